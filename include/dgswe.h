/*
 * dgswe.h -- C interface of the GB300 (sm_103a) library that advances the rainfall-augmented
 * 2D shallow water equations with the discontinuous Galerkin method of Wichitrnithed et al.,
 * "A Discontinuous Galerkin Finite Element Model for Compound Flood Simulations"
 * (arXiv 2307.14302).
 *
 * The calls follow the paper's problem statement (Sec. 2.1, Eq. SWE): find (zeta, q = H u) on a
 * triangulated domain whose boundary is split into ocean (specified elevation) and land (zero
 * normal flow) parts, given bathymetry h_b (positive downward), a Manning field, nodal rainfall
 * (Sec. 2.3, Eq. rain) and tidal boundary data.  The state is advanced by the DG right-hand side
 * (Eq. elem_weak_form, Eq. RKSSP) and an SSP Runge-Kutta scheme (Sec. 2.2) with the positive-
 * depth operator of Sec. 2.4 applied after every stage.
 *
 * Conventions shared by every entry point
 *   - Return value: 0 on success, a negative DGSWE_E* code otherwise; dgswe_last_error() then
 *     holds a message for the calling thread.
 *   - All input pointers are borrowed for the duration of the call and copied before return
 *     (host pointers unless the name says _device).  Output pointers are written before return
 *     (host) or enqueued on the context's stream (device).  Nothing is retained.
 *   - Units are SI: metres, seconds, m/s for rain (the grid helper alone takes mm/h).
 *   - Triangles are given counter-clockwise; a clockwise triangle is made counter-clockwise by
 *     swapping its second and third vertices (modal outputs then refer to that order).
 *   - Element order in every output is the caller's input order; internal renumbering for L2
 *     locality is invisible.
 *   - Modal arrays are [Np][E] per variable (mode-major), Np = (p+1)(p+2)/2, in the orthonormal
 *     Dubiner basis on the reference triangle (-1,-1),(1,-1),(-1,1) (Eq. dubiner), local
 *     vertex order as given, modes ordered by total degree then by the second index.
 *   - Calls on one context must not overlap from several host threads.
 *   - Call order: create, set_params, set_mesh, set_fields, forcing setters (any order),
 *     set_state, then step / get_* freely.  Out-of-order calls return DGSWE_ESTATE.
 */
#ifndef DGSWE_H
#define DGSWE_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

enum {
  DGSWE_OK = 0,
  DGSWE_EINVAL = -1,     /* bad argument */
  DGSWE_ENOMEM = -2,     /* device or host allocation failed */
  DGSWE_ECUDA = -3,      /* a CUDA call failed; message in dgswe_last_error() */
  DGSWE_ENONFINITE = -4, /* a stage produced a non-finite value (device error word) */
  DGSWE_ENEGDEPTH = -5,  /* an element mean depth fell below zero (device error word) */
  DGSWE_ETIMEOUT = -6,   /* a bounded device-side wait ran out */
  DGSWE_ESTATE = -7,     /* call out of order */
  DGSWE_ENOLIB = -8      /* the CUDA device or kernel image is unavailable */
};

enum { DGSWE_FLUX_ROE = 0, DGSWE_FLUX_LLF = 1 };             /* Sec. 2.3 numerical fluxes */
enum { DGSWE_FP64 = 0, DGSWE_MIXED = 1 };                    /* arithmetic of the device path */
enum { DGSWE_MANNING = 0, DGSWE_QUADRATIC = 1, DGSWE_NOFRICTION = 2 };
enum { DGSWE_BT_LAND = 0, DGSWE_BT_OCEAN = 1, DGSWE_BT_RIVER = 2 };  /* boundary types, Sec. 2.1 */
enum { DGSWE_LAYOUT_MODAL = 0, DGSWE_LAYOUT_NODAL = 1 };

typedef struct dgswe_ctx* dgswe_h;

/* Run parameters (Sec. 2.2-2.4, Sec. 3).
 *   p           polynomial degree 1 or 2 (Eq. dubiner);
 *   flux        DGSWE_FLUX_ROE or DGSWE_FLUX_LLF;
 *   ssp_stages  2, 3 or 5: SSP(2,2) or SSP(3,3) in Shu-Osher form (Sec. 2.2; order p+1 is the
 *               usual choice), or the five-stage second-order SSP(5,2) (four forward-Euler
 *               substeps of dt/4, then w = w^n/5 + 4/5 (w4 + dt/4 L(w4)); SSP coefficient 4,
 *               so CFL numbers up to four times those of SSP(2,2) keep its stability bound)
 *               for the five-stage runs of Sec. 3;
 *   precision   DGSWE_FP64 (every operation in double) or DGSWE_MIXED (FP32 bulk; float-float
 *               element means; FP64 for the depth test near H0 and the global ledger);
 *   g           gravity [m/s^2];  H0 thin-layer depth threshold [m] (Sec. 2.4);
 *   cfl, dt     dt > 0 is used as given, otherwise dt = cfl * min_e(2 r_in) / ((2p+1) lambda_e)
 *               with lambda_e = max over vertices of |u| + sqrt(g max(H, H0)) of the state
 *               passed to dgswe_set_state (fixed for the run);
 *   friction    DGSWE_MANNING (tau = g n^2 |u| / H^{4/3}), DGSWE_QUADRATIC (tau = cf |u| / H,
 *               Sec. 3.1) or none;  cf quadratic coefficient;
 *   limiter     1: the optional slope limiter (Sec. 2.3 offers one for shocks without giving its
 *               form) as the TVB minmod moment limiter of Cockburn and Shu for P1 triangles,
 *               applied componentwise after each stage's positive-depth operator and followed
 *               by the operator again; wet elements with three neighbours only; p = 1 only
 *               (DGSWE_EINVAL otherwise);  lim_nu its minmod weight (1.5 is usual, >= 1 keeps
 *               linear data), lim_M its TVB constant (0: TVD). */
typedef struct {
  int32_t p;
  int32_t flux;
  int32_t ssp_stages;
  int32_t precision;
  double g;
  double H0;
  double cfl;
  double dt;
  int32_t friction;
  double cf;
  int32_t limiter;
  double lim_nu;
  double lim_M;
} dgswe_params;

/* Moving radially symmetric rain cell (stand-in for the parametric model of Sec. 2.5):
 * centre (x0, y0) + speed * (t - t0) * (cos heading, sin heading); rate at distance r:
 * rpeak (1/2 + r / (2 rm)) for r < rm, rpeak exp(-(r - rm) / re) beyond.  m, s, rad, m/s. */
typedef struct {
  double x0, y0, heading, speed, rpeak, rm, re, t0;
} dgswe_storm;

/* Gaussian surface set-up eta_p = peak exp(-|x - x0|^2 / (2 sigma^2)) entering the momentum
 * source as F = g H grad(eta_p) (the F_x, F_y of Eq. SWE). */
typedef struct {
  double x0, y0, sigma, peak;
} dgswe_gauss_setup;

/* Mass ledger (Eq. SWE integrated over the domain):  V = sum_e A_e mean(zeta_e);
 * rain_in = sum over stages of b_s dt sum_e A_e R_e;  bdry_in = inflow through ocean edges;
 * rel_err = |V - V0 - rain_in - bdry_in| / VH0 with VH0 the initial water volume. */
typedef struct {
  double t;
  int64_t steps;
  double V0, V, rain_in, bdry_in, VH0, rel_err, wet_frac;
} dgswe_ledger;

/* No counterpart in the paper (lifetime).  Creates a context on CUDA device `device`;
 * `cuda_stream` is a cudaStream_t on which all device
 * work of this context is enqueued (NULL: the library creates a private non-blocking stream).
 * *out receives the handle.  Errors: EINVAL (null out), ENOLIB (no device, or a device other
 * than sm_103a), ECUDA. */
int dgswe_create(dgswe_h* out, int device, void* cuda_stream);

/* Sets the run parameters of the method (Sec. 2.2-2.4, fields listed above; copied).  EINVAL on
 * values outside the ranges above. */
int dgswe_set_params(dgswe_h, const dgswe_params* params);

/* Sets the triangulation (Sec. 2.1, ADCIRC-style arrays).
 *   xy [n_nodes][2] float64 coordinates;  tri [n_tri][3] int32 node indices;
 *   bedge [n_bedge][2] node pairs of boundary edges with btype (DGSWE_BT_*) and bseg (tidal
 *   segment of ocean edges, 0 <= bseg < n_tide_segments); boundary edges not listed are land.
 * Builds edge connectivity, renumbers elements and nodes along a space-filling curve and
 * computes geometry.  EINVAL on out-of-range indices, degenerate triangles, an edge shared by
 * more than two triangles, or an unknown boundary type. */
int dgswe_set_mesh(dgswe_h, int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri, int32_t n_bedge,
                   const int32_t* bedge, const int32_t* btype, const int32_t* bseg);

/* Sets nodal bathymetry hb [n_nodes] (the h_b of Eq. SWE: positive downward, m; continuous
 * piecewise linear) and Manning n (the bottom friction tau_b of Eq. SWE), per element [n_tri]
 * (manning_nodal = 0) or per node [n_nodes] (element value = mean of its nodes).  manning may be
 * NULL when friction is not Manning. */
int dgswe_set_fields(dgswe_h, const double* hb_nodal, const double* manning, int32_t manning_nodal);

/* Rain sources (Sec. 2.3, Eq. rain): the element rate is the mean of its three nodal rates and
 * is added to every element, wet or dry.  Each setter replaces the previous rain source. */
int dgswe_set_rain_nodal(dgswe_h, const double* r_nodal); /* constant in time [n_nodes] m/s */
/* The moving rain cell of dgswe_storm (the parametric rainfall of Sec. 2.5), copied. */
int dgswe_set_rain_parametric(dgswe_h, const dgswe_storm* storm);
/* Gridded records [nt][ny][nx] float32 in mm/h on x0 + i dx, y0 + j dy, times t0 + k dt_rec:
 * bilinear in space, linear in time, clamped at the grid and record ends (Sec. 2.5). */
int dgswe_set_rain_grid(dgswe_h, int32_t nx, int32_t ny, int32_t nt, double x0, double y0, double dx, double dy,
                        double t0, double dt_rec, const float* mm_per_h);

/* Tidal elevation on ocean edges of segment s (the specified-elevation boundary of Sec. 2.1):
 * amp[s] sin(2 pi t / period[s] + phase[s]); the ghost state takes it with the interior
 * discharge.  Copied; n_seg in [1, 8]. */
int dgswe_set_tide(dgswe_h, int32_t n_seg, const double* amp, const double* period, const double* phase);

/* River (specified normal flow) boundaries, Sec. 2.1 Eq. river_bc: edges of type
 * DGSWE_BT_RIVER with bseg = river segment in [0, 8).  q is [n_t][n_seg]: discharge per unit
 * width in m^2/s, positive INTO the domain, n_t records from t0 every dt_rec seconds, linear in
 * time and held constant before the first and after the last record (n_t = 1: constant).
 * The mass component of the numerical flux on a river edge is exactly -q (outward), the
 * momentum components are those of the numerical flux between the interior trace and the ghost
 * state (zeta, -q n); the inflow counts as boundary inflow in the ledger.  Copied; a later call
 * replaces the series.  Returns DGSWE_EINVAL for n_seg outside [1, 8], n_t < 1, dt_rec <= 0
 * with n_t > 1, or non-finite values. */
int dgswe_set_river(dgswe_h, int32_t n_seg, int32_t n_t, double t0, double dt_rec, const double* q);

/* Gaussian pressure set-up forcing (F_x, F_y of Eq. SWE); NULL removes it. */
int dgswe_set_pressure_setup(dgswe_h, const dgswe_gauss_setup* setup);

/* Sets the state (zeta, q) of Eq. SWE at t = t0 (the initial condition of the problem of
 * Sec. 2.1).  layout MODAL: zeta, qx, qy are [Np][n_tri] modal coefficients;
 * NODAL: [n_nodes] nodal values, interpolated linearly on each element.  The positive-depth
 * operator is applied once (it defines the wet/dry flags), the ledger is reset (V0, VH0) and,
 * when params.dt <= 0, dt is fixed from the CFL condition. */
int dgswe_set_state(dgswe_h, const double* zeta, const double* qx, const double* qy, int32_t layout, double t0);

/* Replaces the state at the current time with modal host arrays [Np][n_tri] (the layout of
 * dgswe_get_state): copied to the device and packed into the element records there, bit for
 * bit.  The state is kept as given (a state read back from the solver satisfies the positive-
 * depth constraints of Sec. 2.4 already); only the mean depths and wet/dry flags are derived
 * from it.  Mesh, fields, forcing, dt, time and ledger are kept (the ledger then also holds the
 * injected change).  For restarts and for couplings that exchange the state every step.
 * Page-locked (pinned) host arrays are read by the packing kernel itself, over the host link, in
 * stream order: the call returns at once, and the arrays must not change until the next call
 * that synchronises (dgswe_sync, dgswe_get_state, dgswe_get_ledger, ...).  Other host memory is
 * staged through a device buffer and the call returns after the stream has consumed it. */
int dgswe_load_state(dgswe_h, const double* zeta, const double* qx, const double* qy);

/* The exchange of a coupling loop in one call: the current state goes out to (zeta_out, qx_out,
 * qy_out) exactly as dgswe_get_state writes it, then (zeta_in, qx_in, qy_in) becomes the state
 * exactly as dgswe_load_state takes it; all six arrays modal [Np][n_tri] in caller order, in and
 * out not overlapping.  Equivalent to dgswe_get_state followed by dgswe_load_state, bit for bit
 * (the problem statement's state in, state out, Sec. 2.1).  When all six are page-locked (pinned)
 * host arrays one kernel reads each element record once, writes its old coefficients out and
 * its new ones in, so both directions of the host link are in use at the same time; otherwise the
 * two calls run in turn through their staged paths.  Returns after the stream has finished the
 * exchange (the outputs are complete and the inputs may change). */
int dgswe_exchange_state(dgswe_h, const double* zeta_in, const double* qx_in, const double* qy_in, double* zeta_out,
                         double* qx_out, double* qy_out);

/* Enqueues n_steps steps of the SSP Runge-Kutta scheme (Eq. RKSSP; each stage the DG right-hand
 * side of Eq. elem_weak_form and the positive-depth operator of Sec. 2.4) on the context's stream
 * (CUDA graph replay) and returns without waiting.  Device errors surface in dgswe_sync. */
int dgswe_step(dgswe_h, int64_t n_steps);

/* No counterpart in the paper (stream plumbing): waits for the stream and returns the first
 * device error word (ENONFINITE, ENEGDEPTH, ETIMEOUT) or 0. */
int dgswe_sync(dgswe_h);

/* The fixed time step [s] in *dt (the runs of Sec. 3 use a fixed dt; here from the CFL
 * condition of dgswe_params unless given). */
int dgswe_get_dt(dgswe_h, double* dt);

/* Copies the modal state (zeta, q) of Eq. SWE, in the basis of Eq. dubiner, to host arrays
 * [Np][n_tri] (synchronises the stream).  Page-locked
 * (pinned) arrays are written by the unpacking kernel itself over the host link; other host
 * memory is staged through a device buffer. */
int dgswe_get_state(dgswe_h, double* zeta, double* qx, double* qy);

/* Copies the modal state (as dgswe_get_state: (zeta, q) of Eq. SWE, basis of Eq. dubiner) into
 * caller-owned device memory: each pointer to
 * Np*n_tri doubles, written on the context's stream (no host round trip). */
int dgswe_get_state_device(dgswe_h, double* zeta_dev, double* qx_dev, double* qy_dev);

/* No counterpart in the paper (memory plumbing).  Device memory that the element records need
 * (the state w^n and the two Runge-Kutta stage
 * buffers, each rounded up to 256 bytes), in *bytes.  Valid after dgswe_set_state or
 * dgswe_ensemble_create. */
int dgswe_record_bytes(dgswe_h, uint64_t* bytes);

/* No counterpart in the paper (memory plumbing).  Places the element records in caller-owned
 * device memory (for example a framework's tensor
 * storage), so that the caller's allocator provides the solver's largest arrays: dev must be
 * device memory of the context's device, 256-byte aligned, at least dgswe_record_bytes long.  The
 * current state is copied there and every later step reads and writes it in place; the library
 * never frees it.  The caller keeps it alive and unmodified until it binds other memory, unbinds
 * (dev = NULL: the library allocates its own records again and copies the state back) or destroys
 * the context.  A later dgswe_set_state keeps the binding when the memory is still large enough and
 * drops it otherwise.  Returns DGSWE_EINVAL for memory that is too small, unaligned or not device
 * memory of the context's device; synchronises the stream. */
int dgswe_bind_device(dgswe_h, void* dev, uint64_t bytes);

/* Per-element dry flags (Sec. 2.4) [n_tri] as 0/1 bytes. */
int dgswe_get_dry(dgswe_h, uint8_t* dry);

/* Mass ledger of dgswe_ledger: Eq. SWE's mass equation integrated over the domain and the
 * steps, water volume against rain and boundary inflow (synchronises the stream). */
int dgswe_get_ledger(dgswe_h, dgswe_ledger* out);

/* Total water volume sum_e A_e mean(zeta_e) of the current state (the V of the mass balance of
 * Eq. SWE, above the datum), reduced on the device in
 * FP64 with Neumaier compensation over per-block partial sums held in library-allocated scratch
 * memory; *out receives the value (synchronises the stream). */
int dgswe_volume(dgswe_h, double* out);

/* No counterpart in the paper: the total water volume of dgswe_volume, for callers that cannot
 * allocate device memory -- callers whose device memory all comes from their own pool or caching
 * allocator, and loops that must not stall on the device-wide synchronisation that cudaFree
 * implies.  This entry point allocates nothing.
 *   w0_dev    [n] device array: mode-0 coefficients of zeta (row 0 of dgswe_get_state_device);
 *   area_dev  [n] device array: element areas [m^2];
 *   out_dev   device pointer to one double, receives sum_e area_e * w0_e / sqrt(2);
 *   cuda_stream  stream for the two kernels (NULL: the legacy default stream); asynchronous.
 * Partial sums live in a fixed 64 KiB __device__ array that every GPU loading the library
 * keeps until exit; n may be 0 .. 16,777,216, larger n returns DGSWE_EINVAL.  All calls share
 * that array (each call writes every slot it reads), so calls whose kernels overlap on the GPU
 * race: order them on one stream.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current) and keeps it for the life of the
 * process; after cudaDeviceReset on that device the kept address is stale, and this entry point
 * must not be called there again.  Pointers must belong to the current device. */
int dgswe_volume_sum_noalloc(const double* w0_dev, const double* area_dev, int64_t n, double* out_dev,
                             void* cuda_stream);

/* No counterpart in the paper (the paper runs one scenario at a time): an ensemble of
 * independent scenarios (different meshes, forcing, Manning fields), each the problem of
 * Sec. 2.1 advanced by the method of dgswe_step, advanced together: one persistent launch per RK
 * stage over all scenarios' tiles, the whole step captured in a CUDA graph.  The members must
 * share p, flux, ssp_stages, precision, g and H0 and have their state set; their data is copied
 * (members keep ownership and are not modified).  Each scenario keeps its own dt and time. */
int dgswe_ensemble_create(dgswe_h* out, int32_t n, const dgswe_h* members, int device, void* cuda_stream);
/* n_steps SSP Runge-Kutta steps (Eq. RKSSP) of every scenario, enqueued (as dgswe_step). */
int dgswe_ensemble_step(dgswe_h ens, int64_t n_steps);
/* Scenario `member` (0-based, creation order): its modal state (as dgswe_get_state: (zeta, q) of
 * Eq. SWE); synchronises the stream.  EINVAL for a bad index. */
int dgswe_ensemble_get_state(dgswe_h ens, int32_t member, double* zeta, double* qx, double* qy);
/* Scenario `member`'s own mass ledger (as dgswe_get_ledger: the mass balance of Eq. SWE);
 * synchronises the stream.  EINVAL for a bad index. */
int dgswe_ensemble_get_ledger(dgswe_h ens, int32_t member, dgswe_ledger* out);

/* No counterpart in the paper (device scheduling).  Launch shape of a stage: block size of the
 * element kernel (64, 128, 256, or 0 = autotune on
 * the next step), waves (1 or 2: the grid holds waves x CTAs resident per SM x SMs CTAs whose
 * warps take the 32-element tiles round-robin), and the form, argument split: 0 one fused kernel
 * in which both neighbours evaluate an interior edge; 1 a separate edge kernel computes every
 * interior edge flux once and the element kernel gathers it; 2 the tile form, one kernel in which
 * each warp evaluates every edge touching its 32-element tile once from records staged in shared
 * memory.  The three forms agree to rounding; for a fixed form results do not depend on block or
 * waves.  Returns DGSWE_EINVAL for other values. */
int dgswe_set_launch(dgswe_h, int32_t block, int32_t waves, int32_t split);
/* No counterpart in the paper (device scheduling): the launch shape in use (after autotuning,
 * the one it chose); NULL pointers are skipped. */
int dgswe_get_launch(dgswe_h, int32_t* block, int32_t* waves, int32_t* split);

/* No counterpart in the paper (diagnostics and tests).  Feature sets: *run, the features of this
 * run as a bit set (1 river
 * boundary edges, 2 tidal boundary edges, 4 pressure set-up, 8 nodal rain, 16 storm rain,
 * 32 gridded rain, 64 Manning friction, 128 quadratic friction, 256 no friction, 512 stages whose
 * Shu-Osher weights are powers of two, 1024 other stage weights, 2048 a scenario without rain).
 * *kernel: the features compiled into the tile-form kernel that a stage launches: the narrowest
 * specialised instantiation that covers the run, else the generic one (4095, every feature).
 * Either pointer may be NULL.  DGSWE_ESTATE before the state is set. */
int dgswe_get_tile_features(dgswe_h, int32_t* run, int32_t* kernel);

/* No counterpart in the paper (device scheduling).  How dgswe_step enqueues its work: 1
 * (default) replays whole steps from CUDA graphs captured
 * once (1-step and 8-step graphs); 0 launches every kernel of every stage directly on the
 * stream.  Results are bit-identical; the direct form exists to measure what the graphs save
 * on small, launch-bound meshes.  Returns DGSWE_EINVAL for other values. */
int dgswe_set_graphs(dgswe_h, int32_t on);

/* No counterpart in the paper (diagnostics): number of kernel launches this context enqueued so
 * far (all kinds). */
int64_t dgswe_launch_count(dgswe_h);

/* No counterpart in the paper (lifetime): releases the context and its device memory (NULL is
 * ignored). */
void dgswe_destroy(dgswe_h);

/* No counterpart in the paper (error reporting): message of the last error on the calling
 * thread ("" if none). */
const char* dgswe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
