// layout.h -- data shared by the host runtime and the sm_103a kernels of libdgswe.
//
// Element state lives in per-element records (array of structures, 16-byte aligned) so that
// both the element's own load and a neighbour's gather are a few full-sector vector loads.
//
//   mixed precision, degree P (NP = (P+1)(P+2)/2 modes), floats:
//     [0..5]   element means of zeta, qx, qy as float-float pairs (hi, lo)
//     [6..]    modal coefficients 1..NP-1 of zeta, then qx, then qy (orthonormal basis)
//     then     mean depth H (float), flag bits, bathymetry slopes hb1, hb2; zero padding
//   fp64, degree P, doubles: the same fields, means as plain doubles.
//
// The element mean is the mode-0 coefficient divided by sqrt(2) (phi_0 = 1/sqrt 2 on the
// reference triangle of area 2).
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define DG_HD __host__ __device__
#else
#define DG_HD
#endif

namespace dg {

constexpr int MAXSEG = 8;   // tidal segments: ocean edge code -2 - seg
constexpr int MAXRIV = 8;   // river segments: river edge code -2 - MAXSEG - seg
constexpr int MAXSTAGE = 5; // Runge-Kutta stages
constexpr int MAXNP = 6;
constexpr int MAXNQ = 7;
constexpr int MAXNQP = 8;  // MAXNQ rounded up to an even number
constexpr int MAXNG = 3;
constexpr int TILE_ALIGN = 256;  // scenario element ranges start on multiples of this
constexpr int TILE = 32;         // elements per warp tile

enum : uint32_t { FLAG_DRY = 1u };
enum : int { ERR_NONFINITE = 1, ERR_NEGDEPTH = 2, ERR_TIMEOUT = 4 };

DG_HD constexpr int np_of(int p) { return (p + 1) * (p + 2) / 2; }

// record size in 16-byte units
DG_HD constexpr int rec_vec_mixed(int p) { return (3 * np_of(p) + 7 + 3) / 4 <= 4 ? 4 : 8; }
DG_HD constexpr int rec_vec_fp64(int p) { return ((3 * np_of(p) + 4) + 1) / 2 <= 8 ? 8 : 12; }

// edge-split path: per interior edge one record {eL<<2|jL, eR<<2|jR, scaled normal of L's edge};
// per (element, local edge) one slot with the edge's lift on that side: zeta modes 1.., qx and
// qy modes 0.., the mass flux integral (outward), and a closed-edge flag.  Sizes in 16-byte units.
DG_HD constexpr int edge_vec(bool fp64) { return fp64 ? 2 : 1; }
DG_HD constexpr int slot_vals(int p) { return (np_of(p) - 1) + 2 * np_of(p); }
DG_HD constexpr int slot_vec_mixed(int p) { return (slot_vals(p) + 2 + 3) / 4; }
DG_HD constexpr int slot_vec_fp64(int p) { return (slot_vals(p) + 2 + 1) / 2; }

// reference-element tables (basis, quadrature), held in constant memory per degree
template <typename T>
struct RefTab {
  int nq, ng, np;
  T qw[MAXNQ];                     // area weights, sum 2
  T ql[MAXNQ][3];                  // barycentric coordinates of the area points
  T qphi[MAXNQ][MAXNP];            // basis at area points
  T qdr[MAXNQ][MAXNP];             // d(basis)/dr at area points
  T qds[MAXNQ][MAXNP];             // d(basis)/ds at area points
  T gw[MAXNG];                     // Gauss-Legendre weights, sum 2
  T ephi[3][MAXNG][MAXNP];         // basis on local edge j (vertex j -> j+1) at point k
  T el[3][MAXNG][3];               // barycentric coordinates of those points
  T vphi[3][MAXNP];                // basis at the three vertices
  T vinv[2][3];                    // modal coefficients 1,2 of a linear function from vertex values
  T vabs[MAXNP];                   // largest |basis| over the three vertices, per mode
  T mphi[3][MAXNP];                // basis at the midpoints of the three edges (slope limiter)
  T phi0;                          // constant mode value 1/sqrt(2)
  // transposed copies for evaluating the area points two at a time: consecutive points of one
  // mode adjacent, padded with zeros to an even number of points
  T qwT[MAXNQP];                   // qw, padded
  T qphiT[MAXNP][MAXNQP];          // qphi transposed
  T qwphiT[MAXNP][MAXNQP];         // qw[q] * qphi[q][m], same order
  T qdrT[MAXNP][MAXNQP];           // qdr transposed
  T qdsT[MAXNP][MAXNQP];           // qds transposed
};

// per-scenario forcing constants in the arithmetic type of a path
template <typename T>
struct ForcingT {
  T t0, dt;                        // stage time = t0 + (step + c) dt
  T storm[10];                     // x0, y0, speed cos(heading), speed sin(heading), rpeak, rm, re, t0,
                                   // then 1 / rm and log2(e) / re
  T tide[MAXSEG][3];               // amplitude, 2 pi / period, phase
  T grid[6];                       // x0, y0, 1/dx, 1/dy, t0, 1/dt_rec
  T ps[4];                         // pressure set-up x0, y0, sigma, peak
};

// per-scenario parameters (device array; an ensemble holds several)
struct ScenDev {
  double t0, dt;
  float bdt_hi[MAXSTAGE], bdt_lo[MAXSTAGE];  // beta_s * dt of each Shu-Osher stage, float-float
  double bdt[MAXSTAGE];            // same in double
  double bw[MAXSTAGE];             // weight of stage s in the final combination (ledger)
  int32_t elem_begin, elem_end;
  int32_t rain_kind;               // 0 none, 1 constant per element, 2 storm, 3 grid
  int32_t gnx, gny, gnt;
  int32_t nseg;
  int32_t press;
  int32_t rnseg, rnt;              // river segments and records
  double rt0, ridt;                // first record time, 1 / record interval
  const double* river;             // [rnt][rnseg] m^2/s into the domain
  const float* grid;               // [gnt][gny][gnx] mm/h
  ForcingT<float> f;
  ForcingT<double> d;
};

// device control block
struct Ctl {
  unsigned long long step;         // completed steps (all scenarios advance together)
  unsigned int tile_counter;       // persistent-grid work counter
  unsigned int ticket;             // CTAs finished in the current launch
  int err;                         // ERR_* bits
  int pad;
};

}  // namespace dg
