// args.h -- kernel argument blocks of libdgswe (plain structs shared by host and device code).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "layout.h"

namespace dg {

struct Mixed;
struct Fp64;
template <class Pol>
struct PolT;
template <>
struct PolT<Mixed> {
  using T = float;
};
template <>
struct PolT<Fp64> {
  using T = double;
};

// ----------------------------------------------------------------------- kernel arguments ---
template <class Pol>
struct StageArgs {
  using T = typename PolT<Pol>::T;
  const uint4* in;         // stage input records
  const uint4* wn;         // step-initial records (Shu-Osher combination)
  uint4* out;              // output records
  const int4* nbr;         // per element: 3 neighbour codes (+ Manning bits in .w, mixed)
  const uint4* geo;        // static geometry records
  const int4* nodes;       // per element: 3 node indices
  const T* node_xy;        // [2 * nodes] coordinates (rain, pressure set-up)
  const double* hb_nodal;  // [nodes] FP64 bathymetry (depth test near H0)
  const T* rain_e;         // [elements] constant element rain (rain_kind 1)
  T* rain_node;            // [nodes] gridded rain at the stage time (rain_kind 3), node kernel output
  const int32_t* node_scen;  // [nodes] scenario of each node
  const T* lim;            // [elements][8] slope limiter data: a_i, c_i (i = 0..2), M h^2, pair bits (-1: off)
  T lim_nu;                // limiter minmod weight
  const ScenDev* scen;
  const int32_t* tile_scen;  // scenario of each 32-element tile
  const int4* tile_meta;   // tile form: per tile {scenario, elements present (0..32), 0, 0}
  const uint4* xy0;        // tile form: first vertex of each element, [E] float2 (mixed) / double2 (FP64)
  double* ledger;          // [scenario][wslots][2]: rain volume, boundary inflow volume per warp
  Ctl* ctl;
  const uint4* edges;      // edge-split path: interior edge records
  uint4* slots;            // edge-split path: per (element, local edge) lift slots
  long long nedges;
  int split;               // form: 0 fused, 1 edge kernel + slots, 2 tile (each edge of a warp tile once)
  int ntiles;              // 32-element tiles, processed round-robin by the launch's warps
  int wslots;              // ledger slots per scenario (>= warps of the launch)
  int stage;               // Shu-Osher stage index
  int last;                // 1 on the final stage of a step
  int tune;                // 1: timing run, no ledger or step bookkeeping
  int classify_only;       // prepare pass: derive depth and dry flag, keep the state as given
  int friction;            // 0 Manning, 1 quadratic, 2 none
  int has_n;               // the stage combines with the step-initial state
  int pow2;                // a_n and a_in are 0 or powers of two (exact float-float scaling)
  float a_n_hi, a_n_lo, a_in_hi, a_in_lo;  // Shu-Osher coefficients as float-float
  double a_n, a_in;
  double cst;
  T g, H0, cf;
};

}  // namespace dg

namespace dg {

// host-side launchers, explicitly instantiated for Mixed (stage_mixed.cu) and Fp64 (stage_fp64.cu)
template <class Pol>
cudaError_t upload_tables(int p, const RefTab<float>& tf, const RefTab<double>& td);
template <class Pol>
cudaError_t launch_stage(int p, int flux, const StageArgs<Pol>& a, int grid, int block, cudaStream_t s);
template <class Pol>
int stage_blocks_per_sm(int p, int flux, int block, int split);
// Features of a run that a tile-kernel instantiation compiles in.  The generic instantiation has
// all of them; a specialised one leaves out the code, and the run-time tests, of the others and
// serves any run whose features it covers (ft_covers).
enum Feature : int {
  FT_RIVER = 1 << 0,     // river boundary edges
  FT_OCEAN = 1 << 1,     // tidal (open) boundary edges
  FT_PRESS = 1 << 2,     // pressure set-up forcing
  FT_RAIN1 = 1 << 3,     // rain: constant nodal rates
  FT_RAIN2 = 1 << 4,     // rain: parametric storm
  FT_RAIN3 = 1 << 5,     // rain: gridded, nodal rates from the node kernel
  FT_MANNING = 1 << 6,   // Manning friction
  FT_QUAD = 1 << 7,      // quadratic friction
  FT_NOFRIC = 1 << 8,    // no friction
  FT_POW2 = 1 << 9,      // stages whose Shu-Osher weights are powers of two
  FT_GENSSP = 1 << 10,   // stages with other weights
  FT_RAIN0 = 1 << 11,    // no rain
  FT_ALL = (1 << 12) - 1
};
// a run has one or more rain kinds (one per scenario), exactly one friction law, and one or both
// stage-weight kinds; an instantiation with exactly one of a group fixes it at compile time
constexpr int FT_RAIN = FT_RAIN0 | FT_RAIN1 | FT_RAIN2 | FT_RAIN3;
constexpr int FT_FRIC = FT_MANNING | FT_QUAD | FT_NOFRIC;
// what an instantiation fixes at compile time (-1: decided at run time)
DG_HD constexpr int ft_rain(int ft) {
  return (ft & FT_RAIN) == FT_RAIN0 ? 0
         : (ft & FT_RAIN) == FT_RAIN1 ? 1
         : (ft & FT_RAIN) == FT_RAIN2 ? 2
         : (ft & FT_RAIN) == FT_RAIN3 ? 3
                                      : -1;
}
DG_HD constexpr int ft_friction(int ft) {
  return (ft & FT_FRIC) == FT_MANNING ? 0 : (ft & FT_FRIC) == FT_QUAD ? 1 : (ft & FT_FRIC) == FT_NOFRIC ? 2 : -1;
}
DG_HD constexpr int ft_pow2(int ft) {
  return (ft & (FT_POW2 | FT_GENSSP)) == FT_POW2 ? 1 : (ft & (FT_POW2 | FT_GENSSP)) == FT_GENSSP ? 0 : -1;
}
DG_HD constexpr bool ft_covers(int ft, int need) { return (need & ~ft) == 0; }

// tile form (split = 2): reference tables and shared-memory limits of its translation units,
// the launch (the specialised instantiation that covers the run's features, else the generic
// one), and resident CTAs per SM of the instantiation the launch would use
template <class Pol>
cudaError_t upload_tile_tables(int p, const RefTab<float>& tf, const RefTab<double>& td);
template <class Pol>
cudaError_t launch_tile(int p, int flux, int feat, const StageArgs<Pol>& a, int grid, int block, cudaStream_t s);
template <class Pol>
int tile_blocks_per_sm(int p, int flux, int feat, int block);
// specialised mixed-precision tile kernels (tile_spec.cu): launch or occupancy of the one that
// covers feat; cudaErrorNotSupported (launch) or -1 (occupancy) when none does
cudaError_t launch_tile_spec(int p, int flux, int feat, const StageArgs<Mixed>& a, int grid, int block,
                             cudaStream_t s);
int tile_spec_blocks_per_sm(int p, int flux, int feat, int block);
// Feature bits of the specialised instantiation that covers feat, or -1 when none does
int tile_spec_features(int p, int flux, int feat);
// reference tables and shared-memory limits of the specialised instantiations' translation unit
cudaError_t upload_tile_spec_tables(int p, const RefTab<float>& tf, const RefTab<double>& td);
// edge kernel of the split path: one thread per interior edge, writes both sides' slots
template <class Pol>
cudaError_t launch_edges(int p, int flux, const StageArgs<Pol>& a, int grid, int block, cudaStream_t s);
// positive-depth operator on records [begin, end) in place (a.in == a.out)
template <class Pol>
cudaError_t launch_prepare(int p, const StageArgs<Pol>& a, long long begin, long long end, cudaStream_t s);
// optional slope limiter (p = 1) on the stage output, in place, then the positive-depth operator
template <class Pol>
cudaError_t launch_limiter(const StageArgs<Pol>& a, long long ne, cudaStream_t s);
// gridded rain (rain_kind 3) interpolated to every node at the stage time: a.rain_node[0, nn)
template <class Pol>
cudaError_t launch_node_rain(const StageArgs<Pol>& a, long long nn, cudaStream_t s);
// partial FP64 sums of A*mean(zeta) and A*mean(H) over [begin, end): partials[4*block]
template <class Pol>
cudaError_t launch_volume(int p, const uint4* rec, const uint4* geo, long long begin, long long end,
                          double* partials, int nblk, cudaStream_t s);
// per-block minimum of the CFL time step over [begin, end): partials[block]
template <class Pol>
cudaError_t launch_dt(int p, const uint4* rec, const int4* nodes, const double* xy64, const double* hb_nodal,
                      long long begin, long long end, double cfl, double g, double H0, double* partials, int nblk,
                      cudaStream_t s);
// modal state [Np][n] of scenario elements [begin, begin + n) in caller order; inv[c] is the
// position of caller element c relative to begin.  The arrays may be device memory or
// device-accessible page-locked host memory (coalesced in caller order).
template <class Pol>
cudaError_t launch_gather(int p, const uint4* rec, long long begin, long long n, const int32_t* inv, double* z,
                          double* x, double* y, cudaStream_t s);

// modal state [Np][n] (caller order) into the records of [begin, begin + n), same conventions
template <class Pol>
cudaError_t launch_scatter(int p, uint4* rec, long long begin, long long n, const int32_t* inv, const double* z,
                           const double* x, const double* y, cudaStream_t s);

// Neumaier-compensated reduction of per-block partial pairs (shared by all precisions)
cudaError_t launch_reduce_pairs(const double* partials, int nblk, int npairs, double* out, cudaStream_t s);

}  // namespace dg
