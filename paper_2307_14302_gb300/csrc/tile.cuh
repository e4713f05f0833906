// tile.cuh -- tile form of the DG stage kernel for sm_103a.
//
// One warp owns a tile of 32 consecutive (Hilbert-ordered) triangles and advances it by one
// Runge-Kutta stage (Sec. 2.2, Eq. RKSSP) in three phases:
//   1. element phase A: each lane loads its triangle's record and static data, and integrates the
//      area terms of Eq. elem_weak_form (flux divergence, balance term g zeta grad(hb), friction,
//      pressure set-up) and the element rain of Eq. rain;
//   2. edge phase: every edge touching the tile is evaluated ONCE (Sec. 2.3: Roe or LLF flux at
//      p+1 Gauss points, land/ocean/river ghost states, the wet/dry closure of Sec. 2.4), about 60
//      edges per tile, one per lane and round.  Both sides' records come from shared memory: the
//      tile's own records, and the records of the ~23 out-of-tile neighbours staged there with
//      cp.async while phase 1 runs.  The flux values at the Gauss points, scaled by the Gauss
//      weight and half the edge length, go into per-(element, local edge) slots in shared memory,
//      each side in its own point order, with the pressure relative to that side's own mean;
//   3. element phase B: each lane lifts its three edge slots into the modal right-hand side,
//      applies the diagonal inverse mass matrix (Eq. dubiner), the Shu-Osher combination, the
//      positive-depth operator M Pi_h (Sec. 2.4), stores its record and books its rain volume.
// Interior edges are oriented canonically (the lower element index is "left"), so an edge on the
// border of two tiles gives the same bits in both, and the two sides of every edge receive
// exactly opposite mass fluxes: mass is conserved to rounding of the element means.
//
// Memory pipeline (per warp): the tile's records, static geometry, neighbour codes, first vertices
// and metadata arrive in shared memory by TMA bulk copies
// (cp.async.bulk, one per array, completing on an mbarrier), double-buffered: the next tile's
// copies are in flight while this tile is computed.  The tile's step-initial records are
// prefetched into L2 by a bulk prefetch at the start of the tile and read in phase 3; the
// out-of-tile neighbour records are gathered with 16-byte cp.async.  Every mbarrier wait is
// bounded: a wait that runs out sets ERR_TIMEOUT in the device error word and the kernel returns.
//
// Records are vector-major in shared memory ([RV][32], as in the tile-blocked device array), so
// the 16-byte reads of a warp, at its own slots or at any mix of neighbour slots, spread over
// the banks.  Shared memory per warp: the two buffers, the halo records [RV][32], the edge
// descriptors [96] {left side, right side, left normal} and the edge slots [3][pairs][32], which
// overlay the consumed static part of the current buffer (about 12 KB in the mixed p = 1 path).
// Neighbours beyond 32 halo slots (none on Hilbert-ordered meshes; kept for generality) are read
// from global memory.
//
// The kernel takes a set of Feature bits (args.h): the generic instantiation has all of them;
// the specialised ones (tile_spec.cu) leave out the code of the features a run does not have.
#pragma once
#include "stage.cuh"

namespace dg {

constexpr int HALO = 32;    // staged out-of-tile neighbour records per tile
static_assert(HALO == TILE, "own and halo records share one vector stride in shared memory");
constexpr int TE_MAX = 96;  // edges touching a 32-element tile (3 per element at most)

// edge descriptor: left side, right side (or boundary code), and the left side's scaled outward
// normal (written by the lane that owns the edge, from its own geometry)
template <class T>
struct EdgeDesc;
template <>
struct alignas(16) EdgeDesc<float> {
  int sL, sR;
  float lnx, lny;
};
template <>
struct alignas(16) EdgeDesc<double> {
  int sL, sR, pad0, pad1;
  double lnx, lny;
};
__device__ __forceinline__ void put_desc(EdgeDesc<float>* d, int i, int sL, int sR, float lnx, float lny) {
  reinterpret_cast<int4*>(d)[i] = make_int4(sL, sR, __float_as_int(lnx), __float_as_int(lny));
}
__device__ __forceinline__ void put_desc(EdgeDesc<double>* d, int i, int sL, int sR, double lnx, double lny) {
  int4* p = reinterpret_cast<int4*>(d) + 2 * i;
  p[0] = make_int4(sL, sR, 0, 0);
  reinterpret_cast<double2*>(p)[1] = make_double2(lnx, lny);
}
__device__ __forceinline__ void get_desc(const EdgeDesc<float>* d, int i, int& sL, int& sR, float& lnx, float& lny) {
  const int4 v = reinterpret_cast<const int4*>(d)[i];
  sL = v.x;
  sR = v.y;
  lnx = __int_as_float(v.z);
  lny = __int_as_float(v.w);
}
__device__ __forceinline__ void get_desc(const EdgeDesc<double>* d, int i, int& sL, int& sR, double& lnx,
                                         double& lny) {
  const int4* p = reinterpret_cast<const int4*>(d) + 2 * i;
  const int4 v = p[0];
  const double2 n = reinterpret_cast<const double2*>(p)[1];
  sL = v.x;
  sR = v.y;
  lnx = n.x;
  lny = n.y;
}

template <int P, class Pol>
struct TileLayout {
  using T = typename Pol::T;
  static constexpr int NG = P + 1;
  static constexpr int RV = Pol::template RV<P>;
  static constexpr int GV = Pol::GV;
  // edge slot of one element side: Gz[NG], Gx[NG], Gy[NG] -- and the mass integral when NG is odd;
  // with an even NG the mass is the sum of the Gz, which is exactly antisymmetric across the edge
  // (the right side holds the negated values in reverse order) -- stored as pairs of T
  static constexpr bool MASSV = (NG % 2) == 1;
  static constexpr int NV = 3 * NG + (MASSV ? 1 : 0);
  static constexpr int NPR = (NV + 1) / 2;
  static constexpr int XV = sizeof(T) == 4 ? 16 : 32;          // first vertices of a tile, 16-byte units
  // one buffer: records [RV][32] (the tile's block of the tile-blocked record array), geometry
  // [32][GV], neighbour codes [32], first vertices, the tile's metadata {scenario, elements
  // present}, all filled by the TMA batch
  static constexpr int O_GEO = TILE * RV;
  static constexpr int O_NBR = O_GEO + TILE * GV;
  static constexpr int O_XY = O_NBR + TILE;
  static constexpr int O_META = O_XY + XV;
  static constexpr int COPIED = O_META + 1;
  // the edge slots [3][NPR][32] (pairs of T) overlay the geometry, codes, vertices and metadata,
  // which every lane has read into registers (or into the edge descriptors) before the edge phase
  static constexpr int O_FLX = O_GEO;
  static constexpr int FLXV = 3 * NPR * 32 * 2 * (int)sizeof(T) / 16;
  static constexpr int BUF = (O_FLX + FLXV > COPIED) ? O_FLX + FLXV : COPIED;
  static constexpr int BUF0 = 0;
  static constexpr int BUF1 = BUF;
  static constexpr int HAL = 2 * BUF;                          // [RV][HALO]
  static constexpr int DESC = HAL + HALO * RV;                 // [96] EdgeDesc<T>
  static constexpr int DV = (int)sizeof(EdgeDesc<T>) / 16;
  static constexpr int BAR = DESC + TE_MAX * DV;               // two 8-byte mbarriers
  static constexpr int VEC = BAR + 1;                          // 16-byte units per warp
  static constexpr unsigned TILE_BYTES = 16u * COPIED;         // bytes of one buffer's copies
};
template <int P, class Pol>
__host__ __device__ constexpr int tile_smem_bytes(int block) {
  return 16 * TileLayout<P, Pol>::VEC * (block / 32);
}

// ------------------------------------------------------------------ TMA bulk copies -----
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16) signalling bar
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
// 16-byte load from a shared-memory address
__device__ __forceinline__ uint4 lds128(uint32_t addr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr));
  return v;
}
// bulk prefetch of global memory into L2 (16-byte aligned, size a multiple of 16)
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// order this thread's earlier generic-proxy accesses to shared memory before later bulk copies
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// wait for the completion of phase `parity` of bar; false if it did not complete in 2^20 tries
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok = 0;
  for (int i = 0; i < (1 << 20) && !ok; ++i)
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
  return ok != 0;
}

// a bulk copy that did not complete: record it in the device error word, give the copy one more
// bounded wait so that it does not land in shared memory after the warp has left, and return
template <class Pol>
__device__ __noinline__ void tile_timeout(const StageArgs<Pol>& a, uint32_t bar, uint32_t parity, int lane) {
  if (lane == 0) atomicOr(&a.ctl->err, ERR_TIMEOUT);
  (void)mbar_wait(bar, parity);
}

// static geometry record from shared memory (layout of load_geo)
__device__ __forceinline__ void geo_from(const uint4* g, const int4& nb, Geo<Mixed>& G) {
  const uint4 a = g[0], b = g[1], c = g[2];
  G.lnx[0] = __uint_as_float(a.x); G.lny[0] = __uint_as_float(a.y);
  G.lnx[1] = __uint_as_float(a.z); G.lny[1] = __uint_as_float(a.w);
  G.lnx[2] = __uint_as_float(b.x); G.lny[2] = __uint_as_float(b.y);
  G.hbm = {__uint_as_float(b.z), __uint_as_float(b.w)};
  G.A = {__uint_as_float(c.x), __uint_as_float(c.y)};
  G.invA = {__uint_as_float(c.z), __uint_as_float(c.w)};
  G.man = __int_as_float(nb.w);
}
__device__ __forceinline__ void geo_from(const uint4* g, const int4&, Geo<Fp64>& G) {
  uint4 v[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) v[i] = g[i];
  G.lnx[0] = u2d(v[0].x, v[0].y); G.lny[0] = u2d(v[0].z, v[0].w);
  G.lnx[1] = u2d(v[1].x, v[1].y); G.lny[1] = u2d(v[1].z, v[1].w);
  G.lnx[2] = u2d(v[2].x, v[2].y); G.lny[2] = u2d(v[2].z, v[2].w);
  G.hbm = u2d(v[3].x, v[3].y);
  G.A = u2d(v[3].z, v[3].w);
  G.invA = u2d(v[4].x, v[4].y);
  G.man = u2d(v[4].z, v[4].w);
}

// ------------------------------------------------------------ scalar / packed arithmetic ---
// The area points are evaluated two at a time in packed FP32x2 (mixed path, p = 1) or one at a
// time; these overloads let one routine serve both.
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) { return fma2(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ f2 vmul(f2 a, f2 b) { return mul2(a, b); }
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ double vadd(double a, double b) { return a + b; }
__device__ __forceinline__ f2 vadd(f2 a, f2 b) { return add2(a, b); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ double vneg(double a) { return -a; }
__device__ __forceinline__ f2 vneg(f2 a) { return neg2(a); }
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double vmax(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ f2 vmax(f2 a, f2 b) { return max2(a, b); }
__device__ __forceinline__ float vrcp(float a) { return frcp(a); }
__device__ __forceinline__ double vrcp(double a) { return frcp(a); }
__device__ __forceinline__ f2 vrcp(f2 a) { return rcp2(a); }
__device__ __forceinline__ float vsqrt0(float a) { return fsqrt0(a); }
__device__ __forceinline__ double vsqrt0(double a) { return fsqrt0(a); }
__device__ __forceinline__ f2 vsqrt0(f2 a) { return make_float2(fsqrt0(a.x), fsqrt0(a.y)); }
__device__ __forceinline__ float vpowm43(float a) { return fpowm43(a); }
__device__ __forceinline__ double vpowm43(double a) { return fpowm43(a); }
__device__ __forceinline__ f2 vpowm43(f2 a) { return make_float2(fpowm43(a.x), fpowm43(a.y)); }
// friction coefficient tau (source -tau q): Manning g n^2 |u| / Hs^(4/3) (friction 0) or
// cf |u| / Hs (friction 1).  In FP32 as cfm 2^(lg2|q|^2 / 2 - c lg2 Hs) with c = 7/3 or 2, three
// special-function operations and no square root (|q| = 0 gives 2^-inf = 0).
__device__ __forceinline__ float vtau(float qx, float qy, float, float, float Hs, float, float cfm, int friction) {
  const float c = friction == 0 ? 2.3333333f : 2.0f;
  return cfm * mufu_ex2(fmaf(0.5f, mufu_lg2(fmaf(qx, qx, qy * qy)), -c * mufu_lg2(Hs)));
}
__device__ __forceinline__ f2 vtau(f2 qx, f2 qy, f2 u, f2 v, f2 Hs, f2 iH, f2 cfm, int friction) {
  return make_float2(vtau(qx.x, qy.x, u.x, v.x, Hs.x, iH.x, cfm.x, friction),
                     vtau(qx.y, qy.y, u.y, v.y, Hs.y, iH.y, cfm.y, friction));
}
__device__ __forceinline__ double vtau(double, double, double u, double v, double Hs, double iH, double cfm,
                                       int friction) {
  return cfm * (fsqrt0(fma(u, u, v * v)) * (friction == 0 ? fpowm43(Hs) : iH));
}
template <class V>
__device__ __forceinline__ V vbc(float x);
template <>
__device__ __forceinline__ float vbc<float>(float x) { return x; }
template <>
__device__ __forceinline__ double vbc<double>(float x) { return (double)x; }
template <>
__device__ __forceinline__ f2 vbc<f2>(float x) { return make_float2(x, x); }

// a pair of constant-table entries (points q, q+1 of one mode) or one entry
template <class V, class T>
__device__ __forceinline__ V vtab(const T* row, int q);
template <>
__device__ __forceinline__ float vtab<float, float>(const float* row, int q) { return row[q]; }
template <>
__device__ __forceinline__ double vtab<double, double>(const double* row, int q) { return row[q]; }
template <>
__device__ __forceinline__ f2 vtab<f2, float>(const float* row, int q) { return make_float2(row[q], row[q + 1]); }

// ------------------------------------------------------------------------ area (p = 1) ---
// Degree-1 elements have constant basis gradients: the flux terms need only the weighted sums of
// F over the points (SF), the sources their moments against each basis function (SS).
template <class V>
struct AreaP1 {
  V SF[6];     // sum_q w_q (Fx_z, Fx_x, Fx_y, Fy_z, Fy_x, Fy_y)
  V SS[3][2];  // sum_q w_q phi_m (s_x, s_y)
};

template <class V, class T>
__device__ __forceinline__ void area_points_p1(AreaP1<V>& A, const RefTab<T>& tab, int q, V zs0, V zs1, V xs0,
                                               V xs1, V ys0, V ys1, V xb, V yb, V Hb, V hb1, V hb2, V H0v, V hg,
                                               V ghbx, V ghby, V cfm, int friction, V Fxs, V Fys) {
  const V ph1 = vtab<V, T>(tab.qphiT[1], q), ph2 = vtab<V, T>(tab.qphiT[2], q);
  // trace at the point(s): d = zeta - mean(zeta), H, qx, qy (same operation order as trace_at)
  const V d = vfma(zs1, ph2, vmul(zs0, ph1));
  const V qx = vfma(xs1, ph2, vfma(xs0, ph1, xb));
  const V qy = vfma(ys1, ph2, vfma(ys0, ph1, yb));
  const V hdev = vfma(hb1, ph1, vmul(hb2, ph2));
  const V H = vadd(Hb, vadd(d, hdev));
  const V Hs = vmax(H, H0v);
  const V iH = vrcp(Hs);
  const V u = vmul(qx, iH), v = vmul(qy, iH);
  const V pp = vmul(vmul(hg, d), vfma(vbc<V>(2.f), H, vneg(d)));  // g/2 d (2H - d)
  V tau = vbc<V>(0.f);
  if (friction <= 1) tau = vtau(qx, qy, u, v, Hs, iH, cfm, friction);
  const V sx = vfma(ghbx, d, vfma(vneg(tau), qx, Fxs));
  const V sy = vfma(ghby, d, vfma(vneg(tau), qy, Fys));
  const V w = vtab<V, T>(tab.qwT, q);
  A.SF[0] = vfma(w, qx, A.SF[0]);
  A.SF[1] = vfma(w, vfma(qx, u, pp), A.SF[1]);
  A.SF[2] = vfma(w, vmul(qy, u), A.SF[2]);
  A.SF[3] = vfma(w, qy, A.SF[3]);
  A.SF[4] = vfma(w, vmul(qx, v), A.SF[4]);
  A.SF[5] = vfma(w, vfma(qy, v, pp), A.SF[5]);
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    const V wp = vtab<V, T>(tab.qwphiT[m], q);
    A.SS[m][0] = vfma(wp, sx, A.SS[m][0]);
    A.SS[m][1] = vfma(wp, sy, A.SS[m][1]);
  }
}

// Gaussian pressure set-up F = g H grad(eta_p) at a point (x, y) with depth H (graded workload)
template <class T>
__device__ __forceinline__ void setup_force(const ForcingT<T>& F, T px, T py, T H, T g, T& Fx, T& Fy) {
  const T dx = px - F.ps[0], dy = py - F.ps[1], is2 = frcp(F.ps[2] * F.ps[2]);
  const T eta = F.ps[3] * fexp(-(dx * dx + dy * dy) * T(0.5) * is2);
  Fx = g * H * (-eta * dx * is2);
  Fy = g * H * (-eta * dy * is2);
}

// area integrals (grad v, F) + (s, v) of one element into Rz, Rx, Ry (weak-form moments)
template <int P, class Pol, int FT>
__device__ __forceinline__ void tile_area(const Elem<P, Pol>& E, const Geo<Pol>& G, const ScenDev& S,
                                          const StageArgs<Pol>& a, int press, const typename Pol::T vx[3],
                                          const typename Pol::T vy[3], typename Pol::T (&Rz)[np_of(P)],
                                          typename Pol::T (&Rx)[np_of(P)], typename Pol::T (&Ry)[np_of(P)]) {
  using T = typename Pol::T;
  constexpr int NP = np_of(P);
  constexpr int NQ = 7;
  const RefTab<T>& tab = ctab<T, P>();
  const ForcingT<T>& F = forcing<T>(S);
  const T g = a.g, H0 = a.H0;
  const T detJ = T(0.5) * acc_r(G.A);
  const T idetJ = T(2) * acc_r(G.invA);
  // inverse Jacobian from the edge vectors: t0 = x1 - x0 = 2 (xr, yr), t2 = x0 - x2 = -2 (xs, ys)
  // and ln_j = (t_j.y, -t_j.x)
  const T xr = T(-0.5) * G.lny[0], yr = T(0.5) * G.lnx[0];
  const T xs = T(0.5) * G.lny[2], ys = T(-0.5) * G.lnx[2];
  const T rx = ys * idetJ, ry = -xs * idetJ, sx = -yr * idetJ, sy = xr * idetJ;
  const T g1x = tab.qdr[0][1] * rx + tab.qds[0][1] * sx, g1y = tab.qdr[0][1] * ry + tab.qds[0][1] * sy;
  const T g2x = tab.qdr[0][2] * rx + tab.qds[0][2] * sx, g2y = tab.qdr[0][2] * ry + tab.qds[0][2] * sy;
  const T hbx = E.hb1 * g1x + E.hb2 * g2x, hby = E.hb1 * g1y + E.hb2 * g2y;  // constant grad(hb)
  const int friction = ft_friction(FT) >= 0 ? ft_friction(FT) : a.friction;
  const T cfm = (friction == 0) ? g * G.man * G.man : a.cf;
  if constexpr (P == 1) {
    const T xb = acc_r(E.xb), yb = acc_r(E.yb);
    T Fx[NQ], Fy[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) Fx[q] = Fy[q] = T(0);
    if (press) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const T px = tab.ql[q][0] * vx[0] + tab.ql[q][1] * vx[1] + tab.ql[q][2] * vx[2];
        const T py = tab.ql[q][0] * vy[0] + tab.ql[q][1] * vy[1] + tab.ql[q][2] * vy[2];
        const T Hq = E.Hb + (fma(E.zs[1], tab.qphi[q][2], E.zs[0] * tab.qphi[q][1]) +
                             fma(E.hb1, tab.qphi[q][1], E.hb2 * tab.qphi[q][2]));
        setup_force<T>(F, px, py, Hq, g, Fx[q], Fy[q]);
      }
    }
    T SF[6], SS[3][2];
    if constexpr (sizeof(T) == 4 && DG_PACKED_FLUX) {
      // points (0,1), (2,3), (4,5) in packed pairs, point 6 alone
      AreaP1<f2> A2;
#pragma unroll
      for (int i = 0; i < 6; ++i) A2.SF[i] = p2(0.f);
#pragma unroll
      for (int m = 0; m < 3; ++m) A2.SS[m][0] = A2.SS[m][1] = p2(0.f);
      const f2 zs0 = p2(E.zs[0]), zs1 = p2(E.zs[1]), xs0 = p2(E.xs[0]), xs1 = p2(E.xs[1]);
      const f2 ys0 = p2(E.ys[0]), ys1 = p2(E.ys[1]), xb2 = p2(xb), yb2 = p2(yb), Hb2 = p2(E.Hb);
      const f2 hb12 = p2(E.hb1), hb22 = p2(E.hb2), H02 = p2(H0), hg2 = p2(0.5f * g);
      const f2 ghbx2 = p2(g * hbx), ghby2 = p2(g * hby), cfm2 = p2(cfm);
#pragma unroll
      for (int q = 0; q < 6; q += 2)
        area_points_p1<f2, float>(A2, tab, q, zs0, zs1, xs0, xs1, ys0, ys1, xb2, yb2, Hb2, hb12, hb22, H02, hg2,
                                  ghbx2, ghby2, cfm2, friction, make_float2(Fx[q], Fx[q + 1]),
                                  make_float2(Fy[q], Fy[q + 1]));
      AreaP1<float> A1;
#pragma unroll
      for (int i = 0; i < 6; ++i) A1.SF[i] = 0.f;
#pragma unroll
      for (int m = 0; m < 3; ++m) A1.SS[m][0] = A1.SS[m][1] = 0.f;
      area_points_p1<float, float>(A1, tab, 6, E.zs[0], E.zs[1], E.xs[0], E.xs[1], E.ys[0], E.ys[1], xb, yb, E.Hb,
                                   E.hb1, E.hb2, H0, 0.5f * g, g * hbx, g * hby, cfm, friction, Fx[6], Fy[6]);
#pragma unroll
      for (int i = 0; i < 6; ++i) SF[i] = (A2.SF[i].x + A2.SF[i].y) + A1.SF[i];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        SS[m][0] = (A2.SS[m][0].x + A2.SS[m][0].y) + A1.SS[m][0];
        SS[m][1] = (A2.SS[m][1].x + A2.SS[m][1].y) + A1.SS[m][1];
      }
    } else {
      AreaP1<T> A1;
#pragma unroll
      for (int i = 0; i < 6; ++i) A1.SF[i] = T(0);
#pragma unroll
      for (int m = 0; m < 3; ++m) A1.SS[m][0] = A1.SS[m][1] = T(0);
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        area_points_p1<T, T>(A1, tab, q, E.zs[0], E.zs[1], E.xs[0], E.xs[1], E.ys[0], E.ys[1], xb, yb, E.Hb, E.hb1,
                             E.hb2, H0, T(0.5) * g, g * hbx, g * hby, cfm, friction, Fx[q], Fy[q]);
#pragma unroll
      for (int i = 0; i < 6; ++i) SF[i] = A1.SF[i];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        SS[m][0] = A1.SS[m][0];
        SS[m][1] = A1.SS[m][1];
      }
    }
    const T gx[3] = {T(0), g1x, g2x}, gy[3] = {T(0), g1y, g2y};
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      Rz[m] = (m > 0) ? detJ * (gx[m] * SF[0] + gy[m] * SF[3]) : T(0);
      Rx[m] = detJ * (gx[m] * SF[1] + gy[m] * SF[4] + SS[m][0]);
      Ry[m] = detJ * (gx[m] * SF[2] + gy[m] * SF[5] + SS[m][1]);
    }
  } else if constexpr (sizeof(T) == 4 && DG_PACKED_FLUX) {
    // FP32: the points in packed pairs (0,1), (2,3), (4,5), (6,7); point 7 has zero weight and zero
    // basis values (the mean state, finite) and adds exact zeros
    static_assert(NQ + 1 == MAXNQP, "one padding point");
    constexpr int NS = NP - 1;
    f2 Rz2[NP], Rx2[NP], Ry2[NP];
#pragma unroll
    for (int m = 0; m < NP; ++m) Rz2[m] = Rx2[m] = Ry2[m] = p2(0.f);
    const f2 rx2 = p2(rx), ry2 = p2(ry), sx2 = p2(sx), sy2 = p2(sy), detJ2 = p2(detJ);
    const f2 H02 = p2(H0), hg = p2(0.5f * g), ghbx = p2(g * hbx), ghby = p2(g * hby), cfm2 = p2(cfm);
    const f2 xb2 = p2(acc_r(E.xb)), yb2 = p2(acc_r(E.yb)), Hb2 = p2(E.Hb), hb12 = p2(E.hb1), hb22 = p2(E.hb2);
#pragma unroll
    for (int q = 0; q < NQ + 1; q += 2) {
      f2 d = p2(0.f), qx = xb2, qy = yb2;
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        const f2 ph = vtab<f2, float>(tab.qphiT[m + 1], q);
        d = fma2(p2(E.zs[m]), ph, d);
        qx = fma2(p2(E.xs[m]), ph, qx);
        qy = fma2(p2(E.ys[m]), ph, qy);
      }
      const f2 H = add2(Hb2, add2(d, fma2(hb12, vtab<f2, float>(tab.qphiT[1], q),
                                          mul2(hb22, vtab<f2, float>(tab.qphiT[2], q)))));
      const f2 Hs = max2(H, H02);
      const f2 iH = rcp2(Hs);
      const f2 u = mul2(qx, iH), v = mul2(qy, iH);
      const f2 pp = mul2(mul2(hg, d), fma2(p2(2.f), H, neg2(d)));  // g/2 d (2H - d)
      f2 tau = p2(0.f);
      if (friction <= 1) tau = vtau(qx, qy, u, v, Hs, iH, cfm2, friction);
      float Fx0 = 0.f, Fy0 = 0.f, Fx1 = 0.f, Fy1 = 0.f;
      if (press) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          if (q + k >= NQ) continue;
          const float px = tab.ql[q + k][0] * vx[0] + tab.ql[q + k][1] * vx[1] + tab.ql[q + k][2] * vx[2];
          const float py = tab.ql[q + k][0] * vy[0] + tab.ql[q + k][1] * vy[1] + tab.ql[q + k][2] * vy[2];
          setup_force<float>(F, px, py, k ? H.y : H.x, g, k ? Fx1 : Fx0, k ? Fy1 : Fy0);
        }
      }
      const f2 sxs = fma2(ghbx, d, fma2(neg2(tau), qx, make_float2(Fx0, Fx1)));
      const f2 sys = fma2(ghby, d, fma2(neg2(tau), qy, make_float2(Fy0, Fy1)));
      const f2 fxx = fma2(qx, u, pp), fyx = mul2(qx, v), fxy = mul2(qy, u), fyy = fma2(qy, v, pp);
      const f2 wq = mul2(vtab<f2, float>(tab.qwT, q), detJ2);
      // fluxes rotated into the reference directions, with the weight
      const f2 zr = mul2(wq, fma2(rx2, qx, mul2(ry2, qy))), zs = mul2(wq, fma2(sx2, qx, mul2(sy2, qy)));
      const f2 xr = mul2(wq, fma2(rx2, fxx, mul2(ry2, fyx))), xs2 = mul2(wq, fma2(sx2, fxx, mul2(sy2, fyx)));
      const f2 yr = mul2(wq, fma2(rx2, fxy, mul2(ry2, fyy))), ys2 = mul2(wq, fma2(sx2, fxy, mul2(sy2, fyy)));
      const f2 wsx = mul2(wq, sxs), wsy = mul2(wq, sys);
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        const f2 dr = vtab<f2, float>(tab.qdrT[m], q), ds = vtab<f2, float>(tab.qdsT[m], q);
        const f2 ph = vtab<f2, float>(tab.qphiT[m], q);
        if (m > 0) Rz2[m] = fma2(dr, zr, fma2(ds, zs, Rz2[m]));
        Rx2[m] = fma2(dr, xr, fma2(ds, xs2, fma2(ph, wsx, Rx2[m])));
        Ry2[m] = fma2(dr, yr, fma2(ds, ys2, fma2(ph, wsy, Ry2[m])));
      }
    }
#pragma unroll
    for (int m = 0; m < NP; ++m) {
      Rz[m] = Rz2[m].x + Rz2[m].y;
      Rx[m] = Rx2[m].x + Rx2[m].y;
      Ry[m] = Ry2[m].x + Ry2[m].y;
    }
  } else {
#pragma unroll
    for (int m = 0; m < NP; ++m) Rz[m] = Rx[m] = Ry[m] = T(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const Trace<T> tq = trace_at<P, Pol>(E, tab.qphi[q]);
      const T Hs = max_r(tq.H, H0);
      const T iH = frcp(Hs);
      const T u = tq.qx * iH, v = tq.qy * iH;
      const T pp = pdev(tq.d, tq.H, g);
      T tau = 0;
      if (friction <= 1) tau = vtau(tq.qx, tq.qy, u, v, Hs, iH, cfm, friction);
      T Fxs = 0, Fys = 0;
      if (press) {
        const T px = tab.ql[q][0] * vx[0] + tab.ql[q][1] * vx[1] + tab.ql[q][2] * vx[2];
        const T py = tab.ql[q][0] * vy[0] + tab.ql[q][1] * vy[1] + tab.ql[q][2] * vy[2];
        setup_force<T>(F, px, py, tq.H, g, Fxs, Fys);
      }
      const T sx_ = g * tq.d * hbx - tau * tq.qx + Fxs;
      const T sy_ = g * tq.d * hby - tau * tq.qy + Fys;
      const T fxx = tq.qx * u + pp, fyx = tq.qx * v;
      const T fxy = tq.qy * u, fyy = tq.qy * v + pp;
      const T wq = tab.qw[q] * detJ;
      // each flux rotated once into the reference directions (grad phi_m = qdr grad r + qds grad s),
      // with the weight: then two products per mode and variable
      const T zr = wq * (rx * tq.qx + ry * tq.qy), zs = wq * (sx * tq.qx + sy * tq.qy);
      const T xr = wq * (rx * fxx + ry * fyx), xs2 = wq * (sx * fxx + sy * fyx);
      const T yr = wq * (rx * fxy + ry * fyy), ys2 = wq * (sx * fxy + sy * fyy);
      const T wsx = wq * sx_, wsy = wq * sy_;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        const T dr = tab.qdr[q][m], ds = tab.qds[q][m], ph = tab.qphi[q][m];
        if (m > 0) Rz[m] = fma(dr, zr, fma(ds, zs, Rz[m]));
        Rx[m] = fma(dr, xr, fma(ds, xs2, fma(ph, wsx, Rx[m])));
        Ry[m] = fma(dr, yr, fma(ds, ys2, fma(ph, wsy, Ry[m])));
      }
    }
  }
}

// ---------------------------------------------------------------------- edge phase ------
// record of a side: own (src < 32: [RV][32]) or staged halo (src < 64: [RV][HALO]) records in
// shared memory, vector-major, else the global record of element src - 64
template <int RV>
__device__ __forceinline__ void fetch_side(const uint4* own, const uint4* halo, const uint4* __restrict__ gin, int src,
                                           Raw<RV>& r) {
  if (src < 64) {  // shared memory, read as such (not through a generic address)
    const uint32_t p = smem_u32(src < 32 ? own + src : halo + (src - 32));
    constexpr uint32_t stride = 16u * TILE;  // HALO == TILE: one stride for both
#pragma unroll
    for (int v = 0; v < RV; ++v) r.v[v] = lds128(p + stride * v);
  } else {
#pragma unroll
    for (int v = 0; v < RV; ++v) r.v[v] = __ldg(gin + rec_at<RV>(src - 64, v));
  }
}

// one side's edge slot at flx[(j NPR + i) 32 + lane], pairs of T: Gz[NG], Gx[NG], Gy[NG] (, mass)
template <class T>
struct Pair;
template <>
struct Pair<float> {
  using V = float2;
};
template <>
struct Pair<double> {
  using V = double2;
};
template <class T, int NPR, int NV>
__device__ __forceinline__ void store_side(void* flx, int lane, int j, const T* vals) {
  using V = typename Pair<T>::V;
  V* f = reinterpret_cast<V*>(flx);
#pragma unroll
  for (int i = 0; i < NPR; ++i) {
    V v;
    v.x = vals[2 * i];
    v.y = (2 * i + 1 < NV) ? vals[2 * i + 1] : T(0);
    f[(j * NPR + i) * 32 + lane] = v;
  }
}
template <class T, int NPR, int NV>
__device__ __forceinline__ void load_side(const void* flx, int lane, int j, T* vals) {
  using V = typename Pair<T>::V;
  const V* f = reinterpret_cast<const V*>(flx);
#pragma unroll
  for (int i = 0; i < NPR; ++i) {
    const V v = f[(j * NPR + i) * 32 + lane];
    vals[2 * i] = v.x;
    if (2 * i + 1 < NV) vals[2 * i + 1] = v.y;
  }
}
// mass integral of a side's slot: stored (odd NG) or the sum of its Gz in point order (even NG)
template <class T, int NG, bool MASSV>
__device__ __forceinline__ T side_mass(const T* vals) {
  if constexpr (MASSV) {
    return vals[3 * NG];
  } else {
    T m = vals[0];
#pragma unroll
    for (int k = 1; k < NG; ++k) m += vals[k];
    return m;
  }
}

// reflective wall seen from a trace, along the unit outward normal n: the numerical flux between
// the trace and its mirror image in closed form (Roe: q.n (q.n / Hs + c) n; LLF adds |q.n| q.n / Hs
// n), plus the pressure relative to the side's own mean; no mass crosses
template <int FLUX, class T>
__device__ __forceinline__ T wall_coef(const Trace<T>& t, T nx, T ny, T g, T H0) {
  const T qn = t.qx * nx + t.qy * ny;
  const T Hs = max_r(t.H, H0);
  const T iH = frcp(Hs);
  const T c = fsqrt_pos(g * Hs);
  const T un = (FLUX == 1) ? (qn + abs_r(qn)) * iH : qn * iH;
  return qn * (un + c) + pdev(t.d, t.H, g);
}

template <int P, int FLUX, class Pol, int FT>
__device__ __forceinline__ void tile_edge(const StageArgs<Pol>& a, const ScenDev& S, const uint4* own,
                                          const uint4* halo, const EdgeDesc<typename Pol::T>* desc, void* flx, int i,
                                          const typename Pol::T (*ephi)[P + 1][np_of(P)], const float4* ephi4,
                                          double t64,
                                          typename Pol::Acc& bdry_acc) {
  using T = typename Pol::T;
  using L = TileLayout<P, Pol>;
  constexpr int NG = P + 1, RV = L::RV, NPR = L::NPR, NV = L::NV;
  constexpr bool MASSV = L::MASSV;
  const RefTab<T>& tab = ctab<T, P>();
  const T g = a.g, H0 = a.H0;
  int sL, sR;
  T lnx, lny;  // L's scaled outward normal
  get_desc(desc, i, sL, sR, lnx, lny);
  const int jL = sL & 3, srcL = sL >> 2;
  Raw<RV> rl;
  fetch_side<RV>(own, halo, a.in, srcL, rl);
  Elem<P, Pol> EL;
  unpack<P>(rl, EL);
  T len, il;  // edge length and its inverse
  if constexpr (sizeof(T) == 4) {
    const T l2 = lnx * lnx + lny * lny;
    il = mufu_rsqrt(l2);
    len = l2 * il;
  } else {
    len = fsqrt_pos(lnx * lnx + lny * lny);
    il = frcp(len);
  }
  const T nx = lnx * il, ny = lny * il;
  constexpr bool P1F = P == 1 && sizeof(T) == 4;  // basis values of both points in one 16-byte read
  Trace<T> tl[NG], tr[NG];
  if constexpr (P1F) {
    const float4 b = ephi4[jL];
    tl[0] = trace_p1(EL, b.x, b.y);
    tl[NG - 1] = trace_p1(EL, b.z, b.w);
  } else {
#pragma unroll
    for (int k = 0; k < NG; ++k) tl[k] = trace_at<P, Pol>(EL, ephi[jL][k]);
  }
  // boundary kind (an instantiation without a kind treats such an edge as a wall; the host never
  // selects it for a run that has one)
  const bool interior = sR >= 0;
  const bool river_e = (FT & FT_RIVER) && sR <= -2 - MAXSEG;
  const bool ocean_e = (FT & FT_OCEAN) && sR <= -2 && sR > -2 - MAXSEG;
  const bool land = !interior && !river_e && !ocean_e;
  const bool dryL = (EL.flags & FLAG_DRY) != 0;
  bool dryR = false, river = false;
  int jR = 0, srcR = 64;
  T dcRL = T(0), qr = T(0);
  if (interior) {
    jR = sR & 3;
    srcR = sR >> 2;
    Raw<RV> rr;
    fetch_side<RV>(own, halo, a.in, srcR, rr);
    Elem<P, Pol> ER;
    unpack<P>(rr, ER);
    dcRL = acc_sub_r(ER.zb, EL.zb);
    dryR = (ER.flags & FLAG_DRY) != 0;
    if constexpr (P1F) {  // R's point 1 - k is L's point k
      const float4 b = ephi4[jR];
      tr[0] = trace_p1(ER, b.z, b.w);
      tr[NG - 1] = trace_p1(ER, b.x, b.y);
    } else {
#pragma unroll
      for (int k = 0; k < NG; ++k) tr[k] = trace_at<P, Pol>(ER, ephi[jR][NG - 1 - k]);  // the same points
    }
  } else if (river_e) {  // river: interior elevation, prescribed normal discharge
    const int rs = min(-2 - MAXSEG - sR, MAXRIV - 1);
    qr = river_at<T>(S, rs, t64);
    river = true;
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      tr[k] = tl[k];
      tr[k].qx = -qr * nx;
      tr[k].qy = -qr * ny;
    }
  } else if (ocean_e) {  // ocean: tidal elevation, interior discharge
    const int seg = min(-2 - sR, MAXSEG - 1);
    const T zbc = tide_at<T>(S, seg, t64);
    const T dgh = acc_r(acc_addr(acc_neg(EL.zb), zbc));  // ghost zeta - mean of L
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      tr[k] = tl[k];
      tr[k].H = tl[k].H + (dgh - tl[k].d);
      tr[k].d = dgh;
    }
  }
  constexpr bool PK = DG_PACKED_FLUX && P == 1 && sizeof(T) == 4;  // both points in packed FP32x2
  T fz[NG], fx[NG], fy[NG];
  T ec = T(0);  // mass flux integral along n (L's outward normal)
  bool closed = land;
  FluxAux2 ax;  // packed path: per-side quantities for the wall flux
  if constexpr (PK) {
    // every edge takes the flux evaluation (a land edge against its own trace: the wall below needs
    // only the left side's quantities), so that no lane takes a separate wall path
    if (land) {
#pragma unroll
      for (int k = 0; k < NG; ++k) tr[k] = tl[k];
    }
    const Trace2 L2{make_float2(tl[0].d, tl[1].d), make_float2(tl[0].H, tl[1].H), make_float2(tl[0].qx, tl[1].qx),
                    make_float2(tl[0].qy, tl[1].qy)};
    const Trace2 R2{make_float2(tr[0].d, tr[1].d), make_float2(tr[0].H, tr[1].H), make_float2(tr[0].qx, tr[1].qx),
                    make_float2(tr[0].qy, tr[1].qy)};
    f2 fz2, fx2, fy2;
    edge_flux_pair<FLUX>(L2, R2, p2(dcRL), p2(nx), p2(ny), g, H0, fz2, fx2, fy2, ax);
    fz[0] = fz2.x; fz[1] = fz2.y;
    fx[0] = fx2.x; fx[1] = fx2.y;
    fy[0] = fy2.x; fy[1] = fy2.y;
  }
  if (!land) {
    if constexpr (!PK && P == 2 && sizeof(T) == 4 && DG_PACKED_FLUX) {  // points 0 and 1 packed, point 2 alone
      const Trace2 L2{make_float2(tl[0].d, tl[1].d), make_float2(tl[0].H, tl[1].H), make_float2(tl[0].qx, tl[1].qx),
                      make_float2(tl[0].qy, tl[1].qy)};
      const Trace2 R2{make_float2(tr[0].d, tr[1].d), make_float2(tr[0].H, tr[1].H), make_float2(tr[0].qx, tr[1].qx),
                      make_float2(tr[0].qy, tr[1].qy)};
      f2 fz2, fx2, fy2;
      FluxAux2 ax2;
      edge_flux_pair<FLUX>(L2, R2, p2(dcRL), p2(nx), p2(ny), g, H0, fz2, fx2, fy2, ax2);
      fz[0] = fz2.x; fz[1] = fz2.y;
      fx[0] = fx2.x; fx[1] = fx2.y;
      fy[0] = fy2.x; fy[1] = fy2.y;
      edge_flux<FLUX, T>(tl[NG - 1], tr[NG - 1], dcRL, nx, ny, g, H0, fz[NG - 1], fx[NG - 1], fy[NG - 1]);
    } else if constexpr (!PK) {
#pragma unroll
      for (int k = 0; k < NG; ++k) edge_flux<FLUX, T>(tl[k], tr[k], dcRL, nx, ny, g, H0, fz[k], fx[k], fy[k]);
    }
    if (river) {
#pragma unroll
      for (int k = 0; k < NG; ++k) fz[k] = -qr;  // the specified normal flow is the mass flux
    }
#pragma unroll
    for (int k = 0; k < NG; ++k) ec = fma(tab.gw[k], fz[k], ec);
    ec = ec * (T(0.5) * len);
    // wet/dry closure: no water leaves a dry element (interior: either side; ocean/river: L)
    closed = interior ? ((dryL && ec > T(0)) || (dryR && ec < T(0))) : (dryL && ec > T(0));
  }
  const T hl = T(0.5) * len;
  T vals[NV + 1];
  if (srcL < TILE) {  // L's slot, in L's point order
    if (!closed) {
      if constexpr (PK) {
        const f2 hq = p2(0.25f * g), dc = p2(dcRL);  // the mean of the sides' g/2 d (2H - d)
        const f2 Ld = make_float2(tl[0].d, tl[1].d), LH = make_float2(tl[0].H, tl[1].H);
        const f2 Rd = add2(make_float2(tr[0].d, tr[1].d), dc), RH = make_float2(tr[0].H, tr[1].H);
        const f2 pp = mul2(hq, fma2(Ld, fma2(p2(2.f), LH, neg2(Ld)), mul2(Rd, fma2(p2(2.f), RH, neg2(Rd)))));
        const f2 wk = mul2(make_float2(tab.gw[0], tab.gw[1]), p2(hl));
        const f2 vz = mul2(wk, make_float2(fz[0], fz[1]));
        const f2 vx = mul2(wk, fma2(pp, p2(nx), make_float2(fx[0], fx[1])));
        const f2 vy = mul2(wk, fma2(pp, p2(ny), make_float2(fy[0], fy[1])));
        vals[0] = vz.x; vals[1] = vz.y; vals[2] = vx.x; vals[3] = vx.y; vals[4] = vy.x; vals[5] = vy.y;
      } else {
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          const T p = T(0.5) * (pdev(tl[k].d, tl[k].H, g) + pdev(tr[k].d + dcRL, tr[k].H, g));
          const T wk = tab.gw[k] * hl;
          vals[k] = wk * fz[k];
          vals[NG + k] = wk * (fx[k] + p * nx);
          vals[2 * NG + k] = wk * (fy[k] + p * ny);
        }
      }
      if (MASSV) vals[3 * NG] = ec;
    } else if constexpr (PK) {  // wall: q.n (q.n / Hs + c) + pressure relative to L's mean (LLF: (q.n + |q.n|) / Hs)
      const f2 Ld = make_float2(tl[0].d, tl[1].d), LH = make_float2(tl[0].H, tl[1].H);
      const f2 un = (FLUX == 1) ? mul2(add2(ax.mL, abs2(ax.mL)), ax.iL) : mul2(ax.mL, ax.iL);
      const f2 wl = fma2(ax.mL, fma2(p2(fsqrt_pos(g)), ax.sL, un), mul2(p2(0.5f * g), mul2(Ld, fma2(p2(2.f), LH, neg2(Ld)))));
      const f2 cw = mul2(mul2(make_float2(tab.gw[0], tab.gw[1]), p2(hl)), wl);
      const f2 vx = mul2(cw, p2(nx)), vy = mul2(cw, p2(ny));
      vals[0] = vals[1] = T(0);
      vals[2] = vx.x; vals[3] = vx.y; vals[4] = vy.x; vals[5] = vy.y;
    } else {
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const T cw = tab.gw[k] * hl * wall_coef<FLUX, T>(tl[k], nx, ny, g, H0);
        vals[k] = T(0);
        vals[NG + k] = cw * nx;
        vals[2 * NG + k] = cw * ny;
      }
      if (MASSV) vals[3 * NG] = T(0);
    }
    store_side<T, NPR, NV>(flx, srcL, jL, vals);
    if (!interior && !land && !closed) bdry_acc = acc_addr(bdry_acc, -side_mass<T, NG, MASSV>(vals));  // inflow
  }
  if (interior && srcR < TILE) {  // R's slot, in R's point order (its point k is L's NG-1-k)
    if (!closed) {
      if constexpr (PK) {  // R's point kr is L's point 1 - kr
        const f2 hq = p2(0.25f * g), dc = p2(dcRL);  // the mean of the sides' g/2 d (2H - d)
        const f2 Rd = make_float2(tr[1].d, tr[0].d), RH = make_float2(tr[1].H, tr[0].H);
        const f2 Ld = sub2(make_float2(tl[1].d, tl[0].d), dc), LH = make_float2(tl[1].H, tl[0].H);
        const f2 pp = mul2(hq, fma2(Rd, fma2(p2(2.f), RH, neg2(Rd)), mul2(Ld, fma2(p2(2.f), LH, neg2(Ld)))));
        const f2 wk = mul2(make_float2(tab.gw[0], tab.gw[1]), p2(-hl));
        const f2 vz = mul2(wk, make_float2(fz[1], fz[0]));
        const f2 vx = mul2(wk, fma2(pp, p2(nx), make_float2(fx[1], fx[0])));
        const f2 vy = mul2(wk, fma2(pp, p2(ny), make_float2(fy[1], fy[0])));
        vals[0] = vz.x; vals[1] = vz.y; vals[2] = vx.x; vals[3] = vx.y; vals[4] = vy.x; vals[5] = vy.y;
      } else {
#pragma unroll
        for (int kr = 0; kr < NG; ++kr) {
          const int k = NG - 1 - kr;
          const T p = T(0.5) * (pdev(tr[k].d, tr[k].H, g) + pdev(tl[k].d - dcRL, tl[k].H, g));
          const T wk = tab.gw[kr] * hl;
          vals[kr] = -(wk * fz[k]);
          vals[NG + kr] = -(wk * (fx[k] + p * nx));
          vals[2 * NG + kr] = -(wk * (fy[k] + p * ny));
        }
      }
      if (MASSV) vals[3 * NG] = -ec;
    } else if constexpr (PK) {  // wall seen from R along -n: q.n_R = -mR
      const f2 mR = neg2(ax.mR);
      const f2 Rd = make_float2(tr[0].d, tr[1].d), RH = make_float2(tr[0].H, tr[1].H);
      const f2 un = (FLUX == 1) ? mul2(add2(mR, abs2(mR)), ax.iR) : mul2(mR, ax.iR);
      const f2 wr = fma2(mR, fma2(p2(fsqrt_pos(g)), ax.sR, un), mul2(p2(0.5f * g), mul2(Rd, fma2(p2(2.f), RH, neg2(Rd)))));
      // R's point kr is L's point 1 - kr
      const f2 cw = mul2(mul2(make_float2(tab.gw[0], tab.gw[1]), p2(-hl)), make_float2(wr.y, wr.x));
      const f2 vx = mul2(cw, p2(nx)), vy = mul2(cw, p2(ny));
      vals[0] = vals[1] = T(0);
      vals[2] = vx.x; vals[3] = vx.y; vals[4] = vy.x; vals[5] = vy.y;
    } else {
#pragma unroll
      for (int kr = 0; kr < NG; ++kr) {
        const int k = NG - 1 - kr;
        const T cw = tab.gw[kr] * hl * wall_coef<FLUX, T>(tr[k], -nx, -ny, g, H0);
        vals[kr] = T(0);
        vals[NG + kr] = -(cw * nx);
        vals[2 * NG + kr] = -(cw * ny);
      }
      if (MASSV) vals[3 * NG] = T(0);
    }
    store_side<T, NPR, NV>(flx, srcR, jR, vals);
  }
}

// -------------------------------------------------------------------------- the kernel ---
#ifndef DG_TILE_MAXNREG
// register budget: mixed p = 1 at 128 (16 warps per SM, as its shared memory allows); elsewhere
// shared memory allows about 10 (mixed p = 2) or 9 (FP64 p = 1) warps, which leaves 200 or more
#define DG_TILE_BOUNDS __maxnreg__(sizeof(typename Pol::T) == 4 ? (P == 1 ? 128 : 200) : 224)
#else
#define DG_TILE_BOUNDS __maxnreg__(DG_TILE_MAXNREG)
#endif

template <int P, int FLUX, class Pol, int FT = FT_ALL>
__global__ void DG_TILE_BOUNDS tile_kernel(const StageArgs<Pol> a) {
  using T = typename Pol::T;
  using Acc = typename Pol::Acc;
  using L = TileLayout<P, Pol>;
  constexpr int NP = np_of(P), NS = NP - 1, NG = P + 1, RV = L::RV, GV = L::GV, NPR = L::NPR, NV = L::NV;
  const RefTab<T>& tab = ctab<T, P>();

  // edge basis values, read at edge-dependent indices; at p = 1 in FP32 also one 16-byte row per
  // edge {phi_1, phi_2 at point 0, phi_1, phi_2 at point 1} (phi_0 is constant and not read)
  __shared__ T s_ephi[3][NG][NP];
  __shared__ float4 s_ephi4[3];
  extern __shared__ uint4 tsm[];
  const int tid = threadIdx.x;
  for (int i = tid; i < 3 * NG * NP; i += blockDim.x) {
    const int j = i / (NG * NP), k = (i / NP) % NG, m = i % NP;
    s_ephi[j][k][m] = tab.ephi[j][k][m];
  }
  if (P == 1 && tid < 3)
    s_ephi4[tid] = make_float4((float)tab.ephi[tid][0][1], (float)tab.ephi[tid][0][2],
                               (float)tab.ephi[tid][NG - 1][1], (float)tab.ephi[tid][NG - 1][2]);
  __syncthreads();
  const int lane = tid & 31;
  uint4* Wm = tsm + (size_t)(tid >> 5) * L::VEC;
  uint4* halo = Wm + L::HAL;                                       // [HALO][RV]
  EdgeDesc<T>* desc = reinterpret_cast<EdgeDesc<T>*>(Wm + L::DESC);  // [96]
  const uint32_t bar0 = smem_u32(Wm + L::BAR), bar1 = bar0 + 8;
  if (lane == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar1, 1);
    mbar_fence_init();
  }
  __syncwarp();
  const unsigned lt = (1u << lane) - 1u;
  const int gw = blockIdx.x * (blockDim.x >> 5) + (tid >> 5);
  const int W = gridDim.x * (blockDim.x >> 5);
  // one TMA batch: the tile's records, geometry and neighbour codes into a buffer (lane 0)
  auto issue = [&](int t, int b) {
    if (lane == 0) {
      uint4* buf = Wm + (b ? L::BUF1 : L::BUF0);
      const uint32_t bar = b ? bar1 : bar0;
      fence_proxy_async();
      mbar_expect_tx(bar, L::TILE_BYTES);
      bulk_g2s(smem_u32(buf), a.in + (size_t)t * TILE * RV, 16u * TILE * RV, bar);
      bulk_g2s(smem_u32(buf + L::O_GEO), a.geo + (size_t)t * TILE * GV, 16u * TILE * GV, bar);
      bulk_g2s(smem_u32(buf + L::O_NBR), a.nbr + (size_t)t * TILE, 16u * TILE, bar);
      bulk_g2s(smem_u32(buf + L::O_XY), a.xy0 + (size_t)t * L::XV, 16u * L::XV, bar);
      bulk_g2s(smem_u32(buf + L::O_META), a.tile_meta + t, 16u, bar);
    }
  };
  const double stepd = (double)a.ctl->step + a.cst;
  Acc rain_acc = acc_make<Acc>(0.f, 0.f, 0.0), bdry_acc = acc_make<Acc>(0.f, 0.f, 0.0);
  int cur = -1;
  // constants of the current scenario, reloaded when a tile of another scenario comes
  const ScenDev* Sp = a.scen;
  double t64 = 0.0;
  int rain_kind = 0, press = 0;
  uint32_t ph = 0;  // parity of the next completion: bit 0 buffer 0, bit 1 buffer 1
  if (gw < a.ntiles) issue(gw, 0);

  int it = 0;
  for (int tile = gw; tile < a.ntiles; tile += W, ++it) {
    const int b = it & 1;
    if (tile + W < a.ntiles) issue(tile + W, b ^ 1);  // the other buffer's tile was consumed last iteration
    if (!__all_sync(0xffffffffu, mbar_wait(b ? bar1 : bar0, (ph >> b) & 1u))) {
      tile_timeout(a, b ? bar1 : bar0, (ph >> b) & 1u, lane);
      return;
    }
    ph ^= 1u << b;
    uint4* const buf = Wm + (b ? L::BUF1 : L::BUF0);
    const uint4* own = buf;                           // [RV][32] records
    const uint4* geoS = own + L::O_GEO;               // [32][GV]
    void* flx = buf + L::O_FLX;                       // [3][NPR][32] pairs, over geoS .. meta
    const int4* nbrS = reinterpret_cast<const int4*>(own + L::O_NBR);
    const int4 meta = reinterpret_cast<const int4*>(own + L::O_META)[0];
    const int sc = meta.x, present = meta.y;
    if (present == 0) {  // padding tile: no element (uniform over the warp)
      __syncwarp();
      continue;
    }
    if (sc != cur) {
      if (cur >= 0 && !a.tune) flush_ledger<P, Pol>(a, cur, gw, rain_acc, bdry_acc);
      cur = sc;
      Sp = a.scen + sc;
      t64 = Sp->d.t0 + stepd * Sp->d.dt;  // stage time, formed in FP64
      rain_kind = ft_rain(FT) >= 0 ? ft_rain(FT) : Sp->rain_kind;
      press = (FT & FT_PRESS) ? Sp->press : 0;
    }
    const ScenDev& S = *Sp;
    const int e0 = tile * TILE, e = e0 + lane;
    const bool valid = lane < present;
    const T t = (T)t64;
    if (a.has_n && lane == 0) bulk_prefetch_l2(a.wn + (size_t)e0 * RV, 16u * TILE * RV);  // read in phase B

    // ---- edge ownership: boundary edges, edges to out-of-tile neighbours, and in-tile edges to a
    // higher index belong to this lane; out-of-tile neighbours get a halo slot.  Edge slots: the
    // interior edges first, then the boundary edges (fewer divergent rounds).
    const int4 nb = valid ? nbrS[lane] : make_int4(-1, -1, -1, -1);
    const int code[3] = {nb.x, nb.y, nb.z};
    bool own_e[3], out[3];
    int eidx[3], hslot[3];
    unsigned bi[3], bb[3];
    int nint = 0, hbase = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int c = code[j];
      const int n = c >> 2;
      const bool inside = c >= 0 && n >= e0 && n < e0 + TILE;
      own_e[j] = valid && (c < 0 || !inside || e < n);
      out[j] = valid && c >= 0 && !inside;
      bi[j] = __ballot_sync(0xffffffffu, own_e[j] && c >= 0);
      bb[j] = __ballot_sync(0xffffffffu, own_e[j] && c < 0);
      const unsigned bh = __ballot_sync(0xffffffffu, out[j]);
      hslot[j] = hbase + __popc(bh & lt);
      hbase += __popc(bh);
      nint += __popc(bi[j]);
    }
    {
      int ib = 0, bbase = nint;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        eidx[j] = code[j] >= 0 ? ib + __popc(bi[j] & lt) : bbase + __popc(bb[j] & lt);
        ib += __popc(bi[j]);
        bbase += __popc(bb[j]);
      }
    }
    const int nedge = nint + __popc(bb[0]) + __popc(bb[1]) + __popc(bb[2]);
#pragma unroll
    for (int j = 0; j < 3; ++j)
      if (out[j] && hslot[j] < HALO) {
#pragma unroll
        for (int v = 0; v < RV; ++v) cp_async16(halo + v * HALO + hslot[j], a.in + rec_at<RV>(code[j] >> 2, v));
      }
    cp_async_commit();
    Geo<Pol> G;
    if (valid) geo_from(geoS + lane * GV, nb, G);
    // edge descriptors {left side, right side or boundary code}
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      if (!own_e[j]) continue;
      const int c = code[j];
      const int me = (lane << 2) | j;
      int sL = me, sR = c;
      T lnx = G.lnx[j], lny = G.lny[j];
      if (c >= 0) {
        const int n = c >> 2, jn = c & 3;
        if (!out[j]) {
          sR = ((n - e0) << 2) | jn;
        } else {
          const int other = (((hslot[j] < HALO) ? (32 + hslot[j]) : (64 + n)) << 2) | jn;
          if (e < n) {
            sR = other;
          } else {  // the neighbour has the lower index: it is the left side
            sL = other;
            sR = me;
            lnx = -lnx;
            lny = -lny;
          }
        }
      }
      put_desc(desc, eidx[j], sL, sR, lnx, lny);
    }

    // ---- element phase A: area integrals and rain, while the halo copies are in flight
    T Rz[NP], Rx[NP], Ry[NP];
    T Re = 0;
    if (valid) {
      // gridded rain: node indices now (coalesced), their nodal rates after the area integrals
      const int4 nd = (rain_kind == 3) ? __ldg(a.nodes + e) : make_int4(0, 0, 0, 0);
      Elem<P, Pol> E;
      {
        Raw<RV> r;
#pragma unroll
        for (int v = 0; v < RV; ++v) r.v[v] = own[v * TILE + lane];
        unpack<P>(r, E);
      }
      // vertex coordinates: the first vertex, then along the edge vectors t_j = (-ln_j.y, ln_j.x)
      T vx[3] = {0, 0, 0}, vy[3] = {0, 0, 0};
      if (press || rain_kind == 2) {
        const T* x0 = reinterpret_cast<const T*>(own + L::O_XY) + 2 * lane;
        vx[0] = x0[0];
        vy[0] = x0[1];
        vx[1] = vx[0] - G.lny[0];
        vy[1] = vy[0] + G.lnx[0];
        vx[2] = vx[0] + G.lny[2];
        vy[2] = vy[0] - G.lnx[2];
      }
      tile_area<P, Pol, FT>(E, G, S, a, press, vx, vy, Rz, Rx, Ry);
      // forcing: element rain = mean of the three nodal rates (Eq. rain)
      if (rain_kind == 1) {
        Re = a.rain_e[e];
      } else if (rain_kind == 2) {  // radial storm profile at the three vertices
        const ForcingT<T>& F = forcing<T>(S);
        const T tt = t - F.storm[7];
        const T cx = F.storm[0] + F.storm[2] * tt, cy = F.storm[1] + F.storm[3] * tt;
        const T rp = F.storm[4], rm = F.storm[5], re = F.storm[6];
        T acc = 0;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const T dx = vx[i] - cx, dy = vy[i] - cy;
          const T r = fsqrt0(dx * dx + dy * dy);
          if constexpr (sizeof(T) == 4)  // with 1 / rm and log2(e) / re formed once on the host
            acc += (r < rm) ? rp * fmaf(0.5f * F.storm[8], r, 0.5f) : rp * mufu_ex2((rm - r) * F.storm[9]);
          else
            acc += (r < rm) ? rp * (T(0.5) + T(0.5) * fdiv(r, rm)) : rp * fexp(-fdiv(r - rm, re));
        }
        Re = acc * T(1.0 / 3.0);
      } else if (rain_kind == 3) {  // gridded: nodal rates interpolated by the node kernel of this stage
        Re = (a.rain_node[nd.x] + a.rain_node[nd.y] + a.rain_node[nd.z]) * T(1.0 / 3.0);
      }
    }
    cp_async_wait_all();
    __syncwarp();

    // ---- edge phase: each edge touching the tile once, one per lane and round
    for (int r = 0; r * 32 < nedge; ++r) {
      const int i = r * 32 + lane;
      if (i < nedge) tile_edge<P, FLUX, Pol, FT>(a, S, own, halo, desc, flx, i, s_ephi, s_ephi4, t64, bdry_acc);
    }
    fence_proxy_async();  // the slots' generic writes before the TMA batch that later refills the buffer
    __syncwarp();

    // ---- element phase B: lift, inverse mass, stage combination, positive-depth operator
    if (valid) {
      Elem<P, Pol> E;
      {
        Raw<RV> r;
#pragma unroll
        for (int v = 0; v < RV; ++v) r.v[v] = own[v * TILE + lane];
        unpack<P>(r, E);
      }
      Acc massout;  // edge mass outflow (volume per second), summed exactly over the three sides
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T vals[NV + 1];
        load_side<T, NPR, NV>(flx, lane, j, vals);
#pragma unroll
        for (int k = 0; k < NG; ++k) {
#pragma unroll
          for (int m = 0; m < NP; ++m) {
            const T ph_ = tab.ephi[j][k][m];
            if (m > 0) Rz[m] = fma(-ph_, vals[k], Rz[m]);
            Rx[m] = fma(-ph_, vals[NG + k], Rx[m]);
            Ry[m] = fma(-ph_, vals[2 * NG + k], Ry[m]);
          }
        }
        const T ms = side_mass<T, NG, L::MASSV>(vals);
        massout = (j == 0) ? acc_make<Acc>(ms, T(0), ms) : acc_addr(massout, ms);
      }
      if (E.flags & FLAG_DRY) {  // the momentum equations are not advanced on dry elements
#pragma unroll
        for (int m = 0; m < NP; ++m) Rx[m] = Ry[m] = 0;
      }
      // Shu-Osher combination: out = a_n w^n + a_in w^in + beta dt M^{-1} R
      const T idetJ = T(2) * acc_r(G.invA);
      const Acc an = acc_make<Acc>(a.a_n_hi, a.a_n_lo, a.a_n);
      const Acc ain = acc_make<Acc>(a.a_in_hi, a.a_in_lo, a.a_in);
      const Acc bdt = acc_make<Acc>(S.bdt_hi[a.stage], S.bdt_lo[a.stage], S.bdt[a.stage]);
      // mean rates: d(zeta_bar)/dt = R_e - massout / A;  d(q_bar)/dt = phi_0 R_0 / detJ
      const Acc zrate = acc_addr(acc_neg(acc_mul(massout, G.invA)), Re);
      const T xrate = tab.phi0 * Rx[0] * idetJ, yrate = tab.phi0 * Ry[0] * idetJ;
      Elem<P, Pol> O = E;
      Elem<P, Pol> Wn = E;
      if (a.has_n) {
        Raw<RV> rn;
#pragma unroll
        for (int v = 0; v < RV; ++v) rn.v[v] = __ldg(a.wn + rec_at<RV>(e, v));
        unpack<P>(rn, Wn);
      }
      const T an_r = (sizeof(T) == 4) ? (T)a.a_n_hi : (T)a.a_n, ain_r = (sizeof(T) == 4) ? (T)a.a_in_hi : (T)a.a_in;
      {
        Acc z, x, y;
        constexpr int PW = ft_pow2(FT);
        if (sizeof(T) == 4 && (PW == 1 || (PW == -1 && a.pow2))) {  // exact scaling of both words by a power of two
          z = acc_scale2(E.zb, ain_r);
          x = acc_scale2(E.xb, ain_r);
          y = acc_scale2(E.yb, ain_r);
          if (a.has_n) {
            z = acc_addf(z, acc_scale2(Wn.zb, an_r));
            x = acc_addf(x, acc_scale2(Wn.xb, an_r));
            y = acc_addf(y, acc_scale2(Wn.yb, an_r));
          }
        } else {
          z = acc_mul(ain, E.zb);
          x = acc_mul(ain, E.xb);
          y = acc_mul(ain, E.yb);
          if (a.has_n) {
            z = acc_add(z, acc_mul(an, Wn.zb));
            x = acc_add(x, acc_mul(an, Wn.xb));
            y = acc_add(y, acc_mul(an, Wn.yb));
          }
        }
        O.zb = acc_addf(z, acc_mul(bdt, zrate));
        O.xb = acc_addr(x, acc_r(bdt) * xrate);
        O.yb = acc_addr(y, acc_r(bdt) * yrate);
      }
      const T bdt_r = acc_r(bdt);
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        T z = ain_r * E.zs[m] + bdt_r * (Rz[m + 1] * idetJ);
        T x = ain_r * E.xs[m] + bdt_r * (Rx[m + 1] * idetJ);
        T y = ain_r * E.ys[m] + bdt_r * (Ry[m + 1] * idetJ);
        if (a.has_n) {
          z = fma(an_r, Wn.zs[m], z);
          x = fma(an_r, Wn.xs[m], x);
          y = fma(an_r, Wn.ys[m], y);
        }
        O.zs[m] = z;
        O.xs[m] = x;
        O.ys[m] = y;
      }
      apply_positivity<P, Pol>(O, G, e, a, &a.ctl->err);
      Raw<RV> ro;
      pack<P>(O, ro);
      store_raw<RV>(a.out, e, ro);
      rain_acc = acc_addf(rain_acc, acc_mulr(G.A, Re));
    }
    __syncwarp();  // this tile's shared data is consumed: its buffers may be refilled
  }
  if (cur >= 0 && !a.tune) flush_ledger<P, Pol>(a, cur, gw, rain_acc, bdry_acc);

  // launch epilogue: the last CTA to finish advances the step counter after the final stage
  if (a.last && !a.tune) {
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      const unsigned tk = atomicAdd(&a.ctl->ticket, 1u);
      if (tk == gridDim.x - 1) {
        a.ctl->ticket = 0;
        a.ctl->step += 1ull;
        __threadfence();
      }
    }
  }
}

}  // namespace dg
