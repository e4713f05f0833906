// stage.cuh -- the fused DG stage kernel for sm_103a.
//
// One thread owns one triangle and, per Runge-Kutta stage (Sec. 2.2, Eq. RKSSP):
//   1. evaluates the numerical flux on its three edges at p+1 Gauss points (Sec. 2.3: Roe or
//      LLF; ghost states for land and ocean boundaries; the wet/dry closure of Sec. 2.4),
//   2. integrates the area terms of Eq. elem_weak_form (flux divergence, balance term
//      g zeta grad(hb), Manning friction, pressure set-up, element rain of Eq. rain),
//   3. applies the diagonal inverse mass matrix of the orthonormal basis (Eq. dubiner),
//   4. forms the Shu-Osher combination with the step's initial state,
//   5. applies the positive-depth operator M Pi_h (Sec. 2.4) and stores the record,
//   6. adds its rain and boundary volumes to per-tile ledger partials.
// Interior edge fluxes are computed by both neighbours in one canonical orientation (the lower
// element index is "left"), so both apply bitwise-opposite mass fluxes and mass is conserved.
//
// Pressure and balance terms are evaluated relative to the element's own mean elevation c:
// the identity  <P_c n, v> - (grad v, P_c) - (g c grad hb, v) = 0  with P_c = g/2 c (c + 2 hb)
// (exact for piecewise-linear hb and the degree-(2p+1) rule) is subtracted from Eq.
// elem_weak_form.  Nothing changes in exact arithmetic; in floating point the large terms
// g hb zeta cancel before rounding, which keeps lake-at-rest exact in FP32.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "args.h"
#include "layout.h"


namespace dg {

// ------------------------------------------------------------ float-float (FP32 pairs) ---
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ ff quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  ff t = two_sum(a.lo, b.lo);
  ff u = quick_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return quick_two_sum(u.hi, __fadd_rn(u.lo, t.lo));
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
  ff s = two_sum(a.hi, b);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ float ff_to_f(ff a) { return __fadd_rn(a.hi, a.lo); }
// a - b rounded to float; exactly antisymmetric under swapping a and b
__device__ __forceinline__ float ff_diff(ff a, ff b) {
  ff s = two_sum(a.hi, -b.hi);
  return __fadd_rn(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}
__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }

// accumulator overloads: double (FP64 path) and ff (mixed path)
__device__ __forceinline__ double acc_r(double a) { return a; }
__device__ __forceinline__ float acc_r(ff a) { return ff_to_f(a); }
__device__ __forceinline__ double acc_d(double a) { return a; }
__device__ __forceinline__ double acc_d(ff a) { return ff_to_d(a); }
__device__ __forceinline__ double acc_diff(double a, double b) { return a - b; }
__device__ __forceinline__ float acc_diff(ff a, ff b) { return ff_diff(a, b); }
__device__ __forceinline__ double acc_add(double a, double b) { return a + b; }
__device__ __forceinline__ ff acc_add(ff a, ff b) { return ff_add(a, b); }
// a + b with one two-sum: the error is within a few ulps of the low word of the larger operand
// (no cancellation between the low words is recovered); for sums of like-signed terms and small
// increments, as in the stage combination and the ledgers
__device__ __forceinline__ double acc_addf(double a, double b) { return a + b; }
__device__ __forceinline__ ff acc_addf(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
// a - b rounded to the working precision (float: within an ulp, from the words' differences)
__device__ __forceinline__ double acc_sub_r(double a, double b) { return a - b; }
__device__ __forceinline__ float acc_sub_r(ff a, ff b) { return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo)); }
// a + b rounded to the working precision (float: within an ulp, without the float-float sum)
__device__ __forceinline__ double acc_sum_r(double a, double b) { return a + b; }
__device__ __forceinline__ float acc_sum_r(ff a, ff b) { return __fadd_rn(__fadd_rn(a.hi, b.hi), __fadd_rn(a.lo, b.lo)); }
__device__ __forceinline__ double acc_addr(double a, double b) { return a + b; }
__device__ __forceinline__ ff acc_addr(ff a, float b) { return ff_add_f(a, b); }
__device__ __forceinline__ double acc_mul(double a, double b) { return a * b; }
__device__ __forceinline__ ff acc_mul(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ double acc_mulr(double a, double b) { return a * b; }
__device__ __forceinline__ ff acc_mulr(ff a, float b) { return ff_mul_f(a, b); }
__device__ __forceinline__ void acc_set(double& a, double v) { a = v; }
__device__ __forceinline__ void acc_set(ff& a, double v) {
  a.hi = (float)v;
  a.lo = (float)(v - (double)a.hi);
}
// scaling by a power of two (exact in both words of a float-float)
__device__ __forceinline__ double acc_scale2(double a, double c) { return a * c; }
__device__ __forceinline__ ff acc_scale2(ff a, float c) { return {a.hi * c, a.lo * c}; }
__device__ __forceinline__ double acc_neg(double a) { return -a; }
__device__ __forceinline__ ff acc_neg(ff a) { return {-a.hi, -a.lo}; }
template <class Acc>
__device__ __forceinline__ Acc acc_make(float hi, float lo, double d);
template <>
__device__ __forceinline__ double acc_make<double>(float, float, double d) { return d; }
template <>
__device__ __forceinline__ ff acc_make<ff>(float hi, float lo, double) { return {hi, lo}; }
__device__ __forceinline__ bool acc_finite(double a) { return isfinite(a); }
__device__ __forceinline__ bool acc_finite(ff a) { return isfinite(a.hi) && isfinite(a.lo); }

__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return sqrt(x); }
__device__ __forceinline__ float rcp_r(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_r(double x) { return 1.0 / x; }
__device__ __forceinline__ float abs_r(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_r(double x) { return fabs(x); }
__device__ __forceinline__ float max_r(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double max_r(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float exp_r(float x) { return __expf(x); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }
__device__ __forceinline__ float sin_r(float x) { return sinf(x); }
__device__ __forceinline__ double sin_r(double x) { return sin(x); }
__device__ __forceinline__ float cos_r(float x) { return cosf(x); }
__device__ __forceinline__ double cos_r(double x) { return cos(x); }
// H^{4/3} as H * cbrt(H)
__device__ __forceinline__ float pow43_r(float h) { return h * cbrtf(h); }
__device__ __forceinline__ double pow43_r(double h) { return h * cbrt(h); }

// FP32 path: single hardware (MUFU) instructions of the PTX ISA -- approximate to a few ulp,
// deterministic, flushing subnormals to zero.  Every argument they get is a depth >= H0 > 0, a
// wave speed, an edge length, a squared speed above 1e-30 or a bounded exponent, far from the
// subnormal range.  FP64 path: correctly rounded operations.
__device__ __forceinline__ float mufu_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_rsqrt(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_lg2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float mufu_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float frcp(float x) { return mufu_rcp(x); }
__device__ __forceinline__ double frcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float fdiv(float a, float b) { return a * mufu_rcp(b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float fsqrt_pos(float x) { return x * mufu_rsqrt(x); }  // x > 0
__device__ __forceinline__ double fsqrt_pos(double x) { return sqrt(x); }
// sqrt(x) for x >= 0 (a squared speed): zero below 1e-30, where the friction is negligible
__device__ __forceinline__ float fsqrt0(float x) { return x > 1e-30f ? x * mufu_rsqrt(x) : 0.f; }
__device__ __forceinline__ double fsqrt0(double x) { return sqrt(x); }
// H^{-4/3} = 2^(-4/3 log2 H)
__device__ __forceinline__ float fpowm43(float h) { return mufu_ex2(-1.3333333f * mufu_lg2(h)); }
__device__ __forceinline__ double fpowm43(double h) { return 1.0 / (h * cbrt(h)); }
// e^x = 2^(x log2 e)
__device__ __forceinline__ float fexp(float x) { return mufu_ex2(x * 1.4426950408889634f); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ float fsin(float x) { return __sinf(x); }
__device__ __forceinline__ double fsin(double x) { return sin(x); }

// tidal elevation A sin(2 pi t / T + phi) of segment k at time t.  Mixed path: the phase is
// formed and reduced to [-1/2, 1/2] turns in FP64 (ocean edges are few), the sine is the
// accurate FP32 sinpi of the reduced phase; the FP64 path evaluates it in FP64.
template <class T>
__device__ __forceinline__ T tide_at(const ScenDev& S, int k, double t);
template <>
__device__ __forceinline__ float tide_at<float>(const ScenDev& S, int k, double t) {
  const double u = fma(t, S.d.tide[k][1], S.d.tide[k][2]) * 0.15915494309189535;  // turns
  const float r = (float)(u - rint(u));
  return S.f.tide[k][0] * sinpif(2.0f * r);
}
template <>
__device__ __forceinline__ double tide_at<double>(const ScenDev& S, int k, double t) {
  return S.d.tide[k][0] * sin(S.d.tide[k][1] * t + S.d.tide[k][2]);
}

// river discharge (m^2/s into the domain) of segment k at time t: linear between records, held
// at both ends (Eq. river_bc)
template <class T>
__device__ __forceinline__ T river_at(const ScenDev& S, int k, double t) {
  if (k >= S.rnseg) return T(0);
  const double* q = S.river;
  if (S.rnt == 1) return (T)q[k];
  const double f = (t - S.rt0) * S.ridt;
  if (f <= 0.0) return (T)q[k];
  if (f >= (double)(S.rnt - 1)) return (T)q[(size_t)(S.rnt - 1) * S.rnseg + k];
  const int i = (int)floor(f);
  const double w = f - (double)i;
  return (T)((1.0 - w) * q[(size_t)i * S.rnseg + k] + w * q[(size_t)(i + 1) * S.rnseg + k]);
}

template <class T>
__device__ __forceinline__ const ForcingT<T>& forcing(const ScenDev& S);
template <>
__device__ __forceinline__ const ForcingT<float>& forcing<float>(const ScenDev& S) { return S.f; }
template <>
__device__ __forceinline__ const ForcingT<double>& forcing<double>(const ScenDev& S) { return S.d; }

// -------------------------------------------------------------------- precision policy ---
struct Mixed {
  using T = float;
  using Acc = ff;
  template <int P>
  static constexpr int RV = rec_vec_mixed(P);
  static constexpr int GV = 3;  // static geometry record, 16-byte units
};
struct Fp64 {
  using T = double;
  using Acc = double;
  template <int P>
  static constexpr int RV = rec_vec_fp64(P);
  static constexpr int GV = 5;
};

template <int P, class Pol>
struct Elem {
  static constexpr int NP = np_of(P);
  using T = typename Pol::T;
  using Acc = typename Pol::Acc;
  Acc zb, xb, yb;          // element means
  T zs[NP - 1], xs[NP - 1], ys[NP - 1];  // modal coefficients 1..NP-1
  T Hb;                    // mean depth
  T hb1, hb2;              // bathymetry modes 1, 2
  uint32_t flags;
};

template <int NV>
struct Raw {
  uint4 v[NV];
};

// Element records in device memory are tile-blocked: the 16-byte vector v of element e sits at
// index ((e / 32) NV + v) 32 + e % 32.  The 32 elements of a tile read vector v as 512 contiguous
// bytes, a tile's records form one contiguous block of NV x 32 vectors, and that block copied to
// shared memory keeps the vector-major order, in which a warp's 16-byte reads spread over the banks.
template <int NV>
__host__ __device__ __forceinline__ long long rec_at(long long e, int v) {
  return ((e >> 5) * NV + v) * 32 + (e & 31);
}
template <int NV>
__device__ __forceinline__ void load_raw(const uint4* __restrict__ base, long long e, Raw<NV>& r) {
#pragma unroll
  for (int i = 0; i < NV; ++i) r.v[i] = __ldg(base + rec_at<NV>(e, i));
}
template <int NV>
__device__ __forceinline__ void store_raw(uint4* __restrict__ base, long long e, const Raw<NV>& r) {
#pragma unroll
  for (int i = 0; i < NV; ++i) base[rec_at<NV>(e, i)] = r.v[i];
}

template <int P>
__device__ __forceinline__ void unpack(const Raw<Mixed::RV<P>>& r, Elem<P, Mixed>& E) {
  constexpr int NP = np_of(P), NS = NP - 1;
  float f[4 * Mixed::RV<P>];
#pragma unroll
  for (int i = 0; i < Mixed::RV<P>; ++i) {
    f[4 * i] = __uint_as_float(r.v[i].x);
    f[4 * i + 1] = __uint_as_float(r.v[i].y);
    f[4 * i + 2] = __uint_as_float(r.v[i].z);
    f[4 * i + 3] = __uint_as_float(r.v[i].w);
  }
  E.zb = {f[0], f[1]};
  E.xb = {f[2], f[3]};
  E.yb = {f[4], f[5]};
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    E.zs[m] = f[6 + m];
    E.xs[m] = f[6 + NS + m];
    E.ys[m] = f[6 + 2 * NS + m];
  }
  constexpr int o = 6 + 3 * NS;
  E.Hb = f[o];
  E.flags = __float_as_uint(f[o + 1]);
  E.hb1 = f[o + 2];
  E.hb2 = f[o + 3];
}
template <int P>
__device__ __forceinline__ void pack(const Elem<P, Mixed>& E, Raw<Mixed::RV<P>>& r) {
  constexpr int NP = np_of(P), NS = NP - 1;
  float f[4 * Mixed::RV<P>];
#pragma unroll
  for (int i = 0; i < 4 * Mixed::RV<P>; ++i) f[i] = 0.f;
  f[0] = E.zb.hi; f[1] = E.zb.lo; f[2] = E.xb.hi; f[3] = E.xb.lo; f[4] = E.yb.hi; f[5] = E.yb.lo;
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    f[6 + m] = E.zs[m];
    f[6 + NS + m] = E.xs[m];
    f[6 + 2 * NS + m] = E.ys[m];
  }
  constexpr int o = 6 + 3 * NS;
  f[o] = E.Hb;
  f[o + 1] = __uint_as_float(E.flags);
  f[o + 2] = E.hb1;
  f[o + 3] = E.hb2;
#pragma unroll
  for (int i = 0; i < Mixed::RV<P>; ++i)
    r.v[i] = make_uint4(__float_as_uint(f[4 * i]), __float_as_uint(f[4 * i + 1]), __float_as_uint(f[4 * i + 2]),
                        __float_as_uint(f[4 * i + 3]));
}

__device__ __forceinline__ double u2d(unsigned lo, unsigned hi) {
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ void d2u(double d, unsigned& lo, unsigned& hi) {
  lo = (unsigned)__double2loint(d);
  hi = (unsigned)__double2hiint(d);
}

template <int P>
__device__ __forceinline__ void unpack(const Raw<Fp64::RV<P>>& r, Elem<P, Fp64>& E) {
  constexpr int NP = np_of(P), NS = NP - 1;
  double f[2 * Fp64::RV<P>];
#pragma unroll
  for (int i = 0; i < Fp64::RV<P>; ++i) {
    f[2 * i] = u2d(r.v[i].x, r.v[i].y);
    f[2 * i + 1] = u2d(r.v[i].z, r.v[i].w);
  }
  E.zb = f[0];
  E.xb = f[1];
  E.yb = f[2];
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    E.zs[m] = f[3 + m];
    E.xs[m] = f[3 + NS + m];
    E.ys[m] = f[3 + 2 * NS + m];
  }
  constexpr int o = 3 + 3 * NS;
  E.Hb = f[o];
  E.flags = (uint32_t)__double2loint(f[o + 1]);
  E.hb1 = f[o + 2];
  E.hb2 = f[o + 3];
}
template <int P>
__device__ __forceinline__ void pack(const Elem<P, Fp64>& E, Raw<Fp64::RV<P>>& r) {
  constexpr int NP = np_of(P), NS = NP - 1;
  double f[2 * Fp64::RV<P>];
#pragma unroll
  for (int i = 0; i < 2 * Fp64::RV<P>; ++i) f[i] = 0.0;
  f[0] = E.zb; f[1] = E.xb; f[2] = E.yb;
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    f[3 + m] = E.zs[m];
    f[3 + NS + m] = E.xs[m];
    f[3 + 2 * NS + m] = E.ys[m];
  }
  constexpr int o = 3 + 3 * NS;
  f[o] = E.Hb;
  f[o + 1] = __hiloint2double(0, (int)E.flags);
  f[o + 2] = E.hb1;
  f[o + 3] = E.hb2;
#pragma unroll
  for (int i = 0; i < Fp64::RV<P>; ++i) {
    d2u(f[2 * i], r.v[i].x, r.v[i].y);
    d2u(f[2 * i + 1], r.v[i].z, r.v[i].w);
  }
}

// static per-element geometry: scaled outward normals of the three local edges, mean
// bathymetry, area and inverse area, Manning n
template <class Pol>
struct Geo {
  using T = typename Pol::T;
  using Acc = typename Pol::Acc;
  T lnx[3], lny[3];
  Acc hbm, A, invA;
  T man;
};
__device__ __forceinline__ void load_geo(const uint4* __restrict__ g, long long e, const int4& nb, Geo<Mixed>& G) {
  uint4 a = __ldg(g + 3 * e), b = __ldg(g + 3 * e + 1), c = __ldg(g + 3 * e + 2);
  G.lnx[0] = __uint_as_float(a.x); G.lny[0] = __uint_as_float(a.y);
  G.lnx[1] = __uint_as_float(a.z); G.lny[1] = __uint_as_float(a.w);
  G.lnx[2] = __uint_as_float(b.x); G.lny[2] = __uint_as_float(b.y);
  G.hbm = {__uint_as_float(b.z), __uint_as_float(b.w)};
  G.A = {__uint_as_float(c.x), __uint_as_float(c.y)};
  G.invA = {__uint_as_float(c.z), __uint_as_float(c.w)};
  G.man = __int_as_float(nb.w);
}
__device__ __forceinline__ void load_geo(const uint4* __restrict__ g, long long e, const int4&, Geo<Fp64>& G) {
  uint4 v[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) v[i] = __ldg(g + 5 * e + i);
  G.lnx[0] = u2d(v[0].x, v[0].y); G.lny[0] = u2d(v[0].z, v[0].w);
  G.lnx[1] = u2d(v[1].x, v[1].y); G.lny[1] = u2d(v[1].z, v[1].w);
  G.lnx[2] = u2d(v[2].x, v[2].y); G.lny[2] = u2d(v[2].z, v[2].w);
  G.hbm = u2d(v[3].x, v[3].y);
  G.A = u2d(v[3].z, v[3].w);
  G.invA = u2d(v[4].x, v[4].y);
  G.man = u2d(v[4].z, v[4].w);
}

// reference tables per degree (index P): FP32 copy for the mixed path, FP64 for the FP64 path
// and for the depth test near H0.  Uploaded once per device by upload_tables().
static __constant__ RefTab<float> c_tab_f[3];
static __constant__ RefTab<double> c_tab_d[3];

template <class T, int P>
__device__ __forceinline__ const RefTab<T>& ctab();
template <>
__device__ __forceinline__ const RefTab<float>& ctab<float, 1>() { return c_tab_f[1]; }
template <>
__device__ __forceinline__ const RefTab<float>& ctab<float, 2>() { return c_tab_f[2]; }
template <>
__device__ __forceinline__ const RefTab<double>& ctab<double, 1>() { return c_tab_d[1]; }
template <>
__device__ __forceinline__ const RefTab<double>& ctab<double, 2>() { return c_tab_d[2]; }

// trace of an element at one point: d = zeta - mean(zeta), depth, discharge
template <class T>
struct Trace {
  T d, H, qx, qy;
};

template <int P, class Pol>
__device__ __forceinline__ Trace<typename Pol::T> trace_at(const Elem<P, Pol>& E, const typename Pol::T* phi) {
  using T = typename Pol::T;
  constexpr int NS = np_of(P) - 1;
  Trace<T> t;
  T d = 0, qx = acc_r(E.xb), qy = acc_r(E.yb);
#pragma unroll
  for (int m = 0; m < NS; ++m) {
    d = fma(E.zs[m], phi[m + 1], d);
    qx = fma(E.xs[m], phi[m + 1], qx);
    qy = fma(E.ys[m], phi[m + 1], qy);
  }
  T hdev = fma(E.hb1, phi[1], E.hb2 * phi[2]);
  t.d = d;
  t.H = E.Hb + (d + hdev);
  t.qx = qx;
  t.qy = qy;
  return t;
}

// trace of a degree-1 element at a point with basis values phi_1, phi_2 (as trace_at)
template <class Pol>
__device__ __forceinline__ Trace<typename Pol::T> trace_p1(const Elem<1, Pol>& E, typename Pol::T p1,
                                                            typename Pol::T p2) {
  using T = typename Pol::T;
  Trace<T> t;
  t.d = fma(E.zs[1], p2, E.zs[0] * p1);
  t.qx = fma(E.xs[1], p2, fma(E.xs[0], p1, acc_r(E.xb)));
  t.qy = fma(E.ys[1], p2, fma(E.ys[0], p1, acc_r(E.yb)));
  t.H = E.Hb + (t.d + fma(E.hb1, p1, E.hb2 * p2));
  return t;
}

// canonical flux across an edge with unit normal n from L to R; returns the mass flux and the
// advective + dissipative momentum flux (the pressure part is added per side)
template <int FLUX, class T>
__device__ __forceinline__ void edge_flux(const Trace<T>& L, const Trace<T>& R, T dcRL, T nx, T ny, T g, T H0, T& fz,
                                          T& fx, T& fy) {
  if constexpr (sizeof(T) == 4) {  // FP32: one reciprocal square root per side (as edge_flux_pair)
    const float HsL = fmaxf(L.H, H0), HsR = fmaxf(R.H, H0);
    const float rL = mufu_rsqrt(HsL), rR = mufu_rsqrt(HsR);
    const float mL = L.qx * nx + L.qy * ny, mR = R.qx * nx + R.qy * ny;
    const float unL = mL * (rL * rL), unR = mR * (rR * rR);
    const float dz = (R.d - L.d) + dcRL;
    const float dqx = R.qx - L.qx, dqy = R.qy - L.qy;
    const float cx = 0.5f * (L.qx * unL + R.qx * unR);
    const float cy = 0.5f * (L.qy * unL + R.qy * unR);
    const float cz = 0.5f * (mL + mR);
    const float sL = HsL * rL, sR = HsR * rR;
    if (FLUX == 1) {
      const float sg = fsqrt_pos(g);
      const float lam = fmaxf(fabsf(unL) + sg * sL, fabsf(unR) + sg * sR);
      fz = cz - 0.5f * lam * dz;
      fx = cx - 0.5f * lam * dqx;
      fy = cy - 0.5f * lam * dqy;
      return;
    }
    const float is = frcp(sL + sR);
    const float ut = (L.qx * rL + R.qx * rR) * is, vt = (L.qy * rL + R.qy * rR) * is;
    const float c2 = 0.5f * g * (HsL + HsR);
    const float ic = mufu_rsqrt(c2), c = c2 * ic;
    const float utn = ut * nx + vt * ny, utt = vt * nx - ut * ny;
    const float dqn = mR - mL, dqt = dqy * nx - dqx * ny;
    const float w = (dqn - utn * dz) * ic;
    const float a1 = 0.5f * (dz - w), a3 = 0.5f * (dz + w), a2 = dqt - utt * dz;
    const float l1 = fabsf(utn - c) * a1, l2 = fabsf(utn) * a2, l3 = fabsf(utn + c) * a3;
    fz = cz - 0.5f * (l1 + l3);
    fx = cx - 0.5f * (l1 * (ut - c * nx) - l2 * ny + l3 * (ut + c * nx));
    fy = cy - 0.5f * (l1 * (vt - c * ny) + l2 * nx + l3 * (vt + c * ny));
    return;
  }
  T HsL = max_r(L.H, H0), HsR = max_r(R.H, H0);
  T iL = frcp(HsL), iR = frcp(HsR);
  T uL = L.qx * iL, vL = L.qy * iL, uR = R.qx * iR, vR = R.qy * iR;
  T unL = uL * nx + vL * ny, unR = uR * nx + vR * ny;
  T mL = L.qx * nx + L.qy * ny, mR = R.qx * nx + R.qy * ny;
  T dz = (R.d - L.d) + dcRL;
  T dqx = R.qx - L.qx, dqy = R.qy - L.qy;
  T cx = T(0.5) * (L.qx * unL + R.qx * unR);
  T cy = T(0.5) * (L.qy * unL + R.qy * unR);
  T cz = T(0.5) * (mL + mR);
  if (FLUX == 1) {  // local Lax-Friedrichs
    T lam = max_r(abs_r(unL) + fsqrt_pos(g * HsL), abs_r(unR) + fsqrt_pos(g * HsR));
    fz = cz - T(0.5) * lam * dz;
    fx = cx - T(0.5) * lam * dqx;
    fy = cy - T(0.5) * lam * dqy;
    return;
  }
  // Roe: averages (arithmetic depth, sqrt-depth-weighted velocity), eigen-decomposition
  T sL = fsqrt_pos(HsL), sR = fsqrt_pos(HsR);
  T is = frcp(sL + sR);
  T ut = (sL * uL + sR * uR) * is, vt = (sL * vL + sR * vR) * is;
  T c = fsqrt_pos(g * T(0.5) * (HsL + HsR));
  T ic = frcp(c);
  T utn = ut * nx + vt * ny, utt = vt * nx - ut * ny;
  T dqn = dqx * nx + dqy * ny, dqt = dqy * nx - dqx * ny;
  T w = (dqn - utn * dz) * ic;
  T a1 = T(0.5) * (dz - w), a3 = T(0.5) * (dz + w), a2 = dqt - utt * dz;
  T l1 = abs_r(utn - c) * a1, l2 = abs_r(utn) * a2, l3 = abs_r(utn + c) * a3;
  T D0 = l1 + l3;
  T D1 = l1 * (ut - c * nx) - l2 * ny + l3 * (ut + c * nx);
  T D2 = l1 * (vt - c * ny) + l2 * nx + l3 * (vt + c * ny);
  fz = cz - T(0.5) * D0;
  fx = cx - T(0.5) * D1;
  fy = cy - T(0.5) * D2;
}

#ifndef DG_PACKED_FLUX
#define DG_PACKED_FLUX 1  // FP32 path, p = 1: both Gauss points of an edge in packed FP32x2 arithmetic
#endif

// packed FP32x2 arithmetic (two edge points per instruction)
using f2 = float2;
__device__ __forceinline__ f2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ f2 add2(f2 a, f2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ f2 neg2(f2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ f2 sub2(f2 a, f2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ f2 mul2(f2 a, f2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ f2 max2(f2 a, f2 b) { return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y)); }
__device__ __forceinline__ f2 abs2(f2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ f2 rcp2(f2 a) { return make_float2(frcp(a.x), frcp(a.y)); }
__device__ __forceinline__ f2 sqrt2(f2 a) { return make_float2(fsqrt_pos(a.x), fsqrt_pos(a.y)); }
__device__ __forceinline__ f2 rsqrt2(f2 a) { return make_float2(mufu_rsqrt(a.x), mufu_rsqrt(a.y)); }  // a > 0
struct Trace2 {
  f2 d, H, qx, qy;  // two edge points
};

// edge_flux for two points at once (FP32), written with packed operations and one reciprocal
// square root per side: with r = 1/sqrt(Hs), 1/Hs = r^2, sqrt(Hs) = Hs r, the Roe velocity is
// (q_L r_L + q_R r_R) / (sqrt(Hs_L) + sqrt(Hs_R)), u.n = (q.n)/Hs, and the jump of q.n is the
// difference of the sides' q.n (the same quantities as edge_flux, fewer operations)
// per-side quantities of edge_flux_pair that the wall flux of a closed edge reuses: q.n, 1/Hs and
// sqrt(Hs) of both sides
struct FluxAux2 {
  f2 mL, mR, iL, iR, sL, sR;
};
template <int FLUX>
__device__ __forceinline__ void edge_flux_pair(const Trace2& L, const Trace2& R, f2 dcRL, f2 nx, f2 ny, float g,
                                               float H0, f2& fz, f2& fx, f2& fy, FluxAux2& ax) {
  const f2 half = p2(0.5f), mhalf = p2(-0.5f);
  const f2 HsL = max2(L.H, p2(H0)), HsR = max2(R.H, p2(H0));
  const f2 rL = rsqrt2(HsL), rR = rsqrt2(HsR);
  const f2 iL = mul2(rL, rL), iR = mul2(rR, rR);
  const f2 mL = fma2(L.qx, nx, mul2(L.qy, ny)), mR = fma2(R.qx, nx, mul2(R.qy, ny));
  const f2 unL = mul2(mL, iL), unR = mul2(mR, iR);
  const f2 dz = add2(sub2(R.d, L.d), dcRL);
  const f2 dqx = sub2(R.qx, L.qx), dqy = sub2(R.qy, L.qy);
  const f2 cx = mul2(half, fma2(L.qx, unL, mul2(R.qx, unR)));
  const f2 cy = mul2(half, fma2(L.qy, unL, mul2(R.qy, unR)));
  const f2 cz = mul2(half, add2(mL, mR));
  const f2 sL = mul2(HsL, rL), sR = mul2(HsR, rR);
  ax = {mL, mR, iL, iR, sL, sR};
  if (FLUX == 1) {  // local Lax-Friedrichs: sqrt(g Hs) = sqrt(g) sqrt(Hs)
    const f2 sg = p2(fsqrt_pos(g));
    const f2 lam = max2(fma2(sg, sL, abs2(unL)), fma2(sg, sR, abs2(unR)));
    const f2 hl = mul2(mhalf, lam);
    fz = fma2(hl, dz, cz);
    fx = fma2(hl, dqx, cx);
    fy = fma2(hl, dqy, cy);
    return;
  }
  // Roe: averages (arithmetic depth, sqrt-depth-weighted velocity), eigen-decomposition
  const f2 is = rcp2(add2(sL, sR));
  const f2 ut = mul2(fma2(L.qx, rL, mul2(R.qx, rR)), is), vt = mul2(fma2(L.qy, rL, mul2(R.qy, rR)), is);
  const f2 c2 = mul2(p2(0.5f * g), add2(HsL, HsR));
  const f2 ic = rsqrt2(c2), c = mul2(c2, ic);
  const f2 utn = fma2(ut, nx, mul2(vt, ny)), utt = fma2(vt, nx, mul2(neg2(ut), ny));
  const f2 dqn = sub2(mR, mL), dqt = fma2(dqy, nx, mul2(neg2(dqx), ny));
  const f2 w = mul2(fma2(neg2(utn), dz, dqn), ic);
  const f2 a1 = mul2(half, sub2(dz, w)), a3 = mul2(half, add2(dz, w)), a2 = fma2(neg2(utt), dz, dqt);
  const f2 l1 = mul2(abs2(sub2(utn, c)), a1), l2 = mul2(abs2(utn), a2), l3 = mul2(abs2(add2(utn, c)), a3);
  const f2 D0 = add2(l1, l3);
  const f2 D1 = fma2(l1, fma2(neg2(c), nx, ut), fma2(neg2(l2), ny, mul2(l3, fma2(c, nx, ut))));
  const f2 D2 = fma2(l1, fma2(neg2(c), ny, vt), fma2(l2, nx, mul2(l3, fma2(c, ny, vt))));
  fz = fma2(mhalf, D0, cz);
  fx = fma2(mhalf, D1, cx);
  fy = fma2(mhalf, D2, cy);
}

// pressure difference P - P_c with P_c the pressure at the reference elevation c:
// g/2 (zeta - c)(zeta + c + 2 hb) = g/2 d (2 H - d)
template <class T>
__device__ __forceinline__ T pdev(T d, T H, T g) {
  return T(0.5) * g * d * (T(2) * H - d);
}

// FP64 positive-depth operator on the linear part (Sec. 2.4).  zs/xs/ys are modes 1.. of
// zeta/qx/qy (double, in place); zbar/xbar/ybar means; returns true if the element is dry.
// At p = 2 the operator acts on the linear part and the quadratic modes are scaled by
// clamp((Hmin - H0) / H0, 0, 1), Hmin the linear part's smallest vertex depth (continuous in
// the state: untouched from 2 H0 up, removed at H0 and below).
template <int P>
__device__ bool positivity_fp64(double zbar, double& xbar, double& ybar, double* zs, double* xs, double* ys,
                                const double hbv[3], double H0, const RefTab<double>& tb, bool& changed) {
  constexpr int NP = np_of(P), NS = NP - 1;
  constexpr int NL = NS < 2 ? NS : 2;  // linear modes among zs
  double H[3];
  changed = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double z = zbar;
#pragma unroll
    for (int m = 0; m < NL; ++m) z = fma(zs[m], tb.vphi[i][m + 1], z);
    H[i] = z + hbv[i];
  }
  if (P >= 2) {
    const double hmin = fmin(fmin(H[0], H[1]), H[2]);
    double th = (hmin - H0) / H0;
    th = th < 0.0 ? 0.0 : th;
    if (th < 1.0) {
#pragma unroll
      for (int m = 2; m < NS; ++m) {
        zs[m] *= th;
        xs[m] *= th;
        ys[m] *= th;
      }
      changed = true;
    }
  }
  if (H[0] >= H0 && H[1] >= H0 && H[2] >= H0) return false;
  changed = true;
  double Hbar = (H[0] + H[1] + H[2]) / 3.0;
  double Ho[3];
  bool dry[3];
  if (Hbar <= H0) {
    Ho[0] = Ho[1] = Ho[2] = Hbar;
    dry[0] = dry[1] = dry[2] = true;
  } else {
    // rank of each vertex in the stable order of the three depths (ties by vertex index): lowest
    // 0, middle 1, highest 2; formed by comparisons, so no array is indexed at run time
    int rk[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      rk[i] = 0;
#pragma unroll
      for (int j = 0; j < 3; ++j)
        if (j != i && (H[j] < H[i] || (H[j] == H[i] && j < i))) ++rk[i];
    }
    double hl = H[0], hm = H[0];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (rk[i] == 0) hl = H[i];
      if (rk[i] == 1) hm = H[i];
    }
    const double d = H0 - hl;
    const bool share = hm - 0.5 * d >= H0;  // the other two vertices give up d/2 each
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      if (rk[i] == 0) Ho[i] = H0;
      else if (share) Ho[i] = H[i] - 0.5 * d;
      else Ho[i] = (rk[i] == 1) ? H0 : H[i] - (H0 - hl) - (H0 - hm);
      dry[i] = Ho[i] < H0;
    }
  }
  // rebuild the linear part of zeta from the redistributed vertex values; the mean is kept
  double zv[3] = {Ho[0] - hbv[0], Ho[1] - hbv[1], Ho[2] - hbv[2]};
  if (NS >= 2) {
    zs[0] = tb.vinv[0][0] * zv[0] + tb.vinv[0][1] * zv[1] + tb.vinv[0][2] * zv[2];
    zs[1] = tb.vinv[1][0] * zv[0] + tb.vinv[1][1] * zv[1] + tb.vinv[1][2] * zv[2];
  }
  int nd = (int)dry[0] + (int)dry[1] + (int)dry[2];
  if (nd == 3) {
    xbar = ybar = 0.0;
#pragma unroll
    for (int m = 0; m < NS; ++m) xs[m] = ys[m] = 0.0;
  } else if (nd > 0 && NS >= 2) {
    double qx[3], qy[3], sx = 0.0, sy = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      qx[i] = xbar + xs[0] * tb.vphi[i][1] + xs[1] * tb.vphi[i][2];
      qy[i] = ybar + ys[0] * tb.vphi[i][1] + ys[1] * tb.vphi[i][2];
      if (dry[i]) { sx += qx[i]; sy += qy[i]; qx[i] = qy[i] = 0.0; }
    }
    const double share = (nd == 1) ? 0.5 : 1.0;  // 1 / (3 - nd), exact
#pragma unroll
    for (int i = 0; i < 3; ++i)
      if (!dry[i]) { qx[i] += sx * share; qy[i] += sy * share; }
    xs[0] = tb.vinv[0][0] * qx[0] + tb.vinv[0][1] * qx[1] + tb.vinv[0][2] * qx[2];
    xs[1] = tb.vinv[1][0] * qx[0] + tb.vinv[1][1] * qx[1] + tb.vinv[1][2] * qx[2];
    ys[0] = tb.vinv[0][0] * qy[0] + tb.vinv[0][1] * qy[1] + tb.vinv[0][2] * qy[2];
    ys[1] = tb.vinv[1][0] * qy[0] + tb.vinv[1][1] * qy[1] + tb.vinv[1][2] * qy[2];
  }
  return nd > 0;
}

// positive-depth operator on a freshly combined element; sets E.Hb and the dry flag.
// FP32 path: the linear part's vertex depths are first bounded in FP32; an element clearly
// above H0 at every vertex is case 1 (unchanged, wet; at p = 2 its quadratic modes are scaled
// by the continuous blend factor when the shallowest vertex is below 2 H0), one whose mean
// depth is clearly below H0 with a vertex clearly below H0 is case 2 (flat depth, dry, no
// momentum: the zeta slopes become minus the bathymetry slopes), and one with a vertex below H0
// but a mean depth clearly above it is case 3 (depth moved to the lowest vertex, wet).  The wet /
// dry decision is thereby the FP64 one: FP32 decides only outside a band wider than the FP32
// evaluation error, and elements inside it (and near ties of case 3) take the FP64 operator; for
// a wet mean, a vertex within that band of H0 only decides a redistribution below the FP32
// resolution of the vertex depths, which FP32 makes.
template <int P, class Pol>
__device__ __forceinline__ void apply_positivity(Elem<P, Pol>& E, const Geo<Pol>& G, long long e,
                                                 const StageArgs<Pol>& a, int* err) {
  using T = typename Pol::T;
  constexpr int NS = np_of(P) - 1;
  const RefTab<T>& tab = ctab<T, P>();
  const T H0 = a.H0;
  const T Hb = acc_sum_r(E.zb, G.hbm);  // mean depth
  constexpr int NL = NS < 2 ? NS : 2;  // linear modes among zs
  bool need64 = true, dry = false;
  if (sizeof(T) == 4) {
    T hv[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T v = Hb;
#pragma unroll
      for (int m = 0; m < NL; ++m) v = fma(E.zs[m], tab.vphi[i][m + 1], v);
      v = fma(E.hb1, tab.vphi[i][1], v);
      hv[i] = fma(E.hb2, tab.vphi[i][2], v);
    }
    // bound on the magnitudes summed at any vertex: |Hb| + sum_m (|zs_m| + |hb_m|) max_i |phi_m(x_i)|
    T bound = (abs_r(E.hb1) + abs_r(E.zs[0])) * tab.vabs[1];
    if (NL > 1) bound = fma(abs_r(E.hb2) + abs_r(E.zs[NL > 1 ? 1 : 0]), tab.vabs[2], bound);
    const T hmin = fminf(hv[0], fminf(hv[1], hv[2]));
    const T tol = T(4.0e-6) * (abs_r(Hb) + bound);
    // mean depth clearly above H0: the element is wet whatever its vertices; a vertex depth within
    // tol of H0 then decides only whether a redistribution smaller than tol (below the FP32
    // resolution of the vertex depths) is made, and FP32 decides it
    const bool wet_mean = Hb > H0 * T(1.00001);
    if (hmin - tol > H0 || (wet_mean && hmin >= H0)) {
      need64 = false;  // case 1
      if (P >= 2 && hmin < T(2) * H0) {  // quadratic modes blended out, continuous in hmin
        const T th = (hmin - H0) * frcp(H0);
#pragma unroll
        for (int m = 2; m < NS; ++m) {
          E.zs[m] *= th;
          E.xs[m] *= th;
          E.ys[m] *= th;
        }
      }
    } else if (Hb < H0 * T(0.99999) && hmin + tol < H0 && Hb >= T(0)) {
      need64 = false;  // case 2
      dry = true;
      E.zs[0] = -E.hb1;
      E.zs[1] = -E.hb2;
#pragma unroll
      for (int m = 2; m < NS; ++m) E.zs[m] = T(0);
#pragma unroll
      for (int m = 0; m < NS; ++m) E.xs[m] = E.ys[m] = T(0);
      E.xb = acc_make<typename Pol::Acc>(0.f, 0.f, 0.0);
      E.yb = acc_make<typename Pol::Acc>(0.f, 0.f, 0.0);
    } else if (wet_mean) {
      // case 3, partially wet: the lowest vertex is raised to H0 and the deficit taken from the
      // others (M Pi^d); no vertex ends dry, so the momentum is unchanged (M Pi^f) and the element
      // is wet.  Formed as vertex changes dH_i (summing to zero: the mean is kept) and added to the
      // slope modes through the vertex-to-mode map, so the bathymetry cancels and FP32 keeps the
      // precision of the small depths.  A near tie of the two upper vertices (where the operator
      // depends on their order) is left to the FP64 operator.
      const T h0 = hmin, h2 = fmaxf(hv[0], fmaxf(hv[1], hv[2]));
      const T h1 = fmaxf(fminf(hv[0], hv[1]), fminf(fmaxf(hv[0], hv[1]), hv[2]));  // median
      const T d = H0 - h0;
      const bool split = h1 - T(0.5) * d >= H0;  // the other two vertices share the deficit
      if (split || h2 - h1 > tol) {
        need64 = false;
        const T e = H0 - h1;
        T dh[3];
#pragma unroll
        for (int i = 0; i < 3; ++i)
          dh[i] = (hv[i] == h0) ? d : (split ? T(-0.5) * d : (hv[i] == h2 ? -(d + e) : e));
#pragma unroll
        for (int m = 0; m < NL; ++m)
          E.zs[m] += tab.vinv[m][0] * dh[0] + tab.vinv[m][1] * dh[1] + tab.vinv[m][2] * dh[2];
#pragma unroll
        for (int m = 2; m < NS; ++m) {  // p = 2: the blend factor is zero below H0
          E.zs[m] = T(0);
          E.xs[m] = T(0);
          E.ys[m] = T(0);
        }
      }
    }
  }
  if (need64) {
    double zs[NS], xs[NS], ys[NS];
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      zs[m] = (double)E.zs[m];
      xs[m] = (double)E.xs[m];
      ys[m] = (double)E.ys[m];
    }
    const int4 nd = __ldg(a.nodes + e);
    double hbv[3] = {a.hb_nodal[nd.x], a.hb_nodal[nd.y], a.hb_nodal[nd.z]};
    double xb = acc_d(E.xb), yb = acc_d(E.yb);
    bool changed;
    dry = positivity_fp64<P>(acc_d(E.zb), xb, yb, zs, xs, ys, hbv, (double)H0, c_tab_d[P], changed);
    if (changed) {
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        E.zs[m] = (T)zs[m];
        E.xs[m] = (T)xs[m];
        E.ys[m] = (T)ys[m];
      }
      if (dry) {
        acc_set(E.xb, xb);
        acc_set(E.yb, yb);
      }
    }
    if (acc_d(E.zb) + acc_d(G.hbm) < 0.0) atomicOr(err, ERR_NEGDEPTH);
  }
  E.Hb = Hb;
  E.flags = dry ? FLAG_DRY : 0u;
  if (!acc_finite(E.zb) || !acc_finite(E.xb) || !acc_finite(E.yb)) atomicOr(err, ERR_NONFINITE);
}

// --------------------------------------------------------------- block reduction helpers ---
__device__ __forceinline__ void warp_reduce2(double& a, double& b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
}
__device__ __forceinline__ ff shfl_ff(ff v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}
__device__ __forceinline__ void warp_reduce2(ff& a, ff& b) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = ff_add(a, shfl_ff(a, o));
    b = ff_add(b, shfl_ff(b, o));
  }
}

// ------------------------------------------------------------------ edge-split path ----
template <class Pol>
struct SlotT;
template <>
struct SlotT<Mixed> {
  template <int P>
  static constexpr int SV = slot_vec_mixed(P);
};
template <>
struct SlotT<Fp64> {
  template <int P>
  static constexpr int SV = slot_vec_fp64(P);
};

// lift values of one side: zeta modes 1..NS, qx modes 0..NS, qy modes 0..NS, then mass, flag
template <int P, class T>
struct Lift {
  static constexpr int NP = np_of(P), NV = slot_vals(P);
  T v[NV];
  T mass;
  uint32_t flag;
};

template <int P>
__device__ __forceinline__ void store_slot(uint4* __restrict__ slots, long long idx, const Lift<P, float>& L) {
  constexpr int SV = slot_vec_mixed(P), NV = slot_vals(P);
  float f[4 * SV];
#pragma unroll
  for (int i = 0; i < 4 * SV; ++i) f[i] = 0.f;
#pragma unroll
  for (int i = 0; i < NV; ++i) f[i] = L.v[i];
  f[NV] = L.mass;
  f[NV + 1] = __uint_as_float(L.flag);
  uint4* p = slots + idx * SV;
#pragma unroll
  for (int i = 0; i < SV; ++i)
    p[i] = make_uint4(__float_as_uint(f[4 * i]), __float_as_uint(f[4 * i + 1]), __float_as_uint(f[4 * i + 2]),
                      __float_as_uint(f[4 * i + 3]));
}
template <int P>
__device__ __forceinline__ void load_slot(const uint4* __restrict__ slots, long long idx, Lift<P, float>& L) {
  constexpr int SV = slot_vec_mixed(P), NV = slot_vals(P);
  float f[4 * SV];
  const uint4* p = slots + idx * SV;
#pragma unroll
  for (int i = 0; i < SV; ++i) {
    const uint4 u = __ldg(p + i);
    f[4 * i] = __uint_as_float(u.x);
    f[4 * i + 1] = __uint_as_float(u.y);
    f[4 * i + 2] = __uint_as_float(u.z);
    f[4 * i + 3] = __uint_as_float(u.w);
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) L.v[i] = f[i];
  L.mass = f[NV];
  L.flag = __float_as_uint(f[NV + 1]);
}
template <int P>
__device__ __forceinline__ void store_slot(uint4* __restrict__ slots, long long idx, const Lift<P, double>& L) {
  constexpr int SV = slot_vec_fp64(P), NV = slot_vals(P);
  double f[2 * SV];
#pragma unroll
  for (int i = 0; i < 2 * SV; ++i) f[i] = 0.0;
#pragma unroll
  for (int i = 0; i < NV; ++i) f[i] = L.v[i];
  f[NV] = L.mass;
  f[NV + 1] = __hiloint2double(0, (int)L.flag);
  uint4* p = slots + idx * SV;
#pragma unroll
  for (int i = 0; i < SV; ++i) {
    uint4 u;
    d2u(f[2 * i], u.x, u.y);
    d2u(f[2 * i + 1], u.z, u.w);
    p[i] = u;
  }
}
template <int P>
__device__ __forceinline__ void load_slot(const uint4* __restrict__ slots, long long idx, Lift<P, double>& L) {
  constexpr int SV = slot_vec_fp64(P), NV = slot_vals(P);
  double f[2 * SV];
  const uint4* p = slots + idx * SV;
#pragma unroll
  for (int i = 0; i < SV; ++i) {
    const uint4 u = __ldg(p + i);
    f[2 * i] = u2d(u.x, u.y);
    f[2 * i + 1] = u2d(u.z, u.w);
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) L.v[i] = f[i];
  L.mass = f[NV];
  L.flag = (uint32_t)__double2loint(f[NV + 1]);
}

// slot read from staged shared memory: vector i at base[i * stride]
template <int P>
__device__ __forceinline__ void load_slot(const uint4* base, long long, Lift<P, float>& L, int stride) {
  constexpr int SV = slot_vec_mixed(P), NV = slot_vals(P);
  float f[4 * SV];
#pragma unroll
  for (int i = 0; i < SV; ++i) {
    const uint4 u = base[(size_t)i * stride];
    f[4 * i] = __uint_as_float(u.x);
    f[4 * i + 1] = __uint_as_float(u.y);
    f[4 * i + 2] = __uint_as_float(u.z);
    f[4 * i + 3] = __uint_as_float(u.w);
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) L.v[i] = f[i];
  L.mass = f[NV];
  L.flag = __float_as_uint(f[NV + 1]);
}
template <int P>
__device__ __forceinline__ void load_slot(const uint4* base, long long, Lift<P, double>& L, int stride) {
  constexpr int SV = slot_vec_fp64(P), NV = slot_vals(P);
  double f[2 * SV];
#pragma unroll
  for (int i = 0; i < SV; ++i) {
    const uint4 u = base[(size_t)i * stride];
    f[2 * i] = u2d(u.x, u.y);
    f[2 * i + 1] = u2d(u.z, u.w);
  }
#pragma unroll
  for (int i = 0; i < NV; ++i) L.v[i] = f[i];
  L.mass = f[NV];
  L.flag = (uint32_t)__double2loint(f[NV + 1]);
}

__device__ __forceinline__ void load_edge(const uint4* e, long long i, int& eL, int& jL, int& eR, int& jR, float& lnx,
                                          float& lny) {
  const uint4 u = __ldg(e + i);
  eL = (int)u.x >> 2; jL = (int)u.x & 3; eR = (int)u.y >> 2; jR = (int)u.y & 3;
  lnx = __uint_as_float(u.z);
  lny = __uint_as_float(u.w);
}
__device__ __forceinline__ void load_edge(const uint4* e, long long i, int& eL, int& jL, int& eR, int& jR,
                                          double& lnx, double& lny) {
  const uint4 u = __ldg(e + 2 * i), v = __ldg(e + 2 * i + 1);
  eL = (int)u.x >> 2; jL = (int)u.x & 3; eR = (int)u.y >> 2; jR = (int)u.y & 3;
  lnx = u2d(v.x, v.y);
  lny = u2d(v.z, v.w);
}

// Edge kernel: one thread per interior edge, in the canonical orientation (L = lower element
// index, normal outward from L).  Computes the numerical flux once, the wet/dry closure, the
// pressure relative to each side's own mean elevation, and writes both sides' lift into their
// slots (mass flux +E to L, -E to R: bitwise opposite).  A closed edge only raises the flag;
// each side then builds its own wall flux in the element kernel.
template <int P, int FLUX, class Pol>
__global__ void __launch_bounds__(256) edge_kernel(const StageArgs<Pol> a) {
  using T = typename Pol::T;
  constexpr int NP = np_of(P), NG = P + 1, RV = Pol::template RV<P>;
  const RefTab<T>& tab = ctab<T, P>();
  __shared__ T s_ephi[3][NG][NP];
  for (int i = threadIdx.x; i < 3 * NG * NP; i += blockDim.x) {
    const int j = i / (NG * NP), k = (i / NP) % NG, m = i % NP;
    s_ephi[j][k][m] = tab.ephi[j][k][m];
  }
  __syncthreads();
  const T g = a.g, H0 = a.H0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.nedges;
       i += (long long)gridDim.x * blockDim.x) {
    int eL, jL, eR, jR;
    T lnx, lny;
    load_edge(a.edges, i, eL, jL, eR, jR, lnx, lny);
    Raw<RV> rl, rr;
    load_raw<RV>(a.in, eL, rl);
    load_raw<RV>(a.in, eR, rr);
    Elem<P, Pol> L, R;
    unpack<P>(rl, L);
    unpack<P>(rr, R);
    const T len = fsqrt_pos(lnx * lnx + lny * lny);
    const T il = frcp(len);
    const T nx = lnx * il, ny = lny * il;
    const T dcRL = acc_diff(R.zb, L.zb);
    Trace<T> tl[NG], tr[NG];
    T fz[NG], fx[NG], fy[NG];
    T ecanon = 0;
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      tl[k] = trace_at<P, Pol>(L, s_ephi[jL][k]);
      tr[k] = trace_at<P, Pol>(R, s_ephi[jR][NG - 1 - k]);
      edge_flux<FLUX, T>(tl[k], tr[k], dcRL, nx, ny, g, H0, fz[k], fx[k], fy[k]);
      ecanon = fma(tab.gw[k], fz[k], ecanon);
    }
    ecanon = ecanon * (T(0.5) * len);
    const bool dryL = (L.flags & FLAG_DRY) != 0, dryR = (R.flags & FLAG_DRY) != 0;
    const bool closed = (dryL && ecanon > T(0)) || (dryR && ecanon < T(0));
    Lift<P, T> ol, orr;
#pragma unroll
    for (int v = 0; v < Lift<P, T>::NV; ++v) ol.v[v] = orr.v[v] = T(0);
    ol.flag = orr.flag = closed ? 1u : 0u;
    ol.mass = closed ? T(0) : ecanon;
    orr.mass = closed ? T(0) : -ecanon;
    if (!closed) {
      constexpr int NS = NP - 1;
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const T pl = T(0.5) * (pdev(tl[k].d, tl[k].H, g) + pdev(tr[k].d + dcRL, tr[k].H, g));
        const T pr = T(0.5) * (pdev(tr[k].d, tr[k].H, g) + pdev(tl[k].d - dcRL, tl[k].H, g));
        const T wk = tab.gw[k] * (T(0.5) * len);
        // L: flux along n_L;  R: flux along n_R = -n_L
        const T lz = fz[k], lx = fx[k] + pl * nx, ly = fy[k] + pl * ny;
        const T rz = -fz[k], rx = -(fx[k] + pr * nx), ry = -(fy[k] + pr * ny);
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const T phl = wk * s_ephi[jL][k][m], phr = wk * s_ephi[jR][NG - 1 - k][m];
          if (m > 0) {
            ol.v[m - 1] = fma(-phl, lz, ol.v[m - 1]);
            orr.v[m - 1] = fma(-phr, rz, orr.v[m - 1]);
          }
          ol.v[NS + m] = fma(-phl, lx, ol.v[NS + m]);
          ol.v[NS + NP + m] = fma(-phl, ly, ol.v[NS + NP + m]);
          orr.v[NS + m] = fma(-phr, rx, orr.v[NS + m]);
          orr.v[NS + NP + m] = fma(-phr, ry, orr.v[NS + NP + m]);
        }
      }
    }
    store_slot<P>(a.slots, 3LL * eL + jL, ol);
    store_slot<P>(a.slots, 3LL * eR + jR, orr);
  }
}

// gridded rain (mm/h records, bilinear in space, linear in time, clamped to the grid) at a
// point and time, in m/s (Sec. 2.5)
template <class T>
__device__ __forceinline__ T grid_rain(const ScenDev& S, const ForcingT<T>& F, T px, T py, T t) {
  T gx = (px - F.grid[0]) * F.grid[2], gy = (py - F.grid[1]) * F.grid[3];
  T gt = (t - F.grid[4]) * F.grid[5];
  gx = fmin(fmax(gx, T(0)), T(S.gnx - 1));
  gy = fmin(fmax(gy, T(0)), T(S.gny - 1));
  gt = fmin(fmax(gt, T(0)), T(S.gnt - 1));
  const int ix = min(max((int)floor(gx), 0), max(S.gnx - 2, 0));
  const int iy = min(max((int)floor(gy), 0), max(S.gny - 2, 0));
  const int it = min(max((int)floor(gt), 0), max(S.gnt - 2, 0));
  const T fx = gx - T(ix), fy = gy - T(iy), ft = gt - T(it);
  const int ix1 = S.gnx > 1 ? ix + 1 : ix, iy1 = S.gny > 1 ? iy + 1 : iy;
  T val[2];
#pragma unroll
  for (int qq = 0; qq < 2; ++qq) {
    const int kk = S.gnt > 1 ? it + qq : 0;
    const float* Gr = S.grid + (size_t)kk * S.gnx * S.gny;
    const T v00 = Gr[(size_t)iy * S.gnx + ix], v10 = Gr[(size_t)iy * S.gnx + ix1];
    const T v01 = Gr[(size_t)iy1 * S.gnx + ix], v11 = Gr[(size_t)iy1 * S.gnx + ix1];
    val[qq] = (T(1) - fy) * ((T(1) - fx) * v00 + fx * v10) + fy * ((T(1) - fx) * v01 + fx * v11);
  }
  return ((T(1) - ft) * val[0] + ft * val[1]) * T(1.0 / 3.6e6);
}

// node kernel: the gridded rain of every node at this stage's time, once per node instead of
// once per (element, vertex)
template <class Pol>
__global__ void __launch_bounds__(256) node_rain_kernel(const StageArgs<Pol> a, long long nn) {
  using T = typename Pol::T;
  const double stepd = (double)a.ctl->step + a.cst;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += (long long)gridDim.x * blockDim.x) {
    const ScenDev& S = a.scen[a.node_scen[n]];
    if (S.rain_kind != 3) continue;
    const ForcingT<T>& F = forcing<T>(S);
    const T t = (T)(S.d.t0 + stepd * S.d.dt);  // stage time, formed in FP64
    a.rain_node[n] = grid_rain<T>(S, F, a.node_xy[2 * n], a.node_xy[2 * n + 1], t);
  }
}

// optional slope limiter (Sec. 2.3 offers one without its form): the TVB minmod moment limiter
// of Cockburn and Shu for P1 triangles, componentwise on zeta, qx, qy of wet elements with three
// neighbours.  Edge i (vertices i, i+1): deviation d_i = w(m_i) - mean at the edge midpoint,
// neighbour estimate a_i (mean_i - mean) + c_i (mean_k - mean) with the barycentric pair
// (i, k) precomputed on the host (a_i, c_i >= 0), limited to minmod(d_i, nu estimate) unless
// |d_i| <= M h^2; positive and negative parts rebalanced to sum to zero; the slopes rebuilt from
// the midpoint deviations (vertex deviation i = l_i + l_{i-1} - l_{i+1}).  Means are untouched,
// so the update runs in place; the positive-depth operator follows.
template <class T>
__device__ __forceinline__ T minmod_r(T a, T b) {
  return (a > T(0) && b > T(0)) ? (a < b ? a : b) : ((a < T(0) && b < T(0)) ? (a > b ? a : b) : T(0));
}

template <class Pol>
__device__ __forceinline__ bool limit_var(typename Pol::T* s, const typename Pol::T dm[3], const typename Pol::T* L,
                                          int bits, typename Pol::T nu, const RefTab<typename Pol::T>& tab) {
  using T = typename Pol::T;
  T d[3], l[3];
  bool changed = false;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    d[i] = s[0] * tab.mphi[i][1] + s[1] * tab.mphi[i][2];
    const int k = (bits >> i) & 1 ? (i + 2) % 3 : (i + 1) % 3;
    const T est = L[2 * i] * dm[i] + L[2 * i + 1] * dm[k];
    l[i] = (abs_r(d[i]) <= L[6]) ? d[i] : minmod_r(d[i], nu * est);
    changed = changed || (l[i] != d[i]);
  }
  if (!changed) return false;
  const T sum = l[0] + l[1] + l[2];
  if (sum != T(0)) {
    T pos = 0, neg = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      pos += l[i] > T(0) ? l[i] : T(0);
      neg += l[i] < T(0) ? -l[i] : T(0);
    }
    const T tp = pos > T(0) ? (neg / pos < T(1) ? neg / pos : T(1)) : T(0);
    const T tn = neg > T(0) ? (pos / neg < T(1) ? pos / neg : T(1)) : T(0);
#pragma unroll
    for (int i = 0; i < 3; ++i) l[i] = tp * (l[i] > T(0) ? l[i] : T(0)) - tn * (l[i] < T(0) ? -l[i] : T(0));
  }
  T f[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) f[i] = l[i] + l[(i + 2) % 3] - l[(i + 1) % 3];
  s[0] = tab.vinv[0][0] * f[0] + tab.vinv[0][1] * f[1] + tab.vinv[0][2] * f[2];
  s[1] = tab.vinv[1][0] * f[0] + tab.vinv[1][1] * f[1] + tab.vinv[1][2] * f[2];
  return true;
}

template <class Pol>
__global__ void __launch_bounds__(256) limit_kernel(const StageArgs<Pol> a, long long ne) {
  using T = typename Pol::T;
  constexpr int RV = Pol::template RV<1>;
  const RefTab<T>& tab = ctab<T, 1>();
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x) {
    const int4 nb = __ldg(a.nbr + e);
    if (nb.x < 0 || nb.y < 0 || nb.z < 0) continue;
    const T* L = a.lim + 8 * e;
    const int bits = (int)L[7];
    if (bits < 0) continue;
    Raw<RV> r;
    load_raw<RV>(a.out, e, r);
    Elem<1, Pol> E;
    unpack<1>(r, E);
    if (E.flags & FLAG_DRY) continue;
    T dz[3], dx[3], dy[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int code = (j == 0) ? nb.x : (j == 1 ? nb.y : nb.z);
      Raw<RV> rn;
      load_raw<RV>(a.out, (long long)(code >> 2), rn);
      Elem<1, Pol> N;
      unpack<1>(rn, N);
      dz[j] = acc_diff(N.zb, E.zb);
      dx[j] = acc_diff(N.xb, E.xb);
      dy[j] = acc_diff(N.yb, E.yb);
    }
    bool ch = limit_var<Pol>(E.zs, dz, L, bits, a.lim_nu, tab);
    ch = limit_var<Pol>(E.xs, dx, L, bits, a.lim_nu, tab) || ch;
    ch = limit_var<Pol>(E.ys, dy, L, bits, a.lim_nu, tab) || ch;
    if (!ch) continue;
    Geo<Pol> G;
    load_geo(a.geo, e, nb, G);
    apply_positivity<1, Pol>(E, G, e, a, &a.ctl->err);
    Raw<RV> ro;
    pack<1>(E, ro);
    store_raw<RV>(a.out, e, ro);
  }
}

// ------------------------------------------------------------------------ stage kernel ----
// Work split: 32-element tiles, warp w of the launch takes tiles w, w + W, w + 2W, ... (W warps
// in the grid).  No block-wide barrier inside the loop; rain and boundary volumes accumulate per
// lane and are reduced per warp when the warp moves to another scenario and at the end, into
// ledger slot (scenario, warp): deterministic for a fixed launch shape.
template <int P, class Pol>
__device__ __forceinline__ void flush_ledger(const StageArgs<Pol>& a, int sc, long long gw, typename Pol::Acc& r,
                                             typename Pol::Acc& b) {
  using Acc = typename Pol::Acc;
  warp_reduce2(r, b);
  if ((threadIdx.x & 31) == 0) {
    const ScenDev& S = a.scen[sc];
    const double wdt = S.bw[a.stage] * S.dt;
    double* L = a.ledger + 2 * ((long long)sc * a.wslots + gw);
    L[0] += wdt * acc_d(r);
    L[1] += wdt * acc_d(b);
  }
  r = acc_make<Acc>(0.f, 0.f, 0.0);
  b = acc_make<Acc>(0.f, 0.f, 0.0);
}

// asynchronous global -> shared copies of 16 bytes (the copying thread owns the data)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// dynamic shared memory of the element kernel: per thread, the three neighbour records (fused)
// or the three edge slots (split), then the step-initial record; interleaved by thread so that
// the 16-byte reads of a warp hit distinct banks
template <int P, class Pol, bool SPLIT>
struct Staging {
  static constexpr int RV = Pol::template RV<P>;
  static constexpr int SV = SlotT<Pol>::template SV<P>;
  static constexpr int PER_EDGE = SPLIT ? SV : RV;
  static constexpr int VEC = 3 * PER_EDGE + RV;  // 16-byte vectors per thread
};
template <int P, class Pol, bool SPLIT>
__host__ __device__ constexpr int staging_bytes(int block) {
  return 16 * Staging<P, Pol, SPLIT>::VEC * block;
}

#ifndef DG_AREA_UNROLL
#define DG_AREA_UNROLL 1  // unroll factor of the area-quadrature loop
#endif
#ifndef DG_EDGE_UNROLL
#define DG_EDGE_UNROLL 1  // unroll factor of the three-edge loop
#endif
constexpr int kAreaUnroll = DG_AREA_UNROLL;
constexpr int kEdgeUnroll = DG_EDGE_UNROLL;

template <int P, int FLUX, class Pol, bool SPLIT>
#ifdef DG_MAXNREG
#define DG_STAGE_BOUNDS __maxnreg__(DG_MAXNREG)
#else
// register budget per thread: mixed p = 1 at 128 (16 warps per SM), mixed p = 2 at 144 (12 warps
// per SM as at the 166 the compiler picks unbounded, but 11-14 % faster code), FP64 unbounded
#define DG_STAGE_BOUNDS __maxnreg__(sizeof(typename Pol::T) == 4 ? (P == 2 ? 144 : 128) : 255)
#endif
__global__ void DG_STAGE_BOUNDS stage_kernel(const StageArgs<Pol> a) {
  using T = typename Pol::T;
  using Acc = typename Pol::Acc;
  using St = Staging<P, Pol, SPLIT>;
  constexpr int NP = np_of(P), NS = NP - 1, NG = P + 1;
  constexpr int RV = Pol::template RV<P>;
  constexpr int NQ = (P == 0) ? 1 : 7;
  const RefTab<T>& tab = ctab<T, P>();

  __shared__ T s_ephi[3][NG][NP];  // edge basis values, read at neighbour-dependent indices
  extern __shared__ uint4 stg[];   // [St::VEC][blockDim]
  const int tid = threadIdx.x, B = blockDim.x;
  for (int i = tid; i < 3 * NG * NP; i += B) {
    const int j = i / (NG * NP), k = (i / NP) % NG, m = i % NP;
    s_ephi[j][k][m] = tab.ephi[j][k][m];
  }
  __syncthreads();
  auto sv = [&](int v) -> uint4* { return stg + (size_t)v * B + tid; };

  const int lane = tid & 31;
  const long long gw = (long long)blockIdx.x * (B >> 5) + (tid >> 5);
  const long long W = (long long)gridDim.x * (B >> 5);
  const double stepd = (double)a.ctl->step + a.cst;
  const T g = a.g, H0 = a.H0;
  Acc rain_acc = acc_make<Acc>(0.f, 0.f, 0.0), bdry_acc = acc_make<Acc>(0.f, 0.f, 0.0);
  int cur = -1;

  for (long long tile = gw; tile < a.ntiles; tile += W) {
    const int sc = a.tile_scen[tile];
    if (sc != cur) {
      if (cur >= 0 && !a.tune) flush_ledger<P, Pol>(a, cur, gw, rain_acc, bdry_acc);
      cur = sc;
    }
    const ScenDev& S = a.scen[sc];
    const ForcingT<T>& F = forcing<T>(S);
    const long long e = tile * TILE + lane;
    if (e >= S.elem_end) continue;
    const T t = (T)(S.d.t0 + stepd * S.d.dt);  // stage time, formed in FP64

    const int4 nb = __ldg(a.nbr + e);
    // stage what the edge loop and the combination need, asynchronously
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int code = (j == 0) ? nb.x : (j == 1 ? nb.y : nb.z);
      if (SPLIT) {
        const uint4* src = a.slots + (3 * e + j) * St::SV;
#pragma unroll
        for (int i = 0; i < St::SV; ++i) cp_async16(sv(j * St::PER_EDGE + i), src + i);
      } else if (code >= 0) {
#pragma unroll
        for (int i = 0; i < RV; ++i) cp_async16(sv(j * St::PER_EDGE + i), a.in + rec_at<RV>(code >> 2, i));
      }
    }
    if (a.has_n) {
#pragma unroll
      for (int i = 0; i < RV; ++i) cp_async16(sv(3 * St::PER_EDGE + i), a.wn + rec_at<RV>(e, i));
    }
    cp_async_commit();

    Geo<Pol> G;
    load_geo(a.geo, e, nb, G);
    Raw<RV> rme;
    load_raw<RV>(a.in, e, rme);
    Elem<P, Pol> E;
    unpack<P>(rme, E);
    const int4 nd = (S.rain_kind >= 2 || S.press) ? __ldg(a.nodes + e) : make_int4(0, 0, 0, 0);
    const bool dry_me = (E.flags & FLAG_DRY) != 0;
    const T detJ = T(0.5) * acc_r(G.A);
    const T idetJ = T(2) * acc_r(G.invA);
    // inverse Jacobian from the edge vectors: t0 = x1 - x0 = 2 (xr, yr), t2 = x0 - x2 = -2 (xs, ys)
    // and ln_j = (t_j.y, -t_j.x)
    const T xr = T(-0.5) * G.lny[0], yr = T(0.5) * G.lnx[0];
    const T xs = T(0.5) * G.lny[2], ys = T(-0.5) * G.lnx[2];
    const T rx = ys * idetJ, ry = -xs * idetJ, sx = -yr * idetJ, sy = xr * idetJ;

    T Rz[NP], Rx[NP], Ry[NP];  // weak-form integrals against each basis function
#pragma unroll
    for (int m = 0; m < NP; ++m) Rz[m] = Rx[m] = Ry[m] = 0;

    // ---- area integrals (grad v, F) + (s, v), while the staged copies are in flight
    const T g1x = tab.qdr[0][1] * rx + tab.qds[0][1] * sx, g1y = tab.qdr[0][1] * ry + tab.qds[0][1] * sy;
    const T g2x = tab.qdr[0][2] * rx + tab.qds[0][2] * sx, g2y = tab.qdr[0][2] * ry + tab.qds[0][2] * sy;
    const T hbx = E.hb1 * g1x + E.hb2 * g2x, hby = E.hb1 * g1y + E.hb2 * g2y;  // constant grad(hb)
    const T cfm = (a.friction == 0) ? g * G.man * G.man : a.cf;
    T vx[3] = {0, 0, 0}, vy[3] = {0, 0, 0};
    if (S.press) {
      vx[0] = a.node_xy[2 * (long long)nd.x]; vy[0] = a.node_xy[2 * (long long)nd.x + 1];
      vx[1] = a.node_xy[2 * (long long)nd.y]; vy[1] = a.node_xy[2 * (long long)nd.y + 1];
      vx[2] = a.node_xy[2 * (long long)nd.z]; vy[2] = a.node_xy[2 * (long long)nd.z + 1];
    }
    // p = 1: the basis gradients are constant, so accumulate flux sums and source moments per
    // point and apply the gradients once
    T SF[6] = {0, 0, 0, 0, 0, 0};       // sum_q w_q (fx_z, fx_x, fx_y, fy_z, fy_x, fy_y)
    T SS[NP][2];                        // sum_q w_q phi_m s_(x,y)
#pragma unroll
    for (int m = 0; m < NP; ++m) SS[m][0] = SS[m][1] = 0;
    int q0 = 0;  // first quadrature point of the scalar loop
    if constexpr (DG_PACKED_FLUX && P == 1 && sizeof(T) == 4) {
      // points in pairs with packed FP32x2 arithmetic; the seventh point joins the scalar loop
      f2 SF2[6], SS2[NP][2];
#pragma unroll
      for (int i = 0; i < 6; ++i) SF2[i] = p2(0.f);
#pragma unroll
      for (int m = 0; m < NP; ++m) SS2[m][0] = SS2[m][1] = p2(0.f);
#pragma unroll 1
      for (int q = 0; q + 1 < NQ; q += 2) {
        const Trace<T> ta = trace_at<P, Pol>(E, tab.qphi[q]), tb = trace_at<P, Pol>(E, tab.qphi[q + 1]);
        const f2 d = make_float2(ta.d, tb.d), H = make_float2(ta.H, tb.H);
        const f2 qx = make_float2(ta.qx, tb.qx), qy = make_float2(ta.qy, tb.qy);
        const f2 Hs = max2(H, p2(H0));
        const f2 iH = rcp2(Hs);
        const f2 u = mul2(qx, iH), v = mul2(qy, iH);
        const f2 pp = mul2(mul2(p2(0.5f * g), d), fma2(p2(2.f), H, neg2(d)));  // pdev
        f2 tau = p2(0.f);
        if (a.friction == 0 || a.friction == 1) {
          const f2 uu = fma2(u, u, mul2(v, v));
          const f2 sp = make_float2(fsqrt0(uu.x), fsqrt0(uu.y));
          const f2 hf = (a.friction == 0) ? make_float2(fpowm43(Hs.x), fpowm43(Hs.y)) : iH;
          tau = mul2(p2(cfm), mul2(sp, hf));
        }
        f2 Fs[2] = {p2(0.f), p2(0.f)};
        if (S.press) {
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int qq = q + h;
            const T px = tab.ql[qq][0] * vx[0] + tab.ql[qq][1] * vx[1] + tab.ql[qq][2] * vx[2];
            const T py = tab.ql[qq][0] * vy[0] + tab.ql[qq][1] * vy[1] + tab.ql[qq][2] * vy[2];
            const T dx = px - F.ps[0], dy = py - F.ps[1], is2 = frcp(F.ps[2] * F.ps[2]);
            const T eta = F.ps[3] * fexp(-(dx * dx + dy * dy) * T(0.5) * is2);
            const T Hh = h ? tb.H : ta.H;
            (h ? Fs[0].y : Fs[0].x) = g * Hh * (-eta * dx * is2);
            (h ? Fs[1].y : Fs[1].x) = g * Hh * (-eta * dy * is2);
          }
        }
        const f2 sxq = fma2(p2(g * hbx), d, fma2(neg2(tau), qx, Fs[0]));
        const f2 syq = fma2(p2(g * hby), d, fma2(neg2(tau), qy, Fs[1]));
        const f2 fxx = fma2(qx, u, pp), fyx = mul2(qx, v);
        const f2 fxy = mul2(qy, u), fyy = fma2(qy, v, pp);
        const f2 w = make_float2(tab.qw[q], tab.qw[q + 1]);
        SF2[0] = fma2(w, qx, SF2[0]);
        SF2[1] = fma2(w, fxx, SF2[1]);
        SF2[2] = fma2(w, fxy, SF2[2]);
        SF2[3] = fma2(w, qy, SF2[3]);
        SF2[4] = fma2(w, fyx, SF2[4]);
        SF2[5] = fma2(w, fyy, SF2[5]);
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const f2 wp = mul2(w, make_float2(tab.qphi[q][m], tab.qphi[q + 1][m]));
          SS2[m][0] = fma2(wp, sxq, SS2[m][0]);
          SS2[m][1] = fma2(wp, syq, SS2[m][1]);
        }
      }
#pragma unroll
      for (int i = 0; i < 6; ++i) SF[i] = SF2[i].x + SF2[i].y;
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        SS[m][0] = SS2[m][0].x + SS2[m][0].y;
        SS[m][1] = SS2[m][1].x + SS2[m][1].y;
      }
      q0 = NQ - (NQ % 2);
    }
#pragma unroll kAreaUnroll
    for (int q = q0; q < NQ; ++q) {
      const Trace<T> tq = trace_at<P, Pol>(E, tab.qphi[q]);
      const T Hs = max_r(tq.H, H0);
      const T iH = frcp(Hs);
      const T u = tq.qx * iH, v = tq.qy * iH;
      const T pp = pdev(tq.d, tq.H, g);
      T tau = 0;
      if (a.friction == 0) tau = cfm * fsqrt0(u * u + v * v) * fpowm43(Hs);
      else if (a.friction == 1) tau = cfm * fsqrt0(u * u + v * v) * iH;
      T Fxs = 0, Fys = 0;
      if (S.press) {
        const T px = tab.ql[q][0] * vx[0] + tab.ql[q][1] * vx[1] + tab.ql[q][2] * vx[2];
        const T py = tab.ql[q][0] * vy[0] + tab.ql[q][1] * vy[1] + tab.ql[q][2] * vy[2];
        const T dx = px - F.ps[0], dy = py - F.ps[1], is2 = frcp(F.ps[2] * F.ps[2]);
        const T eta = F.ps[3] * fexp(-(dx * dx + dy * dy) * T(0.5) * is2);
        Fxs = g * tq.H * (-eta * dx * is2);
        Fys = g * tq.H * (-eta * dy * is2);
      }
      const T sx_ = g * tq.d * hbx - tau * tq.qx + Fxs;
      const T sy_ = g * tq.d * hby - tau * tq.qy + Fys;
      const T fxx = tq.qx * u + pp, fyx = tq.qx * v;
      const T fxy = tq.qy * u, fyy = tq.qy * v + pp;
      const T w = tab.qw[q];
      if (P == 1) {
        SF[0] = fma(w, tq.qx, SF[0]);
        SF[1] = fma(w, fxx, SF[1]);
        SF[2] = fma(w, fxy, SF[2]);
        SF[3] = fma(w, tq.qy, SF[3]);
        SF[4] = fma(w, fyx, SF[4]);
        SF[5] = fma(w, fyy, SF[5]);
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const T wp = w * tab.qphi[q][m];
          SS[m][0] = fma(wp, sx_, SS[m][0]);
          SS[m][1] = fma(wp, sy_, SS[m][1]);
        }
      } else {
        const T wq = w * detJ;
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const T dxm = tab.qdr[q][m] * rx + tab.qds[q][m] * sx;
          const T dym = tab.qdr[q][m] * ry + tab.qds[q][m] * sy;
          const T ph = tab.qphi[q][m];
          if (m > 0) Rz[m] = fma(wq, dxm * tq.qx + dym * tq.qy, Rz[m]);
          Rx[m] = fma(wq, dxm * fxx + dym * fyx + ph * sx_, Rx[m]);
          Ry[m] = fma(wq, dxm * fxy + dym * fyy + ph * sy_, Ry[m]);
        }
      }
    }
    if (P == 1) {
      const T gx[3] = {T(0), g1x, g2x}, gy[3] = {T(0), g1y, g2y};
#pragma unroll
      for (int m = 0; m < NP; ++m) {
        if (m > 0) Rz[m] = detJ * (gx[m] * SF[0] + gy[m] * SF[3]);
        Rx[m] = detJ * (gx[m] * SF[1] + gy[m] * SF[4] + SS[m][0]);
        Ry[m] = detJ * (gx[m] * SF[2] + gy[m] * SF[5] + SS[m][1]);
      }
    }

    // ---- forcing: element rain = mean of the three nodal rates (Eq. rain)
    T Re = 0;
    if (S.rain_kind == 1) {
      Re = a.rain_e[e];
    } else if (S.rain_kind >= 2) {
      T acc = 0;
      if (S.rain_kind == 2) {  // radial storm profile at the three vertices
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const long long n = (i == 0) ? nd.x : (i == 1 ? nd.y : nd.z);
          const T px = a.node_xy[2 * n], py = a.node_xy[2 * n + 1];
          const T tt = t - F.storm[7];
          const T dx = px - (F.storm[0] + F.storm[2] * tt), dy = py - (F.storm[1] + F.storm[3] * tt);
          const T r = fsqrt0(dx * dx + dy * dy);
          const T rp = F.storm[4], rm = F.storm[5], re = F.storm[6];
          acc += (r < rm) ? rp * (T(0.5) + T(0.5) * fdiv(r, rm)) : rp * fexp(-fdiv(r - rm, re));
        }
      } else {  // gridded: nodal rates interpolated by the node kernel of this stage
        acc = a.rain_node[nd.x];
        acc += a.rain_node[nd.y];
        acc += a.rain_node[nd.z];
      }
      Re = acc * T(1.0 / 3.0);
    }

    // ---- edge integrals <Fhat.n, v>, from the staged neighbour records or edge slots
    cp_async_wait_all();
    Acc massout = acc_make<Acc>(0.f, 0.f, 0.0);  // edge mass outflow (volume per second)
#pragma unroll kEdgeUnroll
    for (int j = 0; j < 3; ++j) {
      const int code = (j == 0) ? nb.x : (j == 1 ? nb.y : nb.z);
      const T lnx = (j == 0) ? G.lnx[0] : (j == 1 ? G.lnx[1] : G.lnx[2]);
      const T lny = (j == 0) ? G.lny[0] : (j == 1 ? G.lny[1] : G.lny[2]);
      bool wall = (code == -1);
      if (SPLIT && code >= 0) {  // interior edge: lift and mass flux from the edge kernel
        Lift<P, T> lf;
        load_slot<P>(sv(j * St::PER_EDGE), 0, lf, B);
        if (!lf.flag) {
#pragma unroll
          for (int m = 1; m < NP; ++m) Rz[m] += lf.v[m - 1];
#pragma unroll
          for (int m = 0; m < NP; ++m) {
            Rx[m] += lf.v[NS + m];
            Ry[m] += lf.v[NS + NP + m];
          }
          massout = acc_addr(massout, lf.mass);
          continue;
        }
        wall = true;  // closed by the wet/dry rule: my own wall flux below
      }
      const T len = fsqrt_pos(lnx * lnx + lny * lny);
      const T il = frcp(len);
      const T nx = lnx * il, ny = lny * il;
      Trace<T> tm[NG], to[NG];  // my trace and the other side's, at my edge points
#pragma unroll
      for (int k = 0; k < NG; ++k) tm[k] = trace_at<P, Pol>(E, s_ephi[j][k]);
      bool me_L = true, dry_o = false, river = false;
      T dcRL = 0, dc_nm = 0, qr = 0;
      if (!SPLIT && code >= 0) {
        const long long ne_ = code >> 2;
        const int jn = code & 3;
        Raw<RV> rnb;
#pragma unroll
        for (int i = 0; i < RV; ++i) rnb.v[i] = *sv(j * St::PER_EDGE + i);
        Elem<P, Pol> N;
        unpack<P>(rnb, N);
        me_L = e < ne_;
        dc_nm = acc_diff(N.zb, E.zb);                   // c_nb - c_me
        dcRL = me_L ? dc_nm : acc_diff(E.zb, N.zb);     // c_R - c_L
        dry_o = (N.flags & FLAG_DRY) != 0;
#pragma unroll
        for (int k = 0; k < NG; ++k) to[k] = trace_at<P, Pol>(N, s_ephi[jn][NG - 1 - k]);  // same point
      } else if (code <= -2 - MAXSEG) {  // river: interior elevation, prescribed normal discharge
        const int rs = min(-2 - MAXSEG - code, MAXRIV - 1);
        qr = river_at<T>(S, rs, S.d.t0 + ((double)a.ctl->step + a.cst) * S.d.dt);
        river = true;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          to[k] = tm[k];
          to[k].qx = -qr * nx;
          to[k].qy = -qr * ny;
        }
      } else if (code < -1) {  // ocean: tidal elevation, interior discharge
        const int seg = min(-2 - code, MAXSEG - 1);
        const double t64 = S.d.t0 + ((double)a.ctl->step + a.cst) * S.d.dt;  // stage time in FP64
        const T zbc = tide_at<T>(S, seg, t64);
        const T dgh = acc_r(acc_addr(acc_neg(E.zb), zbc));  // ghost zeta - my mean
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          to[k] = tm[k];
          to[k].H = tm[k].H + (dgh - tm[k].d);
          to[k].d = dgh;
        }
      }
      T Fz[NG], Fx[NG], Fy[NG];  // flux along my outward normal at my points
      T emine = 0;              // mass flux integral along my outward normal
      if (!wall) {
        const T sgn = me_L ? T(1) : T(-1);
        T fzc[NG], fxc[NG], fyc[NG];
        if constexpr (DG_PACKED_FLUX && P == 1 && sizeof(T) == 4) {
          const Trace<T> a0 = me_L ? tm[0] : to[0], b0 = me_L ? to[0] : tm[0];
          const Trace<T> a1 = me_L ? tm[1] : to[1], b1 = me_L ? to[1] : tm[1];
          const Trace2 L2{make_float2(a0.d, a1.d), make_float2(a0.H, a1.H), make_float2(a0.qx, a1.qx),
                          make_float2(a0.qy, a1.qy)};
          const Trace2 R2{make_float2(b0.d, b1.d), make_float2(b0.H, b1.H), make_float2(b0.qx, b1.qx),
                          make_float2(b0.qy, b1.qy)};
          f2 fz2, fx2, fy2;
          FluxAux2 ax;
          edge_flux_pair<FLUX>(L2, R2, p2(dcRL), p2(sgn * nx), p2(sgn * ny), g, H0, fz2, fx2, fy2, ax);
          fzc[0] = fz2.x; fzc[1] = fz2.y;
          fxc[0] = fx2.x; fxc[1] = fx2.y;
          fyc[0] = fy2.x; fyc[1] = fy2.y;
          if (river) fzc[0] = fzc[1] = -qr;
        } else {
#pragma unroll
          for (int k = 0; k < NG; ++k) {
            const Trace<T> tL = me_L ? tm[k] : to[k];
            const Trace<T> tR = me_L ? to[k] : tm[k];
            edge_flux<FLUX, T>(tL, tR, dcRL, sgn * nx, sgn * ny, g, H0, fzc[k], fxc[k], fyc[k]);
            if (river) fzc[k] = -qr;  // the specified normal flow is the mass flux
          }
        }
        T ecanon = 0;  // in L's point order: identical bits on both sides of the edge
#pragma unroll
        for (int kc = 0; kc < NG; ++kc) ecanon = fma(tab.gw[kc], me_L ? fzc[kc] : fzc[NG - 1 - kc], ecanon);
        ecanon = ecanon * (T(0.5) * len);
        const bool dry_L = me_L ? dry_me : dry_o, dry_R = me_L ? dry_o : dry_me;
        // wet/dry closure: no water leaves a dry element (interior: either side; ocean: mine)
        wall = (code >= 0) ? ((dry_L && ecanon > T(0)) || (dry_R && ecanon < T(0))) : (dry_me && ecanon > T(0));
        if (!wall) {
          emine = sgn * ecanon;
#pragma unroll
          for (int k = 0; k < NG; ++k) {
            const T p = T(0.5) * (pdev(tm[k].d, tm[k].H, g) + pdev(to[k].d + dc_nm, to[k].H, g));
            Fz[k] = sgn * fzc[k];
            Fx[k] = sgn * fxc[k] + p * nx;
            Fy[k] = sgn * fyc[k] + p * ny;
          }
        }
      }
      if (wall) {  // land edge or closed edge: reflective wall built from my own trace, no mass
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          const T qn = tm[k].qx * nx + tm[k].qy * ny;
          Trace<T> gh = tm[k];
          gh.qx = tm[k].qx - T(2) * qn * nx;
          gh.qy = tm[k].qy - T(2) * qn * ny;
          T fz, fx, fy;
          edge_flux<FLUX, T>(tm[k], gh, T(0), nx, ny, g, H0, fz, fx, fy);
          const T p = pdev(tm[k].d, tm[k].H, g);
          Fz[k] = 0;
          Fx[k] = fx + p * nx;
          Fy[k] = fy + p * ny;
        }
      }
      massout = acc_addr(massout, emine);
      if (code < -1) bdry_acc = acc_addr(bdry_acc, -emine);
      // lift: R_m -= sum_k w_k (len/2) F_k phi_m(edge j, point k)
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const T wk = tab.gw[k] * (T(0.5) * len);
#pragma unroll
        for (int m = 0; m < NP; ++m) {
          const T ph = wk * s_ephi[j][k][m];
          if (m > 0) Rz[m] = fma(-ph, Fz[k], Rz[m]);
          Rx[m] = fma(-ph, Fx[k], Rx[m]);
          Ry[m] = fma(-ph, Fy[k], Ry[m]);
        }
      }
    }
    if (dry_me) {  // the momentum equations are not advanced on dry elements
#pragma unroll
      for (int m = 0; m < NP; ++m) Rx[m] = Ry[m] = 0;
    }

    // ---- Shu-Osher combination: out = a_n w^n + a_in w^in + beta dt M^{-1} R
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
      for (int i = 0; i < RV; ++i) rn.v[i] = *sv(3 * St::PER_EDGE + i);
      unpack<P>(rn, Wn);
    }
    const T an_r = (sizeof(T) == 4) ? (T)a.a_n_hi : (T)a.a_n, ain_r = (sizeof(T) == 4) ? (T)a.a_in_hi : (T)a.a_in;
    {
      Acc z, x, y;
      if (sizeof(T) == 4 && a.pow2) {  // exact scaling of both words by a power of two
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

    // ---- positive-depth operator, store
    apply_positivity<P, Pol>(O, G, e, a, &a.ctl->err);
    Raw<RV> ro;
    pack<P>(O, ro);
    store_raw<RV>(a.out, e, ro);

    // ---- ledger: rain volume rate of the element
    rain_acc = acc_addf(rain_acc, acc_mulr(G.A, Re));
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

namespace dg {

// ------------------------------------------------------------------ auxiliary kernels ----
template <int P, class Pol>
__global__ void __launch_bounds__(256) prepare_kernel(const StageArgs<Pol> a, long long begin, long long end) {
  constexpr int RV = Pol::template RV<P>;
  for (long long e = begin + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < end;
       e += (long long)gridDim.x * blockDim.x) {
    const int4 nb = __ldg(a.nbr + e);
    Geo<Pol> G;
    load_geo(a.geo, e, nb, G);
    Raw<RV> r;
    load_raw<RV>(a.in, e, r);
    Elem<P, Pol> E;
    unpack<P>(r, E);
    Elem<P, Pol> O = E;
    apply_positivity<P, Pol>(O, G, e, a, &a.ctl->err);
    if (a.classify_only) {
      E.Hb = O.Hb;
      E.flags = O.flags;
      O = E;
    }
    pack<P>(O, r);
    store_raw<RV>(a.out, e, r);
  }
}

__device__ __forceinline__ void neu_add(double& s, double& c, double v) {
  const double t = s + v;
  c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
  s = t;
}
// merge two compensated sums (s, c) + (s2, c2)
__device__ __forceinline__ void neu_merge(double& s, double& c, double s2, double c2) {
  neu_add(s, c, s2);
  c += c2;
}

template <int P, class Pol>
__global__ void __launch_bounds__(256) volume_kernel(const uint4* rec, const uint4* geo, long long begin,
                                                     long long end, double* partials) {
  constexpr int RV = Pol::template RV<P>;
  double s0 = 0, c0 = 0, s1 = 0, c1 = 0;
  for (long long e = begin + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < end;
       e += (long long)gridDim.x * blockDim.x) {
    Geo<Pol> G;
    load_geo(geo, e, make_int4(0, 0, 0, 0), G);
    Raw<RV> r;
    load_raw<RV>(rec, e, r);
    Elem<P, Pol> E;
    unpack<P>(r, E);
    const double A = acc_d(G.A), z = acc_d(E.zb);
    neu_add(s0, c0, A * z);
    neu_add(s1, c1, A * z + A * acc_d(G.hbm));
  }
  __shared__ double sh[4][8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double a0 = __shfl_xor_sync(0xffffffffu, s0, o), b0 = __shfl_xor_sync(0xffffffffu, c0, o);
    const double a1 = __shfl_xor_sync(0xffffffffu, s1, o), b1 = __shfl_xor_sync(0xffffffffu, c1, o);
    neu_merge(s0, c0, a0, b0);
    neu_merge(s1, c1, a1, b1);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { sh[0][w] = s0; sh[1][w] = c0; sh[2][w] = s1; sh[3][w] = c1; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
      neu_merge(s0, c0, sh[0][k], sh[1][k]);
      neu_merge(s1, c1, sh[2][k], sh[3][k]);
    }
    partials[4 * blockIdx.x] = s0;
    partials[4 * blockIdx.x + 1] = c0;
    partials[4 * blockIdx.x + 2] = s1;
    partials[4 * blockIdx.x + 3] = c1;
  }
}

template <int P, class Pol>
__global__ void __launch_bounds__(256) dt_kernel(const uint4* rec, const int4* nodes, const double* xy,
                                                 const double* hbn, long long begin, long long end, double cfl,
                                                 double g, double H0, double* partials) {
  constexpr int RV = Pol::template RV<P>, NS = np_of(P) - 1;
  const RefTab<double>& tb = c_tab_d[P];
  double best = 1e300;
  for (long long e = begin + blockIdx.x * (long long)blockDim.x + threadIdx.x; e < end;
       e += (long long)gridDim.x * blockDim.x) {
    Raw<RV> r;
    load_raw<RV>(rec, e, r);
    Elem<P, Pol> E;
    unpack<P>(r, E);
    const int4 nd = nodes[e];
    const int v[3] = {nd.x, nd.y, nd.z};
    double per = 0, lam = 0;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int a0 = v[i], b0 = v[(i + 1) % 3];
      const double dx = xy[2 * (long long)b0] - xy[2 * (long long)a0], dy = xy[2 * (long long)b0 + 1] - xy[2 * (long long)a0 + 1];
      per += sqrt(dx * dx + dy * dy);
      double z = acc_d(E.zb), qx = acc_d(E.xb), qy = acc_d(E.yb);
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        z += (double)E.zs[m] * tb.vphi[i][m + 1];
        qx += (double)E.xs[m] * tb.vphi[i][m + 1];
        qy += (double)E.ys[m] * tb.vphi[i][m + 1];
      }
      const double H = z + hbn[v[i]], Hs = H > H0 ? H : H0;
      const double l = sqrt(qx * qx + qy * qy) / Hs + sqrt(g * Hs);
      lam = l > lam ? l : lam;
    }
    const double x0 = xy[2 * (long long)v[0]], y0 = xy[2 * (long long)v[0] + 1];
    const double A = 0.5 * ((xy[2 * (long long)v[1]] - x0) * (xy[2 * (long long)v[2] + 1] - y0) -
                            (xy[2 * (long long)v[2]] - x0) * (xy[2 * (long long)v[1] + 1] - y0));
    const double dt = cfl * (4.0 * A / per) / ((2.0 * P + 1.0) * lam);
    best = dt < best ? dt : best;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ double sh[8];
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) best = fmin(best, sh[k]);
    partials[blockIdx.x] = best;
  }
}

// modal state [Np][n] in caller order from the records of elements [begin, begin + n): thread c
// writes caller element c (consecutive threads write consecutive addresses, which keeps the
// stores coalesced when the arrays are page-locked host memory read over the C2C link) and reads
// the record of inv[c], its position in the library's order
template <int P, class Pol>
__global__ void __launch_bounds__(256) gather_kernel(const uint4* rec, long long begin, long long n,
                                                     const int32_t* inv, double* z, double* x, double* y) {
  constexpr int RV = Pol::template RV<P>, NS = np_of(P) - 1;
  const double s2 = 1.4142135623730951;  // mode-0 coefficient = sqrt(2) * mean
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    Raw<RV> r;
    load_raw<RV>(rec, begin + inv[c], r);
    Elem<P, Pol> E;
    unpack<P>(r, E);
    z[c] = s2 * acc_d(E.zb);
    x[c] = s2 * acc_d(E.xb);
    y[c] = s2 * acc_d(E.yb);
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      z[(m + 1) * n + c] = (double)E.zs[m];
      x[(m + 1) * n + c] = (double)E.xs[m];
      y[(m + 1) * n + c] = (double)E.ys[m];
    }
  }
}

// modal state [Np][n] in caller order -> records of elements [begin, begin + n) (thread c reads
// caller element c, coalesced); bathymetry modes are kept, depth and flags are recomputed by the
// positive-depth pass that follows
template <int P, class Pol>
__global__ void __launch_bounds__(256) scatter_kernel(uint4* rec, long long begin, long long n, const int32_t* inv,
                                                      const double* z, const double* x, const double* y) {
  constexpr int RV = Pol::template RV<P>, NS = np_of(P) - 1;
  const double is2 = 0.7071067811865476;  // mean = mode-0 coefficient / sqrt(2)
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n; c += (long long)gridDim.x * blockDim.x) {
    const long long e = begin + inv[c];
    Raw<RV> r;
    load_raw<RV>(rec, e, r);
    Elem<P, Pol> E;
    unpack<P>(r, E);
    acc_set(E.zb, is2 * z[c]);
    acc_set(E.xb, is2 * x[c]);
    acc_set(E.yb, is2 * y[c]);
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      E.zs[m] = (typename Pol::T)z[(m + 1) * n + c];
      E.xs[m] = (typename Pol::T)x[(m + 1) * n + c];
      E.ys[m] = (typename Pol::T)y[(m + 1) * n + c];
    }
    pack<P>(E, r);
    store_raw<RV>(rec, e, r);
  }
}

// ---------------------------------------------------------------- launcher instantiation ----
static inline int grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  return (int)(g < 1 ? 1 : (g > 65535 * 8 ? 65535 * 8 : g));
}

#define DG_DEFINE_LAUNCHERS(POL)                                                                             \
  template <>                                                                                                \
  cudaError_t upload_tables<POL>(int p, const RefTab<float>& tf, const RefTab<double>& td) {                 \
    cudaError_t e = cudaMemcpyToSymbol(c_tab_f, &tf, sizeof(RefTab<float>), p * sizeof(RefTab<float>));     \
    if (e != cudaSuccess) return e;                                                                          \
    const int m1 = staging_bytes<1, POL, false>(256), m1s = staging_bytes<1, POL, true>(256);                \
    const int m2 = staging_bytes<2, POL, false>(256), m2s = staging_bytes<2, POL, true>(256);                \
    const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;                                 \
    cudaFuncSetAttribute(stage_kernel<1, 0, POL, false>, A, m1);                                             \
    cudaFuncSetAttribute(stage_kernel<1, 1, POL, false>, A, m1);                                             \
    cudaFuncSetAttribute(stage_kernel<1, 0, POL, true>, A, m1s);                                             \
    cudaFuncSetAttribute(stage_kernel<1, 1, POL, true>, A, m1s);                                             \
    cudaFuncSetAttribute(stage_kernel<2, 0, POL, false>, A, m2);                                             \
    cudaFuncSetAttribute(stage_kernel<2, 1, POL, false>, A, m2);                                             \
    cudaFuncSetAttribute(stage_kernel<2, 0, POL, true>, A, m2s);                                             \
    cudaFuncSetAttribute(stage_kernel<2, 1, POL, true>, A, m2s);                                             \
    return cudaMemcpyToSymbol(c_tab_d, &td, sizeof(RefTab<double>), p * sizeof(RefTab<double>));            \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_stage<POL>(int p, int flux, const StageArgs<POL>& a, int grid, int block, cudaStream_t s) { \
    const int k = (p == 1 ? 0 : 4) + (flux ? 2 : 0) + (a.split ? 1 : 0);                                     \
    switch (k) {                                                                                             \
      case 0: stage_kernel<1, 0, POL, false><<<grid, block, staging_bytes<1, POL, false>(block), s>>>(a); break; \
      case 1: stage_kernel<1, 0, POL, true><<<grid, block, staging_bytes<1, POL, true>(block), s>>>(a); break; \
      case 2: stage_kernel<1, 1, POL, false><<<grid, block, staging_bytes<1, POL, false>(block), s>>>(a); break; \
      case 3: stage_kernel<1, 1, POL, true><<<grid, block, staging_bytes<1, POL, true>(block), s>>>(a); break; \
      case 4: stage_kernel<2, 0, POL, false><<<grid, block, staging_bytes<2, POL, false>(block), s>>>(a); break; \
      case 5: stage_kernel<2, 0, POL, true><<<grid, block, staging_bytes<2, POL, true>(block), s>>>(a); break; \
      case 6: stage_kernel<2, 1, POL, false><<<grid, block, staging_bytes<2, POL, false>(block), s>>>(a); break; \
      default: stage_kernel<2, 1, POL, true><<<grid, block, staging_bytes<2, POL, true>(block), s>>>(a); break; \
    }                                                                                                        \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_edges<POL>(int p, int flux, const StageArgs<POL>& a, int grid, int block, cudaStream_t s) { \
    if (p == 1 && flux == 0) edge_kernel<1, 0, POL><<<grid, block, 0, s>>>(a);                                \
    else if (p == 1) edge_kernel<1, 1, POL><<<grid, block, 0, s>>>(a);                                        \
    else if (flux == 0) edge_kernel<2, 0, POL><<<grid, block, 0, s>>>(a);                                     \
    else edge_kernel<2, 1, POL><<<grid, block, 0, s>>>(a);                                                   \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  template <>                                                                                                \
  int stage_blocks_per_sm<POL>(int p, int flux, int block, int split) {                                      \
    int n = 0;                                                                                               \
    const int k = (p == 1 ? 0 : 4) + (flux ? 2 : 0) + (split ? 1 : 0);                                       \
    switch (k) {                                                                                             \
      case 0: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<1, 0, POL, false>, block, staging_bytes<1, POL, false>(block)); break; \
      case 1: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<1, 0, POL, true>, block, staging_bytes<1, POL, true>(block)); break; \
      case 2: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<1, 1, POL, false>, block, staging_bytes<1, POL, false>(block)); break; \
      case 3: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<1, 1, POL, true>, block, staging_bytes<1, POL, true>(block)); break; \
      case 4: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<2, 0, POL, false>, block, staging_bytes<2, POL, false>(block)); break; \
      case 5: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<2, 0, POL, true>, block, staging_bytes<2, POL, true>(block)); break; \
      case 6: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<2, 1, POL, false>, block, staging_bytes<2, POL, false>(block)); break; \
      default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_kernel<2, 1, POL, true>, block, staging_bytes<2, POL, true>(block)); break; \
    }                                                                                                        \
    return n;                                                                                                \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_prepare<POL>(int p, const StageArgs<POL>& a, long long b, long long e, cudaStream_t s) { \
    int g = grid_for(e - b, 256);                                                                            \
    if (p == 1) prepare_kernel<1, POL><<<g, 256, 0, s>>>(a, b, e);                                           \
    else prepare_kernel<2, POL><<<g, 256, 0, s>>>(a, b, e);                                                  \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_limiter<POL>(const StageArgs<POL>& a, long long ne, cudaStream_t s) {                   \
    limit_kernel<POL><<<grid_for(ne, 256), 256, 0, s>>>(a, ne);                                              \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_node_rain<POL>(const StageArgs<POL>& a, long long nn, cudaStream_t s) {                 \
    node_rain_kernel<POL><<<grid_for(nn, 256), 256, 0, s>>>(a, nn);                                          \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_volume<POL>(int p, const uint4* rec, const uint4* geo, long long b, long long e,        \
                                 double* partials, int nblk, cudaStream_t s) {                               \
    if (p == 1) volume_kernel<1, POL><<<nblk, 256, 0, s>>>(rec, geo, b, e, partials);                        \
    else volume_kernel<2, POL><<<nblk, 256, 0, s>>>(rec, geo, b, e, partials);                               \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_dt<POL>(int p, const uint4* rec, const int4* nodes, const double* xy, const double* hbn, \
                             long long b, long long e, double cfl, double g, double H0, double* partials,     \
                             int nblk, cudaStream_t s) {                                                     \
    if (p == 1) dt_kernel<1, POL><<<nblk, 256, 0, s>>>(rec, nodes, xy, hbn, b, e, cfl, g, H0, partials);      \
    else dt_kernel<2, POL><<<nblk, 256, 0, s>>>(rec, nodes, xy, hbn, b, e, cfl, g, H0, partials);             \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_gather<POL>(int p, const uint4* rec, long long b, long long n, const int32_t* inv,       \
                                 double* z, double* x, double* y, cudaStream_t s) {                          \
    int g = grid_for(n, 256);                                                                                \
    if (p == 1) gather_kernel<1, POL><<<g, 256, 0, s>>>(rec, b, n, inv, z, x, y);                            \
    else gather_kernel<2, POL><<<g, 256, 0, s>>>(rec, b, n, inv, z, x, y);                                   \
    return cudaGetLastError();                                                                               \
  }                                                                                                          \
  template <>                                                                                                \
  cudaError_t launch_scatter<POL>(int p, uint4* rec, long long b, long long n, const int32_t* inv,           \
                                  const double* z, const double* x, const double* y, cudaStream_t s) {       \
    int g = grid_for(n, 256);                                                                                \
    if (p == 1) scatter_kernel<1, POL><<<g, 256, 0, s>>>(rec, b, n, inv, z, x, y);                           \
    else scatter_kernel<2, POL><<<g, 256, 0, s>>>(rec, b, n, inv, z, x, y);                                  \
    return cudaGetLastError();                                                                               \
  }

}  // namespace dg
