// api.cu -- C interface and host runtime of libdgswe (declarations and contracts: dgswe.h).
//
// A context holds one or more scenarios (host copies of preprocessed mesh, fields, forcing and
// initial state).  At dgswe_set_state (or dgswe_ensemble_create) the scenarios are packed into
// one device layout: element records, static geometry, connectivity and per-scenario parameter
// blocks, scenario element ranges aligned to 256 so tiles never straddle two scenarios.  A step
// is one launch of the fused stage kernel per Runge-Kutta stage; steps are replayed from CUDA
// graphs (1 step and 8 steps) captured on a private stream and launched on the caller's.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "args.h"
#include "exchange.h"
#include "dgswe.h"
#include "host.h"
#include "layout.h"

using namespace dg;

static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

// lets the other translation units of the library report an error message
void dg::set_last_error(const std::string& msg) { g_err = msg; }

#define CU(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(DGSWE_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

namespace {

struct Scenario {
  HostMesh m;
  std::vector<double> hb;          // nodal bathymetry, new node order
  std::vector<double> man;         // element Manning n, new element order
  int rain_kind = 0;               // 0 none, 1 nodal constant, 2 storm, 3 grid
  std::vector<double> rain_n;      // nodal constant rain, new node order
  dgswe_storm storm{};
  int gnx = 0, gny = 0, gnt = 0;
  double gx0 = 0, gy0 = 0, gdx = 1, gdy = 1, gt0 = 0, gdt = 1;
  std::vector<float> grid;
  std::vector<double> tamp, tper, tpha;
  int rnseg = 0, rnt = 0;          // river segments and records
  double rt0 = 0.0, rdt = 1.0;
  std::vector<double> river;       // [rnt][rnseg] m^2/s into the domain
  bool press = false;
  dgswe_gauss_setup ps{};
  std::vector<double> w;           // caller's state, modal [ne][3][np], new element order
  double t0 = 0.0;
  double dt = 0.0;                 // fixed time step (known after set_state)
  int level = 0;                   // 1 mesh, 2 fields, 3 state
};

struct Stage {
  double a_n, a_in, beta, c, bw;
};

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  bool own = true;  // false: memory bound by the caller (dgswe_bind_device), never freed here
  ~DevBuf() { release(); }
  void release() {
    if (p && own) cudaFree(p);
    p = nullptr;
    own = true;
  }
  int alloc(size_t bytes) {
    release();
    n = bytes;
    if (bytes == 0) return 0;
    return cudaMalloc(&p, bytes) == cudaSuccess ? 0 : -1;
  }
  void bind(void* ptr, size_t bytes) {
    release();
    p = ptr;
    n = bytes;
    own = false;
  }
  template <class T>
  T* as() const { return reinterpret_cast<T*>(p); }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() { if (prev >= 0) cudaSetDevice(prev); }
};

}  // namespace

struct dgswe_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;   // caller's stream (launches)
  cudaStream_t cap = nullptr;      // private stream (graph capture)
  bool own_stream = false;
  dgswe_params prm{};
  bool has_params = false;
  std::vector<Scenario> sc;
  bool ensemble = false;
  // device layout
  bool ready = false;
  int np = 0, rv = 0, gv = 0;      // modes, record and geometry sizes (16-byte units)
  long long E = 0, N = 0;          // padded element count, node count
  std::vector<long long> eoff, noff;
  DevBuf rec[3], nbr, geo, nodes, node_xy, xy64, hbn, rain_e, rain_node, node_scen, lim, scen, tile_scen, tile_meta, xy0,
      ledger, ctl,
      einv, grids, rivers, scratch,
      gather_buf, edges, slots;
  long long nedges = 0;
  int ntiles = 0;                          // 32-element tiles
  int wslots = 0;                          // ledger slots per scenario
  int wcur = 0;                            // warps of the current launch shape
  std::vector<double> led_rain, led_bdry;  // host-folded ledger of retired launch shapes
  std::vector<double> V0, VH0;
  std::vector<Stage> stages;
  // launch configuration
  int block = 128, waves = 1, split = 1;
  bool autotune = true;
  bool graphs = true;  // replay steps from CUDA graphs (else direct launches)
  bool grid_rain = false;  // some scenario has gridded rain: a node kernel runs before each stage
  int feat = FT_ALL;       // features of the run (Feature bits): selects the tile-kernel instantiation
  long long nn_total = 0;
  int grid = 0;
  cudaGraphExec_t g1 = nullptr, gK = nullptr;
  int K = 8;
  long long launches = 0;
  char* bound = nullptr;           // caller memory holding the three record buffers (dgswe_bind_device)
  size_t bound_bytes = 0;

  ~dgswe_ctx() {
    DeviceGuard dg_(device);
    DevBuf* bufs[] = {&rec[0], &rec[1], &rec[2], &nbr, &geo, &nodes, &node_xy, &xy64, &hbn, &rain_e, &scen,
                      &tile_scen, &tile_meta, &xy0, &ledger, &ctl, &einv, &grids, &rivers, &scratch, &gather_buf,
                      &edges, &slots,
                      &rain_node, &node_scen, &lim};
    for (DevBuf* b : bufs) b->alloc(0);
    if (g1) cudaGraphExecDestroy(g1);
    if (gK) cudaGraphExecDestroy(gK);
    if (cap) cudaStreamDestroy(cap);
    if (own_stream && stream) cudaStreamDestroy(stream);
  }
};

// ------------------------------------------------------------------------------ helpers --
// Neumaier-compensated sum of per-block (sum, compensation) pairs, one CTA, fixed order
__global__ void __launch_bounds__(256) reduce_pairs_kernel(const double* part, int nblk, int npairs, double* out) {
  __shared__ double sh[2][8];
  for (int k = 0; k < npairs; ++k) {
    double s = 0.0, c = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      const double v = part[4 * b + 2 * k], t = s + v;
      c += (fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s;
      s = t;
      c += part[4 * b + 2 * k + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double v = __shfl_xor_sync(0xffffffffu, s, o), vc = __shfl_xor_sync(0xffffffffu, c, o);
      const double t = s + v;
      c += ((fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s) + vc;
      s = t;
    }
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = s; sh[1][threadIdx.x >> 5] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        const double v = sh[0][w], t = s + v;
        c += ((fabs(s) >= fabs(v)) ? (s - t) + v : (v - t) + s) + sh[1][w];
        s = t;
      }
      out[2 * k] = s;
      out[2 * k + 1] = c;
    }
    __syncthreads();
  }
}

cudaError_t dg::launch_reduce_pairs(const double* partials, int nblk, int npairs, double* out, cudaStream_t s) {
  reduce_pairs_kernel<<<1, 256, 0, s>>>(partials, nblk, npairs, out);
  return cudaGetLastError();
}

static void split_ff(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

static bool mixed(const dgswe_ctx* h) { return h->prm.precision == DGSWE_MIXED; }

static std::vector<Stage> ssp_table(int s) {
  std::vector<Stage> t;
  if (s == 2) {
    t = {{0.0, 1.0, 1.0, 0.0, 0}, {0.5, 0.5, 0.5, 1.0, 0}};
  } else if (s == 5) {
    // optimal five-stage second-order SSP: four forward-Euler substeps of dt/4, then a convex
    // combination with w^n
    t = {{0.0, 1.0, 0.25, 0.0, 0}, {0.0, 1.0, 0.25, 0.25, 0}, {0.0, 1.0, 0.25, 0.5, 0},
         {0.0, 1.0, 0.25, 0.75, 0}, {0.2, 0.8, 0.2, 1.0, 0}};
  } else {
    t = {{0.0, 1.0, 1.0, 0.0, 0}, {0.75, 0.25, 0.25, 1.0, 0}, {1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 0.5, 0}};
  }
  // weight of dt L(w^(s)) in the final stage: c_{i+1} = a_n c_0 + a_in c_i + beta_i e_i, c_0 = 0
  const int n = (int)t.size();
  std::vector<std::vector<double>> c(n + 1, std::vector<double>(n, 0.0));
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < n; ++k) c[i + 1][k] = t[i].a_n * c[0][k] + t[i].a_in * c[i][k] + (k == i ? t[i].beta : 0.0);
  for (int k = 0; k < n; ++k) t[k].bw = c[n][k];
  return t;
}

// slope limiter data per element (new order): for local edge i the coefficients a_i, c_i >= 0
// of m_i - b_0 = a_i (b_i - b_0) + c_i (b_k - b_0), k = i+1 (bit i clear) or i+2 (bit i set)
// trying i+1 first; M h^2 with h the longest edge; pair bits, or -1 when the element has a
// boundary edge or an edge without such a pair (not limited)
static std::vector<double> limiter_data(dgswe_h h, long long E) {
  std::vector<double> L(8 * (size_t)E, 0.0);
  for (long long e = 0; e < E; ++e) L[8 * e + 7] = -1.0;
  for (size_t s = 0; s < h->sc.size(); ++s) {
    const HostMesh& M = h->sc[s].m;
    const long long eo = h->eoff[s];
    auto bary = [&](int e, double& x, double& y) {
      const int32_t* v = &M.tri[3 * (size_t)e];
      x = (M.x[v[0]] + M.x[v[1]] + M.x[v[2]]) / 3.0;
      y = (M.y[v[0]] + M.y[v[1]] + M.y[v[2]]) / 3.0;
    };
    for (int e = 0; e < M.ne; ++e) {
      int nb[3];
      bool interior = true;
      for (int j = 0; j < 3; ++j) {
        const int32_t c = M.code[3 * (size_t)e + j];
        interior = interior && c >= 0;
        nb[j] = c >= 0 ? (c >> 2) : -1;
      }
      if (!interior) continue;
      const int32_t* v = &M.tri[3 * (size_t)e];
      double bx[4], by[4];
      bary(e, bx[0], by[0]);
      for (int j = 0; j < 3; ++j) bary(nb[j], bx[j + 1], by[j + 1]);
      double hmax = 0.0;
      for (int j = 0; j < 3; ++j)
        hmax = std::max(hmax, std::hypot(M.x[v[(j + 1) % 3]] - M.x[v[j]], M.y[v[(j + 1) % 3]] - M.y[v[j]]));
      double* out = &L[8 * (size_t)(eo + e)];
      int bits = 0;
      bool ok = true;
      for (int i = 0; i < 3 && ok; ++i) {
        const double mx = 0.5 * (M.x[v[i]] + M.x[v[(i + 1) % 3]]) - bx[0];
        const double my = 0.5 * (M.y[v[i]] + M.y[v[(i + 1) % 3]]) - by[0];
        bool found = false;
        for (int t = 1; t <= 2 && !found; ++t) {
          const int k = (i + t) % 3;
          const double ax = bx[i + 1] - bx[0], ay = by[i + 1] - by[0], cx = bx[k + 1] - bx[0], cy = by[k + 1] - by[0];
          const double det = ax * cy - ay * cx;
          if (det == 0.0) continue;
          const double a = (mx * cy - my * cx) / det, c = (ax * my - ay * mx) / det;
          if (a >= 0.0 && c >= 0.0) {
            out[2 * i] = a;
            out[2 * i + 1] = c;
            if (t == 2) bits |= 1 << i;
            found = true;
          }
        }
        ok = found;
      }
      out[6] = h->prm.lim_M * hmax * hmax;
      out[7] = ok ? (double)bits : -1.0;
    }
  }
  return L;
}

static int check_handle(dgswe_h h) {
  if (!h) return fail(DGSWE_EINVAL, "null handle");
  return 0;
}

static RefTab<double> g_tabd[3];
static RefTab<float> g_tabf[3];
static bool g_tab_built[3] = {false, false, false};

static int upload_all_tables(int p) {
  if (!g_tab_built[p]) {
    build_tables(p, g_tabd[p]);
    tables_to_float(g_tabd[p], g_tabf[p]);
    g_tab_built[p] = true;
  }
  CU(upload_tables<Mixed>(p, g_tabf[p], g_tabd[p]));
  CU(upload_tables<Fp64>(p, g_tabf[p], g_tabd[p]));
  CU(upload_tile_tables<Mixed>(p, g_tabf[p], g_tabd[p]));
  CU(upload_tile_spec_tables(p, g_tabf[p], g_tabd[p]));
  CU(upload_tile_tables<Fp64>(p, g_tabf[p], g_tabd[p]));
  return 0;
}

// one record buffer's share of bound memory: its size rounded up to 256 bytes
static size_t record_stride(size_t rbytes) { return (rbytes + 255) / 256 * 256; }

// Element records on the device are tile-blocked (the layout the kernels read): the 16-byte
// vector v of element e is vector ((e / 32) rv + v) 32 + e % 32 of the array.
static size_t rec_vec(size_t e, size_t v, size_t rv) { return ((e >> 5) * rv + v) * 32 + (e & 31); }
// 32-bit word w of element e's record in a tile-blocked array (e counted from the array's start,
// which is tile-aligned)
static uint32_t rec_word(const std::vector<uint32_t>& blk, size_t e, size_t w, size_t rv) {
  return blk[4 * rec_vec(e, w / 4, rv) + w % 4];
}
// element-major records (rw = 4 rv words each) -> tile-blocked, E a multiple of 32
static std::vector<uint32_t> to_blocked(const std::vector<uint32_t>& rec, size_t E, size_t rv) {
  std::vector<uint32_t> blk(rec.size());
  for (size_t e = 0; e < E; ++e)
    for (size_t v = 0; v < rv; ++v) std::memcpy(&blk[4 * rec_vec(e, v, rv)], &rec[4 * (rv * e + v)], 16);
  return blk;
}

// device-visible address of page-locked host memory (zero-copy), or nullptr when p is pageable
// memory, device memory or not known to the runtime
static const void* host_mapped(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return (at.type == cudaMemoryTypeHost && at.devicePointer) ? at.devicePointer : nullptr;
}

// --------------------------------------------------------------------- device layout -------
template <class T>
static void put(std::vector<uint32_t>& w, size_t at, T v) {
  std::memcpy(&w[at], &v, sizeof(T));
}

// a Shu-Osher weight that scales a float-float value exactly: zero or a positive power of two
static bool pow2_or_0(double c) {
  int ex = 0;
  return c == 0.0 || (c > 0.0 && std::frexp(c, &ex) == 0.5);
}

// the Feature bits of the run: boundary kinds present in the neighbour codes, forcing kinds of
// every scenario, the friction law and the kinds of Runge-Kutta stage weights
static int run_features(dgswe_h h, const std::vector<int32_t>& nbr) {
  int f = 0;
  for (size_t i = 0; i < nbr.size(); i += 4)
    for (int j = 0; j < 3; ++j) {
      const int32_t c = nbr[i + j];
      if (c <= -2 - MAXSEG) f |= FT_RIVER;
      else if (c <= -2) f |= FT_OCEAN;
    }
  for (const Scenario& S : h->sc) {
    if (S.rain_kind == 0) f |= FT_RAIN0;
    if (S.rain_kind == 1) f |= FT_RAIN1;
    if (S.rain_kind == 2) f |= FT_RAIN2;
    if (S.rain_kind == 3) f |= FT_RAIN3;
    if (S.press) f |= FT_PRESS;
  }
  f |= h->prm.friction == DGSWE_MANNING ? FT_MANNING : h->prm.friction == DGSWE_QUADRATIC ? FT_QUAD : FT_NOFRIC;
  for (const Stage& st : h->stages) f |= (pow2_or_0(st.a_n) && pow2_or_0(st.a_in)) ? FT_POW2 : FT_GENSSP;
  return f;
}

static int build_layout(dgswe_h h) {
  DeviceGuard dg_(h->device);
  const int p = h->prm.p, np = np_of(p);
  const bool mx = mixed(h);
  h->np = np;
  h->rv = mx ? rec_vec_mixed(p) : rec_vec_fp64(p);
  h->gv = mx ? 3 : 5;
  const size_t ns = h->sc.size();
  h->eoff.assign(ns, 0);
  h->noff.assign(ns, 0);
  long long E = 0, N = 0;
  for (size_t s = 0; s < ns; ++s) {
    h->eoff[s] = E;
    h->noff[s] = N;
    E += (h->sc[s].m.ne + TILE_ALIGN - 1) / TILE_ALIGN * TILE_ALIGN;
    N += h->sc[s].m.nn;
  }
  h->E = E;
  h->N = N;
  if (upload_all_tables(p)) return DGSWE_ECUDA;
  const RefTab<double>& tb = g_tabd[p];
  // host images
  const size_t rw = 4 * (size_t)h->rv, gw = 4 * (size_t)h->gv;  // 32-bit words per element
  std::vector<uint32_t> rec(rw * E, 0u), geo(gw * E, 0u);
  std::vector<int32_t> nbr(4 * E, -1), nodes(4 * E, 0), einv(E, 0);
  std::vector<float> xy0f(mx ? 2 * E : 0, 0.f);     // first vertex of each element (tile form)
  std::vector<double> xy0d(mx ? 0 : 2 * E, 0.0);
  std::vector<double> xy64(2 * N), hbn(N);
  std::vector<int32_t> nscen(N, 0);
  std::vector<float> xyf(mx ? 2 * N : 0), rainf(mx ? E : 0);
  std::vector<double> rain64(mx ? 0 : E);
  std::vector<float> grids;
  std::vector<size_t> grid_off(ns, 0);
  std::vector<double> rivers;
  std::vector<size_t> river_off(ns, 0);
  for (size_t s = 0; s < ns; ++s) {
    const Scenario& S = h->sc[s];
    const HostMesh& M = S.m;
    const long long eo = h->eoff[s], no = h->noff[s];
    for (int i = 0; i < M.nn; ++i) {
      nscen[no + i] = (int32_t)s;
      xy64[2 * (no + i)] = M.x[i];
      xy64[2 * (no + i) + 1] = M.y[i];
      hbn[no + i] = S.hb[i];
      if (mx) { xyf[2 * (no + i)] = (float)M.x[i]; xyf[2 * (no + i) + 1] = (float)M.y[i]; }
    }
    if (S.rain_kind == 3) { grid_off[s] = grids.size(); grids.insert(grids.end(), S.grid.begin(), S.grid.end()); }
    if (S.rnseg > 0) { river_off[s] = rivers.size(); rivers.insert(rivers.end(), S.river.begin(), S.river.end()); }
    for (int e = 0; e < M.ne; ++e) {
      const long long ge = eo + e;
      const int32_t* v = &M.tri[3 * (size_t)e];
      einv[eo + M.eorig[e]] = e;  // caller element -> position in the library's order
      if (mx) {
        xy0f[2 * ge] = (float)M.x[v[0]];
        xy0f[2 * ge + 1] = (float)M.y[v[0]];
      } else {
        xy0d[2 * ge] = M.x[v[0]];
        xy0d[2 * ge + 1] = M.y[v[0]];
      }
      for (int j = 0; j < 3; ++j) {
        const int32_t c = M.code[3 * (size_t)e + j];
        nbr[4 * ge + j] = c >= 0 ? (int32_t)((((c >> 2) + eo) << 2) | (c & 3)) : c;
        nodes[4 * ge + j] = (int32_t)(v[j] + no);
      }
      const double hv[3] = {S.hb[v[0]], S.hb[v[1]], S.hb[v[2]]};
      const double hbm = (hv[0] + hv[1] + hv[2]) / 3.0;
      const double hb1 = tb.vinv[0][0] * hv[0] + tb.vinv[0][1] * hv[1] + tb.vinv[0][2] * hv[2];
      const double hb2 = tb.vinv[1][0] * hv[0] + tb.vinv[1][1] * hv[1] + tb.vinv[1][2] * hv[2];
      const double A = M.area[e], invA = 1.0 / A;
      const double man = S.man.empty() ? 0.0 : S.man[e];
      double re = 0.0;
      if (S.rain_kind == 1) re = (S.rain_n[v[0]] + S.rain_n[v[1]] + S.rain_n[v[2]]) / 3.0;
      // state record
      const double* w = &S.w[(size_t)e * 3 * np];
      const double s2 = 1.0 / std::sqrt(2.0);
      uint32_t* R = &rec[rw * ge];
      uint32_t* Gm = &geo[gw * ge];
      const int NS = np - 1;
      if (mx) {
        float hi, lo;
        for (int var = 0; var < 3; ++var) {
          split_ff(w[var * np] * s2, hi, lo);
          put(rec, rw * ge + 2 * var, hi);
          put(rec, rw * ge + 2 * var + 1, lo);
          for (int m = 0; m < NS; ++m) put(rec, rw * ge + 6 + var * NS + m, (float)w[var * np + m + 1]);
        }
        const size_t o = rw * ge + 6 + 3 * NS;
        put(rec, o + 2, (float)hb1);
        put(rec, o + 3, (float)hb2);
        for (int j = 0; j < 3; ++j) {
          put(geo, gw * ge + 2 * j, (float)M.lnx[3 * (size_t)e + j]);
          put(geo, gw * ge + 2 * j + 1, (float)M.lny[3 * (size_t)e + j]);
        }
        split_ff(hbm, hi, lo); put(geo, gw * ge + 6, hi); put(geo, gw * ge + 7, lo);
        split_ff(A, hi, lo); put(geo, gw * ge + 8, hi); put(geo, gw * ge + 9, lo);
        split_ff(invA, hi, lo); put(geo, gw * ge + 10, hi); put(geo, gw * ge + 11, lo);
        float mf = (float)man;
        std::memcpy(&nbr[4 * ge + 3], &mf, 4);
        rainf[ge] = (float)re;
      } else {
        for (int var = 0; var < 3; ++var) {
          put(rec, rw * ge + 2 * var, w[var * np] * s2);
          for (int m = 0; m < NS; ++m) put(rec, rw * ge + 2 * (3 + var * NS + m), w[var * np + m + 1]);
        }
        const size_t o = rw * ge + 2 * (3 + 3 * NS);
        put(rec, o + 4, hb1);
        put(rec, o + 6, hb2);
        for (int j = 0; j < 3; ++j) {
          put(geo, gw * ge + 4 * j, M.lnx[3 * (size_t)e + j]);
          put(geo, gw * ge + 4 * j + 2, M.lny[3 * (size_t)e + j]);
        }
        put(geo, gw * ge + 12, hbm);
        put(geo, gw * ge + 14, A);
        put(geo, gw * ge + 16, invA);
        put(geo, gw * ge + 18, man);
        nbr[4 * ge + 3] = 0;
        rain64[ge] = re;
      }
      (void)R;
      (void)Gm;
    }
  }
  // interior edges for the edge-split path, canonical orientation (L = lower element index)
  const int ev = mx ? 1 : 2;
  std::vector<uint32_t> edg;
  for (size_t s = 0; s < ns; ++s) {
    const HostMesh& M = h->sc[s].m;
    const long long eo = h->eoff[s];
    for (int e = 0; e < M.ne; ++e)
      for (int j = 0; j < 3; ++j) {
        const int32_t c = M.code[3 * (size_t)e + j];
        if (c < 0 || (c >> 2) < e) continue;
        const uint32_t wl = (uint32_t)(((e + eo) << 2) | j), wr = (uint32_t)((((c >> 2) + eo) << 2) | (c & 3));
        const double lx = M.lnx[3 * (size_t)e + j], ly = M.lny[3 * (size_t)e + j];
        const size_t at = edg.size();
        edg.resize(at + 4 * ev, 0u);
        edg[at] = wl;
        edg[at + 1] = wr;
        if (mx) {
          const float fx = (float)lx, fy = (float)ly;
          std::memcpy(&edg[at + 2], &fx, 4);
          std::memcpy(&edg[at + 3], &fy, 4);
        } else {
          std::memcpy(&edg[at + 4], &lx, 8);
          std::memcpy(&edg[at + 6], &ly, 8);
        }
      }
  }
  h->nedges = (long long)(edg.size() / (4 * ev));
  const int sv = mx ? slot_vec_mixed(p) : slot_vec_fp64(p);
  if (h->edges.alloc(std::max<size_t>(16, 4 * edg.size())) || h->slots.alloc(16 * (size_t)sv * 3 * E))
    return fail(DGSWE_ENOMEM, "device allocation of the edge-split buffers failed");
  if (!edg.empty()) CU(cudaMemcpy(h->edges.p, edg.data(), 4 * edg.size(), cudaMemcpyHostToDevice));
  CU(cudaMemset(h->slots.p, 0, 16 * (size_t)sv * 3 * E));
  // upload
  const size_t rbytes = 16 * (size_t)h->rv * E;
  if (h->bound && h->bound_bytes >= 3 * record_stride(rbytes)) {  // keep the caller's binding
    for (int b = 0; b < 3; ++b) h->rec[b].bind(h->bound + b * record_stride(rbytes), rbytes);
  } else {
    h->bound = nullptr;
    h->bound_bytes = 0;
    for (int b = 0; b < 3; ++b)
      if (h->rec[b].alloc(rbytes)) return fail(DGSWE_ENOMEM, "device allocation of %zu bytes failed", rbytes);
  }
  if (h->geo.alloc(16 * (size_t)h->gv * E) || h->nbr.alloc(16 * (size_t)E) || h->nodes.alloc(16 * (size_t)E) ||
      h->xy64.alloc(16 * (size_t)N) || h->hbn.alloc(8 * (size_t)N) || h->einv.alloc(4 * (size_t)E) ||
      h->node_xy.alloc(mx ? 8 * (size_t)N : 16 * (size_t)N) || h->rain_e.alloc(mx ? 4 * (size_t)E : 8 * (size_t)E) ||
      h->ctl.alloc(sizeof(Ctl)) || h->scen.alloc(sizeof(ScenDev) * ns) || h->grids.alloc(4 * grids.size()) ||
      h->rivers.alloc(8 * rivers.size()) || h->node_scen.alloc(4 * (size_t)N) ||
      h->rain_node.alloc((mx ? 4 : 8) * (size_t)N) ||
      h->scratch.alloc(sizeof(double) * 4 * 4096))
    return fail(DGSWE_ENOMEM, "device allocation failed");
  const std::vector<uint32_t> blk = to_blocked(rec, (size_t)E, (size_t)h->rv);
  CU(cudaMemcpy(h->rec[0].p, blk.data(), rbytes, cudaMemcpyHostToDevice));
  CU(cudaMemset(h->rec[1].p, 0, rbytes));
  CU(cudaMemset(h->rec[2].p, 0, rbytes));
  CU(cudaMemcpy(h->geo.p, geo.data(), 4 * geo.size(), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->nbr.p, nbr.data(), 4 * nbr.size(), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->nodes.p, nodes.data(), 4 * nodes.size(), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->xy64.p, xy64.data(), 8 * xy64.size(), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->hbn.p, hbn.data(), 8 * hbn.size(), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->einv.p, einv.data(), 4 * einv.size(), cudaMemcpyHostToDevice));
  if (h->xy0.alloc(mx ? 8 * (size_t)E : 16 * (size_t)E)) return fail(DGSWE_ENOMEM, "device allocation failed");
  if (mx) CU(cudaMemcpy(h->xy0.p, xy0f.data(), 4 * xy0f.size(), cudaMemcpyHostToDevice));
  else CU(cudaMemcpy(h->xy0.p, xy0d.data(), 8 * xy0d.size(), cudaMemcpyHostToDevice));
  if (mx) {
    CU(cudaMemcpy(h->node_xy.p, xyf.data(), 4 * xyf.size(), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->rain_e.p, rainf.data(), 4 * rainf.size(), cudaMemcpyHostToDevice));
  } else {
    CU(cudaMemcpy(h->node_xy.p, xy64.data(), 8 * xy64.size(), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(h->rain_e.p, rain64.data(), 8 * rain64.size(), cudaMemcpyHostToDevice));
  }
  if (!grids.empty()) CU(cudaMemcpy(h->grids.p, grids.data(), 4 * grids.size(), cudaMemcpyHostToDevice));
  if (!rivers.empty()) CU(cudaMemcpy(h->rivers.p, rivers.data(), 8 * rivers.size(), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->node_scen.p, nscen.data(), 4 * (size_t)N, cudaMemcpyHostToDevice));
  CU(cudaMemset(h->rain_node.p, 0, (mx ? 4 : 8) * (size_t)N));
  if (h->prm.limiter) {
    std::vector<double> limd = limiter_data(h, E);
    if (h->lim.alloc((mx ? 4 : 8) * limd.size())) return fail(DGSWE_ENOMEM, "device allocation failed");
    if (mx) {
      std::vector<float> lf(limd.begin(), limd.end());
      CU(cudaMemcpy(h->lim.p, lf.data(), 4 * lf.size(), cudaMemcpyHostToDevice));
    } else {
      CU(cudaMemcpy(h->lim.p, limd.data(), 8 * limd.size(), cudaMemcpyHostToDevice));
    }
  }
  h->nn_total = N;
  h->grid_rain = false;
  for (size_t s = 0; s < ns; ++s) h->grid_rain = h->grid_rain || h->sc[s].rain_kind == 3;
  CU(cudaMemset(h->ctl.p, 0, sizeof(Ctl)));
  // per-scenario parameter blocks (dt filled in later)
  std::vector<ScenDev> sd(ns);
  for (size_t s = 0; s < ns; ++s) {
    const Scenario& S = h->sc[s];
    ScenDev& D = sd[s];
    std::memset(&D, 0, sizeof D);
    D.t0 = S.t0;
    D.elem_begin = (int32_t)h->eoff[s];
    D.elem_end = (int32_t)(h->eoff[s] + S.m.ne);
    D.rain_kind = S.rain_kind;
    D.gnx = S.gnx; D.gny = S.gny; D.gnt = S.gnt;
    D.grid = S.rain_kind == 3 ? h->grids.as<float>() + grid_off[s] : nullptr;
    D.nseg = (int32_t)S.tamp.size();
    D.rnseg = S.rnseg;
    D.rnt = S.rnt;
    D.rt0 = S.rt0;
    D.ridt = 1.0 / S.rdt;
    D.river = S.rnseg > 0 ? h->rivers.as<double>() + river_off[s] : nullptr;
    D.press = S.press ? 1 : 0;
    const double st[8] = {S.storm.x0, S.storm.y0, S.storm.speed * std::cos(S.storm.heading),
                          S.storm.speed * std::sin(S.storm.heading), S.storm.rpeak, S.storm.rm, S.storm.re, S.storm.t0};
    const double gr[6] = {S.gx0, S.gy0, 1.0 / S.gdx, 1.0 / S.gdy, S.gt0, 1.0 / S.gdt};
    const double ps[4] = {S.ps.x0, S.ps.y0, S.ps.sigma, S.ps.peak};
    for (int k = 0; k < 8; ++k) { D.d.storm[k] = st[k]; D.f.storm[k] = (float)st[k]; }
    D.d.storm[8] = st[5] != 0.0 ? 1.0 / st[5] : 0.0;
    D.d.storm[9] = st[6] != 0.0 ? 1.4426950408889634 / st[6] : 0.0;
    D.f.storm[8] = (float)D.d.storm[8];
    D.f.storm[9] = (float)D.d.storm[9];
    for (int k = 0; k < 6; ++k) { D.d.grid[k] = gr[k]; D.f.grid[k] = (float)gr[k]; }
    for (int k = 0; k < 4; ++k) { D.d.ps[k] = ps[k]; D.f.ps[k] = (float)ps[k]; }
    for (size_t k = 0; k < S.tamp.size() && k < (size_t)MAXSEG; ++k) {
      // FP64: amp sin(omega t + phase); FP32: amp sin(2 pi frac(t / period + phase / (2 pi)))
      D.d.tide[k][0] = S.tamp[k];
      D.d.tide[k][1] = 2.0 * M_PI / S.tper[k];
      D.d.tide[k][2] = S.tpha[k];
      D.f.tide[k][0] = (float)S.tamp[k];
      D.f.tide[k][1] = (float)(1.0 / S.tper[k]);
      D.f.tide[k][2] = (float)(S.tpha[k] / (2.0 * M_PI));
    }
  }
  // scenario of each 32-element tile; ledger slots per scenario cover the widest launch
  h->ntiles = (int)(E / TILE);
  std::vector<int32_t> ts(h->ntiles, 0);
  for (size_t s = 0; s < ns; ++s) {
    const long long t0 = h->eoff[s] / TILE;
    const long long t1 = (h->eoff[s] + (h->sc[s].m.ne + TILE_ALIGN - 1) / TILE_ALIGN * TILE_ALIGN) / TILE;
    for (long long t = t0; t < t1 && t < h->ntiles; ++t) ts[t] = (int32_t)s;
  }
  int sms = 0;
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  h->wslots = sms * 64 * 2;
  std::vector<int32_t> tm(4 * (size_t)h->ntiles, 0);
  for (long long t = 0; t < h->ntiles; ++t) {
    const size_t s = (size_t)ts[t];
    const long long n = h->eoff[s] + h->sc[s].m.ne - t * TILE;
    tm[4 * t] = ts[t];
    tm[4 * t + 1] = (int32_t)std::max(0LL, std::min<long long>(TILE, n));
  }
  if (h->tile_scen.alloc(4 * (size_t)h->ntiles) || h->tile_meta.alloc(16 * (size_t)h->ntiles) ||
      h->ledger.alloc(16 * (size_t)h->wslots * ns))
    return fail(DGSWE_ENOMEM, "device allocation failed");
  CU(cudaMemcpy(h->tile_scen.p, ts.data(), 4 * ts.size(), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(h->tile_meta.p, tm.data(), 4 * tm.size(), cudaMemcpyHostToDevice));
  CU(cudaMemset(h->ledger.p, 0, 16 * (size_t)h->wslots * ns));
  h->wcur = 0;
  CU(cudaMemcpy(h->scen.p, sd.data(), sizeof(ScenDev) * ns, cudaMemcpyHostToDevice));
  h->led_rain.assign(ns, 0.0);
  h->led_bdry.assign(ns, 0.0);
  h->V0.assign(ns, 0.0);
  h->VH0.assign(ns, 0.0);
  h->stages = ssp_table(h->prm.ssp_stages);
  h->feat = run_features(h, nbr);
  return 0;
}

// fill the per-scenario time-step fields once dt is known
static int upload_dt(dgswe_h h) {
  std::vector<ScenDev> sd(h->sc.size());
  CU(cudaMemcpy(sd.data(), h->scen.p, sizeof(ScenDev) * sd.size(), cudaMemcpyDeviceToHost));
  for (size_t s = 0; s < sd.size(); ++s) {
    ScenDev& D = sd[s];
    D.dt = h->sc[s].dt;
    D.d.t0 = D.t0;
    D.d.dt = D.dt;
    D.f.t0 = (float)D.t0;
    D.f.dt = (float)D.dt;
    for (size_t k = 0; k < h->stages.size(); ++k) {
      D.bdt[k] = h->stages[k].beta * D.dt;
      split_ff(D.bdt[k], D.bdt_hi[k], D.bdt_lo[k]);
      D.bw[k] = h->stages[k].bw;
    }
  }
  CU(cudaMemcpy(h->scen.p, sd.data(), sizeof(ScenDev) * sd.size(), cudaMemcpyHostToDevice));
  return 0;
}

// launch shape change: fold the ledger slots of the old shape into the host accumulators
static int fold_ledger(dgswe_h h) {
  if (h->wcur > 0) {
    const size_t ns = h->sc.size();
    std::vector<double> part(2 * (size_t)h->wslots * ns);
    CU(cudaMemcpy(part.data(), h->ledger.p, 8 * part.size(), cudaMemcpyDeviceToHost));
    for (size_t s = 0; s < ns; ++s)
      for (int w = 0; w < h->wcur; ++w) {
        h->led_rain[s] += part[2 * (s * h->wslots + w)];
        h->led_bdry[s] += part[2 * (s * h->wslots + w) + 1];
      }
    CU(cudaMemset(h->ledger.p, 0, 8 * part.size()));
  }
  if (h->g1) { cudaGraphExecDestroy(h->g1); h->g1 = nullptr; }
  if (h->gK) { cudaGraphExecDestroy(h->gK); h->gK = nullptr; }
  return 0;
}

template <class Pol>
static StageArgs<Pol> make_args(dgswe_h h, int stage, int tune) {
  using T = typename PolT<Pol>::T;
  StageArgs<Pol> a;
  std::memset(&a, 0, sizeof a);
  const int S = (int)h->stages.size();
  const Stage& st = h->stages[stage];
  // rec[0] holds w^n (and receives the step's result); stage outputs alternate in rec[1], rec[2]
  a.in = h->rec[stage == 0 ? 0 : 1 + (stage - 1) % 2].as<uint4>();
  a.wn = h->rec[0].as<uint4>();
  a.out = (stage == S - 1) ? h->rec[0].as<uint4>() : h->rec[1 + stage % 2].as<uint4>();
  if (tune) a.out = h->rec[1 + stage % 2].as<uint4>();  // timing runs never overwrite w^n
  a.nbr = h->nbr.as<int4>();
  a.geo = h->geo.as<uint4>();
  a.nodes = h->nodes.as<int4>();
  a.node_xy = h->node_xy.as<T>();
  a.hb_nodal = h->hbn.as<double>();
  a.rain_e = h->rain_e.as<T>();
  a.rain_node = h->rain_node.as<T>();
  a.lim = h->lim.as<T>();
  a.lim_nu = (T)h->prm.lim_nu;
  a.node_scen = h->node_scen.as<int32_t>();
  a.scen = h->scen.as<ScenDev>();
  a.tile_scen = h->tile_scen.as<int32_t>();
  a.tile_meta = h->tile_meta.as<int4>();
  a.xy0 = h->xy0.as<uint4>();
  a.ledger = h->ledger.as<double>();
  a.ctl = h->ctl.as<Ctl>();
  a.edges = h->edges.as<uint4>();
  a.slots = h->slots.as<uint4>();
  a.nedges = h->nedges;
  a.split = h->split;
  a.ntiles = h->ntiles;
  a.wslots = h->wslots;
  a.stage = stage;
  a.last = (stage == S - 1) ? 1 : 0;
  a.has_n = st.a_n != 0.0 ? 1 : 0;
  a.pow2 = (pow2_or_0(st.a_n) && pow2_or_0(st.a_in)) ? 1 : 0;
  a.tune = tune;
  a.friction = h->prm.friction;
  split_ff(st.a_n, a.a_n_hi, a.a_n_lo);
  split_ff(st.a_in, a.a_in_hi, a.a_in_lo);
  a.a_n = st.a_n;
  a.a_in = st.a_in;
  a.cst = st.c;
  a.g = (T)h->prm.g;
  a.H0 = (T)h->prm.H0;
  a.cf = (T)h->prm.cf;
  return a;
}

static int edge_grid(dgswe_h h) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  const long long need = (h->nedges + 255) / 256;
  return (int)std::max<long long>(1, std::min<long long>(need, 16LL * sms));
}

// one Runge-Kutta stage: (edge kernel, when split = 1) then the element kernel (fused, split or
// tile form)
static int launch_stage_once(dgswe_h h, int stage, int tune, cudaStream_t s) {
  const int grid = h->grid;
  cudaError_t e = cudaSuccess;
  if (h->grid_rain) {  // nodal gridded rain at this stage's time
    e = mixed(h) ? launch_node_rain<Mixed>(make_args<Mixed>(h, stage, tune), h->nn_total, s)
                 : launch_node_rain<Fp64>(make_args<Fp64>(h, stage, tune), h->nn_total, s);
    if (e != cudaSuccess) return fail(DGSWE_ECUDA, "node rain launch: %s", cudaGetErrorString(e));
    h->launches++;
  }
  if (h->split == 1 && h->nedges > 0) {
    if (mixed(h)) e = launch_edges<Mixed>(h->prm.p, h->prm.flux, make_args<Mixed>(h, stage, tune), edge_grid(h), 256, s);
    else e = launch_edges<Fp64>(h->prm.p, h->prm.flux, make_args<Fp64>(h, stage, tune), edge_grid(h), 256, s);
    if (e != cudaSuccess) return fail(DGSWE_ECUDA, "edge launch: %s", cudaGetErrorString(e));
    h->launches++;
  }
  if (h->split == 2)
    e = mixed(h) ? launch_tile<Mixed>(h->prm.p, h->prm.flux, h->feat, make_args<Mixed>(h, stage, tune), grid, h->block, s)
                 : launch_tile<Fp64>(h->prm.p, h->prm.flux, h->feat, make_args<Fp64>(h, stage, tune), grid, h->block, s);
  else if (mixed(h))
    e = launch_stage<Mixed>(h->prm.p, h->prm.flux, make_args<Mixed>(h, stage, tune), grid, h->block, s);
  else
    e = launch_stage<Fp64>(h->prm.p, h->prm.flux, make_args<Fp64>(h, stage, tune), grid, h->block, s);
  if (e != cudaSuccess) return fail(DGSWE_ECUDA, "stage launch: %s", cudaGetErrorString(e));
  h->launches++;
  if (h->prm.limiter && !tune) {  // slope limiter on the stage output, then the positive-depth operator
    const long long ne = (long long)h->ntiles * TILE;
    e = mixed(h) ? launch_limiter<Mixed>(make_args<Mixed>(h, stage, tune), ne, s)
                 : launch_limiter<Fp64>(make_args<Fp64>(h, stage, tune), ne, s);
    if (e != cudaSuccess) return fail(DGSWE_ECUDA, "limiter launch: %s", cudaGetErrorString(e));
    h->launches++;
  }
  return 0;
}

static int launches_per_stage(dgswe_h h) {
  return 1 + ((h->split == 1 && h->nedges > 0) ? 1 : 0) + (h->grid_rain ? 1 : 0) + (h->prm.limiter ? 1 : 0);
}

static int occupancy(dgswe_h h, int block) {
  if (h->split == 2)
    return mixed(h) ? tile_blocks_per_sm<Mixed>(h->prm.p, h->prm.flux, h->feat, block)
                    : tile_blocks_per_sm<Fp64>(h->prm.p, h->prm.flux, h->feat, block);
  return mixed(h) ? stage_blocks_per_sm<Mixed>(h->prm.p, h->prm.flux, block, h->split)
                  : stage_blocks_per_sm<Fp64>(h->prm.p, h->prm.flux, block, h->split);
}

// grid = SMs x resident CTAs per SM x waves; its warps take the 32-element tiles round-robin
static int apply_launch(dgswe_h h, int block, int waves, int split) {
  int sms = 0;
  CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
  if (int rc = fold_ledger(h)) return rc;
  h->block = block;
  h->waves = waves;
  h->split = split;
  const int occ = occupancy(h, block);
  if (occ < 1) return fail(DGSWE_EINVAL, "form %d does not fit a block of %d threads on this device", split, block);
  const int want = sms * occ * waves;
  const int need = (h->ntiles + block / 32 - 1) / (block / 32);  // one tile per warp
  h->grid = std::max(1, std::min(want, need));
  h->wcur = h->grid * (block / 32);
  if (h->wcur > h->wslots) return fail(DGSWE_EINVAL, "launch shape needs %d ledger slots, %d allocated", h->wcur, h->wslots);
  return 0;
}

// time whole steps (every stage; timing runs write only the two scratch records) for each form
// (fused, edge kernel + element kernel, tile), block size and number of waves
static int autotune(dgswe_h h) {
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  float best = 1e30f;
  int bb = 128, bp = 0;
  const int blocks[3] = {64, 128, 256};
  int bs = 1;
  for (int sp = 0; sp <= 2; ++sp)
  for (int pi = 1; pi <= 2; ++pi)
    for (int bi = 0; bi < 3; ++bi) {
      h->split = sp;
      if (occupancy(h, blocks[bi]) < 1) continue;
      if (int rc = apply_launch(h, blocks[bi], pi, sp)) return rc;
      const int ns = (int)h->stages.size();
      for (int w = 0; w < 2; ++w)
        for (int st = 0; st < ns; ++st)
          if (int rc = launch_stage_once(h, st, 1, h->stream)) return rc;
      CU(cudaEventRecord(e0, h->stream));
      for (int r = 0; r < 5; ++r)
        for (int st = 0; st < ns; ++st)
          if (int rc = launch_stage_once(h, st, 1, h->stream)) return rc;
      CU(cudaEventRecord(e1, h->stream));
      CU(cudaEventSynchronize(e1));
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) { best = ms; bb = blocks[bi]; bp = pi; bs = sp; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->autotune = false;
  return apply_launch(h, bb, bp, bs);
}

static int build_graphs(dgswe_h h) {
  for (int which = 0; which < 2; ++which) {
    const int nsteps = which == 0 ? 1 : h->K;
    cudaGraph_t g;
    CU(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    int rc = 0;
    for (int k = 0; k < nsteps && !rc; ++k)
      for (size_t s = 0; s < h->stages.size() && !rc; ++s) rc = launch_stage_once(h, (int)s, 0, h->cap);
    cudaError_t ce = cudaStreamEndCapture(h->cap, &g);
    if (rc) return rc;
    if (ce != cudaSuccess) return fail(DGSWE_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
    h->launches -= nsteps * (long long)h->stages.size() * launches_per_stage(h);  // counted when the graph runs
    cudaGraphExec_t ex;
    ce = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return fail(DGSWE_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
    (which == 0 ? h->g1 : h->gK) = ex;
  }
  return 0;
}

static int reduce_volume(dgswe_h h, size_t s, double& V, double& VH) {
  const long long b = h->eoff[s], e = b + h->sc[s].m.ne;
  const int nblk = (int)std::min<long long>(1024, std::max<long long>(1, (e - b + 255) / 256));
  double* part = h->scratch.as<double>();
  cudaError_t ce = mixed(h) ? launch_volume<Mixed>(h->prm.p, h->rec[0].as<uint4>(), h->geo.as<uint4>(), b, e, part, nblk, h->stream)
                            : launch_volume<Fp64>(h->prm.p, h->rec[0].as<uint4>(), h->geo.as<uint4>(), b, e, part, nblk, h->stream);
  if (ce != cudaSuccess) return fail(DGSWE_ECUDA, "volume launch: %s", cudaGetErrorString(ce));
  h->launches++;
  ce = launch_reduce_pairs(part, nblk, 2, part + 4 * 1024, h->stream);
  if (ce != cudaSuccess) return fail(DGSWE_ECUDA, "reduce launch: %s", cudaGetErrorString(ce));
  h->launches++;
  double out[4];
  CU(cudaMemcpyAsync(out, part + 4 * 1024, sizeof out, cudaMemcpyDeviceToHost, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  V = out[0] + out[1];
  VH = out[2] + out[3];
  return 0;
}

// positive-depth operator on the initial state, then dt and the initial volumes
static int prepare(dgswe_h h) {
  DeviceGuard dg_(h->device);
  const double cfl = h->prm.cfl;
  for (size_t s = 0; s < h->sc.size(); ++s) {
    const long long b = h->eoff[s], e = b + h->sc[s].m.ne;
    cudaError_t ce;
    if (mixed(h)) {
      StageArgs<Mixed> a = make_args<Mixed>(h, 0, 1);
      a.in = h->rec[0].as<uint4>();
      a.out = h->rec[0].as<uint4>();
      ce = launch_prepare<Mixed>(h->prm.p, a, b, e, h->stream);
    } else {
      StageArgs<Fp64> a = make_args<Fp64>(h, 0, 1);
      a.in = h->rec[0].as<uint4>();
      a.out = h->rec[0].as<uint4>();
      ce = launch_prepare<Fp64>(h->prm.p, a, b, e, h->stream);
    }
    if (ce != cudaSuccess) return fail(DGSWE_ECUDA, "prepare launch: %s", cudaGetErrorString(ce));
    h->launches++;
    if (h->sc[s].dt <= 0.0) {
      if (h->prm.dt > 0.0) {
        h->sc[s].dt = h->prm.dt;
      } else {
        if (!(cfl > 0.0)) return fail(DGSWE_EINVAL, "neither dt nor cfl is positive");
        const int nblk = (int)std::min<long long>(1024, std::max<long long>(1, (e - b + 255) / 256));
        double* part = h->scratch.as<double>();
        ce = mixed(h) ? launch_dt<Mixed>(h->prm.p, h->rec[0].as<uint4>(), h->nodes.as<int4>(), h->xy64.as<double>(),
                                         h->hbn.as<double>(), b, e, cfl, h->prm.g, h->prm.H0, part, nblk, h->stream)
                      : launch_dt<Fp64>(h->prm.p, h->rec[0].as<uint4>(), h->nodes.as<int4>(), h->xy64.as<double>(),
                                        h->hbn.as<double>(), b, e, cfl, h->prm.g, h->prm.H0, part, nblk, h->stream);
        if (ce != cudaSuccess) return fail(DGSWE_ECUDA, "dt launch: %s", cudaGetErrorString(ce));
        h->launches++;
        std::vector<double> mins(nblk);
        CU(cudaMemcpyAsync(mins.data(), part, 8 * (size_t)nblk, cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        h->sc[s].dt = *std::min_element(mins.begin(), mins.end());
      }
    }
    if (int rc = reduce_volume(h, s, h->V0[s], h->VH0[s])) return rc;
  }
  if (int rc = upload_dt(h)) return rc;
  if (int rc = apply_launch(h, h->block, h->waves, h->split)) return rc;
  CU(cudaStreamSynchronize(h->stream));
  h->ready = true;
  return 0;
}

// ------------------------------------------------------------------------------ C ABI ---
extern "C" {

const char* dgswe_last_error(void) { return g_err.c_str(); }

int dgswe_create(dgswe_h* out, int device, void* cuda_stream) {
  if (!out) return fail(DGSWE_EINVAL, "null output handle");
  *out = nullptr;
  int n = 0;
  cudaError_t ce = cudaGetDeviceCount(&n);
  if (ce != cudaSuccess || n == 0) return fail(DGSWE_ENOLIB, "no CUDA device: %s", cudaGetErrorString(ce));
  if (device < 0 || device >= n) return fail(DGSWE_EINVAL, "device %d outside [0,%d)", device, n);
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
  if (major != 10 || minor != 3)
    return fail(DGSWE_ENOLIB, "device %d is sm_%d%d; this library is built for sm_103a only", device, major, minor);
  std::unique_ptr<dgswe_ctx> h(new dgswe_ctx());
  h->device = device;
  DeviceGuard dg_(device);
  if (cuda_stream) {
    h->stream = (cudaStream_t)cuda_stream;
  } else {
    CU(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  CU(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  *out = h.release();
  return 0;
}

void dgswe_destroy(dgswe_h h) {
  if (!h) return;
  {
    DeviceGuard dg_(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
  }
  delete h;
}

int dgswe_set_params(dgswe_h h, const dgswe_params* p) {
  if (int rc = check_handle(h)) return rc;
  if (!p) return fail(DGSWE_EINVAL, "null params");
  if (p->p < 1 || p->p > 2) return fail(DGSWE_EINVAL, "p = %d: the device path supports p = 1 and p = 2", p->p);
  if (p->flux != DGSWE_FLUX_ROE && p->flux != DGSWE_FLUX_LLF) return fail(DGSWE_EINVAL, "unknown flux %d", p->flux);
  if (p->ssp_stages != 2 && p->ssp_stages != 3 && p->ssp_stages != 5)
    return fail(DGSWE_EINVAL, "ssp_stages must be 2, 3 or 5");
  if (p->precision != DGSWE_FP64 && p->precision != DGSWE_MIXED) return fail(DGSWE_EINVAL, "unknown precision");
  if (!(p->g > 0) || !(p->H0 > 0)) return fail(DGSWE_EINVAL, "g and H0 must be positive");
  if (p->friction < 0 || p->friction > 2) return fail(DGSWE_EINVAL, "unknown friction law");
  if (p->limiter != 0 && p->limiter != 1) return fail(DGSWE_EINVAL, "limiter must be 0 or 1");
  if (p->limiter && p->p != 1) return fail(DGSWE_EINVAL, "the slope limiter is defined for p = 1");
  if (p->limiter && !(p->lim_nu >= 0.0 && p->lim_M >= 0.0)) return fail(DGSWE_EINVAL, "limiter constants must be >= 0");
  if (!h->sc.empty() && h->sc[0].level > 0) return fail(DGSWE_ESTATE, "set_params must precede set_mesh");
  h->prm = *p;
  h->has_params = true;
  return 0;
}

int dgswe_set_mesh(dgswe_h h, int32_t n_nodes, const double* xy, int32_t n_tri, const int32_t* tri, int32_t n_bedge,
                   const int32_t* bedge, const int32_t* btype, const int32_t* bseg) {
  if (int rc = check_handle(h)) return rc;
  if (!h->has_params) return fail(DGSWE_ESTATE, "set_params must precede set_mesh");
  if (h->ensemble) return fail(DGSWE_ESTATE, "an ensemble's members are fixed");
  Scenario S;
  std::string err;
  int rc = build_mesh(n_nodes, xy, n_tri, tri, n_bedge, bedge, btype, bseg, S.m, err);
  if (rc) return fail(rc, "%s", err.c_str());
  S.level = 1;
  h->sc.clear();
  h->sc.push_back(std::move(S));
  h->ready = false;
  return 0;
}

static Scenario* scen_at(dgswe_h h, int level) {
  if (h->sc.empty() || h->sc[0].level < level || h->ensemble) return nullptr;
  return &h->sc[0];
}

int dgswe_set_fields(dgswe_h h, const double* hb, const double* man, int32_t manning_nodal) {
  if (int rc = check_handle(h)) return rc;
  Scenario* S = scen_at(h, 1);
  if (!S) return fail(DGSWE_ESTATE, "set_mesh must precede set_fields");
  if (!hb) return fail(DGSWE_EINVAL, "null bathymetry");
  const HostMesh& M = S->m;
  S->hb.resize(M.nn);
  for (int i = 0; i < M.nn; ++i) {
    S->hb[i] = hb[M.norig[i]];
    if (!std::isfinite(S->hb[i])) return fail(DGSWE_EINVAL, "non-finite bathymetry at node %d", M.norig[i]);
  }
  S->man.assign(M.ne, 0.0);
  if (man) {
    for (int e = 0; e < M.ne; ++e) {
      if (manning_nodal) {
        const int32_t* v = &M.tri[3 * (size_t)e];
        S->man[e] = (man[M.norig[v[0]]] + man[M.norig[v[1]]] + man[M.norig[v[2]]]) / 3.0;
      } else {
        S->man[e] = man[M.eorig[e]];
      }
    }
  } else if (h->prm.friction == DGSWE_MANNING) {
    return fail(DGSWE_EINVAL, "Manning friction needs a Manning field");
  }
  S->level = std::max(S->level, 2);
  h->ready = false;
  return 0;
}

int dgswe_set_rain_nodal(dgswe_h h, const double* r) {
  if (int rc = check_handle(h)) return rc;
  Scenario* S = scen_at(h, 1);
  if (!S) return fail(DGSWE_ESTATE, "set_mesh must precede the rain source");
  if (!r) return fail(DGSWE_EINVAL, "null rain");
  S->rain_n.resize(S->m.nn);
  for (int i = 0; i < S->m.nn; ++i) S->rain_n[i] = r[S->m.norig[i]];
  S->rain_kind = 1;
  h->ready = false;
  return 0;
}

int dgswe_set_rain_parametric(dgswe_h h, const dgswe_storm* st) {
  if (int rc = check_handle(h)) return rc;
  Scenario* S = scen_at(h, 1);
  if (!S) return fail(DGSWE_ESTATE, "set_mesh must precede the rain source");
  if (!st || !(st->rm > 0) || !(st->re > 0)) return fail(DGSWE_EINVAL, "storm radii must be positive");
  S->storm = *st;
  S->rain_kind = 2;
  h->ready = false;
  return 0;
}

int dgswe_set_rain_grid(dgswe_h h, int32_t nx, int32_t ny, int32_t nt, double x0, double y0, double dx, double dy,
                        double t0, double dt_rec, const float* mmh) {
  if (int rc = check_handle(h)) return rc;
  Scenario* S = scen_at(h, 1);
  if (!S) return fail(DGSWE_ESTATE, "set_mesh must precede the rain source");
  if (nx < 1 || ny < 1 || nt < 1 || !(dx > 0) || !(dy > 0) || !(dt_rec > 0) || !mmh)
    return fail(DGSWE_EINVAL, "bad rain grid");
  S->gnx = nx; S->gny = ny; S->gnt = nt; S->gx0 = x0; S->gy0 = y0; S->gdx = dx; S->gdy = dy; S->gt0 = t0; S->gdt = dt_rec;
  S->grid.assign(mmh, mmh + (size_t)nx * ny * nt);
  S->rain_kind = 3;
  h->ready = false;
  return 0;
}

int dgswe_set_tide(dgswe_h h, int32_t n, const double* amp, const double* per, const double* pha) {
  if (int rc = check_handle(h)) return rc;
  Scenario* S = scen_at(h, 1);
  if (!S) return fail(DGSWE_ESTATE, "set_mesh must precede set_tide");
  if (n < 0 || n > MAXSEG || (n > 0 && (!amp || !per || !pha))) return fail(DGSWE_EINVAL, "at most %d tidal segments", MAXSEG);
  for (int k = 0; k < n; ++k)
    if (!(per[k] > 0)) return fail(DGSWE_EINVAL, "tidal period must be positive");
  S->tamp.assign(amp, amp + n);
  S->tper.assign(per, per + n);
  S->tpha.assign(pha, pha + n);
  h->ready = false;
  return 0;
}

int dgswe_set_river(dgswe_h h, int32_t n, int32_t nt, double t0, double dt_rec, const double* q) {
  if (int rc = check_handle(h)) return rc;
  Scenario* S = scen_at(h, 1);
  if (!S) return fail(DGSWE_ESTATE, "set_mesh must precede set_river");
  if (n < 1 || n > MAXRIV || nt < 1 || !q) return fail(DGSWE_EINVAL, "river: 1 to %d segments and at least one record", MAXRIV);
  if (nt > 1 && !(dt_rec > 0)) return fail(DGSWE_EINVAL, "river: record interval must be positive");
  if (!std::isfinite(t0)) return fail(DGSWE_EINVAL, "river: non-finite t0");
  for (size_t k = 0; k < (size_t)n * nt; ++k)
    if (!std::isfinite(q[k])) return fail(DGSWE_EINVAL, "river: non-finite discharge");
  S->rnseg = n;
  S->rnt = nt;
  S->rt0 = t0;
  S->rdt = nt > 1 ? dt_rec : 1.0;
  S->river.assign(q, q + (size_t)n * nt);
  h->ready = false;
  return 0;
}

int dgswe_set_pressure_setup(dgswe_h h, const dgswe_gauss_setup* ps) {
  if (int rc = check_handle(h)) return rc;
  Scenario* S = scen_at(h, 1);
  if (!S) return fail(DGSWE_ESTATE, "set_mesh must precede set_pressure_setup");
  if (ps && !(ps->sigma > 0)) return fail(DGSWE_EINVAL, "sigma must be positive");
  S->press = ps != nullptr;
  if (ps) S->ps = *ps;
  h->ready = false;
  return 0;
}

int dgswe_set_state(dgswe_h h, const double* zeta, const double* qx, const double* qy, int32_t layout, double t0) {
  if (int rc = check_handle(h)) return rc;
  Scenario* S = scen_at(h, 2);
  if (!S) return fail(DGSWE_ESTATE, "set_fields must precede set_state");
  if (!zeta || !qx || !qy) return fail(DGSWE_EINVAL, "null state array");
  const int p = h->prm.p, np = np_of(p);
  const HostMesh& M = S->m;
  if (M.nseg > (int)S->tamp.size()) return fail(DGSWE_EINVAL, "ocean edges use %d tidal segments, %zu given", M.nseg, S->tamp.size());
  if (M.nriv > S->rnseg) return fail(DGSWE_EINVAL, "river edges use %d river segments, %d given", M.nriv, S->rnseg);
  S->w.assign((size_t)M.ne * 3 * np, 0.0);
  const double* f[3] = {zeta, qx, qy};
  if (layout == DGSWE_LAYOUT_MODAL) {
    for (int e = 0; e < M.ne; ++e)
      for (int v = 0; v < 3; ++v)
        for (int m = 0; m < np; ++m) S->w[((size_t)e * 3 + v) * np + m] = f[v][(size_t)m * M.ne + M.eorig[e]];
  } else if (layout == DGSWE_LAYOUT_NODAL) {
    if (!g_tab_built[p]) {
      build_tables(p, g_tabd[p]);
      tables_to_float(g_tabd[p], g_tabf[p]);
      g_tab_built[p] = true;
    }
    const RefTab<double>& tb = g_tabd[p];
    for (int e = 0; e < M.ne; ++e) {
      const int32_t* vt = &M.tri[3 * (size_t)e];
      for (int v = 0; v < 3; ++v) {
        const double fv[3] = {f[v][M.norig[vt[0]]], f[v][M.norig[vt[1]]], f[v][M.norig[vt[2]]]};
        for (int m = 0; m < np; ++m) {  // projection of the linear interpolant (exact rule)
          double s = 0.0;
          for (int q = 0; q < tb.nq; ++q)
            s += tb.qw[q] * (tb.ql[q][0] * fv[0] + tb.ql[q][1] * fv[1] + tb.ql[q][2] * fv[2]) * tb.qphi[q][m];
          S->w[((size_t)e * 3 + v) * np + m] = s;
        }
      }
    }
  } else {
    return fail(DGSWE_EINVAL, "unknown layout %d", layout);
  }
  for (double v : S->w)
    if (!std::isfinite(v)) return fail(DGSWE_EINVAL, "non-finite initial state");
  S->t0 = t0;
  S->dt = 0.0;
  S->level = 3;
  h->ready = false;
  if (int rc = build_layout(h)) return rc;
  return prepare(h);
}

int dgswe_step(dgswe_h h, int64_t n) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "set_state must precede step");
  if (n < 0) return fail(DGSWE_EINVAL, "negative step count");
  if (n == 0) return 0;
  DeviceGuard dg_(h->device);
  if (h->autotune)
    if (int rc = autotune(h)) return rc;
  if (!h->graphs) {  // every stage launched directly
    for (int64_t i = 0; i < n; ++i)
      for (size_t s = 0; s < h->stages.size(); ++s)
        if (int rc = launch_stage_once(h, (int)s, 0, h->stream)) return rc;
    return 0;
  }
  if (!h->g1)
    if (int rc = build_graphs(h)) return rc;
  const long long per = (long long)h->stages.size() * launches_per_stage(h);
  for (int64_t i = 0; i < n / h->K; ++i) CU(cudaGraphLaunch(h->gK, h->stream));
  for (int64_t i = 0; i < n % h->K; ++i) CU(cudaGraphLaunch(h->g1, h->stream));
  h->launches += n * per;
  return 0;
}

int dgswe_set_graphs(dgswe_h h, int32_t on) {
  if (int rc = check_handle(h)) return rc;
  if (on != 0 && on != 1) return fail(DGSWE_EINVAL, "graphs must be 0 or 1");
  h->graphs = on != 0;
  return 0;
}

int dgswe_sync(dgswe_h h) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return 0;
  DeviceGuard dg_(h->device);
  CU(cudaStreamSynchronize(h->stream));
  Ctl c;
  CU(cudaMemcpy(&c, h->ctl.p, sizeof c, cudaMemcpyDeviceToHost));
  if (c.err & ERR_NONFINITE) return fail(DGSWE_ENONFINITE, "a stage produced a non-finite state");
  if (c.err & ERR_NEGDEPTH) return fail(DGSWE_ENEGDEPTH, "an element mean depth fell below zero");
  if (c.err & ERR_TIMEOUT) return fail(DGSWE_ETIMEOUT, "a bulk copy into shared memory did not complete");
  return 0;
}

int dgswe_get_dt(dgswe_h h, double* dt) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready || !dt) return fail(DGSWE_ESTATE, "no state");
  *dt = h->sc[0].dt;
  return 0;
}

static int gather_state(dgswe_h h, size_t s, double* z, double* x, double* y, bool device_out) {
  DeviceGuard dg_(h->device);
  const long long n = h->sc[s].m.ne, b = h->eoff[s];
  const size_t cnt = (size_t)h->np * n;
  double *dz = z, *dx = x, *dy = y;
  bool staged = false;
  if (!device_out) {
    // page-locked host arrays are written directly by the gather kernel (coalesced, over the
    // host link); other host memory goes through a device staging buffer and three copies
    const void *mz = host_mapped(z), *mx = host_mapped(x), *my = host_mapped(y);
    if (mz && mx && my) {
      dz = (double*)mz;
      dx = (double*)mx;
      dy = (double*)my;
    } else {
      staged = true;
      if (h->gather_buf.n < 3 * cnt * sizeof(double))
        if (h->gather_buf.alloc(3 * cnt * sizeof(double))) return fail(DGSWE_ENOMEM, "gather buffer");
      dz = h->gather_buf.as<double>();
      dx = dz + cnt;
      dy = dx + cnt;
    }
  }
  cudaError_t ce = mixed(h) ? launch_gather<Mixed>(h->prm.p, h->rec[0].as<uint4>(), b, n, h->einv.as<int32_t>() + b, dz, dx, dy, h->stream)
                            : launch_gather<Fp64>(h->prm.p, h->rec[0].as<uint4>(), b, n, h->einv.as<int32_t>() + b, dz, dx, dy, h->stream);
  if (ce != cudaSuccess) return fail(DGSWE_ECUDA, "gather launch: %s", cudaGetErrorString(ce));
  h->launches++;
  if (!device_out && !staged) {
    CU(cudaStreamSynchronize(h->stream));
  } else if (!device_out) {
    CU(cudaMemcpyAsync(z, dz, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(x, dx, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaMemcpyAsync(y, dy, cnt * 8, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  return 0;
}

// after records [b, b + n) received a state: their mean depths and wet/dry flags from it, the
// state kept as given (positive-depth pass in classify mode)
static cudaError_t classify_loaded(dgswe_h h, long long b, long long n) {
  if (mixed(h)) {
    StageArgs<Mixed> a = make_args<Mixed>(h, 0, 1);
    a.in = a.out = h->rec[0].as<uint4>();
    a.classify_only = 1;
    return launch_prepare<Mixed>(h->prm.p, a, b, b + n, h->stream);
  }
  StageArgs<Fp64> a = make_args<Fp64>(h, 0, 1);
  a.in = a.out = h->rec[0].as<uint4>();
  a.classify_only = 1;
  return launch_prepare<Fp64>(h->prm.p, a, b, b + n, h->stream);
}

int dgswe_get_state(dgswe_h h, double* z, double* x, double* y) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "no state");
  if (!z || !x || !y) return fail(DGSWE_EINVAL, "null output");
  if (h->ensemble) return fail(DGSWE_EINVAL, "use dgswe_ensemble_get_state");
  return gather_state(h, 0, z, x, y, false);
}

int dgswe_get_state_device(dgswe_h h, double* z, double* x, double* y) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "no state");
  if (!z || !x || !y) return fail(DGSWE_EINVAL, "null output");
  if (h->ensemble) return fail(DGSWE_EINVAL, "use dgswe_ensemble_get_state");
  return gather_state(h, 0, z, x, y, true);
}

int dgswe_exchange_state(dgswe_h h, const double* zi, const double* xi, const double* yi, double* zo, double* xo,
                         double* yo) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "set_state must precede exchange_state");
  if (!zi || !xi || !yi || !zo || !xo || !yo) return fail(DGSWE_EINVAL, "null state array");
  if (h->ensemble) return fail(DGSWE_EINVAL, "not available on an ensemble");
  DeviceGuard dg_(h->device);
  const void* m[6] = {host_mapped(zi), host_mapped(xi), host_mapped(yi), host_mapped(zo), host_mapped(xo), host_mapped(yo)};
  bool direct = true;
  for (const void* q : m) direct = direct && q != nullptr;
  if (!direct) {  // some array is not page-locked: the state out, then in, through the staged paths
    if (int rc = gather_state(h, 0, zo, xo, yo, false)) return rc;
    if (int rc = dgswe_load_state(h, zi, xi, yi)) return rc;
    CU(cudaStreamSynchronize(h->stream));
    return 0;
  }
  const long long n = h->sc[0].m.ne, b = h->eoff[0];
  const double *dzi = (const double*)m[0], *dxi = (const double*)m[1], *dyi = (const double*)m[2];
  double *dzo = (double*)m[3], *dxo = (double*)m[4], *dyo = (double*)m[5];
  const int32_t* inv = h->einv.as<int32_t>() + b;
  cudaError_t ce = mixed(h) ? launch_exchange<Mixed>(h->prm.p, h->rec[0].as<uint4>(), b, n, inv, dzi, dxi, dyi, dzo, dxo, dyo, h->stream)
                            : launch_exchange<Fp64>(h->prm.p, h->rec[0].as<uint4>(), b, n, inv, dzi, dxi, dyi, dzo, dxo, dyo, h->stream);
  if (ce == cudaSuccess) ce = classify_loaded(h, b, n);
  if (ce != cudaSuccess) return fail(DGSWE_ECUDA, "exchange_state launch: %s", cudaGetErrorString(ce));
  h->launches += 2;
  CU(cudaStreamSynchronize(h->stream));
  return 0;
}

int dgswe_load_state(dgswe_h h, const double* z, const double* x, const double* y) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "set_state must precede load_state");
  if (!z || !x || !y) return fail(DGSWE_EINVAL, "null state array");
  if (h->ensemble) return fail(DGSWE_EINVAL, "not available on an ensemble");
  DeviceGuard dg_(h->device);
  const long long n = h->sc[0].m.ne, b = h->eoff[0];
  const size_t cnt = (size_t)h->np * n;
  // page-locked host arrays are read directly by the scatter kernel (coalesced, over the host
  // link) and the call returns at once; other memory is staged through three copies first
  const void *mz = host_mapped(z), *mx = host_mapped(x), *my = host_mapped(y);
  const bool direct = mz && mx && my;
  const double *sz, *sx, *sy;
  if (direct) {
    sz = (const double*)mz;
    sx = (const double*)mx;
    sy = (const double*)my;
  } else {
    if (h->gather_buf.n < 3 * cnt * sizeof(double))
      if (h->gather_buf.alloc(3 * cnt * sizeof(double))) return fail(DGSWE_ENOMEM, "staging buffer");
    double* dz = h->gather_buf.as<double>();
    CU(cudaMemcpyAsync(dz, z, cnt * 8, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(dz + cnt, x, cnt * 8, cudaMemcpyHostToDevice, h->stream));
    CU(cudaMemcpyAsync(dz + 2 * cnt, y, cnt * 8, cudaMemcpyHostToDevice, h->stream));
    sz = dz;
    sx = dz + cnt;
    sy = dz + 2 * cnt;
  }
  cudaError_t ce = mixed(h) ? launch_scatter<Mixed>(h->prm.p, h->rec[0].as<uint4>(), b, n, h->einv.as<int32_t>() + b, sz, sx, sy, h->stream)
                            : launch_scatter<Fp64>(h->prm.p, h->rec[0].as<uint4>(), b, n, h->einv.as<int32_t>() + b, sz, sx, sy, h->stream);
  if (ce == cudaSuccess) ce = classify_loaded(h, b, n);
  if (ce != cudaSuccess) return fail(DGSWE_ECUDA, "load_state launch: %s", cudaGetErrorString(ce));
  h->launches += 2;
  if (!direct) CU(cudaStreamSynchronize(h->stream));
  return 0;
}

int dgswe_record_bytes(dgswe_h h, uint64_t* bytes) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "set_state must precede record_bytes");
  if (!bytes) return fail(DGSWE_EINVAL, "null output");
  *bytes = 3 * record_stride(16 * (size_t)h->rv * h->E);
  return 0;
}

int dgswe_bind_device(dgswe_h h, void* dev, uint64_t bytes) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "set_state must precede bind_device");
  DeviceGuard dg_(h->device);
  const size_t rbytes = 16 * (size_t)h->rv * h->E, st = record_stride(rbytes);
  if (dev) {
    if (bytes < 3 * st) return fail(DGSWE_EINVAL, "bind_device: %llu bytes given, %zu needed", (unsigned long long)bytes, 3 * st);
    if ((uintptr_t)dev % 256 != 0) return fail(DGSWE_EINVAL, "bind_device: the memory must be 256-byte aligned");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, dev) != cudaSuccess || at.type != cudaMemoryTypeDevice || at.device != h->device) {
      cudaGetLastError();
      return fail(DGSWE_EINVAL, "bind_device: not device memory of device %d", h->device);
    }
  }
  CU(cudaStreamSynchronize(h->stream));
  if (int rc = fold_ledger(h)) return rc;  // the captured graphs name the old buffers
  // the state w^n moves to the new home; the two stage buffers need no contents
  DevBuf keep;
  keep.bind(h->rec[0].p, h->rec[0].n);
  keep.own = h->rec[0].own;
  h->rec[0].own = false;  // handed to keep, freed (if owned) after the copy
  if (dev) {
    char* base = static_cast<char*>(dev);
    for (int b = 0; b < 3; ++b) {
      if (b > 0) h->rec[b].release();
      h->rec[b].bind(base + b * st, rbytes);
    }
  } else {
    for (int b = 0; b < 3; ++b)
      if (h->rec[b].alloc(rbytes)) return fail(DGSWE_ENOMEM, "device allocation of %zu bytes failed", rbytes);
  }
  CU(cudaMemcpyAsync(h->rec[0].p, keep.p, rbytes, cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaStreamSynchronize(h->stream));
  h->bound = static_cast<char*>(dev);
  h->bound_bytes = dev ? bytes : 0;
  return 0;
}

int dgswe_get_dry(dgswe_h h, uint8_t* dry) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "no state");
  if (!dry) return fail(DGSWE_EINVAL, "null output");
  DeviceGuard dg_(h->device);
  const HostMesh& M = h->sc[0].m;
  const size_t rw = 4 * (size_t)h->rv;
  std::vector<uint32_t> rec(rw * ((size_t)(M.ne + TILE - 1) / TILE * TILE));  // whole tiles
  CU(cudaStreamSynchronize(h->stream));
  CU(cudaMemcpy(rec.data(), h->rec[0].p, 4 * rec.size(), cudaMemcpyDeviceToHost));
  const int NS = h->np - 1;
  const size_t off = mixed(h) ? (size_t)(6 + 3 * NS + 1) : (size_t)2 * (3 + 3 * NS + 1);
  for (int e = 0; e < M.ne; ++e) dry[M.eorig[e]] = (rec_word(rec, e, off, h->rv) & FLAG_DRY) ? 1 : 0;
  return 0;
}

static int ledger_of(dgswe_h h, size_t s, dgswe_ledger* out) {
  DeviceGuard dg_(h->device);
  CU(cudaStreamSynchronize(h->stream));
  double V, VH;
  if (int rc = reduce_volume(h, s, V, VH)) return rc;
  (void)VH;
  Ctl c;
  CU(cudaMemcpy(&c, h->ctl.p, sizeof c, cudaMemcpyDeviceToHost));
  std::vector<double> part(2 * (size_t)h->wcur);
  CU(cudaMemcpy(part.data(), h->ledger.as<double>() + 2 * (size_t)s * h->wslots, 16 * (size_t)h->wcur,
                cudaMemcpyDeviceToHost));
  double rs = h->led_rain[s], rc_ = 0.0, bs = h->led_bdry[s], bc = 0.0;
  auto neu = [](double& sum, double& comp, double v) {
    const double t = sum + v;
    comp += (std::fabs(sum) >= std::fabs(v)) ? (sum - t) + v : (v - t) + sum;
    sum = t;
  };
  for (int w = 0; w < h->wcur; ++w) {
    neu(rs, rc_, part[2 * w]);
    neu(bs, bc, part[2 * w + 1]);
  }
  out->steps = (int64_t)c.step;
  out->t = h->sc[s].t0 + (double)c.step * h->sc[s].dt;
  out->V0 = h->V0[s];
  out->V = V;
  out->rain_in = rs + rc_;
  out->bdry_in = bs + bc;
  out->VH0 = h->VH0[s];
  out->rel_err = std::fabs(V - h->V0[s] - out->rain_in - out->bdry_in) / h->VH0[s];
  // wet fraction from the dry flags
  const HostMesh& M = h->sc[s].m;
  const size_t rw = 4 * (size_t)h->rv;
  std::vector<uint32_t> rec(rw * ((size_t)(M.ne + TILE - 1) / TILE * TILE));  // whole tiles
  CU(cudaMemcpy(rec.data(), h->rec[0].as<uint32_t>() + rw * h->eoff[s], 4 * rec.size(), cudaMemcpyDeviceToHost));
  const int NS = h->np - 1;
  const size_t off = mixed(h) ? (size_t)(6 + 3 * NS + 1) : (size_t)2 * (3 + 3 * NS + 1);
  long long wet = 0;
  for (int e = 0; e < M.ne; ++e) wet += (rec_word(rec, e, off, h->rv) & FLAG_DRY) ? 0 : 1;
  out->wet_frac = (double)wet / M.ne;
  return 0;
}

int dgswe_get_ledger(dgswe_h h, dgswe_ledger* out) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "no state");
  if (!out) return fail(DGSWE_EINVAL, "null output");
  return ledger_of(h, 0, out);
}

int dgswe_volume(dgswe_h h, double* out) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "no state");
  if (!out) return fail(DGSWE_EINVAL, "null output");
  DeviceGuard dg_(h->device);
  double VH;
  return reduce_volume(h, 0, *out, VH);
}

int dgswe_ensemble_create(dgswe_h* out, int32_t n, const dgswe_h* members, int device, void* stream) {
  if (!out) return fail(DGSWE_EINVAL, "null output handle");
  *out = nullptr;
  if (n < 1 || !members) return fail(DGSWE_EINVAL, "empty ensemble");
  for (int i = 0; i < n; ++i) {
    if (!members[i] || !members[i]->ready || members[i]->ensemble)
      return fail(DGSWE_ESTATE, "member %d has no state", i);
    const dgswe_params& a = members[0]->prm;
    const dgswe_params& b = members[i]->prm;
    if (a.p != b.p || a.flux != b.flux || a.ssp_stages != b.ssp_stages || a.precision != b.precision || a.g != b.g ||
        a.H0 != b.H0 || a.friction != b.friction || a.cf != b.cf || a.limiter != b.limiter ||
        a.lim_nu != b.lim_nu || a.lim_M != b.lim_M)
      return fail(DGSWE_EINVAL, "member %d differs in p, flux, ssp_stages, precision, g, H0 or friction", i);
  }
  dgswe_h h = nullptr;
  if (int rc = dgswe_create(&h, device, stream)) return rc;
  h->prm = members[0]->prm;
  h->has_params = true;
  h->ensemble = true;
  for (int i = 0; i < n; ++i) h->sc.push_back(members[i]->sc[0]);
  int rc = build_layout(h);
  if (!rc) rc = prepare(h);
  if (rc) {
    dgswe_destroy(h);
    return rc;
  }
  *out = h;
  return 0;
}

int dgswe_ensemble_step(dgswe_h ens, int64_t n) {
  if (int rc = check_handle(ens)) return rc;
  if (!ens->ensemble) return fail(DGSWE_EINVAL, "not an ensemble");
  return dgswe_step(ens, n);
}

int dgswe_ensemble_get_state(dgswe_h ens, int32_t i, double* z, double* x, double* y) {
  if (int rc = check_handle(ens)) return rc;
  if (!ens->ensemble || i < 0 || i >= (int)ens->sc.size()) return fail(DGSWE_EINVAL, "bad member index");
  if (!z || !x || !y) return fail(DGSWE_EINVAL, "null output");
  return gather_state(ens, (size_t)i, z, x, y, false);
}

int dgswe_ensemble_get_ledger(dgswe_h ens, int32_t i, dgswe_ledger* out) {
  if (int rc = check_handle(ens)) return rc;
  if (!ens->ensemble || i < 0 || i >= (int)ens->sc.size()) return fail(DGSWE_EINVAL, "bad member index");
  if (!out) return fail(DGSWE_EINVAL, "null output");
  return ledger_of(ens, (size_t)i, out);
}

int dgswe_set_launch(dgswe_h h, int32_t block, int32_t waves, int32_t split) {
  if (int rc = check_handle(h)) return rc;
  if (block != 0 && block != 64 && block != 128 && block != 256) return fail(DGSWE_EINVAL, "block must be 0, 64, 128 or 256");
  if (block == 0) {
    h->autotune = true;
    return 0;
  }
  if (waves < 1 || waves > 2) return fail(DGSWE_EINVAL, "waves must be 1 or 2");
  if (split < 0 || split > 2) return fail(DGSWE_EINVAL, "split must be 0, 1 or 2");
  h->autotune = false;
  if (!h->ready) {
    h->block = block;
    h->waves = waves;
    h->split = split;
    return 0;
  }
  DeviceGuard dg_(h->device);
  CU(cudaStreamSynchronize(h->stream));
  return apply_launch(h, block, waves, split);
}

int dgswe_get_launch(dgswe_h h, int32_t* block, int32_t* waves, int32_t* split) {
  if (int rc = check_handle(h)) return rc;
  if (block) *block = h->block;
  if (waves) *waves = h->waves;
  if (split) *split = h->split;
  return 0;
}

int dgswe_get_tile_features(dgswe_h h, int32_t* run, int32_t* kernel) {
  if (int rc = check_handle(h)) return rc;
  if (!h->ready) return fail(DGSWE_ESTATE, "no state");
  if (run) *run = h->feat;
  if (kernel) {
    const int ft = mixed(h) ? tile_spec_features(h->prm.p, h->prm.flux, h->feat) : -1;
    *kernel = ft >= 0 ? ft : FT_ALL;
  }
  return 0;
}

int64_t dgswe_launch_count(dgswe_h h) { return h ? h->launches : 0; }

}  // extern "C"
