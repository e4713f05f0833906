/*
 * dgswe_oracle.c -- plain, slow, FP64 CPU reference ("oracle") of the discontinuous Galerkin
 * finite element method for the rainfall-augmented shallow water equations of Wichitrnithed,
 * Valseth, Kubatko, Kang, Hudson and Dawson, arXiv 2307.14302.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's CPU-baseline leg
 * load this library.  It shares no code, header, table or constant generator with the CUDA
 * library: its own basis, quadrature, mesh connectivity and geometry are built here.
 *
 * What it computes, in the paper's order (Sec. 2.2-2.4):
 *   Eq. SWE             mass: d(zeta)/dt + div(q) = R; momentum with flux q q/H + g/2 (H^2-hb^2) I,
 *                       balance term g zeta grad(hb), friction -tau_b q, forcing F.
 *   Eq. elem_weak_form  (dw/dt, v) - (grad v, F) + <Fhat.n, v> = (s, v), element by element.
 *   Eq. dubiner         modal orthonormal Dubiner basis, diagonal mass matrix M = detJ * I.
 *   Sec. 2.3            edge integrals first (elevation-specified, land, then inner edges), then
 *                       forcing (nodal rain), then area integrals.
 *   Eq. rain            element rain = mean of the three nodal rain rates.
 *   Eq. RKSSP           dw/dt = L_h(w), advanced by Shu-Osher SSP Runge-Kutta.
 *   Sec. 2.4            positive-depth operator M Pi_h = (M Pi^d, M Pi^f) after every stage.
 *
 * Readings of points the paper leaves open (each also listed in the design notes):
 *   - pressure flux is g/2 (H^2 - hb^2) (Eq. SWE); the flux-matrix display drops the 1/2; it is
 *     evaluated as g/2 zeta (zeta + 2 hb), the same value with H = zeta + hb (Sec. 2.1);
 *   - Manning: tau_b = g n^2 |u| / H^{4/3}; quadratic (bathtub, Sec. 3.1): tau_b = Cf |u| / H;
 *     velocities and celerities use Hs = max(H, H0);
 *   - Roe flux with Roe averages (arithmetic Hs, sqrt(Hs)-weighted velocity), no entropy fix;
 *     LLF with the larger of |u.n| + sqrt(g Hs) over both sides; the jump is in (zeta, q);
 *   - ghost states: land mirrors q.n and carries zero mass flux; ocean takes zeta = tide(t)
 *     with the interior q; river edges (Eq. river_bc) carry exactly the prescribed normal
 *     discharge as the mass component of the flux, and the momentum components of the
 *     numerical flux between the interior trace and the ghost (zeta, -q_river n); an interior
 *     edge listed as a river edge is an internal river boundary (Sec. 2.3): the river enters the
 *     element to the left of the listed direction a -> b and the element on the other side sees
 *     a wall (an interior land edge is a wall on both sides); "exact" boundaries (verification
 *     only) take a prescribed field;
 *   - bathymetry is continuous and piecewise linear from nodal values;
 *   - area rule exact to degree 2p+1 (p=1: 7-point degree 3; p=2: 7-point degree 5), edge
 *     rule Gauss-Legendre with p+1 points;
 *   - SSP(2,2) and SSP(3,3) in Shu-Osher form (SSP(1,1) for the finite-volume check); the
 *     five-stage scheme of the production runs (Sec. 3) as the optimal five-stage second-order
 *     SSP method, its DG-optimised coefficients not being given;
 *   - M Pi^d case 3 lifts the lowest vertex to H0 and takes the deficit evenly from the other
 *     two, or lifts the middle one too when that would push it below H0;  a vertex is dry
 *     when its updated depth is below H0 and all three are dry in case 2;  M Pi^f zeroes dry
 *     vertex momentum and spreads it evenly over the wet ones (all dry: momentum lost);
 *     the element mean is never touched, the linear part is rebuilt from vertex values;
 *     at p=2 the operator acts on the linear part (modes 0..2) and the quadratic modes are
 *     scaled by theta = clamp((Hmin - H0) / H0, 0, 1), Hmin the smallest vertex depth of the
 *     linear part: untouched when Hmin >= 2 H0, removed when Hmin <= H0, blended between, so
 *     the result depends continuously on the state (no knife-edge switch at H0);
 *   - an element is dry when any vertex is dry; a dry element keeps receiving rain and edge
 *     inflow but its momentum right-hand side is zero; an edge whose total mass flux would
 *     leave a dry element is closed (each side sees a wall built from its own state);
 *   - dt = CFL * min_e(2 r_in) / ((2p+1) max_vertices(|u| + sqrt(g Hs))) at t = 0.
 */
#include "dgswe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NPMAX 6
#define NQMAX 7
#define NGMAX 3

struct orc {
  int p, np, flux, nstage, friction;
  double g, H0, cf, dt, t;
  long nstep;
  double alpha[5][5], beta[5], cst[5], bw[5];
  /* mesh */
  int nn, ne, ned;
  double *x, *y;
  int32_t* tri;
  int *edn, *ede, *edj, *edt, *eds, *order;
  double *det, *rx, *ry, *sx, *sy, *area, *hb, *man;
  /* reference tables */
  int nq, ng;
  double lq[NQMAX][3], qw[NQMAX];
  double phq[NQMAX][NPMAX], phr[NQMAX][NPMAX], phs[NQMAX][NPMAX];
  double gxi[NGMAX], gw[NGMAX];
  double le[3][NGMAX][3];          /* barycentrics of edge j, point k (param from vertex j to j+1) */
  double phe[3][NGMAX][NPMAX];     /* basis at those points */
  double phv[3][NPMAX];            /* basis at the three vertices */
  /* forcing */
  int rain_kind;
  double* rain_nodal;
  double st[8];
  int gnx, gny, gnt;
  double gx0, gy0, gdx, gdy, gt0, gdt;
  float* grid;
  int ntide;
  int lim_on;            /* optional slope limiter (p = 1) */
  double lim_nu, lim_M;
  int* nb3;              /* [ne][3] neighbour across local edge j, -1 on the boundary */
  int nriv, rnt;
  double rt0, rdt;
  double* rq; /* [rnt][nriv] */
  double *tamp, *tper, *tpha;
  int press;
  double pr[4];
  int exact;
  double ex[9];
  /* state and work */
  double *w, *wk[6], *Lw, *rhs, *rnode, *Re;
  uint8_t* dry;
  /* ledger (Neumaier-compensated) */
  double V0, VH0, rain_s, rain_c, bd_s, bd_c, stage_bdry;
};

/* Neumaier-compensated addition of v to the pair (sum s, compensation c): the mass ledger's sums
 * (the volume balance of Eq. SWE over the domain) kept free of cancellation */
static void neu_add(double* s, double* c, double v) {
  double t = *s + v;
  if (fabs(*s) >= fabs(v))
    *c += (*s - t) + v;
  else
    *c += (v - t) + *s;
  *s = t;
}

/* ---------------------------------------------------------------- basis (Eq. dubiner) --- */
/* phi_ij = sqrt((2i+1)(i+j+1)/2) * P_i(a) ((1-b)/2)^i * P_j^{(2i+1,0)}(b) on the reference triangle
 * (-1,-1),(1,-1),(-1,1) with collapsed coordinates a = 2(1+r)/(1-s) - 1, b = s.  The factor
 * P_i(a) ((1-s)/2)^i is evaluated as a polynomial in (r,s) by the Legendre recurrence written in
 * homogeneous form, so the vertex s = 1 needs no special case.  Ordering: total degree, then j
 * (the paper fixes no ordering of the modes of Eq. dubiner). */
static void legendre_hom(int n, double r, double s, double* Q, double* Qr, double* Qs) {
  double A = r + 0.5 * (1.0 + s), u = 0.5 * (1.0 - s);
  Q[0] = 1.0; Qr[0] = 0.0; Qs[0] = 0.0;
  if (n >= 1) { Q[1] = A; Qr[1] = 1.0; Qs[1] = 0.5; }
  for (int k = 1; k < n; ++k) {
    Q[k + 1] = ((2 * k + 1) * A * Q[k] - k * u * u * Q[k - 1]) / (k + 1);
    Qr[k + 1] = ((2 * k + 1) * (Q[k] + A * Qr[k]) - k * u * u * Qr[k - 1]) / (k + 1);
    Qs[k + 1] = ((2 * k + 1) * (0.5 * Q[k] + A * Qs[k]) - k * (-u * Q[k - 1] + u * u * Qs[k - 1])) / (k + 1);
  }
}

/* Jacobi polynomials P_k^(al,0)(x), k = 0..n, and their derivatives by the three-term recurrence:
 * the factor in s of the Dubiner basis (Eq. dubiner) */
static void jacobi_a0(int n, double al, double x, double* P, double* dP) {
  P[0] = 1.0; dP[0] = 0.0;
  if (n >= 1) { P[1] = 0.5 * ((al + 2.0) * x + al); dP[1] = 0.5 * (al + 2.0); }
  for (int k = 1; k < n; ++k) {
    double a1 = 2.0 * (k + 1) * (k + al + 1) * (2 * k + al);
    double a2 = (2 * k + al + 1);
    double b = (2 * k + al + 2) * (2 * k + al);
    double a4 = 2.0 * (k + al) * k * (2 * k + al + 2);
    P[k + 1] = (a2 * (b * x + al * al) * P[k] - a4 * P[k - 1]) / a1;
    dP[k + 1] = (a2 * (b * P[k] + (b * x + al * al) * dP[k]) - a4 * dP[k - 1]) / a1;
  }
}

/* The orthonormal Dubiner basis of Eq. dubiner at (r, s) and its derivatives in r and s */
void orc_basis(int p, double r, double s, double* phi, double* dr, double* ds) {
  double Q[NGMAX + 1], Qr[NGMAX + 1], Qs[NGMAX + 1];
  legendre_hom(p, r, s, Q, Qr, Qs);
  int m = 0;
  for (int d = 0; d <= p; ++d)
    for (int j = 0; j <= d; ++j) {
      int i = d - j;
      double P[NGMAX + 1], dP[NGMAX + 1];
      jacobi_a0(j, 2.0 * i + 1.0, s, P, dP);
      double c = sqrt((2.0 * i + 1.0) * (i + j + 1.0) / 2.0);
      phi[m] = c * Q[i] * P[j];
      if (dr) dr[m] = c * Qr[i] * P[j];
      if (ds) ds[m] = c * (Qs[i] * P[j] + Q[i] * dP[j]);
      ++m;
    }
}

/* ------------------------------------------------------------------------- quadrature --- */
/* barycentric coordinates -> (r, s) on the reference triangle (-1,-1), (1,-1), (-1,1) of Eq. dubiner */
static void bary_to_rs(const double l[3], double* r, double* s) {
  *r = -l[0] + l[1] - l[2];
  *s = -l[0] - l[1] + l[2];
}

/* Symmetric area rules for the element integrals of Eq. elem_weak_form (the paper names no rule), weights
 * summing to the reference area 2:
 *  p=0: centroid (degree 1);
 *  p=1: centroid 27/60, edge midpoints 8/60, vertices 3/60 (degree 3, Stroud);
 *  p=2: centroid 9/40, orbits (a,a,1-2a) with a = (6 -/+ sqrt 15)/21 and weights
 *       (155 -/+ sqrt 15)/1200 (degree 5, Radon). */
static int area_rule_bary(int p, double l[NQMAX][3], double* w) {
  int n = 0;
  l[n][0] = l[n][1] = l[n][2] = 1.0 / 3.0;
  if (p <= 0) { w[0] = 2.0; return 1; }
  if (p == 1) {
    w[n++] = 2.0 * 27.0 / 60.0;
    for (int i = 0; i < 3; ++i) { l[n][i] = 0.5; l[n][(i + 1) % 3] = 0.5; l[n][(i + 2) % 3] = 0.0; w[n++] = 2.0 * 8.0 / 60.0; }
    for (int i = 0; i < 3; ++i) { l[n][i] = 1.0; l[n][(i + 1) % 3] = 0.0; l[n][(i + 2) % 3] = 0.0; w[n++] = 2.0 * 3.0 / 60.0; }
    return n;
  }
  w[n++] = 2.0 * 9.0 / 40.0;
  double r15 = sqrt(15.0);
  double a[2] = {(6.0 - r15) / 21.0, (6.0 + r15) / 21.0};
  double wa[2] = {(155.0 - r15) / 1200.0, (155.0 + r15) / 1200.0};
  for (int o = 0; o < 2; ++o)
    for (int i = 0; i < 3; ++i) {
      l[n][i] = 1.0 - 2.0 * a[o]; l[n][(i + 1) % 3] = a[o]; l[n][(i + 2) % 3] = a[o];
      w[n++] = 2.0 * wa[o];
    }
  return n;
}

/* the area rule of the element integrals of Eq. elem_weak_form in (r, s) (test hook) */
int orc_area_rule(int p, double* r, double* s, double* w) {
  double l[NQMAX][3];
  int n = area_rule_bary(p, l, w);
  for (int q = 0; q < n; ++q) bary_to_rs(l[q], &r[q], &s[q]);
  return n;
}

/* Gauss-Legendre on [-1,1] with p+1 points: the edge integrals of Sec. 2.3 (the paper names no rule). */
int orc_edge_rule(int p, double* xi, double* w) {
  if (p <= 0) { xi[0] = 0.0; w[0] = 2.0; return 1; }
  if (p == 1) { double a = 1.0 / sqrt(3.0); xi[0] = -a; xi[1] = a; w[0] = w[1] = 1.0; return 2; }
  double a = sqrt(3.0 / 5.0);
  xi[0] = -a; xi[1] = 0.0; xi[2] = a; w[0] = w[2] = 5.0 / 9.0; w[1] = 8.0 / 9.0;
  return 3;
}

/* --------------------------------------------------------------------------- setup --- */
/* A solver of the method of Sec. 2.2-2.4 with degree p (Eq. dubiner), the Roe or LLF flux
 * (Sec. 2.3), the Shu-Osher SSP scheme of Eq. RKSSP with ssp_stages stages, gravity g, the
 * thin-layer threshold H0 (Sec. 2.4) and the friction law of Eq. SWE's tau_b (Manning, or the quadratic law of Sec. 3.1) */
orc_t* orc_create(int p, int flux, int ssp_stages, double g, double H0, int friction, double cf) {
  if (p < 0 || p > 2 || ssp_stages < 1 || ssp_stages > 5 || ssp_stages == 4) return NULL;
  orc_t* o = (orc_t*)calloc(1, sizeof(orc_t));
  o->p = p; o->np = (p + 1) * (p + 2) / 2; o->flux = flux; o->nstage = ssp_stages;
  o->g = g; o->H0 = H0; o->friction = friction; o->cf = cf;
  /* Shu-Osher coefficients: w(i+1) = sum_k alpha[i][k] w(k) + beta[i] dt L(w(i)) */
  if (ssp_stages == 1) {
    o->alpha[0][0] = 1.0; o->beta[0] = 1.0; o->cst[0] = 0.0;
  } else if (ssp_stages == 2) {
    o->alpha[0][0] = 1.0; o->beta[0] = 1.0;
    o->alpha[1][0] = 0.5; o->alpha[1][1] = 0.5; o->beta[1] = 0.5;
    o->cst[0] = 0.0; o->cst[1] = 1.0;
  } else if (ssp_stages == 3) {
    o->alpha[0][0] = 1.0; o->beta[0] = 1.0;
    o->alpha[1][0] = 0.75; o->alpha[1][1] = 0.25; o->beta[1] = 0.25;
    o->alpha[2][0] = 1.0 / 3.0; o->alpha[2][1] = 0.0; o->alpha[2][2] = 2.0 / 3.0; o->beta[2] = 2.0 / 3.0;
    o->cst[0] = 0.0; o->cst[1] = 1.0; o->cst[2] = 0.5;
  } else {
    /* optimal five-stage second-order SSP method: four forward-Euler substeps of dt/4, then
     * w(5) = w(0)/5 + 4/5 (w(4) + dt/4 L(w(4))); stage times t + i dt / 4 */
    for (int i = 0; i < 4; ++i) {
      o->alpha[i][i] = 1.0; o->beta[i] = 0.25; o->cst[i] = 0.25 * i;
    }
    o->alpha[4][0] = 0.2; o->alpha[4][4] = 0.8; o->beta[4] = 0.2; o->cst[4] = 1.0;
  }
  /* weight of dt*L(w(s)) in the final stage, for the mass ledger */
  double coef[6][5] = {{0}};
  for (int i = 0; i < ssp_stages; ++i)
    for (int s = 0; s < ssp_stages; ++s) {
      double c = (s == i) ? o->beta[i] : 0.0;
      for (int k = 0; k <= i; ++k) c += o->alpha[i][k] * coef[k][s];
      coef[i + 1][s] = c;
    }
  for (int s = 0; s < ssp_stages; ++s) o->bw[s] = coef[ssp_stages][s];
  /* tables */
  o->nq = area_rule_bary(p, o->lq, o->qw);
  for (int q = 0; q < o->nq; ++q) {
    double r, s;
    bary_to_rs(o->lq[q], &r, &s);
    orc_basis(p, r, s, o->phq[q], o->phr[q], o->phs[q]);
  }
  o->ng = orc_edge_rule(p, o->gxi, o->gw);
  for (int j = 0; j < 3; ++j) {
    for (int k = 0; k < o->ng; ++k) {
      double l[3] = {0, 0, 0}, r, s;
      l[j] = 0.5 * (1.0 - o->gxi[k]);
      l[(j + 1) % 3] = 0.5 * (1.0 + o->gxi[k]);
      memcpy(o->le[j][k], l, sizeof l);
      bary_to_rs(l, &r, &s);
      orc_basis(p, r, s, o->phe[j][k], NULL, NULL);
    }
    double l[3] = {0, 0, 0}, r, s;
    l[j] = 1.0;
    bary_to_rs(l, &r, &s);
    orc_basis(p, r, s, o->phv[j], NULL, NULL);
  }
  return o;
}

/* memory release helper (no counterpart in the paper) */
static void freep(void* p) { free(p); }

/* releases the solver (no counterpart in the paper) */
void orc_destroy(orc_t* o) {
  if (!o) return;
  void* ptrs[] = {o->x, o->y, o->tri, o->edn, o->ede, o->edj, o->edt, o->eds, o->order, o->det, o->rx, o->ry,
                  o->sx, o->sy, o->area, o->hb, o->man, o->rain_nodal, o->grid, o->tamp, o->tper, o->tpha,
                  o->w, o->wk[0], o->wk[1], o->wk[2], o->wk[3], o->wk[4], o->wk[5], o->Lw, o->rhs, o->rnode,
                  o->Re, o->dry, o->rq, o->nb3};
  for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; ++i) freep(ptrs[i]);
  free(o);
}

typedef struct { int64_t key; int e, j; } halfedge;

/* order of half edges by node pair, then element and local edge: pairs the two sides of each
 * interior edge of the triangulation (Sec. 2.1) */
static int cmp_he(const void* a, const void* b) {
  const halfedge *x = (const halfedge*)a, *y = (const halfedge*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->e != y->e) return x->e < y->e ? -1 : 1;
  return x->j - y->j;
}

/* key of an undirected node pair (mesh connectivity, Sec. 2.1) */
static int64_t pair_key(int a, int b, int nn) {
  int lo = a < b ? a : b, hi = a < b ? b : a;
  return (int64_t)lo * nn + hi;
}

/* The triangulation of the domain and its boundary parts (Sec. 2.1: ocean, land, river edges;
 * internal river edges of Sec. 2.3): element geometry, edges with both sides, edge order of
 * Sec. 2.3 (boundary edges before inner edges) */
int orc_set_mesh(orc_t* o, int nn, const double* xy, int ne, const int32_t* tri, int nb, const int32_t* bedge,
                 const int32_t* btype, const int32_t* bseg) {
  o->nn = nn; o->ne = ne;
  o->x = (double*)malloc(sizeof(double) * nn);
  o->y = (double*)malloc(sizeof(double) * nn);
  for (int i = 0; i < nn; ++i) { o->x[i] = xy[2 * i]; o->y[i] = xy[2 * i + 1]; }
  o->tri = (int32_t*)malloc(sizeof(int32_t) * 3 * ne);
  memcpy(o->tri, tri, sizeof(int32_t) * 3 * ne);
  o->det = (double*)malloc(sizeof(double) * ne);
  o->rx = (double*)malloc(sizeof(double) * ne);
  o->ry = (double*)malloc(sizeof(double) * ne);
  o->sx = (double*)malloc(sizeof(double) * ne);
  o->sy = (double*)malloc(sizeof(double) * ne);
  o->area = (double*)malloc(sizeof(double) * ne);
  for (int e = 0; e < ne; ++e) {
    int32_t* v = o->tri + 3 * e;
    double xr = 0.5 * (o->x[v[1]] - o->x[v[0]]), xs = 0.5 * (o->x[v[2]] - o->x[v[0]]);
    double yr = 0.5 * (o->y[v[1]] - o->y[v[0]]), ys = 0.5 * (o->y[v[2]] - o->y[v[0]]);
    double d = xr * ys - xs * yr;
    if (d < 0) { int32_t t = v[1]; v[1] = v[2]; v[2] = t; e--; continue; } /* make it CCW, redo */
    if (d == 0) return -1;
    o->det[e] = d; o->area[e] = 2.0 * d;
    o->rx[e] = ys / d; o->ry[e] = -xs / d; o->sx[e] = -yr / d; o->sy[e] = xr / d;
  }
  /* edges: pair up the 3*ne half-edges by their node pair */
  halfedge* he = (halfedge*)malloc(sizeof(halfedge) * 3 * ne);
  for (int e = 0; e < ne; ++e)
    for (int j = 0; j < 3; ++j) {
      he[3 * e + j].key = pair_key(o->tri[3 * e + j], o->tri[3 * e + (j + 1) % 3], nn);
      he[3 * e + j].e = e; he[3 * e + j].j = j;
    }
  qsort(he, 3 * ne, sizeof(halfedge), cmp_he);
  halfedge* bk = (halfedge*)malloc(sizeof(halfedge) * (nb > 0 ? nb : 1)); /* e = boundary index */
  for (int b = 0; b < nb; ++b) {
    if (btype[b] != ORC_BT_LAND && btype[b] != ORC_BT_OCEAN && btype[b] != ORC_BT_RIVER && btype[b] != ORC_BT_EXACT) {
      free(he); free(bk); return -2;
    }
    bk[b].key = pair_key(bedge[2 * b], bedge[2 * b + 1], nn); bk[b].e = b; bk[b].j = 0;
  }
  qsort(bk, nb, sizeof(halfedge), cmp_he);
  int cap = 3 * ne;
  o->edn = (int*)malloc(sizeof(int) * 2 * cap);
  o->ede = (int*)malloc(sizeof(int) * 2 * cap);
  o->edj = (int*)malloc(sizeof(int) * 2 * cap);
  o->edt = (int*)malloc(sizeof(int) * cap);
  o->eds = (int*)malloc(sizeof(int) * cap);
  int ned = 0;
  for (int i = 0; i < 3 * ne;) {
    int e = he[i].e, j = he[i].j;
    o->edn[2 * ned] = o->tri[3 * e + j];
    o->edn[2 * ned + 1] = o->tri[3 * e + (j + 1) % 3];
    o->ede[2 * ned] = e; o->edj[2 * ned] = j;
    o->eds[ned] = 0;
    if (i + 1 < 3 * ne && he[i + 1].key == he[i].key) {
      o->ede[2 * ned + 1] = he[i + 1].e; o->edj[2 * ned + 1] = he[i + 1].j;
      o->edt[ned] = -1;
      /* an interior edge listed as a boundary: a river edge (Sec. 2.3, internal river boundaries)
       * lets the river enter the element to the left of its listed direction a -> b, and that
       * element's neighbour sees a wall; a land edge is a wall on both sides */
      int lo = 0, hi = nb - 1, bi = -1;
      while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (bk[mid].key == he[i].key) { bi = bk[mid].e; break; }
        if (bk[mid].key < he[i].key) lo = mid + 1; else hi = mid - 1;
      }
      if (bi >= 0) {
        if (btype[bi] != ORC_BT_RIVER && btype[bi] != ORC_BT_LAND) { free(he); free(bk); return -3; }
        int h0 = i, h1 = i + 1;  /* h0: the receiving half-edge (traversed a -> b) */
        if (o->tri[3 * he[h0].e + he[h0].j] != bedge[2 * bi]) { h0 = i + 1; h1 = i; }
        o->ede[2 * ned] = he[h0].e; o->edj[2 * ned] = he[h0].j;
        o->edn[2 * ned] = o->tri[3 * he[h0].e + he[h0].j];
        o->edn[2 * ned + 1] = o->tri[3 * he[h0].e + (he[h0].j + 1) % 3];
        o->ede[2 * ned + 1] = -1; o->edj[2 * ned + 1] = -1;
        o->edt[ned] = btype[bi];
        o->eds[ned] = bseg ? bseg[bi] : 0;
        ++ned;
        o->ede[2 * ned] = he[h1].e; o->edj[2 * ned] = he[h1].j;
        o->edn[2 * ned] = o->tri[3 * he[h1].e + he[h1].j];
        o->edn[2 * ned + 1] = o->tri[3 * he[h1].e + (he[h1].j + 1) % 3];
        o->ede[2 * ned + 1] = -1; o->edj[2 * ned + 1] = -1;
        o->edt[ned] = ORC_BT_LAND;
        o->eds[ned] = 0;
      }
      i += 2;
    } else {
      o->ede[2 * ned + 1] = -1; o->edj[2 * ned + 1] = -1;
      o->edt[ned] = ORC_BT_LAND;
      int lo = 0, hi = nb - 1;
      while (lo <= hi) {
        int mid = (lo + hi) / 2;
        if (bk[mid].key == he[i].key) { o->edt[ned] = btype[bk[mid].e]; o->eds[ned] = bseg ? bseg[bk[mid].e] : 0; break; }
        if (bk[mid].key < he[i].key) lo = mid + 1; else hi = mid - 1;
      }
      i += 1;
    }
    ++ned;
  }
  o->ned = ned;
  free(he); free(bk);
  /* loop order of Sec. 2.3: elevation-specified edges, land edges, river edges, (verification)
   * exact edges, then inner edges */
  o->order = (int*)malloc(sizeof(int) * ned);
  int k = 0;
  const int seq[5] = {ORC_BT_OCEAN, ORC_BT_LAND, ORC_BT_RIVER, ORC_BT_EXACT, -1};
  for (int q = 0; q < 5; ++q)
    for (int i = 0; i < ned; ++i)
      if (o->edt[i] == seq[q]) o->order[k++] = i;
  o->ned = k;
  size_t nw = (size_t)ne * 3 * o->np;
  o->w = (double*)calloc(nw, sizeof(double));
  for (int i = 0; i < 6; ++i) o->wk[i] = (double*)calloc(nw, sizeof(double));
  o->Lw = (double*)calloc(nw, sizeof(double));
  o->rhs = (double*)calloc(nw, sizeof(double));
  o->rnode = (double*)calloc(nn, sizeof(double));
  o->Re = (double*)calloc(ne, sizeof(double));
  o->dry = (uint8_t*)calloc(ne, 1);
  o->hb = (double*)calloc(nn, sizeof(double));
  o->man = (double*)calloc(ne, sizeof(double));
  return ned;
}

/* nodal bathymetry h_b and element Manning coefficients of Eq. SWE */
int orc_set_fields(orc_t* o, const double* hb, const double* man) {
  memcpy(o->hb, hb, sizeof(double) * o->nn);
  if (man) memcpy(o->man, man, sizeof(double) * o->ne);
  return 0;
}

/* constant nodal rain rates (Eq. rain) */
void orc_set_rain_nodal(orc_t* o, const double* r) {
  o->rain_kind = 1;
  free(o->rain_nodal);
  o->rain_nodal = (double*)malloc(sizeof(double) * o->nn);
  memcpy(o->rain_nodal, r, sizeof(double) * o->nn);
}

/* the moving radial rain cell standing in for the parametric rainfall of Sec. 2.5 (whose own profile is not available) */
void orc_set_rain_parametric(orc_t* o, double x0, double y0, double heading, double speed, double rpeak, double rm,
                             double re, double t0) {
  o->rain_kind = 2;
  double v[8] = {x0, y0, heading, speed, rpeak, rm, re, t0};
  memcpy(o->st, v, sizeof v);
}

/* gridded rainfall records in mm/h, interpolated to the nodes (Sec. 2.5: bilinear in space, linear in time) */
void orc_set_rain_grid(orc_t* o, int nx, int ny, int nt, double x0, double y0, double dx, double dy, double t0,
                       double dt_rec, const float* mmh) {
  o->rain_kind = 3;
  o->gnx = nx; o->gny = ny; o->gnt = nt; o->gx0 = x0; o->gy0 = y0; o->gdx = dx; o->gdy = dy; o->gt0 = t0;
  o->gdt = dt_rec;
  free(o->grid);
  o->grid = (float*)malloc(sizeof(float) * (size_t)nx * ny * nt);
  memcpy(o->grid, mmh, sizeof(float) * (size_t)nx * ny * nt);
}

/* tidal constituents of the specified-elevation (ocean) boundary segments (Sec. 2.1) */
void orc_set_tide(orc_t* o, int nseg, const double* amp, const double* per, const double* pha) {
  o->ntide = nseg;
  free(o->tamp); free(o->tper); free(o->tpha);
  o->tamp = (double*)malloc(sizeof(double) * nseg);
  o->tper = (double*)malloc(sizeof(double) * nseg);
  o->tpha = (double*)malloc(sizeof(double) * nseg);
  memcpy(o->tamp, amp, sizeof(double) * nseg);
  memcpy(o->tper, per, sizeof(double) * nseg);
  memcpy(o->tpha, pha, sizeof(double) * nseg);
}

/* the Gaussian set-up eta_p whose forcing F = g H grad(eta_p) enters Eq. SWE (a storm-surge set-up forcing) */
void orc_set_pressure(orc_t* o, double x0, double y0, double sigma, double peak) {
  o->press = 1;
  o->pr[0] = x0; o->pr[1] = y0; o->pr[2] = sigma; o->pr[3] = peak;
}

/* verification only: the travelling-wave manufactured solution (exact ghost states and its
 * momentum residual as forcing; the convergence pin of the method's order) */
void orc_set_exact_wave(orc_t* o, double a, double k, double l, double c, double h0) {
  o->exact = 1;
  o->ex[0] = a; o->ex[1] = k; o->ex[2] = l; o->ex[3] = c; o->ex[4] = h0;
}

/* verification only: a linear exact field for the ghost states (hand-integral pin of the weak
 * form, Eq. elem_weak_form) */
void orc_set_exact_linear(orc_t* o, const double* c9) {
  o->exact = 2;
  memcpy(o->ex, c9, sizeof(double) * 9);
}

/* ------------------------------------------------------------------- point functions --- */
/* verification only: the exact field of the manufactured or linear modes at (x, y, t) */
static void exact_state(const orc_t* o, double x, double y, double t, double w[3]) {
  if (o->exact == 1) { /* zeta = a sin(k(x - ct)) cos(l y), q = (c zeta, 0) */
    double z = o->ex[0] * sin(o->ex[1] * (x - o->ex[3] * t)) * cos(o->ex[2] * y);
    w[0] = z; w[1] = o->ex[3] * z; w[2] = 0.0;
  } else { /* linear field: (zeta, qx, qy) = c0 + c1 x + c2 y per variable */
    for (int v = 0; v < 3; ++v) w[v] = o->ex[3 * v] + o->ex[3 * v + 1] * x + o->ex[3 * v + 2] * y;
  }
}

/* verification only: momentum residual of Eq. SWE for the travelling-wave manufactured solution on
 * a flat bottom h0 (entered as the forcing F) */
static void exact_forcing(const orc_t* o, double x, double y, double t, double f[2]) {
  f[0] = f[1] = 0.0;
  if (o->exact != 1) return;
  double a = o->ex[0], k = o->ex[1], l = o->ex[2], c = o->ex[3], h0 = o->ex[4];
  double th = k * (x - c * t);
  double z = a * sin(th) * cos(l * y);
  double zx = a * k * cos(th) * cos(l * y);
  double zy = -a * l * sin(th) * sin(l * y);
  double zt = -c * zx;
  double H = h0 + z;
  f[0] = c * zt + c * c * zx * z * (2.0 * H - z) / (H * H) + o->g * H * zx;
  f[1] = o->g * H * zy;
}

/* rain rate at node n and time t (m/s): constant nodal, moving radial cell (Sec. 2.5)
 * or gridded records (Sec. 2.5); the element rate is the mean of its nodes (Eq. rain) */
static double rain_at(const orc_t* o, int n, double t) {
  if (o->rain_kind == 1) return o->rain_nodal[n];
  if (o->rain_kind == 2) {
    double x0 = o->st[0], y0 = o->st[1], th = o->st[2], v = o->st[3], rp = o->st[4], rm = o->st[5], re = o->st[6];
    double xc = x0 + v * (t - o->st[7]) * cos(th), yc = y0 + v * (t - o->st[7]) * sin(th);
    double dx = o->x[n] - xc, dy = o->y[n] - yc;
    double r = sqrt(dx * dx + dy * dy);
    return r < rm ? rp * (0.5 + 0.5 * r / rm) : rp * exp(-(r - rm) / re);
  }
  if (o->rain_kind == 3) { /* bilinear in space, linear in time between records */
    double gx = (o->x[n] - o->gx0) / o->gdx, gy = (o->y[n] - o->gy0) / o->gdy, gt = (t - o->gt0) / o->gdt;
    gx = gx < 0 ? 0 : (gx > o->gnx - 1 ? o->gnx - 1 : gx);
    gy = gy < 0 ? 0 : (gy > o->gny - 1 ? o->gny - 1 : gy);
    gt = gt < 0 ? 0 : (gt > o->gnt - 1 ? o->gnt - 1 : gt);
    int i = (int)floor(gx), j = (int)floor(gy), k = (int)floor(gt);
    i = i > o->gnx - 2 ? o->gnx - 2 : i; i = i < 0 ? 0 : i;
    j = j > o->gny - 2 ? o->gny - 2 : j; j = j < 0 ? 0 : j;
    k = k > o->gnt - 2 ? o->gnt - 2 : k; k = k < 0 ? 0 : k;
    double fx = gx - i, fy = gy - j, ft = gt - k;
    double val[2];
    for (int q = 0; q < 2; ++q) {
      int kk = (o->gnt == 1) ? 0 : k + q;
      const float* G = o->grid + (size_t)kk * o->gnx * o->gny;
      int i1 = (o->gnx == 1) ? i : i + 1, j1 = (o->gny == 1) ? j : j + 1;
      double v00 = G[(size_t)j * o->gnx + i], v10 = G[(size_t)j * o->gnx + i1];
      double v01 = G[(size_t)j1 * o->gnx + i], v11 = G[(size_t)j1 * o->gnx + i1];
      val[q] = (1 - fy) * ((1 - fx) * v00 + fx * v10) + fy * ((1 - fx) * v01 + fx * v11);
    }
    double mmh = (1 - ft) * val[0] + ft * val[1];
    return mmh / 3.6e6;
  }
  return 0.0;
}

/* river discharge of segment seg at time t (m^2/s into the domain; Eq. river_bc, linear in time between records) */
static double river_at(const orc_t* o, int seg, double t) {
  if (seg < 0 || seg >= o->nriv || o->rnt < 1) return 0.0;
  if (o->rnt == 1) return o->rq[seg];
  double f = (t - o->rt0) / o->rdt;
  if (f <= 0.0) return o->rq[seg];
  if (f >= o->rnt - 1) return o->rq[(size_t)(o->rnt - 1) * o->nriv + seg];
  int i = (int)floor(f);
  double a = f - i;
  return (1.0 - a) * o->rq[(size_t)i * o->nriv + seg] + a * o->rq[(size_t)(i + 1) * o->nriv + seg];
}

/* discharge series of the river boundary segments (Sec. 2.1, Eq. river_bc) */
void orc_set_river(orc_t* o, int nseg, int nt, double t0, double dt, const double* q) {
  free(o->rq);
  o->rq = NULL;
  o->nriv = o->rnt = 0;
  if (nseg <= 0 || nt <= 0 || !q) return;
  o->rq = (double*)malloc(sizeof(double) * (size_t)nseg * nt);
  memcpy(o->rq, q, sizeof(double) * (size_t)nseg * nt);
  o->nriv = nseg;
  o->rnt = nt;
  o->rt0 = t0;
  o->rdt = dt > 0.0 ? dt : 1.0;
}

/* elevation of ocean segment seg at time t (Sec. 2.1: A sin(2 pi t / T + phase), no ramp) */
static double tide_at(const orc_t* o, int seg, double t) {
  if (seg < 0 || seg >= o->ntide) return 0.0;
  return o->tamp[seg] * sin(2.0 * M_PI * t / o->tper[seg] + o->tpha[seg]);
}

/* normal physical flux F(w).n with pressure g/2 (H^2 - hb^2) (Eq. SWE), evaluated as
 * g/2 zeta (zeta + 2 hb) -- the same quantity since H = zeta + hb (Sec. 2.1), without the
 * cancellation of two ~H^2 terms in deep water */
static void phys_flux(const orc_t* o, const double* w, double hb, double nx, double ny, double* f, double* un_out,
                      double* Hs_out) {
  double H = w[0] + hb, Hs = H > o->H0 ? H : o->H0;
  double u = w[1] / Hs, v = w[2] / Hs, un = u * nx + v * ny;
  double P = 0.5 * o->g * w[0] * (w[0] + 2.0 * hb);
  f[0] = w[1] * nx + w[2] * ny;
  f[1] = w[1] * un + P * nx;
  f[2] = w[2] * un + P * ny;
  *un_out = un;
  *Hs_out = Hs;
}

/* the numerical flux Fhat.n of Sec. 2.3 between traces wl and wr along the unit normal n: LLF, or
 * Roe with Roe averages and no entropy fix, the jump taken in (zeta, q) */
static void numflux_o(const orc_t* o, int flux, const double* wl, double hbl, const double* wr, double hbr, double nx,
                      double ny, double* f) {
  double FL[3], FR[3], unL, unR, HsL, HsR;
  phys_flux(o, wl, hbl, nx, ny, FL, &unL, &HsL);
  phys_flux(o, wr, hbr, nx, ny, FR, &unR, &HsR);
  double g = o->g;
  if (flux == ORC_LLF) {
    double lL = fabs(unL) + sqrt(g * HsL), lR = fabs(unR) + sqrt(g * HsR);
    double lam = lL > lR ? lL : lR;
    for (int v = 0; v < 3; ++v) f[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (wr[v] - wl[v]);
    return;
  }
  double sL = sqrt(HsL), sR = sqrt(HsR);
  double ut = (sL * wl[1] / HsL + sR * wr[1] / HsR) / (sL + sR);
  double vt = (sL * wl[2] / HsL + sR * wr[2] / HsR) / (sL + sR);
  double ct = sqrt(g * 0.5 * (HsL + HsR));
  double utn = ut * nx + vt * ny, utt = -ut * ny + vt * nx;
  double dz = wr[0] - wl[0];
  double dqx = wr[1] - wl[1], dqy = wr[2] - wl[2];
  double dqn = dqx * nx + dqy * ny, dqt = -dqx * ny + dqy * nx;
  double a1 = 0.5 * (dz - (dqn - utn * dz) / ct);
  double a3 = 0.5 * (dz + (dqn - utn * dz) / ct);
  double a2 = dqt - utt * dz;
  double l1 = fabs(utn - ct), l2 = fabs(utn), l3 = fabs(utn + ct);
  double D0 = l1 * a1 + l3 * a3;
  double D1 = l1 * a1 * (ut - ct * nx) + l2 * a2 * (-ny) + l3 * a3 * (ut + ct * nx);
  double D2 = l1 * a1 * (vt - ct * ny) + l2 * a2 * (nx) + l3 * a3 * (vt + ct * ny);
  f[0] = 0.5 * (FL[0] + FR[0]) - 0.5 * D0;
  f[1] = 0.5 * (FL[1] + FR[1]) - 0.5 * D1;
  f[2] = 0.5 * (FL[2] + FR[2]) - 0.5 * D2;
}

/* the numerical flux of Sec. 2.3 alone (test hook) */
void orc_numflux(int flux, double g, double H0, const double* wl, double hbl, const double* wr, double hbr, double nx,
                 double ny, double* f) {
  orc_t tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.g = g; tmp.H0 = H0;
  numflux_o(&tmp, flux, wl, hbl, wr, hbr, nx, ny, f);
}

/* reflective wall seen from the inside state w (land boundary of Sec. 2.1): ghost
 * mirrors q.n; the wall carries no mass */
static void wall_flux(const orc_t* o, const double* w, double hb, double nx, double ny, double* f) {
  double qn = w[1] * nx + w[2] * ny;
  double wr[3] = {w[0], w[1] - 2.0 * qn * nx, w[2] - 2.0 * qn * ny};
  numflux_o(o, o->flux, w, hb, wr, hb, nx, ny, f);
  f[0] = 0.0;
}

/* ---------------------------------------------------------------- right-hand side L_h --- */
/* the trace of element e's modal state at a point with basis values phi (Eq. dubiner expansion) */
static void eval_w(const orc_t* o, const double* W, int e, const double* phi, double out[3]) {
  const double* we = W + (size_t)e * 3 * o->np;
  for (int v = 0; v < 3; ++v) {
    double s = 0.0;
    for (int m = 0; m < o->np; ++m) s += we[v * o->np + m] * phi[m];
    out[v] = s;
  }
}

/* a nodal field (bathymetry, coordinates) interpolated linearly at barycentrics l of element e
 * (continuous piecewise linear h_b) */
static double interp_nodal(const orc_t* o, const double* f, int e, const double l[3]) {
  const int32_t* v = o->tri + 3 * e;
  return l[0] * f[v[0]] + l[1] * f[v[1]] + l[2] * f[v[2]];
}

/* unit outward normal and length of local edge j of element e (the n of Sec. 2.3's edge integrals) */
static void edge_geom(const orc_t* o, int e, int j, double* nx, double* ny, double* len) {
  int a = o->tri[3 * e + j], b = o->tri[3 * e + (j + 1) % 3];
  double tx = o->x[b] - o->x[a], ty = o->y[b] - o->y[a];
  double l = sqrt(tx * tx + ty * ty);
  *nx = ty / l; *ny = -tx / l; *len = l;
}

/* L_h(W) of Eq. RKSSP at time t (Eq. elem_weak_form in the order of Sec. 2.3: edge integrals,
 * forcing, area integrals; the wet/dry edge closure of Sec. 2.4): fills o->Lw = M^{-1} rhs, returns
 * the boundary mass outflow in *bdry_out and the rain volume rate in *rain_out. */
static void compute_L(orc_t* o, const double* W, double t, double* rain_out, double* bdry_out) {
  const int np = o->np, ng = o->ng;
  const double g = o->g;
  memset(o->rhs, 0, sizeof(double) * (size_t)o->ne * 3 * np);
  double bd_s = 0.0, bd_c = 0.0;
  /* 1. edge integrals <Fhat.n, v> (Sec. 2.3: boundary edges, then inner edges) */
  for (int ii = 0; ii < o->ned; ++ii) {
    int i = o->order[ii];
    int L = o->ede[2 * i], jL = o->edj[2 * i], R = o->ede[2 * i + 1], jR = o->edj[2 * i + 1];
    int type = o->edt[i];
    double nx, ny, len;
    edge_geom(o, L, jL, &nx, &ny, &len);
    double fl[NGMAX][3], fr[NGMAX][3], wl[NGMAX][3], wr[NGMAX][3], hbl[NGMAX], hbr[NGMAX];
    double phiR[NGMAX][NPMAX];
    double massflux = 0.0;
    for (int k = 0; k < ng; ++k) {
      eval_w(o, W, L, o->phe[jL][k], wl[k]);
      hbl[k] = interp_nodal(o, o->hb, L, o->le[jL][k]);
      if (type == -1) {
        /* the neighbour traverses the edge the other way: its parameter is -xi_k */
        double lR[3] = {0, 0, 0}, r, s;
        lR[jR] = 0.5 * (1.0 + o->gxi[k]);
        lR[(jR + 1) % 3] = 0.5 * (1.0 - o->gxi[k]);
        bary_to_rs(lR, &r, &s);
        orc_basis(o->p, r, s, phiR[k], NULL, NULL);
        eval_w(o, W, R, phiR[k], wr[k]);
        hbr[k] = interp_nodal(o, o->hb, R, lR);
        numflux_o(o, o->flux, wl[k], hbl[k], wr[k], hbr[k], nx, ny, fl[k]);
      } else if (type == ORC_BT_LAND) {
        wall_flux(o, wl[k], hbl[k], nx, ny, fl[k]);
      } else {
        double xp = interp_nodal(o, o->x, L, o->le[jL][k]), yp = interp_nodal(o, o->y, L, o->le[jL][k]);
        double qr = 0.0;
        if (type == ORC_BT_OCEAN) {
          wr[k][0] = tide_at(o, o->eds[i], t); wr[k][1] = wl[k][1]; wr[k][2] = wl[k][2];
        } else if (type == ORC_BT_RIVER) {
          qr = river_at(o, o->eds[i], t);
          wr[k][0] = wl[k][0]; wr[k][1] = -qr * nx; wr[k][2] = -qr * ny;
        } else {
          exact_state(o, xp, yp, t, wr[k]);
        }
        numflux_o(o, o->flux, wl[k], hbl[k], wr[k], hbl[k], nx, ny, fl[k]);
        if (type == ORC_BT_RIVER) fl[k][0] = -qr; /* the specified normal flow, outward positive */
      }
      massflux += o->gw[k] * 0.5 * len * fl[k][0];
    }
    int closeL = 0, closeR = 0;
    if (type == -1) {
      if ((o->dry[L] && massflux > 0.0) || (o->dry[R] && massflux < 0.0)) closeL = closeR = 1;
    } else if (type != ORC_BT_LAND) {
      if (o->dry[L] && massflux > 0.0) closeL = 1;
    }
    for (int k = 0; k < ng; ++k) {
      if (closeL) wall_flux(o, wl[k], hbl[k], nx, ny, fl[k]);
      if (type == -1) {
        if (closeR) {
          wall_flux(o, wr[k], hbr[k], -nx, -ny, fr[k]);
          for (int v = 0; v < 3; ++v) fr[k][v] = -fr[k][v]; /* express along L's normal */
        } else {
          for (int v = 0; v < 3; ++v) fr[k][v] = fl[k][v];
        }
      }
    }
    double* rL = o->rhs + (size_t)L * 3 * np;
    for (int k = 0; k < ng; ++k) {
      double wq = o->gw[k] * 0.5 * len;
      for (int v = 0; v < 3; ++v)
        for (int m = 0; m < np; ++m) rL[v * np + m] -= wq * fl[k][v] * o->phe[jL][k][m];
      if (type != -1) neu_add(&bd_s, &bd_c, wq * fl[k][0]);
    }
    if (type == -1) {
      double* rR = o->rhs + (size_t)R * 3 * np;
      for (int k = 0; k < ng; ++k) {
        double wq = o->gw[k] * 0.5 * len;
        for (int v = 0; v < 3; ++v)
          for (int m = 0; m < np; ++m) rR[v * np + m] += wq * fr[k][v] * phiR[k][m];
      }
    }
  }
  /* 2. forcing: rain at each node, element rain = mean of its three nodes (Eq. rain) */
  double rs = 0.0, rc = 0.0;
  if (o->rain_kind) {
    for (int n = 0; n < o->nn; ++n) o->rnode[n] = rain_at(o, n, t);
    for (int e = 0; e < o->ne; ++e) {
      const int32_t* v = o->tri + 3 * e;
      o->Re[e] = (o->rnode[v[0]] + o->rnode[v[1]] + o->rnode[v[2]]) / 3.0;
      neu_add(&rs, &rc, o->area[e] * o->Re[e]);
    }
  } else {
    memset(o->Re, 0, sizeof(double) * o->ne);
  }
  /* 3. area integrals (grad v, F) + (s, v) */
  for (int e = 0; e < o->ne; ++e) {
    const int32_t* vt = o->tri + 3 * e;
    double det = o->det[e];
    double hbr_ = 0.5 * (o->hb[vt[1]] - o->hb[vt[0]]), hbs_ = 0.5 * (o->hb[vt[2]] - o->hb[vt[0]]);
    double hbx = hbr_ * o->rx[e] + hbs_ * o->sx[e], hby = hbr_ * o->ry[e] + hbs_ * o->sy[e];
    double* re = o->rhs + (size_t)e * 3 * np;
    for (int q = 0; q < o->nq; ++q) {
      double wq[3];
      eval_w(o, W, e, o->phq[q], wq);
      double hb = interp_nodal(o, o->hb, e, o->lq[q]);
      double H = wq[0] + hb, Hs = H > o->H0 ? H : o->H0;
      double u = wq[1] / Hs, v = wq[2] / Hs;
      double P = 0.5 * g * wq[0] * (wq[0] + 2.0 * hb); /* = g/2 (H^2 - hb^2) */
      double fx[3] = {wq[1], wq[1] * u + P, wq[2] * u};
      double fy[3] = {wq[2], wq[1] * v, wq[2] * v + P};
      double tau = 0.0, sp = sqrt(u * u + v * v);
      if (o->friction == ORC_MANNING)
        tau = g * o->man[e] * o->man[e] * sp / pow(Hs, 4.0 / 3.0);
      else if (o->friction == ORC_QUADRATIC)
        tau = o->cf * sp / Hs;
      double Fx = 0.0, Fy = 0.0;
      if (o->press || o->exact == 1) {
        double xp = interp_nodal(o, o->x, e, o->lq[q]), yp = interp_nodal(o, o->y, e, o->lq[q]);
        if (o->press) {
          double dx = xp - o->pr[0], dy = yp - o->pr[1], s2 = o->pr[2] * o->pr[2];
          double eta = o->pr[3] * exp(-(dx * dx + dy * dy) / (2.0 * s2));
          Fx += g * H * (-eta * dx / s2);
          Fy += g * H * (-eta * dy / s2);
        }
        if (o->exact == 1) {
          double f2[2];
          exact_forcing(o, xp, yp, t, f2);
          Fx += f2[0]; Fy += f2[1];
        }
      }
      double s[3] = {o->Re[e], g * wq[0] * hbx - tau * wq[1] + Fx, g * wq[0] * hby - tau * wq[2] + Fy};
      double wdet = o->qw[q] * det;
      for (int m = 0; m < np; ++m) {
        double dx = o->phr[q][m] * o->rx[e] + o->phs[q][m] * o->sx[e];
        double dy = o->phr[q][m] * o->ry[e] + o->phs[q][m] * o->sy[e];
        for (int vv = 0; vv < 3; ++vv) re[vv * np + m] += wdet * (dx * fx[vv] + dy * fy[vv] + o->phq[q][m] * s[vv]);
      }
    }
    /* dry elements: the momentum equations are not advanced */
    if (o->dry[e])
      for (int m = 0; m < np; ++m) re[np + m] = re[2 * np + m] = 0.0;
    /* 4. M^{-1}: the orthonormal basis gives M = detJ * I */
    double* Le = o->Lw + (size_t)e * 3 * np;
    for (int k = 0; k < 3 * np; ++k) Le[k] = re[k] / det;
  }
  *rain_out = rs + rc;
  *bdry_out = bd_s + bd_c;
}

/* L_h of Eq. RKSSP (the DG right-hand side of Eq. elem_weak_form after M^-1) on the current state */
void orc_rhs(orc_t* o, double* L) {
  double r, b;
  compute_L(o, o->w, o->t, &r, &b);
  memcpy(L, o->Lw, sizeof(double) * (size_t)o->ne * 3 * o->np);
}

/* ----------------------------------------------------------- positivity (Sec. 2.4) --- */
int orc_positivity_vertex(double H0, const double* H, double* Ho, const double* qx, const double* qy, double* qxo,
                          double* qyo, uint8_t* dry) {
  int cas;
  for (int i = 0; i < 3; ++i) { Ho[i] = H[i]; qxo[i] = qx[i]; qyo[i] = qy[i]; dry[i] = 0; }
  if (H[0] >= H0 && H[1] >= H0 && H[2] >= H0) return 1; /* case 1: unchanged */
  double Hbar = (H[0] + H[1] + H[2]) / 3.0;
  if (Hbar <= H0) { /* case 2: flatten; every vertex is dry */
    cas = 2;
    for (int i = 0; i < 3; ++i) { Ho[i] = Hbar; dry[i] = 1; }
  } else { /* case 3: lift the shallow vertices to H0 keeping the sum */
    cas = 3;
    int id[3] = {0, 1, 2};
    for (int a = 0; a < 3; ++a)
      for (int b = a + 1; b < 3; ++b)
        if (H[id[b]] < H[id[a]] || (H[id[b]] == H[id[a]] && id[b] < id[a])) { int t = id[a]; id[a] = id[b]; id[b] = t; }
    double d = H0 - H[id[0]];
    Ho[id[0]] = H0;
    if (H[id[1]] - 0.5 * d >= H0) {
      Ho[id[1]] = H[id[1]] - 0.5 * d;
      Ho[id[2]] = H[id[2]] - 0.5 * d;
    } else {
      Ho[id[1]] = H0;
      Ho[id[2]] = H[id[2]] - (H0 - H[id[0]]) - (H0 - H[id[1]]);
    }
    for (int i = 0; i < 3; ++i) dry[i] = Ho[i] < H0;
  }
  /* M Pi^f: move momentum off dry vertices onto wet ones */
  int nd = dry[0] + dry[1] + dry[2];
  if (nd == 3) {
    for (int i = 0; i < 3; ++i) qxo[i] = qyo[i] = 0.0;
  } else if (nd > 0) {
    double dx = 0.0, dy = 0.0;
    for (int i = 0; i < 3; ++i)
      if (dry[i]) { dx += qx[i]; dy += qy[i]; qxo[i] = qyo[i] = 0.0; }
    for (int i = 0; i < 3; ++i)
      if (!dry[i]) { qxo[i] += dx / (3 - nd); qyo[i] += dy / (3 - nd); }
  }
  return cas;
}

/* rebuild modes 1..2 of one variable from three vertex values (the linear interpolant projected
 * on the orthonormal basis with the exact area rule); mode 0 is left as it is (the vertex-value
 * form of M Pi_h, Sec. 2.4) */
static void set_linear_part(int p, double* we, const double f[3]) {
  double l[NQMAX][3], qw[NQMAX];
  int nq = area_rule_bary(p < 1 ? 1 : p, l, qw);
  for (int m = 1; m < 3 && m < (p + 1) * (p + 2) / 2; ++m) {
    double s = 0.0;
    for (int q = 0; q < nq; ++q) {
      double r, ss, phi[NPMAX];
      bary_to_rs(l[q], &r, &ss);
      orc_basis(p, r, ss, phi, NULL, NULL);
      s += qw[q] * (l[q][0] * f[0] + l[q][1] * f[1] + l[q][2] * f[2]) * phi[m];
    }
    we[m] = s;
  }
}

/* M Pi_h of Sec. 2.4 (as read at the top of this file) on one element's modes we[3][np] (zeta, qx, qy) with nodal
 * bathymetry hbv at its
 * vertices and phv the basis at the vertices; returns 1 if the element is dry */
static int element_positivity(int p, const double phv[3][NPMAX], double H0, const double hbv[3], double* we) {
  const int np = (p + 1) * (p + 2) / 2;
  const int nl = np < 3 ? np : 3; /* modes of the linear part */
  double qx[3], qy[3], H[3];
  for (int i = 0; i < 3; ++i) {
    double s0 = 0, s1 = 0, s2 = 0;
    for (int m = 0; m < nl; ++m) {
      s0 += we[m] * phv[i][m]; s1 += we[np + m] * phv[i][m]; s2 += we[2 * np + m] * phv[i][m];
    }
    qx[i] = s1; qy[i] = s2; H[i] = s0 + hbv[i];
  }
  if (p >= 2) { /* quadratic modes blended out as the linear part's shallowest vertex nears H0 */
    double hmin = H[0] < H[1] ? H[0] : H[1];
    hmin = hmin < H[2] ? hmin : H[2];
    double th = (hmin - H0) / H0;
    th = th < 0.0 ? 0.0 : th;
    if (th < 1.0)
      for (int v = 0; v < 3; ++v)
        for (int m = 3; m < np; ++m) we[v * np + m] *= th;
  }
  double Ho[3], qxo[3], qyo[3];
  uint8_t dv[3];
  int cas = orc_positivity_vertex(H0, H, Ho, qx, qy, qxo, qyo, dv);
  if (cas != 1 && np > 1) {
    double zo[3] = {Ho[0] - hbv[0], Ho[1] - hbv[1], Ho[2] - hbv[2]};
    set_linear_part(p, we, zo);
  }
  int nd = dv[0] + dv[1] + dv[2];
  if (nd == 3) {
    for (int m = 0; m < np; ++m) we[np + m] = we[2 * np + m] = 0.0;
  } else if (nd > 0 && np > 1) {
    set_linear_part(p, we + np, qxo);
    set_linear_part(p, we + 2 * np, qyo);
  }
  return nd > 0;
}

/* ------------------------------------------- optional slope limiter (Sec. 2.3 mentions one) ---
 * The paper offers "an optional slope limiter" for shocks without giving its form.  This is the
 * TVB minmod moment limiter of Cockburn and Shu for P1 on triangles (J. Comput. Phys. 141,
 * 1998), applied componentwise to zeta, qx, qy: for edge i of element K with midpoint m_i and
 * barycentre b_0, write m_i - b_0 = a (b_j - b_0) + c (b_k - b_0) with two neighbour barycentres
 * and a, c >= 0; compare the P1 deviation d_i = w(m_i) - mean_0 with nu (a (mean_j - mean_0) +
 * c (mean_k - mean_0)) through minmod (kept when |d_i| <= M h^2); if the limited deviations do
 * not sum to zero, scale the positive and negative parts to balance; rebuild the linear part
 * from the midpoint deviations.  Means are untouched.  Limited: wet elements with three
 * neighbours whose edges all have a valid pair; others are left as they are. */
/* switches the optional limiter of Sec. 2.3 (the Cockburn-Shu form below) on or off, with its weight and constant */
void orc_set_limiter(orc_t* o, int on, double nu, double M) {
  o->lim_on = on;
  o->lim_nu = nu;
  o->lim_M = M;
}

/* neighbour across each local edge, for the limiter's barycentric pairs (Sec. 2.3's optional limiter) */
static void build_nb3(orc_t* o) {
  o->nb3 = (int*)malloc(sizeof(int) * 3 * (size_t)o->ne);
  for (int k = 0; k < 3 * o->ne; ++k) o->nb3[k] = -1;
  for (int i = 0; i < o->ned; ++i) {
    int L = o->ede[2 * i], jL = o->edj[2 * i], R = o->ede[2 * i + 1], jR = o->edj[2 * i + 1];
    if (o->edt[i] != -1 || R < 0) continue;
    o->nb3[3 * L + jL] = R;
    o->nb3[3 * R + jR] = L;
  }
}

/* minmod of two values (Sec. 2.3's optional limiter) */
static double minmod2(double a, double b) {
  if (a > 0.0 && b > 0.0) return a < b ? a : b;
  if (a < 0.0 && b < 0.0) return a > b ? a : b;
  return 0.0;
}

/* the optional slope limiter of Sec. 2.3 on state W, in place (the Cockburn-Shu form described above) */
static void limiter(orc_t* o, double* W) {
  if (!o->lim_on || o->p != 1) return;
  if (!o->nb3) build_nb3(o);
  const int np = o->np, ne = o->ne;
  const double phi0 = 1.0 / sqrt(2.0);
  double* out = (double*)malloc(sizeof(double) * (size_t)ne * 3 * np);
  memcpy(out, W, sizeof(double) * (size_t)ne * 3 * np);
  /* basis at the three edge midpoints of the reference triangle */
  double phm[3][NPMAX];
  for (int i = 0; i < 3; ++i) {
    double l[3] = {0, 0, 0}, r, s2;
    l[i] = 0.5;
    l[(i + 1) % 3] = 0.5;
    bary_to_rs(l, &r, &s2);
    orc_basis(o->p, r, s2, phm[i], NULL, NULL);
  }
  for (int e = 0; e < ne; ++e) {
    const int* nb = o->nb3 + 3 * e;
    if (o->dry[e] || nb[0] < 0 || nb[1] < 0 || nb[2] < 0) continue;
    const int32_t* vt = o->tri + 3 * e;
    double bx[4], by[4];
    bx[0] = (o->x[vt[0]] + o->x[vt[1]] + o->x[vt[2]]) / 3.0;
    by[0] = (o->y[vt[0]] + o->y[vt[1]] + o->y[vt[2]]) / 3.0;
    for (int j = 0; j < 3; ++j) {
      const int32_t* vn = o->tri + 3 * nb[j];
      bx[j + 1] = (o->x[vn[0]] + o->x[vn[1]] + o->x[vn[2]]) / 3.0;
      by[j + 1] = (o->y[vn[0]] + o->y[vn[1]] + o->y[vn[2]]) / 3.0;
    }
    double h = 0.0;
    for (int j = 0; j < 3; ++j) {
      double dx = o->x[vt[(j + 1) % 3]] - o->x[vt[j]], dy = o->y[vt[(j + 1) % 3]] - o->y[vt[j]];
      double len = sqrt(dx * dx + dy * dy);
      h = len > h ? len : h;
    }
    /* barycentric pairs: neighbour i with one of the other two, coefficients >= 0 */
    int pj[3], pk[3], ok = 1;
    double pa[3], pc[3];
    for (int i = 0; i < 3 && ok; ++i) {
      double mx = 0.5 * (o->x[vt[i]] + o->x[vt[(i + 1) % 3]]) - bx[0];
      double my = 0.5 * (o->y[vt[i]] + o->y[vt[(i + 1) % 3]]) - by[0];
      int found = 0;
      for (int t = 1; t <= 2 && !found; ++t) {
        int j = i, k = (i + t) % 3;
        double ax = bx[j + 1] - bx[0], ay = by[j + 1] - by[0], cx = bx[k + 1] - bx[0], cy = by[k + 1] - by[0];
        double det = ax * cy - ay * cx;
        if (det == 0.0) continue;
        double a = (mx * cy - my * cx) / det, c = (ax * my - ay * mx) / det;
        if (a >= 0.0 && c >= 0.0) { pj[i] = j; pk[i] = k; pa[i] = a; pc[i] = c; found = 1; }
      }
      ok = found;
    }
    if (!ok) continue;
    for (int v = 0; v < 3; ++v) {
      const double* we = W + ((size_t)e * 3 + v) * np;
      double m0 = we[0] * phi0, mb[3];
      for (int j = 0; j < 3; ++j) mb[j] = W[((size_t)nb[j] * 3 + v) * np] * phi0;
      double d[3], lim[3];
      int changed = 0;
      for (int i = 0; i < 3; ++i) {
        d[i] = we[1] * phm[i][1] + we[2] * phm[i][2];
        double dm = pa[i] * (mb[pj[i]] - m0) + pc[i] * (mb[pk[i]] - m0);
        lim[i] = (fabs(d[i]) <= o->lim_M * h * h) ? d[i] : minmod2(d[i], o->lim_nu * dm);
        if (lim[i] != d[i]) changed = 1;
      }
      if (!changed) continue;
      double sum = lim[0] + lim[1] + lim[2];
      if (sum != 0.0) {
        double pos = 0.0, neg = 0.0;
        for (int i = 0; i < 3; ++i) { pos += lim[i] > 0.0 ? lim[i] : 0.0; neg += lim[i] < 0.0 ? -lim[i] : 0.0; }
        double tp = pos > 0.0 ? (neg / pos < 1.0 ? neg / pos : 1.0) : 0.0;
        double tn = neg > 0.0 ? (pos / neg < 1.0 ? pos / neg : 1.0) : 0.0;
        for (int i = 0; i < 3; ++i) lim[i] = tp * (lim[i] > 0.0 ? lim[i] : 0.0) - tn * (lim[i] < 0.0 ? -lim[i] : 0.0);
      }
      /* vertex values of the linear function with midpoint deviations lim (edge i joins
       * vertices i and i+1): f(v_i) = lim_i + lim_{i-1} - lim_{i+1} */
      double f[3];
      for (int i = 0; i < 3; ++i) f[i] = m0 + lim[i] + lim[(i + 2) % 3] - lim[(i + 1) % 3];
      set_linear_part(o->p, out + ((size_t)e * 3 + v) * np, f);
    }
  }
  memcpy(W, out, sizeof(double) * (size_t)ne * 3 * np);
  free(out);
}

static void positivity(orc_t* o, double* W);
/* the limiter alone on the current state (test hook of Sec. 2.3's optional limiter) */
void orc_apply_limiter(orc_t* o) { limiter(o, o->w); }

/* M Pi_h of Sec. 2.4 on every element of W, setting the element dry flags */
static void positivity(orc_t* o, double* W) {
  for (int e = 0; e < o->ne; ++e) {
    const int32_t* vt = o->tri + 3 * e;
    const double hbv[3] = {o->hb[vt[0]], o->hb[vt[1]], o->hb[vt[2]]};
    o->dry[e] = (uint8_t)element_positivity(o->p, (const double(*)[NPMAX])o->phv, o->H0, hbv, W + (size_t)e * 3 * o->np);
  }
}

/* M Pi_h of Sec. 2.4 on one element's modes (test hook) */
int orc_positivity_modal(int p, double H0, const double* hbv, double* w) {
  if (p < 0 || p > 2) return -1;
  double phv[3][NPMAX];
  for (int i = 0; i < 3; ++i) {
    double l[3] = {0, 0, 0}, r, s;
    l[i] = 1.0;
    bary_to_rs(l, &r, &s);
    orc_basis(p, r, s, phv[i], NULL, NULL);
  }
  return element_positivity(p, (const double(*)[NPMAX])phv, H0, hbv, w);
}

/* ------------------------------------------------------------------- state and time --- */
/* water volume of the mass balance of Eq. SWE: sum_e A_e mean(zeta_e), or of the depth with_hb
 * (the volume above the bed), compensated */
static double ledger_V(const orc_t* o, const double* W, int with_hb) {
  double s = 0.0, c = 0.0;
  for (int e = 0; e < o->ne; ++e) {
    double zbar = W[(size_t)e * 3 * o->np] / sqrt(2.0); /* phi_0 = 1/sqrt(2) on the area-2 reference */
    if (with_hb) {
      const int32_t* v = o->tri + 3 * e;
      zbar += (o->hb[v[0]] + o->hb[v[1]] + o->hb[v[2]]) / 3.0;
    }
    neu_add(&s, &c, o->area[e] * zbar);
  }
  return s + c;
}

/* after a new state: M Pi_h (Sec. 2.4) defines the dry flags; the ledger's V0, VH0 and sums restart */
static void reset_ledger(orc_t* o) {
  positivity(o, o->w);
  o->V0 = ledger_V(o, o->w, 0);
  o->VH0 = ledger_V(o, o->w, 1);
  o->rain_s = o->rain_c = o->bd_s = o->bd_c = 0.0;
  o->nstep = 0;
}

/* the initial state (zeta, q) of Eq. SWE from nodal values, L2-projected on the basis of
 * Eq. dubiner (exact for the linear interpolant at p >= 1) */
int orc_set_state_nodal(orc_t* o, const double* zeta, const double* qx, const double* qy) {
  const double* f[3] = {zeta, qx, qy};
  for (int e = 0; e < o->ne; ++e) {
    const int32_t* vt = o->tri + 3 * e;
    double* we = o->w + (size_t)e * 3 * o->np;
    for (int v = 0; v < 3; ++v)
      for (int m = 0; m < o->np; ++m) {
        double s = 0.0;
        for (int q = 0; q < o->nq; ++q)
          s += o->qw[q] * (o->lq[q][0] * f[v][vt[0]] + o->lq[q][1] * f[v][vt[1]] + o->lq[q][2] * f[v][vt[2]]) *
               o->phq[q][m];
        we[v * o->np + m] = s;
      }
  }
  reset_ledger(o);
  return 0;
}

/* the state (zeta, q) of Eq. SWE as modal coefficients (Eq. dubiner) */
int orc_set_state_modal(orc_t* o, const double* w) {
  memcpy(o->w, w, sizeof(double) * (size_t)o->ne * 3 * o->np);
  reset_ledger(o);
  return 0;
}

/* the modal state (zeta, q) of Eq. SWE (Eq. dubiner coefficients) */
void orc_get_state(const orc_t* o, double* w) { memcpy(w, o->w, sizeof(double) * (size_t)o->ne * 3 * o->np); }

/* the state at the three vertices of every element (the values M Pi_h of Sec. 2.4 acts on) */
void orc_get_vertex_values(const orc_t* o, double* out) {
  for (int e = 0; e < o->ne; ++e)
    for (int v = 0; v < 3; ++v)
      for (int i = 0; i < 3; ++i) {
        double s = 0.0;
        for (int m = 0; m < o->np; ++m) s += o->w[((size_t)e * 3 + v) * o->np + m] * o->phv[i][m];
        out[((size_t)e * 3 + v) * 3 + i] = s;
      }
}

/* the element dry flags of Sec. 2.4 (dry when any vertex is dry) */
void orc_get_dry(const orc_t* o, uint8_t* dry) { memcpy(dry, o->dry, o->ne); }

/* the fixed time step of the runs (Sec. 3 uses a fixed dt) from the CFL condition at the current
 * state: cfl min_e 2 r_in / ((2p+1) max_vertices(|u| + sqrt(g Hs))) */
double orc_cfl_dt(const orc_t* o, double cfl) {
  double best = 1e300;
  for (int e = 0; e < o->ne; ++e) {
    const int32_t* vt = o->tri + 3 * e;
    double per = 0.0, lam = 0.0;
    for (int i = 0; i < 3; ++i) {
      int a = vt[i], b = vt[(i + 1) % 3];
      per += sqrt((o->x[b] - o->x[a]) * (o->x[b] - o->x[a]) + (o->y[b] - o->y[a]) * (o->y[b] - o->y[a]));
      double z = 0, qx = 0, qy = 0;
      for (int m = 0; m < o->np; ++m) {
        z += o->w[((size_t)e * 3) * o->np + m] * o->phv[i][m];
        qx += o->w[((size_t)e * 3 + 1) * o->np + m] * o->phv[i][m];
        qy += o->w[((size_t)e * 3 + 2) * o->np + m] * o->phv[i][m];
      }
      double H = z + o->hb[vt[i]], Hs = H > o->H0 ? H : o->H0;
      double l = sqrt(qx * qx + qy * qy) / Hs + sqrt(o->g * Hs);
      if (l > lam) lam = l;
    }
    double din = 4.0 * o->area[e] / per; /* twice the inradius */
    double dt = cfl * din / ((2.0 * o->p + 1.0) * lam);
    if (dt < best) best = dt;
  }
  return best;
}

/* time step and time of the SSP scheme (Eq. RKSSP) */
void orc_set_dt(orc_t* o, double dt) { o->dt = dt; }
/* the current time t of Eq. RKSSP (forcing and tide are evaluated at stage times) */
void orc_set_time(orc_t* o, double t) { o->t = t; }

/* n steps of the Shu-Osher SSP scheme of Eq. RKSSP: per stage L_h (Eq. elem_weak_form) at the
 * stage time, the combination, then M Pi_h (Sec. 2.4, after every stage) and the
 * optional limiter; rain and boundary volumes booked with the stage's final weight */
void orc_step(orc_t* o, long n) {
  size_t nw = (size_t)o->ne * 3 * o->np;
  for (long it = 0; it < n; ++it) {
    double* st[6] = {o->wk[0], o->wk[1], o->wk[2], o->wk[3], o->wk[4], o->wk[5]};
    memcpy(st[0], o->w, sizeof(double) * nw);
    for (int i = 0; i < o->nstage; ++i) {
      double rain, bdry;
      compute_L(o, st[i], o->t + o->cst[i] * o->dt, &rain, &bdry);
      neu_add(&o->rain_s, &o->rain_c, o->bw[i] * o->dt * rain);
      neu_add(&o->bd_s, &o->bd_c, -o->bw[i] * o->dt * bdry);
      double* out = st[i + 1];
      for (size_t k = 0; k < nw; ++k) {
        double s = o->beta[i] * o->dt * o->Lw[k];
        for (int j = 0; j <= i; ++j) s += o->alpha[i][j] * st[j][k];
        out[k] = s;
      }
      positivity(o, out);
      if (o->lim_on) {
        limiter(o, out);
        positivity(o, out);
      }
    }
    memcpy(o->w, st[o->nstage], sizeof(double) * nw);
    o->nstep++;
    o->t += o->dt;
  }
}

/* the mass ledger: t, V0, V, rain in, boundary in, VH0, the relative balance error |V - V0 - rain - bdry| / VH0
 * (Eq. SWE's mass equation integrated over domain and time) and the wet fraction */
void orc_get_ledger(const orc_t* o, double* out) {
  double V = ledger_V(o, o->w, 0);
  double rain = o->rain_s + o->rain_c, bd = o->bd_s + o->bd_c;
  int wet = 0;
  for (int e = 0; e < o->ne; ++e) wet += !o->dry[e];
  out[0] = o->t; out[1] = o->V0; out[2] = V; out[3] = rain; out[4] = bd; out[5] = o->VH0;
  out[6] = fabs(V - o->V0 - rain - bd) / o->VH0;
  out[7] = (double)wet / o->ne;
}

/* verification only: L2 error of variable var against the manufactured solution (the method's
 * order p + 1) */
double orc_l2_error_exact(const orc_t* o, int var) {
  double s = 0.0;
  for (int e = 0; e < o->ne; ++e)
    for (int q = 0; q < o->nq; ++q) {
      double wq[3], ex[3];
      eval_w(o, o->w, e, o->phq[q], wq);
      double xp = interp_nodal(o, o->x, e, o->lq[q]), yp = interp_nodal(o, o->y, e, o->lq[q]);
      exact_state(o, xp, yp, o->t, ex);
      s += o->qw[q] * o->det[e] * (wq[var] - ex[var]) * (wq[var] - ex[var]);
    }
  return sqrt(s);
}

/* amplification factor of the stepper's Shu-Osher table (Eq. RKSSP) on y' = lambda y, z = lambda dt */
double orc_ssp_amplification(int stages, double z) {
  orc_t* o = orc_create(1, 0, stages, 9.81, 0.01, 2, 0.0);
  double y[6] = {1.0, 0, 0, 0, 0, 0};
  for (int i = 0; i < stages; ++i) {
    double s = o->beta[i] * z * y[i];
    for (int j = 0; j <= i; ++j) s += o->alpha[i][j] * y[j];
    y[i + 1] = s;
  }
  double r = y[stages];
  orc_destroy(o);
  return r;
}
