/*
 * dgswe_oracle.h -- plain FP64 CPU reference ("oracle") of the discontinuous Galerkin
 * rainfall shallow-water method (Wichitrnithed et al., arXiv 2307.14302, Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
 * baseline leg may load this library.  It shares no code, header, table or constant generator
 * with the CUDA library; the two meet only through the seeded input generator.
 *
 * All quantities are SI; the state is w = (zeta, qx, qy) with q = H u (Sec. 2.2), stored modal
 * as w[(e*3 + var)*np + m] in the orthonormal Dubiner basis (Eq. dubiner).
 */
#ifndef DGSWE_ORACLE_H
#define DGSWE_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc orc_t;

enum { ORC_ROE = 0, ORC_LLF = 1 };
enum { ORC_MANNING = 0, ORC_QUADRATIC = 1, ORC_NOFRICTION = 2 };
enum { ORC_BT_LAND = 0, ORC_BT_OCEAN = 1, ORC_BT_RIVER = 2, ORC_BT_EXACT = 3 };

orc_t* orc_create(int p, int flux, int ssp_stages, double g, double H0, int friction, double cf);
void orc_destroy(orc_t*);
int orc_set_mesh(orc_t*, int nn, const double* xy, int ne, const int32_t* tri, int nb, const int32_t* bedge,
                 const int32_t* btype, const int32_t* bseg);
int orc_set_fields(orc_t*, const double* hb_nodal, const double* manning_elem);
void orc_set_rain_nodal(orc_t*, const double* r);
void orc_set_rain_parametric(orc_t*, double x0, double y0, double heading, double speed, double rpeak, double rm,
                             double re, double t0);
void orc_set_rain_grid(orc_t*, int nx, int ny, int nt, double x0, double y0, double dx, double dy, double t0,
                       double dt_rec, const float* mm_per_h);
void orc_set_tide(orc_t*, int nseg, const double* amp, const double* period, const double* phase);
/* River boundaries (Sec. 2.1, Eq. river_bc): specified normal discharge q_river (m^2/s, positive
 * into the domain) per river segment, nt records from t0 every dt (linear in time, held at the
 * ends; nt = 1: constant).  q is [nt][nseg]. */
void orc_set_river(orc_t* o, int nseg, int nt, double t0, double dt, const double* q);
/* Optional slope limiter (p = 1): Cockburn-Shu TVB minmod moment limiter after each stage's
 * positive-depth operator (then the operator again); nu the minmod weight (1.5), M the TVB
 * constant (0: TVD). */
void orc_set_limiter(orc_t*, int on, double nu, double M);
/* the limiter alone on the current state (test hook) */
void orc_apply_limiter(orc_t*);
void orc_set_pressure(orc_t*, double x0, double y0, double sigma, double peak);
void orc_set_exact_wave(orc_t*, double a, double k, double l, double c, double h0);
void orc_set_exact_linear(orc_t*, const double* coef9);
int orc_set_state_nodal(orc_t*, const double* zeta, const double* qx, const double* qy);
int orc_set_state_modal(orc_t*, const double* w);
void orc_get_state(const orc_t*, double* w);
void orc_get_vertex_values(const orc_t*, double* v);
void orc_get_dry(const orc_t*, uint8_t* dry);
double orc_cfl_dt(const orc_t*, double cfl);
void orc_set_dt(orc_t*, double dt);
void orc_set_time(orc_t*, double t);
void orc_step(orc_t*, long n);
void orc_rhs(orc_t*, double* L);
void orc_get_ledger(const orc_t*, double* out8);
double orc_l2_error_exact(const orc_t*, int var);

/* component hooks for the pin tests */
void orc_basis(int p, double r, double s, double* phi, double* dphidr, double* dphids);
int orc_area_rule(int p, double* r, double* s, double* w);
int orc_edge_rule(int p, double* xi, double* w);
void orc_numflux(int flux, double g, double H0, const double* wl, double hbl, const double* wr, double hbr,
                 double nx, double ny, double* f);
int orc_positivity_vertex(double H0, const double* H, double* Hout, const double* qx, const double* qy, double* qxo,
                          double* qyo, uint8_t* dry);
/* M Pi_h (Sec. 2.4) on one element: w[3][Np] modal zeta, qx, qy in/out, hbv nodal bathymetry
 * at the three vertices; at p = 2 the quadratic modes are blended out continuously as the
 * linear part's shallowest vertex depth falls from 2 H0 to H0.  Returns 1 if the element is
 * dry, 0 if wet, -1 for p outside 0..2. */
int orc_positivity_modal(int p, double H0, const double* hbv, double* w);
double orc_ssp_amplification(int stages, double z);

#ifdef __cplusplus
}
#endif
#endif
