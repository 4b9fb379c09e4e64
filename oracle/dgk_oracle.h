/*
 * dgk_oracle.h -- plain FP64 CPU reference ("oracle") of one explicit time step of
 * the DGSEM discretisation of the relaxed, non-isothermal Navier-Stokes-Korteweg
 * equations of Keim, Munz & Rohde (arXiv 2208.05310).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or call
 * this code; only the tests, the smoke check and the CPU-baseline leg of the bench
 * use it.  It shares no code, header, table or constant generator with the CUDA
 * library: every formula here is written out again from the paper.
 *
 * State layout (conserved variables, structure of arrays):
 *   U[v][e][n], v = 0..nv-1, e = element, n = node (x index fastest)
 *   relaxation models (model 1, 2): nv = dim+3, U = (rho, rho*u_1..rho*u_dim, rho*e, c)
 *   original NSK (model 0):          nv = dim+2, U = (rho, rho*u_1..rho*u_dim, rho*e)
 * Element e = ix + nx*(iy + ny*iz); node n = i + P*(j + P*k), P = N+1.
 */
#ifndef DGK_ORACLE_H
#define DGK_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int dim;            /* 2 or 3 */
    int N;              /* polynomial degree */
    int n[3];           /* elements per direction */
    double lo[3], hi[3];
    int periodic[3];
    /* faces of the box: -x, +x, -y, +y, -z, +z.  kind 0: no wall (direction must be
       periodic); kind 1: isothermal no-slip wall with static contact angle; kind 2:
       generalized Navier-slip wall, Eq. (bc_nsk_alpha), with the positive parameters
       gamma_1 (contact-angle hysteresis), gamma_2 (slip friction), gamma_3 (heat
       transfer; the wall temperature is wall_T) and gamma_4 (relaxation).
       wall_u: velocity of a kind-1 wall sliding in its own plane (the moving isothermal
       no-slip wall of the sliding-droplet case, Sec. 4; on the box its normal component
       must be zero, on curved elements it is projected on the local tangent plane); zero
       for kind 2, whose solid is at rest (Sec. 2.4). */
    int wall_kind[6];
    double wall_T[6];
    double wall_theta_deg[6];
    double wall_gamma[6][4];
    double wall_u[6][3];
    /* Curved elements (optional; xgeo = NULL: the straight box lo..hi).  Element e maps
       the reference cube [-1,1]^dim by the polynomial of degree ngeo per direction that
       interpolates xgeo[k][e][g] (coordinate k) at the equispaced points
       t_a = -1 + 2a/ngeo, g = a + (ngeo+1)(b + (ngeo+1)c).  The element connectivity is
       the box's (n, periodic, walls); neighbouring elements must share their face
       points.  Requires ngeo <= N (2D) or 2 ngeo <= N (3D), so that the metric terms
       are polynomials the scheme differentiates exactly.  Walls as above, along the local
       normal; a wall velocity is projected on the local tangent plane. */
    int ngeo;
    const double *xgeo;
    /* Unstructured connectivity (optional, with xgeo; NULL: the box's).  For face
       f = 2 dir + side of element e, conn[(e * 2dim + f) * 3 + 0..2] = (neighbour element,
       the neighbour's face, orientation), or (-1 - w, 0, 0) for a face on wall w of the
       wall table above.  Orientation o maps the face point (a, b) of e's face (tangential
       indices in increasing direction order, a fastest) to the neighbour's face point
       (a', b'): (u, v) = o & 1 ? (b, a) : (a, b); a' = o & 2 ? N - u : u;
       b' = o & 4 ? N - v : v (2D: one index, bit 1 only).  Elements may have any
       orientation-preserving local frame.
       Mortars (non-conforming 2:1 faces, Sec. 3.1): a big face facing 2 (2D) or 4 (3D)
       half-size faces has conn = (-100 - m, 0, 0), and mortar[m * 2^(dim-1) + p] =
       (small element, its face, orientation) for the sub-face p (bit 0: upper half along
       the big face's first tangential axis, bit 1: along its second); a small face has
       conn = (big element, its face, o | (p + 1) << 3), o mapping the small face's points
       onto the sub-face's points in the big face's frame. */
    const int *conn;
    const int *mortar;
    int nmortar;
} or_mesh;

typedef struct {
    int model;          /* 0 original NSK (periodic boxes only), 1 relaxation model 1, 2 relaxation model 2 */
    double gammaK, mu, kappa, cv, alpha, beta;
    int flux;           /* convective numerical flux: 0 Rusanov, 1 HLLC (model 2 only, Sec. 4) */
} or_params;

/* ---- point fluxes, for the tests of the numerical flux functions ----
   Convective flux F^C(U) in +e_dir at temperature T, and the HLLC flux between the
   states UL (at xi_dir = -) and UR (at xi_dir = +).  p: the model's convective pressure,
   a: the signal speed of the Rusanov flux. */
int or_conv_point(const or_params *p, int dim, int dir, const double *U, double T, double *F);
int or_hllc_point(const or_params *p, int dim, int dir, const double *UL, double TL, const double *UR, double TR,
                  double *F);
int or_rusanov_point(const or_params *p, int dim, int dir, const double *UL, double TL, const double *UR, double TR,
                     double *F);

/* ---- thermodynamics (Sec. 2.1) ---- */
double or_psi(double rho, double T, double cv);
double or_pressure(double rho, double T);
double or_dpdrho_T(double rho, double T);
double or_cs2(double rho, double T, double cv);
double or_chem(double rho, double T, double cv);
double or_inner_energy(double rho, double T, double cv);
double or_entropy_vol(double rho, double T, double cv);
int    or_spinodal(double T, double *rho_sv, double *rho_sl);
int    or_maxwell(double T, double *rho_v, double *rho_l);
double or_sigma_vl(double T, double cv, double gammaK);
double or_interface_width(double T, double cv, double gammaK);
int    or_rho_from_p(double T, double p, int liquid, double *rho);
double or_wall_dpsi_dc(double c, double rho_v, double rho_l, double sigma, double theta_deg);

/* ---- 1D operators (Sec. 3.1) ---- */
int  or_gauss_legendre(int npts, double *x, double *w);
void or_lagrange_at(int N, const double *xi, double x, double *l);
void or_dmatrix(int N, const double *xi, double *D);

/* ---- discretisation ---- */
int  or_sizes(const or_mesh *m, const or_params *p, long *nelem, int *np, int *nv);
int  or_node_coords(const or_mesh *m, double *x);
int  or_node_weights(const or_mesh *m, double *W); /* J times the Gauss weights, [e][n] */
int  or_set_primitive(const or_mesh *m, const or_params *p, const double *prim, double *U);
int  or_temperature(const or_mesh *m, const or_params *p, const double *U, double *T);
typedef void (*or_forcing_fn)(int dim, const double *x, double t, double *q, void *user);
int  or_rhs(const or_mesh *m, const or_params *p, const double *U, double *Ut);
int  or_rhs_forced(const or_mesh *m, const or_params *p, const double *U, double *Ut,
                   double t, or_forcing_fn f, void *user);
int  or_rk_coeffs(int rk, int *nstages, double *A, double *B, double *c);
int  or_run(const or_mesh *m, const or_params *p, double *U, int nsteps, double dt, int rk,
            double t0, or_forcing_fn f, void *user);
int  or_max_dt(const or_mesh *m, const or_params *p, const double *U, double cfl, double dfl, double *dt);
int  or_diagnostics(const or_mesh *m, const or_params *p, const double *U, double *out);
int  or_num_threads(void);
/* Threads of the parallel element loops from now on (OpenMP; n >= 1). */
void or_set_num_threads(int n);

#define OR_NDIAG 9  /* mass, mom_x, mom_y, mom_z, energy, -entropy, ||rho-c||_2, max|u|,
                        int Pi (rate of entropy production) */

#ifdef __cplusplus
}
#endif
#endif
