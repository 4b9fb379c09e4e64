/*
 * dgk_oracle.c -- plain, slow, FP64 CPU reference of the hot path of
 * Keim, Munz & Rohde, "A relaxation model for the non-isothermal
 * Navier-Stokes-Korteweg equations in confined domains" (arXiv 2208.05310).
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the bench).
 * The product path never includes, links or calls this file.
 *
 * Written for a reader who checks it against the paper by eye: loops in the order of
 * the method, no tiling, no fusion.  Every stage of the right-hand side is computed
 * for all elements before the next stage starts.  Built with -ffp-contract=off.
 *
 * Citations are to the paper's sections and equations:
 *   Sec. 2.1  van der Waals thermodynamics, Eq. (helmholtzfreeenergyvol), (pressure)
 *   Sec. 2.3  relaxation models 1 and 2, Eq. (navierstokeskorteweg_p), (..._palpha)
 *   Sec. 2.4  wall boundary conditions, Eq. (bc_nsk_alpha), (helmfreesurftot_derivative),
 *             (surftenscoef)
 *   Sec. 3.1  DGSEM on Legendre-Gauss nodes, Rusanov and HLLC fluxes (Toro 2009, the
 *             paper's reference for both; Sec. 4: HLLC for model 2), BR1 lifting (twice for the
 *             second derivative), point-wise non-conservative sources, low-storage RK
 *   Sec. 3.2  15-point Gauss quadrature for the surface tension integral
 *   Sec. 4    interface width L_i(T), initial tanh profiles
 *
 * Readings of the paper where it is silent or garbled are listed in the design notes
 * and restated at the point of use below.
 */
#include "dgk_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* van der Waals constants in the paper's non-dimensional form (Sec. 2.1). */
static const double RV = 8.0 / 3.0;
static const double AV = 3.0;
static const double BV = 1.0 / 3.0;

#define MAXP 10
#define MAXG 9 /* geometry points per direction of a curved element */
#define IDX(v, e, n, ne, np) (((size_t)(v) * (size_t)(ne) + (size_t)(e)) * (size_t)(np) + (size_t)(n))
#define FIDX(v, e, f, fp, ne, nf, nfp) \
    ((((size_t)(v) * (size_t)(ne) + (size_t)(e)) * (size_t)(nf) + (size_t)(f)) * (size_t)(nfp) + (size_t)(fp))

/* ======================================================================== */
/* Thermodynamics, Sec. 2.1                                                 */
/* ======================================================================== */

/* Helmholtz free energy per unit volume, Eq. (helmholtzfreeenergyvol). */
double or_psi(double rho, double T, double cv)
{
    return rho * RV * T * cv * (1.0 - log(T)) + rho * RV * T * log(BV * rho / (1.0 - BV * rho))
           - AV * rho * rho;
}

/* Pressure, Eq. (pressure). */
double or_pressure(double rho, double T)
{
    return rho * RV * T / (1.0 - BV * rho) - AV * rho * rho;
}

/* (dp/drho) at constant T, differentiated from Eq. (pressure). */
double or_dpdrho_T(double rho, double T)
{
    return RV * T / ((1.0 - BV * rho) * (1.0 - BV * rho)) - 2.0 * AV * rho;
}

/* Chemical potential dpsi/drho at constant T, differentiated from Eq. (helmholtzfreeenergyvol). */
double or_chem(double rho, double T, double cv)
{
    return RV * T * cv * (1.0 - log(T)) + RV * T * log(BV * rho / (1.0 - BV * rho))
           + RV * T / (1.0 - BV * rho) - 2.0 * AV * rho;
}

/* Internal energy per unit volume rho*eps = psi - T dpsi/dT = rho R cv T - a rho^2. */
double or_inner_energy(double rho, double T, double cv)
{
    return rho * RV * cv * T - AV * rho * rho;
}

/* Entropy per unit volume rho*eta = -dpsi/dT. */
double or_entropy_vol(double rho, double T, double cv)
{
    return rho * RV * cv * log(T) - rho * RV * log(BV * rho / (1.0 - BV * rho));
}

/* Isentropic speed of sound squared, Eq. (speedofsound), for the van der Waals fluid:
   (dp/drho)_T + (dp/dT)_rho (dT/drho)_eta, with (dT/drho)_eta = T / (cv rho (1 - b rho)). */
double or_cs2(double rho, double T, double cv)
{
    double dpdT = rho * RV / (1.0 - BV * rho);
    double dTdrho = T / (cv * rho * (1.0 - BV * rho));
    return or_dpdrho_T(rho, T) + dpdT * dTdrho;
}

/* Spinodal densities: zeros of (dp/drho)_T, one on each side of rho = 1 (Sec. 2.1). */
int or_spinodal(double T, double *rho_sv, double *rho_sl)
{
    if (!(T > 0.0 && T < 1.0)) return -1;
    /* (dp/drho)_T > 0 for small rho, < 0 at rho = 1 (T < 1), > 0 again near 1/b. */
    double a = 1e-12, b = 1.0;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (a + b);
        if (or_dpdrho_T(mid, T) > 0.0) a = mid; else b = mid;
    }
    *rho_sv = 0.5 * (a + b);
    a = 1.0; b = 1.0 / BV - 1e-12;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (a + b);
        if (or_dpdrho_T(mid, T) < 0.0) a = mid; else b = mid;
    }
    *rho_sl = 0.5 * (a + b);
    return 0;
}

/* Root of p(rho, T) = P on the vapour branch (0, rho_sv) or the liquid branch
   (rho_sl, 1/b); p is increasing on both, so bisection is exact to the last bit. */
static double branch_root(double T, double P, double lo, double hi)
{
    for (int it = 0; it < 300; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        if (or_pressure(mid, T) < P) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

int or_rho_from_p(double T, double p, int liquid, double *rho)
{
    if (T >= 1.0) { *rho = branch_root(T, p, 1e-14, 1.0 / BV - 1e-14); return 0; }
    double sv, sl;
    if (or_spinodal(T, &sv, &sl)) return -1;
    if (liquid) *rho = branch_root(T, p, sl, 1.0 / BV - 1e-14);
    else        *rho = branch_root(T, p, 1e-14, sv);
    return 0;
}

/* Maxwell (saturation) densities at temperature T < 1 (Sec. 2.1): the vapour and liquid
   states with equal pressure and equal chemical potential.  Bisection on the common
   pressure P: for each P the two branch roots are found and the chemical potential
   difference mu(rho_l) - mu(rho_v) changes sign at the Maxwell pressure.  Finished by
   Newton steps on the 2x2 system to full precision. */
int or_maxwell(double T, double *rho_v, double *rho_l)
{
    double sv, sl;
    if (or_spinodal(T, &sv, &sl)) return -1;
    const double cv = 1.0; /* the cv term of mu does not depend on rho and cancels */
    double Plo = or_pressure(sl, T), Phi = or_pressure(sv, T);
    if (Plo < 1e-14) Plo = 1e-14;
    double rv = 0, rl = 0;
    for (int it = 0; it < 200; ++it) {
        double P = 0.5 * (Plo + Phi);
        rv = branch_root(T, P, 1e-14, sv);
        rl = branch_root(T, P, sl, 1.0 / BV - 1e-14);
        double g = or_chem(rl, T, cv) - or_chem(rv, T, cv);
        /* raising P moves rho_v up and rho_l up; mu_l - mu_v decreases through zero */
        if (g > 0.0) Plo = P; else Phi = P;
        if (Phi - Plo < 1e-17) break;
    }
    for (int it = 0; it < 8; ++it) {
        double F1 = or_pressure(rl, T) - or_pressure(rv, T);
        double F2 = or_chem(rl, T, cv) - or_chem(rv, T, cv);
        double pv = or_dpdrho_T(rv, T), pl = or_dpdrho_T(rl, T);
        double J11 = -pv, J12 = pl, J21 = -pv / rv, J22 = pl / rl;
        double det = J11 * J22 - J12 * J21;
        if (det == 0.0) break;
        double dv = (F1 * J22 - F2 * J12) / det;
        double dl = (J11 * F2 - J21 * F1) / det;
        rv -= dv; rl -= dl;
    }
    *rho_v = rv; *rho_l = rl;
    return 0;
}

/* Gauss-Legendre points and weights on [-1, 1] by Newton iteration on P_n. */
int or_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1 || n > 64) return -1;
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double pn = (n == 1) ? z : p1;
            double pnm1 = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pnm1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) {
                /* one more evaluation of the derivative at the converged point */
                p0 = 1.0; p1 = z;
                for (int k = 2; k <= n; ++k) {
                    double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1; p1 = p2;
                }
                pn = (n == 1) ? z : p1;
                pnm1 = (n == 1) ? 1.0 : p0;
                dp = n * (z * pn - pnm1) / (z * z - 1.0);
                break;
            }
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    return 0;
}

/* Equilibrium surface tension, Eq. (surftenscoef), with the prefactor read as
   sqrt(2 gamma_K) (the printed sqrt(2/gamma_K) does not reproduce the paper's own
   sigma = 0.0052 at T = 0.85, gamma_K = 1e-4).  The integral of sqrt(psi - bitangent)
   between the Maxwell densities is taken with 15-point Gauss quadrature (Sec. 3.2). */
double or_sigma_vl(double T, double cv, double gammaK)
{
    double rv, rl;
    if (or_maxwell(T, &rv, &rl)) return NAN;
    double x[15], w[15];
    or_gauss_legendre(15, x, w);
    double muv = or_chem(rv, T, cv), pv = or_pressure(rv, T);
    double sum = 0.0;
    for (int q = 0; q < 15; ++q) {
        double rho = 0.5 * (rl + rv) + 0.5 * (rl - rv) * x[q];
        double bitangent = rho * muv - pv;
        double diff = or_psi(rho, T, cv) - bitangent;
        if (diff < 0.0) diff = 0.0;
        sum += w[q] * sqrt(diff);
    }
    return sqrt(2.0 * gammaK) * 0.5 * (rl - rv) * sum;
}

/* Initial interface width L_i(T) = sqrt(2) gamma_K (rho_l - rho_v)^2 / sigma (Sec. 4). */
double or_interface_width(double T, double cv, double gammaK)
{
    double rv, rl;
    if (or_maxwell(T, &rv, &rl)) return NAN;
    return sqrt(2.0) * gammaK * (rl - rv) * (rl - rv) / or_sigma_vl(T, cv, gammaK);
}

/* Derivative of the cubic wall free energy, Eq. (helmfreesurftot_derivative). */
double or_wall_dpsi_dc(double c, double rho_v, double rho_l, double sigma, double theta_deg)
{
    double d = rho_l - rho_v;
    return 6.0 * (c - rho_l) * (c - rho_v) / (d * d * d) * sigma * cos(theta_deg * M_PI / 180.0);
}

/* ======================================================================== */
/* 1D operators on Legendre-Gauss nodes, Sec. 3.1                           */
/* ======================================================================== */

/* Lagrange basis l_j(x) = prod_{k != j} (x - xi_k) / (xi_j - xi_k). */
void or_lagrange_at(int N, const double *xi, double x, double *l)
{
    for (int j = 0; j <= N; ++j) {
        double v = 1.0;
        for (int k = 0; k <= N; ++k)
            if (k != j) v *= (x - xi[k]) / (xi[j] - xi[k]);
        l[j] = v;
    }
}

/* Derivative matrix D[i][j] = l_j'(xi_i), from the product rule applied to l_j. */
void or_dmatrix(int N, const double *xi, double *D)
{
    for (int i = 0; i <= N; ++i)
        for (int j = 0; j <= N; ++j) {
            double s = 0.0;
            for (int m = 0; m <= N; ++m) {
                if (m == j) continue;
                double prod = 1.0 / (xi[j] - xi[m]);
                for (int k = 0; k <= N; ++k)
                    if (k != j && k != m) prod *= (xi[i] - xi[k]) / (xi[j] - xi[k]);
                s += prod;
            }
            D[i * (N + 1) + j] = s;
        }
}

/* ======================================================================== */
/* Discretisation context                                                    */
/* ======================================================================== */

typedef struct {
    int d, N, P, np, nfp, nv, nl;
    long ne;
    int n[3];
    double h[3], lo[3];
    int periodic[3];
    int wall_kind[6];
    double wall_T[6], wall_rv[6], wall_rl[6], wall_sigma[6], wall_theta[6];
    double wall_g[6][4]; /* kind 2: gamma_1..gamma_4 */
    double wall_u[6][3]; /* kind 1: velocity of the wall (tangential) */
    double xi[MAXP], w[MAXP], Dhat[MAXP * MAXP], lm[MAXP], lp[MAXP];
    double Dm[MAXP * MAXP]; /* D_il = l_l'(xi_i) */
    or_params prm;
    /* curved elements (Sec. 3.1: curvilinear hexahedra with metric terms) */
    int curved, ngeo;
    const double *xgeo; /* [d][e][(ngeo+1)^d], the caller's */
    const int *conn;    /* unstructured connectivity [e][2d][3], the caller's, or NULL */
    const int *mortar;  /* mortar table [m][2^(d-1)][3], the caller's */
    int nmortar, nsub;  /* mortars, sub-faces per mortar 2^(d-1) */
    /* 1D mortar operators for the two halves h of a big face, eta_h(xi) = (xi + 2h - 1)/2:
       Im[h][j][i] = l_i(eta_h(xi_j)) (big face point i to sub-face point j),
       Pm[h][i][j] = w_j/(2 w_i) l_i(eta_h(xi_j)) (L2 projection back) */
    double Im[2][MAXP * MAXP], Pm[2][MAXP * MAXP];
    double *Ja;         /* [e][n][dir][k]: J a^dir_k (contravariant basis times J) at the nodes */
    double *Jn;         /* [e][n]: Jacobian J at the nodes */
    double *Jf;         /* [e][f][fp][k]: J a^dir_k at the face points, f = 2 dir + side */
    double *xn;         /* [e][n][k]: node coordinates */
} ctx_t;

static int setup_curved(ctx_t *c);

static int ipow(int a, int b) { int r = 1; while (b-- > 0) r *= a; return r; }

static int setup(const or_mesh *m, const or_params *p, ctx_t *c)
{
    memset(c, 0, sizeof(*c));
    if (m->dim != 2 && m->dim != 3) return -1;
    if (m->N < 1 || m->N + 1 > MAXP) return -1;
    if (p->model < 0 || p->model > 2) return -1;
    if (p->flux != 0 && p->flux != 1) return -1;
    if (p->flux == 1 && p->model != 2) return -1; /* HLLC: model 2 (its hyperbolic part) */
    c->d = m->dim; c->N = m->N; c->P = m->N + 1;
    c->np = ipow(c->P, c->d);
    c->nfp = ipow(c->P, c->d - 1);
    c->prm = *p;
    c->nv = (p->model == 0) ? c->d + 2 : c->d + 3;
    c->nl = (p->model == 0) ? c->d + 1 : c->d + 2;
    c->ne = 1;
    for (int d = 0; d < 3; ++d) c->n[d] = 1;
    for (int d = 0; d < c->d; ++d) {
        if (m->n[d] < 1) return -1;
        c->n[d] = m->n[d];
        c->ne *= m->n[d];
        c->h[d] = (m->hi[d] - m->lo[d]) / m->n[d];
        c->lo[d] = m->lo[d];
        c->periodic[d] = m->periodic[d];
        for (int s = 0; s < 2; ++s) {
            int f = 2 * d + s;
            c->wall_kind[f] = m->periodic[d] ? 0 : m->wall_kind[f];
            if (!m->periodic[d] && m->wall_kind[f] != 1 && m->wall_kind[f] != 2) return -1;
            if (c->wall_kind[f] == 2) {
                for (int k = 0; k < 4; ++k) {
                    if (!(m->wall_gamma[f][k] >= 0.0)) return -1;
                    c->wall_g[f][k] = m->wall_gamma[f][k];
                }
            }
            for (int k = 0; k < 3; ++k) {
                double uk = c->wall_kind[f] != 0 && k < c->d ? m->wall_u[f][k] : 0.0;
                /* box walls: tangential; curved walls: projected on the tangent plane per point */
                if (!isfinite(uk) || (uk != 0.0 && (c->wall_kind[f] != 1 || (k == d && !m->xgeo)))) return -1;
                c->wall_u[f][k] = uk;
            }
            if (c->wall_kind[f] != 0) {
                if (p->model == 0) return -1; /* original NSK: periodic boxes only */
                c->wall_T[f] = m->wall_T[f];
                c->wall_theta[f] = m->wall_theta_deg[f];
                if (or_maxwell(m->wall_T[f], &c->wall_rv[f], &c->wall_rl[f])) return -1;
                c->wall_sigma[f] = or_sigma_vl(m->wall_T[f], p->cv, p->gammaK);
            }
        }
    }
    or_gauss_legendre(c->P, c->xi, c->w);
    double *D = c->Dm;
    or_dmatrix(c->N, c->xi, D);
    for (int i = 0; i < c->P; ++i)
        for (int j = 0; j < c->P; ++j)
            c->Dhat[i * c->P + j] = -(c->w[j] / c->w[i]) * D[j * c->P + i];
    or_lagrange_at(c->N, c->xi, -1.0, c->lm);
    or_lagrange_at(c->N, c->xi, 1.0, c->lp);
    if (m->conn && !m->xgeo) return -1;
    if (m->nmortar && !m->conn) return -1;
    c->mortar = m->mortar;
    c->nmortar = m->nmortar;
    c->nsub = c->d == 2 ? 2 : 4;
    for (int h = 0; h < 2; ++h)
        for (int j = 0; j < c->P; ++j) {
            double l[MAXP];
            or_lagrange_at(c->N, c->xi, 0.5 * (c->xi[j] + 2.0 * h - 1.0), l);
            for (int i = 0; i < c->P; ++i) {
                c->Im[h][j * c->P + i] = l[i];
                c->Pm[h][i * c->P + j] = c->w[j] / (2.0 * c->w[i]) * l[i];
            }
        }
    if (m->xgeo) {
        c->ngeo = m->ngeo;
        c->xgeo = m->xgeo;
        c->conn = m->conn;
        if (m->ngeo < 1 || m->ngeo > MAXG - 1) return -1;
        if (c->d == 2 ? m->ngeo > c->N : 2 * m->ngeo > c->N) return -1;
        c->curved = 1;
        return setup_curved(c);
    }
    return 0;
}

static void teardown(ctx_t *c)
{
    free(c->Ja); free(c->Jn); free(c->Jf); free(c->xn);
    c->Ja = c->Jn = c->Jf = c->xn = NULL;
}

/* coordinate of node n along direction d */
static int ncoord(const ctx_t *c, int n, int d) { return (n / ipow(c->P, d)) % c->P; }

/* face-point index of node n on the faces normal to direction d: the remaining node
   coordinates in increasing direction order */
static int node_to_fp(const ctx_t *c, int n, int d)
{
    int fp = 0, mul = 1;
    for (int dd = 0; dd < c->d; ++dd) {
        if (dd == d) continue;
        fp += ncoord(c, n, dd) * mul;
        mul *= c->P;
    }
    return fp;
}

/* node at position l along direction d through face point fp */
static int fp_to_node(const ctx_t *c, int fp, int d, int l)
{
    int co[3] = {0, 0, 0};
    co[d] = l;
    int rest = fp;
    for (int dd = 0; dd < c->d; ++dd) {
        if (dd == d) continue;
        co[dd] = rest % c->P;
        rest /= c->P;
    }
    return co[0] + c->P * (co[1] + c->P * co[2]);
}

/* neighbour of element e across face (d, s) (s = 0: minus side, 1: plus side); -1 at a wall */
static long neighbour(const ctx_t *c, long e, int d, int s)
{
    if (c->conn) {
        long v = c->conn[((size_t)e * 2 * c->d + 2 * d + s) * 3];
        return v >= 0 ? v : -1;
    }
    long co[3];
    co[0] = e % c->n[0];
    co[1] = (e / c->n[0]) % c->n[1];
    co[2] = e / ((long)c->n[0] * c->n[1]);
    co[d] += s ? 1 : -1;
    if (co[d] < 0 || co[d] >= c->n[d]) {
        if (!c->periodic[d]) return -1;
        co[d] = (co[d] + c->n[d]) % c->n[d];
    }
    return co[0] + c->n[0] * (co[1] + (long)c->n[1] * co[2]);
}

/* The neighbour's face facing face f of element e (box: the opposite face). */
static int nb_face(const ctx_t *c, long e, int f)
{
    if (c->conn) return c->conn[((size_t)e * 2 * c->d + f) * 3 + 1];
    return 2 * (f / 2) + 1 - f % 2;
}

/* The neighbour's face point matching face point fp of face f of element e (box: fp). */
static int map_fp(const ctx_t *c, int o, int fp)
{
    int a = fp % c->P, b = fp / c->P, N = c->N;
    int u = (o & 1) ? b : a, v = (o & 1) ? a : b;
    if (o & 2) u = N - u;
    if (o & 4) v = N - v;
    return u + c->P * v;
}

static int nb_fp(const ctx_t *c, long e, int f, int fp)
{
    if (!c->conn) return fp;
    int o = c->conn[((size_t)e * 2 * c->d + f) * 3 + 2] & 7, N = c->N;
    int a = fp % c->P, b = fp / c->P;
    int u = (o & 1) ? b : a, v = (o & 1) ? a : b;
    if (o & 2) u = N - u;
    if (o & 4) v = N - v;
    return u + c->P * v;
}

/* Face kinds: conforming, wall, the small or the big side of a mortar. */
#define F_CONF 0
#define F_WALL 1
#define F_SMALL 2
#define F_BIG 3
static int face_kind(const ctx_t *c, long e, int f)
{
    if (!c->conn) return neighbour(c, e, f / 2, f % 2) >= 0 ? F_CONF : F_WALL;
    const int *t = c->conn + ((size_t)e * 2 * c->d + f) * 3;
    if (t[0] <= -100) return F_BIG;
    if (t[0] < 0) return F_WALL;
    return (t[2] >> 3) ? F_SMALL : F_CONF;
}

/* Facing sign of two faces' metric orientations (J a^dir along +xi_dir of each element):
   +1 for a plus and a minus face, -1 for two of the same side. */
static double facing(int f, int fo) { return ((f ^ fo) & 1) ? 1.0 : -1.0; }

/* The neighbour's values of the face field tr (variable v, layout FIDX) at the points of
   face f of element e: conforming: the neighbour's trace at the matching points; small
   side of a mortar: the big face's trace interpolated to the sub-face's points; big side:
   the L2 projection of the small faces' traces.  scale multiplies the small faces'
   values in the projection and divides the big face's in the interpolation (1 for plain
   traces, 2^(d-1) for quantities carrying the surface element); with signed, each
   neighbour value is multiplied by the facing sign of the two faces. */
static void nb_trace(const ctx_t *c, const double *tr, int v, long e, int f, double scale, int signed_, double *out)
{
    long ne = c->ne;
    int nf = 2 * c->d, nfp = c->nfp, P = c->P;
    int kind = face_kind(c, e, f);
    const int *t = c->conn ? c->conn + ((size_t)e * nf + f) * 3 : NULL;
    if (kind == F_CONF) {
        long nb = neighbour(c, e, f / 2, f % 2);
        int fo = nb_face(c, e, f);
        double sg = signed_ ? facing(f, fo) : 1.0;
        for (int fp = 0; fp < nfp; ++fp) out[fp] = sg * tr[FIDX(v, nb, fo, nb_fp(c, e, f, fp), ne, nf, nfp)];
        return;
    }
    if (kind == F_SMALL) {
        long B = t[0];
        int fB = t[1], o = t[2] & 7, pos = (t[2] >> 3) - 1, h0 = pos & 1, h1 = (pos >> 1) & 1;
        double sg = (signed_ ? facing(f, fB) : 1.0) / scale;
        for (int fp = 0; fp < nfp; ++fp) {
            int q = map_fp(c, o, fp), u = q % P, w = q / P;
            double acc = 0.0;
            if (c->d == 2) {
                for (int i = 0; i < P; ++i) acc += c->Im[h0][u * P + i] * tr[FIDX(v, B, fB, i, ne, nf, nfp)];
            } else {
                for (int j = 0; j < P; ++j)
                    for (int i = 0; i < P; ++i)
                        acc += c->Im[h0][u * P + i] * c->Im[h1][w * P + j] * tr[FIDX(v, B, fB, i + P * j, ne, nf, nfp)];
            }
            out[fp] = sg * acc;
        }
        return;
    }
    /* big side */
    int m = -100 - t[0];
    for (int fp = 0; fp < nfp; ++fp) out[fp] = 0.0;
    for (int p = 0; p < c->nsub; ++p) {
        const int *sb = c->mortar + ((size_t)m * c->nsub + p) * 3;
        long S = sb[0];
        int fS = sb[1], o = sb[2], h0 = p & 1, h1 = (p >> 1) & 1;
        double sg = (signed_ ? facing(f, fS) : 1.0) * scale;
        for (int fq = 0; fq < nfp; ++fq) {
            int q = map_fp(c, o, fq), u = q % P, w = q / P;
            double val = sg * tr[FIDX(v, S, fS, fq, ne, nf, nfp)];
            if (c->d == 2) {
                for (int i = 0; i < P; ++i) out[i] += c->Pm[h0][i * P + u] * val;
            } else {
                for (int j = 0; j < P; ++j)
                    for (int i = 0; i < P; ++i) out[i + P * j] += c->Pm[h0][i * P + u] * c->Pm[h1][j * P + w] * val;
            }
        }
    }
}

/* Wall table entry of face f of element e (box: f itself). */
static int wall_of(const ctx_t *c, long e, int f)
{
    if (c->conn) return -1 - c->conn[((size_t)e * 2 * c->d + f) * 3];
    return f;
}

/* ======================================================================== */
/* Curved elements: geometry and metric terms (Sec. 3.1)                     */
/* ======================================================================== */

/* Derivative of the Lagrange basis of the points t_0..t_n at x:
   l_j'(x) = sum_{m != j} 1/(t_j - t_m) prod_{k != j, m} (x - t_k)/(t_j - t_k). */
static void lagrange_deriv_at(int n, const double *t, double x, double *dl)
{
    for (int j = 0; j <= n; ++j) {
        double s = 0.0;
        for (int m = 0; m <= n; ++m) {
            if (m == j) continue;
            double prod = 1.0 / (t[j] - t[m]);
            for (int k = 0; k <= n; ++k)
                if (k != j && k != m) prod *= (x - t[k]) / (t[j] - t[k]);
            s += prod;
        }
        dl[j] = s;
    }
}

/* Position X and derivatives dX[j][k] = d X_k / d xi_j of element e's map at the
   reference point xi (interpolation of the caller's equispaced geometry points). */
static void geo_eval(const ctx_t *c, long e, const double *xi, double *X, double dX[3][3])
{
    int G = c->ngeo + 1, d = c->d, ng = ipow(G, d);
    double t[MAXG], l[3][MAXG], dl[3][MAXG];
    for (int a = 0; a < G; ++a) t[a] = -1.0 + 2.0 * a / c->ngeo;
    for (int j = 0; j < d; ++j) {
        or_lagrange_at(c->ngeo, t, xi[j], l[j]);
        lagrange_deriv_at(c->ngeo, t, xi[j], dl[j]);
    }
    for (int k = 0; k < 3; ++k) {
        X[k] = 0.0;
        for (int j = 0; j < 3; ++j) dX[j][k] = 0.0;
    }
    for (int g = 0; g < ng; ++g) {
        int a[3] = {g % G, (g / G) % G, g / (G * G)};
        for (int k = 0; k < d; ++k) {
            double x = c->xgeo[((size_t)k * c->ne + e) * ng + g];
            double wv = 1.0;
            for (int j = 0; j < d; ++j) wv *= l[j][a[j]];
            X[k] += wv * x;
            for (int j = 0; j < d; ++j) {
                double wd = 1.0;
                for (int jj = 0; jj < d; ++jj) wd *= (jj == j) ? dl[jj][a[jj]] : l[jj][a[jj]];
                dX[j][k] += wd * x;
            }
        }
    }
}

/* Metric terms of the map at one point: J a^i = dX/dxi_{i+1} x dX/dxi_{i+2} (cyclic;
   in 2D J a^1 = (y_eta, -x_eta), J a^2 = (-y_xi, x_xi)), returned in Ja[i][k], and the
   Jacobian J = dX/dxi_1 . (J a^1).  For a map of degree ngeo these are polynomials of
   degree <= 2 ngeo (3D) or ngeo (2D) per direction, so with 2 ngeo <= N (ngeo <= N) they
   satisfy the discrete metric identities sum_i D (J a^i) = 0 exactly. */
static double cofactor(int d, double dX[3][3], double Ja[3][3])
{
    if (d == 2) {
        Ja[0][0] = dX[1][1];
        Ja[0][1] = -dX[1][0];
        Ja[1][0] = -dX[0][1];
        Ja[1][1] = dX[0][0];
        return dX[0][0] * dX[1][1] - dX[1][0] * dX[0][1];
    }
    for (int i = 0; i < 3; ++i) {
        const double *a = dX[(i + 1) % 3], *b = dX[(i + 2) % 3];
        Ja[i][0] = a[1] * b[2] - a[2] * b[1];
        Ja[i][1] = a[2] * b[0] - a[0] * b[2];
        Ja[i][2] = a[0] * b[1] - a[1] * b[0];
    }
    return dX[0][0] * Ja[0][0] + dX[0][1] * Ja[0][1] + dX[0][2] * Ja[0][2];
}

/* Node coordinates, J a^dir at the nodes and at the face points, J at the nodes.  A face
   shared by two elements takes the face metric of the element on its minus side (the
   element whose plus face it is), so that both elements see one normal and one surface
   element (conservation). */
static int setup_curved(ctx_t *c)
{
    long ne = c->ne;
    int np = c->np, d = c->d, nf = 2 * d, nfp = c->nfp;
    c->Ja = (double *)malloc(sizeof(double) * ne * np * 9);
    c->Jn = (double *)malloc(sizeof(double) * ne * np);
    c->Jf = (double *)malloc(sizeof(double) * ne * nf * nfp * 3);
    c->xn = (double *)malloc(sizeof(double) * ne * np * 3);
    if (!c->Ja || !c->Jn || !c->Jf || !c->xn) { teardown(c); return -2; }
    int bad = 0;
    for (long e = 0; e < ne; ++e) {
        for (int n = 0; n < np; ++n) {
            double xi[3] = {0, 0, 0}, X[3], dX[3][3], Ja[3][3];
            for (int k = 0; k < d; ++k) xi[k] = c->xi[ncoord(c, n, k)];
            geo_eval(c, e, xi, X, dX);
            double J = cofactor(d, dX, Ja);
            if (!(J > 0.0)) bad = 1;
            c->Jn[(size_t)e * np + n] = J;
            for (int i = 0; i < 3; ++i) {
                c->xn[((size_t)e * np + n) * 3 + i] = X[i];
                for (int k = 0; k < 3; ++k) c->Ja[(((size_t)e * np + n) * 3 + i) * 3 + k] = Ja[i][k];
            }
        }
        for (int f = 0; f < nf; ++f) {
            int dir = f / 2, s = f % 2;
            if (!c->conn && s == 0 && neighbour(c, e, dir, 0) >= 0) continue;
            for (int fp = 0; fp < nfp; ++fp) {
                int n0 = fp_to_node(c, fp, dir, 0);
                double xi[3] = {0, 0, 0}, X[3], dX[3][3], Ja[3][3];
                for (int k = 0; k < d; ++k) xi[k] = c->xi[ncoord(c, n0, k)];
                xi[dir] = s ? 1.0 : -1.0;
                geo_eval(c, e, xi, X, dX);
                cofactor(d, dX, Ja);
                for (int k = 0; k < 3; ++k) c->Jf[(((size_t)e * nf + f) * nfp + fp) * 3 + k] = Ja[dir][k];
            }
        }
    }
    if (c->conn) {
        /* unstructured: a shared face takes the metric of the element with the smaller
           index (of the smaller face for an element facing itself), in the other
           element's frame: the outward normals are opposite, J a^dir = nsign * outward */
        for (long e = 0; e < ne; ++e)
            for (int f = 0; f < nf; ++f) {
                long nb = neighbour(c, e, f / 2, f % 2);
                int fo = nb_face(c, e, f);
                if (face_kind(c, e, f) != F_CONF || nb < e || (nb == e && fo < f)) continue;
                double sg = -((f % 2) ? 1.0 : -1.0) * ((fo % 2) ? 1.0 : -1.0);
                for (int fp = 0; fp < nfp; ++fp) {
                    int fq = nb_fp(c, e, f, fp);
                    for (int k = 0; k < 3; ++k)
                        c->Jf[(((size_t)nb * nf + fo) * nfp + fq) * 3 + k] = sg * c->Jf[(((size_t)e * nf + f) * nfp + fp) * 3 + k];
                }
            }
    } else {
        for (long e = 0; e < ne; ++e)
            for (int dir = 0; dir < d; ++dir) {
                long nb = neighbour(c, e, dir, 0);
                if (nb < 0) continue;
                for (int fp = 0; fp < nfp; ++fp)
                    for (int k = 0; k < 3; ++k)
                        c->Jf[(((size_t)e * nf + 2 * dir) * nfp + fp) * 3 + k] =
                            c->Jf[(((size_t)nb * nf + 2 * dir + 1) * nfp + fp) * 3 + k];
            }
    }
    if (bad) { teardown(c); return -3; }
    return 0;
}

#define JA(c, e, n, i, k) ((c)->Ja[((((size_t)(e)) * (c)->np + (n)) * 3 + (i)) * 3 + (k)])
#define JN(c, e, n) ((c)->Jn[((size_t)(e)) * (c)->np + (n)])
#define JF(c, e, f, fp, k) ((c)->Jf[((((size_t)(e)) * 2 * (c)->d + (f)) * (c)->nfp + (fp)) * 3 + (k)])

/* trace of a nodal field of one element on face (d, s): sum_l l_l(+-1) f_l along lines */
static void trace_elem(const ctx_t *c, const double *f, int d, int s, double *out)
{
    const double *L = s ? c->lp : c->lm;
    for (int fp = 0; fp < c->nfp; ++fp) {
        double acc = 0.0;
        for (int l = 0; l < c->P; ++l) acc += L[l] * f[fp_to_node(c, fp, d, l)];
        out[fp] = acc;
    }
}

/* BR1 lifting in direction d (Sec. 3.1, weak form with collocated Gauss quadrature):
   g_i = (2/h_d) [ sum_l Dhat_il f_l + (l_i(+1) q*_+ - l_i(-1) q*_-) / w_i ] */
static void lift_elem(const ctx_t *c, const double *f, int d, const double *qm, const double *qp,
                      double *out)
{
    for (int n = 0; n < c->np; ++n) {
        int i = ncoord(c, n, d), fp = node_to_fp(c, n, d);
        double acc = 0.0;
        for (int l = 0; l < c->P; ++l) acc += c->Dhat[i * c->P + l] * f[fp_to_node(c, fp, d, l)];
        acc += (c->lp[i] * qp[fp] - c->lm[i] * qm[fp]) / c->w[i];
        out[n] = (2.0 / c->h[d]) * acc;
    }
}

/* ======================================================================== */
/* Point-wise model (Sec. 2.3)                                               */
/* ======================================================================== */

/* Index helpers into one node's or face point's local arrays.
   Conserved:  0 rho, 1..d momentum, d+1 rho*e, d+2 c (relaxation models)
   Lifted pass-1 variables (gradients g[dir*nl + v]): 0 rho, 1..d u_k, d+1 c (relaxation)
   For the original NSK model (model 0) "c" stands for rho itself. */

/* Temperature from the total energy, Eq. (totalenergyalpha) with the vdW internal energy
   rho eps = rho R cv T - a rho^2:
   rho eps = rho e - rho|u|^2/2 - alpha/2 (rho - c)^2 - gamma_K/2 |grad c|^2.
   For the original model the last two terms are replaced by gamma_K/2 |grad rho|^2. */
static double temperature(const ctx_t *c, const double *U, const double *g)
{
    const or_params *p = &c->prm;
    int d = c->d, nl = c->nl;
    double rho = U[0];
    double kin = 0.0;
    for (int k = 0; k < d; ++k) kin += U[1 + k] * U[1 + k];
    kin = 0.5 * kin / rho;
    int vc = (p->model == 0) ? 0 : d + 1;
    double g2 = 0.0;
    for (int k = 0; k < d; ++k) g2 += g[k * nl + vc] * g[k * nl + vc];
    double reps = U[d + 1] - kin - 0.5 * p->gammaK * g2;
    if (p->model != 0) {
        double dc = rho - U[d + 2];
        reps -= 0.5 * p->alpha * dc * dc;
    }
    return (reps + AV * rho * rho) / (rho * RV * p->cv);
}

/* Signal speed used by the Rusanov flux.  Relaxation models: sqrt(cs^2 + alpha rho), the
   sound speed of the modified pressure p + alpha/2 rho^2 (Sec. 2.3), used for both
   models.  Original NSK: sqrt(|cs^2|). */
static double sound_speed(const ctx_t *c, double rho, double T)
{
    const or_params *p = &c->prm;
    double s2 = or_cs2(rho, T, p->cv);
    if (p->model == 0) return sqrt(fabs(s2));
    s2 += p->alpha * rho;
    return s2 > 0.0 ? sqrt(s2) : 0.0;
}

/* Pressure entering the convective flux: p (models 0, 1) or p_alpha = p + alpha/2 rho^2
   (model 2, Eq. (modified_pressure)). */
static double flux_pressure(const ctx_t *c, double rho, double T)
{
    double pr = or_pressure(rho, T);
    if (c->prm.model == 2) pr += 0.5 * c->prm.alpha * rho * rho;
    return pr;
}

/* Convective flux F^C in direction dir (Eq. (navierstokeskorteweg_p)/(..._palpha)). */
static void conv_flux(const ctx_t *c, const double *U, double pr, int dir, double *F)
{
    int d = c->d;
    double u = U[1 + dir] / U[0];
    F[0] = U[1 + dir];
    for (int k = 0; k < d; ++k) F[1 + k] = U[1 + k] * u + (k == dir ? pr : 0.0);
    F[d + 1] = (U[d + 1] + pr) * u;
    if (c->prm.model != 0) F[d + 2] = U[d + 2] * u;
}

/* HLLC flux of the convective part in +e_dir (Toro, Riemann Solvers and Numerical
   Methods for Fluid Dynamics, 3rd ed., Sec. 10.4): wave-speed estimates
   S_L = min(u_L - a_L, u_R - a_R), S_R = max(u_L + a_L, u_R + a_R); contact speed
     S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R))
          / (rho_L (S_L - u_L) - rho_R (S_R - u_R));
   star states U*_K = chi_K (1, S* e_dir + tangential u_K, E_K/rho_K + (S* - u_K)(S* +
   p_K/(rho_K (S_K - u_K))), c_K/rho_K), chi_K = rho_K (S_K - u_K)/(S_K - S*), the order
   parameter carried like a passive scalar; F = F_L, F_L + S_L (U*_L - U_L),
   F_R + S_R (U*_R - U_R) or F_R by the sign pattern of S_L, S*, S_R.  p is the
   model's convective pressure (model 2: p + alpha/2 rho^2) and a its sound speed
   sqrt(cs^2 + alpha rho). */
static void hllc_flux(const ctx_t *c, const double *UL, double pL, double aL, const double *UR, double pR,
                      double aR, int dir, double *F)
{
    int d = c->d, nv = c->nv;
    double rL = UL[0], rR = UR[0];
    double uL = UL[1 + dir] / rL, uR = UR[1 + dir] / rR;
    double SL = fmin(uL - aL, uR - aR), SR = fmax(uL + aL, uR + aR);
    double FL[8], FR[8];
    conv_flux(c, UL, pL, dir, FL);
    conv_flux(c, UR, pR, dir, FR);
    if (SL >= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FL[v]; return; }
    if (SR <= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FR[v]; return; }
    double Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
    const double *UK = Ss >= 0.0 ? UL : UR;
    const double *FK = Ss >= 0.0 ? FL : FR;
    double SK = Ss >= 0.0 ? SL : SR, pK = Ss >= 0.0 ? pL : pR;
    double rK = UK[0], uK = UK[1 + dir] / rK;
    double chi = rK * (SK - uK) / (SK - Ss);
    double Us[8];
    Us[0] = chi;
    for (int k = 0; k < d; ++k) Us[1 + k] = chi * (k == dir ? Ss : UK[1 + k] / rK);
    Us[d + 1] = chi * (UK[d + 1] / rK + (Ss - uK) * (Ss + pK / (rK * (SK - uK))));
    Us[d + 2] = chi * UK[d + 2] / rK;
    for (int v = 0; v < nv; ++v) F[v] = FK[v] + SK * (Us[v] - UK[v]);
}

/* Convective flux along the vector a: sum_k a_k F^C_k. */
static void conv_along(const ctx_t *c, const double *U, double pr, const double *a, double *Fa)
{
    double F[8];
    for (int v = 0; v < c->nv; ++v) Fa[v] = 0.0;
    for (int k = 0; k < c->d; ++k) {
        conv_flux(c, U, pr, k, F);
        for (int v = 0; v < c->nv; ++v) Fa[v] += a[k] * F[v];
    }
}

/* HLLC flux along the unit normal nh (hllc_flux with e_dir replaced by nh): normal
   velocities u.n; the star states keep the tangential velocity,
   U*_K = chi_K (1, u_K + (S* - u_K.n) n, E_K/rho_K + (S* - u_K.n)(S* + p_K/(rho_K (S_K - u_K.n))),
   c_K/rho_K). */
static void hllc_normal(const ctx_t *c, const double *UL, double pL, double aL, const double *UR, double pR,
                        double aR, const double *nh, double *F)
{
    int d = c->d, nv = c->nv;
    double rL = UL[0], rR = UR[0], uL = 0.0, uR = 0.0;
    for (int k = 0; k < d; ++k) {
        uL += UL[1 + k] * nh[k];
        uR += UR[1 + k] * nh[k];
    }
    uL /= rL;
    uR /= rR;
    double SL = fmin(uL - aL, uR - aR), SR = fmax(uL + aL, uR + aR);
    double FL[8], FR[8];
    conv_along(c, UL, pL, nh, FL);
    conv_along(c, UR, pR, nh, FR);
    if (SL >= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FL[v]; return; }
    if (SR <= 0.0) { for (int v = 0; v < nv; ++v) F[v] = FR[v]; return; }
    double Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
    const double *UK = Ss >= 0.0 ? UL : UR;
    const double *FK = Ss >= 0.0 ? FL : FR;
    double SK = Ss >= 0.0 ? SL : SR, pK = Ss >= 0.0 ? pL : pR, uK = Ss >= 0.0 ? uL : uR;
    double rK = UK[0];
    double chi = rK * (SK - uK) / (SK - Ss);
    double Us[8];
    Us[0] = chi;
    for (int k = 0; k < d; ++k) Us[1 + k] = chi * (UK[1 + k] / rK + (Ss - uK) * nh[k]);
    Us[d + 1] = chi * (UK[d + 1] / rK + (Ss - uK) * (Ss + pK / (rK * (SK - uK))));
    Us[d + 2] = chi * UK[d + 2] / rK;
    for (int v = 0; v < nv; ++v) F[v] = FK[v] + SK * (Us[v] - UK[v]);
}

/* Viscous flux F^V in direction dir.
   Relaxation models (Eq. (navierstokeskorteweg_p)): (0, tau_{k,dir}, tau_{dir,k} u_k + j_e,
   gamma_K beta c_{x_dir}), with tau = mu (grad u + grad u^T - 2/3 div u I) (Stokes
   hypothesis) and the simplified energy flux
   j_e = kappa grad T - gamma_K c grad c div u + gamma_K grad c zeta_c,
   zeta_c = beta (gamma_K lap c + alpha (rho - c)).
   Original NSK (Eq. (navierstokeskorteweg), (cauchystressnsk), (energyfluxnsk)): the
   Korteweg stress gamma_K [(|grad rho|^2/2 + rho lap rho) I - grad rho (x) grad rho] is
   added to tau, and j_e = kappa grad T - gamma_K rho grad rho div u. */
static void visc_flux(const ctx_t *c, const double *U, const double *g, const double *gT,
                      double lap, int dir, double *F)
{
    const or_params *p = &c->prm;
    int d = c->d, nl = c->nl;
    double rho = U[0];
    double u[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) u[k] = U[1 + k] / rho;
    /* du[i][k] = d u_k / d x_i */
    double du[3][3] = {{0}};
    for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) du[i][k] = g[i * nl + 1 + k];
    double divu = 0.0;
    for (int k = 0; k < d; ++k) divu += du[k][k];
    double tau[3];
    for (int k = 0; k < d; ++k)
        tau[k] = p->mu * (du[dir][k] + du[k][dir] - (k == dir ? 2.0 / 3.0 * divu : 0.0));
    if (p->model == 0) {
        double gr2 = 0.0;
        for (int k = 0; k < d; ++k) gr2 += g[k * nl] * g[k * nl];
        for (int k = 0; k < d; ++k) {
            double tk = -p->gammaK * g[k * nl] * g[dir * nl];
            if (k == dir) tk += p->gammaK * (0.5 * gr2 + rho * lap);
            tau[k] += tk;
        }
        double je = p->kappa * gT[dir] - p->gammaK * rho * g[dir * nl] * divu;
        F[0] = 0.0;
        double work = 0.0;
        for (int k = 0; k < d; ++k) { F[1 + k] = tau[k]; work += tau[k] * u[k]; }
        F[d + 1] = work + je;
        return;
    }
    double cc = U[d + 2];
    double gc = g[dir * nl + d + 1];
    double zeta = p->beta * (p->gammaK * lap + p->alpha * (rho - cc));
    double je = p->kappa * gT[dir] - p->gammaK * cc * gc * divu + p->gammaK * gc * zeta;
    F[0] = 0.0;
    double work = 0.0;
    for (int k = 0; k < d; ++k) { F[1 + k] = tau[k]; work += tau[k] * u[k]; }
    F[d + 1] = work + je;
    F[d + 2] = p->gammaK * p->beta * gc;
}

/* Point-wise non-conservative source S (Eq. (navierstokeskorteweg_p) for model 1,
   Eq. (navierstokeskorteweg_palpha) for model 2), evaluated with the lifted gradients.
   The third momentum row of model 2 is read as alpha rho c_{x_3} (printed c_{x_2}). */
static void source(const ctx_t *c, const double *U, const double *g, double *S)
{
    const or_params *p = &c->prm;
    int d = c->d, nl = c->nl;
    for (int v = 0; v < c->nv; ++v) S[v] = 0.0;
    if (p->model == 0) return;
    double rho = U[0], cc = U[d + 2];
    double u[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) u[k] = U[1 + k] / rho;
    double divu = 0.0;
    for (int k = 0; k < d; ++k) divu += g[k * nl + 1 + k];
    double gc2 = 0.0, cc_du = 0.0;
    for (int k = 0; k < d; ++k) gc2 += g[k * nl + d + 1] * g[k * nl + d + 1];
    /* grad c (x) grad c : grad (x) u = sum_ij c_i c_j du_j/dx_i */
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) cc_du += g[i * nl + d + 1] * g[j * nl + d + 1] * g[i * nl + 1 + j];
    double korteweg = p->gammaK * (0.5 * gc2 * divu - cc_du);
    double work = 0.0;
    for (int k = 0; k < d; ++k) {
        double drive = (p->model == 1) ? (g[k * nl + d + 1] - g[k * nl]) : g[k * nl + d + 1];
        S[1 + k] = p->alpha * rho * drive;
        work += p->alpha * rho * drive * u[k];
    }
    if (p->model == 1) S[d + 1] = work + 0.5 * p->alpha * (cc * cc - rho * rho) * divu + korteweg;
    else               S[d + 1] = work + 0.5 * p->alpha * cc * cc * divu + korteweg;
    S[d + 2] = p->alpha * p->beta * (rho - cc);
}

/* ======================================================================== */
/* Right-hand side, Sec. 3.1                                                 */
/* ======================================================================== */


/* Pass-1 lifted variables: (rho, u_1..u_d, c) at the nodes; the original model lifts
   (rho, u_1..u_d). */
static void primitives(const ctx_t *c, const double *U, double *q)
{
    long ne = c->ne;
    int np = c->np, d = c->d;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e)
        for (int n = 0; n < np; ++n) {
            double rho = U[IDX(0, e, n, ne, np)];
            q[IDX(0, e, n, ne, np)] = rho;
            for (int k = 0; k < d; ++k) q[IDX(1 + k, e, n, ne, np)] = U[IDX(1 + k, e, n, ne, np)] / rho;
            if (c->prm.model != 0) q[IDX(d + 1, e, n, ne, np)] = U[IDX(d + 2, e, n, ne, np)];
        }
}

/* Traces of nl fields on all 2d faces of every element: tr[v][e][f][fp]. */
static void traces(const ctx_t *c, const double *q, int nvar, double *tr)
{
    long ne = c->ne;
    int np = c->np, nf = 2 * c->d, nfp = c->nfp;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e)
        for (int v = 0; v < nvar; ++v)
            for (int f = 0; f < nf; ++f)
                trace_elem(c, q + IDX(v, e, 0, ne, np), f / 2, f % 2, tr + FIDX(v, e, f, 0, ne, nf, nfp));
}

/* BR1 pass 1 (Sec. 3.1): central face values q* = (q- + q+)/2 of the interpolated nodal
   (rho, u, c); at a no-slip wall rho* = rho-, u* = the wall's velocity (zero unless the
   wall slides), c* = c- (Eq. (bc_assumptions)). */
static void lift_pass1(const ctx_t *c, const double *q, const double *tr, double *grad)
{
    long ne = c->ne;
    int np = c->np, nf = 2 * c->d, nfp = c->nfp, nl = c->nl, d = c->d;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e) {
        double qs[2][MAXP * MAXP];
        for (int dir = 0; dir < d; ++dir)
            for (int v = 0; v < nl; ++v) {
                for (int s = 0; s < 2; ++s) {
                    int f = 2 * dir + s, fo = 2 * dir + (1 - s);
                    long nb = neighbour(c, e, dir, s);
                    for (int fp = 0; fp < nfp; ++fp) {
                        double own = tr[FIDX(v, e, f, fp, ne, nf, nfp)];
                        if (nb >= 0) qs[s][fp] = 0.5 * (own + tr[FIDX(v, nb, fo, fp, ne, nf, nfp)]);
                        else if (v >= 1 && v <= d)
                            /* no-slip: u* = the wall's velocity; Navier slip: no normal
                               velocity, the tangential velocity of the fluid */
                            qs[s][fp] = (c->wall_kind[f] == 2 && v != 1 + dir) ? own : c->wall_u[f][v - 1];
                        else qs[s][fp] = own;
                    }
                }
                lift_elem(c, q + IDX(v, e, 0, ne, np), dir, qs[0], qs[1], grad + IDX(dir * nl + v, e, 0, ne, np));
            }
    }
}

/* gather one node's pass-1 gradients into g[dir*nl + v] */
static void gather_grad(const ctx_t *c, const double *grad, long e, int n, double *g)
{
    for (int dir = 0; dir < c->d; ++dir)
        for (int v = 0; v < c->nl; ++v) g[dir * c->nl + v] = grad[IDX(dir * c->nl + v, e, n, c->ne, c->np)];
}

static void node_temperature(const ctx_t *c, const double *U, const double *grad, double *T)
{
    long ne = c->ne;
    int np = c->np;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e)
        for (int n = 0; n < np; ++n) {
            double Ul[8], g[3 * 8];
            for (int v = 0; v < c->nv; ++v) Ul[v] = U[IDX(v, e, n, ne, np)];
            gather_grad(c, grad, e, n, g);
            T[(size_t)e * np + n] = temperature(c, Ul, g);
        }
}

/* Contact-angle boundary value of the wall-normal gradient of the order parameter,
   Eq. (bc_contactangle_alpha): grad c . n = (1/gamma_K) [gamma_1 div u- - dpsi_wall/dc]
   (gamma_1 = 0 at kind-1 walls). */
static double wall_gn(const ctx_t *c, int f, double cminus, double divu)
{
    double g1 = c->wall_kind[f] == 2 ? c->wall_g[f][0] : 0.0;
    return (g1 * divu - or_wall_dpsi_dc(cminus, c->wall_rv[f], c->wall_rl[f], c->wall_sigma[f], c->wall_theta[f]))
           / c->prm.gammaK;
}

/* BR1 pass 2: grad T (central T*, T* = T_wall at isothermal walls) and the Laplacian of
   the order parameter as the BR1 divergence of its lifted gradient (BR1 applied twice,
   Sec. 3.1); its face value is the central mean of the interpolated d c/dx_dir, and at a
   wall the contact-angle value n_dir * (grad c . n). */
static void lift_pass2(const ctx_t *c, const double *T, const double *grad, const double *trq,
                       double *gT, double *lap)
{
    long ne = c->ne;
    int np = c->np, nf = 2 * c->d, nfp = c->nfp, nl = c->nl, d = c->d;
    int vc = (c->prm.model == 0) ? 0 : d + 1;
    double *trT = (double *)malloc(sizeof(double) * ne * nf * nfp);
    double *trD = (double *)malloc(sizeof(double) * ne * nf * nfp);
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e)
        for (int f = 0; f < nf; ++f) {
            int dir = f / 2, s = f % 2;
            trace_elem(c, T + (size_t)e * np, dir, s, trT + ((size_t)e * nf + f) * nfp);
            trace_elem(c, grad + IDX(dir * nl + vc, e, 0, ne, np), dir, s, trD + ((size_t)e * nf + f) * nfp);
        }
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e) {
        double Ts[2][MAXP * MAXP], Ds[2][MAXP * MAXP], tmp[MAXP * MAXP * MAXP];
        for (int n = 0; n < np; ++n) lap[(size_t)e * np + n] = 0.0;
        for (int dir = 0; dir < d; ++dir) {
            for (int s = 0; s < 2; ++s) {
                int f = 2 * dir + s, fo = 2 * dir + (1 - s);
                long nb = neighbour(c, e, dir, s);
                for (int fp = 0; fp < nfp; ++fp) {
                    double tOwn = trT[((size_t)e * nf + f) * nfp + fp];
                    double dOwn = trD[((size_t)e * nf + f) * nfp + fp];
                    if (nb >= 0) {
                        Ts[s][fp] = 0.5 * (tOwn + trT[((size_t)nb * nf + fo) * nfp + fp]);
                        Ds[s][fp] = 0.5 * (dOwn + trD[((size_t)nb * nf + fo) * nfp + fp]);
                    } else {
                        double cm = trq[FIDX(vc, e, f, fp, ne, nf, nfp)];
                        /* isothermal wall: T* = T_wall; heat-transfer wall (kind 2): the
                           fluid's own trace, the wall heat flux enters the energy flux */
                        Ts[s][fp] = c->wall_kind[f] == 2 ? tOwn : c->wall_T[f];
                        double divu = 0.0;
                        if (c->wall_kind[f] == 2)
                            for (int k = 0; k < d; ++k) {
                                double tk[MAXP * MAXP];
                                trace_elem(c, grad + IDX(k * nl + 1 + k, e, 0, ne, np), dir, s, tk);
                                divu += tk[fp];
                            }
                        Ds[s][fp] = (s ? 1.0 : -1.0) * wall_gn(c, f, cm, divu);
                    }
                }
            }
            lift_elem(c, T + (size_t)e * np, dir, Ts[0], Ts[1], gT + IDX(dir, e, 0, ne, np));
            lift_elem(c, grad + IDX(dir * nl + vc, e, 0, ne, np), dir, Ds[0], Ds[1], tmp);
            for (int n = 0; n < np; ++n) lap[(size_t)e * np + n] += tmp[n];
        }
    }
    free(trT);
    free(trD);
}

/* Full flux F = F^C - F^V of one point in direction dir, and its Rusanov signal speed
   |u_dir| + s. */
static void point_flux(const ctx_t *c, const double *U, const double *g, const double *gT, double lap,
                       int dir, double *F, double *lam)
{
    double T = temperature(c, U, g);
    double pr = flux_pressure(c, U[0], T);
    double Fc[8], Fv[8];
    conv_flux(c, U, pr, dir, Fc);
    visc_flux(c, U, g, gT, lap, dir, Fv);
    for (int v = 0; v < c->nv; ++v) F[v] = Fc[v] - Fv[v];
    *lam = fabs(U[1 + dir] / U[0]) + sound_speed(c, U[0], T);
}

/* Numerical flux through a wall face in the outward normal direction n = nsign * e_dir
   (Sec. 2.4, Eq. (bc_nsk_alpha); kind 1: isothermal no-slip wall with static contact
   angle, gamma_1 = gamma_2 = gamma_4 = 0; kind 2: generalized Navier slip, below):
   convective part: Rusanov flux against the mirrored ghost state (rho, m - 2(m.n)n, rho e, c)
   with the same pressure and signal speed;
   viscous part: tau(grad u-).n, energy (tau(grad u-).n).u_wall + kappa grad T-.n
   - gamma_K c- (grad c.n) div u- (the work of the traction on the wall's velocity, zero
   unless the wall slides; zeta_c = 0 from the relaxation condition with gamma_4 = 0),
   order parameter gamma_K beta (grad c.n), with grad c.n from the contact-angle
   condition. */
static void wall_flux(const ctx_t *c, int f, const double *U, const double *g, const double *gT,
                      double *Fn)
{
    const or_params *p = &c->prm;
    int d = c->d, nl = c->nl, nv = c->nv;
    int dir = f / 2;
    double nsign = (f % 2) ? 1.0 : -1.0;
    double T = temperature(c, U, g);
    double pr = flux_pressure(c, U[0], T);
    double lam = fabs(U[1 + dir] / U[0]) + sound_speed(c, U[0], T);
    double Ug[8], FL[8], FR[8];
    for (int v = 0; v < nv; ++v) Ug[v] = U[v];
    Ug[1 + dir] = -U[1 + dir];
    conv_flux(c, U, pr, dir, FL);
    conv_flux(c, Ug, pr, dir, FR);
    double Fconv[8];
    /* flux in +e_dir computed as for an interior face with the ghost on the outside */
    if (p->flux == 1) {
        double a = sound_speed(c, U[0], T);
        if (nsign > 0) hllc_flux(c, U, pr, a, Ug, pr, a, dir, Fconv);
        else           hllc_flux(c, Ug, pr, a, U, pr, a, dir, Fconv);
    } else {
        for (int v = 0; v < nv; ++v) {
            double Fin = FL[v], Fout = FR[v], Uin = U[v], Uout = Ug[v];
            double Fl = nsign > 0 ? Fin : Fout, Fr = nsign > 0 ? Fout : Fin;
            double Ul = nsign > 0 ? Uin : Uout, Ur = nsign > 0 ? Uout : Uin;
            Fconv[v] = 0.5 * (Fl + Fr) - 0.5 * lam * (Ur - Ul);
        }
    }
    /* viscous normal flux, outward */
    double rho = U[0], cm = U[d + 2];
    double divu = 0.0;
    for (int k = 0; k < d; ++k) divu += g[k * nl + 1 + k];
    double gn = wall_gn(c, f, cm, divu);
    double Fv[8];
    Fv[0] = 0.0;
    if (c->wall_kind[f] == 2) {
        /* generalized Navier slip, Eq. (bc_nsk_alpha): the tangential traction is
           gamma_1 div u grad_wall c - gamma_2 u_t (Eq. (bc_navierstokes_alpha)), the normal
           traction that of the fluid; the wall moves with the fluid's tangential velocity,
           so the traction does work t . u_t; heat flux kappa grad T . n =
           -gamma_3 (1/T_wall - 1/T-) (Eq. (bc_energy_alpha)); zeta_c = -gamma_1 gamma_4 div u
           (Eq. (bc_relaxation_alpha)); grad c . n with the gamma_1 term. */
        double g1 = c->wall_g[f][0], g2 = c->wall_g[f][1], g3 = c->wall_g[f][2], g4 = c->wall_g[f][3];
        double work = 0.0;
        for (int k = 0; k < d; ++k) {
            double uk = U[1 + k] / rho;
            if (k == dir) {
                double tnn = p->mu * (2.0 * g[dir * nl + 1 + dir] - 2.0 / 3.0 * divu);
                Fv[1 + k] = tnn * nsign;
            } else {
                double tk = g1 * divu * g[k * nl + d + 1] - g2 * uk;
                Fv[1 + k] = tk;
                work += tk * uk;
            }
        }
        double zeta = -g1 * g4 * divu;
        double Tm = temperature(c, U, g);
        Fv[d + 1] = work - g3 * (1.0 / c->wall_T[f] - 1.0 / Tm) - p->gammaK * cm * gn * divu + p->gammaK * gn * zeta;
        Fv[d + 2] = p->gammaK * p->beta * gn;
    } else {
        for (int k = 0; k < d; ++k) {
            double tau = p->mu * (g[dir * nl + 1 + k] + g[k * nl + 1 + dir] - (k == dir ? 2.0 / 3.0 * divu : 0.0));
            Fv[1 + k] = tau * nsign;
        }
        double work = 0.0;
        for (int k = 0; k < d; ++k) work += Fv[1 + k] * c->wall_u[f][k];
        Fv[d + 1] = work + p->kappa * gT[dir] * nsign - p->gammaK * cm * gn * divu;
        Fv[d + 2] = p->gammaK * p->beta * gn;
    }
    /* outward normal flux = nsign * Fconv - Fv */
    for (int v = 0; v < nv; ++v) Fn[v] = nsign * Fconv[v] - Fv[v];
}

typedef struct {
    double *q, *trq, *grad, *T, *gT, *lap;
} work_t;

static int work_alloc(const ctx_t *c, work_t *w)
{
    size_t ne = c->ne, np = c->np, nf = 2 * c->d, nfp = c->nfp;
    w->q = (double *)malloc(sizeof(double) * c->nl * ne * np);
    w->trq = (double *)malloc(sizeof(double) * c->nl * ne * nf * nfp);
    w->grad = (double *)malloc(sizeof(double) * c->d * c->nl * ne * np);
    w->T = (double *)malloc(sizeof(double) * ne * np);
    w->gT = (double *)malloc(sizeof(double) * c->d * ne * np);
    w->lap = (double *)malloc(sizeof(double) * ne * np);
    return (w->q && w->trq && w->grad && w->T && w->gT && w->lap) ? 0 : -1;
}

static void work_free(work_t *w)
{
    free(w->q); free(w->trq); free(w->grad); free(w->T); free(w->gT); free(w->lap);
}

static void node_coord(const ctx_t *c, long e, int n, double *x)
{
    if (c->curved) {
        for (int d = 0; d < c->d; ++d) x[d] = c->xn[((size_t)e * c->np + n) * 3 + d];
        return;
    }
    long co[3];
    co[0] = e % c->n[0];
    co[1] = (e / c->n[0]) % c->n[1];
    co[2] = e / ((long)c->n[0] * c->n[1]);
    for (int d = 0; d < c->d; ++d)
        x[d] = c->lo[d] + c->h[d] * (co[d] + 0.5 * (c->xi[ncoord(c, n, d)] + 1.0));
}

static int rhs_core(const ctx_t *c, const double *U, double *Ut, double t, or_forcing_fn forcing, void *user)
{
    long ne = c->ne;
    int np = c->np, nf = 2 * c->d, nfp = c->nfp, nl = c->nl, nv = c->nv, d = c->d, P = c->P;
    work_t w;
    if (work_alloc(c, &w)) { work_free(&w); return -2; }

    /* 1. pass-1 lifted variables, their face traces, BR1 lifting */
    primitives(c, U, w.q);
    traces(c, w.q, nl, w.trq);
    lift_pass1(c, w.q, w.trq, w.grad);
    /* 2. temperature at the nodes from the total energy */
    node_temperature(c, U, w.grad, w.T);
    /* 3. pass 2: grad T and lap c */
    lift_pass2(c, w.T, w.grad, w.trq, w.gT, w.lap);

    /* 4. face traces of the conserved state and of all lifted quantities */
    int nq = nv + d * nl + d + 1; /* U, pass-1 gradients, grad T, lap */
    double *trall = (double *)malloc(sizeof(double) * (size_t)nq * ne * nf * nfp);
    if (!trall) { work_free(&w); return -2; }
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e)
        for (int f = 0; f < nf; ++f) {
            int dir = f / 2, s = f % 2;
            for (int v = 0; v < nv; ++v)
                trace_elem(c, U + IDX(v, e, 0, ne, np), dir, s, trall + FIDX(v, e, f, 0, ne, nf, nfp));
            for (int k = 0; k < d * nl; ++k)
                trace_elem(c, w.grad + IDX(k, e, 0, ne, np), dir, s, trall + FIDX(nv + k, e, f, 0, ne, nf, nfp));
            for (int k = 0; k < d; ++k)
                trace_elem(c, w.gT + IDX(k, e, 0, ne, np), dir, s, trall + FIDX(nv + d * nl + k, e, f, 0, ne, nf, nfp));
            trace_elem(c, w.lap + (size_t)e * np, dir, s, trall + FIDX(nv + d * nl + d, e, f, 0, ne, nf, nfp));
        }

    /* 5. volume integral and point-wise sources */
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e) {
        double (*F)[MAXP * MAXP * MAXP][8] = malloc(sizeof(double) * 3 * MAXP * MAXP * MAXP * 8);
        double Ul[8], g[24], gT[3], S[8];
        for (int n = 0; n < np; ++n) {
            for (int v = 0; v < nv; ++v) Ul[v] = U[IDX(v, e, n, ne, np)];
            gather_grad(c, w.grad, e, n, g);
            for (int k = 0; k < d; ++k) gT[k] = w.gT[IDX(k, e, n, ne, np)];
            double lap = w.lap[(size_t)e * np + n];
            for (int dir = 0; dir < d; ++dir) {
                double lam;
                point_flux(c, Ul, g, gT, lap, dir, F[dir][n], &lam);
            }
            source(c, Ul, g, S);
            for (int v = 0; v < nv; ++v) Ut[IDX(v, e, n, ne, np)] = S[v];
        }
        /* U_t,i -= sum_dir (2/h_dir) sum_l Dhat_il F_dir,l */
        for (int n = 0; n < np; ++n)
            for (int dir = 0; dir < d; ++dir) {
                int i = ncoord(c, n, dir), fp = node_to_fp(c, n, dir);
                for (int v = 0; v < nv; ++v) {
                    double acc = 0.0;
                    for (int l = 0; l < P; ++l) acc += c->Dhat[i * P + l] * F[dir][fp_to_node(c, fp, dir, l)][v];
                    Ut[IDX(v, e, n, ne, np)] -= (2.0 / c->h[dir]) * acc;
                }
            }
        free(F);
    }

    /* 6. surface integral: numerical flux in +e_dir on every face point, lifted to the
          nodes with l_i(+-1)/w_i; Rusanov flux for the convective part and the BR1
          central flux for the viscous part. */
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e) {
        for (int f = 0; f < nf; ++f) {
            int dir = f / 2, s = f % 2, fo = 2 * dir + (1 - s);
            long nb = neighbour(c, e, dir, s);
            for (int fp = 0; fp < nfp; ++fp) {
                double Uo[8], go[24], gTo[3], lapo;
                double Fstar[8];
                for (int v = 0; v < nv; ++v) Uo[v] = trall[FIDX(v, e, f, fp, ne, nf, nfp)];
                for (int k = 0; k < d * nl; ++k) go[k] = trall[FIDX(nv + k, e, f, fp, ne, nf, nfp)];
                for (int k = 0; k < d; ++k) gTo[k] = trall[FIDX(nv + d * nl + k, e, f, fp, ne, nf, nfp)];
                lapo = trall[FIDX(nv + d * nl + d, e, f, fp, ne, nf, nfp)];
                if (nb >= 0) {
                    double Un[8], gn[24], gTn[3], lapn;
                    for (int v = 0; v < nv; ++v) Un[v] = trall[FIDX(v, nb, fo, fp, ne, nf, nfp)];
                    for (int k = 0; k < d * nl; ++k) gn[k] = trall[FIDX(nv + k, nb, fo, fp, ne, nf, nfp)];
                    for (int k = 0; k < d; ++k) gTn[k] = trall[FIDX(nv + d * nl + k, nb, fo, fp, ne, nf, nfp)];
                    lapn = trall[FIDX(nv + d * nl + d, nb, fo, fp, ne, nf, nfp)];
                    const double *UL = s ? Uo : Un, *UR = s ? Un : Uo;
                    const double *gL = s ? go : gn, *gR = s ? gn : go;
                    const double *tL = s ? gTo : gTn, *tR = s ? gTn : gTo;
                    double lL = s ? lapo : lapn, lR = s ? lapn : lapo;
                    if (c->prm.flux == 1) {
                        /* HLLC for the convective part, central BR1 flux for the viscous part */
                        double TL = temperature(c, UL, gL), TR = temperature(c, UR, gR);
                        double Fc[8], FvL[8], FvR[8];
                        hllc_flux(c, UL, flux_pressure(c, UL[0], TL), sound_speed(c, UL[0], TL), UR,
                                  flux_pressure(c, UR[0], TR), sound_speed(c, UR[0], TR), dir, Fc);
                        visc_flux(c, UL, gL, tL, lL, dir, FvL);
                        visc_flux(c, UR, gR, tR, lR, dir, FvR);
                        for (int v = 0; v < nv; ++v) Fstar[v] = Fc[v] - 0.5 * (FvL[v] + FvR[v]);
                    } else {
                        double FL[8], FR[8], laL, laR;
                        point_flux(c, UL, gL, tL, lL, dir, FL, &laL);
                        point_flux(c, UR, gR, tR, lR, dir, FR, &laR);
                        double lam = laL > laR ? laL : laR;
                        for (int v = 0; v < nv; ++v) Fstar[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (UR[v] - UL[v]);
                    }
                } else {
                    double Fn[8];
                    wall_flux(c, f, Uo, go, gTo, Fn);
                    double nsign = s ? 1.0 : -1.0;
                    for (int v = 0; v < nv; ++v) Fstar[v] = nsign * Fn[v];
                }
                /* U_t,i -= (2/h) [l_i(+1) F*_+ - l_i(-1) F*_-] / w_i along the line */
                for (int l = 0; l < P; ++l) {
                    int n = fp_to_node(c, fp, dir, l);
                    double coef = s ? c->lp[l] / c->w[l] : -c->lm[l] / c->w[l];
                    for (int v = 0; v < nv; ++v) Ut[IDX(v, e, n, ne, np)] -= (2.0 / c->h[dir]) * coef * Fstar[v];
                }
            }
        }
    }

    /* 7. optional manufactured-solution forcing */
    if (forcing) {
#pragma omp parallel for schedule(static)
        for (long e = 0; e < ne; ++e)
            for (int n = 0; n < np; ++n) {
                double x[3] = {0, 0, 0}, q[8];
                node_coord(c, e, n, x);
                forcing(d, x, t, q, user);
                for (int v = 0; v < nv; ++v) Ut[IDX(v, e, n, ne, np)] += q[v];
            }
    }
    free(trall);
    work_free(&w);
    return 0;
}

/* ======================================================================== */
/* Right-hand side on curved elements (Sec. 3.1 with metric terms)           */
/* ======================================================================== */

/* BR1 gradient of one nodal field f of element e, strong (chain-rule) form: with
   D_il = l_l'(xi_i), f- the trace of f on a face and f* its face value,
     J d f/d x_k = sum_dir [ J a^dir_k (sum_l D_il f_l)
                             + l_i(+1)/w_i (f*_+ - f-_+) (J a^dir_k)_+
                             - l_i(-1)/w_i (f*_- - f-_-) (J a^dir_k)_- ],
   where _+ and _- are the face points of the line through node i along dir.  On an
   affine element this is the weak form of lift_elem (Gauss collocation sums by parts
   exactly).  fs[f * nfp + fp] holds f* on face f; out[k * np + n] = d f / d x_k. */
static void grad_curved(const ctx_t *c, long e, const double *f, const double *fs, double *out)
{
    int P = c->P, d = c->d, np = c->np, nfp = c->nfp;
    for (int n = 0; n < np; ++n) {
        double acc[3] = {0, 0, 0};
        for (int dir = 0; dir < d; ++dir) {
            int i = ncoord(c, n, dir), fp = node_to_fp(c, n, dir);
            double df = 0.0, tm = 0.0, tp = 0.0;
            for (int l = 0; l < P; ++l) {
                double x = f[fp_to_node(c, fp, dir, l)];
                df += c->Dm[i * P + l] * x;
                tm += c->lm[l] * x;
                tp += c->lp[l] * x;
            }
            double jp = c->lp[i] / c->w[i] * (fs[(2 * dir + 1) * nfp + fp] - tp);
            double jm = c->lm[i] / c->w[i] * (fs[(2 * dir) * nfp + fp] - tm);
            for (int k = 0; k < d; ++k)
                acc[k] += JA(c, e, n, dir, k) * df + jp * JF(c, e, 2 * dir + 1, fp, k) - jm * JF(c, e, 2 * dir, fp, k);
        }
        for (int k = 0; k < d; ++k) out[k * np + n] = acc[k] / JN(c, e, n);
    }
}

/* Outward unit normal and surface element of face point fp of face f of element e */
static double face_normal(const ctx_t *c, long e, int f, int fp, double *nh)
{
    double s2 = 0.0;
    for (int k = 0; k < c->d; ++k) s2 += JF(c, e, f, fp, k) * JF(c, e, f, fp, k);
    double sa = sqrt(s2), sg = (f % 2) ? 1.0 : -1.0;
    for (int k = 0; k < 3; ++k) nh[k] = k < c->d ? sg * JF(c, e, f, fp, k) / sa : 0.0;
    return sa;
}

/* BR1 pass 1 on curved elements: face values as in lift_pass1 (central; at a wall
   rho* = rho-, c* = c-, and u* the part of the wall's velocity (no slip) or of the fluid's
   velocity (Navier slip) tangential to the wall, u* = b - (b.n) n), gradients by
   grad_curved. */
static void lift_pass1_c(const ctx_t *c, const double *q, const double *tr, double *grad)
{
    long ne = c->ne;
    int np = c->np, nf = 2 * c->d, nfp = c->nfp, nl = c->nl, d = c->d;
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e) {
        double fs[6 * MAXP * MAXP], out[3 * MAXP * MAXP * MAXP];
        for (int v = 0; v < nl; ++v) {
            for (int f = 0; f < nf; ++f) {
                int wall = face_kind(c, e, f) == F_WALL;
                double nbt[MAXP * MAXP];
                if (!wall) nb_trace(c, tr, v, e, f, 1.0, 0, nbt);
                for (int fp = 0; fp < nfp; ++fp) {
                    double own = tr[FIDX(v, e, f, fp, ne, nf, nfp)];
                    if (!wall) fs[f * nfp + fp] = 0.5 * (own + nbt[fp]);
                    else if (v >= 1 && v <= d) {
                        int w = wall_of(c, e, f);
                        double nh[3], b[3], bn = 0.0;
                        face_normal(c, e, f, fp, nh);
                        for (int k = 0; k < d; ++k) {
                            b[k] = c->wall_kind[w] == 2 ? tr[FIDX(1 + k, e, f, fp, ne, nf, nfp)] : c->wall_u[w][k];
                            bn += b[k] * nh[k];
                        }
                        fs[f * nfp + fp] = b[v - 1] - bn * nh[v - 1];
                    } else fs[f * nfp + fp] = own;
                }
            }
            grad_curved(c, e, q + IDX(v, e, 0, ne, np), fs, out);
            for (int k = 0; k < d; ++k)
                for (int n = 0; n < np; ++n) grad[IDX(k * nl + v, e, n, ne, np)] = out[k * np + n];
        }
    }
}

/* BR1 pass 2 on curved elements: grad T (T* central; at walls T_wall, or the fluid's
   trace at a Navier-slip wall) and lap c = sum_k [BR1 gradient of the lifted
   d c/d x_k]_k, whose face values are the central means of the interpolated d c/d x_k;
   at a wall the interpolated gradient with its normal component replaced by the
   contact-angle value, g* = g- + (g_n - g-.n) n (only g*.n enters the lifting), with
   the gamma_1 div u- term of a Navier-slip wall (div u- traced from the pass-1
   gradients). */
static void lift_pass2_c(const ctx_t *c, const double *T, const double *grad, const double *trq,
                         double *gT, double *lap)
{
    long ne = c->ne;
    int np = c->np, nf = 2 * c->d, nfp = c->nfp, nl = c->nl, d = c->d;
    int vc = (c->prm.model == 0) ? 0 : d + 1;
    /* traces: trT[e][f][fp], trG[k][e][f][fp] */
    double *trT = (double *)malloc(sizeof(double) * ne * nf * nfp);
    double *trG = (double *)malloc(sizeof(double) * d * ne * nf * nfp);
    double *gJf = (double *)malloc(sizeof(double) * ne * nf * nfp); /* grad c . J a^dir on each face */
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e)
        for (int f = 0; f < nf; ++f) {
            int dir = f / 2, s = f % 2;
            trace_elem(c, T + (size_t)e * np, dir, s, trT + ((size_t)e * nf + f) * nfp);
            for (int k = 0; k < d; ++k)
                trace_elem(c, grad + IDX(k * nl + vc, e, 0, ne, np), dir, s, trG + FIDX(k, e, f, 0, ne, nf, nfp));
            for (int fp = 0; fp < nfp; ++fp) {
                double acc = 0.0;
                for (int k = 0; k < d; ++k) acc += trG[FIDX(k, e, f, fp, ne, nf, nfp)] * JF(c, e, f, fp, k);
                gJf[((size_t)e * nf + f) * nfp + fp] = acc;
            }
        }
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e) {
        double Ts[6 * MAXP * MAXP], Gs[3][6 * MAXP * MAXP], out[3 * MAXP * MAXP * MAXP];
        for (int f = 0; f < nf; ++f) {
            int fo = nb_face(c, e, f), kind = face_kind(c, e, f);
            long nb = neighbour(c, e, f / 2, f % 2);
            double nbT[MAXP * MAXP], nbD[MAXP * MAXP];
            if (kind != F_WALL) nb_trace(c, trT, 0, e, f, 1.0, 0, nbT);
            if (kind == F_SMALL || kind == F_BIG) nb_trace(c, gJf, 0, e, f, c->d == 2 ? 2.0 : 4.0, 1, nbD);
            for (int fp = 0; fp < nfp; ++fp) {
                double tOwn = trT[((size_t)e * nf + f) * nfp + fp];
                int fq = nb_fp(c, e, f, fp);
                if (kind != F_WALL) Ts[f * nfp + fp] = 0.5 * (tOwn + nbT[fp]);
                if (kind == F_CONF) {
                    for (int k = 0; k < d; ++k)
                        Gs[k][f * nfp + fp] = 0.5 * (trG[FIDX(k, e, f, fp, ne, nf, nfp)] +
                                                     trG[FIDX(k, nb, fo, fq, ne, nf, nfp)]);
                } else if (kind != F_WALL) {
                    /* mortar: (grad c)* . J a = (own + neighbour's, interpolated or
                       projected) / 2; only that product enters the lifting, so the face
                       value is the own trace shifted along J a */
                    double own = gJf[((size_t)e * nf + f) * nfp + fp], a2 = 0.0;
                    for (int k = 0; k < d; ++k) a2 += JF(c, e, f, fp, k) * JF(c, e, f, fp, k);
                    double dl = 0.5 * (nbD[fp] - own) / a2;
                    for (int k = 0; k < d; ++k) Gs[k][f * nfp + fp] = trG[FIDX(k, e, f, fp, ne, nf, nfp)] + dl * JF(c, e, f, fp, k);
                } else {
                    double nh[3], gm[3] = {0, 0, 0}, gmn = 0.0;
                    face_normal(c, e, f, fp, nh);
                    for (int k = 0; k < d; ++k) {
                        gm[k] = trG[FIDX(k, e, f, fp, ne, nf, nfp)];
                        gmn += gm[k] * nh[k];
                    }
                    int w = wall_of(c, e, f);
                    double divu = 0.0;
                    if (c->wall_kind[w] == 2)
                        for (int k = 0; k < d; ++k) {
                            double tk[MAXP * MAXP];
                            trace_elem(c, grad + IDX(k * nl + 1 + k, e, 0, ne, np), f / 2, f % 2, tk);
                            divu += tk[fp];
                        }
                    double gn = wall_gn(c, w, trq[FIDX(vc, e, f, fp, ne, nf, nfp)], divu);
                    Ts[f * nfp + fp] = c->wall_kind[w] == 2 ? tOwn : c->wall_T[w];
                    for (int k = 0; k < d; ++k) Gs[k][f * nfp + fp] = gm[k] + (gn - gmn) * nh[k];
                }
            }
        }
        grad_curved(c, e, T + (size_t)e * np, Ts, out);
        for (int k = 0; k < d; ++k)
            for (int n = 0; n < np; ++n) gT[IDX(k, e, n, ne, np)] = out[k * np + n];
        for (int n = 0; n < np; ++n) lap[(size_t)e * np + n] = 0.0;
        for (int k = 0; k < d; ++k) {
            grad_curved(c, e, grad + IDX(k * nl + vc, e, 0, ne, np), Gs[k], out);
            for (int n = 0; n < np; ++n) lap[(size_t)e * np + n] += out[k * np + n];
        }
    }
    free(trT);
    free(trG);
    free(gJf);
}

/* F . a = sum_k a_k F_k of the full flux F = F^C - F^V along the vector a, from the
   Cartesian point fluxes; lam = |u.a| + s |a| (the Rusanov signal speed along a). */
static void flux_along(const ctx_t *c, const double *U, const double *g, const double *gT, double lap,
                       const double *a, double *Fa, double *lam)
{
    int d = c->d, nv = c->nv;
    double F[8], l, un = 0.0, an = 0.0;
    for (int v = 0; v < nv; ++v) Fa[v] = 0.0;
    for (int k = 0; k < d; ++k) {
        point_flux(c, U, g, gT, lap, k, F, &l);
        for (int v = 0; v < nv; ++v) Fa[v] += a[k] * F[v];
        un += a[k] * U[1 + k] / U[0];
        an += a[k] * a[k];
    }
    *lam = fabs(un) + sound_speed(c, U[0], temperature(c, U, g)) * sqrt(an);
}

/* Outward normal flux through a wall with unit outward normal nh, per unit area
   (wall_flux for a general normal): Rusanov against the ghost (rho, m - 2(m.n)n, rho e, c)
   with equal pressure and signal speed, minus the viscous flux.  Kind 1 (no slip):
   tau(grad u-).n, (tau n).u_w + kappa grad T-.n - gamma_K c- g_n div u-, gamma_K beta g_n,
   with u_w the wall's velocity projected on the tangent plane.  Kind 2 (Navier slip,
   Eq. (bc_nsk_alpha)): the normal traction (n.tau n) n of the fluid plus the tangential
   traction t = gamma_1 div u- (grad c- - (grad c-.n) n) - gamma_2 (u- - (u-.n) n), its work
   t.u-, the heat flux -gamma_3 (1/T_wall - 1/T-), zeta_c = -gamma_1 gamma_4 div u-, and
   g_n with the gamma_1 term. */
static void wall_flux_c(const ctx_t *c, int f, const double *U, const double *g, const double *gT,
                        const double *nh, double *Fn)
{
    const or_params *p = &c->prm;
    int d = c->d, nl = c->nl, nv = c->nv;
    double T = temperature(c, U, g);
    double pr = flux_pressure(c, U[0], T);
    double a = sound_speed(c, U[0], T);
    double mn = 0.0;
    for (int k = 0; k < d; ++k) mn += U[1 + k] * nh[k];
    double lam = fabs(mn / U[0]) + a;
    double Ug[8], Fi[8], Fg[8], F[8];
    for (int v = 0; v < nv; ++v) { Ug[v] = U[v]; Fi[v] = Fg[v] = 0.0; }
    for (int k = 0; k < d; ++k) Ug[1 + k] = U[1 + k] - 2.0 * mn * nh[k];
    for (int k = 0; k < d; ++k) {
        conv_flux(c, U, pr, k, F);
        for (int v = 0; v < nv; ++v) Fi[v] += nh[k] * F[v];
        conv_flux(c, Ug, pr, k, F);
        for (int v = 0; v < nv; ++v) Fg[v] += nh[k] * F[v];
    }
    double Fc[8];
    if (p->flux == 1) {
        /* HLLC against the ghost along the outward normal, the fluid on the left */
        hllc_normal(c, U, pr, a, Ug, pr, a, nh, Fc);
    } else {
        for (int v = 0; v < nv; ++v) Fc[v] = 0.5 * (Fi[v] + Fg[v]) - 0.5 * lam * (Ug[v] - U[v]);
    }
    double divu = 0.0;
    for (int k = 0; k < d; ++k) divu += g[k * nl + 1 + k];
    double cm = U[d + 2];
    double gn = wall_gn(c, f, cm, divu);
    double Fv[8];
    Fv[0] = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = 0.0;
        for (int j = 0; j < d; ++j)
            t += p->mu * (g[j * nl + 1 + k] + g[k * nl + 1 + j] - (k == j ? 2.0 / 3.0 * divu : 0.0)) * nh[j];
        Fv[1 + k] = t;
    }
    if (c->wall_kind[f] == 2) {
        double g1 = c->wall_g[f][0], g2 = c->wall_g[f][1], g3 = c->wall_g[f][2], g4 = c->wall_g[f][3];
        double tnn = 0.0, gcn = 0.0, un = 0.0, work = 0.0, u[3];
        for (int k = 0; k < d; ++k) {
            u[k] = U[1 + k] / U[0];
            tnn += Fv[1 + k] * nh[k];
            gcn += g[k * nl + d + 1] * nh[k];
            un += u[k] * nh[k];
        }
        for (int k = 0; k < d; ++k) {
            double tk = g1 * divu * (g[k * nl + d + 1] - gcn * nh[k]) - g2 * (u[k] - un * nh[k]);
            Fv[1 + k] = tnn * nh[k] + tk;
            work += tk * u[k];
        }
        double zeta = -g1 * g4 * divu;
        Fv[d + 1] = work - g3 * (1.0 / c->wall_T[f] - 1.0 / T) - p->gammaK * cm * gn * divu + p->gammaK * gn * zeta;
        Fv[d + 2] = p->gammaK * p->beta * gn;
    } else {
        double gTn = 0.0, uwn = 0.0, work = 0.0;
        for (int k = 0; k < d; ++k) {
            gTn += gT[k] * nh[k];
            uwn += c->wall_u[f][k] * nh[k];
        }
        for (int k = 0; k < d; ++k) work += Fv[1 + k] * (c->wall_u[f][k] - uwn * nh[k]);
        Fv[d + 1] = work + p->kappa * gTn - p->gammaK * cm * gn * divu;
        Fv[d + 2] = p->gammaK * p->beta * gn;
    }
    for (int v = 0; v < nv; ++v) Fn[v] = Fc[v] - Fv[v];
}

/* rhs_core on curved elements: the same stages with the metric terms,
   U_t,i = S_i - (1/J_i) sum_dir [ sum_l Dhat_il (F . J a^dir)_l
                                   + l_i(+1)/w_i F~*_+ - l_i(-1)/w_i F~*_- ],
   with F~* the numerical flux along the face metric J a^dir (oriented along +xi_dir):
   Rusanov F~* = (F_L.Ja + F_R.Ja)/2 - max(lam_L, lam_R)/2 (U_R - U_L), lam = |u.Ja| + s|Ja|
   (L on the minus side of the face), and at a wall |Ja| times the outward wall flux. */
/* Rusanov flux along the face metric J a at the points of face f of element e (a
   conforming face or the small side of a mortar): from the element's own traced record
   (U, pass-1 gradients, grad T, lap c) and the neighbour's, at the matching points or
   interpolated from the big face; F~* = (F_L . Ja + F_R . Ja)/2 - max(lam)/2 (U_R - U_L),
   L the minus side along +xi_dir. */
static void face_flux_pts(const ctx_t *c, const double *trall, int nq, long e, int f, double Fst[][MAXP * MAXP])
{
    long ne = c->ne;
    int nf = 2 * c->d, nfp = c->nfp, nl = c->nl, nv = c->nv, d = c->d, s = f % 2;
    double (*nbr)[MAXP * MAXP] = malloc(sizeof(double) * nq * MAXP * MAXP);
    for (int q = 0; q < nq; ++q) nb_trace(c, trall, q, e, f, 1.0, 0, nbr[q]);
    for (int fp = 0; fp < nfp; ++fp) {
        double Uo[8], go[24], gTo[3], lapo, Un[8], gn[24], gTn[3], lapn, a[3];
        for (int k = 0; k < 3; ++k) a[k] = JF(c, e, f, fp, k);
        for (int v = 0; v < nv; ++v) { Uo[v] = trall[FIDX(v, e, f, fp, ne, nf, nfp)]; Un[v] = nbr[v][fp]; }
        for (int k = 0; k < d * nl; ++k) { go[k] = trall[FIDX(nv + k, e, f, fp, ne, nf, nfp)]; gn[k] = nbr[nv + k][fp]; }
        for (int k = 0; k < d; ++k) {
            gTo[k] = trall[FIDX(nv + d * nl + k, e, f, fp, ne, nf, nfp)];
            gTn[k] = nbr[nv + d * nl + k][fp];
        }
        lapo = trall[FIDX(nv + d * nl + d, e, f, fp, ne, nf, nfp)];
        lapn = nbr[nv + d * nl + d][fp];
        const double *UL = s ? Uo : Un, *UR = s ? Un : Uo;
        const double *gL = s ? go : gn, *gR = s ? gn : go;
        const double *tL = s ? gTo : gTn, *tR = s ? gTn : gTo;
        double lL = s ? lapo : lapn, lR = s ? lapn : lapo;
        double FL[8], FR[8], laL, laR;
        flux_along(c, UL, gL, tL, lL, a, FL, &laL);
        flux_along(c, UR, gR, tR, lR, a, FR, &laR);
        if (c->prm.flux == 1) {
            /* HLLC for the convective part along the unit normal (times the surface
               element), central for the viscous part: F^V . a = F^C . a - F . a */
            double TL = temperature(c, UL, gL), TR = temperature(c, UR, gR), sa = 0.0, nh[3] = {0, 0, 0};
            for (int k = 0; k < d; ++k) sa += a[k] * a[k];
            sa = sqrt(sa);
            for (int k = 0; k < d; ++k) nh[k] = a[k] / sa;
            double pL = flux_pressure(c, UL[0], TL), pR = flux_pressure(c, UR[0], TR), Fh[8], CL[8], CR[8];
            hllc_normal(c, UL, pL, sound_speed(c, UL[0], TL), UR, pR, sound_speed(c, UR[0], TR), nh, Fh);
            conv_along(c, UL, pL, a, CL);
            conv_along(c, UR, pR, a, CR);
            for (int v = 0; v < nv; ++v) Fst[v][fp] = sa * Fh[v] - 0.5 * ((CL[v] - FL[v]) + (CR[v] - FR[v]));
        } else {
            double lam = laL > laR ? laL : laR;
            for (int v = 0; v < nv; ++v) Fst[v][fp] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (UR[v] - UL[v]);
        }
    }
    free(nbr);
}

static int rhs_core_c(const ctx_t *c, const double *U, double *Ut, double t, or_forcing_fn forcing, void *user)
{
    long ne = c->ne;
    int np = c->np, nf = 2 * c->d, nfp = c->nfp, nl = c->nl, nv = c->nv, d = c->d, P = c->P;
    work_t w;
    if (work_alloc(c, &w)) { work_free(&w); return -2; }
    primitives(c, U, w.q);
    traces(c, w.q, nl, w.trq);
    lift_pass1_c(c, w.q, w.trq, w.grad);
    node_temperature(c, U, w.grad, w.T);
    lift_pass2_c(c, w.T, w.grad, w.trq, w.gT, w.lap);

    int nq = nv + d * nl + d + 1;
    double *trall = (double *)malloc(sizeof(double) * (size_t)nq * ne * nf * nfp);
    if (!trall) { work_free(&w); return -2; }
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e)
        for (int f = 0; f < nf; ++f) {
            int dir = f / 2, s = f % 2;
            for (int v = 0; v < nv; ++v)
                trace_elem(c, U + IDX(v, e, 0, ne, np), dir, s, trall + FIDX(v, e, f, 0, ne, nf, nfp));
            for (int k = 0; k < d * nl; ++k)
                trace_elem(c, w.grad + IDX(k, e, 0, ne, np), dir, s, trall + FIDX(nv + k, e, f, 0, ne, nf, nfp));
            for (int k = 0; k < d; ++k)
                trace_elem(c, w.gT + IDX(k, e, 0, ne, np), dir, s, trall + FIDX(nv + d * nl + k, e, f, 0, ne, nf, nfp));
            trace_elem(c, w.lap + (size_t)e * np, dir, s, trall + FIDX(nv + d * nl + d, e, f, 0, ne, nf, nfp));
        }

    /* volume integral of the contravariant fluxes and point-wise sources */
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e) {
        double (*F)[MAXP * MAXP * MAXP][8] = malloc(sizeof(double) * 3 * MAXP * MAXP * MAXP * 8);
        double Ul[8], g[24], gT[3], S[8];
        for (int n = 0; n < np; ++n) {
            for (int v = 0; v < nv; ++v) Ul[v] = U[IDX(v, e, n, ne, np)];
            gather_grad(c, w.grad, e, n, g);
            for (int k = 0; k < d; ++k) gT[k] = w.gT[IDX(k, e, n, ne, np)];
            double lap = w.lap[(size_t)e * np + n];
            for (int dir = 0; dir < d; ++dir) {
                double a[3], lam;
                for (int k = 0; k < 3; ++k) a[k] = JA(c, e, n, dir, k);
                flux_along(c, Ul, g, gT, lap, a, F[dir][n], &lam);
            }
            source(c, Ul, g, S);
            for (int v = 0; v < nv; ++v) Ut[IDX(v, e, n, ne, np)] = S[v];
        }
        for (int n = 0; n < np; ++n)
            for (int dir = 0; dir < d; ++dir) {
                int i = ncoord(c, n, dir), fp = node_to_fp(c, n, dir);
                for (int v = 0; v < nv; ++v) {
                    double acc = 0.0;
                    for (int l = 0; l < P; ++l) acc += c->Dhat[i * P + l] * F[dir][fp_to_node(c, fp, dir, l)][v];
                    Ut[IDX(v, e, n, ne, np)] -= acc / JN(c, e, n);
                }
            }
        free(F);
    }

    /* surface integral: F~* at the points of every face (walls: the wall flux; big sides
       of mortars: the projection of the sub-faces' fluxes), lifted to the nodes */
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e) {
        for (int f = 0; f < nf; ++f) {
            int dir = f / 2, s = f % 2, kind = face_kind(c, e, f);
            double Fst[8][MAXP * MAXP];
            if (kind == F_WALL) {
                for (int fp = 0; fp < nfp; ++fp) {
                    double Uo[8], go[24], gTo[3], nh[3], Fn[8];
                    for (int v = 0; v < nv; ++v) Uo[v] = trall[FIDX(v, e, f, fp, ne, nf, nfp)];
                    for (int k = 0; k < d * nl; ++k) go[k] = trall[FIDX(nv + k, e, f, fp, ne, nf, nfp)];
                    for (int k = 0; k < d; ++k) gTo[k] = trall[FIDX(nv + d * nl + k, e, f, fp, ne, nf, nfp)];
                    double sa = face_normal(c, e, f, fp, nh);
                    wall_flux_c(c, wall_of(c, e, f), Uo, go, gTo, nh, Fn);
                    for (int v = 0; v < nv; ++v) Fst[v][fp] = (s ? 1.0 : -1.0) * sa * Fn[v];
                }
            } else if (kind == F_BIG) {
                /* the sub-faces' fluxes, as their elements compute them, turned to this
                   face's orientation and surface element (x 2^(d-1)) and projected */
                int m = -100 - c->conn[((size_t)e * nf + f) * 3], P_ = c->P;
                for (int v = 0; v < nv; ++v)
                    for (int fp = 0; fp < nfp; ++fp) Fst[v][fp] = 0.0;
                for (int p = 0; p < c->nsub; ++p) {
                    const int *sb = c->mortar + ((size_t)m * c->nsub + p) * 3;
                    double Fs[8][MAXP * MAXP];
                    face_flux_pts(c, trall, nq, sb[0], sb[1], Fs);
                    double sg = facing(f, sb[1]) * (d == 2 ? 2.0 : 4.0);
                    int h0 = p & 1, h1 = (p >> 1) & 1;
                    for (int fq = 0; fq < nfp; ++fq) {
                        int q = map_fp(c, sb[2], fq), u = q % P_, w = q / P_;
                        for (int v = 0; v < nv; ++v) {
                            double val = sg * Fs[v][fq];
                            if (d == 2) {
                                for (int i = 0; i < P_; ++i) Fst[v][i] += c->Pm[h0][i * P_ + u] * val;
                            } else {
                                for (int jj = 0; jj < P_; ++jj)
                                    for (int i = 0; i < P_; ++i)
                                        Fst[v][i + P_ * jj] += c->Pm[h0][i * P_ + u] * c->Pm[h1][jj * P_ + w] * val;
                            }
                        }
                    }
                }
            } else {
                face_flux_pts(c, trall, nq, e, f, Fst);
            }
            for (int fp = 0; fp < nfp; ++fp)
                for (int l = 0; l < P; ++l) {
                    int n = fp_to_node(c, fp, dir, l);
                    double coef = s ? c->lp[l] / c->w[l] : -c->lm[l] / c->w[l];
                    for (int v = 0; v < nv; ++v) Ut[IDX(v, e, n, ne, np)] -= coef * Fst[v][fp] / JN(c, e, n);
                }
        }
    }

    if (forcing) {
#pragma omp parallel for schedule(static)
        for (long e = 0; e < ne; ++e)
            for (int n = 0; n < np; ++n) {
                double x[3] = {0, 0, 0}, q[8];
                node_coord(c, e, n, x);
                forcing(d, x, t, q, user);
                for (int v = 0; v < nv; ++v) Ut[IDX(v, e, n, ne, np)] += q[v];
            }
    }
    free(trall);
    work_free(&w);
    return 0;
}

/* ======================================================================== */
/* Public entry points                                                       */
/* ======================================================================== */

int or_sizes(const or_mesh *m, const or_params *p, long *nelem, int *np, int *nv)
{
    ctx_t c;
    if (setup(m, p, &c)) return -1;
    *nelem = c.ne; *np = c.np; *nv = c.nv;
    teardown(&c);
    return 0;
}

int or_node_coords(const or_mesh *m, double *x)
{
    or_params p = {1, 1e-4, 0.01, 1.0 / 150.0, 5.0, 100.0, 100.0, 0};
    or_mesh mm = *m;
    for (int f = 0; f < 6; ++f) if (mm.wall_kind[f] != 0) mm.wall_T[f] = 0.85;
    ctx_t c;
    if (setup(&mm, &p, &c)) return -1;
    for (long e = 0; e < c.ne; ++e)
        for (int n = 0; n < c.np; ++n) {
            double xx[3];
            node_coord(&c, e, n, xx);
            for (int d = 0; d < c.d; ++d) x[IDX(d, e, n, c.ne, c.np)] = xx[d];
        }
    teardown(&c);
    return 0;
}

/* Conserved state from nodal (rho, u_1..u_d, T, c): the total energy of Eq.
   (totalenergyalpha) with grad c the BR1-lifted gradient of the given c, so that the
   temperature recovered by the scheme at t = 0 is the given T. */
int or_set_primitive(const or_mesh *m, const or_params *p, const double *prim, double *U)
{
    ctx_t c;
    if (setup(m, p, &c)) return -1;
    long ne = c.ne;
    int np = c.np, d = c.d, nv = c.nv;
    for (long e = 0; e < ne; ++e)
        for (int n = 0; n < np; ++n) {
            double rho = prim[IDX(0, e, n, ne, np)];
            U[IDX(0, e, n, ne, np)] = rho;
            for (int k = 0; k < d; ++k) U[IDX(1 + k, e, n, ne, np)] = rho * prim[IDX(1 + k, e, n, ne, np)];
            U[IDX(d + 1, e, n, ne, np)] = 0.0;
            if (p->model != 0) U[IDX(d + 2, e, n, ne, np)] = prim[IDX(d + 2, e, n, ne, np)];
        }
    work_t w;
    if (work_alloc(&c, &w)) { work_free(&w); teardown(&c); return -2; }
    primitives(&c, U, w.q);
    traces(&c, w.q, c.nl, w.trq);
    if (c.curved) lift_pass1_c(&c, w.q, w.trq, w.grad);
    else lift_pass1(&c, w.q, w.trq, w.grad);
    int vc = (p->model == 0) ? 0 : d + 1;
    for (long e = 0; e < ne; ++e)
        for (int n = 0; n < np; ++n) {
            double rho = prim[IDX(0, e, n, ne, np)], T = prim[IDX(d + 1, e, n, ne, np)];
            double kin = 0.0, g2 = 0.0;
            for (int k = 0; k < d; ++k) {
                double u = prim[IDX(1 + k, e, n, ne, np)];
                kin += rho * u * u;
                double gc = w.grad[IDX(k * c.nl + vc, e, n, ne, np)];
                g2 += gc * gc;
            }
            double E = or_inner_energy(rho, T, p->cv) + 0.5 * kin + 0.5 * p->gammaK * g2;
            if (p->model != 0) {
                double dc = rho - prim[IDX(d + 2, e, n, ne, np)];
                E += 0.5 * p->alpha * dc * dc;
            }
            U[IDX(d + 1, e, n, ne, np)] = E;
        }
    work_free(&w);
    teardown(&c);
    (void)nv;
    return 0;
}

int or_temperature(const or_mesh *m, const or_params *p, const double *U, double *T)
{
    ctx_t c;
    if (setup(m, p, &c)) return -1;
    work_t w;
    if (work_alloc(&c, &w)) { work_free(&w); teardown(&c); return -2; }
    primitives(&c, U, w.q);
    traces(&c, w.q, c.nl, w.trq);
    if (c.curved) lift_pass1_c(&c, w.q, w.trq, w.grad);
    else lift_pass1(&c, w.q, w.trq, w.grad);
    node_temperature(&c, U, w.grad, T);
    work_free(&w);
    teardown(&c);
    return 0;
}

int or_rhs(const or_mesh *m, const or_params *p, const double *U, double *Ut)
{
    return or_rhs_forced(m, p, U, Ut, 0.0, NULL, NULL);
}

int or_rhs_forced(const or_mesh *m, const or_params *p, const double *U, double *Ut, double t,
                  or_forcing_fn f, void *user)
{
    ctx_t c;
    if (setup(m, p, &c)) return -1;
    int rc = c.curved ? rhs_core_c(&c, U, Ut, t, f, user) : rhs_core(&c, U, Ut, t, f, user);
    teardown(&c);
    return rc;
}

/* Low-storage Runge-Kutta coefficients (Sec. 3.1; Kennedy & Carpenter):
   rk = 3: Williamson's three-stage third-order 2N scheme;
   rk = 4: Carpenter & Kennedy's five-stage fourth-order 2N scheme. */
int or_rk_coeffs(int rk, int *nstages, double *A, double *B, double *c)
{
    if (rk == 3) {
        const double a[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
        const double b[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
        const double cc[3] = {0.0, 1.0 / 3.0, 3.0 / 4.0};
        *nstages = 3;
        for (int s = 0; s < 3; ++s) { A[s] = a[s]; B[s] = b[s]; c[s] = cc[s]; }
        return 0;
    }
    if (rk == 4) {
        const double a[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                             -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
        const double b[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                             1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                             2277821191437.0 / 14882151754819.0};
        const double cc[5] = {0.0, 1432997174477.0 / 9575080441755.0, 2526269341429.0 / 6820363962896.0,
                              2006345519317.0 / 3224310063776.0, 2802321613138.0 / 2924317926251.0};
        *nstages = 5;
        for (int s = 0; s < 5; ++s) { A[s] = a[s]; B[s] = b[s]; c[s] = cc[s]; }
        return 0;
    }
    return -1;
}

/* nsteps explicit low-storage RK steps: per stage G = A_s G + dt U_t(U); U = U + B_s G. */
int or_run(const or_mesh *m, const or_params *p, double *U, int nsteps, double dt, int rk, double t0,
           or_forcing_fn f, void *user)
{
    ctx_t c;
    if (setup(m, p, &c)) return -1;
    int ns;
    double A[5], B[5], cs[5];
    if (or_rk_coeffs(rk, &ns, A, B, cs)) { teardown(&c); return -1; }
    size_t n = (size_t)c.nv * c.ne * c.np;
    double *G = (double *)calloc(n, sizeof(double));
    double *Ut = (double *)malloc(n * sizeof(double));
    if (!G || !Ut) { free(G); free(Ut); teardown(&c); return -2; }
    double t = t0;
    int rc = 0;
    for (int step = 0; step < nsteps && !rc; ++step) {
        for (int s = 0; s < ns; ++s) {
            rc = c.curved ? rhs_core_c(&c, U, Ut, t + cs[s] * dt, f, user)
                          : rhs_core(&c, U, Ut, t + cs[s] * dt, f, user);
            if (rc) break;
            for (size_t i = 0; i < n; ++i) {
                G[i] = A[s] * G[i] + dt * Ut[i];
                U[i] = U[i] + B[s] * G[i];
            }
        }
        t += dt;
    }
    free(G);
    free(Ut);
    teardown(&c);
    return rc;
}

/* Time step held fixed for a run: the smallest of a convective (CFL), a diffusive (DFL)
   and a relaxation-source bound, with the degree-dependent scaling 1/(2N+1) and the
   direction sums of Sec. 3.1's explicit scheme:
   dt_c = CFL / ((2N+1) max_nodes sum_d (|u_d| + s)/h_d)
   dt_v = DFL / ((2N+1)^2 nu_max sum_d 1/h_d^2),  nu = max(4 mu/(3 rho), kappa/(rho R cv), gamma_K beta)
   dt_s = 2 / (alpha beta).
   On curved elements the spacing along xi_dir at a node is h_dir = 2 J / |J a^dir| and the
   velocity along it u.(J a^dir)/|J a^dir|: the sums are taken per node,
   sum_dir (|u.J a^dir| + s |J a^dir|) / (2J) and sum_dir (|J a^dir| / (2J))^2 (both reduce
   to the box's). */
int or_max_dt(const or_mesh *m, const or_params *p, const double *U, double cfl, double dfl, double *dt)
{
    ctx_t c;
    if (setup(m, p, &c)) return -1;
    long ne = c.ne;
    int np = c.np, d = c.d;
    double *T = (double *)malloc(sizeof(double) * ne * np);
    if (!T) { teardown(&c); return -2; }
    or_temperature(m, p, U, T);
    double lmax = 0.0, numax = 0.0, ih2 = 0.0;
    for (long e = 0; e < ne; ++e)
        for (int n = 0; n < np; ++n) {
            double rho = U[IDX(0, e, n, ne, np)];
            double s = sound_speed(&c, rho, T[(size_t)e * np + n]);
            double lam = 0.0;
            if (c.curved) {
                double J2 = 2.0 * JN(&c, e, n), h2 = 0.0;
                for (int dir = 0; dir < d; ++dir) {
                    double un = 0.0, a2 = 0.0;
                    for (int k = 0; k < d; ++k) {
                        un += U[IDX(1 + k, e, n, ne, np)] / rho * JA(&c, e, n, dir, k);
                        a2 += JA(&c, e, n, dir, k) * JA(&c, e, n, dir, k);
                    }
                    lam += (fabs(un) + s * sqrt(a2)) / J2;
                    h2 += a2 / (J2 * J2);
                }
                if (h2 > ih2) ih2 = h2;
            } else {
                for (int k = 0; k < d; ++k) lam += (fabs(U[IDX(1 + k, e, n, ne, np)] / rho) + s) / c.h[k];
            }
            if (lam > lmax) lmax = lam;
            double nu = 4.0 * p->mu / (3.0 * rho);
            double nk = p->kappa / (rho * RV * p->cv);
            if (nk > nu) nu = nk;
            if (p->model != 0 && p->gammaK * p->beta > nu) nu = p->gammaK * p->beta;
            if (nu > numax) numax = nu;
        }
    free(T);
    if (!c.curved)
        for (int k = 0; k < d; ++k) ih2 += 1.0 / (c.h[k] * c.h[k]);
    teardown(&c);
    double k1 = 2.0 * c.N + 1.0;
    double dtc = cfl / (k1 * lmax);
    double dtv = numax > 0.0 ? dfl / (k1 * k1 * numax * ih2) : 1e300;
    double dts = (p->model != 0 && p->alpha * p->beta > 0.0) ? 2.0 / (p->alpha * p->beta) : 1e300;
    double r = dtc;
    if (dtv < r) r = dtv;
    if (dts < r) r = dts;
    *dt = r;
    return 0;
}

/* Rate of entropy production at the nodes (Sec. 2.3: the relaxation model's production
   rate after Eq. (navierstokeskorteweg_alpha), the original model's after
   Eq. (energyfluxnsk)), from the thermodynamic fluxes of the scheme:
     Pi = tau : grad u / T + kappa |grad T|^2 / T^2 + beta chi^2 / T,
     tau = mu (grad u + grad u^T - 2/3 div u I),  chi = gamma_K lap c + alpha (rho - c),
   the last term for the relaxation models only.  Reading: the printed viscous part
   (4/3 mu |div u|^2 + mu |D_dev|^2) does not follow from the stress of the same section
   under the Stokes hypothesis; the dissipation of that stress, tau : grad u
   (= 2 mu |D_dev|^2 in 3D), is used, and the heat term is the Fourier flux kappa grad T
   paired with grad(1/T).  Gradients are the scheme's: lifted grad u (pass 1), grad T and
   lap c (pass 2).  Pi[e][n]. */
static int entropy_production(const ctx_t *c, const double *U, double *Pi)
{
    long ne = c->ne;
    int np = c->np, d = c->d, nl = c->nl;
    const or_params *p = &c->prm;
    work_t w;
    if (work_alloc(c, &w)) { work_free(&w); return -2; }
    primitives(c, U, w.q);
    traces(c, w.q, nl, w.trq);
    if (c->curved) lift_pass1_c(c, w.q, w.trq, w.grad);
    else lift_pass1(c, w.q, w.trq, w.grad);
    node_temperature(c, U, w.grad, w.T);
    if (c->curved) lift_pass2_c(c, w.T, w.grad, w.trq, w.gT, w.lap);
    else lift_pass2(c, w.T, w.grad, w.trq, w.gT, w.lap);
#pragma omp parallel for schedule(static)
    for (long e = 0; e < ne; ++e)
        for (int n = 0; n < np; ++n) {
            double g[3 * 8], du[3][3];
            gather_grad(c, w.grad, e, n, g);
            /* du[i][k] = d u_k / d x_i */
            for (int i = 0; i < d; ++i)
                for (int k = 0; k < d; ++k) du[i][k] = g[i * nl + 1 + k];
            double divu = 0.0;
            for (int k = 0; k < d; ++k) divu += du[k][k];
            double diss = 0.0; /* tau : grad u = sum_ik tau_ik du_k/dx_i */
            for (int i = 0; i < d; ++i)
                for (int k = 0; k < d; ++k) {
                    double tik = p->mu * (du[i][k] + du[k][i] - (i == k ? 2.0 / 3.0 * divu : 0.0));
                    diss += tik * du[i][k];
                }
            double T = w.T[(size_t)e * np + n], gT2 = 0.0;
            for (int k = 0; k < d; ++k) {
                double gk = w.gT[IDX(k, e, n, ne, np)];
                gT2 += gk * gk;
            }
            double pi = diss / T + p->kappa * gT2 / (T * T);
            if (p->model != 0) {
                double chi = p->gammaK * w.lap[(size_t)e * np + n] + p->alpha * (U[IDX(0, e, n, ne, np)] - U[IDX(d + 2, e, n, ne, np)]);
                pi += p->beta * chi * chi / T;
            }
            Pi[(size_t)e * np + n] = pi;
        }
    work_free(&w);
    return 0;
}

/* Integral diagnostics with the collocated Gauss quadrature:
   out = (mass, momentum x, y, z, total energy, mathematical entropy -int rho eta,
          ||rho - c||_2, max |u|, int Pi (the rate of entropy production, above)). */
int or_diagnostics(const or_mesh *m, const or_params *p, const double *U, double *out)
{
    ctx_t c;
    if (setup(m, p, &c)) return -1;
    long ne = c.ne;
    int np = c.np, d = c.d;
    double *T = (double *)malloc(sizeof(double) * ne * np);
    double *Pi = (double *)malloc(sizeof(double) * ne * np);
    if (!T || !Pi || entropy_production(&c, U, Pi)) { free(T); free(Pi); teardown(&c); return -2; }
    or_temperature(m, p, U, T);
    double J = 1.0;
    for (int k = 0; k < d; ++k) J *= 0.5 * c.h[k];
    for (int k = 0; k < OR_NDIAG; ++k) out[k] = 0.0;
    for (long e = 0; e < ne; ++e)
        for (int n = 0; n < np; ++n) {
            double W = c.curved ? JN(&c, e, n) : J;
            for (int k = 0; k < d; ++k) W *= c.w[ncoord(&c, n, k)];
            double rho = U[IDX(0, e, n, ne, np)];
            out[0] += W * rho;
            double u2 = 0.0;
            for (int k = 0; k < d; ++k) {
                double mk = U[IDX(1 + k, e, n, ne, np)];
                out[1 + k] += W * mk;
                u2 += (mk / rho) * (mk / rho);
            }
            out[4] += W * U[IDX(d + 1, e, n, ne, np)];
            out[5] += -W * or_entropy_vol(rho, T[(size_t)e * np + n], p->cv);
            if (p->model != 0) {
                double dc = rho - U[IDX(d + 2, e, n, ne, np)];
                out[6] += W * dc * dc;
            }
            if (sqrt(u2) > out[7]) out[7] = sqrt(u2);
            out[8] += W * Pi[(size_t)e * np + n];
        }
    out[6] = sqrt(out[6]);
    free(T);
    free(Pi);
    teardown(&c);
    return 0;
}

/* Quadrature weight of every node, W[e][n] = J w_i w_j (w_k): the collocated Gauss
   quadrature of the diagnostics (J = prod h/2 on the straight box). */
int or_node_weights(const or_mesh *m, double *W)
{
    or_params p = {1, 1e-4, 0.01, 1.0 / 150.0, 5.0, 100.0, 100.0, 0};
    or_mesh mm = *m;
    for (int f = 0; f < 6; ++f) if (mm.wall_kind[f] != 0) mm.wall_T[f] = 0.85;
    ctx_t c;
    if (setup(&mm, &p, &c)) return -1;
    double J = 1.0;
    for (int k = 0; k < c.d; ++k) J *= 0.5 * c.h[k];
    for (long e = 0; e < c.ne; ++e)
        for (int n = 0; n < c.np; ++n) {
            double w = c.curved ? JN(&c, e, n) : J;
            for (int k = 0; k < c.d; ++k) w *= c.w[ncoord(&c, n, k)];
            W[(size_t)e * c.np + n] = w;
        }
    teardown(&c);
    return 0;
}

/* point fluxes for the tests: a 1-element periodic context gives d, nv and the model */
static int point_ctx(const or_params *p, int dim, ctx_t *c)
{
    or_mesh m;
    memset(&m, 0, sizeof(m));
    m.dim = dim;
    m.N = 1;
    for (int d = 0; d < 3; ++d) { m.n[d] = 1; m.hi[d] = 1.0; m.periodic[d] = 1; }
    return setup(&m, p, c);
}

int or_conv_point(const or_params *p, int dim, int dir, const double *U, double T, double *F)
{
    ctx_t c;
    if (point_ctx(p, dim, &c) || dir < 0 || dir >= dim) return -1;
    conv_flux(&c, U, flux_pressure(&c, U[0], T), dir, F);
    return 0;
}

int or_hllc_point(const or_params *p, int dim, int dir, const double *UL, double TL, const double *UR, double TR,
                  double *F)
{
    ctx_t c;
    if (point_ctx(p, dim, &c) || dir < 0 || dir >= dim || c.nv < dim + 3) return -1;
    hllc_flux(&c, UL, flux_pressure(&c, UL[0], TL), sound_speed(&c, UL[0], TL), UR, flux_pressure(&c, UR[0], TR),
              sound_speed(&c, UR[0], TR), dir, F);
    return 0;
}

int or_rusanov_point(const or_params *p, int dim, int dir, const double *UL, double TL, const double *UR, double TR,
                     double *F)
{
    ctx_t c;
    if (point_ctx(p, dim, &c) || dir < 0 || dir >= dim) return -1;
    double FL[8], FR[8];
    conv_flux(&c, UL, flux_pressure(&c, UL[0], TL), dir, FL);
    conv_flux(&c, UR, flux_pressure(&c, UR[0], TR), dir, FR);
    double lL = fabs(UL[1 + dir] / UL[0]) + sound_speed(&c, UL[0], TL);
    double lR = fabs(UR[1 + dir] / UR[0]) + sound_speed(&c, UR[0], TR);
    double lam = lL > lR ? lL : lR;
    for (int v = 0; v < c.nv; ++v) F[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * lam * (UR[v] - UL[v]);
    return 0;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
