// dgk_host_math.cpp -- host-side set-up math of libdgk: Legendre-Gauss nodes and the
// DGSEM operators (Sec. 3.1), and the van der Waals saturation states and surface
// tension (Sec. 2.1, Eq. surftenscoef, Sec. 3.2).  Computed once per mesh, in double.
#include "dgk_host_math.h"

#include <cmath>

namespace dgk {
namespace host {

static const double kR = 8.0 / 3.0, kA = 3.0, kB = 1.0 / 3.0;

// Legendre polynomial P_n and its derivative at x by the three-term recurrence.
static void legendre(int n, double x, double &p, double &dp)
{
    double pm1 = 1.0, pc = x;
    if (n == 0) { p = 1.0; dp = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double pn = ((2 * k + 1) * x * pc - k * pm1) / (k + 1);
        pm1 = pc;
        pc = pn;
    }
    p = pc;
    dp = n * (pm1 - x * pc) / (1.0 - x * x);
}

bool gauss_legendre(int n, double *x, double *w)
{
    if (n < 1 || n > 64) return false;
    for (int k = 0; k < (n + 1) / 2; ++k) {
        // root k from the top, Chebyshev-like first guess, Newton to convergence
        double r = std::cos(M_PI * (4.0 * k + 3.0) / (4.0 * n + 2.0));
        double p, dp;
        for (int it = 0; it < 60; ++it) {
            legendre(n, r, p, dp);
            double step = p / dp;
            r -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        legendre(n, r, p, dp);
        double wk = 2.0 / ((1.0 - r * r) * dp * dp);
        x[n - 1 - k] = r;
        w[n - 1 - k] = wk;
        x[k] = -r;
        w[k] = wk;
    }
    if (n % 2) x[n / 2] = 0.0;
    return true;
}

// Barycentric weights lam_j = 1 / prod_{k != j} (x_j - x_k).
static void bary(int P, const double *x, double *lam)
{
    for (int j = 0; j < P; ++j) {
        double pr = 1.0;
        for (int k = 0; k < P; ++k)
            if (k != j) pr *= x[j] - x[k];
        lam[j] = 1.0 / pr;
    }
}

// l_j(t) in barycentric form (t not a node).
static void lagrange_eval(int P, const double *x, const double *lam, double t, double *l)
{
    double den = 0.0;
    for (int j = 0; j < P; ++j) den += lam[j] / (t - x[j]);
    for (int j = 0; j < P; ++j) l[j] = lam[j] / (t - x[j]) / den;
}

bool dg_operators(int N, Operators1D &op)
{
    const int P = N + 1;
    if (P > 16) return false;
    op.P = P;
    if (!gauss_legendre(P, op.xi, op.w)) return false;
    double lam[16];
    bary(P, op.xi, lam);
    // D_ij = l_j'(x_i): off-diagonal (lam_j/lam_i)/(x_i - x_j), diagonal = -row sum
    for (int i = 0; i < P; ++i) {
        double s = 0.0;
        for (int j = 0; j < P; ++j) {
            if (j == i) continue;
            double v = (lam[j] / lam[i]) / (op.xi[i] - op.xi[j]);
            op.D[i * P + j] = v;
            s += v;
        }
        op.D[i * P + i] = -s;
    }
    for (int i = 0; i < P; ++i)
        for (int j = 0; j < P; ++j) op.Dhat[i * P + j] = -(op.w[j] / op.w[i]) * op.D[j * P + i];
    lagrange_eval(P, op.xi, lam, -1.0, op.lm);
    lagrange_eval(P, op.xi, lam, 1.0, op.lp);
    for (int h = 0; h < 2; ++h)
        for (int j = 0; j < P; ++j) lagrange_eval(P, op.xi, lam, 0.5 * (op.xi[j] + 2.0 * h - 1.0), &op.Im[h][j * P]);
    return true;
}

// ---------------------------------------------------------------- thermodynamics

double pressure(double rho, double T) { return rho * kR * T / (1.0 - kB * rho) - kA * rho * rho; }

static double dpdrho(double rho, double T)
{
    double o = 1.0 - kB * rho;
    return kR * T / (o * o) - 2.0 * kA * rho;
}

// chemical potential without the rho-independent cv term (it cancels in every use here)
static double chem(double rho, double T)
{
    double o = 1.0 - kB * rho;
    return kR * T * std::log(kB * rho / o) + kR * T / o - 2.0 * kA * rho;
}

// free energy per volume without the term linear in rho that carries cv
static double psi_red(double rho, double T)
{
    return rho * kR * T * std::log(kB * rho / (1.0 - kB * rho)) - kA * rho * rho;
}

static double bisect_increasing(double (*f)(double, double), double T, double target, double lo, double hi)
{
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (f(mid, T) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

static double neg_dpdrho(double r, double T) { return -dpdrho(r, T); }

bool maxwell(double T, double &rv, double &rl)
{
    if (!(T > 0.0 && T < 1.0)) return false;
    const double rmax = 1.0 / kB;
    // spinodals: dp/drho decreasing through 0 on (0, 1), increasing on (1, 1/b)
    double sv = bisect_increasing(neg_dpdrho, T, 0.0, 1e-12, 1.0);
    double sl = bisect_increasing(dpdrho, T, 0.0, 1.0, rmax - 1e-12);
    double pmin = pressure(sl, T);
    // bracket on the vapour density: P = p(rho_v) must admit a liquid root (P > pmin, P > 0)
    double lo = 1e-12;
    if (pmin > 0.0) lo = bisect_increasing(pressure, T, pmin, 1e-12, sv);
    double hi = sv;
    auto h = [&](double r) {
        double P = pressure(r, T);
        double rL = bisect_increasing(pressure, T, P, sl, rmax - 1e-13);
        return chem(rL, T) - chem(r, T);
    };
    // h > 0 at the low end, < 0 at the vapour spinodal
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (h(mid) > 0.0) lo = mid; else hi = mid;
    }
    rv = 0.5 * (lo + hi);
    rl = bisect_increasing(pressure, T, pressure(rv, T), sl, rmax - 1e-13);
    // Newton polish on (p_l - p_v, mu_l - mu_v) = 0; dmu/drho = (dp/drho)/rho
    for (int it = 0; it < 6; ++it) {
        double f1 = pressure(rl, T) - pressure(rv, T);
        double f2 = chem(rl, T) - chem(rv, T);
        double av = dpdrho(rv, T), al = dpdrho(rl, T);
        double det = (-av) * (al / rl) - al * (-av / rv);
        if (det == 0.0 || !std::isfinite(det)) break;
        double dv = (f1 * (al / rl) - al * f2) / det;
        double dl = ((-av) * f2 - (-av / rv) * f1) / det;
        rv -= dv;
        rl -= dl;
    }
    return std::isfinite(rv) && std::isfinite(rl) && rv > 0.0 && rl > rv;
}

bool sigma_vl(double T, double gammaK, double &sigma)
{
    double rv, rl;
    if (!maxwell(T, rv, rl)) return false;
    double x[15], w[15];
    gauss_legendre(15, x, w);
    const double mv = chem(rv, T), pv = pressure(rv, T);
    const double half = 0.5 * (rl - rv), mid = 0.5 * (rl + rv);
    double acc = 0.0;
    for (int q = 0; q < 15; ++q) {
        double r = mid + half * x[q];
        double d = psi_red(r, T) - (r * mv - pv);
        acc += w[q] * std::sqrt(d > 0.0 ? d : 0.0);
    }
    sigma = std::sqrt(2.0 * gammaK) * half * acc;
    return std::isfinite(sigma);
}

}  // namespace host
}  // namespace dgk
