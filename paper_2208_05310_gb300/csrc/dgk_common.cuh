// dgk_common.cuh -- device-side data structures, node indexing and the point-wise model
// of the relaxed non-isothermal NSK equations (Keim, Munz & Rohde, arXiv 2208.05310).
//
// R is the "bulk" arithmetic type (double for the FP64 form, float for the FP32-bulk
// form).  The energy balance of the temperature recovery is always done in double.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dgk {

// van der Waals constants in the paper's non-dimensional form (Sec. 2.1).
constexpr double kRgas = 8.0 / 3.0;
constexpr double kAvdw = 3.0;
constexpr double kBvdw = 1.0 / 3.0;
constexpr int kMaxP = 6;  // polynomial degree N <= 5

// device status bits (latched with atomicOr, read by dgk_status)
constexpr unsigned kStatNonFinite = 1u;
constexpr unsigned kStatDomain = 2u;
constexpr unsigned kStatBarrier = 4u;  // batched kernel: a grid barrier timed out

struct Phys {
    int model;  // 1 or 2
    double gK, mu, kap, cv, alpha, beta;
    double half_alpha, half_gK, inv_Rcv;  // derived on the host
};

// The same constants in the bulk type R, derived on the host so that kernels of the
// FP32-bulk form convert nothing from double per node.
template <typename R>
struct PhysR {
    int model;
    R gK, mu, kap, alpha, beta;
    R gKbeta, alphabeta, half_alpha, half_gK, two_thirds_mu;
    R s_coef;   // R_gas (1 + 1/cv)
    R inv_Rcv;  // 1 / (R_gas cv)
    R half_alpha_p;  // alpha/2 in the model-2 pressure, 0 for model 1
    int flux;        // convective numerical flux: 0 Rusanov, 1 HLLC (model 2)
};

// Per box face (-x,+x,-y,+y,-z,+z): isothermal no-slip wall with static contact angle.
// Contact-angle gradient: grad c . n = K (c - rl)(c - rv), K = -6 sigma cos(theta) /
// (gamma_K (rl - rv)^3)  (Eq. bc_contactangle_alpha with gamma_1 = 0 and Eq.
// helmfreesurftot_derivative).
struct Walls {
    int kind[6];
    double Tw[6], rv[6], rl[6], K[6];
    double g[6][4];  // kind 2 (generalized Navier slip): gamma_1..gamma_4
    double u[6][3];  // kind 1: velocity of a sliding wall (tangential)
};

// Division of 32-bit unsigned integers by an invariant divisor d >= 1 with a multiply-high
// and two shifts (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994, Sec. 4): l = ceil(log2 d), m = floor(2^32 (2^l - d)/d) + 1,
// then x / d = (t + ((x - t) >> s1)) >> s2 with t = mulhi(m, x), s1 = min(l, 1),
// s2 = max(l - 1, 0).  Valid for every 32-bit x and every d < 2^31.
struct FastDiv {
    unsigned m;
    int s1, s2;
    __host__ void init(unsigned d)
    {
        int l = 0;
        while ((1ull << l) < (unsigned long long)d) ++l;
        m = (unsigned)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
        s1 = l < 1 ? l : 1;
        s2 = l > 1 ? l - 1 : 0;
    }
    __device__ __forceinline__ unsigned div(unsigned x) const
    {
        const unsigned t = __umulhi(m, x);
        return (t + ((x - t) >> s1)) >> s2;
    }
};

struct Geom {
    int n[3];
    int periodic[3];
    double inv2h[3];  // 2 / h_d: d/dx = (2/h) d/dxi on the affine element
    long long ne;
    FastDiv div0, div1;  // by n[0], by n[1] (element index -> Cartesian coordinates)
    long long nslot;     // mortar slots (unstructured meshes with mortars), else 0
    long long nmort;     // mortars
};

template <typename R>
struct GeomR {
    R inv2h[3];
};

template <typename R>
struct WallsR {
    R K[6], rl[6], rv[6], Tw[6];
    int kind[6];                        // 1 no-slip isothermal, 2 generalized Navier slip
    R g1[6], g2[6], g3[6], g1gK[6], g1g4[6];  // kind 2: gamma_1, gamma_2, gamma_3, gamma_1/gamma_K, gamma_1 gamma_4
    R uw[6][3];                         // kind 1: velocity of a sliding wall (tangential; zero at rest)
};

// 1D operators on the P = N+1 Legendre-Gauss nodes (Sec. 3.1):
//   Dhat_ij = -(w_j / w_i) D_ji, Lp_i = l_i(+1)/w_i, Lm_i = l_i(-1)/w_i, lp/lm = l_i(+-1),
//   w = quadrature weights.
struct Ops {
    double Dhat[kMaxP * kMaxP];
    double Dm[kMaxP * kMaxP];  // D_ij = l_j'(xi_i)
    double Im[2][kMaxP * kMaxP], Pm[2][kMaxP * kMaxP];  // mortar interpolation / projection (see OpsR)
    double Lp[kMaxP], Lm[kMaxP], lp[kMaxP], lm[kMaxP], w[kMaxP];
};

// ------------------------------------------------------------------ sizes

// EB: elements per block (tile shape); 0 = as many as fit in 256 threads.
template <int D, int N, int EB = 0>
struct Shape {
    static constexpr int P = N + 1;
    static constexpr int NP = D == 2 ? P * P : P * P * P;   // nodes per element
    static constexpr int NFP = D == 2 ? P : P * P;          // points per face
    static constexpr int NF = 2 * D;                        // faces per element
    static constexpr int NV = D + 3;                        // conserved variables
    static constexpr int NL = D + 2;                        // pass-1 lifted variables (rho, u, c)
    static constexpr int NQ = NV + D * D + 2 * D + 1;       // face quantities: U, grad u, grad T, grad c, lap c
    static constexpr int NFQ = NF * NFP;                    // face points per element
    static constexpr int EPB = EB > 0 ? EB : ((256 / NP) > 0 ? (256 / NP) : 1);  // elements per block
    static constexpr int NT = EPB * NP;                     // threads per block
};

// node n = i + P*(j + P*k); coordinate along direction d
template <int P>
__device__ __forceinline__ int ncoord(int n, int d)
{
    return d == 0 ? n % P : (d == 1 ? (n / P) % P : n / (P * P));
}

// face-point index of node n on the faces normal to d (remaining coordinates in order)
template <int P>
__device__ __forceinline__ int node_fp(int n, int d)
{
    return d == 0 ? n / P : (d == 1 ? (n % P) + P * (n / (P * P)) : n % (P * P));
}

// first node of the line through face point fp along d, and the stride along d
template <int P>
__device__ __forceinline__ int line_base(int fp, int d)
{
    return d == 0 ? P * fp : (d == 1 ? (fp % P) + P * P * (fp / P) : fp);
}
template <int P>
__device__ __forceinline__ int line_stride(int d)
{
    return d == 0 ? 1 : (d == 1 ? P : P * P);
}


// ------------------------------------------------------------------ conversions
//
// binary64 <-> binary32 conversions written from the IEEE 754 encodings, in integer
// arithmetic.  On this GPU every FP64-pipe instruction, conversions included, issues at
// 1/64 of the FP32 rate, so the FP32-bulk kernels convert with integer instructions.
// d2f rounds to nearest even; results below the float normal range flush to signed
// zero, results above it round to +-inf, NaN stays NaN.  f2d is exact (subnormal floats
// become signed zero).

__device__ __forceinline__ float d2f(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const unsigned ed = (hi >> 20) & 0x7ffu;
    const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // leading 23 fraction bits
    const unsigned rest = lo & 0x1fffffffu;                  // the 29 dropped bits
    const int ef = (int)ed - 896;                            // exponent bias 1023 -> 127
    unsigned r = ((unsigned)ef << 23) + m;
    r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
    if (ef <= 0) r = 0u;
    if (ef >= 255) r = 0x7f800000u;
    if (ed == 0x7ffu) r = (m | rest) ? 0x7fc00000u : 0x7f800000u;
    return __uint_as_float(sign | r);
}

__device__ __forceinline__ double f2d(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned sign = u & 0x80000000u, ef = (u >> 23) & 0xffu, m = u & 0x7fffffu;
    unsigned hi = sign | ((ef + 896u) << 20) | (m >> 3);
    unsigned lo = m << 29;
    if (ef == 0u) { hi = sign; lo = 0u; }
    if (ef == 255u) { hi = sign | 0x7ff00000u | (m >> 3) | (m ? 0x80000u : 0u); lo = m << 29; }
    return __hiloint2double((int)hi, (int)lo);
}

// bulk <- double and double <- bulk (identity for the FP64 form)
template <typename R>
__device__ __forceinline__ R to_bulk(double x)
{
    if constexpr (sizeof(R) == 8) return x;
    else return d2f(x);
}
template <typename R>
__device__ __forceinline__ double to_f64(R x)
{
    if constexpr (sizeof(R) == 8) return x;
    else return f2d(x);
}


// ------------------------------------------------------------------ thermodynamics

// Temperature from the total energy, Eq. (totalenergyalpha), with the vdW internal
// energy rho eps = rho R cv T - a rho^2:
//   rho R cv T = rho e + a rho^2 - (|m|^2/(2 rho) + alpha/2 (rho-c)^2 + gamma_K/2 |grad c|^2).
// FP64 form: all in double.  FP32-bulk form: bal = rho e + a rho^2 formed in double from
// the FP64 state (the caller passes it rounded to float), the small kinetic / relaxation
// / capillary terms and the scaling by 1/(rho R cv) in float.  irho = 1/rho, d = rho - c,
// msq = |m|^2, gc2 = |grad c|^2.
__device__ __forceinline__ double temperature_f64(const Phys &ph, double rho, double irho, double E, double d,
                                                  double msq, double gc2)
{
    const double num = E + kAvdw * rho * rho - 0.5 * msq * irho - ph.half_alpha * d * d - ph.half_gK * gc2;
    return num * irho * ph.inv_Rcv;
}
template <typename R>
__device__ __forceinline__ R temperature_bulk(const PhysR<R> &pr, R bal, R irho, R d, R msq, R gc2)
{
    const R small = R(0.5) * msq * irho + pr.half_alpha * d * d + pr.half_gK * gc2;
    return (bal - small) * irho * pr.inv_Rcv;
}

// Pressure in the convective flux, Eq. (pressure), plus alpha/2 rho^2 for model 2
// (Eq. modified_pressure); iomb = 1/(1 - b rho).
template <typename R>
__device__ __forceinline__ R flux_pressure(const PhysR<R> &pr, R rho, R T, R iomb)
{
    return rho * R(kRgas) * T * iomb + (pr.half_alpha_p - R(kAvdw)) * rho * rho;
}

// Signal speed sqrt(c_s^2 + alpha rho) with the vdW isentropic
// c_s^2 = R T (1 + 1/cv)/(1 - b rho)^2 - 2 a rho (Eq. speedofsound, Sec. 2.3).
// Original NSK (model 0): sqrt(|c_s^2|).
template <typename R>
__device__ __forceinline__ R signal_speed(const PhysR<R> &pr, R rho, R T, R iomb)
{
    if (pr.model == 0) return sqrt(fabs(pr.s_coef * T * iomb * iomb - R(2.0 * kAvdw) * rho));
    R s2 = pr.s_coef * T * iomb * iomb + (pr.alpha - R(2.0 * kAvdw)) * rho;
    return s2 > R(0) ? sqrt(s2) : R(0);
}

// ------------------------------------------------------------------ fluxes and sources
//
// du[i][k] = d u_k / d x_i, gT = grad T, gc = grad c, lap = lap c.

// F = F^C - F^V in direction dir (Eq. navierstokeskorteweg_p / _palpha):
//   F^C = (m_dir, m u_dir + p^ e_dir, (rho e + p^) u_dir, c u_dir)
//   F^V = (0, tau_{., dir}, tau_{dir, .}.u + j_e,dir, gamma_K beta c_dir)
//   tau = mu (grad u + grad u^T - 2/3 div u I),
//   j_e = kappa grad T - gamma_K c grad c div u + gamma_K grad c zeta,
//   zeta = beta (gamma_K lap c + alpha (rho - c)).
template <int D, typename R>
__device__ __forceinline__ void flux_dir(const PhysR<R> &ph, int dir, R rho, const R *m, const R *u, R E, R c, R ph_,
                                         const R du[D][D], const R *gT, const R *gc, R lap, R *F)
{
    R divu = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) divu += du[k][k];
    const R mu = ph.mu;
    R ud = u[dir];
    R work = R(0);
    F[0] = m[dir];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        R tau = mu * (du[dir][k] + du[k][dir]);
        if (k == dir) tau -= ph.two_thirds_mu * divu;
        work += tau * u[k];
        F[1 + k] = m[k] * ud - tau;
        if (k == dir) F[1 + k] += ph_;
    }
    if (ph.model == 0) {
        // original NSK (Eq. navierstokeskorteweg): Korteweg stress gamma_K [(|grad rho|^2/2
        // + rho lap rho) I - grad rho (x) grad rho] (Eq. cauchystressnsk) and energy flux
        // kappa grad T - gamma_K rho grad rho div u (Eq. energyfluxnsk).  The c slot holds
        // rho: gc = grad rho, lap = lap rho; its flux is the mass flux, so c stays rho.
        R gr2 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) gr2 += gc[k] * gc[k];
        R kwork = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            R tk = -ph.gK * gc[k] * gc[dir];
            if (k == dir) tk += ph.gK * (R(0.5) * gr2 + rho * lap);
            F[1 + k] -= tk;
            kwork += tk * u[k];
        }
        const R je = ph.kap * gT[dir] - ph.gK * rho * gc[dir] * divu;
        F[D + 1] = (E + ph_) * ud - (work + kwork + je);
        F[D + 2] = F[0];
        return;
    }
    R zeta = ph.beta * (ph.gK * lap + ph.alpha * (rho - c));
    R je = ph.kap * gT[dir] - ph.gK * c * gc[dir] * divu + ph.gK * gc[dir] * zeta;
    F[D + 1] = (E + ph_) * ud - (work + je);
    F[D + 2] = c * ud - ph.gKbeta * gc[dir];
}

// Point-wise source with the lifted gradients (Sec. 3.1); model 1 / model 2 rows of
// Eq. (navierstokeskorteweg_p) / (..._palpha).  g[i][v]: gradient in direction i of
// lifted variable v = (rho, u_1..u_D, c).
template <int D, typename R>
__device__ __forceinline__ void source_terms(const PhysR<R> &ph, R rho, const R *u, R c, const R g[D][D + 2], R *S)
{
    if (ph.model == 0) {  // the original NSK system has no source
#pragma unroll
        for (int v = 0; v < D + 3; ++v) S[v] = R(0);
        return;
    }
    const R al = ph.alpha;
    R divu = R(0), gc2 = R(0), ccdu = R(0), work = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        divu += g[k][1 + k];
        gc2 += g[k][D + 1] * g[k][D + 1];
    }
#pragma unroll
    for (int i = 0; i < D; ++i)
#pragma unroll
        for (int j = 0; j < D; ++j) ccdu += g[i][D + 1] * g[j][D + 1] * g[i][1 + j];
    S[0] = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        R drive = ph.model == 1 ? g[k][D + 1] - g[k][0] : g[k][D + 1];
        S[1 + k] = al * rho * drive;
        work += S[1 + k] * u[k];
    }
    R pw = ph.model == 1 ? R(0.5) * al * (c * c - rho * rho) : R(0.5) * al * c * c;
    S[D + 1] = work + pw * divu + ph.gK * (R(0.5) * gc2 * divu - ccdu);
    S[D + 2] = ph.alphabeta * (rho - c);
}

// Rate of entropy production at a node (Sec. 2.3; the relaxation model's rate after
// Eq. navierstokeskorteweg_alpha, the original model's after Eq. energyfluxnsk), from the
// scheme's lifted gradients du[i][k] = d u_k / d x_i, grad T and lap c:
//   Pi = tau : grad u / T + kappa |grad T|^2 / T^2 + beta chi^2 / T,
//   tau = mu (grad u + grad u^T - 2/3 div u I),  chi = gamma_K lap c + alpha (rho - c),
// the last term for the relaxation models only (the dissipation of the stated stress
// under the Stokes hypothesis; the Fourier flux kappa grad T paired with grad(1/T)).
template <int D, typename R>
__device__ __forceinline__ R entropy_production(const PhysR<R> &ph, R rho, R c, R T, const R du[D][D], const R *gT,
                                                R lap)
{
    R divu = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) divu += du[k][k];
    R diss = R(0), gT2 = R(0);
#pragma unroll
    for (int i = 0; i < D; ++i) {
        gT2 += gT[i] * gT[i];
#pragma unroll
        for (int k = 0; k < D; ++k)
            diss += ph.mu * (du[i][k] + du[k][i] - (i == k ? R(2.0 / 3.0) * divu : R(0))) * du[i][k];
    }
    const R iT = R(1) / T;
    R pi = diss * iT + ph.kap * gT2 * iT * iT;
    if (ph.model != 0) {
        const R chi = ph.gK * lap + ph.alpha * (rho - c);
        pi += ph.beta * chi * chi * iT;
    }
    return pi;
}

}  // namespace dgk
