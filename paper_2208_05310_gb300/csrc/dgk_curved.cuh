// dgk_curved.cuh -- the stage kernels on curved elements (Sec. 3.1 on curvilinear
// hexahedra / quadrilaterals).  Element e maps the reference cube by a polynomial; the
// host computes its metric terms J a^dir_k (the contravariant basis times the Jacobian)
// at the nodes and at the face points, and 1/J at the nodes.  Differences from the box
// kernels of dgk_kernels.cuh:
//   - BR1 liftings in the strong form with the chain rule:
//       J d q/d x_k = sum_dir [ J a^dir_k (D q)_dir + Lp (q* - q-)_+ (J a^dir_k)_+
//                                                   - Lm (q* - q-)_- (J a^dir_k)_- ],
//     (_+/_-: the face points of the node's line along dir; D_il = l_l'(xi_i)), which on
//     an affine element equals the weak form the box kernels use;
//   - lap c = sum_k [BR1 gradient of d c/d x_k]_k; its face data are traces of
//     grad c . J a^dir (one scalar per face point, the same vector on both sides);
//   - volume integral of the contravariant fluxes F . J a^dir, face data along the face
//     metric (flux and signal speed scaled by the surface element), and 1/J in place of
//     2/h in the volume and surface terms.
// The metric arrays: met [D*D+1][ne][NP] (plane dir*D + k: J a^dir_k; plane D*D: 1/J) and
// fmet [D][ne][NF][NFP] (J a^dir_k at face f = 2 dir + side, oriented along +xi_dir and
// identical in the two elements that share the face).  Walls: isothermal no-slip
// contact-angle walls, at rest or sliding, and generalized Navier-slip walls, along the
// local normal; Rusanov or (model 2) HLLC flux along the face normal.
#pragma once

#include "dgk_kernels.cuh"

// Resident threads per SM requested for the curved lifting kernels, as a register budget
// (65536 / threads); 0 leaves the choice to the compiler.  The FP64 form asks for half.
#ifndef DGK_THREADS_LIFT1C
#define DGK_THREADS_LIFT1C 1728
#endif
#ifndef DGK_THREADS_LIFT2C
#define DGK_THREADS_LIFT2C 864
#endif
// 1: ask for the largest shared-memory carveout for k_lift2volc (its blocks hold 43 KB
// in the 3D N = 5 FP32-bulk form)
#ifndef DGK_CURVED_CARVEOUT
#define DGK_CURVED_CARVEOUT 1
#endif

namespace dgk {

__host__ __device__ constexpr int curved_min_blocks(int threads_per_block, int threads_per_sm)
{
    return threads_per_sm > 0 ? min_blocks(threads_per_block, threads_per_sm) : 1;
}

// Face record of a curved face point:
//   U (NV) | d u_k/d x_j at DU + j D + k (D*D) | grad T (D) | grad c (D) | lap c
template <int D>
struct FaceRecC {
    static constexpr int NV = D + 3;
    static constexpr int DU = NV, GT = NV + D * D, GC = GT + D, LAP = GC + D, NQ = LAP + 1;
};

template <int P, typename R>
__device__ __forceinline__ R sel(const R *v, int i)
{
    R x = v[0];
#pragma unroll
    for (int l = 1; l < P; ++l) x = l == i ? v[l] : x;
    return x;
}

// y_i = sum_l D_il x_l (strong derivative of one line)
template <int P, typename R>
__device__ __forceinline__ void dm_line(const OpsR<R> &o, const R x[P], R y[P])
{
#pragma unroll
    for (int i = 0; i < P; ++i) {
        R acc = R(0);
#pragma unroll
        for (int l = 0; l < P; ++l) acc += o.Dm[i * P + l] * x[l];
        y[i] = acc;
    }
}

// F . a of the point flux F = F^C - F^V for a vector a (flux_dir with e_dir replaced by a):
//   F^C . a = (m.a, m (u.a) + p^ a, (rho e + p^)(u.a), c (u.a)),
//   F^V . a = (0, tau a, (tau a).u + j_e.a, gamma_K beta grad c.a); du[j][k] = d u_k/d x_j.
template <int D, typename R>
__device__ __forceinline__ void flux_vec(const PhysR<R> &ph, const R *a, R rho, const R *m, const R *u, R E, R c, R pf,
                                         const R du[D][D], const R *gT, const R *gc, R lap, R *F)
{
    R divu = R(0), un = R(0), mn = R(0), gTa = R(0), gca = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        divu += du[k][k];
        un += u[k] * a[k];
        mn += m[k] * a[k];
        gTa += gT[k] * a[k];
        gca += gc[k] * a[k];
    }
    R work = R(0);
    F[0] = mn;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        R s = R(0);
#pragma unroll
        for (int j = 0; j < D; ++j) s += (du[j][k] + du[k][j]) * a[j];
        const R ta = ph.mu * s - ph.two_thirds_mu * divu * a[k];
        work += ta * u[k];
        F[1 + k] = m[k] * un + pf * a[k] - ta;
    }
    if (ph.model == 0) {
        // original NSK: Korteweg stress and energy flux along a (see flux_dir)
        R gr2 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) gr2 += gc[k] * gc[k];
        R kwork = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const R tk = -ph.gK * gc[k] * gca + ph.gK * (R(0.5) * gr2 + rho * lap) * a[k];
            F[1 + k] -= tk;
            kwork += tk * u[k];
        }
        const R je = ph.kap * gTa - ph.gK * rho * gca * divu;
        F[D + 1] = (E + pf) * un - (work + kwork + je);
        F[D + 2] = F[0];
        return;
    }
    const R zeta = ph.beta * (ph.gK * lap + ph.alpha * (rho - c));
    const R je = ph.kap * gTa - ph.gK * c * gca * divu + ph.gK * gca * zeta;
    F[D + 1] = (E + pf) * un - (work + je);
    F[D + 2] = c * un - ph.gKbeta * gca;
}

// Face data of one curved face point from its record r, along the face metric a
// (oriented along +xi_dir; w: the wall-table entry of a wall face).  Interior: the one-sided flux F . a and the scaled signal
// speed |u.a| + s |a|.  Wall (side: 0 minus, 1 plus face): the complete flux along a,
// |a| nsign F_n with F_n the outward wall flux per unit area for the outward unit normal
// n = nsign a/|a|: Rusanov against the ghost (rho, m - 2(m.n)n, rho e, c) with equal
// pressure and signal speed, minus the viscous flux tau(grad u-).n,
// kappa grad T-.n - gamma_K c- g_n div u-, gamma_K beta g_n (contact-angle g_n).
template <int D, typename R>
__device__ __forceinline__ void face_flux_c(const Ctx<R> &a, int f, int w, bool wall, const R *r, const R *av, R *F, R &lam,
                                            R &pf_out, R &s_out)
{
    using FR = FaceRecC<D>;
    const PhysR<R> &ph = a.pr;
    const R rho = r[0], E = r[D + 1], c = r[D + 2], irho = R(1) / rho;
    R m[D], u[D], gc[D], gT[D], du[D][D], msq = R(0), gc2 = R(0), a2 = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        m[k] = r[1 + k];
        u[k] = m[k] * irho;
        msq += m[k] * m[k];
        gc[k] = r[FR::GC + k];
        gc2 += gc[k] * gc[k];
        gT[k] = r[FR::GT + k];
        a2 += av[k] * av[k];
#pragma unroll
        for (int j = 0; j < D; ++j) du[k][j] = r[FR::DU + k * D + j];
    }
    const R T = (E + R(kAvdw) * rho * rho - R(0.5) * msq * irho - ph.half_alpha * (rho - c) * (rho - c) -
                 ph.half_gK * gc2) * irho * ph.inv_Rcv;
    const R iomb = R(1) / (R(1) - R(kBvdw) * rho);
    const R pf = flux_pressure<R>(ph, rho, T, iomb);
    const R sig = signal_speed<R>(ph, rho, T, iomb);
    const R sa = sqrt(a2);
    pf_out = pf;
    s_out = sig;
    if (!wall) {
        flux_vec<D, R>(ph, av, rho, m, u, E, c, pf, du, gT, gc, r[FR::LAP], F);
        R un = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) un += u[k] * av[k];
        lam = fabs(un) + sig * sa;
        return;
    }
    const R nsign = (f & 1) ? R(1) : R(-1);
    R nh[D], mn = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        nh[k] = nsign * av[k] / sa;
        mn += m[k] * nh[k];
    }
    const R un = mn * irho;
    lam = fabs(un) + sig;
    R Fi[D + 3], Fg[D + 3], Ui[D + 3], Ug[D + 3];
    Fi[0] = mn;
    Fg[0] = -mn;
    Ui[0] = Ug[0] = rho;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const R mg = m[k] - R(2) * mn * nh[k];
        Fi[1 + k] = m[k] * un + pf * nh[k];
        Fg[1 + k] = -mg * un + pf * nh[k];
        Ui[1 + k] = m[k];
        Ug[1 + k] = mg;
    }
    Fi[D + 1] = (E + pf) * un;
    Fg[D + 1] = -(E + pf) * un;
    Fi[D + 2] = c * un;
    Fg[D + 2] = -c * un;
    Ui[D + 1] = Ug[D + 1] = E;
    Ui[D + 2] = Ug[D + 2] = c;
    R divu = R(0), gTn = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        divu += du[k][k];
        gTn += gT[k] * nh[k];
    }
    const R gn = a.v.wr.K[w] * (c - a.v.wr.rl[w]) * (c - a.v.wr.rv[w]);
    R Fv[D + 3];
    Fv[0] = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        R s = R(0);
#pragma unroll
        for (int j = 0; j < D; ++j) s += (du[j][k] + du[k][j]) * nh[j];
        Fv[1 + k] = ph.mu * s - ph.two_thirds_mu * divu * nh[k];
    }
    if (a.v.wr.kind[w] == 2) {
        // generalized Navier slip (Eq. bc_nsk_alpha) along the unit normal: the fluid's
        // normal traction plus the tangential traction gamma_1 div u (grad c)_t - gamma_2 u_t,
        // its work on the fluid, the heat flux -gamma_3 (1/T_wall - 1/T),
        // zeta = -gamma_1 gamma_4 div u, grad c . n with the gamma_1 div u term
        R tnn = R(0), gcn = R(0), work = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            tnn += Fv[1 + k] * nh[k];
            gcn += gc[k] * nh[k];
        }
        const R g1d = a.v.wr.g1[w] * divu, g2 = a.v.wr.g2[w];
        const R gnn = gn + a.v.wr.g1gK[w] * divu;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const R tk = g1d * (gc[k] - gcn * nh[k]) - g2 * (u[k] - un * nh[k]);
            Fv[1 + k] = tnn * nh[k] + tk;
            work += tk * u[k];
        }
        const R qn = -a.v.wr.g3[w] * (R(1) / a.v.wr.Tw[w] - R(1) / T);
        Fv[D + 1] = work + qn - ph.gK * c * gnn * divu - ph.gK * gnn * a.v.wr.g1g4[w] * divu;
        Fv[D + 2] = ph.gKbeta * gnn;
    } else {
        // no slip: the traction works on the wall's velocity, projected on the tangent plane
        R uwn = R(0), work = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) uwn += a.v.wr.uw[w][k] * nh[k];
#pragma unroll
        for (int k = 0; k < D; ++k) work += Fv[1 + k] * (a.v.wr.uw[w][k] - uwn * nh[k]);
        Fv[D + 1] = work + ph.kap * gTn - ph.gK * c * gn * divu;
        Fv[D + 2] = ph.gKbeta * gn;
    }
    const R scale = nsign * sa;
    R Fc[D + 3];
    if (ph.flux == 1) {
        // HLLC against the ghost along the outward normal, the fluid on the left
        hllc_vec<D, R>(Ui, Fi, pf, sig, irho, Ug, Fg, pf, sig, irho, nh, Fc);
    } else {
#pragma unroll
        for (int v = 0; v < D + 3; ++v) Fc[v] = R(0.5) * (Fi[v] + Fg[v]) - R(0.5) * lam * (Ug[v] - Ui[v]);
    }
#pragma unroll
    for (int v = 0; v < D + 3; ++v) F[v] = scale * (Fc[v] - Fv[v]);
}

// Neighbour across face f of the slot's element: the element index (negative at a wall),
// the neighbour's facing face fo, the face-point orientation o and the wall-table entry
// w of a wall face.  Unstructured tables (v.conn) or the box's connectivity.  A mortar face
// returns kMortar - slot (<= kMortar), with fo = 1 on the big side: its neighbour data are
// in the mortar slot, already interpolated or projected to this face's points.
constexpr int kMortar = -1000;

template <int D, int N, typename R>
__device__ __forceinline__ long long face_nbr(const KView<R> &v, const Slot<D, N> &t, int f, int &fo, int &o, int &w)
{
    if (v.conn) {
        const int *c = v.conn + (t.e * (2 * D) + f) * 3;
        const int nb = c[0];
        fo = c[1];
        o = c[2];
        w = nb < 0 ? -1 - nb : f;
        return nb;
    }
    fo = 2 * (f >> 1) + 1 - (f & 1);
    o = 0;
    w = f;
    return t.nbr(v.g, f);
}

// Metric plane p of node n of element e (p = dir*D + k: J a^dir_k; p = D*D: 1/J).
template <int NP, typename R>
__device__ __forceinline__ R metric(const KView<R> &v, int p, long long e, int n)
{
    return nat<NP>(v.met, v.g.ne, p, e, n);
}

// Stage the element's face metrics into sJf[k][f][fp] (one face point per task).
template <int D, int N, typename R>
__device__ __forceinline__ void stage_face_metrics(const Ctx<R> &a, const Slot<D, N> &t, R *sJf)
{
    using S = Shape<D, N>;
    constexpr int NP = S::NP, NF = S::NF, NFP = S::NFP;
    for (int q = t.n; q < NF * NFP; q += NP) {
#pragma unroll
        for (int k = 0; k < D; ++k) sJf[k * NF * NFP + q] = fat<NF, NFP>(a.v.fmet, a.v.g.ne, k, t.e, q / NFP, q % NFP);
    }
}

// Gradient of one nodal field at this thread's node from its reference derivatives
// r[dir] and the jumps q* - q- of its line ends (sJump[f * jstride + fp], f = 2 dir + side):
// out[k] = (1/J) sum_dir [J a^dir_k r_dir + Lp_i jump_+ Jf_k,+ - Lm_i jump_- Jf_k,-].
template <int D, int N, typename R>
__device__ __forceinline__ void chain_gradient(const Ctx<R> &a, int n, const R Ja[D][D], R iJ, const R *r,
                                               const R *sJump, int jstride, const R *sJf, R *out)
{
    using S = Shape<D, N>;
    constexpr int P = S::P, NF = S::NF, NFP = S::NFP;
    R acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) acc[k] = R(0);
#pragma unroll
    for (int dir = 0; dir < D; ++dir) {
        const int i = ncoord<P>(n, dir), fp = node_fp<P>(n, dir);
        const R jp = sel<P, R>(a.op.Lp, i) * sJump[(2 * dir + 1) * jstride + fp];
        const R jm = sel<P, R>(a.op.Lm, i) * sJump[(2 * dir) * jstride + fp];
#pragma unroll
        for (int k = 0; k < D; ++k)
            acc[k] += Ja[dir][k] * r[dir] + jp * sJf[(k * NF + 2 * dir + 1) * NFP + fp] - jm * sJf[(k * NF + 2 * dir) * NFP + fp];
    }
#pragma unroll
    for (int k = 0; k < D; ++k) out[k] = acc[k] * iJ;
}

// ------------------------------------------------------------------ c-lifting on curved elements
//
// On return sDc[k][n] = d c/d x_k.  sR: D*NP scratch for the reference derivatives; sCs:
// face values, overwritten by the jumps; sJf: the staged face metrics.
template <int D, int N, typename R>
struct CLiftC {
    using S = Shape<D, N>;
    static constexpr int smem_per_elem = S::NP + S::NF * S::NFP + D * S::NP + D * S::NP + D * S::NF * S::NFP + S::NP;
    // c, c*/jumps, reference derivatives, grad c, face metrics, T

    __device__ static void run(const Ctx<R> &a, const Slot<D, N> &t, R c, R *sC, R *sCs, R *sR, R *sJf, R *sDc,
                               const R (*Jpre)[D] = nullptr, R iJpre = R(0))
    {
        constexpr int P = S::P, NP = S::NP, NF = S::NF, NFP = S::NFP;
        const long long ne = a.v.g.ne;
        if (t.valid) {
            for (int q = t.n; q < NF * NFP; q += NP) {
                const int f = q / NFP, fp = q % NFP;
                const R own = fat<NF, NFP>(a.v.tr1, ne, D + 1, t.e, f, fp);
                int fo, o, w;
                const long long b = face_nbr<D, N, R>(a.v, t, f, fo, o, w);
                if (b >= 0) sCs[q] = R(0.5) * (own + fat<NF, NFP>(a.v.tr1, ne, D + 1, b, fo, map_fp<S::P>(o, fp)));
                else if (b <= kMortar) sCs[q] = R(0.5) * (own + a.v.mtr1[((long long)(D + 1) * a.v.g.nslot + (kMortar - b)) * NFP + fp]);
                else sCs[q] = own;
            }
            stage_face_metrics<D, N, R>(a, t, sJf);
            sC[t.n] = c;  // after the face loads, so that c's own load is not waited for first
        }
        __syncthreads();
        if (t.valid) {
            for (int q = t.n; q < D * NFP; q += NP) {
                const int dir = q / NFP, line = q % NFP;
                const int base = line_base<P>(line, dir), stride = line_stride<P>(dir);
                R x[P], y[P], tm, tp;
                load_line<P, R>(sC, base, stride, x);
                dm_line<P, R>(a.op, x, y);
                trace_pair<P, R>(a.op, x, tm, tp);
                store_line<P, R>(sR + dir * NP, base, stride, y);
                sCs[(2 * dir) * NFP + line] -= tm;
                sCs[(2 * dir + 1) * NFP + line] -= tp;
            }
        }
        __syncthreads();
        if (t.valid) {
            R Ja[D][D], r[D], gc[D];
#pragma unroll
            for (int dir = 0; dir < D; ++dir) {
                r[dir] = sR[dir * NP + t.n];
#pragma unroll
                for (int k = 0; k < D; ++k) Ja[dir][k] = Jpre ? Jpre[dir][k] : metric<NP, R>(a.v, dir * D + k, t.e, t.n);
            }
            chain_gradient<D, N, R>(a, t.n, Ja, Jpre ? iJpre : metric<NP, R>(a.v, D * D, t.e, t.n), r, sCs, NFP, sJf, gc);
#pragma unroll
            for (int k = 0; k < D; ++k) sDc[k * NP + t.n] = gc[k];
        }
        __syncthreads();
    }
};

// ------------------------------------------------------------------ kernel 1 (curved)
//
// Lifts c, recovers T, and writes the face traces of T and of grad c . J a^dir (tr2[0],
// tr2[1]).

template <int D, int N, typename R>
__device__ __forceinline__ void lift1c_body(const Ctx<R> &a, long long blk, unsigned char *smraw)
{
    using S = Shape<D, N>;
    using L = CLiftC<D, N, R>;
    constexpr int P = S::P, NP = S::NP, NFP = S::NFP, NF = S::NF;
    const Slot<D, N> t(a.v.g, blk);
    R *sC = reinterpret_cast<R *>(smraw) + (size_t)t.le * L::smem_per_elem;
    R *sCs = sC + NP, *sR = sCs + NF * NFP, *sDc = sR + D * NP, *sJf = sDc + D * NP, *sT = sJf + D * NF * NFP;
    // the node's metric terms are loaded with the state: their latency then overlaps the
    // face values and the line derivatives instead of stalling the chain rule
    NodeState<D, R> q;
    R Jm[D][D], iJm = R(0);
    if (t.valid) {
        q.load(a.v, t.e, t.n, NP);
#pragma unroll
        for (int dir = 0; dir < D; ++dir)
#pragma unroll
            for (int k = 0; k < D; ++k) Jm[dir][k] = metric<NP, R>(a.v, dir * D + k, t.e, t.n);
        iJm = metric<NP, R>(a.v, D * D, t.e, t.n);
    }
    L::run(a, t, q.c, sC, sCs, sR, sJf, sDc, Jm, iJm);
    if (t.valid) {
        R gc[D];
#pragma unroll
        for (int d = 0; d < D; ++d) gc[d] = sDc[d * NP + t.n];
        const R T = node_temperature<D, R>(a, q, gc);
        check_state<R>(a.v.status, q.rho, T, q.E);
        sT[t.n] = T;
    }
    __syncthreads();
    if (t.valid) {
        const long long ne = a.v.g.ne;
        for (int qq = t.n; qq < D * NFP; qq += NP) {
            const int dir = qq / NFP, line = qq % NFP;
            const int base = line_base<P>(line, dir), stride = line_stride<P>(dir);
            R x[P], tm, tp;
            load_line<P, R>(sT, base, stride, x);
            trace_pair<P, R>(a.op, x, tm, tp);
            fat<NF, NFP>(a.v.tr2, ne, 0, t.e, 2 * dir, line) = tm;
            fat<NF, NFP>(a.v.tr2, ne, 0, t.e, 2 * dir + 1, line) = tp;
            R dm = R(0), dp = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                load_line<P, R>(sDc + k * NP, base, stride, x);
                trace_pair<P, R>(a.op, x, tm, tp);
                dm += tm * sJf[(k * NF + 2 * dir) * NFP + line];
                dp += tp * sJf[(k * NF + 2 * dir + 1) * NFP + line];
            }
            fat<NF, NFP>(a.v.tr2, ne, 1, t.e, 2 * dir, line) = dm;
            fat<NF, NFP>(a.v.tr2, ne, 1, t.e, 2 * dir + 1, line) = dp;
        }
    }
}

template <int D, int N, typename R>
__global__ void __launch_bounds__(Shape<D, N>::NT, curved_min_blocks(Shape<D, N>::NT, DGK_THREADS_LIFT1C / (int)(sizeof(R) / 4)))
    k_lift1c(KArgs<R> args)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    lift1c_body<D, N, R>(a, blockIdx.x, smraw);
}

// Set-up kernel on curved elements, as k_node_T: mode 0 nodal T into a.v.out; mode 1
// rho e from the temperature in a.v.out.
template <int D, int N, typename R>
__device__ __forceinline__ void node_Tc_body(const Ctx<R> &a, long long blk, unsigned char *smraw, int mode)
{
    using S = Shape<D, N>;
    using L = CLiftC<D, N, R>;
    constexpr int NP = S::NP, NF = S::NF, NFP = S::NFP, NV = S::NV;
    const Slot<D, N> t(a.v.g, blk);
    R *sC = reinterpret_cast<R *>(smraw) + (size_t)t.le * L::smem_per_elem;
    R *sCs = sC + NP, *sR = sCs + NF * NFP, *sDc = sR + D * NP, *sJf = sDc + D * NP;
    double Ud[NV];
    NodeState<D, R> q;
    if (t.valid) {
#pragma unroll
        for (int v = 0; v < NV; ++v) Ud[v] = a.v.U[((long long)v * a.v.g.ne + t.e) * NP + t.n];
        q.from_double(Ud);
    }
    L::run(a, t, q.c, sC, sCs, sR, sJf, sDc);
    if (!t.valid) return;
    R gc[D];
#pragma unroll
    for (int d = 0; d < D; ++d) gc[d] = sDc[d * NP + t.n];
    const long long idx = t.e * NP + t.n;
    if (mode == 0) {
        a.v.out[idx] = to_f64<R>(node_temperature<D, R>(a, q, gc));
        return;
    }
    const double rho = Ud[0], T = a.v.out[idx];
    double msq = 0.0, gc2 = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        msq += Ud[1 + k] * Ud[1 + k];
        gc2 += (double)gc[k] * (double)gc[k];
    }
    const double dc = rho - Ud[D + 2];
    a.v.U[((long long)(D + 1) * a.v.g.ne + t.e) * NP + t.n] =
        rho * (kRgas * a.ph.cv * T - kAvdw * rho) + 0.5 * msq / rho + 0.5 * a.ph.alpha * dc * dc + 0.5 * a.ph.gK * gc2;
}

template <int D, int N, typename R>
__global__ void __launch_bounds__(Shape<D, N>::NT) k_node_Tc(KArgs<R> args, int mode)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    node_Tc_body<D, N, R>(a, blockIdx.x, smraw, mode);
}

// ------------------------------------------------------------------ kernel 2 (curved)

template <int D, int N, typename R>
struct K2CSmem {
    using S = Shape<D, N>;
    static constexpr int G = D * S::NL * S::NP;    // reference derivatives, then gradients [k][v][n]
    static constexpr int GT = D * S::NP;           // grad T
    static constexpr int JF = D * S::NF * S::NFP;  // face metrics [k][f][fp]
    static constexpr int X1 = S::NL * S::NP + S::NF * S::NL * S::NFP;                // prims, q*/jumps
    static constexpr int X2 = S::NP + 2 * S::NF * S::NFP + D * S::NP + D * D * S::NP;  // T, jumps, D T, D grad c
    static constexpr int X4 = D * S::NV * S::NP;                                       // volume: F and its integral per direction
    static constexpr int SR = S::NF * FaceRecC<D>::NQ * S::NFP;                        // traced records
    static constexpr int XN = X4 > SR ? X4 : SR;                                       // nodal U, lap (sN)
    static constexpr int X3 = XN + (S::NV + 1) * S::NP;
    static constexpr int XA = X1 > X2 ? X1 : X2;
    static constexpr int X = XA > X3 ? XA : X3;
    static constexpr int WG = XA;                  // per face: gamma_1/gamma_K of a Navier-slip wall, else 0
    static_assert(WG + S::NF <= X, "no room for the wall factors");
    static constexpr int per_elem = G + GT + JF + X;
};

// Nodal array of record quantity k (FaceRecC order).
template <int D, int N, typename R>
__device__ __forceinline__ const R *face_source_c(int k, const R *sG, const R *sGT, const R *sN)
{
    using S = Shape<D, N>;
    using FR = FaceRecC<D>;
    constexpr int NP = S::NP, NL = S::NL, NV = S::NV;
    if (k < FR::DU) return sN + k * NP;
    if (k < FR::GT) {
        const int j = (k - FR::DU) / D, kk = (k - FR::DU) % D;
        return sG + (j * NL + 1 + kk) * NP;
    }
    if (k < FR::GC) return sGT + (k - FR::GT) * NP;
    if (k < FR::LAP) return sG + ((k - FR::GC) * NL + D + 1) * NP;
    return sN + NV * NP;
}

// DIAG 1: the same liftings, then the rate of entropy production of each node into
// a.v.out[e][n] (double) in place of the volume integral and the face data.
template <int D, int N, typename R, int DIAG = 0>
__device__ __forceinline__ void lift2volc_body(const Ctx<R> &a, long long blk, unsigned char *smraw)
{
    using S = Shape<D, N>;
    using M = K2CSmem<D, N, R>;
    using FR = FaceRecC<D>;
    constexpr int P = S::P, NP = S::NP, NFP = S::NFP, NF = S::NF, NL = S::NL, NV = S::NV, NQ = FR::NQ;
    const Slot<D, N> t(a.v.g, blk);
    R *sG = reinterpret_cast<R *>(smraw) + (size_t)t.le * M::per_elem;
    R *sGT = sG + M::G, *sJf = sGT + M::GT, *sX = sJf + M::JF;
    const long long ne = a.v.g.ne;
    const int n = t.n;
    // one face point per thread when NF NFP = NP (3D, N = 5): its neighbour once
    int fo0 = 0, o0 = 0, w0 = 0;
    const long long b0 = (NF * NFP == NP && t.valid) ? face_nbr<D, N, R>(a.v, t, n / NFP, fo0, o0, w0) : -1;
    // the node's metric terms, loaded first so that their latency overlaps pass 1
    R Ja[D][D], iJ = R(0);
    if (t.valid) {
#pragma unroll
        for (int dir = 0; dir < D; ++dir)
#pragma unroll
            for (int k = 0; k < D; ++k) Ja[dir][k] = metric<NP, R>(a.v, dir * D + k, t.e, n);
        iJ = metric<NP, R>(a.v, D * D, t.e, n);
    }

    // ---- pass 1 inputs: prims (rho, u, c), central face values (walls: rho*, c* one-sided,
    //      u* = 0), face metrics
    R *sQ = sX, *sQs = sX + NL * NP;
    NodeState<D, R> ns;
    if (t.valid) {
        ns.load(a.v, t.e, n, NP);
        for (int q = n; q < NF * NFP; q += NP) {
            const int f = q / NFP, fp = q % NFP;
            int fo = fo0, o = o0, w = w0;
            const long long b = NF * NFP == NP ? b0 : face_nbr<D, N, R>(a.v, t, f, fo, o, w);
            // one branch per kind of face, so that each point issues only its own loads
            if (b >= 0) {
                const int fq = map_fp<P>(o, fp);
                R own[NL], nbv[NL];  // all loads issued before the first use
#pragma unroll
                for (int v = 0; v < NL; ++v) {
                    own[v] = fat<NF, NFP>(a.v.tr1, ne, v, t.e, f, fp);
                    nbv[v] = fat<NF, NFP>(a.v.tr1, ne, v, b, fo, fq);
                }
#pragma unroll
                for (int v = 0; v < NL; ++v) sQs[(f * NL + v) * NFP + fp] = R(0.5) * (own[v] + nbv[v]);
            } else if (b <= kMortar) {
                const long long sl = kMortar - b;
#pragma unroll
                for (int v = 0; v < NL; ++v)
                    sQs[(f * NL + v) * NFP + fp] = R(0.5) * (fat<NF, NFP>(a.v.tr1, ne, v, t.e, f, fp) +
                                                             a.v.mtr1[((long long)v * a.v.g.nslot + sl) * NFP + fp]);
            } else {
                // walls: rho*, c* one-sided; u* the part of the wall's velocity (no slip) or
                // of the fluid's (Navier slip) tangential to the wall, b - (b.Ja/|Ja|^2) Ja
                const bool slip = a.v.wr.kind[w] == 2;
                R bv[D], av[D], ba = R(0), aa = R(0);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    av[k] = fat<NF, NFP>(a.v.fmet, ne, k, t.e, f, fp);
                    bv[k] = slip ? fat<NF, NFP>(a.v.tr1, ne, 1 + k, t.e, f, fp) : a.v.wr.uw[w][k];
                    ba += bv[k] * av[k];
                    aa += av[k] * av[k];
                }
                const R sb = ba / aa;
#pragma unroll
                for (int v = 0; v < NL; ++v)
                    sQs[(f * NL + v) * NFP + fp] =
                        (v >= 1 && v <= D) ? bv[v - 1] - sb * av[v - 1] : fat<NF, NFP>(a.v.tr1, ne, v, t.e, f, fp);
            }
        }
        stage_face_metrics<D, N, R>(a, t, sJf);
        sQ[n] = ns.rho;  // the state's shared copies after the face loads
#pragma unroll
        for (int k = 0; k < D; ++k) sQ[(1 + k) * NP + n] = ns.m[k] * ns.irho;
        sQ[(D + 1) * NP + n] = ns.c;
    }
    // pass-2 face values: T* (T_wall at walls) and (grad c)* . J a^dir (at walls
    // nsign |J a^dir| g_n from the contact angle)
    constexpr int KF = (NF * NFP + NP - 1) / NP;
    R pT[KF], pD[KF];
#pragma unroll
    for (int j = 0; j < KF; ++j) {
        const int q = n + j * NP;
        pT[j] = pD[j] = R(0);
        if (t.valid && q < NF * NFP) {
            const int f = q / NFP, fp = q % NFP, side = f & 1;
            int fo = fo0, o = o0, w = w0;
            const long long b = NF * NFP == NP ? b0 : face_nbr<D, N, R>(a.v, t, f, fo, o, w);
            const R ownT = fat<NF, NFP>(a.v.tr2, ne, 0, t.e, f, fp);
            const R ownD = fat<NF, NFP>(a.v.tr2, ne, 1, t.e, f, fp);
            if (b <= kMortar) {
                const long long sl = kMortar - b, ns = a.v.g.nslot;
                pT[j] = R(0.5) * (ownT + a.v.mtr2[sl * NFP + fp]);
                pD[j] = R(0.5) * (ownD + a.v.mtr2[(ns + sl) * NFP + fp]);
                if (fp == 0) sX[M::WG + f] = R(0);
            } else if (b >= 0) {
                const int fq = map_fp<P>(o, fp);
                pT[j] = R(0.5) * (ownT + fat<NF, NFP>(a.v.tr2, ne, 0, b, fo, fq));
                // the neighbour traced grad c . J a along its own face orientation
                pD[j] = R(0.5) * (ownD + R(facing_sign(f, fo)) * fat<NF, NFP>(a.v.tr2, ne, 1, b, fo, fq));
                if (fp == 0) sX[M::WG + f] = R(0);
            } else {
                const R cm = fat<NF, NFP>(a.v.tr1, ne, D + 1, t.e, f, fp);
                const R gn = a.v.wr.K[w] * (cm - a.v.wr.rl[w]) * (cm - a.v.wr.rv[w]);
                R a2 = R(0);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const R x = fat<NF, NFP>(a.v.fmet, ne, k, t.e, f, fp);
                    a2 += x * x;
                }
                // isothermal wall: T* = T_wall; Navier-slip wall: the fluid's trace (the wall
                // heat flux enters the energy flux) and, added with the pass-2 lines once
                // div u is known, (gamma_1/gamma_K) div u in the contact-angle value
                const bool slip = a.v.wr.kind[w] == 2;
                pT[j] = slip ? ownT : a.v.wr.Tw[w];
                pD[j] = (side ? R(1) : R(-1)) * sqrt(a2) * gn;
                if (fp == 0) sX[M::WG + f] = slip ? a.v.wr.g1gK[w] : R(0);
            }
        }
    }
    __syncthreads();
    // ---- pass 1 lines: reference derivatives (-> sG[dir][v]) and jumps q* - q- (-> sQs)
    if (t.valid) {
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
            const int stride = line_stride<P>(dir);
            for (int q = n; q < NL * NFP; q += NP) {
                const int v = q / NFP, line = q % NFP;
                const int base = line_base<P>(line, dir);
                R x[P], y[P], tm, tp;
                load_line<P, R>(sQ + v * NP, base, stride, x);
                dm_line<P, R>(a.op, x, y);
                trace_pair<P, R>(a.op, x, tm, tp);
                store_line<P, R>(sG + (dir * NL + v) * NP, base, stride, y);
                sQs[((2 * dir) * NL + v) * NFP + line] -= tm;
                sQs[((2 * dir + 1) * NL + v) * NFP + line] -= tp;
            }
        }
    }
    __syncthreads();

    // ---- node: physical gradients, temperature
    R g[D][D + 2];
    R T = R(0);
    if (t.valid) {
#pragma unroll
        for (int v = 0; v < NL; ++v) {
            R r[D], gv[D];
#pragma unroll
            for (int dir = 0; dir < D; ++dir) r[dir] = sG[(dir * NL + v) * NP + n];
            chain_gradient<D, N, R>(a, n, Ja, iJ, r, sQs + v * NFP, NL * NFP, sJf, gv);
#pragma unroll
            for (int k = 0; k < D; ++k) g[k][v] = gv[k];
        }
        R gc[D];
#pragma unroll
        for (int k = 0; k < D; ++k) gc[k] = g[k][D + 1];
        T = node_temperature<D, R>(a, ns, gc);
    }
    __syncthreads();  // the jumps in sQs are read; sX is reused below
    R *sT = sX, *sTs = sT + NP, *sDs = sTs + NF * NFP, *sRT = sDs + NF * NFP, *sRG = sRT + D * NP;
    if (t.valid) {
#pragma unroll
        for (int k = 0; k < D; ++k)
#pragma unroll
            for (int v = 0; v < NL; ++v) sG[(k * NL + v) * NP + n] = g[k][v];
        sT[n] = T;
#pragma unroll
        for (int j = 0; j < KF; ++j) {
            const int q = n + j * NP;
            if (q < NF * NFP) {
                sTs[q] = pT[j];
                sDs[q] = pD[j];
            }
        }
    }
    __syncthreads();

    // ---- pass 2 lines: tasks (dir, line) lift T and form the jumps of T and of
    //      grad c . J a^dir; tasks (dir, k, line) differentiate d c/d x_k along dir
    if (t.valid) {
        for (int q = n; q < D * NFP + D * D * NFP; q += NP) {
            if (q < D * NFP) {
                const int dir = q / NFP, line = q % NFP;
                const int base = line_base<P>(line, dir), stride = line_stride<P>(dir);
                R x[P], y[P], tm, tp;
                load_line<P, R>(sT, base, stride, x);
                dm_line<P, R>(a.op, x, y);
                trace_pair<P, R>(a.op, x, tm, tp);
                store_line<P, R>(sRT + dir * NP, base, stride, y);
                sTs[(2 * dir) * NFP + line] -= tm;
                sTs[(2 * dir + 1) * NFP + line] -= tp;
                R om = R(0), op = R(0);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    load_line<P, R>(sG + (k * NL + D + 1) * NP, base, stride, x);
                    trace_pair<P, R>(a.op, x, tm, tp);
                    om += tm * sJf[(k * NF + 2 * dir) * NFP + line];
                    op += tp * sJf[(k * NF + 2 * dir + 1) * NFP + line];
                }
                sDs[(2 * dir) * NFP + line] -= om;
                sDs[(2 * dir + 1) * NFP + line] -= op;
            } else {
                const int qq = q - D * NFP;
                const int dir = qq / (D * NFP), k = (qq / NFP) % D, line = qq % NFP;
                const int base = line_base<P>(line, dir), stride = line_stride<P>(dir);
                R x[P], y[P];
                load_line<P, R>(sG + (k * NL + D + 1) * NP, base, stride, x);
                dm_line<P, R>(a.op, x, y);
                store_line<P, R>(sRG + (dir * D + k) * NP, base, stride, y);
            }
        }
        // Navier-slip wall ends of the (dir, line) tasks above, by the same threads:
        // nsign |J a| (gamma_1/gamma_K) div u- joins the contact-angle value
        for (int q = n; q < D * NFP; q += NP) {
            const int dir = q / NFP, line = q % NFP;
            const R wgm = sX[M::WG + 2 * dir], wgp = sX[M::WG + 2 * dir + 1];
            if (wgm != R(0) || wgp != R(0)) {
                const int base = line_base<P>(line, dir), stride = line_stride<P>(dir);
                R x[P], tm, tp, dvm = R(0), dvp = R(0), am = R(0), ap = R(0);
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    load_line<P, R>(sG + (k * NL + 1 + k) * NP, base, stride, x);
                    trace_pair<P, R>(a.op, x, tm, tp);
                    dvm += tm;
                    dvp += tp;
                    const R jm = sJf[(k * NF + 2 * dir) * NFP + line], jp = sJf[(k * NF + 2 * dir + 1) * NFP + line];
                    am += jm * jm;
                    ap += jp * jp;
                }
                sDs[(2 * dir) * NFP + line] -= sqrt(am) * wgm * dvm;
                sDs[(2 * dir + 1) * NFP + line] += sqrt(ap) * wgp * dvp;
            }
        }
    }
    __syncthreads();
    R gT[D], lap = R(0);
    R rho = R(0), E = R(0), c = R(0), m[D], u[D], du[D][D], gc[D], S_[NV], pf = R(0);
    if (t.valid) {
        R r[D];
#pragma unroll
        for (int dir = 0; dir < D; ++dir) r[dir] = sRT[dir * NP + n];
        chain_gradient<D, N, R>(a, n, Ja, iJ, r, sTs, NFP, sJf, gT);
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
            const int i = ncoord<P>(n, dir), fp = node_fp<P>(n, dir);
            R vol = R(0);
#pragma unroll
            for (int k = 0; k < D; ++k) vol += Ja[dir][k] * sRG[(dir * D + k) * NP + n];
            lap += vol + sel<P, R>(a.op.Lp, i) * sDs[(2 * dir + 1) * NFP + fp] - sel<P, R>(a.op.Lm, i) * sDs[(2 * dir) * NFP + fp];
        }
        lap *= iJ;
#pragma unroll
        for (int k = 0; k < D; ++k) sGT[k * NP + n] = gT[k];
        rho = ns.rho;
        E = ns.E;
        c = ns.c;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            m[k] = ns.m[k];
            u[k] = m[k] * ns.irho;
            gc[k] = g[k][D + 1];
#pragma unroll
            for (int kk = 0; kk < D; ++kk) du[k][kk] = g[k][1 + kk];
        }
        pf = flux_pressure<R>(a.pr, rho, T, R(1) / (R(1) - R(kBvdw) * rho));
        source_terms<D, R>(a.pr, rho, u, c, g, S_);
    }
    if constexpr (DIAG != 0) {
        if (t.valid) a.v.out[t.e * NP + n] = to_f64<R>(entropy_production<D, R>(a.pr, rho, c, T, du, gT, lap));
        return;
    }
    __syncthreads();  // pass-2 buffers dead before the volume buffers reuse sX

    // ---- volume integral of the contravariant fluxes: acc_i = sum_dir sum_l Dhat_il (F.Ja^dir)_l;
    //      the fluxes of all directions first, then every line contracted in place
    R *sF = sX;  // [D][NV][NP]
    if (t.valid) {
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
            R F[NV];
            flux_vec<D, R>(a.pr, Ja[dir], rho, m, u, E, c, pf, du, gT, gc, lap, F);
#pragma unroll
            for (int v = 0; v < NV; ++v) sF[(dir * NV + v) * NP + n] = F[v];
        }
    }
    __syncthreads();
    if (t.valid) {
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
            const int stride = line_stride<P>(dir);
            for (int q = n; q < NV * NFP; q += NP) {
                int v, line;
                line_task<NV, NFP>(dir, q, v, line);
                const int base = line_base<P>(line, dir);
                R x[P], y[P];
                load_line_d<P, R, M::per_elem>(dir, sF + (dir * NV + v) * NP, base, stride, x);
                dhat_line<P, R>(a.op, x, R(1), y);
                store_line_d<P, R, M::per_elem>(dir, sF + (dir * NV + v) * NP, base, stride, y);
            }
        }
    }
    __syncthreads();
    R *sN = sX + M::XN;
    if (t.valid) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R acc = sF[v * NP + n];
#pragma unroll
            for (int d = 1; d < D; ++d) acc = sF[(d * NV + v) * NP + n] + acc;
            nat<NP>(a.v.Utv, ne, v, t.e, n) = S_[v] - iJ * acc;
        }
        sN[n] = rho;
#pragma unroll
        for (int k = 0; k < D; ++k) sN[(1 + k) * NP + n] = m[k];
        sN[(D + 1) * NP + n] = E;
        sN[(D + 2) * NP + n] = c;
        sN[NV * NP + n] = lap;
    }
    __syncthreads();

    // ---- face records (one task per line of one direction, both ends)
    R *sR = sX;
    if (t.valid) {
        for (int q = n; q < D * NFP; q += NP) {
            const int dir = q / NFP, line = q % NFP;
            const int base = line_base<P>(line, dir), stride = line_stride<P>(dir);
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const R *src = face_source_c<D, N, R>(k, sG, sGT, sN);
                R x[P], am, ap;
                load_line<P, R>(src, base, stride, x);
                trace_pair<P, R>(a.op, x, am, ap);
                sR[((2 * dir) * NQ + k) * NFP + line] = am;
                sR[((2 * dir + 1) * NQ + k) * NFP + line] = ap;
            }
        }
    }
    __syncthreads();

    // ---- face data (one face point per task): U-, F.Ja, scaled signal speed; walls: the
    //      complete flux along the face metric
    if (t.valid) {
        const long long st = ne * NF * NFP;
        for (int q = n; q < NF * NFP; q += NP) {
            const int f = q / NFP, fp = q % NFP;
            int f_nb = fo0, o_nb = o0, w = w0;
            const long long bn = NF * NFP == NP ? b0 : face_nbr<D, N, R>(a.v, t, f, f_nb, o_nb, w);
            const bool wall = bn < 0 && bn > kMortar;
            R r[NQ], av[D];
#pragma unroll
            for (int k = 0; k < NQ; ++k) r[k] = sR[(f * NQ + k) * NFP + fp];
            if (bn <= kMortar && f_nb == 1) {
                // big side of a mortar: its records go to the mortar kernel, which
                // evaluates this side's flux at the small faces' points
#pragma unroll
                for (int k = 0; k < NQ; ++k) a.v.mrec[((long long)k * a.v.g.nslot + (kMortar - bn)) * NFP + fp] = r[k];
            }
#pragma unroll
            for (int k = 0; k < D; ++k) av[k] = sJf[(k * NF + f) * NFP + fp];
            R F[NV], lam, pf, sig;
            face_flux_c<D, R>(a, f, w, wall, r, av, F, lam, pf, sig);
            const unsigned fo = foff<NF, NFP>(t.e, f, fp);
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                (a.v.fd + v * st)[fo] = r[v];
                (a.v.fd + (NV + v) * st)[fo] = F[v];
            }
            (a.v.fd + (2 * NV) * st)[fo] = lam;
            if (a.pr.flux == 1) {
                (a.v.fd + (2 * NV + 1) * st)[fo] = pf;
                (a.v.fd + (2 * NV + 2) * st)[fo] = sig;
            }
        }
    }
}

template <int D, int N, typename R>
__global__ void __launch_bounds__(Shape<D, N>::NT, curved_min_blocks(Shape<D, N>::NT, DGK_THREADS_LIFT2C / (int)(sizeof(R) / 4)))
    k_lift2volc(KArgs<R> args)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    lift2volc_body<D, N, R>(a, blockIdx.x, smraw);
}

// rate of entropy production at the nodes (diagnostics; needs the pass-2 traces of the
// current state, written by k_lift1c and its mortar kernel)
template <int D, int N, typename R>
__global__ void __launch_bounds__(Shape<D, N>::NT) k_entropy_prodc(KArgs<R> args)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    lift2volc_body<D, N, R, 1>(a, blockIdx.x, smraw);
}

// ------------------------------------------------------------------ mortars
//
// A big face facing 2 (2D) or 4 (3D) half-size faces: the small sides' neighbour data are
// the big side's interpolated to their points, the big side's the L2 projection of the
// small sides' (Sec. 3.1, mortar method).  One block per mortar; the results go to the
// mortar slots that the stage kernels read for these faces.

template <int D>
__host__ __device__ constexpr int mortar_stride() { return 4 + 4 * (D == 2 ? 2 : 4); }

// which 0: the pass-1 traces (rho, u, c); which 1: the pass-2 traces (T and grad c . J a,
// the latter signed to the receiving face's orientation and scaled by the surface-element
// ratio 2^(D-1)).
template <int D, int N, typename R>
__global__ void __launch_bounds__(256) k_mortar_traces(KArgs<R> args, int which)
{
    using S = Shape<D, N>;
    constexpr int P = S::P, NF = S::NF, NFP = S::NFP, NL = S::NL, NSUB = D == 2 ? 2 : 4;
    const KView<R> &v = args.v;
    const OpsR<R> &op = args.op;
    const int *mt = v.mort + (long long)blockIdx.x * mortar_stride<D>();
    const long long ne = v.g.ne, ns = v.g.nslot, B = mt[0];
    const int fB = mt[1], sB = mt[2];
    const int nvar = which ? 2 : NL;
    const R *src = which ? v.tr2 : v.tr1;
    R *dst = which ? v.mtr2 : v.mtr1;
    const R scale = R(D == 2 ? 2 : 4);
    for (int q = threadIdx.x; q < nvar * NSUB * NFP; q += blockDim.x) {
        const int var = q / (NSUB * NFP), p = (q / NFP) % NSUB, fq = q % NFP;
        const int *sb = mt + 4 + 4 * p;
        const int qq = map_fp<P>(sb[2], fq), u = qq % P, w = qq / P, h0 = p & 1, h1 = (p >> 1) & 1;
        R acc = R(0);
        if (D == 2) {
#pragma unroll
            for (int i = 0; i < P; ++i) acc += op.Im[h0][u * P + i] * fat<NF, NFP>(src, ne, var, B, fB, i);
        } else {
            for (int j = 0; j < P; ++j) {
                R row = R(0);
#pragma unroll
                for (int i = 0; i < P; ++i) row += op.Im[h0][u * P + i] * fat<NF, NFP>(src, ne, var, B, fB, i + P * j);
                acc += op.Im[h1][w * P + j] * row;
            }
        }
        if (which && var == 1) acc *= R(facing_sign(sb[1], fB)) / scale;
        dst[((long long)var * ns + sb[3]) * NFP + fq] = acc;
    }
    for (int q = threadIdx.x; q < nvar * NFP; q += blockDim.x) {
        const int var = q / NFP, ib = q % NFP, i = ib % P, j = ib / P;
        R acc = R(0);
        for (int p = 0; p < NSUB; ++p) {
            const int *sb = mt + 4 + 4 * p;
            const int h0 = p & 1, h1 = (p >> 1) & 1;
            const R sg = which && var == 1 ? R(facing_sign(fB, sb[1])) * scale : R(1);
            for (int fq = 0; fq < NFP; ++fq) {
                const int qq = map_fp<P>(sb[2], fq), u = qq % P, w = qq / P;
                const R wt = D == 2 ? op.Pm[h0][i * P + u] : op.Pm[h0][i * P + u] * op.Pm[h1][j * P + w];
                acc += wt * sg * fat<NF, NFP>(src, ne, var, sb[0], sb[1], fq);
            }
        }
        dst[((long long)var * ns + sB) * NFP + ib] = acc;
    }
}

// Face data of mortars: at each small face point the big side's face record is
// interpolated and its one-sided flux evaluated along the small face's metric (the small
// side's slot); the small side's Rusanov flux, as k_surf_rk forms it, turned to the big
// face's orientation and surface element (x 2^(D-1)) and projected, is the big side's
// complete flux (written to its own face data, read by k_surf_rk as at a wall).
template <int D, int N, typename R>
__global__ void __launch_bounds__(256) k_mortar_flux(KArgs<R> args)
{
    using S = Shape<D, N>;
    using FR = FaceRecC<D>;
    constexpr int P = S::P, NF = S::NF, NFP = S::NFP, NV = S::NV, NQ = FR::NQ, NSUB = D == 2 ? 2 : 4;
    extern __shared__ __align__(16) unsigned char smraw[];
    R *sF = reinterpret_cast<R *>(smraw);  // [NSUB][NV][NFP]
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    const KView<R> &v = args.v;
    const OpsR<R> &op = args.op;
    const int *mt = v.mort + (long long)blockIdx.x * mortar_stride<D>();
    const long long ne = v.g.ne, ns = v.g.nslot, B = mt[0], st = ne * NF * NFP;
    const int fB = mt[1], sB = mt[2];
    const R scale = R(D == 2 ? 2 : 4);
    for (int q = threadIdx.x; q < NSUB * NFP; q += blockDim.x) {
        const int p = q / NFP, fq = q % NFP;
        const int *sb = mt + 4 + 4 * p;
        const long long Se = sb[0];
        const int fS = sb[1], sS = sb[3];
        const int qq = map_fp<P>(sb[2], fq), u = qq % P, w = qq / P, h0 = p & 1, h1 = (p >> 1) & 1;
        R r[NQ], av[D];
#pragma unroll
        for (int k = 0; k < NQ; ++k) {
            const R *rec = v.mrec + ((long long)k * ns + sB) * NFP;
            R acc = R(0);
            if (D == 2) {
#pragma unroll
                for (int i = 0; i < P; ++i) acc += op.Im[h0][u * P + i] * rec[i];
            } else {
                for (int j = 0; j < P; ++j) {
                    R row = R(0);
#pragma unroll
                    for (int i = 0; i < P; ++i) row += op.Im[h0][u * P + i] * rec[i + P * j];
                    acc += op.Im[h1][w * P + j] * row;
                }
            }
            r[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < D; ++k) av[k] = fat<NF, NFP>(v.fmet, ne, k, Se, fS, fq);
        R F[NV], lam, pf, sig;
        face_flux_c<D, R>(a, fS, fS, false, r, av, F, lam, pf, sig);
        const long long so = sS * NFP + fq, sst = ns * NFP;
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            v.mfd[k * sst + so] = r[k];
            v.mfd[(NV + k) * sst + so] = F[k];
        }
        v.mfd[(2 * NV) * sst + so] = lam;
        v.mfd[(2 * NV + 1) * sst + so] = pf;
        v.mfd[(2 * NV + 2) * sst + so] = sig;
        // the small side's numerical flux, as k_surf_rk forms it
        const long long oo = (Se * NF + fS) * NFP + fq;
        R Uo[NV], Fo[NV], Fs[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            Uo[k] = v.fd[k * st + oo];
            Fo[k] = v.fd[(NV + k) * st + oo];
        }
        const R lo = v.fd[(2 * NV) * st + oo];
        if (a.pr.flux == 1)
            pair_flux_c<D, R, 1>(fS & 1, Uo, Fo, lo, v.fd[(2 * NV + 1) * st + oo], v.fd[(2 * NV + 2) * st + oo], r, F, lam,
                                 pf, sig, av, Fs);
        else
            pair_flux_c<D, R, 0>(fS & 1, Uo, Fo, lo, R(0), R(0), r, F, lam, R(0), R(0), av, Fs);
        const R sg = R(facing_sign(fB, fS)) * scale;
#pragma unroll
        for (int k = 0; k < NV; ++k) sF[(p * NV + k) * NFP + fq] = sg * Fs[k];
    }
    __syncthreads();
    // the projection accumulates in double: its weights and the small sides' fluxes are
    // bulk-type values whose products are exact in double, so the big side's flux is the
    // projection of the small sides' fluxes to one rounding.  (With model 2 the momentum
    // flux carries p + alpha/2 rho^2 ~ 1e2 |J a|; summed in float over the 2^(D-1) NFP
    // terms, its rounding broke the mortar's conservation by ~1e-5 |J a| per face and step.)
    for (int q = threadIdx.x; q < NV * NFP; q += blockDim.x) {
        const int k = q / NFP, ib = q % NFP, i = ib % P, j = ib / P;
        double acc = 0.0;
        for (int p = 0; p < NSUB; ++p) {
            const int *sb = mt + 4 + 4 * p;
            const int h0 = p & 1, h1 = (p >> 1) & 1;
            for (int fq = 0; fq < NFP; ++fq) {
                const int qq = map_fp<P>(sb[2], fq), u = qq % P, w = qq / P;
                const double wt = D == 2 ? to_f64<R>(op.Pm[h0][i * P + u])
                                         : to_f64<R>(op.Pm[h0][i * P + u]) * to_f64<R>(op.Pm[h1][j * P + w]);
                acc += wt * to_f64<R>(sF[(p * NV + k) * NFP + fq]);
            }
        }
        v.fd[(NV + k) * st + (B * NF + fB) * NFP + ib] = to_bulk<R>(acc);
    }
}

// ------------------------------------------------------------------ launchers

struct CurvedTable {
    cudaError_t (*prepare)();
    cudaError_t (*lift1)(const void *args, cudaStream_t s);
    cudaError_t (*lift2vol)(const void *args, cudaStream_t s);
    cudaError_t (*surf)(const void *args, int mode, int stage, cudaStream_t s);
    cudaError_t (*nodeT)(const void *args, int mode, cudaStream_t s);
    cudaError_t (*mortar_traces)(const void *args, int which, int nmort, cudaStream_t s);
    cudaError_t (*mortar_flux)(const void *args, int nmort, cudaStream_t s);
    cudaError_t (*entropy_prod)(const void *args, cudaStream_t s);
};

template <int D, int N, typename R>
struct CurvedLauncher {
    using S = Shape<D, N>;
    static constexpr size_t sm_lift1 = (size_t)S::EPB * CLiftC<D, N, R>::smem_per_elem * sizeof(R);
    static constexpr size_t sm_lift2 = (size_t)S::EPB * K2CSmem<D, N, R>::per_elem * sizeof(R);
    static constexpr size_t sm_surf = (size_t)S::EPB * K3Smem<D, N, R>::per_elem * sizeof(R);

    static unsigned blocks(const KArgs<R> &a) { return (unsigned)((a.v.g.ne + S::EPB - 1) / S::EPB); }

    static cudaError_t prepare()
    {
        cudaError_t err;
        if ((err = cudaFuncSetAttribute(k_lift1c<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_lift1))) return err;
        if ((err = cudaFuncSetAttribute(k_lift2volc<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_lift2)))
            return err;
        if (DGK_CURVED_CARVEOUT &&
            (err = cudaFuncSetAttribute(k_lift2volc<D, N, R>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                        (int)cudaSharedmemCarveoutMaxShared)))
            return err;
        if ((err = cudaFuncSetAttribute(k_surf_rk<D, N, R, 0, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_surf)))
            return err;
        if ((err = cudaFuncSetAttribute(k_surf_rk<D, N, R, 0, 1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_surf)))
            return err;
        if ((err = cudaFuncSetAttribute(k_entropy_prodc<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_lift2)))
            return err;
        return cudaFuncSetAttribute(k_node_Tc<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_lift1);
    }
    static cudaError_t entropy_prod(const void *p, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_entropy_prodc<D, N, R><<<blocks(a), S::NT, sm_lift2, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t lift1(const void *p, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_lift1c<D, N, R><<<blocks(a), S::NT, sm_lift1, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t lift2vol(const void *p, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_lift2volc<D, N, R><<<blocks(a), S::NT, sm_lift2, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t surf(const void *p, int mode, int stage, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        if (a.pr.flux == 1) k_surf_rk<D, N, R, 0, 1, 1><<<blocks(a), S::NT, sm_surf, s>>>(a, mode, stage);
        else k_surf_rk<D, N, R, 0, 0, 1><<<blocks(a), S::NT, sm_surf, s>>>(a, mode, stage);
        return cudaGetLastError();
    }
    static cudaError_t nodeT(const void *p, int mode, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_node_Tc<D, N, R><<<blocks(a), S::NT, sm_lift1, s>>>(a, mode);
        return cudaGetLastError();
    }
    static cudaError_t mortar_traces(const void *p, int which, int nmort, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_mortar_traces<D, N, R><<<nmort, 128, 0, s>>>(a, which);
        return cudaGetLastError();
    }
    static cudaError_t mortar_flux(const void *p, int nmort, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        constexpr size_t sm = (size_t)(D == 2 ? 2 : 4) * S::NV * S::NFP * sizeof(R);
        k_mortar_flux<D, N, R><<<nmort, 128, sm, s>>>(a);
        return cudaGetLastError();
    }
    static const CurvedTable *table()
    {
        static const CurvedTable t = {prepare, lift1, lift2vol, surf, nodeT, mortar_traces, mortar_flux, entropy_prod};
        return &t;
    }
};

}  // namespace dgk

#define DGK_DEFINE_CURVED_TABLE(FNAME, DIM, REAL)                      \
    const dgk::CurvedTable *FNAME(int N)                               \
    {                                                                  \
        switch (N) {                                                   \
        case 2: return dgk::CurvedLauncher<DIM, 2, REAL>::table();     \
        case 3: return dgk::CurvedLauncher<DIM, 3, REAL>::table();     \
        case 4: return dgk::CurvedLauncher<DIM, 4, REAL>::table();     \
        case 5: return dgk::CurvedLauncher<DIM, 5, REAL>::table();     \
        default: return nullptr;                                       \
        }                                                              \
    }
