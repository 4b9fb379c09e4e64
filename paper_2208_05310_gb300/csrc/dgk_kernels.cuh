// dgk_kernels.cuh -- the three kernels of one RK stage of the DGSEM relaxed-NSK scheme,
// plus set-up kernels (pass-1 traces of a new state, nodal temperature / energy).
//
// One stage = three launches; each kernel depends on face data of its neighbours that
// the previous launch produced (BR1 pass 1 -> temperature -> pass 2 -> face flux):
//   k_lift1      lifts c only (the temperature needs grad c), recovers T at the nodes and
//                writes the face traces of T and of dc/dx_normal (inputs of pass 2)
//   k_lift2vol   BR1 pass 1 of (rho, u, c) (recomputed, not stored), T, pass 2 (grad T,
//                lap c), point fluxes and sources, volume integral with Dhat per
//                direction -> U_t(vol); face traces -> one-sided face data (U-, F-, lambda-)
//   k_surf_rk    Rusanov (or HLLC) + central viscous flux per face point, surface lifting
//                with l(+-1)/w, Jacobian 2/h, RK stage update in FP64, new pass-1 traces
//
// Thread layout: one thread per node for point-wise work (EPB elements per block).  The
// tensor-product contractions are done line by line ("sum factorisation"): a thread
// loads the P values of one line into registers and produces all P outputs, and both
// end-point traces, with the operator entries read as uniform kernel-parameter
// constants.  Element-local fields are staged in shared memory.
#pragma once

#include "dgk_common.cuh"

// Resident threads per SM requested from the compiler for each stage kernel, as a
// register budget (65536 / threads).  Measured on the 3D N = 5 FP32-bulk workload:
// k_lift1 gains 8% at 1728 threads, k_lift2vol 4% at 1080; k_surf_rk runs 27% faster
// at 896 (72 registers, four 216-thread blocks per SM) than with the compiler's 92
// registers (two blocks), and slower again at 1120, where it starts to spill.  0 leaves
// the choice to the compiler.  The FP64 form asks for half the threads (its values take
// two registers).
#ifndef DGK_THREADS_LIFT1
#define DGK_THREADS_LIFT1 1728
#endif
#ifndef DGK_THREADS_LIFT2
#define DGK_THREADS_LIFT2 1080
#endif
#ifndef DGK_THREADS_SURF
#define DGK_THREADS_SURF 896
#endif
// k_surf_rk with the HLLC flux loads U and G after the face phase: its face phase needs
// the registers that hold them otherwise (1.77 against 2.10 ms on the 3D N = 5 workload).
#ifndef DGK_SURF_HLLC_LATE
#define DGK_SURF_HLLC_LATE 1
#endif
#ifndef DGK_THREADS_SURF_HLLC
#define DGK_THREADS_SURF_HLLC 896  // k_surf_rk with the HLLC flux
#endif

namespace dgk {

__host__ __device__ constexpr int min_blocks(int threads_per_block, int threads_per_sm)
{
    return threads_per_sm / threads_per_block > 0 ? threads_per_sm / threads_per_block : 1;
}

// 1D operators in the bulk type (see Ops).
template <typename R>
struct OpsR {
    // Row pairs of Dhat for the packed float contractions: Dh2[2 (p P + l) + h] =
    // Dhat_{2p+h, l} (rows 2p and 2p+1 side by side); traces side by side:
    // lmp[2 l] = l_l(-1), lmp[2 l + 1] = l_l(+1).  Filled by fill_pairs() from Dh, lm, lp.
    alignas(8) R Dh2[kMaxP * kMaxP];
    alignas(8) R lmp[2 * kMaxP];
    R Dh[kMaxP * kMaxP];
    R Dm[kMaxP * kMaxP];  // D_ij = l_j'(xi_i) (strong form, curved elements)
    alignas(8) R Lp[kMaxP];
    alignas(8) R Lm[kMaxP];
    R lp[kMaxP], lm[kMaxP];
    // mortars of half-size faces h = 0, 1 (eta = (xi + 2h - 1)/2): Im[h][j*P+i] = l_i(eta_h(xi_j)),
    // Pm[h][i*P+j] = w_j/(2 w_i) l_i(eta_h(xi_j))
    R Im[2][kMaxP * kMaxP], Pm[2][kMaxP * kMaxP];
};

// The packed layouts of OpsR (Dh2, lmp) from its Dh, lm, lp, for P nodes per line.
template <typename R>
__host__ void fill_pairs(OpsR<R> &o, int P)
{
    for (int p = 0; 2 * p + 1 < P; ++p)
        for (int l = 0; l < P; ++l) {
            o.Dh2[2 * (p * P + l)] = o.Dh[(2 * p) * P + l];
            o.Dh2[2 * (p * P + l) + 1] = o.Dh[(2 * p + 1) * P + l];
        }
    for (int l = 0; l < P; ++l) {
        o.lmp[2 * l] = o.lm[l];
        o.lmp[2 * l + 1] = o.lp[l];
    }
}

// Per-problem data: geometry, walls and device arrays.  Kernel parameters for a single
// problem; shared memory in the batched kernel.
template <typename R>
struct KView {
    Geom g;
    GeomR<R> gr;
    WallsR<R> wr;
    double *U;           // [NV][ne][NP]
    double *G;           // [NV][ne][NP]
    R *Us;               // FP32-bulk form: [NV+1][ne][NP] shadow of U (see NodeState); FP64 form: null
    R *Utv;              // [NV][ne][NP] volume part of U_t
    R *tr1;              // [NL][ne][NF][NFP] pass-1 traces of (rho, u, c)
    R *tr2;              // [2][ne][NF][NFP] traces of T and of d c / d x_normal
    R *fd;               // [2NV+3][ne][NF][NFP] one-sided face data: U, F = F^C - F^V, lambda, and
                         // for the HLLC flux the convective pressure and the sound speed
    const R *met;        // curved elements: [D*D+1][ne][NP] J a^dir_k (plane dir*D + k) and 1/J; box: null
    const R *fmet;       // curved elements: [D][ne][NF][NFP] J a^dir_k at the face points; box: null
    const int *conn;     // unstructured connectivity [ne][NF][3] (neighbour or -1 - wall, its face,
                         // face-point orientation; mortar faces: -1000 - slot, 1 on the big side);
                         // null: the box's
    R *mtr1, *mtr2, *mfd;  // mortar slots: the effective neighbour data of mortar faces ([NL], [2],
                           // [2NV+1] x [nslot][NFP]); big sides' face records mrec [NQ][nslot][NFP]
    R *mrec;
    const int *mort;       // mortars [nmort][4 + 4 nsub]: (big element, its face, its slot, -), then per
                           // sub-face p (small element, its face, orientation, its slot)
    double *out;         // rhs output [NV][ne][NP], or nodal T [ne][NP]
    const double *coef;  // device [A_0..A_4, B_0..B_4, dt] of this problem
    unsigned *status;
};

template <typename R>
struct KArgs {
    KView<R> v;
    Phys ph;
    PhysR<R> pr;
    OpsR<R> op;
};

// What a kernel body sees: the problem's view plus the physics and the operators of
// its degree (kernel parameters in both forms, so operator entries stay uniform
// constant-bank operands).
template <typename R>
struct Ctx {
    const KView<R> &v;
    const Phys &ph;
    const PhysR<R> &pr;
    const OpsR<R> &op;
};

// ------------------------------------------------------------------ line helpers

template <int P, typename R>
__device__ __forceinline__ void load_line(const R *f, int base, int stride, R x[P])
{
#pragma unroll
    for (int l = 0; l < P; ++l) x[l] = f[base + l * stride];
}

template <int P, typename R>
__device__ __forceinline__ void store_line(R *f, int base, int stride, const R y[P])
{
#pragma unroll
    for (int l = 0; l < P; ++l) f[base + l * stride] = y[l];
}

// ---- packed float arithmetic: fma.rn.f32x2 / mul.rn.f32x2 on two floats side by side
// in a 64-bit register pair, rounded as the two scalar operations are.  The line
// contractions below are instruction-issue bound; packing halves their FMA instructions.
// A translation unit may switch it off before including this header: the batched
// ensemble's grouped kernels (three degrees' bodies per kernel) ran 15% slower packed
// (17.9 against 15.6 ms per step), the single-problem kernels 2-5% faster.
#ifndef DGK_PACKED_LINES
#define DGK_PACKED_LINES 1
#endif
__device__ __forceinline__ unsigned long long f2_pack(float a, float b)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long r, float &a, float &b)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b)
{
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
template <typename R>
__device__ __forceinline__ unsigned long long f2_at(const R *p)  // two adjacent floats
{
    const float2 v = *reinterpret_cast<const float2 *>(p);
    return f2_pack(v.x, v.y);
}

// task q -> (plane v, line) of a line task over NPL planes of NFP lines.  Lines along z
// (stride NFP, consecutive lines in consecutive banks) with NFP > 32: warp w takes lines
// 0..31 of plane w, the last NFP-32 lines of every plane follow, so that no warp spans
// two planes (plane offsets of NP words shift the banks); other directions: plane-major.
template <int NPL, int NFP>
__device__ __forceinline__ void line_task(int dir, int q, int &v, int &line)
{
    if (NFP > 32 && dir == 2) {
        if (q < 32 * NPL) {
            v = q >> 5;
            line = q & 31;
        } else {
            const int r = q - 32 * NPL;
            v = r / (NFP - 32);
            line = 32 + r % (NFP - 32);
        }
    } else {
        v = q / NFP;
        line = q % NFP;
    }
}

// x-lines (stride 1) of an even number of floats starting on an 8-byte boundary: float2
template <int P, typename R>
__device__ __forceinline__ void load_line_v2(const R *f, int base, R x[P])
{
    const float2 *p = reinterpret_cast<const float2 *>(f + base);
#pragma unroll
    for (int l = 0; l < P / 2; ++l) { const float2 t = p[l]; x[2 * l] = t.x; x[2 * l + 1] = t.y; }
}
template <int P, typename R>
__device__ __forceinline__ void store_line_v2(R *f, int base, const R y[P])
{
    float2 *p = reinterpret_cast<float2 *>(f + base);
#pragma unroll
    for (int l = 0; l < P / 2; ++l) p[l] = make_float2(y[2 * l], y[2 * l + 1]);
}
template <int P, typename R, int PER_ELEM>
__device__ __forceinline__ void load_line_d(int dir, const R *f, int base, int stride, R x[P])
{
    if (sizeof(R) == 4 && P % 2 == 0 && PER_ELEM % 2 == 0 && dir == 0) load_line_v2<P, R>(f, base, x);
    else load_line<P, R>(f, base, stride, x);
}
template <int P, typename R, int PER_ELEM>
__device__ __forceinline__ void store_line_d(int dir, R *f, int base, int stride, const R y[P])
{
    if (sizeof(R) == 4 && P % 2 == 0 && PER_ELEM % 2 == 0 && dir == 0) store_line_v2<P, R>(f, base, y);
    else store_line<P, R>(f, base, stride, y);
}

// BR1 lifting along one line (Sec. 3.1, weak form, collocated Gauss quadrature):
//   y_i = (2/h) [ sum_l Dhat_il x_l + Lp_i q*_+ - Lm_i q*_- ]
// (float: rows in pairs, packed; the face terms as two FMAs after the sum)
template <int P, typename R>
__device__ __forceinline__ void lift_line(const OpsR<R> &o, const R x[P], R qm, R qp, R s, R y[P])
{
    if constexpr (sizeof(R) == 4 && DGK_PACKED_LINES) {
        unsigned long long xb[P];
#pragma unroll
        for (int l = 0; l < P; ++l) xb[l] = f2_pack(x[l], x[l]);
        const unsigned long long qpb = f2_pack(qp, qp), qmb = f2_pack(-qm, -qm), sb = f2_pack(s, s);
#pragma unroll
        for (int p = 0; 2 * p + 1 < P; ++p) {
            unsigned long long acc = f2_pack(0.0f, 0.0f);
#pragma unroll
            for (int l = 0; l < P; ++l) acc = f2_fma(f2_at(&o.Dh2[2 * (p * P + l)]), xb[l], acc);
            acc = f2_fma(f2_at(&o.Lp[2 * p]), qpb, acc);
            acc = f2_fma(f2_at(&o.Lm[2 * p]), qmb, acc);
            f2_unpack(f2_mul(sb, acc), y[2 * p], y[2 * p + 1]);
        }
        if (P % 2) {
            constexpr int i = P - 1;
            R acc = R(0);
#pragma unroll
            for (int l = 0; l < P; ++l) acc += o.Dh[i * P + l] * x[l];
            acc += o.Lp[i] * qp;
            acc += o.Lm[i] * (-qm);
            y[i] = s * acc;
        }
    } else {
        // the operations of the packed form, in its order (the scalar and packed forms
        // give the same bits)
#pragma unroll
        for (int i = 0; i < P; ++i) {
            R acc = R(0);
#pragma unroll
            for (int l = 0; l < P; ++l) acc += o.Dh[i * P + l] * x[l];
            acc += o.Lp[i] * qp;
            acc += o.Lm[i] * (-qm);
            y[i] = s * acc;
        }
    }
}

// y_i = s sum_l Dhat_il x_l (volume integral of one flux line)
template <int P, typename R>
__device__ __forceinline__ void dhat_line(const OpsR<R> &o, const R x[P], R s, R y[P])
{
    if constexpr (sizeof(R) == 4 && DGK_PACKED_LINES) {
        unsigned long long xb[P];
#pragma unroll
        for (int l = 0; l < P; ++l) xb[l] = f2_pack(x[l], x[l]);
        const unsigned long long sb = f2_pack(s, s);
#pragma unroll
        for (int p = 0; 2 * p + 1 < P; ++p) {
            unsigned long long acc = f2_pack(0.0f, 0.0f);
#pragma unroll
            for (int l = 0; l < P; ++l) acc = f2_fma(f2_at(&o.Dh2[2 * (p * P + l)]), xb[l], acc);
            f2_unpack(f2_mul(sb, acc), y[2 * p], y[2 * p + 1]);
        }
        if (P % 2) {
            constexpr int i = P - 1;
            R acc = R(0);
#pragma unroll
            for (int l = 0; l < P; ++l) acc += o.Dh[i * P + l] * x[l];
            y[i] = s * acc;
        }
    } else {
#pragma unroll
        for (int i = 0; i < P; ++i) {
            R acc = R(0);
#pragma unroll
            for (int l = 0; l < P; ++l) acc += o.Dh[i * P + l] * x[l];
            y[i] = s * acc;
        }
    }
}

// traces of one line at xi = -1 and xi = +1 (float: the two traces packed)
template <int P, typename R>
__device__ __forceinline__ void trace_pair(const OpsR<R> &o, const R x[P], R &tm, R &tp)
{
    if constexpr (sizeof(R) == 4 && DGK_PACKED_LINES) {
        unsigned long long acc = f2_pack(0.0f, 0.0f);
#pragma unroll
        for (int l = 0; l < P; ++l) acc = f2_fma(f2_at(&o.lmp[2 * l]), f2_pack(x[l], x[l]), acc);
        f2_unpack(acc, tm, tp);
    } else {
        R am = R(0), ap = R(0);
#pragma unroll
        for (int l = 0; l < P; ++l) {
            am += o.lm[l] * x[l];
            ap += o.lp[l] * x[l];
        }
        tm = am;
        tp = ap;
    }
}

// Device arrays are [plane][element][...]: an element-node array has planes of ne NP
// values, a face array planes of ne NF NFP.  An access takes the plane's base (the same
// for every thread of a launch) plus a 32-bit offset inside the plane: the library
// refuses meshes whose planes exceed 2^32 values, so the offset never wraps, and the
// address costs one wide multiply-add instead of 64-bit index arithmetic per access.
template <int NF, int NFP, typename T>
__device__ __forceinline__ T &fat(T *p, long long ne, int v, long long e, int f, int fp)
{
    return (p + (long long)v * (ne * (NF * NFP)))[((unsigned)e * NF + (unsigned)f) * NFP + (unsigned)fp];
}
template <int NP, typename T>
__device__ __forceinline__ T &nat(T *p, long long ne, int v, long long e, int n)
{
    return (p + (long long)v * (ne * NP))[(unsigned)e * NP + (unsigned)n];
}
// offset of (e, f, fp) inside a face-array plane, and the plane base
template <int NF, int NFP>
__device__ __forceinline__ unsigned foff(long long e, int f, int fp)
{
    return ((unsigned)e * NF + (unsigned)f) * NFP + (unsigned)fp;
}

// The neighbour's face point matching face point fp under orientation o: (u, v) = o & 1 ?
// (b, a) : (a, b) of fp = a + P b; u and v reversed by bits 1 and 2.
template <int P>
__device__ __forceinline__ int map_fp(int o, int fp)
{
    const int a = fp % P, b = fp / P;
    int u = (o & 1) ? b : a, v = (o & 1) ? a : b;
    if (o & 2) u = P - 1 - u;
    if (o & 4) v = P - 1 - v;
    return u + P * v;
}

// Sign between the face-metric orientations of two facing faces (J a^dir along +xi_dir
// of each element): +1 when one is a plus and the other a minus face, else -1.
__device__ __forceinline__ int facing_sign(int f, int fo) { return ((f ^ fo) & 1) ? 1 : -1; }

template <typename R>
__device__ __forceinline__ void check_state(unsigned *status, R rho, R T, R E)
{
    unsigned s = 0;
    if (!isfinite(rho) || !isfinite(T) || !isfinite(E)) s |= kStatNonFinite;
    else if (!(rho > R(0) && rho < R(1.0 / kBvdw) && T > R(0))) s |= kStatDomain;
    if (s) atomicOr(status, s);
}

// Common per-thread prologue: local element, node, validity, element coordinates.
// Neighbours are computed on demand (no per-thread array indexed at run time).
template <int D, int N, int EB = 0>
struct Slot {
    using S = Shape<D, N, EB>;
    int le, n;
    long long e;
    bool valid;
    int cx, cy, cz;
    __device__ Slot(const Geom &g, long long blk)
    {
        le = threadIdx.x / S::NP;
        n = threadIdx.x % S::NP;
        e = blk * S::EPB + le;
        valid = (int)threadIdx.x < S::NT && e < g.ne;
        const unsigned ue = valid ? (unsigned)e : 0u, n0 = (unsigned)g.n[0], n1 = (unsigned)g.n[1];
        const unsigned q0 = g.div0.div(ue), q1 = g.div1.div(q0);
        cx = (int)(ue - q0 * n0);
        cy = (int)(q0 - q1 * n1);
        cz = D == 3 ? (int)q1 : 0;
    }
    // neighbour across face f = 2*dir + side, or -1 at a wall
    __device__ __forceinline__ long long nbr(const Geom &g, int f) const
    {
        const int dir = f >> 1;
        const bool plus = f & 1;
        const int cd = dir == 0 ? cx : (dir == 1 ? cy : cz);
        const int nd = dir == 0 ? g.n[0] : (dir == 1 ? g.n[1] : g.n[2]);
        const int per = dir == 0 ? g.periodic[0] : (dir == 1 ? g.periodic[1] : g.periodic[2]);
        const long long stride = dir == 0 ? 1LL : (dir == 1 ? (long long)g.n[0] : (long long)g.n[0] * g.n[1]);
        int cn = cd + (plus ? 1 : -1);
        if (cn < 0 || cn >= nd) {
            if (!per) return -1;
            cn = plus ? 0 : nd - 1;
        }
        return e + (long long)(cn - cd) * stride;
    }
};

// ------------------------------------------------------------------ c-lifting (k_lift1, k_node_T)
//
// Lifts c in every direction (BR1 with central c*, one-sided at walls).  On return
// sDc[d][n] holds dc/dx_d; with write_tr2 the traces of dc/dx_d on the two faces normal
// to d are written to tr2[1].

template <int D, int N, typename R, int EB = 0>
struct CLift {
    using S = Shape<D, N, EB>;
    static constexpr int smem_per_elem = S::NP + S::NF * S::NFP + D * S::NP + S::NP;  // c, c*, dc, T

    __device__ static void run(const Ctx<R> &a, const Slot<D, N, EB> &t, R c, R *sC, R *sCs, R *sDc, bool write_tr2)
    {
        constexpr int P = S::P, NP = S::NP, NF = S::NF, NFP = S::NFP;
        const long long ne = a.v.g.ne;
        if (t.valid) {
            for (int q = t.n; q < NF * NFP; q += NP) {
                const int f = q / NFP, fp = q % NFP, dir = f >> 1, side = f & 1;
                const R own = fat<NF, NFP>(a.v.tr1, ne, D + 1, t.e, f, fp);
                const long long b = t.nbr(a.v.g, f);
                sCs[q] = b >= 0 ? R(0.5) * (own + fat<NF, NFP>(a.v.tr1, ne, D + 1, b, 2 * dir + 1 - side, fp)) : own;
            }
            sC[t.n] = c;  // after the face loads, so that c's own load is not waited for first
        }
        __syncthreads();
        if (t.valid) {
            for (int q = t.n; q < D * NFP; q += NP) {
                const int dir = q / NFP, line = q % NFP;
                const int base = line_base<P>(line, dir), stride = line_stride<P>(dir);
                R x[P], y[P];
                load_line<P, R>(sC, base, stride, x);
                lift_line<P, R>(a.op, x, sCs[(2 * dir) * NFP + line], sCs[(2 * dir + 1) * NFP + line], a.v.gr.inv2h[dir], y);
                store_line<P, R>(sDc + dir * NP, base, stride, y);
                if (write_tr2) {
                    R tm, tp;
                    trace_pair<P, R>(a.op, y, tm, tp);
                    fat<NF, NFP>(a.v.tr2, ne, 1, t.e, 2 * dir, line) = tm;
                    fat<NF, NFP>(a.v.tr2, ne, 1, t.e, 2 * dir + 1, line) = tp;
                }
            }
        }
        __syncthreads();
    }
};

// One node's conserved state in the bulk type, plus (FP32-bulk form) the energy balance
// bal = rho e + a rho^2 of the temperature recovery (Eq. totalenergyalpha), formed in
// double from the FP64 state and then rounded: near the spinodal the two terms nearly
// cancel, so the sum is taken before any rounding to float.
//
// The FP64 form reads the double state.  The FP32-bulk form reads the shadow Us, which
// every writer of the FP64 state (the RK update, the trace kernel after set-up) fills
// from it: U in float and bal -- the same roundings the kernels would otherwise apply
// to the double state per node and per kernel, done once per stage.
template <int D, typename R>
struct NodeState {
    static constexpr int NV = D + 3;
    R rho, irho, m[D], E, c;
    R bal;  // FP32-bulk form only
    __device__ __forceinline__ void from_double(const double *Ud)
    {
        rho = to_bulk<R>(Ud[0]);
        irho = R(1) / rho;
#pragma unroll
        for (int k = 0; k < D; ++k) m[k] = to_bulk<R>(Ud[1 + k]);
        E = to_bulk<R>(Ud[D + 1]);
        c = to_bulk<R>(Ud[D + 2]);
        bal = sizeof(R) == 4 ? to_bulk<R>(fma(kAvdw * Ud[0], Ud[0], Ud[D + 1])) : R(0);
    }
    __device__ __forceinline__ void load(const KView<R> &v, long long e, int n, int np)
    {
        if constexpr (sizeof(R) == 8) {
            double Ud[NV];
#pragma unroll
            for (int k = 0; k < NV; ++k) Ud[k] = (v.U + (long long)k * (v.g.ne * np))[(unsigned)e * np + (unsigned)n];
            from_double(Ud);
        } else {
            R u[NV + 1];
#pragma unroll
            for (int k = 0; k <= NV; ++k) u[k] = (v.Us + (long long)k * (v.g.ne * np))[(unsigned)e * np + (unsigned)n];
            rho = u[0];
            irho = R(1) / rho;
#pragma unroll
            for (int k = 0; k < D; ++k) m[k] = u[1 + k];
            E = u[D + 1];
            c = u[D + 2];
            bal = u[NV];
        }
    }
    // FP32-bulk form: write the shadow of this state (built by from_double)
    __device__ __forceinline__ void store_shadow(const KView<R> &v, long long e, int n, int np) const
    {
        if constexpr (sizeof(R) == 4) {
            const long long st = v.g.ne * np;
            const unsigned o = (unsigned)e * np + (unsigned)n;
            v.Us[o] = rho;
#pragma unroll
            for (int k = 0; k < D; ++k) (v.Us + (1 + k) * st)[o] = m[k];
            (v.Us + (D + 1) * st)[o] = E;
            (v.Us + (D + 2) * st)[o] = c;
            (v.Us + NV * st)[o] = bal;
        }
    }
};

template <int D, typename R>
__device__ __forceinline__ R node_temperature(const Ctx<R> &a, const NodeState<D, R> &q, const R *gc)
{
    R msq = R(0), gc2 = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        msq += q.m[k] * q.m[k];
        gc2 += gc[k] * gc[k];
    }
    const R d = q.rho - q.c;
    if constexpr (sizeof(R) == 8) return temperature_f64(a.ph, q.rho, q.irho, q.E, d, msq, gc2);
    else return temperature_bulk(a.pr, q.bal, q.irho, d, msq, gc2);
}

// ------------------------------------------------------------------ kernel 1

template <int D, int N, typename R, int EB = 0>
__device__ __forceinline__ void lift1_body(const Ctx<R> &a, long long blk, unsigned char *smraw)
{
    using S = Shape<D, N, EB>;
    using L = CLift<D, N, R, EB>;
    constexpr int P = S::P, NP = S::NP, NFP = S::NFP, NF = S::NF, NV = S::NV;
        const Slot<D, N, EB> t(a.v.g, blk);
    R *sC = reinterpret_cast<R *>(smraw) + (size_t)t.le * L::smem_per_elem;
    R *sCs = sC + NP, *sDc = sCs + NF * NFP, *sT = sDc + D * NP;
    NodeState<D, R> q;
    if (t.valid) q.load(a.v, t.e, t.n, NP);
    L::run(a, t, q.c, sC, sCs, sDc, true);
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
        for (int q = t.n; q < D * NFP; q += NP) {
            const int dir = q / NFP, line = q % NFP;
            R x[P], tm, tp;
            load_line<P, R>(sT, line_base<P>(line, dir), line_stride<P>(dir), x);
            trace_pair<P, R>(a.op, x, tm, tp);
            fat<NF, NFP>(a.v.tr2, ne, 0, t.e, 2 * dir, line) = tm;
            fat<NF, NFP>(a.v.tr2, ne, 0, t.e, 2 * dir + 1, line) = tp;
        }
    }
}

template <int D, int N, typename R, int EB = 0>
__global__ void __launch_bounds__(Shape<D, N, EB>::NT, min_blocks(Shape<D, N, EB>::NT, DGK_THREADS_LIFT1 / (int)(sizeof(R) / 4))) k_lift1(KArgs<R> args)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    lift1_body<D, N, R, EB>(a, blockIdx.x, smraw);
}

// ------------------------------------------------------------------ face flux

// Face record of one face point of a face normal to dir, in the order
//   U (NV) | d u_k / d x_dir (D) | d u_dir / d x_k, k != dir (D-1) | div u | dT/dx_dir |
//   grad c (D) | lap c
template <int D>
struct FaceRec {
    static constexpr int NV = D + 3;
    static constexpr int DDU = NV, DUD = NV + D, DIV = NV + 2 * D - 1, GT = NV + 2 * D, GC = NV + 2 * D + 1,
                         LAP = NV + 3 * D + 1, NQ = NV + 3 * D + 2;
};

// v[d] for a run-time direction d, by selection (no run-time index into a register array)
template <int D, typename R>
__device__ __forceinline__ R pick(int d, const R *v)
{
    R x = v[0];
#pragma unroll
    for (int k = 1; k < D; ++k) x = d == k ? v[k] : x;
    return x;
}

// Convective flux F^C in +e_dir of the state U with convective pressure p and
// irho = 1/rho (Eq. navierstokeskorteweg_palpha for model 2).
template <int D, typename R>
__device__ __forceinline__ void conv_flux(int dir, const R *U, R p, R irho, R *F)
{
    R m[D];
#pragma unroll
    for (int k = 0; k < D; ++k) m[k] = U[1 + k];
    const R mn = pick<D, R>(dir, m), un = mn * irho;
    F[0] = mn;
#pragma unroll
    for (int k = 0; k < D; ++k) F[1 + k] = m[k] * un + (k == dir ? p : R(0));
    F[D + 1] = (U[D + 1] + p) * un;
    F[D + 2] = U[D + 2] * un;
}

// HLLC flux in +e_dir between UL (the - side) and UR (the + side), with their convective
// fluxes FL, FR, pressures, sound speeds and 1/rho (Toro 2009, Sec. 10.4): wave speeds
// S_L = min(u_L - a_L, u_R - a_R), S_R = max(u_L + a_L, u_R + a_R); contact speed S* from
// the pressures and momenta; star state of the side the contact leaves behind,
// chi (1, S* e_dir + tangential u, E/rho + (S* - u)(S* + p/(rho (S - u))), c/rho) with
// chi = rho (S - u)/(S - S*), the order parameter carried like a passive scalar.
template <int D, typename R>
__device__ __forceinline__ void hllc_flux(int dir, const R *UL, const R *FL, R pL, R aL, R irL, const R *UR,
                                          const R *FR, R pR, R aR, R irR, R *F)
{
    constexpr int NV = D + 3;
    R mL[D], mR[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        mL[k] = UL[1 + k];
        mR[k] = UR[1 + k];
    }
    const R rL = UL[0], rR = UR[0];
    const R uL = pick<D, R>(dir, mL) * irL, uR = pick<D, R>(dir, mR) * irR;
    const R SL = fmin(uL - aL, uR - aR), SR = fmax(uL + aL, uR + aR);
    if (SL >= R(0) || SR <= R(0)) {
        const bool left = SL >= R(0);
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = left ? FL[v] : FR[v];
        return;
    }
    const R Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
    const bool left = Ss >= R(0);
    R UK[NV], FK[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        UK[v] = left ? UL[v] : UR[v];
        FK[v] = left ? FL[v] : FR[v];
    }
    const R SK = left ? SL : SR, pK = left ? pL : pR, rK = UK[0], irK = left ? irL : irR, uK = left ? uL : uR;
    const R chi = rK * (SK - uK) / (SK - Ss);
    R Us[NV];
    Us[0] = chi;
#pragma unroll
    for (int k = 0; k < D; ++k) Us[1 + k] = chi * (k == dir ? Ss : UK[1 + k] * irK);
    Us[D + 1] = chi * (UK[D + 1] * irK + (Ss - uK) * (Ss + pK * irK / (SK - uK)));
    Us[D + 2] = chi * UK[D + 2] * irK;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = FK[v] + SK * (Us[v] - UK[v]);
}

// Numerical flux of one interior face point from the one-sided face data fd of its two
// sides (indices iL on the - side, iR on the + side, array stride st): HLLC for the
// convective part, central for the viscous part, F* = HLLC(F^C) - (F^V_L + F^V_R)/2 with
// F^V = F^C - F.  Written to out[v * ostride].
template <int D, typename R>
__device__ __forceinline__ void hllc_face(const R *fd, long long st, unsigned iL, unsigned iR, int dir, R *out,
                                       int ostride)
{
    constexpr int NV = D + 3;
    R UL[NV], UR[NV], FcL[NV], FcR[NV], Fh[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        UL[v] = (fd + v * st)[iL];
        UR[v] = (fd + v * st)[iR];
    }
    const R pL = (fd + (2 * NV + 1) * st)[iL], aL = (fd + (2 * NV + 2) * st)[iL];
    const R pR = (fd + (2 * NV + 1) * st)[iR], aR = (fd + (2 * NV + 2) * st)[iR];
    const R irL = R(1) / UL[0], irR = R(1) / UR[0];
    conv_flux<D, R>(dir, UL, pL, irL, FcL);
    conv_flux<D, R>(dir, UR, pR, irR, FcR);
    hllc_flux<D, R>(dir, UL, FcL, pL, aL, irL, UR, FcR, pR, aR, irR, Fh);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        const R FvL = FcL[v] - (fd + (NV + v) * st)[iL], FvR = FcR[v] - (fd + (NV + v) * st)[iR];
        out[v * ostride] = Fh[v] - R(0.5) * (FvL + FvR);
    }
}

// One-sided flux F(U-, grads-) in direction dir (interior faces), or the complete wall
// flux in +e_dir (wall faces; Sec. 2.4, Eq. bc_nsk_alpha with gamma_1 = gamma_2 =
// gamma_4 = 0: Rusanov against the mirrored ghost (rho, m - 2(m.n)n, rho e, c) with equal
// pressure and signal speed, minus the wall viscous flux with u_wall = 0, zeta = 0 and
// grad c . n from the contact angle), and the Rusanov signal speed |u_dir| + s.  The
// direction is a run-time value: the normal components are selected, so that face
// points of all directions share one instruction stream.
template <int D, typename R>
__device__ __forceinline__ void face_flux(const Ctx<R> &a, int f, int dir, bool wall, const R *r, R *F, R &lam, R &pf_out,
                                          R &s_out)
{
    using FR = FaceRec<D>;
    const PhysR<R> &ph = a.pr;
    const R rho = r[0], E = r[D + 1], c = r[D + 2], irho = R(1) / rho;
    R m[D], u[D], gc[D], ddu[D], msq = R(0), gc2 = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        m[k] = r[1 + k];
        u[k] = m[k] * irho;
        msq += m[k] * m[k];
        gc[k] = r[FR::GC + k];
        gc2 += gc[k] * gc[k];
        ddu[k] = r[FR::DDU + k];
    }
    // temperature of the interpolated face state (bulk type: the face state itself is
    // an interpolation in the bulk type)
    const R T = (E + R(kAvdw) * rho * rho - R(0.5) * msq * irho - ph.half_alpha * (rho - c) * (rho - c) -
                 ph.half_gK * gc2) * irho * ph.inv_Rcv;
    const R iomb = R(1) / (R(1) - R(kBvdw) * rho);
    const R pf = flux_pressure<R>(ph, rho, T, iomb);
    const R un = pick<D, R>(dir, u), mn = pick<D, R>(dir, m), dnn = pick<D, R>(dir, ddu);
    const R sig = signal_speed<R>(ph, rho, T, iomb);
    lam = fabs(un) + sig;
    pf_out = pf;
    s_out = sig;
    const R divu = r[FR::DIV];
    // viscous stress column tau_{k, dir} = mu (du_k/dx_dir + du_dir/dx_k) - 2/3 mu div u delta;
    // du_dir/dx_k (k != dir) sits in slot k of the record's second block if k < dir, else k-1
    R tau[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const R below = k < D - 1 ? r[FR::DUD + (k < D - 1 ? k : 0)] : R(0);
        const R above = k > 0 ? r[FR::DUD + (k > 0 ? k - 1 : 0)] : R(0);
        const R dud = k == dir ? dnn : (k < dir ? below : above);
        tau[k] = ph.mu * (ddu[k] + dud) - (k == dir ? ph.two_thirds_mu * divu : R(0));
    }
    const R gTd = r[FR::GT], gcd = pick<D, R>(dir, gc), lap = r[FR::LAP];
    if (!wall && ph.model == 0) {
        // original NSK: viscous plus Korteweg stress, NSK energy flux; the c slot (= rho)
        // carries the mass flux (see flux_dir)
        R gr2 = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) gr2 += gc[k] * gc[k];
        R work = R(0);
        F[0] = mn;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            R tk = tau[k] - ph.gK * gc[k] * gcd;
            if (k == dir) tk += ph.gK * (R(0.5) * gr2 + rho * lap);
            work += tk * u[k];
            F[1 + k] = m[k] * un - tk + (k == dir ? pf : R(0));
        }
        const R je = ph.kap * gTd - ph.gK * rho * gcd * divu;
        F[D + 1] = (E + pf) * un - (work + je);
        F[D + 2] = mn;
        return;
    }
    if (!wall) {
        R work = R(0);
        F[0] = mn;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            work += tau[k] * u[k];
            F[1 + k] = m[k] * un - tau[k] + (k == dir ? pf : R(0));
        }
        const R zeta = ph.beta * (ph.gK * lap + ph.alpha * (rho - c));
        const R je = ph.kap * gTd - ph.gK * c * gcd * divu + ph.gK * gcd * zeta;
        F[D + 1] = (E + pf) * un - (work + je);
        F[D + 2] = c * un - ph.gKbeta * gcd;
        return;
    }
    const R nsign = (f & 1) ? R(1) : R(-1);
    const R gn = a.v.wr.K[f] * (c - a.v.wr.rl[f]) * (c - a.v.wr.rv[f]);
    R Fi[D + 3], Fg[D + 3], Ui[D + 3], Ug[D + 3];
    const R ui = un, ug = -un;
    Fi[0] = mn;
    Fg[0] = -mn;
    Ui[0] = Ug[0] = rho;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const R mg = k == dir ? -m[k] : m[k];
        const R pk = k == dir ? pf : R(0);
        Fi[1 + k] = m[k] * ui + pk;
        Fg[1 + k] = mg * ug + pk;
        Ui[1 + k] = m[k];
        Ug[1 + k] = mg;
    }
    Fi[D + 1] = (E + pf) * ui;
    Fg[D + 1] = (E + pf) * ug;
    Fi[D + 2] = c * ui;
    Fg[D + 2] = c * ug;
    Ui[D + 1] = Ug[D + 1] = E;
    Ui[D + 2] = Ug[D + 2] = c;
    const bool plus = nsign > R(0);
    if (ph.flux == 1) {
        // HLLC against the ghost, same pressure and sound speed on both sides
        if (plus) hllc_flux<D, R>(dir, Ui, Fi, pf, sig, irho, Ug, Fg, pf, sig, irho, F);
        else hllc_flux<D, R>(dir, Ug, Fg, pf, sig, irho, Ui, Fi, pf, sig, irho, F);
    } else {
#pragma unroll
        for (int v = 0; v < D + 3; ++v) {
            const R FL = plus ? Fi[v] : Fg[v], FRr = plus ? Fg[v] : Fi[v];
            const R UL = plus ? Ui[v] : Ug[v], UR = plus ? Ug[v] : Ui[v];
            F[v] = R(0.5) * (FL + FRr) - R(0.5) * lam * (UR - UL);
        }
    }
    if (a.v.wr.kind[f] == 2) {
        // generalized Navier slip (Eq. bc_nsk_alpha): outward tangential traction
        // gamma_1 div u (grad c)_k - gamma_2 u_k, normal traction of the fluid; work on the
        // slipping fluid; heat flux -gamma_3 (1/T_wall - 1/T); zeta = -gamma_1 gamma_4 div u;
        // grad c . n with the gamma_1 div u term.  F is the flux in +e_dir: outward
        // quantities enter with nsign.
        const R gnn = gn + a.v.wr.g1gK[f] * divu;
        R work = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const R tk = a.v.wr.g1[f] * divu * gc[k] - a.v.wr.g2[f] * u[k];
            if (k == dir) F[1 + k] -= tau[k];
            else {
                F[1 + k] -= nsign * tk;
                work += tk * u[k];
            }
        }
        const R zeta = -a.v.wr.g1g4[f] * divu;
        const R qn = -a.v.wr.g3[f] * (R(1) / a.v.wr.Tw[f] - R(1) / T);
        F[D + 1] -= nsign * (work + qn - ph.gK * c * gnn * divu + ph.gK * gnn * zeta);
        F[D + 2] -= nsign * ph.gKbeta * gnn;
        return;
    }
    // isothermal no-slip wall: the traction does work on the wall's velocity (a sliding wall)
    R work = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        F[1 + k] -= tau[k];
        work += tau[k] * a.v.wr.uw[f][k];
    }
    F[D + 1] -= work + ph.kap * gTd - nsign * ph.gK * c * gn * divu;
    F[D + 2] -= nsign * ph.gKbeta * gn;
}

// Nodal array holding record quantity k of the faces normal to dir (FaceRec order):
// conserved U and div u, lap c in sN; lifted gradients in sG[d][v] (v = rho, u_1..u_D, c);
// grad T in sGT.
template <int D, int N, typename R, int EB = 0>
__device__ __forceinline__ const R *face_source(int k, int dir, const R *sG, const R *sGT, const R *sN)
{
    using S = Shape<D, N, EB>;
    using FR = FaceRec<D>;
    constexpr int NP = S::NP, NL = S::NL, NV = S::NV;
    if (k < FR::DDU) return sN + k * NP;
    if (k < FR::DUD) return sG + (dir * NL + 1 + (k - FR::DDU)) * NP;
    if (k < FR::DIV) {
        const int j = k - FR::DUD, kabs = j < dir ? j : j + 1;
        return sG + (kabs * NL + 1 + dir) * NP;
    }
    if (k == FR::DIV) return sN + NV * NP;
    if (k == FR::GT) return sGT + dir * NP;
    if (k < FR::LAP) return sG + ((k - FR::GC) * NL + D + 1) * NP;
    return sN + (NV + 1) * NP;
}

// ------------------------------------------------------------------ kernel 2

// One line of BR1 pass 2 along the compile-time direction DIR: q < NFP lifts T along
// line q into grad T, otherwise dc/dx_DIR along line q - NFP into the DIR part of lap c.
// (A compile-time direction turns the line's base, stride and buffer offsets into
// constants: one loop per direction over 2 NFP tasks ran faster than one loop over all
// 2 D NFP tasks with a run-time direction, although it takes D rounds instead of one.)
template <int DIR, int P, int NP, int NFP, int NL, int D, typename R>
__device__ __forceinline__ void pass2_line(const Ctx<R> &a, int q, const R *sT, const R *sTs, const R *sDs, const R *sG,
                                           R *sGT, R *sLp)
{
    const bool isT = q < NFP;
    const int line = isT ? q : q - NFP;
    const int base = line_base<P>(line, DIR), stride = line_stride<P>(DIR);
    const R *src = isT ? sT : sG + (DIR * NL + D + 1) * NP;
    const R *qs = isT ? sTs : sDs;
    R *dst = isT ? sGT + DIR * NP : sLp + DIR * NP;
    R x[P], y[P];
    load_line<P, R>(src, base, stride, x);
    lift_line<P, R>(a.op, x, qs[(2 * DIR) * NFP + line], qs[(2 * DIR + 1) * NFP + line], a.v.gr.inv2h[DIR], y);
    store_line<P, R>(dst, base, stride, y);
}

template <int D, int N, typename R, int EB = 0>
struct K2Smem {
    using S = Shape<D, N, EB>;
    static constexpr int G = D * S::NL * S::NP;  // pass-1 gradients sG[d][v][n]
    static constexpr int GT = D * S::NP;         // grad T
    static constexpr int X1 = S::NL * S::NP + S::NF * S::NL * S::NFP;  // prims, q*
    static constexpr int X2 = S::NP + 2 * S::NF * S::NFP + D * S::NP;  // T, T*, Dc*, lap parts
    static constexpr int X4 = D * S::NV * S::NP;                       // volume: F and its integral per direction
    static constexpr int SR = S::NF * FaceRec<D>::NQ * S::NFP;         // traced face records
    static constexpr int XN = X4 > SR ? X4 : SR;                       // nodal U/div/lap (sN) offset
    static constexpr int X3 = XN + (S::NV + 2) * S::NP;
    static constexpr int XA = X1 > X2 ? X1 : X2;
    static constexpr int X = XA > X3 ? XA : X3;
    static constexpr int per_elem = G + GT + X;
};

// DIAG 1: the same liftings, then the rate of entropy production of each node into
// a.v.out[e][n] (double) in place of the volume integral and the face data.
template <int D, int N, typename R, int EB = 0, int DIAG = 0>
__device__ __forceinline__ void lift2vol_body(const Ctx<R> &a, long long blk, unsigned char *smraw)
{
    using S = Shape<D, N, EB>;
    using M = K2Smem<D, N, R, EB>;
    constexpr int P = S::P, NP = S::NP, NFP = S::NFP, NF = S::NF, NL = S::NL, NV = S::NV;
        const Slot<D, N, EB> t(a.v.g, blk);
    // one face point per thread when NF NFP = NP (3D, N = 5): its neighbour once
    const long long bn = (NF * NFP == NP && t.valid) ? t.nbr(a.v.g, t.n / NFP) : -1;
    R *sG = reinterpret_cast<R *>(smraw) + (size_t)t.le * M::per_elem;
    R *sGT = sG + M::G, *sX = sGT + M::GT;
    const long long ne = a.v.g.ne;
    const int n = t.n;

    // ---- pass 1: prims (rho, u, c) and central face values (one-sided rho, c and u* = 0 at walls)
    R *sQ = sX, *sQs = sX + NL * NP;
    NodeState<D, R> ns;
    if (t.valid) {
        ns.load(a.v, t.e, n, NP);
        for (int q = n; q < NF * NFP; q += NP) {
            const int f = q / NFP, fp = q % NFP, dir = f >> 1, side = f & 1;
            const long long b = NF * NFP == NP ? bn : t.nbr(a.v.g, f);
            // two branches, so that interior points issue no loads of wall constants (a
            // select over both would cost 13% of the kernel)
            if (b >= 0) {
                R own[NL], nbv[NL];  // all loads issued before the first use
#pragma unroll
                for (int v = 0; v < NL; ++v) {
                    own[v] = fat<NF, NFP>(a.v.tr1, ne, v, t.e, f, fp);
                    nbv[v] = fat<NF, NFP>(a.v.tr1, ne, v, b, 2 * dir + 1 - side, fp);
                }
#pragma unroll
                for (int v = 0; v < NL; ++v) sQs[(f * NL + v) * NFP + fp] = R(0.5) * (own[v] + nbv[v]);
            } else {
                // walls: u* = the wall's velocity (no slip; zero unless the wall slides), or
                // the fluid's tangential velocity (Navier slip)
                const bool slip = a.v.wr.kind[f] == 2;
#pragma unroll
                for (int v = 0; v < NL; ++v) {
                    const R own = fat<NF, NFP>(a.v.tr1, ne, v, t.e, f, fp);
                    sQs[(f * NL + v) * NFP + fp] =
                        (v >= 1 && v <= D && (!slip || v == 1 + dir)) ? a.v.wr.uw[f][v - 1] : own;
                }
            }
        }
        sQ[n] = ns.rho;
#pragma unroll
        for (int k = 0; k < D; ++k) sQ[(1 + k) * NP + n] = ns.m[k] * ns.irho;
        sQ[(D + 1) * NP + n] = ns.c;
    }
    // pass-2 central face values (T*, and dc/dx_dir* for the lap c lifting; at walls T_wall
    // and the contact-angle gradient), loaded now so that their latency overlaps pass 1
    constexpr int KF = (NF * NFP + NP - 1) / NP;  // face points per thread
    R pT[KF], pD[KF];
#pragma unroll
    for (int j = 0; j < KF; ++j) {
        const int q = n + j * NP;
        pT[j] = pD[j] = R(0);
        if (t.valid && q < NF * NFP) {
            const int f = q / NFP, fp = q % NFP, dir = f >> 1, side = f & 1;
            const long long b = NF * NFP == NP ? bn : t.nbr(a.v.g, f);
            const R ownT = fat<NF, NFP>(a.v.tr2, ne, 0, t.e, f, fp);
            const R ownD = fat<NF, NFP>(a.v.tr2, ne, 1, t.e, f, fp);
            if (b >= 0) {
                const int fo = 2 * dir + 1 - side;
                pT[j] = R(0.5) * (ownT + fat<NF, NFP>(a.v.tr2, ne, 0, b, fo, fp));
                pD[j] = R(0.5) * (ownD + fat<NF, NFP>(a.v.tr2, ne, 1, b, fo, fp));
            } else {
                // isothermal wall: T* = T_wall; Navier-slip wall: the fluid's trace (the
                // wall heat flux enters the energy flux); contact-angle gradient (its
                // gamma_1 div u part is added once div u is known, in the node phase)
                const R cm = fat<NF, NFP>(a.v.tr1, ne, D + 1, t.e, f, fp);
                const R gn = a.v.wr.K[f] * (cm - a.v.wr.rl[f]) * (cm - a.v.wr.rv[f]);
                pT[j] = a.v.wr.kind[f] == 2 ? ownT : a.v.wr.Tw[f];
                pD[j] = side ? gn : -gn;
            }
        }
    }
    __syncthreads();
    if (t.valid) {
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
            const int stride = line_stride<P>(dir);
            for (int q = n; q < NL * NFP; q += NP) {
                int v, line;
                line_task<NL, NFP>(dir, q, v, line);
                const int base = line_base<P>(line, dir);
                R x[P], y[P];
                load_line_d<P, R, M::per_elem>(dir, sQ + v * NP, base, stride, x);
                lift_line<P, R>(a.op, x, sQs[((2 * dir) * NL + v) * NFP + line], sQs[((2 * dir + 1) * NL + v) * NFP + line],
                                a.v.gr.inv2h[dir], y);
                store_line_d<P, R, M::per_elem>(dir, sG + (dir * NL + v) * NP, base, stride, y);
            }
        }
    }
    __syncthreads();

    // ---- node: gradients, temperature; pass-2 central face values
    R g[D][D + 2];
    R T = R(0);
    // the nodal region: written only after the volume integral, which reuses sX
    static_assert(M::X2 <= (NV + 2) * NP, "pass-2 buffers fit the nodal region");
    R *sT = sX + M::XN, *sTs = sT + NP, *sDs = sTs + NF * NFP, *sLp = sDs + NF * NFP;
    if (t.valid) {
#pragma unroll
        for (int d = 0; d < D; ++d)
#pragma unroll
            for (int v = 0; v < NL; ++v) g[d][v] = sG[(d * NL + v) * NP + n];
        R gc[D];
#pragma unroll
        for (int d = 0; d < D; ++d) gc[d] = g[d][D + 1];
        T = node_temperature<D, R>(a, ns, gc);
        sT[n] = T;
#pragma unroll
        for (int j = 0; j < KF; ++j) {
            const int q = n + j * NP;
            if (q < NF * NFP) {
                sTs[q] = pT[j];
                R dD = R(0);
                const int f = q / NFP;
                if (a.v.wr.kind[f] == 2 && a.v.wr.g1gK[f] != R(0) && (NF * NFP == NP ? bn : t.nbr(a.v.g, f)) < 0) {
                    // Eq. bc_contactangle_alpha: + (gamma_1/gamma_K) div u- at the face point
                    const int dir = f >> 1, fp = q % NFP;
                    const int base = line_base<P>(fp, dir), stride = line_stride<P>(dir);
                    R divu = R(0);
#pragma unroll
                    for (int k = 0; k < D; ++k)
#pragma unroll
                        for (int l = 0; l < P; ++l)
                            divu += ((f & 1) ? a.op.lp[l] : a.op.lm[l]) * sG[(k * NL + 1 + k) * NP + base + l * stride];
                    dD = ((f & 1) ? R(1) : R(-1)) * a.v.wr.g1gK[f] * divu;
                }
                sDs[q] = pD[j] + dD;
            }
        }
    }
    __syncthreads();

    // ---- pass 2: grad T (-> sGT) and the per-direction parts of lap c (-> sLp);
    //      per direction, tasks 0..NFP-1 lift T, the next NFP lift dc/dx_dir along dir
    if (t.valid) {
        for (int q = n; q < 2 * NFP; q += NP) pass2_line<0, P, NP, NFP, NL, D, R>(a, q, sT, sTs, sDs, sG, sGT, sLp);
        for (int q = n; q < 2 * NFP; q += NP) pass2_line<1, P, NP, NFP, NL, D, R>(a, q, sT, sTs, sDs, sG, sGT, sLp);
        if constexpr (D == 3)
            for (int q = n; q < 2 * NFP; q += NP) pass2_line<D - 1, P, NP, NFP, NL, D, R>(a, q, sT, sTs, sDs, sG, sGT, sLp);
    }
    __syncthreads();
    R gT[D], lap = R(0);
    R rho = R(0), E = R(0), c = R(0), m[D], u[D], du[D][D], gc[D], S_[NV], pf = R(0);
    if (t.valid) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
            gT[d] = sGT[d * NP + n];
            lap += sLp[d * NP + n];
        }
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

    // ---- volume integral: the fluxes of all directions, then in place along each line
    //      (2/h) sum_l Dhat_il F_l; acc = the sum over the directions
    R *sF = sX;  // [D][NV][NP]
    if (t.valid) {
#pragma unroll
        for (int dir = 0; dir < D; ++dir) {
            R F[NV];
            flux_dir<D, R>(a.pr, dir, rho, m, u, E, c, pf, du, gT, gc, lap, F);
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
                dhat_line<P, R>(a.op, x, a.v.gr.inv2h[dir], y);
                store_line_d<P, R, M::per_elem>(dir, sF + (dir * NV + v) * NP, base, stride, y);
            }
        }
    }
    __syncthreads();
    R *sN = sX + M::XN;  // nodal U, div u, lap c (clear of sF and the traced records)
    if (t.valid) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R acc = sF[v * NP + n];
#pragma unroll
            for (int d = 1; d < D; ++d) acc += sF[(d * NV + v) * NP + n];
            nat<NP>(a.v.Utv, ne, v, t.e, n) = S_[v] - acc;
        }
        sN[n] = rho;
#pragma unroll
        for (int k = 0; k < D; ++k) sN[(1 + k) * NP + n] = m[k];
        sN[(D + 1) * NP + n] = E;
        sN[(D + 2) * NP + n] = c;
        R divu = R(0);
#pragma unroll
        for (int k = 0; k < D; ++k) divu += du[k][k];
        sN[NV * NP + n] = divu;
        sN[(NV + 1) * NP + n] = lap;
    }
    __syncthreads();

    // ---- face records: one task per line of one direction traces every record quantity
    //      (FaceRec order) to both ends of the line, into sR[f][k][fp] (the line's values
    //      are loaded once for the two faces)
    using FR = FaceRec<D>;
    constexpr int NQ = FR::NQ;
    R *sR = sX;  // clear of sN; sF is dead
    if (t.valid) {
        for (int q = n; q < D * NFP; q += NP) {
            int dir, line;
            if (NFP > 32) {
                if (q < 32 * D) { dir = q >> 5; line = q & 31; }
                else { const int r = q - 32 * D; dir = r / (NFP - 32); line = 32 + r % (NFP - 32); }
            } else {
                dir = q / NFP;
                line = q % NFP;
            }
            const int base = line_base<P>(line, dir), stride = line_stride<P>(dir);
#pragma unroll
            for (int k = 0; k < NQ; ++k) {
                const R *src = face_source<D, N, R, EB>(k, dir, sG, sGT, sN);
                R x[P], am, ap;
                load_line<P, R>(src, base, stride, x);
                trace_pair<P, R>(a.op, x, am, ap);
                sR[((2 * dir) * NQ + k) * NFP + line] = am;
                sR[((2 * dir + 1) * NQ + k) * NFP + line] = ap;
            }
        }
    }
    __syncthreads();

    // ---- face data: one face point per task (interior: one-sided data; wall: the
    //      complete wall flux).  The direction is a run-time value: all face points of
    //      an element share one instruction stream.
    if (t.valid) {
        const long long st = ne * NF * NFP;
        for (int q = n; q < NF * NFP; q += NP) {
            const int f = q / NFP, fp = q % NFP, dir = f >> 1;
            const bool wall = (NF * NFP == NP ? bn : t.nbr(a.v.g, f)) < 0;
            R r[NQ];
#pragma unroll
            for (int k = 0; k < NQ; ++k) r[k] = sR[(f * NQ + k) * NFP + fp];
            R F[NV], lam, pf, sig;
            face_flux<D, R>(a, f, dir, wall, r, F, lam, pf, sig);
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

template <int D, int N, typename R, int EB = 0>
__global__ void __launch_bounds__(Shape<D, N, EB>::NT, min_blocks(Shape<D, N, EB>::NT, DGK_THREADS_LIFT2 / (int)(sizeof(R) / 4))) k_lift2vol(KArgs<R> args)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    lift2vol_body<D, N, R, EB>(a, blockIdx.x, smraw);
}

// rate of entropy production at the nodes (diagnostics; needs the pass-2 traces of the
// current state, written by k_lift1)
template <int D, int N, typename R, int EB = 0>
__global__ void __launch_bounds__(Shape<D, N, EB>::NT) k_entropy_prod(KArgs<R> args)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    lift2vol_body<D, N, R, EB, 1>(a, blockIdx.x, smraw);
}

// ------------------------------------------------------------------ kernel 3

template <int D, int N, typename R, int EB = 0>
struct K3Smem {
    using S = Shape<D, N, EB>;
    static constexpr int a1 = S::NF * S::NV * S::NFP;
    static constexpr int a2 = S::NL * S::NP;
    static constexpr int per_elem = a1 > a2 ? a1 : a2;
};

// New pass-1 traces of (rho, u, c) of the element's state (double U -> bulk type), and in
// the FP32-bulk form the shadow of the state.
template <int D, int N, typename R, int EB = 0>
__device__ __forceinline__ void write_traces(const Ctx<R> &a, const Slot<D, N, EB> &t, R *sQ, const double *Ud)
{
    using S = Shape<D, N, EB>;
    constexpr int P = S::P, NP = S::NP, NFP = S::NFP, NF = S::NF, NL = S::NL;
    if (t.valid) {
        NodeState<D, R> q;
        q.from_double(Ud);
        q.store_shadow(a.v, t.e, t.n, NP);
        sQ[t.n] = q.rho;
#pragma unroll
        for (int k = 0; k < D; ++k) sQ[(1 + k) * NP + t.n] = q.m[k] * q.irho;
        sQ[(D + 1) * NP + t.n] = q.c;
    }
    __syncthreads();
    if (t.valid) {
        const long long ne = a.v.g.ne;
        // One loop per direction (compile-time line base and stride: no run-time
        // direction selects or strided address arithmetic) where that takes no more
        // rounds of NP tasks than one loop over all directions does.
        constexpr int RD = (NL * NFP + NP - 1) / NP, RA = (D * NL * NFP + NP - 1) / NP;
        if constexpr (D * RD <= RA) {
#pragma unroll
            for (int dir = 0; dir < D; ++dir)
                for (int q = t.n; q < NL * NFP; q += NP) {
                    const int v = q / NFP, line = q % NFP;
                    R x[P], tm, tp;
                    load_line<P, R>(sQ + v * NP, line_base<P>(line, dir), line_stride<P>(dir), x);
                    trace_pair<P, R>(a.op, x, tm, tp);
                    fat<NF, NFP>(a.v.tr1, ne, v, t.e, 2 * dir, line) = tm;
                    fat<NF, NFP>(a.v.tr1, ne, v, t.e, 2 * dir + 1, line) = tp;
                }
        } else {
            for (int q = t.n; q < D * NL * NFP; q += NP) {
                const int dir = q / (NL * NFP), v = (q / NFP) % NL, line = q % NFP;
                R x[P], tm, tp;
                load_line<P, R>(sQ + v * NP, line_base<P>(line, dir), line_stride<P>(dir), x);
                trace_pair<P, R>(a.op, x, tm, tp);
                fat<NF, NFP>(a.v.tr1, ne, v, t.e, 2 * dir, line) = tm;
                fat<NF, NFP>(a.v.tr1, ne, v, t.e, 2 * dir + 1, line) = tp;
            }
        }
    }
}

// Convective flux along the vector a: (m.a, m (u.a) + p a, (rho e + p)(u.a), c (u.a)),
// irho = 1/rho.
template <int D, typename R>
__device__ __forceinline__ void conv_vec(const R *U, R p, R irho, const R *a, R *F)
{
    R mn = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) mn += U[1 + k] * a[k];
    const R un = mn * irho;
    F[0] = mn;
#pragma unroll
    for (int k = 0; k < D; ++k) F[1 + k] = U[1 + k] * un + p * a[k];
    F[D + 1] = (U[D + 1] + p) * un;
    F[D + 2] = U[D + 2] * un;
}

// HLLC flux along the unit normal nh (hllc_flux with e_dir replaced by nh; FL, FR the
// convective fluxes along nh): the star states keep the tangential velocity,
// U*_K = chi (1, u_K + (S* - u_K.n) n, E/rho + (S* - u_K.n)(S* + p/(rho (S_K - u_K.n))), c/rho).
template <int D, typename R>
__device__ __forceinline__ void hllc_vec(const R *UL, const R *FL, R pL, R aL, R irL, const R *UR, const R *FR, R pR,
                                         R aR, R irR, const R *nh, R *F)
{
    constexpr int NV = D + 3;
    R mL = R(0), mR = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        mL += UL[1 + k] * nh[k];
        mR += UR[1 + k] * nh[k];
    }
    const R rL = UL[0], rR = UR[0], uL = mL * irL, uR = mR * irR;
    const R SL = fmin(uL - aL, uR - aR), SR = fmax(uL + aL, uR + aR);
    if (SL >= R(0) || SR <= R(0)) {
        const bool left = SL >= R(0);
#pragma unroll
        for (int v = 0; v < NV; ++v) F[v] = left ? FL[v] : FR[v];
        return;
    }
    const R Ss = (pR - pL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR));
    const bool left = Ss >= R(0);
    R UK[NV], FK[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        UK[v] = left ? UL[v] : UR[v];
        FK[v] = left ? FL[v] : FR[v];
    }
    const R SK = left ? SL : SR, pK = left ? pL : pR, rK = UK[0], irK = left ? irL : irR, uK = left ? uL : uR;
    const R chi = rK * (SK - uK) / (SK - Ss);
    R Us[NV];
    Us[0] = chi;
#pragma unroll
    for (int k = 0; k < D; ++k) Us[1 + k] = chi * (UK[1 + k] * irK + (Ss - uK) * nh[k]);
    Us[D + 1] = chi * (UK[D + 1] * irK + (Ss - uK) * (Ss + pK * irK / (SK - uK)));
    Us[D + 2] = chi * UK[D + 2] * irK;
#pragma unroll
    for (int v = 0; v < NV; ++v) F[v] = FK[v] + SK * (Us[v] - UK[v]);
}

// Numerical flux along the face metric av of an interior curved face point, from the
// one-sided data of this face (o: U, F = (F^C - F^V).av, lambda, convective pressure,
// sound speed) and of the neighbour (n: the same, F already along av); side 1: this
// element is on the minus side along +xi_dir.  Rusanov, or (FLUX 1) HLLC along the unit
// normal times |av| for the convective part with the central viscous part
// F^V.av = F^C.av - F.av.
template <int D, typename R, int FLUX>
__device__ __forceinline__ void pair_flux_c(bool side, const R *Uo, const R *Fo, R lo, R po, R so, const R *Un,
                                            const R *Fn, R ln, R pn, R sn, const R *av, R *out)
{
    constexpr int NV = D + 3;
    const R *UL = side ? Uo : Un, *UR = side ? Un : Uo, *FL = side ? Fo : Fn, *FR = side ? Fn : Fo;
    if (FLUX == 0) {
        const R lam = fmax(lo, ln);
#pragma unroll
        for (int v = 0; v < NV; ++v) out[v] = R(0.5) * (FL[v] + FR[v]) - R(0.5) * lam * (UR[v] - UL[v]);
        return;
    }
    const R pL = side ? po : pn, pR = side ? pn : po, aL = side ? so : sn, aR = side ? sn : so;
    R a2 = R(0);
#pragma unroll
    for (int k = 0; k < D; ++k) a2 += av[k] * av[k];
    const R sa = sqrt(a2);
    R nh[D];
#pragma unroll
    for (int k = 0; k < D; ++k) nh[k] = av[k] / sa;
    const R irL = R(1) / UL[0], irR = R(1) / UR[0];
    R hL[NV], hR[NV], Fh[NV], CL[NV], CR[NV];
    conv_vec<D, R>(UL, pL, irL, nh, hL);
    conv_vec<D, R>(UR, pR, irR, nh, hR);
    hllc_vec<D, R>(UL, hL, pL, aL, irL, UR, hR, pR, aR, irR, nh, Fh);
    conv_vec<D, R>(UL, pL, irL, av, CL);
    conv_vec<D, R>(UR, pR, irR, av, CR);
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = sa * Fh[v] - R(0.5) * ((CL[v] - FL[v]) + (CR[v] - FR[v]));
}

// mode 0: write U_t (double) to a.v.out; mode 1: RK stage `stage` with coefficients from
// a.v.coef (G = A G + dt U_t; U = U + B G) and new traces.
// FLUX: 0 Rusanov, 1 HLLC (a template parameter, so that each form keeps the register
// allocation of its own flux).  GEO 1: curved elements, whose face data are already
// scaled by the surface element; the surface term takes 1/J of the node (a.v.met) in
// place of 2/h.
template <int D, int N, typename R, int EB = 0, int FLUX = 0, int GEO = 0>
__device__ __forceinline__ void surf_rk_body(const Ctx<R> &a, long long blk, unsigned char *smraw, int mode, int stage)
{
    using S = Shape<D, N, EB>;
    using M = K3Smem<D, N, R, EB>;
    constexpr int P = S::P, NP = S::NP, NFP = S::NFP, NF = S::NF, NV = S::NV;
    constexpr bool SURF_LATE = FLUX == 1 && DGK_SURF_HLLC_LATE;
        const Slot<D, N, EB> t(a.v.g, blk);
    R *sFs = reinterpret_cast<R *>(smraw) + (size_t)t.le * M::per_elem;
    const long long ne = a.v.g.ne;
    // The RK register G is not read at a stage with A = 0 (the first stage of both schemes:
    // G = dt U_t there), nor written at the last stage of a step (the next step's first
    // stage does not read it): 96 B of FP64 traffic per node and step saved.
    // coef = [A_0..A_4, B_0..B_4, dt, number of stages].
    const bool readG = mode != 0 && a.v.coef[stage] != 0.0;
    const bool writeG = mode != 0 && stage + 1 < (int)a.v.coef[11];
    // issue the node loads first so that their latency overlaps the face phase
    R utv[NV];
    double u0[NV], g0[NV];
    R iJ = R(0);  // curved elements: 1/J of the node
    if (t.valid) {
        if (GEO) iJ = a.v.met[((long long)(D * D) * ne + t.e) * NP + t.n];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const long long idx = ((long long)v * ne + t.e) * NP + t.n;
            utv[v] = a.v.Utv[idx];
            if (mode != 0 && !SURF_LATE) {
                u0[v] = a.v.U[idx];
                g0[v] = readG ? a.v.G[idx] : 0.0;
            }
        }
    }
    if (t.valid) {
        const long long st = ne * NF * NFP;
        for (int q = t.n; q < NF * NFP; q += NP) {
            const int f = q / NFP, fp = q % NFP, dir = f >> 1, side = f & 1;
            // curved elements may come with unstructured connectivity (neighbour, its
            // face, face-point orientation); the neighbour's one-sided flux is along its
            // own face metric, of the sign facing_sign relative to this element's
            long long b;
            int fo = 2 * dir + 1 - side, fq = fp;
            long long slot = -1;  // the small side of a mortar: the neighbour's data are in the slot
            if (GEO && a.v.conn) {
                const int *cn = a.v.conn + (t.e * NF + f) * 3;
                b = cn[0] < 0 ? -1 : cn[0];
                fo = cn[1];
                fq = map_fp<P>(cn[2], fp);
                if (cn[0] <= -1000 && cn[1] == 0) {
                    slot = -1000 - cn[0];
                    b = 0;
                }
                // the big side of a mortar holds its complete flux, as a wall does
            } else {
                b = t.nbr(a.v.g, f);
            }
            const long long oo = ((long long)t.e * NF + f) * NFP + fp;
            if (b < 0) {
#pragma unroll
                for (int v = 0; v < NV; ++v) sFs[(f * NV + v) * NFP + fp] = a.v.fd[(NV + v) * st + oo];
            } else if (GEO) {
                // curved elements: the neighbour's one-sided data, at the matching point of
                // its face (its flux signed to this face's orientation) or in the mortar slot
                const R *fN = a.v.fd;
                long long sN = st, iN = ((long long)b * NF + fo) * NFP + fq;
                R sg = R(facing_sign(f, fo));
                if (slot >= 0) {
                    fN = a.v.mfd;
                    sN = a.v.g.nslot * NFP;
                    iN = slot * NFP + fp;
                    sg = R(1);
                }
                R Uo[NV], Fo[NV], Un[NV], Fn[NV], Fs[NV], av[D];
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    Uo[v] = a.v.fd[v * st + oo];
                    Fo[v] = a.v.fd[(NV + v) * st + oo];
                    Un[v] = fN[v * sN + iN];
                    Fn[v] = sg * fN[(NV + v) * sN + iN];
                }
                R po = R(0), so = R(0), pn = R(0), sn = R(0);
                if (FLUX == 1) {
                    po = a.v.fd[(2 * NV + 1) * st + oo];
                    so = a.v.fd[(2 * NV + 2) * st + oo];
                    pn = fN[(2 * NV + 1) * sN + iN];
                    sn = fN[(2 * NV + 2) * sN + iN];
#pragma unroll
                    for (int k = 0; k < D; ++k) av[k] = fat<NF, NFP>(a.v.fmet, ne, k, t.e, f, fp);
                }
                pair_flux_c<D, R, FLUX>(side, Uo, Fo, a.v.fd[(2 * NV) * st + oo], po, so, Un, Fn, fN[(2 * NV) * sN + iN],
                                        pn, sn, av, Fs);
#pragma unroll
                for (int v = 0; v < NV; ++v) sFs[(f * NV + v) * NFP + fp] = Fs[v];
            } else {
                const long long ob = ((long long)b * NF + fo) * NFP + fq;
                const long long iL = side ? oo : ob, iR = side ? ob : oo;
                const R sL = R(1), sR = R(1);
                if (FLUX == 1) {
                    hllc_face<D, R>(a.v.fd, st, iL, iR, dir, sFs + f * NV * NFP + fp, NFP);
                } else {
                    const R lam = fmax(a.v.fd[(2 * NV) * st + iL], a.v.fd[(2 * NV) * st + iR]);
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const R FL = sL * a.v.fd[(NV + v) * st + iL], FR = sR * a.v.fd[(NV + v) * st + iR];
                        const R UL = a.v.fd[v * st + iL], UR = a.v.fd[v * st + iR];
                        sFs[(f * NV + v) * NFP + fp] = R(0.5) * (FL + FR) - R(0.5) * lam * (UR - UL);
                    }
                }
            }
        }
    }
    __syncthreads();
    R Ut[NV];
    if (t.valid) {
        // (2/h) l_i(+-1)/w_i of this node's index in each direction, selected into registers
        // (curved elements: (1/J) l_i(+-1)/w_i)
        R Lp[D], Lm[D];
        int fpd[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int i = ncoord<P>(t.n, d);
            fpd[d] = node_fp<P>(t.n, d);
            R vp = R(0), vm = R(0);
#pragma unroll
            for (int l = 0; l < P; ++l)
                if (l == i) { vp = a.op.Lp[l]; vm = a.op.Lm[l]; }
            Lp[d] = vp * (GEO ? iJ : a.v.gr.inv2h[d]);
            Lm[d] = vm * (GEO ? iJ : a.v.gr.inv2h[d]);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            R acc = utv[v];
#pragma unroll
            for (int d = 0; d < D; ++d)
                acc -= Lp[d] * sFs[((2 * d + 1) * NV + v) * NFP + fpd[d]] - Lm[d] * sFs[((2 * d) * NV + v) * NFP + fpd[d]];
            Ut[v] = acc;
        }
    }
    if (mode == 0) {
        if (t.valid) {
#pragma unroll
            for (int v = 0; v < NV; ++v) a.v.out[((long long)v * ne + t.e) * NP + t.n] = to_f64<R>(Ut[v]);
        }
        return;
    }
    if (SURF_LATE && t.valid) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const long long idx = ((long long)v * ne + t.e) * NP + t.n;
            u0[v] = a.v.U[idx];
            g0[v] = readG ? a.v.G[idx] : 0.0;
        }
    }
    double Ud[NV];
    if (t.valid) {
        // FP64 accumulation: G = A G + dt U_t, U = U + B G (two FP64 FMAs per variable;
        // in the FP32-bulk form dt U_t is formed in float, as U_t itself is)
        const double A = a.v.coef[stage], B = a.v.coef[5 + stage], dt = a.v.coef[10];
        const R dtR = to_bulk<R>(dt);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const long long idx = ((long long)v * ne + t.e) * NP + t.n;
            double gg;
            if constexpr (sizeof(R) == 8) gg = A * g0[v] + dt * Ut[v];
            else gg = fma(A, g0[v], to_f64<R>(dtR * Ut[v]));
            const double uu = fma(B, gg, u0[v]);
            if (writeG) a.v.G[idx] = gg;
            a.v.U[idx] = uu;
            Ud[v] = uu;
        }
    }
    __syncthreads();  // sFs dead; reuse as sQ
    write_traces<D, N, R, EB>(a, t, sFs, Ud);
}

template <int D, int N, typename R, int EB = 0, int FLUX = 0, int GEO = 0>
__global__ void __launch_bounds__(Shape<D, N, EB>::NT,
                                  min_blocks(Shape<D, N, EB>::NT, (FLUX ? DGK_THREADS_SURF_HLLC : DGK_THREADS_SURF) / (int)(sizeof(R) / 4)))
    k_surf_rk(KArgs<R> args, int mode, int stage)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    surf_rk_body<D, N, R, EB, FLUX, GEO>(a, blockIdx.x, smraw, mode, stage);
}

// ------------------------------------------------------------------ set-up kernels

// pass-1 traces of the current state
template <int D, int N, typename R, int EB = 0>
__device__ __forceinline__ void traces_body(const Ctx<R> &a, long long blk, unsigned char *smraw)
{
    using S = Shape<D, N, EB>;
    constexpr int NP = S::NP, NV = S::NV;
        const Slot<D, N, EB> t(a.v.g, blk);
    R *sQ = reinterpret_cast<R *>(smraw) + (size_t)t.le * (size_t)S::NL * NP;
    double Ud[NV];
    if (t.valid) {
#pragma unroll
        for (int v = 0; v < NV; ++v) Ud[v] = a.v.U[((long long)v * a.v.g.ne + t.e) * NP + t.n];
    }
    write_traces<D, N, R, EB>(a, t, sQ, Ud);
}

template <int D, int N, typename R, int EB = 0>
__global__ void __launch_bounds__(Shape<D, N, EB>::NT) k_traces(KArgs<R> args)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    traces_body<D, N, R, EB>(a, blockIdx.x, smraw);
}

// mode 0: nodal temperature into a.v.out[ne][NP]; mode 1: set rho e from the temperature in
// a.v.out (dgk_set_primitive): rho e = rho (R cv T - a rho) + |m|^2/(2 rho)
// + alpha/2 (rho - c)^2 + gamma_K/2 |grad c|^2, grad c lifted from the current traces.
template <int D, int N, typename R, int EB = 0>
__device__ __forceinline__ void node_T_body(const Ctx<R> &a, long long blk, unsigned char *smraw, int mode)
{
    using S = Shape<D, N, EB>;
    using L = CLift<D, N, R, EB>;
    constexpr int NP = S::NP, NF = S::NF, NFP = S::NFP, NV = S::NV;
        const Slot<D, N, EB> t(a.v.g, blk);
    R *sC = reinterpret_cast<R *>(smraw) + (size_t)t.le * L::smem_per_elem;
    R *sCs = sC + NP, *sDc = sCs + NF * NFP;
    double Ud[NV];
    NodeState<D, R> q;
    if (t.valid) {
#pragma unroll
        for (int v = 0; v < NV; ++v) Ud[v] = a.v.U[((long long)v * a.v.g.ne + t.e) * NP + t.n];
        q.from_double(Ud);
    }
    L::run(a, t, q.c, sC, sCs, sDc, false);
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

template <int D, int N, typename R, int EB = 0>
__global__ void __launch_bounds__(Shape<D, N, EB>::NT) k_node_T(KArgs<R> args, int mode)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    const Ctx<R> a{args.v, args.ph, args.pr, args.op};
    node_T_body<D, N, R, EB>(a, blockIdx.x, smraw, mode);
}

}  // namespace dgk
