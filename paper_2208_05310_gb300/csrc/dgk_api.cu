// dgk_api.cu -- host runtime and C ABI of libdgk (declared in include/dgk.h).
//
// The context owns every device buffer of one problem: the FP64 state U and RK register
// G, the bulk-type volume residual and face traces, a small coefficient block read by
// the RK kernel (so one captured graph serves every dt), and the device status word.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dgk.h"
#include "dgk_host_math.h"
#include "dgk_curved.cuh"
#include "dgk_launch.cuh"

const dgk::KernelTable *dgk_table_2d_f64(int N);
const dgk::KernelTable *dgk_table_2d_f32(int N);
const dgk::KernelTable *dgk_table_3d_f64(int N);
const dgk::KernelTable *dgk_table_3d_f32(int N);
const dgk::CurvedTable *dgk_ctable_2d_f64(int N);
const dgk::CurvedTable *dgk_ctable_2d_f32(int N);
const dgk::CurvedTable *dgk_ctable_3d_f64(int N);
const dgk::CurvedTable *dgk_ctable_3d_f32(int N);


namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

#define DGK_CUDA(call)                                                                             \
    do {                                                                                           \
        cudaError_t err_ = (call);                                                                 \
        if (err_ != cudaSuccess)                                                                   \
            return fail(err_ == cudaErrorMemoryAllocation ? DGK_ERR_NOMEM : DGK_ERR_CUDA,           \
                        std::string(#call) + ": " + cudaGetErrorString(err_));                     \
    } while (0)

// LSRK coefficients (Sec. 3.1): Williamson's 3-stage and Carpenter-Kennedy's 5-stage
// fourth-order 2N-storage schemes.
void rk_table(int rk, int &ns, double *A, double *B)
{
    if (rk == 3) {
        static const double a[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
        static const double b[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
        ns = 3;
        for (int s = 0; s < 3; ++s) { A[s] = a[s]; B[s] = b[s]; }
    } else {
        static const double a[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                                    -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
        static const double b[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                                    1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                                    2277821191437.0 / 14882151754819.0};
        ns = 5;
        for (int s = 0; s < 5; ++s) { A[s] = a[s]; B[s] = b[s]; }
    }
}

// primitive (rho, u, T, c) -> partial conserved state; T kept in Tbuf for the energy kernel
// (original NSK model: the c slot holds rho)
__global__ void k_prim_partial(const double *prim, double *U, double *Tbuf, long long nn, int D, int model)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const double rho = prim[i];
    U[i] = rho;
    for (int k = 0; k < D; ++k) U[(1 + k) * nn + i] = rho * prim[(1 + k) * nn + i];
    U[(D + 1) * nn + i] = 0.0;
    U[(D + 2) * nn + i] = model == 0 ? rho : prim[(D + 2) * nn + i];
    Tbuf[i] = prim[(D + 1) * nn + i];
}

struct NodeInfo {
    int D, P, NP;
    double h[3];
    double J;
    double w[dgk::kMaxP];
    const double *met;  // curved elements: [D*D+1][ne][NP] J a^i_k and 1/J in double; box: null
};

// Largest stable dt contribution per node, reduced with atomicMax on the bit pattern
// of non-negative doubles (monotone for non-negative values).
__global__ void k_dt_reduce(const double *U, const double *T, long long ne, NodeInfo ni, dgk::Phys ph,
                            unsigned long long *lam_max, unsigned long long *nu_max)
{
    __shared__ double sl[256], sn[256];
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = ne * ni.NP;
    double lam = 0.0, nu = 0.0;
    if (i < nn) {
        const double rho = U[i], t = T[i];
        double omb = 1.0 - dgk::kBvdw * rho;
        double s2 = dgk::kRgas * t * (1.0 + 1.0 / ph.cv) / (omb * omb) - 2.0 * dgk::kAvdw * rho;
        double s = ph.model == 0 ? sqrt(fabs(s2)) : (s2 + ph.alpha * rho > 0.0 ? sqrt(s2 + ph.alpha * rho) : 0.0);
        for (int k = 0; k < ni.D; ++k) lam += (fabs(U[(1 + k) * nn + i] / rho) + s) / ni.h[k];
        nu = fmax(4.0 * ph.mu / (3.0 * rho), ph.kap / (rho * dgk::kRgas * ph.cv));
        if (ph.model != 0) nu = fmax(nu, ph.gK * ph.beta);
        if (!isfinite(lam)) lam = INFINITY;
    }
    sl[threadIdx.x] = lam;
    sn[threadIdx.x] = nu;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sl[threadIdx.x] = fmax(sl[threadIdx.x], sl[threadIdx.x + o]);
            sn[threadIdx.x] = fmax(sn[threadIdx.x], sn[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicMax(lam_max, (unsigned long long)__double_as_longlong(sl[0]));
        atomicMax(nu_max, (unsigned long long)__double_as_longlong(sn[0]));
    }
}

// k_dt_reduce on curved elements: the spacing along xi_dir at a node is h_dir = 2J/|J a^dir|
// and the velocity along it u.J a^dir/|J a^dir|, so the node's convective sum is
// sum_dir (|u.J a^dir| + s |J a^dir|)/(2J) and its diffusive factor
// sum_dir (|J a^dir|/(2J))^2 (reduced into ih2_max).
__global__ void k_dt_reduce_c(const double *U, const double *T, long long ne, NodeInfo ni, dgk::Phys ph,
                              unsigned long long *lam_max, unsigned long long *nu_max, unsigned long long *ih2_max)
{
    __shared__ double sl[256], sn[256], sh[256];
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = ne * ni.NP;
    double lam = 0.0, nu = 0.0, ih2 = 0.0;
    if (i < nn) {
        const double rho = U[i], t = T[i];
        double omb = 1.0 - dgk::kBvdw * rho;
        double s2 = dgk::kRgas * t * (1.0 + 1.0 / ph.cv) / (omb * omb) - 2.0 * dgk::kAvdw * rho;
        double s = ph.model == 0 ? sqrt(fabs(s2)) : (s2 + ph.alpha * rho > 0.0 ? sqrt(s2 + ph.alpha * rho) : 0.0);
        const double half_iJ = 0.5 * ni.met[(long long)(ni.D * ni.D) * nn + i];
        for (int d = 0; d < ni.D; ++d) {
            double un = 0.0, a2 = 0.0;
            for (int k = 0; k < ni.D; ++k) {
                const double a = ni.met[(long long)(d * ni.D + k) * nn + i];
                un += U[(1 + k) * nn + i] / rho * a;
                a2 += a * a;
            }
            lam += (fabs(un) + s * sqrt(a2)) * half_iJ;
            ih2 += a2 * half_iJ * half_iJ;
        }
        nu = fmax(4.0 * ph.mu / (3.0 * rho), ph.kap / (rho * dgk::kRgas * ph.cv));
        if (ph.model != 0) nu = fmax(nu, ph.gK * ph.beta);
        if (!isfinite(lam)) lam = INFINITY;
    }
    sl[threadIdx.x] = lam;
    sn[threadIdx.x] = nu;
    sh[threadIdx.x] = ih2;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sl[threadIdx.x] = fmax(sl[threadIdx.x], sl[threadIdx.x + o]);
            sn[threadIdx.x] = fmax(sn[threadIdx.x], sn[threadIdx.x + o]);
            sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        atomicMax(lam_max, (unsigned long long)__double_as_longlong(sl[0]));
        atomicMax(nu_max, (unsigned long long)__double_as_longlong(sn[0]));
        atomicMax(ih2_max, (unsigned long long)__double_as_longlong(sh[0]));
    }
}

// Per-block partial sums of the integral diagnostics (fixed tree order), reduced over the
// blocks by k_diag_final in a fixed order, so that the result is deterministic.  Pi: the
// nodal rate of entropy production (k_entropy_prod).
constexpr int kNDiag = DGK_NDIAG;
__global__ void k_diag_partial(const double *U, const double *T, const double *Pi, long long ne, NodeInfo ni,
                               dgk::Phys ph, double *partial)
{
    __shared__ double s[kNDiag][256];
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = ne * ni.NP;
    double q[kNDiag];
    for (int k = 0; k < kNDiag; ++k) q[k] = 0.0;
    if (i < nn) {
        const int n = (int)(i % ni.NP);
        double W = ni.met ? 1.0 / ni.met[(long long)(ni.D * ni.D) * nn + i] : ni.J;
        int r = n;
        for (int k = 0; k < ni.D; ++k) { W *= ni.w[r % ni.P]; r /= ni.P; }
        const double rho = U[i], t = T[i];
        q[0] = W * rho;
        double u2 = 0.0;
        for (int k = 0; k < ni.D; ++k) {
            double mk = U[(1 + k) * nn + i];
            q[1 + k] = W * mk;
            u2 += (mk / rho) * (mk / rho);
        }
        q[4] = W * U[(ni.D + 1) * nn + i];
        // -rho eta = -(rho R cv ln T - rho R ln(b rho / (1 - b rho)))
        q[5] = -W * (rho * dgk::kRgas * ph.cv * log(t) - rho * dgk::kRgas * log(dgk::kBvdw * rho / (1.0 - dgk::kBvdw * rho)));
        double dc = rho - U[(ni.D + 2) * nn + i];
        q[6] = ph.model != 0 ? W * dc * dc : 0.0;
        q[7] = sqrt(u2);
        q[8] = W * Pi[i];
    }
    for (int k = 0; k < kNDiag; ++k) s[k][threadIdx.x] = q[k];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            for (int k = 0; k < kNDiag; ++k)
                s[k][threadIdx.x] = k == 7 ? fmax(s[k][threadIdx.x], s[k][threadIdx.x + o]) : s[k][threadIdx.x] + s[k][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x < kNDiag) partial[(long long)blockIdx.x * kNDiag + threadIdx.x] = s[threadIdx.x][0];
}

// Sum (max for max|u|) of the nb block partials: thread j takes the fixed block range
// [j nb/256, (j+1) nb/256) in order, then a fixed tree over the 256 threads.  Writes
// out[0..kNDiag) (||rho - c||_2 as the square root of its sum); with a counter, at the
// slot out + kNDiag * (*counter) and then advances the counter (samples of a run).
__global__ void __launch_bounds__(256) k_diag_final(const double *partial, long long nb, double *out, unsigned *counter)
{
    __shared__ double s[kNDiag][256];
    const long long lo = nb * threadIdx.x / 256, hi = nb * (threadIdx.x + 1) / 256;
    double q[kNDiag];
    for (int k = 0; k < kNDiag; ++k) q[k] = 0.0;
    for (long long b = lo; b < hi; ++b)
        for (int k = 0; k < kNDiag; ++k) {
            const double v = partial[b * kNDiag + k];
            q[k] = k == 7 ? fmax(q[k], v) : q[k] + v;
        }
    for (int k = 0; k < kNDiag; ++k) s[k][threadIdx.x] = q[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < kNDiag; ++k)
                s[k][threadIdx.x] = k == 7 ? fmax(s[k][threadIdx.x], s[k][threadIdx.x + o]) : s[k][threadIdx.x] + s[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < kNDiag) {
        double *dst = out + (counter ? (long long)kNDiag * (*counter) : 0);
        dst[threadIdx.x] = threadIdx.x == 6 ? sqrt(s[6][0]) : s[threadIdx.x][0];
    }
    __syncthreads();
    if (counter && threadIdx.x == 0) *counter += 1;
}

// p(rho, T) at the nodes (Eq. pressure), from the nodal temperature in T
__global__ void k_pressure(const double *U, const double *T, double *p, long long nn)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const double rho = U[i];
    p[i] = rho * dgk::kRgas * T[i] / (1.0 - dgk::kBvdw * rho) - dgk::kAvdw * rho * rho;
}

// Bitwise comparison of the integer-arithmetic conversions of dgk_common.cuh with the
// hardware conversions (round to nearest) on normal-range inputs.
__global__ void k_check_conv(const double *x, long long n, unsigned long long *bad)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float hw = __double2float_rn(v);
    const float mine = dgk::d2f(v);
    unsigned long long b = 0;
    const bool hw_normal = isnan(hw) || isinf(hw) || hw == 0.0f || fabsf(hw) >= 1.17549435e-38f;
    if (hw_normal && __float_as_uint(hw) != __float_as_uint(mine) && !(isnan(hw) && isnan(mine))) b |= 1ull;
    const float f = hw;
    const double back = dgk::f2d(f);
    if (fabsf(f) >= 1.17549435e-38f || f == 0.0f || isinf(f)) {
        const double ref = (double)f;
        if (__double_as_longlong(ref) != __double_as_longlong(back)) b |= 2ull;
    }
    if (b) atomicAdd(bad, 1ull);
}

}  // namespace

namespace dgk {
// Lets other translation units of the library set the text dgk_last_error() returns.
void set_last_error(const std::string &msg) { g_last_error = msg; }
}  // namespace dgk

struct dgk_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    dgk_params prm{};
    bool have_params = false;
    dgk_box_mesh mesh{};
    bool have_mesh = false;
    int D = 0, N = 0, P = 0, NP = 0, NFP = 0, NF = 0, NV = 0, NL = 0;
    long long ne = 0;
    dgk::host::Operators1D op1{};
    dgk::KArgs<double> a64{};
    dgk::KArgs<float> a32{};
    const dgk::KernelTable *kt = nullptr;
    size_t rsize = 8;
    double *U = nullptr, *G = nullptr, *Tbuf = nullptr, *coef = nullptr, *rhsbuf = nullptr, *partial = nullptr;
    void *Utv = nullptr, *tr1 = nullptr, *tr2 = nullptr, *fd = nullptr;
    void *Us = nullptr;  // FP32-bulk form: shadow of U in float plus the energy balance
    // curved elements (dgk_mesh_curved): metric terms in the bulk type for the kernels
    // (met, fmet) and in double for the time step and the diagnostics (metd; the same
    // buffer as met in the FP64 form); host copy of the node coordinates
    bool curved = false;
    const dgk::CurvedTable *ct = nullptr;
    void *met = nullptr, *fmet = nullptr;
    double *metd = nullptr;
    int *conn = nullptr;  // unstructured connectivity on the device (mortar faces: slot entries), or null
    // mortars: device table, slots, and the slot buffers of the effective neighbour data
    long long nmort = 0, nslot = 0;
    int *mort = nullptr;
    void *mtr1 = nullptr, *mtr2 = nullptr, *mfd = nullptr, *mrec = nullptr;
    std::vector<double> xnodes;
    unsigned *status = nullptr;
    unsigned long long *redbuf = nullptr;
    // diagnostics: nodal entropy production, block partials, one result, the samples of
    // dgk_run and their counter, and the captured graph of one sample
    double *pibuf = nullptr, *diagout = nullptr, *samples = nullptr;
    unsigned *diag_counter = nullptr;
    size_t samples_cap = 0;
    cudaGraphExec_t diag_graph = nullptr;
    double coef_h[12] = {0};  // A_0..A_4, B_0..B_4, dt, number of stages
    bool coef_valid = false;
    cudaGraphExec_t graph = nullptr;
    // dgk_run_host: three item buffers (item i steps in hbuf[i % 3] while item i+1 is
    // copied in and item i-1 out), a captured step graph per buffer, copy streams and events
    double *hbuf[3] = {nullptr, nullptr, nullptr};
    size_t stage_count = 0;
    cudaGraphExec_t hgraph[3] = {nullptr, nullptr, nullptr};
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_start = nullptr, ev_in_ready[3] = {}, ev_done[3] = {}, ev_out_done[3] = {};
    bool timing = false;
    std::vector<cudaEvent_t> events;
    size_t events_used = 0;
    std::vector<int> event_class;
    double t_ms[3] = {0, 0, 0};
    long long t_cnt[3] = {0, 0, 0};

    const void *args() const { return prm.precision == DGK_PREC_FP32BULK ? (const void *)&a32 : (const void *)&a64; }
};

namespace {

void free_buffers(dgk_ctx *c)
{
    if (c->metd && (void *)c->metd != c->met) cudaFree(c->metd);
    void *ptrs[] = {c->U,  c->G,   c->Tbuf, c->coef, c->rhsbuf, c->partial, c->Utv,
                    c->tr1, c->tr2, c->fd,   c->Us,   c->status, c->redbuf, c->met, c->fmet, c->conn,
                    c->mort, c->mtr1, c->mtr2, c->mfd, c->mrec, c->pibuf, c->diagout, c->samples, c->diag_counter};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    c->U = c->G = c->Tbuf = c->coef = c->rhsbuf = c->partial = nullptr;
    c->Utv = c->tr1 = c->tr2 = c->fd = c->Us = nullptr;
    c->met = c->fmet = nullptr;
    c->metd = nullptr;
    c->conn = nullptr;
    c->mort = nullptr;
    c->mtr1 = c->mtr2 = c->mfd = c->mrec = nullptr;
    c->nmort = c->nslot = 0;
    c->curved = false;
    c->ct = nullptr;
    c->xnodes.clear();
    c->status = nullptr;
    c->redbuf = nullptr;
    c->pibuf = c->diagout = c->samples = nullptr;
    c->diag_counter = nullptr;
    c->samples_cap = 0;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    if (c->diag_graph) cudaGraphExecDestroy(c->diag_graph);
    c->diag_graph = nullptr;
    for (int k = 0; k < 3; ++k) {
        if (c->hgraph[k]) cudaGraphExecDestroy(c->hgraph[k]);
        c->hgraph[k] = nullptr;
        if (c->hbuf[k]) cudaFree(c->hbuf[k]);
        c->hbuf[k] = nullptr;
    }
    c->stage_count = 0;
}

void drop_graph(dgk_ctx *c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    if (c->diag_graph) cudaGraphExecDestroy(c->diag_graph);
    c->diag_graph = nullptr;
    for (int k = 0; k < 3; ++k) {
        if (c->hgraph[k]) cudaGraphExecDestroy(c->hgraph[k]);
        c->hgraph[k] = nullptr;
    }
}

template <typename R>
void fill_args(dgk_ctx *c, dgk::KArgs<R> &a)
{
    a.v.U = c->U;
    a.v.G = c->G;
    a.v.Utv = (R *)c->Utv;
    a.v.Us = sizeof(R) == 4 ? (R *)c->Us : nullptr;
    a.v.tr1 = (R *)c->tr1;
    a.v.tr2 = (R *)c->tr2;
    a.v.fd = (R *)c->fd;
    a.v.met = (const R *)c->met;
    a.v.fmet = (const R *)c->fmet;
    a.v.conn = c->conn;
    a.v.mtr1 = (R *)c->mtr1;
    a.v.mtr2 = (R *)c->mtr2;
    a.v.mfd = (R *)c->mfd;
    a.v.mrec = (R *)c->mrec;
    a.v.mort = c->mort;
    a.v.out = c->Tbuf;
    a.v.coef = c->coef;
    a.v.status = c->status;
}

// constants in the bulk type, derived once on the host
template <typename R>
void fill_bulk(dgk::KArgs<R> &a, const dgk::Geom &g, const dgk::Phys &ph, const dgk::Walls &w, const dgk::Ops &o,
               int flux, int P)
{
    for (int i = 0; i < dgk::kMaxP * dgk::kMaxP; ++i) {
        a.op.Dh[i] = (R)o.Dhat[i];
        a.op.Dm[i] = (R)o.Dm[i];
        for (int h = 0; h < 2; ++h) {
            a.op.Im[h][i] = (R)o.Im[h][i];
            a.op.Pm[h][i] = (R)o.Pm[h][i];
        }
    }
    for (int i = 0; i < dgk::kMaxP; ++i) {
        a.op.Lp[i] = (R)o.Lp[i];
        a.op.Lm[i] = (R)o.Lm[i];
        a.op.lp[i] = (R)o.lp[i];
        a.op.lm[i] = (R)o.lm[i];
    }
    for (int d = 0; d < 3; ++d) a.v.gr.inv2h[d] = (R)g.inv2h[d];
    dgk::fill_pairs(a.op, P);
    dgk::PhysR<R> &p = a.pr;
    p.model = ph.model;
    p.gK = (R)ph.gK;
    p.mu = (R)ph.mu;
    p.kap = (R)ph.kap;
    p.alpha = (R)ph.alpha;
    p.beta = (R)ph.beta;
    p.gKbeta = (R)(ph.gK * ph.beta);
    p.alphabeta = (R)(ph.alpha * ph.beta);
    p.half_alpha = (R)(0.5 * ph.alpha);
    p.half_gK = (R)(0.5 * ph.gK);
    p.two_thirds_mu = (R)(2.0 / 3.0 * ph.mu);
    p.s_coef = (R)(dgk::kRgas * (1.0 + 1.0 / ph.cv));
    p.inv_Rcv = (R)(1.0 / (dgk::kRgas * ph.cv));
    p.half_alpha_p = ph.model == 2 ? (R)(0.5 * ph.alpha) : (R)0;
    p.flux = flux;
    for (int f = 0; f < 6; ++f) {
        a.v.wr.kind[f] = w.kind[f];
        a.v.wr.g1[f] = (R)w.g[f][0];
        a.v.wr.g2[f] = (R)w.g[f][1];
        a.v.wr.g3[f] = (R)w.g[f][2];
        a.v.wr.g1gK[f] = (R)(w.g[f][0] / ph.gK);
        a.v.wr.g1g4[f] = (R)(w.g[f][0] * w.g[f][3]);
        for (int k = 0; k < 3; ++k) a.v.wr.uw[f][k] = (R)w.u[f][k];
        a.v.wr.K[f] = (R)w.K[f];
        a.v.wr.rl[f] = (R)w.rl[f];
        a.v.wr.rv[f] = (R)w.rv[f];
        a.v.wr.Tw[f] = (R)w.Tw[f];
    }
}

// geometry, physics, walls and operators into both argument blocks
int build_consts(dgk_ctx *c)
{
    const dgk_box_mesh &m = c->mesh;
    dgk::Geom g{};
    g.ne = c->ne;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = d < c->D ? m.n[d] : 1;
        g.periodic[d] = d < c->D ? m.periodic[d] : 1;
        g.inv2h[d] = d < c->D ? 2.0 / ((m.hi[d] - m.lo[d]) / m.n[d]) : 0.0;
    }
    g.div0.init((unsigned)g.n[0]);
    g.div1.init((unsigned)g.n[1]);
    g.nslot = c->nslot;
    g.nmort = c->nmort;
    const dgk_params &q = c->prm;
    dgk::Phys ph{q.model, q.gammaK, q.mu, q.kappa, q.cv, q.alpha, q.beta,
                 0.5 * q.alpha, 0.5 * q.gammaK, 1.0 / (dgk::kRgas * q.cv)};
    dgk::Walls w{};
    for (int f = 0; f < 2 * c->D; ++f) {
        int d = f / 2;
        if (m.periodic[d]) continue;
        const dgk_wall &wf = m.wall[f];
        double rv, rl, sig;
        if (!dgk::host::maxwell(wf.T_wall, rv, rl) || !dgk::host::sigma_vl(wf.T_wall, c->prm.gammaK, sig))
            return fail(DGK_ERR_THERMO, "wall temperature has no saturation states (need 0 < T_wall < 1)");
        w.kind[f] = wf.kind;
        for (int k = 0; k < 4; ++k) w.g[f][k] = wf.kind == 2 ? wf.gamma[k] : 0.0;
        for (int k = 0; k < c->D; ++k) w.u[f][k] = wf.kind == 1 ? wf.u_wall[k] : 0.0;
        w.Tw[f] = wf.T_wall;
        w.rv[f] = rv;
        w.rl[f] = rl;
        double dr = rl - rv;
        w.K[f] = -6.0 * sig * std::cos(wf.theta_deg * M_PI / 180.0) / (c->prm.gammaK * dr * dr * dr);
    }
    dgk::Ops o{};
    const int P = c->P;
    for (int i = 0; i < P; ++i) {
        for (int j = 0; j < P; ++j) {
            o.Dhat[i * P + j] = c->op1.Dhat[i * P + j];
            o.Dm[i * P + j] = c->op1.D[i * P + j];
            for (int h = 0; h < 2; ++h) {
                o.Im[h][j * P + i] = c->op1.Im[h][j * P + i];
                o.Pm[h][i * P + j] = c->op1.w[j] / (2.0 * c->op1.w[i]) * c->op1.Im[h][j * P + i];
            }
        }
        o.Lp[i] = c->op1.lp[i] / c->op1.w[i];
        o.Lm[i] = c->op1.lm[i] / c->op1.w[i];
        o.lp[i] = c->op1.lp[i];
        o.lm[i] = c->op1.lm[i];
        o.w[i] = c->op1.w[i];
    }
    c->a64.v.g = c->a32.v.g = g;
    c->a64.ph = c->a32.ph = ph;
    fill_bulk(c->a64, g, ph, w, o, c->prm.flux, c->P);
    fill_bulk(c->a32, g, ph, w, o, c->prm.flux, c->P);
    return DGK_OK;
}

int set_coef(dgk_ctx *c, double dt)
{
    int ns;
    double A[5] = {0}, B[5] = {0};
    rk_table(c->prm.rk, ns, A, B);
    double h[12];
    for (int s = 0; s < 5; ++s) { h[s] = A[s]; h[5 + s] = B[s]; }
    h[10] = dt;
    h[11] = ns;
    if (c->coef_valid && std::memcmp(h, c->coef_h, sizeof(h)) == 0) return DGK_OK;
    std::memcpy(c->coef_h, h, sizeof(h));
    DGK_CUDA(cudaMemcpyAsync(c->coef, c->coef_h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
    c->coef_valid = true;
    return DGK_OK;
}

int nstages(const dgk_ctx *c) { return c->prm.rk == 3 ? 3 : 5; }

int event_pair(dgk_ctx *c, int cls, cudaEvent_t &a, cudaEvent_t &b)
{
    if (c->events_used + 2 > c->events.size()) {
        for (int k = 0; k < 64; ++k) {
            cudaEvent_t e;
            DGK_CUDA(cudaEventCreate(&e));
            c->events.push_back(e);
        }
        c->event_class.resize(c->events.size() / 2, 0);
    }
    a = c->events[c->events_used];
    b = c->events[c->events_used + 1];
    c->event_class[c->events_used / 2] = cls;
    c->events_used += 2;
    return DGK_OK;
}

// stage and set-up kernels of the mesh kind (box or curved elements)
// (meshes with mortars: each stage kernel is followed by the mortar kernel that turns its
// face output into the mortar slots' neighbour data)
cudaError_t run_lift1(const dgk_ctx *c, const void *a)
{
    if (!c->curved) return c->kt->lift1(a, c->stream);
    cudaError_t err = c->ct->lift1(a, c->stream);
    if (err == cudaSuccess && c->nmort) err = c->ct->mortar_traces(a, 1, (int)c->nmort, c->stream);
    return err;
}
cudaError_t run_lift2vol(const dgk_ctx *c, const void *a)
{
    if (!c->curved) return c->kt->lift2vol(a, c->stream);
    cudaError_t err = c->ct->lift2vol(a, c->stream);
    if (err == cudaSuccess && c->nmort) err = c->ct->mortar_flux(a, (int)c->nmort, c->stream);
    return err;
}
cudaError_t run_surf(const dgk_ctx *c, const void *a, int mode, int stage)
{
    if (!c->curved) return c->kt->surf(a, mode, stage, c->stream);
    cudaError_t err = c->ct->surf(a, mode, stage, c->stream);
    if (err == cudaSuccess && c->nmort && mode == 1) err = c->ct->mortar_traces(a, 0, (int)c->nmort, c->stream);
    return err;
}
// new pass-1 traces of the current state (and their mortar slots)
cudaError_t run_traces(const dgk_ctx *c)
{
    cudaError_t err = c->kt->traces(c->args(), c->stream);
    if (err == cudaSuccess && c->curved && c->nmort) err = c->ct->mortar_traces(c->args(), 0, (int)c->nmort, c->stream);
    return err;
}
cudaError_t run_nodeT(const dgk_ctx *c, int mode)
{
    return c->curved ? c->ct->nodeT(c->args(), mode, c->stream) : c->kt->nodeT(c->args(), mode, c->stream);
}

// one full RK step, kernel by kernel (optionally bracketed by timing events)
int launch_step(dgk_ctx *c, bool timed)
{
    const void *a = c->args();
    for (int s = 0; s < nstages(c); ++s) {
        for (int k = 0; k < 3; ++k) {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            if (timed) {
                int rc = event_pair(c, k, e0, e1);
                if (rc) return rc;
                DGK_CUDA(cudaEventRecord(e0, c->stream));
            }
            cudaError_t err = k == 0 ? run_lift1(c, a) : k == 1 ? run_lift2vol(c, a) : run_surf(c, a, 1, s);
            if (err != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("stage kernel launch: ") + cudaGetErrorString(err));
            if (timed) DGK_CUDA(cudaEventRecord(e1, c->stream));
        }
    }
    return DGK_OK;
}

int ready(const dgk_ctx *c)
{
    if (!c) return fail(DGK_ERR_ARG, "null context");
    if (!c->have_params || !c->have_mesh) return fail(DGK_ERR_STATE, "set params and mesh first");
    return DGK_OK;
}

int copy_in(dgk_ctx *c, double *dst, const double *src, size_t count, int on_device)
{
    DGK_CUDA(cudaMemcpyAsync(dst, src, count * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream));
    if (!on_device) DGK_CUDA(cudaStreamSynchronize(c->stream));
    return DGK_OK;
}

int after_state_change(dgk_ctx *c)
{
    size_t nstate = (size_t)c->NV * c->ne * c->NP;
    DGK_CUDA(cudaMemsetAsync(c->G, 0, nstate * sizeof(double), c->stream));
    cudaError_t err = run_traces(c);
    if (err != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("trace kernel: ") + cudaGetErrorString(err));
    return DGK_OK;
}

NodeInfo node_info(const dgk_ctx *c)
{
    NodeInfo ni{};
    ni.D = c->D;
    ni.P = c->P;
    ni.NP = c->NP;
    ni.J = 1.0;
    for (int d = 0; d < c->D; ++d) {
        ni.h[d] = (c->mesh.hi[d] - c->mesh.lo[d]) / c->mesh.n[d];
        ni.J *= 0.5 * ni.h[d];
    }
    for (int i = 0; i < c->P; ++i) ni.w[i] = c->op1.w[i];
    ni.met = c->curved ? c->metd : nullptr;
    return ni;
}

// Buffers of the diagnostics (allocated on first use).
int diag_buffers(dgk_ctx *c)
{
    const long long nn = c->ne * c->NP;
    const long long nb = (nn + 255) / 256;
    if (!c->pibuf) DGK_CUDA(cudaMalloc(&c->pibuf, (size_t)nn * sizeof(double)));
    if (!c->partial) DGK_CUDA(cudaMalloc(&c->partial, (size_t)nb * kNDiag * sizeof(double)));
    if (!c->diagout) DGK_CUDA(cudaMalloc(&c->diagout, kNDiag * sizeof(double)));
    if (!c->diag_counter) DGK_CUDA(cudaMalloc(&c->diag_counter, sizeof(unsigned)));
    return DGK_OK;
}

// The integral diagnostics of the current state, reduced on the device into dst
// (DGK_NDIAG doubles; with a counter at dst + DGK_NDIAG * (*counter), which then
// advances): nodal temperature, the pass-2 traces of the state (k_lift1, which the next
// stage recomputes identically), the nodal rate of entropy production, block partials,
// the fixed-order final sum.  Enqueued on the context's stream; capturable.
int enqueue_diag(dgk_ctx *c, double *dst, unsigned *counter)
{
    cudaError_t err = run_nodeT(c, 0);
    if (err == cudaSuccess) err = run_lift1(c, c->args());
    if (err == cudaSuccess) {
        if (c->prm.precision == DGK_PREC_FP32BULK) {
            dgk::KArgs<float> b = c->a32;
            b.v.out = c->pibuf;
            err = c->curved ? c->ct->entropy_prod(&b, c->stream) : c->kt->entropy_prod(&b, c->stream);
        } else {
            dgk::KArgs<double> b = c->a64;
            b.v.out = c->pibuf;
            err = c->curved ? c->ct->entropy_prod(&b, c->stream) : c->kt->entropy_prod(&b, c->stream);
        }
    }
    if (err != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("diagnostics: ") + cudaGetErrorString(err));
    const long long nn = c->ne * c->NP;
    const long long nb = (nn + 255) / 256;
    k_diag_partial<<<(unsigned)nb, 256, 0, c->stream>>>(c->U, c->Tbuf, c->pibuf, c->ne, node_info(c), c->a64.ph,
                                                        c->partial);
    k_diag_final<<<1, 256, 0, c->stream>>>(c->partial, nb, dst, counter);
    DGK_CUDA(cudaGetLastError());
    return DGK_OK;
}

}  // namespace

extern "C" {

const char *dgk_last_error(void) { return g_last_error.c_str(); }

const char *dgk_status_string(int s)
{
    switch (s) {
    case DGK_OK: return "ok";
    case DGK_ERR_ARG: return "invalid argument";
    case DGK_ERR_CUDA: return "CUDA error";
    case DGK_ERR_NONFINITE: return "non-finite value in the state";
    case DGK_ERR_DOMAIN: return "density outside (0, 1/b) or temperature <= 0";
    case DGK_ERR_STATE: return "call order: missing params, mesh or state";
    case DGK_ERR_UNSUPPORTED: return "dimension / degree / option not supported";
    case DGK_ERR_NOMEM: return "device allocation failed";
    case DGK_ERR_THERMO: return "no saturation states at this temperature";
    case DGK_ERR_TIMEOUT: return "a grid barrier of the batched kernel timed out";
    default: return "unknown status";
    }
}

int dgk_create(dgk_ctx **out, int device, void *cuda_stream)
{
    if (!out) return fail(DGK_ERR_ARG, "null output pointer");
    *out = nullptr;
    int ndev = 0;
    DGK_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(DGK_ERR_ARG, "device index out of range");
    DGK_CUDA(cudaSetDevice(device));
    dgk_ctx *c = new (std::nothrow) dgk_ctx();
    if (!c) return fail(DGK_ERR_NOMEM, "host allocation failed");
    c->device = device;
    if (cuda_stream) {
        c->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t err = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) {
            delete c;
            return fail(DGK_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(err));
        }
        c->own_stream = true;
    }
    *out = c;
    return DGK_OK;
}

void dgk_destroy(dgk_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (c->s_in) cudaStreamSynchronize(c->s_in);
    if (c->s_out) cudaStreamSynchronize(c->s_out);
    free_buffers(c);
    for (cudaEvent_t e : c->events) cudaEventDestroy(e);
    if (c->ev_start) cudaEventDestroy(c->ev_start);
    for (int k = 0; k < 3; ++k)
        for (cudaEvent_t e : {c->ev_in_ready[k], c->ev_done[k], c->ev_out_done[k]})
            if (e) cudaEventDestroy(e);
    if (c->s_in) cudaStreamDestroy(c->s_in);
    if (c->s_out) cudaStreamDestroy(c->s_out);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

static bool has_walls(const dgk_box_mesh &m)
{
    for (int d = 0; d < m.dim; ++d)
        if (!m.periodic[d]) return true;
    return false;
}

int dgk_set_params(dgk_ctx *c, const dgk_params *p)
{
    if (!c || !p) return fail(DGK_ERR_ARG, "null argument");
    if (p->model < 0 || p->model > 2) return fail(DGK_ERR_UNSUPPORTED, "model must be 0, 1 or 2");
    if (p->model == 0 && c->have_mesh && has_walls(c->mesh))
        return fail(DGK_ERR_UNSUPPORTED, "the original NSK model runs on periodic boxes");
    if (p->rk != 3 && p->rk != 4) return fail(DGK_ERR_ARG, "rk must be 3 or 4");
    if (p->precision != DGK_PREC_FP64 && p->precision != DGK_PREC_FP32BULK) return fail(DGK_ERR_ARG, "bad precision");
    if (!(p->gammaK > 0) || !(p->mu >= 0) || !(p->kappa >= 0) || !(p->cv > 0) || !(p->alpha >= 0) || !(p->beta >= 0))
        return fail(DGK_ERR_ARG, "parameters out of range");
    if (p->flux != DGK_FLUX_RUSANOV && p->flux != DGK_FLUX_HLLC) return fail(DGK_ERR_ARG, "flux must be Rusanov or HLLC");
    if (p->flux == DGK_FLUX_HLLC && p->model != 2) return fail(DGK_ERR_UNSUPPORTED, "the HLLC flux is for model 2");
    if (c->have_mesh && p->precision != c->prm.precision)
        return fail(DGK_ERR_STATE, "precision is fixed once the mesh is built");
    c->prm = *p;
    c->have_params = true;
    c->coef_valid = false;
    drop_graph(c);
    if (c->have_mesh) return build_consts(c);
    return DGK_OK;
}

// curved_walls: a wall velocity may have a component along the wall's box axis (it is
// projected on the tangent plane of the curved wall at each point)
static int mesh_box_impl(dgk_ctx *c, const dgk_box_mesh *m, bool curved_walls)
{
    if (!c || !m) return fail(DGK_ERR_ARG, "null argument");
    if (!c->have_params) return fail(DGK_ERR_STATE, "set params before the mesh");
    if (m->dim != 2 && m->dim != 3) return fail(DGK_ERR_UNSUPPORTED, "dim must be 2 or 3");
    if (m->N < 2 || m->N > 5) return fail(DGK_ERR_UNSUPPORTED, "N must be 2..5");
    long long ne = 1;
    for (int d = 0; d < m->dim; ++d) {
        if (m->n[d] < 1 || !(m->hi[d] > m->lo[d])) return fail(DGK_ERR_ARG, "bad element count or extent");
        ne *= m->n[d];
        if (ne >= (1LL << 32)) return fail(DGK_ERR_ARG, "more than 2^32 - 1 elements");
        if (!m->periodic[d]) {
            for (int s = 0; s < 2; ++s) {
                const dgk_wall &w = m->wall[2 * d + s];
                if (w.kind != 1 && w.kind != 2) return fail(DGK_ERR_ARG, "non-periodic direction needs walls on both faces");
                if (w.kind == 2)
                    for (int k = 0; k < 4; ++k)
                        if (!(w.gamma[k] >= 0.0) || !std::isfinite(w.gamma[k]))
                            return fail(DGK_ERR_ARG, "wall parameters gamma_1..gamma_4 must be finite and non-negative");
                for (int k = 0; k < m->dim; ++k)
                    if (!std::isfinite(w.u_wall[k]) || (w.u_wall[k] != 0.0 && (w.kind != 1 || (k == d && !curved_walls))))
                        return fail(DGK_ERR_ARG, "a wall velocity must be finite, tangential and on a no-slip wall");
            }
        }
    }
    if (c->prm.model == 0 && has_walls(*m)) return fail(DGK_ERR_UNSUPPORTED, "the original NSK model runs on periodic boxes");
    {
        // the kernels index inside one plane of a node or face array with 32 bits
        long long ne = 1, P = m->N + 1;
        for (int d = 0; d < m->dim; ++d) ne *= m->n[d];
        const long long np = m->dim == 2 ? P * P : P * P * P, nfq = m->dim == 2 ? 4 * P : 6 * P * P;
        if (ne * (np > nfq ? np : nfq) >= (1LL << 32)) return fail(DGK_ERR_ARG, "more than 2^32 - 1 nodes or face points");
    }
    DGK_CUDA(cudaSetDevice(c->device));
    cudaStreamSynchronize(c->stream);
    free_buffers(c);
    c->have_mesh = false;
    c->mesh = *m;
    c->D = m->dim;
    c->N = m->N;
    c->P = m->N + 1;
    c->NP = c->D == 2 ? c->P * c->P : c->P * c->P * c->P;
    c->NFP = c->D == 2 ? c->P : c->P * c->P;
    c->NF = 2 * c->D;
    c->NV = c->D + 3;
    c->NL = c->D + 2;
    c->ne = ne;
    if (!dgk::host::dg_operators(c->N, c->op1)) return fail(DGK_ERR_ARG, "operator set-up failed");
    const bool f32 = c->prm.precision == DGK_PREC_FP32BULK;
    c->rsize = f32 ? sizeof(float) : sizeof(double);
    c->kt = c->D == 2 ? (f32 ? dgk_table_2d_f32(c->N) : dgk_table_2d_f64(c->N))
                      : (f32 ? dgk_table_3d_f32(c->N) : dgk_table_3d_f64(c->N));
    if (!c->kt) return fail(DGK_ERR_UNSUPPORTED, "no kernels for this (dim, N, precision)");
    int rc = build_consts(c);
    if (rc) return rc;
    DGK_CUDA(c->kt->prepare());
    const size_t nstate = (size_t)c->NV * ne * c->NP;
    const size_t nface = (size_t)ne * c->NF * c->NFP;
    DGK_CUDA(cudaMalloc(&c->U, nstate * sizeof(double)));
    DGK_CUDA(cudaMalloc(&c->G, nstate * sizeof(double)));
    DGK_CUDA(cudaMalloc(&c->Tbuf, (size_t)ne * c->NP * sizeof(double)));
    DGK_CUDA(cudaMalloc(&c->coef, 16 * sizeof(double)));
    DGK_CUDA(cudaMalloc(&c->status, sizeof(unsigned)));
    DGK_CUDA(cudaMalloc(&c->redbuf, 3 * sizeof(unsigned long long)));
    DGK_CUDA(cudaMalloc(&c->Utv, nstate * c->rsize));
    DGK_CUDA(cudaMalloc(&c->tr1, (size_t)c->NL * nface * c->rsize));
    DGK_CUDA(cudaMalloc(&c->tr2, (size_t)2 * nface * c->rsize));
    DGK_CUDA(cudaMalloc(&c->fd, (size_t)(2 * c->NV + 3) * nface * c->rsize));
    if (f32) DGK_CUDA(cudaMalloc(&c->Us, (size_t)(c->NV + 1) * ne * c->NP * sizeof(float)));
    DGK_CUDA(cudaMemsetAsync(c->U, 0, nstate * sizeof(double), c->stream));
    DGK_CUDA(cudaMemsetAsync(c->G, 0, nstate * sizeof(double), c->stream));
    DGK_CUDA(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    DGK_CUDA(cudaMemsetAsync(c->tr1, 0, (size_t)c->NL * nface * c->rsize, c->stream));
    fill_args(c, c->a64);
    fill_args(c, c->a32);
    c->coef_valid = false;
    c->have_mesh = true;
    DGK_CUDA(cudaStreamSynchronize(c->stream));
    return DGK_OK;
}

int dgk_mesh_box(dgk_ctx *c, const dgk_box_mesh *m) { return mesh_box_impl(c, m, false); }

static int mesh_curved_impl(dgk_ctx *c, const dgk_box_mesh *m, int ngeo, const double *xgeo, const int *conn,
                            const int *mortar, int nmortar)
{
    if (!c || !m || !xgeo) return fail(DGK_ERR_ARG, "null argument");
    if (!c->have_params) return fail(DGK_ERR_STATE, "set params before the mesh");
    if (m->dim != 2 && m->dim != 3) return fail(DGK_ERR_UNSUPPORTED, "dim must be 2 or 3");
    if (ngeo < 1 || (m->dim == 2 ? ngeo > m->N : 2 * ngeo > m->N))
        return fail(DGK_ERR_UNSUPPORTED, "curved elements need 1 <= ngeo <= N (2D) or 1 <= 2 ngeo <= N (3D)");
    if (conn) {
        // the tables: neighbours in range and pointing back, orientations of the
        // dimension, walls of the box's wall table
        long long ne = 1;
        for (int d = 0; d < m->dim; ++d) ne *= m->n[d];
        if (ne >= (1LL << 31)) return fail(DGK_ERR_ARG, "unstructured meshes take fewer than 2^31 elements");
        const int NF = 2 * m->dim, nsub = m->dim == 2 ? 2 : 4;
        if (nmortar < 0 || (nmortar > 0 && !mortar)) return fail(DGK_ERR_ARG, "bad mortar table");
        auto o_ok = [&](int o) { return m->dim == 3 ? (o >= 0 && o < 8) : (o == 0 || o == 2); };
        for (long long e = 0; e < ne; ++e)
            for (int f = 0; f < NF; ++f) {
                const int *t = conn + (e * NF + f) * 3;
                if (t[0] <= -100) {  // the big side of mortar -100 - t[0]
                    const long long mm = -100LL - t[0];
                    if (mm >= nmortar) return fail(DGK_ERR_ARG, "a face names a mortar outside the table");
                    for (int p = 0; p < nsub; ++p) {
                        const int *sb = mortar + (mm * nsub + p) * 3;
                        if (sb[0] < 0 || sb[0] >= ne || sb[1] < 0 || sb[1] >= NF || !o_ok(sb[2]))
                            return fail(DGK_ERR_ARG, "mortar entry out of range");
                        const int *back = conn + ((long long)sb[0] * NF + sb[1]) * 3;
                        if (back[0] != e || back[1] != f || back[2] != (sb[2] | ((p + 1) << 3)))
                            return fail(DGK_ERR_ARG, "a mortar's small face does not name the big face back");
                    }
                    continue;
                }
                if (t[0] < 0) {
                    const int w = -1 - t[0];
                    if (w >= NF || m->periodic[w / 2] || (m->wall[w].kind != 1 && m->wall[w].kind != 2))
                        return fail(DGK_ERR_ARG, "a boundary face names no wall of the wall table");
                    continue;
                }
                if (t[0] >= ne || t[1] < 0 || t[1] >= NF) return fail(DGK_ERR_ARG, "connectivity entry out of range");
                const int pos = t[2] >> 3;
                if (pos) {  // the small side of a mortar
                    const int *big = conn + ((long long)t[0] * NF + t[1]) * 3;
                    const long long mm = -100LL - big[0];
                    if (big[0] > -100 || mm >= nmortar || pos > nsub) return fail(DGK_ERR_ARG, "a small face names no mortar");
                    const int *sb = mortar + (mm * nsub + pos - 1) * 3;
                    if (sb[0] != e || sb[1] != f || sb[2] != (t[2] & 7)) return fail(DGK_ERR_ARG, "mortar table mismatch");
                    continue;
                }
                if (!o_ok(t[2])) return fail(DGK_ERR_ARG, "connectivity entry out of range");
                const int *back = conn + ((long long)t[0] * NF + t[1]) * 3;
                if (back[0] != e || back[1] != f) return fail(DGK_ERR_ARG, "connectivity is not symmetric");
            }
    }
    int rc = mesh_box_impl(c, m, true);  // validates the rest and allocates the stage buffers
    if (rc) return rc;
    c->have_mesh = false;
    int n[3], per[3];
    for (int d = 0; d < 3; ++d) {
        n[d] = d < c->D ? m->n[d] : 1;
        per[d] = d < c->D ? m->periodic[d] : 1;
    }
    dgk::host::CurvedGeometry geo;
    std::string err;
    if (!dgk::host::curved_geometry(c->D, c->op1, ngeo, n, per, c->ne, xgeo, conn, geo, err)) return fail(DGK_ERR_ARG, err);
    if (conn) {
        // mortar faces become slot entries (-1000 - slot, 1 on the big side); the device
        // mortar table lists each mortar's faces and slots
        const size_t nc = (size_t)c->ne * c->NF * 3;
        const int nsub = c->D == 2 ? 2 : 4, MT = 4 + 4 * nsub;
        std::vector<int> cn(conn, conn + nc), mt((size_t)nmortar * MT, 0);
        for (long long mm = 0; mm < nmortar; ++mm) {
            const long long base = mm * (1 + nsub);
            long long B = -1;
            int fB = 0;
            for (int p = 0; p < nsub; ++p) {
                const int *sb = mortar + (mm * nsub + p) * 3;
                const int *t = conn + ((long long)sb[0] * c->NF + sb[1]) * 3;
                B = t[0];
                fB = t[1];
                mt[mm * MT + 4 + 4 * p + 0] = sb[0];
                mt[mm * MT + 4 + 4 * p + 1] = sb[1];
                mt[mm * MT + 4 + 4 * p + 2] = sb[2];
                mt[mm * MT + 4 + 4 * p + 3] = (int)(base + 1 + p);
                int *ts = &cn[((size_t)sb[0] * c->NF + sb[1]) * 3];
                ts[0] = (int)(-1000 - (base + 1 + p));
                ts[1] = 0;
                ts[2] = 0;
            }
            mt[mm * MT + 0] = (int)B;
            mt[mm * MT + 1] = fB;
            mt[mm * MT + 2] = (int)base;
            int *tb = &cn[((size_t)B * c->NF + fB) * 3];
            tb[0] = (int)(-1000 - base);
            tb[1] = 1;
            tb[2] = 0;
        }
        DGK_CUDA(cudaMalloc(&c->conn, nc * sizeof(int)));
        DGK_CUDA(cudaMemcpy(c->conn, cn.data(), nc * sizeof(int), cudaMemcpyHostToDevice));
        if (nmortar > 0) {
            c->nmort = nmortar;
            c->nslot = (long long)nmortar * (1 + nsub);
            const size_t sl = (size_t)c->nslot * c->NFP * c->rsize;
            const int NQ = c->NV + c->D * c->D + 2 * c->D + 1;
            DGK_CUDA(cudaMalloc(&c->mort, mt.size() * sizeof(int)));
            DGK_CUDA(cudaMemcpy(c->mort, mt.data(), mt.size() * sizeof(int), cudaMemcpyHostToDevice));
            DGK_CUDA(cudaMalloc(&c->mtr1, c->NL * sl));
            DGK_CUDA(cudaMalloc(&c->mtr2, 2 * sl));
            DGK_CUDA(cudaMalloc(&c->mfd, (2 * c->NV + 3) * sl));
            DGK_CUDA(cudaMalloc(&c->mrec, NQ * sl));
            rc = build_consts(c);
            if (rc) return rc;
        }
    }
    const bool f32 = c->prm.precision == DGK_PREC_FP32BULK;
    c->ct = c->D == 2 ? (f32 ? dgk_ctable_2d_f32(c->N) : dgk_ctable_2d_f64(c->N))
                      : (f32 ? dgk_ctable_3d_f32(c->N) : dgk_ctable_3d_f64(c->N));
    if (!c->ct) return fail(DGK_ERR_UNSUPPORTED, "no curved-element kernels for this (dim, N, precision)");
    DGK_CUDA(c->ct->prepare());
    DGK_CUDA(cudaMalloc(&c->metd, geo.met.size() * sizeof(double)));
    DGK_CUDA(cudaMemcpy(c->metd, geo.met.data(), geo.met.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (f32) {
        std::vector<float> h(geo.met.begin(), geo.met.end());
        DGK_CUDA(cudaMalloc(&c->met, h.size() * sizeof(float)));
        DGK_CUDA(cudaMemcpy(c->met, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice));
        std::vector<float> hf(geo.fmet.begin(), geo.fmet.end());
        DGK_CUDA(cudaMalloc(&c->fmet, hf.size() * sizeof(float)));
        DGK_CUDA(cudaMemcpy(c->fmet, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice));
    } else {
        c->met = c->metd;
        DGK_CUDA(cudaMalloc(&c->fmet, geo.fmet.size() * sizeof(double)));
        DGK_CUDA(cudaMemcpy(c->fmet, geo.fmet.data(), geo.fmet.size() * sizeof(double), cudaMemcpyHostToDevice));
    }
    c->xnodes = std::move(geo.x);
    c->curved = true;
    fill_args(c, c->a64);
    fill_args(c, c->a32);
    drop_graph(c);
    c->coef_valid = false;
    c->have_mesh = true;
    return DGK_OK;
}

int dgk_mesh_curved(dgk_ctx *c, const dgk_box_mesh *m, int ngeo, const double *xgeo)
{
    return mesh_curved_impl(c, m, ngeo, xgeo, nullptr, nullptr, 0);
}

int dgk_mesh_unstructured(dgk_ctx *c, const dgk_box_mesh *m, int ngeo, const double *xgeo, const int *conn,
                          const int *mortar, int nmortar)
{
    if (!conn) return fail(DGK_ERR_ARG, "null connectivity");
    return mesh_curved_impl(c, m, ngeo, xgeo, conn, mortar, nmortar);
}

int dgk_sizes(const dgk_ctx *c, long long *nelem, int *np, int *nv)
{
    int rc = ready(c);
    if (rc) return rc;
    if (nelem) *nelem = c->ne;
    if (np) *np = c->NP;
    if (nv) *nv = c->NV;
    return DGK_OK;
}

int dgk_node_coords(dgk_ctx *c, double *x, int on_device)
{
    int rc = ready(c);
    if (rc) return rc;
    if (!x) return fail(DGK_ERR_ARG, "null output");
    const size_t nn = (size_t)c->ne * c->NP;
    std::vector<double> h((size_t)c->D * nn);
    if (c->curved) {
        h = c->xnodes;
    } else {
        for (long long e = 0; e < c->ne; ++e) {
            long long co[3] = {e % c->mesh.n[0], (e / c->mesh.n[0]) % c->mesh.n[1],
                               c->D == 3 ? e / ((long long)c->mesh.n[0] * c->mesh.n[1]) : 0};
            for (int n = 0; n < c->NP; ++n) {
                int r = n;
                for (int d = 0; d < c->D; ++d) {
                    const int i = r % c->P;
                    r /= c->P;
                    const double hd = (c->mesh.hi[d] - c->mesh.lo[d]) / c->mesh.n[d];
                    h[(size_t)d * nn + (size_t)e * c->NP + n] = c->mesh.lo[d] + hd * (co[d] + 0.5 * (c->op1.xi[i] + 1.0));
                }
            }
        }
    }
    DGK_CUDA(cudaMemcpyAsync(x, h.data(), h.size() * sizeof(double), on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                             c->stream));
    DGK_CUDA(cudaStreamSynchronize(c->stream));
    return DGK_OK;
}

int dgk_set_primitive(dgk_ctx *c, const double *prim, size_t count, int on_device)
{
    int rc = ready(c);
    if (rc) return rc;
    const size_t nstate = (size_t)c->NV * c->ne * c->NP;
    if (!prim || count != nstate) return fail(DGK_ERR_ARG, "primitive array has the wrong size");
    // stage the primitives in G (reset afterwards)
    rc = copy_in(c, c->G, prim, count, on_device);
    if (rc) return rc;
    const long long nn = c->ne * c->NP;
    k_prim_partial<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(c->G, c->U, c->Tbuf, nn, c->D, c->prm.model);
    DGK_CUDA(cudaGetLastError());
    cudaError_t err = run_traces(c);
    if (err != cudaSuccess) return fail(DGK_ERR_CUDA, cudaGetErrorString(err));
    err = run_nodeT(c, 1);
    if (err != cudaSuccess) return fail(DGK_ERR_CUDA, cudaGetErrorString(err));
    rc = after_state_change(c);
    if (rc) return rc;
    DGK_CUDA(cudaStreamSynchronize(c->stream));
    return DGK_OK;
}

int dgk_upload_state(dgk_ctx *c, const double *U, size_t count, int on_device)
{
    int rc = ready(c);
    if (rc) return rc;
    const size_t nstate = (size_t)c->NV * c->ne * c->NP;
    if (!U || count != nstate) return fail(DGK_ERR_ARG, "state array has the wrong size");
    rc = copy_in(c, c->U, U, count, on_device);
    if (rc) return rc;
    return after_state_change(c);
}

int dgk_download_state(dgk_ctx *c, double *U, size_t count, int on_device)
{
    int rc = ready(c);
    if (rc) return rc;
    const size_t nstate = (size_t)c->NV * c->ne * c->NP;
    if (!U || count != nstate) return fail(DGK_ERR_ARG, "state array has the wrong size");
    DGK_CUDA(cudaMemcpyAsync(U, c->U, count * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
    if (!on_device) DGK_CUDA(cudaStreamSynchronize(c->stream));
    return DGK_OK;
}

int dgk_rhs(dgk_ctx *c, double *Ut, size_t count, int on_device)
{
    int rc = ready(c);
    if (rc) return rc;
    const size_t nstate = (size_t)c->NV * c->ne * c->NP;
    if (!Ut || count != nstate) return fail(DGK_ERR_ARG, "output array has the wrong size");
    double *dst = Ut;
    if (!on_device) {
        if (!c->rhsbuf) DGK_CUDA(cudaMalloc(&c->rhsbuf, nstate * sizeof(double)));
        dst = c->rhsbuf;
    }
    cudaError_t err;
    const void *a = c->args();
    if ((err = run_lift1(c, a))) return fail(DGK_ERR_CUDA, cudaGetErrorString(err));
    if ((err = run_lift2vol(c, a))) return fail(DGK_ERR_CUDA, cudaGetErrorString(err));
    if (c->prm.precision == DGK_PREC_FP32BULK) {
        dgk::KArgs<float> b = c->a32;
        b.v.out = dst;
        err = run_surf(c, &b, 0, 0);
    } else {
        dgk::KArgs<double> b = c->a64;
        b.v.out = dst;
        err = run_surf(c, &b, 0, 0);
    }
    if (err) return fail(DGK_ERR_CUDA, cudaGetErrorString(err));
    if (!on_device) {
        DGK_CUDA(cudaMemcpyAsync(Ut, dst, nstate * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        DGK_CUDA(cudaStreamSynchronize(c->stream));
    }
    return DGK_OK;
}

int dgk_rk_step(dgk_ctx *c, double dt)
{
    int rc = ready(c);
    if (rc) return rc;
    if (!(dt > 0) || !std::isfinite(dt)) return fail(DGK_ERR_ARG, "dt must be positive");
    if ((rc = set_coef(c, dt))) return rc;
    return launch_step(c, c->timing);
}

int dgk_run(dgk_ctx *c, int nsteps, double dt, int diag_every, double *diag_out)
{
    int rc = ready(c);
    if (rc) return rc;
    if (nsteps < 0) return fail(DGK_ERR_ARG, "nsteps < 0");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(DGK_ERR_ARG, "dt must be positive");
    if (diag_every < 0) return fail(DGK_ERR_ARG, "diag_every < 0");
    if ((rc = set_coef(c, dt))) return rc;
    const int nsamp = (diag_every > 0 && diag_out) ? nsteps / diag_every : 0;
    if (nsamp > 0) {
        if ((rc = diag_buffers(c))) return rc;
        const size_t need = (size_t)nsamp * kNDiag;
        if (need > c->samples_cap) {
            if (c->diag_graph) cudaGraphExecDestroy(c->diag_graph);
            c->diag_graph = nullptr;
            if (c->samples) cudaFree(c->samples);
            c->samples = nullptr;
            c->samples_cap = 0;
            DGK_CUDA(cudaMalloc(&c->samples, need * sizeof(double)));
            c->samples_cap = need;
        }
        DGK_CUDA(cudaMemsetAsync(c->diag_counter, 0, sizeof(unsigned), c->stream));
    }
    if (c->timing) {
        for (int s = 0; s < nsteps; ++s) {
            if ((rc = launch_step(c, true))) return rc;
            if (nsamp > 0 && (s + 1) % diag_every == 0 && (s + 1) / diag_every <= nsamp &&
                (rc = enqueue_diag(c, c->samples, c->diag_counter)))
                return rc;
        }
    } else {
        if (!c->graph && nsteps > 0) {
            cudaGraph_t g;
            DGK_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            rc = launch_step(c, false);
            cudaError_t err = cudaStreamEndCapture(c->stream, &g);
            if (rc) return rc;
            if (err != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(err));
            err = cudaGraphInstantiate(&c->graph, g, 0);
            cudaGraphDestroy(g);
            if (err != cudaSuccess) {
                c->graph = nullptr;
                return fail(DGK_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(err));
            }
        }
        if (nsamp > 0 && !c->diag_graph) {
            cudaGraph_t g;
            DGK_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
            rc = enqueue_diag(c, c->samples, c->diag_counter);
            cudaError_t err = cudaStreamEndCapture(c->stream, &g);
            if (rc) return rc;
            if (err != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("diagnostics capture: ") + cudaGetErrorString(err));
            err = cudaGraphInstantiate(&c->diag_graph, g, 0);
            cudaGraphDestroy(g);
            if (err != cudaSuccess) {
                c->diag_graph = nullptr;
                return fail(DGK_ERR_CUDA, std::string("diagnostics instantiate: ") + cudaGetErrorString(err));
            }
        }
        for (int s = 0; s < nsteps; ++s) {
            DGK_CUDA(cudaGraphLaunch(c->graph, c->stream));
            if (nsamp > 0 && (s + 1) % diag_every == 0 && (s + 1) / diag_every <= nsamp)
                DGK_CUDA(cudaGraphLaunch(c->diag_graph, c->stream));
        }
    }
    if (nsamp > 0) {
        DGK_CUDA(cudaMemcpyAsync(diag_out, c->samples, (size_t)nsamp * kNDiag * sizeof(double), cudaMemcpyDefault,
                                 c->stream));
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, diag_out) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            DGK_CUDA(cudaStreamSynchronize(c->stream));
        }
    }
    return DGK_OK;
}

// the state array the kernels of both argument blocks work on
static void set_state_ptr(dgk_ctx *c, double *U)
{
    c->a64.v.U = U;
    c->a32.v.U = U;
}

int dgk_run_host(dgk_ctx *c, const double *const *in, double *const *out, int nitems, size_t count, int nsteps,
                 double dt)
{
    int rc = ready(c);
    if (rc) return rc;
    const size_t nstate = (size_t)c->NV * c->ne * c->NP;
    if (!in || !out || nitems < 0 || count != nstate) return fail(DGK_ERR_ARG, "bad arrays, count or nitems");
    if (nsteps < 0 || !(dt > 0) || !std::isfinite(dt)) return fail(DGK_ERR_ARG, "nsteps < 0 or dt not positive");
    for (int i = 0; i < nitems; ++i)
        if (!in[i] || !out[i]) return fail(DGK_ERR_ARG, "null host pointer");
    if (nitems == 0) return DGK_OK;
    DGK_CUDA(cudaSetDevice(c->device));
    if ((rc = set_coef(c, dt))) return rc;
    if (c->stage_count != nstate) {
        for (int k = 0; k < 3; ++k) {
            if (c->hgraph[k]) cudaGraphExecDestroy(c->hgraph[k]);
            c->hgraph[k] = nullptr;
            if (c->hbuf[k]) cudaFree(c->hbuf[k]);
            c->hbuf[k] = nullptr;
        }
        c->stage_count = 0;
        for (int k = 0; k < 3; ++k) DGK_CUDA(cudaMalloc(&c->hbuf[k], nstate * sizeof(double)));
        c->stage_count = nstate;
    }
    for (cudaStream_t *st : {&c->s_in, &c->s_out})
        if (!*st) DGK_CUDA(cudaStreamCreateWithFlags(st, cudaStreamNonBlocking));
    if (!c->ev_start) DGK_CUDA(cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming));
    for (int k = 0; k < 3; ++k)
        for (cudaEvent_t *e : {&c->ev_in_ready[k], &c->ev_done[k], &c->ev_out_done[k]})
            if (!*e) DGK_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    const size_t bytes = nstate * sizeof(double);
    const int nbuf = nitems < 3 ? nitems : 3;
    // one captured step graph per item buffer (the arrays are kernel parameters)
    if (nsteps > 0 && !c->timing) {
        for (int k = 0; k < nbuf; ++k) {
            if (c->hgraph[k]) continue;
            set_state_ptr(c, c->hbuf[k]);
            cudaGraph_t g;
            cudaError_t err = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (err == cudaSuccess) {
                rc = launch_step(c, false);
                err = cudaStreamEndCapture(c->stream, &g);
            }
            set_state_ptr(c, c->U);
            if (rc) return rc;
            if (err != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(err));
            err = cudaGraphInstantiate(&c->hgraph[k], g, 0);
            cudaGraphDestroy(g);
            if (err != cudaSuccess) {
                c->hgraph[k] = nullptr;
                return fail(DGK_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(err));
            }
        }
    }
    // The pipeline: item i steps in buffer i % 3 on the context's stream while item i+1 is
    // copied in on s_in and item i-1 out on s_out; a buffer takes a new item once its
    // previous item has left it.  No device-to-device copies: the step graphs work on the
    // buffers themselves.  On an error it stops enqueueing; the streams are drained below
    // so that no copy touches the caller's buffers after the return.
    auto pipeline = [&]() -> int {
        DGK_CUDA(cudaEventRecord(c->ev_start, c->stream));  // after the work already queued
        DGK_CUDA(cudaStreamWaitEvent(c->s_in, c->ev_start, 0));
        DGK_CUDA(cudaStreamWaitEvent(c->s_out, c->ev_start, 0));
        DGK_CUDA(cudaMemcpyAsync(c->hbuf[0], in[0], bytes, cudaMemcpyHostToDevice, c->s_in));
        DGK_CUDA(cudaEventRecord(c->ev_in_ready[0], c->s_in));
        for (int i = 0; i < nitems; ++i) {
            const int b = i % 3;
            if (i + 1 < nitems) {
                const int nb = (i + 1) % 3;
                if (i + 1 >= 3) DGK_CUDA(cudaStreamWaitEvent(c->s_in, c->ev_out_done[nb], 0));
                DGK_CUDA(cudaMemcpyAsync(c->hbuf[nb], in[i + 1], bytes, cudaMemcpyHostToDevice, c->s_in));
                DGK_CUDA(cudaEventRecord(c->ev_in_ready[nb], c->s_in));
            }
            DGK_CUDA(cudaStreamWaitEvent(c->stream, c->ev_in_ready[b], 0));
            set_state_ptr(c, c->hbuf[b]);
            // the new state's traces (as dgk_upload_state; the first RK stage of both
            // schemes does not read the RK register, so it needs no reset)
            cudaError_t err = run_traces(c);
            if (err != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("trace kernel: ") + cudaGetErrorString(err));
            for (int st = 0; st < nsteps; ++st) {
                if (c->timing) {
                    int r = launch_step(c, true);
                    if (r) return r;
                } else {
                    DGK_CUDA(cudaGraphLaunch(c->hgraph[b], c->stream));
                }
            }
            DGK_CUDA(cudaEventRecord(c->ev_done[b], c->stream));
            DGK_CUDA(cudaStreamWaitEvent(c->s_out, c->ev_done[b], 0));
            DGK_CUDA(cudaMemcpyAsync(out[i], c->hbuf[b], bytes, cudaMemcpyDeviceToHost, c->s_out));
            DGK_CUDA(cudaEventRecord(c->ev_out_done[b], c->s_out));
        }
        // the context keeps the last item's state
        DGK_CUDA(cudaMemcpyAsync(c->U, c->hbuf[(nitems - 1) % 3], bytes, cudaMemcpyDeviceToDevice, c->stream));
        return DGK_OK;
    };
    rc = pipeline();
    set_state_ptr(c, c->U);
    const cudaError_t e1 = cudaStreamSynchronize(c->s_in), e2 = cudaStreamSynchronize(c->s_out),
                      e3 = cudaStreamSynchronize(c->stream);
    if (rc) return rc;
    for (cudaError_t e : {e1, e2, e3})
        if (e != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("dgk_run_host: ") + cudaGetErrorString(e));
    return DGK_OK;
}

int dgk_max_dt(dgk_ctx *c, double cfl, double dfl, double *dt)
{
    int rc = ready(c);
    if (rc) return rc;
    if (!dt || !(cfl > 0) || !(dfl > 0)) return fail(DGK_ERR_ARG, "bad arguments");
    cudaError_t err = run_nodeT(c, 0);
    if (err) return fail(DGK_ERR_CUDA, cudaGetErrorString(err));
    DGK_CUDA(cudaMemsetAsync(c->redbuf, 0, 3 * sizeof(unsigned long long), c->stream));
    const long long nn = c->ne * c->NP;
    dgk::Phys ph = c->a64.ph;
    if (c->curved)
        k_dt_reduce_c<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(c->U, c->Tbuf, c->ne, node_info(c), ph, c->redbuf,
                                                                           c->redbuf + 1, c->redbuf + 2);
    else
        k_dt_reduce<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(c->U, c->Tbuf, c->ne, node_info(c), ph, c->redbuf,
                                                                         c->redbuf + 1);
    DGK_CUDA(cudaGetLastError());
    unsigned long long hv[3];
    DGK_CUDA(cudaMemcpyAsync(hv, c->redbuf, sizeof(hv), cudaMemcpyDeviceToHost, c->stream));
    DGK_CUDA(cudaStreamSynchronize(c->stream));
    double lam, nu, ih2 = 0.0;
    std::memcpy(&lam, &hv[0], 8);
    std::memcpy(&nu, &hv[1], 8);
    if (c->curved) {
        std::memcpy(&ih2, &hv[2], 8);
    } else {
        for (int d = 0; d < c->D; ++d) {
            double h = (c->mesh.hi[d] - c->mesh.lo[d]) / c->mesh.n[d];
            ih2 += 1.0 / (h * h);
        }
    }
    const double k1 = 2.0 * c->N + 1.0;
    double r = cfl / (k1 * lam);
    if (nu > 0) r = std::fmin(r, dfl / (k1 * k1 * nu * ih2));
    if (c->prm.model != 0 && c->prm.alpha * c->prm.beta > 0) r = std::fmin(r, 2.0 / (c->prm.alpha * c->prm.beta));
    if (!std::isfinite(r) || !(r > 0)) return fail(DGK_ERR_NONFINITE, "non-finite time step (state invalid)");
    *dt = r;
    return DGK_OK;
}

int dgk_diagnostics(dgk_ctx *c, double *out)
{
    int rc = ready(c);
    if (rc) return rc;
    if (!out) return fail(DGK_ERR_ARG, "null output");
    if ((rc = diag_buffers(c))) return rc;
    if ((rc = enqueue_diag(c, c->diagout, nullptr))) return rc;
    DGK_CUDA(cudaMemcpyAsync(out, c->diagout, kNDiag * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    DGK_CUDA(cudaStreamSynchronize(c->stream));
    return DGK_OK;
}

int dgk_node_temperature_pressure(dgk_ctx *c, double *T, double *p, size_t count, int on_device)
{
    int rc = ready(c);
    if (rc) return rc;
    const size_t nn = (size_t)c->ne * c->NP;
    if (count != nn || (!T && !p)) return fail(DGK_ERR_ARG, "output arrays must hold nelem*np doubles");
    cudaError_t err = run_nodeT(c, 0);
    if (err) return fail(DGK_ERR_CUDA, cudaGetErrorString(err));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (T) DGK_CUDA(cudaMemcpyAsync(T, c->Tbuf, nn * sizeof(double), kind, c->stream));
    if (p) {
        if (!c->rhsbuf) DGK_CUDA(cudaMalloc(&c->rhsbuf, (size_t)c->NV * nn * sizeof(double)));
        k_pressure<<<(unsigned)((nn + 255) / 256), 256, 0, c->stream>>>(c->U, c->Tbuf, c->rhsbuf, (long long)nn);
        DGK_CUDA(cudaGetLastError());
        DGK_CUDA(cudaMemcpyAsync(p, c->rhsbuf, nn * sizeof(double), kind, c->stream));
    }
    DGK_CUDA(cudaStreamSynchronize(c->stream));
    return DGK_OK;
}

int dgk_status(dgk_ctx *c)
{
    if (!c) return fail(DGK_ERR_ARG, "null context");
    DGK_CUDA(cudaStreamSynchronize(c->stream));
    DGK_CUDA(cudaGetLastError());
    if (!c->status) return DGK_OK;
    unsigned s = 0;
    DGK_CUDA(cudaMemcpy(&s, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost));
    DGK_CUDA(cudaMemset(c->status, 0, sizeof(unsigned)));
    if (s & dgk::kStatNonFinite) return fail(DGK_ERR_NONFINITE, "device reported a non-finite state");
    if (s & dgk::kStatDomain) return fail(DGK_ERR_DOMAIN, "device reported a state outside the EoS domain");
    return DGK_OK;
}

int dgk_set_timing(dgk_ctx *c, int enable)
{
    if (!c) return fail(DGK_ERR_ARG, "null context");
    c->timing = enable != 0;
    c->events_used = 0;
    for (int k = 0; k < 3; ++k) { c->t_ms[k] = 0; c->t_cnt[k] = 0; }
    return DGK_OK;
}

int dgk_kernel_time(dgk_ctx *c, int which, double *ms_total, long long *launches)
{
    if (!c || which < 0 || which > 2 || !ms_total) return fail(DGK_ERR_ARG, "bad arguments");
    // resolve outstanding event pairs
    for (size_t i = 0; i + 1 < c->events_used; i += 2) {
        DGK_CUDA(cudaEventSynchronize(c->events[i + 1]));
        float ms = 0.f;
        DGK_CUDA(cudaEventElapsedTime(&ms, c->events[i], c->events[i + 1]));
        int cls = c->event_class[i / 2];
        c->t_ms[cls] += ms;
        c->t_cnt[cls] += 1;
    }
    c->events_used = 0;
    *ms_total = c->t_ms[which];
    if (launches) *launches = c->t_cnt[which];
    return DGK_OK;
}

int dgk_check_conversions(const double *x, size_t n, int on_device, unsigned long long *mismatches)
{
    if (!x || !mismatches) return fail(DGK_ERR_ARG, "null argument");
    double *dx = nullptr;
    unsigned long long *dbad = nullptr;
    DGK_CUDA(cudaMalloc(&dbad, sizeof(unsigned long long)));
    DGK_CUDA(cudaMemset(dbad, 0, sizeof(unsigned long long)));
    if (on_device) {
        dx = const_cast<double *>(x);
    } else {
        DGK_CUDA(cudaMalloc(&dx, n * sizeof(double)));
        DGK_CUDA(cudaMemcpy(dx, x, n * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (n) k_check_conv<<<(unsigned)((n + 255) / 256), 256>>>(dx, (long long)n, dbad);
    cudaError_t err = cudaDeviceSynchronize();
    if (err == cudaSuccess) err = cudaMemcpy(mismatches, dbad, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (!on_device) cudaFree(dx);
    cudaFree(dbad);
    if (err != cudaSuccess) return fail(DGK_ERR_CUDA, cudaGetErrorString(err));
    return DGK_OK;
}

int dgk_maxwell(double T, double *rv, double *rl)
{
    if (!rv || !rl) return fail(DGK_ERR_ARG, "null output");
    if (!dgk::host::maxwell(T, *rv, *rl)) return fail(DGK_ERR_THERMO, "no saturation states at this temperature");
    return DGK_OK;
}

int dgk_sigma_vl(double T, double cv, double gammaK, double *sigma)
{
    (void)cv;  // the cv term of the free energy is linear in rho and drops out
    if (!sigma || !(gammaK > 0)) return fail(DGK_ERR_ARG, "bad arguments");
    if (!dgk::host::sigma_vl(T, gammaK, *sigma)) return fail(DGK_ERR_THERMO, "no saturation states at this temperature");
    return DGK_OK;
}

int dgk_interface_width(double T, double cv, double gammaK, double *width)
{
    double rv, rl, sig;
    int rc = dgk_maxwell(T, &rv, &rl);
    if (rc) return rc;
    if ((rc = dgk_sigma_vl(T, cv, gammaK, &sig))) return rc;
    if (!width) return fail(DGK_ERR_ARG, "null output");
    *width = std::sqrt(2.0) * gammaK * (rl - rv) * (rl - rv) / sig;
    return DGK_OK;
}

}  // extern "C"

// ====================================================================== batched ensembles

// default spin limit of the persistent form's grid barriers: about 2 s at 2 GHz
constexpr long long kBarrierLimitDefault = 4000000000LL;

struct dgk_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    dgk_params prm{};
    std::vector<dgk_ctx *> probs;
    std::vector<int> probN;
    dgk::BatchLaunch L{};
    dgk::KView<float> *d_views = nullptr;
    int *d_probN = nullptr, *d_tiles = nullptr;
    unsigned *d_bar = nullptr;  // [0..1] barrier, [2] status
    int form = 0;               // 0 persistent launch per stage (80-register allocation), 1 grouped
                                // launches per phase, 2 persistent with the 128-register allocation
    int sms = 0, max_bps = 1, max_bps_wide = 1, bps = 1;
    int k[3] = {1, 1, 1};
    size_t tiles_cap = 0;
    cudaGraphExec_t graph = nullptr;
};

namespace {

void batch_drop_graph(dgk_batch *b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
}

// tile table: runs of k_N element blocks of one problem; sorted by degree (N = 3, 4, 5),
// problems of one degree interleaved
int batch_build_tiles(dgk_batch *b)
{
    std::vector<int> tp, tb, tl;
    std::vector<long long> nblk(b->probs.size());
    for (size_t p = 0; p < b->probs.size(); ++p) nblk[p] = (b->probs[p]->ne + b->probs[p]->kt->elems_per_block - 1) /
                                                          b->probs[p]->kt->elems_per_block;
    for (int N = 3; N <= 5; ++N) {
        std::vector<long long> next(b->probs.size(), 0);
        bool more = true;
        while (more) {
            more = false;
            for (size_t p = 0; p < b->probs.size(); ++p) {
                if (b->probN[p] != N || next[p] >= nblk[p]) continue;
                const int kk = b->form == 1 ? 1 : b->k[N - 3];  // grouped form: one element block per CTA
                const long long len = std::min<long long>(kk, nblk[p] - next[p]);
                tp.push_back((int)p);
                tb.push_back((int)next[p]);
                tl.push_back((int)len);
                next[p] += len;
                more = true;
            }
        }
        if (N < 5) b->L.tile_split[N - 3] = (int)tp.size();
    }
    const size_t nt = tp.size();
    if (nt > b->tiles_cap) {
        if (b->d_tiles) cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        DGK_CUDA(cudaMalloc(&b->d_tiles, 3 * nt * sizeof(int)));
        b->tiles_cap = nt;
    }
    std::vector<int> h(3 * nt);
    std::copy(tp.begin(), tp.end(), h.begin());
    std::copy(tb.begin(), tb.end(), h.begin() + nt);
    std::copy(tl.begin(), tl.end(), h.begin() + 2 * nt);
    DGK_CUDA(cudaMemcpy(b->d_tiles, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice));
    b->L.tile_prob = b->d_tiles;
    b->L.tile_blk = b->d_tiles + nt;
    b->L.tile_len = b->d_tiles + 2 * nt;
    b->L.ntiles = (int)nt;
    batch_drop_graph(b);  // the launches carry the tile table and the parameters by value
    return DGK_OK;
}

int batch_launch_step(dgk_batch *b)
{
    const int ns = b->prm.rk == 3 ? 3 : 5;
    for (int s = 0; s < ns; ++s) {
        cudaError_t err = b->form != 1 ? dgk::batch_stage_launch(b->L, b->sms * b->bps, s, b->stream, b->form == 2)
                                       : dgk::batch_phase_launches(b->L, s, b->stream);
        if (err != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("batched stage launch: ") + cudaGetErrorString(err));
    }
    return DGK_OK;
}

}  // namespace

extern "C" {

int dgk_batch_create(dgk_batch **out, int device, void *cuda_stream, const dgk_params *p, int nprob,
                     const dgk_box_mesh *meshes)
{
    if (!out || !p || nprob < 1 || !meshes) return fail(DGK_ERR_ARG, "bad arguments");
    *out = nullptr;
    if (p->precision != DGK_PREC_FP32BULK) return fail(DGK_ERR_UNSUPPORTED, "batched ensembles run the FP32-bulk form");
    if (p->flux != DGK_FLUX_RUSANOV) return fail(DGK_ERR_UNSUPPORTED, "batched ensembles use the Rusanov flux");
    for (int i = 0; i < nprob; ++i)
        if (meshes[i].dim != 2 || meshes[i].N < 3 || meshes[i].N > 5)
            return fail(DGK_ERR_UNSUPPORTED, "batched ensembles take 2D meshes with N = 3..5");
    DGK_CUDA(cudaSetDevice(device));
    dgk_batch *b = new (std::nothrow) dgk_batch();
    if (!b) return fail(DGK_ERR_NOMEM, "host allocation failed");
    b->device = device;
    b->prm = *p;
    int rc = DGK_OK;
    if (cuda_stream) b->stream = (cudaStream_t)cuda_stream;
    else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return fail(DGK_ERR_CUDA, "cudaStreamCreate failed");
        }
        b->own_stream = true;
    }
    for (int i = 0; i < nprob && !rc; ++i) {
        dgk_ctx *c = nullptr;
        rc = dgk_create(&c, device, b->stream);
        if (!rc) b->probs.push_back(c);
        if (!rc) rc = dgk_set_params(c, p);
        if (!rc) rc = dgk_mesh_box(c, &meshes[i]);
        if (!rc) rc = set_coef(c, 1e-6);
        b->probN.push_back(meshes[i].N);
    }
    std::vector<dgk::KView<float>> views;
    for (dgk_ctx *c : b->probs) views.push_back(c->a32.v);
    int maxb = 0, maxw = 0;
    if (!rc && dgk::batch_prepare(&maxb, &maxw) != cudaSuccess) rc = fail(DGK_ERR_CUDA, "batched kernel set-up failed");
    if (!rc && maxb < 1) rc = fail(DGK_ERR_UNSUPPORTED, "batched kernel does not fit on an SM");
    if (!rc && (cudaMalloc(&b->d_views, views.size() * sizeof(views[0])) != cudaSuccess ||
                cudaMalloc(&b->d_probN, b->probN.size() * sizeof(int)) != cudaSuccess ||
                cudaMalloc(&b->d_bar, 4 * sizeof(unsigned)) != cudaSuccess))
        rc = fail(DGK_ERR_NOMEM, "batch tables");
    if (!rc && (cudaMemcpy(b->d_views, views.data(), views.size() * sizeof(views[0]), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(b->d_probN, b->probN.data(), b->probN.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemset(b->d_bar, 0, 4 * sizeof(unsigned)) != cudaSuccess))
        rc = fail(DGK_ERR_CUDA, "batch table upload");
    if (!rc) {
        cudaDeviceProp prop;
        cudaGetDeviceProperties(&prop, device);
        b->sms = prop.multiProcessorCount;
        b->max_bps = maxb;
        b->max_bps_wide = maxw > 0 ? maxw : 1;
        b->bps = maxb;
        b->L.views = b->d_views;
        b->L.prob_N = b->d_probN;
        b->L.ph = b->probs[0]->a32.ph;
        b->L.pr = b->probs[0]->a32.pr;
        for (int n = 3; n <= 5; ++n) {
            dgk::host::Operators1D op;
            dgk::host::dg_operators(n, op);
            dgk::OpsR<float> &o = b->L.op[n - 3];
            std::memset(&o, 0, sizeof(o));
            for (int i = 0; i <= n; ++i) {
                for (int j = 0; j <= n; ++j) o.Dh[i * (n + 1) + j] = (float)op.Dhat[i * (n + 1) + j];
                o.Lp[i] = (float)(op.lp[i] / op.w[i]);
                o.Lm[i] = (float)(op.lm[i] / op.w[i]);
                o.lp[i] = (float)op.lp[i];
                o.lm[i] = (float)op.lm[i];
            }
            dgk::fill_pairs(o, n + 1);
        }
        b->L.bar = b->d_bar;
        b->L.status = b->d_bar + 2;
        b->L.bar_limit = kBarrierLimitDefault;
        rc = batch_build_tiles(b);
    }
    if (rc) {
        dgk_batch_destroy(b);
        return rc;
    }
    *out = b;
    return DGK_OK;
}

void dgk_batch_destroy(dgk_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    batch_drop_graph(b);
    for (dgk_ctx *c : b->probs) dgk_destroy(c);
    if (b->d_views) cudaFree(b->d_views);
    if (b->d_probN) cudaFree(b->d_probN);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_bar) cudaFree(b->d_bar);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
}

dgk_ctx *dgk_batch_problem(dgk_batch *b, int i)
{
    if (!b || i < 0 || i >= (int)b->probs.size()) return nullptr;
    return b->probs[i];
}

int dgk_batch_set_dt(dgk_batch *b, const double *dt)
{
    if (!b || !dt) return fail(DGK_ERR_ARG, "null argument");
    for (size_t i = 0; i < b->probs.size(); ++i) {
        if (!(dt[i] > 0) || !std::isfinite(dt[i])) return fail(DGK_ERR_ARG, "dt must be positive");
        int rc = set_coef(b->probs[i], dt[i]);
        if (rc) return rc;
    }
    return DGK_OK;
}

int dgk_batch_run(dgk_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return fail(DGK_ERR_ARG, "bad arguments");
    if (nsteps == 0) return DGK_OK;
    if (!b->graph) {
        cudaGraph_t g;
        DGK_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int rc = batch_launch_step(b);
        cudaError_t err = cudaStreamEndCapture(b->stream, &g);
        if (rc) return rc;
        if (err != cudaSuccess) return fail(DGK_ERR_CUDA, std::string("batched graph capture: ") + cudaGetErrorString(err));
        err = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (err != cudaSuccess) {
            b->graph = nullptr;
            return fail(DGK_ERR_CUDA, std::string("batched graph instantiate: ") + cudaGetErrorString(err));
        }
    }
    for (int s = 0; s < nsteps; ++s) DGK_CUDA(cudaGraphLaunch(b->graph, b->stream));
    return DGK_OK;
}

int dgk_batch_set_config(dgk_batch *b, const int *cfg)
{
    if (!b || !cfg) return fail(DGK_ERR_ARG, "null argument");
    if (cfg[0] < 0 || cfg[0] > 2)
        return fail(DGK_ERR_ARG, "form must be 0 (persistent), 1 (grouped) or 2 (persistent, wide allocation)");
    if (cfg[1] < 1 || cfg[1] > (cfg[0] == 2 ? b->max_bps_wide : b->max_bps)) return fail(DGK_ERR_ARG, "blocks per SM out of range");
    for (int i = 2; i < 5; ++i)
        if (cfg[i] < 1) return fail(DGK_ERR_ARG, "element blocks per tile must be positive");
    DGK_CUDA(cudaStreamSynchronize(b->stream));
    b->form = cfg[0];
    b->bps = cfg[1];
    for (int i = 0; i < 3; ++i) b->k[i] = cfg[i + 2];
    return batch_build_tiles(b);
}

int dgk_batch_status(dgk_batch *b, int *per_problem)
{
    if (!b) return fail(DGK_ERR_ARG, "null batch");
    DGK_CUDA(cudaStreamSynchronize(b->stream));
    unsigned s = 0;
    DGK_CUDA(cudaMemcpy(&s, b->d_bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost));
    DGK_CUDA(cudaMemset(b->d_bar + 2, 0, sizeof(unsigned)));
    // after a timeout the arrival counter is stale: start the next launch from zero
    if (s & dgk::kStatBarrier) DGK_CUDA(cudaMemset(b->d_bar, 0, 2 * sizeof(unsigned)));
    int first = (s & dgk::kStatBarrier) ? fail(DGK_ERR_TIMEOUT, "a grid barrier of the batched kernel timed out") : DGK_OK;
    for (size_t i = 0; i < b->probs.size(); ++i) {
        const int rc = dgk_status(b->probs[i]);
        if (per_problem) per_problem[i] = rc;
        if (!first && rc) first = rc;
    }
    return first;
}

int dgk_batch_set_barrier_limit(dgk_batch *b, long long cycles)
{
    if (!b || cycles < 1) return fail(DGK_ERR_ARG, "the barrier limit must be at least one cycle");
    DGK_CUDA(cudaStreamSynchronize(b->stream));
    b->L.bar_limit = cycles;
    batch_drop_graph(b);  // a kernel parameter: the step graph is captured again
    return DGK_OK;
}

int dgk_batch_autotune(dgk_batch *b, int *out)
{
    if (!b) return fail(DGK_ERR_ARG, "null batch");
    // refuse to tune on a state that already reports an error (the tuning runs clear the
    // status words at the end)
    int rc = dgk_batch_status(b, nullptr);
    if (rc) return rc;
    // keep the states: U and G of every problem
    std::vector<double *> keep;
    for (dgk_ctx *c : b->probs) {
        const size_t n = (size_t)c->NV * c->ne * c->NP;
        double *k2 = nullptr;
        if (cudaMalloc(&k2, 2 * n * sizeof(double)) != cudaSuccess) {
            for (double *q : keep) cudaFree(q);
            return fail(DGK_ERR_NOMEM, "autotune backup");
        }
        cudaMemcpyAsync(k2, c->U, n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(k2 + n, c->G, n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
        keep.push_back(k2);
    }
    auto restore = [&]() {
        for (size_t i = 0; i < b->probs.size(); ++i) {
            dgk_ctx *c = b->probs[i];
            const size_t n = (size_t)c->NV * c->ne * c->NP;
            cudaMemcpyAsync(c->U, keep[i], n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
            cudaMemcpyAsync(c->G, keep[i] + n, n * sizeof(double), cudaMemcpyDeviceToDevice, b->stream);
            c->kt->traces(c->args(), b->stream);
        }
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // every candidate starts from the kept state: one warm-up step, then two timed steps
    auto time_config = [&](float &ms) -> int {
        restore();
        int r = batch_launch_step(b);
        if (r) return r;
        cudaEventRecord(e0, b->stream);
        for (int k = 0; k < 2 && !r; ++k) r = batch_launch_step(b);
        cudaEventRecord(e1, b->stream);
        if (r) return r;
        if (cudaEventSynchronize(e1) != cudaSuccess) return fail(DGK_ERR_CUDA, "autotune timing");
        cudaEventElapsedTime(&ms, e0, e1);
        return DGK_OK;
    };
    float best = 1e30f;
    // persistent form over resident blocks per SM, then the grouped form; then element
    // blocks per tile for each degree in the faster form (greedy)
    int best_bps = b->bps, best_form = b->form;
    float best_form_ms[2] = {1e30f, 1e30f};
    b->form = 0;
    rc = batch_build_tiles(b);
    for (int bps = 1; bps <= b->max_bps && !rc; ++bps) {
        b->bps = bps;
        float ms = 0;
        rc = time_config(ms);
        if (!rc && ms < best) { best = ms; best_bps = bps; best_form = 0; }
        if (!rc && ms < best_form_ms[0]) best_form_ms[0] = ms;
    }
    // the persistent form with the 128-register allocation
    if (!rc) {
        b->form = 2;
        rc = batch_build_tiles(b);
        for (int bps = 1; bps <= b->max_bps_wide && !rc; ++bps) {
            b->bps = bps;
            float ms = 0;
            rc = time_config(ms);
            if (!rc && ms < best) { best = ms; best_bps = bps; best_form = 2; }
            if (!rc && ms < best_form_ms[0]) best_form_ms[0] = ms;
        }
    }
    b->bps = best_bps;
    if (!rc) {
        b->form = 1;
        float ms = 0;
        if (!(rc = batch_build_tiles(b))) rc = time_config(ms);
        if (!rc && ms < best) { best = ms; best_form = 1; }
        if (!rc) best_form_ms[1] = ms;
    }
    b->form = best_form;
    if (!rc) rc = batch_build_tiles(b);
    // element blocks per tile: the persistent forms only
    for (int n = 0; n < 3 && !rc && b->form != 1; ++n) {
        bool used = false;
        for (int q : b->probN) used |= (q == n + 3);
        if (!used) continue;
        int best_k = b->k[n];
        for (int kk : {1, 2, 4}) {
            b->k[n] = kk;
            if ((rc = batch_build_tiles(b))) break;
            float ms = 0;
            if ((rc = time_config(ms))) break;
            if (ms < best) { best = ms; best_k = kk; }
            if (ms < best_form_ms[0]) best_form_ms[0] = ms;
        }
        b->k[n] = best_k;
    }
    if (!rc) rc = batch_build_tiles(b);
    restore();
    cudaStreamSynchronize(b->stream);
    for (double *q : keep) cudaFree(q);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // statuses latched by the tuning runs say nothing about the restored states
    for (dgk_ctx *c : b->probs)
        if (c->status) cudaMemset(c->status, 0, sizeof(unsigned));
    cudaMemset(b->d_bar + 2, 0, sizeof(unsigned));
    if (out) {
        out[0] = b->form;
        out[1] = b->bps;
        out[2] = b->k[0];
        out[3] = b->k[1];
        out[4] = b->k[2];
        out[5] = (int)(500.0f * best_form_ms[0]);  // two timed steps -> microseconds per step
        out[6] = (int)(500.0f * best_form_ms[1]);
    }
    return rc;
}

}  // extern "C"
