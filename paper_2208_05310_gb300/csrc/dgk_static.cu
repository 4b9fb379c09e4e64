// dgk_static.cu -- dgk_rhs_static: the right-hand side of dgk_rhs evaluated with no
// device allocation at all.
//
// Why: some callers cannot call cudaMalloc.  Examples are applications whose device
// memory is entirely reserved by another allocator's pool (a framework's caching
// allocator that owns the GPU), and loops that must never synchronise the device
// (cudaMalloc and cudaFree may synchronise implicitly).  Such callers pass their own
// state and output buffers; every intermediate array of the three stage kernels lives in
// one file-scope device array of fixed size, DGK_STATIC_SCRATCH_BYTES.
//
// Consequences, stated once here and in include/dgk.h:
//   - every GPU that loads libdgk holds this array until the process exits;
//   - all calls share the array and it keeps the last call's contents; the only value
//     that must start at zero (the device status word) is cleared by each call, and its
//     value after the kernels is copied to the caller's status pointer if one is given;
//   - calls that overlap on the GPU (on different streams, or from different host
//     threads) race on the array: the caller must serialise them;
//   - the first call on a device looks up the array's device address (once per device,
//     with that device current); make that first call before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "dgk.h"
#include "dgk_host_math.h"
#include "dgk_launch.cuh"

const dgk::KernelTable *dgk_table_2d_f64(int N);
const dgk::KernelTable *dgk_table_2d_f32(int N);
const dgk::KernelTable *dgk_table_3d_f64(int N);
const dgk::KernelTable *dgk_table_3d_f32(int N);
namespace dgk {
void set_last_error(const std::string &msg);  // dgk_api.cu: the text dgk_last_error() returns
}

static __device__ __align__(256) unsigned char g_rhs_scratch[DGK_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {nullptr};

int fail_static(int code, const char *msg)
{
    dgk::set_last_error(msg);
    return code;
}

// Host-side stand-in -> device address, once per device, with that device current.
int scratch_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) return fail_static(DGK_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[device]) {
        void *p = nullptr;
        cudaError_t err = cudaGetSymbolAddress(&p, g_rhs_scratch);
        if (err != cudaSuccess || !p) return fail_static(DGK_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
        g_scratch_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[device]);
    return DGK_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename R>
int fill(dgk::KArgs<R> &a, const dgk_params &q, const dgk_box_mesh &m, const dgk::host::Operators1D &op, int D, long long ne)
{
    std::memset(&a, 0, sizeof(a));
    a.v.g.ne = ne;
    for (int d = 0; d < 3; ++d) {
        a.v.g.n[d] = d < D ? m.n[d] : 1;
        a.v.g.periodic[d] = d < D ? m.periodic[d] : 1;
        a.v.g.inv2h[d] = d < D ? 2.0 / ((m.hi[d] - m.lo[d]) / m.n[d]) : 0.0;
        a.v.gr.inv2h[d] = (R)a.v.g.inv2h[d];
    }
    a.v.g.div0.init((unsigned)a.v.g.n[0]);
    a.v.g.div1.init((unsigned)a.v.g.n[1]);
    a.ph = dgk::Phys{q.model, q.gammaK, q.mu, q.kappa, q.cv, q.alpha, q.beta, 0.5 * q.alpha, 0.5 * q.gammaK,
                     1.0 / (dgk::kRgas * q.cv)};
    dgk::PhysR<R> &p = a.pr;
    p.model = q.model;
    p.gK = (R)q.gammaK;
    p.mu = (R)q.mu;
    p.kap = (R)q.kappa;
    p.alpha = (R)q.alpha;
    p.beta = (R)q.beta;
    p.gKbeta = (R)(q.gammaK * q.beta);
    p.alphabeta = (R)(q.alpha * q.beta);
    p.half_alpha = (R)(0.5 * q.alpha);
    p.half_gK = (R)(0.5 * q.gammaK);
    p.two_thirds_mu = (R)(2.0 / 3.0 * q.mu);
    p.s_coef = (R)(dgk::kRgas * (1.0 + 1.0 / q.cv));
    p.inv_Rcv = (R)(1.0 / (dgk::kRgas * q.cv));
    p.half_alpha_p = q.model == 2 ? (R)(0.5 * q.alpha) : (R)0;
    p.flux = q.flux;
    for (int f = 0; f < 2 * D; ++f) {
        if (m.periodic[f / 2]) continue;
        double rv, rl, sig;
        if (!dgk::host::maxwell(m.wall[f].T_wall, rv, rl) || !dgk::host::sigma_vl(m.wall[f].T_wall, q.gammaK, sig))
            return fail_static(DGK_ERR_THERMO, "wall temperature has no saturation states (need 0 < T_wall < 1)");
        const double dr = rl - rv;
        a.v.wr.K[f] = (R)(-6.0 * sig * std::cos(m.wall[f].theta_deg * M_PI / 180.0) / (q.gammaK * dr * dr * dr));
        const dgk_wall &wf = m.wall[f];
        const double g1 = wf.kind == 2 ? wf.gamma[0] : 0.0, g2 = wf.kind == 2 ? wf.gamma[1] : 0.0;
        const double g3 = wf.kind == 2 ? wf.gamma[2] : 0.0, g4 = wf.kind == 2 ? wf.gamma[3] : 0.0;
        a.v.wr.kind[f] = wf.kind;
        a.v.wr.g1[f] = (R)g1;
        a.v.wr.g2[f] = (R)g2;
        a.v.wr.g3[f] = (R)g3;
        a.v.wr.g1gK[f] = (R)(g1 / q.gammaK);
        a.v.wr.g1g4[f] = (R)(g1 * g4);
        for (int k = 0; k < 3; ++k) a.v.wr.uw[f][k] = (R)(wf.kind == 1 && k < D ? wf.u_wall[k] : 0.0);
        a.v.wr.rl[f] = (R)rl;
        a.v.wr.rv[f] = (R)rv;
        a.v.wr.Tw[f] = (R)m.wall[f].T_wall;
    }
    const int P = op.P;
    for (int i = 0; i < P; ++i) {
        for (int j = 0; j < P; ++j) a.op.Dh[i * P + j] = (R)op.Dhat[i * P + j];
        a.op.Lp[i] = (R)(op.lp[i] / op.w[i]);
        a.op.Lm[i] = (R)(op.lm[i] / op.w[i]);
        a.op.lp[i] = (R)op.lp[i];
        a.op.lm[i] = (R)op.lm[i];
    }
    dgk::fill_pairs(a.op, P);
    return DGK_OK;
}

template <typename R>
void place(dgk::KArgs<R> &a, unsigned char *base, const double *U, double *Ut, int D, int NP, int NFP, long long ne)
{
    const int NV = D + 3, NL = D + 2, NF = 2 * D;
    size_t off = 0;
    a.v.status = reinterpret_cast<unsigned *>(base + off);
    off += 256;
    a.v.Utv = reinterpret_cast<R *>(base + off);
    off += align256((size_t)NV * ne * NP * sizeof(R));
    a.v.tr1 = reinterpret_cast<R *>(base + off);
    off += align256((size_t)NL * ne * NF * NFP * sizeof(R));
    a.v.tr2 = reinterpret_cast<R *>(base + off);
    off += align256((size_t)2 * ne * NF * NFP * sizeof(R));
    a.v.fd = reinterpret_cast<R *>(base + off);
    off += align256((size_t)(2 * NV + 3) * ne * NF * NFP * sizeof(R));
    a.v.Us = sizeof(R) == 4 ? reinterpret_cast<R *>(base + off) : nullptr;
    a.v.U = const_cast<double *>(U);
    a.v.G = nullptr;
    a.v.met = nullptr;  // box meshes: no metric terms, no connectivity tables
    a.v.fmet = nullptr;
    a.v.conn = nullptr;
    a.v.out = Ut;
    a.v.coef = nullptr;
}

}  // namespace

extern "C" int dgk_rhs_static(const dgk_params *p, const dgk_box_mesh *m, const double *U, double *Ut, size_t count,
                              void *cuda_stream, unsigned *status)
{
    if (!p || !m || !U || !Ut) return fail_static(DGK_ERR_ARG, "null argument");
    // the mesh's shape first: every later check indexes by dim
    if (m->dim != 2 && m->dim != 3) return fail_static(DGK_ERR_UNSUPPORTED, "dim must be 2 or 3");
    if (m->N < 2 || m->N > 5) return fail_static(DGK_ERR_UNSUPPORTED, "N must be 2..5");
    if (p->model < 0 || p->model > 2) return fail_static(DGK_ERR_UNSUPPORTED, "model must be 0, 1 or 2");
    for (int d = 0; d < m->dim && p->model == 0; ++d)
        if (!m->periodic[d]) return fail_static(DGK_ERR_UNSUPPORTED, "the original NSK model runs on periodic boxes");
    if (p->precision != DGK_PREC_FP64 && p->precision != DGK_PREC_FP32BULK) return fail_static(DGK_ERR_ARG, "bad precision");
    if (p->flux != DGK_FLUX_RUSANOV && p->flux != DGK_FLUX_HLLC) return fail_static(DGK_ERR_ARG, "bad flux");
    if (p->flux == DGK_FLUX_HLLC && p->model != 2) return fail_static(DGK_ERR_UNSUPPORTED, "the HLLC flux is for model 2");
    if (!(p->gammaK > 0) || !(p->mu >= 0) || !(p->kappa >= 0) || !(p->cv > 0) || !(p->alpha >= 0) || !(p->beta >= 0))
        return fail_static(DGK_ERR_ARG, "parameters out of range");
    const int D = m->dim, P = m->N + 1;
    const int NP = D == 2 ? P * P : P * P * P, NFP = D == 2 ? P : P * P, NV = D + 3, NL = D + 2, NF = 2 * D;
    long long ne = 1;
    for (int d = 0; d < D; ++d) {
        if (m->n[d] < 1 || !(m->hi[d] > m->lo[d])) return fail_static(DGK_ERR_ARG, "bad element count or extent");
        for (int s = 0; s < 2 && !m->periodic[d]; ++s) {
            const dgk_wall &w = m->wall[2 * d + s];
            if (w.kind != 1 && w.kind != 2) return fail_static(DGK_ERR_ARG, "non-periodic direction needs walls on both faces");
            if (w.kind == 2)
                for (int k = 0; k < 4; ++k)
                    if (!(w.gamma[k] >= 0.0) || !std::isfinite(w.gamma[k]))
                        return fail_static(DGK_ERR_ARG, "wall parameters gamma_1..gamma_4 must be finite and non-negative");
            for (int k = 0; k < D; ++k)
                if (!std::isfinite(w.u_wall[k]) || (w.u_wall[k] != 0.0 && (w.kind != 1 || k == d)))
                    return fail_static(DGK_ERR_ARG, "a wall velocity must be finite, tangential and on a no-slip wall");
        }
        // n[d] < 2^31 and ne < 2^32 before the multiply: the product stays below 2^63
        ne *= m->n[d];
        if (ne >= (1LL << 32)) return fail_static(DGK_ERR_ARG, "mesh too large for the static scratch of dgk_rhs_static (DGK_STATIC_SCRATCH_BYTES)");
    }
    if (ne * (long long)(NP > NF * NFP ? NP : NF * NFP) >= (1LL << 32))
        return fail_static(DGK_ERR_ARG, "mesh too large for the static scratch of dgk_rhs_static (DGK_STATIC_SCRATCH_BYTES)");
    if (count != (size_t)NV * (size_t)ne * (size_t)NP)
        return fail_static(DGK_ERR_ARG, "count must be nvar * nelem * np of the mesh");
    const bool f32 = p->precision == DGK_PREC_FP32BULK;
    const size_t rs = f32 ? sizeof(float) : sizeof(double);
    const size_t need = 256 + align256((size_t)NV * ne * NP * rs) + align256((size_t)NL * ne * NF * NFP * rs) +
                        align256((size_t)2 * ne * NF * NFP * rs) + align256((size_t)(2 * NV + 3) * ne * NF * NFP * rs) +
                        (f32 ? align256((size_t)(NV + 1) * ne * NP * rs) : 0);
    if (need > (size_t)DGK_STATIC_SCRATCH_BYTES)
        return fail_static(DGK_ERR_ARG, "mesh too large for the static scratch of dgk_rhs_static (DGK_STATIC_SCRATCH_BYTES)");
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return fail_static(DGK_ERR_CUDA, "no current CUDA device");
    unsigned char *base = nullptr;
    int rc = scratch_address(device, &base);
    if (rc) return rc;
    dgk::host::Operators1D op;
    if (!dgk::host::dg_operators(m->N, op)) return fail_static(DGK_ERR_ARG, "operator set-up failed");
    const dgk::KernelTable *kt = D == 2 ? (f32 ? dgk_table_2d_f32(m->N) : dgk_table_2d_f64(m->N))
                                        : (f32 ? dgk_table_3d_f32(m->N) : dgk_table_3d_f64(m->N));
    if (!kt) return fail_static(DGK_ERR_UNSUPPORTED, "no kernels for this (dim, N, precision)");
    if (kt->prepare() != cudaSuccess) return fail_static(DGK_ERR_CUDA, "kernel attribute set-up failed");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    dgk::KArgs<double> a64;
    dgk::KArgs<float> a32;
    const void *args;
    if (f32) {
        if ((rc = fill(a32, *p, *m, op, D, ne))) return rc;
        place(a32, base, U, Ut, D, NP, NFP, ne);
        args = &a32;
    } else {
        if ((rc = fill(a64, *p, *m, op, D, ne))) return rc;
        place(a64, base, U, Ut, D, NP, NFP, ne);
        args = &a64;
    }
    if (cudaMemsetAsync(base, 0, 256, s) != cudaSuccess) return fail_static(DGK_ERR_CUDA, "clearing the status word failed");
    if (kt->traces(args, s) != cudaSuccess || kt->lift1(args, s) != cudaSuccess || kt->lift2vol(args, s) != cudaSuccess ||
        kt->surf(args, 0, 0, s) != cudaSuccess)
        return fail_static(DGK_ERR_CUDA, "kernel launch failed");
    // the status word of this call, in stream order (pageable host memory: the copy, and
    // so the call, waits for the kernels)
    if (status && cudaMemcpyAsync(status, base, sizeof(unsigned), cudaMemcpyDefault, s) != cudaSuccess)
        return fail_static(DGK_ERR_CUDA, "reading the status word failed");
    return DGK_OK;
}
