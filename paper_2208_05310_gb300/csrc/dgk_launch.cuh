// dgk_launch.cuh -- typed launchers of the stage kernels and the (dim, N, precision)
// dispatch table the host runtime uses.  Each instantiation translation unit includes
// this header and defines one dgk_table_<dim>d_<prec>(N) function.
#pragma once

#include "dgk_kernels.cuh"

namespace dgk {

struct KernelTable {
    cudaError_t (*prepare)();  // one-time function attributes (call before any capture)
    cudaError_t (*lift1)(const void *args, cudaStream_t s);
    cudaError_t (*lift2vol)(const void *args, cudaStream_t s);
    cudaError_t (*surf)(const void *args, int mode, int stage, cudaStream_t s);
    cudaError_t (*traces)(const void *args, cudaStream_t s);
    cudaError_t (*nodeT)(const void *args, int mode, cudaStream_t s);
    cudaError_t (*entropy_prod)(const void *args, cudaStream_t s);  // rate of entropy production into out
    int elems_per_block;
    int threads_per_block;
    size_t smem_lift1, smem_lift2vol, smem_surf;
};

template <int D, int N, typename R>
struct Launcher {
    using S = Shape<D, N>;
    static constexpr size_t sm_lift1 = (size_t)S::EPB * CLift<D, N, R>::smem_per_elem * sizeof(R);
    static constexpr size_t sm_lift2 = (size_t)S::EPB * K2Smem<D, N, R>::per_elem * sizeof(R);
    static constexpr size_t sm_surf = (size_t)S::EPB * K3Smem<D, N, R>::per_elem * sizeof(R);
    static constexpr size_t sm_traces = (size_t)S::EPB * S::NL * S::NP * sizeof(R);

    static unsigned blocks(const KArgs<R> &a) { return (unsigned)((a.v.g.ne + S::EPB - 1) / S::EPB); }

    static cudaError_t prepare()
    {
        cudaError_t err;
        if ((err = cudaFuncSetAttribute(k_lift1<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_lift1))) return err;
        if ((err = cudaFuncSetAttribute(k_lift2vol<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_lift2))) return err;
        if ((err = cudaFuncSetAttribute(k_surf_rk<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_surf))) return err;
        if ((err = cudaFuncSetAttribute(k_surf_rk<D, N, R, 0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_surf)))
            return err;
        if ((err = cudaFuncSetAttribute(k_traces<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_traces))) return err;
        if ((err = cudaFuncSetAttribute(k_entropy_prod<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_lift2)))
            return err;
        return cudaFuncSetAttribute(k_node_T<D, N, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm_lift1);
    }
    static cudaError_t entropy_prod(const void *p, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_entropy_prod<D, N, R><<<blocks(a), S::NT, sm_lift2, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t lift1(const void *p, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_lift1<D, N, R><<<blocks(a), S::NT, sm_lift1, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t lift2vol(const void *p, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_lift2vol<D, N, R><<<blocks(a), S::NT, sm_lift2, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t surf(const void *p, int mode, int stage, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        if (a.pr.flux == 1) k_surf_rk<D, N, R, 0, 1><<<blocks(a), S::NT, sm_surf, s>>>(a, mode, stage);
        else k_surf_rk<D, N, R><<<blocks(a), S::NT, sm_surf, s>>>(a, mode, stage);
        return cudaGetLastError();
    }
    static cudaError_t traces(const void *p, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_traces<D, N, R><<<blocks(a), S::NT, sm_traces, s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t nodeT(const void *p, int mode, cudaStream_t s)
    {
        const KArgs<R> &a = *static_cast<const KArgs<R> *>(p);
        k_node_T<D, N, R><<<blocks(a), S::NT, sm_lift1, s>>>(a, mode);
        return cudaGetLastError();
    }
    static const KernelTable *table()
    {
        static const KernelTable t = {prepare, lift1,  lift2vol, surf,     traces,   nodeT, entropy_prod,
                                      S::EPB,  S::NT, sm_lift1, sm_lift2, sm_surf};
        return &t;
    }
};

// Arguments of the batched persistent stage kernel (dgk_batch.cu), FP32-bulk form.
struct BatchLaunch {
    const KView<float> *views;                         // [nprob]
    const int *prob_N, *tile_prob, *tile_blk, *tile_len;
    int ntiles;
    int tile_split[2];                                 // tiles sorted by degree (see dgk_batch.cu)
    Phys ph;
    PhysR<float> pr;
    OpsR<float> op[3];                                 // N = 3, 4, 5
    unsigned *bar, *status;                            // barrier words, batch status
    long long bar_limit;                               // barrier spin limit (cycles)
};
size_t batch_smem();
cudaError_t batch_prepare(int *max_blocks_per_sm, int *max_blocks_per_sm_wide);
cudaError_t batch_stage_launch(const BatchLaunch &L, int grid, int stage, cudaStream_t s, bool wide);
cudaError_t batch_phase_launches(const BatchLaunch &L, int stage, cudaStream_t s);

}  // namespace dgk

#define DGK_DEFINE_TABLE(FNAME, DIM, REAL)                            \
    const dgk::KernelTable *FNAME(int N)                              \
    {                                                                 \
        switch (N) {                                                  \
        case 2: return dgk::Launcher<DIM, 2, REAL>::table();          \
        case 3: return dgk::Launcher<DIM, 3, REAL>::table();          \
        case 4: return dgk::Launcher<DIM, 4, REAL>::table();          \
        case 5: return dgk::Launcher<DIM, 5, REAL>::table();          \
        default: return nullptr;                                      \
        }                                                             \
    }
