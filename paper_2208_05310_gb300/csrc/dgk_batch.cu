// dgk_batch.cu -- one persistent launch per RK stage for an ensemble of independent 2D
// problems of different degree N (3, 4, 5), mesh size, temperature and contact angle
// (FP32-bulk form).
//
// The launch runs the three phases of a stage (c-lifting + temperature; both liftings +
// volume + face data; surface flux + RK update) for every problem.  Between phases all
// blocks meet at a grid barrier: a counter and a generation word in device memory,
// waited on with a bounded spin.  If the wait exceeds its cycle limit the block records
// kStatBarrier in the status word and the kernel returns, so a fault in residency can
// never hang the GPU.  The launch is cooperative so that every block is resident.
//
// Work items ("tiles") are runs of K consecutive element blocks of one problem; the
// tile table is built on the host from the autotuned K per degree.  Each block copies
// the tile's problem view (geometry, walls, array pointers) into shared memory; physics
// constants and the operators of the three degrees stay kernel parameters.
#include <cuda_runtime.h>

#include "dgk_launch.cuh"

namespace dgk {

constexpr int kBatchThreads = 256;
constexpr int kBatchViewBytes = ((int)sizeof(KView<float>) + 127) / 128 * 128;

template <typename R>
struct BatchArgs {
    const KView<R> *views;  // [nprob]
    const int *prob_N;      // [nprob] degree of each problem
    const int *tile_prob;   // [ntiles]
    const int *tile_blk;    // [ntiles] first element block of the tile
    const int *tile_len;    // [ntiles] element blocks in the tile
    int ntiles;
    Phys ph;
    PhysR<R> pr;
    OpsR<R> op[3];          // N = 3, 4, 5
    unsigned *bar;          // [2]: arrivals, generation
    unsigned *status;       // batch status (barrier timeouts)
    long long bar_limit;    // spin limit, clock cycles
};

// Bounded grid barrier (all blocks resident: cooperative launch).  Returns false after a
// timeout, with kStatBarrier latched.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks, unsigned *status, long long limit)
{
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned *gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > limit) {
                    atomicOr(status, kStatBarrier);
                    ok = 0;
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Batch parameters in constant memory: refreshed from the batch's device copy by a
// device-to-device copy at the start of every step, so that the per-(degree, phase)
// functions below read physics constants and operators as constant-bank operands.
__constant__ BatchArgs<float> c_batch;

// One element block of one problem for one phase, in a function of its own (not
// inlined), so that the nine (degree, phase) bodies get separate register allocations.
#ifndef DGK_BATCH_INLINE
#define DGK_BATCH_BLOCK_ATTR __noinline__
#else
#define DGK_BATCH_BLOCK_ATTR __forceinline__
#endif

template <int N, int PHASE>
__device__ DGK_BATCH_BLOCK_ATTR void batch_block(long long blk, int stage)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    const KView<float> &v = *reinterpret_cast<const KView<float> *>(smraw);
    const Ctx<float> a{v, c_batch.ph, c_batch.pr, c_batch.op[N - 3]};
    unsigned char *sm = smraw + kBatchViewBytes;
    if (PHASE == 0) lift1_body<2, N, float>(a, blk, sm);
    else if (PHASE == 1) lift2vol_body<2, N, float>(a, blk, sm);
    else surf_rk_body<2, N, float>(a, blk, sm, 1, stage);
}

template <int PHASE>
__device__ __forceinline__ void batch_dispatch(int N, long long blk, int stage)
{
    if (N == 3) batch_block<3, PHASE>(blk, stage);
    else if (N == 4) batch_block<4, PHASE>(blk, stage);
    else batch_block<5, PHASE>(blk, stage);
}

#ifndef DGK_BATCH_MIN_BLOCKS
#define DGK_BATCH_MIN_BLOCKS 4  // resident blocks per SM the register allocation targets
#endif

__global__ void __launch_bounds__(kBatchThreads, DGK_BATCH_MIN_BLOCKS) k_batch_stage(int stage)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    KView<float> *sv = reinterpret_cast<KView<float> *>(smraw);
    __shared__ int sN, sblk, slen;
    const BatchArgs<float> &b = c_batch;
    for (int phase = 0; phase < 3; ++phase) {
        for (int tile = blockIdx.x; tile < b.ntiles; tile += gridDim.x) {
            const int p = b.tile_prob[tile];
            const unsigned *src = reinterpret_cast<const unsigned *>(b.views + p);
            unsigned *dst = reinterpret_cast<unsigned *>(sv);
            for (int i = threadIdx.x; i < (int)(sizeof(KView<float>) / 4); i += blockDim.x) dst[i] = src[i];
            if (threadIdx.x == 0) {
                sN = b.prob_N[p];
                sblk = b.tile_blk[tile];
                slen = b.tile_len[tile];
            }
            __syncthreads();
            const int N = sN, len = slen;
            for (int j = 0; j < len; ++j) {
                const long long blk = sblk + j;
                if (phase == 0) batch_dispatch<0>(N, blk, stage);
                else if (phase == 1) batch_dispatch<1>(N, blk, stage);
                else batch_dispatch<2>(N, blk, stage);
                __syncthreads();
            }
        }
        if (phase < 2 && !grid_barrier(b.bar, gridDim.x, b.status, b.bar_limit)) return;
    }
}

// shared memory of one block: the view plus the largest phase of the three degrees
template <typename R>
constexpr size_t batch_smem_bytes()
{
    size_t m = 0;
    const size_t c[9] = {Launcher<2, 3, R>::sm_lift1, Launcher<2, 3, R>::sm_lift2, Launcher<2, 3, R>::sm_surf,
                         Launcher<2, 4, R>::sm_lift1, Launcher<2, 4, R>::sm_lift2, Launcher<2, 4, R>::sm_surf,
                         Launcher<2, 5, R>::sm_lift1, Launcher<2, 5, R>::sm_lift2, Launcher<2, 5, R>::sm_surf};
    for (size_t x : c) m = x > m ? x : m;
    return kBatchViewBytes + m;
}

}  // namespace dgk

// Host-side launcher used by dgk_api.cu (FP32-bulk form).
namespace dgk {

size_t batch_smem() { return batch_smem_bytes<float>(); }

cudaError_t batch_prepare(int *max_blocks_per_sm)
{
    cudaError_t err = cudaFuncSetAttribute(k_batch_stage, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)batch_smem_bytes<float>());
    if (err) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, k_batch_stage, kBatchThreads,
                                                         batch_smem_bytes<float>());
}

size_t batch_args_bytes() { return sizeof(BatchArgs<float>); }

// Fill the batch's device copy of the kernel parameters (host -> device, synchronous).
cudaError_t batch_upload_args(const BatchLaunch &L, void *dev)
{
    BatchArgs<float> b;
    b.views = L.views;
    b.prob_N = L.prob_N;
    b.tile_prob = L.tile_prob;
    b.tile_blk = L.tile_blk;
    b.tile_len = L.tile_len;
    b.ntiles = L.ntiles;
    b.ph = L.ph;
    b.pr = L.pr;
    for (int i = 0; i < 3; ++i) b.op[i] = L.op[i];
    b.bar = L.bar;
    b.status = L.status;
    b.bar_limit = L.bar_limit;
    return cudaMemcpy(dev, &b, sizeof(b), cudaMemcpyHostToDevice);
}

// One step's parameters into constant memory (device-to-device, capturable).
cudaError_t batch_bind_args(const void *dev, cudaStream_t s)
{
    return cudaMemcpyToSymbolAsync(c_batch, dev, sizeof(BatchArgs<float>), 0, cudaMemcpyDeviceToDevice, s);
}

cudaError_t batch_stage_launch(int grid, int stage, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = batch_smem_bytes<float>();
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_stage, stage);
}

}  // namespace dgk
