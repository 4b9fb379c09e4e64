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
// constants and the operators of the three degrees are a kernel parameter.
//
// A second, grouped form runs each phase as an ordinary launch over all tiles (three
// launches per stage, no grid barrier): one kernel holds the bodies of all three phases
// and degrees, and its register allocation is that of the heaviest of the nine, which
// caps the persistent form's occupancy; the grouped kernels each carry one phase.  The
// autotuner times the grouped form and the persistent kernel compiled for three and for
// two resident blocks per SM.
#include <cuda_runtime.h>

// scalar line contractions here: packed, the grouped kernels ran 15% slower
#define DGK_PACKED_LINES 0
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
    int tile_split[2];      // tiles sorted by degree: [0, s0) N = 3, [s0, s1) N = 4, [s1, ntiles) N = 5
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

// The batch parameters are a kernel parameter (__grid_constant__): physics constants and
// the operators of the three degrees are read as parameter-bank operands, also as the
// 64-bit pairs of the packed float contractions.

// One element block of one problem for one phase.
template <int N, int PHASE>
__device__ __forceinline__ void phase_block(const BatchArgs<float> &b, const KView<float> &v, long long blk,
                                            unsigned char *sm, int stage)
{
    const Ctx<float> a{v, b.ph, b.pr, b.op[N - 3]};
    if (PHASE == 0) lift1_body<2, N, float>(a, blk, sm);
    else if (PHASE == 1) lift2vol_body<2, N, float>(a, blk, sm);
    else surf_rk_body<2, N, float>(a, blk, sm, 1, stage);
}

// Persistent form.  The tiles are sorted by degree, and each block walks its grid-stride
// sequence of tiles as three consecutive loops, one per degree, each with one inlined
// body: a single loop around a branch over the three degrees' bodies leaves the
// register allocator with the union of their live ranges across the back edge and
// spills heavily, whereas three single-body loops allocate about like the bodies alone.
template <int N, int PHASE>
__device__ __forceinline__ int run_tiles(const BatchArgs<float> &b, int tile, int end, int stage, KView<float> *sv, int *sh)
{
    unsigned char *sm = reinterpret_cast<unsigned char *>(sv) + kBatchViewBytes;
    for (; tile < end; tile += gridDim.x) {
        const int p = b.tile_prob[tile];
        const unsigned *src = reinterpret_cast<const unsigned *>(b.views + p);
        unsigned *dst = reinterpret_cast<unsigned *>(sv);
        for (int i = threadIdx.x; i < (int)(sizeof(KView<float>) / 4); i += blockDim.x) dst[i] = src[i];
        if (threadIdx.x == 0) {
            sh[0] = b.tile_blk[tile];
            sh[1] = b.tile_len[tile];
        }
        __syncthreads();
        const int blk0 = sh[0], len = sh[1];
        for (int j = 0; j < len; ++j) {
            phase_block<N, PHASE>(b, *sv, blk0 + j, sm, stage);
            __syncthreads();
        }
    }
    return tile;
}

template <int PHASE>
__device__ __forceinline__ void run_phase(const BatchArgs<float> &b, int stage, KView<float> *sv, int *sh)
{
    int tile = blockIdx.x;
    tile = run_tiles<3, PHASE>(b, tile, b.tile_split[0], stage, sv, sh);
    tile = run_tiles<4, PHASE>(b, tile, b.tile_split[1], stage, sv, sh);
    run_tiles<5, PHASE>(b, tile, b.ntiles, stage, sv, sh);
}

// MB: resident blocks per SM the register allocation targets.  One kernel holds the
// bodies of all three phases and degrees, so its allocation is that of the heaviest of
// the nine: 80 registers with spills at MB = 3, 128 registers with few spills at MB = 2
// (the autotuner times both).
template <int MB>
__global__ void __launch_bounds__(kBatchThreads, MB) k_batch_stage(const __grid_constant__ BatchArgs<float> b, int stage)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    KView<float> *sv = reinterpret_cast<KView<float> *>(smraw);
    __shared__ int sh[2];
    run_phase<0>(b, stage, sv, sh);
    if (!grid_barrier(b.bar, gridDim.x, b.status, b.bar_limit)) return;
    run_phase<1>(b, stage, sv, sh);
    if (!grid_barrier(b.bar, gridDim.x, b.status, b.bar_limit)) return;
    run_phase<2>(b, stage, sv, sh);
}

// Grouped form: one ordinary launch per phase over the element blocks of all problems
// (one element block per CTA: the tile table is built with k_N = 1).  Each phase kernel
// holds only that phase's three bodies, so its register allocation is that of the phase
// (the budgets of the single-problem kernels), not of the union of all nine bodies; and
// with no loop around the three-way branch the allocation fits those budgets without
// spilling, which a loop over element blocks around the same branch does not.
template <int PHASE>
struct PhaseBudget;  // resident blocks of kBatchThreads per SM the allocation targets
template <> struct PhaseBudget<0> { static constexpr int min_blocks = 6; };
template <> struct PhaseBudget<1> { static constexpr int min_blocks = 4; };
template <> struct PhaseBudget<2> { static constexpr int min_blocks = 3; };

template <int PHASE>
__global__ void __launch_bounds__(kBatchThreads, PhaseBudget<PHASE>::min_blocks)
    k_batch_phase(const __grid_constant__ BatchArgs<float> b, int stage)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    KView<float> *sv = reinterpret_cast<KView<float> *>(smraw);
    __shared__ int sN, sblk;
    const int tile = blockIdx.x;
    const int p = b.tile_prob[tile];
    const unsigned *src = reinterpret_cast<const unsigned *>(b.views + p);
    unsigned *dst = reinterpret_cast<unsigned *>(sv);
    for (int i = threadIdx.x; i < (int)(sizeof(KView<float>) / 4); i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
        sN = b.prob_N[p];
        sblk = b.tile_blk[tile];
    }
    __syncthreads();
    const int N = sN;
    unsigned char *sm = smraw + kBatchViewBytes;
    if (N == 3) phase_block<3, PHASE>(b, *sv, sblk, sm, stage);
    else if (N == 4) phase_block<4, PHASE>(b, *sv, sblk, sm, stage);
    else phase_block<5, PHASE>(b, *sv, sblk, sm, stage);
}

template <typename R, int PHASE>
constexpr size_t phase_smem_bytes()
{
    size_t m = 0;
    const size_t c[3] = {
        PHASE == 0 ? Launcher<2, 3, R>::sm_lift1 : PHASE == 1 ? Launcher<2, 3, R>::sm_lift2 : Launcher<2, 3, R>::sm_surf,
        PHASE == 0 ? Launcher<2, 4, R>::sm_lift1 : PHASE == 1 ? Launcher<2, 4, R>::sm_lift2 : Launcher<2, 4, R>::sm_surf,
        PHASE == 0 ? Launcher<2, 5, R>::sm_lift1 : PHASE == 1 ? Launcher<2, 5, R>::sm_lift2 : Launcher<2, 5, R>::sm_surf};
    for (size_t x : c) m = x > m ? x : m;
    return kBatchViewBytes + m;
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

cudaError_t batch_prepare(int *max_blocks_per_sm, int *max_blocks_per_sm_wide)
{
    cudaError_t err = cudaFuncSetAttribute(k_batch_stage<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)batch_smem_bytes<float>());
    if (err) return err;
    if ((err = cudaFuncSetAttribute(k_batch_stage<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)batch_smem_bytes<float>())))
        return err;
    if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm_wide, k_batch_stage<2>, kBatchThreads,
                                                             batch_smem_bytes<float>())))
        return err;
    if ((err = cudaFuncSetAttribute(k_batch_phase<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)phase_smem_bytes<float, 0>())))
        return err;
    if ((err = cudaFuncSetAttribute(k_batch_phase<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)phase_smem_bytes<float, 1>())))
        return err;
    if ((err = cudaFuncSetAttribute(k_batch_phase<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)phase_smem_bytes<float, 2>())))
        return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(max_blocks_per_sm, k_batch_stage<3>, kBatchThreads,
                                                         batch_smem_bytes<float>());
}

namespace {
BatchArgs<float> batch_args(const BatchLaunch &L)
{
    BatchArgs<float> b;
    b.views = L.views;
    b.prob_N = L.prob_N;
    b.tile_prob = L.tile_prob;
    b.tile_blk = L.tile_blk;
    b.tile_len = L.tile_len;
    b.ntiles = L.ntiles;
    b.tile_split[0] = L.tile_split[0];
    b.tile_split[1] = L.tile_split[1];
    b.ph = L.ph;
    b.pr = L.pr;
    for (int i = 0; i < 3; ++i) b.op[i] = L.op[i];
    b.bar = L.bar;
    b.status = L.status;
    b.bar_limit = L.bar_limit;
    return b;
}
}  // namespace

// wide: the 128-register allocation (k_batch_stage<2>)
cudaError_t batch_stage_launch(const BatchLaunch &L, int grid, int stage, cudaStream_t s, bool wide)
{
    const BatchArgs<float> b = batch_args(L);
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
    return wide ? cudaLaunchKernelEx(&cfg, k_batch_stage<2>, b, stage) : cudaLaunchKernelEx(&cfg, k_batch_stage<3>, b, stage);
}

cudaError_t batch_phase_launches(const BatchLaunch &L, int stage, cudaStream_t s)
{
    const BatchArgs<float> b = batch_args(L);
    k_batch_phase<0><<<L.ntiles, kBatchThreads, phase_smem_bytes<float, 0>(), s>>>(b, stage);
    k_batch_phase<1><<<L.ntiles, kBatchThreads, phase_smem_bytes<float, 1>(), s>>>(b, stage);
    k_batch_phase<2><<<L.ntiles, kBatchThreads, phase_smem_bytes<float, 2>(), s>>>(b, stage);
    return cudaGetLastError();
}

}  // namespace dgk
