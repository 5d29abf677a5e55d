// Persistent sweep kernel: every member of a batch (many simulations of
// uneven lattice sizes, Sec. 3.3's parameter study) advanced over many time
// steps by ONE launch.
//
// The launch is cooperative: its grid is the number of blocks the device
// keeps resident, and every block stays until the last step.  A time step
// is a list of work items over all members (body slots first, then the
// edge tiles, then the interior tiles member by member in row-major order)
// that the blocks take from a queue.  After each step the blocks meet at a
// grid-wide barrier: the writes of step k (populations, poses, outlet
// columns, the tails' reset tickets) are then visible to every block of
// step k + 1.
//
// Each item runs the tile code of the one-lattice kernels with the item's
// member parameters, so every member's populations, forces and trajectory
// equal those of its own step kernel at the same block shape, bit for bit:
//   body slot:   the scalar tile (one node per thread) that the member's
//                current solid node range maps the slot to, with the
//                solid-node sums (Eqs. 25-27); the last body tile of the
//                member runs its tail (Eqs. 23-24); slot 0 also advances
//                a body on a prescribed path;
//   pair tile:   two x-adjacent nodes per thread (step_pair.cuh);
//   scalar tile: one node per thread, no sums.
//
// The populations and poses that a step reads were written by this launch,
// so this translation unit reads them with ld.global.cg
// (VPLBM_COHERENT_LOADS) instead of the read-only path.
//
// Every barrier wait is bounded (SweepLaunch::timeout_ns on the global
// timer): a block whose wait gives up latches ERR_TIMEOUT, sets the abort
// word, and every block leaves at its next barrier.
#define VPLBM_COHERENT_LOADS 1
#include "step_pair.cuh"

namespace vplbm {
namespace {

// 64 registers: 4 blocks of 256 threads per SM (at 48 the pair-tile loop
// spills: the member parameters come from memory, not the constant bank).
constexpr int SWEEP_MINB = 4;

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier: thread 0 of each block publishes the block's writes
// (fence, then one arrival) and waits until `target` arrivals are counted;
// the acquire load and the fence after it order the block's next reads
// after every other block's writes.  Returns false if the launch is being
// abandoned (this wait gave up, or another block's did).
__device__ __forceinline__ bool sweep_barrier(const SweepLaunch &sl, unsigned target, int *s_go)
{
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        int go = 1;
        __threadfence();
        atomicAdd(&sl.ctl->arrive, 1u);
        const unsigned long long t0 = global_ns();
        while (ld_acquire_gpu(&sl.ctl->arrive) < target) {
            if (*reinterpret_cast<volatile int *>(&sl.ctl->abort)) {
                go = 0;
                break;
            }
            if (global_ns() - t0 > sl.timeout_ns) {
                atomicOr(&sl.ctl->err, ERR_TIMEOUT);
                atomicExch(&sl.ctl->abort, 1);
                go = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        *s_go = go;
    }
    __syncthreads();
    return *s_go != 0;
}

// The items that run one node per thread (rare: the body slots, and the
// tiles of members whose nodes cannot be paired) are functions of their
// own, so that their larger register demand does not shape the register
// allocation of the pair-tile loop.
template <int P, int COLL, int SHAPE>
__device__ __noinline__ void sweep_body_item(const StepParams &p, const int4 it, double (*red)[NPART],
                                             float (*rows)[256], int *s_last)
{
    const int b = it.z;
    const int4 range = VPLBM_LDG(reinterpret_cast<const int4 *>(&p.bs_in->ilo));
    int tx0 = 0, ty0 = 0, rw = 1, nrect = 1;   // no solid node: tile (0, 0) runs the tail
    if (range.x <= range.y) {
        tx0 = range.x / (int)blockDim.x;
        ty0 = range.z / (int)blockDim.y;
        rw = range.y / (int)blockDim.x - tx0 + 1;
        nrect = rw * (range.w / (int)blockDim.y - ty0 + 1);
    }
    if (b < nrect) scalar_tile<P, COLL, SHAPE>(p, tx0 + b % rw, ty0 + b / rw, red, rows, s_last, true);
    if (b == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        if (nrect > it.w) *p.err |= ERR_INTERNAL;
        if (prescribed_motion(p)) advance_prescribed(p);
    }
}

template <int P, int COLL, int SHAPE>
__device__ __noinline__ void sweep_scalar_item(const StepParams &p, const int4 it, double (*red)[NPART],
                                               float (*rows)[256], int *s_last)
{
    scalar_tile<P, COLL, SHAPE>(p, it.z, it.w, red, rows, s_last, false);
}

// One work item with its member's parameters p.
template <int P, int COLL, int SHAPE>
__device__ __forceinline__ void sweep_item(const StepParams &p, const int4 it, double (*red)[NPART],
                                           float (*rows)[256], int *s_last)
{
    if (it.y == SWEEP_PAIR) {
        if constexpr (COLL == VPLBM_COLLISION_MRT && P != VPLBM_F64) pair_tile<P, SHAPE>(p, it.z, it.w);
    } else if (it.y == SWEEP_BODY) {
        sweep_body_item<P, COLL, SHAPE>(p, it, red, rows, s_last);
    } else {
        sweep_scalar_item<P, COLL, SHAPE>(p, it, red, rows, s_last);
    }
}

// Blocks take the items of a step from a queue: one atomic counter that
// runs over all steps of the launch hands out `chunk` consecutive items at
// a time (a block that draws a chunk of the next step keeps it for after
// the barrier).  The queue is pipelined so that neither the counter nor the
// item list is waited for: while a block runs chunk c, its thread 0 draws
// the start of chunk c + 2 and the first `chunk` threads copy the items of
// chunk c + 1 into shared memory (cp.async), both complete by the block
// barrier that ends chunk c.  The list starts with the body slots, so the
// members' tails run early in the step.
//
// PSMEM: the item's member parameters are copied to shared memory when
// the member (or the step parity) changes; otherwise they are read from
// global memory where they are used.
constexpr int SWEEP_MAX_CHUNK = 16;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <int P, int COLL, int SHAPE, bool PSMEM>
__global__ void __launch_bounds__(256, SWEEP_MINB) vp_mrt_sweep(const SweepLaunch sl)
{
    __shared__ double red[8][NPART];
    __shared__ float rows[NPART - 1][256];
    __shared__ int s_last, s_go, s_key;
    __shared__ unsigned s_g[3];                               // chunk starts, chunk c in slot c % 3
    __shared__ __align__(16) int4 s_items[2][SWEEP_MAX_CHUNK]; // items of chunk c in slot c % 2
    __shared__ __align__(16) StepParams s_p;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nthreads = blockDim.x * blockDim.y;
    const unsigned V = sl.items_per_step, CH = sl.chunk;
    if (tid == 0) {
        s_g[0] = atomicAdd(&sl.ctl->grab, CH);
        s_g[1] = atomicAdd(&sl.ctl->grab, CH);
        s_key = -1;
    }
    __syncthreads();
    if (tid < (int)CH) {
        cp_async16(&s_items[0][tid], sl.items + s_g[0] % V + tid);
        cp_async_wait_all();
    }
    __syncthreads();
    int c3 = 0, c2 = 0;   // chunk c's slots in s_g and s_items
    for (int k = 0; k < sl.nsteps; ++k) {
        const int par = (int)((sl.step0 + k) & 1);
        const StepParams *pp = sl.params + (size_t)par * sl.n;
        const unsigned v1 = (unsigned)(k + 1) * V;
        while (s_g[c3] < v1) {   // uniform: written before the last block barrier
            const int n3 = c3 == 2 ? 0 : c3 + 1, nn3 = n3 == 2 ? 0 : n3 + 1;
            // chunk c + 1's items into the other slot (its readers, chunk
            // c - 1, are past the last barrier), chunk c + 2's start
            if (tid < (int)CH) cp_async16(&s_items[c2 ^ 1][tid], sl.items + s_g[n3] % V + tid);
            unsigned g2 = 0;
            if (tid == 0) g2 = atomicAdd(&sl.ctl->grab, CH);
            for (unsigned c = 0; c < CH; ++c) {
                const int4 it = s_items[c2][c];
                if (it.x < 0) continue;   // padding (uniform over the block)
                if constexpr (PSMEM) {
                    const int key = par * sl.n + it.x;
                    if (key != s_key) {
                        __syncthreads();   // the previous item is done with s_p
                        const uint32_t *src = reinterpret_cast<const uint32_t *>(pp + it.x);
                        uint32_t *dst = reinterpret_cast<uint32_t *>(&s_p);
                        for (int q = tid; q < (int)(sizeof(StepParams) / 4); q += nthreads) dst[q] = __ldg(src + q);
                        if (tid == 0) s_key = key;
                        __syncthreads();
                    }
                    sweep_item<P, COLL, SHAPE>(s_p, it, red, rows, &s_last);
                } else {
                    sweep_item<P, COLL, SHAPE>(pp[it.x], it, red, rows, &s_last);
                }
            }
            if (tid < (int)CH) cp_async_wait_all();
            // slot nn3 last held chunk c - 1's start, read before the last barrier
            if (tid == 0) s_g[nn3] = g2;
            __syncthreads();
            c3 = n3;
            c2 ^= 1;
        }
        if (k + 1 < sl.nsteps && !sweep_barrier(sl, (unsigned)(k + 1) * gridDim.x + sl.extra_arrivals, &s_go)) return;
    }
}

template <int P, int COLL, int SHAPE, bool PSMEM>
cudaError_t launch_sweep_t(const SweepLaunch &sl, int grid, int bx, int by, cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(bx, by);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, vp_mrt_sweep<P, COLL, SHAPE, PSMEM>, sl);
}

template <int P, int COLL, int SHAPE, bool PSMEM>
cudaError_t max_grid_t(int bx, int by, int *grid)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, vp_mrt_sweep<P, COLL, SHAPE, PSMEM>, bx * by, 0);
    *grid = sms * per_sm;
    return e;
}

// The instantiations: FP32 and FP16 storage, MRT, the disk or any shape,
// parameters in global or shared memory.
template <int P, int SHAPE>
cudaError_t dispatch_psmem(bool psmem, bool launch, const SweepLaunch *sl, int grid, int bx, int by,
                           cudaStream_t stream, int *max_grid)
{
    constexpr int C = VPLBM_COLLISION_MRT;
    if (launch)
        return psmem ? launch_sweep_t<P, C, SHAPE, true>(*sl, grid, bx, by, stream)
                     : launch_sweep_t<P, C, SHAPE, false>(*sl, grid, bx, by, stream);
    return psmem ? max_grid_t<P, C, SHAPE, true>(bx, by, max_grid) : max_grid_t<P, C, SHAPE, false>(bx, by, max_grid);
}

cudaError_t dispatch(int precision, bool disk, bool psmem, bool launch, const SweepLaunch *sl, int grid, int bx,
                     int by, cudaStream_t stream, int *max_grid)
{
    switch (precision) {
    case VPLBM_F32_DEV:
        return disk ? dispatch_psmem<VPLBM_F32_DEV, VPLBM_SHAPE_DISK>(psmem, launch, sl, grid, bx, by, stream, max_grid)
                    : dispatch_psmem<VPLBM_F32_DEV, SHAPE_ANY>(psmem, launch, sl, grid, bx, by, stream, max_grid);
    case VPLBM_F16_DEV:
        return disk ? dispatch_psmem<VPLBM_F16_DEV, VPLBM_SHAPE_DISK>(psmem, launch, sl, grid, bx, by, stream, max_grid)
                    : dispatch_psmem<VPLBM_F16_DEV, SHAPE_ANY>(psmem, launch, sl, grid, bx, by, stream, max_grid);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int sweep_supported(int precision, int collision)
{
    return (precision == VPLBM_F32_DEV || precision == VPLBM_F16_DEV) && collision == VPLBM_COLLISION_MRT;
}

cudaError_t sweep_max_grid(int precision, bool disk, bool psmem, int bx, int by, int *grid)
{
    *grid = 0;
    return dispatch(precision, disk, psmem, false, nullptr, 0, bx, by, nullptr, grid);
}

cudaError_t launch_sweep(int precision, bool disk, bool psmem, const SweepLaunch &sl, int grid, int bx, int by,
                         cudaStream_t stream)
{
    return dispatch(precision, disk, psmem, true, &sl, grid, bx, by, stream, nullptr);
}

}  // namespace vplbm
