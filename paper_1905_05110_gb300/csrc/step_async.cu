// Software-pipelined variant of the fused VP-MRT step (FP32 / FP16 storage).
//
// Each thread updates NK nodes down its column (rows j, j + by, ...).  The
// nine populations a node pulls are copied global -> shared memory with
// per-thread asynchronous copies (cp.async, 4 bytes each) D - 1 nodes ahead
// of the node being collided, so a thread keeps loads in flight while it
// computes and the bytes in flight per SM are bounded by shared memory, not
// by registers.  Completion is tracked with cp.async groups (a hardware
// wait, no spinning); each thread reads back only the slots it filled, so
// no block barrier is needed on this path.
//
// Edge nodes (boundary rules) and the solid-node sums use the scalar code of
// vplbm_node.cuh on global memory, as every other step kernel does.
#include "vplbm_node.cuh"

namespace vplbm {
namespace {

constexpr int ANK = 4;   // nodes per thread (down the column)
constexpr int AD = 3;    // pipeline depth (stages of shared memory)

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// 4-byte word holding element e of a buffer of S (for FP16, the aligned
// pair that contains it); the buffer base is 256-byte aligned.
template <typename S> __device__ __forceinline__ const void *word_of(const S *base, long long e);
template <> __device__ __forceinline__ const void *word_of<float>(const float *base, long long e) { return base + e; }
template <> __device__ __forceinline__ const void *word_of<__half>(const __half *base, long long e)
{
    return base + (e & ~1LL);
}
template <typename S> __device__ __forceinline__ float from_word(uint32_t w, long long e);
template <> __device__ __forceinline__ float from_word<float>(uint32_t w, long long) { return __uint_as_float(w); }
template <> __device__ __forceinline__ float from_word<__half>(uint32_t w, long long e)
{
    const unsigned short h = (e & 1) ? (unsigned short)(w >> 16) : (unsigned short)(w & 0xffffu);
    return __half2float(__ushort_as_half(h));
}

template <int P>
__global__ void __launch_bounds__(256, 4) vp_mrt_step_async(const StepParams p)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;
    extern __shared__ uint32_t sbuf[];   // [AD][NQ][nthreads]
    __shared__ double red[8][NPART];
    __shared__ int s_last;

    const int nt = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int nx = p.nx, ny = p.ny;
    const long long ps = p.ps;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int tile_h = blockDim.y * ANK;
    const int jb = blockIdx.y * tile_h + threadIdx.y;
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const BodyState *__restrict__ bs = p.bs_in;

    auto interior = [&](int j) { return i > 0 && i < nx - 1 && j > 0 && j < ny - 1; };
    auto issue = [&](int k) {
        const int j = jb + k * blockDim.y;
        if (j < ny && interior(j)) {
            const long long b = (long long)j * nx + i;
            uint32_t *slot = sbuf + (k % AD) * NQ * nt + tid;
#pragma unroll
            for (int a = 0; a < NQ; ++a)
                cp_async4(slot + a * nt, word_of<S>(fin, a * ps + b - cx_of(a) - (long long)cy_of(a) * nx));
        }
        cp_async_commit();   // one group per node, empty or not, keeps the counting uniform
    };

    const int4 range = __ldg(reinterpret_cast<const int4 *>(&bs->ilo));   // ilo, ihi, jlo, jhi
    const bool part_block = tile_near_body(range, blockIdx.x * blockDim.x, blockIdx.y * tile_h, blockDim.x, tile_h,
                                           blockIdx.x == 0 && blockIdx.y == 0);

#pragma unroll
    for (int k = 0; k < AD - 1; ++k) issue(k);

    double part[NPART - 1];
#pragma unroll
    for (int q = 0; q < NPART - 1; ++q) part[q] = 0.0;
    bool any_chi = false;

#pragma unroll 1
    for (int k = 0; k < ANK; ++k) {
        if (k + AD - 1 < ANK) issue(k + AD - 1);
        else cp_async_commit();
        cp_async_wait<AD - 1>();   // the copies of node k have landed
        const int j = jb + k * blockDim.y;
        if (i >= nx || j >= ny) continue;
        T f[NQ];
        if (interior(j)) {
            const uint32_t *slot = sbuf + (k % AD) * NQ * nt + tid;
            const long long b = (long long)j * nx + i;
#pragma unroll
            for (int a = 0; a < NQ; ++a)
                f[a] = from_word<S>(slot[a * nt], a * ps + b - cx_of(a) - (long long)cy_of(a) * nx);
        } else {
            pull_all<P>(p, fin, i, j, f);
        }
        T cr = 0, cax = 0, cay = 0;
        const bool chi = node_update<P>(p, bs, part_block && range.x <= range.y, i, j, f, fout, cr, cax, cay);
        if (chi) {
            double one[NPART - 1];
            solid_node_sums<P>(p, fin, i, j, (double)cr, (double)cax, (double)cay, one);
#pragma unroll
            for (int q = 0; q < NPART - 1; ++q) part[q] += one[q];
            any_chi = true;
        }
    }
    if (part_block) tile_reduce(p, range, blockIdx.x, blockIdx.y, blockDim.x, tile_h, any_chi, part, red, &s_last);
}

}  // namespace

int async_rows_per_thread() { return ANK; }

cudaError_t launch_step_async(int precision, const StepParams &p, int bx, int by, cudaStream_t stream)
{
    dim3 block(bx, by);
    dim3 grid((p.nx + bx - 1) / bx, (p.ny + by * ANK - 1) / (by * ANK));
    const size_t smem = (size_t)AD * NQ * bx * by * sizeof(uint32_t);
    if (precision == VPLBM_F32_DEV)
        vp_mrt_step_async<VPLBM_F32_DEV><<<grid, block, smem, stream>>>(p);
    else if (precision == VPLBM_F16_DEV)
        vp_mrt_step_async<VPLBM_F16_DEV><<<grid, block, smem, stream>>>(p);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace vplbm
