// Warp-pipelined, paired variant of the fused VP-MRT step (FP32 / FP16).
//
// Each warp owns a strip of 64 columns (two x-adjacent nodes per lane) and
// walks PNK rows of it.  For every row, the lanes copy the nine population
// rows it pulls from -- one aligned pair per lane plus one halo element at
// each end of the strip -- global -> shared memory with asynchronous copies
// (cp.async), PD - 1 rows ahead of the row being collided.  A warp barrier
// (__syncwarp) publishes the copies to the whole warp, and each lane reads
// its shifted pulls from the shared row, so the c_ax = +-1 planes need no
// shuffles and no misaligned global loads.  The collision of the two nodes
// runs on the packed FP32x2 pipe (vplbm_pair.cuh).
//
// Lattice edges and blocks whose tile meets the disk's bounding box take the
// scalar path (boundary rules, chi, FP64 sums, tail) of vplbm_node.cuh.
// Waits are cp.async group waits (hardware), no spinning.
#include "vplbm_pair.cuh"

namespace vplbm {
namespace {

constexpr int PNK = 4;     // rows per warp
constexpr int PD = 3;      // pipeline stages
constexpr int PROW = 68;   // shared row: elements i0 - 2 .. i0 + 65

template <int P> struct Pipe {
    using S = typename Prec<P>::S;
    static constexpr int ES = sizeof(S);
    static constexpr int PLANE = (PROW * ES + 15) / 16 * 16;
    static constexpr int STAGE = NQ * PLANE;
    static constexpr int WARP_BYTES = PD * STAGE;
};

__device__ __forceinline__ void cp_async(void *smem_dst, const void *gmem_src, int bytes)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(gmem_src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ float2 lds2(const float *row, int pos) { return *reinterpret_cast<const float2 *>(row + pos); }
__device__ __forceinline__ float2 lds2(const __half *row, int pos) { return __half22float2(*reinterpret_cast<const __half2 *>(row + pos)); }
__device__ __forceinline__ float lds1(const float *row, int pos) { return row[pos]; }
__device__ __forceinline__ float lds1(const __half *row, int pos) { return __half2float(row[pos]); }

// One tile (64 x nwarps*PNK nodes) of the step; tile_x / tile_y index the
// tile in the lattice, p may live in shared memory (batched launch).
template <int P>
__device__ __forceinline__ void pipe_tile(const StepParams &p, int tile_x, int tile_y, unsigned char *smem,
                                          double (*red)[NPART], int *s_last)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;
    using C = Pipe<P>;

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int tile_h = nwarps * PNK;
    const int nx = p.nx, ny = p.ny;
    const long long ps = p.ps;
    const int i0 = tile_x * 64;
    const int i = i0 + 2 * lane;
    const int jw = tile_y * tile_h + warp * PNK;
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const BodyState *__restrict__ bs = p.bs_in;

    const int4 range = __ldg(reinterpret_cast<const int4 *>(&bs->ilo));   // ilo, ihi, jlo, jhi
    const bool part_block = tile_near_body(range, i0, tile_y * tile_h, 64, tile_h, tile_x == 0 && tile_y == 0);

    if (!part_block) {   // uniform over the block
        unsigned char *wbuf = smem + warp * C::WARP_BYTES;
        auto issue = [&](int k) {
            const int j = jw + k;
            unsigned char *stage = wbuf + (k % PD) * C::STAGE;
            if (j < ny) {
#pragma unroll
                for (int a = 0; a < NQ; ++a) {
                    const int sj = j - cy_of(a);
                    if (sj < 0 || sj >= ny) continue;
                    const S *src = fin + a * ps + (long long)sj * nx;
                    S *row = reinterpret_cast<S *>(stage + a * C::PLANE);
                    if (i < nx) cp_async(row + 2 + 2 * lane, src + i, 2 * C::ES);
                    if (cx_of(a) == 1 && lane == 0 && i0 >= 2)   // element i0 - 1 (F16: its aligned word)
                        cp_async(C::ES == 4 ? (void *)(row + 1) : (void *)row, C::ES == 4 ? (const void *)(src + i0 - 1) : (const void *)(src + i0 - 2), 4);
                    if (cx_of(a) == -1 && lane == 31 && i0 + 64 < nx)   // element i0 + 64
                        cp_async(row + 66, src + i0 + 64, 4);
                }
            }
            cp_commit();   // one group per row, empty or not
        };
#pragma unroll
        for (int k = 0; k < PD - 1; ++k) issue(k);
#pragma unroll 1
        for (int k = 0; k < PNK; ++k) {
            __syncwarp();   // every lane is done with the stage refilled next
            if (k + PD - 1 < PNK) issue(k + PD - 1);
            else cp_commit();
            cp_wait<PD - 1>();
            __syncwarp();   // the copies of row k, by every lane, are visible
            const int j = jw + k;
            if (i < nx && j < ny) {
                if (i > 0 && i + 2 < nx && j > 0 && j < ny - 1) {
                    const unsigned char *stage = wbuf + (k % PD) * C::STAGE;
                    V2 f[NQ];
#pragma unroll
                    for (int a = 0; a < NQ; ++a) {
                        const S *row = reinterpret_cast<const S *>(stage + a * C::PLANE);
                        const int pos = 2 + 2 * lane - cx_of(a);   // position of element i - c_ax
                        if (cx_of(a) == 0) f[a].v = lds2(row, pos);
                        else f[a].v = make_float2(lds1(row, pos), lds1(row, pos + 1));
                    }
                    pair_update<P>(p, f, fout, (long long)j * nx + i);
                } else {
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        T g[NQ];
                        pull_all<P>(p, fin, i + q, j, g);
                        T cr, cax, cay;
                        (void)node_update<P>(p, bs, false, i + q, j, g, fout, cr, cax, cay);
                    }
                }
            }
        }
        return;
    }

    // a block near the body: scalar path, with the FP64 sums
    double part[NPART - 1];
#pragma unroll
    for (int q = 0; q < NPART - 1; ++q) part[q] = 0.0;
    bool any_chi = false;
#pragma unroll 1
    for (int k = 0; k < PNK; ++k) {
        const int j = jw + k;
        if (i >= nx || j >= ny) continue;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            T g[NQ];
            pull_all<P>(p, fin, i + q, j, g);
            T cr = 0, cax = 0, cay = 0;
            const bool chi = node_update<P>(p, bs, range.x <= range.y, i + q, j, g, fout, cr, cax, cay);
            if (chi) {
                double one[NPART - 1];
                solid_node_sums<P>(p, fin, i + q, j, (double)cr, (double)cax, (double)cay, one);
#pragma unroll
                for (int t = 0; t < NPART - 1; ++t) part[t] += one[t];
                any_chi = true;
            }
        }
    }
    tile_reduce(p, range, tile_x, tile_y, 64, tile_h, any_chi, part, red, s_last);
}


template <int P>
__global__ void __launch_bounds__(256, 3) vp_mrt_step_pipe(const StepParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[8][NPART];
    __shared__ int s_last;
    pipe_tile<P>(p, blockIdx.x, blockIdx.y, smem, red, &s_last);
}

// Every member of a batch in one launch: block b runs tile b of the
// concatenated tile lists; its member is found in the tile prefix and its
// step parameters are staged in shared memory.
template <int P>
__global__ void __launch_bounds__(256, 3) vp_mrt_step_pipe_batch(const BatchLaunch bl)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[8][NPART];
    __shared__ int s_last;
    __shared__ __align__(16) StepParams sp;
    __shared__ int s_member, s_local;
    if (threadIdx.x == 0) {
        int lo = 0, hi = bl.n - 1;   // last member whose first tile is <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bl.tile_start[mid] <= (int)blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_member = lo;
        s_local = (int)blockIdx.x - bl.tile_start[lo];
    }
    __syncthreads();
    const uint32_t *src = reinterpret_cast<const uint32_t *>(bl.params + s_member);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
    for (int k = threadIdx.x; k < (int)(sizeof(StepParams) / 4); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    const int ntx = (sp.nx + 63) / 64;
    pipe_tile<P>(sp, s_local % ntx, s_local / ntx, smem, red, &s_last);
}

}  // namespace

int pipe_rows_per_warp() { return PNK; }

cudaError_t pipe_prepare(int precision, int bx)
{
    const int smem = (bx / 32) * (precision == VPLBM_F32_DEV ? Pipe<VPLBM_F32_DEV>::WARP_BYTES : Pipe<VPLBM_F16_DEV>::WARP_BYTES);
    const void *fn = precision == VPLBM_F32_DEV ? (const void *)vp_mrt_step_pipe<VPLBM_F32_DEV>
                                                : (const void *)vp_mrt_step_pipe<VPLBM_F16_DEV>;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t pipe_batch_prepare(int precision, int bx)
{
    const int smem = (bx / 32) * (precision == VPLBM_F32_DEV ? Pipe<VPLBM_F32_DEV>::WARP_BYTES : Pipe<VPLBM_F16_DEV>::WARP_BYTES);
    const void *fn = precision == VPLBM_F32_DEV ? (const void *)vp_mrt_step_pipe_batch<VPLBM_F32_DEV>
                                                : (const void *)vp_mrt_step_pipe_batch<VPLBM_F16_DEV>;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_step_pipe_batch(int precision, const BatchLaunch &bl, int total_tiles, int bx, cudaStream_t stream)
{
    const int nwarps = bx / 32;
    if (precision == VPLBM_F32_DEV)
        vp_mrt_step_pipe_batch<VPLBM_F32_DEV><<<total_tiles, bx, nwarps * Pipe<VPLBM_F32_DEV>::WARP_BYTES, stream>>>(bl);
    else if (precision == VPLBM_F16_DEV)
        vp_mrt_step_pipe_batch<VPLBM_F16_DEV><<<total_tiles, bx, nwarps * Pipe<VPLBM_F16_DEV>::WARP_BYTES, stream>>>(bl);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_step_pipe(int precision, const StepParams &p, int bx, cudaStream_t stream)
{
    const int nwarps = bx / 32;
    dim3 block(bx, 1);
    dim3 grid((p.nx + 63) / 64, (p.ny + nwarps * PNK - 1) / (nwarps * PNK));
    if (precision == VPLBM_F32_DEV)
        vp_mrt_step_pipe<VPLBM_F32_DEV><<<grid, block, nwarps * Pipe<VPLBM_F32_DEV>::WARP_BYTES, stream>>>(p);
    else if (precision == VPLBM_F16_DEV)
        vp_mrt_step_pipe<VPLBM_F16_DEV><<<grid, block, nwarps * Pipe<VPLBM_F16_DEV>::WARP_BYTES, stream>>>(p);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace vplbm
