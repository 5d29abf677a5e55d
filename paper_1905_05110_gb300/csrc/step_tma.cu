// TMA-staged variant of the fused VP-MRT step (FP32 / FP16 storage).
//
// Same arithmetic as vp_mrt_step (vplbm_node.cuh), different data movement:
// persistent CTAs walk a static list of 128 x 4 node chunks; for each chunk
// one thread issues nine cp.async.bulk.tensor loads (one per population
// plane a, rows shifted by c_ay, 16 bytes of halo on each side for the c_ax
// shift) into a 4-stage shared-memory ring, completion tracked by mbarriers
// with transaction counts.  The pull of interior nodes then reads shared
// memory; edge nodes (boundary rules) read global memory as in the plain
// kernel.  Bytes in flight per SM come from shared memory, not registers,
// which is what a streaming stencil at GB300 bandwidth needs.
//
// Every wait on an mbarrier is bounded (about one second of global time);
// on expiry the CTA latches ERR_TIMEOUT, waits (bounded again) for the
// copies it issued, and returns.
#include <cuda.h>

#include "vplbm_node.cuh"

namespace vplbm {
namespace {

constexpr int TW = 128;        // chunk width = blockDim.x
constexpr int TY = 2;          // blockDim.y
constexpr int CR = TMA_TILE_H; // chunk rows (one node per thread)
constexpr int NSTAGE = 3;      // shared-memory ring depth
constexpr unsigned long long WAIT_LIMIT_NS = 1000000000ull;

template <int P> struct Tma {
    using S = typename Prec<P>::S;
    static constexpr int ES = sizeof(S);
    static constexpr int HALO = 16 / ES;                 // 16 bytes of halo: TMA x alignment
    static constexpr int BOXW = TW + 2 * HALO;
    static constexpr int PLANE_BYTES = (CR * BOXW * ES + 127) / 128 * 128;
    static constexpr int STAGE_BYTES = NQ * PLANE_BYTES;
    static constexpr unsigned TX_BYTES = NQ * CR * BOXW * ES;   // delivered per stage
    static constexpr int SMEM = NSTAGE * STAGE_BYTES + 128;      // + alignment slack
};
// each plane's box lands at a 128-byte aligned offset of the stage
static_assert(Tma<VPLBM_F32_DEV>::PLANE_BYTES % 128 == 0 && Tma<VPLBM_F16_DEV>::PLANE_BYTES % 128 == 0, "plane alignment");

__device__ __forceinline__ uint32_t smem_u32(const void *ptr)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase `parity` of an mbarrier.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        for (int k = 0; k < 32; ++k)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > WAIT_LIMIT_NS) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <int P>
__global__ void __launch_bounds__(256, 4) vp_mrt_step_tma(const StepParams p, const __grid_constant__ CUtensorMap tmap)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;
    using C = Tma<P>;

    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bar[NSTAGE];
    __shared__ double red[8][NPART];
    __shared__ int s_last;

    unsigned char *ring = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TW + tx;
    const int nchx = (p.nx + TW - 1) / TW;
    const int nch = nchx * ((p.ny + CR - 1) / CR);
    const int G = gridDim.x;
    const int nmine = (int)blockIdx.x < nch ? (nch - 1 - (int)blockIdx.x) / G + 1 : 0;

    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const BodyState *__restrict__ bs = p.bs_in;

    auto issue = [&](int k) {
        const int c = (int)blockIdx.x + k * G;
        const int stage = k % NSTAGE;
        const int i0 = (c % nchx) * TW, j0 = (c / nchx) * CR;
        unsigned char *dst = ring + stage * C::STAGE_BYTES;
        mbar_expect_tx(&bar[stage], C::TX_BYTES + (k == 0 ? p.tx_extra : 0u));
#pragma unroll
        for (int a = 0; a < NQ; ++a)
            tma_load_3d(dst + a * C::PLANE_BYTES, &tmap, i0 - C::HALO, j0 - cy_of(a), a, &bar[stage]);
    };

    if (tid == 0) {
        for (int s = 0; s < NSTAGE; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int k = 0; k < NSTAGE && k < nmine; ++k) issue(k);

    const int4 range = __ldg(reinterpret_cast<const int4 *>(&bs->ilo));   // ilo, ihi, jlo, jhi

    for (int k = 0; k < nmine; ++k) {
        const int c = (int)blockIdx.x + k * G;
        const int stage = k % NSTAGE;
        const int cxi = c % nchx, cyi = c / nchx;
        const int i0 = cxi * TW, j0 = cyi * CR;
        const bool ok = mbar_wait(&bar[stage], (unsigned)((k / NSTAGE) & 1));
        if (__syncthreads_or(!ok)) {
            // give up on this launch: latch the error, let the copies this
            // CTA issued land (bounded), then leave
            if (tid == 0) {
                atomicOr(p.err, ERR_TIMEOUT);
                for (int kk = k; kk < k + NSTAGE && kk < nmine; ++kk)
                    (void)mbar_wait(&bar[kk % NSTAGE], (unsigned)((kk / NSTAGE) & 1));
            }
            __syncthreads();
            return;
        }
        const unsigned char *st = ring + stage * C::STAGE_BYTES;
        const bool near = tile_near_body(range, i0, j0, TW, CR, c == 0);

        using A = typename SumT<P>::A;
        A part[NPART - 1];
#pragma unroll
        for (int q = 0; q < NPART - 1; ++q) acc_zero(part[q]);
        bool any_chi = false;
#pragma unroll
        for (int rr = 0; rr < CR / TY; ++rr) {
            const int r = ty + rr * TY;
            const int i = i0 + tx, j = j0 + r;
            if (i < p.nx && j < p.ny) {
                T f[NQ];
                if (i > 0 && i < p.nx - 1 && j > 0 && j < p.ny - 1) {
#pragma unroll
                    for (int a = 0; a < NQ; ++a) {
                        const S *plane = reinterpret_cast<const S *>(st + a * C::PLANE_BYTES);
                        if constexpr (P == VPLBM_F16_DEV) f[a] = __half2float(plane[r * C::BOXW + tx + C::HALO - cx_of(a)]);
                        else f[a] = plane[r * C::BOXW + tx + C::HALO - cx_of(a)];
                    }
                } else {
                    pull_all<P>(p, fin, i, j, f);
                    if (i == p.nx - 1 && p.bc[VPLBM_EAST] == VPLBM_BC_CONVECTIVE) record_outlet<P>(p, j, f);
                }
                T cr = 0, cax = 0, cay = 0;
                const bool chi = node_update<P>(p, bs, near && range.x <= range.y, i, j, f, fout, cr, cax, cay);
                if (chi) {
                    float one[NPART - 1];
                    solid_node_terms<P>(p, fin, i, j, cr, cax, cay, one);
#pragma unroll
                    for (int q = 0; q < NPART - 1; ++q) acc_add(part[q], one[q]);
                    any_chi = true;
                }
            }
        }
        if (near) tile_reduce<A>(p, range, cxi, cyi, TW, CR, any_chi, part, red, &s_last);
        __syncthreads();   // every thread is done with this stage
        if (tid == 0 && k + NSTAGE < nmine) issue(k + NSTAGE);
    }
    if (blockIdx.x == 0 && tid == 0 && prescribed_motion(p)) advance_prescribed(p);
}

}  // namespace

int tma_smem_bytes(int precision)
{
    return precision == VPLBM_F32_DEV ? Tma<VPLBM_F32_DEV>::SMEM
         : precision == VPLBM_F16_DEV ? Tma<VPLBM_F16_DEV>::SMEM : 0;
}

int tma_halo(int precision) { return precision == VPLBM_F32_DEV ? 4 : (precision == VPLBM_F16_DEV ? 8 : 0); }

cudaError_t tma_prepare(int precision, int *blocks_per_sm)
{
    const void *fn = precision == VPLBM_F32_DEV ? (const void *)vp_mrt_step_tma<VPLBM_F32_DEV>
                                                : (const void *)vp_mrt_step_tma<VPLBM_F16_DEV>;
    const int smem = tma_smem_bytes(precision);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, TW * TY, smem);
}

cudaError_t launch_step_tma(int precision, const StepParams &p, const CUtensorMap &map, int grid,
                            cudaStream_t stream)
{
    const int nch = ((p.nx + TW - 1) / TW) * ((p.ny + CR - 1) / CR);
    if (grid > nch) grid = nch;
    dim3 block(TW, TY);
    if (precision == VPLBM_F32_DEV)
        vp_mrt_step_tma<VPLBM_F32_DEV><<<grid, block, Tma<VPLBM_F32_DEV>::SMEM, stream>>>(p, map);
    else if (precision == VPLBM_F16_DEV)
        vp_mrt_step_tma<VPLBM_F16_DEV><<<grid, block, Tma<VPLBM_F16_DEV>::SMEM, stream>>>(p, map);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace vplbm
