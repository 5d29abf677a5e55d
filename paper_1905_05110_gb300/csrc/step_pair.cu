// Paired variant of the fused VP-MRT step for FP32 / FP16 storage.
//
// Each thread updates two x-adjacent nodes (i, i+1), i even.  Populations
// move as aligned 8-byte (FP32) / 4-byte (FP16) pairs: the unshifted planes
// load their pair directly; a plane shifted by c_ax = +1 takes its first
// element from the left neighbour lane (warp shuffle) and one of the lanes
// at the warp's edge loads that element itself; c_ax = -1 mirrors this.
// The collision runs on Blackwell's packed FP32x2 pipe (FFMA2 / FADD2 /
// FMUL2), two nodes per instruction.  Nodes on the lattice edges and every
// node of a block whose tile meets the disk's bounding box take the scalar
// path of vplbm_node.cuh (boundary rules, chi, the FP64 sums and the tail),
// so the arithmetic of the method is unchanged; only rounding differs.
#include "vplbm_pair.cuh"

namespace vplbm {
namespace {

template <int P>
__global__ void __launch_bounds__(256, 3) vp_mrt_step_pair(const StepParams p)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;

    __shared__ double red[8][NPART];
    __shared__ int s_last;

    const int tile_w = 2 * blockDim.x;
    const int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int nx = p.nx, ny = p.ny;
    const bool inside = i < nx && j < ny;   // nx is even: i + 1 < nx too
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const BodyState *__restrict__ bs = p.bs_in;
    const long long ps = p.ps;

    const int4 range = __ldg(reinterpret_cast<const int4 *>(&bs->ilo));   // ilo, ihi, jlo, jhi
    const bool part_block = tile_near_body(range, blockIdx.x * tile_w, blockIdx.y * blockDim.y, tile_w, blockDim.y,
                                           blockIdx.x == 0 && blockIdx.y == 0);

    if (!part_block) {   // uniform over the block
        const int lane = threadIdx.x & 31;
        V2 f[NQ];
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
            const int sj = j - cy_of(a);
            const bool row_ok = inside && sj >= 0 && sj < ny;
            const S *row = fin + a * ps + (long long)sj * nx;
            const float2 pr = row_ok ? ld2(row + i) : make_float2(0.f, 0.f);
            if (cx_of(a) == 0) {
                f[a].v = pr;
            } else if (cx_of(a) == 1) {      // needs (i - 1, i)
                float left = __shfl_up_sync(0xffffffffu, pr.y, 1);
                if (lane == 0) left = (row_ok && i >= 1) ? (float)ldv(row + i - 1) : 0.f;
                f[a].v = make_float2(left, pr.x);
            } else {                          // needs (i + 1, i + 2)
                float right = __shfl_down_sync(0xffffffffu, pr.x, 1);
                if (lane == 31) right = (row_ok && i + 2 < nx) ? (float)ldv(row + i + 2) : 0.f;
                f[a].v = make_float2(pr.y, right);
            }
        }
        if (!inside) return;
        if (i > 0 && i + 2 < nx && j > 0 && j < ny - 1) {
            pair_update<P>(p, f, fout, (long long)j * nx + i);
        } else {
            // an edge node in the pair: both nodes through the scalar path
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                T g[NQ];
                pull_all<P>(p, fin, i + q, j, g);
                T cr, cax, cay;
                (void)node_update<P>(p, bs, false, i + q, j, g, fout, cr, cax, cay);
            }
        }
        return;
    }

    // a block near the body: scalar path for both nodes, with the FP64 sums
    double part[NPART - 1];
#pragma unroll
    for (int k = 0; k < NPART - 1; ++k) part[k] = 0.0;
    bool any_chi = false;
    if (inside) {
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
                for (int k = 0; k < NPART - 1; ++k) part[k] += one[k];
                any_chi = true;
            }
        }
    }
    tile_reduce(p, range, blockIdx.x, blockIdx.y, tile_w, blockDim.y, any_chi, part, red, &s_last);
}

}  // namespace

cudaError_t launch_step_pair(int precision, const StepParams &p, int bx, int by, cudaStream_t stream)
{
    dim3 block(bx, by);
    dim3 grid((p.nx / 2 + bx - 1) / bx, (p.ny + by - 1) / by);
    if (precision == VPLBM_F32_DEV)
        vp_mrt_step_pair<VPLBM_F32_DEV><<<grid, block, 0, stream>>>(p);
    else if (precision == VPLBM_F16_DEV)
        vp_mrt_step_pair<VPLBM_F16_DEV><<<grid, block, 0, stream>>>(p);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace vplbm
