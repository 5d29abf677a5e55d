// Streaming, paired variant of the fused VP-MRT step (FP32 / FP16 storage).
//
// A persistent grid: block b walks a contiguous run of work items (an item
// is a 2*bx x by tile; consecutive items are consecutive row groups of one
// column strip).  Each thread owns a pair of x-adjacent nodes per item and
// prefetches the next item's population pairs into registers before it
// collides the current one, so every thread keeps one item of loads in
// flight while it computes.  The c_ax = +-1 planes take their shifted
// element from the neighbour lane (warp shuffle, after the loads landed);
// the lanes at the warp's edges load that element themselves.  The
// collision of the pair runs on the packed FP32x2 pipe (vplbm_pair.cuh);
// lattice edges and items near the body use the scalar code of
// vplbm_node.cuh (boundary rules, chi, FP64 sums, tail).
#include "vplbm_pair.cuh"

namespace vplbm {
namespace {

template <typename S> struct Raw {
    float2 pr[NQ];     // aligned pair (i, i+1) of each plane's source row
    float edge[6];     // warp-edge element of the shifted planes 1, 5, 8 (left) and 3, 6, 7 (right)
};

// Planes shifted by c_ax = +1 (need element i - 1) and -1 (need i + 2).
__device__ __forceinline__ int edge_slot(int a)
{
    return a == 1 ? 0 : a == 5 ? 1 : a == 8 ? 2 : a == 3 ? 3 : a == 6 ? 4 : 5;
}

struct Item {
    int i, j;          // the thread's first node
    int i0, j0;        // tile origin
    int tx, ty;        // tile index
};

__device__ __forceinline__ Item item_of(int t, int nrg, int bx, int by)
{
    Item it;
    const int strip = t / nrg, rg = t - strip * nrg;
    it.tx = strip;
    it.ty = rg;
    it.i0 = strip * 2 * bx;
    it.j0 = rg * by;
    it.i = it.i0 + 2 * threadIdx.x;
    it.j = it.j0 + threadIdx.y;
    return it;
}

template <int P>
__device__ __forceinline__ void fetch(const StepParams &p, const typename Prec<P>::S *__restrict__ fin, const Item &it,
                                      Raw<typename Prec<P>::S> &r)
{
    const int nx = p.nx, ny = p.ny;
    const int lane = threadIdx.x & 31;
    const bool inside = it.i < nx && it.j < ny;
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
        const int sj = it.j - cy_of(a);
        const bool row_ok = inside && sj >= 0 && sj < ny;
        const typename Prec<P>::S *row = fin + a * p.ps + (long long)sj * nx;
        r.pr[a] = row_ok ? ld2(row + it.i) : make_float2(0.f, 0.f);
        if (cx_of(a) == 1)
            r.edge[edge_slot(a)] = (lane == 0 && row_ok && it.i >= 1) ? (float)ldv(row + it.i - 1) : 0.f;
        else if (cx_of(a) == -1)
            r.edge[edge_slot(a)] = (lane == 31 && row_ok && it.i + 2 < nx) ? (float)ldv(row + it.i + 2) : 0.f;
    }
}

template <int P>
__device__ __forceinline__ void process(const StepParams &p, const typename Prec<P>::S *__restrict__ fin,
                                        typename Prec<P>::S *__restrict__ fout, const BodyState *__restrict__ bs,
                                        const int4 range, const Item &it, const Raw<typename Prec<P>::S> &r,
                                        double (*red)[NPART], int *s_last)
{
    using T = typename Prec<P>::T;
    const int nx = p.nx, ny = p.ny;
    const int bx = blockDim.x, by = blockDim.y;
    const bool inside = it.i < nx && it.j < ny;
    const bool near = tile_near_body(range, it.i0, it.j0, 2 * bx, by, it.tx == 0 && it.ty == 0);
    if (!near) {   // uniform over the block
        const int lane = threadIdx.x & 31;
        V2 f[NQ];
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
            const float2 pr = r.pr[a];
            if (cx_of(a) == 0) {
                f[a].v = pr;
            } else if (cx_of(a) == 1) {
                float left = __shfl_up_sync(0xffffffffu, pr.y, 1);
                if (lane == 0) left = r.edge[edge_slot(a)];
                f[a].v = make_float2(left, pr.x);
            } else {
                float right = __shfl_down_sync(0xffffffffu, pr.x, 1);
                if (lane == 31) right = r.edge[edge_slot(a)];
                f[a].v = make_float2(pr.y, right);
            }
        }
        if (!inside) return;
        if (it.i > 0 && it.i + 2 < nx && it.j > 0 && it.j < ny - 1) {
            pair_update<P>(p, f, fout, (long long)it.j * nx + it.i);
        } else {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                T g[NQ];
                pull_all<P>(p, fin, it.i + q, it.j, g);
                T cr, cax, cay;
                (void)node_update<P>(p, bs, false, it.i + q, it.j, g, fout, cr, cax, cay);
            }
        }
        return;
    }
    // an item near the body: scalar path with the FP64 sums
    double part[NPART - 1];
#pragma unroll
    for (int k = 0; k < NPART - 1; ++k) part[k] = 0.0;
    bool any_chi = false;
    if (inside) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            T g[NQ];
            pull_all<P>(p, fin, it.i + q, it.j, g);
            T cr = 0, cax = 0, cay = 0;
            const bool chi = node_update<P>(p, bs, range.x <= range.y, it.i + q, it.j, g, fout, cr, cax, cay);
            if (chi) {
                double one[NPART - 1];
                solid_node_sums<P>(p, fin, it.i + q, it.j, (double)cr, (double)cax, (double)cay, one);
#pragma unroll
                for (int k = 0; k < NPART - 1; ++k) part[k] += one[k];
                any_chi = true;
            }
        }
    }
    tile_reduce(p, range, it.tx, it.ty, 2 * bx, by, any_chi, part, red, s_last);
}

// The work of one block: items [t_begin, t_end) of the row-group-major item
// list, with the next item prefetched while the current one is collided.
template <int P>
__device__ __forceinline__ void stream_items(const StepParams &p, int t_begin, int t_end, double (*red)[NPART],
                                             int *s_last)
{
    using S = typename Prec<P>::S;
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const BodyState *__restrict__ bs = p.bs_in;
    const int bx = blockDim.x, by = blockDim.y;
    const int nrg = (p.ny + by - 1) / by;
    const int4 range = __ldg(reinterpret_cast<const int4 *>(&bs->ilo));   // ilo, ihi, jlo, jhi

    Raw<S> ra, rb;
    int t = t_begin;
    if (t < t_end) fetch<P>(p, fin, item_of(t, nrg, bx, by), ra);
#pragma unroll 1
    for (; t < t_end; t += 2) {
        if (t + 1 < t_end) fetch<P>(p, fin, item_of(t + 1, nrg, bx, by), rb);
        process<P>(p, fin, fout, bs, range, item_of(t, nrg, bx, by), ra, red, s_last);
        if (t + 1 >= t_end) break;
        if (t + 2 < t_end) fetch<P>(p, fin, item_of(t + 2, nrg, bx, by), ra);
        process<P>(p, fin, fout, bs, range, item_of(t + 1, nrg, bx, by), rb, red, s_last);
    }
}

template <int P>
__global__ void __launch_bounds__(256, 2) vp_mrt_step_stream(const StepParams p)
{
    __shared__ double red[8][NPART];
    __shared__ int s_last;
    const int nstrips = (p.nx / 2 + blockDim.x - 1) / blockDim.x;
    const int nrg = (p.ny + blockDim.y - 1) / blockDim.y;
    const long long W = (long long)nstrips * nrg;
    const int t_begin = (int)(W * blockIdx.x / gridDim.x);
    const int t_end = (int)(W * (blockIdx.x + 1) / gridDim.x);
    stream_items<P>(p, t_begin, t_end, red, &s_last);
}

}  // namespace

cudaError_t stream_prepare(int precision, int bx, int by, int *blocks_per_sm)
{
    const void *fn = precision == VPLBM_F32_DEV ? (const void *)vp_mrt_step_stream<VPLBM_F32_DEV>
                                                : (const void *)vp_mrt_step_stream<VPLBM_F16_DEV>;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, bx * by, 0);
}

cudaError_t launch_step_stream(int precision, const StepParams &p, int bx, int by, int grid, cudaStream_t stream)
{
    const long long W = (long long)((p.nx / 2 + bx - 1) / bx) * ((p.ny + by - 1) / by);
    if (grid > W) grid = (int)W;
    dim3 block(bx, by);
    if (precision == VPLBM_F32_DEV)
        vp_mrt_step_stream<VPLBM_F32_DEV><<<grid, block, 0, stream>>>(p);
    else if (precision == VPLBM_F16_DEV)
        vp_mrt_step_stream<VPLBM_F16_DEV><<<grid, block, 0, stream>>>(p);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace vplbm
