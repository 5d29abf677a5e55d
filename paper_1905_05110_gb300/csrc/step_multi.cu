// The fused step for a lattice that holds several bodies (2 ..
// VPLBM_MAX_BODIES, each a disk, ellipse or rectangle).  Eq. (2) is applied
// body by body: a node is solid for the first body whose chi holds there
// and takes that body's rigid velocity u_s in Eq. (22); the force and
// torque of each body (Eqs. 25-27) sum its own solid nodes, and each body
// has its own tail (history record, motion of Eqs. 23-24).
//
// The launch follows the one-body kernel: the grid's first rows hold the
// body blocks (body k's blocks take the tiles of its node range, reduce
// its sums and elect its tail with its own ticket), the other rows one
// block per tile without sums.  Per-body parameters come from the views
// in device memory (StepParams::views), so the tile reduction and the tail
// are the one-body code run on body k's view.
#include "vplbm_node.cuh"

namespace vplbm {
namespace {

// One tile: pulls, the owner of each node (first body whose chi holds),
// the node update with the owner's rigid velocity, and, in a body block
// of body kb (kb >= 0), the solid-node sums of the nodes kb owns.
template <int P, int COLL>
__device__ __forceinline__ void multi_tile(const StepParams &p, int tile_x, int tile_y, int kb, double (*red)[NPART],
                                           float (*rows)[256], int *s_last)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;
    const int bi0 = tile_x * blockDim.x, bj0 = tile_y * blockDim.y;
    const int i = bi0 + threadIdx.x;
    const int j = bj0 + threadIdx.y;
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const bool block_interior = bi0 > 0 && bj0 > 0 && bi0 + (int)blockDim.x < p.nx && bj0 + (int)blockDim.y < p.ny;
    const bool inside = block_interior || (i < p.nx && j < p.ny);

    T f[NQ];
    if (block_interior) {
        pull_all<P, true>(p, fin, i, j, f);
    } else if (inside) {
        pull_all<P>(p, fin, i, j, f);
        if (i == p.nx - 1 && p.bc[VPLBM_EAST] == VPLBM_BC_CONVECTIVE) record_outlet<P>(p, j, f);
    }

    // bodies whose solid-node range meets the tile (uniform over the block)
    int4 rng[VPLBM_MAX_BODIES];
    unsigned near = 0u;
#pragma unroll
    for (int k = 0; k < VPLBM_MAX_BODIES; ++k) {
        rng[k] = make_int4(1, 0, 1, 0);
        if (k < p.nbodies) {
            rng[k] = __ldg(reinterpret_cast<const int4 *>(&p.bs_in[k].ilo));
            if (tile_near_body(rng[k], bi0, bj0, blockDim.x, blockDim.y, false)) near |= 1u << k;
        }
    }
    int owner = -1;
    T dxl = 0, dyl = 0;
    if (near != 0u && inside) {
#pragma unroll
        for (int k = 0; k < VPLBM_MAX_BODIES; ++k) {
            if (owner < 0 && ((near >> k) & 1u) && i >= rng[k].x && i <= rng[k].y && j >= rng[k].z &&
                j <= rng[k].w) {
                const StepParams &v = p.views[k];
                T dx, dy;
                if (body_chi<P, SHAPE_ANY>(v.body, v.r2f, p.bs_in + k, i, j, dx, dy)) {
                    owner = k;
                    dxl = dx;
                    dyl = dy;
                }
            }
        }
    }
    bool chi = false;
    T cr = 0, cax = 0, cay = 0;
    if (inside)
        chi = node_collide<P, COLL>(p, p.bs_in + (owner < 0 ? 0 : owner), owner >= 0, dxl, dyl, i, j, f, fout, cr, cax,
                                    cay);
    if (kb < 0) return;   // uniform over the block
    const int4 rk = __ldg(reinterpret_cast<const int4 *>(&p.bs_in[kb].ilo));
    tile_solid_sums<P>(p.views[kb], fin, rk, tile_x, tile_y, blockDim.x, blockDim.y, chi && owner == kb, i, j, cr,
                       cax, cay, red, rows, s_last);
}

// MINB: blocks of 256 threads per SM the register budget is sized for.
// Programmatic dependent launch as in the one-body kernel.  Body k's body
// blocks are [body_blocks[k], body_blocks[k + 1]); the first of them also
// computes the next pose of body k when it moves on a prescribed path.
template <int P, int MINB, int COLL>
__global__ void __launch_bounds__(256, MINB) vp_mrt_step_multi(const StepParams p)
{
    __shared__ double red[8][NPART];
    __shared__ float rows[NPART - 1][256];
    __shared__ int s_last;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int nbr = p.nbody_rows;
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    int tx = -1, ty = 0, kb = -1, first_of = -1;
    if ((int)blockIdx.y < nbr) {
        if (b >= p.nbody) return;
        int k = 0, b0 = p.body_blocks[0], b1 = p.body_blocks[1];
#pragma unroll
        for (int m = 1; m < VPLBM_MAX_BODIES; ++m)
            if (m < p.nbodies && b >= p.body_blocks[m]) {
                k = m;
                b0 = p.body_blocks[m];
                b1 = p.body_blocks[m + 1];
            }
        const int lb = b - b0;
        const int4 range = __ldg(reinterpret_cast<const int4 *>(&p.bs_in[k].ilo));
        int tx0 = 0, ty0 = 0, rw = 1, nrect = 1;   // no solid node: tile (0, 0) runs the tail
        if (range.x <= range.y) {
            tx0 = range.x / (int)blockDim.x;
            ty0 = range.z / (int)blockDim.y;
            rw = range.y / (int)blockDim.x - tx0 + 1;
            nrect = rw * (range.w / (int)blockDim.y - ty0 + 1);
        }
        if (lb < nrect) {
            tx = tx0 + lb % rw;
            ty = ty0 + lb / rw;
            kb = k;
        }
        if (lb == 0) {
            first_of = k;
            if (nrect > b1 - b0 && threadIdx.x == 0 && threadIdx.y == 0) *p.err |= ERR_INTERNAL;
        }
    } else {
        tx = blockIdx.x;
        ty = blockIdx.y - nbr;
    }
    if (tx >= 0) multi_tile<P, COLL>(p, tx, ty, kb, red, rows, &s_last);
    if (first_of >= 0 && threadIdx.x == 0 && threadIdx.y == 0) {
        const StepParams &v = p.views[first_of];
        if (prescribed_motion(v)) advance_prescribed(v);
    }
}

template <int P>
cudaError_t launch_multi_t(const StepParams &p0, int bx, int by, int minb, cudaStream_t stream)
{
    StepParams p = p0;
    int acc = 0;
    for (int k = 0; k <= VPLBM_MAX_BODIES; ++k) {
        p.body_blocks[k] = acc;
        if (k < p.nbodies) acc += (int)max_reduction_blocks(p.nx, p.ny, p.body_radius[k], 1, bx, by);
    }
    p.nbody = acc;
    const int ntx = (p.nx + bx - 1) / bx, nty = (p.ny + by - 1) / by;
    const int nbr = (acc + ntx - 1) / ntx;
    p.nbody_rows = nbr;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ntx, nty + nbr);
    cfg.blockDim = dim3(bx, by);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.collision == VPLBM_COLLISION_BGK) {
        if (minb == 6) return cudaLaunchKernelEx(&cfg, vp_mrt_step_multi<P, 6, VPLBM_COLLISION_BGK>, p);
        if (minb == 5) return cudaLaunchKernelEx(&cfg, vp_mrt_step_multi<P, 5, VPLBM_COLLISION_BGK>, p);
        return cudaLaunchKernelEx(&cfg, vp_mrt_step_multi<P, 4, VPLBM_COLLISION_BGK>, p);
    }
    if (minb == 6) return cudaLaunchKernelEx(&cfg, vp_mrt_step_multi<P, 6, VPLBM_COLLISION_MRT>, p);
    if (minb == 5) return cudaLaunchKernelEx(&cfg, vp_mrt_step_multi<P, 5, VPLBM_COLLISION_MRT>, p);
    return cudaLaunchKernelEx(&cfg, vp_mrt_step_multi<P, 4, VPLBM_COLLISION_MRT>, p);
}

}  // namespace

cudaError_t launch_step_multi(int precision, const StepParams &p, int bx, int by, cudaStream_t stream, int minb)
{
    if (p.nbodies < 2 || p.nbodies > VPLBM_MAX_BODIES || !p.views) return cudaErrorInvalidValue;
    switch (precision) {
    case VPLBM_F64: return launch_multi_t<VPLBM_F64>(p, bx, by, minb, stream);
    case VPLBM_F32_DEV: return launch_multi_t<VPLBM_F32_DEV>(p, bx, by, minb, stream);
    case VPLBM_F16_DEV: return launch_multi_t<VPLBM_F16_DEV>(p, bx, by, minb, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vplbm
