// The fused VP-MRT step kernel for one lattice (scalar tiles), templated on
// the storage precision, register budget, collision operator and body
// shape; instantiated for the disk in step_kernels.cu and for the ellipse in
// step_ellipse.cu (two translation units compiled in parallel).
#pragma once

#include "vplbm_node.cuh"

namespace vplbm {
namespace {

// ---- the fused step ----------------------------------------------------

// One tile of the step: blockDim.x x blockDim.y nodes at tile (tile_x,
// tile_y); p may live in shared memory (batched launch).  sums: this block
// also reduces the tile's solid-node sums (and may run the tail).
template <int P, int COLL, int SHAPE = SHAPE_ANY>
__device__ __forceinline__ void scalar_tile(const StepParams &p, int tile_x, int tile_y, double (*red)[NPART],
                                            float (*rows)[256], int *s_last, bool sums)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;
    const int bi0 = tile_x * blockDim.x, bj0 = tile_y * blockDim.y;
    const int i = bi0 + threadIdx.x;
    const int j = bj0 + threadIdx.y;
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const BodyState *__restrict__ bs = p.bs_in;
    // no node of the tile on a lattice edge (uniform over the block)
    const bool block_interior = bi0 > 0 && bj0 > 0 && bi0 + (int)blockDim.x < p.nx && bj0 + (int)blockDim.y < p.ny;
    const bool inside = block_interior || (i < p.nx && j < p.ny);

    // streaming loads first: nothing below them waits on the pose
    T f[NQ];
    if (block_interior) {
        pull_all<P, true>(p, fin, i, j, f);
    } else if (inside) {
        pull_all<P>(p, fin, i, j, f);
        if (i == p.nx - 1 && p.bc[VPLBM_EAST] == VPLBM_BC_CONVECTIVE) record_outlet<P>(p, j, f);
    }

    const int4 range = VPLBM_LDG(reinterpret_cast<const int4 *>(&bs->ilo));   // ilo, ihi, jlo, jhi
    const bool part_block = tile_near_body(range, bi0, bj0, blockDim.x, blockDim.y, tile_x == 0 && tile_y == 0);
    bool chi = false;
    T cr = 0, cax = 0, cay = 0;   // kept for the solid-node sums (converted there)
    if (inside)
        chi = node_update<P, COLL, SHAPE>(p, bs, part_block && range.x <= range.y, i, j, f, fout, cr, cax, cay);
    if (!part_block || !sums) return;   // uniform over the block
    tile_solid_sums<P>(p, fin, range, tile_x, tile_y, blockDim.x, blockDim.y, chi, i, j, cr, cax, cay, red, rows,
                       s_last);
}

// MINB: blocks of 256 threads per SM the register budget is sized for
// (4: 64 registers, 5: 48, 6: 40).
//
// Launched with programmatic dependent launch: every block lets the next
// step's grid start launching at once, and waits (in hardware) until the
// previous step's grid has completed and its writes are visible before it
// reads anything, so the next launch overlaps the end of this one.
//
// The grid's first rows hold p.nbody body blocks, the rest one block per
// tile.  The body blocks are dispatched first: they take the
// tiles that meet the body's node range, reduce the solid-node sums and
// run the tail, so the step's FP64 critical path starts at the beginning
// of the grid instead of wherever the body sits in it.  The row-major
// blocks update every tile without the sums (a body tile is updated twice,
// to identical values) and never wait on the pose before their streaming
// loads.  Body block 0 also computes the next pose of a body on a
// prescribed path.
template <int P, int MINB, int COLL, int SHAPE>
__global__ void __launch_bounds__(256, MINB) vp_mrt_step(const StepParams p)
{
    __shared__ double red[8][NPART];
    __shared__ float rows[NPART - 1][256];
    __shared__ int s_last;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int nbr = p.nbody_rows;
    const int b = blockIdx.y * gridDim.x + blockIdx.x;   // body block index (first rows)
    int tx = -1, ty = 0;
    bool sums = false;
    if ((int)blockIdx.y < nbr) {
        if (b >= p.nbody) return;
        const int4 range = VPLBM_LDG(reinterpret_cast<const int4 *>(&p.bs_in->ilo));
        int tx0 = 0, ty0 = 0, rw = 1, nrect = 1;   // no solid node: tile (0, 0) runs the tail
        if (range.x <= range.y) {
            tx0 = range.x / (int)blockDim.x;
            ty0 = range.z / (int)blockDim.y;
            rw = range.y / (int)blockDim.x - tx0 + 1;
            nrect = rw * (range.w / (int)blockDim.y - ty0 + 1);
        }
        if (b < nrect) {
            tx = tx0 + b % rw;
            ty = ty0 + b / rw;
            sums = true;
        }
        if (b == 0 && nrect > p.nbody && threadIdx.x == 0 && threadIdx.y == 0) *p.err |= ERR_INTERNAL;
    } else {
        tx = blockIdx.x;
        ty = blockIdx.y - nbr;
    }
    if (tx >= 0) scalar_tile<P, COLL, SHAPE>(p, tx, ty, red, rows, &s_last, sums);
    if (b == 0 && threadIdx.x == 0 && threadIdx.y == 0 && prescribed_motion(p)) advance_prescribed(p);
}

template <int P, int SHAPE>
cudaError_t launch_step_t(const StepParams &p0, int bx, int by, int minb, cudaStream_t stream)
{
    StepParams p = p0;
    p.nbody = (int)max_reduction_blocks(p.nx, p.ny, p.body.radius, p.body.present, bx, by);
    const int ntx = (p.nx + bx - 1) / bx, nty = (p.ny + by - 1) / by;
    const int nbr = (p.nbody + ntx - 1) / ntx;
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
        if (minb == 6) return cudaLaunchKernelEx(&cfg, vp_mrt_step<P, 6, VPLBM_COLLISION_BGK, SHAPE>, p);
        if (minb == 5) return cudaLaunchKernelEx(&cfg, vp_mrt_step<P, 5, VPLBM_COLLISION_BGK, SHAPE>, p);
        return cudaLaunchKernelEx(&cfg, vp_mrt_step<P, 4, VPLBM_COLLISION_BGK, SHAPE>, p);
    }
    if (minb == 6) return cudaLaunchKernelEx(&cfg, vp_mrt_step<P, 6, VPLBM_COLLISION_MRT, SHAPE>, p);
    if (minb == 5) return cudaLaunchKernelEx(&cfg, vp_mrt_step<P, 5, VPLBM_COLLISION_MRT, SHAPE>, p);
    return cudaLaunchKernelEx(&cfg, vp_mrt_step<P, 4, VPLBM_COLLISION_MRT, SHAPE>, p);
}


// Step launch for one body shape (all precisions).
template <int SHAPE>
cudaError_t launch_step_shape(int precision, const StepParams &p, int bx, int by, cudaStream_t stream, int minb)
{
    switch (precision) {
    case VPLBM_F64: return launch_step_t<VPLBM_F64, SHAPE>(p, bx, by, minb, stream);
    case VPLBM_F32_DEV: return launch_step_t<VPLBM_F32_DEV, SHAPE>(p, bx, by, minb, stream);
    case VPLBM_F16_DEV: return launch_step_t<VPLBM_F16_DEV, SHAPE>(p, bx, by, minb, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace vplbm
