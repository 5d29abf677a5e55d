// The node-pair tile of the one-step update for FP32- and FP16-deviation
// storage (two x-adjacent nodes per thread), shared by the node-pair step
// kernel (step_pair.cu) and the persistent sweep kernel (sweep.cu).
//
// A thread of an interior tile away from the body loads the two nodes'
// pulls (one aligned pair load for the three populations with c_ax = 0,
// two single loads for the others), runs the MRT update once on float2
// lanes with paired FP32 instructions (mrt_dev_lanes<Lane2>: every lane
// rounds as the scalar update does, so the populations are those of the
// one-node kernel bit for bit) and stores the nine results as pairs.
// Tiles meeting the body's node range take the one-node code for each of
// their nodes; tiles on a lattice edge pull each node with the boundary
// rules and then, in FP16 storage away from the body, update the pair on
// paired lanes, otherwise node by node.  Requires an even nx, so that every
// row starts on a 4-byte boundary of the planes.
#pragma once

#include "step_scalar.cuh"

namespace vplbm {
namespace {

// Blocks of 256 threads per SM the register budget is sized for (48
// registers; 40 and 64 measured within 2 % of it, 5 blocks per SM ahead).
constexpr int PAIR_MINB = 5;

// Nodes (i, j), (i + 1, j) of one pair tile, i even.
template <int P, int SHAPE>
__device__ __forceinline__ void pair_tile(const StepParams &p, int tile_x, int tile_y)
{
    using S = typename Prec<P>::S;
    const int w = 2 * (int)blockDim.x;
    const int bi0 = tile_x * w, bj0 = tile_y * (int)blockDim.y;
    const int i = bi0 + 2 * (int)threadIdx.x, j = bj0 + (int)threadIdx.y;
    const S *__restrict__ fin = static_cast<const S *>(p.fin);
    S *__restrict__ fout = static_cast<S *>(p.fout);
    const BodyState *__restrict__ bs = p.bs_in;
    float cr, cax, cay;
    if (!(bi0 > 0 && bj0 > 0 && bi0 + w < p.nx && bj0 + (int)blockDim.y < p.ny)) {
        // a tile on a lattice edge: each node pulled with the boundary rules
        // (nx even and i even: i < nx gives i + 1 < nx)
        if (i >= p.nx || j >= p.ny) return;
        const int4 range = VPLBM_LDG(reinterpret_cast<const int4 *>(&bs->ilo));
        const bool near = range.x <= range.y && tile_near_body(range, bi0, bj0, w, blockDim.y, false);
        if (P == VPLBM_F16_DEV && !near) {
            // FP16 storage, away from the body: the pair updated on paired
            // lanes (in FP32 storage the one-node code below measured faster)
            float2 f2[NQ];
            {
                float f[NQ];
                pull_all<P>(p, fin, i, j, f);
#pragma unroll
                for (int a = 0; a < NQ; ++a) f2[a].x = f[a];
                pull_all<P>(p, fin, i + 1, j, f);
                if (i + 1 == p.nx - 1 && p.bc[VPLBM_EAST] == VPLBM_BC_CONVECTIVE) record_outlet<P>(p, j, f);
#pragma unroll
                for (int a = 0; a < NQ; ++a) f2[a].y = f[a];
            }
            S *const *dp = reinterpret_cast<S *const *>(p.dst_plane);
            const int b = j * p.nx + i;
            float ax, ay;
            mrt_dev_lanes<Lane2>(p, f2, false, 0.f, 0.f, bs, [&](int a, float2 v) { st_pair(dp[a] + b, v); }, ax,
                                 ay);
            return;
        }
        for (int k = 0; k < 2; ++k) {
            float f[NQ];
            pull_all<P>(p, fin, i + k, j, f);
            if (i + k == p.nx - 1 && p.bc[VPLBM_EAST] == VPLBM_BC_CONVECTIVE) record_outlet<P>(p, j, f);
            node_update<P, VPLBM_COLLISION_MRT, SHAPE>(p, bs, near, i + k, j, f, fout, cr, cax, cay);
        }
        return;
    }
    // streaming loads first: nothing below them waits on the pose
    const int b = j * p.nx + i;
    float2 f2[NQ];
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
        const S *src = static_cast<const S *>(p.src_plane[a]) + b;
        f2[a] = cx_of(a) == 0 ? ld_pair_g(src) : ld_two_g(src);
    }
    const int4 range = VPLBM_LDG(reinterpret_cast<const int4 *>(&bs->ilo));
    if (range.x <= range.y && tile_near_body(range, bi0, bj0, w, blockDim.y, false)) {
        // the tile meets the body's node range: chi node by node
        for (int k = 0; k < 2; ++k) {
            float f[NQ];
#pragma unroll
            for (int a = 0; a < NQ; ++a) f[a] = k ? f2[a].y : f2[a].x;
            node_update<P, VPLBM_COLLISION_MRT, SHAPE>(p, bs, true, i + k, j, f, fout, cr, cax, cay);
        }
        return;
    }
    S *const *dp = reinterpret_cast<S *const *>(p.dst_plane);
    float ax, ay;
    mrt_dev_lanes<Lane2>(p, f2, false, 0.f, 0.f, bs,
                         [&](int a, float2 v) { st_pair(dp[a] + b, v); },
                         ax, ay);
}

}  // namespace
}  // namespace vplbm
