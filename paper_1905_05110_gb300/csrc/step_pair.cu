// The node-pair step kernel for FP32- and FP16-deviation storage: the
// one-step fused update of Algorithm 1 with two x-adjacent nodes per thread.
//
// The one-node-per-thread kernel runs out of instruction issue before it
// runs out of bandwidth in FP16 storage, and comes close to it in FP32;
// the pair tile (step_pair.cuh) halves the per-node instruction count.
//
// Grid: the scalar kernel's body blocks first (tiles of blockDim.x x
// blockDim.y nodes, one node per thread: they reduce the solid-node sums
// and run the tail), then one block per pair tile of 2 blockDim.x x
// blockDim.y nodes, edge rows and columns first.  Requires an even nx, so that every
// row starts on a 4-byte boundary of the planes.
#include "step_pair.cuh"

namespace vplbm {
namespace {

// MINB: blocks of 256 threads per SM the register budget is sized for.
// Programmatic dependent launch as in the one-node kernel.
template <int P, int MINB, int SHAPE>
__global__ void __launch_bounds__(256, MINB) vp_mrt_step_pair(const StepParams p)
{
    __shared__ double red[8][NPART];
    __shared__ float rows[NPART - 1][256];
    __shared__ int s_last;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int nbr = p.nbody_rows;
    if ((int)blockIdx.y < nbr) {
        // body blocks: one node per thread on tiles of blockDim.x x blockDim.y
        const int b = blockIdx.y * gridDim.x + blockIdx.x;
        if (b >= p.nbody) return;
        const int4 range = VPLBM_LDG(reinterpret_cast<const int4 *>(&p.bs_in->ilo));
        int tx0 = 0, ty0 = 0, rw = 1, nrect = 1;   // no solid node: tile (0, 0) runs the tail
        if (range.x <= range.y) {
            tx0 = range.x / (int)blockDim.x;
            ty0 = range.z / (int)blockDim.y;
            rw = range.y / (int)blockDim.x - tx0 + 1;
            nrect = rw * (range.w / (int)blockDim.y - ty0 + 1);
        }
        if (b < nrect)
            scalar_tile<P, VPLBM_COLLISION_MRT, SHAPE>(p, tx0 + b % rw, ty0 + b / rw, red, rows, &s_last, true);
        if (b == 0 && nrect > p.nbody && threadIdx.x == 0 && threadIdx.y == 0) *p.err |= ERR_INTERNAL;
        if (b == 0 && threadIdx.x == 0 && threadIdx.y == 0 && prescribed_motion(p)) advance_prescribed(p);
        return;
    }
    // row-major over the pair tiles, the two edge rows first and, in each
    // row, its two edge columns first: an edge tile runs the one-node code
    // and takes about twice as long, so it should not be among the last
    // blocks of the launch
    const int ntx = gridDim.x, nty = gridDim.y - nbr;
    const int c = blockIdx.x, r = blockIdx.y - nbr;
    pair_tile<P, SHAPE>(p, c == 0 ? 0 : (c == 1 ? ntx - 1 : c - 1), r == 0 ? 0 : (r == 1 ? nty - 1 : r - 1));
}

template <int P, int SHAPE>
cudaError_t launch_pair_t(const StepParams &p0, int bx, int by, cudaStream_t stream)
{
    StepParams p = p0;
    p.nbody = (int)max_reduction_blocks(p.nx, p.ny, p.body.radius, p.body.present, bx, by);
    const int ntx = (p.nx + 2 * bx - 1) / (2 * bx), nty = (p.ny + by - 1) / by;
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
    return cudaLaunchKernelEx(&cfg, vp_mrt_step_pair<P, PAIR_MINB, SHAPE>, p);
}

}  // namespace

long long pair_grid_rows(int nx, int ny, double radius, int present, int bx, int by)
{
    const long long nbody = max_reduction_blocks(nx, ny, radius, present, bx, by);
    const long long ntx = (nx + 2LL * bx - 1) / (2LL * bx), nty = (ny + by - 1) / by;
    return nty + (nbody + ntx - 1) / ntx;
}

cudaError_t launch_step_pair(int precision, const StepParams &p, int bx, int by, cudaStream_t stream)
{
    if (p.collision != VPLBM_COLLISION_MRT || p.nbodies > 1 || (p.nx & 1)) return cudaErrorInvalidValue;
    const bool disk = !p.body.present || p.body.shape == VPLBM_SHAPE_DISK;
    switch (precision) {
    case VPLBM_F32_DEV:
        return disk ? launch_pair_t<VPLBM_F32_DEV, VPLBM_SHAPE_DISK>(p, bx, by, stream)
                    : launch_pair_t<VPLBM_F32_DEV, SHAPE_ANY>(p, bx, by, stream);
    case VPLBM_F16_DEV:
        return disk ? launch_pair_t<VPLBM_F16_DEV, VPLBM_SHAPE_DISK>(p, bx, by, stream)
                    : launch_pair_t<VPLBM_F16_DEV, SHAPE_ANY>(p, bx, by, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace vplbm
