// The two-step kernel: time steps n and n + 1 of Algorithm 1 in one launch,
// for a lattice whose body moves on a prescribed path (fixed or imposed) or
// that has none, so that the pose of step n + 1 does not depend on the
// force of step n.
//
// A block owns a FUSED2_W x FUSED2_H tile.  It first computes step n (pull,
// chi, Eq. 22, collision) for the tile and a one-node ring around it, the
// nodes the pulls of step n + 1 reach, and keeps the post-collision
// populations in shared memory, rounded to the storage precision; then it
// computes step n + 1 for the tile from there and stores it.  Each step
// reads and writes HBM once per two steps instead of once per step, and the
// launch boundary is paid once per two steps.  The node arithmetic is the
// one-step kernel's (node_collide_to, body_chi, the same pull rules through
// a shared-memory source), so the populations are those of two one-step
// launches, bit for bit.  A convective outlet's rule at step n + 1 takes
// the values its outlet nodes pulled at step n: the block keeps those of its
// rows in shared memory, and only step n + 1 writes the outlet state (for
// step n + 2, into the other slot than the one step n reads).
//
// Tiles are dispatched edge first: a tile whose region reaches a lattice
// edge takes the boundary rules node by node and runs about twice as long
// as an interior one, and the blocks dispatched last set the end of the
// launch.  The grid runs column by column (blockIdx.x over the tile rows;
// row by row where the tile columns exceed the grid's y limit), the two
// edge columns first and, in each column, its two edge rows first.
//
// Body blocks come first, as in the one-step kernel: they take the tiles
// that meet the union of the node ranges of poses n and n + 1, reduce the
// solid-node sums of both steps (float-float in FP32) and elect a tail for
// each step (record only: the motion is prescribed).  One more block after
// them, with no tile, computes poses n + 2 and n + 3 for the next launch
// in one FP64 thread from the start of the launch, off the tiles' path.
//
// Interior tiles away from the body run both steps on pairs of x-adjacent
// nodes (an even nx keeps every pair on one aligned word): aligned pair
// loads where c_ax = 0, the MRT update on paired FP32 instructions in the
// lane form every FP32 / FP16 kernel shares (mrt_dev_lanes), pair stores;
// the populations stay those of two one-step launches bit for bit.
#include "vplbm_node.cuh"

namespace vplbm {
namespace {

constexpr int F2_TX = FUSED2_W, F2_TY = 256 / FUSED2_W;    // threads per block (x, y): 256
constexpr int F2_NT = F2_TX * F2_TY;                      // 256
// First-step region in the stage: the tile, its one-node ring and one more
// column on each side, so that the region starts on an even column (two
// x-adjacent nodes then sit in one aligned 8-byte pair); the tile's first
// node is at region column F2_X0, row 1.
constexpr int F2_X0 = 2;
constexpr int F2_RW = FUSED2_W + 2 * F2_X0, F2_RH = FUSED2_H + 2;
constexpr int F2_RN = F2_RW * F2_RH;                      // 680 nodes (64 x 8 tiles)
constexpr int F2_ITER = (F2_RN + F2_NT - 1) / F2_NT;      // region nodes per thread at most
constexpr int F2_PN = F2_RN / 2;                          // region node pairs
constexpr int F2_PITER = (F2_PN + F2_NT - 1) / F2_NT;     // region pairs per thread at most
constexpr int F2_ROWS = FUSED2_H / F2_TY;                 // tile nodes per thread
static_assert(FUSED2_W == F2_TX && FUSED2_H % F2_TY == 0, "tile and block shapes");
static_assert(F2_RW % 2 == 0 && FUSED2_W * FUSED2_H / 2 == F2_NT, "one tile pair per thread in the second step");

// Inward populations (a = 3, 6, 7) pulled by the tile's east-outlet nodes at
// step n, [outlet_slot(a)][row in the tile].
__shared__ float f2_outlet[3 * FUSED2_H];

__device__ __forceinline__ float ld_stage(const float *s) { return *s; }
__device__ __forceinline__ float ld_stage(const __half *s) { return __half2float(*s); }


// Stage reader: lattice node (i, j) -> its slot in the region of the tile
// at (bi0, bj0).  A node reached across a periodic edge sits at its
// unwrapped position in the region (the first step computed it there).
// The outlet's previous values are the tile rows' record of step n (CONV:
// the lattice has a convective outlet; otherwise the outlet rule is never
// reached).
template <int P, bool CONV> struct StageSrc {
    const typename Prec<P>::S *stage;
    int bi0, bj0, nx, ny;
    __device__ __forceinline__ typename Prec<P>::T operator()(int a, int i, int j) const
    {
        int li = i - bi0 + F2_X0, lj = j - bj0 + 1;
        if (li >= F2_RW) li -= nx;
        else if (li < 0) li += nx;
        if (lj >= F2_RH) lj -= ny;
        else if (lj < 0) lj += ny;
        return ld_stage(stage + a * F2_RN + lj * F2_RW + li);
    }
    __device__ __forceinline__ float outlet_prev(const StepParams &, int a, int j) const
    {
        if constexpr (CONV) return f2_outlet[outlet_slot(a) * FUSED2_H + (j - bj0)];
        else return 0.f;
    }
};

// Poses n + 2 and n + 3 of a prescribed path from pose n + 1 (the same
// operations as advance_prescribed, twice).
__device__ __noinline__ void advance_two(const StepParams &pb, BodyState *next0, BodyState *next1)
{
    BodyState s = *pb.bs_in;
    const double F0[3] = {0.0, 0.0, 0.0};
    body_advance(pb.body, s.step, F0, s.q, s.v);
    s.step += 1;
    derive_pose(s, pb.body.present, pb.body.radius, pb.nx, pb.ny, pb.body.shape);
    *next0 = s;
    body_advance(pb.body, s.step, F0, s.q, s.v);
    s.step += 1;
    derive_pose(s, pb.body.present, pb.body.radius, pb.nx, pb.ny, pb.body.shape);
    *next1 = s;
}

// Both steps of one tile.  sums: this block also reduces both steps'
// solid-node sums into partial `slot` of `nparts` and may run the tails.
template <int P, int COLL, int SHAPE, bool CONV>
__device__ __forceinline__ void two_steps(const Fused2Params &q, typename Prec<P>::S *stage, int tx, int ty,
                                          bool sums, int slot, int nparts, int4 ra, int4 rb, double (*red)[NPART],
                                          int *s_last)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;
    using A = typename SumT<P>::A;
    using V = typename SumT<P>::V;
    const StepParams &pa = q.a;
    const StepParams &pb = q.b;
    const int nx = pa.nx, ny = pa.ny;
    const int bi0 = tx * FUSED2_W, bj0 = ty * FUSED2_H;
    const int tid = threadIdx.y * F2_TX + threadIdx.x;
    // every region node is at least one node away from the lattice edges
    const bool interior = bi0 >= F2_X0 + 1 && bj0 >= 2 && bi0 + FUSED2_W + F2_X0 + 1 <= nx && bj0 + FUSED2_H + 2 <= ny;
    const S *__restrict__ fin = static_cast<const S *>(pa.fin);
    const BodyState *__restrict__ bsa = pa.bs_in;
    const BodyState *__restrict__ bsb = pb.bs_in;

    // ---- step n on the region, into the stage ----
    const bool near_a =
        ra.x <= ra.y && (!interior || tile_near_body(ra, bi0 - F2_X0, bj0 - 1, F2_RW, F2_RH, false));
    A part[NPART - 1];
#pragma unroll
    for (int k = 0; k < NPART - 1; ++k) acc_zero(part[k]);
    bool any_chi = false;
    // pairs need an even nx: every row of a plane then starts on an even
    // element, so a pair at an even column is one aligned 8-byte (FP32) or
    // 4-byte (FP16) word
    const bool even_rows = (nx & 1) == 0;
    bool pairs = false;
    if constexpr (COLL == VPLBM_COLLISION_MRT) pairs = even_rows && interior && !near_a;
    if (pairs) {
        // an interior region away from the body: two x-adjacent nodes per
        // thread, on paired FP32 instructions (each lane rounds as the
        // one-node update does), aligned pair loads and stage stores
        for (int it = 0; it < F2_PITER; ++it) {
            const int k = it * F2_NT + tid;
            if (k >= F2_PN) break;
            const int lj = k / (F2_RW / 2), li = 2 * (k - lj * (F2_RW / 2));
            const int b = (bj0 - 1 + lj) * nx + bi0 - F2_X0 + li;
            float2 f2[NQ];
#pragma unroll
            for (int a = 0; a < NQ; ++a) {
                const S *src = static_cast<const S *>(pa.src_plane[a]) + b;
                f2[a] = cx_of(a) == 0 ? ld_pair_g(src) : ld_two_g(src);
            }
            S *dst = stage + lj * F2_RW + li;
            float ax, ay;
            mrt_dev_lanes<Lane2>(pa, f2, false, 0.f, 0.f, bsa, [&](int a, float2 v) { st_pair(dst + a * F2_RN, v); },
                                 ax, ay);
        }
    } else {
        for (int it = 0; it < F2_ITER; ++it) {
            const int k = it * F2_NT + tid;
            if (k >= F2_RN) break;
            const int lj = k / F2_RW, li = k - lj * F2_RW;
            const int ui = bi0 - F2_X0 + li, uj = bj0 - 1 + lj;   // unwrapped lattice position
            int i = ui, j = uj;
            if (!interior) {
                if (i < 0 || i >= nx) {   // beyond a wall, or across a periodic edge
                    if (pa.bc[VPLBM_WEST] != VPLBM_BC_PERIODIC) continue;
                    i = ((i % nx) + nx) % nx;
                }
                if (j < 0 || j >= ny) {
                    if (pa.bc[VPLBM_SOUTH] != VPLBM_BC_PERIODIC) continue;
                    j = ((j % ny) + ny) % ny;
                }
            }
            T f[NQ];
            if (interior) {
                pull_all<P, true>(pa, fin, i, j, f);
            } else {
                pull_all<P>(pa, fin, i, j, f);
                if (CONV && ui == nx - 1 && lj >= 1 && lj <= FUSED2_H) {
                    f2_outlet[outlet_slot(3) * FUSED2_H + lj - 1] = f[3];
                    f2_outlet[outlet_slot(6) * FUSED2_H + lj - 1] = f[6];
                    f2_outlet[outlet_slot(7) * FUSED2_H + lj - 1] = f[7];
                }
            }
            T dxl = 0, dyl = 0;
            bool chi = false;
            if (near_a && i >= ra.x && i <= ra.y && j >= ra.z && j <= ra.w)
                chi = body_chi<P, SHAPE>(pa.body, pa.r2f, bsa, i, j, dxl, dyl);
            T cr = 0, cax = 0, cay = 0;
            S *dst = stage + k;
            chi = node_collide_to<P, COLL>(pa, bsa, chi, dxl, dyl, f, [&](int a, T v) { stv(dst + a * F2_RN, v); }, cr,
                                           cax, cay);
            // the tile's own nodes (not the ring, not a wrapped copy) enter the sums
            if (sums && chi && li >= F2_X0 && li < F2_X0 + FUSED2_W && lj >= 1 && lj <= FUSED2_H && ui < nx && uj < ny) {
                V one[NPART - 1];
                solid_node_terms<P>(pa, fin, i, j, (V)cr, (V)cax, (V)cay, one);
    #pragma unroll
                for (int m = 0; m < NPART - 1; ++m) acc_add(part[m], one[m]);
                any_chi = true;
            }
        }
    }
    if (sums) {
        block_reduce<A>(any_chi, part, red);
        publish_slot<A>(pa, slot, nparts, reinterpret_cast<A *>(red[0]), s_last);
    }
    __syncthreads();   // the stage and the outlet record are complete

    // ---- step n + 1 on the tile, from the stage ----
    const bool near_b = rb.x <= rb.y && tile_near_body(rb, bi0, bj0, FUSED2_W, FUSED2_H, false);
    const StageSrc<P, CONV> src{stage, bi0, bj0, nx, ny};
#pragma unroll
    for (int k = 0; k < NPART - 1; ++k) acc_zero(part[k]);
    any_chi = false;
    pairs = false;
    if constexpr (COLL == VPLBM_COLLISION_MRT) pairs = even_rows && interior && !near_b;
    if (pairs) {
        // the tile away from the body: one pair of x-adjacent nodes per
        // thread, from the stage (aligned where c_ax = 0), to HBM as pairs
        const int ly = tid / (FUSED2_W / 2), px = tid - ly * (FUSED2_W / 2);
        const int k0 = (ly + 1) * F2_RW + F2_X0 + 2 * px;
        float2 f2[NQ];
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
            const S *src = stage + a * F2_RN + k0 - cy_of(a) * F2_RW - cx_of(a);
            f2[a] = cx_of(a) == 0 ? ld_pair_s(src) : ld_two_s(src);
        }
        const int b = (bj0 + ly) * nx + bi0 + 2 * px;
        S *const *dp = reinterpret_cast<S *const *>(pb.dst_plane);
        float ax, ay;
        mrt_dev_lanes<Lane2>(pb, f2, false, 0.f, 0.f, bsb, [&](int a, float2 v) { st_pair(dp[a] + b, v); }, ax, ay);
    } else {
        for (int r = 0; r < F2_ROWS; ++r) {
            const int lx = threadIdx.x, ly = threadIdx.y + r * F2_TY;
            const int i = bi0 + lx, j = bj0 + ly;
            if (i >= nx || j >= ny) continue;
            const int k0 = (ly + 1) * F2_RW + lx + F2_X0;
            const bool plain = interior || (i > 0 && i < nx - 1 && j > 0 && j < ny - 1);
            T f[NQ];
            if (plain) {
    #pragma unroll
                for (int a = 0; a < NQ; ++a) f[a] = ld_stage(stage + a * F2_RN + k0 - cy_of(a) * F2_RW - cx_of(a));
            } else {
    #pragma unroll
                for (int a = 0; a < NQ; ++a) f[a] = pull_edge_src<P>(pb, src, a, i, j);
                if (CONV && i == nx - 1) record_outlet<P>(pb, j, f);
            }
            T dxl = 0, dyl = 0;
            bool chi = false;
            if (near_b) chi = body_chi<P, SHAPE>(pb.body, pb.r2f, bsb, i, j, dxl, dyl);
            T cr = 0, cax = 0, cay = 0;
            chi = node_collide<P, COLL>(pb, bsb, chi, dxl, dyl, i, j, f, nullptr, cr, cax, cay);
            if (sums && chi) {
                T g[NQ];   // pulled again: not kept live across the stores
                if (plain) {
    #pragma unroll
                    for (int a = 0; a < NQ; ++a) g[a] = ld_stage(stage + a * F2_RN + k0 - cy_of(a) * F2_RW - cx_of(a));
                } else {
    #pragma unroll
                    for (int a = 0; a < NQ; ++a) g[a] = pull_edge_src<P>(pb, src, a, i, j);
                }
                V one[NPART - 1];
                solid_terms_from<P>(bsb, g, [&](int a) { return ld_stage(stage + a * F2_RN + k0); }, i, j, (V)cr,
                                    (V)cax, (V)cay, one);
    #pragma unroll
                for (int m = 0; m < NPART - 1; ++m) acc_add(part[m], one[m]);
                any_chi = true;
            }
        }
    }
    if (sums) {
        block_reduce<A>(any_chi, part, red);
        publish_slot<A>(pb, slot, nparts, reinterpret_cast<A *>(red[0]), s_last);
    }
}

// Grid: (tile rows) x (body-block lines + tile columns), or (tile columns) x
// (body-block lines + tile rows) for a lattice of more than 65 535 - lines
// tile columns; programmatic dependent launch as in the one-step kernel.
template <int P, int COLL, int SHAPE, bool CONV>
__device__ __forceinline__ void step2_grid(const Fused2Params &q)
{
    using S = typename Prec<P>::S;
    extern __shared__ __align__(16) unsigned char f2_smem[];
    S *stage = reinterpret_cast<S *>(f2_smem);   // [NQ][F2_RN]
    __shared__ double red[8][NPART];
    __shared__ int s_last;
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int tid = threadIdx.y * F2_TX + threadIdx.x;
    const int nbr = q.a.nbody_rows;
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    const int4 ra = __ldg(reinterpret_cast<const int4 *>(&q.a.bs_in->ilo));
    const int4 rb = __ldg(reinterpret_cast<const int4 *>(&q.b.bs_in->ilo));
    int tx = -1, ty = 0, slot = 0, nparts = 1;
    bool sums = false;
    if ((int)blockIdx.y < nbr) {
        if (b == q.a.nbody) {   // the pose block: poses n + 2, n + 3 for the next launch
            if (tid == 0) advance_two(q.b, q.next0, q.next1);
            return;
        }
        if (b > q.a.nbody) return;
        // union of the two solid-node ranges (ilo > ihi: empty)
        int4 u = ra;
        if (rb.x <= rb.y) {
            if (u.x <= u.y)
                u = make_int4(min(u.x, rb.x), max(u.y, rb.y), min(u.z, rb.z), max(u.w, rb.w));
            else
                u = rb;
        }
        int tx0 = 0, ty0 = 0, rw = 1, nrect = 1;   // no solid node: tile (0, 0) runs the tails
        if (u.x <= u.y) {
            tx0 = u.x / FUSED2_W;
            ty0 = u.z / FUSED2_H;
            rw = u.y / FUSED2_W - tx0 + 1;
            nrect = rw * (u.w / FUSED2_H - ty0 + 1);
        }
        if (b < nrect) {
            tx = tx0 + b % rw;
            ty = ty0 + b / rw;
            sums = true;
            slot = b;
            nparts = nrect;
        }
        if (b == 0 && nrect > q.a.nbody && tid == 0) *q.a.err |= ERR_INTERNAL;
    } else {
        const bool colmajor = (int)gridDim.x == (q.a.ny + FUSED2_H - 1) / FUSED2_H;
        const int lines = gridDim.y - nbr;
        const int ntx = colmajor ? lines : gridDim.x, nty = colmajor ? gridDim.x : lines;
        const int c = colmajor ? blockIdx.y - nbr : blockIdx.x, r = colmajor ? blockIdx.x : blockIdx.y - nbr;
        tx = c == 0 ? 0 : (c == 1 ? ntx - 1 : c - 1);   // edge columns first
        ty = r == 0 ? 0 : (r == 1 ? nty - 1 : r - 1);   // edge rows first
    }
    if (tx >= 0) two_steps<P, COLL, SHAPE, CONV>(q, stage, tx, ty, sums, slot, nparts, ra, rb, red, &s_last);
}

template <int P, int COLL, int SHAPE>
__global__ void __launch_bounds__(F2_NT, 5) vp_mrt_step2(const Fused2Params q)
{
    step2_grid<P, COLL, SHAPE, false>(q);
}

// The same for a lattice with a convective east outlet (any body shape).
template <int P, int COLL>
__global__ void __launch_bounds__(F2_NT, 5) vp_mrt_step2_conv(const Fused2Params q)
{
    step2_grid<P, COLL, SHAPE_ANY, true>(q);
}

__global__ void lookahead_kernel(const StepParams p)
{
    if (threadIdx.x == 0) advance_prescribed(p);
}

template <int P>
cudaError_t launch_p(const Fused2Params &q0, cudaStream_t stream)
{
    Fused2Params q = q0;
    const int nx = q.a.nx, ny = q.a.ny;
    const int ntx = (nx + FUSED2_W - 1) / FUSED2_W, nty = (ny + FUSED2_H - 1) / FUSED2_H;
    // the union of two node ranges one step apart: one node more of radius
    const long long nbody = max_reduction_blocks(nx, ny, q.a.body.radius + 1.0, q.a.body.present, FUSED2_W, FUSED2_H);
    q.a.nbody = (int)nbody;
    // grid lines (rows of a row-major grid, columns of a column-major one)
    // of body blocks; column-major where the tile columns fit the y limit
    const bool colmajor = ntx + (nbody + nty - 1) / nty <= 65535;
    const int line = colmajor ? nty : ntx;
    q.a.nbody_rows = (int)((nbody + 1 + line - 1) / line);   // the body blocks and the pose block
    const size_t smem = (size_t)NQ * F2_RN * sizeof(typename Prec<P>::S);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = colmajor ? dim3(nty, ntx + q.a.nbody_rows) : dim3(ntx, nty + q.a.nbody_rows);
    cfg.blockDim = dim3(F2_TX, F2_TY);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool bgk = q.a.collision == VPLBM_COLLISION_BGK;
    const bool disk = !q.a.body.present || q.a.body.shape == VPLBM_SHAPE_DISK;
    if (q.a.bc[VPLBM_EAST] == VPLBM_BC_CONVECTIVE)
        return bgk ? cudaLaunchKernelEx(&cfg, vp_mrt_step2_conv<P, VPLBM_COLLISION_BGK>, q)
                   : cudaLaunchKernelEx(&cfg, vp_mrt_step2_conv<P, VPLBM_COLLISION_MRT>, q);
    if (bgk)
        return disk ? cudaLaunchKernelEx(&cfg, vp_mrt_step2<P, VPLBM_COLLISION_BGK, VPLBM_SHAPE_DISK>, q)
                    : cudaLaunchKernelEx(&cfg, vp_mrt_step2<P, VPLBM_COLLISION_BGK, SHAPE_ANY>, q);
    return disk ? cudaLaunchKernelEx(&cfg, vp_mrt_step2<P, VPLBM_COLLISION_MRT, VPLBM_SHAPE_DISK>, q)
                : cudaLaunchKernelEx(&cfg, vp_mrt_step2<P, VPLBM_COLLISION_MRT, SHAPE_ANY>, q);
}

}  // namespace

cudaError_t launch_step_fused2(int precision, const Fused2Params &q, cudaStream_t stream)
{
    if (q.a.body.present && q.a.body.motion == VPLBM_MOTION_FREE) return cudaErrorInvalidValue;
    switch (precision) {
    case VPLBM_F32_DEV: return launch_p<VPLBM_F32_DEV>(q, stream);
    case VPLBM_F16_DEV: return launch_p<VPLBM_F16_DEV>(q, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_lookahead(const StepParams &p, cudaStream_t stream)
{
    lookahead_kernel<<<1, 32, 0, stream>>>(p);
    return cudaGetLastError();
}

}  // namespace vplbm
