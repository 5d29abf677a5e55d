// Fused VP-MRT D2Q9 step for sm_103a, and the small kernels around it.
//
// One launch is one time step of Algorithm 1 (Sec. 2.3) for every node:
//   pull-stream the post-collision populations of the previous step
//   (Eq. 18) with the boundary rules of Sec. 3.1/3.2 -> rho, j (Eq. 19)
//   -> chi and u_s from the body pose, in registers (Eq. 2) -> penalized
//   velocity (Eq. 22) -> MRT collision with forcing in moment space
//   (Eqs. 14-17) -> store.  Blocks whose tile meets the disk's bounding box
//   also reduce, in FP64, the penalization reaction and the momentum
//   exchanged through solid/fluid links (Eqs. 25-27); the last of them sums
//   the block partials in a fixed order and one thread advances the body
//   (Eqs. 23-24, RK4), writes the history record and the next pose.
//
// Storage is structure-of-arrays f[a][j][i] with a padded plane stride;
// consecutive threads own consecutive i, so every one of the 9 loads and 9
// stores of a warp is a contiguous 128-byte (FP32) run.  chi is never
// stored.  The collision uses the closed forms of M, M^-1 and M F
// (the rows of Eq. 15 are orthogonal: M^-1 = M^T diag(1/9, 1/36, 1/36,
// 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)).
#include <math.h>

#include "step_scalar.cuh"

namespace vplbm {

const int SHAPES[N_SHAPES][2] = {{128, 2}, {256, 1}, {64, 4}, {32, 8}, {128, 1}, {64, 2}, {32, 4}};

namespace {

// Every member of a batch in one launch: block b runs macro tile b of the
// concatenated macro-tile lists (bl.rows tiles of blockDim.x x blockDim.y
// stacked in y); its member and its macro tile within the member come from
// the tile map (one load), and the member's step parameters are staged in
// shared memory.  The lookup and the staging read only data that no step
// writes, so they run before the wait on the previous step's grid
// (programmatic dependent launch).
template <int P, int COLL>
__global__ void __launch_bounds__(256, 5) vp_mrt_step_batch(const BatchLaunch bl)
{
    __shared__ double red[8][NPART];
    __shared__ float rows[NPART - 1][256];
    __shared__ int s_last;
    __shared__ __align__(16) StepParams sp;
    __shared__ int s_member, s_local;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const int2 ml = __ldg(bl.tile_map + blockIdx.x);
        s_member = ml.x;
        s_local = ml.y;
    }
    __syncthreads();
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(bl.params + s_member);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
    for (int k = tid; k < (int)(sizeof(StepParams) / 4); k += blockDim.x * blockDim.y) dst[k] = src[k];
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const int ntx = (sp.nx + blockDim.x - 1) / blockDim.x;
    const int nty = (sp.ny + blockDim.y - 1) / blockDim.y;
    const int tx = s_local % ntx, ty0 = (s_local / ntx) * bl.rows;
#pragma unroll 1
    for (int r = 0; r < bl.rows && ty0 + r < nty; ++r) scalar_tile<P, COLL, SHAPE_ANY>(sp, tx, ty0 + r, red, rows, &s_last, true);
    if (s_local == 0 && tid == 0 && prescribed_motion(sp)) advance_prescribed(sp);
}

// ---- equilibrium initialisation (Eq. 11) -------------------------------

template <int P>
__global__ void init_equilibrium_kernel(const StepParams p, const double *rho_f, const double *ux_f, const double *uy_f)
{
    using S = typename Prec<P>::S;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    const long long k = (long long)j * p.nx + i;
    const double rho = rho_f ? rho_f[k] : p.rho0;
    const double ux = ux_f ? ux_f[k] : 0.0;
    const double uy = uy_f ? uy_f[k] : 0.0;
    const double u2 = ux * ux + uy * uy;
    S *fout = static_cast<S *>(p.fout);
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
        const double cu = cx_of(a) * ux + cy_of(a) * uy;
        const double poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * u2;
        double val;
        if (Prec<P>::DEV) val = w_of(a) * ((rho - p.rho0) + rho * poly);
        else val = w_of(a) * rho * (1.0 + poly);
        stv(fout + a * p.ps + k, (typename Prec<P>::T)val);
    }
}

// ---- convective outlet: previous values := the state's outlet column -----

template <int P>
__global__ void outlet_reset_kernel(const StepParams p)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.ny) return;
    const S *fin = static_cast<const S *>(p.fin);
    T *out = static_cast<T *>(const_cast<void *>(p.conv_in));
    const long long b = (long long)j * p.nx + p.nx - 1;
    out[outlet_slot(3) * p.ny + j] = ldv(fin + 3 * p.ps + b);
    out[outlet_slot(6) * p.ny + j] = ldv(fin + 6 * p.ps + b);
    out[outlet_slot(7) * p.ny + j] = ldv(fin + 7 * p.ps + b);
}

// ---- macroscopic fields of the current step (Eqs. 19-22) ---------------

template <int P>
__global__ void fields_kernel(const StepParams p, double *rho_o, double *ux_o, double *uy_o)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx || j >= p.ny) return;
    const S *fin = static_cast<const S *>(p.fin);
    T f[NQ];
    pull_all<P>(p, fin, i, j, f);
    double rs = 0, jx = 0, jy = 0;
#pragma unroll
    for (int a = 0; a < NQ; ++a) {
        rs += (double)f[a];
        jx += cx_of(a) * (double)f[a];
        jy += cy_of(a) * (double)f[a];
    }
    const double rho = Prec<P>::DEV ? p.rho0 + rs : rs;
    // chi: the first body whose predicate holds (Eq. 2)
    auto chi_of = [&](const DevBody &body, const BodyState &s) {
        return body.present && (body.shape == VPLBM_SHAPE_ELLIPSE     ? chi_exact_ellipse(i, j, &s, body)
                                : body.shape == VPLBM_SHAPE_RECTANGLE ? chi_exact_rect(i, j, &s, body)
                                                                      : chi_exact(i, j, s.q[0], s.q[1], body.r2));
    };
    BodyState bs = *p.bs_in;
    bool chi = false;
    if (p.nbodies > 1) {
        for (int k = 0; k < p.nbodies && !chi; ++k) {
            bs = p.bs_in[k];
            chi = chi_of(p.views[k].body, bs);
        }
    } else {
        chi = chi_of(p.body, bs);
    }
    double vx = jx / rho + 0.5 * p.gx, vy = jy / rho + 0.5 * p.gy;
    double ax = 0, ay = 0;
    if (chi) {
        const double dx = (double)i - bs.q[0], dy = (double)j - bs.q[1];
        const double usx = bs.v[0] - bs.v[2] * dy, usy = bs.v[1] + bs.v[2] * dx;
        ax = -(vx - usx) / (p.eta + 0.5);
        ay = -(vy - usy) / (p.eta + 0.5);
    }
    const long long k = (long long)j * p.nx + i;
    if (rho_o) rho_o[k] = rho;
    if (ux_o) ux_o[k] = vx + 0.5 * ax;
    if (uy_o) uy_o[k] = vy + 0.5 * ay;
}

}  // namespace

long long max_reduction_blocks(int nx, int ny, double radius, int present, int bx, int by)
{
    if (!present) return 1;
    const long long span = (long long)ceil(2.0 * radius) + 5;
    long long tx = span / bx + 2, ty = span / by + 2;
    const long long gx = (nx + bx - 1) / bx, gy = (ny + by - 1) / by;
    if (tx > gx) tx = gx;
    if (ty > gy) ty = gy;
    return tx * ty;
}

cudaError_t launch_step_batch(int precision, const BatchLaunch &bl, int total_tiles, int bx, int by,
                              cudaStream_t stream)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(total_tiles);
    cfg.blockDim = dim3(bx, by);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const bool bgk = bl.collision == VPLBM_COLLISION_BGK;
    switch (precision) {
    case VPLBM_F32_DEV:
        return bgk ? cudaLaunchKernelEx(&cfg, vp_mrt_step_batch<VPLBM_F32_DEV, VPLBM_COLLISION_BGK>, bl)
                   : cudaLaunchKernelEx(&cfg, vp_mrt_step_batch<VPLBM_F32_DEV, VPLBM_COLLISION_MRT>, bl);
    case VPLBM_F16_DEV:
        return bgk ? cudaLaunchKernelEx(&cfg, vp_mrt_step_batch<VPLBM_F16_DEV, VPLBM_COLLISION_BGK>, bl)
                   : cudaLaunchKernelEx(&cfg, vp_mrt_step_batch<VPLBM_F16_DEV, VPLBM_COLLISION_MRT>, bl);
    case VPLBM_F64:
        return bgk ? cudaLaunchKernelEx(&cfg, vp_mrt_step_batch<VPLBM_F64, VPLBM_COLLISION_BGK>, bl)
                   : cudaLaunchKernelEx(&cfg, vp_mrt_step_batch<VPLBM_F64, VPLBM_COLLISION_MRT>, bl);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(int precision, const StepParams &p, int bx, int by, cudaStream_t stream, int minb)
{
    if (p.nbodies > 1) return launch_step_multi(precision, p, bx, by, stream, minb);
    if (p.body.present && p.body.shape == VPLBM_SHAPE_ELLIPSE)
        return launch_step_ellipse(precision, p, bx, by, stream, minb);
    if (p.body.present && p.body.shape == VPLBM_SHAPE_RECTANGLE)
        return launch_step_rectangle(precision, p, bx, by, stream, minb);
    return launch_step_shape<VPLBM_SHAPE_DISK>(precision, p, bx, by, stream, minb);
}

cudaError_t launch_init_equilibrium(int precision, const StepParams &p, const double *rho_dev,
                                    const double *ux_dev, const double *uy_dev, cudaStream_t stream)
{
    dim3 block(128);
    dim3 grid((p.nx + 127) / 128, p.ny);
    switch (precision) {
    case VPLBM_F64: init_equilibrium_kernel<VPLBM_F64><<<grid, block, 0, stream>>>(p, rho_dev, ux_dev, uy_dev); break;
    case VPLBM_F32_DEV: init_equilibrium_kernel<VPLBM_F32_DEV><<<grid, block, 0, stream>>>(p, rho_dev, ux_dev, uy_dev); break;
    case VPLBM_F16_DEV: init_equilibrium_kernel<VPLBM_F16_DEV><<<grid, block, 0, stream>>>(p, rho_dev, ux_dev, uy_dev); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_outlet_reset(int precision, const StepParams &p, cudaStream_t stream)
{
    const int grid = (p.ny + 127) / 128;
    switch (precision) {
    case VPLBM_F64: outlet_reset_kernel<VPLBM_F64><<<grid, 128, 0, stream>>>(p); break;
    case VPLBM_F32_DEV: outlet_reset_kernel<VPLBM_F32_DEV><<<grid, 128, 0, stream>>>(p); break;
    case VPLBM_F16_DEV: outlet_reset_kernel<VPLBM_F16_DEV><<<grid, 128, 0, stream>>>(p); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fields(int precision, const StepParams &p, double *rho_dev, double *ux_dev,
                          double *uy_dev, cudaStream_t stream)
{
    dim3 block(128);
    dim3 grid((p.nx + 127) / 128, p.ny);
    switch (precision) {
    case VPLBM_F64: fields_kernel<VPLBM_F64><<<grid, block, 0, stream>>>(p, rho_dev, ux_dev, uy_dev); break;
    case VPLBM_F32_DEV: fields_kernel<VPLBM_F32_DEV><<<grid, block, 0, stream>>>(p, rho_dev, ux_dev, uy_dev); break;
    case VPLBM_F16_DEV: fields_kernel<VPLBM_F16_DEV><<<grid, block, 0, stream>>>(p, rho_dev, ux_dev, uy_dev); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace vplbm
