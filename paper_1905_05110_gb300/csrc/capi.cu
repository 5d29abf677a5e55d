// Host runtime behind the C ABI of include/vplbm.h: descriptor checks,
// device memory, CUDA-graph replay of the time loop, host transfers,
// launch-shape autotuning and checkpoints.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "vplbm_ctx.cuh"

using namespace vplbm;

namespace {

thread_local std::string g_error = "no error";

vplbm_status fail(vplbm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_error = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                        \
    do {                                                                                      \
        cudaError_t e_ = (expr);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(VPLBM_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));         \
    } while (0)

constexpr size_t ALIGN = 256;
constexpr int GRAPH_STEPS = 32;   // steps per captured graph (even)
constexpr int MAX_GRID_ROWS = 65535;   // gridDim.y limit of the scalar kernels
constexpr char CKPT_MAGIC[8] = {'V', 'P', 'L', 'B', 'M', 'C', 'K', '3'};

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t elem_size(int precision)
{
    return precision == VPLBM_F64 ? 8 : (precision == VPLBM_F32_DEV ? 4 : 2);
}

double w_host(int a) { return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

// IEEE half <-> double on the host (round to nearest even).
double half_to_double(uint16_t h)
{
    const int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(m | 1024), e - 25);
    return s ? -v : v;
}

uint16_t double_to_half(double x)
{
    // via float, then float -> half with round-to-nearest-even
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t sign = (u >> 16) & 0x8000u;
    u &= 0x7fffffffu;
    if (u >= 0x7f800000u) return (uint16_t)(sign | (u > 0x7f800000u ? 0x7e00u : 0x7c00u));
    if (u >= 0x477ff000u) return (uint16_t)(sign | 0x7c00u);   // overflow to inf
    if (u < 0x38800000u) {                                       // subnormal half
        if (u < 0x33000000u) return (uint16_t)sign;
        const int e = (int)(u >> 23);
        uint32_t m = (u & 0x7fffffu) | 0x800000u;
        const int shift = 126 - e;                                // 14..24
        uint32_t hm = m >> shift;
        const uint32_t rem = m & ((1u << shift) - 1u), half = 1u << (shift - 1);
        if (rem > half || (rem == half && (hm & 1u))) ++hm;
        return (uint16_t)(sign | hm);
    }
    uint32_t hb = ((u >> 13) - (112u << 10));
    const uint32_t rem = u & 0x1fffu;
    if (rem > 0x1000u || (rem == 0x1000u && (hb & 1u))) ++hb;
    return (uint16_t)(sign | hb);
}

}  // namespace

namespace vplbm {
// Error reporting for the other translation units of the library.
vplbm_status report_error(vplbm_status st, const char *msg) { return fail(st, "%s", msg); }
}  // namespace vplbm


namespace {

vplbm_status check_lattice(const vplbm_lattice_desc *lat)
{
    if (!lat) return fail(VPLBM_EINVAL, "lattice descriptor is NULL");
    if (lat->nx < 3 || lat->ny < 3) return fail(VPLBM_EINVAL, "nx and ny must be >= 3 (got %d x %d)", lat->nx, lat->ny);
    if ((long long)lat->nx * lat->ny >= (1LL << 31)) return fail(VPLBM_EINVAL, "lattice too large");
    if (lat->nx > (1 << 22) || lat->ny > 65535) return fail(VPLBM_EINVAL, "nx must be <= 2^22 and ny <= 65535");
    for (int k = 0; k < 9; ++k)
        if (!(lat->s[k] > 0.0 && lat->s[k] < 2.0)) return fail(VPLBM_EINVAL, "relaxation rate s[%d]=%g outside (0,2)", k, lat->s[k]);
    if (!(lat->eta > 0.0) || !isfinite(lat->eta)) return fail(VPLBM_EINVAL, "eta must be > 0");
    if (!(lat->rho0 > 0.0) || !isfinite(lat->rho0)) return fail(VPLBM_EINVAL, "rho0 must be > 0");
    if (!isfinite(lat->gx) || !isfinite(lat->gy)) return fail(VPLBM_EINVAL, "fluid acceleration not finite");
    if (lat->precision < VPLBM_F64 || lat->precision > VPLBM_F16_DEV) return fail(VPLBM_EINVAL, "unknown precision %d", lat->precision);
    if (lat->collision != VPLBM_COLLISION_MRT && lat->collision != VPLBM_COLLISION_BGK)
        return fail(VPLBM_EINVAL, "unknown collision operator %d", lat->collision);
    for (int s = 0; s < 4; ++s) {
        const int k = lat->bc[s].kind;
        if (k < VPLBM_BC_PERIODIC || k > VPLBM_BC_CONVECTIVE) return fail(VPLBM_EINVAL, "edge %d: unknown boundary kind %d", s, k);
        if (k == VPLBM_BC_ZEROGRAD && s >= VPLBM_SOUTH) return fail(VPLBM_EUNSUPPORTED, "zero-gradient is supported on west/east edges only");
        if (k == VPLBM_BC_SYMMETRY && s < VPLBM_SOUTH) return fail(VPLBM_EUNSUPPORTED, "symmetry is supported on south/north edges only");
        if (k == VPLBM_BC_CONVECTIVE && s != VPLBM_EAST) return fail(VPLBM_EUNSUPPORTED, "the convective outlet is supported on the east edge only");
        if (k == VPLBM_BC_CONVECTIVE && !(lat->bc[s].ux >= 0.0 && lat->bc[s].ux < 1e6))
            return fail(VPLBM_EINVAL, "convective velocity (east ux) must be >= 0 and finite");
    }
    if ((lat->bc[VPLBM_WEST].kind == VPLBM_BC_PERIODIC) != (lat->bc[VPLBM_EAST].kind == VPLBM_BC_PERIODIC))
        return fail(VPLBM_EINVAL, "west and east must both be periodic or neither");
    if ((lat->bc[VPLBM_SOUTH].kind == VPLBM_BC_PERIODIC) != (lat->bc[VPLBM_NORTH].kind == VPLBM_BC_PERIODIC))
        return fail(VPLBM_EINVAL, "south and north must both be periodic or neither");
    return VPLBM_OK;
}

vplbm_status check_body(const vplbm_body_desc *b)
{
    if (!b) return VPLBM_OK;
    if (!(b->radius >= 0.0) || b->radius > 1e6) return fail(VPLBM_EINVAL, "radius must be in [0, 1e6]");
    if (b->shape != VPLBM_SHAPE_DISK && b->shape != VPLBM_SHAPE_ELLIPSE && b->shape != VPLBM_SHAPE_RECTANGLE)
        return fail(VPLBM_EINVAL, "unknown shape %d", b->shape);
    if (b->shape != VPLBM_SHAPE_DISK && (!(b->radius > 0.0) || !(b->radius_b > 0.0) || b->radius_b > 1e6))
        return fail(VPLBM_EINVAL, "semi-axes / half-sides must be in (0, 1e6]");
    const double vals[6] = {b->x, b->y, b->theta, b->vx, b->vy, b->omega};
    for (double v : vals)
        if (!isfinite(v) || fabs(v) > 1e7) return fail(VPLBM_EINVAL, "body pose/velocity must be finite and < 1e7");
    if (b->motion < VPLBM_MOTION_FIXED || b->motion > VPLBM_MOTION_FREE) return fail(VPLBM_EINVAL, "unknown motion %d", b->motion);
    if (b->motion == VPLBM_MOTION_IMPOSED && (b->axis < 0 || b->axis > 2)) return fail(VPLBM_EINVAL, "imposed axis must be 0, 1 or 2");
    if (b->motion == VPLBM_MOTION_FREE) {
        if (!(b->mass > 0.0) || !(b->inertia > 0.0)) return fail(VPLBM_EINVAL, "free motion needs mass > 0 and inertia > 0");
        if (b->dof_mask & ~7u) return fail(VPLBM_EINVAL, "dof_mask has bits beyond x|y|theta");
    }
    return VPLBM_OK;
}

void tile_of(int kernel, int bx, int by, int *w, int *h);
long long grid_rows(const vplbm_ctx *c, int bx, int by, int kernel = KERNEL_SCALAR);

// Bodies of a context: nb descriptors (nb = 0: no body); per-body buffers
// have max(nb, 1) slots.
inline int body_slots(int nb) { return nb > 1 ? nb : 1; }

void sizes_for(const vplbm_lattice_desc *lat, const vplbm_body_desc *bodies, int nb, long long cap,
               vplbm_buffer_sizes *s, long long *ps_out, long long *parts_out)
{
    const long long n = (long long)lat->nx * lat->ny;
    const long long ps = (long long)round_up((size_t)n, 128);
    const int slots = body_slots(nb);
    long long parts = 1;   // per body: the largest over the kernels' tilings
    for (int b = 0; b < slots; ++b) {
        const vplbm_body_desc *body = nb > 0 ? &bodies[b] : nullptr;
        const long long m0 = max_reduction_blocks(lat->nx, lat->ny, bounding_radius(body), body != nullptr,
                                                  TMA_TILE_W, TMA_TILE_H);
        if (m0 > parts) parts = m0;
        for (int k = 0; k < N_SHAPES; ++k)
            for (int kern = KERNEL_SCALAR; kern <= KERNEL_TMA; ++kern) {   // every kernel's tiling
                int w, h;
                tile_of(kern, SHAPES[k][0], SHAPES[k][1], &w, &h);
                const long long m = max_reduction_blocks(lat->nx, lat->ny, bounding_radius(body), body != nullptr, w, h);
                if (m > parts) parts = m;
            }
        // the two-step kernel: the union of two consecutive node ranges
        const long long m2 = max_reduction_blocks(lat->nx, lat->ny, bounding_radius(body) + 1.0, body != nullptr,
                                                  FUSED2_W, FUSED2_H);
        if (m2 > parts) parts = m2;
    }
    s->populations = round_up((size_t)(9 * ps) * elem_size(lat->precision), ALIGN);
    // the body states [parity][slot] (one body: two more, the two-step
    // kernel's other pose pair), then (several bodies) the per-body
    // parameter views [parity][body]
    s->body_state = round_up((nb > 1 ? 2 * (size_t)nb : 4) * sizeof(BodyState) +
                                 (nb > 1 ? 2 * (size_t)nb * sizeof(StepParams) : 0),
                             ALIGN);
    // one partials region per body; one body: two (one per step of the
    // two-step kernel)
    s->partials = round_up((size_t)(slots > 2 ? slots : 2) * parts * NPART * sizeof(double), ALIGN);
    s->history = round_up((size_t)slots * cap * sizeof(vplbm_record), ALIGN);
    // FP64 profiles, then their FP32 copies: [side][comp][maxlen] each; then
    // the convective outlet state: [parity][3][ny] 8-byte slots
    s->profiles = round_up((size_t)8 * (lat->nx > lat->ny ? lat->nx : lat->ny) * (sizeof(double) + sizeof(float)), ALIGN) +
                  round_up((size_t)6 * lat->ny * sizeof(double), ALIGN);
    s->control = sizeof(Control);
    if (ps_out) *ps_out = ps;
    if (parts_out) *parts_out = parts;
}

BodyState initial_state(const vplbm_ctx *c, int k)
{
    BodyState s{};
    const bool present = k < c->nbodies;
    if (present) {
        const vplbm_body_desc &b = c->bodies[k];
        s.q[0] = b.x; s.q[1] = b.y; s.q[2] = b.theta;
        s.v[0] = b.vx; s.v[1] = b.vy; s.v[2] = b.omega;
    }
    s.step = 0;
    derive_pose(s, present ? 1 : 0, present ? bounding_radius(&c->bodies[k]) : 0.0, c->nx, c->ny,
                present ? c->bodies[k].shape : VPLBM_SHAPE_DISK);
    return s;
}

StepParams params_for(const vplbm_ctx *c, long long step)
{
    StepParams p = c->base;
    const int par = (int)(step & 1);
    p.fin = c->f[par];
    p.fout = c->f[par ^ 1];
    const int slots = body_slots(c->nbodies);
    p.bs_in = c->bs + par * slots;
    p.bs_out = c->bs + (par ^ 1) * slots;
    p.views = c->views ? c->views + (size_t)par * c->nbodies : nullptr;
    set_planes(p, (int)elem_size(c->precision));
    double *ob = static_cast<double *>(c->outlet);
    p.conv_in = ob + (size_t)par * 3 * c->ny;
    p.conv_out = ob + (size_t)(par ^ 1) * 3 * c->ny;
    return p;
}

// One time step with the context's kernel choice.
cudaError_t launch_one(const vplbm_ctx *c, long long step, cudaStream_t stream)
{
    const StepParams p = params_for(c, step);
    if (c->kernel == KERNEL_TMA) return launch_step_tma(c->precision, p, c->tmap[step & 1], c->tma_grid, stream);
    if (c->kernel == KERNEL_PAIR) return launch_step_pair(c->precision, p, c->bx, c->by, stream);
    // a single step of a two-step choice runs the 40-register scalar kernel
    const int minb = c->kernel == KERNEL_SCALAR_40 || c->kernel == KERNEL_FUSED2 ? 6 : c->kernel == KERNEL_SCALAR_48 ? 5 : 4;
    return launch_step(c->precision, p, c->bx, c->by, stream, minb);
}

// Launch L of a run of two-step launches that starts at a step of parity P
// with the state in f[P] and poses n, n + 1 in bs[P], bs[P ^ 1]: even
// launches go f[P] -> f[P ^ 1] and take their poses from that pair of
// slots, writing the next pair to bs[2 + P], bs[2 + (P ^ 1)]; odd launches
// go back.  After an even number of launches the state, pose and lookahead
// pose are where single steps of the same parity expect them (a two-step
// launch advances the step by two, the buffers by one, so runs come in
// pairs).
cudaError_t launch_two(const vplbm_ctx *c, int L, int P, cudaStream_t stream)
{
    const int odd = L & 1, src = P ^ odd;
    Fused2Params q;
    q.a = params_for(c, 0);
    q.b = params_for(c, 1);
    const int es = (int)elem_size(c->precision);
    q.a.fin = c->f[src];
    q.a.fout = c->f[src ^ 1];
    set_planes(q.a, es);
    q.b.fin = c->f[src ^ 1];
    q.b.fout = c->f[src ^ 1];
    set_planes(q.b, es);
    BodyState *cur = c->bs + (odd ? 2 : 0), *nxt = c->bs + (odd ? 0 : 2);
    q.a.bs_in = cur + P;
    q.b.bs_in = cur + (P ^ 1);
    q.a.bs_out = q.b.bs_out = nullptr;
    q.next0 = nxt + P;
    q.next1 = nxt + (P ^ 1);
    q.b.partials = c->partials + (size_t)c->max_parts * NPART;
    q.b.ticket = &c->ctrl->ticket[1];
    // convective outlet: step n reads the record of step n - 1 and step
    // n + 1 writes the one of step n + 1, alternating between the two slots
    // with the launch (the same slot would race with other blocks' reads);
    // step n's own record stays in each block's shared memory
    double *ob = static_cast<double *>(c->outlet);
    q.a.conv_in = q.b.conv_in = ob + (size_t)src * 3 * c->ny;
    q.a.conv_out = q.b.conv_out = ob + (size_t)(src ^ 1) * 3 * c->ny;
    return launch_step_fused2(c->precision, q, stream);
}

// Why the two-step kernel cannot run this context (nullptr: it can).
const char *fused2_refusal(const vplbm_ctx *c)
{
    if (c->precision == VPLBM_F64) return "the two-step kernel needs FP32 or FP16 storage";
    if (c->nbodies > 1) return "the two-step kernel takes one body";
    if (c->has_body && c->body_desc.motion == VPLBM_MOTION_FREE)
        return "the two-step kernel needs a body on a prescribed path (fixed or imposed)";
    if (max_reduction_blocks(c->nx, c->ny, c->has_body ? bounding_radius(&c->body_desc) + 1.0 : 0.0, c->has_body,
                             FUSED2_W, FUSED2_H) > c->max_parts)
        return "the two-step kernel needs more reduction scratch than allocated";
    return nullptr;
}

// Why the node-pair kernel cannot run this context (nullptr: it can).
const char *pair_refusal(const vplbm_ctx *c)
{
    if (c->precision == VPLBM_F64) return "the node-pair kernel needs FP32 or FP16 storage";
    if (c->collision != VPLBM_COLLISION_MRT) return "the node-pair kernel runs the MRT collision";
    if (c->nbodies > 1) return "the node-pair kernel takes one body";
    if (c->nx & 1) return "the node-pair kernel needs an even nx";
    return nullptr;
}

// Steps of one captured graph, launches per graph.
int graph_launches(const vplbm_ctx *c) { return c->kernel == KERNEL_FUSED2 ? 1 + GRAPH_STEPS / 2 : GRAPH_STEPS; }


// Reduction tile of a launch choice: the block for the scalar kernels, the
// TMA kernel's fixed tile otherwise.
// Rows of a scalar kernel's grid for blocks of bx x by: one row of blocks
// per row of tiles plus the rows of the body blocks.
long long grid_rows(const vplbm_ctx *c, int bx, int by, int kernel)
{
    if (kernel == KERNEL_PAIR)
        return pair_grid_rows(c->nx, c->ny, c->has_body ? bounding_radius(&c->body_desc) : 0.0, c->has_body, bx, by);
    const long long ntx = (c->nx + bx - 1) / bx, nty = (c->ny + by - 1) / by;
    long long nbody = 0;
    for (int k = 0; k < body_slots(c->nbodies); ++k) {
        const bool present = k < c->nbodies;
        nbody += max_reduction_blocks(c->nx, c->ny, present ? bounding_radius(&c->bodies[k]) : 0.0, present, bx, by);
    }
    return nty + (nbody + ntx - 1) / ntx;
}

void tile_of(int kernel, int bx, int by, int *w, int *h)
{
    if (kernel == KERNEL_TMA) { *w = TMA_TILE_W; *h = TMA_TILE_H; }
    else { *w = bx; *h = by; }   // the scalar kernels
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor maps and grid of the TMA-staged kernel, when the lattice allows
// it (row pitch a multiple of 16 bytes, lattice at least one box wide).
void setup_tma(vplbm_ctx *c)
{
    c->tma_ok = false;
    if (c->precision != VPLBM_F32_DEV && c->precision != VPLBM_F16_DEV) return;
    if (c->nbodies > 1) return;   // the TMA-staged kernel takes one body
    if (c->collision != VPLBM_COLLISION_MRT) return;
    const int es = (int)elem_size(c->precision);
    const int halo = tma_halo(c->precision);
    const int boxw = TMA_TILE_W + 2 * halo;
    if ((c->nx * es) % 16 != 0 || c->nx < boxw || c->ny < TMA_BOX_H + 2) return;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        (void)cudaGetLastError();
        return;
    }
    EncodeTiledFn encode = (EncodeTiledFn)fn;
    const cuuint64_t dims[3] = {(cuuint64_t)c->nx, (cuuint64_t)c->ny, 9};
    const cuuint64_t strides[2] = {(cuuint64_t)c->nx * es, (cuuint64_t)c->ps * es};
    const cuuint32_t box[3] = {(cuuint32_t)boxw, (cuuint32_t)TMA_BOX_H, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        c->precision == VPLBM_F32_DEV ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    for (int b = 0; b < 2; ++b) {
        CUresult r = encode(&c->tmap[b], dt, 3, c->f[b], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return;
    }
    int per_sm = 0, nsm = 0;
    if (tma_prepare(c->precision, &per_sm) != cudaSuccess || per_sm < 1 ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        (void)cudaGetLastError();
        return;
    }
    c->tma_grid = per_sm * nsm;
    c->tma_ok = true;
}

// Reset step counter, body state and control word (after a new state).
vplbm_status reset_run(vplbm_ctx *c)
{
    if (c->base.bc[VPLBM_EAST] == VPLBM_BC_CONVECTIVE) CUDA_TRY(launch_outlet_reset(c->precision, params_for(c, 0), c->stream));
    // [parity][body]; one body: also the two-step kernel's other pose pair
    const int slots = body_slots(c->nbodies);
    const int nstates = c->nbodies > 1 ? 2 * slots : 4;
    BodyState s[2 * VPLBM_MAX_BODIES];
    for (int m = 0; m < nstates; ++m) s[m] = initial_state(c, m % slots);
    CUDA_TRY(cudaMemcpyAsync(c->bs, s, nstates * sizeof(BodyState), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->ctrl, 0, sizeof(Control), c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->nstep = 0;
    return VPLBM_OK;
}

}  // namespace

namespace vplbm {
// Body constants of a launch's parameters from the public descriptors
// (also used by the allocation-free entry point).
void fill_dev_body(StepParams &p, const vplbm_lattice_desc *lat, const vplbm_body_desc *body)
{
    DevBody &b = p.body;
    memset(&b, 0, sizeof b);
    b.present = body ? 1 : 0;
    if (!body) return;
    b.motion = body->motion;
    b.axis = body->axis;
    b.dof_mask = body->dof_mask;
    b.radius = bounding_radius(body);
    b.r2 = body->radius * body->radius;
    b.shape = body->shape;
    // FP32 predicate b^2 u^2 + a^2 v^2 <= a^2 b^2 of both shapes (disk: a = b)
    const double ra = body->radius, rb = body->shape == VPLBM_SHAPE_DISK ? body->radius : body->radius_b;
    b.a2 = ra * ra;
    b.b2 = rb * rb;
    b.ab2 = b.a2 * b.b2;
    b.a2f = (float)b.a2; b.b2f = (float)b.b2; b.ab2f = (float)b.ab2;
    // its FP32 error stays below ~1e-6 a^2 b^2 (max / min semi-axis); 100x margin
    const double ratio = ra > 0.0 && rb > 0.0 ? fmax(ra, rb) / fmin(ra, rb) : 1.0;
    b.bandf = (float)(1e-4 * b.ab2 * ratio + 1e-5);
    // rectangle: |u| <= a, |v| <= b; the FP32 error of u, v stays below
    // ~3e-7 of the bounding radius, 30x margin
    b.ra = ra;
    b.rb = rb;
    b.raf = (float)ra;
    b.rbf = (float)rb;
    b.bandr = (float)(1e-5 * bounding_radius(body) + 1e-5);
    p.r2f = (float)b.r2;
    b.r2f = p.r2f;
    b.amp = body->amp;
    b.freq = body->freq;
    b.phase = body->phase;
    const double q0[3] = {body->x, body->y, body->theta};
    b.q_center = body->motion == VPLBM_MOTION_IMPOSED ? q0[body->axis] - body->amp * sin(body->phase) : 0.0;
    b.mass = body->mass;
    b.inertia = body->inertia;
    b.inv_mass = body->mass > 0.0 ? 1.0 / body->mass : 0.0;
    b.inv_inertia = body->inertia > 0.0 ? 1.0 / body->inertia : 0.0;
    for (int d = 0; d < 3; ++d) {
        b.damp[d] = body->damp[d];
        b.stiff[d] = body->stiff[d];
        b.q0[d] = body->q0[d];
        b.f_ext[d] = body->f_ext[d];
    }
    b.qref = 0.5 * lat->rho0 * body->d_ref * body->u_ref * body->u_ref;
    b.inv_qref = b.qref > 0.0 ? 1.0 / b.qref : 0.0;
}
}  // namespace vplbm

namespace {

vplbm_status setup(vplbm_ctx *c, const vplbm_lattice_desc *lat, const vplbm_body_desc *bodies, int nb,
                   long long cap, void *stream)
{
    const vplbm_body_desc *body = nb > 0 ? &bodies[0] : nullptr;
    c->stream = (cudaStream_t)stream;
    CUDA_TRY(cudaGetDevice(&c->device));
    CUDA_TRY(cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking));
    c->precision = lat->precision;
    c->collision = lat->collision;
    c->nx = lat->nx;
    c->ny = lat->ny;
    c->hist_cap = cap;
    c->has_body = body != nullptr;
    if (body) c->body_desc = *body;
    c->nbodies = nb;
    for (int k = 0; k < nb; ++k) c->bodies[k] = bodies[k];

    StepParams &p = c->base;
    p.nx = lat->nx;
    p.collision = lat->collision;
    p.ny = lat->ny;
    p.ps = c->ps;
    for (int k = 0; k < 9; ++k) p.s[k] = lat->s[k];
    p.eta = lat->eta;
    p.pen_k = 1.0 / (lat->eta + 0.5);
    p.rho0 = lat->rho0;
    p.gx = lat->gx;
    p.gy = lat->gy;
    for (int k = 0; k < 9; ++k) p.sf[k] = (float)lat->s[k];
    p.rho0f = (float)lat->rho0;
    p.gxf = (float)lat->gx;
    p.gyf = (float)lat->gy;
    p.pen_kf = (float)p.pen_k;
    fold_consts(p.pc, lat->s, lat->gx, lat->gy);
    fold_consts(p.pcd, lat->s, lat->gx, lat->gy);
    // wall velocity profiles: [side][comp][maxlen]
    const int maxlen = lat->nx > lat->ny ? lat->nx : lat->ny;
    const size_t nprof = (size_t)8 * maxlen;
    std::vector<double> prof(nprof, 0.0);
    std::vector<float> proff(nprof, 0.f);
    float *proff_dev = reinterpret_cast<float *>(c->prof + nprof);
    for (int s = 0; s < 4; ++s) {
        p.bc[s] = lat->bc[s].kind;
        p.wall_u0[s][0] = lat->bc[s].ux;
        p.wall_u0[s][1] = lat->bc[s].uy;
        p.wall_u0f[s][0] = (float)lat->bc[s].ux;
        p.wall_u0f[s][1] = (float)lat->bc[s].uy;
        const int len = s < 2 ? lat->ny : lat->nx;
        const double *src[2] = {lat->bc[s].ux_profile, lat->bc[s].uy_profile};
        for (int comp = 0; comp < 2; ++comp) {
            p.wall_prof[s][comp] = nullptr;
            p.wall_proff[s][comp] = nullptr;
            if (src[comp] && lat->bc[s].kind == VPLBM_BC_VELOCITY) {
                const size_t off = (size_t)(s * 2 + comp) * maxlen;
                for (int k = 0; k < len; ++k) {
                    if (!isfinite(src[comp][k])) return fail(VPLBM_EINVAL, "edge %d: wall velocity not finite", s);
                    prof[off + k] = src[comp][k];
                    proff[off + k] = (float)src[comp][k];
                }
                p.wall_prof[s][comp] = c->prof + off;
                p.wall_proff[s][comp] = proff_dev + off;
            }
        }
    }
    CUDA_TRY(cudaMemcpyAsync(c->prof, prof.data(), nprof * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->outlet = reinterpret_cast<char *>(c->prof) + round_up(nprof * (sizeof(double) + sizeof(float)), ALIGN);
    CUDA_TRY(cudaMemsetAsync(c->outlet, 0, (size_t)6 * lat->ny * sizeof(double), c->stream));
    {
        const double U = lat->bc[VPLBM_EAST].kind == VPLBM_BC_CONVECTIVE ? lat->bc[VPLBM_EAST].ux : 0.0;
        p.conv_k1 = 1.0 / (1.0 + U);
        p.conv_k2 = U / (1.0 + U);
        p.conv_k1f = (float)p.conv_k1;
        p.conv_k2f = (float)p.conv_k2;
    }
    CUDA_TRY(cudaMemcpyAsync(proff_dev, proff.data(), nprof * sizeof(float), cudaMemcpyHostToDevice, c->stream));

    fill_dev_body(p, lat, body);
    p.partials = c->partials;
    p.max_parts = c->max_parts;
    p.ticket = &c->ctrl->ticket[0];
    p.err = &c->ctrl->err;
    p.hist = c->hist;
    p.hist_cap = cap;
    p.nbodies = nb;
    for (int k = 0; k < nb; ++k) p.body_radius[k] = bounding_radius(&bodies[k]);
    if (nb > 1) {
        // per-body views of each parity's parameters
        std::vector<StepParams> views((size_t)2 * nb);
        for (int par = 0; par < 2; ++par) {
            const StepParams q = params_for(c, par);
            for (int k = 0; k < nb; ++k) {
                StepParams &w = views[(size_t)par * nb + k];
                w = q;
                fill_dev_body(w, lat, &bodies[k]);
                w.bs_in = q.bs_in + k;
                w.bs_out = q.bs_out + k;
                w.partials = c->partials + (size_t)k * c->max_parts * NPART;
                w.ticket = &c->ctrl->ticket[k];
                w.hist = c->hist + (size_t)k * cap;
                w.views = nullptr;
                w.nbodies = 1;
            }
        }
        CUDA_TRY(cudaMemcpyAsync(c->views, views.data(), views.size() * sizeof(StepParams), cudaMemcpyHostToDevice,
                                 c->stream));
    }

    setup_tma(c);
    // default: the scalar kernel sized for 6 blocks of 256 threads per SM
    // (FP32 / FP16: no spills at 40 registers), 4 for the FP64 one
    c->kernel = c->precision == VPLBM_F64 ? KERNEL_SCALAR : KERNEL_SCALAR_40;
    c->bx = 256;
    c->by = 1;
    // a lattice too tall for 256 x 1 blocks (grid rows <= 65535) takes
    // taller blocks; 32 x 8 fits every lattice check_lattice accepts
    static const int taller[3][2] = {{128, 2}, {64, 4}, {32, 8}};
    for (int k = 0; k < 3 && grid_rows(c, c->bx, c->by) > MAX_GRID_ROWS; ++k) {
        c->bx = taller[k][0];
        c->by = taller[k][1];
    }
    // populations at rest
    StepParams q = params_for(c, 0);
    q.fout = c->f[0];
    CUDA_TRY(launch_init_equilibrium(c->precision, q, nullptr, nullptr, nullptr, c->stream));
    CUDA_TRY(cudaMemsetAsync(c->hist, 0, (size_t)body_slots(nb) * cap * sizeof(vplbm_record), c->stream));
    return reset_run(c);
}

vplbm_status create_impl(const vplbm_lattice_desc *lat, const vplbm_body_desc *bodies, int nb, long long cap,
                         void *stream, const vplbm_buffers *user, vplbm_ctx **out)
{
    if (!out) return fail(VPLBM_EINVAL, "out pointer is NULL");
    *out = nullptr;
    vplbm_status st = check_lattice(lat);
    if (st != VPLBM_OK) return st;
    if (nb < 0 || nb > VPLBM_MAX_BODIES || (nb > 0 && !bodies))
        return fail(VPLBM_EINVAL, "number of bodies must be in [1, %d] with a non-NULL array", VPLBM_MAX_BODIES);
    for (int k = 0; k < nb; ++k) {
        st = check_body(&bodies[k]);
        if (st != VPLBM_OK) return st;
    }
    if (nb > 1 && user) return fail(VPLBM_EUNSUPPORTED, "several bodies need library-allocated memory");
    if (cap < 1) return fail(VPLBM_EINVAL, "history capacity must be >= 1");
    vplbm_buffer_sizes sz;
    long long ps = 0, parts = 0;
    sizes_for(lat, bodies, nb, cap, &sz, &ps, &parts);

    vplbm_ctx *c = new (std::nothrow) vplbm_ctx();
    if (!c) return fail(VPLBM_ENOMEM, "host allocation failed");
    c->ps = ps;
    c->pop_bytes = sz.populations;
    c->max_parts = parts;
    if (user) {
        const void *ptrs[7] = {user->populations_dev[0], user->populations_dev[1], user->body_state_dev,
                               user->partials_dev, user->history_dev, user->profiles_dev, user->control_dev};
        for (const void *q : ptrs)
            if (!q || ((uintptr_t)q % ALIGN)) {
                delete c;
                return fail(VPLBM_EINVAL, "caller buffers must be non-NULL and 256-byte aligned");
            }
        c->f[0] = user->populations_dev[0];
        c->f[1] = user->populations_dev[1];
        c->bs = (BodyState *)user->body_state_dev;
        c->partials = (double *)user->partials_dev;
        c->hist = (vplbm_record *)user->history_dev;
        c->prof = (double *)user->profiles_dev;
        c->ctrl = (Control *)user->control_dev;
    } else {
        const size_t total = 2 * sz.populations + sz.body_state + sz.partials + sz.history + sz.profiles + sz.control;
        cudaError_t e = cudaMalloc(&c->owned, total);
        if (e != cudaSuccess) {
            delete c;
            (void)cudaGetLastError();
            return fail(VPLBM_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", total, cudaGetErrorString(e));
        }
        char *base = (char *)c->owned;
        c->f[0] = base; base += sz.populations;
        c->f[1] = base; base += sz.populations;
        c->bs = (BodyState *)base;
        if (nb > 1) c->views = reinterpret_cast<StepParams *>(base + 2 * (size_t)nb * sizeof(BodyState));
        base += sz.body_state;
        c->partials = (double *)base; base += sz.partials;
        c->hist = (vplbm_record *)base; base += sz.history;
        c->prof = (double *)base; base += sz.profiles;
        c->ctrl = (Control *)base;
    }
    st = setup(c, lat, bodies, nb, cap, stream);
    if (st != VPLBM_OK) {
        vplbm_destroy(c);
        return st;
    }
    *out = c;
    return VPLBM_OK;
}

vplbm_status ensure_graph(vplbm_ctx *c)
{
    if (c->graph && c->graph_kernel == c->kernel && c->graph_bx == c->bx && c->graph_by == c->by) return VPLBM_OK;
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
    CUDA_TRY(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
    cudaError_t err = cudaSuccess;
    if (c->kernel == KERNEL_FUSED2) {
        // pose n + 1 ahead, then GRAPH_STEPS / 2 (even) two-step launches
        err = launch_lookahead(params_for(c, 0), c->capture);
        for (int L = 0; L < GRAPH_STEPS / 2 && err == cudaSuccess; ++L) err = launch_two(c, L, 0, c->capture);
    } else {
        for (int k = 0; k < GRAPH_STEPS && err == cudaSuccess; ++k) err = launch_one(c, k, c->capture);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->capture, &g);
    if (err != cudaSuccess || e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return fail(VPLBM_ECUDA, "graph capture failed: %s", cudaGetErrorString(err != cudaSuccess ? err : e2));
    }
    cudaError_t e3 = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) return fail(VPLBM_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e3));
    c->graph_kernel = c->kernel;
    c->graph_bx = c->bx;
    c->graph_by = c->by;
    return VPLBM_OK;
}

// One single step on the context's kernel choice (the 40-register scalar
// kernel for a two-step choice).
vplbm_status step_one(vplbm_ctx *c)
{
    CUDA_TRY(launch_one(c, c->nstep, c->stream));
    c->kcount[c->kernel == KERNEL_TMA ? VPLBM_LAUNCH_TMA : VPLBM_LAUNCH_ONE_STEP] += 1;
    c->nstep += 1;
    c->launches += 1;
    return VPLBM_OK;
}

// 4 * pairs steps as 2 * pairs two-step launches from the current step
// (either parity), after a lookahead launch that computes pose n + 1.
vplbm_status step_pairs(vplbm_ctx *c, long long pairs)
{
    const int P = (int)(c->nstep & 1);
    CUDA_TRY(launch_lookahead(params_for(c, c->nstep), c->stream));
    for (long long L = 0; L < 2 * pairs; ++L) CUDA_TRY(launch_two(c, (int)(L & 1), P, c->stream));
    c->kcount[VPLBM_LAUNCH_LOOKAHEAD] += 1;
    c->kcount[VPLBM_LAUNCH_TWO_STEP] += 2 * pairs;
    c->nstep += 4 * pairs;
    c->launches += 1 + 2 * pairs;
    return VPLBM_OK;
}

// The time loop.  Graphs of GRAPH_STEPS steps from even steps; with the
// two-step kernel, shorter runs (and runs from an odd step that a graph
// cannot take) go as pairs of two-step launches, so every run of 4 or more
// steps is made of two-step launches but for at most 3 single steps at its
// end (and one at its start, from an odd step, before a graph).
vplbm_status step_impl(vplbm_ctx *c, long long n)
{
    const bool two = c->kernel == KERNEL_FUSED2;
    while (n > 0) {
        vplbm_status st = VPLBM_OK;
        if ((c->nstep & 1) == 0 && n >= GRAPH_STEPS) {
            st = ensure_graph(c);
            if (st != VPLBM_OK) return st;
            CUDA_TRY(cudaGraphLaunch(c->graph, c->stream));
            c->nstep += GRAPH_STEPS;
            c->launches += graph_launches(c);
            if (two) {
                c->kcount[VPLBM_LAUNCH_LOOKAHEAD] += 1;
                c->kcount[VPLBM_LAUNCH_TWO_STEP] += GRAPH_STEPS / 2;
            } else {
                c->kcount[c->kernel == KERNEL_TMA ? VPLBM_LAUNCH_TMA : VPLBM_LAUNCH_ONE_STEP] += GRAPH_STEPS;
            }
            n -= GRAPH_STEPS;
            continue;
        }
        if (two && n >= 4 && !((c->nstep & 1) && n > GRAPH_STEPS)) {
            const long long pairs = (n < GRAPH_STEPS ? n : GRAPH_STEPS) / 4;
            st = step_pairs(c, pairs);
            n -= 4 * pairs;
        } else {
            st = step_one(c);
            n -= 1;
        }
        if (st != VPLBM_OK) return st;
    }
    return VPLBM_OK;
}

vplbm_status read_error(vplbm_ctx *c)
{
    Control ctl;
    CUDA_TRY(cudaMemcpyAsync(&ctl, c->ctrl, sizeof ctl, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (ctl.err & ERR_NONFINITE) return fail(VPLBM_ENONFINITE, "a density became non-positive or non-finite");
    if (ctl.err & ERR_INTERNAL) return fail(VPLBM_ECUDA, "internal reduction capacity exceeded");
    if (ctl.err & ERR_TIMEOUT) return fail(VPLBM_ETIMEOUT, "a bounded wait for a tensor copy gave up");
    return VPLBM_OK;
}

// Host copy of the stored populations <-> full f in FP64.
void stored_to_full(const vplbm_ctx *c, const void *raw, double *f)
{
    const long long n = (long long)c->nx * c->ny;
    const double rho0 = c->base.rho0;
    for (int a = 0; a < 9; ++a) {
        const double base = c->precision == VPLBM_F64 ? 0.0 : w_host(a) * rho0;
        for (long long k = 0; k < n; ++k) {
            const long long idx = a * c->ps + k;
            double v;
            if (c->precision == VPLBM_F64) v = ((const double *)raw)[idx];
            else if (c->precision == VPLBM_F32_DEV) v = (double)((const float *)raw)[idx];
            else v = half_to_double(((const uint16_t *)raw)[idx]);
            f[a * n + k] = v + base;
        }
    }
}

void full_to_stored(const vplbm_ctx *c, const double *f, void *raw)
{
    const long long n = (long long)c->nx * c->ny;
    const double rho0 = c->base.rho0;
    for (int a = 0; a < 9; ++a) {
        const double base = c->precision == VPLBM_F64 ? 0.0 : w_host(a) * rho0;
        for (long long k = 0; k < n; ++k) {
            const long long idx = a * c->ps + k;
            const double v = f[a * n + k] - base;
            if (c->precision == VPLBM_F64) ((double *)raw)[idx] = v;
            else if (c->precision == VPLBM_F32_DEV) ((float *)raw)[idx] = (float)v;
            else ((uint16_t *)raw)[idx] = double_to_half(v);
        }
    }
}

// Checkpoint layout: header, the body states of the current parity
// (extra_bodies + 1), the stored populations, the history rings
// ([body][hist_cap]), the outlet state.
struct CkptHeader {
    char magic[8];
    int nx, ny, precision, extra_bodies;
    long long ps, nstep, hist_cap, launches;
};

}  // namespace

namespace vplbm {
StepParams ctx_params(const vplbm_ctx *c, long long step) { return params_for(c, step); }
cudaError_t ctx_launch(const vplbm_ctx *c, long long step, cudaStream_t stream) { return launch_one(c, step, stream); }
vplbm_status ctx_read_error(vplbm_ctx *c) { return read_error(c); }
}  // namespace vplbm

// ---------------------------------------------------------------- C ABI

extern "C" {

const char *vplbm_last_error(void) { return g_error.c_str(); }

const char *vplbm_version(void) { return "vplbm 0.1.0 (sm_103a)"; }

vplbm_status vplbm_buffer_sizes_for(const vplbm_lattice_desc *lat, const vplbm_body_desc *body,
                                    long long history_capacity, vplbm_buffer_sizes *out)
{
    if (!out) return fail(VPLBM_EINVAL, "out pointer is NULL");
    vplbm_status st = check_lattice(lat);
    if (st != VPLBM_OK) return st;
    st = check_body(body);
    if (st != VPLBM_OK) return st;
    if (history_capacity < 1) return fail(VPLBM_EINVAL, "history capacity must be >= 1");
    sizes_for(lat, body, body ? 1 : 0, history_capacity, out, nullptr, nullptr);
    return VPLBM_OK;
}

vplbm_status vplbm_create(const vplbm_lattice_desc *lat, const vplbm_body_desc *body,
                          long long history_capacity, void *cuda_stream, vplbm_ctx **out)
{
    try {
        return create_impl(lat, body, body ? 1 : 0, history_capacity, cuda_stream, nullptr, out);
    } catch (...) {
        return fail(VPLBM_ENOMEM, "host allocation failed");
    }
}

vplbm_status vplbm_create_with_buffers(const vplbm_lattice_desc *lat, const vplbm_body_desc *body,
                                       long long history_capacity, void *cuda_stream,
                                       const vplbm_buffers *buffers, vplbm_ctx **out)
{
    if (!buffers) return fail(VPLBM_EINVAL, "buffers is NULL");
    try {
        return create_impl(lat, body, body ? 1 : 0, history_capacity, cuda_stream, buffers, out);
    } catch (...) {
        return fail(VPLBM_ENOMEM, "host allocation failed");
    }
}

vplbm_status vplbm_create_bodies(const vplbm_lattice_desc *lat, const vplbm_body_desc *bodies, int nbodies,
                                 long long history_capacity, void *cuda_stream, vplbm_ctx **out)
{
    if (out) *out = nullptr;
    if (nbodies < 1 || nbodies > VPLBM_MAX_BODIES || !bodies)
        return fail(VPLBM_EINVAL, "number of bodies must be in [1, %d] with a non-NULL array", VPLBM_MAX_BODIES);
    try {
        return create_impl(lat, bodies, nbodies, history_capacity, cuda_stream, nullptr, out);
    } catch (...) {
        return fail(VPLBM_ENOMEM, "host allocation failed");
    }
}

void vplbm_destroy(vplbm_ctx *c)
{
    if (!c) return;
    if (c->stream || c->owned) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->capture) cudaStreamDestroy(c->capture);
    if (c->owned) cudaFree(c->owned);
    if (c->adj_ws) cudaFree(c->adj_ws);
    delete c;
}

// Device address of a page-locked, device-mapped host buffer (the kernels
// then read or write it in place over the CPU-GPU link); null for pageable
// memory, which is staged through device memory instead.
void *mapped_host(const void *host)
{
    if (!host) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
        cudaGetLastError();   // an unknown pointer: pageable
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

vplbm_status vplbm_init_equilibrium(vplbm_ctx *c, const double *rho, const double *ux, const double *uy)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    const size_t n = (size_t)c->nx * c->ny;
    double *tmp = nullptr;
    double *d[3] = {nullptr, nullptr, nullptr};
    const double *h[3] = {rho, ux, uy};
    int nf = 0;
    for (int m = 0; m < 3; ++m) {
        d[m] = static_cast<double *>(mapped_host(h[m]));
        if (h[m] && !d[m]) ++nf;
    }
    if (nf) CUDA_TRY(cudaMallocAsync((void **)&tmp, nf * n * sizeof(double), c->stream));
    int k = 0;
    for (int m = 0; m < 3; ++m)
        if (h[m] && !d[m]) {
            d[m] = tmp + k++ * n;
            CUDA_TRY(cudaMemcpyAsync(d[m], h[m], n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        }
    StepParams p = params_for(c, 0);
    p.fout = c->f[0];
    CUDA_TRY(launch_init_equilibrium(c->precision, p, d[0], d[1], d[2], c->stream));
    if (tmp) CUDA_TRY(cudaFreeAsync(tmp, c->stream));
    return reset_run(c);
}

vplbm_status vplbm_set_populations(vplbm_ctx *c, const double *f)
{
    if (!c || !f) return fail(VPLBM_EINVAL, "NULL argument");
    try {
        std::vector<char> raw(c->pop_bytes, 0);
        full_to_stored(c, f, raw.data());
        CUDA_TRY(cudaMemcpyAsync(c->f[0], raw.data(), c->pop_bytes, cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    } catch (const std::bad_alloc &) {
        return fail(VPLBM_ENOMEM, "host allocation failed");
    }
    return reset_run(c);
}

vplbm_status vplbm_step(vplbm_ctx *c, long long nsteps)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    if (nsteps < 0) return fail(VPLBM_EINVAL, "nsteps must be >= 0");
    return step_impl(c, nsteps);
}

vplbm_status vplbm_sync(vplbm_ctx *c)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return read_error(c);
}

vplbm_status vplbm_get_populations(vplbm_ctx *c, double *f)
{
    if (!c || !f) return fail(VPLBM_EINVAL, "NULL argument");
    try {
        std::vector<char> raw(c->pop_bytes);
        CUDA_TRY(cudaMemcpyAsync(raw.data(), c->f[c->nstep & 1], c->pop_bytes, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        stored_to_full(c, raw.data(), f);
    } catch (const std::bad_alloc &) {
        return fail(VPLBM_ENOMEM, "host allocation failed");
    }
    return read_error(c);
}

vplbm_status vplbm_get_fields_dev(vplbm_ctx *c, double *rho_dev, double *ux_dev, double *uy_dev)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    CUDA_TRY(launch_fields(c->precision, params_for(c, c->nstep), rho_dev, ux_dev, uy_dev, c->stream));
    return VPLBM_OK;
}

vplbm_status vplbm_get_fields(vplbm_ctx *c, double *rho, double *ux, double *uy)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    const size_t n = (size_t)c->nx * c->ny;
    {   // page-locked outputs: the fields kernel writes them in place
        double *h[3] = {rho, ux, uy}, *m[3];
        bool all = true;
        for (int q = 0; q < 3; ++q) {
            m[q] = static_cast<double *>(mapped_host(h[q]));
            all = all && (!h[q] || m[q]);
        }
        if (all) {
            vplbm_status st = vplbm_get_fields_dev(c, m[0], m[1], m[2]);
            if (st != VPLBM_OK) return st;
            CUDA_TRY(cudaStreamSynchronize(c->stream));
            return read_error(c);
        }
    }
    double *tmp = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&tmp, 3 * n * sizeof(double), c->stream));
    vplbm_status st = vplbm_get_fields_dev(c, tmp, tmp + n, tmp + 2 * n);
    if (st != VPLBM_OK) {
        cudaFreeAsync(tmp, c->stream);
        return st;
    }
    double *h[3] = {rho, ux, uy};
    for (int m = 0; m < 3; ++m)
        if (h[m]) CUDA_TRY(cudaMemcpyAsync(h[m], tmp + m * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaFreeAsync(tmp, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return read_error(c);
}

vplbm_status vplbm_get_history(vplbm_ctx *c, long long first, long long count, vplbm_record *dst)
{
    return vplbm_get_history_body(c, 0, first, count, dst);
}

vplbm_status vplbm_get_history_body(vplbm_ctx *c, int k, long long first, long long count, vplbm_record *dst)
{
    if (!c || (!dst && count > 0)) return fail(VPLBM_EINVAL, "NULL argument");
    if (k < 0 || k >= body_slots(c->nbodies)) return fail(VPLBM_EINVAL, "body %d out of range", k);
    const vplbm_record *ring = c->hist + (size_t)k * c->hist_cap;
    if (first < 0 || count < 0) return fail(VPLBM_EINVAL, "negative range");
    if (first + count > c->nstep || first < c->nstep - c->hist_cap)
        return fail(VPLBM_ERANGE, "records [%lld, %lld) not available (step %lld, capacity %lld)", first,
                    first + count, c->nstep, c->hist_cap);
    long long done = 0;
    while (done < count) {
        const long long slot = (first + done) % c->hist_cap;
        long long len = c->hist_cap - slot;
        if (len > count - done) len = count - done;
        CUDA_TRY(cudaMemcpyAsync(dst + done, ring + slot, (size_t)len * sizeof(vplbm_record),
                                 cudaMemcpyDeviceToHost, c->stream));
        done += len;
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return read_error(c);
}

vplbm_status vplbm_get_body(vplbm_ctx *c, double q[3], double v[3], long long *step)
{
    return vplbm_get_body_k(c, 0, q, v, step);
}

vplbm_status vplbm_get_num_bodies(vplbm_ctx *c, int *nbodies)
{
    if (!c || !nbodies) return fail(VPLBM_EINVAL, "NULL argument");
    *nbodies = c->nbodies;
    return VPLBM_OK;
}

vplbm_status vplbm_get_body_k(vplbm_ctx *c, int k, double q[3], double v[3], long long *step)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    if (k < 0 || k >= body_slots(c->nbodies)) return fail(VPLBM_EINVAL, "body %d out of range", k);
    BodyState s;
    CUDA_TRY(cudaMemcpyAsync(&s, c->bs + (c->nstep & 1) * body_slots(c->nbodies) + k, sizeof s, cudaMemcpyDeviceToHost,
                             c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int d = 0; d < 3; ++d) {
        if (q) q[d] = s.q[d];
        if (v) v[d] = s.v[d];
    }
    if (step) *step = s.step;
    return read_error(c);
}

vplbm_status vplbm_set_launch(vplbm_ctx *c, int kernel, int bx, int by)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    if (kernel == KERNEL_TMA) {
        if (!c->tma_ok)
            return fail(VPLBM_EUNSUPPORTED, "the TMA-staged kernel needs the MRT operator, FP32/FP16 storage, nx*elem a multiple of 16 bytes and nx >= 136/144");
        c->kernel = KERNEL_TMA;
        c->bx = TMA_TILE_W;
        c->by = 2;
        return VPLBM_OK;
    }
    if (kernel == KERNEL_FUSED2) {
        const char *why = fused2_refusal(c);
        if (why) return fail(VPLBM_EUNSUPPORTED, "%s", why);
        // (bx, by): the 40-register scalar kernel's blocks for single
        // steps; 0 x 0 keeps the current scalar blocks (TMA: 256 x 1)
        if (bx == 0 && by == 0) {
            bx = c->kernel == KERNEL_TMA ? 256 : c->bx;
            by = c->kernel == KERNEL_TMA ? 1 : c->by;
        }
        const int k0 = c->kernel, bx0 = c->bx, by0 = c->by;
        vplbm_status st = vplbm_set_launch(c, KERNEL_SCALAR_40, bx, by);
        if (st != VPLBM_OK) {
            c->kernel = k0; c->bx = bx0; c->by = by0;
            return st;
        }
        c->kernel = KERNEL_FUSED2;
        return VPLBM_OK;
    }
    if (kernel == KERNEL_PAIR) {
        const char *why = pair_refusal(c);
        if (why) return fail(VPLBM_EUNSUPPORTED, "%s", why);
    } else if (kernel != KERNEL_SCALAR && kernel != KERNEL_SCALAR_48 && kernel != KERNEL_SCALAR_40) {
        return fail(VPLBM_EINVAL, "unknown kernel %d", kernel);
    }
    const int t = bx * by;
    if (bx < 32 || bx % 32 || by < 1 || (t != 128 && t != 256))
        return fail(VPLBM_EINVAL, "launch shape %dx%d not allowed", bx, by);
    int w, h;
    tile_of(kernel, bx, by, &w, &h);
    for (int k = 0; k < body_slots(c->nbodies); ++k) {
        const bool present = k < c->nbodies;
        if (max_reduction_blocks(c->nx, c->ny, present ? bounding_radius(&c->bodies[k]) : 0.0, present, w, h) > c->max_parts)
            return fail(VPLBM_EINVAL, "launch shape %dx%d needs more reduction scratch than allocated", bx, by);
    }
    if (grid_rows(c, bx, by, kernel) > MAX_GRID_ROWS)
        return fail(VPLBM_EINVAL, "launch shape %dx%d needs more than %d grid rows on this lattice", bx, by,
                    MAX_GRID_ROWS);
    c->kernel = kernel;
    c->bx = bx;
    c->by = by;
    return VPLBM_OK;
}

vplbm_status vplbm_get_launch(vplbm_ctx *c, int *kernel, int *bx, int *by)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    if (kernel) *kernel = c->kernel;
    if (bx) *bx = c->bx;
    if (by) *by = c->by;
    return VPLBM_OK;
}

vplbm_status vplbm_inject_wait_timeout(vplbm_ctx *c, int enable)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    if (enable && c->kernel != KERNEL_TMA) return fail(VPLBM_EUNSUPPORTED, "the TMA-staged kernel is not selected");
    c->base.tx_extra = enable ? 16u : 0u;
    c->graph_kernel = -1;   // recapture graphs with the new parameters
    return VPLBM_OK;
}

vplbm_status vplbm_get_launch_count(vplbm_ctx *c, long long *launches)
{
    if (!c || !launches) return fail(VPLBM_EINVAL, "NULL argument");
    *launches = c->launches;
    return VPLBM_OK;
}

vplbm_status vplbm_get_kernel_launches(vplbm_ctx *c, long long counts[VPLBM_LAUNCH_KINDS])
{
    if (!c || !counts) return fail(VPLBM_EINVAL, "NULL argument");
    for (int k = 0; k < VPLBM_LAUNCH_KINDS; ++k) counts[k] = c->kcount[k];
    return VPLBM_OK;
}

vplbm_status vplbm_autotune(vplbm_ctx *c, int steps_per_trial)
{
    if (!c) return fail(VPLBM_EINVAL, "context is NULL");
    if (steps_per_trial < 4) steps_per_trial = 4;
    steps_per_trial = (steps_per_trial + 3) / 4 * 4;   // whole pairs of two-step launches
    // save the run state
    void *save_f = nullptr, *save_h = nullptr;
    BodyState save_bs[2 * VPLBM_MAX_BODIES];
    const size_t bsbytes = (c->nbodies > 1 ? 2 * (size_t)c->nbodies : 4) * sizeof(BodyState);
    const size_t hbytes = (size_t)body_slots(c->nbodies) * c->hist_cap * sizeof(vplbm_record);
    CUDA_TRY(cudaMalloc(&save_f, c->pop_bytes));
    if (cudaMalloc(&save_h, hbytes) != cudaSuccess) {
        cudaFree(save_f);
        return fail(VPLBM_ENOMEM, "autotune scratch allocation failed");
    }
    const long long nstep0 = c->nstep;
    const int k0 = c->kernel, bx0 = c->bx, by0 = c->by;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    vplbm_status st = VPLBM_OK;
    float best = 1e30f;
    int best_kernel = -1, best_bx = 0, best_by = 0;
    std::vector<double> save_outlet((size_t)3 * c->ny);
    void *outlet0 = const_cast<void *>(params_for(c, nstep0).conv_in);
    auto restore = [&]() -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(c->f[nstep0 & 1], save_f, c->pop_bytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(outlet0, save_outlet.data(), save_outlet.size() * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->hist, save_h, hbytes, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->bs, save_bs, bsbytes, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        c->nstep = nstep0;
        return e;
    };
    do {
        if (cudaMemcpyAsync(save_f, c->f[nstep0 & 1], c->pop_bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(save_h, c->hist, hbytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(save_bs, c->bs, bsbytes, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
            cudaMemcpyAsync(save_outlet.data(), outlet0, save_outlet.size() * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess ||
            cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            st = fail(VPLBM_ECUDA, "autotune setup failed");
            break;
        }
        // candidates: the TMA-staged kernel, every block shape of the three
        // register budgets of the scalar kernel, then the two-step kernel
        // (from an even step only: its runs start there)
        static const int kinds[4] = {KERNEL_SCALAR_48, KERNEL_SCALAR_40, KERNEL_SCALAR, KERNEL_PAIR};
        for (int cand = -1; cand <= 4 * N_SHAPES; ++cand) {
            const bool two = cand == 4 * N_SHAPES;
            const int ck = cand < 0 ? KERNEL_TMA : two ? KERNEL_FUSED2 : kinds[cand / N_SHAPES];
            const int cbx = cand < 0 || two ? 0 : SHAPES[cand % N_SHAPES][0];
            const int cby = cand < 0 ? 1 : two ? 0 : SHAPES[cand % N_SHAPES][1];
            if (two) {   // single steps of the two-step choice: 256 x 1 blocks where allowed
                if ((nstep0 & 1) || (vplbm_set_launch(c, KERNEL_FUSED2, 256, 1) != VPLBM_OK &&
                                     vplbm_set_launch(c, KERNEL_FUSED2, 128, 2) != VPLBM_OK))
                    continue;
            } else if (vplbm_set_launch(c, ck, cbx, cby) != VPLBM_OK) {
                continue;
            }
            for (int rep = 0; rep < 2; ++rep) {   // first pass warms up
                if (restore() != cudaSuccess) { st = fail(VPLBM_ECUDA, "autotune restore failed"); break; }
                cudaEventRecord(e0, c->stream);
                if (two) {
                    if (launch_lookahead(params_for(c, c->nstep), c->stream) != cudaSuccess)
                        st = fail(VPLBM_ECUDA, "autotune launch failed");
                    for (int L = 0; L < steps_per_trial / 2 && st == VPLBM_OK; ++L)
                        if (launch_two(c, L, 0, c->stream) != cudaSuccess) st = fail(VPLBM_ECUDA, "autotune launch failed");
                    c->nstep += steps_per_trial;
                }
                for (int s = 0; !two && s < steps_per_trial && st == VPLBM_OK; ++s) {
                    if (launch_one(c, c->nstep, c->stream) != cudaSuccess)
                        st = fail(VPLBM_ECUDA, "autotune launch failed");
                    c->nstep++;
                }
                cudaEventRecord(e1, c->stream);
                if (st != VPLBM_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                    if (st == VPLBM_OK) st = fail(VPLBM_ECUDA, "autotune timing failed");
                    break;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep == 1 && ms < best) { best = ms; best_kernel = c->kernel; best_bx = c->bx; best_by = c->by; }
            }
            if (st != VPLBM_OK) break;
        }
    } while (0);
    if (restore() != cudaSuccess && st == VPLBM_OK) st = fail(VPLBM_ECUDA, "autotune restore failed");
    // the trials may have latched errors on a state that was restored
    cudaMemsetAsync(&c->ctrl->err, 0, sizeof(int), c->stream);
    cudaStreamSynchronize(c->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save_f);
    cudaFree(save_h);
    if (best_kernel >= 0) {
        c->kernel = best_kernel;
        c->bx = best_bx;
        c->by = best_by;
    } else {
        c->kernel = k0;
        c->bx = bx0;
        c->by = by0;
    }
    return st;
}

vplbm_status vplbm_save(vplbm_ctx *c, const char *path)
{
    if (!c || !path) return fail(VPLBM_EINVAL, "NULL argument");
    try {
        const int slots = body_slots(c->nbodies);
        std::vector<char> raw(c->pop_bytes);
        std::vector<vplbm_record> hist((size_t)slots * c->hist_cap);
        std::vector<double> outlet((size_t)3 * c->ny);
        BodyState bs[VPLBM_MAX_BODIES];
        CUDA_TRY(cudaMemcpyAsync(outlet.data(), params_for(c, c->nstep).conv_in, outlet.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(raw.data(), c->f[c->nstep & 1], c->pop_bytes, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(hist.data(), c->hist, hist.size() * sizeof(vplbm_record), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(bs, c->bs + (c->nstep & 1) * slots, slots * sizeof(BodyState), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        CkptHeader h{};
        memcpy(h.magic, CKPT_MAGIC, 8);
        h.nx = c->nx; h.ny = c->ny; h.precision = c->precision; h.extra_bodies = slots - 1;
        h.ps = c->ps; h.nstep = c->nstep; h.hist_cap = c->hist_cap; h.launches = c->launches;
        FILE *fp = fopen(path, "wb");
        if (!fp) return fail(VPLBM_EIO, "cannot open %s for writing", path);
        bool ok = fwrite(&h, sizeof h, 1, fp) == 1 && fwrite(bs, sizeof(BodyState), slots, fp) == (size_t)slots &&
                  fwrite(raw.data(), 1, raw.size(), fp) == raw.size() &&
                  fwrite(hist.data(), sizeof(vplbm_record), hist.size(), fp) == hist.size() &&
                  fwrite(outlet.data(), sizeof(double), outlet.size(), fp) == outlet.size();
        ok = (fclose(fp) == 0) && ok;
        if (!ok) return fail(VPLBM_EIO, "write to %s failed", path);
    } catch (const std::bad_alloc &) {
        return fail(VPLBM_ENOMEM, "host allocation failed");
    }
    return read_error(c);
}

vplbm_status vplbm_load(vplbm_ctx *c, const char *path)
{
    if (!c || !path) return fail(VPLBM_EINVAL, "NULL argument");
    try {
        FILE *fp = fopen(path, "rb");
        if (!fp) return fail(VPLBM_EIO, "cannot open %s", path);
        const int slots = body_slots(c->nbodies);
        CkptHeader h;
        BodyState bs[VPLBM_MAX_BODIES];
        bool ok = fread(&h, sizeof h, 1, fp) == 1;
        if (!ok || memcmp(h.magic, CKPT_MAGIC, 8) != 0) {
            fclose(fp);
            return fail(VPLBM_EIO, "%s is not a checkpoint", path);
        }
        if (h.nx != c->nx || h.ny != c->ny || h.precision != c->precision || h.ps != c->ps || h.hist_cap != c->hist_cap ||
            h.extra_bodies != slots - 1) {
            fclose(fp);
            return fail(VPLBM_EINVAL, "checkpoint %s does not match this context", path);
        }
        if (fread(bs, sizeof(BodyState), slots, fp) != (size_t)slots) {
            fclose(fp);
            return fail(VPLBM_EIO, "%s is truncated", path);
        }
        std::vector<char> raw(c->pop_bytes);
        std::vector<vplbm_record> hist((size_t)slots * c->hist_cap);
        std::vector<double> outlet((size_t)3 * c->ny);
        ok = fread(raw.data(), 1, raw.size(), fp) == raw.size() &&
             fread(hist.data(), sizeof(vplbm_record), hist.size(), fp) == hist.size() &&
             fread(outlet.data(), sizeof(double), outlet.size(), fp) == outlet.size();
        fclose(fp);
        if (!ok) return fail(VPLBM_EIO, "%s is truncated", path);
        const int par = (int)(h.nstep & 1);
        CUDA_TRY(cudaMemcpyAsync(const_cast<void *>(params_for(c, h.nstep).conv_in), outlet.data(),
                                 outlet.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->f[par], raw.data(), raw.size(), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->hist, hist.data(), hist.size() * sizeof(vplbm_record), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemcpyAsync(c->bs + par * slots, bs, slots * sizeof(BodyState), cudaMemcpyHostToDevice, c->stream));
        CUDA_TRY(cudaMemsetAsync(c->ctrl, 0, sizeof(Control), c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        c->nstep = h.nstep;
    } catch (const std::bad_alloc &) {
        return fail(VPLBM_ENOMEM, "host allocation failed");
    }
    return VPLBM_OK;
}

}  // extern "C"
