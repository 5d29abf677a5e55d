// Allocation-free variant of the time step (vplbm_step_noalloc).
//
// Who needs it: callers that must not allocate device memory once they are
// running -- for example a host application whose device memory is owned by
// another framework's caching allocator (an extra cudaMalloc would fail or
// fragment its pool), or a control loop with a fixed memory budget that
// forbids allocation after start-up because cudaMalloc/cudaFree can
// synchronize the device and take unbounded time.  Such a caller already
// owns its populations, body state and history buffers; what the fused step
// kernel needs besides them is scratch memory (the per-block force partials,
// the ticket counter that elects the tail block, the error word and the
// internal pose records).  Here that scratch is a file-scope __device__
// array of fixed size, so no call allocates anything.
//
// The step kernel itself is the one every other entry point uses
// (launch_step); only where its scratch lives differs.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "vplbm_internal.cuh"

namespace vplbm {

// Reports an error message through vplbm_last_error (capi.cu).
vplbm_status report_error(vplbm_status st, const char *msg);

namespace {

// Capacity of the static scratch: block partials for at most this many
// blocks meeting the disk's bounding box (with the 128 x 2 launch shape a
// disk of radius up to about 450 lattice units on a large lattice).
constexpr int NOALLOC_MAX_PARTS = 4096;
constexpr int NOALLOC_BX = 128, NOALLOC_BY = 2;

struct __align__(256) NoallocScratch {
    BodyState bs[2];                         // internal pose records (ping-pong)
    Control ctrl;                            // ticket + error word
    vplbm_record record;                     // history slot when the caller keeps none
    double partials[NOALLOC_MAX_PARTS * NPART];
};

// 256-byte aligned scratch shared by every call on a device; it lives
// until the process exits.
static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Device address of the scratch, looked up once per device.
constexpr int MAX_DEVICES = 64;
std::mutex g_lookup_mutex;
NoallocScratch *g_scratch_addr[MAX_DEVICES] = {};

// Copy the caller's body state into the internal record, derive the
// pose-dependent values and clear the words that must start at zero.
__global__ void noalloc_prepare(const vplbm_body_state *state, int present, double radius, int nx, int ny, int shape)
{
    NoallocScratch &s = g_noalloc_scratch;
    BodyState b{};
    for (int d = 0; d < 3; ++d) {
        b.q[d] = state->q[d];
        b.v[d] = state->v[d];
    }
    b.step = state->step;
    derive_pose(b, present, radius, nx, ny, shape);
    s.bs[0] = b;
    for (unsigned &t : s.ctrl.ticket) t = 0u;
    s.ctrl.err = 0;
}

// Copy the final internal record back to the caller's body state.
__global__ void noalloc_finish(vplbm_body_state *state, int last)
{
    const NoallocScratch &s = g_noalloc_scratch;
    const BodyState &b = s.bs[last];
    for (int d = 0; d < 3; ++d) {
        state->q[d] = b.q[d];
        state->v[d] = b.v[d];
    }
    state->step = b.step;
    state->error = s.ctrl.err;
    state->pad = 0;
}

vplbm_status scratch_address(NoallocScratch **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_error(VPLBM_ECUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return report_error(VPLBM_EUNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_lookup_mutex);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        // the array's name in host code is only a stand-in: ask the runtime
        // for its address on the current device
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess || !ptr) {
            char msg[256];
            snprintf(msg, sizeof msg, "cudaGetSymbolAddress of the step scratch failed: %s", cudaGetErrorString(e));
            return report_error(VPLBM_ECUDA, msg);
        }
        g_scratch_addr[dev] = static_cast<NoallocScratch *>(ptr);
    }
    *out = g_scratch_addr[dev];
    return VPLBM_OK;
}

}  // namespace
}  // namespace vplbm

using namespace vplbm;

extern "C" vplbm_status vplbm_step_noalloc(const vplbm_lattice_desc *lat, const vplbm_body_desc *body,
                                           void *const populations_dev[2], vplbm_body_state *state_dev,
                                           vplbm_record *history_dev, long long history_capacity,
                                           long long nsteps, void *cuda_stream)
{
    // host-side checks of the descriptors (no device work, no allocation)
    vplbm_buffer_sizes sizes;
    vplbm_status st = vplbm_buffer_sizes_for(lat, body, 1, &sizes);
    if (st != VPLBM_OK) return st;
    if (!populations_dev || !populations_dev[0] || !populations_dev[1] || !state_dev)
        return report_error(VPLBM_EINVAL, "populations_dev[0..1] and state_dev must be device pointers");
    // misaligned buffers would fault in the kernels: refuse them here
    const uintptr_t es = lat->precision == VPLBM_F64 ? 8 : (lat->precision == VPLBM_F32_DEV ? 4 : 2);
    if ((uintptr_t)populations_dev[0] % es || (uintptr_t)populations_dev[1] % es)
        return report_error(VPLBM_EINVAL, "populations_dev[0..1] must be aligned to the storage element size");
    if ((uintptr_t)state_dev % 8 || (uintptr_t)history_dev % 8)
        return report_error(VPLBM_EINVAL, "state_dev and history_dev must be 8-byte aligned");
    if (nsteps < 0) return report_error(VPLBM_EINVAL, "nsteps must be >= 0");
    if (history_dev && history_capacity < 1) return report_error(VPLBM_EINVAL, "history_capacity must be >= 1");
    for (int s = 0; s < 4; ++s)
        if (lat->bc[s].ux_profile || lat->bc[s].uy_profile)
            return report_error(VPLBM_EUNSUPPORTED, "vplbm_step_noalloc takes uniform wall velocities only");
    if (lat->bc[VPLBM_EAST].kind == VPLBM_BC_CONVECTIVE)
        return report_error(VPLBM_EUNSUPPORTED, "vplbm_step_noalloc has no outlet state (convective outlet)");
    const int present = body ? 1 : 0;
    const double radius = bounding_radius(body);
    const long long parts = max_reduction_blocks(lat->nx, lat->ny, radius, present, NOALLOC_BX, NOALLOC_BY);
    if (parts > NOALLOC_MAX_PARTS) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "disk of radius %g needs %lld reduction slots; vplbm_step_noalloc has %d (radius up to about 450)",
                 radius, parts, NOALLOC_MAX_PARTS);
        return report_error(VPLBM_ERANGE, msg);
    }

    NoallocScratch *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != VPLBM_OK) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;

    // step parameters, filled as vplbm_create fills them
    StepParams p{};
    p.nx = lat->nx;
    p.collision = lat->collision;
    p.ny = lat->ny;
    p.ps = ((long long)lat->nx * lat->ny + 127) / 128 * 128;
    for (int k = 0; k < 9; ++k) {
        p.s[k] = lat->s[k];
        p.sf[k] = (float)lat->s[k];
    }
    p.eta = lat->eta;
    p.pen_k = 1.0 / (lat->eta + 0.5);
    p.rho0 = lat->rho0;
    p.gx = lat->gx;
    p.gy = lat->gy;
    p.rho0f = (float)lat->rho0;
    p.gxf = (float)lat->gx;
    p.gyf = (float)lat->gy;
    p.pen_kf = (float)p.pen_k;
    fold_consts(p.pc, lat->s, lat->gx, lat->gy);
    fold_consts(p.pcd, lat->s, lat->gx, lat->gy);
    for (int s = 0; s < 4; ++s) {
        p.bc[s] = lat->bc[s].kind;
        p.wall_u0[s][0] = lat->bc[s].ux;
        p.wall_u0[s][1] = lat->bc[s].uy;
        p.wall_u0f[s][0] = (float)lat->bc[s].ux;
        p.wall_u0f[s][1] = (float)lat->bc[s].uy;
        p.wall_prof[s][0] = p.wall_prof[s][1] = nullptr;
        p.wall_proff[s][0] = p.wall_proff[s][1] = nullptr;
    }
    fill_dev_body(p, lat, body);
    p.partials = scratch->partials;
    p.max_parts = NOALLOC_MAX_PARTS;
    p.ticket = &scratch->ctrl.ticket[0];
    p.err = &scratch->ctrl.err;
    p.hist = history_dev ? history_dev : &scratch->record;
    p.hist_cap = history_dev ? history_capacity : 1;

    noalloc_prepare<<<1, 1, 0, stream>>>(state_dev, present, radius, lat->nx, lat->ny,
                                         body ? body->shape : VPLBM_SHAPE_DISK);
    cudaError_t e = cudaGetLastError();
    for (long long k = 0; k < nsteps && e == cudaSuccess; ++k) {
        const int par = (int)(k & 1);
        p.fin = populations_dev[par];
        p.fout = populations_dev[par ^ 1];
        p.bs_in = &scratch->bs[par];
        p.bs_out = &scratch->bs[par ^ 1];
        set_planes(p, lat->precision == VPLBM_F64 ? 8 : (lat->precision == VPLBM_F32_DEV ? 4 : 2));
        e = launch_step(lat->precision, p, NOALLOC_BX, NOALLOC_BY, stream);
    }
    if (e == cudaSuccess) {
        noalloc_finish<<<1, 1, 0, stream>>>(state_dev, (int)(nsteps & 1));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof msg, "vplbm_step_noalloc launch failed: %s", cudaGetErrorString(e));
        return report_error(VPLBM_ECUDA, msg);
    }
    return VPLBM_OK;
}
