// Batched sweep: many simulations of uneven lattice sizes stepped together,
// each member with its own body, reduction and tail, captured as CUDA graphs
// of 32 steps.  Two modes:
//   branches: every member's own step kernel (parameters in the constant
//             bank, its own launch shape), one graph branch per member, so
//             the members' kernels run concurrently and fill each other's
//             waves and tails;
//   tiles:    one launch per time step covering every member's tiles (the
//             scalar step's tile code, member found per block, parameters
//             staged in shared memory).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "vplbm_ctx.cuh"

using namespace vplbm;

namespace {

constexpr int BATCH_GRAPH_STEPS = 32;

vplbm_status berr(vplbm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return report_error(st, buf);
}

}  // namespace

struct vplbm_batch {
    int n = 0;
    std::vector<vplbm_ctx *> members;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;
    int precision = 0;
    int collision = 0;
    int bx = 256, by = 1;             // block (tile) shape of the batched kernel
    int rows = 8;                     // tiles per block, stacked in y
    StepParams *params_dev = nullptr; // [2][n]: parameters of each member per step parity
    int *tile_start_dev = nullptr;    // [n + 1]
    int2 *tile_map_dev = nullptr;     // [total_tiles]: (member, macro tile within the member)
    long long tile_map_cap = 0;
    int total_tiles = 0;
    int mode = VPLBM_BATCH_BRANCHES;
    std::vector<cudaStream_t> branch;  // capture streams of the per-member graph branches
    std::vector<cudaEvent_t> join;     // [0]: fork, [1 + k]: end of branch k
    cudaGraphExec_t graph = nullptr;
    int graph_bx = -1, graph_by = -1, graph_rows = -1, graph_mode = -1;
    std::vector<int> graph_members;   // branch mode: each member's (kernel, bx, by) when captured
    long long launches = 0;
};

namespace {

// Macro-tile prefix of the members for blocks of bx x by threads that run
// `rows` tiles each, and the map from a block (macro tile) to its member
// and its macro tile within the member, so that a block finds both with
// one load.
vplbm_status build_tiles(vplbm_batch *b)
{
    std::vector<int> start(b->n + 1, 0);
    long long total = 0;
    for (int k = 0; k < b->n; ++k) {
        const vplbm_ctx *c = b->members[k];
        start[k] = (int)total;
        const long long nty = (c->ny + b->by - 1) / b->by;
        total += (long long)((c->nx + b->bx - 1) / b->bx) * ((nty + b->rows - 1) / b->rows);
    }
    if (total > (1LL << 30)) return berr(VPLBM_EINVAL, "batch too large (%lld tiles)", total);
    start[b->n] = (int)total;
    std::vector<int2> map;
    try {
        map.resize((size_t)total);
    } catch (...) {
        return berr(VPLBM_ENOMEM, "host allocation failed");
    }
    for (int k = 0; k < b->n; ++k)
        for (int t = start[k]; t < start[k + 1]; ++t) map[(size_t)t] = make_int2(k, t - start[k]);
    if (total > b->tile_map_cap) {
        if (b->tile_map_dev) cudaFree(b->tile_map_dev);
        b->tile_map_dev = nullptr;
        b->tile_map_cap = 0;
        if (cudaMalloc(&b->tile_map_dev, (size_t)total * sizeof(int2)) != cudaSuccess)
            return berr(VPLBM_ENOMEM, "tile map allocation failed");
        b->tile_map_cap = total;
    }
    b->total_tiles = (int)total;
    cudaError_t e = cudaMemcpyAsync(b->tile_start_dev, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->tile_map_dev, map.data(), map.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return berr(VPLBM_ECUDA, "tile table upload failed: %s", cudaGetErrorString(e));
    return VPLBM_OK;
}

vplbm_status upload_params(vplbm_batch *b)
{
    std::vector<StepParams> ps(2 * (size_t)b->n);
    for (int par = 0; par < 2; ++par)
        for (int k = 0; k < b->n; ++k) ps[(size_t)par * b->n + k] = ctx_params(b->members[k], par);
    cudaError_t e = cudaMemcpyAsync(b->params_dev, ps.data(), ps.size() * sizeof(StepParams), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return berr(VPLBM_ECUDA, "parameter upload failed: %s", cudaGetErrorString(e));
    return VPLBM_OK;
}

cudaError_t launch_batch_step(const vplbm_batch *b, long long step, cudaStream_t stream)
{
    if (b->mode == VPLBM_BATCH_BRANCHES) {
        for (int k = 0; k < b->n; ++k) {
            const cudaError_t e = ctx_launch(b->members[k], step, stream);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    BatchLaunch bl;
    bl.params = b->params_dev + (size_t)(step & 1) * b->n;
    bl.tile_map = b->tile_map_dev;
    bl.n = b->n;
    bl.rows = b->rows;
    bl.collision = b->collision;
    return launch_step_batch(b->precision, bl, b->total_tiles, b->bx, b->by, stream);
}

// All members must stand at the same step (they advance together).
vplbm_status common_step(const vplbm_batch *b, long long *step)
{
    const long long s = b->members[0]->nstep;
    for (int k = 1; k < b->n; ++k)
        if (b->members[k]->nstep != s)
            return berr(VPLBM_EINVAL, "batch members are at different steps (%lld vs %lld)", s, b->members[k]->nstep);
    *step = s;
    return VPLBM_OK;
}

// Streams and events of the branch graph, created on first use.
cudaError_t ensure_branches(vplbm_batch *b)
{
    if ((int)b->branch.size() == b->n) return cudaSuccess;
    b->branch.assign(b->n, nullptr);
    b->join.assign(b->n + 1, nullptr);
    for (int k = 0; k < b->n; ++k) {
        const cudaError_t e = cudaStreamCreateWithFlags(&b->branch[k], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
    }
    for (int k = 0; k <= b->n; ++k) {
        const cudaError_t e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// BATCH_GRAPH_STEPS steps of every member: tile mode, one launch per step;
// branch mode, one branch per member forked from and joined into the
// capture stream.
cudaError_t capture_batch_steps(vplbm_batch *b)
{
    if (b->mode != VPLBM_BATCH_BRANCHES) {
        for (int k = 0; k < BATCH_GRAPH_STEPS; ++k) {
            const cudaError_t e = launch_batch_step(b, k, b->capture);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    cudaError_t e = cudaEventRecord(b->join[0], b->capture);
    for (int m = 0; m < b->n && e == cudaSuccess; ++m) {
        e = cudaStreamWaitEvent(b->branch[m], b->join[0], 0);
        for (int k = 0; k < BATCH_GRAPH_STEPS && e == cudaSuccess; ++k) e = ctx_launch(b->members[m], k, b->branch[m]);
        if (e == cudaSuccess) e = cudaEventRecord(b->join[1 + m], b->branch[m]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->capture, b->join[1 + m], 0);
    }
    return e;
}

// The members' launch choices a branch graph bakes in.
std::vector<int> member_launches(const vplbm_batch *b)
{
    std::vector<int> v;
    v.reserve(3 * (size_t)b->n);
    for (const vplbm_ctx *c : b->members) {
        v.push_back(c->kernel);
        v.push_back(c->bx);
        v.push_back(c->by);
    }
    return v;
}

vplbm_status ensure_batch_graph(vplbm_batch *b)
{
    const std::vector<int> ml = b->mode == VPLBM_BATCH_BRANCHES ? member_launches(b) : std::vector<int>();
    if (b->graph && b->graph_mode == b->mode && b->graph_bx == b->bx && b->graph_by == b->by &&
        b->graph_rows == b->rows && b->graph_members == ml)
        return VPLBM_OK;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    if (b->mode == VPLBM_BATCH_BRANCHES) {
        const cudaError_t e = ensure_branches(b);
        if (e != cudaSuccess) return berr(VPLBM_ECUDA, "branch streams: %s", cudaGetErrorString(e));
    }
    cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return berr(VPLBM_ECUDA, "capture begin failed: %s", cudaGetErrorString(e));
    const cudaError_t err = capture_batch_steps(b);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->capture, &g);
    if (err != cudaSuccess || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return berr(VPLBM_ECUDA, "batch graph capture failed: %s", cudaGetErrorString(err != cudaSuccess ? err : e));
    }
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return berr(VPLBM_ECUDA, "batch graph instantiate failed: %s", cudaGetErrorString(e));
    b->graph_mode = b->mode;
    b->graph_bx = b->bx;
    b->graph_by = b->by;
    b->graph_rows = b->rows;
    b->graph_members = ml;
    return VPLBM_OK;
}

vplbm_status batch_step_impl(vplbm_batch *b, long long n)
{
    long long step;
    vplbm_status st = common_step(b, &step);
    if (st != VPLBM_OK) return st;
    long long done = 0;
    while (done < n) {
        long long adv;
        if (((step + done) & 1) == 0 && n - done >= BATCH_GRAPH_STEPS) {
            st = ensure_batch_graph(b);
            if (st != VPLBM_OK) break;
            cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) { st = berr(VPLBM_ECUDA, "batch graph launch failed: %s", cudaGetErrorString(e)); break; }
            adv = BATCH_GRAPH_STEPS;
        } else {
            cudaError_t e = launch_batch_step(b, step + done, b->stream);
            if (e != cudaSuccess) { st = berr(VPLBM_ECUDA, "batch launch failed: %s", cudaGetErrorString(e)); break; }
            adv = 1;
        }
        done += adv;
        b->launches += adv;
    }
    for (int k = 0; k < b->n; ++k) b->members[k]->nstep = step + done;
    return st;
}

}  // namespace

extern "C" {

void vplbm_batch_destroy(vplbm_batch *b)
{
    if (!b) return;
    if (b->stream || b->params_dev) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (cudaStream_t st : b->branch)
        if (st) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->join)
        if (ev) cudaEventDestroy(ev);
    if (b->capture) cudaStreamDestroy(b->capture);
    if (b->params_dev) cudaFree(b->params_dev);
    if (b->tile_start_dev) cudaFree(b->tile_start_dev);
    if (b->tile_map_dev) cudaFree(b->tile_map_dev);
    for (vplbm_ctx *c : b->members) vplbm_destroy(c);
    delete b;
}

vplbm_status vplbm_batch_create(const vplbm_lattice_desc *lats, const vplbm_body_desc *const *bodies, int n,
                                long long history_capacity, void *cuda_stream, vplbm_batch **out)
{
    if (!out || !lats || n < 1) return berr(VPLBM_EINVAL, "need n >= 1 lattice descriptors and an out pointer");
    *out = nullptr;
    const int prec = lats[0].precision;
    for (int k = 0; k < n; ++k)
        if (lats[k].precision != prec) return berr(VPLBM_EINVAL, "member %d: all members need the same precision", k);
    for (int k = 0; k < n; ++k)
        if (lats[k].collision != lats[0].collision)
            return berr(VPLBM_EINVAL, "member %d: all members need the same collision operator", k);
    vplbm_batch *b = new (std::nothrow) vplbm_batch();
    if (!b) return berr(VPLBM_ENOMEM, "host allocation failed");
    b->n = n;
    b->stream = (cudaStream_t)cuda_stream;
    b->precision = prec;
    b->collision = lats[0].collision;
    vplbm_status st = VPLBM_OK;
    try {
        b->members.assign(n, nullptr);
    } catch (...) {
        delete b;
        return berr(VPLBM_ENOMEM, "host allocation failed");
    }
    for (int k = 0; k < n && st == VPLBM_OK; ++k)
        st = vplbm_create(&lats[k], bodies ? bodies[k] : nullptr, history_capacity, cuda_stream, &b->members[k]);
    cudaError_t e = cudaSuccess;
    if (st == VPLBM_OK) {
        e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMalloc(&b->params_dev, 2 * (size_t)n * sizeof(StepParams));
        if (e == cudaSuccess) e = cudaMalloc(&b->tile_start_dev, (size_t)(n + 1) * sizeof(int));
        if (e != cudaSuccess) st = berr(VPLBM_ECUDA, "batch setup failed: %s", cudaGetErrorString(e));
    }
    if (st == VPLBM_OK) st = upload_params(b);
    if (st == VPLBM_OK) st = build_tiles(b);
    if (st != VPLBM_OK) {
        vplbm_batch_destroy(b);
        return st;
    }
    *out = b;
    return VPLBM_OK;
}

vplbm_status vplbm_batch_member(vplbm_batch *b, int k, vplbm_ctx **member)
{
    if (!b || !member || k < 0 || k >= b->n) return berr(VPLBM_EINVAL, "no member %d", k);
    *member = b->members[k];
    return VPLBM_OK;
}

vplbm_status vplbm_batch_step(vplbm_batch *b, long long nsteps)
{
    if (!b) return berr(VPLBM_EINVAL, "batch is NULL");
    if (nsteps < 0) return berr(VPLBM_EINVAL, "nsteps must be >= 0");
    return batch_step_impl(b, nsteps);
}

vplbm_status vplbm_batch_sync(vplbm_batch *b)
{
    if (!b) return berr(VPLBM_EINVAL, "batch is NULL");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return berr(VPLBM_ECUDA, "stream synchronize failed: %s", cudaGetErrorString(e));
    for (int k = 0; k < b->n; ++k) {
        vplbm_status st = ctx_read_error(b->members[k]);
        if (st != VPLBM_OK) return st;
    }
    return VPLBM_OK;
}

vplbm_status vplbm_batch_set_launch(vplbm_batch *b, int block_x, int block_y, int tiles_per_block)
{
    if (!b) return berr(VPLBM_EINVAL, "batch is NULL");
    const int t = block_x * block_y;
    if (block_x < 32 || block_x % 32 || block_y < 1 || (t != 128 && t != 256))
        return berr(VPLBM_EINVAL, "block shape %dx%d not allowed", block_x, block_y);
    if (tiles_per_block < 1 || tiles_per_block > 64)
        return berr(VPLBM_EINVAL, "tiles per block %d not in [1, 64]", tiles_per_block);
    for (int k = 0; k < b->n; ++k) {
        const vplbm_ctx *c = b->members[k];
        if (max_reduction_blocks(c->nx, c->ny, c->has_body ? bounding_radius(&c->body_desc) : 0.0, c->has_body, block_x, block_y) >
            c->max_parts)
            return berr(VPLBM_EINVAL, "member %d: block shape needs more reduction scratch than allocated", k);
    }
    const int obx = b->bx, oby = b->by, orows = b->rows;
    b->bx = block_x;
    b->by = block_y;
    b->rows = tiles_per_block;
    vplbm_status st = build_tiles(b);
    if (st != VPLBM_OK) {
        b->bx = obx;
        b->by = oby;
        b->rows = orows;
        build_tiles(b);
    }
    return st;
}

vplbm_status vplbm_batch_set_mode(vplbm_batch *b, int mode)
{
    if (!b) return berr(VPLBM_EINVAL, "batch is NULL");
    if (mode != VPLBM_BATCH_BRANCHES && mode != VPLBM_BATCH_TILES) return berr(VPLBM_EINVAL, "unknown batch mode %d", mode);
    b->mode = mode;
    return VPLBM_OK;
}

vplbm_status vplbm_batch_get_mode(vplbm_batch *b, int *mode)
{
    if (!b || !mode) return berr(VPLBM_EINVAL, "NULL argument");
    *mode = b->mode;
    return VPLBM_OK;
}

vplbm_status vplbm_batch_get_launch(vplbm_batch *b, int *block_x, int *block_y, int *tiles_per_block,
                                   long long *launches)
{
    if (!b) return berr(VPLBM_EINVAL, "batch is NULL");
    if (block_x) *block_x = b->bx;
    if (block_y) *block_y = b->by;
    if (tiles_per_block) *tiles_per_block = b->rows;
    if (launches) *launches = b->launches;
    return VPLBM_OK;
}

vplbm_status vplbm_batch_autotune(vplbm_batch *b, int steps_per_trial)
{
    if (!b) return berr(VPLBM_EINVAL, "batch is NULL");
    // whole graphs: the modes are compared as they run (a branch-mode step
    // outside a graph launches the members one after another)
    if (steps_per_trial < BATCH_GRAPH_STEPS) steps_per_trial = BATCH_GRAPH_STEPS;
    steps_per_trial = (steps_per_trial + BATCH_GRAPH_STEPS - 1) / BATCH_GRAPH_STEPS * BATCH_GRAPH_STEPS;
    {   // start the trials at an even step so that they run as graphs
        long long step;
        vplbm_status st0 = common_step(b, &step);
        if (st0 != VPLBM_OK) return st0;
        if (step & 1) {
            st0 = batch_step_impl(b, 1);
            if (st0 != VPLBM_OK) return st0;
        }
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return berr(VPLBM_ECUDA, "event creation failed");
    float best = 1e30f, best_tiles = 1e30f;
    int best_bx = b->bx, best_by = b->by, best_rows = b->rows, best_mode = b->mode;
    int tile_bx = b->bx, tile_by = b->by, tile_rows = b->rows;   // the fastest tile-mode shape
    int best_mk = -1, best_mbx = 0, best_mby = 0;   // branch mode: the members' launch choice
    vplbm_status st = VPLBM_OK;
    // branch mode with every member on one scalar kernel and block shape
    // (mode, kernel, bx, by), then tile-mode shapes (mode, bx, by, rows)
    const int cands[12][4] = {{VPLBM_BATCH_BRANCHES, KERNEL_SCALAR_40, 256, 1},
                              {VPLBM_BATCH_BRANCHES, KERNEL_SCALAR_48, 256, 1},
                              {VPLBM_BATCH_BRANCHES, KERNEL_SCALAR_48, 128, 2},
                              {VPLBM_BATCH_BRANCHES, KERNEL_SCALAR_40, 64, 2},
                              {VPLBM_BATCH_BRANCHES, KERNEL_PAIR, 32, 8},
                              {VPLBM_BATCH_BRANCHES, KERNEL_PAIR, 64, 4},
                              {VPLBM_BATCH_TILES, 256, 1, 8}, {VPLBM_BATCH_TILES, 256, 1, 4},
                              {VPLBM_BATCH_TILES, 256, 1, 16}, {VPLBM_BATCH_TILES, 128, 2, 4},
                              {VPLBM_BATCH_TILES, 128, 1, 8}, {VPLBM_BATCH_TILES, 256, 1, 1}};
    for (const auto &cb : cands) {
        if (cb[0] == VPLBM_BATCH_BRANCHES) {
            bool ok = true;
            for (vplbm_ctx *m : b->members) ok = ok && vplbm_set_launch(m, cb[1], cb[2], cb[3]) == VPLBM_OK;
            if (!ok) continue;   // a member's reduction scratch does not fit this shape
            b->mode = VPLBM_BATCH_BRANCHES;
        } else {
            b->mode = VPLBM_BATCH_TILES;
            st = vplbm_batch_set_launch(b, cb[1], cb[2], cb[3]);
            if (st != VPLBM_OK) break;
        }
        for (int rep = 0; rep < 2 && st == VPLBM_OK; ++rep) {
            cudaEventRecord(e0, b->stream);
            st = batch_step_impl(b, steps_per_trial);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = berr(VPLBM_ECUDA, "autotune timing failed");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep == 1 && cb[0] == VPLBM_BATCH_TILES && ms < best_tiles) {
                best_tiles = ms;
                tile_bx = b->bx;
                tile_by = b->by;
                tile_rows = b->rows;
            }
            if (rep == 1 && ms < best) {
                best = ms;
                best_mode = b->mode;
                best_bx = b->bx;
                best_by = b->by;
                best_rows = b->rows;
                if (cb[0] == VPLBM_BATCH_BRANCHES) {
                    best_mk = cb[1];
                    best_mbx = cb[2];
                    best_mby = cb[3];
                }
            }
        }
        if (st != VPLBM_OK) break;
    }
    if (best_mk >= 0)
        for (vplbm_ctx *m : b->members) vplbm_set_launch(m, best_mk, best_mbx, best_mby);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->mode = best_mode;
    // the tile mode keeps its own fastest shape whichever mode won
    vplbm_status st2 = best_mode == VPLBM_BATCH_TILES ? vplbm_batch_set_launch(b, best_bx, best_by, best_rows)
                                                      : vplbm_batch_set_launch(b, tile_bx, tile_by, tile_rows);
    return st != VPLBM_OK ? st : st2;
}

}  // extern "C"
