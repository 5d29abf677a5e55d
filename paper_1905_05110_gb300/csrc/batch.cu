// Batched sweep: many simulations of uneven lattice sizes stepped together,
// each member with its own body, reduction and tail.  Three modes:
//   branches:   every member's own step kernel (parameters in the constant
//               bank, its own launch shape), one graph branch per member,
//               so the members' kernels run concurrently and fill each
//               other's waves and tails; CUDA graphs of 32 steps;
//   tiles:      one launch per time step covering every member's tiles (the
//               scalar step's tile code, member found per block, parameters
//               staged in shared memory); CUDA graphs of 32 steps;
//   persistent: one cooperative launch for up to 1024 time steps of every
//               member (sweep.cu: a work queue of body slots and node-pair
//               tiles, a grid-wide barrier per step), captured with the
//               reset of its queue and barrier counters as a CUDA graph.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "vplbm_ctx.cuh"

using namespace vplbm;

namespace {

constexpr int BATCH_GRAPH_STEPS = 32;
// Steps of one persistent launch (and of its graph).
constexpr int PERSIST_STEPS = 1024;
// A barrier wait of the persistent kernel gives up after this long (a step
// of the largest batch that fits in device memory takes well under 0.1 s);
// with the test hook, after this.
constexpr unsigned long long PERSIST_TIMEOUT_NS = 2000000000ull;
constexpr unsigned long long PERSIST_TEST_TIMEOUT_NS = 20000000ull;

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
    // persistent mode (sweep.cu)
    int pbx = 32, pby = 8;             // block shape: pair tiles of 2 pbx x pby nodes, body tiles pbx x pby
    int pchunk = 4;                    // work items a block takes at a time
    int ppsmem = 1;                    // member parameters staged in shared memory
    bool disk = true;                  // every body a disk (or none): the disk instantiation
    int4 *items_dev = nullptr;         // [items_per_step]
    long long items_cap = 0;
    unsigned items_per_step = 0;
    int pgrid = 0;                     // resident blocks of the chosen variant
    vplbm::SweepCtl *sweep_ctl = nullptr;
    unsigned extra_arrivals = 0;       // test hook (vplbm_batch_inject_barrier_timeout)
    bool pgraph_failed = false;        // capture refused: direct launches
    int graph_pkey[4] = {-1, -1, -1, -1};
    long long kernel_launches = 0;     // persistent launches
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

// Work items of one step of the persistent kernel (SweepLaunch::items):
// every member's body slots (as many as the member's step kernel has body
// blocks at this block shape), then the edge tiles of every member (they
// take the one-node code and about twice as long, so they should not be
// among the last items of a step), then the interior tiles member by
// member in row-major order; padded with empty items to a whole number of
// chunks.  A member's tiles are node-pair tiles (2 pbx x pby) if the
// member's nodes can be paired (FP32/FP16, MRT, even nx), else scalar tiles.
vplbm_status build_items(vplbm_batch *b)
{
    std::vector<int4> items;
    const int bx = b->pbx, by = b->pby;
    try {
        for (int k = 0; k < b->n; ++k) {
            const vplbm_ctx *c = b->members[k];
            const long long nb = max_reduction_blocks(c->nx, c->ny, c->has_body ? bounding_radius(&c->body_desc) : 0.0,
                                                      c->has_body, bx, by);
            if (nb > c->max_parts)
                return berr(VPLBM_EINVAL, "member %d: block shape %dx%d needs more reduction scratch than allocated", k,
                            bx, by);
            for (long long s = 0; s < nb; ++s) items.push_back(make_int4(k, SWEEP_BODY, (int)s, (int)nb));
        }
        for (int pass = 0; pass < 2; ++pass)
            for (int k = 0; k < b->n; ++k) {
                const vplbm_ctx *c = b->members[k];
                const bool pair = (c->nx & 1) == 0 && c->nbodies <= 1;
                const int w = pair ? 2 * bx : bx, kind = pair ? SWEEP_PAIR : SWEEP_SCALAR;
                const int ntx = (c->nx + w - 1) / w, nty = (c->ny + by - 1) / by;
                for (int ty = 0; ty < nty; ++ty)
                    for (int tx = 0; tx < ntx; ++tx) {
                        const bool edge = ty == 0 || ty == nty - 1 || tx == 0 || tx == ntx - 1;
                        if (edge == (pass == 0)) items.push_back(make_int4(k, kind, tx, ty));
                    }
            }
        while (items.size() % (size_t)b->pchunk) items.push_back(make_int4(-1, 0, 0, 0));
    } catch (...) {
        return berr(VPLBM_ENOMEM, "host allocation failed");
    }
    if (items.size() >= (1u << 30)) return berr(VPLBM_EINVAL, "batch too large (%zu work items)", items.size());
    if ((long long)items.size() > b->items_cap) {
        if (b->items_dev) cudaFree(b->items_dev);
        b->items_dev = nullptr;
        b->items_cap = 0;
        if (cudaMalloc(&b->items_dev, items.size() * sizeof(int4)) != cudaSuccess)
            return berr(VPLBM_ENOMEM, "work item allocation failed");
        b->items_cap = (long long)items.size();
    }
    b->items_per_step = (unsigned)items.size();
    cudaError_t e = cudaMemcpyAsync(b->items_dev, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return berr(VPLBM_ECUDA, "work item upload failed: %s", cudaGetErrorString(e));
    e = sweep_max_grid(b->precision, b->disk, b->ppsmem != 0, bx, by, &b->pgrid);
    if (e != cudaSuccess || b->pgrid < 1)
        return berr(VPLBM_ECUDA, "persistent kernel occupancy query failed: %s", cudaGetErrorString(e));
    // no more blocks than chunks of a step
    const long long chunks = (long long)b->items_per_step / b->pchunk;
    if (b->pgrid > chunks) b->pgrid = (int)chunks;
    return VPLBM_OK;
}

// Steps one persistent launch may run: the queue counter runs over all of
// them (and two chunks per block beyond) and must stay below 2^32.
long long persist_max_steps(const vplbm_batch *b)
{
    const unsigned long long room = 0xffffffffull - 3ull * b->pgrid * b->pchunk;
    const long long m = (long long)(room / b->items_per_step) - 1;
    return m < PERSIST_STEPS ? m : PERSIST_STEPS;
}

// One persistent launch of nsteps steps from step `step` (parity only),
// after the reset of its queue and barrier counters.
cudaError_t launch_persistent(const vplbm_batch *b, long long step, int nsteps, cudaStream_t stream)
{
    cudaError_t e = cudaMemsetAsync(b->sweep_ctl, 0, offsetof(SweepCtl, err), stream);
    if (e != cudaSuccess) return e;
    SweepLaunch sl;
    sl.params = b->params_dev;
    sl.items = b->items_dev;
    sl.ctl = b->sweep_ctl;
    sl.n = b->n;
    sl.items_per_step = b->items_per_step;
    sl.chunk = (unsigned)b->pchunk;
    sl.step0 = step & 1;
    sl.nsteps = nsteps;
    sl.timeout_ns = b->extra_arrivals ? PERSIST_TEST_TIMEOUT_NS : PERSIST_TIMEOUT_NS;
    sl.extra_arrivals = b->extra_arrivals;
    return launch_sweep(b->precision, b->disk, b->ppsmem != 0, sl, b->pgrid, b->pbx, b->pby, stream);
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
// capture stream; persistent mode: PERSIST_STEPS steps in one launch.
cudaError_t capture_batch_steps(vplbm_batch *b)
{
    if (b->mode == VPLBM_BATCH_PERSISTENT) return launch_persistent(b, 0, PERSIST_STEPS, b->capture);
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
    const int pkey[4] = {b->pbx * 1024 + b->pby, b->pchunk, b->ppsmem, (int)b->extra_arrivals};
    const bool same_p = b->mode != VPLBM_BATCH_PERSISTENT || memcmp(pkey, b->graph_pkey, sizeof pkey) == 0;
    if (b->graph && b->graph_mode == b->mode && b->graph_bx == b->bx && b->graph_by == b->by &&
        b->graph_rows == b->rows && b->graph_members == ml && same_p)
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
    memcpy(b->graph_pkey, pkey, sizeof pkey);
    return VPLBM_OK;
}

vplbm_status batch_step_impl(vplbm_batch *b, long long n)
{
    long long step;
    vplbm_status st = common_step(b, &step);
    if (st != VPLBM_OK) return st;
    long long done = 0;
    if (b->mode == VPLBM_BATCH_PERSISTENT) {
        // graphs of PERSIST_STEPS steps from an even step (if the capture of a
        // cooperative launch is refused: the same launches made directly)
        const long long maxs = persist_max_steps(b);
        if (maxs < 1) return berr(VPLBM_EINVAL, "batch too large for one persistent launch per step");
        while (done < n && st == VPLBM_OK) {
            long long adv = n - done < maxs ? n - done : maxs;
            cudaError_t e = cudaSuccess;
            if (((step + done) & 1) == 0 && adv == PERSIST_STEPS && !b->pgraph_failed) {
                if (ensure_batch_graph(b) != VPLBM_OK) {
                    b->pgraph_failed = true;
                    continue;
                }
                e = cudaGraphLaunch(b->graph, b->stream);
            } else {
                e = launch_persistent(b, step + done, (int)adv, b->stream);
            }
            if (e != cudaSuccess) {
                st = berr(VPLBM_ECUDA, "persistent launch failed: %s", cudaGetErrorString(e));
                break;
            }
            done += adv;
            b->launches += adv;
            b->kernel_launches += 1;
        }
        for (int k = 0; k < b->n; ++k) b->members[k]->nstep = step + done;
        return st;
    }
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
    if (b->items_dev) cudaFree(b->items_dev);
    if (b->sweep_ctl) cudaFree(b->sweep_ctl);
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
        if (e == cudaSuccess) e = cudaMalloc(&b->sweep_ctl, sizeof(SweepCtl));
        if (e == cudaSuccess) e = cudaMemsetAsync(b->sweep_ctl, 0, sizeof(SweepCtl), b->stream);
        if (e != cudaSuccess) st = berr(VPLBM_ECUDA, "batch setup failed: %s", cudaGetErrorString(e));
    }
    if (st == VPLBM_OK)
        for (const vplbm_ctx *c : b->members)
            if (c->has_body && c->body_desc.shape != VPLBM_SHAPE_DISK) b->disk = false;
    if (st == VPLBM_OK && sweep_supported(prec, b->collision)) st = build_items(b);
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
    int err = 0;
    e = cudaMemcpyAsync(&err, &b->sweep_ctl->err, sizeof err, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return berr(VPLBM_ECUDA, "sweep status read failed: %s", cudaGetErrorString(e));
    if (err & ERR_TIMEOUT) {
        // reported once: the members hold the state of an unfinished step
        cudaMemsetAsync(&b->sweep_ctl->err, 0, sizeof err, b->stream);
        cudaStreamSynchronize(b->stream);
        return berr(VPLBM_ETIMEOUT, "a grid-wide barrier wait of the persistent sweep gave up");
    }
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
    if (mode != VPLBM_BATCH_BRANCHES && mode != VPLBM_BATCH_TILES && mode != VPLBM_BATCH_PERSISTENT)
        return berr(VPLBM_EINVAL, "unknown batch mode %d", mode);
    if (mode == VPLBM_BATCH_PERSISTENT && !sweep_supported(b->precision, b->collision))
        return berr(VPLBM_EUNSUPPORTED, "the persistent sweep runs FP32 or FP16 storage with MRT collision");
    b->mode = mode;
    return VPLBM_OK;
}

vplbm_status vplbm_batch_set_persistent(vplbm_batch *b, int block_x, int block_y, int chunk, int params_in_shared)
{
    if (!b) return berr(VPLBM_EINVAL, "batch is NULL");
    if (!sweep_supported(b->precision, b->collision))
        return berr(VPLBM_EUNSUPPORTED, "the persistent sweep runs FP32 or FP16 storage with MRT collision");
    if (block_x < 32 || block_x % 32 || block_y < 1 || block_x * block_y != 256)
        return berr(VPLBM_EINVAL, "block shape %dx%d not allowed", block_x, block_y);
    if (chunk < 1 || chunk > 16) return berr(VPLBM_EINVAL, "chunk %d not in [1, 16]", chunk);
    const int o[4] = {b->pbx, b->pby, b->pchunk, b->ppsmem};
    b->pbx = block_x;
    b->pby = block_y;
    b->pchunk = chunk;
    b->ppsmem = params_in_shared ? 1 : 0;
    vplbm_status st = build_items(b);
    if (st != VPLBM_OK) {
        b->pbx = o[0];
        b->pby = o[1];
        b->pchunk = o[2];
        b->ppsmem = o[3];
        build_items(b);
    }
    return st;
}

vplbm_status vplbm_batch_get_persistent(vplbm_batch *b, int *block_x, int *block_y, int *chunk, int *params_in_shared,
                                        int *grid, long long *kernel_launches)
{
    if (!b) return berr(VPLBM_EINVAL, "batch is NULL");
    if (block_x) *block_x = b->pbx;
    if (block_y) *block_y = b->pby;
    if (chunk) *chunk = b->pchunk;
    if (params_in_shared) *params_in_shared = b->ppsmem;
    if (grid) *grid = b->pgrid;
    if (kernel_launches) *kernel_launches = b->kernel_launches;
    return VPLBM_OK;
}

vplbm_status vplbm_batch_inject_barrier_timeout(vplbm_batch *b, int enable)
{
    if (!b) return berr(VPLBM_EINVAL, "batch is NULL");
    b->extra_arrivals = enable ? 1u : 0u;
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
    float best = 1e30f, best_tiles = 1e30f, best_pers = 1e30f;
    int best_bx = b->bx, best_by = b->by, best_rows = b->rows, best_mode = b->mode;
    int tile_bx = b->bx, tile_by = b->by, tile_rows = b->rows;   // the fastest tile-mode shape
    int pers[4] = {b->pbx, b->pby, b->pchunk, b->ppsmem};        // the fastest persistent variant
    int best_mk = -1, best_mbx = 0, best_mby = 0;   // branch mode: the members' launch choice
    vplbm_status st = VPLBM_OK;
    // branch mode with every member on one scalar or node-pair kernel and
    // block shape (mode, kernel, bx, by), tile-mode shapes (mode, bx, by,
    // rows), persistent variants (mode, bx, by, chunk, parameters in shared
    // memory)
    const int cands[18][5] = {{VPLBM_BATCH_BRANCHES, KERNEL_SCALAR_40, 256, 1, 0},
                              {VPLBM_BATCH_BRANCHES, KERNEL_SCALAR_48, 256, 1, 0},
                              {VPLBM_BATCH_BRANCHES, KERNEL_SCALAR_48, 128, 2, 0},
                              {VPLBM_BATCH_BRANCHES, KERNEL_SCALAR_40, 64, 2, 0},
                              {VPLBM_BATCH_BRANCHES, KERNEL_PAIR, 32, 8, 0},
                              {VPLBM_BATCH_BRANCHES, KERNEL_PAIR, 64, 4, 0},
                              {VPLBM_BATCH_TILES, 256, 1, 8, 0}, {VPLBM_BATCH_TILES, 256, 1, 4, 0},
                              {VPLBM_BATCH_TILES, 256, 1, 16, 0}, {VPLBM_BATCH_TILES, 128, 2, 4, 0},
                              {VPLBM_BATCH_TILES, 128, 1, 8, 0}, {VPLBM_BATCH_TILES, 256, 1, 1, 0},
                              {VPLBM_BATCH_PERSISTENT, 32, 8, 4, 1}, {VPLBM_BATCH_PERSISTENT, 32, 8, 4, 0},
                              {VPLBM_BATCH_PERSISTENT, 32, 8, 2, 1}, {VPLBM_BATCH_PERSISTENT, 32, 8, 8, 1},
                              {VPLBM_BATCH_PERSISTENT, 64, 4, 4, 1}, {VPLBM_BATCH_PERSISTENT, 128, 2, 4, 1}};
    for (const auto &cb : cands) {
        if (cb[0] == VPLBM_BATCH_BRANCHES) {
            bool ok = true;
            for (vplbm_ctx *m : b->members) ok = ok && vplbm_set_launch(m, cb[1], cb[2], cb[3]) == VPLBM_OK;
            if (!ok) continue;   // a member's reduction scratch does not fit this shape
            b->mode = VPLBM_BATCH_BRANCHES;
        } else if (cb[0] == VPLBM_BATCH_TILES) {
            b->mode = VPLBM_BATCH_TILES;
            st = vplbm_batch_set_launch(b, cb[1], cb[2], cb[3]);
            if (st != VPLBM_OK) break;
        } else {
            if (!sweep_supported(b->precision, b->collision)) continue;
            if (vplbm_batch_set_persistent(b, cb[1], cb[2], cb[3], cb[4]) != VPLBM_OK) continue;
            b->mode = VPLBM_BATCH_PERSISTENT;
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
            if (rep == 1 && cb[0] == VPLBM_BATCH_PERSISTENT && ms < best_pers) {
                best_pers = ms;
                for (int q = 0; q < 4; ++q) pers[q] = cb[1 + q];
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
    // the tile and persistent modes keep their own fastest variant whichever
    // mode won
    vplbm_status st2 = best_mode == VPLBM_BATCH_TILES ? vplbm_batch_set_launch(b, best_bx, best_by, best_rows)
                                                      : vplbm_batch_set_launch(b, tile_bx, tile_by, tile_rows);
    if (st2 == VPLBM_OK && sweep_supported(b->precision, b->collision))
        st2 = vplbm_batch_set_persistent(b, pers[0], pers[1], pers[2], pers[3]);
    return st != VPLBM_OK ? st : st2;
}

}  // extern "C"
