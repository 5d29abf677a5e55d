// The simulation context behind vplbm_ctx (internal to the library).
#pragma once

#include "vplbm_internal.cuh"

using vplbm::BodyState;
using vplbm::Control;
using vplbm::StepParams;

struct vplbm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;        // caller's stream
    cudaStream_t capture = nullptr;       // private stream used only to capture graphs
    int precision = 0;
    int collision = 0;
    int nx = 0, ny = 0;
    long long ps = 0;                     // plane stride (elements)
    size_t pop_bytes = 0;
    StepParams base{};
    vplbm_body_desc body_desc{};          // body 0
    bool has_body = false;
    int nbodies = 0;                      // 0 .. VPLBM_MAX_BODIES
    vplbm_body_desc bodies[VPLBM_MAX_BODIES] = {};
    void *f[2] = {nullptr, nullptr};
    BodyState *bs = nullptr;              // [parity][max(nbodies, 1)]
    StepParams *views = nullptr;          // [parity][nbodies] per-body parameters (nbodies > 1)
    double *partials = nullptr;
    long long max_parts = 0;
    Control *ctrl = nullptr;
    vplbm_record *hist = nullptr;         // [max(nbodies, 1)][hist_cap]
    long long hist_cap = 0;
    double *prof = nullptr;
    void *outlet = nullptr;               // convective outlet state, 2 parities x 3 x ny (8-byte slots)
    void *owned = nullptr;                // single allocation when the library owns memory
    long long nstep = 0;
    int kernel = vplbm::KERNEL_SCALAR;    // KERNEL_SCALAR / _48 / _40 / KERNEL_TMA
    int bx = 128, by = 2;
    cudaGraphExec_t graph = nullptr;
    int graph_kernel = -1, graph_bx = -1, graph_by = -1;
    long long launches = 0;
    long long kcount[VPLBM_LAUNCH_KINDS] = {};   // launches by kernel kind (vplbm_launch_kind)
    // TMA-staged kernel (FP32/FP16 storage): tensor maps of the two
    // population buffers as sources, persistent grid size
    bool tma_ok = false;
    CUtensorMap tmap[2];
    int tma_grid = 0;
    // device workspace of vplbm_adjoint (checkpoints, segment stores,
    // adjoint fields, accumulators), kept between calls; grown when a call
    // needs more, freed by vplbm_destroy
    void *adj_ws = nullptr;
    size_t adj_ws_bytes = 0;
};

namespace vplbm {
// Shared runtime helpers (capi.cu).
StepParams ctx_params(const vplbm_ctx *c, long long step);        // parameters of step `step`
cudaError_t ctx_launch(const vplbm_ctx *c, long long step, cudaStream_t stream);
vplbm_status ctx_read_error(vplbm_ctx *c);                          // latched device errors (syncs)
vplbm_status report_error(vplbm_status st, const char *msg);
}  // namespace vplbm
