// Internal declarations shared by the kernel and runtime translation units.
// Not part of the public ABI (include/vplbm.h is).
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "vplbm.h"

namespace vplbm {

constexpr int NQ = 9;

// Pose and velocity of the body at the start of a step, the step counter,
// and values derived from the pose that every thread of the step kernel
// needs (so the kernel's main path needs no FP64 and no block barrier).
// Two copies alternate: a step reads one and its tail writes the other, so
// late blocks of the same launch never see a half-updated pose.
struct BodyState {
    double q[3];       // x_G, y_G, theta                      (offset 0)
    double v[3];       // vx, vy, omega                        (24)
    long long step;    // time step this state belongs to      (48)
    long long pad0;    //                                      (56)
    int ilo, ihi;      // node range [ilo, ihi] x [jlo, jhi]   (64, read as one int4)
    int jlo, jhi;      //   that may hold solid nodes (ilo > ihi: none)
    int xi, yi;        // floor(x_G), floor(y_G)               (80, int2)
    float xf, yf;      // x_G - xi, y_G - yi, rounded to FP32   (88, float2)
    float vxf, vyf, omf, pad1;   // velocities in FP32          (96, float4)
    float cthf, sthf;  // cos(theta), sin(theta) in FP32 (ellipse) (112, float2)
    int pad[2];        //                                      (120)
    double cth, sth;   // cos(theta), sin(theta) (ellipse)      (128)
};
static_assert(sizeof(BodyState) == 144, "BodyState layout");
// the step kernel reads these groups with vector loads
static_assert(offsetof(BodyState, ilo) % 16 == 0, "int4 load of the solid range");
static_assert(offsetof(BodyState, xi) % 8 == 0, "int2 load of floor(x_G)");
static_assert(offsetof(BodyState, xf) % 8 == 0, "float2 load of the fractions");
static_assert(offsetof(BodyState, vxf) % 16 == 0, "float4 load of the velocities");
static_assert(offsetof(BodyState, cthf) % 8 == 0, "float2 load of the orientation");

// Body constants over a run (copied into every launch's parameters).
struct DevBody {
    int present;
    int motion;
    int axis;
    unsigned dof_mask;
    double radius, r2;
    double amp, freq, phase, q_center;
    double mass, inertia;
    double inv_mass, inv_inertia;   // 1 / mass, 1 / inertia (free motion), host-computed
    double damp[3], stiff[3], q0[3], f_ext[3];
    double qref;       // rho0 d_ref u_ref^2 / 2 (0: no C_D / C_L)
    double inv_qref;   // 1 / qref (0 when qref is 0)
    int shape;         // vplbm_shape; radius above is the bounding radius
    float r2f;         // r2 in FP32 (the disk predicate of the storage kernels)
    double a2, b2, ab2;          // ellipse: semi-axes squared and their product
    float a2f, b2f, ab2f, bandf; // FP32 copies; bandf: FP32 test band of the ellipse predicate
    double ra, rb;               // rectangle: half-sides
    float raf, rbf, bandr, pad_r; // FP32 copies; bandr: FP32 test band of |u| - a, |v| - b
};

// Number of doubles per block partial: fpen_x, fpen_y, tpen, fh_x, fh_y,
// th, n_solid, (pad).
constexpr int NPART = 8;

// Host-folded relaxation factors (uniform over a run): 1 - s_k, the
// (1 - s_k/2) factors of Eq. (17) with the signs and integer factors of the
// closed-form M F folded in, and g/2.
template <typename R> struct FoldedConsts {
    R hgx, hgy;
    R om1, om2, om4, om6, om7, om8;
    R h1x6, mh2x6, mh4, mh6, h7x2, h8;
};

// Fill the folded factors from the relaxation rates and fluid acceleration.
template <typename R> inline void fold_consts(FoldedConsts<R> &k, const double *sv, double gx, double gy)
{
    k.hgx = (R)(0.5 * gx);
    k.hgy = (R)(0.5 * gy);
    k.om1 = (R)(1.0 - sv[1]); k.om2 = (R)(1.0 - sv[2]); k.om4 = (R)(1.0 - sv[4]);
    k.om6 = (R)(1.0 - sv[6]); k.om7 = (R)(1.0 - sv[7]); k.om8 = (R)(1.0 - sv[8]);
    k.h1x6 = (R)(6.0 * (1.0 - 0.5 * sv[1]));
    k.mh2x6 = (R)(-6.0 * (1.0 - 0.5 * sv[2]));
    k.mh4 = (R)(-(1.0 - 0.5 * sv[4]));
    k.mh6 = (R)(-(1.0 - 0.5 * sv[6]));
    k.h7x2 = (R)(2.0 * (1.0 - 0.5 * sv[7]));
    k.h8 = (R)(1.0 - 0.5 * sv[8]);
}

struct StepParams {
    int nx, ny;
    long long ps;                 // plane stride (elements) of a population buffer
    double s[NQ];
    double eta, rho0, gx, gy;
    double pen_k;                 // 1 / (eta + 1/2)
    // FP32 copies for the FP32/FP16 kernels (a double->float conversion
    // runs on the FP64 pipe, which is narrow on GB300)
    float sf[NQ];
    float rho0f, gxf, gyf, pen_kf, r2f;
    FoldedConsts<float> pc;       // FP32 folded factors
    FoldedConsts<double> pcd;     // FP64 folded factors
    int bc[4];
    double wall_u0[4][2];
    const double *wall_prof[4][2];
    // FP32 copies for the FP32/FP16 kernels' wall terms
    float wall_u0f[4][2];
    const float *wall_proff[4][2];
    // convective outlet (east): the previous step's inward pulled values
    // [3][ny] (a = 3, 6, 7; FP64 for the FP64 kernel, FP32 otherwise), read
    // from conv_in and written to conv_out (parity buffers);
    // f = k1 f_prev + k2 f_zero-gradient, k1 = 1/(1+U), k2 = U/(1+U)
    const void *conv_in;
    void *conv_out;
    double conv_k1, conv_k2;
    float conv_k1f, conv_k2f;
    DevBody body;
    const void *fin;
    void *fout;
    // per-plane pointers (set_planes): src_plane[a] = &fin[a][-c_ay][-c_ax],
    // so the pull of an interior node b = j*nx + i reads src_plane[a][b];
    // dst_plane[a] = &fout[a][0][0]
    const void *src_plane[NQ];
    void *dst_plane[NQ];
    const BodyState *bs_in;
    BodyState *bs_out;
    double *partials;
    long long max_parts;          // capacity of partials, in blocks
    unsigned *ticket;
    int *err;
    vplbm_record *hist;
    long long hist_cap;
    unsigned tx_extra;            // test hook: bytes the first TMA stage waits for in vain
    int collision;                // vplbm_collision: picks the kernel instantiation on the host
    // body blocks of a scalar launch: blocks 0 .. nbody-1 take the tiles
    // that meet the body (and the tail); the others take every tile in
    // row-major order without the solid-node sums.  Set by the launcher,
    // with the number of grid rows they occupy.
    int nbody;
    int nbody_rows;
    // several bodies in the lattice (nbodies > 1, step_multi.cu).  views:
    // one copy of these parameters per body for this step's parity, in
    // device memory, whose body, r2f, bs_in, bs_out, partials, ticket and
    // hist are that body's; bs_in / bs_out above then point at the first of
    // nbodies consecutive states.  body_blocks: the body blocks of body k
    // are [body_blocks[k], body_blocks[k + 1]) (set by the launcher from
    // the bounding radii).
    const StepParams *views;
    int nbodies;
    int body_blocks[VPLBM_MAX_BODIES + 1];
    double body_radius[VPLBM_MAX_BODIES];
};

// Error bits latched in the control word.
constexpr int ERR_NONFINITE = 1;
constexpr int ERR_INTERNAL = 2;
constexpr int ERR_TIMEOUT = 4;

// Control block: ticket counter of each body and error word.
struct Control {
    unsigned ticket[VPLBM_MAX_BODIES];
    int err;
    unsigned pad[59];
};
static_assert(sizeof(Control) == 256, "Control layout");

// Per-plane pointers of the step's source and destination buffers; call
// whenever fin / fout change.  es: bytes per stored population.
inline void set_planes(StepParams &p, int es)
{
    static const int cx[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    static const int cy[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    for (int a = 0; a < NQ; ++a) {
        const long long off = (long long)a * p.ps - cx[a] - (long long)cy[a] * p.nx;
        p.src_plane[a] = static_cast<const char *>(p.fin) + off * es;
        p.dst_plane[a] = static_cast<char *>(p.fout) + (long long)a * p.ps * es;
    }
}

// Fill the derived fields of s from its pose (host and device, same IEEE
// operations on both).
__host__ __device__ inline void derive_pose(BodyState &s, int present, double radius, int nx, int ny,
                                            int shape = VPLBM_SHAPE_DISK)
{
    s.ilo = 1; s.ihi = 0; s.jlo = 1; s.jhi = 0;
    s.xi = s.yi = 0;
    s.xf = s.yf = 0.f;
    s.vxf = (float)s.v[0]; s.vyf = (float)s.v[1]; s.omf = (float)s.v[2];
    s.pad0 = 0;
    s.pad1 = 0.f;
    s.pad[0] = s.pad[1] = 0;
    s.cth = 1.0; s.sth = 0.0;
    if (shape != VPLBM_SHAPE_DISK && isfinite(s.q[2])) {
        s.cth = cos(s.q[2]);
        s.sth = sin(s.q[2]);
    }
    s.cthf = (float)s.cth; s.sthf = (float)s.sth;
    if (!present || !isfinite(s.q[0]) || !isfinite(s.q[1])) return;
    // nodes that may satisfy the chi predicate, one node of margin
    const double ilo = fmax(floor(s.q[0] - radius) - 1.0, 0.0), ihi = fmin(ceil(s.q[0] + radius) + 1.0, (double)(nx - 1));
    const double jlo = fmax(floor(s.q[1] - radius) - 1.0, 0.0), jhi = fmin(ceil(s.q[1] + radius) + 1.0, (double)(ny - 1));
    if (!(ilo <= ihi) || !(jlo <= jhi)) return;   // disk outside the lattice
    s.ilo = (int)ilo; s.ihi = (int)ihi; s.jlo = (int)jlo; s.jhi = (int)jhi;
    const double fx = floor(s.q[0]), fy = floor(s.q[1]);
    s.xi = (int)fx; s.yi = (int)fy;
    s.xf = (float)(s.q[0] - fx); s.yf = (float)(s.q[1] - fy);
}

// Body constants of a launch's parameters (capi.cu).
void fill_dev_body(StepParams &p, const vplbm_lattice_desc *lat, const vplbm_body_desc *body);

// Radius of the disk, or of the circle around the ellipse: sizes the node
// range and the reduction scratch.
inline double bounding_radius(const vplbm_body_desc *b)
{
    if (!b) return 0.0;
    if (b->shape == VPLBM_SHAPE_ELLIPSE) return fmax(b->radius, b->radius_b);
    if (b->shape == VPLBM_SHAPE_RECTANGLE) return sqrt(b->radius * b->radius + b->radius_b * b->radius_b);
    return b->radius;
}

// Step kernels a context can launch: the scalar kernel with the register
// budget of 4 / 5 / 6 blocks of 256 threads per SM, the TMA-staged one, and
// the two-step kernel (two time steps per launch).
enum { KERNEL_SCALAR = 0, KERNEL_SCALAR_48 = 1, KERNEL_SCALAR_40 = 2, KERNEL_TMA = 3, KERNEL_FUSED2 = 4, KERNEL_PAIR = 5 };

// Node-pair kernel (step_pair.cu): FP16 storage, MRT, one body, even nx;
// blocks of bx x by threads on tiles of 2 bx x by nodes (the body blocks on
// tiles of bx x by, one node per thread).  Grid rows it needs.
cudaError_t launch_step_pair(int precision, const StepParams &p, int bx, int by, cudaStream_t stream);
long long pair_grid_rows(int nx, int ny, double radius, int present, int bx, int by);

// Two-step kernel (step_fused2.cu): a block computes time step n on its
// tile and a one-node ring around it into shared memory, then step n + 1 on
// the tile from there.  Tile of the second step: FUSED2_W x FUSED2_H nodes.
constexpr int FUSED2_W = 64, FUSED2_H = 8;
struct Fused2Params {
    StepParams a;      // step n: fin, src planes, pose n (bs_in), partials region 0, ticket 0
    StepParams b;      // step n + 1: dst planes, pose n + 1 (bs_in), partials region 1, ticket 1
    BodyState *next0;  // receives pose n + 2 (prescribed motion)
    BodyState *next1;  // receives pose n + 3
};
// Steps n and n + 1 (asynchronous on `stream`); bodies on a prescribed path
// only, FP32 / FP16 storage.  max_parts of both views
// must cover the union of the node ranges of poses n and n + 1 in
// FUSED2_W x FUSED2_H tiles.
cudaError_t launch_step_fused2(int precision, const Fused2Params &q, cudaStream_t stream);
// Pose n + 1 := the prescribed motion applied to pose n (one thread;
// p.bs_in -> p.bs_out), so that a run of two-step launches can start at n.
cudaError_t launch_lookahead(const StepParams &p, cudaStream_t stream);

// Batched launch of the scalar step over many lattices.
struct BatchLaunch {
    const StepParams *params;   // one per member (device), for this step's parity
    const int2 *tile_map;       // per macro tile (block): its member and its macro tile within the member (device)
    int n;
    int rows;                   // tiles per macro tile (stacked in y), one macro tile per block
    int collision;              // shared by every member (host-side dispatch)
};
// Batched scalar step (step_kernels.cu): macro tiles of bx x (by * rows) nodes.
cudaError_t launch_step_batch(int precision, const BatchLaunch &bl, int total_tiles, int bx, int by,
                              cudaStream_t stream);

// Persistent sweep (sweep.cu): one launch runs nsteps time steps of every
// member of a batch.  Its blocks take work items from a queue (an atomic
// counter over the launch's steps, `chunk` items at a time) and meet at a
// grid-wide barrier after each step; the launch is cooperative, so every
// block is resident and the barrier can complete.
struct SweepCtl {
    unsigned grab;      // work items handed out so far (over the launch)
    unsigned arrive;    // barrier arrivals so far (over the launch)
    int abort;          // set by a block whose barrier wait gave up: all leave
    int err;            // ERR_TIMEOUT: a barrier wait gave up (kept until read)
    unsigned pad[60];
};
static_assert(sizeof(SweepCtl) == 256, "SweepCtl layout");
// Kinds of work item: a body slot (the scalar tile with the solid-node sums
// that the member's current node range maps slot z to; slot 0 also checks
// the slot count w and advances a prescribed body), a pair tile (2 bx x by
// nodes at tile (z, w)), a scalar tile (bx x by nodes at (z, w), no sums).
enum : int { SWEEP_BODY = 0, SWEEP_PAIR = 1, SWEEP_SCALAR = 2 };
struct SweepLaunch {
    const StepParams *params;      // [2][n]: each member's parameters by step parity (device)
    const int4 *items;             // [items_per_step]: (member or -1, kind, z, w) (device)
    SweepCtl *ctl;                 // grab, arrive and abort zeroed before the launch (device)
    int n;
    unsigned items_per_step;       // a multiple of chunk
    unsigned chunk;                // items a block takes at a time
    long long step0;               // step of the launch's first step (its parity picks the parameters)
    int nsteps;
    unsigned long long timeout_ns; // a barrier wait gives up after this long
    unsigned extra_arrivals;       // test hook: arrivals every barrier waits for in vain (0)
};
// 1 if the persistent kernel is built for this precision and collision.
int sweep_supported(int precision, int collision);
// Blocks of bx x by threads the kernel variant keeps resident on the device.
cudaError_t sweep_max_grid(int precision, bool disk, bool psmem, int bx, int by, int *grid);
cudaError_t launch_sweep(int precision, bool disk, bool psmem, const SweepLaunch &sl, int grid, int bx, int by,
                         cudaStream_t stream);

// Launchers (step_kernels.cu).  All are asynchronous on `stream`.
cudaError_t launch_step(int precision, const StepParams &p, int bx, int by, cudaStream_t stream, int minb = 4);
// The same for an elliptic body (step_ellipse.cu) and a rectangular one (step_rectangle.cu).
cudaError_t launch_step_ellipse(int precision, const StepParams &p, int bx, int by, cudaStream_t stream, int minb);
cudaError_t launch_step_rectangle(int precision, const StepParams &p, int bx, int by, cudaStream_t stream, int minb);
// Several bodies of any shapes (step_multi.cu); p.nbodies > 1.
cudaError_t launch_step_multi(int precision, const StepParams &p, int bx, int by, cudaStream_t stream, int minb);
cudaError_t launch_init_equilibrium(int precision, const StepParams &p, const double *rho_dev,
                                    const double *ux_dev, const double *uy_dev, cudaStream_t stream);
// Convective outlet: previous values := the outlet column of p.fin (into p.conv_in).
cudaError_t launch_outlet_reset(int precision, const StepParams &p, cudaStream_t stream);
cudaError_t launch_fields(int precision, const StepParams &p, double *rho_dev, double *ux_dev,
                          double *uy_dev, cudaStream_t stream);

// TMA-staged step (step_tma.cu), FP32/FP16 storage.  The tensor map
// describes the source population buffer as (x: nx, y: ny, plane: 9).
int tma_smem_bytes(int precision);
int tma_halo(int precision);
cudaError_t tma_prepare(int precision, int *blocks_per_sm);
cudaError_t launch_step_tma(int precision, const StepParams &p, const CUtensorMap &map, int grid,
                            cudaStream_t stream);
constexpr int TMA_TILE_W = 128, TMA_TILE_H = 2, TMA_BOX_H = 2;

// Largest number of blocks that can take part in the force reduction for
// a disk of this radius under launch shape (bx, by) on an nx x ny lattice.
long long max_reduction_blocks(int nx, int ny, double radius, int present, int bx, int by);

// Launch shapes the runtime may pick from.
constexpr int N_SHAPES = 7;
extern const int SHAPES[N_SHAPES][2];

}  // namespace vplbm
