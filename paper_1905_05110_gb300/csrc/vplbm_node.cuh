// Device code shared by the step kernels: precision traits, the pull with
// boundary rules, the per-node VP-MRT update (Eqs. 14-22), the solid-node
// sums (Eqs. 25-27), the rigid-body update (Eqs. 23-24) and the tail.
// Internal to the library; every function is inlined into its kernel.
#pragma once

#include <math.h>

#include "vplbm_internal.cuh"

namespace vplbm {
namespace {

// ---- precision traits -------------------------------------------------

template <int P> struct Prec;
template <> struct Prec<VPLBM_F64> { using S = double; using T = double; static constexpr bool DEV = false; };
template <> struct Prec<VPLBM_F32_DEV> { using S = float; using T = float; static constexpr bool DEV = true; };
template <> struct Prec<VPLBM_F16_DEV> { using S = __half; using T = float; static constexpr bool DEV = true; };

// Loads of the populations and the pose written by the previous time step.
// A kernel launched once per step reads them through the read-only path
// (ld.global.nc: they do not change while it runs).  A kernel that runs
// several steps in one launch reads data it wrote itself after a grid-wide
// barrier, which the non-coherent path may serve stale: its translation unit
// defines VPLBM_COHERENT_LOADS before including this header, and its loads
// go to L2 (ld.global.cg).
#ifdef VPLBM_COHERENT_LOADS
#define VPLBM_LDG(ptr) __ldcg(ptr)
#else
#define VPLBM_LDG(ptr) __ldg(ptr)
#endif

__device__ __forceinline__ double ldv(const double *p) { return VPLBM_LDG(p); }
__device__ __forceinline__ float ldv(const float *p) { return VPLBM_LDG(p); }
__device__ __forceinline__ float ldv(const __half *p) { return __half2float(VPLBM_LDG(p)); }
__device__ __forceinline__ void stv(double *p, double x) { *p = x; }
__device__ __forceinline__ void stv(float *p, float x) { *p = x; }
__device__ __forceinline__ void stv(__half *p, float x) { *p = __float2half_rn(x); }

// Pairs of x-adjacent populations (the node-pair paths): an aligned pair
// from global memory or a shared-memory stage, two single values (a pair
// that straddles the alignment), an aligned pair store.
__device__ __forceinline__ float2 ld_pair_g(const float *p) { return VPLBM_LDG(reinterpret_cast<const float2 *>(p)); }
__device__ __forceinline__ float2 ld_pair_g(const __half *p) { return __half22float2(VPLBM_LDG(reinterpret_cast<const __half2 *>(p))); }
__device__ __forceinline__ float2 ld_two_g(const float *p) { return make_float2(VPLBM_LDG(p), VPLBM_LDG(p + 1)); }
__device__ __forceinline__ float2 ld_two_g(const __half *p) { return make_float2(__half2float(VPLBM_LDG(p)), __half2float(VPLBM_LDG(p + 1))); }
__device__ __forceinline__ float2 ld_pair_s(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ float2 ld_pair_s(const __half *p) { return __half22float2(*reinterpret_cast<const __half2 *>(p)); }
__device__ __forceinline__ float2 ld_two_s(const float *p) { return make_float2(p[0], p[1]); }
__device__ __forceinline__ float2 ld_two_s(const __half *p) { return make_float2(__half2float(p[0]), __half2float(p[1])); }
__device__ __forceinline__ void st_pair(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ void st_pair(__half *p, float2 v) { *reinterpret_cast<__half2 *>(p) = __floats2half2_rn(v.x, v.y); }

// D2Q9 velocity set in the order of Eq. (10), weights of Eq. (13).
__host__ __device__ constexpr int cx_of(int a) { return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0); }
__host__ __device__ constexpr int cy_of(int a) { return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp_of(int a) { return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 5 + 2) % 4) + 5); }
__host__ __device__ constexpr int miry_of(int a) { return a == 2 ? 4 : a == 4 ? 2 : a == 5 ? 8 : a == 8 ? 5 : a == 6 ? 7 : a == 7 ? 6 : a; }
// Slot of an inward population of the east outlet (c_ax = -1: a = 3, 6, 7).
__host__ __device__ constexpr int outlet_slot(int a) { return a == 3 ? 0 : (a == 6 ? 1 : 2); }
__host__ __device__ constexpr double w_of(int a) { return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

static_assert(opp_of(1) == 3 && opp_of(2) == 4 && opp_of(3) == 1 && opp_of(4) == 2, "opp axis");
static_assert(opp_of(5) == 7 && opp_of(6) == 8 && opp_of(7) == 5 && opp_of(8) == 6, "opp diag");
static_assert(cx_of(miry_of(6)) == cx_of(6) && cy_of(miry_of(6)) == -cy_of(6) && cy_of(miry_of(2)) == -1, "mirror");

// 1/x: FP64 division, or in FP32 the hardware reciprocal estimate refined
// by one Newton-Raphson step, r1 = r0 + r0 (1 - x r0) (within an ulp or two).
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip(float x)
{
    float r0;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(x));
    return fmaf(r0, fmaf(-x, r0, 1.0f), r0);
}

// A parameter in the kernel's arithmetic type: the FP64 value for the FP64
// kernel, the host-rounded FP32 copy otherwise (no conversion on the device).
template <typename T> __device__ __forceinline__ T par(double d, float f);
template <> __device__ __forceinline__ double par<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float par<float>(double, float f) { return f; }

// Host-folded relaxation factors in the arithmetic type of the kernel.
template <typename T> __device__ __forceinline__ const auto &folded(const StepParams &p);
template <> __device__ __forceinline__ const auto &folded<float>(const StepParams &p) { return p.pc; }
template <> __device__ __forceinline__ const auto &folded<double>(const StepParams &p) { return p.pcd; }

__device__ __forceinline__ double wall_u(const StepParams &p, int side, int comp, int k)
{
    const double *prof = p.wall_prof[side][comp];
    return prof ? prof[k] : p.wall_u0[side][comp];
}
__device__ __forceinline__ float wall_uf(const StepParams &p, int side, int comp, int k)
{
    const float *prof = p.wall_proff[side][comp];
    return prof ? prof[k] : p.wall_u0f[side][comp];
}

// Moving-wall term 6 w_a rho0 (c_a . u_w) of the velocity rule, in the
// kernel's arithmetic type (FP32 for the FP32/FP16 kernels: no FP64 on the
// edge path).
template <typename T>
__device__ __forceinline__ T wall_term(const StepParams &p, int a, int side, int k);
template <>
__device__ __forceinline__ double wall_term<double>(const StepParams &p, int a, int side, int k)
{
    const double cu = cx_of(a) * wall_u(p, side, 0, k) + cy_of(a) * wall_u(p, side, 1, k);
    return 6.0 * w_of(a) * p.rho0 * cu;
}
template <>
__device__ __forceinline__ float wall_term<float>(const StepParams &p, int a, int side, int k)
{
    const float cu = (float)cx_of(a) * wall_uf(p, side, 0, k) + (float)cy_of(a) * wall_uf(p, side, 1, k);
    return ((float)(6.0 * w_of(a)) * p.rho0f) * cu;
}

// Source of a pull: population a of the previous post-collision field at
// lattice node (i, j) (inside the lattice), and the convective outlet's
// previous pulled value of inward population a at row j.  GlobalSrc reads
// the population buffer and the outlet state; the two-step kernel reads its
// shared-memory stage and its own record of the first step instead.
template <int P> struct GlobalSrc {
    const typename Prec<P>::S *fin;
    long long ps;
    int nx;
    __device__ __forceinline__ typename Prec<P>::T operator()(int a, int i, int j) const
    {
        return ldv(fin + a * ps + (long long)j * nx + i);
    }
    __device__ __forceinline__ typename Prec<P>::T outlet_prev(const StepParams &p, int a, int j) const
    {
        return static_cast<const typename Prec<P>::T *>(p.conv_in)[outlet_slot(a) * p.ny + j];
    }
};

// Pull of population a into edge node (i, j), with the boundary rules.
template <int P, class Src>
__device__ __forceinline__ typename Prec<P>::T pull_edge_src(const StepParams &p, const Src &src, int a, int i, int j)
{
    using T = typename Prec<P>::T;
    const int nx = p.nx, ny = p.ny;
    int si = i - cx_of(a);
    int sj = j - cy_of(a);
    if (sj < 0 || sj >= ny) {
        const int side = sj < 0 ? VPLBM_SOUTH : VPLBM_NORTH;
        const int kind = p.bc[side];
        if (kind == VPLBM_BC_PERIODIC) {
            sj = sj < 0 ? sj + ny : sj - ny;
        } else if (kind == VPLBM_BC_SYMMETRY) {   // specular reflection at the half-way wall
            int mi = i - cx_of(a);
            if (mi < 0 || mi >= nx) mi = p.bc[VPLBM_WEST] == VPLBM_BC_PERIODIC ? (mi < 0 ? mi + nx : mi - nx) : i;
            return src(miry_of(a), mi, j);
        } else {
            T val = src(opp_of(a), i, j);
            if (kind == VPLBM_BC_VELOCITY) val += wall_term<T>(p, a, side, i);
            return val;
        }
    }
    if (si < 0 || si >= nx) {
        const int side = si < 0 ? VPLBM_WEST : VPLBM_EAST;
        const int kind = p.bc[side];
        if (kind == VPLBM_BC_PERIODIC) {
            si = si < 0 ? si + nx : si - nx;
        } else if (kind == VPLBM_BC_ZEROGRAD) {
            return src(a, i, sj);
        } else if (kind == VPLBM_BC_CONVECTIVE) {   // east only (checked on the host)
            const T z = src(a, i, sj);
            const T prev = src.outlet_prev(p, a, j);
            return par<T>(p.conv_k1, p.conv_k1f) * prev + par<T>(p.conv_k2, p.conv_k2f) * z;
        } else {
            T val = src(opp_of(a), i, j);
            if (kind == VPLBM_BC_VELOCITY) val += wall_term<T>(p, a, side, j);
            return val;
        }
    }
    return src(a, si, sj);
}

template <int P>
__device__ typename Prec<P>::T pull_edge(const StepParams &p, const typename Prec<P>::S *fin, int a, int i, int j)
{
    return pull_edge_src<P>(p, GlobalSrc<P>{fin, p.ps, p.nx}, a, i, j);
}

// Pull-stream all 9 populations of node (i, j); INTERIOR: the caller knows
// the node is not on a lattice edge.
template <int P, bool INTERIOR = false>
__device__ __forceinline__ void pull_all(const StepParams &p, const typename Prec<P>::S *__restrict__ fin,
                                         int i, int j, typename Prec<P>::T f[NQ])
{
    using S = typename Prec<P>::S;
    if (INTERIOR || (i > 0 && i < p.nx - 1 && j > 0 && j < p.ny - 1)) {
        const int b = j * p.nx + i;
#pragma unroll
        for (int a = 0; a < NQ; ++a) f[a] = ldv(static_cast<const S *>(p.src_plane[a]) + b);
    } else {
#pragma unroll
        for (int a = 0; a < NQ; ++a) f[a] = pull_edge<P>(p, fin, a, i, j);
    }
}

// Convective outlet: keep this step's pulled inward populations of an
// outlet node for the next step's rule.
template <int P>
__device__ __forceinline__ void record_outlet(const StepParams &p, int j, const typename Prec<P>::T f[NQ])
{
    using T = typename Prec<P>::T;
    T *out = static_cast<T *>(p.conv_out);
    out[outlet_slot(3) * p.ny + j] = f[3];
    out[outlet_slot(6) * p.ny + j] = f[6];
    out[outlet_slot(7) * p.ny + j] = f[7];
}

// Exact chi predicate of Eq. (2) in FP64 without contraction.
__device__ __forceinline__ bool chi_exact(int i, int j, double xg, double yg, double r2)
{
    double dx = __dsub_rn((double)i, xg);
    double dy = __dsub_rn((double)j, yg);
    double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    return d2 <= r2;
}

// Rectangle: |u| <= a and |v| <= b with (u, v) the node in the body frame,
// FP64 without contraction.
__device__ __forceinline__ bool chi_exact_rect(int i, int j, const BodyState *bs, const DevBody &b)
{
    const double dx = __dsub_rn((double)i, bs->q[0]);
    const double dy = __dsub_rn((double)j, bs->q[1]);
    const double c = bs->cth, s = bs->sth;
    const double u = __dadd_rn(__dmul_rn(dx, c), __dmul_rn(dy, s));
    const double v = __dsub_rn(__dmul_rn(dy, c), __dmul_rn(dx, s));
    return fabs(u) <= b.ra && fabs(v) <= b.rb;
}

// Ellipse: b^2 u^2 + a^2 v^2 <= a^2 b^2 with (u, v) the node in the body
// frame, FP64 without contraction, in a fixed order.
__device__ __forceinline__ bool chi_exact_ellipse(int i, int j, const BodyState *bs, const DevBody &b)
{
    const double dx = __dsub_rn((double)i, bs->q[0]);
    const double dy = __dsub_rn((double)j, bs->q[1]);
    const double c = bs->cth, s = bs->sth;
    const double u = __dadd_rn(__dmul_rn(dx, c), __dmul_rn(dy, s));
    const double v = __dsub_rn(__dmul_rn(dy, c), __dmul_rn(dx, s));
    const double lhs = __dadd_rn(__dmul_rn(b.b2, __dmul_rn(u, u)), __dmul_rn(b.a2, __dmul_rn(v, v)));
    return lhs <= b.ab2;
}

// ---- rigid body (Eqs. 23-24 and Algorithm 1 step 3) --------------------

__device__ void body_acc(const DevBody &b, const double F[3], const double q[3], const double v[3], double acc[3])
{
    for (int d = 0; d < 3; ++d) {
        const double inv_m = d < 2 ? b.inv_mass : b.inv_inertia;   // a multiply: FP64 divides are long on GB300
        acc[d] = (F[d] + b.f_ext[d] - b.damp[d] * v[d] - b.stiff[d] * (q[d] - b.q0[d])) * inv_m;
    }
}

__device__ void body_advance(const DevBody &b, long long step, const double F[3], double q[3], double v[3])
{
    if (!b.present || b.motion == VPLBM_MOTION_FIXED) return;
    if (b.motion == VPLBM_MOTION_IMPOSED) {
        const double two_pi = 6.283185307179586;
        const double ph = two_pi * b.freq * (double)(step + 1) + b.phase;
        double sn, cs;
        sincos(ph, &sn, &cs);
        q[b.axis] = b.q_center + b.amp * sn;
        v[b.axis] = two_pi * b.freq * b.amp * cs;
        return;
    }
    // classic RK4, h = 1, force held over the step
    double k1v[3], k2v[3], k3v[3], k4v[3], k2q[3], k3q[3], k4q[3], qt[3], vt[3];
    body_acc(b, F, q, v, k1v);
    for (int d = 0; d < 3; ++d) { qt[d] = q[d] + 0.5 * v[d]; vt[d] = v[d] + 0.5 * k1v[d]; }
    for (int d = 0; d < 3; ++d) k2q[d] = vt[d];
    body_acc(b, F, qt, vt, k2v);
    for (int d = 0; d < 3; ++d) { qt[d] = q[d] + 0.5 * k2q[d]; vt[d] = v[d] + 0.5 * k2v[d]; }
    for (int d = 0; d < 3; ++d) k3q[d] = vt[d];
    body_acc(b, F, qt, vt, k3v);
    for (int d = 0; d < 3; ++d) { qt[d] = q[d] + k3q[d]; vt[d] = v[d] + k3v[d]; }
    for (int d = 0; d < 3; ++d) k4q[d] = vt[d];
    body_acc(b, F, qt, vt, k4v);
    for (int d = 0; d < 3; ++d) {
        if (!((b.dof_mask >> d) & 1u)) continue;
        const double nq = q[d] + (v[d] + 2.0 * k2q[d] + 2.0 * k3q[d] + k4q[d]) / 6.0;
        const double nv = v[d] + (k1v[d] + 2.0 * k2v[d] + 2.0 * k3v[d] + k4v[d]) / 6.0;
        q[d] = nq;
        v[d] = nv;
    }
}

// ---- the 7 solid-node sums (Eqs. 25-27 and the penalization reaction) ---
//
// FP64 kernel: the terms and their sums in FP64.  FP32 / FP16 kernels: the
// terms in FP32 and their sums in float-float (hi + lo): GB300's FP64 pipe
// is narrow, and a block that meets the body would otherwise spend most of
// its time on FP64 adds.  A float-float sum carries about 44 bits, and the
// block's sum is converted to FP64 exactly before it is published.

// Float-float addition: Knuth's TwoSum of the high parts, the low parts
// added to its error term, then a fast renormalisation (Dekker).
__device__ __forceinline__ float2 ff_add(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = ((a.x - (s - bb)) + (b.x - bb)) + (a.y + b.y);
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}

template <int P> struct SumT { using A = float2; using V = float; };
template <> struct SumT<VPLBM_F64> { using A = double; using V = double; };

__device__ __forceinline__ void acc_add(double &a, double b) { a += b; }
__device__ __forceinline__ void acc_add(float2 &a, float2 b) { a = ff_add(a, b); }
__device__ __forceinline__ void acc_add(float2 &a, float b) { a = ff_add(a, make_float2(b, 0.f)); }
__device__ __forceinline__ void acc_zero(double &a) { a = 0.0; }
__device__ __forceinline__ void acc_zero(float2 &a) { a = make_float2(0.f, 0.f); }
__device__ __forceinline__ double acc_shfl_down(double a, int off) { return __shfl_down_sync(0xffffffffu, a, off); }
__device__ __forceinline__ float2 acc_shfl_down(float2 a, int off)
{
    return make_float2(__shfl_down_sync(0xffffffffu, a.x, off), __shfl_down_sync(0xffffffffu, a.y, off));
}
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(float2 a) { return (double)a.x + (double)a.y; }   // exact

// Bodies on a prescribed path (absent, fixed or imposed) move independently
// of the forces: their next pose is computed by one thread of the first
// block of the step (advance_prescribed), off the tail's critical path.
__device__ __forceinline__ bool prescribed_motion(const StepParams &p)
{
    return !p.body.present || p.body.motion != VPLBM_MOTION_FREE;
}

__device__ __noinline__ void advance_prescribed(const StepParams &p)
{
    BodyState nb = *p.bs_in;
    const double F0[3] = {0.0, 0.0, 0.0};   // not used by fixed / imposed motion
    body_advance(p.body, nb.step, F0, nb.q, nb.v);
    nb.step += 1;
    derive_pose(nb, p.body.present, p.body.radius, p.nx, p.ny, p.body.shape);
    *p.bs_out = nb;
}

// Last participating block: fixed-order sum of the partials (accumulator
// type A, as the blocks published them), history record, and for a free
// body the RK4 update and next pose.  Runs on warp 0.
template <typename A>
__device__ __noinline__ void step_tail(const StepParams &p, int nparts)
{
    const int lane = threadIdx.x & 31;
    BodyState cur;
    if (lane == 0) cur = *p.bs_in;   // issued before the partial loads
    A acc[NPART - 1];
#pragma unroll
    for (int k = 0; k < NPART - 1; ++k) acc_zero(acc[k]);
    // two partials per lane are loaded together (one memory round trip up
    // to 64 partials), then added in lane order
    for (int s0 = 0; s0 < nparts; s0 += 64) {
        const int sa = s0 + lane, sb = s0 + 32 + lane;
        A va[NPART - 1], vb[NPART - 1];
#pragma unroll
        for (int k = 0; k < NPART - 1; ++k) {
            acc_zero(va[k]);
            acc_zero(vb[k]);
        }
        if (sa < nparts) {
            const A *src = reinterpret_cast<const A *>(p.partials + (size_t)sa * NPART);
#pragma unroll
            for (int k = 0; k < NPART - 1; ++k) va[k] = __ldcg(src + k);
        }
        if (sb < nparts) {
            const A *src = reinterpret_cast<const A *>(p.partials + (size_t)sb * NPART);
#pragma unroll
            for (int k = 0; k < NPART - 1; ++k) vb[k] = __ldcg(src + k);
        }
#pragma unroll
        for (int k = 0; k < NPART - 1; ++k) {
            acc_add(acc[k], va[k]);
            acc_add(acc[k], vb[k]);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int k = 0; k < NPART - 1; ++k) acc_add(acc[k], acc_shfl_down(acc[k], off));
    if (lane != 0) return;
    double sum[NPART - 1];
#pragma unroll
    for (int k = 0; k < NPART - 1; ++k) sum[k] = acc_value(acc[k]);

    const double Fh[3] = {sum[3], sum[4], sum[5]};
    vplbm_record r;
    r.t = (double)cur.step;
    r.fx = Fh[0]; r.fy = Fh[1]; r.torque = Fh[2];
    r.cd = Fh[0] * p.body.inv_qref;
    r.cl = Fh[1] * p.body.inv_qref;
    r.x = cur.q[0]; r.y = cur.q[1]; r.theta = cur.q[2];
    r.vx = cur.v[0]; r.vy = cur.v[1]; r.omega = cur.v[2];
    r.fpen_x = sum[0]; r.fpen_y = sum[1]; r.tpen = sum[2];
    r.n_solid = sum[6];
    p.hist[cur.step % p.hist_cap] = r;

    if (!prescribed_motion(p)) {
        BodyState nb = cur;
        body_advance(p.body, cur.step, Fh, nb.q, nb.v);
        nb.step = cur.step + 1;
        derive_pose(nb, p.body.present, p.body.radius, p.nx, p.ny, p.body.shape);
        *p.bs_out = nb;
    }
    *p.ticket = 0u;   // ready for the next launch (stream order)
}

// Terms of one solid node: penalization reaction (force, torque about x_G),
// momentum exchanged through its links during the streaming into this step
// (force, torque), and the node count.  The pulled populations are loaded
// again (cache hits) so that they are not live across the stores.
// f: the node's pulled populations; own(a): its own previous post-collision
// population a.
template <int P, class Own>
__device__ __forceinline__ void solid_terms_from(const BodyState *bs, const typename Prec<P>::T f[NQ], const Own &own,
                                                 int i, int j, typename SumT<P>::V rho, typename SumT<P>::V ax,
                                                 typename SumT<P>::V ay, typename SumT<P>::V out[NPART - 1])
{
    using V = typename SumT<P>::V;
    V dx, dy;
    if constexpr (P == VPLBM_F64) {
        dx = (double)i - bs->q[0];
        dy = (double)j - bs->q[1];
    } else {
        const int2 xy = VPLBM_LDG(reinterpret_cast<const int2 *>(&bs->xi));
        const float2 fr = VPLBM_LDG(reinterpret_cast<const float2 *>(&bs->xf));
        dx = (float)(i - xy.x) - fr.x;
        dy = (float)(j - xy.y) - fr.y;
    }
    const V px = -rho * ax, py = -rho * ay;
    V ex = 0, ey = 0;
#pragma unroll
    for (int a = 1; a < NQ; ++a) {
        const V d = (V)f[a] - (V)own(a);   // pulled minus own
        ex += cx_of(a) * d;
        ey += cy_of(a) * d;
    }
    out[0] = px;
    out[1] = py;
    out[2] = dx * py - dy * px;
    out[3] = ex;
    out[4] = ey;
    out[5] = dx * ey - dy * ex;
    out[6] = 1;
}

template <int P>
__device__ __forceinline__ void solid_node_terms(const StepParams &p, const typename Prec<P>::S *fin, int i, int j,
                                                 typename SumT<P>::V rho, typename SumT<P>::V ax,
                                                 typename SumT<P>::V ay, typename SumT<P>::V out[NPART - 1])
{
    using T = typename Prec<P>::T;
    T f[NQ];
    pull_all<P>(p, fin, i, j, f);
    const long long b = (long long)j * p.nx + i;
    solid_terms_from<P>(p.bs_in, f, [&](int a) { return ldv(fin + a * p.ps + b); }, i, j, rho, ax, ay, out);
}


// Body shape read from the parameters instead of fixed at compile time.
constexpr int SHAPE_ANY = -1;

// chi of node (i, j) for one body (Eq. 2, Alg. 1 step 4) and its lever arm
// (dxl, dyl) = x - x_G.  The storage kernels test in FP32 and re-test in
// FP64 where the FP32 value is within the band of the boundary, so the
// result is the exact FP64 predicate.  SHAPE: VPLBM_SHAPE_DISK, _ELLIPSE or
// _RECTANGLE fixed at compile time, or SHAPE_ANY to read it from the body.
template <int P, int SHAPE>
__device__ __forceinline__ bool body_chi(const DevBody &body, float r2f, const BodyState *__restrict__ bs, int i,
                                         int j, typename Prec<P>::T &dxl, typename Prec<P>::T &dyl)
{
    using T = typename Prec<P>::T;
    constexpr bool DEV = Prec<P>::DEV;
    bool chi = false;
    if constexpr (DEV) {
        const int2 xy = VPLBM_LDG(reinterpret_cast<const int2 *>(&bs->xi));
        const float2 fr = VPLBM_LDG(reinterpret_cast<const float2 *>(&bs->xf));
        const float dxf = (float)(i - xy.x) - fr.x;
        const float dyf = (float)(j - xy.y) - fr.y;
        const int shape = SHAPE == SHAPE_ANY ? body.shape : SHAPE;
        if (shape == VPLBM_SHAPE_RECTANGLE) {
            // |u| <= a and |v| <= b in the body frame, in FP32, exact
            // FP64 re-test where either is within the band of its edge
            const float2 cs = VPLBM_LDG(reinterpret_cast<const float2 *>(&bs->cthf));
            const float uf = fabsf(dxf * cs.x + dyf * cs.y);
            const float vf = fabsf(dyf * cs.x - dxf * cs.y);
            const float band = body.bandr;
            if (fabsf(uf - body.raf) <= band || fabsf(vf - body.rbf) <= band)
                chi = chi_exact_rect(i, j, bs, body);
            else
                chi = uf <= body.raf && vf <= body.rbf;
        } else if (shape == VPLBM_SHAPE_ELLIPSE) {
            // b^2 u^2 + a^2 v^2 <= a^2 b^2 in the body frame, in FP32,
            // exact FP64 re-test inside the band
            const float2 cs = VPLBM_LDG(reinterpret_cast<const float2 *>(&bs->cthf));
            const float uf = dxf * cs.x + dyf * cs.y;
            const float vf = dyf * cs.x - dxf * cs.y;
            const float lhs = body.b2f * (uf * uf) + body.a2f * (vf * vf);
            if (fabsf(lhs - body.ab2f) <= body.bandf) chi = chi_exact_ellipse(i, j, bs, body);
            else chi = lhs <= body.ab2f;
        } else {
            const float d2 = dxf * dxf + dyf * dyf;
            const float r2 = r2f;
            const float band = 1e-5f * r2 + 1e-5f;
            if (fabsf(d2 - r2) <= band) chi = chi_exact(i, j, bs->q[0], bs->q[1], body.r2);
            else chi = d2 <= r2;
        }
        dxl = dxf; dyl = dyf;
    } else {
        const double xg = VPLBM_LDG(&bs->q[0]), yg = VPLBM_LDG(&bs->q[1]);
        const int shape = SHAPE == SHAPE_ANY ? body.shape : SHAPE;
        chi = shape == VPLBM_SHAPE_ELLIPSE   ? chi_exact_ellipse(i, j, bs, body)
              : shape == VPLBM_SHAPE_RECTANGLE ? chi_exact_rect(i, j, bs, body)
                                               : chi_exact(i, j, xg, yg, body.r2);
        dxl = (double)i - xg;
        dyl = (double)j - yg;
    }
    return chi;
}

// ---- FP16-storage MRT update in explicit lane operations ---------------
//
// The FP16-deviation kernels run the MRT update through these lane types:
// Lane1 on one node (a float per quantity), Lane2 on two x-adjacent nodes
// at once (a float2 per quantity, one paired FP32 instruction per
// operation).  Every operation rounds once, as written, with no
// contraction left to the compiler, and a paired instruction rounds each
// lane like its scalar counterpart, so a node updated in a pair gets the
// bits it gets alone.
struct Lane1 {
    using L = float;
    static constexpr bool SCALAR = true;
    static __device__ __forceinline__ L c(float x) { return x; }
    static __device__ __forceinline__ L add(L a, L b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ L sub(L a, L b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ L mul(L a, L b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ L fma(L a, L b, L d) { return __fmaf_rn(a, b, d); }
    static __device__ __forceinline__ L fms(L a, L b, L d) { return __fmaf_rn(a, b, -d); }   // a b - d
    static __device__ __forceinline__ L recip(L x) { return vplbm::recip(x); }
    static __device__ __forceinline__ bool bad(L rho) { return !(rho > 0.f) || !(rho < 1e30f); }
};
struct Lane2 {
    using L = float2;
    static constexpr bool SCALAR = false;
    static __device__ __forceinline__ L c(float x) { return make_float2(x, x); }
    static __device__ __forceinline__ L add(L a, L b) { return __fadd2_rn(a, b); }
    // a - b: the product b (-1) is exact, so one rounding, as __fsub_rn
    static __device__ __forceinline__ L sub(L a, L b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
    static __device__ __forceinline__ L mul(L a, L b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ L fma(L a, L b, L d) { return __ffma2_rn(a, b, d); }
    static __device__ __forceinline__ L fms(L a, L b, L d) { return __ffma2_rn(a, b, make_float2(-d.x, -d.y)); }
    static __device__ __forceinline__ L recip(L x)
    {
        // the hardware estimate per lane, the Newton-Raphson step paired:
        // the same two roundings as recip(float)
        float r0x, r0y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0x) : "f"(x.x));
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0y) : "f"(x.y));
        const float2 r0 = make_float2(r0x, r0y);
        return __ffma2_rn(r0, __ffma2_rn(make_float2(-x.x, -x.y), r0, make_float2(1.f, 1.f)), r0);
    }
    static __device__ __forceinline__ bool bad(L rho) { return Lane1::bad(rho.x) || Lane1::bad(rho.y); }
};

// The MRT update (Eqs. 14-17 with the closed-form M F) of the pulled
// deviation populations f (f_a - w_a rho0) of one node or a pair, from
// rho, j and the penalized velocity u with forcing G = rho (g + a) (Eq. 22;
// a = 0 off the body: u = j / rho + g / 2), stored through store(a, value).
// Returns rho.  Lane1 only: chi and the lever arm (dxl, dyl) of the node,
// and (ax, ay) = a for the solid-node sums.
template <class Ln, class Store>
__device__ __forceinline__ typename Ln::L mrt_dev_lanes(const StepParams &p, const typename Ln::L f[NQ], bool chi,
                                                        float dxl, float dyl, const BodyState *__restrict__ bs,
                                                        const Store &store, float &ax_out, float &ay_out)
{
    using L = typename Ln::L;
    const L d13 = Ln::sub(f[1], f[3]), d24 = Ln::sub(f[2], f[4]), b13 = Ln::add(f[1], f[3]), b24 = Ln::add(f[2], f[4]);
    const L d56 = Ln::sub(f[5], f[6]), d87 = Ln::sub(f[8], f[7]), a56 = Ln::add(f[5], f[6]), a78 = Ln::add(f[7], f[8]);
    const L sx = Ln::add(d56, d87), ty = Ln::sub(a56, a78), sa = Ln::add(b13, b24), sd = Ln::add(a56, a78);
    const L rs = Ln::add(Ln::add(f[0], sa), sd);
    const L rho = Ln::add(Ln::c(p.rho0f), rs);
    const L jx = Ln::add(d13, sx), jy = Ln::add(d24, ty);
    const L inv_rho = Ln::recip(rho);
    L ux = Ln::fma(jx, inv_rho, Ln::c(p.pc.hgx)), uy = Ln::fma(jy, inv_rho, Ln::c(p.pc.hgy));
    L Gx = Ln::mul(rho, Ln::c(p.gxf)), Gy = Ln::mul(rho, Ln::c(p.gyf));
    ax_out = 0.f;
    ay_out = 0.f;
    if constexpr (Ln::SCALAR) {
        if (chi) {   // Eq. (22), eta-stable form: a = (u_s - v) / (eta + 1/2), u = v + a / 2
            const float4 vv = VPLBM_LDG(reinterpret_cast<const float4 *>(&bs->vxf));
            const float usx = __fmaf_rn(-vv.z, dyl, vv.x), usy = __fmaf_rn(vv.z, dxl, vv.y);
            const float ax = __fmul_rn(__fsub_rn(usx, ux), p.pen_kf), ay = __fmul_rn(__fsub_rn(usy, uy), p.pen_kf);
            Gx = __fmul_rn(rho, __fadd_rn(p.gxf, ax));
            Gy = __fmul_rn(rho, __fadd_rn(p.gyf, ay));
            ux = __fmaf_rn(0.5f, ax, ux);
            uy = __fmaf_rn(0.5f, ay, uy);
            ax_out = ax;
            ay_out = ay;
        }
    }
    const auto &k = p.pc;
    const L e = Ln::fma(Ln::c(-4.f), f[0], Ln::fms(Ln::c(2.f), sd, sa));
    const L ep = Ln::fma(Ln::c(4.f), f[0], Ln::fma(Ln::c(-2.f), sa, sd));
    const L qx = Ln::fma(Ln::c(-2.f), d13, sx), qy = Ln::fma(Ln::c(-2.f), d24, ty);
    const L pxx = Ln::sub(b13, b24);
    const L pxy = Ln::sub(Ln::add(f[5], f[7]), Ln::add(f[6], f[8]));
    const L ux2 = Ln::mul(ux, ux), uy2 = Ln::mul(uy, uy);
    const L u2r = Ln::mul(rho, Ln::add(ux2, uy2));
    const L uG = Ln::fma(ux, Gx, Ln::mul(uy, Gy));
    const L es = Ln::fma(Ln::c(k.om1), e,
                         Ln::fma(Ln::c(p.sf[1]), Ln::fma(Ln::c(3.f), u2r, Ln::mul(Ln::c(-2.f), rs)),
                                 Ln::mul(Ln::c(k.h1x6), uG)));
    const L eps = Ln::fma(Ln::c(k.om2), ep,
                          Ln::fma(Ln::c(p.sf[2]), Ln::fma(Ln::c(-3.f), u2r, rs), Ln::mul(Ln::c(k.mh2x6), uG)));
    const L jxs = Ln::add(jx, Gx), jys = Ln::add(jy, Gy);
    const L qxs = Ln::fma(Ln::c(k.om4), qx, Ln::fma(Ln::c(-p.sf[4]), Ln::mul(rho, ux), Ln::mul(Ln::c(k.mh4), Gx)));
    const L qys = Ln::fma(Ln::c(k.om6), qy, Ln::fma(Ln::c(-p.sf[6]), Ln::mul(rho, uy), Ln::mul(Ln::c(k.mh6), Gy)));
    const L cxx = Ln::fms(ux, Gx, Ln::mul(uy, Gy)), cxy = Ln::fma(ux, Gy, Ln::mul(uy, Gx));
    const L pxxs = Ln::fma(Ln::c(k.om7), pxx,
                           Ln::fma(Ln::c(p.sf[7]), Ln::mul(rho, Ln::sub(ux2, uy2)), Ln::mul(Ln::c(k.h7x2), cxx)));
    const L pxys = Ln::fma(Ln::c(k.om8), pxy,
                           Ln::fma(Ln::c(p.sf[8]), Ln::mul(rho, Ln::mul(ux, uy)), Ln::mul(Ln::c(k.h8), cxy)));
    // back to populations, M^-1 = M^T diag(1/|row|^2)
    const L r9 = Ln::mul(rs, Ln::c(1.f / 9.f));
    const L A = Ln::fma(eps, Ln::c(-1.f / 18.f), Ln::fma(es, Ln::c(-1.f / 36.f), r9));
    const L B = Ln::fma(eps, Ln::c(1.f / 36.f), Ln::fma(es, Ln::c(1.f / 18.f), r9));
    const L X1 = Ln::mul(Ln::sub(jxs, qxs), Ln::c(1.f / 6.f)), Y1 = Ln::mul(Ln::sub(jys, qys), Ln::c(1.f / 6.f));
    const L X2 = Ln::fma(qxs, Ln::c(1.f / 12.f), Ln::mul(jxs, Ln::c(1.f / 6.f)));
    const L Y2 = Ln::fma(qys, Ln::c(1.f / 12.f), Ln::mul(jys, Ln::c(1.f / 6.f)));
    const L Pq = Ln::mul(pxxs, Ln::c(0.25f)), Rq = Ln::mul(pxys, Ln::c(0.25f));
    store(0, Ln::fma(eps, Ln::c(1.f / 9.f), Ln::fma(es, Ln::c(-1.f / 9.f), r9)));
    store(1, Ln::add(Ln::add(A, X1), Pq));
    store(2, Ln::sub(Ln::add(A, Y1), Pq));
    store(3, Ln::add(Ln::sub(A, X1), Pq));
    store(4, Ln::sub(Ln::sub(A, Y1), Pq));
    store(5, Ln::add(Ln::add(Ln::add(B, X2), Y2), Rq));
    store(6, Ln::sub(Ln::add(Ln::sub(B, X2), Y2), Rq));
    store(7, Ln::add(Ln::sub(Ln::sub(B, X2), Y2), Rq));
    store(8, Ln::sub(Ln::sub(Ln::add(B, X2), Y2), Rq));
    if (Ln::bad(rho)) *p.err = ERR_NONFINITE;
    return rho;
}

// The VP-MRT (or BGK) update of one node from its pulled populations f
// given chi and the lever arm from body_chi: moments, u_s of the body
// state bs, penalized velocity (Eq. 22), collision with forcing (Eq. 17)
// and the store of f~.  Returns chi and keeps rho, a for the solid-node
// sums.
template <int P, int COLL, class Store>
__device__ __forceinline__ bool node_collide_to(const StepParams &p, const BodyState *__restrict__ bs, bool chi,
                                                typename Prec<P>::T dxl, typename Prec<P>::T dyl,
                                                const typename Prec<P>::T f[NQ], const Store &store,
                                                typename Prec<P>::T &cr, typename Prec<P>::T &cax,
                                                typename Prec<P>::T &cay)
{
    using T = typename Prec<P>::T;
    constexpr bool DEV = Prec<P>::DEV;
    if constexpr (Prec<P>::DEV && COLL == VPLBM_COLLISION_MRT) {
        // FP32 / FP16 storage: the lane form, shared with the node-pair kernels
        float ax, ay;
        cr = mrt_dev_lanes<Lane1>(p, f, chi, dxl, dyl, bs, store, ax, ay);
        cax = ax;
        cay = ay;
        return chi;
    }
    // sums shared by the moments (rows of Eq. 15)
    const T d13 = f[1] - f[3], d24 = f[2] - f[4], b13 = f[1] + f[3], b24 = f[2] + f[4];
    const T d56 = f[5] - f[6], d87 = f[8] - f[7], a56 = f[5] + f[6], a78 = f[7] + f[8];
    const T sx = d56 + d87, ty = a56 - a78, sa = b13 + b24, sd = a56 + a78;
    const T rs = (f[0] + sa) + sd;
    const T rho = DEV ? par<T>(p.rho0, p.rho0f) + rs : rs;
    const T jx = d13 + sx;
    const T jy = d24 + ty;

    // penalized velocity, Eq. (22) in the eta-stable form
    const T inv_rho = recip(rho);
    const T gx = par<T>(p.gx, p.gxf), gy = par<T>(p.gy, p.gyf);
    T vx, vy;
    if constexpr (DEV) {   // (vx, vy) = j / rho + g / 2 as one paired FMA (g / 2 host-folded, exact)
        const float2 v = __ffma2_rn(make_float2(jx, jy), make_float2(inv_rho, inv_rho),
                                    make_float2(p.pc.hgx, p.pc.hgy));
        vx = v.x;
        vy = v.y;
    } else {
        vx = jx * inv_rho + (T)0.5 * gx;
        vy = jy * inv_rho + (T)0.5 * gy;
    }
    T ax = 0, ay = 0;
    if (chi) {
        T usx, usy;
        if constexpr (DEV) {
            const float4 vv = VPLBM_LDG(reinterpret_cast<const float4 *>(&bs->vxf));
            usx = vv.x - vv.z * dyl; usy = vv.y + vv.z * dxl;
        } else {
            usx = bs->v[0] - bs->v[2] * dyl; usy = bs->v[1] + bs->v[2] * dxl;
        }
        const T k = par<T>(p.pen_k, p.pen_kf);
        ax = -(vx - usx) * k;
        ay = -(vy - usy) * k;
    }
    const T ux = vx + (T)0.5 * ax;
    const T uy = vy + (T)0.5 * ay;
    const T Gx = rho * (gx + ax);
    const T Gy = rho * (gy + ay);

    if constexpr (COLL == VPLBM_COLLISION_BGK) {
        // Sec. 2.1: f~ = (1 - omega) f + omega f_eq + (1 - omega/2) F with
        // f_eq of Eq. (11) and F of Eq. (12), by pairs of opposite
        // directions a, a': f~_a = (1 - omega) f_a + w_a (even +- odd),
        //   even = omega (base + rho (9/2 (c.u)^2 - 3/2 u^2)) + 3k (3 (c.u)(c.G) - u.G),
        //   odd  = 3 omega rho (c.u) + 3k (c.G),   k = 1 - omega/2,
        // base = rho (FP64 storage) or rho - rho0 (deviation storage).
        const T om = par<T>(p.s[7], p.sf[7]);
        const T om1 = (T)1 - om;
        const T k3 = fma((T)-1.5, om, (T)3);
        const T k9 = (T)3 * k3;
        const T orho = om * rho;
        const T orho3 = (T)3 * orho, orho45 = (T)4.5 * orho;
        const T u2 = fma(ux, ux, uy * uy);
        const T uG = fma(ux, Gx, uy * Gy);
        const T c0 = fma(om, fma((T)-1.5 * rho, u2, DEV ? rs : rho), -k3 * uG);
        auto pair = [&](int a, int ao, T cu, T cG, T w) {
            const T we = w * fma(cu, fma(orho45, cu, k9 * cG), c0);
            const T wo = w * fma(orho3, cu, k3 * cG);
            store(a, fma(om1, f[a], we + wo));
            store(ao, fma(om1, f[ao], we - wo));
        };
        store(0, fma(om1, f[0], (T)(4.0 / 9.0) * c0));
        pair(1, 3, ux, Gx, (T)(1.0 / 9.0));
        pair(2, 4, uy, Gy, (T)(1.0 / 9.0));
        pair(5, 7, ux + uy, Gx + Gy, (T)(1.0 / 36.0));
        pair(6, 8, uy - ux, Gy - Gx, (T)(1.0 / 36.0));
        if (!(rho > (T)0) || !(rho < (T)1e30)) *p.err = ERR_NONFINITE;
        cr = rho; cax = ax; cay = ay;
        return chi;
    }

    // moments (rows of Eq. 15); equilibria (Eq. 14); M F closed form;
    // Eq. (17) with the host-folded factors 1 - s_k and (1 - s_k/2)
    const T e = fma((T)-4, f[0], fma((T)2, sd, -sa));
    const T ep = fma((T)4, f[0], fma((T)-2, sa, sd));
    const T qx = fma((T)-2, d13, sx);
    const T qy = fma((T)-2, d24, ty);
    const T pxx = b13 - b24;
    const T pxy = (f[5] + f[7]) - (f[6] + f[8]);

    const auto &k = folded<T>(p);
    T e_s, ep_s, A, B, X1, Y1, X2, Y2, Pq, Rq, r9;
    if constexpr (DEV) {
        // the same operations with the (x, y) and (e, eps) pairs on the
        // paired FP32 instructions (each lane rounds like the scalar op)
        const float2 U = make_float2(ux, uy), G = make_float2(Gx, Gy);
        const float2 rr = make_float2(rho, rho);
        const float2 U2 = __fmul2_rn(U, U);
        const T u2r = rho * (U2.x + U2.y);
        const T uG = fma(ux, Gx, uy * Gy);
        const float2 t1 = __ffma2_rn(make_float2(3.f, -3.f), make_float2(u2r, u2r), make_float2(-2.f * rs, rs));
        const float2 t2 = __fmul2_rn(make_float2(k.h1x6, k.mh2x6), make_float2(uG, uG));
        const float2 t3 = __ffma2_rn(make_float2(p.sf[1], p.sf[2]), t1, t2);
        const float2 ES = __ffma2_rn(make_float2(k.om1, k.om2), make_float2(e, ep), t3);
        e_s = ES.x;
        ep_s = ES.y;
        const float2 JS = __fadd2_rn(make_float2(jx, jy), G);
        const float2 Q = make_float2(qx, qy);
        const float2 QS = __ffma2_rn(make_float2(k.om4, k.om6), Q,
                                     __ffma2_rn(make_float2(-p.sf[4], -p.sf[6]), __fmul2_rn(rr, U),
                                                __fmul2_rn(make_float2(k.mh4, k.mh6), G)));
        const float2 D = make_float2(U2.x - U2.y, ux * uy);
        const float2 C = make_float2(fma(ux, Gx, -uy * Gy), fma(ux, Gy, uy * Gx));
        const float2 PS = __ffma2_rn(make_float2(k.om7, k.om8), make_float2(pxx, pxy),
                                     __ffma2_rn(make_float2(p.sf[7], p.sf[8]), __fmul2_rn(rr, D),
                                                __fmul2_rn(make_float2(k.h7x2, k.h8), C)));
        r9 = rs * (T)(1.0 / 9.0);
        A = r9 - e_s * (T)(1.0 / 36.0) - ep_s * (T)(1.0 / 18.0);
        B = r9 + e_s * (T)(1.0 / 18.0) + ep_s * (T)(1.0 / 36.0);
        const float2 XY1 = __fmul2_rn(__ffma2_rn(QS, make_float2(-1.f, -1.f), JS), make_float2(1.f / 6.f, 1.f / 6.f));
        const float2 XY2 = __ffma2_rn(QS, make_float2(1.f / 12.f, 1.f / 12.f), __fmul2_rn(JS, make_float2(1.f / 6.f, 1.f / 6.f)));
        const float2 PR = __fmul2_rn(PS, make_float2(0.25f, 0.25f));
        X1 = XY1.x; Y1 = XY1.y; X2 = XY2.x; Y2 = XY2.y; Pq = PR.x; Rq = PR.y;
    } else {
        const T ux2 = ux * ux, uy2 = uy * uy;
        const T u2r = rho * (ux2 + uy2);
        const T uG = fma(ux, Gx, uy * Gy);
        e_s = fma((T)k.om1, e, fma(par<T>(p.s[1], p.sf[1]), fma((T)3, u2r, (T)-2 * rs), (T)k.h1x6 * uG));
        ep_s = fma((T)k.om2, ep, fma(par<T>(p.s[2], p.sf[2]), fma((T)-3, u2r, rs), (T)k.mh2x6 * uG));
        const T jx_s = jx + Gx;
        const T jy_s = jy + Gy;
        const T qx_s = fma((T)k.om4, qx, fma(-par<T>(p.s[4], p.sf[4]), rho * ux, (T)k.mh4 * Gx));
        const T qy_s = fma((T)k.om6, qy, fma(-par<T>(p.s[6], p.sf[6]), rho * uy, (T)k.mh6 * Gy));
        const T pxx_s = fma((T)k.om7, pxx, fma(par<T>(p.s[7], p.sf[7]), rho * (ux2 - uy2), (T)k.h7x2 * fma(ux, Gx, -uy * Gy)));
        const T pxy_s = fma((T)k.om8, pxy, fma(par<T>(p.s[8], p.sf[8]), rho * (ux * uy), (T)k.h8 * fma(ux, Gy, uy * Gx)));

        // back to populations, M^-1 = M^T diag(1/|row|^2)
        r9 = rs * (T)(1.0 / 9.0);
        A = r9 - e_s * (T)(1.0 / 36.0) - ep_s * (T)(1.0 / 18.0);
        B = r9 + e_s * (T)(1.0 / 18.0) + ep_s * (T)(1.0 / 36.0);
        X1 = (jx_s - qx_s) * (T)(1.0 / 6.0);
        Y1 = (jy_s - qy_s) * (T)(1.0 / 6.0);
        X2 = jx_s * (T)(1.0 / 6.0) + qx_s * (T)(1.0 / 12.0);
        Y2 = jy_s * (T)(1.0 / 6.0) + qy_s * (T)(1.0 / 12.0);
        Pq = pxx_s * (T)0.25;
        Rq = pxy_s * (T)0.25;
    }

    store(0, r9 - e_s * (T)(1.0 / 9.0) + ep_s * (T)(1.0 / 9.0));
    store(1, A + X1 + Pq);
    store(2, A + Y1 - Pq);
    store(3, A - X1 + Pq);
    store(4, A - Y1 - Pq);
    store(5, B + X2 + Y2 + Rq);
    store(6, B - X2 + Y2 - Rq);
    store(7, B - X2 - Y2 + Rq);
    store(8, B + X2 - Y2 - Rq);

    if (!(rho > (T)0) || !(rho < (T)1e30)) *p.err = ERR_NONFINITE;
    cr = rho; cax = ax; cay = ay;
    return chi;
}

// node_collide_to storing f~ into the step's destination buffer.
template <int P, int COLL>
__device__ __forceinline__ bool node_collide(const StepParams &p, const BodyState *__restrict__ bs, bool chi,
                                             typename Prec<P>::T dxl, typename Prec<P>::T dyl, int i, int j,
                                             const typename Prec<P>::T f[NQ], typename Prec<P>::S *__restrict__ fout,
                                             typename Prec<P>::T &cr, typename Prec<P>::T &cax,
                                             typename Prec<P>::T &cay)
{
    using S = typename Prec<P>::S;
    using T = typename Prec<P>::T;
    S *const *dp = reinterpret_cast<S *const *>(p.dst_plane);
    const int b = j * p.nx + i;
    (void)fout;
    return node_collide_to<P, COLL>(p, bs, chi, dxl, dyl, f, [&](int a, T v) { stv(dp[a] + b, v); }, cr, cax, cay);
}

// The update of one interior-or-edge node of a lattice with one body: chi
// where the body can be (near_body, uniform over the block), then
// node_collide.
template <int P, int COLL = VPLBM_COLLISION_MRT, int SHAPE = SHAPE_ANY>
__device__ __forceinline__ bool node_update(const StepParams &p, const BodyState *__restrict__ bs, bool near_body,
                                            int i, int j, const typename Prec<P>::T f[NQ],
                                            typename Prec<P>::S *__restrict__ fout, typename Prec<P>::T &cr,
                                            typename Prec<P>::T &cax, typename Prec<P>::T &cay)
{
    typename Prec<P>::T dxl = 0, dyl = 0;
    bool chi = false;
    if (near_body) chi = body_chi<P, SHAPE>(p.body, p.r2f, bs, i, j, dxl, dyl);
    return node_collide<P, COLL>(p, bs, chi, dxl, dyl, i, j, f, fout, cr, cax, cay);
}

// Does the tile [i0, i0+w) x [j0, j0+h) meet the node range that may hold
// solid nodes?  With no solid node anywhere, tile (0, 0) stands in so that
// one block still runs the tail.
__device__ __forceinline__ bool tile_near_body(const int4 range, int i0, int j0, int w, int h, bool first_tile)
{
    if (range.x > range.y) return first_tile;
    return i0 + w - 1 >= range.x && i0 <= range.y && j0 + h - 1 >= range.z && j0 <= range.w;
}

// Partial slot of tile (tx, ty) of a w x h tiling, the ticket, and the
// tail in the last tile to publish.  sums (shared memory) holds the tile's
// 7 sums in accumulator type A; every thread of the block calls it (it
// contains block barriers).
// publish_slot: the same with the slot and the number of partials given.
template <typename A>
__device__ __forceinline__ void publish_slot(const StepParams &p, int slot, int nparts, const A *sums, int *s_last)
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    if (nparts > p.max_parts) {          // cannot happen for a finite pose; never overrun
        if (tid == 0) *p.err |= ERR_INTERNAL;
        __syncthreads();
        return;
    }
    if (tid == 0) {
        A *dst = reinterpret_cast<A *>(p.partials + (size_t)slot * NPART);
#pragma unroll
        for (int k = 0; k < NPART - 1; ++k) __stcg(dst + k, sums[k]);
        __threadfence();
        const unsigned t = atomicAdd(p.ticket, 1u);
        *s_last = (t == (unsigned)(nparts - 1));
    }
    __syncthreads();
    if (*s_last && tid < 32) {
        __threadfence();
        step_tail<A>(p, nparts);
    }
    __syncthreads();   // the shared scratch and s_last are reused by the next tile
}

template <typename A>
__device__ __forceinline__ void publish_tile(const StepParams &p, const int4 range, int tx, int ty, int w, int h,
                                             const A *sums, int *s_last)
{
    int tx0 = 0, tx1 = 0, ty0 = 0, ty1 = 0;
    if (range.x <= range.y) {
        tx0 = range.x / w; tx1 = range.y / w;
        ty0 = range.z / h; ty1 = range.w / h;
    }
    const int ntx = tx1 - tx0 + 1;
    const int nparts = ntx * (ty1 - ty0 + 1);
    publish_slot<A>(p, (ty - ty0) * ntx + (tx - tx0), nparts, sums, s_last);
}

// Block-wide fixed-order reduction of per-thread accumulators (type A:
// double, or float2 float-float), then publish_tile.  Used where a thread
// has accumulated several nodes (TMA-staged kernel).
// block_reduce leaves the block's sums in red_mem[0] (type A).
template <typename A>
__device__ __forceinline__ void block_reduce(bool any_chi_thread, A part[NPART - 1], double (*red_mem)[NPART])
{
    static_assert(sizeof(A) == sizeof(double), "the shared scratch holds one A per entry");
    A (*red)[NPART] = reinterpret_cast<A (*)[NPART]>(red_mem);
    const int nthreads = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nwarps = nthreads >> 5;
    if (__any_sync(0xffffffffu, any_chi_thread)) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < NPART - 1; ++k) acc_add(part[k], acc_shfl_down(part[k], off));
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NPART - 1; ++k) red[warp][k] = part[k];
    __syncthreads();
    if (warp == 0) {
        A v[NPART - 1];
#pragma unroll
        for (int k = 0; k < NPART - 1; ++k) {
            if (lane < nwarps) v[k] = red[lane][k];
            else acc_zero(v[k]);
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1)
#pragma unroll
            for (int k = 0; k < NPART - 1; ++k) acc_add(v[k], acc_shfl_down(v[k], off));
        __syncwarp();
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NPART - 1; ++k) red[0][k] = v[k];
    }
    __syncthreads();
}

template <typename A>
__device__ __forceinline__ void tile_reduce(const StepParams &p, const int4 range, int tx, int ty, int w, int h,
                                            bool any_chi_thread, A part[NPART - 1], double (*red_mem)[NPART],
                                            int *s_last)
{
    block_reduce<A>(any_chi_thread, part, red_mem);
    publish_tile<A>(p, range, tx, ty, w, h, reinterpret_cast<A *>(red_mem[0]), s_last);
}

// Solid-node sums of a tile where every thread owns one node: the terms go
// to shared memory as rows [quantity][thread], and warp q reduces row q
// (8 float-float adds per lane in thread order, then a shuffle tree), so
// the 7 quantities are summed by 7 warps at once instead of one after the
// other by every warp.  rows holds 7 x 256 floats.
template <int P>
__device__ __forceinline__ void tile_solid_sums(const StepParams &p, const typename Prec<P>::S *fin, const int4 range,
                                                int tx, int ty, int w, int h, bool chi, int i, int j,
                                                typename Prec<P>::T rho, typename Prec<P>::T ax,
                                                typename Prec<P>::T ay, double (*red)[NPART], float (*rows)[256],
                                                int *s_last)
{
    using A = typename SumT<P>::A;
    using V = typename SumT<P>::V;
    if constexpr (P == VPLBM_F64) {
        (void)rows;
        A part[NPART - 1];
#pragma unroll
        for (int k = 0; k < NPART - 1; ++k) acc_zero(part[k]);
        if (chi) {
            V one[NPART - 1];
            solid_node_terms<P>(p, fin, i, j, (V)rho, (V)ax, (V)ay, one);
#pragma unroll
            for (int k = 0; k < NPART - 1; ++k) acc_add(part[k], one[k]);
        }
        tile_reduce<A>(p, range, tx, ty, w, h, chi, part, red, s_last);
    } else {
        const int nthreads = blockDim.x * blockDim.y;
        const int tid = threadIdx.y * blockDim.x + threadIdx.x;
        const int lane = tid & 31, warp = tid >> 5, nwarps = nthreads >> 5;
        float one[NPART - 1];
#pragma unroll
        for (int k = 0; k < NPART - 1; ++k) one[k] = 0.f;
        if (chi) solid_node_terms<P>(p, fin, i, j, (float)rho, (float)ax, (float)ay, one);
#pragma unroll
        for (int k = 0; k < NPART - 1; ++k) rows[k][tid] = one[k];
        __syncthreads();
        float2 *sums = reinterpret_cast<float2 *>(red[0]);
        for (int q = warp; q < NPART - 1; q += nwarps) {
            float2 a = make_float2(0.f, 0.f);
            for (int t = lane; t < nthreads; t += 32) acc_add(a, rows[q][t]);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc_add(a, acc_shfl_down(a, off));
            if (lane == 0) sums[q] = a;
        }
        __syncthreads();
        publish_tile<float2>(p, range, tx, ty, w, h, sums, s_last);
    }
}

}  // namespace
}  // namespace vplbm
