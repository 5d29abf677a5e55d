// Reverse-time discrete adjoint of the fused step for a body on a prescribed
// path (fixed or imposed motion), with sqrt(N) checkpointing.
//
// State S_n = post-collision populations entering step n; one step is
// S_{n+1}(x) = C(Pull(S_n)(x)); the force of step n is
// F_h(n) = sum_{x in R(n)} [j(Pull(S_n))(x) - j(S_n)(x)] (Eqs. 25-27 as a
// node sum).  With J = w_cd mean C_D + w_cl RMS C_L over [w0, N), the
// reverse sweep carries L_n = dJ/dS_n:
//   (a) mu(x) = (dC/df)^T L_{n+1}(x) + [x in R(n)] dJ/dF_h(n) . c   (node local)
//   (b) L_n(y) = (Pull^T mu)(y) - [y in R(n)] dJ/dF_h(n) . c        (a gather)
// and the parameter gradients: dJ/ds_e, dJ/ds_nu (= s7 = s8), dJ/deta from
// (a), dJ/du_in(j) of the west wall's u_x profile from (b).
// The reverse of C is written on the closed-form moments of the forward
// kernel (vplbm_node.cuh): M^-T = diag(1/|row|^2) M for the incoming
// adjoint, M^T for the outgoing one.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <new>
#include <vector>

#include "vplbm_ctx.cuh"
#include "vplbm_node.cuh"

namespace vplbm {
namespace {

// Per-step inputs of the reverse kernels, with the FP32 copies and the
// pose-derived values the FP32 kernels use (no FP64 on their main path:
// GB300's FP64 pipe is narrow).
struct AdjStep {
    double xg, yg, vx, vy, om;   // pose and velocity of step n
    double wx, wy;               // dJ/dF_h(n)
    int ilo, ihi, jlo, jhi;      // node range that may be solid (ilo > ihi: none)
    int xi, yi;                  // floor(x_G), floor(y_G)
    float xf, yf;                // x_G - xi, y_G - yi
    float vxf, vyf, omf, wxf, wyf;
};

// chi of node (i, j) at the pose of a, decided exactly as by the forward
// kernel (FP32 test relative to floor(x_G), FP64 re-test inside the band).
template <typename T>
__device__ __forceinline__ bool chi_adj(const StepParams &p, const AdjStep &a, int i, int j, T &dx, T &dy)
{
    dx = 0;
    dy = 0;
    if (!p.body.present || i < a.ilo || i > a.ihi || j < a.jlo || j > a.jhi) return false;
    if constexpr (sizeof(T) == 4) {
        dx = (float)(i - a.xi) - a.xf;
        dy = (float)(j - a.yi) - a.yf;
        const float d2 = dx * dx + dy * dy;
        const float r2 = p.r2f;
        if (fabsf(d2 - r2) <= 1e-5f * r2 + 1e-5f) return chi_exact(i, j, a.xg, a.yg, p.body.r2);
        return d2 <= r2;
    } else {
        dx = (double)i - a.xg;
        dy = (double)j - a.yg;
        return chi_exact(i, j, a.xg, a.yg, p.body.r2);
    }
}

// Moments of a 9-vector with the rows of Eq. (15): (rho, e, eps, jx, qx, jy, qy, pxx, pxy).
template <typename T> __device__ __forceinline__ void moments9(const T f[NQ], T m[NQ])
{
    const T sa = (f[1] + f[2]) + (f[3] + f[4]);
    const T sd = (f[5] + f[6]) + (f[7] + f[8]);
    m[0] = f[0] + sa + sd;
    m[1] = (T)-4 * f[0] - sa + (T)2 * sd;
    m[2] = (T)4 * f[0] - (T)2 * sa + sd;
    m[3] = (f[1] - f[3]) + (f[5] - f[6]) + (f[8] - f[7]);
    m[4] = (T)2 * (f[3] - f[1]) + (f[5] - f[6]) + (f[8] - f[7]);
    m[5] = (f[2] - f[4]) + (f[5] + f[6]) - (f[7] + f[8]);
    m[6] = (T)2 * (f[4] - f[2]) + (f[5] + f[6]) - (f[7] + f[8]);
    m[7] = (f[1] + f[3]) - (f[2] + f[4]);
    m[8] = (f[5] + f[7]) - (f[6] + f[8]);
}

// M^T applied to moment-space values (column a of M dotted with L).
template <typename T> __device__ __forceinline__ void mt9(const T L[NQ], T out[NQ])
{
    out[0] = L[0] - (T)4 * L[1] + (T)4 * L[2];
    out[1] = L[0] - L[1] - (T)2 * L[2] + L[3] - (T)2 * L[4] + L[7];
    out[2] = L[0] - L[1] - (T)2 * L[2] + L[5] - (T)2 * L[6] - L[7];
    out[3] = L[0] - L[1] - (T)2 * L[2] - L[3] + (T)2 * L[4] + L[7];
    out[4] = L[0] - L[1] - (T)2 * L[2] - L[5] + (T)2 * L[6] - L[7];
    out[5] = L[0] + (T)2 * L[1] + L[2] + L[3] + L[4] + L[5] + L[6] + L[8];
    out[6] = L[0] + (T)2 * L[1] + L[2] - L[3] - L[4] + L[5] + L[6] - L[8];
    out[7] = L[0] + (T)2 * L[1] + L[2] - L[3] - L[4] - L[5] - L[6] + L[8];
    out[8] = L[0] + (T)2 * L[1] + L[2] + L[3] + L[4] - L[5] - L[6] - L[8];
}

// (a) mu = (dC/df)^T lam_next + objective term; parameter-gradient partials
// acc[block][0..3] += (d_eta, d_s1, d_s7, d_s8).
template <int P>
__global__ void __launch_bounds__(256) adj_collide(const StepParams p, const AdjStep a, const typename Prec<P>::T *lam_next,
                                                   typename Prec<P>::T *mu, double *acc)
{
    using T = typename Prec<P>::T;
    using S = typename Prec<P>::S;
    constexpr bool DEV = Prec<P>::DEV;
    __shared__ double red[8][4];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    T g4[4] = {0, 0, 0, 0};
    if (i < p.nx) {
        const S *fin = static_cast<const S *>(p.fin);
        T f[NQ];
        pull_all<P>(p, fin, i, j, f);
        const long long b = (long long)j * p.nx + i;
        T xi[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) xi[q] = lam_next[q * p.ps + b];

        // forward intermediates (as in node_update)
        T m[NQ];
        moments9<T>(f, m);
        const T rs = m[0];
        const T rho = DEV ? par<T>(p.rho0, p.rho0f) + rs : rs;
        const T inv_rho = recip(rho);
        const T jx = m[3], jy = m[5];
        T dx, dy;
        const bool chi = chi_adj<T>(p, a, i, j, dx, dy);
        const T gx = par<T>(p.gx, p.gxf), gy = par<T>(p.gy, p.gyf);
        const T vx = jx * inv_rho + (T)0.5 * gx, vy = jy * inv_rho + (T)0.5 * gy;
        T ax = 0, ay = 0, usx = 0, usy = 0, k = 0;
        if (chi) {
            usx = par<T>(a.vx, a.vxf) - par<T>(a.om, a.omf) * dy;
            usy = par<T>(a.vy, a.vyf) + par<T>(a.om, a.omf) * dx;
            k = par<T>(p.pen_k, p.pen_kf);
            ax = -k * (vx - usx);
            ay = -k * (vy - usy);
        }
        const T ux = vx + (T)0.5 * ax, uy = vy + (T)0.5 * ay;
        const T Gx = rho * (gx + ax), Gy = rho * (gy + ay);
        const T u2r = rho * (ux * ux + uy * uy);
        const T uG = ux * Gx + uy * Gy;
        const T W1 = rho * (ux * ux - uy * uy), W2 = ux * Gx - uy * Gy;
        const T W3 = rho * ux * uy, W4 = ux * Gy + uy * Gx;
        const T s1 = par<T>(p.s[1], p.sf[1]), s2 = par<T>(p.s[2], p.sf[2]), s4 = par<T>(p.s[4], p.sf[4]);
        const T s6 = par<T>(p.s[6], p.sf[6]), s7 = par<T>(p.s[7], p.sf[7]), s8 = par<T>(p.s[8], p.sf[8]);
        const T h1 = (T)1 - (T)0.5 * s1, h2 = (T)1 - (T)0.5 * s2, h4 = (T)1 - (T)0.5 * s4;
        const T h6 = (T)1 - (T)0.5 * s6, h7 = (T)1 - (T)0.5 * s7, h8 = (T)1 - (T)0.5 * s8;

        // adjoint of the post-collision moments: M^-T xi = diag(1/|row|^2) M xi
        T L[NQ];
        moments9<T>(xi, L);
        L[0] *= (T)(1.0 / 9.0); L[1] *= (T)(1.0 / 36.0); L[2] *= (T)(1.0 / 36.0);
        L[3] *= (T)(1.0 / 6.0); L[4] *= (T)(1.0 / 12.0); L[5] *= (T)(1.0 / 6.0);
        L[6] *= (T)(1.0 / 12.0); L[7] *= (T)0.25; L[8] *= (T)0.25;

        // parameter partials (before L is consumed)
        const T e_eq = (T)-2 * rs + (T)3 * u2r;
        g4[1] = L[1] * (-(m[1] - e_eq) - (T)3 * uG);
        g4[2] = L[7] * (-(m[7] - W1) - W2);
        g4[3] = L[8] * (-(m[8] - W3) - (T)0.5 * W4);

        // back through the relaxation (Eq. 17 in closed form)
        T lm[NQ];   // adjoint of the pre-collision moments
        lm[1] = ((T)1 - s1) * L[1];
        lm[2] = ((T)1 - s2) * L[2];
        lm[4] = ((T)1 - s4) * L[4];
        lm[6] = ((T)1 - s6) * L[6];
        lm[7] = ((T)1 - s7) * L[7];
        lm[8] = ((T)1 - s8) * L[8];
        T l_rs = L[0] - (T)2 * s1 * L[1] + s2 * L[2];
        const T l_u2r = (T)3 * s1 * L[1] - (T)3 * s2 * L[2];
        const T l_uG = (T)6 * h1 * L[1] - (T)6 * h2 * L[2];
        T l_jx = L[3], l_jy = L[5];
        T l_Gx = L[3] - h4 * L[4], l_Gy = L[5] - h6 * L[6];
        T l_rho = -s4 * L[4] * ux - s6 * L[6] * uy;
        T l_ux = -s4 * L[4] * rho, l_uy = -s6 * L[6] * rho;
        const T lW1 = s7 * L[7], lW2 = (T)2 * h7 * L[7], lW3 = s8 * L[8], lW4 = h8 * L[8];
        l_rho += lW1 * (ux * ux - uy * uy) + lW3 * ux * uy + l_u2r * (ux * ux + uy * uy);
        l_ux += lW1 * (T)2 * rho * ux + lW2 * Gx + lW3 * rho * uy + lW4 * Gy + l_u2r * (T)2 * rho * ux + l_uG * Gx;
        l_uy += -lW1 * (T)2 * rho * uy - lW2 * Gy + lW3 * rho * ux + lW4 * Gx + l_u2r * (T)2 * rho * uy + l_uG * Gy;
        l_Gx += lW2 * ux + lW4 * uy + l_uG * ux;
        l_Gy += -lW2 * uy + lW4 * ux + l_uG * uy;
        // G = rho (g + a)
        l_rho += l_Gx * (gx + ax) + l_Gy * (gy + ay);
        T l_ax = rho * l_Gx + (T)0.5 * l_ux, l_ay = rho * l_Gy + (T)0.5 * l_uy;
        T l_vx = l_ux, l_vy = l_uy;
        if (chi) {
            l_vx += -k * l_ax;
            l_vy += -k * l_ay;
            g4[0] = k * k * ((vx - usx) * l_ax + (vy - usy) * l_ay);
        }
        // v = j / rho + g/2
        l_jx += l_vx * inv_rho;
        l_jy += l_vy * inv_rho;
        l_rho += -(l_vx * jx + l_vy * jy) * (inv_rho * inv_rho);
        l_rs += l_rho;
        lm[0] = l_rs;
        lm[3] = l_jx;
        lm[5] = l_jy;
        T out[NQ];
        mt9<T>(lm, out);
        if (chi) {
            const T wx = par<T>(a.wx, a.wxf), wy = par<T>(a.wy, a.wyf);
#pragma unroll
            for (int q = 0; q < NQ; ++q) out[q] += (T)cx_of(q) * wx + (T)cy_of(q) * wy;
        }
#pragma unroll
        for (int q = 0; q < NQ; ++q) mu[q * p.ps + b] = out[q];
    }
    // deterministic block sums of the parameter partials
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        T v = g4[q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[warp][q] = (double)v;
    }
    __syncthreads();
    if (tid < 4) {
        double s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][tid];
        double *dst = acc + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 4 + tid;
        *dst += s;
    }
}

// Is the pull of population a into node (i, j) a plain (possibly periodic)
// pull, a wall rule (then *side), or a zero-gradient copy?
enum { PULL_PLAIN = 0, PULL_WALL = 1, PULL_ZEROGRAD = 2 };
__device__ __forceinline__ int pull_kind(const StepParams &p, int a, int i, int j, int *side)
{
    const int si = i - cx_of(a), sj = j - cy_of(a);
    if (sj < 0 || sj >= p.ny) {
        const int sd = sj < 0 ? VPLBM_SOUTH : VPLBM_NORTH;
        if (p.bc[sd] != VPLBM_BC_PERIODIC) { *side = sd; return PULL_WALL; }
    }
    if (si < 0 || si >= p.nx) {
        const int sd = si < 0 ? VPLBM_WEST : VPLBM_EAST;
        if (p.bc[sd] == VPLBM_BC_ZEROGRAD) return PULL_ZEROGRAD;
        if (p.bc[sd] != VPLBM_BC_PERIODIC) { *side = sd; return PULL_WALL; }
    }
    return PULL_PLAIN;
}

// (b) L_n(y) = sum of mu over the pulls that read population (b, y), minus
// the momentum-exchange own term; west velocity-wall pulls give dJ/du_in.
template <int P>
__global__ void __launch_bounds__(256) adj_stream(const StepParams p, const AdjStep a, const typename Prec<P>::T *mu,
                                                  typename Prec<P>::T *lam, double *grad_uin)
{
    using T = typename Prec<P>::T;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= p.nx) return;
    const int nx = p.nx, ny = p.ny;
    const long long ps = p.ps;
    auto MU = [&](int q, int ii, int jj) { return mu[q * ps + (long long)jj * nx + ii]; };
    T dxu, dyu;
    const bool chi = chi_adj<T>(p, a, i, j, dxu, dyu);
    const T wx = par<T>(a.wx, a.wxf), wy = par<T>(a.wy, a.wyf);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        T acc = 0;
        // plain pull into (q, y + c_q), with periodic wrap
        int ti = i + cx_of(q), tj = j + cy_of(q);
        bool ok = true;
        if (tj < 0 || tj >= ny) {
            if (p.bc[tj < 0 ? VPLBM_SOUTH : VPLBM_NORTH] == VPLBM_BC_PERIODIC) tj = (tj + ny) % ny;
            else ok = false;
        }
        if (ok && (ti < 0 || ti >= nx)) {
            if (p.bc[ti < 0 ? VPLBM_WEST : VPLBM_EAST] == VPLBM_BC_PERIODIC) ti = (ti + nx) % nx;
            else ok = false;
        }
        if (ok) {
            int sd;
            if (pull_kind(p, q, ti, tj, &sd) == PULL_PLAIN) acc += MU(q, ti, tj);
        }
        // wall pull into (opp(q), y) reads (q, y)
        {
            int sd;
            if (pull_kind(p, opp_of(q), i, j, &sd) == PULL_WALL) acc += MU(opp_of(q), i, j);
        }
        // zero-gradient pull into (q, (i, j + c_qy)) reads (q, (i, j)) at an edge column
        if (cx_of(q) != 0 && ((cx_of(q) == 1 && i == 0) || (cx_of(q) == -1 && i == nx - 1))) {
            int zj = j + cy_of(q);
            bool zok = true;
            if (zj < 0 || zj >= ny) {
                if (p.bc[zj < 0 ? VPLBM_SOUTH : VPLBM_NORTH] == VPLBM_BC_PERIODIC) zj = (zj + ny) % ny;
                else zok = false;
            }
            if (zok) {
                int sd;
                if (pull_kind(p, q, i, zj, &sd) == PULL_ZEROGRAD) acc += MU(q, i, zj);
            }
        }
        if (chi) acc -= (T)cx_of(q) * wx + (T)cy_of(q) * wy;
        lam[q * ps + (long long)j * nx + i] = acc;
    }
    // inlet profile: the west velocity-wall pulls of this node
    if (i == 0 && grad_uin && p.bc[VPLBM_WEST] == VPLBM_BC_VELOCITY && p.wall_prof[VPLBM_WEST][0]) {
        double g = 0;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            if (cx_of(q) != 1) continue;
            int sd = -1;
            if (pull_kind(p, q, i, j, &sd) == PULL_WALL && sd == VPLBM_WEST)
                g += (double)MU(q, i, j) * 6.0 * w_of(q) * p.rho0;
        }
        grad_uin[j] += g;
    }
}

template <int P>
cudaError_t launch_adjoint_step(const StepParams &p, const AdjStep &a, const void *lam_next, void *mu, void *lam,
                                double *acc, double *grad_uin, cudaStream_t stream)
{
    using T = typename Prec<P>::T;
    dim3 block(256);
    dim3 grid((p.nx + 255) / 256, p.ny);
    adj_collide<P><<<grid, block, 0, stream>>>(p, a, static_cast<const T *>(lam_next), static_cast<T *>(mu), acc);
    adj_stream<P><<<grid, block, 0, stream>>>(p, a, static_cast<const T *>(mu), static_cast<T *>(lam), grad_uin);
    return cudaGetLastError();
}

vplbm_status aerr(vplbm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return report_error(st, buf);
}

}  // namespace
}  // namespace vplbm

using namespace vplbm;

extern "C" vplbm_status vplbm_adjoint(vplbm_ctx *c, const vplbm_adjoint_desc *d, double *grad, double *j_out)
{
    if (!c || !d || !grad) return aerr(VPLBM_EINVAL, "NULL argument");
    if (c->precision != VPLBM_F64 && c->precision != VPLBM_F32_DEV)
        return aerr(VPLBM_EUNSUPPORTED, "the adjoint runs FP64 or FP32 deviation storage");
    if (c->has_body && c->body_desc.motion == VPLBM_MOTION_FREE)
        return aerr(VPLBM_EUNSUPPORTED, "the adjoint needs a body on a prescribed path (fixed or imposed)");
    if (c->collision != VPLBM_COLLISION_MRT) return aerr(VPLBM_EUNSUPPORTED, "the adjoint differentiates the MRT operator only");
    if (c->has_body && c->body_desc.shape != VPLBM_SHAPE_DISK) return aerr(VPLBM_EUNSUPPORTED, "the adjoint takes a disk");
    if (c->nbodies > 1) return aerr(VPLBM_EUNSUPPORTED, "the adjoint takes one body");
    for (int e = VPLBM_SOUTH; e <= VPLBM_NORTH; ++e)
        if (c->base.bc[e] == VPLBM_BC_SYMMETRY) return aerr(VPLBM_EUNSUPPORTED, "the adjoint has no symmetry-wall rule");
    if (c->base.bc[VPLBM_EAST] == VPLBM_BC_CONVECTIVE) return aerr(VPLBM_EUNSUPPORTED, "the adjoint has no convective-outlet rule");
    const long long N = d->nsteps;
    if (N < 1 || d->window_start < 0 || d->window_start >= N) return aerr(VPLBM_EINVAL, "need 0 <= window_start < nsteps");
    if (c->hist_cap < N) return aerr(VPLBM_EINVAL, "history capacity %lld < nsteps %lld", c->hist_cap, N);
    const long long K = d->checkpoint_interval > 0 ? d->checkpoint_interval : (long long)ceil(sqrt((double)N));
    const long long nck = (N + K - 1) / K;
    const size_t es = c->precision == VPLBM_F64 ? 8 : 4;
    const size_t pop = c->pop_bytes;
    const size_t lam_bytes = (size_t)9 * c->ps * es;
    cudaStream_t st = c->stream;
    const long long step0 = c->nstep;

    char *ckpt = nullptr, *store = nullptr, *work = nullptr;
    double *dacc = nullptr;
    void *final_f = nullptr;
    BodyState final_bs[2];
    const dim3 grid((c->nx + 255) / 256, c->ny);
    const size_t nacc = (size_t)grid.x * grid.y * 4;
    auto cleanup = [&]() {
        cudaFree(ckpt); cudaFree(store); cudaFree(work); cudaFree(dacc); cudaFree(final_f);
    };
#define ATRY(expr)                                                                     \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            cleanup();                                                                 \
            return aerr(VPLBM_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));  \
        }                                                                              \
    } while (0)
    ATRY(cudaMalloc(&ckpt, pop * nck));
    ATRY(cudaMalloc(&store, pop * K));
    ATRY(cudaMalloc(&work, lam_bytes * 3));
    ATRY(cudaMalloc(&dacc, (nacc + (size_t)c->ny) * sizeof(double)));
    ATRY(cudaMalloc(&final_f, pop));
    double *grad_uin = dacc + nacc;
    ATRY(cudaMemsetAsync(work, 0, lam_bytes * 3, st));
    ATRY(cudaMemsetAsync(dacc, 0, (nacc + c->ny) * sizeof(double), st));

    // forward with a checkpoint every K steps
    for (long long s = 0; s < nck; ++s) {
        ATRY(cudaMemcpyAsync(ckpt + pop * s, c->f[c->nstep & 1], pop, cudaMemcpyDeviceToDevice, st));
        vplbm_status r = vplbm_step(c, std::min(K, N - s * K));
        if (r != VPLBM_OK) { cleanup(); return r; }
    }
    vplbm_status r = vplbm_sync(c);
    if (r != VPLBM_OK) { cleanup(); return r; }
    // keep the final state to restore after the recomputations
    ATRY(cudaMemcpyAsync(final_f, c->f[c->nstep & 1], pop, cudaMemcpyDeviceToDevice, st));
    ATRY(cudaMemcpyAsync(final_bs, c->bs, sizeof final_bs, cudaMemcpyDeviceToHost, st));
    const long long nfinal = c->nstep;

    // objectives and dJ/dF_h(n) from the recorded forces
    std::vector<vplbm_record> h;
    try {
        h.resize((size_t)N);
    } catch (...) {
        cleanup();
        return aerr(VPLBM_ENOMEM, "host allocation failed");
    }
    r = vplbm_get_history(c, step0, N, h.data());
    if (r != VPLBM_OK) { cleanup(); return r; }
    const double qref = c->base.body.qref;
    const double nh = (double)(N - d->window_start);
    double scd = 0, scl2 = 0;
    for (long long n = d->window_start; n < N; ++n) {
        scd += h[n].fx / qref;
        scl2 += (h[n].fy / qref) * (h[n].fy / qref);
    }
    const double J1 = qref > 0 ? scd / nh : 0.0, J2 = qref > 0 ? sqrt(scl2 / nh) : 0.0;
    if (j_out) { j_out[0] = J1; j_out[1] = J2; }

    // reverse sweep, segment by segment; the recomputation runs the
    // context's scalar step kernel (a TMA-staged choice falls back to the
    // 48-register scalar kernel on 256 x 1 blocks, a two-step choice to its
    // single-step blocks)
    const bool scalar = c->kernel != KERNEL_TMA;
    const int rbx = scalar ? c->bx : 256, rby = scalar ? c->by : 1;
    const int rminb = !scalar ? 5 : c->kernel == KERNEL_SCALAR_40 || c->kernel == KERNEL_FUSED2 ? 6 : c->kernel == KERNEL_SCALAR_48 ? 5 : 4;
    int cur = 0;   // work: lam[0], lam[1], mu
    for (long long s = nck - 1; s >= 0; --s) {
        const long long s0 = s * K, len = std::min(K, N - s0);
        // recompute the segment's states S_{s0} .. S_{s0+len-1}
        c->nstep = step0 + s0;
        BodyState b{};
        b.q[0] = h[s0].x; b.q[1] = h[s0].y; b.q[2] = h[s0].theta;
        b.v[0] = h[s0].vx; b.v[1] = h[s0].vy; b.v[2] = h[s0].omega;
        b.step = step0 + s0;
        derive_pose(b, c->has_body, c->has_body ? c->body_desc.radius : 0.0, c->nx, c->ny);
        ATRY(cudaMemcpyAsync(c->bs + (c->nstep & 1), &b, sizeof b, cudaMemcpyHostToDevice, st));
        ATRY(cudaMemcpyAsync(store, ckpt + pop * s, pop, cudaMemcpyDeviceToDevice, st));
        for (long long k = 0; k + 1 < len; ++k) {
            // S_{s0+k} -> S_{s0+k+1} straight from one slot of the store to
            // the next (the context's scalar kernel and block shape)
            StepParams q = ctx_params(c, step0 + s0 + k);
            q.fin = store + pop * k;
            q.fout = store + pop * (k + 1);
            set_planes(q, (int)es);
            ATRY(launch_step(c->precision, q, rbx, rby, st, rminb));
        }
        for (long long n = s0 + len - 1; n >= s0; --n) {
            StepParams p = ctx_params(c, step0 + n);
            p.fin = store + pop * (n - s0);
            set_planes(p, (int)es);
            AdjStep a;
            a.xg = h[n].x; a.yg = h[n].y;
            a.vx = h[n].vx; a.vy = h[n].vy; a.om = h[n].omega;
            a.wx = 0; a.wy = 0;
            if (n >= d->window_start && qref > 0) {
                a.wx = d->w_cd / (qref * nh);
                a.wy = J2 > 0 ? d->w_cl * (h[n].fy / qref) / (J2 * qref * nh) : 0.0;
            }
            {   // the pose-derived values, as the forward step derived them
                BodyState bsn{};
                bsn.q[0] = a.xg; bsn.q[1] = a.yg;
                bsn.v[0] = a.vx; bsn.v[1] = a.vy; bsn.v[2] = a.om;
                derive_pose(bsn, c->has_body, c->has_body ? c->body_desc.radius : 0.0, c->nx, c->ny);
                a.ilo = bsn.ilo; a.ihi = bsn.ihi; a.jlo = bsn.jlo; a.jhi = bsn.jhi;
                a.xi = bsn.xi; a.yi = bsn.yi; a.xf = bsn.xf; a.yf = bsn.yf;
                a.vxf = bsn.vxf; a.vyf = bsn.vyf; a.omf = bsn.omf;
                a.wxf = (float)a.wx; a.wyf = (float)a.wy;
            }
            void *lam_next = work + lam_bytes * cur, *lam_new = work + lam_bytes * (cur ^ 1), *mu = work + 2 * lam_bytes;
            cudaError_t e = c->precision == VPLBM_F64
                                ? launch_adjoint_step<VPLBM_F64>(p, a, lam_next, mu, lam_new, dacc, grad_uin, st)
                                : launch_adjoint_step<VPLBM_F32_DEV>(p, a, lam_next, mu, lam_new, dacc, grad_uin, st);
            ATRY(e);
            cur ^= 1;
        }
    }
    // gradients
    std::vector<double> acc(nacc + c->ny);
    ATRY(cudaMemcpyAsync(acc.data(), dacc, acc.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    // restore the state after the forward run
    ATRY(cudaMemcpyAsync(c->f[nfinal & 1], final_f, pop, cudaMemcpyDeviceToDevice, st));
    ATRY(cudaMemcpyAsync(c->bs, final_bs, sizeof final_bs, cudaMemcpyHostToDevice, st));
    ATRY(cudaStreamSynchronize(st));
    c->nstep = nfinal;
    double g4[4] = {0, 0, 0, 0};
    for (size_t blk = 0; blk < nacc / 4; ++blk)
        for (int q = 0; q < 4; ++q) g4[q] += acc[blk * 4 + q];
    for (int jj = 0; jj < c->ny; ++jj) grad[jj] = acc[nacc + jj];
    grad[c->ny] = g4[0];
    grad[c->ny + 1] = g4[2] + g4[3];
    grad[c->ny + 2] = g4[1];
    cleanup();
#undef ATRY
    return VPLBM_OK;
}
