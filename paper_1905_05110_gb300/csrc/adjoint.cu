// Reverse-time discrete adjoint of the fused step for a body on a prescribed
// path (fixed or imposed motion), with sqrt(N) checkpointing.
//
// State S_n = post-collision populations entering step n; one step is
// S_{n+1}(x) = C(Pull(S_n)(x)); the force of step n is
// F_h(n) = sum_{x in R(n)} [j(Pull(S_n))(x) - j(S_n)(x)] (Eqs. 25-27 as a
// node sum).  With J = w_cd mean C_D + w_cl RMS C_L over [w0, N), the
// reverse sweep carries L_n = dJ/dS_n:
//   (a) mu(x) = (dC/df)^T L_{n+1}(x) + [x in R(n)] dJ/dF_h(n) . c   (node local)
//   (b) L_n(y) = (Pull^T mu)(y) - [y in R(n)] dJ/dF_h(n) . c
// and the parameter gradients: dJ/ds_e, dJ/ds_nu (= s7 = s8), dJ/deta from
// (a), dJ/du_in(j) of the west wall's u_x profile from (b).
// One kernel per reverse step does both: a node computes mu(x) and pushes
// each mu_q(x) to the one population its pull read (Pull^T as a scatter:
// every population but those of a zero-gradient outlet column has exactly
// one reader), so mu never reaches memory.  A zero-gradient column's
// populations have a second reader, the outlet's own copy rule; those
// contributions go to a per-row buffer that the next reverse step adds in
// as it loads L there.
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

constexpr int ADJ_BX = 32, ADJ_BY = 4;   // block of the reverse kernel (a tile of nodes)
// an interior thread takes ADJ_ROWS nodes of its column, ADJ_BY rows apart
// (at 1024 x 512 the interior then fits in one wave of resident blocks)
constexpr int ADJ_ROWS = 4;
constexpr int ADJ_BLOCK = ADJ_BX * ADJ_BY;
// blocks of 128 threads per SM the reverse kernel's register budget is
// sized for: 64 registers in FP32, 128 in FP64 (no spills)
template <int P> constexpr int adj_minb() { return P == VPLBM_F64 ? 4 : 8; }
inline int cx_host(int q) { static const int c[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1}; return c[q]; }
inline int cy_host(int q) { static const int c[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1}; return c[q]; }

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

// Slot of a population crossing the west (c_ax = +1) or east (c_ax = -1)
// edge in a zero-gradient buffer [side][3][ny]: side 0 west, 1 east.
__device__ __forceinline__ int zg_slot(int q)
{
    const int side = cx_of(q) == 1 ? 0 : 1;
    const int k = cy_of(q) == 0 ? 0 : (cy_of(q) == 1 ? 1 : 2);
    return side * 3 + k;
}

// Per-plane pointers of the adjoint fields: src[q] = &lam_next[q][0][0],
// dst[q] = &lam[q][-c_qy][-c_qx], so that the push of mu_q from interior
// node b writes dst[q][b].
template <typename T> struct LamPlanes {
    const T *src[NQ];
    T *dst[NQ];
};

// The reverse step at node (i, j) with its pulled populations f: (a) mu =
// (dC/df)^T L_{n+1} + objective term, (b) mu pushed into L_n, the
// parameter partials into g.
template <int P, bool EDGE>
__device__ __forceinline__ void adj_one_node(const StepParams &p, const AdjStep &a,
                                             const LamPlanes<typename Prec<P>::T> &lp,
                                             const typename Prec<P>::T *zg_in, typename Prec<P>::T *lam,
                                             typename Prec<P>::T *zg_out, double *grad_uin, int i, int j,
                                             const typename Prec<P>::T f[NQ], typename Prec<P>::T g[4])
{
    using T = typename Prec<P>::T;
    constexpr bool DEV = Prec<P>::DEV;
    const long long b = (long long)j * p.nx + i;
    T xi[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) xi[q] = lp.src[q][b];
    if (EDGE && (i == 0 || i == p.nx - 1)) {   // pending zero-gradient contributions of a column
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if ((cx_of(q) == 1 && i == 0) || (cx_of(q) == -1 && i == p.nx - 1)) xi[q] += zg_in[zg_slot(q) * p.ny + j];
    }

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
    g[1] = L[1] * (-(m[1] - e_eq) - (T)3 * uG);
    g[2] = L[7] * (-(m[7] - W1) - W2);
    g[3] = L[8] * (-(m[8] - W3) - (T)0.5 * W4);

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
        g[0] = k * k * ((vx - usx) * l_ax + (vy - usy) * l_ay);
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
    const T wx = par<T>(a.wx, a.wxf), wy = par<T>(a.wy, a.wyf);
    if (chi) {   // the objective's momentum-exchange term at a solid node
#pragma unroll
        for (int q = 0; q < NQ; ++q) out[q] += (T)cx_of(q) * wx + (T)cy_of(q) * wy;
    }
    // (b): mu_q(x) goes to the population its pull read, less the
    // momentum-exchange own term [y in R(n)] dJ/dF_h . c of that node; a
    // target can be solid only if the node's 3 x 3 neighbourhood meets the
    // body's node range
    const bool near = p.body.present && i + 1 >= a.ilo && i - 1 <= a.ihi && j + 1 >= a.jlo && j - 1 <= a.jhi;
    auto own = [&](int q, int ti, int tj) -> T {
        T ddx, ddy;
        return near && chi_adj<T>(p, a, ti, tj, ddx, ddy) ? (T)cx_of(q) * wx + (T)cy_of(q) * wy : (T)0;
    };
    const long long ps = p.ps;
    if (!EDGE || (i > 0 && i < p.nx - 1 && j > 0 && j < p.ny - 1)) {
        if (near) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) lp.dst[q][b] = out[q] - own(q, i - cx_of(q), j - cy_of(q));
        } else {
#pragma unroll
            for (int q = 0; q < NQ; ++q) lp.dst[q][b] = out[q];
        }
        return;
    }
    if constexpr (!EDGE) return;
    double gu = 0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        int sd = -1;
        const int kind = pull_kind(p, q, i, j, &sd);
        if (kind == PULL_PLAIN) {
            int ti = i - cx_of(q), tj = j - cy_of(q);
            ti = ti < 0 ? ti + p.nx : (ti >= p.nx ? ti - p.nx : ti);
            tj = tj < 0 ? tj + p.ny : (tj >= p.ny ? tj - p.ny : tj);
            lam[q * ps + (long long)tj * p.nx + ti] = out[q] - own(q, ti, tj);
        } else if (kind == PULL_WALL) {
            const int o = opp_of(q);
            lam[o * ps + b] = out[q] - own(o, i, j);
            if (sd == VPLBM_WEST && cx_of(q) == 1 && grad_uin && p.bc[VPLBM_WEST] == VPLBM_BC_VELOCITY &&
                p.wall_prof[VPLBM_WEST][0])
                gu += (double)out[q] * 6.0 * w_of(q) * p.rho0;
        } else {   // zero-gradient copy from (i, j - c_qy), picked up by the next reverse step
            int tj = j - cy_of(q);
            tj = tj < 0 ? tj + p.ny : (tj >= p.ny ? tj - p.ny : tj);
            zg_out[zg_slot(q) * p.ny + tj] = out[q];
        }
        // a population that no pull reads (its opposite's pull here is a
        // zero-gradient copy): only the own term
        int sd2 = -1;
        if (pull_kind(p, opp_of(q), i, j, &sd2) == PULL_ZEROGRAD) lam[q * ps + b] = -own(q, i, j);
    }
    if (i == 0 && grad_uin && p.bc[VPLBM_WEST] == VPLBM_BC_VELOCITY && p.wall_prof[VPLBM_WEST][0]) grad_uin[j] += gu;
}

// Layout of the reverse kernel's grid (1-D): the interior nodes
// [1, nx - 2] x [1, ny - 2] in tiles of ADJ_BX x (ADJ_BY * ADJ_ROWS) aligned on x = 0
// (rows of a warp stay on 128-byte boundaries; the lanes on columns 0 and
// nx - 1 idle), which take no boundary rule, so their warps never diverge
// into one; the perimeter nodes, ADJ_BLOCK per block, come first (their
// blocks take the boundary rules and run longest, and the last blocks of a
// launch set its end; a lattice less than 3 nodes wide or high is all
// perimeter, taken row by row).
struct AdjLayout {
    int itx, ity;    // interior tiles in x and y (0 when there is no interior)
    int nper;        // perimeter nodes
    int blocks;      // interior tiles + perimeter blocks
};

inline AdjLayout adj_layout(int nx, int ny)
{
    AdjLayout l;
    if (nx >= 3 && ny >= 3) {
        l.itx = (nx + ADJ_BX - 1) / ADJ_BX;
        l.ity = (ny - 2 + ADJ_BY * ADJ_ROWS - 1) / (ADJ_BY * ADJ_ROWS);
        l.nper = 2 * nx + 2 * (ny - 2);
    } else {
        l.itx = l.ity = 0;
        l.nper = nx * ny;
    }
    l.blocks = l.itx * l.ity + (l.nper + ADJ_BLOCK - 1) / ADJ_BLOCK;
    return l;
}

// Perimeter node k of an nx x ny lattice (the layout above).
__device__ __forceinline__ void perimeter_node(int nx, int ny, int k, int &i, int &j)
{
    if (nx < 3 || ny < 3) {
        i = k % nx;
        j = k / nx;
    } else if (k < nx) {
        i = k;
        j = 0;
    } else if (k < 2 * nx) {
        i = k - nx;
        j = ny - 1;
    } else {
        const int r = k - 2 * nx;
        j = 1 + (r >> 1);
        i = (r & 1) ? nx - 1 : 0;
    }
}

// The reverse step of one lattice step n (ADJ_ROWS interior nodes or one
// perimeter node per thread): (a) mu =
// (dC/df)^T L_{n+1} + objective term at every node, pushed (b) into L_n;
// parameter partials into the warps' accumulators acc[warp][4]
// (float-float in FP32, so no FP64 work and no block barrier; one writer
// per slot and launch, hence deterministic sums); dJ/du_in at the west
// inlet.  zg_in: the zero-gradient contributions to L_{n+1} left by the
// previous reverse step (added as L_{n+1} is loaded); zg_out: this
// step's, [6][ny].  Launched with programmatic dependent launch: a block
// reads its first pulled state before it waits for the previous reverse
// step to complete, so those loads overlap that step's last blocks.
template <int P>
__global__ void __launch_bounds__(ADJ_BLOCK, adj_minb<P>()) adj_fused(const StepParams p, const AdjStep a,
                                                                 const LamPlanes<typename Prec<P>::T> lp,
                                                                 const typename Prec<P>::T *zg_in,
                                                                 typename Prec<P>::T *lam, typename Prec<P>::T *zg_out,
                                                                 typename SumT<P>::A *acc, double *grad_uin,
                                                                 const AdjLayout lay)
{
    using T = typename Prec<P>::T;
    using S = typename Prec<P>::S;
    const int tid = threadIdx.y * ADJ_BX + threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int nperb = (lay.nper + ADJ_BLOCK - 1) / ADJ_BLOCK;
    T g[4] = {0, 0, 0, 0};
    const S *fin = static_cast<const S *>(p.fin);
    if ((int)blockIdx.x >= nperb) {
        const int bi = (int)blockIdx.x - nperb;
        const int i = (bi % lay.itx) * ADJ_BX + threadIdx.x;
        const int j0 = 1 + (bi / lay.itx) * ADJ_BY * ADJ_ROWS + threadIdx.y;
        const bool col = i >= 1 && i < p.nx - 1;
#pragma unroll 1
        for (int r = 0; r < ADJ_ROWS; ++r) {
            const int j = j0 + r * ADJ_BY;
            const bool in = col && j < p.ny - 1;
            T f[NQ];
            if (in) pull_all<P, true>(p, fin, i, j, f);
            if (r == 0) {   // the first row's pulled state S_n is read before waiting on the
                            // previous reverse step: no reverse step writes the segment store
                asm volatile("griddepcontrol.wait;" ::: "memory");
                asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
            }
            if (in) {
                T gn[4] = {0, 0, 0, 0};   // the node's partials (adj_one_node assigns them)
                adj_one_node<P, false>(p, a, lp, zg_in, lam, zg_out, grad_uin, i, j, f, gn);
#pragma unroll
                for (int q = 0; q < 4; ++q) g[q] += gn[q];
            }
        }
    } else {
        asm volatile("griddepcontrol.wait;" ::: "memory");
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        const int k = (int)blockIdx.x * ADJ_BLOCK + tid;
        if (k < lay.nper) {
            int i, j;
            perimeter_node(p.nx, p.ny, k, i, j);
            T f[NQ];
            pull_all<P>(p, fin, i, j, f);
            adj_one_node<P, true>(p, a, lp, zg_in, lam, zg_out, grad_uin, i, j, f, g);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) g[q] += __shfl_down_sync(0xffffffffu, g[q], off);
    }
    if (lane == 0) {
        using A = typename SumT<P>::A;
        A *dst = acc + ((size_t)blockIdx.x * (ADJ_BLOCK / 32) + warp) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            A t = dst[q];
            acc_add(t, g[q]);
            dst[q] = t;
        }
    }
}

template <int P>
cudaError_t launch_adjoint_step(const StepParams &p, const AdjStep &a, const void *lam_next, const void *zg_in, void *lam,
                                void *zg_out, void *acc, double *grad_uin, cudaStream_t stream, bool pdl)
{
    using T = typename Prec<P>::T;
    LamPlanes<T> lp;
    for (int q = 0; q < NQ; ++q) {
        lp.src[q] = static_cast<const T *>(lam_next) + q * p.ps;
        lp.dst[q] = static_cast<T *>(lam) + q * p.ps - cx_host(q) - (long long)cy_host(q) * p.nx;
    }
    const AdjLayout lay = adj_layout(p.nx, p.ny);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(lay.blocks);
    cfg.blockDim = dim3(ADJ_BX, ADJ_BY);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, adj_fused<P>, p, a, lp, static_cast<const T *>(zg_in), static_cast<T *>(lam),
                              static_cast<T *>(zg_out), static_cast<typename SumT<P>::A *>(acc), grad_uin, lay);
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

    char *ckpt = nullptr, *store = nullptr, *work = nullptr;   // work: lam[0], lam[1], zero-gradient rows [2][6][ny]
    double *dacc = nullptr;   // the warps' parameter accumulators, then dJ/du_in [ny]
    void *final_f = nullptr;
    BodyState final_bs[2];
    // parameter partials: 4 accumulators per warp of the reverse kernel
    // (FP32: float-float pairs, FP64: doubles), then the inlet gradient
    const size_t nwarps = (size_t)adj_layout(c->nx, c->ny).blocks * (ADJ_BLOCK / 32);
    const size_t acc_bytes = nwarps * 4 * (c->precision == VPLBM_F64 ? sizeof(double) : sizeof(float2));
    // the reverse sweep recomputes segment s - 1 on a second stream while
    // segment s runs its reverse steps: two segment stores, and events
    // that order the two streams
    cudaStream_t sr = nullptr;
    BodyState *seg_bs = nullptr;   // [nck] body state at each segment's start
    cudaEvent_t ev_rec[2] = {nullptr, nullptr}, ev_rev[2] = {nullptr, nullptr};
    auto cleanup = [&]() {
        if (sr) cudaStreamSynchronize(sr);
        cudaStreamSynchronize(st);
        for (int q = 0; q < 2; ++q) {
            if (ev_rec[q]) cudaEventDestroy(ev_rec[q]);
            if (ev_rev[q]) cudaEventDestroy(ev_rev[q]);
        }
        if (sr) cudaStreamDestroy(sr);
    };
#define ATRY(expr)                                                                     \
    do {                                                                               \
        cudaError_t e_ = (expr);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            cleanup();                                                                 \
            return aerr(VPLBM_ECUDA, "%s failed: %s", #expr, cudaGetErrorString(e_));  \
        }                                                                              \
    } while (0)
    // the device workspace, kept in the context between calls: checkpoints
    // [nck], two segment stores [2][K], segment-start body states [nck],
    // work, accumulators and inlet gradient, the final state
    const size_t zg_bytes = (size_t)6 * c->ny * es;
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t o_store = al(pop * nck), o_segbs = o_store + al(pop * K * 2);
    const size_t o_work = o_segbs + al((size_t)nck * sizeof(BodyState));
    const size_t o_dacc = o_work + al(lam_bytes * 2 + 2 * zg_bytes);
    const size_t o_final = o_dacc + al(acc_bytes + (size_t)c->ny * sizeof(double));
    const size_t ws_bytes = o_final + al(pop);
    if (c->adj_ws_bytes < ws_bytes) {
        if (c->adj_ws) {
            cudaStreamSynchronize(st);
            cudaFree(c->adj_ws);
            c->adj_ws = nullptr;
            c->adj_ws_bytes = 0;
        }
        ATRY(cudaMalloc(&c->adj_ws, ws_bytes));
        c->adj_ws_bytes = ws_bytes;
    }
    {
        char *ws = static_cast<char *>(c->adj_ws);
        ckpt = ws;
        store = ws + o_store;
        seg_bs = reinterpret_cast<BodyState *>(ws + o_segbs);
        work = ws + o_work;
        dacc = reinterpret_cast<double *>(ws + o_dacc);
        final_f = ws + o_final;
    }
    ATRY(cudaStreamCreateWithFlags(&sr, cudaStreamNonBlocking));
    for (int q = 0; q < 2; ++q) {
        ATRY(cudaEventCreateWithFlags(&ev_rec[q], cudaEventDisableTiming));
        ATRY(cudaEventCreateWithFlags(&ev_rev[q], cudaEventDisableTiming));
    }
    double *grad_uin = reinterpret_cast<double *>(reinterpret_cast<char *>(dacc) + acc_bytes);
    ATRY(cudaMemsetAsync(work, 0, lam_bytes * 2 + 2 * zg_bytes, st));
    ATRY(cudaMemsetAsync(dacc, 0, acc_bytes + (size_t)c->ny * sizeof(double), st));

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
    int cur = 0;   // lam[cur] holds L_{n+1}, zero-gradient rows [cur] its pending column contributions
    // recompute the states S_{s0} .. S_{s0+len-1} of segment s into store
    // slot set s & 1, on stream sr, straight from one slot to the next (the
    // context's scalar kernel and block shape)
    auto recompute = [&](long long s) -> cudaError_t {
        const long long s0 = s * K, len = std::min(K, N - s0);
        char *seg = store + pop * K * (s & 1);
        c->nstep = step0 + s0;
        cudaError_t e = cudaMemcpyAsync(c->bs + (c->nstep & 1), seg_bs + s, sizeof(BodyState), cudaMemcpyDeviceToDevice, sr);
        if (e == cudaSuccess) e = cudaMemcpyAsync(seg, ckpt + pop * s, pop, cudaMemcpyDeviceToDevice, sr);
        for (long long k = 0; k + 1 < len && e == cudaSuccess; ++k) {
            StepParams q = ctx_params(c, step0 + s0 + k);
            q.fin = seg + pop * k;
            q.fout = seg + pop * (k + 1);
            set_planes(q, (int)es);
            e = launch_step(c->precision, q, rbx, rby, sr, rminb);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev_rec[s & 1], sr);
        return e;
    };
    // the body state at each segment's start, from the records (uploaded
    // once: a copy from host memory per segment could stall the host)
    {
        std::vector<BodyState> bsv((size_t)nck);
        for (long long q = 0; q < nck; ++q) {
            const long long s0 = q * K;
            BodyState &b = bsv[(size_t)q];
            b = BodyState{};
            b.q[0] = h[s0].x; b.q[1] = h[s0].y; b.q[2] = h[s0].theta;
            b.v[0] = h[s0].vx; b.v[1] = h[s0].vy; b.v[2] = h[s0].omega;
            b.step = step0 + s0;
            derive_pose(b, c->has_body, c->has_body ? c->body_desc.radius : 0.0, c->nx, c->ny);
        }
        ATRY(cudaMemcpyAsync(seg_bs, bsv.data(), bsv.size() * sizeof(BodyState), cudaMemcpyHostToDevice, st));
        ATRY(cudaStreamSynchronize(st));
    }
    // the first segments' slot sets are free
    ATRY(cudaEventRecord(ev_rev[0], st));
    ATRY(cudaEventRecord(ev_rev[1], st));
    ATRY(cudaStreamWaitEvent(sr, ev_rev[0], 0));   // after the forward run
    ATRY(recompute(nck - 1));
    for (long long s = nck - 1; s >= 0; --s) {
        const long long s0 = s * K, len = std::min(K, N - s0);
        if (s > 0) {   // segment s - 1 reuses the slots of segment s + 1, once its reverse steps are done
            ATRY(cudaStreamWaitEvent(sr, ev_rev[(s - 1) & 1], 0));
            ATRY(recompute(s - 1));
        }
        ATRY(cudaStreamWaitEvent(st, ev_rec[s & 1], 0));
        const char *seg = store + pop * K * (s & 1);
        for (long long n = s0 + len - 1; n >= s0; --n) {
            StepParams p = ctx_params(c, step0 + n);
            p.fin = seg + pop * (n - s0);
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
            // programmatic dependent launch between the reverse steps of a
            // segment; the first one follows the wait on the recomputation
            // (a full dependency)
            const bool pdl = n < s0 + len - 1;
            void *lam_next = work + lam_bytes * cur, *lam_new = work + lam_bytes * (cur ^ 1);
            void *zg_in = work + 2 * lam_bytes + zg_bytes * cur, *zg_out = work + 2 * lam_bytes + zg_bytes * (cur ^ 1);
            cudaError_t e =
                c->precision == VPLBM_F64
                    ? launch_adjoint_step<VPLBM_F64>(p, a, lam_next, zg_in, lam_new, zg_out, dacc, grad_uin, st, pdl)
                    : launch_adjoint_step<VPLBM_F32_DEV>(p, a, lam_next, zg_in, lam_new, zg_out, dacc, grad_uin, st, pdl);
            ATRY(e);
            cur ^= 1;
        }
        ATRY(cudaEventRecord(ev_rev[s & 1], st));
    }
    // gradients
    std::vector<char> accb(acc_bytes);
    std::vector<double> guin(c->ny);
    ATRY(cudaMemcpyAsync(accb.data(), dacc, acc_bytes, cudaMemcpyDeviceToHost, st));
    ATRY(cudaMemcpyAsync(guin.data(), grad_uin, guin.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    // restore the state after the forward run
    ATRY(cudaMemcpyAsync(c->f[nfinal & 1], final_f, pop, cudaMemcpyDeviceToDevice, st));
    ATRY(cudaMemcpyAsync(c->bs, final_bs, sizeof final_bs, cudaMemcpyHostToDevice, st));
    ATRY(cudaStreamSynchronize(st));
    c->nstep = nfinal;
    double g4[4] = {0, 0, 0, 0};   // fixed-order sum over the warps' accumulators
    for (size_t w = 0; w < nwarps; ++w)
        for (int q = 0; q < 4; ++q) {
            if (c->precision == VPLBM_F64) {
                g4[q] += reinterpret_cast<const double *>(accb.data())[w * 4 + q];
            } else {
                const float2 v = reinterpret_cast<const float2 *>(accb.data())[w * 4 + q];
                g4[q] += (double)v.x + (double)v.y;
            }
        }
    for (int jj = 0; jj < c->ny; ++jj) grad[jj] = guin[jj];
    grad[c->ny] = g4[0];
    grad[c->ny + 1] = g4[2] + g4[3];
    grad[c->ny + 2] = g4[1];
    cleanup();
#undef ATRY
    return VPLBM_OK;
}
