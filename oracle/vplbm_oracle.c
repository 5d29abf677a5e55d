/*
 * Plain FP64 CPU oracle of the volume-penalization lattice Boltzmann method
 * (VP-LBM, D2Q9, multiple relaxation time) with a rigid disk.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  It is used by the test-suite,
 * by the package's smoke check and by the CPU-baseline leg of the benchmark;
 * no product code path may call it.  It shares no code, header, table or
 * constant with the CUDA implementation.
 *
 * Every step follows the paper in its own order (Algorithm 1, Sec. 2.3):
 *   1. streaming of the post-collision populations (Eq. 18) with the
 *      boundary rules of Sec. 3.1 / 3.2;
 *   2. macroscopic moments (Eq. 19) with the penalized velocity of
 *      Eqs. (20)-(22);
 *   3. MRT collision with a source term (Eqs. 8, 17), moments by the
 *      matrix M of Eq. (15), equilibria of Eq. (14), forcing of Eq. (12);
 *      or, when the lattice asks for it, the single-relaxation-time (BGK)
 *      operator of Sec. 2.1 in velocity space with the Eq. (12) forcing;
 *   4. force and torque on the body, then the rigid-body update of
 *      Eqs. (23)-(24) by fourth-order Runge-Kutta (Algorithm 1, step 3).
 * Matrix-vector products are written as plain loops over the 9x9 matrices;
 * M^-1 is obtained by Gauss-Jordan elimination, not from a closed form.
 *
 * Readings taken where the paper is silent or ambiguous (all restated in
 * the design notes of the repository):
 *   - Eq. (22) is evaluated in the algebraically identical form
 *     a = -chi (j/rho + g/2 - u_s) / (eta + chi/2), u = j/rho + g/2 + a/2,
 *     which stays finite for eta -> 0.
 *   - The forcing term of Eq. (12) is used without its (1 - 1/(2 tau))
 *     prefactor, because Eqs. (8)/(17) already apply (I - S/2) in moment
 *     space; it is added with a plus sign as the body acceleration
 *     a = -chi/eta (u - u_s) (the minus of Eq. 1 folded into a).
 *   - chi(x) = 1 iff (i - x_G)^2 + (j - y_G)^2 <= R^2, evaluated in FP64
 *     exactly as written (the file is compiled with -ffp-contract=off).
 *   - The force that drives the body is the momentum exchanged through the
 *     links between the solid region R(n) = {chi = 1 at step n} and the
 *     rest of the lattice during the streaming into step n, i.e. Eqs.
 *     (25)-(27) with u_Gamma = 0, summed here node by node over R(n):
 *       F_h(n) = sum_{x in R(n)} [ j(x, n) - j~(x, n-1) ],
 *       T_h(n) = sum_{x in R(n)} (x - x_G) x [ j(x, n) - j~(x, n-1) ],
 *     j = sum_a c_a f_a after streaming, j~ = sum_a c_a f~_a of the node's
 *     own post-collision populations.  The reaction of the penalization
 *     force, sum_solid rho chi (u - u_s)/eta, and its torque are reduced
 *     as well and recorded beside it.
 *   - Walls are half-way bounce-back; a velocity wall adds
 *     6 w_a rho0 (c_a . u_w); a zero-gradient edge copies the population of
 *     the edge column itself.  When the source node of a pull lies outside
 *     in y, the south/north rule wins over the west/east rule.
 *
 * Storage: f[(a*ny + j)*nx + i], node (i, j) at x = i, y = j.
 * The state after n steps is the post-collision population field of step
 * n - 1 (for n = 0: the equilibrium given at initialisation).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define Q 9

/* Planted mistakes, for the test that checks that the pins catch them
 * (tests/test_oracle_plants.py builds this file with -DORACLE_PLANT=k into
 * a library of its own); the oracle itself is built with ORACLE_PLANT = 0,
 * where every PLANT(k) is a constant false and plants nothing. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif
#define PLANT(k) (ORACLE_PLANT == (k))

/* ---- lattice constants, restated from Sec. 2.2 ---------------------- */

static int C[Q][2];      /* Eq. (10) */
static double W[Q];      /* Eq. (13) */
static int OPP[Q];       /* index of -c_a */
static int MIRY[Q];      /* index of (c_ax, -c_ay): mirror image about a wall of constant y */
/* Eq. (15): rows rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy */
static const double M[Q][Q] = {
    { 1,  1,  1,  1,  1,  1,  1,  1,  1},
    {-4, -1, -1, -1, -1,  2,  2,  2,  2},
    { 4, -2, -2, -2, -2,  1,  1,  1,  1},
    { 0,  1,  0, -1,  0,  1, -1, -1,  1},
    { 0, -2,  0,  2,  0,  1, -1, -1,  1},
    { 0,  0,  1,  0, -1,  1,  1, -1, -1},
    { 0,  0, -2,  0,  2,  1,  1, -1, -1},
    { 0,  1, -1,  1, -1,  0,  0,  0,  0},
    { 0,  0,  0,  0,  0,  1, -1,  1, -1}};
static double MINV[Q][Q];
static int constants_ready = 0;

static void setup_constants(void)
{
    if (constants_ready) return;
    const double pi = 3.14159265358979323846;
    /* Eq. (10): c_0 = 0; c_1..4 at angles (a-1) pi/2; c_5..8 at (2a-9) pi/4,
     * length sqrt(2); rounded to the integer lattice vectors. */
    C[0][0] = 0; C[0][1] = 0;
    for (int a = 1; a <= 4; ++a) {
        double ang = (a - 1) * pi / 2.0;
        C[a][0] = (int)lround(cos(ang));
        C[a][1] = (int)lround(sin(ang));
    }
    for (int a = 5; a <= 8; ++a) {
        double ang = (2 * a - 9) * pi / 4.0;
        C[a][0] = (int)lround(sqrt(2.0) * cos(ang));
        C[a][1] = (int)lround(sqrt(2.0) * sin(ang));
    }
    /* Eq. (13) */
    W[0] = 4.0 / 9.0;
    for (int a = 1; a <= 4; ++a) W[a] = 1.0 / 9.0;
    for (int a = 5; a <= 8; ++a) W[a] = PLANT(3) ? 1.0 / 18.0 : 1.0 / 36.0;
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b)
            if (C[b][0] == -C[a][0] && C[b][1] == -C[a][1]) OPP[a] = b;
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b)
            if (C[b][0] == C[a][0] && C[b][1] == -C[a][1]) MIRY[a] = b;
    /* M^-1 by Gauss-Jordan elimination with partial pivoting. */
    double A[Q][2 * Q];
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < 2 * Q; ++c)
            A[r][c] = (c < Q) ? M[r][c] : (c - Q == r ? 1.0 : 0.0);
    for (int col = 0; col < Q; ++col) {
        int piv = col;
        for (int r = col + 1; r < Q; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (piv != col)
            for (int c = 0; c < 2 * Q; ++c) {
                double t = A[col][c]; A[col][c] = A[piv][c]; A[piv][c] = t;
            }
        double p = A[col][col];
        for (int c = 0; c < 2 * Q; ++c) A[col][c] /= p;
        for (int r = 0; r < Q; ++r) {
            if (r == col) continue;
            double fct = A[r][col];
            if (fct == 0.0) continue;
            for (int c = 0; c < 2 * Q; ++c) A[r][c] -= fct * A[col][c];
        }
    }
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) MINV[r][c] = A[r][Q + c];
    constants_ready = 1;
}

/* ---- public descriptors (ctypes mirrors them) ------------------------ */

enum { ORC_PERIODIC = 0, ORC_NOSLIP = 1, ORC_VELOCITY = 2, ORC_ZEROGRAD = 3, ORC_SYMMETRY = 4,
       ORC_CONVECTIVE = 5 };
enum { ORC_WEST = 0, ORC_EAST = 1, ORC_SOUTH = 2, ORC_NORTH = 3 };
enum { ORC_FIXED = 0, ORC_IMPOSED = 1, ORC_FREE = 2 };
enum { ORC_MRT = 0, ORC_BGK = 1 };
enum { ORC_DISK = 0, ORC_ELLIPSE = 1, ORC_RECT = 2 };

typedef struct {
    int nx, ny;
    double s[Q];          /* diagonal of S, Eq. (16) */
    double eta;           /* penalization factor, Eq. (2) */
    double rho0;          /* reference density of the walls */
    double gx, gy;        /* uniform body acceleration of the fluid */
    int bc_kind[4];       /* west, east, south, north */
    double bc_u[4][2];    /* uniform wall velocity per edge */
    const double *bc_ux[4]; /* optional per-node wall velocity, edge length */
    const double *bc_uy[4];
    int collision;        /* ORC_MRT (Eq. 17) or ORC_BGK (Sec. 2.1, rate s[7]) */
} orc_lattice;

typedef struct {
    int present;
    double radius;
    double x, y, theta, vx, vy, omega;   /* initial pose and velocity */
    int motion;                          /* ORC_FIXED / ORC_IMPOSED / ORC_FREE */
    int axis;                            /* imposed coordinate: 0 x, 1 y, 2 theta */
    double amp, freq, phase;             /* q(t) = q_c + amp sin(2 pi freq t + phase) */
    double mass, inertia;
    double damp[3], stiff[3], q0[3], f_ext[3];  /* Eqs. (23)-(24), per x, y, theta */
    unsigned dof_mask;                   /* bit0 x, bit1 y, bit2 theta */
    double u_ref, d_ref;                 /* C_D, C_L normalisation (Sec. 3.1) */
    int shape;                           /* ORC_DISK or ORC_ELLIPSE */
    double radius_b;                     /* ellipse: semi-axis along the body's y axis (radius: along its x axis) */
} orc_body;

/* One record per step n: force and torque of that step, pose used by it. */
typedef struct {
    double t, fx, fy, torque, cd, cl, x, y, theta, vx, vy, omega;
    double fpen_x, fpen_y, tpen, n_solid;
} orc_record;

#define ORC_MAXB 4   /* bodies per lattice */

typedef struct {
    orc_lattice lat;
    int nb;                        /* number of bodies, 0 .. ORC_MAXB */
    orc_body body[ORC_MAXB];
    double *prof_ux[4], *prof_uy[4];
    double *ft;            /* post-collision populations (the state) */
    double *fn;            /* scratch for the next state */
    long long step;
    double q[ORC_MAXB][3], v[ORC_MAXB][3];   /* pose (x, y, theta) and velocity of each body */
    double q_center[ORC_MAXB];               /* centre of an imposed sinusoid */
    orc_record *hist;      /* [max(nb, 1)][hist_cap] */
    long long hist_cap;
    double *conv_prev;     /* convective outlet: pulled f_a(nx-1, j) of the previous step, [a][j] */
    double *conv_next;
} orc_sim;

/* ---- small building blocks ------------------------------------------ */

static double edge_u(const orc_sim *s, int side, int comp, int k)
{
    const double *p = comp == 0 ? s->prof_ux[side] : s->prof_uy[side];
    if (p) return p[k];
    return s->lat.bc_u[side][comp];
}

/* chi of Eq. (2) for body k at its current pose (reading R1).  Disk:
 * |x - x_G| <= R.  Ellipse of semi-axes a (along the body's x axis, at the
 * angle theta of the pose) and b: with u, v the node's coordinates in the
 * body frame, b^2 u^2 + a^2 v^2 <= a^2 b^2.  Rectangle of half-sides a, b
 * along the same axes: |u| <= a and |v| <= b. */
static int chi_body(const orc_sim *s, int k, int i, int j)
{
    const orc_body *b = &s->body[k];
    if (!b->present) return 0;
    double dx = (double)i - s->q[k][0];
    double dy = (double)j - s->q[k][1];
    if (b->shape == ORC_ELLIPSE) {
        double c = cos(s->q[k][2]), sn = sin(s->q[k][2]);
        double a2 = b->radius * b->radius, b2 = b->radius_b * b->radius_b;
        double u = dx * c + dy * sn;
        double v = dy * c - dx * sn;
        return PLANT(14) ? a2 * (u * u) + b2 * (v * v) <= a2 * b2 : b2 * (u * u) + a2 * (v * v) <= a2 * b2;
    }
    if (b->shape == ORC_RECT) {
        double c = cos(s->q[k][2]), sn = sin(s->q[k][2]);
        double u = PLANT(15) ? dx * c - dy * sn : dx * c + dy * sn;
        double v = PLANT(15) ? dy * c + dx * sn : dy * c - dx * sn;
        return fabs(u) <= b->radius && fabs(v) <= b->radius_b;
    }
    double d2 = dx * dx + dy * dy;
    double r2 = b->radius * b->radius;
    return d2 <= r2;
}

/* The body a node belongs to (-1: fluid).  Bodies do not overlap (the
 * caller's responsibility); where they would, the first one listed wins. */
static int owner_at(const orc_sim *s, int i, int j)
{
    for (int k = 0; k < s->nb; ++k)
        if (chi_body(s, k, i, j)) return k;
    return -1;
}

/* 0: fluid, else 1 + the index of the body the node belongs to. */
int orc_chi(const orc_sim *s, int i, int j) { return owner_at(s, i, j) + 1; }

/* Equilibrium of Eq. (11). */
static void equilibrium(double rho, double ux, double uy, double feq[Q])
{
    const double cs2 = 1.0 / 3.0;
    for (int a = 0; a < Q; ++a) {
        double cu = C[a][0] * ux + C[a][1] * uy;
        /* uu : (cc - cs^2 I) */
        double uucc = ux * ux * (C[a][0] * C[a][0] - cs2)
                    + 2.0 * ux * uy * (C[a][0] * C[a][1])
                    + uy * uy * (C[a][1] * C[a][1] - cs2);
        feq[a] = W[a] * rho * (1.0 + cu / cs2 + uucc / (2.0 * cs2 * cs2));
    }
}

/* Moment equilibria of Eq. (14). */
static void moment_equilibrium(double rho, double ux, double uy, double meq[Q])
{
    double u2 = ux * ux + uy * uy;
    meq[0] = rho;
    meq[1] = rho * (-2.0 + 3.0 * u2);
    meq[2] = rho * (1.0 - 3.0 * u2);
    meq[3] = rho * ux;
    meq[4] = PLANT(1) ? rho * ux : -rho * ux;
    meq[5] = rho * uy;
    meq[6] = -rho * uy;
    meq[7] = rho * (ux * ux - uy * uy);
    meq[8] = rho * ux * uy;
}

/* Forcing term of Eq. (12) for the force density G = rho F, without the
 * (1 - 1/(2 tau)) prefactor (it is replaced by (I - S/2) of Eq. 17). */
static void guo_forcing(double ux, double uy, double Gx, double Gy, double F[Q])
{
    const double cs2 = 1.0 / 3.0;
    for (int a = 0; a < Q; ++a) {
        double cu = C[a][0] * ux + C[a][1] * uy;
        double vx = (C[a][0] - ux) / cs2 + (PLANT(2) ? 0.0 : cu * C[a][0] / (cs2 * cs2));
        double vy = (C[a][1] - uy) / cs2 + (PLANT(2) ? 0.0 : cu * C[a][1] / (cs2 * cs2));
        F[a] = W[a] * (vx * Gx + vy * Gy);
    }
}

/* Velocity of Eq. (22) in the eta-stable form; returns the penalization
 * acceleration a and the velocity u. */
static void penalized_velocity(double rho, double jx, double jy, int chi,
                               double usx, double usy, double eta,
                               double gx, double gy,
                               double *ux, double *uy, double *ax, double *ay)
{
    double vx = jx / rho + 0.5 * gx;
    double vy = jy / rho + 0.5 * gy;
    double c = (double)chi;
    *ax = -c * (vx - usx) / (eta + (PLANT(4) ? 1.0 : 0.5) * c);
    *ay = -c * (vy - usy) / (eta + (PLANT(4) ? 1.0 : 0.5) * c);
    *ux = vx + 0.5 * *ax;
    *uy = vy + 0.5 * *ay;
}

/* MRT collision with source, Eq. (17): m* = m - S (m - m_eq) + (I - S/2) M F. */
static void collide(const double f[Q], const double s[Q], double rho,
                    double ux, double uy, double Gx, double Gy, double ft[Q])
{
    double m[Q], meq[Q], F[Q], MF[Q], ms[Q];
    for (int r = 0; r < Q; ++r) {
        m[r] = 0.0;
        for (int a = 0; a < Q; ++a) m[r] += M[r][a] * f[a];
    }
    moment_equilibrium(rho, ux, uy, meq);
    guo_forcing(ux, uy, Gx, Gy, F);
    for (int r = 0; r < Q; ++r) {
        MF[r] = 0.0;
        for (int a = 0; a < Q; ++a) MF[r] += M[r][a] * F[a];
    }
    for (int r = 0; r < Q; ++r)
        ms[r] = m[r] - s[r] * (m[r] - meq[r]) + (1.0 - 0.5 * s[r]) * MF[r];
    for (int a = 0; a < Q; ++a) {
        ft[a] = 0.0;
        for (int r = 0; r < Q; ++r) ft[a] += MINV[a][r] * ms[r];
    }
}

/* Single-relaxation-time (BGK) collision of Sec. 2.1 with the forcing
 * term of Eq. (12) as printed there, (1 - 1/(2 tau)) prefactor included:
 *   f~ = f - (f - f_eq) / tau + (1 - 1/(2 tau)) F,   1/tau = omega.
 * Written in velocity space, independent of M. */
static void collide_bgk(const double f[Q], double omega, double rho,
                        double ux, double uy, double Gx, double Gy, double ft[Q])
{
    double feq[Q], F[Q];
    equilibrium(rho, ux, uy, feq);
    guo_forcing(ux, uy, Gx, Gy, F);
    for (int a = 0; a < Q; ++a)
        ft[a] = f[a] - omega * (f[a] - feq[a]) + (PLANT(12) ? 1.0 : 1.0 - 0.5 * omega) * F[a];
}

/* ---- streaming with boundary rules (Eq. 18) ------------------------- */

static double pulled(const orc_sim *s, int a, int i, int j)
{
    const int nx = s->lat.nx, ny = s->lat.ny;
    const double *ft = s->ft;
#define FT(b, ii, jj) ft[((size_t)(b) * ny + (jj)) * nx + (ii)]
    int si = i - C[a][0];
    int sj = j - C[a][1];
    if (sj < 0 || sj >= ny) {
        int side = sj < 0 ? ORC_SOUTH : ORC_NORTH;
        int kind = s->lat.bc_kind[side];
        if (kind == ORC_PERIODIC) {
            sj = (sj + ny) % ny;
        } else if (kind == ORC_SYMMETRY) {
            /* specular reflection at the half-way wall (u.n = 0, no shear
             * stress): the population left node (i - c_ax, j) in the
             * mirrored direction; at a corner whose x edge is not periodic
             * the node's own mirrored population is taken */
            int mi = i - C[a][0];
            if (mi < 0 || mi >= nx) mi = s->lat.bc_kind[ORC_WEST] == ORC_PERIODIC ? (mi + nx) % nx : i;
            return FT(PLANT(13) ? OPP[a] : MIRY[a], mi, j);
        } else {
            /* half-way bounce-back at y = -1/2 or y = ny - 1/2 */
            double val = FT(OPP[a], i, j);
            if (kind == ORC_VELOCITY) {
                double cu = C[a][0] * edge_u(s, side, 0, i) + C[a][1] * edge_u(s, side, 1, i);
                val += (PLANT(7) ? -6.0 : 6.0) * W[a] * s->lat.rho0 * cu;
            }
            return val;
        }
    }
    if (si < 0 || si >= nx) {
        int side = si < 0 ? ORC_WEST : ORC_EAST;
        int kind = s->lat.bc_kind[side];
        if (kind == ORC_PERIODIC) {
            si = (si + nx) % nx;
        } else if (kind == ORC_ZEROGRAD) {
            return FT(a, i, PLANT(8) ? j : sj);
        } else if (kind == ORC_CONVECTIVE) {
            /* advection of f_a out of the domain, d f/dt + U d f/dx = 0,
             * implicit in time and upwind in space between the outlet node
             * and its inner neighbour (whose pulled value is the
             * zero-gradient one): f(N, n+1) = (f(N, n) + U f(N-1, n+1)) / (1 + U) */
            const double U = s->lat.bc_u[side][0];
            if (PLANT(18)) return (U * s->conv_prev[(size_t)a * ny + j] + FT(a, i, sj)) / (1.0 + U);
            return (s->conv_prev[(size_t)a * ny + j] + U * FT(a, i, PLANT(8) ? j : sj)) / (1.0 + U);
        } else {
            double val = FT(OPP[a], i, j);
            if (kind == ORC_VELOCITY) {
                double cu = C[a][0] * edge_u(s, side, 0, j) + C[a][1] * edge_u(s, side, 1, j);
                val += (PLANT(7) ? -6.0 : 6.0) * W[a] * s->lat.rho0 * cu;
            }
            return val;
        }
    }
    return FT(a, si, sj);
#undef FT
}

/* Macroscopic state of node (i, j) at the current step: the pulled
 * populations f, rho, j, chi, u_s, velocity u and penalization a. */
typedef struct {
    double f[Q];
    double rho, jx, jy, ux, uy, ax, ay, usx, usy, dx, dy;
    int chi;
    int owner;   /* body of a solid node (-1: fluid) */
} node_state;

static void node_macro(const orc_sim *s, int i, int j, node_state *ns)
{
    ns->rho = 0.0; ns->jx = 0.0; ns->jy = 0.0;
    for (int a = 0; a < Q; ++a) {
        ns->f[a] = pulled(s, a, i, j);
        ns->rho += ns->f[a];                 /* Eq. (19) */
        ns->jx += C[a][0] * ns->f[a];
        ns->jy += C[a][1] * ns->f[a];
    }
    ns->owner = owner_at(s, i, j);
    ns->chi = ns->owner >= 0;
    const int k = ns->owner >= 0 ? ns->owner : 0;
    ns->dx = (double)i - s->q[k][0];
    ns->dy = (double)j - s->q[k][1];
    /* rigid-body velocity at the node (of the body it belongs to) */
    ns->usx = s->v[k][0] - s->v[k][2] * ns->dy;
    ns->usy = s->v[k][1] + s->v[k][2] * ns->dx;
    penalized_velocity(ns->rho, ns->jx, ns->jy, ns->chi, ns->usx, ns->usy,
                       s->lat.eta, s->lat.gx, s->lat.gy,
                       &ns->ux, &ns->uy, &ns->ax, &ns->ay);
}

/* ---- rigid body (Eqs. 23-24, Algorithm 1 step 3) -------------------- */

static void body_rhs(const orc_body *b, const double F[3], const double q[3],
                     const double v[3], double acc[3])
{
    for (int d = 0; d < 3; ++d) {
        double m = d < 2 ? b->mass : b->inertia;
        acc[d] = (F[d] + b->f_ext[d] - b->damp[d] * v[d] - b->stiff[d] * (q[d] - b->q0[d])) / m;
    }
}

/* Advance pose and velocity by one time step (h = 1) with the hydrodynamic
 * force and torque F held over the step. */
static void body_advance(const orc_body *b, long long step, double q_center,
                         const double F[3], double q[3], double v[3])
{
    const double pi = 3.14159265358979323846;
    if (b->motion == ORC_FIXED) return;
    if (b->motion == ORC_IMPOSED) {
        double t1 = (double)(step + 1);
        double ph = 2.0 * pi * b->freq * t1 + b->phase;
        q[b->axis] = q_center + b->amp * sin(ph);
        v[b->axis] = 2.0 * pi * b->freq * b->amp * (PLANT(19) ? sin(ph) : cos(ph));
        return;
    }
    /* classic fourth-order Runge-Kutta on (q, v) for the free DOFs */
    const double h = 1.0;
    double k1q[3], k1v[3], k2q[3], k2v[3], k3q[3], k3v[3], k4q[3], k4v[3];
    double qt[3], vt[3];
    for (int d = 0; d < 3; ++d) k1q[d] = v[d];
    body_rhs(b, F, q, v, k1v);
    for (int d = 0; d < 3; ++d) { qt[d] = q[d] + 0.5 * h * k1q[d]; vt[d] = v[d] + 0.5 * h * k1v[d]; }
    for (int d = 0; d < 3; ++d) k2q[d] = vt[d];
    body_rhs(b, F, qt, vt, k2v);
    for (int d = 0; d < 3; ++d) { qt[d] = q[d] + 0.5 * h * k2q[d]; vt[d] = v[d] + 0.5 * h * k2v[d]; }
    for (int d = 0; d < 3; ++d) k3q[d] = vt[d];
    body_rhs(b, F, qt, vt, k3v);
    for (int d = 0; d < 3; ++d) { qt[d] = q[d] + h * k3q[d]; vt[d] = v[d] + h * k3v[d]; }
    for (int d = 0; d < 3; ++d) k4q[d] = vt[d];
    body_rhs(b, F, qt, vt, k4v);
    for (int d = 0; d < 3; ++d) {
        if (!((b->dof_mask >> d) & 1u)) continue;
        q[d] = PLANT(5) ? q[d] + h * k1q[d] : q[d] + h / 6.0 * (k1q[d] + 2.0 * k2q[d] + 2.0 * k3q[d] + k4q[d]);
        v[d] = PLANT(5) ? v[d] + h * k1v[d] : v[d] + h / 6.0 * (k1v[d] + 2.0 * k2v[d] + 2.0 * k3v[d] + k4v[d]);
    }
}

/* ---- public API ------------------------------------------------------ */

void orc_free(orc_sim *s);

orc_sim *orc_create_bodies(const orc_lattice *lat, const orc_body *bodies, int nb, long long hist_cap)
{
    setup_constants();
    if (lat->nx < 2 || lat->ny < 2) return NULL;
    if (lat->bc_kind[ORC_WEST] == ORC_SYMMETRY || lat->bc_kind[ORC_EAST] == ORC_SYMMETRY) return NULL;   /* y walls only */
    for (int side = 0; side < 4; ++side)
        if (lat->bc_kind[side] == ORC_CONVECTIVE && (side != ORC_EAST || !(lat->bc_u[side][0] >= 0.0)))
            return NULL;   /* east outlet only, convective velocity >= 0 */
    if (nb < 0 || nb > ORC_MAXB || (nb > 0 && !bodies)) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    if (!s) return NULL;
    s->lat = *lat;
    s->nb = nb;
    for (int k = 0; k < nb; ++k) s->body[k] = bodies[k];
    for (int side = 0; side < 4; ++side) {
        int len = side < 2 ? lat->ny : lat->nx;
        s->lat.bc_ux[side] = NULL; s->lat.bc_uy[side] = NULL;
        if (lat->bc_ux[side]) {
            s->prof_ux[side] = (double *)malloc(sizeof(double) * len);
            memcpy(s->prof_ux[side], lat->bc_ux[side], sizeof(double) * len);
        }
        if (lat->bc_uy[side]) {
            s->prof_uy[side] = (double *)malloc(sizeof(double) * len);
            memcpy(s->prof_uy[side], lat->bc_uy[side], sizeof(double) * len);
        }
    }
    size_t n = (size_t)Q * lat->nx * lat->ny;
    s->ft = (double *)calloc(n, sizeof(double));
    s->fn = (double *)calloc(n, sizeof(double));
    s->conv_prev = (double *)calloc((size_t)Q * lat->ny, sizeof(double));
    s->conv_next = (double *)calloc((size_t)Q * lat->ny, sizeof(double));
    s->hist_cap = hist_cap > 0 ? hist_cap : 1;
    s->hist = (orc_record *)calloc((size_t)s->hist_cap * (nb > 0 ? nb : 1), sizeof(orc_record));
    if (!s->ft || !s->fn || !s->hist) { orc_free(s); return NULL; }
    for (int k = 0; k < nb; ++k) {
        const orc_body *b = &s->body[k];
        s->q[k][0] = b->x; s->q[k][1] = b->y; s->q[k][2] = b->theta;
        s->v[k][0] = b->vx; s->v[k][1] = b->vy; s->v[k][2] = b->omega;
        if (b->present && b->motion == ORC_IMPOSED)
            s->q_center[k] = s->q[k][b->axis] - b->amp * sin(b->phase);
    }
    s->step = 0;
    return s;
}

orc_sim *orc_create(const orc_lattice *lat, const orc_body *body, long long hist_cap)
{
    return orc_create_bodies(lat, body, body && body->present ? 1 : 0, hist_cap);
}

void orc_free(orc_sim *s)
{
    if (!s) return;
    for (int side = 0; side < 4; ++side) { free(s->prof_ux[side]); free(s->prof_uy[side]); }
    free(s->ft); free(s->fn); free(s->hist); free(s->conv_prev); free(s->conv_next); free(s);
}

static void reset_outlet(orc_sim *s);

/* State = equilibrium (Eq. 11) of the given fields (NULL: rho0, 0). */
void orc_init_equilibrium(orc_sim *s, const double *rho, const double *ux, const double *uy)
{
    const int nx = s->lat.nx, ny = s->lat.ny;
    double feq[Q];
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = (size_t)j * nx + i;
            equilibrium(rho ? rho[k] : s->lat.rho0, ux ? ux[k] : 0.0, uy ? uy[k] : 0.0, feq);
            for (int a = 0; a < Q; ++a) s->ft[((size_t)a * ny + j) * nx + i] = feq[a];
        }
    reset_outlet(s);
}

/* The convective outlet's "previous step" values at step 0 are the given
 * populations of the outlet column. */
static void reset_outlet(orc_sim *s)
{
    const int nx = s->lat.nx, ny = s->lat.ny;
    for (int a = 0; a < Q; ++a)
        for (int j = 0; j < ny; ++j) s->conv_prev[(size_t)a * ny + j] = s->ft[((size_t)a * ny + j) * nx + nx - 1];
}

void orc_set_populations(orc_sim *s, const double *f)
{
    memcpy(s->ft, f, sizeof(double) * (size_t)Q * s->lat.nx * s->lat.ny);
    reset_outlet(s);
}

void orc_get_populations(const orc_sim *s, double *f)
{
    memcpy(f, s->ft, sizeof(double) * (size_t)Q * s->lat.nx * s->lat.ny);
}

/* rho(n), u(n) of Eqs. (19)-(22) at the current step. */
void orc_get_fields(const orc_sim *s, double *rho, double *ux, double *uy)
{
    const int nx = s->lat.nx, ny = s->lat.ny;
    node_state ns;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            node_macro(s, i, j, &ns);
            size_t k = (size_t)j * nx + i;
            if (rho) rho[k] = ns.rho;
            if (ux) ux[k] = ns.ux;
            if (uy) uy[k] = ns.uy;
        }
}

/* One time step of Algorithm 1. */
static void one_step(orc_sim *s)
{
    const int nx = s->lat.nx, ny = s->lat.ny;
    node_state ns;
    double ft[Q];
    double fpen[ORC_MAXB][3] = {{0}}, fh[ORC_MAXB][3] = {{0}};
    double nsolid[ORC_MAXB] = {0};
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            node_macro(s, i, j, &ns);
            if (i == nx - 1)
                for (int a = 0; a < Q; ++a) s->conv_next[(size_t)a * ny + j] = ns.f[a];
            double Gx = ns.rho * (s->lat.gx + ns.ax);
            double Gy = ns.rho * (s->lat.gy + ns.ay);
            if (s->lat.collision == ORC_BGK)
                collide_bgk(ns.f, s->lat.s[7], ns.rho, ns.ux, ns.uy, Gx, Gy, ft);
            else
                collide(ns.f, s->lat.s, ns.rho, ns.ux, ns.uy, Gx, Gy, ft);
            for (int a = 0; a < Q; ++a) s->fn[((size_t)a * ny + j) * nx + i] = ft[a];
            if (ns.chi) {
                const int k = ns.owner;
                /* reaction of the penalization force on the body */
                double px = (PLANT(16) ? 1.0 : -1.0) * ns.rho * ns.ax, py = (PLANT(16) ? 1.0 : -1.0) * ns.rho * ns.ay;
                fpen[k][0] += px;
                fpen[k][1] += py;
                fpen[k][2] += ns.dx * py - ns.dy * px;
                /* momentum brought into the node by the streaming (Eq. 25) */
                double ox = 0.0, oy = 0.0;
                for (int a = 0; a < Q; ++a) {
                    double own = s->ft[((size_t)a * ny + j) * nx + i];
                    ox += C[a][0] * own;
                    oy += C[a][1] * own;
                }
                double ex = PLANT(17) ? ns.jx : ns.jx - ox, ey = PLANT(17) ? ns.jy : ns.jy - oy;
                fh[k][0] += ex;
                fh[k][1] += ey;
                fh[k][2] += PLANT(6) ? ns.dy * ex - ns.dx * ey : ns.dx * ey - ns.dy * ex;   /* Eq. (27) */
                nsolid[k] += 1.0;
            }
        }
    double *t = s->ft; s->ft = s->fn; s->fn = t;
    t = s->conv_prev; s->conv_prev = s->conv_next; s->conv_next = t;

    for (int k = 0; k < (s->nb > 0 ? s->nb : 1); ++k) {
        const orc_body *b = &s->body[k];
        orc_record *r = &s->hist[(size_t)k * s->hist_cap + s->step % s->hist_cap];
        r->t = (double)s->step;
        r->fx = fh[k][0]; r->fy = fh[k][1]; r->torque = fh[k][2];
        double qref = 0.5 * s->lat.rho0 * b->d_ref * b->u_ref * b->u_ref;
        r->cd = qref > 0 ? fh[k][0] / qref : 0.0;
        r->cl = qref > 0 ? fh[k][1] / qref : 0.0;
        r->x = s->q[k][0]; r->y = s->q[k][1]; r->theta = s->q[k][2];
        r->vx = s->v[k][0]; r->vy = s->v[k][1]; r->omega = s->v[k][2];
        r->fpen_x = fpen[k][0]; r->fpen_y = fpen[k][1]; r->tpen = fpen[k][2];
        r->n_solid = nsolid[k];
        if (b->present) body_advance(b, s->step, s->q_center[k], fh[k], s->q[k], s->v[k]);
    }
    s->step += 1;
}

void orc_step(orc_sim *s, long long n)
{
    for (long long k = 0; k < n; ++k) one_step(s);
}

long long orc_get_step(const orc_sim *s) { return s->step; }

/* Copies records first .. first+count-1 of body k (must still be in the ring). */
int orc_get_history_body(const orc_sim *s, int k, long long first, long long count, orc_record *dst)
{
    if (k < 0 || k >= (s->nb > 0 ? s->nb : 1)) return -1;
    if (first < 0 || count < 0 || first + count > s->step) return -1;
    if (first < s->step - s->hist_cap) return -1;
    for (long long n = 0; n < count; ++n) dst[n] = s->hist[(size_t)k * s->hist_cap + (first + n) % s->hist_cap];
    return 0;
}

int orc_get_history(const orc_sim *s, long long first, long long count, orc_record *dst)
{
    return orc_get_history_body(s, 0, first, count, dst);
}

void orc_get_body_k(const orc_sim *s, int k, double q[3], double v[3])
{
    for (int d = 0; d < 3; ++d) { q[d] = s->q[k][d]; v[d] = s->v[k][d]; }
}

void orc_get_body(const orc_sim *s, double q[3], double v[3]) { orc_get_body_k(s, 0, q, v); }

/* ---- single-node entry points used by the pinning tests ------------- */

void orc_constants(int c[Q][2], double w[Q], double m[Q][Q], double minv[Q][Q])
{
    setup_constants();
    memcpy(c, C, sizeof(C)); memcpy(w, W, sizeof(W));
    memcpy(m, M, sizeof(M)); memcpy(minv, MINV, sizeof(MINV));
}

void orc_equilibrium(double rho, double ux, double uy, double feq[Q])
{
    setup_constants();
    equilibrium(rho, ux, uy, feq);
}

void orc_moment_equilibrium(double rho, double ux, double uy, double meq[Q])
{
    moment_equilibrium(rho, ux, uy, meq);
}

void orc_guo_forcing(double ux, double uy, double Gx, double Gy, double F[Q])
{
    setup_constants();
    guo_forcing(ux, uy, Gx, Gy, F);
}

void orc_collide(const double f[Q], const double s[Q], double rho, double ux,
                 double uy, double Gx, double Gy, double ft[Q])
{
    setup_constants();
    collide(f, s, rho, ux, uy, Gx, Gy, ft);
}

void orc_collide_bgk(const double f[Q], double omega, double rho, double ux,
                     double uy, double Gx, double Gy, double ft[Q])
{
    setup_constants();
    collide_bgk(f, omega, rho, ux, uy, Gx, Gy, ft);
}

void orc_penalized_velocity(double rho, double jx, double jy, int chi, double usx,
                            double usy, double eta, double gx, double gy, double out[4])
{
    penalized_velocity(rho, jx, jy, chi, usx, usy, eta, gx, gy, &out[0], &out[1], &out[2], &out[3]);
}

void orc_body_advance(const orc_body *b, long long step, double q_center,
                      const double F[3], double q[3], double v[3])
{
    body_advance(b, step, q_center, F, q, v);
}

/* ---- discrete adjoint of Algorithm 1 (body on a prescribed path) -------
 *
 * The state S_n is the post-collision population field entering step n;
 * one step is S_{n+1} = C(Pull(S_n)) node by node, and the force of step n
 * is F_h(n) = sum_{x in R(n)} [ sum_a c_a Pull(S_n)_a(x) - sum_a c_a S_n(a, x) ].
 * The objective (the second half-window [w0, N) of the run) is
 *   J = w_cd * J1 + w_cl * J2,  J1 = mean C_D(n),  J2 = sqrt(mean C_L(n)^2).
 * The reverse sweep carries L_n = dJ/dS_n:
 *   mu(x)  = (dC/df at f = Pull(S_n)(x))^T L_{n+1}(x) + [x in R(n)] dJ/dF_h(n) . c
 *   L_n    = Pull^T mu - [x in R(n)] dJ/dF_h(n) . c
 * and collects dJ/dtheta = sum_n L_{n+1}^T dC/dtheta + mu^T dPull/dtheta for
 * theta = the west wall's u_x profile, eta, s_nu (= s_7 = s_8), s_e (= s_1).
 * The collision is differentiated in reverse through its own steps (moments
 * by M, equilibria, Guo forcing, penalized velocity); Pull^T is the scatter
 * of each pulled value back onto the population it came from.  The body
 * pose only depends on time, so chi and u_s are fixed per step.
 */

typedef struct {
    long long nsteps;   /* N */
    long long w0;       /* objective window [w0, N) */
    double w_cd, w_cl;  /* weights of J1 and J2 */
} orc_adjoint_desc;

/* Source of the pull of population a into node (i, j): population b at
 * (si, sj); *wall = side of a velocity wall whose term 6 w_a rho0 c_a.u_w
 * is added (-1: none). */
static void pull_source(const orc_sim *s, int a, int i, int j, int *b, int *si_out, int *sj_out, int *wall)
{
    const int nx = s->lat.nx, ny = s->lat.ny;
    int si = i - C[a][0], sj = j - C[a][1];
    *wall = -1;
    if (sj < 0 || sj >= ny) {
        int side = sj < 0 ? ORC_SOUTH : ORC_NORTH;
        if (s->lat.bc_kind[side] == ORC_PERIODIC) {
            sj = (sj + ny) % ny;
        } else if (s->lat.bc_kind[side] == ORC_SYMMETRY) {
            int mi = i - C[a][0];
            if (mi < 0 || mi >= nx) mi = s->lat.bc_kind[ORC_WEST] == ORC_PERIODIC ? (mi + nx) % nx : i;
            *b = MIRY[a]; *si_out = mi; *sj_out = j;
            return;
        } else {
            *b = OPP[a]; *si_out = i; *sj_out = j;
            if (s->lat.bc_kind[side] == ORC_VELOCITY) *wall = side;
            return;
        }
    }
    if (si < 0 || si >= nx) {
        int side = si < 0 ? ORC_WEST : ORC_EAST;
        int kind = s->lat.bc_kind[side];
        if (kind == ORC_PERIODIC) {
            si = (si + nx) % nx;
        } else if (kind == ORC_ZEROGRAD) {
            *b = a; *si_out = i; *sj_out = sj;
            return;
        } else {
            *b = OPP[a]; *si_out = i; *sj_out = j;
            if (kind == ORC_VELOCITY) *wall = side;
            return;
        }
    }
    *b = a; *si_out = si; *sj_out = sj;
}

/* Reverse of the node update f -> f~ = C(f): given xi = dJ/df~, returns
 * mu = (dC/df)^T xi, and adds xi^T dC/d(eta) to *d_eta and xi^T dC/ds_r to
 * d_s[r]. */
static void collide_adjoint(const double f[Q], const double s[Q], int chi, double usx, double usy, double eta,
                            double gx, double gy, const double xi[Q], double mu[Q], double *d_eta, double d_s[Q])
{
    /* forward intermediates */
    double rho = 0, jx = 0, jy = 0;
    for (int a = 0; a < Q; ++a) { rho += f[a]; jx += C[a][0] * f[a]; jy += C[a][1] * f[a]; }
    const double c = (double)chi;
    const double k = 1.0 / (eta + 0.5 * c);
    const double vx = jx / rho + 0.5 * gx, vy = jy / rho + 0.5 * gy;
    const double ax = -c * k * (vx - usx), ay = -c * k * (vy - usy);
    const double ux = vx + 0.5 * ax, uy = vy + 0.5 * ay;
    const double Gx = rho * (gx + ax), Gy = rho * (gy + ay);
    double m[Q], meq[Q], F[Q], MF[Q];
    for (int r = 0; r < Q; ++r) { m[r] = 0; for (int a = 0; a < Q; ++a) m[r] += M[r][a] * f[a]; }
    moment_equilibrium(rho, ux, uy, meq);
    guo_forcing(ux, uy, Gx, Gy, F);
    for (int r = 0; r < Q; ++r) { MF[r] = 0; for (int a = 0; a < Q; ++a) MF[r] += M[r][a] * F[a]; }

    /* f~ = M^-1 m*  ->  lam_ms = M^-T xi */
    double lam_ms[Q], lam_m[Q], lam_meq[Q], lam_MF[Q], lam_F[Q];
    for (int r = 0; r < Q; ++r) { lam_ms[r] = 0; for (int a = 0; a < Q; ++a) lam_ms[r] += MINV[a][r] * xi[a]; }
    /* m*_r = m_r - s_r (m_r - meq_r) + (1 - s_r/2) MF_r */
    for (int r = 0; r < Q; ++r) {
        lam_m[r] = (1.0 - s[r]) * lam_ms[r];
        lam_meq[r] = s[r] * lam_ms[r];
        lam_MF[r] = (PLANT(10) ? 1.0 - s[r] : 1.0 - 0.5 * s[r]) * lam_ms[r];
        d_s[r] += lam_ms[r] * (-(m[r] - meq[r]) - 0.5 * MF[r]);
    }
    for (int a = 0; a < Q; ++a) { lam_F[a] = 0; for (int r = 0; r < Q; ++r) lam_F[a] += M[r][a] * lam_MF[r]; }
    double lam_rho = 0, lam_ux = 0, lam_uy = 0, lam_Gx = 0, lam_Gy = 0;
    /* meq(rho, u), Eq. (14) */
    {
        const double u2 = ux * ux + uy * uy;
        const double br[Q] = {1.0, -2.0 + 3.0 * u2, 1.0 - 3.0 * u2, ux, -ux, uy, -uy, ux * ux - uy * uy, ux * uy};
        const double dux[Q] = {0, 6 * ux, -6 * ux, 1, -1, 0, 0, 2 * ux, uy};
        const double duy[Q] = {0, 6 * uy, -6 * uy, 0, 0, 1, -1, -2 * uy, ux};
        for (int r = 0; r < Q; ++r) {
            lam_rho += lam_meq[r] * br[r];
            lam_ux += lam_meq[r] * rho * dux[r];
            lam_uy += lam_meq[r] * rho * duy[r];
        }
    }
    /* F(u, G), Eq. (12) without the prefactor: F_a = W_a [3 (c - u) + 9 (c.u) c] . G */
    for (int a = 0; a < Q; ++a) {
        const double cx = C[a][0], cy = C[a][1];
        const double cu = cx * ux + cy * uy;
        lam_Gx += lam_F[a] * W[a] * (3.0 * (cx - ux) + 9.0 * cu * cx);
        lam_Gy += lam_F[a] * W[a] * (3.0 * (cy - uy) + 9.0 * cu * cy);
        lam_ux += lam_F[a] * W[a] * ((-3.0 + 9.0 * cx * cx) * Gx + 9.0 * cx * cy * Gy);
        lam_uy += lam_F[a] * W[a] * (9.0 * cy * cx * Gx + (-3.0 + 9.0 * cy * cy) * Gy);
    }
    /* G = rho (g + a) */
    lam_rho += lam_Gx * (gx + ax) + lam_Gy * (gy + ay);
    double lam_ax = rho * lam_Gx, lam_ay = rho * lam_Gy;
    /* u = v + a/2 */
    double lam_vx = lam_ux, lam_vy = lam_uy;
    lam_ax += 0.5 * lam_ux;
    lam_ay += 0.5 * lam_uy;
    /* a = -chi k (v - u_s), k = 1/(eta + chi/2) */
    lam_vx += -c * k * lam_ax;
    lam_vy += -c * k * lam_ay;
    *d_eta += (lam_ax * (c * k * k * (vx - usx)) + lam_ay * (c * k * k * (vy - usy)));
    /* v = j / rho + g/2 */
    const double lam_jx = lam_vx / rho, lam_jy = lam_vy / rho;
    lam_rho += -(lam_vx * jx + lam_vy * jy) / (rho * rho);
    /* m = M f (direct path), rho = sum f, j = sum c f */
    for (int a = 0; a < Q; ++a) {
        double acc = 0;
        for (int r = 0; r < Q; ++r) acc += M[r][a] * lam_m[r];
        mu[a] = acc + lam_rho + C[a][0] * lam_jx + C[a][1] * lam_jy;
    }
}

/* Runs the forward from the current state for d->nsteps steps (the state
 * advances), then the reverse sweep.  grad (ny + 3 entries): dJ/du_in(j)
 * for the west wall's u_x profile, dJ/deta, dJ/ds_nu, dJ/ds_e.  out_j: J1,
 * J2.  Returns 0, or -1 if the body is free or the history ring is short. */
int orc_adjoint(orc_sim *s, const orc_adjoint_desc *d, double *grad, double out_j[2])
{
    const int nx = s->lat.nx, ny = s->lat.ny;
    const long long N = d->nsteps;
    if (s->nb > 1) return -1;
    if (s->body[0].present && s->body[0].motion == ORC_FREE) return -1;
    if (s->lat.collision != ORC_MRT) return -1;
    if (s->body[0].present && s->body[0].shape != ORC_DISK) return -1;
    for (int side = 0; side < 4; ++side)
        if (s->lat.bc_kind[side] == ORC_CONVECTIVE) return -1;
    if (N < 1 || d->w0 < 0 || d->w0 >= N || s->hist_cap < s->step + N) return -1;
    const size_t nf = (size_t)Q * nx * ny;
    const long long step0 = s->step;
    double *states = (double *)malloc(sizeof(double) * nf * (size_t)N);
    double *lam = (double *)calloc(nf, sizeof(double));
    double *nlam = (double *)calloc(nf, sizeof(double));
    double *mu = (double *)calloc(nf, sizeof(double));
    if (!states || !lam || !nlam || !mu) { free(states); free(lam); free(nlam); free(mu); return -1; }
    for (long long n = 0; n < N; ++n) {
        memcpy(states + nf * (size_t)n, s->ft, sizeof(double) * nf);
        one_step(s);
    }
    /* objectives from the recorded forces */
    const double qref = 0.5 * s->lat.rho0 * s->body[0].d_ref * s->body[0].u_ref * s->body[0].u_ref;
    const double nh = (double)(N - d->w0);
    double sum_cd = 0, sum_cl2 = 0;
    for (long long n = d->w0; n < N; ++n) {
        const orc_record *r = &s->hist[(step0 + n) % s->hist_cap];
        sum_cd += r->fx / qref;
        sum_cl2 += (r->fy / qref) * (r->fy / qref);
    }
    const double J1 = sum_cd / nh, J2 = sqrt(sum_cl2 / nh);
    out_j[0] = J1; out_j[1] = J2;

    for (int k = 0; k < ny + 3; ++k) grad[k] = 0.0;
    double d_eta = 0, d_s[Q] = {0};
    double *saved_ft = s->ft;
    double saved_q[3], saved_v[3];
    for (int dd = 0; dd < 3; ++dd) { saved_q[dd] = s->q[0][dd]; saved_v[dd] = s->v[0][dd]; }
    node_state ns;
    for (long long n = N - 1; n >= 0; --n) {
        const orc_record *r = &s->hist[(step0 + n) % s->hist_cap];
        s->ft = states + nf * (size_t)n;
        s->q[0][0] = r->x; s->q[0][1] = r->y; s->q[0][2] = r->theta;
        s->v[0][0] = r->vx; s->v[0][1] = r->vy; s->v[0][2] = r->omega;
        double wx = 0, wy = 0;   /* dJ/dF_h(n) */
        if (n >= d->w0) {
            wx = d->w_cd / (qref * nh);
            wy = (J2 > 0) ? d->w_cl * (r->fy / qref) / (J2 * qref * nh) : 0.0;
        }
        /* mu at every node */
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                node_macro(s, i, j, &ns);
                double xi[Q], m_loc[Q];
                for (int a = 0; a < Q; ++a) xi[a] = lam[((size_t)a * ny + j) * nx + i];
                collide_adjoint(ns.f, s->lat.s, ns.chi, ns.usx, ns.usy, s->lat.eta, s->lat.gx, s->lat.gy, xi, m_loc,
                                &d_eta, d_s);
                if (ns.chi)
                    for (int a = 0; a < Q; ++a) m_loc[a] += wx * C[a][0] + wy * C[a][1];
                for (int a = 0; a < Q; ++a) mu[((size_t)a * ny + j) * nx + i] = m_loc[a];
            }
        /* L_n = Pull^T mu - own term */
        memset(nlam, 0, sizeof(double) * nf);
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                for (int a = 0; a < Q; ++a) {
                    int b, si, sj, wall;
                    pull_source(s, a, i, j, &b, &si, &sj, &wall);
                    const double g = mu[((size_t)a * ny + j) * nx + i];
                    nlam[((size_t)b * ny + sj) * nx + si] += g;
                    if (wall == ORC_WEST && s->prof_ux[ORC_WEST])
                        grad[j] += (PLANT(11) ? -g : g) * 6.0 * W[a] * s->lat.rho0 * C[a][0];
                }
                if (!PLANT(9) && owner_at(s, i, j) >= 0)
                    for (int a = 0; a < Q; ++a) nlam[((size_t)a * ny + j) * nx + i] -= wx * C[a][0] + wy * C[a][1];
            }
        double *t = lam; lam = nlam; nlam = t;
    }
    grad[ny] = d_eta;
    grad[ny + 1] = d_s[7] + d_s[8];
    grad[ny + 2] = d_s[1];
    /* leave the simulation after its forward run */
    s->ft = saved_ft;
    for (int dd = 0; dd < 3; ++dd) { s->q[0][dd] = saved_q[dd]; s->v[0][dd] = saved_v[dd]; }
    free(states); free(lam); free(nlam); free(mu);
    return 0;
}
