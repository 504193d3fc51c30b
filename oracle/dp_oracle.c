/*
 * dp_oracle.c -- FP64 CPU oracle for the semi-Lagrangian (SL) Bellman scheme of
 * Ciancarelli, Ferretti, Intelisano, Villani, "Dynamic Programming Techniques
 * for Planar Orbital Transfer of Low Earth Orbit Satellites" (arXiv 2407.14675).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the GPU path computes.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the library path
 * never calls it.  It shares no code, header or table with the CUDA sources.
 *
 * Everything is double precision, single threaded, one node at a time, in the
 * order the paper states the steps:
 *   - dynamics: polar form of the planar two-body problem, §3 "Grid and polar
 *     coordinates" (unnumbered system), with the angle coordinate dropped, the
 *     mass added as a state (m' = -a/c), the centrifugal term taken with a plus
 *     sign (the printed minus sign contradicts the circular-orbit equilibrium)
 *     and the thrust angle measured from the local horizontal (sin -> radial,
 *     cos -> tangential);
 *   - one-step map: second-order Runge-Kutta (Heun) over dt, §3 after Eq. (10);
 *   - interpolation: multilinear Q1 over the 2^4 corners of the cell, §3 after
 *     Eq. (10); a foot outside the box, or in a cell with a corner outside the
 *     reduced node set, is charged the penalty M (§3 "Grid and polar
 *     coordinates");
 *   - the fixed-point scheme Eq. (10) with running cost l = 1 (minimum time),
 *     value iteration Eq. (12), policy evaluation Eq. (13) and improvement
 *     Eq. (14);
 *   - the minimisation of §3 "Efficient computation of the minimum": tabulated
 *     angles, local walk from the previous optimum, golden-section refinement
 *     (in its discrete form, the Fibonacci search, on the 16-bit angle lattice);
 *   - the approximate optimal feedback Eq. (15) and its fourth-order
 *     Runge-Kutta closed loop (§3 "Computation of the approximate optimal
 *     solution");
 *   - the paper's own Example 1 setting (§4): the polar system with the angle
 *     theta kept as a periodic coordinate and no mass, the running cost of
 *     Eq. (11) in polar form (semi-major axis by the vis-viva relation, the
 *     eccentricity components e cos(omega), e sin(omega) from the
 *     eccentricity vector), and a thrust-off control besides the angles;
 *   - Example 2 (§4): the closed loop of the same feedback on a "real"
 *     system with aerodynamic drag, whose components are printed as
 *     -C v_rho^2 and -C v_theta^2 with C = C_D S rho_D / (2 m).
 *
 * Parity unpinned: the paper prints no value function, policy or trajectory
 * value (its figures are not available); the pins of this oracle are closed
 * forms and invariants checked by the test suite.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NCODES 65536
#define ORC_PI 3.14159265358979323846

enum { ORC_DYN_ORBIT = 0, ORC_DYN_UNIT_SPEED = 1, ORC_DYN_POLAR = 2 };
#define ORC_CODE_OFF 65535   /* policy code of the thrust-off control (grids with off_control) */
enum { ORC_VI = 0, ORC_IMPROVE_FULL = 1, ORC_IMPROVE_WALK = 2, ORC_EVAL = 3 };

typedef struct orc_problem {
    int n[4];            /* nodes per dimension (r, v_r, v_t, m) */
    double lo[4], hi[4]; /* box */
    int dynamics;
    double mu, accel, exhaust_c;
    double dt, beta, M;  /* pseudo-time step, discount exp(-lambda dt), penalty */
    double tgt_c[4], tgt_w[4]; /* open target box; tgt_w[d] <= 0: any value */
    int K;               /* tabulated angles 2 pi k / K */
    int refine;          /* golden-section refinement */
    double refine_tol;   /* rad */
    int reduced;         /* energy-band node set */
    double e_lo, e_hi;
    /* Example 1 (ORC_DYN_POLAR): state (rho, v_rho, v_theta, theta), theta
     * periodic with n[3] nodes over 2 pi; running cost of Eq. (11) */
    int off_control;     /* 1: a thrust-off control besides the angles */
    double cost_alpha, cost_beta, cost_gamma;   /* weights of |u|, (a - a_bar)^2, eccentricity */
    double a_bar, e_bar, omega_bar;             /* target orbit */
} orc_problem;

/* ------------------------------------------------------------------ grid -- */

static double spacing(const orc_problem* p, int d)
{
    return (p->hi[d] - p->lo[d]) / (double)(p->n[d] - 1);
}

/* The last coordinate is periodic (the orbital angle) in Example 1. */
static int periodic(const orc_problem* p, int d)
{
    return p->dynamics == ORC_DYN_POLAR && d == 3;
}

long orc_node_count(const orc_problem* p)
{
    return (long)p->n[0] * p->n[1] * p->n[2] * p->n[3];
}

static void node_index(const orc_problem* p, long j, int idx[4])
{
    for (int d = 3; d >= 0; --d) {
        idx[d] = (int)(j % p->n[d]);
        j /= p->n[d];
    }
}

static long flat_index(const orc_problem* p, const int idx[4])
{
    long j = 0;
    for (int d = 0; d < 4; ++d) j = j * p->n[d] + idx[d];
    return j;
}

static void node_state(const orc_problem* p, const int idx[4], double x[4])
{
    for (int d = 0; d < 4; ++d) x[d] = p->lo[d] + idx[d] * spacing(p, d);
}

int orc_in_target(const orc_problem* p, const double x[4])
{
    for (int d = 0; d < 4; ++d)
        if (p->tgt_w[d] > 0.0 && !(fabs(x[d] - p->tgt_c[d]) < p->tgt_w[d])) return 0;
    return 1;
}

/* Specific orbital energy v^2/2 - mu/r, §3 (definition of the energy). */
double orc_energy(const orc_problem* p, const double x[4])
{
    return 0.5 * (x[1] * x[1] + x[2] * x[2]) - p->mu / x[0];
}

/* Orbital elements of a polar state (rho, v_rho, v_theta, theta) (§3 "Grid and
 * polar coordinates"): semi-major axis by the vis-viva relation
 * a = mu rho / (2 mu - rho v^2), and the eccentricity vector
 * e = ((v^2 - mu/rho) r - (r . v) v) / mu, whose radial and transverse
 * components are rho v_theta^2 / mu - 1 and -rho v_rho v_theta / mu; rotated by
 * theta they give e cos(omega) and e sin(omega). */
void orc_elements(const orc_problem* p, const double x[4], double* a, double* ex, double* ey)
{
    double r = x[0], vr = x[1], vt = x[2], th = x[3];
    double v2 = vr * vr + vt * vt;
    *a = p->mu * r / (2.0 * p->mu - r * v2);
    double er = r * vt * vt / p->mu - 1.0;
    double et = -r * vr * vt / p->mu;
    *ex = er * cos(th) - et * sin(th);
    *ey = er * sin(th) + et * cos(th);
}

/* Running cost l(x, u) of Eq. (11) in polar form: alpha |u| + beta (a - a_bar)^2
 * + gamma ((e cos w - e_bar cos w_bar)^2 + (e sin w - e_bar sin w_bar)^2);
 * |u| = thrust acceleration (0 when off).  Minimum time (l = 1) otherwise. */
double orc_running_cost(const orc_problem* p, const double x[4], int thrust_on)
{
    if (p->dynamics != ORC_DYN_POLAR) return 1.0;
    double a, ex, ey;
    orc_elements(p, x, &a, &ex, &ey);
    double dx = ex - p->e_bar * cos(p->omega_bar), dy = ey - p->e_bar * sin(p->omega_bar);
    return p->cost_alpha * (thrust_on ? p->accel : 0.0) + p->cost_beta * (a - p->a_bar) * (a - p->a_bar) +
           p->cost_gamma * (dx * dx + dy * dy);
}

/* Reduced grid: keep the node iff its energy lies in [e_lo, e_hi]. */
static int node_active(const orc_problem* p, const double x[4])
{
    if (!p->reduced) return 1;
    double e = orc_energy(p, x);
    return e >= p->e_lo && e <= p->e_hi;
}

/* Fills active[] and target[] (one byte per box node); returns active count. */
long orc_build_masks(const orc_problem* p, unsigned char* active, unsigned char* target)
{
    long N = orc_node_count(p), count = 0;
    for (long j = 0; j < N; ++j) {
        int idx[4];
        double x[4];
        node_index(p, j, idx);
        node_state(p, idx, x);
        active[j] = (unsigned char)node_active(p, x);
        target[j] = (unsigned char)(active[j] && orc_in_target(p, x));
        count += active[j];
    }
    return count;
}

/* -------------------------------------------------------------- dynamics -- */

/* Right-hand side b(x, alpha).  Orbit: r' = v_r, v_r' = v_t^2/r - mu/r^2 +
 * (a/m) sin alpha, v_t' = -v_r v_t / r + (a/m) cos alpha, m' = -a/c.
 * Polar (Example 1): the same with thrust acceleration a (no mass) and the
 * angle theta' = v_t / r as last coordinate; alpha = NAN is thrust off. */
void orc_dynamics(const orc_problem* p, const double x[4], double alpha, double f[4])
{
    if (p->dynamics == ORC_DYN_POLAR) {
        double r = x[0], vr = x[1], vt = x[2];
        double u = isnan(alpha) ? 0.0 : p->accel;
        double sa = isnan(alpha) ? 0.0 : sin(alpha), ca = isnan(alpha) ? 0.0 : cos(alpha);
        f[0] = vr;
        f[1] = vt * vt / r - p->mu / (r * r) + u * sa;
        f[2] = -vr * vt / r + u * ca;
        f[3] = vt / r;
    } else if (p->dynamics == ORC_DYN_ORBIT) {
        double r = x[0], vr = x[1], vt = x[2], m = x[3];
        double am = p->accel / m;
        f[0] = vr;
        f[1] = vt * vt / r - p->mu / (r * r) + am * sin(alpha);
        f[2] = -vr * vt / r + am * cos(alpha);
        f[3] = -p->accel / p->exhaust_c;
    } else {
        /* test dynamics: unit speed in the (x0, x1) plane; components below
         * 1e-12 are exact zeros so that axis-aligned moves stay on grid lines */
        double c = cos(alpha), s = sin(alpha);
        if (fabs(c) < 1e-12) c = 0.0;
        if (fabs(s) < 1e-12) s = 0.0;
        f[0] = c;
        f[1] = s;
        f[2] = 0.0;
        f[3] = 0.0;
    }
}

/* Second-order Runge-Kutta (Heun) displacement over h with the control held:
 * k1 = b(x), k2 = b(x + h k1), delta = h (k1 + k2) / 2. */
void orc_heun_displacement(const orc_problem* p, const double x[4], double alpha, double h,
                           double delta[4])
{
    double k1[4], k2[4], xt[4];
    orc_dynamics(p, x, alpha, k1);
    for (int d = 0; d < 4; ++d) xt[d] = x[d] + h * k1[d];
    orc_dynamics(p, xt, alpha, k2);
    for (int d = 0; d < 4; ++d) delta[d] = 0.5 * h * (k1[d] + k2[d]);
}

/* The "real" system of Example 2: the model plus aerodynamic drag with the
 * printed components -C v_rho^2 (radial) and -C v_theta^2 (transverse);
 * polar dynamics only (drag_c = 0 gives the model). */
void orc_dynamics_drag(const orc_problem* p, const double x[4], double alpha, double drag_c, double f[4])
{
    orc_dynamics(p, x, alpha, f);
    if (p->dynamics == ORC_DYN_POLAR && drag_c != 0.0) {
        f[1] -= drag_c * x[1] * x[1];
        f[2] -= drag_c * x[2] * x[2];
    }
}

/* Classical fourth-order Runge-Kutta step of the true dynamics (with drag). */
static void rk4_step_drag(const orc_problem* p, const double x[4], double alpha, double h, double drag_c,
                          double out[4])
{
    double k1[4], k2[4], k3[4], k4[4], y[4];
    orc_dynamics_drag(p, x, alpha, drag_c, k1);
    for (int d = 0; d < 4; ++d) y[d] = x[d] + 0.5 * h * k1[d];
    orc_dynamics_drag(p, y, alpha, drag_c, k2);
    for (int d = 0; d < 4; ++d) y[d] = x[d] + 0.5 * h * k2[d];
    orc_dynamics_drag(p, y, alpha, drag_c, k3);
    for (int d = 0; d < 4; ++d) y[d] = x[d] + h * k3[d];
    orc_dynamics_drag(p, y, alpha, drag_c, k4);
    for (int d = 0; d < 4; ++d) out[d] = x[d] + h / 6.0 * (k1[d] + 2.0 * k2[d] + 2.0 * k3[d] + k4[d]);
}

/* Classical fourth-order Runge-Kutta step of the true dynamics. */
void orc_rk4_step(const orc_problem* p, const double x[4], double alpha, double h, double out[4])
{
    rk4_step_drag(p, x, alpha, h, 0.0, out);
}

/* --------------------------------------------------------- interpolation -- */

/* Q1 interpolation of V at the point s given in grid units (s_d = 0 at lo_d,
 * n_d - 1 at hi_d).  Returns 0 when the point is outside the box (strictly)
 * or a corner of its cell is not in the node set; the caller then uses M. */
/* Q1 interpolation of §3 (after Eq. (10)) at grid coordinates s: the flat
 * indices and weights of the 2^4 cell corners, weights the products of
 * (1 - t_d) or t_d.  Returns 0 when s leaves the box (in a non-periodic
 * dimension) or a corner is outside the node set (active may be NULL). */
static int interp_corners(const orc_problem* p, const unsigned char* active, const double s[4], long idx16[16],
                          double w16[16])
{
    int cell[4];
    double t[4];
    for (int d = 0; d < 4; ++d) {
        if (periodic(p, d)) {
            /* the angle wraps: cells run from node n-1 back to node 0 */
            if (!isfinite(s[d])) return 0;
            double f = floor(s[d]);
            t[d] = s[d] - f;
            long c = (long)f % p->n[d];
            cell[d] = (int)(c < 0 ? c + p->n[d] : c);
            continue;
        }
        if (!(s[d] >= 0.0 && s[d] <= (double)(p->n[d] - 1))) return 0;
        int c = (int)floor(s[d]);
        if (c > p->n[d] - 2) c = p->n[d] - 2;
        cell[d] = c;
        t[d] = s[d] - c;
    }
    for (int b = 0; b < 16; ++b) {
        int idx[4];
        double w = 1.0;
        for (int d = 0; d < 4; ++d) {
            int bit = (b >> (3 - d)) & 1;
            idx[d] = cell[d] + bit;
            if (periodic(p, d) && idx[d] == p->n[d]) idx[d] = 0;
            w *= bit ? t[d] : 1.0 - t[d];
        }
        long j = flat_index(p, idx);
        if (active && !active[j]) return 0;
        idx16[b] = j;
        w16[b] = w;
    }
    return 1;
}

int orc_interp(const orc_problem* p, const double* V, const unsigned char* active,
               const double s[4], double* out)
{
    long idx[16];
    double w[16];
    if (!interp_corners(p, active, s, idx, w)) return 0;
    double acc = 0.0;
    for (int b = 0; b < 16; ++b) acc += w[b] * V[idx[b]];
    *out = acc;
    return 1;
}

/* ------------------------------------------------------ Bellman operator -- */

static double code_angle(long code)
{
    long c = code % ORC_NCODES;
    if (c < 0) c += ORC_NCODES;
    return 2.0 * ORC_PI * (double)c / (double)ORC_NCODES;
}

/* Control of a policy code: the angle, or NAN for thrust off. */
static double code_control(const orc_problem* p, long code)
{
    if (p->off_control && code == ORC_CODE_OFF) return NAN;
    return code_angle(code);
}

/* Code of the k-th tabulated angle 2 pi k / K on the 16-bit lattice. */
static long table_code(int K, long k)
{
    return (k * ORC_NCODES + K / 2) / K;
}

/* Nearest tabulated index to a code (start of the local walk). */
static int nearest_table_index(int K, long code)
{
    return (int)(((code * K + ORC_NCODES / 2) / ORC_NCODES) % K);
}

/* Term of Eq. (10) at grid node idx for control alpha (NAN: thrust off):
 * dt * l(x_j, alpha) + beta * I[V](x_j + dt Phi(x_j, alpha)). */
double orc_q_node(const orc_problem* p, const double* V, const unsigned char* active,
                  const int idx[4], double alpha)
{
    double x[4], delta[4], s[4], I;
    node_state(p, idx, x);
    orc_heun_displacement(p, x, alpha, p->dt, delta);
    for (int d = 0; d < 4; ++d) s[d] = idx[d] + delta[d] / spacing(p, d);
    if (!orc_interp(p, V, active, s, &I)) I = p->M;
    return p->dt * orc_running_cost(p, x, !isnan(alpha)) + p->beta * I;
}

/* Row j of the policy-evaluation system, Eq. (13) at a frozen control code:
 * the update of node j is affine in V,
 *     V_j = b_j + beta * sum_c w_c V_{idx_c},
 * with w_c the Q1 weights of the node's foot.  b_j is dt l(x_j, control),
 * plus beta M when the foot leaves the box or the node set (the row is then
 * empty).  A target node has V_j = 0 and an inactive node V_j = M: b_j is
 * that value and the row is empty.  Returns the number of weights (16 or 0). */
int orc_policy_row(const orc_problem* p, const unsigned char* active, const unsigned char* target, long j,
                   unsigned code, long idx16[16], double w16[16], double* b)
{
    if (!active[j]) { *b = p->M; return 0; }
    if (target[j]) { *b = 0.0; return 0; }
    int node[4];
    double x[4], delta[4], s[4];
    node_index(p, j, node);
    node_state(p, node, x);
    double a = code_control(p, code);
    orc_heun_displacement(p, x, a, p->dt, delta);
    for (int d = 0; d < 4; ++d) s[d] = node[d] + delta[d] / spacing(p, d);
    double run = p->dt * orc_running_cost(p, x, !isnan(a));
    if (!interp_corners(p, active, s, idx16, w16)) {
        *b = run + p->beta * p->M;
        return 0;
    }
    *b = run;
    return 16;
}

/* Every row of the policy-evaluation system (orc_policy_row): idx and w hold
 * 16 entries per node (count[j] of them used), b one value per node. */
void orc_policy_system(const orc_problem* p, const unsigned char* active, const unsigned char* target,
                       const uint16_t* code, long* idx, double* w, double* b, int* count)
{
    long N = orc_node_count(p);
    for (long j = 0; j < N; ++j)
        count[j] = orc_policy_row(p, active, target, j, code[j], idx + 16 * j, w + 16 * j, b + j);
}

/* Foot of the one-step map from grid node idx in grid units (test helper:
 * tells how close a foot lies to a cell face). */
void orc_foot_node(const orc_problem* p, const int idx[4], double alpha, double s[4])
{
    double x[4], delta[4];
    node_state(p, idx, x);
    orc_heun_displacement(p, x, alpha, p->dt, delta);
    for (int d = 0; d < 4; ++d) s[d] = idx[d] + delta[d] / spacing(p, d);
}

/* Term of Eq. (15) at an arbitrary state y with feedback step tau: the
 * discount over tau is beta^(tau/dt) = exp(-lambda tau). */
double orc_q_state(const orc_problem* p, const double* V, const unsigned char* active,
                   const double y[4], double alpha, double tau)
{
    double delta[4], s[4], I;
    orc_heun_displacement(p, y, alpha, tau, delta);
    for (int d = 0; d < 4; ++d) s[d] = (y[d] + delta[d] - p->lo[d]) / spacing(p, d);
    if (!orc_interp(p, V, active, s, &I)) I = p->M;
    return tau * orc_running_cost(p, y, !isnan(alpha)) + pow(p->beta, tau / p->dt) * I;
}

typedef struct {
    const orc_problem* p;
    const double* V;
    const unsigned char* active;
    const int* idx;   /* grid node, or NULL for an arbitrary state */
    const double* y;
    double tau;
    long evals;
} q_ctx;

static double q_of_code(q_ctx* c, long code)
{
    c->evals++;
    double a = code_control(c->p, code);
    if (c->idx) return orc_q_node(c->p, c->V, c->active, c->idx, a);
    return orc_q_state(c->p, c->V, c->active, c->y, a, c->tau);
}

/* Full enumeration of the tabulated angles; ties go to the lowest index. */
static int enumerate_table(q_ctx* c, double* qbest)
{
    int K = c->p->K, kb = 0;
    double qb = q_of_code(c, table_code(K, 0));
    for (int k = 1; k < K; ++k) {
        double q = q_of_code(c, table_code(K, k));
        if (q < qb) { qb = q; kb = k; }
    }
    *qbest = qb;
    return kb;
}

/* Local walk from the previous optimum: move one tabulated step towards the
 * strictly lower neighbour (left wins a tie between neighbours) until neither
 * neighbour is lower. */
static int walk_table(q_ctx* c, int k0, double* qbest)
{
    int K = c->p->K, k = k0;
    double qk = q_of_code(c, table_code(K, k));
    for (int step = 0; step < K; ++step) {
        int kl = (k + K - 1) % K, kr = (k + 1) % K;
        double ql = q_of_code(c, table_code(K, kl));
        double qr = q_of_code(c, table_code(K, kr));
        if (ql < qk && ql <= qr) { k = kl; qk = ql; }
        else if (qr < qk) { k = kr; qk = qr; }
        else break;
    }
    *qbest = qk;
    return k;
}

/* A refinement point that the search may not evaluate: beyond the upper
 * tabulated neighbour, or (grids with the off control) the lattice code that
 * stands for thrust off. */
static int excluded(const q_ctx* c, long ck, long x, long hi_off)
{
    if (x >= hi_off) return 1;
    long w = (ck + x) % ORC_NCODES;
    if (w < 0) w += ORC_NCODES;
    return c->p->off_control && w == ORC_CODE_OFF;
}

/* Golden-section refinement in its discrete form (Fibonacci search) on the
 * 16-bit angle lattice, inside the bracket formed by the two tabulated
 * neighbours of the tabulated minimiser k.  The interval is extended to a
 * Fibonacci length with +inf beyond the upper neighbour.  Returns the best
 * evaluated code (the tabulated minimiser included); *qbest its value. */
static long fibonacci_refine(q_ctx* c, int k, double qk, double* qbest)
{
    const orc_problem* p = c->p;
    int K = p->K;
    long ck = table_code(K, k);
    long cl = (k == 0) ? table_code(K, K - 1) - ORC_NCODES : table_code(K, k - 1);
    long cr = (k == K - 1) ? ORC_NCODES : table_code(K, k + 1);
    long lo_off = cl - ck, hi_off = cr - ck, L = hi_off - lo_off;

    long F[64];
    F[1] = 1; F[2] = 1;
    int n = 2;
    while (F[n] < L) { ++n; F[n] = F[n - 1] + F[n - 2]; }

    long best = ck;
    double qb = qk;
    const double step_rad = 2.0 * ORC_PI / ORC_NCODES;
    long a = lo_off;
    long x1 = a + F[n - 2], x2 = a + F[n - 1];
    double f1 = excluded(c, ck, x1, hi_off) ? INFINITY : q_of_code(c, ck + x1);
    double f2 = excluded(c, ck, x2, hi_off) ? INFINITY : q_of_code(c, ck + x2);
    if (f1 < qb) { qb = f1; best = ck + x1; }
    if (f2 < qb) { qb = f2; best = ck + x2; }
    /* interval [a, a + F[kk]] holds the points a + F[kk-2] and a + F[kk-1] */
    for (int kk = n; kk > 4 && F[kk] * step_rad > p->refine_tol; --kk) {
        if (f1 <= f2) {          /* keep [a, x2] */
            x2 = x1; f2 = f1;
            x1 = a + F[kk - 3];
            f1 = excluded(c, ck, x1, hi_off) ? INFINITY : q_of_code(c, ck + x1);
            if (f1 < qb) { qb = f1; best = ck + x1; }
        } else {                 /* keep [x1, a + F[kk]] */
            a = x1;
            x1 = x2; f1 = f2;
            x2 = a + F[kk - 2];
            f2 = excluded(c, ck, x2, hi_off) ? INFINITY : q_of_code(c, ck + x2);
            if (f2 < qb) { qb = f2; best = ck + x2; }
        }
    }
    *qbest = qb;
    long w = best % ORC_NCODES;
    return w < 0 ? w + ORC_NCODES : w;
}

/* One Bellman update at node j (Eq. (12), (13) or (14)).  code_in is the
 * frozen policy (EVAL) or the previous optimum (IMPROVE_WALK).  Writes the
 * new value and, for the improvement modes, the new policy code.  Returns
 * the number of control evaluations. */
long orc_bellman_node(const orc_problem* p, const double* V, const unsigned char* active,
                      const unsigned char* target, long j, int mode, unsigned code_in,
                      double* v_out, unsigned* code_out)
{
    int idx[4];
    node_index(p, j, idx);
    if (target[j]) { *v_out = 0.0; *code_out = code_in; return 0; }
    q_ctx c = { p, V, active, idx, NULL, 0.0, 0 };
    double q;
    if (mode == ORC_EVAL) {
        *v_out = q_of_code(&c, code_in);
        *code_out = code_in;
        return c.evals;
    }
    int k;
    /* a node whose previous control was off has no angle to walk from: it
     * tabulates in full */
    int walk = mode == ORC_IMPROVE_WALK && !(p->off_control && code_in == ORC_CODE_OFF);
    if (walk) k = walk_table(&c, nearest_table_index(p->K, code_in), &q);
    else k = enumerate_table(&c, &q);
    long code = table_code(p->K, k) % ORC_NCODES;
    if (mode != ORC_VI && p->refine) code = fibonacci_refine(&c, k, q, &q);
    if (p->off_control) {
        /* thrust off is one more control; it wins a tie */
        double q_off = q_of_code(&c, ORC_CODE_OFF);
        if (q_off <= q) { q = q_off; code = ORC_CODE_OFF; }
    }
    *v_out = q;
    *code_out = (unsigned)code;
    return c.evals;
}

/* A full Jacobi sweep: V_out = T(V_in) at every active node (inactive nodes
 * get M, target nodes 0).  codes may be NULL for VI.  Returns the sup-norm of
 * V_out - V_in over the node set; *evals accumulates control evaluations. */
double orc_sweep(const orc_problem* p, const double* V_in, double* V_out,
                 const unsigned char* active, const unsigned char* target,
                 int mode, const uint16_t* code_in, uint16_t* code_out, long* evals)
{
    long N = orc_node_count(p);
    double res = 0.0;
    for (long j = 0; j < N; ++j) {
        if (!active[j]) { V_out[j] = p->M; if (code_out) code_out[j] = code_in ? code_in[j] : 0; continue; }
        unsigned ci = code_in ? code_in[j] : 0, co = 0;
        double v;
        long e = orc_bellman_node(p, V_in, active, target, j, mode, ci, &v, &co);
        if (evals) *evals += e;
        V_out[j] = v;
        if (code_out) code_out[j] = (uint16_t)co;
        double dv = fabs(v - V_in[j]);
        if (dv > res || isnan(dv)) res = dv;
    }
    return res;
}

/* The same update at a list of nodes only (sampled parity at full size). */
void orc_bellman_nodes(const orc_problem* p, const double* V, const unsigned char* active,
                       const unsigned char* target, const long* nodes, long count, int mode,
                       const uint16_t* code_in, double* v_out, uint16_t* code_out)
{
    for (long i = 0; i < count; ++i) {
        unsigned co = 0;
        orc_bellman_node(p, V, active, target, nodes[i], mode, code_in ? code_in[i] : 0,
                         &v_out[i], &co);
        if (code_out) code_out[i] = (uint16_t)co;
    }
}

/* q at a list of (node, code) pairs: used to check near-tie decisions. */
void orc_q_nodes(const orc_problem* p, const double* V, const unsigned char* active,
                 const long* nodes, const uint16_t* codes, long count, double* q_out)
{
    for (long i = 0; i < count; ++i) {
        int idx[4];
        node_index(p, nodes[i], idx);
        q_out[i] = orc_q_node(p, V, active, idx, code_control(p, codes[i]));
    }
}

/* Value iteration Eq. (12): Jacobi sweeps until sup|V^{k+1} - V^k| < tol. */
long orc_value_iterate(const orc_problem* p, double* V, const unsigned char* active,
                       const unsigned char* target, double tol, long max_sweeps, double* res_out)
{
    long N = orc_node_count(p), s = 0;
    double* W = (double*)malloc(sizeof(double) * N);
    double res = INFINITY;
    while (s < max_sweeps) {
        res = orc_sweep(p, V, W, active, target, ORC_VI, NULL, NULL, NULL);
        memcpy(V, W, sizeof(double) * N);
        ++s;
        if (res < tol) break;
    }
    free(W);
    *res_out = res;
    return s;
}

/* Value iteration, Eq. (12), with each node's own coefficient solved: for a
 * control a the update of node j is V_j = c_a + beta w_jj^a V_j + beta R_a,
 * w_jj^a the node's own Q1 weight at its foot and R_a the rest of the blend,
 * and the sweep takes V'_j = min_a (c_a + beta R_a) / (1 - beta w_jj^a) over
 * the tabulated angles (ties to the lowest index).  A foot outside the box or
 * the node set gives c_a = dt + beta M.  The affine maps have slopes below 1,
 * so the fixed point of this sweep is that of Eq. (12).  Minimum time only
 * (l = 1, no thrust-off control).  Returns max |V' - V| over the node set. */
double orc_vi_diag_sweep(const orc_problem* p, const double* V_in, double* V_out, const unsigned char* active,
                         const unsigned char* target)
{
    long N = orc_node_count(p);
    double res = 0.0;
    for (long j = 0; j < N; ++j) {
        if (!active[j]) { V_out[j] = p->M; continue; }
        if (target[j]) { V_out[j] = 0.0; continue; }
        int node[4];
        double x[4];
        node_index(p, j, node);
        node_state(p, node, x);
        double best = INFINITY;
        for (int k = 0; k < p->K; ++k) {
            double a = code_angle(table_code(p->K, k)), delta[4], sgrid[4], w[16];
            long idx[16];
            orc_heun_displacement(p, x, a, p->dt, delta);
            for (int d = 0; d < 4; ++d) sgrid[d] = node[d] + delta[d] / spacing(p, d);
            double q;
            if (!interp_corners(p, active, sgrid, idx, w)) {
                q = p->dt + p->beta * p->M;
            } else {
                double self = 0.0, rest = 0.0;
                for (int b = 0; b < 16; ++b) {
                    if (idx[b] == j) self += w[b];
                    else rest += w[b] * V_in[idx[b]];
                }
                q = (p->dt + p->beta * rest) / (1.0 - p->beta * self);
            }
            if (q < best) best = q;
        }
        V_out[j] = best;
        double dv = fabs(best - V_in[j]);
        if (dv > res || isnan(dv)) res = dv;
    }
    return res;
}

/* Modified policy iteration: improvement Eq. (14) (full enumeration first,
 * then walk), n_eval Jacobi sweeps of Eq. (13) at the frozen policy, repeat
 * until an improvement sweep moves V by less than tol.  Returns the number of
 * improvement sweeps; *eval_sweeps the evaluation sweeps. */
long orc_policy_iterate(const orc_problem* p, double* V, uint16_t* code,
                        const unsigned char* active, const unsigned char* target,
                        double tol, long max_outer, int n_eval, int walk,
                        long* eval_sweeps, double* res_out)
{
    long N = orc_node_count(p), outer = 0;
    double* W = (double*)malloc(sizeof(double) * N);
    uint16_t* C = (uint16_t*)malloc(sizeof(uint16_t) * N);
    double res = INFINITY;
    *eval_sweeps = 0;
    while (outer < max_outer) {
        int mode = (outer == 0 || !walk) ? ORC_IMPROVE_FULL : ORC_IMPROVE_WALK;
        res = orc_sweep(p, V, W, active, target, mode, code, C, NULL);
        memcpy(V, W, sizeof(double) * N);
        memcpy(code, C, sizeof(uint16_t) * N);
        ++outer;
        if (res < tol) break;
        for (int e = 0; e < n_eval; ++e) {
            orc_sweep(p, V, W, active, target, ORC_EVAL, code, NULL, NULL);
            memcpy(V, W, sizeof(double) * N);
            ++*eval_sweeps;
        }
    }
    free(W);
    free(C);
    *res_out = res;
    return outer;
}

/* -------------------------------------------- feedback and closed loop -- */

/* Approximate optimal feedback Eq. (15) at n states: full tabulation, then the
 * same golden-section refinement as the improvement sweep. */
void orc_feedback(const orc_problem* p, const double* V, const unsigned char* active,
                  const double* states, long n, double tau, uint16_t* code_out, double* q_out)
{
    for (long i = 0; i < n; ++i) {
        q_ctx c = { p, V, active, NULL, states + 4 * i, tau, 0 };
        double q;
        int k = enumerate_table(&c, &q);
        long code = table_code(p->K, k) % ORC_NCODES;
        if (p->refine) code = fibonacci_refine(&c, k, q, &q);
        if (p->off_control) {
            double q_off = q_of_code(&c, ORC_CODE_OFF);
            if (q_off <= q) { q = q_off; code = ORC_CODE_OFF; }
        }
        code_out[i] = (uint16_t)code;
        if (q_out) q_out[i] = q;
    }
}

/* Closed loop: the feedback is recomputed every step of length h (held over
 * the step) and the true dynamics advance by one RK4 step.  Arrival is the
 * end of the first step inside the target; t_arrive = -1 if none before
 * t_max. */
void orc_simulate_drag(const orc_problem* p, const double* V, const unsigned char* active,
                       const double* x0, long n, double tau, double h, double t_max, double drag_c,
                       double* t_arrive, double* x_final);

void orc_simulate(const orc_problem* p, const double* V, const unsigned char* active,
                  const double* x0, long n, double tau, double h, double t_max,
                  double* t_arrive, double* x_final)
{
    orc_simulate_drag(p, V, active, x0, n, tau, h, t_max, 0.0, t_arrive, x_final);
}

/* The same closed loop on the "real" system with drag (Example 2). */
void orc_simulate_drag(const orc_problem* p, const double* V, const unsigned char* active,
                       const double* x0, long n, double tau, double h, double t_max, double drag_c,
                       double* t_arrive, double* x_final)
{
    long steps = (long)ceil(t_max / h - 1e-9);
    for (long i = 0; i < n; ++i) {
        double y[4], z[4];
        memcpy(y, x0 + 4 * i, sizeof y);
        t_arrive[i] = -1.0;
        for (long s = 0; s < steps; ++s) {
            uint16_t code;
            orc_feedback(p, V, active, y, 1, tau, &code, NULL);
            rk4_step_drag(p, y, code_control(p, code), h, drag_c, z);
            memcpy(y, z, sizeof y);
            if (orc_in_target(p, y)) { t_arrive[i] = (s + 1) * h; break; }
        }
        memcpy(x_final + 4 * i, y, sizeof y);
    }
}
