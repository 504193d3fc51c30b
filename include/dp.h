/*
 * dp.h -- C ABI of the GB300 semi-Lagrangian Bellman solver for planar
 * low-thrust orbit transfer (Ciancarelli, Ferretti, Intelisano, Villani,
 * "Dynamic Programming Techniques for Planar Orbital Transfer of Low Earth
 * Orbit Satellites", arXiv 2407.14675).
 *
 * The library solves the fixed-point scheme of §3, Eq. (10),
 *
 *     v_j = min_f { dt l(x_j, f) + beta I[V](x_j + dt Phi(x_j, f)) },
 *
 * on a 4-D grid of states x = (r, v_r, v_t, m) with running cost l = 1
 * (minimum time), beta = exp(-lambda dt), Phi a second-order Runge-Kutta
 * (Heun) step of the polar two-body dynamics with thrust (§3 "Grid and polar
 * coordinates", angle coordinate dropped, mass added with m' = -a/c), I[V]
 * the multilinear (Q1) interpolation, and I[V] = M for a foot outside the box
 * or the reduced node set.  The control is the thrust angle alpha (sin alpha
 * radial, cos alpha tangential); every policy is stored as a 16-bit angle
 * code, alpha = 2 pi code / 65536.
 *
 * Conventions for every call:
 *   - Return value: a DP_* status code.  On failure dp_last_error() gives a
 *     message (thread-local, valid until the next call on that thread).
 *   - Host pointers are owned by the caller and only read or written during
 *     the call; the library copies in and out and keeps no reference.
 *   - The library owns all device memory of a grid (allocated by
 *     dp_grid_create and by the first FP64 polish, freed by dp_grid_destroy).
 *   - All GPU work of a grid is issued on desc.stream (NULL: the legacy
 *     default stream) on the device that was current at dp_grid_create; calls
 *     that return host data synchronise that stream.
 *   - One grid handle must not be used by two threads at the same time.
 *
 * Node order: a box node (i_r, i_vr, i_vt, i_m) has box index
 * ((i_r n1 + i_vr) n2 + i_vt) n3 + i_m (mass fastest), coordinates
 * x_d = lo_d + i_d (hi_d - lo_d)/(n_d - 1).  Values and policies are exchanged
 * in "compact order": the stored nodes in ascending box index.  Without the
 * reduced grid every box node is stored and compact order is box order.
 */
#ifndef DP_H
#define DP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define DP_OK         0
#define DP_EINVAL     1  /* invalid argument or descriptor                     */
#define DP_ENOMEM     2  /* device or host allocation failed                   */
#define DP_ECUDA      3  /* a CUDA call failed                                 */
#define DP_ENOCONV    4  /* sweep budget reached before the tolerance; results
                            and statistics are valid                           */
#define DP_ETIMEOUT   5  /* a bounded device-side wait expired                 */
#define DP_ENONFINITE 6  /* a non-finite value met (input or iterate)          */

/* ---- enums ---- */
#define DP_FP64 0            /* FP64 geometry and FP64 values                     */
#define DP_FP32 1            /* FP32 geometry and values, FP64 residual / polish  */

#define DP_DYN_ORBIT      0  /* planar orbit (r, v_r, v_t, m), §3 polar dynamics   */
#define DP_DYN_UNIT_SPEED 1  /* test dynamics x' = (cos a, sin a, 0, 0); components
                                below 1e-12 in magnitude are taken as exact zeros  */
#define DP_DYN_POLAR      2  /* the paper's Example 1 (§4): state (rho, v_rho,
                                v_theta, theta), the polar system of §3 with thrust
                                acceleration `accel` and no mass; theta periodic
                                (n[3] nodes over 2 pi: hi[3] = lo[3] + 2 pi
                                (n[3]-1)/n[3]); running cost of Eq. (11); FP64 only */

#define DP_CODE_OFF 65535    /* policy code of the thrust-off control (off_control) */

#define DP_SWEEP_VI           0  /* Eq. (12): min over the tabulated angles        */
#define DP_SWEEP_IMPROVE_FULL 1  /* Eq. (14): full tabulation (+ refinement)       */
#define DP_SWEEP_IMPROVE_WALK 2  /* Eq. (14): walk from the previous optimum
                                    (+ refinement), §3 "Efficient computation of
                                    the minimum"                                   */
#define DP_SWEEP_EVAL         3  /* Eq. (13): one Jacobi sweep at the frozen policy */
#define DP_SWEEP_EVAL_DIAG    4  /* Eq. (13) as a linear system: one Jacobi iteration
                                    with each node's own coefficient solved,
                                    V'_j = V_j + (T_f(V)_j - V_j) / (1 - beta w_jj),
                                    w_jj the node's own weight among the Q1
                                    corners of its foot (same fixed point)     */
#define DP_SWEEP_VI_DIAG      5  /* Eq. (12) with each node's own coefficient solved
                                    inside the minimisation:
                                    V'_j = min_a (c_a + beta R_a) / (1 - beta w_jj^a)
                                    (same fixed point; minimum-time dynamics)   */

/* How policy iteration evaluates a frozen policy (dp_solve_opts.eval_solver). */
#define DP_EVAL_JACOBI 0     /* n_eval Jacobi sweeps (modified policy iteration)   */
#define DP_EVAL_GMRES  1     /* the linear system of Eq. (13) by restarted GMRES,
                                as §3 prescribes after Eq. (14)                    */
#define DP_EVAL_DIAG   2     /* n_eval DP_SWEEP_EVAL_DIAG iterations: the Jacobi
                                method proper on that system (the node's own
                                coefficient solved), same fixed point          */
#define DP_GMRES_MAX_RESTART 64

typedef struct dp_grid dp_grid;

/* Grid, dynamics, target and control-set description (§3, §4). */
typedef struct dp_grid_desc {
    int32_t n[4];          /* nodes per dimension (r, v_r, v_t, m), each in [2, 1024] */
    double  lo[4], hi[4];  /* box, lo < hi; r > 0 and m > 0 on the box for ORBIT     */
    int32_t dynamics;      /* DP_DYN_*                                               */
    double  mu;            /* gravitational parameter (nondimensional 1)             */
    double  accel;         /* thrust acceleration a at unit mass (>= 0)              */
    double  exhaust_c;     /* exhaust speed c (> 0), m' = -a/c                       */
    double  dt;            /* pseudo-time step of the scheme (> 0)                   */
    double  beta;          /* discount exp(-lambda dt), in (0, 1)                    */
    double  penalty_M;     /* I[V] outside the domain; <= 0 means dt / (1 - beta)    */
    double  target_c[4];   /* target: open box |x_d - c_d| < w_d over the d with     */
    double  target_w[4];   /*   w_d > 0; V = 0 there and those nodes are not updated */
    int32_t n_angles;      /* K tabulated angles 2 pi k / K, K in [2, 1024]          */
    int32_t refine;        /* 1: golden-section refinement in improvement sweeps     */
    double  refine_tol;    /* refinement bracket width, rad (> 0)                    */
    int32_t reduced;       /* 1: keep only nodes with energy in [energy_lo, hi]      */
    double  energy_lo, energy_hi; /* specific energy (v_r^2 + v_t^2)/2 - mu/r band   */
    int32_t precision;     /* DP_FP64 or DP_FP32                                     */
    void*   stream;        /* cudaStream_t for all work of this grid (may be NULL)   */
    /* DP_DYN_POLAR only (ignored otherwise): */
    int32_t off_control;   /* 1: thrust off (DP_CODE_OFF) is a control besides the
                              angles; it wins a tie                                  */
    double  cost_alpha, cost_beta, cost_gamma; /* Eq. (11): alpha |u| + beta (a - a_bar)^2
                              + gamma |(e cos w, e sin w) - (e_bar cos w_bar, ...)|^2 */
    double  a_bar, e_bar, omega_bar;           /* target orbit: semi-major axis (length
                              unit of the box), eccentricity, argument of perigee  */
} dp_grid_desc;

/* Solver options. */
typedef struct dp_solve_opts {
    double  tol;           /* stop when an improvement (PI) or VI sweep moves V by
                              less than tol in the sup norm                         */
    int64_t max_sweeps;    /* VI: sweep budget; PI: improvement-sweep budget        */
    int32_t n_eval;        /* PI: evaluation sweeps per improvement (>= 0)          */
    int32_t walk;          /* PI: 1 = local walk from the previous optimum after the
                              first improvement, 0 = full tabulation every time     */
    int32_t warm;          /* 0: start from V = 0 (PI: full tabulation first);
                              1: start from the resident V and policy               */
    int32_t polish;        /* FP32 grids: 1 = finish with FP64 values once FP32
                              stalls; 0 = stay FP32                                 */
    double  switch_tol;    /* FP32 -> FP64 switch when the improvement residual is
                              below this (<= 0: 16 FP32 epsilons of M, automatic);
                              the switch also happens after 3 improvements without
                              a 0.1 % gain over the best FP32 residual when it is
                              below 64 times that tolerance, or after 30 anywhere   */
    int32_t time_kernels;  /* 1: time every sweep with CUDA events (small overhead) */
    double* history;       /* nullable host array: the residual of every stopping
                              test (VI: every sweep; PI: every improvement sweep),
                              in order, up to history_capacity entries          */
    int64_t history_capacity;
    /* Evaluation of the frozen policy in policy iteration (§3 after Eq. (14)):
     * with the control fixed, Eq. (13) is the sparse linear system
     * (I - beta W_f) V = b, W_f holding the Q1 weights of each node's foot.
     * DP_EVAL_GMRES replaces the n_eval Jacobi sweeps by restarted GMRES on it:
     * each cycle starts from the residual T_f(V) - V of the value the
     * improvement sweep produced and adds the minimal-residual correction
     * from an Arnoldi basis of up to gmres_restart vectors. */
    int32_t eval_solver;   /* DP_EVAL_JACOBI (0), DP_EVAL_GMRES or DP_EVAL_DIAG        */
    int32_t gmres_restart; /* Arnoldi steps per cycle, 1..DP_GMRES_MAX_RESTART
                              (0: 30)                                              */
    int32_t gmres_cycles;  /* cycles per evaluation (0: 1); cycles after the first
                              cost one evaluation sweep each for their residual    */
    int32_t gmres_reorth;  /* 1: classical Gram-Schmidt twice (0: once)            */
    double  gmres_rtol;    /* a cycle ends early once the 2-norm residual estimate
                              falls below gmres_rtol times its start (0: 1e-3)     */
    int32_t n_eval_fp64;   /* PI on FP32 grids with polish: evaluation sweeps per
                              improvement once the values are FP64 (>= 0; 0:
                              automatic, max(n_eval, 80) for DP_EVAL_DIAG and
                              max(n_eval, 160) for DP_EVAL_JACOBI, 0 when n_eval
                              is 0).  Batches ignore it and keep n_eval           */
    int32_t eval_levels;   /* PI on FP32 grids (DP_EVAL_JACOBI, DP_EVAL_DIAG):
                              evaluation sweeps run per launch, 1..32 (0:
                              automatic).  Above 1 a launch runs that many
                              consecutive Jacobi sweeps as a wavefront over the
                              nodes, each sweep's chunk starting once the
                              previous sweep has finished every chunk within
                              the frozen feet's reach; the values are the same
                              as one sweep per launch, bit for bit.  Automatic
                              (0): one sweep per launch.  A launch that gives
                              up a bounded wait (2 s) makes the call return
                              DP_ETIMEOUT                                    */
} dp_solve_opts;

/* Test hook for the bounded waits of the multi-level evaluation
 * (eval_levels > 1): a launch whose chunk waits longer than ns nanoseconds for
 * the previous sweep gives up, every block of it returns, and the call
 * returns DP_ETIMEOUT with the value not valid (a later call starts clean).
 * ns >= 0 (0: give up at the first unmet dependency), -1 restores the default
 * of 2 s.  Process-wide. */
int dp_set_wave_wait_limit(int64_t ns);

/* Solver statistics (filled on DP_OK and on DP_ENOCONV). */
typedef struct dp_solve_stats {
    int64_t sweeps_vi;
    int64_t sweeps_improve;       /* storage-precision improvement sweeps            */
    int64_t sweeps_eval;          /* storage-precision evaluation sweeps             */
    int64_t sweeps_improve_fp64;  /* FP64-value improvement sweeps (polish)          */
    int64_t sweeps_eval_fp64;     /* FP64-value evaluation sweeps (polish)           */
    double  residual;             /* last stopping-test sup norm                     */
    int32_t converged;
    double  ms_wall;              /* host wall time of the call                      */
    double  ms_vi, ms_improve, ms_eval, ms_improve_fp64, ms_eval_fp64; /* GPU time by
                                     sweep type when time_kernels = 1               */
    int64_t node_updates;         /* stored non-target nodes x sweeps               */
    int64_t launches;             /* kernels launched by the call                    */
    int64_t history_count;        /* entries written to opts->history                */
    int64_t switch_outer;         /* PI: improvement sweeps before the FP64 switch
                                     (-1: no switch)                                 */
    int64_t gmres_cycles;         /* GMRES: cycles run                               */
    int64_t gmres_matvecs;        /* GMRES: products with I - beta W_f (Arnoldi
                                     steps); their GPU time is in ms_eval /
                                     ms_eval_fp64 when time_kernels = 1             */
} dp_solve_stats;

/* Sizes of a grid. */
typedef struct dp_grid_info {
    int64_t n_box;      /* n0 n1 n2 n3                                             */
    int64_t n_active;   /* stored nodes                                            */
    int64_t n_target;   /* stored nodes inside the target                          */
    double  penalty_M;  /* the M in use                                            */
    int32_t fp64_values;/* 1 when the resident value is held in FP64               */
    int64_t device_bytes;
} dp_grid_info;

/* Validates desc, builds the node set (the energy-band reduction of §3 "Grid
 * and polar coordinates" when desc->reduced), the target set and the angle
 * tables, and allocates double-buffered V (= 0) and the policy (code 0).
 * Errors: DP_EINVAL (bad descriptor; empty node set; reduced grid needs v_t > 0
 * on the box), DP_ENOMEM, DP_ECUDA.  *out is NULL on failure. */
int dp_grid_create(const dp_grid_desc* desc, dp_grid** out);

/* Frees all device memory of the grid (synchronises its stream).  NULL is a
 * no-op. */
int dp_grid_destroy(dp_grid* grid);

int dp_grid_get_info(const dp_grid* grid, dp_grid_info* info);

/* Box index of every stored node, compact order (count == n_active). */
int dp_get_active_index(const dp_grid* grid, int64_t* box_index, int64_t count);

/* Copy V in / out, compact order, count == n_active.  dp_set_value rejects
 * non-finite input (DP_ENONFINITE) and forces target nodes to 0; it loads the
 * storage precision of the grid (FP32 grids round to nearest). */
int dp_set_value(dp_grid* grid, const double* host_V, int64_t count);
int dp_get_value(const dp_grid* grid, double* host_V, int64_t count);
/* The same with FP32 host values: half the bytes over the host link for FP32
 * grids, whose stored values they are exactly (dp_get_value_f32 copies them
 * without conversion; dp_set_value_f32 stores them unchanged).  On FP64
 * grids, and on FP32 grids whose values have moved to FP64 (after a polish),
 * dp_get_value_f32 rounds to nearest and dp_set_value_f32 widens exactly and
 * returns the grid to FP32 values, as dp_set_value does.  Same errors as the
 * FP64 calls. */
int dp_set_value_f32(dp_grid* grid, const float* host_V, int64_t count);
int dp_get_value_f32(const dp_grid* grid, float* host_V, int64_t count);

/* Copy the policy (16-bit angle codes) in / out, compact order. */
int dp_set_policy(dp_grid* grid, const uint16_t* host_codes, int64_t count);
int dp_get_policy(const dp_grid* grid, uint16_t* host_codes, int64_t count);

/* Frozen feet (FP32 grids).  An improvement sweep stores, per node, the cell
 * and fractions of the foot of its new control (the semi-Lagrangian step of
 * §3 after Eq. (10)), and the evaluation sweeps that follow (Eq. (13)) read
 * them instead of repeating the step.  With FP32 values a foot is one 8-byte
 * word (18-bit fractions) or a word pair (24-bit fractions, 12 bytes); with
 * FP64 values always the pair.  DP_SWEEP_EVAL reads either; DP_SWEEP_EVAL_DIAG
 * reads the pair (its step divides by 1 - beta w_jj, which the 18-bit
 * fractions do not resolve where w_jj is near 1) and otherwise recomputes the
 * feet, exactly as for a policy set from the host.
 *   DP_FOOT_AUTO (default): dp_policy_iterate stores the pair for
 *     DP_EVAL_DIAG and 8-byte words otherwise; dp_bellman_sweep stores
 *     8-byte words.
 *   DP_FOOT_WORD8 / DP_FOOT_PAIR: every FP32-value improvement stores that
 *     format.
 * The format changes a result by the fraction quantisation only (at most
 * 3 * 2^-19 of a cell's value spread per evaluation sweep with 8-byte words).
 * Returns DP_EINVAL for another format. */
#define DP_FOOT_AUTO  0
#define DP_FOOT_WORD8 1
#define DP_FOOT_PAIR  2
int dp_set_foot_format(dp_grid* grid, int32_t format);

/* One Jacobi sweep of the scheme on the resident V and policy (mode =
 * DP_SWEEP_*): Eq. (12), (13) or (14).  Improvement modes rewrite the policy;
 * EVAL and EVAL_DIAG read it.  On FP32 grids whose value has moved to FP64 (after a
 * polish) the sweep runs with FP64 values.  *residual (nullable) receives
 * max_j |V'_j - V_j| over the stored nodes, accumulated in FP64. */
int dp_bellman_sweep(dp_grid* grid, int32_t mode, double* residual);

/* Value iteration, §3 Eq. (12): sweeps until the residual < opts->tol or
 * opts->max_sweeps (DP_ENOCONV).  opts->eval_solver = DP_EVAL_DIAG runs
 * DP_SWEEP_VI_DIAG sweeps instead (minimum-time dynamics).  stats nullable. */
int dp_value_iterate(dp_grid* grid, const dp_solve_opts* opts, dp_solve_stats* stats);

/* Modified policy iteration, §3 Eq. (13)-(14): an improvement sweep (full
 * tabulation first, then the local walk, each followed by golden-section
 * refinement when desc.refine) and opts->n_eval Jacobi evaluation sweeps at
 * the frozen policy, repeated until an improvement sweep moves V by less than
 * opts->tol.  FP32 grids with opts->polish switch to FP64 values once the FP32
 * residual stalls and finish there.  With opts->eval_solver = DP_EVAL_GMRES
 * the evaluation is GMRES on the linear system instead of n_eval sweeps (the
 * paper's policy iteration); the host then checks every improvement sweep.
 * stats nullable. */
int dp_policy_iterate(dp_grid* grid, const dp_solve_opts* opts, dp_solve_stats* stats);

/* Policy evaluation, §3 Eq. (13) solved as a linear system: restarted GMRES
 * on (I - beta W_f) V = b at the resident policy, from the resident V, until
 * an evaluation sweep moves V by less than opts->tol (sup norm) or after
 * opts->max_sweeps cycles (DP_ENOCONV).  Each round is one evaluation sweep
 * (V <- T_f(V), whose change is the stopping test) and one GMRES cycle of
 * opts->gmres_restart steps; opts->gmres_cycles is ignored.  FP32 grids build
 * the frozen feet of the policy first when no improvement sweep has stored
 * them.  The basis takes (gmres_restart + 1) x n_active values of the
 * storage precision (FP32 grids: FP32) of device memory, allocated on first
 * use and kept with the grid.  Uses tol, max_sweeps, gmres_*, time_kernels;
 * stats nullable (sweeps_eval / sweeps_eval_fp64, gmres_*, residual). */
int dp_policy_evaluate(dp_grid* grid, const dp_solve_opts* opts, dp_solve_stats* stats);

/* Approximate optimal feedback, §3 Eq. (15), at n arbitrary states
 * (host, n x 4 row-major) with step tau > 0: full tabulation then refinement
 * (when desc.refine) of tau l(y, alpha) + beta^(tau/dt) I[V](y + tau Phi(y, alpha))
 * (l = 1, or Eq. (11) for DP_DYN_POLAR, where the thrust-off control is also
 * compared).  alpha_out (n, rad in [0, 2 pi); NaN = thrust off) required,
 * q_out (n) nullable. */
int dp_feedback_control(const dp_grid* grid, const double* states, int32_t n, double tau,
                        double* alpha_out, double* q_out);

/* Closed loop, §3 "Computation of the approximate optimal solution": per
 * trajectory, the feedback of Eq. (15) with step tau is recomputed every
 * h_rk4 and held over one classical RK4 step of the dynamics, until the state
 * enters the target (t_arrive = end of that step) or t_max (t_arrive = -1).
 * x0 and x_final are n x 4 row-major host arrays. */
/* The same closed loop on a perturbed "real" system (§4 Example 2): the
 * feedback comes from the grid's model, while the RK4 steps add aerodynamic
 * drag with the printed components -drag_c v_rho^2 and -drag_c v_theta^2
 * (drag_c = C_D S rho_D / (2 m) in 1/length unit; DP_DYN_POLAR grids only;
 * drag_c = 0 is dp_simulate_closed_loop). */
int dp_simulate_closed_loop_drag(const dp_grid* grid, const double* x0, int32_t n, double tau, double h_rk4,
                                 double t_max, double drag_c, double* t_arrive, double* x_final);
int dp_simulate_closed_loop(const dp_grid* grid, const double* x0, int32_t n, double tau,
                            double h_rk4, double t_max, double* t_arrive, double* x_final);

/* ---- learned warm start (not in the paper) ----
 *
 * A multilayer perceptron 4 -> 256 -> 256 -> 256 -> 3 (GELU, exact erf form,
 * after each hidden layer; linear output) maps a state, normalised to [-1, 1]^4
 * over the network's input box, to (V / M, cos alpha, sin alpha).  Weights are
 * FP32 master copies; the two 256 x 256 layers run as BF16 x BF16 -> FP32
 * tensor-core GEMMs (tcgen05).  Training minimises the mean squared error over
 * the three outputs with Adam (beta1 0.9, beta2 0.999, eps 1e-8) on every node
 * of a solved grid; the trained network then initialises V and the policy of
 * another grid for policy iteration (dp_solve_opts.warm = 1).  The sweeps still
 * decide the result: the warm start only changes where policy iteration starts.
 *
 * Parameter order of the flat FP32 vector (dp_mlp_param_count() floats):
 * W1 (256 x 4, row = output), b1 (256), W2 (256 x 256), b2, W3 (256 x 256), b3,
 * W4 (3 x 256), b4 (3). */
typedef struct dp_mlp dp_mlp;

typedef struct dp_mlp_train_opts {
    int32_t  epochs;       /* passes over the grid's nodes                          */
    int32_t  batch;        /* samples per step, multiple of 512, <= capacity        */
    double   lr;           /* Adam step size                                        */
    uint64_t seed;         /* permutation seeds (0: 14675)                          */
    double   lr_final;     /* > 0: step size of the last epoch, reached geometrically
                              from lr epoch by epoch; 0: lr throughout           */
} dp_mlp_train_opts;

typedef struct dp_mlp_train_stats {
    int64_t epochs, steps, samples;
    double  first_epoch_loss, last_epoch_loss;   /* mean squared error per output */
    double  ms;                                  /* GPU time of the training       */
    double  flops;                               /* nominal forward + backward FLOPs */
} dp_mlp_train_stats;

int64_t dp_mlp_param_count(void);

/* Creates a network with zeroed parameters (set them with dp_mlp_set_params)
 * for inputs in the box [lo, hi] (4 each), processing up to batch_capacity
 * (multiple of 512) samples per launch on `stream`. */
int dp_mlp_create(const double* lo, const double* hi, int32_t batch_capacity, void* stream, dp_mlp** out);
int dp_mlp_destroy(dp_mlp* mlp);
/* Host copies of the flat FP32 parameter vector (resets Adam's moments). */
int dp_mlp_set_params(dp_mlp* mlp, const float* params, int64_t count);
int dp_mlp_get_params(const dp_mlp* mlp, float* params, int64_t count);
/* Outputs (n x 3: V / M, cos, sin) at n host states (n x 4). */
int dp_mlp_forward(dp_mlp* mlp, const double* states, int32_t n, float* out);
/* Gradient of the mean squared error of one batch (n a multiple of 512, <=
 * capacity) with respect to every parameter, and the loss; no update. */
int dp_mlp_gradients(dp_mlp* mlp, const double* states, const float* targets, int32_t n, float* grads,
                     float* loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step size lr; the step
 * count and moments carry over from earlier steps and dp_mlp_train_grid)
 * with a caller-supplied gradient of count = dp_mlp_param_count() entries,
 * in the flat parameter order of dp_mlp_set_params: for gradients computed
 * elsewhere (dp_mlp_gradients, or another process).  Synchronises the
 * network's stream. */
int dp_mlp_apply_gradients(dp_mlp* mlp, const float* grads, int64_t count, double lr);
/* Test hook for the bounded wait of the tensor-core GEMMs: the number of
 * polls of each GEMM's wait for its MMAs before it gives up (polls >= 0; 0
 * gives up at once), -1 restores the default (2^22).  A GEMM that gives up
 * sets an error flag, still waits (with the default limit) for the MMAs it
 * committed, skips its epilogue, frees its TMEM and returns; the call then
 * returns DP_ETIMEOUT and clears the flag, so the next call runs normally. */
int dp_mlp_set_wait_limit(dp_mlp* mlp, int32_t polls);
/* Trains on every stored node of a grid: targets V / M and the (cos, sin) of
 * the grid's resident value and policy.  stats nullable. */
int dp_mlp_train_grid(dp_mlp* mlp, dp_grid* grid, const dp_mlp_train_opts* opts, dp_mlp_train_stats* stats);
/* Writes V = M clamp(V/M-hat, 0, 1) (0 on target nodes) and the policy code of
 * atan2(sin-hat, cos-hat) at every stored node of a grid, in the grid's
 * storage precision (an FP32 grid that held FP64 values after a polish goes
 * back to FP32 values).  *ms (nullable): GPU time. */
int dp_warm_start(dp_mlp* mlp, dp_grid* grid, double* ms);

/* ---- batched transfers ----
 *
 * Many independent transfers (each its own full-box grid: sizes, thrust,
 * target, box) solved by modified policy iteration (§3, Eq. (13)/(14)) at
 * once.  Every sweep kind is one persistent launch over all live transfers,
 * and the outer steps are replayed from a CUDA graph; the decisions a single
 * grid's dp_policy_iterate takes on the host (stopping test, the confirming
 * full-table improvement after a converged walk, the FP32 -> FP64 switch)
 * are taken per transfer on the device, so each transfer runs the same sweep
 * sequence as dp_policy_iterate on a grid of its own.
 *
 * Device memory per node: 2 x 4 (FP32 V) + 2 x 8 (FP64 V) + 2 (policy) + 12
 * (frozen foot: an 8-byte word in the FP32-value phase of plain evaluation,
 * the word pair otherwise) + 4 (increment sum) = 42 bytes, plus the line
 * tables.
 * Node and value order inside a transfer: box order, as for a grid. */
typedef struct dp_batch dp_batch;

/* Per-transfer results of dp_batch_policy_iterate. */
typedef struct dp_batch_stats {
    int64_t sweeps_improve;       /* FP32 improvement sweeps                          */
    int64_t sweeps_eval;          /* FP32 evaluation sweeps                           */
    int64_t sweeps_improve_fp64;  /* FP64-value improvement sweeps                    */
    int64_t sweeps_eval_fp64;     /* FP32 increment sweeps of the FP64-value phase    */
    double  residual;             /* last improvement residual (sup norm, FP64)      */
    int32_t converged;
    int32_t nonfinite;
    int64_t switch_outer;         /* improvements before the FP64 switch (-1: none)  */
    int64_t nodes;                /* nodes of the transfer                            */
} dp_batch_stats;

/* Builds a batch of `count` (1 .. 65536) transfers from descs[0 .. count-1]:
 * each must be valid for dp_grid_create, full-box (reduced = 0) and FP32, and
 * all must share one dynamics.  V = 0, policy code 0.  GPU work is issued on
 * `stream` (NULL: a stream the batch creates; the legacy default stream cannot
 * be captured into a graph).  Errors: DP_EINVAL (the message names the
 * transfer), DP_ENOMEM, DP_ECUDA. */
int dp_batch_create(const dp_grid_desc* descs, int32_t count, void* stream, dp_batch** out);
int dp_batch_destroy(dp_batch* batch);
/* Sizes and tuning of a batch; every output pointer is nullable.
 * nodes_target: nodes inside the targets (never updated).  item_eval /
 * item_improve: nodes per work item of the evaluation and improvement
 * launches. */
int dp_batch_get_info(const dp_batch* batch, int32_t* count, int64_t* nodes_total, int64_t* nodes_target,
                      int32_t* item_eval, int32_t* item_improve, int64_t* device_bytes);
/* Sets the work-item sizes (multiples of 256 in [256, 2^20]). */
int dp_batch_set_items(dp_batch* batch, int32_t item_eval, int32_t item_improve);
/* Times the candidate work-item sizes (512 .. 32768 nodes) of the evaluation
 * and walk-improvement launches on this batch with CUDA events and keeps the
 * fastest of each (returned through the nullable outputs).  It runs sweeps,
 * so it leaves every transfer at V = 0 and policy code 0: call it before
 * setting a warm start. */
int dp_batch_autotune(dp_batch* batch, int32_t* item_eval, int32_t* item_improve);
/* Modified policy iteration of every transfer with the options of
 * dp_policy_iterate (tol, max_sweeps = improvement budget per transfer,
 * n_eval <= 1024, walk, warm, polish, switch_tol; time_kernels and history are
 * ignored; eval_solver DP_EVAL_JACOBI or DP_EVAL_DIAG).  total (nullable): sums of the sweep counts, node_updates,
 * launches, the largest residual and switch_outer, converged = all converged.
 * per (nullable): count entries.  Returns DP_ENOCONV if some transfer missed
 * the tolerance (statistics valid), DP_ENONFINITE if one produced a non-finite
 * value. */
int dp_batch_policy_iterate(dp_batch* batch, const dp_solve_opts* opts, dp_solve_stats* total,
                            dp_batch_stats* per);
/* One Jacobi sweep of every transfer on its FP32 values (a transfer whose
 * value is held in FP64 after a polished solve is first rounded to FP32):
 * DP_SWEEP_IMPROVE_FULL, DP_SWEEP_IMPROVE_WALK or DP_SWEEP_EVAL (at the
 * resident policy).  residual (nullable): count entries, max |V_out - V_in|
 * per transfer.  ms (nullable): GPU time of the sweep launch. */
int dp_batch_sweep(dp_batch* batch, int32_t mode, double* residual, double* ms);
/* Value and policy of transfer `index` (count = its n0 n1 n2 n3 nodes). */
int dp_batch_set_value(dp_batch* batch, int32_t index, const double* host_V, int64_t count);
int dp_batch_get_value(const dp_batch* batch, int32_t index, double* host_V, int64_t count);
int dp_batch_set_policy(dp_batch* batch, int32_t index, const uint16_t* host_codes, int64_t count);
int dp_batch_get_policy(const dp_batch* batch, int32_t index, uint16_t* host_codes, int64_t count);

/* One Jacobi sweep that allocates nothing (the paper has no counterpart: this
 * call exists for callers that cannot allocate device memory).
 *
 * Who needs it: software that may not call cudaMalloc once it is running --
 * flight or other real-time code that forbids allocation after start-up, or a
 * host whose device memory belongs to another allocator (a framework's
 * caching allocator, a fixed pool that accounts for every byte), where an
 * extra cudaMalloc can fail or fragment that pool.  dp_grid_create allocates,
 * so such callers cannot hold a grid; this call needs none.
 *
 * It runs the same sweep as dp_bellman_sweep (mode = DP_SWEEP_VI ... EVAL) for the
 * full-box grid that desc describes (desc->reduced must be 0), on buffers the
 * caller owns, in desc->stream on the current device:
 *   V_in   device, n0 n1 n2 n3 values in box order, double (DP_FP64) or float
 *          (DP_FP32); target nodes should hold 0
 *   V_out  device, same size and type, distinct from V_in; receives T(V_in)
 *   codes  device, n0 n1 n2 n3 16-bit angle codes: read by EVAL and WALK,
 *          written by the improvement modes; may be NULL for DP_SWEEP_VI
 *   residual  host, nullable: max |V_out - V_in| (FP64)
 * The call synchronises desc->stream before it returns.
 *
 * Scratch: the node-set and angle tables, the residual slot and the control
 * block live in one file-scope __device__ array of 1,127,168 bytes, which every
 * GPU that loads this library holds until the process exits.  That bounds the
 * grid: n0 n1 <= 4096 and n0 n1 n2 <= 262144, else DP_EINVAL with a message.
 * Every call shares the array and leaves its contents behind; the call rebuilds
 * the tables and clears the residual slot and control block itself.  Calls
 * that overlap on the GPU (two streams, two threads) race on the array and give
 * wrong results: issue them one after another.
 *
 * Set-up: make one warm-up call per device at start-up, before the phase in
 * which the caller may not allocate.  With lazy module loading (the CUDA
 * default since 12.2) the library's device code, this array included, is
 * loaded into a context on first use, and that load allocates device memory;
 * after the warm-up call the array is resident until the context ends.  Every
 * call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, a host-side query), so a context re-created after
 * cudaDeviceReset needs one more warm-up call and nothing else.  Apart from
 * that first load the call never calls cudaMalloc, cudaFree or any
 * allocating library routine.
 *
 * Errors: DP_EINVAL (descriptor, mode, NULL or aliased buffers, grid beyond
 * the scratch bound), DP_ECUDA, DP_ENONFINITE (V_out holds a non-finite value). */
int dp_bellman_sweep_noalloc(const dp_grid_desc* desc, int32_t mode, const void* V_in, void* V_out,
                             uint16_t* codes, double* residual);

/* Warm start of grid dst from the solved value and policy of grid src, the
 * same problem at another resolution or box (no network; the plain baseline
 * of the learned warm start): at every stored node of dst, V = the Q1
 * interpolation of src's resident value (dst's M where the node lies outside
 * src's box or its src cell leaves src's node set; 0 on dst's target) and
 * the policy code of the nearest src node (0 where that node is not stored).
 * Written in dst's storage precision; dst then starts with warm = 1.  Both
 * grids must have the same dynamics and live on one device; src's stream is
 * synchronised first.  *ms (nullable): GPU time. */
int dp_warm_start_from_grid(const dp_grid* src, dp_grid* dst, double* ms);

/* Message of the last failed call on this thread ("" if none). */
const char* dp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DP_H */
