/*
 * oca.h -- C-ABI of the GB300-native scale-based collision-avoidance library.
 *
 * Method: "GPU-Accelerated Optimization-Based Collision Avoidance" (Wu, Wang,
 * Zhang, arXiv 2406.07048).  Robot parts and obstacles are H-polyhedra
 * (Sec. III-A); a part i and an obstacle j are collision-free at step t iff
 * the scale LP eqn:scale_opt has alpha* >= 1, which its dual
 * eqn:scale_opt_dual turns into constraints linear in (lambda, mu)
 * (eqn:poly_colli_free_conts).  An MPC problem over these constraints
 * (eqn:MPC_opt_origin) is split by ADMM (Sec. IV-B) into a batch of small
 * per-pair QPs (eqn:const_least_square), a per-scenario trajectory QP, and
 * elementwise dual updates.
 *
 * Conventions for every entry point
 *   - Plain C: no CUDA or torch types.  `stream` is a cudaStream_t passed as
 *     void* (NULL = legacy default stream).  Every call is stream-ordered and
 *     asynchronous unless stated otherwise; argument errors are reported
 *     before anything is launched.
 *   - Device arrays are caller-owned and must stay valid until the work on
 *     `stream` has finished.  Floating arrays all have the scene's dtype
 *     (OCA_F32 = float, OCA_F64 = double).
 *   - Pair-indexed arrays are component-major with the pair index fastest:
 *     element c of pair p is at [c * P + p], P = total pairs of the scene.
 *   - Pairs of scenario s are enumerated
 *       p = pair_begin[s] + (j * n_parts_s + part) * N_s + (t - 1)
 *     (obstacle j slowest, step t = 1..N_s fastest); pair_begin is the CSR of
 *     M_s * n_parts_s * N_s, available from oca_scene_info.
 *   - y = [lambda; mu; gamma] of a pair is stored padded: lambda_k at
 *     component k (k < fr_max), mu_m at fr_max + m (m < fo_max), gamma at
 *     fr_max + fo_max; ny_max = fr_max + fo_max + 1.  Components beyond a
 *     pair's own face counts are neither read nor written.
 *   - Per-element failures (iteration caps, non-finite data) are reported
 *     through status arrays; nothing traps on the device.
 */
#ifndef OCA_H
#define OCA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OCA_OK = 0,
    OCA_ERR_INVALID_ARGUMENT = 1, /* bad pointer, size, dtype or geometry          */
    OCA_ERR_CUDA = 2,             /* a CUDA runtime call failed                    */
    OCA_ERR_NO_MEMORY = 3,        /* device allocation failed (scene creation)     */
    OCA_ERR_UNSUPPORTED = 4,      /* valid request the library does not implement  */
    OCA_ERR_CAPACITY = 5          /* a size exceeds a compiled-in maximum           */
} oca_status;

typedef enum { OCA_F32 = 0, OCA_F64 = 1 } oca_dtype;

typedef enum {
    OCA_MODEL_BICYCLE = 0, /* s = (x, y, theta, v), u = (accel, steer), dim 2          */
    OCA_MODEL_TRAILER = 1, /* s = (x, y, theta, v, psi), u = (accel, steer), dim 2     */
    OCA_MODEL_QUAD = 2     /* s = (p, v, roll, pitch, yaw, body rates), u = 4 rotor
                              thrusts relative to hover, dim 3                        */
} oca_model_kind;

/* per-pair status values (status_out of oca_pair_qp_batch / oca_scale_detect_batch) */
enum {
    OCA_PAIR_OK = 0,
    OCA_PAIR_ITER_CAP = 1,   /* solver hit its iteration cap; result is the last iterate */
    OCA_PAIR_DEGENERATE = 2, /* singular working set; result is the last valid iterate   */
    OCA_PAIR_NONFINITE = 3   /* non-finite input or iterate                               */
};

/* per-scenario status values of oca_admm_solve */
enum {
    OCA_SCEN_CONVERGED = 0, /* both stopping tests of Sec. IV-B met      */
    OCA_SCEN_MAX_ITER = 1,  /* max_iter iterations without meeting them   */
    OCA_SCEN_FAILED = 2,    /* singular or non-finite trajectory QP       */
    OCA_SCEN_ACTIVE = 3     /* internal: still iterating                   */
};

/* Compiled-in maxima (OCA_ERR_CAPACITY beyond them). */
#define OCA_MAX_OBS_FACES 24
#define OCA_MAX_PART_FACES 8
#define OCA_MAX_HORIZON 256

/* ------------------------------------------------------------------------ */
/* Context                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct oca_ctx oca_ctx;

/* Create a context bound to CUDA device `device` (makes it current).
 * Owns nothing per-problem; scenes own their workspaces.
 * Errors: OCA_ERR_INVALID_ARGUMENT (out == NULL, no such device), OCA_ERR_CUDA. */
oca_status oca_create(oca_ctx **out, int device);

/* Destroy a context.  Scenes created from it must be destroyed first. */
void oca_destroy(oca_ctx *ctx);

/* Human-readable name of a status code (static storage). */
const char *oca_status_string(oca_status st);

/* ------------------------------------------------------------------------ */
/* Scene: H-polyhedra of robot parts and obstacles (Sec. III-A, IV-A)       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t dim;     /* 2 or 3                                                    */
    int32_t dtype;   /* oca_dtype of every floating array of this scene          */
    int32_t n_scen;  /* S >= 1 independent scenarios                            */
    int32_t fo_max;  /* row stride (max faces) of the obstacle arrays, <= OCA_MAX_OBS_FACES  */
    int32_t fr_max;  /* row stride of the part arrays, <= OCA_MAX_PART_FACES    */
    /* host metadata, read only during oca_scene_create: */
    const int32_t *obs_begin;  /* [S+1] CSR of obstacles over scenarios         */
    const int32_t *obs_nf;     /* [M_tot] obstacle face counts, 1..fo_max       */
    const int32_t *part_begin; /* [S+1] CSR of robot parts over scenarios       */
    const int32_t *part_nf;    /* [P_tot] part face counts, 1..fr_max           */
    const int32_t *part_link;  /* [P_tot] 0 = vehicle body, 1 = trailer link    */
    const int32_t *horizon;    /* [S] N_s, 1..OCA_MAX_HORIZON                   */
    /* device geometry, caller-owned, must outlive the scene: */
    const void *obs_C;    /* [M_tot][fo_max][dim] outward normals c_m (world)   */
    const void *obs_d;    /* [M_tot][fo_max] offsets d_m:  C y <= d             */
    const void *part_A;   /* [P_tot][fr_max][dim] body-frame normals a_k        */
    const void *part_b;   /* [P_tot][fr_max] offsets b_k > 0 (centre inside)    */
    const void *part_off; /* [P_tot][dim] part centre in its link frame         */
} oca_scene_desc;

typedef struct oca_scene oca_scene;

typedef struct {
    int64_t n_pairs;   /* P = sum_s M_s * n_parts_s * N_s                       */
    int64_t n_states;  /* sum_s (N_s + 1): rows of the state arrays             */
    int64_t n_ctrls;   /* sum_s N_s: rows of the control arrays                 */
    int32_t ny_max;    /* fr_max + fo_max + 1                                   */
    int32_t n_tiles;   /* work tiles of the pair kernels                        */
    const int64_t *pair_begin; /* host [S+1], owned by the scene                */
    const int64_t *state_begin;/* host [S+1]                                     */
    const int64_t *ctrl_begin; /* host [S+1]                                     */
} oca_scene_info;

/* Validate a scene and allocate its device workspace (the only allocating
 * call besides oca_create).  Reads the host metadata and checks, on the
 * device, that part offsets are > 0 and all geometry is finite.
 * Errors: OCA_ERR_INVALID_ARGUMENT, OCA_ERR_CAPACITY, OCA_ERR_NO_MEMORY,
 * OCA_ERR_CUDA.  Synchronous. */
oca_status oca_scene_create(oca_ctx *ctx, const oca_scene_desc *desc, oca_scene **out);
void oca_scene_destroy(oca_scene *scene);
oca_status oca_scene_info_get(const oca_scene *scene, oca_scene_info *info);

/* Work shape of the pair kernels: warps per 32-lane tile (1..16); each warp
 * sweeps every W-th obstacle of the tile's scenario.  oca_scene_create picks
 * about eight obstacles per warp at the median obstacle count;
 * DeviceScene.autotune_warps in the Python binding times the fused pair
 * kernel of short solves for each candidate and sets the fastest.
 * Errors: OCA_ERR_INVALID_ARGUMENT (warps outside 1..16), OCA_ERR_CAPACITY
 * (more warps per tile than the pair kernels are compiled for -- 16 for
 * FP32 2-D scenes, 12 for FP64 2-D, 8 for 3-D -- or their shared memory for
 * that many warps exceeds the device's per-block limit: per warp,
 * (ls + fr_max + fo_max + dim + 2 + nstat) * 32 + 4 nob elements and 16
 * bytes, with ls = 4 (fo_max | 1) in FP32 and 4 fo_max + 2 in FP64,
 * nob = fo_max (nc + 1) rounded up to a multiple of 4, nc = 2 in 2-D and 4
 * in 3-D, nstat = 9 in 2-D and 18 in 3-D). */
oca_status oca_scene_set_warps(oca_scene *scene, int warps);
int oca_scene_get_warps(const oca_scene *scene); /* -1 if scene == NULL */

/* ------------------------------------------------------------------------ */
/* Model and ADMM parameters                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t kind;     /* oca_model_kind; must match the scene's dim           */
    double dt;        /* Euler step of eqn:system_eqn: s+ = s + dt f_c(s,u)   */
    double param[8];  /* bicycle [L]; trailer [L, M_hitch, L2]; quad
                         [m, g, Jx, Jy, Jz, arm, yaw_coeff]                     */
    double Qs[12];    /* diagonal of Q_s (eqn:navigation_cost)                 */
    double Qu[4];     /* diagonal of Q_u                                        */
    double s_lo[12], s_hi[12]; /* state box of eqn:MPC_opt_origin; +-inf (or
                                  magnitude >= 1e30) leaves a component free    */
    double u_lo[4], u_hi[4];   /* control box                                    */
} oca_model;

typedef struct {
    double sigma;     /* ADMM penalty (eqn:ADMM_Lagrangian), paper: 300            */
    double eps_pri;   /* stop when sum(dzeta^2 + |dxi|^2) <= eps_pri (Sec. IV-B)    */
    double eps_dual;  /* and sum(|dlambda|^2 + |dmu|^2) <= eps_dual                  */
    double prox;      /* >= 0; proximal weight 0.5*prox*sum_g |K_g|^2 (y_g - y^k_g)^2 in
                         step 1, each generator's step measured in residual space
                         (0 = the paper's QP as printed)                               */
    int32_t max_iter; /* iteration cap                                                */
    int32_t flags;    /* OCA_ADMM_* bits                                              */
    double rho_box;   /* >= 0; penalty of the box block: the state/control boxes are
                         a bounded copy z of (s, u) with scaled dual w, updated
                         after each trajectory step (z = clip(s + w), w += s - z);
                         its residuals |s - z|^2 and |dz|^2 join r_pri and r_dual  */
    double damp;      /* >= 0; proximal weight 0.5*damp*|(s,u) - (s,u)^k|^2 in step 2 */
} oca_admm_params;

#define OCA_ADMM_RICCATI_F32 1  /* factorise the trajectory QP in FP32 (default FP64) */
#define OCA_ADMM_FIXED_POINT 2  /* differentiate the fixed point (oca_admm_solve_taped,
                                   oca_admm_backward): see below                   */

/* Per-scenario results, all device arrays of length S (float arrays: scene dtype). */
typedef struct {
    int32_t *iters;  /* iterations performed                                    */
    int32_t *status; /* OCA_SCEN_*                                               */
    void *r_pri;     /* primal residual sum of the last iteration                */
    void *r_dual;    /* dual residual sum of the last iteration                  */
    void *cost;      /* F of eqn:navigation_cost at the returned trajectory     */
} oca_admm_report;

/* ------------------------------------------------------------------------ */
/* Hot-path entry points                                                    */
/* ------------------------------------------------------------------------ */

/* Scale-based collision detection, Sec. III-A eqn:scale_opt, per pair:
 *   alpha* = min alpha s.t. A x <= alpha b, C' x <= d'  (body frame of the part,
 *   C' = C R(s_t), d' = d - C rho(s_t)), solved through the dual
 *   eqn:scale_opt_dual; alpha* >= 1 means collision-free.
 * states : [n_states][ns] row-major (s_t of scenario s at row state_begin[s]+t).
 * alpha  : [P] out.  lambda: [fr_max][P] out or NULL.  mu: [fo_max][P] out or NULL.
 * margin : [P] double out or NULL: FP64 weak-duality lower bound
 *          -d'^T mu / (b^T lambda + |A^T lambda + C'^T mu| D_R) on alpha*
 *          (D_R = largest vertex norm of the part), Sec. III-B.
 * verdict: [P] int32 out or NULL: 1 if alpha* >= 1 (free), else 0.
 * status : [P] int32 out or NULL: OCA_PAIR_*. */
oca_status oca_scale_detect_batch(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                                  const void *states, void *alpha, void *lambda, void *mu,
                                  double *margin, int32_t *verdict, int32_t *status, void *stream);

/* FP64 certificate margin of caller-given dual variables, per pair
 * (Sec. III-B, weak duality of eqn:scale_opt / eqn:scale_opt_dual): for any
 * lambda, mu >= 0,
 *   alpha* >= -d'^T mu / (b^T lambda + |A^T lambda + C'^T mu| D_R),
 * D_R the part's largest vertex norm, C' = C R(s_t), d' = d - C rho(s_t).
 * A margin >= 1 certifies the pair collision-free without solving the LP;
 * the final check of an ADMM solve passes its returned y (lambda = y,
 * mu = y + fr_max * P in the padded layout) and states.  The poses are formed
 * in FP64 from the stored states and every sum is FP64, so the bound holds for
 * the geometry as stored.
 * states: [n_states][ns] (scene dtype).  lambda: [fr_max][P], mu: [fo_max][P]
 * (scene dtype; only a pair's own components are read).  margin: [P] double
 * out; -DBL_MAX where a component is negative or non-finite, or the
 * denominator is not positive.
 * Errors: OCA_ERR_INVALID_ARGUMENT (a NULL pointer, a model that does not
 * match the scene), OCA_ERR_CUDA. */
oca_status oca_cert_margin_batch(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                                 const void *states, const void *lambda, const void *mu, double *margin,
                                 void *stream);

/* ADMM step 1 alone, Sec. IV-C eqn:const_least_square, per pair:
 *   min 0.5 |K^T y + bq|^2 + 0.5 prox sum_g |K_g|^2 (y_g - y_in,g)^2
 *   s.t. b_i^T lambda = 1, y = [lambda; mu; gamma] >= 0,
 * with K built at the pose of s_t and bq = [1 + zeta; xi].
 * zeta: [P], xi: [dim][P] in.  y_in: [ny_max][P] in (warm start; also the
 * proximal centre); y_out: [ny_max][P] out (may alias y_in).
 * v_out: [dim+1][P] = K^T y + bq out or NULL.  obj_out: [P] = 0.5|v|^2 or NULL.
 * status_out: [P] int32 OCA_PAIR_* or NULL. */
oca_status oca_pair_qp_batch(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                             const void *states, const void *zeta, const void *xi, double prox,
                             const void *y_in, void *y_out, void *v_out, void *obj_out,
                             int32_t *status_out, void *stream);

/* The same pair QPs as oca_pair_qp_batch by the paper's own route
 * (Sec. IV-C): y_e of the robot face with the largest b eliminated through
 * b^T lambda = 1 (eqn:const_least_square_ineq), the KKT conditions
 * (eqn:kkt_conditions) as the LCP w = M z + q (eqn:linear_complementarity_problem),
 * solved by Lemke's complementary pivoting with one GPU thread per LCP row
 * (one warp per pair).  A comparison kernel for the semismooth Newton /
 * active-set solvers of oca_pair_qp_batch (same arguments and outputs;
 * y_out must not alias y_in).  Requires fr_max + fo_max + 1 <= 32
 * (else OCA_ERR_UNSUPPORTED).  status_out: OCA_PAIR_OK, OCA_PAIR_ITER_CAP
 * (pivot cap), OCA_PAIR_DEGENERATE (ray termination). */
oca_status oca_pair_qp_lemke_batch(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                                   const void *states, const void *zeta, const void *xi, double prox,
                                   const void *y_in, void *y_out, void *v_out, void *obj_out,
                                   int32_t *status_out, void *stream);
/* Whole ADMM solves of every scenario (Sec. IV-B), Gauss-Seidel order:
 * step 1 pair QPs, step 2 one LQ (SQP) step of the trajectory problem with
 * linearised dynamics and Gauss-Newton-linearised pair residuals, solved by
 * a Riccati recursion, step 3 zeta += T, xi += R; per-scenario stopping rule.
 * s_ref: [n_states][ns] in.  s: [n_states][ns] in/out (row t=0 of each
 * scenario is the fixed initial state).  u: [n_ctrls][nu] in/out.
 * y: [ny_max][P] in/out (initial y^0 / result).  zeta: [P], xi: [dim][P] in/out.
 * report: device arrays, out.  Runs to completion on `stream` (the host waits
 * between iteration chunks to test whether every scenario has stopped). */
oca_status oca_admm_solve(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                          const oca_admm_params *params, const void *s_ref, void *s, void *u,
                          void *y, void *zeta, void *xi, const oca_admm_report *report,
                          void *stream);

/* ------------------------------------------------------------------------ */
/* Differentiation: adjoint of the unrolled ADMM                            */
/* ------------------------------------------------------------------------ */
/* The paper solves the MPC problem and stops there; these three calls add a
 * reverse-mode gradient of the solution with respect to the obstacles.
 * A taped solve records every iterate (s^k, u^k, y^k, zeta^k, xi^k, the box
 * block and the Gauss-Newton statistics) so that oca_admm_backward can run
 * the iterations of Sec. IV-B backwards: per pair it differentiates the pair
 * QP through its optimality conditions on the active set (implicit function
 * theorem; prox > 0 makes the QP strictly convex and its solution unique),
 * per scenario it solves the adjoint of each trajectory LQ with the same
 * Riccati factorisation (FP64) and differentiates the linearisation point
 * through the second derivatives of the dynamics and of the part poses.
 * The result is the exact derivative of the map the solve executed (its
 * iteration count held fixed); it is defined where no pair's active set
 * changes, i.e. at strictly complementary pair solutions. */

/* Size in bytes of the tape for this scene, model and iteration cap: the
 * iterates of a solve with max_iter iterations and the backward pass's work
 * area.  About (max_iter + 1) * (ny_max + dim + 1) * n_pairs elements.
 * Errors: OCA_ERR_INVALID_ARGUMENT. */
oca_status oca_admm_tape_bytes(const oca_scene *scene, const oca_model *model, int32_t max_iter, int64_t *bytes);
/* Size in bytes of the one-iterate tape of the fixed-point form
 * (OCA_ADMM_FIXED_POINT): the final iterate and the same work area, about
 * (2 ny_max + 2 dim + 2) * n_pairs elements, independent of max_iter.
 * Errors: OCA_ERR_INVALID_ARGUMENT. */
oca_status oca_admm_fixed_point_tape_bytes(const oca_scene *scene, const oca_model *model, int64_t *bytes);
/* oca_admm_solve that also records its iterates in `tape` (caller-owned
 * device memory, 256-byte aligned, tape_bytes >= oca_admm_tape_bytes(...,
 * params->max_iter); else OCA_ERR_INVALID_ARGUMENT / OCA_ERR_CAPACITY).
 * Same results as oca_admm_solve; runs without iteration graphs.
 * With OCA_ADMM_FIXED_POINT in params->flags it records only the returned
 * iterate (tape_bytes >= oca_admm_fixed_point_tape_bytes) and runs as
 * oca_admm_solve does, iteration graphs included. */
oca_status oca_admm_solve_taped(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                                const oca_admm_params *params, const void *s_ref, void *s, void *u, void *y,
                                void *zeta, void *xi, const oca_admm_report *report, void *tape, int64_t tape_bytes,
                                void *stream);
/* Gradient of L = sum_s grad_cost[s] * F_s + sum_p grad_alpha[p] * alpha*_p,
 * F_s the trajectory cost of eqn:navigation_cost returned by the taped
 * solve for scenario s and alpha*_p the scale of eqn:scale_opt of pair p at
 * the returned trajectory, with respect to the obstacle offsets d, the
 * obstacle translations and the initial states.  alpha* enters through the
 * LP envelope theorem (Sec. III-B): its derivative is -mu_m with respect to
 * d'_m and mu_m x_i with respect to C'_mi, at the optimal certificate mu and
 * primal point x; valid where the LP's optimal basis is unique.  Arguments: the scene, model, params and
 * s_ref of the taped solve; tape, tape_bytes as given to it (its work area
 * is overwritten); iters = report.iters of that solve (device, [S]);
 * grad_cost [S] (device, scene dtype); grad_alpha [P] or NULL.
 * Outputs (device, scene dtype, each may be NULL but not all three):
 *   grad_obs_offset [M_tot][fo_max]  dL/dd_m (pad faces 0);
 *   grad_obs_center [M_tot][dim]     dL/ddelta for a translation delta of the
 *                                    obstacle (offsets d_m + c_m . delta);
 *   grad_state0     [S][ns]          dL/ds_0.
 * prox must be > 0 (else OCA_ERR_UNSUPPORTED).  Scenarios whose solve
 * FAILED, or that ran no iteration, get meaningless gradients.
 *
 * Fixed-point form (OCA_ADMM_FIXED_POINT in params->flags, the tape of a
 * fixed-point taped solve): the derivative of the solve's limit xs = T(xs)
 * instead of the executed iterations, by the implicit function theorem,
 * d xs / d theta = (I - dT/dx)^-1 dT/dtheta, its transpose applied as the
 * Neumann series sum_i (dT/dx^T)^i: params->max_iter reverse steps of the
 * same adjoint iteration, every one at the taped iterate.  Valid for
 * scenarios that converged; the series converges at the rate the forward
 * iteration did, so max_iter should be of the order of the iterations the
 * forward took to converge tightly.  Memory: one iterate, whatever the count. */
oca_status oca_admm_backward(oca_ctx *ctx, const oca_scene *scene, const oca_model *model,
                             const oca_admm_params *params, const void *s_ref, void *tape, int64_t tape_bytes,
                             const int32_t *iters, const void *grad_cost, const void *grad_alpha,
                             void *grad_obs_offset, void *grad_obs_center, void *grad_state0, void *stream);
/* ------------------------------------------------------------------------ */
/* Closed-loop receding-horizon control                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t n_steps;   /* control steps C >= 1                                        */
    int32_t reserved;  /* 0                                                           */
    double window[3];  /* sensing box half-widths around the position (Sec. V-B senses
                          20 x 20 x 6 m: 10, 10, 3); <= 0 leaves an axis unlimited      */
} oca_mpc_params;
/* The paper's closed loop (Sec. V-B), every scenario at once.  Per control
 * step c = 0..C-1:
 *   1. the horizon window: s_ref rows t = 0..N <- ref[c + t] (clamped to the
 *      last row); for c > 0 the warm start is shifted one step (s_t <- s_{t+1},
 *      u_t <- u_{t+1}, and y, zeta, xi of pair (j, part, t) <- (j, part, t+1));
 *      s_0 <- the true state;
 *   2. the sensing cull: obstacles whose centre lies outside the box
 *      |centre - position| <= window take no part in this step's solve (their
 *      pairs keep y, zeta, xi);
 *   3. the ADMM of oca_admm_solve with `params`;
 *   4. the plant: x <- x + dt f_c(x, u_0), u_0 the plan's first control clipped
 *      to the control box (0 where non-finite);
 *   5. collision of the true state with every obstacle (alpha* < 1 of the
 *      scale LP, sensed or not).
 * ref        [S][T_ref][ns] device: the reference state of every control step.
 * obs_center [M_tot][dim] device: the point the sensing window tests.
 * x          [S][ns] device in/out: the true state.
 * s_ref, s, u, y, zeta, xi: as for oca_admm_solve (in: the first warm start,
 *            out: the last window and plan).
 * x_hist [S][C+1][ns], u_hist [S][C][nu] (scene dtype), iters_hist [S][C],
 * collided [S] (int32; the first control step whose true state collides, -1
 * if none) out.
 * Synchronous with the host between control steps (the ADMM's chunk checks).
 * Errors: OCA_ERR_INVALID_ARGUMENT, OCA_ERR_CUDA. */
oca_status oca_mpc_run(oca_ctx *ctx, const oca_scene *scene, const oca_model *model, const oca_admm_params *params,
                       const oca_mpc_params *mpc, const void *ref, int32_t T_ref, const void *obs_center, void *x,
                       void *s_ref, void *s, void *u, void *y, void *zeta, void *xi, void *x_hist, void *u_hist,
                       int32_t *iters_hist, int32_t *collided, void *stream);
/* ------------------------------------------------------------------------ */
/* Collision detection without allocation                                   */
/* ------------------------------------------------------------------------ */

/* The same results as oca_scale_detect_batch (alpha*, optional lambda*, mu*,
 * verdict, status; no certificate margin) for a scene of exactly one
 * scenario, without creating an oca_scene and without allocating anything,
 * on the device or the host.  For callers that cannot allocate: a real-time
 * control loop that must stay out of the CUDA allocator (which can block or
 * synchronise), or code under a host that forbids heap use.  The paper has
 * no counterpart of this entry point.
 * desc: as for oca_scene_create with n_scen == 1 (host metadata, device
 * geometry); the face counts and part links are copied into a file-scope
 * device scratch array of 1 MiB that also holds the poses, so
 * 4 * (M + 2 * n_parts) (rounded up to 256) + (dim + dim^2) * n_parts * N *
 * sizeof(element) must not exceed 1 MiB, else OCA_ERR_CAPACITY; other argument
 * errors give OCA_ERR_INVALID_ARGUMENT before any work is queued.
 * The host metadata (obs_nf, part_nf, part_link) is copied on `stream` with
 * cudaMemcpyAsync: from page-locked (pinned) memory the copy stays
 * asynchronous, and the arrays must then stay valid until it has run on the
 * stream; from pageable memory the driver stages the data before the call
 * returns, which can block the calling thread.
 * Every GPU that loads the library holds the 1 MiB until the process exits.
 * The first call on a device looks up the array's device address (make that
 * call before any stream capture); all calls on a device share the array, so
 * calls whose work overlaps on the GPU race. */
oca_status oca_scale_detect_noalloc(const oca_scene_desc *desc, const oca_model *model, const void *states,
                                    void *alpha, void *lambda, void *mu, int32_t *verdict, int32_t *status,
                                    void *stream);

/* ------------------------------------------------------------------------ */
/* The step-2 LQ problem, batched, sequential or parallel in time            */
/* ------------------------------------------------------------------------ */
/* Step 2 of the ADMM (Sec. IV-B eqn:ADMM_state_updates, solved as one QP per
 * iteration) is an LQ problem of the form
 *   min  sum_{t=0..N} 0.5 s_t^T Q_t s_t + q_t^T s_t + sum_{t<N} 0.5 u_t^T R_t u_t + r_t^T u_t
 *   s.t. s_{t+1} = A_t s_t + B_t u_t + c_t,  s_0 given,
 * with Q_t positive semidefinite and R_t positive definite.  oca_lq_solve
 * solves a batch of S independent such problems (same ns, nu, N) in FP64:
 *   OCA_LQ_SEQUENTIAL  the backward Riccati recursion over t, one CTA per problem;
 *   OCA_LQ_SCAN        parallel in time: the stage relations of the optimality
 *                      conditions (state and costate, s_{t+1} = A s + b - C lam_{t+1},
 *                      lam_t = J s - eta + A^T lam_{t+1}) composed associatively in
 *                      ceil(log2(N + 1)) rounds, one CTA per composition, giving
 *                      every stage's value function at once; it trades about
 *                      log2(N) times the recursion's arithmetic for a dependent
 *                      chain of log2(N) rounds instead of N steps (for long
 *                      horizons with few problems).
 * Both then form the gains K_t, k_t of every stage in parallel and roll the
 * closed loop out from s_0 (one warp per problem).
 * Layouts (device, row-major, problem-major):
 *   A [S][N][ns][ns], B [S][N][ns][nu], c [S][N][ns], Q [S][N+1][ns][ns],
 *   q [S][N+1][ns], R [S][N][nu][nu], r [S][N][nu], s0 [S][ns];
 *   out: s [S][N+1][ns], u [S][N][nu], P [S][N+1][ns][ns] and p [S][N+1][ns]
 *   (value functions V_t(s) = 0.5 s^T P_t s + p_t^T s + const, each may be NULL),
 *   status [S] int32 (0 solved; 1 a singular R_t, R_t + B^T P B or elimination
 *   pivot, or a non-finite value: that problem's outputs are meaningless).
 * work: caller-owned device workspace, 256-byte aligned, at least
 * oca_lq_workspace_bytes(...) bytes; nothing is allocated.  ns <= 12, nu <= 4,
 * N <= OCA_MAX_LQ_HORIZON, S <= 65535 (else OCA_ERR_CAPACITY).
 * Errors: OCA_ERR_INVALID_ARGUMENT, OCA_ERR_CAPACITY, OCA_ERR_CUDA. */
#define OCA_LQ_SEQUENTIAL 0
#define OCA_LQ_SCAN 1
#define OCA_MAX_LQ_HORIZON 65535
oca_status oca_lq_workspace_bytes(int32_t ns, int32_t nu, int32_t N, int32_t n_problems, int64_t *bytes);
oca_status oca_lq_solve(oca_ctx *ctx, int32_t method, int32_t ns, int32_t nu, int32_t N, int32_t n_problems,
                        const double *A, const double *B, const double *c, const double *Q, const double *q,
                        const double *R, const double *r, const double *s0, double *s, double *u, double *P,
                        double *p, int32_t *status, void *work, int64_t work_bytes, void *stream);

/* ------------------------------------------------------------------------ */
/* Kernel timing                                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double pair_ms;        /* summed device time of the fused pair kernel launches */
    double traj_ms;        /* summed device time of the trajectory (Riccati) launches */
    int64_t pair_launches; /* launches that did work (iteration index <= max_iter) */
    int64_t traj_launches;
} oca_profile_stats;

/* Start (enable != 0) or stop timing oca_admm_solve's kernels on this
 * context with CUDA events recorded around each launch (also inside the
 * captured iteration graphs); starting resets the counters.  The events are
 * read when the host tests for convergence between iteration chunks, so the
 * timed solve runs in its normal configuration.  Errors: OCA_ERR_CUDA. */
oca_status oca_profile_enable(oca_ctx *ctx, int enable);
oca_status oca_profile_read(const oca_ctx *ctx, oca_profile_stats *out);

/* FP64 FMA throughput of `device` in GFLOP/s (*gflops), measured by a
 * synthetic kernel: 2,048 threads per SM, each advancing 8 independent FMA
 * chains for 8,192 steps; the best of three timed launches after one warm-up
 * (about 0.1 s in all).  The denominator of the trajectory kernel's FP64
 * roofline.  Synchronous; allocates 8 bytes and two events and frees them;
 * the calling thread's current device is restored.
 * Errors: OCA_ERR_INVALID_ARGUMENT (gflops == NULL, no such device),
 * OCA_ERR_CUDA. */
oca_status oca_fp64_peak(int device, double *gflops);

#ifdef __cplusplus
}
#endif
#endif /* OCA_H */
