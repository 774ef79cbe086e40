/*
 * dmx.h -- C ABI of the GB300-native batched soft-contact rollout library.
 *
 * The library integrates many independent environments of a rigid-body
 * system with MuJoCo-style soft contacts (arXiv 2506.14186, "Differentiable
 * Simulation of Hard Contacts with Soft Gradients for Learning and Control"):
 *
 *   state x = [q, v], q in R^nq (free joints carry a unit quaternion), v in R^nv
 *   (Sec. 2: x_{k+1} = step(x_k, a_k, p), loss L(x~_{k+1}, x_k, a_k, p))
 *   v' = M^-1 (tau - c + J^T f)                              (Sec. 2, Eq. EOM)
 *   f from the relaxed Gauss principle with reference acceleration
 *   a_ref = -b (J v) - k d(r) r and regulariser R = A_hat (1 - d) / d
 *                                           (Sec. 2.1, Eq. primal-problem)
 *   integrated by adaptive Dormand-Prince 5(4) with a PID step-size
 *   controller per environment                   (Sec. 3.1, App. B, App. C.2)
 *   differentiated by the discrete adjoint over the accepted steps
 *   (discretize-then-optimize, App. C.2), optionally with the straight-through
 *   contacts-from-distance (CFD) right-hand side in the backward pass (Sec. 4).
 *
 * Conventions
 *   - Batched arrays are structure-of-arrays: element (i, e) of an [n][B]
 *     array is at i * B + e (environment index fastest).
 *   - Unless a call says otherwise, array pointers are DEVICE pointers owned
 *     by the caller; the library never frees caller memory.  Work is ordered
 *     on the CUDA stream passed as `stream` (NULL = legacy default stream).
 *   - Models, tapes and servers are owned by the library (create/destroy).
 *   - Every call returns a dmx_status; on failure dmx_last_error() returns a
 *     thread-local message.  No exception crosses the ABI.
 *   - Per-environment failures do not fail a call: they are reported in the
 *     caller's status[B] array (DMX_ENV_*), and that environment's outputs
 *     hold its last accepted state.
 */
#ifndef DMX_H
#define DMX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DMX_OK = 0,
  DMX_ERR_INVALID = 1,        /* bad argument or model description */
  DMX_ERR_OOM = 2,            /* device or host allocation failed */
  DMX_ERR_CUDA = 3,           /* a CUDA call failed */
  DMX_NOT_READY = 4,          /* dmx_poll: request still running */
  DMX_ERR_TIMEOUT = 5,        /* a bounded wait ran out */
  DMX_ERR_UNIMPLEMENTED = 6
} dmx_status;

/* per-environment status codes (status[B]) */
enum {
  DMX_ENV_OK = 0,
  DMX_ENV_MAX_STEPS = 1,      /* step attempts reached max_steps before T (App. D budget) */
  DMX_ENV_H_UNDERFLOW = 2,    /* step size fell below 1e-12 s */
  DMX_ENV_NONFINITE = 3,      /* non-finite initial state */
  DMX_ENV_SOLVER_NOCONV = 4,  /* constraint Newton solve exceeded 50 iterations */
  DMX_ENV_ROW_OVERFLOW = 5    /* more included constraint rows than the workspace holds (row capacity =
                                 min(rows of all contact slots, 64), dmx_model_info) */
};

enum { DMX_JNT_FREE = 0, DMX_JNT_HINGE = 1 };
enum { DMX_GEOM_SPHERE = 0, DMX_GEOM_CAPSULE = 1, DMX_GEOM_BOX = 2 };
enum { DMX_ACT_MOTOR = 0, DMX_ACT_POSITION = 1 };
enum { DMX_FORM_PERSISTENT = 0, DMX_FORM_STEP = 1, DMX_FORM_STEP_GRAPH = 2 };
/* integration schemes (dmx_rollout_args.method): adaptive Dormand-Prince 5(4)
 * (App. C.2) and Tsitouras 5(4) (the paper's default solver, Fig. 12), both with
 * the PID step-size controller of App. B; semi-implicit Euler with the fixed
 * step h0 (the MuJoCo XLA integrator the paper compares against, Sec. 3.1:
 * v_{n+1} = v_n + h F(q_n, v_n), q_{n+1} = q_n (+) h v_{n+1}; rtol/atol unused). */
enum { DMX_METHOD_DOPRI5 = 0, DMX_METHOD_TSIT5 = 1, DMX_METHOD_EULER = 2 };
/* adjoint kernels of dmx_rollout_grad (dmx_set_adjoint) */
enum { DMX_ADJ_REVERSE = 0, DMX_ADJ_TANGENT = 1, DMX_ADJ_RECOMPUTE = 2 };

/* ------------------------------------------------------------------ model */
/* Body of a kinematic tree.  parent < own index (-1 = world).  A free joint
 * (7 qpos: position, quaternion w,x,y,z; 6 dof: linear velocity in world
 * axes, angular velocity in body axes) is allowed on children of the world
 * only; a hinge rotates about `axis` (body frame) through the body origin. */
typedef struct {
  int32_t parent, joint;
  double pos[3], quat[4];     /* body frame in the parent frame at q = 0 */
  double axis[3];             /* hinge axis, body frame */
  double mass, com[3];        /* COM in the body frame */
  double inertia[3];          /* principal moments about the COM, body axes */
  double damping;             /* joint damping (generalised force -damping * v) */
} dmx_body_desc;

/* Collision geometry fixed to a body.  size: sphere {r}, capsule {r, half
 * length along local x}, box {half extents}. */
typedef struct {
  int32_t type, body;
  double pos[3], quat[4], size[3];
} dmx_geom_desc;

/* Contact pair: geom1 against the ground plane z = 0 (geom2 = -1: sphere 1
 * contact, capsule 2 end-sphere contacts, box 8 vertex contacts), capsule
 * geom1 against box geom2, or a sphere / capsule against a sphere / capsule
 * of another body (closest points of the two segments, one contact; the
 * ball-ball contact of the billiard, Sec. 4).  condim 1 = frictionless normal
 * row, condim 3 = pyramidal cone with 4 edge rows n +- mu t1, n +- mu t2. */
typedef struct {
  int32_t geom1, geom2, condim;
  double mu;
} dmx_pair_desc;

/* Actuator on a hinge body: motor tau += gear * u; position servo
 * tau += kp (u - q) - kd v. */
typedef struct {
  int32_t type, body;
  double gear, kp, kd;
} dmx_actuator_desc;

/* Whole model (Sec. 2.1 parameters: solref = (t_c, phi_d), solimp =
 * (d_o, d_w, width, midpoint, power); Sec. 4 solimp-CFD = (d_c, d_0, w_c,
 * m_c, p_c) and the width of the softplus replacing the ReLU in a_ref). */
typedef struct {
  int32_t nbody, ngeom, npair, nact;
  const dmx_body_desc* body;
  const dmx_geom_desc* geom;
  const dmx_pair_desc* pair;
  const dmx_actuator_desc* act;
  double gravity[3];
  double solref[2];
  double solimp[5];
  double solimp_cfd[5];
  double softplus;
  const double* qpos0;        /* [nq] reference pose for A_hat (host pointer) */
} dmx_model_desc;

typedef struct dmx_model dmx_model;
typedef struct dmx_tape dmx_tape;
typedef struct dmx_server dmx_server;

/* Validates the description (host memory, copied) and uploads the compiled
 * model to the current CUDA device.  Errors: DMX_ERR_INVALID (unsupported
 * joint/pair, sizes over the compiled limits), DMX_ERR_CUDA, DMX_ERR_OOM. */
dmx_status dmx_create_model(const dmx_model_desc* desc, dmx_model** out);
void dmx_destroy_model(dmx_model* m);
/* nq, nv, nu of the model; any pointer may be NULL. */
dmx_status dmx_model_dims(const dmx_model* m, int32_t* nq, int32_t* nv, int32_t* nu);

/* ------------------------------------------------------------------ rollout */
typedef struct {
  int32_t B;                  /* environments, >= 0 (0 = no work) */
  const double* x0;           /* [nx][B] initial states (nx = nq + nv) */
  const double* ctrl;         /* [NI][nu][B] piecewise-constant controls, NULL iff nu == 0 */
  const double* T;            /* [B] horizons (s), > 0 */
  int32_t NI;                 /* control intervals over [0, T], >= 1 */
  double rtol, atol;          /* error-norm tolerances: rtol >= 0, atol > 0 */
  double h0;                  /* first trial step (s), > 0 */
  int32_t max_steps;          /* step-attempt budget per environment, >= 1 */
  int32_t K;                  /* checkpoint interval (accepted steps) of the tape, >= 1 */
  int32_t form;               /* DMX_FORM_*: persistent refill kernel, or one launch per step attempt
                                 (plain stream launches / CUDA-graph replay) */
  int32_t lanes;              /* lanes per environment (1,2,4,8,16,32), 0 = autotuned */
  int32_t host;               /* 1: x0, ctrl, T and all outputs are HOST pointers; the call stages
                                 them through library device memory and returns after the copies */
  double* xT;                 /* out [nx][B] final states */
  double* xb;                 /* out [NI+1][nx][B] states at the interval boundaries, or NULL */
  int32_t* nsteps;            /* out [B] accepted steps, or NULL */
  int32_t* nrej;              /* out [B] rejected attempts, or NULL */
  int32_t* status;            /* out [B] DMX_ENV_* codes, or NULL */
  dmx_tape** tape;            /* out: tape for dmx_rollout_grad (checkpoints every K accepted
                                 steps + accepted step sizes), or NULL for forward only */
  int32_t method;             /* DMX_METHOD_*: integration scheme (0 = adaptive Dormand-Prince 5(4)) */
} dmx_rollout_args;

/* Batched adaptive rollout x0 -> x(T) (Sec. 3.1; one independent step-size
 * sequence per environment, Fig. 14).  Errors: DMX_ERR_INVALID for bad sizes or
 * NULL required pointers, DMX_ERR_OOM when the tape does not fit, DMX_ERR_CUDA. */
dmx_status dmx_rollout(dmx_model* m, const dmx_rollout_args* a, void* stream);

/* Discrete adjoint of the taped rollout (App. C.2, discretize-then-optimize),
 * accepted step sizes held constant, for the loss gradient cotangents
 * xT_bar [nx][B] and xb_bar [NI+1][nx][B] (or NULL).  Writes x0_bar [nx][B]
 * and ctrl_bar [NI][nu][B] (NULL iff nu == 0).  cfd = 1 applies the
 * straight-through estimator of Sec. 4: stage derivatives of the CFD
 * right-hand side evaluated on the stored (CFD-free) trajectory.  Device
 * pointers, ordered on `stream`.  The tape stays valid (may be reused). */
dmx_status dmx_rollout_grad(dmx_model* m, dmx_tape* tape, int32_t cfd, const double* xT_bar,
                            const double* xb_bar, double* x0_bar, double* ctrl_bar, void* stream);
/* Model parameters of the gradient below (the parameters tuned by the
 * system identification of Sec. 5.1 / App. E.2): np = 6 + npair + nbody +
 * nbox, values (host, may be NULL) = t_c, phi_d (solref), d_o, d_w, width,
 * midpoint (solimp), the friction coefficient mu of every pair, the mass of
 * every body (its rotational inertia scaled in proportion: equal density,
 * fixed shape), then the side length of every box geom in geom order (2 x
 * its x half size; the half sizes scale together, and the inertia of a body
 * whose only geom is the box scales with the square, mass fixed). */
dmx_status dmx_model_params(const dmx_model* m, int32_t* np, double* values);
/* dmx_rollout_grad plus the gradient of the same loss with respect to the
 * model parameters (p of the problem statement in Sec. 2, differentiated
 * through the discrete adjoint with the accepted step sizes held constant;
 * A_hat, the model constant computed at qpos0 at creation, carries its
 * derivative with respect to the masses and box sides).  p_bar [np][B] receives
 * it per environment; p_bar_sum [np] (may be NULL) the sum over the
 * environments (a fixed-order reduction: the batch's gradient when every
 * environment shares the model).  Computed by the forward-mode adjoint kernel
 * (one derivative direction per lane: the states, controls and parameters),
 * whatever dmx_set_adjoint selects.  Device pointers, ordered on `stream`. */
dmx_status dmx_rollout_grad_params(dmx_model* m, dmx_tape* tape, int32_t cfd, const double* xT_bar,
                                   const double* xb_bar, double* x0_bar, double* ctrl_bar, double* p_bar,
                                   double* p_bar_sum, void* stream);
/* Optimize-then-discretize gradient (App. C.2, Eq. adjoint-equations:
 * BacksolveAdjoint; with cfd = 1 the straight-through variant of App. C.4).
 * The continuous adjoint a_x' = -a_x^T df/dx, a_u' = -a_x^T df/du of
 * x' = f(x, u) = (G(q) v, F(q, v, u)) is integrated backward from x(T)
 * together with the state itself, with its own adaptive steps (the scheme
 * `method` and the PID controller of the forward pass, error norm over the
 * state's tangent components and every adjoint component, tolerances
 * rtol / atol, first trial step h0), so it needs only the final states and
 * no tape (constant memory).  The gradient is that of the continuous map up
 * to the backward solve's tolerance, not of the discretisation (contrast
 * dmx_rollout_grad).  Backward integration of dissipative contacts runs them
 * anti-damped: a tolerance too tight for that may end an environment with
 * DMX_ENV_H_UNDERFLOW in status. */
typedef struct {
  int32_t B, NI;
  const double* xT;           /* [nx][B] final states of the forward rollout */
  const double* ctrl;         /* [NI][nu][B] controls, NULL iff nu == 0 */
  const double* T;            /* [B] horizons */
  double rtol, atol, h0;      /* backward error control (rtol >= 0, atol > 0, h0 > 0) */
  int32_t max_steps;          /* backward step-attempt budget per environment */
  int32_t method;             /* DMX_METHOD_* of the backward solve */
  int32_t cfd;                /* 1: VJPs of F~ (straight-through) */
  const double* xT_bar;       /* [nx][B] dL/dx(T) */
  const double* xb_bar;       /* [NI+1][nx][B] cotangents of the interval-boundary states, or NULL */
  double* x0_bar;             /* out [nx][B] a_x(0) */
  double* ctrl_bar;           /* out [NI][nu][B], NULL iff nu == 0 */
  int32_t* steps;             /* out [B] accepted backward steps, or NULL */
  int32_t* status;            /* out [B] DMX_ENV_* of the backward solve, or NULL */
} dmx_otd_args;
dmx_status dmx_rollout_grad_otd(dmx_model* m, const dmx_otd_args* a, void* stream);
/* Kernel that dmx_rollout_grad runs for this model (both compute the same
 * derivative; results agree to rounding):
 *   DMX_ADJ_REVERSE (default): reverse mode, a group of lanes per environment
 *     (lanes from dmx_set_lanes(m, B, 2, G), G in {2, 4, 8, 16, 32}, else a
 *     default that fills the SMs); per accepted step it transposes the
 *     Dormand-Prince stages with one right-hand-side VJP per stage.  With
 *     cfd = 0 the workspace of every stage's right-hand side is kept in
 *     library device memory while a segment between two checkpoints is
 *     recomputed (K steps x 6 stages per resident environment, used when it
 *     fits 1/8 of the free device memory and 8 GiB), so each stage is
 *     evaluated once; otherwise as DMX_ADJ_RECOMPUTE.  An environment whose
 *     right-hand side overflowed the row workspace during the adjoint gets
 *     NaN in x0_bar.
 *   DMX_ADJ_RECOMPUTE: the same reverse mode, evaluating each stage's
 *     right-hand side again during the reverse sweep (no stage snapshots).
 *   DMX_ADJ_TANGENT: forward-mode derivative scalars, one warp per
 *     environment and one input direction per lane (the Jacobian of every
 *     step, column by column); kept as an independent check.
 * DMX_ERR_INVALID for another mode. */
dmx_status dmx_set_adjoint(dmx_model* m, int32_t mode);
void dmx_tape_free(dmx_tape* t);
/* Copies a tape into caller DEVICE buffers (any may be NULL), on `stream`:
 * hlog [max_steps][B] accepted step sizes (entries past nsteps[e] undefined),
 * nsteps [B] accepted-step counts, ckpt [ncheck][nx+1][B] the state and time
 * after every K accepted steps (checkpoint c holds step c*K; c = 0 is x0).
 * dims[6] (host, may be NULL) receives B, NI, max_steps, K, ncheck, nx.  The
 * step sizes let a reference integrator replay the exact step sequence. */
dmx_status dmx_tape_read(const dmx_tape* t, double* hlog, int32_t* nsteps, double* ckpt, int32_t* dims,
                         void* stream);

/* Lanes per environment used for (model, B, forward/gradient) when
 * dmx_rollout_args.lanes == 0: the value recorded by dmx_set_lanes (the
 * autotuner's choice), else a default that gives every SM sub-partition a
 * warp of FP64 work.  `stream` is unused (may be NULL). */
dmx_status dmx_autotune(dmx_model* m, int32_t B, int32_t grad, int32_t* lanes, void* stream);
/* Records the lanes per environment for (model, B, kind): kind 0 = forward
 * rollout, 1 = taped rollout, 2 = reverse-mode adjoint kernel; lanes in
 * {1, 2, 4, 8, 16, 32} (kind 2: {2, ..., 32}).  DMX_ERR_INVALID otherwise. */
dmx_status dmx_set_lanes(dmx_model* m, int32_t B, int32_t grad, int32_t lanes);
/* Model facts for tests and tools: invw[nbody] (host, may be NULL) receives the
 * translational inverse weight of every body at qpos0 (the A_hat of Sec. 2.1,
 * model constant); info[8] (host, may be NULL) receives nslot, nrowid,
 * row capacity of the forward right-hand side (the CFD right-hand side holds
 * every row id up to 128), workspace doubles, workspace ints, nbody. */
dmx_status dmx_model_info(const dmx_model* m, double* invw, int32_t* info);

/* ------------------------------------------------------------------ serving */
typedef struct {
  int64_t device_bytes;       /* admission budget for request state (tapes, staging) */
  int32_t max_inflight;       /* concurrent requests on the device */
  int32_t nstreams;           /* CUDA streams the server overlaps requests on */
  int64_t host_stage_bytes;   /* page-locked host staging, split into max_inflight equal blocks (one per
                                 in-flight request); 0 = 32 MiB per in-flight request */
} dmx_server_cfg;

/* A request owns its host buffers until dmx_poll reports it done.  Host
 * pointers, pageable or pinned; layouts as in dmx_rollout_args.  The server
 * copies the inputs into its own page-locked block when it admits the
 * request and the outputs out of it when the device work has finished, so
 * no copy of one request waits for the device work of another. */
typedef struct {
  dmx_model* model;
  int32_t B, NI, max_steps, K;
  double rtol, atol, h0;
  const double* x0;           /* [nx][B] */
  const double* ctrl;         /* [NI][nu][B] or NULL */
  const double* T;            /* [B] */
  int32_t grad;               /* 1: also run the adjoint with xT_bar */
  int32_t cfd;
  const double* xT_bar;       /* [nx][B] when grad */
  double* xT;                 /* out [nx][B] */
  double* x0_bar;             /* out [nx][B] when grad */
  double* ctrl_bar;           /* out [NI][nu][B] when grad and nu > 0 */
  int32_t* status;            /* out [B] or NULL */
} dmx_request;

/* Continuous batching (served MPC requests): dmx_submit queues a request and
 * returns at once; a worker thread admits queued requests in arrival order as
 * soon as an in-flight slot and enough of the device budget are free (also
 * while others run) and issues each on one of the server's streams, where its
 * kernels overlap with those of the requests already on the device. */
dmx_status dmx_server_create(const dmx_server_cfg* cfg, dmx_server** out);
/* Queues the request (non-blocking).  Admitted to the device once its memory
 * fits the budget and a slot is free.  DMX_ERR_INVALID if it can never fit
 * (device budget, or the host staging block of one in-flight request). */
dmx_status dmx_submit(dmx_server* s, const dmx_request* r, uint64_t* ticket);
/* DMX_OK when the request's outputs are in its host buffers, DMX_NOT_READY
 * while it runs; non-blocking.  latency_s (optional) = submit -> completion. */
dmx_status dmx_poll(dmx_server* s, uint64_t ticket, double* latency_s);
/* Waits (bounded by timeout_s) for all requests, then frees the server. */
dmx_status dmx_server_destroy(dmx_server* s, double timeout_s);

/* Allocation-free rollout (the paper has no counterpart: this is a service of
 * the library).  Some callers cannot let a library call cudaMalloc: real-time
 * control loops, because cudaMalloc may synchronise the whole device and take
 * milliseconds at an unpredictable moment; hosts that hand out all device
 * memory from their own fixed arena or budget; processes whose device
 * footprint must stay constant after start-up.  For them this entry point
 * runs the same integration as dmx_rollout in the plain one-launch-per-attempt
 * form, with the per-environment integrator state kept in one fixed device
 * array compiled into the library (DMX_STATIC_SCRATCH_BYTES, present on every
 * GPU that loads the library until the process exits).  It calls no
 * cudaMalloc, cudaFree or other allocating routine.
 *   - Arguments as in dmx_rollout, with device buffers only (host = 0) and no
 *     tape (tape = NULL); `form` is ignored.  The caller passes all inputs and
 *     outputs; the model must come from dmx_create_model on this device.
 *   - State needed: B * (8 * (nq + 2 nv + 3) + 40) + 8 bytes.  A larger B is
 *     rejected with DMX_ERR_INVALID and a message naming both sizes.
 *   - The first call on a device looks up the array's device address (with
 *     that device current); make that first call before any stream capture.
 *   - Every call on a device uses the same array and leaves its contents
 *     behind: calls whose work overlaps on the GPU (other streams, other host
 *     threads) race and corrupt each other.  Serialise them.
 *   - Returns after the rollout has finished on `stream` (it polls a counter). */
#define DMX_STATIC_SCRATCH_BYTES (4 << 20)
dmx_status dmx_rollout_static(dmx_model* m, const dmx_rollout_args* a, void* stream);

/* Right-hand side v' = F(q, v, u) of Eq. (EOM) for B independent states (no
 * integration): q [nq][B], v [nv][B], u [nu][B] (NULL iff nu == 0) device
 * arrays; cfd = 1 evaluates the CFD right-hand side F~ of Sec. 4.  Writes
 * a [nv][B] and info [4][B] (DMX_ENV_* status, constraint rows, active rows,
 * 0).  The constraint solve starts from an empty active set.  lanes as in
 * dmx_rollout_args (0 = default). */
dmx_status dmx_eval_rhs(dmx_model* m, int32_t B, const double* q, const double* v, const double* u, int32_t cfd,
                        int32_t lanes, double* a, int32_t* info, void* stream);

/* Vector-Jacobian product of the right-hand side (Eq. (EOM) with the
 * constraint solve of Sec. 2.1; cfd = 1: of F~, Sec. 4) for B independent
 * states: qbar [nq][B], vbar [nv][B], ubar [nu][B] (NULL iff nu == 0) receive
 * (dF/dq)^T abar, (dF/dv)^T abar, (dF/du)^T abar for abar [nv][B] at
 * q [nq][B], v [nv][B], u [nu][B] (device arrays).  The constraint solve is
 * differentiated through its final active set.  status [B] = the right-hand
 * side's DMX_ENV_* status.  lanes in {0 (default), 2, 4, 8, 16, 32}. */
dmx_status dmx_eval_rhs_vjp(dmx_model* m, int32_t B, const double* q, const double* v, const double* u,
                            const double* abar, int32_t cfd, int32_t lanes, double* qbar, double* vbar, double* ubar,
                            int32_t* status, void* stream);

/* FP64 throughput probe (the paper has no counterpart: it measures the
 * machine).  Launches blocks x threads threads on `stream`, each running
 * eight independent FP64 fused multiply-add chains of `iters` links: one
 * launch performs 16 * blocks * threads * iters FP64 flops.  The caller
 * times it (CUDA events on `stream`) to obtain the FP64 peak that the
 * rollout and adjoint kernels are reported against.  sink: a device double
 * the kernel may write (it never does for these inputs).  threads must be a
 * multiple of 32 in [32, 1024]; DMX_ERR_INVALID otherwise. */
dmx_status dmx_fp64_peak(int32_t blocks, int32_t threads, int32_t iters, double* sink, void* stream);

const char* dmx_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DMX_H */
