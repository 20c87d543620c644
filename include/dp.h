/*
 * dp.h - C ABI of the GB300 differentiable rigid-body rollout library (libdphys.so).
 *
 * The library steps a batch of independent robots with the impulse-based velocity-stepping
 * engine of "A Differentiable Physics Engine for Deep Learning in Robotics" (arXiv 1611.01652,
 * section 2.1) and returns the reverse-mode gradient of the rollout loss (Eq. L, section 2.2)
 * with respect to the initial state, the per-instance model parameters and the controller
 * weights (Eq. g), by back-propagation through time (section 2.1.1).
 *
 * Problem statement followed by the calls (section 2.2):
 *     x^{t+1} = f_ph(x^t, u^t),   u^t = g_deep(s(x^t) | W),   L = sum_t l(x^t, p).
 *
 * Conventions
 *   - All calls are asynchronous and ordered on the CUDA stream given to dp_create_world.
 *   - Pointer arguments documented as "host or device" may point to either; the library
 *     copies with cudaMemcpyDefault. Caller-owned buffers must stay valid until the stream
 *     has passed the call (cudaStreamSynchronize or dp_sync).
 *   - Nothing aborts: every call returns a dp_status; dp_last_error() gives a message.
 *     Numerical failures (non-finite states) are reported by dp_sync() as DP_ENAN.
 *   - Instances of one world share one topology (bodies, joints, spheres, pairs and the
 *     controller shape); every parameter below is per instance.
 *   - State layout per body: p[3], R[9] (row-major rotation matrix, body-to-world), v[3], w[3]
 *     (world-frame linear and angular velocity) = 18 floats; a state is [B][n_bodies][18].
 */
#ifndef DP_H
#define DP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DP_OK = 0,
  DP_EINVAL = 1,   /* invalid descriptor or argument (nothing was enqueued) */
  DP_ENOMEM = 2,   /* device allocation failed */
  DP_ECUDA = 3,    /* a CUDA call failed; see dp_last_error */
  DP_ETIMEOUT = 4, /* a bounded wait ran out (reserved: no kernel of this library waits on another
                      thread or device, so no call returns it) */
  DP_ENAN = 5,     /* a rollout produced a non-finite state or loss */
  DP_ESTATE = 6    /* call out of order (e.g. dp_backward without a matching dp_rollout) */
} dp_status;

/* Limits of one world's topology. */
#define DP_MAX_BODIES 32
#define DP_MAX_JOINTS 32
#define DP_MAX_SPHERES 32
#define DP_MAX_PAIRS 32
#define DP_MAX_LAYERS 6

enum { DP_JOINT_BALL = 0, DP_JOINT_HINGE = 1 };
enum { DP_FLAG_LIMIT = 1, DP_FLAG_MOTOR = 2 };
/* Controller input blocks, in this order (section 3.1 sensors; section 3.3 sin/cos clock). */
enum {
  DP_F_ANGLES = 1,  /* hinge angle of every motorised hinge, joint order */
  DP_F_RATES = 2,   /* hinge rate of every motorised hinge */
  DP_F_CLOCK = 4,   /* sin(2 pi f t dt), cos(2 pi f t dt) */
  DP_F_IMU = 8,     /* gravity direction and angular velocity of imu_body, in its frame */
  DP_F_TARGET = 16  /* loss point minus loss target (world frame) */
};
/* Loss l(x) of Eq. L, evaluated on the point q = p_b + R_b c of body loss_body. */
enum {
  DP_LOSS_SQDIST = 0, /* |q - target|^2 */
  DP_LOSS_DIST = 1,   /* |q - target| */
  DP_LOSS_LINEAR = 2, /* target . q  (target used as a direction) */
  DP_LOSS_DISP = 3    /* target . (q - q_0) */
};
enum { DP_MODE_FINAL = 0 /* l(x_T) */, DP_MODE_MEAN = 1 /* (1/T) sum_{t=1..T} l(x_t) */ };

/*
 * Batch descriptor, read once by dp_create_world. All arrays are caller-owned host memory.
 * Per-instance arrays have a leading dimension n_instances (B) and are float32.
 */
typedef struct {
  int32_t n_instances;            /* B >= 1 */
  int32_t n_bodies, n_joints, n_spheres, n_pairs;
  /* topology, shared by all instances */
  const int32_t* joint_type;      /* [nj] DP_JOINT_* */
  const int32_t* joint_body;      /* [nj][2] parent a (-1 = world), child b (>= 0, != a) */
  const int32_t* joint_flags;     /* [nj] DP_FLAG_* (hinges only) */
  const int32_t* sphere_body;     /* [ns] body carrying each sphere */
  const int32_t* pair_sphere;     /* [np][2] sphere-sphere candidate pairs (different bodies) */
  /* per-instance parameters */
  const float* mass;              /* [B][nb] kg */
  const float* inertia;           /* [B][nb][3] principal moments in the body frame */
  const float* anchor;            /* [B][nj][2][3] joint point in the parent / child frame
                                     (world frame for a world parent) */
  const float* axis;              /* [B][nj][2][3] hinge axis (unit) in parent / child frame */
  const float* ref;               /* [B][nj][2][3] unit reference vectors perpendicular to the
                                     axis; the hinge angle is the angle between them */
  const float* limit;             /* [B][nj][2] lower, upper angle (rad), lower < upper */
  const float* motor;             /* [B][nj][3] servo gain (1/s), max torque (N m), max rate */
  const float* sph_off;           /* [B][ns][3] sphere centre in its body frame */
  const float* sph_rad;           /* [B][ns] radius */
  const float* sph_mu;            /* [B][ns] Coulomb friction coefficient */
  const float* sph_e;             /* [B][ns] restitution */
  const float* loss_point;        /* [B][3] point c on loss_body (body frame) */
  const float* loss_target;       /* [B][3] target point or direction */
  const float* state0;            /* [B][nb][18] initial state */
  /* controller: dense ReLU network, linear output (Eq. g), bfloat16 storage, fp32 accumulate */
  int32_t n_layers;               /* 0 = no controller (servo targets are 0) */
  int32_t widths[DP_MAX_LAYERS + 1];
  int32_t skip;                   /* 1: the output layer also reads the input layer */
  int32_t features;               /* DP_F_* mask; the input width must equal their count */
  int32_t imu_body;
  float clock_hz;
  /* constants */
  float gravity[3];
  float dt, ground_z, beta, gamma, slop;
  int32_t iters;                  /* projected Gauss-Seidel sweeps per step, >= 1 */
  int32_t horizon;                /* T, steps per rollout, >= 1 */
  int32_t ckpt_every;             /* store a state every K steps for the backward pass;
                                     0 = choose K from free device memory */
  int32_t loss_kind, loss_mode, loss_body;
  int32_t ctrl_fp32;              /* 0: bfloat16 storage points (default); 1: the controller keeps its
                                     input, weights and hidden activations in fp32 (no rounding) */
  int32_t warmstart;              /* 1: reserve room for the learned warm start (dp_set_warmstart) */
  const int32_t* horizons;        /* [B] per-instance horizons in [1, horizon], or NULL (all = horizon).
                                     In dp_rollout an instance's loss of Eq. L ends at its own
                                     horizon; a warp of 32 instances steps to the largest horizon
                                     among them (instances past their horizon keep stepping with a
                                     zero loss weight and get zero adjoints); the trajectory rows
                                     beyond a warp's largest horizon are not written. */
  int32_t rows_global;            /* 1: keep the constraint rows in global memory even when they fit
                                     in shared memory (a launch-configuration choice) */
  int32_t dw_splits;              /* split count of the controller-gradient reduction (0 = automatic) */
  float grad_decay;               /* alpha of section 3.2: the state adjoint passed from step t+1 back to
                                     step t is multiplied by alpha (0 or 1: no decay) */
  int32_t n_recurrent;            /* H >= 0: the recurrent controller state h^t of Eq. g (section 2.2):
                                     the last H network inputs are h^t (a bfloat16 storage point
                                     unless ctrl_fp32), the last H outputs z give
                                     h^{t+1} = tanh(z), h^0 = 0 at the start of a rollout; the
                                     first outputs stay the motor signals. Needs n_layers >= 1,
                                     no skip layer, widths[0] >= features + H and
                                     widths[n_layers] >= motors + H. 0 = feed-forward. */
  int32_t one_warp;               /* launch mapping (a configuration choice, not a change of the
                                     method): 0 = four warps per group of 32 instances for the
                                     recorded rollout and the reverse pass of the topologies the
                                     library compiles (the quadruped, arms of 3-7 links) when the
                                     whole solver tape is kept; 1 = one warp per group for every
                                     launch. Other topologies always run one warp per group. */
} dp_batch_desc;

typedef struct dp_world dp_world; /* opaque; owned by the library */

/* Gradients with respect to the per-instance parameters; each pointer (host or device) may be
   NULL. Shapes are those of the matching dp_batch_desc arrays. Axes and reference vectors are
   model structure and get no gradient. */
typedef struct {
  float *mass, *inertia, *anchor, *limit, *motor, *sph_off, *sph_rad, *sph_mu, *sph_e, *loss_point, *loss_target;
} dp_param_grads;

/*
 * Validate the descriptor, build the static row schedule, pick the checkpoint interval and
 * allocate every device buffer the world needs (parameters, state, checkpoints, per-step tape,
 * controller activations). `stream` is a cudaStream_t (NULL = legacy default stream).
 * Errors: DP_EINVAL (descriptor), DP_ENOMEM, DP_ECUDA. On error *out is NULL.
 */
dp_status dp_create_world(const dp_batch_desc* desc, void* stream, dp_world** out);

/* Release every resource of the world (synchronises its stream first). NULL is a no-op. */
void dp_free(dp_world* w);

/* Number of controller parameters of the world (flat layout: for each layer W[out][in] then
   b[out]; with skip, a final W_skip[out][in0], b_skip[out]). */
int64_t dp_num_params(const dp_world* w);

/* Number of constraint-row slots per instance and the static schedule (host arrays of that
   length, each may be NULL): row kind, owning joint/sphere/pair index, sub-row, bodies a and b
   (-1 = world), colour, and the sweep order (slot indices, colour-major then slot). Kinds:
   0 joint linear, 1 hinge angular, 2 limit, 3 motor, 4 ground normal, 5 ground friction,
   6 pair normal, 7 pair friction. */
int32_t dp_num_slots(const dp_world* w);
dp_status dp_schedule(const dp_world* w, int32_t* kind, int32_t* idx, int32_t* sub, int32_t* body_a,
                      int32_t* body_b, int32_t* colour, int32_t* order);

/* Replace the initial state used by dp_rollout. `state` (host or device) is [B][nb][18]. */
dp_status dp_set_initial_state(dp_world* w, const float* state);

/* Set the current state and step index used by dp_step. */
dp_status dp_set_state(dp_world* w, const float* state, int32_t t);
/* Copy the current state ([B][nb][18]) to `state` (host or device). */
dp_status dp_get_state(dp_world* w, float* state);

/*
 * Advance the current state by n_steps steps of section 2.1 (no gradient bookkeeping).
 * W (host or device, dp_num_params floats, fp32 master weights; NULL if no controller).
 * active (device, optional): [n_steps][B][n_slots] bytes, 1 where a constraint slot was active.
 */
dp_status dp_step(dp_world* w, int32_t n_steps, const float* W, uint8_t* active);

/*
 * Roll all instances from the initial state over the horizon with controller weights W and
 * write the per-instance loss of Eq. L to loss ([B], host or device). Stores the checkpoints
 * needed by dp_backward. traj (device, optional): [T+1][B][nb][18] states; active (device,
 * optional): [T][B][n_slots] bytes. After the call the current state is x_T.
 */
dp_status dp_rollout(dp_world* w, const float* W, float* loss, float* traj, uint8_t* active);

/*
 * Reverse mode through the last dp_rollout: given dL_total/dloss_i in dloss ([B], host or
 * device), write dL/dW (dp_num_params floats), dL/dstate0 ([B][nb][18]) and the parameter
 * gradients (each output optional, host or device). Recomputes every checkpoint segment and
 * replays each step's solver in reverse. Errors: DP_ESTATE without a preceding rollout.
 */
dp_status dp_backward(dp_world* w, const float* dloss, float* dW, float* dstate0, const dp_param_grads* dparams);

/*
 * dp_backward_noalloc: dL/dW through the last dp_rollout, for callers that must not allocate
 * device memory once they are running: an application that reserves all of its device memory up
 * front (a fixed budget shared with other processes, or a pool that owns the GPU), or one that
 * runs on a thread or in a phase where an allocation could block or fail. The paper has no
 * counterpart to this call.
 *
 * It computes the same controller gradient as dp_backward (the other gradients are not
 * produced) and calls no cudaMalloc, cudaFree or other allocating routine: besides the world's
 * own buffers it uses one static device array of DP_NOALLOC_SCRATCH_FLOATS floats (4 MiB),
 * which every GPU that loads the library holds until the process exits, for the split partial
 * sums of the gradient reduction.
 *   - The first call on a device looks up that device's address of the array; make that first
 *     call before any stream capture. The world's device must be current (DP_EINVAL otherwise),
 *     and a cudaDeviceReset after the first call is not supported (the array may move).
 *   - A controller layer with more than DP_NOALLOC_SCRATCH_FLOATS weights is rejected with
 *     DP_EINVAL before anything is enqueued.
 *   - All calls on a device share the array. Every value a call reads from it is written
 *     earlier by the same call, but calls that overlap on the GPU (unordered streams) race:
 *     order them on one stream.
 * dloss ([B]) and dW (dp_num_params floats) may be host or device pointers.
 */
#define DP_NOALLOC_SCRATCH_FLOATS (1 << 20)
dp_status dp_backward_noalloc(dp_world* w, const float* dloss, float* dW);

/* Synchronise the world's stream; DP_ENAN if the last rollout (or dp_step) produced a non-finite
   state or loss, or the last dp_backward a non-finite gradient, naming the first such instance in
   dp_last_error(). */
dp_status dp_sync(dp_world* w);

/* Per-instance status flags (the failure report of the problem statement's batch, section 2.2:
   one robot's non-finite values do not stop the others): bit DP_INST_NAN_STATE is set when the
   instance met a non-finite state or loss in the rollout or steps since the last dp_rollout, bit
   DP_INST_NAN_GRAD when its state or parameter adjoint in the last dp_backward was non-finite.
   dp_instance_status copies the B words to status ([B] int32, host or device, caller-owned),
   stream-ordered. dp_last_error_detail synchronises the stream and writes a one-line report to
   buf (at most n bytes including the terminating NUL): how many instances carry each flag, the
   first eight of them, and the thread's last error message; it returns DP_ENAN when any flag is
   set, DP_OK otherwise, DP_EINVAL for a NULL world (or a NULL buf with n > 0). */
#define DP_INST_NAN_STATE 1
#define DP_INST_NAN_GRAD 2
dp_status dp_instance_status(dp_world* w, int32_t* status);
dp_status dp_last_error_detail(dp_world* w, char* buf, size_t n);

/* Measurement utility (not part of the method): enqueues on `stream` a kernel that keeps every
   SM's FP32 FMA pipes busy (8 blocks of 256 threads per SM, 8 independent FMA chains per thread,
   iters x 16 FMAs per chain) and writes the FLOPs it performs (2 per FMA) to *flops (host).
   sink: a device buffer of at least 8 x SMs x 256 floats that the kernel may write. The caller
   times the kernel on the stream; FLOPs / time is the device's measured FP32 peak, the
   denominator of the roofline of the FP32-bound kernels. DP_EINVAL for iters < 1 or NULLs. */
dp_status dp_fma_peak(int64_t iters, float* sink, int64_t* flops, void* stream);

/* Message of the last failed call on this thread (never NULL). */
const char* dp_last_error(void);

/* Checkpoint interval K chosen at create (states stored every K steps). */
int32_t dp_ckpt_every(const dp_world* w);

/*
 * How the world evaluates its controller u = g(s(x) | W) (section 2.2, Eq. g), chosen at create:
 * DP_CTRL_NONE (no controller), DP_CTRL_SIMT (in the step, one lane per instance, fp32 FMA),
 * DP_CTRL_TENSOR (in the step on the tensor cores: bfloat16 networks K0-H-H-NO with K0 <= 32,
 * NO <= 16, H in {64, 128, 256}; the warp's 32 instances are the rows of each product),
 * DP_CTRL_WIDE (bfloat16 networks with a hidden layer wider than 256: batched tensor-core
 * products between per-step launches). -1 for a NULL world.
 */
enum { DP_CTRL_NONE = 0, DP_CTRL_SIMT = 1, DP_CTRL_TENSOR = 2, DP_CTRL_WIDE = 3 };
int32_t dp_controller_kind(const dp_world* w);

/*
 * Learned warm start of the solver (not in the paper; its solver starts from zero impulses).
 *
 * The rows are taken in groups of three: the linear rows of each joint (x, y, z), the angular
 * rows of each hinge with its motor row, the normal, t1, t2 rows of each contact (groups in slot
 * order of their first row). Each group is described by 16 features taken after row assembly,
 * before the first sweep (rows of inactive slots give zeros):
 *   0-2   J v of the three rows (pre-solve velocities)   3-5  their biases
 *   6-8   their effective masses
 *   9     contact: friction coefficient; hinge: the motor's bound tau_max h; joint: 0
 *   10-11 horizontal offset of the group's point from the centre of mass
 *   12    number of active contacts of the instance
 *   13    weight share M |g| h / max(1, active contacts)
 *   14    height above the ground of the group's point (contact point, or the joint's anchor on
 *         its child body)
 *   15    group type: 0 ground contact, 1 sphere-pair contact, 2 joint, 3 hinge.
 * A 16-64-64-3 network y (ReLU hidden layers, linear output; bfloat16 inputs, weights and
 * hidden activations, fp32 accumulation; flat fp32 parameters W1[64][16], b1[64], W2[64][64],
 * b2[64], W3[3][64], b3[3], DP_WS_PARAMS floats) gives a velocity-scale correction y per row,
 * and the start is alpha lambda_prev + m_eff y (m_eff: the row's effective mass), where
 * lambda_prev are the impulses the rows ended the previous step with (zero before the first step
 * of a rollout and after dp_set_state; the network does not see them), projected
 * on the rows' bounds (normal >= 0, |friction| <= mu normal, |motor| <= tau_max h; inactive rows
 * and limit rows start at zero) and applied in slot order before the sweeps. A zero network is
 * the damped warm start from the previous step. Reverse mode treats the start as a constant.
 */
#define DP_WS_PARAMS 5443
#define DP_WS_ROW 19 /* a harvested row: 16 features, then the network's ideal output y */

/* Enable the warm start with the network W (host or device, DP_WS_PARAMS floats, copied) and
   the weight alpha in [0, 1] of the previous impulses, or disable it (W = NULL; alpha is kept
   for dp_harvest). The world must have been created with desc.warmstart = 1 (DP_EINVAL
   otherwise). Takes effect from the next dp_step / dp_rollout; a recorded rollout is dropped. */
dp_status dp_set_warmstart(dp_world* w, const float* W, float alpha);

/* Replace per-instance parameters in place, for system identification and hardware-parameter
   search by gradient descent through the engine (the section 4 Discussion's outlook; the gradients are
   dp_backward's dp_param_grads): each non-NULL pointer of p (host or device, caller-owned,
   shapes of the matching dp_batch_desc arrays, [B][n], float) overwrites that group for every
   instance; NULL groups are kept. The values are not validated (a non-positive mass or inertia
   gives non-finite states, reported by dp_sync). A recorded rollout is dropped: dp_backward needs
   a new dp_rollout. DP_EINVAL for a NULL world or p. Stream-ordered. */
dp_status dp_set_params(dp_world* w, const dp_param_grads* p);

/* The controller's recurrent state h^t of Eq. g (section 2.2; n_recurrent > 0): set h
   [B][n_recurrent] (float, host or device, caller-owned, copied) as the state the next dp_step
   starts from, or read the current one into h. dp_set_state and every dp_rollout start from
   h = 0. Stream-ordered. DP_EINVAL for a NULL world or h, or a world without recurrent state. */
dp_status dp_set_recurrent(dp_world* w, const float* h);
dp_status dp_get_recurrent(dp_world* w, float* h);

/* The impulses every slot ended the last step with, [B][n_slots] (host or device): read them,
   or set them as the lambda_prev of the next dp_step. */
dp_status dp_set_impulses(dp_world* w, const float* lam);
dp_status dp_get_impulses(dp_world* w, float* lam);

/* Rollout from the initial state with the world's solver (cold, or warm-started) that harvests
   one training row per active group per step: rows (device, [max_rows][DP_WS_ROW]) receives the
   16 features and the network's ideal output, (impulses after the solve - alpha previous
   impulses) / m_eff per row (0 for inactive rows); u_noise (device, [horizon][B][n_motors], or NULL) is added to the controller
   output at every step. *n_rows (host) = rows written (<= max_rows). Synchronises the stream.
   Leaves no rollout for dp_backward. */
dp_status dp_harvest(dp_world* w, const float* W, const float* u_noise, float* rows, int64_t max_rows,
                     int64_t* n_rows);

/* Residual of the solve: with on = 1 every later dp_rollout (which restarts the count) and
   dp_step accumulates, per instance, the RMS over the active rows of the complementarity
   residual after the sweeps (w = J v + bias + gamma lambda: |w| for joint rows, |min(lambda, w)|
   for limits and normals, |lambda - clamp(lambda - w, lo, hi)| for motors and friction).
   dp_get_residual writes the mean over the accumulated steps (device or host, [B]). */
dp_status dp_set_residual(dp_world* w, int32_t on);
dp_status dp_get_residual(dp_world* w, float* resid);

/* Training of the warm-start network on harvested rows (all pointers device memory, ordered on
   `stream`, a cudaStream_t or NULL). dp_ws_loss_grad: loss = (1/n) sum_rows sum_k (y_k -
   lambda_k)^2 and dW = dloss/dW ([DP_WS_PARAMS]; straight-through bfloat16 roundings), using
   `work` of dp_ws_workspace_floats(n) floats. dp_ws_forward: outputs y [n][3] for features
   [n][16]. dp_ws_adam: one Adam step (bias-corrected, step >= 1) on count parameters. */
int64_t dp_ws_workspace_floats(int64_t n);
int32_t dp_ws_param_count(void);
dp_status dp_ws_loss_grad(const float* W, const float* rows, int64_t n, float* loss, float* dW, float* work,
                          void* stream);
dp_status dp_ws_forward(const float* W, const float* feats, int64_t n, float* y, float* work, void* stream);
dp_status dp_ws_adam(float* W, const float* dW, float* m, float* v, int64_t count, int32_t step, float lr, float beta1,
                     float beta2, float eps, void* stream);

/* ------------------------------------------------------------------------------------------
   Differentiable camera (section 3.4: the inverted pendulum observed by a camera). A pinhole ray
   tracer over textured objects carried by the bodies (oriented boxes, spheres, planes), batched
   over instances. The pixel
   (row i, column j) ray leaves the camera centre C along
       d = R_c^T (P ((j + 1/2) - W/2) / f, P ((i + 1/2) - H/2) / f, P),
   so t = 1 is the projection plane at distance P; of the object hits at t >= 1 (in front of the
   projection plane) the nearest is seen. Texture coordinates from the hit point x in the
   object's frame (centre c in the body frame, axes of the body): a box's entry face (box axis k)
   gives u = (x_a / h_a + 1) / 2, v = (x_b / h_b + 1) / 2 (a = k+1, b = k+2 mod 3, h: half extents);
   a sphere of radius h_0 gives u = atan2(x_1, x_0) / (2 pi) + 1/2, v = acos(x_2 / h_0) / pi; a plane
   (the plane x_2 = 0, seen from either side) gives u = frac(x_0 / (2 h_0) + 1/2),
   v = frac(x_1 / (2 h_1) + 1/2) (the texture repeats). The colour is the bilinear interpolation of the object's texture
   (texel centres at ((c + 1/2) / Wt, (r + 1/2) / Ht), clamped at the edges). Rays that hit
   nothing are black. Reverse mode keeps the forward pass's discrete choices (object, face,
   texels, the period of a plane's texture) and differentiates the rest, so the frame's
   derivatives with respect to the body poses and the texels are those of the bilinear
   interpolation. */
#define DP_CAMERA_MAX_OBJECTS 16

typedef struct {
  int32_t width, height; /* pixels; width * height < 2^24 (DP_EINVAL otherwise) */
  float focal;           /* focal length f in pixels */
  float plane;           /* distance P of the projection plane from the camera centre (world units) */
  float position[3];     /* camera centre C (world) */
  float rotation[9];     /* R_c, row-major: rows are the image-right, image-down and optical axes (world) */
} dp_camera;

enum { DP_OBJ_BOX = 0, DP_OBJ_SPHERE = 1, DP_OBJ_PLANE = 2 };
typedef struct {
  int32_t n_obj;           /* objects, <= DP_CAMERA_MAX_OBJECTS */
  const int32_t* body;     /* [n_obj] body carrying the object, -1 = the world frame (host) */
  const float* center;     /* [n_obj][3] object centre in the body frame (host) */
  const float* half;       /* [n_obj][3] box half extents along the body axes; sphere: radius in
                              [0]; plane: texture half periods in [0], [1]; all > 0 (host) */
  const int32_t* tex;      /* [n_obj] texture index (host) */
  int32_t n_tex, tex_h, tex_w; /* textures [n_tex][tex_h][tex_w][3] */
  const int32_t* kind;     /* [n_obj] DP_OBJ_* (host), or NULL: every object is a box */
} dp_scene;

/* Frames image [B][H][W][3] (device) of B instances with body states state [B][nb][18]
   (device; p, R row-major, v, w as dp_get_state) and textures [n_tex][tex_h][tex_w][3]
   (device); hit [B][H][W] (device, optional) receives the object each pixel sees (-1: none). All
   buffers are caller-owned; ordered on `stream` (a cudaStream_t or NULL). DP_EINVAL for a
   malformed camera or scene (dp_camera_last_error says why). */
dp_status dp_render(const dp_camera* cam, const dp_scene* scene, int32_t n_instances, int32_t n_bodies,
                    const float* state, const float* textures, float* image, int32_t* hit, void* stream);

/* Reverse mode of dp_render for the scalar sum(dimage * image): dstate [B][nb][18] (device,
   overwritten; the velocity entries stay zero) and, when not NULL, dtextures [n_tex][tex_h]
   [tex_w][3] (device, overwritten). */
dp_status dp_render_backward(const dp_camera* cam, const dp_scene* scene, int32_t n_instances, int32_t n_bodies,
                             const float* state, const float* textures, const float* dimage, float* dstate,
                             float* dtextures, void* stream);

/* Message of the last camera call that failed on this thread. */
const char* dp_camera_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DP_H */
