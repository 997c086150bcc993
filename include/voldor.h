/*
 * voldor.h -- C ABI of the GB300 (sm_103a) implementation of VOLDOR's
 * generalized-EM inference (Min, Yang, Dunn, "VOLDOR: Visual Odometry from
 * Log-logistic Dense Optical flow Residuals", CVPR 2020).
 *
 * Problem statement (Sec. 3, Table 1): the input is a window of T dense optical
 * flow fields X_1..X_T, X_t mapping image I_{t-1} to I_t and living on the
 * pixel grid of I_{t-1}; the outputs are the relative camera poses
 * T_1..T_T (T_t maps camera t-1 coordinates to camera t: x_t = R x_{t-1} + t),
 * the depth map theta of I_0 (z-depth) and the rigidness maps W_1..W_T
 * (per-pixel inlier probabilities on the grid of I_0).
 *
 * Conventions shared by every call:
 *  - All calls are extern "C", take plain pointers and sizes, and return a
 *    voldor_status. Nothing aborts, traps or throws across the ABI.
 *  - Images are row-major: pixel j = y * width + x, x = column, y = row.
 *  - Flow stacks are [T][H][W][2] with (u, v) interleaved, float32
 *    (VOLDOR_FLOW_F32) or IEEE binary16 (VOLDOR_FLOW_F16).
 *  - Poses are row-major 4x4 float64 matrices, T of them back to back.
 *  - A context owns all of its device memory and works on the CUDA stream given
 *    at creation (NULL = the legacy default stream). Host-side outputs are
 *    caller-owned; calls that return host data synchronise that stream.
 *  - One context must not be used from two host threads at once; separate
 *    contexts are independent.
 *  - After VOLDOR_ERR_CUDA the context is poisoned: every later call on it
 *    returns VOLDOR_ERR_CUDA until it is destroyed.
 */
#ifndef VOLDOR_H
#define VOLDOR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct voldor_ctx voldor_ctx;
typedef struct voldor_net voldor_net;

typedef enum {
    VOLDOR_OK = 0,
    VOLDOR_ERR_INVALID_ARG = 1,      /* bad size, NULL pointer, NaN/Inf input, unknown enum */
    VOLDOR_ERR_CUDA = 2,             /* a CUDA runtime call failed; context poisoned */
    VOLDOR_ERR_OOM = 3,              /* device allocation failed */
    VOLDOR_ERR_NOT_BOOTSTRAPPED = 4, /* em_step / stage call before voldor_bootstrap or set_state */
    VOLDOR_ERR_DEGENERATE = 5,       /* a frame had no weighted pose hypothesis and kept its pose */
    VOLDOR_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up */
    VOLDOR_ERR_INTERNAL = 7          /* a device-side consistency check failed */
} voldor_status;

enum { VOLDOR_FLOW_F32 = 0, VOLDOR_FLOW_F16 = 1 };
enum { VOLDOR_BOOT_GIVEN_POSE = 0, VOLDOR_BOOT_EPIPOLAR = 2 };

typedef struct { double fx, fy, cx, cy; } voldor_intrinsics;

/* Method parameters. voldor_default_params() fills the paper's values
 * (Sec. 6.1: a1 = 0.01, a2 = 0.09, b1 = -0.0022, b2 = 1.0, lambda = 0.15,
 * gamma = 0.9, Sigma = diag(0.1 x3 translation, 0.004 x3 rotation)) and the
 * numerical guards of this implementation. */
typedef struct {
    double a1, a2, b1, b2;        /* Fisk parameter functions A, B (Eqs. 5-6) */
    double lambda_;               /* adaptive uniform outlier density (Eq. 7) */
    double gamma;                 /* HMM transition probability (Eq. 11) */
    double sigma_t, sigma_r;      /* pose kernel covariance diagonal, variances (Eq. 18) */
    double inv_depth_min, inv_depth_max;  /* depth samples: uniform in inverse depth */
    double x_min, x_max;          /* floor and cap of the squared flow residual, px^2 */
    double beta_min;              /* floor of the Fisk shape B */
    double ms_tol;                /* meanshift stops when |dx| < ms_tol */
    int hyps_per_frame;           /* S: P3P pose hypotheses kept per frame (<= 65536) */
    int groups_per_frame;         /* G: budget of minimal groups per frame (>= 1, <= 262144). Groups
                                     are drawn over the frame's pixels with a 3D-2D correspondence
                                     and solved in order until S hypotheses exist or G groups are
                                     spent; 4 S (the default's ratio) reaches S on every frame of
                                     the driving and handheld workloads */
    int ms_max_iter;              /* meanshift iteration cap */
    int criterion;                /* VOLDOR_CRITERION_MIE (Eq. 10, default) or _MLE (Eq. 9) for the
                                     depth update and the dense pose scores; the E-step posterior
                                     rho/(rho+mu) is the same under both */
    int residual;                 /* VOLDOR_RESIDUAL_FISK (Eqs. 3-6, default) or _GAUSSIAN: the
                                     ablation study's alternative model (Sec. 6.3), an isotropic
                                     normal 2-D residual whose squared EPE is exponential with the
                                     Fisk median alpha(|v_ob|) (Eq. 5); used for rho and mu (Eq. 7)
                                     everywhere the density enters */
    uint64_t seed, window_id;     /* Philox4x64-10 key of the window */
} voldor_params;

enum { VOLDOR_CRITERION_MIE = 0, VOLDOR_CRITERION_MLE = 1 };
enum { VOLDOR_RESIDUAL_FISK = 0, VOLDOR_RESIDUAL_GAUSSIAN = 1 };

void voldor_default_params(voldor_params* p);

/* Creates a context for a W x H image and T flows, copies the flow stack into
 * library-owned device memory (converting nothing: F16 stays F16, F32 stays
 * F32) and allocates the state (theta, W, smoothed W, poses, scratch).
 *  flows:           T*H*W*2 elements of flow_dtype; host memory when
 *                   flows_on_device == 0, device memory of the current device
 *                   otherwise. Copied on `cuda_stream` (a cudaStream_t or NULL).
 *  params:          NULL = voldor_default_params().
 * Errors: INVALID_ARG (width or height < 2 or > 4096, T < 1 or > 16, non-finite or
 * non-positive focal lengths, invalid params, a non-finite flow or a flow
 * vector longer than 16384 px: four times the largest image side; the Fisk
 * model's outlier density (Eq. 7, with alpha = a1 e^{a2 |v|} of Eq. 5) leaves
 * FP32's normal range just beyond it), OOM, CUDA. *out is NULL on error. */
voldor_status voldor_init_window(voldor_ctx** out, int width, int height, int T,
                                 const voldor_intrinsics* K, const voldor_params* params,
                                 const void* flows, int flow_dtype, int flows_on_device,
                                 void* cuda_stream);

/* Replaces the flow stack of an existing context (same size and dtype), with
 * no allocation. The state is unchanged; call voldor_bootstrap next.
 * INVALID_ARG for flows voldor_init_window would reject; the context then
 * holds zero flows and must be bootstrapped again (NOT_BOOTSTRAPPED until). */
voldor_status voldor_set_flows(voldor_ctx* ctx, const void* flows, int flows_on_device);

/* Bootstrap (Table 1, first three lines): W := 1 everywhere; T_1 := the given
 * pose (mode VOLDOR_BOOT_GIVEN_POSE, Sec. 5.3 "from previous estimates"), or
 * (mode VOLDOR_BOOT_EPIPOLAR, T1_rowmajor_4x4 ignored and may be NULL) the
 * epipolar estimate of voldor_bootstrap_epipolar with 512 samples and
 * |t_1| = 1 (the monocular scale convention of that mode); the learned
 * bootstrap is voldor_bootstrap_learned (it needs the network);
 * T_t := T_1 for t >= 2 (used only when a frame has no weighted hypothesis);
 * theta by two-view triangulation of x_j + X_1^j along the ray of pixel j
 * (least squares over the two projection equations, inverse depth clamped to
 * [inv_depth_min, inv_depth_max], non-positive depth sent to the far end).
 * Resets the iteration counter k to 0. T1_rowmajor_4x4: host, 16 doubles.
 * Errors: INVALID_ARG (unknown mode, NULL or non-finite T_1 for GIVEN_POSE),
 * CUDA; with EPIPOLAR also those of voldor_bootstrap_epipolar. */
voldor_status voldor_bootstrap(voldor_ctx* ctx, int mode, const double* T1_rowmajor_4x4);

/* Epipolar bootstrap (Sec. 5.3 and Table 1, second line: T_1 from the
 * epipolar geometry of X_1 by least median of squares), then the bootstrap of
 * voldor_bootstrap with that T_1. Correspondences: every pixel of I_0 whose
 * flow target lies inside I_1, in calibrated coordinates. n_samples minimal
 * samples of 8 pixels (Philox counters (m, 0, 0, 3) and (m, 1, 0, 3) under the
 * window key) give 8-point essential matrices, each scored by the lower median
 * of its Sampson errors over all valid pixels; the best is refined by least
 * squares over its inliers (error <= (2.5 s)^2, s = 1.4826 (1 + 5/(n - 8))
 * sqrt(median)); (R, t) is the decomposition with the most pixels in front of
 * both cameras, and |t| = baseline (a monocular window's scale is free).
 * T1_out (host, 16 doubles, may be NULL) receives T_1. Synchronises the
 * context's stream. VOLDOR_ERR_DEGENERATE if no sample is valid (the state is
 * then unchanged). n_samples in [1, VOLDOR_EPI_MAX_SAMPLES]; scratch of about
 * 25 KB per sample is allocated on first use and kept by the context. */
#define VOLDOR_EPI_MAX_SAMPLES 4096
voldor_status voldor_bootstrap_epipolar(voldor_ctx* ctx, int n_samples, double baseline, double* T1_out);

/* Runs n_iters iterations of the VOLDOR loop (Table 1): for t = 1..T the pose
 * update of Eq. 19 (Philox-drawn minimal groups, P3P, dense scoring of every
 * hypothesis against every pixel, weighted meanshift on se(3)); the E-step
 * with forward-backward smoothing of W (Eqs. 11-14); the MIE depth update by
 * sampling-propagation along directed 1-D chains (Eq. 10, Fig. 5); the
 * unsmoothed W update. Iteration k uses sweep direction
 * [left->right, top->bottom, right->left, bottom->top][k mod 4] and smoothing
 * along rows for even k mod 4, columns otherwise. The iterations run as one
 * CUDA graph on the context's stream; the call then synchronises that stream
 * to read the device status word, from which it learns DEGENERATE and
 * TIMEOUT. Errors: NOT_BOOTSTRAPPED, CUDA, DEGENERATE (state stays valid),
 * TIMEOUT. */
voldor_status voldor_em_step(voldor_ctx* ctx, int n_iters);

/* Copies the outputs into caller-owned host buffers and synchronises.
 *  poses: T*16 doubles (T_t row-major 4x4), depth: H*W floats, rigidness:
 *  T*H*W floats (unsmoothed W_t). Any pointer may be NULL to skip it. */
voldor_status voldor_get_pose_depth_rigidness(voldor_ctx* ctx, double* poses, float* depth,
                                              float* rigidness);

/* Releases the context (NULL is ignored). */
void voldor_destroy(voldor_ctx* ctx);

const char* voldor_status_string(voldor_status s);

/* ---------------------------------------------------------------------------
 * Stage calls: the building blocks voldor_em_step runs, exposed for
 * checkpoint/resume and for parity tests that feed the same state to both
 * sides. All are asynchronous on the context's stream unless stated.
 * ------------------------------------------------------------------------- */

/* Overwrites the state: poses (T*16 doubles, host), depth (H*W floats, host),
 * rigidness (T*H*W floats, host), iteration counter k. NULL leaves that part
 * unchanged. Marks the context bootstrapped. Synchronises. */
voldor_status voldor_set_state(voldor_ctx* ctx, const double* poses, const float* depth,
                               const float* rigidness, int iteration);

/* Pose update of frame t (1..T) at iteration k (Eqs. 15-19): Philox groups,
 * P3P (FP64), dense scores L_h (FP32 per pair, FP64 sums), meanshift seeded at
 * argmax L_h. Results stay readable through voldor_get_buffer. */
voldor_status voldor_pose_update(voldor_ctx* ctx, int k, int t);

/* Dense scoring alone (the step that dominates the EM): scores n caller-given
 * hypotheses of frame t against every valid pixel under the current state.
 *  R: n*9 doubles row-major, tv: n*3 doubles (host); L: n doubles (host).
 *  L_h = sum_j [pi_{t-1}(theta_j) valid] W_t^j log(rho/(rho+mu)), the Eq. 10
 *  criterion with T_t = h. Synchronises. n <= hyps_per_frame. */
voldor_status voldor_score_hypotheses(voldor_ctx* ctx, int t, int n, const double* R,
                                      const double* tv, double* L);

/* E-step of iteration k: emissions rho/(rho+mu) at the current theta and
 * poses, then forward-backward along rows (k mod 4 in {0, 2}) or columns
 * (Eqs. 11-14) into the smoothed map (buffer VOLDOR_BUF_SMOOTHED). */
voldor_status voldor_rigidness_smooth(voldor_ctx* ctx, int k);

/* M-step of iteration k: MIE sampling-propagation sweep (Eq. 10, Fig. 5)
 * using the smoothed map; updates theta and the label map. */
voldor_status voldor_depth_update(voldor_ctx* ctx, int k);

/* Unsmoothed W update (Table 1, last line): W_t^j = rho/(rho+mu). */
voldor_status voldor_rigidness_update(voldor_ctx* ctx);

/* Readable / writable device buffers (host copies; synchronise). */
enum {
    VOLDOR_BUF_SMOOTHED = 0,  /* float [T][H][W] smoothed q(W_t^j = 1), read/write */
    VOLDOR_BUF_LABELS = 1,    /* uint8 [H][W] last sweep's choice: 0 prev, 1 nbr, 2 smp */
    VOLDOR_BUF_HYPS = 2,      /* double [S][12] last pose update's hypotheses: R (9), t (3) */
    VOLDOR_BUF_HYP_INFO = 3,  /* int64 [S][2] group index, solution slot */
    VOLDOR_BUF_HYP_WEIGHT = 4,/* double [S] group weight (product of W) */
    VOLDOR_BUF_SCORES = 5,    /* double [S] dense scores L_h */
    VOLDOR_BUF_POSE_INFO = 6, /* int32 [4] n_hyp, seed index, meanshift steps, status */
    VOLDOR_BUF_DEPTH_SAMPLES = 7, /* float [H][W] last sweep's smp candidates */
    VOLDOR_BUF_HYPS_F32 = 8,  /* float [S][12] scoring form of the hypotheses */
    /* after voldor_bootstrap_epipolar with M samples: */
    VOLDOR_BUF_EPI_E = 9,       /* double [M][9] each sample's essential matrix (row-major; 0 if invalid) */
    VOLDOR_BUF_EPI_MEDIANS = 10,/* float [M] each sample's median Sampson error (+inf if invalid) */
    VOLDOR_BUF_EPI_VALID = 11,  /* int32 [M] 1 valid; rejected: -1 repeated pixel, -2 a flow target outside
                                   I_1, -3 the 8 x 9 system has rank < 8, -4 its null vector has rank < 2 */
    VOLDOR_BUF_EPI_INFO = 12,   /* int64 [8] chosen sample, chosen candidate, valid pixels, inliers,
                                   candidates' cheirality counts [4] */
    VOLDOR_BUF_EPI_REFINED = 13 /* double [27] refined E, then its U and V (row-major) */
};
voldor_status voldor_get_buffer(voldor_ctx* ctx, int which, void* host, size_t bytes);
voldor_status voldor_set_buffer(voldor_ctx* ctx, int which, const void* host, size_t bytes);

/* Per-launch device times (ms, CUDA events on the context's stream) of the
 * dense-scoring kernel during the last voldor_em_step, in launch order, and
 * (if `pairs` is not NULL) the (hypothesis, pixel) pairs each launch scored
 * and (if `hyps` is not NULL) its hypothesis count.
 * Writes min(count, max) values; *count gets the number recorded. Requires
 * timing to be enabled with voldor_enable_timing(ctx, 1) before the step.
 * Synchronises. */
voldor_status voldor_enable_timing(voldor_ctx* ctx, int on);
voldor_status voldor_get_score_times(voldor_ctx* ctx, float* ms, long long* pairs, long long* hyps, int max,
                                     int* count);

/* Number of library kernels enqueued on this context so far (graph replays
 * count every kernel node of the graph). */
long long voldor_kernel_launches(const voldor_ctx* ctx);

/* The CUDA runtime's description of the error that poisoned the context
 * ("no CUDA error" if none). The string is static. */
const char* voldor_last_error_string(const voldor_ctx* ctx);

/* ---------------------------------------------------------------------------
 * Allocation-free dense scoring. The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory when they need
 * a score -- code recording a CUDA graph that must not contain allocations,
 * a process that gives this library a fixed memory budget, or a caller whose
 * own allocator owns the device. It allocates nothing (no cudaMalloc, no
 * cudaFree, no allocating library routine): its only scratch is a 4 MiB
 * array compiled into the library, which every GPU that loads the library
 * holds until the process exits.
 *
 * It computes, on the device and asynchronously on `cuda_stream`,
 *   L[h] = - sum_j records[j].wq * log(1 + mu_j / rho_j(h))
 * for h < n_hyps: the dense score voldor_score_hypotheses returns, but for
 * pixel records and hypotheses the caller supplies.
 *  records: device, n_pix records of 12 floats (48 bytes, 16-byte aligned):
 *           {xb, yb2, w, ut, vt, beta, beta_k, Cp, wq, 0, 0, 0} with, for the
 *           pixel's point P in camera t-1, xb = P_x/P_z, yb2 = (fy/fx) P_y/P_z,
 *           w = 1/P_z, (ut, vt) = X_t(pi_{t-1}) / fx, beta = B(|X_t|),
 *           beta_k = beta * log2(fx^2 / A(|X_t|)), Cp = fx^2 * mu / beta
 *           (mu of Eq. 7), wq = W_t^j. Every record given is scored.
 *  hyps:    device, n_hyps x 12 floats: E (9, row-major) and tt (3) with
 *           E = S (R - I) S^-1, tt = S t, S = diag(1, fy/fx, 1).
 *  xs_min, xs_max: floor and cap of the squared residual divided by fx^2.
 *  L:       device, n_hyps doubles, written.
 * Limits: 1 <= n_hyps <= 8192, n_pix >= 0, records 16-byte aligned, hyps
 * 4-byte aligned, L 8-byte aligned; otherwise INVALID_ARG before any device
 * work. The first call on a device looks up the scratch array's device
 * address (with that device current); make that first call before any stream
 * capture. Every call writes each scratch cell it later reads, so nothing
 * carries over between calls -- but all calls share the one array, so calls
 * that overlap on the GPU (different streams, or different host threads) race
 * and must be serialised by the caller. Errors: INVALID_ARG, CUDA. */
voldor_status voldor_score_records_noalloc(const float* records, int n_pix, const float* hyps, int n_hyps,
                                           double xs_min, double xs_max, double* L, void* cuda_stream);

/* Diagnostic for rooflines (no counterpart in the paper): measures the SFU
 * (special-function unit) throughput of the current GPU in results per SM
 * clock for op 0 = exp2, 1 = log2, 2 = reciprocal (approximate forms). One
 * wave of 4 blocks per SM runs 16 independent chains per thread; the grid is
 * timed with CUDA events and divided by the SM clock measured during the run
 * (cycle counter over the global nanosecond timer, median over blocks), which
 * is returned in *sm_mhz (may be NULL). Allocates and frees a few KB;
 * synchronises the device. Errors: INVALID_ARG, OOM, CUDA. */
voldor_status voldor_probe_sfu_rate(int op, double* results_per_sm_clock, double* sm_mhz);

/* Exercises the expiry path of the bounded device-side waits (every mbarrier
 * wait of the library's kernels gives up after a poll limit and the call
 * reports VOLDOR_ERR_TIMEOUT): one block of 128 threads waits, with the dense
 * scoring's bounded wait, on an mbarrier phase that nothing completes, for
 * `polls` polls (0 .. 2^26, the kernels' own limit). Returns VOLDOR_ERR_TIMEOUT when every thread gave
 * up (the expected result), with the SM cycles the wait took in *cycles (may
 * be NULL); the device stays usable. Synchronises the device. Errors:
 * INVALID_ARG, OOM, CUDA. */
voldor_status voldor_probe_bounded_wait(long long polls, long long* cycles);

/* ---------------------------------------------------------------------------
 * Batching and tuning of many windows (no counterpart in the paper).
 * ------------------------------------------------------------------------- */

/* Autotunes the dense-scoring tile shape of one window: hypotheses per thread
 * (2, 4 or 8, i.e. 512, 1024 or 2048 hypotheses per block, 3, 2 or 1 blocks
 * per SM) and pixel chunks (1, 2, 4
 * or 8 waves of resident blocks), timing each candidate with CUDA events on
 * the window's own frame-1 hypotheses and records. Keeps the fastest;
 * discards captured graphs that used another shape. Overwrites the stage
 * buffers (hypotheses, records), not the state (poses, depth, W, k).
 * Synchronises. Outputs may be NULL. */
voldor_status voldor_autotune(voldor_ctx* ctx, int* hyps_per_thread, int* chunks, float* best_ms);

/* Sets the dense-scoring tile shape directly (hyps_per_thread 2, 4 or 8). */
voldor_status voldor_set_score_shape(voldor_ctx* ctx, int hyps_per_thread, int chunks);

/* A batch of windows run as one CUDA graph: every window's n_iters
 * iterations (the graph voldor_em_step would replay) become independent
 * branches of a single graph launch, so windows of different sizes and T run
 * concurrently. Each window must be bootstrapped and appear once; windows
 * must outlive the batch. */
typedef struct voldor_batch voldor_batch;
voldor_status voldor_batch_create(voldor_ctx* const* ctxs, int n, int n_iters, voldor_batch** out);

/* Launches the batch on `cuda_stream` and synchronises. latency_ms (n floats,
 * or NULL) receives, per window, the time from the batch start to the end of
 * that window's last kernel (CUDA events). Returns DEGENERATE if any window
 * had a frame without weighted hypotheses. */
voldor_status voldor_batch_run(voldor_batch* batch, void* cuda_stream, float* latency_ms);
void voldor_batch_destroy(voldor_batch* batch);

/* One-shot form: create, run on the legacy stream, destroy. */
voldor_status voldor_em_batch(voldor_ctx* const* ctxs, int n, int n_iters);

/* ---------------------------------------------------------------------------
 * Absolute scale from the ground plane (Sec. 6.1: the scale is taken from the
 * mode over the pixels whose surface normal is near the vertical; the paper's
 * details are in an appendix that is not part of its text). From the current
 * depth of I_0: normals by central differences of the back-projected depth
 * map; rigid pixels (mean W >= 1/2) below the camera (image y axis down) whose
 * normal is within max_tilt_rad of the camera's y axis, with all five depths of
 * the stencil strictly inside the depth range, give the distance of their
 * tangent plane from the camera; the mode of log2 of those heights (4096 bins
 * over [-8, 8), argmax of the 5-bin box-filtered histogram, centroid of the raw
 * bins around it) gives scale = camera_height / 2^mode. With apply != 0 the
 * depth and every translation are multiplied by it. Synchronises the
 * context's stream. VOLDOR_ERR_DEGENERATE if no pixel qualifies.
 * ------------------------------------------------------------------------- */
voldor_status voldor_ground_scale(voldor_ctx* ctx, double camera_height, double max_tilt_rad, int apply,
                                  double* scale_out);

/* ---------------------------------------------------------------------------
 * Learned proposal (no counterpart in the paper): a 6-layer
 * 3x3 convolutional network, 2T -> 32 -> 32 -> 32 -> 32 -> 32 -> 2 channels
 * with ReLU between layers, reads the flows (divided by 32 px, 2 channels per
 * frame, T <= 8) and predicts per pixel a log-depth and a rigidness logit. BF16
 * weights and activations, FP32 accumulation on tensor cores, FP32 Adam on
 * master weights. Parameters: per layer W[Cout][3][3][Cin] then bias[Cout],
 * FP32, layers in order.
 * ------------------------------------------------------------------------- */
size_t voldor_net_num_params(int T);                 /* 0 if T is not in [1, 8] */
voldor_status voldor_net_create(int T, voldor_net** out);   /* parameters start at zero */
void voldor_net_destroy(voldor_net* net);
voldor_status voldor_net_set_weights(voldor_net* net, const float* host, size_t count);   /* resets Adam */
voldor_status voldor_net_get_weights(voldor_net* net, float* host, size_t count);
/* Gradient of the last voldor_net_train_step's loss (before its update). */
voldor_status voldor_net_get_grads(voldor_net* net, float* host, size_t count);
/* Forward pass on B images of H x W: flows device [B][T][H][W][2], pred device
 * [B][H][W][8] floats (channel 0 log-depth, 1 rigidness logit, rest zero).
 * The last layer writes pred directly when it is 16-byte aligned memory of
 * the current device, else the network's own buffer, copied to pred on the
 * stream; the results are the same. Synchronises the stream. */
voldor_status voldor_net_forward(voldor_net* net, const void* flows, int flow_dtype, int B, int H, int W, float* pred,
                                 void* cuda_stream);
/* One training step: forward, loss = mean over pixels of Huber(delta 0.1) on
 * log-depth + lam_r * BCE on the rigidness logit (target device
 * [B][H][W][2]: log-depth, rigidness in [0, 1]; a non-finite log-depth skips
 * the pixel), backward, Adam (lr; lr = 0 computes gradients only). *loss
 * (host, may be NULL) gets the loss before the update. Synchronises. */
voldor_status voldor_net_train_step(voldor_net* net, const void* flows, int flow_dtype, const float* target, int B,
                                    int H, int W, float lr, float lam_r, float* loss, void* cuda_stream);
/* Learned bootstrap: poses, depth and W as in voldor_bootstrap (T_1 given,
 * triangulated depth), then the network's prediction replaces
 *   - with VOLDOR_LEARNED_DEPTH: the depth, exp(log-depth + s) clamped to the
 *     depth range, where s = median over pixels of log(theta_tri) - log-depth
 *     (pixels whose triangulated depth is strictly inside the range) puts the
 *     prediction on the metric scale that T_1 fixes;
 *   - with VOLDOR_LEARNED_RIGIDNESS: every W_t, by sigmoid(logit).
 * flags = 0 is the plain bootstrap. The network's T must equal the window's. */
enum { VOLDOR_LEARNED_DEPTH = 1, VOLDOR_LEARNED_RIGIDNESS = 2 };
voldor_status voldor_bootstrap_learned(voldor_ctx* ctx, const double* T1_rowmajor_4x4, voldor_net* net, int flags);

/* Device memory held by the context, bytes. */
size_t voldor_device_bytes(const voldor_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* VOLDOR_H */
