/*
 * nasgabor.h -- C ABI of libnasgabor.so: NASGabor appearance evaluation on GB300 (sm_103a).
 *
 * The library evaluates, for every primitive i, the view-dependent colour of
 * the appearance model of "Beyond Spherical Harmonics" (arXiv 2606.09794,
 * Sec. 4.2, eq:app_model)
 *
 *     f_C(d_i) = c0_i + sum_{l=1..L} w_il G(d_i; [x_il, y_il, z_il], lam_il, a_il, k_il)
 *
 * with G the Normalized Anisotropic Spherical Gabor lobe (Sec. 5.1 definition,
 * normalised by the approximate constant of Supp. E/F), at the central-ray
 * direction d_i = (mu_i - cam)/|mu_i - cam| (Sec. 5.2: one evaluation per
 * primitive per frame), plus the matching backward pass (Supp. F derivatives,
 * chained through the Supp. C activations) and the comparison real-SH model
 * (Sec. 3.2, Spherical Harmonics).
 *
 * Conventions for every entry point:
 *   - Device pointers live on the CUDA device current on the calling thread;
 *     "host" pointers are read during the call only.
 *   - The caller owns and allocates every buffer; no entry point allocates
 *     device memory unless its comment says otherwise.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream). Arguments are validated on the host before any launch; a
 *     rejected call launches nothing and returns a negative status.
 *   - n == 0 (or n_idx == 0) is valid and launches nothing.
 *   - No C++ exception crosses this boundary.
 *   - The library looks up the device addresses of its own device variables (an
 *     error word, the fixed scratch of nasg_frustum_compact_noalloc) once per
 *     device and keeps them for the life of the process: after cudaDeviceReset, or
 *     any release of a device's primary context, those addresses are stale, so do
 *     not call into the library on that device again in the same process.
 *
 * Parameter layout ("planes"): a lobe has P raw scalars, P = 10 in QUAT frame
 * mode (q_w q_x q_y q_z lam_r a_r k_r w_r w_g w_b) and P = 9 in COS frame mode
 * (ct_r cp_r cpsi_r lam_r a_r k_r w_r w_g w_b; Supp. C). Parameters are stored
 * plane-major, lobe-minor: element (plane p, primitive i, lobe l) sits at
 * p*N*L + i*L + l. Diffuse colours c0 are planar [3][N]; means, colours and
 * colour gradients are interleaved [N][3].
 *
 * Activations (Supp. C table; act_mode RAW): lam = exp(lam_r), a = exp(a_r),
 * k = 20 (tanh(k_r) + 1), w = tanh(w_r), COS cosines c = tanh(r). In act_mode
 * IDENTITY the stored values are the activated quantities themselves.
 */
#ifndef NASGABOR_H_
#define NASGABOR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t nasg_status;
#define NASG_OK               0
#define NASG_ERR_NULL        -1  /* a required pointer is NULL                         */
#define NASG_ERR_RANGE       -2  /* a size, count or mode is out of range              */
#define NASG_ERR_ALIGN       -3  /* a pointer is not aligned to its element type       */
#define NASG_ERR_UNSUPPORTED -4  /* valid but not built (e.g. an unsupported mode mix) */
#define NASG_ERR_CUDA        -5  /* a CUDA runtime call or launch failed               */
#define NASG_ERR_DEVICE      -6  /* a kernel reported a device-side error (see nasg_device_status) */
#define NASG_ERR_CAPACITY    -7  /* larger than a fixed-capacity entry point can take   */

#define NASG_FRAME_QUAT 0   /* frame from a quaternion (4 raw scalars)              */
#define NASG_FRAME_COS  1   /* frame from three cosines (Supp. C parameterisation)  */

#define NASG_DTYPE_F32  0   /* parameters stored as float32                         */
#define NASG_DTYPE_BF16 1   /* parameters stored as bfloat16 (math stays float32)   */

#define NASG_NORM_APPROX 0  /* C^-1 = lam sqrt(1+a) / (2 pi (1 - e^{-2 lam})) (Sec. 5.1, used for all results) */
#define NASG_NORM_NONE   1  /* the unnormalised Sec. 5.1 kernel (G(z) = 1)          */
#define NASG_NORM_EXACT  2  /* 1 / (Sec. 5.1 closed-form integral): the approximate C^-1 times
                               2 / (1 + Psi), Psi = 2 Lam e^{-Lam} sinhc(sqrt(Lam^2 - k^2)) / (1 - e^{-2 Lam}),
                               Lam = lam (1+a); the paper's "Exact" variant. The printed integral is
                               exact for a = 0 or k = 0 and approximate otherwise.               */

/* Lobe families: the NASGabor lobe and its specialisations. Stored per lobe, after the
 * frame scalars (4 quaternion or 3 cosine planes), in this order:
 *   NASG_FAMILY_NASGABOR  lam, a, k, w_r, w_g, w_b       (P = 10 QUAT / 9 COS)
 *   NASG_FAMILY_NASG      lam, a, w_r, w_g, w_b          (k = 0: no carrier; P = 9)
 *   NASG_FAMILY_SG        lam, w_r, w_g, w_b             (a = 0, k = 0: the normalised
 *                                                          spherical Gaussian; P = 8)
 *   NASG_FAMILY_PHASE     lam, a, k, phi, w_r, w_g, w_b  (carrier (1 + cos(k v + phi))/2,
 *                                                          phi stored as is; P = 11)
 * NASG and SG are the Sec. 5.1 lobe at k = 0 (and a = 0), the distributions of the
 * Supp. A table; the phase carrier is not in the paper (its integral: the
 * closed form with Psi scaled by cos(phi), since the envelope is even in d.x).
 * The families other than NASGabor take QUAT frames and the evaluation entry
 * points (fwd, bwd, fused fwd+bwd) only. */
#define NASG_FAMILY_NASGABOR 0
#define NASG_FAMILY_NASG     1
#define NASG_FAMILY_SG       2
#define NASG_FAMILY_PHASE    3

#define NASG_ACT_RAW      0 /* stored values are raw; Supp. C activations applied   */
#define NASG_ACT_IDENTITY 1 /* stored values are the activated quantities           */

#define NASG_MAX_LOBES 32

/* Shape and mode of one parameter set. */
typedef struct nasg_desc {
  int64_t n;            /* number of primitives N (>= 0)                              */
  int32_t n_lobes;      /* lobes per primitive L, 1..NASG_MAX_LOBES                   */
  int32_t frame_mode;   /* NASG_FRAME_*                                                */
  int32_t param_dtype;  /* NASG_DTYPE_* of `params` and `c0`                           */
  int32_t norm_mode;    /* NASG_NORM_*                                                 */
  int32_t act_mode;     /* NASG_ACT_*                                                  */
  int32_t accumulate;   /* backward outputs: 0 overwrite, 1 add into (g += ...)        */
  int32_t lobe_family;  /* NASG_FAMILY_* (0 = the NASGabor lobe)                       */
  int32_t reserved;     /* must be 0                                                   */
} nasg_desc;

/* Raw scalars per lobe for a frame mode: 10 (QUAT) or 9 (COS); -1 if invalid. */
int32_t nasg_lobe_planes(int32_t frame_mode);

/* Raw scalars per lobe for a frame mode and lobe family (see NASG_FAMILY_*); -1 if
 * the combination is invalid or not supported. */
int32_t nasg_param_planes(int32_t frame_mode, int32_t lobe_family);

/* Static description of a status code (never NULL). */
const char* nasg_status_string(nasg_status status);

/* The cudaError_t of the most recent failed CUDA call made by this library on
 * the calling thread (0 if none); reading it does not clear it. */
int32_t nasg_last_cuda_error(void);

/* Synchronises `stream` and reads the library's device error word, which a
 * kernel sets when one of its bounded waits (on a bulk-copy barrier) gives up
 * instead of hanging. Returns NASG_OK if clear, NASG_ERR_DEVICE if set (and
 * clears it), NASG_ERR_CUDA if the query itself failed. */
nasg_status nasg_device_status(void* stream);

/* ABI version of this header (bumped on any incompatible change). */
#define NASG_ABI_VERSION 4
int32_t nasg_abi_version(void);

/*
 * Forward pass (eq:app_model with the Sec. 5.1 / Supp. F lobe):
 *   rgb[i][c] = c0[c][i] + sum_l w_il[c] G_il(d_i),  d_i = normalize(means[i] - cam).
 *
 * params  device, [P][N*L] of desc->param_dtype (f32 or bf16)
 * c0      device, [3][N] of desc->param_dtype
 * means   device, [N][3] f32
 * cam     HOST, 3 f32 (camera centre)
 * idx     device, nullable: evaluate only primitives idx[0..n_idx) (each in
 *         [0, N)); rgb rows of other primitives are left untouched. NULL
 *         evaluates every primitive (n_idx ignored).
 * rgb     device, [N][3] f32 output
 * Errors: NASG_ERR_NULL (params/c0/means/cam/rgb NULL), NASG_ERR_RANGE (bad
 * desc fields, n_idx < 0), NASG_ERR_ALIGN (misaligned element pointers),
 * NASG_ERR_CUDA (launch failure).
 */
nasg_status nasgabor_eval_fwd(const nasg_desc* desc, const void* params, const void* c0,
                              const float* means, const float* cam, const int32_t* idx,
                              int64_t n_idx, float* rgb, void* stream);

/*
 * Backward pass (Supp. F derivatives, recomputed from the inputs; nothing is
 * saved by the forward): for the upstream gradient g_rgb = dLoss/drgb,
 *   g_params = dLoss/d(raw params) [P][N*L] f32, g_c0 = dLoss/dc0 [3][N] f32,
 *   g_means  = dLoss/dmeans [N][3] f32 (through d = normalize(mu - cam)).
 * g_means may be NULL (not computed). With desc->accumulate = 1 the results are
 * added into the outputs. With idx, only the listed primitives' entries are
 * written. Same errors as the forward; g_rgb, g_params, g_c0 must be non-NULL.
 */
nasg_status nasgabor_eval_bwd(const nasg_desc* desc, const void* params, const float* means,
                              const float* cam, const int32_t* idx, int64_t n_idx,
                              const float* g_rgb, float* g_params, float* g_c0, float* g_means,
                              void* stream);

/*
 * Forward and backward in one pass over the parameters, for a given upstream
 * gradient: writes rgb as nasgabor_eval_fwd and the gradients as
 * nasgabor_eval_bwd, reading params, c0, means and g_rgb once. Every primitive
 * is processed (no index list). g_means may be NULL.
 */
nasg_status nasgabor_fused_fwd_bwd(const nasg_desc* desc, const void* params, const void* c0,
                                   const float* means, const float* cam, const float* g_rgb,
                                   float* rgb, float* g_params, float* g_c0, float* g_means,
                                   void* stream);

/* Adam hyperparameters of one step (bias-corrected, torch.optim.Adam order). */
typedef struct nasg_adam_hparams {
  float lr;       /* learning rate (>= 0)                        */
  float beta1;    /* [0, 1)                                      */
  float beta2;    /* [0, 1)                                      */
  float eps;      /* > 0                                         */
  int32_t step;   /* t >= 1: the step being taken (bias corrections 1 - beta^t) */
} nasg_adam_hparams;

/* Optimiser state of one parameter set, all device pointers, updated in place. */
typedef struct nasg_train_state {
  float* master;        /* [P][N*L] f32 raw lobe parameters (FP32 master)          */
  float* m;             /* [P][N*L] f32 first moments                              */
  float* v;             /* [P][N*L] f32 second moments                             */
  void* params_bf16;    /* [P][N*L] bf16 copy: RNE(master) of the updated entries; nullable */
  float* c0_master;     /* [3][N] f32 diffuse colours                              */
  float* c0_m;          /* [3][N] f32                                              */
  float* c0_v;          /* [3][N] f32                                              */
  void* c0_bf16;        /* [3][N] bf16 copy, nullable                              */
} nasg_train_state;

/* Upstream gradient of nasgabor_fused_step. */
#define NASG_LOSS_GIVEN 0   /* g_rgb_or_target is dLoss/dRGB [N][3]                            */
#define NASG_LOSS_MSE   1   /* g_rgb_or_target is a target colour t [N][3]; the loss is the mean
                               over the listed primitives i and channels c of (c_ic - t_ic)^2, so
                               dLoss/dc_ic = 2 (c_ic - t_ic) / (3 n_listed), formed in the kernel */

/*
 * Fused training step for the listed primitives: forward (eq:app_model), the
 * Supp. F backward for the upstream gradient, and one Adam update of master, m,
 * v (lobe parameters and c0) in one pass, the gradients never being written to
 * memory. The upstream gradient is given (loss_mode NASG_LOSS_GIVEN: g_rgb_or_target
 * holds dLoss/dRGB [N][3] f32), or formed in the kernel from each primitive's colour
 * and a target colour (NASG_LOSS_MSE: g_rgb_or_target holds the target [N][3] f32;
 * fitting the appearance model of Sec. 4.2, eq:app_model, to per-primitive colours
 * without a residual kernel or a gradient buffer). With desc->param_dtype = BF16 the
 * model is evaluated at RNE_bf16(master) (the stored BF16 copy); with F32 at master.
 * Primitives not listed are left untouched (their m, v do not advance).
 *   idx/n_idx     device list of primitives (NULL: all N). Entries outside [0, N) are
 *                 skipped (and still counted in n_listed).
 *   n_idx_device  device int32, nullable: when given, the list length is
 *                 min(n_idx, *n_idx_device) (so the count produced by
 *                 nasg_frustum_compact can be used without a host round trip);
 *                 n_listed is that length.
 *   rgb, g_means  device [N][3] f32 outputs for the listed primitives, nullable.
 * desc->accumulate must be 0. Errors as nasgabor_eval_bwd; NASG_ERR_RANGE for
 * bad hyperparameters or an unknown loss_mode.
 */
nasg_status nasgabor_fused_step(const nasg_desc* desc, const nasg_train_state* state, const float* means,
                                const float* cam, const int32_t* idx, int64_t n_idx,
                                const int32_t* n_idx_device, const float* g_rgb_or_target, int32_t loss_mode,
                                const nasg_adam_hparams* hparams, float* rgb, float* g_means, void* stream);

/*
 * Writes the BF16 copies of a training state from its FP32 masters, for all N
 * primitives: params_bf16 = RNE_bf16(master) [P][N*L] and c0_bf16 = RNE_bf16(c0_master)
 * [3][N] (a NULL copy is skipped); m and v are not touched. The copies the fused step
 * and the fitting step evaluate and write are these roundings (the model is
 * evaluated at the stored BF16 values); use this after initialising or loading the
 * masters. P = nasg_param_planes(desc->frame_mode, desc->lobe_family). Errors:
 * NASG_ERR_NULL (a copy without its master), NASG_ERR_ALIGN, NASG_ERR_RANGE (desc).
 */
nasg_status nasg_train_state_refresh_bf16(const nasg_desc* desc, const nasg_train_state* state, void* stream);

/* Bytes of device workspace nasg_frustum_compact needs for n primitives. */
size_t nasg_frustum_workspace_bytes(int64_t n);

/*
 * Ordered list of the primitives whose centre lies in a pinhole frustum (the
 * primitives a frame sees, Sec. 5.2): with p = R (mu - center), visible iff
 * p_z > near_z, |p_x| <= t p_z and |p_y| <= t p_z, t = tan_half_fov.
 *   rot      HOST 9 f32, row-major world->camera rotation (rows right, up, forward)
 *   center   HOST 3 f32
 *   idx      device [n] int32 output, ascending primitive indices of the visible set
 *   n_visible device int32 output (the list length)
 *   workspace device scratch of nasg_frustum_workspace_bytes(n) bytes, 16-byte aligned
 * Deterministic. n < 2^31. Three kernel launches on `stream`, no host synchronisation.
 */
nasg_status nasg_frustum_compact(int64_t n, const float* means, const float* rot, const float* center,
                                 float tan_half_fov, float near_z, int32_t* idx, int32_t* n_visible,
                                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * nasg_frustum_compact without a workspace argument, for callers that cannot
 * allocate device memory where they need the list: a renderer plugged into a
 * host application that owns every device allocation through its own pool, or
 * a per-frame loop with a fixed memory budget in which a cudaMalloc would
 * synchronise the device. The paper has no counterpart; this is a library
 * convenience.
 *
 * Same arguments, results and determinism as nasg_frustum_compact, except:
 *   - the scratch lives in a fixed array of this library's device memory sized
 *     for NASG_NOALLOC_MAX_PRIMS primitives (about 8 MiB), which every GPU that
 *     loads the library holds until the process exits; larger n is rejected
 *     with NASG_ERR_CAPACITY before anything is launched;
 *   - the first call on a device looks up the array's device address (once per
 *     device, with that device current) and keeps it for the process (see the
 *     conventions above on cudaDeviceReset); make that first call before any
 *     stream capture;
 *   - every call shares the one array: calls that may overlap on the GPU (on
 *     different streams without ordering between them) race and corrupt each
 *     other's lists. Calls ordered on one stream are safe; the array keeps the
 *     last call's contents, and each call writes every scratch byte it reads.
 * No entry point here allocates device memory.
 */
#define NASG_NOALLOC_MAX_PRIMS (1 << 23)
nasg_status nasg_frustum_compact_noalloc(int64_t n, const float* means, const float* rot, const float* center,
                                         float tan_half_fov, float near_z, int32_t* idx, int32_t* n_visible,
                                         void* stream);

/* ------------------------------------------------------------------------
 * Batched persistent forward+backward over many scenes in one launch.
 * A scene is one parameter set with its own N, L, camera and buffers (the
 * layouts of nasgabor_fused_fwd_bwd). The computation per scene is exactly
 * nasgabor_fused_fwd_bwd's (eq:app_model, Supp. F), for the upstream gradient
 * g_rgb given per scene; outputs are overwritten.
 * ------------------------------------------------------------------------ */
#define NASG_MAX_SCENES 256

typedef struct nasg_scene {
  int64_t n;              /* primitives (>= 0)                                  */
  int32_t n_lobes;        /* 1..NASG_MAX_LOBES                                  */
  int32_t reserved0;
  const void* params;     /* device [P][N*L] (f32 or bf16, per nasg_batch_modes) */
  const void* c0;         /* device [3][N]                                      */
  const float* means;     /* device [N][3]                                      */
  float cam[3];           /* camera centre (copied into the table)              */
  float reserved1;
  const float* g_rgb;     /* device [N][3] upstream dLoss/dRGB                  */
  float* rgb;             /* device [N][3] output                               */
  float* g_params;        /* device [P][N*L] f32 output                         */
  float* g_c0;            /* device [3][N] f32 output                           */
  float* g_means;         /* device [N][3] f32 output, nullable                 */
} nasg_scene;

typedef struct nasg_batch_modes {
  int32_t frame_mode, param_dtype, norm_mode, act_mode;  /* shared by every scene */
} nasg_batch_modes;

/* Filled by nasgabor_batched_prepare; pass it to nasgabor_batched_run. */
typedef struct nasg_batch_plan {
  int32_t n_scenes, frame_mode, param_dtype, norm_mode, act_mode, sub_tiles;
  int32_t pair_path;  /* 1: every scene has even L, 2-element aligned parameter planes, 8-byte aligned
                         gradient planes and P N L < 2^31, so the launch runs the pair-load/store
                         kernel with 32-bit offsets; 0: the general kernel */
  int32_t reserved;
  int64_t total_tiles, total_prims, total_lobes;
  void* workspace;
} nasg_batch_plan;

/* Launch schedule: dynamic (1: tiles from an atomic counter, 0: round-robin),
 * blocks per SM (0: as many as fit), sub_tiles (the k prepare was called with),
 * staged (1: each sub-tile's parameter spans, means, upstream gradients and
 * diffuse colours moved into shared memory by bulk copies, three sub-tiles
 * ahead, for the scenes with even L >= 4, N L sizeof(T) a multiple of 16 bytes
 * and 16-byte aligned buffers; the others are loaded directly; 0: every load
 * direct, one sub-tile ahead). */
typedef struct nasg_batch_tuning {
  int32_t dynamic, blocks_per_sm, sub_tiles, staged;
} nasg_batch_tuning;

/* Device workspace bytes for a batch of n_scenes (1..NASG_MAX_SCENES); 0 if out of range. */
size_t nasgabor_batched_workspace_bytes(int32_t n_scenes);

/*
 * Validates the scenes (HOST array of n_scenes) and writes their device table
 * and tile ranges (tiles of sub_tiles sub-tiles of I x 256/S primitives, S the
 * lanes per primitive of the scene's L, I = 2 for BF16 and 1 for FP32 parameters,
 * 1 <= sub_tiles <= 64)
 * into `workspace` (16-byte aligned, >= nasgabor_batched_workspace_bytes).
 * Synchronises `stream` (not for use inside a stream capture). The buffers the
 * scenes point to are read/written by later runs, not by this call.
 */
nasg_status nasgabor_batched_prepare(const nasg_scene* scenes, int32_t n_scenes, const nasg_batch_modes* modes,
                                     int32_t sub_tiles, void* workspace, size_t workspace_bytes,
                                     nasg_batch_plan* plan, void* stream);

/*
 * One persistent launch over every tile of the prepared batch (tuning may be
 * NULL: dynamic scheduling, as many blocks as fit). Enqueues at most a 4-byte
 * memset and one kernel on `stream` and makes no host synchronisation or
 * allocation, so a stream capture of it records a replayable CUDA graph.
 * Runs sharing one workspace must not overlap on the GPU.
 */
nasg_status nasgabor_batched_run(const nasg_batch_plan* plan, const nasg_batch_tuning* tuning, void* stream);

/*
 * Small autotuner: times every schedule (sub_tiles in {1, 2, 4, 8}, static or
 * dynamic, staged or direct, 1 or 2 blocks per SM) on this batch, `reps` runs each, writes the
 * fastest to *best (and its time to *best_ms, nullable) and leaves `workspace`
 * and *plan prepared for it. Runs the batch's kernels (outputs are overwritten).
 */
nasg_status nasgabor_batched_autotune(const nasg_scene* scenes, int32_t n_scenes, const nasg_batch_modes* modes,
                                      void* workspace, size_t workspace_bytes, int32_t reps,
                                      nasg_batch_plan* plan, nasg_batch_tuning* best, float* best_ms,
                                      void* stream);

/* Bytes of device workspace nasgabor_fit_step needs (per-block loss partials). */
size_t nasgabor_fit_workspace_bytes(void);

/*
 * One step of fitting the student mixture (desc: N, L_s even, QUAT frames; the
 * student lives in `state` as for nasgabor_fused_step, evaluated at the BF16
 * values when desc->param_dtype is BF16) to a teacher field (teacher_params
 * [P][N*L_t] raw f32, teacher_c0 [3][N] f32, L_t even with L_t/2 a power of two
 * dividing the student's lanes per primitive) at the n_dirs unit directions
 * dirs [n_dirs][3] (device, shared by all primitives). Per primitive the loss is
 * the mean over (direction, channel) of (student - teacher colour)^2; its
 * gradient summed over the directions takes one Adam step of every primitive
 * (lobe parameters and c0). *loss (device f32) receives the mean squared error
 * over all (primitive, direction, channel). workspace: device scratch of
 * nasgabor_fit_workspace_bytes() bytes. Deterministic. NASG_ERR_UNSUPPORTED for
 * COS frames or lobe counts outside the stated shapes.
 */
nasg_status nasgabor_fit_step(const nasg_desc* desc, const nasg_train_state* state, const float* teacher_params,
                              const float* teacher_c0, int32_t teacher_lobes, const float* dirs, int32_t n_dirs,
                              const nasg_adam_hparams* hparams, float* loss, void* workspace,
                              size_t workspace_bytes, void* stream);

/*
 * Real spherical harmonics of degree 0..3 (Sec. 3.2): orthonormal real basis
 * with the Condon-Shortley phase, coefficient j = l^2 + l + m (m = -l..l).
 *   rgb[i][c] = sum_j coeffs[j][c][i] Y_j(d_i),  d_i = normalize(means[i] - cam).
 * coeffs device [(degree+1)^2][3][N] f32, means device [N][3] f32, cam HOST 3 f32,
 * rgb device [N][3] f32. No offset and no clamp are applied.
 */
nasg_status sh_eval_fwd(int32_t degree, int64_t n, const float* coeffs, const float* means,
                        const float* cam, float* rgb, void* stream);

/* Backward of sh_eval_fwd: g_coeffs [(degree+1)^2][3][N] f32 (overwritten) and
 * g_means [N][3] f32 (nullable, overwritten). */
nasg_status sh_eval_bwd(int32_t degree, int64_t n, const float* coeffs, const float* means,
                        const float* cam, const float* g_rgb, float* g_coeffs, float* g_means,
                        void* stream);

/*
 * Diagnostic: evaluates one of the library's FP32 elementary functions on the
 * device so that tests can measure its error against a float64 reference. The
 * paper has no counterpart; the functions are the kernels' building blocks.
 *   fn 0: y = e^x - 1 for x <= 0            (y2 unused, may be NULL)
 *   fn 1: y = tanh(x), y2 = 1 - tanh(x)^2
 *   fn 2: y = sin(x),  y2 = cos(x)          (|x| <= 6400)
 *   fn 3: fn 1 by the BF16 weight table the BF16 kernels use (x BF16-valued, finite)
 * x, y, y2 device [n] f32. Errors: NASG_ERR_RANGE (fn or n), NASG_ERR_NULL.
 */
nasg_status nasg_math_probe(int32_t fn, const float* x, float* y, float* y2, int64_t n, void* stream);

/*
 * Diagnostic microbenchmark: launches SMs x blocks_per_sm blocks of 256 threads,
 * each thread running `iters` rounds of eight independent dependency chains of one
 * instruction kind, so that the kernel's duration (timed by the caller on
 * `stream`) gives the device's issue rate for it. The paper has no counterpart;
 * it measures the ceilings the arithmetic-bound kernels are graded against.
 *   pipe 0: ex2.approx.ftz.f32 (the multi-function unit: exponentials, reciprocals);
 *   pipe 1: packed FP32x2 fused multiply-add (two FMAs per instruction);
 *   pipe 2: scalar FP32 fused multiply-add.
 * *ops (host) receives the number of lane operations the launch performs (a packed
 * FMA counts two). out: device scratch of SMs x blocks_per_sm floats (written only
 * in a case that does not occur). iters 1..2^24, blocks_per_sm 1..8.
 */
nasg_status nasg_pipe_probe(int32_t pipe, int64_t iters, int32_t blocks_per_sm, float* out, int64_t* ops,
                            void* stream);

/* ------------------------------------------------------------------------- */
/* Host-resident data                                                         */
/* ------------------------------------------------------------------------- */

/* Device workspace bytes of nasgabor_fused_fwd_bwd_host for desc and chunk
 * (a multiple of 8, 8..2^26 primitives); 0 if invalid. */
size_t nasgabor_fused_host_workspace_bytes(const nasg_desc* desc, int64_t chunk);

/*
 * nasgabor_fused_fwd_bwd with every array in HOST memory (the same layouts).
 * When every array is page-locked (mapped into the device's address space,
 * e.g. cudaHostAlloc or torch pin_memory), the kernel reads its inputs and
 * writes its outputs in place over the host link, with plain loads and stores
 * (no copies; chunk and workspace are validated but not used). Otherwise the
 * primitives flow in chunks of `chunk` through three device slots in
 * `workspace` (device, 256-byte aligned, >= nasgabor_fused_host_workspace_bytes),
 * the copies in both directions overlapping the kernel of the neighbouring
 * chunks on two internal copy streams (created once per device). Ordered after
 * the work already queued on `stream`; when `stream` reaches the point after
 * this call, the outputs are in host memory. desc->accumulate must be 0.
 * Errors as nasgabor_fused_fwd_bwd, plus NASG_ERR_RANGE for a bad chunk or
 * workspace.
 */
nasg_status nasgabor_fused_fwd_bwd_host(const nasg_desc* desc, const void* params, const void* c0,
                                        const float* means, const float* cam, const float* g_rgb, float* rgb,
                                        float* g_params, float* g_c0, float* g_means, int64_t chunk,
                                        void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------- */
/* Alpha compositing of the primitives (the consumer of their colours)        */
/* ------------------------------------------------------------------------- */

/* Pinhole camera of the compositing calls. */
typedef struct nasg_raster_camera {
  float rot[9];          /* world -> camera rotation, row-major, rows (right, up, forward)  */
  float centre[3];       /* camera centre (world)                                            */
  float fx, fy, cx, cy;  /* focal lengths and principal point, pixels; image y grows downward */
  float near_z;          /* primitives with camera depth <= near_z are not drawn             */
  int32_t width, height; /* image size, 1..16384                                             */
} nasg_raster_camera;

/* Device workspace bytes for n primitives, a width x height image and room for
 * max_pairs (tile, primitive) pairs; 0 if out of range. */
size_t nasg_raster_workspace_bytes(int64_t n, int32_t width, int32_t height, int64_t max_pairs);

/*
 * Front-to-back compositing of the primitives into an image (Sec. 3.1:
 * C = sum_i T_i alpha_i c_i, alpha_i = sigma_i rho_i, T_i = prod_{j<i}(1 - alpha_j)),
 * with the projection and rules of the Gaussian-splatting rasterizer the paper
 * builds on: p = R (mu - centre), x = cx + fx p_x/p_z, y = cy - fy p_y/p_z, pixel
 * (i, j) sampled at (i + 0.5, j + 0.5); rho = exp(-q/2) of the EWA-projected
 * covariance J R Sigma R^T J^T + 0.3 I, Sigma = Rq diag(s^2) Rq^T;
 * alpha = min(0.99, sigma rho), counted iff alpha >= 1/255; order by p_z (ties by
 * index); a pixel stops before the contribution that would take T below 1e-4.
 *   means [n][3], scales [n][3] (activated, > 0), quats [n][4] (w, x, y, z; any norm),
 *   opacity [n] (sigma in (0, 1)), colours [n][3]: device f32.
 *   image  device [height][width][3] f32 output; final_t device [height][width] f32
 *          output (transmittance left at each pixel).
 *   workspace: device, 256-byte aligned, >= nasg_raster_workspace_bytes(n, w, h,
 *          max_pairs); it keeps the forward's state for nasg_raster_backward.
 *   n_pairs: nullable host output, the number of (tile, primitive) pairs.
 * Synchronises the stream once (to size the sort). NASG_ERR_CAPACITY when the
 * pairs exceed max_pairs (n_pairs still reports the count); n < 2^31.
 */
nasg_status nasg_raster_forward(int64_t n, const float* means, const float* scales, const float* quats,
                                const float* opacity, const float* colours, const nasg_raster_camera* camera,
                                float* image, float* final_t, int64_t max_pairs, void* workspace,
                                size_t workspace_bytes, int64_t* n_pairs, void* stream);

/*
 * Gradients of <g_image, image> of the last nasg_raster_forward with this
 * workspace (same n, colours, camera, max_pairs) wrt the colours and the
 * opacities: g_colours [n][3] and g_opacity [n] (device f32, overwritten):
 *   dC/dc_i = alpha_i T_i,  dC/dalpha_i = c_i T_i - (sum_{later j} c_j alpha_j T_j)/(1 - alpha_i),
 *   dalpha_i/dsigma_i = rho_i where alpha_i < 0.99.
 * final_t: the forward's output; g_image device [height][width][3] f32. Sums over
 * pixels use float atomics (the summation order is not fixed).
 */
nasg_status nasg_raster_backward(int64_t n, const float* colours, const nasg_raster_camera* camera,
                                 const float* final_t, const float* g_image, float* g_colours, float* g_opacity,
                                 int64_t max_pairs, void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------- */
/* Learning-rate rules (host side, no device work)                            */
/* ------------------------------------------------------------------------- */

/*
 * Camera-spacing learning-rate heuristic (Sec. 4.2). d_knn = mean over the
 * cameras of the mean Euclidean distance from the camera centre to its k nearest
 * other centres (all others when n_cams - 1 < k); then
 *   *eta_f     = eta_f_base     * (d_ref / d_knn)^beta    (spherical / feature parameters)
 *   *eta_sigma = eta_sigma_base * (d_knn / d_ref)^gamma   (kernel opacities).
 * The paper uses k = 3, beta = 2, gamma = 0.6 and, as d_ref, the same spacing of a
 * reference capture (a dataset constant supplied by the caller).
 * centres: HOST [n_cams][3] f32, read only. d_knn: nullable output.
 * Errors: NASG_ERR_NULL; NASG_ERR_RANGE for n_cams < 2, k < 1, d_ref not a
 * positive finite number, or all cameras at one point. O(n_cams^2) work.
 */
nasg_status nasg_lr_heuristic(const float* centres, int32_t n_cams, int32_t k, double d_ref, double eta_f_base,
                              double eta_sigma_base, double beta, double gamma, double* eta_f, double* eta_sigma,
                              double* d_knn);

/*
 * Cosine learning-rate factor (Supp. C, LR scheduling): 1 before t_start, then
 * (1 + cos(pi s / S)) / 2 with s = t - t_start and S = t_max - t_start, and 0 from
 * s >= S on (also when S <= 0). The factor multiplies the base rates of the
 * appearance parameters from the start of the schedule (the paper starts it once
 * the model has largely converged). Never fails.
 */
double nasg_cosine_lr_factor(int64_t t, int64_t t_start, int64_t t_max);

/*
 * Diagnostic: launches one block that waits, with an iteration limit of
 * `limit` (1..2^20), on a shared-memory barrier that nothing completes, so that
 * tests can check the bounded-wait path: afterwards nasg_device_status()
 * returns NASG_ERR_DEVICE. The paper has no counterpart; this exercises the
 * library's failure detection without faulting or hanging the GPU.
 */
nasg_status nasg_probe_wait_timeout(int32_t limit, void* stream);

#ifdef __cplusplus
}  /* extern "C" */
#endif

#endif  /* NASGABOR_H_ */
