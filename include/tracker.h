/*
 * tracker.h -- C ABI of the GB300 (sm_103a) silhouette-fitness library for the
 * CMA-ES surgical-instrument tracker of arXiv 2603.11404 (Hu, Liang, Richter,
 * Yip, "Real-time Rendering-based Surgical Instrument Tracking via
 * Evolutionary Optimization").
 *
 * The hot path is the fitness of a whole CMA-ES population (Sec. III-A.1,
 * Sec. III-A.2): for every candidate state Theta = (T_r^c, q) the library
 * runs the kinematics of the instrument links, projects the link meshes
 * through a pinhole camera, rasterises a binary silhouette S and reduces it
 * against the observed mask M to integer counts, all inside one kernel launch
 * (no silhouette is written to memory).  Around it sit the device-resident
 * CMA-ES update of Eq. (cmaes_update) and a per-frame tracking call.
 *
 * Conventions shared by every entry point
 * - Status: every function returns trk_status; nothing throws across the ABI.
 *   TRK_EINVAL means an argument was rejected before any device work was
 *   queued.  TRK_ECUDA means a CUDA call failed (tracker_last_error() gives the
 *   CUDA error string).
 * - Streams: `stream` is a cudaStream_t passed as void*; NULL is the legacy
 *   default stream.  Functions named *_host synchronise that stream before they
 *   return; all others only enqueue work and return immediately.
 * - Memory: pointers named *_dev are device pointers owned by the caller and
 *   must stay valid until the queued work completes; pointers named *_host are
 *   host pointers, read or written before the call returns.  The tracker owns
 *   its copies of the mesh, chain and camera and its scratch buffers.
 * - A state vector has d = 9 * n_instruments floats per candidate:
 *   [r0 r1 r2 | x y z | qh1 qh2 qh3] per instrument (Sec. III-A.3): the
 *   rotation (axis-angle vector, or look-at angles alpha, beta, gamma), the
 *   translation in mm, and the unconstrained joint coordinates q-hat whose
 *   inverse cosine map gives wrist pitch, wrist yaw and jaw angle.  Two
 *   instruments are laid out [Theta_L, Theta_R] (Sec. III-B).
 * - Masks: bit-packed rows, word w of row i holds pixels (i, 32w .. 32w+31),
 *   bit b = pixel 32w+b; row stride ceil(W/32) words; bits past W are zero.
 * - Pixel (i, j) samples the image point (u, v) = (j, i).  Vertices are
 *   snapped to 1/256 px with round-half-even; a pixel is covered by a triangle
 *   under integer edge functions with the top-left rule.
 */
#ifndef TRACKER_H
#define TRACKER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TRK_OK = 0,
    TRK_EINVAL = 1,   /* rejected argument (nothing was enqueued)                 */
    TRK_ENOMEM = 2,   /* device or host allocation failed                          */
    TRK_ECUDA = 3,    /* a CUDA runtime call failed                                */
    TRK_EDEVICE = 4,  /* a kernel raised an error bit of the device error word      */
    TRK_EBUSY = 6     /* admission refused (not enough free memory or slots)       */
} trk_status;       /* (5 is unused: no kernel of this library waits on the device) */

/* Bits of a tracker's device error word (tracker_get_error). */
#define TRK_DEVERR_WORKLIST 0x1u    /* error: the binned rasteriser's work list overflowed
                                       (an internal limit; the launch's counts are incomplete) */
#define TRK_DEVERR_NONFINITE 0x8u   /* warning: a candidate's state held a NaN or an infinity
                                       (its vertices were flagged, its triangles culled)  */

#define TRK_MAX_FRAMES 16     /* kinematic frames per instrument                  */
#define TRK_MAX_INSTRUMENTS 2 /* single arm or bi-manual (Sec. III-B)             */
#define TRK_MAX_D 18          /* 9 * TRK_MAX_INSTRUMENTS                          */
#define TRK_MAX_LAMBDA 1024   /* largest CMA-ES population                         */
#define TRK_MAX_PIXELS (1280 * 1280) /* silhouette bitmap must fit one CTA's smem */

enum { TRK_AXIS_NONE = 0, TRK_AXIS_X = 1, TRK_AXIS_Y = 2, TRK_AXIS_Z = 3 };
enum { TRK_ROT_AXIS_ANGLE = 0, TRK_ROT_LOOKAT = 1 };
enum { TRK_LOSS_XOR = 0, TRK_LOSS_ONE_MINUS_IOU = 1, TRK_LOSS_MSE_APP = 2 };
/* Rasteriser of the fitness path (trk_config.raster); both give identical counts.
 *  CLUSTER: one thread-block cluster per candidate draws every triangle into
 *           per-CTA full-image bitmaps in shared memory, OR-ed through
 *           distributed shared memory (images up to TRK_MAX_PIXELS).
 *  BINNED:  a cluster per candidate projects, sets up and bins the live
 *           triangles by 64 x 32-pixel screen tile (an exact counting sort);
 *           a persistent grid then rasterises the bins in chunks of 256
 *           triangles into shared-memory tile bitmaps and popcounts them
 *           against the mask (images up to 16384 x 8192).
 *  AUTO:    CLUSTER (the faster on every workload measured), BINNED only
 *           where the full-image bitmap would not fit one CTA's shared memory. */
enum { TRK_RASTER_AUTO = 0, TRK_RASTER_CLUSTER = 1, TRK_RASTER_BINNED = 2 };

/* One rigid link mesh in the coordinates of kinematic frame `frame`
 * (the CAD vertices v_m of Sec. III-A.2).  Host arrays, copied at create. */
typedef struct {
    int32_t frame;         /* 0 .. n_frames-1                                  */
    int32_t n_verts;
    const float *verts;    /* [n_verts * 3], mm                                */
    int32_t n_tris;
    const int32_t *tris;   /* [n_tris * 3], indices into this mesh's verts     */
} trk_link_mesh;

/* Forward kinematics T_m^r(q) of one instrument (Sec. III-A.2), as a tree of
 * frames below the end-effector frame E (the wrist-pitch frame, Sec. III-A):
 *   T_f = T_parent(f) * Trans(offset_f) * Rot(axis_f, coef_f * q[joint_f]),
 * parent -1 meaning E, parents listed before children.  q_i is recovered
 * from the state's q-hat_i by the inverse cosine map with limits
 * [q_lb_i, q_ub_i] (Sec. III-A.3).  The camera pose is T_r^c = [R | t]. */
typedef struct {
    int32_t n_frames;
    int32_t parent[TRK_MAX_FRAMES];
    double offset[TRK_MAX_FRAMES][3];
    int32_t axis[TRK_MAX_FRAMES];
    int32_t joint[TRK_MAX_FRAMES];  /* 0 .. 2                                */
    double coef[TRK_MAX_FRAMES];
    double q_lb[3], q_ub[3];
    int32_t rot_param;     /* TRK_ROT_AXIS_ANGLE or TRK_ROT_LOOKAT               */
    int32_t n_instruments; /* 1, or 2 for the bi-manual joint render            */
} trk_chain;

/* Pinhole intrinsics K (Sec. III-A.2).  256*cx and 256*cy must be integers. */
typedef struct {
    double fx, fy, cx, cy;
    int32_t width, height;
    double z_near;         /* mm; vertices closer are flagged                    */
} trk_intrinsics;

typedef struct {
    int32_t loss_kind;     /* TRK_LOSS_*                                         */
    float lambda_app;      /* appearance weight of Eq. render_loss (MSE_APP)     */
    int32_t cull_backfaces;/* 0: union of all faces (default)                    */
    int32_t lambda_max;    /* largest population eval_population will accept     */
    int32_t cluster;       /* CTAs per candidate, 1..8 (0 = auto)                */
    int32_t block_threads; /* threads per CTA: multiple of 32, >= 32 per instrument,
                              <= 256 (0 = auto)                                  */
    int32_t raster;        /* TRK_RASTER_* (0 = auto)                            */
} trk_config;

typedef struct trk_tracker trk_tracker;
typedef struct trk_cmaes trk_cmaes;

/* Human-readable name of a status, and the last CUDA error text seen by this
 * library on the calling thread (empty if none). */
const char *trk_status_string(trk_status s);
const char *tracker_last_error(void);

/* Create a tracker on the current CUDA device: validates and copies the link
 * meshes, the chain and the intrinsics to the device and allocates the
 * per-candidate scratch (snapped vertices) for lambda_max candidates.  Every
 * fitness launch on the tracker uses that scratch, so launches that could
 * overlap on the GPU (other streams, other host threads) race on it: issue
 * them on one stream, or order them with events.
 * Errors: TRK_EINVAL for out-of-range indices, frames, sizes, non-integer
 * 256*cx, images larger than TRK_MAX_PIXELS; TRK_ENOMEM; TRK_ECUDA.
 * Sec. III-A.2 (renderer inputs: v_m, T_m^r, K). */
trk_status tracker_create(const trk_link_mesh *meshes, int32_t n_meshes, const trk_chain *chain,
                          const trk_intrinsics *K, const trk_config *cfg, trk_tracker **out);
trk_status tracker_destroy(trk_tracker *t);

/* The tracker's device error word: every kernel launched for this tracker
 * (fitness, fused generations, batches, servers) ORs TRK_DEVERR_* bits into
 * it instead of trapping.  Synchronises `stream`, copies the word to
 * *device_code (may be NULL) and clears it.  Returns TRK_EDEVICE if an error
 * bit was set, else TRK_OK (warning bits alone still return TRK_OK).  Not a
 * paper feature: the boundary's error reporting. */
trk_status tracker_get_error(trk_tracker *t, uint32_t *device_code, void *stream);

/* Sizes the tracker was created with (any pointer may be NULL). */
trk_status tracker_info(const trk_tracker *t, int32_t *d, int32_t *n_verts, int32_t *n_tris,
                        int32_t *width, int32_t *height, int32_t *words_per_row);

/* Bit-pack an observed mask M_ref (Sec. III-A.2): mask_dev [H*W] bytes, nonzero
 * = tool, into packed_dev [H*ceil(W/32)] words (layout above).  Asynchronous. */
trk_status tracker_pack_mask(trk_tracker *t, const uint8_t *mask_dev, uint32_t *packed_dev, void *stream);

/* THE HOT PATH.  Fitness of lam candidates (Sec. III-A.1-2):
 *   params_dev [lam*d] FP32 states (layout above),
 *   mask_packed_dev the packed observed mask,
 *   loss_dev [lam] FP32 loss of the configured kind:
 *     XOR            s + m - 2I          (MSE of binary images, Eq. render_loss)
 *     ONE_MINUS_IOU  1 - I/(s + m - I)   (0 when the union is empty; Sec. IV-B metric)
 *     MSE_APP        XOR + lambda_app |s - m|   (Eq. render_loss),
 *   counts_dev [lam*4] int32 (s, I, m, culled) or NULL, with s = sum S,
 *     I = sum S&M, m = sum M, culled = triangles skipped because a vertex was
 *     behind z_near or outside the guard band (|u-cx|, |v-cy| > 2^14 px).
 * One launch: kinematics, projection and 1/256 px snapping of every vertex,
 * triangle setup and integer top-left rasterisation into a shared-memory
 * bitmap per candidate, and the popcount reduction against the mask.
 * lam = 0 is a no-op.  Errors: TRK_EINVAL if lam > lambda_max or a pointer is
 * NULL; TRK_ECUDA on a launch failure.  Asynchronous on `stream`. */
trk_status eval_population(trk_tracker *t, const float *params_dev, int32_t lam,
                           const uint32_t *mask_packed_dev, float *loss_dev, int32_t *counts_dev,
                           void *stream);

/* Parity hook: the same launch as eval_population, additionally writing the
 * snapped vertices snap_dev [lam*n_instruments*n_verts*2] int32 (1/256 px;
 * INT32_MIN for a flagged vertex) and the unsnapped offsets from the principal
 * point uv_dev [same shape] FP32 (u - cx, v - cy in px); either may be NULL. */
trk_status eval_population_debug(trk_tracker *t, const float *params_dev, int32_t lam,
                                 const uint32_t *mask_packed_dev, float *loss_dev, int32_t *counts_dev,
                                 int32_t *snap_dev, float *uv_dev, void *stream);

/* Largest lam * n_instruments * n_verts that eval_population_noalloc accepts
 * (the size, in snapped vertices, of its fixed scratch array: 16 MiB). */
#define TRK_NOALLOC_MAX_SNAP (1 << 21)

/* Allocation-free fitness evaluation.  The paper has no counterpart: this is
 * a service for callers that must not allocate device memory at the point
 * where they evaluate a population -- code running inside another framework's
 * memory pool or arena (which forbids cudaMalloc behind its back), real-time
 * control loops that cannot take the allocator's locks or latency, and hosts
 * that only hand out pre-registered buffers.  It computes exactly what
 * eval_population computes, but needs no tracker: the caller passes the mesh,
 * chain, camera and configuration together with the population, and the
 * call allocates nothing (no cudaMalloc, cudaFree or allocating library
 * routine).  The one scratch buffer the kernel needs (every candidate's
 * snapped vertices) is a fixed device array inside this library, 16 MiB,
 * held by every GPU that loads the library until the process exits.
 *   verts_dev [n_verts*4] FP32: x, y, z (mm) and the vertex's frame index
 *     stored as a float; tris_dev [n_tris*4] int32: three vertex indices and
 *     one unused word.  The host cannot validate device memory, so the kernel
 *     checks them: a vertex whose frame is not an integer in [0, n_frames) is
 *     treated as flagged, and a triangle with an index outside [0, n_verts)
 *     is not drawn; both count as culled (counts_dev[4k+3]).
 *   chain, K, cfg: host structs as for tracker_create (cfg.lambda_max is
 *     ignored); params_dev, lam, mask_packed_dev, loss_dev, counts_dev: as
 *     for eval_population.
 * Errors: TRK_EINVAL (reason in tracker_last_error()) for bad arguments (the
 * host-side checks of tracker_create, lam > 65535, more than 2^24 vertices
 * or triangles) or lam * n_instruments * n_verts > TRK_NOALLOC_MAX_SNAP;
 * TRK_ECUDA.  Every call looks up the scratch array's device address on the
 * current device (cudaGetSymbolAddress, which allocates nothing); the first
 * call on a device also loads the library's kernels there, so make it before
 * any stream capture.
 * Every call shares the array: calls whose kernels can overlap on the GPU
 * (other streams, other host threads) race on it and must be serialised by
 * the caller.  Asynchronous on `stream`. */
trk_status eval_population_noalloc(const float *verts_dev, int32_t n_verts, const int32_t *tris_dev, int32_t n_tris,
                                   const trk_chain *chain, const trk_intrinsics *K, const trk_config *cfg,
                                   const float *params_dev, int32_t lam, const uint32_t *mask_packed_dev,
                                   float *loss_dev, int32_t *counts_dev, void *stream);

/* Render the union silhouette of one state into a packed bitmap
 * (silhouette_dev [H*ceil(W/32)] words): used to make synthetic observations
 * and for inspection, not by the fitness path.  Asynchronous. */
trk_status tracker_render(trk_tracker *t, const float *params_dev, uint32_t *silhouette_dev, void *stream);

/* ---------------------------------------------------------------------------
 * Device-resident CMA-ES (Sec. III-A.1, Eq. cmaes_update; Sec. III-B block
 * form).  The state (mean, sigma, C, its symmetric square root and inverse
 * square root, the paths p_sigma and p_c, the generation counters and the
 * best candidate) lives on the device in FP64; populations are FP32.
 * Search coordinates are normalised: state = scales (.) x, C^(0) = I.
 * Samples: x_k = m + sigma C^(1/2) z_k with z from Philox4x32-10 (counter
 * (block, total generation, stream_id, 0), key = seed): 24-bit uniforms
 * ((r >> 8) + 1/2) 2^-24 and the Box-Muller transform in FP32; the
 * covariance, its eigendecomposition, the paths and the step size are FP64.
 * Constants: Hansen's CMA-ES tutorial defaults for n = d, c_m = 1.
 * ------------------------------------------------------------------------- */

/* Create an optimiser for populations of lam (2..TRK_MAX_LAMBDA, <= the
 * tracker's lambda_max) around mean_host [d] (physical units) with per-
 * coordinate scales_host [d] and initial step sigma0 (normalised units).
 * block_diag != 0 keeps C block-diagonal with 9x9 blocks (Sec. III-B).
 * Synchronous (uploads the initial state). */
trk_status cmaes_create(trk_tracker *t, int32_t lam, const double *mean_host, const double *scales_host,
                        double sigma0, uint64_t seed, uint32_t stream_id, int32_t block_diag,
                        trk_cmaes **out);
trk_status cmaes_destroy(trk_cmaes *es);

/* Restart the search around mean_dev [d] FP64 (physical units) on the device:
 * C = I, sigma = sigma0, paths 0, frame-best cleared.  The total generation
 * counter (the random-number stream position) keeps counting. */
trk_status cmaes_reset_device(trk_cmaes *es, const double *mean_dev, void *stream);
trk_status cmaes_reset_host(trk_cmaes *es, const double *mean_host, void *stream);

/* Sample the next population into the optimiser's own buffer and, if
 * params_dev is not NULL, copy it there ([lam*d] FP32).  Asynchronous. */
trk_status cmaes_ask(trk_cmaes *es, float *params_dev, void *stream);

/* The same as cmaes_ask with the standard normals supplied by the caller:
 * z_dev [lam*d] FP64 replaces the Philox draw (for reproducing a sample or
 * checking the update against another implementation).  Asynchronous. */
trk_status cmaes_ask_normals(trk_cmaes *es, const double *z_dev, float *params_dev, void *stream);

/* Copy the standard normals of the last population (z_dev [lam*d] FP64). */
trk_status cmaes_last_normals(trk_cmaes *es, double *z_dev, void *stream);

/* Update from loss_dev [lam] (lower is better; NaN ranks last) for the
 * population of the last ask: stable ranking by (loss, index), weighted
 * recombination, p_sigma, p_c, rank-one and rank-mu update of C, cumulative
 * step-size adaptation, and C^(1/2), C^(-1/2) from an eigenbasis of C warm-
 * started from the previous one (an FP32 one-sided Jacobi pass, then FP64
 * Newton-Schulz orthogonalisation and two Newton steps for the square root).
 * Asynchronous. */
trk_status cmaes_tell(trk_cmaes *es, const float *loss_dev, void *stream);

/* One generation in one launch: every candidate is sampled, evaluated against
 * mask_packed_dev and the update is applied (the same arithmetic as
 * cmaes_ask, eval_population and cmaes_tell in sequence). */
trk_status cmaes_step(trk_cmaes *es, const uint32_t *mask_packed_dev, void *stream);

/* Read the state (synchronises the stream).  Any output pointer may be NULL.
 * mean/p_sigma/p_c [d] normalised, C [d*d], best_x [d] FP32 physical. */
trk_status cmaes_get_state_host(trk_cmaes *es, double *mean, double *sigma, double *C, double *p_sigma,
                                double *p_c, int32_t *gen, int32_t *gen_total, float *best_x,
                                float *best_loss, void *stream);

/* Device pointers of the optimiser's population and loss buffers. */
trk_status cmaes_buffers(trk_cmaes *es, float **params_dev, float **loss_dev, float **best_x_dev);

/* Per-frame tracking (Sec. III-A: the previous estimate seeds the next frame;
 * joint readings, when given, replace the propagated joints).  Restarts the
 * search around the current estimate (the previous frame's best, or the
 * creation mean for the first frame), runs `generations` CMA-ES generations
 * against the packed mask and makes the frame's best candidate the estimate.
 * joint_reading_dev [3*n_instruments] FP32 measured joint angles q, or NULL.
 * pose_out_dev [d] FP32 or NULL.  Asynchronous. */
trk_status track_frame_device(trk_cmaes *es, const uint32_t *mask_packed_dev, int32_t generations,
                              const float *joint_reading_dev, float *pose_out_dev, void *stream);

/* The same from host memory: copies mask_host [H*W] bytes (pinned memory
 * gives an asynchronous copy) and the optional joint_reading_host to the
 * device, packs the mask, tracks, and copies the estimate back to
 * pose_out_host [d] (and its loss to best_loss_out, if not NULL).
 * Synchronises `stream` before returning. */
trk_status track_frame_host(trk_cmaes *es, const uint8_t *mask_host, int32_t generations,
                            const float *joint_reading_host, float *pose_out_host, float *best_loss_out,
                            void *stream);

/* Keypoint term of the objective (Eq. kpts_loss): L = L_render + lambda_kpts
 * sum over instruments of L_kpts, with L_kpts = min over the two assignments
 * of sum_i (|t_i^r - t_sigma(i)^p| - tau)_+ + (|t_mean^r - t_mean^p| - tau)_+,
 * t^p the candidate's projected keypoints (px, image coordinates) and t^r the
 * detections.  The keypoints are two points (mm) in kinematic frames
 * frame[0], frame[1] (the jaw tips).  The term is evaluated for an instrument
 * only when its detection is valid (the paper's "exactly two keypoints").
 * Default: lambda_kpts = 0 (off).  Synchronous, host-side settings. */
typedef struct {
    int32_t frame[2];
    double point[2][3];
    double tau;          /* px */
    double lambda_kpts;  /* weight in loss units per px */
} trk_keypoints;
trk_status tracker_set_keypoints(trk_tracker *t, const trk_keypoints *kp);

/* Detections for the following launches: obs_dev [n_instruments * 5] floats
 * (x1, y1, x2, y2, valid) per instrument, device memory owned by the caller
 * and read by every later fitness launch of this tracker (update its contents
 * on the launching stream between frames); NULL turns the term off.  Batches
 * and servers take the pointer when they are created. */
trk_status tracker_set_keypoint_obs(trk_tracker *t, const float *obs_dev);

/* Projected keypoints of n states [n*d] (device): out_dev [n * n_inst * 4]
 * = (u1, v1, u2, v2) per instrument, image coordinates.  Asynchronous. */
trk_status tracker_project_keypoints(trk_tracker *t, const float *states_dev, int32_t n, float *out_dev,
                                     void *stream);

/* ---------------------------------------------------------------------------
 * Soft (differentiable) silhouette.  The paper fits with a differentiable
 * renderer (Sec. III-A.2) and the MSE term of Eq. (render_loss); this is the
 * soft form of that term, with a hand-written gradient:
 *   d_t(p) = signed distance (px) from pixel centre p to projected triangle t
 *            (+ inside, - outside; unsnapped projection),
 *   a_t(p) = sigmoid(d_t(p) / sigma), 0 where d_t(p) < -14 sigma,
 *   S(p)   = 1 - prod_t (1 - a_t(p)) over every triangle of every link,
 *   L      = sum_p (S(p) - M(p))^2.
 * Triangles with a flagged vertex or zero area are left out.  FP32
 * arithmetic; the loss sums the tiles' squared errors in a fixed order and
 * the gradient sums are exact 64-bit fixed-point integers, so repeated calls
 * give identical results.
 * ------------------------------------------------------------------------- */

/* loss_dev[lam] = L of each candidate of params_dev [lam*d]; with grad_dev
 * [lam*d] not NULL also dL/dparams (physical units: rad, mm, rad of q-hat).
 * The backward recomputes the forward tile by tile: no per-pixel state is
 * kept between the passes.  sigma in [0.05, 64] px.  Asynchronous. */
trk_status soft_eval(trk_tracker *t, const float *params_dev, int32_t lam, const uint32_t *mask_packed_dev,
                     float sigma, float *loss_dev, float *grad_dev, void *stream);

/* Gradient refinement after a tracked frame (call after track_frame_device
 * on the same stream): the top_k candidates of the optimiser's last
 * generation (lowest loss, then lowest index; top_k <= 32) take `steps` Adam
 * steps (beta 0.9 / 0.999, eps 1e-8, step size lr in the optimiser's
 * normalised units) on the soft loss; the refined candidate with the lowest
 * fitness loss (the tracker's loss_kind, binary silhouette) replaces the
 * frame's estimate if it beats the frame's best.  The estimate is written to
 * pose_out_dev [d] (may be NULL); *picked_host (may be NULL; then the call is
 * asynchronous) receives the index of the adopted refined candidate, or -1. */
trk_status soft_refine(trk_cmaes *es, const uint32_t *mask_packed_dev, int32_t top_k, int32_t steps, float lr,
                       float sigma, float *pose_out_dev, int32_t *picked_host, void *stream);

/* ---------------------------------------------------------------------------
 * Heterogeneous batches: many instances (one- or two-instrument scenes with
 * their own meshes, image sizes and population sizes) in one persistent launch
 * per generation and image-size group (instances whose shared-memory bitmaps
 * allow the same number of CTAs per SM form a group; the groups' launches run
 * side by side).  Not a paper feature: the paper tracks one scene per call;
 * batching serves several scenes or camera streams per GPU pass.
 * ------------------------------------------------------------------------- */
typedef struct trk_batch trk_batch;

/* n instances; instance i uses trackers[i] and, if optimisers is not NULL,
 * optimisers[i] (created on trackers[i]) for its populations; otherwise lam[i]
 * gives its population size.  Trackers may be shared between instances (the
 * batch owns its scratch).  cluster (CTAs per candidate, 1..8) and threads
 * (per CTA, multiple of 32, <= 256) may be 0 for the default (8, 256).
 * Synchronous (allocates and uploads the batch's tables). */
trk_status batch_create(trk_tracker *const *trackers, trk_cmaes *const *optimisers, const int32_t *lam, int32_t n,
                        int32_t cluster, int32_t threads, trk_batch **out);
trk_status batch_destroy(trk_batch *b);

/* Launch shape of the persistent kernel: set, or read back (n_clusters = the
 * clusters of the persistent grids, summed over the image-size groups). */
trk_status batch_set_launch(trk_batch *b, int32_t cluster, int32_t threads);
trk_status batch_get_launch(const trk_batch *b, int32_t *cluster, int32_t *threads, int32_t *n_clusters);

/* Fitness of every instance in one persistent launch: host arrays of n device
 * pointers (params [lam_i*d_i], packed masks, loss [lam_i] or a NULL array,
 * counts [lam_i*4] or a NULL array), results identical to eval_population per
 * instance.  Asynchronous on `stream` (the small descriptor upload is staged
 * from host memory before the call returns). */
trk_status batch_eval(trk_batch *b, const float *const *params_dev, const uint32_t *const *masks_dev,
                      float *const *loss_dev, int32_t *const *counts_dev, void *stream);

/* One tracked frame of every instance (the batch must have optimisers): reset
 * around each instance's estimate, `generations` x (one persistent fitness
 * launch that also samples + one launch running every instance's CMA-ES
 * update), then each frame's best becomes its estimate and is written to
 * poses_dev[i] [d_i].  With use_graph != 0 the sequence is recorded once as a
 * CUDA graph and replayed (re-recorded when `generations` changes).  Results
 * are identical to track_frame_device on each instance alone.  Waits for the
 * stream's previous work, then enqueues asynchronously. */
trk_status batch_track_frame(trk_batch *b, const uint32_t *const *masks_dev, int32_t generations,
                             float *const *poses_dev, int32_t use_graph, void *stream);

/* Autotuner: times the persistent fitness launch for every launch shape
 * (CTAs per candidate 1, 2, 4, 8 x threads 128, 256) on this batch's own
 * populations (params_dev per instance, or NULL to use the optimisers'
 * buffers) and masks, keeps the fastest and reports it (any output may be
 * NULL; us_out = microseconds per launch).  Synchronises the stream. */
trk_status batch_autotune(trk_batch *b, const float *const *params_dev, const uint32_t *const *masks_dev,
                          int32_t reps, int32_t *cluster_out, int32_t *threads_out, float *us_out, void *stream);

/* ---------------------------------------------------------------------------
 * Serving: frames from several camera streams with continuous batching.  Not
 * a paper feature: the paper tracks one video stream per process.  Each camera
 * stream keeps its CMA-ES state (an optimiser from cmaes_create) resident on
 * the device and warm-starts it frame to frame.  Submitted frames wait on the
 * host; server_step admits waiting frames into free slots (one frame per
 * stream at a time, at most max_active in all) and enqueues one *tick*: one
 * CMA-ES generation of every admitted frame, their candidates evaluated
 * together in one persistent launch in which the last CTA of each frame's
 * candidates runs that frame's update (a tick with a single frame launches
 * track_frame_device's fused per-frame kernel instead).  A frame
 * finishes after its stream's `generations` ticks; frames admitted later join
 * at the next tick.  Every frame is computed by the kernels of
 * track_frame_device, so its pose is bit-identical to tracking it alone.
 * The server owns one CUDA stream; its calls are not thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct trk_server trk_server;

/* A finished frame.  Times are seconds on the clock of server_now(); t_done
 * is the device completion time of the frame's last tick (its pose download
 * included), mapped onto that clock. */
typedef struct {
    uint64_t tag;                /* the caller's tag from server_submit           */
    double t_submit, t_admit, t_done;
    int32_t stream, d;
    float pose[TRK_MAX_D];       /* the frame's estimate, d entries                */
    float best_loss;
    int32_t pad;
} trk_frame_result;

/* Monotonic host clock (seconds) used for all server times. */
double server_now(void);

/* max_active: frames in slots at once; max_streams: camera streams that can
 * be open; max_pending: frames submitted but not yet admitted, over all
 * streams (each holds a pinned staging copy of max_pixels bytes); max_lambda:
 * largest population of a stream; hbm_reserve_bytes: device memory that
 * server_add_stream must leave free; cluster / threads: launch shape of the
 * fitness launch (0 = 4 CTAs x 256 threads).  Synchronous. */
trk_status server_create(int32_t max_active, int32_t max_streams, int32_t max_pending, int64_t max_pixels,
                         int32_t max_lambda, int64_t hbm_reserve_bytes, int32_t cluster, int32_t threads,
                         trk_server **out);
trk_status server_destroy(trk_server *v);

/* Open a camera stream served by optimiser es (its tracker's image must have
 * at most max_pixels pixels); each frame runs `generations` generations; with
 * use_joint_reading != 0 every submitted frame carries joint readings that
 * reset the joint coordinates of the mean.  Admission by device memory: the
 * stream's raster scratch (lam * n_instruments * n_verts * 8 bytes) is
 * allocated only if hbm_reserve_bytes stay free; otherwise TRK_EBUSY.
 * Synchronous.  *stream_id receives the stream's index. */
trk_status server_add_stream(trk_server *v, trk_cmaes *es, int32_t generations, int32_t use_joint_reading,
                             int32_t *stream_id);
/* Close an idle stream (TRK_EBUSY while it has frames queued or in flight). */
trk_status server_remove_stream(trk_server *v, int32_t stream_id);

/* Queue a frame: copies mask_host [H*W] bytes (0/1) and, for streams opened
 * with joint readings, joint_reading_host [3*n_instruments] into a staging
 * buffer before returning.  t_submit < 0 stamps server_now().  TRK_EBUSY when
 * max_pending frames are already waiting. */
trk_status server_submit(trk_server *v, int32_t stream_id, const uint8_t *mask_host, const float *joint_reading_host,
                         uint64_t tag, double t_submit);

/* Admit waiting frames into free slots and enqueue one tick for every frame
 * in a slot (no-op when none).  Never waits for the device: while two ticks
 * are still running it enqueues nothing, so a newly admitted frame waits for
 * at most one tick; callers loop over server_step / server_poll.
 * n_active_out / n_queued_out (may be NULL): frames in slots, frames still
 * waiting. */
trk_status server_step(trk_server *v, int32_t *n_active_out, int32_t *n_queued_out);

/* Move up to max_out finished frames, in completion order, into out; with
 * wait != 0 first waits for every enqueued tick. */
trk_status server_poll(trk_server *v, trk_frame_result *out, int32_t max_out, int32_t wait, int32_t *n_out);

/* Counters: ticks enqueued so far, frames in slots, frames waiting, free
 * staging buffers (any output may be NULL). */
trk_status server_stats(const trk_server *v, int64_t *ticks, int32_t *n_active, int32_t *n_queued,
                        int32_t *free_staging);

/* Temporal filter (Sec. III-A, temporal filtering): a constant-velocity
 * Kalman filter on the frame estimates, state (Theta, dTheta/dt) with the joint
 * coordinates as joint angles q.  Process noise is block-diagonal with one
 * 2x2 block diag(q_pos[i], q_vel[i]) per coordinate, measurement noise
 * diagonal r[i], so the filter runs as one (position, velocity) filter per
 * coordinate.  The first frame initialises s = (z, 0), P = diag(r, p_vel0);
 * every later frame predicts at its reset (s <- F s, P <- F P F^T + Q with
 * F = [[1, dt], [0, 1]]) and updates with the frame's best candidate as the
 * measurement.  The filtered state, joint angles clamped to their limits, is
 * the frame's estimate and pose output; with seed_mean != 0 the prediction
 * (rather than the last estimate) is the next frame's search mean.  Joint
 * readings, when given, still replace the joints of the mean.  Units: rad,
 * mm, rad of joint angle; dt in the caller's time unit.  Arrays have d
 * entries (up to TRK_MAX_D).  Setting the filter clears its state.
 * Synchronises `stream`. */
typedef struct {
    int32_t enabled, seed_mean;
    double dt;
    double q_pos[TRK_MAX_D], q_vel[TRK_MAX_D], r[TRK_MAX_D], p_vel0[TRK_MAX_D];
} trk_filter;
trk_status cmaes_set_filter(trk_cmaes *es, const trk_filter *f, void *stream);

/* Checkpoint: the whole optimiser state as a plain blob.  cmaes_save with
 * blob = NULL sets *n to the size needed.  A loaded optimiser continues
 * bit-identically.  Both synchronise the stream. */
trk_status cmaes_save(trk_cmaes *es, void *blob, size_t *n, void *stream);
trk_status cmaes_load(trk_cmaes *es, const void *blob, size_t n, void *stream);

/* Roofline denominator of the fitness kernel, measured.  The paper has no
 * counterpart: the fitness path (edge functions, bounding boxes, bit
 * operations) is bound by integer ALU issue, and this call measures that peak
 * on the current device.  One kernel fills every SM to its thread limit; each
 * thread advances eight independent chains of 32-bit LOP3 operations for
 * iters x 16 steps.  *tops_out = operations / kernel time (CUDA events) in
 * 10^12 operations per second; *ms_out (may be NULL) the kernel time;
 * *derived_tops_out (may be NULL) SMs x 64 lanes x the device's maximum SM
 * clock.  About 4 ms at iters = 2000 on a GB300.  Allocates and frees a small
 * buffer (4 bytes per thread) and synchronises the device's default stream.
 * Errors: TRK_EINVAL (iters <= 0, tops_out NULL), TRK_ENOMEM, TRK_ECUDA. */
trk_status trk_probe_int_issue(int32_t iters, double *tops_out, double *ms_out, double *derived_tops_out);

#ifdef __cplusplus
}
#endif

#endif /* TRACKER_H */
