// Internal declarations shared by the CUDA translation units of the tracker
// library (kernels in raster.cu and cmaes.cu, the C ABI in abi.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <math.h>

#include "../../include/tracker.h"

namespace trk {

constexpr int kMaxFrames = TRK_MAX_FRAMES;
constexpr int kMaxD = TRK_MAX_D;
constexpr int kSnapFlag = INT32_MIN;          // snapped x of a flagged vertex
constexpr int kBigListCap = 1024;              // large triangles deferred per CTA
constexpr double kGuardPx = 16384.0;           // |u - cx|, |v - cy| limit (2^14 px)

// Kinematic chain of one instrument in device-friendly form (Sec. III-A.2).
// Constants also carry double-float (hi, lo) copies, split on the host, for the
// per-candidate kinematics that run on the FP32 pipes.
struct ChainDev {
    int n_frames, n_inst, rot_param, pad;
    int parent[kMaxFrames], axis[kMaxFrames], joint[kMaxFrames];
    double offset[kMaxFrames][3];
    double coef[kMaxFrames];
    double q_lb[3], q_ub[3];
    float2 offset_df[kMaxFrames][3];
    float2 coef_df[kMaxFrames];
    float2 lb_df[3], half_range_df[3], pi_over_range_df[3];  // lb, (ub-lb)/2, pi/(ub-lb)
};

// Pinhole camera (Sec. III-A.2) and image geometry.
struct CamDev {
    double fx, fy, z_near, guard;
    int W, H, Wq, cx256, cy256;
    float2 fx_df, fy_df;
};

// Binned pipeline (binned.cu): the screen is cut into tiles of kTileW x kTileH
// pixels (two mask words by 32 rows); each candidate's live triangles are
// binned by tile, and a tile's bin is rasterised in work items of up to
// kBinChunk entries.
constexpr int kTileW = 64;
constexpr int kTileH = 32;
constexpr int kTileWords = kTileH * (kTileW / 32);
constexpr int kBinChunk = 1024;   // records per raster work item (taken 32 at a time by the warps of a CTA)
constexpr int kBinMaxTilesPerAxis = 256;  // tile ranges are packed in 8-bit fields

// Scratch of the binned pipeline, sized when the tracker is created.
struct BinDev {
    float *frames;       // [lam][n_inst][n_frames][24] projective rows of every candidate (hi, lo)
    int2 *pool;          // [lam][pool_cap][3] snapped vertices of the binned triangles, grouped by tile
    int4 *items;         // [max_items] raster work items: candidate, tile | tx << 16 | ty << 24,
                         // first pool record, records | chunks of the tile << 9
    uint32_t *merge;     // [lam][n_tiles][kTileWords] OR of a multi-chunk tile (zero between launches)
    int *tile_done;      // [lam][n_tiles] finished chunks of a multi-chunk tile (zero between launches)
    int *acc;            // [lam][4] s, I, culled, unused (zeroed by the front kernel)
    unsigned *ctl;       // [4] items, item ticket, exit ticket, m (zero between launches)
    int n_tx, n_ty, n_tiles, pool_cap, max_items, live_cap, tiles_grid, pad[3];
};

// Everything one fitness launch needs (a multiple of 16 bytes: batched
// launches copy it into shared memory in 16-byte pieces).
struct __align__(16) EvalArgs {
    ChainDev ch;
    CamDev cam;
    const float4 *verts;   // [V] x, y, z, frame index (exact small float)
    const int4 *tris;      // [T] i0, i1, i2, 0
    int V, T;
    // [P] the mesh as primitives: (a, b, c, d) is the pair of triangles (a, b, c)
    // and (a, c, d) sharing the edge a-c, (a, b, c, -1) a single triangle; NULL
    // in the index-checked launch, which draws tris[]
    const int4 *prims;
    int P, pad_p;
    const float *params;   // [lam * d]
    int d, lam;
    const uint32_t *mask;  // packed [H * Wq]
    int2 *snap;            // scratch [lam * n_inst * V]
    float *loss;           // [lam] or null
    int *counts;           // [lam * 4] or null
    int2 *snap_dbg;        // optional export of snapped vertices
    float2 *uv_dbg;        // optional export of unsnapped offsets
    uint32_t *silhouette;  // optional: write the union bitmap (render mode, lam == 1)
    int loss_kind;
    float lambda_app;
    int cull;
    // fused CMA-ES generation (all NULL for a plain fitness launch): every
    // cluster samples its own candidate, the last CTA to finish runs the update
    const struct CmaConst *cma_k;
    struct CmaState *cma_st;
    double *cma_y, *cma_z;     // [lam * d] steps and normals of the population
    unsigned *cma_done;        // CTA ticket counter, zero between launches
    float *cma_pose_out;       // frame estimate output (finish only), may be NULL
    int cma_finish;            // 1: also make the frame's best the estimate
    // keypoint term of the objective (Eq. kpts_loss): two keypoints per
    // instrument (frame, point in that frame), threshold tau, weight lambda;
    // kp_obs [n_inst * 5] = detected (x1, y1, x2, y2, valid) or NULL (term off)
    int kp_frame[2];
    float kp_pt[2][3];
    float kp_tau, kp_lambda;
    const float *kp_obs;
    BinDev bin;            // binned pipeline scratch (unused by the cluster-bitmap kernel)
    unsigned *err;         // the tracker's device error word (TRK_DEVERR_*), or NULL
    int pad_err[2];
};

struct LaunchCfg {
    int cluster;           // CTAs per candidate
    int threads;           // threads per CTA
    size_t smem;           // dynamic shared memory per CTA
};

// Constant-velocity Kalman filter on the frame estimates (temporal filtering,
// Sec. III-A): state (Theta, dTheta/dt) with the joint coordinates as joint
// angles q; process noise block-diagonal, one 2x2 block diag(q_pos, q_vel)
// per coordinate, measurement noise diagonal, so the filter splits into one
// (position, velocity) filter per coordinate.
struct KfConst {
    int enabled, seed_mean;  // seed_mean: the prediction is the next frame's mean
    double dt;
    double q_pos[kMaxD], q_vel[kMaxD], r[kMaxD], p_vel0[kMaxD];
};
struct KfState {
    int initialized, pad;
    double s[kMaxD][2];      // position, velocity
    double P[kMaxD][3];      // covariance p00, p01, p11
};

// CMA-ES constants, host-computed in FP64 (Hansen's tutorial defaults).
struct CmaConst {
    int d, lam, mu, block;
    double w[TRK_MAX_LAMBDA / 2];
    double mu_eff, c_sigma, d_sigma, c_c, c_1, c_mu, c_m, chi_n, sigma0;
    // derived on the host: sqrt(c_s (2 - c_s) mu_eff), sqrt(c_c (2 - c_c) mu_eff),
    // ((1.4 + 2/(n+1)) chi_n)^2, c_s / d_s, 1 / chi_n
    double ps_coef, pc_coef, hs_thr2, cs_over_ds, inv_chi;
    double scales[kMaxD];
    float2 scales_df[kMaxD];
    double q_lb[3], q_ub[3];
    unsigned long long seed;
    unsigned stream_id;
    KfConst kf;
};

// Device-resident CMA-ES state (FP64 except the FP32 population and best).
struct CmaState {
    double m[kMaxD], p_sigma[kMaxD], p_c[kMaxD];
    double C[kMaxD * kMaxD], B[kMaxD * kMaxD], ev[kMaxD];
    double C_half[kMaxD * kMaxD], C_inv_half[kMaxD * kMaxD];
    double est[kMaxD];     // current estimate (physical units), seeds the next frame
    double sigma;
    double cs_pow;         // (1 - c_sigma)^(2 gen), for the h_sigma test
    int gen, gen_total;
    int jacobi_sweeps;     // sweeps of the last eigen-path update, or minus its Newton-Schulz steps
    int warn;              // bit 0: an eigenvalue was not positive; bit 1: Newton-Schulz did not
                           // converge, the eigen path serves until the next reset
    float best_loss;       // best of the current frame (since the last reset)
    float best_x[kMaxD];
    // double-float copies for the sampler (FP32 pipes): C^(1/2), mean, sigma
    float2 C_half_df[kMaxD * kMaxD];
    float2 m_df[kMaxD];
    float2 sigma_df;
    KfState kf;
};

// hi/lo split of a double into a double-float pair (host or device).
__host__ __device__ inline float2 split_df(double x)
{
    float hi = (float)x;
    return make_float2(hi, (float)(x - (double)hi));
}

cudaError_t launch_eval(const EvalArgs &a, const LaunchCfg &cfg, cudaStream_t s);
// The cluster-bitmap kernel with index checks (meshes in the caller's device
// memory): a vertex whose frame index is out of range is flagged, a triangle
// with a vertex index out of range is culled.
cudaError_t launch_eval_checked(const EvalArgs &a, const LaunchCfg &cfg, cudaStream_t s);
// Binned pipeline: the front kernel (cluster of cfg.cluster CTAs per candidate)
// and the persistent tile kernel; fused CMA-ES generations when a.cma_st is set.
cudaError_t launch_binned(const EvalArgs &a, const LaunchCfg &cfg, cudaStream_t s);
size_t binned_front_smem_bytes(const EvalArgs &a, int threads);
size_t binned_tiles_smem_bytes();
cudaError_t prepare_binned(size_t front_smem, int *tiles_per_sm);
// Raise a kernel's dynamic shared memory limit on the current device to at
// least smem (kept per device and kernel; thread-safe).
cudaError_t ensure_smem_attr(const void *func, size_t smem);
cudaError_t launch_project_keypoints(const EvalArgs &a, const float *states, int n, float *out, cudaStream_t s);
size_t tell_smem_bytes();
cudaError_t launch_eval_batch(const EvalArgs *descs_dev, const uint32_t *const *masks_dev, const int2 *items_dev,
                              int n_items, unsigned *next_item_dev, const LaunchCfg &cfg, int n_clusters,
                              cudaStream_t s, const int *tell_last_dev = nullptr);
cudaError_t prepare_eval_batch(size_t smem, int cluster, int threads, int *max_clusters);
cudaError_t launch_pack_mask(const uint8_t *mask, uint32_t *packed, int W, int H, int Wq, cudaStream_t s);
size_t eval_smem_bytes(const EvalArgs &a);
cudaError_t prepare_eval(size_t smem);
void set_last_error(const char *msg);  // the text tracker_last_error() returns
int eval_max_threads();

cudaError_t launch_cma_reset(const CmaConst *k, CmaState *st, const double *mean_dev, bool from_est,
                             const float *joint_reading_dev, int n_inst, cudaStream_t s);
cudaError_t launch_cma_ask(const CmaConst *k, int lam, CmaState *st, double *y, double *z_keep, float *params,
                           const double *z_in, cudaStream_t s);
cudaError_t launch_cma_tell(const CmaConst *k, CmaState *st, const double *y, const float *params,
                            const float *loss, cudaStream_t s);
cudaError_t launch_cma_finish_frame(const CmaConst *k, CmaState *st, float *pose_out, cudaStream_t s);
// C^(1/2), C^(-1/2) and the eigenbasis of the stored C (completes an update
// made without them).
cudaError_t launch_cma_sqrt(const CmaConst *k, CmaState *st, cudaStream_t s);
// Device tables (one entry per instance) for the batched CMA-ES kernels.
struct BatchTables {
    const CmaConst **k = nullptr;
    CmaState **st = nullptr;
    const double **y = nullptr;
    const float **params = nullptr, **loss = nullptr;
    const float **joint = nullptr;   // joint readings for the reset, entries may be NULL; NULL table = none
    float **pose = nullptr;          // frame estimates written by the epilogue
    int *ninst = nullptr;
};
// op 0 reset from the estimate, 1 update, 2 frame epilogue, 3 update without
// the square roots (a frame's last generation), 4 update where a selected
// entry with kSelNoSqrt set leaves them out; one block per selected instance
// (sel[n] device indices, or NULL for instances 0..n-1)
constexpr int kSelNoSqrt = 1 << 30;
cudaError_t launch_cma_batch(int op, int n, const int *sel, const BatchTables &t, cudaStream_t s);

static_assert(sizeof(EvalArgs) % 16 == 0, "batched launches copy EvalArgs in 16-byte pieces");

}  // namespace trk

// Objects behind the opaque handles of the C ABI.
struct trk_tracker {
    int device = 0;
    trk::ChainDev ch{};
    trk::CamDev cam{};
    trk_config cfg{};
    int V = 0, T = 0, d = 0;
    float4 *verts = nullptr;
    int4 *tris = nullptr;
    int4 *prims = nullptr;     // the mesh as quadrilateral pairs and single triangles (EvalArgs::prims)
    int P = 0;
    int2 *snap = nullptr;       // scratch [lambda_max * n_inst * V]
    int raster = 0;             // TRK_RASTER_CLUSTER or TRK_RASTER_BINNED (resolved at create)
    trk::BinDev bin{};          // binned pipeline scratch (raster == TRK_RASTER_BINNED)
    trk::LaunchCfg lc_front{};  // launch shape of the binned front kernel
    uint32_t *zero_mask = nullptr;
    unsigned *err = nullptr;    // device error word (TRK_DEVERR_* bits)
    trk::LaunchCfg lc{};
    void *soft = nullptr;       // soft-silhouette scratch, allocated on first use
    // keypoint term (tracker_set_keypoints / tracker_set_keypoint_obs)
    int kp_frame[2] = {0, 0};
    float kp_pt[2][3] = {{0, 0, 0}, {0, 0, 0}};
    float kp_tau = 0.0f, kp_lambda = 0.0f;
    const float *kp_obs = nullptr;
};

// The tracker's mesh into a launch's arguments: vertices, triangles and the
// primitive records the fitness kernel draws.
inline void apply_mesh(trk::EvalArgs &a, const trk_tracker *t)
{
    a.verts = t->verts;
    a.tris = t->tris;
    a.V = t->V;
    a.T = t->T;
    a.prims = t->prims;
    a.P = t->P;
}

// The tracker's keypoint term into a launch's arguments.
inline void apply_keypoints(trk::EvalArgs &a, const trk_tracker *t)
{
    a.err = t->err;
    for (int k = 0; k < 2; ++k) {
        a.kp_frame[k] = t->kp_frame[k];
        for (int j = 0; j < 3; ++j) a.kp_pt[k][j] = t->kp_pt[k][j];
    }
    a.kp_tau = t->kp_tau;
    a.kp_lambda = t->kp_lambda;
    a.kp_obs = t->kp_obs;
}

struct trk_cmaes {
    trk_tracker *t = nullptr;
    trk::CmaConst hk{};
    trk::CmaConst *k = nullptr;      // device copy
    trk::CmaState *st = nullptr;
    double *y = nullptr;        // [lam*d]
    double *z = nullptr;        // [lam*d] normals of the last population
    float *params = nullptr;    // [lam*d]
    float *loss = nullptr;      // [lam]
    double *mean0 = nullptr;    // [d] creation mean (physical)
    uint8_t *mask_bytes = nullptr;
    uint32_t *mask_packed = nullptr;
    float *joint = nullptr;     // [3*n_inst]
    float *pose = nullptr;      // [d]
    unsigned *done = nullptr;   // CTA ticket counter of the fused generation kernel
    void *refine = nullptr;     // gradient-refinement buffers, allocated on first use
    int lam = 0, d = 0;
    // the last update left out the square roots (a frame's last generation):
    // work that samples or updates again without a reset runs them first
    bool sqrt_pending = false;
};

namespace trk {
void soft_free(trk_tracker *t);      // releases trk_tracker::soft
void refine_free(trk_cmaes *es);     // releases trk_cmaes::refine
}  // namespace trk


