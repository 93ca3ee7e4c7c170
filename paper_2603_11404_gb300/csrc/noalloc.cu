// Allocation-free fitness evaluation: eval_population_noalloc (include/tracker.h).
//
// Some callers cannot allocate device memory at the point where they evaluate
// a population: code that runs under a memory pool or arena owned by another
// framework (which forbids cudaMalloc behind its back), real-time control
// loops that must not take the allocator's locks or risk its latency, and
// embedded hosts that only hand out pre-registered buffers.  This entry point
// serves them: the caller passes every input and output as device memory it
// already owns, and the one piece of scratch the fitness kernel needs (the
// snapped screen coordinates of every vertex of every candidate) lives in a
// fixed, file-scope device array that is part of the loaded library.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "internal.cuh"

using namespace trk;

namespace {

// The scratch array.  Every GPU that loads this library keeps it (16 MiB)
// until the process exits.  All calls share it: calls whose kernels overlap on
// the GPU (different streams, or different host threads) race on it.
static __device__ __align__(256) int2 g_noalloc_snap[TRK_NOALLOC_MAX_SNAP];

trk_status fail(trk_status s, const char *why)
{
    set_last_error(why);  // reported by tracker_last_error()
    return s;
}

// The array's device address on the current device.  Host code cannot use the
// array's name as an address, so every call asks the runtime (a host-side
// lookup that allocates nothing; looking it up each time keeps it right after
// the device's context is reset or recreated).
trk_status scratch_address(int2 **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_snap);
    if (e != cudaSuccess) return fail(TRK_ECUDA, cudaGetErrorString(e));
    *out = static_cast<int2 *>(p);
    return TRK_OK;
}

}  // namespace

extern "C" {

trk_status eval_population_noalloc(const float *verts_dev, int32_t n_verts, const int32_t *tris_dev, int32_t n_tris,
                                   const trk_chain *chain, const trk_intrinsics *K, const trk_config *cfg,
                                   const float *params_dev, int32_t lam, const uint32_t *mask_packed_dev,
                                   float *loss_dev, int32_t *counts_dev, void *stream)
{
    if (!chain || !K || !cfg) return fail(TRK_EINVAL, "NULL chain, intrinsics or config");
    if (lam < 0 || lam > 65535) return fail(TRK_EINVAL, "lam out of range (0..65535)");
    if (lam == 0) return TRK_OK;
    if (!verts_dev || !tris_dev || !params_dev || !mask_packed_dev || n_verts <= 0 || n_tris < 0)
        return fail(TRK_EINVAL, "NULL device pointer or empty mesh");
    if (n_verts > (1 << 24) || n_tris > (1 << 24)) return fail(TRK_EINVAL, "mesh too large");
    if (chain->n_frames <= 0 || chain->n_frames > TRK_MAX_FRAMES) return fail(TRK_EINVAL, "n_frames out of range");
    if (chain->n_instruments < 1 || chain->n_instruments > TRK_MAX_INSTRUMENTS)
        return fail(TRK_EINVAL, "n_instruments must be 1 or 2");
    if (chain->rot_param != TRK_ROT_AXIS_ANGLE && chain->rot_param != TRK_ROT_LOOKAT)
        return fail(TRK_EINVAL, "rot_param");
    for (int f = 0; f < chain->n_frames; ++f) {
        if (chain->parent[f] >= f || chain->parent[f] < -1 || chain->axis[f] < 0 || chain->axis[f] > 3 ||
            chain->joint[f] < 0 || chain->joint[f] > 2)
            return fail(TRK_EINVAL, "chain frame fields");
        for (int k = 0; k < 3; ++k)
            if (!isfinite(chain->offset[f][k])) return fail(TRK_EINVAL, "offset not finite");
        if (!isfinite(chain->coef[f])) return fail(TRK_EINVAL, "coef not finite");
    }
    for (int i = 0; i < 3; ++i)
        if (!(chain->q_lb[i] <= chain->q_ub[i]) || !isfinite(chain->q_lb[i]) || !isfinite(chain->q_ub[i]))
            return fail(TRK_EINVAL, "joint limits");
    if (K->width <= 0 || K->height <= 0 || (long long)K->width * K->height > TRK_MAX_PIXELS)
        return fail(TRK_EINVAL, "image size out of range");
    if (!(K->fx > 0) || !(K->fy > 0) || !isfinite(K->fx) || !isfinite(K->fy)) return fail(TRK_EINVAL, "focal length");
    if (!(K->z_near > 0) || !isfinite(K->z_near)) return fail(TRK_EINVAL, "z_near");
    const double cx256 = K->cx * 256.0, cy256 = K->cy * 256.0;
    if (cx256 != floor(cx256) || cy256 != floor(cy256) || fabs(cx256) > (1 << 22) || fabs(cy256) > (1 << 22))
        return fail(TRK_EINVAL, "256*cx and 256*cy must be integers");
    if (cfg->loss_kind < 0 || cfg->loss_kind > 2) return fail(TRK_EINVAL, "loss_kind");
    if (cfg->cluster < 0 || cfg->cluster > 8) return fail(TRK_EINVAL, "cluster must be 0..8");
    if (cfg->block_threads < 0 || cfg->block_threads > 256 || cfg->block_threads % 32 ||
        (cfg->block_threads > 0 && cfg->block_threads < 32 * chain->n_instruments))
        return fail(TRK_EINVAL, "block_threads");
    const long long need = (long long)lam * chain->n_instruments * n_verts;
    if (need > TRK_NOALLOC_MAX_SNAP)
        return fail(TRK_EINVAL, "lam * n_instruments * n_verts exceeds TRK_NOALLOC_MAX_SNAP (the static scratch)");

    int2 *scratch = nullptr;
    trk_status st = scratch_address(&scratch);
    if (st != TRK_OK) return st;

    EvalArgs a{};
    ChainDev &ch = a.ch;
    ch.n_frames = chain->n_frames;
    ch.n_inst = chain->n_instruments;
    ch.rot_param = chain->rot_param;
    for (int f = 0; f < chain->n_frames; ++f) {
        ch.parent[f] = chain->parent[f];
        ch.axis[f] = chain->axis[f];
        ch.joint[f] = chain->joint[f];
        ch.coef[f] = chain->coef[f];
        ch.coef_df[f] = split_df(chain->coef[f]);
        for (int k = 0; k < 3; ++k) {
            ch.offset[f][k] = chain->offset[f][k];
            ch.offset_df[f][k] = split_df(chain->offset[f][k]);
        }
    }
    for (int i = 0; i < 3; ++i) {
        double range = chain->q_ub[i] - chain->q_lb[i];
        ch.q_lb[i] = chain->q_lb[i];
        ch.q_ub[i] = chain->q_ub[i];
        ch.lb_df[i] = split_df(chain->q_lb[i]);
        ch.half_range_df[i] = split_df(0.5 * range);
        ch.pi_over_range_df[i] = split_df(range > 0 ? M_PI / range : 0.0);
    }
    CamDev &cam = a.cam;
    cam.fx = K->fx;
    cam.fy = K->fy;
    cam.z_near = K->z_near;
    cam.guard = kGuardPx;
    cam.W = K->width;
    cam.H = K->height;
    cam.Wq = (K->width + 31) / 32;
    cam.cx256 = (int)cx256;
    cam.cy256 = (int)cy256;
    cam.fx_df = split_df(K->fx);
    cam.fy_df = split_df(K->fy);
    a.verts = reinterpret_cast<const float4 *>(verts_dev);
    a.tris = reinterpret_cast<const int4 *>(tris_dev);
    a.V = n_verts;
    a.T = n_tris;
    a.params = params_dev;
    a.d = 9 * chain->n_instruments;
    a.lam = lam;
    a.mask = mask_packed_dev;
    a.snap = scratch;  // fully overwritten by every call before it is read
    a.loss = loss_dev;
    a.counts = counts_dev;
    a.loss_kind = cfg->loss_kind;
    a.lambda_app = cfg->lambda_app;
    a.cull = cfg->cull_backfaces;

    LaunchCfg lc;
    lc.threads = cfg->block_threads > 0 ? cfg->block_threads : 256;
    if (cfg->cluster > 0) {
        lc.cluster = cfg->cluster;
    } else {
        long long work = (long long)(n_verts + n_tris) * chain->n_instruments;
        long long per_cta = (long long)lc.threads * 2;
        lc.cluster = (int)std::min<long long>(8, std::max<long long>(1, (work + per_cta - 1) / per_cta));
    }
    lc.smem = eval_smem_bytes(a);
    if (lc.smem > 227 * 1024) return fail(TRK_EINVAL, "image too large for the shared-memory bitmap");
    // the index-checked kernel: the mesh is in the caller's device memory; its
    // dynamic shared-memory limit is a kernel attribute, not an allocation
    cudaError_t e = launch_eval_checked(a, lc, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail(TRK_ECUDA, cudaGetErrorString(e));
    return TRK_OK;
}

}  // extern "C"
