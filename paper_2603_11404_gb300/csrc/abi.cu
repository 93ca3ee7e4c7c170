// C ABI of the tracker library (declared in include/tracker.h): validation,
// device allocation and the host-side sequencing of the kernels in raster.cu
// and cmaes.cu.  All compute runs in those kernels; nothing here touches the
// data on the host beyond validation and the copies the caller asks for.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace trk;

namespace {

thread_local std::string g_last_error;

trk_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return TRK_ECUDA;
}

trk_status inval(const char *why)
{
    g_last_error = why;
    return TRK_EINVAL;
}

#define CU(call, what)                                  \
    do {                                                \
        cudaError_t _e = (call);                        \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

void trk::set_last_error(const char *msg) { g_last_error = msg; }

extern "C" {

const char *trk_status_string(trk_status s)
{
    switch (s) {
    case TRK_OK: return "ok";
    case TRK_EINVAL: return "invalid argument";
    case TRK_ENOMEM: return "out of memory";
    case TRK_ECUDA: return "CUDA error";
    case TRK_EDEVICE: return "device error";
    case TRK_EBUSY: return "busy";
    }
    return "unknown status";
}

const char *tracker_last_error(void) { return g_last_error.c_str(); }

static void binned_free(BinDev &b)
{
    cudaFree(b.frames);
    cudaFree(b.pool);
    cudaFree(b.items);
    cudaFree(b.merge);
    cudaFree(b.tile_done);
    cudaFree(b.acc);
    cudaFree(b.ctl);
    b = BinDev{};
}

// The mesh as primitives for the fitness kernel: triangles that share an edge
// with opposite directions (a consistently wound pair) become one record
// (a, b, c, d) for the triangles (a, b, c) and (a, c, d); the rest stay single
// (a, b, c, -1).  Greedy in mesh order: each triangle not yet taken pairs with
// the first later free triangle across one of its edges, so the records keep
// the mesh's order (neighbouring records draw neighbouring pixels).  Whether a
// pair is drawn as one quadrilateral is decided per candidate on the device
// (convexity of the projected corners); the union of pixels is the same.
static std::vector<int4> pair_triangles(const std::vector<int4> &tris, long long T)
{
    struct DirEdge {
        int u, v, t;
    };
    std::vector<DirEdge> edges;
    edges.reserve((size_t)(3 * T));
    for (int t = 0; t < (int)T; ++t) {
        const int4 &r = tris[t];
        edges.push_back({r.x, r.y, t});
        edges.push_back({r.y, r.z, t});
        edges.push_back({r.z, r.x, t});
    }
    auto key_less = [](const DirEdge &a, const DirEdge &b) {
        return a.u != b.u ? a.u < b.u : (a.v != b.v ? a.v < b.v : a.t < b.t);
    };
    std::sort(edges.begin(), edges.end(), key_less);
    std::vector<char> taken((size_t)std::max<long long>(T, 1), 0);
    std::vector<int4> prims;
    prims.reserve((size_t)T);
    for (int t = 0; t < (int)T; ++t) {
        if (taken[t]) continue;
        taken[t] = 1;
        const int c[3] = {tris[t].x, tris[t].y, tris[t].z};
        int best = -1, best_k = 0;
        for (int k = 0; k < 3; ++k) {
            const int u = c[k], v = c[(k + 1) % 3];
            // triangles holding the reverse edge v -> u
            auto it = std::lower_bound(edges.begin(), edges.end(), DirEdge{v, u, 0}, key_less);
            for (; it != edges.end() && it->u == v && it->v == u; ++it) {
                const int o = it->t;
                if (taken[o] || (best >= 0 && o >= best)) continue;
                const int4 &r = tris[o];
                const int w = r.x + r.y + r.z - u - v;  // the other triangle's third corner
                if (w == c[0] || w == c[1] || w == c[2]) continue;  // a folded duplicate, not a pair
                best = o;
                best_k = k;
            }
        }
        if (best < 0) {
            prims.push_back(make_int4(c[0], c[1], c[2], -1));
            continue;
        }
        taken[best] = 1;
        // shared edge c[k] -> c[k+1]: rotate so that it is the closing edge c -> a
        const int a0 = c[(best_k + 1) % 3], b0 = c[(best_k + 2) % 3], c0 = c[best_k];
        const int4 &r = tris[best];
        const int d0 = r.x + r.y + r.z - a0 - c0;
        prims.push_back(make_int4(a0, b0, c0, d0));
    }
    return prims;
}

static void tracker_free(trk_tracker *t)
{
    if (!t) return;
    cudaFree(t->verts);
    cudaFree(t->tris);
    cudaFree(t->prims);
    cudaFree(t->snap);
    cudaFree(t->zero_mask);
    cudaFree(t->err);
    binned_free(t->bin);
    soft_free(t);
    delete t;
}

static LaunchCfg auto_launch(const trk_tracker *t, const EvalArgs &a)
{
    LaunchCfg lc;
    lc.threads = t->cfg.block_threads > 0 ? t->cfg.block_threads : 256;
    if (t->cfg.cluster > 0) {
        lc.cluster = t->cfg.cluster;
    } else {
        // about 2 work items (vertices + triangles) per thread, at most 8 CTAs
        // (2048 threads) per candidate: the kernel is latency-bound, so more
        // threads per candidate help until the cluster barriers dominate
        long long work = (long long)(t->V + t->T) * t->ch.n_inst;
        long long per_cta = (long long)lc.threads * 2;
        lc.cluster = (int)std::min<long long>(8, std::max<long long>(1, (work + per_cta - 1) / per_cta));
    }
    lc.smem = eval_smem_bytes(a);
    return lc;
}

// Binned pipeline layout for tracker t (front launch shape from auto_launch).
// Returns false when the image or the mesh is too large for it.
static bool binned_layout(trk_tracker *t, const EvalArgs &probe)
{
    BinDev &b = t->bin;
    b.n_tx = (t->cam.W + kTileW - 1) / kTileW;
    b.n_ty = (t->cam.H + kTileH - 1) / kTileH;
    if (b.n_tx > kBinMaxTilesPerAxis || b.n_ty > kBinMaxTilesPerAxis) return false;
    b.n_tiles = b.n_tx * b.n_ty;
    const long long NT = (long long)t->T * t->ch.n_inst;
    const long long per_launch = (long long)t->lc_front.cluster * t->lc_front.threads;
    b.live_cap = (int)(((NT + per_launch - 1) / per_launch) * t->lc_front.threads);
    // the bins of one candidate: every live triangle once per tile its box
    // touches (about 0.6 entries per triangle at 640 x 512), with room for two
    // entries per triangle; more than that draws the candidate's tiles from
    // every triangle instead
    const long long pool = 2 * NT + 8192;
    const long long items = pool / kBinChunk + b.n_tiles + 1;
    if (pool > (1LL << 28) || items * t->cfg.lambda_max > (1LL << 30)) return false;
    b.pool_cap = (int)pool;
    b.max_items = (int)(items * t->cfg.lambda_max);
    EvalArgs a = probe;
    a.bin = b;
    t->lc_front.smem = binned_front_smem_bytes(a, t->lc_front.threads);
    return t->lc_front.smem <= 227 * 1024;
}

static cudaError_t binned_alloc(trk_tracker *t)
{
    BinDev &b = t->bin;
    const size_t lam = (size_t)t->cfg.lambda_max, nT = (size_t)b.n_tiles;
    cudaError_t e;
    if ((e = cudaMalloc(&b.frames, lam * t->ch.n_inst * t->ch.n_frames * 24 * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&b.pool, lam * b.pool_cap * 3 * sizeof(int2))) != cudaSuccess ||
        (e = cudaMalloc(&b.items, (size_t)b.max_items * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc(&b.merge, lam * nT * kTileWords * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMalloc(&b.tile_done, lam * nT * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&b.acc, lam * 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&b.ctl, 4 * sizeof(unsigned))) != cudaSuccess)
        return e;
    if ((e = cudaMemset(b.merge, 0, lam * nT * kTileWords * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset(b.tile_done, 0, lam * nT * sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(b.ctl, 0, 4 * sizeof(unsigned))) != cudaSuccess)
        return e;
    int per_sm = 0, n_sm = 0;
    if ((e = prepare_binned(t->lc_front.smem, &per_sm)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, t->device)) != cudaSuccess)
        return e;
    b.tiles_grid = std::max(1, per_sm) * std::max(1, n_sm);
    return cudaSuccess;
}

trk_status tracker_create(const trk_link_mesh *meshes, int32_t n_meshes, const trk_chain *chain,
                          const trk_intrinsics *K, const trk_config *cfg, trk_tracker **out)
{
    if (!out) return inval("out is NULL");
    *out = nullptr;
    if (!meshes || n_meshes <= 0 || !chain || !K || !cfg) return inval("NULL argument");
    if (chain->n_frames <= 0 || chain->n_frames > TRK_MAX_FRAMES) return inval("n_frames out of range");
    if (chain->n_instruments < 1 || chain->n_instruments > TRK_MAX_INSTRUMENTS)
        return inval("n_instruments must be 1 or 2");
    if (chain->rot_param != TRK_ROT_AXIS_ANGLE && chain->rot_param != TRK_ROT_LOOKAT)
        return inval("rot_param");
    for (int f = 0; f < chain->n_frames; ++f) {
        if (chain->parent[f] >= f || chain->parent[f] < -1) return inval("parent must precede child");
        if (chain->axis[f] < 0 || chain->axis[f] > 3) return inval("axis");
        if (chain->joint[f] < 0 || chain->joint[f] > 2) return inval("joint");
        for (int k = 0; k < 3; ++k)
            if (!isfinite(chain->offset[f][k])) return inval("offset not finite");
        if (!isfinite(chain->coef[f])) return inval("coef not finite");
    }
    for (int i = 0; i < 3; ++i)
        if (!(chain->q_lb[i] <= chain->q_ub[i]) || !isfinite(chain->q_lb[i]) || !isfinite(chain->q_ub[i]))
            return inval("joint limits");
    if (K->width <= 0 || K->height <= 0 || (long long)K->width * K->height > TRK_MAX_PIXELS)
        return inval("image size out of range");
    if (!(K->fx > 0) || !(K->fy > 0) || !isfinite(K->fx) || !isfinite(K->fy)) return inval("focal length");
    if (!(K->z_near > 0) || !isfinite(K->z_near)) return inval("z_near");
    double cx256 = K->cx * 256.0, cy256 = K->cy * 256.0;
    if (cx256 != floor(cx256) || cy256 != floor(cy256) || fabs(cx256) > (1 << 22) || fabs(cy256) > (1 << 22))
        return inval("256*cx and 256*cy must be integers");
    if (cfg->loss_kind < 0 || cfg->loss_kind > 2) return inval("loss_kind");
    if (cfg->lambda_max < 1 || cfg->lambda_max > 65535) return inval("lambda_max out of range");
    if (cfg->cluster < 0 || cfg->cluster > 8) return inval("cluster must be 0..8");
    if (cfg->block_threads < 0 || cfg->block_threads > 256 || cfg->block_threads % 32 ||
        (cfg->block_threads > 0 && cfg->block_threads < 32 * chain->n_instruments))
        return inval("block_threads: multiple of 32, at least 32 per instrument, at most 256");
    if (cfg->raster < TRK_RASTER_AUTO || cfg->raster > TRK_RASTER_BINNED) return inval("raster");

    long long V = 0, T = 0;
    for (int i = 0; i < n_meshes; ++i) {
        const trk_link_mesh &m = meshes[i];
        if (m.frame < 0 || m.frame >= chain->n_frames) return inval("mesh frame out of range");
        if (m.n_verts < 0 || m.n_tris < 0 || (m.n_verts && !m.verts) || (m.n_tris && !m.tris))
            return inval("mesh arrays");
        for (long long j = 0; j < 3LL * m.n_tris; ++j)
            if (m.tris[j] < 0 || m.tris[j] >= m.n_verts) return inval("triangle index out of range");
        for (long long j = 0; j < 3LL * m.n_verts; ++j)
            if (!isfinite(m.verts[j])) return inval("vertex not finite");
        V += m.n_verts;
        T += m.n_tris;
    }
    if (V > (1 << 24) || T > (1 << 24)) return inval("mesh too large");

    trk_tracker *t = new (std::nothrow) trk_tracker();
    if (!t) return TRK_ENOMEM;
    cudaError_t e = cudaGetDevice(&t->device);
    if (e != cudaSuccess) {
        delete t;
        return cuda_fail(e, "cudaGetDevice");
    }
    t->cfg = *cfg;
    t->V = (int)V;
    t->T = (int)T;
    t->d = 9 * chain->n_instruments;
    ChainDev &ch = t->ch;
    ch.n_frames = chain->n_frames;
    ch.n_inst = chain->n_instruments;
    ch.rot_param = chain->rot_param;
    for (int f = 0; f < chain->n_frames; ++f) {
        ch.parent[f] = chain->parent[f];
        ch.axis[f] = chain->axis[f];
        ch.joint[f] = chain->joint[f];
        ch.coef[f] = chain->coef[f];
        for (int k = 0; k < 3; ++k) ch.offset[f][k] = chain->offset[f][k];
    }
    for (int i = 0; i < 3; ++i) {
        ch.q_lb[i] = chain->q_lb[i];
        ch.q_ub[i] = chain->q_ub[i];
        double range = chain->q_ub[i] - chain->q_lb[i];
        ch.lb_df[i] = split_df(chain->q_lb[i]);
        ch.half_range_df[i] = split_df(0.5 * range);
        ch.pi_over_range_df[i] = split_df(range > 0 ? M_PI / range : 0.0);
    }
    for (int f = 0; f < chain->n_frames; ++f) {
        ch.coef_df[f] = split_df(chain->coef[f]);
        for (int k = 0; k < 3; ++k) ch.offset_df[f][k] = split_df(chain->offset[f][k]);
    }
    CamDev &cam = t->cam;
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

    std::vector<float4> hv(std::max<long long>(V, 1));
    std::vector<int4> ht(std::max<long long>(T, 1));
    long long vb = 0, tb = 0;
    for (int i = 0; i < n_meshes; ++i) {
        const trk_link_mesh &m = meshes[i];
        for (int j = 0; j < m.n_verts; ++j)
            hv[vb + j] = make_float4(m.verts[3 * j], m.verts[3 * j + 1], m.verts[3 * j + 2], (float)m.frame);
        for (int j = 0; j < m.n_tris; ++j)
            ht[tb + j] = make_int4((int)(m.tris[3 * j] + vb), (int)(m.tris[3 * j + 1] + vb),
                                   (int)(m.tris[3 * j + 2] + vb), 0);
        vb += m.n_verts;
        tb += m.n_tris;
    }
    std::vector<int4> hp = pair_triangles(ht, T);
    // draw order: the reverse of the mesh's.  Instrument meshes list the links
    // from the shaft to the jaws and the shaft from its far end, so the tip
    // (the largest primitives on screen) is drawn first and the small far end
    // is left for when the cluster's warps run out of work.  Within a link
    // neighbouring primitives stay together, so a chunk's 32 lanes draw
    // primitives of similar size.  Any order gives the same union.
    std::reverse(hp.begin(), hp.end());
    t->P = (int)hp.size();
    if (hp.empty()) hp.push_back(make_int4(0, 0, 0, -1));
    size_t snap_elems = (size_t)cfg->lambda_max * ch.n_inst * std::max<long long>(V, 1);
    if ((e = cudaMalloc(&t->verts, hv.size() * sizeof(float4))) != cudaSuccess ||
        (e = cudaMalloc(&t->tris, ht.size() * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc(&t->prims, hp.size() * sizeof(int4))) != cudaSuccess ||
        (e = cudaMalloc(&t->snap, snap_elems * sizeof(int2))) != cudaSuccess ||
        (e = cudaMalloc(&t->zero_mask, (size_t)cam.H * cam.Wq * 4)) != cudaSuccess ||
        (e = cudaMalloc(&t->err, sizeof(unsigned))) != cudaSuccess) {
        tracker_free(t);
        g_last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA;
    }
    if ((e = cudaMemcpy(t->verts, hv.data(), hv.size() * sizeof(float4), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(t->tris, ht.data(), ht.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(t->prims, hp.data(), hp.size() * sizeof(int4), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(t->zero_mask, 0, (size_t)cam.H * cam.Wq * 4)) != cudaSuccess ||
        (e = cudaMemset(t->err, 0, sizeof(unsigned))) != cudaSuccess) {
        tracker_free(t);
        return cuda_fail(e, "tracker upload");
    }
    EvalArgs probe{};
    probe.ch = t->ch;
    probe.cam = t->cam;
    t->lc = auto_launch(t, probe);
    t->lc_front = t->lc;
    const bool binned_ok = binned_layout(t, probe);
    if (cfg->raster == TRK_RASTER_BINNED && !binned_ok) {
        tracker_free(t);
        return inval("image or mesh too large for the binned rasteriser");
    }
    // AUTO takes the cluster-bitmap kernel, the faster of the two on every
    // workload measured (640 x 512, 20k triangles, 64 candidates: 43 us against
    // 72.5 us), and the binned form only for an image whose bitmap does not fit
    // one CTA's shared memory
    const bool cluster_fits = t->lc.smem <= 227 * 1024;
    if (cfg->raster == TRK_RASTER_BINNED)
        t->raster = TRK_RASTER_BINNED;
    else if (cfg->raster == TRK_RASTER_CLUSTER || cluster_fits || !binned_ok)
        t->raster = TRK_RASTER_CLUSTER;
    else
        t->raster = TRK_RASTER_BINNED;
    if (t->raster == TRK_RASTER_BINNED) {
        if ((e = binned_alloc(t)) != cudaSuccess) {
            tracker_free(t);
            g_last_error = std::string("binned rasteriser set-up: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA;
        }
    } else {
        t->bin = BinDev{};
    }
    // the cluster-bitmap kernel also serves batches, servers and images the
    // binned form cannot take: it needs its full-image bitmap in shared memory
    if (t->lc.smem > 227 * 1024) {
        if (t->raster == TRK_RASTER_CLUSTER) {
            tracker_free(t);
            return inval("image too large for the shared-memory bitmap");
        }
    } else if ((e = prepare_eval(t->lc.smem)) != cudaSuccess) {
        tracker_free(t);
        return cuda_fail(e, "eval kernel attributes");
    }
    *out = t;
    return TRK_OK;
}

trk_status tracker_set_keypoints(trk_tracker *t, const trk_keypoints *kp)
{
    if (!t || !kp) return inval("NULL argument");
    for (int k = 0; k < 2; ++k)
        if (kp->frame[k] < 0 || kp->frame[k] >= t->ch.n_frames) return inval("keypoint frame out of range");
    if (!(kp->tau >= 0.0) || !(kp->lambda_kpts >= 0.0)) return inval("tau and lambda_kpts must be >= 0");
    for (int k = 0; k < 2; ++k) {
        t->kp_frame[k] = kp->frame[k];
        for (int j = 0; j < 3; ++j) t->kp_pt[k][j] = (float)kp->point[k][j];
    }
    t->kp_tau = (float)kp->tau;
    t->kp_lambda = (float)kp->lambda_kpts;
    return TRK_OK;
}

trk_status tracker_set_keypoint_obs(trk_tracker *t, const float *obs_dev)
{
    if (!t) return inval("NULL tracker");
    t->kp_obs = obs_dev;
    return TRK_OK;
}

trk_status tracker_project_keypoints(trk_tracker *t, const float *states_dev, int32_t n, float *out_dev, void *stream)
{
    if (!t) return inval("NULL tracker");
    if (n < 0) return inval("n < 0");
    if (n == 0) return TRK_OK;
    if (!states_dev || !out_dev) return inval("NULL device pointer");
    EvalArgs a{};
    a.ch = t->ch;
    a.cam = t->cam;
    a.d = t->d;
    apply_keypoints(a, t);
    CU(launch_project_keypoints(a, states_dev, n, out_dev, as_stream(stream)), "project keypoints");
    return TRK_OK;
}

trk_status tracker_destroy(trk_tracker *t)
{
    if (!t) return inval("NULL tracker");
    tracker_free(t);
    return TRK_OK;
}

trk_status tracker_get_error(trk_tracker *t, uint32_t *device_code, void *stream)
{
    if (!t) return inval("NULL tracker");
    cudaStream_t s = as_stream(stream);
    unsigned w = 0;
    CU(cudaMemcpyAsync(&w, t->err, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "error word copy");
    CU(cudaMemsetAsync(t->err, 0, sizeof(unsigned), s), "error word clear");
    CU(cudaStreamSynchronize(s), "error word sync");
    if (device_code) *device_code = w;
    if (w & TRK_DEVERR_WORKLIST) {
        g_last_error = "device error word: the binned rasteriser's work list overflowed";
        return TRK_EDEVICE;
    }
    return TRK_OK;
}

trk_status tracker_info(const trk_tracker *t, int32_t *d, int32_t *n_verts, int32_t *n_tris, int32_t *width,
                        int32_t *height, int32_t *words_per_row)
{
    if (!t) return inval("NULL tracker");
    if (d) *d = t->d;
    if (n_verts) *n_verts = t->V;
    if (n_tris) *n_tris = t->T;
    if (width) *width = t->cam.W;
    if (height) *height = t->cam.H;
    if (words_per_row) *words_per_row = t->cam.Wq;
    return TRK_OK;
}

trk_status tracker_pack_mask(trk_tracker *t, const uint8_t *mask_dev, uint32_t *packed_dev, void *stream)
{
    if (!t || !mask_dev || !packed_dev) return inval("NULL argument");
    CU(launch_pack_mask(mask_dev, packed_dev, t->cam.W, t->cam.H, t->cam.Wq, as_stream(stream)), "pack_mask");
    return TRK_OK;
}

static trk_status eval_impl(trk_tracker *t, const float *params, int32_t lam, const uint32_t *mask, float *loss,
                            int32_t *counts, int32_t *snap_dbg, float *uv_dbg, uint32_t *sil, void *stream)
{
    if (!t) return inval("NULL tracker");
    if (lam < 0 || lam > t->cfg.lambda_max) return inval("lam out of range (0..lambda_max)");
    if (lam == 0) return TRK_OK;
    if (!params || !mask) return inval("NULL params or mask");
    EvalArgs a{};
    a.ch = t->ch;
    a.cam = t->cam;
    apply_mesh(a, t);
    a.params = params;
    a.d = t->d;
    a.lam = lam;
    a.mask = mask;
    a.snap = t->snap;
    a.loss = loss;
    a.counts = counts;
    a.snap_dbg = reinterpret_cast<int2 *>(snap_dbg);
    a.uv_dbg = reinterpret_cast<float2 *>(uv_dbg);
    a.silhouette = sil;
    a.loss_kind = t->cfg.loss_kind;
    a.lambda_app = t->cfg.lambda_app;
    a.cull = t->cfg.cull_backfaces;
    apply_keypoints(a, t);
    if (t->raster == TRK_RASTER_BINNED) {
        a.bin = t->bin;
        CU(launch_binned(a, t->lc_front, as_stream(stream)), "eval_population launch");
    } else {
        CU(launch_eval(a, t->lc, as_stream(stream)), "eval_population launch");
    }
    return TRK_OK;
}

trk_status eval_population(trk_tracker *t, const float *params_dev, int32_t lam, const uint32_t *mask_packed_dev,
                           float *loss_dev, int32_t *counts_dev, void *stream)
{
    return eval_impl(t, params_dev, lam, mask_packed_dev, loss_dev, counts_dev, nullptr, nullptr, nullptr, stream);
}

trk_status eval_population_debug(trk_tracker *t, const float *params_dev, int32_t lam,
                                 const uint32_t *mask_packed_dev, float *loss_dev, int32_t *counts_dev,
                                 int32_t *snap_dev, float *uv_dev, void *stream)
{
    return eval_impl(t, params_dev, lam, mask_packed_dev, loss_dev, counts_dev, snap_dev, uv_dev, nullptr, stream);
}

trk_status tracker_render(trk_tracker *t, const float *params_dev, uint32_t *silhouette_dev, void *stream)
{
    if (!t || !silhouette_dev) return inval("NULL argument");
    return eval_impl(t, params_dev, 1, t->zero_mask, nullptr, nullptr, nullptr, nullptr, silhouette_dev, stream);
}

// ---------------------------------------------------------------------------
// CMA-ES
// ---------------------------------------------------------------------------
static void cmaes_free(trk_cmaes *es)
{
    if (!es) return;
    cudaFree(es->k);
    cudaFree(es->st);
    cudaFree(es->y);
    cudaFree(es->z);
    cudaFree(es->params);
    cudaFree(es->loss);
    cudaFree(es->mean0);
    cudaFree(es->mask_bytes);
    cudaFree(es->mask_packed);
    cudaFree(es->joint);
    cudaFree(es->pose);
    cudaFree(es->done);
    refine_free(es);
    delete es;
}

// Hansen's CMA-ES tutorial defaults for dimension n and population lam.
static void default_constants(CmaConst &k, int n, int lam)
{
    k.d = n;
    k.lam = lam;
    k.mu = lam / 2;
    double sw = 0.0;
    for (int i = 0; i < k.mu; ++i) {
        k.w[i] = log((lam + 1) / 2.0) - log((double)(i + 1));
        sw += k.w[i];
    }
    double sw2 = 0.0;
    for (int i = 0; i < k.mu; ++i) {
        k.w[i] /= sw;
        sw2 += k.w[i] * k.w[i];
    }
    k.mu_eff = 1.0 / sw2;
    k.c_sigma = (k.mu_eff + 2.0) / (n + k.mu_eff + 5.0);
    k.d_sigma = 1.0 + 2.0 * std::max(0.0, sqrt((k.mu_eff - 1.0) / (n + 1.0)) - 1.0) + k.c_sigma;
    k.c_c = (4.0 + k.mu_eff / n) / (n + 4.0 + 2.0 * k.mu_eff / n);
    k.c_1 = 2.0 / ((n + 1.3) * (n + 1.3) + k.mu_eff);
    k.c_mu = std::min(1.0 - k.c_1, 2.0 * (k.mu_eff - 2.0 + 1.0 / k.mu_eff) / ((n + 2.0) * (n + 2.0) + k.mu_eff));
    k.c_m = 1.0;
    k.chi_n = sqrt((double)n) * (1.0 - 1.0 / (4.0 * n) + 1.0 / (21.0 * n * n));
    k.ps_coef = sqrt(k.c_sigma * (2.0 - k.c_sigma) * k.mu_eff);
    k.pc_coef = sqrt(k.c_c * (2.0 - k.c_c) * k.mu_eff);
    double thr = (1.4 + 2.0 / (n + 1)) * k.chi_n;
    k.hs_thr2 = thr * thr;
    k.cs_over_ds = k.c_sigma / k.d_sigma;
    k.inv_chi = 1.0 / k.chi_n;
}

trk_status cmaes_create(trk_tracker *t, int32_t lam, const double *mean_host, const double *scales_host,
                        double sigma0, uint64_t seed, uint32_t stream_id, int32_t block_diag, trk_cmaes **out)
{
    if (!out) return inval("out is NULL");
    *out = nullptr;
    if (!t || !mean_host || !scales_host) return inval("NULL argument");
    if (lam < 2 || lam > TRK_MAX_LAMBDA || lam > t->cfg.lambda_max) return inval("lam out of range");
    if (!(sigma0 > 0) || !isfinite(sigma0)) return inval("sigma0");
    const int d = t->d;
    for (int i = 0; i < d; ++i)
        if (!(scales_host[i] > 0) || !isfinite(scales_host[i]) || !isfinite(mean_host[i]))
            return inval("mean/scales");
    if (block_diag && d % 9) return inval("block_diag needs d multiple of 9");
    trk_cmaes *es = new (std::nothrow) trk_cmaes();
    if (!es) return TRK_ENOMEM;
    es->t = t;
    es->lam = lam;
    es->d = d;
    CmaConst &k = es->hk;
    default_constants(k, d, lam);
    k.block = block_diag ? 9 : 0;
    k.sigma0 = sigma0;
    for (int i = 0; i < d; ++i) {
        k.scales[i] = scales_host[i];
        k.scales_df[i] = split_df(scales_host[i]);
    }
    for (int i = 0; i < 3; ++i) {
        k.q_lb[i] = t->ch.q_lb[i];
        k.q_ub[i] = t->ch.q_ub[i];
    }
    k.seed = seed;
    k.stream_id = stream_id;
    const int H = t->cam.H, W = t->cam.W, Wq = t->cam.Wq;
    cudaError_t e;
    if ((e = cudaMalloc(&es->k, sizeof(CmaConst))) != cudaSuccess ||
        (e = cudaMalloc(&es->st, sizeof(CmaState))) != cudaSuccess ||
        (e = cudaMalloc(&es->y, sizeof(double) * lam * d)) != cudaSuccess ||
        (e = cudaMalloc(&es->z, sizeof(double) * lam * d)) != cudaSuccess ||
        (e = cudaMalloc(&es->params, sizeof(float) * lam * d)) != cudaSuccess ||
        (e = cudaMalloc(&es->loss, sizeof(float) * lam)) != cudaSuccess ||
        (e = cudaMalloc(&es->mean0, sizeof(double) * d)) != cudaSuccess ||
        (e = cudaMalloc(&es->mask_bytes, (size_t)H * W)) != cudaSuccess ||
        (e = cudaMalloc(&es->mask_packed, (size_t)H * Wq * 4)) != cudaSuccess ||
        (e = cudaMalloc(&es->joint, sizeof(float) * 3 * TRK_MAX_INSTRUMENTS)) != cudaSuccess ||
        (e = cudaMalloc(&es->pose, sizeof(float) * d)) != cudaSuccess ||
        (e = cudaMalloc(&es->done, sizeof(unsigned))) != cudaSuccess) {
        cmaes_free(es);
        g_last_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA;
    }
    CmaState zero{};
    zero.gen_total = 0;
    if ((e = cudaMemcpy(es->k, &k, sizeof(CmaConst), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(es->st, &zero, sizeof(CmaState), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(es->mean0, mean_host, sizeof(double) * d, cudaMemcpyHostToDevice)) != cudaSuccess) {
        cmaes_free(es);
        return cuda_fail(e, "cmaes upload");
    }
    if ((e = cudaMemset(es->done, 0, sizeof(unsigned))) != cudaSuccess ||
        (t->raster == TRK_RASTER_CLUSTER && (e = prepare_eval(std::max(t->lc.smem, tell_smem_bytes()))) != cudaSuccess) ||
        (e = launch_cma_reset(es->k, es->st, es->mean0, false, nullptr, t->ch.n_inst, 0)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        cmaes_free(es);
        return cuda_fail(e, "cmaes reset");
    }
    *out = es;
    return TRK_OK;
}

trk_status cmaes_set_filter(trk_cmaes *es, const trk_filter *f, void *stream)
{
    if (!es || !f) return inval("NULL argument");
    const int d = es->d;
    if (f->enabled) {
        if (!(f->dt > 0.0)) return inval("filter dt must be > 0");
        for (int i = 0; i < d; ++i)
            if (!(f->q_pos[i] >= 0.0) || !(f->q_vel[i] >= 0.0) || !(f->r[i] > 0.0) || !(f->p_vel0[i] >= 0.0))
                return inval("filter noise: q_pos, q_vel, p_vel0 >= 0 and r > 0 required");
    }
    KfConst &c = es->hk.kf;
    c = KfConst{};
    c.enabled = f->enabled ? 1 : 0;
    c.seed_mean = f->seed_mean ? 1 : 0;
    c.dt = f->dt;
    for (int i = 0; i < d; ++i) {
        c.q_pos[i] = f->q_pos[i];
        c.q_vel[i] = f->q_vel[i];
        c.r[i] = f->r[i];
        c.p_vel0[i] = f->p_vel0[i];
    }
    cudaStream_t s = as_stream(stream);
    const int zero = 0;
    CU(cudaMemcpyAsync(es->k, &es->hk, sizeof(CmaConst), cudaMemcpyHostToDevice, s), "filter upload");
    CU(cudaMemcpyAsync(&es->st->kf.initialized, &zero, sizeof(int), cudaMemcpyHostToDevice, s), "filter reset");
    CU(cudaStreamSynchronize(s), "filter upload sync");
    return TRK_OK;
}

trk_status cmaes_destroy(trk_cmaes *es)
{
    if (!es) return inval("NULL optimiser");
    cmaes_free(es);
    return TRK_OK;
}

trk_status cmaes_reset_device(trk_cmaes *es, const double *mean_dev, void *stream)
{
    if (!es || !mean_dev) return inval("NULL argument");
    CU(launch_cma_reset(es->k, es->st, mean_dev, false, nullptr, es->t->ch.n_inst, as_stream(stream)), "reset");
    es->sqrt_pending = false;
    return TRK_OK;
}

// Square roots left out by a frame's last generation, before work that needs
// them (a reset makes them unnecessary).
static trk_status ensure_sqrt(trk_cmaes *es, cudaStream_t s)
{
    if (!es->sqrt_pending) return TRK_OK;
    CU(launch_cma_sqrt(es->k, es->st, s), "square roots");
    es->sqrt_pending = false;
    return TRK_OK;
}

trk_status cmaes_reset_host(trk_cmaes *es, const double *mean_host, void *stream)
{
    if (!es || !mean_host) return inval("NULL argument");
    CU(cudaMemcpyAsync(es->mean0, mean_host, sizeof(double) * es->d, cudaMemcpyHostToDevice, as_stream(stream)),
       "reset upload");
    CU(cudaStreamSynchronize(as_stream(stream)), "reset upload sync");
    return cmaes_reset_device(es, es->mean0, stream);
}

static trk_status ask_impl(trk_cmaes *es, const double *z_in, float *params_dev, void *stream)
{
    cudaStream_t s = as_stream(stream);
    trk_status r = ensure_sqrt(es, s);
    if (r != TRK_OK) return r;
    CU(launch_cma_ask(es->k, es->lam, es->st, es->y, es->z, es->params, z_in, s), "ask");
    if (params_dev && params_dev != es->params)
        CU(cudaMemcpyAsync(params_dev, es->params, sizeof(float) * es->lam * es->d, cudaMemcpyDeviceToDevice, s),
           "ask copy");
    return TRK_OK;
}

trk_status cmaes_ask(trk_cmaes *es, float *params_dev, void *stream)
{
    if (!es) return inval("NULL optimiser");
    return ask_impl(es, nullptr, params_dev, stream);
}

trk_status cmaes_ask_normals(trk_cmaes *es, const double *z_dev, float *params_dev, void *stream)
{
    if (!es || !z_dev) return inval("NULL argument");
    return ask_impl(es, z_dev, params_dev, stream);
}

trk_status cmaes_last_normals(trk_cmaes *es, double *z_dev, void *stream)
{
    if (!es || !z_dev) return inval("NULL argument");
    CU(cudaMemcpyAsync(z_dev, es->z, sizeof(double) * es->lam * es->d, cudaMemcpyDeviceToDevice, as_stream(stream)),
       "normals copy");
    return TRK_OK;
}

trk_status cmaes_tell(trk_cmaes *es, const float *loss_dev, void *stream)
{
    if (!es || !loss_dev) return inval("NULL argument");
    trk_status r = ensure_sqrt(es, as_stream(stream));
    if (r != TRK_OK) return r;
    CU(launch_cma_tell(es->k, es->st, es->y, es->params, loss_dev, as_stream(stream)), "tell");
    return TRK_OK;
}

// One generation in one launch: every cluster samples its candidate, the
// fitness is evaluated, and the last CTA to finish runs the update (and, on a
// frame's last generation, makes the frame's best the estimate).
static trk_status fused_generation(trk_cmaes *es, const uint32_t *mask, int finish, float *pose_out, void *stream)
{
    trk_tracker *t = es->t;
    trk_status r = ensure_sqrt(es, as_stream(stream));
    if (r != TRK_OK) return r;
    es->sqrt_pending = finish != 0;  // the finishing update leaves out the square roots
    EvalArgs a{};
    a.ch = t->ch;
    a.cam = t->cam;
    apply_mesh(a, t);
    a.params = es->params;
    a.d = t->d;
    a.lam = es->lam;
    a.mask = mask;
    a.snap = t->snap;
    a.loss = es->loss;
    a.loss_kind = t->cfg.loss_kind;
    a.lambda_app = t->cfg.lambda_app;
    a.cull = t->cfg.cull_backfaces;
    apply_keypoints(a, t);
    a.cma_k = es->k;
    a.cma_st = es->st;
    a.cma_y = es->y;
    a.cma_z = es->z;
    a.cma_done = es->done;
    a.cma_pose_out = pose_out;
    a.cma_finish = finish;
    if (t->raster == TRK_RASTER_BINNED) {
        a.bin = t->bin;
        CU(launch_binned(a, t->lc_front, as_stream(stream)), "fused generation launch");
        return TRK_OK;
    }
    LaunchCfg lc = t->lc;
    lc.smem = std::max(lc.smem, tell_smem_bytes());
    CU(launch_eval(a, lc, as_stream(stream)), "fused generation launch");
    return TRK_OK;
}

trk_status cmaes_step(trk_cmaes *es, const uint32_t *mask_packed_dev, void *stream)
{
    if (!es || !mask_packed_dev) return inval("NULL argument");
    return fused_generation(es, mask_packed_dev, 0, nullptr, stream);
}

trk_status cmaes_get_state_host(trk_cmaes *es, double *mean, double *sigma, double *C, double *p_sigma, double *p_c,
                                int32_t *gen, int32_t *gen_total, float *best_x, float *best_loss, void *stream)
{
    if (!es) return inval("NULL optimiser");
    CmaState h;
    CU(cudaMemcpyAsync(&h, es->st, sizeof(CmaState), cudaMemcpyDeviceToHost, as_stream(stream)), "state copy");
    CU(cudaStreamSynchronize(as_stream(stream)), "state sync");
    const int d = es->d;
    if (mean) memcpy(mean, h.m, sizeof(double) * d);
    if (sigma) *sigma = h.sigma;
    if (C) memcpy(C, h.C, sizeof(double) * d * d);
    if (p_sigma) memcpy(p_sigma, h.p_sigma, sizeof(double) * d);
    if (p_c) memcpy(p_c, h.p_c, sizeof(double) * d);
    if (gen) *gen = h.gen;
    if (gen_total) *gen_total = h.gen_total;
    if (best_x) memcpy(best_x, h.best_x, sizeof(float) * d);
    if (best_loss) *best_loss = h.best_loss;
    return TRK_OK;
}

trk_status cmaes_buffers(trk_cmaes *es, float **params_dev, float **loss_dev, float **best_x_dev)
{
    if (!es) return inval("NULL optimiser");
    if (params_dev) *params_dev = es->params;
    if (loss_dev) *loss_dev = es->loss;
    if (best_x_dev) *best_x_dev = es->st->best_x;
    return TRK_OK;
}

trk_status track_frame_device(trk_cmaes *es, const uint32_t *mask_packed_dev, int32_t generations,
                              const float *joint_reading_dev, float *pose_out_dev, void *stream)
{
    if (!es || !mask_packed_dev) return inval("NULL argument");
    if (generations < 1 || generations > 1000) return inval("generations out of range");
    cudaStream_t s = as_stream(stream);
    CU(launch_cma_reset(es->k, es->st, nullptr, true, joint_reading_dev, es->t->ch.n_inst, s), "frame reset");
    es->sqrt_pending = false;
    for (int g = 0; g < generations; ++g) {
        trk_status r = fused_generation(es, mask_packed_dev, g == generations - 1, pose_out_dev, stream);
        if (r != TRK_OK) return r;
    }
    return TRK_OK;
}

trk_status track_frame_host(trk_cmaes *es, const uint8_t *mask_host, int32_t generations,
                            const float *joint_reading_host, float *pose_out_host, float *best_loss_out, void *stream)
{
    if (!es || !mask_host || !pose_out_host) return inval("NULL argument");
    cudaStream_t s = as_stream(stream);
    trk_tracker *t = es->t;
    CU(cudaMemcpyAsync(es->mask_bytes, mask_host, (size_t)t->cam.H * t->cam.W, cudaMemcpyHostToDevice, s),
       "mask upload");
    if (joint_reading_host)
        CU(cudaMemcpyAsync(es->joint, joint_reading_host, sizeof(float) * 3 * t->ch.n_inst, cudaMemcpyHostToDevice, s),
           "joint upload");
    CU(launch_pack_mask(es->mask_bytes, es->mask_packed, t->cam.W, t->cam.H, t->cam.Wq, s), "pack");
    trk_status r = track_frame_device(es, es->mask_packed, generations, joint_reading_host ? es->joint : nullptr,
                                      es->pose, stream);
    if (r != TRK_OK) return r;
    CU(cudaMemcpyAsync(pose_out_host, es->pose, sizeof(float) * es->d, cudaMemcpyDeviceToHost, s), "pose download");
    if (best_loss_out)
        CU(cudaMemcpyAsync(best_loss_out, &es->st->best_loss, sizeof(float), cudaMemcpyDeviceToHost, s),
           "loss download");
    CU(cudaStreamSynchronize(s), "track_frame sync");
    return TRK_OK;
}

// Blob: magic, version, d, lam, sizeof(CmaState), then the state.
struct BlobHeader {
    uint32_t magic, version, d, lam, state_bytes, pad;
};
static const uint32_t kBlobMagic = 0x434d4145u;  // "CMAE"

trk_status cmaes_save(trk_cmaes *es, void *blob, size_t *n, void *stream)
{
    if (!es || !n) return inval("NULL argument");
    size_t need = sizeof(BlobHeader) + sizeof(CmaState);
    if (!blob) {
        *n = need;
        return TRK_OK;
    }
    if (*n < need) return inval("blob too small");
    trk_status r = ensure_sqrt(es, as_stream(stream));
    if (r != TRK_OK) return r;
    BlobHeader h{kBlobMagic, 2u, (uint32_t)es->d, (uint32_t)es->lam, (uint32_t)sizeof(CmaState), 0u};
    memcpy(blob, &h, sizeof h);
    CU(cudaMemcpyAsync((char *)blob + sizeof h, es->st, sizeof(CmaState), cudaMemcpyDeviceToHost, as_stream(stream)),
       "save copy");
    CU(cudaStreamSynchronize(as_stream(stream)), "save sync");
    *n = need;
    return TRK_OK;
}

trk_status cmaes_load(trk_cmaes *es, const void *blob, size_t n, void *stream)
{
    if (!es || !blob) return inval("NULL argument");
    if (n < sizeof(BlobHeader) + sizeof(CmaState)) return inval("blob too small");
    BlobHeader h;
    memcpy(&h, blob, sizeof h);
    if (h.magic != kBlobMagic || h.version != 2u || h.d != (uint32_t)es->d || h.lam != (uint32_t)es->lam ||
        h.state_bytes != sizeof(CmaState))
        return inval("blob does not match this optimiser");
    CU(cudaMemcpyAsync(es->st, (const char *)blob + sizeof h, sizeof(CmaState), cudaMemcpyHostToDevice,
                       as_stream(stream)),
       "load copy");
    es->sqrt_pending = false;  // saved states carry their square roots
    CU(cudaStreamSynchronize(as_stream(stream)), "load sync");
    return TRK_OK;
}

}  // extern "C"
