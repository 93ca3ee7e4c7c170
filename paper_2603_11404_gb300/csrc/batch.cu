// Heterogeneous batches (C ABI batch_* in include/tracker.h): many instances --
// one- or two-instrument scenes with their own meshes, image sizes and
// population sizes -- evaluated by one persistent launch per generation.
//
//   k_eval_batch   a fixed grid of co-resident clusters pulls (instance,
//                  candidate) items, largest instances first, from an atomic
//                  queue; each item is the single-candidate fitness body.
//                  Instances are grouped by how many CTAs of their shared-
//                  memory bitmap fit an SM, and each group has its own grid,
//                  queue and bitmap size (the groups' launches run side by
//                  side on forked streams), so a small image is not held to
//                  the occupancy of the batch's largest one
//   cma batch      the CMA-ES update of every instance in one launch, one CTA
//                  per instance (the updates run side by side on the SMs)
//
// batch_track_frame records reset + generations + epilogue once as a CUDA graph
// and replays it every frame; the per-frame mask and pose pointers are read from
// device tables that are refreshed before each replay.  batch_autotune times
// the launch shapes (CTAs per candidate, threads per CTA) on the batch itself.
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "internal.cuh"

using namespace trk;

struct trk_batch {
    int n = 0;
    bool cma = false;
    std::vector<trk_tracker *> tr;
    std::vector<trk_cmaes *> es;
    std::vector<int> lam;
    std::vector<EvalArgs> hdescs;
    EvalArgs *descs = nullptr;          // [n] device
    const uint32_t **masks = nullptr;   // [n] device table
    float **poses = nullptr;            // [n] device table
    int2 *items = nullptr;              // [n_items] device: by group, largest instances first in each
    int n_items = 0;
    unsigned *next_item = nullptr;      // [groups] device queue heads
    struct Group {
        int item_off = 0, n_items = 0;
        size_t smem = 0;                // the largest bitmap of the group's instances
        LaunchCfg lc{};
        int n_clusters = 0;
    };
    std::vector<Group> groups;          // largest shared-memory footprint first
    std::vector<cudaStream_t> aux;      // [groups - 1] streams the later groups launch on
    std::vector<cudaEvent_t> joined;    // [groups - 1] their completion
    cudaEvent_t forked = nullptr;
    int2 *snap = nullptr;               // batch-owned scratch for every instance
    BatchTables tb;                     // CMA-ES tables (tb.pose aliases poses)
    const void **pin = nullptr;         // pinned staging for the two pointer tables
    LaunchCfg lc{};
    int n_clusters = 0;
    cudaStream_t cap = nullptr;         // capture stream
    cudaGraphExec_t gexec = nullptr;
    int g_gens = -1;
};

static void batch_free(trk_batch *b)
{
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (cudaStream_t x : b->aux)
        if (x) cudaStreamDestroy(x);
    for (cudaEvent_t x : b->joined)
        if (x) cudaEventDestroy(x);
    if (b->forked) cudaEventDestroy(b->forked);
    cudaFree(b->descs);
    cudaFree(b->masks);
    cudaFree(b->poses);
    cudaFree(b->items);
    cudaFree(b->next_item);
    cudaFree(b->snap);
    cudaFree(b->tb.k);
    cudaFree(b->tb.st);
    cudaFree(b->tb.y);
    cudaFree(b->tb.params);
    cudaFree(b->tb.loss);
    cudaFree(b->tb.ninst);
    cudaFreeHost(b->pin);
    delete b;
}

static trk_status bfail(trk_status s, const char *why)
{
    set_last_error(why);
    return s;
}

// Shared memory and occupancy for a launch shape, per group; fills the
// groups' launch configurations, b->lc (the shape) and b->n_clusters (summed).
static trk_status batch_configure(trk_batch *b, int cluster, int threads)
{
    int max_inst = 1;
    size_t smem = 0;
    for (int i = 0; i < b->n; ++i) {
        max_inst = std::max(max_inst, b->tr[i]->ch.n_inst);
        smem = std::max(smem, eval_smem_bytes(b->hdescs[i]));
    }
    if (threads <= 0) threads = 256;
    if (threads > 256 || threads % 32 || threads < 32 * max_inst) return bfail(TRK_EINVAL, "batch threads");
    if (cluster <= 0) cluster = 8;
    if (cluster > 8) return bfail(TRK_EINVAL, "batch cluster must be 1..8");
    if (smem > 227 * 1024) return bfail(TRK_EINVAL, "largest image too large for the shared-memory bitmap");
    int total = 0;
    for (trk_batch::Group &g : b->groups) {
        int maxc = 0;
        cudaError_t e = prepare_eval_batch(g.smem, cluster, threads, &maxc);
        if (e != cudaSuccess) return bfail(TRK_ECUDA, cudaGetErrorString(e));
        if (maxc <= 0) return bfail(TRK_EINVAL, "launch shape does not fit on the device");
        g.lc.cluster = cluster;
        g.lc.threads = threads;
        g.lc.smem = g.smem;
        g.n_clusters = std::min(maxc, g.n_items);
        total += g.n_clusters;
    }
    b->lc.cluster = cluster;
    b->lc.threads = threads;
    b->lc.smem = smem;
    b->n_clusters = total;
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        b->g_gens = -1;
    }
    return TRK_OK;
}

extern "C" {

trk_status batch_create(trk_tracker *const *trackers, trk_cmaes *const *optimisers, const int32_t *lam, int32_t n,
                        int32_t cluster, int32_t threads, trk_batch **out)
{
    if (!out) return bfail(TRK_EINVAL, "out is NULL");
    *out = nullptr;
    if (!trackers || n < 1 || n > 4096) return bfail(TRK_EINVAL, "need 1..4096 instances");
    if (!optimisers && !lam) return bfail(TRK_EINVAL, "population sizes or optimisers required");
    trk_batch *b = new (std::nothrow) trk_batch();
    if (!b) return TRK_ENOMEM;
    b->n = n;
    b->cma = optimisers != nullptr;
    long long snap_total = 0;
    for (int i = 0; i < n; ++i) {
        trk_tracker *t = trackers[i];
        trk_cmaes *es = optimisers ? optimisers[i] : nullptr;
        if (!t || (optimisers && (!es || es->t != t))) {
            batch_free(b);
            return bfail(TRK_EINVAL, "instance needs a tracker (and, with optimisers, one created on it)");
        }
        int l = es ? es->lam : lam[i];
        if (l < 1 || l > 65535) {
            batch_free(b);
            return bfail(TRK_EINVAL, "population size out of range");
        }
        b->tr.push_back(t);
        b->es.push_back(es);
        b->lam.push_back(l);
        snap_total += (long long)l * t->ch.n_inst * std::max(t->V, 1);
        b->n_items += l;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&b->descs, sizeof(EvalArgs) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->masks, sizeof(void *) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->poses, sizeof(void *) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->items, sizeof(int2) * b->n_items)) != cudaSuccess ||
        (e = cudaMalloc(&b->snap, sizeof(int2) * snap_total)) != cudaSuccess ||
        (e = cudaMalloc(&b->tb.k, sizeof(void *) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->tb.st, sizeof(void *) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->tb.y, sizeof(void *) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->tb.params, sizeof(void *) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->tb.loss, sizeof(void *) * n)) != cudaSuccess ||
        (e = cudaMalloc(&b->tb.ninst, sizeof(int) * n)) != cudaSuccess ||
        (e = cudaMallocHost(&b->pin, sizeof(void *) * 2 * n)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        batch_free(b);
        set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA;
    }
    // descriptors: per-instance constants, batch-owned scratch
    b->hdescs.resize(n);
    long long off = 0;
    std::vector<const CmaConst *> hk(n);
    std::vector<CmaState *> hst(n);
    std::vector<const double *> hy(n);
    std::vector<const float *> hp(n), hl(n);
    std::vector<int> hni(n);
    for (int i = 0; i < n; ++i) {
        trk_tracker *t = b->tr[i];
        EvalArgs a{};
        a.ch = t->ch;
        a.cam = t->cam;
        apply_mesh(a, t);
        a.d = t->d;
        a.lam = b->lam[i];
        a.snap = b->snap + off;
        a.loss_kind = t->cfg.loss_kind;
        a.lambda_app = t->cfg.lambda_app;
        a.cull = t->cfg.cull_backfaces;
        apply_keypoints(a, t);
        off += (long long)b->lam[i] * t->ch.n_inst * std::max(t->V, 1);
        if (trk_cmaes *es = b->es[i]) {
            a.params = es->params;
            a.loss = es->loss;
            a.cma_k = es->k;
            a.cma_st = es->st;
            a.cma_y = es->y;
            a.cma_z = es->z;
            hk[i] = es->k;
            hst[i] = es->st;
            hy[i] = es->y;
            hp[i] = es->params;
            hl[i] = es->loss;
        }
        hni[i] = t->ch.n_inst;
        b->hdescs[i] = a;
    }
    // groups: instances by the number of CTAs with their bitmap that fit an
    // SM's shared memory (a few KB of other shared memory per CTA included),
    // fewest first; items: (instance, candidate) by group, and within a group
    // instances with more work first
    int dev = 0, sm_smem = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) {
        batch_free(b);
        set_last_error(cudaGetErrorString(e));
        return TRK_ECUDA;
    }
    auto per_sm = [&](int i) { return (long long)sm_smem / (long long)(eval_smem_bytes(b->hdescs[i]) + 4096); };
    auto cost = [&](int i) { return (long long)(b->tr[i]->V + b->tr[i]->T) * b->tr[i]->ch.n_inst; };
    std::vector<int> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const long long px = per_sm(x), py = per_sm(y);
        return px != py ? px < py : cost(x) > cost(y);
    });
    std::vector<int2> items;
    items.reserve(b->n_items);
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        if (k == 0 || per_sm(i) != per_sm(order[k - 1])) {
            b->groups.emplace_back();
            b->groups.back().item_off = (int)items.size();
        }
        trk_batch::Group &g = b->groups.back();
        g.n_items += b->lam[i];
        g.smem = std::max(g.smem, eval_smem_bytes(b->hdescs[i]));
        for (int c = 0; c < b->lam[i]; ++c) items.push_back(make_int2(i, c));
    }
    const int G = (int)b->groups.size();
    b->aux.assign(G - 1, nullptr);
    b->joined.assign(G - 1, nullptr);
    if ((e = cudaMalloc(&b->next_item, sizeof(unsigned) * G)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming)) != cudaSuccess) {
        batch_free(b);
        set_last_error(cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA;
    }
    for (int g = 0; g + 1 < G; ++g)
        if ((e = cudaStreamCreateWithFlags(&b->aux[g], cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&b->joined[g], cudaEventDisableTiming)) != cudaSuccess) {
            batch_free(b);
            set_last_error(cudaGetErrorString(e));
            return TRK_ECUDA;
        }
    if ((e = cudaMemcpy(b->descs, b->hdescs.data(), sizeof(EvalArgs) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->tb.k, hk.data(), sizeof(void *) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->tb.st, hst.data(), sizeof(void *) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->tb.y, hy.data(), sizeof(void *) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->tb.params, hp.data(), sizeof(void *) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->tb.loss, hl.data(), sizeof(void *) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(b->tb.ninst, hni.data(), sizeof(int) * n, cudaMemcpyHostToDevice)) != cudaSuccess) {
        batch_free(b);
        set_last_error(cudaGetErrorString(e));
        return TRK_ECUDA;
    }
    b->tb.pose = b->poses;
    trk_status st = batch_configure(b, cluster, threads);
    if (st != TRK_OK) {
        batch_free(b);
        return st;
    }
    *out = b;
    return TRK_OK;
}

trk_status batch_destroy(trk_batch *b)
{
    if (!b) return bfail(TRK_EINVAL, "NULL batch");
    batch_free(b);
    return TRK_OK;
}

trk_status batch_set_launch(trk_batch *b, int32_t cluster, int32_t threads)
{
    if (!b) return bfail(TRK_EINVAL, "NULL batch");
    return batch_configure(b, cluster, threads);
}

trk_status batch_get_launch(const trk_batch *b, int32_t *cluster, int32_t *threads, int32_t *n_clusters)
{
    if (!b) return bfail(TRK_EINVAL, "NULL batch");
    if (cluster) *cluster = b->lc.cluster;
    if (threads) *threads = b->lc.threads;
    if (n_clusters) *n_clusters = b->n_clusters;
    return TRK_OK;
}

// Descriptors for a launch over explicit per-instance buffers (fitness only).
static trk_status stage_eval(trk_batch *b, const float *const *params, const uint32_t *const *masks,
                             float *const *loss, int32_t *const *counts, cudaStream_t s)
{
    std::vector<EvalArgs> d = b->hdescs;
    for (int i = 0; i < b->n; ++i) {
        if (!params[i] || !masks[i]) return bfail(TRK_EINVAL, "NULL params or mask");
        d[i].params = params[i];
        d[i].mask = masks[i];
        d[i].loss = loss ? loss[i] : nullptr;
        d[i].counts = counts ? counts[i] : nullptr;
        d[i].cma_k = nullptr;
        d[i].cma_st = nullptr;
        d[i].cma_y = d[i].cma_z = nullptr;
    }
    // pageable source: the call returns once d has been staged, so d may go out of scope
    cudaError_t e = cudaMemcpyAsync(b->descs, d.data(), sizeof(EvalArgs) * b->n, cudaMemcpyHostToDevice, s);
    return e == cudaSuccess ? TRK_OK : bfail(TRK_ECUDA, cudaGetErrorString(e));
}

// One persistent fitness launch per group: the first group on s, the others
// on streams forked from s and joined back into it (under stream capture the
// fork and join become graph edges).
static cudaError_t launch_groups(trk_batch *b, const uint32_t *const *masks, cudaStream_t s)
{
    const int G = (int)b->groups.size();
    auto one = [&](int g, cudaStream_t st) {
        const trk_batch::Group &x = b->groups[g];
        return launch_eval_batch(b->descs, masks, b->items + x.item_off, x.n_items, b->next_item + g, x.lc,
                                 x.n_clusters, st);
    };
    cudaError_t e = cudaMemsetAsync(b->next_item, 0, sizeof(unsigned) * G, s);
    if (e != cudaSuccess) return e;
    if (G > 1 && (e = cudaEventRecord(b->forked, s)) != cudaSuccess) return e;
    for (int g = 1; g < G; ++g)
        if ((e = cudaStreamWaitEvent(b->aux[g - 1], b->forked, 0)) != cudaSuccess ||
            (e = one(g, b->aux[g - 1])) != cudaSuccess ||
            (e = cudaEventRecord(b->joined[g - 1], b->aux[g - 1])) != cudaSuccess)
            return e;
    if ((e = one(0, s)) != cudaSuccess) return e;
    for (int g = 1; g < G; ++g)
        if ((e = cudaStreamWaitEvent(s, b->joined[g - 1], 0)) != cudaSuccess) return e;
    return cudaSuccess;
}

static trk_status launch_staged(trk_batch *b, cudaStream_t s)
{
    cudaError_t e = launch_groups(b, nullptr, s);
    return e == cudaSuccess ? TRK_OK : bfail(TRK_ECUDA, cudaGetErrorString(e));
}

trk_status batch_eval(trk_batch *b, const float *const *params_dev, const uint32_t *const *masks_dev,
                      float *const *loss_dev, int32_t *const *counts_dev, void *stream)
{
    if (!b || !params_dev || !masks_dev) return bfail(TRK_EINVAL, "NULL argument");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    trk_status st = stage_eval(b, params_dev, masks_dev, loss_dev, counts_dev, s);
    if (st == TRK_OK) st = launch_staged(b, s);
    if (st != TRK_OK) return st;
    // restore the resident descriptors for batch_track_frame
    cudaError_t e = cudaMemcpyAsync(b->descs, b->hdescs.data(), sizeof(EvalArgs) * b->n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bfail(TRK_ECUDA, cudaGetErrorString(e));
    return TRK_OK;
}

// reset, generations x (fitness + updates), epilogue: enqueued on s
static cudaError_t enqueue_frame(trk_batch *b, int generations, cudaStream_t s)
{
    cudaError_t e = launch_cma_batch(0, b->n, nullptr, b->tb, s);
    for (int g = 0; g < generations && e == cudaSuccess; ++g) {
        if ((e = launch_groups(b, b->masks, s)) != cudaSuccess) break;
        // the last generation's updates leave out the square roots (the next frame resets)
        e = launch_cma_batch(g == generations - 1 ? 3 : 1, b->n, nullptr, b->tb, s);
    }
    if (e == cudaSuccess)
        e = launch_cma_batch(2, b->n, nullptr, b->tb, s);
    return e;
}

trk_status batch_track_frame(trk_batch *b, const uint32_t *const *masks_dev, int32_t generations,
                             float *const *poses_dev, int32_t use_graph, void *stream)
{
    if (!b || !masks_dev || !poses_dev) return bfail(TRK_EINVAL, "NULL argument");
    if (!b->cma) return bfail(TRK_EINVAL, "batch was created without optimisers");
    // every frame ends with updates that leave out the square roots: later
    // single-optimiser work that samples without a reset runs them first
    for (trk_cmaes *o : b->es)
        if (o) o->sqrt_pending = true;
    if (generations < 1 || generations > 1000) return bfail(TRK_EINVAL, "generations out of range");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    // the previous frame's replay must be done with the pinned tables before they change
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bfail(TRK_ECUDA, cudaGetErrorString(e));
    for (int i = 0; i < b->n; ++i) {
        if (!masks_dev[i] || !poses_dev[i]) return bfail(TRK_EINVAL, "NULL mask or pose pointer");
        b->pin[i] = masks_dev[i];
        b->pin[b->n + i] = poses_dev[i];
    }
    if ((e = cudaMemcpyAsync(b->masks, b->pin, sizeof(void *) * b->n, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(b->poses, b->pin + b->n, sizeof(void *) * b->n, cudaMemcpyHostToDevice, s)) !=
            cudaSuccess)
        return bfail(TRK_ECUDA, cudaGetErrorString(e));
    if (!use_graph) {
        e = enqueue_frame(b, generations, s);
        return e == cudaSuccess ? TRK_OK : bfail(TRK_ECUDA, cudaGetErrorString(e));
    }
    if (!b->gexec || b->g_gens != generations) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return bfail(TRK_ECUDA, cudaGetErrorString(e));
        cudaError_t e2 = enqueue_frame(b, generations, b->cap);
        e = cudaStreamEndCapture(b->cap, &g);
        if (e2 != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return bfail(TRK_ECUDA, cudaGetErrorString(e2 != cudaSuccess ? e2 : e));
        }
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(TRK_ECUDA, cudaGetErrorString(e));
        b->g_gens = generations;
    }
    e = cudaGraphLaunch(b->gexec, s);
    return e == cudaSuccess ? TRK_OK : bfail(TRK_ECUDA, cudaGetErrorString(e));
}

trk_status batch_autotune(trk_batch *b, const float *const *params_dev, const uint32_t *const *masks_dev,
                          int32_t reps, int32_t *cluster_out, int32_t *threads_out, float *us_out, void *stream)
{
    if (!b || !masks_dev) return bfail(TRK_EINVAL, "NULL argument");
    if (reps < 1 || reps > 1000) return bfail(TRK_EINVAL, "reps out of range");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<const float *> p(b->n);
    std::vector<float *> l(b->n);
    for (int i = 0; i < b->n; ++i) {
        p[i] = params_dev ? params_dev[i] : (b->es[i] ? b->es[i]->params : nullptr);
        l[i] = b->es[i] ? b->es[i]->loss : nullptr;
        if (!p[i]) return bfail(TRK_EINVAL, "params required for an instance without an optimiser");
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int clusters[] = {1, 2, 4, 8};
    const int threads[] = {128, 256};
    float best = 1e30f;
    int bc = b->lc.cluster, bt = b->lc.threads;
    if (stage_eval(b, p.data(), masks_dev, l.data(), nullptr, s) != TRK_OK) return TRK_EINVAL;
    for (int c : clusters)
        for (int t : threads) {
            if (batch_configure(b, c, t) != TRK_OK) continue;
            if (launch_staged(b, s) != TRK_OK) continue;  // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps; ++r) launch_staged(b, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            float us = ms * 1000.f / reps;
            if (us < best) {
                best = us;
                bc = c;
                bt = t;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    trk_status st = batch_configure(b, bc, bt);
    cudaMemcpyAsync(b->descs, b->hdescs.data(), sizeof(EvalArgs) * b->n, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    if (cluster_out) *cluster_out = bc;
    if (threads_out) *threads_out = bt;
    if (us_out) *us_out = best;
    return st;
}

}  // extern "C"
