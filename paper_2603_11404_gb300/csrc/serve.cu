// Serving runtime (C ABI server_* in include/tracker.h): frames from several
// camera streams tracked with continuous batching.
//
// Every camera stream owns a device-resident CMA-ES state (mean, covariance,
// step size, estimate) that is warm-started frame to frame.  Frames are
// queued on the host and admitted into a fixed number of slots; one *tick*
// advances every admitted frame by one CMA-ES generation:
//
//   uploads of newly admitted masks -> reset of their optimisers ->
//   one persistent fitness launch over all admitted frames' candidates, in
//   which the last CTA of each frame's candidates runs that frame's CMA-ES
//   update (and, after its last generation, the frame epilogue) ->
//   pose download for the frames that ran their last generation
//
// A tick with a single frame in the slots runs the fused per-frame kernel
// instead (the one track_frame_device launches, same arithmetic).
//
// so a frame that arrives while others are on the GPU joins at the next tick
// and its work shares launches with theirs (iteration-level batching), and a
// slot freed by a finishing frame is reused at the next tick.  Ticks are
// queued on one CUDA stream; a ring of tick records (device tables, pinned
// staging, completion event) lets the host prepare tick k+1 while the device
// runs tick k.  Each frame is computed by exactly the per-instance kernels of
// track_frame_device, so its result does not depend on what else is admitted.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <new>
#include <vector>

#include "internal.cuh"

using namespace trk;

namespace {

constexpr int kRing = 4;      // tick records
constexpr int kInflight = 2;  // ticks queued on the device at most: a newly admitted frame
                              // waits for at most one tick before its first

struct Pending {
    int buf = -1;             // pinned staging buffer (mask bytes, then joint readings)
    uint64_t tag = 0;
    double t_submit = 0.0;
    double t_admit = 0.0;
    bool joint = false;
};

struct CamStream {
    trk_cmaes *es = nullptr;
    int gens = 0;
    bool use_joint = false;
    bool open = false;
    int2 *snap = nullptr;     // this stream's raster scratch
    size_t bytes = 0;         // device bytes admitted for it
    std::deque<Pending> queue;
    bool active = false;      // a frame occupies a slot
    int gen = 0;              // generations already enqueued for it
    Pending cur;
    long long cost = 0;       // fitness work per candidate, for item ordering
};

struct DoneRec {
    int stream;
    uint64_t tag;
    double t_submit, t_admit;
    int d;
};

struct Tick {
    cudaEvent_t ev = nullptr;
    bool in_flight = false;
    void *pin = nullptr;      // mapped pinned: tick table, then results
    void *pin_dev = nullptr;  // the device's address of pin
    int *dev = nullptr;       // device: the streams admitted at this tick
    std::vector<DoneRec> done;
    std::vector<int> release; // staging buffers free once this tick has run
    double t_enqueue = 0.0;
};

double host_now()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct trk_server {
    int max_active = 0, max_streams = 0, max_pending = 0;
    size_t max_pixels = 0, reserve = 0, stage_bytes = 0;
    std::vector<CamStream> cs;
    std::vector<EvalArgs> hdescs;
    EvalArgs *descs = nullptr;
    unsigned *queue = nullptr; // fitness queue counter: zero between ticks (the kernel leaves it so)
    BatchTables tb;
    uint8_t *stage = nullptr;  // pinned [max_pending][stage_bytes]
    std::vector<int> free_bufs;
    Tick ring[kRing];
    int ring_next = 0;
    size_t items_cap = 0;      // int2 entries per tick table
    cudaStream_t s = nullptr;
    cudaEvent_t ref = nullptr;
    double t_ref = 0.0;
    LaunchCfg lc{};
    int max_clusters = 0;
    // light ticks: the widest cluster (up to 8 CTAs per candidate) whose
    // persistent grid holds every candidate of the tick at once
    int max_clusters_by_size[9] = {};
    std::vector<trk_frame_result> completed;
    int rr = 0;                // round-robin start for admission
    int n_active = 0;
    long long ticks = 0;
};

namespace {

trk_status sfail(trk_status st, const char *why)
{
    set_last_error(why);
    return st;
}

#define SCU(call, what)                                                            \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) return sfail(TRK_ECUDA, cudaGetErrorString(e_));    \
    } while (0)

// Tick table layout, in mapped pinned memory that the fitness launch reads in
// place (no upload): the streams admitted at this tick, one last-generation
// flag per stream, then the items; the results of finished frames follow.
// Only the admitted streams are copied to the device, for the reset launch.
size_t tick_items_offset(const trk_server *v) { return (2 * v->max_streams * sizeof(int) + 15) & ~(size_t)15; }
size_t tick_table_bytes(const trk_server *v) { return tick_items_offset(v) + v->items_cap * sizeof(int2); }
size_t tick_result_bytes(const trk_server *v) { return (size_t)v->max_streams * (TRK_MAX_D + 1) * sizeof(float); }

void server_free(trk_server *v)
{
    if (!v) return;
    if (v->s) cudaStreamSynchronize(v->s);
    for (Tick &t : v->ring) {
        if (t.ev) cudaEventDestroy(t.ev);
        cudaFreeHost(t.pin);
        cudaFree(t.dev);
    }
    for (CamStream &c : v->cs) cudaFree(c.snap);
    cudaFree(v->queue);
    cudaFree(v->descs);
    cudaFree(v->tb.k);
    cudaFree(v->tb.st);
    cudaFree(v->tb.joint);
    cudaFree(v->tb.ninst);
    cudaFreeHost(v->stage);
    if (v->ref) cudaEventDestroy(v->ref);
    if (v->s) cudaStreamDestroy(v->s);
    delete v;
}

// Collect the results of every completed tick, oldest first.
trk_status harvest(trk_server *v)
{
    for (int k = 0; k < kRing; ++k) {
        // oldest in-flight tick: the ring is filled in order starting at ring_next
        Tick &t = v->ring[(v->ring_next + k) % kRing];
        if (!t.in_flight) continue;
        cudaError_t e = cudaEventQuery(t.ev);
        if (e == cudaErrorNotReady) break;
        if (e != cudaSuccess) return sfail(TRK_ECUDA, cudaGetErrorString(e));
        float ms = 0.f;
        SCU(cudaEventElapsedTime(&ms, v->ref, t.ev), "tick time");
        const double t_done = v->t_ref + 1e-3 * ms;
        const float *res = reinterpret_cast<const float *>(static_cast<const char *>(t.pin) + tick_table_bytes(v));
        for (size_t i = 0; i < t.done.size(); ++i) {
            const DoneRec &r = t.done[i];
            trk_frame_result out{};
            out.stream = r.stream;
            out.tag = r.tag;
            out.t_submit = r.t_submit;
            out.t_admit = r.t_admit;
            out.t_done = t_done;
            out.d = r.d;
            memcpy(out.pose, res + i * (TRK_MAX_D + 1), sizeof(float) * r.d);
            out.best_loss = res[i * (TRK_MAX_D + 1) + TRK_MAX_D];
            v->completed.push_back(out);
        }
        for (int b : t.release) v->free_bufs.push_back(b);
        t.done.clear();
        t.release.clear();
        t.in_flight = false;
    }
    return TRK_OK;
}

trk_status reconfigure(trk_server *v)
{
    size_t smem = 0;
    int max_inst = 1;
    for (size_t i = 0; i < v->cs.size(); ++i)
        if (v->cs[i].open) {
            smem = std::max(smem, std::max(eval_smem_bytes(v->hdescs[i]), tell_smem_bytes()));
            max_inst = std::max(max_inst, v->cs[i].es->t->ch.n_inst);
            // single-frame ticks launch the tracker's fused kernel on this device
            const trk_tracker *t = v->cs[i].es->t;
            if (t->raster == TRK_RASTER_CLUSTER)
                SCU(prepare_eval(std::max(t->lc.smem, tell_smem_bytes())), "fused kernel shared memory");
        }
    if (v->lc.threads < 32 * max_inst) return sfail(TRK_EINVAL, "threads too few for two instruments");
    int maxc = 0, maxw = 0;
    SCU(prepare_eval_batch(smem, v->lc.cluster, v->lc.threads, &maxc), "server launch shape");
    if (maxc <= 0) return sfail(TRK_EINVAL, "launch shape does not fit on the device");
    v->lc.smem = smem;
    v->max_clusters = maxc;
    // a light tick (few admitted frames) runs its candidates on as many CTAs
    // each as lets them all run at once: its latency is one candidate's, which
    // more CTAs per candidate shorten
    for (int c = 0; c <= 8; ++c) v->max_clusters_by_size[c] = 0;
    for (int c = v->lc.cluster + 1; c <= 8; ++c) {
        SCU(prepare_eval_batch(smem, c, v->lc.threads, &maxw), "server wide launch shape");
        v->max_clusters_by_size[c] = maxw;
    }
    return TRK_OK;
}

}  // namespace

extern "C" {

double server_now(void) { return host_now(); }

trk_status server_create(int32_t max_active, int32_t max_streams, int32_t max_pending, int64_t max_pixels,
                         int32_t max_lambda, int64_t hbm_reserve_bytes, int32_t cluster, int32_t threads,
                         trk_server **out)
{
    if (!out) return sfail(TRK_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_active < 1 || max_streams < 1 || max_streams > 4096 || max_pending < 1 || max_pending > 65536)
        return sfail(TRK_EINVAL, "slot, stream or pending counts out of range");
    if (max_pixels < 1 || max_pixels > TRK_MAX_PIXELS) return sfail(TRK_EINVAL, "max_pixels out of range");
    if (max_lambda < 1 || max_lambda > TRK_MAX_LAMBDA) return sfail(TRK_EINVAL, "max_lambda out of range");
    if (hbm_reserve_bytes < 0) return sfail(TRK_EINVAL, "hbm_reserve_bytes < 0");
    if (cluster < 0 || cluster > 8) return sfail(TRK_EINVAL, "cluster must be 0..8");
    if (threads < 0 || threads > 256 || threads % 32) return sfail(TRK_EINVAL, "threads");
    trk_server *v = new (std::nothrow) trk_server();
    if (!v) return sfail(TRK_ENOMEM, "host allocation");
    v->max_active = std::min(max_active, max_streams);
    v->max_streams = max_streams;
    v->max_pending = max_pending;
    v->max_pixels = (size_t)max_pixels;
    v->reserve = (size_t)hbm_reserve_bytes;
    v->stage_bytes = ((size_t)max_pixels + sizeof(float) * 3 * TRK_MAX_INSTRUMENTS + 255) & ~(size_t)255;
    v->items_cap = (size_t)v->max_active * max_lambda;
    v->lc.cluster = cluster > 0 ? cluster : 4;  // 4: one population of 64 fits one wave of the persistent grid
    v->lc.threads = threads > 0 ? threads : 256;
    v->cs.resize(max_streams);
    v->hdescs.resize(max_streams);
    const size_t P = sizeof(void *) * max_streams;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&v->s, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreate(&v->ref)) != cudaSuccess ||
        (e = cudaMalloc(&v->descs, sizeof(EvalArgs) * max_streams)) != cudaSuccess ||
        (e = cudaMalloc(&v->queue, sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMemsetAsync(v->queue, 0, sizeof(unsigned), v->s)) != cudaSuccess ||
        (e = cudaMalloc(&v->tb.k, P)) != cudaSuccess || (e = cudaMalloc(&v->tb.st, P)) != cudaSuccess ||
        (e = cudaMalloc(&v->tb.joint, P)) != cudaSuccess ||
        (e = cudaMalloc(&v->tb.ninst, sizeof(int) * max_streams)) != cudaSuccess ||
        (e = cudaMallocHost(&v->stage, v->stage_bytes * max_pending)) != cudaSuccess) {
        server_free(v);
        return sfail(e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA, cudaGetErrorString(e));
    }
    for (Tick &t : v->ring) {
        if ((e = cudaEventCreate(&t.ev)) != cudaSuccess ||
            (e = cudaHostAlloc(&t.pin, tick_table_bytes(v) + tick_result_bytes(v), cudaHostAllocMapped)) !=
                cudaSuccess ||
            (e = cudaHostGetDevicePointer(&t.pin_dev, t.pin, 0)) != cudaSuccess ||
            (e = cudaMalloc(&t.dev, sizeof(int) * max_streams)) != cudaSuccess) {
            server_free(v);
            return sfail(e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA, cudaGetErrorString(e));
        }
    }
    for (int i = max_pending - 1; i >= 0; --i) v->free_bufs.push_back(i);
    // time origin: device event timestamps are mapped onto the host clock
    if ((e = cudaEventRecord(v->ref, v->s)) != cudaSuccess || (e = cudaEventSynchronize(v->ref)) != cudaSuccess) {
        server_free(v);
        return sfail(TRK_ECUDA, cudaGetErrorString(e));
    }
    v->t_ref = host_now();
    *out = v;
    return TRK_OK;
}

trk_status server_destroy(trk_server *v)
{
    if (!v) return sfail(TRK_EINVAL, "NULL server");
    server_free(v);
    return TRK_OK;
}

trk_status server_add_stream(trk_server *v, trk_cmaes *es, int32_t generations, int32_t use_joint_reading,
                             int32_t *stream_id)
{
    if (!v || !es || !stream_id) return sfail(TRK_EINVAL, "NULL argument");
    if (generations < 1 || generations > 1000) return sfail(TRK_EINVAL, "generations out of range");
    trk_tracker *t = es->t;
    if ((size_t)t->cam.W * t->cam.H > v->max_pixels) return sfail(TRK_EINVAL, "image larger than max_pixels");
    if ((size_t)es->lam * v->max_active > v->items_cap) return sfail(TRK_EINVAL, "population larger than max_lambda");
    int id = -1;
    for (int i = 0; i < v->max_streams; ++i)
        if (!v->cs[i].open) {
            id = i;
            break;
        }
    if (id < 0) return sfail(TRK_EBUSY, "all stream slots are open");
    for (int i = 0; i < v->max_streams; ++i)
        if (v->cs[i].open && v->cs[i].es == es) return sfail(TRK_EINVAL, "optimiser already serves a stream");
    // admission by device memory: the stream's raster scratch must leave the reserve free
    const size_t bytes = sizeof(int2) * (size_t)es->lam * t->ch.n_inst * std::max(t->V, 1);
    size_t free_b = 0, total_b = 0;
    SCU(cudaMemGetInfo(&free_b, &total_b), "memory query");
    if (free_b < bytes + v->reserve) return sfail(TRK_EBUSY, "not enough free device memory for another stream");
    CamStream &c = v->cs[id];
    c = CamStream{};
    if (cudaMalloc(&c.snap, bytes) != cudaSuccess) {
        cudaGetLastError();
        c = CamStream{};
        return sfail(TRK_EBUSY, "device allocation for the stream failed");
    }
    c.es = es;
    c.gens = generations;
    c.use_joint = use_joint_reading != 0;
    c.bytes = bytes;
    c.cost = (long long)(t->V + t->T) * t->ch.n_inst;
    c.open = true;
    EvalArgs a{};
    a.ch = t->ch;
    a.cam = t->cam;
    apply_mesh(a, t);
    a.d = t->d;
    a.lam = es->lam;
    a.snap = c.snap;
    a.mask = es->mask_packed;
    a.params = es->params;
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
    a.cma_pose_out = es->pose;
    v->hdescs[id] = a;
    const void *kp = es->k, *stp = es->st;
    const void *jp = c.use_joint ? es->joint : nullptr;
    const int ni = t->ch.n_inst;
    const size_t o = sizeof(void *) * id;
    SCU(cudaMemcpyAsync(v->descs + id, &v->hdescs[id], sizeof(EvalArgs), cudaMemcpyHostToDevice, v->s), "desc");
    SCU(cudaMemcpyAsync((char *)v->tb.k + o, &kp, sizeof(void *), cudaMemcpyHostToDevice, v->s), "table");
    SCU(cudaMemcpyAsync((char *)v->tb.st + o, &stp, sizeof(void *), cudaMemcpyHostToDevice, v->s), "table");
    SCU(cudaMemcpyAsync((char *)v->tb.joint + o, &jp, sizeof(void *), cudaMemcpyHostToDevice, v->s), "table");
    SCU(cudaMemcpyAsync(v->tb.ninst + id, &ni, sizeof(int), cudaMemcpyHostToDevice, v->s), "table");
    SCU(cudaStreamSynchronize(v->s), "stream registration");  // the sources above are host stack values
    trk_status st = reconfigure(v);
    if (st != TRK_OK) {
        cudaFree(c.snap);
        c = CamStream{};
        reconfigure(v);
        return st;
    }
    *stream_id = id;
    return TRK_OK;
}

trk_status server_remove_stream(trk_server *v, int32_t stream_id)
{
    if (!v || stream_id < 0 || stream_id >= v->max_streams || !v->cs[stream_id].open)
        return sfail(TRK_EINVAL, "no such stream");
    CamStream &c = v->cs[stream_id];
    if (c.active || !c.queue.empty()) return sfail(TRK_EBUSY, "stream has frames queued or in flight");
    SCU(cudaStreamSynchronize(v->s), "drain");
    cudaFree(c.snap);
    c = CamStream{};
    return TRK_OK;
}

trk_status server_submit(trk_server *v, int32_t stream_id, const uint8_t *mask_host, const float *joint_reading_host,
                         uint64_t tag, double t_submit)
{
    if (!v || !mask_host) return sfail(TRK_EINVAL, "NULL argument");
    if (stream_id < 0 || stream_id >= v->max_streams || !v->cs[stream_id].open)
        return sfail(TRK_EINVAL, "no such stream");
    CamStream &c = v->cs[stream_id];
    if (c.use_joint && !joint_reading_host) return sfail(TRK_EINVAL, "stream expects joint readings");
    trk_status st = harvest(v);
    if (st != TRK_OK) return st;
    if (v->free_bufs.empty()) return sfail(TRK_EBUSY, "no free staging buffer (max_pending frames queued)");
    const int b = v->free_bufs.back();
    v->free_bufs.pop_back();
    trk_tracker *t = c.es->t;
    uint8_t *dst = v->stage + v->stage_bytes * b;
    const size_t n = (size_t)t->cam.W * t->cam.H;
    memcpy(dst, mask_host, n);
    if (c.use_joint) memcpy(dst + ((n + 15) & ~(size_t)15), joint_reading_host, sizeof(float) * 3 * t->ch.n_inst);
    Pending p;
    p.buf = b;
    p.tag = tag;
    p.t_submit = t_submit >= 0.0 ? t_submit : host_now();
    p.joint = c.use_joint;
    c.queue.push_back(p);
    return TRK_OK;
}

trk_status server_step(trk_server *v, int32_t *n_active_out, int32_t *n_queued_out)
{
    if (!v) return sfail(TRK_EINVAL, "NULL server");
    trk_status st = harvest(v);
    if (st != TRK_OK) return st;
    int inflight = 0;
    for (const Tick &t : v->ring) inflight += t.in_flight ? 1 : 0;
    if (inflight >= kInflight) {  // back-pressure without blocking: admit at a later call
        int queued = 0;
        for (const CamStream &c : v->cs) queued += (int)c.queue.size();
        if (n_active_out) *n_active_out = v->n_active;
        if (n_queued_out) *n_queued_out = queued;
        return TRK_OK;
    }
    Tick &tk = v->ring[v->ring_next];
    if (tk.in_flight) {  // cannot happen with kInflight < kRing; kept as a guard
        SCU(cudaEventSynchronize(tk.ev), "tick wait");
        if ((st = harvest(v)) != TRK_OK) return st;
    }
    // admission: streams without a frame in a slot, round robin, while slots remain
    std::vector<int> admitted;
    const double now = host_now();
    for (int k = 0; k < v->max_streams && v->n_active < v->max_active; ++k) {
        const int i = (v->rr + k) % v->max_streams;
        CamStream &c = v->cs[i];
        if (!c.open || c.active || c.queue.empty()) continue;
        c.cur = c.queue.front();
        c.queue.pop_front();
        c.cur.t_admit = now;
        c.active = true;
        c.gen = 0;
        ++v->n_active;
        admitted.push_back(i);
    }
    v->rr = (v->rr + 1) % v->max_streams;
    int queued = 0;
    for (const CamStream &c : v->cs) queued += (int)c.queue.size();
    if (n_queued_out) *n_queued_out = queued;
    if (v->n_active == 0) {
        if (n_active_out) *n_active_out = 0;
        return TRK_OK;
    }
    // this tick's tables: items of every admitted frame (costliest streams first) and selections
    std::vector<int> act;
    for (int i = 0; i < v->max_streams; ++i)
        if (v->cs[i].open && v->cs[i].active) act.push_back(i);
    std::stable_sort(act.begin(), act.end(), [&](int x, int y) { return v->cs[x].cost > v->cs[y].cost; });
    char *pin = static_cast<char *>(tk.pin);
    int *sel_new = reinterpret_cast<int *>(pin);
    int *tell_last = sel_new + v->max_streams;
    int2 *items = reinterpret_cast<int2 *>(pin + tick_items_offset(v));
    int n_items = 0, n_new = 0, n_done = 0;
    std::vector<int> sel_done(act.size());
    for (int i : act)
        for (int c = 0; c < v->cs[i].es->lam; ++c) items[n_items++] = make_int2(i, c);
    for (int i : admitted) sel_new[n_new++] = i;
    for (int i : act) {
        // a frame's last generation: its update leaves out the square roots
        // (the next frame restarts from C = I) and ends with the epilogue
        const bool last = v->cs[i].gen + 1 == v->cs[i].gens;
        tell_last[i] = last ? 1 : 0;
        if (last) {
            sel_done[n_done++] = i;
            v->cs[i].es->sqrt_pending = true;
        }
    }
    // the fitness launch reads the items and flags where the host wrote them
    const char *pd = static_cast<const char *>(tk.pin_dev);
    const int *d_tell_last = reinterpret_cast<const int *>(pd) + v->max_streams;
    const int2 *d_items = reinterpret_cast<const int2 *>(pd + tick_items_offset(v));
    cudaStream_t s = v->s;
    if (n_new) SCU(cudaMemcpyAsync(tk.dev, sel_new, sizeof(int) * n_new, cudaMemcpyHostToDevice, s), "selections");
    // uploads of the newly admitted frames
    for (int i : admitted) {
        CamStream &c = v->cs[i];
        trk_tracker *t = c.es->t;
        const uint8_t *src = v->stage + v->stage_bytes * c.cur.buf;
        const size_t n = (size_t)t->cam.W * t->cam.H;
        SCU(cudaMemcpyAsync(c.es->mask_bytes, src, n, cudaMemcpyHostToDevice, s), "mask upload");
        if (c.cur.joint)
            SCU(cudaMemcpyAsync(c.es->joint, src + ((n + 15) & ~(size_t)15), sizeof(float) * 3 * t->ch.n_inst,
                                cudaMemcpyHostToDevice, s),
                "joint upload");
        SCU(launch_pack_mask(c.es->mask_bytes, c.es->mask_packed, t->cam.W, t->cam.H, t->cam.Wq, s), "pack");
        tk.release.push_back(c.cur.buf);
        c.cur.buf = -1;
    }
    SCU(launch_cma_batch(0, n_new, tk.dev, v->tb, s), "reset");
    const trk_tracker *t1 = act.size() == 1 ? v->cs[act[0]].es->t : nullptr;
    if (t1 && t1->raster == TRK_RASTER_CLUSTER) {
        // one frame in the slots: the fused per-frame kernel of
        // track_frame_device, in the tracker's own launch shape
        EvalArgs a = v->hdescs[act[0]];
        a.cma_finish = tell_last[act[0]];
        LaunchCfg lc1 = t1->lc;
        lc1.smem = std::max(lc1.smem, tell_smem_bytes());
        SCU(launch_eval(a, lc1, s), "fitness and update");
    } else {
        LaunchCfg lc = v->lc;
        int n_clusters = std::min(v->max_clusters, n_items);
        for (int c = 8; c > v->lc.cluster; --c)
            if (n_items <= v->max_clusters_by_size[c]) {
                lc.cluster = c;
                n_clusters = n_items;
                break;
            }
        SCU(launch_eval_batch(v->descs, nullptr, d_items, n_items, v->queue, lc, n_clusters, s, d_tell_last),
            "fitness and updates");
    }
    float *res = reinterpret_cast<float *>(static_cast<char *>(tk.pin) + tick_table_bytes(v));
    for (int k = 0; k < n_done; ++k) {
        CamStream &c = v->cs[sel_done[k]];
        SCU(cudaMemcpyAsync(res + k * (TRK_MAX_D + 1), c.es->pose, sizeof(float) * c.es->d, cudaMemcpyDeviceToHost, s),
            "pose download");
        SCU(cudaMemcpyAsync(res + k * (TRK_MAX_D + 1) + TRK_MAX_D, &c.es->st->best_loss, sizeof(float),
                            cudaMemcpyDeviceToHost, s),
            "loss download");
        tk.done.push_back(DoneRec{sel_done[k], c.cur.tag, c.cur.t_submit, c.cur.t_admit, c.es->d});
    }
    SCU(cudaEventRecord(tk.ev, s), "tick event");
    tk.in_flight = true;
    tk.t_enqueue = now;
    v->ring_next = (v->ring_next + 1) % kRing;
    ++v->ticks;
    for (int i : act) {
        CamStream &c = v->cs[i];
        if (++c.gen == c.gens) {
            c.active = false;
            --v->n_active;
        }
    }
    if (n_active_out) *n_active_out = v->n_active;
    return TRK_OK;
}

trk_status server_poll(trk_server *v, trk_frame_result *out, int32_t max_out, int32_t wait, int32_t *n_out)
{
    if (!v || !n_out || (max_out > 0 && !out)) return sfail(TRK_EINVAL, "NULL argument");
    if (wait) SCU(cudaStreamSynchronize(v->s), "drain");
    trk_status st = harvest(v);
    if (st != TRK_OK) return st;
    const int n = std::min<int>(max_out, (int)v->completed.size());
    for (int i = 0; i < n; ++i) out[i] = v->completed[i];
    v->completed.erase(v->completed.begin(), v->completed.begin() + n);
    *n_out = n;
    return TRK_OK;
}

trk_status server_stats(const trk_server *v, int64_t *ticks, int32_t *n_active, int32_t *n_queued,
                        int32_t *free_staging)
{
    if (!v) return sfail(TRK_EINVAL, "NULL server");
    if (ticks) *ticks = v->ticks;
    if (n_active) *n_active = v->n_active;
    int q = 0;
    for (const CamStream &c : v->cs) q += (int)c.queue.size();
    if (n_queued) *n_queued = q;
    if (free_staging) *free_staging = (int)v->free_bufs.size();
    return TRK_OK;
}

}  // extern "C"
