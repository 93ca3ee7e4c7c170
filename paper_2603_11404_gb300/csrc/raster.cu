// Fitness of a CMA-ES population in one launch (arXiv 2603.11404, Sec. III-A.2):
//   S = R(K(Pi(T_r^c T_m^r(q) v_m))),  counts (s, I, m) of S against M_ref,
//   loss of Eq. render_loss / the 1 - IoU mask error of Sec. IV-B.
//
// Launch shape: one thread-block cluster of `cluster` CTAs per candidate.
//   prologue every CTA of the cluster (in the fused CMA-ES mode) samples the
//            candidate and composes its link transforms in double-float
//            arithmetic (redundantly: no CTA waits for another).
//   phase 1  every CTA projects its share of the vertices in compensated FP32
//            (double-float, error-free TwoSum/TwoProd), snapping them to 1/256 px
//            with round-half-even; the snapped vertices go to an L2-resident
//            scratch array.
//   phase 2  after a cluster barrier the warps of all CTAs take chunks of 32
//            primitive records (edge-sharing triangle pairs, drawn as convex
//            quadrilaterals where the projected corners allow, else as their
//            triangles) from a counter in CTA 0's shared memory until none
//            are left: integer setup (orientation, top-left bias, bbox), then
//            small primitives are rasterised by one thread each with int32
//            incremental edge functions; larger ones are deferred and, after
//            a second cluster barrier, drawn by the warps of the whole
//            cluster with int64 edge functions and __ballot_sync coverage
//            words.  Coverage is OR-ed into the CTA's own full-image bitmap
//            in shared memory.
//   phase 3  after a further cluster barrier CTA r ORs band r of all the
//            cluster's bitmaps through distributed shared memory, ANDs with
//            the observed mask, popcounts, and the cluster's counts meet in
//            CTA 0, which writes counts and loss.
// No silhouette image is written to global memory.
#include <cooperative_groups.h>

#include "raster_dev.cuh"

namespace cg = cooperative_groups;

namespace trk {


// Projected keypoints of given states (synthetic detections, diagnostics):
// one warp per state composes its frames and writes (u, v) of both keypoints
// of every instrument.
__global__ void k_project_keypoints(EvalArgs a, const float *states, int n, float *out)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nI = a.ch.n_inst, nF = a.ch.n_frames;
    float2 *scr = reinterpret_cast<float2 *>(smem);
    float *sM = reinterpret_cast<float *>(scr + nI * kComposeScratch);
    const int st = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (st >= n) return;
    if (warp < nI)
        compose_frames_warp(a.ch, a.cam, states + (size_t)st * a.d + 9 * warp, sM + warp * nF * 24,
                            scr + warp * kComposeScratch, lane);
    __syncthreads();
    if (threadIdx.x < 2 * nI) {
        const int b = threadIdx.x >> 1, k = threadIdx.x & 1;
        const float2 p = project_keypoint(sM + (b * nF + a.kp_frame[k]) * 24, a.kp_pt[k], a.cam);
        out[((size_t)st * nI + b) * 4 + 2 * k] = p.x;
        out[((size_t)st * nI + b) * 4 + 2 * k + 1] = p.y;
    }
}

cudaError_t launch_project_keypoints(const EvalArgs &a, const float *states, int n, float *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const size_t smem = (size_t)a.ch.n_inst * (kComposeScratch * sizeof(float2) + a.ch.n_frames * 24 * sizeof(float));
    k_project_keypoints<<<n, 32 * a.ch.n_inst, smem, s>>>(a, states, n, out);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// The fused fitness kernel.
// ----------------------------------------------------------------------------

// One candidate c of one evaluation (all CTAs of the cluster call it together).
// mask_override replaces a.mask when not NULL (batched launches).  A non-zero
// tell_ctas is the number of CTAs that evaluate a's population in this launch:
// the last of them to finish runs the CMA-ES update (and, when a.cma_finish is
// set, the frame epilogue).
// Consecutive fused generations are launched with programmatic stream
// serialisation (see griddep_wait).
// Triangle t's vertex indices.  kChecked (meshes in the caller's device memory,
// which the host cannot validate): an index outside [0, V) marks the triangle
// bad (w = 1) and points it at vertex 0, so nothing outside the candidate's
// vertices is read; gather3 then flags it, and it is culled.
template <bool kChecked>
__device__ __forceinline__ int4 load_tri(const EvalArgs &a, int t)
{
    const int b = t >= a.T;  // instrument (at most 2): no division
    int4 tri = a.tris[t - b * a.T];
    if (kChecked) {
        const bool ok = (unsigned)tri.x < (unsigned)a.V && (unsigned)tri.y < (unsigned)a.V &&
                        (unsigned)tri.z < (unsigned)a.V;
        tri = ok ? make_int4(tri.x, tri.y, tri.z, 0) : make_int4(0, 0, 0, 1);
    }
    return tri;
}

// The three snapped vertices of a loaded triangle (written by other CTAs of
// the cluster: read through L2).
template <bool kChecked>
__device__ __forceinline__ void gather3(const int2 *sv, int4 tri, int2 &v0, int2 &v1, int2 &v2)
{
    v0 = __ldcg(sv + tri.x);
    v1 = __ldcg(sv + tri.y);
    v2 = __ldcg(sv + tri.z);
    if (kChecked && tri.w) v0.x = kSnapFlag;
}

// Chunk tickets of phase 2: lane 0 takes the next chunk from the counter in
// CTA 0's shared memory and broadcasts it.
__device__ __forceinline__ int chunk_ticket(int *ctr, int lane)
{
    int v = 0;
    if (lane == 0) v = atomicAdd(ctr, 1);
    return __shfl_sync(0xffffffffu, v, 0);
}

__device__ __forceinline__ bool small_box(int spanx, int spany) { return spanx < 32 * 256 && spany < 64 * 256; }

// One triangle of phase 2: drawn by this lane when small, otherwise deferred to
// a whole warp through the CTA's list (entry `ent`).  Returns 1 when the
// triangle is culled for a flagged vertex.
template <bool kInlineFallback>
__device__ __forceinline__ int draw_one_tri(int2 v0, int2 v1, int2 v2, int ent, const EvalArgs &a, uint32_t *bm,
                                            int *big, int *sacc)
{
    TriSetup t;
    const int st = tri_setup(v0, v1, v2, a.cam.W, a.cam.H, a.cull, t);
    if (st == 1) {
        if (small_box(t.spanx, t.spany)) {
            raster_small(t, bm, a.cam.Wq);
        } else {
            // larger triangles wait for a whole warp.  If the list is full: the
            // plain launch redraws every large primitive after the loop (raster
            // code here would make its loop spill); the batched launch,
            // compiled with more registers, draws the triangle in this lane
            const int slot = atomicAdd(&sacc[4], 1);
            if (slot < kBigListCap) big[slot] = ent;
            else if constexpr (kInlineFallback) raster_serial(t, bm, a.cam.Wq);
            else sacc[6] = 1;
        }
    }
    return st == 2;
}

// Primitive t's record and snapped corners (written by other CTAs of the
// cluster: read through L2).  A single triangle has w = -1 and no 4th corner.
__device__ __forceinline__ int4 load_prim(const EvalArgs &a, int t)
{
    const int b = t >= a.P;  // instrument (at most 2): no division
    return a.prims[t - b * a.P];
}

__device__ __forceinline__ void gather_prim(const EvalArgs &a, const int2 *snapc0, int t, int4 p, int2 &v0, int2 &v1,
                                            int2 &v2, int2 &v3)
{
    const int2 *sv = snapc0 + (t >= a.P) * a.V;
    v0 = __ldcg(sv + p.x);
    v1 = __ldcg(sv + p.y);
    v2 = __ldcg(sv + p.z);
    if (p.w >= 0) v3 = __ldcg(sv + p.w);
}

// One primitive of phase 2 drawn by this lane: a convex quadrilateral in one
// pass, anything else as its triangles; large ones are deferred to a whole
// warp.  Returns the number of its triangles culled for a flagged vertex.
template <bool kInlineFallback>
__device__ __forceinline__ int draw_prim_lane(const EvalArgs &a, int t, int d, int2 v0, int2 v1, int2 v2, int2 v3,
                                              uint32_t *bm, int *big, int *sacc)
{
    const int W = a.cam.W, H = a.cam.H, Wq = a.cam.Wq;
    int st = 3, culled = 0;
    if (d >= 0) {
        QuadSetup q;
        st = quad_setup(v0, v1, v2, v3, W, H, a.cull, q);
        if (st == 1) {
            if (small_box(q.spanx, q.spany)) {
                raster_quad_small(q, bm, Wq);
            } else {
                const int slot = atomicAdd(&sacc[4], 1);
                if (slot < kBigListCap) {
                    big[slot] = 4 * t;
                } else if constexpr (kInlineFallback) {
                    TriSetup ts;
                    if (tri_setup(v0, v1, v2, W, H, a.cull, ts) == 1) raster_serial(ts, bm, Wq);
                    if (tri_setup(v0, v2, v3, W, H, a.cull, ts) == 1) raster_serial(ts, bm, Wq);
                } else {
                    sacc[6] = 1;
                }
            }
        }
    }
    if (st == 3) {
        culled += draw_one_tri<kInlineFallback>(v0, v1, v2, 4 * t + 1, a, bm, big, sacc);
        if (d >= 0) culled += draw_one_tri<kInlineFallback>(v0, v2, v3, 4 * t + 2, a, bm, big, sacc);
    }
    return culled;
}

// One deferred entry drawn by the whole warp into this CTA's bitmap: the
// triangles of primitive ent / 4 (part 0 both, 1 the first, 2 the second), a
// pixel per lane with int64 edge functions.
__device__ __forceinline__ void draw_deferred(const EvalArgs &a, const int2 *snapc0, int ent, uint32_t *bm, int lane)
{
    const int W = a.cam.W, H = a.cam.H, Wq = a.cam.Wq;
    const int t = ent >> 2, part = ent & 3;
    const int b = t >= a.P;
    const int4 p = a.prims[t - b * a.P];
    const int2 *sv = snapc0 + b * a.V;
    const int2 u0 = __ldcg(sv + p.x), u1 = __ldcg(sv + p.y), u2 = __ldcg(sv + p.z);
    TriSetup ts;
    if (part != 2 && tri_setup(u0, u1, u2, W, H, a.cull, ts) == 1) raster_warp(ts, bm, Wq, lane);
    if (part != 1 && tri_setup(u0, u2, __ldcg(sv + p.w), W, H, a.cull, ts) == 1) raster_warp(ts, bm, Wq, lane);
}

// Phase 2 over the tracker's primitive list (quadrilateral pairs and single
// triangles, prims[] of EvalArgs).  A warp takes a chunk of 32 primitives
// (one per lane) from the cluster's counter and takes the next chunk's ticket
// while it draws: a warp holds at most one chunk beyond the one it draws, so
// the warps of a cluster run out of work together.  Deferred-list entries are
// 4 * primitive + part: part 0 the whole quadrilateral (its two triangles), 1
// its first triangle (a, b, c), 2 its second (a, c, d); they are drawn after
// the cluster barrier that follows, shared out over the whole cluster (in
// eval_candidate).  Returns this thread's count of triangles culled for a
// flagged vertex.
template <bool kInlineFallback>
__device__ __forceinline__ int draw_prims(const EvalArgs &a, cg::cluster_group &cluster, const int2 *snapc0, uint32_t *bm,
                                          int *big, int *sacc, int lane, int warp, int nwarp)
{
    const int W = a.cam.W, H = a.cam.H, Wq = a.cam.Wq;
    const int NP = a.ch.n_inst * a.P, V = a.V, P = a.P;
    int culled = 0;
    int *ctr = cluster.map_shared_rank(&sacc[5], 0);
    int cur = chunk_ticket(ctr, lane);
    while (cur * 32 < NP) {  // tickets of one warp increase: once past the end, done
        int tk = 0;
        if (lane == 0) tk = atomicAdd(ctr, 1);  // the next chunk, read after drawing this one
        const int t = cur * 32 + lane;
        if (t < NP) {
            const int4 p = load_prim(a, t);
            int2 v0, v1, v2, v3 = make_int2(0, 0);
            gather_prim(a, snapc0, t, p, v0, v1, v2, v3);
            culled += draw_prim_lane<kInlineFallback>(a, t, p.w, v0, v1, v2, v3, bm, big, sacc);
        }
        cur = __shfl_sync(0xffffffffu, tk, 0);
    }
    __syncthreads();
    if (!kInlineFallback && sacc[6]) {
        // the list overflowed: every large primitive of the candidate, a warp
        // per triangle (drawing twice is harmless under the union); a primitive
        // counts as large exactly as in the loop above
        for (int base = warp * 32; base < NP; base += nwarp * 32) {
            const int tt = base + lane;
            bool l1 = false, l2 = false;
            if (tt < NP) {
                const int b = tt >= P;
                const int4 p = a.prims[tt - b * P];
                const int2 *sv = snapc0 + b * V;
                const int2 u0 = __ldcg(sv + p.x), u1 = __ldcg(sv + p.y), u2 = __ldcg(sv + p.z);
                int st = 3;
                if (p.w >= 0) {
                    const int2 u3 = __ldcg(sv + p.w);
                    QuadSetup q;
                    st = quad_setup(u0, u1, u2, u3, W, H, a.cull, q);
                    if (st == 1) l1 = l2 = !small_box(q.spanx, q.spany);
                    if (st == 3) {
                        TriSetup ts;
                        l2 = tri_setup(u0, u2, u3, W, H, a.cull, ts) == 1 && !small_box(ts.spanx, ts.spany);
                    }
                }
                if (st == 3) {
                    TriSetup ts;
                    l1 = tri_setup(u0, u1, u2, W, H, a.cull, ts) == 1 && !small_box(ts.spanx, ts.spany);
                }
            }
            for (int part = 1; part <= 2; ++part)
                for (unsigned mm = __ballot_sync(0xffffffffu, part == 1 ? l1 : l2); mm; mm &= mm - 1) {
                    const int tu = __shfl_sync(0xffffffffu, tt, __ffs(mm) - 1);
                    const int b = tu >= P;
                    const int4 p = a.prims[tu - b * P];
                    const int2 *sv = snapc0 + b * V;
                    const int2 u0 = __ldcg(sv + p.x);
                    const int2 u1 = __ldcg(sv + (part == 1 ? p.y : p.z));
                    const int2 u2 = __ldcg(sv + (part == 1 ? p.z : p.w));
                    TriSetup ts;
                    if (tri_setup(u0, u1, u2, W, H, a.cull, ts) == 1) raster_warp(ts, bm, Wq, lane);
                }
        }
    }
    return culled;
}

// Phase 2 over plain triangles (tris[] of EvalArgs; the index-checked launch on
// meshes in caller memory).  Deferred-list entries are triangle indices.
template <bool kInlineFallback, bool kChecked>
__device__ __forceinline__ int draw_tris(const EvalArgs &a, cg::cluster_group &cluster, const int2 *snapc, uint32_t *bm,
                                      int *big, int *sacc, int lane, int warp, int nwarp)
{
    const int W = a.cam.W, H = a.cam.H, Wq = a.cam.Wq;
    int culled = 0;
    const int NT = a.ch.n_inst * a.T;
    int *ctr = cluster.map_shared_rank(&sacc[5], 0);
    int cur = chunk_ticket(ctr, lane), nx1 = chunk_ticket(ctr, lane), nx2 = chunk_ticket(ctr, lane);
    int t0 = cur * 32 + lane, t1 = nx1 * 32 + lane;
    int4 tri1 = make_int4(0, 0, 0, 0);
    int b1 = 0;
    int2 v0 = make_int2(0, 0), v1 = v0, v2 = v0;
    if (t0 < NT) {
        const int b0 = t0 >= a.T;  // instrument (at most 2): no division
        gather3<kChecked>(snapc + b0 * a.V, load_tri<kChecked>(a, t0), v0, v1, v2);
    }
    if (t1 < NT) {
        b1 = t1 >= a.T;
        tri1 = load_tri<kChecked>(a, t1);
    }
    while (cur * 32 < NT) {
        const int nx3 = chunk_ticket(ctr, lane);
        int2 w0 = make_int2(0, 0), w1 = w0, w2 = w0;
        if (t1 < NT) gather3<kChecked>(snapc + b1 * a.V, tri1, w0, w1, w2);
        const int t2 = nx2 * 32 + lane;
        int4 tri2 = make_int4(0, 0, 0, 0);
        int b2 = 0;
        if (t2 < NT) {
            b2 = t2 >= a.T;
            tri2 = load_tri<kChecked>(a, t2);
        }
        if (t0 < NT) culled += draw_one_tri<kInlineFallback>(v0, v1, v2, t0, a, bm, big, sacc);
        cur = nx1;
        t0 = t1;
        v0 = w0;
        v1 = w1;
        v2 = w2;
        nx1 = nx2;
        t1 = t2;
        tri1 = tri2;
        b1 = b2;
        nx2 = nx3;
    }
    __syncthreads();
    const int nbig = min(sacc[4], kBigListCap);
    for (int e = warp; e < nbig; e += nwarp) {
        int tt = big[e];
        int b = tt >= a.T;
        int2 u0, u1, u2;
        gather3<kChecked>(snapc + b * a.V, load_tri<kChecked>(a, tt), u0, u1, u2);
        TriSetup t;
        tri_setup(u0, u1, u2, W, H, a.cull, t);
        raster_warp(t, bm, Wq, lane);
    }
    if (!kInlineFallback && sacc[6]) {  // the list overflowed: every large triangle of the candidate, a warp each (drawing twice is harmless)
        for (int base = warp * 32; base < NT; base += nwarp * 32) {
            const int tt = base + lane;
            bool large = false;
            TriSetup t;
            if (tt < NT) {
                const int b = tt >= a.T;
                int2 u0, u1, u2;
                gather3<kChecked>(snapc + b * a.V, load_tri<kChecked>(a, tt), u0, u1, u2);
                large = tri_setup(u0, u1, u2, W, H, a.cull, t) == 1 && !small_box(t.spanx, t.spany);
            }
            for (unsigned mm = __ballot_sync(0xffffffffu, large); mm; mm &= mm - 1) {
                const int src = __ffs(mm) - 1, tu = __shfl_sync(0xffffffffu, tt, src);
                const int b = tu >= a.T;
                int2 u0, u1, u2;
                gather3<kChecked>(snapc + b * a.V, load_tri<kChecked>(a, tu), u0, u1, u2);
                TriSetup u;
                tri_setup(u0, u1, u2, W, H, a.cull, u);
                raster_warp(u, bm, Wq, lane);
            }
        }
    }
    return culled;
}

template <bool kInlineFallback, bool kChecked = false, bool kQuads = true>
__device__ __forceinline__ void eval_candidate(const EvalArgs &a, int c, const uint32_t *mask_override,
                                               unsigned tell_ctas, bool dependent_launch)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int K = (int)cluster.num_blocks();
    const uint32_t *maskp = mask_override ? mask_override : a.mask;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int nI = a.ch.n_inst, nF = a.ch.n_frames;
    const int H = a.cam.H, Wq = a.cam.Wq;
    const int nwords = H * Wq;

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *scr = reinterpret_cast<float2 *>(smem);                           // [nI*kComposeScratch]
    uint32_t *bm = reinterpret_cast<uint32_t *>(scr + nI * kComposeScratch);  // [H*Wq]
    float *sM = reinterpret_cast<float *>(bm + ((nwords + 3) & ~3));          // [nI*nF*24]
    int *big = reinterpret_cast<int *>(sM + nI * nF * 24);                    // [kBigListCap]
    // [8]: s I m culled, big-list count, chunk ticket counter, big-list
    // overflow, deferred-entry ticket counter
    int *sacc = big + kBigListCap;
    __shared__ int red[4][32];
    __shared__ float s_par[kMaxD];
    __shared__ float2 s_z[kMaxD];
    __shared__ int s_last;

    {  // the warps that do not compose frames clear the bitmap (16-byte stores)
        const int c0 = nwarp > nI ? 32 * nI : 0;
        uint4 *bm4 = reinterpret_cast<uint4 *>(bm);
        for (int w = tid - c0; w >= 0 && w < (nwords + 3) >> 2; w += nthr - c0) bm4[w] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid < 8) sacc[tid] = 0;
    // everything above touches only this CTA's shared memory; from here on the
    // launch reads what the previous generation wrote
    if (dependent_launch) griddep_wait();
    // ---- prologue: every CTA samples the candidate (fused CMA-ES mode; the
    //      draws are the same in every CTA and CTA 0 stores them) and composes
    //      its frames in double-float, so no CTA waits for another ----
    {
        const float *par = a.params + (size_t)c * a.d;
        if (a.cma_st) {
            if (warp == 0) {
                const bool owner = rank == 0;
                cma_sample_warp(*a.cma_k, a.cma_st, c, nullptr, owner ? a.cma_y : nullptr,
                                owner ? a.cma_z : nullptr, owner ? const_cast<float *>(a.params) : nullptr, s_par,
                                s_z, lane);
            }
            __syncthreads();
            par = s_par;
        }
        if (warp < nI)
            compose_frames_warp(a.ch, a.cam, par + 9 * warp, sM + warp * nF * 24, scr + warp * kComposeScratch,
                                lane);
        if (rank == 0 && warp == nwarp - 1) check_state_finite(par, a.d, a.err, lane);
    }
    __syncthreads();

    // ---- phase 1: project and snap this CTA's share of the vertices, two in flight ----
    const int gtid = rank * nthr + tid, gstride = K * nthr;
    int2 *snapc = a.snap + (size_t)c * nI * a.V;
    const int NV = nI * a.V;
    for (int idx0 = gtid; idx0 < NV; idx0 += 2 * gstride) {
        const int idx1 = idx0 + gstride;
        const bool has1 = idx1 < NV;
        int b0 = idx0 >= a.V, b1 = has1 ? (idx1 >= a.V) : b0;  // instrument (at most 2): no division
        float4 p0 = a.verts[idx0 - b0 * a.V];
        float4 p1 = has1 ? a.verts[idx1 - b1 * a.V] : p0;
        float2 uv0, uv1;
        int2 o0, o1;
        const int f0 = (int)p0.w, f1 = (int)p1.w;
        if (kChecked && !((unsigned)f0 < (unsigned)nF && (float)f0 == p0.w)) {  // a frame index out of range: flagged
            o0 = make_int2(kSnapFlag, kSnapFlag);
            uv0 = make_float2(0.0f, 0.0f);
        } else {
            o0 = project_vertex(p0, sM + (b0 * nF + f0) * 24, a.cam, uv0);
        }
        if (kChecked && !((unsigned)f1 < (unsigned)nF && (float)f1 == p1.w)) {
            o1 = make_int2(kSnapFlag, kSnapFlag);
            uv1 = make_float2(0.0f, 0.0f);
        } else {
            o1 = project_vertex(p1, sM + (b1 * nF + f1) * 24, a.cam, uv1);
        }
        snapc[idx0] = o0;
        if (a.snap_dbg) a.snap_dbg[(size_t)c * NV + idx0] = o0;
        if (a.uv_dbg) a.uv_dbg[(size_t)c * NV + idx0] = uv0;
        if (has1) {
            snapc[idx1] = o1;
            if (a.snap_dbg) a.snap_dbg[(size_t)c * NV + idx1] = o1;
            if (a.uv_dbg) a.uv_dbg[(size_t)c * NV + idx1] = uv1;
        }
    }
    cluster.sync();  // arrive.release / wait.acquire: the snapped vertices are visible cluster-wide

    // ---- phase 2: primitives -> this CTA's bitmap.  Warps of the whole cluster
    //      take chunks of 32 primitives (one per lane) from a counter in CTA 0's
    //      shared memory, so the cluster finishes together whatever they cost;
    //      the bitmaps are OR-ed in phase 3, so which CTA draws a primitive does
    //      not change the result ----
    int culled = kQuads ? draw_prims<kInlineFallback>(a, cluster, snapc, bm, big, sacc, lane, warp, nwarp)
                        : draw_tris<kInlineFallback, kChecked>(a, cluster, snapc, bm, big, sacc, lane, warp, nwarp);
    cluster.sync();
    if (kQuads) {
        // the large primitives deferred by every CTA of the cluster, shared out
        // over all its warps: the tip of a coarse mesh close to the camera lands
        // in a few chunks, and a CTA drawing its own list alone would hold the
        // whole cluster up.  Entry e of the cluster is entry e - start(r) of
        // CTA r's list (lists read through DSMEM, complete at the barrier above)
        const int cnt = lane < K ? min(*cluster.map_shared_rank(&sacc[4], lane), kBigListCap) : 0;
        int incl = cnt;
        for (int o = 1; o < 8; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 7);
        if (total > 0) {  // the same in every CTA: the barrier below is uniform
            int *ctr = cluster.map_shared_rank(&sacc[7], 0);
            for (int e = chunk_ticket(ctr, lane); e < total; e = chunk_ticket(ctr, lane)) {
                const int r = __popc(__ballot_sync(0xffffffffu, lane < K && incl <= e));
                const int start = __shfl_sync(0xffffffffu, incl - cnt, r);
                const int ent = cluster.map_shared_rank(big, r)[e - start];
                draw_deferred(a, snapc, ent, bm, lane);
            }
            cluster.sync();  // every deferred primitive drawn before the bitmaps are read
        }
    }

    // ---- phase 3: OR the cluster's bitmaps over this CTA's band, count ----
    const int per = (nwords + K - 1) / K;
    const int w0 = rank * per, w1 = min(nwords, w0 + per);
    const uint32_t *rbm[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) rbm[q] = cluster.map_shared_rank(bm, q < K ? q : 0);
    int s = 0, I = 0, m = 0;
    for (int w = w0 + tid; w < w1; w += nthr) {
        uint32_t part[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) part[q] = (q < K) ? rbm[q][w] : 0u;
        uint32_t M = maskp[w];
        uint32_t S = 0u;
#pragma unroll
        for (int q = 0; q < 8; ++q) S |= part[q];
        s += __popc(S);
        I += __popc(S & M);
        m += __popc(M);
        if (a.silhouette) a.silhouette[w] = S;
    }
    for (int o = 16; o; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        I += __shfl_xor_sync(0xffffffffu, I, o);
        m += __shfl_xor_sync(0xffffffffu, m, o);
        culled += __shfl_xor_sync(0xffffffffu, culled, o);
    }
    if (lane == 0) {
        red[0][warp] = s;
        red[1][warp] = I;
        red[2][warp] = m;
        red[3][warp] = culled;
    }
    __syncthreads();
    if (tid < 4) {
        int acc = 0;
        for (int w = 0; w < nwarp; ++w) acc += red[tid][w];
        atomicAdd(cluster.map_shared_rank(&sacc[tid], 0), acc);
    }
    cluster.sync();
    if (rank == 0 && tid == 0) {
        int S_ = sacc[0], I_ = sacc[1], M_ = sacc[2], C_ = sacc[3];
        if (a.counts) {
            a.counts[4 * c + 0] = S_;
            a.counts[4 * c + 1] = I_;
            a.counts[4 * c + 2] = M_;
            a.counts[4 * c + 3] = C_;
        }
        if (a.loss) {
            int x = S_ + M_ - 2 * I_;
            float L;
            if (a.loss_kind == TRK_LOSS_ONE_MINUS_IOU) {
                int U = S_ + M_ - I_;
                L = (U > 0) ? __fsub_rn(1.0f, __fdiv_rn((float)I_, (float)U)) : 0.0f;
            } else if (a.loss_kind == TRK_LOSS_MSE_APP) {
                L = __fadd_rn((float)x, __fmul_rn(a.lambda_app, (float)abs(S_ - M_)));
            } else {
                L = (float)x;
            }
            if (a.kp_obs && a.kp_lambda != 0.0f) L = __fadd_rn(L, keypoint_loss(a, sM));
            a.loss[c] = L;
        }
    }
    if (a.cma_st && tell_ctas) {  // the last CTA to finish updates the search distribution
        if (tid == 0) {
            __threadfence();
            unsigned ticket = atomicAdd(a.cma_done, 1u);
            s_last = (ticket == tell_ctas - 1);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            TellSmem &S = *reinterpret_cast<TellSmem *>(smem);  // the cluster no longer reads this CTA's smem
            // a frame's last generation leaves out the square roots: the next
            // frame restarts from C = I (the host runs them if it does not)
            cma_tell_block(*a.cma_k, a.cma_st, a.cma_y, a.params, a.loss, S, tid, nthr, !a.cma_finish);
            __syncthreads();
            if (a.cma_finish) cma_finish_frame(*a.cma_k, a.cma_st, a.cma_pose_out, tid, nthr);
            if (tid == 0) *a.cma_done = 0u;
        }
    }
}

__global__ void __launch_bounds__(256, 4) k_eval(EvalArgs a)
{
    griddep_launch_dependents();
    eval_candidate<false>(a, blockIdx.y, nullptr, gridDim.x * gridDim.y, true);
}

// The same with index checks: meshes in the caller's device memory
// (eval_population_noalloc), whose indices the host cannot validate.
__global__ void __launch_bounds__(256, 4) k_eval_checked(EvalArgs a)
{
    eval_candidate<false, true, false>(a, blockIdx.y, nullptr, 0u, false);
}

// Persistent batched evaluation: a fixed grid of clusters pulls (instance,
// candidate) items from a queue (largest first) until it is empty.  CTA 0 of
// each cluster takes the ticket and the others read it through DSMEM, so the
// cluster stays in lockstep.  kTell (serving ticks): tell_last holds one flag
// per instance (1 for a frame's last generation) and the last CTA of each
// instance's items runs that instance's CMA-ES update, as k_eval does for one
// instance; items and flags sit in mapped pinned host memory that the host
// rewrites between ticks (read with ld.cv, never from a cached line), and the
// cluster that draws the launch's last ticket leaves the queue counter at zero
// for the next tick.  Without kTell the updates are a separate launch.
template <bool kTell>
__global__ void __launch_bounds__(256, 3) k_eval_batch(const EvalArgs *descs, const uint32_t *const *masks,
                                                       const int2 *items, int n_items, unsigned *next_item,
                                                       const int *tell_last)
{
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ int s_item;
    __shared__ int s_tick[3];  // kTell: the item and its instance's flag, read once by CTA 0's thread 0
    __shared__ __align__(16) EvalArgs s_args;  // this item's descriptor, read from shared memory
    for (;;) {
        if (cluster.block_rank() == 0 && threadIdx.x == 0) {
            s_item = (int)atomicAdd(next_item, 1u);
            if (kTell && s_item < n_items) {
                const int2 v = __ldcv(items + s_item);
                s_tick[0] = v.x;
                s_tick[1] = v.y;
                s_tick[2] = __ldcv(tell_last + v.x);
            }
        }
        cluster.sync();
        const int it = *cluster.map_shared_rank(&s_item, 0);
        int2 ic = make_int2(0, 0);
        int last = 0;
        if (kTell && it < n_items) {
            const int *t0 = cluster.map_shared_rank(s_tick, 0);
            ic = make_int2(t0[0], t0[1]);
            last = t0[2];
        }
        cluster.sync();  // every CTA has its ticket before CTA 0 takes the next
        if (it >= n_items) {
            // every cluster draws exactly one ticket past the items: the last of
            // them is the launch's last atomic on the counter
            if (kTell && cluster.block_rank() == 0 && threadIdx.x == 0 && it == n_items + (int)gridDim.y - 1)
                *next_item = 0u;
            break;
        }
        if (!kTell) ic = items[it];
        const int4 *src = reinterpret_cast<const int4 *>(descs + ic.x);
        int4 *dst = reinterpret_cast<int4 *>(&s_args);
        for (int i = threadIdx.x; i < (int)(sizeof(EvalArgs) / 16); i += blockDim.x) dst[i] = src[i];
        __syncthreads();
        unsigned tell = 0;
        if (kTell) {
            if (threadIdx.x == 0) s_args.cma_finish = last;
            __syncthreads();
            tell = (unsigned)s_args.lam * gridDim.x;  // every CTA of every candidate of the instance
        }
        eval_candidate<true>(s_args, ic.y, masks ? masks[ic.x] : nullptr, tell, false);
    }
}

cudaError_t launch_eval_batch(const EvalArgs *descs_dev, const uint32_t *const *masks_dev, const int2 *items_dev,
                              int n_items, unsigned *next_item_dev, const LaunchCfg &cfg, int n_clusters,
                              cudaStream_t s, const int *tell_last_dev)
{
    if (n_items == 0) return cudaSuccess;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.cluster, n_clusters, 1);
    lc.blockDim = dim3(cfg.threads, 1, 1);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cfg.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return tell_last_dev ? cudaLaunchKernelEx(&lc, k_eval_batch<true>, descs_dev, masks_dev, items_dev, n_items,
                                              next_item_dev, tell_last_dev)
                         : cudaLaunchKernelEx(&lc, k_eval_batch<false>, descs_dev, masks_dev, items_dev, n_items,
                                              next_item_dev, tell_last_dev);
}

cudaError_t prepare_eval_batch(size_t smem, int cluster, int threads, int *max_clusters)
{
    cudaError_t e = ensure_smem_attr((const void *)k_eval_batch<false>, smem);
    if (e == cudaSuccess) e = ensure_smem_attr((const void *)k_eval_batch<true>, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cluster, 1, 1);
    lc.blockDim = dim3(threads, 1, 1);
    lc.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    // both forms (with and without the fused updates) must fit the shape
    int with_tell = 0;
    if ((e = cudaOccupancyMaxActiveClusters(max_clusters, k_eval_batch<false>, &lc)) != cudaSuccess ||
        (e = cudaOccupancyMaxActiveClusters(&with_tell, k_eval_batch<true>, &lc)) != cudaSuccess)
        return e;
    *max_clusters = std::min(*max_clusters, with_tell);
    return cudaSuccess;
}

size_t tell_smem_bytes() { return sizeof(TellSmem); }

size_t eval_smem_bytes(const EvalArgs &a)
{
    size_t nwords = (size_t)a.cam.H * a.cam.Wq;
    return (size_t)a.ch.n_inst * kComposeScratch * sizeof(float2) + ((nwords + 3) & ~(size_t)3) * 4 +
           (size_t)a.ch.n_inst * a.ch.n_frames * 24 * 4 + (size_t)kBigListCap * 4 + 8 * 4;
}

int eval_max_threads() { return 1024; }

cudaError_t prepare_eval(size_t smem) { return ensure_smem_attr((const void *)k_eval, smem); }

cudaError_t launch_eval_checked(const EvalArgs &a, const LaunchCfg &cfg, cudaStream_t s)
{
    if (a.lam == 0) return cudaSuccess;
    cudaError_t e = ensure_smem_attr((const void *)k_eval_checked, cfg.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.cluster, a.lam, 1);
    lc.blockDim = dim3(cfg.threads, 1, 1);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cfg.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    return cudaLaunchKernelEx(&lc, k_eval_checked, a);
}

cudaError_t launch_eval(const EvalArgs &a, const LaunchCfg &cfg, cudaStream_t s)
{
    if (a.lam == 0) return cudaSuccess;
    if (!a.prims) return cudaErrorInvalidValue;  // k_eval draws the primitive records (apply_mesh)
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.cluster, a.lam, 1);
    lc.blockDim = dim3(cfg.threads, 1, 1);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cfg.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    // fused generations follow each other: overlap the next one's launch with
    // this one's tail (see griddep_wait)
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = a.cma_st ? 1 : 0;
    lc.attrs = attr;
    lc.numAttrs = 2;
    return cudaLaunchKernelEx(&lc, k_eval, a);
}

// ----------------------------------------------------------------------------
// Mask packing: one warp per 32-pixel word, coverage by __ballot_sync.
// ----------------------------------------------------------------------------
__global__ void k_pack_mask(const uint8_t *mask, uint32_t *packed, int W, int H, int Wq)
{
    long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (gw >= (long long)H * Wq) return;
    int i = (int)(gw / Wq), w = (int)(gw - (long long)i * Wq);
    int j = w * 32 + lane;
    bool on = (j < W) && mask[(size_t)i * W + j] != 0;
    unsigned b = __ballot_sync(0xffffffffu, on);
    if (lane == 0) packed[gw] = b;
}

cudaError_t launch_pack_mask(const uint8_t *mask, uint32_t *packed, int W, int H, int Wq, cudaStream_t s)
{
    long long threads = (long long)H * Wq * 32;
    int blocks = (int)((threads + 255) / 256);
    if (blocks == 0) return cudaSuccess;
    k_pack_mask<<<blocks, 256, 0, s>>>(mask, packed, W, H, Wq);
    return cudaGetLastError();
}

}  // namespace trk
