// Fitness of a CMA-ES population by a binned, tiled rasteriser (arXiv
// 2603.11404, Sec. III-A.2): S = R(K(Pi(T_r^c T_m^r(q) v_m))), counts (s, I, m)
// of S against M_ref and the loss of Eq. render_loss / the 1 - IoU mask error
// of Sec. IV-B.  Two launches per evaluation, both with programmatic stream
// serialisation so each is resident before its predecessor ends:
//
// k_front  one thread-block cluster per candidate.
//   prologue  every CTA samples the candidate (fused CMA-ES mode) and composes
//             its frames in double-float arithmetic; CTA 0 keeps the frames
//             for the keypoint term; every CTA popcounts a slice of the mask.
//   phase 1   the cluster projects and snaps the candidate's vertices to an
//             L2-resident scratch array (compensated FP32, round-half-even).
//   phase 2   after a cluster barrier each thread sets up a fixed share of the
//             triangles (orientation, top-left bias, clipped pixel box); the
//             live ones (box holding a pixel centre) are compacted into the
//             CTA's shared-memory list and counted per screen tile.
//   phase 3   after a second barrier every CTA reads all the cluster's tile
//             counts through distributed shared memory and scans them: an
//             exact counting sort, so each tile's bin is one contiguous run of
//             the candidate's pool.  The CTA that owns a tile records it and
//             appends one work item per kBinChunk entries of its bin.
//   phase 4   after a third barrier each CTA scatters its live triangles
//             (their three snapped vertices, oriented) into the bins of the
//             tiles their boxes touch.
// k_tiles  a persistent grid over the work items (whole GPU).  An item is up
//   to kBinChunk triangles of one tile's bin; the warps of a CTA take them 32
//   at a time (each triangle: the three snapped vertices stored in the bin).
//   One thread sets up a triangle again, clips its box to the tile and
//   rasterises it with int32 incremental edge functions into its warp's
//   32 x 64-pixel shared-memory tile bitmap; triangles too large for that go
//   to a warp that covers 32 pixels per step with int64 edges and
//   __ballot_sync.  The warps' bitmaps are OR-ed.  A tile drawn by one item is popcounted against
//   the mask at once; the items of a larger bin OR their words into an
//   L2-resident tile and the last of them counts it.  Counts meet in per-
//   candidate integer accumulators; the last CTA to leave writes every loss
//   (and, for a fused CMA-ES generation, runs the update).
// No silhouette image is written to global memory (except on request by
// tracker_render).  Counts are exact integers, so the result does not depend
// on which CTA draws a triangle or in which order.
#include <cooperative_groups.h>

#include <mutex>
#include <vector>

#include "raster_dev.cuh"

namespace cg = cooperative_groups;

namespace trk {

// Inclusive warp scan of v.
__device__ __forceinline__ int warp_incl_scan(int v, int lane)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// The front kernel.
// ---------------------------------------------------------------------------
// Order a live triangle's vertices as tri_setup does (positive orientation
// under the edge functions), so the tile kernel can skip that step.
__device__ __forceinline__ void orient(int2 &a, int2 &b, int2 &c)
{
    const int spanx = max(a.x, max(b.x, c.x)) - min(a.x, min(b.x, c.x));
    const int spany = max(a.y, max(b.y, c.y)) - min(a.y, min(b.y, c.y));
    long long A;
    if (spanx < (1 << 15) && spany < (1 << 15))
        A = (long long)((b.x - a.x) * (c.y - a.y) - (c.x - a.x) * (b.y - a.y));
    else
        A = (long long)(b.x - a.x) * (long long)(c.y - a.y) - (long long)(c.x - a.x) * (long long)(b.y - a.y);
    if (A < 0) {
        const int2 tmp = b;
        b = c;
        c = tmp;
    }
}
// The three snapped vertices of triangle t of the candidate (snapc: its
// vertices; written by other CTAs of the cluster, so read through L2).
__device__ __forceinline__ void tri_vertices(const EvalArgs &a, const int2 *snapc, int4 tri, int b, int2 &v0,
                                             int2 &v1, int2 &v2)
{
    const int2 *sv = snapc + b * a.V;
    v0 = __ldcg(sv + tri.x);
    v1 = __ldcg(sv + tri.y);
    v2 = __ldcg(sv + tri.z);
}

__global__ void __launch_bounds__(256, 4) k_front(EvalArgs a)
{
    griddep_launch_dependents();
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int K = (int)cluster.num_blocks();
    const int c = blockIdx.y;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int nI = a.ch.n_inst, nF = a.ch.n_frames;
    const int W = a.cam.W, H = a.cam.H, Wq = a.cam.Wq;
    const int nT = a.bin.n_tiles, ntx = a.bin.n_tx;

    extern __shared__ __align__(16) unsigned char smem[];
    float2 *scr = reinterpret_cast<float2 *>(smem);                          // [nI * kComposeScratch]
    float *sM = reinterpret_cast<float *>(scr + nI * kComposeScratch);       // [nI * nF * 24]
    int *cnt = reinterpret_cast<int *>(sM + nI * nF * 24);                   // [nT] this CTA's tile counts
    int *cur = cnt + nT;                                                     // [nT] scatter cursors
    int *tot = cur + nT;                                                     // [nT] tile totals, then bases
    int2 *live = reinterpret_cast<int2 *>(tot + ((nT + 1) & ~1));            // [live_cap] (triangle, tiles)
    __shared__ ChainDev s_ch;  // the chain in shared memory: the lanes of a warp read different entries
    __shared__ int s_nlive, s_grand;
    __shared__ int s_red[32];
    __shared__ float s_par[kMaxD];
    __shared__ float2 s_z[kMaxD];

    {
        const int2 *src = reinterpret_cast<const int2 *>(&a.ch);
        int2 *dst = reinterpret_cast<int2 *>(&s_ch);
        for (int i = tid; i < (int)(sizeof(ChainDev) / sizeof(int2)); i += nthr) dst[i] = src[i];
    }
    for (int i = tid; i < nT; i += nthr) cnt[i] = 0;
    if (tid == 0) s_nlive = 0;
    __syncthreads();
    // everything above touches only this CTA's shared memory; from here on the
    // launch reads and writes what the previous kernel on the stream used
    griddep_wait();
    if (rank == 0 && tid < 4) a.bin.acc[4 * c + tid] = 0;
    const int nwords = H * Wq;
    if (a.silhouette)  // render mode (one candidate): tiles without triangles stay empty
        for (int w = rank * nthr + tid; w < nwords; w += K * nthr) a.silhouette[w] = 0u;
    {  // m = popcount of the observed mask, a slice per CTA of the launch
        const int q = c * K + rank, nq = (int)gridDim.y * K;
        int mm = 0;
        for (int w = q * nthr + tid; w < nwords; w += nq * nthr) mm += __popc(a.mask[w]);
        mm = warp_sum(mm);
        if (lane == 0 && mm) atomicAdd(&a.bin.ctl[3], (unsigned)mm);
    }

    // ---- prologue: sample (fused CMA-ES mode: the draws are the same in
    //      every CTA and CTA 0 stores them) and compose the candidate's frames ----
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
            compose_frames_warp(s_ch, a.cam, par + 9 * warp, sM + warp * nF * 24, scr + warp * kComposeScratch, lane);
        if (rank == 0 && warp == nwarp - 1) check_state_finite(par, a.d, a.err, lane);
    }
    __syncthreads();
    if (rank == 0)
        for (int i = tid; i < nI * nF * 24; i += nthr) a.bin.frames[(size_t)c * nI * nF * 24 + i] = sM[i];

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
        int2 o0 = project_vertex(p0, sM + (b0 * nF + (int)p0.w) * 24, a.cam, uv0);
        int2 o1 = project_vertex(p1, sM + (b1 * nF + (int)p1.w) * 24, a.cam, uv1);
        snapc[idx0] = o0;
        if (a.snap_dbg) a.snap_dbg[(size_t)c * NV + idx0] = o0;
        if (a.uv_dbg) a.uv_dbg[(size_t)c * NV + idx0] = uv0;
        if (has1) {
            snapc[idx1] = o1;
            if (a.snap_dbg) a.snap_dbg[(size_t)c * NV + idx1] = o1;
            if (a.uv_dbg) a.uv_dbg[(size_t)c * NV + idx1] = uv1;
        }
    }
    cluster.sync();  // the snapped vertices are visible cluster-wide

    // ---- phase 2: set-up of a fixed share of the triangles (warp-uniform
    //      trip counts, so the ballots below see every lane), software-
    //      pipelined: the vertices of the next triangle and the indices of the
    //      one after are in flight while a triangle is set up ----
    int culled = 0;
    const int NT = nI * a.T;
    {
        const int tw0 = rank * nthr + warp * 32;
        int tA = tw0 + lane, tB = tA + gstride;
        int4 triB = make_int4(0, 0, 0, 0);
        int2 a0 = make_int2(0, 0), a1 = a0, a2 = a0;
        if (tA < NT) {
            const int b = tA >= a.T;
            tri_vertices(a, snapc, a.tris[tA - b * a.T], b, a0, a1, a2);
        }
        if (tB < NT) triB = a.tris[tB - (tB >= a.T) * a.T];
        for (int tw = tw0; tw < NT; tw += gstride) {
            const int t = tw + lane, tC = tB + gstride;
            int4 triC = make_int4(0, 0, 0, 0);
            if (tC < NT) triC = a.tris[tC - (tC >= a.T) * a.T];
            int2 b0 = make_int2(0, 0), b1 = b0, b2 = b0;
            if (tB < NT) tri_vertices(a, snapc, triB, tB >= a.T, b0, b1, b2);
            bool is_live = false;
            int pk = 0;
            if (t < NT) {
                TriSetup ts;
                const int st = tri_setup(a0, a1, a2, W, H, a.cull, ts);
                culled += st == 2;
                if (st == 1) {
                    is_live = true;
                    const int tx0 = ts.j0 / kTileW, tx1 = ts.j1 / kTileW, ty0 = ts.i0 / kTileH, ty1 = ts.i1 / kTileH;
                    pk = tx0 | (tx1 << 8) | (ty0 << 16) | (ty1 << 24);
                    for (int ty = ty0; ty <= ty1; ++ty)
                        for (int tx = tx0; tx <= tx1; ++tx) atomicAdd(&cnt[ty * ntx + tx], 1);
                }
            }
            const unsigned lm = __ballot_sync(0xffffffffu, is_live);
            int base = 0;
            if (lane == 0 && lm) base = atomicAdd(&s_nlive, __popc(lm));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (is_live) live[base + __popc(lm & ((1u << lane) - 1u))] = make_int2(t, pk);
            a0 = b0;
            a1 = b1;
            a2 = b2;
            tB = tC;
            triB = triC;
        }
    }
    culled = warp_sum(culled);
    if (lane == 0) s_red[warp] = culled;
    __syncthreads();
    if (tid == 0) {
        int sum = 0;
        for (int w = 0; w < nwarp; ++w) sum += s_red[w];
        if (sum) atomicAdd(&a.bin.acc[4 * c + 2], sum);
    }
    cluster.sync();  // every CTA's tile counts are final

    // ---- phase 3: the counting sort's offsets.  tot[tile] = the cluster's
    //      entries in the tile, cur[tile] = those of lower-ranked CTAs ----
    for (int i = tid; i < nT; i += nthr) {
        int total = 0, before = 0;
        for (int q = 0; q < K; ++q) {
            const int v = cluster.map_shared_rank(cnt, q)[i];
            total += v;
            before += q < rank ? v : 0;
        }
        tot[i] = total;
        cur[i] = before;
    }
    __syncthreads();
    {  // exclusive scan of tot over the tiles, in place; s_grand = all entries
        const int per = (nT + nthr - 1) / nthr;
        const int i0 = min(nT, tid * per), i1 = min(nT, i0 + per);
        int sum = 0;
        for (int i = i0; i < i1; ++i) sum += tot[i];
        const int incl = warp_incl_scan(sum, lane);
        __syncthreads();  // s_red is reused
        if (lane == 31) s_red[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const int v = lane < nwarp ? s_red[lane] : 0;
            const int wi = warp_incl_scan(v, lane);
            if (lane < nwarp) s_red[lane] = wi - v;  // exclusive prefix of the warps
            if (lane == nwarp - 1) s_grand = wi;
        }
        __syncthreads();
        int run = s_red[warp] + incl - sum;
        for (int i = i0; i < i1; ++i) {
            const int v = tot[i];
            tot[i] = run;
            cur[i] += run;
            run += v;
        }
    }
    __syncthreads();
    const int grand = s_grand;
    const bool ovf = grand > a.bin.pool_cap;  // bins do not fit: draw the tiles from every triangle
    // tiles owned by this CTA (tile % K == rank): append their work items, one
    // per kBinChunk records of the tile's bin (or one drawing the tile from
    // every triangle: zero chunks)
    for (int j0 = 0; rank + K * j0 < nT; j0 += nthr) {
        const int tile = rank + K * (j0 + tid);
        int n = 0, first = 0, count = 0;
        if (tile < nT) {
            first = tot[tile];
            count = (tile + 1 < nT ? tot[tile + 1] : grand) - first;
            n = count == 0 ? 0 : (ovf ? 1 : (count + kBinChunk - 1) / kBinChunk);
        }
        const int incl = warp_incl_scan(n, lane);
        int wbase = 0;
        if (lane == 31 && incl) wbase = (int)atomicAdd(&a.bin.ctl[0], (unsigned)incl);
        wbase = __shfl_sync(0xffffffffu, wbase, 31);
        const int tw = tile | ((tile % ntx) << 16) | ((tile / ntx) << 24);
        for (int k = 0; k < n; ++k) {
            const int slot = wbase + incl - n + k;
            const int4 it = ovf ? make_int4(c, tw, 0, 0)
                                : make_int4(c, tw, first + k * kBinChunk,
                                            min(kBinChunk, count - k * kBinChunk) | (n << 11));
            if (slot < a.bin.max_items) a.bin.items[slot] = it;
            else if (a.err) atomicOr(a.err, TRK_DEVERR_WORKLIST);
        }
    }
    cluster.sync();  // no CTA reads another's counts any more (nor exits before they are read)

    // ---- phase 4: scatter this CTA's live triangles (their three snapped
    //      vertices) into the bins of the tiles their boxes touch ----
    if (!ovf) {
        int2 *pool = a.bin.pool + (size_t)c * a.bin.pool_cap * 3;
        const int nl = s_nlive;
        int i = tid;
        int2 e = i < nl ? live[i] : make_int2(0, 0);
        int4 tri = make_int4(0, 0, 0, 0);
        if (i < nl) tri = a.tris[e.x - (e.x >= a.T) * a.T];
        for (; i < nl; i += nthr) {
            int2 v0, v1, v2;
            tri_vertices(a, snapc, tri, e.x >= a.T, v0, v1, v2);
            orient(v0, v1, v2);
            const int pk = e.y;
            if (i + nthr < nl) {  // the next triangle's indices in flight
                e = live[i + nthr];
                tri = a.tris[e.x - (e.x >= a.T) * a.T];
            }
            const int tx0 = pk & 255, tx1 = (pk >> 8) & 255, ty0 = (pk >> 16) & 255, ty1 = (pk >> 24) & 255;
            for (int ty = ty0; ty <= ty1; ++ty)
                for (int tx = tx0; tx <= tx1; ++tx) {
                    int2 *r = pool + (size_t)atomicAdd(&cur[ty * ntx + tx], 1) * 3;
                    r[0] = v0;
                    r[1] = v1;
                    r[2] = v2;
                }
        }
    }
}

// ---------------------------------------------------------------------------
// The tile kernel.
// ---------------------------------------------------------------------------
// Triangle (v0, v1, v2) in the tile at (X0, Y0): set-up, box clipped to the
// tile, int32 raster into the tile bitmap `bm` (rows of two words).  Larger
// triangles are queued for a warp (big != NULL: their record `rec` within the
// work item) or drawn by this thread (big == NULL).
// The box and spans of an oriented live triangle (what tri_setup would give).
__device__ __forceinline__ void tri_box(int2 a, int2 b, int2 c, int W, int H, TriSetup &t)
{
    const int xmn = min(a.x, min(b.x, c.x)), xmx = max(a.x, max(b.x, c.x));
    const int ymn = min(a.y, min(b.y, c.y)), ymx = max(a.y, max(b.y, c.y));
    t.j0 = max(0, (xmn + 255) >> 8);
    t.j1 = min(W - 1, xmx >> 8);
    t.i0 = max(0, (ymn + 255) >> 8);
    t.i1 = min(H - 1, ymx >> 8);
    t.spanx = xmx - xmn;
    t.spany = ymx - ymn;
    t.x[0] = a.x; t.y[0] = a.y;
    t.x[1] = b.x; t.y[1] = b.y;
    t.x[2] = c.x; t.y[2] = c.y;
}

// oriented != 0: (v0, v1, v2) is a bin record (live, oriented); else raw
// snapped vertices that still need the full set-up.
__device__ __forceinline__ void tile_triangle(const EvalArgs &a, int2 v0, int2 v1, int2 v2, int X0, int Y0,
                                              uint32_t *bm, int rec, int *big, int *n_big, bool oriented = true)
{
    TriSetup ts;
    if (oriented)
        tri_box(v0, v1, v2, a.cam.W, a.cam.H, ts);
    else if (tri_setup(v0, v1, v2, a.cam.W, a.cam.H, a.cull, ts) != 1)
        return;
    const int j0 = max(ts.j0, X0), j1 = min(ts.j1, X0 + kTileW - 1);
    const int i0 = max(ts.i0, Y0), i1 = min(ts.i1, Y0 + kTileH - 1);
    if (j0 > j1 || i0 > i1) return;  // (from every triangle: not in this tile)
    ts.j0 = j0;
    ts.j1 = j1;
    ts.i0 = i0;
    ts.i1 = i1;
    if (ts.spanx < 32 * 256 && ts.spany < 64 * 256) {
        raster_small_at(ts, bm + (i0 - Y0) * 2 + (((j0 & ~31) - X0) >> 5), 2);
    } else if (big) {
        big[atomicAdd(n_big, 1)] = rec;
    } else {
        for (int i = i0; i <= i1; ++i)
            for (int j = j0; j <= j1; ++j) {
                const long long Px = 256LL * j, Py = 256LL * i;
                if ((edge64(ts, 0, Px, Py) | edge64(ts, 1, Px, Py) | edge64(ts, 2, Px, Py)) >= 0)
                    atomicOr(bm + (i - Y0) * 2 + ((j - X0) >> 5), 1u << (j & 31));
            }
    }
}

// A large triangle by one warp: lane l tests pixel 32 w + l of tile word w.
__device__ __forceinline__ void tile_triangle_warp(const EvalArgs &a, int2 v0, int2 v1, int2 v2, int X0, int Y0,
                                                   uint32_t *bm, int lane)
{
    TriSetup ts;
    tri_box(v0, v1, v2, a.cam.W, a.cam.H, ts);
    const int j0 = max(ts.j0, X0), j1 = min(ts.j1, X0 + kTileW - 1);
    const int i0 = max(ts.i0, Y0), i1 = min(ts.i1, Y0 + kTileH - 1);
    for (int i = i0; i <= i1; ++i) {
        const long long Py = 256LL * i;
        for (int w = (j0 - X0) >> 5; w <= ((j1 - X0) >> 5); ++w) {
            const int j = X0 + (w << 5) + lane;
            bool in = j >= j0 && j <= j1;
            if (in) {
                const long long Px = 256LL * j;
                in = (edge64(ts, 0, Px, Py) | edge64(ts, 1, Px, Py) | edge64(ts, 2, Px, Py)) >= 0;
            }
            const unsigned m = __ballot_sync(0xffffffffu, in);
            if (lane == 0 && m) atomicOr(bm + (i - Y0) * 2 + w, m);
        }
    }
}

static __device__ __noinline__ void tiles_epilogue(const EvalArgs &a, unsigned char *smem, int tid, int nthr);

// A tile whose candidate's bins overflowed: every triangle, filtered by the tile.
static __device__ __noinline__ void tile_from_every_triangle(const EvalArgs &a, int c, int X0, int Y0, uint32_t *bm,
                                                             int tid, int nthr)
{
    const int NT = a.ch.n_inst * a.T;
    const int2 *snapc = a.snap + (size_t)c * a.ch.n_inst * a.V;
    for (int t = tid; t < NT; t += nthr) {
        const int b = t >= a.T;
        int2 v0, v1, v2;
        tri_vertices(a, snapc, a.tris[t - b * a.T], b, v0, v1, v2);
        tile_triangle(a, v0, v1, v2, X0, Y0, bm, 0, nullptr, nullptr, false);
    }
}

constexpr int kTilesWarps = 8;  // k_tiles runs 256-thread CTAs

__global__ void __launch_bounds__(256, 4) k_tiles(EvalArgs a)
{
    griddep_launch_dependents();
    extern __shared__ __align__(16) unsigned char smem[];  // the CMA-ES update's shared memory (fused mode)
    __shared__ uint32_t tbm[kTilesWarps][kTileWords];     // one tile bitmap per warp
    __shared__ int s_big[kBinChunk];
    __shared__ int s_nbig, s_next, s_last, s_sub;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    const int H = a.cam.H, Wq = a.cam.Wq;
    const int nT = a.bin.n_tiles;
    uint32_t *bm = tbm[warp];
    griddep_wait();  // the front kernel is complete: bins, items and counters are final
    const int n_items = min((int)__ldcg(&a.bin.ctl[0]), a.bin.max_items);
    if (tid == 0) {
        s_next = (int)atomicAdd(&a.bin.ctl[1], 1u);
        s_nbig = 0;
        s_sub = 0;
    }
    for (;;) {
        __syncthreads();  // the ticket is visible; the last item's readers are done
        const int it = s_next;
        if (it >= n_items) break;
        const int4 item = a.bin.items[it];
        const int c = item.x, tile = item.y & 0xffff;
        const int X0 = ((item.y >> 16) & 255) * kTileW, Y0 = ((unsigned)item.y >> 24) * kTileH;
        const int n_ch = item.w >> 11;
        bm[lane] = 0u;
        bm[lane + 32] = 0u;
        __syncwarp();
        if (n_ch > 0) {
            // the item's records, 32 at a time: each warp takes the next group
            // when it is done with one, so a slow triangle holds up only its warp
            const int n = item.w & 2047;
            const int2 *pool = a.bin.pool + ((size_t)c * a.bin.pool_cap + item.z) * 3;
            for (;;) {
                int g = 0;
                if (lane == 0) g = atomicAdd(&s_sub, 32);
                g = __shfl_sync(0xffffffffu, g, 0);
                if (g >= n) break;
                const int e = g + lane;
                if (e < n)
                    tile_triangle(a, pool[3 * e], pool[3 * e + 1], pool[3 * e + 2], X0, Y0, bm, e, s_big, &s_nbig);
            }
        } else {
            tile_from_every_triangle(a, c, X0, Y0, bm, tid, nthr);
        }
        __syncthreads();
        if (tid == 0) s_next = (int)atomicAdd(&a.bin.ctl[1], 1u);  // the next item's ticket
        for (int k = warp; k < s_nbig; k += nwarp) {
            const int2 *r = a.bin.pool + ((size_t)c * a.bin.pool_cap + item.z + s_big[k]) * 3;
            tile_triangle_warp(a, r[0], r[1], r[2], X0, Y0, bm, lane);
        }
        __syncthreads();
        // count (one thread per tile word): at once for a tile drawn by one
        // item, else after OR-ing this item's words into the L2 copy, by the
        // item that finishes the tile last
        uint32_t S = 0u;
        if (tid < kTileWords)
            for (int w = 0; w < nwarp; ++w) S |= tbm[w][tid];
        if (tid == 0) {
            s_nbig = 0;
            s_sub = 0;
        }
        bool count = true;
        if (n_ch > 1) {
            uint32_t *mg = a.bin.merge + ((size_t)c * nT + tile) * kTileWords;
            if (tid < kTileWords && S) atomicOr(mg + tid, S);
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = atomicAdd(&a.bin.tile_done[(size_t)c * nT + tile], 1) == n_ch - 1;
            __syncthreads();
            count = s_last;
            if (count) {
                __threadfence();
                if (tid < kTileWords) S = atomicExch(mg + tid, 0u);  // read, and leave zero for the next launch
                if (tid == 0) a.bin.tile_done[(size_t)c * nT + tile] = 0;
            }
        }
        if (count && tid < kTileWords) {
            const int row = Y0 + (tid >> 1), col = (X0 >> 5) + (tid & 1);
            int s = 0, I = 0;
            if (row < H && col < Wq) {
                const uint32_t M = a.mask[(size_t)row * Wq + col];
                s = __popc(S);
                I = __popc(S & M);
                if (a.silhouette) a.silhouette[(size_t)row * Wq + col] = S;
            }
            s = warp_sum(s);
            I = warp_sum(I);
            if (lane == 0) {
                if (s) atomicAdd(&a.bin.acc[4 * c], s);
                if (I) atomicAdd(&a.bin.acc[4 * c + 1], I);
            }
        }
    }
    // the last CTA to leave writes every candidate's counts and loss, then (a
    // fused CMA-ES generation) runs the update
    if (tid == 0) {
        __threadfence();
        s_last = atomicAdd(&a.bin.ctl[2], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    tiles_epilogue(a, smem, tid, nthr);
}

// Counts and loss of every candidate, then (fused CMA-ES mode) the update; run
// by the last CTA of k_tiles.
static __device__ __noinline__ void tiles_epilogue(const EvalArgs &a, unsigned char *smem, int tid, int nthr)
{
    const int M_ = (int)__ldcg(&a.bin.ctl[3]);
    const int nF = a.ch.n_frames, nI = a.ch.n_inst;
    for (int c = tid; c < a.lam; c += nthr) {
        const int S_ = __ldcg(&a.bin.acc[4 * c]), I_ = __ldcg(&a.bin.acc[4 * c + 1]);
        const int C_ = __ldcg(&a.bin.acc[4 * c + 2]);
        if (a.counts) {
            a.counts[4 * c + 0] = S_;
            a.counts[4 * c + 1] = I_;
            a.counts[4 * c + 2] = M_;
            a.counts[4 * c + 3] = C_;
        }
        if (a.loss) {
            const int x = S_ + M_ - 2 * I_;
            float L;
            if (a.loss_kind == TRK_LOSS_ONE_MINUS_IOU) {
                const int U = S_ + M_ - I_;
                L = (U > 0) ? __fsub_rn(1.0f, __fdiv_rn((float)I_, (float)U)) : 0.0f;
            } else if (a.loss_kind == TRK_LOSS_MSE_APP) {
                L = __fadd_rn((float)x, __fmul_rn(a.lambda_app, (float)abs(S_ - M_)));
            } else {
                L = (float)x;
            }
            if (a.kp_obs && a.kp_lambda != 0.0f)
                L = __fadd_rn(L, keypoint_loss(a, a.bin.frames + (size_t)c * nI * nF * 24));
            a.loss[c] = L;
        }
    }
    __syncthreads();
    if (a.cma_st) {
        TellSmem &S = *reinterpret_cast<TellSmem *>(smem);
        cma_tell_block(*a.cma_k, a.cma_st, a.cma_y, a.params, a.loss, S, tid, nthr, !a.cma_finish);
        __syncthreads();
        if (a.cma_finish) cma_finish_frame(*a.cma_k, a.cma_st, a.cma_pose_out, tid, nthr);
    }
    if (tid < 4) a.bin.ctl[tid] = 0u;
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
size_t binned_front_smem_bytes(const EvalArgs &a, int threads)
{
    const size_t nT = (size_t)a.bin.n_tiles;
    return (size_t)a.ch.n_inst * kComposeScratch * sizeof(float2) + (size_t)a.ch.n_inst * a.ch.n_frames * 24 * 4 +
           (2 * nT + ((nT + 1) & ~(size_t)1)) * 4 + (size_t)a.bin.live_cap * sizeof(int2);
}

size_t binned_tiles_smem_bytes() { return sizeof(TellSmem); }

cudaError_t ensure_smem_attr(const void *func, size_t smem)
{
    // The limit is a property of the function on one device: remember the
    // largest value set per (function, device).
    struct Entry {
        const void *func;
        int device;
        size_t smem;
    };
    static std::mutex mu;
    static std::vector<Entry> done;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    for (Entry &x : done)
        if (x.func == func && x.device == dev) {
            if (smem <= x.smem) return cudaSuccess;
            e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e == cudaSuccess) x.smem = smem;
            return e;
        }
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) done.push_back(Entry{func, dev, smem});
    return e;
}

cudaError_t prepare_binned(size_t front_smem, int *tiles_per_sm)
{
    cudaError_t e = ensure_smem_attr((const void *)k_front, front_smem);
    if (e != cudaSuccess) return e;
    const size_t ts = binned_tiles_smem_bytes();
    if ((e = ensure_smem_attr((const void *)k_tiles, ts)) != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(tiles_per_sm, k_tiles, 256, ts);
}

cudaError_t launch_binned(const EvalArgs &a, const LaunchCfg &cfg, cudaStream_t s)
{
    if (a.lam == 0) return cudaSuccess;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    attr[1].id = cudaLaunchAttributeClusterDimension;
    attr[1].val.clusterDim.x = cfg.cluster;
    attr[1].val.clusterDim.y = 1;
    attr[1].val.clusterDim.z = 1;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.cluster, a.lam, 1);
    lc.blockDim = dim3(cfg.threads, 1, 1);
    lc.dynamicSmemBytes = cfg.smem;
    lc.stream = s;
    lc.attrs = attr;
    lc.numAttrs = 2;
    cudaError_t e = cudaLaunchKernelEx(&lc, k_front, a);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t lt = {};
    lt.gridDim = dim3(a.bin.tiles_grid, 1, 1);
    lt.blockDim = dim3(256, 1, 1);
    lt.dynamicSmemBytes = a.cma_st ? binned_tiles_smem_bytes() : 0;
    lt.stream = s;
    lt.attrs = attr;
    lt.numAttrs = 1;
    return cudaLaunchKernelEx(&lt, k_tiles, a);
}

}  // namespace trk
