/*
 * CPU oracle for the silhouette fitness of arXiv 2603.11404 (test infrastructure).
 *
 * This file is the plain, slow, obviously-correct reference that the CUDA path
 * is checked against.  Only tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load it; the product library never does.  It shares no
 * code with the CUDA sources.
 *
 * What it computes, in the paper's order (Sec. III-A):
 *   state Theta = (T_r^c, q)                                  Eq. (1), Sec. III-A
 *   q_i from the unconstrained q-hat_i (inverse cosine map)   Sec. III-A.3
 *   R: axis-angle (Rodrigues) or look-at Ry(gamma)Rx(alpha)Rz(beta)  Sec. III-A.3
 *   T_r^c T_m^r(q) v_m, pinhole K, canonical projection       Sec. III-A.2 (renderer)
 *   S = R(...): binary silhouette, union over all triangles    Sec. III-A.2
 *   counts s = sum S, m = sum M, I = sum S&M -> losses         Eq. render_loss, Sec. IV (1 - IoU)
 *
 * Readings where the paper is silent (all arithmetic in FP64 / exact int64):
 *   - pixel (i, j) samples the image point (u, v) = (j, i);
 *   - projected coordinates are snapped to 1/256 px with round-half-even:
 *       U = nearbyint(256 (u - cx)) + 256 cx,  u - cx = fx X / Z  (256 cx integer);
 *   - a vertex with Z < z_near or |u - cx| or |v - cy| > guard px is flagged; a
 *     triangle touching a flagged vertex is not drawn and is counted as culled;
 *   - coverage: normalise the triangle to positive doubled area
 *       A = (b - a) x (c - a) > 0 (swap b, c when A < 0, skip when A == 0);
 *     edge p0->p1 has E(P) = dx (Py - y0) - dy (Px - x0); P is covered iff every
 *     edge has E > 0, or E == 0 and the edge is top-left (dy < 0, or dy == 0 and
 *     dx > 0);
 *   - optional back-face culling skips triangles whose unnormalised A > 0 (the
 *     meshes are wound counter-clockwise seen from outside; with y pointing down
 *     a front face has A < 0).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_FRAMES 16

/* ------------------------------------------------------------------------- */
/* Kinematic chain description (one instrument).                             */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n_frames;
    const int *parent;      /* [nf], -1 = end-effector frame E               */
    const double *offset;   /* [nf*3] translation in the parent frame (mm)    */
    const int *axis;        /* [nf] 0 none, 1 x, 2 y, 3 z                    */
    const int *joint;       /* [nf] joint index 0..2                          */
    const double *coef;     /* [nf] angle = coef * q[joint]                   */
    const double *q_lb;     /* [3]                                            */
    const double *q_ub;     /* [3]                                            */
    int rot_param;          /* 0 axis-angle, 1 look-at                        */
} orc_chain;

/* Sec. III-A.3, inverse map: q = lb + (ub-lb)/2 (1 - cos(pi (qh - lb)/(ub - lb))). */
double orc_q_from_qhat(double qh, double lb, double ub)
{
    if (ub == lb) return lb;
    return lb + 0.5 * (ub - lb) * (1.0 - cos(M_PI * (qh - lb) / (ub - lb)));
}

/* Sec. III-A.3, forward map: qh = lb + (ub-lb)/pi arccos(1 - 2 (q - lb)/(ub - lb)). */
double orc_qhat_from_q(double q, double lb, double ub)
{
    if (ub == lb) return lb;
    double a = 1.0 - 2.0 * (q - lb) / (ub - lb);
    if (a > 1.0) a = 1.0;
    if (a < -1.0) a = -1.0;
    return lb + (ub - lb) / M_PI * acos(a);
}

static void mat_rx(double a, double R[9])
{
    double c = cos(a), s = sin(a);
    double M[9] = {1, 0, 0, 0, c, -s, 0, s, c};
    memcpy(R, M, sizeof M);
}
static void mat_ry(double a, double R[9])
{
    double c = cos(a), s = sin(a);
    double M[9] = {c, 0, s, 0, 1, 0, -s, 0, c};
    memcpy(R, M, sizeof M);
}
static void mat_rz(double a, double R[9])
{
    double c = cos(a), s = sin(a);
    double M[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
    memcpy(R, M, sizeof M);
}
static void mat_mul3(const double A[9], const double B[9], double C[9])
{
    double T[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * B[3 * k + j];
            T[3 * i + j] = acc;
        }
    memcpy(C, T, sizeof T);
}

/* Rotation of T_r^c.  rot_param 0: axis-angle vector r, Rodrigues' formula
 * R = I + sin(t) [k]x + (1 - cos(t)) [k]x^2 with t = |r|, k = r / t (first order
 * I + [r]x when t < 1e-8).  rot_param 1: look-at R = Ry(gamma) Rx(alpha) Rz(beta)
 * with r = (alpha, beta, gamma), Sec. III-A.3. */
void orc_rotation(int rot_param, const double r[3], double R[9])
{
    if (rot_param == 1) {
        double Ry[9], Rx[9], Rz[9], T[9];
        mat_ry(r[2], Ry);
        mat_rx(r[0], Rx);
        mat_rz(r[1], Rz);
        mat_mul3(Ry, Rx, T);
        mat_mul3(T, Rz, R);
        return;
    }
    double t = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    if (t < 1e-8) {
        double M[9] = {1, -r[2], r[1], r[2], 1, -r[0], -r[1], r[0], 1};
        memcpy(R, M, sizeof M);
        return;
    }
    double k[3] = {r[0] / t, r[1] / t, r[2] / t};
    double K[9] = {0, -k[2], k[1], k[2], 0, -k[0], -k[1], k[0], 0};
    double K2[9];
    mat_mul3(K, K, K2);
    double s = sin(t), c1 = 1.0 - cos(t);
    for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? 1.0 : 0.0) + s * K[i] + c1 * K2[i];
}

/* 3x4 rigid transforms, row-major [R | t]. */
static void tf_mul(const double A[12], const double B[12], double C[12])
{
    double T[12];
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 4; ++j) {
            double acc = (j == 3) ? A[4 * i + 3] : 0.0;
            for (int k = 0; k < 3; ++k) acc += A[4 * i + k] * B[4 * k + j];
            T[4 * i + j] = acc;
        }
    }
    memcpy(C, T, sizeof T);
}

/* Camera-from-frame transforms T_cam_f = T_r^c * T_f(q) for every frame of the
 * chain, given one 9-vector state [r(3), t(3), qhat(3)].  T_f = T_parent *
 * Trans(offset_f) * Rot(axis_f, coef_f * q[joint_f]) (forward kinematics of the
 * wrist, Sec. III-A.2 "T_m^r(q)"). */
void orc_frame_transforms(const orc_chain *ch, const double *state, double *T_out)
{
    double q[3];
    for (int i = 0; i < 3; ++i) q[i] = orc_q_from_qhat(state[6 + i], ch->q_lb[i], ch->q_ub[i]);
    double R[9];
    orc_rotation(ch->rot_param, state, R);
    double Tc[12] = {R[0], R[1], R[2], state[3], R[3], R[4], R[5], state[4], R[6], R[7], R[8], state[5]};
    double Tf[ORC_MAX_FRAMES][12];
    for (int f = 0; f < ch->n_frames; ++f) {
        double J[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        double ang = ch->coef[f] * q[ch->joint[f]];
        if (ch->axis[f] == 1) mat_rx(ang, J);
        if (ch->axis[f] == 2) mat_ry(ang, J);
        if (ch->axis[f] == 3) mat_rz(ang, J);
        double L[12] = {J[0], J[1], J[2], ch->offset[3 * f + 0],
                        J[3], J[4], J[5], ch->offset[3 * f + 1],
                        J[6], J[7], J[8], ch->offset[3 * f + 2]};
        if (ch->parent[f] < 0) memcpy(Tf[f], L, sizeof L);
        else tf_mul(Tf[ch->parent[f]], L, Tf[f]);
    }
    for (int f = 0; f < ch->n_frames; ++f) tf_mul(Tc, Tf[f], T_out + 12 * f);
}

/* Project and snap the vertices of one instrument (Sec. III-A.2:
 * K(Pi(T_r^c T_m^r(q) v_m))).  Writes the unsnapped offsets from the principal
 * point (u - cx, v - cy) in px, the snapped 1/256 px coordinates and a flag byte
 * (1 = behind z_near or outside the guard band).  Returns the number flagged. */
int orc_project(const orc_chain *ch, const double *state, int n_verts, const float *verts,
                const int *vframe, double fx, double fy, double cx, double cy, double z_near,
                double guard, double *uv, int64_t *snap, uint8_t *flag)
{
    double T[ORC_MAX_FRAMES * 12];
    orc_frame_transforms(ch, state, T);
    int64_t cx256 = (int64_t)llround(256.0 * cx), cy256 = (int64_t)llround(256.0 * cy);
    int n_flag = 0;
    for (int v = 0; v < n_verts; ++v) {
        const double *M = T + 12 * vframe[v];
        double p[3] = {verts[3 * v], verts[3 * v + 1], verts[3 * v + 2]};
        double X = M[0] * p[0] + M[1] * p[1] + M[2] * p[2] + M[3];
        double Y = M[4] * p[0] + M[5] * p[1] + M[6] * p[2] + M[7];
        double Z = M[8] * p[0] + M[9] * p[1] + M[10] * p[2] + M[11];
        double du = 0.0, dv = 0.0;
        int bad = !(Z >= z_near);
        if (!bad) {
            du = fx * X / Z;
            dv = fy * Y / Z;
            bad = !(fabs(du) <= guard && fabs(dv) <= guard);
        }
        uv[2 * v] = du;
        uv[2 * v + 1] = dv;
        flag[v] = (uint8_t)bad;
        if (bad) {
            snap[2 * v] = 0;
            snap[2 * v + 1] = 0;
            ++n_flag;
        } else {
            snap[2 * v] = (int64_t)nearbyint(256.0 * du) + cx256;
            snap[2 * v + 1] = (int64_t)nearbyint(256.0 * dv) + cy256;
        }
    }
    return n_flag;
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}
static int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }

/* Rasterise triangles over snapped vertices into the byte image S (OR union) by
 * brute force over each triangle's bounding box.  frag_out receives the number
 * of (triangle, pixel) coverages, so a watertight tessellation has frags equal
 * to the covered area.  Returns the number of triangles culled for flags. */
int64_t orc_raster(int n_tris, const int32_t *tris, int vert_base, const int64_t *snap,
                   const uint8_t *flag, int W, int H, int cull_back, uint8_t *S,
                   int64_t *frag_out, int64_t *bbox_px_out)
{
    int64_t culled = 0, frags = 0, bbox_px = 0;
    for (int t = 0; t < n_tris; ++t) {
        int id[3] = {tris[3 * t] + vert_base, tris[3 * t + 1] + vert_base, tris[3 * t + 2] + vert_base};
        if (flag[id[0]] || flag[id[1]] || flag[id[2]]) { ++culled; continue; }
        int64_t x[3], y[3];
        for (int k = 0; k < 3; ++k) { x[k] = snap[2 * id[k]]; y[k] = snap[2 * id[k] + 1]; }
        int64_t A = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
        if (A == 0) continue;
        if (cull_back && A > 0) continue;
        if (A < 0) {
            int64_t tx = x[1], ty = y[1];
            x[1] = x[2]; y[1] = y[2];
            x[2] = tx; y[2] = ty;
        }
        int64_t dx[3], dy[3], x0[3], y0[3];
        int tl[3];
        for (int k = 0; k < 3; ++k) {
            int k1 = (k + 1) % 3;
            x0[k] = x[k]; y0[k] = y[k];
            dx[k] = x[k1] - x[k];
            dy[k] = y[k1] - y[k];
            tl[k] = (dy[k] < 0) || (dy[k] == 0 && dx[k] > 0);
        }
        int64_t xmn = x[0], xmx = x[0], ymn = y[0], ymx = y[0];
        for (int k = 1; k < 3; ++k) {
            if (x[k] < xmn) xmn = x[k];
            if (x[k] > xmx) xmx = x[k];
            if (y[k] < ymn) ymn = y[k];
            if (y[k] > ymx) ymx = y[k];
        }
        int64_t j0 = ceil_div(xmn, 256), j1 = floor_div(xmx, 256);
        int64_t i0 = ceil_div(ymn, 256), i1 = floor_div(ymx, 256);
        if (j0 < 0) j0 = 0;
        if (i0 < 0) i0 = 0;
        if (j1 > W - 1) j1 = W - 1;
        if (i1 > H - 1) i1 = H - 1;
        if (j0 > j1 || i0 > i1) continue;
        bbox_px += (j1 - j0 + 1) * (i1 - i0 + 1);
        for (int64_t i = i0; i <= i1; ++i) {
            for (int64_t j = j0; j <= j1; ++j) {
                int64_t Px = 256 * j, Py = 256 * i;
                int in = 1;
                for (int k = 0; k < 3 && in; ++k) {
                    int64_t E = dx[k] * (Py - y0[k]) - dy[k] * (Px - x0[k]);
                    in = (E > 0) || (E == 0 && tl[k]);
                }
                if (in) {
                    S[i * W + j] = 1;
                    ++frags;
                }
            }
        }
    }
    if (frag_out) *frag_out += frags;
    if (bbox_px_out) *bbox_px_out += bbox_px;
    return culled;
}

/* Counts of Eq. render_loss / the IoU metric: s = sum S, m = sum M, I = sum S&M,
 * plus the XOR count taken by a direct per-pixel loop as a self-check. */
void orc_counts(int W, int H, const uint8_t *S, const uint8_t *M, int64_t out[4])
{
    int64_t s = 0, m = 0, I = 0, x = 0;
    for (int64_t p = 0; p < (int64_t)W * H; ++p) {
        int a = S[p] != 0, b = M[p] != 0;
        s += a;
        m += b;
        I += a & b;
        x += (a - b) * (a - b);
    }
    out[0] = s; out[1] = m; out[2] = I; out[3] = x;
}

/* ------------------------------------------------------------------------- */
/* Whole-population evaluation (the fitness of every CMA-ES sample).          */
/* ------------------------------------------------------------------------- */
typedef struct {
    const orc_chain *ch;
    int n_inst, d, lam;
    const double *params;           /* [lam*d] */
    int n_verts, n_tris;
    const float *verts;
    const int *vframe;
    const int32_t *tris;
    double fx, fy, cx, cy, z_near, guard;
    int W, H, cull_back;
    const uint8_t *mask;
    int64_t *out;                   /* [lam*8]: s, m, I, xor, frags, culled, flagged, bbox_px */
    int next;
    pthread_mutex_t lock;
} orc_job;

static void eval_one(orc_job *J, int c, uint8_t *S, double *uv, int64_t *snap, uint8_t *flag)
{
    int nv = J->n_verts;
    int64_t flagged = 0, culled = 0, frags = 0, bbox_px = 0;
    for (int b = 0; b < J->n_inst; ++b)
        flagged += orc_project(J->ch, J->params + (size_t)c * J->d + 9 * b, nv, J->verts, J->vframe,
                               J->fx, J->fy, J->cx, J->cy, J->z_near, J->guard,
                               uv + 2 * (size_t)nv * b, snap + 2 * (size_t)nv * b, flag + (size_t)nv * b);
    memset(S, 0, (size_t)J->W * J->H);
    for (int b = 0; b < J->n_inst; ++b)
        culled += orc_raster(J->n_tris, J->tris, nv * b, snap, flag, J->W, J->H, J->cull_back, S,
                             &frags, &bbox_px);
    int64_t cnt[4];
    orc_counts(J->W, J->H, S, J->mask, cnt);
    int64_t *o = J->out + 8 * (size_t)c;
    o[0] = cnt[0]; o[1] = cnt[1]; o[2] = cnt[2]; o[3] = cnt[3];
    o[4] = frags; o[5] = culled; o[6] = flagged; o[7] = bbox_px;
}

static void *worker(void *arg)
{
    orc_job *J = (orc_job *)arg;
    size_t nv = (size_t)J->n_verts * J->n_inst;
    uint8_t *S = malloc((size_t)J->W * J->H);
    double *uv = malloc(nv * 2 * sizeof(double));
    int64_t *snap = malloc(nv * 2 * sizeof(int64_t));
    uint8_t *flag = malloc(nv);
    for (;;) {
        pthread_mutex_lock(&J->lock);
        int c = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (c >= J->lam) break;
        eval_one(J, c, S, uv, snap, flag);
    }
    free(S); free(uv); free(snap); free(flag);
    return NULL;
}

/* Evaluate lam candidate states (each n_inst*9 doubles) against the byte mask
 * M [H*W]; out [lam*8] = s, m, I, xor, frags, culled, flagged, bbox_px.  The
 * union over instruments implements the bi-manual joint render (Sec. III-B).
 * n_threads > 1 splits candidates over POSIX threads. */
int orc_eval_population(int n_frames, const int *parent, const double *offset, const int *axis,
                        const int *joint, const double *coef, const double *q_lb, const double *q_ub,
                        int rot_param, int n_inst, int lam, const double *params, int n_verts,
                        const float *verts, const int *vframe, int n_tris, const int32_t *tris,
                        double fx, double fy, double cx, double cy, double z_near, double guard,
                        int W, int H, int cull_back, const uint8_t *mask, int64_t *out, int n_threads)
{
    if (n_frames > ORC_MAX_FRAMES) return -1;
    orc_chain ch = {n_frames, parent, offset, axis, joint, coef, q_lb, q_ub, rot_param};
    orc_job J;
    memset(&J, 0, sizeof J);
    J.ch = &ch; J.n_inst = n_inst; J.d = 9 * n_inst; J.lam = lam; J.params = params;
    J.n_verts = n_verts; J.n_tris = n_tris; J.verts = verts; J.vframe = vframe; J.tris = tris;
    J.fx = fx; J.fy = fy; J.cx = cx; J.cy = cy; J.z_near = z_near; J.guard = guard;
    J.W = W; J.H = H; J.cull_back = cull_back; J.mask = mask; J.out = out; J.next = 0;
    pthread_mutex_init(&J.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    pthread_t th[256];
    for (int i = 1; i < n_threads; ++i) pthread_create(&th[i], NULL, worker, &J);
    worker(&J);
    for (int i = 1; i < n_threads; ++i) pthread_join(th[i], NULL);
    pthread_mutex_destroy(&J.lock);
    return 0;
}

/* Single-candidate helpers for tests: project one instrument, render the union
 * silhouette of one candidate into S. */
int orc_project_state(int n_frames, const int *parent, const double *offset, const int *axis,
                      const int *joint, const double *coef, const double *q_lb, const double *q_ub,
                      int rot_param, const double *state, int n_verts, const float *verts,
                      const int *vframe, double fx, double fy, double cx, double cy, double z_near,
                      double guard, double *uv, int64_t *snap, uint8_t *flag, double *T_out)
{
    if (n_frames > ORC_MAX_FRAMES) return -1;
    orc_chain ch = {n_frames, parent, offset, axis, joint, coef, q_lb, q_ub, rot_param};
    if (T_out) orc_frame_transforms(&ch, state, T_out);
    return orc_project(&ch, state, n_verts, verts, vframe, fx, fy, cx, cy, z_near, guard, uv, snap, flag);
}
