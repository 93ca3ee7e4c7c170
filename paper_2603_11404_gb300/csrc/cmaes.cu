// Stand-alone device-resident CMA-ES kernels (arXiv 2603.11404, Sec. III-A.1,
// Eq. cmaes_update; block-diagonal covariance of Sec. III-B): reset, sample
// (ask), update (tell) and the frame epilogue.  The arithmetic lives in
// cma_device.cuh and is shared with the fused per-generation fitness kernel.
#include "cma_device.cuh"

namespace trk {

__device__ void cma_reset_body(const CmaConst &k, CmaState *st, const double *mean_dev, int from_est,
                               const float *joint_reading, int n_inst, int tid, int nt)
{
    const int d = k.d;
    // a new frame: the Kalman prediction, whose position seeds the mean if asked to
    const bool predict = from_est && k.kf.enabled && st->kf.initialized;
    for (int i = tid; i < d; i += nt) {
        double mi = from_est ? st->est[i] : mean_dev[i];
        if (predict) {
            kf_predict(k.kf, st->kf, i);
            if (k.kf.seed_mean) mi = kf_to_state(k, st->kf, i);
        }
        int b = i / 9, r = i - 9 * b;
        if (joint_reading && r >= 6 && b < n_inst)
            mi = qhat_from_q((double)joint_reading[3 * b + (r - 6)], k.q_lb[r - 6], k.q_ub[r - 6]);
        st->est[i] = mi;
        st->m[i] = mi / k.scales[i];
        st->m_df[i] = split_df(st->m[i]);
        st->p_sigma[i] = 0.0;
        st->p_c[i] = 0.0;
        st->ev[i] = 1.0;
        st->best_x[i] = 0.0f;
    }
    for (int e = tid; e < d * d; e += nt) {
        double v = (e / d == e % d) ? 1.0 : 0.0;
        st->C[e] = v;
        st->B[e] = v;
        st->C_half[e] = v;
        st->C_half_df[e] = make_float2((float)v, 0.0f);
        st->C_inv_half[e] = v;
    }
    if (tid == 0) {
        st->sigma = k.sigma0;
        st->sigma_df = split_df(k.sigma0);
        st->cs_pow = 1.0;
        st->gen = 0;
        st->best_loss = INFINITY;
        st->jacobi_sweeps = 0;
        st->warn = 0;
    }
}

__global__ void k_cma_reset(const CmaConst *__restrict__ kp, CmaState *st, const double *mean_dev, int from_est,
                            const float *joint_reading, int n_inst)
{
    cma_reset_body(*kp, st, mean_dev, from_est, joint_reading, n_inst, threadIdx.x, blockDim.x);
}

__global__ void k_cma_ask(const CmaConst *__restrict__ kp, CmaState *st, double *y, double *z_keep,
                          float *params, const double *z_in)
{
    __shared__ float2 zs[kMaxD];
    cma_sample_warp(*kp, st, blockIdx.x, z_in, y, z_keep, params, nullptr, zs, threadIdx.x);
}

constexpr int kTellThreads = 128;  // 4 warps: one per SM sub-partition's FP64 pipe

__global__ void __launch_bounds__(kTellThreads) k_cma_tell(const CmaConst *__restrict__ kp, CmaState *st,
                                                           const double *y, const float *params, const float *loss)
{
    __shared__ TellSmem S;
    cma_tell_block(*kp, st, y, params, loss, S, threadIdx.x, blockDim.x);
}

// The square roots and eigenbasis of the stored covariance (after an update
// that left them out).
__global__ void __launch_bounds__(kTellThreads) k_cma_sqrt(const CmaConst *__restrict__ kp, CmaState *st)
{
    __shared__ TellSmem S;
    cma_sqrt_block(*kp, st, S, threadIdx.x, blockDim.x);
}

__global__ void k_cma_finish(const CmaConst *__restrict__ kp, CmaState *st, float *pose_out)
{
    cma_finish_frame(*kp, st, pose_out, threadIdx.x, blockDim.x);
}

// Batched forms: block b serves instance sel[b] (or b when sel is NULL) of
// tables of device pointers indexed by instance.
// Selected entries may carry kSelNoSqrt (op 4: that instance's update leaves
// out the square roots).
__device__ __forceinline__ int batch_instance(const int *sel)
{
    return sel ? (sel[blockIdx.x] & ~kSelNoSqrt) : (int)blockIdx.x;
}

__global__ void k_cma_reset_batch(const int *sel, const CmaConst *const *kp, CmaState *const *st, const int *n_inst,
                                  const float *const *joint)
{
    const int i = batch_instance(sel);
    cma_reset_body(*kp[i], st[i], nullptr, 1, joint ? joint[i] : nullptr, n_inst[i], threadIdx.x, blockDim.x);
}

__global__ void __launch_bounds__(kTellThreads) k_cma_tell_batch(const int *sel, const CmaConst *const *kp,
                                                                 CmaState *const *st, const double *const *y,
                                                                 const float *const *params,
                                                                 const float *const *loss, int do_sqrt)
{
    __shared__ TellSmem S;
    const int i = batch_instance(sel);
    const bool sq = do_sqrt == 2 ? !(sel[blockIdx.x] & kSelNoSqrt) : do_sqrt != 0;
    cma_tell_block(*kp[i], st[i], y[i], params[i], loss[i], S, threadIdx.x, blockDim.x, sq);
}

__global__ void k_cma_finish_batch(const int *sel, const CmaConst *const *kp, CmaState *const *st,
                                   float *const *pose_out)
{
    const int i = batch_instance(sel);
    cma_finish_frame(*kp[i], st[i], pose_out[i], threadIdx.x, blockDim.x);
}

cudaError_t launch_cma_batch(int op, int n, const int *sel, const BatchTables &t, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    if (op == 0) k_cma_reset_batch<<<n, 128, 0, s>>>(sel, t.k, t.st, t.ninst, t.joint);
    if (op == 1 || op == 3 || op == 4)
        k_cma_tell_batch<<<n, kTellThreads, 0, s>>>(sel, t.k, t.st, t.y, t.params, t.loss, op == 4 ? 2 : op == 1);
    if (op == 2) k_cma_finish_batch<<<n, 32, 0, s>>>(sel, t.k, t.st, t.pose);
    return cudaGetLastError();
}

cudaError_t launch_cma_reset(const CmaConst *k, CmaState *st, const double *mean_dev, bool from_est,
                             const float *joint_reading_dev, int n_inst, cudaStream_t s)
{
    k_cma_reset<<<1, 128, 0, s>>>(k, st, mean_dev, from_est ? 1 : 0, joint_reading_dev, n_inst);
    return cudaGetLastError();
}

cudaError_t launch_cma_ask(const CmaConst *k, int lam, CmaState *st, double *y, double *z_keep, float *params,
                           const double *z_in, cudaStream_t s)
{
    k_cma_ask<<<lam, 32, 0, s>>>(k, st, y, z_keep, params, z_in);
    return cudaGetLastError();
}

cudaError_t launch_cma_tell(const CmaConst *k, CmaState *st, const double *y, const float *params,
                            const float *loss, cudaStream_t s)
{
    k_cma_tell<<<1, kTellThreads, 0, s>>>(k, st, y, params, loss);
    return cudaGetLastError();
}

cudaError_t launch_cma_sqrt(const CmaConst *k, CmaState *st, cudaStream_t s)
{
    k_cma_sqrt<<<1, kTellThreads, 0, s>>>(k, st);
    return cudaGetLastError();
}

cudaError_t launch_cma_finish_frame(const CmaConst *k, CmaState *st, float *pose_out, cudaStream_t s)
{
    k_cma_finish<<<1, 32, 0, s>>>(k, st, pose_out);
    return cudaGetLastError();
}

}  // namespace trk
