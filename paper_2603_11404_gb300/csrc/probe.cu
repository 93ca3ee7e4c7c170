// Integer-issue probe: the denominator of the fitness kernel's roofline.
//
// The fitness path (edge functions, bounding boxes, bit operations) is bound by
// integer ALU issue, not by HBM or a tensor contraction, so its roofline peak is
// the rate at which the SMs retire plain 32-bit integer operations.  This kernel
// measures that rate on the device it runs on: every thread advances eight
// independent chains of LOP3 (three-input logic) operations, enough
// independent work per warp to cover the pipe latency, with every SM filled to
// its thread limit.  Hand-written PTX keeps the compiler from folding the
// chains away; the result is stored so that nothing is dead.
#include "internal.cuh"

namespace trk {

constexpr int kProbeChains = 8;
constexpr int kProbeUnroll = 16;

__global__ void __launch_bounds__(256) k_int_issue(uint32_t *out, int iters, uint32_t b, uint32_t c)
{
    uint32_t x[kProbeChains];
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) x[k] = (threadIdx.x + blockIdx.x * blockDim.x) * 0x9E3779B9u + k;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kProbeUnroll; ++u) {
#pragma unroll
            for (int k = 0; k < kProbeChains; ++k)
                asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(x[k]) : "r"(b), "r"(c));
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) r ^= x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace trk

using namespace trk;

static trk_status probe_fail(trk_status st, const char *why)
{
    set_last_error(why);
    return st;
}

extern "C" trk_status trk_probe_int_issue(int32_t iters, double *tops_out, double *ms_out, double *derived_tops_out)
{
    if (iters <= 0) return probe_fail(TRK_EINVAL, "iters must be > 0");
    if (!tops_out) return probe_fail(TRK_EINVAL, "tops_out is NULL");
    int dev = 0, sms = 0, max_threads = 0, khz = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&max_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev)) != cudaSuccess)
        return probe_fail(TRK_ECUDA, cudaGetErrorString(e));
    const int threads = 256;
    const int blocks = sms * (max_threads / threads);
    uint32_t *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.0f;
    if ((e = cudaMalloc(&out, (size_t)blocks * threads * sizeof(uint32_t))) != cudaSuccess)
        return probe_fail(e == cudaErrorMemoryAllocation ? TRK_ENOMEM : TRK_ECUDA, cudaGetErrorString(e));
    if ((e = cudaEventCreate(&e0)) == cudaSuccess && (e = cudaEventCreate(&e1)) == cudaSuccess) {
        k_int_issue<<<blocks, threads>>>(out, iters / 8 + 1, 0x5bd1e995u, 0x27d4eb2fu);  // warm-up
        cudaEventRecord(e0);
        k_int_issue<<<blocks, threads>>>(out, iters, 0x5bd1e995u, 0x27d4eb2fu);
        cudaEventRecord(e1);
        if ((e = cudaGetLastError()) == cudaSuccess && (e = cudaEventSynchronize(e1)) == cudaSuccess)
            e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess) return probe_fail(TRK_ECUDA, cudaGetErrorString(e));
    if (!(ms > 0.0f)) return probe_fail(TRK_ECUDA, "probe kernel reported no elapsed time");
    const double ops = (double)blocks * threads * iters * kProbeUnroll * kProbeChains;
    *tops_out = ops / ((double)ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
    // 64 INT32 lanes per SM per clock at the device's reported maximum SM clock
    if (derived_tops_out) *derived_tops_out = (double)sms * 64.0 * (double)khz * 1e3 / 1e12;
    return TRK_OK;
}
