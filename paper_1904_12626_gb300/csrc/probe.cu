// probe.cu -- a throughput probe of the FP64 pipe, the denominator the
// all-FP64 tile kernel's roofline is reported against (the FP32 kernels are
// reported against the FP32 issue rate, fixed by the SM count and clock).
//
// Each thread runs eight independent chains of fused multiply-adds in FP64,
// so the pipe, not the dependency latency, sets the rate; the grid holds 32
// warps per SM.  The result is FP64 lane-operations per second over three
// timed launches after a warm-up, at whatever clock the GPU runs.  Nothing is
// allocated: the chains' sum is written to a device variable only when it
// equals a value it never takes, which keeps the arithmetic live.
#include "internal.cuh"

namespace {

constexpr int kProbeIters = 2048;
constexpr int kProbeThreads = 256;
constexpr int kProbeBlocksPerSm = 4;

__device__ double g_probe_sink;

__global__ void __launch_bounds__(kProbeThreads) fp64_probe_kernel(double a, double b)
{
    double c[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) c[i] = threadIdx.x * 1e-3 + i;
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) c[i] = fma(c[i], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += c[i];
    if (s == -1.2345e300) g_probe_sink = s;
}

}  // namespace

extern "C" mp_status mp_probe_fp64_rate(double *lane_ops_per_s)
{
    if (!lane_ops_per_s) return MP_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return MP_ECUDA;
    const int blocks = sms * kProbeBlocksPerSm;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    mp_status st = MP_OK;
    float ms = 0.0f;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        st = MP_ECUDA;
    } else {
        fp64_probe_kernel<<<blocks, kProbeThreads>>>(1.0000001, 1e-9);
        cudaEventRecord(e0);
        for (int r = 0; r < 3; ++r) fp64_probe_kernel<<<blocks, kProbeThreads>>>(1.0000001, 1e-9);
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
            cudaGetLastError() != cudaSuccess || ms <= 0.0f)
            st = MP_ECUDA;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != MP_OK) return st;
    *lane_ops_per_s = 3.0 * blocks * kProbeThreads * (double)kProbeIters * 8.0 / (ms * 1e-3);
    return MP_OK;
}
