// Throughput probes for the roofline of the FP32 pair passes: the FP32 (FMA)
// pipe through packed f32x2 FMAs, and the MUFU pipe through rsqrt.approx.
// Each thread runs independent chains so that issue, not latency, limits the
// loop; results go to a file-scope sink that is written only for an
// impossible value, so nothing is allocated and nothing is optimised away.
#include <cuda_runtime.h>

#include <string>

#include "../../include/cphremd.h"
#include "cph_device.cuh"

void cph_internal_set_error(const std::string& m);

namespace {

constexpr int kProbeIters = 2048;
constexpr int kProbeThreads = 256;

__device__ float g_probe_sink;

__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(float s) {
    float2 a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = make_float2(threadIdx.x * 1e-3f + k, threadIdx.x * 1e-3f - k);
    const float2 m = make_float2(s, s), c = make_float2(0.5f, 0.25f);
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = __ffma2_rn(a[k], m, c);
    }
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) r += a[k].x + a[k].y;
    if (r == -1.2345f) g_probe_sink = r;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_mufu(float s) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = s + threadIdx.x * 1e-3f + k;
    for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = cph::rsqrt_ftz(a[k]);
    }
    float r = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) r += a[k];
    if (r == -1.2345f) g_probe_sink = r;
}

int pfail(const char* m) {
    cph_internal_set_error(m);
    return CPH_E_CUDA;
}

} // namespace

extern "C" int cph_probe_pipe_rates(double* fp32_ops_per_s, double* mufu_ops_per_s, void* stream) {
    if (!fp32_ops_per_s || !mufu_ops_per_s) {
        cph_internal_set_error("cph_probe_pipe_rates: NULL argument");
        return CPH_E_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return pfail("cph_probe_pipe_rates: no device");
    const int blocks = sms * 8;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return pfail("cph_probe_pipe_rates: cudaEventCreate failed");
    const double threads = (double)blocks * kProbeThreads;
    double rate[2] = {0.0, 0.0};
    for (int which = 0; which < 2; ++which) {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) { // the first run warms up
            cudaEventRecord(e0, st);
            if (which == 0) k_probe_fma<<<blocks, kProbeThreads, 0, st>>>(0.999f);
            else k_probe_mufu<<<blocks, kProbeThreads, 0, st>>>(1.5f);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                return pfail("cph_probe_pipe_rates: probe kernel failed");
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        // FP32 lane operations (one FMA counts once) or MUFU operations
        const double ops = threads * kProbeIters * (which == 0 ? 16.0 : 8.0);
        rate[which] = ops / (best * 1e-3);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) return pfail("cph_probe_pipe_rates: launch failed");
    *fp32_ops_per_s = rate[0];
    *mufu_ops_per_s = rate[1];
    return CPH_OK;
}
