// probe.cu -- measured peak rate of single-precision fused multiply-adds on
// the current device (libenuf_probe.so, a helper of the benchmark; not part
// of the ENUF library).  It is the denominator of the FMA roofline that is
// reported beside the HBM roofline for the spreading and interpolation
// kernels, whose algorithmic work is p^3 and f p^3 multiply-adds per
// particle (plus the window evaluations).
#include <cuda_runtime.h>

#include <string>

#include "../../include/enuf_probe.h"

namespace {

thread_local std::string g_probe_err;

__device__ float fma_sink;  // written only if the chains hit an impossible value

constexpr int kChains = 8, kUnroll = 16;

// kChains independent chains a <- a m + c per thread (m < 1: the chains
// settle near c / (1 - m) and never overflow or go subnormal).
__global__ void __launch_bounds__(256) k_fma_peak(int iters, float seed)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = seed + 1e-6f * (float)(threadIdx.x + k);
    const float m = 0.99999994f, c = 5.9604645e-08f;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], m, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == -1.0f) fma_sink = s;
}

int pfail(int code, const std::string& msg)
{
    g_probe_err = msg;
    return code;
}

}  // namespace

extern "C" const char* enuf_probe_last_error(void) { return g_probe_err.c_str(); }

extern "C" int enuf_fma_peak_tflops(double* tflops, void* cuda_stream)
{
    g_probe_err.clear();
    if (!tflops) return pfail(-1, "tflops is NULL");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return pfail(-4, std::string("device query: ") + cudaGetErrorString(e));
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    const int blocks = sms * 8, threads = 256, iters = 2048, reps = 3;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fma_peak<<<blocks, threads, 0, st>>>(iters, 1.0f);  // warm-up
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps; r++) k_fma_peak<<<blocks, threads, 0, st>>>(iters, 1.0f);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return pfail(-4, std::string("FMA probe: ") + cudaGetErrorString(e));
    }
    const double fmas = (double)blocks * threads * iters * kUnroll * kChains * reps;
    *tflops = 2.0 * fmas / ((double)ms * 1e-3) / 1e12;
    return 0;
}
