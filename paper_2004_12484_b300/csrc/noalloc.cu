// noalloc.cu -- real-space pair sum for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// electrostatics: code running inside a host framework whose device memory is
// fully reserved by its own pool allocator, plugins that are handed only
// input and output buffers, and code paths that must not allocate after an
// initial set-up phase (allocation can synchronise the device and can fail
// under memory pressure).  For them this file provides one entry point,
// enuf_real_space_noalloc, that allocates nothing: it is a variant of the
// library's all-pairs real-space kernel that reads raw positions (it does no
// sorting, which would need scratch buffers) and keeps its only scratch --
// the per-block partial sums of the energy and virial and a completion
// counter -- in a fixed array in device global memory declared below.
//
// The array exists once per GPU that loads the library and lives until the
// process exits.  Its size bounds the problem: at most kMaxBlocks blocks of
// 256 particles, i.e. N <= 262,144 particles.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so on the first call on each device this file
// looks up the device address with cudaGetSymbolAddress while that device is
// current, and passes the pointer to the kernel.  That first call performs
// the look-up and therefore should happen before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/enuf.h"
#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;
constexpr int kMaxDevices = 64;

// Scratch: kMaxBlocks x 8 partial sums (energy, six virial components, pad)
// followed by one completion counter.  Shared by every call on the device.
struct NoAllocScratch {
    double partial[kMaxBlocks * 8];
    unsigned int counter;
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

NoAllocScratch* g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mu;

}  // namespace

namespace enuf {
void set_last_error(const std::string& msg);  // enuf.cu: backs enuf_last_error()
}

namespace {

int nfail(int code, const std::string& msg)
{
    enuf::set_last_error(msg);
    return code;
}

// x wrapped into [0, L) (iL = 1/L, passed in so that no division runs per
// particle or pair)
template <typename R> __device__ __forceinline__ R wrap_to_box(R x, R L, R iL) { return x - L * floor(x * iL); }

template <typename R>
__device__ __forceinline__ void pair_sum(R dx, R dy, R dz, R qi, R qj, R rc2, R alpha, R two_a_sqpi, R (&f)[3], R& ph,
                                         R (&acc)[7])
{
    const R r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= rc2 || r2 <= R(0)) return;
    const R r = enuf::dsqrt(r2);
    const R ar = alpha * r;
    const R ec = enuf::derfc(ar) / r;
    const R fs = qi * qj * (ec + two_a_sqpi * enuf::dexp(-ar * ar)) / r2;
    f[0] += fs * dx;
    f[1] += fs * dy;
    f[2] += fs * dz;
    ph += qj * ec;
    acc[0] += R(0.5) * qi * qj * ec;
    acc[1] += R(0.5) * fs * dx * dx;
    acc[2] += R(0.5) * fs * dy * dy;
    acc[3] += R(0.5) * fs * dz * dz;
    acc[4] += R(0.5) * fs * dx * dy;
    acc[5] += R(0.5) * fs * dx * dz;
    acc[6] += R(0.5) * fs * dy * dz;
}

// All pairs within r_c under the minimum image (r_c <= L/2).  Each block
// stages tiles of 256 particles in shared memory.  Its partial sums go to
// the scratch array; the last block to finish adds them in block order
// (deterministic), writes `out` and resets the counter.
template <typename R>
__global__ void __launch_bounds__(kThreads) k_real_space_noalloc(int N, const R* __restrict__ pos,
                                                                 const R* __restrict__ q, R L0, R L1, R L2, R iL0,
                                                                 R iL1, R iL2, R rc2,
                                                                 R alpha, R two_a_sqpi, double ke,
                                                                 R* __restrict__ F, R* __restrict__ phi,
                                                                 NoAllocScratch* __restrict__ scratch,
                                                                 double* __restrict__ out)
{
    __shared__ R sx[kThreads], sy[kThreads], sz[kThreads], sq[kThreads];
    __shared__ double red[32 * 7];
    __shared__ bool last;
    const int i = blockIdx.x * kThreads + threadIdx.x;
    R xi = R(0), yi = R(0), zi = R(0), qi = R(0);
    if (i < N) {
        xi = wrap_to_box(pos[3 * (size_t)i], L0, iL0);
        yi = wrap_to_box(pos[3 * (size_t)i + 1], L1, iL1);
        zi = wrap_to_box(pos[3 * (size_t)i + 2], L2, iL2);
        qi = q[i];
    }
    R f[3] = {R(0), R(0), R(0)}, ph = R(0);
    R acc[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    for (int j0 = 0; j0 < N; j0 += kThreads) {
        const int j = j0 + threadIdx.x;
        if (j < N) {
            sx[threadIdx.x] = wrap_to_box(pos[3 * (size_t)j], L0, iL0);
            sy[threadIdx.x] = wrap_to_box(pos[3 * (size_t)j + 1], L1, iL1);
            sz[threadIdx.x] = wrap_to_box(pos[3 * (size_t)j + 2], L2, iL2);
            sq[threadIdx.x] = q[j];
        }
        __syncthreads();
        const int nt = min(kThreads, N - j0);
        if (i < N) {
            for (int t = 0; t < nt; t++) {
                if (j0 + t == i) continue;
                R dx = xi - sx[t], dy = yi - sy[t], dz = zi - sz[t];
                dx -= L0 * rint(dx * iL0);
                dy -= L1 * rint(dy * iL1);
                dz -= L2 * rint(dz * iL2);
                pair_sum<R>(dx, dy, dz, qi, sq[t], rc2, alpha, two_a_sqpi, f, ph, acc);
            }
        }
        __syncthreads();
    }
    if (i < N) {
        if (F) {
            F[3 * (size_t)i] = (R)ke * f[0];
            F[3 * (size_t)i + 1] = (R)ke * f[1];
            F[3 * (size_t)i + 2] = (R)ke * f[2];
        }
        if (phi) phi[i] = (R)ke * ph;
    }
    enuf::block_reduce_to_double<R, 7>(acc, scratch->partial + 8 * (size_t)blockIdx.x, red);
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(&scratch->counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // last block: warp w < 7 sums component w over the blocks in order
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w < 7) {
        double a = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) a += __ldcg(scratch->partial + 8 * b + w);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) red[w] = ke * a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = red[0];
        out[1] = red[1]; out[2] = red[4]; out[3] = red[5];
        out[4] = red[4]; out[5] = red[2]; out[6] = red[6];
        out[7] = red[5]; out[8] = red[6]; out[9] = red[3];
        scratch->counter = 0u;
    }
}

// Device address of the scratch array on the current device (looked up once
// per device, with that device current).
int scratch_for_current_device(NoAllocScratch** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return nfail(ENUF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return nfail(ENUF_EUNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return nfail(ENUF_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = static_cast<NoAllocScratch*>(p);
    }
    *out = g_scratch_ptr[dev];
    return ENUF_OK;
}

}  // namespace

extern "C" {

int enuf_real_space_noalloc(const void* pos, const void* q, int64_t N, const double* L, double alpha, double r_c,
                            double coulomb_k, int precision, void* F, void* phi, double* out, void* cuda_stream)
{
    enuf::set_last_error("");
    if (!pos || !q || !L || !out) return nfail(ENUF_EINVAL, "pos, q, L and out are required");
    if (N < 1) return nfail(ENUF_EINVAL, "N must be >= 1");
    if (N > (int64_t)kMaxBlocks * kThreads)
        return nfail(ENUF_EUNSUPPORTED, "N exceeds the fixed scratch of enuf_real_space_noalloc (at most " +
                                            std::to_string((long long)kMaxBlocks * kThreads) + " particles)");
    for (int t = 0; t < 3; t++)
        if (!(L[t] > 0.0)) return nfail(ENUF_EINVAL, "box edges must be positive");
    const double Lmin = std::fmin(L[0], std::fmin(L[1], L[2]));
    if (!(r_c > 0.0) || r_c > 0.5 * Lmin) return nfail(ENUF_EINVAL, "r_c must satisfy 0 < r_c <= min(L)/2");
    if (!(alpha > 0.0)) return nfail(ENUF_EINVAL, "alpha must be positive");
    if (precision != ENUF_FP64 && precision != ENUF_MIXED) return nfail(ENUF_EINVAL, "unknown precision");
    if (coulomb_k == 0.0) coulomb_k = 1.0;
    NoAllocScratch* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != ENUF_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // the counter must start at zero (a previous call may have been cut short)
    cudaError_t e = cudaMemsetAsync(&scratch->counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return nfail(ENUF_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int nb = (int)((N + kThreads - 1) / kThreads);
    const double two_a_sqpi = 2.0 * alpha / std::sqrt(3.14159265358979323846);
    if (precision == ENUF_FP64)
        k_real_space_noalloc<double><<<nb, kThreads, 0, st>>>(
            (int)N, (const double*)pos, (const double*)q, L[0], L[1], L[2], 1.0 / L[0], 1.0 / L[1], 1.0 / L[2],
            r_c * r_c, alpha, two_a_sqpi, coulomb_k,
            (double*)F, (double*)phi, scratch, out);
    else
        k_real_space_noalloc<float><<<nb, kThreads, 0, st>>>(
            (int)N, (const float*)pos, (const float*)q, (float)L[0], (float)L[1], (float)L[2], (float)(1.0 / L[0]),
            (float)(1.0 / L[1]), (float)(1.0 / L[2]), (float)(r_c * r_c),
            (float)alpha, (float)two_a_sqpi, coulomb_k, (float*)F, (float*)phi, scratch, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return nfail(ENUF_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return ENUF_OK;
}

}  // extern "C"
