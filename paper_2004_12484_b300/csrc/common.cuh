// common.cuh -- small device types and helpers shared by the ENUF kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace enuf {

// complex value types
template <typename R> struct Cpx;
template <> struct Cpx<float> { using T = float2; };
template <> struct Cpx<double> { using T = double2; };

// sorted particle record: offset inside its bin (x, y, z) and charge
struct __align__(16) f4 { float x, y, z, w; };
struct __align__(32) d4 { double x, y, z, w; };
template <typename R> struct Rec;
template <> struct Rec<float> { using T = f4; };
template <> struct Rec<double> { using T = d4; };

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return V{a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return V{a.x - b.x, a.y - b.y}; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b)
{
    return V{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename V> __device__ __forceinline__ V cconj(V a) { return V{a.x, -a.y}; }

__device__ __forceinline__ float dexp(float x) { return expf(x); }
__device__ __forceinline__ double dexp(double x) { return exp(x); }
__device__ __forceinline__ float derfc(float x) { return erfcf(x); }
__device__ __forceinline__ double derfc(double x) { return erfc(x); }
__device__ __forceinline__ float dsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }

// Asynchronous global -> shared copies (cp.async): a thread issues all of
// its copies before waiting, so their latencies overlap instead of following
// one another.  Copies of !valid elements read nothing and fill zeros.
// cp_async_wait_all waits for all of the thread's copies (a barrier then
// publishes them to the CTA).
__device__ __forceinline__ void cp_async_bytes8(void* dst, const void* src, bool valid)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 8u : 0u)
                 : "memory");
}
__device__ __forceinline__ void cp_async_bytes16(void* dst, const void* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(valid ? 16u : 0u)
                 : "memory");
}
// one complex value (8 bytes in single, 16 in double precision)
__device__ __forceinline__ void cp_async_cpx(float2* dst, const float2* src, bool valid)
{
    cp_async_bytes8(dst, src, valid);
}
__device__ __forceinline__ void cp_async_cpx(double2* dst, const double2* src, bool valid)
{
    cp_async_bytes16(dst, src, valid);
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Programmatic dependent launch.  The chain's kernels are launched with
// programmatic stream serialisation: a kernel may be launched as soon as its
// predecessor's CTAs have exited, before the predecessor grid is retired, and
// calls this before it reads or writes anything an earlier kernel of the
// chain touches (griddepcontrol.wait returns once the predecessor grid has
// completed and its memory is visible; at once when the launch had no such
// predecessor).  No kernel signals its dependents early: dependents made
// resident while the predecessor's last wave still ran crowded onto the
// SMs that wave had left free and cost 10 % of the step (measured).
__device__ __forceinline__ void pdl_wait()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Division by a divisor d (1 <= d < 2^16) fixed at launch, for dividends
// n < 2^16: q = (n m) >> 32 with m = floor(2^32 / d) + 1 is exact in that
// range (the error n (m - 2^32 / d) / 2^32 < 2^-16 < 1 / d cannot carry the
// fraction n / d past an integer), and costs a multiply instead of the ~20
// instructions of a general integer division.
struct FDiv {
    uint32_t d;
    unsigned long long m;
    static FDiv make(uint32_t dv)
    {
        FDiv f;
        f.d = dv;
        f.m = 0x100000000ull / dv + 1;
        return f;
    }
    __device__ __forceinline__ uint32_t div(uint32_t n) const { return (uint32_t)(((unsigned long long)n * m) >> 32); }
};

template <typename R> __device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Bytes of dynamic shared memory the block was launched with.
__device__ __forceinline__ unsigned dynamic_smem_bytes()
{
    unsigned v;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
    return v;
}

// ------------------------------------------------------------------ bounds checks
// The checked build of the library (compiled with ENUF_BOUNDS_CHECK) tests
// every index derived from the particle data, the bin counts, the work lists
// and the thread decomposition of the kernels against the extent it must stay
// within, before the access it guards.  A failed test counts the failure,
// records the first one (source file, line, index and extent; read by
// enuf_bounds_status) and skips the access, so that the kernel carries on
// and never traps.  In the normal build ENUF_IN is the constant true and
// the checks vanish at compile time.
#ifdef ENUF_BOUNDS_CHECK
struct BoundsLog {
    unsigned long long fails;
    long long index, extent;
    int line;
    char file[44];
};
static __device__ BoundsLog g_bounds;

static __device__ __noinline__ bool bounds_fail(long long i, long long n, int line, const char* file)
{
    if (atomicAdd(&g_bounds.fails, 1ull) == 0ull) {
        g_bounds.index = i;
        g_bounds.extent = n;
        g_bounds.line = line;
        const char* base = file;
        for (const char* c = file; *c; c++)
            if (*c == '/') base = c + 1;
        int k = 0;
        for (; k < (int)sizeof(g_bounds.file) - 1 && base[k]; k++) g_bounds.file[k] = base[k];
        g_bounds.file[k] = 0;
    }
    return false;
}
#define ENUF_IN(i, n)                                                                        \
    ((unsigned long long)(long long)(i) < (unsigned long long)(long long)(n) ||             \
     ::enuf::bounds_fail((long long)(i), (long long)(n), __LINE__, __FILE__))
#else
#define ENUF_IN(i, n) true
#endif
// An index of the thread decomposition, checked and, when out of range,
// replaced by 0 (kernels with block-wide barriers cannot leave early).
#define ENUF_CLAMP(i, n) (ENUF_IN(i, n) ? (i) : 0)

// Status bits written by kernels into the workspace status word.
enum : int {
    ST_NONFINITE = 1,  // a non-finite position or charge was seen
    ST_WORKLIST = 2,   // the bin work list overflowed its bound (internal error)
    ST_TIMEOUT = 4,    // a bounded wait for asynchronous copies gave up (internal error)
};

// ------------------------------------------------------------------ bulk copies
// Copies by the TMA engine from global to shared memory, completed on an
// mbarrier in the CTA's shared memory: non-tensor ("bulk") copies of a
// multiple of 16 bytes between 16-byte aligned addresses, and boxes of a
// tensor described by a tensor map.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the asynchronous proxy
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of transactions still to come.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// One box of a 4-dimensional tensor (tile mode) from global to shared memory
// through the tensor map at `tmap` (a __grid_constant__ kernel parameter);
// coordinates are element indices, innermost first, and may lie outside the
// tensor (those elements are filled with zeros).  The destination must be
// 128-byte aligned.
__device__ __forceinline__ void tma_load_4d(void* dst, const void* tmap, int c0, int c1, int c2, int c3, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

// Waits for the barrier's phase `parity` to complete, giving up after
// `limit` polls (each poll may suspend the thread for a while); returns
// whether the phase completed.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit)
{
    const uint32_t a = smem_addr(bar);
    for (int i = 0; i < limit; i++) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Block reduction of NV values per thread.  Each warp sums in type R, the
// warp totals are added in double; threads 0..NV-1 write out[0..NV).
// Must be called by every thread of the block.
template <typename R, int NV>
__device__ __forceinline__ void block_reduce_to_double(R (&v)[NV], double* out, double* smem /* 32*NV */)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < NV; k++) {
        R s = warp_sum(v[k]);
        if (lane == 0) smem[warp * NV + k] = (double)s;
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double t = 0.0;
        for (int w = 0; w < nw; w++) t += smem[w * NV + threadIdx.x];
        out[threadIdx.x] = t;
    }
    __syncthreads();
}

}  // namespace enuf
