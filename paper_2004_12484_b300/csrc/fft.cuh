// fft.cuh -- hand-written 3D FFT of the ENUF grid, pruned to the retained
// frequency cube |n_t| <= n_c, with the reciprocal-space step fused into the
// middle (z) pass.
//
// Forward chain (the spreading, transform and scaling stages of Sec. 3.1):
//   k_fx  real rows along x -> half spectrum, keep kx = 0..n_c
//   k_fy  along y for each kx, keep ky in the band (2 n_c + 1 values)
//         (k_fxy: both in one kernel per z-plane where the kept plane fits
//         in shared memory, grids 32-256)
//   k_fz  along z for each (ky, kx) pencil, then for every retained n:
//         S(n) = D(n) ghat(n) (scaling by the window's Fourier coefficients),
//         energy and virial (Eq. 38), and the subdivided spectra of the
//         force field and potential (Eq. 41-42), then the inverse transform
//         along z of each field (the split into field spectra and the first
//         inverse pass); k_fzw does the same with radix-8 passes and the
//         fields one after the other (512, and 128 and 256 in single
//         precision)
// Inverse chain (the inverse transforms ahead of the interpolation):
//   k_iy  along y (band -> full length) for each field and kx
//   k_ix  half spectrum kx = 0..n_c -> real rows (complex-to-real)
//         (k_iyx: both in one kernel per z-plane and field, grids 32-256)
//
// Every 1D transform is a Stockham autosort FFT: each thread holds R (16,
// 8, 4 or 2) elements in registers per pass, applies the twiddles and a
// radix-R butterfly; the passes exchange through shared memory, the first
// loads from and the last stores to global memory directly.  The
// real-to-complex rows use the half-length complex transform of the packed
// row (x_{2j} + i x_{2j+1}) and the usual even/odd split.
// Sign conventions: forward sum_l g_l exp(-2 pi i k l / M), inverse with
// exp(+...), both unnormalised.
#pragma once
#include "common.cuh"

namespace enuf {

// ---------------------------------------------------------------- butterflies
template <typename V, bool INV> __device__ __forceinline__ void dft2(V* v)
{
    V a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
}

// multiply by -i (forward) or +i (inverse)
template <typename V, bool INV> __device__ __forceinline__ V mul_mi(V d)
{
    return INV ? V{-d.y, d.x} : V{d.y, -d.x};
}

template <typename V, bool INV> __device__ __forceinline__ void dft4(V* v)
{
    V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]), t2 = cadd(v[1], v[3]);
    V t3 = mul_mi<V, INV>(csub(v[1], v[3]));
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
}

template <typename V, bool INV> __device__ __forceinline__ void dft8(V* v)
{
    using R = decltype(v[0].x);
    V e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<V, INV>(e);
    dft4<V, INV>(o);
    const R s = (R)0.70710678118654752440;
    // o[k] *= exp(-+ 2 pi i k / 8)
    V o1 = o[1], o3 = o[3];
    if (!INV) {
        o[1] = V{(o1.x + o1.y) * s, (o1.y - o1.x) * s};
        o[3] = V{(o3.y - o3.x) * s, -(o3.x + o3.y) * s};
    } else {
        o[1] = V{(o1.x - o1.y) * s, (o1.x + o1.y) * s};
        o[3] = V{-(o3.x + o3.y) * s, (o3.x - o3.y) * s};
    }
    o[2] = mul_mi<V, INV>(o[2]);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        v[k] = cadd(e[k], o[k]);
        v[k + 4] = csub(e[k], o[k]);
    }
}

// 16-point DFT in registers as 4 x 4: DFT4 over n1 of x[4 n1 + n2] for each
// n2, twiddles W16^(n2 k1), DFT4 over n2; outputs in natural order.
template <typename V, bool INV> __device__ __forceinline__ void dft16(V* v)
{
    using R = decltype(v[0].x);
    V a[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; n2++) {
        V t[4] = {v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]};
        dft4<V, INV>(t);
#pragma unroll
        for (int k1 = 0; k1 < 4; k1++) a[n2][k1] = t[k1];
    }
    // W16^j = exp(-+ 2 pi i j / 16) for the products n2 k1 in {1, 2, 3, 4, 6, 9}
    const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173, h = (R)0.70710678118654752440;
    const R sg = INV ? R(1) : R(-1);  // sign of the imaginary part of W16^1
    auto tw = [&](V x, R c, R sn) { return V{x.x * c - x.y * sn, x.x * sn + x.y * c}; };
    a[1][1] = tw(a[1][1], c1, sg * s1);
    a[1][2] = tw(a[1][2], h, sg * h);
    a[1][3] = tw(a[1][3], s1, sg * c1);
    a[2][1] = tw(a[2][1], h, sg * h);
    a[2][2] = tw(a[2][2], R(0), sg);
    a[2][3] = tw(a[2][3], -h, sg * h);
    a[3][1] = tw(a[3][1], s1, sg * c1);
    a[3][2] = tw(a[3][2], -h, sg * h);
    a[3][3] = tw(a[3][3], -c1, -sg * s1);
#pragma unroll
    for (int k1 = 0; k1 < 4; k1++) {
        V t[4] = {a[0][k1], a[1][k1], a[2][k1], a[3][k1]};
        dft4<V, INV>(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; k2++) v[k1 + 4 * k2] = t[k2];
    }
}

template <typename V, int R, bool INV> __device__ __forceinline__ void dftR(V* v)
{
    if constexpr (R == 16) dft16<V, INV>(v);
    else if constexpr (R == 8) dft8<V, INV>(v);
    else if constexpr (R == 4) dft4<V, INV>(v);
    else dft2<V, INV>(v);
}

// Threads serving one transform of length N when passes use radix MR (16,
// 8 or 4) and below: each thread holds MR elements per pass.
template <int N, int MR = 8> struct FftThreads {
    static constexpr int NT = N >= MR ? N / MR : 1;
};

// Radix of the register passes of the x-row kernels (k_fx, k_ix): 16 for
// the half-length 256 of a 512 grid (two radix-16 passes, one exchange),
// else 8.
template <int N> struct RowMR {
    static constexpr int V = N == 256 ? 16 : 8;
};

// Radix of the passes of N points in the fused x-y kernels of an M grid
// (k_fxy, INV = false; k_iyx, INV = true): 16 in single precision for the
// 256-point columns and 128-point rows of a 256 grid and for the 128-point
// columns of the inverse kernel of a 128 grid (two passes, one exchange,
// instead of radix 8, 8 and 2 or 4); else 8.  At 128 the forward kernel
// keeps radix 8: its 128 CTAs (one per plane) need the threads of the
// 16-point columns for the row batches (12.3 against 14.3 us).  The block
// size (the host's xy_threads) stays within XyBounds<R, M, INV>::T, which
// leaves the radix-16 kernels room for their registers.
template <typename R, int N, int M, bool INV> struct XyMR {
    static constexpr int V = (sizeof(R) == 4 && (N == 256 || (N == 128 && (M == 256 || INV)))) ? 16 : 8;
};
template <typename R, int M, bool INV> struct XyBounds {
    static constexpr int T = sizeof(R) != 4 ? 1024 : (M == 256 ? 544 : (M == 128 ? (INV ? 288 : 544) : 1024));
};

// Shared-memory layout of one transform: element e lives at pidx(e) = e +
// e/16, which spreads the stride-R writes of the first Stockham passes over
// all banks.  A transform of length N occupies PadLen<N>::V slots.
__device__ __forceinline__ int pidx(int e) { return e + (e >> 4); }
template <int N> struct PadLen {
    static constexpr int V = N + N / 16;
};

// One Stockham pass of radix R on NTR contiguous transforms of length N in
// shared memory (transform r starts at x + r * trs), served by NT = max(1,
// N/8) threads (t = 0..NT-1) that each handle the same butterflies of all NTR
// transforms.  All threads of the CTA must call it (it contains barriers).
// W is the table exp(-2 pi i k / Mtab), k < Mtab, and ws = Mtab / N.  Element e of a
// transform is stored at pidx(e).
template <typename V, int N, int R, int Ns, bool INV, int NTR, int MR>
__device__ __forceinline__ void stockham_pass(V* x, int trs, int t, const V* __restrict__ W, int ws)
{
    constexpr int NT = FftThreads<N, MR>::NT;
    constexpr int NB = N / R;
    constexpr int PER = NB / NT;
    V v[NTR][PER][R];
#pragma unroll
    for (int b = 0; b < PER; b++) {
        const int j = t + b * NT;
        const int k = j & (Ns - 1);
        V tw[R];
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; r++) {
                tw[r] = W[(r * k * (N / (Ns * R))) * ws];
                if (INV) tw[r].y = -tw[r].y;
            }
        }
#pragma unroll
        for (int q = 0; q < NTR; q++) {
#pragma unroll
            for (int r = 0; r < R; r++) v[q][b][r] = x[q * trs + pidx(j + r * NB)];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; r++) v[q][b][r] = cmul(v[q][b][r], tw[r]);
            }
            dftR<V, R, INV>(v[q][b]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < PER; b++) {
        const int j = t + b * NT;
        const int k = j & (Ns - 1);
        const int d = (j - k) * R + k;
#pragma unroll
        for (int q = 0; q < NTR; q++) {
#pragma unroll
            for (int r = 0; r < R; r++) x[q * trs + pidx(d + r * Ns)] = v[q][b][r];
        }
    }
    __syncthreads();
}

template <typename V, int N, int Ns, bool INV, int NTR, int MR> struct FftPasses {
    static __device__ __forceinline__ void run(V* x, int trs, int t, const V* __restrict__ W, int ws)
    {
        constexpr int R = (MR >= 8 && Ns * 8 <= N) ? 8 : ((Ns * 4 <= N) ? 4 : 2);
        stockham_pass<V, N, R, Ns, INV, NTR, MR>(x, trs, t, W, ws);
        FftPasses<V, N, Ns * R, INV, NTR, MR>::run(x, trs, t, W, ws);
    }
};
template <typename V, int N, bool INV, int NTR, int MR> struct FftPasses<V, N, N, INV, NTR, MR> {
    static __device__ __forceinline__ void run(V*, int, int, const V* __restrict__, int) {}
};

template <typename V, int N, bool INV, int MR = 8>
__device__ __forceinline__ void fft_smem(V* x, int t, const V* __restrict__ W, int ws)
{
    FftPasses<V, N, 1, INV, 1, MR>::run(x, 0, t, W, ws);
}

// NTR transforms at x, x + trs, ... handled together by the same threads.
template <typename V, int N, bool INV, int NTR, int MR = 8>
__device__ __forceinline__ void fft_smem_multi(V* x, int trs, int t, const V* __restrict__ W, int ws)
{
    FftPasses<V, N, 1, INV, NTR, MR>::run(x, trs, t, W, ws);
}

// ---------------------------------------------------------------- register passes
// The same Stockham passes with the data of the first pass taken from, and
// the results of the last pass left in, registers: thread t of the NT
// threads serving a transform holds v[m] = x[t + NT m] (m < E = N / NT) on
// entry and v[m] = X[t + NT m] on exit, so a transform loaded from and
// stored to global memory directly touches shared memory only between
// passes (passes - 1 exchanges through the transform's buffer at x, PadLen
// slots).  NTR transforms (buffers x + q trs) per thread, as in
// stockham_pass.  All threads of the CTA must call it (it contains
// barriers).
template <typename V, int N, int Ns, bool INV, int NTR, int MR> struct RegPasses {
    static constexpr int R =
        (MR >= 16 && Ns * 16 <= N) ? 16 : ((MR >= 8 && Ns * 8 <= N) ? 8 : ((Ns * 4 <= N) ? 4 : 2));
    static constexpr int NT = FftThreads<N, MR>::NT;
    static constexpr int NB = N / R, PER = NB / NT, E = N / NT;
    // v[q][m]: element m of transform q (m = b + PER r for butterfly b, leg r)
    static __device__ __forceinline__ void run(V (&v)[NTR][E], V* x, int trs, int t, const V* __restrict__ W, int ws)
    {
#pragma unroll
        for (int b = 0; b < PER; b++) {
            const int j = t + b * NT;
            const int k = j & (Ns - 1);
            V tw[R];
            if (Ns > 1) {
#pragma unroll
                for (int r = 1; r < R; r++) {
                    tw[r] = W[(r * k * (N / (Ns * R))) * ws];
                    if (INV) tw[r].y = -tw[r].y;
                }
            }
#pragma unroll
            for (int q = 0; q < NTR; q++) {
                V u[R];
#pragma unroll
                for (int r = 0; r < R; r++) u[r] = v[q][b + PER * r];
                if (Ns > 1) {
#pragma unroll
                    for (int r = 1; r < R; r++) u[r] = cmul(u[r], tw[r]);
                }
                dftR<V, R, INV>(u);
#pragma unroll
                for (int r = 0; r < R; r++) v[q][b + PER * r] = u[r];
            }
        }
        if constexpr (Ns * R < N) {
            // exchange: results to their autosort positions, then the next
            // pass's inputs x[j + r N / R'] into the same register slots
            using Next = RegPasses<V, N, Ns * R, INV, NTR, MR>;
#pragma unroll
            for (int b = 0; b < PER; b++) {
                const int j = t + b * NT;
                const int k = j & (Ns - 1);
                const int d = (j - k) * R + k;
#pragma unroll
                for (int q = 0; q < NTR; q++) {
#pragma unroll
                    for (int r = 0; r < R; r++) x[q * trs + pidx(d + r * Ns)] = v[q][b + PER * r];
                }
            }
            __syncthreads();
#pragma unroll
            for (int b = 0; b < Next::PER; b++) {
                const int j = t + b * NT;
#pragma unroll
                for (int q = 0; q < NTR; q++) {
#pragma unroll
                    for (int r = 0; r < Next::R; r++) v[q][b + Next::PER * r] = x[q * trs + pidx(j + r * Next::NB)];
                }
            }
            __syncthreads();
            Next::run(v, x, trs, t, W, ws);
        }
    }
};

template <typename V, int N, bool INV, int MR = 8>
__device__ __forceinline__ void fft_reg(V (&v)[1][N / FftThreads<N, MR>::NT], V* x, int t, const V* __restrict__ W,
                                        int ws)
{
    RegPasses<V, N, 1, INV, 1, MR>::run(v, x, 0, t, W, ws);
}

// Copies the twiddle table exp(-2 pi i k / M), k < M, into shared memory
// (asynchronously: complete after the kernel's next cp_async_wait_all and
// barrier).
template <typename V>
__device__ __forceinline__ const V* stage_twiddles(V* dst, const V* __restrict__ src, int M)
{
    for (int i = threadIdx.x; i < M; i += blockDim.x) cp_async_cpx(dst + i, src + i, true);
    return dst;
}

// Row of a batch served by row slot r of the x pass of k_iyx (NTX threads
// a row, RB rows a batch).  A half-warp (the unit of a 64-bit
// shared-memory access) holds 16 / NTX row slots; within each full block of
// 16 slots they take rows NTX apart instead of consecutive ones, so that
// the half-warp's accesses to one kx column of the plane buffer (element kx
// LD + pidx(y)) fall on 16 distinct bank pairs: LD tx + y mod 16 is distinct
// for tx < NTX and y = h + NTX i (i < 16 / NTX) whenever LD is odd, where
// consecutive rows (LD = 1 mod 16 at M = 256) gave only NTX + 1 values.
// The blocks must start on multiples of 16 rows (pidx pads after every 16),
// so a batch covers RBU = RB rounded down to whole blocks where that takes
// no more batches (slots RBU.. then stay idle), else RB rows with the slots
// past the last full block on their own row.  (Measured: k_iyx 19.8 -> 18.4
// us at M = 128, 129.0 -> 124.9 us at 256; the same order in the x pass of
// k_fxy, whose plane accesses are stores, made it slower, 12.5 -> 14.0 us.)
__device__ __forceinline__ int batch_rows(int RB, int M)
{
    const int RBU = RB & ~15;
    return (RBU > 0 && (M + RBU - 1) / RBU == (M + RB - 1) / RB) ? RBU : RB;
}
template <int NTX> __device__ __forceinline__ int batch_row(int r, int RB)
{
    static_assert(NTX >= 1 && (NTX & (NTX - 1)) == 0, "a power of two");
    if constexpr (NTX >= 16) {
        return r;  // a half-warp serves one row
    } else {
        constexpr int Q = 16 / NTX;
        if (r >= (RB & ~15)) return r;
        const int s = r & 15;
        return (r & ~15) + s / Q + NTX * (s % Q);
    }
}

// ---------------------------------------------------------------- geometry
struct FftGeom {
    int nc;    // retained cutoff
    int Kx;    // nc + 1 stored kx values
    int Kb;    // 2 nc + 1 band values along y and z
    int P;     // Kb * Kx pencils along z
    int W;     // transforms (columns / pencils) per CTA in k_fy / k_fz / k_iy
    int rows;  // rows per CTA in k_fx / k_ix
    FDiv fKx, fW, fKxR;  // division by Kx, W and (k_iyx) Kx rounded up to its column batch
};

// Launch bounds of the separate passes of the 512 grid in single precision:
// CTAs of at most 512 threads for the y passes, three of them an SM (at
// most 40 registers; ionic-liquid inverse y 0.495 -> 0.395 ms, forward y
// 0.156 -> 0.137 ms against two), and for the 256-thread x-row passes five
// (forward x, 0.238 -> 0.225 ms) or four (inverse x: with five, 0.608 ->
// 0.614 ms; with six both spill).
template <typename R, int M> struct SepBounds {
    static constexpr bool big = M >= 512 && sizeof(R) == 4;
    static constexpr int YT = big ? 512 : 1024, YB = big ? 3 : 1, FXB = big ? 5 : 1, IXB = big ? 4 : 1;
};

// ---------------------------------------------------------------- k_fx
// grid: ceil(M*M / rows) blocks, rows * NT(M/2) threads.  Clears the grid
// rows it reads (the spreading accumulates into a zeroed grid).  Thread t of
// a row loads the packed pairs z_j = x_{2j} + i x_{2j+1}, j = t + NT m,
// straight from the grid row, transforms with register passes, and the
// even/odd split X_k = (Z_k + conj Z_{M/2-k})/2 - i/2 e^{-2 pi i k/M}
// (Z_k - conj Z_{M/2-k}) of the kept kx <= n_c reads the partners from
// shared memory.
template <typename R, int M>
__global__ void __launch_bounds__(256, SepBounds<R, M>::FXB) k_fx(R* __restrict__ grid, typename Cpx<R>::T* __restrict__ C1, FftGeom g,
                     const typename Cpx<R>::T* __restrict__ Wg)
{
    using V = typename Cpx<R>::T;
    constexpr int MH = M / 2, MRX = RowMR<MH>::V, NT = FftThreads<MH, MRX>::NT, RS = PadLen<MH>::V, E = MH / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* s = reinterpret_cast<V*>(smraw);
    const int rows = g.rows, row0 = blockIdx.x * rows, nrows = M * M;
    const V* sW = stage_twiddles(s + rows * RS, Wg, M);
    const int r0 = threadIdx.x / NT, t = threadIdx.x % NT, r = ENUF_CLAMP(r0, rows), row = row0 + r;
    const bool live = row < nrows;
    V* gin = reinterpret_cast<V*>(grid) + (size_t)(live ? row : 0) * MH;
    V v[1][E];
#pragma unroll
    for (int m = 0; m < E; m++) v[0][m] = live ? gin[t + NT * m] : V{R(0), R(0)};
    cp_async_wait_all();
    __syncthreads();
    V* x = s + r * RS;
    fft_reg<V, MH, false, MRX>(v, x, t, sW, 2);
    // the grid is left zeroed for the next spreading (each element is
    // cleared by the thread that read it, once its value is in use: a
    // store right behind the load of the same address waits for it)
    if (live) {
#pragma unroll
        for (int m = 0; m < E; m++) gin[t + NT * m] = V{R(0), R(0)};
    }
#pragma unroll
    for (int m = 0; m < E; m++) x[pidx(t + NT * m)] = v[0][m];
    __syncthreads();
    if (!live) return;
    const int Kx = g.Kx;
    for (int k = t; k < Kx; k += NT) {
        const V zk = x[pidx(k % MH)];
        const V zc = cconj(x[pidx((MH - k) % MH)]);
        const V fe = V{R(0.5) * (zk.x + zc.x), R(0.5) * (zk.y + zc.y)};
        const V d = csub(zk, zc);
        const V fo = V{R(0.5) * d.y, R(-0.5) * d.x};  // -i/2 (zk - zc)
        if (ENUF_IN((size_t)row * Kx + k, (size_t)nrows * Kx)) C1[(size_t)row * Kx + k] = cadd(fe, cmul(sW[k], fo));
    }
}

// ---------------------------------------------------------------- k_fxy
// Fused forward x and y passes for grids whose pruned plane fits in shared
// memory: one CTA per z-plane (grid: M blocks, CB * NT(M) threads, CB
// columns per batch).  Clears the grid plane it reads (the spreading
// accumulates into a zeroed grid).  The x-rows are transformed in batches
// (loaded straight into registers), their kept kx columns stored transposed
// in a plane buffer, transformed along y (thread (w, t) = (tid % CB, tid /
// CB) on column k0 + w) and the band rows stored to C2 from registers.
template <typename R, int M>
__global__ void __launch_bounds__(XyBounds<R, M, false>::T) k_fxy(R* __restrict__ grid, typename Cpx<R>::T* __restrict__ C2,
                                              FftGeom g, const typename Cpx<R>::T* __restrict__ Wg)
{
    using V = typename Cpx<R>::T;
    constexpr int MH = M / 2, MRX = XyMR<R, MH, M, false>::V, MRY = XyMR<R, M, M, false>::V;
    constexpr int NTX = FftThreads<MH, MRX>::NT, NTY = FftThreads<M, MRY>::NT, LD = PadLen<M>::V + 1;
    constexpr int RS = PadLen<MH>::V, EX = MH / NTX, EY = M / NTY;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int Kx = g.Kx, Kb = g.Kb, nc = g.nc;
    const int RB = blockDim.x / NTX;  // rows per batch
    const int CB = blockDim.x / NTY;  // columns per batch
    V* rowbuf = reinterpret_cast<V*>(smraw);
    V* plane = rowbuf + RB * RS;  // [Kx (rounded to CB)][LD]
    V* sW = plane + ((Kx + CB - 1) / CB) * CB * LD;
    stage_twiddles(sW, Wg, M);
    pdl_wait();
    const int z0 = blockIdx.x, z = ENUF_CLAMP(z0, M);
    V* gin = reinterpret_cast<V*>(grid + (size_t)z * M * M);
    const int r0 = threadIdx.x / NTX, tx = threadIdx.x % NTX, r = ENUF_CLAMP(r0, RB);
    cp_async_wait_all();
    __syncthreads();
    for (int y0 = 0; y0 < M; y0 += RB) {
        const int y = y0 + r;
        const bool live = y < M;
        V* row = gin + (size_t)(live ? y : 0) * MH;
        V v[1][EX];
#pragma unroll
        for (int m = 0; m < EX; m++) v[0][m] = live ? row[tx + NTX * m] : V{R(0), R(0)};
        V* x = rowbuf + r * RS;
        fft_reg<V, MH, false, MRX>(v, x, tx, sW, 2);
        // the grid is left zeroed for the next spreading (each element is
        // cleared by the thread that read it, once its value is in use)
        if (live) {
#pragma unroll
            for (int m = 0; m < EX; m++) row[tx + NTX * m] = V{R(0), R(0)};
        }
#pragma unroll
        for (int m = 0; m < EX; m++) x[pidx(tx + NTX * m)] = v[0][m];
        __syncthreads();
        if (live) {
            for (int k = tx; k < Kx; k += NTX) {
                const V zk = x[pidx(k % MH)];
                const V zc = cconj(x[pidx((MH - k) % MH)]);
                const V fe = V{R(0.5) * (zk.x + zc.x), R(0.5) * (zk.y + zc.y)};
                const V d = csub(zk, zc);
                const V fo = V{R(0.5) * d.y, R(-0.5) * d.x};
                plane[k * LD + pidx(y)] = cadd(fe, cmul(sW[k], fo));
            }
        }
        __syncthreads();
    }
    const int ty0 = threadIdx.x / CB, w = threadIdx.x - ty0 * CB;
    const int ty = ENUF_CLAMP(ty0, NTY);  // ty < NT(M): blockDim = CB NT(M)
    V* dst = C2 + (size_t)z * Kb * Kx;
    for (int k0 = 0; k0 < Kx; k0 += CB) {
        const int kx = ENUF_CLAMP(k0 + w, ((Kx + CB - 1) / CB) * CB);
        V* col = plane + kx * LD;
        V v[1][EY];
#pragma unroll
        for (int m = 0; m < EY; m++) v[0][m] = col[pidx(ty + NTY * m)];
        __syncthreads();
        fft_reg<V, M, false, MRY>(v, col, ty, sW, 1);
        if (kx < Kx) {
#pragma unroll
            for (int m = 0; m < EY; m++) {
                const int ky = ty + NTY * m;
                int kb = -1;
                if (ky <= nc) kb = ky;
                else if (ky >= M - nc) kb = ky - (M - Kb);
                if (kb >= 0 && ENUF_IN(kb, Kb)) dst[(size_t)kb * Kx + kx] = v[0][m];
            }
        }
    }
}

// ---------------------------------------------------------------- k_fy
// grid: (ceil(Kx / W), M) blocks, W * NT(M) threads.  Thread (w, t) = (tid %
// W, tid / W) serves column kx0 + w: loads y = t + NT m straight from C1,
// register passes, stores the band rows to C2.
template <typename R, int M>
__global__ void __launch_bounds__(SepBounds<R, M>::YT, SepBounds<R, M>::YB) k_fy(const typename Cpx<R>::T* __restrict__ C1, typename Cpx<R>::T* __restrict__ C2, FftGeom g,
                     const typename Cpx<R>::T* __restrict__ Wg)
{
    using V = typename Cpx<R>::T;
    constexpr int NT = FftThreads<M>::NT, LD = PadLen<M>::V + 1, E = M / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* s = reinterpret_cast<V*>(smraw);
    const int Wc = g.W, Kx = g.Kx, Kb = g.Kb, nc = g.nc;
    const int kx0 = blockIdx.x * Wc, z = ENUF_CLAMP((int)blockIdx.y, M);
    const V* sW = stage_twiddles(s + Wc * LD, Wg, M);
    const int t0 = (int)g.fW.div(threadIdx.x), w = threadIdx.x - t0 * Wc, kx = kx0 + w;
    const int t = ENUF_CLAMP(t0, NT);
    V v[1][E];
#pragma unroll
    for (int m = 0; m < E; m++)
        v[0][m] = kx < Kx ? C1[((size_t)z * M + t + NT * m) * Kx + kx] : V{R(0), R(0)};
    cp_async_wait_all();
    __syncthreads();
    fft_reg<V, M, false>(v, s + w * LD, t, sW, 1);
    if (kx >= Kx) return;
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int ky = t + NT * m;
        int kb = -1;
        if (ky <= nc) kb = ky;
        else if (ky >= M - nc) kb = ky - (M - Kb);
        if (kb >= 0 && ENUF_IN(kb, Kb)) C2[((size_t)z * Kb + kb) * Kx + kx] = v[0][m];
    }
}

// ---------------------------------------------------------------- k_fz
// Reciprocal-space tables (per dimension t, index n + n_c):
//   tk[t][.] = k_t = 2 pi n / L_t,  te[t][.] = exp(-k_t^2 / (4 alpha^2)),
//   td[t][.] = D_t(n)^2 = exp(2 b pi^2 n^2 / M^2)  (square of the scaling).
template <typename R> struct KTables {
    const R* tk;  // 3 * Kb
    const R* te;
    const R* td;
    R cE;        // coulomb_k * 2 pi / V   (energy prefactor, Eq. 22)
    R cF;        // coulomb_k * 4 pi / V   (field prefactor, Eq. 41)
    R inv4a2;    // 1 / (4 alpha^2)
};

// grid: ceil(P / W) blocks, W * NT(M) threads (a multiple of 32).
// Writes NF inverse-z-transformed field spectra C3[f][z][kb][kx] and the
// block's energy/virial partials part[blockIdx][0..6] =
// (E, Wxx, Wyy, Wzz, Wxy, Wxz, Wyz).  NF = 0 gives the energy only, NF = 1
// the potential's spectrum alone, NF = 3 the field -i k (ik forces), NF = 4
// the field and the potential.
// Shared memory: max(NF, 1) buffers of W pencils (the first also holds the
// forward transform), the twiddles, the reciprocal tables, the reduction.
template <typename R, int M, int NF>
__global__ void __launch_bounds__(512) k_fz(const typename Cpx<R>::T* __restrict__ C2, typename Cpx<R>::T* __restrict__ C3, FftGeom g,
                     const typename Cpx<R>::T* __restrict__ Wg, KTables<R> ktg, double* __restrict__ part)
{
    using V = typename Cpx<R>::T;
    // radix-4 passes: twice the threads of the radix-8 kernels, for more
    // parallelism in this small kernel
    constexpr int MR = 4, NT = FftThreads<M, MR>::NT, LD = PadLen<M>::V + 1, NB = NF > 0 ? NF : 1, E = M / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* X = reinterpret_cast<V*>(smraw);
    const int Wc = g.W, Kx = g.Kx, Kb = g.Kb, nc = g.nc, P = g.P;
    const int FS = Wc * LD;  // field buffer stride
    double* red = reinterpret_cast<double*>(X + NB * FS);
    V* sW = reinterpret_cast<V*>(red + 32 * 7);
    stage_twiddles(sW, Wg, M);
    R* stab = reinterpret_cast<R*>(sW + M);
    for (int i = threadIdx.x; i < 3 * Kb; i += blockDim.x) {
        stab[i] = ktg.tk[i];
        stab[3 * Kb + i] = ktg.te[i];
        stab[6 * Kb + i] = ktg.td[i];
    }
    const R* tk = stab;
    const R* te = stab + 3 * Kb;
    const R* td = stab + 6 * Kb;
    pdl_wait();
    // thread (w, t) = (tid % W, tid / W) serves pencil p0 + w, elements
    // z = t + NT m (neighbouring threads read neighbouring pencils)
    const int p0 = blockIdx.x * Wc;
    const int t0 = (int)g.fW.div(threadIdx.x), w = threadIdx.x - t0 * Wc, p = p0 + w;
    const int t = ENUF_CLAMP(t0, NT);
    V v[1][E];
#pragma unroll
    for (int m = 0; m < E; m++) v[0][m] = p < P ? C2[(size_t)(t + NT * m) * P + p] : V{R(0), R(0)};
    cp_async_wait_all();
    __syncthreads();
    fft_reg<V, M, false, MR>(v, X + w * LD, t, sW, 1);

    // scaling, energy / virial, subdivided field spectra
    R acc[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    V fv[NB][E];
    int nx = 0, ny = 0;
    bool pv = false;
    if (p < P) {
        const int kb = (int)g.fKx.div(p);
        nx = p - kb * Kx;
        ny = kb <= nc ? kb : kb - Kb;
        pv = ENUF_IN(nx, Kx) && ENUF_IN(ny + nc, Kb);
    }
    const R kxv = pv ? tk[nx + nc] : R(0), kyv = pv ? tk[Kb + ny + nc] : R(0);
    const R exy = pv ? te[nx + nc] * te[Kb + ny + nc] : R(0), dxy = pv ? td[nx + nc] * td[Kb + ny + nc] : R(0);
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int z = t + NT * m;
        const int nz = z <= nc ? z : (z >= M - nc ? z - M : (1 << 20));
        V val = V{R(0), R(0)};
        R kzv = R(0);
        if (pv && nz != (1 << 20) && (nx != 0 || ny != 0 || nz != 0)) {
            kzv = tk[2 * Kb + nz + nc];
            const R k2 = kxv * kxv + kyv * kyv + kzv * kzv;
            const R G = exy * te[2 * Kb + nz + nc] / k2;
            const R D2 = dxy * td[2 * Kb + nz + nc];
            const V gh = v[0][m];
            const R s2 = D2 * (gh.x * gh.x + gh.y * gh.y);  // |S(n)|^2
            const R e = (nx == 0 ? R(1) : R(2)) * ktg.cE * G * s2;
            const R c = R(2) * (R(1) / k2 + ktg.inv4a2);
            acc[0] += e;
            acc[1] += e * (R(1) - c * kxv * kxv);
            acc[2] += e * (R(1) - c * kyv * kyv);
            acc[3] += e * (R(1) - c * kzv * kzv);
            acc[4] -= e * c * kxv * kyv;
            acc[5] -= e * c * kxv * kzv;
            acc[6] -= e * c * kyv * kzv;
            const R f = ktg.cF * G * D2;
            val = V{f * gh.x, f * gh.y};
        }
        if (NF == 1) {
            // the potential alone (forces by analytic differentiation)
            fv[0][m] = val;
        } else if (NF > 0) {
            // -i k_t val for the three field components, val for the potential
            fv[0][m] = V{kxv * val.y, -kxv * val.x};
            if (NF > 1) fv[1 % NB][m] = V{kyv * val.y, -kyv * val.x};
            if (NF > 2) fv[2 % NB][m] = V{kzv * val.y, -kzv * val.x};
            if (NF > 3) fv[3 % NB][m] = val;
        }
    }
    block_reduce_to_double<R, 7>(acc, part + 8 * (size_t)blockIdx.x, red);
    if (NF == 0) return;
    RegPasses<V, M, 1, true, NB, MR>::run(fv, X + w * LD, FS, t, sW, 1);
    if (p < P) {
#pragma unroll
        for (int f = 0; f < NB; f++) {
#pragma unroll
            for (int m = 0; m < E; m++)
                if (ENUF_IN(((size_t)f * M + t + NT * m) * P + p, (size_t)NB * M * P))
                    C3[((size_t)f * M + t + NT * m) * P + p] = fv[f][m];
        }
    }
}

// The z pass for large grids (M = 512, and 128 and 256 in single
// precision): the same steps as k_fz with radix-8 register passes, W
// pencils per CTA of W * M/8 threads (8 at 512: two CTAs an SM; 16 at 128
// and 256: the loads and stores of a z row are 128-byte runs of 16
// neighbouring pencils), and the NF field transforms done one after the
// other through one buffer per pencil (the spectrum S~ and k_z stay in
// registers between them).  At 128 the CTA has 256 threads and the
// launch bounds leave it 80 registers.
template <typename R, int M, int NF>
__global__ void __launch_bounds__(sizeof(R) == 4 ? (M == 128 ? 256 : 1024) : 512) k_fzw(const typename Cpx<R>::T* __restrict__ C2, typename Cpx<R>::T* __restrict__ C3, FftGeom g,
                      const typename Cpx<R>::T* __restrict__ Wg, KTables<R> ktg, double* __restrict__ part)
{
    using V = typename Cpx<R>::T;
    constexpr int MR = 8, NT = FftThreads<M, MR>::NT, LD = PadLen<M>::V + 1, E = M / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* X = reinterpret_cast<V*>(smraw);
    const int Wc = g.W, Kx = g.Kx, Kb = g.Kb, nc = g.nc, P = g.P;
    double* red = reinterpret_cast<double*>(X + Wc * LD);
    V* sW = reinterpret_cast<V*>(red + 32 * 7);
    stage_twiddles(sW, Wg, M);
    R* stab = reinterpret_cast<R*>(sW + M);
    for (int i = threadIdx.x; i < 3 * Kb; i += blockDim.x) {
        stab[i] = ktg.tk[i];
        stab[3 * Kb + i] = ktg.te[i];
        stab[6 * Kb + i] = ktg.td[i];
    }
    const R* tk = stab;
    const R* te = stab + 3 * Kb;
    const R* td = stab + 6 * Kb;
    pdl_wait();
    const int p0 = blockIdx.x * Wc;
    const int t0 = (int)g.fW.div(threadIdx.x), w = threadIdx.x - t0 * Wc, p = p0 + w;
    const int t = ENUF_CLAMP(t0, NT);
    V v[1][E];
#pragma unroll
    for (int m = 0; m < E; m++) v[0][m] = p < P ? C2[(size_t)(t + NT * m) * P + p] : V{R(0), R(0)};
    cp_async_wait_all();
    __syncthreads();
    V* buf = X + w * LD;
    fft_reg<V, M, false, MR>(v, buf, t, sW, 1);

    // scaling, energy / virial; v becomes val = (ke 4 pi / V) G D S~, zero
    // outside the retained cube
    R acc[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    R kz[E];
    int nx = 0, ny = 0;
    bool pv = false;
    if (p < P) {
        const int kb = (int)g.fKx.div(p);
        nx = p - kb * Kx;
        ny = kb <= nc ? kb : kb - Kb;
        pv = ENUF_IN(nx, Kx) && ENUF_IN(ny + nc, Kb);
    }
    const R kxv = pv ? tk[nx + nc] : R(0), kyv = pv ? tk[Kb + ny + nc] : R(0);
    const R exy = pv ? te[nx + nc] * te[Kb + ny + nc] : R(0), dxy = pv ? td[nx + nc] * td[Kb + ny + nc] : R(0);
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int z = t + NT * m;
        const int nz = z <= nc ? z : (z >= M - nc ? z - M : (1 << 20));
        V val = V{R(0), R(0)};
        R kzv = R(0);
        if (pv && nz != (1 << 20) && (nx != 0 || ny != 0 || nz != 0)) {
            kzv = tk[2 * Kb + nz + nc];
            const R k2 = kxv * kxv + kyv * kyv + kzv * kzv;
            const R G = exy * te[2 * Kb + nz + nc] / k2;
            const R D2 = dxy * td[2 * Kb + nz + nc];
            const V gh = v[0][m];
            const R s2 = D2 * (gh.x * gh.x + gh.y * gh.y);  // |S(n)|^2
            const R e = (nx == 0 ? R(1) : R(2)) * ktg.cE * G * s2;
            const R c = R(2) * (R(1) / k2 + ktg.inv4a2);
            acc[0] += e;
            acc[1] += e * (R(1) - c * kxv * kxv);
            acc[2] += e * (R(1) - c * kyv * kyv);
            acc[3] += e * (R(1) - c * kzv * kzv);
            acc[4] -= e * c * kxv * kyv;
            acc[5] -= e * c * kxv * kzv;
            acc[6] -= e * c * kyv * kzv;
            const R f = ktg.cF * G * D2;
            val = V{f * gh.x, f * gh.y};
        }
        v[0][m] = val;
        kz[m] = kzv;
    }
    block_reduce_to_double<R, 7>(acc, part + 8 * (size_t)blockIdx.x, red);
    if (NF == 0) return;
#pragma unroll 1
    for (int f = 0; f < (NF > 0 ? NF : 1); f++) {
        // NF = 1: the potential; else -i k_t val for the three field
        // components and val for the potential (f = 3)
        V fv[1][E];
#pragma unroll
        for (int m = 0; m < E; m++) {
            const V val = v[0][m];
            const R kk = f == 0 ? kxv : (f == 1 ? kyv : kz[m]);
            fv[0][m] = (NF == 1 || f == 3) ? val : V{kk * val.y, -kk * val.x};
        }
        fft_reg<V, M, true, MR>(fv, buf, t, sW, 1);
        if (p < P) {
#pragma unroll
            for (int m = 0; m < E; m++)
                if (ENUF_IN(((size_t)f * M + t + NT * m) * P + p, (size_t)NF * M * P))
                    C3[((size_t)f * M + t + NT * m) * P + p] = fv[0][m];
        }
    }
}

// ---------------------------------------------------------------- k_fz_spectrum
// The forward z pass alone, for the entry points that return the retained
// spectrum instead of forces: the same pencils and transform as k_fz, then
// for every retained n the value ghat(n) (scale = 0) or the approximated
// structure factor S~(n) = D(n) ghat(n) (scale = 1, the scaling step of Sec.
// 3.1), written to out[((n_z + n_c) Kb + (n_y + n_c)) Kx + n_x].
// grid: ceil(P / W) blocks, W * NT(M) threads.
template <typename R, int M>
__global__ void __launch_bounds__(512) k_fz_spectrum(const typename Cpx<R>::T* __restrict__ C2,
                                                     typename Cpx<R>::T* __restrict__ out, FftGeom g,
                                                     const typename Cpx<R>::T* __restrict__ Wg,
                                                     const R* __restrict__ td, int scale)
{
    using V = typename Cpx<R>::T;
    constexpr int MR = 4, NT = FftThreads<M, MR>::NT, LD = PadLen<M>::V + 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* X = reinterpret_cast<V*>(smraw);
    const int Wc = g.W, Kx = g.Kx, Kb = g.Kb, nc = g.nc, P = g.P;
    V* sW = X + Wc * LD;
    stage_twiddles(sW, Wg, M);
    pdl_wait();
    const int p0 = blockIdx.x * Wc;
    for (int i = threadIdx.x; i < Wc * M; i += blockDim.x) {
        const int z = (int)g.fW.div(i), w = i - z * Wc, p = p0 + w;
        cp_async_cpx(X + w * LD + pidx(z), C2 + (p < P ? (size_t)z * P + p : 0), p < P);
    }
    cp_async_wait_all();
    __syncthreads();
    fft_smem<V, M, false, MR>(X + (threadIdx.x / NT) * LD, threadIdx.x % NT, sW, 1);
    for (int i = threadIdx.x; i < Wc * Kb; i += blockDim.x) {
        const int kbz = (int)g.fW.div(i), w = i - kbz * Wc, p = p0 + w;
        if (p >= P) continue;
        const int nz = kbz - nc, z = nz >= 0 ? nz : nz + M;
        const int kb = (int)g.fKx.div(p), kx = p - kb * Kx;
        const int ny = kb <= nc ? kb : kb - Kb;
        V v = X[w * LD + pidx(z)];
        if (scale) {
            const R d = sqrt(td[kx + nc] * td[Kb + ny + nc] * td[2 * Kb + kbz]);
            v = V{d * v.x, d * v.y};
        }
        if (ENUF_IN(((size_t)kbz * Kb + (ny + nc)) * Kx + kx, (size_t)Kb * Kb * Kx))
            out[((size_t)kbz * Kb + (ny + nc)) * Kx + kx] = v;
    }
}

// ---------------------------------------------------------------- k_iy
// grid: (ceil(Kx / W), M, NF) blocks, W * NT(M) threads.  Thread (w, t) =
// (tid % W, tid / W) serves column kx0 + w: it loads its band elements
// y = t + NT m straight from C3 (neighbouring threads read neighbouring
// columns), transforms with register passes and stores its outputs to C4.
template <typename R, int M>
__global__ void __launch_bounds__(SepBounds<R, M>::YT, SepBounds<R, M>::YB) k_iy(const typename Cpx<R>::T* __restrict__ C3, typename Cpx<R>::T* __restrict__ C4, FftGeom g,
                     const typename Cpx<R>::T* __restrict__ Wg)
{
    using V = typename Cpx<R>::T;
    constexpr int NT = FftThreads<M>::NT, LD = PadLen<M>::V + 1, E = M / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* s = reinterpret_cast<V*>(smraw);
    const int Wc = g.W, Kx = g.Kx, Kb = g.Kb, nc = g.nc, P = g.P;
    const int kx0 = blockIdx.x * Wc, z = ENUF_CLAMP((int)blockIdx.y, M), f = blockIdx.z;
    const V* W = stage_twiddles(s + Wc * LD, Wg, M);
    const int t0 = (int)g.fW.div(threadIdx.x), w = threadIdx.x - t0 * Wc, kx = kx0 + w;
    const int t = ENUF_CLAMP(t0, NT);
    const V* src = C3 + ((size_t)f * M + z) * P;
    V v[1][E];
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int y = t + NT * m;
        int kb = -1;
        if (kx < Kx) {
            if (y <= nc) kb = y;
            else if (y >= M - nc) kb = y - (M - Kb);
        }
        v[0][m] = (kb >= 0 && ENUF_IN(kb, Kb)) ? src[(size_t)kb * Kx + kx] : V{R(0), R(0)};
    }
    cp_async_wait_all();
    __syncthreads();
    fft_reg<V, M, true>(v, s + w * LD, t, W, 1);
    if (kx < Kx) {
        V* dst = C4 + ((size_t)f * M + z) * M * Kx + kx;
#pragma unroll
        for (int m = 0; m < E; m++) dst[(size_t)(t + NT * m) * Kx] = v[0][m];
    }
}

// ---------------------------------------------------------------- k_iyx
// Fused inverse y and x (complex-to-real) passes: one CTA per (z-plane,
// field) (grid: (M, NF) blocks, 1024 threads).
// Launch bounds of k_iyx: in single precision with M = 128 the CTA has 264
// threads (33 kept kx columns x 8) and three CTAs share an SM, so that the
// 3 * 128 CTAs of three fields run in one wave on 148 SMs.
template <typename R, int M> struct IyxBounds {
    static constexpr bool small = sizeof(R) == 4 && M == 128;
    static constexpr int T = XyBounds<R, M, true>::T, B = small ? 3 : 1;
};

template <typename R, int M>
__global__ void __launch_bounds__(IyxBounds<R, M>::T, IyxBounds<R, M>::B) k_iyx(const typename Cpx<R>::T* __restrict__ C3, R* __restrict__ fld,
                                              FftGeom g, const typename Cpx<R>::T* __restrict__ Wg)
{
    using V = typename Cpx<R>::T;
    constexpr int MH = M / 2, MRX = XyMR<R, MH, M, true>::V, MRY = XyMR<R, M, M, true>::V;
    constexpr int NTX = FftThreads<MH, MRX>::NT, NTY = FftThreads<M, MRY>::NT, LD = PadLen<M>::V + 1;
    constexpr int RS = PadLen<MH>::V, EX = MH / NTX, EY = M / NTY;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int Kx = g.Kx, Kb = g.Kb, nc = g.nc, P = g.P;
    const int RB = blockDim.x / NTX;
    const int CB = blockDim.x / NTY;
    V* rowbuf = reinterpret_cast<V*>(smraw);
    V* plane = rowbuf + RB * RS;
    const int KxR = ((Kx + CB - 1) / CB) * CB;
    V* sW = plane + KxR * LD;
    stage_twiddles(sW, Wg, M);
    pdl_wait();
    const int z0 = blockIdx.x, z = ENUF_CLAMP(z0, M), f = blockIdx.y;
    const V* src = C3 + ((size_t)f * M + z) * P;
    // inverse y: thread (w, t) = (tid % CB, tid / CB) on column k0 + w loads
    // its band elements y = t + NT m straight from C3 (neighbouring threads
    // read neighbouring kx)
    const int ty0 = threadIdx.x / CB, w = threadIdx.x - ty0 * CB;
    const int ty = ENUF_CLAMP(ty0, NTY);  // ty < NT(M): blockDim = CB NT(M)
    cp_async_wait_all();
    __syncthreads();
    for (int k0 = 0; k0 < Kx; k0 += CB) {
        const int kx = ENUF_CLAMP(k0 + w, KxR);
        V v[1][EY];
#pragma unroll
        for (int m = 0; m < EY; m++) {
            const int y = ty + NTY * m;
            int kb = -1;
            if (kx < Kx) {
                if (y <= nc) kb = y;
                else if (y >= M - nc) kb = y - (M - Kb);
            }
            v[0][m] = (kb >= 0 && ENUF_IN(kb, Kb)) ? src[(size_t)kb * Kx + kx] : V{R(0), R(0)};
        }
        V* col = plane + kx * LD;
        fft_reg<V, M, true, MRY>(v, col, ty, sW, 1);
#pragma unroll
        for (int m = 0; m < EY; m++) col[pidx(ty + NTY * m)] = v[0][m];
    }
    __syncthreads();
    // complex-to-real x per row: thread t of row r forms its inputs from the
    // plane and stores its outputs straight to the field row
    V* out = reinterpret_cast<V*>(fld + ((size_t)f * M + z) * M * M);
    const int r0 = threadIdx.x / NTX, tx = threadIdx.x % NTX, r = ENUF_CLAMP(r0, RB);
    const int RBU = batch_rows(RB, M), yr = batch_row<NTX>(r, RBU);
    for (int y0 = 0; y0 < M; y0 += RBU) {
        const int y = y0 + yr;
        const bool live = r < RBU && y < M;
        const int yy = live ? y : 0;
        V v[1][EX];
#pragma unroll
        for (int m = 0; m < EX; m++) {
            const int k = tx + NTX * m;
            const V a = k <= nc ? plane[k * LD + pidx(yy)] : V{R(0), R(0)};
            const int kb = MH - k;
            const V b = kb <= nc ? cconj(plane[kb * LD + pidx(yy)]) : V{R(0), R(0)};
            const V fe = cadd(a, b);
            const V fo = cmul(csub(a, b), cconj(sW[k]));
            v[0][m] = V{fe.x - fo.y, fe.y + fo.x};
        }
        fft_reg<V, MH, true, MRX>(v, rowbuf + r * RS, tx, sW, 2);
        if (live) {
#pragma unroll
            for (int m = 0; m < EX; m++) out[(size_t)y * MH + tx + NTX * m] = v[0][m];
        }
    }
}

// ---------------------------------------------------------------- k_ix
// grid: ceil(NF*M*M / rows) blocks, rows * NT(M/2) threads.  Complex-to-real
// rows: X_k (k = 0..n_c, zero above) -> x_j = sum_k X_k e^{2 pi i k j/M} over
// the Hermitian-completed spectrum, as a half-length complex transform of
// z_k = (X_k + conj X_{M/2-k}) + i e^{2 pi i k / M} (X_k - conj X_{M/2-k})
// whose outputs are the packed pairs (x_{2j}, x_{2j+1}).  Thread t of a row
// forms its inputs z_{t + NT m} from the row in global memory, transforms
// with register passes and stores its outputs straight to the field row.
template <typename R, int M>
__global__ void __launch_bounds__(256, SepBounds<R, M>::IXB) k_ix(const typename Cpx<R>::T* __restrict__ C4, R* __restrict__ fld, FftGeom g, int nrows,
                     const typename Cpx<R>::T* __restrict__ Wg)
{
    using V = typename Cpx<R>::T;
    constexpr int MH = M / 2, MRX = RowMR<MH>::V, NT = FftThreads<MH, MRX>::NT, RS = PadLen<MH>::V, E = MH / NT;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* s = reinterpret_cast<V*>(smraw);
    const int rows = g.rows, row0 = blockIdx.x * rows, Kx = g.Kx, nc = g.nc;
    const V* W = stage_twiddles(s + rows * RS, Wg, M);
    cp_async_wait_all();
    __syncthreads();
    const int r0 = threadIdx.x / NT, t = threadIdx.x % NT, r = ENUF_CLAMP(r0, rows), row = row0 + r;
    const bool live = row < nrows;
    const V* src = C4 + (size_t)(live ? row : 0) * Kx;
    V v[1][E];
#pragma unroll
    for (int m = 0; m < E; m++) {
        const int k = t + NT * m;
        const V a = (live && k <= nc) ? src[k] : V{R(0), R(0)};
        const int kb = MH - k;
        const V b = (live && kb <= nc) ? cconj(src[kb]) : V{R(0), R(0)};
        const V fe = cadd(a, b);
        const V fo = cmul(csub(a, b), cconj(W[k]));  // (a - b) e^{+2 pi i k / M}
        v[0][m] = V{fe.x - fo.y, fe.y + fo.x};       // fe + i fo
    }
    fft_reg<V, MH, true, MRX>(v, s + r * RS, t, W, 2);
    if (live) {
        V* out = reinterpret_cast<V*>(fld) + (size_t)row * MH;
#pragma unroll
        for (int m = 0; m < E; m++) out[t + NT * m] = v[0][m];
    }
}

}  // namespace enuf
