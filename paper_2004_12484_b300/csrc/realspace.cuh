// realspace.cuh -- real-space part of the Ewald sum (Sec. 2.1) and the
// final FP64 assembly.
//
// Pair energy  q_i q_j erfc(alpha r) / r                        (Eq. 17)
// (times B_U, and the force times B_F, for the smeared charges of ENUF-DPD,
// Eq. 51-58)
// Pair force   q_i q_j [erfc(alpha r)/r + 2 alpha/sqrt(pi) e^{-alpha^2 r^2}]
//              r_ij / r^2                  (Eq. 29, textbook form)
// Potential    phi_i += q_j erfc(alpha r) / r
// within r < r_c.  Particles are counting-sorted into linked cells of edge
// >= r_c / 2 (at least 5 per dimension; else edge >= r_c, at least 3); one
// thread serves one particle and visits the 125 (27) neighbouring cells
// (Sec. 3.2: linked-cell list).  Each ordered
// pair is visited from both ends, so no atomics are needed; the energy and
// virial take half of each visit.  Boxes too small for 3 cells per dimension
// use the all-pairs kernel with the minimum image (r_c <= L/2 is required).
#pragma once
#include "common.cuh"

namespace enuf {

template <typename R> struct RealParams {
    int nc[3];   // cells per dimension
    R h[3];      // cell edges
    R L[3];      // box (all-pairs kernel)
    R rc2, alpha, two_a_sqpi, ke;
    R self_phi;  // -2 alpha / sqrt(pi) (self term of dE/dq_i, times ke inside)
    R inv_lam;   // 1 / lambda_e of Slater-type smeared charges (kernels with SL)
};

// ENUF-DPD factors of Slater-type charges (Eq. 57-58) at x = r / lambda_e:
// B_U = 1 - (1 + x) e^{-2x}, B_F = 1 - (1 + 2x (1 + x)) e^{-2x}, written with
// em = 1 - e^{-2x} from expm1 so that B_U keeps its relative accuracy for
// close pairs (its leading term is x); e^{-2x} = 1 - em then costs no second
// exponential (for large x its relative error grows, but it only enters
// multiplied by terms that B_U and B_F approach 1 against).
template <typename R> __device__ __forceinline__ void slater_factors(R x, R& bu, R& bf)
{
    R em;
    if constexpr (sizeof(R) == 4) em = -expm1f(-2.0f * x);
    else em = -expm1(-2.0 * x);
    const R e = R(1) - em;
    bu = em - x * e;
    bf = em - R(2) * x * (R(1) + x) * e;
}

// SL: smeared Slater-type charges (ENUF-DPD): the erfc pair energy scaled by
// B_U and the pair force by B_F; coincident charges add the finite energy of
// Eq. 59 (erfc(0) B_U / r -> 1 / lambda_e) and no force (Eq. 60).
template <typename R, bool SL = false>
__device__ __forceinline__ void pair_term(R dx, R dy, R dz, R qi, R qj, const RealParams<R>& rp, R (&f)[3], R& ph,
                                          R (&acc)[7])
{
    const R r2 = dx * dx + dy * dy + dz * dz;
    if (r2 >= rp.rc2) return;
    if (r2 <= R(0)) {
        if constexpr (SL) {
            ph += qj * rp.inv_lam;
            acc[0] += R(0.5) * qi * qj * rp.inv_lam;
        }
        return;
    }
    R ec, fs;
    R r;
    if constexpr (sizeof(R) == 4) {
        // single precision: one reciprocal square root instead of a square
        // root and two divisions (rsqrtf is within 2 ulp)
        const float rinv = rsqrtf(r2);
        r = r2 * rinv;
        const float ar = rp.alpha * r;
        ec = erfcf(ar) * rinv;
        fs = qi * qj * (ec + rp.two_a_sqpi * expf(-ar * ar)) * (rinv * rinv);
    } else {
        r = dsqrt(r2);
        const R ar = rp.alpha * r;
        ec = derfc(ar) / r;
        fs = qi * qj * (ec + rp.two_a_sqpi * dexp(-ar * ar)) / r2;
    }
    if constexpr (SL) {
        R bu, bf;
        slater_factors<R>(r * rp.inv_lam, bu, bf);
        ec *= bu;
        fs *= bf;
    }
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

// Adds the real-space force and potential (and the self term of phi) to F
// and phi in the caller's particle order (zeroed buffers; global atomics);
// part[block] gets (E, W..) partials.  SR: stencil radius in cells ((2 SR +
// 1)^3 cells of edge >= r_c / SR).  Block row blockIdx.y = dz + SR takes one
// z-layer of the stencil, so a particle is served by 2 SR + 1 threads and
// small systems still fill the GPU.
template <typename R, int SR, bool SL = false>
__global__ void __launch_bounds__(256) k_realspace_cells(int N, const typename Rec<R>::T* __restrict__ rec,
                                                         const uint32_t* __restrict__ cell_of,
                                                         const uint32_t* __restrict__ offset,
                                                         const uint32_t* __restrict__ perm, RealParams<R> rp,
                                                         R* __restrict__ F, R* __restrict__ phi,
                                                         double* __restrict__ part)
{
    __shared__ double red[32 * 7];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    R acc[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    if (i < N) {
        const typename Rec<R>::T ri = rec[i];
        const uint32_t c0 = cell_of[i];
        const uint32_t c = ENUF_CLAMP(c0, (uint32_t)(rp.nc[0] * rp.nc[1] * rp.nc[2]));
        const int cx = c % rp.nc[0], cy = (c / rp.nc[0]) % rp.nc[1], cz = c / (rp.nc[0] * rp.nc[1]);
        R f[3] = {R(0), R(0), R(0)}, ph = R(0);
        {
            const int dz = (int)blockIdx.y - SR;
            const int nz = (cz + dz + rp.nc[2]) % rp.nc[2];
            for (int dy = -SR; dy <= SR; dy++) {
                const int ny = (cy + dy + rp.nc[1]) % rp.nc[1];
                for (int dx = -SR; dx <= SR; dx++) {
                    const int nx = (cx + dx + rp.nc[0]) % rp.nc[0];
                    const uint32_t nb = nx + rp.nc[0] * (ny + rp.nc[1] * nz);
                    const R sx = ri.x - (R)dx * rp.h[0], sy = ri.y - (R)dy * rp.h[1], sz = ri.z - (R)dz * rp.h[2];
                    const uint32_t e0 = offset[nb + 1];
                    const uint32_t e = ENUF_IN(e0, N + 1) ? e0 : 0u;
                    for (uint32_t j = offset[nb]; j < e; j++) {
                        if ((int)j == i) continue;
                        const typename Rec<R>::T rj = rec[j];
                        pair_term<R, SL>(sx - rj.x, sy - rj.y, sz - rj.z, ri.w, rj.w, rp, f, ph, acc);
                    }
                }
            }
        }
        const uint32_t oi = perm[i];
        if (!ENUF_IN(oi, N)) {
            F = nullptr;
            phi = nullptr;
        }
        if (F) {
            atomicAdd(F + 3 * (size_t)oi, rp.ke * f[0]);
            atomicAdd(F + 3 * (size_t)oi + 1, rp.ke * f[1]);
            atomicAdd(F + 3 * (size_t)oi + 2, rp.ke * f[2]);
        }
        if (phi) atomicAdd(phi + oi, rp.ke * (ph + (blockIdx.y == 0 ? rp.self_phi * ri.w : R(0))));
    }
    block_reduce_to_double<R, 7>(acc, part + 8 * ((size_t)blockIdx.y * gridDim.x + blockIdx.x), red);
}

// All pairs with the minimum image; records hold wrapped absolute positions.
template <typename R, bool SL = false>
__global__ void __launch_bounds__(256) k_realspace_allpairs(int N, const typename Rec<R>::T* __restrict__ rec,
                                                            const uint32_t* __restrict__ perm, RealParams<R> rp,
                                                            R* __restrict__ F, R* __restrict__ phi,
                                                            double* __restrict__ part)
{
    __shared__ double red[32 * 7];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    R acc[7] = {R(0), R(0), R(0), R(0), R(0), R(0), R(0)};
    if (i < N) {
        const typename Rec<R>::T ri = rec[i];
        R f[3] = {R(0), R(0), R(0)}, ph = R(0);
        for (int j = 0; j < N; j++) {
            if (j == i) continue;
            const typename Rec<R>::T rj = rec[j];
            R d[3] = {ri.x - rj.x, ri.y - rj.y, ri.z - rj.z};
#pragma unroll
            for (int t = 0; t < 3; t++) {
                if (d[t] > R(0.5) * rp.L[t]) d[t] -= rp.L[t];
                else if (d[t] < R(-0.5) * rp.L[t]) d[t] += rp.L[t];
            }
            pair_term<R, SL>(d[0], d[1], d[2], ri.w, rj.w, rp, f, ph, acc);
        }
        const uint32_t oi = perm[i];
        if (!ENUF_IN(oi, N)) {
            F = nullptr;
            phi = nullptr;
        }
        if (F) {
            F[3 * (size_t)oi] = rp.ke * f[0];
            F[3 * (size_t)oi + 1] = rp.ke * f[1];
            F[3 * (size_t)oi + 2] = rp.ke * f[2];
        }
        if (phi) phi[oi] = rp.ke * (ph + rp.self_phi * ri.w);
    }
    block_reduce_to_double<R, 7>(acc, part + 8 * (size_t)blockIdx.x, red);
}

// Adds the real-space force and potential (computed beside the reciprocal
// part into their own buffers) to the reciprocal ones, and clears those
// buffers for the next evaluation.
template <typename R>
__global__ void __launch_bounds__(256) k_combine(int N, R* __restrict__ Fr, R* __restrict__ phir,
                                                 R* __restrict__ F, R* __restrict__ phi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (F) {
#pragma unroll
        for (int t = 0; t < 3; t++) {
            F[3 * (size_t)i + t] += Fr[3 * (size_t)i + t];
            Fr[3 * (size_t)i + t] = R(0);
        }
    }
    if (phi) {
        phi[i] += phir[i];
        phir[i] = R(0);
    }
}

// ---------------------------------------------------------------- assembly
struct FinalParams {
    int nq, nk, nr;      // partial counts (nr = 0: no real-space part)
    double ke, alpha, V, sqrt_pi;
    int kspace_only;
};

// Blocks of 512 threads (16 warps): in block b, warp w sums quantity w over
// block b's fixed chunk of the per-block partials (lane-strided, then a
// fixed shuffle tree); the last block to finish (no block waits for another)
// adds the blocks' sums in block order, so the result is deterministic, adds
// the self energy (Eq. 24) and the background term and writes the ENUF_NOUT
// results.  scratch: 16 doubles per block; done: kept zero between calls.
__global__ void __launch_bounds__(512) k_finalize(const double* __restrict__ qpart, const double* __restrict__ kpart,
                                                  const double* __restrict__ rpart, FinalParams fp,
                                                  int* __restrict__ status, double* __restrict__ out,
                                                  double* __restrict__ scratch, unsigned* __restrict__ done)
{
    __shared__ double s[16];
    __shared__ bool s_last;
    pdl_wait();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nb = gridDim.x, b = blockIdx.x;
    auto chunk = [&](int n, int& lo, int& hi) {
        const int c = (n + nb - 1) / nb;
        lo = min(n, b * c);
        hi = min(n, lo + c);
    };
    double a = 0.0;
    int lo, hi;
    if (w < 2) {
        chunk(fp.nq, lo, hi);
        for (int k = lo + lane; k < hi; k += 32) a += qpart[2 * k + w];
    } else if (w < 9) {
        chunk(fp.nk, lo, hi);
        for (int k = lo + lane; k < hi; k += 32) a += kpart[8 * k + (w - 2)];
    } else {
        chunk(fp.nr, lo, hi);
        for (int k = lo + lane; k < hi; k += 32) a += rpart[8 * k + (w - 9)];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (nb > 1) {
        if (lane == 0) scratch[16 * b + w] = a;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = atomicAdd(done, 1u) == (unsigned)nb - 1;
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        if (threadIdx.x < 16) {
            double t = 0.0;
            for (int k = 0; k < nb; k++) t += __ldcg(scratch + 16 * k + threadIdx.x);
            s[threadIdx.x] = t;
        }
    } else if (lane == 0) {
        s[w] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (nb > 1) *done = 0u;  // ready for the next evaluation
        const double q2 = s[0], Q = s[1];
        const double Ek = s[2];
        const double Er = fp.nr ? fp.ke * s[9] : 0.0;
        double Es = 0.0, Eb = 0.0;
        if (!fp.kspace_only) {
            Es = -fp.ke * fp.alpha / fp.sqrt_pi * q2;
            Eb = -fp.ke * 3.14159265358979323846 * Q * Q / (2.0 * fp.V * fp.alpha * fp.alpha);
        }
        // virial components (xx, yy, zz, xy, xz, yz) -> row-major 3x3
        double w6[6];
        for (int k = 0; k < 6; k++) w6[k] = s[3 + k] + (fp.nr ? fp.ke * s[10 + k] : 0.0);
        out[0] = fp.kspace_only ? Ek : (Er + Ek + Es + Eb);
        out[1] = Er;
        out[2] = Ek;
        out[3] = Es;
        out[4] = Eb;
        out[5] = Q;
        out[6] = w6[0] + Eb; out[7] = w6[3]; out[8] = w6[4];
        out[9] = w6[3]; out[10] = w6[1] + Eb; out[11] = w6[5];
        out[12] = w6[4]; out[13] = w6[5]; out[14] = w6[2] + Eb;
        out[15] = (double)(*status);
        *status = 0;  // cleared for the next evaluation
    }
}

// d(E_background)/dq_i = -ke pi Q / (V alpha^2), the same for every particle.
template <typename R>
__global__ void k_phi_background(int N, const double* __restrict__ out, double scale, R* __restrict__ phi)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) phi[i] += (R)(scale * out[5]);
}

// Net force removal: per-block sums, one-block mean, shift.
template <typename R>
__global__ void __launch_bounds__(256) k_force_sum(int N, const R* __restrict__ F, double* __restrict__ part)
{
    __shared__ double red[32 * 3];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    R v[3] = {R(0), R(0), R(0)};
    if (i < N) { v[0] = F[3 * (size_t)i]; v[1] = F[3 * (size_t)i + 1]; v[2] = F[3 * (size_t)i + 2]; }
    block_reduce_to_double<R, 3>(v, part + 4 * (size_t)blockIdx.x, red);
}

__global__ void __launch_bounds__(256) k_force_mean(int nb, int N, const double* __restrict__ part,
                                                    double* __restrict__ mean)
{
    __shared__ double s[256][3];
    double a[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x)
        for (int k = 0; k < 3; k++) a[k] += part[4 * b + k];
    for (int k = 0; k < 3; k++) s[threadIdx.x][k] = a[k];
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int k = 0; k < 3; k++) s[threadIdx.x][k] += s[threadIdx.x + o][k];
        __syncthreads();
    }
    if (threadIdx.x < 3) mean[threadIdx.x] = s[0][threadIdx.x] / (double)N;
}

template <typename R>
__global__ void k_force_shift(int N, const double* __restrict__ mean, R* __restrict__ F)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        F[3 * (size_t)i] -= (R)mean[0];
        F[3 * (size_t)i + 1] -= (R)mean[1];
        F[3 * (size_t)i + 2] -= (R)mean[2];
    }
}

// Backward: dpos = -gE F, dq = gE phi.
template <typename R>
__global__ void k_backward_scale(int N, const R* __restrict__ F, const R* __restrict__ phi,
                                 const double* __restrict__ gE, R* __restrict__ dpos, R* __restrict__ dq)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const R g = gE ? (R)(*gE) : R(1);
    if (dpos) {
        dpos[3 * (size_t)i] = -g * F[3 * (size_t)i];
        dpos[3 * (size_t)i + 1] = -g * F[3 * (size_t)i + 1];
        dpos[3 * (size_t)i + 2] = -g * F[3 * (size_t)i + 2];
    }
    if (dq) dq[i] = g * phi[i];
}

}  // namespace enuf
