// sort.cuh -- wrap positions into the box and counting-sort the particles
// into bins (grid tiles for the NFFT, linked cells for the real-space sum).
//
// Positions are normalised x = r / L and wrapped, x - floor(x) (Sec. 2.3.1
// defines x_i = r_i / L).  The bin index and the offset inside the bin are
// computed once here: in double for double plans, and for float plans with a
// float-float product (Dekker's exact product via fma) so that the offset is
// accurate to float rounding even for large boxes.
#pragma once
#include "common.cuh"

namespace enuf {

struct BinGeom {
    int S[3];          // cells per dimension (M for the NFFT grid, n_cell for real space)
    int T;             // cells per bin edge (tile edge; 1 for real space)
    int nb[3];         // bins per dimension = S / T
    double scale[3];   // S_t / L_t
    float scale_hi[3]; // float split of scale: scale ~ hi + lo
    float scale_lo[3];
    double unit[3];    // length of one cell in the offset's unit: 1 (grid units) or L_t/S_t
};

// Cell index c in [0, S) and fraction f in [0, 1) of u = r * scale.
__device__ __forceinline__ void locate(double r, const BinGeom& g, int t, int& c, double& f)
{
    double u = r * g.scale[t];
    double k = floor(u);
    f = u - k;
    if (f >= 1.0) { f = 0.0; k += 1.0; }
    long long kk = (long long)k % g.S[t];
    if (kk < 0) kk += g.S[t];
    c = (int)kk;
}

__device__ __forceinline__ void locate(float r, const BinGeom& g, int t, int& c, float& f)
{
    const float hi = g.scale_hi[t], lo = g.scale_lo[t];
    float p = r * hi;
    float e = fmaf(r, hi, -p);   // exact rounding error of r * hi
    float l = fmaf(r, lo, e);
    float k = floorf(p);
    f = (p - k) + l;             // p - k is exact
    if (f < 0.f) { f += 1.f; k -= 1.f; }
    if (f >= 1.f) { f -= 1.f; k += 1.f; }
    if (f >= 1.f || f < 0.f) f = 0.f;
    int kk = (int)k % g.S[t];
    if (kk < 0) kk += g.S[t];
    c = kk;
}

// Pass 1: bin key, rank inside the bin (atomic counter), unsorted record,
// per-block sums of q^2 and q (for the self and background terms).  The
// counter of bin b is count[b * cs]: with few bins, a stride of one 128-byte
// line per counter spreads the atomics over many L2 lines instead of a few
// hot ones.
template <typename R>
__global__ void __launch_bounds__(256) k_bin_keys(int N, const R* __restrict__ pos, const R* __restrict__ q,
                                                  BinGeom g, uint32_t* __restrict__ key,
                                                  uint32_t* __restrict__ rank,
                                                  typename Rec<R>::T* __restrict__ rec,
                                                  uint32_t* __restrict__ count, int cs, int* __restrict__ status,
                                                  double* __restrict__ qpart)
{
    __shared__ double red[32 * 2];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    R qq = R(0);
    if (i < N) {
        R r3[3] = {pos[3 * (size_t)i], pos[3 * (size_t)i + 1], pos[3 * (size_t)i + 2]};
        qq = q[i];
        bool ok = isfinite(r3[0]) && isfinite(r3[1]) && isfinite(r3[2]) && isfinite(qq);
        int c[3] = {0, 0, 0};
        R off[3] = {R(0), R(0), R(0)};
        if (ok) {
#pragma unroll
            for (int t = 0; t < 3; t++) {
                R f;
                locate(r3[t], g, t, c[t], f);
                off[t] = ((R)(c[t] % g.T) + f) * (R)g.unit[t];
            }
        } else {
            atomicOr(status, ST_NONFINITE);
            qq = R(0);
        }
        uint32_t b = (uint32_t)(c[0] / g.T) +
                     (uint32_t)g.nb[0] * ((uint32_t)(c[1] / g.T) + (uint32_t)g.nb[1] * (uint32_t)(c[2] / g.T));
        key[i] = b;
        rank[i] = atomicAdd(&count[(size_t)b * cs], 1u);
        typename Rec<R>::T rr;
        rr.x = off[0]; rr.y = off[1]; rr.z = off[2]; rr.w = qq;
        rec[i] = rr;
    }
    if (qpart) {
        R v[2] = {qq * qq, qq};
        block_reduce_to_double<R, 2>(v, qpart + 2 * (size_t)blockIdx.x, red);
    }
}

// Pass 2 (one block of 1024 threads): exclusive scan of the bin counts into
// offsets, and a work list of (bin, begin, end) items of at most `cap`
// particles each for the kernels that process bins (heavy bins are split).
// Each thread sums a contiguous chunk of bins; the per-thread totals are
// scanned with warp shuffles and one pass over the 32 warp totals.  The
// counts are cleared after use, ready for the next evaluation.
__global__ void __launch_bounds__(1024) k_scan_bins(int nbins, uint32_t* __restrict__ count, int cs,
                                                    uint32_t* __restrict__ offset, int cap,
                                                    int4* __restrict__ work, int* __restrict__ nwork, int max_work,
                                                    int* __restrict__ status)
{
    __shared__ uint32_t s_cnt[32], s_wrk[32];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarp = nt >> 5;
    const int chunk = (nbins + nt - 1) / nt;
    const int b0 = min(nbins, tid * chunk), b1 = min(nbins, b0 + chunk);
    uint32_t c = 0, w = 0;
    for (int b = b0; b < b1; b++) {
        uint32_t n = count[(size_t)b * cs];
        c += n;
        if (work) w += (n + cap - 1) / cap;
    }
    // inclusive scans inside each warp, then over the warp totals
    uint32_t ic = c, iw = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t a = __shfl_up_sync(0xffffffffu, ic, o), bw = __shfl_up_sync(0xffffffffu, iw, o);
        if (lane >= o) { ic += a; iw += bw; }
    }
    if (lane == 31) { s_cnt[warp] = ic; s_wrk[warp] = iw; }
    __syncthreads();
    if (warp == 0) {
        uint32_t x = lane < nwarp ? s_cnt[lane] : 0u, y = lane < nwarp ? s_wrk[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t a = __shfl_up_sync(0xffffffffu, x, o), bw = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) { x += a; y += bw; }
        }
        s_cnt[lane] = x;
        s_wrk[lane] = y;
    }
    __syncthreads();
    uint32_t base = (warp ? s_cnt[warp - 1] : 0u) + ic - c, wbase = (warp ? s_wrk[warp - 1] : 0u) + iw - w;
    for (int b = b0; b < b1; b++) {
        uint32_t n = count[(size_t)b * cs];
        count[(size_t)b * cs] = 0u;
        offset[b] = base;
        if (work) {
            for (uint32_t s = 0; s < n; s += cap) {
                if ((int)wbase < max_work) work[wbase] = make_int4(b, (int)(base + s), (int)(base + min(n, s + cap)), 0);
                wbase++;
            }
        }
        base += n;
    }
    if (tid == nt - 1) {
        offset[nbins] = s_cnt[nwarp - 1];
        if (work) {
            int nw = (int)s_wrk[nwarp - 1];
            if (nw > max_work) { atomicOr(status, ST_WORKLIST); nw = max_work; }
            *nwork = nw;
        }
    }
}

// Pass 3: scatter the records into bin order; perm[sorted] = original index.
template <typename R>
__global__ void __launch_bounds__(256) k_scatter(int N, const uint32_t* __restrict__ key,
                                                 const uint32_t* __restrict__ rank,
                                                 const uint32_t* __restrict__ offset,
                                                 const typename Rec<R>::T* __restrict__ rec_in,
                                                 typename Rec<R>::T* __restrict__ rec_out, uint32_t* __restrict__ perm,
                                                 uint32_t* __restrict__ bin_of_sorted)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t b = key[i];
    const uint32_t d = offset[b] + rank[i];
    rec_out[d] = rec_in[i];
    perm[d] = (uint32_t)i;
    if (bin_of_sorted) bin_of_sorted[d] = b;
}

}  // namespace enuf
