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
    int T;             // cells per tile edge (1 for real space)
    int nb[3];         // tiles per dimension = S / T
    int sub, lr;       // sub-tile edge and log2(T / sub): a bin is one of the
                       // (T / sub)^3 sub-tiles of a tile, numbered tile-major
    int lT, lsub;      // log2(T), log2(sub) (both powers of two)
    int smask[3];      // S - 1 when S is a power of two, else -1
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
    long long kk;
    if (g.smask[t] >= 0) kk = (long long)k & g.smask[t];
    else {
        kk = (long long)k % g.S[t];
        if (kk < 0) kk += g.S[t];
    }
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
    int kk;
    if (g.smask[t] >= 0) kk = (int)k & g.smask[t];
    else {
        kk = (int)k % g.S[t];
        if (kk < 0) kk += g.S[t];
    }
    c = kk;
}

// The scan, run by the last block of k_bin_keys to finish (the bins are
// complete once every other block has counted its particles): exclusive
// scan of the bin counts into offsets, the work list `work` of (group,
// begin, end) items over groups of GROUP consecutive bins (the tiles) with
// at most `cap` particles per item (heavy groups are split, empty ones get
// no item), and, for the per-bin work list that the scatter pass writes,
// the index item2[b] of bin b's first item when bins are cut into items of
// at most `cap2` particles.  The bins go through shared memory in segments
// of NT * 8: one coalesced read of the counts (which are cleared, ready for
// the next evaluation), 8 bins per thread, a shuffle scan of the per-thread
// totals, and coalesced writes of the offsets and item indices.
struct ScanArgs {
    int nbins;
    uint32_t* count;
    int cs;             // word stride of the counters
    uint32_t* offset;   // nbins + 1
    int cap;
    int4* work;         // NULL: no group work list
    int* nwork;
    int max_work;
    int cap2;
    uint32_t* item2;    // NULL: no per-bin item indices
    int* nwork2;
    int max_work2;
    unsigned* done;     // blocks finished (kept zero between evaluations)
};

constexpr int kScanPer = 8;  // bins per thread and segment

// Scans bins [lo, hi) starting from the running totals base0 (particles,
// items of `work`, items of the per-bin list; NULL: zero); `final`: this
// block ends the scan and writes the totals.
template <int GROUP, int NT>
__device__ __forceinline__ void scan_bins_block(const ScanArgs& a, int* status, uint32_t* s_a, uint32_t* s_b,
                                                uint32_t (*s_sum)[32], int lo, int hi, const uint32_t* base0,
                                                bool final)
{
    constexpr int PER = kScanPer, SEG = NT * PER, NWARP = NT / 32;
    static_assert(PER % GROUP == 0, "a thread's bins hold whole groups");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    uint32_t base[3] = {0u, 0u, 0u};  // particles, items of work, items of the per-bin list
    if (base0) {
#pragma unroll
        for (int e = 0; e < 3; e++) base[e] = base0[e];
    }
    // the thread's counts of a segment, all loads in flight at once; the next
    // segment's are loaded while this one is scanned
    uint32_t t[PER];
    auto load_segment = [&](int s0) {
        const int ns = min(SEG, hi - s0);
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = tid + k * NT;
            t[k] = i < ns ? __ldcg(a.count + (size_t)(s0 + i) * a.cs) : 0u;
        }
    };
    if (lo < hi) load_segment(lo);
    for (int s0 = lo; s0 < hi; s0 += SEG) {
        const int ns = min(SEG, hi - s0);
#pragma unroll
        for (int k = 0; k < PER; k++) {
            const int i = tid + k * NT;
            if (i < ns) {
                s_a[i] = t[k];
                a.count[(size_t)(s0 + i) * a.cs] = 0u;
            }
        }
        if (s0 + SEG < hi) load_segment(s0 + SEG);
        __syncthreads();
        const int b0 = tid * PER;
        uint32_t n[PER];
        uint32_t v[3] = {0u, 0u, 0u};
#pragma unroll
        for (int k = 0; k < PER; k++) {
            n[k] = b0 + k < ns ? s_a[b0 + k] : 0u;
            v[0] += n[k];
            if (a.item2) v[2] += (n[k] + a.cap2 - 1) / a.cap2;
        }
        if (a.work) {
#pragma unroll
            for (int gg = 0; gg < PER / GROUP; gg++) {
                uint32_t ng = 0;
#pragma unroll
                for (int k = 0; k < GROUP; k++) ng += n[gg * GROUP + k];
                v[1] += (ng + a.cap - 1) / a.cap;
            }
        }
        // inclusive scans inside each warp, then over the warp totals
        uint32_t inc[3] = {v[0], v[1], v[2]};
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int e = 0; e < 3; e++) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, inc[e], o);
                if (lane >= o) inc[e] += t;
            }
        }
        if (lane == 31) {
#pragma unroll
            for (int e = 0; e < 3; e++) s_sum[e][warp] = inc[e];
        }
        __syncthreads();
        if (warp == 0) {
            uint32_t x[3];
#pragma unroll
            for (int e = 0; e < 3; e++) x[e] = lane < NWARP ? s_sum[e][lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
                for (int e = 0; e < 3; e++) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, x[e], o);
                    if (lane >= o) x[e] += t;
                }
            }
#pragma unroll
            for (int e = 0; e < 3; e++) s_sum[e][lane] = x[e];
        }
        __syncthreads();
        uint32_t ex[3];
#pragma unroll
        for (int e = 0; e < 3; e++) ex[e] = base[e] + (warp ? s_sum[e][warp - 1] : 0u) + inc[e] - v[e];
        uint32_t o = ex[0], it2 = ex[2], wb = ex[1];
#pragma unroll
        for (int gg = 0; gg < PER / GROUP; gg++) {
            const uint32_t gstart = o;
#pragma unroll
            for (int k = gg * GROUP; k < (gg + 1) * GROUP; k++) {
                if (b0 + k < ns) {
                    s_a[b0 + k] = o;
                    s_b[b0 + k] = it2;
                }
                o += n[k];
                if (a.item2) it2 += (n[k] + a.cap2 - 1) / a.cap2;
            }
            if (a.work) {
                const uint32_t ng = o - gstart;
                const int gidx = (s0 + b0) / GROUP + gg;
                for (uint32_t s = 0; s < ng; s += a.cap) {
                    if ((int)wb < a.max_work)
                        a.work[wb] = make_int4(gidx, (int)(gstart + s), (int)(gstart + min(ng, s + a.cap)), 0);
                    wb++;
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < ns; i += NT) {
            if (!ENUF_IN(s0 + i, a.nbins)) continue;
            a.offset[s0 + i] = s_a[i];
            if (a.item2) a.item2[s0 + i] = s_b[i];
        }
#pragma unroll
        for (int e = 0; e < 3; e++) base[e] += s_sum[e][NWARP - 1];
        __syncthreads();
    }
    if (final && tid == 0) {
        a.offset[a.nbins] = base[0];
        if (a.work) {
            int nw = (int)base[1];
            if (nw > a.max_work) { atomicOr(status, ST_WORKLIST); nw = a.max_work; }
            *a.nwork = nw;
        }
        if (a.item2) {
            int nw = (int)base[2];
            if (nw > a.max_work2) { atomicOr(status, ST_WORKLIST); nw = a.max_work2; }
            *a.nwork2 = nw;
        }
    }
}

// Pass 1: bin key, rank inside the bin (atomic counter), unsorted record,
// per-block sums of q^2 and q (for the self and background terms); the
// last block to finish then runs pass 2 (scan_bins_block).  The
// counter of bin b is count[b * cs]: with few bins, a stride of one 128-byte
// line per counter spreads the atomics over many L2 lines instead of a few
// hot ones.
template <typename R, int GROUP>
__global__ void __launch_bounds__(256) k_bin_keys(int N, const R* __restrict__ pos, const R* __restrict__ q,
                                                  BinGeom g, uint32_t* __restrict__ key,
                                                  uint32_t* __restrict__ rank,
                                                  typename Rec<R>::T* __restrict__ rec, ScanArgs sa,
                                                  int* __restrict__ status, double* __restrict__ qpart)
{
    __shared__ double red[32 * 2];
    __shared__ uint32_t s_scan[2 * 256 * kScanPer];
    __shared__ uint32_t s_sum[3][32];
    __shared__ bool s_last;
    pdl_wait();
    uint32_t* __restrict__ count = sa.count;
    const int cs = sa.cs;
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
                off[t] = ((R)(c[t] & (g.T - 1)) + f) * (R)g.unit[t];
            }
        } else {
            atomicOr(status, ST_NONFINITE);
            qq = R(0);
        }
        uint32_t b = (uint32_t)(c[0] >> g.lT) +
                     (uint32_t)g.nb[0] * ((uint32_t)(c[1] >> g.lT) + (uint32_t)g.nb[1] * (uint32_t)(c[2] >> g.lT));
        if (g.lr > 0) {
            // sub-tile of the cell index the kernels split from the stored
            // offset (same truncation and clamp as split_offset)
            uint32_t sb = 0;
#pragma unroll
            for (int t = 0; t < 3; t++) {
                int ci = (int)off[t];
                if (ci > g.T - 1) ci = g.T - 1;
                sb |= (uint32_t)(ci >> g.lsub) << (g.lr * t);
            }
            b = (b << (3 * g.lr)) | sb;
        }
        key[i] = b;
        rank[i] = ENUF_IN(b, sa.nbins) ? atomicAdd(&count[(size_t)b * cs], 1u) : 0u;
        typename Rec<R>::T rr;
        rr.x = off[0]; rr.y = off[1]; rr.z = off[2]; rr.w = qq;
        rec[i] = rr;
    }
    if (qpart) {
        R v[2] = {qq * qq, qq};
        block_reduce_to_double<R, 2>(v, qpart + 2 * (size_t)blockIdx.x, red);
    }
    // the last block to finish scans the bins (no block waits for another);
    // large bin counts are scanned by the k_scan_* passes instead
    if (!sa.done) return;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(sa.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    scan_bins_block<GROUP, 256>(sa, status, s_scan, s_scan + 256 * kScanPer, s_sum, 0, sa.nbins, nullptr, true);
    if (threadIdx.x == 0) *sa.done = 0u;  // ready for the next evaluation
}

// Pass 2 for large bin counts, in three launches over chunks of
// kScanChunk bins: (a) per-chunk totals, (b) one block scans the totals
// into chunk bases and writes the overall totals, (c) every chunk is scanned
// from its base (offsets, item indices, work items; counts cleared).
constexpr int kScanChunk = 256 * kScanPer;

template <int GROUP>
__global__ void __launch_bounds__(256) k_scan_sums(ScanArgs a, uint32_t* __restrict__ csum)
{
    constexpr int PER = kScanPer;
    __shared__ uint32_t s_red[3][8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lo = blockIdx.x * kScanChunk, hi = min(a.nbins, lo + kScanChunk);
    const int b0 = lo + tid * PER;
    uint32_t n[PER];
    uint32_t v[3] = {0u, 0u, 0u};
#pragma unroll
    for (int k = 0; k < PER; k++) {
        n[k] = b0 + k < hi ? __ldcg(a.count + (size_t)(b0 + k) * a.cs) : 0u;
        v[0] += n[k];
        if (a.item2) v[2] += (n[k] + a.cap2 - 1) / a.cap2;
    }
    if (a.work) {
#pragma unroll
        for (int gg = 0; gg < PER / GROUP; gg++) {
            uint32_t ng = 0;
#pragma unroll
            for (int k = 0; k < GROUP; k++) ng += n[gg * GROUP + k];
            v[1] += (ng + a.cap - 1) / a.cap;
        }
    }
#pragma unroll
    for (int e = 0; e < 3; e++) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[e] += __shfl_xor_sync(0xffffffffu, v[e], o);
        if (lane == 0) s_red[e][warp] = v[e];
    }
    __syncthreads();
    if (tid < 3) {
        uint32_t t = 0;
        for (int w = 0; w < 8; w++) t += s_red[tid][w];
        csum[3 * blockIdx.x + tid] = t;
    }
}

__global__ void __launch_bounds__(1024) k_scan_bases(ScanArgs a, int nchunks, const uint32_t* __restrict__ csum,
                                                     uint32_t* __restrict__ cbase, int* __restrict__ status)
{
    __shared__ uint32_t s_sum[3][32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int per = (nchunks + 1023) / 1024;
    const int c0 = min(nchunks, tid * per), c1 = min(nchunks, c0 + per);
    uint32_t v[3] = {0u, 0u, 0u};
    for (int c = c0; c < c1; c++) {
#pragma unroll
        for (int e = 0; e < 3; e++) v[e] += csum[3 * c + e];
    }
    uint32_t inc[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int e = 0; e < 3; e++) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, inc[e], o);
            if (lane >= o) inc[e] += t;
        }
    }
    if (lane == 31) {
#pragma unroll
        for (int e = 0; e < 3; e++) s_sum[e][warp] = inc[e];
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t x[3];
#pragma unroll
        for (int e = 0; e < 3; e++) x[e] = s_sum[e][lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int e = 0; e < 3; e++) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, x[e], o);
                if (lane >= o) x[e] += t;
            }
        }
#pragma unroll
        for (int e = 0; e < 3; e++) s_sum[e][lane] = x[e];
    }
    __syncthreads();
    uint32_t run[3];
#pragma unroll
    for (int e = 0; e < 3; e++) run[e] = (warp ? s_sum[e][warp - 1] : 0u) + inc[e] - v[e];
    for (int c = c0; c < c1; c++) {
#pragma unroll
        for (int e = 0; e < 3; e++) {
            cbase[3 * c + e] = run[e];
            run[e] += csum[3 * c + e];
        }
    }
    if (tid == 1023) {
        a.offset[a.nbins] = s_sum[0][31];
        if (a.work) {
            int nw = (int)s_sum[1][31];
            if (nw > a.max_work) { atomicOr(status, ST_WORKLIST); nw = a.max_work; }
            *a.nwork = nw;
        }
        if (a.item2) {
            int nw = (int)s_sum[2][31];
            if (nw > a.max_work2) { atomicOr(status, ST_WORKLIST); nw = a.max_work2; }
            *a.nwork2 = nw;
        }
    }
}

template <int GROUP>
__global__ void __launch_bounds__(256) k_scan_apply(ScanArgs a, const uint32_t* __restrict__ cbase,
                                                    int* __restrict__ status)
{
    __shared__ uint32_t s_scan[2 * 256 * kScanPer];
    __shared__ uint32_t s_sum[3][32];
    const int lo = blockIdx.x * kScanChunk, hi = min(a.nbins, lo + kScanChunk);
    scan_bins_block<GROUP, 256>(a, status, s_scan, s_scan + 256 * kScanPer, s_sum, lo, hi, cbase + 3 * blockIdx.x,
                                false);
}

// Pass 3: scatter the records into bin order; perm[sorted] = original index.
// With `work2`, the particle of rank r in bin b with r % cap2 == 0 also
// writes the per-bin work item (b, begin, end) of the cap2 particles from
// it, at index item2[b] + r / cap2.
template <typename R>
__global__ void __launch_bounds__(256) k_scatter(int N, const uint32_t* __restrict__ key,
                                                 const uint32_t* __restrict__ rank,
                                                 const uint32_t* __restrict__ offset,
                                                 const typename Rec<R>::T* __restrict__ rec_in,
                                                 typename Rec<R>::T* __restrict__ rec_out, uint32_t* __restrict__ perm,
                                                 uint32_t* __restrict__ bin_of_sorted,
                                                 const uint32_t* __restrict__ item2, int cap2,
                                                 int4* __restrict__ work2, int max_work2, int nbins)
{
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const uint32_t b = key[i];
    const uint32_t r = rank[i];
    if (!ENUF_IN(b, nbins)) return;
    const uint32_t d = offset[b] + r;
    if (!ENUF_IN(d, N)) return;
    rec_out[d] = rec_in[i];
    perm[d] = (uint32_t)i;
    if (bin_of_sorted) bin_of_sorted[d] = b;
    if (work2 && r % (uint32_t)cap2 == 0u) {
        const uint32_t it = item2[b] + r / (uint32_t)cap2;
        const uint32_t nb = offset[b + 1] - offset[b];
        if ((int)it < max_work2) work2[it] = make_int4((int)b, (int)d, (int)(offset[b] + min(nb, r + (uint32_t)cap2)), 0);
    }
}

}  // namespace enuf
