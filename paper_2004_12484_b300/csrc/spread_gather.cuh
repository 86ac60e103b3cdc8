// spread_gather.cuh -- the two non-equispaced steps of the NFFT (Sec. 3.1):
//
//   spreading:      g_l = sum_j q_j prod_t phi(u_{j,t} - l_t)           (a3)
//   interpolating:  v_j = sum_l prod_t phi(u_{j,t} - l_t) w_l           (a7)
//
// with the Gaussian window phi(u) = (pi b)^(-1/2) exp(-u^2/b) on the p grid
// points l = floor(u) - p/2 + 1 ... floor(u) + p/2 of each dimension.  The
// window values are evaluated on the fly in registers, never tabulated in
// global memory (as Sec. 3.2 prescribes for the GPU kernels).
//
// Particles were counting-sorted into sub-tiles (S^3 cells, S = min(T, 8))
// numbered tile-major, so every tile of T^3 cells is one contiguous range.
// Both kernels keep a padded shared-memory box covering every cell their
// particles touch (edge + p - 1 cells in y and z; in x widened to 16-byte
// aligned rows).  Spreading gives each warp one sub-tile and a private box,
// updated without atomics and flushed with one global vector atomic per
// non-zero aligned group of four cells (scalar atomics in double).
// Interpolation gives each CTA one tile (or one z-half of it), stages the
// box of every field -- by the TMA engine for p = 8 and 6 in single
// precision, else with 16-byte loads -- and then reads only shared memory.  In both, a group of G >=
// p lanes serves one particle: lane a takes the x-offset a, so a group reads
// or writes p consecutive cells of one grid row per step; the partial sums
// are combined with shuffles.
#pragma once
#include <cuda.h>  // CUtensorMap

#include "common.cuh"

namespace enuf {

template <int P> struct GroupOf {
    static constexpr int G = P <= 2 ? 2 : (P <= 4 ? 4 : (P <= 8 ? 8 : 16));
};

// Entries of the per-warp table of y-z weight products that visit_window
// uses for the window widths without a register path (p = 4, 6 and 8 keep
// the weights in registers).
template <int P> struct WyzTable {
    static constexpr int N = (P == 4 || P == 6 || P == 8) ? 0 : P * P;
};

// Per-plan window constants: 1/b, log2(e)/b and c[a] = exp(-a^2 / b), a < P.
template <typename R> struct WinC {
    R inv_b;
    R l2b;
    R c[16];
};

// exp(-s / b).  Single precision evaluates 2^(-s log2(e) / b) with the
// factor folded into one constant, by the PTX instruction ex2.approx.ftz
// (relative error about 2^-22; the arguments, at least -(p/2)^2 log2(e)/b
// >= -60 for the supported widths, never reach the denormal range that the
// flush to zero would change); double calls exp.
__device__ __forceinline__ float win_exp(float s, const WinC<float>& wc)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-s * wc.l2b));
    return y;
}
__device__ __forceinline__ double win_exp(double s, const WinC<double>& wc) { return exp(-s * wc.inv_b); }

// Window weights of one dimension for the in-cell fraction d in [0, 1]:
// w[a] = exp(-(d + j)^2 / b) with j = m - 1 - a, a = 0..P-1 (normalisation
// applied by the caller).  Fast Gaussian gridding (Greengard and Lee, the
// gridding of Sec. 3.1), centred on the particle's cell so that no factor
// is raised beyond the power m: (d + j)^2 = d^2 + 2 d j + j^2 gives
// w = exp(-d^2/b) g^j c[j] for j >= 0 and exp(-d^2/b) (1/g)^(-j) c[-j] for
// j < 0, with g = exp(-2d/b) and c[j] = exp(-j^2/b): three exponentials per
// dimension instead of P.
template <typename R, int P>
__device__ __forceinline__ void window_weights(R d, const WinC<R>& wc, R (&w)[P])
{
    constexpr int m = P / 2;
    const R e0 = win_exp(d * d, wc);
    const R g = win_exp(R(2) * d, wc);
    const R gi = win_exp(R(-2) * d, wc);
    R up = e0, dn = e0;
#pragma unroll
    for (int j = 0; j < m; j++) {       // a = m - 1 - j
        w[m - 1 - j] = up * wc.c[j];
        up *= g;
    }
#pragma unroll
    for (int j = 1; j <= m; j++) {      // a = m - 1 + j
        dn *= gi;
        w[m - 1 + j] = dn * wc.c[j];
    }
}

template <typename R, int T>
__device__ __forceinline__ void split_offset(R o, int& i, R& d)
{
    int c = (int)o;          // o >= 0
    if (c > T - 1) c = T - 1; // float rounding can give o == T
    i = c;
    d = o - (R)c;
}

// Products wy[b] * wz[c] of one particle's y and z window weights, written
// by the warp into `wyz` (row rr = b + P c): lane k < P evaluates the two
// exponentials of offset k and the products are formed with shuffles.
template <typename R, int P>
__device__ __forceinline__ void pair_weights(R dy, R dz, const WinC<R>& wc, R* wyz, int lane)
{
    constexpr int m = P / 2;
    const int k = lane < P ? lane : 0;
    const R uy = dy + (R)(m - 1 - k), uz = dz + (R)(m - 1 - k);
    const R wy = win_exp(uy * uy, wc), wz = win_exp(uz * uz, wc);
#pragma unroll
    for (int r0 = 0; r0 < P * P; r0 += 32) {
        const int rr = r0 + lane;
        const int b = rr % P, c = (rr / P) % P;
        const R vy = __shfl_sync(0xffffffffu, wy, b);
        const R vz = __shfl_sync(0xffffffffu, wz, c);
        if (rr < P * P) wyz[rr] = vy * vz;
    }
}

// Visits the P*P window rows of one particle with a whole warp, 32/G rows
// per step: lane G g + a handles x-offset a (if a < P) of row rr = (32/G) it
// + g, so the rows of one instruction start on different banks; f(it, rr, b,
// c) with b = rr % P, c = rr / P.
template <int P, typename Fn>
__device__ __forceinline__ void window_rows(int a, int g, Fn&& f)
{
    constexpr int RPI = 32 / GroupOf<P>::G;
    if (a >= P) return;
#pragma unroll
    for (int it = 0; it < (P * P + RPI - 1) / RPI; it++) {
        const int rr = RPI * it + g;
        if (rr < P * P) f(it, rr, rr % P, rr / P);
    }
}

// Calls f(s, b, c, w) for the window rows this lane serves (see
// window_rows), with w = wx * wy[b] * wz[c] (wx: the lane's own x weight)
// and s = 0, 1, ... the lane's step.  For p = 8 and p = 4 the lane's rows
// fall on fixed y offsets, so the weights stay in registers (p = 8: the
// lane's two y weights evaluated in the lane; p = 4: one shuffle; wx folded
// into the y weights); other widths go through the per-warp product table
// `wyz` in shared memory.
template <typename R, int P, typename Fn>
__device__ __forceinline__ void visit_window(R dy, R dz, R wx, const WinC<R>& wc, R* wyz, int lane, Fn&& f)
{
    constexpr int G = GroupOf<P>::G;
    const int g = lane / G, a = lane % G;
    if constexpr (P == 8) {
        R wz[8];
        window_weights<R, 8>(dz, wc, wz);
        const R uy0 = dy + (R)(3 - g), uy1 = dy - (R)(1 + g);
        const R t0 = wx * win_exp(uy0 * uy0, wc), t1 = wx * win_exp(uy1 * uy1, wc);
#pragma unroll
        for (int c = 0; c < 8; c++) {
            f(2 * c, g, c, t0 * wz[c]);
            f(2 * c + 1, g + 4, c, t1 * wz[c]);
        }
    } else if constexpr (P == 6) {
        // lane (g, a < 6): planes g and (g < 2) g + 4, all six rows; the six
        // y weights and the lane's z weights evaluated in the lane (the four
        // groups of one access touch four consecutive planes)
        if (a >= P) return;
        R wy[6];
        window_weights<R, 6>(dy, wc, wy);
        const R uz0 = dz + (R)(2 - g), uz1 = dz - (R)(2 + g);
        const R t0 = wx * win_exp(uz0 * uz0, wc), t1 = wx * win_exp(uz1 * uz1, wc);
#pragma unroll
        for (int b = 0; b < 6; b++) f(b, b, g, t0 * wy[b]);
        if (g < 2) {
#pragma unroll
            for (int b = 0; b < 6; b++) f(6 + b, b, g + 4, t1 * wy[b]);
        }
    } else if constexpr (P == 4) {
        R wz[4];
        window_weights<R, 4>(dz, wc, wz);
        const R u = dy + (R)(1 - a);
        const R wyo = win_exp(u * u, wc);
        const int b = g & 3, hi = g >> 2;
        const R t = wx * __shfl_sync(0xffffffffu, wyo, b);
#pragma unroll
        for (int it = 0; it < 2; it++) f(it, b, 2 * it + hi, t * (hi ? wz[2 * it + 1] : wz[2 * it]));
    } else {
        pair_weights<R, P>(dy, dz, wc, wyz, lane);
        __syncwarp();
        window_rows<P>(a, g, [&](int it, int rr, int b, int c) { f(it, b, c, wx * wyz[rr]); });
        __syncwarp();
    }
}

// Sum over the warp of four values per lane, transposed: the lanes exchange
// half of their values at each of the first two steps, so that 6 shuffles
// replace 20.  Returns, in lane l, the total of value (l >> 3) & 3 (lanes 0,
// 8, 16, 24 hold totals 0, 1, 2, 3).
template <typename R>
__device__ __forceinline__ R warp_sum4(const R (&v)[4], int lane)
{
    const bool h16 = lane & 16, h8 = lane & 8;
    R k0 = h16 ? v[2] : v[0], k1 = h16 ? v[3] : v[1];
    k0 += __shfl_xor_sync(0xffffffffu, h16 ? v[0] : v[2], 16);
    k1 += __shfl_xor_sync(0xffffffffu, h16 ? v[1] : v[3], 16);
    R k = h8 ? k1 : k0;
    k += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    return k;
}

// Shared-memory box of a work unit of T x T x ZS cells (a tile, ZS = T, or
// one z-half of it, ZS = T / 2): x from tile_x0 - XA to tile_x0 - XA + BX
// (XA >= m - 1 and BX multiples of 4 so that rows start on 16-byte
// boundaries in global memory), y from the tile origin - (m - 1) over
// PT = T + p - 1 cells, z from the unit's origin - (m - 1) over PZ = ZS + p - 1.
template <int P, int T, int ZS = T> struct Box {
    static constexpr int m = P / 2;
    static constexpr int XA = (m - 1 + 3) / 4 * 4;
    static constexpr int BX = (XA + T + m + 3) / 4 * 4;
    static constexpr int PT = T + P - 1;
    static constexpr int PZ = ZS + P - 1;
    static constexpr int CELLS = BX * PT * PZ;
    static constexpr int XOFF = XA - (m - 1);  // box x of window point 0 minus floor(u)
};

// Spreading, one warp (the whole CTA) per work item = (sub-tile, particle
// range).  A sub-tile is S^3 cells of a T^3 tile, S = min(T, 8); the warp
// accumulates its particles into a private shared-memory box (S + p - 1
// cells in y and z, 16-byte aligned rows in x) with plain read-add-write:
// no other warp touches the box, so no shared-memory atomics are needed,
// and the P*P/(32/G) rows a lane updates for one particle are distinct
// cells, so their reads are all issued before their writes.  The box is then
// added to the grid with one vector atomic per non-zero aligned group of four
// cells (scalar atomics in double).  Work item index x = tile << (3 lr) |
// sub-tile (lr = log2(T / S)).
// The spreading box of a sub-tile (S^3 cells): the Box geometry with row
// stride BX and plane stride PS padded so that the four rows one warp
// instruction touches start on disjoint groups of 8 banks -- the same row of
// four consecutive planes for p = 8 (PS = 24 banks mod 32), for p = 6 on
// 8-cell sub-tiles rows 24 and planes 16 banks apart (see RowsP6), four
// consecutive rows otherwise.
template <int P, int S> struct SBox {
    using B0 = Box<P, S>;
    static constexpr int m = P / 2, XA = B0::XA, XOFF = B0::XOFF, PT = B0::PT;
    static constexpr int BX = (P != 8 && B0::BX % 16 == 0) ? B0::BX + 8 : B0::BX;
    static constexpr bool P6 = P == 6 && BX == 24;
    static constexpr int PS0 = PT * BX;
    static constexpr int PS = P6 ? PS0 + (48 - PS0 % 32) % 32 : PS0 + ((P == 8 && PS0 % 16 == 0) ? 8 : 0);
    static constexpr int CELLS = PT * PS;
};

// The window rows of one lane for p = 6 (lane 8 g + a, x offset a < 6): the
// 36 rows (y offset b, z offset c) of a window split into 12 runs of three
// planes (b, c = 3h .. 3h + 2), and group g takes the three runs with
// 3 b + 2 h = g (mod 4).  Every lane then visits 9 points instead of the 12
// (two planes of six rows) of the lanes that do most in a plane-wise split,
// and where rows lie 24 banks and planes 16 banks apart (mod 32) the four
// groups of one access touch disjoint groups of 8 banks: (3 b + 2 c) mod 4 =
// g + 2j for the run's plane j.  Runs 0 and 1 have h = 0 and 1; run 2 the
// h of the remaining class member (b + 4 < 6).
struct RowsP6 {
    int b[3];
    bool h2;  // run 2 on planes 3..5
    __device__ __forceinline__ explicit RowsP6(int g)
    {
        const int r0 = (3 * g) & 3, r1 = (3 * g + 2) & 3;
        b[0] = r0;
        b[1] = r1;
        h2 = r0 >= 2;
        b[2] = (h2 ? r1 : r0) + 4;
    }
};

template <typename R, int P, int T>
__global__ void __launch_bounds__(32) k_spread(const int4* __restrict__ work, const int* __restrict__ nwork,
                                               const typename Rec<R>::T* __restrict__ rec, int M, int lnb, int lr,
                                               WinC<R> wc, R cnorm3, R* __restrict__ grid, int N)
{
    constexpr int S = T < 8 ? T : 8;
    using B = SBox<P, S>;
    constexpr int PT = B::PT, BX = B::BX, PS = B::PS, m = P / 2, G = GroupOf<P>::G;
    extern __shared__ __align__(32) unsigned char smraw_sg[];
    R* acc = reinterpret_cast<R*>(smraw_sg);
    R* wyz = acc + B::CELLS;  // P*P products (window widths without a register path)
    using RecT = typename Rec<R>::T;
    pdl_wait();
    if ((int)blockIdx.x >= *nwork) return;  // uniform for the whole CTA
    const int4 w = work[blockIdx.x];
    const int lane = threadIdx.x;
    for (int i = lane; i < B::CELLS * (int)sizeof(R) / 16; i += 32)
        reinterpret_cast<float4*>(acc)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int sub = w.x & ((1 << (3 * lr)) - 1), tile = w.x >> (3 * lr), rm = (1 << lr) - 1;
    const int sx = sub & rm, sy = (sub >> lr) & rm, sz = sub >> (2 * lr);
    const int nbm = (1 << lnb) - 1;
    const int tx = tile & nbm, ty = (tile >> lnb) & nbm, tz = tile >> (2 * lnb);
    const int a = lane % G;
    if (!(ENUF_IN(tz, nbm + 1) && ENUF_IN(w.y, w.z) && ENUF_IN(w.z - 1, N))) return;
    __syncwarp();

    // p = 8 and 6: the warp's 32 records go through shared memory (one
    // broadcast load per particle; shuffles would share the shared-memory
    // pipe that bounds this kernel, four per particle)
    constexpr bool SREC = P == 8 || B::P6;
    __shared__ RecT srecs[SREC ? 32 : 1];
    const RowsP6 rows6(lane >> 3);  // p = 6: the lane's window rows
    int o6[3];                      // and their offsets in the box
#pragma unroll
    for (int k = 0; k < 3; k++) o6[k] = (k == 1 || (k == 2 && rows6.h2) ? 3 * PS : 0) + rows6.b[k] * BX;
    for (int j0 = w.y; j0 < w.z; j0 += 32) {
        // one record per lane, handed to the warp with shuffles (or, p = 8
        // and 6, through shared memory)
        RecT mine;
        if (j0 + lane < w.z) mine = rec[j0 + lane];
        else mine.x = mine.y = mine.z = mine.w = R(0);
        if constexpr (SREC) {
            srecs[lane] = mine;
            __syncwarp();
        }
        const int nj = min(32, w.z - j0);
        for (int jj = 0; jj < nj; jj++) {
            R rx, ry, rz, rq;
            if constexpr (SREC) {
                const RecT rr = srecs[jj];
                rx = rr.x;
                ry = rr.y;
                rz = rr.z;
                rq = rr.w;
            } else {
                rx = __shfl_sync(0xffffffffu, mine.x, jj);
                ry = __shfl_sync(0xffffffffu, mine.y, jj);
                rz = __shfl_sync(0xffffffffu, mine.z, jj);
                rq = __shfl_sync(0xffffffffu, mine.w, jj);
            }
            int ix, iy, iz;
            R dx, dy, dz;
            split_offset<R, T>(rx, ix, dx);
            split_offset<R, T>(ry, iy, dy);
            split_offset<R, T>(rz, iz, dz);
            ix -= sx * S;  // cell inside the sub-tile, 0..S-1 (the bin was
            iy -= sy * S;  // chosen from the same split)
            iz -= sz * S;
            if (!(ENUF_IN(ix, S) && ENUF_IN(iy, S) && ENUF_IN(iz, S))) {  // uniform for the warp
                __syncwarp();
                continue;
            }
            const R ua = dx + (R)(m - 1 - (a % P));
            const R wx = rq * cnorm3 * win_exp(ua * ua, wc);
            constexpr int RPI = 32 / G;
            constexpr int NV = P == 8 ? 16 : (P == 6 ? 12 : (P == 4 ? 2 : (P * P + RPI - 1) / RPI));
            if constexpr (P == 8) {
                // lane 8 g + a: x-offset a of planes g and g + 4 and all eight
                // rows; every lane evaluates the eight y weights (fast Gaussian
                // gridding: three exponentials) and its two z weights itself
                // rather than taking them by shuffles.  The four lane groups
                // of one access touch planes g + 4 s, PS apart: disjoint
                // groups of 8 banks.
                const int g = lane >> 3;
                R wy8[8];
                window_weights<R, 8>(dy, wc, wy8);
                const R uz0 = dz + (R)(3 - g), uz1 = dz - (R)(1 + g);
                const R t0 = wx * win_exp(uz0 * uz0, wc), t1 = wx * win_exp(uz1 * uz1, wc);
                R* base = acc + (iz + g) * PS + iy * BX + ix + B::XOFF + a;
                R old[16];
#pragma unroll
                for (int s = 0; s < 2; s++) {
#pragma unroll
                    for (int i = 0; i < 8; i++) old[8 * s + i] = base[4 * s * PS + i * BX];
                }
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    base[i * BX] = old[i] + t0 * wy8[i];
                    base[4 * PS + i * BX] = old[8 + i] + t1 * wy8[i];
                }
            } else if constexpr (B::P6) {
                // lane 8 g + a: x-offset a of the three runs of RowsP6 (9
                // points); the y weights of its rows and the six z weights
                // evaluated in the lane
                R wz6[6];
                window_weights<R, 6>(dz, wc, wz6);
                R t[3];
#pragma unroll
                for (int k = 0; k < 3; k++) {
                    const R uy = dy + (R)(2 - rows6.b[k]);
                    t[k] = wx * win_exp(uy * uy, wc);
                }
                if (a < P) {
                    R* base = acc + iz * PS + iy * BX + ix + B::XOFF + a;
                    R old[9];
#pragma unroll
                    for (int k = 0; k < 3; k++) {
#pragma unroll
                        for (int j = 0; j < 3; j++) old[3 * k + j] = base[o6[k] + j * PS];
                    }
#pragma unroll
                    for (int j = 0; j < 3; j++) {
                        const R z2 = rows6.h2 ? wz6[3 + j] : wz6[j];
                        base[o6[0] + j * PS] = old[j] + t[0] * wz6[j];
                        base[o6[1] + j * PS] = old[3 + j] + t[1] * wz6[3 + j];
                        base[o6[2] + j * PS] = old[6 + j] + t[2] * z2;
                    }
                }
            } else if constexpr (NV <= 16) {
                R* base = acc + (iz * PS) + iy * BX + ix + B::XOFF + a;
                int off[NV];
                R vv[NV];
                unsigned valid = 0u;
                visit_window<R, P>(dy, dz, wx, wc, wyz, lane, [&](int st, int b, int c, R wv) {
                    off[st] = c * PS + b * BX;
                    vv[st] = wv;
                    valid |= 1u << st;
                });
                if (a < P) {
                    R old[NV];
#pragma unroll
                    for (int k = 0; k < NV; k++)
                        if (valid >> k & 1u) old[k] = base[off[k]];
#pragma unroll
                    for (int k = 0; k < NV; k++)
                        if (valid >> k & 1u) base[off[k]] = old[k] + vv[k];
                }
            } else {
                R* base = acc + (iz * PS) + iy * BX + ix + B::XOFF + a;
                visit_window<R, P>(dy, dz, wx, wc, wyz, lane, [&](int, int b, int c, R wv) {
                    if (a < P) base[c * PS + b * BX] += wv;
                });
            }
            __syncwarp();
        }
    }

    const int ox = tx * T + sx * S - B::XA, oy = ty * T + sy * S - (m - 1), oz = tz * T + sz * S - (m - 1);
    const int mask = M - 1;  // M is a power of two (and a multiple of 4)
    if constexpr (sizeof(R) == 4) {
        // one 16-byte vector atomic per aligned group of 4 cells
        constexpr int NV4 = B::B0::BX / 4;  // vectors per row that hold cells
        for (int i = lane; i < NV4 * PT * PT; i += 32) {
            const int vx = i % NV4, ly = (i / NV4) % PT, lz = i / (NV4 * PT);
            const float4 v = *reinterpret_cast<const float4*>(acc + lz * PS + ly * BX + 4 * vx);
            if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) {
                const int gx = (ox + 4 * vx) & mask, gy = (oy + ly) & mask, gz = (oz + lz) & mask;
                const size_t gi = ((size_t)gz * M + gy) * M + gx;
                if (ENUF_IN(gi + 3, (size_t)M * M * M)) atomicAdd(reinterpret_cast<float4*>(grid + gi), v);
            }
        }
    } else {
        constexpr int NX = B::B0::BX;
        for (int i = lane; i < NX * PT * PT; i += 32) {
            const int lx = i % NX, ly = (i / NX) % PT, lz = i / (NX * PT);
            const R v = acc[lz * PS + ly * BX + lx];
            if (v != R(0)) {
                const int gx = (ox + lx) & mask, gy = (oy + ly) & mask, gz = (oz + lz) & mask;
                const size_t gi = ((size_t)gz * M + gy) * M + gx;
                if (ENUF_IN(gi, (size_t)M * M * M)) atomicAdd(grid + gi, v);
            }
        }
    }
}

// Interpolates the n particles of one staged work unit from its box s (NF
// fields of Box<P, T, ZS>::CELLS cells; z0 = the unit's first cell inside its
// tile): one warp per particle, rows spread over the lanes as in k_spread.
// wyz: the warp's weight-product table; srec: the unit's records; oidx(k):
// the caller's index of the unit's particle k.  Fields 0..2 give the force
// per unit charge (F_i = q_i * value), field 3 (NF = 4) the potential.
template <typename R, int P, int T, int NF, int ZS, typename OIdx>
__device__ __forceinline__ void interp_unit(const R* s, R* wyz, const typename Rec<R>::T* srec, int n, int z0,
                                            const WinC<R>& wc, R cnorm3, R* __restrict__ F, R* __restrict__ phi,
                                            OIdx&& oidx, int N)
{
    using B = Box<P, T, ZS>;
    constexpr int PT = B::PT, BX = B::BX, C = B::CELLS, m = P / 2, G = GroupOf<P>::G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int a = lane % G;
    for (int k = warp; k < n; k += nwarp) {
        const typename Rec<R>::T r = srec[k];
        int ix, iy, iz;
        R dx, dy, dz;
        split_offset<R, T>(r.x, ix, dx);
        split_offset<R, T>(r.y, iy, dy);
        split_offset<R, T>(r.z, iz, dz);
        iz -= z0;
        if (!(ENUF_IN(ix, T) && ENUF_IN(iy, T) && ENUF_IN(iz, ZS))) continue;  // uniform for the warp
        const R ua = dx + (R)(m - 1 - (a % P));
        const R wx = win_exp(ua * ua, wc);
        const R* base = s + (iz * PT + iy) * BX + ix + B::XOFF + a;
        R acc[4] = {R(0), R(0), R(0), R(0)};
        visit_window<R, P>(dy, dz, wx, wc, wyz, lane, [&](int, int b, int c, R ww) {
            if (a < P) {
                const int o = (c * PT + b) * BX;
#pragma unroll
                for (int f = 0; f < NF; f++) acc[f] += ww * base[f * C + o];
            }
        });
        // warp sum of the four partials, transposed: after it lane 8 f
        // holds the total of field f
        const R tot = warp_sum4(acc, lane);
        if ((lane & 7) == 0) {
            const int f = lane >> 3;
            const uint32_t oi = oidx(k);
            if (!ENUF_IN(oi, N)) {
            } else if (f < 3) {
                if (F) F[3 * (size_t)oi + f] = r.w * cnorm3 * tot;
            } else if (NF == 4 && phi) {
                phi[oi] = cnorm3 * tot;
            }
        }
        __syncwarp();
    }
}

// Interpolation of NF real fields (planes of M^3, plane stride M^3).  Fields
// 0..2 give the force per unit charge (F_i = q_i * value), field 3 (when
// NF = 4) the potential phi_i.  F is written (not accumulated) in the
// caller's particle order through perm.  A work item covers a whole tile
// (ZS = T, item x = tile) or one z-half of a tile (ZS = T / 2, item x =
// 2 tile + half): the half box lets two CTAs share an SM, so one stages its
// box while the other interpolates.
template <typename R, int P, int T, int NF, int NTH, int ZS = T>
__global__ void __launch_bounds__(NTH) k_gather(const int4* __restrict__ work, const int* __restrict__ nwork,
                                                const typename Rec<R>::T* __restrict__ rec,
                                                const uint32_t* __restrict__ perm, int M, int lnbx, int lnby,
                                                WinC<R> wc, R cnorm3, const R* __restrict__ fld, R* __restrict__ F,
                                                R* __restrict__ phi, int N)
{
    using B = Box<P, T, ZS>;
    constexpr int PT = B::PT, PZ = B::PZ, BX = B::BX, C = B::CELLS, m = P / 2, G = GroupOf<P>::G;
    static_assert(ZS == T || 2 * ZS == T, "a work unit is a tile or half of one");
    extern __shared__ __align__(32) unsigned char smraw_sg[];
    R* s = reinterpret_cast<R*>(smraw_sg);
    pdl_wait();
    if ((int)blockIdx.x >= *nwork) return;
    const int4 w = work[blockIdx.x];
    const int tile = ZS < T ? w.x >> 1 : w.x;
    const int z0 = ZS < T ? (w.x & 1) * ZS : 0;  // the unit's first cell inside the tile
    const int tx = tile & ((1 << lnbx) - 1), ty = (tile >> lnbx) & ((1 << lnby) - 1), tz = tile >> (lnbx + lnby);
    const int ox = tx * T - B::XA, oy = ty * T - (m - 1), oz = tz * T + z0 - (m - 1);
    const int mask = M - 1;
    const size_t M3 = (size_t)M * M * M;
    if (!(ENUF_IN(tz, M / T) && ENUF_IN(w.y, w.z) && ENUF_IN(w.z - 1, N) &&
          ENUF_IN((NF * C + (blockDim.x >> 5) * WyzTable<P>::N) * sizeof(R) +
                      (size_t)(w.z - w.y) * (sizeof(typename Rec<R>::T) + 4) - 1,
                  dynamic_smem_bytes())))
        return;  // uniform for the CTA
    // stage the box of every field with 16-byte loads
    constexpr int EV = 16 / sizeof(R);  // elements per 16-byte vector
    constexpr int NV = BX / EV;
    for (int i = threadIdx.x; i < NV * PT * PZ; i += blockDim.x) {
        const int vx = i % NV, ly = (i / NV) % PT, lz = i / (NV * PT);
        const size_t gi = ((size_t)((oz + lz) & mask) * M + ((oy + ly) & mask)) * M + ((ox + EV * vx) & mask);
        const int si = (lz * PT + ly) * BX + EV * vx;
#pragma unroll
        for (int f = 0; f < NF; f++)
            *reinterpret_cast<float4*>(s + f * C + si) = __ldg(reinterpret_cast<const float4*>(fld + f * M3 + gi));
    }
    using RecT = typename Rec<R>::T;
    RecT* srec = reinterpret_cast<RecT*>(s + NF * C + (blockDim.x >> 5) * WyzTable<P>::N);
    uint32_t* sperm = reinterpret_cast<uint32_t*>(srec + (w.z - w.y));
    for (int i = threadIdx.x; i < w.z - w.y; i += blockDim.x) {
        srec[i] = rec[w.y + i];
        sperm[i] = perm[w.y + i];
    }
    __syncthreads();

    interp_unit<R, P, T, NF, ZS>(s, s + NF * C + (threadIdx.x >> 5) * WyzTable<P>::N, srec, w.z - w.y, z0, wc,
                                 cnorm3, F, phi, [&](int k) { return sperm[k]; }, N);
}

// Staging of one work unit of the TMA interpolation kernels (k_gather_p8,
// k_gather_p6): one thread has the TMA engine copy the unit's box of each
// field plane (a tensor-map box of BX x PY x PZ cells from (ox, oy, oz),
// plane f at s + f C) and the unit's n particle records into shared memory,
// completing on the mbarrier `bar`; cells of a box that crosses the edge of
// the periodic grid arrive as zeros and are then filled from their periodic
// images by the threads (16-byte copies of whole aligned groups of four
// cells, all in flight before the wait).  Needs M >= BX (a box crosses each
// edge at most once).  Returns false (the status word flagged) if the copies
// did not complete within the wait's bound.
template <int NF, int BX, int PY, int PZ, int C>
__device__ __forceinline__ bool stage_unit_tma(float* s, f4* srec, uint64_t* bar, const CUtensorMap* tmap,
                                               const f4* rec, int n, int ox, int oy, int oz, int M,
                                               const float* __restrict__ fld, int* status)
{
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)(NF * BX * PY * PZ * 4 + n * 16));
#pragma unroll
        for (int f = 0; f < NF; f++) tma_load_4d(s + f * C, tmap, ox, oy, oz, f, bar);
        bulk_g2s(srec, rec, (uint32_t)n * 16u, bar);
    }
    if (!mbar_wait(bar, 0, 1 << 22)) {
        // should not happen: report, and wait (bounded) for the copies still
        // writing this CTA's shared memory before leaving
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        mbar_wait(bar, 0, 1 << 22);
        return false;
    }
    if (ox < 0 || ox + BX > M || oy < 0 || oy + PY > M || oz < 0 || oz + PZ > M) {
        const int mask = M - 1;
        const size_t M3 = (size_t)M * M * M;
        constexpr int NV = BX / 4;
        for (int i = threadIdx.x; i < NV * PY * PZ; i += blockDim.x) {
            const int vx = i % NV, ly = (i / NV) % PY, lz = i / (NV * PY);
            const int gx = ox + 4 * vx, gy = oy + ly, gz = oz + lz;
            if (gx >= 0 && gx < M && gy >= 0 && gy < M && gz >= 0 && gz < M) continue;
            const size_t gi = ((size_t)(gz & mask) * M + (gy & mask)) * M + (gx & mask);
            const int si = (lz * PY + ly) * BX + 4 * vx;
            if (!ENUF_IN(gi + 3, M3)) continue;
#pragma unroll
            for (int f = 0; f < NF; f++) cp_async_bytes16(s + f * C + si, fld + f * M3 + gi, true);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    return true;
}

// Interpolation for windows of p = 8 on 16-cell tiles in z-halves, single
// precision (the configuration of the large workloads and the benchmark).
// Staging by stage_unit_tma (boxes of BX x PT x PZ cells).  Compute: one
// warp per particle, lane (g, a) = (lane / 8, lane % 8) takes x offset a of
// rows g and g + 4 and all eight planes, and sums each of its two rows
// along z with the z weights before applying the x and y weights, so a
// window point costs one shared load and one FMA per field.
template <int NF> struct GatherP8 {
    using B = Box<8, 16, 8>;
    static constexpr int PY = B::PT;                       // box rows (y)
    static constexpr int CP = (B::CELLS + 31) / 32 * 32;  // field stride in shared memory, 128-byte aligned
    static constexpr int CAP = 256;                        // particles per work item
    static constexpr size_t SMEM = (size_t)NF * CP * 4 + CAP * sizeof(f4) + 16;
};

template <int NF>
__global__ void __launch_bounds__(512, 2) k_gather_p8(const int4* __restrict__ work, const int* __restrict__ nwork,
                                                      const f4* __restrict__ rec, const uint32_t* __restrict__ perm,
                                                      int M, int lnb, WinC<float> wc, float cnorm3,
                                                      const float* __restrict__ fld,
                                                      const __grid_constant__ CUtensorMap tmap, float* __restrict__ F,
                                                      float* __restrict__ phi, int* __restrict__ status, int N)
{
    using G8 = GatherP8<NF>;
    using B = typename G8::B;
    constexpr int PT = B::PT, PZ = B::PZ, BX = B::BX, C = G8::CP, XOFF = B::XOFF;
    extern __shared__ __align__(128) unsigned char smraw_g8[];
    float* s = reinterpret_cast<float*>(smraw_g8);
    f4* srec = reinterpret_cast<f4*>(s + NF * C);
    uint64_t* bar = reinterpret_cast<uint64_t*>(srec + G8::CAP);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    pdl_wait();
    if ((int)blockIdx.x >= *nwork) return;  // uniform for the whole CTA
    const int4 w = work[blockIdx.x];
    const int n = w.z - w.y;                 // 1..CAP (the scan splits larger units)
    const int tile = w.x >> 1, z0 = (w.x & 1) * 8;
    const int nbm = (1 << lnb) - 1;
    const int tx = tile & nbm, ty = (tile >> lnb) & nbm, tz = tile >> (2 * lnb);
    const int ox = tx * 16 - B::XA, oy = ty * 16 - 3, oz = tz * 16 + z0 - 3;
    if (!(ENUF_IN(tz, nbm + 1) && ENUF_IN(n - 1, G8::CAP) && ENUF_IN(w.z - 1, N))) return;  // uniform for the CTA
    if (!stage_unit_tma<NF, BX, PT, PZ, C>(s, srec, bar, &tmap, rec + w.y, n, ox, oy, oz, M, fld, status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 3, a = lane & 7;
    for (int k = warp; k < n; k += 16) {
        // the output index is needed last: its load runs under the window sums
        const uint32_t oi = perm[w.y + k];
        const f4 r = srec[k];
        int ix, iy, iz;
        float dx, dy, dz;
        split_offset<float, 16>(r.x, ix, dx);
        split_offset<float, 16>(r.y, iy, dy);
        split_offset<float, 16>(r.z, iz, dz);
        iz -= z0;
        if (!(ENUF_IN(ix, 16) && ENUF_IN(iy, 16) && ENUF_IN(iz, 8))) continue;  // uniform for the warp
        // the lane's x weight and the y weights of its rows g and g + 4, each
        // evaluated in the lane (an exponential costs less than a shuffle
        // through the shared-memory pipe that bounds this kernel)
        const float ux = dx + (float)(3 - a), uy0 = dy + (float)(3 - g), uy1 = dy - (float)(1 + g);
        const float wx = win_exp(ux * ux, wc), wy0 = win_exp(uy0 * uy0, wc), wy1 = win_exp(uy1 * uy1, wc);
        float wz[8];
        window_weights<float, 8>(dz, wc, wz);
        const float* base = s + (iz * PT + iy + g) * BX + ix + XOFF + a;
        float s0[NF], s1[NF];
#pragma unroll
        for (int f = 0; f < NF; f++) s0[f] = s1[f] = 0.f;
#pragma unroll
        for (int c = 0; c < 8; c++) {
#pragma unroll
            for (int f = 0; f < NF; f++) {
                s0[f] = fmaf(wz[c], base[f * C + c * PT * BX], s0[f]);
                s1[f] = fmaf(wz[c], base[f * C + c * PT * BX + 4 * BX], s1[f]);
            }
        }
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int f = 0; f < NF; f++) acc[f] = wx * fmaf(wy0, s0[f], wy1 * s1[f]);
        // lane 8 f holds the total of field f
        const float tot = warp_sum4(acc, lane);
        if ((lane & 7) == 0 && ENUF_IN(oi, N)) {
            const int f = lane >> 3;
            if (f < 3) {
                if (F) F[3 * (size_t)oi + f] = r.w * cnorm3 * tot;
            } else if (NF == 4 && phi) {
                phi[oi] = cnorm3 * tot;
            }
        }
    }
}

// Interpolation for windows of p = 6 on 16-cell tiles in z-halves, single
// precision: k_gather_p8's staging with boxes of BX x PY x PZ cells, PY one
// row more than the window needs (PT) so that planes lie 16 banks apart
// (mod 32) and rows 24.  Compute: one warp per particle, lane (g, a) takes
// x offset a (< 6) of the three runs of three planes of RowsP6 and sums each
// run along z before applying the x and y weights (9 shared loads and FMAs
// a field; lanes a = 6, 7 read lane 5's cells, a broadcast, with weight 0).
template <int NF> struct GatherP6 {
    using B = Box<6, 16, 8>;
    static constexpr int PY = B::PT + 1;                    // box rows (y)
    static constexpr int CELLS = B::BX * PY * B::PZ;
    static constexpr int CP = (CELLS + 31) / 32 * 32;       // field stride in shared memory, 128-byte aligned
    static constexpr int CAP = 256;                          // particles per work item
    static constexpr size_t SMEM = (size_t)NF * CP * 4 + CAP * sizeof(f4) + 16;
    static_assert(B::BX == 24 && (PY * B::BX) % 32 == 16, "rows 24 and planes 16 banks apart");
};

template <int NF>
__global__ void __launch_bounds__(512, 2) k_gather_p6(const int4* __restrict__ work, const int* __restrict__ nwork,
                                                      const f4* __restrict__ rec, const uint32_t* __restrict__ perm,
                                                      int M, int lnb, WinC<float> wc, float cnorm3,
                                                      const float* __restrict__ fld,
                                                      const __grid_constant__ CUtensorMap tmap, float* __restrict__ F,
                                                      float* __restrict__ phi, int* __restrict__ status, int N)
{
    using G6 = GatherP6<NF>;
    using B = typename G6::B;
    constexpr int PY = G6::PY, PZ = B::PZ, BX = B::BX, C = G6::CP, XOFF = B::XOFF;
    extern __shared__ __align__(128) unsigned char smraw_g6[];
    float* s = reinterpret_cast<float*>(smraw_g6);
    f4* srec = reinterpret_cast<f4*>(s + NF * C);
    uint64_t* bar = reinterpret_cast<uint64_t*>(srec + G6::CAP);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    pdl_wait();
    if ((int)blockIdx.x >= *nwork) return;  // uniform for the whole CTA
    const int4 w = work[blockIdx.x];
    const int n = w.z - w.y;                 // 1..CAP (the scan splits larger units)
    const int tile = w.x >> 1, z0 = (w.x & 1) * 8;
    const int nbm = (1 << lnb) - 1;
    const int tx = tile & nbm, ty = (tile >> lnb) & nbm, tz = tile >> (2 * lnb);
    const int ox = tx * 16 - B::XA, oy = ty * 16 - 2, oz = tz * 16 + z0 - 2;
    if (!(ENUF_IN(tz, nbm + 1) && ENUF_IN(n - 1, G6::CAP) && ENUF_IN(w.z - 1, N))) return;  // uniform for the CTA
    if (!stage_unit_tma<NF, BX, PY, PZ, C>(s, srec, bar, &tmap, rec + w.y, n, ox, oy, oz, M, fld, status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a = lane & 7, ax = a < 6 ? a : 5;
    const RowsP6 rows(lane >> 3);
    // the lane's three runs: offsets of their first cells from the window's corner
    const int o0 = rows.b[0] * BX, o1 = (3 * PY + rows.b[1]) * BX, o2 = ((rows.h2 ? 3 * PY : 0) + rows.b[2]) * BX;
    for (int k = warp; k < n; k += 16) {
        const uint32_t oi = perm[w.y + k];
        const f4 r = srec[k];
        int ix, iy, iz;
        float dx, dy, dz;
        split_offset<float, 16>(r.x, ix, dx);
        split_offset<float, 16>(r.y, iy, dy);
        split_offset<float, 16>(r.z, iz, dz);
        iz -= z0;
        if (!(ENUF_IN(ix, 16) && ENUF_IN(iy, 16) && ENUF_IN(iz, 8))) continue;  // uniform for the warp
        const float ux = dx + (float)(2 - ax);
        const float uy0 = dy + (float)(2 - rows.b[0]), uy1 = dy + (float)(2 - rows.b[1]),
                    uy2 = dy + (float)(2 - rows.b[2]);
        const float wx = a < 6 ? win_exp(ux * ux, wc) : 0.f;
        const float wy0 = win_exp(uy0 * uy0, wc), wy1 = win_exp(uy1 * uy1, wc), wy2 = win_exp(uy2 * uy2, wc);
        float wz[6];
        window_weights<float, 6>(dz, wc, wz);
        const float* base = s + (iz * PY + iy) * BX + ix + XOFF + ax;
        float s0[NF], s1[NF], s2[NF];
#pragma unroll
        for (int f = 0; f < NF; f++) s0[f] = s1[f] = s2[f] = 0.f;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float z2 = rows.h2 ? wz[3 + j] : wz[j];
#pragma unroll
            for (int f = 0; f < NF; f++) {
                s0[f] = fmaf(wz[j], base[f * C + o0 + j * PY * BX], s0[f]);
                s1[f] = fmaf(wz[3 + j], base[f * C + o1 + j * PY * BX], s1[f]);
                s2[f] = fmaf(z2, base[f * C + o2 + j * PY * BX], s2[f]);
            }
        }
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int f = 0; f < NF; f++) acc[f] = wx * fmaf(wy0, s0[f], fmaf(wy1, s1[f], wy2 * s2[f]));
        // lane 8 f holds the total of field f
        const float tot = warp_sum4(acc, lane);
        if ((lane & 7) == 0 && ENUF_IN(oi, N)) {
            const int f = lane >> 3;
            if (f < 3) {
                if (F) F[3 * (size_t)oi + f] = r.w * cnorm3 * tot;
            } else if (NF == 4 && phi) {
                phi[oi] = cnorm3 * tot;
            }
        }
    }
}

// Interpolation for the analytic-differentiation forces: one real potential
// grid A (plane of M^3) and, per particle, the window sum of A together with
// the three sums weighted by the window's derivative, d phi/du = -(2u/b) phi
// (u = particle minus grid point, in grid units).  With
//   s = sum_l w_l A_l,   g_t = sum_l u_t w_l A_l,
// the potential is phi_i = cnorm3 s and the force F_{i,t} = q_i fa_t g_t,
// fa_t = cnorm3 (M / L_t) (2 / b): the gradient of the approximated energy
// through the window values.  The staged box holds the one grid, so the
// tile's staging is a third of the three-field interpolation's and every
// window point costs one shared-memory load.
template <typename R, int P, int T, int NTH, int ZS = T>
__global__ void __launch_bounds__(NTH) k_gather_ad(const int4* __restrict__ work, const int* __restrict__ nwork,
                                                   const typename Rec<R>::T* __restrict__ rec,
                                                   const uint32_t* __restrict__ perm, int M, int lnbx, int lnby,
                                                   WinC<R> wc, R cnorm3, R fa0, R fa1, R fa2,
                                                   const R* __restrict__ fld, R* __restrict__ F, R* __restrict__ phi,
                                                   int N)
{
    using B = Box<P, T, ZS>;
    constexpr int PT = B::PT, PZ = B::PZ, BX = B::BX, C = B::CELLS, m = P / 2, G = GroupOf<P>::G;
    static_assert(ZS == T || 2 * ZS == T, "a work unit is a tile or half of one");
    extern __shared__ __align__(32) unsigned char smraw_sg[];
    R* s = reinterpret_cast<R*>(smraw_sg);
    pdl_wait();
    if ((int)blockIdx.x >= *nwork) return;
    const int4 w = work[blockIdx.x];
    const int tile = ZS < T ? w.x >> 1 : w.x;
    const int z0 = ZS < T ? (w.x & 1) * ZS : 0;  // the unit's first cell inside the tile
    const int tx = tile & ((1 << lnbx) - 1), ty = (tile >> lnbx) & ((1 << lnby) - 1), tz = tile >> (lnbx + lnby);
    const int ox = tx * T - B::XA, oy = ty * T - (m - 1), oz = tz * T + z0 - (m - 1);
    const int mask = M - 1;
    if (!(ENUF_IN(tz, M / T) && ENUF_IN(w.y, w.z) && ENUF_IN(w.z - 1, N) &&
          ENUF_IN((C + (blockDim.x >> 5) * WyzTable<P>::N) * sizeof(R) +
                      (size_t)(w.z - w.y) * (sizeof(typename Rec<R>::T) + 4) - 1,
                  dynamic_smem_bytes())))
        return;  // uniform for the CTA
    constexpr int EV = 16 / sizeof(R);
    constexpr int NV = BX / EV;
    for (int i = threadIdx.x; i < NV * PT * PZ; i += blockDim.x) {
        const int vx = i % NV, ly = (i / NV) % PT, lz = i / (NV * PT);
        const size_t gi = ((size_t)((oz + lz) & mask) * M + ((oy + ly) & mask)) * M + ((ox + EV * vx) & mask);
        *reinterpret_cast<float4*>(s + (lz * PT + ly) * BX + EV * vx) = __ldg(reinterpret_cast<const float4*>(fld + gi));
    }
    using RecT = typename Rec<R>::T;
    RecT* srec = reinterpret_cast<RecT*>(s + C + (blockDim.x >> 5) * WyzTable<P>::N);
    uint32_t* sperm = reinterpret_cast<uint32_t*>(srec + (w.z - w.y));
    for (int i = threadIdx.x; i < w.z - w.y; i += blockDim.x) {
        srec[i] = rec[w.y + i];
        sperm[i] = perm[w.y + i];
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int g = lane / G, a = lane % G;
    R* wyz = s + C + warp * WyzTable<P>::N;
    for (int j = w.y + warp; j < w.z; j += nwarp) {
        const RecT r = srec[j - w.y];
        int ix, iy, iz;
        R dx, dy, dz;
        split_offset<R, T>(r.x, ix, dx);
        split_offset<R, T>(r.y, iy, dy);
        split_offset<R, T>(r.z, iz, dz);
        iz -= z0;
        if (!(ENUF_IN(ix, T) && ENUF_IN(iy, T) && ENUF_IN(iz, ZS))) continue;  // uniform for the warp
        const R ux = dx + (R)(m - 1 - (a % P));
        const R wx = win_exp(ux * ux, wc);
        const R* base = s + (iz * PT + iy) * BX + ix + B::XOFF + a;
        // acc = (s, g_x, g_y, g_z) partials of this lane
        R acc[4];
        if constexpr (P == 8) {
            // lane (g, a): rows y = g and g + 4, all eight z; the z sums
            // with weights wz and u_z wz, then the y weights
            R wz[8];
            window_weights<R, 8>(dz, wc, wz);
            const R uy0 = dy + (R)(3 - g), uy1 = dy - (R)(1 + g);
            const R wy0 = win_exp(uy0 * uy0, wc), wy1 = win_exp(uy1 * uy1, wc);
            R s0 = R(0), d0 = R(0), s1 = R(0), d1 = R(0);
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const R wzu = wz[c] * (dz + (R)(3 - c));
                const R v0 = base[(c * PT + g) * BX], v1 = base[(c * PT + g + 4) * BX];
                s0 += wz[c] * v0;
                d0 += wzu * v0;
                s1 += wz[c] * v1;
                d1 += wzu * v1;
            }
            acc[0] = wx * (wy0 * s0 + wy1 * s1);
            acc[1] = ux * acc[0];
            acc[2] = wx * (wy0 * uy0 * s0 + wy1 * uy1 * s1);
            acc[3] = wx * (wy0 * d0 + wy1 * d1);
        } else {
            R sa = R(0), sy = R(0), sz = R(0);
            visit_window<R, P>(dy, dz, wx, wc, wyz, lane, [&](int, int b, int c, R ww) {
                if (a < P) {
                    const R t = ww * base[(c * PT + b) * BX];
                    sa += t;
                    sy += t * (dy + (R)(m - 1 - b));
                    sz += t * (dz + (R)(m - 1 - c));
                }
            });
            acc[0] = sa;
            acc[1] = a < P ? ux * sa : R(0);
            acc[2] = sy;
            acc[3] = sz;
        }
        const R tot = warp_sum4(acc, lane);
        if ((lane & 7) == 0 && ENUF_IN(sperm[j - w.y], N)) {
            const int f = lane >> 3;
            const uint32_t oi = sperm[j - w.y];
            if (f == 0) {
                if (phi) phi[oi] = cnorm3 * tot;
            } else if (F) {
                F[3 * (size_t)oi + f - 1] = r.w * (f == 1 ? fa0 : (f == 2 ? fa1 : fa2)) * tot;
            }
        }
        __syncwarp();
    }
}

// The analytic-differentiation interpolation of k_gather_ad for p = 6 on
// 16-cell tiles in z-halves, single precision: the potential grid's box
// staged by stage_unit_tma (the geometry of k_gather_p6, field plane 0 of
// the same tensor map) and the three-plane runs of RowsP6, each summed
// along z twice, with the z weights and with u_z times them, before the x
// and y weights are applied.  (The same staging for p = 8, with the rows of
// k_gather_p8, was slower than k_gather_ad's: 26.0 -> 28.7 us at RPM size.)
__global__ void __launch_bounds__(512, 2) k_gather_ad_p6(const int4* __restrict__ work, const int* __restrict__ nwork,
                                                         const f4* __restrict__ rec, const uint32_t* __restrict__ perm,
                                                         int M, int lnb, WinC<float> wc, float cnorm3, float fa0,
                                                         float fa1, float fa2, const float* __restrict__ fld,
                                                         const __grid_constant__ CUtensorMap tmap,
                                                         float* __restrict__ F, float* __restrict__ phi,
                                                         int* __restrict__ status, int N)
{
    using G = GatherP6<1>;
    using B = typename G::B;
    constexpr int PY = G::PY, PZ = B::PZ, BX = B::BX, C = G::CP, XOFF = B::XOFF;
    extern __shared__ __align__(128) unsigned char smraw_ga[];
    float* s = reinterpret_cast<float*>(smraw_ga);
    f4* srec = reinterpret_cast<f4*>(s + C);
    uint64_t* bar = reinterpret_cast<uint64_t*>(srec + G::CAP);
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    pdl_wait();
    if ((int)blockIdx.x >= *nwork) return;  // uniform for the whole CTA
    const int4 w = work[blockIdx.x];
    const int n = w.z - w.y;                 // 1..CAP (the scan splits larger units)
    const int tile = w.x >> 1, z0 = (w.x & 1) * 8;
    const int nbm = (1 << lnb) - 1;
    const int tx = tile & nbm, ty = (tile >> lnb) & nbm, tz = tile >> (2 * lnb);
    const int ox = tx * 16 - B::XA, oy = ty * 16 - 2, oz = tz * 16 + z0 - 2;
    if (!(ENUF_IN(tz, nbm + 1) && ENUF_IN(n - 1, G::CAP) && ENUF_IN(w.z - 1, N))) return;  // uniform for the CTA
    if (!stage_unit_tma<1, BX, PY, PZ, C>(s, srec, bar, &tmap, rec + w.y, n, ox, oy, oz, M, fld, status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int a = lane & 7, ax = a < 6 ? a : 5;  // lanes 6, 7 read lane 5's cells with weight 0
    const RowsP6 rows(lane >> 3);
    // the lane's three runs: offsets of their first cells from the window's corner
    const int o0 = rows.b[0] * BX, o1 = (3 * PY + rows.b[1]) * BX, o2 = ((rows.h2 ? 3 * PY : 0) + rows.b[2]) * BX;
    for (int k = warp; k < n; k += 16) {
        const uint32_t oi = perm[w.y + k];
        const f4 r = srec[k];
        int ix, iy, iz;
        float dx, dy, dz;
        split_offset<float, 16>(r.x, ix, dx);
        split_offset<float, 16>(r.y, iy, dy);
        split_offset<float, 16>(r.z, iz, dz);
        iz -= z0;
        if (!(ENUF_IN(ix, 16) && ENUF_IN(iy, 16) && ENUF_IN(iz, 8))) continue;  // uniform for the warp
        const float ux = dx + (float)(2 - ax);
        const float wx = a < 6 ? win_exp(ux * ux, wc) : 0.f;
        const float* base = s + (iz * PY + iy) * BX + ix + XOFF + ax;
        float wz[6];
        window_weights<float, 6>(dz, wc, wz);
        float sk[3] = {0.f, 0.f, 0.f}, dk[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; j++) {
            // planes j (runs with h = 0) and 3 + j (h = 1); u_z = dz + 2 - c
            const float z2w = rows.h2 ? wz[3 + j] : wz[j];
            const float u0 = dz + (float)(2 - j), u1 = dz - (float)(1 + j), u2 = rows.h2 ? u1 : u0;
            const float v0 = base[o0 + j * PY * BX], v1 = base[o1 + j * PY * BX], v2 = base[o2 + j * PY * BX];
            sk[0] = fmaf(wz[j], v0, sk[0]);
            dk[0] = fmaf(wz[j] * u0, v0, dk[0]);
            sk[1] = fmaf(wz[3 + j], v1, sk[1]);
            dk[1] = fmaf(wz[3 + j] * u1, v1, dk[1]);
            sk[2] = fmaf(z2w, v2, sk[2]);
            dk[2] = fmaf(z2w * u2, v2, dk[2]);
        }
        float ss = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const float uy = dy + (float)(2 - rows.b[q]);
            const float wy = win_exp(uy * uy, wc);
            ss = fmaf(wy, sk[q], ss);
            sy = fmaf(wy * uy, sk[q], sy);
            sz = fmaf(wy, dk[q], sz);
        }
        // (s, g_x, g_y, g_z) partials of this lane; lane 8 f holds total f
        float acc[4] = {wx * ss, 0.f, wx * sy, wx * sz};
        acc[1] = ux * acc[0];
        const float tot = warp_sum4(acc, lane);
        if ((lane & 7) == 0 && ENUF_IN(oi, N)) {
            const int f = lane >> 3;
            if (f == 0) {
                if (phi) phi[oi] = cnorm3 * tot;
            } else if (F) {
                F[3 * (size_t)oi + f - 1] = r.w * (f == 1 ? fa0 : (f == 2 ? fa1 : fa2)) * tot;
            }
        }
    }
}

// Interpolation without staging, for grids whose field planes stay resident
// in L2 (the whole set is at most a few tens of MB): one group of G lanes per
// particle in sorted order, reading each window row of p consecutive cells
// straight from global memory (tile-sorted particles keep the reads of a CTA
// close together, so most hit in L1).
template <typename R, int P, int T, int NF>
__global__ void __launch_bounds__(256) k_gather_direct(int N, const typename Rec<R>::T* __restrict__ rec,
                                                       const uint32_t* __restrict__ tile_of,
                                                       const uint32_t* __restrict__ perm, int M, int lnbx, int lnby,
                                                       WinC<R> wc, R cnorm3, const R* __restrict__ fld,
                                                       R* __restrict__ F, R* __restrict__ phi)
{
    constexpr int m = P / 2, G = GroupOf<P>::G;
    pdl_wait();
    const int lane = threadIdx.x % G;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (j >= N) return;  // whole groups leave together
    const unsigned gmask = (G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G)));
    const int M3 = M * M * M;  // < 2^31 for M <= 512
    const int mask = M - 1;
    const typename Rec<R>::T r = rec[j];
    const int tile = (int)tile_of[j];
    const int tx = tile & ((1 << lnbx) - 1), ty = (tile >> lnbx) & ((1 << lnby) - 1), tz = tile >> (lnbx + lnby);
    int ix, iy, iz;
    R dx, dy, dz;
    split_offset<R, T>(r.x, ix, dx);
    split_offset<R, T>(r.y, iy, dy);
    split_offset<R, T>(r.z, iz, dz);
    if (!(ENUF_IN(tz, M / T) && ENUF_IN(perm[j], N))) return;  // whole groups leave together
    R wy[P], wz[P];
    window_weights<R, P>(dy, wc, wy);
    window_weights<R, P>(dz, wc, wz);
    R acc[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) acc[f] = R(0);
    if (lane < P) {
        R u = dx + (R)(m - 1 - lane);
        const R wx = win_exp(u * u, wc);
        const int gx = (tx * T + ix - (m - 1) + lane) & mask;
        const int y0 = ty * T + iy - (m - 1), z0 = tz * T + iz - (m - 1);
        int yo[P];
#pragma unroll
        for (int b = 0; b < P; b++) yo[b] = ((y0 + b) & mask) * M;
#pragma unroll
        for (int c = 0; c < P; c++) {
            const R wxz = wx * wz[c];
            const R* zb = fld + (((z0 + c) & mask) * M * M + gx);
#pragma unroll
            for (int b = 0; b < P; b++) {
                const R ww = wxz * wy[b];
#pragma unroll
                for (int f = 0; f < NF; f++) acc[f] += ww * __ldg(zb + f * M3 + yo[b]);
            }
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int f = 0; f < NF; f++) acc[f] += __shfl_xor_sync(gmask, acc[f], o, G);
    }
    if (lane == 0) {
        const uint32_t oi = perm[j];
        if (F) {
            const R qc = r.w * cnorm3;
            F[3 * (size_t)oi] = qc * acc[0];
            F[3 * (size_t)oi + 1] = qc * acc[1];
            F[3 * (size_t)oi + 2] = qc * acc[2];
        }
        if (NF == 4 && phi) phi[oi] = cnorm3 * acc[NF - 1];
    }
}

// The analytic-differentiation interpolation without staging (same
// selection rule as k_gather_direct): one group of G lanes per particle,
// lane a < P the x offset a; the row sums over y carry the weights wy and
// u_y wy, the plane sums over z the weights wz and u_z wz.
template <typename R, int P, int T>
__global__ void __launch_bounds__(256) k_gather_direct_ad(int N, const typename Rec<R>::T* __restrict__ rec,
                                                          const uint32_t* __restrict__ tile_of,
                                                          const uint32_t* __restrict__ perm, int M, int lnbx,
                                                          int lnby, WinC<R> wc, R cnorm3, R fa0, R fa1, R fa2,
                                                          const R* __restrict__ fld, R* __restrict__ F,
                                                          R* __restrict__ phi)
{
    constexpr int m = P / 2, G = GroupOf<P>::G;
    pdl_wait();
    const int lane = threadIdx.x % G;
    const int j = (blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (j >= N) return;  // whole groups leave together
    const unsigned gmask = (G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) / G * G)));
    const int mask = M - 1;
    const typename Rec<R>::T r = rec[j];
    const int tile = (int)tile_of[j];
    const int tx = tile & ((1 << lnbx) - 1), ty = (tile >> lnbx) & ((1 << lnby) - 1), tz = tile >> (lnbx + lnby);
    int ix, iy, iz;
    R dx, dy, dz;
    split_offset<R, T>(r.x, ix, dx);
    split_offset<R, T>(r.y, iy, dy);
    split_offset<R, T>(r.z, iz, dz);
    if (!(ENUF_IN(tz, M / T) && ENUF_IN(perm[j], N))) return;  // whole groups leave together
    R wy[P], wz[P];
    window_weights<R, P>(dy, wc, wy);
    window_weights<R, P>(dz, wc, wz);
    R acc[4] = {R(0), R(0), R(0), R(0)};
    if (lane < P) {
        const R ux = dx + (R)(m - 1 - lane);
        const R wx = win_exp(ux * ux, wc);
        const int gx = (tx * T + ix - (m - 1) + lane) & mask;
        const int y0 = ty * T + iy - (m - 1), z0 = tz * T + iz - (m - 1);
        int yo[P];
#pragma unroll
        for (int b = 0; b < P; b++) yo[b] = ((y0 + b) & mask) * M;
        R sa = R(0), sy = R(0), sz = R(0);
#pragma unroll
        for (int c = 0; c < P; c++) {
            const R* zb = fld + (((z0 + c) & mask) * M * M + gx);
            R rs = R(0), ry = R(0);
#pragma unroll
            for (int b = 0; b < P; b++) {
                const R v = __ldg(zb + yo[b]);
                rs += wy[b] * v;
                ry += wy[b] * (dy + (R)(m - 1 - b)) * v;
            }
            sa += wz[c] * rs;
            sy += wz[c] * ry;
            sz += wz[c] * (dz + (R)(m - 1 - c)) * rs;
        }
        acc[0] = wx * sa;
        acc[1] = ux * acc[0];
        acc[2] = wx * sy;
        acc[3] = wx * sz;
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
#pragma unroll
        for (int f = 0; f < 4; f++) acc[f] += __shfl_xor_sync(gmask, acc[f], o, G);
    }
    if (lane == 0) {
        const uint32_t oi = perm[j];
        if (F) {
            F[3 * (size_t)oi] = r.w * fa0 * acc[1];
            F[3 * (size_t)oi + 1] = r.w * fa1 * acc[2];
            F[3 * (size_t)oi + 2] = r.w * fa2 * acc[3];
        }
        if (phi) phi[oi] = cnorm3 * acc[0];
    }
}

}  // namespace enuf
