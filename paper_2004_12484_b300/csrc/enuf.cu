// enuf.cu -- host side of the ENUF library: parameter checks, workspace
// layout, window / twiddle / reciprocal tables, the launch sequence of one
// evaluation, CUDA-graph replay, and the C ABI declared in include/enuf.h.
//
// One evaluation (Sec. 3.1-3.2 of the paper, everything on the device):
//   bin keys -> scan -> scatter        counting sort into grid tiles (a1, a2)
//   spread                             window spreading (a3)
//   fx, fy, fz                         forward FFT; fz fuses scaling, the
//                                      energy/virial (Eq. 38) and subdividing
//   iy, ix                             inverse FFT of 3 or 4 fields packed
//                                      into one pass (a6)
//   gather                             interpolation, F = q E (a7)
//   real-space sort + pair kernel      erfc sum (a8)
//   finalize                           FP64 assembly of E and the virial (a9)
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/enuf.h"
#include "common.cuh"
#include "fft.cuh"
#include "realspace.cuh"
#include "sort.cuh"
#include "md.cuh"
#include "spread_gather.cuh"

using namespace enuf;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

// On a CUDA error: clear the runtime's pending (non-sticky) error so that
// later, unrelated launch checks do not see it, and report it.
#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) {                                                              \
            cudaGetLastError();                                                               \
            return fail(ENUF_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
        }                                                                                     \
    } while (0)

constexpr int kWorkCap = 512;    // particles per work item of the interpolation (a tile)
constexpr int kSpreadCap = 128;  // particles per work item of the spreading (a sub-tile)
constexpr int kMaxSmem = 227 * 1024;
constexpr double kPi = 3.14159265358979323846;

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Resolved {
    enuf_params prm;
    bool fp64;
    size_t rsz;    // sizeof(real)
    int nc, Kx, Kb, P;
    int T, nbt[3], ntiles, max_work;  // tiles of T^3 cells, interpolation work items
    // interpolation work units: z-halves of the 16-cell tiles (zhalf), the
    // sub-tile bins per unit (ggroup) and particles per work item (gcap)
    bool zhalf;
    int ggroup, gcap;
    int S, lr, nbins, max_work2;      // sub-tiles of S^3 (the sort's bins), lr = log2(T/S), spreading items
    bool cells;    // linked cells (else all pairs)
    int ncell[3], nrbins;
    int sr;        // stencil radius of the linked cells: 2 (edge >= r_c / 2) or 1 (edge >= r_c)
    double h[3];
    FftGeom gfx, gy, gz;
    int fxy_threads;  // > 0: fused x-y kernels, k_fxy with this block size
    int iyx_threads;  // and k_iyx with this one
    size_t fxy_smem, iyx_smem;
    bool gather_direct;  // interpolate straight from L2-resident field planes
    bool fz_wide;        // the z pass is k_fzw (M = 512)
};

int ffthreads(int n) { return n >= 8 ? n / 8 : 1; }
// threads per row of the x-row kernels k_fx, k_ix (radix RowMR of fft.cuh)
int rowthreads(int mh) { return mh == 256 ? mh / 16 : ffthreads(mh); }
// threads of one transform of n points in k_fxy / k_iyx of an M grid (the
// radix of XyMR) and their largest block (XyBounds)
int xythreads(bool fp64, int n, int M, bool inv)
{
    const bool r16 = !fp64 && (n == 256 || (n == 128 && (M == 256 || inv)));
    return r16 ? n / 16 : ffthreads(n);
}
int xy_max_threads(bool fp64, int M, bool inv)
{
    if (fp64) return XyBounds<double, 512, false>::T;
    if (M == 256) return XyBounds<float, 256, false>::T;
    if (M == 128) return inv ? XyBounds<float, 128, true>::T : XyBounds<float, 128, false>::T;
    return XyBounds<float, 64, false>::T;
}
// slots of one transform of length n in shared memory (PadLen in fft.cuh)
int padlen(int n) { return n + n / 16; }

int resolve(const enuf_params* in, Resolved& r)
{
    if (!in) return fail(ENUF_EINVAL, "params is NULL");
    r.prm = *in;
    enuf_params& p = r.prm;
    for (int t = 0; t < 3; t++)
        if (!(p.L[t] > 0.0) || !std::isfinite(p.L[t])) return fail(ENUF_EINVAL, "box edges must be positive");
    if (p.N < 1 || p.N >= (int64_t(1) << 31)) return fail(ENUF_EINVAL, "N must be in [1, 2^31)");
    if (!(p.alpha > 0.0)) return fail(ENUF_EINVAL, "alpha must be positive");
    if (!is_pow2(p.M) || p.M < 8 || p.M > 512) return fail(ENUF_EUNSUPPORTED, "M must be a power of two in [8, 512]");
    if (p.p < 2 || p.p > 12 || (p.p & 1) || p.p > p.M) return fail(ENUF_EUNSUPPORTED, "p must be even, 2..12, <= M");
    if (p.n_c == 0) p.n_c = p.M / 4;
    if (p.n_c < 1 || 2 * p.n_c >= p.M) return fail(ENUF_EINVAL, "n_c must satisfy 1 <= n_c < M/2");
    if (p.precision != ENUF_FP64 && p.precision != ENUF_MIXED) return fail(ENUF_EINVAL, "unknown precision");
    if (p.coulomb_k == 0.0) p.coulomb_k = 1.0;
    if (p.flags != 0) return fail(ENUF_EINVAL, "params.flags is reserved and must be 0");
    if (!(p.slater_lambda >= 0.0) || !std::isfinite(p.slater_lambda))
        return fail(ENUF_EINVAL, "slater_lambda must be finite and >= 0");
    const double Lmin = std::min(p.L[0], std::min(p.L[1], p.L[2]));
    if (!(p.r_c > 0.0) || p.r_c > 0.5 * Lmin) return fail(ENUF_EINVAL, "r_c must satisfy 0 < r_c <= min(L)/2");

    r.fp64 = p.precision == ENUF_FP64;
    r.rsz = r.fp64 ? 8 : 4;
    r.nc = p.n_c;
    r.Kx = r.nc + 1;
    r.Kb = 2 * r.nc + 1;
    r.P = r.Kb * r.Kx;
    // tile edge: 16 for float grids of edge >= 128, else 8, else 4 -- the
    // largest for which the interpolation box of 4 fields fits in shared
    // memory (the same box geometry as Box<P, T> in spread_gather.cuh)
    auto box_bytes = [&](int T) {
        const int m = p.p / 2, XA = (m - 1 + 3) / 4 * 4, BX = (XA + T + m + 3) / 4 * 4, PT = T + p.p - 1;
        return ((size_t)BX * PT * PT * 4 + (size_t)32 * p.p * p.p) * r.rsz + (size_t)kWorkCap * (4 * r.rsz + 4);
    };
    // windows of p <= 4 interpolate faster straight from L2-resident fields
    // (8-cell tiles) than from a staged 16-cell box; p = 6 and 8 have a
    // TMA-staged interpolation of their own on 16-cell tiles
    const bool fields_in_l2 = (size_t)4 * p.M * p.M * p.M * r.rsz <= (size_t)64 << 20;
    r.T = (!r.fp64 && p.M >= 128 && !(p.p <= 4 && fields_in_l2)) ? 16 : 8;
    if (const char* tv = std::getenv("ENUF_TILE")) {  // tuning knob: tile edge 4, 8 or 16
        const int t = std::atoi(tv);
        if ((t == 4 || t == 8 || t == 16) && t <= p.M) r.T = t;
    }
    while (r.T > 4 && box_bytes(r.T) > (size_t)kMaxSmem) r.T /= 2;
    if (box_bytes(r.T) > (size_t)kMaxSmem) return fail(ENUF_EUNSUPPORTED, "window too wide for the tile box");
    for (int t = 0; t < 3; t++) r.nbt[t] = p.M / r.T;
    r.ntiles = r.nbt[0] * r.nbt[1] * r.nbt[2];
    r.S = std::min(r.T, 8);
    r.lr = r.T / r.S == 2 ? 1 : 0;
    // 16-cell tiles interpolate in z-halves (sub-tiles 0-3 and 4-7 of a tile,
    // each a contiguous particle range): two CTAs share an SM
    r.zhalf = r.lr == 1 && !std::getenv("ENUF_GATHER_FULL_TILE");
    r.ggroup = r.lr ? (r.zhalf ? 4 : 8) : 1;
    r.gcap = r.zhalf ? kWorkCap / 2 : kWorkCap;
    r.max_work = (r.zhalf ? 2 : 1) * r.ntiles + (int)(p.N / r.gcap) + 1;
    r.nbins = r.ntiles << (3 * r.lr);
    r.max_work2 = (int)std::min<int64_t>(r.nbins, p.N) + (int)(p.N / kSpreadCap) + 1;
    // linked cells of edge >= r_c, at least 3 per dimension
    // linked cells of edge >= r_c / 2 with a 5^3 stencil where every
    // dimension holds at least 5 of them (the stencil's volume is 15.6 r_c^3
    // instead of 27 r_c^3), else of edge >= r_c with 3^3
    r.cells = true;
    r.sr = 2;
    for (int t = 0; t < 3; t++)
        if ((int)std::floor(2.0 * p.L[t] / p.r_c) < 5 || std::getenv("ENUF_CELL_STENCIL3")) r.sr = 1;
    for (int t = 0; t < 3; t++) {
        r.ncell[t] = (int)std::floor(r.sr * p.L[t] / p.r_c);
        if (r.ncell[t] > 256) r.ncell[t] = 256;
        if (r.ncell[t] < 2 * r.sr + 1) r.cells = false;
    }
    if (!r.cells) r.ncell[0] = r.ncell[1] = r.ncell[2] = 1;
    for (int t = 0; t < 3; t++) r.h[t] = p.L[t] / r.ncell[t];
    r.nrbins = r.ncell[0] * r.ncell[1] * r.ncell[2];

    const size_t vsz = 2 * r.rsz;
    const int M = p.M;
    // k_fx / k_ix rows per block
    r.gfx = FftGeom{r.nc, r.Kx, r.Kb, r.P, 0, 256 / rowthreads(M / 2)};
    const int NT = ffthreads(M), gran = std::max(1, 32 / NT);
    auto round_up = [](int v, int g) { return (v + g - 1) / g * g; };
    // k_fy / k_iy: columns per block, about 16 but balanced over Kx (about 8
    // at M = 512, where 16 columns of 64 threads made one CTA of 960 threads
    // an SM by registers)
    {
        const int cw = M >= 512 ? 8 : 16;
        int nch = (r.Kx + cw - 1) / cw;
        int W = round_up((r.Kx + nch - 1) / nch, gran);
        while (W * NT > (M >= 512 ? 512 : 1024)) W -= gran;  // the launch bounds of k_fy / k_iy
        while ((size_t)(W * (padlen(M) + 1) + M) * vsz > (size_t)kMaxSmem) W -= gran;
        r.gy = FftGeom{r.nc, r.Kx, r.Kb, r.P, W, 0};
    }
    // k_fzw for M = 512: 8 pencils a CTA of 8 M/8 threads, one buffer per
    // pencil (two CTAs an SM: 0.293 ms at the ionic-liquid size against
    // 0.307 with 16 pencils in one CTA of 1024 threads)
    r.fz_wide = (M >= 512 || ((M == 128 || M == 256) && !r.fp64)) && !std::getenv("ENUF_FZ_NARROW");
    if (r.fz_wide) {
        // at 128 and 256 (single precision) 16 pencils: polyelectrolyte z
        // pass 0.0573 -> 0.0368 ms against k_fz (0.0389 with 8 pencils); RPM
        // step 0.1065 -> 0.1048 ms (8 pencils: no change)
        int W = (M == 128 || M == 256) ? 16 : 8;
        if (const char* wv = std::getenv("ENUF_FZ_W")) {  // tuning knob: 4, 8 or 16 pencils a CTA
            const int w = std::atoi(wv);
            if (w == 4 || w == 8 || (w == 16 && !r.fp64)) W = w;
        }
        r.gz = FftGeom{r.nc, r.Kx, r.Kb, r.P, W, 0};
    } else
    // k_fz: pencils per block (at most 512 threads: the batched inverse
    // transforms of four fields need up to 128 registers per thread); its
    // passes use radix 4, so M/4 threads serve one pencil
    {
        const int NTZ = M >= 4 ? M / 4 : 1, granz = std::max(1, 32 / NTZ);
        // 8 pencils a CTA: at M = 128 the 2145 pencils make 269 CTAs of 256
        // threads, so every SM works (0.1271 against 0.1274 ms a step with 16)
        int W = round_up(8, granz);
        if (const char* wv = std::getenv("ENUF_FZ_W")) {  // tuning knob: pencils per CTA of the z pass
            const int w = std::atoi(wv);
            if (w >= 1 && w <= 64) W = round_up(w, granz);
        }
        while (W * NTZ > 512) W -= granz;
        while ((size_t)(4 * W * (padlen(M) + 1) + M) * vsz + 32 * 7 * 8 + (size_t)9 * r.Kb * r.rsz > (size_t)kMaxSmem)
            W -= granz;
        r.gz = FftGeom{r.nc, r.Kx, r.Kb, r.P, W, 0};
    }
    if (r.gy.W < 1 || r.gz.W < 1) return fail(ENUF_EUNSUPPORTED, "FFT block shape does not fit");
    // the four field planes stay in L2 (126 MB) when they total <= 64 MB
    r.gather_direct = r.T < 16 && r.lr == 0 && (size_t)4 * M * M * M * r.rsz <= (size_t)64 << 20 && !std::getenv("ENUF_STAGED_GATHER");
    // fused x-y passes (one CTA per z-plane) where the pruned plane fits:
    // the kept kx columns are transformed in as few batches as the 1024-thread
    // limit allows, each batch CB columns wide with no idle column slots;
    // the rows then go through in batches of blockDim / NTX
    r.fxy_threads = r.iyx_threads = 0;
    r.fxy_smem = r.iyx_smem = 0;
    if (M >= 32 && M <= 256) {
        for (int inv = 0; inv < 2; inv++) {
            const int NTX = xythreads(r.fp64, M / 2, M, inv), NTY = xythreads(r.fp64, M, M, inv);
            const int tmax = xy_max_threads(r.fp64, M, inv);
            for (int nbatch = (r.Kx * NTY + tmax - 1) / tmax; nbatch <= r.Kx; nbatch++) {
                const int CB = (r.Kx + nbatch - 1) / nbatch, t = CB * NTY;
                if (t > tmax || t % NTX) continue;
                const int RB = t / NTX, KxR = (r.Kx + CB - 1) / CB * CB;
                const size_t sm = ((size_t)RB * padlen(M / 2) + (size_t)KxR * (padlen(M) + 1) + M) * vsz;
                if (sm <= (size_t)kMaxSmem) {
                    (inv ? r.iyx_threads : r.fxy_threads) = t;
                    (inv ? r.iyx_smem : r.fxy_smem) = sm;
                    break;
                }
            }
        }
        if (!r.fxy_threads || !r.iyx_threads) r.fxy_threads = r.iyx_threads = 0;
    }
    // launch-time divisors of the FFT kernels' index arithmetic
    for (FftGeom* gm : {&r.gfx, &r.gy, &r.gz}) {
        gm->fKx = FDiv::make((uint32_t)r.Kx);
        gm->fW = FDiv::make((uint32_t)std::max(1, gm->W));
        gm->fKxR = FDiv::make(1);
    }
    if (r.iyx_threads > 0) {
        const int CB = r.iyx_threads / xythreads(r.fp64, M, M, true);
        r.gy.fKxR = FDiv::make((uint32_t)((r.Kx + CB - 1) / CB * CB));
    }
    return ENUF_OK;
}

// ------------------------------------------------------------------ workspace
struct Layout {
    size_t status, out, mean, md_step;
    size_t counts, offsets, work, nwork, work2, nwork2, item2;
    size_t csum_g, cbase_g, csum_r, cbase_r;  // chunk totals / bases of the chunked scans
    size_t key, rank, rec_tmp, rec, perm, tile_of;
    size_t rcounts, roffsets, rrec, rperm, rcell;
    size_t rkey, rrank, rrec_tmp, Fr, phir;  // real-space sort scratch and outputs
    size_t qpart, kpart, rpart, fpart, fscratch;
    size_t twid, tk, te, td;
    size_t grid, C1, C2, C3, C4, fld;
    size_t s_pos, s_q, s_F, s_phi;
    size_t total;
};

// Word stride of the bin counters: with few bins, one 128-byte line each
// (the particles' atomics spread over many L2 lines), one 32-byte sector
// each up to 8192 bins, packed beyond.
int count_stride(int nbins) { return nbins <= 1024 ? 32 : (nbins <= 8192 ? 8 : 1); }

Layout layout(const Resolved& r)
{
    Layout L{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + std::max<size_t>(bytes, 1));
        return at;
    };
    const size_t N = (size_t)r.prm.N, M = (size_t)r.prm.M, rs = r.rsz, vs = 2 * r.rsz;
    const size_t recsz = r.fp64 ? sizeof(d4) : sizeof(f4);
    const size_t nblkN = (N + 255) / 256;
    const size_t nblkZ = ((size_t)r.P + r.gz.W - 1) / r.gz.W;
    L.status = take(16);  // status word; at +4 the assembly's block counter, at +8 and +12 those of the two sorts
    L.out = take(ENUF_NOUT * 8);
    L.mean = take(4 * 8);
    L.md_step = take(16);  // step counter of the time-stepping harness
    L.counts = take((size_t)(r.nbins + 1) * 4 * count_stride(r.nbins));
    L.offsets = take((r.nbins + 1) * 4);
    L.work = take((size_t)r.max_work * 16);
    L.nwork = take(4);
    L.work2 = take((size_t)r.max_work2 * 16);
    L.nwork2 = take(4);
    L.item2 = take((size_t)r.nbins * 4);
    const size_t nchg = (size_t)(r.nbins + kScanChunk - 1) / kScanChunk, nchr = (size_t)(r.nrbins + kScanChunk - 1) / kScanChunk;
    L.csum_g = take(nchg * 12);
    L.cbase_g = take(nchg * 12);
    L.csum_r = take(nchr * 12);
    L.cbase_r = take(nchr * 12);
    L.key = take(N * 4);
    L.rank = take(N * 4);
    L.rec_tmp = take(N * recsz);
    L.rec = take(N * recsz);
    L.perm = take(N * 4);
    L.tile_of = take(N * 4);
    L.rcounts = take((size_t)(r.nrbins + 1) * 4 * count_stride(r.nrbins));
    L.roffsets = take((r.nrbins + 1) * 4);
    L.rrec = take(N * recsz);
    L.rperm = take(N * 4);
    L.rcell = take(N * 4);
    L.rkey = take(N * 4);
    L.rrank = take(N * 4);
    L.rrec_tmp = take(N * recsz);
    L.Fr = take(3 * N * rs);
    L.phir = take(N * rs);
    L.qpart = take(nblkN * 2 * 8);
    L.kpart = take(nblkZ * 8 * 8);
    L.rpart = take(nblkN * 5 * 8 * 8);  // up to 5 stencil layers of blocks
    L.fpart = take(nblkN * 4 * 8);
    L.fscratch = take(64 * 16 * 8);  // assembly: 16 sums per block, at most 64 blocks
    L.twid = take(M * vs);
    L.tk = take(3 * r.Kb * rs);
    L.te = take(3 * r.Kb * rs);
    L.td = take(3 * r.Kb * rs);
    L.grid = take(M * M * M * rs);
    L.C1 = take(M * M * r.Kx * vs);
    L.C2 = take(M * (size_t)r.P * vs);
    L.C3 = take(4 * M * (size_t)r.P * vs);
    L.C4 = take(4 * M * M * r.Kx * vs);
    L.fld = take(4 * M * M * M * rs);
    L.s_pos = take(3 * N * rs);
    L.s_q = take(N * rs);
    L.s_F = take(3 * N * rs);
    L.s_phi = take(N * rs);
    L.total = o;
    return L;
}

struct GraphEntry {
    const void *pos, *q;
    void *F, *phi;
    double* out;
    int flags;
    cudaGraphExec_t exec;
    unsigned long long stamp;
};

}  // namespace

struct enuf_plan {
    Resolved r;
    Layout lay;
    char* ws = nullptr;
    bool own_ws = false;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t aux_stream = nullptr;  // side branch (assembly beside the interpolation)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    double* hout = nullptr;  // pinned host copy of the results (host-buffer entry point)
    bool use_graph = true;
    bool profile = false;
    bool pdl = true;  // programmatic dependent launch along the chain (ENUF_NO_PDL=1 turns it off)
    bool legacy_gather = false;  // ENUF_LEGACY_GATHER=1: the generic interpolation kernel for p = 8 and 6 as well
    bool gather_tma = false;     // k_gather_p8 / k_gather_p6 serve the interpolation (its tensor map is set)
    CUtensorMap fld_tmap;        // the field planes, for the TMA boxes of k_gather_p8 / k_gather_p6
    bool attrs_done = false;
    std::vector<GraphEntry> graphs;
    // one time step of the harness (enuf_md_run) as a graph, for one set of
    // buffers, flags and step
    struct {
        const void *pos, *vel, *q, *inv_mass, *F;
        double* energies;
        int flags, cap;
        double dt;
        cudaGraphExec_t exec = nullptr;
    } md;
    unsigned long long stamp = 0;
    // derived constants
    double b = 0, inv_b = 0, cnorm3 = 0;
    int lnb = 0;  // log2 of tiles per dimension
    // profiling
    std::vector<std::string> tnames;
    std::vector<cudaEvent_t> tevents;
    std::vector<float> ttimes;
    cudaGraphExec_t prof_exec = nullptr;
};

namespace {

template <typename T> T* at(enuf_plan* pl, size_t off) { return reinterpret_cast<T*>(pl->ws + off); }

// Window constants for the kernels: 1/b, log2(e)/b and exp(-a^2/b), a < 16
// (computed in double on the host, rounded to the kernel's type).
template <typename R> WinC<R> winc(const enuf_plan* pl)
{
    WinC<R> w{};
    w.inv_b = (R)pl->inv_b;
    w.l2b = (R)(pl->inv_b / std::log(2.0));
    for (int a = 0; a < 16; a++) w.c[a] = (R)std::exp(-(double)a * a * pl->inv_b);
    return w;
}

// ------------------------------------------------------------------ launching
// Kernels that begin with pdl_wait() and may therefore be
// launched with programmatic stream serialisation.
inline bool pdl_kernel(const char* name)
{
    static const char* const names[] = {"bin_keys", "real_bin_keys", "scatter", "real_scatter", "spread",
                                        "fft_xy", "fft_z_kspace", "ifft_yx", "gather", "finalize"};
    for (const char* n : names)
        if (std::strcmp(n, name) == 0) return true;
    return false;
}

struct Launcher {
    enuf_plan* pl;
    cudaStream_t st;
    bool attr_only;
    int count = 0;

    template <typename... KArgs, typename... Args>
    int go(const char* name, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, Args... args)
    {
        if (smem > 48 * 1024 && attr_only) {
            cudaError_t e = cudaFuncSetAttribute((const void*)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return fail(ENUF_ECUDA, std::string("cudaFuncSetAttribute(") + name + "): " + cudaGetErrorString(e));
        }
        if (attr_only) { count++; return ENUF_OK; }
        if (pl->profile && pl->tnames.size() + 1 < pl->tevents.size()) {
            CK(cudaEventRecordWithFlags(pl->tevents[pl->tnames.size()], st, cudaEventRecordExternal));
            pl->tnames.push_back(name);
        }
        cudaError_t e;
        if (pl->pdl && pdl_kernel(name)) {
            // may start while the previous kernel on the stream finishes; the
            // kernel waits for it (pdl_wait) before using its data
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = grid;
            cfg.blockDim = block;
            cfg.dynamicSmemBytes = smem;
            cfg.stream = st;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
            if (e == cudaSuccess) e = cudaGetLastError();
        } else {
            k<<<grid, block, smem, st>>>(args...);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) return fail(ENUF_ECUDA, std::string("launch ") + name + ": " + cudaGetErrorString(e));
        count++;
        return ENUF_OK;
    }
};

#define LCHK(x)                      \
    do {                             \
        int rc_ = (x);               \
        if (rc_ != ENUF_OK) return rc_; \
    } while (0)

template <typename R, int P, int T>
int launch_spread_t(Launcher& L, enuf_plan* pl)
{
    const Resolved& r = pl->r;
    const Layout& y = pl->lay;
    constexpr int S = T < 8 ? T : 8;
    // the box and (widths without a register path) the weight-product table;
    // p = 8 needs no table, which lets 14 of its CTAs share an SM instead of 13
    return L.go("spread", k_spread<R, P, T>, dim3(r.max_work2), dim3(32),
                (size_t)(SBox<P, S>::CELLS + WyzTable<P>::N) * sizeof(R), at<const int4>(pl, y.work2),
                at<const int>(pl, y.nwork2), at<const typename Rec<R>::T>(pl, y.rec), r.prm.M, pl->lnb, r.lr,
                winc<R>(pl), (R)pl->cnorm3, at<R>(pl, y.grid), (int)r.prm.N);
}

template <typename R, int P, int T>
int launch_gather_t(Launcher& L, enuf_plan* pl, int nf, R* F, R* phi)
{
    const Resolved& r = pl->r;
    const Layout& y = pl->lay;
    if (r.gather_direct) {
        constexpr int G = GroupOf<P>::G;
        const int N = (int)r.prm.N;
        const dim3 grid((unsigned)(((size_t)N * G + 255) / 256));
        if (nf == 4)
            return L.go("gather", k_gather_direct<R, P, T, 4>, grid, dim3(256), 0, N,
                        at<const typename Rec<R>::T>(pl, y.rec), at<const uint32_t>(pl, y.tile_of),
                        at<const uint32_t>(pl, y.perm), r.prm.M, pl->lnb, pl->lnb, winc<R>(pl), (R)pl->cnorm3,
                        at<const R>(pl, y.fld), F, phi);
        return L.go("gather", k_gather_direct<R, P, T, 3>, grid, dim3(256), 0, N,
                    at<const typename Rec<R>::T>(pl, y.rec), at<const uint32_t>(pl, y.tile_of),
                    at<const uint32_t>(pl, y.perm), r.prm.M, pl->lnb, pl->lnb, winc<R>(pl), (R)pl->cnorm3,
                    at<const R>(pl, y.fld), F, phi);
    }
    using RecT = typename Rec<R>::T;
    if constexpr (T == 16 && (P == 8 || P == 6) && sizeof(R) == 4) {
        if (pl->gather_tma) {
            // p = 8 and 6 in single precision: boxes staged by the TMA
            // engine, z-accumulated window rows
            int* st = at<int>(pl, y.status);
            auto go = [&](auto kern, size_t smem) {
                return L.go("gather", kern, dim3(r.max_work), dim3(512), smem, at<const int4>(pl, y.work),
                            at<const int>(pl, y.nwork), at<const f4>(pl, y.rec), at<const uint32_t>(pl, y.perm),
                            r.prm.M, pl->lnb, winc<float>(pl), (float)pl->cnorm3, at<const float>(pl, y.fld),
                            pl->fld_tmap, (float*)F, (float*)phi, st, (int)r.prm.N);
            };
            if constexpr (P == 8) {
                if (nf == 4) return go(k_gather_p8<4>, GatherP8<4>::SMEM);
                return go(k_gather_p8<3>, GatherP8<3>::SMEM);
            } else {
                if (nf == 4) return go(k_gather_p6<4>, GatherP6<4>::SMEM);
                return go(k_gather_p6<3>, GatherP6<3>::SMEM);
            }
        }
    }
    if constexpr (T == 16) {
        if (r.zhalf) {
            // z-halves of the tiles, 512 threads: two CTAs (three-field boxes
            // of 99 KB) share an SM
            constexpr int NTH = 512, ZS = 8;
            const size_t smem = ((size_t)nf * Box<P, T, ZS>::CELLS + (NTH / 32) * WyzTable<P>::N) * sizeof(R) +
                                (size_t)r.gcap * (sizeof(RecT) + 4);
            if (nf == 4)
                return L.go("gather", k_gather<R, P, T, 4, NTH, ZS>, dim3(r.max_work), dim3(NTH), smem,
                            at<const int4>(pl, y.work), at<const int>(pl, y.nwork), at<const RecT>(pl, y.rec),
                            at<const uint32_t>(pl, y.perm), r.prm.M, pl->lnb, pl->lnb, winc<R>(pl), (R)pl->cnorm3,
                            at<const R>(pl, y.fld), F, phi, (int)r.prm.N);
            return L.go("gather", k_gather<R, P, T, 3, NTH, ZS>, dim3(r.max_work), dim3(NTH), smem,
                        at<const int4>(pl, y.work), at<const int>(pl, y.nwork), at<const RecT>(pl, y.rec),
                        at<const uint32_t>(pl, y.perm), r.prm.M, pl->lnb, pl->lnb, winc<R>(pl), (R)pl->cnorm3,
                        at<const R>(pl, y.fld), F, phi, (int)r.prm.N);
        }
    }
    // 1024 threads for whole 16-cell tiles (one CTA per SM holds the box),
    // 256 for the smaller tiles
    constexpr int NTH = T == 16 ? 1024 : 256;
    const size_t smem = ((size_t)nf * Box<P, T>::CELLS + (NTH / 32) * WyzTable<P>::N) * sizeof(R) +
                        (size_t)r.gcap * (sizeof(RecT) + 4);
    if (nf == 4)
        return L.go("gather", k_gather<R, P, T, 4, NTH>, dim3(r.max_work), dim3(NTH), smem, at<const int4>(pl, y.work),
                    at<const int>(pl, y.nwork), at<const typename Rec<R>::T>(pl, y.rec), at<const uint32_t>(pl, y.perm),
                    r.prm.M, pl->lnb, pl->lnb, winc<R>(pl), (R)pl->cnorm3, at<const R>(pl, y.fld), F, phi, (int)r.prm.N);
    return L.go("gather", k_gather<R, P, T, 3, NTH>, dim3(r.max_work), dim3(NTH), smem, at<const int4>(pl, y.work),
                at<const int>(pl, y.nwork), at<const typename Rec<R>::T>(pl, y.rec), at<const uint32_t>(pl, y.perm),
                r.prm.M, pl->lnb, pl->lnb, winc<R>(pl), (R)pl->cnorm3, at<const R>(pl, y.fld), F, phi, (int)r.prm.N);
}

// Interpolation of the potential grid with the window gradient (forces by
// analytic differentiation); k_gather_ad_p6 for p = 6 in single precision
// on 16-cell tiles, else k_gather_ad: 512 threads for the 16-cell
// tiles (the box of one grid lets several CTAs share an SM), 256 for the
// smaller tiles.
template <typename R, int P, int T>
int launch_gather_ad_t(Launcher& L, enuf_plan* pl, R* F, R* phi)
{
    const Resolved& r = pl->r;
    const Layout& y = pl->lay;
    const R cn = (R)pl->cnorm3;
    R fa[3];
    for (int t = 0; t < 3; t++) fa[t] = (R)(pl->cnorm3 * r.prm.M / r.prm.L[t] * 2.0 / pl->b);
    if (r.gather_direct) {
        constexpr int G = GroupOf<P>::G;
        const int N = (int)r.prm.N;
        const dim3 grid((unsigned)(((size_t)N * G + 255) / 256));
        return L.go("gather", k_gather_direct_ad<R, P, T>, grid, dim3(256), 0, N,
                    at<const typename Rec<R>::T>(pl, y.rec), at<const uint32_t>(pl, y.tile_of),
                    at<const uint32_t>(pl, y.perm), r.prm.M, pl->lnb, pl->lnb, winc<R>(pl), cn, fa[0], fa[1], fa[2],
                    at<const R>(pl, y.fld), F, phi);
    }
    if constexpr (T == 16 && P == 6 && sizeof(R) == 4) {
        if (pl->gather_tma) {
            // p = 6 in single precision: the potential's boxes staged by the
            // TMA engine, z-accumulated window runs
            return L.go("gather", k_gather_ad_p6, dim3(r.max_work), dim3(512), GatherP6<1>::SMEM,
                        at<const int4>(pl, y.work), at<const int>(pl, y.nwork), at<const f4>(pl, y.rec),
                        at<const uint32_t>(pl, y.perm), r.prm.M, pl->lnb, winc<float>(pl), (float)cn, (float)fa[0],
                        (float)fa[1], (float)fa[2], at<const float>(pl, y.fld), pl->fld_tmap, (float*)F, (float*)phi,
                        at<int>(pl, y.status), (int)r.prm.N);
        }
    }
    using RecT = typename Rec<R>::T;
    constexpr int NTH = T == 16 ? 512 : 256;
    if constexpr (T == 16) {
        if (r.zhalf) {  // the sort's work units are z-halves of the tiles
            constexpr int ZS = 8;
            const size_t smem = ((size_t)Box<P, T, ZS>::CELLS + (NTH / 32) * WyzTable<P>::N) * sizeof(R) +
                                (size_t)r.gcap * (sizeof(RecT) + 4);
            return L.go("gather", k_gather_ad<R, P, T, NTH, ZS>, dim3(r.max_work), dim3(NTH), smem,
                        at<const int4>(pl, y.work), at<const int>(pl, y.nwork), at<const RecT>(pl, y.rec),
                        at<const uint32_t>(pl, y.perm), r.prm.M, pl->lnb, pl->lnb, winc<R>(pl), cn, fa[0], fa[1],
                        fa[2], at<const R>(pl, y.fld), F, phi, (int)r.prm.N);
        }
    }
    const size_t smem = ((size_t)Box<P, T>::CELLS + (NTH / 32) * WyzTable<P>::N) * sizeof(R) +
                        (size_t)r.gcap * (sizeof(RecT) + 4);
    return L.go("gather", k_gather_ad<R, P, T, NTH>, dim3(r.max_work), dim3(NTH), smem, at<const int4>(pl, y.work),
                at<const int>(pl, y.nwork), at<const RecT>(pl, y.rec), at<const uint32_t>(pl, y.perm),
                r.prm.M, pl->lnb, pl->lnb, winc<R>(pl), cn, fa[0], fa[1], fa[2], at<const R>(pl, y.fld), F, phi, (int)r.prm.N);
}

#define DISPATCH_P(T_, FN, ...)                                           \
    switch (pl->r.prm.p) {                                                \
    case 2: return FN<R, 2, T_>(__VA_ARGS__);                             \
    case 4: return FN<R, 4, T_>(__VA_ARGS__);                             \
    case 6: return FN<R, 6, T_>(__VA_ARGS__);                             \
    case 8: return FN<R, 8, T_>(__VA_ARGS__);                             \
    case 10: return FN<R, 10, T_>(__VA_ARGS__);                           \
    case 12: return FN<R, 12, T_>(__VA_ARGS__);                           \
    default: return fail(ENUF_EUNSUPPORTED, "unsupported p");             \
    }

template <typename R> int launch_spread(Launcher& L, enuf_plan* pl)
{
    if (pl->r.T == 16) { DISPATCH_P(16, launch_spread_t, L, pl) }
    if (pl->r.T == 4) { DISPATCH_P(4, launch_spread_t, L, pl) }
    DISPATCH_P(8, launch_spread_t, L, pl)
}

template <typename R> int launch_gather(Launcher& L, enuf_plan* pl, int nf, R* F, R* phi)
{
    if (pl->r.T == 16) { DISPATCH_P(16, launch_gather_t, L, pl, nf, F, phi) }
    if (pl->r.T == 4) { DISPATCH_P(4, launch_gather_t, L, pl, nf, F, phi) }
    DISPATCH_P(8, launch_gather_t, L, pl, nf, F, phi)
}

template <typename R> int launch_gather_ad(Launcher& L, enuf_plan* pl, R* F, R* phi)
{
    if (pl->r.T == 16) { DISPATCH_P(16, launch_gather_ad_t, L, pl, F, phi) }
    if (pl->r.T == 4) { DISPATCH_P(4, launch_gather_ad_t, L, pl, F, phi) }
    DISPATCH_P(8, launch_gather_ad_t, L, pl, F, phi)
}

// The FFT chain of one evaluation: forward x and y, the z pass with the
// reciprocal-space step and the inverse z transforms of nf fields, inverse y
// and x.  With `spec` set, the chain stops after the forward z transform and
// writes the retained spectrum there instead (ghat, or S~ = D ghat when
// scale is 1; k_fz_spectrum).
template <typename R, int M>
int launch_fft_chain_m(Launcher& L, enuf_plan* pl, int nf, void* spec = nullptr, int scale = 0)
{
    using V = typename Cpx<R>::T;
    const Resolved& r = pl->r;
    const Layout& y = pl->lay;
    const V* W = at<const V>(pl, y.twid);
    const size_t vs = sizeof(V);
    const bool fused = r.fxy_threads > 0 && !std::getenv("ENUF_NO_FUSED_XY");
    if (fused) {
        LCHK(L.go("fft_xy", k_fxy<R, M>, dim3(M), dim3(r.fxy_threads), r.fxy_smem, at<R>(pl, y.grid),
                  at<V>(pl, y.C2), r.gy, W));
    }
    // forward x
    if (!fused) {
        const int NT = rowthreads(M / 2), rows = r.gfx.rows;
        const int nblk = (M * M + rows - 1) / rows;
        LCHK(L.go("fft_x", k_fx<R, M>, dim3(nblk), dim3(rows * NT), (size_t)(rows * padlen(M / 2) + M) * vs, at<R>(pl, y.grid),
                  at<V>(pl, y.C1), r.gfx, W));
    }
    const int NT = ffthreads(M);
    // forward y
    if (!fused) {
        const int Wc = r.gy.W;
        LCHK(L.go("fft_y", k_fy<R, M>, dim3((r.Kx + Wc - 1) / Wc, M), dim3(Wc * NT), (size_t)(Wc * (padlen(M) + 1) + M) * vs,
                  at<const V>(pl, y.C1), at<V>(pl, y.C2), r.gy, W));
    }
    if (spec) {
        // pencils per CTA of the spectrum pass (radix 4: M/4 threads a
        // pencil, at most 512 threads)
        FftGeom gs = r.gz;
        gs.W = std::max(1, std::min(gs.W, 512 / std::max(1, M / 4)));
        gs.fW = FDiv::make((uint32_t)gs.W);
        const int Wc = gs.W;
        const size_t smem = (size_t)(Wc * (padlen(M) + 1) + M) * vs;
        if (smem > 48 * 1024 && !L.attr_only) {
            cudaError_t e = cudaFuncSetAttribute((const void*)k_fz_spectrum<R, M>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return fail(ENUF_ECUDA, std::string("cudaFuncSetAttribute(fft_z_spectrum): ") +
                                                              cudaGetErrorString(e));
        }
        const int NTZ = M >= 4 ? M / 4 : 1;
        return L.go("fft_z_spectrum", k_fz_spectrum<R, M>, dim3((r.P + Wc - 1) / Wc), dim3(Wc * NTZ), smem,
                    at<const V>(pl, y.C2), reinterpret_cast<V*>(spec), gs, W, at<const R>(pl, y.td), scale);
    }
    // z + reciprocal-space step + inverse z
    bool wide_done = false;
    if constexpr (M >= 128) {
        if (r.fz_wide) {
        const int Wc = r.gz.W;
        const size_t smem = (size_t)(Wc * (padlen(M) + 1) + M) * vs + 32 * 7 * 8 + (size_t)9 * r.Kb * sizeof(R);
        KTables<R> kt;
        kt.tk = at<const R>(pl, y.tk);
        kt.te = at<const R>(pl, y.te);
        kt.td = at<const R>(pl, y.td);
        const double V3 = r.prm.L[0] * r.prm.L[1] * r.prm.L[2];
        kt.cE = (R)(r.prm.coulomb_k * 2.0 * kPi / V3);
        kt.cF = (R)(r.prm.coulomb_k * 4.0 * kPi / V3);
        kt.inv4a2 = (R)(1.0 / (4.0 * r.prm.alpha * r.prm.alpha));
        const dim3 g((r.P + Wc - 1) / Wc), b(Wc * (M / 8));
        if (nf == 0)
            LCHK(L.go("fft_z_kspace", k_fzw<R, M, 0>, g, b, smem, at<const V>(pl, y.C2), at<V>(pl, y.C3), r.gz, W, kt,
                      at<double>(pl, y.kpart)));
        else if (nf == 1)
            LCHK(L.go("fft_z_kspace", k_fzw<R, M, 1>, g, b, smem, at<const V>(pl, y.C2), at<V>(pl, y.C3), r.gz, W, kt,
                      at<double>(pl, y.kpart)));
        else if (nf == 3)
            LCHK(L.go("fft_z_kspace", k_fzw<R, M, 3>, g, b, smem, at<const V>(pl, y.C2), at<V>(pl, y.C3), r.gz, W, kt,
                      at<double>(pl, y.kpart)));
        else
            LCHK(L.go("fft_z_kspace", k_fzw<R, M, 4>, g, b, smem, at<const V>(pl, y.C2), at<V>(pl, y.C3), r.gz, W, kt,
                      at<double>(pl, y.kpart)));
        wide_done = true;
        }
    }
    if (!wide_done) {
        const int Wc = r.gz.W;
        const size_t smem = (size_t)(std::max(nf, 1) * Wc * (padlen(M) + 1) + M) * vs + 32 * 7 * 8 + (size_t)9 * r.Kb * sizeof(R);
        KTables<R> kt;
        kt.tk = at<const R>(pl, y.tk);
        kt.te = at<const R>(pl, y.te);
        kt.td = at<const R>(pl, y.td);
        const double V3 = r.prm.L[0] * r.prm.L[1] * r.prm.L[2];
        kt.cE = (R)(r.prm.coulomb_k * 2.0 * kPi / V3);
        kt.cF = (R)(r.prm.coulomb_k * 4.0 * kPi / V3);
        kt.inv4a2 = (R)(1.0 / (4.0 * r.prm.alpha * r.prm.alpha));
        const dim3 g((r.P + Wc - 1) / Wc);
        const int NT = M >= 4 ? M / 4 : 1;  // threads per pencil in k_fz (radix-4 passes)
        if (nf == 0)
            LCHK(L.go("fft_z_kspace", k_fz<R, M, 0>, g, dim3(Wc * NT), smem, at<const V>(pl, y.C2), at<V>(pl, y.C3), r.gz,
                      W, kt, at<double>(pl, y.kpart)));
        else if (nf == 1)
            LCHK(L.go("fft_z_kspace", k_fz<R, M, 1>, g, dim3(Wc * NT), smem, at<const V>(pl, y.C2), at<V>(pl, y.C3), r.gz,
                      W, kt, at<double>(pl, y.kpart)));
        else if (nf == 3)
            LCHK(L.go("fft_z_kspace", k_fz<R, M, 3>, g, dim3(Wc * NT), smem, at<const V>(pl, y.C2), at<V>(pl, y.C3), r.gz,
                      W, kt, at<double>(pl, y.kpart)));
        else
            LCHK(L.go("fft_z_kspace", k_fz<R, M, 4>, g, dim3(Wc * NT), smem, at<const V>(pl, y.C2), at<V>(pl, y.C3), r.gz,
                      W, kt, at<double>(pl, y.kpart)));
    }
    if (nf == 0) return ENUF_OK;
    if (fused) {
        return L.go("ifft_yx", k_iyx<R, M>, dim3(M, nf), dim3(r.iyx_threads), r.iyx_smem, at<const V>(pl, y.C3),
                    at<R>(pl, y.fld), r.gy, W);
    }
    // inverse y
    {
        const int Wc = r.gy.W;
        LCHK(L.go("ifft_y", k_iy<R, M>, dim3((r.Kx + Wc - 1) / Wc, M, nf), dim3(Wc * NT), (size_t)(Wc * (padlen(M) + 1) + M) * vs,
                  at<const V>(pl, y.C3), at<V>(pl, y.C4), r.gy, W));
    }
    // inverse x (complex to real)
    {
        const int NTh = rowthreads(M / 2), rows = r.gfx.rows;
        const int nrows = nf * M * M;
        LCHK(L.go("ifft_x", k_ix<R, M>, dim3((nrows + rows - 1) / rows), dim3(rows * NTh), (size_t)(rows * padlen(M / 2) + M) * vs,
                  at<const V>(pl, y.C4), at<R>(pl, y.fld), r.gfx, nrows, W));
    }
    return ENUF_OK;
}

template <typename R> int launch_fft_chain(Launcher& L, enuf_plan* pl, int nf, void* spec = nullptr, int scale = 0)
{
    switch (pl->r.prm.M) {
    case 8: return launch_fft_chain_m<R, 8>(L, pl, nf, spec, scale);
    case 16: return launch_fft_chain_m<R, 16>(L, pl, nf, spec, scale);
    case 32: return launch_fft_chain_m<R, 32>(L, pl, nf, spec, scale);
    case 64: return launch_fft_chain_m<R, 64>(L, pl, nf, spec, scale);
    case 128: return launch_fft_chain_m<R, 128>(L, pl, nf, spec, scale);
    case 256: return launch_fft_chain_m<R, 256>(L, pl, nf, spec, scale);
    case 512: return launch_fft_chain_m<R, 512>(L, pl, nf, spec, scale);
    default: return fail(ENUF_EUNSUPPORTED, "unsupported M");
    }
}

// Bin counts above this are scanned by the chunked passes (k_scan_sums,
// k_scan_bases, k_scan_apply) rather than by the key pass's last block.
constexpr int kFusedScanMax = 16384;

int launch_chunked_scan(Launcher& L, enuf_plan* pl, const ScanArgs& sa, int group, size_t csum_off,
                        size_t cbase_off)
{
    const int nch = (sa.nbins + kScanChunk - 1) / kScanChunk;
    uint32_t* cs = at<uint32_t>(pl, csum_off);
    uint32_t* cb = at<uint32_t>(pl, cbase_off);
    int* status = at<int>(pl, pl->lay.status);
    if (group == 8) LCHK(L.go("scan_sums", k_scan_sums<8>, dim3(nch), dim3(256), 0, sa, cs));
    else if (group == 4) LCHK(L.go("scan_sums", k_scan_sums<4>, dim3(nch), dim3(256), 0, sa, cs));
    else LCHK(L.go("scan_sums", k_scan_sums<1>, dim3(nch), dim3(256), 0, sa, cs));
    LCHK(L.go("scan_bases", k_scan_bases, dim3(1), dim3(1024), 0, sa, nch, (const uint32_t*)cs, cb, status));
    if (group == 8) LCHK(L.go("scan_apply", k_scan_apply<8>, dim3(nch), dim3(256), 0, sa, (const uint32_t*)cb, status));
    else if (group == 4)
        LCHK(L.go("scan_apply", k_scan_apply<4>, dim3(nch), dim3(256), 0, sa, (const uint32_t*)cb, status));
    else LCHK(L.go("scan_apply", k_scan_apply<1>, dim3(nch), dim3(256), 0, sa, (const uint32_t*)cb, status));
    return ENUF_OK;
}

// Blocks of the assembly: one up to 4096 partials of a quantity, at most 64.
int fin_blocks(const FinalParams& fp)
{
    const int n = std::max(fp.nq, std::max(fp.nk, fp.nr));
    return std::max(1, std::min(64, (n + 4095) / 4096));
}

BinGeom make_geom(const int S[3], int T, const double L3[3], bool grid_units, int sub = 1, int lr = 0)
{
    BinGeom g{};
    g.sub = sub;
    g.lr = lr;
    for (int t = 0; t < 3; t++) {
        g.S[t] = S[t];
        g.nb[t] = S[t] / T;
        g.scale[t] = (double)S[t] / L3[t];
        g.scale_hi[t] = (float)g.scale[t];
        g.scale_lo[t] = (float)(g.scale[t] - (double)g.scale_hi[t]);
        g.unit[t] = grid_units ? 1.0 : L3[t] / S[t];
    }
    g.T = T;
    while ((1 << g.lT) < T) g.lT++;
    while ((1 << g.lsub) < sub) g.lsub++;
    for (int t = 0; t < 3; t++) g.smask[t] = (S[t] & (S[t] - 1)) == 0 ? S[t] - 1 : -1;
    return g;
}

// The whole evaluation on stream L.st.
// With `spec` set: the transposed NFFT alone (sort, spread, forward FFT,
// scaling), the structure factor S~ written to spec; nothing else runs.
template <typename R>
int launch_sequence(Launcher& L, enuf_plan* pl, const R* pos, const R* q, R* F, R* phi, double* out, int flags,
                    void* spec = nullptr)
{
    const Resolved& r = pl->r;
    const Layout& y = pl->lay;
    const int N = (int)r.prm.N;
    const int nblkN = (N + 255) / 256;
    const bool want_phi = (flags & ENUF_WANT_PHI) && phi;
    const bool konly = (flags & ENUF_KSPACE_ONLY) || spec;
    // forces by analytic differentiation: the potential's grid alone
    const bool ad = (flags & ENUF_AD_FORCES) && (F || want_phi);
    const int nf = ad ? 1 : (want_phi ? 4 : (F ? 3 : 0));
    using RecT = typename Rec<R>::T;

    // the status word, the bin counts and the block counters are kept
    // zeroed between calls by the kernels that consume them (k_finalize, the
    // scan in the last block of k_bin_keys)
    // (a8) real space: its own sort scratch and output buffers, so that it
    // can run on a side branch beside the whole reciprocal chain; the
    // outputs are added to the reciprocal ones after both
    auto real_space = [&]() -> int {
        const BinGeom gr = make_geom(r.ncell, 1, r.prm.L, false);
        const bool rbig = r.nrbins > kFusedScanMax;
        ScanArgs sr{r.nrbins, at<uint32_t>(pl, y.rcounts), count_stride(r.nrbins), at<uint32_t>(pl, y.roffsets),
                    kWorkCap, (int4*)nullptr, (int*)nullptr, 0, kSpreadCap, (uint32_t*)nullptr, (int*)nullptr, 0,
                    rbig ? (unsigned*)nullptr : at<unsigned>(pl, y.status + 12)};
        LCHK(L.go("real_bin_keys", k_bin_keys<R, 1>, dim3(nblkN), dim3(256), 0, N, pos, q, gr, at<uint32_t>(pl, y.rkey),
                  at<uint32_t>(pl, y.rrank), at<RecT>(pl, y.rrec_tmp), sr, at<int>(pl, y.status), (double*)nullptr));
        if (rbig) LCHK(launch_chunked_scan(L, pl, sr, 1, y.csum_r, y.cbase_r));
        LCHK(L.go("real_scatter", k_scatter<R>, dim3(nblkN), dim3(256), 0, N, at<const uint32_t>(pl, y.rkey),
                  at<const uint32_t>(pl, y.rrank), at<const uint32_t>(pl, y.roffsets), at<const RecT>(pl, y.rrec_tmp),
                  at<RecT>(pl, y.rrec), at<uint32_t>(pl, y.rperm), at<uint32_t>(pl, y.rcell), (const uint32_t*)nullptr,
                  kSpreadCap, (int4*)nullptr, 0, r.nrbins));
        RealParams<R> rp;
        for (int t = 0; t < 3; t++) {
            rp.nc[t] = r.ncell[t];
            rp.h[t] = (R)r.h[t];
            rp.L[t] = (R)r.prm.L[t];
        }
        rp.rc2 = (R)(r.prm.r_c * r.prm.r_c);
        rp.alpha = (R)r.prm.alpha;
        rp.two_a_sqpi = (R)(2.0 * r.prm.alpha / std::sqrt(kPi));
        rp.ke = (R)r.prm.coulomb_k;
        rp.self_phi = (R)(-2.0 * r.prm.alpha / std::sqrt(kPi));
        R* Fo = F ? at<R>(pl, y.Fr) : nullptr;
        R* po = want_phi ? at<R>(pl, y.phir) : nullptr;
        rp.inv_lam = r.prm.slater_lambda > 0.0 ? (R)(1.0 / r.prm.slater_lambda) : R(0);
        const bool sl = r.prm.slater_lambda > 0.0;
        const RecT* rrec = at<const RecT>(pl, y.rrec);
        const uint32_t* rperm = at<const uint32_t>(pl, y.rperm);
        double* rpart = at<double>(pl, y.rpart);
        if (r.cells) {
            const uint32_t* rcell = at<const uint32_t>(pl, y.rcell);
            const uint32_t* roff = at<const uint32_t>(pl, y.roffsets);
            const dim3 g(nblkN, 2 * r.sr + 1);
            if (r.sr == 2)
                LCHK(L.go("realspace", sl ? k_realspace_cells<R, 2, true> : k_realspace_cells<R, 2, false>, g,
                          dim3(256), 0, N, rrec, rcell, roff, rperm, rp, Fo, po, rpart));
            else
                LCHK(L.go("realspace", sl ? k_realspace_cells<R, 1, true> : k_realspace_cells<R, 1, false>, g,
                          dim3(256), 0, N, rrec, rcell, roff, rperm, rp, Fo, po, rpart));
        } else {
            LCHK(L.go("realspace", sl ? k_realspace_allpairs<R, true> : k_realspace_allpairs<R, false>, dim3(nblkN),
                      dim3(256), 0, N, rrec, rperm, rp, Fo, po, rpart));
        }
        return ENUF_OK;
    };
    const int nr = konly ? 0 : nblkN * (r.cells ? 2 * r.sr + 1 : 1);
    const bool real_side = !konly && !L.attr_only && !pl->profile;
    if (real_side) {
        CK(cudaEventRecord(pl->ev_fork, L.st));
        CK(cudaStreamWaitEvent(pl->aux_stream, pl->ev_fork, 0));
        const cudaStream_t main_st = L.st;
        L.st = pl->aux_stream;
        const int rc = real_space();
        L.st = main_st;
        cudaEventRecord(pl->ev_join, pl->aux_stream);
        if (rc != ENUF_OK) {
            cudaStreamWaitEvent(L.st, pl->ev_join, 0);  // a capture must end joined
            return rc;
        }
    } else if (!konly) {
        LCHK(real_space());
    }

    // (a1, a2) counting sort into grid tiles
    const int Sg[3] = {r.prm.M, r.prm.M, r.prm.M};
    const BinGeom gg = make_geom(Sg, r.T, r.prm.L, true, r.S, r.lr);
    {
        const bool big = r.nbins > kFusedScanMax;
        ScanArgs sa{r.nbins, at<uint32_t>(pl, y.counts), count_stride(r.nbins), at<uint32_t>(pl, y.offsets),
                    r.gcap, at<int4>(pl, y.work), at<int>(pl, y.nwork), r.max_work, kSpreadCap,
                    at<uint32_t>(pl, y.item2), at<int>(pl, y.nwork2), r.max_work2,
                    big ? (unsigned*)nullptr : at<unsigned>(pl, y.status + 8)};
        LCHK(L.go("bin_keys", r.ggroup == 8 ? k_bin_keys<R, 8> : (r.ggroup == 4 ? k_bin_keys<R, 4> : k_bin_keys<R, 1>),
                  dim3(nblkN), dim3(256), 0, N, pos, q, gg,
                  at<uint32_t>(pl, y.key), at<uint32_t>(pl, y.rank), at<RecT>(pl, y.rec_tmp), sa, at<int>(pl, y.status),
                  at<double>(pl, y.qpart)));
        if (big) LCHK(launch_chunked_scan(L, pl, sa, r.ggroup, y.csum_g, y.cbase_g));
    }
    LCHK(L.go("scatter", k_scatter<R>, dim3(nblkN), dim3(256), 0, N, at<const uint32_t>(pl, y.key),
              at<const uint32_t>(pl, y.rank), at<const uint32_t>(pl, y.offsets), at<const RecT>(pl, y.rec_tmp),
              at<RecT>(pl, y.rec), at<uint32_t>(pl, y.perm),
              r.gather_direct ? at<uint32_t>(pl, y.tile_of) : (uint32_t*)nullptr,  // read only by the direct gathers
              at<const uint32_t>(pl, y.item2), kSpreadCap, at<int4>(pl, y.work2), r.max_work2, r.nbins));
    // (a3) spread (into a zeroed grid: zeroed at binding, then by the
    // forward FFT that reads it)
    LCHK(launch_spread<R>(L, pl));
    if (spec) return launch_fft_chain<R>(L, pl, 0, spec, 1);
    // (a4-a6) FFT chain with the fused reciprocal step
    LCHK(launch_fft_chain<R>(L, pl, nf));
    // (a9) assembly parameters
    FinalParams fp;
    fp.nq = nblkN;
    fp.nk = (r.P + r.gz.W - 1) / r.gz.W;
    fp.nr = 0;
    fp.ke = r.prm.coulomb_k;
    fp.alpha = r.prm.alpha;
    fp.V = r.prm.L[0] * r.prm.L[1] * r.prm.L[2];
    fp.sqrt_pi = std::sqrt(kPi);
    fp.kspace_only = konly ? 1 : 0;
    double* o = out ? out : at<double>(pl, y.out);
    // k-space only: the assembly needs nothing from the interpolation, so it
    // runs on a side branch beside it (not in profiling mode, whose timing
    // events follow one stream)
    const bool side = konly && nf > 0 && !L.attr_only && !pl->profile;
    if (side) {
        CK(cudaEventRecord(pl->ev_fork, L.st));
        CK(cudaStreamWaitEvent(pl->aux_stream, pl->ev_fork, 0));
        const cudaStream_t main_st = L.st;
        L.st = pl->aux_stream;
        const int rc = L.go("finalize", k_finalize, dim3(fin_blocks(fp)), dim3(512), 0, at<const double>(pl, y.qpart),
                            at<const double>(pl, y.kpart), at<const double>(pl, y.rpart), fp, at<int>(pl, y.status), o,
                            at<double>(pl, y.fscratch), at<unsigned>(pl, y.status + 4));
        L.st = main_st;
        if (rc != ENUF_OK) {
            // rejoin the side branch before returning (a capture must end joined)
            cudaEventRecord(pl->ev_join, pl->aux_stream);
            cudaStreamWaitEvent(L.st, pl->ev_join, 0);
            return rc;
        }
        CK(cudaEventRecord(pl->ev_join, pl->aux_stream));
    }
    // (a7) interpolation
    if (ad) LCHK(launch_gather_ad<R>(L, pl, F, want_phi ? phi : (R*)nullptr));
    else if (nf > 0) LCHK(launch_gather<R>(L, pl, nf, F, want_phi ? phi : (R*)nullptr));
    // (a9) assembly
    fp.nr = nr;
    if (real_side) CK(cudaStreamWaitEvent(L.st, pl->ev_join, 0));
    if (!konly && (F || want_phi))
        LCHK(L.go("combine", k_combine<R>, dim3(nblkN), dim3(256), 0, N, at<R>(pl, y.Fr), at<R>(pl, y.phir), F,
                  want_phi ? phi : (R*)nullptr));
    if (side) CK(cudaStreamWaitEvent(L.st, pl->ev_join, 0));
    else
        LCHK(L.go("finalize", k_finalize, dim3(fin_blocks(fp)), dim3(512), 0, at<const double>(pl, y.qpart),
                  at<const double>(pl, y.kpart), at<const double>(pl, y.rpart), fp, at<int>(pl, y.status), o,
                  at<double>(pl, y.fscratch), at<unsigned>(pl, y.status + 4)));
    if (want_phi && !konly)
        LCHK(L.go("phi_background", k_phi_background<R>, dim3(nblkN), dim3(256), 0, N, (const double*)o,
                  -r.prm.coulomb_k * kPi / (fp.V * r.prm.alpha * r.prm.alpha), phi));
    if ((flags & ENUF_REMOVE_NET_FORCE) && F) {
        LCHK(L.go("force_sum", k_force_sum<R>, dim3(nblkN), dim3(256), 0, N, (const R*)F, at<double>(pl, y.fpart)));
        LCHK(L.go("force_mean", k_force_mean, dim3(1), dim3(256), 0, nblkN, N, at<const double>(pl, y.fpart),
                  at<double>(pl, y.mean)));
        LCHK(L.go("force_shift", k_force_shift<R>, dim3(nblkN), dim3(256), 0, N, at<const double>(pl, y.mean), F));
    }
    return ENUF_OK;
}

int run_sequence(enuf_plan* pl, cudaStream_t st, bool attr_only, const void* pos, const void* q, void* F, void* phi,
                 double* out, int flags, int* count = nullptr)
{
    Launcher L{pl, st, attr_only};
    int rc;
    if (pl->r.fp64)
        rc = launch_sequence<double>(L, pl, (const double*)pos, (const double*)q, (double*)F, (double*)phi, out, flags);
    else
        rc = launch_sequence<float>(L, pl, (const float*)pos, (const float*)q, (float*)F, (float*)phi, out, flags);
    if (count) *count = L.count;
    return rc;
}

int prepare_attrs(enuf_plan* pl)
{
    if (pl->attrs_done) return ENUF_OK;
    // walk every variant once in attribute-only mode (no launches)
    int flags[4] = {ENUF_WANT_PHI, 0, ENUF_REMOVE_NET_FORCE, ENUF_AD_FORCES | ENUF_WANT_PHI};
    for (int k = 0; k < 4; k++) {
        void* dummy = (void*)pl->ws;
        int rc = run_sequence(pl, pl->stream, true, dummy, dummy, dummy, dummy, nullptr, flags[k]);
        if (rc != ENUF_OK) return rc;
    }
    int rc = run_sequence(pl, pl->stream, true, pl->ws, pl->ws, nullptr, nullptr, nullptr, 0);
    if (rc != ENUF_OK) return rc;
    pl->attrs_done = true;
    return ENUF_OK;
}

int upload_tables(enuf_plan* pl)
{
    const Resolved& r = pl->r;
    const int M = r.prm.M, Kb = r.Kb, nc = r.nc;
    std::vector<double> tw(2 * M), tk(3 * Kb), te(3 * Kb), td(3 * Kb);
    for (int k = 0; k < M; k++) {
        double a = -2.0 * kPi * (double)k / (double)M;
        tw[2 * k] = std::cos(a);
        tw[2 * k + 1] = std::sin(a);
    }
    for (int t = 0; t < 3; t++)
        for (int n = -nc; n <= nc; n++) {
            const double kk = 2.0 * kPi * n / r.prm.L[t];
            const double s = kPi * n / (double)M;
            tk[t * Kb + n + nc] = kk;
            te[t * Kb + n + nc] = std::exp(-kk * kk / (4.0 * r.prm.alpha * r.prm.alpha));
            td[t * Kb + n + nc] = std::exp(2.0 * pl->b * s * s);
        }
    auto put = [&](size_t off, const std::vector<double>& v) -> int {
        if (r.fp64) {
            CK(cudaMemcpy(pl->ws + off, v.data(), v.size() * 8, cudaMemcpyHostToDevice));
        } else {
            std::vector<float> f(v.begin(), v.end());
            CK(cudaMemcpy(pl->ws + off, f.data(), f.size() * 4, cudaMemcpyHostToDevice));
        }
        return ENUF_OK;
    };
    LCHK(put(pl->lay.twid, tw));
    LCHK(put(pl->lay.tk, tk));
    LCHK(put(pl->lay.te, te));
    LCHK(put(pl->lay.td, td));
    return ENUF_OK;
}

void drop_graphs(enuf_plan* pl)
{
    for (auto& g : pl->graphs) cudaGraphExecDestroy(g.exec);
    pl->graphs.clear();
    if (pl->md.exec) cudaGraphExecDestroy(pl->md.exec);
    pl->md.exec = nullptr;
}

// Tensor map of the four field planes (x, y, z, field) for the TMA boxes of
// k_gather_p8 / k_gather_p6: boxes of BX x PY x PZ x 1 cells (the kernel's
// geometry for the plan's p), no swizzle, zeros outside.
int encode_field_map(enuf_plan* pl)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return fail(ENUF_ECUDA, "the driver does not provide cuTensorMapEncodeTiled");
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const bool p8 = pl->r.prm.p == 8;
    const cuuint64_t M = (cuuint64_t)pl->r.prm.M;
    const cuuint64_t dims[4] = {M, M, M, 4};
    const cuuint64_t strides[3] = {M * 4, M * M * 4, M * M * M * 4};
    const cuuint32_t box[4] = {(cuuint32_t)(p8 ? GatherP8<3>::B::BX : GatherP6<3>::B::BX),
                               (cuuint32_t)(p8 ? GatherP8<3>::PY : GatherP6<3>::PY),
                               (cuuint32_t)(p8 ? GatherP8<3>::B::PZ : GatherP6<3>::B::PZ), 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult rc = encode(&pl->fld_tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, pl->ws + pl->lay.fld, dims, strides,
                               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) return fail(ENUF_ECUDA, "cuTensorMapEncodeTiled failed with code " + std::to_string((int)rc));
    return ENUF_OK;
}

int bind_workspace(enuf_plan* pl, void* ptr)
{
    drop_graphs(pl);
    pl->ws = (char*)ptr;
    // the p = 8 and 6 single-precision interpolation on z-halves of 16-cell
    // tiles stages its boxes through a tensor map of this workspace's field
    // planes
    const Resolved& r = pl->r;
    pl->gather_tma = !r.fp64 && r.T == 16 && r.zhalf && (r.prm.p == 8 || r.prm.p == 6) && r.prm.M >= 32 &&
                     r.gcap == 256 && !r.gather_direct && !pl->legacy_gather;
    if (pl->gather_tma) LCHK(encode_field_map(pl));
    // the status word and the bin counts start (and are kept) zeroed
    CK(cudaMemset(pl->ws, 0, pl->lay.total));
    LCHK(upload_tables(pl));
    pl->attrs_done = false;
    return prepare_attrs(pl);
}

// Restores the buffers that evaluations expect zeroed (after an evaluation
// was cut short).
void reset_zeroed(enuf_plan* pl)
{
    const Layout& y = pl->lay;
    const Resolved& r = pl->r;
    const size_t M3 = (size_t)r.prm.M * r.prm.M * r.prm.M;
    cudaMemsetAsync(pl->ws + y.status, 0, 16, pl->stream);
    cudaMemsetAsync(pl->ws + y.counts, 0, (size_t)(r.nbins + 1) * 4 * count_stride(r.nbins), pl->stream);
    cudaMemsetAsync(pl->ws + y.rcounts, 0, (size_t)(r.nrbins + 1) * 4 * count_stride(r.nrbins), pl->stream);
    cudaMemsetAsync(pl->ws + y.grid, 0, M3 * r.rsz, pl->stream);
    cudaMemsetAsync(pl->ws + y.Fr, 0, (size_t)3 * r.prm.N * r.rsz, pl->stream);
    cudaMemsetAsync(pl->ws + y.phir, 0, (size_t)r.prm.N * r.rsz, pl->stream);
    cudaGetLastError();
}

// Instantiates a captured graph, adds it to the plan's cache (evicting the
// least recently used of 8) and launches it on the plan's stream.
int cache_and_launch(enuf_plan* pl, GraphEntry ge, cudaGraph_t graph)
{
    cudaError_t e = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ENUF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    if (pl->graphs.size() >= 8) {
        auto old = std::min_element(pl->graphs.begin(), pl->graphs.end(),
                                    [](const GraphEntry& a, const GraphEntry& b) { return a.stamp < b.stamp; });
        cudaGraphExecDestroy(old->exec);
        pl->graphs.erase(old);
    }
    pl->graphs.push_back(ge);
    CK(cudaGraphLaunch(ge.exec, pl->stream));
    return ENUF_OK;
}

int compute_impl(enuf_plan* pl, const void* pos, const void* q, void* F, void* phi, double* out, int flags)
{
    if (!pl) return fail(ENUF_EINVAL, "plan is NULL");
    if (!pl->ws) return fail(ENUF_EINVAL, "plan has no workspace");
    if (!pos || !q) return fail(ENUF_EINVAL, "pos and q are required");
    if ((flags & ENUF_WANT_PHI) && !phi) return fail(ENUF_EINVAL, "ENUF_WANT_PHI needs a phi buffer");
    if (flags & ~(ENUF_WANT_VIRIAL | ENUF_WANT_PHI | ENUF_REMOVE_NET_FORCE | ENUF_KSPACE_ONLY | ENUF_AD_FORCES))
        return fail(ENUF_EINVAL, "unknown flag bits");
    if (!(flags & ENUF_WANT_PHI)) phi = nullptr;
    if (pl->profile) {
        // a fresh graph per call with an event-record node before every
        // kernel and one after the last, so kernel times carry no launch gaps
        if (pl->prof_exec) {
            cudaGraphExecDestroy(pl->prof_exec);
            pl->prof_exec = nullptr;
        }
        pl->tnames.clear();
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = run_sequence(pl, pl->cap_stream, false, pos, q, F, phi, out, flags);
        if (rc == ENUF_OK) cudaEventRecordWithFlags(pl->tevents[pl->tnames.size()], pl->cap_stream, cudaEventRecordExternal);
        cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &graph);
        if (rc != ENUF_OK) {
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ENUF_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
        e = cudaGraphInstantiate(&pl->prof_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ENUF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
        CK(cudaGraphLaunch(pl->prof_exec, pl->stream));
        return ENUF_OK;
    }
    if (!pl->use_graph) {
        int rc = run_sequence(pl, pl->stream, false, pos, q, F, phi, out, flags);
        if (rc != ENUF_OK) reset_zeroed(pl);
        return rc;
    }
    for (auto& g : pl->graphs) {
        if (g.pos == pos && g.q == q && g.F == F && g.phi == phi && g.out == out && g.flags == flags) {
            g.stamp = ++pl->stamp;
            CK(cudaGraphLaunch(g.exec, pl->stream));
            return ENUF_OK;
        }
    }
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = run_sequence(pl, pl->cap_stream, false, pos, q, F, phi, out, flags);
    cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &graph);
    if (rc != ENUF_OK) {
        if (e == cudaSuccess) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ENUF_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    GraphEntry ge{pos, q, F, phi, out, flags, nullptr, ++pl->stamp};
    return cache_and_launch(pl, ge, graph);
}

// Host-buffer call as one graph: the copies of positions and charges in,
// the evaluation, and the copies of forces, potentials and results out
// (pinned host buffers only; cached by the host pointers, flag bit 30 marks
// these entries).
int host_graph_call(enuf_plan* pl, const void* pos_host, const void* q_host, void* F_host, void* phi_host,
                    int flags, void* F, void* phi, double* dout)
{
    const size_t N = (size_t)pl->r.prm.N, rs = pl->r.rsz;
    const Layout& y = pl->lay;
    const int key = flags | (1 << 30);
    for (auto& g : pl->graphs) {
        if (g.pos == pos_host && g.q == q_host && g.F == F_host && g.phi == phi_host && g.out == pl->hout &&
            g.flags == key) {
            g.stamp = ++pl->stamp;
            CK(cudaGraphLaunch(g.exec, pl->stream));
            return ENUF_OK;
        }
    }
    const cudaStream_t cs = pl->cap_stream;
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaMemcpyAsync(pl->ws + y.s_pos, pos_host, 3 * N * rs, cudaMemcpyHostToDevice, cs);
    cudaMemcpyAsync(pl->ws + y.s_q, q_host, N * rs, cudaMemcpyHostToDevice, cs);
    int rc = run_sequence(pl, cs, false, pl->ws + y.s_pos, pl->ws + y.s_q, F, phi, dout, flags);
    if (rc == ENUF_OK) {
        if (F_host) cudaMemcpyAsync(F_host, F, 3 * N * rs, cudaMemcpyDeviceToHost, cs);
        if (phi) cudaMemcpyAsync(phi_host, phi, N * rs, cudaMemcpyDeviceToHost, cs);
        cudaMemcpyAsync(pl->hout, dout, ENUF_NOUT * sizeof(double), cudaMemcpyDeviceToHost, cs);
    }
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (rc != ENUF_OK) {
        if (e == cudaSuccess) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ENUF_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    }
    GraphEntry ge{pos_host, q_host, F_host, phi_host, pl->hout, key, nullptr, ++pl->stamp};
    return cache_and_launch(pl, ge, graph);
}

// True for host memory the GPU can copy to and from directly (pinned or
// registered); a NULL pointer counts as such.
bool host_pinned(const void* p)
{
    if (!p) return true;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

int check_status(const double* parts)
{
    const int st = (int)parts[ENUF_OUT_STATUS];
    if (st & ST_NONFINITE) return fail(ENUF_ENONFINITE, "a position or charge is NaN or infinite");
    if (st) return fail(ENUF_EDEVICE, "a kernel reported internal status " + std::to_string(st));
    return ENUF_OK;
}

}  // namespace

namespace enuf {
// Lets the other translation unit of the library report through
// enuf_last_error().
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace enuf

// ====================================================================== C ABI
extern "C" {

const char* enuf_last_error(void) { return g_err.c_str(); }

const char* enuf_version(void) { return "enuf-b300 0.1 (sm_103a)"; }

int enuf_plan_workspace_bytes(const enuf_params* params, size_t* bytes)
{
    Resolved r;
    LCHK(resolve(params, r));
    if (!bytes) return fail(ENUF_EINVAL, "bytes is NULL");
    *bytes = layout(r).total;
    return ENUF_OK;
}

int enuf_plan_create(const enuf_params* params, void* cuda_stream, int allocate, enuf_plan** out)
{
    g_err.clear();
    if (!out) return fail(ENUF_EINVAL, "out is NULL");
    *out = nullptr;
    Resolved r;
    LCHK(resolve(params, r));
    enuf_plan* pl = new enuf_plan();
    pl->r = r;
    pl->lay = layout(r);
    pl->stream = (cudaStream_t)cuda_stream;
    const double sigma = (double)r.prm.M / (2.0 * r.nc), m = 0.5 * r.prm.p;
    pl->b = 2.0 * sigma * m / ((2.0 * sigma - 1.0) * kPi);
    pl->inv_b = 1.0 / pl->b;
    pl->cnorm3 = std::pow(kPi * pl->b, -1.5);
    while ((1 << pl->lnb) < r.nbt[0]) pl->lnb++;
    const char* ev = std::getenv("ENUF_NO_GRAPH");
    pl->use_graph = !(ev && ev[0] == '1');
    ev = std::getenv("ENUF_PROFILE");
    pl->profile = ev && ev[0] == '1';
    ev = std::getenv("ENUF_NO_PDL");
    pl->pdl = !(ev && ev[0] == '1');
    ev = std::getenv("ENUF_LEGACY_GATHER");
    pl->legacy_gather = ev && ev[0] == '1';
    if (pl->profile) {
        pl->tevents.resize(48);
        for (auto& x : pl->tevents) cudaEventCreate(&x);
    }
    cudaError_t e = cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->aux_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess && cudaMallocHost((void**)&pl->hout, ENUF_NOUT * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();  // pinned memory is an optimisation: fall back to a pageable copy
        pl->hout = nullptr;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
        if (pl->ev_join) cudaEventDestroy(pl->ev_join);
        if (pl->aux_stream) cudaStreamDestroy(pl->aux_stream);
        if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
        for (auto x : pl->tevents) cudaEventDestroy(x);
        delete pl;
        return fail(ENUF_ECUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    }
    if (allocate) {
        void* p = nullptr;
        e = cudaMalloc(&p, pl->lay.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaEventDestroy(pl->ev_fork);
            cudaEventDestroy(pl->ev_join);
            cudaStreamDestroy(pl->aux_stream);
            cudaStreamDestroy(pl->cap_stream);
            if (pl->hout) cudaFreeHost(pl->hout);
            for (auto x : pl->tevents) cudaEventDestroy(x);
            const size_t want = pl->lay.total;
            delete pl;
            return fail(ENUF_ENOMEM, "cudaMalloc of " + std::to_string(want) + " bytes failed: " +
                                         cudaGetErrorString(e));
        }
        pl->own_ws = true;
        int rc = bind_workspace(pl, p);
        if (rc != ENUF_OK) {
            std::string msg = g_err;
            enuf_plan_destroy(pl);
            return fail(rc, msg);
        }
    }
    *out = pl;
    return ENUF_OK;
}

int enuf_plan_set_workspace(enuf_plan* pl, void* dev_ptr, size_t bytes)
{
    if (!pl || !dev_ptr) return fail(ENUF_EINVAL, "plan or pointer is NULL");
    if (bytes < pl->lay.total) return fail(ENUF_EINVAL, "workspace too small");
    if (((uintptr_t)dev_ptr) & 255) return fail(ENUF_EINVAL, "workspace must be 256-byte aligned");
    if (pl->own_ws && pl->ws) {
        cudaFree(pl->ws);
        pl->own_ws = false;
    }
    return bind_workspace(pl, dev_ptr);
}

int enuf_plan_set_stream(enuf_plan* pl, void* cuda_stream)
{
    if (!pl) return fail(ENUF_EINVAL, "plan is NULL");
    pl->stream = (cudaStream_t)cuda_stream;
    return ENUF_OK;
}

int enuf_plan_get_params(const enuf_plan* pl, enuf_params* out)
{
    if (!pl || !out) return fail(ENUF_EINVAL, "NULL argument");
    *out = pl->r.prm;
    return ENUF_OK;
}

// One velocity-Verlet step on stream st (see md.cuh).
int md_step_sequence(enuf_plan* pl, cudaStream_t st, void* pos, void* vel, const void* q, const void* im, void* F,
                     double dt, int flags, double* energies, int cap)
{
    const Resolved& r = pl->r;
    const Layout& y = pl->lay;
    const int N = (int)r.prm.N, nb = (N + 255) / 256;
    Launcher L{pl, st, false};
    double* out = at<double>(pl, y.out);
    double* part = at<double>(pl, y.fpart);
    unsigned* step = at<unsigned>(pl, y.md_step);
    if (r.fp64) {
        using R = double;
        LCHK(L.go("md_kick_drift", k_md_kick_drift<R>, dim3(nb), dim3(256), 0, N, (R*)pos, (R*)vel, (const R*)F,
                  (const R*)im, (R)(0.5 * dt), (R)dt, (R)r.prm.L[0], (R)r.prm.L[1], (R)r.prm.L[2]));
    } else {
        using R = float;
        LCHK(L.go("md_kick_drift", k_md_kick_drift<R>, dim3(nb), dim3(256), 0, N, (R*)pos, (R*)vel, (const R*)F,
                  (const R*)im, (R)(0.5 * dt), (R)dt, (R)r.prm.L[0], (R)r.prm.L[1], (R)r.prm.L[2]));
    }
    LCHK(run_sequence(pl, st, false, pos, q, F, nullptr, out, flags));
    if (r.fp64) {
        using R = double;
        LCHK(L.go("md_kick", k_md_kick<R>, dim3(nb), dim3(256), 0, N, (R*)vel, (const R*)F, (const R*)im, (R)(0.5 * dt),
                  part));
    } else {
        using R = float;
        LCHK(L.go("md_kick", k_md_kick<R>, dim3(nb), dim3(256), 0, N, (R*)vel, (const R*)F, (const R*)im, (R)(0.5 * dt),
                  part));
    }
    LCHK(L.go("md_record", k_md_record, dim3(1), dim3(256), 0, nb, (const double*)part, (const double*)out, energies,
              step, cap));
    return ENUF_OK;
}

int enuf_md_run(enuf_plan* pl, void* pos, void* vel, const void* q, const void* inv_mass, void* F, int have_forces,
                double dt, int nsteps, int flags, double* energies)
{
    if (!pl) return fail(ENUF_EINVAL, "plan is NULL");
    if (!pl->ws) return fail(ENUF_EINVAL, "plan has no workspace");
    if (!pos || !vel || !q || !inv_mass || !F || !energies) return fail(ENUF_EINVAL, "a buffer is NULL");
    if (nsteps < 0) return fail(ENUF_EINVAL, "nsteps must be >= 0");
    if (!std::isfinite(dt)) return fail(ENUF_EINVAL, "dt must be finite");
    if (flags & ~(ENUF_WANT_VIRIAL | ENUF_REMOVE_NET_FORCE | ENUF_KSPACE_ONLY | ENUF_AD_FORCES))
        return fail(ENUF_EINVAL, "unknown or unsupported flag bits");
    LCHK(prepare_attrs(pl));
    double* out = at<double>(pl, pl->lay.out);
    if (!have_forces) LCHK(compute_impl(pl, pos, q, F, nullptr, out, flags));
    CK(cudaMemsetAsync(pl->ws + pl->lay.md_step, 0, 16, pl->stream));
    if (nsteps == 0) return ENUF_OK;
    if (!pl->use_graph || pl->profile) {
        for (int s = 0; s < nsteps; s++) {
            int rc = md_step_sequence(pl, pl->stream, pos, vel, q, inv_mass, F, dt, flags, energies, nsteps);
            if (rc != ENUF_OK) {
                reset_zeroed(pl);
                return rc;
            }
        }
        return ENUF_OK;
    }
    auto& m = pl->md;
    const bool same = m.exec && m.pos == pos && m.vel == vel && m.q == q && m.inv_mass == inv_mass && m.F == F &&
                      m.energies == energies && m.flags == flags && m.dt == dt && m.cap == nsteps;
    if (!same) {
        if (m.exec) cudaGraphExecDestroy(m.exec);
        m.exec = nullptr;
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = md_step_sequence(pl, pl->cap_stream, pos, vel, q, inv_mass, F, dt, flags, energies, nsteps);
        cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &graph);
        if (rc != ENUF_OK) {
            if (e == cudaSuccess) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ENUF_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&m.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            m.exec = nullptr;
            return fail(ENUF_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
        }
        m.pos = pos;
        m.vel = vel;
        m.q = q;
        m.inv_mass = inv_mass;
        m.F = F;
        m.energies = energies;
        m.flags = flags;
        m.dt = dt;
        m.cap = nsteps;
    }
    for (int s = 0; s < nsteps; s++) CK(cudaGraphLaunch(m.exec, pl->stream));
    return ENUF_OK;
}

int enuf_plan_destroy(enuf_plan* pl)
{
    if (!pl) return ENUF_OK;
    drop_graphs(pl);
    if (pl->prof_exec) cudaGraphExecDestroy(pl->prof_exec);
    for (auto e : pl->tevents) cudaEventDestroy(e);
    if (pl->own_ws && pl->ws) cudaFree(pl->ws);
    if (pl->ev_fork) cudaEventDestroy(pl->ev_fork);
    if (pl->ev_join) cudaEventDestroy(pl->ev_join);
    if (pl->aux_stream) cudaStreamDestroy(pl->aux_stream);
    if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
    if (pl->hout) cudaFreeHost(pl->hout);
    delete pl;
    return ENUF_OK;
}

int enuf_compute(enuf_plan* pl, const void* pos, const void* q, void* F, void* phi, double* out, int flags)
{
    return compute_impl(pl, pos, q, F, phi, out, flags);
}

int enuf_energy_forces(enuf_plan* pl, const void* pos, const void* q, double* E_host, void* F, double* virial_host,
                       void* phi, double* parts_host, int flags)
{
    if (!pl) return fail(ENUF_EINVAL, "plan is NULL");
    double* dout = at<double>(pl, pl->lay.out);
    LCHK(compute_impl(pl, pos, q, F, phi, dout, flags));
    double hl[ENUF_NOUT];
    double* h = pl->hout ? pl->hout : hl;  // pinned: the copy queues behind the evaluation
    CK(cudaMemcpyAsync(h, dout, ENUF_NOUT * sizeof(double), cudaMemcpyDeviceToHost, pl->stream));
    CK(cudaStreamSynchronize(pl->stream));
    if (E_host) *E_host = h[ENUF_OUT_E];
    if (virial_host) std::memcpy(virial_host, h + ENUF_OUT_VIRIAL, 9 * sizeof(double));
    if (parts_host) std::memcpy(parts_host, h, ENUF_NOUT * sizeof(double));
    return check_status(h);
}

int enuf_energy_forces_host(enuf_plan* pl, const void* pos_host, const void* q_host, double* E_host, void* F_host,
                            double* virial_host, void* phi_host, int flags)
{
    if (!pl || !pl->ws) return fail(ENUF_EINVAL, "plan is NULL or has no workspace");
    if (!pos_host || !q_host) return fail(ENUF_EINVAL, "pos_host and q_host are required");
    const size_t N = (size_t)pl->r.prm.N, rs = pl->r.rsz;
    const Layout& y = pl->lay;
    void* F = F_host ? (void*)(pl->ws + y.s_F) : nullptr;
    void* phi = (phi_host && (flags & ENUF_WANT_PHI)) ? (void*)(pl->ws + y.s_phi) : nullptr;
    if ((flags & ENUF_WANT_PHI) && !phi) flags &= ~ENUF_WANT_PHI;
    double* dout = at<double>(pl, y.out);
    if (flags & ~(ENUF_WANT_VIRIAL | ENUF_WANT_PHI | ENUF_REMOVE_NET_FORCE | ENUF_KSPACE_ONLY | ENUF_AD_FORCES))
        return fail(ENUF_EINVAL, "unknown flag bits");
    if (pl->use_graph && !pl->profile && pl->hout && host_pinned(pos_host) && host_pinned(q_host) &&
        host_pinned(F_host) && host_pinned(phi ? phi_host : nullptr)) {
        // one graph launch and one synchronisation per call
        LCHK(host_graph_call(pl, pos_host, q_host, F_host, phi ? phi_host : nullptr, flags, F, phi, dout));
        CK(cudaStreamSynchronize(pl->stream));
        const double* h = pl->hout;
        if (E_host) *E_host = h[ENUF_OUT_E];
        if (virial_host) std::memcpy(virial_host, h + ENUF_OUT_VIRIAL, 9 * sizeof(double));
        return check_status(h);
    }
    CK(cudaMemcpyAsync(pl->ws + y.s_pos, pos_host, 3 * N * rs, cudaMemcpyHostToDevice, pl->stream));
    CK(cudaMemcpyAsync(pl->ws + y.s_q, q_host, N * rs, cudaMemcpyHostToDevice, pl->stream));
    LCHK(compute_impl(pl, pl->ws + y.s_pos, pl->ws + y.s_q, F, phi, dout, flags));
    // every copy queued behind the evaluation, one synchronisation (the
    // results go to the plan's pinned buffer: a copy into pageable memory
    // would return only when it is done)
    if (F_host) CK(cudaMemcpyAsync(F_host, F, 3 * N * rs, cudaMemcpyDeviceToHost, pl->stream));
    if (phi) CK(cudaMemcpyAsync(phi_host, phi, N * rs, cudaMemcpyDeviceToHost, pl->stream));
    double hl[ENUF_NOUT];
    double* h = pl->hout ? pl->hout : hl;
    CK(cudaMemcpyAsync(h, dout, ENUF_NOUT * sizeof(double), cudaMemcpyDeviceToHost, pl->stream));
    CK(cudaStreamSynchronize(pl->stream));
    if (E_host) *E_host = h[ENUF_OUT_E];
    if (virial_host) std::memcpy(virial_host, h + ENUF_OUT_VIRIAL, 9 * sizeof(double));
    return check_status(h);
}

int enuf_backward_flags(enuf_plan* pl, const void* pos, const void* q, const double* gE, void* dpos, void* dq,
                        int flags)
{
    if (!pl || !pl->ws) return fail(ENUF_EINVAL, "plan is NULL or has no workspace");
    if (flags & ~ENUF_AD_FORCES) return fail(ENUF_EINVAL, "only ENUF_AD_FORCES is accepted");
    const Layout& y = pl->lay;
    void* F = pl->ws + y.s_F;
    void* phi = pl->ws + y.s_phi;
    LCHK(compute_impl(pl, pos, q, F, phi, at<double>(pl, y.out), ENUF_WANT_PHI | flags));
    const int N = (int)pl->r.prm.N, nb = (N + 255) / 256;
    if (pl->r.fp64)
        k_backward_scale<double><<<nb, 256, 0, pl->stream>>>(N, (const double*)F, (const double*)phi, gE, (double*)dpos,
                                                             (double*)dq);
    else
        k_backward_scale<float><<<nb, 256, 0, pl->stream>>>(N, (const float*)F, (const float*)phi, gE, (float*)dpos,
                                                           (float*)dq);
    CK(cudaGetLastError());
    return ENUF_OK;
}

int enuf_backward(enuf_plan* pl, const void* pos, const void* q, const double* gE, void* dpos, void* dq)
{
    return enuf_backward_flags(pl, pos, q, gE, dpos, dq, 0);
}

int enuf_last_timings(enuf_plan* pl, const char** names, float* times_ms, int cap)
{
    if (!pl) return fail(ENUF_EINVAL, "plan is NULL");
    const int n = (int)pl->tnames.size();
    if (!pl->profile || n == 0) return 0;
    CK(cudaEventSynchronize(pl->tevents[n]));
    pl->ttimes.assign(n, 0.f);
    for (int i = 0; i < n; i++) cudaEventElapsedTime(&pl->ttimes[i], pl->tevents[i], pl->tevents[i + 1]);
    const int m = std::min(n, cap);
    for (int i = 0; i < m; i++) {
        if (names) names[i] = pl->tnames[i].c_str();
        if (times_ms) times_ms[i] = pl->ttimes[i];
    }
    return m;
}

int enuf_structure_factor(enuf_plan* pl, const void* pos, const void* q, void* S)
{
    if (!pl || !pl->ws) return fail(ENUF_EINVAL, "plan is NULL or has no workspace");
    if (!pos || !q || !S) return fail(ENUF_EINVAL, "pos, q and S are required");
    LCHK(prepare_attrs(pl));
    Launcher L{pl, pl->stream, false};
    int rc = pl->r.fp64 ? launch_sequence<double>(L, pl, (const double*)pos, (const double*)q, nullptr, nullptr,
                                                  nullptr, ENUF_KSPACE_ONLY, S)
                        : launch_sequence<float>(L, pl, (const float*)pos, (const float*)q, nullptr, nullptr,
                                                 nullptr, ENUF_KSPACE_ONLY, S);
    if (rc != ENUF_OK) {
        reset_zeroed(pl);
        return rc;
    }
    // the key pass records non-finite inputs in the status word, which the
    // assembly of an evaluation would otherwise read and clear
    int st = 0;
    CK(cudaMemcpyAsync(&st, pl->ws + pl->lay.status, sizeof(int), cudaMemcpyDeviceToHost, pl->stream));
    CK(cudaStreamSynchronize(pl->stream));
    if (st) {
        CK(cudaMemsetAsync(pl->ws + pl->lay.status, 0, sizeof(int), pl->stream));
        CK(cudaStreamSynchronize(pl->stream));
        if (st & ST_NONFINITE) return fail(ENUF_ENONFINITE, "a position or charge is NaN or infinite");
        return fail(ENUF_EDEVICE, "a kernel reported internal status " + std::to_string(st));
    }
    return ENUF_OK;
}

int enuf_fft_forward(enuf_plan* pl, const void* grid, void* ghat)
{
    if (!pl || !pl->ws) return fail(ENUF_EINVAL, "plan is NULL or has no workspace");
    if (!grid || !ghat) return fail(ENUF_EINVAL, "grid and ghat are required");
    LCHK(prepare_attrs(pl));
    const size_t M = (size_t)pl->r.prm.M;
    // the forward passes read the plan's grid buffer (and leave it zeroed)
    CK(cudaMemcpyAsync(pl->ws + pl->lay.grid, grid, M * M * M * pl->r.rsz, cudaMemcpyDeviceToDevice, pl->stream));
    Launcher L{pl, pl->stream, false};
    int rc = pl->r.fp64 ? launch_fft_chain<double>(L, pl, 0, ghat, 0) : launch_fft_chain<float>(L, pl, 0, ghat, 0);
    if (rc != ENUF_OK) reset_zeroed(pl);
    return rc;
}

int enuf_bounds_checked(void)
{
#ifdef ENUF_BOUNDS_CHECK
    return 1;
#else
    return 0;
#endif
}

int enuf_bounds_status(unsigned long long* fails, char* where, int where_len, int clear)
{
    if (!fails) return fail(ENUF_EINVAL, "fails is NULL");
    *fails = 0;
    if (where && where_len > 0) where[0] = 0;
#ifdef ENUF_BOUNDS_CHECK
    CK(cudaDeviceSynchronize());
    BoundsLog log;
    CK(cudaMemcpyFromSymbol(&log, g_bounds, sizeof(log)));
    *fails = log.fails;
    if (log.fails && where && where_len > 0) {
        log.file[sizeof(log.file) - 1] = 0;
        snprintf(where, (size_t)where_len, "%s:%d index %lld of %lld", log.file, log.line, log.index, log.extent);
    }
    if (clear) {
        const BoundsLog zero{};
        CK(cudaMemcpyToSymbol(g_bounds, &zero, sizeof(zero)));
    }
#else
    (void)clear;
#endif
    return ENUF_OK;
}

#ifdef ENUF_BOUNDS_CHECK
// n + 2 threads write a buffer of n + 2 elements through checks against n:
// the last two writes must be refused and recorded (the buffer has room
// for them, so the test stays in bounds even if the checks did not work).
__global__ void k_bounds_selftest(int* buf, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n + 2 && ENUF_IN(i, n)) buf[i] = 1;
}
#endif

int enuf_bounds_selftest(void)
{
#ifdef ENUF_BOUNDS_CHECK
    constexpr int n = 1000;
    int* d = nullptr;
    CK(cudaMalloc(&d, (n + 2) * sizeof(int)));
    std::vector<int> h(n + 2, 0);
    const BoundsLog zero{};
    cudaError_t e = cudaMemset(d, 0, (n + 2) * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bounds, &zero, sizeof(zero));
    if (e == cudaSuccess) {
        k_bounds_selftest<<<(n + 2 + 255) / 256, 256>>>(d, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), d, (n + 2) * sizeof(int), cudaMemcpyDeviceToHost);
    BoundsLog log{};
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&log, g_bounds, sizeof(log));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bounds, &zero, sizeof(zero));
    cudaFree(d);
    if (e != cudaSuccess) return fail(ENUF_ECUDA, std::string("bounds self-test: ") + cudaGetErrorString(e));
    int written = 0;
    for (int i = 0; i < n; i++) written += h[i];
    if (written != n || h[n] != 0 || h[n + 1] != 0 || log.fails != 2 || log.extent != n ||
        (log.index != n && log.index != n + 1))
        return fail(ENUF_EDEVICE, "bounds self-test: the checks did not refuse and record the two writes");
    return ENUF_OK;
#else
    return fail(ENUF_EINVAL, "the library was built without bounds checks");
#endif
}

int enuf_launch_count(enuf_plan* pl, int flags, int with_forces)
{
    if (!pl || !pl->ws) return fail(ENUF_EINVAL, "plan is NULL or has no workspace");
    int n = 0;
    void* d = pl->ws;
    int rc = run_sequence(pl, pl->stream, true, d, d, with_forces ? d : nullptr, (flags & ENUF_WANT_PHI) ? d : nullptr,
                          nullptr, flags, &n);
    return rc == ENUF_OK ? n : rc;
}

}  // extern "C"
