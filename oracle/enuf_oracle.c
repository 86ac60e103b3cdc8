/*
 * enuf_oracle.c -- plain FP64 CPU oracle for the ENUF method (Ewald summation
 * with the reciprocal-space sum evaluated by non-uniform FFTs).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite,
 * __graft_entry__.smoke() and the CPU-baseline leg of bench.py may load it.
 * It shares no source, header, table or constant with the CUDA library.
 *
 * Two oracles live here (Yang et al., "The ENUF method", arXiv:2004.12484):
 *
 *   O1  direct Ewald (Sec. 2.1): real-space erfc pair sum (Eq. 17, force
 *       Eq. 29 in its textbook form), reciprocal sum over an explicit set of
 *       wave vectors with S(k) = sum_j q_j exp(-i k.r_j) (Eq. 22, 25, 26),
 *       self energy (Eq. 24), reciprocal force from the gradient of Eq. 22
 *       (Eq. 39-41).
 *
 *   O2  plain NFFT-Ewald (Sec. 2.3 and 3.1): the structure factor of Eq. 37 is
 *       obtained as a transposed NFFT (Eq. 36): spread the charges with a
 *       Gaussian window onto an equispaced grid, FFT, scale by the window's
 *       Fourier coefficients; the energy follows Eq. 38; the force follows
 *       Eq. 41-42 as a conjugated NFFT (Eq. 35) of g_n = n G S(n): subdivide
 *       (place on the grid, scaled), inverse FFT, interpolate with the same
 *       window.
 *
 * Readings of the paper that the text leaves open (each one is a decision,
 * listed again in the design notes):
 *   - S uses exp(-i k.r) (Eq. 26, 37); Eq. 22's exp(+i k.r) gives the same
 *     energy.
 *   - The window is the Gaussian of the NFFT literature, in grid units
 *     phi(u) = (pi b)^(-1/2) exp(-u^2/b), b = 2 sigma m / ((2 sigma - 1) pi),
 *     m = p/2, sigma = M / (2 n_c), truncated to the p grid points
 *     l = floor(u) - m + 1 ... floor(u) + m.  Its continuous Fourier
 *     transform times M is exp(-b pi^2 n^2 / M^2).
 *   - The frequency set is the symmetric cube |n_t| <= n_c, n != 0, with
 *     n_c < M/2 (Eq. 33 read as symmetric so that S(-n) = conj S(n) pairs are
 *     complete).
 *   - Units: energies carry the factor ke = 1/(4 pi eps0) (1 in Gaussian
 *     units).  Orthorhombic boxes use k = 2 pi (n_x/L_x, n_y/L_y, n_z/L_z);
 *     for a cube this is exactly Eq. 38 and Eq. 42.
 *   - A non-neutral system gets the uniform-background term
 *     -ke pi Q^2 / (2 V alpha^2) (the paper assumes neutrality).
 *   - Virial: the textbook Ewald pressure tensor, W_ab = -dE/d(eps_ab).
 *
 * All arithmetic is IEEE double.  Loops are the definitions written out; the
 * only parallelism is OpenMP over independent outputs, which does not change
 * any sum's order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* small helpers                                                        */
/* ------------------------------------------------------------------ */

/* Fractional coordinate in [0,1): x - floor(x), with a result that rounds up
 * to 1.0 folded back to 0. */
static double wrap01(double x)
{
    double w = x - floor(x);
    if (w >= 1.0) w = 0.0;
    return w;
}

static int64_t imod(int64_t a, int64_t m)
{
    int64_t r = a % m;
    return r < 0 ? r + m : r;
}

/* ------------------------------------------------------------------ */
/* Gaussian window of the NFFT (Sec. 2.2, Sec. 3.1: "Gaussian window")  */
/* ------------------------------------------------------------------ */

/* Shape parameter b for oversampling sigma = M/(2 n_c) and m = p/2. */
double orc_window_b(int M, int n_c, int p)
{
    double sigma = (double)M / (2.0 * (double)n_c);
    double m = 0.5 * (double)p;
    return 2.0 * sigma * m / ((2.0 * sigma - 1.0) * M_PI);
}

/* phi(u) in grid units. */
double orc_window(double u, double b)
{
    return exp(-u * u / b) / sqrt(M_PI * b);
}

/* M times the window's continuous Fourier transform at integer frequency n:
 * M c(n) = exp(-b pi^2 n^2 / M^2).  The scaling step divides by this. */
double orc_window_hat(int n, int M, double b)
{
    double t = M_PI * (double)n / (double)M;
    return exp(-b * t * t);
}

/* ------------------------------------------------------------------ */
/* FFT: recursive radix-2 decimation in time, in place on interleaved   */
/* complex doubles.  sign = -1: sum_l x_l exp(-2 pi i k l / n);         */
/* sign = +1: the same with exp(+...).  Unnormalised.  n a power of 2.  */
/* ------------------------------------------------------------------ */

static void fft_rec(int n, double *x, int sign, double *tmp)
{
    if (n == 1) return;
    int h = n / 2;
    /* split into even and odd samples */
    for (int i = 0; i < h; i++) {
        tmp[2 * i] = x[4 * i];
        tmp[2 * i + 1] = x[4 * i + 1];
        tmp[2 * (h + i)] = x[4 * i + 2];
        tmp[2 * (h + i) + 1] = x[4 * i + 3];
    }
    memcpy(x, tmp, sizeof(double) * 2 * n);
    fft_rec(h, x, sign, tmp);
    fft_rec(h, x + 2 * h, sign, tmp);
    for (int k = 0; k < h; k++) {
        double ang = sign * 2.0 * M_PI * (double)k / (double)n;
        double wr = cos(ang), wi = sin(ang);
        double er = x[2 * k], ei = x[2 * k + 1];
        double orr = x[2 * (h + k)], oi = x[2 * (h + k) + 1];
        double tr = wr * orr - wi * oi, ti = wr * oi + wi * orr;
        x[2 * k] = er + tr;
        x[2 * k + 1] = ei + ti;
        x[2 * (h + k)] = er - tr;
        x[2 * (h + k) + 1] = ei - ti;
    }
}

int orc_fft1d(int n, double *x, int sign)
{
    if (n <= 0 || (n & (n - 1)) != 0) return -1;
    double *tmp = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    if (!tmp) return -2;
    fft_rec(n, x, sign, tmp);
    free(tmp);
    return 0;
}

/* 3D transform of a complex M^3 array stored [z][y][x] (x fastest): the 1D
 * transform applied along x, then y, then z. */
int orc_fft3d(int M, double *a, int sign)
{
    if (M <= 0 || (M & (M - 1)) != 0) return -1;
    int64_t M2 = (int64_t)M * M;
    int err = 0;
    for (int axis = 0; axis < 3; axis++) {
        int64_t stride = axis == 0 ? 1 : (axis == 1 ? M : M2);
#pragma omp parallel for schedule(static) reduction(| : err)
        for (int64_t line = 0; line < M2; line++) {
            /* the two indices that are not along `axis` */
            int64_t i0 = line % M, i1 = line / M;
            int64_t base;
            if (axis == 0) base = i0 * M + i1 * M2;
            else if (axis == 1) base = i0 + i1 * M2;
            else base = i0 + i1 * M;
            double *buf = (double *)malloc(sizeof(double) * 2 * (size_t)M);
            if (!buf) { err |= 1; continue; }
            for (int64_t t = 0; t < M; t++) {
                buf[2 * t] = a[2 * (base + t * stride)];
                buf[2 * t + 1] = a[2 * (base + t * stride) + 1];
            }
            err |= orc_fft1d(M, buf, sign) != 0;
            for (int64_t t = 0; t < M; t++) {
                a[2 * (base + t * stride)] = buf[2 * t];
                a[2 * (base + t * stride) + 1] = buf[2 * t + 1];
            }
            free(buf);
        }
    }
    return err ? -2 : 0;
}

/* ------------------------------------------------------------------ */
/* Real-space pair sum, Eq. 17 (energy) and Eq. 29 (force, textbook    */
/* form: F_i = ke q_i sum_j q_j [erfc(a r)/r + 2a/sqrt(pi) e^{-a^2 r^2}]  */
/*                       r_ij / r^2, r_ij = r_i - r_j).                */
/* Every periodic image with |r_ij + n L| < r_c is included.           */
/* If idx != NULL only the particles idx[0..nsub) are evaluated (all j  */
/* are still summed) and the energy/virial outputs are not written.    */
/* ------------------------------------------------------------------ */
/* ENUF-DPD correction factors of Slater-type smeared charges (Eq. 51-58):
 * with x = r / lambda_e,
 *   B_U = 1 - (1 + x) exp(-2x)                (energy, Eq. 57),
 *   B_F = 1 - (1 + 2x (1 + x)) exp(-2x)       (force, Eq. 58);
 * the pair energy and force of two such charges are the point-charge ones
 * times B_U and B_F (Eq. 53-56). */
void orc_slater_factors(double r, double lambda_e, double *BU, double *BF)
{
    double x = r / lambda_e, e = exp(-2.0 * x);
    *BU = 1.0 - (1.0 + x) * e;
    *BF = 1.0 - (1.0 + 2.0 * x * (1.0 + x)) * e;
}

/* Real-space sum; lambda_e > 0 applies the ENUF-DPD factors to each pair's
 * erfc terms (the real-space part of the smeared-charge interaction within
 * r_c, the method's r_c = 3 R_c); lambda_e = 0 is the point-charge sum.
 * Two distinct smeared charges at the same point interact with the finite
 * limit of Eq. 59 (erfc(0) B_U/r -> 1/lambda_e) and no force (Eq. 60). */
static int real_space_core(int64_t N, const double *pos, const double *q, const double *L,
                           double alpha, double rc, double ke, double lambda_e,
                           int64_t nsub, const int64_t *idx,
                           double *E, double *F, double *phi, double *vir)
{
    /* the nearest-image vector has |d_t| <= L_t/2, so image shells up to
     * |n_t| <= floor(r_c/L_t + 1/2) can lie inside the cutoff */
    int nimg[3];
    for (int t = 0; t < 3; t++) nimg[t] = (int)floor(rc / L[t] + 0.5);
    const double two_a_sqpi = 2.0 * alpha / sqrt(M_PI);
    const double rc2 = rc * rc;
    int64_t count = idx ? nsub : N;
    double Esum = 0.0, W[9] = {0};

#pragma omp parallel
    {
        double Eloc = 0.0, Wloc[9] = {0};
#pragma omp for schedule(dynamic, 16)
        for (int64_t s = 0; s < count; s++) {
            int64_t i = idx ? idx[s] : s;
            double fi[3] = {0, 0, 0}, ph = 0.0;
            for (int64_t j = 0; j < N; j++) {
                double d0[3];
                for (int t = 0; t < 3; t++) {
                    /* nearest image first, then the image shells around it */
                    double d = pos[3 * i + t] - pos[3 * j + t];
                    d0[t] = d - L[t] * floor(d / L[t] + 0.5);
                }
                for (int a = -nimg[0]; a <= nimg[0]; a++)
                for (int b = -nimg[1]; b <= nimg[1]; b++)
                for (int c = -nimg[2]; c <= nimg[2]; c++) {
                    if (j == i && a == 0 && b == 0 && c == 0) continue;
                    double dx = d0[0] + a * L[0], dy = d0[1] + b * L[1], dz = d0[2] + c * L[2];
                    double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 >= rc2) continue;
                    double e, fs;
                    if (r2 == 0.0) {
                        if (!(lambda_e > 0.0)) continue;  /* coincident point charges: no finite term */
                        e = 1.0 / lambda_e;
                        fs = 0.0;
                    } else {
                        double r = sqrt(r2);
                        e = erfc(alpha * r) / r;
                        fs = ke * q[i] * q[j] * (e + two_a_sqpi * exp(-alpha * alpha * r2)) / r2;
                        if (lambda_e > 0.0) {
                            double BU, BF;
                            orc_slater_factors(r, lambda_e, &BU, &BF);
                            e *= BU;
                            fs *= BF;
                        }
                    }
                    fi[0] += fs * dx; fi[1] += fs * dy; fi[2] += fs * dz;
                    ph += ke * q[j] * e;
                    /* each unordered pair is seen twice (from i and from j):
                     * half of the pair energy and virial per visit */
                    Eloc += 0.5 * ke * q[i] * q[j] * e;
                    double dv[3] = {dx, dy, dz}, fv[3] = {fs * dx, fs * dy, fs * dz};
                    for (int u = 0; u < 3; u++)
                        for (int v = 0; v < 3; v++) Wloc[3 * u + v] += 0.5 * dv[u] * fv[v];
                }
            }
            if (F) { F[3 * s] = fi[0]; F[3 * s + 1] = fi[1]; F[3 * s + 2] = fi[2]; }
            if (phi) phi[s] = ph;
        }
#pragma omp critical
        {
            Esum += Eloc;
            for (int u = 0; u < 9; u++) W[u] += Wloc[u];
        }
    }
    if (!idx) {
        if (E) *E = Esum;
        if (vir) for (int u = 0; u < 9; u++) vir[u] = W[u];
    }
    return 0;
}

int orc_real_space(int64_t N, const double *pos, const double *q, const double *L,
                   double alpha, double rc, double ke,
                   int64_t nsub, const int64_t *idx,
                   double *E, double *F, double *phi, double *vir)
{
    return real_space_core(N, pos, q, L, alpha, rc, ke, 0.0, nsub, idx, E, F, phi, vir);
}

int orc_real_space_slater(int64_t N, const double *pos, const double *q, const double *L,
                          double alpha, double rc, double ke, double lambda_e,
                          int64_t nsub, const int64_t *idx,
                          double *E, double *F, double *phi, double *vir)
{
    if (!(lambda_e > 0.0)) return -1;
    return real_space_core(N, pos, q, L, alpha, rc, ke, lambda_e, nsub, idx, E, F, phi, vir);
}

/* ------------------------------------------------------------------ */
/* Self energy (Eq. 24) and the neutralising-background term.          */
/* ------------------------------------------------------------------ */
void orc_self_and_background(int64_t N, const double *q, const double *L, double alpha, double ke,
                             double *E_self, double *E_bg, double *Q_out)
{
    double s2 = 0.0, Q = 0.0;
    for (int64_t j = 0; j < N; j++) { s2 += q[j] * q[j]; Q += q[j]; }
    double V = L[0] * L[1] * L[2];
    *E_self = -ke * alpha / sqrt(M_PI) * s2;
    *E_bg = -ke * M_PI * Q * Q / (2.0 * V * alpha * alpha);
    if (Q_out) *Q_out = Q;
}

/* ------------------------------------------------------------------ */
/* Reciprocal part, shared constants                                   */
/* ------------------------------------------------------------------ */

/* k = 2 pi (n_x/L_x, n_y/L_y, n_z/L_z); G(k) = exp(-k^2/4a^2)/k^2 (Eq. 22). */
static void wave_vector(const int n[3], const double *L, double k[3])
{
    for (int t = 0; t < 3; t++) k[t] = 2.0 * M_PI * (double)n[t] / L[t];
}

static double green(const double k[3], double alpha)
{
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    return exp(-k2 / (4.0 * alpha * alpha)) / k2;
}

/* Adds one wave vector's energy and virial contribution (2 pi/V) G |S|^2
 * (delta_ab - 2 k_a k_b (1/k^2 + 1/4a^2)). */
static void add_energy_virial(const double k[3], double G, double S2, double pref,
                              double alpha, double *E, double *W)
{
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    double e = pref * G * S2;
    *E += e;
    double c = 2.0 * (1.0 / k2 + 1.0 / (4.0 * alpha * alpha));
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) W[3 * a + b] += e * ((a == b ? 1.0 : 0.0) - c * k[a] * k[b]);
}

/* ------------------------------------------------------------------ */
/* O1 reciprocal part, direct: explicit sum over wave vectors.         */
/* Set: cube |n_t| <= nmax (sphere = 0) or sphere |n| <= nmax (1).     */
/* Phase factors by Euler recurrence exp(i 2 pi n x) = (exp(i 2 pi x))^n */
/* per dimension.  F_i (Eq. 41) = ke (4 pi q_i / V) sum_k k G Im{S e^{ik.r_i}}, */
/* phi_i = ke (4 pi / V) sum_k G Re{S e^{ik.r_i}} (so E = 1/2 sum q phi). */
/* ------------------------------------------------------------------ */
int orc_kspace_direct(int64_t N, const double *pos, const double *q, const double *L,
                      double alpha, double ke, int nmax, int sphere,
                      double *E, double *F, double *phi, double *vir,
                      int64_t nsub, const int64_t *idx)
{
    int nn = 2 * nmax + 1;
    double V = L[0] * L[1] * L[2];
    /* enumerate the wave vectors of the set */
    int64_t K = 0;
    int *nlist = (int *)malloc(sizeof(int) * 3 * (size_t)nn * nn * nn);
    if (!nlist) return -2;
    for (int a = -nmax; a <= nmax; a++)
        for (int b = -nmax; b <= nmax; b++)
            for (int c = -nmax; c <= nmax; c++) {
                if (a == 0 && b == 0 && c == 0) continue;
                if (sphere && a * a + b * b + c * c > nmax * nmax) continue;
                nlist[3 * K] = a; nlist[3 * K + 1] = b; nlist[3 * K + 2] = c;
                K++;
            }
    double *S = (double *)calloc(2 * (size_t)K, sizeof(double));
    if (!S) { free(nlist); return -2; }

    /* S(k) = sum_j q_j exp(-i k.r_j)  (Eq. 26) */
#pragma omp parallel
    {
        double *Sl = (double *)calloc(2 * (size_t)K, sizeof(double));
        double *ph = (double *)malloc(sizeof(double) * 2 * 3 * nn);
#pragma omp for schedule(static)
        for (int64_t j = 0; j < N; j++) {
            for (int t = 0; t < 3; t++) {
                double x = pos[3 * j + t] / L[t];
                double cr = cos(2.0 * M_PI * x), ci = -sin(2.0 * M_PI * x); /* exp(-i 2 pi x) */
                double *pt = ph + 2 * t * nn;
                pt[2 * nmax] = 1.0; pt[2 * nmax + 1] = 0.0;
                for (int n = 1; n <= nmax; n++) {
                    double pr = pt[2 * (nmax + n - 1)], pi = pt[2 * (nmax + n - 1) + 1];
                    pt[2 * (nmax + n)] = pr * cr - pi * ci;
                    pt[2 * (nmax + n) + 1] = pr * ci + pi * cr;
                    pt[2 * (nmax - n)] = pt[2 * (nmax + n)];       /* conjugate */
                    pt[2 * (nmax - n) + 1] = -pt[2 * (nmax + n) + 1];
                }
            }
            for (int64_t kk = 0; kk < K; kk++) {
                const double *px = ph + 2 * (0 * nn + nlist[3 * kk] + nmax);
                const double *py = ph + 2 * (1 * nn + nlist[3 * kk + 1] + nmax);
                const double *pz = ph + 2 * (2 * nn + nlist[3 * kk + 2] + nmax);
                double ar = px[0] * py[0] - px[1] * py[1], ai = px[0] * py[1] + px[1] * py[0];
                double br = ar * pz[0] - ai * pz[1], bi = ar * pz[1] + ai * pz[0];
                Sl[2 * kk] += q[j] * br;
                Sl[2 * kk + 1] += q[j] * bi;
            }
        }
#pragma omp critical
        for (int64_t kk = 0; kk < 2 * K; kk++) S[kk] += Sl[kk];
        free(Sl); free(ph);
    }

    /* energy and virial, Eq. 22/25 */
    double Eacc = 0.0, W[9] = {0};
    for (int64_t kk = 0; kk < K; kk++) {
        double k[3];
        wave_vector(nlist + 3 * kk, L, k);
        double S2 = S[2 * kk] * S[2 * kk] + S[2 * kk + 1] * S[2 * kk + 1];
        add_energy_virial(k, green(k, alpha), S2, ke * 2.0 * M_PI / V, alpha, &Eacc, W);
    }
    if (E) *E = Eacc;
    if (vir) for (int u = 0; u < 9; u++) vir[u] = W[u];

    /* forces and potentials at the requested particles */
    int64_t count = idx ? nsub : N;
    if (F || phi) {
#pragma omp parallel for schedule(dynamic, 8)
        for (int64_t s = 0; s < count; s++) {
            int64_t i = idx ? idx[s] : s;
            double f[3] = {0, 0, 0}, pv = 0.0;
            for (int64_t kk = 0; kk < K; kk++) {
                double k[3];
                wave_vector(nlist + 3 * kk, L, k);
                double arg = k[0] * pos[3 * i] + k[1] * pos[3 * i + 1] + k[2] * pos[3 * i + 2];
                double er = cos(arg), ei = sin(arg);              /* exp(+i k.r_i) */
                double pr = S[2 * kk] * er - S[2 * kk + 1] * ei;   /* Re(S e^{ik.r}) */
                double pim = S[2 * kk] * ei + S[2 * kk + 1] * er;  /* Im(S e^{ik.r}) */
                double G = green(k, alpha);
                for (int t = 0; t < 3; t++) f[t] += k[t] * G * pim;
                pv += G * pr;
            }
            double c = ke * 4.0 * M_PI / V;
            if (F) for (int t = 0; t < 3; t++) F[3 * s + t] = c * q[i] * f[t];
            if (phi) phi[s] = c * pv;
        }
    }
    free(S); free(nlist);
    return 0;
}

/* Structure factor on the cube |n_t| <= nc, stored [(nz+nc)][(ny+nc)][(nx+nc)]
 * as interleaved complex: direct definition (Eq. 37). */
int orc_structure_factor_direct(int64_t N, const double *pos, const double *q, const double *L,
                                int nc, double *S)
{
    int nn = 2 * nc + 1;
    int64_t K = (int64_t)nn * nn * nn;
    memset(S, 0, sizeof(double) * 2 * (size_t)K);
#pragma omp parallel for schedule(static)
    for (int64_t kk = 0; kk < K; kk++) {
        int n[3] = {(int)(kk % nn) - nc, (int)((kk / nn) % nn) - nc, (int)(kk / ((int64_t)nn * nn)) - nc};
        double sr = 0.0, si = 0.0;
        for (int64_t j = 0; j < N; j++) {
            double arg = 0.0;
            for (int t = 0; t < 3; t++) arg += 2.0 * M_PI * (double)n[t] * pos[3 * j + t] / L[t];
            sr += q[j] * cos(arg);
            si -= q[j] * sin(arg);
        }
        S[2 * kk] = sr; S[2 * kk + 1] = si;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* O2: plain NFFT-Ewald reciprocal part (Sec. 2.3.1, Sec. 3.1).        */
/* ------------------------------------------------------------------ */

/* Window weights of one particle along one axis: the p grid indices
 * l = floor(u) - m + 1 + a (a = 0..p-1, not yet reduced mod M) and
 * phi(u - l). */
static void particle_window(double u, int p, double b, int64_t *l0, double *w)
{
    int m = p / 2;
    int64_t f = (int64_t)floor(u);
    *l0 = f - m + 1;
    for (int a = 0; a < p; a++) w[a] = orc_window(u - (double)(*l0 + a), b);
}

/* Spreading step: g_l = sum_j q_j prod_t phi(u_{j,t} - l_t) on the
 * periodic M^3 grid (real values stored in a complex array). */
int orc_spread(int64_t N, const double *pos, const double *q, const double *L,
               int M, int p, double b, double *grid /* complex M^3 */)
{
    int64_t M2 = (int64_t)M * M;
    memset(grid, 0, sizeof(double) * 2 * (size_t)(M2 * M));
    double wx[64], wy[64], wz[64];
    if (p > 64) return -1;
    for (int64_t j = 0; j < N; j++) {
        int64_t lx, ly, lz;
        particle_window(M * wrap01(pos[3 * j] / L[0]), p, b, &lx, wx);
        particle_window(M * wrap01(pos[3 * j + 1] / L[1]), p, b, &ly, wy);
        particle_window(M * wrap01(pos[3 * j + 2] / L[2]), p, b, &lz, wz);
        for (int c = 0; c < p; c++)
            for (int bb = 0; bb < p; bb++)
                for (int a = 0; a < p; a++) {
                    int64_t cell = imod(lx + a, M) + M * imod(ly + bb, M) + M2 * imod(lz + c, M);
                    grid[2 * cell] += q[j] * wx[a] * wy[bb] * wz[c];
                }
    }
    return 0;
}

/* Interpolation step: value_j = sum_l prod_t phi(u_{j,t} - l_t) a_l for a
 * complex grid a; writes the complex result. */
static void interpolate(int64_t N, const double *pos, const double *L, int M, int p, double b,
                        const double *a, double *out)
{
    int64_t M2 = (int64_t)M * M;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; j++) {
        double wx[64], wy[64], wz[64];
        int64_t lx, ly, lz;
        particle_window(M * wrap01(pos[3 * j] / L[0]), p, b, &lx, wx);
        particle_window(M * wrap01(pos[3 * j + 1] / L[1]), p, b, &ly, wy);
        particle_window(M * wrap01(pos[3 * j + 2] / L[2]), p, b, &lz, wz);
        double sr = 0.0, si = 0.0;
        for (int c = 0; c < p; c++)
            for (int bb = 0; bb < p; bb++)
                for (int aa = 0; aa < p; aa++) {
                    int64_t cell = imod(lx + aa, M) + M * imod(ly + bb, M) + M2 * imod(lz + c, M);
                    double w = wx[aa] * wy[bb] * wz[c];
                    sr += w * a[2 * cell];
                    si += w * a[2 * cell + 1];
                }
        out[2 * j] = sr;
        out[2 * j + 1] = si;
    }
}

/* Transposed NFFT (Eq. 36): S~(n) on the cube |n_t| <= nc, same storage as
 * orc_structure_factor_direct.  Spread, forward FFT, scale by 1/(M c(n)). */
int orc_structure_factor_nfft(int64_t N, const double *pos, const double *q, const double *L,
                              int M, int p, int nc, double *S)
{
    if (2 * nc >= M || p > M) return -1;
    int64_t M2 = (int64_t)M * M;
    double b = orc_window_b(M, nc, p);
    double *grid = (double *)malloc(sizeof(double) * 2 * (size_t)(M2 * M));
    if (!grid) return -2;
    orc_spread(N, pos, q, L, M, p, b, grid);
    orc_fft3d(M, grid, -1);
    int nn = 2 * nc + 1;
    for (int c = -nc; c <= nc; c++)
        for (int bb = -nc; bb <= nc; bb++)
            for (int a = -nc; a <= nc; a++) {
                int64_t cell = imod(a, M) + M * imod(bb, M) + M2 * imod(c, M);
                double scale = 1.0 / (orc_window_hat(a, M, b) * orc_window_hat(bb, M, b) * orc_window_hat(c, M, b));
                int64_t o = (int64_t)(a + nc) + nn * ((int64_t)(bb + nc) + nn * (int64_t)(c + nc));
                S[2 * o] = scale * grid[2 * cell];
                S[2 * o + 1] = scale * grid[2 * cell + 1];
            }
    free(grid);
    return 0;
}

/* Full O2 reciprocal evaluation: E_K (Eq. 38), virial, F^K (Eq. 41-42) and
 * the reciprocal potential phi^K at every particle. */
int orc_kspace_nfft(int64_t N, const double *pos, const double *q, const double *L,
                    double alpha, double ke, int M, int p, int nc,
                    double *E, double *F, double *phi, double *vir)
{
    if (2 * nc >= M || p > M || p < 2 || (p & 1)) return -1;
    int64_t M2 = (int64_t)M * M, M3 = M2 * M;
    double b = orc_window_b(M, nc, p);
    double V = L[0] * L[1] * L[2];

    /* forward: spreading, FFT, scaling -> S~(n) (Eq. 36-37) */
    double *grid = (double *)malloc(sizeof(double) * 2 * (size_t)M3);
    /* four conjugated-NFFT inputs: the three components of g_n and the
     * potential's coefficients */
    double *ga[4];
    for (int f = 0; f < 4; f++) ga[f] = (double *)calloc(2 * (size_t)M3, sizeof(double));
    double *val = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    if (!grid || !ga[0] || !ga[1] || !ga[2] || !ga[3] || !val) return -2;
    orc_spread(N, pos, q, L, M, p, b, grid);
    orc_fft3d(M, grid, -1);

    double Eacc = 0.0, W[9] = {0};
    for (int c = -nc; c <= nc; c++)
        for (int bb = -nc; bb <= nc; bb++)
            for (int a = -nc; a <= nc; a++) {
                if (a == 0 && bb == 0 && c == 0) continue;
                int n[3] = {a, bb, c};
                int64_t cell = imod(a, M) + M * imod(bb, M) + M2 * imod(c, M);
                double chat = orc_window_hat(a, M, b) * orc_window_hat(bb, M, b) * orc_window_hat(c, M, b);
                double Sr = grid[2 * cell] / chat, Si = grid[2 * cell + 1] / chat;
                double k[3];
                wave_vector(n, L, k);
                double G = green(k, alpha);
                /* Eq. 38 (general box form ke 2pi/V G|S|^2) */
                add_energy_virial(k, G, Sr * Sr + Si * Si, ke * 2.0 * M_PI / V, alpha, &Eacc, W);
                /* subdividing: g_n = k G S(n) (Eq. 41, in k units), divided
                 * by the window's coefficient so that the interpolation
                 * returns sum_n g_n exp(2 pi i n.x_j) */
                for (int t = 0; t < 3; t++) {
                    ga[t][2 * cell] = k[t] * G * Sr / chat;
                    ga[t][2 * cell + 1] = k[t] * G * Si / chat;
                }
                ga[3][2 * cell] = G * Sr / chat;
                ga[3][2 * cell + 1] = G * Si / chat;
            }
    if (E) *E = Eacc;
    if (vir) for (int u = 0; u < 9; u++) vir[u] = W[u];

    /* inverse: inverse FFT, interpolating; F = ke 4 pi q/V Im(g_j)
     * (Eq. 42), phi = ke 4 pi/V Re(sum G S e^{2 pi i n.x}) */
    double cF = ke * 4.0 * M_PI / V;
    for (int f = 0; f < 4; f++) {
        if (f < 3 && !F) continue;
        if (f == 3 && !phi) continue;
        orc_fft3d(M, ga[f], +1);
        interpolate(N, pos, L, M, p, b, ga[f], val);
        for (int64_t j = 0; j < N; j++) {
            if (f < 3) F[3 * j + f] = cF * q[j] * val[2 * j + 1];
            else phi[j] = cF * val[2 * j];
        }
    }
    free(grid); free(val);
    for (int f = 0; f < 4; f++) free(ga[f]);
    (void)M2;
    return 0;
}

/* ------------------------------------------------------------------ */
/* O2-ad: the same reciprocal energy with forces by analytic             */
/* differentiation.  E~ of Eq. 38 depends on r_j only through the window */
/* values phi(u_{j,t} - l_t), u_{j,t} = M x_{j,t}/L_t, so its gradient is */
/*   dE~/dx_{j,t} = q_j (ke 4 pi/V) (M/L_t) sum_l d_t[prod_s phi] A_l,    */
/* with A_l = sum_n G(k_n) S~(n)/(M c(n)) exp(2 pi i n.l/M) the potential  */
/* on the grid (one inverse FFT instead of the three of Eq. 41-42).  The  */
/* forces F = -grad E~ are then the exact gradient of the approximated    */
/* energy, the variant beside the ik forces of Eq. 41-42.                */
/* ------------------------------------------------------------------ */

/* d phi/du in grid units: -(2u/b) phi(u). */
double orc_window_deriv(double u, double b)
{
    return -2.0 * u / b * orc_window(u, b);
}

int orc_kspace_nfft_ad(int64_t N, const double *pos, const double *q, const double *L,
                       double alpha, double ke, int M, int p, int nc,
                       double *E, double *F, double *phi, double *vir)
{
    if (2 * nc >= M || p > M || p < 2 || (p & 1) || p > 64) return -1;
    int64_t M2 = (int64_t)M * M, M3 = M2 * M;
    double b = orc_window_b(M, nc, p);
    double V = L[0] * L[1] * L[2];
    double *grid = (double *)malloc(sizeof(double) * 2 * (size_t)M3);
    double *A = (double *)calloc(2 * (size_t)M3, sizeof(double));
    if (!grid || !A) { free(grid); free(A); return -2; }

    /* forward: spreading, FFT, scaling (Eq. 36-37); energy and virial
     * (Eq. 38); potential coefficients G S~(n) / (M c(n)) */
    orc_spread(N, pos, q, L, M, p, b, grid);
    orc_fft3d(M, grid, -1);
    double Eacc = 0.0, W[9] = {0};
    for (int c = -nc; c <= nc; c++)
        for (int bb = -nc; bb <= nc; bb++)
            for (int a = -nc; a <= nc; a++) {
                if (a == 0 && bb == 0 && c == 0) continue;
                int n[3] = {a, bb, c};
                int64_t cell = imod(a, M) + M * imod(bb, M) + M2 * imod(c, M);
                double chat = orc_window_hat(a, M, b) * orc_window_hat(bb, M, b) * orc_window_hat(c, M, b);
                double Sr = grid[2 * cell] / chat, Si = grid[2 * cell + 1] / chat;
                double k[3];
                wave_vector(n, L, k);
                double G = green(k, alpha);
                add_energy_virial(k, G, Sr * Sr + Si * Si, ke * 2.0 * M_PI / V, alpha, &Eacc, W);
                A[2 * cell] = G * Sr / chat;
                A[2 * cell + 1] = G * Si / chat;
            }
    if (E) *E = Eacc;
    if (vir) for (int u = 0; u < 9; u++) vir[u] = W[u];

    /* one inverse FFT: the potential on the grid */
    orc_fft3d(M, A, +1);

    /* interpolation of the potential and of its gradient: the window
     * product and its three partial derivatives in u */
    double cF = ke * 4.0 * M_PI / V;
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < N; j++) {
        double w[3][64], d[3][64];
        int64_t l0[3];
        for (int t = 0; t < 3; t++) {
            double u = M * wrap01(pos[3 * j + t] / L[t]);
            particle_window(u, p, b, &l0[t], w[t]);
            for (int a = 0; a < p; a++) d[t][a] = orc_window_deriv(u - (double)(l0[t] + a), b);
        }
        double s = 0.0, g[3] = {0.0, 0.0, 0.0};
        for (int c = 0; c < p; c++)
            for (int bb = 0; bb < p; bb++)
                for (int a = 0; a < p; a++) {
                    int64_t cell = imod(l0[0] + a, M) + M * imod(l0[1] + bb, M) + M2 * imod(l0[2] + c, M);
                    double v = A[2 * cell];  /* the potential grid is real */
                    s += w[0][a] * w[1][bb] * w[2][c] * v;
                    g[0] += d[0][a] * w[1][bb] * w[2][c] * v;
                    g[1] += w[0][a] * d[1][bb] * w[2][c] * v;
                    g[2] += w[0][a] * w[1][bb] * d[2][c] * v;
                }
        if (phi) phi[j] = cF * s;
        if (F)
            for (int t = 0; t < 3; t++) F[3 * j + t] = -q[j] * cF * ((double)M / L[t]) * g[t];
    }
    free(grid);
    free(A);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Brute-force image sum (Eq. 1), spherical summation order: all image */
/* vectors n with |n| <= shell (in box units), E = 1/2 sum_n sum_{i,j}'  */
/* q_i q_j / |r_ij + nL|.  Used only to pin O1 on tiny boxes.           */
/* ------------------------------------------------------------------ */
double orc_image_sum(int64_t N, const double *pos, const double *q, const double *L,
                     double ke, int shell)
{
    double E = 0.0;
#pragma omp parallel for reduction(+ : E) schedule(dynamic, 1)
    for (int a = -shell; a <= shell; a++) {
        for (int bb = -shell; bb <= shell; bb++)
            for (int c = -shell; c <= shell; c++) {
                if (a * a + bb * bb + c * c > shell * shell) continue;
                double part = 0.0;
                for (int64_t i = 0; i < N; i++)
                    for (int64_t j = 0; j < N; j++) {
                        if (a == 0 && bb == 0 && c == 0 && i == j) continue;
                        double dx = pos[3 * i] - pos[3 * j] + a * L[0];
                        double dy = pos[3 * i + 1] - pos[3 * j + 1] + bb * L[1];
                        double dz = pos[3 * i + 2] - pos[3 * j + 2] + c * L[2];
                        part += q[i] * q[j] / sqrt(dx * dx + dy * dy + dz * dz);
                    }
                E += 0.5 * ke * part;
            }
    }
    return E;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
