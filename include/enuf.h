/*
 * enuf.h -- C ABI of the ENUF library: Ewald summation with the
 * reciprocal-space sum evaluated by non-uniform FFTs, on one NVIDIA B300.
 *
 * Method: Yang, Li, Zhu, Laaksonen, Wang, "The ENUF method -- Ewald summation
 * based on non-uniform fast Fourier transform: implementation,
 * parallelization, and application" (arXiv:2004.12484).
 *
 * Problem statement (Sec. 2.1): N point charges q_j at positions r_j in a
 * periodic orthorhombic box L_x x L_y x L_z.  The library returns the total
 * electrostatic energy
 *     E = E_real (Eq. 17) + E_recip (Eq. 22 / 38) + E_self (Eq. 24)
 *         [+ E_background = -k pi Q^2 / (2 V alpha^2) when Q = sum q != 0],
 * the forces F_i = -dE/dr_i (real part Eq. 29 in textbook form, reciprocal
 * part Eq. 41-42), optionally the potentials phi_i = dE/dq_i (Eq. 5) and the
 * virial W_ab = -dE/d eps_ab.  The reciprocal part follows Sec. 3.1:
 * spread (Gaussian window) -> 3D FFT -> scale -> energy (Eq. 38); subdivide ->
 * inverse FFT (the three force components packed in one pass) -> interpolate.
 *
 * Variants: forces by analytic differentiation of the approximated energy
 * (flag ENUF_AD_FORCES: the potential alone is transformed back and the
 * window's gradient interpolated); smeared Slater-type charges of ENUF-DPD
 * (enuf_params.slater_lambda, Eq. 51-60: real-space pair terms scaled by
 * B_U and B_F); velocity-Verlet time stepping driven by a plan (enuf_md_run).
 *
 * Conventions
 *   - Every array argument of the compute calls is a DEVICE pointer unless
 *     its name ends in _host.  Positions are N x 3 row-major (x, y, z per
 *     particle), charges N, forces N x 3, potentials N.  Element type is
 *     float for ENUF_MIXED plans and double for ENUF_FP64 plans.
 *   - Positions may lie anywhere; they are wrapped into the box.
 *   - Energies and the virial are always double.
 *   - The caller owns every input and output buffer.  A plan owns its device
 *     workspace (or borrows one given with enuf_plan_set_workspace) and a
 *     private CUDA stream used only to capture CUDA graphs.
 *   - Calls are ordered on the stream given at plan creation (or
 *     enuf_plan_set_stream); asynchronous calls return before the work ends.
 *   - Return value: 0 on success, a negative ENUF_E* code on failure; the
 *     message of the last failure on the calling thread is returned by
 *     enuf_last_error().  Outputs are undefined after a failure.
 *   - A plan is not thread safe: one host thread at a time per plan.
 */
#ifndef ENUF_H
#define ENUF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* precision */
#define ENUF_FP64 0   /* every step in IEEE double                                  */
#define ENUF_MIXED 1  /* spread, FFT, interpolate, real-space pairs in float;       */
                      /* energy/virial reductions, self, background terms in double */

/* flags (per call; OR-ed) */
#define ENUF_WANT_VIRIAL 1       /* fill the 3x3 virial                              */
#define ENUF_WANT_PHI 2          /* fill phi_i = dE/dq_i (a 4th inverse transform)    */
#define ENUF_REMOVE_NET_FORCE 4  /* subtract (1/N) sum_i F_i from every force         */
#define ENUF_KSPACE_ONLY 8       /* reciprocal part only (no real-space, self, bg)    */
/* Reciprocal forces by analytic differentiation instead of the ik scheme of
 * Eq. 41-42: one inverse transform of the potential (G S~ on the grid) and
 * the window's gradient in the interpolation, F_i = -q_i grad phi~(r_i).  The
 * forces are then the exact gradient of the approximated energy of Eq. 38
 * (the ik forces are not), at one inverse transform instead of three; phi
 * comes from the same grid.  Energy and virial are unchanged. */
#define ENUF_AD_FORCES 16

/* error codes */
#define ENUF_OK 0
#define ENUF_EINVAL -1       /* invalid argument                                */
#define ENUF_EUNSUPPORTED -2 /* size or option outside what the plan supports   */
#define ENUF_ENOMEM -3       /* device allocation failed                        */
#define ENUF_ECUDA -4        /* a CUDA call failed                              */
#define ENUF_ENONFINITE -5   /* a position or charge was NaN or infinite        */
#define ENUF_EDEVICE -6      /* a kernel reported an internal error             */

/* Layout of the results vector (ENUF_NOUT doubles) written by enuf_compute. */
#define ENUF_OUT_E 0         /* total energy                      */
#define ENUF_OUT_E_REAL 1    /* Eq. 17                            */
#define ENUF_OUT_E_RECIP 2   /* Eq. 38                            */
#define ENUF_OUT_E_SELF 3    /* Eq. 24                            */
#define ENUF_OUT_E_BG 4      /* neutralising background           */
#define ENUF_OUT_Q 5         /* net charge sum_i q_i              */
#define ENUF_OUT_VIRIAL 6    /* 9 entries, row-major W_ab         */
#define ENUF_OUT_STATUS 15   /* 0 ok, else the kernels' status bits (as a double) */
#define ENUF_NOUT 16

typedef struct enuf_params {
    double L[3];       /* box edges (> 0)                                        */
    int64_t N;         /* number of particles, 1 <= N < 2^31                     */
    double alpha;      /* Ewald splitting parameter alpha = 1/(sqrt(2) sigma)    */
    double r_c;        /* real-space cutoff, 0 < r_c <= min(L)/2                 */
    int M;             /* FFT grid edge, a power of two in [8, 512]              */
    int p;             /* window support points per dimension, even, 2..12, <= M */
    int n_c;           /* reciprocal cutoff |n_t| <= n_c; 0 selects M/4;         */
                       /* must satisfy 1 <= n_c < M/2                            */
    int precision;     /* ENUF_FP64 or ENUF_MIXED                                */
    double coulomb_k;  /* 1/(4 pi eps0) in the caller's units; 0 selects 1.0     */
    int flags;         /* reserved, must be 0                                    */
    double slater_lambda; /* ENUF-DPD smeared charges (Eq. 51): decay length   */
                       /* lambda_e > 0 of the Slater-type densities; each      */
                       /* real-space pair energy is scaled by B_U and each     */
                       /* pair force by B_F (Eq. 57-58), coincident charges    */
                       /* interact with the finite limit of Eq. 59; the        */
                       /* reciprocal part stays the point-charge one (the      */
                       /* method takes r_c = 3 R_c for this).  0: point charges */
} enuf_params;

typedef struct enuf_plan enuf_plan;

/* Device bytes the plan's workspace needs (lets the caller's allocator own
 * the memory; see enuf_plan_set_workspace).  Validates the parameters. */
int enuf_plan_workspace_bytes(const enuf_params* params, size_t* bytes);

/* Creates a plan.  `cuda_stream` is a cudaStream_t (NULL = legacy default
 * stream).  If `allocate` is nonzero the plan allocates its workspace with
 * cudaMalloc; otherwise enuf_plan_set_workspace must be called before the
 * first compute call.  Window constants, twiddle tables and reciprocal
 * tables are computed here in double on the host and copied to the device
 * (this call synchronises the stream). */
int enuf_plan_create(const enuf_params* params, void* cuda_stream, int allocate, enuf_plan** out);

/* Gives the plan a caller-owned device workspace of at least
 * enuf_plan_workspace_bytes() bytes, 256-byte aligned.  The plan does not
 * free it.  Drops captured graphs. */
int enuf_plan_set_workspace(enuf_plan* plan, void* dev_ptr, size_t bytes);

/* Changes the stream later calls are ordered on. */
int enuf_plan_set_stream(enuf_plan* plan, void* cuda_stream);

/* Reads back the parameters the plan resolved (n_c, coulomb_k defaults). */
int enuf_plan_get_params(const enuf_plan* plan, enuf_params* out);

/* Frees the plan, its own workspace and its graphs.  NULL is accepted. */
int enuf_plan_destroy(enuf_plan* plan);

/* Asynchronous evaluation on the plan's stream; every step of the method
 * runs in the library's kernels.  pos, q: inputs (device).  F: N x 3 output
 * (device; NULL gives the energy only).  phi: N output (device; required when
 * ENUF_WANT_PHI is set, else ignored).  out: ENUF_NOUT doubles (device, may
 * be NULL).  With ENUF_KSPACE_ONLY, F and phi hold the reciprocal parts only
 * and out[ENUF_OUT_E] is E_recip.  The work is replayed from a CUDA graph
 * captured on the first call with the same pointers and flags (set the
 * environment variable ENUF_NO_GRAPH=1 before plan creation to launch the
 * kernels directly).  Non-finite inputs and internal errors are reported in
 * out[ENUF_OUT_STATUS] and by the synchronous wrappers. */
int enuf_compute(enuf_plan* plan, const void* pos, const void* q, void* F, void* phi, double* out, int flags);

/* Synchronous wrapper of enuf_compute: device inputs/outputs, energy parts
 * returned to host memory (E_host: 1 double or NULL; virial_host: 9 doubles
 * or NULL; parts_host: ENUF_NOUT doubles or NULL).  Synchronises the plan's
 * stream and checks the status word (ENUF_ENONFINITE / ENUF_EDEVICE). */
int enuf_energy_forces(enuf_plan* plan, const void* pos, const void* q, double* E_host, void* F,
                       double* virial_host, void* phi, double* parts_host, int flags);

/* End-to-end call with HOST buffers: copies pos_host and q_host (N x 3 and N
 * elements of the plan's type, ideally page-locked) to plan-owned device
 * buffers, computes, and copies F (and phi when ENUF_WANT_PHI is set) back
 * into F_host / phi_host.  Synchronises. */
int enuf_energy_forces_host(enuf_plan* plan, const void* pos_host, const void* q_host, double* E_host,
                            void* F_host, double* virial_host, void* phi_host, int flags);

/* Backward pass of E with respect to the inputs (Eq. 27 and Eq. 5):
 * dpos = gE * (-F), dq = gE * phi, where gE points to one double on the
 * device (NULL means 1).  Recomputes the grids instead of reading stored
 * state.  dpos: N x 3, dq: N (device; either may be NULL).  Asynchronous. */
int enuf_backward(enuf_plan* plan, const void* pos, const void* q, const double* gE, void* dpos, void* dq);

/* enuf_backward with flags: ENUF_AD_FORCES takes -F by analytic
 * differentiation, which is the exact gradient of the energy the forward
 * call returns (the ik forces of enuf_backward are that gradient only within
 * the method's accuracy).  Any other flag bit is ENUF_EINVAL. */
int enuf_backward_flags(enuf_plan* plan, const void* pos, const void* q, const double* gE, void* dpos, void* dq,
                        int flags);

/* Time stepping driven by the plan: nsteps velocity-Verlet steps
 *   v += (dt/2) F/m;  r += dt v (wrapped into the box);  F = F(r);  v += (dt/2) F/m
 * with the forces of enuf_compute under `flags` (ENUF_AD_FORCES,
 * ENUF_REMOVE_NET_FORCE, ENUF_KSPACE_ONLY, ENUF_WANT_VIRIAL; not
 * ENUF_WANT_PHI), a harness for the conservation of energy and momentum
 * along a trajectory.  pos, vel: N x 3, updated in place; q: N; inv_mass: N
 * values 1/m_i (0 fixes a particle); F: N x 3, the forces at pos on return,
 * and on entry when have_forces is nonzero (else computed first); all device
 * buffers of the plan's type.  energies: 4 * nsteps doubles on the device,
 * per step (E_pot, E_kin, E_pot + E_kin, status word).  Units are the
 * caller's (F in coulomb_k q^2 / length^2, dt and m consistent with them).
 * Each step is one CUDA graph launch (captured on the first call with the
 * same buffers, flags, dt and nsteps).  Asynchronous on the plan's stream. */
int enuf_md_run(enuf_plan* plan, void* pos, void* vel, const void* q, const void* inv_mass, void* F,
                int have_forces, double dt, int nsteps, int flags, double* energies);

/* The transposed NFFT of Sec. 3.1 alone (spread, 3D FFT, scaling by the
 * window's Fourier coefficients; Eq. 36-37): the approximated structure
 * factor S~(n) ~ sum_j q_j exp(-2 pi i n.x_j), x_j = r_j / L, on the
 * retained half cube n_x in [0, n_c], n_y, n_z in [-n_c, n_c].  S: device,
 * (2 n_c + 1)^2 (n_c + 1) complex values of the plan's type (re, im pairs),
 * element n at ((n_z + n_c)(2 n_c + 1) + (n_y + n_c))(n_c + 1) + n_x; the
 * other half follows from S~(-n) = conj S~(n).  The structure factor is
 * additive over any partition of the particles (the partial structure
 * factors of Sec. 3.3 sum to the whole).  pos, q as for enuf_compute.
 * Synchronises the plan's stream and checks the inputs (ENUF_ENONFINITE). */
int enuf_structure_factor(enuf_plan* plan, const void* pos, const void* q, void* S);

/* The library's hand-written forward 3D FFT alone, for checking it against
 * another FFT: ghat(k) = sum_l g_l exp(-2 pi i k.l / M) (unnormalised, the
 * sign of Sec. 3.1's forward transform) of the caller's real grid g
 * ([z][y][x], M^3 values of the plan's type, device, not modified), on the
 * same retained half cube and layout as enuf_structure_factor, without the
 * scaling.  Asynchronous on the plan's stream. */
int enuf_fft_forward(enuf_plan* plan, const void* grid, void* ghat);

/* Per-kernel device times (milliseconds) of the last enuf_compute, measured
 * with CUDA events when ENUF_PROFILE=1 was set at plan creation (graphs are
 * then not used).  Fills up to `cap` entries; returns the count. */
int enuf_last_timings(enuf_plan* plan, const char** names, float* times_ms, int cap);

/* Number of kernel launches one enuf_compute call with `flags` performs
 * (memset nodes not counted). */
int enuf_launch_count(enuf_plan* plan, int flags, int with_forces);

/* Real-space erfc pair sum only, for callers that cannot allocate device
 * memory: code running inside a framework whose
 * device memory is reserved by its own pool allocator, plugins handed only
 * their input and output buffers, or code that must not allocate (and so
 * possibly synchronise or fail) after set-up.  The paper has no counterpart
 * of this entry point; it is a variant of the library's all-pairs real-space
 * kernel that allocates nothing: it reads the raw positions (no sorting) and
 * keeps its only scratch, per-block partial sums and a completion counter, in
 * a fixed array in device memory that every GPU loading the library holds
 * until the process exits.
 *   pos, q: N x 3 and N inputs (device; float for ENUF_MIXED, double for
 *   ENUF_FP64).  L: 3 box edges (host).  r_c <= min(L)/2 (minimum image).
 *   F, phi: N x 3 and N outputs (device, may be NULL): the pair force
 *   coulomb_k q_i sum_j ... and the pair potential coulomb_k sum_j q_j
 *   erfc(alpha r)/r, written, not accumulated.  out: 10 doubles (device):
 *   E_real followed by the 9 entries of its virial, row-major.
 *   cuda_stream: cudaStream_t the work is ordered on (NULL = legacy stream).
 * Limits and behaviour: N <= 262,144 (the fixed scratch holds 1024 blocks of
 * 256 particles); larger N returns ENUF_EUNSUPPORTED with a message.  The
 * cost grows as N^2 (every pair is visited).  The first call on each device looks up the scratch
 * array's device address (cudaGetSymbolAddress with that device current);
 * make that first call before any stream capture.  All calls on a device
 * share the scratch, so calls whose kernels overlap on the GPU (different
 * streams, or different host threads) race and give wrong results; order
 * them.  Each call clears the counter it needs before its kernel runs.
 * Asynchronous; errors are reported by the return code and enuf_last_error. */
int enuf_real_space_noalloc(const void* pos, const void* q, int64_t N, const double* L, double alpha, double r_c,
                            double coulomb_k, int precision, void* F, void* phi, double* out, void* cuda_stream);

/* ---------------------------------------------------------------------
 * Learned parameter selector (the paper chooses alpha, r_c, n_c by the
 * procedure of Sec. 2.3.2 / Eq. 31-32; the build adds a small network that
 * predicts the time-optimal choice from a system descriptor).  Network:
 * 6 -> 64 -> 64 -> 4 with SiLU activations; parameters packed row-major as
 * W1[64][6], b1[64], W2[64][64], b2[64], W3[4][64], b3[4].  Weights used by
 * the forward pass are bfloat16; accumulation is float.
 * --------------------------------------------------------------------- */
#define ENUF_MLP_NPARAM 4868

/* Inference: y[n][4] = net(x[n][6]).  w_bf16: ENUF_MLP_NPARAM bfloat16
 * values; x, y: float, device.  Asynchronous on `stream`. */
int enuf_mlp_forward(const void* w_bf16, const float* x, int64_t n, float* y, void* stream);

/* One fused training step on a mini-batch (x: batch x 6, y_target: batch x 4,
 * out_weight: 4 loss weights; all device float): forward, backward of
 * L = 1/(4 batch) sum out_weight_c (y - y_target)^2, gradients summed over the
 * batch, then (if apply_update) Adam on the float master weights w_master
 * (moments adam_m, adam_v; 1-based step) and the bfloat16 copy w_bf16 that
 * the forward pass reads.  loss_out (1 float) and grad_out (ENUF_MLP_NPARAM
 * floats) may be NULL.  Runs as one CTA; asynchronous on `stream`. */
int enuf_mlp_train_step(float* w_master, void* w_bf16, float* adam_m, float* adam_v, const float* x,
                        const float* y_target, const float* out_weight, int batch, float lr, float beta1,
                        float beta2, float eps, int step, float* loss_out, float* grad_out, int apply_update,
                        void* stream);

/* ---------------------------------------------------------------------
 * Checked build.  libenuf_check.so is this library compiled with bounds
 * checks (in place of a memory checker): every index that the kernels derive
 * from particle data, bin counts, work lists or their thread decomposition is
 * tested against its extent before the access; a failed test is counted and
 * the access skipped (a kernel never traps).  Same entry points and results
 * as libenuf.so while no check fails; slower.
 * --------------------------------------------------------------------- */

/* 1 in the checked build, 0 in libenuf.so. */
int enuf_bounds_checked(void);

/* Synchronises the device and returns in *fails the number of failed checks
 * since the last clear (always 0 in libenuf.so).  If where (host, where_len
 * bytes) is given it receives the first failure as "file:line index i of n"
 * ("" if none).  clear != 0 resets the count.  Errors: ENUF_EINVAL (fails
 * NULL), ENUF_ECUDA. */
int enuf_bounds_status(unsigned long long* fails, char* where, int where_len, int clear);

/* Checked build: runs a kernel whose last two of n + 2 writes fail their
 * check (the buffer has room for them) and verifies that exactly those were
 * refused and recorded; clears the count.  0 on success, ENUF_EDEVICE if the
 * checks misbehaved, ENUF_EINVAL in libenuf.so. */
int enuf_bounds_selftest(void);

/* Thread-local description of the last failure ("" if none). */
const char* enuf_last_error(void);

/* Library version string. */
const char* enuf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ENUF_H */
