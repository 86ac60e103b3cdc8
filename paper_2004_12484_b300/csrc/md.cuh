// md.cuh -- velocity-Verlet time stepping driven by the evaluation (a
// harness for the conservation the method is used for: energy and momentum
// over a trajectory).  One step:
//   v += (dt/2) F / m;  r += dt v (wrapped into the box);  F = F(r);
//   v += (dt/2) F / m;  record E_pot, E_kin = 1/2 sum m v^2, their sum.
#pragma once
#include "common.cuh"

namespace enuf {

// First half kick and drift; positions are wrapped into [0, L).
template <typename R>
__global__ void __launch_bounds__(256) k_md_kick_drift(int N, R* __restrict__ pos, R* __restrict__ vel,
                                                       const R* __restrict__ F, const R* __restrict__ inv_mass,
                                                       R hdt, R dt, R L0, R L1, R L2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const R w = hdt * inv_mass[i];
    const R Lb[3] = {L0, L1, L2};
#pragma unroll
    for (int t = 0; t < 3; t++) {
        const size_t k = 3 * (size_t)i + t;
        const R v = vel[k] + w * F[k];
        vel[k] = v;
        R x = pos[k] + dt * v;
        x -= Lb[t] * floor(x / Lb[t]);
        if (x >= Lb[t]) x -= Lb[t];  // rounding of a value just below 0
        pos[k] = x;
    }
}

// Second half kick; per-block partial sums of the kinetic energy (a
// particle with 1/m = 0 is fixed and carries none).
template <typename R>
__global__ void __launch_bounds__(256) k_md_kick(int N, R* __restrict__ vel, const R* __restrict__ F,
                                                 const R* __restrict__ inv_mass, R hdt, double* __restrict__ part)
{
    __shared__ double red[32];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    R ke[1] = {R(0)};
    if (i < N) {
        const R im = inv_mass[i];
        const R w = hdt * im;
        R v2 = R(0);
#pragma unroll
        for (int t = 0; t < 3; t++) {
            const size_t k = 3 * (size_t)i + t;
            const R v = vel[k] + w * F[k];
            vel[k] = v;
            v2 += v * v;
        }
        ke[0] = im > R(0) ? R(0.5) * v2 / im : R(0);
    }
    block_reduce_to_double<R, 1>(ke, part + 4 * (size_t)blockIdx.x, red);
}

// One block: the step's kinetic energy from the partials (fixed order),
// the potential energy and status from the evaluation's results, written to
// energies[4 s ..] for the step s counted on the device.
__global__ void __launch_bounds__(256) k_md_record(int nb, const double* __restrict__ part,
                                                   const double* __restrict__ out, double* __restrict__ energies,
                                                   unsigned* __restrict__ step, int cap)
{
    __shared__ double red[32];
    __shared__ double tot[1];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[4 * (size_t)b];
    double v[1] = {s};
    block_reduce_to_double<double, 1>(v, tot, red);
    if (threadIdx.x == 0) {
        const double ke = tot[0];
        const unsigned k = *step;
        if ((int)k < cap) {
            energies[4 * (size_t)k] = out[ENUF_OUT_E];
            energies[4 * (size_t)k + 1] = ke;
            energies[4 * (size_t)k + 2] = out[ENUF_OUT_E] + ke;
            energies[4 * (size_t)k + 3] = out[ENUF_OUT_STATUS];
        }
        *step = k + 1;
    }
}

}  // namespace enuf
