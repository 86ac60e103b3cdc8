// mlp.cu -- the learned parameter selector's network: 6 -> 64 -> 64 -> 4
// with SiLU activations, bfloat16 weights and float accumulation, as two
// hand-written kernels: batched inference, and one fused training step
// (forward, mean-squared-error backward, gradient accumulation over the
// mini-batch, Adam update of the float master weights and their bfloat16
// copies).
//
// Parameter layout (ENUF_MLP_NPARAM = 4868 values, row-major):
//   W1[64][6], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <string>

#include "../../include/enuf.h"

namespace enuf {
void set_last_error(const std::string& msg);
}

namespace {

constexpr int NI = 6, NH = 64, NO = 4;
constexpr int OW1 = 0, OB1 = OW1 + NH * NI, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH, OB3 = OW3 + NO * NH;
constexpr int NP = OB3 + NO;
static_assert(NP == ENUF_MLP_NPARAM, "parameter count");

__device__ __forceinline__ float silu(float x) { return x / (1.f + expf(-x)); }
__device__ __forceinline__ float silu_grad(float x)
{
    const float s = 1.f / (1.f + expf(-x));
    return s * (1.f + x * (1.f - s));
}

// ------------------------------------------------------------------ inference
// One thread per sample; the weights (converted to float) live in shared
// memory and every thread reads the same weight at the same time.
__global__ void __launch_bounds__(256) k_mlp_forward(const __nv_bfloat16* __restrict__ wq, const float* __restrict__ x,
                                                     int n, float* __restrict__ y)
{
    __shared__ float w[NP];
    for (int i = threadIdx.x; i < NP; i += blockDim.x) w[i] = __bfloat162float(wq[i]);
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float in[NI];
#pragma unroll
    for (int i = 0; i < NI; i++) in[i] = x[(size_t)s * NI + i];
    float h1[NH];
#pragma unroll
    for (int j = 0; j < NH; j++) {
        float a = w[OB1 + j];
#pragma unroll
        for (int i = 0; i < NI; i++) a = fmaf(w[OW1 + j * NI + i], in[i], a);
        h1[j] = silu(a);
    }
    float out[NO];
#pragma unroll
    for (int c = 0; c < NO; c++) out[c] = w[OB3 + c];
    for (int o = 0; o < NH; o++) {
        float a = w[OB2 + o];
#pragma unroll
        for (int k = 0; k < NH; k++) a = fmaf(w[OW2 + o * NH + k], h1[k], a);
        const float h2 = silu(a);
#pragma unroll
        for (int c = 0; c < NO; c++) out[c] = fmaf(w[OW3 + c * NH + o], h2, out[c]);
    }
#pragma unroll
    for (int c = 0; c < NO; c++) y[(size_t)s * NO + c] = out[c];
}

// ------------------------------------------------------------------ training
constexpr int CH = 64;         // samples per chunk held in shared memory
constexpr int TT = 512;        // threads of the training CTA

struct TrainArgs {
    float* wm;                 // float master weights (NP)
    __nv_bfloat16* wq;         // bfloat16 copy used by the forward pass (NP)
    float* m;                  // Adam first moment (NP)
    float* v;                  // Adam second moment (NP)
    const float* x;            // batch x NI
    const float* t;            // batch x NO targets
    const float* ow;           // NO output weights of the loss
    int batch;
    float lr, beta1, beta2, eps;
    int step;                  // 1-based Adam step
    float* loss;               // 1 value: mean weighted squared error
    float* grad;               // NP values or nullptr
    int apply;                 // 0: gradients only
};

// One CTA: the mini-batch is processed in chunks of CH samples; each layer is
// a small batched matrix product over (sample, unit) pairs, the backward pass
// mirrors it, and the gradients accumulate in shared memory.  Loss L = 1/(B
// NO) sum_s sum_c ow_c (y_sc - t_sc)^2.
__global__ void __launch_bounds__(TT) k_mlp_train(TrainArgs a)
{
    extern __shared__ __align__(16) float sm[];
    float* w = sm;                 // NP   (bfloat16 weights as float)
    float* g = w + NP;             // NP   gradient accumulator
    float* X = g + NP;             // CH x NI
    float* A1 = X + CH * NI;       // CH x NH  pre-activations
    float* H1 = A1 + CH * NH;      // CH x NH
    float* A2 = H1 + CH * NH;      // CH x NH
    float* H2 = A2 + CH * NH;      // CH x NH
    float* D = H2 + CH * NH;       // CH x NH  (delta of layer 2, then layer 1)
    float* DY = D + CH * NH;       // CH x NO
    __shared__ float red[TT / 32];
    const int tid = threadIdx.x;
    for (int i = tid; i < NP; i += TT) {
        w[i] = __bfloat162float(a.wq[i]);
        g[i] = 0.f;
    }
    float lsum = 0.f;
    __syncthreads();
    const float inv = 1.f / ((float)a.batch * NO);
    for (int c0 = 0; c0 < a.batch; c0 += CH) {
        const int ns = min(CH, a.batch - c0);
        for (int i = tid; i < CH * NI; i += TT) X[i] = (i / NI) < ns ? a.x[(size_t)c0 * NI + i] : 0.f;
        __syncthreads();
        for (int i = tid; i < CH * NH; i += TT) {
            const int s = i / NH, j = i % NH;
            float z = w[OB1 + j];
#pragma unroll
            for (int k = 0; k < NI; k++) z = fmaf(w[OW1 + j * NI + k], X[s * NI + k], z);
            A1[i] = z;
            H1[i] = silu(z);
        }
        __syncthreads();
        for (int i = tid; i < CH * NH; i += TT) {
            const int s = i / NH, o = i % NH;
            float z = w[OB2 + o];
#pragma unroll 16
            for (int k = 0; k < NH; k++) z = fmaf(w[OW2 + o * NH + k], H1[s * NH + k], z);
            A2[i] = z;
            H2[i] = silu(z);
        }
        __syncthreads();
        for (int i = tid; i < CH * NO; i += TT) {
            const int s = i / NO, c = i % NO;
            float z = w[OB3 + c];
#pragma unroll 16
            for (int k = 0; k < NH; k++) z = fmaf(w[OW3 + c * NH + k], H2[s * NH + k], z);
            float d = 0.f;
            if (s < ns) {
                const float e = z - a.t[(size_t)(c0 + s) * NO + c];
                lsum += a.ow[c] * e * e;
                d = 2.f * a.ow[c] * e * inv;
            }
            DY[i] = d;
        }
        __syncthreads();
        // layer 3 gradients and the layer-2 delta
        for (int i = tid; i < NO * NH + NO; i += TT) {
            if (i < NO * NH) {
                const int c = i / NH, k = i % NH;
                float s2 = 0.f;
                for (int s = 0; s < CH; s++) s2 = fmaf(DY[s * NO + c], H2[s * NH + k], s2);
                g[OW3 + i] += s2;
            } else {
                const int c = i - NO * NH;
                float s2 = 0.f;
                for (int s = 0; s < CH; s++) s2 += DY[s * NO + c];
                g[OB3 + c] += s2;
            }
        }
        for (int i = tid; i < CH * NH; i += TT) {
            const int s = i / NH, k = i % NH;
            float z = 0.f;
#pragma unroll
            for (int c = 0; c < NO; c++) z = fmaf(w[OW3 + c * NH + k], DY[s * NO + c], z);
            D[i] = z * silu_grad(A2[i]);
        }
        __syncthreads();
        // layer 2 gradients
        for (int i = tid; i < NH * NH + NH; i += TT) {
            if (i < NH * NH) {
                const int o = i / NH, k = i % NH;
                float s2 = 0.f;
                for (int s = 0; s < CH; s++) s2 = fmaf(D[s * NH + o], H1[s * NH + k], s2);
                g[OW2 + i] += s2;
            } else {
                const int o = i - NH * NH;
                float s2 = 0.f;
                for (int s = 0; s < CH; s++) s2 += D[s * NH + o];
                g[OB2 + o] += s2;
            }
        }
        __syncthreads();
        // layer-1 delta (reuses A2 as scratch), then layer 1 gradients
        for (int i = tid; i < CH * NH; i += TT) {
            const int s = i / NH, j = i % NH;
            float z = 0.f;
#pragma unroll 16
            for (int o = 0; o < NH; o++) z = fmaf(w[OW2 + o * NH + j], D[s * NH + o], z);
            A2[i] = z * silu_grad(A1[i]);
        }
        __syncthreads();
        for (int i = tid; i < NH * NI + NH; i += TT) {
            if (i < NH * NI) {
                const int j = i / NI, k = i % NI;
                float s2 = 0.f;
                for (int s = 0; s < CH; s++) s2 = fmaf(A2[s * NH + j], X[s * NI + k], s2);
                g[OW1 + i] += s2;
            } else {
                const int j = i - NH * NI;
                float s2 = 0.f;
                for (int s = 0; s < CH; s++) s2 += A2[s * NH + j];
                g[OB1 + j] += s2;
            }
        }
        __syncthreads();
    }
    // loss
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((tid & 31) == 0) red[tid >> 5] = lsum;
    __syncthreads();
    if (tid == 0) {
        float l = 0.f;
        for (int k = 0; k < TT / 32; k++) l += red[k];
        if (a.loss) *a.loss = l * inv;
    }
    // Adam
    const float bc1 = 1.f - powf(a.beta1, (float)a.step), bc2 = 1.f - powf(a.beta2, (float)a.step);
    for (int i = tid; i < NP; i += TT) {
        const float gi = g[i];
        if (a.grad) a.grad[i] = gi;
        if (a.apply) {
            const float mi = a.beta1 * a.m[i] + (1.f - a.beta1) * gi;
            const float vi = a.beta2 * a.v[i] + (1.f - a.beta2) * gi * gi;
            a.m[i] = mi;
            a.v[i] = vi;
            const float wn = a.wm[i] - a.lr * (mi / bc1) / (sqrtf(vi / bc2) + a.eps);
            a.wm[i] = wn;
            a.wq[i] = __float2bfloat16(wn);
        }
    }
}

int mfail(int code, const std::string& msg)
{
    enuf::set_last_error(msg);
    return code;
}

}  // namespace

extern "C" {

int enuf_mlp_forward(const void* w_bf16, const float* x, int64_t n, float* y, void* stream)
{
    if (!w_bf16 || !x || !y) return mfail(ENUF_EINVAL, "NULL argument");
    if (n < 0 || n > (int64_t(1) << 31) - 1) return mfail(ENUF_EINVAL, "bad sample count");
    if (n == 0) return ENUF_OK;
    k_mlp_forward<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16*)w_bf16, x, (int)n,
                                                                                    y);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mfail(ENUF_ECUDA, std::string("k_mlp_forward: ") + cudaGetErrorString(e));
    return ENUF_OK;
}

int enuf_mlp_train_step(float* w_master, void* w_bf16, float* adam_m, float* adam_v, const float* x,
                        const float* y_target, const float* out_weight, int batch, float lr, float beta1, float beta2,
                        float eps, int step, float* loss_out, float* grad_out, int apply_update, void* stream)
{
    if (!w_master || !w_bf16 || !adam_m || !adam_v || !x || !y_target || !out_weight)
        return mfail(ENUF_EINVAL, "NULL argument");
    if (batch < 1 || step < 1) return mfail(ENUF_EINVAL, "batch and step must be >= 1");
    TrainArgs a{w_master, (__nv_bfloat16*)w_bf16, adam_m, adam_v, x, y_target, out_weight, batch, lr, beta1, beta2,
                eps, step, loss_out, grad_out, apply_update};
    const size_t smem = (size_t)(2 * NP + CH * NI + 5 * CH * NH + CH * NO) * sizeof(float);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return mfail(ENUF_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
        attr = true;
    }
    k_mlp_train<<<1, TT, smem, (cudaStream_t)stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mfail(ENUF_ECUDA, std::string("k_mlp_train: ") + cudaGetErrorString(e));
    return ENUF_OK;
}

}  // extern "C"
