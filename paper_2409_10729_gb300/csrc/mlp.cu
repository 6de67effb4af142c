// mlp.cu -- the troubled-cell network of the gated form: training kernels
// (loss + gradient, Adam), inference on sample batches, and the generation of
// labelled training samples from a solver state.
//
// Network: 5 -> 32 -> 32 -> 1, ReLU hidden layers, logistic output; input is
// a 5-cell stencil of one sensor field (mixture density or pressure)
// normalised as (v_k - v_i)/max_k |v_k - v_i|; a stencil whose variation is
// at most MFC_GATE_FLOOR |v_i| is flat and never shown to the network.
// Parameters (1281 floats): W1[32][5], b1[32], W2[32][32], b2[32], w3[32],
// b3.  Label of a cell and direction: troubled (1) when, for some primitive
// field whose stencil is not flat, a nonlinear WENO5-JS weight at either
// face departs from its linear weight by more than tau relative; smooth (0)
// otherwise (below the floor the two reconstructions differ by round-off).  Loss: weighted binary
// cross-entropy on the logit (positive-class weight wp).  Training is FP32;
// the samples are formed in FP64 from reference-order primitives (this file is
// built with -fmad=false).
#include <cuda_runtime.h>
#include <math.h>

#include "mfc.h"
#include "mfc_internal.cuh"
#include "sweep.cuh"

namespace mfc5 {

constexpr int kMlpH = 32, kMlpIn = 5;
constexpr int kMlpParams = kMlpH * kMlpIn + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;
constexpr int OW1 = 0, OB1 = kMlpH * kMlpIn, OW2 = OB1 + kMlpH, OB2 = OW2 + kMlpH * kMlpH, OW3 = OB2 + kMlpH,
              OB3 = OW3 + kMlpH;
static_assert(kMlpParams == 1281, "parameter layout");

__device__ __forceinline__ float softplusf(float t) { return t > 0.f ? t + log1pf(expf(-t)) : log1pf(expf(t)); }

// Loss and gradient over n samples.  Block = kGradThreads threads; each pass
// of a block takes kGradThreads samples: one thread per sample runs the
// forward and backward pass and stages its activations in shared memory,
// then every thread accumulates ~10 parameters over the staged samples.
// Block partial sums go to global memory with one atomic add per parameter.
constexpr int kGradThreads = 128;
constexpr int kStage = kMlpIn + 4 * kMlpH + 1;  // x, h1, d1, d2, dz*h2, dz

__global__ void __launch_bounds__(kGradThreads)
mlp_grad_kernel(const float* __restrict__ X, const float* __restrict__ Y, long long n,
                const float* __restrict__ theta, float wp, float inv_n, float* grad, float* loss) {
    extern __shared__ float sm[];
    float* th = sm;                        // kMlpParams
    float* st = sm + kMlpParams;           // kGradThreads * kStage
    for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) th[k] = theta[k];
    __syncthreads();
    constexpr int PER = (kMlpParams + kGradThreads - 1) / kGradThreads;
    float acc[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) acc[r] = 0.f;
    float lsum = 0.f;
    for (long long base = (long long)blockIdx.x * kGradThreads; base < n;
         base += (long long)gridDim.x * kGradThreads) {
        long long s = base + threadIdx.x;
        float* me = st + threadIdx.x * kStage;
        if (s < n) {
            float x[kMlpIn], h1[kMlpH], h2[kMlpH], d2[kMlpH];
#pragma unroll
            for (int i = 0; i < kMlpIn; ++i) x[i] = X[s * kMlpIn + i];
#pragma unroll 4
            for (int j = 0; j < kMlpH; ++j) {
                float a = th[OB1 + j];
#pragma unroll
                for (int i = 0; i < kMlpIn; ++i) a = fmaf(th[OW1 + j * kMlpIn + i], x[i], a);
                h1[j] = fmaxf(a, 0.f);
            }
#pragma unroll 4
            for (int j = 0; j < kMlpH; ++j) {
                float a = th[OB2 + j];
#pragma unroll
                for (int i = 0; i < kMlpH; ++i) a = fmaf(th[OW2 + j * kMlpH + i], h1[i], a);
                h2[j] = fmaxf(a, 0.f);
            }
            float z = th[OB3];
#pragma unroll
            for (int i = 0; i < kMlpH; ++i) z = fmaf(th[OW3 + i], h2[i], z);
            float y = Y[s];
            lsum += wp * y * softplusf(-z) + (1.f - y) * softplusf(z);
            float sg = 1.f / (1.f + expf(-z));
            float dz = (wp * y * (sg - 1.f) + (1.f - y) * sg) * inv_n;
#pragma unroll
            for (int i = 0; i < kMlpH; ++i) d2[i] = h2[i] > 0.f ? dz * th[OW3 + i] : 0.f;
#pragma unroll
            for (int i = 0; i < kMlpIn; ++i) me[i] = x[i];
#pragma unroll 4
            for (int i = 0; i < kMlpH; ++i) {
                float a = 0.f;
#pragma unroll
                for (int j = 0; j < kMlpH; ++j) a = fmaf(th[OW2 + j * kMlpH + i], d2[j], a);
                me[kMlpIn + i] = h1[i];
                me[kMlpIn + kMlpH + i] = h1[i] > 0.f ? a : 0.f;
                me[kMlpIn + 2 * kMlpH + i] = d2[i];
                me[kMlpIn + 3 * kMlpH + i] = dz * h2[i];
            }
            me[kStage - 1] = dz;
        } else {
            for (int i = 0; i < kStage; ++i) me[i] = 0.f;
        }
        __syncthreads();
        // parameter k: sum over the staged samples of its per-sample gradient
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            int k = threadIdx.x + r * kGradThreads;
            if (k >= kMlpParams) break;
            float a = acc[r];
            if (k < OB1) {                 // W1[j][i] += d1_j x_i
                int j = k / kMlpIn, i = k % kMlpIn;
                for (int t = 0; t < kGradThreads; ++t) a = fmaf(st[t * kStage + kMlpIn + kMlpH + j], st[t * kStage + i], a);
            } else if (k < OW2) {          // b1[j] += d1_j
                int j = k - OB1;
                for (int t = 0; t < kGradThreads; ++t) a += st[t * kStage + kMlpIn + kMlpH + j];
            } else if (k < OB2) {          // W2[j][i] += d2_j h1_i
                int j = (k - OW2) / kMlpH, i = (k - OW2) % kMlpH;
                for (int t = 0; t < kGradThreads; ++t)
                    a = fmaf(st[t * kStage + kMlpIn + 2 * kMlpH + j], st[t * kStage + kMlpIn + i], a);
            } else if (k < OW3) {          // b2[j] += d2_j
                int j = k - OB2;
                for (int t = 0; t < kGradThreads; ++t) a += st[t * kStage + kMlpIn + 2 * kMlpH + j];
            } else if (k < OB3) {          // w3[i] += dz h2_i
                int i = k - OW3;
                for (int t = 0; t < kGradThreads; ++t) a += st[t * kStage + kMlpIn + 3 * kMlpH + i];
            } else {                       // b3 += dz
                for (int t = 0; t < kGradThreads; ++t) a += st[t * kStage + kStage - 1];
            }
            acc[r] = a;
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        int k = threadIdx.x + r * kGradThreads;
        if (k < kMlpParams) atomicAdd(&grad[k], acc[r]);
    }
    // loss: warp reduction, then one atomic per warp
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum * inv_n);
}

__global__ void mlp_adam_kernel(float* theta, const float* __restrict__ g, float* m, float* v, float lr, float b1,
                                float b2, float eps, float c1, float c2) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= kMlpParams) return;
    float gk = g[k];
    float mk = b1 * m[k] + (1.f - b1) * gk;
    float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    theta[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

// Logit of one normalised stencil x[5] with parameters th (any memory space).
__device__ __forceinline__ float mlp_logit(const float* th, const float* x) {
    float h1[kMlpH];
#pragma unroll 4
    for (int j = 0; j < kMlpH; ++j) {
        float a = th[OB1 + j];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) a = fmaf(th[OW1 + j * kMlpIn + i], x[i], a);
        h1[j] = fmaxf(a, 0.f);
    }
    float z = th[OB3];
#pragma unroll 2
    for (int j = 0; j < kMlpH; ++j) {
        float a = th[OB2 + j];
#pragma unroll
        for (int i = 0; i < kMlpH; ++i) a = fmaf(th[OW2 + j * kMlpH + i], h1[i], a);
        z = fmaf(th[OW3 + j], fmaxf(a, 0.f), z);
    }
    return z;
}

__global__ void mlp_forward_kernel(const float* __restrict__ X, long long n, const float* __restrict__ theta,
                                   float* z) {
    __shared__ float th[kMlpParams];
    for (int k = threadIdx.x; k < kMlpParams; k += blockDim.x) th[k] = theta[k];
    __syncthreads();
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        float x[kMlpIn];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) x[i] = X[s * kMlpIn + i];
        z[s] = mlp_logit(th, x);
    }
}

// Training samples from an FP64 state: for every cell c and direction d,
// two samples (density sensor, pressure sensor) sharing the cell's label.
// Layout: sample index ((d * ncell + c) * 2 + sensor).
template <int NDIM>
__global__ void gate_samples_kernel(const double* __restrict__ q, int n0, int n1, int n2, int per0, int per1,
                                    int per2, Eos eos, double eps, float tau, float* X, float* Y) {
    using FL = Fields<NDIM>;
    const long long nc = (long long)n0 * n1 * n2;
    const int n[3] = {n0, n1, n2}, per[3] = {per0, per1, per2};
    const long long stride[3] = {1, n0, (long long)n0 * n1};
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nc * NDIM;
         t += (long long)gridDim.x * blockDim.x) {
        const int d = (int)(t / nc);
        const long long c = t % nc;
        const int idx = (int)((c / stride[d]) % n[d]);
        const long long base = c - (long long)idx * stride[d];
        double w[5][FL::NEQ];
        for (int k = 0; k < 5; ++k) {
            long long cc = base + (long long)bc_index(idx - 2 + k, n[d], per[d]) * stride[d];
            double v[FL::NEQ];
            for (int f = 0; f < FL::NEQ; ++f) v[f] = q[f * nc + cc];
            exact::cons_to_prim<NDIM>(eos, v, w[k]);   // reference-order primitives
        }
        bool troubled = false;
        const double dm[3] = {0.1, 0.6, 0.3}, dp[3] = {0.3, 0.6, 0.1};
        for (int f = 0; f < FL::NEQ; ++f) {
            const double c13 = 13.0 / 12.0;
            double v0 = w[0][f], v1 = w[1][f], v2 = w[2][f], v3 = w[3][f], v4 = w[4][f];
            double mf = 0.0;
            for (int k = 0; k < 5; ++k) mf = fmax(mf, fabs(w[k][f] - v2));
            if (!(mf > MFC_GATE_FLOOR * fabs(v2))) continue;   // flat: round-off only
            double b[3];
            b[0] = c13 * (v0 - 2.0 * v1 + v2) * (v0 - 2.0 * v1 + v2) + 0.25 * (v0 - 4.0 * v1 + 3.0 * v2) * (v0 - 4.0 * v1 + 3.0 * v2);
            b[1] = c13 * (v1 - 2.0 * v2 + v3) * (v1 - 2.0 * v2 + v3) + 0.25 * (v1 - v3) * (v1 - v3);
            b[2] = c13 * (v2 - 2.0 * v3 + v4) * (v2 - 2.0 * v3 + v4) + 0.25 * (3.0 * v2 - 4.0 * v3 + v4) * (3.0 * v2 - 4.0 * v3 + v4);
            double am[3], ap[3], sm = 0.0, sp = 0.0;
            for (int k = 0; k < 3; ++k) {
                double s2 = (eps + b[k]) * (eps + b[k]);
                am[k] = dm[k] / s2;
                ap[k] = dp[k] / s2;
                sm += am[k];
                sp += ap[k];
            }
            for (int k = 0; k < 3; ++k) {
                troubled |= fabs(am[k] / sm - dm[k]) > tau * dm[k];
                troubled |= fabs(ap[k] / sp - dp[k]) > tau * dp[k];
            }
        }
        for (int sensor = 0; sensor < 2; ++sensor) {
            double v[5], m = 0.0;
            for (int k = 0; k < 5; ++k) v[k] = sensor == 0 ? w[k][0] + w[k][1] : w[k][FL::IE];
            for (int k = 0; k < 5; ++k) m = fmax(m, fabs(v[k] - v[2]));
            long long sidx = t * 2 + sensor;
            const bool live = m > MFC_GATE_FLOOR * fabs(v[2]);
            for (int k = 0; k < 5; ++k) X[sidx * 5 + k] = live ? float((v[k] - v[2]) / m) : 0.f;
            Y[sidx] = !live ? -1.f : (troubled ? 1.f : 0.f);
        }
    }
}

cudaError_t launch_gate_samples(int ndim, const double* q, const int* n, const int* periodic, const Eos& e,
                                double eps, float tau, float* X, float* Y, cudaStream_t s) {
    long long total = (long long)n[0] * n[1] * n[2] * ndim;
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    if (blocks < 1) blocks = 1;
    if (ndim == 1)
        gate_samples_kernel<1><<<(unsigned)blocks, 256, 0, s>>>(q, n[0], n[1], n[2], periodic[0], periodic[1],
                                                                periodic[2], e, eps, tau, X, Y);
    else if (ndim == 2)
        gate_samples_kernel<2><<<(unsigned)blocks, 256, 0, s>>>(q, n[0], n[1], n[2], periodic[0], periodic[1],
                                                                periodic[2], e, eps, tau, X, Y);
    else
        gate_samples_kernel<3><<<(unsigned)blocks, 256, 0, s>>>(q, n[0], n[1], n[2], periodic[0], periodic[1],
                                                                periodic[2], e, eps, tau, X, Y);
    return cudaGetLastError();
}

}  // namespace mfc5

using namespace mfc5;

extern "C" int mfc_mlp_nparams(void) { return kMlpParams; }

extern "C" int mfc_mlp_loss_grad(const float* X, const float* Y, long long n, const float* theta, float pos_weight,
                                 float* grad, float* loss, void* cuda_stream) {
    if (!X || !Y || !theta || !grad || !loss || n <= 0 || !(pos_weight > 0.f)) return MFC_EINVAL;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const size_t smem = sizeof(float) * (kMlpParams + kGradThreads * kStage);
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return MFC_ECUDA;
        attr = true;
    }
    if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, s) != cudaSuccess ||
        cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess)
        return MFC_ECUDA;
    long long blocks = (n + kGradThreads - 1) / kGradThreads;
    if (blocks > 152LL * 2) blocks = 152LL * 2;
    mlp_grad_kernel<<<(unsigned)blocks, kGradThreads, smem, s>>>(X, Y, n, theta, pos_weight, 1.0f / (float)n, grad,
                                                                 loss);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ECUDA;
}

extern "C" int mfc_mlp_adam(float* theta, const float* grad, float* m, float* v, int t, float lr, float beta1,
                            float beta2, float eps, void* cuda_stream) {
    if (!theta || !grad || !m || !v || t < 1) return MFC_EINVAL;
    // bias corrections 1 - beta^t formed in FP64: in FP32, 1 - 0.999^t loses
    // about 1e-5 relative to cancellation
    float c1 = (float)(1.0 - pow((double)beta1, (double)t));
    float c2 = (float)(1.0 - pow((double)beta2, (double)t));
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(theta, grad, m, v, lr, beta1,
                                                                                      beta2, eps, c1, c2);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ECUDA;
}

extern "C" int mfc_mlp_forward(const float* X, long long n, const float* theta, float* z, void* cuda_stream) {
    if (!X || !theta || !z || n <= 0) return MFC_EINVAL;
    long long blocks = (n + 255) / 256;
    if (blocks > 152LL * 16) blocks = 152LL * 16;
    mlp_forward_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)cuda_stream>>>(X, n, theta, z);
    return cudaGetLastError() == cudaSuccess ? MFC_OK : MFC_ECUDA;
}
