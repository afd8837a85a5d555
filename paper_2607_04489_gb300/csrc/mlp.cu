// The learned variant selector's network: a small FP32 multilayer perceptron
// 12 -> 64 -> 64 -> 15 (ReLU, softmax) over the runtime statistics of a join
// (Sec. 4: statistics drive the choice of algorithm and knobs). Parameters
// are one contiguous float array: W1[64][12], b1[64], W2[64][64], b2[64],
// W3[15][64], b3[15] (row-major, out x in).
//
// Two training losses over the relative slowdowns R_ic = t_ic / min_c t_ic - 1
// (capped) of plan class c on sample i:
//   tau = 0: the expected regret of the softmax choice,
//            L = mean_i sum_c p_ic R_ic, dL/dz_ic = p_ic (R_ic - sum_k p_ik R_ik) / n;
//   tau > 0: the cross-entropy toward the soft target q_i = softmax(-R_i / tau),
//            L = mean_i -sum_c q_ic log p_ic, dL/dz_ic = (p_ic - q_ic) / n.
// Kernels: forward (one CTA of 64 threads per sample), per-sample gradients
// written to a [n][P] buffer and summed in sample order by a second kernel
// (deterministic), and Adam.
#include "eiger.h"
#include "kernels.cuh"

namespace eiger {

namespace {

constexpr int kIn = EIGER_MLP_IN;
constexpr int kHid = EIGER_MLP_HIDDEN;
constexpr int kOut = EIGER_MLP_OUT;
constexpr int kW1 = 0;
constexpr int kB1 = kW1 + kHid * kIn;
constexpr int kW2 = kB1 + kHid;
constexpr int kB2 = kW2 + kHid * kHid;
constexpr int kW3 = kB2 + kHid;
constexpr int kB3 = kW3 + kOut * kHid;
constexpr int kP = kB3 + kOut;
static_assert(kHid == 64, "one thread per hidden unit");

struct Acts {
    float x[kIn];
    float h1[kHid];
    float h2[kHid];
    float z[kOut];
};

// CTA-collective (64 threads): forward pass of sample `x` into `a`.
__device__ void forward_cta(const float* __restrict__ P, const float* __restrict__ x, Acts& a) {
    const int t = threadIdx.x;
    if (t < kIn) a.x[t] = x[t];
    __syncthreads();
    float s = P[kB1 + t];
#pragma unroll
    for (int f = 0; f < kIn; ++f) s += P[kW1 + t * kIn + f] * a.x[f];
    a.h1[t] = s > 0.f ? s : 0.f;
    __syncthreads();
    s = P[kB2 + t];
#pragma unroll 8
    for (int i = 0; i < kHid; ++i) s += P[kW2 + t * kHid + i] * a.h1[i];
    a.h2[t] = s > 0.f ? s : 0.f;
    __syncthreads();
    if (t < kOut) {
        s = P[kB3 + t];
#pragma unroll 8
        for (int i = 0; i < kHid; ++i) s += P[kW3 + t * kHid + i] * a.h2[i];
        a.z[t] = s;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kHid)
    mlp_forward_kernel(const float* __restrict__ P, const float* __restrict__ X, int n, float* __restrict__ Z) {
    __shared__ Acts a;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        forward_cta(P, X + (size_t)i * kIn, a);
        if (threadIdx.x < kOut) Z[(size_t)i * kOut + threadIdx.x] = a.z[threadIdx.x];
        __syncthreads();
    }
}

// Per-sample loss and gradient (already divided by n) into G[i][P], L[i].
__global__ void __launch_bounds__(kHid)
    mlp_grad_kernel(const float* __restrict__ P, const float* __restrict__ X, const float* __restrict__ C, int n,
                    float tau, float* __restrict__ G, float* __restrict__ L) {
    __shared__ Acts a;
    __shared__ float p[kOut], dz[kOut], da2[kHid], da1[kHid];
    const int t = threadIdx.x;
    const float inv_n = 1.0f / (float)n;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        forward_cta(P, X + (size_t)i * kIn, a);
        const float* c = C + (size_t)i * kOut;
        if (t == 0) {
            float m = a.z[0];
            for (int k = 1; k < kOut; ++k) m = fmaxf(m, a.z[k]);
            float den = 0.f;
            for (int k = 0; k < kOut; ++k) {
                p[k] = expf(a.z[k] - m);
                den += p[k];
            }
            for (int k = 0; k < kOut; ++k) p[k] /= den;
            if (tau > 0.f) {
                float cmin = c[0];
                for (int k = 1; k < kOut; ++k) cmin = fminf(cmin, c[k]);
                float qden = 0.f;
                for (int k = 0; k < kOut; ++k) {
                    dz[k] = expf(-(c[k] - cmin) / tau);  // unnormalised target
                    qden += dz[k];
                }
                const float lse = m + logf(den);  // log p_k = z_k - lse
                float ce = 0.f;
                for (int k = 0; k < kOut; ++k) {
                    const float q = dz[k] / qden;
                    ce -= q * (a.z[k] - lse);
                    dz[k] = (p[k] - q) * inv_n;
                }
                L[i] = ce;
            } else {
                float er = 0.f;
                for (int k = 0; k < kOut; ++k) er += p[k] * c[k];
                for (int k = 0; k < kOut; ++k) dz[k] = p[k] * (c[k] - er) * inv_n;
                L[i] = er;
            }
        }
        __syncthreads();
        float* g = G + (size_t)i * kP;
        // layer 3
        if (t < kOut) g[kB3 + t] = dz[t];
        for (int c3 = 0; c3 < kOut; ++c3) g[kW3 + c3 * kHid + t] = dz[c3] * a.h2[t];
        float d = 0.f;
        for (int c3 = 0; c3 < kOut; ++c3) d += P[kW3 + c3 * kHid + t] * dz[c3];
        da2[t] = a.h2[t] > 0.f ? d : 0.f;
        __syncthreads();
        // layer 2
        g[kB2 + t] = da2[t];
        for (int r = 0; r < kHid; ++r) g[kW2 + r * kHid + t] = da2[r] * a.h1[t];
        d = 0.f;
        for (int r = 0; r < kHid; ++r) d += P[kW2 + r * kHid + t] * da2[r];
        da1[t] = a.h1[t] > 0.f ? d : 0.f;
        __syncthreads();
        // layer 1
        g[kB1 + t] = da1[t];
        for (int f = 0; f < kIn; ++f) g[kW1 + t * kIn + f] = da1[t] * a.x[f];
        __syncthreads();
    }
}

// grad[q] = sum_i G[i][q] in sample order; loss = mean_i L[i] (thread 0 of block 0).
__global__ void mlp_reduce_kernel(const float* __restrict__ G, const float* __restrict__ L, int n,
                                  float* __restrict__ grad, float* __restrict__ loss) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < kP) {
        float s = 0.f;
        for (int i = 0; i < n; ++i) s += G[(size_t)i * kP + q];
        grad[q] = s;
    }
    if (loss && blockIdx.x == 0 && threadIdx.x == 0) {
        float s = 0.f;
        for (int i = 0; i < n; ++i) s += L[i];
        *loss = s / (float)n;
    }
}

__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ grad, float* __restrict__ M,
                                float* __restrict__ V, int step, float lr, float b1, float b2, float eps) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kP) return;
    const float g = grad[q];
    const float m = b1 * M[q] + (1.f - b1) * g;
    const float v = b2 * V[q] + (1.f - b2) * g * g;
    M[q] = m;
    V[q] = v;
    const float mh = m / (1.f - powf(b1, (float)step));
    const float vh = v / (1.f - powf(b2, (float)step));
    P[q] -= lr * mh / (sqrtf(vh) + eps);
}

}  // namespace

int mlp_param_count() { return kP; }

size_t mlp_grad_ws_bytes(int n) {
    return align_up((size_t)n * kP * sizeof(float), 256) + align_up((size_t)n * sizeof(float), 256);
}

cudaError_t mlp_forward(const float* P, const float* X, int n, float* Z, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int grid = n < 4096 ? n : 4096;
    mlp_forward_kernel<<<grid, kHid, 0, s>>>(P, X, n, Z);
    return cudaGetLastError();
}

cudaError_t mlp_grad(const float* P, const float* X, const float* C, int n, float tau, float* grad, float* loss,
                     void* ws, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    float* G = static_cast<float*>(ws);
    float* L = reinterpret_cast<float*>(static_cast<char*>(ws) + align_up((size_t)n * kP * sizeof(float), 256));
    const int grid = n < 4096 ? n : 4096;
    mlp_grad_kernel<<<grid, kHid, 0, s>>>(P, X, C, n, tau, G, L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mlp_reduce_kernel<<<(kP + 255) / 256, 256, 0, s>>>(G, L, n, grad, loss);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float* P, const float* grad, float* M, float* V, int step, float lr, cudaStream_t s) {
    mlp_adam_kernel<<<(kP + 255) / 256, 256, 0, s>>>(P, grad, M, V, step, lr, 0.9f, 0.999f, 1e-8f);
    return cudaGetLastError();
}

}  // namespace eiger
