// k_mlp.cu -- the learned k-ladder predictor: a 64 -> 128 -> 128 -> 33 ReLU MLP
// trained on the GPU (FP32 master weights, Adam) and run for inference in
// BF16 (a component of this library, not of the paper).
//
// Loss of a batch: mean over its samples of the cross-entropy between
// softmax(y[0:32]) and the target fractions t[0:32], plus (y[32] - t[32])^2.
//
// A training step is two launches: k_mlp_grad (one block per tile of 16
// samples: forward, loss, backward, the tile's gradient written to its own
// slice of a partial-gradient buffer) and k_mlp_adam (one thread per
// parameter: the tiles' partial gradients summed in tile order, then Adam).
// Every sum runs in a fixed order, so training is deterministic.  The layer
// products are a few MFLOP per step; they run on the FP32 pipes from shared
// memory, where the launch latency, not the arithmetic, sets the time.
#include <cmath>

#include <cuda_bf16.h>

#include "qsg_launch.h"

namespace qsg {

constexpr int kIn = 64, kH = 128, kOut = 33, kTile = 16;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kOut * kH, kParams = oB3 + kOut;
static_assert(kParams == 29089, "parameter layout");

int mlp_param_count() { return kParams; }

// One tile of samples idx[t0 .. t0+nt): forward, loss, backward.
__global__ void __launch_bounds__(128) k_mlp_grad(const float *__restrict__ P, const float *__restrict__ X,
                                                  const float *__restrict__ T, const int *__restrict__ idx,
                                                  int batch, float *__restrict__ partial,
                                                  float *__restrict__ loss_partial) {
    __shared__ float x[kTile][kIn];
    __shared__ float z1[kTile][kH], z2[kTile][kH];
    __shared__ float y[kTile][kOut], dy[kTile][kOut];
    __shared__ float d2[kTile][kH], d1[kTile][kH];
    __shared__ float lsum[kTile];
    const int tid = threadIdx.x, t0 = blockIdx.x * kTile;
    const int nt = min(kTile, batch - t0);
    const float inv_b = 1.0f / (float)batch;
    for (int i = tid; i < kTile * kIn; i += 128) {
        const int s = i / kIn, f = i % kIn;
        x[s][f] = s < nt ? X[(size_t)idx[t0 + s] * kIn + f] : 0.0f;
    }
    __syncthreads();
    // layer 1 and 2: thread = hidden unit
    {
        const int j = tid;
        for (int s = 0; s < nt; ++s) {
            float a = P[oB1 + j];
            for (int i = 0; i < kIn; ++i) a = fmaf(P[oW1 + j * kIn + i], x[s][i], a);
            z1[s][j] = a;
        }
    }
    __syncthreads();
    {
        const int j = tid;
        for (int s = 0; s < nt; ++s) {
            float a = P[oB2 + j];
            for (int i = 0; i < kH; ++i) a = fmaf(P[oW2 + j * kH + i], fmaxf(z1[s][i], 0.0f), a);
            z2[s][j] = a;
        }
    }
    __syncthreads();
    for (int e = tid; e < nt * kOut; e += 128) {
        const int s = e / kOut, o = e % kOut;
        float a = P[oB3 + o];
        for (int i = 0; i < kH; ++i) a = fmaf(P[oW3 + o * kH + i], fmaxf(z2[s][i], 0.0f), a);
        y[s][o] = a;
    }
    __syncthreads();
    // loss and dL/dy per sample (thread = sample)
    if (tid < nt) {
        const int s = tid;
        const float *t = T + (size_t)idx[t0 + s] * kOut;
        float mx = y[s][0];
        for (int o = 1; o < 32; ++o) mx = fmaxf(mx, y[s][o]);
        float se = 0.0f, tsum = 0.0f;
        for (int o = 0; o < 32; ++o) {
            se += expf(y[s][o] - mx);
            tsum += t[o];
        }
        const float lse = logf(se);
        float ce = 0.0f;
        for (int o = 0; o < 32; ++o) {
            const float logp = y[s][o] - mx - lse;
            ce -= t[o] * logp;
            dy[s][o] = (expf(logp) * tsum - t[o]) * inv_b;
        }
        const float r = y[s][32] - t[32];
        dy[s][32] = 2.0f * r * inv_b;
        lsum[s] = ce + r * r;
    }
    __syncthreads();
    if (tid == 0) {
        float l = 0.0f;
        for (int s = 0; s < nt; ++s) l += lsum[s];
        loss_partial[blockIdx.x] = l * inv_b;
    }
    float *G = partial + (size_t)blockIdx.x * kParams;
    // layer 3 gradients; dL/dz2
    for (int e = tid; e < kOut * kH; e += 128) {
        const int o = e / kH, i = e % kH;
        float a = 0.0f;
        for (int s = 0; s < nt; ++s) a = fmaf(dy[s][o], fmaxf(z2[s][i], 0.0f), a);
        G[oW3 + e] = a;
    }
    if (tid < kOut) {
        float a = 0.0f;
        for (int s = 0; s < nt; ++s) a += dy[s][tid];
        G[oB3 + tid] = a;
    }
    {
        const int j = tid;
        for (int s = 0; s < nt; ++s) {
            float a = 0.0f;
            for (int o = 0; o < kOut; ++o) a = fmaf(dy[s][o], P[oW3 + o * kH + j], a);
            d2[s][j] = z2[s][j] > 0.0f ? a : 0.0f;
        }
    }
    __syncthreads();
    // layer 2 gradients; dL/dz1
    for (int e = tid; e < kH * kH; e += 128) {
        const int j = e / kH, i = e % kH;
        float a = 0.0f;
        for (int s = 0; s < nt; ++s) a = fmaf(d2[s][j], fmaxf(z1[s][i], 0.0f), a);
        G[oW2 + e] = a;
    }
    {
        const int j = tid;
        float a = 0.0f;
        for (int s = 0; s < nt; ++s) a += d2[s][j];
        G[oB2 + j] = a;
        for (int s = 0; s < nt; ++s) {
            float c = 0.0f;
            for (int k = 0; k < kH; ++k) c = fmaf(d2[s][k], P[oW2 + k * kH + j], c);
            d1[s][j] = z1[s][j] > 0.0f ? c : 0.0f;
        }
    }
    __syncthreads();
    // layer 1 gradients
    for (int e = tid; e < kH * kIn; e += 128) {
        const int j = e / kIn, i = e % kIn;
        float a = 0.0f;
        for (int s = 0; s < nt; ++s) a = fmaf(d1[s][j], x[s][i], a);
        G[oW1 + e] = a;
    }
    {
        const int j = tid;
        float a = 0.0f;
        for (int s = 0; s < nt; ++s) a += d1[s][j];
        G[oB1 + j] = a;
    }
}

// Sum the tiles' partial gradients (tile order) and apply one Adam step
// (Kingma & Ba 2015) at step number t, or only write the gradient (adam = 0).
__global__ void k_mlp_adam(float *__restrict__ P, float *__restrict__ M, float *__restrict__ V,
                           const float *__restrict__ partial, int ntiles, float *__restrict__ grad_out,
                           int adam, float lr, float c1, float c2, const float *__restrict__ loss_partial,
                           float *__restrict__ loss_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && loss_out) {
        float l = 0.0f;
        for (int b = 0; b < ntiles; ++b) l += loss_partial[b];
        *loss_out = l;
    }
    if (p >= kParams) return;
    float g = 0.0f;
    for (int b = 0; b < ntiles; ++b) g += partial[(size_t)b * kParams + p];
    if (grad_out) grad_out[p] = g;
    if (!adam) return;
    const float m = 0.9f * M[p] + 0.1f * g;
    const float v = 0.999f * V[p] + 0.001f * g * g;
    M[p] = m;
    V[p] = v;
    // c1 = 1 - 0.9^t, c2 = 1 - 0.999^t (host FP64, rounded once)
    P[p] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
}

cudaError_t launch_mlp_step(float *P, float *M, float *V, const float *X, const float *T, const int *idx, int batch,
                            float *partial, float *loss_partial, float *grad_out, int adam, float lr, int t,
                            float *loss_out, cudaStream_t st) {
    const int ntiles = (batch + kTile - 1) / kTile;
    count_launches(2);
    k_mlp_grad<<<ntiles, 128, 0, st>>>(P, X, T, idx, batch, partial, loss_partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const float c1 = (float)(1.0 - std::pow(0.9, (double)t)), c2 = (float)(1.0 - std::pow(0.999, (double)t));
    k_mlp_adam<<<(kParams + 255) / 256, 256, 0, st>>>(P, M, V, partial, ntiles, grad_out, adam, lr, c1, c2,
                                                       loss_partial, loss_out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Inference.  FP32: plain forward.  BF16: weights, inputs and hidden
// activations rounded to bfloat16 (nearest even), products and sums in FP32.
// One block per sample.
// ---------------------------------------------------------------------------
__global__ void k_mlp_to_bf16(const float *__restrict__ P, __nv_bfloat16 *__restrict__ Pb) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < kParams) Pb[p] = __float2bfloat16_rn(P[p]);
}

template <bool BF16>
__global__ void __launch_bounds__(128) k_mlp_infer(const float *__restrict__ P, const __nv_bfloat16 *__restrict__ Pb,
                                                   const float *__restrict__ X, float *__restrict__ Y) {
    __shared__ float h0[kIn], h1[kH], h2[kH];
    const int s = blockIdx.x, tid = threadIdx.x;
    auto w = [&](int i) { return BF16 ? __bfloat162float(Pb[i]) : P[i]; };
    auto act = [&](float v) { return BF16 ? __bfloat162float(__float2bfloat16_rn(v)) : v; };
    if (tid < kIn) h0[tid] = act(X[(size_t)s * kIn + tid]);
    __syncthreads();
    {
        float a = w(oB1 + tid);
        for (int i = 0; i < kIn; ++i) a = fmaf(w(oW1 + tid * kIn + i), h0[i], a);
        h1[tid] = act(fmaxf(a, 0.0f));
    }
    __syncthreads();
    {
        float a = w(oB2 + tid);
        for (int i = 0; i < kH; ++i) a = fmaf(w(oW2 + tid * kH + i), h1[i], a);
        h2[tid] = act(fmaxf(a, 0.0f));
    }
    __syncthreads();
    if (tid < kOut) {
        float a = w(oB3 + tid);
        for (int i = 0; i < kH; ++i) a = fmaf(w(oW3 + tid * kH + i), h2[i], a);
        Y[(size_t)s * kOut + tid] = a;
    }
}

cudaError_t launch_mlp_infer(const float *P, __nv_bfloat16 *Pb, const float *X, float *Y, long long n, int bf16,
                             cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (bf16) {
        count_launches(2);
        k_mlp_to_bf16<<<(kParams + 255) / 256, 256, 0, st>>>(P, Pb);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_mlp_infer<true><<<(unsigned)n, 128, 0, st>>>(P, Pb, X, Y);
    } else {
        count_launches(1);
        k_mlp_infer<false><<<(unsigned)n, 128, 0, st>>>(P, Pb, X, Y);
    }
    return cudaGetLastError();
}

}  // namespace qsg
