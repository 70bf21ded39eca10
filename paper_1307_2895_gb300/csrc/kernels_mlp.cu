// Rank-prediction MLP: three layers of width 64 with ReLU, target
// log(1 + k), Huber loss (delta 1) averaged over samples.  FP32 training
// (forward + backward written out, per-block gradient partials summed in
// block order, Adam), BF16-weight inference with FP32 accumulation.
//
// Parameter layout (flat float): W1 (H x F) row-major | b1 (H) | W2 (H x H) |
// b2 (H) | W3 (1 x H) | b3 (1).  F = kFeat, H = kHid.
#include <cuda_bf16.h>

#include <atomic>

#include "hif_internal.h"
#include "kernels.h"

namespace hif {

constexpr int kChunk = 64;      // samples per block
constexpr int kMlpThreads = 256;

struct MlpOffsets {
  static constexpr int W1 = 0;
  static constexpr int b1 = W1 + kHid * kFeat;
  static constexpr int W2 = b1 + kHid;
  static constexpr int b2 = W2 + kHid * kHid;
  static constexpr int W3 = b2 + kHid;
  static constexpr int b3 = W3 + kHid;
  static constexpr int P = b3 + 1;
};
static_assert(MlpOffsets::P == kMlpParams, "parameter count");

// One block: samples [s0, s0 + kChunk) of the (optionally indexed) batch.
// Writes its partial gradient (sum over its samples of dL_i/dtheta / n) to
// partial[blockIdx.x * P ..] and its partial loss sum to ploss[blockIdx.x].
__global__ void k_mlp_fwd_bwd(const float* __restrict__ X, const float* __restrict__ t,
                              const int* __restrict__ idx, int nb, float inv_n,
                              const float* __restrict__ prm, float* __restrict__ partial,
                              float* __restrict__ ploss) {
  extern __shared__ __align__(16) float sm[];
  float* W1 = sm;                                // H x F
  float* b1 = W1 + kHid * kFeat;
  float* W2 = b1 + kHid;                         // H x H
  float* b2 = W2 + kHid * kHid;
  float* W3 = b2 + kHid;
  float* xs = W3 + kHid;                         // chunk x F
  float* Z1 = xs + kChunk * kFeat;               // chunk x H
  float* Z2 = Z1 + kChunk * kHid;                // chunk x H
  float* G2 = Z2 + kChunk * kHid;                // chunk x H  (dL/dZ2)
  float* G1 = G2 + kChunk * kHid;                // chunk x H  (dL/dZ1)
  float* gy = G1 + kChunk * kHid;                // chunk
  __shared__ float s_b3, s_loss;
  const int tid = threadIdx.x;
  const int s0 = blockIdx.x * kChunk;
  const int ns = min(kChunk, nb - s0);
  for (int e = tid; e < MlpOffsets::W3 + kHid; e += blockDim.x) sm[e] = prm[e];
  if (tid == 0) { s_b3 = prm[MlpOffsets::b3]; s_loss = 0.f; }
  for (int e = tid; e < kChunk * kFeat; e += blockDim.x) {
    const int s = e / kFeat, f = e % kFeat;
    float v = 0.f;
    if (s < ns) {
      const int row = idx ? idx[s0 + s] : s0 + s;
      v = X[(int64_t)row * kFeat + f];
    }
    xs[e] = v;
  }
  __syncthreads();
  for (int e = tid; e < kChunk * kHid; e += blockDim.x) {      // Z1 = x W1^T + b1
    const int s = e / kHid, i = e % kHid;
    float a = b1[i];
    for (int f = 0; f < kFeat; ++f) a = fmaf(W1[i * kFeat + f], xs[s * kFeat + f], a);
    Z1[e] = a;
  }
  __syncthreads();
  for (int e = tid; e < kChunk * kHid; e += blockDim.x) {      // Z2 = relu(Z1) W2^T + b2
    const int s = e / kHid, i = e % kHid;
    float a = b2[i];
    for (int j = 0; j < kHid; ++j) a = fmaf(W2[i * kHid + j], fmaxf(Z1[s * kHid + j], 0.f), a);
    Z2[e] = a;
  }
  __syncthreads();
  for (int s = tid; s < kChunk; s += blockDim.x) {              // y, residual, dL/dy
    float g = 0.f;
    if (s < ns) {
      float y = s_b3;
      for (int j = 0; j < kHid; ++j) y = fmaf(W3[j], fmaxf(Z2[s * kHid + j], 0.f), y);
      const int row = idx ? idx[s0 + s] : s0 + s;
      const float d = y - t[row];
      const float ad = fabsf(d);
      atomicAdd(&s_loss, ad <= 1.f ? 0.5f * d * d : ad - 0.5f);
      g = fminf(fmaxf(d, -1.f), 1.f) * inv_n;
    }
    gy[s] = g;
  }
  __syncthreads();
  for (int e = tid; e < kChunk * kHid; e += blockDim.x) {      // dL/dZ2
    const int s = e / kHid, i = e % kHid;
    G2[e] = Z2[e] > 0.f ? gy[s] * W3[i] : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < kChunk * kHid; e += blockDim.x) {      // dL/dZ1 = (G2 W2) * (Z1 > 0)
    const int s = e / kHid, j = e % kHid;
    float a = 0.f;
    for (int i = 0; i < kHid; ++i) a = fmaf(G2[s * kHid + i], W2[i * kHid + j], a);
    G1[e] = Z1[e] > 0.f ? a : 0.f;
  }
  __syncthreads();
  float* out = partial + (int64_t)blockIdx.x * MlpOffsets::P;
  for (int p = tid; p < MlpOffsets::P; p += blockDim.x) {       // weight gradients of this chunk
    float a = 0.f;
    if (p < MlpOffsets::b1) {
      const int i = p / kFeat, f = p % kFeat;
      for (int s = 0; s < kChunk; ++s) a = fmaf(G1[s * kHid + i], xs[s * kFeat + f], a);
    } else if (p < MlpOffsets::W2) {
      const int i = p - MlpOffsets::b1;
      for (int s = 0; s < kChunk; ++s) a += G1[s * kHid + i];
    } else if (p < MlpOffsets::b2) {
      const int q = p - MlpOffsets::W2, i = q / kHid, j = q % kHid;
      for (int s = 0; s < kChunk; ++s) a = fmaf(G2[s * kHid + i], fmaxf(Z1[s * kHid + j], 0.f), a);
    } else if (p < MlpOffsets::W3) {
      const int i = p - MlpOffsets::b2;
      for (int s = 0; s < kChunk; ++s) a += G2[s * kHid + i];
    } else if (p < MlpOffsets::b3) {
      const int j = p - MlpOffsets::W3;
      for (int s = 0; s < kChunk; ++s) a = fmaf(gy[s], fmaxf(Z2[s * kHid + j], 0.f), a);
    } else {
      for (int s = 0; s < kChunk; ++s) a += gy[s];
    }
    out[p] = a;
  }
  if (tid == 0) ploss[blockIdx.x] = s_loss;
}

// grad[p] = sum_b partial[b][p] (block order); loss = sum_b ploss[b] * inv_n
__global__ void k_mlp_reduce(const float* __restrict__ partial, const float* __restrict__ ploss, int nblk,
                             float inv_n, float* __restrict__ grad, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < MlpOffsets::P) {
    float a = 0.f;
    for (int b = 0; b < nblk; ++b) a += partial[(int64_t)b * MlpOffsets::P + p];
    grad[p] = a;
  }
  if (p == 0 && loss) {
    float a = 0.f;
    for (int b = 0; b < nblk; ++b) a += ploss[b];
    *loss = a * inv_n;
  }
}

// Adam (beta1 0.9, beta2 0.999, eps 1e-8), step count t >= 1
__global__ void k_mlp_adam(float* __restrict__ prm, const float* __restrict__ grad, float* __restrict__ m,
                           float* __restrict__ v, float lr, int t) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= MlpOffsets::P) return;
  const float b1 = 0.9f, b2 = 0.999f;
  const float g = grad[p];
  const float mm = b1 * m[p] + (1.f - b1) * g;
  const float vv = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.f - powf(b1, (float)t));
  const float vh = vv / (1.f - powf(b2, (float)t));
  prm[p] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// Inference with BF16 weights and FP32 accumulation: one warp per sample.
__global__ void k_mlp_predict(const float* __restrict__ X, int n, const __nv_bfloat16* __restrict__ w,
                              float* __restrict__ y) {
  __shared__ float h1[kMlpThreads / 32][kHid];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = blockIdx.x * (blockDim.x >> 5) + warp;
  if (s >= n) return;
  const float* x = X + (int64_t)s * kFeat;
  for (int i = lane; i < kHid; i += 32) {
    float a = __bfloat162float(w[MlpOffsets::b1 + i]);
    for (int f = 0; f < kFeat; ++f) a = fmaf(__bfloat162float(w[MlpOffsets::W1 + i * kFeat + f]), x[f], a);
    h1[warp][i] = fmaxf(a, 0.f);
  }
  __syncwarp();
  float acc = 0.f;
  for (int i = lane; i < kHid; i += 32) {
    float a = __bfloat162float(w[MlpOffsets::b2 + i]);
    for (int j = 0; j < kHid; ++j) a = fmaf(__bfloat162float(w[MlpOffsets::W2 + i * kHid + j]), h1[warp][j], a);
    acc = fmaf(__bfloat162float(w[MlpOffsets::W3 + i]), fmaxf(a, 0.f), acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[s] = acc + __bfloat162float(w[MlpOffsets::b3]);
}

__global__ void k_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

// ---------------------------------------------------------------------------
static size_t fwd_bwd_smem() {
  return sizeof(float) * (size_t)(kHid * kFeat + kHid + kHid * kHid + kHid + kHid + kChunk * kFeat +
                                  4 * kChunk * kHid + kChunk);
}

void mlp_grad(const float* X, const float* t, const int* idx, int nb, float inv_n, const float* prm,
              float* partial, float* ploss, float* grad, float* loss, cudaStream_t st) {
  const int nblk = (nb + kChunk - 1) / kChunk;
  const size_t smem = fwd_bwd_smem();
  static std::atomic<bool> attr{false};
  if (!attr) {
    cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  note_launches(2);
  k_mlp_fwd_bwd<<<nblk, kMlpThreads, smem, st>>>(X, t, idx, nb, inv_n, prm, partial, ploss);
  k_mlp_reduce<<<(kMlpParams + 255) / 256, 256, 0, st>>>(partial, ploss, nblk, inv_n, grad, loss);
}

void mlp_adam(float* prm, const float* grad, float* m, float* v, float lr, int t, cudaStream_t st) {
  note_launches(1);
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(prm, grad, m, v, lr, t);
}

void mlp_to_bf16(const float* prm, void* wbf16, cudaStream_t st) {
  note_launches(1);
  k_to_bf16<<<(kMlpParams + 255) / 256, 256, 0, st>>>(prm, reinterpret_cast<__nv_bfloat16*>(wbf16), kMlpParams);
}

void mlp_predict(const float* X, int n, const void* wbf16, float* y, cudaStream_t st) {
  if (n <= 0) return;
  note_launches(1);
  const int per = kMlpThreads / 32;
  k_mlp_predict<<<(n + per - 1) / per, kMlpThreads, 0, st>>>(X, n, reinterpret_cast<const __nv_bfloat16*>(wbf16),
                                                              y);
}

int mlp_chunks(int nb) { return (nb + kChunk - 1) / kChunk; }

}  // namespace hif
