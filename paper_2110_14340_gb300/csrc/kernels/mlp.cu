// mlp.cu - the learned launch-configuration cost model: MLP 4 -> 64 -> 64 -> 64 -> 1.
//
// No counterpart in the paper (auto-tuning is named as future work, §8).
// FP32 FFMA kernels (the network is far too small for tensor cores to pay):
//   jacc_k_mlp_fwd_bwd  one CTA per chunk of 32 samples: parameters and the
//                       chunk's activations in shared memory, forward pass,
//                       squared-error loss and backward pass; writes the
//                       chunk's gradient to its own row of `partial`.
//   jacc_k_mlp_adam     sums the chunk gradients in fixed order (deterministic)
//                       and applies one Adam step with bias correction.
//   jacc_k_mlp_forward  predictions only.
//   jacc_k_mlp_pick     per query, the argmin of the predictions over the valid
//                       tile configurations and the gap to the second best.
// Parameter layout: W1[64][4] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64] b4.
// Shared-memory activation rows are padded to 65 floats so that lanes indexed
// by sample read distinct banks.
#include <cuda_runtime.h>

#include "../host/jacc_internal.h"
#include "mlp.h"

namespace {

constexpr int H = 64;
constexpr int NIN = 4;
constexpr int S = 32;   // samples per CTA (one per lane)
constexpr int NT = 256; // 8 warps
constexpr int LD = H + 1;
constexpr int OFF_W1 = 0, OFF_B1 = 256, OFF_W2 = 320, OFF_B2 = 4416, OFF_W3 = 4480, OFF_B3 = 8576, OFF_W4 = 8640,
              OFF_B4 = 8704;

struct Smem {
  float p[JACC_MLP_NPARAM];
  float x[S][NIN];
  float z1[S][LD], z2[S][LD], z3[S][LD];  // pre-activations
  float d[S][LD], d2[S][LD];              // back-propagated dz buffers
  float y[S], dy[S];
  float red[NT / 32];
};

__device__ __forceinline__ float relu(float z) { return z > 0.f ? z : 0.f; }

// Layer: zo[s][o] = b[o] + sum_i W[o][i] act(zi[s][i]) for o in this warp's 8 outputs.
template <bool RELU_IN>
__device__ __forceinline__ void dense64(const float* W, const float* b, const float (*zi)[LD], float (*zo)[LD]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = b[w * 8 + k];
  for (int i = 0; i < H; ++i) {
    const float h = RELU_IN ? relu(zi[lane][i]) : zi[lane][i];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = fmaf(W[(w * 8 + k) * H + i], h, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) zo[lane][w * 8 + k] = acc[k];
}

__device__ void forward_chunk(Smem& sm, const float* __restrict__ X, long long s0, int nvalid) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < S * NIN; t += NT) {
    const int s = t / NIN, i = t % NIN;
    sm.x[s][i] = s < nvalid ? X[(s0 + s) * NIN + i] : 0.f;
  }
  __syncthreads();
  {  // layer 1 (4 inputs)
    float acc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int o = w * 8 + k;
      float a = sm.p[OFF_B1 + o];
#pragma unroll
      for (int i = 0; i < NIN; ++i) a = fmaf(sm.p[OFF_W1 + o * NIN + i], sm.x[lane][i], a);
      acc[k] = a;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) sm.z1[lane][w * 8 + k] = acc[k];
  }
  __syncthreads();
  dense64<true>(sm.p + OFF_W2, sm.p + OFF_B2, sm.z1, sm.z2);
  __syncthreads();
  dense64<true>(sm.p + OFF_W3, sm.p + OFF_B3, sm.z2, sm.z3);
  __syncthreads();
  if (w == 0) {
    float a = sm.p[OFF_B4];
    for (int i = 0; i < H; ++i) a = fmaf(sm.p[OFF_W4 + i], relu(sm.z3[lane][i]), a);
    sm.y[lane] = a;
  }
  __syncthreads();
}

__device__ void load_params(Smem& sm, const float* __restrict__ P) {
  for (int j = threadIdx.x; j < JACC_MLP_NPARAM; j += NT) sm.p[j] = P[j];
}

// gW[o][i] = sum_s dz[s][o] * act(h[s][i]) ; gb[o] = sum_s dz[s][o]; rows of length nin.
template <int NINL, bool RELU_IN>
__device__ void weight_grad(const float (*dz)[LD], const float* hin, int hld, float* gW, float* gb) {
  for (int t = threadIdx.x; t < H * NINL; t += NT) {
    const int o = t / NINL, i = t % NINL;
    float a = 0.f;
    for (int s = 0; s < S; ++s) {
      const float h = hin[s * hld + i];
      a = fmaf(dz[s][o], RELU_IN ? relu(h) : h, a);
    }
    gW[o * NINL + i] = a;
  }
  for (int o = threadIdx.x; o < H; o += NT) {
    float a = 0.f;
    for (int s = 0; s < S; ++s) a += dz[s][o];
    gb[o] = a;
  }
}

// dzi[s][i] = (z[s][i] > 0) * sum_o W[o][i] dzo[s][o], for this warp's 8 inputs i.
__device__ __forceinline__ void back64(const float* W, const float (*dzo)[LD], const float (*z)[LD], float (*dzi)[LD]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = 0.f;
  for (int o = 0; o < H; ++o) {
    const float g = dzo[lane][o];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] = fmaf(W[o * H + w * 8 + k], g, acc[k]);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int i = w * 8 + k;
    dzi[lane][i] = z[lane][i] > 0.f ? acc[k] : 0.f;
  }
}

__global__ void __launch_bounds__(NT) jacc_k_mlp_fwd_bwd(const float* __restrict__ P, const float* __restrict__ X,
                                                         const float* __restrict__ Y, int n, float* __restrict__ partial,
                                                         float* __restrict__ loss_partial, unsigned* step) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem& sm = *reinterpret_cast<Smem*>(smraw);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long s0 = (long long)blockIdx.x * S;
  const int nvalid = (int)((n - s0) < S ? (n - s0) : S);
  if (step && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(step, 1u);  // Adam step counter for this step
  load_params(sm, P);
  __syncthreads();
  forward_chunk(sm, X, s0, nvalid);
  // loss and dL/dy (mean over all n samples)
  if (w == 0) {
    const float e = lane < nvalid ? sm.y[lane] - Y[s0 + lane] : 0.f;
    sm.dy[lane] = 2.f * e / (float)n;
    float l = e * e;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if (lane == 0) loss_partial[blockIdx.x] = l;
  }
  __syncthreads();
  float* g = partial + (long long)blockIdx.x * JACC_MLP_NPARAM;
  // layer 4
  for (int i = threadIdx.x; i < H; i += NT) {
    float a = 0.f;
    for (int s = 0; s < S; ++s) a = fmaf(sm.dy[s], relu(sm.z3[s][i]), a);
    g[OFF_W4 + i] = a;
  }
  if (threadIdx.x == 0) {
    float a = 0.f;
    for (int s = 0; s < S; ++s) a += sm.dy[s];
    g[OFF_B4] = a;
  }
  // dz3[s][o] = dy[s] W4[o] (z3 > 0)
  for (int t = threadIdx.x; t < S * H; t += NT) {
    const int s = t / H, o = t % H;
    sm.d[s][o] = sm.z3[s][o] > 0.f ? sm.dy[s] * sm.p[OFF_W4 + o] : 0.f;
  }
  __syncthreads();
  weight_grad<H, true>(sm.d, &sm.z2[0][0], LD, g + OFF_W3, g + OFF_B3);
  back64(sm.p + OFF_W3, sm.d, sm.z2, sm.d2);  // dz2
  __syncthreads();
  weight_grad<H, true>(sm.d2, &sm.z1[0][0], LD, g + OFF_W2, g + OFF_B2);
  back64(sm.p + OFF_W2, sm.d2, sm.z1, sm.d);  // dz1 (overwrites dz3, no longer needed)
  __syncthreads();
  weight_grad<NIN, false>(sm.d, &sm.x[0][0], NIN, g + OFF_W1, g + OFF_B1);
}

// One thread per parameter: fixed-order sum of the chunk gradients, then Adam.
__global__ void __launch_bounds__(256) jacc_k_mlp_adam(float* __restrict__ P, float* __restrict__ M,
                                                       float* __restrict__ V, const float* __restrict__ partial,
                                                       int nparts, const float* __restrict__ loss_partial, int n,
                                                       float* loss_out, const unsigned* step, float lr, float b1,
                                                       float b2, float eps, float* grad_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (loss_out && j == 0) {
    float l = 0.f;
    for (int c = 0; c < nparts; ++c) l += loss_partial[c];
    *loss_out = l / (float)n;
  }
  if (j >= JACC_MLP_NPARAM) return;
  float gsum = 0.f;
  for (int c = 0; c < nparts; ++c) gsum += partial[(long long)c * JACC_MLP_NPARAM + j];
  if (grad_out) grad_out[j] = gsum;
  if (!step) return;  // gradient only
  const float t = (float)(*step);
  const float m = b1 * M[j] + (1.f - b1) * gsum;
  const float v = b2 * V[j] + (1.f - b2) * gsum * gsum;
  M[j] = m;
  V[j] = v;
  const float mh = m / (1.f - powf(b1, t));
  const float vh = v / (1.f - powf(b2, t));
  P[j] = P[j] - lr * mh / (sqrtf(vh) + eps);
}

__global__ void __launch_bounds__(NT) jacc_k_mlp_forward(const float* __restrict__ P, const float* __restrict__ X, int n,
                                                         float* __restrict__ Yout) {
  extern __shared__ __align__(16) unsigned char smraw[];
  Smem& sm = *reinterpret_cast<Smem*>(smraw);
  const long long s0 = (long long)blockIdx.x * S;
  const int nvalid = (int)((n - s0) < S ? (n - s0) : S);
  load_params(sm, P);
  __syncthreads();
  forward_chunk(sm, X, s0, nvalid);
  if (threadIdx.x < nvalid) Yout[s0 + threadIdx.x] = sm.y[threadIdx.x];
}

// Queries of JACC_NUM_TILES rows each: pick[q] = argmin over valid rows (ties
// to the lowest tile id), gap[q] = second-lowest valid prediction - lowest.
__global__ void jacc_k_mlp_pick(const float* __restrict__ pred, const int* __restrict__ valid, int nq, int ntile,
                                int* pick, float* gap) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  float best = 3.4e38f, second = 3.4e38f;
  int bi = -1;
  for (int t = 0; t < ntile; ++t) {
    if (!valid[q * ntile + t]) continue;
    const float v = pred[q * ntile + t];
    if (v < best) {
      second = best;
      best = v;
      bi = t;
    } else if (v < second) {
      second = v;
    }
  }
  pick[q] = bi;
  gap[q] = (bi >= 0 && second < 3.0e38f) ? second - best : 3.4e38f;
}

}  // namespace

namespace jacc {

size_t mlp_smem_bytes() { return sizeof(Smem); }

cudaError_t mlp_setup() {
  cudaError_t e = cudaFuncSetAttribute(jacc_k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(jacc_k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
}

int mlp_nparts(int n) { return (n + S - 1) / S; }

cudaError_t mlp_fwd_bwd(const float* P, const float* X, const float* Y, int n, float* partial, float* loss_partial,
                        unsigned* step, cudaStream_t s) {
  jacc_k_mlp_fwd_bwd<<<mlp_nparts(n), NT, sizeof(Smem), s>>>(P, X, Y, n, partial, loss_partial, step);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* P, float* M, float* V, const float* partial, int nparts, const float* loss_partial, int n,
                     float* loss_out, const unsigned* step, float lr, float b1, float b2, float eps, float* grad_out,
                     cudaStream_t s) {
  jacc_k_mlp_adam<<<(JACC_MLP_NPARAM + 255) / 256, 256, 0, s>>>(P, M, V, partial, nparts, loss_partial, n, loss_out,
                                                                 step, lr, b1, b2, eps, grad_out);
  return cudaGetLastError();
}

cudaError_t mlp_forward(const float* P, const float* X, int n, float* Y, cudaStream_t s) {
  jacc_k_mlp_forward<<<mlp_nparts(n), NT, sizeof(Smem), s>>>(P, X, n, Y);
  return cudaGetLastError();
}

cudaError_t mlp_pick(const float* pred, const int* valid, int nq, int ntile, int* pick, float* gap, cudaStream_t s) {
  jacc_k_mlp_pick<<<(nq + 127) / 128, 128, 0, s>>>(pred, valid, nq, ntile, pick, gap);
  return cudaGetLastError();
}

}  // namespace jacc
