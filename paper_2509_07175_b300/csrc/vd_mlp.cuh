// vd_mlp.cuh -- the learned proposal: a small MLP that ranks the 32 nearest
// sites of a site by how likely each one is a bisector neighbour (shares a face
// of the cell, Sec. 2.2).  The ranking only orders the point-in-cell search of
// the learned form; the exact tests still decide every clip.
//
// Input of site i: the offsets (v_k - v_i) / d_1 of its 32 nearest sites in
// distance order, d_1 the distance to the nearest one (96 values; z = 0 in 2D,
// so the 2D network uses 64 of them), bf16.  Network 96 -> 64 -> 64 -> 32 with
// ReLU, one logit per slot of the 32-NN list.  Weights: FP32 master copy (Adam)
// and a bf16 copy for the products.  Every product runs on the tensor cores
// (mma.sync m16n8k16, bf16 x bf16 with FP32 accumulation); one warp owns a tile
// of 16 rows (sites).
//
// Rounding points (the CPU check rounds at the same places): the inputs, the
// weights and the hidden activations after ReLU are bf16; in the backward pass
// dZ, dH2 and dH1 are rounded to bf16 where they enter a product.  Biases,
// logits, bias gradients and weight gradients stay FP32.
//
// Loss: mean binary cross-entropy over rows x 32 slots, label 1 when the slot's
// site is a neighbour of the row's site.
#pragma once

#include <cuda_bf16.h>

#include "vd_dev.cuh"

namespace vd {
namespace mlp {

constexpr int NIN = 96, NH = 64, NOUT = 32;
// flat parameter layout (row-major weights, in x out)
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NIN * NH, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NH * NOUT, NPARAM = OFF_B3 + NOUT;
static_assert(NPARAM == 12448, "parameter layout");

using bf16 = __nv_bfloat16;

__device__ __forceinline__ unsigned pack2(bf16 lo, bf16 hi) {
  __nv_bfloat162 v;
  v.x = lo;  // low 16 bits: the lower column / row index
  v.y = hi;
  return *reinterpret_cast<unsigned*>(&v);
}

// D[16x8] += A[16x16] B[16x8]; bf16 operands, FP32 accumulators
__device__ __forceinline__ void mma16816(float* d, const unsigned* a, const unsigned* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C[16 x N] = A[16 x K] B[K x N] for one warp, operands read through element
// accessors A(r, k), B(k, n), each result element handed to store(r, n, v).
// Fragment layout of m16n8k16 (g = lane / 4, t = lane % 4): A holds rows g, g+8
// x columns 2t, 2t+1, 2t+8, 2t+9; B rows 2t, 2t+1, 2t+8, 2t+9 x column g; C rows
// g, g+8 x columns 2t, 2t+1.
template <int K, int N, typename FA, typename FB, typename FS>
__device__ __forceinline__ void warp_gemm(FA A, FB B, FS store, int lane) {
  const int g = lane >> 2, t = lane & 3;
  unsigned a[K / 16][4];
#pragma unroll
  for (int kk = 0; kk < K / 16; ++kk) {
    const int k0 = kk * 16;
    a[kk][0] = pack2(A(g, k0 + 2 * t), A(g, k0 + 2 * t + 1));
    a[kk][1] = pack2(A(g + 8, k0 + 2 * t), A(g + 8, k0 + 2 * t + 1));
    a[kk][2] = pack2(A(g, k0 + 2 * t + 8), A(g, k0 + 2 * t + 9));
    a[kk][3] = pack2(A(g + 8, k0 + 2 * t + 8), A(g + 8, k0 + 2 * t + 9));
  }
#pragma unroll 2
  for (int n0 = 0; n0 < N; n0 += 8) {
    float d[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kk = 0; kk < K / 16; ++kk) {
      const int k0 = kk * 16;
      unsigned b[2];
      b[0] = pack2(B(k0 + 2 * t, n0 + g), B(k0 + 2 * t + 1, n0 + g));
      b[1] = pack2(B(k0 + 2 * t + 8, n0 + g), B(k0 + 2 * t + 9, n0 + g));
      mma16816(d, a[kk], b);
    }
    store(g, n0 + 2 * t, d[0]);
    store(g, n0 + 2 * t + 1, d[1]);
    store(g + 8, n0 + 2 * t, d[2]);
    store(g + 8, n0 + 2 * t + 1, d[3]);
  }
}

// bf16 weights and FP32 biases staged in shared memory
struct Wsh {
  bf16 w1[NIN * NH];
  bf16 w2[NH * NH];
  bf16 w3[NH * NOUT];
  float b1[NH], b2[NH], b3[NOUT];
};

__device__ __forceinline__ void stage_weights(Wsh& S, const bf16* wb, const float* params) {
  for (int t = threadIdx.x; t < NIN * NH; t += blockDim.x) S.w1[t] = wb[OFF_W1 + t];
  for (int t = threadIdx.x; t < NH * NH; t += blockDim.x) S.w2[t] = wb[OFF_W2 + t];
  for (int t = threadIdx.x; t < NH * NOUT; t += blockDim.x) S.w3[t] = wb[OFF_W3 + t];
  for (int t = threadIdx.x; t < NH; t += blockDim.x) {
    S.b1[t] = params[OFF_B1 + t];
    S.b2[t] = params[OFF_B2 + t];
  }
  for (int t = threadIdx.x; t < NOUT; t += blockDim.x) S.b3[t] = params[OFF_B3 + t];
  __syncthreads();
}

// activations of one warp's 16 rows
struct Act {
  bf16 x[16 * NIN];
  bf16 h1[16 * NH];
  bf16 h2[16 * NH];
  float z[16 * NOUT];
};

// forward pass of the 16 rows in A.x; logits to A.z
__device__ __forceinline__ void forward16(const Wsh& S, Act& A, int lane) {
  warp_gemm<NIN, NH>([&](int r, int k) { return A.x[r * NIN + k]; },
                     [&](int k, int n) { return S.w1[k * NH + n]; },
                     [&](int r, int n, float v) { A.h1[r * NH + n] = __float2bfloat16_rn(fmaxf(v + S.b1[n], 0.f)); },
                     lane);
  __syncwarp();
  warp_gemm<NH, NH>([&](int r, int k) { return A.h1[r * NH + k]; },
                    [&](int k, int n) { return S.w2[k * NH + n]; },
                    [&](int r, int n, float v) { A.h2[r * NH + n] = __float2bfloat16_rn(fmaxf(v + S.b2[n], 0.f)); },
                    lane);
  __syncwarp();
  warp_gemm<NH, NOUT>([&](int r, int k) { return A.h2[r * NH + k]; },
                      [&](int k, int n) { return S.w3[k * NOUT + n]; },
                      [&](int r, int n, float v) { A.z[r * NOUT + n] = v + S.b3[n]; }, lane);
  __syncwarp();
}

// lane's three inputs (slot `lane` of the 32-NN list) of site i
template <typename T>
__device__ __forceinline__ void features_of(const Dev<T>& C, const int* knn, const T* delta, int i, int lane,
                                            float& fx, float& fy, float& fz) {
  int k = knn[(long long)i * 32 + lane];
  float s = 0.5f / (float)delta[i];  // delta = half the nearest distance
  fx = fy = fz = 0.f;
  if (k >= 0 && k < C.n) {
    fx = (float)(C.sites[3 * k] - C.sites[3 * i]) * s;
    fy = (float)(C.sites[3 * k + 1] - C.sites[3 * i + 1]) * s;
    fz = (float)(C.sites[3 * k + 2] - C.sites[3 * i + 2]) * s;
  }
}

struct RankSmem {
  Wsh W;
  Act A[4];
};

// Inference fused with feature construction and top-k selection: the candidate
// mask of site i has bit s set when slot s of its 32-NN list is among the topk
// largest logits (equal logits: the lower slot first).  Nothing but the mask is
// written.  4 warps per block, a tile of 16 sites per warp.
template <typename T>
__global__ void __launch_bounds__(128) k_mlp_rank(const __grid_constant__ Dev<T> C, const int* knn, const T* delta, const bf16* wb,
                                                  const float* params, int topk, unsigned* cmask) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RankSmem& SM = *reinterpret_cast<RankSmem*>(smem_raw);
  stage_weights(SM.W, wb, params);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Act& A = SM.A[warp];
  const int ntiles = (C.n + 15) / 16;
  for (int tile = blockIdx.x * 4 + warp; tile < ntiles; tile += gridDim.x * 4) {
    const int i0 = tile * 16;
    for (int r = 0; r < 16; ++r) {
      float fx = 0.f, fy = 0.f, fz = 0.f;
      if (i0 + r < C.n) features_of(C, knn, delta, i0 + r, lane, fx, fy, fz);
      A.x[r * NIN + 3 * lane] = __float2bfloat16_rn(fx);
      A.x[r * NIN + 3 * lane + 1] = __float2bfloat16_rn(fy);
      A.x[r * NIN + 3 * lane + 2] = __float2bfloat16_rn(fz);
    }
    __syncwarp();
    forward16(SM.W, A, lane);
    for (int r = 0; r < 16 && i0 + r < C.n; ++r) {
      const int i = i0 + r;
      const bool valid = knn[(long long)i * 32 + lane] >= 0;
      const float z = valid ? A.z[r * NOUT + lane] : -3.0e38f;
      int rank = 0;
#pragma unroll 8
      for (int j = 0; j < 32; ++j) {
        float zj = __shfl_sync(FULL, z, j);
        rank += (zj > z) || (zj == z && j < lane);
      }
      const unsigned m = __ballot_sync(FULL, valid && rank < topk);
      if (lane == 0) cmask[i] = m;
    }
    __syncwarp();
  }
}

// ----- training ----------------------------------------------------------------

struct TrainSmem {
  Wsh W;
  Act A[4];
  bf16 dz[4][16 * NOUT];
  bf16 dh2[4][16 * NH];
  bf16 dh1[4][16 * NH];
  float g[NPARAM];  // the block's gradient sum
};

// Forward and backward of `count` rows; row t of the batch is the stored row
// (pa * (start + t) + pc) mod rows, an affine permutation of all stored rows.
// Adds the gradient of the batch's mean loss to grads and the batch's summed
// (not averaged) loss to *loss_sum.  x: bf16 [rows*96], y: [rows] bit masks.
__global__ void __launch_bounds__(128) k_mlp_train(const bf16* wb, const float* params, const bf16* x,
                                                   const unsigned* y, long long rows, long long start, int count,
                                                   long long pa, long long pc, float* grads, float* loss_sum) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& SM = *reinterpret_cast<TrainSmem*>(smem_raw);
  for (int t = threadIdx.x; t < NPARAM; t += blockDim.x) SM.g[t] = 0.f;
  stage_weights(SM.W, wb, params);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Act& A = SM.A[warp];
  bf16* dz = SM.dz[warp];
  bf16* dh2 = SM.dh2[warp];
  bf16* dh1 = SM.dh1[warp];
  float* G = SM.g;
  const float inv = 1.f / ((float)count * (float)NOUT);
  const int ntiles = (count + 15) / 16;
  float lsum = 0.f, gb3 = 0.f;
  for (int tile = blockIdx.x * 4 + warp; tile < ntiles; tile += gridDim.x * 4) {
    const int r0 = tile * 16, nr = min(16, count - r0);
    long long myrow = -1;
    unsigned myy = 0;
    if (lane < nr) {
      myrow = (long long)(((unsigned long long)pa * (unsigned long long)(start + r0 + lane) + (unsigned long long)pc) %
                          (unsigned long long)rows);
      myy = y[myrow];
    }
    for (int r = 0; r < 16; ++r) {
      long long row = __shfl_sync(FULL, myrow, r);
      for (int k = lane; k < NIN; k += 32) A.x[r * NIN + k] = row >= 0 ? x[row * NIN + k] : __float2bfloat16_rn(0.f);
    }
    __syncwarp();
    forward16(SM.W, A, lane);
    // dZ = (sigmoid(z) - y) / (count * 32); loss = softplus(z) - y z
    for (int r = 0; r < 16; ++r) {
      const unsigned yy = __shfl_sync(FULL, myy, r);
      float g = 0.f;
      if (r < nr) {
        const float z = A.z[r * NOUT + lane];
        const float lab = (float)((yy >> lane) & 1u);
        const float sg = 1.f / (1.f + __expf(-z));
        g = (sg - lab) * inv;
        lsum += fmaxf(z, 0.f) + log1pf(__expf(-fabsf(z))) - lab * z;
        gb3 += g;
      }
      dz[r * NOUT + lane] = __float2bfloat16_rn(g);
    }
    __syncwarp();
    // dW3 += H2^T dZ  (64 x 32; the contraction runs over the tile's 16 rows)
#pragma unroll 1
    for (int m0 = 0; m0 < NH; m0 += 16)
      warp_gemm<16, NOUT>([&](int r, int k) { return A.h2[k * NH + m0 + r]; },
                          [&](int k, int n) { return dz[k * NOUT + n]; },
                          [&](int r, int n, float v) { atomicAdd(&G[OFF_W3 + (m0 + r) * NOUT + n], v); }, lane);
    // dH2 = (dZ W3^T) * [H2 > 0]
    warp_gemm<NOUT, NH>([&](int r, int k) { return dz[r * NOUT + k]; },
                        [&](int k, int n) { return SM.W.w3[n * NOUT + k]; },
                        [&](int r, int n, float v) {
                          float u = __bfloat162float(A.h2[r * NH + n]) > 0.f ? v : 0.f;
                          dh2[r * NH + n] = __float2bfloat16_rn(u);
                          atomicAdd(&G[OFF_B2 + n], u);
                        },
                        lane);
    __syncwarp();
    // dW2 += H1^T dH2
#pragma unroll 1
    for (int m0 = 0; m0 < NH; m0 += 16)
      warp_gemm<16, NH>([&](int r, int k) { return A.h1[k * NH + m0 + r]; },
                        [&](int k, int n) { return dh2[k * NH + n]; },
                        [&](int r, int n, float v) { atomicAdd(&G[OFF_W2 + (m0 + r) * NH + n], v); }, lane);
    // dH1 = (dH2 W2^T) * [H1 > 0]
    warp_gemm<NH, NH>([&](int r, int k) { return dh2[r * NH + k]; },
                      [&](int k, int n) { return SM.W.w2[n * NH + k]; },
                      [&](int r, int n, float v) {
                        float u = __bfloat162float(A.h1[r * NH + n]) > 0.f ? v : 0.f;
                        dh1[r * NH + n] = __float2bfloat16_rn(u);
                        atomicAdd(&G[OFF_B1 + n], u);
                      },
                      lane);
    __syncwarp();
    // dW1 += X^T dH1
#pragma unroll 1
    for (int m0 = 0; m0 < NIN; m0 += 16)
      warp_gemm<16, NH>([&](int r, int k) { return A.x[k * NIN + m0 + r]; },
                        [&](int k, int n) { return dh1[k * NH + n]; },
                        [&](int r, int n, float v) { atomicAdd(&G[OFF_W1 + (m0 + r) * NH + n], v); }, lane);
    __syncwarp();
  }
  atomicAdd(&G[OFF_B3 + lane], gb3);
  lsum = warp_sum(lsum);
  if (lane == 0) atomicAdd(loss_sum, lsum);
  __syncthreads();
  for (int t = threadIdx.x; t < NPARAM; t += blockDim.x) {
    float v = G[t];
    if (v != 0.f) atomicAdd(&grads[t], v);
  }
}

// one Adam step (Kingma and Ba, bias-corrected moments; c1 = 1 - b1^t,
// c2 = 1 - b2^t) on the FP32 master weights, then the bf16 copy
__global__ void k_adam(float* params, const float* grads, float* m, float* v, bf16* wb, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NPARAM) return;
  float g = grads[t];
  float mt = b1 * m[t] + (1.f - b1) * g;
  float vt = b2 * v[t] + (1.f - b2) * g * g;
  m[t] = mt;
  v[t] = vt;
  float p = params[t] - lr * (mt / c1) / (sqrtf(vt / c2) + eps);
  params[t] = p;
  wb[t] = __float2bfloat16_rn(p);
}

// out[t] = in[t] * scale, t < count
__global__ void k_scale(const float* in, float* out, int count, float scale) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) out[t] = in[t] * scale;
}

// bf16 copy of the master weights
__global__ void k_to_bf16(const float* params, bf16* wb) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < NPARAM) wb[t] = __float2bfloat16_rn(params[t]);
}

// He-uniform weights (bound sqrt(6 / fan_in)), zero biases, zero Adam moments;
// one 64-bit mix of (seed, index) per weight
__global__ void k_mlp_init(float* params, float* m, float* v, bf16* wb, unsigned long long seed) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= NPARAM) return;
  int fan = 0;
  if (t < OFF_B1) fan = NIN;
  else if (t >= OFF_W2 && t < OFF_B2) fan = NH;
  else if (t >= OFF_W3 && t < OFF_B3) fan = NH;
  float w = 0.f;
  if (fan) {
    unsigned long long h = mix64(seed ^ mix64(0x9E3779B97F4A7C15ull * (unsigned long long)(t + 1)));
    float u = (float)(h >> 40) * (1.f / 16777216.f);  // [0, 1)
    w = (2.f * u - 1.f) * sqrtf(6.f / (float)fan);
  }
  params[t] = w;
  m[t] = 0.f;
  v[t] = 0.f;
  wb[t] = __float2bfloat16_rn(w);
}

// logits of `rows` stored rows (evaluation and tests)
__global__ void __launch_bounds__(128) k_mlp_forward(const bf16* wb, const float* params, const bf16* x,
                                                     long long rows, float* logits) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RankSmem& SM = *reinterpret_cast<RankSmem*>(smem_raw);
  stage_weights(SM.W, wb, params);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  Act& A = SM.A[warp];
  const long long ntiles = (rows + 15) / 16;
  for (long long tile = blockIdx.x * 4 + warp; tile < ntiles; tile += gridDim.x * 4) {
    const long long r0 = tile * 16;
    const int nr = (int)min(16ll, rows - r0);
    for (int t = lane; t < 16 * NIN; t += 32) {
      int r = t / NIN;
      A.x[t] = r < nr ? x[(r0 + r) * NIN + (t - r * NIN)] : __float2bfloat16_rn(0.f);
    }
    __syncwarp();
    forward16(SM.W, A, lane);
    for (int r = 0; r < nr; ++r) logits[(r0 + r) * NOUT + lane] = A.z[r * NOUT + lane];
    __syncwarp();
  }
}

// features of every site, bf16 [n*96] (training data)
template <typename T>
__global__ void k_features(Dev<T> C, const int* knn, const T* delta, bf16* x) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)C.n * 32) return;
  int i = (int)(t >> 5), lane = (int)(t & 31);
  float f[3];
  features_of(C, knn, delta, i, lane, f[0], f[1], f[2]);
  for (int d = 0; d < 3; ++d) x[(long long)i * NIN + 3 * lane + d] = __float2bfloat16_rn(f[d]);
}

// labels: bit s of site i set when slot s of its 32-NN list is one of its
// neighbours in the CSR of the last computation (neighbours are ascending)
__global__ void k_labels(int n, const int* knn, const long long* noff, const int* nidx, unsigned* y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned m = 0;
  const long long b = noff[i], e = noff[i + 1];
  for (int s = 0; s < 32; ++s) {
    int k = knn[(long long)i * 32 + s];
    if (k < 0) continue;
    long long lo = b, hi = e;
    while (lo < hi) {
      long long mid = (lo + hi) >> 1;
      if (nidx[mid] < k) lo = mid + 1;
      else hi = mid;
    }
    if (lo < e && nidx[lo] == k) m |= 1u << s;
  }
  y[i] = m;
}

}  // namespace mlp
}  // namespace vd
