// tds_mlp.cu -- learned warm start: per-contact features, and the
// 10 -> 64 -> 64 -> 3 ReLU network on BF16 tensor cores (mma.sync m16n8k16,
// FP32 accumulation) for inference inside the step and for training
// (forward, backward, Adam on FP32 master weights).
//
// The paper suggests data-driven models as future work (section
// "Discussion"); here a small network predicts the initial normal and
// friction impulses of every contact from local features, and the plain
// projected Gauss-Seidel solve still judges the result (it converges to the
// same residual; only the number of sweeps changes).
//
// Features (one row of 10 per contact): (J_n v*)/(|g| h), overlap/dbar,
// Lambda_n0/W, |Lambda_t0|/W, (Lambda_t0 . s)/W, persisted, Z_a, Z_b,
// depth below the column surface / dbar, contact type (0 pair, 1 terrain or
// wall, 2 tool); W = |g| h / (1/m_a + 1/m_b), s the unit tangential slip
// velocity at v* (or, below 1e-6 m/s, unit n x e_k with e_k the axis least
// aligned with n). Outputs: Lambda_n/W, (Lambda_t . s)/W, (Lambda_t . (n x s))/W.
#include <cuda_bf16.h>

#include "tds_internal.cuh"

namespace {

constexpr int kIn = 10, kHid = 64, kOut = 3;
// FP32 parameter vector, row-major: W1[64][10], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid,
              kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kOut * kHid,
              kParams = kOffB3 + kOut;

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t *>(&v);
}
__device__ __forceinline__ uint32_t pack_raw(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
// D += A B with A 16x16 (row), B 16x8 (col), BF16 inputs, FP32 accumulators.
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Weights as the kernels read them: BF16, K padded to multiples of 16 and the
// output layer padded to 8 rows; biases FP32.
struct Packed {
  __nv_bfloat16 W1[kHid][16];
  __nv_bfloat16 W2[kHid][kHid];
  __nv_bfloat16 W3[8][kHid];
  float b1[kHid], b2[kHid], b3[8];
};

__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16 *p) {  // two adjacent BF16
  return *reinterpret_cast<const uint32_t *>(p);
}

// Forward pass of one 16-row tile in one warp. X rows come as FP32 (10 used);
// keeps pre-activations z1, z2 (C layout) and the BF16 A fragments of h1, h2.
struct Fwd {
  float z1[8][4], z2[8][4], y[4];
  uint32_t A2[4][4], A3[4][4];
};

__device__ __forceinline__ void forward_tile(const Packed &P, const float *X, uint32_t row0, uint32_t m,
                                             Fwd &f) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  auto xv = [&](int r, int k) -> float {
    uint32_t row = row0 + r;
    return (row < m && k < kIn) ? X[(size_t)row * kIn + k] : 0.f;
  };
  uint32_t A1[4] = {pack_bf16(xv(g, 2 * t), xv(g, 2 * t + 1)), pack_bf16(xv(g + 8, 2 * t), xv(g + 8, 2 * t + 1)),
                    pack_bf16(xv(g, 2 * t + 8), xv(g, 2 * t + 9)),
                    pack_bf16(xv(g + 8, 2 * t + 8), xv(g + 8, 2 * t + 9))};
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16 *w = &P.W1[nt * 8 + g][0];
    mma16816(acc, A1, ld_pair(w + 2 * t), ld_pair(w + 2 * t + 8));
    const int c = nt * 8 + 2 * t;
    f.z1[nt][0] = acc[0] + P.b1[c];
    f.z1[nt][1] = acc[1] + P.b1[c + 1];
    f.z1[nt][2] = acc[2] + P.b1[c];
    f.z1[nt][3] = acc[3] + P.b1[c + 1];
  }
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    f.A2[kc][0] = pack_bf16(fmaxf(f.z1[2 * kc][0], 0.f), fmaxf(f.z1[2 * kc][1], 0.f));
    f.A2[kc][1] = pack_bf16(fmaxf(f.z1[2 * kc][2], 0.f), fmaxf(f.z1[2 * kc][3], 0.f));
    f.A2[kc][2] = pack_bf16(fmaxf(f.z1[2 * kc + 1][0], 0.f), fmaxf(f.z1[2 * kc + 1][1], 0.f));
    f.A2[kc][3] = pack_bf16(fmaxf(f.z1[2 * kc + 1][2], 0.f), fmaxf(f.z1[2 * kc + 1][3], 0.f));
  }
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16 *w = &P.W2[nt * 8 + g][0];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) mma16816(acc, f.A2[kc], ld_pair(w + kc * 16 + 2 * t), ld_pair(w + kc * 16 + 2 * t + 8));
    const int c = nt * 8 + 2 * t;
    f.z2[nt][0] = acc[0] + P.b2[c];
    f.z2[nt][1] = acc[1] + P.b2[c + 1];
    f.z2[nt][2] = acc[2] + P.b2[c];
    f.z2[nt][3] = acc[3] + P.b2[c + 1];
  }
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    f.A3[kc][0] = pack_bf16(fmaxf(f.z2[2 * kc][0], 0.f), fmaxf(f.z2[2 * kc][1], 0.f));
    f.A3[kc][1] = pack_bf16(fmaxf(f.z2[2 * kc][2], 0.f), fmaxf(f.z2[2 * kc][3], 0.f));
    f.A3[kc][2] = pack_bf16(fmaxf(f.z2[2 * kc + 1][0], 0.f), fmaxf(f.z2[2 * kc + 1][1], 0.f));
    f.A3[kc][3] = pack_bf16(fmaxf(f.z2[2 * kc + 1][2], 0.f), fmaxf(f.z2[2 * kc + 1][3], 0.f));
  }
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const __nv_bfloat16 *w = &P.W3[g][0];
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) mma16816(acc, f.A3[kc], ld_pair(w + kc * 16 + 2 * t), ld_pair(w + kc * 16 + 2 * t + 8));
  const int c = 2 * t;
  f.y[0] = acc[0] + P.b3[c];
  f.y[1] = acc[1] + P.b3[c + 1];
  f.y[2] = acc[2] + P.b3[c];
  f.y[3] = acc[3] + P.b3[c + 1];
}

// FP32 master parameters -> packed BF16 weights.
__global__ void k_pack(const float *params, Packed *P) {
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < kHid * 16; i += blockDim.x * gridDim.x) {
    int o = i / 16, k = i % 16;
    P->W1[o][k] = __float2bfloat16_rn(k < kIn ? params[kOffW1 + o * kIn + k] : 0.f);
  }
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < kHid * kHid; i += blockDim.x * gridDim.x)
    P->W2[i / kHid][i % kHid] = __float2bfloat16_rn(params[kOffW2 + i]);
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < 8 * kHid; i += blockDim.x * gridDim.x) {
    int o = i / kHid, k = i % kHid;
    P->W3[o][k] = __float2bfloat16_rn(o < kOut ? params[kOffW3 + o * kHid + k] : 0.f);
  }
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < kHid; i += blockDim.x * gridDim.x) {
    P->b1[i] = params[kOffB1 + i];
    P->b2[i] = params[kOffB2 + i];
  }
  for (int i = threadIdx.x + blockIdx.x * blockDim.x; i < 8; i += blockDim.x * gridDim.x)
    P->b3[i] = i < kOut ? params[kOffB3 + i] : 0.f;
}

// Inference on m rows of FP32 features (row-major, 10 per row) -> Y (3 per row).
__global__ void __launch_bounds__(256) k_forward(const Packed *gP, const float *X, uint32_t m, float *Y) {
  __shared__ Packed P;
  for (int i = threadIdx.x; i < (int)(sizeof(Packed) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t *>(&P)[i] = reinterpret_cast<const uint32_t *>(gP)[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t warps = (blockDim.x >> 5) * gridDim.x;
  for (uint32_t tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < m; tile += warps) {
    Fwd f;
    forward_tile(P, X, tile * 16, m, f);
    float y2a = __shfl_down_sync(0xffffffffu, f.y[0], 1), y2b = __shfl_down_sync(0xffffffffu, f.y[2], 1);
    if (t == 0) {
      uint32_t ra = tile * 16 + g, rb = ra + 8;
      if (ra < m) { Y[ra * 3] = f.y[0]; Y[ra * 3 + 1] = f.y[1]; Y[ra * 3 + 2] = y2a; }
      if (rb < m) { Y[rb * 3] = f.y[2]; Y[rb * 3 + 1] = f.y[3]; Y[rb * 3 + 2] = y2b; }
    }
  }
}

// ---------------------------------------------------------------------------
// training: loss and gradients of L = (1/(3m)) sum (y - t)^2
// ---------------------------------------------------------------------------
constexpr int kTrainWarps = 8;
constexpr int kRows = 16 * kTrainWarps;  // rows per block iteration

struct Stage {  // per block: the tiles the weight-gradient products read (BF16)
  __nv_bfloat16 X[kRows][16];
  __nv_bfloat16 h1[kRows][kHid];
  __nv_bfloat16 h2[kRows][kHid];
  __nv_bfloat16 dz1[kRows][kHid];
  __nv_bfloat16 dz2[kRows][kHid];
  __nv_bfloat16 dy[kRows][16];
};

// A fragment of S^T (S row-major [rows][cols]): A[m][k] = S[k0 + k][m0 + m].
template <int C>
__device__ __forceinline__ void frag_at(const __nv_bfloat16 (*S)[C], int k0, int m0, uint32_t (&a)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  a[0] = pack_raw(S[k0 + 2 * t][m0 + g], S[k0 + 2 * t + 1][m0 + g]);
  a[1] = pack_raw(S[k0 + 2 * t][m0 + g + 8], S[k0 + 2 * t + 1][m0 + g + 8]);
  a[2] = pack_raw(S[k0 + 2 * t + 8][m0 + g], S[k0 + 2 * t + 9][m0 + g]);
  a[3] = pack_raw(S[k0 + 2 * t + 8][m0 + g + 8], S[k0 + 2 * t + 9][m0 + g + 8]);
}
// B fragment of S itself (B[k][n] = S[k0 + k][n0 + n]).
template <int C>
__device__ __forceinline__ void frag_b(const __nv_bfloat16 (*S)[C], int k0, int n0, uint32_t &b0, uint32_t &b1) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  b0 = pack_raw(S[k0 + 2 * t][n0 + g], S[k0 + 2 * t + 1][n0 + g]);
  b1 = pack_raw(S[k0 + 2 * t + 8][n0 + g], S[k0 + 2 * t + 9][n0 + g]);
}

// Sum over the 8 lanes sharing t (the 16 rows) of a per-column value; lane t
// (< 4) adds it to dst when valid.
__device__ __forceinline__ void col_sum_add(float v, float *dst, bool valid = true) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  if ((threadIdx.x & 31) < 4 && valid) atomicAdd(dst, v);
}

__global__ void __launch_bounds__(kTrainWarps * 32) k_loss_grad(const Packed *gP, const float *X,
                                                                 const float *T, uint32_t m,
                                                                 float *grad, float *loss) {
  __shared__ Packed P;
  extern __shared__ __align__(16) unsigned char dyn[];
  Stage &S = *reinterpret_cast<Stage *>(dyn);
  for (int i = threadIdx.x; i < (int)(sizeof(Packed) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t *>(&P)[i] = reinterpret_cast<const uint32_t *>(gP)[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const float scale = 2.0f / (3.0f * (float)m);
  float lsum = 0.f;
  for (uint32_t base = blockIdx.x * kRows; base < m; base += gridDim.x * kRows) {
    const uint32_t row0 = base + warp * 16;
    const int r0 = warp * 16;  // this warp's rows in the stage
    Fwd f;
    forward_tile(P, X, row0, m, f);
    // dL/dy (C layout: rows g, g+8; cols 2t, 2t+1; 3 outputs used)
    float dy[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int col = 2 * t + (q & 1);
      const uint32_t row = row0 + g + (q >> 1) * 8;
      float e = 0.f;
      if (col < kOut && row < m) e = f.y[q] - T[(size_t)row * kOut + col];
      lsum += e * e;
      dy[q] = scale * e;
    }
    col_sum_add(dy[0] + dy[2], &grad[kOffB3 + min(2 * t, kOut - 1)], 2 * t < kOut);
    col_sum_add(dy[1] + dy[3], &grad[kOffB3 + min(2 * t + 1, kOut - 1)], 2 * t + 1 < kOut);
    // dh2 = dy W3 (K = 8 outputs, padded to 16)
    uint32_t Ady[4] = {pack_bf16(dy[0], dy[1]), pack_bf16(dy[2], dy[3]), 0u, 0u};
    float dz2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      uint32_t b0 = pack_raw(P.W3[2 * t][nt * 8 + g], P.W3[2 * t + 1][nt * 8 + g]);
      mma16816(acc, Ady, b0, 0u);
#pragma unroll
      for (int q = 0; q < 4; ++q) dz2[nt][q] = f.z2[nt][q] > 0.f ? acc[q] : 0.f;
    }
    // dh1 = dz2 W2
    uint32_t Adz2[4][4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      Adz2[kc][0] = pack_bf16(dz2[2 * kc][0], dz2[2 * kc][1]);
      Adz2[kc][1] = pack_bf16(dz2[2 * kc][2], dz2[2 * kc][3]);
      Adz2[kc][2] = pack_bf16(dz2[2 * kc + 1][0], dz2[2 * kc + 1][1]);
      Adz2[kc][3] = pack_bf16(dz2[2 * kc + 1][2], dz2[2 * kc + 1][3]);
    }
    float dz1[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) {
        uint32_t b0 = pack_raw(P.W2[kc * 16 + 2 * t][nt * 8 + g], P.W2[kc * 16 + 2 * t + 1][nt * 8 + g]);
        uint32_t b1 = pack_raw(P.W2[kc * 16 + 2 * t + 8][nt * 8 + g], P.W2[kc * 16 + 2 * t + 9][nt * 8 + g]);
        mma16816(acc, Adz2[kc], b0, b1);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) dz1[nt][q] = f.z1[nt][q] > 0.f ? acc[q] : 0.f;
    }
    // bias gradients (FP32 column sums)
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = nt * 8 + 2 * t;
      col_sum_add(dz2[nt][0] + dz2[nt][2], &grad[kOffB2 + c]);
      col_sum_add(dz2[nt][1] + dz2[nt][3], &grad[kOffB2 + c + 1]);
      col_sum_add(dz1[nt][0] + dz1[nt][2], &grad[kOffB1 + c]);
      col_sum_add(dz1[nt][1] + dz1[nt][3], &grad[kOffB1 + c + 1]);
    }
    // stage the tiles the weight gradients read
    for (int k = lane; k < 16 * 16; k += 32) {
      const int r = k / 16, c = k % 16;
      const uint32_t row = row0 + r;
      S.X[r0 + r][c] = __float2bfloat16_rn((row < m && c < kIn) ? X[(size_t)row * kIn + c] : 0.f);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = r0 + g + (q >> 1) * 8, c = nt * 8 + 2 * t + (q & 1);
        S.h1[r][c] = __float2bfloat16_rn(fmaxf(f.z1[nt][q], 0.f));
        S.h2[r][c] = __float2bfloat16_rn(fmaxf(f.z2[nt][q], 0.f));
        S.dz1[r][c] = __float2bfloat16_rn(dz1[nt][q]);
        S.dz2[r][c] = __float2bfloat16_rn(dz2[nt][q]);
      }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = r0 + g + (q >> 1) * 8, c = 2 * t + (q & 1);
      S.dy[r][c] = __float2bfloat16_rn(dy[q]);
      S.dy[r][c + 8] = __float2bfloat16_rn(0.f);
    }
    __syncthreads();
    // weight gradients over the block's kRows rows: 8 tiles of dW1 (64x16),
    // 32 of dW2 (64x64), 8 of dW3 (8x64, M padded to 16)
    for (int tile = warp; tile < 48; tile += kTrainWarps) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      int which, mt, nt;
      if (tile < 8) { which = 1; mt = tile >> 1; nt = tile & 1; }
      else if (tile < 40) { which = 2; mt = (tile - 8) >> 3; nt = (tile - 8) & 7; }
      else { which = 3; mt = 0; nt = tile - 40; }
      for (int kc = 0; kc < kRows / 16; ++kc) {
        uint32_t a[4], b0, b1;
        if (which == 1) { frag_at<kHid>(S.dz1, kc * 16, mt * 16, a); frag_b<16>(S.X, kc * 16, nt * 8, b0, b1); }
        else if (which == 2) { frag_at<kHid>(S.dz2, kc * 16, mt * 16, a); frag_b<kHid>(S.h1, kc * 16, nt * 8, b0, b1); }
        else { frag_at<16>(S.dy, kc * 16, 0, a); frag_b<kHid>(S.h2, kc * 16, nt * 8, b0, b1); }
        mma16816(acc, a, b0, b1);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int o = mt * 16 + g + (q >> 1) * 8, i = nt * 8 + 2 * t + (q & 1);
        if (which == 1) { if (i < kIn) atomicAdd(&grad[kOffW1 + o * kIn + i], acc[q]); }
        else if (which == 2) atomicAdd(&grad[kOffW2 + o * kHid + i], acc[q]);
        else if (o < kOut) atomicAdd(&grad[kOffW3 + o * kHid + i], acc[q]);
      }
    }
    __syncthreads();
  }
  // loss
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 1);
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 2);
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 4);
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 8);
  lsum += __shfl_xor_sync(0xffffffffu, lsum, 16);
  if (lane == 0) atomicAdd(loss, lsum / (3.0f * (float)m));
}

__global__ void k_adam(float *params, float *grad, float *mom, float *vel, uint32_t step, float lr) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kParams; i += blockDim.x * gridDim.x) {
    float g = grad[i];
    float m = b1 * mom[i] + (1.f - b1) * g;
    float v = b2 * vel[i] + (1.f - b2) * g * g;
    mom[i] = m;
    vel[i] = v;
    params[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    grad[i] = 0.f;
  }
}

// ---------------------------------------------------------------------------
// inside the step: surface columns, features, learned initial impulses
// ---------------------------------------------------------------------------
__device__ __forceinline__ int ordered(float f) {  // float -> int with the same order
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float unordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

// Column of a centre in its scene: heightfield cells grouped cf x cf, FP32
// with explicit rounding (the same decision as the oracle's).
__device__ __forceinline__ uint32_t column_of(const SceneGeo &G, float px, float py) {
  const float w = __fmul_rn(G.hf_cell, (float)G.cf);
  const float tx = __fdiv_rn(__fsub_rn(px, G.hf_x0), w), ty = __fdiv_rn(__fsub_rn(py, G.hf_y0), w);
  const float fx = floorf(tx), fy = floorf(ty);
  int i, j;
  if (!(fx >= 0.0f)) i = 0; else if (fx > (float)(G.ncx - 1)) i = G.ncx - 1; else i = (int)fx;
  if (!(fy >= 0.0f)) j = 0; else if (fy > (float)(G.ncy - 1)) j = G.ncy - 1; else j = (int)fy;
  return G.col_off + (uint32_t)(j * G.ncx + i);
}

__global__ void k_columns_clear(uint32_t ncols, int *surf) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < ncols; c += gridDim.x * blockDim.x)
    surf[c] = ordered(-INFINITY);
}
__global__ void k_columns(DevPtrs d, StepConsts k, int *surf) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k.n; i += gridDim.x * blockDim.x) {
    const SceneGeo &G = k.geo[d.sid[i]];
    if (G.cf <= 0) continue;
    const float4 P = d.pos[i];
    if (P.w == 0.0f) continue;  // dormant reserve slot
    atomicMax(surf + column_of(G, P.x, P.y), ordered(__fadd_rn(P.z, P.w)));
  }
}

// Slip direction fallback: unit n x e_k with e_k the axis least aligned with n.
__device__ __forceinline__ float3 axis_tangent(float3 n) {
  float3 e = make_float3(1.f, 0.f, 0.f);
  float best = fabsf(n.x);
  if (fabsf(n.y) < best) { best = fabsf(n.y); e = make_float3(0.f, 1.f, 0.f); }
  if (fabsf(n.z) < best) e = make_float3(0.f, 0.f, 1.f);
  float3 t = cross(n, e);
  return rsqrtf(dot(t, t)) * t;
}

// The contacts without previous-step impulses, appended to new_idx (the
// only ones the network starts when no training data are recorded).
__global__ void k_new_contacts(DevPtrs d) {
  const uint32_t nc = d.ctr[CTR_NC];
  const uint32_t lane = threadIdx.x & 31;
  for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < nc;
       base += gridDim.x * blockDim.x) {
    const uint32_t c = base + lane;
    const bool fresh = c < nc && d.c_flag[c] == 0;
    const unsigned m = __ballot_sync(0xffffffffu, fresh);
    uint32_t at = 0;
    if (lane == 0 && m) at = atomicAdd(d.ctr + CTR_NEW, (uint32_t)__popc(m));
    at = __shfl_sync(0xffffffffu, at, 0);
    if (fresh) d.new_idx[at + __popc(m & ((1u << lane) - 1u))] = c;
  }
}

// Features at v* with the previous-step impulses, and the slip direction s
// and scale W for the outputs: of every contact (row c of feat), or with
// compact != 0 of the contacts listed in new_idx (row j for new_idx[j]).
__global__ void k_features(DevPtrs d, StepConsts k, const int *surf, int compact) {
  const uint32_t nrows = compact ? d.ctr[CTR_NEW] : d.ctr[CTR_NC];
  const float gh = sqrtf(k.g[0] * k.g[0] + k.g[1] * k.g[1] + k.g[2] * k.g[2]) * k.dt;
  for (uint32_t row = blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += gridDim.x * blockDim.x) {
    const uint32_t c = compact ? d.new_idx[row] : row;
    const uint2 ab = d.c_ab[c];
    const bool dyn = (ab.y & TDS_STATIC) == 0u;
    const float4 rn = d.c_rn[c], rq = d.c_rq[c];
    const float3 n = f3(rn);
    const float la = rn.w, lb = rq.x;
    const float4 P = d.pos[ab.x];
    const SceneGeo &G = k.geo[d.sid[ab.x]];
    const float4 va = d.pv[2 * ab.x], wa = d.pv[2 * ab.x + 1];
    float3 vb, wb;
    float imb = 0.f, rb = 0.f;
    if (dyn) {
      const float4 v4 = d.pv[2 * ab.y], w4 = d.pv[2 * ab.y + 1];
      vb = f3(v4); wb = f3(w4); imb = v4.w; rb = d.pos[ab.y].w;
    } else {
      vb = f3(d.c_sv[c]); wb = f3(d.c_sw[c]);
    }
    const float delta = 2.f * (P.w - la);
    const float dbar = dyn ? P.w + rb : 2.f * P.w;
    const float3 dv = vb - f3(va);
    const float3 u = dv - cross(lb * wb + la * f3(wa), n);
    const float3 ut = u - dot(u, n) * n;
    const float ms2 = dot(ut, ut);
    const float3 s = ms2 > 1e-12f ? rsqrtf(ms2) * ut : axis_tangent(n);
    const float W = gh / (va.w + imb);
    const float4 l0 = d.c_la[c];
    float3 t1, t2;
    onb(n, t1, t2);
    const float3 lt = l0.y * t1 + l0.z * t2;
    float depth = 0.f;
    if (G.cf > 0) depth = (unordered(surf[column_of(G, P.x, P.y)]) - P.z) / dbar;
    const uint32_t sid = ab.y & ~TDS_STATIC;
    float *F = d.feat + (size_t)row * 10;
    F[0] = dot(n, dv) / gh;
    F[1] = delta / dbar;
    F[2] = l0.x / W;
    F[3] = sqrtf(dot(lt, lt)) / W;
    F[4] = dot(lt, s) / W;
    F[5] = (float)d.c_flag[c];
    F[6] = (float)d.inc_cnt[ab.x];
    F[7] = dyn ? (float)d.inc_cnt[ab.y] : 0.f;
    F[8] = depth;
    F[9] = dyn ? 0.f : (sid >= 1u + G.nwall ? 2.f : 1.f);
    d.sdirw[row] = make_float4(s.x, s.y, s.z, W);
  }
}

// Network on the features, and the initial impulses it predicts for the
// contacts without previous-step impulses (a contact that persisted keeps
// those, which already start it near its solution):
// Lambda_n = W y0, Lambda_t = W (y1 s + y2 n x s), no rolling impulse; all
// projected into the bounds (normal >= -f_c, Coulomb disk).
__global__ void __launch_bounds__(256) k_learned(DevPtrs d, const Packed *gP, int compact) {
  __shared__ Packed P;
  for (int i = threadIdx.x; i < (int)(sizeof(Packed) / 4); i += blockDim.x)
    reinterpret_cast<uint32_t *>(&P)[i] = reinterpret_cast<const uint32_t *>(gP)[i];
  __syncthreads();
  const uint32_t nc = compact ? d.ctr[CTR_NEW] : d.ctr[CTR_NC];  // rows of feat
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const uint32_t warps = (blockDim.x >> 5) * gridDim.x;
  for (uint32_t tile = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); tile * 16 < nc; tile += warps) {
    Fwd f;
    forward_tile(P, d.feat, tile * 16, nc, f);
    const float y2a = __shfl_down_sync(0xffffffffu, f.y[0], 1), y2b = __shfl_down_sync(0xffffffffu, f.y[2], 1);
    if (t != 0) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const uint32_t row = tile * 16 + g + 8 * h;
      if (row >= nc) continue;
      const uint32_t c = compact ? d.new_idx[row] : row;
      if (d.c_flag[c]) continue;
      const float y0 = h ? f.y[2] : f.y[0], y1 = h ? f.y[3] : f.y[1], y2 = h ? y2b : y2a;
      const float4 sw = d.sdirw[row], rn = d.c_rn[c], rq = d.c_rq[c];
      const float2 rm = d.c_rm[c];
      const float3 n = f3(rn), s = f3(sw);
      const float W = sw.w;
      const float ln = fmaxf(W * y0, -rq.w);
      const float3 lt = W * (y1 * s + y2 * cross(n, s));
      float3 t1, t2;
      onb(n, t1, t2);
      float a1 = dot(lt, t1), a2 = dot(lt, t2);
      const float bt = rm.x * fabsf(ln), m2 = a1 * a1 + a2 * a2;
      if (m2 > bt * bt) { const float sc = bt > 0.f ? bt * rsqrtf(m2) : 0.f; a1 *= sc; a2 *= sc; }
      d.c_la[c] = make_float4(ln, a1, a2, 0.f);
      d.c_lb[c] = make_float2(0.f, 0.f);
    }
  }
}

}  // namespace

// compact != 0: features of the new contacts only (listed first), for the
// learned warm start when no training data are recorded.
int tds_launch_features(const DevPtrs &d, const StepConsts &k, int *surf, uint32_t ncols, uint32_t cap,
                        int compact, cudaStream_t st) {
  int launches = 1;
  if (ncols > 0) {
    k_columns_clear<<<(ncols + 255) / 256, 256, 0, st>>>(ncols, surf);
    k_columns<<<(k.n + 255) / 256, 256, 0, st>>>(d, k, surf);
    launches += 2;
  }
  unsigned blocks = (cap + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (compact) {
    cudaMemsetAsync(d.ctr + CTR_NEW, 0, sizeof(uint32_t), st);
    k_new_contacts<<<blocks, 256, 0, st>>>(d);
    launches += 1;
  }
  k_features<<<blocks, 256, 0, st>>>(d, k, surf, compact);
  return launches;
}
void tds_launch_learned(const DevPtrs &d, const void *packed, uint32_t cap, int compact, cudaStream_t st) {
  unsigned blocks = (cap + 127) / 128;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks == 0) blocks = 1;
  k_learned<<<blocks, 256, 0, st>>>(d, static_cast<const Packed *>(packed), compact);
}

size_t tds_mlp_packed_bytes() { return (sizeof(Packed) + 255) & ~(size_t)255; }
int tds_mlp_params() { return kParams; }

void tds_mlp_pack(const float *params, void *packed, cudaStream_t st) {
  k_pack<<<8, 256, 0, st>>>(params, static_cast<Packed *>(packed));
}
void tds_mlp_forward_launch(const void *packed, const float *X, uint32_t m, float *Y, cudaStream_t st) {
  unsigned blocks = (m + 16 * 8 - 1) / (16 * 8);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks == 0) blocks = 1;
  k_forward<<<blocks, 256, 0, st>>>(static_cast<const Packed *>(packed), X, m, Y);
}
cudaError_t tds_mlp_loss_grad_launch(const void *packed, const float *X, const float *T, uint32_t m,
                                     float *grad, float *loss, cudaStream_t st) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute((const void *)k_loss_grad,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Stage));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  unsigned blocks = (m + kRows - 1) / kRows;
  if (blocks > 152 * 2) blocks = 152 * 2;
  if (blocks == 0) blocks = 1;
  k_loss_grad<<<blocks, kTrainWarps * 32, sizeof(Stage), st>>>(static_cast<const Packed *>(packed), X, T, m,
                                                              grad, loss);
  return cudaGetLastError();
}
void tds_mlp_adam_launch(float *params, float *grad, float *mom, float *vel, uint32_t step, float lr,
                         cudaStream_t st) {
  k_adam<<<(kParams + 255) / 256, 256, 0, st>>>(params, grad, mom, vel, step, lr);
}
