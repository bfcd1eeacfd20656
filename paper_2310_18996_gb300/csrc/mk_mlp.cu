// Surrogate MLP kernels: 4 -> 128 -> 128 -> 128 -> 35, GELU hidden units.
//
// Tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation) run
// every 128-wide product: the hidden layers, the output layer, the backward
// products dh = dz W and the weight gradients dW = dz^T h.  Operand precision
// in training (the same on the FP64 oracle's BF16 path): weights BF16
// (rounded from an FP32 master copy that Adam updates); hidden activations
// stored as BF16; the output y in FP32; the backward operands dy and
// dz = dh * GELU'(z) rounded to BF16, with GELU'(z) from the FP32
// pre-activation.  Inference takes each hidden activation as two BF16 terms
// (hi + lo), so that its outputs are smooth in the inputs: the tuning
// differentiates them.  The 4-wide first layer and its weight gradient run
// on the FP32 cores with FP32 inputs.
//
// Training: one cluster of 8 CTAs runs a whole epoch in one launch.  Each CTA
// takes 32 samples of a step; per layer it writes its partial weight and bias
// gradients to shared memory, and after a cluster barrier every CTA sums one
// eighth of that layer's parameters over the 8 CTAs' partials (distributed
// shared memory, fixed order), applies Adam to them and writes the new
// weights into every CTA's shared-memory copy (no CTA uses that layer again
// in the step).  The weights reach global memory only through the host,
// which refreshes the global image from the FP32 master after the launch.
//
// Parameter vector: W0 [128x4], b0, W1 [128x128], b1, W2 [128x128], b2,
// W3 [35x128], b3, each W row-major [out][in].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mk_mlp.h"

namespace mk {
namespace {

constexpr int kS = 32;        // samples per CTA pass
constexpr int kCl = 8;        // CTAs of the training cluster
constexpr int kThr = 256;     // threads per CTA (8 warps)
constexpr int kLd = 136;      // BF16 row stride of 128-wide buffers (272 B: conflict-free ldmatrix rows)
constexpr int kLdY = 56;      // BF16 row stride of the output-gradient buffer (48 columns used)
constexpr int kW3R = 48;      // rows of W3 in the image (35 real, zero rows after)
constexpr int kLdP = 136;     // FP32 row stride of the gradient partials
constexpr int kOutP = 40;     // outputs padded to 5 tiles of 8

__host__ __device__ constexpr int dim(int l) { return l == 0 ? 4 : (l == 4 ? 35 : 128); }

// canonical offsets of W_l and b_l in the parameter vector
__host__ __device__ constexpr int w_off(int l) {
  return l == 0 ? 0 : w_off(l - 1) + dim(l) * dim(l - 1) + dim(l);
}
__host__ __device__ constexpr int b_off(int l) { return w_off(l) + dim(l + 1) * dim(l); }

// Weight image (bytes), identical in global and shared memory.
struct Img {
  static constexpr int W1 = 0;
  static constexpr int W2 = W1 + 128 * kLd * 2;
  static constexpr int W3 = W2 + 128 * kLd * 2;
  static constexpr int W0 = W3 + kW3R * kLd * 2;  // FP32 [128][4]
  static constexpr int B0 = W0 + 128 * 4 * 4;
  static constexpr int B1 = B0 + 128 * 4;
  static constexpr int B2 = B1 + 128 * 4;
  static constexpr int B3 = B2 + 128 * 4;
  static constexpr int BYTES = B3 + kOutP * 4;
};
static_assert(Img::BYTES % 16 == 0, "image is copied in 16-byte pieces");

// Work buffers after the image (bytes from the start of shared memory).
struct Wk {
  static constexpr int X = Img::BYTES;          // FP32 [32][4]
  static constexpr int H0 = X + kS * 4 * 4;      // BF16 [32][kLd] each
  static constexpr int H1 = H0 + kS * kLd * 2;
  static constexpr int H2 = H1 + kS * kLd * 2;
  static constexpr int Y = H2 + kS * kLd * 2;    // FP32 [32][kOutP]
  static constexpr int FWD_END = Y + kS * kOutP * 4;
  // inference keeps each hidden activation as two BF16 terms: the low terms
  // (BF16 [32][kLd] each) in space the training buffers use
  static constexpr int HL0 = FWD_END;
  static constexpr int HL1 = HL0 + kS * kLd * 2;
  static constexpr int HL2 = HL1 + kS * kLd * 2;
  static constexpr int INFER_END = HL2 + kS * kLd * 2;
  static constexpr int DA = FWD_END;             // BF16 [32][kLd]: dz ping-pong
  static constexpr int DB = DA + kS * kLd * 2;
  static constexpr int DY = DB + kS * kLd * 2;   // BF16 [32][kLdY]
  static constexpr int P = DY + kS * kLdY * 2;   // FP32 [128][kLdP] weight-gradient partials
  static constexpr int PB = P + 128 * kLdP * 4;  // FP32 [128] bias-gradient partials
  static constexpr int RED = PB + 128 * 4;       // FP64 [8] warp loss partials, [8] CTA loss
  static constexpr int TG = RED + 16 * 8;        // FP32 [32][36] targets of the pass
  static constexpr int ROWS = TG + kS * 36 * 4;  // int64 [32] sample rows of the pass
  static constexpr int END = ROWS + kS * 8;
};
static_assert(Wk::END <= 227 * 1024, "shared memory plan exceeds 227 KB");

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t saddr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void ldsm4(uint32_t a, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm4t(uint32_t a, uint32_t (&r)[4]) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
// d += a b: A 16x16 (row), B 16x8 (col), BF16 in, FP32 accumulate
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// the same shared-memory location in CTA `rank` of the cluster (generic pointer)
template <typename T>
__device__ __forceinline__ const T *remote(const T *p, uint32_t rank) {
  return static_cast<const T *>(__cluster_map_shared_rank(const_cast<T *>(p), rank));
}

// GELU(x) = x Phi(x) and its derivative Phi(x) + x phi(x), from one erfc
__device__ __forceinline__ float normal_cdf(float x) { return 0.5f * erfcf(-x * 0.70710678118654752f); }
__device__ __forceinline__ float gelu_deriv_from(float x, float cdf) {
  return cdf + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&v);
}
__device__ __forceinline__ float bf16_val(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }

// Adam (Kingma & Ba 2015, Algorithm 1) on one parameter; c1 = 1/(1 - b1^t),
// c2 = 1/(1 - b2^t).  Returns the new value.
__device__ __forceinline__ float adam_one(float &p, float &m, float &v, float g, float lr, float b1, float b2,
                                          float eps, float c1, float c2) {
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * (g * g);
  p = p - lr * (m * c1) / (sqrtf(v * c2) + eps);
  return p;
}

// Where canonical parameter i sits in the image: byte offset, and whether it
// is kept as BF16 (the 128-wide weights) or as FP32 (biases; W0 as the FP32
// value of its BF16 rounding).
struct Slot {
  int off;
  bool bf16;
};
__device__ __forceinline__ Slot image_slot(int i) {
  if (i < b_off(0)) return {Img::W0 + 4 * i, false};
  if (i < w_off(1)) return {Img::B0 + 4 * (i - b_off(0)), false};
  if (i < b_off(1)) {
    const int q = i - w_off(1);
    return {Img::W1 + 2 * ((q / 128) * kLd + q % 128), true};
  }
  if (i < w_off(2)) return {Img::B1 + 4 * (i - b_off(1)), false};
  if (i < b_off(2)) {
    const int q = i - w_off(2);
    return {Img::W2 + 2 * ((q / 128) * kLd + q % 128), true};
  }
  if (i < w_off(3)) return {Img::B2 + 4 * (i - b_off(2)), false};
  if (i < b_off(3)) {
    const int q = i - w_off(3);
    return {Img::W3 + 2 * ((q / 128) * kLd + q % 128), true};
  }
  return {Img::B3 + 4 * (i - b_off(3)), false};
}

// The value the kernels keep for parameter i (p its FP32 master value).
__device__ __forceinline__ float image_value(int i, float p) { return i < b_off(0) ? bf16_val(p) : p; }

// Write the kernels' copy of canonical parameter i (value p) into an image.
__device__ __forceinline__ void image_put(unsigned char *img, int i, float p) {
  const Slot sl = image_slot(i);
  if (sl.bf16) {
    *reinterpret_cast<__nv_bfloat16 *>(img + sl.off) = __float2bfloat16_rn(p);
  } else {
    *reinterpret_cast<float *>(img + sl.off) = image_value(i, p);
  }
}

// The same, into the shared-memory image of every CTA of the cluster.
__device__ __forceinline__ void image_put_cluster(unsigned char *sm, int i, float p) {
  const Slot sl = image_slot(i);
  if (sl.bf16) {
    const __nv_bfloat16 v = __float2bfloat16_rn(p);
#pragma unroll
    for (int c = 0; c < kCl; ++c)
      *static_cast<__nv_bfloat16 *>(__cluster_map_shared_rank(static_cast<void *>(sm + sl.off), c)) = v;
  } else {
    const float v = image_value(i, p);
#pragma unroll
    for (int c = 0; c < kCl; ++c)
      *static_cast<float *>(__cluster_map_shared_rank(static_cast<void *>(sm + sl.off), c)) = v;
  }
}

// Copy the image from global memory (L2, bypassing L1: other CTAs wrote it).
__device__ __forceinline__ void load_image(unsigned char *sm, const unsigned char *gimg) {
  const uint4 *src = reinterpret_cast<const uint4 *>(gimg);
  uint4 *dst = reinterpret_cast<uint4 *>(sm);
  for (int i = threadIdx.x; i < Img::BYTES / 16; i += blockDim.x) dst[i] = __ldcg(src + i);
}

// ------------------------------------------------------------------ products
// Sample-major product out[32][N] = A[32][K] B, A BF16 [s][k] (row stride lda
// elements).  TRANS_W = false: B(k, n) = W[n][k] (forward); true: B(k, n) =
// W[k][n] (backward).  Warp w: rows 16 (w & 1) .. + 15, columns
// 32 (w >> 1) .. + 31 (4 tiles of 8); acc[nt][0..3] is the m16n8 fragment.
template <bool TRANS_W, bool ZERO = true>
__device__ __forceinline__ void gemm_s(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *W, int ldw, int K,
                                       float (&acc)[4][4]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int s0 = 16 * (w & 1), n0 = 32 * (w >> 1);
  const int q = lane >> 3, r8 = lane & 7;
  if (ZERO) {
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[nt][i] = 0.f;
  }
  const uint32_t a_base = saddr(A + (s0 + r8 + 8 * (q & 1)) * lda + 8 * (q >> 1));
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    ldsm4(a_base + 2 * k0, a);
#pragma unroll
    for (int np = 0; np < 2; ++np) {  // pairs of n tiles
      const int nb = n0 + 16 * np;
      uint32_t b[4];
      if (!TRANS_W) {
        ldsm4(saddr(W + (nb + 8 * (q >> 1) + r8) * ldw + k0 + 8 * (q & 1)), b);
      } else {
        ldsm4t(saddr(W + (k0 + 8 * (q & 1) + r8) * ldw + nb + 8 * (q >> 1)), b);
      }
      mma16816(acc[2 * np], a, b[0], b[1]);
      mma16816(acc[2 * np + 1], a, b[2], b[3]);
    }
  }
}

// sum over the 32 samples of column j of a BF16 [32][ld] buffer (four
// independent partial sums, added in a fixed order)
__device__ __forceinline__ float column_sum(const __nv_bfloat16 *D, int ld, int j) {
  float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int i = 0; i < kS; ++i) a[i & 3] += __bfloat162float(D[i * ld + j]);
  return (a[0] + a[1]) + (a[2] + a[3]);
}

// Element (s, j) of fragment slot (nt, i) of gemm_s: s = s0 + g + 8 (i >> 1),
// j = n0 + 8 nt + 2 t + (i & 1).
__device__ __forceinline__ void frag_pos(int nt, int i, int &s, int &j) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  s = 16 * (w & 1) + (lane >> 2) + 8 * (i >> 1);
  j = 32 * (w >> 1) + 8 * nt + 2 * (lane & 3) + (i & 1);
}

// Weight-gradient product P[j][k] = sum_s D[s][j] H[s][k] over 32 samples: M
// tile mt (rows 16 mt ..), NT tiles of 8 columns from column k0.  D BF16 [s][j]
// (stride ldd), H BF16 [s][k] (stride kLd).
template <int NT>
__device__ __forceinline__ void gemm_w(const __nv_bfloat16 *D, int ldd, const __nv_bfloat16 *H, int mt, int k0,
                                       float *P) {
  const int lane = threadIdx.x & 31;
  const int q = lane >> 3, r8 = lane & 7;
  float acc[NT][4];
#pragma unroll
  for (int nt = 0; nt < NT; ++nt)
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[nt][i] = 0.f;
#pragma unroll
  for (int s0 = 0; s0 < kS; s0 += 16) {
    uint32_t a[4];
    ldsm4t(saddr(D + (s0 + 8 * (q >> 1) + r8) * ldd + 16 * mt + 8 * (q & 1)), a);
#pragma unroll
    for (int np = 0; np < NT / 2; ++np) {
      uint32_t b[4];
      ldsm4t(saddr(H + (s0 + 8 * (q & 1) + r8) * kLd + k0 + 16 * np + 8 * (q >> 1)), b);
      mma16816(acc[2 * np], a, b[0], b[1]);
      mma16816(acc[2 * np + 1], a, b[2], b[3]);
    }
  }
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int col = k0 + 8 * nt + 2 * t;
    *reinterpret_cast<float2 *>(P + (16 * mt + g) * kLdP + col) = make_float2(acc[nt][0], acc[nt][1]);
    *reinterpret_cast<float2 *>(P + (16 * mt + g + 8) * kLdP + col) = make_float2(acc[nt][2], acc[nt][3]);
  }
}

// ------------------------------------------------------------------ forward of 32 samples
// X (FP32 [32][4]) in shared memory -> H0, H1, H2 (BF16) and Y (FP32
// [32][kOutP], 35 used).  With KEEP_G the GELU derivatives of the three hidden
// layers stay in G[l] in the fragment layout of gemm_s.  SPLIT (inference):
// each activation h is kept as hi = bf16(h) in H and lo = bf16(h - hi) in
// HL, and every product takes both terms, so the activations enter the
// tensor cores with ~16 significant bits and the outputs are a smooth
// function of the inputs (training rounds them to one BF16 term).
template <bool KEEP_G, bool SPLIT = false>
__device__ __forceinline__ void forward32(unsigned char *sm, float (&G)[3][4][4]) {
  const float *X = reinterpret_cast<const float *>(sm + Wk::X);
  const float *W0 = reinterpret_cast<const float *>(sm + Img::W0);
  __nv_bfloat16 *H[3] = {reinterpret_cast<__nv_bfloat16 *>(sm + Wk::H0),
                         reinterpret_cast<__nv_bfloat16 *>(sm + Wk::H1),
                         reinterpret_cast<__nv_bfloat16 *>(sm + Wk::H2)};
  __nv_bfloat16 *HL[3] = {reinterpret_cast<__nv_bfloat16 *>(sm + Wk::HL0),
                          reinterpret_cast<__nv_bfloat16 *>(sm + Wk::HL1),
                          reinterpret_cast<__nv_bfloat16 *>(sm + Wk::HL2)};
  const float *B[3] = {reinterpret_cast<const float *>(sm + Img::B0), reinterpret_cast<const float *>(sm + Img::B1),
                       reinterpret_cast<const float *>(sm + Img::B2)};
  const __nv_bfloat16 *Wl[3] = {nullptr, reinterpret_cast<const __nv_bfloat16 *>(sm + Img::W1),
                                reinterpret_cast<const __nv_bfloat16 *>(sm + Img::W2)};
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    float acc[4][4];
    if (l == 0) {  // 4 inputs: FP32 cores, FP32 inputs
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          int s, j;
          frag_pos(nt, i, s, j);
          const float4 wv = *reinterpret_cast<const float4 *>(W0 + 4 * j);
          const float4 xv = *reinterpret_cast<const float4 *>(X + 4 * s);
          acc[nt][i] = fmaf(wv.w, xv.w, fmaf(wv.z, xv.z, fmaf(wv.y, xv.y, wv.x * xv.x)));
        }
    } else {
      gemm_s<false>(H[l - 1], kLd, Wl[l], kLd, 128, acc);
      if (SPLIT) gemm_s<false, false>(HL[l - 1], kLd, Wl[l], kLd, 128, acc);
    }
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int s, j;
        frag_pos(nt, 2 * h, s, j);
        const float z0 = acc[nt][2 * h] + B[l][j], z1 = acc[nt][2 * h + 1] + B[l][j + 1];
        const float p0 = normal_cdf(z0), p1 = normal_cdf(z1);
        if (KEEP_G) {
          G[l][nt][2 * h] = gelu_deriv_from(z0, p0);
          G[l][nt][2 * h + 1] = gelu_deriv_from(z1, p1);
        }
        const float h0 = z0 * p0, h1 = z1 * p1;
        *reinterpret_cast<uint32_t *>(H[l] + s * kLd + j) = pack_bf16(h0, h1);
        if (SPLIT)
          *reinterpret_cast<uint32_t *>(HL[l] + s * kLd + j) = pack_bf16(h0 - bf16_val(h0), h1 - bf16_val(h1));
      }
    __syncthreads();
  }
  // output layer: 5 column tiles (40 columns, 35 real), both row tiles, warps 0..4
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (w < 5) {
    const __nv_bfloat16 *W3 = reinterpret_cast<const __nv_bfloat16 *>(sm + Img::W3);
    const int q = lane >> 3, r8 = lane & 7;
    float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
    for (int k0 = 0; k0 < 128; k0 += 16) {
      uint32_t b[4];  // tiles w and w + 1 (rows up to 47 exist: zero padding)
      ldsm4(saddr(W3 + (8 * w + 8 * (q >> 1) + r8) * kLd + k0 + 8 * (q & 1)), b);
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        uint32_t a[4];
        ldsm4(saddr(H[2] + (16 * mt + r8 + 8 * (q & 1)) * kLd + k0 + 8 * (q >> 1)), a);
        mma16816(acc[mt], a, b[0], b[1]);
        if (SPLIT) {
          ldsm4(saddr(HL[2] + (16 * mt + r8 + 8 * (q & 1)) * kLd + k0 + 8 * (q >> 1)), a);
          mma16816(acc[mt], a, b[0], b[1]);
        }
      }
    }
    float *Y = reinterpret_cast<float *>(sm + Wk::Y);
    const float *B3 = reinterpret_cast<const float *>(sm + Img::B3);
    const int g = lane >> 2, t = lane & 3, j = 8 * w + 2 * t;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      Y[(16 * mt + g) * kOutP + j] = acc[mt][0] + B3[j];
      Y[(16 * mt + g) * kOutP + j + 1] = acc[mt][1] + B3[j + 1];
      Y[(16 * mt + g + 8) * kOutP + j] = acc[mt][2] + B3[j];
      Y[(16 * mt + g + 8) * kOutP + j + 1] = acc[mt][3] + B3[j + 1];
    }
  }
  __syncthreads();
}

// Load the inputs of samples [i0, i0 + cnt) (cnt <= 32; rows or base + i) as
// X; rows past cnt are zero.  Returns nothing; ends with a barrier.
__device__ __forceinline__ void load_x(unsigned char *sm, const float *x, const int32_t *rows, int64_t base,
                                       int64_t i0, int cnt) {
  float *X = reinterpret_cast<float *>(sm + Wk::X);
  if (threadIdx.x < kS * 4) {
    const int s = threadIdx.x >> 2, k = threadIdx.x & 3;
    float v = 0.f;
    if (s < cnt) {
      const int64_t i = i0 + s;
      const int64_t row = rows ? rows[base + i] : base + i;
      v = x[row * 4 + k];
    }
    X[threadIdx.x] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Training pass of samples [i0, i0 + cnt): their rows, their inputs X (ready
// on return), and their targets, copied asynchronously into TG (complete
// after cp_async_wait_all and a barrier).
__device__ __forceinline__ void load_pass(unsigned char *sm, const MlpRun &R, int64_t i0, int cnt) {
  int64_t *rows = reinterpret_cast<int64_t *>(sm + Wk::ROWS);
  if (threadIdx.x < kS) {
    const int64_t i = i0 + threadIdx.x;
    rows[threadIdx.x] = threadIdx.x < cnt ? (R.rows ? R.rows[R.base + i] : R.base + i) : 0;
  }
  __syncthreads();
  float *X = reinterpret_cast<float *>(sm + Wk::X);
  if (threadIdx.x < kS * 4) {
    const int s = threadIdx.x >> 2, k = threadIdx.x & 3;
    X[threadIdx.x] = s < cnt ? R.x[rows[s] * 4 + k] : 0.f;
  }
  float *T = reinterpret_cast<float *>(sm + Wk::TG);
  for (int e = threadIdx.x; e < cnt * kMlpOut; e += blockDim.x) {
    const int s = e / kMlpOut, j = e % kMlpOut;
    cp_async4(T + s * 36 + j, R.t + rows[s] * kMlpOut + j);
  }
  cp_async_commit();
  __syncthreads();
}

// ------------------------------------------------------------------ inference
__global__ void __launch_bounds__(kThr, 1) k_mlp_forward(const unsigned char *__restrict__ gimg,
                                                          const float *__restrict__ x, int64_t n, float *y) {
  extern __shared__ __align__(16) unsigned char sm[];
  load_image(sm, gimg);
  const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kS;
  const int cnt = static_cast<int>(n - i0 < kS ? n - i0 : kS);
  load_x(sm, x, nullptr, 0, i0, cnt);  // (its barrier also covers the image)
  float G[3][4][4];
  forward32<false, true>(sm, G);
  const float *Y = reinterpret_cast<const float *>(sm + Wk::Y);
  for (int e = threadIdx.x; e < cnt * kMlpOut; e += blockDim.x) {
    const int s = e / kMlpOut, j = e % kMlpOut;
    y[(i0 + s) * kMlpOut + j] = Y[s * kOutP + j];
  }
}

// ------------------------------------------------------------------ training cluster
// Four consecutive parameters i .. i + 3 (i a multiple of 4, inside one
// weight row or among the biases) into every CTA's shared-memory image.
__device__ __forceinline__ void image_put4_cluster(unsigned char *sm, int i, float4 p) {
  const Slot sl = image_slot(i);
  if (sl.bf16) {
    uint2 v;
    v.x = pack_bf16(p.x, p.y);
    v.y = pack_bf16(p.z, p.w);
#pragma unroll
    for (int c = 0; c < kCl; ++c)
      *static_cast<uint2 *>(__cluster_map_shared_rank(static_cast<void *>(sm + sl.off), c)) = v;
  } else {
    const float4 v = make_float4(image_value(i, p.x), image_value(i, p.y), image_value(i, p.z), image_value(i, p.w));
#pragma unroll
    for (int c = 0; c < kCl; ++c)
      *static_cast<float4 *>(__cluster_map_shared_rank(static_cast<void *>(sm + sl.off), c)) = v;
  }
}

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 add4(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// Owned slice of layer l's gradient (weights then bias, canonical order), in
// groups of four parameters: groups [rank G / 8, (rank + 1) G / 8) of the
// layer's G = ceil(L / 4), L = dim(l+1) (dim(l) + 1).  Sums the 8 CTAs'
// partials (ranks in order).  adam: apply the Adam step to the slice at once
// (the step has one pass) and write the new weights into every CTA's
// shared-memory image; otherwise store (or add) the sums into grad.
struct AdamArgs {
  float lr, b1, b2, eps, c1, c2;
};
__device__ __forceinline__ void reduce_owned(unsigned char *sm, int l, uint32_t rank, const MlpRun &R, bool add,
                                             bool adam, const AdamArgs &A) {
  const int ni = dim(l), no = dim(l + 1), L = no * (ni + 1), G = (L + 3) / 4;
  const int g0 = static_cast<int>(rank) * G / kCl, g1 = (static_cast<int>(rank) + 1) * G / kCl;
  const float *P = reinterpret_cast<const float *>(sm + Wk::P);
  const float *PB = reinterpret_cast<const float *>(sm + Wk::PB);
  float *__restrict__ master = R.master;
  float *__restrict__ mm = R.m;
  float *__restrict__ vv = R.v;
  float *__restrict__ grad = R.grad;
  for (int gi = g0 + threadIdx.x; gi < g1; gi += blockDim.x) {
    const int q = 4 * gi, i = w_off(l) + q;
    const bool full = q + 4 <= L;  // only the last group of a layer may be short
    float4 p = make_float4(0.f, 0.f, 0.f, 0.f), m = p, v = p;
    if (adam && full) {  // issued before the partials are read
      p = ld4(master + i);
      m = ld4(mm + i);
      v = ld4(vv + i);
    }
    // (rows of P and the bias partials both hold the whole group, in bounds)
    const float *a = q < no * ni ? P + (q / ni) * kLdP + q % ni : PB + (q - no * ni);
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int c = 0; c < kCl; ++c) s = add4(s, ld4(remote(a, c)));
    if (full) {
      if (adam) {
        adam_one(p.x, m.x, v.x, s.x, A.lr, A.b1, A.b2, A.eps, A.c1, A.c2);
        adam_one(p.y, m.y, v.y, s.y, A.lr, A.b1, A.b2, A.eps, A.c1, A.c2);
        adam_one(p.z, m.z, v.z, s.z, A.lr, A.b1, A.b2, A.eps, A.c1, A.c2);
        adam_one(p.w, m.w, v.w, s.w, A.lr, A.b1, A.b2, A.eps, A.c1, A.c2);
        st4(master + i, p);
        st4(mm + i, m);
        st4(vv + i, v);
        image_put4_cluster(sm, i, p);
      } else {
        st4(grad + i, add ? add4(ld4(grad + i), s) : s);
      }
    } else {
      const float sv[4] = {s.x, s.y, s.z, s.w};
      for (int e = 0; e < L - q; ++e) {
        if (adam) {
          float pe = master[i + e], me = mm[i + e], ve = vv[i + e];
          adam_one(pe, me, ve, sv[e], A.lr, A.b1, A.b2, A.eps, A.c1, A.c2);
          master[i + e] = pe;
          mm[i + e] = me;
          vv[i + e] = ve;
          image_put_cluster(sm, i + e, pe);
        } else {
          grad[i + e] = add ? grad[i + e] + sv[e] : sv[e];
        }
      }
    }
  }
}

// Samples of chunk `c` of step `st` for this CTA: [i0, i0 + cnt) of the launch.
__device__ __forceinline__ void chunk_range(const MlpRun &R, int st, int c, uint32_t rank, int64_t &i0, int &cnt,
                                            int &step_n) {
  const int64_t s0 = static_cast<int64_t>(st) * R.batch;
  const int64_t s1 = s0 + R.batch < R.n ? s0 + R.batch : R.n;
  step_n = static_cast<int>(s1 - s0);
  i0 = s0 + static_cast<int64_t>(c) * kMlpChunk + static_cast<int64_t>(rank) * kS;
  const int64_t e = i0 + kS < s1 ? i0 + kS : s1;
  cnt = e > i0 ? static_cast<int>(e - i0) : 0;
}

__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kThr, 1) k_mlp_train(MlpRun R) {
  extern __shared__ __align__(16) unsigned char sm[];
  const uint32_t rank = cluster_rank();
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const unsigned char *gimg = static_cast<const unsigned char *>(R.img);
  __nv_bfloat16 *H0 = reinterpret_cast<__nv_bfloat16 *>(sm + Wk::H0);
  __nv_bfloat16 *H1 = reinterpret_cast<__nv_bfloat16 *>(sm + Wk::H1);
  __nv_bfloat16 *H2 = reinterpret_cast<__nv_bfloat16 *>(sm + Wk::H2);
  __nv_bfloat16 *DA = reinterpret_cast<__nv_bfloat16 *>(sm + Wk::DA);
  __nv_bfloat16 *DB = reinterpret_cast<__nv_bfloat16 *>(sm + Wk::DB);
  __nv_bfloat16 *DY = reinterpret_cast<__nv_bfloat16 *>(sm + Wk::DY);
  const __nv_bfloat16 *W1 = reinterpret_cast<const __nv_bfloat16 *>(sm + Img::W1);
  const __nv_bfloat16 *W2 = reinterpret_cast<const __nv_bfloat16 *>(sm + Img::W2);
  const __nv_bfloat16 *W3 = reinterpret_cast<const __nv_bfloat16 *>(sm + Img::W3);
  float *P = reinterpret_cast<float *>(sm + Wk::P);
  float *PB = reinterpret_cast<float *>(sm + Wk::PB);
  double *RED = reinterpret_cast<double *>(sm + Wk::RED);
  const float *X = reinterpret_cast<const float *>(sm + Wk::X);
  const float *Y = reinterpret_cast<const float *>(sm + Wk::Y);

  load_image(sm, gimg);
  __syncthreads();

  for (int st = 0; st < R.steps; ++st) {
    int64_t i0;
    int cnt, step_n;
    chunk_range(R, st, 0, rank, i0, cnt, step_n);
    const int chunks = (step_n + kMlpChunk - 1) / kMlpChunk;
    const double inv = R.inv_count > 0.0 ? R.inv_count : 1.0 / (static_cast<double>(step_n) * kMlpOut);
    // a one-pass training step updates each layer right after its gradient is
    // summed (no CTA uses that layer's weights again in this step)
    const bool fuse = R.train && chunks == 1;
    AdamArgs A{};
    if (R.train) {
      const int64_t t = R.t0 + 1 + st;
      A = AdamArgs{R.lr, R.b1, R.b2, R.eps,
                   static_cast<float>(1.0 / (1.0 - pow(static_cast<double>(R.b1), static_cast<double>(t)))),
                   static_cast<float>(1.0 / (1.0 - pow(static_cast<double>(R.b2), static_cast<double>(t))))};
    }
    double step_loss = 0.0;  // CTA 0
    for (int c = 0; c < chunks; ++c) {
      chunk_range(R, st, c, rank, i0, cnt, step_n);
      const bool add = R.accumulate || c > 0;
      load_pass(sm, R, i0, cnt);
      float G[3][4][4];
      forward32<true>(sm, G);
      cp_async_wait_all();  // the targets (copied during the forward pass)
      __syncthreads();

      // ---- loss and output gradient dy (BF16), zero past the valid samples and outputs
      const float *T = reinterpret_cast<const float *>(sm + Wk::TG);
      float lf = 0.f;  // this thread's few squared residuals
      const float two_inv = static_cast<float>(2.0 * inv);
      for (int e = tid; e < kS * 48; e += kThr) {
        const int s = e / 48, j = e % 48;
        float d = 0.f;
        if (s < cnt && j < kMlpOut) {
          const float r = Y[s * kOutP + j] - T[s * 36 + j];
          lf = fmaf(r, r, lf);
          d = two_inv * r;
        }
        DY[s * kLdY + j] = __float2bfloat16_rn(d);
      }
      double lsum = static_cast<double>(lf) * inv;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
      if (lane == 0) RED[w] = lsum;
      __syncthreads();
      if (tid == 0) {
        double s = 0.0;
        for (int i = 0; i < kThr / 32; ++i) s += RED[i];
        RED[8] = s;  // this CTA's loss of the chunk
      }

      // ---- layer 3: dW3 = dy^T h2 (48 x 128 tiles on warps 0..5), db3; dh2 = dy W3
      if (w < 6) gemm_w<8>(DY, kLdY, H2, w % 3, 64 * (w / 3), P);
      if (tid < kMlpOut) PB[tid] = column_sum(DY, kLdY, tid);
      {
        float acc[4][4];
        gemm_s<true>(DY, kLdY, W3, kLd, 48, acc);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            int s, j;
            frag_pos(nt, 2 * h, s, j);
            *reinterpret_cast<uint32_t *>(DA + s * kLd + j) =
                pack_bf16(acc[nt][2 * h] * G[2][nt][2 * h], acc[nt][2 * h + 1] * G[2][nt][2 * h + 1]);
          }
      }
      cluster_sync();  // partials of layer 3 complete everywhere
      if (rank == 0 && tid == 0)
        for (int cc = 0; cc < kCl; ++cc) step_loss += *remote(RED + 8, cc);
      reduce_owned(sm, 3, rank, R, add, fuse, A);
      cluster_sync();  // partials read

      // ---- layers 2 and 1: dW = dz^T h, db; dh = dz W, dz' = dh * GELU'(z)
#pragma unroll
      for (int l = 2; l >= 1; --l) {
        const __nv_bfloat16 *D = (l == 2) ? DA : DB;
        __nv_bfloat16 *Dn = (l == 2) ? DB : DA;
        const __nv_bfloat16 *Hin = (l == 2) ? H1 : H0;
        const __nv_bfloat16 *Wm = (l == 2) ? W2 : W1;
        gemm_w<8>(D, kLd, Hin, w, 0, P);  // two halves of 8 column tiles keep registers for G
        gemm_w<8>(D, kLd, Hin, w, 64, P);
        if (tid < 128) PB[tid] = column_sum(D, kLd, tid);
        float acc[4][4];
        gemm_s<true>(D, kLd, Wm, kLd, 128, acc);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            int s, j;
            frag_pos(nt, 2 * h, s, j);
            *reinterpret_cast<uint32_t *>(Dn + s * kLd + j) = pack_bf16(acc[nt][2 * h] * G[l - 1][nt][2 * h],
                                                                       acc[nt][2 * h + 1] * G[l - 1][nt][2 * h + 1]);
          }
        cluster_sync();
        reduce_owned(sm, l, rank, R, add, fuse, A);
        cluster_sync();
      }

      // ---- layer 0 (FP32 inputs): dW0 = dz0^T x, db0 (dz0 in DA)
      for (int e = tid; e < 128 * 4; e += kThr) {
        const int j = e >> 2, k = e & 3;
        float a[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int i = 0; i < kS; ++i) a[i & 3] = fmaf(__bfloat162float(DA[i * kLd + j]), X[i * 4 + k], a[i & 3]);
        P[j * kLdP + k] = (a[0] + a[1]) + (a[2] + a[3]);
      }
      if (tid < 128) PB[tid] = column_sum(DA, kLd, tid);
      cluster_sync();
      reduce_owned(sm, 0, rank, R, add, fuse, A);
      cluster_sync();  // partials read (the next chunk rewrites them)
    }
    if (rank == 0 && tid == 0 && R.loss_out) R.loss_out[st] = step_loss;
    if (R.train && !fuse) {
      // several passes: Adam on this CTA's eighth of every layer from the
      // summed gradient; the new weights go to every CTA's image
      for (int l = 0; l < 4; ++l) {  // the groups reduce_owned wrote
        const int L = dim(l + 1) * (dim(l) + 1), G = (L + 3) / 4;
        const int g0 = static_cast<int>(rank) * G / kCl, g1 = (static_cast<int>(rank) + 1) * G / kCl;
        for (int q = 4 * g0 + tid; q < min(4 * g1, L); q += kThr) {
          const int i = w_off(l) + q;
          float p = R.master[i], m = R.m[i], v = R.v[i];
          adam_one(p, m, v, R.grad[i], A.lr, A.b1, A.b2, A.eps, A.c1, A.c2);
          R.master[i] = p;
          R.m[i] = m;
          R.v[i] = v;
          image_put_cluster(sm, i, p);
        }
      }
      cluster_sync();  // every CTA's image is complete before the next forward
    }
  }
  cluster_sync();  // no CTA leaves while others may read its shared memory
}

// ------------------------------------------------------------------ small kernels
__global__ void k_mlp_pack(const float *__restrict__ master, unsigned char *img, __nv_bfloat16 *wbf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float p = master[i];
  image_put(img, i, p);
  if (wbf) wbf[i] = __float2bfloat16_rn(p);
}

__global__ void k_mlp_adam(float *master, float *m, float *v, const float *__restrict__ g, unsigned char *img,
                           float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  float p = master[i], mi = m[i], vi = v[i];
  adam_one(p, mi, vi, g[i], lr, b1, b2, eps, c1, c2);
  master[i] = p;
  m[i] = mi;
  v[i] = vi;
  image_put(img, i, p);
}

}  // namespace

// ---------------------------------------------------------------- launchers
size_t mlp_image_bytes() { return Img::BYTES; }

cudaError_t mlp_pack(const float *master, void *img, void *wbf, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(img, 0, Img::BYTES, st);  // padding rows and columns stay zero
  if (e != cudaSuccess) return e;
  k_mlp_pack<<<(kMlpParams + 255) / 256, 256, 0, st>>>(master, static_cast<unsigned char *>(img),
                                                        static_cast<__nv_bfloat16 *>(wbf));
  return cudaGetLastError();
}

cudaError_t mlp_forward(const void *img, const float *x, int64_t n, float *y, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int smem = Wk::INFER_END;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int64_t grid = (n + kS - 1) / kS;
  k_mlp_forward<<<static_cast<unsigned>(grid), kThr, smem, st>>>(static_cast<const unsigned char *>(img), x, n, y);
  return cudaGetLastError();
}

cudaError_t mlp_cluster_run(const MlpRun &R, cudaStream_t st) {
  if (R.steps == 0) return cudaSuccess;
  const int smem = Wk::END;
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  k_mlp_train<<<kCl, kThr, smem, st>>>(R);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float *master, float *m, float *v, const float *grad, void *img, float lr, float b1, float b2,
                     float eps, int64_t step, cudaStream_t st) {
  const double c1 = 1.0 / (1.0 - pow(static_cast<double>(b1), static_cast<double>(step)));
  const double c2 = 1.0 / (1.0 - pow(static_cast<double>(b2), static_cast<double>(step)));
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(master, m, v, grad, static_cast<unsigned char *>(img), lr,
                                                        b1, b2, eps, static_cast<float>(c1),
                                                        static_cast<float>(c2));
  return cudaGetLastError();
}

}  // namespace mk
