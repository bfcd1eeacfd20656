// Surrogate MLP kernels: 4 -> 128 -> 128 -> 128 -> 35, GELU hidden units.
//
// Weights are used in BF16 (a copy refreshed from the FP32 master after each
// Adam step); biases, activations and every accumulation are FP32.  Layout of
// the parameter vector: W0 [128x4], b0, W1 [128x128], b1, W2 [128x128], b2,
// W3 [35x128], b3, each W row-major [out][in].
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mk_mlp.h"

namespace mk {

__host__ __device__ constexpr int mlp_dim(int l) { return l == 0 ? 4 : (l == 4 ? 35 : 128); }
constexpr int kTile = 32;  // samples per CTA
constexpr int kThreads = 128;

struct MlpOffsets {
  int w[4], b[4];
};

__host__ __device__ inline MlpOffsets mlp_offsets() {
  MlpOffsets o;
  int p = 0;
  for (int l = 0; l < 4; ++l) {
    o.w[l] = p;
    p += mlp_dim(l + 1) * mlp_dim(l);
    o.b[l] = p;
    p += mlp_dim(l + 1);
  }
  return o;
}

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * erfcf(-x * 0.70710678118654752f); }

__device__ __forceinline__ float gelu_deriv(float x) {
  return 0.5f * erfcf(-x * 0.70710678118654752f) + x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

// Forward over a tile of kTile samples.  rows[i] (or i) selects the sample.
// When acts is set, stores z_l and h_l of the three hidden layers
// (acts + l * 2 * n * 128: z, then h) and the outputs y for the backward pass.
__global__ void __launch_bounds__(kThreads) k_mlp_fwd(const __nv_bfloat16 *__restrict__ wbf,
                                                      const float *__restrict__ master, const float *__restrict__ x,
                                                      const int32_t *__restrict__ rows, int64_t n, float *y,
                                                      float *acts) {
  __shared__ float in[kTile][128];         // inputs of the current layer, then its outputs
  __shared__ __nv_bfloat16 wt[128][128];  // transposed weights of the current layer: wt[k][j]
  const MlpOffsets O = mlp_offsets();
  const int64_t s0 = static_cast<int64_t>(blockIdx.x) * kTile;
  const int j = threadIdx.x;
  for (int i = threadIdx.x; i < kTile * 4; i += kThreads) {
    const int s = i / 4, k = i % 4;
    const int64_t g = s0 + s;
    float v = 0.f;
    if (g < n) v = x[(rows ? rows[g] : g) * 4 + k];
    in[s][k] = v;
  }
  for (int l = 0; l < 4; ++l) {
    const int ni = mlp_dim(l), no = mlp_dim(l + 1);
    __syncthreads();
    for (int i = threadIdx.x; i < ni * no; i += kThreads) {
      const int jj = i / ni, kk = i % ni;
      wt[kk][jj] = wbf[O.w[l] + i];
    }
    __syncthreads();
    float acc[kTile];
    if (j < no) {
      const float b = master[O.b[l] + j];
#pragma unroll
      for (int s = 0; s < kTile; ++s) acc[s] = b;
      for (int k = 0; k < ni; ++k) {
        const float w = __bfloat162float(wt[k][j]);
#pragma unroll
        for (int s = 0; s < kTile; ++s) acc[s] = fmaf(in[s][k], w, acc[s]);
      }
    }
    __syncthreads();  // every thread has read `in`
    if (j < no) {
#pragma unroll
      for (int s = 0; s < kTile; ++s) {
        const int64_t g = s0 + s;
        const float h = (l < 3) ? gelu(acc[s]) : acc[s];
        in[s][j] = h;
        if (g < n) {
          if (l < 3) {
            if (acts) {
              acts[(static_cast<int64_t>(l) * 2 * n + g) * 128 + j] = acc[s];
              acts[(static_cast<int64_t>(l) * 2 * n + n + g) * 128 + j] = h;
            }
          } else {
            y[g * 35 + j] = h;
          }
        }
      }
    }
  }
}

// dy = 2 (y - t) / (n_total * 35) and the per-CTA loss partial (FP64).
__global__ void k_mlp_loss(const float *__restrict__ y, const float *__restrict__ t,
                           const int32_t *__restrict__ rows, int64_t n, double inv_count, float *dy,
                           double *loss_part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n * 35;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t s = i / 35, o = i % 35;
    const float r = y[i] - t[(rows ? rows[s] : s) * 35 + o];
    dy[i] = static_cast<float>(2.0 * inv_count) * r;
    acc += static_cast<double>(r) * r * inv_count;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// Backward through the hidden layers for a tile: dz_l = (W_{l+1}^T dz_{l+1}) * GELU'(z_l),
// l = 2, 1, 0, stored in dzs + l * n * 128.
__global__ void __launch_bounds__(kThreads) k_mlp_bwd(const __nv_bfloat16 *__restrict__ wbf,
                                                      const float *__restrict__ acts, const float *__restrict__ dy,
                                                      int64_t n, float *dzs) {
  __shared__ float din[kTile][128];      // dz of layer l + 1, then of layer l
  __shared__ __nv_bfloat16 w[128][128];  // W_{l+1} as [out j][in k]
  const MlpOffsets O = mlp_offsets();
  const int64_t s0 = static_cast<int64_t>(blockIdx.x) * kTile;
  const int k = threadIdx.x;
  for (int i = threadIdx.x; i < kTile * 35; i += kThreads) {
    const int s = i / 35, o = i % 35;
    const int64_t g = s0 + s;
    din[s][o] = g < n ? dy[g * 35 + o] : 0.f;
  }
  for (int l = 2; l >= 0; --l) {
    const int no = mlp_dim(l + 2);  // outputs of layer l + 1
    __syncthreads();
    for (int i = threadIdx.x; i < no * 128; i += kThreads) w[i / 128][i % 128] = wbf[O.w[l + 1] + i];
    __syncthreads();
    float acc[kTile];
#pragma unroll
    for (int s = 0; s < kTile; ++s) acc[s] = 0.f;
    for (int jj = 0; jj < no; ++jj) {
      const float wv = __bfloat162float(w[jj][k]);
#pragma unroll
      for (int s = 0; s < kTile; ++s) acc[s] = fmaf(din[s][jj], wv, acc[s]);
    }
    __syncthreads();  // every thread has read `din`
#pragma unroll
    for (int s = 0; s < kTile; ++s) {
      const int64_t g = s0 + s;
      float d = 0.f;
      if (g < n) {
        const float z = acts[(static_cast<int64_t>(l) * 2 * n + g) * 128 + k];
        d = acc[s] * gelu_deriv(z);
        dzs[(static_cast<int64_t>(l) * n + g) * 128 + k] = d;
      }
      din[s][k] = d;
    }
  }
}

// Weight and bias gradients of layer l: dW[j][k] = sum_s d[s][j] in[s][k],
// db[j] = sum_s d[s][j]; one thread per entry, samples summed in order.
__global__ void k_mlp_wgrad(const float *__restrict__ d, int64_t ldd, const float *__restrict__ in, int64_t ldi,
                            const float *__restrict__ x, const int32_t *__restrict__ rows, int no, int ni,
                            int64_t n, float *gw, float *gb) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < no * ni) {
    const int j = idx / ni, k = idx % ni;
    float acc = 0.f;
    for (int64_t s = 0; s < n; ++s) {
      const float a = in ? in[s * ldi + k] : x[(rows ? rows[s] : s) * 4 + k];
      acc = fmaf(d[s * ldd + j], a, acc);
    }
    gw[idx] = acc;
  } else if (idx < no * ni + no) {
    const int j = idx - no * ni;
    float acc = 0.f;
    for (int64_t s = 0; s < n; ++s) acc += d[s * ldd + j];
    gb[j] = acc;
  }
}

// Adam on the FP32 master, then the BF16 copy.
__global__ void k_mlp_adam(float *master, __nv_bfloat16 *wbf, const float *__restrict__ g, float *m, float *v,
                           int np, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
  const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
  m[i] = mi;
  v[i] = vi;
  const float p = master[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  master[i] = p;
  wbf[i] = __float2bfloat16_rn(p);
}

__global__ void k_mlp_to_bf16(const float *master, __nv_bfloat16 *wbf, int np) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) wbf[i] = __float2bfloat16_rn(master[i]);
}

// ---------------------------------------------------------------- launchers
cudaError_t mlp_to_bf16(const float *master, void *wbf, cudaStream_t st) {
  k_mlp_to_bf16<<<(kMlpParams + 255) / 256, 256, 0, st>>>(master, static_cast<__nv_bfloat16 *>(wbf), kMlpParams);
  return cudaGetLastError();
}

cudaError_t mlp_forward(const void *wbf, const float *master, const float *x, const int32_t *rows, int64_t n,
                        float *y, float *acts, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int64_t grid = (n + kTile - 1) / kTile;
  k_mlp_fwd<<<static_cast<unsigned>(grid), kThreads, 0, st>>>(static_cast<const __nv_bfloat16 *>(wbf), master, x,
                                                             rows, n, y, acts);
  return cudaGetLastError();
}

// One gradient evaluation on n samples: forward with activations, loss and
// dy, backward, weight gradients into grad (kMlpParams floats).  loss_part
// holds kLossParts doubles (the caller sums them).
cudaError_t mlp_gradient(const void *wbf, const float *master, const float *x, const float *t,
                         const int32_t *rows, int64_t n, double inv_count, float *y, float *dy, float *acts,
                         float *dzs, float *grad, double *loss_part, cudaStream_t st) {
  cudaError_t e = mlp_forward(wbf, master, x, rows, n, y, acts, st);
  if (e != cudaSuccess) return e;
  k_mlp_loss<<<kLossParts, 256, 0, st>>>(y, t, rows, n, inv_count, dy, loss_part);
  const int64_t grid = (n + kTile - 1) / kTile;
  k_mlp_bwd<<<static_cast<unsigned>(grid), kThreads, 0, st>>>(static_cast<const __nv_bfloat16 *>(wbf), acts, dy,
                                                              n, dzs);
  const MlpOffsets O = mlp_offsets();
  for (int l = 0; l < 4; ++l) {
    const int no = mlp_dim(l + 1), ni = mlp_dim(l);
    const float *d = (l == 3) ? dy : dzs + static_cast<int64_t>(l) * n * 128;
    const int64_t ldd = (l == 3) ? 35 : 128;
    const float *in = (l == 0) ? nullptr : acts + (static_cast<int64_t>(l - 1) * 2 * n + n) * 128;
    const int cnt = no * ni + no;
    k_mlp_wgrad<<<(cnt + 127) / 128, 128, 0, st>>>(d, ldd, in, 128, x, rows, no, ni, n, grad + O.w[l],
                                                    grad + O.b[l]);
  }
  return cudaGetLastError();
}

cudaError_t mlp_adam(float *master, void *wbf, const float *grad, float *m, float *v, float lr, float b1, float b2,
                     float eps, int64_t step, cudaStream_t st) {
  const double c1 = 1.0 / (1.0 - pow(static_cast<double>(b1), static_cast<double>(step)));
  const double c2 = 1.0 / (1.0 - pow(static_cast<double>(b2), static_cast<double>(step)));
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(master, static_cast<__nv_bfloat16 *>(wbf), grad, m, v,
                                                        kMlpParams, lr, b1, b2, eps, static_cast<float>(c1),
                                                        static_cast<float>(c2));
  return cudaGetLastError();
}

}  // namespace mk
