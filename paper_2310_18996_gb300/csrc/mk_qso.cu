// Quasars from lognormal quasar-density fields (Sec. 2.2, App. A): the
// Hankel-transform pair that turns the matter spectrum into the spectrum of
// the Gaussian field delta_q, and the voxel draw from three delta_q boxes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/mockskewer.h"
#include "mk_device.cuh"
#include "mk_host.h"
#include "mk_trace.h"

using namespace mk;

namespace {

int qfail(mk_ctx *ctx, int code, const char *msg) { return mkhost::ctx_fail(ctx, code, msg); }

#define CKQ(ctx, call)                                                                  \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) {                                                            \
      char b_[256];                                                                     \
      snprintf(b_, sizeof(b_), "%s: %s", #call, cudaGetErrorString(e_));                 \
      return qfail(ctx, MK_ECUDA, b_);                                                  \
    }                                                                                   \
  } while (0)

double sinc_j0(double x) {
  if (std::fabs(x) < 1e-4) return 1.0 - x * x / 6.0 + x * x * x * x / 120.0;
  return std::sin(x) / x;
}

// xi(r) of a tabulated P(k) (trapezoid rule on k_i = i dk)
double xi_at(const double *pk, int n, double dk, double r) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) {
    const double k = i * dk, w = (i == 0 || i == n - 1) ? 0.5 : 1.0;
    s += w * pk[i] * k * k * sinc_j0(k * r);
  }
  return s * dk / (2.0 * M_PI * M_PI);
}

// -------------------------------------------------------------------------- draw kernels
struct DrawParams {
  const float *box[3];
  int32_t stride;
  int32_t n, lgn;  // n = 2^lgn
  float cell;
  float origin[3];
  const float4 *tab;  // per r node: (a_1, a_2, a_3, nbar cell^3 / E[p]), (w_1, w_2, w_3, 0)
  int32_t n_tab;
  float r0, inv_dr;
  uint32_t key0, key1;
  int32_t *count32;       // per sub-range (count pass)
  const int64_t *offset;  // per sub-range (write pass)
  mk_qso *out;
  int64_t capacity;
  double origin_d[3], cell_d;
};

// Accept decision of voxel v (and its Philox words for the position).
__device__ __forceinline__ bool voxel_accept(const DrawParams &P, int64_t v, u32x4 &w, int &x, int &y, int &z) {
  const int mask = P.n - 1;
  x = static_cast<int>(v) & mask;
  y = static_cast<int>(v >> P.lgn) & mask;
  z = static_cast<int>(v >> (2 * P.lgn));
  const float cx = P.origin[0] + (x + 0.5f) * P.cell, cy = P.origin[1] + (y + 0.5f) * P.cell,
              cz = P.origin[2] + (z + 0.5f) * P.cell;
  const float r = sqrtf(cx * cx + cy * cy + cz * cz);
  float s = (r - P.r0) * P.inv_dr;
  s = fminf(fmaxf(s, 0.0f), static_cast<float>(P.n_tab - 1));
  int k = min(static_cast<int>(s), P.n_tab - 2);
  const float f = s - static_cast<float>(k);
  const float4 a0 = __ldg(P.tab + 2 * k), a1 = __ldg(P.tab + 2 * k + 2);
  const float4 w0 = __ldg(P.tab + 2 * k + 1), w1 = __ldg(P.tab + 2 * k + 3);
  const float aa[3] = {fmaf(f, a1.x - a0.x, a0.x), fmaf(f, a1.y - a0.y, a0.y), fmaf(f, a1.z - a0.z, a0.z)};
  const float ww[3] = {fmaf(f, w1.x - w0.x, w0.x), fmaf(f, w1.y - w0.y, w0.y), fmaf(f, w1.z - w0.z, w0.z)};
  const float norm = fmaf(f, a1.w - a0.w, a0.w);
  float p = 0.0f;
#pragma unroll
  for (int i = 0; i < 3; ++i) p = fmaf(ww[i], expf(aa[i] * __ldg(P.box[i] + v * P.stride)), p);
  const float prob = fminf(1.0f, norm * fmaxf(p, 0.0f));
  w = philox4x32_10(u32x4{static_cast<uint32_t>(v), static_cast<uint32_t>(static_cast<uint64_t>(v) >> 32), 0x51534Fu, 0u},
                    P.key0, P.key1);
  return (__uint2float_rn(w.x) + 0.5f) * 0x1p-32f < prob;  // (w0 + 1/2) 2^-32 < P in FP32
}

constexpr int kDrawThreads = 256;
constexpr int kSub = 1024;  // voxels per warp sub-range (count and write passes)

// Record of an accepted voxel.  Out of line, so that its FP64 arithmetic runs
// only for accepted voxels instead of being predicated into every iteration.
__device__ __noinline__ void write_qso(const DrawParams &P, int64_t o, int64_t v, u32x4 w, int x, int y, int z) {
  mk_qso q;
  q.pos[0] = P.origin_d[0] + (x + (static_cast<double>(w.y) + 0.5) * 0x1p-32) * P.cell_d;
  q.pos[1] = P.origin_d[1] + (y + (static_cast<double>(w.z) + 0.5) * 0x1p-32) * P.cell_d;
  q.pos[2] = P.origin_d[2] + (z + (static_cast<double>(w.w) + 0.5) * 0x1p-32) * P.cell_d;
  q.id = static_cast<uint64_t>(v);
  P.out[o] = q;
}

// One warp per sub-range of kSub voxels: the accepted count (ballot/popc).
__global__ void __launch_bounds__(kDrawThreads) k_qso_count(DrawParams P) {
  const int64_t nv = static_cast<int64_t>(P.n) * P.n * P.n;
  const int64_t subs = (nv + kSub - 1) / kSub;
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (kDrawThreads / 32);
  for (int64_t s = blockIdx.x * static_cast<int64_t>(kDrawThreads / 32) + (threadIdx.x >> 5); s < subs; s += warps) {
    const int64_t v0 = s * kSub, v1 = min(nv, v0 + kSub);
    int c = 0;
    for (int64_t c0 = v0; c0 < v1; c0 += 32) {
      const int64_t v = c0 + lane;
      u32x4 w;
      int x, y, z;
      const bool acc = v < v1 && voxel_accept(P, v, w, x, y, z);
      c += __popc(__ballot_sync(0xffffffffu, acc));
    }
    if (lane == 0) P.count32[s] = c;
  }
}

// The same decisions, written in voxel order from each sub-range's offset.
__global__ void __launch_bounds__(kDrawThreads) k_qso_write(DrawParams P) {
  const int64_t nv = static_cast<int64_t>(P.n) * P.n * P.n;
  const int64_t subs = (nv + kSub - 1) / kSub;
  const int lane = threadIdx.x & 31;
  const int64_t warps = static_cast<int64_t>(gridDim.x) * (kDrawThreads / 32);
  for (int64_t s = blockIdx.x * static_cast<int64_t>(kDrawThreads / 32) + (threadIdx.x >> 5); s < subs; s += warps) {
    const int64_t v0 = s * kSub, v1 = min(nv, v0 + kSub);
    int64_t base = P.offset[s];
    for (int64_t c0 = v0; c0 < v1; c0 += 32) {
      const int64_t v = c0 + lane;
      u32x4 w{0u, 0u, 0u, 0u};
      int x = 0, y = 0, z = 0;
      const bool acc = v < v1 && voxel_accept(P, v, w, x, y, z);
      const uint32_t m = __ballot_sync(0xffffffffu, acc);
      if (m != 0u) {  // warp-uniform: most chunks of 32 voxels accept none
        const int64_t o = base + __popc(m & ((1u << lane) - 1u));
        if (acc && o < P.capacity) write_qso(P, o, v, w, x, y, z);
      }
      base += __popc(m);
    }
  }
}

// Sums of delta_q,i^2 (FP32 over runs of 32 elements per thread, FP64 across
// runs and threads), one partial per block, summed on the host in order.
__global__ void __launch_bounds__(kDrawThreads) k_box_sq_sum(const float *b0, const float *b1, const float *b2,
                                                             int32_t stride, int64_t nv, double *partial) {
  __shared__ double red[3][kDrawThreads];
  double s[3] = {0.0, 0.0, 0.0};
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
  int64_t v = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  while (v < nv) {
    float f[3] = {0.f, 0.f, 0.f};
#pragma unroll 8
    for (int r = 0; r < 32 && v < nv; ++r, v += step) {
      const float a = __ldg(b0 + v * stride), b = __ldg(b1 + v * stride), c = __ldg(b2 + v * stride);
      f[0] = fmaf(a, a, f[0]);
      f[1] = fmaf(b, b, f[1]);
      f[2] = fmaf(c, c, f[2]);
    }
    for (int i = 0; i < 3; ++i) s[i] += f[i];
  }
  for (int i = 0; i < 3; ++i) red[i][threadIdx.x] = s[i];
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int i = 0; i < 3; ++i) red[i][threadIdx.x] += red[i][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int i = 0; i < 3; ++i) partial[3 * blockIdx.x + i] = red[i][0];
}

double bias_of(const double *bl, double z) { return bl[0] * std::pow((1.0 + z) / (1.0 + bl[1]), bl[2]); }

}  // namespace

extern "C" int mk_xi_of_pk(const double *h_pk, int32_t n_pk, double dk, const double *h_r, int32_t n_r,
                           double *h_xi) {
  if (!h_pk || n_pk < 2 || !(dk > 0.0) || (n_r > 0 && (!h_r || !h_xi)) || n_r < 0) return MK_EINVAL;
  for (int j = 0; j < n_r; ++j) h_xi[j] = xi_at(h_pk, n_pk, dk, h_r[j]);
  return MK_OK;
}

extern "C" int mk_lognormal_pk(const double *h_pk, int32_t n_pk, double dk, double B, double *h_pq) {
  if (!h_pk || !h_pq || n_pk < 2 || !(dk > 0.0) || !(B >= 0.0)) return MK_EINVAL;
  const int n = n_pk;
  const double dr = M_PI / (dk * (n - 1));
  std::vector<double> g(n);
  for (int j = 0; j < n; ++j) {
    const double r = j * dr, arg = 1.0 + B * xi_at(h_pk, n, dk, r);
    if (!(arg > 0.0)) return MK_EINVAL;
    const double w = (j == 0 || j == n - 1) ? 0.5 : 1.0;
    g[j] = w * dr * std::log(arg) * r * r;
  }
  for (int i = 0; i < n; ++i) {
    const double k = i * dk;
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += g[j] * sinc_j0(k * j * dr);
    h_pq[i] = std::max(0.0, 4.0 * M_PI * s);  // ringing of the finite sums where P_q is small
  }
  return MK_OK;
}

extern "C" int mk_draw_qso(mk_ctx *ctx, const mk_qso_draw_params *q, const float *const d_box_q[3], int32_t box_stride,
                           mk_qso *d_qso, int64_t capacity, int64_t *h_count) {
  MK_TRACE("mk_draw_qso");
  if (!ctx) return MK_EINVAL;
  if (!q || !d_box_q || !d_box_q[0] || !d_box_q[1] || !d_box_q[2] || !h_count || (capacity > 0 && !d_qso) ||
      capacity < 0)
    return qfail(ctx, MK_EINVAL, "mk_draw_qso: NULL argument");
  int lgn = 0;
  while (lgn < 12 && (1 << lgn) < q->n) ++lgn;
  if (q->n < 2 || q->n > 2048 || (1 << lgn) != q->n || !(q->cell > 0.0) || (box_stride != 1 && box_stride != 2))
    return qfail(ctx, MK_EINVAL, "mk_draw_qso: box side must be a power of two in [2, 2048]; bad cell or stride");
  if (!(q->z_box[0] < q->z_box[1] && q->z_box[1] < q->z_box[2]) || !(q->bias[0] > 0.0))
    return qfail(ctx, MK_EINVAL, "mk_draw_qso: box redshifts must increase and the bias be > 0");
  if (!q->h_nbar || q->n_nbar < 2 || !(q->nbar_dz > 0.0)) return qfail(ctx, MK_EINVAL, "mk_draw_qso: bad nbar table");
  CKQ(ctx, cudaSetDevice(mkhost::ctx_device(ctx)));
  const cudaStream_t st = mkhost::ctx_stream(ctx);
  const int64_t n = q->n, nv = n * n * n;
  // sigma_i^2 = mean delta_q,i^2 (fixed grid, partials summed in order)
  const int red_blocks = std::min<int64_t>(4 * mkhost::ctx_sms(ctx), (nv + kDrawThreads - 1) / kDrawThreads);
  double *d_part = nullptr;
  CKQ(ctx, cudaMalloc(&d_part, sizeof(double) * 3 * red_blocks));
  k_box_sq_sum<<<red_blocks, kDrawThreads, 0, st>>>(d_box_q[0], d_box_q[1], d_box_q[2], box_stride, nv, d_part);
  std::vector<double> part(3 * red_blocks);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(part.data(), d_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_part);
  CKQ(ctx, e);
  double sig2[3] = {0.0, 0.0, 0.0};
  for (int b = 0; b < red_blocks; ++b)
    for (int i = 0; i < 3; ++i) sig2[i] += part[3 * b + i];
  for (int i = 0; i < 3; ++i) sig2[i] /= static_cast<double>(nv);

  // coefficient table over the box's range of distances
  double rmin2 = 0.0, rmax2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double lo = q->origin[d], hi = q->origin[d] + n * q->cell;
    const double near = (lo > 0.0) ? lo : (hi < 0.0 ? -hi : 0.0);
    const double far = std::max(std::fabs(lo), std::fabs(hi));
    rmin2 += near * near;
    rmax2 += far * far;
  }
  const int n_tab = 8192;
  const double r0 = std::sqrt(rmin2), r1 = std::sqrt(rmax2) + 1e-6;
  const double dr = (r1 - r0) / (n_tab - 1);
  double bz[3], xi0[3];
  for (int i = 0; i < 3; ++i) {
    const double g = mkhost::ctx_growth(ctx, q->z_box[i]);
    bz[i] = bias_of(q->bias, q->z_box[i]);
    xi0[i] = bz[i] * bz[i] * g * g * q->xi_m5;
  }
  std::vector<float4> tab(2 * n_tab);
  for (int k = 0; k < n_tab; ++k) {
    const double r = r0 + k * dr, z = mkhost::ctx_z_of(ctx, r), g = mkhost::ctx_growth(ctx, z);
    const double b = bias_of(q->bias, z);
    double a[3], xi[3];
    for (int i = 0; i < 3; ++i) {
      a[i] = b * (1.0 + q->z_box[i]) / (bz[i] * (1.0 + z));
      xi[i] = std::pow(1.0 + xi0[i], a[i] * a[i]) - 1.0;
    }
    const double t12 = (z - q->z_box[0]) / (q->z_box[1] - q->z_box[0]);
    const double t23 = (z - q->z_box[1]) / (q->z_box[2] - q->z_box[1]);
    const double xi12 = (1.0 - t12) * xi[0] + t12 * xi[1], xi23 = (1.0 - t23) * xi[1] + t23 * xi[2];
    const double xmod = b * b * g * g * q->xi_m5;
    double lam = std::fabs(xi12 - xi23) > 0.0 ? (xmod - xi23) / (xi12 - xi23) : 0.5;
    lam = std::min(1.0, std::max(0.0, lam));
    const double w[3] = {lam * (1.0 - t12), lam * t12 + (1.0 - lam) * (1.0 - t23), (1.0 - lam) * t23};
    double ep = 0.0;
    for (int i = 0; i < 3; ++i) ep += w[i] * std::exp(0.5 * a[i] * a[i] * sig2[i]);
    double nb = 0.0;
    const double s = (z - q->nbar_z0) / q->nbar_dz;
    if (s >= 0.0 && s <= q->n_nbar - 1) {
      const int j = std::min(static_cast<int>(std::floor(s)), q->n_nbar - 2);
      nb = q->h_nbar[j] + (s - j) * (q->h_nbar[j + 1] - q->h_nbar[j]);
    }
    const double norm = ep > 0.0 ? nb * q->cell * q->cell * q->cell / ep : 0.0;
    tab[2 * k] = make_float4(static_cast<float>(a[0]), static_cast<float>(a[1]), static_cast<float>(a[2]),
                             static_cast<float>(norm));
    tab[2 * k + 1] = make_float4(static_cast<float>(w[0]), static_cast<float>(w[1]), static_cast<float>(w[2]), 0.f);
  }
  DrawParams P{};
  for (int i = 0; i < 3; ++i) P.box[i] = d_box_q[i];
  P.stride = box_stride;
  P.n = q->n;
  P.lgn = lgn;
  P.cell = static_cast<float>(q->cell);
  for (int d = 0; d < 3; ++d) {
    P.origin[d] = static_cast<float>(q->origin[d]);
    P.origin_d[d] = q->origin[d];
  }
  P.cell_d = q->cell;
  P.n_tab = n_tab;
  P.r0 = static_cast<float>(r0);
  P.inv_dr = static_cast<float>(1.0 / dr);
  P.key0 = static_cast<uint32_t>(q->seed);
  P.key1 = static_cast<uint32_t>(q->seed >> 32);
  P.out = d_qso;
  P.capacity = capacity;
  const int64_t subs = (nv + kSub - 1) / kSub;
  float4 *d_tab = nullptr;
  int32_t *d_cnt = nullptr;
  int64_t *d_off = nullptr;
  std::vector<int32_t> cnt(subs);
  std::vector<int64_t> off(subs);
  e = cudaMalloc(&d_tab, sizeof(float4) * tab.size());
  if (e == cudaSuccess) e = cudaMalloc(&d_cnt, sizeof(int32_t) * subs);
  if (e == cudaSuccess) e = cudaMalloc(&d_off, sizeof(int64_t) * subs);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, tab.data(), sizeof(float4) * tab.size(), cudaMemcpyHostToDevice, st);
  const int64_t warps_per_block = kDrawThreads / 32;
  const int grid = static_cast<int>(
      std::min<int64_t>((subs + warps_per_block - 1) / warps_per_block, 8 * mkhost::ctx_sms(ctx)));
  P.tab = d_tab;
  P.count32 = d_cnt;
  P.offset = d_off;
  if (e == cudaSuccess) {
    k_qso_count<<<grid, kDrawThreads, 0, st>>>(P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int32_t) * subs, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  int64_t total = 0;
  if (e == cudaSuccess) {
    for (int64_t t = 0; t < subs; ++t) {
      off[t] = total;
      total += cnt[t];
    }
    e = cudaMemcpyAsync(d_off, off.data(), sizeof(int64_t) * subs, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess && capacity > 0) {
    k_qso_write<<<grid, kDrawThreads, 0, st>>>(P);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_tab);
  cudaFree(d_cnt);
  cudaFree(d_off);
  CKQ(ctx, e);
  *h_count = total;
  if (total > capacity) return qfail(ctx, MK_ERANGE, "mk_draw_qso: more quasars than capacity (count returned)");
  return MK_OK;
}
