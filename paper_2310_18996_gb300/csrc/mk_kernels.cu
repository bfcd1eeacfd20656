// Kernels of the skewer-synthesis path (sm_103a) and their host launchers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mk_device.cuh"
#include "mk_kernels.h"

namespace mk {

// =================================================================== geometry
// D_C(z) by cubic Hermite interpolation of the FP64 table (values + slopes).
__device__ __forceinline__ double dc_eval(const DcTable &T, double z) {
  double s = z / T.h;
  int i = static_cast<int>(floor(s));
  i = max(0, min(i, T.n - 2));
  const double t = s - i;
  const double2 a = T.dc[i], b = T.dc[i + 1];
  const double t2 = t * t, t3 = t2 * t;
  return (2.0 * t3 - 3.0 * t2 + 1.0) * a.x + (t3 - 2.0 * t2 + t) * T.h * a.y +
         (-2.0 * t3 + 3.0 * t2) * b.x + (t3 - t2) * T.h * b.y;
}

// z(r): linear interpolation in the z(r) table (error ~1e-7), then two
// Newton steps on the Hermite D_C, dz = (D_C(z) - r) E(z) H0/c.
__device__ double z_of_dc(const DcTable &T, double r) {
  const double s = r * T.inv_hr;
  const int i = max(0, min(static_cast<int>(s), T.n_r - 2));
  const double z0 = T.zr[i], z1 = T.zr[i + 1];
  double z = fma(s - i, z1 - z0, z0);
  for (int it = 0; it < 2; ++it) {
    const double zp = 1.0 + z;
    const double e = sqrt(fma(T.omega_m * zp, zp * zp, 1.0 - T.omega_m));
    z -= (dc_eval(T, z) - r) * e * (1.0 / 2997.92458);
  }
  return z;
}

__global__ void k_geometry(const mk_qso *__restrict__ q, int64_t nq, GeomParams P, mk_skewer *sk,
                           int64_t *cnt_px, int64_t *cnt_seg, int *err) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i >= nq) return;
  const mk_qso Q = q[i];
  mk_skewer s;
  s.offset = 0;
  s.n = 0;
  s.j_lo = 0;
  s.id = Q.id;
  for (int d = 0; d < 3; ++d) s.p0[d] = s.step[d] = 0;
  const double r = sqrt(Q.pos[0] * Q.pos[0] + Q.pos[1] * Q.pos[1] + Q.pos[2] * Q.pos[2]);
  if (r > 0.0) {
    const double zmax = (P.tab.n - 2) * P.tab.h;
    const double zq = z_of_dc(P.tab, r);
    double z_lo = (1.0 + zq) * P.lrf_min / P.lambda_lya - 1.0;
    const double z_hi = (1.0 + zq) * P.lrf_max / P.lambda_lya - 1.0;
    if (P.lobs_min > 0.0) z_lo = fmax(z_lo, P.lobs_min / P.lambda_lya - 1.0);
    z_lo = fmax(z_lo, 0.0);
    int64_t jl = 0, n = 0;
    if (z_hi > z_lo) {
      if (z_hi >= zmax) {
        raise_error(err, ERR_RANGE);
      } else {
        const double r_lo = dc_eval(P.tab, z_lo), r_hi = dc_eval(P.tab, z_hi);
        jl = static_cast<int64_t>(ceil(r_lo / P.dr - 0.5));
        const int64_t jh = static_cast<int64_t>(ceil(r_hi / P.dr - 0.5));
        n = jh > jl ? jh - jl : 0;
        if (P.n_max > 0 && n > P.n_max) {
          jl = jh - P.n_max;
          n = P.n_max;
        }
        if (n < P.n_min) n = 0;
        if (n > 0 && (jl < 0 || jl + n > P.j_max)) {
          raise_error(err, ERR_RANGE);
          n = 0;
        }
      }
    }
    s.n = static_cast<int32_t>(n);
    s.j_lo = static_cast<int32_t>(jl);
    // Q20.44 cell coordinates of the first pixel and the step (rounding at
    // 2^-44 cells; the pixel decisions above use the exact divisions)
    const double rc = (static_cast<double>(jl) + 0.5) * P.dr;
    const double inv_r = 1.0 / r, inv_cell = 1.0 / P.cell;
    for (int d = 0; d < 3; ++d) {
      const double u = Q.pos[d] * inv_r;
      const double c0 = fma(rc * u - P.origin[d], inv_cell, -0.5);
      s.p0[d] = llrint(c0 * 0x1p44);
      s.step[d] = llrint(P.dr * u * inv_cell * 0x1p44);
    }
  }
  sk[i] = s;
  cnt_px[i] = P.rebin > 0 ? s.n / P.rebin : s.n;
  cnt_seg[i] = P.n_fft > 0 ? (s.n + P.n_fft - 1) / P.n_fft : 0;
}

// =================================================================== scan
// Exclusive prefix sums of two int64 sequences (pixels, segments) in three
// passes over tiles of SCAN_TILE elements.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

struct Pair {
  int64_t a, b;
};

__device__ __forceinline__ Pair block_exclusive_scan(Pair v, Pair *sh, Pair &total) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int off = 1; off < SCAN_THREADS; off <<= 1) {
    Pair add = {0, 0};
    if (t >= off) add = sh[t - off];
    __syncthreads();
    sh[t].a += add.a;
    sh[t].b += add.b;
    __syncthreads();
  }
  total = sh[SCAN_THREADS - 1];
  Pair ex = {sh[t].a - v.a, sh[t].b - v.b};
  __syncthreads();
  return ex;
}

__global__ void k_scan_tiles(const int64_t *a, const int64_t *b, int64_t n, Pair *tile_sum) {
  __shared__ Pair sh[SCAN_THREADS];
  const int64_t base = blockIdx.x * static_cast<int64_t>(SCAN_TILE) + threadIdx.x * SCAN_ITEMS;
  Pair v = {0, 0};
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) {
      v.a += a[base + k];
      v.b += b ? b[base + k] : 0;
    }
  }
  Pair tot;
  block_exclusive_scan(v, sh, tot);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void k_scan_tile_sums(Pair *tile_sum, int64_t ntiles) {
  __shared__ Pair sh[SCAN_THREADS];
  Pair carry = {0, 0};
  for (int64_t base = 0; base < ntiles; base += SCAN_THREADS) {
    const int64_t i = base + threadIdx.x;
    Pair v = (i < ntiles) ? tile_sum[i] : Pair{0, 0};
    Pair tot;
    Pair ex = block_exclusive_scan(v, sh, tot);
    if (i < ntiles) tile_sum[i] = Pair{ex.a + carry.a, ex.b + carry.b};
    carry.a += tot.a;
    carry.b += tot.b;
  }
}

__global__ void k_scan_apply(const int64_t *a, const int64_t *b, int64_t n, const Pair *tile_sum,
                             int64_t *out_a, int64_t *out_b, mk_skewer *sk) {
  __shared__ Pair sh[SCAN_THREADS];
  const int64_t base = blockIdx.x * static_cast<int64_t>(SCAN_TILE) + threadIdx.x * SCAN_ITEMS;
  Pair v = {0, 0};
  int64_t va[SCAN_ITEMS], vb[SCAN_ITEMS];
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    va[k] = (base + k < n) ? a[base + k] : 0;
    vb[k] = (base + k < n && b) ? b[base + k] : 0;
    v.a += va[k];
    v.b += vb[k];
  }
  Pair tot;
  Pair ex = block_exclusive_scan(v, sh, tot);
  const Pair ts = tile_sum[blockIdx.x];
  int64_t ra = ts.a + ex.a, rb = ts.b + ex.b;
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) {
      out_a[base + k] = ra;
      if (out_b) out_b[base + k] = rb;
      if (sk) sk[base + k].offset = ra;
    }
    ra += va[k];
    rb += vb[k];
  }
  // the thread holding element n - 1 writes the totals at index n
  if (base <= n - 1 && n - 1 < base + SCAN_ITEMS) {
    out_a[n] = ra;
    if (out_b) out_b[n] = rb;
  }
}

// =================================================================== tables
__global__ void k_pixtab(const double *__restrict__ zpix, const float *__restrict__ gpix, int32_t j_max,
                         NodeParams nd, float4 *pixtab) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= j_max) return;
  const double z = zpix[j];
  double la, b, c;
  const int k = nd.count;
  if (z <= nd.z[0]) {
    la = nd.ln_a[0]; b = nd.b[0]; c = nd.c[0];
  } else if (z >= nd.z[k - 1]) {
    la = nd.ln_a[k - 1]; b = nd.b[k - 1]; c = nd.c[k - 1];
  } else {
    int i = 0;
    while (i + 2 < k && z >= nd.z[i + 1]) ++i;
    const double w = (z - nd.z[i]) / (nd.z[i + 1] - nd.z[i]);
    la = (1.0 - w) * nd.ln_a[i] + w * nd.ln_a[i + 1];
    b = (1.0 - w) * nd.b[i] + w * nd.b[i + 1];
    c = (1.0 - w) * nd.c[i] + w * nd.c[i + 1];
  }
  const double log2e = 1.4426950408889634;
  pixtab[j] = make_float4(gpix[j], static_cast<float>(exp(la) * log2e), static_cast<float>(b * log2e),
                          static_cast<float>(c));
}

__device__ __forceinline__ int16_t bin_of(double z, double z_lo, double dz, int n_z) {
  const double f = floor((z - z_lo) / dz);
  return static_cast<int16_t>(f < 0.0 ? -1 : (f >= n_z ? n_z : static_cast<int>(f)));
}

// Pixel z bins and, for segments of n_seg pixels starting at J, the z bin of
// the segment's mean z (n_z where the segment leaves the tables).
__global__ void k_zbin(const double *__restrict__ zpix, const double *__restrict__ cumz, int32_t j_max,
                       double z_lo, double dz, int n_z, int n_seg, int16_t *zbin, int16_t *segzbin) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= j_max) return;
  zbin[j] = bin_of(zpix[j], z_lo, dz, n_z);
  segzbin[j] = (j + n_seg <= j_max) ? bin_of((cumz[j + n_seg] - cumz[j]) / n_seg, z_lo, dz, n_z)
                                    : static_cast<int16_t>(n_z);
}

// bin_end[k + 1] for k = -1 .. n_z: the first J whose z bin exceeds k (zbin is
// non-decreasing in J); kBinEndNever where no tabulated pixel does.  One CTA.
__global__ void k_bin_end(const int16_t *__restrict__ zbin, int32_t j_max, int n_z, int32_t *bin_end) {
  for (int k = threadIdx.x; k <= n_z + 1; k += blockDim.x) bin_end[k] = kBinEndNever;
  __syncthreads();
  for (int j = threadIdx.x; j < j_max; j += blockDim.x) {
    const int z = zbin[j];
    const int zp = j ? max(static_cast<int>(zbin[j - 1]), -1) : -1;
    for (int k = zp; k < z; ++k) bin_end[k + 1] = j;
  }
}

// Difference array of the pixel count per global pixel J: +1 at j_lo, -1 at
// j_lo + n of every skewer (diff has j_max + 1 entries, zeroed by the caller).
__global__ void k_jcount(const mk_skewer *__restrict__ sk, int64_t n_sk, int32_t j_max, int32_t *diff) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n_sk;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int32_t a = sk[i].j_lo, n = sk[i].n;
    if (n <= 0 || a < 0 || a + n > j_max) continue;
    atomicAdd(diff + a, 1);
    atomicAdd(diff + a + n, -1);
  }
}

// zwin[J] = mean z of pixels J .. J+n-1 (the window of a delta_S segment
// starting at J), cut at the end of the tables.
__global__ void k_zwin(const double *__restrict__ cumz, int32_t j_max, int n, float *zwin) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= j_max) return;
  const int e = min(j + n, j_max);
  zwin[j] = static_cast<float>((cumz[e] - cumz[j]) / (e - j));
}

// out[i] = off[i n / k], i = 0..k: the offsets at the slice boundaries.
__global__ void k_pick(const int64_t *__restrict__ off, int64_t n, int k, int64_t *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= k) out[i] = off[static_cast<int64_t>(i) * n / k];
}

// (n+1)^3 padded pairs from planar n^3 boxes (periodic ghost layer).
__global__ void k_pack_padded(const float *__restrict__ d, const float *__restrict__ e, int lgn, float2 *out) {
  const int64_t n = int64_t(1) << lgn, n1 = n + 1, total = n1 * n1 * n1;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t x = i % n1, y = (i / n1) % n1, z = i / (n1 * n1);
    const int64_t src = ((z & (n - 1)) << (2 * lgn)) | ((y & (n - 1)) << lgn) | (x & (n - 1));
    out[i] = make_float2(d[src], e[src]);
  }
}

// (n+6)^3 pairs with a periodic margin of 3 from planar n^3 boxes.
__global__ void k_pack_halo(const float *__restrict__ d, const float *__restrict__ e, int lgn, float2 *out) {
  const int64_t n = int64_t(1) << lgn, p = n + 6, total = p * p * p;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t x = i % p - 3, y = (i / p) % p - 3, z = i / (p * p) - 3;
    const int64_t src = ((z & (n - 1)) << (2 * lgn)) | ((y & (n - 1)) << lgn) | (x & (n - 1));
    out[i] = make_float2(d[src], e[src]);
  }
}

// (n+1)^3 points of {delta, eta_xx, eta_yy, eta_zz, eta_xy, eta_xz, eta_yz, 0}
// from planar boxes (e6: six n^3 boxes), periodic ghost layer as k_pack_padded.
__global__ void k_pack_tensor(const float *__restrict__ d, const float *__restrict__ e6, int lgn, float4 *out) {
  const int64_t n = int64_t(1) << lgn, n1 = n + 1, total = n1 * n1 * n1, n3 = n * n * n;
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t x = i % n1, y = (i / n1) % n1, z = i / (n1 * n1);
    const int64_t src = ((z & (n - 1)) << (2 * lgn)) | ((y & (n - 1)) << lgn) | (x & (n - 1));
    out[2 * i] = make_float4(d[src], e6[src], e6[n3 + src], e6[2 * n3 + src]);
    out[2 * i + 1] = make_float4(e6[3 * n3 + src], e6[4 * n3 + src], e6[5 * n3 + src], 0.f);
  }
}

__global__ void k_pack(const float *__restrict__ d, const float *__restrict__ e, int64_t n, float2 *out) {
  for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x)
    out[i] = make_float2(d[i], e[i]);
}

__global__ void k_out_counts(const mk_skewer *sk, int64_t n, int rebin, int64_t *cnt) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) cnt[i] = sk[i].n / rebin;
}

__global__ void k_seg_counts(const int64_t *off, int64_t n, int n_fft, int64_t *cnt) {
  const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
  if (i < n) cnt[i] = (off[i + 1] - off[i] + n_fft - 1) / n_fft;
}

// =================================================================== flux kernel
__global__ void __launch_bounds__(256) k_flux(FluxParams P) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i = warp; i < P.n_sk; i += nwarps) {
    const mk_skewer sk = P.sk[i];
    const int64_t o = P.off_out[i];
    const int64_t nout = P.off_out[i + 1] - o;
    if (o + nout > P.capacity) {
      if (lane == 0) raise_error(P.err, ERR_CAPACITY);
      continue;
    }
    // records made for another pixel length (read back from a file) may run
    // past the pixel tables
    if (sk.j_lo < 0 || sk.j_lo + nout * P.rebin > P.j_max) {
      if (lane == 0) raise_error(P.err, ERR_RANGE);
      continue;
    }
    for (int64_t k = lane; k < nout; k += 32) {
      float s = 0.f;
      for (int r = 0; r < P.rebin; ++r) {
        const int64_t j = k * P.rebin + r;
        const float4 tb = __ldg(P.pixtab + sk.j_lo + j);
        s += fgpa(tb, P.delta[sk.offset + j], P.eta[sk.offset + j]);
      }
      P.flux[o + k] = P.rebin == 1 ? s : s / static_cast<float>(P.rebin);
    }
  }
}

// =================================================================== finalize
__global__ void k_finalize(const double *__restrict__ partials, int nparts, int n_z, int n_k, int n_fft,
                           mk_stats_out *out) {
  extern __shared__ double tot[];
  const StatLayout L{n_z, n_k};
  const int size = L.size();
  for (int idx = threadIdx.x; idx < size; idx += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += partials[static_cast<size_t>(c) * size + idx];
    tot[idx] = s;
  }
  // zero the output struct
  double *o = reinterpret_cast<double *>(out);
  for (int idx = threadIdx.x; idx < static_cast<int>(sizeof(mk_stats_out) / sizeof(double)); idx += blockDim.x)
    o[idx] = 0.0;
  __syncthreads();
  const double per_bin = static_cast<double>(n_fft / 2) / n_k;
  for (int zb = threadIdx.x; zb < n_z; zb += blockDim.x) {
    for (int i = 0; i < MK_NSUM; ++i) out->sums[zb][i] = tot[L.sums(zb, i)];
    for (int k = 0; k < n_k; ++k) out->p1d_sum[zb][k] = tot[L.p1d(zb, k)];
    out->n_seg[zb] = tot[L.nseg(zb)];
    finalize_bin(out, zb, n_k, per_bin);
  }
}

// =================================================================== launchers
static int blocks_for(int64_t n, int threads) { return static_cast<int>((n + threads - 1) / threads); }

cudaError_t launch_geometry(const mk_qso *q, int64_t nq, const GeomParams &P, mk_skewer *sk, int64_t *cnt_px,
                            int64_t *cnt_seg, int *err, cudaStream_t st) {
  if (nq == 0) return cudaSuccess;
  k_geometry<<<blocks_for(nq, 128), 128, 0, st>>>(q, nq, P, sk, cnt_px, cnt_seg, err);
  return cudaGetLastError();
}

size_t scan_workspace_bytes(int64_t n) {
  return sizeof(Pair) * static_cast<size_t>((n + SCAN_TILE - 1) / SCAN_TILE + 1);
}

cudaError_t launch_scan(const int64_t *a, const int64_t *b, int64_t n, int64_t *out_a, int64_t *out_b,
                        mk_skewer *sk, void *ws, cudaStream_t st) {
  if (n == 0) {
    cudaError_t e = cudaMemsetAsync(out_a, 0, sizeof(int64_t), st);
    if (e == cudaSuccess && out_b) e = cudaMemsetAsync(out_b, 0, sizeof(int64_t), st);
    return e;
  }
  const int64_t ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  Pair *ts = static_cast<Pair *>(ws);
  k_scan_tiles<<<static_cast<unsigned>(ntiles), SCAN_THREADS, 0, st>>>(a, b, n, ts);
  k_scan_tile_sums<<<1, SCAN_THREADS, 0, st>>>(ts, ntiles);
  k_scan_apply<<<static_cast<unsigned>(ntiles), SCAN_THREADS, 0, st>>>(a, b, n, ts, out_a, out_b, sk);
  return cudaGetLastError();
}

cudaError_t launch_pixtab(const double *zpix, const float *gpix, int32_t j_max, const NodeParams &nd,
                          float4 *pixtab, cudaStream_t st) {
  k_pixtab<<<blocks_for(j_max, 256), 256, 0, st>>>(zpix, gpix, j_max, nd, pixtab);
  return cudaGetLastError();
}

cudaError_t launch_zbin(const double *zpix, const double *cumz, int32_t j_max, double z_lo, double dz, int n_z,
                        int n_seg, int16_t *zbin, int16_t *segzbin, cudaStream_t st) {
  k_zbin<<<blocks_for(j_max, 256), 256, 0, st>>>(zpix, cumz, j_max, z_lo, dz, n_z, n_seg, zbin, segzbin);
  return cudaGetLastError();
}

cudaError_t launch_jcount(const mk_skewer *sk, int64_t n_sk, int32_t j_max, int32_t *diff, int sms, cudaStream_t st) {
  if (n_sk == 0) return cudaSuccess;
  k_jcount<<<sms * 4, 256, 0, st>>>(sk, n_sk, j_max, diff);
  return cudaGetLastError();
}

cudaError_t launch_zwin(const double *cumz, int32_t j_max, int n, float *zwin, cudaStream_t st) {
  k_zwin<<<blocks_for(j_max, 256), 256, 0, st>>>(cumz, j_max, n, zwin);
  return cudaGetLastError();
}

cudaError_t launch_pick(const int64_t *off, int64_t n, int k, int64_t *out, cudaStream_t st) {
  k_pick<<<blocks_for(k + 1, 64), 64, 0, st>>>(off, n, k, out);
  return cudaGetLastError();
}

cudaError_t launch_bin_end(const int16_t *zbin, int32_t j_max, int n_z, int32_t *bin_end, cudaStream_t st) {
  k_bin_end<<<1, 256, 0, st>>>(zbin, j_max, n_z, bin_end);
  return cudaGetLastError();
}

cudaError_t launch_pack_tensor(const float *d, const float *e6, int lgn, float *out, int sms, cudaStream_t st) {
  k_pack_tensor<<<sms * 8, 256, 0, st>>>(d, e6, lgn, reinterpret_cast<float4 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_pack_halo(const float *d, const float *e, int lgn, float *out, int sms, cudaStream_t st) {
  k_pack_halo<<<sms * 8, 256, 0, st>>>(d, e, lgn, reinterpret_cast<float2 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_pack_padded(const float *d, const float *e, int lgn, float *out, int sms, cudaStream_t st) {
  k_pack_padded<<<sms * 8, 256, 0, st>>>(d, e, lgn, reinterpret_cast<float2 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_pack(const float *d, const float *e, int64_t n, float *out, int sms, cudaStream_t st) {
  k_pack<<<sms * 8, 256, 0, st>>>(d, e, n, reinterpret_cast<float2 *>(out));
  return cudaGetLastError();
}

cudaError_t launch_out_counts(const mk_skewer *sk, int64_t n, int rebin, int64_t *cnt, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_out_counts<<<blocks_for(n, 256), 256, 0, st>>>(sk, n, rebin, cnt);
  return cudaGetLastError();
}

cudaError_t launch_seg_counts(const int64_t *off, int64_t n, int n_fft, int64_t *cnt, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_seg_counts<<<blocks_for(n, 256), 256, 0, st>>>(off, n, n_fft, cnt);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ dispatch by FFT length
#define MK_SWITCH(EXPR, FAIL)                  \
  switch (n_fft) {                             \
    case 256: return SkewerUnit<256>::EXPR;    \
    case 512: return SkewerUnit<512>::EXPR;    \
    case 1024: return SkewerUnit<1024>::EXPR;  \
    case 2048: return SkewerUnit<2048>::EXPR;  \
  }                                            \
  return FAIL;

size_t skewer_smem_bytes(int n_fft, int threads, int n_z, int n_k, bool stats) {
  MK_SWITCH(smem_bytes(threads, n_z, n_k, stats), 0)
}

int skewer_blocks_per_sm(int n_fft, int variant, int lgn, int minb, int threads, int n_z, int n_k, bool stats) {
  MK_SWITCH(blocks_per_sm(variant, lgn, minb, threads, n_z, n_k, stats), 1)
}

cudaError_t launch_skewer(const SkewerParams &P, int n_fft, int variant, int minb, int grid, int threads,
                          cudaStream_t st) {
  MK_SWITCH(launch(P, variant, minb, grid, threads, st), cudaErrorInvalidValue)
}

int stats_blocks_per_sm(int n_fft, int threads, int n_z, int n_k, bool tune) {
  MK_SWITCH(stats_blocks_per_sm(threads, n_z, n_k, tune), 1)
}

cudaError_t launch_stats(const StatParams &P, int n_fft, int grid, int threads, cudaStream_t st) {
  MK_SWITCH(launch_stats(P, grid, threads, st), cudaErrorInvalidValue)
}
#undef MK_SWITCH

cudaError_t launch_flux(const FluxParams &P, int sms, cudaStream_t st) {
  if (P.n_sk == 0) return cudaSuccess;
  const int64_t warps = P.n_sk;
  int grid = blocks_for(warps * 32, 256);
  if (grid > sms * 16) grid = sms * 16;
  k_flux<<<grid, 256, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double *partials, int nparts, int n_z, int n_k, int n_fft, mk_stats_out *out,
                            cudaStream_t st) {
  const size_t smem = sizeof(double) * StatLayout{n_z, n_k}.size();
  cudaError_t e = cudaFuncSetAttribute(k_finalize, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_finalize<<<1, 512, smem, st>>>(partials, nparts, n_z, n_k, n_fft, out);
  return cudaGetLastError();
}

}  // namespace mk
