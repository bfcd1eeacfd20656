// Templates of the fused skewer kernel and the statistics kernel; each FFT
// length is instantiated in its own translation unit (mk_skewer_<N>.cu).
#pragma once

#include "mk_device.cuh"

namespace mk {

// =================================================================== shared-memory plan
// Per CTA: per-warp statistic accumulators (when statistics are on), the
// twiddle table, then one FFT buffer of N/2 + 2 complex values per team.
template <int N>
struct TeamSmem {
  static constexpr int T = N / 8;
  static constexpr int BUF = N == 256 ? kBuf256 : N / 2 + 2;  // complex slots per team buffer
  __host__ __device__ static size_t acc_bytes(int threads, int n_z, int n_k, bool stats) {
    return stats ? static_cast<size_t>(threads / 32) * WarpAcc::bytes(n_z, n_k) : 0;
  }
  __host__ __device__ static size_t bytes(int threads, int n_z, int n_k, bool stats) {
    return acc_bytes(threads, n_z, n_k, stats) + TwTab<N>::BYTES +
           static_cast<size_t>(threads / T) * BUF * sizeof(float2);
  }
};

// largest i with a[i] <= v over a[0..n] (a non-decreasing)
__device__ __forceinline__ int64_t upper_index(const int64_t *a, int64_t n, int64_t v) {
  int64_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void zero_warp_acc(unsigned char *base, size_t wbytes) {
  float *f = reinterpret_cast<float *>(base);
  for (size_t i = threadIdx.x & 31; i < wbytes / sizeof(float); i += 32) f[i] = 0.f;
  __syncwarp();
}

// Sum the warps' compensated FP32 accumulators in FP64 and write this CTA's
// partials in the StatLayout order.
__device__ __forceinline__ void flush_warp_partials(unsigned char *smem, int nwarps, size_t wbytes, int n_z, int n_k,
                                    double *partials) {
  __syncthreads();
  const StatLayout L{n_z, n_k};
  const int ns = n_z * MK_NSUM, np = n_z * n_k;
  for (int idx = threadIdx.x; idx < L.size(); idx += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < nwarps; ++w) {
      const WarpAcc A = WarpAcc::at(smem + w * wbytes, n_z, n_k);
      if (idx < ns) {
        const float2 v = A.sums[idx];
        s += static_cast<double>(v.x) - static_cast<double>(v.y);
      } else if (idx < ns + np) {
        const float2 v = A.p1d[idx - ns];
        s += static_cast<double>(v.x) - static_cast<double>(v.y);
      } else {
        s += static_cast<double>(A.nseg[idx - ns - np]);
      }
    }
    partials[static_cast<size_t>(blockIdx.x) * L.size() + idx] = s;
  }
}

// =================================================================== fused skewer kernel
// One team per segment of N pixels: small-scale modes -> inverse real FFT ->
// per pixel gather, growth, FGPA, stores and pixel sums -> forward FFT of the
// flux -> P1D.  Teams take contiguous ranges of segments (all segments cost
// the same).  Pixel sums stay in registers, across segments, for as long as
// the warp's pixels stay in one z bin: the warp flushes them to its shared
// accumulators when its pixels reach the end of the bin (bin_end) or a
// segment starts in another bin.
// INTERP: MK_INTERP_TRILINEAR, or MK_INTERP_GAUSS7 (LAYOUT must be MK_BOX_HALO).
// PSZ: P_s given at several redshifts (P.ps_nodes >= 2), interpolated per segment
// FIXLGN > 0: a padded box of side 2^FIXLGN (constant strides in the gather)
template <int N, int LAYOUT, bool BIG, int MINB, int INTERP = MK_INTERP_TRILINEAR, bool PSZ = false, int FIXLGN = 0>
__global__ void __launch_bounds__(256, MINB) k_skewer(SkewerParams P) {
  constexpr int T = N / 8;
  constexpr int BUF = TeamSmem<N>::BUF;
  const int teams = blockDim.x / T;
  const int team = threadIdx.x / T, t = threadIdx.x % T, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int wlo0 = t & ~31;  // first team pixel of this warp
  const int nwarps = blockDim.x >> 5;
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t wbytes = P.do_stats ? WarpAcc::bytes(P.n_z, P.n_k) : 0;
  float2 *tws = reinterpret_cast<float2 *>(smem + nwarps * wbytes);
  float2 *buf = tws + TwTab<N>::SLOTS * T + team * BUF;
  float *fb = reinterpret_cast<float *>(buf);
  const WarpAcc W = WarpAcc::at(smem + warp * wbytes, P.n_z, P.n_k);
  if (P.do_stats) zero_warp_acc(smem + warp * wbytes, wbytes);
  fill_twiddles<N>(tws, P.tw);

  // segments segoff[0] .. segoff[n_sk] (a slice of a larger catalogue may
  // start at segoff[0] > 0)
  const int64_t u0 = P.segoff[0], nunits = P.segoff[P.n_sk] - u0;
  const int64_t g = static_cast<int64_t>(blockIdx.x) * teams + team;
  const int64_t G = static_cast<int64_t>(gridDim.x) * teams;
  int64_t u = u0 + g * nunits / G;
  const int64_t uend = u0 + (g + 1) * nunits / G;
  int64_t i = u < uend ? upper_index(P.segoff, P.n_sk, u) : 0;

  PixelSums acc;
  acc.zero();
  int zc = -2;  // z bin of acc (warp-uniform), -2 before the first segment

  for (; u < uend; ++u) {
    while (P.segoff[i + 1] <= u) ++i;
    const int s = static_cast<int>(u - P.segoff[i]);
    const mk_skewer sk = P.sk[i];
    const int64_t j0 = static_cast<int64_t>(s) * N;
    const int npx = static_cast<int>(min(static_cast<int64_t>(N), sk.n - j0));
    if ((P.delta_out || P.flux_out) && sk.offset + sk.n > P.capacity) {
      if (t == 0) raise_error(P.err, ERR_CAPACITY);
      continue;
    }
    // ---- start the box rows of this segment's stencils on their way to L2:
    // lane t samples pixel 8t + 4 (the modes and the inverse FFT below hide
    // the latency)
    {
      const int64_t ps = j0 + min(npx - 1, 8 * t + 4);
      prefetch_stencil<LAYOUT, BIG>(P.box_d, P.lgn, sk.p0[0] + kRoundQ + ps * sk.step[0],
                                    sk.p0[1] + kRoundQ + ps * sk.step[1], sk.p0[2] + kRoundQ + ps * sk.step[2]);
    }
    // ---- small-scale field of this segment
    if constexpr (PSZ) {  // P_s at the mean z of the segment's window, linear between nodes
      const float zw = __ldg(P.zwin + sk.j_lo + static_cast<int>(j0));
      const int k = P.ps_nodes;
      int n0 = 0;
      while (n0 + 2 < k && zw >= P.ps_z[n0 + 1]) ++n0;
      const float w_hi = fminf(fmaxf((zw - P.ps_z[n0]) / (P.ps_z[n0 + 1] - P.ps_z[n0]), 0.f), 1.f);
      const float *amp = P.amp + n0 * (N / 2 + 1);
      small_scale_modes<N, true>(buf, amp, amp + (N / 2 + 1), w_hi, static_cast<uint32_t>(s), sk.id, P.seed, t);
    } else {
      small_scale_modes<N, false>(buf, P.amp, nullptr, 0.f, static_cast<uint32_t>(s), sk.id, P.seed, t);
    }
    team_sync<T>(team);
    inverse_real_fft<N>(buf, tws, t, team);

    // ---- per pixel: gather, growth, FGPA, stores, pixel sums
    const int jb = sk.j_lo + static_cast<int>(j0);
    int pend = 0;  // segment pixel where bin zc ends
    if (P.do_stats) {
      const int zs = __ldg(P.zbin + jb);
      if (zs != zc) {
        if (zc != -2) flush_bin_sums(W, P.n_z, zc, acc, lane);
        acc.zero();
        zc = zs;
      }
      pend = __ldg(P.bin_end + zc + 1) - jb;
    }
    // sight-line weights of the velocity-gradient tensor (Eq. eta)
    float uu[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if constexpr (LAYOUT == MK_BOX_TENSOR) {
      const float ux = static_cast<float>(sk.step[0]), uy = static_cast<float>(sk.step[1]),
                  uz = static_cast<float>(sk.step[2]);
      const float inv = rsqrtf(ux * ux + uy * uy + uz * uz);
      const float vx = ux * inv, vy = uy * inv, vz = uz * inv;
      uu[0] = vx * vx;
      uu[1] = vy * vy;
      uu[2] = vz * vz;
      uu[3] = 2.f * vx * vy;
      uu[4] = 2.f * vx * vz;
      uu[5] = 2.f * vy * vz;
    }
    int64_t px = sk.p0[0] + kRoundQ + (j0 + t) * sk.step[0];
    int64_t py = sk.p0[1] + kRoundQ + (j0 + t) * sk.step[1];
    int64_t pz = sk.p0[2] + kRoundQ + (j0 + t) * sk.step[2];
    const int64_t sx = T * sk.step[0], sy = T * sk.step[1], sz = T * sk.step[2];
    const int64_t out0 = sk.offset + j0;
    // warp-uniform: this warp's pixels of the segment all lie before pend
    const bool one_bin = min(T * 7 + wlo0 + 32, npx) <= pend;
    // pixel p: gather, growth, small-scale field, FGPA, stores; returns F
    auto synth = [&](int p, float2 &x) -> float {
      float2 de;
      if constexpr (INTERP == MK_INTERP_GAUSS7) {
        static_assert(LAYOUT == MK_BOX_HALO, "the Gaussian kernel reads a halo box");
        de = gather_gauss7<BIG>(P.box_d, P.lgn, px, py, pz);
      } else if constexpr (LAYOUT == MK_BOX_TENSOR) {
        de = gather_tensor<BIG>(P.box_d, P.lgn, px, py, pz, uu);
      } else {
        de = gather<LAYOUT, BIG, FIXLGN>(P.box_d, P.box_e, P.lgn, px, py, pz);
      }
      const float4 tb = __ldg(P.pixtab + jb + p);
      x = make_float2(fmaf(tb.x, de.x, fb[p]), tb.x * de.y);
      const float f = fgpa(tb, x.x, x.y);
      if (P.delta_out) {
        P.delta_out[out0 + p] = x.x;
        P.eta_out[out0 + p] = x.y;
      }
      if (P.flux_out) P.flux_out[out0 + p] = f;
      return f;
    };
    // (the tensor and Gaussian-kernel gathers keep one loop: their registers
    // do not leave room for a second copy)
    constexpr bool kLean = LAYOUT != MK_BOX_TENSOR && INTERP == MK_INTERP_TRILINEAR;
    if (kLean && npx == N && (!P.do_stats || one_bin)) {
      // a full segment inside one z bin (most segments): no per-pixel bounds or bin checks
#pragma unroll 2
      for (int k = 0; k < 8; ++k) {
        const int p = t + T * k;
        float2 x;
        const float f = synth(p, x);
        if (P.do_stats) acc.add_sums(f, x);
        fb[p] = f;
        px += sx;
        py += sy;
        pz += sz;
      }
      acc.n += 8.f;  // this thread's pixels of the segment
    } else {
#pragma unroll 2
    for (int k = 0; k < 8; ++k) {
      const int p = t + T * k;
      float f = 0.f;
      float2 x = make_float2(0.f, 0.f);
      if (p < npx) f = synth(p, x);
      if (P.do_stats && one_bin) {
        if (p < npx) acc.add(f, x);
      } else if (P.do_stats) {
        // this warp's pixels at k: T k + wlo0 + lane; flush while they pass pend
        const int hi = min(T * k + wlo0 + 32, npx);
        bool todo = p < npx;
        while (hi > pend) {
          if (todo && p < pend) {
            acc.add(f, x);
            todo = false;
          }
          flush_bin_sums(W, P.n_z, zc, acc, lane);
          acc.zero();
          ++zc;
          pend = __ldg(P.bin_end + zc + 1) - jb;
        }
        if (todo) acc.add(f, x);
      }
      fb[p] = f;
      px += sx;
      py += sy;
      pz += sz;
    }
    }

    // ---- P1D of the segment
    if (P.do_stats && npx == N) {
      const int zs = __ldg(P.segzbin + jb);
      if (zs >= 0 && zs < P.n_z) {
        forward_packed_fft<N>(buf, tws, t, team);
        float pk[4];
        power_of_modes<N>(buf, P.tw, t, pk);
        accumulate_p1d<N>(W, P.n_k, pk, P.p1d_scale, zs, t);
        if (t == 0) W.nseg[zs] += 1u;
      }
    }
    team_sync<T>(team);
  }
  if (P.do_stats) {
    if (zc != -2) flush_bin_sums(W, P.n_z, zc, acc, lane);
    flush_warp_partials(smem, nwarps, wbytes, P.n_z, P.n_k, P.partials);
  }
}

// =================================================================== statistics kernel
template <int N>
__global__ void __launch_bounds__(256, 2) k_stats(StatParams P) {
  constexpr int T = N / 8;
  constexpr int BUF = TeamSmem<N>::BUF;
  const int teams = blockDim.x / T;
  const int team = threadIdx.x / T, t = threadIdx.x % T, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t wbytes = WarpAcc::bytes(P.n_z, P.n_k);
  float2 *tws = reinterpret_cast<float2 *>(smem + nwarps * wbytes);
  float2 *buf = tws + TwTab<N>::SLOTS * T + team * BUF;
  float *fb = reinterpret_cast<float *>(buf);
  const WarpAcc W = WarpAcc::at(smem + warp * wbytes, P.n_z, P.n_k);
  zero_warp_acc(smem + warp * wbytes, wbytes);
  fill_twiddles<N>(tws, P.tw);

  const int64_t nunits = P.segoff[P.n_sk];
  const int64_t g = static_cast<int64_t>(blockIdx.x) * teams + team;
  const int64_t G = static_cast<int64_t>(gridDim.x) * teams;
  int64_t u = g * nunits / G;
  const int64_t uend = (g + 1) * nunits / G;
  int64_t i = u < uend ? upper_index(P.segoff, P.n_sk, u) : 0;
  const int R = P.rebin;
  const int wlo0 = t & ~31;  // first team pixel of this warp
  // R = 1: pixel sums in registers across segments while the warp's pixels
  // stay in one z bin, flushed at the bin's end (as in k_skewer)
  PixelSums acc;
  acc.zero();
  int zc = -2;
  team_sync<T>(team);

  for (; u < uend; ++u) {
    while (P.segoff[i + 1] <= u) ++i;
    const int s = static_cast<int>(u - P.segoff[i]);
    const mk_skewer sk = P.sk[i];
    const int64_t o = P.off_out[i];
    const int64_t nout = P.off_out[i + 1] - o;
    // records made for another pixel length may run past the pixel tables
    // (team-uniform: the whole team skips the segment)
    if (sk.j_lo < 0 || sk.j_lo + nout * R > P.j_max) {
      if (t == 0) raise_error(P.err, ERR_RANGE);
      continue;
    }
    const int64_t k0 = static_cast<int64_t>(s) * N;
    const int npx = static_cast<int>(min(static_cast<int64_t>(N), nout - k0));
    auto zbin_of = [&](int64_t kk) -> int {
      const int64_t J = sk.j_lo + kk * R;
      if (R == 1) return __ldg(P.zbin + J);
      const double fz = floor(((P.cumz[J + R] - P.cumz[J]) / R - P.z_lo) / P.dz);
      return fz < 0.0 ? -1 : (fz >= P.n_z ? P.n_z : static_cast<int>(fz));
    };
    if (R == 1) {
      const int jb = sk.j_lo + static_cast<int>(k0);
      const int zs = __ldg(P.zbin + jb);
      if (zs != zc) {
        if (zc != -2) flush_bin_sums(W, P.n_z, zc, acc, lane);
        acc.zero();
        zc = zs;
      }
      int pend = __ldg(P.bin_end + zc + 1) - jb;  // segment pixel where bin zc ends
      // warp-uniform: this warp's pixels of the segment all lie before pend
      const bool one_bin = min(T * 7 + wlo0 + 32, npx) <= pend;
      if (npx == N && one_bin && P.pixtab) {
        // tuning pass over a full segment inside one z bin: no bounds or bin checks
        const float *dp = P.delta + sk.offset + k0 + t, *ep = P.eta + sk.offset + k0 + t;
        const float4 *tp = P.pixtab + sk.j_lo + k0 + t;
        float dv[8], ev[8];
        float4 tb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          dv[q] = __ldg(dp + T * q);
          ev[q] = __ldg(ep + T * q);
          tb[q] = __ldg(tp + T * q);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float f = fgpa(tb[q], dv[q], ev[q]);
          acc.add_sums(f, make_float2(dv[q], ev[q]));
          fb[t + T * q] = f;
        }
        acc.n += 8.f;
      } else {
      // streaming case: issue every load of the thread's 8 pixels before any use
      float dv[8], ev[8], fv[8];
      float4 tb[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int p = t + T * q;
        const bool ok = p < npx;
        const int64_t kk = k0 + (ok ? p : 0);
        dv[q] = (ok && P.delta) ? __ldg(P.delta + sk.offset + kk) : 0.f;
        ev[q] = (ok && P.delta) ? __ldg(P.eta + sk.offset + kk) : 0.f;
        if (P.pixtab) {
          tb[q] = __ldg(P.pixtab + sk.j_lo + kk);
          fv[q] = 0.f;
        } else {
          fv[q] = ok ? __ldg(P.flux + o + kk) : 0.f;
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int p = t + T * q;
        float f = 0.f;
        if (p < npx) f = P.pixtab ? fgpa(tb[q], dv[q], ev[q]) : fv[q];
        const float2 x = make_float2(dv[q], ev[q]);
        if (one_bin) {
          if (p < npx) acc.add(f, x);
        } else {
          // this warp's pixels at q: T q + wlo0 + lane; flush while they pass pend
          const int hi = min(T * q + wlo0 + 32, npx);
          bool todo = p < npx;
          while (hi > pend) {
            if (todo && p < pend) {
              acc.add(f, x);
              todo = false;
            }
            flush_bin_sums(W, P.n_z, zc, acc, lane);
            acc.zero();
            ++zc;
            pend = __ldg(P.bin_end + zc + 1) - jb;
          }
          if (todo) acc.add(f, x);
        }
        fb[p] = f;
      }
      }
    } else {
      const int zf = zbin_of(k0), zl = zbin_of(k0 + npx - 1);
      float a0[MK_NSUM], a1[MK_NSUM];
#pragma unroll
      for (int q = 0; q < MK_NSUM; ++q) a0[q] = a1[q] = 0.f;
#pragma unroll 2
      for (int q = 0; q < 8; ++q) {
        const int p = t + T * q;
        float f = 0.f;
        if (p < npx) {
          const int64_t kk = k0 + p;
          float ds = 0.f, es = 0.f;
          if (P.delta) {
            for (int r = 0; r < R; ++r) {
              ds += P.delta[sk.offset + kk * R + r];
              es += P.eta[sk.offset + kk * R + r];
            }
            ds /= static_cast<float>(R);
            es /= static_cast<float>(R);
          }
          f = P.flux[o + kk];
          const int zb = zbin_of(kk);
          if (zb == zf) add_pixel(a0, f, ds, es);
          else if (zb == zf + 1) add_pixel(a1, f, ds, es);
          else if (zb >= 0 && zb < P.n_z) add_pixel_slow(W, zb, f, ds, es);
        }
        fb[p] = f;
      }
      flush_pixel_sums(W, P.n_z, zf, zl > zf, a0, a1, lane);
    }
    if (npx == N) {
      int zs;
      if (R == 1) {
        zs = __ldg(P.segzbin + sk.j_lo + k0);
      } else {
        const int64_t J0 = sk.j_lo + k0 * R;
        const double zm =
            (P.cumz[J0 + static_cast<int64_t>(N) * R] - P.cumz[J0]) / (static_cast<double>(N) * R);
        const double fz = floor((zm - P.z_lo) / P.dz);
        zs = fz < 0.0 ? -1 : (fz >= P.n_z ? P.n_z : static_cast<int>(fz));
      }
      if (zs >= 0 && zs < P.n_z) {
        forward_packed_fft<N>(buf, tws, t, team);
        float pk[4];
        power_of_modes<N>(buf, P.tw, t, pk);
        accumulate_p1d<N>(W, P.n_k, pk, P.p1d_scale, zs, t);
        if (t == 0) W.nseg[zs] += 1u;
      }
    }
    team_sync<T>(team);
  }
  if (R == 1 && zc != -2) flush_bin_sums(W, P.n_z, zc, acc, lane);
  flush_warp_partials(smem, nwarps, wbytes, P.n_z, P.n_k, P.partials);
}

}  // namespace mk
