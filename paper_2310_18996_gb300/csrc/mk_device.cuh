// Device building blocks of the skewer-synthesis kernels (sm_103a).
//
// A "team" of T = N/8 threads owns one segment of N pixels of one skewer:
// thread t holds pixels t + T i, i = 0..7, in registers, and the team shares
// one buffer of N/2 + 1 complex values in shared memory for the FFTs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mk_params.h"

namespace mk {

// ------------------------------------------------------------------ errors
__device__ __forceinline__ void raise_error(int *err, int bit) { atomicOr(err, bit); }

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror & Shaw, SC'11: ten rounds of (hi, lo) = M * x on
// words 0 and 2, xor with words 1, 3 and the round key; the key advances by
// the Weyl constants between rounds.
struct u32x4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox4x32_10(u32x4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = u32x4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// ln(u) for u = (x + 1/2) 2^-32 without losing the small distance to 1:
// the upper half of the range goes through log1p of the complement.
__device__ __forceinline__ float log_uniform(uint32_t x) {
  if (x & 0x80000000u) {
    const float d = (__uint2float_rn(~x) + 0.5f) * 0x1p-32f;
    return log1pf(-d);
  }
  return logf((__uint2float_rn(x) + 0.5f) * 0x1p-32f);
}

// (cos, sin)(2 pi u), u = (x + 1/2) 2^-32: the angle is taken in (-pi, pi)
// and both outputs negated, cos(phi + pi) = -cos(phi).
__device__ __forceinline__ float2 unit_phase(uint32_t x) {
  const float phi =
      (static_cast<float>(static_cast<int32_t>(x ^ 0x80000000u)) + 0.5f) * 1.4629180792671596e-09f;
  float s, c;
  __sincosf(phi, &s, &c);
  return make_float2(-c, -s);
}

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by +i (SIGN > 0) or -i (SIGN < 0)
template <int SIGN>
__device__ __forceinline__ float2 cmul_i(float2 a) {
  return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------------------ team barrier
template <int T>
__device__ __forceinline__ void team_sync(int team) {
  if constexpr (T == 32) {
    __syncwarp();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(T) : "memory");
  }
}

// ------------------------------------------------------------------ FFT plan
template <int N>
struct Fft {
  static constexpr int M = N / 2;  // complex points
  static constexpr int T = N / 8;  // threads per team (M/4)
  static constexpr int LOGM = (M == 128) ? 7 : (M == 256) ? 8 : (M == 512) ? 9 : 10;
  static constexpr int P4 = LOGM / 2;        // radix-4 passes
  static constexpr bool R2 = (LOGM & 1) != 0;  // one radix-2 pass at the end
  static_assert(N == 256 || N == 512 || N == 1024 || N == 2048, "unsupported N");
};

// Per-thread twiddles, fixed for the kernel's lifetime (the thread's
// butterfly index does not change between segments).  Stored for the
// forward sign e^{-i...}; the inverse uses conjugates.
template <int N>
struct Twiddles {
  float2 w4[Fft<N>::P4][3];  // radix-4 pass p, r = 1..3
  float2 w2[2];              // radix-2 pass, butterflies t and t + T
  float2 wu[4];              // e^{-2 pi i k/N}, k = t + r T (real-FFT untangle)
};

// tw[k] = e^{-2 pi i k/N}, k < N (FP64-rounded table in global memory)
template <int N>
__device__ __forceinline__ void load_twiddles(Twiddles<N> &tw, const float2 *__restrict__ tab, int t) {
  constexpr int T = Fft<N>::T;
  int ns = 1;
#pragma unroll
  for (int p = 0; p < Fft<N>::P4; ++p) {
    const int jm = t % ns;
#pragma unroll
    for (int r = 1; r < 4; ++r) tw.w4[p][r - 1] = tab[(r * jm * (N / (4 * ns))) % N];
    ns *= 4;
  }
  if constexpr (Fft<N>::R2) {
    // Ns = M/2: angle 2 pi (j mod Ns)/M -> index 2 (j mod Ns)
    tw.w2[0] = tab[(2 * (t % ns)) % N];
    tw.w2[1] = tab[(2 * ((t + T) % ns)) % N];
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) tw.wu[r] = tab[t + r * T];
}

template <int SIGN>
__device__ __forceinline__ void dft4(float2 &v0, float2 &v1, float2 &v2, float2 &v3) {
  const float2 a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = cmul_i<SIGN>(csub(v1, v3));
  v0 = cadd(a, c);
  v2 = csub(a, c);
  v1 = cadd(b, d);
  v3 = csub(b, d);
}

// Stockham passes 1.. on buf (pass 0 already applied by the caller, whose
// outputs sit in v[] for butterfly j = t).  SIGN = -1 forward, +1 inverse.
// On return buf holds the transform in natural order.
template <int N, int SIGN>
__device__ __forceinline__ void fft_finish(float2 *buf, float2 (&v)[4], const Twiddles<N> &tw, int t,
                                           int team) {
  constexpr int T = Fft<N>::T;
  constexpr int M = Fft<N>::M;
  // pass 0 (Ns = 1): outputs at 4 t + r
  team_sync<T>(team);
#pragma unroll
  for (int r = 0; r < 4; ++r) buf[4 * t + r] = v[r];
  int ns = 4;
#pragma unroll
  for (int p = 1; p < Fft<N>::P4; ++p) {
    team_sync<T>(team);
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = buf[t + r * T];
#pragma unroll
    for (int r = 1; r < 4; ++r) v[r] = cmul(v[r], SIGN < 0 ? tw.w4[p][r - 1] : cconj(tw.w4[p][r - 1]));
    dft4<SIGN>(v[0], v[1], v[2], v[3]);
    const int jm = t % ns;
    const int base = (t / ns) * ns * 4 + jm;
    team_sync<T>(team);
#pragma unroll
    for (int r = 0; r < 4; ++r) buf[base + r * ns] = v[r];
    ns *= 4;
  }
  if constexpr (Fft<N>::R2) {
    team_sync<T>(team);
    float2 a0 = buf[t], b0 = buf[t + M / 2], a1 = buf[t + T], b1 = buf[t + T + M / 2];
    b0 = cmul(b0, SIGN < 0 ? tw.w2[0] : cconj(tw.w2[0]));
    b1 = cmul(b1, SIGN < 0 ? tw.w2[1] : cconj(tw.w2[1]));
    team_sync<T>(team);
    buf[t] = cadd(a0, b0);
    buf[t + M / 2] = csub(a0, b0);
    buf[t + T] = cadd(a1, b1);
    buf[t + T + M / 2] = csub(a1, b1);
  }
  team_sync<T>(team);
}

// Inverse real FFT of the Hermitian modes Y_0..Y_M held in buf (already
// scaled by 1/N); on return the float view of buf holds the N real outputs
// in pixel order.
template <int N>
__device__ __forceinline__ void inverse_real_fft(float2 *buf, const Twiddles<N> &tw, int t, int team) {
  constexpr int T = Fft<N>::T;
  constexpr int M = Fft<N>::M;
  float2 v[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int k = t + r * T;
    const float2 yk = buf[k];
    const float2 ym = cconj(buf[M - k]);
    // Z_k = (Y_k + conj Y_{M-k}) + i (Y_k - conj Y_{M-k}) e^{+2 pi i k/N}
    v[r] = cadd(cadd(yk, ym), cmul_i<1>(cmul(csub(yk, ym), cconj(tw.wu[r]))));
  }
  dft4<1>(v[0], v[1], v[2], v[3]);  // pass 0: Ns = 1, no twiddle
  fft_finish<N, 1>(buf, v, tw, t, team);
}

// Forward complex FFT of the N real values in the float view of buf
// (z_n = x_{2n} + i x_{2n+1}); on return buf holds Z_0..Z_{M-1}.
template <int N>
__device__ __forceinline__ void forward_packed_fft(float2 *buf, const Twiddles<N> &tw, int t, int team) {
  constexpr int T = Fft<N>::T;
  float2 v[4];
  team_sync<T>(team);
#pragma unroll
  for (int r = 0; r < 4; ++r) v[r] = buf[t + r * T];
  dft4<-1>(v[0], v[1], v[2], v[3]);
  fft_finish<N, -1>(buf, v, tw, t, team);
}

// |X_k|^2 of the real input for k = 4t+1 .. 4t+4 after forward_packed_fft:
// X_k = E_k + e^{-2 pi i k/N} O_k with E = (Z_k + conj Z_{M-k})/2,
// O = (Z_k - conj Z_{M-k})/(2i); Z_M = Z_0.
template <int N>
__device__ __forceinline__ void power_of_modes(const float2 *buf, const float2 *__restrict__ tab, int t,
                                               float (&pk)[4]) {
  constexpr int M = Fft<N>::M;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int k = 4 * t + 1 + r;
    const float2 zk = buf[k & (M - 1)];
    const float2 zm = cconj(buf[(M - k) & (M - 1)]);
    const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
    const float2 dd = csub(zk, zm);
    const float2 o = make_float2(0.5f * dd.y, -0.5f * dd.x);  // (Z - conj Z')/(2i)
    const float2 w = tab[k & (N - 1)];                          // e^{-2 pi i k/N}
    const float2 x = cadd(e, cmul(w, o));
    pk[r] = fmaf(x.x, x.x, x.y * x.y);
  }
}

// ------------------------------------------------------------------ small-scale modes
// Writes Y_m = X_m/N for m = 0..M into buf (Philox words -> Box-Muller).
template <int N>
__device__ __forceinline__ void small_scale_modes(float2 *buf, const float *__restrict__ amp, uint32_t seg,
                                                  uint64_t id, uint32_t seed, int t) {
  constexpr int T = Fft<N>::T;
  constexpr int M = Fft<N>::M;
  const uint32_t id_lo = static_cast<uint32_t>(id), id_hi = static_cast<uint32_t>(id >> 32);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const uint32_t c = t + q * T;  // modes 2c, 2c+1 (< M)
    const u32x4 w = philox4x32_10(u32x4{c, seg, id_hi, 0u}, seed, id_lo);
    const int m0 = 2 * c, m1 = 2 * c + 1;
    const float2 p0 = unit_phase(w.y), p1 = unit_phase(w.w);
    const float r0 = sqrtf(-log_uniform(w.x)), r1 = sqrtf(-log_uniform(w.z));
    const float a0 = amp[m0] * r0, a1 = amp[m1] * r1;
    buf[m0] = (m0 == 0) ? make_float2(0.f, 0.f) : make_float2(a0 * p0.x, a0 * p0.y);
    buf[m1] = make_float2(a1 * p1.x, a1 * p1.y);
  }
  if (t == 0) {  // Nyquist mode m = M from counter M/2, words (0, 1): real A e1
    const u32x4 w = philox4x32_10(u32x4{static_cast<uint32_t>(M / 2), seg, id_hi, 0u}, seed, id_lo);
    const float e1 = sqrtf(-2.0f * log_uniform(w.x)) * unit_phase(w.y).x;
    buf[M] = make_float2(amp[M] * e1, 0.f);
  }
}

// ------------------------------------------------------------------ fixed-point gather
// Q20.44 cell coordinate (minus 1/2) -> base cell index and weight in [0, 1].
__device__ __forceinline__ void split_coord(int64_t p, int mask, int &i0, int &i1, float &t) {
  const int base = static_cast<int>(p >> 44);
  i0 = base & mask;
  i1 = (base + 1) & mask;
  t = __uint2float_rn(static_cast<uint32_t>(static_cast<uint64_t>(p) >> 12)) * 0x1p-32f;
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Trilinear (delta, eta) at fixed-point coordinate (px, py, pz).
template <int LAYOUT>
__device__ __forceinline__ float2 gather(const float *__restrict__ d, const float *__restrict__ e, int lgn,
                                         int64_t px, int64_t py, int64_t pz) {
  const int mask = (1 << lgn) - 1;
  int x0, x1, y0, y1, z0, z1;
  float tx, ty, tz;
  split_coord(px, mask, x0, x1, tx);
  split_coord(py, mask, y0, y1, ty);
  split_coord(pz, mask, z0, z1, tz);
  // row index (z n + y) n in 64 bits: boxes up to 2048^3 cells
  const size_t r00 = static_cast<size_t>((static_cast<uint32_t>(z0) << lgn) | static_cast<uint32_t>(y0)) << lgn;
  const size_t r10 = static_cast<size_t>((static_cast<uint32_t>(z0) << lgn) | static_cast<uint32_t>(y1)) << lgn;
  const size_t r01 = static_cast<size_t>((static_cast<uint32_t>(z1) << lgn) | static_cast<uint32_t>(y0)) << lgn;
  const size_t r11 = static_cast<size_t>((static_cast<uint32_t>(z1) << lgn) | static_cast<uint32_t>(y1)) << lgn;
  float2 v[8];
  if constexpr (LAYOUT == MK_BOX_INTERLEAVED) {
    const float2 *b = reinterpret_cast<const float2 *>(d);
    v[0] = __ldg(b + r00 + x0); v[1] = __ldg(b + r00 + x1);
    v[2] = __ldg(b + r10 + x0); v[3] = __ldg(b + r10 + x1);
    v[4] = __ldg(b + r01 + x0); v[5] = __ldg(b + r01 + x1);
    v[6] = __ldg(b + r11 + x0); v[7] = __ldg(b + r11 + x1);
  } else {
    const size_t idx[8] = {r00 + x0, r00 + x1, r10 + x0, r10 + x1, r01 + x0, r01 + x1, r11 + x0, r11 + x1};
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = make_float2(__ldg(d + idx[k]), __ldg(e + idx[k]));
  }
  float2 out;
  {
    const float a = lerpf(v[0].x, v[1].x, tx), b = lerpf(v[2].x, v[3].x, tx);
    const float c = lerpf(v[4].x, v[5].x, tx), dd = lerpf(v[6].x, v[7].x, tx);
    out.x = lerpf(lerpf(a, b, ty), lerpf(c, dd, ty), tz);
  }
  {
    const float a = lerpf(v[0].y, v[1].y, tx), b = lerpf(v[2].y, v[3].y, tx);
    const float c = lerpf(v[4].y, v[5].y, tx), dd = lerpf(v[6].y, v[7].y, tx);
    out.y = lerpf(lerpf(a, b, ty), lerpf(c, dd, ty), tz);
  }
  return out;
}

// ------------------------------------------------------------------ FGPA
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// tab = {G, a log2 e, b log2 e, c}:  F = 2^(-a' 2^(b' (delta + c eta)))
__device__ __forceinline__ float fgpa(float4 tab, float delta, float eta) {
  return ex2_approx(-tab.y * ex2_approx(tab.z * fmaf(tab.w, eta, delta)));
}

// ------------------------------------------------------------------ statistics
// Team-wide sum of v[NSUM]; the result is valid in thread t == 0.
template <int T>
__device__ __forceinline__ void team_reduce(float (&v)[MK_NSUM], float *red, int t, int team) {
#pragma unroll
  for (int i = 0; i < MK_NSUM; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  if constexpr (T > 32) {
    const int wid = t >> 5;
    if ((t & 31) == 0) {
#pragma unroll
      for (int i = 0; i < MK_NSUM; ++i) red[wid * MK_NSUM + i] = v[i];
    }
    team_sync<T>(team);
    if (t == 0) {
#pragma unroll
      for (int i = 0; i < MK_NSUM; ++i) {
        float s = red[i];
        for (int w = 1; w < T / 32; ++w) s += red[w * MK_NSUM + i];
        v[i] = s;
      }
    }
    team_sync<T>(team);
  }
}

// Pixel statistics of the team's 8 pixels per thread.  zb[i] is the
// pixel's z bin (-1 below the range, n_z above, also for invalid pixels).
template <int T>
__device__ __forceinline__ void accumulate_pixels(double *acc, const StatLayout &L, const float (&f)[8],
                                                  const float (&d)[8], const float (&e)[8],
                                                  const int (&zb)[8], int zb_first, int zb_last, float *red,
                                                  int t, int team) {
  if (zb_first < 0) zb_first = 0;
  if (zb_last > L.n_z - 1) zb_last = L.n_z - 1;
  for (int b = zb_first; b <= zb_last; ++b) {
    float v[MK_NSUM];
#pragma unroll
    for (int i = 0; i < MK_NSUM; ++i) v[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      if (zb[i] == b) {
        v[0] += 1.f;
        v[1] += f[i];
        v[2] = fmaf(f[i], f[i], v[2]);
        v[3] += d[i];
        v[4] += e[i];
        v[5] = fmaf(d[i], d[i], v[5]);
        v[6] = fmaf(e[i], e[i], v[6]);
        v[7] = fmaf(d[i], e[i], v[7]);
        v[8] = fmaf(f[i], d[i], v[8]);
        v[9] = fmaf(f[i], e[i], v[9]);
      }
    }
    team_reduce<T>(v, red, t, team);
    if (t == 0) {
#pragma unroll
      for (int i = 0; i < MK_NSUM; ++i) acc[L.sums(b, i)] += static_cast<double>(v[i]);
    }
  }
}

// Add the 4 mode powers of thread t (modes 4t+1..4t+4) to the P1D bins of z bin zb.
template <int N>
__device__ __forceinline__ void accumulate_p1d(double *acc, const StatLayout &L, const float (&pk)[4],
                                               float scale, int zb, int t) {
  constexpr int M = Fft<N>::M;
  const int per_bin = M / L.n_k;  // modes per k bin
  if (per_bin >= 4) {
    float s = (pk[0] + pk[1]) + (pk[2] + pk[3]);
    const int group = per_bin / 4;  // threads sharing a bin (power of two <= 32)
    for (int o = 1; o < group && o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (group > 32) {
      // only when n_k is tiny; fall back to one add per warp leader
      if ((t & 31) == 0) atomicAdd(&acc[L.p1d(zb, (4 * t) / per_bin)], static_cast<double>(s * scale));
    } else if ((t & (group - 1)) == 0) {
      acc[L.p1d(zb, (4 * t) / per_bin)] += static_cast<double>(s * scale);
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int k = 4 * t + r;  // mode k+1, bin (k * n_k)/M
      atomicAdd(&acc[L.p1d(zb, (k * L.n_k) / M)], static_cast<double>(pk[r] * scale));
    }
  }
  if (t == 0) acc[L.nseg(zb)] += 1.0;
}

}  // namespace mk
