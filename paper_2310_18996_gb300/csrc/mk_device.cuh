// Device building blocks of the skewer-synthesis kernels (sm_103a).
//
// A "team" of T = N/8 threads owns one segment of N pixels of one skewer:
// thread t handles pixels t + T k, k = 0..7, and the team shares one buffer
// of N/2 + 1 complex values in shared memory for the FFTs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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

__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// -ln(u) for u = (x + 1/2) 2^-32, branch-free and accurate in relative terms
// over the whole range.  Below 1/2 the SFU log2 is accurate to ~2^-22
// relative (|log2 u| >= 1).  Above, u = 1 - d with d = (~x + 1/2) 2^-32 known
// exactly, and -ln(1 - d) = 2 atanh(s), s = d/(2 - d) <= 1/3, summed from the
// Gregory series 2 (s + s^3/3 + ... + s^17/17) (truncation < 1e-10).
__device__ __forceinline__ float neg_log_uniform(uint32_t x) {
  const float u = (__uint2float_rn(x) + 0.5f) * 0x1p-32f;
  const float lo = -0.69314718055994531f * lg2_approx(u);
  const float d = (__uint2float_rn(~x) + 0.5f) * 0x1p-32f;
  const float s = __fdividef(d, 2.0f - d);
  const float s2 = s * s;
  float p = 1.0f / 17.0f;
  p = fmaf(p, s2, 1.0f / 15.0f);
  p = fmaf(p, s2, 1.0f / 13.0f);
  p = fmaf(p, s2, 1.0f / 11.0f);
  p = fmaf(p, s2, 1.0f / 9.0f);
  p = fmaf(p, s2, 1.0f / 7.0f);
  p = fmaf(p, s2, 1.0f / 5.0f);
  p = fmaf(p, s2, 1.0f / 3.0f);
  p = fmaf(p, s2, 1.0f);
  const float hi = 2.0f * s * p;
  return (x & 0x80000000u) ? hi : lo;
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

__device__ __forceinline__ float sqrt_pos(float x) { return x * rsqrtf(x); }  // x > 0

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
template <int SIGN>
__device__ __forceinline__ float2 cmul_i(float2 a) {  // times +i (SIGN > 0) or -i
  return SIGN > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// ------------------------------------------------------------------ packed FP32 pairs
// sm_100 and later execute add, sub, mul and fma on the two FP32 halves of a
// 64-bit register pair in one instruction; each half rounds exactly as the
// scalar instruction (round to nearest even, no flush to zero).
#define MK_F2_BINOP(name, op)                                                                  \
  __device__ __forceinline__ float2 name(float2 a, float2 b) {                                 \
    float2 r;                                                                                  \
    asm("{.reg .b64 a, b, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\t" op        \
        " d, a, b;\n\tmov.b64 {%0, %1}, d;}"                                                  \
        : "=f"(r.x), "=f"(r.y)                                                                 \
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                                             \
    return r;                                                                                  \
  }
MK_F2_BINOP(f2add, "add.rn.f32x2")
MK_F2_BINOP(f2sub, "sub.rn.f32x2")
MK_F2_BINOP(f2mul, "mul.rn.f32x2")
#undef MK_F2_BINOP

// a * b + c per half, one rounding
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
  float2 r;
  asm("{.reg .b64 a, b, c, d;\n\tmov.b64 a, {%2, %3};\n\tmov.b64 b, {%4, %5};\n\tmov.b64 c, {%6, %7};\n\t"
      "fma.rn.f32x2 d, a, b, c;\n\tmov.b64 {%0, %1}, d;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return r;
}

// a + t (b - a) per half, t the same for both: the scalar lerp's rounding
__device__ __forceinline__ float2 f2lerp(float2 a, float2 b, float t) {
  return f2fma(make_float2(t, t), f2sub(b, a), a);
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
  static constexpr int LOGM = (M == 128) ? 7 : (M == 256) ? 8 : (M == 512) ? 9 : (M == 1024) ? 10 : 11;
  static constexpr int P4 = LOGM / 2;          // radix-4 passes
  static constexpr bool R2 = (LOGM & 1) != 0;  // one radix-2 pass at the end
  // 4096: complex lines of 2048 (box synthesis only)
  static_assert(N == 256 || N == 512 || N == 1024 || N == 2048 || N == 4096, "unsupported N");
};

// Shared-memory swizzle of complex index i: xor the low bits with 5 times
// bits 4-5.  Every Stockham access pattern (strided reads t + r T, writes at
// base + r Ns for Ns = 1, 4, 16, ..., the mode and power reads) then hits 16
// distinct 8-byte slots per half warp.
__device__ __forceinline__ int sw(int i) { return i ^ (5 * ((i >> 4) & 3)); }

// Per-thread twiddles, one shared-memory table per CTA (its teams share it):
// slot s of team thread t at tws[s T + t], so a warp's reads of one slot are
// conflict-free.  Stored for the forward sign e^{-i...}; the inverse uses
// conjugates.
//   slots 3 (p - 1) + r - 1, p = 1 .. P4 - 1, r = 1 .. 3: radix-4 pass p
//     (pass 0 has unit twiddles), e^{-2 pi i r (t mod 4^p) / 4^(p+1)}
//   slots R2 + q, q = 0, 1: radix-2 pass, butterflies t and t + T
//   slots U + r, r = 0 .. 3: e^{-2 pi i k/N}, k = t + r T (real-FFT untangle)
template <int N>
struct TwTab {
  static constexpr int T = Fft<N>::T;
  static constexpr int R2 = 3 * (Fft<N>::P4 - 1);
  static constexpr int U = R2 + 2;
  static constexpr int SLOTS = U + 4;
  static constexpr size_t BYTES = sizeof(float2) * SLOTS * T;
};

// tab[k] = e^{-2 pi i k/N}, k < N (FP64-rounded table in global memory).
// Called by every thread of the CTA; ends with a CTA barrier.
template <int N>
__device__ __forceinline__ void fill_twiddles(float2 *tws, const float2 *__restrict__ tab) {
  constexpr int T = Fft<N>::T;
  for (int i = threadIdx.x; i < TwTab<N>::SLOTS * T; i += blockDim.x) {
    const int s = i / T, t = i % T;
    int k;
    if (s < TwTab<N>::R2) {
      const int p = s / 3 + 1, r = s % 3 + 1, ns = 1 << (2 * p);
      k = (r * (t % ns) * (N / (4 * ns))) % N;
    } else if (s < TwTab<N>::U) {
      const int ns = 1 << (2 * Fft<N>::P4);
      k = (2 * ((t + (s - TwTab<N>::R2) * T) % ns)) % N;
    } else {
      k = t + (s - TwTab<N>::U) * T;
    }
    tws[i] = tab[k];
  }
  __syncthreads();
}

// 4-point DFT in place (SIGN = -1 forward, +1 inverse); the sums run on
// packed pairs, the rotated difference b +- i^SIGN e on scalars.
template <int SIGN>
__device__ __forceinline__ void dft4(float2 &v0, float2 &v1, float2 &v2, float2 &v3) {
  const float2 a = f2add(v0, v2), b = f2sub(v0, v2), c = f2add(v1, v3), e = f2sub(v1, v3);
  v0 = f2add(a, c);
  v2 = f2sub(a, c);
  const float2 d = cmul_i<SIGN>(e);
  v1 = make_float2(b.x + d.x, b.y + d.y);
  v3 = make_float2(b.x - d.x, b.y - d.y);
}

// Stockham passes after pass 0 (whose butterfly j = t outputs are in v[]).
// SIGN = -1 forward, +1 inverse.  On return buf holds the transform in
// natural order, through the swizzle, or with PLAIN at plain indices: the
// last pass writes t + r T (radix-4 ending: base t, stride T; radix-2
// ending: t, t + T, t + 2T, t + 3T), consecutive per lane, so the plain
// layout is conflict-free there.
template <int N, int SIGN, bool PLAIN = false>
__device__ __forceinline__ void fft_finish(float2 *buf, float2 (&v)[4], const float2 *tws, int t, int team) {
  constexpr int T = Fft<N>::T;
  constexpr int M = Fft<N>::M;
  team_sync<T>(team);
#pragma unroll
  for (int r = 0; r < 4; ++r) buf[sw(4 * t + r)] = v[r];
  int ns = 4;
#pragma unroll
  for (int p = 1; p < Fft<N>::P4; ++p) {
    team_sync<T>(team);
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = buf[sw(t + r * T)];
#pragma unroll
    for (int r = 1; r < 4; ++r) {
      const float2 w = tws[(3 * (p - 1) + r - 1) * T + t];
      v[r] = cmul(v[r], SIGN < 0 ? w : cconj(w));
    }
    dft4<SIGN>(v[0], v[1], v[2], v[3]);
    const int base = (t / ns) * ns * 4 + t % ns;
    const bool plain = PLAIN && !Fft<N>::R2 && p == Fft<N>::P4 - 1;
    team_sync<T>(team);
#pragma unroll
    for (int r = 0; r < 4; ++r) buf[plain ? base + r * ns : sw(base + r * ns)] = v[r];
    ns *= 4;
  }
  if constexpr (Fft<N>::R2) {
    team_sync<T>(team);
    float2 a0 = buf[sw(t)], b0 = buf[sw(t + M / 2)], a1 = buf[sw(t + T)], b1 = buf[sw(t + T + M / 2)];
    const float2 w0 = tws[TwTab<N>::R2 * T + t], w1 = tws[(TwTab<N>::R2 + 1) * T + t];
    b0 = cmul(b0, SIGN < 0 ? w0 : cconj(w0));
    b1 = cmul(b1, SIGN < 0 ? w1 : cconj(w1));
    team_sync<T>(team);
    buf[PLAIN ? t : sw(t)] = f2add(a0, b0);
    buf[PLAIN ? t + M / 2 : sw(t + M / 2)] = f2sub(a0, b0);
    buf[PLAIN ? t + T : sw(t + T)] = f2add(a1, b1);
    buf[PLAIN ? t + T + M / 2 : sw(t + T + M / 2)] = f2sub(a1, b1);
  }
  team_sync<T>(team);
}

// ------------------------------------------------------------------ 256-point layouts
// With N = 256 (a team is one warp) the skewer transforms keep their buffer
// in two padded layouts instead of the swizzle: LA(i) = i + i/16 and
// LB(i) = i + 4 (i/16) for complex index i <= M.  Every access of the
// 256-point transforms is then a per-lane base plus a compile-time offset (no
// index arithmetic per access), and each half warp still hits 16 distinct
// 8-byte slots (apart from two 2-way conflicts among the mirror reads of the
// untangle step).  LA holds the modes, the outputs of the first write and of
// radix-4 pass 2, and the forward result; LB the output of radix-4 pass 1.
// The arithmetic is that of fft_finish, so results are unchanged.
constexpr int kBuf256 = 156;  // complex slots of a 256-point team buffer: LB(127) + 1
__device__ __forceinline__ int lay_a(int i) { return i + (i >> 4); }
__device__ __forceinline__ int lay_b(int i) { return i + 4 * (i >> 4); }

// fft_finish for N = 256 in the padded layouts (input layout LA after the
// first write; output plain with PLAIN, else LA)
template <int SIGN, bool PLAIN>
__device__ __forceinline__ void fft_finish256(float2 *buf, float2 (&v)[4], const float2 *tws, int t) {
  constexpr int T = 32;
  constexpr int R2 = TwTab<256>::R2;
  __syncwarp();
  {  // 4t + r -> LA: lay_a(4t) + r
    const int b = lay_a(4 * t);
#pragma unroll
    for (int r = 0; r < 4; ++r) buf[b + r] = v[r];
  }
#pragma unroll
  for (int p = 1; p <= 2; ++p) {
    __syncwarp();
    // reads at t + 32 r: LA (pass 1) lay_a(t) + 34 r, LB (pass 2) lay_b(t) + 40 r
    const int rb = p == 1 ? lay_a(t) : lay_b(t);
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = buf[rb + (p == 1 ? 34 : 40) * r];
#pragma unroll
    for (int r = 1; r < 4; ++r) {
      const float2 w = tws[(3 * (p - 1) + r - 1) * T + t];
      v[r] = cmul(v[r], SIGN < 0 ? w : cconj(w));
    }
    dft4<SIGN>(v[0], v[1], v[2], v[3]);
    __syncwarp();
    // writes at base + r ns: pass 1 (ns 4) into LB, lay_b(16 (t/4) + t%4) + 4 r;
    // pass 2 (ns 16) into LA, lay_a(64 (t/16) + t%16) + 17 r
    const int wb = p == 1 ? lay_b(16 * (t >> 2) + (t & 3)) : lay_a(64 * (t >> 4) + (t & 15));
#pragma unroll
    for (int r = 0; r < 4; ++r) buf[wb + (p == 1 ? 4 : 17) * r] = v[r];
  }
  __syncwarp();
  // radix-2 pass: t, t + M/2, t + T, t + T + M/2 in LA = lay_a(t) + 0, 68, 34, 102
  const int rb = lay_a(t);
  float2 a0 = buf[rb], b0 = buf[rb + 68], a1 = buf[rb + 34], b1 = buf[rb + 102];
  const float2 w0 = tws[R2 * T + t], w1 = tws[(R2 + 1) * T + t];
  b0 = cmul(b0, SIGN < 0 ? w0 : cconj(w0));
  b1 = cmul(b1, SIGN < 0 ? w1 : cconj(w1));
  __syncwarp();
  if (PLAIN) {
    buf[t] = f2add(a0, b0);
    buf[t + 64] = f2sub(a0, b0);
    buf[t + 32] = f2add(a1, b1);
    buf[t + 96] = f2sub(a1, b1);
  } else {
    buf[rb] = f2add(a0, b0);
    buf[rb + 68] = f2sub(a0, b0);
    buf[rb + 34] = f2add(a1, b1);
    buf[rb + 102] = f2sub(a1, b1);
  }
  __syncwarp();
}

// Inverse real FFT of the Hermitian modes Y_0..Y_M held in buf (already
// scaled by 1/N); on return the float view holds the N real outputs at plain
// indices (pixel p at float p).
template <int N>
__device__ __forceinline__ void inverse_real_fft(float2 *buf, const float2 *tws, int t, int team) {
  constexpr int T = Fft<N>::T;
  constexpr int M = Fft<N>::M;
  float2 v[4];
  // N = 256: k = t + 32 r at lay_a(t) + 34 r, M - k at lay_a(32 - t) + 34 (3 - r)
  const int ka = N == 256 ? lay_a(t) : 0, kb = N == 256 ? lay_a(32 - t) : 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int k = t + r * T;
    const float2 yk = buf[N == 256 ? ka + 34 * r : sw(k)];
    const float2 ym = cconj(buf[N == 256 ? kb + 34 * (3 - r) : sw(M - k)]);
    // Z_k = (Y_k + conj Y_{M-k}) + i (Y_k - conj Y_{M-k}) e^{+2 pi i k/N}
    v[r] = cadd(cadd(yk, ym), cmul_i<1>(cmul(csub(yk, ym), cconj(tws[(TwTab<N>::U + r) * T + t]))));
  }
  dft4<1>(v[0], v[1], v[2], v[3]);
  if constexpr (N == 256) {
    fft_finish256<1, true>(buf, v, tws, t);
  } else {
    fft_finish<N, 1, true>(buf, v, tws, t, team);
  }
}

// Forward complex FFT of the N reals in the float view of buf (plain
// indices, pixel p at float p); on return buf holds Z_0..Z_{M-1} through the
// swizzle.
template <int N>
__device__ __forceinline__ void forward_packed_fft(float2 *buf, const float2 *tws, int t, int team) {
  constexpr int T = Fft<N>::T;
  float2 v[4];
  team_sync<T>(team);
#pragma unroll
  for (int r = 0; r < 4; ++r) v[r] = buf[t + r * T];
  dft4<-1>(v[0], v[1], v[2], v[3]);
  if constexpr (N == 256) {
    fft_finish256<-1, false>(buf, v, tws, t);
  } else {
    fft_finish<N, -1>(buf, v, tws, t, team);
  }
}

// |X_k|^2 of the real input for k = 4t+1 .. 4t+4 after forward_packed_fft:
// X_k = E_k + e^{-2 pi i k/N} O_k, E = (Z_k + conj Z_{M-k})/2,
// O = (Z_k - conj Z_{M-k})/(2i), Z_M = Z_0.
template <int N>
__device__ __forceinline__ void power_of_modes(const float2 *buf, const float2 *__restrict__ tab, int t,
                                               float (&pk)[4]) {
  constexpr int M = Fft<N>::M;
  // N = 256 (layout LA): k = 4t + 1 + r at lay_a(4t) + 1 + r (r < 3), M - k at
  // lay_a(4 (31 - t)) + 3 - r
  const int pa = N == 256 ? lay_a(4 * t) : 0, pb = N == 256 ? lay_a(4 * (31 - t)) : 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int k = 4 * t + 1 + r;
    const int ik = N != 256 ? sw(k & (M - 1)) : (r < 3 ? pa + 1 + r : lay_a(k & (M - 1)));
    const float2 zk = buf[ik];
    const float2 zm = cconj(buf[N == 256 ? pb + 3 - r : sw((M - k) & (M - 1))]);
    const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y + zm.y));
    const float2 dd = csub(zk, zm);
    const float2 o = make_float2(0.5f * dd.y, -0.5f * dd.x);
    const float2 w = __ldg(tab + (k & (N - 1)));
    const float2 x = cadd(e, cmul(w, o));
    pk[r] = fmaf(x.x, x.x, x.y * x.y);
  }
}

// ------------------------------------------------------------------ small-scale modes
// Y_m = X_m / N for m = 0..M into buf (Philox words -> Box-Muller):
// X_m = A_m sqrt(-ln u1) e^{2 pi i u2} (= A (e1 + i e2)/sqrt 2), X_M = A e1.
// Counter c serves modes 2c (words 0, 1) and 2c + 1 (words 2, 3); the words
// of counter 0 that mode 0 (X_0 = 0) would use serve the Nyquist mode M.
// ZNODES: amp and amp_hi hold (A_m / N)^2 at two z nodes, mixed with weight
// w_hi; otherwise amp holds A_m / N and amp_hi is unused.
template <int N, bool ZNODES>
__device__ __forceinline__ void small_scale_modes(float2 *buf, const float *__restrict__ amp,
                                                  const float *__restrict__ amp_hi, float w_hi, uint32_t seg,
                                                  uint64_t id, uint32_t seed, int t) {
  constexpr int T = Fft<N>::T;
  constexpr int M = Fft<N>::M;
  const uint32_t id_lo = static_cast<uint32_t>(id), id_hi = static_cast<uint32_t>(id >> 32);
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const uint32_t c = t + q * T;  // modes 2c, 2c+1 (< M)
    const u32x4 w = philox4x32_10(u32x4{c, seg, id_hi, 0u}, seed, id_lo);
    const bool nyq = (c == 0);
    const int m0 = nyq ? M : 2 * c, m1 = 2 * c + 1;
    float s0 = __ldg(amp + m0), s1 = __ldg(amp + m1);
    if (ZNODES) {  // interpolate P_s between the nodes, then the root
      s0 = sqrtf(fmaf(w_hi, __ldg(amp_hi + m0) - s0, s0));
      s1 = sqrtf(fmaf(w_hi, __ldg(amp_hi + m1) - s1, s1));
    }
    const float2 p0 = unit_phase(w.y), p1 = unit_phase(w.w);
    const float a0 = s0 * sqrt_pos((nyq ? 2.0f : 1.0f) * neg_log_uniform(w.x));
    const float a1 = s1 * sqrt_pos(neg_log_uniform(w.z));
    // N = 256 (layout LA): mode 2c + e, c = t + 32 q, at lay_a(2t) + e + 68 q
    const int i0 = N != 256 ? sw(m0) : (nyq ? lay_a(M) : lay_a(2 * t) + 68 * q);
    const int i1 = N != 256 ? sw(m1) : lay_a(2 * t) + 1 + 68 * q;
    buf[i0] = make_float2(a0 * p0.x, nyq ? 0.f : a0 * p0.y);
    buf[i1] = make_float2(a1 * p1.x, a1 * p1.y);
  }
  if (t == 0) buf[0] = make_float2(0.f, 0.f);  // sw(0) = lay_a(0) = 0
}

// ------------------------------------------------------------------ fixed-point gather
// Positions are Q20.44 cell coordinates (minus 1/2, so that integer values
// fall on cell centres).  The kernels add kRoundQ to a skewer's start so that
// the weight below, the top 23 fraction bits, is the fraction rounded to
// nearest; a fraction that rounds up to 1 moves to the next cell with weight 0.
constexpr int64_t kRoundQ = int64_t(1) << 20;

// base cell index (periodic, n = mask + 1)
__device__ __forceinline__ int cell_of(int64_t p, int mask) { return static_cast<int>(p >> 44) & mask; }

// weight in [0, 1): 1.m - 1 with m the fraction bits 43..21 (exact)
__device__ __forceinline__ float weight_of(int64_t p) {
  const uint32_t m = static_cast<uint32_t>(static_cast<uint64_t>(p) >> 21) & 0x7FFFFFu;
  return __uint_as_float(0x3F800000u | m) - 1.0f;
}

__device__ __forceinline__ float lerpf(float a, float b, float t) { return fmaf(t, b - a, a); }

// Trilinear (delta, eta) at fixed-point coordinate (px, py, pz).  BIG: box
// with more than 2^30 cells (64-bit indices).
//   MK_BOX_PLANAR / MK_BOX_INTERLEAVED: n^3 cells, periodic indices.
//   MK_BOX_PADDED: (delta, eta) pairs on (n+1)^3 points whose last plane,
//   row and column repeat index 0, so the 8 corners sit at fixed offsets
//   from the base corner and no index wraps.
//   MK_BOX_HALO: pairs on (n+6)^3 points, a periodic margin of 3 on every
//   side; the same fixed offsets from base index (x+3, y+3, z+3).
// FIXLGN > 0 (padded layout, 32-bit indices): the box side is 2^FIXLGN, so
// the row and plane strides are constants and the eight loads take immediate
// offsets from one pointer (placed mid-way between the two planes, so that
// every offset stays within the immediate range).
template <int LAYOUT, bool BIG, int FIXLGN = 0>
__device__ __forceinline__ float2 gather(const float *__restrict__ d, const float *__restrict__ e, int lgn,
                                         int64_t px, int64_t py, int64_t pz) {
  const int mask = FIXLGN > 0 ? (1 << FIXLGN) - 1 : (1 << lgn) - 1;
  const int x0 = cell_of(px, mask), y0 = cell_of(py, mask), z0 = cell_of(pz, mask);
  const float tx = weight_of(px), ty = weight_of(py), tz = weight_of(pz);
  using I = typename std::conditional<BIG, int64_t, int32_t>::type;
  float2 v[8];
  if constexpr (FIXLGN > 0) {
    static_assert(LAYOUT == MK_BOX_PADDED && !BIG, "fixed strides serve the padded layout with 32-bit indices");
    constexpr int n1 = (1 << FIXLGN) + 1, plane = n1 * n1, half = plane / 2;
    const float2 *mid = reinterpret_cast<const float2 *>(d) + (z0 * plane + y0 * n1 + x0 + half);
    const float2 *a00 = mid - half, *a01 = a00 + n1;
    const float2 *a10 = mid + (plane - half), *a11 = a10 + n1;
    v[0] = __ldg(a00); v[1] = __ldg(a00 + 1);
    v[2] = __ldg(a01); v[3] = __ldg(a01 + 1);
    v[4] = __ldg(a10); v[5] = __ldg(a10 + 1);
    v[6] = __ldg(a11); v[7] = __ldg(a11 + 1);
  } else if constexpr (LAYOUT == MK_BOX_PADDED || LAYOUT == MK_BOX_HALO) {
    constexpr int h = LAYOUT == MK_BOX_HALO ? 3 : 0;
    const I n1 = mask + 1 + (LAYOUT == MK_BOX_HALO ? 6 : 1);
    const float2 *a00 =
        reinterpret_cast<const float2 *>(d) + ((static_cast<I>(z0 + h) * n1 + (y0 + h)) * n1 + (x0 + h));
    const float2 *a01 = a00 + n1, *a10 = a00 + n1 * n1;
    const float2 *a11 = a10 + n1;
    v[0] = __ldg(a00); v[1] = __ldg(a00 + 1);
    v[2] = __ldg(a01); v[3] = __ldg(a01 + 1);
    v[4] = __ldg(a10); v[5] = __ldg(a10 + 1);
    v[6] = __ldg(a11); v[7] = __ldg(a11 + 1);
  } else {
    const int x1 = (x0 + 1) & mask, y1 = (y0 + 1) & mask, z1 = (z0 + 1) & mask;
    using U = typename std::conditional<BIG, size_t, uint32_t>::type;
    const U zz0 = static_cast<U>(z0) << (2 * lgn), zz1 = static_cast<U>(z1) << (2 * lgn);
    const U yy0 = static_cast<U>(y0) << lgn, yy1 = static_cast<U>(y1) << lgn;
    const U r00 = zz0 | yy0, r10 = zz0 | yy1, r01 = zz1 | yy0, r11 = zz1 | yy1;
    if constexpr (LAYOUT == MK_BOX_INTERLEAVED) {
      const float2 *b = reinterpret_cast<const float2 *>(d);
      v[0] = __ldg(b + (r00 | x0)); v[1] = __ldg(b + (r00 | x1));
      v[2] = __ldg(b + (r10 | x0)); v[3] = __ldg(b + (r10 | x1));
      v[4] = __ldg(b + (r01 | x0)); v[5] = __ldg(b + (r01 | x1));
      v[6] = __ldg(b + (r11 | x0)); v[7] = __ldg(b + (r11 | x1));
    } else {
      const U idx[8] = {r00 | x0, r00 | x1, r10 | x0, r10 | x1, r01 | x0, r01 | x1, r11 | x0, r11 | x1};
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = make_float2(__ldg(d + idx[k]), __ldg(e + idx[k]));
    }
  }
  // x, then y, then z; delta and eta as one packed pair
  const float2 c0 = f2lerp(v[0], v[1], tx), c1 = f2lerp(v[2], v[3], tx);
  const float2 c2 = f2lerp(v[4], v[5], tx), c3 = f2lerp(v[6], v[7], tx);
  return f2lerp(f2lerp(c0, c1, ty), f2lerp(c2, c3, ty), tz);
}

// Trilinear (delta, eta_par) from an MK_BOX_TENSOR box: all seven fields are
// interpolated (x, then y, then z, on packed pairs) and the velocity-gradient
// tensor is contracted with the sight line, eta_par = u_p u_q eta_pq (Eq. eta);
// uu = {ux^2, uy^2, uz^2, 2 ux uy, 2 ux uz, 2 uy uz}.
struct F7 {
  float2 a, b, c;  // (delta, xx), (yy, zz), (xy, xz)
  float d;         // yz
};
__device__ __forceinline__ F7 lerp7(const F7 &p, const F7 &q, float t) {
  return F7{f2lerp(p.a, q.a, t), f2lerp(p.b, q.b, t), f2lerp(p.c, q.c, t), lerpf(p.d, q.d, t)};
}
// the two points (x0, x0 + 1) of a row, lerped in x
__device__ __forceinline__ F7 tensor_row(const float4 *r, float tx) {
  const float4 a0 = __ldg(r), b0 = __ldg(r + 1), a1 = __ldg(r + 2), b1 = __ldg(r + 3);
  const F7 p{make_float2(a0.x, a0.y), make_float2(a0.z, a0.w), make_float2(b0.x, b0.y), b0.z};
  const F7 q{make_float2(a1.x, a1.y), make_float2(a1.z, a1.w), make_float2(b1.x, b1.y), b1.z};
  return lerp7(p, q, tx);
}

template <bool BIG>
__device__ __forceinline__ float2 gather_tensor(const float *__restrict__ d, int lgn, int64_t px, int64_t py,
                                                int64_t pz, const float (&uu)[6]) {
  const int mask = (1 << lgn) - 1;
  const int x0 = cell_of(px, mask), y0 = cell_of(py, mask), z0 = cell_of(pz, mask);
  const float tx = weight_of(px), ty = weight_of(py), tz = weight_of(pz);
  using I = typename std::conditional<BIG, int64_t, int32_t>::type;
  const I n1 = mask + 2;
  const float4 *b = reinterpret_cast<const float4 *>(d);
  const I i00 = (static_cast<I>(z0) * n1 + y0) * n1 + x0;
  const F7 c0 = tensor_row(b + 2 * i00, tx), c1 = tensor_row(b + 2 * (i00 + n1), tx);
  const F7 c2 = tensor_row(b + 2 * (i00 + n1 * n1), tx), c3 = tensor_row(b + 2 * (i00 + n1 * n1 + n1), tx);
  const F7 v = lerp7(lerp7(c0, c1, ty), lerp7(c2, c3, ty), tz);
  const float eta = fmaf(uu[0], v.a.y, fmaf(uu[1], v.b.x, fmaf(uu[2], v.b.y,
                    fmaf(uu[3], v.c.x, fmaf(uu[4], v.c.y, uu[5] * v.d)))));
  return make_float2(v.a.x, eta);
}

// Normalised 1D weights of the Gaussian-kernel average (Sec. 2.3) along one
// axis: voxels c - 3 .. c + 3 around the voxel c containing the point, whose
// centre is at distance e = 1/2 - f (f the point's offset inside voxel c, in
// cells); voxel c + m sits at m + e, w_m ~ exp(-(m + e)^2 / 2).  With
// q = exp(-e), w_m ~ q^m C_m, C_m = exp(-m^2/2) (the common factor
// exp(-e^2/2) cancels in the normalisation): two exponentials per axis.
static __constant__ float kGauss7C[7] = {0.011108996538242306f, 0.13533528323661270f, 0.60653065971263342f, 1.0f,
                                         0.60653065971263342f, 0.13533528323661270f, 0.011108996538242306f};

// q = exp(-e), qi = 1/q and the reciprocal of sum_m q^m C_m
__device__ __forceinline__ void gauss7_axis(float f, float &q, float &qi, float &inv) {
  const float e = 0.5f - f;
  q = expf(-e);
  qi = expf(e);
  const float q2 = q * q, qi2 = qi * qi;
  const float c1 = kGauss7C[2], c2 = kGauss7C[1], c3 = kGauss7C[0];
  inv = 1.0f / ((c3 * (qi2 * qi) + c3 * (q2 * q)) + (c2 * qi2 + c2 * q2) + (c1 * qi + c1 * q) + 1.0f);
}

__device__ __forceinline__ void gauss7_weights(float f, float (&w)[7]) {
  float q, qi, inv;
  gauss7_axis(f, q, qi, inv);
  float pw = qi * qi * qi * inv;  // q^m inv for m = -3
#pragma unroll
  for (int m = 0; m < 7; ++m) {
    w[m] = pw * kGauss7C[m];
    pw *= q;
  }
}

// Gaussian-kernel average of (delta, eta) over 7^3 voxels (Sec. 2.3) from an
// MK_BOX_HALO box, as three nested 1D contractions (the weights are
// separable): per z plane, 7 x-rows of 7 pairs contracted with the x weights,
// then with the y weights; the z weights come as a running product.
template <bool BIG>
__device__ __forceinline__ float2 gather_gauss7(const float *__restrict__ d, int lgn, int64_t px, int64_t py,
                                                int64_t pz) {
  const int mask = (1 << lgn) - 1;
  // containing voxel: floor(p + 1/2) of the centre-based coordinate p
  const int64_t hx = px + (int64_t(1) << 43), hy = py + (int64_t(1) << 43), hz = pz + (int64_t(1) << 43);
  const int cx = cell_of(hx, mask), cy = cell_of(hy, mask), cz = cell_of(hz, mask);
  float wx[7], wy[7];
  gauss7_weights(weight_of(hx), wx);
  gauss7_weights(weight_of(hy), wy);
  float qz, qiz, invz;
  gauss7_axis(weight_of(hz), qz, qiz, invz);
  float pz_run = qiz * qiz * qiz * invz;
  using I = typename std::conditional<BIG, int64_t, int32_t>::type;
  const I n6 = mask + 7;
  // voxel (c - 3) per axis sits at halo index c
  const float2 *row = reinterpret_cast<const float2 *>(d) + ((static_cast<I>(cz) * n6 + cy) * n6 + cx);
  float2 acc = make_float2(0.f, 0.f);
#pragma unroll 1
  for (int k = 0; k < 7; ++k) {
    float2 ay = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      const float2 *r = row + j * n6;
      float2 ax = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < 7; ++i) ax = f2fma(make_float2(wx[i], wx[i]), __ldg(r + i), ax);
      ay = f2fma(make_float2(wy[j], wy[j]), ax, ay);
    }
    const float wk = pz_run * kGauss7C[k];
    acc = f2fma(make_float2(wk, wk), ay, acc);
    pz_run *= qz;
    row += n6 * n6;
  }
  return acc;
}

// Prefetch into L2 the four voxel rows (y0|y1, z0|z1) that the trilinear
// stencil at (px, py, pz) reads, for the paired layouts (each row's two
// corners x0, x0 + 1 are adjacent).
template <int LAYOUT, bool BIG>
__device__ __forceinline__ void prefetch_stencil(const float *__restrict__ d, int lgn, int64_t px, int64_t py,
                                                 int64_t pz) {
  if constexpr (LAYOUT == MK_BOX_PLANAR) return;
  if constexpr (LAYOUT == MK_BOX_TENSOR) {
    const int mask = (1 << lgn) - 1;
    const int x0 = cell_of(px, mask), y0 = cell_of(py, mask), z0 = cell_of(pz, mask);
    using I = typename std::conditional<BIG, int64_t, int32_t>::type;
    const I n1 = mask + 2;
    const float4 *b = reinterpret_cast<const float4 *>(d);
    const I i00 = (static_cast<I>(z0) * n1 + y0) * n1 + x0;
    const I rows[4] = {i00, i00 + n1, i00 + n1 * n1, i00 + n1 * n1 + n1};
#pragma unroll
    for (int r = 0; r < 4; ++r) asm volatile("prefetch.global.L2 [%0];" ::"l"(b + 2 * rows[r]));
    return;
  }
  const int mask = (1 << lgn) - 1;
  const int x0 = cell_of(px, mask), y0 = cell_of(py, mask), z0 = cell_of(pz, mask);
  using I = typename std::conditional<BIG, int64_t, int32_t>::type;
  const float2 *b = reinterpret_cast<const float2 *>(d);
  const float2 *a[4];
  if constexpr (LAYOUT == MK_BOX_PADDED || LAYOUT == MK_BOX_HALO) {
    constexpr int h = LAYOUT == MK_BOX_HALO ? 3 : 0;
    const I n1 = mask + 1 + (LAYOUT == MK_BOX_HALO ? 6 : 1);
    a[0] = b + ((static_cast<I>(z0 + h) * n1 + (y0 + h)) * n1 + (x0 + h));
    a[1] = a[0] + n1;
    a[2] = a[0] + n1 * n1;
    a[3] = a[2] + n1;
  } else {
    const int y1 = (y0 + 1) & mask, z1 = (z0 + 1) & mask;
    using U = typename std::conditional<BIG, size_t, uint32_t>::type;
    a[0] = b + ((static_cast<U>(z0) << (2 * lgn)) | (static_cast<U>(y0) << lgn) | x0);
    a[1] = b + ((static_cast<U>(z0) << (2 * lgn)) | (static_cast<U>(y1) << lgn) | x0);
    a[2] = b + ((static_cast<U>(z1) << (2 * lgn)) | (static_cast<U>(y0) << lgn) | x0);
    a[3] = b + ((static_cast<U>(z1) << (2 * lgn)) | (static_cast<U>(y1) << lgn) | x0);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) asm volatile("prefetch.global.L2 [%0];" ::"l"(a[r]));
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
// Per-warp accumulators in shared memory, FP32 with Kahan compensation
// (each slot has one writer lane), flushed to FP64 at the end of the kernel:
//   sums[n_z][NSUM] (float2 {sum, compensation}), p1d[n_z][n_k] (float2),
//   nseg[n_z] (uint32)
struct WarpAcc {
  float2 *sums, *p1d;
  uint32_t *nseg;
  __host__ __device__ static size_t bytes(int n_z, int n_k) {
    return ((sizeof(float2) * n_z * (MK_NSUM + n_k) + sizeof(uint32_t) * n_z) + 15) / 16 * 16;
  }
  __device__ static WarpAcc at(unsigned char *base, int n_z, int n_k) {
    WarpAcc a;
    a.sums = reinterpret_cast<float2 *>(base);
    a.p1d = a.sums + n_z * MK_NSUM;
    a.nseg = reinterpret_cast<uint32_t *>(a.p1d + n_z * n_k);
    return a;
  }
};

__device__ __forceinline__ void kahan_add(float2 &acc, float x) {
  const float y = x - acc.y;
  const float t = acc.x + y;
  acc.y = (t - acc.x) - y;
  acc.x = t;
}

// Warp reduce-scatter of 16 values: afterwards lanes l and l + 16 hold the
// warp total of v[l & 15].
__device__ __forceinline__ float reduce_scatter16(float (&v)[16], int lane) {
#pragma unroll
  for (int s = 8; s >= 1; s >>= 1) {
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const bool up = lane & s;
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// Warp reduce-scatter of 32 values: lane l holds the warp total of v[l].
__device__ __forceinline__ float reduce_scatter32(float (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const bool up = lane & s;
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  return v[0];
}

// Pixel sums of one pixel: n, F, F^2, d, e, d^2, e^2, d e, F d, F e.
__device__ __forceinline__ void add_pixel(float *a, float f, float d, float e) {
  a[0] += 1.f;
  a[1] += f;
  a[2] = fmaf(f, f, a[2]);
  a[3] += d;
  a[4] += e;
  a[5] = fmaf(d, d, a[5]);
  a[6] = fmaf(e, e, a[6]);
  a[7] = fmaf(d, e, a[7]);
  a[8] = fmaf(f, d, a[8]);
  a[9] = fmaf(f, e, a[9]);
}

// Pixel sums of one thread for one z bin, in the StatLayout order
// n, F, F^2, d, e, d^2, e^2, d e, F d, F e; the (d, e) pairs run packed.
struct PixelSums {
  float n, f, ff, de;
  float2 m1, m2, fm;  // (d, e), (d^2, e^2), (F d, F e)
  __device__ __forceinline__ void zero() {
    n = f = ff = de = 0.f;
    m1 = m2 = fm = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void add(float F, float2 x) {
    n += 1.f;
    add_sums(F, x);
  }
  // the sums without the count (a full segment adds its count once)
  __device__ __forceinline__ void add_sums(float F, float2 x) {
    f += F;
    ff = fmaf(F, F, ff);
    de = fmaf(x.x, x.y, de);
    m1 = f2add(m1, x);
    m2 = f2fma(x, x, m2);
    fm = f2fma(make_float2(F, F), x, fm);
  }
};

// Add the warp's PixelSums of bin zb to the warp accumulators (warp-uniform
// call; bins outside [0, n_z) are dropped).
__device__ __forceinline__ void flush_bin_sums(const WarpAcc &W, int n_z, int zb, const PixelSums &a, int lane) {
  float v[16] = {a.n, a.f, a.ff, a.m1.x, a.m1.y, a.m2.x, a.m2.y, a.de, a.fm.x, a.fm.y,
                 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const float s = reduce_scatter16(v, lane);
  if (lane < MK_NSUM && zb >= 0 && zb < n_z) kahan_add(W.sums[zb * MK_NSUM + lane], s);
}

// Flush the thread sums of bins zf (a0) and zf + 1 (a1) into the warp
// accumulators (warp-uniform call).
__device__ __forceinline__ void flush_pixel_sums(const WarpAcc &W, int n_z, int zf, bool two, const float *a0,
                                                 const float *a1, int lane) {
  if (!two) {
    float v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = i < MK_NSUM ? a0[i] : 0.f;
    const float s = reduce_scatter16(v, lane);
    if (lane < MK_NSUM && zf >= 0 && zf < n_z) kahan_add(W.sums[zf * MK_NSUM + lane], s);
  } else {
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = i < MK_NSUM ? a0[i] : (i < 2 * MK_NSUM ? a1[i - MK_NSUM] : 0.f);
    const float s = reduce_scatter32(v, lane);
    const int b = zf + (lane >= MK_NSUM ? 1 : 0);
    if (lane < 2 * MK_NSUM && b >= 0 && b < n_z) kahan_add(W.sums[b * MK_NSUM + lane % MK_NSUM], s);
  }
}

// Pixel sums of bins beyond zf + 1 (only when a segment spans three or more
// bins): the lanes that need it take turns adding into the warp accumulators.
__device__ __forceinline__ void add_pixel_slow(const WarpAcc &W, int zb, float f, float d, float e) {
  float a[MK_NSUM] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  add_pixel(a, f, d, e);
  const unsigned active = __activemask();
  const int lane = threadIdx.x & 31;
  for (int l = 0; l < 32; ++l) {
    if (((active >> l) & 1u) && l == lane) {
#pragma unroll
      for (int i = 0; i < MK_NSUM; ++i) kahan_add(W.sums[zb * MK_NSUM + i], a[i]);
    }
    __syncwarp(active);
  }
}

// Add the 4 mode powers of thread t (modes 4t+1..4t+4) to the P1D bins of z
// bin zb (warp-uniform call).  Every bin slot of a warp has one writer.
template <int N>
__device__ __forceinline__ void accumulate_p1d(const WarpAcc &W, int n_k, const float (&pk)[4], float scale,
                                               int zb, int t) {
  constexpr int M = Fft<N>::M;
  const int per_bin = M / n_k;
  const int lane = t & 31;
  if (per_bin >= 4) {
    float s = (pk[0] + pk[1]) + (pk[2] + pk[3]);
    const int group = per_bin / 4;  // threads sharing a bin
    const int g32 = group < 32 ? group : 32;
    for (int o = 1; o < g32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((lane & (g32 - 1)) == 0) kahan_add(W.p1d[zb * n_k + (4 * t) / per_bin], s * scale);
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) kahan_add(W.p1d[zb * n_k + ((4 * t + r) * n_k) / M], pk[r] * scale);
  }
}

}  // namespace mk
