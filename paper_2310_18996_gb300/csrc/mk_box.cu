// Gaussian box synthesis (Sec. 2.1, Eq. deltaL, Eq. eta): Philox white noise,
// a 3D FFT made of batched line FFTs in shared memory, the sqrt(P(k)) filter
// and the velocity-gradient filters -k_p k_q / k^2, written straight into the
// library's box layouts.
//
// Five passes make one (delta, eta_pq) pair of boxes, each reading and writing
// the n^3 complex work box once:
//   noise + FFT x | FFT y | FFT z, filter, inverse FFT z | inverse y | inverse x + layout
// Two real boxes come out of one complex inverse transform: the modes of
// delta and eta are Hermitian, so IFFT(D f1 + i D f2) = (delta f1-box) + i (f2-box).
#include <algorithm>

#include "mk_device.cuh"
#include "mk_kernels.h"

namespace mk {
namespace {

constexpr int kLines = 8;     // lines per CTA group
constexpr int kLinePad = 2;   // complex slots of padding per line buffer
constexpr int kBoxThreads = 512;

// Lines of 1024 points take the warp-register FFT (REG): one warp per line,
// 256 threads, line buffers of 1024 + 34 slots (the 32 x 33 transpose fits).
template <int N2, bool REG>
struct BoxSmem {
  static constexpr int M = N2 / 2;  // line length n
  static constexpr int PAD = REG ? 34 : kLinePad;
  static constexpr int THREADS = REG ? 256 : kBoxThreads;
  static constexpr size_t TW = REG ? 256 : TwTab<N2>::BYTES;  // REG: 16 twiddles of the 32-point DFT
  static constexpr size_t bytes() { return TW + sizeof(float2) * kLines * (M + PAD); }
};

// bit reversal of a 5-bit index
__host__ __device__ constexpr int rev5(int k) {
  return ((k & 1) << 4) | ((k & 2) << 2) | (k & 4) | ((k & 8) >> 2) | ((k & 16) >> 4);
}

// 32-point DFT in registers: radix-2 decimation in frequency, natural order in,
// bit-reversed order out (X[k] = x[rev5(k)]); w32[m] = e^{-2 pi i m / 32}, m < 16.
template <int SIGN>
__device__ __forceinline__ void dft32_reg(float2 (&x)[32], const float2 *w32) {
#pragma unroll
  for (int span = 16; span >= 1; span >>= 1) {
#pragma unroll
    for (int blk = 0; blk < 32; blk += 2 * span) {
#pragma unroll
      for (int j = 0; j < span; ++j) {
        const float2 a = x[blk + j], b = x[blk + j + span];
        x[blk + j] = f2add(a, b);
        const float2 d = f2sub(a, b);
        const int m = j * (16 / span);
        if (m == 0) {
          x[blk + j + span] = d;
        } else {
          const float2 w = w32[m];
          x[blk + j + span] = cmul(d, SIGN < 0 ? w : cconj(w));
        }
      }
    }
  }
}

// 1024-point FFT of one line by one warp (four-step, 32 x 32): a 32-point DFT
// over n2 of x[lane + 32 n2], the twiddles W_1024^(lane k2), a transpose
// through the line buffer (rows of 33), a 32-point DFT over n1; natural order
// in and out.  tab[k] = e^{-2 pi i k / 2048}.
template <int SIGN>
__device__ __forceinline__ void fft1024_warp(float2 *b, const float2 *__restrict__ tab, const float2 *w32, int lane) {
  float2 x[32];
#pragma unroll
  for (int n2 = 0; n2 < 32; ++n2) x[n2] = b[lane + 32 * n2];
  dft32_reg<SIGN>(x, w32);
  // W_1024^(lane k2) for k2 = 8 q + r: (W^(8 lane))^q (W^lane)^r, W_1024^m = tab[2 m]
  const float2 t1 = __ldg(tab + 2 * lane), t8 = __ldg(tab + ((16 * lane) & 2047));
  float2 p1[8];
  p1[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int r = 1; r < 8; ++r) p1[r] = cmul(p1[r - 1], t1);
  float2 q = make_float2(1.f, 0.f);
#pragma unroll
  for (int qq = 0; qq < 4; ++qq) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int k2 = 8 * qq + r;
      if (k2 == 0) continue;
      const float2 w = cmul(q, p1[r]);
      x[rev5(k2)] = cmul(x[rev5(k2)], SIGN < 0 ? w : cconj(w));
    }
    q = cmul(q, t8);
  }
  __syncwarp();
#pragma unroll
  for (int k2 = 0; k2 < 32; ++k2) b[k2 * 33 + lane] = x[rev5(k2)];
  __syncwarp();
#pragma unroll
  for (int n1 = 0; n1 < 32; ++n1) x[n1] = b[lane * 33 + n1];
  dft32_reg<SIGN>(x, w32);
  __syncwarp();
#pragma unroll
  for (int k1 = 0; k1 < 32; ++k1) b[lane + 32 * k1] = x[rev5(k1)];
  __syncwarp();
}

// Asynchronous global-to-shared copies (no register round trip, all of a
// thread's copies in flight at once).
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t s = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ int wrap_index(int j, int n) { return j < n / 2 ? j : j - n; }

// Filter pair p of the Sec. 2.1 boxes at wave vector k (k2 = |k|^2 > 0):
// (f1, f2) with eta_pq = -k_p k_q / k^2 delta.
__device__ __forceinline__ float2 pair_filter(int pair, float kx, float ky, float kz, float inv_k2) {
  switch (pair) {
    case 0: return make_float2(1.0f, -kx * kx * inv_k2);
    case 1: return make_float2(-ky * ky * inv_k2, -kz * kz * inv_k2);
    case 2: return make_float2(-kx * ky * inv_k2, -kx * kz * inv_k2);
    default: return make_float2(-ky * kz * inv_k2, 0.0f);
  }
}

// Address of element e of line c in group g along `axis` (box side n).
__device__ __forceinline__ int64_t line_addr(int axis, int64_t g, int c, int e, int n) {
  const int64_t nn = static_cast<int64_t>(n) * n;
  if (axis == 0) return (g * kLines + c) * n + e;
  const int64_t row = g / (n / kLines), x = (g % (n / kLines)) * kLines + c;
  return axis == 1 ? row * nn + static_cast<int64_t>(e) * n + x : row * n + static_cast<int64_t>(e) * nn + x;
}

// Flat index i of a group's kLines * n elements to (line c, element e): along
// x whole lines are contiguous; along y and z the kLines lines of one
// element are.
__device__ __forceinline__ void flat_to_ce(int axis, int i, int n, int &c, int &e) {
  if (axis == 0) {
    c = i / n;
    e = i % n;
  } else {
    e = i / kLines;
    c = i % kLines;
  }
}

template <int N2, int MODE, bool REG>
__global__ void __launch_bounds__(BoxSmem<N2, REG>::THREADS, 2) k_box_pass(BoxPassParams P) {
  constexpr int M = N2 / 2;  // box side
  constexpr int THREADS = BoxSmem<N2, REG>::THREADS;
  constexpr int T = Fft<N2>::T;
  constexpr int TEAMS = THREADS / T;
  static_assert(REG || T == 32 || TEAMS <= 15, "teams of more than one warp use named barriers 1..TEAMS");
  static_assert(!REG || (N2 == 2048 && THREADS == 32 * kLines), "the register FFT: 1024-point lines, a warp each");
  constexpr int LS = M + BoxSmem<N2, REG>::PAD;
  constexpr int SIGN = (MODE == kBoxNoiseX || MODE == kBoxFwd || MODE == kBoxShapeZ) ? -1 : 1;
  constexpr int AXIS_FIXED = (MODE == kBoxNoiseX || MODE == kBoxInvXOut) ? 0
                             : (MODE == kBoxShapeZ || MODE == kBoxSpecZ) ? 2 : -1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2 *tws = reinterpret_cast<float2 *>(smem_raw);
  float2 *lines = reinterpret_cast<float2 *>(smem_raw + BoxSmem<N2, REG>::TW);
  if constexpr (REG) {
    if (threadIdx.x < 16) tws[threadIdx.x] = __ldg(P.tw + 64 * threadIdx.x);  // e^{-2 pi i m / 32}
    __syncthreads();
  } else {
    fill_twiddles<N2>(tws, P.tw);
  }
  const int axis = AXIS_FIXED >= 0 ? AXIS_FIXED : P.axis;
  const int team = threadIdx.x / T, t = threadIdx.x % T;
  const int64_t groups = static_cast<int64_t>(M) * M / kLines;

  for (int64_t g = blockIdx.x; g < groups; g += gridDim.x) {
    // ---- load (or draw) the group's lines
    if constexpr (MODE == kBoxNoiseX) {
      // 4 voxels per Philox call: (w0, w1) and (w2, w3) through Box-Muller
      const int64_t v0 = g * kLines * M;
      for (int i = 4 * threadIdx.x; i < kLines * M; i += 4 * THREADS) {
        const uint64_t q = static_cast<uint64_t>(v0 + i) >> 2;
        const u32x4 w = philox4x32_10(u32x4{static_cast<uint32_t>(q), static_cast<uint32_t>(q >> 32), 0u, 0u},
                                      P.key0, P.key1);
        const float r0 = sqrt_pos(2.0f * neg_log_uniform(w.x)), r1 = sqrt_pos(2.0f * neg_log_uniform(w.z));
        const float2 p0 = unit_phase(w.y), p1 = unit_phase(w.w);
        const int c = i / M, e = i % M;  // 4 | M: the 4 voxels share a line
        float2 *b = lines + c * LS + e;
        b[0] = make_float2(r0 * p0.x, 0.f);
        b[1] = make_float2(r0 * p0.y, 0.f);
        b[2] = make_float2(r1 * p1.x, 0.f);
        b[3] = make_float2(r1 * p1.y, 0.f);
      }
    } else {
      const float2 *src = (MODE == kBoxSpecZ) ? P.spec : P.work;
      if (axis == 0) {  // whole lines: 16-byte copies of element pairs
        for (int i = 2 * threadIdx.x; i < kLines * M; i += 2 * THREADS) {
          const int c = i / M, e = i % M;
          cp_async16(lines + c * LS + e, src + line_addr(0, g, c, e, M));
        }
      } else {          // kLines adjacent columns: 8-byte copies, 64 B per row
        for (int i = threadIdx.x; i < kLines * M; i += THREADS) {
          int c, e;
          flat_to_ce(axis, i, M, c, e);
          cp_async8(lines + c * LS + e, src + line_addr(axis, g, c, e, M));
        }
      }
      cp_async_wait_all();
    }
    __syncthreads();

    // ---- FFT along the line (forward, or inverse for the inverse modes)
    if constexpr (MODE != kBoxSpecZ) {
      if constexpr (REG) {
        fft1024_warp<SIGN>(lines + (threadIdx.x >> 5) * LS, P.tw, tws, threadIdx.x & 31);
      } else {
        for (int c = team; c < kLines; c += TEAMS) {
          float2 *b = lines + c * LS;
          float2 v[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) v[r] = b[t + r * T];
          dft4<SIGN>(v[0], v[1], v[2], v[3]);
          fft_finish<N2, SIGN, true>(b, v, tws, t, team);
        }
      }
      __syncthreads();
    }

    // ---- filter in mode space (z lines: element e is k_z)
    if constexpr (MODE == kBoxShapeZ || MODE == kBoxSpecZ) {
      const int64_t yrow = g / (M / kLines);
      const int x0 = static_cast<int>(g % (M / kLines)) * kLines;
      const int ky_i = static_cast<int>(yrow);
      for (int i = threadIdx.x; i < kLines * M; i += THREADS) {
        const int e = i / kLines, c = i % kLines;
        const int xi = x0 + c;
        float2 d = lines[c * LS + e];
        const float kx = P.kf * wrap_index(xi, M), ky = P.kf * wrap_index(ky_i, M), kz = P.kf * wrap_index(e, M);
        const float k2 = kx * kx + ky * ky + kz * kz;
        if constexpr (MODE == kBoxShapeZ) {
          const bool zero = (xi == M / 2) || (ky_i == M / 2) || (e == M / 2) || k2 == 0.0f;
          float s = 0.0f;
          if (!zero) {
            // linear in the table, 0 beyond its last entry (n_pk <= 2^24: the
            // comparison is exact and j <= n_pk - 2 below); |k| and the roots
            // through rsqrt (a few ulp, far inside the synthesis tolerance)
            const float u = k2 * rsqrtf(k2) * P.inv_dk, last = static_cast<float>(P.n_pk - 1);
            float pk = -1.0f;
            if (u < last) {
              const int j = static_cast<int>(u);
              const float f = u - static_cast<float>(j);
              pk = fmaf(f, __ldg(P.pk + j + 1) - __ldg(P.pk + j), __ldg(P.pk + j));
            } else if (u == last) {
              pk = __ldg(P.pk + P.n_pk - 1);
            }
            s = pk > 0.0f ? pk * rsqrtf(pk) * P.amp : 0.0f;
          }
          d = make_float2(d.x * s, d.y * s);
          if (P.spec) P.spec[line_addr(2, g, c, e, M)] = d;
        }
        const float2 f = k2 > 0.0f ? pair_filter(P.pair, kx, ky, kz, __frcp_rn(k2)) : make_float2(0.f, 0.f);
        lines[c * LS + e] = make_float2(d.x * f.x - d.y * f.y, d.y * f.x + d.x * f.y);
      }
      __syncthreads();
      // inverse FFT along z
      if constexpr (REG) {
        fft1024_warp<1>(lines + (threadIdx.x >> 5) * LS, P.tw, tws, threadIdx.x & 31);
      } else {
        for (int c = team; c < kLines; c += TEAMS) {
          float2 *b = lines + c * LS;
          float2 v[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) v[r] = b[t + r * T];
          dft4<1>(v[0], v[1], v[2], v[3]);
          fft_finish<N2, 1, true>(b, v, tws, t, team);
        }
      }
      __syncthreads();
    }

    // ---- store
    if constexpr (MODE == kBoxInvXOut) {
      if (P.out) {
        // lines l = g kLines + c of x at (y, z) = (l mod n, l / n); each goes to every
        // periodic copy of its row in the (side)^2 rows of the layout
        const int S = P.out_side, mg = P.out_margin;
        for (int c = 0; c < kLines; ++c) {
          const int64_t l = g * kLines + c;
          const int y = static_cast<int>(l % M), z = static_cast<int>(l / M);
          for (int rz = -1; rz <= 1; ++rz) {
            const int zp = z + mg + rz * M;
            if (zp < 0 || zp >= S) continue;
            for (int ry = -1; ry <= 1; ++ry) {
              const int yp = y + mg + ry * M;
              if (yp < 0 || yp >= S) continue;
              float *row = P.out + ((static_cast<int64_t>(zp) * S + yp) * S) * P.out_stride + P.out_slot;
              for (int xp = threadIdx.x; xp < S; xp += THREADS) {
                const int x = ((xp - mg) % M + M) % M;
                const float2 v = lines[c * LS + x];
                if (P.out_stride == 1) {  // delta alone
                  row[xp] = v.x;
                } else {
                  *reinterpret_cast<float2 *>(row + static_cast<int64_t>(xp) * P.out_stride) =
                      make_float2(v.x, (P.pair == 3) ? 0.0f : v.y);
                }
              }
            }
          }
        }
      } else {
        for (int i = threadIdx.x; i < kLines * M; i += THREADS) {
          int c, e;
          flat_to_ce(0, i, M, c, e);
          P.work[line_addr(0, g, c, e, M)] = lines[c * LS + e];
        }
      }
    } else if (axis == 0) {
      for (int i = 2 * threadIdx.x; i < kLines * M; i += 2 * THREADS) {
        const int c = i / M, e = i % M;
        const float2 a = lines[c * LS + e], b = lines[c * LS + e + 1];
        *reinterpret_cast<float4 *>(P.work + line_addr(0, g, c, e, M)) = make_float4(a.x, a.y, b.x, b.y);
      }
    } else {
#pragma unroll 4
      for (int i = threadIdx.x; i < kLines * M; i += THREADS) {
        int c, e;
        flat_to_ce(axis, i, M, c, e);
        P.work[line_addr(axis, g, c, e, M)] = lines[c * LS + e];
      }
    }
    __syncthreads();
  }
}

template <int N2, int MODE>
cudaError_t launch_mode(const BoxPassParams &P, int sms, cudaStream_t st) {
  constexpr bool REG = N2 == 2048;
  constexpr int THREADS = BoxSmem<N2, REG>::THREADS;
  const size_t smem = BoxSmem<N2, REG>::bytes();
  cudaError_t e = cudaFuncSetAttribute(k_box_pass<N2, MODE, REG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_box_pass<N2, MODE, REG>, THREADS, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int64_t groups = static_cast<int64_t>(N2 / 2) * (N2 / 2) / kLines;
  const int grid = static_cast<int>(std::min<int64_t>(groups, static_cast<int64_t>(sms) * per_sm));
  k_box_pass<N2, MODE, REG><<<grid, THREADS, smem, st>>>(P);
  return cudaGetLastError();
}

template <int N2>
cudaError_t launch_n(const BoxPassParams &P, int mode, int sms, cudaStream_t st) {
  switch (mode) {
    case kBoxNoiseX: return launch_mode<N2, kBoxNoiseX>(P, sms, st);
    case kBoxFwd: return launch_mode<N2, kBoxFwd>(P, sms, st);
    case kBoxShapeZ: return launch_mode<N2, kBoxShapeZ>(P, sms, st);
    case kBoxSpecZ: return launch_mode<N2, kBoxSpecZ>(P, sms, st);
    case kBoxInv: return launch_mode<N2, kBoxInv>(P, sms, st);
    default: return launch_mode<N2, kBoxInvXOut>(P, sms, st);
  }
}

}  // namespace

cudaError_t launch_box_pass(const BoxPassParams &P, int mode, int sms, cudaStream_t st) {
  switch (P.lgn) {
    case 7: return launch_n<256>(P, mode, sms, st);
    case 8: return launch_n<512>(P, mode, sms, st);
    case 9: return launch_n<1024>(P, mode, sms, st);
    case 10: return launch_n<2048>(P, mode, sms, st);
    case 11: return launch_n<4096>(P, mode, sms, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mk
