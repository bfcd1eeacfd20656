// The tuning-pass kernel: the FGPA of stored delta, eta and its statistics,
// with each team's next segment of the fields staged in shared memory.
#pragma once

#include "mk_skewer.cuh"

namespace mk {

// =================================================================== tuning-pass kernel
// The tuning pass (FGPA of stored delta, eta at full resolution, then the
// statistics): k_stats's pixel and P1D work, with each team's next segment of
// delta and eta copied into shared memory by the bulk-copy (TMA) engine while
// the current one is processed, so that the HBM latency hides behind the
// current segment's FFT.
// Shared memory: per-warp accumulators, the twiddle table, per team two stage
// buffers of delta and eta (a segment's FFT runs in its own stage buffer once
// its fields are read), then per team one mbarrier per stage buffer.
template <int N>
struct TuneSmem {
  static constexpr int STAGE = N + 4;  // floats per field and buffer (a segment plus its 16-byte misalignment)
  static_assert(2 * STAGE >= 2 * TeamSmem<N>::BUF, "a stage buffer holds the FFT buffer");
  static_assert((STAGE * sizeof(float)) % 16 == 0, "stage buffers start on 16 bytes");
  __host__ __device__ static size_t stage_bytes(int threads) {
    return static_cast<size_t>(threads / (N / 8)) * 4 * STAGE * sizeof(float);
  }
  static size_t bytes(int threads, int n_z, int n_k) {
    return TeamSmem<N>::acc_bytes(threads, n_z, n_k, true) + TwTab<N>::BYTES + stage_bytes(threads) +
           static_cast<size_t>(threads / (N / 8)) * 2 * sizeof(uint64_t);
  }
};

// ------------------------------------------------------------------ bulk copies
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
// the initialised barriers are visible to the bulk-copy engine
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// the one expected arrival of a phase, with the bytes its copies will bring
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for the phase of the given parity for at most `limit` clock cycles
// (the copies of a segment take microseconds); false when the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// earlier generic accesses of shared memory are ordered before later bulk copies into it
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// bytes (a multiple of 16, both addresses 16-byte aligned) from global to shared memory
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// true when pred holds on every thread of the team (a barrier of the team)
template <int T>
__device__ __forceinline__ bool team_all(int team, bool pred) {
  if constexpr (T == 32) {
    return __all_sync(0xffffffffu, pred);
  } else {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred pi, po;\n\tsetp.ne.u32 pi, %1, 0;\n\tbar.red.and.pred po, %2, %3, pi;\n\t"
        "selp.u32 %0, 1, 0, po;\n\t}"
        : "=r"(r)
        : "r"(static_cast<uint32_t>(pred)), "r"(team + 1), "r"(T)
        : "memory");
    return r != 0;
  }
}

// Where the tuning pass finds a segment: its first field index, pixels,
// first pixel-table index, whether its pixels lie inside the tables, and the
// segment's last (shift + npx) mod 4 floats of delta and eta (thread t holds
// float t of them), which the whole 16-byte pieces of the bulk copies leave.
struct TuneSeg {
  int64_t start;
  int npx, jb;
  bool ok;
  float td, te;
};

// P: a tuning pass (rebin 1, fields and FGPA table set; delta, eta 16-byte aligned).
template <int N>
__global__ void __launch_bounds__(256, 2) k_tune_stats(StatParams P) {
  constexpr int T = N / 8;
  constexpr int STAGE = TuneSmem<N>::STAGE;
  const int teams = blockDim.x / T;
  const int team = threadIdx.x / T, t = threadIdx.x % T, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  extern __shared__ __align__(16) unsigned char smem[];
  const size_t wbytes = WarpAcc::bytes(P.n_z, P.n_k);
  float2 *tws = reinterpret_cast<float2 *>(smem + nwarps * wbytes);
  // stage buffers b = 0, 1: delta at stage + 2 b STAGE, eta at stage + (2 b + 1) STAGE
  unsigned char *stage_base = smem + nwarps * wbytes + TwTab<N>::BYTES;
  float *stage_buf = reinterpret_cast<float *>(stage_base) + team * 4 * STAGE;
  uint64_t *bars = reinterpret_cast<uint64_t *>(stage_base + TuneSmem<N>::stage_bytes(blockDim.x)) + 2 * team;
  const WarpAcc W = WarpAcc::at(smem + warp * wbytes, P.n_z, P.n_k);
  zero_warp_acc(smem + warp * wbytes, wbytes);
  if (t == 0) {
    mbar_init(bars);
    mbar_init(bars + 1);
    mbar_init_fence();
  }
  fill_twiddles<N>(tws, P.tw);  // (ends with a CTA barrier)

  const int64_t nunits = P.segoff[P.n_sk];
  const int64_t g = static_cast<int64_t>(blockIdx.x) * teams + team;
  const int64_t G = static_cast<int64_t>(gridDim.x) * teams;
  int64_t u = g * nunits / G;
  const int64_t u_first = u;
  const int64_t uend = (g + 1) * nunits / G;
  int64_t i = u < uend ? upper_index(P.segoff, P.n_sk, u) : 0;
  int64_t inext = i;  // skewer of the segment to describe next
  const int wlo0 = t & ~31;
  PixelSums acc;
  acc.zero();
  int zc = -2;

  // describe segment uu (of skewer inext, advanced as needed); team-uniform
  auto describe = [&](int64_t uu) -> TuneSeg {
    while (P.segoff[inext + 1] <= uu) ++inext;
    const int64_t o = P.off_out[inext], nout = P.off_out[inext + 1] - o;
    const int64_t k0 = (uu - P.segoff[inext]) * N;
    const int64_t off = P.sk[inext].offset;
    const int j_lo = P.sk[inext].j_lo;
    TuneSeg d;
    d.start = off + k0;
    d.npx = static_cast<int>(min(static_cast<int64_t>(N), nout - k0));
    // records made for another pixel length may run past the pixel tables
    d.ok = j_lo >= 0 && j_lo + nout <= P.j_max;
    d.jb = d.ok ? j_lo + static_cast<int>(k0) : 0;
    return d;
  };
  // Copy segment d's fields into stage buffer b: thread 0 of the team issues
  // two bulk copies of the whole 16-byte pieces from d.start rounded down to
  // 16 bytes (pixel p lands at (start & 3) + p), completing on bars[b]; the
  // threads t < (shift + npx) mod 4 load the floats after the last piece.
  auto stage = [&](TuneSeg &d, int b) {
    const int shift = static_cast<int>(d.start & 3);
    const int nfl = (shift + d.npx) & ~3, tail = shift + d.npx - nfl;
    const float *bd = P.delta + (d.start - shift), *be = P.eta + (d.start - shift);
    d.td = t < tail ? __ldg(bd + nfl + t) : 0.f;
    d.te = t < tail ? __ldg(be + nfl + t) : 0.f;
    if (t == 0) {
      fence_async_shared();
      mbar_arrive_tx(bars + b, static_cast<uint32_t>(8 * nfl));
      if (nfl > 0 && !P.wait_test) {  // (the test hook leaves the expected bytes missing)
        bulk_g2s(stage_buf + 2 * b * STAGE, bd, static_cast<uint32_t>(4 * nfl), bars + b);
        bulk_g2s(stage_buf + (2 * b + 1) * STAGE, be, static_cast<uint32_t>(4 * nfl), bars + b);
      }
    }
  };
  uint32_t parity = 0;  // bit b: parity of stage buffer b's next phase
  bool staged_next = false;
  TuneSeg cur{0, 0, 0, false, 0.f, 0.f};
  if (u < uend) {
    cur = describe(u);
    stage(cur, 0);
  }

  for (; u < uend; ++u) {
    const int b = static_cast<int>((u - u_first) & 1);
    TuneSeg nxt = cur;
    staged_next = u + 1 < uend;
    if (staged_next) {
      nxt = describe(u + 1);
      stage(nxt, b ^ 1);
    }
    const int npx = cur.npx, jb = cur.jb;
    // the FGPA table and bin entries of this segment, requested before the
    // wait for the staged fields so that their latency overlaps it
    // (indices clamped to the segment's last pixel)
    const float4 *tp = P.pixtab + jb + t;
    float4 tb[8];
    int zs0 = 0;
    if (cur.ok) {
#pragma unroll
      for (int q = 0; q < 8; ++q) tb[q] = __ldg(tp + min(T * q, npx - 1 - t));
      zs0 = __ldg(P.zbin + jb);
    }
    // this segment's copies are in; its last floats join them from registers
    const long long limit = P.wait_test ? (1LL << 20) : (1LL << 31);  // cycles: ~0.5 ms, ~1 s
    const bool arrived = mbar_wait(bars + b, (parity >> b) & 1u, limit);
    parity ^= 1u << b;
    if (!team_all<T>(team, arrived)) {  // (team-uniform) the copies never completed
      if (t == 0) raise_error(P.err, ERR_TIMEOUT);
      if (staged_next) mbar_wait(bars + (b ^ 1), (parity >> (b ^ 1)) & 1u, limit);  // before leaving
      break;
    }
    {
      const int shift = static_cast<int>(cur.start & 3);
      const int nfl = (shift + npx) & ~3;
      if (t < shift + npx - nfl) {
        stage_buf[2 * b * STAGE + nfl + t] = cur.td;
        stage_buf[(2 * b + 1) * STAGE + nfl + t] = cur.te;
      }
    }
    team_sync<T>(team);
    if (!cur.ok) {  // skip the segment, as k_stats does
      if (t == 0) raise_error(P.err, ERR_RANGE);
      team_sync<T>(team);
      cur = nxt;
      continue;
    }
    const int shift = static_cast<int>(cur.start & 3);
    const float *sd = stage_buf + 2 * b * STAGE + shift, *se = stage_buf + (2 * b + 1) * STAGE + shift;
    // the segment's FFT buffer: its own stage buffer, written once every
    // field value of the segment has been read
    float2 *buf = reinterpret_cast<float2 *>(stage_buf + 2 * b * STAGE);
    float *fb = reinterpret_cast<float *>(buf);
    if (zs0 != zc) {
      if (zc != -2) flush_bin_sums(W, P.n_z, zc, acc, lane);
      acc.zero();
      zc = zs0;
    }
    int pend = __ldg(P.bin_end + zc + 1) - jb;
    const bool one_bin = min(T * 7 + wlo0 + 32, npx) <= pend;
    float2 xv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      xv[q] = t + T * q < npx ? make_float2(sd[t + T * q], se[t + T * q]) : make_float2(0.f, 0.f);
    team_sync<T>(team);  // every field value read before fb overwrites the buffer
    if (npx == N && one_bin) {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float f = fgpa(tb[q], xv[q].x, xv[q].y);
        acc.add_sums(f, xv[q]);
        fb[t + T * q] = f;
      }
      acc.n += 8.f;  // this thread's pixels of the segment
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {  // (unrolled: tb[q] and xv[q] stay in registers)
        const int p = t + T * q;
        float f = 0.f;
        const float2 x = xv[q];
        if (p < npx) f = fgpa(tb[q], x.x, x.y);
        if (one_bin) {
          if (p < npx) acc.add(f, x);
        } else {
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
    if (npx == N) {
      const int zs = __ldg(P.segzbin + jb);
      if (zs >= 0 && zs < P.n_z) {
        forward_packed_fft<N>(buf, tws, t, team);
        float pk[4];
        power_of_modes<N>(buf, P.tw, t, pk);
        accumulate_p1d<N>(W, P.n_k, pk, P.p1d_scale, zs, t);
        if (t == 0) W.nseg[zs] += 1u;
      }
    }
    team_sync<T>(team);  // the stage buffer b and fb are free again
    cur = nxt;
  }
  if (zc != -2) flush_bin_sums(W, P.n_z, zc, acc, lane);
  flush_warp_partials(smem, nwarps, wbytes, P.n_z, P.n_k, P.partials);
}

}  // namespace mk
