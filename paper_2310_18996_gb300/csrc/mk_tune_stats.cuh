// The tuning-pass kernel: the FGPA of stored delta, eta and its statistics,
// with each team's next segment of the fields staged in shared memory.
#pragma once

#include "mk_skewer.cuh"

namespace mk {

// =================================================================== tuning-pass kernel
// The tuning pass (FGPA of stored delta, eta at full resolution, then the
// statistics): k_stats's pixel and P1D work, with each team's next segment of
// delta and eta copied into shared memory (cp.async, 16-byte pieces) while
// the current one is processed, so that the HBM latency hides behind the
// current segment's FFT.
// Shared memory: per-warp accumulators, the twiddle table, then per team two
// stage buffers of delta and eta (a segment's FFT runs in its own stage
// buffer once its fields are read).
template <int N>
struct TuneSmem {
  static constexpr int STAGE = N + 4;  // floats per field and buffer (a segment plus its 16-byte misalignment)
  static_assert(2 * STAGE >= 2 * TeamSmem<N>::BUF, "a stage buffer holds the FFT buffer");
  static size_t bytes(int threads, int n_z, int n_k) {
    return TeamSmem<N>::acc_bytes(threads, n_z, n_k, true) + TwTab<N>::BYTES +
           static_cast<size_t>(threads / (N / 8)) * 4 * STAGE * sizeof(float);
  }
};

// 16-byte copy of which the first nb bytes come from src and the rest are zero
// (nb = 0 reads nothing)
__device__ __forceinline__ void cp_async16z(void *dst, const void *src, int nb) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src), "r"(nb)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Where the tuning pass finds a segment: its first field index, pixels,
// first pixel-table index, and whether its pixels lie inside the tables.
struct TuneSeg {
  int64_t start;
  int npx, jb;
  bool ok;
};

// Stage the npx floats of a field from global index `start` into sd: N/4 + 1
// 16-byte pieces from start rounded down to 16 bytes (pixel p lands at
// sd[(start & 3) + p]); a piece's bytes past the segment are zero-filled, not
// read.  Thread t of the team copies pieces t and t + T (and t = 0 the last).
template <int N>
__device__ __forceinline__ void stage_field(float *sd, const float *__restrict__ f, int64_t start, int npx, int t) {
  constexpr int T = N / 8;
  const int shift = static_cast<int>(start & 3);
  const float *base = f + (start - shift);
  const int end = shift + npx;  // floats of the staged range that belong to the segment
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const int c = r < 2 ? t + r * T : N / 4;
    if (r == 2 && t != 0) break;
    const int nb = min(max(4 * (end - 4 * c), 0), 16);
    cp_async16z(sd + 4 * c, nb ? base + 4 * c : base, nb);
  }
}

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
  float *stage_buf = reinterpret_cast<float *>(smem + nwarps * wbytes + TwTab<N>::BYTES) + team * 4 * STAGE;
  const WarpAcc W = WarpAcc::at(smem + warp * wbytes, P.n_z, P.n_k);
  zero_warp_acc(smem + warp * wbytes, wbytes);
  fill_twiddles<N>(tws, P.tw);

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
  auto stage = [&](const TuneSeg &d, int b) {
    stage_field<N>(stage_buf + 2 * b * STAGE, P.delta, d.start, d.npx, t);
    stage_field<N>(stage_buf + (2 * b + 1) * STAGE, P.eta, d.start, d.npx, t);
  };
  TuneSeg cur{0, 0, 0, false};
  if (u < uend) {
    cur = describe(u);
    stage(cur, 0);
  }
  cp_async_commit();
  team_sync<T>(team);

  for (; u < uend; ++u) {
    const int b = static_cast<int>((u - u_first) & 1);
    TuneSeg nxt = cur;
    if (u + 1 < uend) {
      nxt = describe(u + 1);
      stage(nxt, b ^ 1);
    }
    cp_async_commit();  // one group per segment (possibly empty)
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
    cp_async_wait_prior();  // this segment's copies are in
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
