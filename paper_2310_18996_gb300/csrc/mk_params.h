// Kernel parameter blocks shared by the host launch code and the kernels.
#pragma once

#include <stdint.h>

#include "../../include/mockskewer.h"

namespace mk {

// error bits of the device error word
enum : int { ERR_RANGE = 1, ERR_CAPACITY = 2, ERR_TIMEOUT = 4 };

// bin_end entry of a z bin that no tabulated pixel leaves
constexpr int32_t kBinEndNever = 1 << 30;

// Cubic-Hermite table of D_C(z) on z_i = i h: values and slopes c/(H0 E(z_i)).
struct DcTable {
  const double2 *dc;  // {D_C(z_i), dD_C/dz(z_i)}
  int n;              // entries
  double h;           // z spacing
  double omega_m;     // for E(z) in the Newton inversion
  const double *zr;   // z(r_i) on r_i = i hr: the starting point of the inversion
  int n_r;            // entries
  double inv_hr;      // 1 / hr
};

struct GeomParams {
  DcTable tab;
  double lambda_lya, dr, lrf_min, lrf_max, lobs_min;
  int32_t n_min, n_max;
  double origin[3], cell;
  int32_t j_max;  // pixel tables cover J < j_max
  int32_t n_fft;  // segment length for the segment count (0: none)
  int32_t rebin;  // > 0: write floor(n / rebin) counts instead (flux offsets)
};

using NodeParams = mk_fgpa_nodes;

// FP64 accumulators of one team in shared memory:
//   sums[n_z][NSUM], p1d[n_z][n_k], nseg[n_z]
struct StatLayout {
  int n_z, n_k;
  __host__ __device__ int sums(int zb, int i) const { return zb * MK_NSUM + i; }
  __host__ __device__ int p1d(int zb, int k) const { return n_z * MK_NSUM + zb * n_k + k; }
  __host__ __device__ int nseg(int zb) const { return n_z * (MK_NSUM + n_k) + zb; }
  __host__ __device__ int size() const { return n_z * (MK_NSUM + n_k + 1); }
};

// Derived statistics of z bin zb from its raw sums (out->sums[zb],
// p1d_sum[zb], n_seg[zb]), which the caller has filled: F-bar, sigma_F,
// P1D_F per mode, P1D_F / F-bar^2, and b_F, beta_F from the least-squares
// fit F ~ F0 + k_d delta + k_e eta (Sec. 2.6, Sec. 4.1).  per_bin: modes per k
// bin, (n_fft / 2) / n_k.  The finalize kernel and the host-side merge of
// per-rank sums (mk_stats_merge) both use it.
__host__ __device__ inline void finalize_bin(mk_stats_out *out, int zb, int n_k, double per_bin) {
  const double *s = out->sums[zb];
  const double n = s[0];
  if (n <= 0.0) return;
  const double fbar = s[1] / n;
  out->mean_flux[zb] = fbar;
  const double varf = s[2] / n - fbar * fbar;
  out->sigma_f[zb] = varf > 0.0 ? sqrt(varf) : 0.0;
  const double md = s[3] / n, me = s[4] / n;
  const double cdd = s[5] / n - md * md, cee = s[6] / n - me * me, cde = s[7] / n - md * me;
  const double vfd = s[8] / n - fbar * md, vfe = s[9] / n - fbar * me;
  const double det = cdd * cee - cde * cde;
  if (det != 0.0) {
    const double kd = (cee * vfd - cde * vfe) / det;
    const double ke = (cdd * vfe - cde * vfd) / det;
    out->b_f[zb] = kd / fbar;
    out->beta_f[zb] = kd != 0.0 ? ke / kd : 0.0;
  }
  const double ns = out->n_seg[zb];
  if (ns > 0.0) {
    for (int k = 0; k < n_k; ++k) {
      out->p1d_f[zb][k] = out->p1d_sum[zb][k] / (ns * per_bin);
      out->p1d_df[zb][k] = out->p1d_f[zb][k] / (fbar * fbar);
    }
  }
}

// Everything the fused / split skewer kernels read.
struct SkewerParams {
  const mk_skewer *sk;
  const int64_t *segoff;  // exclusive prefix of segments per skewer, n_sk + 1
  int64_t n_sk;
  // box
  const float *box_d;  // planar delta, or (delta, eta) pairs (interleaved, padded)
  const float *box_e;  // planar eta or NULL
  int32_t lgn;
  // tables
  const float4 *pixtab;  // per global pixel J: {G, a log2e, b log2e, c}
  const int16_t *zbin;     // per J: z bin, -1 below, n_z above
  const int16_t *segzbin;  // per J: z bin of the mean z of pixels J .. J+N-1
  const int32_t *bin_end;  // [k + 1], k = -1 .. n_z: first J with zbin > k (large beyond the tables)
  const double *cumz;      // per J: sum_{J' < J} z_J'
  const float *amp;        // A_m / N, m = 0..N/2; with ps_nodes >= 2: (A_m / N)^2 per node, node-major
  int32_t ps_nodes;        // z-dependent small-scale power: tables at ps_z (>= 2), else one
  float ps_z[MK_MAX_NODES];
  const float *zwin;       // per J: mean z of pixels J .. J+N-1 (with ps_nodes >= 2)
  const float2 *tw;      // e^{-2 pi i k/N}, k < N
  uint32_t seed;
  int32_t j_max;
  // outputs
  float *delta_out, *eta_out, *flux_out;
  int64_t capacity;
  // statistics
  int32_t do_stats;
  int32_t n_z, n_k;
  double z_lo, dz, dr;
  float p1d_scale;   // dr / N
  double *partials;  // [gridDim.x][layout size]
  int *err;
};

// Statistics pass over stored flux (any rebin).
struct StatParams {
  const mk_skewer *sk;
  const int64_t *off_out;  // output offsets, n_sk + 1
  const int64_t *segoff;   // prefix of ceil(n_out / N) per skewer
  int64_t n_sk;
  const float *flux;         // stored flux, or NULL with pixtab set
  const float *delta, *eta;  // fine fields or NULL
  const float4 *pixtab;      // tuning pass: FGPA table; the flux is computed from delta, eta
  int32_t rebin;
  const int16_t *zbin;
  const int16_t *segzbin;
  const int32_t *bin_end;  // first pixel J past each z bin (index zbin + 1), as in SkewerParams
  const double *cumz;
  const float2 *tw;
  int32_t j_max;
  int32_t n_z, n_k;
  double z_lo, dz, dr;
  float p1d_scale;  // rebin dr / N
  double *partials;
  int *err;
  int32_t wait_test;  // test hook: the tuning pass issues no bulk copies and waits ~2^20 cycles at most
};

struct FluxParams {
  const mk_skewer *sk;
  const int64_t *off_out;
  int64_t n_sk;
  const float *delta, *eta;
  const float4 *pixtab;
  int32_t rebin;
  int32_t j_max;
  float *flux;
  int64_t capacity;
  int *err;
};

}  // namespace mk
