// C-ABI of the skewer-synthesis library: context, tables, entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/mockskewer.h"
#include "mk_kernels.h"
#include "mk_trace.h"

using namespace mk;

namespace {

constexpr double kCH = 2997.92458;  // c/H0 [Mpc/h]
constexpr double kZMax = 12.0;      // redshift range of the tables
constexpr double kDcStep = 1.0 / 512.0;
constexpr double kZrStep = 1.0;  // Mpc/h, spacing of the z(r) starting table

// ------------------------------------------------------------------ host cosmology
// Flat LCDM, Omega_L = 1 - Omega_M (Table 1).  D_C is tabulated on a uniform
// z grid by composite Simpson integration of c/(H0 E); values between nodes
// come from cubic Hermite interpolation with the exact slopes.  The growth
// factor solves the linear growth equation in ln a by classical RK4.
struct HostCosmo {
  double om = 0.3147;
  std::vector<double> dc, slope;  // on z_i = i kDcStep
  std::vector<double> lna, gD, gDp;  // growth D(ln a) and dD/dln a
  double lna0 = 0.0, dlna = 0.0, d_today = 1.0;

  double e(double z) const {
    const double zp = 1.0 + z;
    return std::sqrt(om * zp * zp * zp + (1.0 - om));
  }

  void build(double omega_m) {
    om = omega_m;
    const int n = static_cast<int>(kZMax / kDcStep) + 2;
    dc.assign(n, 0.0);
    slope.assign(n, 0.0);
    const int sub = 32;  // Simpson panels per table step
    for (int i = 0; i < n; ++i) {
      const double z = i * kDcStep;
      slope[i] = kCH / e(z);
      if (i == 0) continue;
      const double a = z - kDcStep, hh = kDcStep / sub;
      double s = kCH / e(a) + kCH / e(z);
      for (int k = 1; k < sub; ++k) s += (k & 1 ? 4.0 : 2.0) * kCH / e(a + k * hh);
      dc[i] = dc[i - 1] + s * hh / 3.0;
    }
    // growth: y = (D, D'), ' = d/dln a;  D'' + (2 - 1.5 Om(a)) D' - 1.5 Om(a) D = 0
    // starting deep in matter domination where D = a is the growing mode.
    const int steps = 24000;
    lna0 = std::log(1e-4);
    dlna = -lna0 / steps;
    lna.resize(steps + 1);
    gD.resize(steps + 1);
    gDp.resize(steps + 1);
    auto om_a = [&](double x) {
      const double a3 = std::exp(3.0 * x);
      return om / (om + (1.0 - om) * a3);
    };
    auto rhs = [&](double x, double d, double dp, double &dd, double &ddp) {
      const double w = om_a(x);
      dd = dp;
      ddp = -(2.0 - 1.5 * w) * dp + 1.5 * w * d;
    };
    double x = lna0, d = std::exp(lna0), dp = d;
    for (int s = 0; s <= steps; ++s) {
      lna[s] = x;
      gD[s] = d;
      gDp[s] = dp;
      if (s == steps) break;
      double k1d, k1p, k2d, k2p, k3d, k3p, k4d, k4p;
      rhs(x, d, dp, k1d, k1p);
      rhs(x + 0.5 * dlna, d + 0.5 * dlna * k1d, dp + 0.5 * dlna * k1p, k2d, k2p);
      rhs(x + 0.5 * dlna, d + 0.5 * dlna * k2d, dp + 0.5 * dlna * k2p, k3d, k3p);
      rhs(x + dlna, d + dlna * k3d, dp + dlna * k3p, k4d, k4p);
      d += dlna / 6.0 * (k1d + 2 * k2d + 2 * k3d + k4d);
      dp += dlna / 6.0 * (k1p + 2 * k2p + 2 * k3p + k4p);
      x += dlna;
    }
    d_today = gD[steps];
  }

  static double hermite(double y0, double y1, double s0, double s1, double h, double t) {
    const double t2 = t * t, t3 = t2 * t;
    return (2 * t3 - 3 * t2 + 1) * y0 + (t3 - 2 * t2 + t) * h * s0 + (-2 * t3 + 3 * t2) * y1 +
           (t3 - t2) * h * s1;
  }

  double distance(double z) const {
    double s = z / kDcStep;
    int i = static_cast<int>(std::floor(s));
    if (i < 0) i = 0;
    if (i > static_cast<int>(dc.size()) - 2) i = static_cast<int>(dc.size()) - 2;
    return hermite(dc[i], dc[i + 1], slope[i], slope[i + 1], kDcStep, s - i);
  }

  double z_of(double r) const {
    int lo = 0, hi = static_cast<int>(dc.size()) - 1;
    while (hi - lo > 1) {
      const int mid = (lo + hi) / 2;
      if (dc[mid] <= r) lo = mid; else hi = mid;
    }
    double z = (lo + (r - dc[lo]) / (dc[hi] - dc[lo])) * kDcStep;
    for (int it = 0; it < 5; ++it) z -= (distance(z) - r) / (kCH / e(z));
    return z;
  }

  double growth(double z) const {
    const double x = -std::log1p(z);
    double s = (x - lna0) / dlna;
    int i = static_cast<int>(std::floor(s));
    if (i < 0) i = 0;
    if (i > static_cast<int>(gD.size()) - 2) i = static_cast<int>(gD.size()) - 2;
    return hermite(gD[i], gD[i + 1], gDp[i], gDp[i + 1], dlna, s - i) / d_today;
  }
};

}  // namespace

// ====================================================================== context
struct mk_box {
  mk_box_desc desc;
  const float *d;
  const float *e;
  int lgn;
};

struct LaunchCfg {
  int threads;  // CTA size of the fused kernel
  int minb;     // register budget of the instance: that of minb 256-thread CTAs per SM (2, 3 or 4)
};

struct mk_ctx {
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  mk_cosmo cosmo{};
  std::string err;
  HostCosmo cos;
  double2 *d_dc = nullptr;
  int n_dc = 0;
  double *d_zr = nullptr;  // z(r) on r_i = i kZrStep
  int n_zr = 0;
  int *d_err = nullptr;
  int *h_err = nullptr;  // pinned
  // pixel tables (per dr)
  double dr = -1.0;
  int32_t j_max = 0;
  double *d_zpix = nullptr, *d_cumz = nullptr;
  float *d_gpix = nullptr;
  float4 *d_pixtab = nullptr;
  int16_t *d_zbin = nullptr, *d_segzbin = nullptr;
  int32_t *d_bin_end = nullptr;  // MK_MAX_ZBINS + 2 entries
  bool pixtab_valid = false;
  mk_fgpa_nodes nodes_key{};
  bool zbin_valid = false;
  mk_stat_bins bins_key{};
  // small-scale amplitudes and twiddles
  float *d_amp = nullptr;
  std::vector<double> amp_key;
  int ps_nodes = 1;  // node tables in d_amp (>= 2: squared amplitudes per node)
  float ps_z[MK_MAX_NODES] = {};
  float *d_pk = nullptr;    // P(k) table of the box synthesis
  int n_pk_cap = 0;
  float *d_zwin = nullptr;  // window mean z per J for segments of zwin_n pixels
  int zwin_n = 0;
  double zwin_dr = -1.0;
  float2 *d_tw[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // N = 256 .. 4096 (4096: box lines of 2048)
  // workspaces
  int64_t *d_cnt_px = nullptr, *d_cnt_seg = nullptr, *d_segoff = nullptr;
  int64_t cnt_cap = 0;
  void *d_scan_ws = nullptr;
  size_t scan_cap = 0;
  double *d_partials = nullptr;
  size_t partials_cap = 0;  // doubles
  mk_stats_out *d_stats = nullptr, *h_stats = nullptr;
  int64_t *h_total = nullptr;  // pinned
  int skewer_threads = 256;
  // launch configurations chosen by the autotuner, per kernel variant
  std::map<uint64_t, LaunchCfg> tuned;
  // captured graph of the last mk_run with MK_GRAPH, and what it was made from
  cudaGraphExec_t graph = nullptr;
  std::vector<unsigned char> graph_key;
  uint64_t generation = 0;  // bumped whenever a table or workspace moves
  bool timing = false;
  bool timed = false;
  unsigned char *static_scratch = nullptr;  // device address of mk_stats_static's array
  int grid_cap = 0;  // at most this many CTAs for the persistent kernels (0: no cap)
  int wait_test = 0;  // test hook of the tuning pass's bounded wait (mk_set_wait_test)
  int fault = 0;      // test hook: MK_FAULT_ALLOC or MK_FAULT_LAUNCH fails the next such step once
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // mk_run_host: device copies of the catalogue and records, two staging
  // buffers, slice boundaries, copy streams and their events
  void *d_hq = nullptr, *d_hsk = nullptr, *d_hoff = nullptr;
  size_t hq_cap = 0, hsk_cap = 0, hoff_cap = 0;
  void *d_stage[2] = {nullptr, nullptr};
  size_t stage_cap[2] = {0, 0};
  int64_t *d_pick = nullptr, *h_pick = nullptr;  // MK_MAX_CHUNKS + 1
  cudaStream_t copy_st[MK_HOST_COPY_STREAMS] = {};
  cudaEvent_t ev_done[MK_MAX_CHUNKS] = {};
  cudaEvent_t ev_copy[MK_HOST_COPY_STREAMS][MK_MAX_CHUNKS] = {};
  bool host_ready = false;
};

namespace {

int fail(mk_ctx *ctx, int code, const char *fmt, ...) {
  char msg[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return fail(ctx, MK_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// the injected failure of kind `kind`, once (mk_inject_fault)
int take_fault(mk_ctx *ctx, int kind) {
  if (ctx->fault != kind) return MK_OK;
  ctx->fault = 0;
  return kind == MK_FAULT_ALLOC ? fail(ctx, MK_ENOMEM, "injected device allocation failure")
                                : fail(ctx, MK_ECUDA, "injected kernel launch failure");
}

int grow(mk_ctx *ctx, void **p, size_t *cap, size_t need) {
  if (*cap >= need && *p) return MK_OK;
  if (int rc = take_fault(ctx, MK_FAULT_ALLOC)) return rc;  // (the old buffer stays as it was)
  ++ctx->generation;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, need) != cudaSuccess) {
    *p = nullptr;
    return fail(ctx, MK_ENOMEM, "device allocation of %zu bytes failed", need);
  }
  *cap = need;
  return MK_OK;
}

int ensure_counts(mk_ctx *ctx, int64_t n) {
  // (the scan workspace is checked as well: an earlier call may have failed to grow it)
  if (ctx->cnt_cap >= n + 1 && ctx->d_cnt_px) return grow(ctx, &ctx->d_scan_ws, &ctx->scan_cap, scan_workspace_bytes(n));
  ++ctx->generation;
  cudaFree(ctx->d_cnt_px);
  cudaFree(ctx->d_cnt_seg);
  cudaFree(ctx->d_segoff);
  ctx->d_cnt_px = ctx->d_cnt_seg = ctx->d_segoff = nullptr;
  ctx->cnt_cap = 0;
  const size_t bytes = sizeof(int64_t) * static_cast<size_t>(n + 1);
  if (cudaMalloc(&ctx->d_cnt_px, bytes) != cudaSuccess || cudaMalloc(&ctx->d_cnt_seg, bytes) != cudaSuccess ||
      cudaMalloc(&ctx->d_segoff, bytes) != cudaSuccess)
    return fail(ctx, MK_ENOMEM, "count workspace (%lld skewers)", static_cast<long long>(n));
  ctx->cnt_cap = n + 1;
  return grow(ctx, &ctx->d_scan_ws, &ctx->scan_cap, scan_workspace_bytes(n));
}

int ensure_pixel_tables(mk_ctx *ctx, double dr) {
  if (ctx->dr == dr && ctx->d_zpix) return MK_OK;
  ++ctx->generation;
  const double rmax = ctx->cos.distance(kZMax - 2 * kDcStep);
  const int32_t jmax = static_cast<int32_t>(std::floor(rmax / dr)) - 1;
  std::vector<double> z(jmax), cz(jmax + 1);
  std::vector<float> g(jmax);
  cz[0] = 0.0;
  for (int32_t j = 0; j < jmax; ++j) {
    z[j] = ctx->cos.z_of((j + 0.5) * dr);
    g[j] = static_cast<float>(ctx->cos.growth(z[j]));
    cz[j + 1] = cz[j] + z[j];
  }
  cudaFree(ctx->d_zpix);
  cudaFree(ctx->d_cumz);
  cudaFree(ctx->d_gpix);
  cudaFree(ctx->d_pixtab);
  cudaFree(ctx->d_zbin);
  cudaFree(ctx->d_segzbin);
  cudaFree(ctx->d_zwin);
  ctx->d_zwin = nullptr;
  ctx->d_zpix = ctx->d_cumz = nullptr;
  ctx->d_gpix = nullptr;
  ctx->d_pixtab = nullptr;
  ctx->d_zbin = ctx->d_segzbin = nullptr;
  if (cudaMalloc(&ctx->d_zpix, sizeof(double) * jmax) != cudaSuccess ||
      cudaMalloc(&ctx->d_cumz, sizeof(double) * (jmax + 1)) != cudaSuccess ||
      cudaMalloc(&ctx->d_gpix, sizeof(float) * jmax) != cudaSuccess ||
      cudaMalloc(&ctx->d_pixtab, sizeof(float4) * jmax) != cudaSuccess ||
      cudaMalloc(&ctx->d_zbin, sizeof(int16_t) * jmax) != cudaSuccess ||
      cudaMalloc(&ctx->d_segzbin, sizeof(int16_t) * jmax) != cudaSuccess)
    return fail(ctx, MK_ENOMEM, "pixel tables");
  CK(cudaMemcpy(ctx->d_zpix, z.data(), sizeof(double) * jmax, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_cumz, cz.data(), sizeof(double) * (jmax + 1), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(ctx->d_gpix, g.data(), sizeof(float) * jmax, cudaMemcpyHostToDevice));
  ctx->dr = dr;
  ctx->j_max = jmax;
  ctx->pixtab_valid = false;
  ctx->zbin_valid = false;
  return MK_OK;
}

int tw_slot(int n_fft) {
  switch (n_fft) {
    case 256: return 0;
    case 512: return 1;
    case 1024: return 2;
    case 2048: return 3;
    case 4096: return 4;
  }
  return -1;
}

// FFT lengths of the skewer and statistics kernels (the 4096 table serves the
// box synthesis only)
bool skewer_fft(int n_fft) { return n_fft == 256 || n_fft == 512 || n_fft == 1024 || n_fft == 2048; }

int ensure_twiddles(mk_ctx *ctx, int n_fft) {
  const int slot = tw_slot(n_fft);
  if (ctx->d_tw[slot]) return MK_OK;
  ++ctx->generation;
  std::vector<float2> tw(n_fft);
  for (int k = 0; k < n_fft; ++k) {
    const double a = 2.0 * M_PI * k / n_fft;
    tw[k] = make_float2(static_cast<float>(std::cos(a)), static_cast<float>(-std::sin(a)));
  }
  CK(cudaMalloc(&ctx->d_tw[slot], sizeof(float2) * n_fft));
  CK(cudaMemcpy(ctx->d_tw[slot], tw.data(), sizeof(float2) * n_fft, cudaMemcpyHostToDevice));
  return MK_OK;
}

int ensure_amp(mk_ctx *ctx, const mk_skewer_params *p) {
  const int m = p->n_fft / 2;
  const int nodes = p->p_s_nodes >= 2 ? p->p_s_nodes : 1;
  std::vector<double> key(3 + nodes * (m + 2));
  key[0] = p->n_fft;
  key[1] = p->dr;
  key[2] = nodes;
  for (int k = 0; k < nodes; ++k) {
    key[3 + k] = nodes > 1 ? p->h_p_s_z[k] : 0.0;
    for (int i = 0; i <= m; ++i) key[3 + nodes + k * (m + 1) + i] = p->h_p_s[k * (m + 1) + i];
  }
  if (!(key == ctx->amp_key && ctx->d_amp)) {
    std::vector<float> amp(static_cast<size_t>(nodes) * (m + 1));
    for (int k = 0; k < nodes; ++k)
      for (int i = 0; i <= m; ++i) {
        const double ps = p->h_p_s[k * (m + 1) + i];
        if (!(ps >= 0.0)) return fail(ctx, MK_EINVAL, "P_S[%d][%d] must be >= 0", k, i);
        const double a2 = p->n_fft * ps / p->dr / (static_cast<double>(p->n_fft) * p->n_fft);
        // one table: A_m / N; node tables: (A_m / N)^2, interpolated in z then square-rooted
        amp[k * (m + 1) + i] = static_cast<float>(i == 0 ? 0.0 : (nodes > 1 ? a2 : std::sqrt(a2)));
      }
    cudaFree(ctx->d_amp);
    ctx->d_amp = nullptr;
    ++ctx->generation;
    CK(cudaMalloc(&ctx->d_amp, sizeof(float) * amp.size()));
    CK(cudaMemcpy(ctx->d_amp, amp.data(), sizeof(float) * amp.size(), cudaMemcpyHostToDevice));
    ctx->amp_key = key;
    ctx->ps_nodes = nodes;
    for (int k = 0; k < nodes && nodes > 1; ++k) ctx->ps_z[k] = static_cast<float>(p->h_p_s_z[k]);
  }
  if (nodes > 1 && (ctx->zwin_n != p->n_fft || ctx->zwin_dr != ctx->dr || !ctx->d_zwin)) {
    if (!ctx->d_zwin) {
      ++ctx->generation;
      CK(cudaMalloc(&ctx->d_zwin, sizeof(float) * ctx->j_max));
    }
    CK(launch_zwin(ctx->d_cumz, ctx->j_max, p->n_fft, ctx->d_zwin, ctx->stream));
    ctx->zwin_n = p->n_fft;
    ctx->zwin_dr = ctx->dr;
  }
  return MK_OK;
}

int check_params(mk_ctx *ctx, const mk_skewer_params *p, bool need_ps) {
  if (!p) return fail(ctx, MK_EINVAL, "params is NULL");
  if (!(p->dr > 0.0) || p->dr > 100.0) return fail(ctx, MK_EINVAL, "dr must be in (0, 100]");
  if (!(p->lrf_min > 0.0) || !(p->lrf_max > p->lrf_min)) return fail(ctx, MK_EINVAL, "bad forest window");
  if (p->n_min < 0 || p->n_max < 0) return fail(ctx, MK_EINVAL, "n_min/n_max must be >= 0");
  if (!skewer_fft(p->n_fft)) return fail(ctx, MK_EINVAL, "n_fft must be 256, 512, 1024 or 2048");
  if (need_ps && !p->h_p_s) return fail(ctx, MK_EINVAL, "h_p_s is NULL");
  if (p->p_s_nodes < 0 || p->p_s_nodes > MK_MAX_NODES)
    return fail(ctx, MK_EINVAL, "p_s_nodes must be in [0, %d]", MK_MAX_NODES);
  if (p->p_s_nodes >= 2) {
    if (!p->h_p_s_z) return fail(ctx, MK_EINVAL, "h_p_s_z is NULL");
    for (int k = 1; k < p->p_s_nodes; ++k)
      if (!(p->h_p_s_z[k] > p->h_p_s_z[k - 1])) return fail(ctx, MK_EINVAL, "h_p_s_z must increase");
  }
  if (p->interp != MK_INTERP_TRILINEAR && p->interp != MK_INTERP_GAUSS7)
    return fail(ctx, MK_EINVAL, "interp must be MK_INTERP_TRILINEAR or MK_INTERP_GAUSS7");
  return MK_OK;
}

int check_nodes(mk_ctx *ctx, const mk_fgpa_nodes *nd) {
  if (!nd || nd->count < 1 || nd->count > MK_MAX_NODES) return fail(ctx, MK_EINVAL, "bad FGPA node count");
  for (int i = 1; i < nd->count; ++i)
    if (!(nd->z[i] > nd->z[i - 1])) return fail(ctx, MK_EINVAL, "FGPA node z must increase");
  return MK_OK;
}

int check_bins(mk_ctx *ctx, const mk_stat_bins *b) {
  if (!b || b->n_z < 1 || b->n_z > MK_MAX_ZBINS) return fail(ctx, MK_EINVAL, "bad n_z");
  if (!(b->dz > 0.0)) return fail(ctx, MK_EINVAL, "dz must be > 0");
  if (!skewer_fft(b->n_fft)) return fail(ctx, MK_EINVAL, "bins n_fft must be 256, 512, 1024 or 2048");
  if (b->n_k < 1 || b->n_k > MK_MAX_KBINS || (b->n_fft / 2) % b->n_k)
    return fail(ctx, MK_EINVAL, "n_k must divide n_fft/2 and be <= %d", MK_MAX_KBINS);
  return MK_OK;
}

int ensure_pixtab(mk_ctx *ctx, const mk_fgpa_nodes *nd) {
  if (ctx->pixtab_valid && std::memcmp(&ctx->nodes_key, nd, sizeof(*nd)) == 0) return MK_OK;
  CK(launch_pixtab(ctx->d_zpix, ctx->d_gpix, ctx->j_max, *nd, ctx->d_pixtab, ctx->stream));
  ctx->nodes_key = *nd;
  ctx->pixtab_valid = true;
  return MK_OK;
}

int ensure_zbin(mk_ctx *ctx, const mk_stat_bins *b) {
  if (ctx->zbin_valid && std::memcmp(&ctx->bins_key, b, sizeof(*b)) == 0) return MK_OK;
  if (!ctx->d_bin_end) {
    ++ctx->generation;
    CK(cudaMalloc(&ctx->d_bin_end, sizeof(int32_t) * (MK_MAX_ZBINS + 2)));
  }
  CK(launch_zbin(ctx->d_zpix, ctx->d_cumz, ctx->j_max, b->z_lo, b->dz, b->n_z, b->n_fft, ctx->d_zbin,
                 ctx->d_segzbin, ctx->stream));
  CK(launch_bin_end(ctx->d_zbin, ctx->j_max, b->n_z, ctx->d_bin_end, ctx->stream));
  ctx->bins_key = *b;
  ctx->zbin_valid = true;
  return MK_OK;
}

int read_error_word(mk_ctx *ctx) {
  CK(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int e = *ctx->h_err;
  if (e) {
    CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (e & ERR_TIMEOUT) return fail(ctx, MK_ETIMEOUT, "a device wait timed out");
    if (e & ERR_CAPACITY) return fail(ctx, MK_ERANGE, "output larger than the stated capacity");
    return fail(ctx, MK_ERANGE, "pixel outside the redshift tables (z > %.1f)", kZMax);
  }
  return MK_OK;
}

int time_begin(mk_ctx *ctx) {
  if (ctx->timing) CK(cudaEventRecord(ctx->ev0, ctx->stream));
  return MK_OK;
}

int time_end(mk_ctx *ctx) {
  if (ctx->timing) {
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    ctx->timed = true;
  }
  return MK_OK;
}

// persistent grids: as many resident CTAs as the SMs hold
// (at most ctx->grid_cap CTAs when a cap is set)
int capped(mk_ctx *ctx, int grid) { return ctx->grid_cap > 0 && grid > ctx->grid_cap ? ctx->grid_cap : grid; }

int skewer_grid(mk_ctx *ctx, int n_fft, int variant, int lgn, LaunchCfg cfg, const mk_stat_bins *bins) {
  return capped(ctx, ctx->sms * skewer_blocks_per_sm(n_fft, variant, lgn, cfg.minb, cfg.threads,
                                                     bins ? bins->n_z : 0, bins ? bins->n_k : 0, bins != nullptr));
}

// default launch: 256-thread CTAs with the register budget of three per SM
// (85 registers; measured fastest on GB300 for N = 256)
LaunchCfg default_cfg(int n_fft) {
  (void)n_fft;
  return LaunchCfg{256, 3};
}

// kernel variant: the box layout, plus kGauss7Variant for the Gaussian kernel,
// plus kPsNodesVariant for P_s tables at several redshifts
int kernel_variant(const mk_box *box, const mk_skewer_params *p) {
  return box->desc.layout | (p->interp == MK_INTERP_GAUSS7 ? kGauss7Variant : 0) |
         (p->p_s_nodes >= 2 ? kPsNodesVariant : 0);
}

int check_interp(mk_ctx *ctx, const mk_box *box, const mk_skewer_params *p) {
  if (p->interp == MK_INTERP_GAUSS7 && box->desc.layout != MK_BOX_HALO)
    return fail(ctx, MK_EINVAL, "MK_INTERP_GAUSS7 needs an MK_BOX_HALO box");
  return MK_OK;
}

uint64_t tune_key(int n_fft, int variant, int lgn, uint32_t flags) {
  return (static_cast<uint64_t>(n_fft) << 32) | (static_cast<uint64_t>(variant) << 16) |
         (static_cast<uint64_t>(lgn > 10) << 8) | (flags & (MK_STORE_FIELDS | MK_STORE_FLUX | MK_STATS));
}

int stats_grid(mk_ctx *ctx, const mk_stat_bins *bins, int threads, bool tune = false) {
  return capped(ctx, ctx->sms * stats_blocks_per_sm(bins->n_fft, threads, bins->n_z, bins->n_k, tune));
}

GeomParams geom_params(mk_ctx *ctx, const mk_box *box, const mk_skewer_params *p) {
  GeomParams G;
  std::memset(&G, 0, sizeof(G));
  G.tab = DcTable{ctx->d_dc, ctx->n_dc, kDcStep, ctx->cosmo.omega_m, ctx->d_zr, ctx->n_zr, 1.0 / kZrStep};
  G.lambda_lya = ctx->cosmo.lambda_lya;
  G.dr = p->dr;
  G.lrf_min = p->lrf_min;
  G.lrf_max = p->lrf_max;
  G.lobs_min = p->lobs_min;
  G.n_min = p->n_min;
  G.n_max = p->n_max;
  for (int d = 0; d < 3; ++d) G.origin[d] = box->desc.origin[d];
  G.cell = box->desc.cell;
  G.j_max = ctx->j_max;
  G.n_fft = p->n_fft;
  G.rebin = 0;
  return G;
}

int enqueue_geometry(mk_ctx *ctx, const GeomParams &G, const mk_qso *d_qso, int64_t n_qso, mk_skewer *d_sk,
                     int64_t *d_offsets) {
  CK(launch_geometry(d_qso, n_qso, G, d_sk, ctx->d_cnt_px, ctx->d_cnt_seg, ctx->d_err, ctx->stream));
  CK(launch_scan(ctx->d_cnt_px, ctx->d_cnt_seg, n_qso, d_offsets, ctx->d_segoff, d_sk, ctx->d_scan_ws,
                 ctx->stream));
  return MK_OK;
}

int run_geometry(mk_ctx *ctx, const mk_box *box, const mk_qso *d_qso, int64_t n_qso, const mk_skewer_params *p,
                 mk_skewer *d_sk, int64_t *d_offsets) {
  return enqueue_geometry(ctx, geom_params(ctx, box, p), d_qso, n_qso, d_sk, d_offsets);
}

SkewerParams skewer_params(mk_ctx *ctx, const mk_box *box, const mk_skewer *d_sk, int64_t n, const mk_skewer_params *p) {
  SkewerParams S;
  std::memset(&S, 0, sizeof(S));
  S.sk = d_sk;
  S.segoff = ctx->d_segoff;
  S.n_sk = n;
  S.box_d = box->d;
  S.box_e = box->e;
  S.lgn = box->lgn;
  S.pixtab = ctx->d_pixtab;
  S.zbin = ctx->d_zbin;
  S.cumz = ctx->d_cumz;
  S.amp = ctx->d_amp;
  S.ps_nodes = ctx->ps_nodes;
  for (int k = 0; k < MK_MAX_NODES; ++k) S.ps_z[k] = ctx->ps_z[k];
  S.zwin = ctx->d_zwin;
  S.tw = ctx->d_tw[tw_slot(p->n_fft)];
  S.seed = p->seed;
  S.j_max = ctx->j_max;
  S.segzbin = ctx->d_segzbin;
  S.bin_end = ctx->d_bin_end;
  S.err = ctx->d_err;
  S.dr = p->dr;
  S.p1d_scale = static_cast<float>(p->dr / p->n_fft);
  return S;
}

int finish_stats(mk_ctx *ctx, int nparts, const mk_stat_bins *b, mk_stats_out *h_out) {
  CK(launch_finalize(ctx->d_partials, nparts, b->n_z, b->n_k, b->n_fft, ctx->d_stats, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_stats, ctx->d_stats, sizeof(mk_stats_out), cudaMemcpyDeviceToHost, ctx->stream));
  int rc = read_error_word(ctx);  // synchronises
  if (rc) return rc;
  std::memcpy(h_out, ctx->h_stats, sizeof(mk_stats_out));
  return MK_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

int mk_create(mk_ctx **out, int device, void *cuda_stream, const mk_cosmo *cosmo) {
  mk_ctx *ctx = nullptr;
  if (!out) return MK_EINVAL;
  *out = nullptr;
  if (!cosmo || !(cosmo->omega_m > 0.0) || cosmo->omega_m > 1.0 || !(cosmo->lambda_lya > 0.0))
    return MK_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return MK_ECUDA;
  ctx = new mk_ctx();
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  ctx->cosmo = *cosmo;
  ctx->cos.build(cosmo->omega_m);
  int rc = MK_OK;
  do {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { rc = MK_ECUDA; break; }
    ctx->sms = prop.multiProcessorCount;
    ctx->n_dc = static_cast<int>(ctx->cos.dc.size());
    std::vector<double2> tab(ctx->n_dc);
    for (int i = 0; i < ctx->n_dc; ++i) tab[i] = make_double2(ctx->cos.dc[i], ctx->cos.slope[i]);
    ctx->n_zr = static_cast<int>(ctx->cos.dc.back() / kZrStep) + 2;
    std::vector<double> zr(ctx->n_zr);
    for (int i = 0; i < ctx->n_zr; ++i) zr[i] = ctx->cos.z_of(i * kZrStep);
    if (cudaMalloc(&ctx->d_dc, sizeof(double2) * ctx->n_dc) != cudaSuccess ||
        cudaMemcpy(ctx->d_dc, tab.data(), sizeof(double2) * ctx->n_dc, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&ctx->d_zr, sizeof(double) * ctx->n_zr) != cudaSuccess ||
        cudaMemcpy(ctx->d_zr, zr.data(), sizeof(double) * ctx->n_zr, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess || cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_total, sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&ctx->d_stats, sizeof(mk_stats_out)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_stats, sizeof(mk_stats_out)) != cudaSuccess) {
      rc = MK_ENOMEM;
      break;
    }
  } while (0);
  if (rc != MK_OK) {
    mk_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return MK_OK;
}

void mk_destroy(mk_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->d_dc);
  cudaFree(ctx->d_zr);
  cudaFree(ctx->d_err);
  cudaFreeHost(ctx->h_err);
  cudaFreeHost(ctx->h_total);
  cudaFree(ctx->d_zpix);
  cudaFree(ctx->d_cumz);
  cudaFree(ctx->d_gpix);
  cudaFree(ctx->d_pixtab);
  cudaFree(ctx->d_zbin);
  cudaFree(ctx->d_segzbin);
  cudaFree(ctx->d_bin_end);
  cudaFree(ctx->d_amp);
  cudaFree(ctx->d_zwin);
  cudaFree(ctx->d_pk);
  for (auto *p : ctx->d_tw) cudaFree(p);
  cudaFree(ctx->d_cnt_px);
  cudaFree(ctx->d_cnt_seg);
  cudaFree(ctx->d_segoff);
  cudaFree(ctx->d_scan_ws);
  cudaFree(ctx->d_partials);
  cudaFree(ctx->d_stats);
  cudaFreeHost(ctx->h_stats);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  cudaFree(ctx->d_hq);
  cudaFree(ctx->d_hsk);
  cudaFree(ctx->d_hoff);
  cudaFree(ctx->d_stage[0]);
  cudaFree(ctx->d_stage[1]);
  cudaFree(ctx->d_pick);
  if (ctx->h_pick) cudaFreeHost(ctx->h_pick);
  if (ctx->host_ready) {
    for (int c = 0; c < MK_HOST_COPY_STREAMS; ++c) {
      cudaStreamDestroy(ctx->copy_st[c]);
      for (int k = 0; k < MK_MAX_CHUNKS; ++k) cudaEventDestroy(ctx->ev_copy[c][k]);
    }
    for (int k = 0; k < MK_MAX_CHUNKS; ++k) cudaEventDestroy(ctx->ev_done[k]);
  }
  delete ctx;
}

const char *mk_last_error(const mk_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int mk_set_stream(mk_ctx *ctx, void *cuda_stream) {
  if (!ctx) return MK_EINVAL;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return MK_OK;
}

int mk_sync(mk_ctx *ctx) {
  if (!ctx) return MK_EINVAL;
  CK(cudaSetDevice(ctx->device));
  return read_error_word(ctx);
}

int mk_load_box(mk_ctx *ctx, mk_box **out, const mk_box_desc *desc, const float *d_delta, const float *d_eta) {
  MK_TRACE("mk_load_box");
  if (!ctx || !out) return MK_EINVAL;
  *out = nullptr;
  if (!desc) return fail(ctx, MK_EINVAL, "desc is NULL");
  const int n = desc->n;
  if (n < 2 || n > 2048 || (n & (n - 1))) return fail(ctx, MK_EINVAL, "box n must be a power of two in [2, 2048]");
  if (!(desc->cell > 0.0)) return fail(ctx, MK_EINVAL, "cell must be > 0");
  if (desc->layout == MK_BOX_PLANAR) {
    if (!d_delta || !d_eta) return fail(ctx, MK_EINVAL, "planar box needs d_delta and d_eta");
  } else if (desc->layout == MK_BOX_INTERLEAVED || desc->layout == MK_BOX_PADDED || desc->layout == MK_BOX_HALO ||
             desc->layout == MK_BOX_TENSOR) {
    if (!d_delta || d_eta) return fail(ctx, MK_EINVAL, "packed box: d_delta holds the records, d_eta must be NULL");
    const int align = desc->layout == MK_BOX_TENSOR ? 16 : 8;
    if (reinterpret_cast<uintptr_t>(d_delta) % align)
      return fail(ctx, MK_EINVAL, "packed box must be %d-byte aligned", align);
  } else {
    return fail(ctx, MK_EINVAL, "unknown layout %d", desc->layout);
  }
  mk_box *b = new mk_box();
  b->desc = *desc;
  b->d = d_delta;
  b->e = d_eta;
  b->lgn = 0;
  while ((1 << b->lgn) < n) ++b->lgn;
  *out = b;
  return MK_OK;
}

void mk_free_box(mk_box *box) { delete box; }

int mk_pack_box(mk_ctx *ctx, int64_t n_voxels, const float *d_delta, const float *d_eta, float *d_out) {
  MK_TRACE("mk_pack_box");
  if (!ctx) return MK_EINVAL;
  if (n_voxels < 0 || !d_delta || !d_eta || !d_out) return fail(ctx, MK_EINVAL, "bad pack arguments");
  CK(cudaSetDevice(ctx->device));
  CK(launch_pack(d_delta, d_eta, n_voxels, d_out, ctx->sms, ctx->stream));
  return MK_OK;
}

int mk_pack_box_padded(mk_ctx *ctx, int32_t n, const float *d_delta, const float *d_eta, float *d_out) {
  MK_TRACE("mk_pack_box_padded");
  if (!ctx) return MK_EINVAL;
  if (n < 2 || n > 2048 || (n & (n - 1))) return fail(ctx, MK_EINVAL, "box n must be a power of two in [2, 2048]");
  if (!d_delta || !d_eta || !d_out) return fail(ctx, MK_EINVAL, "bad pack arguments");
  if (reinterpret_cast<uintptr_t>(d_out) % 8) return fail(ctx, MK_EINVAL, "d_out must be 8-byte aligned");
  int lgn = 0;
  while ((1 << lgn) < n) ++lgn;
  CK(cudaSetDevice(ctx->device));
  CK(launch_pack_padded(d_delta, d_eta, lgn, d_out, ctx->sms, ctx->stream));
  return MK_OK;
}

int mk_pack_box_halo(mk_ctx *ctx, int32_t n, const float *d_delta, const float *d_eta, float *d_out) {
  MK_TRACE("mk_pack_box_halo");
  if (!ctx) return MK_EINVAL;
  if (n < 2 || n > 2048 || (n & (n - 1))) return fail(ctx, MK_EINVAL, "box n must be a power of two in [2, 2048]");
  if (!d_delta || !d_eta || !d_out) return fail(ctx, MK_EINVAL, "bad pack arguments");
  if (reinterpret_cast<uintptr_t>(d_out) % 8) return fail(ctx, MK_EINVAL, "d_out must be 8-byte aligned");
  int lgn = 0;
  while ((1 << lgn) < n) ++lgn;
  CK(cudaSetDevice(ctx->device));
  CK(launch_pack_halo(d_delta, d_eta, lgn, d_out, ctx->sms, ctx->stream));
  return MK_OK;
}

int mk_pack_box_tensor(mk_ctx *ctx, int32_t n, const float *d_delta, const float *d_eta6, float *d_out) {
  MK_TRACE("mk_pack_box_tensor");
  if (!ctx) return MK_EINVAL;
  if (n < 2 || n > 2048 || (n & (n - 1))) return fail(ctx, MK_EINVAL, "box n must be a power of two in [2, 2048]");
  if (!d_delta || !d_eta6 || !d_out) return fail(ctx, MK_EINVAL, "bad pack arguments");
  if (reinterpret_cast<uintptr_t>(d_out) % 16) return fail(ctx, MK_EINVAL, "d_out must be 16-byte aligned");
  int lgn = 0;
  while ((1 << lgn) < n) ++lgn;
  CK(cudaSetDevice(ctx->device));
  CK(launch_pack_tensor(d_delta, d_eta6, lgn, d_out, ctx->sms, ctx->stream));
  return MK_OK;
}

int mk_make_skewers(mk_ctx *ctx, const mk_box *box, const mk_qso *d_qso, int64_t n_qso,
                    const mk_skewer_params *params, mk_skewer *d_sk, int64_t *d_offsets, float *d_delta_out,
                    float *d_eta_out, int64_t capacity_px, int64_t *h_total_px) {
  MK_TRACE("mk_make_skewers");
  if (!ctx) return MK_EINVAL;
  int rc = check_params(ctx, params, d_delta_out != nullptr);
  if (rc) return rc;
  if (!box || n_qso < 0 || (n_qso > 0 && !d_qso) || !d_sk || !d_offsets)
    return fail(ctx, MK_EINVAL, "bad box, catalogue or skewer arguments");
  if ((rc = check_interp(ctx, box, params))) return rc;
  if ((d_delta_out == nullptr) != (d_eta_out == nullptr))
    return fail(ctx, MK_EINVAL, "d_delta_out and d_eta_out go together");
  CK(cudaSetDevice(ctx->device));
  if ((rc = ensure_pixel_tables(ctx, params->dr)) || (rc = ensure_counts(ctx, n_qso))) return rc;
  if ((rc = run_geometry(ctx, box, d_qso, n_qso, params, d_sk, d_offsets))) return rc;
  if (h_total_px) {
    CK(cudaMemcpyAsync(ctx->h_total, d_offsets + n_qso, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    if ((rc = read_error_word(ctx))) return rc;
    *h_total_px = *ctx->h_total;
  }
  if (!d_delta_out) return MK_OK;
  if ((rc = ensure_twiddles(ctx, params->n_fft)) || (rc = ensure_amp(ctx, params))) return rc;
  // the growth factor is the only table entry this pass reads
  mk_fgpa_nodes unit{};
  unit.count = 1;
  unit.z[0] = 0.0;
  if (!ctx->pixtab_valid && (rc = ensure_pixtab(ctx, &unit))) return rc;
  SkewerParams S = skewer_params(ctx, box, d_sk, n_qso, params);
  S.delta_out = d_delta_out;
  S.eta_out = d_eta_out;
  S.flux_out = nullptr;
  S.capacity = capacity_px;
  S.do_stats = 0;
  const LaunchCfg cfg = default_cfg(params->n_fft);
  const int variant = kernel_variant(box, params);
  const int grid = skewer_grid(ctx, params->n_fft, variant, box->lgn, cfg, nullptr);
  if ((rc = time_begin(ctx))) return rc;
  CK(launch_skewer(S, params->n_fft, variant, cfg.minb, grid, cfg.threads, ctx->stream));
  return time_end(ctx);
}

int mk_flux(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk, const float *d_delta,
            const float *d_eta, const mk_fgpa_nodes *nodes, int32_t rebin, float *d_flux, int64_t *d_offsets_out,
            int64_t capacity_out) {
  MK_TRACE("mk_flux");
  if (!ctx) return MK_EINVAL;
  int rc = check_params(ctx, params, false);
  if (rc || (rc = check_nodes(ctx, nodes))) return rc;
  if (rebin < 1 || rebin > 4096) return fail(ctx, MK_EINVAL, "rebin must be in [1, 4096]");
  if (n_sk < 0 || (n_sk > 0 && (!d_sk || !d_delta || !d_eta || !d_flux)) || !d_offsets_out)
    return fail(ctx, MK_EINVAL, "bad flux arguments");
  CK(cudaSetDevice(ctx->device));
  if ((rc = ensure_pixel_tables(ctx, params->dr)) || (rc = ensure_counts(ctx, n_sk)) ||
      (rc = ensure_pixtab(ctx, nodes)))
    return rc;
  CK(launch_out_counts(d_sk, n_sk, rebin, ctx->d_cnt_px, ctx->stream));
  CK(launch_scan(ctx->d_cnt_px, nullptr, n_sk, d_offsets_out, nullptr, nullptr, ctx->d_scan_ws, ctx->stream));
  FluxParams F{};
  F.sk = d_sk;
  F.off_out = d_offsets_out;
  F.n_sk = n_sk;
  F.delta = d_delta;
  F.eta = d_eta;
  F.pixtab = ctx->d_pixtab;
  F.rebin = rebin;
  F.j_max = ctx->j_max;
  F.flux = d_flux;
  F.capacity = capacity_out;
  F.err = ctx->d_err;
  CK(launch_flux(F, ctx->sms, ctx->stream));
  return MK_OK;
}

namespace {
// Statistics pass shared by mk_stats (stored flux) and mk_flux_stats (flux
// computed from stored fields with the FGPA table of `nodes`).
int stats_pass(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
               const int64_t *d_offsets_out, const float *d_flux, int32_t rebin, const float *d_delta,
               const float *d_eta, const mk_fgpa_nodes *nodes, const mk_stat_bins *bins, mk_stats_out *h_out) {
  if (!ctx) return MK_EINVAL;
  int rc = check_params(ctx, params, false);
  if (rc || (rc = check_bins(ctx, bins))) return rc;
  if (rebin < 1 || rebin > 4096) return fail(ctx, MK_EINVAL, "rebin must be in [1, 4096]");
  if (!h_out || n_sk < 0 || (n_sk > 0 && (!d_sk || !d_offsets_out || (!d_flux && !nodes))))
    return fail(ctx, MK_EINVAL, "bad stats arguments");
  if (nodes && (rebin != 1 || !d_delta)) return fail(ctx, MK_EINVAL, "the tuning pass needs rebin 1 and the fields");
  if ((d_delta == nullptr) != (d_eta == nullptr)) return fail(ctx, MK_EINVAL, "d_delta and d_eta go together");
  CK(cudaSetDevice(ctx->device));
  if ((rc = ensure_pixel_tables(ctx, params->dr)) || (rc = ensure_counts(ctx, n_sk)) ||
      (rc = ensure_twiddles(ctx, bins->n_fft)) || (rc = ensure_zbin(ctx, bins)))
    return rc;
  if (nodes && (rc = ensure_pixtab(ctx, nodes))) return rc;
  const int threads = 256;
  const StatLayout L{bins->n_z, bins->n_k};
  const int grid = stats_grid(ctx, bins, threads, tune_kernel(nodes ? ctx->d_pixtab : nullptr, d_delta, d_eta, rebin));
  if ((rc = grow(ctx, reinterpret_cast<void **>(&ctx->d_partials), &ctx->partials_cap,
                 sizeof(double) * static_cast<size_t>(grid) * L.size())))
    return rc;
  if (n_sk > 0) CK(launch_seg_counts(d_offsets_out, n_sk, bins->n_fft, ctx->d_cnt_seg, ctx->stream));
  CK(launch_scan(ctx->d_cnt_seg, nullptr, n_sk, ctx->d_segoff, nullptr, nullptr, ctx->d_scan_ws, ctx->stream));
  StatParams P{};
  P.sk = d_sk;
  P.off_out = d_offsets_out;
  P.segoff = ctx->d_segoff;
  P.n_sk = n_sk;
  P.flux = nodes ? nullptr : d_flux;
  P.pixtab = nodes ? ctx->d_pixtab : nullptr;
  P.delta = d_delta;
  P.eta = d_eta;
  P.rebin = rebin;
  P.zbin = ctx->d_zbin;
  P.segzbin = ctx->d_segzbin;
  P.bin_end = ctx->d_bin_end;
  P.p1d_scale = static_cast<float>(rebin * params->dr / bins->n_fft);
  P.cumz = ctx->d_cumz;
  P.tw = ctx->d_tw[tw_slot(bins->n_fft)];
  P.j_max = ctx->j_max;
  P.n_z = bins->n_z;
  P.n_k = bins->n_k;
  P.z_lo = bins->z_lo;
  P.dz = bins->dz;
  P.dr = params->dr;
  P.partials = ctx->d_partials;
  P.err = ctx->d_err;
  P.wait_test = ctx->wait_test;
  if ((rc = take_fault(ctx, MK_FAULT_LAUNCH))) return rc;
  if ((rc = time_begin(ctx))) return rc;
  CK(launch_stats(P, bins->n_fft, grid, threads, ctx->stream));
  if ((rc = time_end(ctx))) return rc;
  return finish_stats(ctx, grid, bins, h_out);
}
}  // namespace

int mk_stats(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
             const int64_t *d_offsets_out, const float *d_flux, int32_t rebin, const float *d_delta,
             const float *d_eta, const mk_stat_bins *bins, mk_stats_out *h_out) {
  MK_TRACE("mk_stats");
  if (!ctx) return MK_EINVAL;
  if (n_sk > 0 && !d_flux) return fail(ctx, MK_EINVAL, "d_flux is NULL");
  return stats_pass(ctx, params, d_sk, n_sk, d_offsets_out, d_flux, rebin, d_delta, d_eta, nullptr, bins, h_out);
}

int mk_flux_stats(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
                  const int64_t *d_offsets, const float *d_delta, const float *d_eta, const mk_fgpa_nodes *nodes,
                  const mk_stat_bins *bins, mk_stats_out *h_out) {
  MK_TRACE("mk_flux_stats");
  if (!ctx) return MK_EINVAL;
  int rc = check_nodes(ctx, nodes);
  if (rc) return rc;
  if (n_sk > 0 && (!d_delta || !d_eta)) return fail(ctx, MK_EINVAL, "the tuning pass needs d_delta and d_eta");
  return stats_pass(ctx, params, d_sk, n_sk, d_offsets, nullptr, 1, d_delta, d_eta, nodes, bins, h_out);
}

int mk_run(mk_ctx *ctx, const mk_box *box, const mk_qso *d_qso, int64_t n_qso, const mk_skewer_params *params,
           const mk_fgpa_nodes *nodes, const mk_stat_bins *bins, uint32_t flags, mk_skewer *d_sk,
           int64_t *d_offsets, float *d_delta_out, float *d_eta_out, float *d_flux_out, int64_t capacity_px,
           mk_stats_out *h_out) {
  MK_TRACE("mk_run");
  if (!ctx) return MK_EINVAL;
  int rc = check_params(ctx, params, true);
  if (rc || (rc = check_nodes(ctx, nodes))) return rc;
  if (flags & ~(MK_STORE_FIELDS | MK_STORE_FLUX | MK_STATS | MK_AUTOTUNE | MK_GRAPH))
    return fail(ctx, MK_EINVAL, "unknown flags 0x%x", flags);
  const bool stats = flags & MK_STATS;
  if (stats) {
    if ((rc = check_bins(ctx, bins))) return rc;
    if (bins->n_fft != params->n_fft) return fail(ctx, MK_EINVAL, "fused statistics need bins n_fft == n_fft");
    if (!h_out) return fail(ctx, MK_EINVAL, "h_out is NULL");
  }
  if (!box || n_qso < 0 || (n_qso > 0 && !d_qso) || !d_sk || !d_offsets)
    return fail(ctx, MK_EINVAL, "bad box, catalogue or skewer arguments");
  if ((rc = check_interp(ctx, box, params))) return rc;
  if ((flags & MK_STORE_FIELDS) && (!d_delta_out || !d_eta_out))
    return fail(ctx, MK_EINVAL, "MK_STORE_FIELDS needs d_delta_out and d_eta_out");
  if ((flags & MK_STORE_FLUX) && !d_flux_out) return fail(ctx, MK_EINVAL, "MK_STORE_FLUX needs d_flux_out");
  if ((flags & MK_GRAPH) && !ctx->stream)
    return fail(ctx, MK_EINVAL, "MK_GRAPH needs a non-default stream (the legacy stream cannot be captured)");
  CK(cudaSetDevice(ctx->device));
  if ((rc = take_fault(ctx, MK_FAULT_LAUNCH))) return rc;
  if ((rc = ensure_pixel_tables(ctx, params->dr)) || (rc = ensure_counts(ctx, n_qso)) ||
      (rc = ensure_twiddles(ctx, params->n_fft)) || (rc = ensure_amp(ctx, params)) ||
      (rc = ensure_pixtab(ctx, nodes)))
    return rc;
  if (stats && (rc = ensure_zbin(ctx, bins))) return rc;
  const StatLayout L{stats ? bins->n_z : 0, stats ? bins->n_k : 0};

  // the launch shape: tuned, or tune now, or the default
  const int variant = kernel_variant(box, params);
  const uint64_t key = tune_key(params->n_fft, variant, box->lgn, flags);
  LaunchCfg cfg = default_cfg(params->n_fft);
  auto it = ctx->tuned.find(key);
  if (it != ctx->tuned.end()) cfg = it->second;

  const GeomParams G = geom_params(ctx, box, params);
  SkewerParams S = skewer_params(ctx, box, d_sk, n_qso, params);
  S.delta_out = (flags & MK_STORE_FIELDS) ? d_delta_out : nullptr;
  S.eta_out = (flags & MK_STORE_FIELDS) ? d_eta_out : nullptr;
  S.flux_out = (flags & MK_STORE_FLUX) ? d_flux_out : nullptr;
  S.capacity = capacity_px;
  S.do_stats = stats ? 1 : 0;
  if (stats) {
    S.n_z = bins->n_z;
    S.n_k = bins->n_k;
    S.z_lo = bins->z_lo;
    S.dz = bins->dz;
  }

  // enqueue geometry, the fused kernel and (with statistics) their readback
  auto enqueue = [&](LaunchCfg c, int grid, bool timed) -> int {
    int r = enqueue_geometry(ctx, G, d_qso, n_qso, d_sk, d_offsets);
    if (r) return r;
    S.partials = ctx->d_partials;
    if (timed && (r = time_begin(ctx))) return r;
    CK(launch_skewer(S, params->n_fft, variant, c.minb, grid, c.threads, ctx->stream));
    if (timed && (r = time_end(ctx))) return r;
    if (stats) {
      CK(launch_finalize(ctx->d_partials, grid, bins->n_z, bins->n_k, bins->n_fft, ctx->d_stats, ctx->stream));
      CK(cudaMemcpyAsync(ctx->h_stats, ctx->d_stats, sizeof(mk_stats_out), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    }
    return MK_OK;
  };
  auto ensure_partials = [&](int grid) -> int {
    if (!stats) return MK_OK;
    return grow(ctx, reinterpret_cast<void **>(&ctx->d_partials), &ctx->partials_cap,
                sizeof(double) * static_cast<size_t>(grid) * L.size());
  };

  if ((flags & MK_AUTOTUNE) && it == ctx->tuned.end()) {
    // time every admissible shape on this call's inputs; outputs are rewritten
    // by the final run below
    const LaunchCfg cand[5] = {{256, 2}, {256, 3}, {256, 4}, {128, 3}, {128, 4}};
    cudaEvent_t a0, a1;
    CK(cudaEventCreate(&a0));
    CK(cudaEventCreate(&a1));
    float best = 1e30f;
    for (const LaunchCfg &c : cand) {
      if (c.threads < params->n_fft / 8) continue;  // a team must fit in a CTA
      const int grid = skewer_grid(ctx, params->n_fft, variant, box->lgn, c, stats ? bins : nullptr);
      if ((rc = ensure_partials(grid))) break;
      if ((rc = enqueue_geometry(ctx, G, d_qso, n_qso, d_sk, d_offsets))) break;
      S.partials = ctx->d_partials;
      float ms = 0.f;
      for (int rep = 0; rep < 2 && rc == MK_OK; ++rep) {  // first launch warms caches
        if (cudaEventRecord(a0, ctx->stream) != cudaSuccess ||
            launch_skewer(S, params->n_fft, variant, c.minb, grid, c.threads, ctx->stream) != cudaSuccess ||
            cudaEventRecord(a1, ctx->stream) != cudaSuccess || cudaEventSynchronize(a1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, a0, a1) != cudaSuccess)
          rc = fail(ctx, MK_ECUDA, "autotune launch failed: %s", cudaGetErrorString(cudaGetLastError()));
      }
      if (rc) break;
      if (ms < best) {
        best = ms;
        cfg = c;
      }
    }
    cudaEventDestroy(a0);
    cudaEventDestroy(a1);
    if (rc) return rc;
    ctx->tuned[key] = cfg;
  }

  const int grid = skewer_grid(ctx, params->n_fft, variant, box->lgn, cfg, stats ? bins : nullptr);
  if ((rc = ensure_partials(grid))) return rc;

  if (flags & MK_GRAPH) {
    // replay the captured step when nothing it depends on has changed
    std::vector<unsigned char> gkey(sizeof(G) + sizeof(S) + 8 * sizeof(int64_t));
    unsigned char *kp = gkey.data();
    S.partials = ctx->d_partials;
    std::memcpy(kp, &G, sizeof(G));
    std::memcpy(kp + sizeof(G), &S, sizeof(S));
    const int64_t extra[8] = {reinterpret_cast<int64_t>(d_qso), n_qso, reinterpret_cast<int64_t>(d_offsets),
                              static_cast<int64_t>(ctx->generation), grid, cfg.threads * 16 + cfg.minb,
                              static_cast<int64_t>(flags & ~MK_AUTOTUNE),
                              stats ? (bins->n_z * 4096 + bins->n_k * 8 + (bins->n_fft >> 8)) : 0};
    std::memcpy(kp + sizeof(G) + sizeof(S), extra, sizeof(extra));
    if (!ctx->graph || gkey != ctx->graph_key) {
      if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      rc = enqueue(cfg, grid, false);
      const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
      if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ce != cudaSuccess) return fail(ctx, MK_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
      const cudaError_t ie = cudaGraphInstantiate(&ctx->graph, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) {
        ctx->graph = nullptr;
        return fail(ctx, MK_ECUDA, "graph instantiate: %s", cudaGetErrorString(ie));
      }
      ctx->graph_key = gkey;
    }
    if ((rc = time_begin(ctx))) return rc;
    CK(cudaGraphLaunch(ctx->graph, ctx->stream));
    if ((rc = time_end(ctx))) return rc;
  } else {
    if ((rc = enqueue(cfg, grid, true))) return rc;
  }
  if (!stats) return MK_OK;
  CK(cudaStreamSynchronize(ctx->stream));
  const int e = *ctx->h_err;
  if (e) return read_error_word(ctx);
  std::memcpy(h_out, ctx->h_stats, sizeof(mk_stats_out));
  return MK_OK;
}

namespace {
int ensure_host_path(mk_ctx *ctx) {
  if (ctx->host_ready) return MK_OK;
  CK(cudaMalloc(&ctx->d_pick, sizeof(int64_t) * (MK_MAX_CHUNKS + 1)));
  CK(cudaMallocHost(&ctx->h_pick, sizeof(int64_t) * (MK_MAX_CHUNKS + 1)));
  for (int c = 0; c < MK_HOST_COPY_STREAMS; ++c) {
    CK(cudaStreamCreateWithFlags(&ctx->copy_st[c], cudaStreamNonBlocking));
    for (int k = 0; k < MK_MAX_CHUNKS; ++k) CK(cudaEventCreateWithFlags(&ctx->ev_copy[c][k], cudaEventDisableTiming));
  }
  for (int k = 0; k < MK_MAX_CHUNKS; ++k) CK(cudaEventCreateWithFlags(&ctx->ev_done[k], cudaEventDisableTiming));
  ctx->host_ready = true;
  return MK_OK;
}
}  // namespace

int mk_run_host(mk_ctx *ctx, const mk_box *box, const mk_qso *h_qso, int64_t n_qso, const mk_skewer_params *params,
                const mk_fgpa_nodes *nodes, const mk_stat_bins *bins, uint32_t flags, int32_t n_chunks,
                float *h_flux_out, int64_t capacity_px, int64_t *h_total_px, mk_stats_out *h_out) {
  MK_TRACE("mk_run_host");
  if (!ctx) return MK_EINVAL;
  int rc = check_params(ctx, params, true);
  if (rc || (rc = check_nodes(ctx, nodes))) return rc;
  if (flags & ~MK_STATS) return fail(ctx, MK_EINVAL, "mk_run_host: flags may hold MK_STATS only");
  const bool stats = flags & MK_STATS;
  if (stats) {
    if ((rc = check_bins(ctx, bins))) return rc;
    if (bins->n_fft != params->n_fft) return fail(ctx, MK_EINVAL, "fused statistics need bins n_fft == n_fft");
    if (!h_out) return fail(ctx, MK_EINVAL, "h_out is NULL");
  }
  if (!box || n_qso < 0 || (n_qso > 0 && !h_qso) || !h_flux_out || !h_total_px)
    return fail(ctx, MK_EINVAL, "bad box, catalogue or output arguments");
  if ((rc = check_interp(ctx, box, params))) return rc;
  if (n_chunks < 1 || n_chunks > MK_MAX_CHUNKS) return fail(ctx, MK_EINVAL, "n_chunks must be in [1, %d]", MK_MAX_CHUNKS);
  CK(cudaSetDevice(ctx->device));
  if ((rc = ensure_pixel_tables(ctx, params->dr)) || (rc = ensure_counts(ctx, n_qso)) ||
      (rc = ensure_twiddles(ctx, params->n_fft)) || (rc = ensure_amp(ctx, params)) ||
      (rc = ensure_pixtab(ctx, nodes)) || (rc = ensure_host_path(ctx)))
    return rc;
  if (stats && (rc = ensure_zbin(ctx, bins))) return rc;
  const size_t nq = static_cast<size_t>(n_qso);
  if ((rc = grow(ctx, &ctx->d_hq, &ctx->hq_cap, sizeof(mk_qso) * (nq ? nq : 1))) ||
      (rc = grow(ctx, &ctx->d_hsk, &ctx->hsk_cap, sizeof(mk_skewer) * (nq ? nq : 1))) ||
      (rc = grow(ctx, &ctx->d_hoff, &ctx->hoff_cap, sizeof(int64_t) * (nq + 1))))
    return rc;
  mk_skewer *d_sk = static_cast<mk_skewer *>(ctx->d_hsk);
  int64_t *d_off = static_cast<int64_t *>(ctx->d_hoff);
  cudaStream_t s0 = ctx->stream;

  // catalogue in, geometry of every quasar, slice boundaries out
  if (n_qso > 0) CK(cudaMemcpyAsync(ctx->d_hq, h_qso, sizeof(mk_qso) * nq, cudaMemcpyHostToDevice, s0));
  const GeomParams G = geom_params(ctx, box, params);
  if ((rc = enqueue_geometry(ctx, G, static_cast<const mk_qso *>(ctx->d_hq), n_qso, d_sk, d_off))) return rc;
  const int K = n_chunks;
  CK(launch_pick(d_off, n_qso, K, ctx->d_pick, s0));
  CK(cudaMemcpyAsync(ctx->h_pick, ctx->d_pick, sizeof(int64_t) * (K + 1), cudaMemcpyDeviceToHost, s0));
  if ((rc = read_error_word(ctx))) return rc;  // synchronises s0
  const int64_t *pk = ctx->h_pick;
  const int64_t total = pk[K];
  *h_total_px = total;
  if (total > capacity_px) return fail(ctx, MK_ERANGE, "flux of %lld pixels exceeds capacity %lld",
                                      static_cast<long long>(total), static_cast<long long>(capacity_px));
  int64_t maxc = 1;
  for (int k = 0; k < K; ++k) maxc = std::max<int64_t>(maxc, pk[k + 1] - pk[k]);
  for (int b = 0; b < 2; ++b)
    if ((rc = grow(ctx, &ctx->d_stage[b], &ctx->stage_cap[b], sizeof(float) * static_cast<size_t>(maxc)))) return rc;

  const uint32_t kflags = MK_STORE_FLUX | (stats ? MK_STATS : 0u);
  LaunchCfg cfg = default_cfg(params->n_fft);
  const int variant = kernel_variant(box, params);
  auto it = ctx->tuned.find(tune_key(params->n_fft, variant, box->lgn, kflags));
  if (it != ctx->tuned.end()) cfg = it->second;
  const int grid = skewer_grid(ctx, params->n_fft, variant, box->lgn, cfg, stats ? bins : nullptr);
  const StatLayout L{stats ? bins->n_z : 0, stats ? bins->n_k : 0};
  if (stats && (rc = grow(ctx, reinterpret_cast<void **>(&ctx->d_partials), &ctx->partials_cap,
                          sizeof(double) * static_cast<size_t>(grid) * K * L.size())))
    return rc;
  SkewerParams S = skewer_params(ctx, box, d_sk, n_qso, params);
  S.do_stats = stats ? 1 : 0;
  if (stats) {
    S.n_z = bins->n_z;
    S.n_k = bins->n_k;
    S.z_lo = bins->z_lo;
    S.dz = bins->dz;
  }

  // slices: compute on s0 into staging buffer k % 2, copy out on the copy
  // streams once the slice is done; slice k + 2 reuses the buffer after them
  for (int k = 0; k < K; ++k) {
    const int64_t q0 = static_cast<int64_t>(k) * n_qso / K, q1 = static_cast<int64_t>(k + 1) * n_qso / K;
    const int64_t p0 = pk[k], p1 = pk[k + 1];
    if (k >= 2)
      for (int c = 0; c < MK_HOST_COPY_STREAMS; ++c) CK(cudaStreamWaitEvent(s0, ctx->ev_copy[c][k - 2], 0));
    float *stage = static_cast<float *>(ctx->d_stage[k & 1]);
    if (q1 > q0) {
      S.sk = d_sk + q0;
      S.segoff = ctx->d_segoff + q0;
      S.n_sk = q1 - q0;
      // records hold absolute offsets: shift the base so that pixel p0 lands at stage[0]
      S.flux_out = reinterpret_cast<float *>(reinterpret_cast<uintptr_t>(stage) - sizeof(float) * p0);
      S.capacity = p1;
      S.partials = stats ? ctx->d_partials + static_cast<size_t>(k) * grid * L.size() : nullptr;
      CK(launch_skewer(S, params->n_fft, variant, cfg.minb, grid, cfg.threads, s0));
    } else if (stats) {
      CK(cudaMemsetAsync(ctx->d_partials + static_cast<size_t>(k) * grid * L.size(), 0,
                         sizeof(double) * static_cast<size_t>(grid) * L.size(), s0));
    }
    CK(cudaEventRecord(ctx->ev_done[k], s0));
    const int64_t n = p1 - p0;
    for (int c = 0; c < MK_HOST_COPY_STREAMS; ++c) {
      const int64_t a = n * c / MK_HOST_COPY_STREAMS, b = n * (c + 1) / MK_HOST_COPY_STREAMS;
      CK(cudaStreamWaitEvent(ctx->copy_st[c], ctx->ev_done[k], 0));
      if (b > a)
        CK(cudaMemcpyAsync(h_flux_out + p0 + a, stage + a, sizeof(float) * (b - a), cudaMemcpyDeviceToHost,
                           ctx->copy_st[c]));
      CK(cudaEventRecord(ctx->ev_copy[c][k], ctx->copy_st[c]));
    }
  }
  if (stats) {
    CK(launch_finalize(ctx->d_partials, grid * K, bins->n_z, bins->n_k, bins->n_fft, ctx->d_stats, s0));
    CK(cudaMemcpyAsync(ctx->h_stats, ctx->d_stats, sizeof(mk_stats_out), cudaMemcpyDeviceToHost, s0));
  }
  for (int c = 0; c < MK_HOST_COPY_STREAMS; ++c) CK(cudaStreamWaitEvent(s0, ctx->ev_copy[c][K - 1], 0));
  if ((rc = read_error_word(ctx))) return rc;  // synchronises s0, after every copy
  if (stats) std::memcpy(h_out, ctx->h_stats, sizeof(mk_stats_out));
  return MK_OK;
}

int mk_launch_config(mk_ctx *ctx, int32_t n_fft, int32_t layout, int32_t big_box, uint32_t flags,
                     int32_t *threads, int32_t *occupancy) {
  if (!ctx || !threads || !occupancy) return MK_EINVAL;
  if (!skewer_fft(n_fft)) return fail(ctx, MK_EINVAL, "bad n_fft");
  LaunchCfg c = default_cfg(n_fft);
  auto it = ctx->tuned.find(tune_key(n_fft, layout, big_box ? 11 : 10, flags));
  if (it != ctx->tuned.end()) c = it->second;
  *threads = c.threads;
  *occupancy = c.minb;
  return it != ctx->tuned.end() ? MK_OK : MK_ERANGE;
}

int mk_set_grid_cap(mk_ctx *ctx, int32_t max_ctas) {
  if (!ctx) return MK_EINVAL;
  if (max_ctas < 0) return fail(ctx, MK_EINVAL, "max_ctas must be >= 0");
  ctx->grid_cap = max_ctas;
  return MK_OK;
}

int mk_inject_fault(mk_ctx *ctx, int32_t kind) {
  if (!ctx) return MK_EINVAL;
  if (kind < 0 || kind > MK_FAULT_LAUNCH) return fail(ctx, MK_EINVAL, "unknown fault kind %d", kind);
  ctx->fault = kind;
  return MK_OK;
}

int mk_set_wait_test(mk_ctx *ctx, int32_t on) {
  if (!ctx) return MK_EINVAL;
  ctx->wait_test = on != 0;
  return MK_OK;
}

int mk_set_timing(mk_ctx *ctx, int on) {
  if (!ctx) return MK_EINVAL;
  CK(cudaSetDevice(ctx->device));
  if (on && !ctx->ev0) {
    CK(cudaEventCreate(&ctx->ev0));
    CK(cudaEventCreate(&ctx->ev1));
  }
  ctx->timing = on != 0;
  ctx->timed = false;
  return MK_OK;
}

int mk_last_kernel_ms(mk_ctx *ctx, double *ms) {
  if (!ctx || !ms) return MK_EINVAL;
  if (!ctx->timed) return fail(ctx, MK_EINVAL, "no timed launch");
  CK(cudaSetDevice(ctx->device));
  CK(cudaEventSynchronize(ctx->ev1));
  float t = 0.f;
  CK(cudaEventElapsedTime(&t, ctx->ev0, ctx->ev1));
  *ms = t;
  return MK_OK;
}

}  // extern "C"

// ====================================================================== merge of per-part statistics
extern "C" int mk_stats_merge(const mk_stats_out *parts, int32_t n_parts, const mk_stat_bins *bins,
                              mk_stats_out *out) {
  if (!parts || !out || !bins || n_parts < 1) return MK_EINVAL;
  if (bins->n_z < 1 || bins->n_z > MK_MAX_ZBINS || bins->n_k < 1 || bins->n_k > MK_MAX_KBINS ||
      !skewer_fft(bins->n_fft) || (bins->n_fft / 2) % bins->n_k)
    return MK_EINVAL;
  mk_stats_out tot;
  std::memset(&tot, 0, sizeof(tot));
  for (int32_t p = 0; p < n_parts; ++p)
    for (int zb = 0; zb < bins->n_z; ++zb) {
      for (int i = 0; i < MK_NSUM; ++i) tot.sums[zb][i] += parts[p].sums[zb][i];
      for (int k = 0; k < bins->n_k; ++k) tot.p1d_sum[zb][k] += parts[p].p1d_sum[zb][k];
      tot.n_seg[zb] += parts[p].n_seg[zb];
    }
  const double per_bin = static_cast<double>(bins->n_fft / 2) / bins->n_k;
  for (int zb = 0; zb < bins->n_z; ++zb) finalize_bin(&tot, zb, bins->n_k, per_bin);
  std::memcpy(out, &tot, sizeof(tot));
  return MK_OK;
}

// ====================================================================== statistics without allocation
// Scratch of mk_stats_static: one fixed array in the library's device memory
// instead of the context's growable workspace.  Layout, in 256-byte aligned
// pieces: the device copy of the result, segment counts, segment offsets,
// scan tile sums, then per-CTA FP64 partial sums in the remaining space.
static __device__ __align__(256) unsigned char g_stats_scratch[MK_STATIC_SCRATCH_BYTES];

namespace {

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

// Device address of the array on the context's device, looked up by the
// first call on each context with its device current.  A context lives in
// one CUDA context of its device, so the address cannot go stale under it
// (a cudaDeviceReset ends the contexts created before it).
int stats_scratch_address(mk_ctx *ctx, unsigned char **out) {
  if (!ctx->static_scratch) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_stats_scratch);
    if (e != cudaSuccess || !p)
      return fail(ctx, MK_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
    ctx->static_scratch = static_cast<unsigned char *>(p);
  }
  *out = ctx->static_scratch;
  return MK_OK;
}

}  // namespace

extern "C" int mk_stats_static(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
                               const int64_t *d_offsets_out, const float *d_flux, int32_t rebin,
                               const float *d_delta, const float *d_eta, const mk_stat_bins *bins,
                               mk_stats_out *h_out) {
  MK_TRACE("mk_stats_static");
  if (!ctx) return MK_EINVAL;
  int rc = check_params(ctx, params, false);
  if (rc || (rc = check_bins(ctx, bins))) return rc;
  if (rebin < 1 || rebin > 4096) return fail(ctx, MK_EINVAL, "rebin must be in [1, 4096]");
  if (!h_out || n_sk < 0 || (n_sk > 0 && (!d_sk || !d_offsets_out || !d_flux)))
    return fail(ctx, MK_EINVAL, "bad stats arguments");
  if (n_sk > MK_STATIC_MAX_SKEWERS)
    return fail(ctx, MK_EINVAL, "n_sk = %lld exceeds MK_STATIC_MAX_SKEWERS = %d", static_cast<long long>(n_sk),
                MK_STATIC_MAX_SKEWERS);
  if ((d_delta == nullptr) != (d_eta == nullptr)) return fail(ctx, MK_EINVAL, "d_delta and d_eta go together");
  CK(cudaSetDevice(ctx->device));
  if (!(ctx->d_zpix && ctx->dr == params->dr))
    return fail(ctx, MK_EINVAL, "no pixel tables for dr = %g on this context: run an allocating call first",
                params->dr);
  if (!ctx->d_tw[tw_slot(bins->n_fft)])
    return fail(ctx, MK_EINVAL, "no FFT twiddles for n_fft = %d on this context: run an allocating call first",
                bins->n_fft);
  // the z-bin tables: the per-pixel ones come with the pixel tables, the
  // bin-end table with the first allocating statistics call; rebuilding them
  // for other bins only runs kernels into that memory
  if (!ctx->d_bin_end)
    return fail(ctx, MK_EINVAL,
                "no z-bin tables on this context: run an allocating statistics call (mk_stats, mk_flux_stats, "
                "or mk_run with MK_STATS) first");
  if ((rc = ensure_zbin(ctx, bins))) return rc;
  unsigned char *base = nullptr;
  if ((rc = stats_scratch_address(ctx, &base))) return rc;

  const size_t off_cnt = align256(sizeof(mk_stats_out));
  const size_t off_seg = off_cnt + align256(sizeof(int64_t) * MK_STATIC_MAX_SKEWERS);
  const size_t off_tiles = off_seg + align256(sizeof(int64_t) * (MK_STATIC_MAX_SKEWERS + 1));
  const size_t off_part = off_tiles + align256(scan_workspace_bytes(MK_STATIC_MAX_SKEWERS));
  if (off_part >= MK_STATIC_SCRATCH_BYTES) return fail(ctx, MK_EINVAL, "static scratch layout overflow");
  mk_stats_out *d_out = reinterpret_cast<mk_stats_out *>(base);
  int64_t *d_cnt = reinterpret_cast<int64_t *>(base + off_cnt);
  int64_t *d_seg = reinterpret_cast<int64_t *>(base + off_seg);
  void *d_tiles = base + off_tiles;
  double *d_part = reinterpret_cast<double *>(base + off_part);
  const size_t part_doubles = (MK_STATIC_SCRATCH_BYTES - off_part) / sizeof(double);

  const int threads = 256;
  const StatLayout L{bins->n_z, bins->n_k};
  int grid = stats_grid(ctx, bins, threads);
  if (static_cast<size_t>(grid) * L.size() > part_doubles) grid = static_cast<int>(part_doubles / L.size());
  if (grid < 1) return fail(ctx, MK_EINVAL, "binning too large for the static scratch");

  // every piece below is fully rewritten by this call, so nothing is cleared
  if (n_sk > 0) CK(launch_seg_counts(d_offsets_out, n_sk, bins->n_fft, d_cnt, ctx->stream));
  CK(launch_scan(d_cnt, nullptr, n_sk, d_seg, nullptr, nullptr, d_tiles, ctx->stream));
  StatParams P{};
  P.sk = d_sk;
  P.off_out = d_offsets_out;
  P.segoff = d_seg;
  P.n_sk = n_sk;
  P.flux = d_flux;
  P.delta = d_delta;
  P.eta = d_eta;
  P.rebin = rebin;
  P.zbin = ctx->d_zbin;
  P.segzbin = ctx->d_segzbin;
  P.bin_end = ctx->d_bin_end;
  P.p1d_scale = static_cast<float>(rebin * params->dr / bins->n_fft);
  P.cumz = ctx->d_cumz;
  P.tw = ctx->d_tw[tw_slot(bins->n_fft)];
  P.j_max = ctx->j_max;
  P.n_z = bins->n_z;
  P.n_k = bins->n_k;
  P.z_lo = bins->z_lo;
  P.dz = bins->dz;
  P.dr = params->dr;
  P.partials = d_part;
  P.err = ctx->d_err;
  if ((rc = time_begin(ctx))) return rc;
  CK(launch_stats(P, bins->n_fft, grid, threads, ctx->stream));
  if ((rc = time_end(ctx))) return rc;
  CK(launch_finalize(d_part, grid, bins->n_z, bins->n_k, bins->n_fft, d_out, ctx->stream));
  CK(cudaMemcpyAsync(ctx->h_stats, d_out, sizeof(mk_stats_out), cudaMemcpyDeviceToHost, ctx->stream));
  if ((rc = read_error_word(ctx))) return rc;  // synchronises
  std::memcpy(h_out, ctx->h_stats, sizeof(mk_stats_out));
  return MK_OK;
}

// ====================================================================== internal accessors
// for the surrogate and tuner translation unit (mk_tune.cu)
namespace mkhost {
cudaStream_t ctx_stream(mk_ctx *c) { return c->stream; }
int ctx_device(mk_ctx *c) { return c->device; }
int ctx_fail(mk_ctx *c, int code, const char *msg) { return fail(c, code, "%s", msg); }
int ctx_sms(mk_ctx *c) { return c->sms; }
double ctx_z_of(mk_ctx *c, double r) { return c->cos.z_of(r); }
double ctx_growth(mk_ctx *c, double z) { return c->cos.growth(z); }
double ctx_distance(mk_ctx *c, double z) { return c->cos.distance(z); }

int ctx_pixel_histogram(mk_ctx *ctx, double dr, const mk_skewer *d_sk, int64_t n_sk, std::vector<double> &z,
                        std::vector<int64_t> &count, double *ms) {
  int rc = ensure_pixel_tables(ctx, dr);
  if (rc) return rc;
  const int32_t jm = ctx->j_max;
  int32_t *d_diff = nullptr;
  CK(cudaMalloc(&d_diff, sizeof(int32_t) * (jm + 1)));
  cudaEvent_t a = nullptr, b = nullptr;
  std::vector<int32_t> diff(jm + 1);
  z.resize(jm);
  cudaError_t e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) e = cudaEventRecord(a, ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_diff, 0, sizeof(int32_t) * (jm + 1), ctx->stream);
  if (e == cudaSuccess) e = launch_jcount(d_sk, n_sk, jm, d_diff, ctx->sms, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(diff.data(), d_diff, sizeof(int32_t) * (jm + 1), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(z.data(), ctx->d_zpix, sizeof(double) * jm, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b, ctx->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  float t = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaFree(d_diff);
  if (e != cudaSuccess) return fail(ctx, MK_ECUDA, "pixel histogram: %s", cudaGetErrorString(e));
  if (ms) *ms += t;
  count.assign(jm, 0);
  int64_t run = 0;
  for (int32_t j = 0; j < jm; ++j) {
    run += diff[j];
    count[j] = run;
  }
  return MK_OK;
}
}  // namespace mkhost

extern "C" int mk_synth_box(mk_ctx *ctx, int32_t n, double cell, uint64_t seed, const double *h_pk, int32_t n_pk,
                            double dk, int32_t layout, float *d_work, float *d_spec, float *d_out) {
  MK_TRACE("mk_synth_box");
  if (!ctx) return MK_EINVAL;
  if (n < 128 || n > 2048 || (n & (n - 1)))
    return fail(ctx, MK_EINVAL, "box side must be 128, 256, 512, 1024 or 2048");
  int lgn = 0;
  while ((1 << lgn) < n) ++lgn;
  if (!(cell > 0.0) || !(dk > 0.0) || !h_pk || n_pk < 2 || n_pk > (1 << 24))
    return fail(ctx, MK_EINVAL, "bad cell, dk or P(k) table (2 .. 2^24 entries)");
  if (!d_work || !d_out || (reinterpret_cast<uintptr_t>(d_work) & 15) || (reinterpret_cast<uintptr_t>(d_out) & 3) ||
      (layout != MK_BOX_PLANAR && (reinterpret_cast<uintptr_t>(d_out) & 7)))
    return fail(ctx, MK_EINVAL, "d_work must be 16-byte and d_out 8-byte (planar: 4-byte) aligned device pointers");
  const int64_t nv = static_cast<int64_t>(n) * n * n;
  int side = n, margin = 0, stride = 2, pairs = 1;
  switch (layout) {
    case MK_BOX_PLANAR: stride = 1; break;
    case MK_BOX_INTERLEAVED: break;
    case MK_BOX_PADDED: side = n + 1; break;
    case MK_BOX_HALO: side = n + 6; margin = 3; break;
    case MK_BOX_TENSOR:
      side = n + 1;
      stride = 8;
      pairs = 4;
      if (!d_spec || (reinterpret_cast<uintptr_t>(d_spec) & 7))
        return fail(ctx, MK_EINVAL, "MK_BOX_TENSOR needs an 8-byte aligned d_spec of 2 n^3 floats");
      if ((reinterpret_cast<uintptr_t>(d_out) & 15)) return fail(ctx, MK_EINVAL, "MK_BOX_TENSOR: d_out not 16-byte aligned");
      break;
    default: return fail(ctx, MK_EINVAL, "layout must be planar, interleaved, padded, halo or tensor");
  }
  auto overlap = [](const float *a, int64_t na, const float *b, int64_t nb) { return a < b + nb && b < a + na; };
  const int64_t nout = static_cast<int64_t>(side) * side * side * stride;
  if (!(layout == MK_BOX_INTERLEAVED && d_out == d_work) && overlap(d_work, 2 * nv, d_out, nout))
    return fail(ctx, MK_EINVAL, "d_work overlaps d_out");
  if (d_spec && (overlap(d_spec, 2 * nv, d_work, 2 * nv) || overlap(d_spec, 2 * nv, d_out, nout)))
    return fail(ctx, MK_EINVAL, "d_spec overlaps d_work or d_out");
  for (int i = 0; i < n_pk; ++i)
    if (!(h_pk[i] >= 0.0)) return fail(ctx, MK_EINVAL, "P(k) must be >= 0");
  CK(cudaSetDevice(ctx->device));
  int rc;
  if ((rc = ensure_twiddles(ctx, 2 * n))) return rc;
  std::vector<float> pk(h_pk, h_pk + n_pk);
  CK(cudaStreamSynchronize(ctx->stream));  // an earlier synthesis may still read the table
  if (n_pk > ctx->n_pk_cap) {
    cudaFree(ctx->d_pk);
    ctx->d_pk = nullptr;
    ctx->n_pk_cap = 0;
    CK(cudaMalloc(&ctx->d_pk, sizeof(float) * n_pk));
    ctx->n_pk_cap = n_pk;
  }
  CK(cudaMemcpy(ctx->d_pk, pk.data(), sizeof(float) * n_pk, cudaMemcpyHostToDevice));
  BoxPassParams P{};
  P.work = reinterpret_cast<float2 *>(d_work);
  P.spec = layout == MK_BOX_TENSOR ? reinterpret_cast<float2 *>(d_spec) : nullptr;
  P.tw = ctx->d_tw[tw_slot(2 * n)];
  P.pk = ctx->d_pk;
  P.n_pk = n_pk;
  P.inv_dk = static_cast<float>(1.0 / dk);
  P.kf = static_cast<float>(2.0 * M_PI / (n * cell));
  P.amp = static_cast<float>(1.0 / (std::pow(cell, 1.5) * static_cast<double>(nv)));
  P.key0 = static_cast<uint32_t>(seed);
  P.key1 = static_cast<uint32_t>(seed >> 32);
  P.lgn = lgn;
  const bool in_place = layout == MK_BOX_INTERLEAVED && d_out == d_work;
  P.out = in_place ? nullptr : d_out;
  P.out_side = side;
  P.out_margin = margin;
  P.out_stride = stride;
  for (int p = 0; p < pairs; ++p) {
    P.pair = p;
    P.out_slot = 2 * p;
    if (p == 0) {
      P.axis = 0;
      CK(launch_box_pass(P, kBoxNoiseX, ctx->sms, ctx->stream));
      P.axis = 1;
      CK(launch_box_pass(P, kBoxFwd, ctx->sms, ctx->stream));
      P.axis = 2;
      CK(launch_box_pass(P, kBoxShapeZ, ctx->sms, ctx->stream));
    } else {
      P.axis = 2;
      CK(launch_box_pass(P, kBoxSpecZ, ctx->sms, ctx->stream));
    }
    P.axis = 1;
    CK(launch_box_pass(P, kBoxInv, ctx->sms, ctx->stream));
    P.axis = 0;
    CK(launch_box_pass(P, kBoxInvXOut, ctx->sms, ctx->stream));
  }
  return MK_OK;
}

extern "C" int mk_cosmo_eval(mk_ctx *ctx, double z, double *d_c, double *growth) {
  if (!ctx) return MK_EINVAL;
  if (!d_c || !growth || !(z >= 0.0 && z < kZMax)) return fail(ctx, MK_EINVAL, "mk_cosmo_eval: z outside [0, 12)");
  *d_c = ctx->cos.distance(z);
  *growth = ctx->cos.growth(z);
  return MK_OK;
}
