// The tuning procedure of Sec. 2.6: a and b sigma_g from the FGPA moments of
// a Gaussian field, c from beta, b from the measured sigma_g, and the ratio
// iteration of the small-scale power P_S, every pass a fused synthesis.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/mockskewer.h"
#include "mk_host.h"
#include "mk_trace.h"

namespace {

int pfail(mk_ctx *ctx, int code, const char *msg) { return mkhost::ctx_fail(ctx, code, msg); }

// Composite Gauss-Legendre rule for E[f(xi)], xi ~ N(0, 1): kPanels panels of
// 8 points over [-10, 10] (the normal density beyond holds < 2e-23), the
// density folded into the weights.  The 8 Legendre nodes come from Newton's
// method on the three-term recurrence.
struct NormalRule {
  static constexpr int kOrder = 8, kPanels = 160;
  static constexpr double kHalfWidth = 10.0;
  std::vector<double> xi, w;
  NormalRule() {
    double x[kOrder], wl[kOrder];
    for (int i = 0; i < kOrder; ++i) {
      double t = std::cos(M_PI * (i + 0.75) / (kOrder + 0.5)), dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = t;
        for (int k = 2; k <= kOrder; ++k) {
          const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = kOrder * (t * p1 - p0) / (t * t - 1.0);
        const double dt = p1 / dp;
        t -= dt;
        if (std::fabs(dt) < 1e-16) break;
      }
      x[i] = t;
      wl[i] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
    const double h = 2.0 * kHalfWidth / kPanels;
    for (int p = 0; p < kPanels; ++p)
      for (int i = 0; i < kOrder; ++i) {
        const double v = -kHalfWidth + h * (p + 0.5) + 0.5 * h * x[i];
        xi.push_back(v);
        w.push_back(0.5 * h * wl[i] * std::exp(-0.5 * v * v) / std::sqrt(2.0 * M_PI));
      }
  }
};

const NormalRule &normal_rule() {
  static const NormalRule r;
  return r;
}

// F-bar, sigma_F and their derivatives in (ln a, ln s): J[0] = dFbar, J[1] = dsigma_F.
void gauss_moments(double a, double s, double *fbar, double *sig, double J[2][2]) {
  const NormalRule &R = normal_rule();
  double m1 = 0, m2 = 0, d1a = 0, d1s = 0, d2a = 0, d2s = 0;
  for (size_t i = 0; i < R.xi.size(); ++i) {
    const double tau = a * std::exp(s * R.xi[i]);  // optical depth
    const double F = std::exp(-tau), wt = R.w[i];
    m1 += wt * F;
    m2 += wt * F * F;
    d1a -= wt * tau * F;  // dF/d ln a = -tau F
    d1s -= wt * tau * s * R.xi[i] * F;  // dF/d ln s = -tau s xi F
    d2a -= 2.0 * wt * tau * F * F;
    d2s -= 2.0 * wt * tau * s * R.xi[i] * F * F;
  }
  const double v = std::max(m2 - m1 * m1, 0.0), sg = std::sqrt(v);
  *fbar = m1;
  *sig = sg;
  if (J) {
    J[0][0] = d1a;
    J[0][1] = d1s;
    const double inv = sg > 0 ? 0.5 / sg : 0.0;
    J[1][0] = (d2a - 2.0 * m1 * d1a) * inv;
    J[1][1] = (d2s - 2.0 * m1 * d1s) * inv;
  }
}

// Newton in (ln a, ln s), steps capped at 0.5 in either; starts from the
// small-dispersion limit (F-bar = e^-a, sigma_F = a F-bar s).
bool fit_a_s(double fbar, double sigf, double *a_out, double *s_out) {
  if (!(fbar > 0.0 && fbar < 1.0) || !(sigf > 0.0 && sigf < std::sqrt(fbar * (1.0 - fbar)))) return false;
  double la = std::log(-std::log(fbar));
  double ls = std::log(sigf / (-std::log(fbar) * fbar));
  for (int it = 0; it < 300; ++it) {
    double f, sg, J[2][2];
    gauss_moments(std::exp(la), std::exp(ls), &f, &sg, J);
    const double r0 = f - fbar, r1 = sg - sigf;
    if (std::fabs(r0) < 1e-14 && std::fabs(r1) < 1e-14) {
      *a_out = std::exp(la);
      *s_out = std::exp(ls);
      return true;
    }
    const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    if (!(std::fabs(det) > 0.0)) return false;
    double d0 = -(J[1][1] * r0 - J[0][1] * r1) / det;
    double d1 = -(-J[1][0] * r0 + J[0][0] * r1) / det;
    const double big = std::max(std::fabs(d0), std::fabs(d1));
    if (big > 0.5) {
      d0 *= 0.5 / big;
      d1 *= 0.5 / big;
    }
    la += d0;
    ls += d1;
  }
  return false;
}

// sigma_F of the target from the DFT-mode sum of its binned P1D_dF.
double sigma_f_of_p1d(double fbar, const double *p1d, int n_k, int n_fft_p1d, double dr) {
  const int q = (n_fft_p1d / 2) / n_k;
  double sum = 0.0;
  for (int k = 0; k < n_k; ++k) sum += p1d[k];
  const double modes = 2.0 * q * sum - p1d[n_k - 1];  // m = 1..N-1; Nyquist counted once
  return fbar * std::sqrt(modes / (n_fft_p1d * dr));
}

// var(delta_tot + c eta) from a bin's pixel sums (0 n, 3 d, 4 e, 5 dd, 6 ee, 7 de).
double var_g(const double *S, double c) {
  const double n = S[0], md = S[3] / n, me = S[4] / n;
  return (S[5] / n - md * md) + c * c * (S[6] / n - me * me) + 2.0 * c * (S[7] / n - md * me);
}

}  // namespace

extern "C" int mk_fgpa_gauss_moments(double a, double s, double *fbar, double *sigma_f) {
  if (!(a > 0.0) || !(s >= 0.0) || !fbar || !sigma_f) return MK_EINVAL;
  gauss_moments(a, s, fbar, sigma_f, nullptr);
  return MK_OK;
}

extern "C" int mk_fit_a_bsigma(double fbar, double sigma_f, double *a, double *s) {
  if (!a || !s) return MK_EINVAL;
  return fit_a_s(fbar, sigma_f, a, s) ? MK_OK : MK_EINVAL;
}

extern "C" int mk_tune_ps(mk_ctx *ctx, const mk_box *box, const mk_qso *d_qso, int64_t n_qso,
                          const mk_skewer_params *params, const mk_stat_bins *bins, const mk_tune_target *target,
                          int32_t n_outer, int32_t n_inner, mk_skewer *d_sk, int64_t *d_offsets, double *h_p_s,
                          mk_fgpa_nodes *out, mk_ps_tune_report *report) {
  MK_TRACE("mk_tune_ps");
  if (!ctx) return MK_EINVAL;
  if (!box || !params || !bins || !target || !h_p_s || !out || !report || !d_sk || !d_offsets)
    return pfail(ctx, MK_EINVAL, "mk_tune_ps: NULL argument");
  if (n_outer < 1 || n_inner < 0 || static_cast<int64_t>(n_outer) * (1 + n_inner) + 1 > MK_PS_TUNE_MAX_PASSES)
    return pfail(ctx, MK_EINVAL, "mk_tune_ps: need n_outer >= 1, n_inner >= 0 and at most MK_PS_TUNE_MAX_PASSES passes");
  const int nz = bins->n_z, nk = bins->n_k;
  if (nz < 1 || nz > MK_MAX_ZBINS || nk < 1 || nk > MK_MAX_KBINS || bins->n_fft < 2 || (bins->n_fft / 2) % nk)
    return pfail(ctx, MK_EINVAL, "mk_tune_ps: bad statistics bins");
  if (target->k_lo < 0 || target->k_hi > nk || target->k_hi <= target->k_lo)
    return pfail(ctx, MK_EINVAL, "mk_tune_ps: bad k range");
  const int nm = params->n_fft / 2 + 1;
  std::vector<int> tuned;
  for (int i = 0; i < nz; ++i) {
    if (!((target->active >> i) & 1u)) continue;
    tuned.push_back(i);
    if (!target->use_beta) return pfail(ctx, MK_EINVAL, "mk_tune_ps: c comes from the target beta (use_beta = 1)");
    if (!(target->mean_flux[i] > 0.0 && target->mean_flux[i] < 1.0))
      return pfail(ctx, MK_EINVAL, "mk_tune_ps: target mean flux outside (0, 1)");
    for (int k = 0; k < nk; ++k)
      if (!(target->p1d[i][k] > 0.0)) return pfail(ctx, MK_EINVAL, "mk_tune_ps: target P1D must be > 0 in every k bin");
  }
  if (tuned.empty()) return pfail(ctx, MK_EINVAL, "mk_tune_ps: no active z bin");
  std::memset(report, 0, sizeof(*report));
  const auto t0 = std::chrono::steady_clock::now();

  // nodes at the bin centres; untuned nodes copy the nearest tuned one
  std::vector<int> src(nz);
  for (int i = 0; i < nz; ++i) {
    int best = tuned[0];
    for (int j : tuned)
      if (std::abs(j - i) < std::abs(best - i)) best = j;
    src[i] = best;
  }
  std::vector<double> zc(nz), a(nz, 1.0), s(nz, 1.0), b(nz, 1.0), c(nz, 1.0);
  for (int i = 0; i < nz; ++i) zc[i] = bins->z_lo + (i + 0.5) * bins->dz;
  // steps 1-2: c from beta, (a, b sigma_g) from F-bar and the P1D integral
  for (int i : tuned) {
    c[i] = target->beta[i];
    const double sf = sigma_f_of_p1d(target->mean_flux[i], target->p1d[i], nk, bins->n_fft, params->dr);
    report->sigma_f_target[i] = sf;
    if (!fit_a_s(target->mean_flux[i], sf, &a[i], &s[i])) {
      char msg[160];
      snprintf(msg, sizeof(msg), "mk_tune_ps: no (a, b sigma_g) gives F-bar %.4g and sigma_F %.4g in z bin %d",
               target->mean_flux[i], sf, i);
      return pfail(ctx, MK_EINVAL, msg);
    }
  }
  auto follow = [&](std::vector<double> &v) {
    for (int i = 0; i < nz; ++i) v[i] = v[src[i]];
  };
  follow(a);
  follow(s);
  follow(c);
  for (int i = 0; i < nz; ++i) report->bsigma[i] = s[i];

  std::vector<double> ps(h_p_s, h_p_s + static_cast<size_t>(nz) * nm);
  // k bin of every P_S mode
  std::vector<int> mbin(nm, 0);
  const int q = (bins->n_fft / 2) / nk;
  for (int m = 1; m < nm; ++m) {
    int mp = static_cast<int>(std::floor(static_cast<double>(m) * bins->n_fft / params->n_fft + 0.5));
    mp = std::min(std::max(mp, 1), bins->n_fft / 2);
    mbin[m] = (mp - 1) / q;
  }

  mk_skewer_params p = *params;
  p.p_s_nodes = nz >= 2 ? nz : 0;
  p.h_p_s_z = zc.data();
  p.h_p_s = ps.data();
  mk_fgpa_nodes nd;
  std::memset(&nd, 0, sizeof(nd));
  nd.count = nz;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return pfail(ctx, MK_ECUDA, "mk_tune_ps: cudaEventCreate failed");
  }
  mk_stats_out st;
  auto run_pass = [&]() -> int {
    for (int i = 0; i < nz; ++i) {
      nd.z[i] = zc[i];
      nd.ln_a[i] = std::log(a[i]);
      nd.b[i] = b[i];
      nd.c[i] = c[i];
    }
    const cudaStream_t stream = mkhost::ctx_stream(ctx);
    cudaEventRecord(e0, stream);
    const int rc = mk_run(ctx, box, d_qso, n_qso, &p, &nd, bins, MK_STATS, d_sk, d_offsets, nullptr, nullptr,
                          nullptr, 0, &st);
    if (rc) return rc;
    cudaEventRecord(e1, stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    report->gpu_ms += ms;
    double dp = 0.0;
    for (int i : tuned)
      for (int k = target->k_lo; k < target->k_hi; ++k)
        dp = std::max(dp, std::fabs(st.p1d_df[i][k] / target->p1d[i][k] - 1.0));
    report->max_rel_p1d_pass[report->passes] = dp;
    report->passes += 1;
    return MK_OK;
  };

  int rc = MK_OK;
  for (int o = 0; o < n_outer && rc == MK_OK; ++o) {
    // step 3: sigma_g on the skewers, b = (b sigma_g) / sigma_g
    if ((rc = run_pass())) break;
    for (int i : tuned) {
      const double v = var_g(st.sums[i], c[i]);
      if (!(v > 0.0)) {
        rc = pfail(ctx, MK_EINVAL, "mk_tune_ps: a tuned z bin has no pixel variance");
        break;
      }
      report->sigma_g[i] = std::sqrt(v);
      b[i] = s[i] / std::sqrt(v);
      if (o > 0) {
        // keep F-bar (Sec. 2.6 makes small adjustments of a between outer
        // loops): one Newton step in ln a on this pass's mean flux, with the
        // slope of the Gaussian-field model at (a, b sigma_g)
        double f, sg, J[2][2];
        gauss_moments(a[i], s[i], &f, &sg, J);
        if (J[0][0] < 0.0) {
          const double dla = (st.mean_flux[i] - target->mean_flux[i]) / (-J[0][0]);
          a[i] *= std::exp(std::max(-0.5, std::min(0.5, dla)));
        }
      }
    }
    if (rc) break;
    follow(a);
    follow(b);
    // step 4: ratio iteration of P_S
    for (int it = 0; it < n_inner && rc == MK_OK; ++it) {
      if ((rc = run_pass())) break;
      for (int i : tuned) {
        double ratio[MK_MAX_KBINS];
        for (int k = 0; k < nk; ++k) {
          if (!(st.p1d_df[i][k] > 0.0)) {
            rc = pfail(ctx, MK_EINVAL, "mk_tune_ps: a tuned z bin has no P1D segment");
            break;
          }
          ratio[k] = target->p1d[i][k] / st.p1d_df[i][k];
        }
        if (rc) break;
        for (int m = 1; m < nm; ++m) ps[static_cast<size_t>(i) * nm + m] *= ratio[mbin[m]];
      }
      for (int i = 0; i < nz; ++i)
        if (src[i] != i)
          std::copy(ps.begin() + static_cast<size_t>(src[i]) * nm, ps.begin() + static_cast<size_t>(src[i] + 1) * nm,
                    ps.begin() + static_cast<size_t>(i) * nm);
    }
  }
  if (rc == MK_OK) rc = run_pass();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  double df = 0.0, db = 0.0;
  for (int i : tuned) {
    df = std::max(df, std::fabs(st.mean_flux[i] - target->mean_flux[i]));
    db = std::max(db, std::fabs(st.beta_f[i] / target->beta[i] - 1.0));
  }
  report->max_abs_dfbar = df;
  report->max_rel_p1d = report->max_rel_p1d_pass[report->passes - 1];
  report->max_rel_beta = db;
  report->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  std::copy(ps.begin(), ps.end(), h_p_s);
  *out = nd;
  return MK_OK;
}
