// Surrogate MLP objects, surrogate training data and the tuning of a, b, c.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "../../include/mockskewer.h"
#include "mk_host.h"
#include "mk_mlp.h"
#include "mk_trace.h"

using namespace mk;

struct mk_mlp {
  mk_ctx *ctx = nullptr;
  int device = 0;  // kept so that destruction does not depend on the context
  int64_t cap = 0;
  float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  void *wbf = nullptr;  // canonical BF16 copy (mk_mlp_get_params)
  void *img = nullptr;  // weight image the tensor-core kernels read
  double *d_loss = nullptr, *h_loss = nullptr;  // per-step losses (pinned host copy)
  int64_t loss_cap = 0;
  int64_t step = 0;
};

namespace {

int mfail(mk_ctx *ctx, int code, const char *msg) { return mkhost::ctx_fail(ctx, code, msg); }

#define CKM(ctx, call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      char b_[256];                                                                        \
      snprintf(b_, sizeof(b_), "%s: %s", #call, cudaGetErrorString(e_));                    \
      return mfail(ctx, MK_ECUDA, b_);                                                     \
    }                                                                                      \
  } while (0)

void mlp_free(mk_mlp *p) {
  cudaFree(p->master);
  cudaFree(p->m);
  cudaFree(p->v);
  cudaFree(p->grad);
  cudaFree(p->wbf);
  cudaFree(p->img);
  cudaFree(p->d_loss);
  cudaFreeHost(p->h_loss);
}

// room for n per-step losses
int ensure_loss(mk_mlp *p, int64_t n) {
  if (n <= p->loss_cap) return MK_OK;
  cudaFree(p->d_loss);
  cudaFreeHost(p->h_loss);
  p->d_loss = nullptr;
  p->h_loss = nullptr;
  p->loss_cap = 0;
  if (cudaMalloc(&p->d_loss, sizeof(double) * n) != cudaSuccess ||
      cudaMallocHost(&p->h_loss, sizeof(double) * n) != cudaSuccess)
    return mfail(p->ctx, MK_ENOMEM, "surrogate MLP loss buffer");
  p->loss_cap = n;
  return MK_OK;
}

MlpRun run_args(mk_mlp *p) {
  MlpRun R{};
  R.b1 = 0.9f;
  R.b2 = 0.999f;
  R.eps = 1e-8f;
  R.master = p->master;
  R.m = p->m;
  R.v = p->v;
  R.grad = p->grad;
  R.img = p->img;
  return R;
}

}  // namespace

// ====================================================================== MLP
extern "C" int mk_mlp_create(mk_ctx *ctx, mk_mlp **out, int64_t max_batch, uint64_t seed) {
  if (!ctx || !out) return MK_EINVAL;
  *out = nullptr;
  if (max_batch < 1 || max_batch > (1 << 24)) return mfail(ctx, MK_EINVAL, "max_batch must be in [1, 2^24]");
  CKM(ctx, cudaSetDevice(mkhost::ctx_device(ctx)));
  mk_mlp *p = new mk_mlp();
  p->ctx = ctx;
  p->device = mkhost::ctx_device(ctx);
  p->cap = max_batch;
  const size_t np = sizeof(float) * kMlpParams;
  if (cudaMalloc(&p->master, np) != cudaSuccess || cudaMalloc(&p->m, np) != cudaSuccess ||
      cudaMalloc(&p->v, np) != cudaSuccess || cudaMalloc(&p->grad, np) != cudaSuccess ||
      cudaMalloc(&p->wbf, sizeof(uint16_t) * kMlpParams) != cudaSuccess ||
      cudaMalloc(&p->img, mlp_image_bytes()) != cudaSuccess) {
    mlp_free(p);
    delete p;
    return mfail(ctx, MK_ENOMEM, "surrogate MLP allocation");
  }
  // He initialisation: W ~ N(0, 2 / fan_in), b = 0
  std::vector<float> h(kMlpParams, 0.f);
  std::mt19937_64 rng(seed);
  const int dims[5] = {kMlpIn, kMlpHidden, kMlpHidden, kMlpHidden, kMlpOut};
  size_t o = 0;
  for (int l = 0; l < 4; ++l) {
    std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / dims[l]));
    for (int i = 0; i < dims[l + 1] * dims[l]; ++i) h[o++] = static_cast<float>(nd(rng));
    o += dims[l + 1];
  }
  *out = p;
  return mk_mlp_set_params(p, h.data());
}

extern "C" void mk_mlp_destroy(mk_mlp *mlp) {
  if (!mlp) return;
  cudaSetDevice(mlp->device);
  cudaDeviceSynchronize();
  mlp_free(mlp);
  delete mlp;
}

extern "C" int mk_mlp_set_params(mk_mlp *p, const float *h_params) {
  if (!p || !h_params) return MK_EINVAL;
  mk_ctx *ctx = p->ctx;
  cudaStream_t st = mkhost::ctx_stream(ctx);
  CKM(ctx, cudaSetDevice(mkhost::ctx_device(ctx)));
  CKM(ctx, cudaMemcpyAsync(p->master, h_params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, st));
  CKM(ctx, cudaMemsetAsync(p->m, 0, sizeof(float) * kMlpParams, st));
  CKM(ctx, cudaMemsetAsync(p->v, 0, sizeof(float) * kMlpParams, st));
  CKM(ctx, mlp_pack(p->master, p->img, p->wbf, st));
  CKM(ctx, cudaStreamSynchronize(st));
  p->step = 0;
  return MK_OK;
}

extern "C" int mk_mlp_get_params(mk_mlp *p, float *h_params, uint16_t *h_bf16) {
  if (!p) return MK_EINVAL;
  mk_ctx *ctx = p->ctx;
  cudaStream_t st = mkhost::ctx_stream(ctx);
  CKM(ctx, cudaSetDevice(mkhost::ctx_device(ctx)));
  if (h_params)
    CKM(ctx, cudaMemcpyAsync(h_params, p->master, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, st));
  if (h_bf16) {
    CKM(ctx, mlp_pack(p->master, p->img, p->wbf, st));  // the BF16 copy of the current master
    CKM(ctx, cudaMemcpyAsync(h_bf16, p->wbf, sizeof(uint16_t) * kMlpParams, cudaMemcpyDeviceToHost, st));
  }
  CKM(ctx, cudaStreamSynchronize(st));
  return MK_OK;
}

extern "C" int mk_mlp_forward(mk_mlp *p, const float *d_x, int64_t n, float *d_y) {
  MK_TRACE("mk_mlp_forward");
  if (!p) return MK_EINVAL;
  if (n < 0 || (n > 0 && (!d_x || !d_y))) return mfail(p->ctx, MK_EINVAL, "bad forward arguments");
  CKM(p->ctx, cudaSetDevice(mkhost::ctx_device(p->ctx)));
  CKM(p->ctx, mlp_forward(p->img, d_x, n, d_y, mkhost::ctx_stream(p->ctx)));
  return MK_OK;
}

extern "C" int mk_mlp_loss_grad(mk_mlp *p, const float *d_x, const float *d_t, int64_t n, double *h_loss,
                                float *h_grad) {
  MK_TRACE("mk_mlp_loss_grad");
  if (!p) return MK_EINVAL;
  if (n < 1 || n > p->cap || !d_x || !d_t) return mfail(p->ctx, MK_EINVAL, "n must be in [1, max_batch]");
  mk_ctx *ctx = p->ctx;
  cudaStream_t st = mkhost::ctx_stream(ctx);
  CKM(ctx, cudaSetDevice(mkhost::ctx_device(ctx)));
  int rc = ensure_loss(p, 1);
  if (rc) return rc;
  // one step over all n samples (passes of kMlpChunk), no update
  MlpRun R = run_args(p);
  R.x = d_x;
  R.t = d_t;
  R.n = n;
  R.batch = static_cast<int32_t>(std::min<int64_t>(n, INT32_MAX));
  R.steps = 1;
  R.inv_count = 1.0 / (static_cast<double>(n) * kMlpOut);
  R.loss_out = p->d_loss;
  CKM(ctx, mlp_cluster_run(R, st));
  if (h_grad)
    CKM(ctx, cudaMemcpyAsync(h_grad, p->grad, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, st));
  CKM(ctx, cudaMemcpyAsync(p->h_loss, p->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  CKM(ctx, cudaStreamSynchronize(st));
  if (h_loss) *h_loss = p->h_loss[0];
  return MK_OK;
}

extern "C" int mk_mlp_adam_step(mk_mlp *p, const float *d_grad, float lr) {
  if (!p) return MK_EINVAL;
  if (!d_grad || !(lr > 0.f)) return mfail(p->ctx, MK_EINVAL, "mk_mlp_adam_step needs a gradient and lr > 0");
  mk_ctx *ctx = p->ctx;
  CKM(ctx, cudaSetDevice(mkhost::ctx_device(ctx)));
  CKM(ctx, mlp_adam(p->master, p->m, p->v, d_grad, p->img, lr, 0.9f, 0.999f, 1e-8f, ++p->step,
                    mkhost::ctx_stream(ctx)));
  return MK_OK;
}

extern "C" int mk_mlp_train(mk_mlp *p, const float *d_x, const float *d_t, int64_t n, int32_t batch,
                            int32_t epochs, float lr, uint64_t seed, double *h_epoch_loss) {
  MK_TRACE("mk_mlp_train");
  if (!p) return MK_EINVAL;
  mk_ctx *ctx = p->ctx;
  if (n < 1 || !d_x || !d_t || batch < 1 || batch > p->cap || epochs < 0 || !(lr > 0.f))
    return mfail(ctx, MK_EINVAL, "bad training arguments (n >= 1, 1 <= batch <= max_batch, lr > 0)");
  if (n > INT32_MAX) return mfail(ctx, MK_EINVAL, "too many samples");
  cudaStream_t st = mkhost::ctx_stream(ctx);
  CKM(ctx, cudaSetDevice(mkhost::ctx_device(ctx)));
  const int64_t steps = (n + batch - 1) / batch;
  int rc = ensure_loss(p, std::max<int64_t>(1, steps * epochs));
  if (rc) return rc;
  // per epoch: a shuffled sample order (host RNG), uploaded through two
  // pinned buffers so that the next shuffle overlaps the running epoch
  int32_t *d_rows[2] = {nullptr, nullptr}, *h_rows[2] = {nullptr, nullptr};
  cudaEvent_t up[2] = {nullptr, nullptr};
  bool ok = true;
  for (int k = 0; k < 2 && ok; ++k)
    ok = cudaMalloc(&d_rows[k], sizeof(int32_t) * n) == cudaSuccess &&
         cudaMallocHost(&h_rows[k], sizeof(int32_t) * n) == cudaSuccess &&
         cudaEventCreateWithFlags(&up[k], cudaEventDisableTiming) == cudaSuccess;
  std::vector<int32_t> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  std::mt19937_64 rng(seed);
  if (!ok) rc = mfail(ctx, MK_ENOMEM, "training index arrays");
  for (int e = 0; e < epochs && rc == MK_OK; ++e) {
    std::shuffle(perm.begin(), perm.end(), rng);
    const int k = e & 1;
    if (e >= 2 && cudaEventSynchronize(up[k]) != cudaSuccess) {  // the copy from this buffer is done
      rc = mfail(ctx, MK_ECUDA, "training index upload");
      break;
    }
    std::memcpy(h_rows[k], perm.data(), sizeof(int32_t) * n);
    if (cudaMemcpyAsync(d_rows[k], h_rows[k], sizeof(int32_t) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaEventRecord(up[k], st) != cudaSuccess) {
      rc = mfail(ctx, MK_ECUDA, "training index upload");
      break;
    }
    MlpRun R = run_args(p);
    R.x = d_x;
    R.t = d_t;
    R.rows = d_rows[k];
    R.n = n;
    R.batch = batch;
    R.steps = static_cast<int32_t>(steps);
    R.train = 1;
    R.lr = static_cast<float>(lr * (0.05 + 0.95 * 0.5 * (1.0 + std::cos(M_PI * e / std::max(1, epochs)))));
    R.t0 = p->step;
    R.loss_out = p->d_loss + static_cast<int64_t>(e) * steps;
    cudaError_t ce = mlp_cluster_run(R, st);
    // the kernel updated the weight images in shared memory only: refresh the
    // global image (the next launch and inference read it)
    if (ce == cudaSuccess) ce = mlp_pack(p->master, p->img, nullptr, st);
    if (ce != cudaSuccess) {
      rc = mfail(ctx, MK_ECUDA, cudaGetErrorString(ce));
      break;
    }
    p->step += steps;
  }
  if (rc == MK_OK && h_epoch_loss && epochs > 0) {
    if (cudaMemcpyAsync(p->h_loss, p->d_loss, sizeof(double) * steps * epochs, cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
      rc = mfail(ctx, MK_ECUDA, "training loss readback");
  }
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == MK_OK) rc = mfail(ctx, MK_ECUDA, "training");
  if (rc == MK_OK && h_epoch_loss) {
    for (int e = 0; e < epochs; ++e) {  // mean over the epoch's samples
      double s = 0.0;
      for (int64_t i = 0; i < steps; ++i) {
        const int64_t nb = std::min<int64_t>(batch, n - i * batch);
        s += p->h_loss[e * steps + i] * nb;
      }
      h_epoch_loss[e] = s / n;
    }
  }
  for (int k = 0; k < 2; ++k) {
    cudaFree(d_rows[k]);
    cudaFreeHost(h_rows[k]);
    if (up[k]) cudaEventDestroy(up[k]);
  }
  return rc;
}

// ====================================================================== surrogate data
namespace {

// Effective parameters of a z bin: the FGPA parameters ln a, b, c are linear
// in z between nodes (clamped at the ends), so the pixels of bin i see a blend
// of nodes i - 1, i, i + 1.  To first order a bin's statistics are those at
// constant parameters equal to the pixel-weighted mean of the interpolated
// parameters, theta_eff = W theta, with W[i][j] the mean interpolation weight
// of node j over the pixels of bin i (inactive nodes folded into the nearest
// active node they follow).  Tuning solves each bin for theta_eff and maps
// back to the nodes through W.
struct EffMap {
  int nz = 0;
  std::vector<int> act;   // active bins (= active nodes), ascending
  std::vector<double> W;  // nz x nz
  bool identity = true;

  int build(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
            const mk_stat_bins *bins, uint32_t active, const mk_fgpa_nodes &nd, double *gpu_ms) {
    nz = bins->n_z;
    act.clear();
    for (int i = 0; i < nz; ++i)
      if ((active >> i) & 1u) act.push_back(i);
    W.assign(static_cast<size_t>(nz) * nz, 0.0);
    for (int i = 0; i < nz; ++i) W[static_cast<size_t>(i) * nz + i] = 1.0;
    identity = true;
    std::vector<double> zj;
    std::vector<int64_t> cnt;
    int rc = mkhost::ctx_pixel_histogram(ctx, params->dr, d_sk, n_sk, zj, cnt, gpu_ms);
    if (rc) return rc;
    std::vector<double> acc(static_cast<size_t>(nz) * nz, 0.0), tot(nz, 0.0);
    const int k = nd.count;
    for (size_t j = 0; j < zj.size(); ++j) {
      if (cnt[j] <= 0) continue;
      const double z = zj[j];
      const double f = std::floor((z - bins->z_lo) / bins->dz);
      if (f < 0.0 || f >= nz) continue;
      const int zb = static_cast<int>(f);
      const double c = static_cast<double>(cnt[j]);
      tot[zb] += c;
      // the node interpolation of the pixel table
      if (z <= nd.z[0]) {
        acc[static_cast<size_t>(zb) * nz] += c;
      } else if (z >= nd.z[k - 1]) {
        acc[static_cast<size_t>(zb) * nz + k - 1] += c;
      } else {
        int i = 0;
        while (i + 2 < k && z >= nd.z[i + 1]) ++i;
        const double w = (z - nd.z[i]) / (nd.z[i + 1] - nd.z[i]);
        acc[static_cast<size_t>(zb) * nz + i] += c * (1.0 - w);
        acc[static_cast<size_t>(zb) * nz + i + 1] += c * w;
      }
    }
    // fold inactive nodes into the active node they follow
    std::vector<int> follow(nz, -1);
    for (int i = 0; i < nz; ++i) {
      if ((active >> i) & 1u) {
        follow[i] = i;
        continue;
      }
      for (int j : act)
        if (follow[i] < 0 || std::abs(j - i) < std::abs(follow[i] - i)) follow[i] = j;
    }
    for (int zb : act) {
      if (!(tot[zb] > 0.0)) continue;
      for (int j = 0; j < nz; ++j) W[static_cast<size_t>(zb) * nz + j] = 0.0;
      for (int j = 0; j < nz; ++j)
        if (follow[j] >= 0) W[static_cast<size_t>(zb) * nz + follow[j]] += acc[static_cast<size_t>(zb) * nz + j] / tot[zb];
    }
    identity = false;
    return MK_OK;
  }

  // theta_eff of the active bins, tb[3 zb + p]
  void eff(const mk_fgpa_nodes &nd, std::vector<double> &tb) const {
    tb.assign(static_cast<size_t>(nz) * 3, 0.0);
    for (int zb : act)
      for (int j : act) {
        const double w = W[static_cast<size_t>(zb) * nz + j];
        tb[3 * zb] += w * nd.ln_a[j];
        tb[3 * zb + 1] += w * nd.b[j];
        tb[3 * zb + 2] += w * nd.c[j];
      }
  }

  // active nodes whose theta_eff is tb (W restricted to the active bins and
  // nodes, Gaussian elimination with partial pivoting); the caller sets the
  // inactive nodes
  void nodes(const std::vector<double> &tb, mk_fgpa_nodes &nd) const {
    const int n = static_cast<int>(act.size());
    std::vector<double> M(static_cast<size_t>(n) * (n + 3));
    for (int r = 0; r < n; ++r) {
      for (int c = 0; c < n; ++c) M[static_cast<size_t>(r) * (n + 3) + c] = W[static_cast<size_t>(act[r]) * nz + act[c]];
      for (int p = 0; p < 3; ++p) M[static_cast<size_t>(r) * (n + 3) + n + p] = tb[3 * act[r] + p];
    }
    bool ok = true;
    for (int c = 0; c < n && ok; ++c) {
      int piv = c;
      for (int r = c + 1; r < n; ++r)
        if (std::fabs(M[static_cast<size_t>(r) * (n + 3) + c]) > std::fabs(M[static_cast<size_t>(piv) * (n + 3) + c])) piv = r;
      if (std::fabs(M[static_cast<size_t>(piv) * (n + 3) + c]) < 1e-9) {
        ok = false;
        break;
      }
      for (int q = 0; q < n + 3; ++q) std::swap(M[static_cast<size_t>(c) * (n + 3) + q], M[static_cast<size_t>(piv) * (n + 3) + q]);
      for (int r = 0; r < n; ++r) {
        if (r == c) continue;
        const double f = M[static_cast<size_t>(r) * (n + 3) + c] / M[static_cast<size_t>(c) * (n + 3) + c];
        for (int q = c; q < n + 3; ++q) M[static_cast<size_t>(r) * (n + 3) + q] -= f * M[static_cast<size_t>(c) * (n + 3) + q];
      }
    }
    for (int r = 0; r < n; ++r) {
      const int j = act[r];
      for (int p = 0; p < 3; ++p) {
        const double v = ok ? M[static_cast<size_t>(r) * (n + 3) + n + p] / M[static_cast<size_t>(r) * (n + 3) + r]
                            : tb[3 * j + p];  // singular map: nodes take the bin values
        (p == 0 ? nd.ln_a : p == 1 ? nd.b : nd.c)[j] = v;
      }
    }
  }
};


bool valid_stat_sample(const mk_stats_out &st, int zb, int n_k) {
  if (st.sums[zb][0] <= 0.0 || st.n_seg[zb] <= 0.0 || !(st.mean_flux[zb] > 1e-3)) return false;
  if (!std::isfinite(st.b_f[zb]) || !std::isfinite(st.beta_f[zb])) return false;
  for (int k = 0; k < n_k; ++k)
    if (!(st.p1d_df[zb][k] > 0.0) || !std::isfinite(std::log(st.p1d_df[zb][k]))) return false;
  return true;
}

void stat_vector(const mk_stats_out &st, int zb, double *t) {
  t[0] = st.mean_flux[zb];
  t[1] = st.b_f[zb];
  t[2] = st.beta_f[zb];
  for (int k = 0; k < 32; ++k) t[3 + k] = std::log(st.p1d_df[zb][k]);
}

mk_fgpa_nodes constant_nodes(const mk_stat_bins *b, double ln_a, double bb, double c) {
  mk_fgpa_nodes nd;
  std::memset(&nd, 0, sizeof(nd));
  nd.count = b->n_z;
  for (int i = 0; i < b->n_z; ++i) {
    nd.z[i] = b->z_lo + (i + 0.5) * b->dz;
    nd.ln_a[i] = ln_a;
    nd.b[i] = bb;
    nd.c[i] = c;
  }
  return nd;
}

}  // namespace

extern "C" int mk_surrogate_labels(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
                                   const int64_t *d_offsets, const float *d_delta, const float *d_eta,
                                   const mk_stat_bins *bins, const mk_surrogate_space *space, int32_t n_draws,
                                   uint64_t seed, double *h_x, double *h_t, int64_t *h_count) {
  MK_TRACE("mk_surrogate_labels");
  if (!ctx) return MK_EINVAL;
  if (!bins || bins->n_k != 32 || !space || n_draws < 0 || !h_x || !h_t || !h_count)
    return mfail(ctx, MK_EINVAL, "surrogate labels need 32 k bins, a parameter space and host outputs");
  std::mt19937_64 rng(seed);
  std::uniform_real_distribution<double> ua(space->ln_a_min, space->ln_a_max), ub(space->b_min, space->b_max),
      uc(space->c_min, space->c_max), unit(-1.0, 1.0);
  const bool sloped = space->dln_a_dz_max > 0.0 || space->db_dz_max > 0.0 || space->dc_dz_max > 0.0;
  EffMap E;
  if (sloped) {
    // every bin counts as active: each node has its own value
    const mk_fgpa_nodes probe = constant_nodes(bins, 0.0, 0.0, 0.0);
    const uint32_t all = bins->n_z >= 32 ? 0xffffffffu : ((1u << bins->n_z) - 1u);
    const int rc = E.build(ctx, params, d_sk, n_sk, bins, all, probe, nullptr);
    if (rc) return rc;
  }
  const double zmid = bins->z_lo + 0.5 * bins->n_z * bins->dz;
  int64_t cnt = 0;
  mk_stats_out st;
  std::vector<double> tb;
  for (int d = 0; d < n_draws; ++d) {
    const double la = ua(rng), b = ub(rng), c = uc(rng);
    mk_fgpa_nodes nd = constant_nodes(bins, la, b, c);
    if (sloped) {
      const double sa = space->dln_a_dz_max * unit(rng), sb = space->db_dz_max * unit(rng),
                   sc = space->dc_dz_max * unit(rng);
      for (int i = 0; i < nd.count; ++i) {
        nd.ln_a[i] += sa * (nd.z[i] - zmid);
        nd.b[i] += sb * (nd.z[i] - zmid);
        nd.c[i] += sc * (nd.z[i] - zmid);
      }
      E.eff(nd, tb);
    }
    const int rc = mk_flux_stats(ctx, params, d_sk, n_sk, d_offsets, d_delta, d_eta, &nd, bins, &st);
    if (rc) return rc;
    for (int zb = 0; zb < bins->n_z; ++zb) {
      if (!valid_stat_sample(st, zb, 32)) continue;
      double *x = h_x + 4 * cnt;
      x[0] = nd.z[zb];
      x[1] = sloped ? tb[3 * zb] : la;
      x[2] = sloped ? tb[3 * zb + 1] : b;
      x[3] = sloped ? tb[3 * zb + 2] : c;
      stat_vector(st, zb, h_t + kMlpOut * cnt);
      ++cnt;
    }
  }
  *h_count = cnt;
  return MK_OK;
}

extern "C" int mk_surrogate_fit(mk_mlp *p, const double *h_x, const double *h_t, int64_t n, int32_t batch,
                                int32_t epochs, float lr, uint64_t seed, mk_surrogate_norm *norm,
                                double *h_epoch_loss) {
  MK_TRACE("mk_surrogate_fit");
  if (!p) return MK_EINVAL;
  mk_ctx *ctx = p->ctx;
  if (n < 2 || !h_x || !h_t || !norm) return mfail(ctx, MK_EINVAL, "surrogate fit needs >= 2 samples and a norm");
  std::memset(norm, 0, sizeof(*norm));
  auto moments = [&](const double *a, int stride, int col, double &mean, double &sd) {
    double s = 0.0, s2 = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i * stride + col];
    mean = s / n;
    for (int64_t i = 0; i < n; ++i) {
      const double d = a[i * stride + col] - mean;
      s2 += d * d;
    }
    sd = std::sqrt(s2 / n);
    if (!(sd > 1e-12)) sd = 1.0;
  };
  for (int c = 0; c < kMlpIn; ++c) moments(h_x, kMlpIn, c, norm->x_mean[c], norm->x_std[c]);
  for (int c = 0; c < kMlpOut; ++c) moments(h_t, kMlpOut, c, norm->t_mean[c], norm->t_std[c]);
  std::vector<float> xs(n * kMlpIn), ts(n * kMlpOut);
  for (int64_t i = 0; i < n; ++i) {
    for (int c = 0; c < kMlpIn; ++c)
      xs[i * kMlpIn + c] = static_cast<float>((h_x[i * kMlpIn + c] - norm->x_mean[c]) / norm->x_std[c]);
    for (int c = 0; c < kMlpOut; ++c)
      ts[i * kMlpOut + c] = static_cast<float>((h_t[i * kMlpOut + c] - norm->t_mean[c]) / norm->t_std[c]);
  }
  cudaStream_t st = mkhost::ctx_stream(ctx);
  CKM(ctx, cudaSetDevice(mkhost::ctx_device(ctx)));
  float *dx = nullptr, *dt = nullptr;
  if (cudaMalloc(&dx, sizeof(float) * xs.size()) != cudaSuccess ||
      cudaMalloc(&dt, sizeof(float) * ts.size()) != cudaSuccess) {
    cudaFree(dx);
    return mfail(ctx, MK_ENOMEM, "surrogate training set");
  }
  int rc = MK_OK;
  if (cudaMemcpyAsync(dx, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dt, ts.data(), sizeof(float) * ts.size(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = mfail(ctx, MK_ECUDA, "surrogate training set upload");
  if (!rc) rc = mk_mlp_train(p, dx, dt, n, batch, epochs, lr, seed, h_epoch_loss);
  cudaStreamSynchronize(st);
  cudaFree(dx);
  cudaFree(dt);
  return rc;
}

// ====================================================================== tuning
namespace {

struct Residuals {
  std::vector<double> r;  // per node, concatenated
  int m = 0;              // residuals per node
};

struct TuneState {
  mk_ctx *ctx;
  const mk_skewer_params *params;
  const mk_skewer *d_sk;
  int64_t n_sk;
  const int64_t *d_offsets;
  const float *d_delta, *d_eta;
  const mk_stat_bins *bins;
  const mk_tune_target *tg;
  mk_tune_report *rep;
  cudaEvent_t e0, e1;
  int nk() const { return tg->k_hi - tg->k_lo; }
  int m() const { return 1 + nk() + (tg->use_beta ? 1 : 0); }
  bool active(int zb) const { return (tg->active >> zb) & 1u; }
};

// Residual vector of one bin from statistic values (Fbar, beta, ln P1D), in
// units of the tolerances; the P1D block is scaled by 1/sqrt(k bins) so that it
// weighs in the least-squares steps like one statistic (F and beta are single
// numbers), and model noise spread over many k bins cannot outvote beta.
void residual(const TuneState &S, int zb, double fbar, double beta, const double *lnp, double *r) {
  const mk_tune_target *t = S.tg;
  r[0] = (fbar - t->mean_flux[zb]) / t->tol_mean_flux;
  const double wp = 1.0 / std::sqrt(static_cast<double>(S.nk()));
  for (int k = t->k_lo; k < t->k_hi; ++k)
    r[1 + k - t->k_lo] = wp * (lnp[k] - std::log(t->p1d[zb][k])) / t->tol_p1d;
  if (t->use_beta) r[1 + S.nk()] = (beta - t->beta[zb]) / (t->tol_beta * std::fabs(t->beta[zb]));
}

// One full tuning pass at `nodes`; residuals of every bin, GPU time added.
int full_pass(TuneState &S, const mk_fgpa_nodes &nodes, mk_stats_out &st, std::vector<double> &r) {
  cudaStream_t stream = mkhost::ctx_stream(S.ctx);
  cudaEventRecord(S.e0, stream);
  const int rc = mk_flux_stats(S.ctx, S.params, S.d_sk, S.n_sk, S.d_offsets, S.d_delta, S.d_eta, &nodes, S.bins, &st);
  if (rc) return rc;
  cudaEventRecord(S.e1, stream);
  cudaEventSynchronize(S.e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, S.e0, S.e1);
  S.rep->gpu_ms += ms;
  S.rep->passes += 1;
  const int m = S.m();
  r.assign(static_cast<size_t>(S.bins->n_z) * m, 0.0);
  double lnp[MK_MAX_KBINS];
  for (int zb = 0; zb < S.bins->n_z; ++zb) {
    if (!S.active(zb)) continue;
    for (int k = 0; k < S.bins->n_k; ++k) lnp[k] = std::log(std::max(st.p1d_df[zb][k], 1e-300));
    residual(S, zb, st.mean_flux[zb], st.beta_f[zb], lnp, &r[static_cast<size_t>(zb) * m]);
  }
  return MK_OK;
}

// Convergence check of a full pass; also fills the report's error measures.
bool converged(TuneState &S, const mk_stats_out &st) {
  const mk_tune_target *t = S.tg;
  double df = 0.0, dp = 0.0, db = 0.0;
  for (int zb = 0; zb < S.bins->n_z; ++zb) {
    if (!S.active(zb)) continue;
    df = std::max(df, std::fabs(st.mean_flux[zb] - t->mean_flux[zb]));
    for (int k = t->k_lo; k < t->k_hi; ++k) dp = std::max(dp, std::fabs(st.p1d_df[zb][k] / t->p1d[zb][k] - 1.0));
    if (t->use_beta) db = std::max(db, std::fabs(st.beta_f[zb] / t->beta[zb] - 1.0));
  }
  S.rep->max_abs_dfbar = df;
  S.rep->max_rel_p1d = dp;
  S.rep->max_rel_beta = db;
  return df <= t->tol_mean_flux && dp <= t->tol_p1d && (!t->use_beta || db <= t->tol_beta);
}

// Levenberg-Marquardt step for 3 parameters: (J^T J + lam diag) d = -J^T r.
void lm_step(const double *J, const double *r, int m, double lam, double *d) {
  double A[3][3] = {{0}}, g[3] = {0, 0, 0};
  for (int i = 0; i < m; ++i)
    for (int p = 0; p < 3; ++p) {
      g[p] += J[i * 3 + p] * r[i];
      for (int q = 0; q < 3; ++q) A[p][q] += J[i * 3 + p] * J[i * 3 + q];
    }
  for (int p = 0; p < 3; ++p) A[p][p] += lam * A[p][p] + 1e-12;
  // Gaussian elimination with partial pivoting on [A | -g]
  double M[3][4];
  for (int p = 0; p < 3; ++p) {
    for (int q = 0; q < 3; ++q) M[p][q] = A[p][q];
    M[p][3] = -g[p];
  }
  for (int c = 0; c < 3; ++c) {
    int piv = c;
    for (int rr = c + 1; rr < 3; ++rr)
      if (std::fabs(M[rr][c]) > std::fabs(M[piv][c])) piv = rr;
    for (int q = 0; q < 4; ++q) std::swap(M[c][q], M[piv][q]);
    for (int rr = c + 1; rr < 3; ++rr) {
      const double f = M[rr][c] / M[c][c];
      for (int q = c; q < 4; ++q) M[rr][q] -= f * M[c][q];
    }
  }
  for (int c = 2; c >= 0; --c) {
    double s = M[c][3];
    for (int q = c + 1; q < 3; ++q) s -= M[c][q] * d[q];
    d[c] = s / M[c][c];
  }
}

constexpr double kSurrogateStop = 1e-4;  // surrogate-only fits stop below this step

// Nodes of bins without data follow the nearest tuned node (ties: the lower).
void fill_inactive(mk_fgpa_nodes &nd, const TuneState &S) {
  const int nz = S.bins->n_z;
  for (int i = 0; i < nz; ++i) {
    if (S.active(i)) continue;
    int best = -1;
    for (int j = 0; j < nz; ++j)
      if (S.active(j) && (best < 0 || std::abs(j - i) < std::abs(best - i))) best = j;
    if (best < 0) return;
    nd.ln_a[i] = nd.ln_a[best];
    nd.b[i] = nd.b[best];
    nd.c[i] = nd.c[best];
  }
}

// Clamped LM step on the effective parameters of bin zb; returns its largest component.
double apply_step_eff(std::vector<double> &tb, int zb, const double *d) {
  const double lim[3] = {1.0, 0.4, 0.4};
  double s = 1.0;
  for (int p = 0; p < 3; ++p)
    if (std::fabs(d[p]) > lim[p]) s = std::min(s, lim[p] / std::fabs(d[p]));
  for (int p = 0; p < 3; ++p) tb[3 * zb + p] += s * d[p];
  return s * std::max(std::fabs(d[0]), std::max(std::fabs(d[1]), std::fabs(d[2])));
}

void shift(mk_fgpa_nodes &nd, int p, double h) {
  for (int i = 0; i < nd.count; ++i) {
    if (p == 0) nd.ln_a[i] += h;
    if (p == 1) nd.b[i] += h;
    if (p == 2) nd.c[i] += h;
  }
}

// Surrogate predictions at `rows` inputs (z, ln a, b, c): host in, host out.
struct Surrogate {
  mk_mlp *mlp;
  const mk_surrogate_norm *norm;
  float *dx = nullptr, *dy = nullptr;
  int cap = 0;
  int eval(TuneState &S, const std::vector<double> &x, std::vector<double> &t) {
    const int n = static_cast<int>(x.size() / 4);
    cudaStream_t st = mkhost::ctx_stream(S.ctx);
    if (n > cap) {
      cudaFree(dx);
      cudaFree(dy);
      dx = dy = nullptr;
      if (cudaMalloc(&dx, sizeof(float) * 4 * n) != cudaSuccess || cudaMalloc(&dy, sizeof(float) * 35 * n) != cudaSuccess)
        return mfail(S.ctx, MK_ENOMEM, "surrogate inference buffers");
      cap = n;
    }
    std::vector<float> xs(4 * n), ys(35 * n);
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 4; ++c) xs[4 * i + c] = static_cast<float>((x[4 * i + c] - norm->x_mean[c]) / norm->x_std[c]);
    cudaEventRecord(S.e0, st);
    CKM(S.ctx, cudaMemcpyAsync(dx, xs.data(), sizeof(float) * xs.size(), cudaMemcpyHostToDevice, st));
    int rc = mk_mlp_forward(mlp, dx, n, dy);
    if (rc) return rc;
    CKM(S.ctx, cudaMemcpyAsync(ys.data(), dy, sizeof(float) * ys.size(), cudaMemcpyDeviceToHost, st));
    cudaEventRecord(S.e1, st);
    CKM(S.ctx, cudaEventSynchronize(S.e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, S.e0, S.e1);
    S.rep->gpu_ms += ms;
    t.resize(35 * static_cast<size_t>(n));
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 35; ++c) t[35 * i + c] = ys[35 * i + c] * norm->t_std[c] + norm->t_mean[c];
    return MK_OK;
  }
  // residuals and central-difference Jacobians of all active bins at the
  // effective parameters tb (3 per bin) and bin centres zc (inference is
  // smooth in its inputs: its activations carry ~16 bits)
  int model(TuneState &S, const double *zc, const std::vector<double> &tb, std::vector<double> &r,
            std::vector<double> &J) {
    const double h[3] = {0.02, 0.02, 0.02};
    constexpr int kV = 7;  // centre, then (+h, -h) per parameter
    const int nz = S.bins->n_z, m = S.m();
    std::vector<double> x(static_cast<size_t>(nz) * kV * 4), t;
    for (int zb = 0; zb < nz; ++zb)
      for (int v = 0; v < kV; ++v) {
        double *xi = &x[(static_cast<size_t>(zb) * kV + v) * 4];
        const int p = (v - 1) / 2;
        const double d = v == 0 ? 0.0 : ((v - 1) % 2 == 0 ? h[p] : -h[p]);
        xi[0] = zc[zb];
        xi[1] = tb[3 * zb] + (v > 0 && p == 0 ? d : 0.0);
        xi[2] = tb[3 * zb + 1] + (v > 0 && p == 1 ? d : 0.0);
        xi[3] = tb[3 * zb + 2] + (v > 0 && p == 2 ? d : 0.0);
      }
    int rc = eval(S, x, t);
    if (rc) return rc;
    r.assign(static_cast<size_t>(nz) * m, 0.0);
    J.assign(static_cast<size_t>(nz) * m * 3, 0.0);
    std::vector<double> rp(m), rm(m);
    for (int zb = 0; zb < nz; ++zb) {
      if (!S.active(zb)) continue;
      const double *t0 = &t[(static_cast<size_t>(zb) * kV) * 35];
      residual(S, zb, t0[0], t0[2], t0 + 3, &r[static_cast<size_t>(zb) * m]);  // t[3 + k] = ln P1D of k bin k
      for (int p = 0; p < 3; ++p) {
        const double *tp = &t[(static_cast<size_t>(zb) * kV + 1 + 2 * p) * 35];
        const double *tm = &t[(static_cast<size_t>(zb) * kV + 2 + 2 * p) * 35];
        residual(S, zb, tp[0], tp[2], tp + 3, rp.data());
        residual(S, zb, tm[0], tm[2], tm + 3, rm.data());
        for (int i = 0; i < m; ++i)
          J[(static_cast<size_t>(zb) * m + i) * 3 + p] = (rp[i] - rm[i]) / (2.0 * h[p]);
      }
    }
    return MK_OK;
  }
  ~Surrogate() {
    cudaFree(dx);
    cudaFree(dy);
  }
};

}  // namespace

extern "C" int mk_tune(mk_ctx *ctx, const mk_skewer_params *params, const mk_skewer *d_sk, int64_t n_sk,
                       const int64_t *d_offsets, const float *d_delta, const float *d_eta, const mk_stat_bins *bins,
                       const mk_tune_target *target, int32_t method, mk_mlp *surrogate,
                       const mk_surrogate_norm *norm, int32_t max_passes, mk_fgpa_nodes *inout,
                       mk_tune_report *report) {
  MK_TRACE("mk_tune");
  if (!ctx) return MK_EINVAL;
  if (!bins || !target || !inout || !report || max_passes < 1)
    return mfail(ctx, MK_EINVAL, "mk_tune needs bins, a target, nodes, a report and max_passes >= 1");
  if (inout->count != bins->n_z) return mfail(ctx, MK_EINVAL, "one node per z bin is required");
  for (int i = 0; i < bins->n_z; ++i)
    if (std::fabs(inout->z[i] - (bins->z_lo + (i + 0.5) * bins->dz)) > 1e-9)
      return mfail(ctx, MK_EINVAL, "nodes must sit at the z bin centres");
  if (target->k_lo < 0 || target->k_hi > bins->n_k || target->k_hi <= target->k_lo)
    return mfail(ctx, MK_EINVAL, "bad k range");
  if (!(target->tol_mean_flux > 0) || !(target->tol_p1d > 0) || (target->use_beta && !(target->tol_beta > 0)))
    return mfail(ctx, MK_EINVAL, "tolerances must be > 0");
  for (int zb = 0; zb < bins->n_z; ++zb) {
    if (!((target->active >> zb) & 1u)) continue;
    for (int k = target->k_lo; k < target->k_hi; ++k)
      if (!(target->p1d[zb][k] > 0)) return mfail(ctx, MK_EINVAL, "P1D targets must be > 0");
  }
  if (method == MK_TUNE_SURROGATE && (!surrogate || !norm || bins->n_k != 32))
    return mfail(ctx, MK_EINVAL, "surrogate tuning needs a fitted surrogate, its norm and 32 k bins");
  if (method != MK_TUNE_PLAIN && method != MK_TUNE_SURROGATE) return mfail(ctx, MK_EINVAL, "unknown method");
  std::memset(report, 0, sizeof(*report));
  CKM(ctx, cudaSetDevice(mkhost::ctx_device(ctx)));
  TuneState S{ctx, params, d_sk, n_sk, d_offsets, d_delta, d_eta, bins, target, report, nullptr, nullptr};
  CKM(ctx, cudaEventCreate(&S.e0));
  CKM(ctx, cudaEventCreate(&S.e1));
  const auto t0 = std::chrono::steady_clock::now();
  const int m = S.m(), nz = bins->n_z;
  mk_fgpa_nodes nd = *inout;
  fill_inactive(nd, S);
  mk_stats_out st;
  std::vector<double> r, J, rp, tb;
  int rc = MK_OK;
  EffMap E;
  if ((rc = E.build(ctx, params, d_sk, n_sk, bins, target->active, nd, &report->gpu_ms))) {
    cudaEventDestroy(S.e0);
    cudaEventDestroy(S.e1);
    return rc;
  }
  if (method == MK_TUNE_PLAIN) {
    // a uniform shift of every node shifts every theta_eff by the same amount,
    // so the three shifted passes give d r / d theta_eff of every bin
    const double h[3] = {0.05, 0.05, 0.05};
    while (rc == MK_OK && report->passes < max_passes) {
      if ((rc = full_pass(S, nd, st, r))) break;
      if (converged(S, st)) {
        report->converged = 1;
        break;
      }
      if (report->passes + 4 > max_passes) break;
      J.assign(static_cast<size_t>(nz) * m * 3, 0.0);
      for (int p = 0; p < 3 && rc == MK_OK; ++p) {
        mk_fgpa_nodes q = nd;
        shift(q, p, h[p]);
        mk_stats_out sq;
        if ((rc = full_pass(S, q, sq, rp))) break;
        for (int zb = 0; zb < nz; ++zb)
          for (int i = 0; i < m; ++i)
            J[(static_cast<size_t>(zb) * m + i) * 3 + p] = (rp[static_cast<size_t>(zb) * m + i] - r[static_cast<size_t>(zb) * m + i]) / h[p];
      }
      if (rc) break;
      E.eff(nd, tb);
      for (int zb = 0; zb < nz; ++zb) {
        if (!S.active(zb)) continue;
        double d[3];
        lm_step(&J[static_cast<size_t>(zb) * m * 3], &r[static_cast<size_t>(zb) * m], m, 1e-3, d);
        (void)apply_step_eff(tb, zb, d);
      }
      E.nodes(tb, nd);
      fill_inactive(nd, S);
      report->iterations += 1;
    }
  } else {
    Surrogate sg{surrogate, norm};
    const double *zc = nd.z;
    E.eff(nd, tb);
    // fit the target on the surrogate alone
    for (int it = 0; it < 25 && rc == MK_OK; ++it) {
      if ((rc = sg.model(S, zc, tb, r, J))) break;
      double big = 0.0;
      for (int zb = 0; zb < nz; ++zb) {
        if (!S.active(zb)) continue;
        double d[3];
        lm_step(&J[static_cast<size_t>(zb) * m * 3], &r[static_cast<size_t>(zb) * m], m, 1e-2, d);
        big = std::max(big, apply_step_eff(tb, zb, d));
      }
      if (big < kSurrogateStop) break;
    }
    E.nodes(tb, nd);
    fill_inactive(nd, S);
    // refit on the surrogate shifted by `off` (true minus predicted residual at
    // theta) plus the per-bin linear term B (theta_eff - theta)
    auto refit = [&](const std::vector<double> &off, const std::vector<double> &theta,
                     const std::vector<double> &B, std::vector<double> &rs) -> int {
      int rr_rc = MK_OK;
      for (int it = 0; it < 12; ++it) {
        if (it > 0 && (rr_rc = sg.model(S, zc, tb, rs, J))) return rr_rc;
        double big = 0.0;
        for (int zb = 0; zb < nz; ++zb) {
          if (!S.active(zb)) continue;
          std::vector<double> rr(m), JJ(static_cast<size_t>(m) * 3);
          for (int i = 0; i < m; ++i) {
            const size_t row = static_cast<size_t>(zb) * m + i;
            double lin = 0.0;
            for (int p = 0; p < 3; ++p) {
              lin += B[row * 3 + p] * (tb[3 * zb + p] - theta[3 * zb + p]);
              JJ[i * 3 + p] = J[row * 3 + p] + B[row * 3 + p];
            }
            rr[i] = rs[row] + off[row] + lin;
          }
          double d[3];
          lm_step(JJ.data(), rr.data(), m, 1e-2, d);
          big = std::max(big, apply_step_eff(tb, zb, d));
        }
        if (big < kSurrogateStop) break;
      }
      return MK_OK;
    };
    std::vector<double> B(static_cast<size_t>(nz) * m * 3, 0.0), prev_off, prev_theta;
    // calibration: a pass over the first calib_skewers skewers gives the
    // surrogate's error at its fit (free of the subset-to-catalogue difference
    // when it was labelled on those skewers)
    if (rc == MK_OK && norm->calib_skewers > 0 && norm->calib_skewers < n_sk && max_passes > 1) {
      TuneState Sc = S;
      Sc.n_sk = norm->calib_skewers;
      std::vector<double> rt, rs;
      mk_stats_out sc;
      const int full_before = report->passes;
      if ((rc = full_pass(Sc, nd, sc, rt)) == MK_OK) {
        report->passes = full_before;  // counted apart: a fraction of a full pass
        report->calib_passes += 1;
        E.eff(nd, tb);
        if ((rc = sg.model(S, zc, tb, rs, J)) == MK_OK) {
          std::vector<double> off(rs.size());
          for (size_t i = 0; i < rs.size(); ++i) off[i] = rt[i] - rs[i];
          const std::vector<double> theta = tb;
          if ((rc = refit(off, theta, B, rs)) == MK_OK) {
            E.nodes(tb, nd);
            fill_inactive(nd, S);
            report->iterations += 1;
          }
        }
      }
    }
    // verify on full passes; between passes re-solve on the surrogate with the
    // last pass's discrepancy (true minus predicted residual) as an offset,
    // plus a per-bin linear term B (theta_eff - theta_eff,i) for how the
    // discrepancy changes with the parameters (Broyden updates from successive passes)
    while (rc == MK_OK && report->passes < max_passes) {
      std::vector<double> rt;
      if ((rc = full_pass(S, nd, st, rt))) break;
      if (converged(S, st)) {
        report->converged = 1;
        break;
      }
      if (report->passes >= max_passes) break;
      std::vector<double> rs, off;
      E.eff(nd, tb);
      if ((rc = sg.model(S, zc, tb, rs, J))) break;
      off.resize(rs.size());
      for (size_t i = 0; i < rs.size(); ++i) off[i] = rt[i] - rs[i];
      const std::vector<double> theta = tb;
      if (!prev_off.empty()) {
        for (int zb = 0; zb < nz; ++zb) {
          if (!S.active(zb)) continue;
          double dth[3], nn = 0.0;
          for (int p = 0; p < 3; ++p) {
            dth[p] = theta[3 * zb + p] - prev_theta[3 * zb + p];
            nn += dth[p] * dth[p];
          }
          if (nn < 1e-14) continue;
          for (int i = 0; i < m; ++i) {
            const size_t row = static_cast<size_t>(zb) * m + i;
            double pred = 0.0;
            for (int p = 0; p < 3; ++p) pred += B[row * 3 + p] * dth[p];
            const double u = (off[row] - prev_off[row]) - pred;
            for (int p = 0; p < 3; ++p) B[row * 3 + p] += u * dth[p] / nn;
          }
        }
      }
      prev_off = off;
      prev_theta = theta;
      if ((rc = refit(off, theta, B, rs))) break;
      E.nodes(tb, nd);
      fill_inactive(nd, S);
      report->iterations += 1;
    }
  }
  report->wall_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  cudaEventDestroy(S.e0);
  cudaEventDestroy(S.e1);
  if (rc) return rc;
  *inout = nd;
  return MK_OK;
}
