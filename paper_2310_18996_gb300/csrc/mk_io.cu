// Saved pre-production (Sec. 3): stored pre-FGPA skewers to and from a file,
// through a pinned staging buffer on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/mockskewer.h"
#include "mk_host.h"
#include "mk_trace.h"

namespace {

constexpr char kMagic[8] = {'M', 'K', 'S', 'K', 'E', 'W', '0', '1'};
constexpr size_t kStage = size_t(64) << 20;  // bytes per staged copy

int iofail(mk_ctx *ctx, int code, const char *msg) { return mkhost::ctx_fail(ctx, code, msg); }

struct Staging {
  void *h = nullptr;
  ~Staging() {
    if (h) cudaFreeHost(h);
  }
};

// device -> file in pieces of kStage bytes
bool dump(FILE *f, const void *d, size_t bytes, void *h, cudaStream_t st) {
  const char *src = static_cast<const char *>(d);
  for (size_t o = 0; o < bytes; o += kStage) {
    const size_t b = std::min(kStage, bytes - o);
    if (cudaMemcpyAsync(h, src + o, b, cudaMemcpyDeviceToHost, st) != cudaSuccess) return false;
    if (cudaStreamSynchronize(st) != cudaSuccess) return false;
    if (std::fwrite(h, 1, b, f) != b) return false;
  }
  return true;
}

// file -> device in pieces of whole elements, at most kStage bytes each;
// check(first element, pointer, count) sees each piece in host memory before
// it is copied and may refuse it
template <class T, class Check>
bool fill(FILE *f, T *d, int64_t count, void *h, cudaStream_t st, Check check) {
  const int64_t per = static_cast<int64_t>(kStage / sizeof(T));
  for (int64_t o = 0; o < count; o += per) {
    const int64_t c = std::min(per, count - o);
    const size_t b = sizeof(T) * static_cast<size_t>(c);
    if (std::fread(h, 1, b, f) != b) return false;
    if (!check(o, static_cast<const T *>(h), c)) return false;
    if (cudaMemcpyAsync(d + o, h, b, cudaMemcpyHostToDevice, st) != cudaSuccess) return false;
    if (cudaStreamSynchronize(st) != cudaSuccess) return false;
  }
  return true;
}

}  // namespace

extern "C" int mk_save_skewers(mk_ctx *ctx, const char *path, const mk_skewer *d_sk, int64_t n_sk,
                               const int64_t *d_offsets, const float *d_delta, const float *d_eta) {
  MK_TRACE("mk_save_skewers");
  if (!ctx) return MK_EINVAL;
  if (!path || n_sk < 0 || !d_offsets || (n_sk > 0 && (!d_sk || !d_delta || !d_eta)))
    return iofail(ctx, MK_EINVAL, "mk_save_skewers: NULL argument");
  if (cudaSetDevice(mkhost::ctx_device(ctx)) != cudaSuccess) return iofail(ctx, MK_ECUDA, "cudaSetDevice");
  const cudaStream_t st = mkhost::ctx_stream(ctx);
  int64_t total = 0;
  if (cudaMemcpyAsync(&total, d_offsets + n_sk, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return iofail(ctx, MK_ECUDA, "mk_save_skewers: reading the pixel total");
  if (total < 0) return iofail(ctx, MK_EINVAL, "mk_save_skewers: negative pixel total");
  Staging s;
  if (cudaMallocHost(&s.h, kStage) != cudaSuccess) return iofail(ctx, MK_ENOMEM, "mk_save_skewers: staging buffer");
  FILE *f = std::fopen(path, "wb");
  if (!f) return iofail(ctx, MK_EINVAL, "mk_save_skewers: cannot open the file for writing");
  bool ok = std::fwrite(kMagic, 1, 8, f) == 8 && std::fwrite(&n_sk, 8, 1, f) == 1 && std::fwrite(&total, 8, 1, f) == 1;
  ok = ok && dump(f, d_sk, sizeof(mk_skewer) * static_cast<size_t>(n_sk), s.h, st);
  ok = ok && dump(f, d_offsets, sizeof(int64_t) * static_cast<size_t>(n_sk + 1), s.h, st);
  ok = ok && dump(f, d_delta, sizeof(float) * static_cast<size_t>(total), s.h, st);
  ok = ok && dump(f, d_eta, sizeof(float) * static_cast<size_t>(total), s.h, st);
  ok = (std::fclose(f) == 0) && ok;
  return ok ? MK_OK : iofail(ctx, MK_EINVAL, "mk_save_skewers: write failed");
}

extern "C" int mk_load_skewers(mk_ctx *ctx, const char *path, mk_skewer *d_sk, int64_t cap_sk, int64_t *d_offsets,
                               float *d_delta, float *d_eta, int64_t cap_px, int64_t *n_sk, int64_t *total_px) {
  MK_TRACE("mk_load_skewers");
  if (!ctx) return MK_EINVAL;
  if (!path || !n_sk || !total_px) return iofail(ctx, MK_EINVAL, "mk_load_skewers: NULL argument");
  FILE *f = std::fopen(path, "rb");
  if (!f) return iofail(ctx, MK_EINVAL, "mk_load_skewers: cannot open the file");
  char magic[8];
  int64_t ns = -1, tp = -1;
  const bool head = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
                    std::fread(&ns, 8, 1, f) == 1 && std::fread(&tp, 8, 1, f) == 1 && ns >= 0 && tp >= 0;
  if (!head) {
    std::fclose(f);
    return iofail(ctx, MK_EINVAL, "mk_load_skewers: not a skewer file");
  }
  *n_sk = ns;
  *total_px = tp;
  if (!d_sk || !d_offsets || !d_delta || !d_eta) {
    std::fclose(f);
    return MK_OK;  // size query
  }
  if (ns > cap_sk || tp > cap_px) {
    std::fclose(f);
    return iofail(ctx, MK_ERANGE, "mk_load_skewers: buffers smaller than the file (sizes returned)");
  }
  if (cudaSetDevice(mkhost::ctx_device(ctx)) != cudaSuccess) {
    std::fclose(f);
    return iofail(ctx, MK_ECUDA, "cudaSetDevice");
  }
  const cudaStream_t st = mkhost::ctx_stream(ctx);
  Staging s;
  if (cudaMallocHost(&s.h, kStage) != cudaSuccess) {
    std::fclose(f);
    return iofail(ctx, MK_ENOMEM, "mk_load_skewers: staging buffer");
  }
  // The records and offsets drive every later index into the pixel arrays,
  // so they must describe consecutive pixel ranges that tile [0, total):
  // record i starts where record i - 1 ends, and offsets[i] is its start.
  std::vector<int64_t> start(static_cast<size_t>(ns) + 1);
  int64_t run = 0;
  const auto records = [&](int64_t i0, const mk_skewer *r, int64_t c) {
    for (int64_t k = 0; k < c; ++k) {
      if (r[k].offset != run || r[k].n < 0 || r[k].j_lo < 0 || r[k].n > tp - run) return false;
      start[static_cast<size_t>(i0 + k)] = run;
      run += r[k].n;
    }
    return true;
  };
  const auto offsets = [&](int64_t i0, const int64_t *v, int64_t c) {
    for (int64_t k = 0; k < c; ++k)
      if (v[k] != start[static_cast<size_t>(i0 + k)]) return false;
    return true;
  };
  const auto any = [](int64_t, const float *, int64_t) { return true; };
  const bool rec_ok = fill(f, d_sk, ns, s.h, st, records) && run == tp;
  start[static_cast<size_t>(ns)] = tp;
  const bool off_ok = rec_ok && fill(f, d_offsets, ns + 1, s.h, st, offsets);
  const bool px_ok = off_ok && fill(f, d_delta, tp, s.h, st, any) && fill(f, d_eta, tp, s.h, st, any);
  std::fclose(f);
  if (!rec_ok || !off_ok)
    return iofail(ctx, MK_EINVAL, "mk_load_skewers: truncated file, or records and offsets that do not tile the pixels");
  return px_ok ? MK_OK : iofail(ctx, MK_EINVAL, "mk_load_skewers: truncated file");
}
