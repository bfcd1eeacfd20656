// Saved pre-production (Sec. 3): stored pre-FGPA skewers to and from a file,
// through a pinned staging buffer on the context's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>

#include "../../include/mockskewer.h"
#include "mk_host.h"

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

// file -> device in pieces of kStage bytes
bool fill(FILE *f, void *d, size_t bytes, void *h, cudaStream_t st) {
  char *dst = static_cast<char *>(d);
  for (size_t o = 0; o < bytes; o += kStage) {
    const size_t b = std::min(kStage, bytes - o);
    if (std::fread(h, 1, b, f) != b) return false;
    if (cudaMemcpyAsync(dst + o, h, b, cudaMemcpyHostToDevice, st) != cudaSuccess) return false;
    if (cudaStreamSynchronize(st) != cudaSuccess) return false;
  }
  return true;
}

}  // namespace

extern "C" int mk_save_skewers(mk_ctx *ctx, const char *path, const mk_skewer *d_sk, int64_t n_sk,
                               const int64_t *d_offsets, const float *d_delta, const float *d_eta) {
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
  bool ok = fill(f, d_sk, sizeof(mk_skewer) * static_cast<size_t>(ns), s.h, st);
  ok = ok && fill(f, d_offsets, sizeof(int64_t) * static_cast<size_t>(ns + 1), s.h, st);
  ok = ok && fill(f, d_delta, sizeof(float) * static_cast<size_t>(tp), s.h, st);
  ok = ok && fill(f, d_eta, sizeof(float) * static_cast<size_t>(tp), s.h, st);
  std::fclose(f);
  return ok ? MK_OK : iofail(ctx, MK_EINVAL, "mk_load_skewers: truncated file");
}
