// Internal accessors of the context for translation units other than mk_api.cu.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/mockskewer.h"

namespace mkhost {
cudaStream_t ctx_stream(mk_ctx *c);
int ctx_device(mk_ctx *c);
int ctx_fail(mk_ctx *c, int code, const char *msg);
int ctx_sms(mk_ctx *c);
// FP64 cosmology of the context (Sec. 2): z(D_C), G(z), D_C(z)
double ctx_z_of(mk_ctx *c, double r);
double ctx_growth(mk_ctx *c, double z);
double ctx_distance(mk_ctx *c, double z);
// Pixel redshifts z_J of the tables for pixel size dr and, per J, the number
// of pixels of the n_sk skewers d_sk at J (synchronous; GPU time added to *ms).
int ctx_pixel_histogram(mk_ctx *c, double dr, const mk_skewer *d_sk, int64_t n_sk, std::vector<double> &z,
                        std::vector<int64_t> &count, double *ms);
}  // namespace mkhost
