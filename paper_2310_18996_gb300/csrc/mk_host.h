// Internal accessors of the context for translation units other than mk_api.cu.
#pragma once

#include <cuda_runtime.h>

#include "../../include/mockskewer.h"

namespace mkhost {
cudaStream_t ctx_stream(mk_ctx *c);
int ctx_device(mk_ctx *c);
int ctx_fail(mk_ctx *c, int code, const char *msg);
}  // namespace mkhost
