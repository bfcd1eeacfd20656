// Launchers of the surrogate MLP kernels (mk_mlp.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mk {

constexpr int kMlpParams = 38179;  // 4-128-128-128-35
constexpr int kMlpIn = 4, kMlpOut = 35, kMlpHidden = 128;
constexpr int kLossParts = 64;

cudaError_t mlp_to_bf16(const float *master, void *wbf, cudaStream_t st);
// y (n x 35); with acts (3 x 2 x n x 128 floats) the hidden z and h are kept
cudaError_t mlp_forward(const void *wbf, const float *master, const float *x, const int32_t *rows, int64_t n,
                        float *y, float *acts, cudaStream_t st);
cudaError_t mlp_gradient(const void *wbf, const float *master, const float *x, const float *t,
                         const int32_t *rows, int64_t n, double inv_count, float *y, float *dy, float *acts,
                         float *dzs, float *grad, double *loss_part, cudaStream_t st);
cudaError_t mlp_adam(float *master, void *wbf, const float *grad, float *m, float *v, float lr, float b1, float b2,
                     float eps, int64_t step, cudaStream_t st);

}  // namespace mk
