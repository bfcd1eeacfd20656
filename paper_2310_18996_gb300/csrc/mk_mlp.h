// Launchers of the surrogate MLP kernels (mk_mlp.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mk {

constexpr int kMlpParams = 38179;  // 4-128-128-128-35
constexpr int kMlpIn = 4, kMlpOut = 35, kMlpHidden = 128;
constexpr int kMlpChunk = 256;     // samples of one pass of the training cluster (8 CTAs x 32)

// Bytes of the weight image: the BF16 weights in the padded layout the
// tensor-core kernels read (W0 as FP32 copies of its BF16 values) and the FP32
// biases; the kernels copy it into shared memory.
size_t mlp_image_bytes();

// Image and canonical BF16 copy (wbf, kMlpParams values, may be NULL) of the
// FP32 master parameters.
cudaError_t mlp_pack(const float *master, void *img, void *wbf, cudaStream_t st);

// y (n x 35) = MLP(x (n x 4)) with the weights of img.
cudaError_t mlp_forward(const void *img, const float *x, int64_t n, float *y, cudaStream_t st);

// One launch of the training cluster: `steps` steps of `batch` samples each
// (the last step may hold fewer), sample i of the launch at row rows[i]
// (rows NULL: row base + i).  Each step: forward and backward of its samples
// in passes of kMlpChunk, the gradient (FP32, summed over the step's samples
// in a fixed order) into grad; with train, one Adam step on master / m / v
// (Adam step count t0 + 1 + step) and the image refreshed.  loss_out[step]:
// the step's mean squared error (scaled by inv_count, or 1/(samples * 35) of
// the step when inv_count is 0).  accumulate: add the gradient to grad
// instead of overwriting it (train off only).
struct MlpRun {
  const float *x, *t;
  const int32_t *rows;
  int64_t base, n;       // samples [base, base + n) of x / t (or of rows)
  int32_t batch, steps;
  int32_t train, accumulate;
  double inv_count;
  float lr, b1, b2, eps;
  int64_t t0;
  float *master, *m, *v, *grad;
  void *img;
  double *loss_out;
};
cudaError_t mlp_cluster_run(const MlpRun &R, cudaStream_t st);

// One Adam step (Adam step count `step` >= 1) with a given gradient; refreshes
// the image.
cudaError_t mlp_adam(float *master, float *m, float *v, const float *grad, void *img, float lr, float b1,
                     float b2, float eps, int64_t step, cudaStream_t st);

}  // namespace mk
