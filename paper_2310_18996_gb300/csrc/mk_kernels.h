// Host-side launchers of the kernels in mk_kernels.cu.
#pragma once

#include <cuda_runtime.h>

#include "mk_params.h"

namespace mk {

constexpr int kGauss7Variant = 16;   // kernel variant bit of MK_INTERP_GAUSS7
constexpr int kPsNodesVariant = 32;  // kernel variant bit of P_s tables at several redshifts

cudaError_t launch_geometry(const mk_qso *q, int64_t nq, const GeomParams &P, mk_skewer *sk, int64_t *cnt_px,
                            int64_t *cnt_seg, int *err, cudaStream_t st);
size_t scan_workspace_bytes(int64_t n);
// exclusive prefix sums (n + 1 outputs) of a (and b if not NULL); also
// stores the pixel offset into sk[i].offset when sk is not NULL
cudaError_t launch_scan(const int64_t *a, const int64_t *b, int64_t n, int64_t *out_a, int64_t *out_b,
                        mk_skewer *sk, void *ws, cudaStream_t st);
cudaError_t launch_pixtab(const double *zpix, const float *gpix, int32_t j_max, const NodeParams &nd,
                          float4 *pixtab, cudaStream_t st);
cudaError_t launch_zbin(const double *zpix, const double *cumz, int32_t j_max, double z_lo, double dz, int n_z,
                        int n_seg, int16_t *zbin, int16_t *segzbin, cudaStream_t st);
cudaError_t launch_pack(const float *d, const float *e, int64_t n, float *out, int sms, cudaStream_t st);
cudaError_t launch_pack_tensor(const float *d, const float *e6, int lgn, float *out, int sms, cudaStream_t st);
cudaError_t launch_pack_halo(const float *d, const float *e, int lgn, float *out, int sms, cudaStream_t st);
cudaError_t launch_pack_padded(const float *d, const float *e, int lgn, float *out, int sms, cudaStream_t st);
cudaError_t launch_jcount(const mk_skewer *sk, int64_t n_sk, int32_t j_max, int32_t *diff, int sms, cudaStream_t st);
cudaError_t launch_zwin(const double *cumz, int32_t j_max, int n, float *zwin, cudaStream_t st);
cudaError_t launch_pick(const int64_t *off, int64_t n, int k, int64_t *out, cudaStream_t st);
cudaError_t launch_bin_end(const int16_t *zbin, int32_t j_max, int n_z, int32_t *bin_end, cudaStream_t st);
cudaError_t launch_out_counts(const mk_skewer *sk, int64_t n, int rebin, int64_t *cnt, cudaStream_t st);
cudaError_t launch_seg_counts(const int64_t *off, int64_t n, int n_fft, int64_t *cnt, cudaStream_t st);
int skewer_blocks_per_sm(int n_fft, int variant, int lgn, int minb, int threads, int n_z, int n_k, bool stats);
// The tuning pass (FGPA table set, rebin 1, 16-byte aligned fields) runs the
// staged kernel k_tune_stats; every other statistics pass runs k_stats.
inline bool tune_kernel(const void *pixtab, const float *delta, const float *eta, int rebin) {
  return pixtab && delta && eta && rebin == 1 &&
         ((reinterpret_cast<uintptr_t>(delta) | reinterpret_cast<uintptr_t>(eta)) & 15) == 0;
}
int stats_blocks_per_sm(int n_fft, int threads, int n_z, int n_k, bool tune);
size_t skewer_smem_bytes(int n_fft, int threads, int n_z, int n_k, bool stats);
// variant: box layout, plus kGauss7Variant for the Gaussian-kernel interpolation,
// plus kPsNodesVariant for z-dependent P_s (built for register budget 3 only);
// minb: register budget of the instance, that of minb 256-thread CTAs per SM
// (2, 3 or 4)
cudaError_t launch_skewer(const SkewerParams &P, int n_fft, int variant, int minb, int grid, int threads,
                          cudaStream_t st);
// The fused skewer kernel and the statistics kernel for FFT length N: launch
// and occupancy helpers, defined in mk_skewer_unit.cuh and instantiated once
// per length (256, 512, 1024, 2048) in mk_skewer_<N>.cu.
template <int N>
struct SkewerUnit {
  static size_t smem_bytes(int threads, int n_z, int n_k, bool stats);
  static int blocks_per_sm(int variant, int lgn, int minb, int threads, int n_z, int n_k, bool stats);
  static cudaError_t launch(const SkewerParams &P, int variant, int minb, int grid, int threads, cudaStream_t st);
  static int stats_blocks_per_sm(int threads, int n_z, int n_k, bool tune);
  static cudaError_t launch_stats(const StatParams &P, int grid, int threads, cudaStream_t st);
};
extern template struct SkewerUnit<256>;
extern template struct SkewerUnit<512>;
extern template struct SkewerUnit<1024>;
extern template struct SkewerUnit<2048>;
cudaError_t launch_flux(const FluxParams &P, int sms, cudaStream_t st);
cudaError_t launch_stats(const StatParams &P, int n_fft, int grid, int threads, cudaStream_t st);
// One pass of the box synthesis: batched line FFTs of an n^3 complex box
// ([z][y][x], x fastest) along one axis, with the pass's extra step (noise,
// mode filter or output layout).
struct BoxPassParams {
  float2 *work;          // n^3, transformed in place
  float2 *spec;          // n^3 delta modes (kept for further filter pairs) or NULL
  const float2 *tw;      // e^{-2 pi i k / 2n}, k < 2n
  const float *pk;       // P(k) at k = i dk, i < n_pk
  int32_t n_pk;
  float inv_dk;
  float kf;              // 2 pi / (n cell)
  float amp;             // 1 / (cell^{3/2} n^3): sqrt(P / cell^3) and the inverse 1/n^3
  uint32_t key0, key1;   // Philox key of the white noise
  int32_t pair;          // filter pair 0..3: (1, eta_xx), (eta_yy, eta_zz), (eta_xy, eta_xz), (eta_yz, 0)
  int32_t axis;          // 0 x, 1 y, 2 z
  int32_t lgn;
  float *out;            // output layout (last pass) or NULL
  int32_t out_side, out_margin, out_stride, out_slot;
};

// Box synthesis passes (mk_box.cu), modes in the order they run:
enum BoxPass : int {
  kBoxNoiseX = 0,  // white noise, forward FFT along x
  kBoxFwd = 1,     // forward FFT along P.axis
  kBoxShapeZ = 2,  // forward FFT along z, filter (delta modes to spec if set), inverse along z
  kBoxSpecZ = 3,   // delta modes from spec, filter, inverse FFT along z
  kBoxInv = 4,     // inverse FFT along P.axis
  kBoxInvXOut = 5  // inverse FFT along x, lines written into the output layout (or in place)
};
cudaError_t launch_box_pass(const BoxPassParams &P, int mode, int sms, cudaStream_t st);
cudaError_t launch_finalize(const double *partials, int nparts, int n_z, int n_k, int n_fft, mk_stats_out *out,
                            cudaStream_t st);

}  // namespace mk
