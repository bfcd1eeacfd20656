// Definitions of SkewerUnit<N> (declared in mk_kernels.h): the launch and
// occupancy helpers of the fused skewer kernel and the statistics kernel for
// one FFT length.  Each length is explicitly instantiated in a translation
// unit of its own (mk_skewer_<N>.cu), so that the lengths compile in parallel.
#pragma once

#include "mk_kernels.h"
#include "mk_skewer.cuh"
#include "mk_tune_stats.cuh"

namespace mk {

namespace skewer_unit_detail {

// minb: register budget of the instance, that of minb 256-thread CTAs per SM;
// psz: P_s tables at several redshifts (one instance per layout, budget 3)
template <int NN, int L, int INTERP, typename F>
cudaError_t with_layout(bool big, bool psz, int minb, F &&fn) {
  if (psz) return big ? fn(k_skewer<NN, L, true, 3, INTERP, true>) : fn(k_skewer<NN, L, false, 3, INTERP, true>);
  if (minb >= 4) return big ? fn(k_skewer<NN, L, true, 4, INTERP>) : fn(k_skewer<NN, L, false, 4, INTERP>);
  if (minb == 3) return big ? fn(k_skewer<NN, L, true, 3, INTERP>) : fn(k_skewer<NN, L, false, 3, INTERP>);
  return big ? fn(k_skewer<NN, L, true, 2, INTERP>) : fn(k_skewer<NN, L, false, 2, INTERP>);
}

// Side 2^kFixLgn of the box whose padded-layout strides are compile-time
// constants in the N = 256 instances (the 1024^3 box of the batched workload);
// other sides take the strides at run time.
constexpr int kFixLgn = 10;

// Calls fn with the kernel instance for (kernel variant, box size, register budget).
template <int NN, typename F>
cudaError_t with_skewer_kernel(int variant, int lgn, int minb, F &&fn) {
  const bool big = lgn > 10;
  const bool psz = (variant & kPsNodesVariant) != 0;
  const int layout = variant & (kGauss7Variant - 1);
  if constexpr (NN == 256) {
    if (variant == MK_BOX_PADDED && lgn == kFixLgn) {
      constexpr int L = MK_BOX_PADDED, I = MK_INTERP_TRILINEAR;
      if (minb >= 4) return fn(k_skewer<NN, L, false, 4, I, false, kFixLgn>);
      if (minb == 3) return fn(k_skewer<NN, L, false, 3, I, false, kFixLgn>);
      return fn(k_skewer<NN, L, false, 2, I, false, kFixLgn>);
    }
  }
  if (variant & kGauss7Variant) return with_layout<NN, MK_BOX_HALO, MK_INTERP_GAUSS7>(big, psz, minb, fn);
  if (layout == MK_BOX_HALO) return with_layout<NN, MK_BOX_HALO, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
  if (layout == MK_BOX_TENSOR) return with_layout<NN, MK_BOX_TENSOR, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
  if (layout == MK_BOX_PADDED) return with_layout<NN, MK_BOX_PADDED, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
  if (layout == MK_BOX_INTERLEAVED) return with_layout<NN, MK_BOX_INTERLEAVED, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
  return with_layout<NN, MK_BOX_PLANAR, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
}

template <typename K>
int occupancy(K kern, int threads, size_t smem) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem) != cudaSuccess || v < 1) return 1;
  return v;
}
}  // namespace skewer_unit_detail

template <int NN>
size_t SkewerUnit<NN>::smem_bytes(int threads, int n_z, int n_k, bool stats) {
  return TeamSmem<NN>::bytes(threads, n_z, n_k, stats);
}

template <int NN>
int SkewerUnit<NN>::blocks_per_sm(int variant, int lgn, int minb, int threads, int n_z, int n_k, bool stats) {
  const size_t smem = TeamSmem<NN>::bytes(threads, n_z, n_k, stats);
  int b = 1;
  skewer_unit_detail::with_skewer_kernel<NN>(variant, lgn, minb, [&](auto kern) {
    b = skewer_unit_detail::occupancy(kern, threads, smem);
    return cudaSuccess;
  });
  return b;
}

template <int NN>
cudaError_t SkewerUnit<NN>::launch(const SkewerParams &P, int variant, int minb, int grid, int threads,
                                   cudaStream_t st) {
  const size_t smem = TeamSmem<NN>::bytes(threads, P.n_z, P.n_k, P.do_stats != 0);
  return skewer_unit_detail::with_skewer_kernel<NN>(variant, P.lgn, minb, [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, smem, st>>>(P);
    return cudaGetLastError();
  });
}

template <int NN>
int SkewerUnit<NN>::stats_blocks_per_sm(int threads, int n_z, int n_k, bool tune) {
  if (tune) return skewer_unit_detail::occupancy(k_tune_stats<NN>, threads, TuneSmem<NN>::bytes(threads, n_z, n_k));
  return skewer_unit_detail::occupancy(k_stats<NN>, threads, TeamSmem<NN>::bytes(threads, n_z, n_k, true));
}

template <int NN>
cudaError_t SkewerUnit<NN>::launch_stats(const StatParams &P, int grid, int threads, cudaStream_t st) {
  if (tune_kernel(P.pixtab, P.delta, P.eta, P.rebin)) {
    const size_t smem = TuneSmem<NN>::bytes(threads, P.n_z, P.n_k);
    cudaError_t e =
        cudaFuncSetAttribute(k_tune_stats<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    k_tune_stats<NN><<<grid, threads, smem, st>>>(P);
    return cudaGetLastError();
  }
  const size_t smem = TeamSmem<NN>::bytes(threads, P.n_z, P.n_k, true);
  cudaError_t e = cudaFuncSetAttribute(k_stats<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_stats<NN><<<grid, threads, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace mk
