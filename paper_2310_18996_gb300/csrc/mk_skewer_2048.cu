// Instances of the fused skewer kernel and the statistics kernel for one
// FFT length, with their launch and occupancy helpers.
#include "mk_kernels.h"
#include "mk_skewer.cuh"

namespace mk {

namespace {
constexpr int NN = 2048;

// minb: register budget of the instance, that of minb 256-thread CTAs per SM;
// psz: P_s tables at several redshifts (one instance per layout, budget 3)
template <int L, int INTERP, typename F>
cudaError_t with_layout(bool big, bool psz, int minb, F &&fn) {
  if (psz) return big ? fn(k_skewer<NN, L, true, 3, INTERP, true>) : fn(k_skewer<NN, L, false, 3, INTERP, true>);
  if (minb >= 4) return big ? fn(k_skewer<NN, L, true, 4, INTERP>) : fn(k_skewer<NN, L, false, 4, INTERP>);
  if (minb == 3) return big ? fn(k_skewer<NN, L, true, 3, INTERP>) : fn(k_skewer<NN, L, false, 3, INTERP>);
  return big ? fn(k_skewer<NN, L, true, 2, INTERP>) : fn(k_skewer<NN, L, false, 2, INTERP>);
}

// Calls fn with the kernel instance for (kernel variant, box size, register budget).
template <typename F>
cudaError_t with_skewer_kernel(int variant, bool big, int minb, F &&fn) {
  const bool psz = (variant & kPsNodesVariant) != 0;
  const int layout = variant & (kGauss7Variant - 1);
  if (variant & kGauss7Variant) return with_layout<MK_BOX_HALO, MK_INTERP_GAUSS7>(big, psz, minb, fn);
  if (layout == MK_BOX_HALO) return with_layout<MK_BOX_HALO, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
  if (layout == MK_BOX_TENSOR) return with_layout<MK_BOX_TENSOR, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
  if (layout == MK_BOX_PADDED) return with_layout<MK_BOX_PADDED, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
  if (layout == MK_BOX_INTERLEAVED) return with_layout<MK_BOX_INTERLEAVED, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
  return with_layout<MK_BOX_PLANAR, MK_INTERP_TRILINEAR>(big, psz, minb, fn);
}

template <typename K>
int occupancy(K kern, int threads, size_t smem) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  int v = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem) != cudaSuccess || v < 1) return 1;
  return v;
}
}  // namespace

size_t skewer_smem_bytes_2048(int threads, int n_z, int n_k, bool stats) {
  return TeamSmem<NN>::bytes(threads, n_z, n_k, stats);
}

int skewer_blocks_per_sm_2048(int variant, int lgn, int minb, int threads, int n_z, int n_k, bool stats) {
  const size_t smem = TeamSmem<NN>::bytes(threads, n_z, n_k, stats);
  int b = 1;
  with_skewer_kernel(variant, lgn > 10, minb, [&](auto kern) {
    b = occupancy(kern, threads, smem);
    return cudaSuccess;
  });
  return b;
}

cudaError_t launch_skewer_2048(const SkewerParams &P, int variant, int minb, int grid, int threads, cudaStream_t st) {
  const size_t smem = TeamSmem<NN>::bytes(threads, P.n_z, P.n_k, P.do_stats != 0);
  return with_skewer_kernel(variant, P.lgn > 10, minb, [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, smem, st>>>(P);
    return cudaGetLastError();
  });
}

int stats_blocks_per_sm_2048(int threads, int n_z, int n_k) {
  return occupancy(k_stats<NN>, threads, TeamSmem<NN>::bytes(threads, n_z, n_k, true));
}

cudaError_t launch_stats_2048(const StatParams &P, int grid, int threads, cudaStream_t st) {
  const size_t smem = TeamSmem<NN>::bytes(threads, P.n_z, P.n_k, true);
  cudaError_t e = cudaFuncSetAttribute(k_stats<NN>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  k_stats<NN><<<grid, threads, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace mk
