// Instantiations and launchers of the tent kernel for one space dimension.
// Compiled once per dimension with -DTP_DIM=1, 2 or 3 (the translation units
// build in parallel).
#include <algorithm>

#include "tp_kernel.cuh"

#ifndef TP_DIM
#error "compile with -DTP_DIM=1, 2 or 3"
#endif

#define TP_CAT2(a, b) a##b
#define TP_CAT(a, b) TP_CAT2(a, b)

namespace tp {

namespace {

template <bool MIXED, bool ADJ, bool PERSIST>
cudaError_t set_attr(size_t smem) {
  return cudaFuncSetAttribute(k_layer<TP_DIM, MIXED, ADJ, PERSIST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

template <bool MIXED, bool ADJ, bool PERSIST>
cudaError_t launch(const KArgs& a, int n_cluster, int cs, int t0, size_t smem, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_cluster * cs));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_layer<TP_DIM, MIXED, ADJ, PERSIST>, a, t0);
}

template <bool MIXED, bool ADJ, bool PERSIST>
cudaError_t occupancy(int cs, size_t smem, int* n) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)cs);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaOccupancyMaxActiveClusters(n, k_layer<TP_DIM, MIXED, ADJ, PERSIST>, &cfg);
}

}  // namespace

// largest static shared memory of the instantiations (bytes)
cudaError_t TP_CAT(layer_static_smem_d, TP_DIM)(size_t* bytes) {
  size_t m = 0;
  cudaFuncAttributes fa;
  cudaError_t e;
  if ((e = cudaFuncGetAttributes(&fa, k_layer<TP_DIM, false, false, false>)) != cudaSuccess) return e;
  m = std::max(m, fa.sharedSizeBytes);
  if ((e = cudaFuncGetAttributes(&fa, k_layer<TP_DIM, true, false, false>)) != cudaSuccess) return e;
  m = std::max(m, fa.sharedSizeBytes);
  if ((e = cudaFuncGetAttributes(&fa, k_layer<TP_DIM, false, true, false>)) != cudaSuccess) return e;
  m = std::max(m, fa.sharedSizeBytes);
  if ((e = cudaFuncGetAttributes(&fa, k_layer<TP_DIM, false, false, true>)) != cudaSuccess) return e;
  m = std::max(m, fa.sharedSizeBytes);
  if ((e = cudaFuncGetAttributes(&fa, k_layer<TP_DIM, true, false, true>)) != cudaSuccess) return e;
  *bytes = std::max(m, fa.sharedSizeBytes);
  return cudaSuccess;
}

cudaError_t TP_CAT(layer_attrs_d, TP_DIM)(size_t smem) {
  cudaError_t e;
  if ((e = set_attr<false, false, false>(smem)) != cudaSuccess) return e;
  if ((e = set_attr<true, false, false>(smem)) != cudaSuccess) return e;
  if ((e = set_attr<false, true, false>(smem)) != cudaSuccess) return e;
  if ((e = set_attr<false, false, true>(smem)) != cudaSuccess) return e;
  return set_attr<true, false, true>(smem);
}

cudaError_t TP_CAT(launch_layer_d, TP_DIM)(const KArgs& a, int n_cluster, int cs, int t0, size_t smem,
                                           cudaStream_t st, int mode, bool persistent) {
  if (persistent) {
    if (mode == 1) return launch<true, false, true>(a, n_cluster, cs, t0, smem, st);
    return launch<false, false, true>(a, n_cluster, cs, t0, smem, st);
  }
  if (mode == 2) return launch<false, true, false>(a, n_cluster, cs, t0, smem, st);
  if (mode == 1) return launch<true, false, false>(a, n_cluster, cs, t0, smem, st);
  return launch<false, false, false>(a, n_cluster, cs, t0, smem, st);
}

cudaError_t TP_CAT(max_clusters_d, TP_DIM)(int cs, size_t smem, int mode, int* n) {
  if (mode == 1) return occupancy<true, false, true>(cs, smem, n);
  return occupancy<false, false, true>(cs, smem, n);
}

}  // namespace tp
