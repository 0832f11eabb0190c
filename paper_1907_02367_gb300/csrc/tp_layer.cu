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
  cudaError_t e = cudaFuncSetAttribute(k_layer<TP_DIM, MIXED, ADJ, PERSIST, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_layer<TP_DIM, MIXED, ADJ, PERSIST, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

template <bool MIXED, bool ADJ, bool PERSIST, bool NEU>
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
  return cudaLaunchKernelEx(&cfg, k_layer<TP_DIM, MIXED, ADJ, PERSIST, NEU>, a, t0);
}

template <bool MIXED, bool ADJ, bool PERSIST, bool NEU>
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
  return cudaOccupancyMaxActiveClusters(n, k_layer<TP_DIM, MIXED, ADJ, PERSIST, NEU>, &cfg);
}

}  // namespace

// largest static shared memory of the instantiations (bytes)
cudaError_t TP_CAT(layer_static_smem_d, TP_DIM)(size_t* bytes) {
  size_t m = 0;
  cudaFuncAttributes fa;
  cudaError_t e;
  const void* k[] = {
      (const void*)k_layer<TP_DIM, false, false, false, false>, (const void*)k_layer<TP_DIM, true, false, false, false>,
      (const void*)k_layer<TP_DIM, false, true, false, false>, (const void*)k_layer<TP_DIM, false, false, true, false>,
      (const void*)k_layer<TP_DIM, true, false, true, false>, (const void*)k_layer<TP_DIM, false, false, false, true>,
      (const void*)k_layer<TP_DIM, true, false, false, true>, (const void*)k_layer<TP_DIM, false, true, false, true>,
      (const void*)k_layer<TP_DIM, false, false, true, true>, (const void*)k_layer<TP_DIM, true, false, true, true>};
  for (const void* f : k) {
    if ((e = cudaFuncGetAttributes(&fa, f)) != cudaSuccess) return e;
    m = std::max(m, fa.sharedSizeBytes);
  }
  *bytes = m;
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
  const bool neu = (mode & 4) != 0;
  mode &= 3;
  if (persistent) {
    if (mode == 1)
      return neu ? launch<true, false, true, true>(a, n_cluster, cs, t0, smem, st)
                 : launch<true, false, true, false>(a, n_cluster, cs, t0, smem, st);
    return neu ? launch<false, false, true, true>(a, n_cluster, cs, t0, smem, st)
               : launch<false, false, true, false>(a, n_cluster, cs, t0, smem, st);
  }
  if (mode == 2)
    return neu ? launch<false, true, false, true>(a, n_cluster, cs, t0, smem, st)
               : launch<false, true, false, false>(a, n_cluster, cs, t0, smem, st);
  if (mode == 1)
    return neu ? launch<true, false, false, true>(a, n_cluster, cs, t0, smem, st)
               : launch<true, false, false, false>(a, n_cluster, cs, t0, smem, st);
  return neu ? launch<false, false, false, true>(a, n_cluster, cs, t0, smem, st)
             : launch<false, false, false, false>(a, n_cluster, cs, t0, smem, st);
}

cudaError_t TP_CAT(max_clusters_d, TP_DIM)(int cs, size_t smem, int mode, int* n) {
  const bool neu = (mode & 4) != 0;
  if ((mode & 3) == 1) return neu ? occupancy<true, false, true, true>(cs, smem, n) : occupancy<true, false, true, false>(cs, smem, n);
  return neu ? occupancy<false, false, true, true>(cs, smem, n) : occupancy<false, false, true, false>(cs, smem, n);
}

}  // namespace tp
