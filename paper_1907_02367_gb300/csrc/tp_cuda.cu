// libtp device side: context, shared-memory plan, launches of the tent
// kernel (per level in a CUDA graph, or one persistent dataflow launch), the
// energy reduction.
//
// One cluster of CTAs solves one tent (Section 4.1, eq. 4.1 with the Section 5
// recovery terms).  For a tent at vertex v with patch star(v), basis U_h = sum_j x_j b_j
// of U^p (Section 3, Remark 3.1 scaling) and front points q of every patch
// element K (one spatial rule mapped onto the faces, Fig. 2):
//
//   top face (t = tau_top(x), n_t dS = dx, n_x dS = -g dx):
//     c^-2 v w + s.t - v (t.g) - (s.g) w = (s - v g).(t - w g) + (c^-2 - |g|^2) v w
//   so the top contribution is a Gram matrix  A += Z^T Z  of the rows
//     z_0 = sqrt(w_q) sqrt(c^-2 - |g|^2) v_j,  z_m = sqrt(w_q) (s_mj - v_j g_m)
//   (c|g| < 1 on a space-like face, Section 2.2), plus the recovery row
//     sqrt(w_q) U_j at the bottom point;
//   bottom data (RHS):  b_i += w_q [ (c^-2 v_b - s_b.g_b) v_i + (s_b - v_b g_b).s_i + U_b U_i ];
//   Dirichlet vertical faces (eq. 4.1):
//     A_ij += w (s_j.n + alpha v_j) v_i,  b_i += w g_D (alpha v_i - s_i.n).
// Then the local solve (a binary32 inverse of the equilibrated matrix and
// refinement in the path's precision, a direct binary64 LU as fallback), and
// (U, v, sigma) at the top points overwrite the front (Section 4.1: only the
// latest values are stored).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <type_traits>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tp_internal.h"

#define TP_CUDA_OK(call)                                                              \
  do {                                                                                \
    cudaError_t e__ = (call);                                                         \
    if (e__ != cudaSuccess) {                                                         \
      tp::set_error(std::string("tp: CUDA error ") + cudaGetErrorString(e__) + " at " + \
                    #call);                                                           \
      return TP_ERR_CUDA;                                                             \
    }                                                                                 \
  } while (0)

#include "tp_kernel.cuh"

namespace {
using namespace tp;

// energy flux through the front, per (rhs, element) partial sums
template <int DIM>
__global__ void k_energy_partial(const KArgs a, double* partial, int nblk_per_rhs) {
  constexpr int NV = DIM + 1, C = DIM + 2;
  __shared__ double red[kThreads];
  const int r = blockIdx.y;
  double acc = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < a.ne;
       k += (int64_t)gridDim.x * blockDim.x) {
    double e[DIM][DIM], dt[DIM], X0[DIM];
    const int v0 = a.elems[k * NV];
    for (int d = 0; d < DIM; ++d) X0[d] = a.X[(int64_t)v0 * DIM + d];
    const double t0 = a.tau[v0];
    for (int i = 0; i < DIM; ++i) {
      const int vi = a.elems[k * NV + i + 1];
      for (int d = 0; d < DIM; ++d) e[i][d] = a.X[(int64_t)vi * DIM + d] - X0[d];
      dt[i] = a.tau[vi] - t0;
    }
    double g[DIM];
    const double det = lin_grad<DIM>(e, dt, g);
    const double ic2 = 1.0 / (a.cK[k] * a.cK[k]);
    const double ad = fabs(det);
    const double* f = a.front + ((int64_t)r * a.ne + k) * a.Q * C;
    for (int q = 0; q < a.Q; ++q) {
      const double vv = f[q * C + 1];
      double s2 = 0.0, sg = 0.0;
      for (int d = 0; d < DIM; ++d) {
        s2 = fma(f[q * C + 2 + d], f[q * C + 2 + d], s2);
        sg = fma(f[q * C + 2 + d], g[d], sg);
      }
      acc = fma(0.5 * __ldg(a.wref + q) * ad, ic2 * vv * vv + s2 - 2.0 * vv * sg, acc);
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[(int64_t)r * nblk_per_rhs + blockIdx.x] = red[0];
}

// E_r into out[r * stride]; with stride 2 the accumulated energy loss D_r
// (zero when diss is null) into out[2 r + 1]
__global__ void k_energy_final(const double* partial, int nblk, int nrhs, double* out, int stride = 1,
                               const double* diss = nullptr) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrhs) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(int64_t)r * nblk + b];
  out[(int64_t)r * stride] = s;
  if (stride == 2) out[2 * (int64_t)r + 1] = diss != nullptr ? diss[r] : 0.0;
}

template <typename T>
int upload(T** dptr, const std::vector<T>& h) {
  *dptr = nullptr;
  if (h.empty()) return TP_OK;
  TP_CUDA_OK(cudaMalloc(dptr, h.size() * sizeof(T)));
  TP_CUDA_OK(cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return TP_OK;
}

}  // namespace

// ===========================================================================
// context
// ===========================================================================
struct tp_ctx {
  int dim = 0, p = 0, nb = 0, nmono = 0, Q = 0, C = 0, nrhs = 1;
  double alpha = 0.5;
  int64_t nv = 0, ne = 0, ntents = 0, n_bnd = 0;
  int32_t n_levels = 0;
  std::vector<int64_t> level_ptr;
  tp::Topology topo;
  tp::SimplexRule rule;
  std::vector<double> bnd_xt, bnd_nrm;
  bool neumann = false;     // the mesh has Neumann facets
  std::vector<int8_t> bnd_kind;
  KArgs args{};
  KArgs args_adj{};        // same tables; front/tau point at the adjoint state
  double T_final = 0.0;
  double* d_adj = nullptr;
  double* d_tau_adj = nullptr;
  // right-hand sides in groups of nrhs_g (the shared-memory plan holds one
  // group; each sweep runs group after group from the same front times)
  int rhs_groups = 1, nrhs_g = 1;
  double* d_tau_save = nullptr;
  cudaGraphExec_t adj_graph = nullptr;
  size_t smem_bytes = 0;
  int energy_blocks = 0;
  std::vector<void*> allocs;
  double* d_front = nullptr;
  double* d_tau = nullptr;
  double* d_gD = nullptr;
  double* d_partial = nullptr;
  double* d_diss = nullptr;   // per right-hand side: energy lost in the tents since tp_set_state (tracked contexts)
  // wave-speed gradient (contexts created with ckpt_stride > 0): the initial
  // front of the last tp_set_state, a work front and its times, forward
  // checkpoints every ckpt_stride levels, the fronts before each level of one
  // segment, and the forward solutions of one segment's tents
  int ckpt_stride = 0;
  double* d_front0 = nullptr;
  double* d_work = nullptr;
  double* d_tau_work = nullptr;
  double* d_ckpt = nullptr;
  double* d_ckpt_tau = nullptr;
  double* d_snap = nullptr;
  double* d_xsave = nullptr;
  long long xs_stride = 0, xsave_tents = 0;
  int* d_status = nullptr;
  long long* d_info = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaStream_t last_stream = nullptr;
  int n_sm = 152, max_cs = 1;
  // right-hand sides split over the CTAs of a tent's cluster (1: not split)
  int rsplit_cs = 1;
  bool tc_used = false;   // tensor-core moments and outflow in the forward sweep
  bool mixed = false;
  // persistent dataflow sweep
  bool persistent = true;
  int persist_clusters = 0;
  int persist_cs = 1;
  int tune_key[5] = {0, 0, 0, 0, 0};   // (dim, p, nrhs, mixed, patch bucket) of the autotuner cache
  int* d_queue = nullptr;
  int* d_done = nullptr;
  int* d_tent_vert = nullptr;
  // dependency lists of the dataflow sweep kept on the host (tp_inject_wait)
  std::vector<int32_t> dep_ptr_h, dep_need_h;
  // vertex stars in the record order (grouped by material) and the tents'
  // vertices and top times (point outputs are assigned to tents on the host)
  std::vector<int> star_sorted;
  std::vector<int32_t> tent_vert_h;
  std::vector<double> tent_ttop_h;
  // point outputs (tp_set_probes)
  int n_probe = 0, n_probe_t = 0;
  double* d_probe_out = nullptr;
  std::vector<void*> probe_allocs;
  int* d_dep_need = nullptr;
  unsigned long long* d_stats = nullptr;   // solve statistics (kMaxRefine + 2 counters)
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  int device = 0;
};

namespace {

template <typename T>
int ctx_upload(tp_ctx* ctx, T** d, const std::vector<T>& h) {
  int rc = upload(d, h);
  if (rc == TP_OK && *d) ctx->allocs.push_back((void*)*d);
  return rc;
}

constexpr size_t kTwoPerSmSmem = 95 * 1024;  // plan that leaves room for two CTAs per SM

// cap of the shared-memory plan: the device's per-block limit less the
// kernel's static shared memory; the attribute is set to it, so contexts of
// any size can share the kernel
int max_dyn_smem(int dim, size_t* cap) {
  int dev = 0, optin = 0;
  size_t stat = 0;
  TP_CUDA_OK(cudaGetDevice(&dev));
  TP_CUDA_OK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  TP_CUDA_OK(dim == 1 ? tp::layer_static_smem_d1(&stat) : dim == 2 ? tp::layer_static_smem_d2(&stat)
                                                                     : tp::layer_static_smem_d3(&stat));
  if ((size_t)optin <= stat + kTwoPerSmSmem) {
    *cap = kTwoPerSmSmem;
  } else {
    *cap = ((size_t)optin - stat) & ~(size_t)1023;
  }
  return TP_OK;
}

int set_smem_attr(int dim, size_t cap) {
  cudaError_t e = dim == 1 ? tp::layer_attrs_d1(cap) : dim == 2 ? tp::layer_attrs_d2(cap) : tp::layer_attrs_d3(cap);
  TP_CUDA_OK(e);
  return TP_OK;
}

cudaError_t launch_layer(tp_ctx* ctx, const KArgs& a, int n_cluster, int cs, int t0, cudaStream_t st, int mode,
                         bool persistent) {
  if (ctx->neumann) mode |= 4;   // the kernel variant with the Neumann facet code
  switch (ctx->dim) {
    case 1: return tp::launch_layer_d1(a, n_cluster, cs, t0, ctx->smem_bytes, st, mode, persistent);
    case 2: return tp::launch_layer_d2(a, n_cluster, cs, t0, ctx->smem_bytes, st, mode, persistent);
    default: return tp::launch_layer_d3(a, n_cluster, cs, t0, ctx->smem_bytes, st, mode, persistent);
  }
}

// resident clusters of the persistent kernel for cluster size cs
int set_persist_cs(tp_ctx* ctx, int cs) {
  int nclu = 0;
  const int mode = (ctx->mixed ? 1 : 0) | (ctx->neumann ? 4 : 0);
  cudaError_t e = ctx->dim == 1 ? tp::max_clusters_d1(cs, ctx->smem_bytes, mode, &nclu)
                : ctx->dim == 2 ? tp::max_clusters_d2(cs, ctx->smem_bytes, mode, &nclu)
                                : tp::max_clusters_d3(cs, ctx->smem_bytes, mode, &nclu);
  if (e != cudaSuccess || nclu < 1) {
    cudaGetLastError();
    return TP_ERR_UNSUPPORTED;
  }
  ctx->persist_cs = cs;
  ctx->persist_clusters = nclu;
  return TP_OK;
}

// autotuner results for this process: (dim, p, nrhs, mixed, patch bucket) -> (cs, dataflow?)
std::mutex g_tune_mu;
std::map<std::vector<int>, std::pair<int, bool>> g_tuned;

bool tuned_lookup(const int* key, int* cs, bool* dataflow) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find(std::vector<int>(key, key + 5));
  if (it == g_tuned.end()) return false;
  *cs = it->second.first;
  *dataflow = it->second.second;
  return true;
}

// cluster size for a level of nt tents: a power of two <= max_cs with
// nt * cs <= 2 CTAs per SM
int level_cluster_size(const tp_ctx* ctx, int64_t nt) {
  if (ctx->rsplit_cs > 1) return ctx->rsplit_cs;   // one CTA per slice of the right-hand sides
  int cs = 1;
  while (cs * 2 <= ctx->max_cs && nt * cs * 2 <= 2LL * ctx->n_sm) cs *= 2;
  return cs;
}

// the arguments of right-hand-side group k: its slice of the front and of
// the boundary data (both right-hand-side major)
KArgs group_args(const tp_ctx* ctx, KArgs a, int k) {
  a.front += (size_t)k * ctx->nrhs_g * ctx->ne * ctx->Q * ctx->C;
  if (a.gD) a.gD += (size_t)k * ctx->nrhs_g * ctx->n_bnd;
  if (a.diss) a.diss += (size_t)k * ctx->nrhs_g;
  if (a.probe_out) a.probe_out += (size_t)k * ctx->nrhs_g * ctx->n_probe_t * ctx->n_probe;
  return a;
}

// one level; group < 0: every right-hand-side group, each from the front
// times before the level (saved, and restored before every group after the first)
int launch_level(tp_ctx* ctx, int32_t L, cudaStream_t st, bool adj = false, int group = -1) {
  const int64_t t0 = ctx->level_ptr[L - 1], t1 = ctx->level_ptr[L];
  if (t1 <= t0) return TP_OK;
  const int nt = (int)(t1 - t0);
  const int cs = level_cluster_size(ctx, nt);
  const int mode = adj ? 2 : (ctx->mixed ? 1 : 0);
  double* tau = adj ? ctx->d_tau_adj : ctx->d_tau;
  const int k0 = group < 0 ? 0 : group, k1 = group < 0 ? ctx->rhs_groups : group + 1;
  const bool restore = group < 0 && ctx->rhs_groups > 1;
  if (restore) TP_CUDA_OK(cudaMemcpyAsync(ctx->d_tau_save, tau, ctx->nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
  for (int k = k0; k < k1; ++k) {
    if (restore && k > 0)
      TP_CUDA_OK(cudaMemcpyAsync(tau, ctx->d_tau_save, ctx->nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
    cudaError_t e = launch_layer(ctx, group_args(ctx, adj ? ctx->args_adj : ctx->args, k), nt, cs, (int)t0, st, mode, false);
    TP_CUDA_OK(e);
    TP_CUDA_OK(cudaGetLastError());
  }
  return TP_OK;
}

// one level with explicit kernel arguments (one right-hand-side group)
int launch_level_with(tp_ctx* ctx, int32_t L, cudaStream_t st, bool adj, const KArgs& a) {
  const int64_t t0 = ctx->level_ptr[L - 1], t1 = ctx->level_ptr[L];
  if (t1 <= t0) return TP_OK;
  const int nt = (int)(t1 - t0);
  TP_CUDA_OK(launch_layer(ctx, a, nt, level_cluster_size(ctx, nt), (int)t0, st, adj ? 2 : (ctx->mixed ? 1 : 0), false));
  TP_CUDA_OK(cudaGetLastError());
  return TP_OK;
}

}  // namespace

extern "C" int tp_create(const tp_mesh_desc* mesh, const tp_tents* tents, const tp_basis* basis,
                         const tp_params* prm, tp_ctx** out) {
  if (!mesh || !tents || !basis || !prm || !out) {
    tp::set_error("tp_create: null argument");
    return TP_ERR_ARG;
  }
  if (mesh->dim != basis->dim || mesh->dim != tents->dim || prm->p != basis->p ||
      mesh->n_vert != tents->nv || prm->nrhs < 1) {
    tp::set_error("tp_create: dim/p/n_vert mismatch between mesh, tents, basis and params");
    return TP_ERR_ARG;
  }
  if (prm->precision != TP_FP64 && prm->precision != TP_MIXED) {
    tp::set_error("tp_create: precision must be TP_FP64 or TP_MIXED");
    return TP_ERR_ARG;
  }
  auto* ctx = new tp_ctx();
  auto fail = [&](int rc) {
    tp_destroy_ctx(ctx);
    return rc;
  };
  if (!tp::build_topology(mesh, &ctx->topo)) return fail(TP_ERR_ARG);
  tp::Topology& T = ctx->topo;
  const int n = T.dim;
  ctx->dim = n;
  ctx->p = basis->p;
  ctx->nb = basis->nb;
  ctx->nmono = basis->nmono;
  ctx->C = n + 2;
  ctx->nrhs = prm->nrhs;
  ctx->alpha = prm->alpha;
  ctx->mixed = (prm->precision == TP_MIXED);
  ctx->persistent = (prm->schedule == TP_SCHED_DATAFLOW);
  ctx->nv = T.nv;
  ctx->ne = T.ne;
  ctx->rule = tp::simplex_rule(n, basis->p + 1);
  ctx->Q = ctx->rule.Q;
  ctx->ntents = (int64_t)tents->vert.size();
  ctx->n_levels = tents->n_levels;
  ctx->level_ptr = tents->level_ptr;
  ctx->neumann = std::find(T.facet_kind.begin(), T.facet_kind.end(), (int8_t)1) != T.facet_kind.end();
  // patch checks: size limits; materials (distinct wave speeds) per tent
  int ngmax = 1, pmax = 1;
  std::vector<std::array<int, 4>> facet_mix;   // distinct (materials, Dirichlet, interface, Neumann facets)
  for (int64_t v = 0; v < T.nv; ++v) {
    const int p0 = T.star_ptr[v], p1 = T.star_ptr[v + 1];
    pmax = std::max(pmax, p1 - p0);
    if ((T.vfac_ptr[v + 1] - T.vfac_ptr[v]) + (T.ifac_ptr[v + 1] - T.ifac_ptr[v]) > tp::kMaxFacets) {
      tp::set_error("tp_create: vertex " + std::to_string(v) + " lies on more than 16 boundary or interface facets");
      return fail(TP_ERR_UNSUPPORTED);
    }
    if (p1 - p0 > tp::kMaxPatch) {
      tp::set_error("tp_create: vertex " + std::to_string(v) + " has more than 64 elements");
      return fail(TP_ERR_UNSUPPORTED);
    }
    std::vector<double> speeds;
    for (int e = p0; e < p1; ++e)
      if (std::find(speeds.begin(), speeds.end(), T.c[T.star_el[e]]) == speeds.end())
        speeds.push_back(T.c[T.star_el[e]]);
    ngmax = std::max(ngmax, (int)speeds.size());
    int nneu_v = 0;
    for (int e = T.vfac_ptr[v]; e < T.vfac_ptr[v + 1]; ++e) nneu_v += T.facet_kind[T.vfac[e]];
    const std::array<int, 4> mix = {(int)speeds.size(), T.vfac_ptr[v + 1] - T.vfac_ptr[v] - nneu_v,
                                    T.ifac_ptr[v + 1] - T.ifac_ptr[v], nneu_v};
    if (std::find(facet_mix.begin(), facet_mix.end(), mix) == facet_mix.end()) facet_mix.push_back(mix);
  }
  if (ngmax > tp::kMaxGroups) {
    tp::set_error("tp_create: a tent has more than 4 materials (wave speeds)");
    return fail(TP_ERR_UNSUPPORTED);
  }
  // replay the tents on the host: anisotropic diameter (eq. 3.3) and the
  // Dirichlet quadrature points of every tent
  std::vector<double> tau(T.nv, 0.0), tent_h(ctx->ntents);
  std::vector<long long> gdoff(ctx->ntents + 1, 0);
  const int Q = ctx->Q;
  for (int64_t it = 0; it < ctx->ntents; ++it) {
    const int v = tents->vert[it];
    double c = 0.0;   // the largest speed of the tent
    for (int e = T.star_ptr[v]; e < T.star_ptr[v + 1]; ++e) c = std::max(c, T.c[T.star_el[e]]);
    const double tb = tau[v], tt = tents->t_top[it];
    std::vector<std::vector<double>> pts;
    auto push = [&](int w, double t) {
      std::vector<double> pnt(n + 1);
      for (int d = 0; d < n; ++d) pnt[d] = T.X[(int64_t)w * n + d];
      pnt[n] = t;
      pts.push_back(pnt);
    };
    push(v, tb);
    push(v, tt);
    for (int e = T.nbr_ptr[v]; e < T.nbr_ptr[v + 1]; ++e) push(T.nbr[e], tau[T.nbr[e]]);
    double best = 0.0;
    for (size_t i = 0; i < pts.size(); ++i)
      for (size_t j = i + 1; j < pts.size(); ++j) {
        double s = 0.0;
        for (int d = 0; d < n; ++d) s += (pts[i][d] - pts[j][d]) * (pts[i][d] - pts[j][d]);
        const double dt = pts[i][n] - pts[j][n];
        s += c * c * dt * dt;
        best = std::max(best, std::sqrt(s));
      }
    tent_h[it] = best;
    const int nf = T.vfac_ptr[v + 1] - T.vfac_ptr[v];
    gdoff[it + 1] = gdoff[it] + (long long)nf * Q;
    for (int f = 0; f < nf; ++f) {
      const int fid = T.vfac[T.vfac_ptr[v] + f];
      double P[4][4];
      for (int d = 0; d < n; ++d) P[0][d] = P[1][d] = T.X[(int64_t)v * n + d];
      P[0][n] = tb;
      P[1][n] = tt;
      int c2 = 2;
      for (int i = 0; i < n; ++i) {
        const int w = T.facet_vert[(int64_t)fid * n + i];
        if (w == v) continue;
        for (int d = 0; d < n; ++d) P[c2][d] = T.X[(int64_t)w * n + d];
        P[c2][n] = tau[w];
        ++c2;
      }
      for (int q = 0; q < Q; ++q) {
        for (int d = 0; d <= n; ++d) {
          double s = 0.0;
          for (int i = 0; i <= n; ++i) s += ctx->rule.bary[q * (n + 1) + i] * P[i][d];
          ctx->bnd_xt.push_back(s);
        }
        for (int d = 0; d < n; ++d) ctx->bnd_nrm.push_back(T.facet_nrm[(int64_t)fid * n + d]);
        ctx->bnd_kind.push_back(T.facet_kind[fid]);
      }
    }
    tau[v] = tt;
  }
  ctx->n_bnd = gdoff[ctx->ntents];
  gdoff.pop_back();

  // dependencies of the dataflow sweep: tent (v, L) waits until every vertex w
  // of {v} and its neighbours has completed its tents of level < L
  std::vector<int32_t> dep_ptr(ctx->ntents + 1, 0), dep_vert, dep_need;
  {
    std::vector<std::vector<int32_t>> lev_at(T.nv);
    for (int64_t it = 0; it < ctx->ntents; ++it) lev_at[tents->vert[it]].push_back(tents->level[it]);
    for (int64_t it = 0; it < ctx->ntents; ++it) {
      const int v = tents->vert[it], L = tents->level[it];
      auto add = [&](int w) {
        const auto& lv = lev_at[w];
        const int need = (int)(std::lower_bound(lv.begin(), lv.end(), L) - lv.begin());
        if (need > 0) {
          dep_vert.push_back(w);
          dep_need.push_back(need);
        }
      };
      add(v);
      for (int e = T.nbr_ptr[v]; e < T.nbr_ptr[v + 1]; ++e) add(T.nbr[e]);
      dep_ptr[it + 1] = (int32_t)dep_vert.size();
    }
  }
  // dataflow queue order: level by level (every awaited tent is earlier in the
  // queue), and within a level the tents with the longest chain of dependent
  // work after them first, so that a cluster that frees up takes a tent on the
  // critical path.  Work of a tent: 1, +0.2 with Dirichlet or interface facets.
  std::vector<int32_t> queue_tent(ctx->ntents);
  {
    std::vector<std::vector<int32_t>> tents_at(T.nv);
    for (int64_t it = 0; it < ctx->ntents; ++it) tents_at[tents->vert[it]].push_back((int32_t)it);
    std::vector<std::vector<int32_t>> succ(ctx->ntents);
    for (int64_t it = 0; it < ctx->ntents; ++it)
      for (int e = dep_ptr[it]; e < dep_ptr[it + 1]; ++e) succ[tents_at[dep_vert[e]][dep_need[e] - 1]].push_back((int32_t)it);
    std::vector<double> height(ctx->ntents, 0.0);
    for (int64_t it = ctx->ntents - 1; it >= 0; --it) {   // tents are sorted by level
      const int v = tents->vert[it];
      double h = 0.0;
      for (int32_t sc : succ[it]) h = std::max(h, height[sc]);
      const bool extra = (T.vfac_ptr[v + 1] > T.vfac_ptr[v]) || (T.ifac_ptr[v + 1] > T.ifac_ptr[v]);
      height[it] = h + (extra ? 1.2 : 1.0);
    }
    for (int64_t it = 0; it < ctx->ntents; ++it) queue_tent[it] = (int32_t)it;
    for (int L = 0; L < tents->n_levels; ++L) {
      const int64_t b = tents->level_ptr[L], e = tents->level_ptr[L + 1];
      std::stable_sort(queue_tent.begin() + b, queue_tent.begin() + e,
                       [&](int32_t x, int32_t y) { return height[x] > height[y]; });
    }
  }

  // device uploads
  int rc = TP_OK;
  KArgs& a = ctx->args;
  double *dX, *dc, *dbary, *dw, *dsqw, *dttop, *dspc;
  int *del, *dtv, *dspp, *dspm, *dpar, *dvar, *drp, *drs, *dtp, *dtd;
  int *ddp, *ddv, *ddn, *dqt;
  double *drf, *dtf;
  float2* dcdd;
  float2* dsqwff = nullptr;
  float *drff, *dtff;
  std::vector<float2> coef_dd(basis->sp_coef.size());
  for (size_t i = 0; i < coef_dd.size(); ++i) {
    const float hi = (float)basis->sp_coef[i];
    coef_dd[i] = make_float2(hi, (float)(basis->sp_coef[i] - (double)hi));
  }
  std::vector<float> rel_ff(basis->rel_fac.begin(), basis->rel_fac.end());
  std::vector<float> relT_ff(basis->relT_fac.begin(), basis->relT_fac.end());
  long long* dgo;
  std::vector<double> sqw(Q);
  for (int q = 0; q < Q; ++q) sqw[q] = std::sqrt(ctx->rule.w[q]);
  // sqrt(w) as a float-float pair (hi = nearest binary32, lo = the rest rounded)
  std::vector<float2> sqw_ff(Q);
  for (int q = 0; q < Q; ++q) {
    const float h = (float)sqw[q];
    sqw_ff[q] = make_float2(h, (float)(sqw[q] - (double)h));
  }
  std::vector<double> ttop(tents->t_top.begin(), tents->t_top.end());
  std::vector<double> tbot(tents->t_bot.begin(), tents->t_bot.end());
  double* dtbot = nullptr;
  std::vector<int> tv(tents->vert.begin(), tents->vert.end());
  // vertex stars grouped by material: speeds in order of first appearance
  // (bitwise-equal c), elements of each material in star order
  std::vector<int> star_sorted(T.star_el.size()), star_grp(T.star_el.size()), vert_ng(T.nv);
  std::vector<double> vert_gc((size_t)T.nv * tp::kMaxGroups, 0.0);
  for (int64_t v = 0; v < T.nv; ++v) {
    const int p0 = T.star_ptr[v], p1 = T.star_ptr[v + 1];
    int ng = 0;
    for (int e = p0; e < p1; ++e) {
      const double ck = T.c[T.star_el[e]];
      int g = 0;
      while (g < ng && vert_gc[(size_t)v * tp::kMaxGroups + g] != ck) ++g;
      if (g == ng) vert_gc[(size_t)v * tp::kMaxGroups + ng++] = ck;
    }
    vert_ng[v] = ng;
    int pos = p0;
    for (int g = 0; g < ng; ++g)
      for (int e = p0; e < p1; ++e)
        if (T.c[T.star_el[e]] == vert_gc[(size_t)v * tp::kMaxGroups + g]) {
          star_sorted[pos] = T.star_el[e];
          star_grp[pos++] = g;
        }
  }
  ctx->star_sorted = star_sorted;
  ctx->tent_vert_h.assign(tents->vert.begin(), tents->vert.end());
  ctx->tent_ttop_h.assign(tents->t_top.begin(), tents->t_top.end());
  int *dftp = nullptr, *dfti = nullptr, *dfmp = nullptr, *dfmi = nullptr;
  float *dftc = nullptr, *dfmc = nullptr;
  if ((rc = ctx_upload(ctx, &dftp, basis->ft_ptr)) || (rc = ctx_upload(ctx, &dfti, basis->ft_idx)) ||
      (rc = ctx_upload(ctx, &dfmp, basis->fm_ptr)) || (rc = ctx_upload(ctx, &dfmi, basis->fm_idx)) ||
      (rc = ctx_upload(ctx, &dftc, basis->ft_coef)) || (rc = ctx_upload(ctx, &dfmc, basis->fm_coef)))
    return fail(rc);
  double *dcgd = nullptr, *dchd = nullptr, *dftd = nullptr, *dfmd = nullptr;   // binary64 copies (exact)
  {
    auto widen = [](const std::vector<float>& f) { return std::vector<double>(f.begin(), f.end()); };
    if ((rc = ctx_upload(ctx, &dcgd, widen(basis->cg_coef))) || (rc = ctx_upload(ctx, &dchd, widen(basis->ch_coef))) ||
        (rc = ctx_upload(ctx, &dftd, widen(basis->ft_coef))) || (rc = ctx_upload(ctx, &dfmd, widen(basis->fm_coef))))
      return fail(rc);
  }
  int *dpij = nullptr, *dcgp = nullptr, *dcgi = nullptr, *dchp = nullptr, *dchi = nullptr;
  float *dcgc = nullptr, *dchc = nullptr;
  if ((rc = ctx_upload(ctx, &dpij, basis->pair_ij)) || (rc = ctx_upload(ctx, &dcgp, basis->cg_ptr)) ||
      (rc = ctx_upload(ctx, &dcgi, basis->cg_idx)) || (rc = ctx_upload(ctx, &dchp, basis->ch_ptr)) ||
      (rc = ctx_upload(ctx, &dchi, basis->ch_idx)) || (rc = ctx_upload(ctx, &dcgc, basis->cg_coef)) ||
      (rc = ctx_upload(ctx, &dchc, basis->ch_coef)))
    return fail(rc);
  // per element: inverse of the edge matrix e (rows X_i - X_0), so that the
  // gradient of a linear function is e^-1 (its increments along the edges), and sqrt|det e|
  std::vector<double> einv((size_t)T.ne * n * n), esdet(T.ne);
  for (int64_t k = 0; k < T.ne; ++k) {
    double e[3][3] = {};
    const int* vk = &T.elems[(size_t)k * (n + 1)];
    for (int i = 0; i < n; ++i)
      for (int d = 0; d < n; ++d) e[i][d] = T.X[(size_t)vk[i + 1] * n + d] - T.X[(size_t)vk[0] * n + d];
    double inv[3][3] = {}, det;
    if (n == 1) {
      det = e[0][0];
      inv[0][0] = 1.0 / det;
    } else if (n == 2) {
      det = e[0][0] * e[1][1] - e[0][1] * e[1][0];
      inv[0][0] = e[1][1] / det;
      inv[0][1] = -e[0][1] / det;
      inv[1][0] = -e[1][0] / det;
      inv[1][1] = e[0][0] / det;
    } else {
      double c[3][3];   // c[i] = cofactor column of edge i: rows of e^-T times det
      c[0][0] = e[1][1] * e[2][2] - e[1][2] * e[2][1];
      c[0][1] = e[1][2] * e[2][0] - e[1][0] * e[2][2];
      c[0][2] = e[1][0] * e[2][1] - e[1][1] * e[2][0];
      c[1][0] = e[2][1] * e[0][2] - e[2][2] * e[0][1];
      c[1][1] = e[2][2] * e[0][0] - e[2][0] * e[0][2];
      c[1][2] = e[2][0] * e[0][1] - e[2][1] * e[0][0];
      c[2][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
      c[2][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
      c[2][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
      det = e[0][0] * c[0][0] + e[0][1] * c[0][1] + e[0][2] * c[0][2];
      for (int d = 0; d < 3; ++d)
        for (int i = 0; i < 3; ++i) inv[d][i] = c[i][d] / det;
    }
    for (int d = 0; d < n; ++d)
      for (int i = 0; i < n; ++i) einv[((size_t)k * n + d) * n + i] = inv[d][i];
    esdet[k] = std::sqrt(std::fabs(det));
  }
  // reciprocals of sqrt|det e| and of the reference weights' square roots
  // (the kept top U-values are unscaled by 1/sqrt(w) = 1/(sqrt(w_ref) sqrt|det e|))
  std::vector<double> eisdet(T.ne), isqw(Q);
  for (int64_t k = 0; k < T.ne; ++k) eisdet[k] = 1.0 / esdet[k];
  for (int q = 0; q < Q; ++q) isqw[q] = 1.0 / sqw[q];
  double *deinv = nullptr, *desdet = nullptr, *deisdet = nullptr, *disqw = nullptr;
  if ((rc = ctx_upload(ctx, &deinv, einv)) || (rc = ctx_upload(ctx, &desdet, esdet)) ||
      (rc = ctx_upload(ctx, &deisdet, eisdet)) || (rc = ctx_upload(ctx, &disqw, isqw)))
    return fail(rc);
  // per vertex: one record with all of its star that does not depend on the
  // sweep, so that a tent reads it in one round of loads.
  //   ints:    per element (el, material, vertex ids[n+1]); per facet (Dirichlet
  //            first, then interface, then Neumann): (elements of the + and -
  //            sides in slots 0, 1, vertex ids other than v in slots 2..n,
  //            material of the + element, of the - element, position among the
  //            vertex's boundary facets = block of its boundary data)
  //   doubles: x_v[n], speeds[kMaxGroups], their 1/c^2 [kMaxGroups]; per element its vertex coordinates
  //            [(n+1) n]; per facet its normal [n] and vertex coordinates [(n+1) n]
  // per tent: (v, int offset, double offset, elements, Dirichlet facets,
  // interface facets, materials, Neumann facets)
  std::vector<int> rec_i, tent_hdr((size_t)ctx->ntents * 8, 0);
  std::vector<double> rec_d;
  std::vector<int> vrec_i(T.nv), vrec_d(T.nv);
  {
    const int NVn = n + 1;
    auto grp_of = [&](int64_t v, double ck) {
      int g = 0;
      while (g < vert_ng[v] - 1 && vert_gc[(size_t)v * tp::kMaxGroups + g] != ck) ++g;
      return g;
    };
    for (int64_t v = 0; v < T.nv; ++v) {
      vrec_i[v] = (int)rec_i.size();
      vrec_d[v] = (int)rec_d.size();
      for (int d = 0; d < n; ++d) rec_d.push_back(T.X[(size_t)v * n + d]);
      for (int g = 0; g < tp::kMaxGroups; ++g) rec_d.push_back(vert_gc[(size_t)v * tp::kMaxGroups + g]);
      for (int g = 0; g < tp::kMaxGroups; ++g) {
        const double cg = vert_gc[(size_t)v * tp::kMaxGroups + g];
        rec_d.push_back(g < vert_ng[v] ? 1.0 / (cg * cg) : 0.0);
      }
      for (int e = T.star_ptr[v]; e < T.star_ptr[v + 1]; ++e) {
        const int el = star_sorted[e];
        rec_i.push_back(el);
        rec_i.push_back(star_grp[e]);
        for (int i = 0; i < NVn; ++i) {
          const int vi = T.elems[(size_t)el * NVn + i];
          rec_i.push_back(vi);
          for (int d = 0; d < n; ++d) rec_d.push_back(T.X[(size_t)vi * n + d]);
        }
      }
      const int nb_v = T.vfac_ptr[v + 1] - T.vfac_ptr[v], ni = T.ifac_ptr[v + 1] - T.ifac_ptr[v];
      // (kind, id, data block): Dirichlet facets, interface facets, Neumann facets
      std::vector<std::array<int, 3>> order;
      for (int pass = 0; pass < 3; ++pass) {
        if (pass == 1) {
          for (int f = 0; f < ni; ++f) order.push_back({2, T.ifac_ptr[v] + f, -1});
          continue;
        }
        for (int f = 0; f < nb_v; ++f) {
          const int fid = T.vfac[T.vfac_ptr[v] + f];
          if (T.facet_kind[fid] == (pass == 0 ? 0 : 1)) order.push_back({pass == 0 ? 0 : 1, fid, f});
        }
      }
      for (const auto& fo : order) {
        const bool bnd = fo[0] != 2;
        const int fid = fo[1];
        const int* fv = bnd ? &T.facet_vert[(size_t)fid * n] : &T.ifac_vert[(size_t)fid * n];
        const double* fn = bnd ? &T.facet_nrm[(size_t)fid * n] : &T.ifac_nrm[(size_t)fid * n];
        int w_[4] = {(int)v, (int)v, -1, -1};
        int c2 = 2;
        for (int i = 0; i < n; ++i)
          if (fv[i] != v) w_[c2++] = fv[i];
        // slots 0 and 1: the elements on the facet's + and - sides (a boundary
        // facet's own element twice; read by the wave-speed gradient), then the
        // facet's other vertices
        rec_i.push_back(bnd ? T.facet_elem[fid] : T.ifac_kp[fid]);
        rec_i.push_back(bnd ? T.facet_elem[fid] : T.ifac_km[fid]);
        for (int i = 2; i < NVn; ++i) rec_i.push_back(w_[i]);
        rec_i.push_back(grp_of(v, T.c[bnd ? T.facet_elem[fid] : T.ifac_kp[fid]]));
        rec_i.push_back(grp_of(v, T.c[bnd ? T.facet_elem[fid] : T.ifac_km[fid]]));
        rec_i.push_back(fo[2]);
        for (int d = 0; d < n; ++d) rec_d.push_back(fn[d]);
        for (int i = 0; i < NVn; ++i)
          for (int d = 0; d < n; ++d) rec_d.push_back(w_[i] >= 0 ? T.X[(size_t)w_[i] * n + d] : 0.0);
      }
    }
    for (int64_t it = 0; it < ctx->ntents; ++it) {
      const int v = tents->vert[it];
      int* h = &tent_hdr[(size_t)it * 8];
      h[0] = v;
      h[1] = vrec_i[v];
      h[2] = vrec_d[v];
      h[3] = T.star_ptr[v + 1] - T.star_ptr[v];
      int nneu = 0;
      for (int e = T.vfac_ptr[v]; e < T.vfac_ptr[v + 1]; ++e) nneu += T.facet_kind[T.vfac[e]];
      h[4] = T.vfac_ptr[v + 1] - T.vfac_ptr[v] - nneu;   // Dirichlet facets
      h[5] = T.ifac_ptr[v + 1] - T.ifac_ptr[v];
      h[6] = vert_ng[v];
      h[7] = nneu;
    }
  }
  std::vector<double> tent_ih(ctx->ntents);
  for (int64_t it = 0; it < ctx->ntents; ++it) tent_ih[it] = 1.0 / tent_h[it];
  int *dthdr = nullptr, *dreci = nullptr;
  double *drecd = nullptr, *dtih = nullptr;
  if ((rc = ctx_upload(ctx, &dthdr, tent_hdr)) || (rc = ctx_upload(ctx, &dreci, rec_i)) ||
      (rc = ctx_upload(ctx, &drecd, rec_d)) || (rc = ctx_upload(ctx, &dtih, tent_ih)))
    return fail(rc);
  if ((rc = ctx_upload(ctx, &dX, T.X)) || (rc = ctx_upload(ctx, &dc, T.c)) ||
      (rc = ctx_upload(ctx, &del, T.elems)) || (rc = ctx_upload(ctx, &dbary, ctx->rule.bary)) ||
      (rc = ctx_upload(ctx, &ddp, dep_ptr)) || (rc = ctx_upload(ctx, &ddv, dep_vert)) ||
      (rc = ctx_upload(ctx, &ddn, dep_need)) || (rc = ctx_upload(ctx, &dqt, queue_tent)) ||
      (rc = ctx_upload(ctx, &dw, ctx->rule.w)) || (rc = ctx_upload(ctx, &dsqw, sqw)) ||
      (rc = ctx_upload(ctx, &dtv, tv)) || (rc = ctx_upload(ctx, &dttop, ttop)) ||
      (rc = ctx_upload(ctx, &dtbot, tbot)) ||
      (rc = ctx_upload(ctx, &dgo, gdoff)) ||
      (rc = ctx_upload(ctx, &dspp, basis->sp_ptr)) || (rc = ctx_upload(ctx, &dspm, basis->sp_mono)) ||
      (rc = ctx_upload(ctx, &dspc, basis->sp_coef)) || (rc = ctx_upload(ctx, &dpar, basis->parent)) ||
      (rc = ctx_upload(ctx, &dvar, basis->var)) || (rc = ctx_upload(ctx, &drp, basis->rel_ptr)) ||
      (rc = ctx_upload(ctx, &drs, basis->rel_src)) || (rc = ctx_upload(ctx, &drf, basis->rel_fac)) ||
      (rc = ctx_upload(ctx, &dtp, basis->relT_ptr)) || (rc = ctx_upload(ctx, &dtd, basis->relT_dst)) ||
      (rc = ctx_upload(ctx, &dtf, basis->relT_fac)) || (rc = ctx_upload(ctx, &dcdd, coef_dd)) || (rc = ctx_upload(ctx, &dsqwff, sqw_ff)) ||
      (rc = ctx_upload(ctx, &drff, rel_ff)) || (rc = ctx_upload(ctx, &dtff, relT_ff)))
    return fail(rc == TP_ERR_CUDA ? TP_ERR_OOM : rc);
  const size_t nfront = (size_t)ctx->nrhs * T.ne * Q * ctx->C;
  if (cudaMalloc(&ctx->d_front, nfront * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_tau, T.nv * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_status, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_info, sizeof(long long)) != cudaSuccess ||
      (ctx->n_bnd > 0 &&
       cudaMalloc(&ctx->d_gD, (size_t)ctx->nrhs * ctx->n_bnd * sizeof(double)) != cudaSuccess)) {
    tp::set_error("tp_create: device allocation of the front state failed");
    return fail(TP_ERR_OOM);
  }
  // (the adjoint state is allocated by the first tp_adjoint)
  ctx->T_final = tents->T;
  if (cudaMalloc(&ctx->d_queue, sizeof(int)) != cudaSuccess ||
      cudaMalloc(&ctx->d_done, T.nv * sizeof(int)) != cudaSuccess) {
    tp::set_error("tp_create: device allocation failed");
    return fail(TP_ERR_OOM);
  }
  if (prm->ckpt_stride < 0) {
    tp::set_error("tp_create: ckpt_stride must be >= 0");
    return fail(TP_ERR_ARG);
  }
  ctx->ckpt_stride = prm->ckpt_stride;
  if (ctx->ckpt_stride > 0 &&
      cudaMalloc(&ctx->d_front0, (size_t)ctx->nrhs * T.ne * Q * ctx->C * sizeof(double)) != cudaSuccess) {
    tp::set_error("tp_create: device allocation of the initial-state copy failed");
    return fail(TP_ERR_OOM);
  }
  if (prm->dissipation && cudaMalloc(&ctx->d_diss, (size_t)ctx->nrhs * sizeof(double)) != cudaSuccess) {
    tp::set_error("tp_create: device allocation failed");
    return fail(TP_ERR_OOM);
  }
  if (ctx->d_diss) cudaMemset(ctx->d_diss, 0, (size_t)ctx->nrhs * sizeof(double));
  ctx->energy_blocks = (int)std::min<int64_t>(1024, (T.ne + kThreads - 1) / kThreads);
  if (cudaMalloc(&ctx->d_partial, (size_t)ctx->nrhs * ctx->energy_blocks * sizeof(double)) != cudaSuccess) {
    tp::set_error("tp_create: device allocation failed");
    return fail(TP_ERR_OOM);
  }
  cudaMemset(ctx->d_front, 0, nfront * sizeof(double));
  cudaMemset(ctx->d_tau, 0, T.nv * sizeof(double));
  cudaMemset(ctx->d_status, 0, sizeof(int));
  cudaMemset(ctx->d_info, 0, sizeof(long long));
  cudaGetDevice(&ctx->device);

  a.nb = ctx->nb;
  a.nmono = ctx->nmono;
  a.p = basis->p;
  {
    // the monomial list is ordered by total degree: offsets of each degree
    std::vector<int> cnt(basis->p + 2, 0);
    for (int g = 0; g < basis->nmono; ++g) {
      int deg = 0;
      for (int d = 0; d <= n; ++d) deg += basis->exps[g * (n + 1) + d];
      ++cnt[deg + 1];
    }
    for (int d = 0; d <= basis->p + 1; ++d) a.mono_lv[d] = (d ? a.mono_lv[d - 1] : 0) + cnt[d];
  }
  {
    // U-value sums: functions ordered by their number of terms (key 0: one
    // term of coefficient 1, a copy)
    const int Cc = n + 2;
    std::vector<std::pair<int, int>> key(basis->nb);
    for (int j = 0; j < basis->nb; ++j) {
      const int e0 = basis->sp_ptr[j * Cc], e1 = basis->sp_ptr[j * Cc + 1];
      key[j] = {(e1 - e0 == 1 && basis->sp_coef[e0] == 1.0) ? 0 : e1 - e0, j};
    }
    std::sort(key.begin(), key.end());
    std::vector<int> ev_order;
    a.ev_ncls = 0;
    for (int j = 0; j < basis->nb; ++j) {
      if (j == 0 || key[j].first != key[j - 1].first) {
        if (a.ev_ncls == tp::kMaxEvCls) {
          tp::set_error("tp_create: basis functions with more than 16 distinct term counts");
          return fail(TP_ERR_UNSUPPORTED);
        }
        a.ev_off[a.ev_ncls] = j;
        a.ev_terms[a.ev_ncls++] = key[j].first;
      }
      ev_order.push_back(key[j].second);
    }
    a.ev_off[a.ev_ncls] = basis->nb;
    int* devo = nullptr;
    if ((rc = ctx_upload(ctx, &devo, ev_order))) return fail(rc);
    a.ev_order = devo;
  }
  a.Q = Q;
  a.nrhs = ctx->nrhs;
  a.ne = T.ne;
  a.n_bnd = ctx->n_bnd;
  a.alpha = ctx->alpha;
  a.beta = prm->beta;
  a.ngmax = ngmax;
  a.dep_ptr = ddp;
  a.dep_vert = ddv;
  a.dep_need = ddn;
  ctx->d_dep_need = ddn;
  ctx->dep_ptr_h = dep_ptr;
  ctx->dep_need_h = dep_need;
  a.max_spin = tp::kMaxSpin;
  a.max_refine = tp::kMaxRefine;
  if (cudaMalloc(&ctx->d_stats, (tp::kMaxRefine + 2) * sizeof(unsigned long long)) != cudaSuccess) {
    tp::set_error("tp_create: device allocation failed");
    return fail(TP_ERR_OOM);
  }
  cudaMemset(ctx->d_stats, 0, (tp::kMaxRefine + 2) * sizeof(unsigned long long));
  a.solve_stats = ctx->d_stats;
  a.queue_tent = dqt;
  a.X = dX;
  a.elems = del;
  a.cK = dc;
  a.ft_ptr = dftp;
  a.ft_idx = dfti;
  a.ft_coef = dftc;
  a.fm_ptr = dfmp;
  a.fm_idx = dfmi;
  a.fm_coef = dfmc;
  a.pair_ij = dpij;
  a.cg_ptr = dcgp;
  a.cg_idx = dcgi;
  a.ch_ptr = dchp;
  a.ch_idx = dchi;
  a.cg_coef = dcgc;
  a.ch_coef = dchc;
  a.cg_coefd = dcgd;
  a.ch_coefd = dchd;
  a.ft_coefd = dftd;
  a.fm_coefd = dfmd;
  a.elem_einv = deinv;
  a.elem_sdet = desdet;
  a.elem_isdet = deisdet;
  a.isqw = disqw;
  a.bary = dbary;
  a.wref = dw;
  a.sqw = dsqw;
  a.tent_v = dtv;
  a.tent_ttop = dttop;
  a.tent_tbot = dtbot;
  a.tent_ih = dtih;
  a.tent_hdr = dthdr;
  a.vrec_i = dreci;
  a.vrec_d = drecd;
  a.tent_gdoff = dgo;
  a.sp_ptr = dspp;
  a.sp_mono = dspm;
  a.sp_coef = dspc;
  a.mono_parent = dpar;
  a.mono_var = dvar;
  a.rel_ptr = drp;
  a.rel_src = drs;
  a.rel_fac = drf;
  a.relT_ptr = dtp;
  a.relT_dst = dtd;
  a.relT_fac = dtf;
  a.sp_coef_dd = dcdd;
  a.sqw_dd = dsqwff;
  a.rel_facf = drff;
  a.relT_facf = dtff;
  a.tau = ctx->d_tau;
  a.queue = ctx->d_queue;
  a.done = ctx->d_done;
  a.tent_end = (int)ctx->ntents;
  a.front = ctx->d_front;
  a.gD = nullptr;
  a.diss = ctx->d_diss;
  a.status = ctx->d_status;
  a.status_info = ctx->d_info;
  // shared-memory plan: the largest chunk of points that fits
  const int nb = ctx->nb, C = ctx->C;
  const int npair = nb * (nb + 1) / 2;
  if (npair > kMaxPair * kThreads) {
    tp::set_error("tp_create: dim U^p too large for this kernel (more than 38)");
    return fail(TP_ERR_UNSUPPORTED);
  }
  a.mono_stride = ctx->nmono | 1;
  a.ustride = nb | 1;
  // shared-memory plan: the largest chunk of points that keeps two CTAs per SM,
  // else the largest that fits one
  int nrg = ctx->nrhs;   // right-hand sides per group
  bool ifneu = false;   // some tent has interface or Neumann facets
  for (const auto& m : facet_mix) ifneu = ifneu || m[2] > 0 || m[3] > 0;
  bool tc_try = false;   // the plan with the tensor-core staging
  auto plan = [&](int CH, int keep) {
    size_t off = 0;
    auto take = [&](int* field, size_t count) {
      if (field) *field = (int)off;
      off += count;
    };
    const size_t nmom = (size_t)nrg * C * nb;
    const size_t NB = (size_t)ngmax * nb;          // unknowns of the largest tent
    const size_t half_nb = (NB + 1) / 2, half_rb = ((size_t)nrg * NB + 1) / 2;
    // region used in turn by the monomials (point phases 1, 2, 4) and by A, the
    // summed Grams and the solve buffers (reduction to solve); A at offset 0
    // (the binary32 sweep buffers of the solve reuse the summed Grams, dead after the congruence)
    const size_t sg_al = std::max((size_t)ngmax * (n + 2) * npair, NB * NB);
    // interface blocks (tents with interface facets) followed by the Dirichlet
    // sums of every material (tents with Dirichlet facets), partials reduced in place
    // (and for tents with Neumann facets the blocks plus a partial b)
    size_t pd = 0;
    for (const auto& m : facet_mix)
      pd = std::max(pd, (m[2] > 0 || m[3] > 0 ? (size_t)m[0] * nb * m[0] * nb : 0) +
                            (m[1] > 0 ? (size_t)m[0] * (n + 1) * (npair + (size_t)nrg * nb) : 0) +
                            (m[3] > 0 ? (size_t)nrg * m[0] * nb : 0));
    const size_t solve_part = NB * NB + sg_al + (size_t)nrg * NB + half_rb;
    const size_t mono_part = (size_t)2 * CH * a.mono_stride;
    a.off_mono = 0;
    take(nullptr, NB * NB);                        // A
    a.off_al = (int)off;                           // two binary32 N x N sweep buffers
    take(&a.off_sg, sg_al);
    take(&a.off_x, (size_t)nrg * NB);
    take(&a.off_z, half_rb);
    off = std::max(solve_part, mono_part);
    take(&a.off_b, (size_t)nrg * NB);
    take(&a.off_pg, (size_t)ngmax * npair);        // G, H_m, Gbot contiguous
    take(&a.off_ph, (size_t)ngmax * n * npair);
    take(&a.off_pgb, (size_t)ngmax * npair);
    take(&a.off_pm, (size_t)ngmax * nmom);        // moments: partials, summed in place, then the outflow vectors
    a.off_sm = a.off_y = a.off_pm;
    // tensor-core staging (bf16 digit planes), in the region of the facet
    // sums (dead during the point passes before phase 2 and during the
    // outflow): the moments' A (rows of data coefficients x CH points) and B
    // (32 basis functions x CH points), or the outflow's A (rows x 32) and B
    // (2 CH points x 32), plus room for the row groups that A's M = 128 tile
    // reads past its stored rows
    size_t tcd = 0;
    if (tc_try) {
      const size_t RG = ((size_t)nrg * C + 7) / 8, NP2 = ((size_t)2 * CH + 15) / 16 * 16;
      const size_t NY = ((size_t)nrg * C + 15) / 16 * 16;
      const size_t mom = (size_t)tp::kTcSlices * CH * (RG * 8 + 32);
      const size_t out = (size_t)tp::kTcSlices * 32 * (NP2 + NY);
      tcd = ((std::max(mom, out) + 512 + 3) / 4 + 1) & ~(size_t)1;
    }
    off += off & 1;                                // 16-byte alignment of the staging
    a.off_tc = (int)off;
    take(&a.off_pd, std::max(pd, tcd));
    // facet Grams of interface and Neumann facets (none on meshes without them)
    take(&a.off_f, ifneu ? npair : 0);
    take(&a.off_f2, ifneu ? npair : 0);
    take(&a.off_fpm, ifneu ? (size_t)nb * nb : 0);
    take(&a.off_del, (size_t)nrg * nb);
    take(&a.off_u, (size_t)2 * CH * (nb | 1));
    take(&a.off_pt, (size_t)2 * CH * (n + 2));
    take(&a.off_cb, (size_t)(CH + 1) * nrg * C);   // data coefficients, rows of CH + 1
    take(&a.off_gd, (size_t)CH * nrg);
    take(&a.off_rd, NB);
    take(&a.off_eq, half_nb);
    take(&a.off_keep, (size_t)keep * nb);          // top U-values of the CTA's slice, kept for the outflow
    take(&a.off_keepw, (size_t)keep);
    // wave-speed gradient (reverse sweep): y(x), y(x'), y(mu') per material and the forward solution
    take(&a.off_yg, prm->ckpt_stride > 0 ? 3 * (size_t)ngmax * nmom + (size_t)nrg * NB : 0);
    return off * sizeof(double);
  };
  int CH = 0;
  size_t bytes = 0, cap_used = 0;
  size_t max_dyn = 0;
  if ((rc = max_dyn_smem(n, &max_dyn)) != TP_OK) return fail(rc);
  // right-hand sides split over the cluster: rs CTAs, each owning a slice of
  // every group's right-hand sides (automatic: 16 or more per CTA; at 3D
  // p = 3 with 64 right-hand sides, 4 CTAs of 16 sweep 1.6x faster than 8 of 8)
  int rs = prm->rhs_split;
  if (rs == 0) {
    rs = 1;
    for (int r : {8, 4, 2})
      if (rs == 1 && ctx->nrhs % r == 0 && ctx->nrhs / r >= 16) rs = r;
  }
  if (!(rs == 1 || rs == 2 || rs == 4 || rs == 8) || ctx->nrhs % rs != 0) {
    tp::set_error("tp_create: rhs_split must be 0, 1, 2, 4 or 8 and divide nrhs");
    return fail(TP_ERR_ARG);
  }
  // the most right-hand sides per group (a divisor of nrhs, a multiple of rs)
  // whose plan fits; the plan holds one CTA's nrg = group / rs of them
  int grp = 0;
  // tensor-core contractions (mixed precision, split right-hand sides): a
  // first search with their staging, over chunks that are multiples of the
  // MMA's K step of 16 points and at most 48 points (the level sums of
  // 48 x 5 digit products of at most 2^16 stay below 2^24), with at most 96
  // rows (right-hand sides x components: the outflow's five level sums of
  // that many columns fill the 512 tensor-memory columns) and 32 basis
  // functions.  The CTA holds all 512 columns: its shared-memory request is
  // raised above half the SM's, so that no second CTA shares the SM.
  int smem_sm = 0, dev_ = 0;
  size_t stat_smem = 0;
  TP_CUDA_OK(cudaGetDevice(&dev_));
  TP_CUDA_OK(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev_));
  TP_CUDA_OK(n == 1 ? tp::layer_static_smem_d1(&stat_smem) : n == 2 ? tp::layer_static_smem_d2(&stat_smem)
                                                                     : tp::layer_static_smem_d3(&stat_smem));
  const bool tc_want = prm->tensor_cores >= 0 && ctx->mixed && rs > 1 && nb <= 32 &&
                       (ctx->nrhs / rs) * C <= 96;
  for (int pass = 0; pass < 2 && CH == 0; ++pass) {
    tc_try = tc_want && pass == 0;
    if (!tc_want && pass == 0) continue;
    for (grp = ctx->nrhs; grp >= 1 && CH == 0; --grp) {
      if (ctx->nrhs % grp || grp % rs) continue;
      nrg = grp / rs;
      if (tc_try && nrg * C > 96) continue;
      for (size_t cap : {kTwoPerSmSmem, max_dyn}) {
        for (int ch : {48, 32, 16, 8}) {
          if (CH != 0 || plan(ch, 0) > cap) continue;
          if (tc_try && (ch % 16 != 0 || ch * tp::kTcSlices * 65536 >= (1 << 24))) continue;
          CH = ch;
        }
        if (CH) {
          cap_used = cap;
          break;
        }
      }
      if (CH) break;
    }
  }
  if (CH == 0) {
    tp::set_error("tp_create: shared-memory plan does not fit (nb/nrhs too large)");
    return fail(TP_ERR_UNSUPPORTED);
  }
  // the rest of the budget keeps the top U-values of up to `keep` points per
  // CTA (a slice that fits skips their second evaluation in the outflow)
  // (split right-hand sides evaluate the top U-values of every point again: no keep buffer)
  int keep = rs > 1 ? 0 : (int)std::min<size_t>((cap_used - plan(CH, 0)) / ((size_t)(nb + 1) * sizeof(double)),
                                                (size_t)pmax * Q);
  while (keep > 0 && plan(CH, keep) > cap_used) --keep;
  bytes = plan(CH, keep);
  // one CTA per SM with the tensor-core contractions (it holds all 512 columns)
  if (tc_try) bytes = std::max(bytes, std::min(max_dyn, (size_t)smem_sm / 2 + 1024 - stat_smem));
  a.CH = CH;
  a.keep_pts = keep;
  a.nrhs = nrg;
  a.rsplit = rs > 1 ? 1 : 0;
  a.tc = tc_try ? 1 : 0;
  a.tc_cols = tc_try ? tp::tc_cols_max : 0;
  ctx->tc_used = tc_try;
  ctx->rsplit_cs = rs;
  ctx->nrhs_g = grp;
  ctx->rhs_groups = ctx->nrhs / grp;
  if (ctx->rhs_groups > 1 && cudaMalloc(&ctx->d_tau_save, T.nv * sizeof(double)) != cudaSuccess) {
    tp::set_error("tp_create: out of device memory");
    return fail(TP_ERR_OOM);
  }
  ctx->args_adj = a;
  ctx->args_adj.front = ctx->d_adj;
  ctx->args_adj.tau = ctx->d_tau_adj;
  ctx->args_adj.gD = nullptr;
  ctx->args_adj.diss = nullptr;
  ctx->smem_bytes = bytes;
  rc = set_smem_attr(n, max_dyn);
  if (rc) return fail(rc);
  {
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) == cudaSuccess && nsm > 0)
      ctx->n_sm = nsm;
    const double avg_pts = (double)T.star_el.size() / (double)T.nv * Q;
    int cs = 1;
    while (cs < 8 && avg_pts / (2.0 * cs) >= 32.0) cs *= 2;
    ctx->max_cs = cs;
  }
  {
    const double avg_star = (double)T.star_el.size() / (double)T.nv;
    const int key[5] = {n, ctx->p, ctx->nrhs, ctx->mixed ? 1 : 0, (int)std::lround(avg_star)};
    std::copy(key, key + 5, ctx->tune_key);
  }
  if (ctx->persistent) {
    int cs = ctx->max_cs;
    bool sched_dataflow = true;
    if (tuned_lookup(ctx->tune_key, &cs, &sched_dataflow)) ctx->persistent = sched_dataflow;
    if (rs > 1) cs = rs;   // the cluster is the right-hand-side split
    if (ctx->persistent && set_persist_cs(ctx, cs) != TP_OK) ctx->persistent = false;   // one launch per level
  }
  if (cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    tp::set_error("tp_create: stream creation failed");
    return fail(TP_ERR_CUDA);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    tp::set_error("tp_create: device error during set-up");
    return fail(TP_ERR_CUDA);
  }
  *out = ctx;
  return TP_OK;
}

extern "C" int tp_ctx_info(const tp_ctx* ctx, int64_t* n_front, int32_t* n_comp, int64_t* n_bnd,
                           int32_t* n_levels) {
  if (!ctx) {
    tp::set_error("tp_ctx_info: null context");
    return TP_ERR_ARG;
  }
  if (n_front) *n_front = ctx->ne * ctx->Q;
  if (n_comp) *n_comp = ctx->C;
  if (n_bnd) *n_bnd = ctx->n_bnd;
  if (n_levels) *n_levels = ctx->n_levels;
  return TP_OK;
}

extern "C" int tp_ctx_schedule(const tp_ctx* ctx, int32_t* dataflow, int32_t* cluster, int32_t* rhs_split,
                               int32_t* rhs_groups) {
  if (!ctx) {
    tp::set_error("tp_ctx_schedule: null context");
    return TP_ERR_ARG;
  }
  if (dataflow) *dataflow = ctx->persistent ? 1 : 0;
  if (cluster) *cluster = ctx->persistent ? ctx->persist_cs : ctx->max_cs;
  if (rhs_split) *rhs_split = ctx->rsplit_cs;
  if (rhs_groups) *rhs_groups = ctx->rhs_groups;
  return TP_OK;
}

extern "C" int tp_ctx_tensor_cores(const tp_ctx* ctx, int32_t* used) {
  if (!ctx || !used) {
    tp::set_error("tp_ctx_tensor_cores: null argument");
    return TP_ERR_ARG;
  }
  *used = ctx->tc_used ? 1 : 0;
  return TP_OK;
}

extern "C" int tp_front_points(const tp_ctx* ctx, double* xq, double* wq) {
  if (!ctx) {
    tp::set_error("tp_front_points: null context");
    return TP_ERR_ARG;
  }
  const tp::Topology& T = ctx->topo;
  const int n = ctx->dim, Q = ctx->Q;
  for (int64_t k = 0; k < T.ne; ++k) {
    const int32_t* el = &T.elems[k * (n + 1)];
    double e[3][3];
    for (int i = 0; i < n; ++i)
      for (int d = 0; d < n; ++d) e[i][d] = T.X[(int64_t)el[i + 1] * n + d] - T.X[(int64_t)el[0] * n + d];
    double det = (n == 1) ? e[0][0]
               : (n == 2) ? e[0][0] * e[1][1] - e[0][1] * e[1][0]
                          : e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                                e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                                e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
    for (int q = 0; q < Q; ++q) {
      if (xq)
        for (int d = 0; d < n; ++d) {
          double s = 0.0;
          for (int i = 0; i <= n; ++i) s += ctx->rule.bary[q * (n + 1) + i] * T.X[(int64_t)el[i] * n + d];
          xq[(k * Q + q) * n + d] = s;
        }
      if (wq) wq[k * Q + q] = ctx->rule.w[q] * std::fabs(det);
    }
  }
  return TP_OK;
}

extern "C" int tp_boundary_points(const tp_ctx* ctx, double* xt) {
  if (!ctx || (!xt && ctx->n_bnd > 0)) {
    tp::set_error("tp_boundary_points: null argument");
    return TP_ERR_ARG;
  }
  std::copy(ctx->bnd_xt.begin(), ctx->bnd_xt.end(), xt);
  return TP_OK;
}

extern "C" int tp_boundary_kinds(const tp_ctx* ctx, double* nrm, int8_t* kind) {
  if (!ctx) {
    tp::set_error("tp_boundary_kinds: null context");
    return TP_ERR_ARG;
  }
  if (nrm) std::copy(ctx->bnd_nrm.begin(), ctx->bnd_nrm.end(), nrm);
  if (kind) std::copy(ctx->bnd_kind.begin(), ctx->bnd_kind.end(), kind);
  return TP_OK;
}

extern "C" int tp_set_state(tp_ctx* ctx, const double* d_front, const double* d_gD, void* stream) {
  if (!ctx || !d_front) {
    tp::set_error("tp_set_state: null argument");
    return TP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nfront = (size_t)ctx->nrhs * ctx->ne * ctx->Q * ctx->C;
  TP_CUDA_OK(cudaMemcpyAsync(ctx->d_front, d_front, nfront * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (ctx->d_front0)   // the wave-speed gradient sweeps forward again from here
    TP_CUDA_OK(cudaMemcpyAsync(ctx->d_front0, d_front, nfront * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TP_CUDA_OK(cudaMemsetAsync(ctx->d_tau, 0, ctx->nv * sizeof(double), st));
  TP_CUDA_OK(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  TP_CUDA_OK(cudaMemsetAsync(ctx->d_info, 0, sizeof(long long), st));
  if (ctx->d_diss) TP_CUDA_OK(cudaMemsetAsync(ctx->d_diss, 0, (size_t)ctx->nrhs * sizeof(double), st));
  TP_CUDA_OK(cudaMemsetAsync(ctx->d_stats, 0, (tp::kMaxRefine + 2) * sizeof(unsigned long long), st));
  if (ctx->d_probe_out)
    TP_CUDA_OK(cudaMemsetAsync(ctx->d_probe_out, 0,
                               (size_t)ctx->nrhs * ctx->n_probe_t * ctx->n_probe * sizeof(double), st));
  if (ctx->n_bnd > 0) {
    if (d_gD) {
      TP_CUDA_OK(cudaMemcpyAsync(ctx->d_gD, d_gD, (size_t)ctx->nrhs * ctx->n_bnd * sizeof(double),
                                 cudaMemcpyDeviceToDevice, st));
      ctx->args.gD = ctx->d_gD;
    } else {
      TP_CUDA_OK(cudaMemsetAsync(ctx->d_gD, 0, (size_t)ctx->nrhs * ctx->n_bnd * sizeof(double), st));
      ctx->args.gD = ctx->d_gD;
    }
  }
  ctx->last_stream = st;
  return TP_OK;
}

extern "C" int tp_set_probes(tp_ctx* ctx, int32_t n_pts, const double* xq, int32_t n_t, const double* times) {
  if (!ctx || n_pts < 0 || n_t < 0 || (n_pts > 0 && !xq) || (n_t > 0 && !times)) {
    tp::set_error("tp_set_probes: invalid argument");
    return TP_ERR_ARG;
  }
  const tp::Topology& T = ctx->topo;
  const int n = ctx->dim, NV = n + 1;
  for (void* g : ctx->probe_allocs) cudaFree(g);
  ctx->probe_allocs.clear();
  ctx->d_probe_out = nullptr;
  ctx->n_probe = ctx->n_probe_t = 0;
  for (KArgs* a : {&ctx->args, &ctx->args_adj}) {
    a->probe_ptr = nullptr;
    a->probe_out = nullptr;
  }
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);   // the graphs hold the old arguments
  ctx->graphs.clear();
  if (n_pts == 0 || n_t == 0) return TP_OK;
  for (int k = 1; k < n_t; ++k)
    if (!(times[k] > times[k - 1])) {
      tp::set_error("tp_set_probes: output times must increase");
      return TP_ERR_ARG;
    }
  // the element of every point (barycentric coordinates >= -1e-12) and its coordinates there
  std::vector<int> pel(n_pts, -1);
  std::vector<double> pbary((size_t)n_pts * NV);
  for (int j = 0; j < n_pts; ++j) {
    for (int64_t k = 0; k < T.ne && pel[j] < 0; ++k) {
      const int32_t* el = &T.elems[(size_t)k * NV];
      double e[3][3] = {}, rhs[3] = {}, lam[4] = {};
      for (int i = 0; i < n; ++i) {
        for (int d = 0; d < n; ++d) e[d][i] = T.X[(size_t)el[i + 1] * n + d] - T.X[(size_t)el[0] * n + d];
      }
      for (int d = 0; d < n; ++d) rhs[d] = xq[(size_t)j * n + d] - T.X[(size_t)el[0] * n + d];
      // solve e lam[1..n] = rhs by Cramer's rule (n <= 3)
      auto det3 = [&](double m[3][3]) {
        if (n == 1) return m[0][0];
        if (n == 2) return m[0][0] * m[1][1] - m[0][1] * m[1][0];
        return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) - m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
               m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
      };
      const double D = det3(e);
      double s = 0.0;
      for (int i = 0; i < n; ++i) {
        double m[3][3];
        for (int r = 0; r < 3; ++r)
          for (int c2 = 0; c2 < 3; ++c2) m[r][c2] = (c2 == i) ? rhs[r] : e[r][c2];
        lam[i + 1] = det3(m) / D;
        s += lam[i + 1];
      }
      lam[0] = 1.0 - s;
      bool in = true;
      for (int i = 0; i <= n; ++i) in = in && lam[i] >= -1e-12;
      if (in) {
        pel[j] = (int)k;
        for (int i = 0; i <= n; ++i) pbary[(size_t)j * NV + i] = lam[i];
      }
    }
    if (pel[j] < 0) {
      tp::set_error("tp_set_probes: point " + std::to_string(j) + " lies in no element of the mesh");
      return TP_ERR_ARG;
    }
  }
  // replay the tents: the sample (x_j, t_k) belongs to the tent whose
  // bottom and top fronts enclose it on x_j's element, t_bot(x_j) <= t_k <
  // t_top(x_j) (at the final time, the tent whose top reaches it)
  std::vector<std::vector<int>> at_el(T.ne);
  for (int j = 0; j < n_pts; ++j) at_el[pel[j]].push_back(j);
  std::vector<double> tau(T.nv, 0.0);
  const double Tf = ctx->T_final;
  std::vector<int32_t> ptr(ctx->ntents + 1, 0), sj, sk, sslot;
  for (int64_t it = 0; it < ctx->ntents; ++it) {
    const int v = ctx->tent_vert_h[it];
    const double ttop = ctx->tent_ttop_h[it];
    for (int e = T.star_ptr[v]; e < T.star_ptr[v + 1]; ++e) {
      const int K = ctx->star_sorted[e];
      for (int j : at_el[K]) {
        double tb = 0.0, tt = 0.0;
        for (int i = 0; i < NV; ++i) {
          const int w = T.elems[(size_t)K * NV + i];
          const double l = pbary[(size_t)j * NV + i];
          tb += l * tau[w];
          tt += l * (w == v ? ttop : tau[w]);
        }
        for (int k = 0; k < n_t; ++k) {
          const double t = times[k];
          if ((tb <= t && t < tt) || (t == Tf && tb < tt && tt == Tf)) {
            sj.push_back(j);
            sk.push_back(k);
            sslot.push_back(e - T.star_ptr[v]);
          }
        }
      }
    }
    tau[v] = ttop;
    ptr[it + 1] = (int32_t)sj.size();
  }
  std::vector<double> tv(times, times + n_t);
  int *dptr = nullptr, *dj = nullptr, *dk = nullptr, *dsl = nullptr;
  double *dbary = nullptr, *dt = nullptr;
  int rc = TP_OK;
  auto up = [&](auto** d, const auto& h) {
    int r = upload(d, h);
    if (r == TP_OK && *d) ctx->probe_allocs.push_back((void*)*d);
    return r;
  };
  if ((rc = up(&dptr, ptr)) || (rc = up(&dj, sj)) || (rc = up(&dk, sk)) || (rc = up(&dsl, sslot)) ||
      (rc = up(&dbary, pbary)) || (rc = up(&dt, tv)))
    return rc;
  const size_t nout = (size_t)ctx->nrhs * n_t * n_pts;
  if (cudaMalloc(&ctx->d_probe_out, nout * sizeof(double)) != cudaSuccess) {
    tp::set_error("tp_set_probes: device allocation failed");
    return TP_ERR_OOM;
  }
  ctx->probe_allocs.push_back(ctx->d_probe_out);
  TP_CUDA_OK(cudaMemset(ctx->d_probe_out, 0, nout * sizeof(double)));
  ctx->n_probe = n_pts;
  ctx->n_probe_t = n_t;
  KArgs& a = ctx->args;
  a.probe_ptr = dptr;
  a.probe_j = dj;
  a.probe_k = dk;
  a.probe_slot = dsl;
  a.probe_bary = dbary;
  a.probe_t = dt;
  a.n_probe = n_pts;
  a.n_probe_t = n_t;
  a.probe_out = ctx->d_probe_out;
  return TP_OK;
}

extern "C" int tp_get_probes(const tp_ctx* ctx, double* d_out, void* stream) {
  if (!ctx || !d_out || !ctx->d_probe_out) {
    tp::set_error("tp_get_probes: null argument or no point outputs set");
    return TP_ERR_ARG;
  }
  TP_CUDA_OK(cudaMemcpyAsync(d_out, ctx->d_probe_out,
                             (size_t)ctx->nrhs * ctx->n_probe_t * ctx->n_probe * sizeof(double),
                             cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
  return TP_OK;
}

extern "C" int tp_set_front(tp_ctx* ctx, const double* d_front, const double* d_tau, void* stream) {
  if (!ctx || !d_front || !d_tau) {
    tp::set_error("tp_set_front: null argument");
    return TP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nfront = (size_t)ctx->nrhs * ctx->ne * ctx->Q * ctx->C;
  TP_CUDA_OK(cudaMemcpyAsync(ctx->d_front, d_front, nfront * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TP_CUDA_OK(cudaMemcpyAsync(ctx->d_tau, d_tau, ctx->nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
  ctx->last_stream = st;
  return TP_OK;
}

namespace {
void drop_graphs(tp_ctx* ctx) {   // captured graphs hold the kernel arguments by value
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
  if (ctx->adj_graph) cudaGraphExecDestroy(ctx->adj_graph);
  ctx->adj_graph = nullptr;
}
}  // namespace

extern "C" int tp_set_limits(tp_ctx* ctx, int64_t max_polls, int32_t max_refine) {
  if (!ctx) {
    tp::set_error("tp_set_limits: null context");
    return TP_ERR_ARG;
  }
  const long long spin = max_polls > 0 ? (long long)max_polls : tp::kMaxSpin;
  const int ref = max_refine >= 0 ? std::min<int>(max_refine, tp::kMaxRefine) : tp::kMaxRefine;
  for (KArgs* a : {&ctx->args, &ctx->args_adj}) {
    a->max_spin = spin;
    a->max_refine = ref;
  }
  drop_graphs(ctx);
  return TP_OK;
}

extern "C" int tp_inject_wait(tp_ctx* ctx, int64_t tent, int32_t extra) {
  if (!ctx || tent < 0 || tent >= ctx->ntents || extra < 0) {
    tp::set_error("tp_inject_wait: invalid argument");
    return TP_ERR_ARG;
  }
  const int d0 = ctx->dep_ptr_h[tent], d1 = ctx->dep_ptr_h[tent + 1];
  if (d1 <= d0) {
    tp::set_error("tp_inject_wait: tent " + std::to_string(tent) + " waits for no earlier tent");
    return TP_ERR_ARG;
  }
  std::vector<int32_t> need(ctx->dep_need_h.begin() + d0, ctx->dep_need_h.begin() + d1);
  for (auto& x : need) x += extra;
  TP_CUDA_OK(cudaMemcpy(ctx->d_dep_need + d0, need.data(), need.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  return TP_OK;
}

extern "C" int tp_solve_stats(tp_ctx* ctx, int64_t* direct_lu, int64_t* hist, int32_t nhist) {
  if (!ctx || (hist && nhist < 0)) {
    tp::set_error("tp_solve_stats: invalid argument");
    return TP_ERR_ARG;
  }
  unsigned long long h[tp::kMaxRefine + 2];
  TP_CUDA_OK(cudaStreamSynchronize(ctx->last_stream));
  TP_CUDA_OK(cudaMemcpy(h, ctx->d_stats, sizeof(h), cudaMemcpyDeviceToHost));
  if (direct_lu) *direct_lu = (int64_t)h[0];
  if (hist)
    for (int k = 0; k < nhist; ++k) hist[k] = k <= tp::kMaxRefine ? (int64_t)h[1 + k] : 0;
  return TP_OK;
}

extern "C" int tp_solve_layer(tp_ctx* ctx, int32_t level, void* stream) {
  if (!ctx || level < 1 || level > ctx->n_levels) {
    tp::set_error("tp_solve_layer: level out of range");
    return TP_ERR_ARG;
  }
  ctx->last_stream = (cudaStream_t)stream;
  return launch_level(ctx, level, (cudaStream_t)stream);
}

namespace {
__global__ void k_sweep_setup(const int* vert, int t_begin, int cs, int* done, int* queue) {
  // completed tents before the range, per vertex (each tent counts once per
  // CTA of its cluster); queue head at the range start
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < t_begin; t += gridDim.x * blockDim.x)
    atomicAdd(done + vert[t], cs);
  if (blockIdx.x == 0 && threadIdx.x == 0) *queue = t_begin;
}
}  // namespace

extern "C" int tp_advance(tp_ctx* ctx, int32_t level_begin, int32_t level_end, void* stream) {
  if (!ctx || level_begin < 1 || level_end > ctx->n_levels + 1 || level_end < level_begin) {
    tp::set_error("tp_advance: level range out of bounds");
    return TP_ERR_ARG;
  }
  if (level_end == level_begin) return TP_OK;
  auto key = std::make_pair((int)level_begin, (int)level_end);
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    cudaGraph_t g = nullptr;
    TP_CUDA_OK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = TP_OK;
    // right-hand-side groups one after the other, each from the front times
    // at the start of the range
    const size_t tau_bytes = ctx->nv * sizeof(double);
    cudaError_t e0 = cudaSuccess;
    if (ctx->rhs_groups > 1)
      e0 = cudaMemcpyAsync(ctx->d_tau_save, ctx->d_tau, tau_bytes, cudaMemcpyDeviceToDevice, ctx->cap_stream);
    for (int k = 0; k < ctx->rhs_groups && rc == TP_OK; ++k) {
      if (k > 0 && e0 == cudaSuccess)
        e0 = cudaMemcpyAsync(ctx->d_tau, ctx->d_tau_save, tau_bytes, cudaMemcpyDeviceToDevice, ctx->cap_stream);
      if (e0 != cudaSuccess) {
        tp::set_error(std::string("tp_advance: CUDA error ") + cudaGetErrorString(e0));
        rc = TP_ERR_CUDA;
        break;
      }
      if (ctx->persistent) {
        const int t_begin = (int)ctx->level_ptr[level_begin - 1], t_end = (int)ctx->level_ptr[level_end - 1];
        KArgs a = group_args(ctx, ctx->args, k);
        a.tent_end = t_end;
        cudaError_t e = cudaMemsetAsync(ctx->d_done, 0, ctx->nv * sizeof(int), ctx->cap_stream);
        if (e == cudaSuccess) {
          k_sweep_setup<<<std::max(1, std::min(1024, (t_begin + 255) / 256)), 256, 0, ctx->cap_stream>>>(
              ctx->args.tent_v, t_begin, ctx->persist_cs, ctx->d_done, ctx->d_queue);
          e = cudaGetLastError();
        }
        if (e == cudaSuccess)
          e = launch_layer(ctx, a, ctx->persist_clusters, ctx->persist_cs, 0, ctx->cap_stream, ctx->mixed ? 1 : 0, true);
        if (e != cudaSuccess) {
          tp::set_error(std::string("tp_advance: CUDA error ") + cudaGetErrorString(e));
          rc = TP_ERR_CUDA;
        }
      } else {
        for (int32_t L = level_begin; L < level_end && rc == TP_OK; ++L)
          rc = launch_level(ctx, L, ctx->cap_stream, false, k);
      }
    }
    cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
    if (rc != TP_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    TP_CUDA_OK(e);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    TP_CUDA_OK(e);
    it = ctx->graphs.emplace(key, ex).first;
  }
  ctx->last_stream = (cudaStream_t)stream;
  TP_CUDA_OK(cudaGraphLaunch(it->second, (cudaStream_t)stream));
  return TP_OK;
}

namespace {
__global__ void k_fill(double* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
}  // namespace

namespace {

// the buffers of the wave-speed gradient, allocated on its first use
int grad_buffers(tp_ctx* ctx) {
  if (ctx->d_work) return TP_OK;
  const size_t nfront = (size_t)ctx->nrhs * ctx->ne * ctx->Q * ctx->C;
  const int S = ctx->ckpt_stride, nseg = (ctx->n_levels + S - 1) / S;
  int64_t most = 0;   // tents of the largest segment
  for (int sg = 0; sg < nseg; ++sg) {
    const int L0 = 1 + sg * S, L1 = std::min(L0 + S, ctx->n_levels + 1);
    most = std::max<int64_t>(most, ctx->level_ptr[L1 - 1] - ctx->level_ptr[L0 - 1]);
  }
  ctx->xs_stride = (long long)ctx->nrhs * ctx->args.ngmax * ctx->nb;
  ctx->xsave_tents = most;
  if (cudaMalloc(&ctx->d_work, nfront * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_tau_work, ctx->nv * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_ckpt, (size_t)nseg * nfront * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_ckpt_tau, (size_t)nseg * ctx->nv * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_snap, (size_t)S * nfront * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&ctx->d_xsave, (size_t)std::max<int64_t>(1, most) * ctx->xs_stride * sizeof(double)) != cudaSuccess) {
    for (double** g : {&ctx->d_work, &ctx->d_tau_work, &ctx->d_ckpt, &ctx->d_ckpt_tau, &ctx->d_snap, &ctx->d_xsave}) {
      cudaFree(*g);
      *g = nullptr;
    }
    cudaGetLastError();
    tp::set_error("tp_adjoint: device allocation of the checkpoints failed");
    return TP_ERR_OOM;
  }
  return TP_OK;
}

// reverse sweep with the wave-speed gradient: forward from the initial state
// of the last tp_set_state keeping a checkpoint (front and times) at the start
// of every segment of ckpt_stride levels; then segment by segment from the
// last: forward again from its checkpoint keeping the front before each level
// and every tent's solution, and the reverse levels of the segment, each
// adding its tents' dJ/dc
int adjoint_with_gradient(tp_ctx* ctx, double* d_dJ_dc, cudaStream_t st) {
  const size_t nfront = (size_t)ctx->nrhs * ctx->ne * ctx->Q * ctx->C;
  const size_t fb = nfront * sizeof(double), tb = ctx->nv * sizeof(double);
  const int S = ctx->ckpt_stride, nseg = (ctx->n_levels + S - 1) / S;
  int rc = grad_buffers(ctx);
  if (rc != TP_OK) return rc;
  TP_CUDA_OK(cudaMemsetAsync(d_dJ_dc, 0, ctx->ne * sizeof(double), st));
  KArgs af = ctx->args;   // forward on the work front
  af.front = ctx->d_work;
  af.tau = ctx->d_tau_work;
  af.diss = nullptr;
  af.xsave = nullptr;
  TP_CUDA_OK(cudaMemcpyAsync(ctx->d_work, ctx->d_front0, fb, cudaMemcpyDeviceToDevice, st));
  TP_CUDA_OK(cudaMemsetAsync(ctx->d_tau_work, 0, tb, st));
  for (int sg = 0; sg < nseg; ++sg) {
    const int L0 = 1 + sg * S, L1 = std::min(L0 + S, ctx->n_levels + 1);
    TP_CUDA_OK(cudaMemcpyAsync(ctx->d_ckpt + (size_t)sg * nfront, ctx->d_work, fb, cudaMemcpyDeviceToDevice, st));
    TP_CUDA_OK(cudaMemcpyAsync(ctx->d_ckpt_tau + (size_t)sg * ctx->nv, ctx->d_tau_work, tb, cudaMemcpyDeviceToDevice, st));
    for (int L = L0; L < L1; ++L)
      if ((rc = launch_level_with(ctx, L, st, false, af)) != TP_OK) return rc;
  }
  KArgs aa = ctx->args_adj;   // reverse, with the forward boundary data and the gradient
  aa.gD = ctx->args.gD;
  aa.dJdc = d_dJ_dc;
  aa.xsave = ctx->d_xsave;
  aa.xs_stride = ctx->xs_stride;
  af.xsave = ctx->d_xsave;
  af.xs_stride = ctx->xs_stride;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int L0 = 1 + sg * S, L1 = std::min(L0 + S, ctx->n_levels + 1);
    af.xbase = aa.xbase = ctx->level_ptr[L0 - 1];
    TP_CUDA_OK(cudaMemcpyAsync(ctx->d_work, ctx->d_ckpt + (size_t)sg * nfront, fb, cudaMemcpyDeviceToDevice, st));
    TP_CUDA_OK(cudaMemcpyAsync(ctx->d_tau_work, ctx->d_ckpt_tau + (size_t)sg * ctx->nv, tb, cudaMemcpyDeviceToDevice, st));
    for (int L = L0; L < L1; ++L) {
      TP_CUDA_OK(cudaMemcpyAsync(ctx->d_snap + (size_t)(L - L0) * nfront, ctx->d_work, fb, cudaMemcpyDeviceToDevice, st));
      if ((rc = launch_level_with(ctx, L, st, false, af)) != TP_OK) return rc;
    }
    for (int L = L1 - 1; L >= L0; --L) {
      aa.front_fwd = ctx->d_snap + (size_t)(L - L0) * nfront;
      if ((rc = launch_level_with(ctx, L, st, true, aa)) != TP_OK) return rc;
    }
  }
  return TP_OK;
}

}  // namespace

extern "C" int tp_adjoint(tp_ctx* ctx, const double* d_lambda_T, double* d_dJ_dc, double* d_lambda_0,
                          void* stream) {
  if (!ctx || !d_lambda_T || !d_lambda_0) {
    tp::set_error("tp_adjoint: null argument");
    return TP_ERR_ARG;
  }
  if (d_dJ_dc && ctx->ckpt_stride <= 0) {
    tp::set_error("tp_adjoint: the wave-speed gradient needs a context created with ckpt_stride > 0");
    return TP_ERR_ARG;
  }
  if (d_dJ_dc && ctx->rhs_groups > 1) {
    tp::set_error("tp_adjoint: the wave-speed gradient needs every right-hand side in one group");
    return TP_ERR_UNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nfront = (size_t)ctx->nrhs * ctx->ne * ctx->Q * ctx->C;
  if (!ctx->d_adj) {   // the adjoint state, on first use
    if (cudaMalloc(&ctx->d_adj, nfront * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&ctx->d_tau_adj, ctx->nv * sizeof(double)) != cudaSuccess) {
      cudaFree(ctx->d_adj);
      ctx->d_adj = nullptr;
      cudaGetLastError();
      tp::set_error("tp_adjoint: device allocation of the adjoint state failed");
      return TP_ERR_OOM;
    }
    ctx->args_adj.front = ctx->d_adj;
    ctx->args_adj.tau = ctx->d_tau_adj;
  }
  TP_CUDA_OK(cudaMemcpyAsync(ctx->d_adj, d_lambda_T, nfront * sizeof(double), cudaMemcpyDeviceToDevice, st));
  k_fill<<<(unsigned)std::min<int64_t>(1024, (ctx->nv + 255) / 256), 256, 0, st>>>(ctx->d_tau_adj, ctx->nv,
                                                                                 ctx->T_final);
  TP_CUDA_OK(cudaGetLastError());
  if (d_dJ_dc && ctx->n_levels > 0) {
    const int rc = adjoint_with_gradient(ctx, d_dJ_dc, st);
    if (rc != TP_OK) return rc;
  } else if (d_dJ_dc) {
    TP_CUDA_OK(cudaMemsetAsync(d_dJ_dc, 0, ctx->ne * sizeof(double), st));
  } else if (ctx->n_levels > 0) {
    if (!ctx->adj_graph) {
      cudaGraph_t g = nullptr;
      TP_CUDA_OK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
      int rc = TP_OK;
      for (int k = 0; k < ctx->rhs_groups && rc == TP_OK; ++k) {   // groups from the final time each
        if (k > 0) {
          k_fill<<<(unsigned)std::min<int64_t>(1024, (ctx->nv + 255) / 256), 256, 0, ctx->cap_stream>>>(
              ctx->d_tau_adj, ctx->nv, ctx->T_final);
          if (cudaGetLastError() != cudaSuccess) rc = TP_ERR_CUDA;
        }
        for (int32_t L = ctx->n_levels; L >= 1 && rc == TP_OK; --L) rc = launch_level(ctx, L, ctx->cap_stream, true, k);
      }
      cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
      if (rc != TP_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      TP_CUDA_OK(e);
      e = cudaGraphInstantiate(&ctx->adj_graph, g, 0);
      cudaGraphDestroy(g);
      TP_CUDA_OK(e);
    }
    TP_CUDA_OK(cudaGraphLaunch(ctx->adj_graph, st));
  }
  TP_CUDA_OK(cudaMemcpyAsync(d_lambda_0, ctx->d_adj, nfront * sizeof(double), cudaMemcpyDeviceToDevice, st));
  ctx->last_stream = st;
  return TP_OK;
}

extern "C" int tp_autotune(tp_ctx* ctx, void* stream, int32_t* chosen, double* best_ms) {
  if (!ctx) {
    tp::set_error("tp_autotune: null context");
    return TP_ERR_ARG;
  }
  if (ctx->n_levels < 1) return TP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nfront = (size_t)ctx->nrhs * ctx->ne * ctx->Q * ctx->C;
  double *save_f = nullptr, *save_t = nullptr;
  if (cudaMalloc(&save_f, nfront * sizeof(double)) != cudaSuccess ||
      cudaMalloc(&save_t, ctx->nv * sizeof(double)) != cudaSuccess) {
    cudaFree(save_f);
    tp::set_error("tp_autotune: allocation failed");
    return TP_ERR_OOM;
  }
  int rc = TP_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemcpyAsync(save_f, ctx->d_front, nfront * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(save_t, ctx->d_tau, ctx->nv * sizeof(double), cudaMemcpyDeviceToDevice, st);
  // candidates: 0 = one launch per level, else the dataflow sweep with clusters of that size
  const int cand[5] = {0, 1, 2, 4, 8};
  int best = -1;
  float best_t = 3.4e38f;
  for (int ci = 0; ci < 5 && rc == TP_OK; ++ci) {
    const int c = cand[ci];
    if (c == 0) {
      ctx->persistent = false;
    } else {
      if ((ctx->rsplit_cs > 1 ? c != ctx->rsplit_cs : c > ctx->max_cs * 2) || set_persist_cs(ctx, c) != TP_OK)
        continue;
      ctx->persistent = true;
    }
    for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
    ctx->graphs.clear();
    float t = 0.f;
    for (int rep = 0; rep < 2 && rc == TP_OK; ++rep) {
      cudaMemcpyAsync(ctx->d_front, save_f, nfront * sizeof(double), cudaMemcpyDeviceToDevice, st);
      cudaMemcpyAsync(ctx->d_tau, save_t, ctx->nv * sizeof(double), cudaMemcpyDeviceToDevice, st);
      cudaEventRecord(e0, st);
      rc = tp_advance(ctx, 1, ctx->n_levels + 1, stream);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = TP_ERR_CUDA;
      cudaEventElapsedTime(&t, e0, e1);
    }
    if (rc == TP_OK && t < best_t) {
      best_t = t;
      best = c;
    }
  }
  if (rc == TP_OK && best >= 0) {
    ctx->persistent = best > 0;
    if (best > 0) set_persist_cs(ctx, best);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[std::vector<int>(ctx->tune_key, ctx->tune_key + 5)] = {best > 0 ? best : 1, best > 0};
  }
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
  cudaMemcpyAsync(ctx->d_front, save_f, nfront * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(ctx->d_tau, save_t, ctx->nv * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaStreamSynchronize(st);
  cudaFree(save_f);
  cudaFree(save_t);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (chosen) *chosen = best;
  if (best_ms) *best_ms = best_t;
  ctx->last_stream = st;
  return rc;
}

extern "C" int tp_energy(tp_ctx* ctx, double* d_out, void* stream) {
  if (!ctx || !d_out) {
    tp::set_error("tp_energy: null argument");
    return TP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 grid(ctx->energy_blocks, ctx->nrhs);
  switch (ctx->dim) {
    case 1: k_energy_partial<1><<<grid, kThreads, 0, st>>>(ctx->args, ctx->d_partial, ctx->energy_blocks); break;
    case 2: k_energy_partial<2><<<grid, kThreads, 0, st>>>(ctx->args, ctx->d_partial, ctx->energy_blocks); break;
    default: k_energy_partial<3><<<grid, kThreads, 0, st>>>(ctx->args, ctx->d_partial, ctx->energy_blocks); break;
  }
  TP_CUDA_OK(cudaGetLastError());
  k_energy_final<<<(ctx->nrhs + 127) / 128, 128, 0, st>>>(ctx->d_partial, ctx->energy_blocks, ctx->nrhs, d_out, 2,
                                                         ctx->d_diss);
  TP_CUDA_OK(cudaGetLastError());
  ctx->last_stream = st;
  return TP_OK;
}

extern "C" int tp_get_state(const tp_ctx* ctx, double* d_front, double* d_tau, void* stream) {
  if (!ctx) {
    tp::set_error("tp_get_state: null context");
    return TP_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (d_front)
    TP_CUDA_OK(cudaMemcpyAsync(d_front, ctx->d_front,
                               (size_t)ctx->nrhs * ctx->ne * ctx->Q * ctx->C * sizeof(double),
                               cudaMemcpyDeviceToDevice, st));
  if (d_tau) TP_CUDA_OK(cudaMemcpyAsync(d_tau, ctx->d_tau, ctx->nv * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return TP_OK;
}

extern "C" int tp_sync_status(tp_ctx* ctx, int32_t* status, int64_t* info) {
  if (!ctx) {
    tp::set_error("tp_sync_status: null context");
    return TP_ERR_ARG;
  }
  TP_CUDA_OK(cudaStreamSynchronize(ctx->last_stream));
  int s = 0;
  long long i = 0;
  TP_CUDA_OK(cudaMemcpy(&s, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  TP_CUDA_OK(cudaMemcpy(&i, ctx->d_info, sizeof(long long), cudaMemcpyDeviceToHost));
  if (status) *status = s;
  if (info) *info = i;
  return TP_OK;
}

extern "C" void tp_destroy_ctx(tp_ctx* ctx) {
  if (!ctx) return;
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  for (void* p : ctx->allocs) cudaFree(p);
  cudaFree(ctx->d_front);
  cudaFree(ctx->d_tau);
  cudaFree(ctx->d_gD);
  cudaFree(ctx->d_partial);
  cudaFree(ctx->d_diss);
  cudaFree(ctx->d_stats);
  for (void* g : ctx->probe_allocs) cudaFree(g);
  for (double* g : {ctx->d_front0, ctx->d_work, ctx->d_tau_work, ctx->d_ckpt, ctx->d_ckpt_tau, ctx->d_snap, ctx->d_xsave})
    cudaFree(g);
  cudaFree(ctx->d_adj);
  cudaFree(ctx->d_queue);
  cudaFree(ctx->d_done);
  cudaFree(ctx->d_tau_adj);
  cudaFree(ctx->d_tau_save);
  if (ctx->adj_graph) cudaGraphExecDestroy(ctx->adj_graph);
  cudaFree(ctx->d_status);
  cudaFree(ctx->d_info);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  delete ctx;
}

// ===========================================================================
// Allocation-free front energy (tp_front_energy_noalloc)
//
// Some callers cannot allocate device memory when they need this number:
// applications whose framework has already reserved the free device memory in
// its own pool (a library cudaMalloc would fail or fragment that pool), and
// long-running or certified services that fix their device-memory budget at
// start-up and forbid allocations afterwards.  This entry point computes the
// same quantity as tp_energy from caller-owned arrays and keeps its only
// scratch -- the per-block partial sums -- in the fixed array below.
//
// The array is a module global: every GPU that loads libtp holds it (256 KiB)
// until the process exits.  In host code its name is only a host-side
// stand-in, so the device address is looked up once per device with
// cudaGetSymbolAddress (done by the first call on that device, which should
// therefore come before any stream capture).  Every call shares the array:
// each partial slot it reads is written earlier in the same call, so nothing
// needs clearing, but two calls that overlap on the GPU (different streams or
// threads) race on it.
// ===========================================================================
namespace {

constexpr int kNoAllocPartials = 32768;   // doubles: nrhs x blocks-per-rhs partial sums
static __device__ __align__(256) double g_noalloc_partials[kNoAllocPartials];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[kMaxDevices] = {};

int noalloc_scratch(double** out) {
  int dev = 0;
  TP_CUDA_OK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    tp::set_error("tp_front_energy_noalloc: device ordinal out of range");
    return TP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || p == nullptr) {
      tp::set_error(std::string("tp_front_energy_noalloc: cudaGetSymbolAddress failed: ") +
                    cudaGetErrorString(e));
      return TP_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return TP_OK;
}

}  // namespace

extern "C" int tp_front_energy_noalloc(int32_t dim, int64_t n_elem, int32_t Q, int32_t nrhs,
                                       const double* d_coords, const int32_t* d_elems,
                                       const double* d_c, const double* d_tau, const double* d_wref,
                                       const double* d_front, double* d_out, void* stream) {
  if (dim < 1 || dim > tp::kMaxDim || n_elem < 1 || Q < 1 || nrhs < 1 || !d_coords || !d_elems ||
      !d_c || !d_tau || !d_wref || !d_front || !d_out) {
    tp::set_error("tp_front_energy_noalloc: invalid argument");
    return TP_ERR_ARG;
  }
  if (nrhs > kNoAllocPartials) {
    tp::set_error("tp_front_energy_noalloc: nrhs = " + std::to_string(nrhs) +
                  " exceeds the fixed scratch of " + std::to_string(kNoAllocPartials) +
                  " partial sums (at most that many right-hand sides)");
    return TP_ERR_ARG;
  }
  double* partial = nullptr;
  int rc = noalloc_scratch(&partial);
  if (rc != TP_OK) return rc;
  KArgs a{};
  a.Q = Q;
  a.nrhs = nrhs;
  a.ne = n_elem;
  a.X = d_coords;
  a.elems = d_elems;
  a.cK = d_c;
  a.tau = const_cast<double*>(d_tau);
  a.wref = d_wref;
  a.front = const_cast<double*>(d_front);
  const int nblk = (int)std::min<int64_t>(
      {(int64_t)1024, (n_elem + kThreads - 1) / kThreads, (int64_t)(kNoAllocPartials / nrhs)});
  cudaStream_t st = (cudaStream_t)stream;
  const dim3 grid(nblk, nrhs);
  switch (dim) {
    case 1: k_energy_partial<1><<<grid, kThreads, 0, st>>>(a, partial, nblk); break;
    case 2: k_energy_partial<2><<<grid, kThreads, 0, st>>>(a, partial, nblk); break;
    default: k_energy_partial<3><<<grid, kThreads, 0, st>>>(a, partial, nblk); break;
  }
  TP_CUDA_OK(cudaGetLastError());
  k_energy_final<<<(nrhs + 127) / 128, 128, 0, st>>>(partial, nblk, nrhs, d_out);
  TP_CUDA_OK(cudaGetLastError());
  return TP_OK;
}

// ===========================================================================
// Arithmetic peaks of the plain ALUs (tp_measure_alu_peaks): the rooflines of
// the tent sweep are set by the binary64 pipe (binary64 path) and the
// binary32 pipe (float-float mixed path), for which no library figure exists.
// Eight independent fused multiply-add chains per thread, enough warps per SM
// to hide the pipe latency; 2 flops per fused multiply-add.
// ===========================================================================
namespace {

template <typename F>
__global__ void k_fma_chains(F* sink, int iters, F m, F c) {
  F a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (F)(threadIdx.x + j) * (F)1e-3;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
  F s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == (F)-1.25) sink[blockIdx.x] = s;   // never true; keeps the chains live
}

template <typename F>
int fma_peak(int n_sm, cudaStream_t st, double* tflops) {
  F* sink = nullptr;
  TP_CUDA_OK(cudaMalloc(&sink, 8 * n_sm * sizeof(F)));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int blocks = 8 * n_sm, threads = 256, iters = 1 << 14;
  float best = 3.4e38f;
  int rc = TP_OK;
  for (int rep = 0; rep < 4 && rc == TP_OK; ++rep) {
    cudaEventRecord(e0, st);
    k_fma_chains<F><<<blocks, threads, 0, st>>>(sink, iters, (F)0.999999, (F)1e-7);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      tp::set_error("tp_measure_alu_peaks: kernel failed");
      rc = TP_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);   // the first launch warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (rc == TP_OK) *tflops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
  return rc;
}

}  // namespace

extern "C" int tp_measure_alu_peaks(double* fp64_tflops, double* fp32_tflops, void* stream) {
  if (!fp64_tflops || !fp32_tflops) {
    tp::set_error("tp_measure_alu_peaks: null argument");
    return TP_ERR_ARG;
  }
  int dev = 0, nsm = 0;
  TP_CUDA_OK(cudaGetDevice(&dev));
  TP_CUDA_OK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  int rc = fma_peak<double>(nsm, st, fp64_tflops);
  if (rc == TP_OK) rc = fma_peak<float>(nsm, st, fp32_tflops);
  return rc;
}
