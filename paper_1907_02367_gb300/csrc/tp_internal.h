// Internal structures of libtp shared by the host code (tp_host.cpp) and the
// CUDA code (tp_cuda.cu).  Not part of the public ABI (include/tp.h).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/tp.h"

namespace tp {

void set_error(const std::string& msg);

constexpr int kMaxDim = 3;
constexpr int kMaxP = 8;
constexpr int kMaxEvCls = 16;   // classes of basis functions by term count
constexpr int kMaxPatch = 64;     // elements in one vertex star handled by one CTA
constexpr int kMaxFacets = 16;    // Dirichlet + interface facets through one vertex
constexpr int kMaxGroups = 4;     // materials (distinct wave speeds) in one tent
constexpr int kTcSlices = 5;      // digits per operand of the tensor-core contractions
constexpr int tc_cols_max = 512;  // tensor-memory columns of an SM, all held by a CTA of the tensor-core path

// ---------------------------------------------------------------------------
// mesh topology built on the host
// ---------------------------------------------------------------------------
struct Topology {
  int dim = 0;
  int64_t nv = 0, ne = 0;
  std::vector<double> X;          // nv * dim
  std::vector<int32_t> elems;     // ne * (dim+1)
  std::vector<double> c;          // ne
  std::vector<int32_t> star_ptr, star_el;     // elements around a vertex (ascending)
  std::vector<int32_t> nbr_ptr, nbr;          // neighbouring vertices (ascending)
  std::vector<int32_t> facet_vert;            // boundary facets: dim sorted vertex ids each
  std::vector<double> facet_nrm;              // boundary facets: outward unit normal (dim)
  std::vector<int32_t> vfac_ptr, vfac;        // boundary facets through a vertex (facet order)
  std::vector<int32_t> facet_elem;            // boundary facets: owning element
  std::vector<int8_t> facet_kind;             // boundary facets: 0 Dirichlet, 1 Neumann
  // time-like interface facets (different wave speed on the two sides), listed
  // per vertex of the facet: dim vertex ids, the two elements (+ = lower index),
  // the unit normal out of the + element
  std::vector<int32_t> ifac_ptr, ifac_vert, ifac_kp, ifac_km;
  std::vector<double> ifac_nrm;
};

bool build_topology(const tp_mesh_desc* m, Topology* t);

// ---------------------------------------------------------------------------
// reference rule on the n-simplex (collapsed Gauss-Jacobi, m points per axis)
// ---------------------------------------------------------------------------
struct SimplexRule {
  int n = 0, m = 0, Q = 0;
  std::vector<double> bary;   // Q * (n+1)
  std::vector<double> w;      // Q, sums to 1/n!
};
SimplexRule simplex_rule(int n, int m);

}  // namespace tp

// ---------------------------------------------------------------------------
// opaque handles
// ---------------------------------------------------------------------------
struct tp_tents {
  int dim = 0;
  int64_t nv = 0;
  double T = 0.0, kappa = 0.0;
  std::vector<int32_t> vert, level, round;
  std::vector<double> t_bot, t_top;
  std::vector<int64_t> level_ptr;   // tents of level L (1-based) are [level_ptr[L-1], level_ptr[L])
  int32_t n_levels = 0;
};

struct tp_basis {
  int dim = 0, p = 0, nb = 0, nmono = 0;
  std::vector<int32_t> exps;        // nmono * (dim+1): exponents of (that, xhat_1..n)
  std::vector<int32_t> parent;      // monomial g = monomial parent[g] * variable var[g] (g >= 1)
  std::vector<int32_t> var;
  std::vector<double> coef;         // nb * nmono, U
  // sparse evaluation table: for basis j and component comp in
  // {U, d/dthat, d/dxhat_1..n}: entries [ptr[j*C+comp], ptr[j*C+comp+1])
  std::vector<int32_t> sp_ptr, sp_mono;
  std::vector<double> sp_coef;
  // derivative relations inside U^p: d/d(var) b_j = sum fac * b_src with
  // var in {that, xhat_1..n}; for (j, var): entries [rel_ptr[j*(n+1)+var], ...)
  std::vector<int32_t> rel_ptr, rel_src;
  std::vector<double> rel_fac;
  // transposed: for (k, var): entries (j, fac) with b_k appearing in d b_j
  std::vector<int32_t> relT_ptr, relT_dst;
  std::vector<double> relT_fac;
  // congruences of the top-face form, merged per entry (i <= j, packed order
  // p = i nb - i (i - 1) / 2 + j - i):
  //   (D_t X D_t^T + sum_m D_m X D_m^T)_ij = sum over [cg_ptr[p], cg_ptr[p+1]) of cg_coef * X[cg_idx]
  //   (sum_m D_m H_m D_t^T + D_t H_m D_m^T)_ij = sum over [ch_ptr[p], ch_ptr[p+1]) of
  //       ch_coef * H_{m}[ch_idx & 0xffff], m = ch_idx >> 16
  // (X, H_m packed symmetric; the coefficients are exact integers)
  // Dirichlet facet congruences, every entry (i, j) of nb x nb (row-major):
  //   (D_t F D_t^T)_ij = sum over [ft_ptr[ij], ft_ptr[ij+1]) of ft_coef * F[ft_idx]
  //   (D_t F D_m^T)_ij = sum over [fm_ptr[ij], fm_ptr[ij+1]) of fm_coef * F[fm_idx & 0xffff], m = fm_idx >> 16
  std::vector<int32_t> ft_ptr, ft_idx, fm_ptr, fm_idx;
  std::vector<float> ft_coef, fm_coef;
  std::vector<int32_t> pair_ij;     // (i << 16) | j of packed entry p
  std::vector<int32_t> cg_ptr, cg_idx, ch_ptr, ch_idx;
  std::vector<float> cg_coef, ch_coef;
};
