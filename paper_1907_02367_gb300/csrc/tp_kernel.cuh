// Device side of libtp shared by the translation units that instantiate the
// tent kernel (one per space dimension) and the context code: the kernel
// arguments, the float-float arithmetic, the basis and congruence helpers,
// and the tent kernel template itself.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "tp_internal.h"
#include "tp_tc.cuh"

namespace cg = cooperative_groups;

namespace tp {

constexpr int kThreads = 256;
constexpr int kMaxPair = 3;      // Gram pairs per thread (nb (nb+1)/2 <= 3 * 256: dim U^p <= 38)
constexpr int kMaxRefine = 40;   // refinement steps of the mixed path
constexpr long long kMaxSpin = 1LL << 20;   // bounded dependency wait: 2^20 polls (well under a second), then TP_ERR_TIMEOUT

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct KArgs {
  int nb, nmono, Q, nrhs, CH, mono_stride, ngmax;
  int ustride;                    // row stride of the U-values of a point in shared memory (nb rounded up to odd)
  // right-hand sides split over the cluster: CTA r of a tent's cluster owns
  // right-hand sides [r nrhs, (r + 1) nrhs) of the group (nrhs = per CTA) for
  // the data moments, the solve and the outflow, over all points of the
  // patch; the Grams stay split by points.  0: every CTA sees all nrhs.
  int rsplit;
  int p;                          // degree of U^p
  int mono_lv[kMaxP + 2];         // monomials of total degree d: [mono_lv[d], mono_lv[d+1])
  // U-value sums: basis functions in classes of equal term count (class with
  // ev_terms 0: one term of coefficient 1); class c is ev_order[ev_off[c] .. ev_off[c+1])
  int ev_ncls;
  int ev_off[kMaxEvCls + 1];
  int ev_terms[kMaxEvCls];
  const int* ev_order;
  int64_t ne, n_bnd;
  double alpha, beta;
  const double* X;
  const int* elems;
  const double* cK;
  const double* elem_einv;    // per element: inverse of the edge matrix e (rows X_i - X_0), dim x dim
  const double* elem_sdet;    // per element: sqrt(|det e|)
  const double* elem_isdet;   // per element: 1 / sqrt(|det e|)
  const double* bary;     // Q * (dim+1)
  const double* wref;     // Q
  const double* sqw;      // Q, sqrt(wref)
  const float2* sqw_dd;   // Q, sqrt(wref) as a float-float pair
  const double* isqw;     // Q, 1 / sqrt(wref)
  const int* tent_v;
  const double* tent_ttop;
  const double* tent_tbot;
  const double* tent_ih;      // 1 / h
  const int* tent_hdr;        // per tent: v, record offsets (int, double), elements, Dirichlet and interface facets, materials, Neumann facets
  const int* vrec_i;          // per vertex: star record, ints (elements, facets)
  const double* vrec_d;       // per vertex: star record, doubles (x_v, speeds, coordinates, normals)
  const long long* tent_gdoff;
  const int* sp_ptr;
  const int* sp_mono;
  const double* sp_coef;
  const float2* sp_coef_dd;   // (hi, lo) binary32 pair of every sp_coef entry
  const int* mono_parent;
  const int* mono_var;
  // merged congruence tables of the top-face form (see tp_basis)
  const int* pair_ij;
  const int *cg_ptr, *cg_idx, *ch_ptr, *ch_idx;
  const float *cg_coef, *ch_coef;
  const int *ft_ptr, *ft_idx, *fm_ptr, *fm_idx;   // Dirichlet facet congruences (see tp_basis)
  const float *ft_coef, *fm_coef;
  const double *cg_coefd, *ch_coefd, *ft_coefd, *fm_coefd;   // the same coefficients in binary64
  double* tau;
  double* front;
  const double* gD;
  double* diss;               // per right-hand side: accumulated energy lost in the tents (nullptr: not tracked)
  // wave-speed gradient: the forward sweep stores each tent's solution
  // (xsave[(tent - xbase) * xs_stride + r * ngmax * nb + row], r over the
  // group's right-hand sides) when xsave is set; the reverse sweep reads it
  // back with the forward front before the level (front_fwd) and adds
  // dJ/dc per element into dJdc when dJdc is set
  double* xsave;
  long long xbase, xs_stride;
  const double* front_fwd;
  double* dJdc;
  int off_yg;                 // shared memory of the gradient: y(x), y(x'), y(mu') and x
  // bounded waits and the solve's refinement: the dependency wait gives up
  // after max_spin polls (TP_ERR_TIMEOUT); a refinement that has not settled
  // after max_refine steps hands the tent to the direct binary64 LU;
  // solve_stats (kMaxRefine + 2 counters, or nullptr): [0] tents solved by
  // the direct LU, [1 + k] tents whose refinement settled after k steps
  long long max_spin;
  int max_refine;
  unsigned long long* solve_stats;
  // point outputs (forward sweep): the samples (probe point, output time)
  // that lie inside tent t are [probe_ptr[t], probe_ptr[t+1]) with the
  // probe's index, the time's index and the patch slot of its element; the
  // forward kernel writes U_h there: probe_out[(r * n_probe_t + k) * n_probe + j]
  const int* probe_ptr;        // nullptr: no point outputs
  const int* probe_j;
  const int* probe_k;
  const int* probe_slot;
  const double* probe_bary;   // per probe point: barycentric coordinates in its element
  const double* probe_t;      // output times
  int n_probe, n_probe_t;
  double* probe_out;
  int* status;
  long long* status_info;
  // persistent sweep: tent queue, completed tents per vertex, dependencies
  // (for tent t: vertices w of its star with the number of their tents that
  // must be complete, [dep_ptr[t], dep_ptr[t+1]))
  int* queue;
  int* done;
  const int* dep_ptr;
  const int* dep_vert;
  const int* dep_need;
  const int* queue_tent;      // tent at each queue position (level order, critical chains first)
  int tent_end;
  // shared-memory carve (offsets in doubles)
  const int* rel_ptr;
  const int* rel_src;
  const double* rel_fac;
  const int* relT_ptr;
  const int* relT_dst;
  const double* relT_fac;
  const float* rel_facf;      // relation factors (small integers) in binary32
  const float* relT_facf;
  int off_al, off_eq, off_z, off_x;             // solve: binary32 inverse and refinement
  int off_pt;                                   // per-point (that, xhat, scale) of the block-wide evaluation
  int keep_pts, off_keep, off_keepw;            // kept top U-values (scaled) and 1/sqrt(w) of a CTA's slice
  int off_b, off_pg, off_ph, off_pgb, off_pm, off_pd, off_sg, off_sm, off_f, off_f2, off_fpm, off_del,
      off_u, off_mono, off_cb, off_gd, off_y, off_rd;
  // tensor-core contractions (mixed forward sweep with split right-hand
  // sides, single-material tents): the data moments and the outflow run as
  // exact digit products on tcgen05 (tp_tc.cuh); off_tc: their staging
  // (bf16 digit planes, in the region of the facet sums, which is dead in
  // the point passes before phase 2 and in the outflow), tc_cols
  // tensor-memory columns held per CTA
  int tc, off_tc, tc_cols;
};

__device__ __forceinline__ void flag_error(const KArgs& a, int code, long long info) {
  if (atomicCAS(a.status, 0, code) == 0) *a.status_info = info;
}

// gradient g of the linear function with increments dv[i] along the edges
// e[i] = X_{i+1} - X_0 (solves e g = dv); returns det(e)
template <int DIM>
__device__ __forceinline__ double lin_grad(const double (&e)[DIM][DIM], const double* dv, double* g) {
  if constexpr (DIM == 1) {
    g[0] = dv[0] / e[0][0];
    return e[0][0];
  } else if constexpr (DIM == 2) {
    const double det = e[0][0] * e[1][1] - e[0][1] * e[1][0];
    const double id = 1.0 / det;
    g[0] = (e[1][1] * dv[0] - e[0][1] * dv[1]) * id;
    g[1] = (-e[1][0] * dv[0] + e[0][0] * dv[1]) * id;
    return det;
  } else {
    // rows of e^-1^T: (e1 x e2, e2 x e0, e0 x e1) / det
    double c0[3], c1[3], c2[3];
    c0[0] = e[1][1] * e[2][2] - e[1][2] * e[2][1];
    c0[1] = e[1][2] * e[2][0] - e[1][0] * e[2][2];
    c0[2] = e[1][0] * e[2][1] - e[1][1] * e[2][0];
    c1[0] = e[2][1] * e[0][2] - e[2][2] * e[0][1];
    c1[1] = e[2][2] * e[0][0] - e[2][0] * e[0][2];
    c1[2] = e[2][0] * e[0][1] - e[2][1] * e[0][0];
    c2[0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];
    c2[1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
    c2[2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
    const double det = e[0][0] * c0[0] + e[0][1] * c0[1] + e[0][2] * c0[2];
    const double id = 1.0 / det;
    for (int d = 0; d < 3; ++d) g[d] = (dv[0] * c0[d] + dv[1] * c1[d] + dv[2] * c2[d]) * id;
    return det;
  }
}

// determinant of a small symmetric Gram matrix
template <int DIM>
__device__ __forceinline__ double small_det(const double (&G)[DIM][DIM]) {
  if constexpr (DIM == 1) {
    return G[0][0];
  } else if constexpr (DIM == 2) {
    return G[0][0] * G[1][1] - G[0][1] * G[1][0];
  } else {
    return G[0][0] * (G[1][1] * G[2][2] - G[1][2] * G[2][1]) -
           G[0][1] * (G[1][0] * G[2][2] - G[1][2] * G[2][0]) +
           G[0][2] * (G[1][0] * G[2][1] - G[1][1] * G[2][0]);
  }
}

// ---------------------------------------------------------------------------
// Arithmetic used by the tent kernel.  The FP64 path computes in binary64.
// The mixed path computes the assembly, the refinement residual and the
// outflow in float-float ("double-float") arithmetic on the binary32 pipes,
// which GB300 runs ~58x faster than binary64: a value is an unevaluated sum
// hi + lo of two binary32 numbers (|lo| <= ulp(hi)/2, ~48 significant bits),
// built from the error-free transformations TwoSum (Knuth), FastTwoSum
// (Dekker) and TwoProd through the fused multiply-add.  The intrinsics
// __fadd_rn/__fsub_rn/__fmul_rn keep the compiler from contracting them.
// ---------------------------------------------------------------------------
struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dd fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  const dd t = two_sum(a.lo, b.lo);
  s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dd dd_mulf(dd a, float f) {   // f exact in binary32
  const float p = __fmul_rn(a.hi, f);
  float e = fmaf(a.hi, f, -p);
  e = fmaf(a.lo, f, e);
  return fast_two_sum(p, e);
}

// float-float split of a binary64 value, hi = x rounded to binary32 and
// lo = x - hi rounded, by integer operations on its bits (the binary64 unit,
// ~2 operations per clock per SM on this GPU, stays free); values outside
// [2^-74, 2^126) in magnitude (where lo would leave binary32's normal range)
// take the conversion instructions.  Equal in value to the conversions (a
// zero lo may carry the sign of x).
__device__ __forceinline__ dd dd_split(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((u >> 52) & 0x7FF) - 1023;
  if (E < -74 || E > 125) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
  }
  const unsigned long long frac = u & ((1ull << 52) - 1);
  const unsigned int low = (unsigned int)(frac & ((1u << 29) - 1));   // the 29 bits below binary32's fraction
  unsigned int hb = ((unsigned int)(u >> 63) << 31) | ((unsigned int)(E + 127) << 23) | (unsigned int)(frac >> 29);
  const bool up = low > (1u << 28) || (low == (1u << 28) && (hb & 1u));
  hb += up ? 1u : 0u;   // a carry out of the fraction raises the exponent
  // lo = x - hi = +-(low - up 2^29) 2^(E - 52), |.| <= 2^28 units
  const int r = (int)low - (up ? (1 << 29) : 0);
  const int k = E - 52, k1 = k / 2;
  float lo = __fmul_rn(__fmul_rn(__int2float_rn(r), __uint_as_float((unsigned int)(127 + k1) << 23)),
                       __uint_as_float((unsigned int)(127 + k - k1) << 23));
  if (u >> 63) lo = -lo;
  return {__uint_as_float(hb), lo};
}

template <typename T>
struct Ar;

template <>
struct Ar<double> {
  static __device__ __forceinline__ float hi(double x) { return (float)x; }
  static __device__ __forceinline__ double addf(double a, float f) { return a + (double)f; }
  static __device__ __forceinline__ double fms(double t, double a, double b) { return ::fma(-a, b, t); }
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double one() { return 1.0; }
  static __device__ __forceinline__ double from(double x) { return x; }
  static __device__ __forceinline__ double to(double x) { return x; }
  static __device__ __forceinline__ double add(double a, double b) { return a + b; }
  static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
  static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
  static __device__ __forceinline__ double mulf(double a, float f) { return a * (double)f; }
  static __device__ __forceinline__ double fmac(double a, float f, double c) { return ::fma(a, (double)f, c); }
  // accumulation of a long sum of products (see the float-float version)
  static __device__ __forceinline__ double acc(double s, double a, double b) { return ::fma(a, b, s); }
  static __device__ __forceinline__ double accf(double s, double a, float f) { return ::fma(a, (double)f, s); }
  static __device__ __forceinline__ double accn(double s, double a, double b) { return ::fma(-a, b, s); }
  static __device__ __forceinline__ double norm(double s) { return s; }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ double coef(const KArgs& a, int e);
};

template <>
struct Ar<dd> {
  static __device__ __forceinline__ float hi(dd x) { return x.hi; }
  static __device__ __forceinline__ dd addf(dd a, float f) { return dd_add(a, {f, 0.f}); }
  static __device__ __forceinline__ dd fms(dd t, dd a, dd b) {
    const dd p = dd_mul(a, b);
    return dd_add(t, {-p.hi, -p.lo});
  }
  static __device__ __forceinline__ dd zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ dd one() { return {1.f, 0.f}; }
  static __device__ __forceinline__ dd from(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
  }
  static __device__ __forceinline__ double to(dd x) { return (double)x.hi + (double)x.lo; }
  static __device__ __forceinline__ dd add(dd a, dd b) { return dd_add(a, b); }
  static __device__ __forceinline__ dd sub(dd a, dd b) { return dd_add(a, {-b.hi, -b.lo}); }
  static __device__ __forceinline__ dd mul(dd a, dd b) { return dd_mul(a, b); }
  static __device__ __forceinline__ dd mulf(dd a, float f) { return dd_mulf(a, f); }
  static __device__ __forceinline__ dd fmac(dd a, float f, dd c) { return dd_add(dd_mulf(a, f), c); }
  // s += a b for a long sum of products, compensated in the manner of Ogita,
  // Rump and Oishi's Dot2: s = (p, e) holds the running binary32 sum p and
  // the sum e of all rounding errors (of the products, exact by fmaf, and of
  // the additions, exact by TwoSum); the pair is not normalised until norm().
  static __device__ __forceinline__ dd acc(dd s, dd a, dd b) {
    const float h = __fmul_rn(a.hi, b.hi);
    float r = fmaf(a.hi, b.hi, -h);
    r = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, r));
    const float pn = __fadd_rn(s.hi, h);
    const float bb = __fsub_rn(pn, s.hi);
    const float q = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(pn, bb)), __fsub_rn(h, bb));
    return {pn, __fadd_rn(s.lo, __fadd_rn(q, r))};
  }
  static __device__ __forceinline__ dd accf(dd s, dd a, float f) {   // s += a f, f exact in binary32
    const float h = __fmul_rn(a.hi, f);
    const float r = fmaf(a.lo, f, fmaf(a.hi, f, -h));
    const float pn = __fadd_rn(s.hi, h);
    const float bb = __fsub_rn(pn, s.hi);
    const float q = __fadd_rn(__fsub_rn(s.hi, __fsub_rn(pn, bb)), __fsub_rn(h, bb));
    return {pn, __fadd_rn(s.lo, __fadd_rn(q, r))};
  }
  static __device__ __forceinline__ dd accn(dd s, dd a, dd b) { return acc(s, {-a.hi, -a.lo}, b); }   // s -= a b
  static __device__ __forceinline__ dd norm(dd s) { return fast_two_sum(s.hi, s.lo); }
  static __device__ __forceinline__ dd fma(dd a, dd b, dd c) { return dd_add(dd_mul(a, b), c); }
  static __device__ __forceinline__ dd coef(const KArgs& a, int e);
};

__device__ __forceinline__ double Ar<double>::coef(const KArgs& a, int e) { return __ldg(a.sp_coef + e); }
__device__ __forceinline__ dd Ar<dd>::coef(const KArgs& a, int e) {
  const float2 c = __ldg(a.sp_coef_dd + e);
  return {c.x, c.y};
}

// U-values at npt points with the whole block: the points' (that, xhat_1..xhat_n,
// scale) are in pt[q * (DIM + 2)]; one pass per monomial degree (m = parent
// monomial times one variable), then the sparse sums u_j = scale * sum c m.
// Monomials go to m[q * mono_stride], U-values to u[q * nb].  Callers write pt
// before the call; the first and last statements that touch shared memory
// are separated from them by barriers.
template <int DIM, typename T, bool SCALE = true>
__device__ __forceinline__ void eval_uvalues_block(const KArgs& a, int npt, const T* pt, T* m, T* u) {
  // Each thread takes one monomial (one basis function) at four points, so
  // that four independent products are in flight per table lookup.
  const int tid = threadIdx.x, ms = a.mono_stride, nb = a.nb;
  const int nq4 = (npt + 3) >> 2;
  // the constant monomial carries the scale, so every monomial and U-value is scaled
  for (int q = tid; q < npt; q += blockDim.x) m[q * ms] = SCALE ? pt[q * (DIM + 2) + DIM + 1] : Ar<T>::one();
  for (int d = 1; d <= a.p; ++d) {
    __syncthreads();   // pt, and the monomials of degree d - 1
    const int g0 = a.mono_lv[d], cnt = a.mono_lv[d + 1] - g0;
    for (int id = tid; id < cnt * nq4; id += blockDim.x) {
      const int g = g0 + id % cnt, q0 = (id / cnt) << 2;
      const int par = __ldg(a.mono_parent + g), vr = __ldg(a.mono_var + g);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int q = min(q0 + t, npt - 1);
        const T v = Ar<T>::mul(m[q * ms + par], pt[q * (DIM + 2) + vr]);
        if (q0 + t < npt) m[q * ms + g] = v;
      }
    }
  }
  __syncthreads();
  // items (function, four points) class after class, so that the lanes of a
  // warp run loops of one length; a one-term function of coefficient 1 is a copy
  for (int id = tid; id < nb * nq4; id += blockDim.x) {
    int c = 0;
    while (id >= a.ev_off[c + 1] * nq4) ++c;
    const int f0 = a.ev_off[c], nj = a.ev_off[c + 1] - f0, loc = id - f0 * nq4;
    const int j = __ldg(a.ev_order + f0 + loc % nj), q0 = (loc / nj) << 2;
    const int e0 = __ldg(a.sp_ptr + j * (DIM + 2)), e1 = __ldg(a.sp_ptr + j * (DIM + 2) + 1);
    int qq[4];
    T acc[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      qq[t] = min(q0 + t, npt - 1);
      acc[t] = Ar<T>::zero();
    }
    if (a.ev_terms[c] == 0) {
      const int g = __ldg(a.sp_mono + e0);
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (q0 + t < npt) u[qq[t] * a.ustride + j] = m[qq[t] * ms + g];
      continue;
    }
    for (int e = e0; e < e1; ++e) {
      const T c = Ar<T>::coef(a, e);
      const int g = __ldg(a.sp_mono + e);
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[t] = Ar<T>::acc(acc[t], c, m[qq[t] * ms + g]);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (q0 + t < npt) u[qq[t] * a.ustride + j] = Ar<T>::norm(acc[t]);
  }
  __syncthreads();
}

// s + y f for a factor f of a table of small exact numbers (derivative
// relations, merged congruence tables): binary64 reads the table's binary64
// copy and takes one fused multiply-add; float-float reads the binary32 copy
// (add: exact product and float-float sum; acc: a compensated long-sum step)
template <typename T>
struct Fac;
template <>
struct Fac<double> {
  static __device__ __forceinline__ double add(double s, double y, const float*, const double* fd, int e) {
    return ::fma(y, __ldg(fd + e), s);
  }
  static __device__ __forceinline__ double acc(double s, double y, const float*, const double* fd, int e) {
    return ::fma(y, __ldg(fd + e), s);
  }
};
template <>
struct Fac<dd> {
  static __device__ __forceinline__ dd add(dd s, dd y, const float* ff, const double*, int e) {
    return dd_add(s, dd_mulf(y, __ldg(ff + e)));
  }
  static __device__ __forceinline__ dd acc(dd s, dd y, const float* ff, const double*, int e) {
    return Ar<dd>::accf(s, y, __ldg(ff + e));
  }
};

// butterfly exchange of a value of the path's arithmetic within a warp
__device__ __forceinline__ double shfl_xor_t(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dd shfl_xor_t(dd v, int o) {
  return {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// packed upper-triangle index of (i, j), i, j < nb
__device__ __forceinline__ int pair_index(int i, int j, int nb) {
  const int lo = min(i, j), hi = max(i, j);
  return lo * nb - lo * (lo - 1) / 2 + (hi - lo);
}

// (D_va X D_vb^T)_ij for a packed symmetric X, D_var given by the relation
// table: (D_var u)_j = sum over entries e of (j, var) of fac_e u[src_e]
// (the factors are small integers, exact in binary32)
template <int DIM, typename T>
__device__ __forceinline__ T congruence(const KArgs& a, int i, int va, int j, int vb, const T* X, int nb) {
  constexpr int NVAR = DIM + 1;
  const int a0 = __ldg(a.rel_ptr + i * NVAR + va), a1 = __ldg(a.rel_ptr + i * NVAR + va + 1);
  const int b0 = __ldg(a.rel_ptr + j * NVAR + vb), b1 = __ldg(a.rel_ptr + j * NVAR + vb + 1);
  T s = Ar<T>::zero();
  for (int e = a0; e < a1; ++e) {
    const int si = __ldg(a.rel_src + e);
    T t = Ar<T>::zero();
    for (int f = b0; f < b1; ++f)
      t = Fac<T>::add(t, X[pair_index(si, __ldg(a.rel_src + f), nb)], a.rel_facf, a.rel_fac, f);
    s = Fac<T>::add(s, t, a.rel_facf, a.rel_fac, e);
  }
  return s;
}

// (D_var y)_i for a vector y
template <int DIM, typename T>
__device__ __forceinline__ T rel_apply(const KArgs& a, int i, int var, const T* y) {
  const int e0 = __ldg(a.rel_ptr + i * (DIM + 1) + var), e1 = __ldg(a.rel_ptr + i * (DIM + 1) + var + 1);
  T s = Ar<T>::zero();
  for (int e = e0; e < e1; ++e) s = Fac<T>::add(s, y[__ldg(a.rel_src + e)], a.rel_facf, a.rel_fac, e);
  return s;
}

// (D_var^T y)_k through the transposed table
template <int DIM, typename T>
__device__ __forceinline__ T relT_apply(const KArgs& a, int k, int var, const T* y) {
  const int e0 = __ldg(a.relT_ptr + k * (DIM + 1) + var), e1 = __ldg(a.relT_ptr + k * (DIM + 1) + var + 1);
  T s = Ar<T>::zero();
  for (int e = e0; e < e1; ++e) s = Fac<T>::add(s, y[__ldg(a.relT_dst + e)], a.relT_facf, a.relT_fac, e);
  return s;
}

// binary32 reciprocal of the hardware's approximate reciprocal instruction
// (about 1 ulp): the binary32 inverse of the solve is refined against A, so its
// last bit does not matter, and the correctly rounded reciprocal costs several
// times as long on the critical path of the elimination
__device__ __forceinline__ float rcp_fast(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// 1/x by two Newton-Raphson steps r <- r + r (1 - x r) from the binary32
// reciprocal (quadratic convergence: 24 -> 48 -> 96 bits); falls back to the
// division outside the binary32 range.
__device__ __forceinline__ double recip(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// (D_va X D_vb^T)_ij for a full row-major nb x nb X (or X^T when TR)
template <int DIM, typename T, bool TR>
__device__ __forceinline__ T congruence_full(const KArgs& a, int i, int va, int j, int vb, const T* X, int nb) {
  constexpr int NVAR = DIM + 1;
  const int a0 = __ldg(a.rel_ptr + i * NVAR + va), a1 = __ldg(a.rel_ptr + i * NVAR + va + 1);
  const int b0 = __ldg(a.rel_ptr + j * NVAR + vb), b1 = __ldg(a.rel_ptr + j * NVAR + vb + 1);
  T s = Ar<T>::zero();
  for (int e = a0; e < a1; ++e) {
    const int si = __ldg(a.rel_src + e);
    T t = Ar<T>::zero();
    for (int f = b0; f < b1; ++f) {
      const int sj = __ldg(a.rel_src + f);
      t = Fac<T>::add(t, TR ? X[sj * nb + si] : X[si * nb + sj], a.rel_facf, a.rel_fac, f);
    }
    s = Fac<T>::add(s, t, a.rel_facf, a.rel_fac, e);
  }
  return s;
}

// n-weighted normal-derivative congruences: (D_a X D_b^T) with a, b in {t, n}
// where D_n = sum_m n_m D_m.  SYM: X packed symmetric, else full (TR: X^T).
template <int DIM, typename T, int MODE>
__device__ __forceinline__ T cong_any(const KArgs& a, int i, int va, int j, int vb, const T* X, int nb) {
  if constexpr (MODE == 0) return congruence<DIM, T>(a, i, va, j, vb, X, nb);
  else if constexpr (MODE == 1) return congruence_full<DIM, T, false>(a, i, va, j, vb, X, nb);
  else return congruence_full<DIM, T, true>(a, i, va, j, vb, X, nb);
}
template <int DIM, typename T, int MODE>
__device__ __forceinline__ void iface_terms(const KArgs& a, int i, int j, const T* X, int nb, const T* nrm,
                                            T* ntn, T* ntt, T* ttn, T* nnn) {
  // ntt = (D_n X D_t^T), ttn = (D_t X D_n^T), nnn = (D_n X D_n^T), ntn unused slot kept for symmetry
  T a1 = Ar<T>::zero(), a2 = Ar<T>::zero(), a3 = Ar<T>::zero();
  for (int m = 0; m < DIM; ++m) {
    a1 = Ar<T>::fma(nrm[m], cong_any<DIM, T, MODE>(a, i, 1 + m, j, 0, X, nb), a1);
    a2 = Ar<T>::fma(nrm[m], cong_any<DIM, T, MODE>(a, i, 0, j, 1 + m, X, nb), a2);
    for (int m2 = 0; m2 < DIM; ++m2)
      a3 = Ar<T>::fma(Ar<T>::mul(nrm[m], nrm[m2]), cong_any<DIM, T, MODE>(a, i, 1 + m, j, 1 + m2, X, nb), a3);
  }
  *ntt = a1;
  *ttn = a2;
  *nnn = a3;
  *ntn = cong_any<DIM, T, MODE>(a, i, 0, j, 0, X, nb);   // (D_t X D_t^T)
}

// One tent per thread-block cluster of CS CTAs (CS = gridDim.x / tents in the
// launch, 1..8).  Each CTA takes a slice of the patch's points.
//
// Materials (Section 4.2).  The patch elements are grouped by wave speed; each
// group g carries its own polynomial x_g in U^p mapped with its own c_g
// (Remark 3.1), so the tent system has ng*nb unknowns.
//
// Assembly through Grams of U-values.  With u the vector of the nb U-values
// at a point and the exact derivative maps of U^p, v = (c/h) D_t u,
// sigma_m = -(1/h) D_m u, the top-face form of group g summed over its points is
//   A_top = h^-2 [ D_t G D_t^T + sum_m D_m G D_m^T + c sum_m (D_m H_m D_t^T + D_t H_m D_m^T) ],
//   G = sum_q w u u^T,  H_m = sum_K g_{K,m} G_K  (g = top front gradient on K),
// the recovery term is A_bot = sum_q w u_b u_b^T, the bottom data give
//   b = gamma + (c/h) D_t alpha - (1/h) sum_m D_m beta_m
// with moments gamma = sum w U_b u_b, alpha = sum w (c^-2 v_b - s_b.g_b) u_b,
// beta_m = sum w (s_b,m - v_b g_b,m) u_b.  A Dirichlet facet with normal n
// adds A_D = (c/h) D_t F E^T, b_D = E' delta, F = sum w u u^T,
// delta = sum w g_D u, E = alpha_D (c/h) D_t - (1/h) D_n, E' = alpha_D (c/h) D_t + (1/h) D_n,
// D_n = sum_m n_m D_m.  A Neumann facet (sigma.n = g_N) adds
// A_N = -(c/h^2) D_n F D_t^T + (beta/h^2) D_n F D_n^T and
// b_N = -(c/h) D_t delta - (beta/h) D_n delta, delta = sum w g_N u (eq. 4.1; the
// code is compiled in only when NEU).  A time-like facet between groups + and - (normal n out
// of +) adds, for test side t and trial side s (signs s_+ = 1, s_- = -1),
//   A^{ts} = s_t h^-2 [ -c_s/2 D_n F^{ts} D_t^T - c_t/2 D_t F^{ts} D_n^T ]
//          + s_t s_s h^-2 [ alpha c_s c_t D_t F^{ts} D_t^T + beta D_n F^{ts} D_n^T ],
//   F^{ts} = sum w u^t u^s^T,
// the {v}[[tau]]_N + {s}.[[w]]_N + alpha [[v]]_N.[[w]]_N + beta [[s]]_N [[tau]]_N
// terms of eq. (2.5).  Every CTA publishes its partial Grams and moments;
// after a cluster barrier every CTA sums them in rank order, forms A and b,
// solves, and writes the outflow of its slice.
//
// MIXED = false: assembly, residual and outflow in binary64; MIXED = true:
// in float-float.  Both: A is equilibrated (D A D, D = |diag A|^-1/2),
// inverted in binary32 and the solution refined against A in the path's
// precision until the correction stops shrinking; a refinement that does not
// settle falls back to a direct binary64 LU.
//
// ADJ = true: the adjoint tent map (reverse sweep).  With g_D = 0 a tent maps
// its bottom values linearly to its top values, b = B f_bot, A x = b,
// f_top = E x; the adjoint takes lambda at the top points to
// mu = A^-T (E^T lambda) and lambda_bot = B^T mu at the bottom points.  In the
// U-value form E^T lambda = zeta_U + (c/h) D_t zeta_v - (1/h) sum_m D_m zeta_m,
// zeta = sum_q lambda_q u_q over the top points (the moment formula of b), and
// B^T mu at a bottom point is w (s0, c^-2 s_t - g_b.s, s_m - g_b,m s_t) with
// s0 = u.mu, s_t = (c/h) u.D_t^T mu, s_m = -(1/h) u.D_m^T mu.  The front and
// time arrays of the arguments are then the adjoint state (tau runs backwards).
//
// PERSIST = true: one resident grid of clusters; each cluster takes the next
// tent of the sorted list from a queue, waits (bounded) until the tents of its
// vertex and neighbours that precede it in level are complete, solves it and
// publishes its completion.  Tents leave the queue in level order, so every
// awaited tent is held by a running cluster: no launch per level, and a tent
// starts as soon as its own inputs are ready.  The front and the front times
// are read through L2 (ld.global.cg) so that no stale L1 line is used.
template <int DIM, bool MIXED, bool ADJ, bool PERSIST, bool NEU>
__global__ void __launch_bounds__(kThreads, 2) k_layer(const KArgs a, const int tent0) {
  using T = typename std::conditional<MIXED, dd, double>::type;
  using R = Ar<T>;
  constexpr int NV = DIM + 1;   // vertices per element
  constexpr int C = DIM + 2;    // U, v, sigma  (and gamma, alpha, beta_m moments)
  extern __shared__ __align__(16) double sm[];
  __shared__ int s_P, s_v, s_nfac, s_nif, s_ng, s_nneu;
  __shared__ double s_ttop, s_tbot, s_tc, s_ih;
  __shared__ double s_gc[tp::kMaxGroups], s_gic2[tp::kMaxGroups];   // speeds and 1/c^2 of the materials
  __shared__ double s_xv[DIM];
  __shared__ int s_el[tp::kMaxPatch], s_grp[tp::kMaxPatch];
  // vertex ids of elements; of facets (slots 2..): for boundary facets slot 0
  // holds the block of their data among the vertex's boundary facets
  __shared__ int s_vid[tp::kMaxPatch][NV], s_fw[tp::kMaxFacets][NV];
  __shared__ double s_X[tp::kMaxPatch][NV][DIM];
  __shared__ double s_tb[tp::kMaxPatch][NV], s_tt[tp::kMaxPatch][NV];
  __shared__ double s_gb[tp::kMaxPatch][DIM], s_gt[tp::kMaxPatch][DIM];
  __shared__ double s_sdet[tp::kMaxPatch], s_isdet[tp::kMaxPatch];
  // mixed path: g_bot (DIM) and sqrt|det| (slot DIM) of each element and c^-2 of each material as float-float pairs
  __shared__ float2 s_gbf[MIXED ? tp::kMaxPatch : 1][DIM + 1];
  __shared__ float2 s_gic2f[tp::kMaxGroups];
  __shared__ double s_fP[tp::kMaxFacets][NV][DIM + 1];   // vertical face simplices (x, t)
  __shared__ double s_fsq[tp::kMaxFacets], s_fn[tp::kMaxFacets][DIM];   // sqrt(n! volume), normal
  __shared__ int s_fg[tp::kMaxFacets], s_fg2[tp::kMaxFacets];   // groups (Dirichlet: one; interface: +, -)
  __shared__ int s_pgrp[2 * 64];
  __shared__ double s_gel[tp::kMaxPatch];   // wave-speed gradient of the tent per patch element
  __shared__ int s_piv;
  __shared__ float s_pb[2][4][32];   // register sweeps: the pivot rows of a block of four steps
  __shared__ float s_red[2][kThreads / 32];

  __shared__ int s_tent;
  // tensor-core contractions: tensor-memory base, completion barrier of the
  // MMAs, binary exponents of the rows of A (0) and the columns of B (1)
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_tcbar;
  __shared__ int s_tce[2][tc::kMaxM];
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int CS = (int)cluster.num_blocks();
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr bool kTC = MIXED && !ADJ;   // the tensor-core path exists for the mixed forward sweep
  uint32_t tc_phase = 0;                // parity of the next completion of s_tcbar
  if (kTC && a.tc) {
    if (warp == 0) tc::tmem_alloc(&s_tmem, a.tc_cols);
    if (tid == 0) tc::mbar_init(&s_tcbar, 1);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  for (;;) {
  int tent;
  if constexpr (PERSIST) {
    // rank 0 takes the next tent and stores its index into every CTA of the
    // cluster (each CTA read its copy of the previous index several cluster
    // barriers ago)
    if (rank == 0 && tid == 0) {
      const int pos = atomicAdd(a.queue, 1);
      const int t_ = pos < a.tent_end ? __ldg(a.queue_tent + pos) : a.tent_end;
      for (int r = 0; r < CS; ++r) *cluster.map_shared_rank(&s_tent, r) = t_;
    }
    cluster.sync();
    tent = s_tent;
    if (tent >= a.tent_end) break;
  } else {
    tent = tent0 + blockIdx.x / CS;
  }
  const int nb = a.nb, Q = a.Q, nrhs = a.nrhs, CH = a.CH, NG = a.ngmax;
  const int us = a.ustride;   // row stride of the U-values in shared memory (odd: no bank conflicts between points)
  // this CTA's right-hand sides (all of the group unless they are split over the cluster)
  const bool rsplit = a.rsplit != 0;
  double* const front = a.front + (rsplit ? (size_t)rank * nrhs * a.ne * Q * C : 0);
  const double* const gD = a.gD != nullptr ? a.gD + (rsplit ? (size_t)rank * nrhs * a.n_bnd : 0) : nullptr;
  const int npair = nb * (nb + 1) / 2;
  const int nmom = nrhs * C * nb;
  T* sA = reinterpret_cast<T*>(sm);                  // N*N        assembled A, then LU factors
  T* sb = reinterpret_cast<T*>(sm + a.off_b);        // nrhs*N     assembled b, then x
  T* sPG = reinterpret_cast<T*>(sm + a.off_pg);      // NG*npair   this CTA: G (top) per group
  T* sPH = reinterpret_cast<T*>(sm + a.off_ph);      // NG*DIM*npair  H_m
  T* sPGb = reinterpret_cast<T*>(sm + a.off_pgb);    // NG*npair   G (bottom, recovery)
  T* sPM = reinterpret_cast<T*>(sm + a.off_pm);      // NG*nmom    moments (gamma, alpha, beta_m) per rhs, this CTA
  T* sPD = reinterpret_cast<T*>(sm + a.off_pd);      // N*N        interface blocks (tents with interface facets)
  T* sSG = reinterpret_cast<T*>(sm + a.off_sg);      // NG*(DIM+2)*npair  summed G, H_m, Gbot
  T* sSM = reinterpret_cast<T*>(sm + a.off_sm);      // NG*nmom    summed moments (in place of sPM)
  T* sF = reinterpret_cast<T*>(sm + a.off_f);        // npair      facet Gram (+ side)
  T* sF2 = reinterpret_cast<T*>(sm + a.off_f2);      // npair      facet Gram (- side)
  T* sFpm = reinterpret_cast<T*>(sm + a.off_fpm);    // nb*nb      facet Gram (+ test, - trial)
  T* sDel = reinterpret_cast<T*>(sm + a.off_del);    // nrhs*nb    facet moments delta
  T* sU = reinterpret_cast<T*>(sm + a.off_u);        // 2*CH*nb    U-values (scaled) per (side, point)
  T* sPt = reinterpret_cast<T*>(sm + a.off_pt);      // 2*CH*(DIM+2)  (that, xhat, scale) per point
  T* sM = reinterpret_cast<T*>(sm + a.off_mono);     // 2*CH*mono_stride
  T* sCB = reinterpret_cast<T*>(sm + a.off_cb);      // nrhs*C*(CH+1) data coefficients, point fastest
  const int cbs = CH + 1;                            // their row stride (odd: no bank conflicts along a row)
  T* sGd = reinterpret_cast<T*>(sm + a.off_gd);      // CH*nrhs    Dirichlet data coefficients
  T* sY = reinterpret_cast<T*>(sm + a.off_y);        // NG*nmom    outflow coefficient vectors (sPM, dead after the congruence)
  double* sRD = sm + a.off_rd;                       // N          reciprocal pivots (binary64 path)

  // ---------------- phase 0: tent, materials and patch geometry ----------------
  // (a) what does not depend on earlier tents: vertex star, coordinates,
  // materials, facets; in the dataflow sweep it is fetched while the tents
  // this one depends on may still be running
  // one round of loads: the tent's header, then its vertex's star record
  const int4 h0 = __ldg(reinterpret_cast<const int4*>(a.tent_hdr) + 2 * (size_t)tent);
  const int4 h1 = __ldg(reinterpret_cast<const int4*>(a.tent_hdr) + 2 * (size_t)tent + 1);
  const int v = h0.x, P = h0.w, nfac = h1.x, nif = h1.y, ng = h1.z;   // Neumann facets: h1.w, s_nneu
  if (tid == 0) {
    s_v = v;
    s_P = P;
    s_ttop = a.tent_ttop[tent];
    s_ih = a.tent_ih[tent];
    s_nfac = nfac;
    s_nif = nif;
    s_ng = ng;
    s_nneu = h1.w;
  }
  for (int id = tid; id < NG * nmom; id += blockDim.x) sPM[id] = R::zero();
  for (int id = tid; id < NG * (DIM + 2) * npair; id += blockDim.x) sPG[id] = R::zero();   // PG, PH, PGb contiguous
  const int N = ng * nb;
  const bool extra = (nfac > 0 || nif > 0 || (NEU && h1.w > 0));
  {
    const int* ri = a.vrec_i + h0.y;
    const double* rd = a.vrec_d + h0.z;
    if (tid < DIM) s_xv[tid] = __ldg(rd + tid);
    if (tid < ng) {
      s_gc[tid] = __ldg(rd + DIM + tid);
      s_gic2[tid] = __ldg(rd + DIM + tp::kMaxGroups + tid);
      if constexpr (MIXED) {
        const T g2 = R::from(s_gic2[tid]);
        s_gic2f[tid] = make_float2(g2.hi, g2.lo);
      }
    }
    const double* rX = rd + DIM + 2 * tp::kMaxGroups;
    for (int k = tid; k < P; k += blockDim.x) {
      s_el[k] = __ldg(ri + k * (2 + NV));
      s_grp[k] = __ldg(ri + k * (2 + NV) + 1);
      for (int i = 0; i < NV; ++i) {
        s_vid[k][i] = __ldg(ri + k * (2 + NV) + 2 + i);
        for (int d = 0; d < DIM; ++d) s_X[k][i][d] = __ldg(rX + (k * NV + i) * DIM + d);
      }
    }
    // vertical face simplices (x_v, t_bot), (x_v, t_top), (x_w, tau_w): Dirichlet
    // facets first, then the time-like interface facets, then Neumann facets
    const int* rfi = ri + P * (2 + NV);
    const double* rfd = rX + P * NV * DIM;
    for (int f = tid; f < nfac + nif + (NEU ? h1.w : 0); f += blockDim.x) {
      for (int i = 2; i < NV; ++i) s_fw[f][i] = __ldg(rfi + f * (NV + 3) + i);
      s_fg[f] = __ldg(rfi + f * (NV + 3) + NV);
      s_fg2[f] = __ldg(rfi + f * (NV + 3) + NV + 1);
      s_fw[f][0] = __ldg(rfi + f * (NV + 3) + NV + 2);
      const double* fd = rfd + f * (DIM + NV * DIM);
      for (int d = 0; d < DIM; ++d) s_fn[f][d] = __ldg(fd + d);
      for (int i = 0; i < NV; ++i)
        for (int d = 0; d < DIM; ++d) s_fP[f][i][d] = __ldg(fd + DIM + i * DIM + d);
    }
  }
  if constexpr (PERSIST) {
    // the earlier tents of this vertex and its neighbours must be complete:
    // every CTA of a tent publishes its own completion, so a vertex whose
    // first `need` tents are done has a count of need * CS; each CTA waits
    // for (and acquires) the counts itself
    {
      const int d0 = a.dep_ptr[tent], d1 = a.dep_ptr[tent + 1];
      for (int e = d0 + tid; e < d1; e += blockDim.x) {
        const int w = a.dep_vert[e], need = a.dep_need[e] * CS;
        long long spins = 0;
        while (ld_acquire(a.done + w) < need) {
          if (++spins > a.max_spin) {
            flag_error(a, TP_ERR_TIMEOUT, tent);
            break;
          }
          // once any tent has flagged an error the sweep's result is void:
          // stop waiting so that the launch ends promptly
          if ((spins & 255) == 0 && ld_acquire(a.status) != 0) break;
          __nanosleep(32);
        }
      }
    }
    __syncthreads();
  } else {
    __syncthreads();
  }
  // (b) the front times: bottom and top fronts over every element, causality
  const double tbot = ADJ ? a.tent_tbot[tent] : __ldcg(a.tau + v);
  if (tid == 0) {
    s_tbot = tbot;
    s_tc = 0.5 * (tbot + s_ttop);
  }
  for (int k = tid; k < P; k += blockDim.x) {
    for (int i = 0; i < NV; ++i) {
      const int vi = s_vid[k][i];
      const double tv = (vi == v) ? tbot : __ldcg(a.tau + vi);
      s_tb[k][i] = tv;
      s_tt[k][i] = (vi == v) ? s_ttop : tv;
    }
    // gradients of the linear fronts: g = e^-1 (tau_i - tau_0), e from the host
    const int el = s_el[k];
    double db[DIM], dt[DIM];
    for (int i = 0; i < DIM; ++i) {
      db[i] = s_tb[k][i + 1] - s_tb[k][0];
      dt[i] = s_tt[k][i + 1] - s_tt[k][0];
    }
    double g2 = 0.0;
    for (int d = 0; d < DIM; ++d) {
      double gb = 0.0, gt = 0.0;
      for (int i = 0; i < DIM; ++i) {
        const double ei = __ldg(a.elem_einv + ((int64_t)el * DIM + d) * DIM + i);
        gb = fma(ei, db[i], gb);
        gt = fma(ei, dt[i], gt);
      }
      s_gb[k][d] = gb;
      s_gt[k][d] = gt;
      g2 = fma(gt, gt, g2);
    }
    s_sdet[k] = __ldg(a.elem_sdet + el);
    s_isdet[k] = __ldg(a.elem_isdet + el);
    if constexpr (MIXED) {
      for (int d = 0; d < DIM; ++d) {
        const dd gf = dd_split(s_gb[k][d]);
        s_gbf[k][d] = make_float2(gf.hi, gf.lo);
      }
      const dd sf = dd_split(s_sdet[k]);
      s_gbf[k][DIM] = make_float2(sf.hi, sf.lo);
    }
    const double ck = s_gc[s_grp[k]];
    if (!(ck * ck * g2 < 1.0)) flag_error(a, TP_ERR_CAUSALITY, tent);   // space-like top face: c |g| < 1
  }
  for (int f = tid; f < nfac + nif + (NEU ? s_nneu : 0); f += blockDim.x) {
    s_fP[f][0][DIM] = tbot;
    s_fP[f][1][DIM] = s_ttop;
    for (int c2 = 2; c2 <= DIM; ++c2) s_fP[f][c2][DIM] = __ldcg(a.tau + s_fw[f][c2]);
    // n! * n-volume = sqrt(det(E^T E)), E = [P_i - P_0] ((n+1) x n)
    double G[DIM][DIM];
    for (int i = 0; i < DIM; ++i)
      for (int j = 0; j < DIM; ++j) {
        double s_ = 0.0;
        for (int d = 0; d <= DIM; ++d) s_ += (s_fP[f][i + 1][d] - s_fP[f][0][d]) * (s_fP[f][j + 1][d] - s_fP[f][0][d]);
        G[i][j] = s_;
      }
    // sqrt(w) = sqrt(w_ref) sqrt(n! volume) at the facet's points
    s_fsq[f] = sqrt(sqrt(fabs(small_det<DIM>(G))));
  }
  // Gram pairs owned by this thread (upper triangle, i <= j, row-major order)
  int pi[kMaxPair], pj[kMaxPair];
  T aK[kMaxPair], aG[kMaxPair], aH[kMaxPair][DIM], aB[kMaxPair];
#pragma unroll
  for (int s = 0; s < kMaxPair; ++s) {
    const int id = tid + s * kThreads;
    int i = 0, j = 0;
    if (id < npair) {
      int rem = id;
      while (rem >= nb - i) {
        rem -= nb - i;
        ++i;
      }
      j = i + rem;
    }
    pi[s] = i;
    pj[s] = j;
    aK[s] = aG[s] = aB[s] = R::zero();
#pragma unroll
    for (int d = 0; d < DIM; ++d) aH[s][d] = R::zero();
  }
  __syncthreads();

  // tensor-core contractions for this tent (single material, split right-hand sides)
  const bool tc_on = kTC && a.tc && ng == 1;
  // ---------------- phase 1: this CTA's slice of the patch points ----------------
  const int NP = P * Q;
  const int slice = (NP + CS - 1) / CS;
  const int q0 = min(NP, rank * slice), q1 = min(NP, q0 + slice);
  const double ih = s_ih, tc = s_tc;
  int curk = q0 / Q, kend = (curk + 1) * Q;
  int curg = (q1 > q0) ? s_grp[curk] : 0;
  // forward sweep: the top U-values of a slice that fits the keep buffer are
  // kept for the outflow instead of being evaluated a second time
  const bool keep = !ADJ && !rsplit && (q1 - q0) <= a.keep_pts;
  T* sKeep = reinterpret_cast<T*>(sm + a.off_keep);   // keep_pts*nb  sqrt(w)-scaled top U-values
  double* sKeepW = sm + a.off_keepw;                   // keep_pts     1 / sqrt(w)
  // element flush: G += G_K, H_m += g_{K,m} G_K;  group flush: publish G, H, Gbot of the group
  auto flush_element = [&](int k) {
    T g[DIM];
    for (int d = 0; d < DIM; ++d) g[d] = R::from(s_gt[k][d]);
#pragma unroll
    for (int s = 0; s < kMaxPair; ++s) {
      const T k_ = R::norm(aK[s]);
      aG[s] = R::add(aG[s], k_);
#pragma unroll
      for (int d = 0; d < DIM; ++d) aH[s][d] = R::fma(g[d], k_, aH[s][d]);
      aK[s] = R::zero();
    }
  };
  auto flush_group = [&](int g) {
#pragma unroll
    for (int s = 0; s < kMaxPair; ++s) {
      const int id = tid + s * kThreads;
      if (id < npair) {
        sPG[g * npair + id] = R::add(sPG[g * npair + id], aG[s]);
#pragma unroll
        for (int d = 0; d < DIM; ++d)
          sPH[(g * DIM + d) * npair + id] = R::add(sPH[(g * DIM + d) * npair + id], aH[s][d]);
        sPGb[g * npair + id] = R::add(sPGb[g * npair + id], R::norm(aB[s]));
      }
      aG[s] = aB[s] = R::zero();
#pragma unroll
      for (int d = 0; d < DIM; ++d) aH[s][d] = R::zero();
    }
  };
  // a patch point q of element k mapped to the tent's reference coordinates
  // (Remark 3.1) on the top (TOP) or bottom face, with sqrt(w) as the scale of
  // its U-values; returns sqrt(w)
  auto map_point = [&](T* pp, int k, int q, bool top) {
    const double cg = s_gc[s_grp[k]];
    double x[DIM], tt = 0.0;
    for (int d = 0; d < DIM; ++d) x[d] = 0.0;
    for (int i = 0; i < NV; ++i) {
      const double l = __ldg(a.bary + q * NV + i);
      for (int d = 0; d < DIM; ++d) x[d] = fma(l, s_X[k][i][d], x[d]);
      tt = fma(l, top ? s_tt[k][i] : s_tb[k][i], tt);
    }
    pp[0] = R::from(cg * (tt - tc) * ih);
    for (int d = 0; d < DIM; ++d) pp[1 + d] = R::from((x[d] - s_xv[d]) * ih);
    const double sw = __ldg(a.sqw + q) * s_sdet[k];
    pp[DIM + 1] = R::from(sw);
    return sw;
  };
  // data coefficients of the points base .. base + nq - 1 (patch point
  // numbering) for every right-hand side, one (point, right-hand side) per
  // thread so that the front loads of a chunk are all in flight at once:
  // forward, the bottom values in the form of the moments (gamma, alpha,
  // beta_m); adjoint, lambda at the top point
  auto data_coefs = [&](int base, int nq) {
    for (int id = tid; id < nq * nrhs; id += blockDim.x) {   // (consecutive threads: consecutive points)
      const int r = id / nq, ql = id % nq, qg = base + ql, k = qg / Q, q = qg % Q;
      const double* f = front + (((int64_t)r * a.ne + s_el[k]) * Q + q) * C;
      double fv[C];
#pragma unroll
      for (int cc = 0; cc < C; ++cc) fv[cc] = __ldcg(f + cc);
      T* cb = sCB + (size_t)r * C * cbs + ql;   // component cc at cb[cc * cbs]
      if constexpr (ADJ) {
        // adjoint: zeta = sum_q lambda_q u_q over the top points
        const double isw = __ldg(a.isqw + q) * s_isdet[k];
#pragma unroll
        for (int cc = 0; cc < C; ++cc) cb[cc * cbs] = R::from(fv[cc] * isw);
      } else if constexpr (MIXED) {
        // the same coefficients in float-float, the stored values split by
        // integer operations (no binary64 arithmetic per point and column)
        const float2 w2 = __ldg(a.sqw_dd + q), d2 = s_gbf[k][DIM], c2 = s_gic2f[s_grp[k]];
        const dd sw = dd_mul({w2.x, w2.y}, {d2.x, d2.y});
        dd f[C];
#pragma unroll
        for (int cc = 0; cc < C; ++cc) f[cc] = dd_split(fv[cc]);
        dd gb[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) gb[d] = {s_gbf[k][d].x, s_gbf[k][d].y};
        dd sg = dd_mul(f[2], gb[0]);
#pragma unroll
        for (int d = 1; d < DIM; ++d) sg = dd_add(sg, dd_mul(f[2 + d], gb[d]));
        cb[0] = dd_mul(sw, f[0]);                                                     // gamma
        cb[cbs] = dd_mul(sw, R::sub(dd_mul({c2.x, c2.y}, f[1]), sg));                   // alpha
#pragma unroll
        for (int d = 0; d < DIM; ++d) cb[(2 + d) * cbs] = dd_mul(sw, R::sub(f[2 + d], dd_mul(f[1], gb[d])));   // beta_m
      } else {
        const double sw = __ldg(a.sqw + q) * s_sdet[k], ic2 = s_gic2[s_grp[k]];
        const double Ub = fv[0], vb = fv[1];
        double sg = 0.0;
        for (int d = 0; d < DIM; ++d) sg = fma(fv[2 + d], s_gb[k][d], sg);
        cb[0] = R::from(sw * Ub);                       // gamma
        cb[cbs] = R::from(sw * (ic2 * vb - sg));          // alpha
        for (int d = 0; d < DIM; ++d) cb[(2 + d) * cbs] = R::from(sw * (fv[2 + d] - vb * s_gb[k][d]));   // beta_m
      }
    }
  };
  // the front records (C values each) that data_coefs(base, nq) will read,
  // prefetched into L2 (their latency then overlaps the work on the chunk before)
  auto prefetch_front = [&](int base, int nq) {
    for (int id = tid; id < nq * nrhs; id += blockDim.x) {
      const int r = id / nq, ql = id % nq, qg = base + ql, k = qg / Q, q = qg % Q;
      const double* f = front + (((int64_t)r * a.ne + s_el[k]) * Q + q) * C;
      asm volatile("prefetch.global.L2 [%0];" ::"l"(f));
      asm volatile("prefetch.global.L2 [%0];" ::"l"(f + C - 1));
    }
  };
  // moments of the data of nq points whose U-values are rows prow.. of sU, per
  // material: one (material, right-hand side, basis function) per group of
  // ps lanes with its C components as independent sums; the lanes of a group
  // take every ps-th point and are added by butterfly shuffles (a fixed order)
  auto data_moments = [&](int nq, int prow) {
    const int nitem = ng * nrhs * nb;
    int ps = 1;
    while (ps < 8 && nitem * ps * 2 <= (int)blockDim.x) ps *= 2;
    for (int id0 = 0; id0 < nitem * ps; id0 += blockDim.x) {
      const int id = id0 + tid, item = id / ps, part = id % ps;
      const int g = item / (nrhs * nb), rest = item % (nrhs * nb), r = rest / nb, i = rest % nb;
      T t[C];
#pragma unroll
      for (int cc = 0; cc < C; ++cc) t[cc] = R::zero();
      if (item < nitem)
        for (int ql = part; ql < nq; ql += ps)
          if (s_pgrp[ql] == g) {
            const T u = sU[(size_t)(prow + ql) * us + i];
            const T* cb = sCB + (size_t)r * C * cbs + ql;
#pragma unroll
            for (int cc = 0; cc < C; ++cc) t[cc] = R::acc(t[cc], cb[cc * cbs], u);
          }
#pragma unroll
      for (int cc = 0; cc < C; ++cc) t[cc] = R::norm(t[cc]);
      for (int o = 1; o < ps; o <<= 1)
#pragma unroll
        for (int cc = 0; cc < C; ++cc) t[cc] = R::add(t[cc], shfl_xor_t(t[cc], o));
      if (part == 0 && item < nitem) {
        T* M = sPM + (size_t)g * nmom + (size_t)r * C * nb + i;
#pragma unroll
        for (int cc = 0; cc < C; ++cc) M[cc * nb] = R::add(M[cc * nb], t[cc]);
      }
    }
  };
  // ---- tensor-core contractions (tp_tc.cuh) ----
  // the digit-plane products of one contraction: level L = i + j sums planes
  // i of A and j of B over ksteps K steps of 16 into tensor-memory columns
  // (L - 2) cstride; one thread issues them (tc_issue), every thread waits
  // (bounded) for their completion (tc_wait, which returns whether they
  // completed, the same in every thread)
  auto tc_issue = [&](uint32_t aA, uint32_t planeA, uint32_t lboA, uint32_t aB, uint32_t planeB, uint32_t lboB,
                      int ksteps, int N, int cstride) {
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      const uint32_t id_ = tc::idesc_bf16(tc::kMaxM, N);
      if (planeB == 0) {
        // B's digit planes stacked along N at cstride-row offsets (plane j at
        // rows (j - 1) cstride): one product per plane i of A and K step puts
        // A_i B_j into the columns of level i + j for every j at once (the
        // columns past level S + 1 take unused pairs and are never read)
        for (int ks = 0; ks < ksteps; ++ks)
          for (int i = 1; i <= tc::kSlices; ++i)
            tc::mma_bf16(s_tmem + (uint32_t)((i - 1) * cstride),
                         tc::sdesc(aA + (uint32_t)(i - 1) * planeA + (uint32_t)ks * 2 * lboA, lboA, 128),
                         tc::sdesc(aB + (uint32_t)ks * 2 * lboB, lboB, 128), id_, ks > 0 || i > 1);
      } else
      // K steps outermost, so that consecutive products go to different
      // level sums; the first product of each level overwrites its columns
      for (int ks = 0; ks < ksteps; ++ks)
        for (int L = 2; L <= tc::kSlices + 1; ++L)
          for (int i = max(1, L - tc::kSlices); i <= min(tc::kSlices, L - 1); ++i) {
            const int j = L - i;
            tc::mma_bf16(s_tmem + (uint32_t)((L - 2) * cstride),
                         tc::sdesc(aA + (uint32_t)(i - 1) * planeA + (uint32_t)ks * 2 * lboA, lboA, 128),
                         tc::sdesc(aB + (uint32_t)(j - 1) * planeB + (uint32_t)ks * 2 * lboB, lboB, 128), id_,
                         ks > 0 || i > max(1, L - tc::kSlices));
          }
      tc::commit(&s_tcbar);
    }
  };
  auto tc_wait = [&]() {
    bool ok = tc::mbar_wait(&s_tcbar, tc_phase, tc::kMaxPolls);
    if (!ok) {
      flag_error(a, TP_ERR_TIMEOUT, tent);
      tc::mbar_wait(&s_tcbar, tc_phase, 16 * tc::kMaxPolls);   // the products still in flight
    }
    tc_phase ^= 1u;
    ok = __syncthreads_and(ok) != 0;
    tc::fence_after();
    return ok;
  };
  auto tc_product = [&](uint32_t aA, uint32_t planeA, uint32_t lboA, uint32_t aB, uint32_t planeB, uint32_t lboB,
                        int ksteps, int N, int cstride) {
    tc_issue(aA, planeA, lboA, aB, planeB, lboB, ksteps, N, cstride);
    return tc_wait();
  };
  // data moments of nq bottom points (U-values in rows 0.. of sU) of a
  // single-material tent on the tensor cores:
  //   M[r, c, i] += sum_q cb[q, r, c] U_i(q)
  // A: the data coefficients, rows (r, c), scaled per row; B: the U-values,
  // rows i (padded to 32), scaled per basis function; K: the points (padded
  // to 16 with zeros, at most CH, so that the level sums stay below 2^24)
  // (tc_mom_start digit-splits the chunk and issues its products; the
  // caller evaluates the next chunk while they run; tc_mom_finish waits and
  // adds the level sums into the moments)
  auto tc_mom_start = [&](int nq) {
    if constexpr (kTC) {
      const int M = nrhs * C, RG = (M + 7) >> 3, KC = ((nq + 15) >> 4) << 1;
      uint16_t* sTA = reinterpret_cast<uint16_t*>(sm + a.off_tc);
      const int planeA = CH * RG * 8;
      uint16_t* sTB = sTA + tc::kSlices * planeA + 512;
      int* eA = s_tce[0];
      int* eB = s_tce[1];
      // two threads per row (M + nb <= 128 rows, so every thread takes part
      // once and the pair's maxima meet by one shuffle)
      {
        const int m = tid >> 1, part = tid & 1;
        float mx = 0.f;
        if (m < M) {
          for (int ql = part; ql < nq; ql += 2) mx = fmaxf(mx, fabsf(sCB[(size_t)m * cbs + ql].hi));
        } else if (m < M + nb) {
          for (int ql = part; ql < nq; ql += 2) mx = fmaxf(mx, fabsf(sU[(size_t)ql * us + (m - M)].hi));
        }
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
        if (part == 0 && m < M) eA[m] = tc::scale_exp(mx);
        if (part == 0 && m >= M && m < M + nb) eB[m - M] = tc::scale_exp(mx);
      }
      __syncthreads();
      // digit planes, one item = 8 consecutive points of one row of A or B
      for (int id = tid; id < (M + 32) * KC; id += blockDim.x) {
        const bool isA = id < M * KC;
        const int id2 = isA ? id : id - M * KC, rows = isA ? M : 32;
        const int kc = id2 / rows, m = id2 % rows;
        const bool live = isA || m < nb;
        const int ex = isA ? eA[m] : (live ? eB[m] : 0);
        float d[8][tc::kSlices];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int ql = kc * 8 + j;
          T x = R::zero();
          if (ql < nq && live) x = isA ? sCB[(size_t)m * cbs + ql] : sU[(size_t)ql * us + m];
          tc::digits(x.hi, x.lo, ex, d[j]);
        }
        if (isA) tc::store_row8(sTA + ((size_t)(kc * RG + (m >> 3)) * 64 + (m & 7) * 8), planeA, d);
        else tc::store_row8(sTB + ((size_t)(kc * 4 * tc::kSlices + (m >> 3)) * 64 + (m & 7) * 8), 4 * 64, d);
      }
      // B: the planes stacked along N, 32 rows each (planeB = 0 selects the stacked products)
      tc_issue(tc::smem_addr(sTA), (uint32_t)planeA * 2, (uint32_t)RG * 128, tc::smem_addr(sTB), 0u,
               (uint32_t)(4 * tc::kSlices) * 128, KC >> 1, 32 * tc::kSlices, 32);
    }
  };
  auto tc_mom_finish = [&]() {
    if constexpr (kTC) {
      const int M = nrhs * C;
      const int* eA = s_tce[0];
      const int* eB = s_tce[1];
      const bool ok = tc_wait();
      // levels -> float-float moments: warp w reads rows 32 (w % 4) .. + 31,
      // basis functions 16 (w / 4) .. + 15
      const int q4 = warp & 3, h = warp >> 2;
      if (ok && 32 * q4 < M) {
        const int m = 32 * q4 + lane;
        for (int c8 = 0; c8 < 2; ++c8) {
          float lv[tc::kSlices][8];
#pragma unroll
          for (int l = 0; l < tc::kSlices; ++l)
            tc::ld8(s_tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(l * 32 + 16 * h + 8 * c8), lv[l]);
          tc::wait_ld();
          if (m < M) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int i = 16 * h + 8 * c8 + j;
              if (i >= nb) continue;
              float acc[tc::kSlices];
#pragma unroll
              for (int l = 0; l < tc::kSlices; ++l) acc[l] = lv[l][j];
              T v;
              tc::combine_ff(acc, v.hi, v.lo);
              tc::ff_scale(v.hi, v.lo, eA[m] + eB[i] - 16);
              T* Mp = sPM + (size_t)m * nb + i;
              *Mp = R::add(*Mp, v);
            }
          }
        }
      }
      tc::fence_before();
      __syncthreads();   // the exponents and columns read above are rewritten by the next chunk
    }
  };
  for (int base = q0; base < q1; base += CH) {
    const int nq = min(CH, q1 - base);
    // (a) one thread per (side, point): mapped coordinates, sqrt(w), data
    // coefficients; then the U-values of all 2 nq points with the whole block
    // (point q = side * nq + ql)
    const int npt = 2 * nq;
    for (int id = tid; id < npt; id += blockDim.x) {
      const int side = id / nq, ql = id % nq, qg = base + ql;
      const int k = qg / Q, q = qg % Q;
      if (side == 0) s_pgrp[ql] = s_grp[k];
      map_point(sPt + id * (DIM + 2), k, q, side == 0);
      if (keep && side == 0) sKeepW[base - q0 + ql] = __ldg(a.isqw + q) * s_isdet[k];
    }
    // (with the right-hand sides split over the cluster the moments take a pass of their own)
    if (!rsplit) data_coefs(base, nq);
    eval_uvalues_block<DIM, T>(a, npt, sPt, sM, sU);
    if (keep)
      for (int id = tid; id < nq * nb; id += blockDim.x) sKeep[(size_t)(base - q0) * nb + id] = sU[(id / nb) * us + id % nb];
    // (b) Grams of U-values: top per element (flushed into G and H_m), bottom; per material
    for (int ql = 0; ql < nq; ++ql) {
      if (base + ql >= kend) {   // the next element's points start
        const int k = (base + ql) / Q;
        flush_element(curk);
        if (s_grp[k] != curg) {
          flush_group(curg);
          curg = s_grp[k];
        }
        curk = k;
        kend = (k + 1) * Q;
      }
      const T* ut = sU + (size_t)ql * us;
      const T* ub = sU + (size_t)(nq + ql) * us;
#pragma unroll
      for (int s = 0; s < kMaxPair; ++s) {
        if (tid + s * kThreads < npair) {
          aK[s] = R::acc(aK[s], ut[pi[s]], ut[pj[s]]);
          aB[s] = R::acc(aB[s], ub[pi[s]], ub[pj[s]]);
        }
      }
    }
    // (c) moments of the data (forward: bottom points; adjoint: top points), per material
    if (!rsplit) data_moments(nq, ADJ ? 0 : nq);
    __syncthreads();
  }
  if (q1 > q0) {
    flush_element(curk);
    flush_group(curg);
  }
  if (rsplit) {
    // this CTA's right-hand sides at every point of the patch (forward: the
    // bottom points; adjoint: the top points): the moments are complete in
    // this CTA and take no cluster reduction
    prefetch_front(0, min(CH, NP));
    for (int base = 0; base < NP; base += CH) {
      const int nq = min(CH, NP - base);
      for (int id = tid; id < nq; id += blockDim.x) {
        const int qg = base + id, k = qg / Q, q = qg % Q;
        s_pgrp[id] = s_grp[k];
        map_point(sPt + id * (DIM + 2), k, q, ADJ);
      }
      data_coefs(base, nq);
      if (base + CH < NP) prefetch_front(base + CH, min(CH, NP - base - CH));
      eval_uvalues_block<DIM, T>(a, nq, sPt, sM, sU);
      if (tc_on) {
        if (base > 0) tc_mom_finish();   // the previous chunk's products ran meanwhile
        tc_mom_start(nq);                // (its issue barrier orders this chunk's reads before the next writes)
      } else {
        data_moments(nq, 0);
        __syncthreads();
      }
    }
    if (tc_on && NP > 0) tc_mom_finish();
  }

  // ---------------- phase 2: vertical faces ----------------
  // Dirichlet facets, per material g, after the interface blocks: the facet
  // Grams summed over g's facets, G_g, and weighted by the facets' normals,
  // Gn_g[d] = sum_f n_f[d] F_f (layout [G_g | Gn_g[0..DIM)] of npair each),
  // then the data moments in the same arrangement (nrhs*nb each).  The
  // congruences with the derivative maps are linear, so these sums carry all
  // a tent needs; they are formed after the cluster reduction.
  // Interface and Neumann facets add their blocks to the partial A (N*N)
  // at once; Neumann facets also to a partial b (nrhs*N, after the
  // Dirichlet sums).
  const int nneu = NEU ? s_nneu : 0;   // (kernels for meshes without Neumann facets leave out their code)
  const bool pblk = nif > 0 || nneu > 0;
  T* sFD = sPD + (pblk ? (size_t)N * N : 0);
  T* sDD = sFD + (size_t)ng * (DIM + 1) * npair;
  const int nfd = nfac > 0 ? ng * (DIM + 1) * (npair + nrhs * nb) : 0;
  T* sPBN = sFD + nfd;
  if (extra) {
    if (pblk)
      for (int id = tid; id < N * N; id += blockDim.x) sPD[id] = R::zero();
    for (int id = tid; id < nfd; id += blockDim.x) sFD[id] = R::zero();
    if (nneu > 0)
      for (int id = tid; id < nrhs * N; id += blockDim.x) sPBN[id] = R::zero();
    for (int id = tid; id < nrhs * nb; id += blockDim.x) sDel[id] = R::zero();
    if (nif > 0)
      for (int id = tid; id < nb * nb; id += blockDim.x) sFpm[id] = R::zero();
    __syncthreads();
    // (a) Dirichlet facets: the points of all of them (facet after facet) in
    // one pass, split over the cluster; a facet's Gram and moments are folded
    // into its material's sums where its points end
    if (nfac > 0) {
      const int NPD = nfac * Q, dsl = (NPD + CS - 1) / CS;
      const int d0 = min(NPD, rank * dsl), d1 = min(NPD, d0 + dsl);
      // the Grams take this CTA's slice [d0, d1); the data moments of split
      // right-hand sides take every point
      const int l0 = rsplit ? 0 : d0, l1 = rsplit ? NPD : d1;
      T aF[kMaxPair];
#pragma unroll
      for (int s = 0; s < kMaxPair; ++s) aF[s] = R::zero();
      auto fold_gram = [&](int f) {
        if (f >= nfac) return;
        T* Fg = sFD + (size_t)s_fg[f] * (DIM + 1) * npair;
#pragma unroll
        for (int s = 0; s < kMaxPair; ++s)
          if (tid + s * kThreads < npair) {
            const int q = tid + s * kThreads;
            Fg[q] = R::add(Fg[q], aF[s]);
            for (int d = 0; d < DIM; ++d)
              Fg[(1 + d) * npair + q] = R::fma(R::from(s_fn[f][d]), aF[s], Fg[(1 + d) * npair + q]);
            aF[s] = R::zero();
          }
      };
      auto fold_mom = [&](int f, int id, T t) {
        if (f >= nfac) return;
        T* Dg = sDD + (size_t)s_fg[f] * (DIM + 1) * nrhs * nb;
        Dg[id] = R::add(Dg[id], t);
        for (int d = 0; d < DIM; ++d)
          Dg[(1 + d) * nrhs * nb + id] = R::fma(R::from(s_fn[f][d]), t, Dg[(1 + d) * nrhs * nb + id]);
      };
      int fc = l0 / Q;   // facet of the points being accumulated (uniform over the CTA)
      for (int base = l0; base < l1; base += CH) {
        const int nq = min(CH, l1 - base);
        for (int id = tid; id < nq; id += blockDim.x) {
          const int q = base + id, f = q / Q, qf = q - f * Q;
          double xt[DIM + 1];
          for (int d = 0; d <= DIM; ++d) xt[d] = 0.0;
          for (int i = 0; i < NV; ++i) {
            const double l = __ldg(a.bary + qf * NV + i);
            for (int d = 0; d <= DIM; ++d) xt[d] = fma(l, s_fP[f][i][d], xt[d]);
          }
          const double sw = __ldg(a.sqw + qf) * s_fsq[f];
          T* pp = sPt + id * (DIM + 2);
          pp[0] = R::from(s_gc[s_fg[f]] * (xt[DIM] - tc) * ih);
          for (int d = 0; d < DIM; ++d) pp[1 + d] = R::from((xt[d] - s_xv[d]) * ih);
          pp[DIM + 1] = R::from(sw);
          // the facet's block of boundary data (without Neumann facets: the facet's own index)
          const long long goff = a.tent_gdoff[tent] + (NEU ? (long long)s_fw[f][0] * Q + qf : (long long)q);
          for (int r = 0; r < nrhs; ++r)
            sGd[id * nrhs + r] = R::from((!ADJ && gD != nullptr) ? sw * gD[(long long)r * a.n_bnd + goff] : 0.0);
        }
        eval_uvalues_block<DIM, T>(a, nq, sPt, sM, sU);
        const int fc0 = fc;
        for (int ql = 0; ql < nq; ++ql) {
          if (base + ql >= (fc + 1) * Q) fold_gram(fc++);
          if (base + ql < d0 || base + ql >= d1) continue;   // another CTA's Gram points
          const T* u = sU + (size_t)ql * us;
#pragma unroll
          for (int s = 0; s < kMaxPair; ++s)
            if (tid + s * kThreads < npair) aF[s] = R::fma(u[pi[s]], u[pj[s]], aF[s]);
        }
        for (int id = tid; id < nrhs * nb; id += blockDim.x) {
          const int r = id / nb, i = id % nb;
          int f = fc0;
          T t = sDel[id];
          for (int ql = 0; ql < nq; ++ql) {
            if (base + ql >= (f + 1) * Q) {
              fold_mom(f++, id, t);
              t = R::zero();
            }
            t = R::fma(sGd[ql * nrhs + r], sU[(size_t)ql * us + i], t);
          }
          sDel[id] = t;
        }
        __syncthreads();
      }
      fold_gram(fc);
      for (int id = tid; id < nrhs * nb; id += blockDim.x) {
        fold_mom(fc, id, sDel[id]);
        sDel[id] = R::zero();
      }
      __syncthreads();
    }
    // (b) time-like interface facets, then Neumann facets, one after the
    // other, each facet's points split over the cluster; their blocks go into
    // the partial A at once.  Neumann facets (eq. 4.1), with F the facet Gram
    // of U-values and delta = sum w g_N u:
    //   A_N = -(c/h^2) D_n F D_t^T + (beta/h^2) D_n F D_n^T,
    //   b_N = -(c/h) D_t delta - (beta/h) D_n delta
    // (v = (c/h) D_t u, sigma.n = -(1/h) D_n u, D_n = sum_m n_m D_m)
    const int fsl = (Q + CS - 1) / CS;
    const int f0 = min(Q, rank * fsl), f1 = min(Q, f0 + fsl);
    for (int f = nfac; f < nfac + nif + nneu; ++f) {
      const bool neu = NEU && f >= nfac + nif;
      const int gp = s_fg[f], gm = s_fg2[f];
      const double cp = s_gc[gp], cm = s_gc[gm];
      T aF[kMaxPair], aF2[kMaxPair];
#pragma unroll
      for (int s = 0; s < kMaxPair; ++s) aF[s] = aF2[s] = R::zero();
      // (a Neumann facet's data moments of split right-hand sides take every point)
      const int l0 = (rsplit && neu) ? 0 : f0, l1 = (rsplit && neu) ? Q : f1;
      for (int base = l0; base < l1; base += CH) {
        const int nq = min(CH, l1 - base);
        const int npt = neu ? nq : 2 * nq;   // interface: + side points, then - side
        for (int id = tid; id < nq; id += blockDim.x) {
          const int q = base + id;
          double xt[DIM + 1];
          for (int d = 0; d <= DIM; ++d) xt[d] = 0.0;
          for (int i = 0; i < NV; ++i) {
            const double l = __ldg(a.bary + q * NV + i);
            for (int d = 0; d <= DIM; ++d) xt[d] = fma(l, s_fP[f][i][d], xt[d]);
          }
          const double sw = __ldg(a.sqw + q) * s_fsq[f];
          T* pp = sPt + id * (DIM + 2);
          pp[0] = R::from(cp * (xt[DIM] - tc) * ih);
          for (int d = 0; d < DIM; ++d) pp[1 + d] = R::from((xt[d] - s_xv[d]) * ih);
          pp[DIM + 1] = R::from(sw);
          if (neu) {
            const long long goff = a.tent_gdoff[tent] + (long long)s_fw[f][0] * Q + q;
            for (int r = 0; r < nrhs; ++r)
              sGd[id * nrhs + r] = R::from((!ADJ && gD != nullptr) ? sw * gD[(long long)r * a.n_bnd + goff] : 0.0);
          } else {
            T* p2 = sPt + (nq + id) * (DIM + 2);
            p2[0] = R::from(cm * (xt[DIM] - tc) * ih);
            for (int d = 0; d < DIM; ++d) p2[1 + d] = pp[1 + d];
            p2[DIM + 1] = pp[DIM + 1];
          }
        }
        eval_uvalues_block<DIM, T>(a, npt, sPt, sM, sU);
        for (int ql = 0; ql < nq; ++ql) {
          if (base + ql < f0 || base + ql >= f1) continue;   // another CTA's Gram points
          const T* u = sU + (size_t)ql * us;
          const T* u2 = sU + (size_t)(nq + ql) * us;
#pragma unroll
          for (int s = 0; s < kMaxPair; ++s)
            if (tid + s * kThreads < npair) {
              aF[s] = R::fma(u[pi[s]], u[pj[s]], aF[s]);
              if (!neu) aF2[s] = R::fma(u2[pi[s]], u2[pj[s]], aF2[s]);
            }
        }
        if (neu) {
          for (int id = tid; id < nrhs * nb; id += blockDim.x) {
            const int r = id / nb, i = id % nb;
            T t = sDel[id];
            for (int ql = 0; ql < nq; ++ql) t = R::fma(sGd[ql * nrhs + r], sU[(size_t)ql * us + i], t);
            sDel[id] = t;
          }
        } else {
          for (int id = tid; id < nb * nb; id += blockDim.x) {
            const int i = id / nb, j = id % nb;
            T t = sFpm[id];
            for (int ql = 0; ql < nq; ++ql) t = R::fma(sU[(size_t)ql * us + i], sU[(size_t)(nq + ql) * us + j], t);
            sFpm[id] = t;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int s = 0; s < kMaxPair; ++s)
        if (tid + s * kThreads < npair) {
          sF[tid + s * kThreads] = aF[s];
          sF2[tid + s * kThreads] = aF2[s];
        }
      __syncthreads();
      T nrm[DIM];
      for (int d = 0; d < DIM; ++d) nrm[d] = R::from(s_fn[f][d]);
      if (neu) {
        const double ih2 = ih * ih;
        for (int id = tid; id < nb * nb; id += blockDim.x) {
          const int i = id / nb, j = id % nb;
          T tt_, nt_, tn_, nn_;
          iface_terms<DIM, T, 0>(a, i, j, sF, nb, nrm, &tt_, &nt_, &tn_, &nn_);
          const T t = R::fma(R::from(-cp * ih2), nt_, R::mul(R::from(a.beta * ih2), nn_));
          T* dst = sPD + (size_t)(gp * nb + i) * N + gp * nb + j;
          *dst = R::add(*dst, t);
        }
        for (int id = tid; id < nrhs * nb; id += blockDim.x) {
          const int r = id / nb, i = id % nb;
          const T* del = sDel + (size_t)r * nb;
          T dn = R::zero();
          for (int d = 0; d < DIM; ++d) dn = R::fma(nrm[d], rel_apply<DIM, T>(a, i, 1 + d, del), dn);
          const T t = R::fma(R::from(-a.beta * ih), dn, R::mul(R::from(-cp * ih), rel_apply<DIM, T>(a, i, 0, del)));
          T* dst = sPBN + (size_t)r * N + gp * nb + i;
          *dst = R::add(*dst, t);
        }
        __syncthreads();
        for (int id = tid; id < nrhs * nb; id += blockDim.x) sDel[id] = R::zero();
        __syncthreads();
        continue;
      }
      {
        const double ih2 = ih * ih;
        for (int id = tid; id < 4 * nb * nb; id += blockDim.x) {
          const int blk = id / (nb * nb), rem = id % (nb * nb), i = rem / nb, j = rem % nb;
          const int tside = blk >> 1, sside = blk & 1;   // 0: +, 1: -
          const double st = tside ? -1.0 : 1.0, ss = sside ? -1.0 : 1.0;
          const double ct = tside ? cm : cp, cs = sside ? cm : cp;
          T tt_, nt_, tn_, nn_;
          if (tside == sside) {
            iface_terms<DIM, T, 0>(a, i, j, tside ? sF2 : sF, nb, nrm, &tt_, &nt_, &tn_, &nn_);
          } else if (tside == 0) {
            iface_terms<DIM, T, 1>(a, i, j, sFpm, nb, nrm, &tt_, &nt_, &tn_, &nn_);
          } else {
            iface_terms<DIM, T, 2>(a, i, j, sFpm, nb, nrm, &tt_, &nt_, &tn_, &nn_);
          }
          T t = R::mul(R::from(-0.5 * st * cs * ih2), nt_);
          t = R::fma(R::from(-0.5 * st * ct * ih2), tn_, t);
          t = R::fma(R::from(st * ss * a.alpha * cs * ct * ih2), tt_, t);
          t = R::fma(R::from(st * ss * a.beta * ih2), nn_, t);
          const int gr = tside ? gm : gp, gcl = sside ? gm : gp;
          T* dst = sPD + (size_t)(gr * nb + i) * N + gcl * nb + j;
          *dst = R::add(*dst, t);
        }
      }
      __syncthreads();
      for (int id = tid; id < nb * nb; id += blockDim.x) sFpm[id] = R::zero();
      __syncthreads();
    }
  }

  // ---------------- cluster reduction (rank order) ----------------
  // every CTA sums every CTA's partials in rank order (all remote loads of an
  // entry are issued before the additions)
  auto cluster_sum = [&](T* src, int id) {
    T t = R::zero();
    for (int r0 = 0; r0 < CS; r0 += 4) {
      T v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r0 + u < CS) v[u] = cluster.map_shared_rank(src, r0 + u)[id];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r0 + u < CS) t = R::add(t, v[u]);
    }
    return t;
  };
  // reduce-scatter: rank r sums its share of every array over the cluster and
  // stores the sums into every CTA's copy
  auto cluster_reduce = [&](T* part, T* sum, int n) {
    const int lo = (n * rank) / CS, hi = (n * (rank + 1)) / CS;
    for (int id = lo + tid; id < hi; id += blockDim.x) {
      const T t = cluster_sum(part, id);
      for (int rr = 0; rr < CS; ++rr) cluster.map_shared_rank(sum, rr)[id] = t;
    }
  };
  cluster.sync();
  // layout [G (NG*npair) | H_m (NG*DIM*npair) | Gbot (NG*npair)]; unused groups hold zeros
  cluster_reduce(sPG, sSG, NG * (DIM + 2) * npair);
  // (split right-hand sides: each CTA's moments, Dirichlet data sums and
  // Neumann partial b already cover every point for its own right-hand sides)
  if (!rsplit) cluster_reduce(sPM, sSM, ng * nmom);   // in place (sSM == sPM): each entry has one owner
  if (pblk) cluster_reduce(sPD, sA, N * N);   // interface and Neumann blocks
  else
    for (int id = tid; id < N * N; id += blockDim.x) sA[id] = R::zero();
  if (NEU && s_nneu > 0) {   // Neumann data (after the Dirichlet sums)
    if (rsplit)
      for (int id = tid; id < nrhs * N; id += blockDim.x) sb[id] = sFD[nfd + id];
    else
      cluster_reduce(sFD + nfd, sb, nrhs * N);
  } else {
    for (int id = tid; id < nrhs * N; id += blockDim.x) sb[id] = R::zero();
  }
  // in place: each entry is read and rewritten by the one thread that owns it
  if (nfac > 0) cluster_reduce(sFD, sFD, rsplit ? ng * (DIM + 1) * npair : nfd);
  cluster.sync();   // no CTA leaves or reuses its partials while another still reads them
  // congruence: rank r forms rows [N r / CS, N (r + 1) / CS) of A and b and
  // stores them into rank 0's A and b; rank 0 alone solves.  Every CTA holds
  // the same summed partials, so the rows do not depend on which rank forms them.
  T* A0 = cluster.map_shared_rank(sA, 0);
  T* b0 = cluster.map_shared_rank(sb, 0);
  const int row0 = (N * rank) / CS, nrow = (N * (rank + 1)) / CS - row0;
  {
    const T ih2 = R::from(ih * ih), mih = R::from(-ih);
    // top-face form of every material block by the merged tables: entries
    // i <= j of the packed upper triangle, split over the cluster; each entry
    // is stored with its mirror (the form is symmetric, the Dirichlet and
    // interface parts already in A are not)
    const int nent = ng * npair, ent0 = (nent * rank) / CS, ent1 = (nent * (rank + 1)) / CS;
    unsigned gdir = 0;   // materials with Dirichlet facets
    for (int f = 0; f < nfac; ++f) gdir |= 1u << s_fg[f];
    if (nfac > 0) {
      // Dirichlet facets, A_D = (c/h) D_t F E^T with E = alpha (c/h) D_t - (1/h) D_n
      // summed over the material's facets, from G_g and Gn_g, added into this
      // CTA's copy of A for the entries this rank forms (each entry and its
      // mirror: one item each)
      for (int id = tid; id < 2 * (ent1 - ent0); id += blockDim.x) {
        const int e_ = ent0 + (id >> 1), g = e_ / npair, pp = e_ % npair;
        const int ij = __ldg(a.pair_ij + pp);
        int i = ij >> 16, j = ij & 0xffff;
        if (((id & 1) && i == j) || !((gdir >> g) & 1u)) continue;
        if (id & 1) {
          const int t_ = i;
          i = j;
          j = t_;
        }
        const int e2 = i * nb + j;
        const T* Fg = sFD + (size_t)g * (DIM + 1) * npair;
        T a0 = R::zero(), am = R::zero();
        for (int e = __ldg(a.ft_ptr + e2), e1 = __ldg(a.ft_ptr + e2 + 1); e < e1; ++e)
          a0 = Fac<T>::acc(a0, Fg[__ldg(a.ft_idx + e)], a.ft_coef, a.ft_coefd, e);
        for (int e = __ldg(a.fm_ptr + e2), e1 = __ldg(a.fm_ptr + e2 + 1); e < e1; ++e) {
          const int c0 = __ldg(a.fm_idx + e);   // (derivative direction << 16) | pair
          am = Fac<T>::acc(am, Fg[(size_t)(1 + (c0 >> 16)) * npair + (c0 & 0xffff)], a.fm_coef, a.fm_coefd, e);
        }
        const double cf = s_gc[g];
        const T ad = R::mul(R::from(cf * ih), R::fma(mih, R::norm(am), R::mul(R::from(a.alpha * cf * ih), R::norm(a0))));
        const size_t o = (size_t)(g * nb + i) * N + g * nb + j;
        sA[o] = R::add(sA[o], ad);
      }
      __syncthreads();
    }
    for (int id = ent0 + tid; id < ent1; id += blockDim.x) {
      const int g = id / npair, pp = id % npair;
      const int ij = __ldg(a.pair_ij + pp), i = ij >> 16, j = ij & 0xffff;
      const T* SG = sSG + (size_t)g * npair;
      const T* SH = sSG + (size_t)(NG + g * DIM) * npair;
      const T* SGb = sSG + (size_t)(NG * (DIM + 1) + g) * npair;
      T tg0 = R::zero(), tg1 = R::zero(), th0 = R::zero(), th1 = R::zero();
      {
        const int e0 = __ldg(a.cg_ptr + pp), e1 = __ldg(a.cg_ptr + pp + 1);
        int e = e0;
        for (; e + 1 < e1; e += 2) {
          tg0 = Fac<T>::acc(tg0, SG[__ldg(a.cg_idx + e)], a.cg_coef, a.cg_coefd, e);
          tg1 = Fac<T>::acc(tg1, SG[__ldg(a.cg_idx + e + 1)], a.cg_coef, a.cg_coefd, e + 1);
        }
        if (e < e1) tg0 = Fac<T>::acc(tg0, SG[__ldg(a.cg_idx + e)], a.cg_coef, a.cg_coefd, e);
      }
      {
        const int e0 = __ldg(a.ch_ptr + pp), e1 = __ldg(a.ch_ptr + pp + 1);
        int e = e0;
        for (; e + 1 < e1; e += 2) {
          const int c0 = __ldg(a.ch_idx + e), c1 = __ldg(a.ch_idx + e + 1);
          th0 = Fac<T>::acc(th0, SH[(c0 >> 16) * npair + (c0 & 0xffff)], a.ch_coef, a.ch_coefd, e);
          th1 = Fac<T>::acc(th1, SH[(c1 >> 16) * npair + (c1 & 0xffff)], a.ch_coef, a.ch_coefd, e + 1);
        }
        if (e < e1) {
          const int c0 = __ldg(a.ch_idx + e);
          th0 = Fac<T>::acc(th0, SH[(c0 >> 16) * npair + (c0 & 0xffff)], a.ch_coef, a.ch_coefd, e);
        }
      }
      const T t = R::fma(R::from(s_gc[g]), R::add(R::norm(th0), R::norm(th1)), R::add(R::norm(tg0), R::norm(tg1)));
      const T val = R::fma(ih2, t, SGb[pp]);
      const size_t o = (size_t)(g * nb + i) * N + g * nb + j;
      A0[o] = R::add(sA[o], val);
      if (i != j) {
        const size_t o2 = (size_t)(g * nb + j) * N + g * nb + i;
        A0[o2] = R::add(sA[o2], val);
      }
    }
    // (split right-hand sides: every row of this CTA's own b, kept in this CTA)
    const int brow0 = rsplit ? 0 : row0, bnrow = rsplit ? N : nrow;
    T* const bdst = rsplit ? sb : b0;
    for (int id = tid; id < nrhs * bnrow; id += blockDim.x) {
      const int r = id / bnrow, Rw = brow0 + id % bnrow;
      const int g = Rw / nb, i = Rw % nb;
      const T* M = sSM + (size_t)g * nmom + (size_t)r * C * nb;   // gamma, alpha, beta_1..beta_n
      T t = R::fma(R::from(s_gc[g] * ih), rel_apply<DIM, T>(a, i, 0, M + nb), M[i]);
      for (int d = 0; d < DIM; ++d) t = R::fma(mih, rel_apply<DIM, T>(a, i, 1 + d, M + (2 + d) * nb), t);
      // Dirichlet data: b_D = E' delta summed over g's facets,
      // E' = alpha (c/h) D_t + (1/h) D_n
      if ((gdir >> g) & 1u) {
        const T* Dg = sDD + (size_t)g * (DIM + 1) * nrhs * nb + (size_t)r * nb;
        T dn = rel_apply<DIM, T>(a, i, 1, Dg + (size_t)nrhs * nb);
        for (int d = 1; d < DIM; ++d) dn = R::add(dn, rel_apply<DIM, T>(a, i, 1 + d, Dg + (size_t)(1 + d) * nrhs * nb));
        const T ac = R::from(a.alpha * s_gc[g] * ih);
        t = R::add(t, R::fma(R::from(ih), dn, R::mul(ac, rel_apply<DIM, T>(a, i, 0, Dg))));
      }
      const size_t o = (size_t)r * N + Rw;
      bdst[o] = R::add(sb[o], t);
    }
  }
  cluster.sync();   // rank 0 holds the assembled A and b
  if (rsplit) {
    // every CTA solves for its own right-hand sides with its own copy of A
    if (rank != 0)
      for (int id = tid; id < N * N; id += blockDim.x) sA[id] = A0[id];
    cluster.sync();   // rank 0's A is read before any CTA's solve overwrites its own
  }
  if (rank == 0 || rsplit) {
  if constexpr (ADJ) {   // solve with A^T
    for (int id = tid; id < N * N; id += blockDim.x) {
      const int i = id / N, j = id % N;
      if (i < j) {
        const T t = sA[id];
        sA[id] = sA[j * N + i];
        sA[j * N + i] = t;
      }
    }
    __syncthreads();
  }

  // ---------------- phase 3: solve ----------------
  // Both precisions: the equilibrated matrix D A D (D = |diag A|^-1/2) is
  // inverted in binary32 by Gauss-Jordan without row interchanges, then
  // x += D F D (b - A x) with the residual in the path's precision (binary64,
  // or float-float for MIXED) until the correction stops shrinking; a
  // refinement that does not settle falls back to a direct binary64 LU.
  // Every tent matrix has a positive definite symmetric part (testing the
  // tent system with V = U_h gives x^T A x = 1/2 int_top Q_g(u) + 1/2 int_bot
  // Q_g(u_b) + int_bot U^2 + the dissipative boundary and interface terms > 0),
  // and so has each of its Schur complements: elimination without
  // interchanges does not break down.  The direct LU of the fallback keeps
  // partial pivoting on Dirichlet and interface tents.
  const bool lu_pivoting = extra || ng > 1;
  bool refined = false;
  {
    float* sG = reinterpret_cast<float*>(sm + a.off_al);    // 2*N*N   ping-pong sweep buffers
    float* sEq = reinterpret_cast<float*>(sm + a.off_eq);   // N       equilibration scales
    float* sZ = reinterpret_cast<float*>(sm + a.off_z);     // nrhs*N  scaled residual (binary32)
    T* sX = reinterpret_cast<T*>(sm + a.off_x);             // nrhs*N  iterate
    // register path with room for the right-hand sides: D b rides along as
    // extra columns (lanes N .. N + nrhs - 1) and the elimination leaves the
    // first iterate (D A D)^-1 D b in them
    const bool regs = N <= 32, aug = regs && N + nrhs <= 32;
    for (int i = tid; i < N; i += blockDim.x) {
      const float d = fabsf(R::hi(sA[i * N + i]));
      sEq[i] = (d > 0.f && isfinite(d)) ? rsqrtf(d) : 1.f;
    }
    // (items from warp 1 on, beside warp 0's scales)
    for (int id = (tid + kThreads - 32) % kThreads; id < nrhs * N; id += blockDim.x) {
      sX[id] = R::zero();
      if (aug) {   // the same scale as sEq, formed here so that one barrier suffices
        const float d = fabsf(R::hi(sA[(id % N) * (N + 1)]));
        sZ[id] = ((d > 0.f && isfinite(d)) ? rsqrtf(d) : 1.f) * R::hi(sb[id]);
      }
    }
    __syncthreads();
    auto bad_pivot = [&](float pv) {
      // binary64: the refinement then fails and the direct LU decides
      if (!(fabsf(pv) > 0.f) || !isfinite(pv)) {
        if (MIXED && lane == 0) flag_error(a, TP_ERR_SINGULAR, tent);
        return true;
      }
      return false;
    };
    // register path (N <= 32): row warp + 8 s of the sweep matrix in gr[s],
    // column = lane.  Blocks of four steps K = {k..k+3} per barrier: with S_K
    // the block's pivot rows at its start, every warp reduces S_K by the four
    // steps itself (P = [S_KK^-1 | S_KK^-1 S_KJ] in the pivot and the other
    // columns), and a row i outside K becomes
    //   (columns of K set to 0, the others kept) - sum_b s_{i,k+b} P_b,
    // which is the four single steps taken at once (block Gauss-Jordan).
    float gr[4] = {0.f, 0.f, 0.f, 0.f};
    if (regs) {
#pragma unroll
      for (int s_ = 0; s_ < 4; ++s_) {
        const int i = warp + 8 * s_;
        if (i < N && lane < N) gr[s_] = R::hi(sA[i * N + lane]) * sEq[i] * sEq[lane];
        else if (aug && i < N && lane < N + nrhs) gr[s_] = sZ[(lane - N) * N + i];
      }
      for (int k = 0, blk = 0; k < N; k += 4, ++blk) {
        const int kb = min(4, N - k);
        float(*pb)[32] = s_pb[blk & 1];
        // the owners publish the block's pivot rows (rows k..k+3 are on warps
        // (k & 7) .. (k & 7) + 3, slot k >> 3)
        if (warp >= (k & 7) && warp < (k & 7) + kb) {
          const int s_ = k >> 3;
          pb[warp - (k & 7)][lane] = s_ == 0 ? gr[0] : s_ == 1 ? gr[1] : s_ == 2 ? gr[2] : gr[3];
        }
        // this warp's rows in the pivot columns (block-start values)
        float ml[4][4];
#pragma unroll
        for (int s_ = 0; s_ < 4; ++s_)
#pragma unroll
          for (int b = 0; b < 4; ++b) ml[s_][b] = __shfl_sync(0xffffffffu, gr[s_], k + b);
        __syncthreads();
        float P[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) P[b] = b < kb ? pb[b][lane] : 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (b >= kb) break;
          const int kc = k + b;
          float mm[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) mm[c] = __shfl_sync(0xffffffffu, P[c], kc);
          float pv = mm[b];
          if (bad_pivot(pv)) pv = 1.f;
          const float rp = rcp_fast(pv);
          const float pn = (lane == kc) ? rp : P[b] * rp;
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (c != b) P[c] = fmaf(-mm[c], pn, lane == kc ? 0.f : P[c]);
          P[b] = pn;
        }
        const bool kcol = lane >= k && lane < k + kb;
#pragma unroll
        for (int s_ = 0; s_ < 4; ++s_) {
          const int i = warp + 8 * s_;
          const int bi = i - k;
          if (bi >= 0 && bi < kb) {
            gr[s_] = bi == 0 ? P[0] : bi == 1 ? P[1] : bi == 2 ? P[2] : P[3];
          } else {
            float x = kcol ? 0.f : gr[s_];
#pragma unroll
            for (int b = 0; b < 4; ++b) x = fmaf(-ml[s_][b], P[b], x);
            gr[s_] = x;
          }
        }
      }
    } else {
      for (int id = tid; id < N * N; id += blockDim.x) sG[id] = R::hi(sA[id]) * sEq[id / N] * sEq[id % N];
      __syncthreads();
      // Gauss-Jordan sweeps: step k reads buffer k % 2 and writes buffer
      // (k + 1) % 2; the final buffer holds F = (D A D)^-1
      for (int k = 0; k < N; ++k) {
        const float* S = sG + (size_t)(k & 1) * N * N;
        float* Gn = sG + (size_t)((k + 1) & 1) * N * N;
        float pv = S[k * N + k];
        if (bad_pivot(pv)) pv = 1.f;
        const float rp = rcp_fast(pv);
        for (int i = warp; i < N; i += kThreads / 32) {   // rows over warps, columns over lanes
          const float lik = -S[i * N + k] * rp;
          for (int j = lane; j < N; j += 32) {
            float g;
            if (i == k) g = (j == k) ? rp : S[k * N + j] * rp;
            else if (j == k) g = lik;
            else g = fmaf(lik, S[k * N + j], S[i * N + j]);
            Gn[i * N + j] = g;
          }
        }
        __syncthreads();
      }
    }
    const float* F = sG + (size_t)(N & 1) * N * N;
    __syncthreads();
    // refinement
    float prev = 3.4e38f;
    const int maxit = min(a.max_refine, kMaxRefine);
    for (int it = 0; it < maxit; ++it) {
      // residual b - A x, each row split over 8 lanes of one warp; stored
      // scaled by D in binary32 (the first iterate is x = 0: the residual is b)
      if (it == 0 && aug) {
        // the first iterate from the extra columns: x = D (D A D)^-1 D b
#pragma unroll
        for (int s_ = 0; s_ < 4; ++s_) {
          const int i = warp + 8 * s_;
          if (i < N && lane >= N && lane < N + nrhs) sZ[(lane - N) * N + i] = sEq[i] * gr[s_];
        }
        __syncthreads();
        float dmax = 0.f;
        for (int id = tid; id < nrhs * N; id += blockDim.x) {
          const float dx = sZ[id];
          sX[id] = R::addf(sX[id], dx);
          dmax = fmaxf(dmax, fabsf(dx));
        }
        for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        if (lane == 0) s_red[1][warp] = dmax;
        __syncthreads();
        continue;
      }
      if (it == 0)
        for (int id = tid; id < nrhs * N; id += blockDim.x) sZ[id] = sEq[id % N] * R::hi(sb[id]);
      for (int base4 = 0; base4 < (it == 0 ? 0 : nrhs * N * 4); base4 += blockDim.x) {
        const int id = base4 + tid, item = id >> 2, sub = id & 3;
        T t = R::zero();
        if (item < nrhs * N) {
          const int r = item / N, i = item % N;
          const T* xr = sX + (size_t)r * N;
          for (int j = sub; j < N; j += 4) t = R::accn(t, sA[i * N + j], xr[j]);
          t = R::norm(t);
        }
        for (int o = 2; o > 0; o >>= 1) {
          T u;
          if constexpr (MIXED) {
            u.hi = __shfl_xor_sync(0xffffffffu, t.hi, o);
            u.lo = __shfl_xor_sync(0xffffffffu, t.lo, o);
          } else {
            u = __shfl_xor_sync(0xffffffffu, t, o);
          }
          t = R::add(t, u);
        }
        if (sub == 0 && item < nrhs * N) sZ[item] = sEq[item % N] * R::hi(R::add(sb[item], t));
      }
      __syncthreads();
      // x += D F r: register path, one row per (warp, slot), summed over lanes
      // (the scale |x| of the stop test is taken from the first iterate)
      float dmax = 0.f;
      if (regs) {
        for (int r = 0; r < nrhs; ++r) {
          const float vj = (lane < N) ? sZ[(size_t)r * N + lane] : 0.f;
          float zs = 0.f;   // lane s_ < 4 ends with the sum of slot s_
#pragma unroll
          for (int s_ = 0; s_ < 4; ++s_) {
            float z = gr[s_] * vj;
            for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
            if (lane == s_) zs = z;
          }
          // one update instruction per warp for its (up to) four rows
          const int i = warp + 8 * lane;
          if (lane < 4 && i < N) {
            const float dx = sEq[i] * zs;
            const size_t o_ = (size_t)r * N + i;
            sX[o_] = R::addf(sX[o_], dx);
            dmax = fmaxf(dmax, fabsf(dx));
          }
        }
      }
      // shared-memory path: each row split over 8 lanes
      for (int base8 = 0; base8 < (regs ? 0 : nrhs * N * 8); base8 += blockDim.x) {
        const int id = base8 + tid, item = id >> 3, sub = id & 7;
        float z = 0.f;
        if (item < nrhs * N) {
          const int r = item / N, i = item % N;
          const float* zr = sZ + (size_t)r * N;
          for (int j = sub; j < N; j += 8) z = fmaf(F[i * N + j], zr[j], z);
        }
        for (int o = 4; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        if (sub == 0 && item < nrhs * N) {
          const float dx = sEq[item % N] * z;
          sX[item] = R::addf(sX[item], dx);
          dmax = fmaxf(dmax, fabsf(dx));
        }
      }
      for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
      if (it == 0) {   // the first correction is the whole binary32 solution: no test
        if (lane == 0) s_red[1][warp] = dmax;
        __syncthreads();
        continue;
      }
      if (lane == 0) s_red[0][warp] = dmax;
      __syncthreads();
      float dm = 0.f, xm = 0.f;
      for (int w = 0; w < kThreads / 32; ++w) {
        dm = fmaxf(dm, s_red[0][w]);
        xm = fmaxf(xm, s_red[1][w]);
      }
      // stop once the correction is at the resolution of the residual's
      // precision, or once it stops shrinking at a small level (the residual's
      // rounding then limits the accuracy)
      // (a correction that stalls above floor_ of the solution, or no
      // convergence in kMaxRefine steps, sends the tent to the direct LU)
      const float tiny = MIXED ? 4e-15f : 2.5e-16f, floor_ = MIXED ? 1e-10f : 1e-12f;
      const float stall = 0.5f;
      if (!(isfinite(dm) && isfinite(xm))) break;   // the direct LU decides
      // (the next correction is predicted as dm * (dm / prev) once the
      // corrections shrink fast; stop when that is below the resolution too)
      const bool done = dm <= tiny * xm || (it >= 2 && dm > stall * prev && dm <= floor_ * xm) ||
                        (it >= 2 && dm <= 0.01f * prev && 4.f * dm * (dm / prev) <= tiny * xm);
      prev = dm;
      if (done) {
        refined = true;
        if (a.solve_stats != nullptr && tid == 0) atomicAdd(a.solve_stats + 1 + min(it + 1, kMaxRefine), 1ull);
        break;
      }
      // (the next iteration writes s_red only after its first barrier)
    }
    if (refined) {
      __syncthreads();
      for (int id = tid; id < nrhs * N; id += blockDim.x) sb[id] = sX[id];
      __syncthreads();
    }
  }
  if (!refined) {   // direct binary64 LU (the mixed path converts A and b to binary64 first)
    if (a.solve_stats != nullptr && tid == 0) atomicAdd(a.solve_stats, 1ull);
    __syncthreads();
    double* dA = reinterpret_cast<double*>(sA);   // in place: a float-float pair and a double share 8 bytes
    double* db = reinterpret_cast<double*>(sb);
    if constexpr (MIXED) {
      for (int id = tid; id < N * N; id += blockDim.x) {
        const T v = sA[id];
        dA[id] = R::to(v);
      }
      for (int id = tid; id < nrhs * N; id += blockDim.x) {
        const T v = sb[id];
        db[id] = R::to(v);
      }
      __syncthreads();
    }
    double* sXd = reinterpret_cast<double*>(sm + a.off_x);   // nrhs*N  solution during back substitution
    auto pivot_recip = [&](double piv, int k) {
      if (!(fabs(piv) > 0.0) || !isfinite(piv)) {
        flag_error(a, TP_ERR_SINGULAR, tent);
        piv = 1.0;
      }
      sRD[k] = recip(piv);
    };
    if (!lu_pivoting) {
      // A is symmetric positive definite: LU without interchanges, b eliminated
      // alongside, one barrier per step.  Step k updates rows and columns > k;
      // every thread forms the multiplier a_ik / a_kk it needs, and the thread
      // that updates a_{k+1,k+1} forms the next reciprocal pivot.
      if (tid == 0) pivot_recip(dA[0], 0);
      __syncthreads();
      for (int k = 0; k + 1 < N; ++k) {
        const double rp = sRD[k];
        const int rem = N - k - 1, wdt = rem + nrhs;
        for (int id = tid; id < rem * wdt; id += blockDim.x) {
          const int i = k + 1 + id / wdt, jj = id % wdt;
          const double l = dA[i * N + k] * rp;
          if (jj < rem) {
            const int j = k + 1 + jj;
            const double t = fma(-l, dA[k * N + j], dA[i * N + j]);
            dA[i * N + j] = t;
            if (id == 0) pivot_recip(t, k + 1);
          } else {
            const int r = jj - rem;
            db[r * N + i] = fma(-l, db[r * N + k], db[r * N + i]);
          }
        }
        __syncthreads();
      }
    } else {
      // LU with partial pivoting (Dirichlet and interface tents), b eliminated alongside
      for (int k = 0; k < N; ++k) {
        if (warp == 0) {
          // |a_ik| compared through the bit patterns (non-negative doubles order as integers)
          unsigned long long best = 0ull;
          int bi = k;
          for (int i = k + lane; i < N; i += 32) {
            const unsigned long long bits = (unsigned long long)__double_as_longlong(fabs(dA[i * N + k]));
            if (bits > best || (bits == best && i < bi)) {
              best = bits;
              bi = i;
            }
          }
          for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) {
              best = ob;
              bi = oi;
            }
          }
          if (lane == 0) {
            s_piv = bi;
            pivot_recip(dA[bi * N + k], k);
          }
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != k) {
          for (int j = tid; j < N; j += blockDim.x) {
            const double t = dA[k * N + j];
            dA[k * N + j] = dA[pr * N + j];
            dA[pr * N + j] = t;
          }
          for (int r = tid; r < nrhs; r += blockDim.x) {
            const double t = db[r * N + k];
            db[r * N + k] = db[r * N + pr];
            db[r * N + pr] = t;
          }
          __syncthreads();
        }
        const double rp = sRD[k];
        const int rem = N - k - 1, wdt = rem + nrhs;
        for (int id = tid; id < rem * wdt; id += blockDim.x) {
          const int i = k + 1 + id / wdt, jj = id % wdt;
          const double l = dA[i * N + k] * rp;
          if (jj < rem) {
            const int j = k + 1 + jj;
            dA[i * N + j] = fma(-l, dA[k * N + j], dA[i * N + j]);
          } else {
            const int r = jj - rem;
            db[r * N + i] = fma(-l, db[r * N + k], db[r * N + i]);
          }
        }
        __syncthreads();
      }
    }
    // back substitution, one barrier per step: x_k = b_k / u_kk into sXd, and
    // b_i -= u_ik x_k for i < k (every thread forms x_k itself)
    for (int k = N - 1; k >= 0; --k) {
      const double rp = sRD[k];
      for (int id = tid; id < (k + 1) * nrhs; id += blockDim.x) {
        const int r = id / (k + 1), i = id % (k + 1);
        const double xk = db[r * N + k] * rp;
        if (i == k) sXd[r * N + k] = xk;
        else db[r * N + i] = fma(-dA[i * N + k], xk, db[r * N + i]);
      }
      __syncthreads();
    }
    for (int id = tid; id < nrhs * N; id += blockDim.x) db[id] = sXd[id];
    if constexpr (MIXED) {
      __syncthreads();
      for (int id = tid; id < nrhs * N; id += blockDim.x) {
        const double v = db[id];
        sb[id] = R::from(v);
      }
    }
  }
  }   // rank 0 (every rank with split right-hand sides)
  cluster.sync();   // the solution is in rank 0's b (split right-hand sides: in each CTA's own)
  if (rank != 0 && !rsplit)
    for (int id = tid; id < nrhs * N; id += blockDim.x) sb[id] = b0[id];
  if constexpr (!ADJ) {
    // the forward solution kept for the reverse sweep of the wave-speed gradient
    if (a.xsave != nullptr && (rank == 0 || rsplit)) {
      const int NBg = NG * nb;
      double* xs = a.xsave + (size_t)(tent - a.xbase) * a.xs_stride + (size_t)(rsplit ? rank * nrhs : 0) * NBg;
      for (int id = tid; id < nrhs * N; id += blockDim.x) xs[(size_t)(id / N) * NBg + id % N] = R::to(sb[id]);
    }
  }
  __syncthreads();

  // ---------------- phase 4: outflow at this CTA's top points (adjoint: bottom points) ----------------
  // coefficient vectors of U_h, v_h, sigma_h in terms of U-values, per material: y = D^T x_g
  for (int id = tid; id < ng * nmom; id += blockDim.x) {
    const int g = id / nmom, rest = id % nmom;
    const int r = rest / (C * nb), rem = rest % (C * nb), cc = rem / nb, kk = rem % nb;
    const T* xg = sb + (size_t)r * N + g * nb;
    T t;
    if (cc == 0) t = xg[kk];
    else t = R::mul(R::from(cc == 1 ? s_gc[g] * ih : -ih), relT_apply<DIM, T>(a, kk, cc - 1, xg));
    sY[id] = t;
  }
  __syncthreads();
  // the points whose front values this CTA overwrites (split right-hand
  // sides: this CTA's own right-hand sides at every point)
  const int o0 = rsplit ? 0 : q0, o1 = rsplit ? NP : q1;
  // ---------------- energy lost in the tent (forward sweep, when tracked) ----------------
  // Testing the tent system with V = U_h and using d/dt e + div(v sigma) = 0
  // inside the Trefftz tent: 1/2 int_top Q_{g_t}(u) = 1/2 int_bot Q_{g_b}(u_b) - D,
  //   D = 1/2 int_bot Q_{g_b}(u - u_b) + int_bot (U - U_b) U
  //     + int_D [alpha v^2 - g_D (alpha v - sigma.n)] + int_N [beta (sigma.n)^2 - g_N (beta sigma.n - v)]
  //     + int_time [alpha (v+ - v-)^2 + beta ((sigma+ - sigma-).n)^2]
  // (eq. 2.5, eq. 4.1, Section 6.5; Q_g(w) = c^-2 w_v^2 + |w_s|^2 - 2 w_v w_s.g).
  // Point values of the solution come from the outflow vectors and U-values
  // scaled by sqrt(w); the stored bottom values are read before this CTA
  // overwrites them below.  Summed over the sweep: E(T) = E(0) - sum D.
  if constexpr (!ADJ) {
    if (a.diss != nullptr) {
      double* sDis = reinterpret_cast<double*>(sDel);   // nrhs partial sums (sDel is dead after phase 2)
      double* sFb = reinterpret_cast<double*>(sCB);     // CH*nrhs*C stored values (sCB is dead after phase 1)
      double* sGdd = reinterpret_cast<double*>(sGd);    // CH*nrhs boundary data (dead after phase 2)
      for (int id = tid; id < nrhs; id += blockDim.x) sDis[id] = 0.0;
      __syncthreads();
      auto fieldv = [&](int g, int r, int cc, const T* u) {   // sqrt(w) times component cc of the solution
        const T* y = sY + (size_t)g * nmom + ((size_t)r * C + cc) * nb;
        T t = R::zero();
        for (int j = 0; j < nb; ++j) t = R::acc(t, y[j], u[j]);
        return R::to(R::norm(t));
      };
      // (a) bottom face: the jump to the stored front and the recovery term
      for (int base = o0; base < o1; base += CH) {
        const int nq = min(CH, o1 - base);
        for (int id = tid; id < nq; id += blockDim.x) {
          const int qg = base + id;
          map_point(sPt + id * (DIM + 2), qg / Q, qg % Q, false);
        }
        for (int id = tid; id < nq * nrhs; id += blockDim.x) {
          const int ql = id / nrhs, r = id % nrhs, qg = base + ql, k = qg / Q, q = qg % Q;
          const double sw = __ldg(a.sqw + q) * s_sdet[k];
          const double* f = front + (((int64_t)r * a.ne + s_el[k]) * Q + q) * C;
#pragma unroll
          for (int cc = 0; cc < C; ++cc) sFb[(size_t)id * C + cc] = sw * __ldcg(f + cc);
        }
        eval_uvalues_block<DIM, T>(a, nq, sPt, sM, sU);
        for (int id = tid; id < nq * nrhs; id += blockDim.x) {
          const int ql = id / nrhs, r = id % nrhs, k = (base + ql) / Q, g = s_grp[k];
          const T* u = sU + (size_t)ql * us;
          const double* fb = sFb + (size_t)id * C;
          const double Uh = fieldv(g, r, 0, u), dv = fieldv(g, r, 1, u) - fb[1];
          double ds2 = 0.0, dsg = 0.0;
          for (int d = 0; d < DIM; ++d) {
            const double ds = fieldv(g, r, 2 + d, u) - fb[2 + d];
            ds2 = fma(ds, ds, ds2);
            dsg = fma(ds, s_gb[k][d], dsg);
          }
          atomicAdd(sDis + r, 0.5 * (s_gic2[g] * dv * dv + ds2 - 2.0 * dv * dsg) + (Uh - fb[0]) * Uh);
        }
        __syncthreads();
      }
      // (b) vertical faces: Dirichlet, then interface, then Neumann facets,
      // each facet's points split over the cluster (split right-hand sides: every point)
      const int fsl = (Q + CS - 1) / CS;
      const int p0 = rsplit ? 0 : min(Q, rank * fsl), p1 = rsplit ? Q : min(Q, p0 + fsl);
      for (int f = 0; f < nfac + nif + nneu; ++f) {
        const bool ifc = f >= nfac && f < nfac + nif, neu = NEU && f >= nfac + nif;
        const int gp = s_fg[f], gm = s_fg2[f];
        for (int base = p0; base < p1; base += CH) {
          const int nq = min(CH, p1 - base);
          for (int id = tid; id < nq; id += blockDim.x) {
            const int q = base + id;
            double xt[DIM + 1];
            for (int d = 0; d <= DIM; ++d) xt[d] = 0.0;
            for (int i = 0; i < NV; ++i) {
              const double l = __ldg(a.bary + q * NV + i);
              for (int d = 0; d <= DIM; ++d) xt[d] = fma(l, s_fP[f][i][d], xt[d]);
            }
            const double sw = __ldg(a.sqw + q) * s_fsq[f];
            T* pp = sPt + id * (DIM + 2);
            pp[0] = R::from(s_gc[gp] * (xt[DIM] - tc) * ih);
            for (int d = 0; d < DIM; ++d) pp[1 + d] = R::from((xt[d] - s_xv[d]) * ih);
            pp[DIM + 1] = R::from(sw);
            if (ifc) {
              T* p2 = sPt + (nq + id) * (DIM + 2);
              p2[0] = R::from(s_gc[gm] * (xt[DIM] - tc) * ih);
              for (int d = 0; d < DIM; ++d) p2[1 + d] = pp[1 + d];
              p2[DIM + 1] = pp[DIM + 1];
            } else {
              // the facet's block of boundary data (without Neumann facets: the facet's own index)
              const long long goff = a.tent_gdoff[tent] + (NEU ? (long long)s_fw[f][0] * Q : (long long)f * Q) + q;
              for (int r = 0; r < nrhs; ++r)
                sGdd[id * nrhs + r] = gD != nullptr ? sw * gD[(long long)r * a.n_bnd + goff] : 0.0;
            }
          }
          eval_uvalues_block<DIM, T>(a, ifc ? 2 * nq : nq, sPt, sM, sU);
          for (int id = tid; id < nq * nrhs; id += blockDim.x) {
            const int ql = id / nrhs, r = id % nrhs;
            const T* u = sU + (size_t)ql * us;
            const double vh = fieldv(gp, r, 1, u);
            double sn = 0.0;
            for (int d = 0; d < DIM; ++d) sn = fma(s_fn[f][d], fieldv(gp, r, 2 + d, u), sn);
            double val;
            if (ifc) {
              const T* u2 = sU + (size_t)(nq + ql) * us;
              double sn2 = 0.0;
              for (int d = 0; d < DIM; ++d) sn2 = fma(s_fn[f][d], fieldv(gm, r, 2 + d, u2), sn2);
              const double jv = vh - fieldv(gm, r, 1, u2), js = sn - sn2;
              val = a.alpha * jv * jv + a.beta * js * js;
            } else {
              const double gv = sGdd[id];
              val = neu ? a.beta * sn * sn - gv * (a.beta * sn - vh) : a.alpha * vh * vh - gv * (a.alpha * vh - sn);
            }
            atomicAdd(sDis + r, val);
          }
          __syncthreads();
        }
      }
      double* diss = a.diss + (rsplit ? (size_t)rank * nrhs : 0);
      for (int r = tid; r < nrhs; r += blockDim.x) atomicAdd(diss + r, sDis[r]);
      __syncthreads();
    }
  }
  // ---------------- point outputs (forward sweep, when requested) ----------------
  // U_h at the samples (x_j, t_k) that lie inside this tent: t_bot(x_j) <=
  // t_k < t_top(x_j) on the element of x_j (the host assigns each sample to
  // the one tent that holds it); U_h = sum_j x_j b_j at the mapped point
  // (Remark 3.1)
  if constexpr (!ADJ) {
    if (a.probe_ptr != nullptr) {
      const int s0 = __ldg(a.probe_ptr + tent), ns = __ldg(a.probe_ptr + tent + 1) - s0;
      const int psl = rsplit ? ns : (ns + CS - 1) / CS;
      const int a0 = rsplit ? 0 : min(ns, rank * psl), a1 = rsplit ? ns : min(ns, a0 + psl);
      for (int base = a0; base < a1; base += 2 * CH) {
        const int nq = min(2 * CH, a1 - base);
        for (int id = tid; id < nq; id += blockDim.x) {
          const int smp = s0 + base + id, j = __ldg(a.probe_j + smp), k = __ldg(a.probe_slot + smp);
          const double t = __ldg(a.probe_t + __ldg(a.probe_k + smp));
          double x[DIM];
          for (int d = 0; d < DIM; ++d) x[d] = 0.0;
          for (int i = 0; i < NV; ++i) {
            const double l = __ldg(a.probe_bary + (size_t)j * NV + i);
            for (int d = 0; d < DIM; ++d) x[d] = fma(l, s_X[k][i][d], x[d]);
          }
          T* pp = sPt + id * (DIM + 2);
          pp[0] = R::from(s_gc[s_grp[k]] * (t - tc) * ih);
          for (int d = 0; d < DIM; ++d) pp[1 + d] = R::from((x[d] - s_xv[d]) * ih);
          pp[DIM + 1] = R::one();
        }
        eval_uvalues_block<DIM, T, false>(a, nq, sPt, sM, sU);
        for (int id = tid; id < nq * nrhs; id += blockDim.x) {
          const int ql = id % nq, r = id / nq, smp = s0 + base + ql;
          const int j = __ldg(a.probe_j + smp), kt = __ldg(a.probe_k + smp), k = __ldg(a.probe_slot + smp);
          const T* y = sY + (size_t)s_grp[k] * nmom + (size_t)r * C * nb;   // U_h = u . x_g
          const T* u = sU + (size_t)ql * us;
          T acc = R::zero();
          for (int jj = 0; jj < nb; ++jj) acc = R::acc(acc, y[jj], u[jj]);
          const int rg = (rsplit ? rank * nrhs : 0) + r;
          a.probe_out[((size_t)rg * a.n_probe_t + kt) * a.n_probe + j] = R::to(R::norm(acc));
        }
        __syncthreads();
      }
    }
  }
  // ---------------- wave-speed gradient (reverse sweep, when requested) ----------------
  // With the tents held fixed, J depends on the speed c_g of material g
  // through every tent's maps b = B f_bot, A x = b, f_top = E x (eq. 4.1), so
  //   dJ/dc_g += lambda_top . (dE/dc_g) x + mu^T ((dB/dc_g) f_bot - (dA/dc_g) x),
  // x the tent's forward solution, f_bot the forward front below it,
  // lambda_top the adjoint front at its top points, mu = A^-T E^T lambda_top.
  // With t^ = c (t - t_c)/h (Remark 3.1) the fields F = (U, v, sigma) of a
  // coefficient vector x move with c as
  //   dF/dc = ((t - t_c)/c) F(x') + (0, v/c, 0),   x' = (c/h) D_t^T x
  // (the time derivative of U_h is again in U^p), so every derivative is a
  // point value of the forms of eq. (4.1) and eq. (2.5) on F and dF; the
  // only explicit c of the forms is c^-2 of the top and bottom faces.  Each
  // point's contribution is booked on its element (a facet's on the element
  // of its side): summed over the elements of a material it is dJ/dc of
  // that material.
  if constexpr (ADJ) {
    if (a.dJdc != nullptr) {
      const int NBg = NG * nb;
      T* sYx = reinterpret_cast<T*>(sm + a.off_yg);   // NG*nmom  y(x)
      T* sYxp = sYx + (size_t)NG * nmom;               // NG*nmom  y(x')
      T* sYmp = sYxp + (size_t)NG * nmom;              // NG*nmom  y(mu')
      T* sXf = sYmp + (size_t)NG * nmom;               // nrhs*N   forward solution
      const int rg0 = rsplit ? rank * nrhs : 0;
      {
        const double* xs = a.xsave + (size_t)(tent - a.xbase) * a.xs_stride;
        for (int id = tid; id < nrhs * N; id += blockDim.x) sXf[id] = R::from(xs[(size_t)(rg0 + id / N) * NBg + id % N]);
      }
      for (int k = tid; k < P; k += blockDim.x) s_gel[k] = 0.0;
      __syncthreads();
      // y = (z_g, (c/h) D_t^T z_g, -(1/h) D_m^T z_g) of a coefficient vector z per material and right-hand side
      auto coefs = [&](T* dst, const T* src, int rstride, int gstride) {
        for (int id = tid; id < ng * nmom; id += blockDim.x) {
          const int g = id / nmom, rest = id % nmom;
          const int r = rest / (C * nb), rem = rest % (C * nb), cc = rem / nb, kk = rem % nb;
          const T* zg = src + (size_t)r * rstride + (size_t)g * gstride;
          dst[id] = cc == 0 ? zg[kk]
                            : R::mul(R::from(cc == 1 ? s_gc[g] * ih : -ih), relT_apply<DIM, T>(a, kk, cc - 1, zg));
        }
      };
      coefs(sYx, sXf, N, nb);
      coefs(sYmp, sY + nb, C * nb, nmom);              // mu' = y_v(mu)
      __syncthreads();
      coefs(sYxp, sYx + nb, C * nb, nmom);             // x' = y_v(x)
      __syncthreads();
      // sqrt(w) times the C components of the field of vectors Y at U-values u
      auto fld = [&](const T* Y, int g, int r, const T* u, double* F) {
        for (int cc = 0; cc < C; ++cc) {
          const T* y = Y + (size_t)g * nmom + ((size_t)r * C + cc) * nb;
          T t = R::zero();
          for (int j = 0; j < nb; ++j) t = R::acc(t, y[j], u[j]);
          F[cc] = R::to(R::norm(t));
        }
      };
      // fields of x and mu and their c-derivatives at a point of material g
      auto fields4 = [&](int g, int r, const T* u, double tq, double* Fx, double* dFx, double* Fm, double* dFm) {
        const double cg = s_gc[g];
        fld(sYx, g, r, u, Fx);
        fld(sYxp, g, r, u, dFx);
        fld(sY, g, r, u, Fm);
        fld(sYmp, g, r, u, dFm);
        for (int cc = 0; cc < C; ++cc) {
          dFx[cc] *= tq / cg;
          dFm[cc] *= tq / cg;
        }
        dFx[1] += Fx[1] / cg;
        dFm[1] += Fm[1] / cg;
      };
      // (a) top points (the map E and the top form) and bottom points (the
      // bottom form of b and the recovery terms), this CTA's points
      for (int side = 0; side < 2; ++side) {
        for (int base = o0; base < o1; base += CH) {
          const int nq = min(CH, o1 - base);
          for (int id = tid; id < nq; id += blockDim.x) {
            const int qg = base + id;
            map_point(sPt + id * (DIM + 2), qg / Q, qg % Q, side == 0);
          }
          eval_uvalues_block<DIM, T>(a, nq, sPt, sM, sU);
          for (int id = tid; id < nq * nrhs; id += blockDim.x) {
            const int ql = id / nrhs, r = id % nrhs, qg = base + ql, k = qg / Q, q = qg % Q, g = s_grp[k];
            double tt = 0.0;
            for (int i = 0; i < NV; ++i) tt = fma(__ldg(a.bary + q * NV + i), side == 0 ? s_tt[k][i] : s_tb[k][i], tt);
            double Fx[C], dFx[C], Fm[C], dFm[C];
            fields4(g, r, sU + (size_t)ql * us, tt - tc, Fx, dFx, Fm, dFm);
            const double ic2 = s_gic2[g], dic2 = -2.0 * ic2 / s_gc[g];   // c^-2 and its derivative
            const double* gk = side == 0 ? s_gt[k] : s_gb[k];
            // c^-2 a_v b_v + a_s.b_s - a_v (b_s.g) - (a_s.g) b_v: the face form of eq. (4.1)
            auto Qf = [&](const double* A_, const double* B_) {
              double s2 = ic2 * A_[1] * B_[1], ag = 0.0, bg = 0.0;
              for (int d = 0; d < DIM; ++d) {
                s2 = fma(A_[2 + d], B_[2 + d], s2);
                ag = fma(A_[2 + d], gk[d], ag);
                bg = fma(B_[2 + d], gk[d], bg);
              }
              return s2 - A_[1] * bg - ag * B_[1];
            };
            double val;
            if (side == 0) {
              const double* lam = front + (((int64_t)r * a.ne + s_el[k]) * Q + q) * C;
              const double isw = __ldg(a.isqw + q) * s_isdet[k];
              double e = 0.0;
              for (int cc = 0; cc < C; ++cc) e = fma(__ldcg(lam + cc) * isw, dFx[cc], e);
              val = e - (Qf(dFx, Fm) + Qf(Fx, dFm) + dic2 * Fx[1] * Fm[1]);
            } else {
              const double sw = __ldg(a.sqw + q) * s_sdet[k];
              const double* f0 = a.front_fwd + (((int64_t)(rg0 + r) * a.ne + s_el[k]) * Q + q) * C;
              double fb[C];
              for (int cc = 0; cc < C; ++cc) fb[cc] = sw * __ldcg(f0 + cc);
              val = Qf(fb, dFm) + dic2 * fb[1] * Fm[1] + fb[0] * dFm[0] - (dFx[0] * Fm[0] + Fx[0] * dFm[0]);
            }
            atomicAdd(s_gel + k, val);
          }
          __syncthreads();
        }
      }
      // (b) vertical faces: Dirichlet, interface and Neumann facets (each
      // facet's points split over the cluster; split right-hand sides: every point)
      const int fsl = (Q + CS - 1) / CS;
      const int p0 = rsplit ? 0 : min(Q, rank * fsl), p1 = rsplit ? Q : min(Q, p0 + fsl);
      const int* rfi = a.vrec_i + h0.y + P * (2 + NV);
      double* sGdd = reinterpret_cast<double*>(sGd);
      for (int f = 0; f < nfac + nif + nneu; ++f) {
        const bool ifc = f >= nfac && f < nfac + nif, neu = NEU && f >= nfac + nif;
        const int gp = s_fg[f], gm = s_fg2[f];
        // patch slots of the elements on the facet's + and - sides (boundary facets: one element)
        int kp = 0, km = 0;
        {
          const int ep = __ldg(rfi + f * (NV + 3)), em = __ldg(rfi + f * (NV + 3) + 1);
          for (int k = 0; k < P; ++k) {
            if (s_el[k] == ep) kp = k;
            if (s_el[k] == em) km = k;
          }
        }
        for (int base = p0; base < p1; base += CH) {
          const int nq = min(CH, p1 - base);
          for (int id = tid; id < nq; id += blockDim.x) {
            const int q = base + id;
            double xt[DIM + 1];
            for (int d = 0; d <= DIM; ++d) xt[d] = 0.0;
            for (int i = 0; i < NV; ++i) {
              const double l = __ldg(a.bary + q * NV + i);
              for (int d = 0; d <= DIM; ++d) xt[d] = fma(l, s_fP[f][i][d], xt[d]);
            }
            const double sw = __ldg(a.sqw + q) * s_fsq[f];
            T* pp = sPt + id * (DIM + 2);
            pp[0] = R::from(s_gc[gp] * (xt[DIM] - tc) * ih);
            for (int d = 0; d < DIM; ++d) pp[1 + d] = R::from((xt[d] - s_xv[d]) * ih);
            pp[DIM + 1] = R::from(sw);
            if (ifc) {
              T* p2 = sPt + (nq + id) * (DIM + 2);
              p2[0] = R::from(s_gc[gm] * (xt[DIM] - tc) * ih);
              for (int d = 0; d < DIM; ++d) p2[1 + d] = pp[1 + d];
              p2[DIM + 1] = pp[DIM + 1];
            } else {
              // the forward boundary data of the facet (g_D or g_N)
              const long long goff = a.tent_gdoff[tent] + (NEU ? (long long)s_fw[f][0] * Q : (long long)f * Q) + q;
              for (int r = 0; r < nrhs; ++r)
                sGdd[id * nrhs + r] = gD != nullptr ? sw * gD[(long long)r * a.n_bnd + goff] : 0.0;
            }
          }
          eval_uvalues_block<DIM, T>(a, ifc ? 2 * nq : nq, sPt, sM, sU);
          for (int id = tid; id < nq * nrhs; id += blockDim.x) {
            const int ql = id / nrhs, r = id % nrhs, q = base + ql;
            double tt = 0.0;
            for (int i = 0; i < NV; ++i) tt = fma(__ldg(a.bary + q * NV + i), s_fP[f][i][DIM], tt);
            double Fx[C], dFx[C], Fm[C], dFm[C];
            fields4(gp, r, sU + (size_t)ql * us, tt - tc, Fx, dFx, Fm, dFm);
            auto sn = [&](const double* F_) {
              double t_ = 0.0;
              for (int d = 0; d < DIM; ++d) t_ = fma(s_fn[f][d], F_[2 + d], t_);
              return t_;
            };
            if (ifc) {
              double Gx[C], dGx[C], Gm[C], dGm[C], Z[C];
              fields4(gm, r, sU + (size_t)(nq + ql) * us, tt - tc, Gx, dGx, Gm, dGm);
              for (int cc = 0; cc < C; ++cc) Z[cc] = 0.0;
              // the interface form of eq. (2.5) with trial fields X+-, test fields M+-
              auto I = [&](const double* Xp, const double* Xm, const double* Mp, const double* Mm) {
                const double jm = sn(Mp) - sn(Mm), dv = Mp[1] - Mm[1];
                return 0.5 * (jm * (Xp[1] + Xm[1]) + dv * (sn(Xp) + sn(Xm))) + a.alpha * dv * (Xp[1] - Xm[1]) +
                       a.beta * jm * (sn(Xp) - sn(Xm));
              };
              atomicAdd(s_gel + kp, -(I(dFx, Z, Fm, Gm) + I(Fx, Gx, dFm, Z)));
              atomicAdd(s_gel + km, -(I(Z, dGx, Fm, Gm) + I(Fx, Gx, Z, dGm)));
            } else {
              const double gv = sGdd[id];
              double val;
              if (neu) {   // A: v (tau.n) + beta (sigma.n)(tau.n); b: g_N (beta tau.n - w)
                val = gv * (a.beta * sn(dFm) - dFm[1]) -
                      (dFx[1] * sn(Fm) + Fx[1] * sn(dFm) + a.beta * (sn(dFx) * sn(Fm) + sn(Fx) * sn(dFm)));
              } else {     // A: (sigma.n + alpha v) w; b: g_D (alpha w - tau.n)
                val = gv * (a.alpha * dFm[1] - sn(dFm)) -
                      ((sn(dFx) + a.alpha * dFx[1]) * Fm[1] + (sn(Fx) + a.alpha * Fx[1]) * dFm[1]);
              }
              atomicAdd(s_gel + kp, val);
            }
          }
          __syncthreads();
        }
      }
      for (int k = tid; k < P; k += blockDim.x) atomicAdd(a.dJdc + s_el[k], s_gel[k]);
      __syncthreads();
    }
  }
  // tensor-core outflow: f(q)[r, c] = sum_j U_j(q) y[r, c, j] for a chunk
  // of up to 2 CH top points, one M = 128 tile of points: A = the digit
  // planes of the points' U-values (rows = points, K = basis functions
  // padded to 32, scaled per point), B = those of y (rows (r, c) padded to
  // 16, scaled per row; formed once per tent); each level sum takes
  // (tc_cols / kSlices) rounded down to 32, i.e. 96 columns (>= NY)
  const int M_tc = nrhs * C, NY = (M_tc + 15) & ~15, planeY = 32 * NY;
  const int planeU = 32 * ((2 * CH + 15) & ~15);
  if constexpr (kTC) {
    if (tc_on) {
      uint16_t* sTB = reinterpret_cast<uint16_t*>(sm + a.off_tc) + tc::kSlices * planeU + 512;
      for (int m = tid; m < NY; m += blockDim.x) {
        float mx = 0.f;
        if (m < M_tc)
          for (int j = 0; j < nb; ++j) mx = fmaxf(mx, fabsf(sY[(size_t)m * nb + j].hi));
        s_tce[0][m] = tc::scale_exp(mx);
      }
      __syncthreads();
      for (int id = tid; id < NY * 4; id += blockDim.x) {
        const int kc = id / NY, m = id % NY;
        float d[8][tc::kSlices];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int jj = kc * 8 + j;
          const T x = (m < M_tc && jj < nb) ? sY[(size_t)m * nb + jj] : R::zero();
          tc::digits(x.hi, x.lo, s_tce[0][m], d[j]);
        }
        tc::store_row8(sTB + ((size_t)(kc * (NY >> 3) + (m >> 3)) * 64 + (m & 7) * 8), planeY, d);
      }
      // (the first chunk's barriers order these writes before the products)
    }
  }
  auto tc_outflow = [&](int base, int nq) {
    if constexpr (kTC) {
      const int NP = (nq + 15) & ~15, RGU = NP >> 3;
      uint16_t* sTA = reinterpret_cast<uint16_t*>(sm + a.off_tc);
      uint16_t* sTB = sTA + tc::kSlices * planeU + 512;
      int* eY = s_tce[0];
      int* eU = s_tce[1];
      for (int ql = tid; ql < NP; ql += blockDim.x) {
        float mx = 0.f;
        if (ql < nq)
          for (int j = 0; j < nb; ++j) mx = fmaxf(mx, fabsf(sU[(size_t)ql * us + j].hi));
        eU[ql] = tc::scale_exp(mx);
      }
      __syncthreads();
      for (int id = tid; id < NP * 4; id += blockDim.x) {
        const int kc = id / NP, n = id % NP;
        float d[8][tc::kSlices];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int jj = kc * 8 + j;
          const T x = (n < nq && jj < nb) ? sU[(size_t)n * us + jj] : R::zero();
          tc::digits(x.hi, x.lo, eU[n], d[j]);
        }
        tc::store_row8(sTA + ((size_t)(kc * RGU + (n >> 3)) * 64 + (n & 7) * 8), planeU, d);
      }
      const int cstride = (a.tc_cols / tc::kSlices) & ~31;   // columns per level sum (>= NY)
      const bool ok = tc_product(tc::smem_addr(sTA), (uint32_t)planeU * 2, (uint32_t)RGU * 128,
                                 tc::smem_addr(sTB), (uint32_t)planeY * 2, (uint32_t)(NY >> 3) * 128, 2, NY, cstride);
      // levels -> binary64 front values: the thread of lane l of warp w holds
      // point 32 (w % 4) + l and the rows (r, c) of half w / 4
      const int q4 = warp & 3, h = warp >> 2, half = NY >> 1;
      if (ok && 32 * q4 < nq) {
        const int ql = 32 * q4 + lane;
        const bool live = ql < nq;
        double* fq = front;
        int ep = 0;
        if (live) {
          const int qg = base + ql, k = qg / Q, q = qg % Q;
          fq = front + ((int64_t)s_el[k] * Q + q) * C;
          ep = eU[ql] - 16;
        }
        const int64_t rstride = (int64_t)a.ne * Q * C;
        for (int c0 = h * half; c0 < (h + 1) * half; c0 += 8) {
          float lv[tc::kSlices][8];
#pragma unroll
          for (int l = 0; l < tc::kSlices; ++l)
            tc::ld8(s_tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(l * cstride + c0), lv[l]);
          tc::wait_ld();
          if (live) {
            int r = c0 / C, cc = c0 - r * C;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              if (c0 + j < M_tc) {
                float acc[tc::kSlices];
#pragma unroll
                for (int l = 0; l < tc::kSlices; ++l) acc[l] = lv[l][j];
                float sh, se;
                tc::combine_ff(acc, sh, se);
                fq[r * rstride + cc] = tc::ff_to_double(sh, se, ep + eY[c0 + j]);
              }
              if (++cc == C) {
                cc = 0;
                ++r;
              }
            }
          }
        }
      }
      tc::fence_before();
      __syncthreads();
    }
  };
  for (int base = o0; base < o1; base += 2 * CH) {
    const int nq = min(2 * CH, o1 - base);
    if (!keep) {
    for (int id = tid; id < nq; id += blockDim.x) {
      const int qg = base + id, k = qg / Q, q = qg % Q;
      const double cg = s_gc[s_grp[k]];
      double x[DIM], tt = 0.0;
      for (int d = 0; d < DIM; ++d) x[d] = 0.0;
      for (int i = 0; i < NV; ++i) {
        const double l = __ldg(a.bary + q * NV + i);
        for (int d = 0; d < DIM; ++d) x[d] = fma(l, s_X[k][i][d], x[d]);
        tt = fma(l, ADJ ? s_tb[k][i] : s_tt[k][i], tt);
      }
      T* pp = sPt + id * (DIM + 2);
      pp[0] = R::from(cg * (tt - tc) * ih);
      for (int d = 0; d < DIM; ++d) pp[1 + d] = R::from((x[d] - s_xv[d]) * ih);
      pp[DIM + 1] = R::one();
    }
    eval_uvalues_block<DIM, T, false>(a, nq, sPt, sM, sU);
    }
    if constexpr (!ADJ) {
      // few right-hand sides: one (point, right-hand side, component) per
      // thread, so that every warp (and every sub-partition's binary64 unit)
      // has work
      if (tc_on) {
        tc_outflow(base, nq);
      } else if (nq * nrhs < (int)blockDim.x) {
        for (int id = tid; id < nq * nrhs * C; id += blockDim.x) {
          const int cc = id % C, rq = id / C, r = rq / nq, ql = rq % nq;
          const int qg = base + ql, k = qg / Q, q = qg % Q;
          const T* u = keep ? sKeep + (size_t)(base - q0 + ql) * nb : sU + (size_t)ql * us;
          const T* y = sY + (size_t)s_grp[k] * nmom + ((size_t)r * C + cc) * nb;
          T t = R::zero();
          for (int j = 0; j < nb; ++j) t = R::acc(t, y[j], u[j]);
          const double val = R::to(R::norm(t));
          front[(((int64_t)r * a.ne + s_el[k]) * Q + q) * C + cc] = keep ? val * sKeepW[base - q0 + ql] : val;
        }
      } else
      // one (point, right-hand side) per thread, its C components as
      // independent sums (consecutive threads: consecutive points)
      for (int id = tid; id < nq * nrhs; id += blockDim.x) {
        const int r = id / nq, ql = id % nq;
        const int qg = base + ql, k = qg / Q, q = qg % Q;
        const T* u = keep ? sKeep + (size_t)(base - q0 + ql) * nb : sU + (size_t)ql * us;
        const T* y = sY + (size_t)s_grp[k] * nmom + (size_t)r * C * nb;
        T t[C];
#pragma unroll
        for (int cc = 0; cc < C; ++cc) t[cc] = R::zero();
        for (int j = 0; j < nb; ++j) {
          const T uj = u[j];
#pragma unroll
          for (int cc = 0; cc < C; ++cc) t[cc] = R::acc(t[cc], y[cc * nb + j], uj);
        }
        double* f = front + (((int64_t)r * a.ne + s_el[k]) * Q + q) * C;
        if (keep) {
          const double sc = sKeepW[base - q0 + ql];
#pragma unroll
          for (int cc = 0; cc < C; ++cc) f[cc] = R::to(R::norm(t[cc])) * sc;
        } else {
#pragma unroll
          for (int cc = 0; cc < C; ++cc) f[cc] = R::to(R::norm(t[cc]));
        }
      }
    } else {
      // lambda_bot = w (s0, c^-2 s_t - g_b.s, s_m - g_b,m s_t)
      for (int id = tid; id < nq * nrhs; id += blockDim.x) {
        const int ql = id / nrhs, r = id % nrhs;
        const int qg = base + ql, k = qg / Q, q = qg % Q;
        const T* u = sU + (size_t)ql * us;
        double sv[C];
        for (int cc = 0; cc < C; ++cc) {
          const T* y = sY + (size_t)s_grp[k] * nmom + ((size_t)r * C + cc) * nb;
          T t = R::zero();
          for (int j = 0; j < nb; ++j) t = R::acc(t, y[j], u[j]);
          t = R::norm(t);
          sv[cc] = R::to(t);
        }
        const double cg = s_gc[s_grp[k]];
        const double sq = __ldg(a.sqw + q) * s_sdet[k];
        const double w = sq * sq;
        double gs = 0.0;
        for (int d = 0; d < DIM; ++d) gs = fma(s_gb[k][d], sv[2 + d], gs);
        double* f = front + (((int64_t)r * a.ne + s_el[k]) * Q + q) * C;
        f[0] = w * sv[0];
        f[1] = w * (sv[1] / (cg * cg) - gs);
        for (int d = 0; d < DIM; ++d) f[2 + d] = w * (sv[2 + d] - s_gb[k][d] * sv[1]);
      }
    }
    __syncthreads();
  }
  if (tid == 0 && rank == 0) a.tau[v] = ADJ ? s_tbot : s_ttop;
  if constexpr (PERSIST) {
    // this CTA's front (and rank 0's time) writes, then its completion count;
    // no CTA reads another's shared memory after the solution copy, and the
    // next tent's first cluster barrier keeps rank 0's b until all have copied it
    __threadfence();
    __syncthreads();
    if (tid == 0) red_release_add(a.done + v, 1);
  } else {
    cluster.sync();   // rank 0's b stays valid until every CTA has read the solution
    break;
  }
  }   // tent loop
  if (kTC && a.tc) {
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_free(s_tmem, a.tc_cols);
  }
}


// launchers, one translation unit per space dimension (tp_layer_d<n>.cu)
// mode: 0 forward binary64, 1 forward mixed, 2 adjoint binary64, plus 4 for
// meshes with Neumann facets;
// persistent: one resident grid of clusters pulling tents from a queue
#define TP_DECLARE_LAUNCHERS(D)                                                                  \
  cudaError_t layer_attrs_d##D(size_t smem);                                                      \
  cudaError_t layer_static_smem_d##D(size_t* bytes);                                              \
  cudaError_t launch_layer_d##D(const KArgs& a, int n_cluster, int cs, int t0, size_t smem,       \
                                cudaStream_t st, int mode, bool persistent);                      \
  cudaError_t max_clusters_d##D(int cs, size_t smem, int mode, int* n);
TP_DECLARE_LAUNCHERS(1)
TP_DECLARE_LAUNCHERS(2)
TP_DECLARE_LAUNCHERS(3)
#undef TP_DECLARE_LAUNCHERS

}  // namespace tp
