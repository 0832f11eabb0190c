// Host side of libtp: mesh topology, reference quadrature, the Trefftz basis
// tables and tent pitching.  Compiled with -ffp-contract=off so that the
// pitching arithmetic is plain IEEE binary64 (no fused multiply-add).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "tp_internal.h"

namespace tp {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

// ===========================================================================
// Topology
// ===========================================================================
bool build_topology(const tp_mesh_desc* m, Topology* t) {
  if (!m || m->dim < 1 || m->dim > kMaxDim || m->n_vert < 2 || m->n_elem < 1 || !m->coords ||
      !m->elems || !m->c) {
    set_error("tp: invalid mesh descriptor");
    return false;
  }
  const int n = m->dim;
  t->dim = n;
  t->nv = m->n_vert;
  t->ne = m->n_elem;
  t->X.assign(m->coords, m->coords + m->n_vert * n);
  t->elems.assign(m->elems, m->elems + m->n_elem * (n + 1));
  t->c.assign(m->c, m->c + m->n_elem);
  for (int64_t k = 0; k < t->ne; ++k) {
    if (!(t->c[k] > 0.0) || !std::isfinite(t->c[k])) {
      set_error("tp: wave speed must be positive and finite (element " + std::to_string(k) + ")");
      return false;
    }
    for (int i = 0; i <= n; ++i) {
      int32_t a = t->elems[k * (n + 1) + i];
      if (a < 0 || a >= t->nv) {
        set_error("tp: element " + std::to_string(k) + " has an invalid vertex id");
        return false;
      }
    }
  }
  // vertex star (elements ascending)
  std::vector<int32_t> cnt(t->nv + 1, 0);
  for (int64_t k = 0; k < t->ne; ++k)
    for (int i = 0; i <= n; ++i) cnt[t->elems[k * (n + 1) + i] + 1]++;
  t->star_ptr.assign(t->nv + 1, 0);
  for (int64_t v = 0; v < t->nv; ++v) t->star_ptr[v + 1] = t->star_ptr[v] + cnt[v + 1];
  t->star_el.assign(t->star_ptr[t->nv], 0);
  std::vector<int32_t> fill(t->star_ptr.begin(), t->star_ptr.end() - 1);
  for (int64_t k = 0; k < t->ne; ++k)
    for (int i = 0; i <= n; ++i) t->star_el[fill[t->elems[k * (n + 1) + i]]++] = (int32_t)k;

  // neighbours
  std::vector<std::vector<int32_t>> nb(t->nv);
  for (int64_t k = 0; k < t->ne; ++k)
    for (int i = 0; i <= n; ++i)
      for (int j = 0; j <= n; ++j)
        if (i != j) nb[t->elems[k * (n + 1) + i]].push_back(t->elems[k * (n + 1) + j]);
  t->nbr_ptr.assign(t->nv + 1, 0);
  t->nbr.clear();
  for (int64_t v = 0; v < t->nv; ++v) {
    auto& l = nb[v];
    std::sort(l.begin(), l.end());
    l.erase(std::unique(l.begin(), l.end()), l.end());
    t->nbr.insert(t->nbr.end(), l.begin(), l.end());
    t->nbr_ptr[v + 1] = (int32_t)t->nbr.size();
  }

  // boundary facets: facets owned by exactly one element
  struct F {
    std::array<int32_t, 3> v;
    int32_t elem, opp;
    int32_t o;   // local index of opp in the element
  };
  std::vector<F> fs;
  fs.reserve(t->ne * (n + 1));
  for (int64_t k = 0; k < t->ne; ++k) {
    const int32_t* el = &t->elems[k * (n + 1)];
    for (int o = 0; o <= n; ++o) {
      F f{{-1, -1, -1}, (int32_t)k, el[o], o};
      int c = 0;
      for (int i = 0; i <= n; ++i)
        if (i != o) f.v[c++] = el[i];
      std::sort(f.v.begin(), f.v.begin() + n);
      fs.push_back(f);
    }
  }
  std::sort(fs.begin(), fs.end(), [](const F& a, const F& b) { return a.v < b.v; });
  t->facet_vert.clear();
  t->facet_nrm.clear();
  t->facet_elem.clear();
  t->facet_kind.clear();
  // unit normal of facet f pointing away from vertex opp
  auto facet_normal = [&](const F& f, int32_t opp, double* nrm) {
    nrm[0] = nrm[1] = nrm[2] = 0.0;
    const double* P0 = &t->X[(int64_t)f.v[0] * n];
    if (n == 1) {
      nrm[0] = 1.0;
    } else if (n == 2) {
      const double* P1 = &t->X[(int64_t)f.v[1] * n];
      nrm[0] = P1[1] - P0[1];
      nrm[1] = -(P1[0] - P0[0]);
    } else {
      const double* P1 = &t->X[(int64_t)f.v[1] * n];
      const double* P2 = &t->X[(int64_t)f.v[2] * n];
      double a[3] = {P1[0] - P0[0], P1[1] - P0[1], P1[2] - P0[2]};
      double b[3] = {P2[0] - P0[0], P2[1] - P0[1], P2[2] - P0[2]};
      nrm[0] = a[1] * b[2] - a[2] * b[1];
      nrm[1] = a[2] * b[0] - a[0] * b[2];
      nrm[2] = a[0] * b[1] - a[1] * b[0];
    }
    double len = 0.0, dotp = 0.0;
    for (int d = 0; d < n; ++d) len += nrm[d] * nrm[d];
    len = std::sqrt(len);
    for (int d = 0; d < n; ++d) {
      nrm[d] /= len;
      dotp += (t->X[(int64_t)opp * n + d] - P0[d]) * nrm[d];
    }
    if (dotp > 0)
      for (int d = 0; d < n; ++d) nrm[d] = -nrm[d];
  };
  struct IF {
    std::array<int32_t, 3> v;
    int32_t kp, km;
    double nrm[3];
  };
  std::vector<IF> ifs;
  for (size_t i = 0; i < fs.size();) {
    size_t j = i;
    while (j < fs.size() && fs[j].v == fs[i].v) ++j;
    if (j - i == 1) {
      const F& f = fs[i];
      double nrm[3];
      facet_normal(f, f.opp, nrm);
      for (int d = 0; d < n; ++d) {
        t->facet_vert.push_back(f.v[d]);
        t->facet_nrm.push_back(nrm[d]);
      }
      t->facet_elem.push_back(f.elem);
      const int8_t kind = m->bnd_type ? m->bnd_type[(int64_t)f.elem * (n + 1) + f.o] : 0;
      if (kind != 0 && kind != 1) {
        set_error("tp: bnd_type of element " + std::to_string(f.elem) + " is neither 0 (Dirichlet) nor 1 (Neumann)");
        return false;
      }
      t->facet_kind.push_back(kind);
    } else if (j - i == 2) {
      const F& f1 = fs[i];
      const F& f2 = fs[i + 1];
      if (t->c[f1.elem] != t->c[f2.elem]) {   // time-like interface facet (Section 4.2)
        const F& fp = (f1.elem < f2.elem) ? f1 : f2;
        const F& fm = (f1.elem < f2.elem) ? f2 : f1;
        IF rec;
        rec.v = fp.v;
        rec.kp = fp.elem;
        rec.km = fm.elem;
        facet_normal(fp, fp.opp, rec.nrm);
        ifs.push_back(rec);
      }
    } else {
      set_error("tp: non-manifold mesh (a facet has more than two elements)");
      return false;
    }
    i = j;
  }
  {
    std::vector<std::vector<int32_t>> vi(t->nv);
    for (size_t f = 0; f < ifs.size(); ++f)
      for (int d = 0; d < n; ++d) vi[ifs[f].v[d]].push_back((int32_t)f);
    t->ifac_ptr.assign(t->nv + 1, 0);
    t->ifac_vert.clear();
    t->ifac_nrm.clear();
    t->ifac_kp.clear();
    t->ifac_km.clear();
    for (int64_t v = 0; v < t->nv; ++v) {
      for (int32_t f : vi[v]) {
        for (int d = 0; d < n; ++d) {
          t->ifac_vert.push_back(ifs[f].v[d]);
          t->ifac_nrm.push_back(ifs[f].nrm[d]);
        }
        t->ifac_kp.push_back(ifs[f].kp);
        t->ifac_km.push_back(ifs[f].km);
      }
      t->ifac_ptr[v + 1] = (int32_t)t->ifac_kp.size();
    }
  }
  const int64_t nf = (int64_t)t->facet_vert.size() / n;
  std::vector<std::vector<int32_t>> vf(t->nv);
  for (int64_t f = 0; f < nf; ++f)
    for (int d = 0; d < n; ++d) vf[t->facet_vert[f * n + d]].push_back((int32_t)f);
  t->vfac_ptr.assign(t->nv + 1, 0);
  t->vfac.clear();
  for (int64_t v = 0; v < t->nv; ++v) {
    t->vfac.insert(t->vfac.end(), vf[v].begin(), vf[v].end());
    t->vfac_ptr[v + 1] = (int32_t)t->vfac.size();
  }
  return true;
}

// ===========================================================================
// Gauss-Jacobi by Newton iteration with deflation; collapsed simplex rule
// ===========================================================================
// Jacobi polynomial P_m^{(a,0)}(x) and P_{m-1} by the three-term recurrence.
static void jacobi_eval(int m, double a, double x, double* pm, double* pm1) {
  const double b = 0.0;
  double p0 = 1.0, p1 = 0.5 * ((a + b + 2.0) * x + (a - b));
  if (m == 0) {
    *pm = p0;
    *pm1 = 0.0;
    return;
  }
  for (int k = 2; k <= m; ++k) {
    double s = 2.0 * k + a + b;
    double c1 = 2.0 * k * (k + a + b) * (s - 2.0);
    double c2 = (s - 1.0) * (s * (s - 2.0) * x + a * a - b * b);
    double c3 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * s;
    double p2 = (c2 * p1 - c3 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  *pm = p1;
  *pm1 = p0;
}

// m-point rule on [0,1] for the weight (1-xi)^a, nodes ascending.
static void gauss_jacobi01(int m, int ai, std::vector<double>* xs, std::vector<double>* ws) {
  const double a = ai, b = 0.0;
  std::vector<double> r;
  for (int i = 0; i < m; ++i) {
    double x = -std::cos(M_PI * (i + 0.5) / m);
    for (int it = 0; it < 200; ++it) {
      double pm, pm1;
      jacobi_eval(m, a, x, &pm, &pm1);
      double s = 2.0 * m + a + b;
      double dp = (m * ((a - b) - s * x) * pm + 2.0 * (m + a) * (m + b) * pm1) / (s * (1.0 - x * x));
      double defl = 0.0;
      for (double y : r) defl += 1.0 / (x - y);
      double dx = pm / (dp - pm * defl);
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    r.push_back(x);
  }
  std::sort(r.begin(), r.end());
  xs->resize(m);
  ws->resize(m);
  const double gm = std::lgamma(m + a + 1.0) + std::lgamma(m + b + 1.0) - std::lgamma(m + a + b + 1.0) -
                    std::lgamma(m + 1.0);
  for (int i = 0; i < m; ++i) {
    double x = r[i], pm, pm1;
    jacobi_eval(m, a, x, &pm, &pm1);
    double s = 2.0 * m + a + b;
    double dp = (m * ((a - b) - s * x) * pm + 2.0 * (m + a) * (m + b) * pm1) / (s * (1.0 - x * x));
    double w = std::exp(gm) * std::pow(2.0, a + b + 1.0) / ((1.0 - x * x) * dp * dp);
    (*xs)[i] = 0.5 * (x + 1.0);
    (*ws)[i] = w / std::pow(2.0, a + 1.0);
  }
}

SimplexRule simplex_rule(int n, int m) {
  SimplexRule R;
  R.n = n;
  R.m = m;
  std::vector<std::vector<double>> x(n), w(n);
  for (int d = 0; d < n; ++d) gauss_jacobi01(m, n - 1 - d, &x[d], &w[d]);
  int Q = 1;
  for (int d = 0; d < n; ++d) Q *= m;
  R.Q = Q;
  R.bary.resize(Q * (n + 1));
  R.w.resize(Q);
  for (int q = 0; q < Q; ++q) {
    int idx[3] = {0, 0, 0}, rem = q;
    for (int d = n - 1; d >= 0; --d) {
      idx[d] = rem % m;
      rem /= m;
    }
    double wt = 1.0, scale = 1.0, sum = 0.0, pt[3];
    for (int d = 0; d < n; ++d) {
      wt *= w[d][idx[d]];
      pt[d] = scale * x[d][idx[d]];
      scale *= (1.0 - x[d][idx[d]]);
      sum += pt[d];
    }
    R.w[q] = wt;
    R.bary[q * (n + 1)] = 1.0 - sum;
    for (int d = 0; d < n; ++d) R.bary[q * (n + 1) + 1 + d] = pt[d];
  }
  return R;
}

}  // namespace tp

// ===========================================================================
// C ABI: errors, basis, pitching
// ===========================================================================
extern "C" const char* tp_last_error(void) { return tp::g_last_error.c_str(); }

namespace {

using Exps = std::array<int, 4>;   // (t, x1, x2, x3)

struct Rat {
  long long num, den;
};
long long gcdll(long long a, long long b) {
  a = a < 0 ? -a : a;
  while (b) {
    long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}
double rat_to_double(long long num, long long den) {
  long long g = gcdll(num, den);
  if (g > 1) {
    num /= g;
    den /= g;
  }
  return (double)num / (double)den;   // both exact in binary64 (< 2^53): one rounding
}
long long factorial(int k) {
  long long f = 1;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

// all x-exponent vectors with |alpha| = d in n variables
void alphas_of_degree(int n, int d, std::vector<Exps>* out) {
  if (n == 1) {
    out->push_back({0, d, 0, 0});
    return;
  }
  if (n == 2) {
    for (int a = d; a >= 0; --a) out->push_back({0, a, d - a, 0});
    return;
  }
  for (int a = d; a >= 0; --a)
    for (int b = d - a; b >= 0; --b) out->push_back({0, a, b, d - a - b});
}

}  // namespace

extern "C" int tp_build_basis(int32_t dim, int32_t p, tp_basis** out) {
  if (!out || dim < 1 || dim > tp::kMaxDim || p < 1 || p > tp::kMaxP) {
    tp::set_error("tp_build_basis: need 1 <= dim <= 3 and 1 <= p <= 8");
    return TP_ERR_ARG;
  }
  auto* B = new tp_basis();
  B->dim = dim;
  B->p = p;
  const int n = dim, C = dim + 2;
  // monomials t^k x^alpha with k + |alpha| <= p, ordered by total degree,
  // then by the power of t (descending), then alpha (descending)
  std::vector<Exps> monos;
  for (int deg = 0; deg <= p; ++deg)
    for (int k = deg; k >= 0; --k) {
      std::vector<Exps> al;
      alphas_of_degree(n, deg - k, &al);
      for (auto e : al) {
        e[0] = k;
        monos.push_back(e);
      }
    }
  std::map<Exps, int> index;
  for (size_t i = 0; i < monos.size(); ++i) index[monos[i]] = (int)i;
  B->nmono = (int)monos.size();
  B->exps.resize(B->nmono * (n + 1));
  B->parent.assign(B->nmono, -1);
  B->var.assign(B->nmono, -1);
  for (int g = 0; g < B->nmono; ++g) {
    for (int d = 0; d <= n; ++d) B->exps[g * (n + 1) + d] = monos[g][d];
    for (int d = 0; d <= n; ++d)
      if (monos[g][d] > 0) {
        Exps e = monos[g];
        e[d] -= 1;
        B->parent[g] = index.at(e);
        B->var[g] = d;
        break;
      }
  }
  // basis: type 0 (U(.,0) = x^beta, U_t(.,0) = 0), |beta| <= p, and type 1
  // (U(.,0) = 0, U_t(.,0) = x^beta), |beta| <= p-1; closed form
  //   U = sum_j t^(2j+type) / (2j+type)! Lap^j x^beta,
  // which is the solution of the recursion (3.1) for these initial data.
  struct Term {
    Exps e;
    long long num, den;
  };
  std::vector<std::vector<Term>> funcs;
  std::vector<int> ftype;
  std::vector<Exps> fbeta;
  for (int type = 0; type <= 1; ++type) {
    for (int deg = 0; deg <= p - type; ++deg) {
      std::vector<Exps> betas;
      alphas_of_degree(n, deg, &betas);
      for (const Exps& beta : betas) {
        std::map<Exps, long long> term;   // Lap^j x^beta with integer coefficients
        term[beta] = 1;
        std::vector<Term> f;
        for (int j = 0; !term.empty(); ++j) {
          int k = 2 * j + type;
          for (auto& kv : term) {
            Exps e = kv.first;
            e[0] = k;
            f.push_back({e, kv.second, factorial(k)});
          }
          std::map<Exps, long long> lap;
          for (auto& kv : term)
            for (int mm = 1; mm <= n; ++mm)
              if (kv.first[mm] >= 2) {
                Exps e = kv.first;
                long long fac = (long long)e[mm] * (e[mm] - 1);
                e[mm] -= 2;
                lap[e] += kv.second * fac;
              }
          for (auto it = lap.begin(); it != lap.end();)
            it = (it->second == 0) ? lap.erase(it) : std::next(it);
          term.swap(lap);
        }
        funcs.push_back(f);
        ftype.push_back(type);
        fbeta.push_back(beta);
      }
    }
  }
  B->nb = (int)funcs.size();
  // derivative relations (exact identities of the closed form, no rounding):
  //   d/dx_m b_{beta,type} = beta_m b_{beta-e_m,type}
  //   d/dt   b_{beta,1}    = b_{beta,0}
  //   d/dt   b_{beta,0}    = sum_m beta_m (beta_m - 1) b_{beta-2e_m,1}
  {
    std::map<std::pair<int, Exps>, int> fidx;
    for (int j = 0; j < B->nb; ++j) fidx[{ftype[j], fbeta[j]}] = j;
    const int NVAR = n + 1;
    std::vector<std::vector<std::pair<int, double>>> rel((size_t)B->nb * NVAR);
    for (int j = 0; j < B->nb; ++j) {
      const Exps& be = fbeta[j];
      if (ftype[j] == 1) {
        rel[(size_t)j * NVAR].push_back({fidx.at({0, be}), 1.0});
      } else {
        for (int mm = 1; mm <= n; ++mm)
          if (be[mm] >= 2) {
            Exps e = be;
            e[mm] -= 2;
            rel[(size_t)j * NVAR].push_back({fidx.at({1, e}), (double)(be[mm] * (be[mm] - 1))});
          }
      }
      for (int mm = 1; mm <= n; ++mm)
        if (be[mm] >= 1) {
          Exps e = be;
          e[mm] -= 1;
          rel[(size_t)j * NVAR + mm].push_back({fidx.at({ftype[j], e}), (double)be[mm]});
        }
    }
    B->rel_ptr.assign((size_t)B->nb * NVAR + 1, 0);
    std::vector<std::vector<std::pair<int, double>>> relT((size_t)B->nb * NVAR);
    for (size_t r = 0; r < rel.size(); ++r) {
      for (auto& e : rel[r]) {
        B->rel_src.push_back(e.first);
        B->rel_fac.push_back(e.second);
        relT[(size_t)e.first * NVAR + r % NVAR].push_back({(int)(r / NVAR), e.second});
      }
      B->rel_ptr[r + 1] = (int32_t)B->rel_src.size();
    }
    B->relT_ptr.assign((size_t)B->nb * NVAR + 1, 0);
    for (size_t r = 0; r < relT.size(); ++r) {
      for (auto& e : relT[r]) {
        B->relT_dst.push_back(e.first);
        B->relT_fac.push_back(e.second);
      }
      B->relT_ptr[r + 1] = (int32_t)B->relT_dst.size();
    }
    // merged congruence tables of the top-face form (entries i <= j)
    const int nb = B->nb;
    auto pidx = [&](int i, int j) {
      const int lo = std::min(i, j), hi = std::max(i, j);
      return lo * nb - lo * (lo - 1) / 2 + (hi - lo);
    };
    auto rel_of = [&](int row, int v, int* b, int* e) {
      *b = B->rel_ptr[(size_t)row * NVAR + v];
      *e = B->rel_ptr[(size_t)row * NVAR + v + 1];
    };
    B->cg_ptr.assign(1, 0);
    B->ch_ptr.assign(1, 0);
    for (int i = 0; i < nb; ++i)
      for (int j = i; j < nb; ++j) {
        std::map<int, double> gm, hm;
        for (int va = 0; va < NVAR; ++va) {   // D_t X D_t^T and D_m X D_m^T
          int b0, e0, b1, e1;
          rel_of(i, va, &b0, &e0);
          rel_of(j, va, &b1, &e1);
          for (int e = b0; e < e0; ++e)
            for (int f = b1; f < e1; ++f) gm[pidx(B->rel_src[e], B->rel_src[f])] += B->rel_fac[e] * B->rel_fac[f];
        }
        for (int m = 1; m < NVAR; ++m) {      // D_m H_m D_t^T + D_t H_m D_m^T
          for (int pass = 0; pass < 2; ++pass) {
            int b0, e0, b1, e1;
            rel_of(i, pass == 0 ? m : 0, &b0, &e0);
            rel_of(j, pass == 0 ? 0 : m, &b1, &e1);
            for (int e = b0; e < e0; ++e)
              for (int f = b1; f < e1; ++f)
                hm[((m - 1) << 16) | pidx(B->rel_src[e], B->rel_src[f])] += B->rel_fac[e] * B->rel_fac[f];
          }
        }
        B->pair_ij.push_back((i << 16) | j);
        for (auto& kv : gm)
          if (kv.second != 0.0) {
            B->cg_idx.push_back(kv.first);
            B->cg_coef.push_back((float)kv.second);
          }
        for (auto& kv : hm)
          if (kv.second != 0.0) {
            B->ch_idx.push_back(kv.first);
            B->ch_coef.push_back((float)kv.second);
          }
        B->cg_ptr.push_back((int32_t)B->cg_idx.size());
        B->ch_ptr.push_back((int32_t)B->ch_idx.size());
      }
    // Dirichlet facet congruences (all entries: the forms are not symmetric)
    B->ft_ptr.assign(1, 0);
    B->fm_ptr.assign(1, 0);
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) {
        std::map<int, double> tm, mm;
        int b0, e0, b1, e1;
        rel_of(i, 0, &b0, &e0);
        rel_of(j, 0, &b1, &e1);
        for (int e = b0; e < e0; ++e)
          for (int f = b1; f < e1; ++f) tm[pidx(B->rel_src[e], B->rel_src[f])] += B->rel_fac[e] * B->rel_fac[f];
        for (int m = 1; m < NVAR; ++m) {
          rel_of(j, m, &b1, &e1);
          for (int e = b0; e < e0; ++e)
            for (int f = b1; f < e1; ++f)
              mm[((m - 1) << 16) | pidx(B->rel_src[e], B->rel_src[f])] += B->rel_fac[e] * B->rel_fac[f];
        }
        for (auto& kv : tm)
          if (kv.second != 0.0) {
            B->ft_idx.push_back(kv.first);
            B->ft_coef.push_back((float)kv.second);
          }
        for (auto& kv : mm)
          if (kv.second != 0.0) {
            B->fm_idx.push_back(kv.first);
            B->fm_coef.push_back((float)kv.second);
          }
        B->ft_ptr.push_back((int32_t)B->ft_idx.size());
        B->fm_ptr.push_back((int32_t)B->fm_idx.size());
      }
  }
  B->coef.assign((size_t)B->nb * B->nmono, 0.0);
  B->sp_ptr.assign(B->nb * C + 1, 0);
  for (int j = 0; j < B->nb; ++j) {
    for (const Term& tm : funcs[j]) B->coef[(size_t)j * B->nmono + index.at(tm.e)] = rat_to_double(tm.num, tm.den);
    for (int comp = 0; comp < C; ++comp) {
      for (const Term& tm : funcs[j]) {
        int var = comp - 1;   // -1: U, 0: t, 1..n: x_m
        if (var < 0) {
          B->sp_mono.push_back(index.at(tm.e));
          B->sp_coef.push_back(rat_to_double(tm.num, tm.den));
        } else if (tm.e[var] > 0) {
          Exps e = tm.e;
          long long f = e[var];
          e[var] -= 1;
          B->sp_mono.push_back(index.at(e));
          B->sp_coef.push_back(rat_to_double(tm.num * f, tm.den));
        }
      }
      B->sp_ptr[j * C + comp + 1] = (int32_t)B->sp_mono.size();
    }
  }
  *out = B;
  return TP_OK;
}

extern "C" int tp_basis_info(const tp_basis* b, int32_t* nb, int32_t* nmono) {
  if (!b) {
    tp::set_error("tp_basis_info: null basis");
    return TP_ERR_ARG;
  }
  if (nb) *nb = b->nb;
  if (nmono) *nmono = b->nmono;
  return TP_OK;
}

extern "C" int tp_basis_export(const tp_basis* b, int32_t* exps, double* coef) {
  if (!b) {
    tp::set_error("tp_basis_export: null basis");
    return TP_ERR_ARG;
  }
  if (exps) std::copy(b->exps.begin(), b->exps.end(), exps);
  if (coef) std::copy(b->coef.begin(), b->coef.end(), coef);
  return TP_OK;
}

extern "C" void tp_destroy_basis(tp_basis* b) { delete b; }

// ---------------------------------------------------------------------------
// pitching
// ---------------------------------------------------------------------------
extern "C" int tp_pitch_mesh(const tp_mesh_desc* mesh, const tp_params* prm, tp_tents** out) {
  if (!out || !prm) {
    tp::set_error("tp_pitch_mesh: null argument");
    return TP_ERR_ARG;
  }
  if (!(prm->kappa > 0.0) || !(prm->T > 0.0) || !std::isfinite(prm->T)) {
    tp::set_error("tp_pitch_mesh: kappa and T must be positive");
    return TP_ERR_ARG;
  }
  tp::Topology topo;
  if (!tp::build_topology(mesh, &topo)) return TP_ERR_ARG;
  const int n = topo.dim;
  const int64_t nv = topo.nv;
  // edge speed: max c over the elements containing the edge
  std::map<std::pair<int32_t, int32_t>, double> ce;
  for (int64_t k = 0; k < topo.ne; ++k) {
    const int32_t* el = &topo.elems[k * (n + 1)];
    for (int i = 0; i <= n; ++i)
      for (int j = i + 1; j <= n; ++j) {
        auto key = std::make_pair(std::min(el[i], el[j]), std::max(el[i], el[j]));
        auto it = ce.find(key);
        if (it == ce.end() || topo.c[k] > it->second) ce[key] = topo.c[k];
      }
  }
  std::vector<double> delta(topo.nbr.size());
  for (int64_t v = 0; v < nv; ++v)
    for (int32_t e = topo.nbr_ptr[v]; e < topo.nbr_ptr[v + 1]; ++e) {
      int32_t w = topo.nbr[e];
      double s = 0.0;
      for (int d = 0; d < n; ++d) {
        double dx = topo.X[w * n + d] - topo.X[v * n + d];
        s = s + dx * dx;
      }
      double len = std::sqrt(s);
      double cc = ce.at(std::make_pair(std::min<int32_t>(v, w), std::max<int32_t>(v, w)));
      delta[e] = (prm->kappa * len) / cc;
    }
  const double T = prm->T;
  std::vector<double> tau(nv, 0.0);
  std::vector<int32_t> lam(nv, 0);
  std::vector<char> kept(nv, 0);
  struct Rec {
    int32_t level, round, v;
    double tb, tt;
  };
  std::vector<Rec> recs;
  std::vector<int32_t> R;
  // R0 of a round: tau_v < T and tau_v <= tau_w for every neighbour w.  Only
  // the pitched vertices and their neighbours change tau or see a change, so
  // the set is kept up to date instead of rescanned; it iterates in
  // increasing vertex order, the order of the greedy independent subset.
  auto in_r0 = [&](int64_t v) {
    if (!(tau[v] < T)) return false;
    for (int32_t e = topo.nbr_ptr[v]; e < topo.nbr_ptr[v + 1]; ++e)
      if (!(tau[v] <= tau[topo.nbr[e]])) return false;
    return true;
  };
  std::vector<char> is_r0(nv, 0);
  std::vector<int32_t> r0, r0_next, added;   // r0 sorted by vertex index
  for (int64_t v = 0; v < nv; ++v)
    if (in_r0(v)) {
      is_r0[v] = 1;
      r0.push_back((int32_t)v);
    }
  int64_t below_T = nv;                     // vertices with tau < T (all, as T > 0)
  std::vector<int32_t> touched;
  std::vector<char> mark(nv, 0);
  for (int32_t rnd = 1; below_T > 0; ++rnd) {
    R.clear();
    for (int32_t v : r0) {
      bool ok = true;
      for (int32_t e = topo.nbr_ptr[v]; e < topo.nbr_ptr[v + 1] && ok; ++e)
        if (kept[topo.nbr[e]]) ok = false;
      if (ok) {
        kept[v] = 1;
        R.push_back(v);
      }
    }
    if (R.empty()) {
      tp::set_error("tp_pitch_mesh: no vertex can advance (internal error)");
      return TP_ERR_CAUSALITY;
    }
    size_t first = recs.size();
    for (int32_t v : R) {
      double tt = T;
      int32_t lv = lam[v];
      for (int32_t e = topo.nbr_ptr[v]; e < topo.nbr_ptr[v + 1]; ++e) {
        double cand = tau[topo.nbr[e]] + delta[e];
        if (cand < tt) tt = cand;
        lv = std::max(lv, lam[topo.nbr[e]]);
      }
      recs.push_back({lv + 1, rnd, v, tau[v], tt});
    }
    touched.clear();
    for (size_t i = first; i < recs.size(); ++i) {
      const int32_t v = recs[i].v;
      tau[v] = recs[i].tt;
      lam[v] = recs[i].level;
      kept[v] = 0;
      if (!(tau[v] < T)) --below_T;
      if (!mark[v]) {
        mark[v] = 1;
        touched.push_back(v);
      }
      for (int32_t e = topo.nbr_ptr[v]; e < topo.nbr_ptr[v + 1]; ++e)
        if (!mark[topo.nbr[e]]) {
          mark[topo.nbr[e]] = 1;
          touched.push_back(topo.nbr[e]);
        }
    }
    added.clear();
    for (int32_t u : touched) {
      mark[u] = 0;
      const char now = in_r0(u) ? 1 : 0;
      if (now && !is_r0[u]) added.push_back(u);
      is_r0[u] = now;
    }
    std::sort(added.begin(), added.end());
    r0_next.clear();
    size_t a = 0;
    for (int32_t v : r0) {                  // merge the kept members with the new ones
      if (!is_r0[v]) continue;
      while (a < added.size() && added[a] < v) r0_next.push_back(added[a++]);
      r0_next.push_back(v);
    }
    while (a < added.size()) r0_next.push_back(added[a++]);
    r0.swap(r0_next);
  }
  // order (level, round, v): recs are in (round, v) order already, so a
  // counting sort on the level keeps the rest
  int32_t n_levels = 0;
  for (const Rec& r : recs) n_levels = std::max(n_levels, r.level);
  std::vector<int64_t> at((size_t)n_levels + 2, 0);
  for (const Rec& r : recs) at[r.level + 1]++;
  for (int32_t L = 1; L <= n_levels + 1; ++L) at[L] += at[L - 1];
  auto* tt = new tp_tents();
  tt->dim = n;
  tt->nv = nv;
  tt->T = T;
  tt->kappa = prm->kappa;
  const size_t nt = recs.size();
  tt->vert.resize(nt);
  tt->level.resize(nt);
  tt->round.resize(nt);
  tt->t_bot.resize(nt);
  tt->t_top.resize(nt);
  for (const Rec& r : recs) {
    const int64_t i = at[r.level]++;
    tt->vert[i] = r.v;
    tt->level[i] = r.level;
    tt->round[i] = r.round;
    tt->t_bot[i] = r.tb;
    tt->t_top[i] = r.tt;
  }
  tt->n_levels = n_levels;
  tt->level_ptr.assign(tt->n_levels + 1, 0);
  for (const Rec& r : recs) tt->level_ptr[r.level]++;
  for (int32_t L = 1; L <= tt->n_levels; ++L) tt->level_ptr[L] += tt->level_ptr[L - 1];
  *out = tt;
  return TP_OK;
}

extern "C" int tp_tents_info(const tp_tents* t, int64_t* n_tents, int32_t* n_levels) {
  if (!t) {
    tp::set_error("tp_tents_info: null tents");
    return TP_ERR_ARG;
  }
  if (n_tents) *n_tents = (int64_t)t->vert.size();
  if (n_levels) *n_levels = t->n_levels;
  return TP_OK;
}

extern "C" int tp_tents_export(const tp_tents* t, int32_t* vert, double* t_bot, double* t_top,
                               int32_t* level) {
  if (!t) {
    tp::set_error("tp_tents_export: null tents");
    return TP_ERR_ARG;
  }
  if (vert) std::copy(t->vert.begin(), t->vert.end(), vert);
  if (t_bot) std::copy(t->t_bot.begin(), t->t_bot.end(), t_bot);
  if (t_top) std::copy(t->t_top.begin(), t->t_top.end(), t_top);
  if (level) std::copy(t->level.begin(), t->level.end(), level);
  return TP_OK;
}

extern "C" void tp_destroy_tents(tp_tents* t) { delete t; }
