// Host-side Ruge-Stuben setup used as INPUT GENERATION for both the CUDA solve path and the
// CPU oracle: strength of connection, PMIS coarsening, BAMG-direct interpolation and ILU(0)
// (row-scaled LDU). The Galerkin product and transposes are done by the Python caller.
//
// Paper references (arXiv:2112.14681):
//   strength  |a_ij| >= theta * max_{k!=i} |a_ik|                         -- Sec. 5.1, eq. (strength)
//   PMIS      Luby-type maximal independent set with random weights       -- Sec. 5.1
//   BAMG-direct closed-form weights w_ij                                   -- Sec. 5.1, eq. (bamgdir)
//   ILU(0) as L (unit lower) * D_U * (I + U_s), rows of U scaled by diag  -- Sec. 5.3.2, Alg. 2 footnote
//
// Conventions: CSR with 0-based int32 indices, columns sorted ascending within each row,
// the diagonal entry present in every row.
#include <cstdint>
#include <cmath>
#include <vector>
#include <algorithm>

namespace {

inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// mode 0: S_i = { j != i : |a_ij| >= theta * max_{k != i} |a_ik| }   (absolute values)
// mode 1: S_i = { j != i : -a_ij >= theta * max_{k != i} (-a_ik) }    (classical sign-aware form:
//         only couplings of the opposite sign to a positive diagonal can be strong)
// stored as a flag per nonzero. The two coincide for M-matrices.
int g_strength_mode = 0;

void strength(int n, const int* rp, const int* ci, const double* v, double theta, std::vector<char>& s) {
  s.assign(rp[n], 0);
  const int mode = g_strength_mode;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double mx = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] != i) mx = std::max(mx, mode ? -v[p] : std::fabs(v[p]));
    if (mx <= 0.0) continue;
    const double thr = theta * mx;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] != i && v[p] != 0.0 && (mode ? -v[p] : std::fabs(v[p])) >= thr) s[p] = 1;
  }
}

}  // namespace

extern "C" {

void nsw_set_strength_mode(int mode) { g_strength_mode = mode; }

// PMIS C/F splitting. cf[i] = coarse index (>= 0) for C-points, -1 for F-points.
// Returns the number of coarse points, or -1 on invalid input.
int nsw_amg_coarsen(int n, const int* rp, const int* ci, const double* v, double theta, uint64_t seed, int* cf) {
  if (n <= 0) return -1;
  std::vector<char> s;
  strength(n, rp, ci, v, theta, s);
  // Transpose strength: ST_j = { i : j in S_i }.
  std::vector<int> strp(n + 1, 0), stci;
  for (int i = 0; i < n; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (s[p]) strp[ci[p] + 1]++;
  for (int i = 0; i < n; ++i) strp[i + 1] += strp[i];
  stci.resize(strp[n]);
  {
    std::vector<int> fill(strp.begin(), strp.end() - 1);
    for (int i = 0; i < n; ++i)
      for (int p = rp[i]; p < rp[i + 1]; ++p)
        if (s[p]) stci[fill[ci[p]]++] = i;
  }
  // Weights lambda_i = |ST_i| + U[0,1) from a counter-based generator.
  std::vector<double> lam(n);
  for (int i = 0; i < n; ++i) {
    const double u = (double)(splitmix64(seed ^ (0xA24BAED4963EE407ull * (uint64_t)(i + 1))) >> 11) * 0x1.0p-53;
    lam[i] = (double)(strp[i + 1] - strp[i]) + u;
  }
  // state: 0 undecided, 1 C, 2 F
  std::vector<char> st(n, 0);
  for (int i = 0; i < n; ++i) {
    bool dep_any = false;
    for (int p = rp[i]; p < rp[i + 1]; ++p) dep_any |= (s[p] != 0);
    const bool infl_any = strp[i + 1] > strp[i];
    if (!infl_any) st[i] = 2;  // influences no one: cannot serve as an interpolation point
    if (!dep_any && !infl_any) st[i] = 2;
  }
  std::vector<int> newc;
  for (int round = 0; round < 10 * n + 10; ++round) {
    newc.clear();
    bool any_undecided = false;
    for (int i = 0; i < n; ++i) {
      if (st[i] != 0) continue;
      any_undecided = true;
      bool is_max = true;
      auto beats = [&](int j) {  // true if undecided j outranks i
        if (j == i || st[j] != 0) return false;
        return lam[j] > lam[i] || (lam[j] == lam[i] && j > i);
      };
      for (int p = rp[i]; p < rp[i + 1] && is_max; ++p)
        if (s[p] && beats(ci[p])) is_max = false;
      for (int q = strp[i]; q < strp[i + 1] && is_max; ++q)
        if (beats(stci[q])) is_max = false;
      if (is_max) newc.push_back(i);
    }
    if (!any_undecided) break;
    for (int c : newc) st[c] = 1;
    for (int c : newc)
      for (int q = strp[c]; q < strp[c + 1]; ++q)
        if (st[stci[q]] == 0) st[stci[q]] = 2;
  }
  // F-points with no strong C-neighbour are promoted to C.
  for (int i = 0; i < n; ++i) {
    if (st[i] != 2) continue;
    bool has_c = false;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (s[p] && st[ci[p]] == 1) { has_c = true; break; }
    if (!has_c) st[i] = 1;
  }
  int nc = 0;
  for (int i = 0; i < n; ++i) cf[i] = (st[i] == 1) ? nc++ : -1;
  return nc;
}

// BAMG-direct interpolation with f = 1:
//   w_ij = -(a_ij + beta_i / |C_i^s|) / (a_ii + sum_{k weak} a_ik),  beta_i = sum_{k in F_i^s} a_ik.
// Output P (n x nc) in CSR; P arrays must hold n+1 row pointers and nnz(A) entries.
// Returns nnz(P) or -1 if a row has a zero denominator.
int64_t nsw_amg_interp(int n, const int* rp, const int* ci, const double* v, double theta, const int* cf,
                       int* prp, int* pci, double* pv) {
  std::vector<char> s;
  strength(n, rp, ci, v, theta, s);
  std::vector<int> cnt(n, 0);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    if (cf[i] >= 0) { cnt[i] = 1; continue; }
    int c = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (s[p] && cf[ci[p]] >= 0) ++c;
    cnt[i] = c;
  }
  prp[0] = 0;
  for (int i = 0; i < n; ++i) prp[i + 1] = prp[i] + cnt[i];
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int i = 0; i < n; ++i) {
    int o = prp[i];
    if (cf[i] >= 0) { pci[o] = cf[i]; pv[o] = 1.0; continue; }
    double aii = 0.0, weak = 0.0, beta = 0.0;
    int nc = 0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int j = ci[p];
      if (j == i) { aii += v[p]; continue; }
      if (!s[p]) weak += v[p];
      else if (cf[j] >= 0) ++nc;
      else beta += v[p];
    }
    const double den = aii + weak;
    if (den == 0.0 || nc == 0) { bad += 1; continue; }
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int j = ci[p];
      if (j == i || !s[p] || cf[j] < 0) continue;
      pci[o] = cf[j];
      pv[o] = -(v[p] + beta / nc) / den;
      ++o;
    }
  }
  // Coarse indices are increasing with fine index, so each row is already sorted.
  return bad ? -1 : (int64_t)prp[n];
}

// ILU(0) on the pattern of A, returned as  A ~ (I + L_s) D_U (I + U_s):
//   L_s strictly lower (multipliers), U_s strictly upper with rows scaled by 1/u_ii, dU_inv = 1/u_ii.
// L arrays hold n+1 / nnz_strict_lower entries, U arrays n+1 / nnz_strict_upper.
// Returns 0, or -(i+1) if a zero pivot appears in row i.
int nsw_ilu0(int n, const int* rp, const int* ci, const double* v, int* lrp, int* lci, double* lv, int* urp,
             int* uci, double* uv, double* dUinv) {
  std::vector<double> a(v, v + rp[n]);
  std::vector<int> diag(n, -1), pos(n, -1);
  for (int i = 0; i < n; ++i)
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) diag[i] = p;
  for (int i = 0; i < n; ++i) {
    if (diag[i] < 0) return -(i + 1);
    for (int p = rp[i]; p < rp[i + 1]; ++p) pos[ci[p]] = p;
    for (int p = rp[i]; p < diag[i]; ++p) {
      const int k = ci[p];
      const double piv = a[diag[k]];
      if (piv == 0.0) return -(k + 1);
      a[p] /= piv;
      const double lik = a[p];
      for (int q = diag[k] + 1; q < rp[k + 1]; ++q) {
        const int j = ci[q];
        if (pos[j] >= 0 && pos[j] > p) a[pos[j]] -= lik * a[q];
      }
    }
    for (int p = rp[i]; p < rp[i + 1]; ++p) pos[ci[p]] = -1;
    if (a[diag[i]] == 0.0) return -(i + 1);
  }
  lrp[0] = 0;
  urp[0] = 0;
  int lo = 0, uo = 0;
  for (int i = 0; i < n; ++i) {
    const double inv = 1.0 / a[diag[i]];
    dUinv[i] = inv;
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] < i) { lci[lo] = ci[p]; lv[lo] = a[p]; ++lo; }
      else if (ci[p] > i) { uci[uo] = ci[p]; uv[uo] = a[p] * inv; ++uo; }
    }
    lrp[i + 1] = lo;
    urp[i + 1] = uo;
  }
  return 0;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Sparse matrix product C = A B (CSR, OpenMP over rows, Gustavson accumulation with a dense
// marker per thread). Each row is formed by one thread in a fixed order, then its columns are
// sorted, so the result does not depend on the thread count. Used for the Galerkin product
// A_c = R (A P) of the hierarchy setup.
// ------------------------------------------------------------------------------------------
#include <omp.h>

extern "C" {

// Pass 1: row counts of C into crp[1..m] (crp[0] = 0, prefix-summed). Returns nnz(C).
int64_t nsw_spgemm_count(int m, int ncols_b, const int* arp, const int* aci, const int* brp, const int* bci, int64_t* crp) {
  std::vector<int64_t> cnt(m, 0);
#pragma omp parallel
  {
    std::vector<int> mark(ncols_b, -1);
#pragma omp for schedule(dynamic, 1024)
    for (int i = 0; i < m; ++i) {
      int64_t c = 0;
      for (int p = arp[i]; p < arp[i + 1]; ++p) {
        const int k = aci[p];
        for (int q = brp[k]; q < brp[k + 1]; ++q) {
          const int j = bci[q];
          if (mark[j] != i) { mark[j] = i; ++c; }
        }
      }
      cnt[i] = c;
    }
  }
  crp[0] = 0;
  for (int i = 0; i < m; ++i) crp[i + 1] = crp[i] + cnt[i];
  return crp[m];
}

// Pass 2: columns (sorted per row) and values of C.
void nsw_spgemm_fill(int m, int ncols_b, const int* arp, const int* aci, const double* av, const int* brp, const int* bci,
                     const double* bv, const int64_t* crp, int* cci, double* cv) {
#pragma omp parallel
  {
    std::vector<int64_t> pos(ncols_b, -1);
    std::vector<std::pair<int, double>> row;
#pragma omp for schedule(dynamic, 1024)
    for (int i = 0; i < m; ++i) {
      row.clear();
      for (int p = arp[i]; p < arp[i + 1]; ++p) {
        const int k = aci[p];
        const double a = av[p];
        for (int q = brp[k]; q < brp[k + 1]; ++q) {
          const int j = bci[q];
          if (pos[j] < 0) { pos[j] = (int64_t)row.size(); row.emplace_back(j, a * bv[q]); }
          else row[pos[j]].second += a * bv[q];
        }
      }
      for (auto& e : row) pos[e.first] = -1;
      std::sort(row.begin(), row.end(), [](const std::pair<int, double>& x, const std::pair<int, double>& y) { return x.first < y.first; });
      int64_t o = crp[i];
      for (auto& e : row) { cci[o] = e.first; cv[o] = e.second; ++o; }
    }
  }
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// ILUT(droptol, lfil) (dual-threshold incomplete LU, row by row) and Ruiz scaling of U, the
// factorisation and scaling of the ILUT smoother of Algorithm 2 (Sec. 5.3.3).
//   A ~ (I + L_s) U, L_s strictly lower, U upper with its diagonal.
//   In row i: tau_i = droptol * ||a_i||_2; multipliers below tau_i are dropped; after the
//   elimination entries below tau_i are dropped and at most lfil entries (largest magnitude)
//   are kept in each of the L and strict-U parts; the diagonal is always kept.
// Output arrays are sized by the caller with the bounds n*lfil (L) and n*(lfil+1) (U); the
// function returns 0 and the actual counts, or -(i+1) on a zero pivot in row i.
// ------------------------------------------------------------------------------------------
#include <set>

extern "C" {

int nsw_ilut(int n, const int* rp, const int* ci, const double* v, double droptol, int lfil, int* lrp, int* lci,
             double* lv, int* urp, int* uci, double* uv, int64_t* counts) {
  std::vector<double> w(n, 0.0);
  std::vector<char> used(n, 0);
  std::vector<int> nz;
  std::vector<int64_t> urow(n + 1, 0);  // filled progressively
  int64_t lo = 0, uo = 0;
  lrp[0] = 0;
  urp[0] = 0;
  std::vector<int> udiag(n, -1);
  for (int i = 0; i < n; ++i) {
    double nrm = 0.0;
    nz.clear();
    std::set<int> lower;  // pending lower columns in increasing order
    for (int p = rp[i]; p < rp[i + 1]; ++p) {
      const int j = ci[p];
      w[j] = v[p];
      used[j] = 1;
      nz.push_back(j);
      nrm += v[p] * v[p];
      if (j < i) lower.insert(j);
    }
    const double tau = droptol * std::sqrt(nrm);
    while (!lower.empty()) {
      const int k = *lower.begin();
      lower.erase(lower.begin());
      const double piv = uv[udiag[k]];
      double lik = w[k] / piv;
      if (std::fabs(lik) < tau) {
        w[k] = 0.0;
        continue;
      }
      w[k] = lik;
      for (int q = udiag[k] + 1; q < urp[k + 1]; ++q) {
        const int j = uci[q];
        if (!used[j]) {
          used[j] = 1;
          w[j] = 0.0;
          nz.push_back(j);
          if (j < i) lower.insert(j);
        }
        w[j] -= lik * uv[q];
      }
    }
    // split, drop small entries, keep the lfil largest per part
    std::vector<std::pair<double, int>> L, U;
    double diag = 0.0;
    bool has_diag = false;
    for (int j : nz) {
      const double x = w[j];
      if (j == i) { diag = x; has_diag = true; }
      else if (x != 0.0 && std::fabs(x) >= tau) (j < i ? L : U).emplace_back(-std::fabs(x), j);
      used[j] = 0;
    }
    auto keep = [&](std::vector<std::pair<double, int>>& part) {
      if ((int)part.size() > lfil) {
        std::nth_element(part.begin(), part.begin() + lfil, part.end());
        part.resize(lfil);
      }
      std::sort(part.begin(), part.end(), [](const std::pair<double, int>& a, const std::pair<double, int>& b) { return a.second < b.second; });
    };
    keep(L);
    keep(U);
    if (!has_diag || diag == 0.0) return -(i + 1);
    for (auto& e : L) { lci[lo] = e.second; lv[lo] = w[e.second]; ++lo; }
    lrp[i + 1] = (int)lo;
    udiag[i] = (int)uo;
    uci[uo] = i; uv[uo] = diag; ++uo;
    for (auto& e : U) { uci[uo] = e.second; uv[uo] = w[e.second]; ++uo; }
    urp[i + 1] = (int)uo;
    for (int j : nz) w[j] = 0.0;
  }
  counts[0] = lo;
  counts[1] = uo;
  return 0;
}

// Ruiz equilibration of a (square, sparse) matrix M: find positive D_r, D_c with every row and
// column of D_r M D_c having largest magnitude 1 (to `tol`), by repeated division with the
// square roots of the current row and column maxima. Returns the sweeps used.
int nsw_ruiz(int n, const int* rp, const int* ci, const double* v, double tol, int maxit, double* dr, double* dc) {
  std::vector<double> rmax(n), cmax(n);
  for (int i = 0; i < n; ++i) dr[i] = dc[i] = 1.0;
  int it = 0;
  for (; it < maxit; ++it) {
    std::fill(rmax.begin(), rmax.end(), 0.0);
    std::fill(cmax.begin(), cmax.end(), 0.0);
    for (int i = 0; i < n; ++i)
      for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const double a = std::fabs(dr[i] * v[p] * dc[ci[p]]);
        rmax[i] = std::max(rmax[i], a);
        cmax[ci[p]] = std::max(cmax[ci[p]], a);
      }
    double dev = 0.0;
    for (int i = 0; i < n; ++i) {
      if (rmax[i] > 0) dev = std::max(dev, std::fabs(1.0 - rmax[i]));
      if (cmax[i] > 0) dev = std::max(dev, std::fabs(1.0 - cmax[i]));
    }
    if (dev <= tol) break;
    for (int i = 0; i < n; ++i) {
      if (rmax[i] > 0) dr[i] /= std::sqrt(rmax[i]);
      if (cmax[i] > 0) dc[i] /= std::sqrt(cmax[i]);
    }
  }
  return it;
}

// Henrici's departure from normality of D_r U D_c for an upper triangular U (Sec. 5.3:
// dep(A)^2 = ||A||_F^2 - ||D||_F^2 with D the eigenvalues, here the diagonal): the Frobenius
// norm of the scaled strictly upper part. Also nu = ||diag(U~)^-1 U~ - I||_F, the ||U_s||_F of the
// unit-diagonal form U~ = diag(U~)(I + U_s) that the theorem's bound is stated for.
static void ruiz_dep(int n, const int* rp, const int* ci, const double* v, const double* dr, const double* dc,
                     double* dep, double* nu) {
  double d2 = 0.0, n2 = 0.0;
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] == i) diag = dr[i] * v[p] * dc[i];
    for (int p = rp[i]; p < rp[i + 1]; ++p)
      if (ci[p] != i) {
        const double a = dr[i] * v[p] * dc[ci[p]];
        d2 += a * a;
        if (diag != 0.0) n2 += (a / diag) * (a / diag);
      }
  }
  *dep = std::sqrt(d2);
  *nu = std::sqrt(n2);
}

// Ruiz scaling of an upper triangular U with the early termination the paper proposes after the
// dep(U) bound (Sec. 5.3, eq. depU): before each sweep k the departure from normality dep_k of
// the current scaled factor is compared with dep_factor * sqrt((2 sqrt(n) + nu_k) nu_k); the
// iteration stops when it is below, when dep_k no longer decreases (then the previous sweep's
// scaling is kept: the paper observes dep(U) reaching its minimum after one or two sweeps), when
// the row and column maxima are within `tol` of one, or after maxit sweeps.
// info (7 doubles): dep and nu of the returned scaling, its bound, dep of the unscaled U,
// the stop reason (0 tol, 1 dep below bound, 2 dep increased, 3 maxit), sweeps, 0.
int nsw_ruiz_dep(int n, const int* rp, const int* ci, const double* v, double tol, int maxit, double dep_factor,
                 double* dr, double* dc, double* info) {
  std::vector<double> rmax(n), cmax(n), pr(n), pc(n);
  for (int i = 0; i < n; ++i) dr[i] = dc[i] = 1.0;
  double dep = 0.0, nu = 0.0;
  ruiz_dep(n, rp, ci, v, dr, dc, &dep, &nu);
  info[3] = dep;
  double prev = INFINITY, prev_nu = 0.0;
  int reason = 3, it = 0;
  for (; it < maxit; ++it) {
    const double bound = std::sqrt((2.0 * std::sqrt((double)n) + nu) * nu);
    if (it > 0 && dep >= prev) {  // no longer decreasing: back to the previous sweep's scaling
      for (int i = 0; i < n; ++i) {
        dr[i] = pr[i];
        dc[i] = pc[i];
      }
      dep = prev;
      nu = prev_nu;
      --it;
      reason = 2;
      break;
    }
    if (dep <= dep_factor * bound) {
      reason = 1;
      break;
    }
    std::fill(rmax.begin(), rmax.end(), 0.0);
    std::fill(cmax.begin(), cmax.end(), 0.0);
    for (int i = 0; i < n; ++i)
      for (int p = rp[i]; p < rp[i + 1]; ++p) {
        const double a = std::fabs(dr[i] * v[p] * dc[ci[p]]);
        rmax[i] = std::max(rmax[i], a);
        cmax[ci[p]] = std::max(cmax[ci[p]], a);
      }
    double dev = 0.0;
    for (int i = 0; i < n; ++i) {
      if (rmax[i] > 0) dev = std::max(dev, std::fabs(1.0 - rmax[i]));
      if (cmax[i] > 0) dev = std::max(dev, std::fabs(1.0 - cmax[i]));
    }
    if (dev <= tol) {
      reason = 0;
      break;
    }
    for (int i = 0; i < n; ++i) {
      pr[i] = dr[i];
      pc[i] = dc[i];
      if (rmax[i] > 0) dr[i] /= std::sqrt(rmax[i]);
      if (cmax[i] > 0) dc[i] /= std::sqrt(cmax[i]);
    }
    prev = dep;
    prev_nu = nu;
    ruiz_dep(n, rp, ci, v, dr, dc, &dep, &nu);
  }
  info[0] = dep;
  info[1] = nu;
  info[2] = std::sqrt((2.0 * std::sqrt((double)n) + nu) * nu);
  info[4] = reason;
  info[5] = it;
  info[6] = 0.0;
  return it;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Input generation for the graded 27-point case: Q1 assembly and symmetric permutation. Both
// reproduce the Python generator's scipy operations bit for bit (same products, sums and order)
// and only make them parallel.
// ------------------------------------------------------------------------------------------
namespace {
inline double tri(const double* d, const double* o, int a, int b) {
  return a == b ? d[a] : o[a < b ? a : b];  // symmetric tridiagonal entry, |a - b| <= 1
}
}  // namespace

extern "C" {

// A = Mz (x) My (x) Kx + Mz (x) Ky (x) Mx + Kz (x) My (x) Mx on e^3 interior nodes (x fastest),
// from the diagonals (d) and off-diagonals (o) of the assembled 1D stiffness K and mass M
// matrices (x and y share Kx, Mx). Each entry is ((mz * my) * kx + (mz * ky) * mx) + (kz * my) * mx
// (the order of scipy's kron products and CSR sums); exact zeros are dropped as scipy's sum does.
// rp: n + 1 entries, ci / v: (3e - 2)^3 entries. Returns nnz.
int64_t nsw_q1_assemble(int e, const double* kxd, const double* kxo, const double* mxd, const double* mxo,
                        const double* kzd, const double* kzo, const double* mzd, const double* mzo, int64_t* rp,
                        int* ci, double* v) {
  const int64_t n = (int64_t)e * e * e;
  rp[0] = 0;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n; ++r) {
    const int ix = (int)(r % e), iy = (int)((r / e) % e), iz = (int)(r / ((int64_t)e * e));
    const int cx = (ix > 0) + 1 + (ix < e - 1), cy = (iy > 0) + 1 + (iy < e - 1), cz = (iz > 0) + 1 + (iz < e - 1);
    rp[r + 1] = (int64_t)cx * cy * cz;
  }
  for (int64_t r = 0; r < n; ++r) rp[r + 1] += rp[r];
  int64_t zeros = 0;
#pragma omp parallel for schedule(static) reduction(+ : zeros)
  for (int64_t r = 0; r < n; ++r) {
    const int ix = (int)(r % e), iy = (int)((r / e) % e), iz = (int)(r / ((int64_t)e * e));
    int64_t p = rp[r];
    for (int jz = iz - 1; jz <= iz + 1; ++jz) {
      if (jz < 0 || jz >= e) continue;
      const double mz = tri(mzd, mzo, iz, jz), kz = tri(kzd, kzo, iz, jz);
      for (int jy = iy - 1; jy <= iy + 1; ++jy) {
        if (jy < 0 || jy >= e) continue;
        const double my = tri(mxd, mxo, iy, jy), ky = tri(kxd, kxo, iy, jy);
        const double t1 = mz * my, t2 = mz * ky, t3 = kz * my;
        for (int jx = ix - 1; jx <= ix + 1; ++jx) {
          if (jx < 0 || jx >= e) continue;
          const double kx = tri(kxd, kxo, ix, jx), mx = tri(mxd, mxo, ix, jx);
          const double val = (t1 * kx + t2 * mx) + t3 * mx;  // built with -ffp-contract=off: no FMAs
          ci[p] = (int)(jx + (int64_t)e * (jy + (int64_t)e * jz));
          v[p] = val;
          zeros += (val == 0.0);
          ++p;
        }
      }
    }
  }
  if (zeros) {  // never expected for these operators; compact serially to match scipy
    int64_t q = 0;
    for (int64_t r = 0; r < n; ++r) {
      const int64_t b = rp[r], end = rp[r + 1];
      rp[r] = q;
      for (int64_t p = b; p < end; ++p)
        if (v[p] != 0.0) {
          ci[q] = ci[p];
          v[q] = v[p];
          ++q;
        }
    }
    rp[n] = q;
  }
  return rp[n];
}

// B = P A P^T for the ordering perm (new row k is old row perm[k]; new column of old column c is
// inv[c] with inv[perm[k]] = k), columns sorted ascending in each row, values copied unchanged:
// scipy's A[perm, :][:, perm] followed by sort_indices.
void nsw_sym_permute(int n, const int* rp, const int* ci, const double* v, const int* perm, int* brp, int* bci,
                     double* bv) {
  std::vector<int> inv(n);
#pragma omp parallel for schedule(static)
  for (int k = 0; k < n; ++k) inv[perm[k]] = k;
  brp[0] = 0;
  for (int k = 0; k < n; ++k) brp[k + 1] = brp[k] + (rp[perm[k] + 1] - rp[perm[k]]);
#pragma omp parallel for schedule(dynamic, 4096)
  for (int k = 0; k < n; ++k) {
    const int o = perm[k];
    int q = brp[k];
    for (int p = rp[o]; p < rp[o + 1]; ++p, ++q) {
      // insertion into the sorted prefix [brp[k], q)
      const int c = inv[ci[p]];
      const double x = v[p];
      int t = q;
      while (t > brp[k] && bci[t - 1] > c) {
        bci[t] = bci[t - 1];
        bv[t] = bv[t - 1];
        --t;
      }
      bci[t] = c;
      bv[t] = x;
    }
  }
}

}  // extern "C"
