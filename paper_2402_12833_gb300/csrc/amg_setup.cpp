// Smoothed-aggregation setup on the host (the hierarchy is built once per
// matrix; the solve runs on the device).  Definitions in amg.h.
#include "amg.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <limits>

namespace mpcg {
namespace amg {

bool check_input(int n, const int* ptr, const int* col, const double* val, std::string& err) {
  char buf[256];
  if (n < 1 || !ptr || !col || !val) {
    err = "matrix: n >= 1 and non-NULL row offsets, columns and values are required";
    return false;
  }
  if (ptr[0] != 0) {
    err = "matrix: row offsets must start at 0";
    return false;
  }
  for (int i = 0; i < n; ++i) {
    if (ptr[i + 1] < ptr[i]) {
      snprintf(buf, sizeof buf, "matrix: row offsets decrease at row %d", i);
      err = buf;
      return false;
    }
    bool diag = false;
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
      const int j = col[e];
      if (j < 0 || j >= n || (e > ptr[i] && j <= col[e - 1])) {
        snprintf(buf, sizeof buf, "matrix: row %d has a column out of range or out of ascending order", i);
        err = buf;
        return false;
      }
      if (!std::isfinite(val[e])) {
        snprintf(buf, sizeof buf, "matrix: row %d has a non-finite value", i);
        err = buf;
        return false;
      }
      if (j == i) {
        diag = true;
        if (!(val[e] > 0.0)) {
          snprintf(buf, sizeof buf, "matrix: diagonal entry %d is not positive", i);
          err = buf;
          return false;
        }
      }
    }
    if (!diag) {
      snprintf(buf, sizeof buf, "matrix: row %d has no diagonal entry", i);
      err = buf;
      return false;
    }
  }
  // symmetry: every a_ij has a partner a_ji equal to 1e-12 of the larger
  for (int i = 0; i < n; ++i)
    for (int e = ptr[i]; e < ptr[i + 1]; ++e) {
      const int j = col[e];
      const int* b = col + ptr[j];
      const int* f = std::lower_bound(b, col + ptr[j + 1], i);
      const double v = val[e];
      const double u = (f != col + ptr[j + 1] && *f == i) ? val[f - col] : 0.0;
      if (std::fabs(u - v) > 1e-12 * std::max(std::fabs(u), std::fabs(v))) {
        snprintf(buf, sizeof buf, "matrix: not symmetric at (%d, %d)", i, j);
        err = buf;
        return false;
      }
    }
  return true;
}

void transpose(const Csr& A, Csr& At) {
  At.rows = A.cols;
  At.cols = A.rows;
  At.ptr.assign((size_t)A.cols + 1, 0);
  for (int j : A.col) ++At.ptr[(size_t)j + 1];
  for (int j = 0; j < A.cols; ++j) At.ptr[(size_t)j + 1] += At.ptr[j];
  At.col.resize(A.col.size());
  At.val.resize(A.val.size());
  std::vector<int> next(At.ptr.begin(), At.ptr.end() - 1);
  for (int i = 0; i < A.rows; ++i)   // rows in ascending order: the transposed rows come out sorted
    for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      const int k = next[A.col[e]]++;
      At.col[k] = i;
      At.val[k] = A.val[e];
    }
}

void multiply(const Csr& A, const Csr& B, Csr& C) {
  C.rows = A.rows;
  C.cols = B.cols;
  C.ptr.assign((size_t)A.rows + 1, 0);
  C.col.clear();
  C.val.clear();
  std::vector<double> acc((size_t)B.cols, 0.0);
  std::vector<int> mark((size_t)B.cols, -1), touched;
  for (int i = 0; i < A.rows; ++i) {
    touched.clear();
    for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      const int k = A.col[e];
      const double a = A.val[e];
      for (int f = B.ptr[k]; f < B.ptr[k + 1]; ++f) {
        const int j = B.col[f];
        if (mark[j] != i) {
          mark[j] = i;
          acc[j] = 0.0;
          touched.push_back(j);
        }
        acc[j] += a * B.val[f];
      }
    }
    std::sort(touched.begin(), touched.end());
    for (int j : touched)
      if (acc[j] != 0.0) {
        C.col.push_back(j);
        C.val.push_back(acc[j]);
      }
    C.ptr[(size_t)i + 1] = (int)C.col.size();
  }
}

void strength(const Csr& A, double theta, Csr& S) {
  const int n = A.rows;
  Csr D;   // directed: j strongly influences i
  D.rows = D.cols = n;
  D.ptr.assign((size_t)n + 1, 0);
  for (int i = 0; i < n; ++i) {
    double m = -std::numeric_limits<double>::infinity();
    for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e)
      if (A.col[e] != i) m = std::max(m, -A.val[e]);
    for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e) {
      const double c = -A.val[e];
      if (A.col[e] != i && c > 0.0 && c >= theta * m) {
        D.col.push_back(A.col[e]);
        D.val.push_back(1.0);
      }
    }
    D.ptr[(size_t)i + 1] = (int)D.col.size();
  }
  Csr Dt;
  transpose(D, Dt);
  S.rows = S.cols = n;
  S.ptr.assign((size_t)n + 1, 0);
  S.col.clear();
  S.val.clear();
  for (int i = 0; i < n; ++i) {   // union of the sorted rows of D and D^T
    int a = D.ptr[i], b = Dt.ptr[i];
    const int ae = D.ptr[i + 1], be = Dt.ptr[i + 1];
    while (a < ae || b < be) {
      int j;
      if (b >= be || (a < ae && D.col[a] < Dt.col[b])) j = D.col[a++];
      else if (a >= ae || Dt.col[b] < D.col[a]) j = Dt.col[b++];
      else {
        j = D.col[a];
        ++a;
        ++b;
      }
      S.col.push_back(j);
      S.val.push_back(1.0);
    }
    S.ptr[(size_t)i + 1] = (int)S.col.size();
  }
}

int aggregate(const Csr& S, std::vector<int>& agg) {
  const int n = S.rows;
  agg.assign((size_t)n, -1);
  std::vector<char> first((size_t)n, 0);
  int na = 0;
  for (int i = 0; i < n; ++i) {   // pass 1
    const int b = S.ptr[i], e = S.ptr[i + 1];
    if (b == e || agg[i] >= 0) continue;
    bool free_nbrs = true;
    for (int k = b; k < e && free_nbrs; ++k) free_nbrs = agg[S.col[k]] < 0;
    if (!free_nbrs) continue;
    agg[i] = na;
    first[i] = 1;
    for (int k = b; k < e; ++k) {
      agg[S.col[k]] = na;
      first[S.col[k]] = 1;
    }
    ++na;
  }
  for (int i = 0; i < n; ++i) {   // pass 2
    if (agg[i] >= 0) continue;
    for (int k = S.ptr[i]; k < S.ptr[i + 1]; ++k)
      if (first[S.col[k]]) {
        agg[i] = agg[S.col[k]];
        break;
      }
  }
  return na;
}

void tentative(const std::vector<int>& agg, int na, Csr& T) {
  const int n = (int)agg.size();
  std::vector<double> size((size_t)na, 0.0);
  for (int a : agg)
    if (a >= 0) size[a] += 1.0;
  T.rows = n;
  T.cols = na;
  T.ptr.assign((size_t)n + 1, 0);
  T.col.clear();
  T.val.clear();
  for (int i = 0; i < n; ++i) {
    if (agg[i] >= 0) {
      T.col.push_back(agg[i]);
      T.val.push_back(1.0 / std::sqrt(size[agg[i]]));
    }
    T.ptr[(size_t)i + 1] = (int)T.col.size();
  }
}

static double diag_of(const Csr& A, int i) {
  for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e)
    if (A.col[e] == i) return A.val[e];
  return 0.0;
}

double gershgorin(const Csr& A) {
  double rho = 0.0;
  for (int i = 0; i < A.rows; ++i) {
    double s = 0.0;
    for (int e = A.ptr[i]; e < A.ptr[i + 1]; ++e) s += std::fabs(A.val[e]);
    rho = std::max(rho, s / std::fabs(diag_of(A, i)));
  }
  return rho;
}

void smoothed_prolongator(const Csr& A, const Csr& T, double w, Csr& P) {
  if (w == 0.0) {
    P = T;
    return;
  }
  const double s = w / gershgorin(A);
  Csr AT;
  multiply(A, T, AT);
  P.rows = T.rows;
  P.cols = T.cols;
  P.ptr.assign((size_t)T.rows + 1, 0);
  P.col.clear();
  P.val.clear();
  for (int i = 0; i < T.rows; ++i) {   // row i of T - diag(s / a_ii) (A T), merged by column
    const double d = s / diag_of(A, i);
    int a = T.ptr[i], b = AT.ptr[i];
    const int ae = T.ptr[i + 1], be = AT.ptr[i + 1];
    while (a < ae || b < be) {
      int j;
      double v;
      if (b >= be || (a < ae && T.col[a] < AT.col[b])) {
        j = T.col[a];
        v = T.val[a++];
      } else if (a >= ae || AT.col[b] < T.col[a]) {
        j = AT.col[b];
        v = 0.0 - d * AT.val[b++];
      } else {
        j = T.col[a];
        v = T.val[a++] - d * AT.val[b++];
      }
      if (v != 0.0) {
        P.col.push_back(j);
        P.val.push_back(v);
      }
    }
    P.ptr[(size_t)i + 1] = (int)P.col.size();
  }
}

void build(const Csr& A, const Params& p, Levels& out) {
  out.A.assign(1, A);
  out.P.clear();
  out.agg.clear();
  while ((int)out.A.size() < p.max_levels && out.A.back().rows > p.coarse_size) {
    const Csr& Af = out.A.back();
    Csr S, T, P, Pt, PtA, Ac;
    strength(Af, p.theta, S);
    std::vector<int> agg;
    const int na = aggregate(S, agg);
    if (na == 0 || na >= Af.rows) break;
    tentative(agg, na, T);
    smoothed_prolongator(Af, T, p.w, P);
    transpose(P, Pt);
    multiply(Pt, Af, PtA);
    multiply(PtA, P, Ac);
    out.P.push_back(std::move(P));
    out.agg.push_back(std::move(agg));
    out.A.push_back(std::move(Ac));
  }
}

bool ell_layout(const Csr& M, Ell& E) {
  E.rows = M.rows;
  E.cols = M.cols;
  const double mean = M.rows ? (double)M.nnz() / M.rows : 0.0;
  E.lg = 0;
  while (E.lg < 5 && (double)(2 << E.lg) <= mean / 6.0) ++E.lg;
  const int g = 1 << E.lg, rps = 32 >> E.lg;   // lanes per row, rows per slice
  E.nslices = (M.rows + rps - 1) / rps;
  E.sptr.assign((size_t)E.nslices + 1, 0);
  long long total = 0;
  for (int sl = 0; sl < E.nslices; ++sl) {
    int w = 0;
    for (int r = rps * sl; r < rps * sl + rps && r < M.rows; ++r) w = std::max(w, (M.ptr[r + 1] - M.ptr[r] + g - 1) / g);
    total += 32LL * w;
    if (total >= (1LL << 31)) return false;
    E.sptr[(size_t)sl + 1] = (int)total;
  }
  E.col.assign((size_t)total, 0);
  E.val.assign((size_t)total, 0.0);
  for (int sl = 0; sl < E.nslices; ++sl)
    for (int r = rps * sl; r < rps * sl + rps && r < M.rows; ++r)
      for (int e = M.ptr[r]; e < M.ptr[r + 1]; ++e) {
        const int idx = e - M.ptr[r];   // entry idx of the row: slot idx / g of lane (r - rps sl) g + idx mod g
        const size_t k = (size_t)E.sptr[sl] + 32 * (size_t)(idx / g) + (size_t)((r - rps * sl) * g + idx % g);
        E.col[k] = M.col[e];
        E.val[k] = M.val[e];
      }
  return true;
}

}  // namespace amg
}  // namespace mpcg
