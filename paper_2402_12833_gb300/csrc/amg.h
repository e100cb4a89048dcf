// Host-side construction of an algebraic grid hierarchy by smoothed
// aggregation (Section 2.1 admits nested spaces built by agglomeration;
// Section 3, Example 2 builds them with an algebraic multigrid setup).  The
// published method restated here is smoothed aggregation after Vanek, Mandel
// and Brezina (Computing 56, 1996), with the classical signed strength
// measure of the Ruge-Stueben setup:
//   * j != i strongly influences i when -a_ij > 0 and
//     -a_ij >= theta * max_{k != i}(-a_ik); i and j are strongly coupled when
//     either influences the other;
//   * aggregation in index order: an unknown whose strong neighbours are all
//     free starts an aggregate with them; a free unknown then joins the
//     aggregate of its first strong neighbour (ascending column order) placed
//     by the first pass; unknowns with no strong neighbour stay outside;
//   * tentative prolongator T[i, a] = 1/sqrt(|a|);
//   * P = (I - (w / rho) D^-1 A) T with rho = max_i sum_j |a_ij| / |a_ii|;
//   * coarse operators P^T A P, coarsening until at most coarse_size
//     unknowns, max_levels grids, or no reduction.
// Sparse products accumulate each row in ascending order of the inner index
// and drop entries that cancel to exactly zero.
#pragma once

#include <string>
#include <vector>

namespace mpcg {
namespace amg {

struct Csr {
  int rows = 0, cols = 0;
  std::vector<int> ptr, col;   // ascending columns within a row
  std::vector<double> val;
  long long nnz() const { return (long long)col.size(); }
};

struct Params {
  double theta;      // strength threshold
  double w;          // prolongator smoothing weight (0: plain aggregation)
  int max_levels;    // grids including the finest
  int coarse_size;   // stop once a grid has at most this many unknowns
};

// Grids finest first: A[0] is the input; P[l] maps grid l+1 to grid l;
// agg[l][i] is the aggregate (unknown of grid l+1) of unknown i of grid l, or -1.
struct Levels {
  std::vector<Csr> A, P;
  std::vector<std::vector<int>> agg;
};

// Square, sorted, in-range, positive diagonal, symmetric to 1e-12 relative.
bool check_input(int n, const int* ptr, const int* col, const double* val, std::string& err);
void strength(const Csr& A, double theta, Csr& S);
int aggregate(const Csr& S, std::vector<int>& agg);
void tentative(const std::vector<int>& agg, int na, Csr& T);
double gershgorin(const Csr& A);
void transpose(const Csr& A, Csr& At);
void multiply(const Csr& A, const Csr& B, Csr& C);
void smoothed_prolongator(const Csr& A, const Csr& T, double w, Csr& P);
void build(const Csr& A, const Params& p, Levels& out);

// Sliced ELLPACK of a CSR matrix, the layout the device kernels read (one
// warp per slice, g = 2^lg lanes per row, slot k of lane l of slice s at
// sptr[s] + 32 k + l; padding: column 0, value 0).  Lanes per row: the
// largest power of two g <= 32 with g <= (mean row length) / 6.  Returns
// false when the stored entries would not fit 32-bit offsets.
struct Ell {
  int rows = 0, cols = 0, nslices = 0, lg = 0;
  std::vector<int> sptr, col;
  std::vector<double> val;
};
bool ell_layout(const Csr& M, Ell& E);

}  // namespace amg
}  // namespace mpcg
