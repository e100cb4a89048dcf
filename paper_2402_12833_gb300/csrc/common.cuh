// Internal definitions shared by the CUDA translation units of libmpcg.
//
// Padded grid layout
// ------------------
// Grid j has n1 = 2^k - 1 interior nodes per side.  Every vector (and every
// stencil plane) of that grid is stored with pitch p = n1 + 1 = 2^k along
// each axis: element (x, y[, z]) lives at  G + x + p*y [+ p*p*z]  for
// 0 <= x, y, z < p.  Coordinates equal to p-1 are pad entries that are always
// zero; because the pitch is exactly n1 + 1, the pad of row y-1 sits at the
// address of (x = -1, y), the pad row of plane z-1 at (y = -1, z), and so on,
// so one pad layer serves as the zero Dirichlet ghost on both sides of every
// axis.  A guard of G = p*p + p + 1 (3D; p + 1 in 2D) zero elements in front
// makes (-1,-1,-1) addressable (G is rounded up to a multiple of 32); a second
// zero guard of G elements follows the box, so every vector occupies
// len = 2G + p^dim rounded up to 32 elements and every neighbour of every
// box entry, pads included, lies inside the vector's own zeroed storage.
// Stencils therefore need no boundary tests,
// interpolation reads zero parents outside the grid, and sums over a whole
// padded array equal sums over the interior unknowns.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpcg.h"

namespace mpcg {

constexpr int kMaxCols = MPCG_MAX_COLS;
constexpr int kMaxWindow = MPCG_MAX_WINDOW;
constexpr int kMaxLevels = 12;
constexpr int kBlock = 256;

// A batch of nb problems on the same grid stores every vector, column and
// stencil plane as nb consecutive padded arrays of len elements: problem b of
// column c starts at c * cp + b * len with the column pitch cp = nb * len.
// Because each padded array carries its own zero guards, stencils and
// transfers never reach from one problem into the next.  Kernels take the
// problem index from blockIdx.y (nb = 1 is the single-problem case).
struct GridDesc {
  int dim;        // 2 or 3
  int n1;         // interior nodes per side
  int lp;         // log2(pitch)
  int p;          // pitch = n1 + 1
  long long G;    // guard elements before the first entry
  long long npts; // p^dim (entries of the padded box)
  long long len;  // 2G + npts rounded up (elements per problem per vector)
  long long n;    // interior unknowns n1^dim
  int nb;         // problems in the batch
  long long cp;   // column / plane pitch = nb * len
};

inline GridDesc make_grid(int dim, int n1, int nb = 1) {
  GridDesc g;
  g.nb = nb;
  g.dim = dim;
  g.n1 = n1;
  g.p = n1 + 1;
  int lp = 0;
  while ((1 << lp) < g.p) ++lp;
  g.lp = lp;
  long long p = g.p;
  // guard rounded up to 32 elements so that every padded box starts on a
  // 128-byte boundary (vector loads of 4 floats / 2 doubles stay aligned)
  const long long guard = dim == 3 ? p * p + p + 1 : p + 1;
  g.G = (guard + 31) / 32 * 32;
  g.npts = dim == 3 ? p * p * p : p * p;
  // a zero guard of G elements after the box as well: the vectorised stencil
  // kernels evaluate pad entries too, and the neighbours of the last pad
  // plane reach up to p*p + p elements past the box
  g.len = (2 * g.G + g.npts + 31) / 32 * 32;
  g.n = dim == 3 ? (long long)n1 * n1 * n1 : (long long)n1 * n1;
  g.cp = (long long)nb * g.len;
  return g;
}

// Linear offset of a stencil neighbour.
__host__ __device__ inline long long nb_offset(int p, int dx, int dy, int dz) {
  return (long long)dx + (long long)dy * p + (long long)dz * p * p;
}

// Solver state kept in device memory so that a captured iteration can run
// without host involvement.
struct DevState {
  int k;          // x updates done
  int count;      // blocks in the window
  int newest;     // ring slot of the newest block
  int done;       // 0 running, 1 converged, 2 maxit, 3 breakdown
  int maxit;
  int ncols;      // active column count C of this solver
  int m;          // window length
  int dropped_total;
  double rtol;
  double bnorm;
  double rnorm;
  double delta;
  double tau;
  double alpha[kMaxCols];
  double beta[kMaxWindow][kMaxCols][kMaxCols];
  double gpinv[kMaxWindow][kMaxCols][kMaxCols];
};

template <typename T>
struct Window {
  T* P[kMaxWindow];
  T* AP[kMaxWindow];
};

}  // namespace mpcg
