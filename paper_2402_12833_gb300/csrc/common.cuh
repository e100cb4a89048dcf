// Internal definitions shared by the CUDA translation units of libmpcg.
//
// Padded grid layout
// ------------------
// A grid has n_a unknown nodes along axis a (the nodes of the axis minus its
// Dirichlet faces).  Every vector (and every stencil plane) of that grid is a
// padded box with pitches px >= nx + 1 (a multiple of 4, so that rows start
// on 16-byte boundaries), py = ny + 1 and, in 3D, pz = nz + 1: unknown
// (x, y[, z]) lives at  G + x + px*y [+ px*py*z].  Entries with x >= nx,
// y >= ny or z >= nz are pads that are always zero; because every pitch
// exceeds the extent, the pad of row y-1 sits at the address of (x = -1, y),
// the pad row of plane z-1 at (y = -1, z), and so on, so one pad layer
// serves as the zero ghost on both sides of every axis -- for Dirichlet
// faces (eliminated nodes) and free faces (no coupling) alike.  A guard of
// G = px*py + px + 1 (3D; px + 1 in 2D) zero elements in front makes
// (-1,-1,-1) addressable (G is rounded up to a multiple of 32); a second zero
// guard of G elements follows the box, so every neighbour of every box
// entry, pads included, lies inside the vector's own zeroed storage.
// Vector unknowns (ncomp = 3 components per node, 3D) stack one such box per
// component: component a of node (x, y, z) lives at
// G + a*cstride + x + px*y + px*py*z with cstride = px*py*pz, and the pad
// plane z = nz of component a is the zero ghost below component a+1.
// Stencils therefore need no boundary tests, interpolation reads zero
// parents outside the grid, and sums over a whole padded array equal sums
// over the unknowns.  For the all-Dirichlet grids with 2^k - 1 unknowns per
// side every pitch is 2^k.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpcg.h"
#include "dw.cuh"

namespace mpcg {

constexpr int kMaxCols = MPCG_MAX_COLS;
constexpr int kMaxVecCols = 8;   // columns of the vector (3 unknowns per node) block SpMM
constexpr int kMaxWindow = MPCG_MAX_WINDOW;
constexpr int kMaxLevels = 12;
constexpr int kBlock = 256;

// Division by a run-time constant d by one 64-bit multiply and a shift
// (the round-up multiplier of Granlund and Montgomery, "Division by
// invariant integers using multiplication", 1994): with l = ceil(log2 d),
// s = 32 + l and m = ceil(2^s / d), q = (n m) >> s equals n / d for all
// 0 <= n < 2^31 (the error n (m - 2^s/d) / 2^s stays below 1/d).
struct FastDiv {
  unsigned long long m;
  int s;
};

inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.s = 32 + l;
  f.m = ((1ull << f.s) + d - 1) / d;
  return f;
}

__host__ __device__ inline unsigned fdiv(unsigned n, const FastDiv& f) {
  return (unsigned)(((unsigned long long)n * f.m) >> f.s);
}

// A batch of nb problems on the same grid stores every vector, column and
// stencil plane as nb consecutive padded arrays of len elements: problem b of
// column c starts at c * cp + b * len with the column pitch cp = nb * len.
// Because each padded array carries its own zero guards, stencils and
// transfers never reach from one problem into the next.  Kernels take the
// problem index from blockIdx.y (nb = 1 is the single-problem case).
struct GridDesc {
  int dim;        // 2 or 3
  int ncomp;      // unknowns per node (1, or 3 for 3D elasticity)
  int nx, ny, nz; // unknown nodes per axis (nz = 1 in 2D)
  int lox, loy, loz;  // 1 where the low face of the axis is Dirichlet (sets the transfer parity)
  int px, py, pz; // pitches (pz = 1 in 2D)
  long long pxy;  // px * py
  long long cstride;  // elements of one component box
  FastDiv dvx, dvy, dvz;  // division by px, py, pz
  int n1;         // nx (all-Dirichlet cubes: unknown nodes per side)
  int lp;         // log2(px) when px is a power of two, else -1
  int p;          // px
  long long G;    // guard elements before the first entry
  long long npts; // ncomp * cstride (entries of the padded boxes)
  long long len;  // 2G + npts rounded up (elements per problem per vector)
  long long n;    // unknowns ncomp * nx * ny * nz
  int nb;         // problems in the batch
  long long cp;   // column / plane pitch = nb * len
};

// Grid with `nodes` nodes per side, Dirichlet faces `faces` (bit 2a: low
// face of axis a, bit 2a+1: high face), ncomp unknowns per node.
inline GridDesc make_grid_nodes(int dim, int nodes, unsigned faces, int ncomp, int nb = 1) {
  GridDesc g;
  g.nb = nb;
  g.dim = dim;
  g.ncomp = ncomp;
  int ext[3] = {1, 1, 1}, lo[3] = {0, 0, 0};
  for (int a = 0; a < dim; ++a) {
    lo[a] = (faces >> (2 * a)) & 1;
    ext[a] = nodes - lo[a] - (int)((faces >> (2 * a + 1)) & 1);
  }
  g.nx = ext[0]; g.ny = ext[1]; g.nz = ext[2];
  g.lox = lo[0]; g.loy = lo[1]; g.loz = lo[2];
  g.px = (g.nx + 1 + 3) / 4 * 4;
  g.py = g.ny + 1;
  g.pz = dim == 3 ? g.nz + 1 : 1;
  g.pxy = (long long)g.px * g.py;
  g.cstride = g.pxy * g.pz;
  g.dvx = make_fastdiv(g.px);
  g.dvy = make_fastdiv(g.py);
  g.dvz = make_fastdiv(g.pz);
  g.n1 = g.nx;
  g.p = g.px;
  g.lp = -1;
  for (int k = 0; k < 31; ++k)
    if ((1 << k) == g.px) g.lp = k;
  // guard rounded up to 32 elements so that every padded box starts on a
  // 128-byte boundary (vector loads of 4 floats / 2 doubles stay aligned)
  const long long guard = dim == 3 ? g.pxy + g.px + 1 : (long long)g.px + 1;
  g.G = (guard + 31) / 32 * 32;
  g.npts = (long long)ncomp * g.cstride;
  // a zero guard of G elements after the box as well: the vectorised stencil
  // kernels evaluate pad entries too, and their neighbours reach up to
  // px*py + px elements past the box
  g.len = (2 * g.G + g.npts + 31) / 32 * 32;
  g.n = (long long)ncomp * g.nx * g.ny * g.nz;
  g.cp = (long long)nb * g.len;
  return g;
}

// Unstructured ("flat") grid of n unknowns for an algebraic hierarchy:
// unknown i lives at G + i of a box of npts = n rounded up to 32 entries,
// the tail of the box and the guards being zero, so the block kernels (which
// only read G, npts, len, cp and nb) run on it unchanged.  It is described as
// one row (nx = n, ny = nz = 1, dim = 1) so that padded_index() maps i to G + i.
inline GridDesc make_grid_flat(long long n, int nb = 1) {
  GridDesc g;
  g.nb = nb;
  g.dim = 1;
  g.ncomp = 1;
  g.nx = (int)n;
  g.ny = 1;
  g.nz = 1;
  g.lox = g.loy = g.loz = 0;
  g.px = (int)((n + 31) / 32 * 32);
  g.py = 1;
  g.pz = 1;
  g.pxy = g.px;
  g.cstride = g.px;
  g.dvx = make_fastdiv(g.px);
  g.dvy = make_fastdiv(1);
  g.dvz = make_fastdiv(1);
  g.n1 = g.nx;
  g.p = g.px;
  g.lp = -1;
  g.G = 32;
  g.npts = g.px;
  g.len = (2 * g.G + g.npts + 31) / 32 * 32;
  g.n = n;
  g.cp = (long long)nb * g.len;
  return g;
}

// A sparse matrix of an algebraic hierarchy on the device, in sliced
// ELLPACK form with one warp per slice and g = 2^lg lanes per row: slice s
// holds the 32/g rows s*32/g ... s*32/g + 32/g - 1; lane l serves row
// l / g of the slice and takes entries q, q + g, q + 2g, ... of it
// (q = l mod g).  Slot k of lane l is stored at sptr[s] + 32 k + l, so a
// warp reads each slot of its rows in one coalesced load; the slice has
// (sptr[s+1] - sptr[s]) / 32 slots.  Missing entries, and the rows past
// `rows` in the last slice, are padded with column 0 and value 0.  g = 1
// suits short rows (one thread per row); long rows (restrictions, the wider
// coarse operators) take several lanes and a shuffle reduction.
template <typename T>
struct EllDev {
  int rows, cols, nslices, lg;
  const int* sptr;
  const int* col;
  const T* val;
};

// All-Dirichlet scalar grid with n1 unknowns per side.
inline GridDesc make_grid(int dim, int n1, int nb = 1) { return make_grid_nodes(dim, n1 + 2, 0x3Fu, 1, nb); }

// Padded offset (from the start of the problem's array) of compact unknown
// i = a + ncomp * node, node lexicographic over the unknown nodes, x fastest.
__host__ __device__ inline long long padded_index(const GridDesc& g, long long i) {
  const int a = (int)(i % g.ncomp);
  const long long node = i / g.ncomp;
  const int x = (int)(node % g.nx);
  const long long q = node / g.nx;
  const int y = (int)(q % g.ny);
  const int z = (int)(q / g.ny);
  return g.G + a * g.cstride + x + (long long)g.px * y + g.pxy * z;
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
  int dropped_total;   // search columns dropped by the drop rule, summed over blocks
  int pinv_fallbacks;  // blocks whose Gram took the eigenvalue pseudo-inverse
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
