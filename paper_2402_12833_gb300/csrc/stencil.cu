// Structured-grid kernels: layout conversion, block stencil SpMM (the A Z
// product of Section 2.2), residual, restriction R = P^T and prolongation P
// (Section 2.1), damped-Jacobi smoothing (Eq. 2), and the Galerkin product
// P^T A P that builds the coarse operators.
//
// The stencil kernels work on the padded layout described in common.cuh and
// give every thread a group of W consecutive x-points (W = 4 floats or
// 2 doubles: one 16-byte load per stencil plane and per grid row, plus one
// scalar on each side for the x-neighbours).  Stencil coefficients are zero
// at pad entries, so every output at a pad entry is exactly zero without a
// test.  blockIdx.y selects the problem of a batch (offset b * len; columns
// and stencil planes are cp = nb * len apart).
#include "kernels.cuh"
#include "tune.h"
#include "vec.cuh"

// stencil.cu compiles the float / double instances; stencil_dw.cu
// (MPCG_STENCIL_DW) the double-word ones and stencil_sym.cu
// (MPCG_STENCIL_SYM) the FP32 kernels on the symmetric half of the stencil.
#if defined(MPCG_STENCIL_DW) || defined(MPCG_STENCIL_SYM)
#define MPCG_STENCIL_PLAIN 0
#else
#define MPCG_STENCIL_PLAIN 1
#endif

namespace mpcg {

namespace {

// ---------------------------------------------------------------------------
template <typename TI, typename TO>
__global__ void k_pack(GridDesc g, const TI* __restrict__ src, long long ld, TO* __restrict__ dst, int ncols) {
  const long long n = g.n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * ncols;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / n);
    const long long i = t - (long long)c * n;
    dst[(long long)c * g.cp + padded_index(g, i)] = (TO)src[(long long)c * ld + i];
  }
}

// Pack of one FP64 column that also records whether it has a nonzero entry
// (nz = 1; the caller zeroes nz first).  Bit patterns are tested (no FP64
// arithmetic); -0.0 counts as nonzero.
template <typename TO>
__global__ void k_pack_flag(GridDesc g, const double* __restrict__ src, TO* __restrict__ dst, int* nz) {
  const long long n = g.n;
  bool any = false;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const double v = src[t];
    any |= __double_as_longlong(v) != 0;
    dst[padded_index(g, t)] = (TO)v;
  }
  if (__any_sync(0xffffffffu, any) && (threadIdx.x & 31) == 0) *nz = 1;
}

template <typename TI, typename TO>
__global__ void k_unpack(GridDesc g, const TI* __restrict__ src, TO* __restrict__ dst, long long ld, int ncols) {
  const long long n = g.n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * ncols;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / n);
    const long long i = t - (long long)c * n;
    dst[(long long)c * ld + i] = (TO)src[(long long)c * g.cp + padded_index(g, i)];
  }
}

// A grid row segment around a group: v[-1], v[0..W-1] (one aligned vector
// load), v[W].  Returned as e[0..W+1] with e[k] = v[k-1].
template <typename T>
__device__ __forceinline__ void load_row(const T* __restrict__ p, T (&e)[Vec<T>::W + 2]) {
  constexpr int W = Vec<T>::W;
  T mid[W];
  Vec<T>::load_keep(p, mid);
  e[0] = p[-1];
#pragma unroll
  for (int w = 0; w < W; ++w) e[w + 1] = mid[w];
  e[W + 1] = p[W];
}

// The same row segment with the neighbours v[-1] and v[W] taken from the
// adjacent lanes' vectors by warp shuffles (lanes of a warp hold consecutive
// groups); a lane whose neighbour lane is idle (warp edge, tail) loads them
// itself.  Every lane of the warp must call it; an idle lane (active =
// false) reads nothing.  Fewer L1 wavefronts than the scalar loads; used by
// the Jacobi sweep, which reads two rows per stencil row (measured faster
// there, slower in the multi-column SpMM, whose loads then wait longer).
template <typename T, int W = Vec<T>::W>
__device__ __forceinline__ void load_row_shfl(const T* __restrict__ p, T (&e)[W + 2], bool active,
                                              unsigned act, int lane) {
  T mid[W];
  if (active) VecN<T, W>::load_keep(p, mid);
  else {
#pragma unroll
    for (int w = 0; w < W; ++w) mid[w] = 0;
  }
  T left = __shfl_up_sync(0xffffffffu, mid[W - 1], 1);
  T right = __shfl_down_sync(0xffffffffu, mid[0], 1);
  const bool lnb = lane > 0 && ((act >> (lane - 1)) & 1u);
  const bool rnb = lane < 31 && ((act >> (lane + 1)) & 1u);
  if (active && !lnb) left = p[-1];
  if (active && !rnb) right = p[W];
  e[0] = left;
#pragma unroll
  for (int w = 0; w < W; ++w) e[w + 1] = mid[w];
  e[W + 1] = right;
}

// Row offsets of the 3^DIM stencil around the group start, row k = dy + 3 dz.
template <int DIM>
__device__ __forceinline__ long long row_offset(int k, long long px, long long pxy) {
  const int dy = k % 3 - 1, dz = DIM == 3 ? k / 3 - 1 : 0;
  return dy * px + dz * pxy;
}

// o[w] = p[w - 1] and o[w] = p[w + 1] for the W values of a group: one
// aligned vector load (evict-first) and one scalar.
template <typename T, int W>
__device__ __forceinline__ void load_left(const T* __restrict__ p, T (&o)[W]) {
  if constexpr (W > 1) {
    T v[W];
    VecN<T, W>::load(p, v);
#pragma unroll
    for (int w = 1; w < W; ++w) o[w] = v[w - 1];
  }
  o[0] = p[-1];
}
template <typename T, int W>
__device__ __forceinline__ void load_right(const T* __restrict__ p, T (&o)[W]) {
  if constexpr (W > 1) {
    T v[W];
    VecN<T, W>::load(p, v);
#pragma unroll
    for (int w = 0; w + 1 < W; ++w) o[w] = v[w + 1];
  }
  o[W - 1] = p[W];
}

// The three couplings a_j = A(i, i + (j - 1) + ro) of stencil row k (row
// offset ro) for the W points i of the group at idx.
//   SYM = false: the full stencil, plane 3k + j at the point itself.
//   SYM = true: the symmetric half (launch_sym_half: plane p holds tap
//   3^dim / 2 + p, the diagonal and the couplings to the later neighbours).
//   A coupling to an earlier neighbour is read transposed, A(i, i - s) =
//   A(i - s, i), from the mirrored tap's plane at the neighbour: rows before
//   the centre row read the mirrored row's three planes at i + ro shifted by
//   -1, 0, +1; the centre row reads its x-1 coupling from the x+1 plane at
//   i - 1.  The later rows' planes are loaded with the default caching, since
//   the groups behind read them again transposed.
template <typename T, int DIM, int W, bool SYM>
__device__ __forceinline__ void row_coeffs(const T* __restrict__ st, long long pitch, long long idx, long long ro,
                                           int k, T (&a0)[W], T (&a1)[W], T (&a2)[W]) {
  if constexpr (!SYM) {
    VecN<T, W>::load(st + (long long)(3 * k + 0) * pitch + idx, a0);
    VecN<T, W>::load(st + (long long)(3 * k + 1) * pitch + idx, a1);
    VecN<T, W>::load(st + (long long)(3 * k + 2) * pitch + idx, a2);
  } else {
    constexpr int R = DIM == 3 ? 9 : 3, kc = R / 2, tc = 3 * kc + 1;
    if (k > kc) {
      VecN<T, W>::load_keep(st + (long long)(3 * k + 0 - tc) * pitch + idx, a0);
      VecN<T, W>::load_keep(st + (long long)(3 * k + 1 - tc) * pitch + idx, a1);
      VecN<T, W>::load_keep(st + (long long)(3 * k + 2 - tc) * pitch + idx, a2);
    } else if (k == kc) {
      VecN<T, W>::load(st + idx, a1);
      VecN<T, W>::load_keep(st + pitch + idx, a2);
#pragma unroll
      for (int w = 1; w < W; ++w) a0[w] = a2[w - 1];
      a0[0] = st[pitch + idx - 1];
    } else {
      const int km = R - 1 - k;
      load_left<T, W>(st + (long long)(3 * km + 2 - tc) * pitch + idx + ro, a0);
      VecN<T, W>::load(st + (long long)(3 * km + 1 - tc) * pitch + idx + ro, a1);
      load_right<T, W>(st + (long long)(3 * km + 0 - tc) * pitch + idx + ro, a2);
    }
  }
}

// acc[c][w] += sum over the stencil of A(point w) * X_c(neighbour), C columns;
// pitch = distance between stencil planes and between columns; SYM as
// row_coeffs.
template <typename T, int DIM, int C, bool SYM = false>
__device__ __forceinline__ void stencil_group(const T* __restrict__ st, long long pitch, const T* __restrict__ X,
                                              long long idx, long long px, long long pxy,
                                              T (&acc)[C][Vec<T>::W]) {
  constexpr int W = Vec<T>::W;
  constexpr int R = DIM == 3 ? 9 : 3;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const long long ro = row_offset<DIM>(k, px, pxy);
    T a0[W], a1[W], a2[W];
    row_coeffs<T, DIM, W, SYM>(st, pitch, idx, ro, k, a0, a1, a2);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      T e[W + 2];
      load_row<T>(X + (long long)c * pitch + idx + ro, e);
#pragma unroll
      for (int w = 0; w < W; ++w) {
        acc[c][w] = fma(a0[w], e[w], acc[c][w]);
        acc[c][w] = fma(a1[w], e[w + 1], acc[c][w]);
        acc[c][w] = fma(a2[w], e[w + 2], acc[c][w]);
      }
    }
  }
}

// The FP32 3D instances with up to 6 columns run three blocks per SM (at most
// 85 registers) in one wave of resident blocks (spmm_blocks): measured faster
// than two blocks per SM over two waves, whose loads wait longer.
template <typename T, int DIM, int C, bool ZAZ, bool SYM = false>
__global__ void __launch_bounds__(kBlock, (sizeof(T) == 4 && DIM == 3 && C <= 6) ? 3 : (kIsDw<T> ? 2 : 1)) k_spmm(GridDesc g, const T* __restrict__ st, const T* __restrict__ X,
                                                 T* __restrict__ Y, double* zaz, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  constexpr int W = Vec<T>::W;
  const long long bo = (long long)pb * g.len;
  T zacc[ZAZ ? C : 1];
#pragma unroll
  for (int c = 0; c < (ZAZ ? C : 1); ++c) zacc[c] = 0;
  const long long ngroups = g.npts / W;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    const long long idx = bo + g.G + q * W;
    T acc[C][W];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int w = 0; w < W; ++w) acc[c][w] = 0;
    stencil_group<T, DIM, C, SYM>(st, g.cp, X, idx, g.px, g.pxy, acc);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      Vec<T>::store(Y + (long long)c * g.cp + idx, acc[c]);
      if (ZAZ) {
        T xc[W];
        Vec<T>::load_keep(X + (long long)c * g.cp + idx, xc);
#pragma unroll
        for (int w = 0; w < W; ++w) zacc[c] = fma(xc[w], acc[c][w], zacc[c]);
      }
    }
  }
  if (ZAZ) block_sum_store<T, ZAZ ? C : 1>(zacc, zaz + (long long)pb * C * gridDim.x, gridDim.x, blockIdx.x);
}

// r = b - A x with the partials of |r|^2 and |b|^2.  xnz (may be null) flags
// per problem whether x can be nonzero; for a zero iterate A x = 0 exactly
// and the stencil is not read (r = b, the same values bit for bit).
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_residual(GridDesc g, const T* __restrict__ st, const T* __restrict__ b,
                                                     const T* __restrict__ xv, T* __restrict__ r, double* part,
                                                     const int* __restrict__ xnz) {
  constexpr int W = Vec<T>::W;
  const int pb = blockIdx.y;
  const bool zero_x = xnz && xnz[pb] == 0;
  const long long bo = (long long)pb * g.len;
  T sums[2] = {0, 0};
  const long long ngroups = g.npts / W;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    const long long idx = bo + g.G + q * W;
    T acc[1][W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[0][w] = 0;
    if (!zero_x) stencil_group<T, DIM, 1>(st, g.cp, xv, idx, g.px, g.pxy, acc);
    T bv[W], rv[W];
    Vec<T>::load(b + idx, bv);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      rv[w] = bv[w] - acc[0][w];
      sums[0] = fma(rv[w], rv[w], sums[0]);
      sums[1] = fma(bv[w], bv[w], sums[1]);
    }
    Vec<T>::store(r + idx, rv);
  }
  block_sum_store<T, 2>(sums, part + (long long)pb * 2 * gridDim.x, gridDim.x, blockIdx.x);
}

// Restriction R = P^T: coarse node I sits on fine node 2I + lo (per axis,
// lo = 1 when the low face is Dirichlet); the fine nodes at distance one
// carry weight 1/2 per differing axis.  Vector unknowns restrict
// componentwise.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_restrict(GridDesc gf, GridDesc gc, const T* __restrict__ rf,
                                                     T* __restrict__ rc, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= gc.npts) return;
  rf += (long long)pb * gf.len;
  rc += (long long)pb * gc.len;
  int X, Y, Z, a;
  decode(gc, t, X, Y, Z, a);
  const long long idc = gc.G + t;
  if (!interior(gc, X, Y, Z)) {
    rc[idc] = (T)0;
    return;
  }
  const long long pf = gf.px, pp = gf.pxy;
  const long long idf = gf.G + a * gf.cstride + (2 * X + gf.lox) + pf * (2 * Y + gf.loy) +
                        (DIM == 3 ? pp * (2 * Z + gf.loz) : 0);
  T acc = 0;
#pragma unroll
  for (int ez = (DIM == 3 ? -1 : 0); ez <= (DIM == 3 ? 1 : 0); ++ez) {
#pragma unroll
    for (int ey = -1; ey <= 1; ++ey) {
#pragma unroll
      for (int ex = -1; ex <= 1; ++ex) {
        const T w = (T)((ex ? 0.5f : 1.f) * (ey ? 0.5f : 1.f) * (ez ? 0.5f : 1.f));
        acc = fma(w, rf[idf + ex + pf * ey + pp * ez], acc);
      }
    }
  }
  rc[idc] = acc;
}

// Damped Jacobi (Eq. 2 with M = D / omega, dinv = omega / diag), c_0 = 0:
//   mode 0: out = dinv r                          (one sweep)
//   mode 1: out = s1 + dinv (r - A s1), s1 = dinv r  (two sweeps, s1 formed
//           at the neighbours on the fly)
//   mode 2: out = sin + dinv (r - A sin)           (a further sweep)
//   W points per thread: Vec<T>::W (one vector load), or 1 on the small
//   grids (modes 0 and 1; mode 2 keeps Vec<T>::W).  Every point's
//   arithmetic is the same whatever W.  SYM: st is the symmetric half
//   (row_coeffs).
template <typename T, int DIM, int W = Vec<T>::W, bool SYM = false>
__global__ void __launch_bounds__(kBlock, 4) k_jacobi(GridDesc g, const T* __restrict__ st, const T* __restrict__ dinv,
                                                   const T* __restrict__ r, const T* __restrict__ sin,
                                                   T* __restrict__ out, int mode, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const long long ngroups = g.npts / W;
  const long long q0 = blockIdx.x * (long long)blockDim.x + (threadIdx.x & ~31);
  if (q0 >= ngroups) return;   // the whole warp is idle
  const int lane = threadIdx.x & 31;
  const long long q = q0 + lane;
  const bool active = q < ngroups;
  const long long idx = (long long)pb * g.len + g.G + q * W;
  T di[W] = {}, ri[W] = {}, o[W];
  if (active) {
    VecN<T, W>::load_keep(dinv + idx, di);
    VecN<T, W>::load_keep(r + idx, ri);
  }
  if (mode == 0) {
    if (!active) return;
#pragma unroll
    for (int w = 0; w < W; ++w) o[w] = di[w] * ri[w];
    VecN<T, W>::store(out + idx, o);
    return;
  }
  T acc[1][W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[0][w] = 0;
  if (mode == 1) {
    const unsigned act = __ballot_sync(0xffffffffu, active);
    constexpr int R = DIM == 3 ? 9 : 3;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const long long ro = row_offset<DIM>(k, g.px, g.pxy);
      T a0[W] = {}, a1[W] = {}, a2[W] = {}, ed[W + 2], er[W + 2];
      if (active) row_coeffs<T, DIM, W, SYM>(st, g.cp, idx, ro, k, a0, a1, a2);
      load_row_shfl<T, W>(dinv + idx + ro, ed, active, act, lane);
      load_row_shfl<T, W>(r + idx + ro, er, active, act, lane);
#pragma unroll
      for (int w = 0; w < W; ++w) {
        acc[0][w] = fma(a0[w], ed[w] * er[w], acc[0][w]);
        acc[0][w] = fma(a1[w], ed[w + 1] * er[w + 1], acc[0][w]);
        acc[0][w] = fma(a2[w], ed[w + 2] * er[w + 2], acc[0][w]);
      }
    }
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const T s1 = di[w] * ri[w];
      o[w] = s1 + di[w] * (ri[w] - acc[0][w]);
    }
  } else if constexpr (W == Vec<T>::W) {   // mode 2 (the launcher uses the full width for it)
    if (!active) return;
    stencil_group<T, DIM, 1, SYM>(st, g.cp, sin, idx, g.px, g.pxy, acc);
    T sv[W];
    Vec<T>::load_keep(sin + idx, sv);
#pragma unroll
    for (int w = 0; w < W; ++w) o[w] = sv[w] + di[w] * (ri[w] - acc[0][w]);
  } else {
    return;
  }
  if (active) VecN<T, W>::store(out + idx, o);
}

// Multicoloured SSOR (Section 3's smoother; the colouring is a reading):
// one Gauss-Seidel update of every unknown of colour `colour` (parity of the
// global node coordinates, bit a for axis a), in place:
// x_i += omega (b_i - sum_s a_is x_(i+s)) / a_ii.  No two unknowns of a
// colour are coupled by the stencil, so the colour updates at once.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_gs_colour(GridDesc g, const T* __restrict__ st, const T* __restrict__ b,
                                                      T* __restrict__ x, int colour, T omega, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.npts) return;
  int px_, py_, pz_, a;
  decode(g, t, px_, py_, pz_, a);
  if (!interior(g, px_, py_, pz_)) return;
  const int c = ((px_ + g.lox) & 1) | (((py_ + g.loy) & 1) << 1) | (DIM == 3 ? (((pz_ + g.loz) & 1) << 2) : 0);
  if (c != colour) return;
  constexpr int S = DIM == 3 ? 27 : 9;
  const long long i = (long long)pb * g.len + g.G + t;
  T acc = 0;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = DIM == 3 ? s / 9 - 1 : 0;
    acc = fma(st[(long long)s * g.cp + i], x[i + dx + (long long)dy * g.px + (long long)dz * g.pxy], acc);
  }
  const T diag = st[(long long)(S / 2) * g.cp + i];
  x[i] += omega * (b[i] - acc) / diag;
}

// d = b - A x over the padded box (zero rows at pads), no norms.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_defect(GridDesc g, const T* __restrict__ st, const T* __restrict__ b,
                                                   const T* __restrict__ x, T* __restrict__ d, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  constexpr int W = Vec<T>::W;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= g.npts / W) return;
  const long long idx = (long long)pb * g.len + g.G + q * W;
  T acc[1][W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[0][w] = 0;
  stencil_group<T, DIM, 1>(st, g.cp, x, idx, g.px, g.pxy, acc);
  T bv[W], o[W];
  Vec<T>::load_keep(b + idx, bv);
#pragma unroll
  for (int w = 0; w < W; ++w) o[w] = bv[w] - acc[0][w];
  Vec<T>::store(d + idx, o);
}

// fine += P coarse (two grids, Section 2.1's interpolation): fine global
// node g sits on coarse node g/2 (even g) or between (g-1)/2 and (g+1)/2.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_prolong_add(GridDesc gc, GridDesc gf, const T* __restrict__ coarse,
                                                        T* __restrict__ fine, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= gf.npts) return;
  int x, y, z, a;
  decode(gf, t, x, y, z, a);
  if (!interior(gf, x, y, z)) return;
  const int gx = x + gf.lox, gy = y + gf.loy, gz = DIM == 3 ? z + gf.loz : 0;
  const T* cb = coarse + (long long)pb * gc.len + gc.G + (long long)a * gc.cstride;
  T v = 0;
#pragma unroll
  for (int kz = 0; kz < (DIM == 3 ? 2 : 1); ++kz) {
    if (DIM == 3 && kz == 1 && !(gz & 1)) continue;
    const int cz = DIM == 3 ? (gz >> 1) + kz - gc.loz : 0;
#pragma unroll
    for (int ky = 0; ky < 2; ++ky) {
      if (ky == 1 && !(gy & 1)) continue;
      const int cy = (gy >> 1) + ky - gc.loy;
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        if (kx == 1 && !(gx & 1)) continue;
        const int cx = (gx >> 1) + kx - gc.lox;
        const T w = (T)((gx & 1) ? 0.5 : 1.0) * (T)((gy & 1) ? 0.5 : 1.0) * (T)((DIM == 3 && (gz & 1)) ? 0.5 : 1.0);
        v = fma(w, cb[cx + (long long)cy * gc.px + (DIM == 3 ? (long long)cz * gc.pxy : 0)], v);
      }
    }
  }
  fine[(long long)pb * gf.len + gf.G + t] += v;
}

// dst += src over the padded box.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_add_to(GridDesc g, const T* __restrict__ src, T* __restrict__ dst,
                                                   const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.npts) return;
  const long long i = (long long)pb * g.len + g.G + t;
  dst[i] += src[i];
}

// Composite prolongation P_J ... P_{j+1} of every coarse grid's correction
// straight to the fine grid (Section 2.1 allows the composite transfers to be
// formed explicitly): the nested Q1 spaces make it the multilinear
// interpolation of grid j's values at the fine nodes.  Along an axis with
// s = 2^(J-j), fine global node g lies between coarse global nodes g >> m
// and (g >> m) + 1 with weights 1 - f/s and f/s, f = g mod s (exact binary
// fractions); coarse parents outside the grid are pad entries (zero).  One
// launch writes columns 0 .. J-1 of Z (column J is the fine smoothing),
// equal to successive two-grid prolongation up to the summation order.  The
// grid count is a template parameter, so that every column's ratio s and
// weights fold to constants (the kernel is bound by instruction issue).
template <typename T>
struct CoarseSrc {
  const T* v[kMaxLevels];      // grid j's correction (padded, problem 0)
  GridDesc g[kMaxLevels];
};

template <typename T, int DIM, int JJ>
__global__ void __launch_bounds__(kBlock) k_prolong_all(GridDesc gf, CoarseSrc<T> src, T* __restrict__ Z,
                                                        const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  constexpr int W = Vec<T>::W;
  constexpr int NR = 3;   // coarse x values a group of W <= 4 fine points needs at s >= 2
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= gf.npts / W) return;
  const long long t0 = q * W;
  int x0, y, z, a;
  decode(gf, t0, x0, y, z, a);
  const long long idf = (long long)pb * gf.len + gf.G + t0;
  if (y >= gf.ny || (DIM == 3 && z >= gf.nz)) {   // pad row
    T o[W];
#pragma unroll
    for (int w = 0; w < W; ++w) o[w] = 0;
#pragma unroll
    for (int j = 0; j < JJ; ++j) Vec<T>::store(Z + (long long)j * gf.cp + idf, o);
    return;
  }
  const int gy = y + gf.loy, gz = DIM == 3 ? z + gf.loz : 0, gx0 = x0 + gf.lox;
#pragma unroll
  for (int j = 0; j < JJ; ++j) {
    // grid j sits m = JJ - j levels below: s = 2^m fine intervals per coarse one
    const int m = JJ - j, s = 1 << m, sm1 = s - 1;
    const T inv_s = (T)(1.f / (float)s);   // exact: s is a power of two
    const GridDesc& gc = src.g[j];
    const int cy0 = (gy >> m) - gc.loy, cz0 = DIM == 3 ? (gz >> m) - gc.loz : 0;
    const T wy1 = (T)(gy & sm1) * inv_s, wz1 = DIM == 3 ? (T)(gz & sm1) * inv_s : (T)0;
    const int X0 = gx0 >> m;
    const T* base = src.v[j] + (long long)pb * gc.len + gc.G + (long long)a * gc.cstride + (X0 - gc.lox);
    T row[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) row[k] = 0;
#pragma unroll
    for (int kz = 0; kz < (DIM == 3 ? 2 : 1); ++kz) {
      const T wz = DIM == 3 ? (kz ? wz1 : (T)1 - wz1) : (T)1;
#pragma unroll
      for (int ky = 0; ky < 2; ++ky) {
        const T wgt = wz * (ky ? wy1 : (T)1 - wy1);
        const T* rp = base + gc.px * (long long)(cy0 + ky) + (DIM == 3 ? gc.pxy * (long long)(cz0 + kz) : 0);
#pragma unroll
        for (int k = 0; k < NR; ++k) row[k] = fma(wgt, rp[k], row[k]);
      }
    }
    // along x: fine node gx0 + w = X0 s + t sits in coarse interval k = t / s
    // at fraction (t mod s) / s; k = 2 only for s = 2, t = 4 (fraction 0)
    const T d0 = row[1] - row[0], d1 = row[2] - row[1];
    const int f0 = gx0 & sm1;
    T o[W];
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int t = f0 + w, k = t >> m;
      const T f = (T)(t & sm1) * inv_s;
      const T v = k == 0 ? fma(f, d0, row[0]) : (k == 1 ? fma(f, d1, row[1]) : row[2]);
      o[w] = x0 + w < gf.nx ? v : (T)0;
    }
    Vec<T>::store(Z + (long long)j * gf.cp + idf, o);
  }
}

// The small-grid tail of the MG chain in one block (scalar unknowns, two
// Jacobi sweeps): the restrictions from grid jt + 1 down to grid 0, the
// damped-Jacobi smoothing of grids 1 .. jt and the exact coarsest solve.
// Grids this small are latency-bound as separate launches; one block of
// 1024 threads takes them in turn with block barriers in between.
template <typename T>
struct TailArgs {
  int jt;                          // finest grid of the tail
  GridDesc g[kMaxLevels];
  const T* st[kMaxLevels];         // stencil planes of grid j
  const T* dinv[kMaxLevels];       // damped inverse diagonal of grid j
  T* r[kMaxLevels];                // restricted residual of grid j (j <= jt)
  T* z[kMaxLevels];                // correction of grid j (grid 0: the coarse solve)
  const T* rin;                    // residual of grid jt + 1
  const double* a0inv;             // explicit inverse of the coarsest operator
};

template <typename T, int DIM>
__global__ void __launch_bounds__(1024) k_coarse_tail(TailArgs<T> a, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  constexpr int S = DIM == 3 ? 27 : 9;
  // restrictions jt + 1 -> jt -> ... -> 0
  for (int j = a.jt; j >= 0; --j) {
    const GridDesc& gf = a.g[j + 1];
    const GridDesc& gc = a.g[j];
    const T* rf = (j == a.jt ? a.rin : a.r[j + 1]) + (long long)pb * gf.len;
    T* rc = a.r[j] + (long long)pb * gc.len;
    for (long long t = threadIdx.x; t < gc.npts; t += blockDim.x) {
      int X, Y, Z, c;
      decode(gc, t, X, Y, Z, c);
      T acc = 0;
      if (interior(gc, X, Y, Z)) {
        const long long pf = gf.px, pp = gf.pxy;
        const long long idf = gf.G + (2 * X + gf.lox) + pf * (2 * Y + gf.loy) + (DIM == 3 ? pp * (2 * Z + gf.loz) : 0);
        for (int ez = (DIM == 3 ? -1 : 0); ez <= (DIM == 3 ? 1 : 0); ++ez)
          for (int ey = -1; ey <= 1; ++ey)
            for (int ex = -1; ex <= 1; ++ex) {
              const T w = (T)((ex ? 0.5f : 1.f) * (ey ? 0.5f : 1.f) * (ez ? 0.5f : 1.f));
              acc = fma(w, rf[idf + ex + pf * ey + pp * ez], acc);
            }
      }
      rc[gc.G + t] = acc;
    }
    __syncthreads();
  }
  // two damped-Jacobi sweeps from zero on grids 1 .. jt (Eq. 2, c_0 = 0):
  // out = s1 + dinv (r - A s1) with s1 = dinv r formed at the neighbours
  for (int j = 1; j <= a.jt; ++j) {
    const GridDesc& g = a.g[j];
    const long long bo = (long long)pb * g.len + g.G;
    const T* st = a.st[j] + bo;
    const T* di = a.dinv[j] + bo;
    const T* rr = a.r[j] + bo;
    T* out = a.z[j] + bo;
    for (long long t = threadIdx.x; t < g.npts; t += blockDim.x) {
      T acc = 0;
      for (int s = 0; s < S; ++s) {
        const long long off = (s % 3 - 1) + g.px * ((s / 3) % 3 - 1) + (DIM == 3 ? g.pxy * (s / 9 - 1) : 0);
        acc = fma(st[(long long)s * g.cp + t], di[t + off] * rr[t + off], acc);
      }
      const T s1 = di[t] * rr[t];
      out[t] = s1 + di[t] * (rr[t] - acc);
    }
  }
  // exact coarsest solve: warp per row of the explicit inverse
  {
    extern __shared__ double yv[];
    const GridDesc& g = a.g[0];
    const int n = (int)g.n;
    const double* inv = a.a0inv + (long long)pb * n * n;
    const T* r0 = a.r[0] + (long long)pb * g.len;
    T* out = a.z[0] + (long long)pb * g.len;
    for (int i = threadIdx.x; i < n; i += blockDim.x) yv[i] = (double)r0[padded_index(g, i)];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x >> 5; i < n; i += blockDim.x >> 5) {
      const double* row = inv + (long long)i * n;
      double s = 0.0;
      for (int k = lane; k < n; k += 32) s = fma(row[k], yv[k], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) out[padded_index(g, i)] = (T)s;
    }
  }
}

// Galerkin product A_c = P^T A_f P, one coarse row per thread.  For vector
// unknowns P interpolates componentwise, so every component pair (a, b) is a
// scalar Galerkin product of its own plane group b * 3^DIM + s.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_galerkin(GridDesc gf, GridDesc gc, const double* __restrict__ stf,
                                                     double* __restrict__ stc) {
  constexpr int S = DIM == 3 ? 27 : 9;
  const int pb = blockIdx.y;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= gc.npts) return;
  stf += (long long)pb * gf.len;
  stc += (long long)pb * gc.len;
  int X, Y, Z, comp;
  decode(gc, t, X, Y, Z, comp);
  const long long idc = gc.G + t;
  if (!interior(gc, X, Y, Z)) {
    for (int s = 0; s < S * gc.ncomp; ++s) stc[s * gc.cp + idc] = 0.0;
    return;
  }
  const long long pf = gf.px, ppf = gf.pxy;
  for (int b = 0; b < gc.ncomp; ++b) {
    double acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0;
    const double* sfb = stf + (long long)b * S * gf.cp;
    for (int ez = (DIM == 3 ? -1 : 0); ez <= (DIM == 3 ? 1 : 0); ++ez)
      for (int ey = -1; ey <= 1; ++ey)
        for (int ex = -1; ex <= 1; ++ex) {
          const double we = (ex ? 0.5 : 1.0) * (ey ? 0.5 : 1.0) * (ez ? 0.5 : 1.0);
          const long long idf = gf.G + comp * gf.cstride + (2 * X + gf.lox + ex) + pf * (2 * Y + gf.loy + ey) +
                                (DIM == 3 ? ppf * (2 * Z + gf.loz + ez) : 0);
          for (int s = 0; s < S; ++s) {
            const double a = sfb[s * gf.cp + idf];
            if (a == 0.0) continue;
            // offset of the fine column node from the fine image of (X, Y, Z);
            // the image has even global index on every axis, so the column's
            // coarse parents are D = f/2 (f even) or (f -+ 1)/2 (f odd)
            const int f[3] = {ex + (s % 3 - 1), ey + ((s / 3) % 3 - 1), DIM == 3 ? ez + (s / 9 - 1) : 0};
            int D0[3], D1[3], np[3];
            double w[3];
            for (int k = 0; k < 3; ++k) {
              if (k == 2 && DIM == 2) { D0[k] = D1[k] = 0; np[k] = 1; w[k] = 1.0; continue; }
              if ((f[k] & 1) == 0) { D0[k] = D1[k] = f[k] / 2; np[k] = 1; w[k] = 1.0; }
              else { D0[k] = (f[k] - 1) / 2; D1[k] = (f[k] + 1) / 2; np[k] = 2; w[k] = 0.5; }
            }
            const double base = we * a * w[0] * w[1] * w[2];
            const int Cc[3] = {X, Y, Z};
            for (int iz = 0; iz < np[2]; ++iz)
              for (int iy = 0; iy < np[1]; ++iy)
                for (int ix = 0; ix < np[0]; ++ix) {
                  const int Dx = ix ? D1[0] : D0[0], Dy = iy ? D1[1] : D0[1], Dz = iz ? D1[2] : D0[2];
                  const int cx = Cc[0] + Dx, cy = Cc[1] + Dy, cz = Cc[2] + Dz;
                  if (cx < 0 || cx >= gc.nx || cy < 0 || cy >= gc.ny) continue;   // Dirichlet parent
                  if (DIM == 3 && (cz < 0 || cz >= gc.nz)) continue;
                  acc[(Dx + 1) + 3 * (Dy + 1) + (DIM == 3 ? 9 * (Dz + 1) : 0)] += base;
                }
          }
        }
    for (int s = 0; s < S; ++s) stc[(b * S + s) * gc.cp + idc] = acc[s];
  }
}

// Damped inverse diagonal omega D^{-1}.  Vector unknowns: D is the 3 x 3
// block of a node's unknowns (the centre planes of the three plane groups);
// dinv plane b at the row of component a holds omega (D^{-1})_{ab}.
template <typename T>
__global__ void k_dinv(GridDesc g, const double* __restrict__ st, T* __restrict__ dinv, double omega) {
  const int pb = blockIdx.y;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.npts) return;
  int x, y, z, comp;
  decode(g, t, x, y, z, comp);
  const long long idx = (long long)pb * g.len + g.G + t;
  const int S = g.dim == 3 ? 27 : 9;
  const int centre = g.dim == 3 ? 13 : 4;
  const bool in = interior(g, x, y, z);
  if (g.ncomp == 1) {
    dinv[idx] = in ? (T)(omega / st[centre * g.cp + idx]) : (T)0;
    return;
  }
  if (!in) {
    for (int b = 0; b < 3; ++b) dinv[b * g.cp + idx] = (T)0;
    return;
  }
  const long long node = idx - comp * g.cstride;
  double D[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) D[a][b] = st[(long long)(b * S + centre) * g.cp + node + a * g.cstride];
  // inverse by the adjugate: (D^{-1})_{ab} = cofactor_{ba} / det
  const double c00 = D[1][1] * D[2][2] - D[1][2] * D[2][1];
  const double c01 = D[1][2] * D[2][0] - D[1][0] * D[2][2];
  const double c02 = D[1][0] * D[2][1] - D[1][1] * D[2][0];
  const double det = D[0][0] * c00 + D[0][1] * c01 + D[0][2] * c02;
  double inv[3][3];
  inv[0][0] = c00;
  inv[1][0] = c01;
  inv[2][0] = c02;
  inv[0][1] = D[0][2] * D[2][1] - D[0][1] * D[2][2];
  inv[1][1] = D[0][0] * D[2][2] - D[0][2] * D[2][0];
  inv[2][1] = D[0][1] * D[2][0] - D[0][0] * D[2][1];
  inv[0][2] = D[0][1] * D[1][2] - D[0][2] * D[1][1];
  inv[1][2] = D[0][2] * D[1][0] - D[0][0] * D[1][2];
  inv[2][2] = D[0][0] * D[1][1] - D[0][1] * D[1][0];
  for (int b = 0; b < 3; ++b) dinv[b * g.cp + idx] = (T)(omega * inv[comp][b] / det);
}

__global__ void k_convert_f32(const double* __restrict__ src, float* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// The symmetric half of a scalar FP64 stencil in FP32 (A is symmetric, so
// A(i, i - s) = A(i - s, i) need not be stored twice): plane p = 0 .. S/2
// (S = 3^dim taps) holds tap S/2 + p, the diagonal and the couplings to the
// later neighbours (offset dx + dy px + dz pxy > 0).  A coupling whose row or
// column is not an unknown (pad or guard entry, zero diagonal) is stored as
// zero, so that the transposed reads leave the rows of pads at zero.  Every
// entry of the cp-element planes (all problems, guards included) is written.
template <int DIM>
__global__ void k_sym_half(GridDesc g, const double* __restrict__ st, float* __restrict__ out) {
  constexpr int S = DIM == 3 ? 27 : 9, tc = S / 2;
  const double* diag = st + (long long)tc * g.cp;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < g.cp;
       e += (long long)gridDim.x * blockDim.x) {
    const bool row = diag[e] != 0.0;
#pragma unroll
    for (int p = 0; p <= tc; ++p) {
      const int t = tc + p;
      const long long off = (t % 3 - 1) + (long long)(t / 3 % 3 - 1) * g.px + (DIM == 3 ? (t / 9 - 1) * g.pxy : 0);
      const long long nb = e + off;
      const bool col = nb < g.cp && diag[nb] != 0.0;
      out[(long long)p * g.cp + e] = row && col ? (float)st[(long long)t * g.cp + e] : 0.0f;
    }
  }
}

// ---------------------------------------------------------------------------
// Vector unknowns (3D elasticity, three components per node).  Plane
// b * 27 + s at the row of component a holds the coupling of unknown
// (node, a) to (node + offset_s, b); component b of a node sits cstride
// after component 0, so the 81 couplings of a row are 27 neighbours in each
// of three component boxes.

// Block SpMM of a vector operator: one thread per (output component a, group
// of W x-points), so that only the C columns' accumulators are live (all
// three components per thread would cap occupancy at one block per SM for
// C = 5).  Consecutive threads take consecutive groups of the same component.
template <typename T, int C, bool ZAZ>
__global__ void __launch_bounds__(kBlock) k_vspmm(GridDesc g, const T* __restrict__ st, const T* __restrict__ X,
                                                  T* __restrict__ Y, double* zaz, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  constexpr int W = Vec<T>::W;
  const long long bo = (long long)pb * g.len;
  const long long cs = g.cstride;
  T zacc[ZAZ ? C : 1];
#pragma unroll
  for (int c = 0; c < (ZAZ ? C : 1); ++c) zacc[c] = 0;
  const long long ngroups = cs / W;
  for (long long item = blockIdx.x * (long long)blockDim.x + threadIdx.x; item < 3 * ngroups;
       item += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(item / ngroups);
    const long long idx0 = bo + g.G + (item - a * ngroups) * W;
    T acc[C][W];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int w = 0; w < W; ++w) acc[c][w] = 0;
#pragma unroll 1
    for (int k = 0; k < 9; ++k) {
      const long long ro = row_offset<3>(k, g.px, g.pxy);
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const T* sp = st + (long long)(b * 27 + 3 * k) * g.cp + idx0 + a * cs;
        T a0[W], a1[W], a2[W];
        Vec<T>::load(sp, a0);
        Vec<T>::load(sp + g.cp, a1);
        Vec<T>::load(sp + 2 * g.cp, a2);
#pragma unroll
        for (int c = 0; c < C; ++c) {
          T e[W + 2];
          load_row<T>(X + (long long)c * g.cp + idx0 + b * cs + ro, e);
#pragma unroll
          for (int w = 0; w < W; ++w) {
            acc[c][w] = fma(a0[w], e[w], acc[c][w]);
            acc[c][w] = fma(a1[w], e[w + 1], acc[c][w]);
            acc[c][w] = fma(a2[w], e[w + 2], acc[c][w]);
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const long long o = (long long)c * g.cp + idx0 + a * cs;
      Vec<T>::store(Y + o, acc[c]);
      if (ZAZ) {
        T xc[W];
        Vec<T>::load_keep(X + o, xc);
#pragma unroll
        for (int w = 0; w < W; ++w) zacc[c] = fma(xc[w], acc[c][w], zacc[c]);
      }
    }
  }
  if (ZAZ) block_sum_store<T, ZAZ ? C : 1>(zacc, zaz + (long long)pb * C * gridDim.x, gridDim.x, blockIdx.x);
}

// r = b - A x for a vector operator, one thread per (component, group), the
// whole 81-coefficient row unrolled so that a thread's loads are in flight
// together (the coarse grids of the hierarchy are latency-bound).  NORMS:
// per-block partial sums of |r|^2 and |b|^2 (grid-stride, for the residual
// of the refinement); otherwise one group per thread (the smoother).
template <typename T, bool NORMS>
__global__ void __launch_bounds__(kBlock, 3) k_vres(GridDesc g, const T* __restrict__ st, const T* __restrict__ b,
                                                    const T* __restrict__ xv, T* __restrict__ r, double* part,
                                                    const DevState* state, const int* __restrict__ xnz) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const bool zero_x = xnz && xnz[pb] == 0;   // zero iterate: r = b
  constexpr int W = Vec<T>::W;
  const long long bo = (long long)pb * g.len;
  const long long cs = g.cstride;
  const long long ngroups = cs / W;
  T sums[2] = {0, 0};
  for (long long item = blockIdx.x * (long long)blockDim.x + threadIdx.x; item < 3 * ngroups;
       item += NORMS ? (long long)gridDim.x * blockDim.x : 3 * ngroups) {
    const int a = (int)(item / ngroups);
    const long long idx0 = bo + g.G + (item - a * ngroups) * W;
    T acc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[w] = 0;
    if (!zero_x) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const long long ro = row_offset<3>(k, g.px, g.pxy);
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          const T* sp = st + (long long)(bb * 27 + 3 * k) * g.cp + idx0 + a * cs;
          T a0[W], a1[W], a2[W], e[W + 2];
          Vec<T>::load(sp, a0);
          Vec<T>::load(sp + g.cp, a1);
          Vec<T>::load(sp + 2 * g.cp, a2);
          load_row<T>(xv + idx0 + bb * cs + ro, e);
#pragma unroll
          for (int w = 0; w < W; ++w) {
            acc[w] = fma(a0[w], e[w], acc[w]);
            acc[w] = fma(a1[w], e[w + 1], acc[w]);
            acc[w] = fma(a2[w], e[w + 2], acc[w]);
          }
        }
      }
    }
    T bv[W], rv[W];
    Vec<T>::load(b + idx0 + a * cs, bv);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      rv[w] = bv[w] - acc[w];
      if (NORMS) {
        sums[0] = fma(rv[w], rv[w], sums[0]);
        sums[1] = fma(bv[w], bv[w], sums[1]);
      }
    }
    Vec<T>::store(r + idx0 + a * cs, rv);
  }
  if (NORMS) block_sum_store<T, 2>(sums, part + (long long)pb * 2 * gridDim.x, gridDim.x, blockIdx.x);
}

// Block-Jacobi update (Eq. 2 with M = D / omega, D the 3 x 3 node blocks):
// out = (sin or 0) + dinv t, pointwise per node (in place is allowed).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_vblock(GridDesc g, const T* __restrict__ dinv, const T* t,
                                                   const T* sin, T* out, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  constexpr int W = Vec<T>::W;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= g.cstride / W) return;
  const long long idx0 = (long long)pb * g.len + g.G + q * W;
  const long long cs = g.cstride;
  T tv[3][W];
#pragma unroll
  for (int b = 0; b < 3; ++b) Vec<T>::load_keep(t + idx0 + b * cs, tv[b]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    T o[W];
    if (sin) Vec<T>::load_keep(sin + idx0 + a * cs, o);
    else {
#pragma unroll
      for (int w = 0; w < W; ++w) o[w] = 0;
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      T d[W];
      Vec<T>::load_keep(dinv + (long long)b * g.cp + idx0 + a * cs, d);
#pragma unroll
      for (int w = 0; w < W; ++w) o[w] = fma(d[w], tv[b][w], o[w]);
    }
    Vec<T>::store(out + idx0 + a * cs, o);
  }
}

// The last block-Jacobi sweep in one pass: t = b - A x for the three
// components of a node group (the arithmetic of k_vres), then
// out = x + dinv t (that of k_vblock); out must not alias x (x is read at
// the neighbours).  Bitwise the results of k_vres followed by k_vblock.
template <typename T>
__global__ void __launch_bounds__(kBlock, 3) k_vres_block(GridDesc g, const T* __restrict__ st,
                                                          const T* __restrict__ b, const T* __restrict__ xv,
                                                          const T* __restrict__ dinv, T* __restrict__ out,
                                                          const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  constexpr int W = Vec<T>::W;
  const long long bo = (long long)pb * g.len;
  const long long cs = g.cstride;
  const long long ngroups = cs / W;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    const long long idx0 = bo + g.G + q * W;
    T tv[3][W];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T acc[W];
#pragma unroll
      for (int w = 0; w < W; ++w) acc[w] = 0;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const long long ro = row_offset<3>(k, g.px, g.pxy);
#pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          const T* sp = st + (long long)(bb * 27 + 3 * k) * g.cp + idx0 + a * cs;
          T a0[W], a1[W], a2[W], e[W + 2];
          Vec<T>::load(sp, a0);
          Vec<T>::load(sp + g.cp, a1);
          Vec<T>::load(sp + 2 * g.cp, a2);
          load_row<T>(xv + idx0 + bb * cs + ro, e);
#pragma unroll
          for (int w = 0; w < W; ++w) {
            acc[w] = fma(a0[w], e[w], acc[w]);
            acc[w] = fma(a1[w], e[w + 1], acc[w]);
            acc[w] = fma(a2[w], e[w + 2], acc[w]);
          }
        }
      }
      T bv[W];
      Vec<T>::load(b + idx0 + a * cs, bv);
#pragma unroll
      for (int w = 0; w < W; ++w) tv[a][w] = bv[w] - acc[w];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T o[W];
      Vec<T>::load_keep(xv + idx0 + a * cs, o);
#pragma unroll
      for (int bb = 0; bb < 3; ++bb) {
        T d[W];
        Vec<T>::load_keep(dinv + (long long)bb * g.cp + idx0 + a * cs, d);
#pragma unroll
        for (int w = 0; w < W; ++w) o[w] = fma(d[w], tv[bb][w], o[w]);
      }
      Vec<T>::store(out + idx0 + a * cs, o);
    }
  }
}

inline int blocks_for(long long n) { return (int)((n + kBlock - 1) / kBlock); }

template <typename T>
constexpr int vw() { return 16 / (int)sizeof(T); }

}  // namespace

// ---------------------------------------------------------------------------
template <typename TI, typename TO>
void launch_pack(const GridDesc& g, const TI* src, long long ld, TO* dst, int ncols, cudaStream_t s) {
  k_pack<TI, TO><<<grid_for(g.n * ncols, 4096), kBlock, 0, s>>>(g, src, ld, dst, ncols);
}
template <typename TO>
void launch_pack_flag(const GridDesc& g, const double* src, TO* dst, int* nz, cudaStream_t s) {
  k_pack_flag<TO><<<grid_for(g.n, 4096), kBlock, 0, s>>>(g, src, dst, nz);
}

#if MPCG_STENCIL_PLAIN
int g_sm_count = 0;
void set_sm_count(int n) { g_sm_count = n; }
int sm_count() { return g_sm_count; }
#else
extern int g_sm_count;
#endif

template <typename T>
int spmm_blocks(const GridDesc& g, int C) {
  const int nb = stream_blocks(g);
  int dflt = nb;
  if (sizeof(T) == 4 && g.dim == 3 && g.ncomp == 1 && C <= 6 && g_sm_count > 0) {
    const long long groups = g.npts / 2;
    const long long need = (groups + kBlock * 16 - 1) / (kBlock * 16);
    long long w = 3LL * g_sm_count;   // one wave at three blocks per SM
    if (w < need) w = need;
    dflt = (int)(w < nb ? w : nb);
  }
  // tuned: between the 64-points-per-thread minimum and the partial-sum
  // slots the solver reserves (stream_blocks_cap)
  const int v = tune::lookup(tune::kSpmm, kind_of<T>(), g.npts, g.nb, C, dflt);
  const int lo = stream_blocks_min(g), hi = stream_blocks_cap(g);
  return v < lo ? lo : (v > hi ? hi : v);
}
#if MPCG_STENCIL_PLAIN
template int spmm_blocks<double>(const GridDesc&, int);
template int spmm_blocks<float>(const GridDesc&, int);
#endif

template <typename TI, typename TO>
void launch_unpack(const GridDesc& g, const TI* src, TO* dst, long long ld, int ncols, cudaStream_t s) {
  k_unpack<TI, TO><<<grid_for(g.n * ncols, 4096), kBlock, 0, s>>>(g, src, dst, ld, ncols);
}
#if MPCG_STENCIL_PLAIN
template void launch_pack<double, double>(const GridDesc&, const double*, long long, double*, int, cudaStream_t);
template void launch_pack<double, float>(const GridDesc&, const double*, long long, float*, int, cudaStream_t);
template void launch_unpack<double, double>(const GridDesc&, const double*, double*, long long, int, cudaStream_t);
template void launch_unpack<float, double>(const GridDesc&, const float*, double*, long long, int, cudaStream_t);
template void launch_pack<float, float>(const GridDesc&, const float*, long long, float*, int, cudaStream_t);
template void launch_unpack<float, float>(const GridDesc&, const float*, float*, long long, int, cudaStream_t);
#endif

template <typename T, int DIM, bool SYM = false>
static void spmm_dim(const GridDesc& g, const T* st, const T* X, T* Y, int C, double* zaz, const DevState* state,
                     cudaStream_t s) {
  const dim3 grid(spmm_blocks<T>(g, C), g.nb);
#define MPCG_SPMM_CASE(CC)                                                                      \
  case CC:                                                                                      \
    if (zaz) k_spmm<T, DIM, CC, true, SYM><<<grid, kBlock, 0, s>>>(g, st, X, Y, zaz, state);    \
    else k_spmm<T, DIM, CC, false, SYM><<<grid, kBlock, 0, s>>>(g, st, X, Y, zaz, state);      \
    break;
  switch (C) {
    MPCG_SPMM_CASE(1) MPCG_SPMM_CASE(2) MPCG_SPMM_CASE(3) MPCG_SPMM_CASE(4) MPCG_SPMM_CASE(5)
    MPCG_SPMM_CASE(6) MPCG_SPMM_CASE(7) MPCG_SPMM_CASE(8) MPCG_SPMM_CASE(9) MPCG_SPMM_CASE(10)
    MPCG_SPMM_CASE(11) MPCG_SPMM_CASE(12)
    default: break;
  }
#undef MPCG_SPMM_CASE
}

template <typename T>
static void vspmm(const GridDesc& g, const T* st, const T* X, T* Y, int C, double* zaz, const DevState* state,
                  cudaStream_t s) {
  const dim3 grid(stream_blocks(g), g.nb);
#define MPCG_VSPMM_CASE(CC)                                                                     \
  case CC:                                                                                      \
    if (zaz) k_vspmm<T, CC, true><<<grid, kBlock, 0, s>>>(g, st, X, Y, zaz, state);             \
    else k_vspmm<T, CC, false><<<grid, kBlock, 0, s>>>(g, st, X, Y, zaz, state);               \
    break;
  switch (C) {
    MPCG_VSPMM_CASE(1) MPCG_VSPMM_CASE(2) MPCG_VSPMM_CASE(3) MPCG_VSPMM_CASE(4) MPCG_VSPMM_CASE(5)
    MPCG_VSPMM_CASE(6) MPCG_VSPMM_CASE(7) MPCG_VSPMM_CASE(8)
    default: break;
  }
#undef MPCG_VSPMM_CASE
}

template <typename T>
void launch_spmm(const GridDesc& g, const T* st, const T* X, T* Y, int C, double* zaz, const DevState* state,
                 cudaStream_t s) {
  if (g.ncomp == 3) vspmm<T>(g, st, X, Y, C, zaz, state, s);
  else if (g.dim == 3) spmm_dim<T, 3>(g, st, X, Y, C, zaz, state, s);
  else spmm_dim<T, 2>(g, st, X, Y, C, zaz, state, s);
}
#if MPCG_STENCIL_PLAIN
template void launch_spmm<double>(const GridDesc&, const double*, const double*, double*, int, double*,
                                  const DevState*, cudaStream_t);
template void launch_spmm<float>(const GridDesc&, const float*, const float*, float*, int, double*,
                                 const DevState*, cudaStream_t);
#endif

template <typename T>
void launch_residual(const GridDesc& g, const T* st, const T* b, const T* x, T* r, double* part, cudaStream_t s,
                     const int* xnz) {
  const dim3 grid(stream_blocks(g), g.nb);
  if (g.ncomp == 3) k_vres<T, true><<<grid, kBlock, 0, s>>>(g, st, b, x, r, part, nullptr, xnz);
  else if (g.dim == 3) k_residual<T, 3><<<grid, kBlock, 0, s>>>(g, st, b, x, r, part, xnz);
  else k_residual<T, 2><<<grid, kBlock, 0, s>>>(g, st, b, x, r, part, xnz);
}
#if MPCG_STENCIL_PLAIN
template void launch_residual<double>(const GridDesc&, const double*, const double*, const double*, double*,
                                      double*, cudaStream_t, const int*);
template void launch_residual<float>(const GridDesc&, const float*, const float*, const float*, float*, double*,
                                     cudaStream_t, const int*);
#endif

template <typename T>
void launch_restrict(const GridDesc& gf, const GridDesc& gc, const T* rf, T* rc, const DevState* state,
                     cudaStream_t s) {
  const dim3 grid(blocks_for(gc.npts), gc.nb);
  if (gc.dim == 3) k_restrict<T, 3><<<grid, kBlock, 0, s>>>(gf, gc, rf, rc, state);
  else k_restrict<T, 2><<<grid, kBlock, 0, s>>>(gf, gc, rf, rc, state);
}
#if MPCG_STENCIL_PLAIN
template void launch_restrict<double>(const GridDesc&, const GridDesc&, const double*, double*, const DevState*,
                                      cudaStream_t);
template void launch_restrict<float>(const GridDesc&, const GridDesc&, const float*, float*, const DevState*,
                                     cudaStream_t);
#endif

template <typename T, bool SYM = false>
static void jacobi_impl(const GridDesc& g, const T* st, const T* dinv, const T* r, const T* sin, T* out, int mode,
                        const DevState* state, cudaStream_t s) {
  // one point per thread where Vec<T>::W points per thread would leave fewer
  // than 4 warps per SM (the small coarse grids, latency-bound): more warps
  // in flight, same sums (measured: 33^3 and 17^3 launches 11.9 -> 7.2 us,
  // the 129^3 solve 4.575 -> 4.557 ms).  Larger grids keep the vector width:
  // their smoothing runs beside the fine grid's, and four times the blocks
  // there slowed the solve.
  const bool narrow_rule = g_sm_count > 0 && g.npts / vw<T>() * g.nb < (long long)g_sm_count * 128;
  const bool narrow = mode != 2 && tune::lookup(tune::kJacobi, kind_of<T>(), g.npts, g.nb, 0, narrow_rule ? 1 : 0) != 0;
  if (narrow) {
    const dim3 grid(blocks_for(g.npts), g.nb);
    if (g.dim == 3) k_jacobi<T, 3, 1, SYM><<<grid, kBlock, 0, s>>>(g, st, dinv, r, sin, out, mode, state);
    else k_jacobi<T, 2, 1, SYM><<<grid, kBlock, 0, s>>>(g, st, dinv, r, sin, out, mode, state);
    return;
  }
  const dim3 grid(blocks_for(g.npts / vw<T>()), g.nb);
  if (g.dim == 3) k_jacobi<T, 3, Vec<T>::W, SYM><<<grid, kBlock, 0, s>>>(g, st, dinv, r, sin, out, mode, state);
  else k_jacobi<T, 2, Vec<T>::W, SYM><<<grid, kBlock, 0, s>>>(g, st, dinv, r, sin, out, mode, state);
}

template <typename T>
void launch_jacobi(const GridDesc& g, const T* st, const T* dinv, const T* r, const T* sin, T* out, int mode,
                   const DevState* state, cudaStream_t s) {
  if (g.ncomp != 1) return;   // vector grids smooth with launch_vres / launch_vblock
  jacobi_impl<T>(g, st, dinv, r, sin, out, mode, state, s);
}
template <typename T>
void launch_vres(const GridDesc& g, const T* st, const T* r, const T* x, T* t, const DevState* state,
                 cudaStream_t s) {
  k_vres<T, false><<<dim3(blocks_for(3 * (g.cstride / vw<T>())), g.nb), kBlock, 0, s>>>(g, st, r, x, t, nullptr,
                                                                                        state, nullptr);
}
#if MPCG_STENCIL_PLAIN
template void launch_vres<double>(const GridDesc&, const double*, const double*, const double*, double*,
                                  const DevState*, cudaStream_t);
template void launch_vres<float>(const GridDesc&, const float*, const float*, const float*, float*,
                                 const DevState*, cudaStream_t);
#endif

template <typename T>
void launch_vres_block(const GridDesc& g, const T* st, const T* r, const T* x, const T* dinv, T* out,
                       const DevState* state, cudaStream_t s) {
  k_vres_block<T><<<dim3(blocks_for(g.cstride / vw<T>()), g.nb), kBlock, 0, s>>>(g, st, r, x, dinv, out, state);
}
#if MPCG_STENCIL_PLAIN
template void launch_vres_block<double>(const GridDesc&, const double*, const double*, const double*,
                                        const double*, double*, const DevState*, cudaStream_t);
template void launch_vres_block<float>(const GridDesc&, const float*, const float*, const float*, const float*,
                                       float*, const DevState*, cudaStream_t);
#endif

template <typename T>
void launch_vblock(const GridDesc& g, const T* dinv, const T* t, const T* sin, T* out, const DevState* state,
                   cudaStream_t s) {
  k_vblock<T><<<dim3(blocks_for(g.cstride / vw<T>()), g.nb), kBlock, 0, s>>>(g, dinv, t, sin, out, state);
}
#if MPCG_STENCIL_PLAIN
template void launch_vblock<double>(const GridDesc&, const double*, const double*, const double*, double*,
                                    const DevState*, cudaStream_t);
template void launch_vblock<float>(const GridDesc&, const float*, const float*, const float*, float*,
                                   const DevState*, cudaStream_t);
#endif

#if MPCG_STENCIL_PLAIN
template void launch_jacobi<double>(const GridDesc&, const double*, const double*, const double*, const double*,
                                    double*, int, const DevState*, cudaStream_t);
template void launch_jacobi<float>(const GridDesc&, const float*, const float*, const float*, const float*, float*,
                                   int, const DevState*, cudaStream_t);
#endif


// out = sum of the ncols columns of Zc (the additive MG correction B r of
// Eq. 3 as a single search direction), columns added in order.
template <typename T>
__global__ void k_sum_columns(GridDesc g, const T* __restrict__ Zc, int ncols, T* __restrict__ out,
                              const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const long long o = (long long)pb * g.len + g.G;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    T v = Zc[o + t];
    for (int c = 1; c < ncols; ++c) v += Zc[(long long)c * g.cp + o + t];
    out[o + t] = v;
  }
}

template <typename T>
void launch_sum_columns(const GridDesc& g, const T* Zc, int ncols, T* out, const DevState* state, cudaStream_t s) {
  k_sum_columns<T><<<dim3(stream_blocks(g), g.nb), kBlock, 0, s>>>(g, Zc, ncols, out, state);
}
#if MPCG_STENCIL_PLAIN
template void launch_sum_columns<double>(const GridDesc&, const double*, int, double*, const DevState*, cudaStream_t);
template void launch_sum_columns<float>(const GridDesc&, const float*, int, float*, const DevState*, cudaStream_t);
#endif

template <typename T>
void launch_coarse_tail(int jt, const GridDesc* g, const T* const* st, const T* const* dinv, T* const* r,
                        T* const* z, const T* rin, const double* a0inv, const DevState* state, cudaStream_t s) {
  TailArgs<T> a = {};
  a.jt = jt;
  for (int j = 0; j <= jt + 1; ++j) {
    a.g[j] = g[j];
    a.st[j] = st[j];
    a.dinv[j] = dinv[j];
    a.r[j] = r[j];
    a.z[j] = z[j];
  }
  a.rin = rin;
  a.a0inv = a0inv;
  const dim3 grid(1, g[0].nb);
  const size_t smem = (size_t)g[0].n * sizeof(double);
  if (g[0].dim == 3) k_coarse_tail<T, 3><<<grid, 1024, smem, s>>>(a, state);
  else k_coarse_tail<T, 2><<<grid, 1024, smem, s>>>(a, state);
}
#if MPCG_STENCIL_PLAIN
template void launch_coarse_tail<double>(int, const GridDesc*, const double* const*, const double* const*,
                                         double* const*, double* const*, const double*, const double*,
                                         const DevState*, cudaStream_t);
template void launch_coarse_tail<float>(int, const GridDesc*, const float* const*, const float* const*,
                                        float* const*, float* const*, const float*, const double*, const DevState*,
                                        cudaStream_t);
#endif

template <typename T>
void launch_gs_colour(const GridDesc& g, const T* st, const T* b, T* x, int colour, double omega, const DevState* state,
                      cudaStream_t s) {
  const dim3 grid(blocks_for(g.npts), g.nb);
  if (g.dim == 3) k_gs_colour<T, 3><<<grid, kBlock, 0, s>>>(g, st, b, x, colour, (T)omega, state);
  else k_gs_colour<T, 2><<<grid, kBlock, 0, s>>>(g, st, b, x, colour, (T)omega, state);
}
#if MPCG_STENCIL_PLAIN
template void launch_gs_colour<double>(const GridDesc&, const double*, const double*, double*, int, double,
                                       const DevState*, cudaStream_t);
template void launch_gs_colour<float>(const GridDesc&, const float*, const float*, float*, int, double,
                                      const DevState*, cudaStream_t);
#endif

template <typename T>
void launch_defect(const GridDesc& g, const T* st, const T* b, const T* x, T* d, const DevState* state,
                   cudaStream_t s) {
  const dim3 grid(blocks_for(g.npts / vw<T>()), g.nb);
  if (g.dim == 3) k_defect<T, 3><<<grid, kBlock, 0, s>>>(g, st, b, x, d, state);
  else k_defect<T, 2><<<grid, kBlock, 0, s>>>(g, st, b, x, d, state);
}
#if MPCG_STENCIL_PLAIN
template void launch_defect<double>(const GridDesc&, const double*, const double*, const double*, double*,
                                    const DevState*, cudaStream_t);
template void launch_defect<float>(const GridDesc&, const float*, const float*, const float*, float*,
                                   const DevState*, cudaStream_t);
#endif

template <typename T>
void launch_prolong_add(const GridDesc& gc, const GridDesc& gf, const T* coarse, T* fine, const DevState* state,
                        cudaStream_t s) {
  const dim3 grid(blocks_for(gf.npts), gf.nb);
  if (gf.dim == 3) k_prolong_add<T, 3><<<grid, kBlock, 0, s>>>(gc, gf, coarse, fine, state);
  else k_prolong_add<T, 2><<<grid, kBlock, 0, s>>>(gc, gf, coarse, fine, state);
}
#if MPCG_STENCIL_PLAIN
template void launch_prolong_add<double>(const GridDesc&, const GridDesc&, const double*, double*, const DevState*,
                                         cudaStream_t);
template void launch_prolong_add<float>(const GridDesc&, const GridDesc&, const float*, float*, const DevState*,
                                        cudaStream_t);
#endif

template <typename T>
void launch_add_to(const GridDesc& g, const T* src, T* dst, const DevState* state, cudaStream_t s) {
  k_add_to<T><<<dim3(blocks_for(g.npts), g.nb), kBlock, 0, s>>>(g, src, dst, state);
}
#if MPCG_STENCIL_PLAIN
template void launch_add_to<double>(const GridDesc&, const double*, double*, const DevState*, cudaStream_t);
template void launch_add_to<float>(const GridDesc&, const float*, float*, const DevState*, cudaStream_t);
#endif

template <typename T>
void launch_prolong_all(const GridDesc& gf, const T* const* coarse, const GridDesc* gcs, int J, T* Z,
                        const DevState* state, cudaStream_t s) {
  CoarseSrc<T> src = {};
  for (int j = 0; j < J; ++j) {
    src.v[j] = coarse[j];
    src.g[j] = gcs[j];
  }
  const dim3 grid(blocks_for(gf.npts / vw<T>()), gf.nb);
  static_assert(kMaxLevels <= 12, "the switch below covers up to 11 coarse grids");
#define MPCG_PROLONG_CASE(JJ)                                                                   \
  case JJ:                                                                                      \
    if (gf.dim == 3) k_prolong_all<T, 3, JJ><<<grid, kBlock, 0, s>>>(gf, src, Z, state);       \
    else k_prolong_all<T, 2, JJ><<<grid, kBlock, 0, s>>>(gf, src, Z, state);                   \
    break;
  switch (J) {
    MPCG_PROLONG_CASE(1) MPCG_PROLONG_CASE(2) MPCG_PROLONG_CASE(3) MPCG_PROLONG_CASE(4) MPCG_PROLONG_CASE(5)
    MPCG_PROLONG_CASE(6) MPCG_PROLONG_CASE(7) MPCG_PROLONG_CASE(8) MPCG_PROLONG_CASE(9) MPCG_PROLONG_CASE(10)
    MPCG_PROLONG_CASE(11)
    default: break;
  }
#undef MPCG_PROLONG_CASE
}
#if MPCG_STENCIL_PLAIN
template void launch_prolong_all<double>(const GridDesc&, const double* const*, const GridDesc*, int, double*,
                                         const DevState*, cudaStream_t);
template void launch_prolong_all<float>(const GridDesc&, const float* const*, const GridDesc*, int, float*,
                                        const DevState*, cudaStream_t);
#endif

#if MPCG_STENCIL_PLAIN
void launch_galerkin(const GridDesc& gf, const GridDesc& gc, const double* stf, double* stc, cudaStream_t s) {
  const dim3 grid(blocks_for(gc.npts), gc.nb);
  if (gc.dim == 3) k_galerkin<3><<<grid, kBlock, 0, s>>>(gf, gc, stf, stc);
  else k_galerkin<2><<<grid, kBlock, 0, s>>>(gf, gc, stf, stc);
}
#endif

template <typename T>
void launch_dinv(const GridDesc& g, const double* st, T* dinv, double omega, cudaStream_t s) {
  k_dinv<T><<<dim3(blocks_for(g.npts), g.nb), kBlock, 0, s>>>(g, st, dinv, omega);
}
#if MPCG_STENCIL_PLAIN
template void launch_dinv<double>(const GridDesc&, const double*, double*, double, cudaStream_t);
template void launch_dinv<float>(const GridDesc&, const double*, float*, double, cudaStream_t);
#endif

#if MPCG_STENCIL_PLAIN
void launch_convert_f32(const double* src, float* dst, long long count, cudaStream_t s) {
  k_convert_f32<<<grid_for(count, 4096), kBlock, 0, s>>>(src, dst, count);
}
#endif

#if MPCG_STENCIL_PLAIN
template void launch_pack_flag<double>(const GridDesc&, const double*, double*, int*, cudaStream_t);
#elif defined(MPCG_STENCIL_DW)
// The double-word instances (FP64 data, double-FP32 arithmetic), compiled in
// their own translation unit (stencil_dw.cu) to keep the build parallel.
template void launch_pack<double, dw>(const GridDesc&, const double*, long long, dw*, int, cudaStream_t);
template void launch_unpack<dw, double>(const GridDesc&, const dw*, double*, long long, int, cudaStream_t);
template void launch_pack_flag<dw>(const GridDesc&, const double*, dw*, int*, cudaStream_t);
template int spmm_blocks<dw>(const GridDesc&, int);
template void launch_spmm<dw>(const GridDesc&, const dw*, const dw*, dw*, int, double*, const DevState*,
                              cudaStream_t);
template void launch_residual<dw>(const GridDesc&, const dw*, const dw*, const dw*, dw*, double*, cudaStream_t,
                                  const int*);
template void launch_restrict<dw>(const GridDesc&, const GridDesc&, const dw*, dw*, const DevState*, cudaStream_t);
template void launch_jacobi<dw>(const GridDesc&, const dw*, const dw*, const dw*, const dw*, dw*, int,
                                const DevState*, cudaStream_t);
template void launch_vres<dw>(const GridDesc&, const dw*, const dw*, const dw*, dw*, const DevState*, cudaStream_t);
template void launch_vblock<dw>(const GridDesc&, const dw*, const dw*, const dw*, dw*, const DevState*,
                                cudaStream_t);
template void launch_vres_block<dw>(const GridDesc&, const dw*, const dw*, const dw*, const dw*, dw*,
                                    const DevState*, cudaStream_t);
template void launch_sum_columns<dw>(const GridDesc&, const dw*, int, dw*, const DevState*, cudaStream_t);
template void launch_coarse_tail<dw>(int, const GridDesc*, const dw* const*, const dw* const*, dw* const*,
                                     dw* const*, const dw*, const double*, const DevState*, cudaStream_t);
template void launch_gs_colour<dw>(const GridDesc&, const dw*, const dw*, dw*, int, double, const DevState*,
                                   cudaStream_t);
template void launch_defect<dw>(const GridDesc&, const dw*, const dw*, const dw*, dw*, const DevState*,
                                cudaStream_t);
template void launch_prolong_add<dw>(const GridDesc&, const GridDesc&, const dw*, dw*, const DevState*,
                                     cudaStream_t);
template void launch_add_to<dw>(const GridDesc&, const dw*, dw*, const DevState*, cudaStream_t);
template void launch_prolong_all<dw>(const GridDesc&, const dw* const*, const GridDesc*, int, dw*,
                                     const DevState*, cudaStream_t);
template void launch_dinv<dw>(const GridDesc&, const double*, dw*, double, cudaStream_t);

namespace {
__global__ void k_convert_dw(const double* __restrict__ src, dw* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = dw_from_double(src[i]);
}
}  // namespace

void launch_convert_dw(const double* src, dw* dst, long long count, cudaStream_t s) {
  k_convert_dw<<<grid_for(count, 4096), kBlock, 0, s>>>(src, dst, count);
}
#endif

#ifdef MPCG_STENCIL_SYM
// FP32 kernels on the symmetric half of a scalar stencil, compiled in their
// own translation unit (stencil_sym.cu).
int sym_planes(int dim) { return dim == 3 ? 14 : 5; }

void launch_sym_half(const GridDesc& g, const double* st, float* half, cudaStream_t s) {
  if (g.dim == 3) k_sym_half<3><<<grid_for(g.cp, 4096), kBlock, 0, s>>>(g, st, half);
  else k_sym_half<2><<<grid_for(g.cp, 4096), kBlock, 0, s>>>(g, st, half);
}

void launch_spmm_sym(const GridDesc& g, const float* half, const float* X, float* Y, int C, double* zaz,
                     const DevState* state, cudaStream_t s) {
  if (g.ncomp != 1) return;
  if (g.dim == 3) spmm_dim<float, 3, true>(g, half, X, Y, C, zaz, state, s);
  else spmm_dim<float, 2, true>(g, half, X, Y, C, zaz, state, s);
}

void launch_jacobi_sym(const GridDesc& g, const float* half, const float* dinv, const float* r, const float* sin,
                       float* out, int mode, const DevState* state, cudaStream_t s) {
  if (g.ncomp != 1) return;
  jacobi_impl<float, true>(g, half, dinv, r, sin, out, mode, state, s);
}
#endif

}  // namespace mpcg
