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
#include "vec.cuh"

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
    const int x = (int)(i % g.n1);
    const long long q = i / g.n1;
    const int y = (int)(q % g.n1);
    const int z = (int)(q / g.n1);
    dst[(long long)c * g.cp + g.G + x + (long long)g.p * y + (long long)g.p * g.p * z] = (TO)src[(long long)c * ld + i];
  }
}

template <typename TI, typename TO>
__global__ void k_unpack(GridDesc g, const TI* __restrict__ src, TO* __restrict__ dst, long long ld, int ncols) {
  const long long n = g.n;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * ncols;
       t += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(t / n);
    const long long i = t - (long long)c * n;
    const int x = (int)(i % g.n1);
    const long long q = i / g.n1;
    const int y = (int)(q % g.n1);
    const int z = (int)(q / g.n1);
    dst[(long long)c * ld + i] = (TO)src[(long long)c * g.cp + g.G + x + (long long)g.p * y + (long long)g.p * g.p * z];
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

// Row offsets of the 3^DIM stencil around the group start, row k = dy + 3 dz.
template <int DIM>
__device__ __forceinline__ long long row_offset(int k, long long p) {
  const int dy = k % 3 - 1, dz = DIM == 3 ? k / 3 - 1 : 0;
  return dy * p + dz * p * p;
}

// acc[c][w] += sum over the stencil of A(point w) * X_c(neighbour), C columns;
// pitch = distance between stencil planes and between columns.
template <typename T, int DIM, int C>
__device__ __forceinline__ void stencil_group(const T* __restrict__ st, long long pitch, const T* __restrict__ X,
                                              long long idx, long long p, T (&acc)[C][Vec<T>::W]) {
  constexpr int W = Vec<T>::W;
  constexpr int R = DIM == 3 ? 9 : 3;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const long long ro = row_offset<DIM>(k, p);
    T a0[W], a1[W], a2[W];
    Vec<T>::load(st + (long long)(3 * k + 0) * pitch + idx, a0);
    Vec<T>::load(st + (long long)(3 * k + 1) * pitch + idx, a1);
    Vec<T>::load(st + (long long)(3 * k + 2) * pitch + idx, a2);
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

template <typename T, int DIM, int C, bool ZAZ>
__global__ void __launch_bounds__(kBlock) k_spmm(GridDesc g, const T* __restrict__ st, const T* __restrict__ X,
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
    stencil_group<T, DIM, C>(st, g.cp, X, idx, g.p, acc);
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

template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_residual(GridDesc g, const T* __restrict__ st, const T* __restrict__ b,
                                                     const T* __restrict__ xv, T* __restrict__ r, double* part) {
  constexpr int W = Vec<T>::W;
  const int pb = blockIdx.y;
  const long long bo = (long long)pb * g.len;
  T sums[2] = {0, 0};
  const long long ngroups = g.npts / W;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    const long long idx = bo + g.G + q * W;
    T acc[1][W];
#pragma unroll
    for (int w = 0; w < W; ++w) acc[0][w] = 0;
    stencil_group<T, DIM, 1>(st, g.cp, xv, idx, g.p, acc);
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

// Restriction R = P^T: coarse node I sits on fine node 2I+1 (per axis); the
// fine nodes at distance one carry weight 1/2 per differing axis.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_restrict(GridDesc gf, GridDesc gc, const T* __restrict__ rf,
                                                     T* __restrict__ rc, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= gc.npts) return;
  rf += (long long)pb * gf.len;
  rc += (long long)pb * gc.len;
  int X, Y, Z;
  decode(gc, t, X, Y, Z);
  const long long idc = gc.G + t;
  if (!interior(gc, X, Y, Z)) {
    rc[idc] = (T)0;
    return;
  }
  const long long pf = gf.p, pp = pf * pf;
  const long long idf = gf.G + (2 * X + 1) + pf * (2 * Y + 1) + (DIM == 3 ? pp * (2 * Z + 1) : 0);
  T acc = 0;
#pragma unroll
  for (int ez = (DIM == 3 ? -1 : 0); ez <= (DIM == 3 ? 1 : 0); ++ez) {
#pragma unroll
    for (int ey = -1; ey <= 1; ++ey) {
#pragma unroll
      for (int ex = -1; ex <= 1; ++ex) {
        const T w = (T)((ex ? 0.5 : 1.0) * (ey ? 0.5 : 1.0) * (ez ? 0.5 : 1.0));
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
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_jacobi(GridDesc g, const T* __restrict__ st, const T* __restrict__ dinv,
                                                   const T* __restrict__ r, const T* __restrict__ sin,
                                                   T* __restrict__ out, int mode, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  constexpr int W = Vec<T>::W;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= g.npts / W) return;
  const long long idx = (long long)pb * g.len + g.G + q * W;
  T di[W], ri[W], o[W];
  Vec<T>::load_keep(dinv + idx, di);
  Vec<T>::load_keep(r + idx, ri);
  if (mode == 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) o[w] = di[w] * ri[w];
    Vec<T>::store(out + idx, o);
    return;
  }
  T acc[1][W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[0][w] = 0;
  if (mode == 1) {
    constexpr int R = DIM == 3 ? 9 : 3;
#pragma unroll
    for (int k = 0; k < R; ++k) {
      const long long ro = row_offset<DIM>(k, g.p);
      T a0[W], a1[W], a2[W], ed[W + 2], er[W + 2];
      Vec<T>::load(st + (long long)(3 * k + 0) * g.cp + idx, a0);
      Vec<T>::load(st + (long long)(3 * k + 1) * g.cp + idx, a1);
      Vec<T>::load(st + (long long)(3 * k + 2) * g.cp + idx, a2);
      load_row<T>(dinv + idx + ro, ed);
      load_row<T>(r + idx + ro, er);
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
  } else {
    stencil_group<T, DIM, 1>(st, g.cp, sin, idx, g.p, acc);
    T sv[W];
    Vec<T>::load_keep(sin + idx, sv);
#pragma unroll
    for (int w = 0; w < W; ++w) o[w] = sv[w] + di[w] * (ri[w] - acc[0][w]);
  }
  Vec<T>::store(out + idx, o);
}

// Prolongation P: bilinear / trilinear interpolation from the coarse grid.
// A group of W fine points starting at even x0 needs the coarse values
// x0/2 - 1 .. x0/2 + W/2 - 1 of each contributing coarse row:
//   fine x0 + 2k     = (c[x0/2 + k - 1] + c[x0/2 + k]) / 2
//   fine x0 + 2k + 1 =  c[x0/2 + k]
// Parents outside the grid are pad entries of the coarse layout (zero).
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_prolong(GridDesc gc, GridDesc gf, const T* __restrict__ coarse,
                                                    T* __restrict__ fine, int ncols, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  constexpr int W = Vec<T>::W;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= gf.npts / W) return;
  const long long t0 = q * W;
  int x0, y, z;
  decode(gf, t0, x0, y, z);
  const long long idf = (long long)pb * gf.len + gf.G + t0;
  // per axis: parents (c0, c1) with weights (w0, w1)
  auto par = [](int i, int& c0, int& c1, T& w0, T& w1) {
    if (i & 1) { c0 = c1 = i >> 1; w0 = (T)1; w1 = (T)0; }
    else { c0 = (i >> 1) - 1; c1 = i >> 1; w0 = w1 = (T)0.5; }
  };
  int cy0, cy1, cz0 = 0, cz1 = 0;
  T wy0, wy1, wz0 = 1, wz1 = 0;
  par(y, cy0, cy1, wy0, wy1);
  if (DIM == 3) par(z, cz0, cz1, wz0, wz1);
  const long long pc = gc.p, ppc = pc * pc;
  const int cx = x0 >> 1;
  for (int c = 0; c < ncols; ++c) {
    const T* C0 = coarse + (long long)c * gc.cp + (long long)pb * gc.len + gc.G;
    T row[W / 2 + 1];
#pragma unroll
    for (int k = 0; k <= W / 2; ++k) row[k] = 0;
#pragma unroll
    for (int kz = 0; kz < (DIM == 3 ? 2 : 1); ++kz) {
      const int czz = kz ? cz1 : cz0;
      const T wz = kz ? wz1 : wz0;
#pragma unroll
      for (int ky = 0; ky < 2; ++ky) {
        const int cyy = ky ? cy1 : cy0;
        const T wgt = wz * (ky ? wy1 : wy0);
        const T* rp = C0 + pc * cyy + (DIM == 3 ? ppc * czz : 0) + cx - 1;
#pragma unroll
        for (int k = 0; k <= W / 2; ++k) row[k] = fma(wgt, rp[k], row[k]);
      }
    }
    T o[W];
#pragma unroll
    for (int k = 0; k < W / 2; ++k) {
      o[2 * k] = (T)0.5 * (row[k] + row[k + 1]);
      o[2 * k + 1] = row[k + 1];
    }
    Vec<T>::store(fine + (long long)c * gf.cp + idf, o);
  }
}

// Galerkin product A_c = P^T A_f P, one coarse row per thread.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_galerkin(GridDesc gf, GridDesc gc, const double* __restrict__ stf,
                                                     double* __restrict__ stc) {
  constexpr int S = DIM == 3 ? 27 : 9;
  const int pb = blockIdx.y;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= gc.npts) return;
  stf += (long long)pb * gf.len;
  stc += (long long)pb * gc.len;
  int X, Y, Z;
  decode(gc, t, X, Y, Z);
  const long long idc = gc.G + t;
  if (!interior(gc, X, Y, Z)) {
    for (int s = 0; s < S; ++s) stc[s * gc.cp + idc] = 0.0;
    return;
  }
  double acc[S];
#pragma unroll
  for (int s = 0; s < S; ++s) acc[s] = 0.0;
  const long long pf = gf.p, ppf = pf * pf;
  const int nc = gc.n1;
  for (int ez = (DIM == 3 ? -1 : 0); ez <= (DIM == 3 ? 1 : 0); ++ez)
    for (int ey = -1; ey <= 1; ++ey)
      for (int ex = -1; ex <= 1; ++ex) {
        const double we = (ex ? 0.5 : 1.0) * (ey ? 0.5 : 1.0) * (ez ? 0.5 : 1.0);
        const long long idf = gf.G + (2 * X + 1 + ex) + pf * (2 * Y + 1 + ey) + (DIM == 3 ? ppf * (2 * Z + 1 + ez) : 0);
        for (int s = 0; s < S; ++s) {
          const double a = stf[s * gf.cp + idf];
          if (a == 0.0) continue;
          const int f[3] = {ex + (s % 3 - 1), ey + ((s / 3) % 3 - 1), DIM == 3 ? ez + (s / 9 - 1) : 0};
          // coarse parents of the fine column node, relative to (X, Y, Z)
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
                if (cx < 0 || cx >= nc || cy < 0 || cy >= nc) continue;
                if (DIM == 3 && (cz < 0 || cz >= nc)) continue;
                acc[(Dx + 1) + 3 * (Dy + 1) + (DIM == 3 ? 9 * (Dz + 1) : 0)] += base;
              }
        }
      }
  for (int s = 0; s < S; ++s) stc[s * gc.cp + idc] = acc[s];
}

template <typename T>
__global__ void k_dinv(GridDesc g, const double* __restrict__ st, T* __restrict__ dinv, double omega) {
  const int pb = blockIdx.y;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.npts) return;
  int x, y, z;
  decode(g, t, x, y, z);
  const long long idx = (long long)pb * g.len + g.G + t;
  const int centre = g.dim == 3 ? 13 : 4;
  dinv[idx] = interior(g, x, y, z) ? (T)(omega / st[centre * g.cp + idx]) : (T)0;
}

__global__ void k_convert_f32(const double* __restrict__ src, float* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
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
template <typename TI, typename TO>
void launch_unpack(const GridDesc& g, const TI* src, TO* dst, long long ld, int ncols, cudaStream_t s) {
  k_unpack<TI, TO><<<grid_for(g.n * ncols, 4096), kBlock, 0, s>>>(g, src, dst, ld, ncols);
}
template void launch_pack<double, double>(const GridDesc&, const double*, long long, double*, int, cudaStream_t);
template void launch_pack<double, float>(const GridDesc&, const double*, long long, float*, int, cudaStream_t);
template void launch_unpack<double, double>(const GridDesc&, const double*, double*, long long, int, cudaStream_t);
template void launch_unpack<float, double>(const GridDesc&, const float*, double*, long long, int, cudaStream_t);
template void launch_pack<float, float>(const GridDesc&, const float*, long long, float*, int, cudaStream_t);
template void launch_unpack<float, float>(const GridDesc&, const float*, float*, long long, int, cudaStream_t);

template <typename T, int DIM>
static void spmm_dim(const GridDesc& g, const T* st, const T* X, T* Y, int C, double* zaz, const DevState* state,
                     cudaStream_t s) {
  const dim3 grid(stream_blocks(g), g.nb);
#define MPCG_SPMM_CASE(CC)                                                                      \
  case CC:                                                                                      \
    if (zaz) k_spmm<T, DIM, CC, true><<<grid, kBlock, 0, s>>>(g, st, X, Y, zaz, state);         \
    else k_spmm<T, DIM, CC, false><<<grid, kBlock, 0, s>>>(g, st, X, Y, zaz, state);           \
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
void launch_spmm(const GridDesc& g, const T* st, const T* X, T* Y, int C, double* zaz, const DevState* state,
                 cudaStream_t s) {
  if (g.dim == 3) spmm_dim<T, 3>(g, st, X, Y, C, zaz, state, s);
  else spmm_dim<T, 2>(g, st, X, Y, C, zaz, state, s);
}
template void launch_spmm<double>(const GridDesc&, const double*, const double*, double*, int, double*,
                                  const DevState*, cudaStream_t);
template void launch_spmm<float>(const GridDesc&, const float*, const float*, float*, int, double*,
                                 const DevState*, cudaStream_t);

template <typename T>
void launch_residual(const GridDesc& g, const T* st, const T* b, const T* x, T* r, double* part, cudaStream_t s) {
  const dim3 grid(stream_blocks(g), g.nb);
  if (g.dim == 3) k_residual<T, 3><<<grid, kBlock, 0, s>>>(g, st, b, x, r, part);
  else k_residual<T, 2><<<grid, kBlock, 0, s>>>(g, st, b, x, r, part);
}
template void launch_residual<double>(const GridDesc&, const double*, const double*, const double*, double*,
                                      double*, cudaStream_t);
template void launch_residual<float>(const GridDesc&, const float*, const float*, const float*, float*, double*,
                                     cudaStream_t);

template <typename T>
void launch_restrict(const GridDesc& gf, const GridDesc& gc, const T* rf, T* rc, const DevState* state,
                     cudaStream_t s) {
  const dim3 grid(blocks_for(gc.npts), gc.nb);
  if (gc.dim == 3) k_restrict<T, 3><<<grid, kBlock, 0, s>>>(gf, gc, rf, rc, state);
  else k_restrict<T, 2><<<grid, kBlock, 0, s>>>(gf, gc, rf, rc, state);
}
template void launch_restrict<double>(const GridDesc&, const GridDesc&, const double*, double*, const DevState*,
                                      cudaStream_t);
template void launch_restrict<float>(const GridDesc&, const GridDesc&, const float*, float*, const DevState*,
                                     cudaStream_t);

template <typename T>
void launch_jacobi(const GridDesc& g, const T* st, const T* dinv, const T* r, const T* sin, T* out, int mode,
                   const DevState* state, cudaStream_t s) {
  const dim3 grid(blocks_for(g.npts / vw<T>()), g.nb);
  if (g.dim == 3) k_jacobi<T, 3><<<grid, kBlock, 0, s>>>(g, st, dinv, r, sin, out, mode, state);
  else k_jacobi<T, 2><<<grid, kBlock, 0, s>>>(g, st, dinv, r, sin, out, mode, state);
}
template void launch_jacobi<double>(const GridDesc&, const double*, const double*, const double*, const double*,
                                    double*, int, const DevState*, cudaStream_t);
template void launch_jacobi<float>(const GridDesc&, const float*, const float*, const float*, const float*, float*,
                                   int, const DevState*, cudaStream_t);

template <typename T>
void launch_prolong(const GridDesc& gc, const GridDesc& gf, const T* coarse, T* fine, int ncols,
                    const DevState* state, cudaStream_t s) {
  const dim3 grid(blocks_for(gf.npts / vw<T>()), gf.nb);
  if (gf.dim == 3) k_prolong<T, 3><<<grid, kBlock, 0, s>>>(gc, gf, coarse, fine, ncols, state);
  else k_prolong<T, 2><<<grid, kBlock, 0, s>>>(gc, gf, coarse, fine, ncols, state);
}
template void launch_prolong<double>(const GridDesc&, const GridDesc&, const double*, double*, int,
                                     const DevState*, cudaStream_t);
template void launch_prolong<float>(const GridDesc&, const GridDesc&, const float*, float*, int, const DevState*,
                                    cudaStream_t);

void launch_galerkin(const GridDesc& gf, const GridDesc& gc, const double* stf, double* stc, cudaStream_t s) {
  const dim3 grid(blocks_for(gc.npts), gc.nb);
  if (gc.dim == 3) k_galerkin<3><<<grid, kBlock, 0, s>>>(gf, gc, stf, stc);
  else k_galerkin<2><<<grid, kBlock, 0, s>>>(gf, gc, stf, stc);
}

template <typename T>
void launch_dinv(const GridDesc& g, const double* st, T* dinv, double omega, cudaStream_t s) {
  k_dinv<T><<<dim3(blocks_for(g.npts), g.nb), kBlock, 0, s>>>(g, st, dinv, omega);
}
template void launch_dinv<double>(const GridDesc&, const double*, double*, double, cudaStream_t);
template void launch_dinv<float>(const GridDesc&, const double*, float*, double, cudaStream_t);

void launch_convert_f32(const double* src, float* dst, long long count, cudaStream_t s) {
  k_convert_f32<<<grid_for(count, 4096), kBlock, 0, s>>>(src, dst, count);
}

}  // namespace mpcg
