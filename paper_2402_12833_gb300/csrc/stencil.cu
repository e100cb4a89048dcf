// Structured-grid kernels: layout conversion, block stencil SpMM (the A Z
// product of Section 2.2), residual, restriction R = P^T and prolongation P
// (Section 2.1), damped-Jacobi smoothing (Eq. 3), and the Galerkin product
// P^T A P that builds the coarse operators.
//
// All kernels work on the padded layout described in common.cuh: one thread
// per entry of the padded box, pad entries written as zero.
#include "kernels.cuh"

namespace mpcg {

namespace {

__device__ __forceinline__ void decode(const GridDesc& g, long long t, int& x, int& y, int& z) {
  const int mask = g.p - 1;
  x = (int)(t & mask);
  y = (int)((t >> g.lp) & mask);
  z = (int)(t >> (2 * g.lp));
}

__device__ __forceinline__ bool interior(const GridDesc& g, int x, int y, int z) {
  return x < g.n1 && y < g.n1 && (g.dim == 2 || z < g.n1);
}

// Sum NV per-thread values over the block, written value-major to
// part[v * stride + blockIdx.x].  Fixed reduction order (deterministic).
template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* part, int stride) {
  __shared__ double sh[kBlock / 32][NV > 0 ? NV : 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double a = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) sh[warp][i] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += blockDim.x) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += sh[w][i];
    part[(long long)i * stride + blockIdx.x] = a;
  }
}

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
    dst[(long long)c * g.len + g.G + x + (long long)g.p * y + (long long)g.p * g.p * z] = (TO)src[(long long)c * ld + i];
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
    dst[(long long)c * ld + i] = (TO)src[(long long)c * g.len + g.G + x + (long long)g.p * y + (long long)g.p * g.p * z];
  }
}

// Apply the 3^DIM stencil at padded index idx to vector v.
template <typename T, int DIM>
__device__ __forceinline__ T stencil_apply(const T (&a)[DIM == 3 ? 27 : 9], const T* __restrict__ v,
                                           long long idx, int p) {
  T acc = 0;
  const long long pp = (long long)p * p;
#pragma unroll
  for (int dz = 0; dz < (DIM == 3 ? 3 : 1); ++dz) {
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      const T* row = v + idx + (long long)(dy - 1) * p + (DIM == 3 ? (long long)(dz - 1) * pp : 0);
      const int s = dz * 9 + dy * 3;
      acc = fma(a[s + 0], row[-1], acc);
      acc = fma(a[s + 1], row[0], acc);
      acc = fma(a[s + 2], row[1], acc);
    }
  }
  return acc;
}

template <typename T, int DIM>
__device__ __forceinline__ void load_stencil(T (&a)[DIM == 3 ? 27 : 9], const T* __restrict__ st, long long len,
                                             long long idx) {
#pragma unroll
  for (int s = 0; s < (DIM == 3 ? 27 : 9); ++s) a[s] = st[s * len + idx];
}

template <typename T, int DIM, int C, bool ZAZ>
__global__ void __launch_bounds__(kBlock) k_spmm(GridDesc g, const T* __restrict__ st, const T* __restrict__ X,
                                                 T* __restrict__ Y, double* zaz, const DevState* state) {
  if (state && state->done) return;
  constexpr int S = DIM == 3 ? 27 : 9;
  double acc[ZAZ ? C : 1];
#pragma unroll
  for (int c = 0; c < (ZAZ ? C : 1); ++c) acc[c] = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    decode(g, t, x, y, z);
    const long long idx = g.G + t;
    if (interior(g, x, y, z)) {
      T a[S];
      load_stencil<T, DIM>(a, st, g.len, idx);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const T* Xc = X + (long long)c * g.len;
        const T yv = stencil_apply<T, DIM>(a, Xc, idx, g.p);
        Y[(long long)c * g.len + idx] = yv;
        if (ZAZ) acc[c] += (double)Xc[idx] * (double)yv;
      }
    } else {
#pragma unroll
      for (int c = 0; c < C; ++c) Y[(long long)c * g.len + idx] = (T)0;
    }
  }
  if (ZAZ) block_sum_store<ZAZ ? C : 1>(acc, zaz, kRedBlocks);
}

template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_residual(GridDesc g, const T* __restrict__ st, const T* __restrict__ b,
                                                     const T* __restrict__ xv, T* __restrict__ r, double* part) {
  constexpr int S = DIM == 3 ? 27 : 9;
  double acc[2] = {0.0, 0.0};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    decode(g, t, x, y, z);
    const long long idx = g.G + t;
    if (interior(g, x, y, z)) {
      T a[S];
      load_stencil<T, DIM>(a, st, g.len, idx);
      const T rv = b[idx] - stencil_apply<T, DIM>(a, xv, idx, g.p);
      r[idx] = rv;
      acc[0] += (double)rv * (double)rv;
      acc[1] += (double)b[idx] * (double)b[idx];
    } else {
      r[idx] = (T)0;
    }
  }
  block_sum_store<2>(acc, part, kRedBlocks);
}

// Restriction R = P^T: coarse node I sits on fine node 2I+1 (per axis); the
// fine nodes at distance one carry weight 1/2 per differing axis.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_restrict(GridDesc gf, GridDesc gc, const T* __restrict__ rf,
                                                     T* __restrict__ rc, const DevState* state) {
  if (state && state->done) return;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= gc.npts) return;
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

// Damped Jacobi (Eq. 3 with M = D / omega, dinv = omega / diag).
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_jacobi(GridDesc g, const T* __restrict__ st, const T* __restrict__ dinv,
                                                   const T* __restrict__ r, const T* __restrict__ sin,
                                                   T* __restrict__ out, int mode, const DevState* state) {
  if (state && state->done) return;
  constexpr int S = DIM == 3 ? 27 : 9;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.npts) return;
  int x, y, z;
  decode(g, t, x, y, z);
  const long long idx = g.G + t;
  if (!interior(g, x, y, z)) {
    out[idx] = (T)0;
    return;
  }
  const T di = dinv[idx], ri = r[idx];
  if (mode == 0) {
    out[idx] = di * ri;
    return;
  }
  T a[S];
  load_stencil<T, DIM>(a, st, g.len, idx);
  if (mode == 1) {
    // s1 = dinv r everywhere; s2 = s1 + dinv (r - A s1), evaluated with s1
    // formed on the fly at the neighbours
    const long long p = g.p, pp = p * p;
    T acc = 0;
#pragma unroll
    for (int dz = 0; dz < (DIM == 3 ? 3 : 1); ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const long long o = (dx - 1) + (dy - 1) * p + (DIM == 3 ? (dz - 1) * pp : 0);
          acc = fma(a[dz * 9 + dy * 3 + dx], dinv[idx + o] * r[idx + o], acc);
        }
    const T s1 = di * ri;
    out[idx] = s1 + di * (ri - acc);
  } else {
    const T ax = stencil_apply<T, DIM>(a, sin, idx, g.p);
    out[idx] = sin[idx] + di * (ri - ax);
  }
}

// Prolongation P: bilinear / trilinear interpolation from the coarse grid.
template <typename T, int DIM>
__global__ void __launch_bounds__(kBlock) k_prolong(GridDesc gc, GridDesc gf, const T* __restrict__ coarse,
                                                    T* __restrict__ fine, int ncols, const DevState* state) {
  if (state && state->done) return;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= gf.npts) return;
  int x, y, z;
  decode(gf, t, x, y, z);
  const long long idf = gf.G + t;
  if (!interior(gf, x, y, z)) {
    for (int c = 0; c < ncols; ++c) fine[(long long)c * gf.len + idf] = (T)0;
    return;
  }
  // per axis: parents (c0, c1) with weights (w0, w1); out-of-grid parents are
  // pad entries of the coarse layout and read as zero
  int cx0, cx1, cy0, cy1, cz0 = 0, cz1 = 0;
  T wx0, wx1, wy0, wy1, wz0 = 1, wz1 = 0;
  auto par = [](int i, int& c0, int& c1, T& w0, T& w1) {
    if (i & 1) { c0 = c1 = i >> 1; w0 = (T)1; w1 = (T)0; }
    else { c0 = (i >> 1) - 1; c1 = i >> 1; w0 = w1 = (T)0.5; }
  };
  par(x, cx0, cx1, wx0, wx1);
  par(y, cy0, cy1, wy0, wy1);
  if (DIM == 3) par(z, cz0, cz1, wz0, wz1);
  const long long pc = gc.p, ppc = pc * pc;
  for (int c = 0; c < ncols; ++c) {
    const T* C0 = coarse + (long long)c * gc.len + gc.G;
    T acc = 0;
#pragma unroll
    for (int kz = 0; kz < (DIM == 3 ? 2 : 1); ++kz) {
      const int cz = kz ? cz1 : cz0;
      const T wz = kz ? wz1 : wz0;
#pragma unroll
      for (int ky = 0; ky < 2; ++ky) {
        const int cy = ky ? cy1 : cy0;
        const T wy = ky ? wy1 : wy0;
        const T* row = C0 + pc * cy + (DIM == 3 ? ppc * cz : 0);
        acc = fma(wz * wy * wx0, row[cx0], acc);
        acc = fma(wz * wy * wx1, row[cx1], acc);
      }
    }
    fine[(long long)c * gf.len + idf] = acc;
  }
}

// Galerkin product A_c = P^T A_f P, one coarse row per thread.
template <int DIM>
__global__ void __launch_bounds__(kBlock) k_galerkin(GridDesc gf, GridDesc gc, const double* __restrict__ stf,
                                                     double* __restrict__ stc) {
  constexpr int S = DIM == 3 ? 27 : 9;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= gc.npts) return;
  int X, Y, Z;
  decode(gc, t, X, Y, Z);
  const long long idc = gc.G + t;
  if (!interior(gc, X, Y, Z)) {
    for (int s = 0; s < S; ++s) stc[s * gc.len + idc] = 0.0;
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
          const double a = stf[s * gf.len + idf];
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
          const int C[3] = {X, Y, Z};
          for (int iz = 0; iz < np[2]; ++iz)
            for (int iy = 0; iy < np[1]; ++iy)
              for (int ix = 0; ix < np[0]; ++ix) {
                const int Dx = ix ? D1[0] : D0[0], Dy = iy ? D1[1] : D0[1], Dz = iz ? D1[2] : D0[2];
                const int cx = C[0] + Dx, cy = C[1] + Dy, cz = C[2] + Dz;
                if (cx < 0 || cx >= nc || cy < 0 || cy >= nc) continue;
                if (DIM == 3 && (cz < 0 || cz >= nc)) continue;
                acc[(Dx + 1) + 3 * (Dy + 1) + (DIM == 3 ? 9 * (Dz + 1) : 0)] += base;
              }
        }
      }
  for (int s = 0; s < S; ++s) stc[s * gc.len + idc] = acc[s];
}

template <typename T>
__global__ void k_dinv(GridDesc g, const double* __restrict__ st, T* __restrict__ dinv, double omega) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= g.npts) return;
  int x, y, z;
  decode(g, t, x, y, z);
  const long long idx = g.G + t;
  const int centre = g.dim == 3 ? 13 : 4;
  dinv[idx] = interior(g, x, y, z) ? (T)(omega / st[centre * g.len + idx]) : (T)0;
}

__global__ void k_convert_f32(const double* __restrict__ src, float* __restrict__ dst, long long count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

inline int blocks_for(long long n) { return (int)((n + kBlock - 1) / kBlock); }

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

template <typename T, int DIM>
static void spmm_dim(const GridDesc& g, const T* st, const T* X, T* Y, int C, double* zaz, const DevState* state,
                     cudaStream_t s) {
  const int nb = grid_for(g.npts, kRedBlocks);
#define MPCG_SPMM_CASE(CC)                                                                      \
  case CC:                                                                                      \
    if (zaz) k_spmm<T, DIM, CC, true><<<nb, kBlock, 0, s>>>(g, st, X, Y, zaz, state);           \
    else k_spmm<T, DIM, CC, false><<<nb, kBlock, 0, s>>>(g, st, X, Y, zaz, state);             \
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
  const int nb = kRedBlocks;   // fixed so the partial count is known
  if (g.dim == 3) k_residual<T, 3><<<nb, kBlock, 0, s>>>(g, st, b, x, r, part);
  else k_residual<T, 2><<<nb, kBlock, 0, s>>>(g, st, b, x, r, part);
}
template void launch_residual<double>(const GridDesc&, const double*, const double*, const double*, double*,
                                      double*, cudaStream_t);
template void launch_residual<float>(const GridDesc&, const float*, const float*, const float*, float*, double*,
                                     cudaStream_t);

template <typename T>
void launch_restrict(const GridDesc& gf, const GridDesc& gc, const T* rf, T* rc, const DevState* state,
                     cudaStream_t s) {
  if (gc.dim == 3) k_restrict<T, 3><<<blocks_for(gc.npts), kBlock, 0, s>>>(gf, gc, rf, rc, state);
  else k_restrict<T, 2><<<blocks_for(gc.npts), kBlock, 0, s>>>(gf, gc, rf, rc, state);
}
template void launch_restrict<double>(const GridDesc&, const GridDesc&, const double*, double*, const DevState*,
                                      cudaStream_t);
template void launch_restrict<float>(const GridDesc&, const GridDesc&, const float*, float*, const DevState*,
                                     cudaStream_t);

template <typename T>
void launch_jacobi(const GridDesc& g, const T* st, const T* dinv, const T* r, const T* sin, T* out, int mode,
                   const DevState* state, cudaStream_t s) {
  if (g.dim == 3) k_jacobi<T, 3><<<blocks_for(g.npts), kBlock, 0, s>>>(g, st, dinv, r, sin, out, mode, state);
  else k_jacobi<T, 2><<<blocks_for(g.npts), kBlock, 0, s>>>(g, st, dinv, r, sin, out, mode, state);
}
template void launch_jacobi<double>(const GridDesc&, const double*, const double*, const double*, const double*,
                                    double*, int, const DevState*, cudaStream_t);
template void launch_jacobi<float>(const GridDesc&, const float*, const float*, const float*, const float*, float*,
                                   int, const DevState*, cudaStream_t);

template <typename T>
void launch_prolong(const GridDesc& gc, const GridDesc& gf, const T* coarse, T* fine, int ncols,
                    const DevState* state, cudaStream_t s) {
  if (gf.dim == 3) k_prolong<T, 3><<<blocks_for(gf.npts), kBlock, 0, s>>>(gc, gf, coarse, fine, ncols, state);
  else k_prolong<T, 2><<<blocks_for(gf.npts), kBlock, 0, s>>>(gc, gf, coarse, fine, ncols, state);
}
template void launch_prolong<double>(const GridDesc&, const GridDesc&, const double*, double*, int,
                                     const DevState*, cudaStream_t);
template void launch_prolong<float>(const GridDesc&, const GridDesc&, const float*, float*, int, const DevState*,
                                    cudaStream_t);

void launch_galerkin(const GridDesc& gf, const GridDesc& gc, const double* stf, double* stc, cudaStream_t s) {
  if (gc.dim == 3) k_galerkin<3><<<blocks_for(gc.npts), kBlock, 0, s>>>(gf, gc, stf, stc);
  else k_galerkin<2><<<blocks_for(gc.npts), kBlock, 0, s>>>(gf, gc, stf, stc);
}

template <typename T>
void launch_dinv(const GridDesc& g, const double* st, T* dinv, double omega, cudaStream_t s) {
  k_dinv<T><<<blocks_for(g.npts), kBlock, 0, s>>>(g, st, dinv, omega);
}
template void launch_dinv<double>(const GridDesc&, const double*, double*, double, cudaStream_t);
template void launch_dinv<float>(const GridDesc&, const double*, float*, double, cudaStream_t);

void launch_convert_f32(const double* src, float* dst, long long count, cudaStream_t s) {
  k_convert_f32<<<grid_for(count, 4096), kBlock, 0, s>>>(src, dst, count);
}

}  // namespace mpcg
