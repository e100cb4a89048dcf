// Operators of an algebraic hierarchy (sliced ELLPACK, EllDev in
// common.cuh): the block SpMM A Z of the Section 2.2 update with the
// z_i^T A z_i partials, the residual, damped Jacobi on every grid (Eq. 2,
// c_0 = 0) and the transfers R_j = P_j^T (restriction) and P_j
// (prolongation) of Section 2.1.  Vectors are flat padded arrays (unknown i
// at G + i); every launcher takes pointers already offset by G.
//
// A warp computes one slice: g lanes per row accumulate every g-th entry and
// a shuffle reduction over the g lanes finishes the row, so the column and
// value loads of a slot are coalesced and the slot count of the warp is
// uniform.  The gathered X entries come through L1/L2: the matrices of a
// grid hierarchy couple nearby unknowns.
#include "kernels.cuh"
#include "vec.cuh"

namespace mpcg {

namespace {

template <typename T>
__device__ __forceinline__ T ldv(const T* p) {
  return __ldg(p);
}

// sum over the g = 2^lg lanes of a row group (all 32 lanes take part)
template <typename T>
__device__ __forceinline__ T group_sum(T v, int lg) {
  for (int o = 1; o < (1 << lg); o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Y[:, c] = A X[:, c] (ADD: Y[:, c] += A X[:, c]) for C columns (column
// pitches ldx, ldy); with ZAZ the per-block partials of X[:, c]^T Y[:, c]
// (value-major, stride gridDim.x).
template <typename T, int C, bool ZAZ, bool ADD = false>
__global__ void __launch_bounds__(kBlock) k_ell_spmm(EllDev<T> A, const T* __restrict__ X, long long ldx,
                                                     T* __restrict__ Y, long long ldy, double* zaz,
                                                     const DevState* state) {
  if (state && state[0].done) return;
  T zacc[ZAZ ? C : 1];
#pragma unroll
  for (int c = 0; c < (ZAZ ? C : 1); ++c) zacc[c] = 0;
  const long long nt = (long long)A.nslices * 32;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nt; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t >> 5), lane = (int)(t & 31);
    const long long r = ((long long)s << (5 - A.lg)) + (lane >> A.lg);
    const int b = A.sptr[s];
    const int w = (A.sptr[s + 1] - b) >> 5;
    T acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = 0;
#pragma unroll 4   // four slots' loads in flight: the short coarse rows are latency-bound
    for (int k = 0; k < w; ++k) {
      const int e = b + 32 * k + lane;
      const int j = ldv(A.col + e);
      const T v = ldv(A.val + e);
#pragma unroll
      for (int c = 0; c < C; ++c) acc[c] = fma(v, X[c * ldx + j], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = group_sum(acc[c], A.lg);
    if (r < A.rows && (lane & ((1 << A.lg) - 1)) == 0) {
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (ADD) Y[c * ldy + r] += acc[c];
        else Y[c * ldy + r] = acc[c];
        if (ZAZ) zacc[c] = fma(X[c * ldx + r], acc[c], zacc[c]);
      }
    }
  }
  if (ZAZ) block_sum_store<T, ZAZ ? C : 1>(zacc, zaz, gridDim.x, blockIdx.x);
}

// r = b - A x with the partials of |r|^2 and |b|^2 (NORMS; without them it
// is the defect of the V-cycle); a zero iterate (xnz[0] == 0) gives r = b
// without reading the matrix.
template <typename T, bool NORMS = true>
__global__ void __launch_bounds__(kBlock) k_ell_residual(EllDev<T> A, const T* __restrict__ b,
                                                         const T* __restrict__ x, T* __restrict__ r,
                                                         double* part, const int* __restrict__ xnz) {
  const bool zero_x = xnz && xnz[0] == 0;
  T sums[2] = {0, 0};
  const long long nt = (long long)A.nslices * 32;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nt; t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t >> 5), lane = (int)(t & 31);
    const long long q = ((long long)s << (5 - A.lg)) + (lane >> A.lg);
    T acc = 0;
    if (!zero_x) {
      const int e0 = A.sptr[s];
      const int w = (A.sptr[s + 1] - e0) >> 5;
#pragma unroll 4
      for (int k = 0; k < w; ++k) {
        const int e = e0 + 32 * k + lane;
        acc = fma(ldv(A.val + e), x[ldv(A.col + e)], acc);
      }
      acc = group_sum(acc, A.lg);
    }
    if (q < A.rows && (lane & ((1 << A.lg) - 1)) == 0) {
      const T bv = b[q];
      const T rv = bv - acc;
      r[q] = rv;
      sums[0] = fma(rv, rv, sums[0]);
      sums[1] = fma(bv, bv, sums[1]);
    }
  }
  if (NORMS) block_sum_store<T, 2>(sums, part, gridDim.x, blockIdx.x);
}

// Damped Jacobi with dinv = omega / a_ii: mode 0: out = dinv g; mode 1: two
// sweeps from zero in one pass, out = s1 + dinv (g - A s1) with s1 = dinv g
// formed on the fly at every gathered column; mode 2: out = sin + dinv (g -
// A sin).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_ell_jacobi(EllDev<T> A, const T* __restrict__ dinv,
                                                       const T* __restrict__ g, const T* __restrict__ sin,
                                                       T* __restrict__ out, int mode, const DevState* state) {
  if (state && state[0].done) return;
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)A.nslices * 32) return;   // whole warps: the grid covers the slices in units of 32 threads
  const int s = (int)(t >> 5), lane = (int)(t & 31);
  const long long q = ((long long)s << (5 - A.lg)) + (lane >> A.lg);
  T acc = 0;
  if (mode != 0) {
    const int e0 = A.sptr[s];
    const int w = (A.sptr[s + 1] - e0) >> 5;
#pragma unroll 4
    for (int k = 0; k < w; ++k) {
      const int e = e0 + 32 * k + lane;
      const int j = ldv(A.col + e);
      const T xj = mode == 1 ? dinv[j] * g[j] : sin[j];
      acc = fma(ldv(A.val + e), xj, acc);
    }
    acc = group_sum(acc, A.lg);
  }
  if (q >= A.rows || (lane & ((1 << A.lg) - 1)) != 0) return;
  const T d = dinv[q], gv = g[q];
  if (mode == 0) out[q] = d * gv;
  else if (mode == 1) out[q] = d * gv + d * (gv - acc);
  else out[q] = sin[q] + d * (gv - acc);
}

template <typename T>
int ell_threads_blocks(const EllDev<T>& A) {
  return (int)(((long long)A.nslices * 32 + kBlock - 1) / kBlock);
}

}  // namespace

template <typename T>
void launch_ell_spmm(const EllDev<T>& A, const T* X, long long ldx, T* Y, long long ldy, int C, double* zaz,
                     int nblocks, const DevState* state, cudaStream_t s) {
  const int grid = nblocks > 0 ? nblocks : ell_threads_blocks(A);
#define MPCG_ELL_CASE(CC)                                                                                \
  case CC:                                                                                               \
    if (zaz) k_ell_spmm<T, CC, true><<<grid, kBlock, 0, s>>>(A, X, ldx, Y, ldy, zaz, state);             \
    else k_ell_spmm<T, CC, false><<<grid, kBlock, 0, s>>>(A, X, ldx, Y, ldy, zaz, state);                \
    break;
  switch (C) {
    MPCG_ELL_CASE(1) MPCG_ELL_CASE(2) MPCG_ELL_CASE(3) MPCG_ELL_CASE(4) MPCG_ELL_CASE(5) MPCG_ELL_CASE(6)
    MPCG_ELL_CASE(7) MPCG_ELL_CASE(8) MPCG_ELL_CASE(9) MPCG_ELL_CASE(10) MPCG_ELL_CASE(11) MPCG_ELL_CASE(12)
    default: break;
  }
#undef MPCG_ELL_CASE
}
template void launch_ell_spmm<double>(const EllDev<double>&, const double*, long long, double*, long long, int,
                                      double*, int, const DevState*, cudaStream_t);
template void launch_ell_spmm<float>(const EllDev<float>&, const float*, long long, float*, long long, int, double*,
                                     int, const DevState*, cudaStream_t);

template <typename T>
void launch_ell_residual(const EllDev<T>& A, const T* b, const T* x, T* r, double* part, int nblocks, cudaStream_t s,
                         const int* xnz) {
  k_ell_residual<T><<<nblocks, kBlock, 0, s>>>(A, b, x, r, part, xnz);
}

template <typename T>
void launch_ell_defect(const EllDev<T>& A, const T* b, const T* x, T* d, const DevState* state, cudaStream_t s) {
  (void)state;   // every problem of an algebraic hierarchy is the single problem 0
  k_ell_residual<T, false><<<ell_threads_blocks(A), kBlock, 0, s>>>(A, b, x, d, nullptr, nullptr);
}
template void launch_ell_defect<double>(const EllDev<double>&, const double*, const double*, double*, const DevState*,
                                        cudaStream_t);
template void launch_ell_defect<float>(const EllDev<float>&, const float*, const float*, float*, const DevState*,
                                       cudaStream_t);

template <typename T>
void launch_ell_spmv_add(const EllDev<T>& A, const T* X, T* Y, const DevState* state, cudaStream_t s) {
  k_ell_spmm<T, 1, false, true><<<ell_threads_blocks(A), kBlock, 0, s>>>(A, X, 0, Y, 0, nullptr, state);
}
template void launch_ell_spmv_add<double>(const EllDev<double>&, const double*, double*, const DevState*,
                                          cudaStream_t);
template void launch_ell_spmv_add<float>(const EllDev<float>&, const float*, float*, const DevState*, cudaStream_t);
template void launch_ell_residual<double>(const EllDev<double>&, const double*, const double*, double*, double*, int,
                                          cudaStream_t, const int*);
template void launch_ell_residual<float>(const EllDev<float>&, const float*, const float*, float*, double*, int,
                                         cudaStream_t, const int*);

template <typename T>
void launch_ell_jacobi(const EllDev<T>& A, const T* dinv, const T* g, const T* sin, T* out, int mode,
                       const DevState* state, cudaStream_t s) {
  k_ell_jacobi<T><<<ell_threads_blocks(A), kBlock, 0, s>>>(A, dinv, g, sin, out, mode, state);
}
template void launch_ell_jacobi<double>(const EllDev<double>&, const double*, const double*, const double*, double*,
                                        int, const DevState*, cudaStream_t);
template void launch_ell_jacobi<float>(const EllDev<float>&, const float*, const float*, const float*, float*, int,
                                       const DevState*, cudaStream_t);

// double-word instances (MPCG_FP64_DW)
template void launch_ell_spmm<dw>(const EllDev<dw>&, const dw*, long long, dw*, long long, int, double*, int,
                                  const DevState*, cudaStream_t);
template void launch_ell_defect<dw>(const EllDev<dw>&, const dw*, const dw*, dw*, const DevState*, cudaStream_t);
template void launch_ell_spmv_add<dw>(const EllDev<dw>&, const dw*, dw*, const DevState*, cudaStream_t);
template void launch_ell_residual<dw>(const EllDev<dw>&, const dw*, const dw*, dw*, double*, int, cudaStream_t,
                                      const int*);
template void launch_ell_jacobi<dw>(const EllDev<dw>&, const dw*, const dw*, const dw*, dw*, int, const DevState*,
                                    cudaStream_t);

}  // namespace mpcg
