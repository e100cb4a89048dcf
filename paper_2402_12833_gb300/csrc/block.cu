// Tall-skinny block kernels of the MPCG step (Section 2.2, Algorithm 1):
//   * the Gram blocks (A P_j)^T Z against the stored window,
//   * the A-orthogonalisation P = Z - sum_j P_j beta_j with the same
//     recurrence for A P, fused with the new Gram matrix sym(P^T A P) and
//     the right-hand side P^T r,
//   * the update x += P alpha, r -= A P alpha with ||r||^2.
//
// Reductions are deterministic: every block writes its partial sums
// (value-major, fixed block count) and one small kernel adds them in a fixed
// order.  Partial sums accumulate in FP64; in the FP32 path each thread first
// sums its own products in FP32 over a short run (at most 16 products per
// value in the Gram kernel, the points of one grid-stride sweep elsewhere).
#include "kernels.cuh"

namespace mpcg {

namespace {

template <int NV>
__device__ __forceinline__ void block_sum_store(double (&v)[NV], double* part, int stride) {
  __shared__ double sh[kBlock / 32][NV];
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

constexpr int kTD = 16;   // points per shared-memory tile of the Gram kernel

template <typename T, int C>
__global__ void __launch_bounds__(kBlock) k_gram_window(GridDesc g, Window<T> win, const T* __restrict__ Z,
                                                        double* part, const DevState* state) {
  if (state->done) return;
  const int cnt = state->count;
  if (cnt == 0) return;
  const int m = state->m, newest = state->newest;
  const int nx = cnt * C;
  constexpr int kMaxE = (kMaxWindow * C * C + kBlock - 1) / kBlock;
  __shared__ T Xs[kMaxWindow * C][kTD];
  __shared__ T Ys[C][kTD];
  __shared__ const T* rowp[kMaxWindow * C];
  for (int r = threadIdx.x; r < nx; r += blockDim.x) {
    const int jj = r / C, a = r % C;
    const int slot = (newest - jj + m) % m;
    rowp[r] = win.AP[slot] + (long long)a * g.len + g.G;
  }
  double acc[kMaxE];
#pragma unroll
  for (int q = 0; q < kMaxE; ++q) acc[q] = 0.0;
  __syncthreads();
  const long long ntiles = (g.npts + kTD - 1) / kTD;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const long long base = tile * kTD;
    for (int e = threadIdx.x; e < (nx + C) * kTD; e += blockDim.x) {
      const int r = e / kTD, d = e % kTD;
      const long long i = base + d;
      if (r < nx) Xs[r][d] = i < g.npts ? rowp[r][i] : (T)0;
      else Ys[r - nx][d] = i < g.npts ? Z[(long long)(r - nx) * g.len + g.G + i] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxE; ++q) {
      const int e = threadIdx.x + q * kBlock;
      if (e < nx * C) {
        const int r = e / C, b = e % C;
        T s = 0;
#pragma unroll
        for (int d = 0; d < kTD; ++d) s = fma(Xs[r][d], Ys[b][d], s);
        acc[q] += (double)s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kMaxE; ++q) {
    const int e = threadIdx.x + q * kBlock;
    if (e < nx * C) part[(long long)e * kGramBlocks + blockIdx.x] = acc[q];
  }
}

template <typename T, int C>
__global__ void __launch_bounds__(kBlock) k_orth_update(GridDesc g, Window<T> win, const T* __restrict__ Z,
                                                        const T* __restrict__ AZ, const T* __restrict__ r,
                                                        double* part, const DevState* state) {
  if (state->done) return;
  const int cnt = state->count, m = state->m, newest = state->newest;
  const int ns = (newest + 1) % m;
  __shared__ T beta[kMaxWindow][C][C];
  __shared__ const T* pp[kMaxWindow];
  __shared__ const T* app[kMaxWindow];
  for (int e = threadIdx.x; e < cnt * C * C; e += blockDim.x) {
    const int jj = e / (C * C), a = (e / C) % C, b = e % C;
    beta[jj][a][b] = (T)state->beta[jj][a][b];
  }
  for (int jj = threadIdx.x; jj < cnt; jj += blockDim.x) {
    const int slot = (newest - jj + m) % m;
    pp[jj] = win.P[slot];
    app[jj] = win.AP[slot];
  }
  __syncthreads();
  T* Pn = win.P[ns];
  T* APn = win.AP[ns];
  constexpr int NG = C * (C + 1) / 2;
  T acc[NG + C];
#pragma unroll
  for (int i = 0; i < NG + C; ++i) acc[i] = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    const long long idx = g.G + t;
    T p[C], ap[C];
#pragma unroll
    for (int b = 0; b < C; ++b) {
      p[b] = Z[(long long)b * g.len + idx];
      ap[b] = AZ[(long long)b * g.len + idx];
    }
    for (int jj = 0; jj < cnt; ++jj) {
      const T* Pj = pp[jj];
      const T* APj = app[jj];
#pragma unroll
      for (int a = 0; a < C; ++a) {
        const T pa = Pj[(long long)a * g.len + idx];
        const T apa = APj[(long long)a * g.len + idx];
#pragma unroll
        for (int b = 0; b < C; ++b) {
          p[b] = fma(-pa, beta[jj][a][b], p[b]);
          ap[b] = fma(-apa, beta[jj][a][b], ap[b]);
        }
      }
    }
    const T rv = r[idx];
    int k = 0;
#pragma unroll
    for (int a = 0; a < C; ++a) {
      Pn[(long long)a * g.len + idx] = p[a];
      APn[(long long)a * g.len + idx] = ap[a];
#pragma unroll
      for (int b = a; b < C; ++b) {
        acc[k] = fma(p[a], ap[b], acc[k]);
        acc[k] = fma(p[b], ap[a], acc[k]);
        ++k;
      }
      acc[NG + a] = fma(p[a], rv, acc[NG + a]);
    }
  }
  double accd[NG + C];
#pragma unroll
  for (int i = 0; i < NG + C; ++i) accd[i] = (double)acc[i];
  block_sum_store<NG + C>(accd, part, kRedBlocks);
}

template <typename T, int C>
__global__ void __launch_bounds__(kBlock) k_update_xr(GridDesc g, Window<T> win, T* __restrict__ x,
                                                      T* __restrict__ r, double* part, const DevState* state) {
  if (state->done) return;
  const int newest = state->newest;
  const T* P = win.P[newest];
  const T* AP = win.AP[newest];
  T al[C];
#pragma unroll
  for (int a = 0; a < C; ++a) al[a] = (T)state->alpha[a];
  T acc = 0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    const long long idx = g.G + t;
    T px = 0, apx = 0;
#pragma unroll
    for (int a = 0; a < C; ++a) {
      px = fma(P[(long long)a * g.len + idx], al[a], px);
      apx = fma(AP[(long long)a * g.len + idx], al[a], apx);
    }
    x[idx] += px;
    const T rv = r[idx] - apx;
    r[idx] = rv;
    acc = fma(rv, rv, acc);
  }
  double v[1] = {(double)acc};
  block_sum_store<1>(v, part, kRedBlocks);
}

}  // namespace

#define MPCG_C_SWITCH(C, BODY)                                                                   \
  switch (C) {                                                                                   \
    case 1: { constexpr int CC = 1; BODY; } break;                                               \
    case 2: { constexpr int CC = 2; BODY; } break;                                               \
    case 3: { constexpr int CC = 3; BODY; } break;                                               \
    case 4: { constexpr int CC = 4; BODY; } break;                                               \
    case 5: { constexpr int CC = 5; BODY; } break;                                               \
    case 6: { constexpr int CC = 6; BODY; } break;                                               \
    case 7: { constexpr int CC = 7; BODY; } break;                                               \
    case 8: { constexpr int CC = 8; BODY; } break;                                               \
    case 9: { constexpr int CC = 9; BODY; } break;                                               \
    case 10: { constexpr int CC = 10; BODY; } break;                                             \
    case 11: { constexpr int CC = 11; BODY; } break;                                             \
    case 12: { constexpr int CC = 12; BODY; } break;                                             \
    default: break;                                                                              \
  }

template <typename T>
void launch_gram_window(const GridDesc& g, Window<T> win, const T* Z, int C, double* part, const DevState* state,
                        cudaStream_t s) {
  const int nb = kGramBlocks;
  MPCG_C_SWITCH(C, (k_gram_window<T, CC><<<nb, kBlock, 0, s>>>(g, win, Z, part, state)));
}

template <typename T>
void launch_orth_update(const GridDesc& g, Window<T> win, const T* Z, const T* AZ, const T* r, int C, double* part,
                        const DevState* state, cudaStream_t s) {
  const int nb = kRedBlocks;
  MPCG_C_SWITCH(C, (k_orth_update<T, CC><<<nb, kBlock, 0, s>>>(g, win, Z, AZ, r, part, state)));
}

template <typename T>
void launch_update_xr(const GridDesc& g, Window<T> win, T* x, T* r, int C, double* part, const DevState* state,
                      cudaStream_t s) {
  const int nb = kRedBlocks;
  MPCG_C_SWITCH(C, (k_update_xr<T, CC><<<nb, kBlock, 0, s>>>(g, win, x, r, part, state)));
}

template void launch_gram_window<double>(const GridDesc&, Window<double>, const double*, int, double*,
                                         const DevState*, cudaStream_t);
template void launch_gram_window<float>(const GridDesc&, Window<float>, const float*, int, double*,
                                        const DevState*, cudaStream_t);
template void launch_orth_update<double>(const GridDesc&, Window<double>, const double*, const double*,
                                         const double*, int, double*, const DevState*, cudaStream_t);
template void launch_orth_update<float>(const GridDesc&, Window<float>, const float*, const float*, const float*,
                                        int, double*, const DevState*, cudaStream_t);
template void launch_update_xr<double>(const GridDesc&, Window<double>, double*, double*, int, double*,
                                       const DevState*, cudaStream_t);
template void launch_update_xr<float>(const GridDesc&, Window<float>, float*, float*, int, double*,
                                      const DevState*, cudaStream_t);

}  // namespace mpcg
