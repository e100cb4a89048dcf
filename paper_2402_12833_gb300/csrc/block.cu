// Tall-skinny block kernels of the MPCG step (Section 2.2, Algorithm 1):
//   * the Gram blocks W_j = (A P_j)^T Z against the stored window,
//   * the A-orthogonalisation P = Z - sum_j P_j beta_j with the same
//     recurrence for A P, fused with the new Gram matrix sym(P^T A P) and
//     the right-hand side P^T r,
//   * the update x += P alpha, r -= A P alpha with ||r||^2.
//
// These kernels stream the padded arrays (pads are zero, so they take part
// harmlessly) in 16-byte vectors: 4 floats or 2 doubles per thread and step;
// blockIdx.y selects the problem of a batch (see common.cuh).
// Reductions are deterministic: every block writes its partial sums
// (value-major, fixed block count) and one small kernel adds them in a fixed
// order.  In the FP32 path each thread sums at most 64 points in FP32 and the
// warp adds its 32 lanes in FP32; everything above the warp is FP64.
#include "kernels.cuh"
#include "tune.h"
#include "vec.cuh"

namespace mpcg {

namespace {

// W_jj[a][b] = sum_i AP_slot(jj)[a][i] Z[b][i].  Block b works on window
// block jj = b % m and on the contiguous point chunk b / m, so that the
// blocks running together read the same chunk of Z (L2 reuse).
// double-word Gram: two blocks per SM (128 registers) without the software
// pipelining of the next point's loads (which needs 24 more registers)
constexpr bool kGramDwPrefetch = false;

template <typename T, int C>
__global__ void __launch_bounds__(kBlock, kIsDw<T> ? 2 : 3) k_gram_window(GridDesc g, Window<T> win, const T* __restrict__ Z,
                                                        double* part, int nchunks, const DevState* state) {
  const int pb = blockIdx.y;
  state += pb;
  if (state->done) return;
  const int m = state->m;
  const int jj = blockIdx.x % m, chunk = blockIdx.x / m;
  if (jj >= state->count) return;
  const int slot = (state->newest - jj + m) % m;
  const long long bo = (long long)pb * g.len + g.G;
  const T* AP = win.AP[slot] + bo;
  const T* Zb = Z + bo;
  // double-word: one point per thread and step (register pressure); the
  // group count per chunk follows the chunking of the vector width
  constexpr int VW = Vec<T>::W;
  constexpr int W = kIsDw<T> ? 1 : VW;
  const long long ngroups = g.npts / VW;
  const long long per = (ngroups + nchunks - 1) / nchunks;
  const long long g0 = (long long)chunk * per * (VW / W);
  const long long g1 = (g0 + per * (VW / W)) < ngroups * (VW / W) ? g0 + per * (VW / W) : ngroups * (VW / W);
  // the chunk count keeps every thread at <= 16 vector groups (64 points in
  // FP32) before its partial sums enter the reduction
  typename Acc<T>::type acc[C * C];
#pragma unroll
  for (int e = 0; e < C * C; ++e) acc[e] = Acc<T>::of(T(0));
  auto load_point = [&](long long q, T (&z)[C][W], T (&ap)[C][W]) {
    const long long i = q * W;
#pragma unroll
    for (int b = 0; b < C; ++b) VecN<T, W>::load_keep(Zb + (long long)b * g.cp + i, z[b]);
#pragma unroll
    for (int a = 0; a < C; ++a) VecN<T, W>::load(AP + (long long)a * g.cp + i, ap[a]);
  };
  auto accumulate = [&](const T (&z)[C][W], const T (&ap)[C][W]) {
#pragma unroll
    for (int a = 0; a < C; ++a)
#pragma unroll
      for (int b = 0; b < C; ++b)
#pragma unroll
        for (int w = 0; w < W; ++w) mac(acc[a * C + b], ap[a][w], z[b][w]);
  };
  if constexpr (kIsDw<T> && kGramDwPrefetch) {
    // the next point's loads are issued before the current point's products
    // (software pipelining)
    long long q = g0 + threadIdx.x;
    T z[C][W], ap[C][W];
    if (q < g1) load_point(q, z, ap);
    while (q < g1) {
      const long long qn = q + blockDim.x;
      T zn[C][W], apn[C][W];
      if (qn < g1) load_point(qn, zn, apn);
      accumulate(z, ap);
#pragma unroll
      for (int b = 0; b < C; ++b)
#pragma unroll
        for (int w = 0; w < W; ++w) {
          z[b][w] = zn[b][w];
          ap[b][w] = apn[b][w];
        }
      q = qn;
    }
  } else {
    for (long long q = g0 + threadIdx.x; q < g1; q += blockDim.x) {
      T z[C][W], ap[C][W];
      load_point(q, z, ap);
      accumulate(z, ap);
    }
  }
  T fin[C * C];
#pragma unroll
  for (int e = 0; e < C * C; ++e) fin[e] = Acc<T>::value(acc[e]);
  double* pj = part + ((long long)pb * m + jj) * C * C * nchunks;
  block_sum_store<T, C * C>(fin, pj, nchunks, chunk);
}

// Gram partials of one point group: G = sym(P^T A P) (upper triangle,
// p_a ap_b + p_b ap_a) and g = P^T r.
template <typename T, int C, int W>
__device__ __forceinline__ void gram_point(const T (&p)[C][W], const T (&ap)[C][W], const T* rp,
                                           typename Acc<T>::type (&acc)[C * (C + 1) / 2 + C]) {
  constexpr int NG = C * (C + 1) / 2;
  T rv[W];
  VecN<T, W>::load(rp, rv);
  int k = 0;
#pragma unroll
  for (int a = 0; a < C; ++a) {
#pragma unroll
    for (int b = a; b < C; ++b) {
#pragma unroll
      for (int w = 0; w < W; ++w) {
        mac(acc[k], p[a][w], ap[b][w]);
        mac(acc[k], p[b][w], ap[a][w]);
      }
      ++k;
    }
#pragma unroll
    for (int w = 0; w < W; ++w) mac(acc[NG + a], p[a][w], rv[w]);
  }
}

// In double-word arithmetic the Gram partials of the new block go to a
// second kernel (k_orth_gram_dw): without their 27 double-word accumulators
// the orthogonalisation fits 128 registers and two blocks per SM.
template <typename T, int C>
__global__ void __launch_bounds__(kBlock, 2) k_orth_update(GridDesc g, Window<T> win, const T* __restrict__ Z,
                                                        const T* __restrict__ AZ, const T* __restrict__ r,
                                                        double* part, const DevState* state) {
  const int pb = blockIdx.y;
  state += pb;
  if (state->done) return;
  const int cnt = state->count, m = state->m, newest = state->newest;
  const int ns = (newest + 1) % m;
  const long long bo = (long long)pb * g.len + g.G;
  __shared__ T beta[kMaxWindow][C][C];
  __shared__ const T* pp[kMaxWindow];
  __shared__ const T* app[kMaxWindow];
  for (int e = threadIdx.x; e < cnt * C * C; e += blockDim.x) {
    const int jj = e / (C * C), a = (e / C) % C, b = e % C;
    beta[jj][a][b] = (T)state->beta[jj][a][b];
  }
  for (int jj = threadIdx.x; jj < cnt; jj += blockDim.x) {
    const int slot = (newest - jj + m) % m;
    pp[jj] = win.P[slot] + bo;
    app[jj] = win.AP[slot] + bo;
  }
  __syncthreads();
  T* Pn = win.P[ns] + bo;
  T* APn = win.AP[ns] + bo;
  const T* Zb = Z + bo;
  const T* AZb = AZ + bo;
  const T* rb = r + bo;
  constexpr int W = kIsDw<T> ? 1 : Vec<T>::W;   // double-word: one point per thread (registers)
  constexpr bool kParts = !kIsDw<T>;             // Gram partials here, or in k_orth_gram_dw
  constexpr int NG = C * (C + 1) / 2;
  using A = typename Acc<T>::type;
  A acc[kParts ? NG + C : 1];
#pragma unroll
  for (int i = 0; i < (kParts ? NG + C : 1); ++i) acc[i] = Acc<T>::of(T(0));
  const long long ngroups = g.npts / W;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = q * W;
    A pacc[C][W], apacc[C][W];
#pragma unroll
    for (int b = 0; b < C; ++b) {
      T zv[W], azv[W];
      VecN<T, W>::load(Zb + (long long)b * g.cp + i, zv);
      VecN<T, W>::load(AZb + (long long)b * g.cp + i, azv);
#pragma unroll
      for (int w = 0; w < W; ++w) {
        pacc[b][w] = Acc<T>::of(zv[w]);
        apacc[b][w] = Acc<T>::of(azv[w]);
      }
    }
    auto load_block = [&](int jj, T (&pa)[C][W], T (&apa)[C][W]) {
#pragma unroll
      for (int a = 0; a < C; ++a) {
        VecN<T, W>::load(pp[jj] + (long long)a * g.cp + i, pa[a]);
        VecN<T, W>::load(app[jj] + (long long)a * g.cp + i, apa[a]);
      }
    };
    auto apply_block = [&](int jj, const T (&pa)[C][W], const T (&apa)[C][W]) {
#pragma unroll
      for (int a = 0; a < C; ++a)
#pragma unroll
        for (int b = 0; b < C; ++b) {
          const T bt = beta[jj][a][b];
#pragma unroll
          for (int w = 0; w < W; ++w) {
            mac(pacc[b][w], -pa[a][w], bt);
            mac(apacc[b][w], -apa[a][w], bt);
          }
        }
    };
    if constexpr (kIsDw<T>) {
      // few warps per SM in double-word: block jj + 1 is loaded while
      // block jj's products run (software pipelining)
      T pa[C][W], apa[C][W];
      if (cnt > 0) load_block(0, pa, apa);
      for (int jj = 0; jj < cnt; ++jj) {
        T pn[C][W], apn[C][W];
        if (jj + 1 < cnt) load_block(jj + 1, pn, apn);
        apply_block(jj, pa, apa);
#pragma unroll
        for (int a = 0; a < C; ++a)
#pragma unroll
          for (int w = 0; w < W; ++w) {
            pa[a][w] = pn[a][w];
            apa[a][w] = apn[a][w];
          }
      }
    } else {
      for (int jj = 0; jj < cnt; ++jj) {
        T pa[C][W], apa[C][W];
        load_block(jj, pa, apa);
        apply_block(jj, pa, apa);
      }
    }
    T p[C][W], ap[C][W];
#pragma unroll
    for (int b = 0; b < C; ++b)
#pragma unroll
      for (int w = 0; w < W; ++w) {
        p[b][w] = Acc<T>::value(pacc[b][w]);
        ap[b][w] = Acc<T>::value(apacc[b][w]);
      }
#pragma unroll
    for (int a = 0; a < C; ++a) {
      VecN<T, W>::store(Pn + (long long)a * g.cp + i, p[a]);
      VecN<T, W>::store(APn + (long long)a * g.cp + i, ap[a]);
    }
    if constexpr (kParts) gram_point<T, C, W>(p, ap, rb + i, acc);
  }
  if constexpr (kParts) {
    T fin[NG + C];
#pragma unroll
    for (int i = 0; i < NG + C; ++i) fin[i] = Acc<T>::value(acc[i]);
    block_sum_store<T, NG + C>(fin, part + (long long)pb * (NG + C) * gridDim.x, gridDim.x, blockIdx.x);
  }
}

// The Gram partials of the new block, double-word: the same points per
// thread and the same order as the fused FP32 / FP64 kernels (same grid).
template <int C>
__global__ void __launch_bounds__(kBlock, 2) k_orth_gram_dw(GridDesc g, Window<dw> win, const dw* __restrict__ r,
                                                             double* part, const DevState* state) {
  const int pb = blockIdx.y;
  state += pb;
  if (state->done) return;
  const int ns = (state->newest + 1) % state->m;
  const long long bo = (long long)pb * g.len + g.G;
  const dw* Pn = win.P[ns] + bo;
  const dw* APn = win.AP[ns] + bo;
  constexpr int NG = C * (C + 1) / 2;
  dwacc acc[NG + C];
#pragma unroll
  for (int i = 0; i < NG + C; ++i) acc[i] = dwacc_of(dw(0));
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < g.npts;
       q += (long long)gridDim.x * blockDim.x) {
    dw p[C][1], ap[C][1];
#pragma unroll
    for (int a = 0; a < C; ++a) {
      VecN<dw, 1>::load(Pn + (long long)a * g.cp + q, p[a]);
      VecN<dw, 1>::load(APn + (long long)a * g.cp + q, ap[a]);
    }
    gram_point<dw, C, 1>(p, ap, r + bo + q, acc);
  }
  dw fin[NG + C];
#pragma unroll
  for (int i = 0; i < NG + C; ++i) fin[i] = dwacc_value(acc[i]);
  block_sum_store<dw, NG + C>(fin, part + (long long)pb * (NG + C) * gridDim.x, gridDim.x, blockIdx.x);
}

template <typename T, int C>
__global__ void __launch_bounds__(kBlock) k_update_xr(GridDesc g, Window<T> win, T* __restrict__ x,
                                                      T* __restrict__ r, double* part, const DevState* state) {
  const int pb = blockIdx.y;
  state += pb;
  if (state->done) return;
  const int newest = state->newest;
  const long long bo = (long long)pb * g.len + g.G;
  const T* P = win.P[newest] + bo;
  const T* AP = win.AP[newest] + bo;
  T* xb = x + bo;
  T* rb = r + bo;
  T al[C];
#pragma unroll
  for (int a = 0; a < C; ++a) al[a] = (T)state->alpha[a];
  constexpr int W = Vec<T>::W;
  T acc[1] = {0};
  const long long ngroups = g.npts / W;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = q * W;
    T px[W] = {}, apx[W] = {};
#pragma unroll
    for (int a = 0; a < C; ++a) {
      T pv[W], av[W];
      Vec<T>::load(P + (long long)a * g.cp + i, pv);
      Vec<T>::load(AP + (long long)a * g.cp + i, av);
#pragma unroll
      for (int w = 0; w < W; ++w) {
        px[w] = fma(pv[w], al[a], px[w]);
        apx[w] = fma(av[w], al[a], apx[w]);
      }
    }
    T xv[W], rv[W];
    Vec<T>::load_keep(xb + i, xv);
    Vec<T>::load_keep(rb + i, rv);
#pragma unroll
    for (int w = 0; w < W; ++w) {
      xv[w] += px[w];
      rv[w] -= apx[w];
      acc[0] = fma(rv[w], rv[w], acc[0]);
    }
    Vec<T>::store(xb + i, xv);
    Vec<T>::store(rb + i, rv);
  }
  block_sum_store<T, 1>(acc, part + (long long)pb * gridDim.x, gridDim.x, blockIdx.x);
}

// Mixed-precision refinement, start of an inner FP32 solve: with the outer
// residual r64 and |r64|^2 in nrm2[2p], b32 = r64 / |r64| (zero for an
// inactive problem, whose inner solve then stops at once).  The inner iterate
// starts at zero, so the inner residual is b32 itself: it is written to r32
// as well, with the block partials of |r32|^2 and |b32|^2 that the residual
// kernel would have produced (value-major, stride gridDim.x).
__global__ void __launch_bounds__(kBlock) k_start_inner(GridDesc g, const double* __restrict__ r64,
                                                        const double* __restrict__ nrm2,
                                                        const int* __restrict__ active, float* __restrict__ b32,
                                                        float* __restrict__ r32, double* part) {
  const int pb = blockIdx.y;
  const bool on = !active || active[pb];
  const double inv = on && nrm2[2 * pb] > 0.0 ? 1.0 / sqrt(nrm2[2 * pb]) : 0.0;
  const long long o = (long long)pb * g.len + g.G;
  float sums[2] = {0.f, 0.f};
  const long long ngroups = g.npts / 4;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = o + q * 4;
    double lo[2], hi[2];
    Vec<double>::load(r64 + i, lo);
    Vec<double>::load(r64 + i + 2, hi);
    const float v[4] = {(float)(lo[0] * inv), (float)(lo[1] * inv), (float)(hi[0] * inv), (float)(hi[1] * inv)};
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      sums[0] = fmaf(v[w], v[w], sums[0]);
      sums[1] = fmaf(v[w], v[w], sums[1]);
    }
    Vec<float>::store(b32 + i, v);
    Vec<float>::store(r32 + i, v);
  }
  block_sum_store<float, 2>(sums, part + (long long)pb * 2 * gridDim.x, gridDim.x, blockIdx.x);
}

// End of an inner solve: x64 += |r64| d32 (nrm2[2p] = |r64|^2).
__global__ void __launch_bounds__(kBlock) k_axpy_mixed(GridDesc g, double* __restrict__ x,
                                                       const float* __restrict__ d, const double* __restrict__ nrm2,
                                                       int* xnz) {
  const int pb = blockIdx.y;
  const double sc = sqrt(nrm2[2 * pb]);
  if (xnz && blockIdx.x == 0 && threadIdx.x == 0) xnz[pb] = 1;   // x may be nonzero from here on
  const long long o = (long long)pb * g.len + g.G;
  const long long ngroups = g.npts / 4;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    const long long i = o + q * 4;
    float dv[4];
    double lo[2], hi[2];
    Vec<float>::load(d + i, dv);
    Vec<double>::load_keep(x + i, lo);
    Vec<double>::load_keep(x + i + 2, hi);
    lo[0] = fma(sc, (double)dv[0], lo[0]);
    lo[1] = fma(sc, (double)dv[1], lo[1]);
    hi[0] = fma(sc, (double)dv[2], hi[0]);
    hi[1] = fma(sc, (double)dv[3], hi[1]);
    Vec<double>::store(x + i, lo);
    Vec<double>::store(x + i + 2, hi);
  }
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

int gram_chunks_default(const GridDesc& g) {
  // 8 vector groups (32 points in FP32, 16 in FP64) per thread and chunk
  const long long groups = g.npts / 4;
  long long c = (groups + kBlock * 8 - 1) / (kBlock * 8);
  if (c < 1) c = 1;
  return (int)(c < kGramChunksMax ? c : kGramChunksMax);
}
// at most 16 vector groups (64 FP32 points) per thread and chunk
int gram_chunks_min(const GridDesc& g) { return (gram_chunks_default(g) + 1) / 2; }
int gram_chunks_cap(const GridDesc& g) {
  const long long c = 4LL * gram_chunks_default(g);
  return (int)(c < kGramChunksMax ? c : kGramChunksMax);
}
int gram_chunks(const GridDesc& g) {
  const int v = tune::lookup(tune::kGram, tune::kAny, g.npts, g.nb, 0, gram_chunks_default(g));
  const int lo = gram_chunks_min(g), hi = gram_chunks_cap(g);
  return v < lo ? lo : (v > hi ? hi : v);
}

int stream_blocks_min(const GridDesc& g) {
  const long long groups = g.npts / 2;
  long long need = (groups + kBlock * 16 - 1) / (kBlock * 16);   // <= 64 points per thread
  if (need < 1) need = 1;
  return (int)(need < kStreamBlocksMax ? need : kStreamBlocksMax);
}
int stream_blocks_default(const GridDesc& g) {
  const long long groups = g.npts / 2;
  long long need = stream_blocks_min(g);
  long long fill = (groups + kBlock - 1) / kBlock;                // no idle threads
  long long nb = kStreamBlocks < fill ? kStreamBlocks : fill;
  if (need > nb) nb = need;
  if (nb < 1) nb = 1;
  return (int)(nb < kStreamBlocksMax ? nb : kStreamBlocksMax);
}
// the most blocks the tuner may choose (and the reduction buffers reserve):
// eight per SM, without idle threads
int stream_blocks_cap(const GridDesc& g) {
  const long long groups = g.npts / 2;
  const long long fill = (groups + kBlock - 1) / kBlock;
  long long c = 8LL * (sm_count() > 0 ? sm_count() : 152);
  if (c > fill) c = fill;
  const long long d = stream_blocks_default(g);
  if (c < d) c = d;
  return (int)(c < kStreamBlocksMax ? c : kStreamBlocksMax);
}
int stream_blocks(const GridDesc& g) {
  const int v = tune::lookup(tune::kStream, tune::kAny, g.npts, g.nb, 0, stream_blocks_default(g));
  const int lo = stream_blocks_min(g), hi = stream_blocks_cap(g);
  return v < lo ? lo : (v > hi ? hi : v);
}

template <typename T>
void launch_gram_window(const GridDesc& g, Window<T> win, const T* Z, int C, int m, double* part,
                        const DevState* state, cudaStream_t s) {
  const int nch = gram_chunks(g);
  MPCG_C_SWITCH(C, (k_gram_window<T, CC><<<dim3(nch * m, g.nb), kBlock, 0, s>>>(g, win, Z, part, nch, state)));
}

template <typename T>
void launch_orth_update(const GridDesc& g, Window<T> win, const T* Z, const T* AZ, const T* r, int C, double* part,
                        const DevState* state, cudaStream_t s) {
  const int nb = stream_blocks(g);
  MPCG_C_SWITCH(C, (k_orth_update<T, CC><<<dim3(nb, g.nb), kBlock, 0, s>>>(g, win, Z, AZ, r, part, state)));
}

void launch_orth_gram_dw(const GridDesc& g, Window<dw> win, const dw* r, int C, double* part, const DevState* state,
                         cudaStream_t s) {
  const int nb = stream_blocks(g);
  MPCG_C_SWITCH(C, (k_orth_gram_dw<CC><<<dim3(nb, g.nb), kBlock, 0, s>>>(g, win, r, part, state)));
}

template <typename T>
void launch_update_xr(const GridDesc& g, Window<T> win, T* x, T* r, int C, double* part, const DevState* state,
                      cudaStream_t s) {
  const int nb = stream_blocks(g);
  MPCG_C_SWITCH(C, (k_update_xr<T, CC><<<dim3(nb, g.nb), kBlock, 0, s>>>(g, win, x, r, part, state)));
}

void launch_start_inner(const GridDesc& g, const double* r64, const double* nrm2, const int* active, float* b32,
                        float* r32, double* part, cudaStream_t s) {
  k_start_inner<<<dim3(stream_blocks(g), g.nb), kBlock, 0, s>>>(g, r64, nrm2, active, b32, r32, part);
}
void launch_axpy_mixed(const GridDesc& g, double* x, const float* d, const double* scale, int* xnz,
                       cudaStream_t s) {
  k_axpy_mixed<<<dim3(stream_blocks(g), g.nb), kBlock, 0, s>>>(g, x, d, scale, xnz);
}

template void launch_gram_window<double>(const GridDesc&, Window<double>, const double*, int, int, double*,
                                         const DevState*, cudaStream_t);
template void launch_gram_window<float>(const GridDesc&, Window<float>, const float*, int, int, double*,
                                        const DevState*, cudaStream_t);
template void launch_orth_update<double>(const GridDesc&, Window<double>, const double*, const double*,
                                         const double*, int, double*, const DevState*, cudaStream_t);
template void launch_orth_update<float>(const GridDesc&, Window<float>, const float*, const float*, const float*,
                                        int, double*, const DevState*, cudaStream_t);
template void launch_update_xr<double>(const GridDesc&, Window<double>, double*, double*, int, double*,
                                       const DevState*, cudaStream_t);
template void launch_update_xr<float>(const GridDesc&, Window<float>, float*, float*, int, double*,
                                      const DevState*, cudaStream_t);
template void launch_gram_window<dw>(const GridDesc&, Window<dw>, const dw*, int, int, double*, const DevState*,
                                     cudaStream_t);
template void launch_orth_update<dw>(const GridDesc&, Window<dw>, const dw*, const dw*, const dw*, int, double*,
                                     const DevState*, cudaStream_t);
template void launch_update_xr<dw>(const GridDesc&, Window<dw>, dw*, dw*, int, double*, const DevState*,
                                   cudaStream_t);

}  // namespace mpcg
