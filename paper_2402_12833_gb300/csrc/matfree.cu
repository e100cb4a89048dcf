// Matrix-free fine-grid operator of the Q1 diffusion problem (Section 1's
// model problem, -div(kappa grad u) with kappa constant on each element),
// the matrix-free direction the paper names as future work (Section 4):
// instead of streaming 27 stored coefficients per unknown, the FP32 kernels
// of the inner solve rebuild each row from the coefficients of the 8
// elements around the node.
//
// 3D Q1 hexahedron of side h: the element stiffness entry between two of its
// nodes depends only on how many coordinates differ: h/3 (same node), 0
// (one), -h/12 (two or three).  Hence, with k_e = -(h/12) kappa_e:
//   centre           -4 * (sum of the 8 k_e around the node)
//   face neighbour    0
//   edge neighbour    sum of the 2 k_e sharing that edge
//   corner neighbour  the 1 k_e sharing that corner.
// 2D Q1 square: 4/6, -1/6, -2/6 for 0, 1, 2 differing coordinates
// (independent of h); with k_e = -kappa_e / 6: centre -4 * (sum of the 4
// k_e), edge neighbour the sum of the 2 k_e sharing the edge, corner twice
// the 1 k_e sharing it (all 9 couplings non-zero).
// k is stored in the padded node layout at the element's lowest node
// (unknown coordinates -1 .. n-1 per axis; the -1 entries sit in pads and
// guards, see common.cuh), zero for elements outside the domain.  Couplings
// to eliminated Dirichlet nodes multiply pad entries of X (zero), and the
// outputs at pad points are set to zero, so the result equals the stored
// operator's.
#include <string.h>

#include "kernels.cuh"
#include "vec.cuh"

namespace mpcg {

namespace {

// k_e of element e (lowest node: global node (ex, ey[, ez])) of problem
// blockIdx.y at its padded slot.
__global__ void k_place_kappa(GridDesc g, const double* __restrict__ kappa, int ne, double scale,
                              float* __restrict__ k32, double* __restrict__ k64) {
  const int pb = blockIdx.y;
  const long long n = g.dim == 3 ? (long long)ne * ne * ne : (long long)ne * ne;
  kappa += (long long)pb * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(e % ne), ey = (int)((e / ne) % ne), ez = g.dim == 3 ? (int)(e / ((long long)ne * ne)) : 0;
    const long long i = (long long)pb * g.len + g.G + (long long)(ex - g.lox) + (long long)(ey - g.loy) * g.px +
                        (g.dim == 3 ? (long long)(ez - g.loz) * g.pxy : 0);
    const double k = scale * kappa[e];
    k64[i] = k;
    k32[i] = (float)k;
  }
}

// Largest |a_stored - a_kappa| and |a_stored| over the couplings between
// unknowns (FP64) of problem blockIdx.y, as order-preserving bit patterns of
// non-negative doubles.
__global__ void k_check_kappa(GridDesc g, const double* __restrict__ st, const double* __restrict__ k64,
                              unsigned long long* out) {
  const int pb = blockIdx.y;
  const int S = g.dim == 3 ? 27 : 9;
  double dmax = 0.0, amax = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    int x, y, z, a;
    decode(g, t, x, y, z, a);
    if (!interior(g, x, y, z)) continue;
    const long long i = (long long)pb * g.len + g.G + t;
    for (int s = 0; s < S; ++s) {
      const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = g.dim == 3 ? s / 9 - 1 : 0;
      const int qx = x + dx, qy = y + dy, qz = z + dz;
      if (qx < 0 || qy < 0 || qx >= g.nx || qy >= g.ny) continue;
      if (g.dim == 3 && (qz < 0 || qz >= g.nz)) continue;
      const int nd = (dx != 0) + (dy != 0) + (dz != 0);
      double sum = 0.0;   // k_e over the elements holding both nodes
      for (int c = (g.dim == 3 ? 0 : 1); c < 2; ++c) {
        if ((dz < 0 && c == 1) || (dz > 0 && c == 0)) continue;
        for (int b = 0; b < 2; ++b) {
          if ((dy < 0 && b == 1) || (dy > 0 && b == 0)) continue;
          for (int e = 0; e < 2; ++e) {
            if ((dx < 0 && e == 1) || (dx > 0 && e == 0)) continue;
            sum += k64[i + (e - 1) + (long long)(b - 1) * g.px + (g.dim == 3 ? (long long)(c - 1) * g.pxy : 0)];
          }
        }
      }
      double ak;
      if (nd == 0) ak = -4.0 * sum;
      else if (g.dim == 3) ak = nd == 1 ? 0.0 : sum;
      else ak = nd == 1 ? sum : 2.0 * sum;
      const double as = st[(long long)s * g.cp + i];
      dmax = fmax(dmax, fabs(as - ak));
      amax = fmax(amax, fabs(as));
    }
  }
  atomicMax(out, (unsigned long long)__double_as_longlong(dmax));
  atomicMax(out + 1, (unsigned long long)__double_as_longlong(amax));
}

// Row segment v[-1 .. 4] around a group of four points: e[k] = v[k - 1].
__device__ __forceinline__ void row6(const float* __restrict__ p, float (&e)[6]) {
  float m[4];
  Vec<float>::load_keep(p, m);
  e[0] = p[-1];
#pragma unroll
  for (int w = 0; w < 4; ++w) e[w + 1] = m[w];
  e[5] = p[4];
}

// k_e of the 8 elements around the points x0 .. x0+3 of a group:
// kq[2b + c][k] for the element whose lowest node is (x0 - 1 + k, y - 1 + b,
// z - 1 + c).
__device__ __forceinline__ void load_kappa(const float* __restrict__ k32, long long idx, long long px, long long pxy,
                                           float (&kq)[4][5]) {
#pragma unroll
  for (int b = 0; b < 2; ++b)
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const float* p = k32 + idx + (long long)(b - 1) * px + (long long)(c - 1) * pxy;
      float m[4];
      Vec<float>::load_keep(p, m);
      kq[2 * b + c][0] = p[-1];
#pragma unroll
      for (int w = 0; w < 4; ++w) kq[2 * b + c][w + 1] = m[w];
    }
}

// Coefficients of stencil row (DY, DZ) for the four points: cf[dx + 1][w].
template <int DY, int DZ>
__device__ __forceinline__ void row_coefs(const float (&kq)[4][5], float (&cf)[3][4]) {
  constexpr int b = DY > 0, c = DZ > 0;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    if (DY == 0 && DZ == 0) {
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) s += kq[q][w] + kq[q][w + 1];
      cf[0][w] = 0.f;
      cf[1][w] = -4.f * s;
      cf[2][w] = 0.f;
    } else if (DZ == 0) {   // edges (+-1, DY, 0); face (0, DY, 0)
      cf[0][w] = kq[2 * b][w] + kq[2 * b + 1][w];
      cf[1][w] = 0.f;
      cf[2][w] = kq[2 * b][w + 1] + kq[2 * b + 1][w + 1];
    } else if (DY == 0) {   // edges (+-1, 0, DZ); face (0, 0, DZ)
      cf[0][w] = kq[c][w] + kq[2 + c][w];
      cf[1][w] = 0.f;
      cf[2][w] = kq[c][w + 1] + kq[2 + c][w + 1];
    } else {                // corners (+-1, DY, DZ); edge (0, DY, DZ)
      cf[0][w] = kq[2 * b + c][w];
      cf[1][w] = kq[2 * b + c][w] + kq[2 * b + c][w + 1];
      cf[2][w] = kq[2 * b + c][w + 1];
    }
  }
}

template <int DY, int DZ, int C>
__device__ __forceinline__ void apply_row(const float (&kq)[4][5], const float* __restrict__ X, long long pitch,
                                          long long idx, long long px, long long pxy, float (&acc)[C][4]) {
  float cf[3][4];
  row_coefs<DY, DZ>(kq, cf);
  const long long ro = (long long)DY * px + (long long)DZ * pxy;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    if (DY == 0 && DZ == 0) {   // the centre only
      float m[4];
      Vec<float>::load_keep(X + (long long)c * pitch + idx, m);
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[c][w] = fmaf(cf[1][w], m[w], acc[c][w]);
    } else {
      float e[6];
      row6(X + (long long)c * pitch + idx + ro, e);
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        acc[c][w] = fmaf(cf[0][w], e[w], acc[c][w]);
        if (DY != 0 && DZ != 0) acc[c][w] = fmaf(cf[1][w], e[w + 1], acc[c][w]);
        acc[c][w] = fmaf(cf[2][w], e[w + 2], acc[c][w]);
      }
    }
  }
}

template <int C>
__device__ __forceinline__ void mf_group(const float (&kq)[4][5], const float* __restrict__ X, long long pitch,
                                         long long idx, long long px, long long pxy, float (&acc)[C][4]) {
  apply_row<-1, -1, C>(kq, X, pitch, idx, px, pxy, acc);
  apply_row<0, -1, C>(kq, X, pitch, idx, px, pxy, acc);
  apply_row<1, -1, C>(kq, X, pitch, idx, px, pxy, acc);
  apply_row<-1, 0, C>(kq, X, pitch, idx, px, pxy, acc);
  apply_row<0, 0, C>(kq, X, pitch, idx, px, pxy, acc);
  apply_row<1, 0, C>(kq, X, pitch, idx, px, pxy, acc);
  apply_row<-1, 1, C>(kq, X, pitch, idx, px, pxy, acc);
  apply_row<0, 1, C>(kq, X, pitch, idx, px, pxy, acc);
  apply_row<1, 1, C>(kq, X, pitch, idx, px, pxy, acc);
}

// Y = A X over C columns (+ partials of z_c^T A z_c), A from k.
template <int C>
__global__ void __launch_bounds__(kBlock, 3) k_spmm_mf(GridDesc g, const float* __restrict__ k32,
                                                    const float* __restrict__ X, float* __restrict__ Y, double* zaz,
                                                    const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  float zacc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) zacc[c] = 0.f;
  const long long ngroups = g.npts / 4;
  const long long bo = (long long)pb * g.len + g.G;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    int x0, y, z, a;
    decode(g, q * 4, x0, y, z, a);
    const long long idx = bo + q * 4;
    const bool row_in = y < g.ny && z < g.nz;
    float kq[4][5];
    load_kappa(k32, idx, g.px, g.pxy, kq);
    float acc[C][4];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[c][w] = 0.f;
    mf_group<C>(kq, X, g.cp, idx, g.px, g.pxy, acc);
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
      for (int w = 0; w < 4; ++w)
        if (!row_in || x0 + w >= g.nx) acc[c][w] = 0.f;   // pad points: zero rows
      Vec<float>::store(Y + (long long)c * g.cp + idx, acc[c]);
      if (zaz) {
        float xc[4];
        Vec<float>::load_keep(X + (long long)c * g.cp + idx, xc);
#pragma unroll
        for (int w = 0; w < 4; ++w) zacc[c] = fmaf(xc[w], acc[c][w], zacc[c]);
      }
    }
  }
  if (zaz) block_sum_store<float, C>(zacc, zaz + (long long)pb * C * gridDim.x, gridDim.x, blockIdx.x);
}

// Two damped-Jacobi sweeps from zero on the fine grid, fused (as k_jacobi
// mode 1): s1 = dinv r, s = s1 + dinv (r - A s1), A from k; dinv (stored)
// is omega / diagonal, zero at pads.
__global__ void __launch_bounds__(kBlock, 4) k_jacobi_mf(GridDesc g, const float* __restrict__ k32,
                                                      const float* __restrict__ dinv, const float* __restrict__ r,
                                                      float* __restrict__ out, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const long long ngroups = g.npts / 4;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= ngroups) return;
  const long long idx = (long long)pb * g.len + g.G + q * 4;
  float kq[4][5];
  load_kappa(k32, idx, g.px, g.pxy, kq);
  // s1 = dinv r on the 3 x 3 row neighbourhood, then A s1 through the rows
  float acc[1][4] = {{0.f, 0.f, 0.f, 0.f}};
  float di[4], ri[4];
  Vec<float>::load_keep(dinv + idx, di);
  Vec<float>::load_keep(r + idx, ri);
#define MPCG_JMF_ROW(DY, DZ)                                                                        \
  {                                                                                                 \
    float cf[3][4];                                                                                 \
    row_coefs<DY, DZ>(kq, cf);                                                                      \
    const long long ro = (long long)(DY) * g.px + (long long)(DZ) * g.pxy;                           \
    float ed[6], er[6];                                                                             \
    row6(dinv + idx + ro, ed);                                                           \
    row6(r + idx + ro, er);                                                              \
    _Pragma("unroll") for (int w = 0; w < 4; ++w) {                                                \
      acc[0][w] = fmaf(cf[0][w], ed[w] * er[w], acc[0][w]);                                         \
      acc[0][w] = fmaf(cf[1][w], ed[w + 1] * er[w + 1], acc[0][w]);                                 \
      acc[0][w] = fmaf(cf[2][w], ed[w + 2] * er[w + 2], acc[0][w]);                                 \
    }                                                                                               \
  }
  MPCG_JMF_ROW(-1, -1) MPCG_JMF_ROW(0, -1) MPCG_JMF_ROW(1, -1)
  MPCG_JMF_ROW(-1, 0) MPCG_JMF_ROW(0, 0) MPCG_JMF_ROW(1, 0)
  MPCG_JMF_ROW(-1, 1) MPCG_JMF_ROW(0, 1) MPCG_JMF_ROW(1, 1)
#undef MPCG_JMF_ROW
  float o[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    const float s1 = di[w] * ri[w];
    o[w] = s1 + di[w] * (ri[w] - acc[0][w]);
  }
  Vec<float>::store(out + idx, o);
}

// ---- 2D: kq[b][k] for the element whose lowest node is (x0 - 1 + k, y - 1 + b)
__device__ __forceinline__ void load_kappa2(const float* __restrict__ k32, long long idx, long long px,
                                            float (&kq)[2][5]) {
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    const float* p = k32 + idx + (long long)(b - 1) * px;
    float m[4];
    Vec<float>::load_keep(p, m);
    kq[b][0] = p[-1];
#pragma unroll
    for (int w = 0; w < 4; ++w) kq[b][w + 1] = m[w];
  }
}

// Coefficients of stencil row DY for the four points: cf[dx + 1][w].
template <int DY>
__device__ __forceinline__ void row_coefs2(const float (&kq)[2][5], float (&cf)[3][4]) {
  constexpr int b = DY > 0;
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    if (DY == 0) {   // edges (+-1, 0), centre
      cf[0][w] = kq[0][w] + kq[1][w];
      cf[1][w] = -4.f * (kq[0][w] + kq[0][w + 1] + kq[1][w] + kq[1][w + 1]);
      cf[2][w] = kq[0][w + 1] + kq[1][w + 1];
    } else {         // corners (+-1, DY), edge (0, DY)
      cf[0][w] = 2.f * kq[b][w];
      cf[1][w] = kq[b][w] + kq[b][w + 1];
      cf[2][w] = 2.f * kq[b][w + 1];
    }
  }
}

template <int C>
__global__ void __launch_bounds__(kBlock, 3) k_spmm_mf2d(GridDesc g, const float* __restrict__ k32,
                                                      const float* __restrict__ X, float* __restrict__ Y, double* zaz,
                                                      const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  float zacc[C];
#pragma unroll
  for (int c = 0; c < C; ++c) zacc[c] = 0.f;
  const long long ngroups = g.npts / 4;
  const long long bo = (long long)pb * g.len + g.G;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < ngroups;
       q += (long long)gridDim.x * blockDim.x) {
    int x0, y, z, a;
    decode(g, q * 4, x0, y, z, a);
    const long long idx = bo + q * 4;
    float kq[2][5];
    load_kappa2(k32, idx, g.px, kq);
    float cf[3][3][4];
    row_coefs2<-1>(kq, cf[0]);
    row_coefs2<0>(kq, cf[1]);
    row_coefs2<1>(kq, cf[2]);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float e[6];
        row6(X + (long long)c * g.cp + idx + (long long)(k - 1) * g.px, e);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          acc[w] = fmaf(cf[k][0][w], e[w], acc[w]);
          acc[w] = fmaf(cf[k][1][w], e[w + 1], acc[w]);
          acc[w] = fmaf(cf[k][2][w], e[w + 2], acc[w]);
        }
      }
#pragma unroll
      for (int w = 0; w < 4; ++w)
        if (y >= g.ny || x0 + w >= g.nx) acc[w] = 0.f;   // pad points: zero rows
      Vec<float>::store(Y + (long long)c * g.cp + idx, acc);
      if (zaz) {
        float xc[4];
        Vec<float>::load_keep(X + (long long)c * g.cp + idx, xc);
#pragma unroll
        for (int w = 0; w < 4; ++w) zacc[c] = fmaf(xc[w], acc[w], zacc[c]);
      }
    }
  }
  if (zaz) block_sum_store<float, C>(zacc, zaz + (long long)pb * C * gridDim.x, gridDim.x, blockIdx.x);
}

__global__ void __launch_bounds__(kBlock, 4) k_jacobi_mf2d(GridDesc g, const float* __restrict__ k32,
                                                        const float* __restrict__ dinv, const float* __restrict__ r,
                                                        float* __restrict__ out, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= g.npts / 4) return;
  const long long idx = (long long)pb * g.len + g.G + q * 4;
  float kq[2][5];
  load_kappa2(k32, idx, g.px, kq);
  float di[4], ri[4], acc[4] = {0.f, 0.f, 0.f, 0.f};
  Vec<float>::load_keep(dinv + idx, di);
  Vec<float>::load_keep(r + idx, ri);
#define MPCG_JMF2_ROW(DY)                                                                           \
  {                                                                                                 \
    float cf[3][4];                                                                                 \
    row_coefs2<DY>(kq, cf);                                                                         \
    float ed[6], er[6];                                                                             \
    row6(dinv + idx + (long long)(DY) * g.px, ed);                                                  \
    row6(r + idx + (long long)(DY) * g.px, er);                                                     \
    _Pragma("unroll") for (int w = 0; w < 4; ++w) {                                                \
      acc[w] = fmaf(cf[0][w], ed[w] * er[w], acc[w]);                                               \
      acc[w] = fmaf(cf[1][w], ed[w + 1] * er[w + 1], acc[w]);                                       \
      acc[w] = fmaf(cf[2][w], ed[w + 2] * er[w + 2], acc[w]);                                       \
    }                                                                                               \
  }
  MPCG_JMF2_ROW(-1) MPCG_JMF2_ROW(0) MPCG_JMF2_ROW(1)
#undef MPCG_JMF2_ROW
  float o[4];
#pragma unroll
  for (int w = 0; w < 4; ++w) o[w] = di[w] * ri[w] + di[w] * (ri[w] - acc[w]);
  Vec<float>::store(out + idx, o);
}

inline int blocks_for(long long n) { return (int)((n + kBlock - 1) / kBlock); }

}  // namespace

mpcg_status place_kappa(const GridDesc& g, const double* kappa, int ne, double h, float* k32, double* k64,
                        unsigned long long* check, const double* st64, double* maxdiff, double* maxabs,
                        cudaStream_t s) {
  if ((g.dim != 2 && g.dim != 3) || g.ncomp != 1) return MPCG_ERR_ARG;
  const long long n = g.dim == 3 ? (long long)ne * ne * ne : (long long)ne * ne;
  const double scale = g.dim == 3 ? -h / 12.0 : -1.0 / 6.0;
  k_place_kappa<<<dim3(grid_for(n, 4096), g.nb), kBlock, 0, s>>>(g, kappa, ne, scale, k32, k64);
  cudaMemsetAsync(check, 0, 2 * sizeof(unsigned long long), s);
  k_check_kappa<<<dim3(grid_for(g.npts, 2048), g.nb), kBlock, 0, s>>>(g, st64, k64, check);
  unsigned long long hv[2] = {0, 0};
  if (cudaMemcpyAsync(hv, check, sizeof(hv), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MPCG_ERR_CUDA;
  memcpy(maxdiff, &hv[0], sizeof(double));
  memcpy(maxabs, &hv[1], sizeof(double));
  return MPCG_OK;
}

#define MPCG_MF_CASES(K, ...)                                                                      \
  case 1: K<1><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                   \
  case 2: K<2><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                   \
  case 3: K<3><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                   \
  case 4: K<4><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                   \
  case 5: K<5><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                   \
  case 6: K<6><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                   \
  case 7: K<7><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                   \
  case 8: K<8><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                   \
  case 9: K<9><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                   \
  case 10: K<10><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                 \
  case 11: K<11><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;                                 \
  case 12: K<12><<<__VA_ARGS__>>>(g, k32, X, Y, zaz, state); break;

bool launch_spmm_mf(const GridDesc& g, const float* k32, const float* X, float* Y, int C, int nblocks, double* zaz,
                    const DevState* state, cudaStream_t s) {
  const dim3 grid(nblocks, g.nb);
  if (g.dim == 3) {
    switch (C) {
      MPCG_MF_CASES(k_spmm_mf, grid, kBlock, 0, s)
      default: return false;
    }
  } else {
    switch (C) {
      MPCG_MF_CASES(k_spmm_mf2d, grid, kBlock, 0, s)
      default: return false;
    }
  }
  return true;
}
#undef MPCG_MF_CASES

void launch_jacobi_mf(const GridDesc& g, const float* k32, const float* dinv, const float* r, float* out,
                      const DevState* state, cudaStream_t s) {
  const dim3 grid(blocks_for(g.npts / 4), g.nb);
  if (g.dim == 3) k_jacobi_mf<<<grid, kBlock, 0, s>>>(g, k32, dinv, r, out, state);
  else k_jacobi_mf2d<<<grid, kBlock, 0, s>>>(g, k32, dinv, r, out, state);
}

}  // namespace mpcg
