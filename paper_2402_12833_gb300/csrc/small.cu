// Small single-block kernels of the MPCG step (Section 2.2, Algorithm 1):
// the deterministic reduction of block partial sums, the coefficient blocks
// beta_j = (P_j^T A P_j)^+ (A P_j)^T Z, the step alpha = (P^T A P)^+ P^T r with
// the column-drop rule and the scaled pseudo-inverse, the convergence test,
// and the exact coarsest-level solve (dense Cholesky, S_0 of Section 2.1).
//
// Scaled pseudo-inverse: with D = diag(G_ii)^{-1/2} on the active columns,
// G^+ = D (D G D)^+ D, where (D G D)^+ keeps the eigenvalues above
// tau * lambda_max.  D G D has unit diagonal, so lambda_max <= n_active and
// lambda_min >= 1 / trace((D G D)^{-1}); when a Cholesky factorisation
// succeeds and 1 / trace(inverse) > tau * n_active, every eigenvalue is kept
// and the pseudo-inverse is the inverse, computed from the factor.  Otherwise
// the cyclic Jacobi eigenvalue method (round-robin ordering, one warp)
// diagonalises D G D and the small eigenvalues are cut.
#include <math.h>

#include "kernels.cuh"

namespace mpcg {

static_assert(kMaxCols <= 12, "MPCG_SMALL_C_SWITCH covers up to 12 columns");
#define MPCG_SMALL_C_SWITCH(C, BODY)                                                             \
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

namespace {

// out[v] = sum_b part[v * stride + b], b < nblk: one warp per value, lanes
// stride over blocks, fixed shuffle tree (deterministic).
__device__ void reduce_values(const double* __restrict__ part, int nv, int nblk, int stride, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = warp; v < nv; v += nw) {
    const double* p = part + (long long)v * stride;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int b = lane;
    for (; b + 96 < nblk; b += 128) {
      a0 += p[b];
      a1 += p[b + 32];
      a2 += p[b + 64];
      a3 += p[b + 96];
    }
    for (; b < nblk; b += 32) a0 += p[b];
    double a = (a0 + a1) + (a2 + a3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) out[v] = a;
  }
}

// Multi-block reduction of value-major partial sums.  Value v (of nv) is
// summed by block v % gridDim.x over its nblk partials in a fixed order and
// written to red[v].  Exactly one block -- the last to finish -- gets true,
// after which every red[v] is visible to it (read them with __ldcg).  The
// counter is zero between launches.  Values below nv_a come from part_a
// (stride stride_a, nblk_a partials), the rest from part_b.
__device__ bool reduce_values_grid(const double* __restrict__ part_a, int nv_a, int nblk_a, int stride_a,
                                   const double* __restrict__ part_b, int nv_b, int nblk_b, int stride_b,
                                   double* red, unsigned* counter) {
  __shared__ double wsum[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = blockIdx.x; v < nv_a + nv_b; v += gridDim.x) {
    const double* p = v < nv_a ? part_a + (long long)v * stride_a : part_b + (long long)(v - nv_a) * stride_b;
    const int nb = v < nv_a ? nblk_a : nblk_b;
    double a = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) a += p[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) wsum[warp] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
      red[v] = t;
    }
    __syncthreads();
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(counter, 1u) == gridDim.x - 1;
  __syncthreads();
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0u;
  }
  return last;
}

constexpr int kPad = 16;   // padded matrix size for the small solvers (>= kMaxCols, even)

// Jacobi eigenvalue pseudo-inverse of the na x na matrix A (ld kPad, active
// part already scaled to unit diagonal); result into Ah (ld kPad).  One warp.
__device__ void warp_jacobi_pinv(double* A, double* V, int na, double tau, double* Ah, double* rot_c, double* rot_s,
                                 int* rot_p, int* rot_q, double* lam) {
  const int lane = threadIdx.x & 31;
  for (int e = lane; e < kPad * kPad; e += 32) V[e] = (e / kPad == e % kPad) ? 1.0 : 0.0;
  __syncwarp();
  const int np = (na + 1) & ~1;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = lane; e < na * na; e += 32) {
      const int i = e / na, j = e % na;
      const double v = A[i * kPad + j];
      tot += v * v;
      if (i != j) off += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (off <= 1e-30 * tot) break;
    for (int round = 0; round < np - 1; ++round) {
      const int npairs = np / 2;
      if (lane < npairs) {
        int p, q;
        if (lane == 0) { p = np - 1; q = round; }
        else { p = (round + lane) % (np - 1); q = (round - lane + np - 1) % (np - 1); }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, s = 0.0;
        if (q < na) {
          const double apq = A[p * kPad + q];
          if (apq != 0.0) {
            const double app = A[p * kPad + p], aqq = A[q * kPad + q];
            const double theta = (aqq - app) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = rsqrt(t * t + 1.0);
            s = t * c;
          }
        }
        rot_p[lane] = p; rot_q[lane] = q; rot_c[lane] = c; rot_s[lane] = s;
      }
      __syncwarp();
      for (int e = lane; e < npairs * np; e += 32) {
        const int k = e / np, i = e % np;
        const int p = rot_p[k], q = rot_q[k];
        const double c = rot_c[k], s = rot_s[k];
        const double aip = A[i * kPad + p], aiq = A[i * kPad + q];
        A[i * kPad + p] = c * aip - s * aiq;
        A[i * kPad + q] = s * aip + c * aiq;
        const double vip = V[i * kPad + p], viq = V[i * kPad + q];
        V[i * kPad + p] = c * vip - s * viq;
        V[i * kPad + q] = s * vip + c * viq;
      }
      __syncwarp();
      for (int e = lane; e < npairs * np; e += 32) {
        const int k = e / np, j = e % np;
        const int p = rot_p[k], q = rot_q[k];
        const double c = rot_c[k], s = rot_s[k];
        const double apj = A[p * kPad + j], aqj = A[q * kPad + j];
        A[p * kPad + j] = c * apj - s * aqj;
        A[q * kPad + j] = s * apj + c * aqj;
      }
      __syncwarp();
    }
  }
  double lmax = 0.0;
  for (int i = 0; i < na; ++i) lmax = fmax(lmax, A[i * kPad + i]);
  if (lane < na) {
    const double l = A[lane * kPad + lane];
    lam[lane] = l > tau * lmax ? 1.0 / l : 0.0;
  }
  __syncwarp();
  for (int e = lane; e < na * na; e += 32) {
    const int i = e / na, j = e % na;
    double s = 0.0;
    for (int k = 0; k < na; ++k) s += V[i * kPad + k] * V[j * kPad + k] * lam[k];
    Ah[i * kPad + j] = s;
  }
  __syncwarp();
}

__global__ void k_set_params(DevState* st, double rtol, int maxit, int m, int C, double delta, double tau) {
  st += blockIdx.x;
  st->rtol = rtol;
  st->maxit = maxit;
  st->m = m;
  st->ncols = C;
  st->delta = delta;
  st->tau = tau;
}

__global__ void k_init(DevState* st, const double* part_res, int nblk, double* res_hist, long long hist_stride,
                       cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double v[2];
  const int pb = blockIdx.x;
  st += pb;
  part_res += (long long)pb * 2 * nblk;
  if (res_hist) res_hist += pb * hist_stride;
  reduce_values(part_res, 2, nblk, nblk, v);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->k = 0;
    st->count = 0;
    st->newest = st->m - 1;
    st->dropped_total = 0;
    st->pinv_fallbacks = 0;
    st->rnorm = sqrt(v[0]);
    st->bnorm = sqrt(v[1]);
    int done = 0;
    // a non-finite b or x_0 is a breakdown, tested first: with b infinite,
    // ||r|| <= rtol ||b|| reads inf <= inf and would pass as converged
    if (!isfinite(st->rnorm) || !isfinite(st->bnorm)) done = 3;
    else if (st->bnorm == 0.0 || st->rnorm <= st->rtol * st->bnorm) done = 1;
    else if (st->maxit <= 0) done = 2;
    st->done = done;
    if (res_hist) res_hist[0] = st->bnorm > 0.0 ? st->rnorm / st->bnorm : 0.0;
    if (use_cond) cudaGraphSetConditional(cond, done == 0 ? 1u : 0u);
  }
}

// beta_j = G_j^+ W_j for the window blocks: the W partial sums are reduced by
// all blocks of the grid, the last block forms beta.
__global__ void k_small_beta(DevState* st, const double* part_W, int nchunks, int C, double* scratch,
                             unsigned* counter) {
  const int pb = blockIdx.y;
  st += pb;
  scratch += (long long)pb * kSmallScratch;
  counter += 2 * pb;
  part_W += (long long)pb * st->m * C * C * nchunks;
  if (st->done) return;
  const int cnt = st->count;
  if (cnt == 0) return;
  const int m = st->m, newest = st->newest;
  if (!reduce_values_grid(part_W, cnt * C * C, nchunks, nchunks, nullptr, 0, 0, 0, scratch, counter)) return;
  __shared__ double W[kMaxWindow * kMaxCols * kMaxCols];
  for (int e = threadIdx.x; e < cnt * C * C; e += blockDim.x) W[e] = __ldcg(scratch + e);
  __syncthreads();
  for (int e = threadIdx.x; e < cnt * C * C; e += blockDim.x) {
    const int jj = e / (C * C), a = (e / C) % C, b = e % C;
    const int slot = (newest - jj + m) % m;
    double s = 0.0;
    for (int c = 0; c < C; ++c) s += st->gpinv[slot][a][c] * W[(jj * C + c) * C + b];
    st->beta[jj][a][b] = s;
  }
}

// Position of G entry (a, b), a <= b, in the packed upper triangle of the
// reduced Gram values ((0,0), (0,1), ..., (0,C-1), (1,1), ...).
__device__ __forceinline__ int tri_index(int a, int b, int C) { return a * C - a * (a - 1) / 2 + (b - a); }

// alpha = G^+ g after the grid reduction of G = sym(P^T A P), g = P^T r and
// the z^T A z of the new block; G^+ also goes to the window ring.  One warp,
// C columns known at compile time.  GB300 issues one FP64 warp instruction
// per 64 cycles per SM sub-partition whatever the active lanes, so the
// factorisation keeps one row per lane in registers and every step is a
// handful of warp-wide instructions: the drop rule and the scaling are one
// pass over the lanes; the Cholesky factor of D G D (right-looking, lane i
// holds row i); the columns of L^{-1} by forward substitution (lane j holds
// column j), whose squares give trace((D G D)^{-1}) for the cut test; and
// row i of (D G D)^{-1} = L^{-T} (L^{-1} e_i) by backward substitution.
template <int C>
__global__ void __launch_bounds__(kBlock) k_small_alpha(DevState* st, const double* part_G, int nblk_G,
                                                        const double* part_zaz, int nblk_zaz, int zaz_stride,
                                                        double* alpha_hist, long long ahist_stride, double* scratch,
                                                        unsigned* counter) {
  constexpr int NG = C * (C + 1) / 2;
  constexpr unsigned kFull = 0xffffffffu;
  const int pb = blockIdx.y;
  st += pb;
  part_G += (long long)pb * (NG + C) * nblk_G;
  part_zaz += (long long)pb * C * zaz_stride;
  if (alpha_hist) alpha_hist += pb * ahist_stride;
  scratch += (long long)pb * kSmallScratch + kSmallScratchAlpha;
  counter += 2 * pb + 1;
  if (st->done) return;
  __shared__ double red[NG + 2 * C];
  __shared__ double Lsm[C][C];
  __shared__ double dsm[C];
  __shared__ int map[C];
  // workspace of the Jacobi eigenvalue fallback
  __shared__ double A[kPad * kPad], V[kPad * kPad], Ah[kPad * kPad];
  __shared__ double rc[kPad], rs[kPad], lam[kPad];
  __shared__ int rp[kPad], rq[kPad];
  if (!reduce_values_grid(part_G, NG + C, nblk_G, nblk_G, part_zaz, C, nblk_zaz, zaz_stride, scratch, counter))
    return;
  for (int e = threadIdx.x; e < NG + 2 * C; e += blockDim.x) red[e] = __ldcg(scratch + e);
  __syncthreads();
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  // column-drop rule on the diagonal (the partials hold p_a ap_b + p_b ap_a)
  double pap = 0.0, gv = 0.0;
  bool act = false, bad = false;
  if (lane < C) {
    pap = 0.5 * red[tri_index(lane, lane, C)];
    const double zaz = red[NG + C + lane];
    gv = red[NG + lane];
    bad = !isfinite(pap) || !isfinite(zaz);
    act = pap > st->delta * zaz && pap > 0.0;
  }
  const unsigned amask = __ballot_sync(kFull, act);
  const int na = __popc(amask);
  bad = __any_sync(kFull, bad);
  if (lane < C) map[lane] = 0;
  __syncwarp();
  if (act) map[__popc(amask & ((1u << lane) - 1u))] = lane;
  const double dsc = act ? rsqrt(pap) : 0.0;
  if (lane < C) dsm[lane] = dsc;
  __syncwarp();
  if (lane == 0) {
    st->dropped_total += C - na;
    if (bad || na == 0) st->done = 3;
  }
  const int ci = na > 0 ? map[lane < na ? lane : 0] : 0;
  const double di = __shfl_sync(kFull, dsc, ci);
  double Z[C];   // row `lane` of (D G D)^+ over the active positions
#pragma unroll
  for (int j = 0; j < C; ++j) Z[j] = 0.0;
  if (na > 0) {
    // row `lane` of D G D (G = 0.5 red; scaling by 0.5 is exact)
    double Ar[C];
    const double hdi = 0.5 * di;
#pragma unroll
    for (int j = 0; j < C; ++j) {
      const int cj = map[j < na ? j : 0];
      const double dj = __shfl_sync(kFull, dsc, cj);
      const int lo = ci < cj ? ci : cj, hi = ci < cj ? cj : ci;
      Ar[j] = (lane < na && j < na) ? hdi * red[tri_index(lo, hi, C)] * dj : 0.0;
    }
    // Cholesky D G D = L L^T; dinv[k] = 1 / L_kk
    double dinv[C];
    bool ok = true;
#pragma unroll
    for (int k = 0; k < C; ++k) {
      dinv[k] = 0.0;
      if (k < na && ok) {
        const double piv = __shfl_sync(kFull, Ar[k], k);
        if (!(piv > 0.0)) {
          ok = false;
        } else {
          const double li = rsqrt(piv);
          dinv[k] = li;
          Ar[k] *= li;   // L_ik; lane k: L_kk = piv / sqrt(piv)
#pragma unroll
          for (int j = k + 1; j < C; ++j)
            if (j < na) Ar[j] = fma(-Ar[k], __shfl_sync(kFull, Ar[k], j), Ar[j]);
        }
      }
    }
    if (ok) {
      if (lane < na) {
#pragma unroll
        for (int j = 0; j < C; ++j) Lsm[lane][j] = Ar[j];
      }
      __syncwarp();
      // column `lane` of L^{-1}
      double X[C];
#pragma unroll
      for (int k = 0; k < C; ++k) {
        X[k] = 0.0;
        if (k < na) {
          double s = k == lane ? 1.0 : 0.0;
#pragma unroll
          for (int m = 0; m < k; ++m) s = fma(-Lsm[k][m], X[m], s);
          X[k] = s * dinv[k];
        }
      }
      // every eigenvalue passes the cut when 1 / trace(inverse) > tau * n
      // (unit diagonal: lambda_max <= n, lambda_min >= 1 / trace(inverse))
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < C; ++k) t = fma(X[k], X[k], t);
      if (lane >= na) t = 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(kFull, t, o);
      ok = t > 0.0 && t * (st->tau * na) < 1.0;
      if (ok) {   // row `lane` of the inverse: L^{-T} times column `lane` of L^{-1}
#pragma unroll
        for (int k = C - 1; k >= 0; --k) {
          if (k < na) {
            double s = X[k];
#pragma unroll
            for (int m = k + 1; m < C; ++m)
              if (m < na) s = fma(-Lsm[m][k], Z[m], s);
            Z[k] = s * dinv[k];
          }
        }
      }
    }
    if (!ok) {   // Jacobi eigenvalue pseudo-inverse of D G D
      if (lane == 0) st->pinv_fallbacks += 1;
      for (int e = lane; e < kPad * kPad; e += 32) {
        const int i = e / kPad, j = e % kPad;
        double v = 0.0;
        if (i < na && j < na) {
          const int a = map[i], b = map[j];
          v = (0.5 * dsm[a]) * red[tri_index(a < b ? a : b, a < b ? b : a, C)] * dsm[b];
        }
        A[e] = v;
      }
      __syncwarp();
      warp_jacobi_pinv(A, V, na, st->tau, Ah, rc, rs, rp, rq, lam);
#pragma unroll
      for (int j = 0; j < C; ++j) Z[j] = (lane < na && j < na) ? Ah[lane * kPad + j] : 0.0;
    }
  }
  // G^+ = D (D G D)^+ D on the active columns (zero rows and columns for
  // dropped ones) into the window ring; alpha = G^+ g
  const int ns = (st->newest + 1) % st->m;
  for (int e = lane; e < C * C; e += 32) st->gpinv[ns][e / C][e % C] = 0.0;
  __syncwarp();
  double al = 0.0;
#pragma unroll
  for (int j = 0; j < C; ++j) {
    const int cj = map[j < na ? j : 0];
    const double dj = __shfl_sync(kFull, dsc, cj);
    const double gj = __shfl_sync(kFull, gv, cj);
    if (lane < na && j < na) {
      const double v = di * Z[j] * dj;
      st->gpinv[ns][ci][cj] = v;
      al = fma(v, gj, al);
    }
  }
  __syncwarp();
  if (lane < C && !act) {
    st->alpha[lane] = 0.0;
    if (alpha_hist) alpha_hist[(long long)st->k * C + lane] = 0.0;
  }
  if (lane < na) {
    st->alpha[ci] = al;
    if (alpha_hist) alpha_hist[(long long)st->k * C + ci] = al;
  }
  __syncwarp();
  if (lane == 0) {
    st->newest = ns;
    if (st->count < st->m) st->count += 1;
  }
}

__global__ void k_check(DevState* st, const double* part_r, int nblk, double* res_hist, long long hist_stride,
                        cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double v[1];
  __shared__ double w[kBlock / 32];
  const int pb = blockIdx.x;
  st += pb;
  part_r += (long long)pb * nblk;
  if (res_hist) res_hist += pb * hist_stride;
  const int was_done = st->done;
  if (!was_done) {
    // one value: every thread takes a strided share, then a fixed tree
    double a = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) a += part_r[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += w[i];
      v[0] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int done = was_done;
    if (!was_done) {
      st->k += 1;
      st->rnorm = sqrt(v[0]);
      if (res_hist) res_hist[st->k] = st->rnorm / st->bnorm;
      if (!isfinite(st->rnorm)) done = 3;
      else if (st->rnorm <= st->rtol * st->bnorm) done = 1;
      else if (st->k >= st->maxit) done = 2;
      st->done = done;
    }
    if (use_cond) cudaGraphSetConditional(cond, done == 0 ? 1u : 0u);
  }
}

// Dense matrix of the coarsest operator: row i = a + ncomp * node takes
// plane b * 3^dim + s at the row's padded entry as the coefficient of the
// unknown (node + offset_s, b).
__global__ void k_dense_from_stencil(GridDesc g, const double* __restrict__ st, double* __restrict__ dense) {
  const long long n = g.n;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long node = i / g.ncomp;
  const int x = (int)(node % g.nx), y = (int)((node / g.nx) % g.ny), z = (int)(node / ((long long)g.nx * g.ny));
  const long long idx = padded_index(g, i);
  const int S = g.dim == 3 ? 27 : 9;
  for (long long j = 0; j < n; ++j) dense[i * n + j] = 0.0;
  for (int b = 0; b < g.ncomp; ++b)
    for (int s = 0; s < S; ++s) {
      const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = g.dim == 3 ? s / 9 - 1 : 0;
      const int ox = x + dx, oy = y + dy, oz = z + dz;
      if (ox < 0 || ox >= g.nx || oy < 0 || oy >= g.ny || oz < 0 || oz >= g.nz) continue;
      const long long j = b + (long long)g.ncomp * (ox + (long long)g.nx * oy + (long long)g.nx * g.ny * oz);
      dense[i * n + j] = st[(long long)(b * S + s) * g.cp + idx];
    }
}

// Right-looking dense Cholesky A = L L^T (lower triangle overwritten), one
// block; rdiag[i] = 1 / L_ii for the solves.
__global__ void k_cholesky(double* a, double* rdiag, int n, int* info) {
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double piv = a[(long long)k * n + k];
      if (!(piv > 0.0) || !isfinite(piv)) fail = k + 1;
      else {
        const double l = sqrt(piv);
        a[(long long)k * n + k] = l;
        rdiag[k] = 1.0 / l;
      }
    }
    __syncthreads();
    if (fail) break;
    const double rk = rdiag[k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) a[(long long)i * n + k] *= rk;
    __syncthreads();
    const int m = n - k - 1;
    for (long long e = threadIdx.x; e < (long long)m * m; e += blockDim.x) {
      const int i = k + 1 + (int)(e / m), j = k + 1 + (int)(e % m);
      if (j <= i) a[(long long)i * n + j] -= a[(long long)i * n + k] * a[(long long)j * n + k];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) info[0] = fail;
}

// A0^{-1} = L^{-T} L^{-1} from the Cholesky factor A0 = L L^T (setup, one
// block): X = L^{-1} by forward substitution, one column per thread, then
// inv = X^T X.  The per-iteration coarse solve is then one parallel
// matrix-vector product instead of two sequential substitutions.
__global__ void k_coarse_inverse(const double* __restrict__ L, const double* __restrict__ rdiag, double* X,
                                 double* inv, int n) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    for (int i = 0; i < j; ++i) X[(long long)i * n + j] = 0.0;
    X[(long long)j * n + j] = rdiag[j];
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += L[(long long)i * n + k] * X[(long long)k * n + j];
      X[(long long)i * n + j] = -s * rdiag[i];
    }
  }
  __syncthreads();
  for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
    const int a = (int)(e / n), b = (int)(e % n);
    double s = 0.0;
    for (int k = a > b ? a : b; k < n; ++k) s += X[(long long)k * n + a] * X[(long long)k * n + b];
    inv[e] = s;
  }
}

// out = A0^{-1} r (the exact coarsest solve S_0): one warp per row, lanes
// striding over the (contiguous) row, a fixed shuffle tree for the sum.
// Every block stages the whole right-hand side in shared memory.
constexpr int kCoarseRowsPerBlock = 8;

template <typename T>
__global__ void __launch_bounds__(32 * kCoarseRowsPerBlock) k_coarse_solve(GridDesc g, const double* __restrict__ inv,
                                                                           const T* __restrict__ r,
                                                                           T* __restrict__ out, const DevState* state) {
  const int pb = blockIdx.y;
  if (state && state[pb].done) return;
  extern __shared__ double y[];
  const int n = (int)g.n;
  inv += (long long)pb * n * n;
  r += (long long)pb * g.len;
  out += (long long)pb * g.len;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = (double)r[padded_index(g, i)];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * kCoarseRowsPerBlock + (threadIdx.x >> 5);
  if (i >= n) return;
  const double* row = inv + (long long)i * n;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma(row[j], y[j], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[padded_index(g, i)] = (T)s;
}

// out[b * nv + v] = sum of problem b's partials of value v.
__global__ void k_sum_partials(const double* part, int nv, int nblk, double* out) {
  const int pb = blockIdx.x;
  reduce_values(part + (long long)pb * nv * nblk, nv, nblk, nblk, out + (long long)pb * nv);
}

// flag |= some problem of the batch is still running.
// Device side of the mixed-precision refinement loop (one graph per solve):
// mix[p] = {inner iterations so far, status (0 running, 1 converged, 2 out
// of iterations or steps, 3 breakdown), active}.
__global__ void k_mix_init(int* mix, int* active, int nb, int* outer) {
  for (int p = threadIdx.x; p < nb; p += blockDim.x) {
    mix[3 * p + 0] = 0;
    mix[3 * p + 1] = 0;
    mix[3 * p + 2] = 1;
    active[p] = 1;
  }
  if (threadIdx.x == 0) *outer = 0;
}

// After the FP64 residual: decide every problem's state from |r|^2 and |b|^2
// (nrm[2p], nrm[2p+1]), hand the running ones their inner parameters
// (tolerance, remaining iterations, window, columns, drop and cutoff
// thresholds), and set the outer loop's condition (some problem running).
__global__ void k_outer_check(int* mix, int* active, int nb, const double* nrm, double rtol, int maxit,
                              int max_outer, int* outer, DevState* st, double inner_rtol, int m, int C,
                              double delta, double tau, cudaGraphConditionalHandle cond) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const int step = *outer;
  for (int p = threadIdx.x; p < nb; p += blockDim.x) {
    int* mp = mix + 3 * p;
    int budget = 0;
    if (mp[2]) {
      const double rn = sqrt(nrm[2 * p]), bn = sqrt(nrm[2 * p + 1]);
      if (!isfinite(rn)) { mp[1] = 3; mp[2] = 0; }
      else if (bn == 0.0 || rn <= rtol * bn) { mp[1] = 1; mp[2] = 0; }
      else if (mp[0] >= maxit || step >= max_outer) { mp[1] = 2; mp[2] = 0; }
      else {
        budget = maxit - mp[0];
        atomicOr(&any, 1);
      }
    }
    active[p] = mp[2];
    st[p].rtol = inner_rtol;
    st[p].maxit = budget;
    st[p].m = m;
    st[p].ncols = C;
    st[p].delta = delta;
    st[p].tau = tau;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *outer = step + 1;
    cudaGraphSetConditional(cond, any ? 1u : 0u);
  }
}

// After an inner solve: count its iterations, stop problems that broke down
// or made no progress.
__global__ void k_outer_accumulate(int* mix, int nb, const DevState* st) {
  for (int p = threadIdx.x; p < nb; p += blockDim.x) {
    int* mp = mix + 3 * p;
    if (!mp[2]) continue;
    const int k = st[p].k;
    mp[0] += k;
    if (st[p].done == 3) { mp[1] = 3; mp[2] = 0; }
    else if (k == 0) { mp[1] = 2; mp[2] = 0; }
  }
}

__global__ void k_any_running(const DevState* st, int nb, int* flag) {
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    if (st[b].done == 0) atomicOr(flag, 1);
}

// out[2b] = iterations, out[2b+1] = done of problem b.
__global__ void k_gather_kd(const DevState* st, int nb, int* out) {
  for (int b = threadIdx.x + blockIdx.x * blockDim.x; b < nb; b += blockDim.x * gridDim.x) {
    out[2 * b] = st[b].k;
    out[2 * b + 1] = st[b].done;
  }
}

// The loop condition of a batched graph: continue while any problem runs.
__global__ void k_set_cond(int* flag, cudaGraphConditionalHandle cond) {
  cudaGraphSetConditional(cond, *flag ? 1u : 0u);
  *flag = 0;
}

}  // namespace

void launch_set_params(DevState* st, int nb, double rtol, int maxit, int m, int C, double delta, double tau,
                       cudaStream_t s) {
  k_set_params<<<nb, 1, 0, s>>>(st, rtol, maxit, m, C, delta, tau);
}
void launch_init(DevState* st, int nb, const double* part_res, int nblk, double* res_hist, long long hist_stride,
                 cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
  k_init<<<nb, kBlock, 0, s>>>(st, part_res, nblk, res_hist, hist_stride, cond, use_cond);
}
void launch_small_beta(DevState* st, int nb, const double* part_W, int nchunks, int C, double* scratch,
                       unsigned* counter, cudaStream_t s) {
  k_small_beta<<<dim3(kSmallGrid, nb), kBlock, 0, s>>>(st, part_W, nchunks, C, scratch, counter);
}
void launch_small_alpha(DevState* st, int nb, const double* part_G, int nblk_G, const double* part_zaz, int nblk_zaz,
                        int zaz_stride, int C, double* alpha_hist, long long ahist_stride, double* scratch,
                        unsigned* counter, cudaStream_t s) {
  MPCG_SMALL_C_SWITCH(C, (k_small_alpha<CC><<<dim3(kSmallGrid, nb), kBlock, 0, s>>>(
                             st, part_G, nblk_G, part_zaz, nblk_zaz, zaz_stride, alpha_hist, ahist_stride, scratch,
                             counter)));
}
void launch_check(DevState* st, int nb, const double* part_r, int nblk, double* res_hist, long long hist_stride,
                  cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s) {
  k_check<<<nb, kBlock, 0, s>>>(st, part_r, nblk, res_hist, hist_stride, cond, use_cond);
}
void launch_dense_from_stencil(const GridDesc& g, const double* st, double* dense, cudaStream_t s) {
  k_dense_from_stencil<<<(int)((g.n + 127) / 128), 128, 0, s>>>(g, st, dense);
}
void launch_cholesky(double* a, double* rdiag, int n, int* info, cudaStream_t s) {
  k_cholesky<<<1, 512, 0, s>>>(a, rdiag, n, info);
}
void launch_coarse_inverse(const double* L, const double* rdiag, double* X, double* inv, int n, cudaStream_t s) {
  k_coarse_inverse<<<1, 256, 0, s>>>(L, rdiag, X, inv, n);
}
template <typename T>
void launch_coarse_solve(const GridDesc& g, const double* inv, const T* r, T* out, const DevState* state,
                         cudaStream_t s) {
  const dim3 grid((unsigned)((g.n + kCoarseRowsPerBlock - 1) / kCoarseRowsPerBlock), g.nb);
  k_coarse_solve<T><<<grid, 32 * kCoarseRowsPerBlock, (size_t)g.n * sizeof(double), s>>>(g, inv, r, out, state);
}
template void launch_coarse_solve<double>(const GridDesc&, const double*, const double*, double*, const DevState*,
                                          cudaStream_t);
template void launch_coarse_solve<float>(const GridDesc&, const double*, const float*, float*, const DevState*,
                                         cudaStream_t);
template void launch_coarse_solve<dw>(const GridDesc&, const double*, const dw*, dw*, const DevState*, cudaStream_t);
void launch_mix_init(int* mix, int* active, int nb, int* outer, cudaStream_t s) {
  k_mix_init<<<1, kBlock, 0, s>>>(mix, active, nb, outer);
}
void launch_outer_check(int* mix, int* active, int nb, const double* nrm, double rtol, int maxit, int max_outer,
                        int* outer, DevState* st, double inner_rtol, int m, int C, double delta, double tau,
                        cudaGraphConditionalHandle cond, cudaStream_t s) {
  k_outer_check<<<1, kBlock, 0, s>>>(mix, active, nb, nrm, rtol, maxit, max_outer, outer, st, inner_rtol, m, C, delta,
                                     tau, cond);
}
void launch_outer_accumulate(int* mix, int nb, const DevState* st, cudaStream_t s) {
  k_outer_accumulate<<<1, kBlock, 0, s>>>(mix, nb, st);
}
void launch_sum_partials(const double* part, int nb, int nv, int nblk, double* out, cudaStream_t s) {
  k_sum_partials<<<nb, kBlock, 0, s>>>(part, nv, nblk, out);
}
void launch_any_running(const DevState* st, int nb, int* flag, cudaStream_t s) {
  k_any_running<<<1, kBlock, 0, s>>>(st, nb, flag);
}
void launch_set_cond(int* flag, cudaGraphConditionalHandle cond, cudaStream_t s) {
  k_set_cond<<<1, 1, 0, s>>>(flag, cond);
}
void launch_gather_kd(const DevState* st, int nb, int* out, cudaStream_t s) {
  k_gather_kd<<<(nb + kBlock - 1) / kBlock, kBlock, 0, s>>>(st, nb, out);
}

}  // namespace mpcg
