// Small single-block kernels of the MPCG step (Section 2.2, Algorithm 1):
// the deterministic reduction of block partial sums, the coefficient blocks
// beta_j = (P_j^T A P_j)^+ (A P_j)^T Z, the step alpha = (P^T A P)^+ P^T r with
// the column-drop rule and the scaled pseudo-inverse, the convergence test,
// and the exact coarsest-level solve (dense Cholesky, S_0 of Section 2.1).
//
// The pseudo-inverse diagonalises D G D (D = diag(G_ii)^{-1/2}) with the
// cyclic Jacobi eigenvalue method in round-robin (parallel) ordering, one
// warp per matrix, and inverts the eigenvalues above tau * lambda_max.
#include <math.h>

#include "kernels.cuh"

namespace mpcg {

namespace {

// out[v] = sum_b part[v * stride + b], b < nblk: one warp per value, lanes
// stride over blocks, fixed shuffle tree (deterministic).
__device__ void reduce_values(const double* __restrict__ part, int nv, int nblk, int stride, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int v = warp; v < nv; v += nw) {
    double a = 0.0;
    for (int b = lane; b < nblk; b += 32) a += part[(long long)v * stride + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) out[v] = a;
  }
}

constexpr int kPad = 16;   // padded matrix size for the eigen solver (>= kMaxCols, even)

// Scaled pseudo-inverse of the symmetric n x n matrix G (row-major, ld kPad)
// restricted to the columns with act[i] != 0.  Result in Gp (ld kPad).  Runs
// on one warp; Gs, V, scratch are shared arrays of kPad*kPad.
__device__ void warp_pinv(const double* G, const int* act, int n, double tau, double* Gp, double* A, double* V,
                          double* d, int* map, double* rot_c, double* rot_s, int* rot_p, int* rot_q) {
  const int lane = threadIdx.x & 31;
  // active index map
  if (lane == 0) {
    int k = 0;
    for (int i = 0; i < n; ++i)
      if (act[i]) map[k++] = i;
    map[kPad - 1] = k;       // count stored in the last slot
  }
  __syncwarp();
  const int na = map[kPad - 1];
  for (int e = lane; e < kPad * kPad; e += 32) Gp[e] = 0.0;
  if (na == 0) { __syncwarp(); return; }
  for (int i = lane; i < na; i += 32) d[i] = 1.0 / sqrt(G[map[i] * kPad + map[i]]);
  __syncwarp();
  const int np = (na + 1) & ~1;   // even size; index na is a dummy when na is odd
  for (int e = lane; e < kPad * kPad; e += 32) {
    const int i = e / kPad, j = e % kPad;
    A[e] = (i < na && j < na) ? d[i] * G[map[i] * kPad + map[j]] * d[j] : 0.0;
    V[e] = (i == j) ? 1.0 : 0.0;
  }
  __syncwarp();
  for (int sweep = 0; sweep < 30; ++sweep) {
    // convergence: off-diagonal Frobenius norm vs total
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
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        }
        rot_p[lane] = p; rot_q[lane] = q; rot_c[lane] = c; rot_s[lane] = s;
      }
      __syncwarp();
      // A <- A J (columns), then A <- J^T A (rows), V <- V J
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
  // eigenvalues on the diagonal; inverse of those above tau * max
  double lmax = 0.0;
  for (int i = 0; i < na; ++i) lmax = fmax(lmax, A[i * kPad + i]);
  __syncwarp();
  for (int e = lane; e < na * na; e += 32) {
    const int i = e / na, j = e % na;
    double s = 0.0;
    for (int k = 0; k < na; ++k) {
      const double lk = A[k * kPad + k];
      if (lk > tau * lmax) s += V[i * kPad + k] * V[j * kPad + k] / lk;
    }
    Gp[map[i] * kPad + map[j]] = d[i] * s * d[j];
  }
  __syncwarp();
}

__global__ void k_set_params(DevState* st, double rtol, int maxit, int m, int C, double delta, double tau) {
  st->rtol = rtol;
  st->maxit = maxit;
  st->m = m;
  st->ncols = C;
  st->delta = delta;
  st->tau = tau;
}

__global__ void k_init(DevState* st, const double* part_res, int nblk, double* res_hist,
                       cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double v[2];
  reduce_values(part_res, 2, nblk, kRedBlocks, v);
  __syncthreads();
  if (threadIdx.x == 0) {
    st->k = 0;
    st->count = 0;
    st->newest = st->m - 1;
    st->dropped_total = 0;
    st->rnorm = sqrt(v[0]);
    st->bnorm = sqrt(v[1]);
    int done = 0;
    if (st->bnorm == 0.0 || st->rnorm <= st->rtol * st->bnorm) done = 1;
    else if (st->maxit <= 0) done = 2;
    else if (!isfinite(st->rnorm)) done = 3;
    st->done = done;
    if (res_hist) res_hist[0] = st->bnorm > 0.0 ? st->rnorm / st->bnorm : 0.0;
    if (use_cond) cudaGraphSetConditional(cond, done == 0 ? 1u : 0u);
  }
}

__global__ void k_small_beta(DevState* st, const double* part_W, int C) {
  if (st->done) return;
  const int cnt = st->count;
  if (cnt == 0) return;
  const int m = st->m, newest = st->newest;
  __shared__ double W[kMaxWindow * kMaxCols * kMaxCols];
  reduce_values(part_W, cnt * C * C, kGramBlocks, kGramBlocks, W);
  __syncthreads();
  for (int e = threadIdx.x; e < cnt * C * C; e += blockDim.x) {
    const int jj = e / (C * C), a = (e / C) % C, b = e % C;
    const int slot = (newest - jj + m) % m;
    double s = 0.0;
    for (int c = 0; c < C; ++c) s += st->gpinv[slot][a][c] * W[(jj * C + c) * C + b];
    st->beta[jj][a][b] = s;
  }
}

__global__ void k_small_alpha(DevState* st, const double* part_G, const double* part_zaz, int C,
                              double* alpha_hist) {
  if (st->done) return;
  const int NG = C * (C + 1) / 2;
  __shared__ double red[kMaxCols * (kMaxCols + 1) / 2 + 2 * kMaxCols];
  __shared__ double G[kPad * kPad], Gp[kPad * kPad], A[kPad * kPad], V[kPad * kPad];
  __shared__ double dsc[kPad], rc[kPad], rs[kPad];
  __shared__ int act[kPad], map[kPad], rp[kPad], rq[kPad];
  reduce_values(part_G, NG + C, kRedBlocks, kRedBlocks, red);
  reduce_values(part_zaz, C, kRedBlocks, kRedBlocks, red + NG + C);
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    // G = sym(P^T A P): the partials hold p_a ap_b + p_b ap_a for a <= b
    for (int e = lane; e < kPad * kPad; e += 32) G[e] = 0.0;
    __syncwarp();
    if (lane == 0) {
      int k = 0, nact = 0;
      for (int a = 0; a < C; ++a)
        for (int b = a; b < C; ++b) {
          const double v = 0.5 * red[k++];
          G[a * kPad + b] = v;
          G[b * kPad + a] = v;
        }
      int bad = 0;
      for (int a = 0; a < C; ++a) {
        const double pap = G[a * kPad + a], zaz = red[NG + C + a];
        if (!isfinite(pap) || !isfinite(zaz)) bad = 1;
        act[a] = pap > st->delta * zaz ? 1 : 0;
        nact += act[a];
      }
      for (int a = 0; a < C; ++a)
        if (!act[a]) {
          for (int b = 0; b < C; ++b) G[a * kPad + b] = G[b * kPad + a] = 0.0;
          st->dropped_total += 1;
        }
      if (bad || nact == 0) st->done = 3;
    }
    __syncwarp();
    warp_pinv(G, act, C, st->tau, Gp, A, V, dsc, map, rc, rs, rp, rq);
    const int ns = (st->newest + 1) % st->m;
    for (int e = lane; e < C * C; e += 32) st->gpinv[ns][e / C][e % C] = Gp[(e / C) * kPad + e % C];
    if (lane < C) {
      double s = 0.0;
      for (int b = 0; b < C; ++b) s += Gp[lane * kPad + b] * red[NG + b];
      st->alpha[lane] = s;
      if (alpha_hist) alpha_hist[(long long)st->k * C + lane] = s;
    }
    __syncwarp();
    if (lane == 0) {
      st->newest = ns;
      if (st->count < st->m) st->count += 1;
    }
  }
}

__global__ void k_check(DevState* st, const double* part_r, int nblk, double* res_hist,
                        cudaGraphConditionalHandle cond, int use_cond) {
  __shared__ double v[1];
  const int was_done = st->done;
  if (!was_done) reduce_values(part_r, 1, nblk, kRedBlocks, v);
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

__global__ void k_dense_from_stencil(GridDesc g, const double* __restrict__ st, double* __restrict__ dense) {
  const long long n = g.n;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int x = (int)(i % g.n1), y = (int)((i / g.n1) % g.n1), z = (int)(i / ((long long)g.n1 * g.n1));
  const long long idx = g.G + x + (long long)g.p * y + (long long)g.p * g.p * z;
  const int S = g.dim == 3 ? 27 : 9;
  for (int j = 0; j < n; ++j) dense[i * n + j] = 0.0;
  for (int s = 0; s < S; ++s) {
    const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = g.dim == 3 ? s / 9 - 1 : 0;
    const int nx = x + dx, ny = y + dy, nz = z + dz;
    if (nx < 0 || nx >= g.n1 || ny < 0 || ny >= g.n1 || nz < 0 || (g.dim == 3 ? nz >= g.n1 : nz != 0)) continue;
    const long long j = nx + (long long)g.n1 * ny + (long long)g.n1 * g.n1 * nz;
    dense[i * n + j] = st[s * g.len + idx];
  }
}

// Right-looking dense Cholesky A = L L^T (lower triangle overwritten), one block.
__global__ void k_cholesky(double* a, int n, int* info) {
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double piv = a[(long long)k * n + k];
      if (!(piv > 0.0) || !isfinite(piv)) fail = k + 1;
      else a[(long long)k * n + k] = sqrt(piv);
    }
    __syncthreads();
    if (fail) break;
    const double lkk = a[(long long)k * n + k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) a[(long long)i * n + k] /= lkk;
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

// out = A0^{-1} r by forward and backward substitution with the Cholesky
// factor; one warp, column-oriented.
template <typename T>
__global__ void k_coarse_solve(GridDesc g, const double* __restrict__ L, const T* __restrict__ r, T* __restrict__ out,
                               const DevState* state) {
  if (state && state->done) return;
  extern __shared__ double y[];
  const int n = (int)g.n, lane = threadIdx.x;
  auto padded = [&](int i) {
    const int x = i % g.n1, yy = (i / g.n1) % g.n1, z = i / (g.n1 * g.n1);
    return g.G + x + (long long)g.p * yy + (long long)g.p * g.p * z;
  };
  for (int i = lane; i < n; i += 32) y[i] = (double)r[padded(i)];
  __syncwarp();
  for (int i = 0; i < n; ++i) {
    const double yi = y[i] / L[(long long)i * n + i];
    __syncwarp();
    if (lane == 0) y[i] = yi;
    for (int k = i + 1 + lane; k < n; k += 32) y[k] -= L[(long long)k * n + i] * yi;
    __syncwarp();
  }
  for (int i = n - 1; i >= 0; --i) {
    const double xi = y[i] / L[(long long)i * n + i];
    __syncwarp();
    if (lane == 0) y[i] = xi;
    for (int k = lane; k < i; k += 32) y[k] -= L[(long long)i * n + k] * xi;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) out[padded(i)] = (T)y[i];
}

__global__ void k_sum_partials(const double* part, int nv, int nblk, double* out) {
  reduce_values(part, nv, nblk, kRedBlocks, out);
}

__global__ void k_axpy_mixed(GridDesc g, double* __restrict__ x, const float* __restrict__ d,
                             const double* __restrict__ nrm2) {
  const double sc = sqrt(nrm2[0]);
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    const long long idx = g.G + t;
    x[idx] = fma(sc, (double)d[idx], x[idx]);
  }
}

__global__ void k_scale_to_f32(GridDesc g, const double* __restrict__ r, const double* __restrict__ nrm2,
                               float* __restrict__ out) {
  const double inv = nrm2[0] > 0.0 ? 1.0 / sqrt(nrm2[0]) : 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    const long long idx = g.G + t;
    out[idx] = (float)(r[idx] * inv);
  }
}

}  // namespace

void launch_set_params(DevState* st, double rtol, int maxit, int m, int C, double delta, double tau,
                       cudaStream_t s) {
  k_set_params<<<1, 1, 0, s>>>(st, rtol, maxit, m, C, delta, tau);
}
void launch_init(DevState* st, const double* part_res, int nblk, double* res_hist, cudaGraphConditionalHandle cond,
                 int use_cond, cudaStream_t s) {
  k_init<<<1, kBlock, 0, s>>>(st, part_res, nblk, res_hist, cond, use_cond);
}
void launch_small_beta(DevState* st, const double* part_W, int C, cudaStream_t s) {
  k_small_beta<<<1, 1024, 0, s>>>(st, part_W, C);
}
void launch_small_alpha(DevState* st, const double* part_G, const double* part_zaz, int C, double* alpha_hist,
                        cudaStream_t s) {
  k_small_alpha<<<1, kBlock, 0, s>>>(st, part_G, part_zaz, C, alpha_hist);
}
void launch_check(DevState* st, const double* part_r, int nblk, double* res_hist, cudaGraphConditionalHandle cond,
                  int use_cond, cudaStream_t s) {
  k_check<<<1, kBlock, 0, s>>>(st, part_r, nblk, res_hist, cond, use_cond);
}
void launch_dense_from_stencil(const GridDesc& g, const double* st, double* dense, cudaStream_t s) {
  k_dense_from_stencil<<<(int)((g.n + 127) / 128), 128, 0, s>>>(g, st, dense);
}
void launch_cholesky(double* a, int n, int* info, cudaStream_t s) { k_cholesky<<<1, 512, 0, s>>>(a, n, info); }
template <typename T>
void launch_coarse_solve(const GridDesc& g, const double* L, const T* r, T* out, const DevState* state,
                         cudaStream_t s) {
  k_coarse_solve<T><<<1, 32, (size_t)g.n * sizeof(double), s>>>(g, L, r, out, state);
}
template void launch_coarse_solve<double>(const GridDesc&, const double*, const double*, double*, const DevState*,
                                          cudaStream_t);
template void launch_coarse_solve<float>(const GridDesc&, const double*, const float*, float*, const DevState*,
                                         cudaStream_t);
void launch_sum_partials(const double* part, int nv, int nblk, double* out, cudaStream_t s) {
  k_sum_partials<<<1, kBlock, 0, s>>>(part, nv, nblk, out);
}
void launch_axpy_mixed(const GridDesc& g, double* x, const float* d, const double* scale, cudaStream_t s) {
  k_axpy_mixed<<<grid_for(g.npts, 4096), kBlock, 0, s>>>(g, x, d, scale);
}
void launch_scale_to_f32(const GridDesc& g, const double* r, const double* nrm2, float* out, cudaStream_t s) {
  k_scale_to_f32<<<grid_for(g.npts, 4096), kBlock, 0, s>>>(g, r, nrm2, out);
}

}  // namespace mpcg
