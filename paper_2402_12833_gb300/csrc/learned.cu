// Learned search direction (an extension beyond the paper): a 3x3
// convolutional network N with channels 2 -> 16 -> 16 -> 16 -> 1 (ReLU after
// the first three, zero padding, no bias) maps the scaled residual r / ||r||
// and the coefficient channel c = log10(diag A)/3 - mean to y; the solver
// appends z = ||r|| y as one more MPCG column.
//
// Activations are bfloat16, channel-last, in the padded grid layout of
// common.cuh (pads hold zeros = the zero padding of the convolution); weights
// are bfloat16 values kept as floats; products are exact in FP32 and summed
// in FP32.  Training kernels: transposed convolutions for the data gradient
// (masked by the ReLU pattern), tiled weight gradients, the A-angle loss and
// Adam.  Weight layout W[co][ci][ky][kx] with tap = 3 ky + kx multiplying the
// input at offset (dx, dy) = (kx - 1, ky - 1).
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "vec.cuh"

namespace mpcg {

namespace {

__device__ __forceinline__ long long tap_offset(int tap, int p) { return (tap % 3 - 1) + (long long)(tap / 3 - 1) * p; }

__device__ __forceinline__ bool interior2(const GridDesc& g, long long t) {
  const int x = (int)(t & (g.p - 1)), y = (int)(t >> g.lp);
  return x < g.n1 && y < g.n1;
}

// Forward layer CIN -> COUT.  in/out: [B][len][C] bf16.  W: [COUT][CIN][9].
template <int CIN, int COUT, bool RELU>
__global__ void __launch_bounds__(kBlock) k_net_layer(GridDesc g, int B, const __nv_bfloat16* __restrict__ in,
                                                      const float* __restrict__ W, __nv_bfloat16* __restrict__ out) {
  __shared__ float Ws[9][CIN][COUT];
  for (int e = threadIdx.x; e < COUT * CIN * 9; e += blockDim.x) {
    const int co = e / (CIN * 9), ci = (e / 9) % CIN, tap = e % 9;
    Ws[tap][ci][co] = W[e];
  }
  __syncthreads();
  const long long total = (long long)B * g.npts;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(u / g.npts);
    const long long t = u - (long long)b * g.npts;
    const long long base = (long long)b * g.len + g.G + t;
    __nv_bfloat16* o = out + base * COUT;
    if (!interior2(g, t)) {
#pragma unroll
      for (int co = 0; co < COUT; ++co) o[co] = __float2bfloat16_rn(0.f);
      continue;
    }
    float acc[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) acc[co] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const __nv_bfloat16* src = in + (base + tap_offset(tap, g.p)) * CIN;
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) {
        const float v = __bfloat162float(src[ci]);
#pragma unroll
        for (int co = 0; co < COUT; ++co) acc[co] = fmaf(Ws[tap][ci][co], v, acc[co]);
      }
    }
#pragma unroll
    for (int co = 0; co < COUT; ++co) o[co] = __float2bfloat16_rn(RELU ? fmaxf(acc[co], 0.f) : acc[co]);
  }
}

// Network input: channel 0 = bf16(r * s), channel 1 = bf16(c), with
// s = 1 / ||r|| taken from the solver state (inference) or 1 (training,
// where r is already scaled).  in0 may be written for the weight gradient.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_net_input(GridDesc g, int B, const T* __restrict__ r, long long r_ld,
                                                      const float* __restrict__ c, const DevState* state,
                                                      __nv_bfloat16* __restrict__ in0) {
  if (state && state->done) return;
  const float s = state ? (float)(state->rnorm > 0.0 ? 1.0 / state->rnorm : 0.0) : 1.f;
  const long long total = (long long)B * g.npts;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(u / g.npts);
    const long long t = u - (long long)b * g.npts;
    const long long base = (long long)b * g.len + g.G + t;
    const bool in = interior2(g, t);
    in0[base * 2 + 0] = __float2bfloat16_rn(in ? (float)r[(long long)b * r_ld + g.G + t] * s : 0.f);
    in0[base * 2 + 1] = __float2bfloat16_rn(in ? c[g.G + t] : 0.f);
  }
}

// Last layer 16 -> 1 without ReLU.  Writes y (float, training) or the MPCG
// column z = ||r|| y (inference, type T).
template <typename T>
__global__ void __launch_bounds__(kBlock) k_net_last(GridDesc g, int B, const __nv_bfloat16* __restrict__ in,
                                                     const float* __restrict__ W, float* __restrict__ y,
                                                     T* __restrict__ z, const DevState* state) {
  if (state && state->done) return;
  __shared__ float Ws[9][16];
  for (int e = threadIdx.x; e < 16 * 9; e += blockDim.x) Ws[e % 9][e / 9] = W[e];
  __syncthreads();
  const double scale = state ? state->rnorm : 1.0;
  const long long total = (long long)B * g.npts;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(u / g.npts);
    const long long t = u - (long long)b * g.npts;
    const long long base = (long long)b * g.len + g.G + t;
    float acc = 0.f;
    if (interior2(g, t)) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const __nv_bfloat16* src = in + (base + tap_offset(tap, g.p)) * 16;
#pragma unroll
        for (int ci = 0; ci < 16; ++ci) acc = fmaf(Ws[tap][ci], __bfloat162float(src[ci]), acc);
      }
    }
    if (y) y[base] = acc;
    if (z) z[base] = (T)(scale * (double)acc);
  }
}

// Data gradient through a layer CIN -> COUT: dIn(p) = mask(p) *
// sum_tap W[tap]^T dOut(p - off(tap)); mask = (act_in > 0) (ReLU of the layer
// below).  dOut, dIn: [B][len][C] float with zero pads.
template <int CIN, int COUT>
__global__ void __launch_bounds__(kBlock) k_net_dgrad(GridDesc g, int B, const float* __restrict__ dOut,
                                                      const float* __restrict__ W,
                                                      const __nv_bfloat16* __restrict__ act_in,
                                                      float* __restrict__ dIn) {
  __shared__ float Ws[9][COUT][CIN];
  for (int e = threadIdx.x; e < COUT * CIN * 9; e += blockDim.x) {
    const int co = e / (CIN * 9), ci = (e / 9) % CIN, tap = e % 9;
    Ws[tap][co][ci] = W[e];
  }
  __syncthreads();
  const long long total = (long long)B * g.npts;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(u / g.npts);
    const long long t = u - (long long)b * g.npts;
    const long long base = (long long)b * g.len + g.G + t;
    float acc[CIN];
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) acc[ci] = 0.f;
    if (interior2(g, t)) {
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const float* src = dOut + (base - tap_offset(tap, g.p)) * COUT;
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
          const float d = src[co];
#pragma unroll
          for (int ci = 0; ci < CIN; ++ci) acc[ci] = fmaf(Ws[tap][co][ci], d, acc[ci]);
        }
      }
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci)
        if (!(__bfloat162float(act_in[base * CIN + ci]) > 0.f)) acc[ci] = 0.f;
    }
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) dIn[base * CIN + ci] = acc[ci];
  }
}

// Weight gradient of a layer CIN -> COUT: dW[co][ci][tap] = sum over items
// and points q of dOut(q)[co] * act_in(q + off(tap))[ci].  Each block takes
// a chunk of kWP consecutive points of one item, stages dOut and the input
// rows it touches in shared memory and writes its COUT*CIN*9 partial sums
// (value-major, stride = gridDim.x).
constexpr int kWP = 128;
template <int CIN, int COUT>
__global__ void __launch_bounds__(kBlock) k_net_wgrad(GridDesc g, int B, const float* __restrict__ dOut,
                                                      const __nv_bfloat16* __restrict__ act_in, double* part,
                                                      int chunks_per_item) {
  extern __shared__ float sm[];
  const int halo = g.p + 1;
  float* dO = sm;                              // [kWP][COUT]
  float* A = sm + kWP * COUT;                  // [kWP + 2 halo][CIN]
  const int b = blockIdx.x / chunks_per_item, chunk = blockIdx.x % chunks_per_item;
  const long long t0 = (long long)chunk * kWP;
  const long long base = (long long)b * g.len + g.G + t0;
  for (int e = threadIdx.x; e < kWP * COUT; e += blockDim.x) {
    const int q = e / COUT;
    dO[e] = t0 + q < g.npts ? dOut[(base + q) * COUT + e % COUT] : 0.f;
  }
  for (int e = threadIdx.x; e < (kWP + 2 * halo) * CIN; e += blockDim.x) {
    const int q = e / CIN - halo;
    // points within one halo of the box lie inside the vector's zero guards
    const bool ok = t0 + q >= -halo && t0 + q < g.npts + halo;
    A[e] = ok ? __bfloat162float(act_in[(base + q) * CIN + e % CIN]) : 0.f;
  }
  __syncthreads();
  constexpr int NV = COUT * CIN * 9;
  constexpr int PER = (NV + kBlock - 1) / kBlock;
  float acc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.f;
  for (int q = 0; q < kWP; ++q) {
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * kBlock;
      if (e < NV) {
        const int co = e / (CIN * 9), ci = (e / 9) % CIN, tap = e % 9;
        const int off = (tap % 3 - 1) + (tap / 3 - 1) * g.p;
        acc[k] = fmaf(dO[q * COUT + co], A[(q + halo + off) * CIN + ci], acc[k]);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * kBlock;
    if (e < NV) part[(long long)e * gridDim.x + blockIdx.x] = (double)acc[k];
  }
}

// Per item b: eAy, eAe, yAy (partials, value-major per item, stride nblk).
__global__ void __launch_bounds__(kBlock) k_net_dots(GridDesc g, const float* __restrict__ y,
                                                     const float* __restrict__ Ay, const float* __restrict__ e,
                                                     const float* __restrict__ Ae, double* part) {
  const int b = blockIdx.y;
  const long long o = (long long)b * g.len + g.G;
  float s[3] = {0.f, 0.f, 0.f};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    const float yv = y[o + t], av = Ay[o + t], ev = e[o + t], aev = Ae[o + t];
    s[0] = fmaf(ev, av, s[0]);
    s[1] = fmaf(ev, aev, s[1]);
    s[2] = fmaf(yv, av, s[2]);
  }
  block_sum_store<float, 3>(s, part + (long long)b * 3 * gridDim.x, gridDim.x, blockIdx.x);
}

// Loss per item and coefficients of dL/dy = -k1 (Ae - k2 Ay) / B.
__global__ void k_net_loss(const double* part, int nblk, int B, double* coef, double* loss_sum) {
  const int b = threadIdx.x;
  if (b >= B) return;
  double d[3];
  for (int v = 0; v < 3; ++v) {
    double a = 0.0;
    for (int k = 0; k < nblk; ++k) a += part[((long long)b * 3 + v) * nblk + k];
    d[v] = a;
  }
  const double eAy = d[0], eAe = d[1], yAy = d[2];
  const bool ok = eAe > 0.0 && yAy > 0.0;
  const double L = ok ? 1.0 - eAy * eAy / (eAe * yAy) : 1.0;
  coef[2 * b + 0] = ok ? 2.0 * eAy / (eAe * yAy) / B : 0.0;
  coef[2 * b + 1] = ok ? eAy / yAy : 0.0;
  atomicAdd(loss_sum, L / B);   // B <= 12 values; the order does not feed back into training
}

__global__ void k_net_dy(GridDesc g, int B, const float* __restrict__ Ay, const float* __restrict__ Ae,
                         const double* __restrict__ coef, float* __restrict__ dy) {
  const long long total = (long long)B * g.len;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(u / g.len);
    const float k1 = (float)coef[2 * b], k2 = (float)coef[2 * b + 1];
    dy[u] = -k1 * (Ae[u] - k2 * Ay[u]);
  }
}

// Reduce the weight-gradient partials of all layers and take one Adam step
// (Kingma & Ba 2015, bias-corrected) on the FP32 master weights; also writes
// the bfloat16-rounded copy used by the forward pass.
__global__ void k_net_adam(const double* const* parts, const int* nblk, int nparams, float* master, float* m,
                           float* v, float* wq, int step, float lr, float b1, float b2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nparams) return;
  int layer = 0, off = i;
  const int sizes[4] = {kNetC1 * kNetIn * 9, kNetW * kNetW * 9, kNetW * kNetW * 9, kNetW * 9};
  while (off >= sizes[layer]) off -= sizes[layer], ++layer;
  double gsum = 0.0;
  const double* p = parts[layer] + (long long)off * nblk[layer];
  for (int k = 0; k < nblk[layer]; ++k) gsum += p[k];
  const float gr = (float)gsum;
  const float mi = b1 * m[i] + (1.f - b1) * gr;
  const float vi = b2 * v[i] + (1.f - b2) * gr * gr;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / (1.f - powf(b1, (float)step));
  const float vh = vi / (1.f - powf(b2, (float)step));
  const float w = master[i] - lr * mh / (sqrtf(vh) + eps);
  master[i] = w;
  wq[i] = __bfloat162float(__float2bfloat16_rn(w));
}

__global__ void k_net_grad_sum(const double* const* parts, const int* nblk, int nparams, double* grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nparams) return;
  int layer = 0, off = i;
  const int sizes[4] = {kNetC1 * kNetIn * 9, kNetW * kNetW * 9, kNetW * kNetW * 9, kNetW * 9};
  while (off >= sizes[layer]) off -= sizes[layer], ++layer;
  double gsum = 0.0;
  const double* p = parts[layer] + (long long)off * nblk[layer];
  for (int k = 0; k < nblk[layer]; ++k) gsum += p[k];
  grad[i] = gsum;
}

__global__ void k_net_acts_export(GridDesc g, int B, NetActs a, float* out) {
  const long long nn = (long long)g.n1 * g.n1;
  const long long total = 4LL * B * nn;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int L = (int)(u / (B * nn));
    const int b = (int)((u / nn) % B);
    const long long q = u % nn;
    const long long t = (q / g.n1) * g.p + q % g.n1;
    const long long base = (long long)b * g.len + g.G + t;
    float* o = out + u * 16;
    const int C = L == 0 ? kNetIn : 16;
    const __nv_bfloat16* src = L == 0 ? a.a0 : L == 1 ? a.a1 : L == 2 ? a.a2 : a.a3;
    for (int ch = 0; ch < 16; ++ch) o[ch] = ch < C ? __bfloat162float(src[base * C + ch]) : 0.f;
  }
}

__global__ void k_round_bf16(const float* src, float* dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __bfloat162float(__float2bfloat16_rn(src[i]));
}

// c = log10(omega / dinv) / 3 at interior points (pads 0); partial sums.
__global__ void k_net_coef(GridDesc g, const double* __restrict__ dinv, double omega, float* c, double* part) {
  double s[1] = {0.0};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x) {
    const bool in = interior2(g, t);
    const double v = in ? log10(omega / dinv[g.G + t]) / 3.0 : 0.0;
    c[g.G + t] = (float)v;
    s[0] += v;
  }
  block_sum_store<double, 1>(s, part, gridDim.x, blockIdx.x);
}

__global__ void k_net_coef_center(GridDesc g, float* c, const double* part, int nblk) {
  __shared__ double mean;
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int k = 0; k < nblk; ++k) a += part[k];
    mean = a / (double)g.n;
  }
  __syncthreads();
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < g.npts;
       t += (long long)gridDim.x * blockDim.x)
    if (interior2(g, t)) c[g.G + t] = (float)((double)c[g.G + t] - mean);
}

}  // namespace

int net_blocks(const GridDesc& g, int B) { return grid_for((long long)B * g.npts, 4096); }

template <typename T>
void launch_net_forward(const GridDesc& g, int B, const T* r, long long r_ld, const float* c, const float* wq,
                        const DevState* state, NetActs acts, float* y, T* z, cudaStream_t s) {
  const int nb = net_blocks(g, B);
  k_net_input<T><<<nb, kBlock, 0, s>>>(g, B, r, r_ld, c, state, acts.a0);
  k_net_layer<kNetIn, kNetC1, true><<<nb, kBlock, 0, s>>>(g, B, acts.a0, wq + kNetOff1, acts.a1);
  k_net_layer<kNetW, kNetW, true><<<nb, kBlock, 0, s>>>(g, B, acts.a1, wq + kNetOff2, acts.a2);
  k_net_layer<kNetW, kNetW, true><<<nb, kBlock, 0, s>>>(g, B, acts.a2, wq + kNetOff3, acts.a3);
  k_net_last<T><<<nb, kBlock, 0, s>>>(g, B, acts.a3, wq + kNetOff4, y, z, state);
}
template void launch_net_forward<double>(const GridDesc&, int, const double*, long long, const float*, const float*,
                                         const DevState*, NetActs, float*, double*, cudaStream_t);
template void launch_net_forward<float>(const GridDesc&, int, const float*, long long, const float*, const float*,
                                        const DevState*, NetActs, float*, float*, cudaStream_t);

int net_wgrad_blocks(const GridDesc& g, int B) { return B * (int)((g.npts + kWP - 1) / kWP); }

void launch_net_backward(const GridDesc& g, int B, const float* wq, NetActs acts, const float* dy, NetGrads gr,
                         cudaStream_t s) {
  const int nb = net_blocks(g, B);
  const int cpi = (int)((g.npts + kWP - 1) / kWP);
  const int nw = B * cpi;
  const int halo = g.p + 1;
  auto shm = [&](int cin, int cout) { return (size_t)(kWP * cout + (kWP + 2 * halo) * cin) * sizeof(float); };
  // layer 4 (16 -> 1)
  k_net_wgrad<kNetW, 1><<<nw, kBlock, shm(kNetW, 1), s>>>(g, B, dy, acts.a3, gr.part[3], cpi);
  k_net_dgrad<kNetW, 1><<<nb, kBlock, 0, s>>>(g, B, dy, wq + kNetOff4, acts.a3, gr.d3);
  // layer 3
  k_net_wgrad<kNetW, kNetW><<<nw, kBlock, shm(kNetW, kNetW), s>>>(g, B, gr.d3, acts.a2, gr.part[2], cpi);
  k_net_dgrad<kNetW, kNetW><<<nb, kBlock, 0, s>>>(g, B, gr.d3, wq + kNetOff3, acts.a2, gr.d2);
  // layer 2
  k_net_wgrad<kNetW, kNetW><<<nw, kBlock, shm(kNetW, kNetW), s>>>(g, B, gr.d2, acts.a1, gr.part[1], cpi);
  k_net_dgrad<kNetW, kNetW><<<nb, kBlock, 0, s>>>(g, B, gr.d2, wq + kNetOff2, acts.a1, gr.d1);
  // layer 1 (weights only)
  k_net_wgrad<kNetIn, kNetC1><<<nw, kBlock, shm(kNetIn, kNetC1), s>>>(g, B, gr.d1, acts.a0, gr.part[0], cpi);
}

size_t net_wgrad_smem(const GridDesc& g) {
  return (size_t)(kWP * kNetW + (kWP + 2 * (g.p + 1)) * kNetW) * sizeof(float);
}

// Opt in to the dynamic shared memory the weight-gradient kernels need on
// grid g (host call, before any capture).
void net_prepare_attributes(const GridDesc& g) {
  const int bytes = (int)net_wgrad_smem(g);
  cudaFuncSetAttribute(k_net_wgrad<kNetW, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_net_wgrad<kNetW, kNetW>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  cudaFuncSetAttribute(k_net_wgrad<kNetIn, kNetC1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

void launch_net_loss_grad(const GridDesc& g, int B, const float* y, const float* Ay, const float* e,
                          const float* Ae, double* part, double* coef, double* loss_sum, float* dy, cudaStream_t s) {
  const int nblk = 64;
  k_net_dots<<<dim3(nblk, B), kBlock, 0, s>>>(g, y, Ay, e, Ae, part);
  k_net_loss<<<1, 32, 0, s>>>(part, nblk, B, coef, loss_sum);
  k_net_dy<<<grid_for((long long)B * g.len, 4096), kBlock, 0, s>>>(g, B, Ay, Ae, coef, dy);
}

void launch_net_adam(const double* const* parts_dev, const int* nblk_dev, float* master, float* m, float* v, float* wq,
                     int step, float lr, float b1, float b2, float eps, cudaStream_t s) {
  k_net_adam<<<(kNetParams + kBlock - 1) / kBlock, kBlock, 0, s>>>(parts_dev, nblk_dev, kNetParams, master, m, v, wq,
                                                                   step, lr, b1, b2, eps);
}

void launch_net_grad_sum(const double* const* parts_dev, const int* nblk_dev, double* grad, cudaStream_t s) {
  k_net_grad_sum<<<(kNetParams + kBlock - 1) / kBlock, kBlock, 0, s>>>(parts_dev, nblk_dev, kNetParams, grad);
}

void launch_net_acts_export(const GridDesc& g, int B, NetActs acts, float* out, cudaStream_t s) {
  k_net_acts_export<<<grid_for(4LL * B * g.n1 * g.n1, 4096), kBlock, 0, s>>>(g, B, acts, out);
}

void launch_round_bf16(const float* src, float* dst, int n, cudaStream_t s) {
  k_round_bf16<<<(n + kBlock - 1) / kBlock, kBlock, 0, s>>>(src, dst, n);
}

void launch_net_coef(const GridDesc& g, const double* dinv, double omega, float* c, double* part, cudaStream_t s) {
  const int nb = 256;
  k_net_coef<<<nb, kBlock, 0, s>>>(g, dinv, omega, c, part);
  k_net_coef_center<<<grid_for(g.npts, 1024), kBlock, 0, s>>>(g, c, part, nb);
}

}  // namespace mpcg
