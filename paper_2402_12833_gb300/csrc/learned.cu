// Learned search direction (an extension beyond the paper): a 3x3
// convolutional network N with channels 2 -> 16 -> 16 -> 16 -> 1 (ReLU after
// the first three, zero padding, no bias) maps the scaled residual r / ||r||
// and the coefficient channel c = log10(diag A)/3 - mean to y; the solver
// appends z = ||r|| y as one more MPCG column.
//
// This file holds the training steps around the tensor-core kernels
// (learned_tc.cu: the forward pass; learned_train_tc.cu: weight and data
// gradients): the A-angle loss and its gradient, the reduction of the
// weight-gradient partials, Adam, and the coefficient channel.  Activations
// are bfloat16, channel-last, in the padded grid layout of common.cuh (pads
// hold zeros = the zero padding of the convolution); weights are bfloat16
// values kept as floats.  Weight layout W[co][ci][ky][kx] with tap = 3 ky +
// kx multiplying the input at offset (dx, dy) = (kx - 1, ky - 1).
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "vec.cuh"

namespace mpcg {

namespace {

__device__ __forceinline__ bool interior2(const GridDesc& g, long long t) {
  const int x = (int)(t & (g.p - 1)), y = (int)(t >> g.lp);
  return x < g.n1 && y < g.n1;
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
// layer sizes of the 2D (3x3) and 3D (3x3x3, 3 -> 16 -> 16 -> 16 -> 3) networks
__device__ __forceinline__ int net_layer_size(int net3, int layer) {
  if (net3) return layer == 0 || layer == 3 ? 3 * 16 * 27 : 16 * 16 * 27;
  return layer == 0 ? kNetC1 * kNetIn * 9 : (layer == 3 ? kNetW * 9 : kNetW * kNetW * 9);
}

__global__ void k_net_adam(const double* const* parts, int nblk, int nparams, int net3, float* master, float* m,
                           float* v, float* wq, int step, float lr, float b1, float b2, float eps) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nparams) return;
  int layer = 0, off = i;
  const int sizes[4] = {net_layer_size(net3, 0), net_layer_size(net3, 1), net_layer_size(net3, 2),
                        net_layer_size(net3, 3)};
  while (off >= sizes[layer]) off -= sizes[layer], ++layer;
  double gsum = 0.0;
  const double* p = parts[layer] + (long long)off * nblk;
  for (int k = 0; k < nblk; ++k) gsum += p[k];
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

__global__ void k_net_grad_sum(const double* const* parts, int nblk, int nparams, int net3, double* grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nparams) return;
  int layer = 0, off = i;
  const int sizes[4] = {net_layer_size(net3, 0), net_layer_size(net3, 1), net_layer_size(net3, 2),
                        net_layer_size(net3, 3)};
  while (off >= sizes[layer]) off -= sizes[layer], ++layer;
  double gsum = 0.0;
  const double* p = parts[layer] + (long long)off * nblk;
  for (int k = 0; k < nblk; ++k) gsum += p[k];
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

// Backward pass on the tensor cores (learned_train_tc.cu): per layer from
// the last, the weight gradient (partials into gr.part[layer]) and the data
// gradient through the layer, masked by the ReLU pattern of its input.
void launch_net_backward(const GridDesc& g, int B, const float* wq, NetActs acts, const float* dy, NetGrads gr,
                         int* err, cudaStream_t s) {
  launch_net_wgrad_tc(g, B, 3, dy, acts.a3, gr.part[3], err, s);
  launch_net_dgrad_tc(g, B, 1, dy, wq + kNetOff4, acts.a3, gr.d3, err, s);
  launch_net_wgrad_tc(g, B, 2, gr.d3, acts.a2, gr.part[2], err, s);
  launch_net_dgrad_tc(g, B, kNetW, gr.d3, wq + kNetOff3, acts.a2, gr.d2, err, s);
  launch_net_wgrad_tc(g, B, 1, gr.d2, acts.a1, gr.part[1], err, s);
  launch_net_dgrad_tc(g, B, kNetW, gr.d2, wq + kNetOff2, acts.a1, gr.d1, err, s);
  launch_net_wgrad_tc(g, B, 0, gr.d1, acts.a0, gr.part[0], err, s);
}

void launch_net_loss_grad(const GridDesc& g, int B, const float* y, const float* Ay, const float* e,
                          const float* Ae, double* part, double* coef, double* loss_sum, float* dy, cudaStream_t s) {
  const int nblk = 64;
  k_net_dots<<<dim3(nblk, B), kBlock, 0, s>>>(g, y, Ay, e, Ae, part);
  k_net_loss<<<1, 32, 0, s>>>(part, nblk, B, coef, loss_sum);
  k_net_dy<<<grid_for((long long)B * g.len, 4096), kBlock, 0, s>>>(g, B, Ay, Ae, coef, dy);
}

void launch_net_adam(const double* const* parts_dev, int nblk, int net3, float* master, float* m, float* v, float* wq,
                     int step, float lr, float b1, float b2, float eps, cudaStream_t s) {
  const int np = net3 ? kNet3Params : kNetParams;
  k_net_adam<<<(np + kBlock - 1) / kBlock, kBlock, 0, s>>>(parts_dev, nblk, np, net3, master, m, v, wq,
                                                                   step, lr, b1, b2, eps);
}

void launch_net_grad_sum(const double* const* parts_dev, int nblk, int net3, double* grad, cudaStream_t s) {
  const int np = net3 ? kNet3Params : kNetParams;
  k_net_grad_sum<<<(np + kBlock - 1) / kBlock, kBlock, 0, s>>>(parts_dev, nblk, np, net3, grad);
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
