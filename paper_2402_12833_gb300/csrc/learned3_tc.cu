// The learned column of 3D vector problems (3D elasticity) on the
// fifth-generation tensor cores: a 3x3x3 convolutional network with channels
// 3 -> 16 -> 16 -> 16 -> 3 (ReLU after the first three, zero padding, no
// bias) maps the three displacement components of r / ||r|| to y; the solver
// appends z = ||r|| y (all three components) as one MPCG column.
//
// Activations live on the node box of the vector grid (node t = x + px (y +
// py z), the same box as each displacement component) as 16 bfloat16
// channels per node, [B][act_len][16] with the grid's zero guards in front;
// nodes outside the unknown grid (pads) hold zeros, the zero padding of the
// convolutions.
//
// One launch per layer (the 3D halo of a fused four-layer tile would cost
// more than the round trip of 32 bytes per node): a CTA owns R = 4 rows of
// up to 128 nodes at one z and stages the 3 x (R + 2) input rows around them
// (x from -1 to 128) as K-major bfloat16 planes.  The MMAs go by staged row:
// per staged row, z plane and x shift the A operand is the staged row
// shifted (SBO = 128 B, LBO = one plane) and B stacks the 16 x 16 weight
// tiles of the y-taps that row feeds along N (16 to 48), into the 16 FP32
// TMEM columns of each output row (tcgen05.mma kind::f16, M = 128 nodes,
// K = 16): 57 MMAs per CTA in the forward pass; the data gradient (the
// transposed convolution, masked by the ReLU pattern of the layer input)
// takes its FP32 input as bfloat16 hi + lo planes, 114 MMAs per CTA.  The weight gradient is
// the pixel-reduction GEMM of the 2D network with 27 taps: A = dOut^T (hi
// rows 0-15, lo rows 16-31), B = the im2col of the layer input (27 taps x 16
// channels = 432 rows, three MMAs of N = 144 per K step), accumulated in 432
// TMEM columns over a CTA's run of 64-node chunks.
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.cuh"
#include "tc.cuh"

namespace mpcg {

namespace {

constexpr int kT3 = 128;                       // threads: TMEM lanes 0..127 = nodes of a row tile
constexpr int kR3 = 4;                         // output rows per CTA
constexpr int kXS3 = 130;                      // staged nodes per row: x = -1 .. 128
constexpr int kRows3 = 3 * (kR3 + 2);          // staged rows (z - 1 .. z + 1) x (y0 - 1 .. y0 + R)
constexpr int kPlane3 = kRows3 * kXS3 * 16;    // bytes of one 8-channel plane
constexpr int kW3Bytes = 27 * 512;             // 27 weight tiles of 16 x 16 bf16
constexpr long long kWait3 = 1LL << 22;
// polls of a first wait before a kernel gives up (set_wait_first_net3; the
// drain after a give-up always uses kWait3)
__constant__ long long c_wait_first3 = kWait3;

__device__ __forceinline__ int canon16(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__host__ __device__ __forceinline__ long long act_len3(const GridDesc& g) {
  return (2 * g.G + g.cstride + 31) / 32 * 32;
}

__device__ __forceinline__ bool inside3(const GridDesc& g, int x, int y, int z) {
  return x >= 0 && y >= 0 && z >= 0 && x < g.nx && y < g.ny && z < g.nz;
}

// smem byte layout of the conv kernel: NPL planes, the weight tiles, the
// row barriers, the TMEM slot
template <int NPL>
struct Conv3Smem {
  static constexpr int kWOff = NPL * kPlane3;
  static constexpr int kBarOff = kWOff + kW3Bytes;
  static constexpr int kBytes = kBarOff + 8 * (kR3 + 2) + 16;   // one mbarrier per staged y row
};

// MODE 0: forward, out = relu?(sum W in(p + off)), in bfloat16 activations;
//         LAST: 3 FP32 outputs to a vector-layout array (y, or z = s y).
// MODE 1: data gradient, dIn = mask(act_in > 0) sum W^T dOut(p - off), dOut
//         FP32 [B][act_len][16] (zero beyond the layer's outputs).
// 16-byte asynchronous copy global -> shared; src_bytes 0 zero-fills
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Packed weights: for layer l and mode m (0 forward, 1 data gradient) the 27
// tap tiles of 16 x 16 bfloat16 in the K-major layout of the B operand, at
// byte (2 l + m) * kW3Bytes, ordered (kz, kx, ky) so that the three y-taps of
// one (kz, kx) are consecutive.  Forward row n = co, column k = ci; gradient
// row n = ci, column k = co; zero beyond the layer's channels.
__global__ void k_net3_pack(const float* __restrict__ wq, unsigned char* __restrict__ wp) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 8 * 27 * 256) return;
  const int lm = e / (27 * 256), l = lm >> 1, mode = lm & 1;
  const int t = (e / 256) % 27, n = (e / 16) % 16, k = e % 16;
  const int cin = l == 0 ? 3 : 16, cout = l == 3 ? 3 : 16;
  const int off = l == 0 ? kNet3Off1 : l == 1 ? kNet3Off2 : l == 2 ? kNet3Off3 : kNet3Off4;
  const int co = mode == 0 ? n : k, ci = mode == 0 ? k : n;
  const float w = (co < cout && ci < cin) ? wq[off + (co * cin + ci) * 27 + t] : 0.f;
  // tap t = kz * 9 + ky * 3 + kx goes to tile (kz * 3 + kx) * 3 + ky (ky fastest)
  const int tp = ((t / 9) * 3 + t % 3) * 3 + (t / 3) % 3;
  *reinterpret_cast<__nv_bfloat16*>(wp + lm * kW3Bytes + tp * 512 + canon16(n, k)) = __float2bfloat16_rn(w);
}

template <int MODE, bool RELU, bool LAST, typename T>
__global__ void __launch_bounds__(kT3, 1)
    k_net3_conv_tc(GridDesc g, int B, const void* __restrict__ in, const unsigned char* __restrict__ wp, int cin,
                   int cout, const __nv_bfloat16* __restrict__ act_in, void* __restrict__ out,
                   float* __restrict__ yv, T* __restrict__ zv, const DevState* state, int* err) {
  constexpr int NPL = MODE == 0 ? 2 : 4;
  using S = Conv3Smem<NPL>;
  if (state && state->done) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + S::kBarOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + S::kBarOff + 8 * (kR3 + 2));
  const int tid = threadIdx.x, warp = tid >> 5;
  const int x0 = blockIdx.x * 128, y0 = blockIdx.y * kR3;
  const int z = blockIdx.z % g.pz, b = blockIdx.z / g.pz;
  const long long alen = act_len3(g);
  const long long abase = (long long)b * alen + g.G;
  const long long px = g.px, pxy = g.pxy;

  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), 64);
  if (tid < kR3 + 2) tc::mbar_init(tc::smem_u32(bar + tid));
  if (tid == 0) tc::mbar_init_fence();
  // the layer's 27 packed weight tiles (13,824 bytes)
  for (int e = tid; e < kW3Bytes / 16; e += kT3)
    cp_async16(smem + S::kWOff + 16 * e, wp + 16 * e, 16);
  // staged rows: slot (dz, sy) = dz * (R + 2) + sy holds node row (y0 - 1 + sy, z - 1 + dz)
  for (int e = tid; e < kRows3 * kXS3; e += kT3) {
    const int row = e / kXS3, xs = e % kXS3;
    const int dz = row / (kR3 + 2), sy = row % (kR3 + 2);
    const int x = x0 - 1 + xs, y = y0 - 1 + sy, zz = z - 1 + dz;
    const bool in_grid = inside3(g, x, y, zz);
    const long long node = in_grid ? abase + x + px * y + pxy * zz : abase;
    const int off = (row * kXS3 + xs) * 16;
    if (MODE == 0) {   // two 16-byte halves (channels 0-7, 8-15), zero-filled off the grid
      const __nv_bfloat16* src = static_cast<const __nv_bfloat16*>(in) + node * 16;
      cp_async16(smem + off, src, in_grid ? 16 : 0);
      cp_async16(smem + kPlane3 + off, src + 8, in_grid ? 16 : 0);
    } else {
      float v[16];
      const float4* src = reinterpret_cast<const float4*>(static_cast<const float*>(in) + node * 16);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float4 f = in_grid ? src[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        v[4 * q] = f.x;
        v[4 * q + 1] = f.y;
        v[4 * q + 2] = f.z;
        v[4 * q + 3] = f.w;
      }
      float hi[16], lo[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) tc::split_bf16(v[c], hi[c], lo[c]);
#pragma unroll
      for (int pl = 0; pl < 4; ++pl) {
        const float* w = pl < 2 ? hi + 8 * pl : lo + 8 * (pl - 2);
        *reinterpret_cast<uint4*>(smem + pl * kPlane3 + off) =
            make_uint4(tc::pack_bf16x2(w[0], w[1]), tc::pack_bf16x2(w[2], w[3]), tc::pack_bf16x2(w[4], w[5]),
                       tc::pack_bf16x2(w[6], w[7]));
      }
    }
  }
  cp_async_wait_all();
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  // Output row r takes the staged rows sy = r .. r + 2; the MMAs go by
  // staged row (sy outer, then sz, then the x shift sx), and the y-taps that
  // one staged row feeds are stacked along N (weights packed y-tap-fastest)
  // into the outputs' TMEM blocks: forward, ky = sy - r, block column
  // 16 (R - 1 - r), descending in r; gradient, ky = r + 2 - sy, column 16 r.
  // An output's first contribution (sy = r, sz = sx = 0, hi plane) sets its
  // block; everything else accumulates.  Commit per staged row: output r is
  // complete with the commit of sy = r + 2.
  if (tid == 0) {
    const uint32_t s0 = tc::smem_u32(smem), w0 = tc::smem_u32(smem + S::kWOff);
    for (int sy = 0; sy < kR3 + 2; ++sy) {
      const int lo = MODE == 0 ? (sy - kR3 + 1 > 0 ? sy - kR3 + 1 : 0) : (2 - sy > 0 ? 2 - sy : 0);
      const int hi = MODE == 0 ? (sy < 2 ? sy : 2) : (kR3 + 1 - sy < 2 ? kR3 + 1 - sy : 2);
      for (int sz = 0; sz < 3; ++sz) {
        for (int sx = 0; sx < 3; ++sx) {
          const int kz = MODE == 0 ? sz : 2 - sz, kx = MODE == 0 ? sx : 2 - sx;
          const uint32_t a = s0 + (uint32_t)(((sz * (kR3 + 2) + sy) * kXS3 + sx) * 16);
          const uint32_t wt = w0 + (uint32_t)((kz * 3 + kx) * 3) * 512;   // the tile of ky = 0
          // output block of tap ky (column of the output it feeds)
          auto col = [&](int ky) { return MODE == 0 ? 16 * (kR3 - 1 - (sy - ky)) : 16 * (sy + ky - 2); };
          int l = lo, h = hi;
          if (sz == 0 && sx == 0 && sy < kR3) {   // output sy's first contribution
            const int kf = MODE == 0 ? 0 : 2;
            const uint64_t bf = tc::sdesc(wt + kf * 512, 128, 256);
            tc::mma_bf16(tmem + col(kf), tc::sdesc(a, kPlane3, 128), bf, tc::idesc_bf16(128, 16), 0u);
            if (MODE == 1)
              tc::mma_bf16(tmem + col(kf), tc::sdesc(a + 2 * kPlane3, kPlane3, 128), bf, tc::idesc_bf16(128, 16), 1u);
            if (MODE == 0) l = 1;
            else h = 1;
          }
          if (l <= h) {
            const uint64_t bd = tc::sdesc(wt + l * 512, 128, 256);
            const uint32_t id = tc::idesc_bf16(128, 16 * (h - l + 1));
            const uint32_t d = tmem + col(l);   // columns ascend with ky in both orientations
            tc::mma_bf16(d, tc::sdesc(a, kPlane3, 128), bd, id, 1u);
            if (MODE == 1) tc::mma_bf16(d, tc::sdesc(a + 2 * kPlane3, kPlane3, 128), bd, id, 1u);
          }
        }
      }
      tc::mma_commit(tc::smem_u32(bar + sy));
    }
  }
  bool failed = false;
  const int x = x0 + tid;
  const double zs = (LAST && state) ? state->rnorm : 1.0;
  for (int r = 0; r < kR3; ++r) {
    const bool ok = tc::mbar_wait(tc::smem_u32(bar + r + 2), 0u, c_wait_first3);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after();
    float v[16];
    const int col = MODE == 0 ? 16 * (kR3 - 1 - r) : 16 * r;
    tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)col, v);
    const int y = y0 + r;
    if (!inside3(g, x, y, z)) continue;   // pads keep their zeros
    const long long t = x + px * y + pxy * z;
    const long long node = abase + t;
    if (MODE == 1) {
      const uint4* m = reinterpret_cast<const uint4*>(act_in + node * 16);
      const uint4 m0 = m[0], m1 = m[1];
      const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
      float o[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const unsigned short hb = (unsigned short)(c & 1 ? mw[c >> 1] >> 16 : mw[c >> 1] & 0xFFFFu);
        o[c] = (c < cin && __bfloat162float(__ushort_as_bfloat16(hb)) > 0.f) ? v[c] : 0.f;
      }
      float4* dst = reinterpret_cast<float4*>(static_cast<float*>(out) + node * 16);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    } else if (LAST) {
      // components a = 0..2 of node t in the vector layout of the grid
      const long long vb = (long long)b * g.len + g.G + t;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (yv) yv[vb + a * g.cstride] = v[a];
        if (zv) zv[vb + a * g.cstride] = (T)(zs * (double)v[a]);
      }
    } else {
      uint32_t q[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float a0 = RELU ? fmaxf(v[2 * k], 0.f) : v[2 * k];
        const float a1 = RELU ? fmaxf(v[2 * k + 1], 0.f) : v[2 * k + 1];
        q[k] = tc::pack_bf16x2(2 * k < cout ? a0 : 0.f, 2 * k + 1 < cout ? a1 : 0.f);
      }
      uint4* dst = reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(out) + node * 16);
      dst[0] = make_uint4(q[0], q[1], q[2], q[3]);
      dst[1] = make_uint4(q[4], q[5], q[6], q[7]);
    }
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    // the last commit covers every MMA issued: let them finish (bounded)
    tc::mbar_wait(tc::smem_u32(bar + kR3 + 1), 0u, kWait3);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 64);
}

// Network input: channels 0..2 = bf16(r_a * s), s = 1 / ||r|| from the
// solver state (or 1), channels 3..15 zero; grid nodes only.
template <typename T>
__global__ void k_net3_input(GridDesc g, int B, const T* __restrict__ r, long long r_ld, const DevState* state,
                             __nv_bfloat16* __restrict__ a0) {
  if (state && state->done) return;
  const float s = state ? (float)(state->rnorm > 0.0 ? 1.0 / state->rnorm : 0.0) : 1.f;
  const long long alen = act_len3(g);
  const long long total = (long long)B * g.cstride;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(u / g.cstride);
    const long long t = u - (long long)b * g.cstride;
    const int x = (int)(t % g.px), y = (int)((t / g.px) % g.py), z = (int)(t / g.pxy);
    if (!inside3(g, x, y, z)) continue;
    const T* rb = r + (long long)b * r_ld + g.G + t;
    float v[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) v[a] = (float)rb[a * g.cstride] * s;
    uint4* dst = reinterpret_cast<uint4*>(a0 + ((long long)b * alen + g.G + t) * 16);
    dst[0] = make_uint4(tc::pack_bf16x2(v[0], v[1]), tc::pack_bf16x2(v[2], 0.f), 0u, 0u);
    dst[1] = make_uint4(0u, 0u, 0u, 0u);
  }
}

// dOut of the last layer: the vector-layout dL/dy to [B][act_len][16] FP32
// (channels 0..2).
__global__ void k_net3_dy_channels(GridDesc g, int B, const float* __restrict__ dy, float* __restrict__ d) {
  const long long alen = act_len3(g);
  const long long total = (long long)B * g.cstride;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(u / g.cstride);
    const long long t = u - (long long)b * g.cstride;
    const int x = (int)(t % g.px), y = (int)((t / g.px) % g.py), z = (int)(t / g.pxy);
    if (!inside3(g, x, y, z)) continue;
    float4* dst = reinterpret_cast<float4*>(d + ((long long)b * alen + g.G + t) * 16);
    const float* src = dy + (long long)b * g.len + g.G + t;
    dst[0] = make_float4(src[0], src[g.cstride], src[2 * g.cstride], 0.f);
  }
}

// Weight gradient, 27 taps: see the file comment.
constexpr int kWChunk3 = 64;
constexpr int kWA3 = 128 * kWChunk3 * 2;      // 16 KB
constexpr int kWB3 = 432 * kWChunk3 * 2;      // 54 KB
constexpr int kWStage3 = kWA3 + kWB3;
constexpr int kWSmem3 = 2 * kWStage3 + 64;    // 140 KB: one CTA per SM (its 512 TMEM columns)

__device__ __forceinline__ int toff64(int row, int k) {
  return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__global__ void __launch_bounds__(kT3, 1)
    k_net3_wgrad_tc(GridDesc g, int cin, int cout, int chunks_per_block, int blocks_per_image,
                    const float* __restrict__ dOut, const __nv_bfloat16* __restrict__ act, double* part, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kWStage3);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * kWStage3 + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x / blocks_per_image, blk = blockIdx.x % blocks_per_image;
  const long long nchunks = (g.cstride + kWChunk3 - 1) / kWChunk3;
  const long long c0 = (long long)blk * chunks_per_block;
  long long c1 = c0 + chunks_per_block;
  if (c1 > nchunks) c1 = nchunks;
  const int n = c0 < c1 ? (int)(c1 - c0) : 0;
  const long long alen = act_len3(g);
  const long long abase = (long long)b * alen + g.G;

  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), 512);
  if (tid < 2) tc::mbar_init(tc::smem_u32(bar + tid));
  if (tid == 0) tc::mbar_init_fence();
  for (int i = tid; i < 2 * kWA3 / 16; i += kT3) {
    const int st = i / (kWA3 / 16), j = i % (kWA3 / 16);
    reinterpret_cast<uint4*>(smem + st * kWStage3)[j] = make_uint4(0, 0, 0, 0);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = tc::idesc_bf16(128, 144);
  bool failed = false;
  int issued = 0;   // chunks whose MMAs were issued
  for (int i = 0; i < n && !failed; ++i) {
    const int st = i & 1;
    unsigned char* A = smem + st * kWStage3;
    unsigned char* Bt = A + kWA3;
    if (i >= 2) {
      const bool ok = tc::mbar_wait(tc::smem_u32(bar + st), (uint32_t)(((i - 2) >> 1) & 1), c_wait_first3);
      failed = __syncthreads_or(!ok);
      if (failed) break;
      tc::fence_after();
    }
    const long long t0 = (c0 + i) * kWChunk3;
    // A: dOut^T, hi rows co, lo rows 16 + co (16 channels, zero beyond
    // cout); thread = (point of the chunk, channel half)
    {
      const int pt = tid & (kWChunk3 - 1), h = tid / kWChunk3;
      const long long t = t0 + pt;
      float4 f0 = make_float4(0.f, 0.f, 0.f, 0.f), f1 = f0;
      if (t < g.cstride) {
        const float4* src = reinterpret_cast<const float4*>(dOut + (abase + t) * 16 + 8 * h);
        f0 = src[0];
        f1 = src[1];
      }
      const float d[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int co = 8 * h + c;
        float hi, lo;
        tc::split_bf16(co < cout ? d[c] : 0.f, hi, lo);
        *reinterpret_cast<__nv_bfloat16*>(A + toff64(co, pt)) = __float2bfloat16_rn(hi);
        *reinterpret_cast<__nv_bfloat16*>(A + toff64(16 + co, pt)) = __float2bfloat16_rn(lo);
      }
    }
    // B: im2col rows (tap, ci), 27 taps x 2 channel halves x 8 point groups
    for (int item = tid; item < 27 * 2 * 8; item += kT3) {
      const int tap = item / 16, half = (item / 8) % 2, pg = item % 8;
      const int kz = tap / 9, ky = (tap / 3) % 3, kx = tap % 3;
      const long long off = (kx - 1) + (long long)(ky - 1) * g.px + (long long)(kz - 1) * g.pxy;
      uint32_t w[8][4];
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const long long t = t0 + pg * 8 + kk;
        if (t >= g.cstride) {
#pragma unroll
          for (int j = 0; j < 4; ++j) w[kk][j] = 0u;
        } else {
          const uint4 v = *reinterpret_cast<const uint4*>(act + (abase + t + off) * 16 + half * 8);
          w[kk][0] = v.x; w[kk][1] = v.y; w[kk][2] = v.z; w[kk][3] = v.w;
        }
      }
#pragma unroll
      for (int ci = 0; ci < 8; ++ci) {
        const unsigned sel = (ci & 1) ? 0x7632u : 0x5410u;
        const int wi = ci >> 1;
        *reinterpret_cast<uint4*>(Bt + toff64(tap * 16 + half * 8 + ci, pg * 8)) =
            make_uint4(__byte_perm(w[0][wi], w[1][wi], sel), __byte_perm(w[2][wi], w[3][wi], sel),
                       __byte_perm(w[4][wi], w[5][wi], sel), __byte_perm(w[6][wi], w[7][wi], sel));
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      const uint32_t a_addr = tc::smem_u32(A), b_addr = tc::smem_u32(Bt);
#pragma unroll
      for (int ks = 0; ks < kWChunk3 / 16; ++ks)
#pragma unroll
        for (int part3 = 0; part3 < 3; ++part3)   // taps 9 part3 .. 9 part3 + 8: B rows from 144 part3
          tc::mma_bf16(tmem + 144 * part3, tc::sdesc(a_addr + ks * 256, 128, 1024),
                       tc::sdesc(b_addr + part3 * 18 * 1024 + ks * 256, 128, 1024), idesc, (i > 0 || ks > 0) ? 1u : 0u);
      tc::mma_commit(tc::smem_u32(bar + st));
    }
    issued = i + 1;
  }
  // every MMA issued has completed once the last issued commit has
  bool drained = true;
  if (issued > 0) {
    const int last = issued - 1;
    drained = tc::mbar_wait(tc::smem_u32(bar + (last & 1)), (uint32_t)((last >> 1) & 1), kWait3);
    if (!drained && issued > 1)
      tc::mbar_wait(tc::smem_u32(bar + ((last - 1) & 1)), (uint32_t)(((last - 1) >> 1) & 1), kWait3);
  }
  failed = __syncthreads_or(failed || !drained);
  tc::fence_after();
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
  } else if (warp == 0) {
#pragma unroll 1
    for (int j = 0; j < 432 / 16; ++j) {
      float v[16];
      if (n > 0) tc::tmem_ld16(tmem + 16 * j, v);
      else {
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = 0.f;
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const float lo = __shfl_down_sync(0xffffffffu, v[c], 16);
        const int ncol = 16 * j + c, tap = ncol / 16, ci = ncol % 16, co = lane;
        if (lane < cout && ci < cin)
          part[(long long)((co * cin + ci) * 27 + tap) * gridDim.x + blockIdx.x] = (double)v[c] + (double)lo;
      }
    }
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

constexpr int kWCpb3 = 16;   // 64-node chunks per CTA

__global__ void k_net3_acts_export(GridDesc g, int B, NetActs a, float* out) {
  const long long alen = act_len3(g);
  const long long nn = (long long)g.nx * g.ny * g.nz;
  const long long total = 4LL * B * nn;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < total;
       u += (long long)gridDim.x * blockDim.x) {
    const int L = (int)(u / (B * nn));
    const int b = (int)((u / nn) % B);
    const long long q = u % nn;
    const int x = (int)(q % g.nx), y = (int)((q / g.nx) % g.ny), z = (int)(q / ((long long)g.nx * g.ny));
    const long long node = (long long)b * alen + g.G + x + g.px * (long long)y + g.pxy * (long long)z;
    const __nv_bfloat16* src = L == 0 ? a.a0 : L == 1 ? a.a1 : L == 2 ? a.a2 : a.a3;
    float* o = out + u * 16;
    for (int c = 0; c < 16; ++c) o[c] = __bfloat162float(src[node * 16 + c]);
  }
}

}  // namespace

void launch_net3_acts_export(const GridDesc& g, int B, NetActs acts, float* out, cudaStream_t s) {
  k_net3_acts_export<<<grid_for(4LL * B * g.nx * g.ny * g.nz, 4096), kBlock, 0, s>>>(g, B, acts, out);
}

long long net3_act_len(const GridDesc& g) { return act_len3(g); }

int net3_wgrad_blocks(const GridDesc& g, int B) {
  const long long nchunks = (g.cstride + kWChunk3 - 1) / kWChunk3;
  return B * (int)((nchunks + kWCpb3 - 1) / kWCpb3);
}

cudaError_t set_wait_first_net3(long long polls) {
  return cudaMemcpyToSymbol(c_wait_first3, &polls, sizeof(polls));
}

int net3_pack_bytes() { return 8 * kW3Bytes; }

void launch_net3_pack(const float* wq, unsigned char* wp, cudaStream_t s) {
  k_net3_pack<<<(8 * 27 * 256 + kBlock - 1) / kBlock, kBlock, 0, s>>>(wq, wp);
}

void net3_prepare_attributes() {
  cudaFuncSetAttribute(k_net3_conv_tc<0, true, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Conv3Smem<2>::kBytes);
  cudaFuncSetAttribute(k_net3_conv_tc<0, false, true, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Conv3Smem<2>::kBytes);
  cudaFuncSetAttribute(k_net3_conv_tc<0, false, true, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Conv3Smem<2>::kBytes);
  cudaFuncSetAttribute(k_net3_conv_tc<0, false, true, dw>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Conv3Smem<2>::kBytes);
  cudaFuncSetAttribute(k_net3_conv_tc<1, false, false, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       Conv3Smem<4>::kBytes);
  cudaFuncSetAttribute(k_net3_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem3);
}

// Forward pass of nimg images: r (type T, vector layout, image stride r_ld,
// scaled by 1 / ||r|| from state when given) -> acts.a0..a3 (bfloat16) and
// y (float, vector layout, may be null) and/or z = ||r|| y (T, may be null);
// wp: the weights packed by launch_net3_pack.
template <typename T>
void launch_net3_forward(const GridDesc& g, int B, const T* r, long long r_ld, const unsigned char* wp,
                         const DevState* state, NetActs acts, float* y, T* z, int* err, cudaStream_t s) {
  const long long total = (long long)B * g.cstride;
  k_net3_input<T><<<grid_for(total, 4096), kBlock, 0, s>>>(g, B, r, r_ld, state, acts.a0);
  const dim3 grid((unsigned)((g.px + 127) / 128), (unsigned)((g.py + kR3 - 1) / kR3), (unsigned)(g.pz * B));
  const int sm2 = Conv3Smem<2>::kBytes;
  const unsigned char* w[4] = {wp, wp + 2 * kW3Bytes, wp + 4 * kW3Bytes, wp + 6 * kW3Bytes};
  k_net3_conv_tc<0, true, false, float><<<grid, kT3, sm2, s>>>(g, B, acts.a0, w[0], 3, 16, nullptr, acts.a1,
                                                               nullptr, nullptr, state, err);
  k_net3_conv_tc<0, true, false, float><<<grid, kT3, sm2, s>>>(g, B, acts.a1, w[1], 16, 16, nullptr, acts.a2,
                                                               nullptr, nullptr, state, err);
  k_net3_conv_tc<0, true, false, float><<<grid, kT3, sm2, s>>>(g, B, acts.a2, w[2], 16, 16, nullptr, acts.a3,
                                                               nullptr, nullptr, state, err);
  k_net3_conv_tc<0, false, true, T><<<grid, kT3, sm2, s>>>(g, B, acts.a3, w[3], 16, 3, nullptr, nullptr, y, z,
                                                           state, err);
}
template void launch_net3_forward<float>(const GridDesc&, int, const float*, long long, const unsigned char*,
                                         const DevState*, NetActs, float*, float*, int*, cudaStream_t);
template void launch_net3_forward<double>(const GridDesc&, int, const double*, long long, const unsigned char*,
                                          const DevState*, NetActs, float*, double*, int*, cudaStream_t);
template void launch_net3_forward<dw>(const GridDesc&, int, const dw*, long long, const unsigned char*,
                                      const DevState*, NetActs, float*, dw*, int*, cudaStream_t);

// Backward pass: dy (vector layout) -> weight-gradient partials per layer
// (stride net3_wgrad_blocks) and the data gradients d3, d2, d1 ([B][act_len][16]).
void launch_net3_backward(const GridDesc& g, int B, const unsigned char* wp, NetActs acts, const float* dy,
                          NetGrads gr, float* d4, int* err, cudaStream_t s) {
  const long long total = (long long)B * g.cstride;
  k_net3_dy_channels<<<grid_for(total, 4096), kBlock, 0, s>>>(g, B, dy, d4);
  const long long nchunks = (g.cstride + kWChunk3 - 1) / kWChunk3;
  const int bpi = (int)((nchunks + kWCpb3 - 1) / kWCpb3);
  const dim3 wgrid((unsigned)(B * bpi));
  const dim3 grid((unsigned)((g.px + 127) / 128), (unsigned)((g.py + kR3 - 1) / kR3), (unsigned)(g.pz * B));
  const int sm4 = Conv3Smem<4>::kBytes;
  const unsigned char* wg[4] = {wp + kW3Bytes, wp + 3 * kW3Bytes, wp + 5 * kW3Bytes, wp + 7 * kW3Bytes};
  k_net3_wgrad_tc<<<wgrid, kT3, kWSmem3, s>>>(g, 16, 3, kWCpb3, bpi, d4, acts.a3, gr.part[3], err);
  k_net3_conv_tc<1, false, false, float><<<grid, kT3, sm4, s>>>(g, B, d4, wg[3], 16, 3, acts.a3, gr.d3, nullptr,
                                                                nullptr, nullptr, err);
  k_net3_wgrad_tc<<<wgrid, kT3, kWSmem3, s>>>(g, 16, 16, kWCpb3, bpi, gr.d3, acts.a2, gr.part[2], err);
  k_net3_conv_tc<1, false, false, float><<<grid, kT3, sm4, s>>>(g, B, gr.d3, wg[2], 16, 16, acts.a2, gr.d2,
                                                                nullptr, nullptr, nullptr, err);
  k_net3_wgrad_tc<<<wgrid, kT3, kWSmem3, s>>>(g, 16, 16, kWCpb3, bpi, gr.d2, acts.a1, gr.part[1], err);
  k_net3_conv_tc<1, false, false, float><<<grid, kT3, sm4, s>>>(g, B, gr.d2, wg[1], 16, 16, acts.a1, gr.d1,
                                                                nullptr, nullptr, nullptr, err);
  k_net3_wgrad_tc<<<wgrid, kT3, kWSmem3, s>>>(g, 3, 16, kWCpb3, bpi, gr.d1, acts.a0, gr.part[0], err);
}

}  // namespace mpcg
