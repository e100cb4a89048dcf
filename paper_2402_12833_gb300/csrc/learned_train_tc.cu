// Training kernels of the learned column on the fifth-generation tensor
// cores: the weight gradient as a pixel-reduction GEMM and the data gradient
// as a transposed implicit GEMM.
//
// Weight gradient of a 3x3 layer CIN -> COUT (both <= 16):
//   dW[co][ci][tap] = sum over images b and points p of
//                     dOut_b(p)[co] * act_b(p + off(tap))[ci],
// i.e. D = A B^T with A = dOut^T (rows co, K = points) and B = the im2col of
// the layer input (rows (tap, ci), K = points), reduced over K in TMEM.
// dOut is FP32; it enters the bfloat16 MMA as hi + lo (hi = bf16(d),
// lo = bf16(d - hi), 16 significant bits): rows 0-15 of A hold hi, rows
// 16-31 lo, rows 32-127 zero (M = 128), and the epilogue adds row co and
// row 16 + co.  The activations are bfloat16 already, so every product is
// exact and the FP32 accumulation is the only rounding besides the split.
// Each CTA reduces a run of 64-point chunks of one image: per chunk the
// threads stage A (8-point x 8-row core matrices, transposed from the
// point-major dOut) and B (the nine shifted windows of the layer input,
// transposed likewise), one thread issues four MMAs (K = 16 points each,
// M = 128, N = 144 = 9 taps x 16 channels) and commits them to the stage's
// mbarrier; two stages let the staging of chunk i + 1 overlap the MMAs of
// chunk i.  Points beyond the padded box contribute zero (dOut is read as
// zero there); the layer input is read in the vector's zero guards, as the
// zero padding of the convolution.
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.cuh"
#include "tc.cuh"

namespace mpcg {

namespace {

constexpr int kWT = 128;                 // threads (four warps: TMEM lanes 0..127)
constexpr int kChunk = 64;               // points per chunk (K of four MMAs)
constexpr int kM = 128;
constexpr int kN = 144;                  // 9 taps x 16 input channels
constexpr int kABytes = kM * kChunk * 2;     // 16 KB
constexpr int kBBytes = kN * kChunk * 2;     // 18 KB
constexpr int kStage = kABytes + kBBytes;
// 80 KB of dynamic shared memory (the two stages take 68 KB): at most two
// CTAs share an SM, so their 2 x 256 TMEM columns always fit and no
// allocation waits for another CTA to finish
constexpr int kWSmem = 80 * 1024;
constexpr int kWTmemCols = 256;
constexpr long long kWaitLimitW = 1LL << 22;
// polls of a first wait before a kernel gives up (set_wait_first_train; the
// drain after a give-up always uses kWaitLimitW)
__constant__ long long c_wait_first_w = kWaitLimitW;

// byte offset of element (row, k) in a tile of 64 K columns: core matrices
// of 8 rows x 8 k (128 B), K-adjacent (LBO = 128 B), row groups 1024 B apart
__device__ __forceinline__ int toff(int row, int k) {
  return (row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kWT, 2)
    k_net_wgrad_tc(GridDesc g, int chunks_per_block, int blocks_per_image, const float* __restrict__ dOut,
                   const __nv_bfloat16* __restrict__ act, double* part, int* err) {
  static_assert(CIN <= 16 && COUT <= 16, "at most 16 channels");
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * kStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + 2 * kStage + 16);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x / blocks_per_image, blk = blockIdx.x % blocks_per_image;
  const long long nchunks = (g.npts + kChunk - 1) / kChunk;
  const long long c0 = (long long)blk * chunks_per_block;
  long long c1 = c0 + chunks_per_block;
  if (c1 > nchunks) c1 = nchunks;
  const int n = c0 < c1 ? (int)(c1 - c0) : 0;
  const long long base = (long long)b * g.len + g.G;
  const long long p = g.p;

  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kWTmemCols);
  if (tid < 2) tc::mbar_init(tc::smem_u32(bar + tid));
  if (tid == 0) tc::mbar_init_fence();
  // rows 32..127 of A stay zero in both stages
  for (int i = tid; i < 2 * kABytes / 16; i += kWT) {
    const int st = i / (kABytes / 16), j = i % (kABytes / 16);
    reinterpret_cast<uint4*>(smem + st * kStage)[j] = make_uint4(0, 0, 0, 0);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = tc::idesc_bf16(kM, kN);
  bool failed = false;
  int issued = 0;   // chunks whose MMAs were issued

  for (int i = 0; i < n && !failed; ++i) {
    const int st = i & 1;
    unsigned char* A = smem + st * kStage;
    unsigned char* Bt = A + kABytes;
    if (i >= 2) {   // the MMAs of chunk i - 2 read this stage
      const bool ok = tc::mbar_wait(tc::smem_u32(bar + st), (uint32_t)(((i - 2) >> 1) & 1), c_wait_first_w);
      failed = __syncthreads_or(!ok);
      if (failed) break;
      tc::fence_after();
    }
    const long long t0 = (c0 + i) * kChunk;
    // A: one core-matrix column (8 points) of one 8-channel group per item;
    // hi rows cg*8 + c, lo rows 16 + cg*8 + c
    constexpr int CG = (COUT + 7) / 8;
    for (int item = tid; item < CG * 8; item += kWT) {
      const int cg = item / 8, pg = item % 8;
#pragma unroll 1
      for (int c = 0; c < 8; ++c) {
        const int co = cg * 8 + c;
        float hi[8], lo[8];
#pragma unroll
        for (int kk = 0; kk < 8; ++kk) {
          const long long t = t0 + pg * 8 + kk;
          const float d = (t < g.npts && co < COUT) ? dOut[(base + t) * COUT + co] : 0.f;
          tc::split_bf16(d, hi[kk], lo[kk]);
        }
        const uint4 vh = make_uint4(tc::pack_bf16x2(hi[0], hi[1]), tc::pack_bf16x2(hi[2], hi[3]),
                                    tc::pack_bf16x2(hi[4], hi[5]), tc::pack_bf16x2(hi[6], hi[7]));
        const uint4 vl = make_uint4(tc::pack_bf16x2(lo[0], lo[1]), tc::pack_bf16x2(lo[2], lo[3]),
                                    tc::pack_bf16x2(lo[4], lo[5]), tc::pack_bf16x2(lo[6], lo[7]));
        *reinterpret_cast<uint4*>(A + toff(co, pg * 8)) = vh;
        *reinterpret_cast<uint4*>(A + toff(16 + co, pg * 8)) = vl;
      }
    }
    // B: rows (tap, ci), the layer input at the tap's offset, 8 points per core matrix
    for (int item = tid; item < 9 * 2 * 8; item += kWT) {
      const int tap = item / 16, half = (item / 8) % 2, pg = item % 8;
      const long long off = (tap % 3 - 1) + (long long)(tap / 3 - 1) * p;
      uint32_t w[8][4];   // [point][channel pair]
#pragma unroll
      for (int kk = 0; kk < 8; ++kk) {
        const long long t = t0 + pg * 8 + kk;
        const long long q = base + t + off;
        if (t >= g.npts) {   // beyond the box: dOut is zero there; stay inside the guards
#pragma unroll
          for (int j = 0; j < 4; ++j) w[kk][j] = 0u;
        } else if (CIN == 16) {
          const uint4 v = *reinterpret_cast<const uint4*>(act + q * 16 + half * 8);
          w[kk][0] = v.x; w[kk][1] = v.y; w[kk][2] = v.z; w[kk][3] = v.w;
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j) w[kk][j] = 0u;
          if (half == 0) {
#pragma unroll
            for (int c = 0; c < CIN; c += 2) {
              const __nv_bfloat16 a0 = act[q * CIN + c];
              const __nv_bfloat16 a1 = c + 1 < CIN ? act[q * CIN + c + 1] : __float2bfloat16_rn(0.f);
              w[kk][c / 2] = (uint32_t)__bfloat16_as_ushort(a0) | ((uint32_t)__bfloat16_as_ushort(a1) << 16);
            }
          }
        }
      }
      // transpose: row ci of the core matrix holds the 8 points of channel ci
#pragma unroll
      for (int ci = 0; ci < 8; ++ci) {
        const unsigned sel = (ci & 1) ? 0x7632u : 0x5410u;
        const int wi = ci >> 1;
        const uint4 r = make_uint4(__byte_perm(w[0][wi], w[1][wi], sel), __byte_perm(w[2][wi], w[3][wi], sel),
                                   __byte_perm(w[4][wi], w[5][wi], sel), __byte_perm(w[6][wi], w[7][wi], sel));
        *reinterpret_cast<uint4*>(Bt + toff(tap * 16 + half * 8 + ci, pg * 8)) = r;
      }
    }
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      const uint32_t a_addr = tc::smem_u32(A), b_addr = tc::smem_u32(Bt);
#pragma unroll
      for (int ks = 0; ks < kChunk / 16; ++ks)
        tc::mma_bf16(tmem, tc::sdesc(a_addr + ks * 256, 128, 1024), tc::sdesc(b_addr + ks * 256, 128, 1024), idesc,
                     (i > 0 || ks > 0) ? 1u : 0u);
      tc::mma_commit(tc::smem_u32(bar + st));
    }
    issued = i + 1;
  }
  // every MMA issued has completed once the last issued commit has
  bool drained = true;
  if (issued > 0) {
    const int last = issued - 1;
    drained = tc::mbar_wait(tc::smem_u32(bar + (last & 1)), (uint32_t)((last >> 1) & 1), kWaitLimitW);
    if (!drained && issued > 1)
      tc::mbar_wait(tc::smem_u32(bar + ((last - 1) & 1)), (uint32_t)(((last - 1) >> 1) & 1), kWaitLimitW);
  }
  failed = __syncthreads_or(failed || !drained);
  tc::fence_after();
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
  } else if (warp == 0) {
    // lane r < 16: row r (hi) plus row 16 + r (lo) of every column
#pragma unroll 1
    for (int j = 0; j < kN / 16; ++j) {
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
        if (lane < COUT && ci < CIN)
          part[(long long)((co * CIN + ci) * 9 + tap) * gridDim.x + blockIdx.x] = (double)v[c] + (double)lo;
      }
    }
  }
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kWTmemCols);
}

// Data gradient through a layer whose input has 16 channels and output COUT
// (16, or 1 for the last layer):
//   dIn(p)[ci] = [act_in(p)[ci] > 0] * sum_tap sum_co W[co][ci][tap] dOut(p - off(tap))[co],
// the transposed convolution masked by the ReLU pattern of the layer below.
// A CTA owns R = 8 rows of 128 points of one image; the R + 2 rows of dOut
// around them (x from -1 to 128) are staged once as four bfloat16 planes
// (hi channels 0-7, hi 8-15, lo 0-7, lo 8-15; hi = bf16(d), lo = bf16(d - hi)).
// Output row r takes the staged rows r .. r + 2 (tap ky = r + 2 - row) at
// the x shift 2 - kx.  The MMAs go by staged row and shift: the A operand is
// the staged row shifted (SBO = 128 B, LBO = one plane) and B stacks the
// 16 x 16 weight tiles of the y-taps that row feeds along N (tiles packed
// ky-fastest), into the outputs' 16-column TMEM blocks (column 16 r,
// ascending with ky); hi planes and lo planes are two MMAs.  An output's
// first contribution (its own staged row, shift 0, hi planes) sets its
// block; one commit per staged row, output r complete with staged row r + 2.
constexpr int kDR = 8;                   // output rows per CTA
constexpr int kDXS = 130;                // stored points per row: x = -1 .. 128
constexpr int kDPlane = (kDR + 2) * kDXS * 16;
constexpr int kDWOff = 4 * kDPlane;      // weight tiles
constexpr int kDBarOff = kDWOff + 9 * 512;
constexpr int kDSmem = kDBarOff + 8 * (kDR + 2) + 16;
constexpr int kDTmemCols = 128;

__device__ __forceinline__ int canon16(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

template <int COUT>
__global__ void __launch_bounds__(kWT, 2)
    k_net_dgrad_tc(GridDesc g, const float* __restrict__ dOut, const float* __restrict__ W,
                   const __nv_bfloat16* __restrict__ act_in, float* __restrict__ dIn, int* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kDBarOff);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kDBarOff + 8 * (kDR + 2));
  const int tid = threadIdx.x, warp = tid >> 5;
  const int x0 = blockIdx.x * 128, y0 = blockIdx.y * kDR, b = blockIdx.z;
  const int n1 = g.n1;
  const long long p = g.p;
  const long long base = (long long)b * g.len + g.G;

  if (warp == 0) tc::tmem_alloc(tc::smem_u32(tmem_slot), kDTmemCols);
  if (tid < kDR + 2) tc::mbar_init(tc::smem_u32(bar + tid));
  if (tid == 0) tc::mbar_init_fence();
  // weight tiles: tap t = ky * 3 + kx at tile kx * 3 + ky, row n = ci, column k = co
  for (int e = tid; e < 9 * 256; e += kWT) {
    const int t = e / 256, ci = (e / 16) % 16, co = e % 16;
    const float w = co < COUT ? W[(co * 16 + ci) * 9 + t] : 0.f;
    *reinterpret_cast<__nv_bfloat16*>(smem + kDWOff + ((t % 3) * 3 + t / 3) * 512 + canon16(ci, co)) =
        __float2bfloat16_rn(w);
  }
  // dOut rows y0 - 1 .. y0 + kDR, x0 - 1 .. x0 + 128 (zero outside the grid)
  for (int e = tid; e < (kDR + 2) * kDXS; e += kWT) {
    const int sr = e / kDXS, xs = e % kDXS;
    const int y = y0 - 1 + sr, x = x0 - 1 + xs;
    const bool in = x >= 0 && x < n1 && y >= 0 && y < n1;
    float hi[16], lo[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      const float d = (in && c < COUT) ? dOut[(base + (long long)y * p + x) * COUT + c] : 0.f;
      tc::split_bf16(d, hi[c], lo[c]);
    }
    const int off = (sr * kDXS + xs) * 16;
#pragma unroll
    for (int pl = 0; pl < 4; ++pl) {
      const float* v = pl < 2 ? hi + 8 * pl : lo + 8 * (pl - 2);
      *reinterpret_cast<uint4*>(smem + pl * kDPlane + off) =
          make_uint4(tc::pack_bf16x2(v[0], v[1]), tc::pack_bf16x2(v[2], v[3]), tc::pack_bf16x2(v[4], v[5]),
                     tc::pack_bf16x2(v[6], v[7]));
    }
  }
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  if (tid == 0) {
    const uint32_t s0 = tc::smem_u32(smem), w0 = tc::smem_u32(smem + kDWOff);
    for (int sr = 0; sr < kDR + 2; ++sr) {
      const int lo = 2 - sr > 0 ? 2 - sr : 0, hi = kDR + 1 - sr < 2 ? kDR + 1 - sr : 2;
#pragma unroll
      for (int sx = 0; sx < 3; ++sx) {
        const int kx = 2 - sx;
        const uint32_t a = s0 + (uint32_t)((sr * kDXS + sx) * 16);
        const uint64_t ah = tc::sdesc(a, kDPlane, 128), al = tc::sdesc(a + 2 * kDPlane, kDPlane, 128);
        int h = hi;
        if (sx == 0 && sr < kDR) {   // output sr's first contribution: tap ky = 2
          const uint64_t bf = tc::sdesc(w0 + (kx * 3 + 2) * 512, 128, 256);
          tc::mma_bf16(tmem + 16 * sr, ah, bf, tc::idesc_bf16(128, 16), 0u);
          tc::mma_bf16(tmem + 16 * sr, al, bf, tc::idesc_bf16(128, 16), 1u);
          h = 1;
        }
        if (lo <= h) {   // taps lo .. h into outputs sr + lo - 2 ..
          const uint64_t bd = tc::sdesc(w0 + (kx * 3 + lo) * 512, 128, 256);
          const uint32_t id = tc::idesc_bf16(128, 16 * (h - lo + 1));
          const uint32_t d = tmem + (uint32_t)(16 * (sr + lo - 2));
          tc::mma_bf16(d, ah, bd, id, 1u);
          tc::mma_bf16(d, al, bd, id, 1u);
        }
      }
      tc::mma_commit(tc::smem_u32(bar + sr));
    }
  }
  bool failed = false;
  const int x = x0 + tid;
  for (int r = 0; r < kDR; ++r) {
    const bool ok = tc::mbar_wait(tc::smem_u32(bar + r + 2), 0u, c_wait_first_w);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    tc::fence_after();
    float v[16];
    tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16 * r, v);
    const int y = y0 + r;
    if (x < p && y < p) {   // a point of the padded box
      const long long o = base + (long long)y * p + x;
      const bool in = x < n1 && y < n1;
      float out[16];
      if (in) {
        const uint4 m0 = *reinterpret_cast<const uint4*>(act_in + o * 16);
        const uint4 m1 = *reinterpret_cast<const uint4*>(act_in + o * 16 + 8);
        const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const unsigned short hb = (unsigned short)(c & 1 ? mw[c >> 1] >> 16 : mw[c >> 1] & 0xFFFFu);
          out[c] = __bfloat162float(__ushort_as_bfloat16(hb)) > 0.f ? v[c] : 0.f;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 16; ++c) out[c] = 0.f;
      }
      float4* dst = reinterpret_cast<float4*>(dIn + o * 16);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_float4(out[4 * q], out[4 * q + 1], out[4 * q + 2], out[4 * q + 3]);
    }
  }
  if (failed) {
    if (tid == 0) atomicExch(err, 1);
    // the last commit covers every MMA issued: let them finish (bounded)
    // before their memory is freed
    tc::mbar_wait(tc::smem_u32(bar + kDR + 1), 0u, kWaitLimitW);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kDTmemCols);
}

}  // namespace

void launch_net_dgrad_tc(const GridDesc& g, int B, int cout, const float* dOut, const float* W,
                         const __nv_bfloat16* act_in, float* dIn, int* err, cudaStream_t s) {
  const dim3 grid((unsigned)((g.p + 127) / 128), (unsigned)((g.p + kDR - 1) / kDR), (unsigned)B);
  if (cout == 1) k_net_dgrad_tc<1><<<grid, kWT, kDSmem, s>>>(g, dOut, W, act_in, dIn, err);
  else k_net_dgrad_tc<16><<<grid, kWT, kDSmem, s>>>(g, dOut, W, act_in, dIn, err);
}

int net_wgrad_tc_chunks_per_block() { return 16; }

int net_wgrad_tc_blocks(const GridDesc& g, int B) {
  const long long nchunks = (g.npts + kChunk - 1) / kChunk;
  const int cpb = net_wgrad_tc_chunks_per_block();
  return B * (int)((nchunks + cpb - 1) / cpb);
}

cudaError_t set_wait_first_train(long long polls) {
  return cudaMemcpyToSymbol(c_wait_first_w, &polls, sizeof(polls));
}

void net_train_tc_prepare_attributes() {
  cudaFuncSetAttribute(k_net_dgrad_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDSmem);
  cudaFuncSetAttribute(k_net_dgrad_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kDSmem);
  cudaFuncSetAttribute(k_net_wgrad_tc<kNetW, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem);
  cudaFuncSetAttribute(k_net_wgrad_tc<kNetW, kNetW>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem);
  cudaFuncSetAttribute(k_net_wgrad_tc<kNetIn, kNetC1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmem);
}

void launch_net_wgrad_tc(const GridDesc& g, int B, int layer, const float* dOut, const __nv_bfloat16* act,
                         double* part, int* err, cudaStream_t s) {
  const long long nchunks = (g.npts + kChunk - 1) / kChunk;
  const int cpb = net_wgrad_tc_chunks_per_block();
  const int bpi = (int)((nchunks + cpb - 1) / cpb);
  const dim3 grid((unsigned)(B * bpi));
  if (layer == 3) k_net_wgrad_tc<kNetW, 1><<<grid, kWT, kWSmem, s>>>(g, cpb, bpi, dOut, act, part, err);
  else if (layer == 0) k_net_wgrad_tc<kNetIn, kNetC1><<<grid, kWT, kWSmem, s>>>(g, cpb, bpi, dOut, act, part, err);
  else k_net_wgrad_tc<kNetW, kNetW><<<grid, kWT, kWSmem, s>>>(g, cpb, bpi, dOut, act, part, err);
}

}  // namespace mpcg
