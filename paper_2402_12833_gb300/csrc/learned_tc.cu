// Learned-column inference on the fifth-generation tensor cores: the whole
// four-layer network (3x3 convolutions 2 -> 16 -> 16 -> 16 -> 1, ReLU after
// the first three, zero padding, bfloat16 weights and activations, FP32
// accumulation) fused in one kernel per output tile.
//
// Each layer is an implicit GEMM over rows of 128 tile pixels (M = 128,
// K = 16 input channels): output row i takes the input rows i, i + 1, i + 2
// (the y-taps), each shifted by the x-tap.  The MMAs go by input row: for
// input row s and x-tap kx the A operand is row s shifted by kx, and the B
// operand stacks the 16 x 16 weight tiles of the y-taps that row feeds along
// N (16, 32 or 48), so the product lands in the TMEM blocks of up to three
// output rows at once (tcgen05.mma kind::f16, bf16 inputs, FP32 accumulator
// in tensor memory; see issue_slot).  One elected thread issues the MMAs
// with one tcgen05.commit per input row; eight warps read the accumulators
// back with tcgen05.ld (two warps per 32-lane quadrant, one per channel
// half), apply ReLU and the domain mask, round to bfloat16 and write the
// next layer's activations to shared memory.  Layer 1 has two input
// channels (zero-padded to 16), layer 4 one output channel (zero-padded
// weights, column 0 read).
//
// Tile: 120 x 8 output pixels with a 4-pixel halo (four layers of 3x3), i.e.
// 128 x 16 activation pixels; layer l computes rows l .. 15 - l, so the halo
// rows and columns become invalid one ring per layer and the central 120 x 8
// outputs are exact.  Pixels outside the problem's grid are held at zero in
// every layer (the zero padding of each convolution).
//
// Operand layouts (shared memory, K-major, no swizzle): a core matrix is 8
// rows x 16 bytes (8 bf16 of K) stored contiguously; the descriptor's
// leading byte offset (LBO) steps between the two K halves, the stride byte
// offset (SBO) between consecutive groups of 8 rows.  Activations are kept as
// two planes (channels 0-7 and 8-15) of [row][x + 1] pixels x 16 bytes, so
// the A operand of input row s at x-tap kx is simply the 128 consecutive
// pixels starting at (s, kx): SBO = 128 bytes, LBO = one plane.  The weights
// are packed once per attach into compact tiles ordered y-tap-fastest
// (LBO = 128, SBO = 256 bytes; consecutive tiles continue the N rows).  The
// activations are updated in place: input row q of layer L lives in slot
// q - L, and output row r is written to slot r - L - 1 (its slot as an input
// of layer L + 1) once it is complete -- with the commit of input row r + 1,
// by which time the MMAs reading slot r - L - 1 are done, since commits
// complete in issue order.  This halves the shared memory, so two CTAs share
// an SM and hide each other's latencies.
#include <cuda_bf16.h>
#include <stdint.h>

#include "kernels.cuh"

namespace mpcg {

namespace {

constexpr int kTW = 120;           // output tile width
constexpr int kTH = 8;             // output tile height
constexpr int kHalo = 4;
constexpr int kEW = kTW + 2 * kHalo;   // 128 = M of one MMA row
constexpr int kEH = kTH + 2 * kHalo;   // 16
constexpr int kXS = kEW + 2;           // stored row length: x = -1 and x = 128 are zero columns
constexpr int kNPix = kEH * kXS;       // pixels of one activation buffer
constexpr int kPlane = kNPix * 16;     // bytes of one channel plane
constexpr int kThreads = 256;          // eight warps: TMEM lanes 0..127, twice (channel halves)
constexpr int kMaxRows = kEH - 2;      // rows computed by the first layer
constexpr int kMaxSlots = kEH;         // input rows (slots) of the first layer: one mbarrier each
constexpr int kTmemCols = 256;         // one 16-column accumulator per output row of a layer (224 used)
constexpr long long kWaitLimit = 1LL << 22;

static_assert(2 * kEW == kThreads, "two threads per tile column: one per channel half");
static_assert(kEH == 16 && kThreads >= 64, "halo-column zeroing maps 16 rows x 2 sides x 2 planes");

// shared memory map (bytes): one activation buffer, updated in place
constexpr int kActBytes = 2 * kPlane;                // two planes
constexpr int kWBytes = 4 * 9 * 16 * 16 * 2;         // four layers x nine taps of B
constexpr int kOffAct0 = 0;
constexpr int kOffW = kOffAct0 + kActBytes;
constexpr int kOffBar = kOffW + kWBytes;
constexpr int kSmemBytes = kOffBar + 8 * kMaxSlots + 16;

// instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M = 128 (>> 4 at bits 24-28)
__host__ __device__ constexpr uint32_t idesc_n(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
}

// TMEM column of output row i of a layer: descending in i, so that the
// three y-taps of one input row land in three consecutive 16-column blocks
constexpr int kColTop = kMaxRows - 1;
__host__ __device__ constexpr int col_of(int i) { return 16 * (kColTop - i); }
static_assert(col_of(0) + 16 <= kTmemCols && col_of(kMaxRows - 1) == 0, "output blocks fit the TMEM allocation");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, LBO and SBO (all >> 4),
// descriptor version 1 at bits 46-47, base offset 0, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// byte offset of element (row, k) in a compact K-major tile of 16 columns
__host__ __device__ __forceinline__ int canon(int row, int k) {
  return (row >> 3) * 256 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// polls of a row's first wait before the kernel gives up (set_wait_first_infer;
// the drain after a give-up always uses kWaitLimit)
__constant__ long long c_wait_first = kWaitLimit;

// bounded wait; false if the phase did not complete within `limit` polls
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit = kWaitLimit) {
  for (long long i = 0; i < limit; ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// 8 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// The MMAs that read input slot s of a layer with nrows output rows.  Output
// row i takes input slots i, i + 1, i + 2 (y-taps ky = 0, 1, 2), so slot s
// feeds the outputs s - ky for ky in [lo, hi] (those in range).  For each
// x-tap kx the A operand is slot s shifted by kx and the B operand stacks the
// tiles of ky = lo .. hi along N (weights packed ky-fastest): block j lands
// in output s - lo - j, whose columns follow those of s - lo.  Output s's
// first contribution (kx = 0, ky = 0) initialises its block; everything else
// accumulates.  Four MMAs per slot instead of nine per output row.
__device__ __forceinline__ void issue_slot(uint32_t tmem, uint32_t act_in, uint32_t w_layer, int s, int nrows) {
  const int lo = s - (nrows - 1) > 0 ? s - (nrows - 1) : 0;
  const int hi = s < 2 ? s : 2;
#pragma unroll
  for (int kx = 0; kx < 3; ++kx) {
    const uint64_t adesc = sdesc(act_in + (uint32_t)((s * kXS + kx) * 16), kPlane, 128);
    int l = lo;
    if (kx == 0 && lo == 0) {
      mma_bf16(tmem + (uint32_t)col_of(s), adesc, sdesc(w_layer + (uint32_t)(kx * 3) * 512, 128, 256), idesc_n(16),
               0u);
      l = 1;
    }
    if (l <= hi)
      mma_bf16(tmem + (uint32_t)col_of(s - l), adesc, sdesc(w_layer + (uint32_t)(kx * 3 + l) * 512, 128, 256),
               idesc_n(16 * (hi - l + 1)), 1u);
  }
}

// The fused forward pass.  r: the residual (type T, padded layout, image b
// at b * r_ld; scaled by 1 / ||r|| from the solver state when state is
// given), c: coefficient channel (padded), wtc: the packed bfloat16 weights,
// y: optional float output, z: optional output ||r|| y (type T), acts:
// optional copy of the bfloat16 activations as floats for inspection,
// [4][B][n1 * n1][16] compact (layer 0 = the two input channels, zero-padded
// to 16; layers 1-3 = the outputs of the first three convolutions); keep:
// optional bfloat16 activations in the padded training layout ([B][len][C],
// interior points only; the pads stay as the caller zeroed them), the forward
// pass of training.
template <typename T>
__global__ void __launch_bounds__(kThreads, 2)
    k_net_infer_tc(GridDesc g, const T* __restrict__ r, long long r_ld, const float* __restrict__ c,
                   const uint4* __restrict__ wtc, const DevState* state, float* __restrict__ y, T* __restrict__ z,
                   int* err, float* __restrict__ acts, NetActs keep) {
  if (state && state->done) return;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kOffBar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + kOffBar + 8 * kMaxSlots);
  // thread = (tile column x, channel half h): the two threads of a column
  // share the staging rows and split every TMEM row read (8 channels each)
  const int tid = threadIdx.x, warp = tid >> 5, x = tid & (kEW - 1), h = tid / kEW;
  const int b = blockIdx.z;
  const int gx0 = blockIdx.x * kTW - kHalo, gy0 = blockIdx.y * kTH - kHalo;
  const int n1 = g.n1;
  const long long p = g.p;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid < kMaxSlots) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar + tid)) : "memory");
  if (tid == 0) asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  // zero the x = -1 and x = 128 columns of every slot and plane (the only
  // activation entries that no layer writes but later layers read)
  if (tid < 64) {
    const int row = tid & 15, side = (tid >> 4) & 1, plane = (tid >> 5) & 1;
    *reinterpret_cast<uint4*>(smem + kOffAct0 + plane * kPlane + (row * kXS + side * (kXS - 1)) * 16) =
        make_uint4(0, 0, 0, 0);
  }
  for (int i = tid; i < kWBytes / 16; i += kThreads) reinterpret_cast<uint4*>(smem + kOffW)[i] = wtc[i];
  // input tile (thread = column x, all 16 rows, loads issued together):
  // channel 0 = bf16(r / ||r||), channel 1 = bf16(c), zero outside the grid
  {
    const float sc = state ? (float)(state->rnorm > 0.0 ? 1.0 / state->rnorm : 0.0) : 1.f;
    const T* rb = r + (long long)b * r_ld;
    const int gxx = gx0 + x;
    const bool colok = gxx >= 0 && gxx < n1;
    constexpr int kHalfRows = kEH / 2;   // rows h * 8 .. h * 8 + 7 of the tile
    const int y0 = h * kHalfRows;
    float v0[kHalfRows], v1[kHalfRows];
#pragma unroll
    for (int k = 0; k < kHalfRows; ++k) {
      const int gy = gy0 + y0 + k;
      const bool ok = colok && gy >= 0 && gy < n1;
      const long long idx = g.G + gxx + p * gy;
      v0[k] = ok ? (float)rb[idx] * sc : 0.f;
      v1[k] = ok ? c[idx] : 0.f;
    }
#pragma unroll
    for (int k = 0; k < kHalfRows; ++k) {
      const int off = ((y0 + k) * kXS + x + 1) * 16;
      *reinterpret_cast<uint4*>(smem + kOffAct0 + off) = make_uint4(pack_bf16x2(v0[k], v1[k]), 0, 0, 0);
      *reinterpret_cast<uint4*>(smem + kOffAct0 + kPlane + off) = make_uint4(0, 0, 0, 0);
    }
    if (keep.a0 && x >= kHalo && x < kHalo + kTW && gxx < n1) {
      for (int k = 0; k < kHalfRows; ++k) {
        const int yy = y0 + k, gy = gy0 + yy;
        if (yy < kHalo || yy >= kHalo + kTH || gy >= n1) continue;
        const long long o = (long long)b * g.len + g.G + gxx + p * gy;
        keep.a0[o * 2 + 0] = __float2bfloat16_rn(v0[k]);
        keep.a0[o * 2 + 1] = __float2bfloat16_rn(v1[k]);
      }
    }
    if (acts && x >= kHalo && x < kHalo + kTW && gxx < n1) {
      const long long nn = (long long)n1 * n1;
      for (int k = 0; k < kHalfRows; ++k) {
        const int yy = y0 + k, gy = gy0 + yy;
        if (yy < kHalo || yy >= kHalo + kTH || gy >= n1) continue;
        float* o = acts + (((long long)b * nn) + (long long)gy * n1 + gxx) * 16;
        o[0] = __bfloat162float(__float2bfloat16_rn(v0[k]));
        o[1] = __bfloat162float(__float2bfloat16_rn(v1[k]));
        for (int ch = 2; ch < 16; ++ch) o[ch] = 0.f;
      }
    }
  }
  fence_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t bar0 = smem_u32(bar), w_addr = smem_u32(smem + kOffW);
  const uint32_t act_addr = smem_u32(smem + kOffAct0);
  unsigned char* act = smem + kOffAct0;
  uint32_t phase = 0;             // bit s: parity of the commits issued to slot barrier s so far
  bool failed = false;
  const double zscale = state ? state->rnorm : 1.0;
  const int gx = gx0 + x;

  for (int L = 0; L < 4 && !failed; ++L) {
    const uint32_t wl = w_addr + L * 9 * 512;
    const int r0 = L + 1, nrows = kEH - 2 * (L + 1), nslots = nrows + 2;
    // input row q of layer L lives in slot q - L; output row r0 + i is
    // written to slot i (its slot as an input of layer L + 1)
    if (tid == 0) {
      fence_after();
      for (int sl = 0; sl < nslots; ++sl) {
        issue_slot(tmem, act_addr, wl, sl, nrows);
        mma_commit(bar0 + 8 * sl);
      }
    }
    for (int i = 0; i < nrows; ++i) {
      // output i is complete once the MMAs of slot i + 2 are (commits
      // complete in issue order), and by then so are those reading slot i
      const int sb = i + 2;
      const bool ok = mbar_wait(bar0 + 8 * sb, (phase >> sb) & 1u, c_wait_first);
      if (!ok) {
        failed = true;
        break;
      }
      fence_after();
      // warps w and w + 4 read the same 32 lanes: channels 8 h .. 8 h + 7
      float v[8];
      tmem_ld8(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(col_of(i) + 8 * h), v);
      const int row = r0 + i, gy = gy0 + row;
      const bool inside = gx >= 0 && gx < n1 && gy >= 0 && gy < n1;
      if (L < 3) {
        uint32_t q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          q[k] = inside ? pack_bf16x2(fmaxf(v[2 * k], 0.f), fmaxf(v[2 * k + 1], 0.f)) : 0u;
        const int off = ((row - L - 1) * kXS + x + 1) * 16;   // in place: slot of input row row - 1
        *reinterpret_cast<uint4*>(act + h * kPlane + off) = make_uint4(q[0], q[1], q[2], q[3]);
        __nv_bfloat16* kept = L == 0 ? keep.a1 : (L == 1 ? keep.a2 : keep.a3);
        if (kept && inside && x >= kHalo && x < kHalo + kTW && row >= kHalo && row < kHalo + kTH) {
          uint4* o = reinterpret_cast<uint4*>(kept + ((long long)b * g.len + g.G + gx + p * gy) * 16);
          o[h] = make_uint4(q[0], q[1], q[2], q[3]);
        }
        if (acts && inside && x >= kHalo && x < kHalo + kTW && row >= kHalo && row < kHalo + kTH) {
          const long long nn = (long long)n1 * n1;
          float* o = acts + ((((long long)(L + 1) * gridDim.z + b) * nn) + (long long)gy * n1 + gx) * 16 + 8 * h;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 h2 = *reinterpret_cast<const __nv_bfloat162*>(&q[k]);
            o[2 * k] = __low2float(h2);
            o[2 * k + 1] = __high2float(h2);
          }
        }
      } else if (h == 0 && inside && x >= kHalo && x < kHalo + kTW && row >= kHalo && row < kHalo + kTH) {
        const long long o = (long long)b * g.len + g.G + gx + p * gy;
        if (y) y[o] = v[0];
        if (z) z[o] = (T)(zscale * (double)v[0]);
      }
    }
    // the layer's outputs feed the next layer's MMAs (async proxy)
    fence_async_smem();
    fence_before();
    failed = __syncthreads_or(failed);
    if (failed) {
      if (tid == 0) atomicExch(err, 1);
      // the layer's last commit covers every MMA it issued: let them finish
      // (bounded) before their memory is freed
      mbar_wait(bar0 + 8 * (nslots - 1), (phase >> (nslots - 1)) & 1u);
    }
    phase ^= (1u << nslots) - 1u;
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Pack the bfloat16-valued weights into the compact B tiles of the four
// layers (zero-padded to 16 x 16 per tap).
__global__ void k_net_pack_tc(const float* __restrict__ wq, __nv_bfloat16* __restrict__ wtc) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 4 * 9 * 256; e += gridDim.x * blockDim.x) {
    const int L = e / (9 * 256), t = (e / 256) % 9, n = (e / 16) % 16, k = e % 16;
    float w = 0.f;
    if (L == 0) { if (k < kNetIn) w = wq[kNetOff1 + (n * kNetIn + k) * 9 + t]; }
    else if (L == 1) w = wq[kNetOff2 + (n * kNetC1 + k) * 9 + t];
    else if (L == 2) w = wq[kNetOff3 + (n * kNetW + k) * 9 + t];
    else { if (n == 0) w = wq[kNetOff4 + k * 9 + t]; }
    // tap t = ky * 3 + kx of the weights goes to tile kx * 3 + ky (ky fastest)
    wtc[((L * 9 + (t % 3) * 3 + t / 3) * 512 + canon(n, k)) / 2] = __float2bfloat16_rn(w);
  }
}

}  // namespace

int net_tc_weight_bytes() { return kWBytes; }

void launch_net_pack_tc(const float* wq, void* wtc, cudaStream_t s) {
  k_net_pack_tc<<<36, 256, 0, s>>>(wq, reinterpret_cast<__nv_bfloat16*>(wtc));
}

template <typename T>
void launch_net_infer(const GridDesc& g, int B, const T* r, long long r_ld, const float* c, const void* wtc,
                      const DevState* state, float* y, T* z, int* err, cudaStream_t s, float* acts, NetActs keep) {
  const dim3 grid((unsigned)((g.n1 + kTW - 1) / kTW), (unsigned)((g.n1 + kTH - 1) / kTH), (unsigned)B);
  k_net_infer_tc<T><<<grid, kThreads, kSmemBytes, s>>>(g, r, r_ld, c, reinterpret_cast<const uint4*>(wtc), state, y,
                                                        z, err, acts, keep);
}
template void launch_net_infer<double>(const GridDesc&, int, const double*, long long, const float*, const void*,
                                       const DevState*, float*, double*, int*, cudaStream_t, float*, NetActs);
template void launch_net_infer<float>(const GridDesc&, int, const float*, long long, const float*, const void*,
                                      const DevState*, float*, float*, int*, cudaStream_t, float*, NetActs);
template void launch_net_infer<dw>(const GridDesc&, int, const dw*, long long, const float*, const void*,
                                   const DevState*, float*, dw*, int*, cudaStream_t, float*, NetActs);

cudaError_t set_wait_first_infer(long long polls) {
  return cudaMemcpyToSymbol(c_wait_first, &polls, sizeof(polls));
}

void net_infer_prepare_attributes() {
  cudaFuncSetAttribute(k_net_infer_tc<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  cudaFuncSetAttribute(k_net_infer_tc<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  cudaFuncSetAttribute(k_net_infer_tc<dw>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
}

}  // namespace mpcg
