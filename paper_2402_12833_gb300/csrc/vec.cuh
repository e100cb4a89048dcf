// Device helpers shared by the streaming kernels: 16-byte vector access to
// the padded arrays (4 floats or 2 doubles per thread and step) and
// deterministic block reductions that write value-major partial sums.
#pragma once

#include "common.cuh"
#include "dw.cuh"

namespace mpcg {

template <typename T>
struct Vec;

template <>
struct Vec<float> {
  static constexpr int W = 4;
  // streamed once: evict-first
  __device__ static __forceinline__ void load(const float* p, float (&v)[4]) {
    const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
  // re-read by neighbours or other blocks: default caching
  __device__ static __forceinline__ void load_keep(const float* p, float (&v)[4]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  }
  __device__ static __forceinline__ void store(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};

template <>
struct Vec<double> {
  static constexpr int W = 2;
  __device__ static __forceinline__ void load(const double* p, double (&v)[2]) {
    const double2 q = __ldcs(reinterpret_cast<const double2*>(p));
    v[0] = q.x; v[1] = q.y;
  }
  __device__ static __forceinline__ void load_keep(const double* p, double (&v)[2]) {
    const double2 q = *reinterpret_cast<const double2*>(p);
    v[0] = q.x; v[1] = q.y;
  }
  __device__ static __forceinline__ void store(double* p, const double (&v)[2]) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  }
};

// double-word pairs: two per 16-byte vector, like doubles
template <>
struct Vec<dw> {
  static constexpr int W = 2;
  __device__ static __forceinline__ void load(const dw* p, dw (&v)[2]) {
    const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
    v[0] = dw(q.x, q.y); v[1] = dw(q.z, q.w);
  }
  __device__ static __forceinline__ void load_keep(const dw* p, dw (&v)[2]) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = dw(q.x, q.y); v[1] = dw(q.z, q.w);
  }
  __device__ static __forceinline__ void store(dw* p, const dw (&v)[2]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
  }
};

// Loads and stores of W consecutive values (W = 1 or the full vector width
// of Vec<T>), for kernels whose points per thread depend on the grid size.
template <typename T, int W>
struct VecN;
template <typename T>
struct VecN<T, 1> {
  __device__ static __forceinline__ void load(const T* p, T (&v)[1]) { v[0] = __ldcs(p); }
  __device__ static __forceinline__ void load_keep(const T* p, T (&v)[1]) { v[0] = *p; }
  __device__ static __forceinline__ void store(T* p, const T (&v)[1]) { *p = v[0]; }
};
template <>
struct VecN<float, 4> : Vec<float> {};
template <>
struct VecN<double, 2> : Vec<double> {};
template <>
struct VecN<dw, 2> : Vec<dw> {};

// Number of values a lane holds after `steps` halvings of nv values.
__host__ __device__ constexpr int rs_count(int nv, int steps) {
  return steps == 0 ? nv : rs_count((nv + 1) / 2, steps - 1);
}

// One butterfly reduce-scatter step across lanes `o` apart: the lane pair
// splits its K values into a lower and an upper half (the upper half padded
// with zeros to H values); the lane without bit o keeps the lower half, the
// other the upper half, each adding its partner's copy.  `base` and `nvalid`
// track the first value index of the lane's half and how many of its values
// are real (an odd split leaves padding that must not claim an index).
template <typename T, int NV, int K, int O>
__device__ __forceinline__ void rs_step(T (&a)[NV], int& base, int& nvalid, int lane) {
  constexpr int H = (K + 1) / 2;
  const bool up = (lane & O) != 0;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    const T lo = a[i];
    const T hi = (H + i < K) ? a[H + i] : T(0);
    const T send = up ? lo : hi;
    const T keep = up ? hi : lo;
    a[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
  }
  if (up) {
    base += H;
    nvalid = nvalid > H ? nvalid - H : 0;
  } else {
    nvalid = nvalid < H ? nvalid : H;
  }
}

// Block sum of NV per-thread values, written to part[i * stride + slot].
// The warp stage sums in T (FP32 in the FP32 path) by a butterfly
// reduce-scatter (lane pairs 16, 8, 4, 2, 1 apart exchange half of their
// values, so a warp spends about NV shuffles instead of 5 NV); the
// cross-warp stage sums in FP64 in a fixed order.  Every thread of the block
// must call it.
template <typename T, int NV>
__device__ __forceinline__ void block_sum_store(const T (&v)[NV], double* part, long long stride, int slot) {
  __shared__ double sh[kBlock / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T a[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) a[i] = v[i];
  int base = 0, nvalid = NV;
  rs_step<T, NV, rs_count(NV, 0), 16>(a, base, nvalid, lane);
  rs_step<T, NV, rs_count(NV, 1), 8>(a, base, nvalid, lane);
  rs_step<T, NV, rs_count(NV, 2), 4>(a, base, nvalid, lane);
  rs_step<T, NV, rs_count(NV, 3), 2>(a, base, nvalid, lane);
  rs_step<T, NV, rs_count(NV, 4), 1>(a, base, nvalid, lane);
  constexpr int K5 = rs_count(NV, 5);
#pragma unroll
  for (int i = 0; i < K5; ++i)
    if (i < nvalid) sh[warp][base + i] = (double)a[i];
  __syncthreads();
  for (int i = threadIdx.x; i < NV; i += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w][i];
    part[(long long)i * stride + slot] = s;
  }
}

// Box index t (0 <= t < npts) -> node (x, y, z) and component.
__device__ __forceinline__ void decode(const GridDesc& g, long long t, int& x, int& y, int& z, int& comp) {
  const unsigned u = (unsigned)t;
  const unsigned q1 = fdiv(u, g.dvx);
  x = (int)(u - q1 * (unsigned)g.px);
  const unsigned q2 = fdiv(q1, g.dvy);
  y = (int)(q1 - q2 * (unsigned)g.py);
  if (g.dim == 3) {
    const unsigned q3 = fdiv(q2, g.dvz);
    z = (int)(q2 - q3 * (unsigned)g.pz);
    comp = (int)q3;
  } else {
    z = 0;
    comp = (int)q2;
  }
}

__device__ __forceinline__ void decode(const GridDesc& g, long long t, int& x, int& y, int& z) {
  int comp;
  decode(g, t, x, y, z, comp);
}

__device__ __forceinline__ bool interior(const GridDesc& g, int x, int y, int z) {
  return x < g.nx && y < g.ny && (g.dim == 2 || z < g.nz);
}

}  // namespace mpcg
