// mg_stencil_apply_noalloc: Y = A X for a fine-grid operator given in the
// stencil format of mg_operator, without any device allocation.
//
// The padded copies of the stencil and of X and Y that the block SpMM kernel
// works on live in one file-scope device array of kScratchDoubles doubles
// (16 MiB).  Every GPU that loads the library holds that array until the
// process exits.  Host code cannot use the array's name as a device address:
// the address is looked up with cudaGetSymbolAddress, with the context that
// will run the kernels current, and cached.  The module holding the array is
// loaded once per CUDA context, so the cache is keyed on the context's
// process-unique ID (cuCtxGetId), not on the device ordinal: after
// cudaDeviceReset, or with a non-primary context current, the ID differs and
// the address is looked up again instead of reusing a stale one.
#include <cuda.h>

#include <mutex>
#include <stdio.h>

#include "kernels.cuh"

namespace {

constexpr long long kScratchDoubles = 1LL << 21;   // 16 MiB
constexpr int kCacheSlots = 16;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct ScratchCache {
  std::mutex mu;
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
  bool resolved = false;
  unsigned long long id[kCacheSlots] = {};   // 0 = empty slot
  double* ptr[kCacheSlots] = {};
  int next = 0;                              // round-robin replacement
};
ScratchCache g_cache;

mpcg_status fail(mpcg_status st, const char* msg) {
  mpcg::set_error_message(msg);
  return st;
}

// The two driver calls, taken through the runtime so that the library keeps
// no link-time dependence on libcuda (it loads on machines without a GPU).
bool resolve_driver_calls() {
  if (g_cache.resolved) return g_cache.get_current && g_cache.get_id;
  g_cache.resolved = true;
  cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = cudaDriverEntryPointSymbolNotFound;
  void* f1 = nullptr;
  void* f2 = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
      cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
      q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return false;
  }
  g_cache.get_current = (CtxGetCurrentFn)f1;
  g_cache.get_id = (CtxGetIdFn)f2;
  return true;
}

// ID of the context current on this thread; 0 if there is none yet.
unsigned long long current_context_id() {
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (g_cache.get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
  if (g_cache.get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

mpcg_status lookup_failed(cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "mg_stencil_apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
  cudaGetLastError();
  return fail(MPCG_ERR_CUDA, buf);
}

// Device address of the scratch array in the context current on this thread
// (looked up once per context).
mpcg_status scratch_for_current_context(double** out) {
  std::lock_guard<std::mutex> lock(g_cache.mu);
  if (!resolve_driver_calls())
    return fail(MPCG_ERR_CUDA, "mg_stencil_apply_noalloc: the CUDA driver does not provide cuCtxGetCurrent/cuCtxGetId");
  unsigned long long id = current_context_id();
  if (id == 0) {
    // no context bound to this thread yet: the runtime binds the current
    // device's primary context on its first call, which this lookup is
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return lookup_failed(e);
    id = current_context_id();
    if (id == 0) return fail(MPCG_ERR_CUDA, "mg_stencil_apply_noalloc: no CUDA context is current");
  }
  for (int i = 0; i < kCacheSlots; ++i)
    if (g_cache.id[i] == id) {
      *out = g_cache.ptr[i];
      return MPCG_OK;
    }
  double* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
  if (e != cudaSuccess || !p) return lookup_failed(e);
  const int slot = g_cache.next;
  g_cache.next = (g_cache.next + 1) % kCacheSlots;
  g_cache.id[slot] = id;
  g_cache.ptr[slot] = p;
  *out = p;
  return MPCG_OK;
}

}  // namespace

extern "C" mpcg_status mg_stencil_apply_noalloc(int dim, int nodes, const double* values_dev, const double* X_dev,
                                                double* Y_dev, int ncols, void* stream) {
  using namespace mpcg;
  set_error_message("");
  if (dim != 2 && dim != 3) return fail(MPCG_ERR_ARG, "mg_stencil_apply_noalloc: dim must be 2 or 3");
  const int q = nodes - 1;
  if (q < 2 || q > (1 << 15)) return fail(MPCG_ERR_ARG, "mg_stencil_apply_noalloc: nodes - 1 must be in [2, 32768]");
  if (ncols < 1 || ncols > MPCG_MAX_COLS)
    return fail(MPCG_ERR_ARG, "mg_stencil_apply_noalloc: ncols must be in 1..MPCG_MAX_COLS");
  if (!values_dev || !X_dev || !Y_dev) return fail(MPCG_ERR_ARG, "mg_stencil_apply_noalloc: NULL pointer");
  const GridDesc g = make_grid(dim, nodes - 2);
  const int S = dim == 3 ? 27 : 9;
  const long long need = (long long)(S + 2 * ncols) * g.len;
  if (need > kScratchDoubles) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "mg_stencil_apply_noalloc: this grid needs %lld doubles of scratch, the fixed maximum is %lld "
             "(use mg_apply_operator for larger grids)",
             need, kScratchDoubles);
    return fail(MPCG_ERR_ARG, buf);
  }
  double* scratch = nullptr;
  const mpcg_status st = scratch_for_current_context(&scratch);
  if (st != MPCG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  double* st_pad = scratch;
  double* x_pad = st_pad + (long long)S * g.len;
  double* y_pad = x_pad + (long long)ncols * g.len;
  // the array keeps the previous call's contents: the pads must read zero
  if (cudaMemsetAsync(scratch, 0, sizeof(double) * (size_t)need, s) != cudaSuccess) {
    cudaGetLastError();
    return fail(MPCG_ERR_CUDA, "mg_stencil_apply_noalloc: cudaMemsetAsync failed");
  }
  launch_pack<double, double>(g, values_dev, g.n, st_pad, S, s);
  launch_pack<double, double>(g, X_dev, g.n, x_pad, ncols, s);
  launch_spmm<double>(g, st_pad, x_pad, y_pad, ncols, nullptr, nullptr, s);
  launch_unpack<double, double>(g, y_pad, Y_dev, g.n, ncols, s);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    char buf[256];
    snprintf(buf, sizeof buf, "mg_stencil_apply_noalloc: kernel launch failed: %s", cudaGetErrorString(e));
    return fail(MPCG_ERR_CUDA, buf);
  }
  return MPCG_OK;
}
