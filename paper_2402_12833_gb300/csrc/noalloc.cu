// mg_stencil_apply_noalloc: Y = A X for a fine-grid operator given in the
// stencil format of mg_operator, without any device allocation.
//
// The padded copies of the stencil and of X and Y that the block SpMM kernel
// works on live in one file-scope device array of kScratchDoubles doubles
// (16 MiB).  Every GPU that loads the library holds that array until the
// process exits.  Host code cannot use the array's name as a device address,
// so the first call on each device, with that device current, looks the
// address up once with cudaGetSymbolAddress and caches it; later calls pass
// the cached address to the kernels.
#include <mutex>
#include <stdio.h>

#include "kernels.cuh"

namespace {

constexpr long long kScratchDoubles = 1LL << 21;   // 16 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) double g_noalloc_scratch[kScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

mpcg_status fail(mpcg_status st, const char* msg) {
  mpcg::set_error_message(msg);
  return st;
}

// Device address of the scratch array on the current device (looked up once).
mpcg_status scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return fail(MPCG_ERR_CUDA, "mg_stencil_apply_noalloc: no usable current CUDA device");
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    double* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      char buf[256];
      snprintf(buf, sizeof buf, "mg_stencil_apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      cudaGetLastError();
      return fail(MPCG_ERR_CUDA, buf);
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MPCG_OK;
}

}  // namespace

extern "C" mpcg_status mg_stencil_apply_noalloc(int dim, int nodes, const double* values_dev, const double* X_dev,
                                                double* Y_dev, int ncols, void* stream) {
  using namespace mpcg;
  if (dim != 2 && dim != 3) return fail(MPCG_ERR_ARG, "mg_stencil_apply_noalloc: dim must be 2 or 3");
  const int q = nodes - 1;
  if (q < 4 || (q & (q - 1)) != 0 || q > (1 << 15))
    return fail(MPCG_ERR_ARG, "mg_stencil_apply_noalloc: nodes - 1 must be a power of two >= 4");
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
  const mpcg_status st = scratch_for_current_device(&scratch);
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
