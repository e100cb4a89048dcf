// The structured-grid kernels of stencil.cu instantiated for double-word
// values (dw.cuh): FP64 data with double-FP32 arithmetic.  A separate
// translation unit so that the build compiles both halves in parallel.
#define MPCG_STENCIL_DW 1
#include "stencil.cu"
