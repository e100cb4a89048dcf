// The FP32 block SpMM and damped-Jacobi kernels of stencil.cu on the
// symmetric half of a scalar stencil (the inner solves of the mixed
// precision), with the conversion that builds the half.  A separate
// translation unit so that the build compiles it in parallel.
#define MPCG_STENCIL_SYM 1
#include "stencil.cu"
