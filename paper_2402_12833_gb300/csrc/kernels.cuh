// Host-side launchers of the libmpcg kernels (internal).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace mpcg {

// Maximum number of thread blocks of the grid-stride reduction kernels; the
// partial-sum buffers are sized for it.
constexpr int kRedBlocks = 1216;         // 152 SMs x 8 (stencil kernels with partial sums)
constexpr int kTailPoints = 512;      // grids this small go through the single-block MG tail
constexpr int kStreamBlocks = 608;       // 152 SMs x 4 (streaming block kernels)
constexpr int kStreamBlocksMax = 8192;
constexpr int kGramChunksMax = 4096;

// Grid sizes of the streaming block kernels and of the window Gram kernel;
// both keep every thread at <= 64 points per FP32 partial sum.
// Launch shapes: the fixed rules, unless the autotuner's table (tune.h) holds
// a value for the grid, clamped to the range the reduction buffers reserve
// (stream_blocks_cap / gram_chunks_cap) and to the accuracy limit of at most
// 64 FP32 points per thread before the partial sums leave the thread.
int stream_blocks(const GridDesc& g);
int gram_chunks(const GridDesc& g);
int stream_blocks_default(const GridDesc& g);
int gram_chunks_default(const GridDesc& g);
int stream_blocks_min(const GridDesc& g);
int stream_blocks_cap(const GridDesc& g);
int gram_chunks_min(const GridDesc& g);
int gram_chunks_cap(const GridDesc& g);
// number of SMs (set at hierarchy setup; 0 before)
int sm_count();
template <typename T>
constexpr int kind_of();
template <>
constexpr int kind_of<float>() { return 0; }
template <>
constexpr int kind_of<double>() { return 1; }
template <>
constexpr int kind_of<dw>() { return 2; }

// Sets the calling thread's message returned by mpcg_last_error().
void set_error_message(const char* msg);
// mpcg_solve_batched_graph takes these classes (mixed precision, graphs on,
// one device, each hierarchy once)
bool batched_graph_eligible(mg_hierarchy* const* hs, int nclass);

inline int grid_for(long long work, int cap) {
  long long b = (work + kBlock - 1) / kBlock;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

// ---- ell.cu (algebraic hierarchies; vectors offset by G) -----------------
// Y[:, c] = A X[:, c], c < C <= 12 (column pitches ldx, ldy); zaz (may be
// null) receives per-block partials of X_c^T Y_c, value-major with stride
// nblocks.  nblocks <= 0: one thread per row.
template <typename T>
void launch_ell_spmm(const EllDev<T>& A, const T* X, long long ldx, T* Y, long long ldy, int C, double* zaz,
                     int nblocks, const DevState* state, cudaStream_t s);
// r = b - A x, partials [|r|^2, |b|^2] over nblocks blocks; xnz as launch_residual
template <typename T>
void launch_ell_residual(const EllDev<T>& A, const T* b, const T* x, T* r, double* part, int nblocks,
                         cudaStream_t s, const int* xnz = nullptr);
// d = b - A x without norms (V-cycle defect)
template <typename T>
void launch_ell_defect(const EllDev<T>& A, const T* b, const T* x, T* d, const DevState* state, cudaStream_t s);
// Y += A X, one column (V-cycle prolongation of the coarse correction)
template <typename T>
void launch_ell_spmv_add(const EllDev<T>& A, const T* X, T* Y, const DevState* state, cudaStream_t s);
// damped Jacobi (dinv = omega / a_ii), modes as launch_jacobi
template <typename T>
void launch_ell_jacobi(const EllDev<T>& A, const T* dinv, const T* g, const T* sin, T* out, int mode,
                       const DevState* state, cudaStream_t s);

// ---- stencil.cu ----------------------------------------------------------
// compact interior <-> padded layout (ncols columns; compact leading dim ld)
template <typename TI, typename TO>
void launch_pack(const GridDesc& g, const TI* src, long long ld, TO* dst, int ncols, cudaStream_t s);
// pack of one FP64 column; *nz = 1 when it has a nonzero entry (zero it first)
template <typename TO>
void launch_pack_flag(const GridDesc& g, const double* src, TO* dst, int* nz, cudaStream_t s);
// SM count used to size one-wave launches (set at hierarchy setup)
void set_sm_count(int n);
// blocks (and zaz partial slots) of launch_spmm on grid g with C columns
template <typename T>
int spmm_blocks(const GridDesc& g, int C);
template <typename TI, typename TO>
void launch_unpack(const GridDesc& g, const TI* src, TO* dst, long long ld, int ncols, cudaStream_t s);

// Y = A X over C columns; if zaz != nullptr also partials of X_b^T Y_b
// (value-major, stride kRedBlocks).  `state` (may be null) gates on done.
template <typename T>
void launch_spmm(const GridDesc& g, const T* st, const T* X, T* Y, int C, double* zaz,
                 const DevState* state, cudaStream_t s);
// r = b - A x; partials [||r||^2, ||b||^2].  xnz (may be null): per problem,
// 0 when x is known to be zero (then r = b without reading the stencil)
template <typename T>
void launch_residual(const GridDesc& g, const T* st, const T* b, const T* x, T* r, double* part,
                     cudaStream_t s, const int* xnz = nullptr);
// coarse = P^T fine
template <typename T>
void launch_restrict(const GridDesc& gf, const GridDesc& gc, const T* rf, T* rc,
                     const DevState* state, cudaStream_t s);
// damped Jacobi: mode 0: out = dinv r; mode 1: two sweeps from zero;
// mode 2: out = sin + dinv (r - A sin)
template <typename T>
void launch_jacobi(const GridDesc& g, const T* st, const T* dinv, const T* r, const T* sin, T* out,
                   int mode, const DevState* state, cudaStream_t s);
// ---- stencil_sym.cu: FP32 on the symmetric half of a scalar stencil ------
// Planes of the half: 14 (3D) or 5 (2D), the diagonal and the couplings to
// the lexicographically later neighbours, same pitch (cp) as the full planes.
int sym_planes(int dim);
// half (sym_planes(g.dim) * g.cp floats) from the full FP64 planes st;
// couplings with a pad row or column stored as zero
void launch_sym_half(const GridDesc& g, const double* st, float* half, cudaStream_t s);
// launch_spmm<float> and launch_jacobi<float> (scalar grids) reading the half
void launch_spmm_sym(const GridDesc& g, const float* half, const float* X, float* Y, int C, double* zaz,
                     const DevState* state, cudaStream_t s);
void launch_jacobi_sym(const GridDesc& g, const float* half, const float* dinv, const float* r, const float* sin,
                       float* out, int mode, const DevState* state, cudaStream_t s);
// Vector operators (3 unknowns per node): t = r - A x (one sweep's residual)
// and the block-Jacobi update out = (sin or 0) + dinv t (in place allowed).
template <typename T>
void launch_vres(const GridDesc& g, const T* st, const T* r, const T* x, T* t, const DevState* state,
                 cudaStream_t s);
// the last block-Jacobi sweep fused: out = x + dinv (r - A x), out != x
template <typename T>
void launch_vres_block(const GridDesc& g, const T* st, const T* r, const T* x, const T* dinv, T* out,
                       const DevState* state, cudaStream_t s);
template <typename T>
void launch_vblock(const GridDesc& g, const T* dinv, const T* t, const T* sin, T* out, const DevState* state,
                   cudaStream_t s);
// out = Zc[0] + ... + Zc[ncols-1] (columns cp apart).
template <typename T>
void launch_sum_columns(const GridDesc& g, const T* Zc, int ncols, T* out, const DevState* state, cudaStream_t s);
// The small-grid tail of the MG chain in one block (scalar unknowns, nu = 2):
// restrictions from grid jt + 1 (residual rin) down to 0 into r[j], Jacobi
// smoothing of grids 1 .. jt into z[j], coarse solve into z[0].
template <typename T>
void launch_coarse_tail(int jt, const GridDesc* g, const T* const* st, const T* const* dinv, T* const* r,
                        T* const* z, const T* rin, const double* a0inv, const DevState* state, cudaStream_t s);
// Z columns 0 .. J-1 on the fine grid gf from grid j's correction coarse[j]
// (grid descriptor gcs[j]) by the composite multilinear interpolation.
template <typename T>
void launch_prolong_all(const GridDesc& gf, const T* const* coarse, const GridDesc* gcs, int J, T* Z,
                        const DevState* state, cudaStream_t s);
// Multicoloured SSOR: one Gauss-Seidel update of the unknowns of `colour`
// (bit a = parity of the global coordinate on axis a), in place on x, scalar
// grids; d = b - A x; fine += P coarse (two grids).
template <typename T>
void launch_gs_colour(const GridDesc& g, const T* st, const T* b, T* x, int colour, double omega, const DevState* state,
                      cudaStream_t s);
template <typename T>
void launch_defect(const GridDesc& g, const T* st, const T* b, const T* x, T* d, const DevState* state,
                   cudaStream_t s);
template <typename T>
void launch_prolong_add(const GridDesc& gc, const GridDesc& gf, const T* coarse, T* fine, const DevState* state,
                        cudaStream_t s);
template <typename T>
void launch_add_to(const GridDesc& g, const T* src, T* dst, const DevState* state, cudaStream_t s);
// coarse stencil = P^T A P (FP64)
void launch_galerkin(const GridDesc& gf, const GridDesc& gc, const double* stf, double* stc,
                     cudaStream_t s);
// dinv = omega / centre coefficient (0 at pads)
template <typename T>
void launch_dinv(const GridDesc& g, const double* st, T* dinv, double omega, cudaStream_t s);
void launch_convert_f32(const double* src, float* dst, long long count, cudaStream_t s);
// double -> double-word pairs (dw.cuh), element by element
void launch_convert_dw(const double* src, dw* dst, long long count, cudaStream_t s);

// ---- block.cu --------------------------------------------------------------
// W partials: rows jj*C+a (window block jj, newest first), cols b:
//   sum_i AP_slot(jj)[a][i] * Z[b][i]
template <typename T>
void launch_gram_window(const GridDesc& g, Window<T> win, const T* Z, int C, int m, double* part,
                        const DevState* state, cudaStream_t s);
// P_new = Z - sum P_j beta_j, AP_new = AZ - sum AP_j beta_j into the next
// ring slot; partials of sym(P^T AP) (upper triangle) and P^T r.
template <typename T>
void launch_orth_update(const GridDesc& g, Window<T> win, const T* Z, const T* AZ, const T* r,
                        int C, double* part, const DevState* state, cudaStream_t s);
// double-word: the Gram partials of the new block (launch_orth_update<dw>
// leaves them to this kernel), same partial layout as the fused kernels
void launch_orth_gram_dw(const GridDesc& g, Window<dw> win, const dw* r, int C, double* part,
                         const DevState* state, cudaStream_t s);
// x += P alpha, r -= AP alpha (newest block); partial of ||r||^2
template <typename T>
void launch_update_xr(const GridDesc& g, Window<T> win, T* x, T* r, int C, double* part,
                      const DevState* state, cudaStream_t s);

// ---- matfree.cu ----------------------------------------------------------
// Element coefficients kappa (FP64, nb problems of ne^dim elements, x
// fastest) into the padded slots k32 / k64 of the fine grid as -(h/12) kappa
// (3D) or -kappa/6 (2D), and the largest difference between the stored FP64
// stencil st64 and the one kappa defines (couplings between unknowns, all
// problems), with the largest stored coefficient.
mpcg_status place_kappa(const GridDesc& g, const double* kappa, int ne, double h, float* k32, double* k64,
                        unsigned long long* check, const double* st64, double* maxdiff, double* maxabs,
                        cudaStream_t s);
// Y = A X (C <= 12 columns, zaz partials as launch_spmm with nblocks blocks;
// false for other C) and the fused two-sweep Jacobi, A rebuilt from k32
// (2D / 3D scalar, FP32).
bool launch_spmm_mf(const GridDesc& g, const float* k32, const float* X, float* Y, int C, int nblocks, double* zaz,
                    const DevState* state, cudaStream_t s);
void launch_jacobi_mf(const GridDesc& g, const float* k32, const float* dinv, const float* r, float* out,
                      const DevState* state, cudaStream_t s);

// ---- small.cu ------------------------------------------------------------
void launch_init(DevState* st, int nb, const double* part_res, int nblk, double* res_hist, long long hist_stride,
                 cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s);
// The small solves reduce their partial sums with kSmallGrid blocks; the last
// block to finish (atomic counter, zero between launches) does the solve.
// scratch holds the reduced values (>= m C^2 + C^2 + 3C doubles).
constexpr int kSmallGrid = 96;
constexpr int kSmallScratchAlpha = kMaxWindow * kMaxCols * kMaxCols;   // offset of small_alpha's values
constexpr int kSmallScratch = kSmallScratchAlpha + kMaxCols * kMaxCols + 3 * kMaxCols;   // per problem
void launch_small_beta(DevState* st, int nb, const double* part_W, int nchunks, int C, double* scratch,
                       unsigned* counter, cudaStream_t s);
void launch_small_alpha(DevState* st, int nb, const double* part_G, int nblk_G, const double* part_zaz, int nblk_zaz,
                        int zaz_stride, int C, double* alpha_hist, long long ahist_stride, double* scratch,
                        unsigned* counter, cudaStream_t s);
void launch_check(DevState* st, int nb, const double* part_r, int nblk, double* res_hist, long long hist_stride,
                  cudaGraphConditionalHandle cond, int use_cond, cudaStream_t s);
void launch_set_params(DevState* st, int nb, double rtol, int maxit, int m, int C, double delta, double tau,
                       cudaStream_t s);
// batched graphs: flag |= any problem running; then cond = flag, flag = 0
void launch_any_running(const DevState* st, int nb, int* flag, cudaStream_t s);
void launch_set_cond(int* flag, cudaGraphConditionalHandle cond, cudaStream_t s);
void launch_gather_kd(const DevState* st, int nb, int* out, cudaStream_t s);
// Cholesky of the dense coarsest matrix (in place, lower); info[0] = 0 or the
// failing pivot + 1
void launch_dense_from_stencil(const GridDesc& g, const double* st, double* dense, cudaStream_t s);
void launch_cholesky(double* a, double* rdiag, int n, int* info, cudaStream_t s);
// inv = A0^{-1} from the Cholesky factor (X: n*n scratch)
void launch_coarse_inverse(const double* L, const double* rdiag, double* X, double* inv, int n, cudaStream_t s);
// out = A0^{-1} r; r, out in the padded layout of grid g
template <typename T>
void launch_coarse_solve(const GridDesc& g, const double* inv, const T* r, T* out, const DevState* state,
                         cudaStream_t s);
// ||r||^2 style sum of partials (value-major) into out[nv]
// Device side of the mixed-precision refinement loop: mix holds per problem
// {inner iterations so far, status, active}.
void launch_mix_init(int* mix, int* active, int nb, int* outer, cudaStream_t s);
void launch_outer_check(int* mix, int* active, int nb, const double* nrm, double rtol, int maxit, int max_outer,
                        int* outer, DevState* st, double inner_rtol, int m, int C, double delta, double tau,
                        cudaGraphConditionalHandle cond, cudaStream_t s);
void launch_outer_accumulate(int* mix, int nb, const DevState* st, cudaStream_t s);
void launch_sum_partials(const double* part, int nb, int nv, int nblk, double* out, cudaStream_t s);
// x64 += scale * d (padded, FP32 d); scale read from device; xnz[p] = 1
void launch_axpy_mixed(const GridDesc& g, double* x, const float* d, const double* scale, int* xnz,
                       cudaStream_t s);
// start of an inner FP32 solve from a zero iterate: b32 = r32 = r64 / ||r64||
// (device norm-squared) and the residual partials of ||r32||^2, ||b32||^2
void launch_start_inner(const GridDesc& g, const double* r64, const double* nrm2, const int* active, float* b32,
                        float* r32, double* part, cudaStream_t s);

// ---- learned.cu ----------------------------------------------------------
// Network 2 -> 16 -> 16 -> 16 -> 1 (3x3), parameters packed layer by layer,
// each W[co][ci][ky][kx].
constexpr int kNetIn = 2, kNetC1 = 16, kNetW = 16;
constexpr int kNetOff1 = 0;
constexpr int kNetOff2 = kNetOff1 + kNetC1 * kNetIn * 9;
constexpr int kNetOff3 = kNetOff2 + kNetW * kNetC1 * 9;
constexpr int kNetOff4 = kNetOff3 + kNetW * kNetW * 9;
constexpr int kNetParams = kNetOff4 + kNetW * 9;
// the 3x3x3 network of 3D vector problems: channels 3 -> 16 -> 16 -> 16 -> 3
constexpr int kNet3Off1 = 0;
constexpr int kNet3Off2 = kNet3Off1 + 16 * 3 * 27;
constexpr int kNet3Off3 = kNet3Off2 + 16 * 16 * 27;
constexpr int kNet3Off4 = kNet3Off3 + 16 * 16 * 27;
constexpr int kNet3Params = kNet3Off4 + 3 * 16 * 27;

struct NetActs {   // [B][len][C] bfloat16, zero pads
  __nv_bfloat16 *a0, *a1, *a2, *a3;
};
struct NetGrads {  // data gradients [B][len][16] float; weight-gradient partials per layer
  float *d1, *d2, *d3;
  double* part[4];
};

// Fused tensor-core inference (all four layers per output tile); wtc holds
// the weights packed by launch_net_pack_tc (net_tc_weight_bytes() bytes);
// err is set to 1 if a bounded wait on the MMA completion runs out; acts
// (may be null) receives the activations [4][B][n1*n1][16] as floats; keep
// (pointers may be null) receives them in the padded bfloat16 layout of
// NetActs (the training forward pass).
template <typename T>
void launch_net_infer(const GridDesc& g, int B, const T* r, long long r_ld, const float* c, const void* wtc,
                      const DevState* state, float* y, T* z, int* err, cudaStream_t s, float* acts = nullptr,
                      NetActs keep = NetActs{nullptr, nullptr, nullptr, nullptr});
// Tensor-core training kernels (learned_train_tc.cu): the weight gradient of
// layer `layer` (0..3) into part (value-major, stride net_wgrad_tc_blocks)
// and the masked data gradient through a layer with cout outputs (1 or 16).
void launch_net_wgrad_tc(const GridDesc& g, int B, int layer, const float* dOut, const __nv_bfloat16* act,
                         double* part, int* err, cudaStream_t s);
void launch_net_dgrad_tc(const GridDesc& g, int B, int cout, const float* dOut, const float* W,
                         const __nv_bfloat16* act_in, float* dIn, int* err, cudaStream_t s);
int net_wgrad_tc_blocks(const GridDesc& g, int B);
void net_train_tc_prepare_attributes();
// The 3x3x3 network of 3D vector problems (learned3_tc.cu): activations are
// [B][net3_act_len(g)][16] bfloat16 on the node box; partials of the weight
// gradient are net3_wgrad_blocks per parameter; d4 is scratch of the size of
// one activation set in FP32.
long long net3_act_len(const GridDesc& g);
int net3_wgrad_blocks(const GridDesc& g, int B);
void net3_prepare_attributes();
// polls of the first bounded wait of each learned-column tensor-core kernel
// (2D inference, 2D training, 3D network) on the current device
cudaError_t set_wait_first_infer(long long polls);
cudaError_t set_wait_first_train(long long polls);
cudaError_t set_wait_first_net3(long long polls);
// bfloat16 tap tiles of all layers, forward and data-gradient orientation
// (net3_pack_bytes() bytes), from the bfloat16-rounded weights wq
int net3_pack_bytes();
void launch_net3_pack(const float* wq, unsigned char* wp, cudaStream_t s);
template <typename T>
void launch_net3_forward(const GridDesc& g, int B, const T* r, long long r_ld, const unsigned char* wp,
                         const DevState* state, NetActs acts, float* y, T* z, int* err, cudaStream_t s);
void launch_net3_backward(const GridDesc& g, int B, const unsigned char* wp, NetActs acts, const float* dy,
                          NetGrads gr, float* d4, int* err, cudaStream_t s);
// activations of the 3D network to the compact float layout
// [4][B][unknown nodes][16], nodes x fastest
void launch_net3_acts_export(const GridDesc& g, int B, NetActs acts, float* out, cudaStream_t s);

void launch_net_pack_tc(const float* wq, void* wtc, cudaStream_t s);
int net_tc_weight_bytes();
void net_infer_prepare_attributes();
void launch_net_backward(const GridDesc& g, int B, const float* wq, NetActs acts, const float* dy, NetGrads gr,
                         int* err, cudaStream_t s);
void launch_net_loss_grad(const GridDesc& g, int B, const float* y, const float* Ay, const float* e,
                          const float* Ae, double* part, double* coef, double* loss_sum, float* dy, cudaStream_t s);
// the weight-gradient partials of every layer are nblk per parameter (the
// block count of the last backward pass: net_wgrad_tc_blocks of its batch)
// net3: the 3D network's layer sizes and parameter count
void launch_net_adam(const double* const* parts_dev, int nblk, int net3, float* master, float* m, float* v, float* wq,
                     int step, float lr, float b1, float b2, float eps, cudaStream_t s);
void launch_round_bf16(const float* src, float* dst, int n, cudaStream_t s);
// grad[i] = sum of the weight-gradient partials of parameter i (all layers)
void launch_net_grad_sum(const double* const* parts_dev, int nblk, int net3, double* grad, cudaStream_t s);
// activations a0..a3 of the training forward ([B][len][C] bfloat16, padded)
// to the compact float layout [4][B][n1*n1][16] (a0 zero-padded to 16)
void launch_net_acts_export(const GridDesc& g, int B, NetActs acts, float* out, cudaStream_t s);
void launch_net_coef(const GridDesc& g, const double* dinv, double omega, float* c, double* part, cudaStream_t s);

}  // namespace mpcg
