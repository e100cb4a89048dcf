// mpcg_solve_batched: many independent problems of uneven size.
//
// Problems of one grid size form one batched hierarchy (mg_hierarchy_setup_batched),
// whose every kernel processes the whole batch at once (the problem index is
// blockIdx.y) with a device-side loop that runs while any problem of the
// batch is unconverged.  The size classes are independent: mixed-precision
// classes with graphs run as branches of one CUDA graph (one launch for the
// whole batch, mpcg_solve_batched_graph in api.cu); otherwise this entry
// point drives them from one host thread each, so that their launches execute
// concurrently on their own streams.
#include <string>
#include <thread>
#include <vector>

#include "kernels.cuh"

extern "C" mpcg_status mpcg_solve_batched(mg_hierarchy* const* hs, int nclass, const double* const* b,
                                          double* const* x, double rtol, int maxit, int* const* iters) {
  if (!hs || nclass < 1 || !b || !x) {
    mpcg::set_error_message("mpcg_solve_batched: bad arguments");
    return MPCG_ERR_ARG;
  }
  // mixed-precision classes with graphs: every class's solve is a branch of
  // one CUDA graph, one launch for the whole batch
  if (nclass > 1 && mpcg::batched_graph_eligible(hs, nclass))
    return mpcg_solve_batched_graph(hs, nclass, b, x, rtol, maxit, iters);
  std::vector<mpcg_status> st(nclass, MPCG_OK);
  std::vector<std::string> err(nclass);
  std::vector<std::thread> th;
  th.reserve(nclass);
  for (int c = 0; c < nclass; ++c)
    th.emplace_back([&, c] {
      st[c] = mpcg_solve(hs[c], b[c], x[c], rtol, maxit, iters ? iters[c] : nullptr, nullptr, nullptr);
      if (st[c] != MPCG_OK) err[c] = mpcg_last_error();
    });
  for (auto& t : th) t.join();
  mpcg_status worst = MPCG_OK;
  std::string msg;
  for (int c = 0; c < nclass; ++c) {
    if (st[c] < 0 && (worst >= 0 || st[c] < worst)) {
      worst = st[c];
      msg = "class " + std::to_string(c) + ": " + err[c];
    } else if (st[c] == MPCG_NOT_CONVERGED && worst == MPCG_OK) {
      worst = st[c];
      msg = "class " + std::to_string(c) + " did not converge";
    }
  }
  mpcg::set_error_message(msg.c_str());
  return worst;
}
