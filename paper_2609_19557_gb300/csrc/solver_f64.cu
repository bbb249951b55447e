// Plain FP64 form of the solver (every vector, matrix value and sum in FP64).
#include "solver_impl.cuh"
#include "batch_impl.cuh"

namespace pdq {
SolverBase *make_solver_f64(cudaStream_t s) { return new Solver<double>(s); }
BatchBase *make_batch_f64(const std::vector<SolverBase *> &sv, const std::vector<int> &g_rows,
                          const std::vector<int> &g_cols, int chunk, std::string *err) {
  return make_batch_impl<double>(sv, g_rows, g_cols, chunk, err);
}
}  // namespace pdq
