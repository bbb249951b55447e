// FP32-bulk form of the solver: SpMVs and vector updates of the inner loop in
// FP32 with FP32 accumulation; acceptance sums, check/restart/termination
// reductions, multiplier and penalty updates and the setup in FP64.
#include "solver_impl.cuh"
#include "batch_impl.cuh"

namespace pdq {
SolverBase *make_solver_f32(cudaStream_t s) { return new Solver<float>(s); }
BatchBase *make_batch_f32(const std::vector<SolverBase *> &sv, const std::vector<int> &g_rows,
                          const std::vector<int> &g_cols, int chunk, std::string *err) {
  return make_batch_impl<float>(sv, g_rows, g_cols, chunk, err);
}
}  // namespace pdq
