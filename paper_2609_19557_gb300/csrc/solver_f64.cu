// Plain FP64 form of the solver (every vector, matrix value and sum in FP64).
#include "solver_impl.cuh"

namespace pdq {
SolverBase *make_solver_f64(cudaStream_t s) { return new Solver<double>(s); }
}  // namespace pdq
