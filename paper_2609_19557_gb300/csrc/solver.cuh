// Host orchestration of the PDNQP solver on one GPU: setup (Sec. 3.1), the
// outer proximal-ALM loop (Algorithm 3) on the host with its vector work in
// kernels, and the inner rAPDHG solve (Algorithm 4) driven entirely by the
// device: a CUDA graph of `chunk` trial slots is replayed, each slot being
// [primal, rows, cols, decide, average, check-rows, check-cols, check-final,
// check-apply]; every kernel reads the device-resident state and does nothing
// once the inner solve has stopped, so the host only polls the status
// between graph launches (Sec. 3.4, "GPU inner iterations").
#pragma once
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/pdnqp.h"
#include "common.cuh"

namespace pdq {

// Problem data after validation, classification (rows E first) and CSR
// construction on the host.
struct HostProblem {
  int n = 0, m = 0, mE = 0;
  std::vector<int> q_rp, q_ci, q_diag;
  std::vector<double> q_v;
  std::vector<int> a_rp, a_ci;
  std::vector<double> a_v;
  std::vector<int> at_rp, at_ci;
  std::vector<double> at_v;
  std::vector<double> c, lc, uc, lx, ux;  // lc/uc in internal row order; +-inf for absent bounds
  std::vector<int> perm;                  // internal row -> original row
};

// Algorithm parameters: Table tab:parameters plus the readings of the rules
// the paper leaves open.
struct Params {
  double time_limit = 1e30;
  long long k_out = 2147483647LL, k_in = 40000;
  double sigma_init = 20.0, theta_sigma = 0.25, delta_gamma = 1e-2;
  double rho_in_min = 0.3, rho_in_max = 0.95, rho_z = 0.95;
  int ruiz_outer = 8, ruiz_inner = 8, lanczos_steps = 64, k_chk = 64;
  double beta_suff = 0.2, beta_nec = 0.8, beta_art = 0.36;
  int rej_limit = 60;
  double kappa_shrink = 0.5;
  double delta_sigma = 2.0, sigma_max = 1e6, tol_floor = 0.1;
  double gamma_override = 0.0;
  int chunk = 128;
  long long iter_budget = 4000000000000000000LL;
  int g_rows = 0, g_cols = 0;  // entries per lane per CSR-stream chunk (0 = from the mean row length)
  int cond_graph = 1;          // 1: device-driven WHILE/IF graph; 0: unrolled slots (profilable)
  int persistent = 1;          // 1: persistent cooperative trial loop (when supported)
  int loop_blocks_per_sm = 0;  // blocks per SM of that loop (0: as many as fit)
  int controller = 0;          // 1: the learned controller proposes rho_in and the next primal weight
  double ctrl_explore = 0.0;   // std. dev. of Gaussian noise added to the actions (trajectory generation)
  long long ctrl_seed = 0;
  double eps_inf = 0.0;        // infeasibility tolerance on l_inf-normalised directions (0: 1e-5)
  int anderson = 1;            // Anderson acceleration of (lambda, z)
  int anderson_mem = 5;        // stored outer iterates m_A (2..5)
  int autotune = 0;            // 1: time the lanes-per-row choices of the graph form once, keep the fastest
  int escalate = 1;            // FP32-bulk: continue in FP64 after a NUMERICAL_ERROR
  int batch_fused = 1;         // pdnqp_solve_batch: 1 = one batched graph for all inner loops, 0 = thread pool
  int batch_chunk = 16;        // trial slots per launch of the batched graph
};

struct Result {
  int status = -1;
  double rp = 0, rd = 0, sp = 1, sd = 1, rel_kkt = 0;
  long long outer = 0, inner = 0, trials = 0, restarts = 0, passes = 0;
  long long rebases = 0;  // FP32-bulk: inner solves re-based at the rejection limit
  double seconds = 0, obj = 0;
  long long launches = 0;
  double inner_seconds = 0, setup_seconds = 0;
  double loop_seconds = 0;
  long long loop_trials = 0;
  int loop_blocks = 0;
  long long loop_launches = 0;
  long long ctrl_used = 0, ctrl_fallbacks = 0;  // outer iterations driven by the network / by the fallback
  double loop_phase_seconds[6] = {0, 0, 0, 0, 0, 0};
};

class SolverBase {
 public:
  virtual ~SolverBase() {}
  virtual int setup(const HostProblem &P, const Params &prm, std::string *err) = 0;
  virtual int solve(double ea, double er, Params &prm, std::string *err) = 0;
  virtual int get(double *x_int_orig, double *lam_int_orig, Result *r) = 0;
  virtual int set_start(const double *x0, const double *lam0_int) = 0;
  virtual int debug_inner(Params &prm, int nck, const int64_t *ck, double *snap, std::string *err) = 0;
  virtual int replay(int which, int reps) = 0;
  virtual int tuned_g(int which) const = 0;
  virtual double kernel_bytes(int which) const = 0;
  virtual double last_replay_ms() const = 0;
  virtual double gamma() const = 0;
  virtual double lambda_min() const = 0;
  virtual void set_gamma(double g) = 0;
  virtual int64_t nnz_q() const = 0;
  virtual int set_controller(const float *w, int count) = 0;
  virtual const std::vector<double> &trace() const = 0;
  virtual long long ctrl_fallbacks() const = 0;
};

SolverBase *make_solver_f64(cudaStream_t s);
SolverBase *make_solver_f32(cudaStream_t s);

// Batched form (fused): the inner iterations of several solvers of one
// precision run in one launch per phase of a captured CUDA graph, while
// each problem's outer iteration (Algorithm 3) runs on its own host thread.
// Built over solvers that have been set up; while it exists, their solves
// hand every inner solve to it.
class BatchBase {
 public:
  virtual ~BatchBase() {}
  // Worker thread of problem idx: its pdnqp_solve has returned.
  virtual void finished(int idx) = 0;
  // Calling thread: launches the batched graph until every problem has
  // finished; returns 0 or a negative code (the waiting solves then fail).
  virtual int schedule() = 0;
  virtual const std::string &error() const = 0;
  // Graph launches and batched kernel launches so far.
  virtual long long graph_launches() const = 0;
  // Device time of the batched graph launches (CUDA events on the batch's stream).
  virtual double graph_seconds() const = 0;
  virtual long long kernel_launches() const = 0;
};
// g_rows[i] / g_cols[i]: lanes per row of problem i's row and column passes
// (the values its solo graph form would use).
BatchBase *make_batch_f64(const std::vector<SolverBase *> &sv, const std::vector<int> &g_rows,
                          const std::vector<int> &g_cols, int chunk, std::string *err);
BatchBase *make_batch_f32(const std::vector<SolverBase *> &sv, const std::vector<int> &g_rows,
                          const std::vector<int> &g_cols, int chunk, std::string *err);

}  // namespace pdq
