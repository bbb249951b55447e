// External KKT test of a point (Sec. 4.1) on problem data held in device
// memory: the residuals of Eqs. outer-residuals / outer-scales on the
// original (unscaled) problem, with variable-bound violations counted in r_p.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/pdnqp.h"
#include "kkt_kernels.cuh"

namespace pdq {
namespace {

static thread_local std::string g_kkt_err;

int check_problem(const pdnqp_device_problem *P, const double *x, const double *y, const double *out) {
  if (!P || !x || !out) {
    g_kkt_err = "NULL argument";
    return PDNQP_ERR_ARG;
  }
  const int n = P->Q.n_rows, m = P->A.n_rows;
  if (n <= 0 || P->Q.n_cols != n || !P->Q.row_ptr || (P->Q.nnz > 0 && (!P->Q.col_idx || !P->Q.val))) {
    g_kkt_err = "Q must be a square n x n device CSR with n >= 1";
    return PDNQP_ERR_ARG;
  }
  if (P->Q.nnz < 0 || P->Q.nnz > 2147483647LL || P->A.nnz < 0 || P->A.nnz > 2147483647LL) {
    g_kkt_err = "nnz must fit the int32 CSR indices";
    return PDNQP_ERR_ARG;
  }
  if (m < 0 || (m > 0 && (P->A.n_cols != n || !P->A.row_ptr || !P->At.row_ptr || P->At.n_rows != n ||
                          P->At.n_cols != m || !P->l_c || !P->u_c || !y))) {
    g_kkt_err = "A (m x n), At (n x m), l_c, u_c and y are required when m > 0";
    return PDNQP_ERR_ARG;
  }
  if (!P->c || !P->l_x || !P->u_x) {
    g_kkt_err = "c, l_x and u_x are required";
    return PDNQP_ERR_ARG;
  }
  return 0;
}

int launch_kkt(const pdnqp_device_problem *P, const double *x, const double *y, double *out, double *scratch,
               cudaStream_t s) {
  const int n = P->Q.n_rows, m = P->A.n_rows;
  const int nb_r = grid_for(m > 0 ? m : 1, kBlock), nb_c = grid_for(n, kBlock);
  if (m > 0)
    k_kkt_rows<<<nb_r, kBlock, 0, s>>>(m, P->A.row_ptr, P->A.col_idx, P->A.val, P->l_c, P->u_c, x, scratch);
  else
    k_kkt_rows<<<1, kBlock, 0, s>>>(0, nullptr, nullptr, nullptr, nullptr, nullptr, x, scratch);
  k_kkt_cols<<<nb_c, kBlock, 0, s>>>(n, P->Q.row_ptr, P->Q.col_idx, P->Q.val, m > 0 ? P->At.row_ptr : nullptr,
                                     m > 0 ? P->At.col_idx : nullptr, m > 0 ? P->At.val : nullptr, P->c, P->l_x,
                                     P->u_x, x, y, scratch);
  k_kkt_final<<<1, kRedThreads, 0, s>>>(scratch, m > 0 ? nb_r : 1, nb_c, out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_kkt_err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return PDNQP_ERR_CUDA;
  }
  return 0;
}

// Scratch of pdnqp_kkt_residuals_noalloc: the block partial sums of one call,
// kKktQ quantities x kMaxBlocks blocks = 5 x 1216 doubles (48,640 bytes).
// Every device that loads the library holds this array until the process
// exits; all calls on a device share it.
static __device__ __align__(256) double g_kkt_noalloc_scratch[kKktQ * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the static scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached for the life of the
// process (a cudaDeviceReset, which unloads the module, invalidates it; the
// header tells callers not to use this entry point on a reset device).
int noalloc_scratch(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    g_kkt_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return PDNQP_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    g_kkt_err = "device ordinal out of range for the static scratch table";
    return PDNQP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_kkt_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      g_kkt_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return PDNQP_ERR_CUDA;
    }
    g_noalloc_ptr[dev] = (double *)p;
  }
  *out = g_noalloc_ptr[dev];
  return 0;
}

}  // namespace
}  // namespace pdq

extern "C" {

int pdnqp_kkt_residuals_noalloc(const pdnqp_device_problem *P, const double *x, const double *y, double *out,
                                void *stream) {
  using namespace pdq;
  int rc = check_problem(P, x, y, out);
  if (rc) return rc;
  // Each pass launches at most kMaxBlocks blocks (grid-stride over rows), so
  // the partial sums of any problem that fits the int32 CSR layout fit the
  // static array; a grid that would not fit is rejected.
  const int nb_r = grid_for(P->A.n_rows > 0 ? P->A.n_rows : 1, kBlock), nb_c = grid_for(P->Q.n_rows, kBlock);
  if (nb_r > kMaxBlocks || nb_c > kMaxBlocks) {
    g_kkt_err = "problem needs more partial sums than the static scratch holds (5 x 1216)";
    return PDNQP_ERR_ARG;
  }
  double *scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  // Every block writes its partial sums before the final kernel reads exactly
  // those entries, so nothing left by a previous call needs clearing.
  return launch_kkt(P, x, y, out, scratch, (cudaStream_t)stream);
}

int pdnqp_kkt_residuals(const pdnqp_device_problem *P, const double *x, const double *y, double *out,
                        void *stream) {
  using namespace pdq;
  int rc = check_problem(P, x, y, out);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  double *scratch = nullptr;
  cudaError_t e = cudaMalloc(&scratch, sizeof(double) * kKktQ * kMaxBlocks);
  if (e != cudaSuccess) {
    g_kkt_err = std::string("cudaMalloc: ") + cudaGetErrorString(e);
    return PDNQP_ERR_OOM;
  }
  rc = launch_kkt(P, x, y, out, scratch, s);
  e = cudaStreamSynchronize(s);
  cudaFree(scratch);
  if (rc) return rc;
  if (e != cudaSuccess) {
    g_kkt_err = std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e);
    return PDNQP_ERR_CUDA;
  }
  return 0;
}

const char *pdnqp_kkt_last_error(void) { return pdq::g_kkt_err.c_str(); }

}  // extern "C"
