// Failure-detection self-test: makes each kind of bounded device wait of the
// trial loop run out on purpose, without a fault.  A grid barrier that one
// block never reaches, and a bulk-copy mbarrier that expects bytes nothing
// sends, are the two waits the persistent loop can be stuck in; both must give
// up after their poll limits, set the fault flag and return, leaving the
// context usable.
#include <cuda_runtime.h>

#include <chrono>

#include "../../include/pdnqp.h"
#include "common.cuh"

namespace pdq {
namespace {

// Block 0 leaves before the barrier: no leader ever releases the others.
__global__ void k_selftest_barrier(unsigned *bar, int *ret) {
  if (blockIdx.x == 0) return;
  const bool ok = grid_sync(bar);
  if (threadIdx.x == 0) ret[blockIdx.x] = ok ? 1 : 0;
}

// One arrival with an expected transaction of 16 bytes and no copy issued:
// the phase never completes.  No asynchronous operation is in flight.
__global__ void k_selftest_tx(unsigned *fault, int *ret) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16u);
  __syncthreads();
  const bool ok = mbar_wait_warp(&bar, 0u, fault);
  if ((threadIdx.x & 31) == 0) ret[threadIdx.x >> 5] = ok ? 1 : 0;
}

}  // namespace
}  // namespace pdq

extern "C" int pdnqp_selftest_wait(int kind, int *gave_up, double *seconds) {
  using namespace pdq;
  if ((kind != 0 && kind != 1) || !gave_up) return PDNQP_ERR_ARG;
  constexpr int kBlocks = 4, kRet = 8;
  unsigned *bar = nullptr;
  int *ret = nullptr;
  if (cudaMalloc(&bar, kBarWords * sizeof(unsigned)) != cudaSuccess) return PDNQP_ERR_OOM;
  if (cudaMalloc(&ret, kRet * sizeof(int)) != cudaSuccess) {
    cudaFree(bar);
    return PDNQP_ERR_OOM;
  }
  int rc = 0;
  int hret[kRet];
  unsigned hbar[kBarWords];
  const auto t0 = std::chrono::steady_clock::now();
  if (cudaMemset(bar, 0, kBarWords * sizeof(unsigned)) != cudaSuccess ||
      cudaMemset(ret, 0xff, kRet * sizeof(int)) != cudaSuccess) {
    rc = PDNQP_ERR_CUDA;
  } else {
    if (kind == 0)
      k_selftest_barrier<<<kBlocks, kBlock>>>(bar, ret);
    else
      k_selftest_tx<<<1, kBlock>>>(bar + kBarFault, ret);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(hret, ret, sizeof(hret), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(hbar, bar, sizeof(hbar), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = PDNQP_ERR_CUDA;
  }
  const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (seconds) *seconds = dt;
  if (rc == 0) {
    // Every waiter reported failure and the fault flag is set.
    bool all = hbar[kBarFault] == 1u;
    const int first = kind == 0 ? 1 : 0, last = kind == 0 ? kBlocks : kBlock / 32;
    for (int b = first; b < last; ++b) all = all && hret[b] == 0;
    *gave_up = all ? 1 : 0;
  }
  cudaFree(bar);
  cudaFree(ret);
  return rc;
}
