// Kernels of the external KKT test (Sec. 4.1): residuals of Eqs.
// outer-residuals / outer-scales on the original data of Eq. qp, with
// variable-bound violations counted in r_p.  Included by each entry-point
// translation unit (internal linkage).
#pragma once
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"

namespace pdq {
namespace {

constexpr int kKktQ = 5;  // partial quantities: rows r_p, rows s_p, cols r_p, cols r_d, cols s_d (all maxima)

__global__ void __launch_bounds__(kBlock) k_kkt_rows(int m, const int *__restrict__ rp, const int *__restrict__ ci,
                                                     const double *__restrict__ v, const double *__restrict__ lc,
                                                     const double *__restrict__ uc, const double *__restrict__ x,
                                                     double *part) {
  double rpv = 0.0, spv = 0.0;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x) {
    double ax = 0.0;
    for (int k = rp[j]; k < rp[j + 1]; ++k) ax += v[k] * x[ci[k]];
    const double lo = lc[j] <= -1e20 ? -INFINITY : lc[j], hi = uc[j] >= 1e20 ? INFINITY : uc[j];
    rpv = fmax(rpv, res_term(ax < lo ? lo - ax : (ax > hi ? ax - hi : 0.0)));
    spv = fmax(spv, scale_term(fabs(ax)));
    if (isfinite(lo)) spv = fmax(spv, fabs(lo));
    if (isfinite(hi)) spv = fmax(spv, fabs(hi));
  }
  double q[2] = {rpv, spv};
  block_reduce_store<2>(q, 3u, part);
}

__global__ void __launch_bounds__(kBlock) k_kkt_cols(int n, const int *__restrict__ qrp, const int *__restrict__ qci,
                                                     const double *__restrict__ qv, const int *__restrict__ trp,
                                                     const int *__restrict__ tci, const double *__restrict__ tv,
                                                     const double *__restrict__ c, const double *__restrict__ lx,
                                                     const double *__restrict__ ux, const double *__restrict__ x,
                                                     const double *__restrict__ y, double *part) {
  double rpv = 0.0, rdv = 0.0, sdv = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double qx = 0.0, aty = 0.0;
    for (int k = qrp[i]; k < qrp[i + 1]; ++k) qx += qv[k] * x[qci[k]];
    if (trp)
      for (int k = trp[i]; k < trp[i + 1]; ++k) aty += tv[k] * y[tci[k]];
    const double lo = lx[i] <= -1e20 ? -INFINITY : lx[i], hi = ux[i] >= 1e20 ? INFINITY : ux[i];
    const double xi = x[i];
    rpv = fmax(rpv, res_term(xi < lo ? lo - xi : (xi > hi ? xi - hi : 0.0)));
    double p = xi - (qx + c[i] + aty);
    p = p < lo ? lo : p;
    p = p > hi ? hi : p;
    rdv = fmax(rdv, res_term(fabs(xi - p)));
    sdv = fmax(sdv, fmax(scale_term(fabs(qx)), fmax(fabs(c[i]), scale_term(fabs(aty)))));
  }
  double q[3] = {rpv, rdv, sdv};
  block_reduce_store<3>(q, 7u, part + 2 * kMaxBlocks);
}

__global__ void __launch_bounds__(kRedThreads) k_kkt_final(const double *part, int nb_r, int nb_c, double *out) {
  double a[2], b[3];
  final_reduce<2>(part, nb_r, 3u, a);
  final_reduce<3>(part + 2 * kMaxBlocks, nb_c, 7u, b);
  if (threadIdx.x == 0) {
    out[0] = fmax(a[0], b[0]);
    out[1] = b[1];
    out[2] = fmax(1.0, a[1]);
    out[3] = fmax(1.0, b[2]);
  }
}

}  // namespace
}  // namespace pdq
