// Kernels of the one-time setup (Sec. 3.1: outer Ruiz scaling, objective
// scalar, Lanczos estimate for gamma, initial penalties) and of the outer
// glue of Algorithm 3 (Eqs. practical-multiplier-update, outer-residuals,
// outer-scales, penalty-trigger-eq).  All of them compute in FP64.
#pragma once
#include <math.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.cuh"

namespace pdq {
namespace {  // internal linkage: each solver TU owns its kernels

// ---------------------------------------------------------------------------
// Outer Ruiz scaling of [[Q, A^T], [A, 0]] (Eq. scaled-problem).
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(kBlock) k_oruiz_rows(Mat<double> A, const double *Dc, const double *Dx, double *rn) {
  GroupIter<G> it;
  for (long long base = it.first; base < A.nrows; base += it.step) {
    const long long j = base + it.sub;
    const bool valid = j < A.nrows;
    const double dj = valid ? Dc[j] : 0.0;
    const double a = row_max<G, double>(A.rp, A.ci, A.val, j, valid, it.lane_g,
                                        [&](int k, double v) { return fabs(dj * v * Dx[k]); });
    if (valid && it.lane_g == 0) rn[j] = a;
  }
}

template <int G>
__global__ void __launch_bounds__(kBlock) k_oruiz_cols(Mat<double> At, Mat<double> Q, const double *Dc,
                                                       const double *Dx, double *cn) {
  GroupIter<G> it;
  for (long long base = it.first; base < Q.nrows; base += it.step) {
    const long long i = base + it.sub;
    const bool valid = i < Q.nrows;
    const double di = valid ? Dx[i] : 0.0;
    const double a = row_max<G, double>(At.rp, At.ci, At.val, i, valid, it.lane_g,
                                        [&](int k, double v) { return fabs(Dc[k] * v * di); });
    const double b = row_max<G, double>(Q.rp, Q.ci, Q.val, i, valid, it.lane_g,
                                        [&](int k, double v) { return fabs(di * v * Dx[k]); });
    if (valid && it.lane_g == 0) cn[i] = fmax(a, b);
  }
}

__global__ void k_ruiz_apply(double *D, const double *nrm, long long len) {
  PDNQP_GRID_STRIDE(i, len) {
    const double c = nrm[i];
    if (c > 0.0) D[i] = D[i] * (1.0 / sqrt(c));
  }
}

// val_k *= mult * rs[row] * cs[col]
__global__ void k_scale_csr(int nrows, const int *rp, const int *ci, double *val, const double *rs, const double *cs,
                            double mult) {
  PDNQP_GRID_STRIDE(i, nrows) {
    const double ri = rs[i] * mult;
    for (int k = rp[i]; k < rp[i + 1]; ++k) val[k] = ri * val[k] * cs[ci[k]];
  }
}

// Max absolute row sum (induced l_inf norm) partials of a CSR matrix.
template <int G>
__global__ void __launch_bounds__(kBlock) k_rowabs_max(Mat<double> M, double *part) {
  double best = 0.0;
  GroupIter<G> it;
  for (long long base = it.first; base < M.nrows; base += it.step) {
    const long long i = base + it.sub;
    const bool valid = i < M.nrows;
    const double s = row_sum<G, double>(M.rp, M.ci, M.val, i, valid, it.lane_g, [&](int, double v) { return fabs(v); });
    if (valid && it.lane_g == 0) best = fmax(best, s);
  }
  double v[1] = {best};
  block_reduce_store<1>(v, 1u, part);
}

__global__ void k_absmax(const double *v, long long n, double *part) {
  double best = 0.0;
  PDNQP_GRID_STRIDE(i, n) best = fmax(best, fabs(v[i]));
  double q[1] = {best};
  block_reduce_store<1>(q, 1u, part);
}

// Reduction of nq quantities (row q of part, nb partials each) -> out[q]:
// block q reduces quantity q (fixed order: lane-strided serial sums, then a
// serial sum of the 32 lane sums).
__global__ void __launch_bounds__(32) k_reduce_rows(const double *part, int nq, int nb, unsigned max_mask, double *out) {
  __shared__ double ls[32];
  const int q = blockIdx.x, lane = threadIdx.x;
  if (q >= nq) return;
  const bool mx = q < 32 && ((max_mask >> q) & 1u);
  double a = 0.0;
  for (int b = lane; b < nb; b += 32) {
    const double p = part[(long long)q * kMaxBlocks + b];
    a = mx ? fmax(a, p) : a + p;
  }
  ls[lane] = a;
  __syncwarp();
  if (lane == 0) {
    double r = ls[0];
    for (int k = 1; k < 32; ++k) r = mx ? fmax(r, ls[k]) : r + ls[k];
    out[q] = r;
  }
}

// Diagonal shift: val[diag[i]] += s (diag[i] = position of (i, i) in row i).
__global__ void k_add_diag(int n, const int *diag, double *val, double s) {
  PDNQP_GRID_STRIDE(i, n) val[diag[i]] += s;
}

__global__ void k_scale_vec(double *v, const double *by, long long n, int divide, double mult) {
  PDNQP_GRID_STRIDE(i, n) v[i] = (divide ? v[i] / by[i] : v[i] * by[i]) * mult;
}

template <typename T>
__global__ void k_to_T(T *dst, const double *src, long long n) {
  PDNQP_GRID_STRIDE(i, n) dst[i] = T(src[i]);
}
template <typename T>
__global__ void k_from_T(double *dst, const T *src, long long n) {
  PDNQP_GRID_STRIDE(i, n) dst[i] = double(src[i]);
}

__global__ void k_fill_d(double *p, long long n, double v) {
  PDNQP_GRID_STRIDE(i, n) p[i] = v;
}
__global__ void k_mul_scalar(double *p, long long n, double a) {
  PDNQP_GRID_STRIDE(i, n) p[i] *= a;
}
__global__ void __launch_bounds__(kBlock) k_dot(const double *a, const double *b, long long n, double *part) {
  double s = 0.0;
  PDNQP_GRID_STRIDE(i, n) s += a[i] * b[i];
  double q[1] = {s};
  block_reduce_store<1>(q, 0u, part);
}
// h = (b_E, 0) (Eq. inner-qp), b_E = l_c on the equality rows.
template <typename T>
__global__ void k_form_h(T *h, const double *lc, long long m, int mE) {
  PDNQP_GRID_STRIDE(j, m) h[j] = j < mE ? T(lc[j]) : T(0);
}

// ---------------------------------------------------------------------------
// Lanczos (Eq. R-choice): SpMV, dot products, full reorthogonalisation by
// classical Gram-Schmidt applied twice.
// ---------------------------------------------------------------------------
// i-th output of the splitmix64 generator seeded with `seed`, mapped to [-0.5, 0.5).
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}
__global__ void k_start_vector(double *v, long long n, uint64_t seed) {
  PDNQP_GRID_STRIDE(i, n) v[i] = splitmix_uniform(seed, (uint64_t)i);
}

template <int G>
__global__ void __launch_bounds__(kBlock) k_spmv(Mat<double> M, const double *x, double *y) {
  GroupIter<G> it;
  for (long long base = it.first; base < M.nrows; base += it.step) {
    const long long i = base + it.sub;
    const bool valid = i < M.nrows;
    const double s = row_sum<G, double>(M.rp, M.ci, M.val, i, valid, it.lane_g, [&](int k, double v) { return v * x[k]; });
    if (valid && it.lane_g == 0) y[i] = s;
  }
}

// Partials of V[p] . w for p = blockIdx.y (rows p of part).
__global__ void __launch_bounds__(kBlock) k_multidot(const double *V, long long n, const double *w, double *part) {
  const double *vp = V + (long long)blockIdx.y * n;
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s += vp[i] * w[i];
  double q[1] = {s};
  block_reduce_store<1>(q, 0u, part + (long long)blockIdx.y * kMaxBlocks);
}

// w -= sum_{p < np} h[p] V[p]
__global__ void k_multiaxpy(const double *V, long long n, const double *h, int np, double *w) {
  PDNQP_GRID_STRIDE(i, n) {
    double s = w[i];
    for (int p = 0; p < np; ++p) s -= h[p] * V[(long long)p * n + i];
    w[i] = s;
  }
}

// w = w - a v - b u   (u may be null)
__global__ void k_lanczos_axpy(double *w, const double *v, const double *u, double a, double b, long long n) {
  PDNQP_GRID_STRIDE(i, n) {
    double s = w[i] - a * v[i];
    if (u) s -= b * u[i];
    w[i] = s;
  }
}
__global__ void k_scale_into(double *dst, const double *src, double a, long long n) {
  PDNQP_GRID_STRIDE(i, n) dst[i] = src[i] * a;
}

// ---------------------------------------------------------------------------
// Initial point and penalties (Sec. 3.2.1).
// ---------------------------------------------------------------------------
// x = P_[lx,ux](x0 / Dx) (x0 already in the original coordinates, or null).
__global__ void k_init_x(long long n, const double *x0, const double *Dx, const double *lx, const double *ux,
                         double *x64, double *z) {
  PDNQP_GRID_STRIDE(i, n) {
    double v = x0 ? x0[i] / Dx[i] : 0.0;
    v = v < lx[i] ? lx[i] : v;
    v = v > ux[i] ? ux[i] : v;
    x64[i] = v;
    z[i] = v;
  }
}

// lambda (scaled) = c_s lambda0 / Dc (internal row order), inner y = -lambda.
__global__ void k_init_lambda(long long m, double *lam, const double *lam0_int, const double *Dc, double cs,
                              double *y64) {
  PDNQP_GRID_STRIDE(j, m) {
    const double l = lam0_int ? cs * lam0_int[j] / Dc[j] : 0.0;
    lam[j] = l;
    y64[j] = -l;
  }
}

// Rows of the initial point: partial sum of dist(Ax, [lc, uc])^2, and the
// residual r = A x - P(A x + lambda / sigma) once sigma is known (pass 2).
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_init_rows(Dev<T> d, Mat<double> Ad, const double *lc, const double *uc,
                                                      double *lam, const double *sig, double *rprev, int pass) {
  const double *__restrict__ x = d.xb;
  double acc = 0.0;
  GroupIter<G> it;
  for (long long base = it.first; base < d.m; base += it.step) {
    const long long j = base + it.sub;
    const bool valid = j < d.m;
    const double ax = row_sum<G, double>(Ad.rp, Ad.ci, Ad.val, j, valid, it.lane_g,
                                         [&](int k, double a) { return a * double(x[k]); });
    if (valid && it.lane_g == 0) {
      const double lo = lc[j], hi = uc[j];
      if (pass == 0) {
        double p = ax;
        p = p < lo ? lo : p;
        p = p > hi ? hi : p;
        acc += (ax - p) * (ax - p);
      } else {
        double s;
        if (j < d.mE) {
          s = lo;
        } else {
          s = ax + lam[j] / sig[j];
          s = s < lo ? lo : s;
          s = s > hi ? hi : s;
        }
        rprev[j] = ax - s;
      }
    }
  }
  double v[1] = {acc};
  block_reduce_store<1>(v, 0u, d.part);
}

// Partials of x'Qx (from H x - gamma^-1 x) and c'x.
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_objective(Dev<T> d, Mat<double> Hd, const double *c, double ginv) {
  const double *__restrict__ x = d.xb;
  double xqx = 0.0, cx = 0.0;
  GroupIter<G> it;
  for (long long base = it.first; base < d.n; base += it.step) {
    const long long i = base + it.sub;
    const bool valid = i < d.n;
    const double hx = row_sum<G, double>(Hd.rp, Hd.ci, Hd.val, i, valid, it.lane_g,
                                         [&](int k, double a) { return a * double(x[k]); });
    if (valid && it.lane_g == 0) {
      const double xi = double(x[i]);
      xqx += xi * (hx - ginv * xi);
      cx += c[i] * xi;
    }
  }
  double v[2] = {xqx, cx};
  block_reduce_store<2>(v, 0u, d.part);
}

// ---------------------------------------------------------------------------
// Outer glue (Algorithm 3).
// ---------------------------------------------------------------------------
// Quantities of the outer residual reduction (rows of part):
//   0 r_p scaled, 1 s_p scaled, 2 r_p unscaled, 3 s_p unscaled, 4 ||r||_inf (rows)
//   5 r_d scaled, 6 s_d scaled, 7 r_d unscaled, 8 s_d unscaled, 9 ||x - z||_inf,
//   10 x'Qx, 11 c'x                         (10, 11 sums; the rest maxima)
constexpr unsigned OUT_MAXMASK = 0x3FFu;

// Eq. practical-multiplier-update (two-sided rows) + row terms of the residuals.
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_outer_rows(Dev<T> d, Mat<double> Ad, const double *lc, const double *uc,
                                                       const double *Dc, double *lam, const double *sig, double *rcur,
                                                       int update) {
  const double *__restrict__ x = d.xb;  // outer x (FP64)
  double q[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) q[k] = 0.0;
  TileIter ti;
  for (long long tile = ti.first; tile < d.m; tile += ti.step) {
    const double ax = tile_row_sum<G, double>(Ad.rp, Ad.ci, Ad.val, tile, d.m,
                                              [&](int k, double a) { return a * double(x[k]); });
    const long long j = tile + ti.lane;
    if (j < d.m) {
      const double lo = lc[j], hi = uc[j];
      if (update) {
        double s;
        if (j < d.mE) {
          s = lo;
        } else {
          s = ax + lam[j] / sig[j];
          s = s < lo ? lo : s;
          s = s > hi ? hi : s;
        }
        const double r = ax - s;
        lam[j] = lam[j] + sig[j] * r;
        rcur[j] = r;
        q[4] = fmax(q[4], fabs(r));
      }
      const double viol = ax < lo ? lo - ax : (ax > hi ? ax - hi : 0.0);
      double spv = scale_term(fabs(ax));
      if (isfinite(lo)) spv = fmax(spv, fabs(lo));
      if (isfinite(hi)) spv = fmax(spv, fabs(hi));
      q[0] = fmax(q[0], res_term(viol));
      q[1] = fmax(q[1], spv);
      const double dc = Dc[j];
      q[2] = fmax(q[2], res_term(viol / dc));
      q[3] = fmax(q[3], spv / dc);
    }
  }
  block_reduce_store<12>(q, OUT_MAXMASK, d.part);
}

// Column terms: Qx = H x - gamma^-1 x, A' lambda, projected stationarity in the
// scaled and the original coordinates (x = Dx xbar, lambda = Dc lambdabar / c_s).
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_outer_cols(Dev<T> d, Mat<double> Hd, Mat<double> Atd, const double *c,
                                                       const double *lx, const double *ux, const double *Dx,
                                                       const double *lam, const double *z, double ginv, double cs) {
  const double *__restrict__ x = d.xb;  // outer x (FP64)
  double q[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) q[k] = 0.0;
  TileIter ti;
  for (long long tile = ti.first; tile < d.n; tile += ti.step) {
    const double hx = tile_row_sum<G, double>(Hd.rp, Hd.ci, Hd.val, tile, d.n,
                                              [&](int k, double a) { return a * double(x[k]); });
    const double atl = tile_row_sum<G, double>(Atd.rp, Atd.ci, Atd.val, tile, d.n,
                                               [&](int k, double a) { return a * lam[k]; });
    const long long i = tile + ti.lane;
    if (i < d.n) {
      const double xi = double(x[i]);
      const double qx = hx - ginv * xi;
      const double g = qx + c[i] + atl;
      const double lo = lx[i], hi = ux[i];
      double p = xi - g;
      p = p < lo ? lo : p;
      p = p > hi ? hi : p;
      q[5] = fmax(q[5], res_term(fabs(xi - p)));
      q[6] = fmax(q[6], fmax(scale_term(fabs(qx)), fmax(fabs(c[i]), scale_term(fabs(atl)))));
      const double f = 1.0 / (cs * Dx[i]);
      const double xo = Dx[i] * xi, loo = lo * Dx[i], hio = hi * Dx[i], go = g * f;
      double po = xo - go;
      po = po < loo ? loo : po;
      po = po > hio ? hio : po;
      q[7] = fmax(q[7], res_term(fabs(xo - po)));
      q[2] = fmax(q[2], res_term(xo < loo ? loo - xo : (xo > hio ? xo - hio : 0.0)));
      q[8] = fmax(q[8], fmax(scale_term(fabs(qx * f)), fmax(fabs(c[i] * f), scale_term(fabs(atl * f)))));
      q[9] = fmax(q[9], fabs(xi - z[i]));
      q[10] += xi * qx;
      q[11] += c[i] * xi;
    }
  }
  block_reduce_store<12>(q, OUT_MAXMASK, d.part + 12 * kMaxBlocks);
}

// Infeasibility tests (Sec. "Infeasibility detection") on the scaled problem,
// from the changes over one outer iteration dlam = lambda^{k+1} - lambda^k and
// dx = x^{k+1} - x^k.  Unnormalised quantities; the host divides by the
// norms.  Rows (4): 0 largest |dlam_j| that would need an infinite row bound
// (sign condition), 1 sum of the finite-bound terms of sigma_C(dlam), 2
// largest departure of (A dx)_j from the recession cone of [l_c, u_c], 3
// ||dlam||_inf.
constexpr unsigned INF_R_MAXMASK = 0xDu;
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_inf_rows(Dev<T> d, Mat<double> Ad, const double *lc, const double *uc,
                                                     const double *lam, const double *lam0, const double *dx) {
  double q[4] = {0.0, 0.0, 0.0, 0.0};
  TileIter ti;
  for (long long tile = ti.first; tile < d.m; tile += ti.step) {
    const double ad = tile_row_sum<G, double>(Ad.rp, Ad.ci, Ad.val, tile, d.m, [&](int k, double a) { return a * dx[k]; });
    const long long j = tile + ti.lane;
    if (j < d.m) {
      const double y = lam[j] - lam0[j], lo = lc[j], hi = uc[j];
      if (y > 0.0) {
        if (isinf(hi)) q[0] = fmax(q[0], y); else q[1] += hi * y;
      } else if (y < 0.0) {
        if (isinf(lo)) q[0] = fmax(q[0], -y); else q[1] += lo * y;
      }
      if (!isinf(lo) && ad < 0.0) q[2] = fmax(q[2], -ad);
      if (!isinf(hi) && ad > 0.0) q[2] = fmax(q[2], ad);
      q[3] = fmax(q[3], fabs(y));
    }
  }
  block_reduce_store<4>(q, INF_R_MAXMASK, d.part);
}

// Columns (7): 0 largest |v_i|, v = -A' dlam, that would need an infinite
// variable bound, 1 sum of the finite-bound terms of sigma_X(v), 2 largest
// departure of dx_i from the recession cone of [l_x, u_x], 3 dx'Q dx, 4 c'dx,
// 5 ||Q dx||_inf, 6 ||dx||_inf (Q dx = H dx - dx / gamma).
constexpr unsigned INF_C_MAXMASK = 0x65u;
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_inf_cols(Dev<T> d, Mat<double> Hd, Mat<double> Atd, const double *c,
                                                     const double *lx, const double *ux, const double *lam,
                                                     const double *lam0, const double *dx, double ginv) {
  double q[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  TileIter ti;
  for (long long tile = ti.first; tile < d.n; tile += ti.step) {
    const double atl = tile_row_sum<G, double>(Atd.rp, Atd.ci, Atd.val, tile, d.n,
                                               [&](int k, double a) { return a * (lam[k] - lam0[k]); });
    const double hd = tile_row_sum<G, double>(Hd.rp, Hd.ci, Hd.val, tile, d.n, [&](int k, double a) { return a * dx[k]; });
    const long long i = tile + ti.lane;
    if (i < d.n) {
      const double v = -atl, di = dx[i], qd = hd - ginv * di, lo = lx[i], hi = ux[i];
      if (v > 0.0) {
        if (isinf(hi)) q[0] = fmax(q[0], v); else q[1] += hi * v;
      } else if (v < 0.0) {
        if (isinf(lo)) q[0] = fmax(q[0], -v); else q[1] += lo * v;
      }
      if (!isinf(lo) && di < 0.0) q[2] = fmax(q[2], -di);
      if (!isinf(hi) && di > 0.0) q[2] = fmax(q[2], di);
      q[3] += di * qd;
      q[4] += c[i] * di;
      q[5] = fmax(q[5], fabs(qd));
      q[6] = fmax(q[6], fabs(di));
    }
  }
  block_reduce_store<7>(q, INF_C_MAXMASK, d.part);
}

// Anderson acceleration (Sec. "Anderson acceleration"): sums of one Type-II
// step over the stored pairs (U_a, G_a), a = 0..L-1 oldest first, physical
// slot (head + a) % cap, D = m + n doubles each.  With f_a = G_a - U_a,
// dF_a = f_{a+1} - f_a (a < nc = L - 1) and f_k = f_{L-1}: out rows
// a * nc + b = dF_a'dF_b, nc * nc + a = dF_a'f_k, nc * nc + nc = f_k'f_k.
template <int NC>
__global__ void __launch_bounds__(kBlock) k_aa_dots(const double *U, const double *G, int head, int cap, long long D,
                                                    double *part) {
  constexpr int NQ = NC * NC + NC + 1;
  double q[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) q[k] = 0.0;
  PDNQP_GRID_STRIDE(i, D) {
    double f[NC + 1];
#pragma unroll
    for (int a = 0; a <= NC; ++a) {
      const long long s = (long long)((head + a) % cap) * D;
      f[a] = G[s + i] - U[s + i];
    }
    double df[NC];
#pragma unroll
    for (int a = 0; a < NC; ++a) df[a] = f[a + 1] - f[a];
#pragma unroll
    for (int a = 0; a < NC; ++a) {
#pragma unroll
      for (int b = 0; b < NC; ++b) q[a * NC + b] += df[a] * df[b];
      q[NC * NC + a] += df[a] * f[NC];
    }
    q[NC * NC + NC] += f[NC] * f[NC];
  }
  block_reduce_store<NQ>(q, 0u, part);
}

// The extrapolated point out = G_{L-1} - sum_a gam_a (G_{a+1} - G_a) and the
// squared norm of the correction (row 0 of part).
__global__ void __launch_bounds__(kBlock) k_aa_apply(const double *G, int head, int cap, int nc, long long D,
                                                     double g0, double g1, double g2, double g3, double *out,
                                                     double *part) {
  const double gam[4] = {g0, g1, g2, g3};
  double sn[1] = {0.0};
  PDNQP_GRID_STRIDE(i, D) {
    double v = 0.0;
    for (int a = 0; a < nc; ++a) {
      const long long s0 = (long long)((head + a) % cap) * D, s1 = (long long)((head + a + 1) % cap) * D;
      v += gam[a] * (G[s1 + i] - G[s0 + i]);
    }
    out[i] = G[(long long)((head + nc) % cap) * D + i] - v;
    sn[0] += v * v;
  }
  block_reduce_store<1>(sn, 0u, part);
}

__global__ void k_sub(long long n, const double *a, const double *b, double *out) {
  PDNQP_GRID_STRIDE(i, n) out[i] = a[i] - b[i];
}

// Eq. penalty-trigger-eq with the growth rule (only when `grow`: the primal
// part of the termination test still fails).  Stores r as the previous residual.
__global__ void k_sigma_update(int m, int mE, double *sig, const double *lam, const double *rcur, double *rprev,
                               double theta, int grow, double rn, double dsig, double smax) {
  PDNQP_GRID_STRIDE(j, m) {
    const double r = rcur[j];
    const bool active = j < mE || lam[j] != 0.0;
    if (grow && active && fabs(r) > theta * fabs(rprev[j]) && rn > 0.0)
      sig[j] = fmin(smax, sig[j] * fmax(1.0, dsig * fabs(r) / rn));
    rprev[j] = r;
  }
}

template <typename T>
__global__ void k_copy_T(T *dst, const T *src, long long n) {
  PDNQP_GRID_STRIDE(i, n) dst[i] = src[i];
}
template <typename T>
__global__ void k_copy_to_double(double *dst, const T *src, long long n) {
  PDNQP_GRID_STRIDE(i, n) dst[i] = double(src[i]);
}

// Unscaling for the result: x_orig = Dx x, lambda_orig = Dc lambda / c_s.
template <typename T>
__global__ void k_unscale(const T *x, const double *Dx, long long n, const double *lam, const double *Dc, long long m,
                          double cs, double *xo, double *lo) {
  PDNQP_GRID_STRIDE(i, n) xo[i] = Dx[i] * double(x[i]);
  PDNQP_GRID_STRIDE(j, m) lo[j] = Dc[j] * lam[j] / cs;
}

}  // namespace
}  // namespace pdq
