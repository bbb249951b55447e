// CUDA kernels of the PDNQP hot path (Algorithm 4) and of its setup and outer
// glue (Algorithm 3, Sec. 3.1), templated on the storage type T of the inner
// iterates and matrix values (double: plain FP64 form; float: FP32-bulk form).
//
// Coordinates.  The inner iterates live in the outer-scaled, inner-UNSCALED
// coordinates of Eq. inner-qp: w = (x, s_I, r_E, r_I), y, stored as
// corrections from the FP64 base point of the solve (the warm start w_b, y_b):
// w = w_b + dw, y = y_b + dy.  The base enters only through the gradient of
// the inner objective at the base (q' = q + H w_b - B'y_b), the residual
// h' = h - B w_b and the shifted bounds, so the iteration is exactly PDHG on
// (dw, dy) and the FP32-bulk form keeps full relative precision in the
// corrections.  The penalty scaling
// (Eq. inner-penalty-scaling) and the inner Ruiz scaling (Sec. 3.3.2) are the
// diagonal change of variables w = E w~, y = D y~; PDHG in the scaled space is
// exactly PDHG in these coordinates with the effective diagonal steps
// tau_eff = e^2 tau~ and eta_eff = d^2 eta~, and the acceptance test (Eq.
// adaptive-condition) is invariant under it.  So the CSR values of A, A^T and
// Q are never rewritten inside the solve: the scalings only enter the step
// vectors and the scaled restart metric.
//
// H_k = diag(Q + gamma^-1 I, 0, sigma_E, sigma_I) and B = [[A_E, 0, -I, 0],
// [A_I, -I, 0, -I]] are never formed: their s and r blocks are diagonal and
// handled inline, and only the x blocks are SpMVs (Sec. 3.4: one product each
// with Q, A and A^T per trial).
#pragma once
#include <math.h>

#include "common.cuh"

namespace pdq {
namespace {  // internal linkage: each solver TU owns its kernels

// Rows of the partial-sums array used by each reduction.
constexpr int P_TR_R = 0;    // trial, row kernel: lhs_tau, lhs_eta, rhs_h, rhs_b
constexpr int P_TR_C = 4;    // trial, column kernel (same 4)
constexpr int P_CK_R = 8;    // check, row kernel: 16 quantities
constexpr int P_CK_C = 24;   // check, column kernel: 16 quantities
constexpr unsigned CK_MAXMASK = 0x0F0Fu;  // quantities 0-3 and 8-11 of a check are maxima
// Counter words (d.ctr): [0] column last-block counter, [1] check last-block
// counter, [2] row last-block counter (long rows), [kCtrBar, kCtrBar + kBarWords) the grid barrier of the persistent loop.
constexpr int kCtrBar = 128, kCtrWords = kCtrBar + kBarWords;
// Rows of A with more entries than this are treated as dense coupling rows
// (at most kMaxLong of them, the longest first; the rest stay row-wise).
constexpr int kLongRowMin = 1024;
constexpr int kMaxLong = 64;

template <typename T>
struct Mat {
  int nrows;
  const int *rp;
  const int *ci;
  const T *val;
};

// Device pointers of one solver (passed by value to the trial kernels).
template <typename T>
struct Dev {
  int n, m, mE;
  Mat<T> H, A, At;  // H = Qbar + gamma^-1 I (x block of H_k), A (rows E then I), A^T
  // n-vectors: corrections dx and their cached products H dx, A' dy, averages
  T *x[2], *Hx[2], *Aty[2], *xbar[2], *Hxbar[2];
  T *qx;          // q'_x = c - z / gamma + H x_b - A' y_b
  T *qx0;         // q_x = c - z / gamma (scale s_d)
  T *Hxb, *Atyb;  // H x_b, A' y_b (scales)
  T *lx, *ux;     // shifted bounds l - x_b, u - x_b
  T *taux, *itaux, *ex, *xst, *Atybar;
  // m-vectors (s is indexed by row; entries of equality rows are unused)
  T *y[2], *s[2], *r[2], *Bw[2], *ybar[2], *sbar[2], *rbar[2];
  T *qs;          // y_b: gradient of the s block at the base (I rows)
  T *qr;          // lambda + sigma r_b + y_b: gradient of the r block at the base
  T *hp;          // h - B w_b
  T *h, *Bwb;     // h and B w_b (scale s_p)
  T *ls, *us;     // shifted slack bounds l_c - s_b, u_c - s_b (I rows)
  T *eta, *taus, *taur, *ieta, *itaus, *itaur, *es, *er, *dy, *yst, *sst, *rst, *Bwbar;
  // FP64 base point and outer data
  const double *xb, *yb, *sb, *rb;  // base: outer x, inner y, warm-start s and r
  const double *lam, *sig;          // multipliers and row penalties
  double *part;
  // Dense coupling rows (more than kLongRowMin entries): their products are
  // split evenly over the blocks of the row pass, and the block that
  // arrives last combines the block partials in block order and updates
  // those rows.  As is A with these rows emptied (As == A when nlr == 0).
  int nlr;
  int lr_nnz;
  Mat<T> As;
  const int *lr_row;   // [nlr] row index of each long row (ascending)
  const int *lr_ptr;   // [nlr + 1] offsets into lr_ci / lr_val
  const int *lr_ci;
  const T *lr_val;
  const unsigned char *lr_flag;  // [m] 1 for a long row
  double *lr_part;     // [kMaxLong][kMaxBlocks] block partial products
  double *lr_acc;      // [4] acceptance-sum terms of the long rows (added to the row sums)
  DevState *st;
  unsigned *ctr;   // arrival counters of the last-block reductions (reset by the last block)
  unsigned long long *ptime;  // persistent loop: ns spent in the primal, row and column(+decision) passes
  cudaGraphConditionalHandle hw, hc;  // device-loop handles (0 when the graph has none)
};

template <typename T>
__device__ __forceinline__ T clampv(T v, T lo, T hi) {
  // Same comparison order as a plain projection: NaN stays NaN.
  v = v < lo ? lo : v;
  v = v > hi ? hi : v;
  return v;
}

// Per-thread accumulator of the acceptance sums: FP64 in the FP64 form; in
// the FP32-bulk form each thread sums its few rows in FP32 and the cross-
// thread reduction is FP64 (block_reduce_store / final_reduce).
template <typename T>
struct SumT {
  typedef T type;
};

#define PDNQP_GRID_STRIDE(i, N) \
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (long long)(N); \
       i += (long long)gridDim.x * blockDim.x)
// The same over the blocks of a GridCtx (one problem's share of a batched launch).
#define PDNQP_VGRID_STRIDE(i, N, g) \
  for (long long i = (long long)(g).b * blockDim.x + threadIdx.x; i < (long long)(N); \
       i += (long long)(g).nb * blockDim.x)

// The single-block kernels work on a shared-memory copy of the device state
// (one coalesced load and store) instead of chains of dependent global
// read-modify-writes.
__device__ __forceinline__ void state_load(DevState &S, const DevState *g) {
  for (int i = threadIdx.x; i < (int)(sizeof(DevState) / 4); i += blockDim.x) ((int *)&S)[i] = __ldcg((const int *)g + i);
  __syncthreads();
}
__device__ __forceinline__ void state_store(DevState *g, const DevState &S) {
  __syncthreads();
  for (int i = threadIdx.x; i < (int)(sizeof(DevState) / 4); i += blockDim.x) ((int *)g)[i] = ((const int *)&S)[i];
}

// Start of one graph launch: at most `chunk` trials before control returns to
// the host.
__global__ void k_loop_begin(DevState *st, long long chunk) { st->slot_left = chunk; }

// Last-block detection: after this block's partial sums are stored, returns
// true in the single block that arrives last (its threads then see every
// block's partials); that block resets the counter at the end of its work.
__device__ __forceinline__ bool arrive_last(unsigned *ctr, int nb = -1) {
  __shared__ bool last;
  if (nb < 0) nb = gridDim.x;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ctr, 1u) == (unsigned)(nb - 1);
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// A kernel that finds the loop stopped ends the device loop (block 0 only).
// COND = false builds kernels without conditional-handle calls (for unrolled
// graphs, which profilers can inspect).
template <bool COND>
__device__ __forceinline__ void stop_loop(cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hc) {
  if (COND && blockIdx.x == 0 && threadIdx.x == 0) {
    if (hw) cudaGraphSetConditional(hw, 0u);
    if (hc) cudaGraphSetConditional(hc, 0u);
  }
}

template <bool COND>
__device__ void decide_body(DevState *stg, const double *part, const double *lacc, int nb_r, int nb_c,
                            cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hc);
template <bool COND>
__device__ void check_final_body(DevState *stg, const double *part, int nb_r, int nb_c,
                                 cudaGraphConditionalHandle hw);
__device__ void inner_begin_body(DevState *st, const double *part, int nb_r, int nb_c);
__device__ __forceinline__ void decide_logic(DevState *st, const double (&a)[4], const double (&b)[4]);

// ===========================================================================
// Trial step (Eq. pdqp-trial) and acceptance test (Eq. adaptive-condition).
// ===========================================================================

// Primal x-block of the trial: x_tr = P_[l,u](x - tau (q + (1-alpha) H xbar +
// alpha H x - A'y)) with the cached products H x, H xbar, A'y.
// The phase functions below read the scalar state through `st` (global
// memory in the one-kernel-per-phase launches, a shared-memory copy in the
// persistent loop) and touch the iterate buffers through plain pointers: in
// the persistent loop the same buffers are written and read across grid
// barriers within one launch, so they must not go through the read-only path.
// 16-byte vectors of the streaming passes (every vector is its own
// allocation, so 256-byte aligned): W elements per load or store.
template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  typedef float4 type;
};
template <>
struct Vec16<double> {
  typedef double2 type;
};
template <typename T>
struct Pack {
  static constexpr int W = 16 / sizeof(T);
  T v[W];
  __device__ __forceinline__ void load(const T *p, long long i) {
    *reinterpret_cast<typename Vec16<T>::type *>(v) = reinterpret_cast<const typename Vec16<T>::type *>(p)[i];
  }
  __device__ __forceinline__ void store(T *p, long long i) const {
    reinterpret_cast<typename Vec16<T>::type *>(p)[i] = *reinterpret_cast<const typename Vec16<T>::type *>(v);
  }
};

template <typename T>
__device__ __forceinline__ void primal_phase(const Dev<T> &d, const DevState *st, GridCtx g = hw_grid()) {
  const int cur = st->cur, a0 = st->acur, acc = st->accepted;
  const double t = (double)st->t;
  const T alpha = T(2.0 / (t + 2.0));
  const T oma = T(1) - alpha;
  const T sc = T(st->kappa / st->omega);
  const T ap = T(st->alpha_acc), omap = T(1) - ap;
  const T *x = d.x[cur];
  const T *Hx = d.Hx[cur];
  const T *Aty = d.Aty[cur];
  T *xt = d.x[1 - cur];
  constexpr int W = Pack<T>::W;
  const long long nv = d.n / W;
  // W elements per thread and trip with 16-byte loads and stores; the same
  // arithmetic per element as the scalar tail below.
  PDNQP_VGRID_STRIDE(c, nv, g) {
    Pack<T> X, HX, HB, Q, AT, TA, L, U, XT;
    X.load(x, c);
    HX.load(Hx, c);
    HB.load(d.Hxbar[a0], c);
    Q.load(d.qx, c);
    AT.load(Aty, c);
    TA.load(d.taux, c);
    L.load(d.lx, c);
    U.load(d.ux, c);
    if (acc) {
      // Running averages of the previous acceptance (Algorithm 4), written to
      // the other buffer: wbar <- (1 - alpha) wbar + alpha w.
      Pack<T> XB;
      XB.load(d.xbar[a0], c);
#pragma unroll
      for (int k = 0; k < W; ++k) {
        HB.v[k] = omap * HB.v[k] + ap * HX.v[k];
        XB.v[k] = omap * XB.v[k] + ap * X.v[k];
      }
      HB.store(d.Hxbar[a0 ^ 1], c);
      XB.store(d.xbar[a0 ^ 1], c);
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
      const T g = Q.v[k] + oma * HB.v[k] + alpha * HX.v[k] - AT.v[k];
      XT.v[k] = clampv<T>(X.v[k] - (sc * TA.v[k]) * g, L.v[k], U.v[k]);
    }
    XT.store(xt, c);
  }
  // Tail (n mod W elements).
  const long long tid = (long long)g.b * blockDim.x + threadIdx.x;
  const long long i = nv * W + tid;
  if (i < d.n) {
    const T xi = x[i], hxi = Hx[i];
    T hxb;
    if (acc) {
      hxb = omap * d.Hxbar[a0][i] + ap * hxi;
      d.Hxbar[a0 ^ 1][i] = hxb;
      d.xbar[a0 ^ 1][i] = omap * d.xbar[a0][i] + ap * xi;
    } else {
      hxb = d.Hxbar[a0][i];
    }
    const T g = d.qx[i] + oma * hxb + alpha * hxi - Aty[i];
    xt[i] = clampv<T>(xi - (sc * d.taux[i]) * g, d.lx[i], d.ux[i]);
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_primal(Dev<T> d) {
  if (d.st->status != ST_RUNNING) return;
  primal_phase<T>(d, d.st);
}

// ---------------------------------------------------------------------------
// Dense coupling rows.  Block b of the row pass forms the products of entries
// [b L / nb, (b + 1) L / nb) of the concatenated long rows (L entries in all)
// and stores one partial per long row it touches (FP64, block order fixed);
// the block that arrives last sums, for each long row, the partials of the
// blocks whose range overlaps it, in block order, and applies the row update
// of the trial to those rows.  Deterministic for a given grid size.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long lr_cut(long long L, int b, int nb) { return L * b / nb; }

// Sum of one double per thread, in a fixed order; the result is in thread 0.
__device__ __forceinline__ double block_sum_fixed(double v) {
  __shared__ double ws[kBlock / 32];
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  double a = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < kBlock / 32; ++w) a += ws[w];
  __syncthreads();
  return a;
}

template <typename T>
__device__ __forceinline__ void long_rows_partial(const Dev<T> &d, const T *xt, GridCtx g = hw_grid()) {
  const long long L = d.lr_nnz;
  const int nb = g.nb, b = g.b;
  const long long e0 = lr_cut(L, b, nb), e1 = lr_cut(L, b + 1, nb);
  if (e0 >= e1) return;
  int s = 0;
  while (s + 1 < d.nlr && d.lr_ptr[s + 1] <= e0) ++s;
  for (; s < d.nlr && d.lr_ptr[s] < e1; ++s) {
    const long long a0 = e0 > d.lr_ptr[s] ? e0 : d.lr_ptr[s];
    const long long a1 = e1 < d.lr_ptr[s + 1] ? e1 : d.lr_ptr[s + 1];
    T acc = T(0);
    for (long long k = a0 + threadIdx.x; k < a1; k += kBlock) acc += d.lr_val[k] * __ldcg(xt + d.lr_ci[k]);
    const double v = block_sum_fixed(double(acc));
    if (threadIdx.x == 0) d.lr_part[(long long)s * kMaxBlocks + b] = v;
  }
}

// Row update of one constraint row with (A x_tr)_j = ax: the same arithmetic
// as the row passes below (one thread).
template <typename T>
__device__ __forceinline__ void row_update_one(const Dev<T> &d, const DevState *st, long long j, T ax, T &Lt, T &Le,
                                               T &RH, T &RB) {
  const int cur = st->cur, nx = 1 - cur, a0 = st->acur, acc = st->accepted;
  const double t = (double)st->t;
  const T alpha = T(2.0 / (t + 2.0)), oma = T(1) - alpha;
  const T beta = T(t / (t + 1.0));
  const T sct = T(st->kappa / st->omega), sce = T(st->kappa * st->omega);
  const T ap = T(st->alpha_acc), omap = T(1) - ap;
  const bool ineq = j >= d.mE;
  const T y = d.y[cur][j], r = d.r[cur][j];
  T rb;
  if (acc) {
    rb = omap * d.rbar[a0][j] + ap * r;
    d.rbar[a0 ^ 1][j] = rb;
    d.ybar[a0 ^ 1][j] = omap * d.ybar[a0][j] + ap * y;
    if (ineq) d.sbar[a0 ^ 1][j] = omap * d.sbar[a0][j] + ap * d.s[cur][j];
  } else {
    rb = d.rbar[a0][j];
  }
  const T sig = T(d.sig[j]);
  const T rt = r - (sct * d.taur[j]) * (d.qr[j] + sig * (oma * rb + alpha * r) + y);
  d.r[nx][j] = rt;
  T bwt = ax - rt, ds = T(0);
  if (ineq) {
    const T s0 = d.s[cur][j];
    const T stv = clampv<T>(s0 - (sct * d.taus[j]) * (d.qs[j] + y), d.ls[j], d.us[j]);
    d.s[nx][j] = stv;
    ds = stv - s0;
    Lt += ds * ds * d.itaus[j];
    bwt -= stv;
  }
  const T yt = y + (sce * d.eta[j]) * (d.hp[j] - bwt - beta * (bwt - d.Bw[cur][j]));
  d.Bw[nx][j] = bwt;
  d.y[nx][j] = yt;
  const T dr = rt - r, dyv = yt - y;
  Lt += dr * dr * d.itaur[j];
  Le += dyv * dyv * d.ieta[j];
  RH += fabs(dr * sig * dr);
  RB += fabs(ds * dyv) + fabs(dr * dyv);
}

// Run by one whole block once every block's partials are visible (nb = the
// row pass's grid size).  Warp w takes long rows w, w + 8, ...; the four
// acceptance-sum terms go to lr_acc (warps combined in order).
template <typename T>
__device__ void long_rows_finish(const Dev<T> &d, const DevState *st, int nb) {
  __shared__ double wacc[kBlock / 32][4];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long L = d.lr_nnz;
  T Lt = T(0), Le = T(0), RH = T(0), RB = T(0);
  for (int s = w; s < d.nlr; s += kBlock / 32) {
    const long long p0 = d.lr_ptr[s], p1 = d.lr_ptr[s + 1];
    double a = 0.0;
    for (int b = lane; b < nb; b += 32) {
      const long long e0 = lr_cut(L, b, nb), e1 = lr_cut(L, b + 1, nb);
      if (e0 < e1 && e0 < p1 && e1 > p0) a += __ldcg(d.lr_part + (long long)s * kMaxBlocks + b);
    }
    a = warp_sum(a);
    if (lane == 0) row_update_one<T>(d, st, d.lr_row[s], T(a), Lt, Le, RH, RB);
  }
  if (lane == 0) {
    wacc[w][0] = double(Lt);
    wacc[w][1] = double(Le);
    wacc[w][2] = double(RH);
    wacc[w][3] = double(RB);
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double v = 0.0;
    for (int k = 0; k < kBlock / 32; ++k) v += wacc[k][threadIdx.x];
    d.lr_acc[threadIdx.x] = v;
  }
  __syncthreads();
}

// Constraint rows: (A x_tr)_j, the s/r blocks of the primal trial, B w_tr,
// the dual trial y_tr = y + eta (h - B w_tr - beta (B w_tr - B w)), and the
// row-local terms of the acceptance sums.  Steps are used as
// tau = (kappa / omega) tau0, eta = (kappa omega) eta0; the sums of
// dw^2 / tau and dy^2 / eta are accumulated with the stored inverses 1/tau0,
// 1/eta0 and scaled once by omega / kappa and 1 / (kappa omega).
template <typename T, int G>
__device__ __forceinline__ void rows_phase(const Dev<T> &d, const DevState *st, GridCtx g = hw_grid()) {
  const int cur = st->cur, nx = 1 - cur, a0 = st->acur, acc = st->accepted;
  const double t = (double)st->t;
  const T alpha = T(2.0 / (t + 2.0)), oma = T(1) - alpha;
  const T beta = T(t / (t + 1.0));
  const T sct = T(st->kappa / st->omega), sce = T(st->kappa * st->omega);
  const T ap = T(st->alpha_acc), omap = T(1) - ap;
  const T *xt = d.x[nx];
  T Lt = T(0), Le = T(0), RH = T(0), RB = T(0);
  TileIter ti(g);
  for (long long tile = ti.first; tile < d.m; tile += ti.step) {
    const long long j = tile + ti.lane;
    const bool valid = j < d.m && !(d.nlr && d.lr_flag[j]), ineq = j >= d.mE;
    // Everything that does not need (A x_tr)_j first (the r and s blocks of
    // the trial and the operands of the dual step), so that these loads
    // overlap the SpMV chain.
    T y = T(0), r = T(0), rt = T(0), stv = T(0), ds = T(0), bw = T(0), etj = T(0), hpj = T(0), sig = T(0);
    if (valid) {
      y = d.y[cur][j];
      r = d.r[cur][j];
      T rb;
      if (acc) {  // running averages of the previous acceptance
        rb = omap * d.rbar[a0][j] + ap * r;
        d.rbar[a0 ^ 1][j] = rb;
        d.ybar[a0 ^ 1][j] = omap * d.ybar[a0][j] + ap * y;
        if (ineq) d.sbar[a0 ^ 1][j] = omap * d.sbar[a0][j] + ap * d.s[cur][j];
      } else {
        rb = d.rbar[a0][j];
      }
      sig = T(d.sig[j]);
      rt = r - (sct * d.taur[j]) * (d.qr[j] + sig * (oma * rb + alpha * r) + y);
      d.r[nx][j] = rt;
      if (ineq) {
        const T s = d.s[cur][j];
        stv = clampv<T>(s - (sct * d.taus[j]) * (d.qs[j] + y), d.ls[j], d.us[j]);
        d.s[nx][j] = stv;
        ds = stv - s;
        Lt += ds * ds * d.itaus[j];
      }
      bw = d.Bw[cur][j];
      etj = d.eta[j];
      hpj = d.hp[j];
    }
    const T ax = tile_row_sum<G, T>(d.As.rp, d.As.ci, d.As.val, tile, d.m, [&](int k, T a) { return a * __ldcg(xt + k); });
    if (valid) {
      T bwt = ax - rt;
      if (ineq) bwt -= stv;
      const T yt = y + (sce * etj) * (hpj - bwt - beta * (bwt - bw));
      d.Bw[nx][j] = bwt;
      d.y[nx][j] = yt;
      const T dr = rt - r, dyv = yt - y;
      Lt += dr * dr * d.itaur[j];
      Le += dyv * dyv * d.ieta[j];
      RH += fabs(dr * sig * dr);
      RB += fabs(ds * dyv) + fabs(dr * dyv);
    }
  }
  double v[4] = {double(Lt), double(Le), double(RH), double(RB)};
  block_reduce_store<4>(v, 0u, d.part + P_TR_R * kMaxBlocks, g.b);
}

// Row pass of one trial over the blocks of g (graph and batched forms).
template <typename T, int G>
__device__ __forceinline__ void rows_trial_body(const Dev<T> &d, GridCtx g) {
  if (d.st->status != ST_RUNNING) return;
  if (d.nlr) long_rows_partial<T>(d, d.x[1 - d.st->cur], g);
  rows_phase<T, G>(d, d.st, g);
  if (d.nlr && arrive_last(d.ctr + 2, g.nb)) {
    long_rows_finish<T>(d, d.st, g.nb);
    if (threadIdx.x == 0) d.ctr[2] = 0u;
  }
}

template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_rows(Dev<T> d) {
  rows_trial_body<T, G>(d, hw_grid());
}

// Variable rows: (H x_tr)_i and (A' y_tr)_i (the products with Q and A^T),
// plus the x terms of the acceptance sums.
template <typename T, int GH, int GT>
__device__ __forceinline__ void cols_phase(const Dev<T> &d, const DevState *st, GridCtx g = hw_grid()) {
  const int cur = st->cur, nx = 1 - cur;
  const T *xt = d.x[nx];
  const T *yt = d.y[nx];
  T Lt = T(0), RH = T(0), RB = T(0);
  TileIter ti(g);
  for (long long tile = ti.first; tile < d.n; tile += ti.step) {
    const long long i = tile + ti.lane;
    // Row-local operands first: their loads overlap the SpMV chains.
    T xti = T(0), xci = T(0), hxc = T(0), atc = T(0), itx = T(0);
    if (i < d.n) {
      xti = xt[i];
      xci = d.x[cur][i];
      hxc = d.Hx[cur][i];
      atc = d.Aty[cur][i];
      itx = d.itaux[i];
    }
    T hx, aty;
    tile_pair_sum<GH, GT, T>(
        d.H.rp, d.H.ci, d.H.val, d.At.rp, d.At.ci, d.At.val, tile, d.n,
        [&](int k, T a) { return a * __ldcg(xt + k); }, [&](int k, T a) { return a * __ldcg(yt + k); }, hx, aty);
    if (i < d.n) {
      d.Hx[nx][i] = hx;
      d.Aty[nx][i] = aty;
      const T dx = xti - xci;
      const T dh = hx - hxc;
      const T da = aty - atc;
      Lt += dx * dx * itx;
      RH += fabs(dx * dh);
      RB += fabs(dx * da);
    }
  }
  double v[4] = {double(Lt), 0.0, double(RH), double(RB)};
  block_reduce_store<4>(v, 0u, d.part + P_TR_C * kMaxBlocks, g.b);
}

// Column pass of one trial over the blocks of g, with the acceptance decision
// in the problem's last block (graph and batched forms).
template <typename T, int G, bool COND>
__device__ __forceinline__ void cols_trial_body(const Dev<T> &d, int nb_r, GridCtx g) {
  if (d.st->status != ST_RUNNING) {
    stop_loop<COND>(d.hw, d.hc);
    return;
  }
  cols_phase<T, G, G>(d, d.st, g);
  if (arrive_last(d.ctr, g.nb)) {
    decide_body<COND>(d.st, d.part, d.nlr ? d.lr_acc : nullptr, nb_r, g.nb, d.hw, d.hc);
    if (threadIdx.x == 0) d.ctr[0] = 0u;
  }
}

template <typename T, int G, bool COND>
__global__ void __launch_bounds__(kBlock) k_cols(Dev<T> d, int nb_r) {
  cols_trial_body<T, G, COND>(d, nb_r, hw_grid());
}

// ===========================================================================
// Panel stream of the persistent loop.  The rows of one or two CSR matrices
// with the same row set are cut into panels of kBlock rows; each block takes
// panels blockIdx.x, blockIdx.x + gridDim.x, ...  For each panel one thread
// issues bulk copies of the panel's column-index and value ranges (rounded
// to 16 bytes) into one of two shared-memory stages while the block works on
// the other stage, so the matrix stream runs ahead of the arithmetic instead
// of behind a chain of dependent loads.  In a stage, the block first forms
// the products a_k x[col_k] over the panel's entries (coalesced, many
// independent gathers per thread, written in place of the values), then
// thread t sums the products of row panel + t in entry order.  A panel whose
// entries do not fit a stage is read directly from global memory (same
// order).  Per row: pre(r, valid) runs before the wait (its loads overlap the
// copies) and returns a context; post(r, valid, ctx, sums) runs after.
// ===========================================================================
constexpr int kStageEntries = 3072;  // entries (index + value) per stage, all matrices of a panel
template <typename T>
constexpr unsigned stage_bytes() {
  return kStageEntries * (4u + (unsigned)sizeof(T));
}
// Dynamic shared memory of the persistent loop: two stages.  (Shared memory
// taken here is L1 capacity lost to the in-flight loads of every pass, so
// the products are formed in place.)
template <typename T>
constexpr unsigned stream_smem_bytes() {
  return 2 * stage_bytes<T>();
}

struct StreamCtl {
  unsigned long long bar[2];
  int done[2];     // per stage: warps finished with the panel in it
  int base[2][2];  // per stage and matrix: first entry copied (multiple of 4)
  int cnt[2][2];   // entries copied (multiple of 4)
  int off[2][2];   // byte offset of the index array in the stage (values follow)
  int fits[2];
};

__device__ __forceinline__ void stream_init(StreamCtl &ctl) {
  if (threadIdx.x == 0) {
    mbar_init(&ctl.bar[0], 1);
    mbar_init(&ctl.bar[1], 1);
    mbar_init_fence();
  }
  __syncthreads();
}

// Row bounds of panel p (thread 0 loads them one panel ahead of the issue).
template <typename T, int NM>
__device__ __forceinline__ void panel_bounds(const Mat<T> *M, long long p, long long nrows, int *lo, int *hi) {
  const long long r0 = p * kBlock;
  const long long r1 = r0 + kBlock < nrows ? r0 + kBlock : nrows;
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    lo[m] = M[m].rp[r0];
    hi[m] = M[m].rp[r1];
  }
}

template <typename T, int NM>
__device__ __forceinline__ void stream_issue(StreamCtl &ctl, unsigned char *buf, int st, const Mat<T> *M,
                                             const int *lo, const int *hi) {
  unsigned total = 0;
  int a[NM], c[NM], o[NM];
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    a[m] = lo[m] & ~3;
    c[m] = ((hi[m] + 3) & ~3) - a[m];
    o[m] = (int)total;
    total += (unsigned)c[m] * (4u + (unsigned)sizeof(T));
  }
  const int fits = total <= stage_bytes<T>() ? 1 : 0;
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    ctl.base[st][m] = a[m];
    ctl.cnt[st][m] = c[m];
    ctl.off[st][m] = o[m];
  }
  ctl.fits[st] = fits;
  unsigned char *dst = buf + (size_t)st * stage_bytes<T>();
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(&ctl.bar[st], fits ? total : 0u);
  if (fits) {
    const unsigned long long pol = l2_evict_first_policy();
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      if (c[m] > 0) {
        bulk_g2s_hint(dst + o[m], M[m].ci + a[m], (unsigned)c[m] * 4u, &ctl.bar[st], pol);
        bulk_g2s_hint(dst + o[m] + 4 * c[m], M[m].val + a[m], (unsigned)c[m] * (unsigned)sizeof(T), &ctl.bar[st], pol);
      }
    }
  }
}

// Warps work through the panels independently: warp w owns rows 32w..32w+31
// of every panel, waits for the panel's copy on the stage's mbarrier, forms
// the products of its own entry ranges (contiguous slices of the stage) and
// the row sums, and reports on the stage's counter; the last warp to finish
// with a stage refills it with the panel two ahead.  Per panel a warp makes a
// single round of dependent memory accesses: load(r) issues the row-local
// loads before the wait, the gathers of all matrices go out in one batch,
// and finish(r, raw, sums) does all the arithmetic and the stores at the end.
// The only block-wide barriers are at the start and end of the pass.  On a
// fault (a copy that never lands) the warps run out the loop without
// touching the stages, the copies in flight get a bounded wait, and the pass
// returns false.
template <typename T, int NM, int GB, typename Load, typename Finish>
__device__ __forceinline__ bool stream_panels(StreamCtl &ctl, unsigned char *buf, unsigned &ph, unsigned *fault,
                                              const Mat<T> *M, const T *const *gx, long long nrows, Load load,
                                              Finish finish) {
  constexpr int kWarps = kBlock / 32;
  const long long np = (nrows + kBlock - 1) / kBlock;
  const long long p0 = blockIdx.x, nb = gridDim.x;
  if (p0 >= np) return true;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    ctl.done[0] = 0;
    ctl.done[1] = 0;
    int lo[NM], hi[NM];
    panel_bounds<T, NM>(M, p0, nrows, lo, hi);
    stream_issue<T, NM>(ctl, buf, 0, M, lo, hi);
    if (p0 + nb < np) {
      panel_bounds<T, NM>(M, p0 + nb, nrows, lo, hi);
      stream_issue<T, NM>(ctl, buf, 1, M, lo, hi);
    }
  }
  __syncthreads();
  bool ok = true;
  for (long long k = 0, p = p0; p < np; ++k, p += nb) {
    const int st = (int)(k & 1);
    const long long r = p * kBlock + threadIdx.x;
    const bool valid = r < nrows;
    int rb[NM], re[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      rb[m] = valid ? M[m].rp[r] : 0;
      re[m] = valid ? M[m].rp[r + 1] : 0;
    }
    const auto raw = load(r, valid);
    // This warp's rows: [rw, rw + 32) clipped to nrows.
    const long long rw = p * kBlock + 32 * w;
    const int last = rw < nrows ? (int)((nrows - 1 - rw) < 31 ? (nrows - 1 - rw) : 31) : -1;
    T sum[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) sum[m] = T(0);
    if (ok) ok = mbar_wait_warp(&ctl.bar[st], (ph >> st) & 1u, fault);
    ph ^= 1u << st;
    if (ok && last >= 0) {
      if (ctl.fits[st]) {
        unsigned char *sb = buf + (size_t)st * stage_bytes<T>();
        int wb[NM], we[NM], b0[NM];
        const int *sci[NM];
        T *sv[NM];
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          const int cnt = ctl.cnt[st][m];
          b0[m] = ctl.base[st][m];
          sci[m] = reinterpret_cast<const int *>(sb + ctl.off[st][m]);
          sv[m] = reinterpret_cast<T *>(sb + ctl.off[st][m] + 4 * cnt);
          // The warp's entries [wb, we) (rows of invalid lanes are empty).
          wb[m] = __shfl_sync(0xffffffffu, rb[m], 0) - b0[m];
          we[m] = __shfl_sync(0xffffffffu, re[m], last) - b0[m];
        }
        // Products in batches of GB entries per lane and matrix: all index
        // and value reads and all gathers of a batch (every matrix) are
        // issued before its stores.
        for (int j0 = lane;; j0 += GB * 32) {
          bool more = false;
#pragma unroll
          for (int m = 0; m < NM; ++m) more |= wb[m] + j0 < we[m];
          if (!__any_sync(0xffffffffu, more)) break;
          int ci[NM][GB];
          T a[NM][GB], xg[NM][GB];
#pragma unroll
          for (int m = 0; m < NM; ++m)
#pragma unroll
            for (int u = 0; u < GB; ++u) {
              const int e = wb[m] + j0 + u * 32;
              ci[m][u] = e < we[m] ? sci[m][e] : 0;
              a[m][u] = e < we[m] ? sv[m][e] : T(0);
            }
#pragma unroll
          for (int m = 0; m < NM; ++m)
#pragma unroll
            for (int u = 0; u < GB; ++u) xg[m][u] = __ldcg(gx[m] + ci[m][u]);
#pragma unroll
          for (int m = 0; m < NM; ++m)
#pragma unroll
            for (int u = 0; u < GB; ++u) {
              const int e = wb[m] + j0 + u * 32;
              if (e < we[m]) sv[m][e] = a[m][u] * xg[m][u];
            }
        }
        __syncwarp();
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          T a = T(0);
          for (int k2 = rb[m]; k2 < re[m]; ++k2) a += sv[m][k2 - b0[m]];
          sum[m] = a;
        }
      } else {
        // The panel does not fit a stage: read it from global memory.  Rows of
        // at most kLongRow entries are summed by their own lane in entry order;
        // longer rows (dense coupling rows) by the whole warp, lane-strided,
        // then a fixed butterfly (deterministic).
        constexpr int kLongRow = 64;
#pragma unroll
        for (int m = 0; m < NM; ++m) {
          const bool lng = valid && re[m] - rb[m] > kLongRow;
          T a = T(0);
          if (!lng)
            for (int k2 = rb[m]; k2 < re[m]; ++k2) a += M[m].val[k2] * __ldcg(gx[m] + M[m].ci[k2]);
          unsigned todo = __ballot_sync(0xffffffffu, lng);
          while (todo) {
            const int l = __ffs(todo) - 1;
            todo &= todo - 1;
            const int b = __shfl_sync(0xffffffffu, rb[m], l), e = __shfl_sync(0xffffffffu, re[m], l);
            T w = T(0);
            for (int k2 = b + lane; k2 < e; k2 += 32) w += M[m].val[k2] * __ldcg(gx[m] + M[m].ci[k2]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
            if (lane == l) a = w;
          }
          sum[m] = a;
        }
      }
    }
    // Done with the stage: the last warp refills it with the panel two ahead.
    // The fences on both sides of the counter order every warp's reads and
    // in-place writes of the stage before the refill's copy.
    __syncwarp();
    bool refill = false;
    if (ok && lane == 0) {
      __threadfence_block();
      refill = atomicAdd(&ctl.done[st], 1) == kWarps - 1;
    }
    if (refill) {
      __threadfence_block();
      ctl.done[st] = 0;
      const long long p2 = p + 2 * nb;
      if (p2 < np) {
        int lo[NM], hi[NM];
        panel_bounds<T, NM>(M, p2, nrows, lo, hi);
        stream_issue<T, NM>(ctl, buf, st, M, lo, hi);
      }
    }
    finish(r, valid, raw, sum);
  }
  __syncthreads();
  if (!ok && threadIdx.x == 0) {
    // Bounded wait for copies that may still be in flight.
    for (int s2 = 0; s2 < 2; ++s2)
      for (unsigned it = 0; it <= kSpinLimitTx && !mbar_test(&ctl.bar[s2], (ph >> s2) & 1u); ++it) __nanosleep(32);
  }
  __syncthreads();
  return ok;
}

// Row pass of the persistent loop: the per-row arithmetic of rows_phase with
// (A x_tr) from the panel stream.
template <typename T, bool LR>
__device__ __forceinline__ bool rows_phase_stream(const Dev<T> &d, const DevState *st, StreamCtl &ctl,
                                                  unsigned char *buf, unsigned &ph, unsigned *fault) {
  const int cur = st->cur, nx = 1 - cur, a0 = st->acur, acc = st->accepted;
  const double t = (double)st->t;
  const T alpha = T(2.0 / (t + 2.0)), oma = T(1) - alpha;
  const T beta = T(t / (t + 1.0));
  const T sct = T(st->kappa / st->omega), sce = T(st->kappa * st->omega);
  const T ap = T(st->alpha_acc), omap = T(1) - ap;
  T Lt = T(0), Le = T(0), RH = T(0), RB = T(0);
  struct Raw {
    T y, r, rb, yb, tr, qr, bw, eta, hp, itr, ie, s, sb, ts, qs, ls, us, its;
    double sig;
  };
  if (LR) long_rows_partial<T>(d, d.x[nx]);
  const Mat<T> M[1] = {d.As};
  const T *gx[1] = {d.x[nx]};
  const bool ok = stream_panels<T, 1, 8>(
      ctl, buf, ph, fault, M, gx, d.m,
      [&](long long j, bool valid) {
        Raw c;
        memset(&c, 0, sizeof(c));
        if (valid) {
          c.y = d.y[cur][j];
          c.r = d.r[cur][j];
          c.rb = d.rbar[a0][j];
          if (acc) c.yb = d.ybar[a0][j];
          c.sig = d.sig[j];
          c.tr = d.taur[j];
          c.qr = d.qr[j];
          c.bw = d.Bw[cur][j];
          c.eta = d.eta[j];
          c.hp = d.hp[j];
          c.itr = d.itaur[j];
          c.ie = d.ieta[j];
          if (j >= d.mE) {
            c.s = d.s[cur][j];
            if (acc) c.sb = d.sbar[a0][j];
            c.ts = d.taus[j];
            c.qs = d.qs[j];
            c.ls = d.ls[j];
            c.us = d.us[j];
            c.its = d.itaus[j];
          }
        }
        return c;
      },
      [&](long long j, bool valid, const Raw &c, const T *sum) {
        if (!valid || (LR && d.lr_flag[j])) return;
        const bool ineq = j >= d.mE;
        T rb = c.rb;
        if (acc) {  // running averages of the previous acceptance
          rb = omap * rb + ap * c.r;
          d.rbar[a0 ^ 1][j] = rb;
          d.ybar[a0 ^ 1][j] = omap * c.yb + ap * c.y;
          if (ineq) d.sbar[a0 ^ 1][j] = omap * c.sb + ap * c.s;
        }
        const T sig = T(c.sig);
        const T rt = c.r - (sct * c.tr) * (c.qr + sig * (oma * rb + alpha * c.r) + c.y);
        d.r[nx][j] = rt;
        T bwt = sum[0] - rt, ds = T(0);
        if (ineq) {
          const T stv = clampv<T>(c.s - (sct * c.ts) * (c.qs + c.y), c.ls, c.us);
          d.s[nx][j] = stv;
          ds = stv - c.s;
          Lt += ds * ds * c.its;
          bwt -= stv;
        }
        const T yt = c.y + (sce * c.eta) * (c.hp - bwt - beta * (bwt - c.bw));
        d.Bw[nx][j] = bwt;
        d.y[nx][j] = yt;
        const T dr = rt - c.r, dyv = yt - c.y;
        Lt += dr * dr * c.itr;
        Le += dyv * dyv * c.ie;
        RH += fabs(dr * sig * dr);
        RB += fabs(ds * dyv) + fabs(dr * dyv);
      });
  double v[4] = {double(Lt), double(Le), double(RH), double(RB)};
  block_reduce_store<4>(v, 0u, d.part + P_TR_R * kMaxBlocks);
  return ok;
}

// Column pass of the persistent loop: H x_tr and A' y_tr from the panel
// stream (both matrices in the same panel), then the per-variable terms.
template <typename T>
__device__ __forceinline__ bool cols_phase_stream(const Dev<T> &d, const DevState *st, StreamCtl &ctl,
                                                  unsigned char *buf, unsigned &ph, unsigned *fault) {
  const int cur = st->cur, nx = 1 - cur;
  T Lt = T(0), RH = T(0), RB = T(0);
  struct Raw {
    T xti, xci, hxc, atc, itx;
  };
  const Mat<T> M[2] = {d.H, d.At};
  const T *gx[2] = {d.x[nx], d.y[nx]};
  const bool ok = stream_panels<T, 2, 6>(
      ctl, buf, ph, fault, M, gx, d.n,
      [&](long long i, bool valid) {
        Raw c = {T(0), T(0), T(0), T(0), T(0)};
        if (valid) {
          c.xti = d.x[nx][i];
          c.xci = d.x[cur][i];
          c.hxc = d.Hx[cur][i];
          c.atc = d.Aty[cur][i];
          c.itx = d.itaux[i];
        }
        return c;
      },
      [&](long long i, bool valid, const Raw &c, const T *sum) {
        if (!valid) return;
        d.Hx[nx][i] = sum[0];
        d.Aty[nx][i] = sum[1];
        const T dx = c.xti - c.xci;
        const T dh = sum[0] - c.hxc;
        const T da = sum[1] - c.atc;
        Lt += dx * dx * c.itx;
        RH += fabs(dx * dh);
        RB += fabs(dx * da);
      });
  double v[4] = {double(Lt), 0.0, double(RH), double(RB)};
  block_reduce_store<4>(v, 0u, d.part + P_TR_C * kMaxBlocks);
  return ok;
}

// Persistent trial loop (one cooperative launch): primal, rows and columns of
// each trial are separated by grid barriers, and the last block to reach the
// third barrier takes the acceptance decision (decide_body) before releasing
// the others, which then reload the scalar state.  The loop leaves when the
// solve stops, a periodic check is due (the check kernels follow this launch)
// or the launch's trial allowance (slot_left) is used up; it does not start
// while a check is pending (the check kernels clear check_due).  All blocks
// take the same branches (the state is block-uniform), so every barrier is
// reached by every block.  Partial sums use this grid's size for both passes.
// LR: the instance has dense coupling rows (d.nlr > 0); a separate
// instantiation keeps their branches out of the common case.
template <typename T, bool LR>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 3 : 2) k_trials(Dev<T> d) {
  __shared__ DevState S;
  __shared__ StreamCtl ctl;
  extern __shared__ __align__(128) unsigned char stage_buf[];
  unsigned *bar = d.ctr + kCtrBar;
  unsigned *fault = bar + kBarFault;
  unsigned ph = 0u;  // parity of the next wait on each stage
  stream_init(ctl);
  state_load(S, d.st);
  const int nb = gridDim.x;
  // Block 0 times each pass: its own work, then its wait at the barrier
  // (imbalance across blocks plus the barrier itself; the last one includes
  // the acceptance decision).
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned long long tp[6] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
  unsigned long long tk = timer ? global_ns() : 0ull;
  auto lap = [&](int k) {
    if (timer) {
      const unsigned long long t = global_ns();
      tp[k] += t - tk;
      tk = t;
    }
  };
  while (S.status == ST_RUNNING && S.slot_left > 0 && !S.check_due) {
    primal_phase<T>(d, &S);
    lap(0);
    if (!grid_sync(bar)) return;
    lap(1);
    if (!rows_phase_stream<T, LR>(d, &S, ctl, stage_buf, ph, fault)) return;
    lap(2);
    if (!grid_sync(bar, [&] {
          if (LR) long_rows_finish<T>(d, &S, nb);
        }))
      return;
    lap(3);
    if (!cols_phase_stream<T>(d, &S, ctl, stage_buf, ph, fault)) return;
    lap(4);
    if (!grid_sync(bar, [&] { decide_body<false>(d.st, d.part, LR ? d.lr_acc : nullptr, nb, nb, 0, 0); })) return;
    state_load(S, d.st);
    lap(5);
  }
  if (timer && d.ptime)
    for (int k = 0; k < 6; ++k) d.ptime[k] += tp[k];
}

// Acceptance decision (single block, deterministic order).  On acceptance the
// trial buffers become current (index flip); on rejection both step vectors
// are shrunk through kappa.

// Acceptance decision (Eq. adaptive-condition), run by the last block of the
// column kernel once every block's partial sums are visible: FP64 sums in a
// fixed order; on acceptance the trial buffers become current (index flip), on
// rejection both step vectors shrink through kappa.  Sets the device-loop
// handles: hw (continue while running and the launch has trials left) and hc
// (a periodic check follows).
// The scalar part of the acceptance decision (one thread), from the row (a)
// and column (b) sums of the trial.
__device__ __forceinline__ void decide_logic(DevState *st, const double (&a)[4], const double (&b)[4]) {
  // Commit the averages materialised by this trial's primal / row passes.
  st->acur ^= st->accepted;
  st->accepted = 0;
  st->restart_flag = 0;
  st->check_due = 0;
  st->trials += 1;
  const double om = st->omega, ka = st->kappa;
  const double lhs = (om / ka) * (a[0] + b[0]) + (a[1] + b[1]) / (ka * om);
  const double rh = a[2] + b[2], rb = a[3] + b[3];
  if (!isfinite(lhs) || !isfinite(rh) || !isfinite(rb)) {
    st->status = ST_NUMERICAL_ERROR;
  } else if (0.5 * lhs >= 0.5 * rh + rb) {
    st->alpha_acc = 2.0 / ((double)st->t + 2.0);
    st->cur ^= 1;
    st->accepted = 1;
    st->t += 1;
    st->t_total += 1;
    st->accepted_all += 1;
    st->rej = 0;
    const bool due = (st->k_chk > 0 && st->t_total % st->k_chk == 0) || st->t_total == st->k_in;
    st->check_due = due ? 1 : 0;
    if (!due && st->t_total == st->pause_at) st->status = ST_PAUSED;
  } else {
    st->kappa *= st->shrink;
    st->rej += 1;
    if (st->rej >= st->rej_limit) st->status = ST_NUMERICAL_ERROR;
  }
  st->slot_left -= 1;
}

template <bool COND>
__device__ void decide_body(DevState *stg, const double *part, const double *lacc, int nb_r, int nb_c,
                            cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hc) {
  __shared__ DevState S;
  state_load(S, stg);
  double a[4], b[4];
  if (nb_r == nb_c) {
    // Row and column partials of one grid (rows 0-3 and 4-7): one pass.
    double ab[8];
    final_reduce<8>(part + P_TR_R * kMaxBlocks, nb_r, 0u, ab);
    for (int k = 0; k < 4; ++k) {
      a[k] = ab[k];
      b[k] = ab[4 + k];
    }
  } else {
    final_reduce<4>(part + P_TR_R * kMaxBlocks, nb_r, 0u, a);
    final_reduce<4>(part + P_TR_C * kMaxBlocks, nb_c, 0u, b);
  }
  if (lacc)
    for (int k = 0; k < 4; ++k) a[k] += __ldcg(lacc + k);
  if (threadIdx.x == 0) {
    decide_logic(&S, a, b);
    if (COND) {
      const bool run = S.status == ST_RUNNING;
      if (hw) cudaGraphSetConditional(hw, (run && S.slot_left > 0) ? 1u : 0u);
      if (hc) cudaGraphSetConditional(hc, (run && S.check_due) ? 1u : 0u);
    }
  }
  state_store(stg, S);
}

// Materialises the running averages of a pending acceptance: bar[acur^1] =
// (1 - alpha) bar[acur] + alpha w (Algorithm 4, "update the weighted
// averages") for x, H x, s, r, y.  The trial kernels do this lazily; this
// kernel is only used before the host reads a paused state.  Reads and writes
// different buffers, so a repeated launch is harmless.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_average(Dev<T> d) {
  const DevState *st = d.st;
  if (!st->accepted) return;
  const int cur = st->cur, a0 = st->acur, a1 = st->acur ^ 1;
  const T alpha = T(st->alpha_acc), oma = T(1) - alpha;
  PDNQP_GRID_STRIDE(i, d.n) {
    d.xbar[a1][i] = oma * d.xbar[a0][i] + alpha * d.x[cur][i];
    d.Hxbar[a1][i] = oma * d.Hxbar[a0][i] + alpha * d.Hx[cur][i];
  }
  PDNQP_GRID_STRIDE(j, d.m) {
    d.ybar[a1][j] = oma * d.ybar[a0][j] + alpha * d.y[cur][j];
    d.rbar[a1][j] = oma * d.rbar[a0][j] + alpha * d.r[cur][j];
    if (j >= d.mE) d.sbar[a1][j] = oma * d.sbar[a0][j] + alpha * d.s[cur][j];
  }
}

// ===========================================================================
// Periodic check (Sec. 3.3.3 inner termination; restart criteria and the
// primal weight, Eqs. primal-weight-movement / primal-weight-update).
// Per candidate (c = current, a = average) 8 quantities:
//   0 r_p (max), 1 s_p (max), 2 r_d (max), 3 s_d (max),
//   4 sum (d (Bw - h))^2, 5 sum ((w - P(w - e^2 g)) / e)^2,
//   6 sum ((w - w_start) / e)^2, 7 sum ((y - y_start) / d)^2
// stored as [c0..c7, a0..a7].  mode 1 = only the current point's 4 and 5
// (restart metric of the inner start).
// ===========================================================================
// Contributions of one row (its s and r components and its dual) to the 8
// quantities of one candidate, in FP64.  Inputs are corrections (bwd = B dw,
// ds, dr, dy, epoch-start corrections) plus the base data of the row.
struct RowIn {
  bool ineq;
  double bwd, hp, bwb, h;        // B dw, h - B w_b, B w_b, h
  double ds, dr, dyv;            // corrections
  double qs, qr, sig, lam;       // base gradients (s, r blocks), penalty, multiplier
  double rb, yb;                 // base r and y
  double ls, us;                 // shifted slack bounds
  double es, er, dsc;            // column scales of s, r and the row scale
  double sst, rst, yst;          // epoch-start corrections
};

__device__ __forceinline__ void row_cand(double *q, const RowIn &a) {
  const double e_bh = a.bwd - a.hp;  // (B w - h)_j
  q[0] = fmax(q[0], fabs(e_bh));
  q[1] = fmax(q[1], fmax(fabs(a.bwb + a.bwd), fabs(a.h)));
  const double gr = a.qr + a.sig * a.dr + a.dyv;  // sigma r + lambda + y at the point
  q[2] = fmax(q[2], fabs(gr));
  q[3] = fmax(q[3], fmax(fabs(a.sig * (a.rb + a.dr)), fmax(fabs(a.lam), fabs(a.yb + a.dyv))));
  q[4] += (a.dsc * e_bh) * (a.dsc * e_bh);
  q[5] += (a.er * gr) * (a.er * gr);
  const double wr = (a.dr - a.rst) / a.er;
  q[6] += wr * wr;
  const double wy = (a.dyv - a.yst) / a.dsc;
  q[7] += wy * wy;
  if (a.ineq) {
    const double gs = a.qs + a.dyv;  // y at the point
    double p = a.ds - gs;
    p = p < a.ls ? a.ls : p;
    p = p > a.us ? a.us : p;
    q[2] = fmax(q[2], fabs(a.ds - p));
    double p2 = a.ds - a.es * a.es * gs;
    p2 = p2 < a.ls ? a.ls : p2;
    p2 = p2 > a.us ? a.us : p2;
    const double ks = (a.ds - p2) / a.es;
    q[5] += ks * ks;
    const double ws = (a.ds - a.sst) / a.es;
    q[6] += ws * ws;
  }
}

template <typename T, int G>
__device__ __forceinline__ void check_rows_body(const Dev<T> &d, int mode, GridCtx g) {
  const DevState *st = d.st;
  if (mode == 0 && !(st->status == ST_RUNNING && st->check_due)) return;
  // Averages of a pending acceptance are formed on the fly (and written for the
  // row blocks); x bar is gathered as (1 - alpha) xbar + alpha x.
  const int cur = st->cur, a0 = st->acur, acc = st->accepted, ab = a0 ^ acc;
  const T ap = T(st->alpha_acc), omap = T(1) - ap;
  const T *__restrict__ xb0 = d.xbar[a0];
  const T *__restrict__ xc = d.x[cur];
  double q[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) q[k] = 0.0;
  TileIter ti(g);
  for (long long tile = ti.first; tile < d.m; tile += ti.step) {
    T axb = T(0);
    if (mode == 0)
      axb = tile_row_sum<G, T>(d.A.rp, d.A.ci, d.A.val, tile, d.m, [&](int k, T a) {
        return a * (acc ? omap * xb0[k] + ap * xc[k] : xb0[k]);
      });
    const long long j = tile + ti.lane;
    if (j < d.m) {
      const bool ineq = j >= d.mE;
      RowIn a;
      a.ineq = ineq;
      a.hp = double(d.hp[j]);
      a.bwb = double(d.Bwb[j]);
      a.h = double(d.h[j]);
      a.qs = ineq ? double(d.qs[j]) : 0.0;
      a.qr = double(d.qr[j]);
      a.sig = d.sig[j];
      a.lam = d.lam[j];
      a.rb = d.rb[j];
      a.yb = d.yb[j];
      a.ls = ineq ? double(d.ls[j]) : 0.0;
      a.us = ineq ? double(d.us[j]) : 0.0;
      a.es = ineq ? double(d.es[j]) : 1.0;
      a.er = double(d.er[j]);
      a.dsc = double(d.dy[j]);
      a.sst = ineq ? double(d.sst[j]) : 0.0;
      a.rst = double(d.rst[j]);
      a.yst = double(d.yst[j]);
      a.bwd = double(d.Bw[cur][j]);
      a.ds = ineq ? double(d.s[cur][j]) : 0.0;
      a.dr = double(d.r[cur][j]);
      a.dyv = double(d.y[cur][j]);
      row_cand(q, a);
      if (mode == 0) {
        T sa = ineq ? d.sbar[a0][j] : T(0), ra = d.rbar[a0][j], ya = d.ybar[a0][j];
        if (acc) {
          ra = omap * ra + ap * d.r[cur][j];
          ya = omap * ya + ap * d.y[cur][j];
          d.rbar[ab][j] = ra;
          d.ybar[ab][j] = ya;
          if (ineq) {
            sa = omap * sa + ap * d.s[cur][j];
            d.sbar[ab][j] = sa;
          }
        }
        const T bwa = axb - sa - ra;
        d.Bwbar[j] = bwa;
        a.bwd = double(bwa);
        a.ds = double(sa);
        a.dr = double(ra);
        a.dyv = double(ya);
        row_cand(q + 8, a);
      }
    }
  }
  block_reduce_store<16>(q, CK_MAXMASK, d.part + P_CK_R * kMaxBlocks, g.b);
}

template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_check_rows(Dev<T> d, int mode) {
  check_rows_body<T, G>(d, mode, hw_grid());
}

// Contributions of one variable (x block) to the 8 quantities of a candidate:
// dx, H dx, A' dy corrections plus the base data of the variable.
__device__ __forceinline__ void col_cand(double *q, double dx, double hdx, double atdy, double qx, double qx0,
                                         double hxb, double atyb, double lx, double ux, double ex, double xst) {
  const double g = hdx + qx - atdy;  // gradient of the inner Lagrangian at the point
  double p = dx - g;
  p = p < lx ? lx : p;
  p = p > ux ? ux : p;
  q[2] = fmax(q[2], fabs(dx - p));
  q[3] = fmax(q[3], fmax(fabs(hxb + hdx), fmax(fabs(qx0), fabs(atyb + atdy))));
  double p2 = dx - ex * ex * g;
  p2 = p2 < lx ? lx : p2;
  p2 = p2 > ux ? ux : p2;
  const double k = (dx - p2) / ex;
  q[5] += k * k;
  const double w = (dx - xst) / ex;
  q[6] += w * w;
}

template <typename T, int G, bool COND>
__device__ __forceinline__ void check_cols_body(const Dev<T> &d, int mode, int nb_r, GridCtx g) {
  const DevState *st = d.st;
  if (mode == 0 && !(st->status == ST_RUNNING && st->check_due)) return;
  // y bar of a pending acceptance was materialised by k_check_rows.
  const int cur = st->cur, a0 = st->acur, acc = st->accepted, ab = a0 ^ acc;
  const T ap = T(st->alpha_acc), omap = T(1) - ap;
  const T *__restrict__ yb = d.ybar[ab];
  double q[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) q[k] = 0.0;
  TileIter ti(g);
  for (long long tile = ti.first; tile < d.n; tile += ti.step) {
    T atyb = T(0);
    if (mode == 0)
      atyb = tile_row_sum<G, T>(d.At.rp, d.At.ci, d.At.val, tile, d.n, [&](int k, T a) { return a * yb[k]; });
    const long long i = tile + ti.lane;
    if (i < d.n) {
      const double qx = double(d.qx[i]), qx0 = double(d.qx0[i]), hxb = double(d.Hxb[i]);
      const double atyb0 = double(d.Atyb[i]), lx = double(d.lx[i]), ux = double(d.ux[i]);
      const double ex = double(d.ex[i]), xst = double(d.xst[i]);
      col_cand(q, double(d.x[cur][i]), double(d.Hx[cur][i]), double(d.Aty[cur][i]), qx, qx0, hxb, atyb0, lx, ux, ex,
               xst);
      if (mode == 0) {
        d.Atybar[i] = atyb;
        T xa = d.xbar[a0][i], ha = d.Hxbar[a0][i];
        if (acc) {
          xa = omap * xa + ap * d.x[cur][i];
          ha = omap * ha + ap * d.Hx[cur][i];
          d.xbar[ab][i] = xa;
          d.Hxbar[ab][i] = ha;
        }
        col_cand(q + 8, double(xa), double(ha), double(atyb), qx, qx0, hxb, atyb0, lx, ux, ex, xst);
      }
    }
  }
  block_reduce_store<16>(q, CK_MAXMASK, d.part + P_CK_C * kMaxBlocks, g.b);
  if (arrive_last(d.ctr + 1, g.nb)) {
    if (mode == 0)
      check_final_body<COND>(d.st, d.part, nb_r, g.nb, d.hw);
    else
      inner_begin_body(d.st, d.part, nb_r, g.nb);
    if (threadIdx.x == 0) d.ctr[1] = 0u;
  }
}

template <typename T, int G, bool COND>
__global__ void __launch_bounds__(kBlock) k_check_cols(Dev<T> d, int mode, int nb_r) {
  check_cols_body<T, G, COND>(d, mode, nb_r, hw_grid());
}

// Decisions of the check (single block): inner termination of both candidates
// (Eq. inner-termination), iteration limit, restart criteria and primal weight.
template <bool COND>
__device__ void check_final_body(DevState *stg, const double *part, int nb_r, int nb_c,
                                 cudaGraphConditionalHandle hw) {
  __shared__ DevState S;
  state_load(S, stg);
  double a[16], b[16];
  final_reduce<16>(part + P_CK_R * kMaxBlocks, nb_r, CK_MAXMASK, a);
  final_reduce<16>(part + P_CK_C * kMaxBlocks, nb_c, CK_MAXMASK, b);
  if (threadIdx.x == 0) {
    DevState *st = &S;
    double q[16];
    for (int k = 0; k < 16; ++k) q[k] = ((CK_MAXMASK >> k) & 1u) ? fmax(a[k], b[k]) : a[k] + b[k];
    for (int k = 0; k < 16; ++k) st->chk[k] = q[k];
    // The averages of this trial's acceptance were materialised by the check
    // kernels.  The check is consumed here (a repeated launch of the check
    // kernels without a trial in between does nothing); the restart itself is
    // applied by k_check_apply on restart_flag.
    st->acur ^= st->accepted;
    st->accepted = 0;
    st->restart_flag = 0;
    st->check_due = 0;
    const double dta = st->dta, dtr = st->dtr;
    const double spc = fmax(1.0, q[1]), sdc = fmax(1.0, q[3]);
    const double spa = fmax(1.0, q[9]), sda = fmax(1.0, q[11]);
    const bool okc = q[0] <= dta + dtr * spc && q[2] <= dta + dtr * sdc;
    const bool oka = q[8] <= dta + dtr * spa && q[10] <= dta + dtr * sda;
    if (!st->ignore_conv && okc) {
      st->status = ST_CONVERGED;
      st->ret_avg = 0;
    } else if (!st->ignore_conv && oka) {
      st->status = ST_CONVERGED;
      st->ret_avg = 1;
    } else if (st->t_total == st->k_in) {
      st->status = ST_ITER_LIMIT;
    } else {
      const double om = st->omega;
      const double kc = sqrt(om * q[4] + q[5] / om);
      const double ka = sqrt(om * q[12] + q[13] / om);
      const bool use_avg = ka < kc;
      const double kcand = use_avg ? ka : kc;
      const bool restart = kcand <= st->beta_suff * st->k_restart ||
                           (kcand <= st->beta_nec * st->k_restart && kcand > st->k_last) ||
                           (double)st->t >= st->beta_art * (double)st->t_total;
      st->k_last = kcand;
      if (restart) {
        const double dW = sqrt(use_avg ? q[14] : q[6]);
        const double dY = sqrt(use_avg ? q[15] : q[7]);
        if (dW > 0.0 && dY > 0.0) st->omega = exp(0.25 * log(dY / dW) + 0.75 * log(om));
        st->kappa = 1.0;
        st->t = 0;
        st->k_restart = kcand;
        st->k_last = INFINITY;
        st->restarts += 1;
        st->restart_flag = 1;
        st->restart_use_avg = use_avg ? 1 : 0;
      }
      if (st->t_total == st->pause_at) st->status = ST_PAUSED;
    }
    if (COND && hw) cudaGraphSetConditional(hw, (st->status == ST_RUNNING && st->slot_left > 0) ? 1u : 0u);
  }
  state_store(stg, S);
}

// Restart (Algorithm 4): optionally move the current point to the average
// (with its cached products), then make it the epoch start and clear the
// averages.  Idempotent, so a repeated launch is harmless.
template <typename T>
__device__ __forceinline__ void check_apply_body(const Dev<T> &d, GridCtx g) {
  const DevState *st = d.st;
  if (!st->restart_flag) return;
  const int cur = st->cur, ab = st->acur;
  const bool ua = st->restart_use_avg;
  PDNQP_VGRID_STRIDE(i, d.n, g) {
    T x = d.x[cur][i], hx = d.Hx[cur][i];
    if (ua) {
      x = d.xbar[ab][i];
      hx = d.Hxbar[ab][i];
      d.x[cur][i] = x;
      d.Hx[cur][i] = hx;
      d.Aty[cur][i] = d.Atybar[i];
    }
    d.xst[i] = x;
    d.xbar[ab][i] = x;
    d.Hxbar[ab][i] = hx;
  }
  PDNQP_VGRID_STRIDE(j, d.m, g) {
    T y = d.y[cur][j], r = d.r[cur][j];
    if (ua) {
      y = d.ybar[ab][j];
      r = d.rbar[ab][j];
      d.y[cur][j] = y;
      d.r[cur][j] = r;
      d.Bw[cur][j] = d.Bwbar[j];
    }
    d.yst[j] = y;
    d.rst[j] = r;
    d.ybar[ab][j] = y;
    d.rbar[ab][j] = r;
    if (j >= d.mE) {
      T s = d.s[cur][j];
      if (ua) {
        s = d.sbar[ab][j];
        d.s[cur][j] = s;
      }
      d.sst[j] = s;
      d.sbar[ab][j] = s;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBlock) k_check_apply(Dev<T> d) {
  check_apply_body<T>(d, hw_grid());
}

// ===========================================================================
// Setup of one inner solve (a0): warm start, penalty + inner Ruiz scaling,
// diagonal steps, cached products.
// ===========================================================================

// Base rows of one inner solve (Eq. inner-warm-start, in FP64): v = A x_b,
// s_b = P_[l_c,u_c](v + lambda / sigma) and r_b = v - s_b on inequality rows,
// r_b = v - b_E on equality rows; then B w_b, h' = h - B w_b, the base
// gradients of the s and r blocks, the shifted slack bounds, and zero
// corrections.
template <typename T>
__global__ void __launch_bounds__(kBlock) k_base_rows(Dev<T> d, Mat<double> Ad, const double *lc, const double *uc,
                                                      double *sb, double *rb) {
  const int cur = d.st->cur;
  const double *__restrict__ x = d.xb;
  PDNQP_GRID_STRIDE(j, d.m) {
    double v = 0.0;
    for (int k = Ad.rp[j]; k < Ad.rp[j + 1]; ++k) v += Ad.val[k] * x[Ad.ci[k]];
    const double lam = d.lam[j], sig = d.sig[j], yb = d.yb[j];
    double s = 0.0, r, bw;
    if (j >= d.mE) {
      s = v + lam / sig;
      s = s < lc[j] ? lc[j] : s;
      s = s > uc[j] ? uc[j] : s;
      r = v - s;
      bw = v - s - r;
      d.ls[j] = T(lc[j] - s);
      d.us[j] = T(uc[j] - s);
      d.qs[j] = T(yb);
      d.s[cur][j] = T(0);
    } else {
      r = v - lc[j];
      bw = v - r;
    }
    const double h = j < d.mE ? lc[j] : 0.0;
    sb[j] = s;
    rb[j] = r;
    d.h[j] = T(h);
    d.Bwb[j] = T(bw);
    d.hp[j] = T(h - bw);
    d.qr[j] = T(lam + sig * r + yb);
    d.r[cur][j] = T(0);
    d.y[cur][j] = T(0);
    d.Bw[cur][j] = T(0);
  }
}

// Base columns: H x_b and A' y_b in FP64, q'_x = c - z / gamma + H x_b - A' y_b,
// q_x, the shifted bounds, and zero corrections with zero cached products.
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_base_cols(Dev<T> d, Mat<double> Hd, Mat<double> Atd, const double *c,
                                                      const double *z, const double *lxd, const double *uxd,
                                                      double ginv) {
  const int cur = d.st->cur;
  const double *__restrict__ x = d.xb;
  const double *__restrict__ y = d.yb;
  TileIter ti;
  for (long long tile = ti.first; tile < d.n; tile += ti.step) {
    const double hx = tile_row_sum<G, double>(Hd.rp, Hd.ci, Hd.val, tile, d.n, [&](int k, double a) { return a * x[k]; });
    const double aty = tile_row_sum<G, double>(Atd.rp, Atd.ci, Atd.val, tile, d.n, [&](int k, double a) { return a * y[k]; });
    const long long i = tile + ti.lane;
    if (i < d.n) {
      const double q0 = c[i] - z[i] * ginv;
      d.qx0[i] = T(q0);
      d.qx[i] = T(q0 + hx - aty);
      d.Hxb[i] = T(hx);
      d.Atyb[i] = T(aty);
      d.lx[i] = T(lxd[i] - x[i]);
      d.ux[i] = T(uxd[i] - x[i]);
      d.x[cur][i] = T(0);
      d.Hx[cur][i] = T(0);
      d.Aty[cur][i] = T(0);
    }
  }
}

// Penalty scaling as the initial column scale of the r block: e_r = 1/sqrt(sigma).
template <typename T>
__global__ void k_iscale_init(Dev<T> d) {
  PDNQP_GRID_STRIDE(i, d.n) d.ex[i] = T(1);
  PDNQP_GRID_STRIDE(j, d.m) {
    d.es[j] = T(1);
    d.er[j] = T(1.0 / sqrt(d.sig[j]));
    d.dy[j] = T(1);
  }
}

// Reciprocal square root in the storage precision.
__device__ __forceinline__ float rsqrt_t(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_t(double v) { return rsqrt(v); }

// Inner Ruiz, l_inf norms of the x columns of [[H~, B~^T], [B~, 0]]:
// max(max_k |e_k H_ki e_i|, max_j |d_j A_ji e_i|), in the storage precision T.
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_iruiz_cols(Dev<T> d, double *cnx) {
  TileIter ti;
  for (long long tile = ti.first; tile < d.n; tile += ti.step) {
    const long long i = tile + ti.lane;
    // e_i is applied after the reduction (max over k of |e_k H_ki| times e_i).
    const T a = tile_row_max<G, T>(d.H.rp, d.H.ci, d.H.val, tile, d.n, [&](int k, T v) { return fabs(d.ex[k] * v); });
    const T b = tile_row_max<G, T>(d.At.rp, d.At.ci, d.At.val, tile, d.n, [&](int k, T v) { return fabs(d.dy[k] * v); });
    if (i < d.n) cnx[i] = double(fmax(a, b) * d.ex[i]);
  }
}

// Inner Ruiz, rows of B~ and the s / r columns: row j: max(max_k |d_j A_jk e_k|,
// d_j e_s (I rows), d_j e_r); s column: d_j e_s; r column: max(e_r^2 sigma_j, d_j e_r).
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_iruiz_rows(Dev<T> d, double *rn, double *cns, double *cnr) {
  TileIter ti;
  for (long long tile = ti.first; tile < d.m; tile += ti.step) {
    const T a = tile_row_max<G, T>(d.A.rp, d.A.ci, d.A.val, tile, d.m, [&](int k, T v) { return fabs(v * d.ex[k]); });
    const long long j = tile + ti.lane;
    if (j < d.m) {
      const T dj = d.dy[j];
      const T er = d.er[j];
      T rowv = fmax(a * dj, dj * er);
      if (j >= d.mE) {
        const T es = d.es[j];
        rowv = fmax(rowv, dj * es);
        cns[j] = double(dj * es);
      }
      rn[j] = double(rowv);
      cnr[j] = double(fmax(er * er * T(d.sig[j]), dj * er));
    }
  }
}

template <typename T>
__global__ void k_iruiz_update(Dev<T> d, const double *cnx, const double *rn, const double *cns, const double *cnr) {
  PDNQP_GRID_STRIDE(i, d.n) {
    const T c = T(cnx[i]);
    if (c > T(0)) d.ex[i] = d.ex[i] * rsqrt_t(c);
  }
  PDNQP_GRID_STRIDE(j, d.m) {
    const T r = T(rn[j]);
    if (r > T(0)) d.dy[j] = d.dy[j] * rsqrt_t(r);
    const T cr = T(cnr[j]);
    if (cr > T(0)) d.er[j] = d.er[j] * rsqrt_t(cr);
    if (j >= d.mE) {
      const T cs = T(cns[j]);
      if (cs > T(0)) d.es[j] = d.es[j] * rsqrt_t(cs);
    }
  }
}

// Eq. diagonal-scales for the x columns (m_w) and the effective primal step
// tau_eff / (kappa / omega) = e^2 * 0.99 / m_w (Eq. diagonal-steps), in the
// storage precision; imwx = 1 / m_w is kept for m_y.
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_mw_cols(Dev<T> d, double *imwx) {
  TileIter ti;
  for (long long tile = ti.first; tile < d.n; tile += ti.step) {
    const T h1 = tile_row_sum<G, T>(d.H.rp, d.H.ci, d.H.val, tile, d.n, [&](int k, T v) { return fabs(d.ex[k] * v); });
    const T b1 = tile_row_sum<G, T>(d.At.rp, d.At.ci, d.At.val, tile, d.n, [&](int k, T v) { return fabs(d.dy[k] * v); });
    const T b2 = tile_row_sum<G, T>(d.At.rp, d.At.ci, d.At.val, tile, d.n, [&](int k, T v) {
      const T bb = d.dy[k] * v;
      return T(d.sig[k]) * bb * bb;
    });
    const long long i = tile + ti.lane;
    if (i < d.n) {
      const T ei = d.ex[i];
      const T mw = h1 * ei + fmax(b1 * ei, sqrt(b2) * ei);
      imwx[i] = double(T(1) / mw);
      d.taux[i] = ei * ei * (T(0.99) / mw);
      d.itaux[i] = mw / (T(0.99) * ei * ei);
    }
  }
}

// m_w of the s and r columns, their steps, and m_y with the dual step
// eta_eff / (kappa omega) = d^2 * 0.99 / m_y.
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) k_my_rows(Dev<T> d, const double *imwx) {
  TileIter ti;
  for (long long tile = ti.first; tile < d.m; tile += ti.step) {
    const T a = tile_row_sum<G, T>(d.A.rp, d.A.ci, d.A.val, tile, d.m, [&](int k, T v) {
      const T bb = v * d.ex[k];
      return bb * bb * T(imwx[k]);
    });
    const long long j = tile + ti.lane;
    if (j < d.m) {
      const T dj = d.dy[j];
      const T sg = T(d.sig[j]);
      const T er = d.er[j];
      const T br = dj * er;
      const T mwr = er * er * sg + br;
      d.taur[j] = er * er * (T(0.99) / mwr);
      d.itaur[j] = mwr / (T(0.99) * er * er);
      T my = a * dj * dj + br * br / mwr;
      if (j >= d.mE) {
        const T es = d.es[j];
        const T bs = dj * es;
        const T mws = fmax(bs, sqrt(sg * bs * bs));
        d.taus[j] = es * es * (T(0.99) / mws);
        d.itaus[j] = mws / (T(0.99) * es * es);
        my += bs * bs / mws;
      }
      d.eta[j] = dj * dj * (T(0.99) / my);
      d.ieta[j] = my / (T(0.99) * dj * dj);
    }
  }
}

// Epoch start and averages of the inner start (buffer 0).
template <typename T>
__global__ void k_inner_init(Dev<T> d) {
  const int cur = d.st->cur;
  PDNQP_GRID_STRIDE(i, d.n) {
    d.xst[i] = d.x[cur][i];
    d.xbar[0][i] = d.x[cur][i];
    d.Hxbar[0][i] = d.Hx[cur][i];
  }
  PDNQP_GRID_STRIDE(j, d.m) {
    d.yst[j] = d.y[cur][j];
    d.rst[j] = d.r[cur][j];
    d.ybar[0][j] = d.y[cur][j];
    d.rbar[0][j] = d.r[cur][j];
    if (j >= d.mE) {
      d.sst[j] = d.s[cur][j];
      d.sbar[0][j] = d.s[cur][j];
    }
  }
}

// End of an inner solve: the outer x and inner y become base + correction
// (the current point, or the average when it is the converged candidate).
template <typename T>
__global__ void k_finish(Dev<T> d, double *x64, double *y64, int use_avg) {
  const int cur = d.st->cur, ab = d.st->acur ^ d.st->accepted;
  const T *__restrict__ dx = use_avg ? d.xbar[ab] : d.x[cur];
  const T *__restrict__ dy = use_avg ? d.ybar[ab] : d.y[cur];
  PDNQP_GRID_STRIDE(i, d.n) x64[i] += double(dx[i]);
  PDNQP_GRID_STRIDE(j, d.m) y64[j] += double(dy[j]);
}

// Totals of the current and averaged points for a snapshot:
// out = [w (dw) | y (m) | wbar (dw) | ybar (m)], w = (x, s_I, r_E, r_I).
template <typename T>
__global__ void k_totals(Dev<T> d, double *out) {
  const int cur = d.st->cur, ab = d.st->acur ^ d.st->accepted;
  const long long n = d.n, m = d.m, mI = m - d.mE, dw = n + mI + m;
  for (int a = 0; a < 2; ++a) {
    const T *x = a ? d.xbar[ab] : d.x[cur];
    const T *s = a ? d.sbar[ab] : d.s[cur];
    const T *r = a ? d.rbar[ab] : d.r[cur];
    const T *y = a ? d.ybar[ab] : d.y[cur];
    double *o = out + a * (dw + m);
    PDNQP_GRID_STRIDE(i, n) o[i] = d.xb[i] + double(x[i]);
    PDNQP_GRID_STRIDE(j, m) {
      if (j >= d.mE) o[n + (j - d.mE)] = d.sb[j] + double(s[j]);
      o[n + mI + j] = d.rb[j] + double(r[j]);
      o[dw + j] = d.yb[j] + double(y[j]);
    }
  }
}

// Restart metric of the inner start (last block of the mode-1 check).
__device__ void inner_begin_body(DevState *st, const double *part, int nb_r, int nb_c) {
  double a[16], b[16];
  final_reduce<16>(part + P_CK_R * kMaxBlocks, nb_r, CK_MAXMASK, a);
  final_reduce<16>(part + P_CK_C * kMaxBlocks, nb_c, CK_MAXMASK, b);
  if (threadIdx.x != 0) return;
  const double om = st->omega;
  st->k_restart = sqrt(om * (a[4] + b[4]) + (a[5] + b[5]) / om);
  st->k_last = INFINITY;
  st->status = st->start_status;
}


// ===========================================================================
// Batched form: the inner iterations of many problems in one launch per
// phase.  Block k of a batched launch works for problem map[k].p as block
// map[k].b of map[k].nb (the problem's own partition, the same as when it
// runs alone, so its reductions and its iterates are bitwise those of its
// solo graph-form solve); the problem's device pointers come from devs[p].
// Every phase skips a problem whose status is not ST_RUNNING, so problems
// that wait for their host outer iteration cost one state read per block.
// ===========================================================================
struct BatchBlk {
  int p, b, nb;
};

// The problem's Dev copied to shared memory once per block (its pointers are
// then read without a global-memory round trip per use).
template <typename T>
__device__ __forceinline__ const Dev<T> &batch_dev(const Dev<T> *devs, int p) {
  __shared__ __align__(16) unsigned char buf[sizeof(Dev<T>)];
  static_assert(sizeof(Dev<T>) % 4 == 0, "Dev must be a whole number of words");
  const int *src = reinterpret_cast<const int *>(devs + p);
  for (int i = threadIdx.x; i < (int)(sizeof(Dev<T>) / 4); i += blockDim.x) reinterpret_cast<int *>(buf)[i] = src[i];
  __syncthreads();
  return *reinterpret_cast<const Dev<T> *>(buf);
}

template <typename T>
__global__ void __launch_bounds__(kBlock) kb_primal(const Dev<T> *devs, const BatchBlk *map) {
  const BatchBlk e = map[blockIdx.x];
  const Dev<T> &d = batch_dev(devs, e.p);
  if (d.st->status != ST_RUNNING) return;
  primal_phase<T>(d, d.st, GridCtx{e.b, e.nb});
}

template <typename T, int G>
__global__ void __launch_bounds__(kBlock) kb_rows(const Dev<T> *devs, const BatchBlk *map) {
  const BatchBlk e = map[blockIdx.x];
  rows_trial_body<T, G>(batch_dev(devs, e.p), GridCtx{e.b, e.nb});
}

// nb_rows[p]: blocks of problem p in the row launches (its row partials).
template <typename T, int G>
__global__ void __launch_bounds__(kBlock) kb_cols(const Dev<T> *devs, const BatchBlk *map, const int *nb_rows) {
  const BatchBlk e = map[blockIdx.x];
  cols_trial_body<T, G, false>(batch_dev(devs, e.p), nb_rows[e.p], GridCtx{e.b, e.nb});
}

template <typename T, int G>
__global__ void __launch_bounds__(kBlock) kb_check_rows(const Dev<T> *devs, const BatchBlk *map) {
  const BatchBlk e = map[blockIdx.x];
  check_rows_body<T, G>(batch_dev(devs, e.p), 0, GridCtx{e.b, e.nb});
}

template <typename T, int G>
__global__ void __launch_bounds__(kBlock) kb_check_cols(const Dev<T> *devs, const BatchBlk *map,
                                                        const int *nb_rows) {
  const BatchBlk e = map[blockIdx.x];
  check_cols_body<T, G, false>(batch_dev(devs, e.p), 0, nb_rows[e.p], GridCtx{e.b, e.nb});
}

template <typename T>
__global__ void __launch_bounds__(kBlock) kb_check_apply(const Dev<T> *devs, const BatchBlk *map) {
  const BatchBlk e = map[blockIdx.x];
  check_apply_body<T>(batch_dev(devs, e.p), GridCtx{e.b, e.nb});
}

// Scheduler edits between graph launches: problems in `go` that are set up
// (ST_READY) start running; problems in `stop` that still run pause (their
// time limit passed).
template <typename T>
__global__ void kb_control(const Dev<T> *devs, const int *go, int ngo, const int *stop, int nstop) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ngo + nstop; k += gridDim.x * blockDim.x) {
    DevState *st = devs[k < ngo ? go[k] : stop[k - ngo]].st;
    if (k < ngo) {
      if (st->status == ST_READY) st->status = ST_RUNNING;
    } else if (st->status == ST_RUNNING) {
      st->status = ST_PAUSED;
    }
  }
}

// Copies every problem's device state into one array (one read-back per launch).
template <typename T>
__global__ void kb_gather_states(const Dev<T> *devs, int count, DevState *out) {
  constexpr int W = (int)(sizeof(DevState) / 4);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < (long long)count * W;
       k += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(k / W), w = (int)(k % W);
    reinterpret_cast<int *>(out + p)[w] = __ldcg(reinterpret_cast<const int *>(devs[p].st) + w);
  }
}

}  // namespace
}  // namespace pdq
