// Templated implementation of SolverBase (T = double: plain FP64 form,
// T = float: FP32-bulk form).  Included by exactly one .cu per T.
#pragma once
#include <algorithm>
#include <cstdio>

#include "kernels.cuh"
#include "kernels_outer.cuh"
#include "solver.cuh"

namespace pdq {

#define PDNQP_CK(expr)                                                            \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      last_err_ = std::string(#expr) + ": " + cudaGetErrorString(_e);             \
      return PDNQP_ERR_CUDA;                                                      \
    }                                                                             \
  } while (0)

#define PDNQP_TRY(x)          \
  do {                        \
    int _r = (x);             \
    if (_r < 0) return _r;    \
  } while (0)

// K = entries per lane per CSR-stream chunk (chunk = 32 K nonzeros per warp).
// Kernels are instantiated for K in {4, 8, 16}; GroupIter kernels read it as
// lanes per row.
template <typename F>
static void with_G(int g, F f) {
  switch (g) {
    case 4: f(std::integral_constant<int, 4>()); break;
    case 8: f(std::integral_constant<int, 8>()); break;
    default: f(std::integral_constant<int, 16>()); break;
  }
}

// K from the mean row length: the smallest power of two >= mean, in [4, 16].
static int pick_g(long long nnz, long long rows) {
  const double mean = rows > 0 ? (double)nnz / (double)rows : 1.0;
  int g = 4;
  while (g < 16 && g < mean) g *= 2;
  return g;
}

// Where a solver in the batched form hands its inner solves (BatchRunner).
struct BatchHook {
  virtual ~BatchHook() {}
  // Blocks until inner solve idx has left the running state; returns 1 when
  // it was stopped at its time limit (deadline, steady-clock seconds), else 0.
  virtual int run_inner(int idx, DevState *S, double deadline) = 0;
};

// Smallest relative inner tolerance of the FP32-bulk form: 8 units of FP32 roundoff (2^-24).
constexpr double kFp32RelTolFloor = 8.0 * 5.9604644775390625e-8;

template <typename T>
class BatchRunner;

template <typename T>
class Solver : public SolverBase {
  friend class BatchRunner<T>;

 public:
  explicit Solver(cudaStream_t s) : s_(s) {
    // Stream capture needs a non-default stream: make one when none is given.
    if (!s_ && cudaStreamCreateWithFlags(&s_, cudaStreamNonBlocking) == cudaSuccess) own_stream_ = true;
  }
  ~Solver() override {
    if (s_) cudaStreamSynchronize(s_);
    if (gexec_) cudaGraphExecDestroy(gexec_);
    for (cudaEvent_t e : replay_ev_)
      if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : loop_ev_)
      if (e) cudaEventDestroy(e);
    for (void *p : allocs_) cudaFree(p);
    if (hst_) cudaFreeHost(hst_);
    if (hfault_) cudaFreeHost(hfault_);
    if (own_stream_) cudaStreamDestroy(s_);
  }

  // ------------------------------------------------------------------ setup
  int setup(const HostProblem &P, const Params &prm, std::string *err) override {
    int rc = setup_impl(P, prm);
    if (rc < 0 && err) *err = last_err_;
    return rc;
  }

  double gamma() const override { return gamma_; }
  double lambda_min() const override { return lam_min_; }
  int64_t nnz_q() const override { return nnzH_; }
  void set_gamma(double g) override { gamma_pending_ = g; }

  // Learned controller: BF16 weights on the device (rounded there from the
  // FP32 copy), evaluated once per outer iteration on the solve's stream.
  int set_controller(const float *w, int count) override {
    has_ctrl_ = false;
    if (!w || count <= 0) return 0;
    if (!ctrl_w_) {
      PDNQP_TRY(dalloc(&ctrl_w32_, (size_t)count));
      PDNQP_TRY(dalloc(&ctrl_w_, (size_t)count));
      PDNQP_TRY(dalloc(&ctrl_x_, 16));
      PDNQP_TRY(dalloc(&ctrl_y_, 2));
    }
    PDNQP_CK(cudaMemcpyAsync(ctrl_w32_, w, sizeof(float) * count, cudaMemcpyHostToDevice, s_));
    if (pdnqp_mlp_to_bf16(ctrl_w32_, ctrl_w_, count, s_) != 0) {
      last_err_ = std::string("controller weights: ") + pdnqp_mlp_last_error();
      return PDNQP_ERR_CUDA;
    }
    PDNQP_CK(cudaStreamSynchronize(s_));
    has_ctrl_ = true;
    return 0;
  }
  const std::vector<double> &trace() const override { return trace_; }
  long long ctrl_fallbacks() const override { return ctrl_fallbacks_; }

  int set_start(const double *x0, const double *lam0_int) override {
    // Stored in original coordinates / internal row order; applied at the next solve.
    if (x0) {
      has_x0_ = true;
      h_x0_.assign(x0, x0 + n_);
    } else {
      has_x0_ = false;
    }
    if (lam0_int && m_) {
      has_l0_ = true;
      h_l0_.assign(lam0_int, lam0_int + m_);
    } else {
      has_l0_ = false;
    }
    return 0;
  }

  int solve(double ea, double er, Params &prm, std::string *err) override {
    int rc = solve_impl(ea, er, prm);
    if (rc < 0 && err) *err = last_err_;
    return rc;
  }

  int debug_inner(Params &prm, int nck, const int64_t *ck, double *snap, std::string *err) override {
    int rc = debug_impl(prm, nck, ck, snap);
    if (rc < 0 && err) *err = last_err_;
    return rc;
  }

  int get(double *x_orig, double *lam_int_orig, Result *r) override {
    if (r) *r = res_;
    if (!solved_once_) return (x_orig || lam_int_orig) ? PDNQP_ERR_STATE : 0;
    if (x_orig && n_) PDNQP_CK(cudaMemcpy(x_orig, xo_, sizeof(double) * n_, cudaMemcpyDeviceToHost));
    if (lam_int_orig && m_) PDNQP_CK(cudaMemcpy(lam_int_orig, lo_, sizeof(double) * m_, cudaMemcpyDeviceToHost));
    return 0;
  }

  // Replays one hot kernel (measurement hook); writes trial buffers only.
  int replay(int which, int reps) override {
    if (!ready_) return PDNQP_ERR_STATE;
    // The kernels are gated on a running status: set it, then restore.
    DevState saved;
    PDNQP_CK(cudaMemcpyAsync(&saved, st_, sizeof(DevState), cudaMemcpyDeviceToHost, s_));
    PDNQP_CK(cudaStreamSynchronize(s_));
    DevState run = saved;
    run.status = ST_RUNNING;
    PDNQP_CK(cudaMemcpyAsync(st_, &run, sizeof(DevState), cudaMemcpyHostToDevice, s_));
    const int kind = which & 3;
    auto one = [&]() {
      if (kind == 0) launch_cols();
      else if (kind == 1) launch_rows();
      else launch_primal();
    };
    if (which & 8) {
      // The same launches captured as one CUDA graph (per-node cost as in the solve).
      cudaGraph_t g;
      PDNQP_CK(cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal));
      for (int k = 0; k < reps; ++k) one();
      PDNQP_CK(cudaStreamEndCapture(s_, &g));
      cudaGraphExec_t ge;
      cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        last_err_ = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
        return PDNQP_ERR_CUDA;
      }
      PDNQP_CK(cudaGraphUpload(ge, s_));
      PDNQP_CK(cudaStreamSynchronize(s_));
      if (replay_ev_[0] == nullptr) {
        PDNQP_CK(cudaEventCreate(&replay_ev_[0]));
        PDNQP_CK(cudaEventCreate(&replay_ev_[1]));
      }
      PDNQP_CK(cudaEventRecord(replay_ev_[0], s_));
      PDNQP_CK(cudaGraphLaunch(ge, s_));
      PDNQP_CK(cudaEventRecord(replay_ev_[1], s_));
      PDNQP_CK(cudaStreamSynchronize(s_));
      float ms = 0.f;
      PDNQP_CK(cudaEventElapsedTime(&ms, replay_ev_[0], replay_ev_[1]));
      last_replay_ms_ = ms;
      cudaGraphExecDestroy(ge);
    } else {
      for (int k = 0; k < reps; ++k) one();
    }
    PDNQP_CK(cudaMemcpyAsync(st_, &saved, sizeof(DevState), cudaMemcpyHostToDevice, s_));
    PDNQP_CK(cudaStreamSynchronize(s_));
    return 0;
  }

  // Compulsory DRAM bytes (each array touched once, int32 indices, value size
  // sizeof(T)); gathers of x / y assumed L2-resident.
  double last_replay_ms() const override { return last_replay_ms_; }

  double kernel_bytes(int which) const override {
    const double v = sizeof(T), n = n_, m = m_, mI = m_ - mE_;
    const double mat_h = (v + 4) * nnzH_ + 4 * (n + 1), mat_a = (v + 4) * nnzA_ + 4 * (m + 1);
    const double mat_at = (v + 4) * nnzA_ + 4 * (n + 1);
    // k_cols: H, A^T; reads x_tr, x, Hx, Aty, taux; writes Hx_tr, Aty_tr; gathers x_tr (n) and y_tr (m).
    const double cols = mat_h + mat_at + v * n * 7 + v * m;
    // k_rows: A; reads y, r, rbar, lam(8), sig(8), taur, Bw, eta, h + s, sbar?, taus, ls, us (I); writes r, Bw, y (+ s).
    const double rows = mat_a + v * n + m * (8 * v + 16) + mI * 5 * v;
    // k_primal: reads qx, Hxbar, Hx, Aty, x, taux, lx, ux; writes x_tr.
    const double primal = 9 * v * n;
    // k_average: reads/writes xbar, Hxbar (read x, Hx), ybar, rbar (+ sbar), (read y, r, s).
    const double avg = 6 * v * n + 6 * v * m + 3 * v * mI;
    if (which == 5) {
      // One trial of the persistent loop (k_trials) after an accepted trial,
      // each array counted once per pass (gathers assumed served from L2):
      // primal: reads x, Hx, Hxbar, xbar, qx, A'y, taux, lx, ux; writes x_tr,
      //   Hxbar', xbar'.
      const double p5 = 12 * v * n;
      // rows: A; gathers x_tr; reads y, r, rbar, ybar, taur, qr, Bw, eta, hp,
      //   itaur, ieta and sig (FP64) per row, s, sbar, taus, qs, ls, us,
      //   itaus per inequality row; writes rbar', ybar', r, Bw, y (+ sbar', s).
      const double r5 = mat_a + v * n + m * (16 * v + 8) + mI * 9 * v;
      // cols: H, A^T; gathers x_tr (also read per row) and y_tr; reads x,
      //   Hx, A'y, taux; writes Hx_tr, A'y_tr.
      const double c5 = mat_h + mat_at + 7 * v * n + v * m;
      return p5 + r5 + c5;
    }
    if (which == 0) return cols;
    if (which == 1) return rows;
    if (which == 2) return primal;
    if (which == 3) return avg;
    return cols + rows + primal + avg;
  }

 private:
  // ------------------------------------------------------------- helpers
  // Every array carries kPad zeroed elements past its end: the bulk copies of
  // the panel stream round their ranges up to 16 bytes and may read them.
  static constexpr size_t kPad = 4;
  template <typename U>
  int dalloc(U **p, size_t count) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, (std::max<size_t>(count, 1) + kPad) * sizeof(U));
    if (e != cudaSuccess) {
      last_err_ = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      return PDNQP_ERR_OOM;
    }
    allocs_.push_back(q);
    *p = (U *)q;
    PDNQP_CK(cudaMemsetAsync((char *)q + count * sizeof(U), 0, kPad * sizeof(U), s_));
    return 0;
  }
  template <typename U>
  int upload(U **p, const std::vector<U> &h) {
    int rc = dalloc(p, h.size());
    if (rc) return rc;
    if (!h.empty()) PDNQP_CK(cudaMemcpyAsync(*p, h.data(), sizeof(U) * h.size(), cudaMemcpyHostToDevice, s_));
    return 0;
  }

  int grid_n() const { return grid_for(n_, kBlock); }
  int grid_m() const { return grid_for(m_, kBlock); }
  int grid_nm() const { return grid_for(std::max(n_, m_), kBlock); }
  int grid_rows_g(long long rows, int g) const { return grid_for(rows, kBlock / g); }

  int reduce_to_host(int nq, int nb, unsigned mask, double *out) {
    k_reduce_rows<<<nq, 32, 0, s_>>>(part_, nq, nb, mask, dred_);
    PDNQP_CK(cudaGetLastError());
    PDNQP_CK(cudaMemcpyAsync(hred_.data(), dred_, sizeof(double) * nq, cudaMemcpyDeviceToHost, s_));
    PDNQP_CK(cudaStreamSynchronize(s_));
    for (int q = 0; q < nq; ++q) out[q] = hred_[q];
    return 0;
  }

  // -------------------------------------------------------- setup_impl
  int setup_impl(const HostProblem &P, const Params &prm) {
    n_ = P.n;
    m_ = P.m;
    mE_ = P.mE;
    nnzA_ = P.a_ci.size();
    nnzH_ = P.q_ci.size();
    PDNQP_TRY(dalloc(&st_, 1));
    PDNQP_CK(cudaMallocHost(&hst_, sizeof(DevState)));
    PDNQP_CK(cudaMallocHost(&hfault_, sizeof(unsigned)));
    *hfault_ = 0u;
    PDNQP_TRY(dalloc(&part_, (size_t)kMaxPartials * kMaxBlocks));
    PDNQP_TRY(dalloc(&xprev_, (size_t)n_));
    PDNQP_TRY(dalloc(&lamprev_, (size_t)std::max(m_, 1)));
    PDNQP_TRY(dalloc(&dxv_, (size_t)n_));
    PDNQP_TRY(dalloc(&dred_, 128));
    hred_.resize(128);
    // FP64 matrices.
    int *qrp, *qci, *qdiag, *arp, *aci, *atrp, *atci;
    PDNQP_TRY(upload(&qrp, P.q_rp));
    PDNQP_TRY(upload(&qci, P.q_ci));
    PDNQP_TRY(upload(&qdiag, P.q_diag));
    PDNQP_TRY(upload(&qv_, P.q_v));
    PDNQP_TRY(upload(&arp, P.a_rp));
    PDNQP_TRY(upload(&aci, P.a_ci));
    PDNQP_TRY(upload(&av_, P.a_v));
    PDNQP_TRY(upload(&atrp, P.at_rp));
    PDNQP_TRY(upload(&atci, P.at_ci));
    PDNQP_TRY(upload(&atv_, P.at_v));
    qdiag_ = qdiag;
    Hd_ = {n_, qrp, qci, qv_};
    Ad_ = {m_, arp, aci, av_};
    Atd_ = {n_, atrp, atci, atv_};
    gA0_ = gA_ = prm.g_rows ? prm.g_rows : pick_g(nnzA_, m_);
    gN0_ = gN_ = prm.g_cols ? prm.g_cols : pick_g(std::max(nnzH_, nnzA_), n_);
    // FP64 vectors.
    PDNQP_TRY(upload(&c_, P.c));
    PDNQP_TRY(upload(&lxd_, P.lx));
    PDNQP_TRY(upload(&uxd_, P.ux));
    PDNQP_TRY(upload(&lcd_, P.lc));
    PDNQP_TRY(upload(&ucd_, P.uc));
    PDNQP_TRY(dalloc(&Dc_, m_));
    PDNQP_TRY(dalloc(&Dx_, n_));
    PDNQP_TRY(dalloc(&lam_, m_));
    PDNQP_TRY(dalloc(&sig_, m_));
    PDNQP_TRY(dalloc(&rprev_, m_));
    PDNQP_TRY(dalloc(&rcur_, m_));
    PDNQP_TRY(dalloc(&z_, n_));
    PDNQP_TRY(dalloc(&xo_, n_));
    PDNQP_TRY(dalloc(&lo_, m_));
    PDNQP_TRY(dalloc(&scn_[0], n_));
    PDNQP_TRY(dalloc(&scn_[1], n_));
    PDNQP_TRY(dalloc(&scm_[0], m_));
    PDNQP_TRY(dalloc(&scm_[1], m_));
    PDNQP_TRY(dalloc(&scm_[2], m_));
    PDNQP_TRY(dalloc(&dx0_, n_));
    PDNQP_TRY(dalloc(&dl0_, m_));
    // ---- outer Ruiz on [[Q, A^T], [A, 0]] (Eq. scaled-problem)
    k_fill_d<<<grid_m(), kBlock, 0, s_>>>(Dc_, m_, 1.0);
    k_fill_d<<<grid_n(), kBlock, 0, s_>>>(Dx_, n_, 1.0);
    for (int sw = 0; sw < prm.ruiz_outer; ++sw) {
      if (m_)
        with_G(gA_, [&](auto GG) {
          k_oruiz_rows<decltype(GG)::value><<<grid_rows_g(m_, gA_), kBlock, 0, s_>>>(Ad_, Dc_, Dx_, scm_[0]);
        });
      with_G(gN_, [&](auto GG) {
        k_oruiz_cols<decltype(GG)::value><<<grid_rows_g(n_, gN_), kBlock, 0, s_>>>(Atd_, Hd_, Dc_, Dx_, scn_[0]);
      });
      if (m_) k_ruiz_apply<<<grid_m(), kBlock, 0, s_>>>(Dc_, scm_[0], m_);
      k_ruiz_apply<<<grid_n(), kBlock, 0, s_>>>(Dx_, scn_[0], n_);
    }
    PDNQP_CK(cudaGetLastError());
    if (m_) {
      k_scale_csr<<<grid_m(), kBlock, 0, s_>>>(m_, arp, aci, av_, Dc_, Dx_, 1.0);
      k_scale_csr<<<grid_n(), kBlock, 0, s_>>>(n_, atrp, atci, atv_, Dx_, Dc_, 1.0);
    }
    k_scale_csr<<<grid_n(), kBlock, 0, s_>>>(n_, qrp, qci, qv_, Dx_, Dx_, 1.0);
    k_scale_vec<<<grid_n(), kBlock, 0, s_>>>(c_, Dx_, n_, 0, 1.0);
    // objective scalar c_s = 1 / max(1, ||Dx Q Dx||_inf, ||Dx c||_inf)
    double qn, cn;
    {
      int nb = grid_rows_g(n_, gN_);
      with_G(gN_, [&](auto GG) { k_rowabs_max<decltype(GG)::value><<<nb, kBlock, 0, s_>>>(Hd_, part_); });
      PDNQP_TRY(reduce_to_host(1, nb, 1u, &qn));
      nb = grid_n();
      k_absmax<<<nb, kBlock, 0, s_>>>(c_, n_, part_);
      PDNQP_TRY(reduce_to_host(1, nb, 1u, &cn));
    }
    cs_ = prm.ruiz_outer >= 0 ? 1.0 / std::max(1.0, std::max(qn, cn)) : 1.0;
    k_mul_scalar<<<grid_for(nnzH_, kBlock), kBlock, 0, s_>>>(qv_, nnzH_, cs_);
    k_mul_scalar<<<grid_n(), kBlock, 0, s_>>>(c_, n_, cs_);
    {
      int nb = grid_rows_g(n_, gN_);
      with_G(gN_, [&](auto GG) { k_rowabs_max<decltype(GG)::value><<<nb, kBlock, 0, s_>>>(Hd_, part_); });
      PDNQP_TRY(reduce_to_host(1, nb, 1u, &qnorm_));
    }
    // bounds in scaled coordinates
    k_scale_vec<<<grid_n(), kBlock, 0, s_>>>(lxd_, Dx_, n_, 1, 1.0);
    k_scale_vec<<<grid_n(), kBlock, 0, s_>>>(uxd_, Dx_, n_, 1, 1.0);
    if (m_) {
      k_scale_vec<<<grid_m(), kBlock, 0, s_>>>(lcd_, Dc_, m_, 0, 1.0);
      k_scale_vec<<<grid_m(), kBlock, 0, s_>>>(ucd_, Dc_, m_, 0, 1.0);
    }
    PDNQP_CK(cudaGetLastError());
    // ---- gamma (Eq. R-choice): two Lanczos starts, the smaller estimate.
    double l1, l2;
    PDNQP_TRY(lanczos(prm.lanczos_steps, 1ULL, &l1));
    PDNQP_TRY(lanczos(prm.lanczos_steps, 2ULL, &l2));
    lam_min_ = std::min(l1, l2);
    gamma_ = prm.gamma_override > 0 ? prm.gamma_override
                                     : 1.0 / (std::max(0.0, -lam_min_) + prm.delta_gamma * std::max(1.0, qnorm_));
    // H = Qbar + gamma^-1 I
    k_add_diag<<<grid_n(), kBlock, 0, s_>>>(n_, qdiag_, qv_, 1.0 / gamma_);
    PDNQP_CK(cudaGetLastError());
    // ---- T-typed copies and inner vectors
    PDNQP_TRY(alloc_T(P.a_rp));
    PDNQP_CK(cudaStreamSynchronize(s_));
    ready_ = true;
    return 0;
  }

  int lanczos(int steps, unsigned long long seed, double *out) {
    const long long n = n_;
    if (n == 0) {
      *out = 0.0;
      return 0;
    }
    const int k = (int)std::min<long long>(std::min(steps, 79), n);  // part_lz() holds 80 rows
    if (!V_) PDNQP_TRY(dalloc(&V_, (size_t)(k + 1) * n));
    if (!hdev_) PDNQP_TRY(dalloc(&hdev_, 256));
    double *w = scn_[1];
    std::vector<double> al(k + 1, 0.0), be(k + 1, 0.0);
    // Hd currently holds the scaled Q (gamma not yet added).
    k_start_vector<<<grid_n(), kBlock, 0, s_>>>(V_, n, seed);
    double nrm;
    PDNQP_TRY(dot(V_, V_, &nrm));
    k_scale_into<<<grid_n(), kBlock, 0, s_>>>(V_, V_, 1.0 / std::sqrt(nrm), n);
    int used = 0;
    const int nbd = grid_n();
    for (int j = 0; j < k; ++j) {
      double *vj = V_ + (long long)j * n;
      with_G(gN_, [&](auto GG) {
        k_spmv<decltype(GG)::value><<<grid_rows_g(n, gN_), kBlock, 0, s_>>>(Hd_, vj, w);
      });
      PDNQP_TRY(dot(w, vj, &al[j]));
      used = j + 1;
      k_lanczos_axpy<<<grid_n(), kBlock, 0, s_>>>(w, vj, j > 0 ? V_ + (long long)(j - 1) * n : nullptr, al[j],
                                                   j > 0 ? be[j - 1] : 0.0, n);
      for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        dim3 grid(nbd, j + 1);
        k_multidot<<<grid, kBlock, 0, s_>>>(V_, n, w, part_lz());
        k_reduce_rows<<<j + 1, 32, 0, s_>>>(part_lz(), j + 1, nbd, 0u, hdev_);
        k_multiaxpy<<<grid_n(), kBlock, 0, s_>>>(V_, n, hdev_, j + 1, w);
      }
      double b2;
      PDNQP_TRY(dot(w, w, &b2));
      const double b = std::sqrt(b2);
      be[j] = b;
      if (j == k - 1) break;
      if (b <= 1e-12 * (std::fabs(al[j]) + (j > 0 ? be[j - 1] : 0.0) + 1e-300)) break;
      k_scale_into<<<grid_n(), kBlock, 0, s_>>>(V_ + (long long)(j + 1) * n, w, 1.0 / b, n);
    }
    PDNQP_CK(cudaGetLastError());
    *out = tridiag_min(al, be, used);
    return 0;
  }

  // Smallest eigenvalue of the Lanczos tridiagonal by Sturm-count bisection.
  static double tridiag_min(const std::vector<double> &a, const std::vector<double> &b, int k) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < k; ++i) {
      const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < k - 1 ? std::fabs(b[i]) : 0.0);
      lo = std::min(lo, a[i] - r);
      hi = std::max(hi, a[i] + r);
    }
    auto below = [&](double x) {
      int cnt = 0;
      double dd = 1.0;
      for (int i = 0; i < k; ++i) {
        dd = (a[i] - x) - (i > 0 ? b[i - 1] * b[i - 1] / dd : 0.0);
        if (dd == 0.0) dd = -1e-300;
        if (dd < 0.0) ++cnt;
      }
      return cnt;
    };
    for (int it = 0; it < 400; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (below(mid) >= 1) hi = mid;
      else lo = mid;
    }
    return 0.5 * (lo + hi);
  }

  double *part_lz() { return lzpart_ ? lzpart_ : (dalloc(&lzpart_, (size_t)80 * kMaxBlocks), lzpart_); }

  int dot(const double *a, const double *b, double *out) {
    const int nb = grid_n();
    k_dot<<<nb, kBlock, 0, s_>>>(a, b, n_, part_);
    return reduce_to_host(1, nb, 0u, out);
  }

  int alloc_T(const std::vector<int> &arp) {
    Dev<T> &d = d_;
    d.n = n_;
    d.m = m_;
    d.mE = mE_;
    if (std::is_same<T, double>::value) {
      d.H = {Hd_.nrows, Hd_.rp, Hd_.ci, (const T *)Hd_.val};
      d.A = {Ad_.nrows, Ad_.rp, Ad_.ci, (const T *)Ad_.val};
      d.At = {Atd_.nrows, Atd_.rp, Atd_.ci, (const T *)Atd_.val};
    } else {
      T *hv, *av, *atv;
      PDNQP_TRY(dalloc(&hv, nnzH_));
      PDNQP_TRY(dalloc(&av, nnzA_));
      PDNQP_TRY(dalloc(&atv, nnzA_));
      k_to_T<T><<<grid_for(nnzH_, kBlock), kBlock, 0, s_>>>(hv, qv_, nnzH_);
      if (nnzA_) {
        k_to_T<T><<<grid_for(nnzA_, kBlock), kBlock, 0, s_>>>(av, av_, nnzA_);
        k_to_T<T><<<grid_for(nnzA_, kBlock), kBlock, 0, s_>>>(atv, atv_, nnzA_);
      }
      d.H = {Hd_.nrows, Hd_.rp, Hd_.ci, hv};
      d.A = {Ad_.nrows, Ad_.rp, Ad_.ci, av};
      d.At = {Atd_.nrows, Atd_.rp, Atd_.ci, atv};
    }
    PDNQP_TRY(split_long_rows(arp));
    for (int b = 0; b < 2; ++b) {
      PDNQP_TRY(dalloc(&d.x[b], n_));
      PDNQP_TRY(dalloc(&d.Hx[b], n_));
      PDNQP_TRY(dalloc(&d.Aty[b], n_));
      PDNQP_TRY(dalloc(&d.xbar[b], n_));
      PDNQP_TRY(dalloc(&d.Hxbar[b], n_));
      PDNQP_TRY(dalloc(&d.y[b], m_));
      PDNQP_TRY(dalloc(&d.s[b], m_));
      PDNQP_TRY(dalloc(&d.r[b], m_));
      PDNQP_TRY(dalloc(&d.Bw[b], m_));
      PDNQP_TRY(dalloc(&d.ybar[b], m_));
      PDNQP_TRY(dalloc(&d.sbar[b], m_));
      PDNQP_TRY(dalloc(&d.rbar[b], m_));
      PDNQP_CK(cudaMemsetAsync(d.s[b], 0, sizeof(T) * std::max(m_, 1), s_));
      PDNQP_CK(cudaMemsetAsync(d.sbar[b], 0, sizeof(T) * std::max(m_, 1), s_));
    }
    T **nv[] = {&d.qx, &d.qx0, &d.Hxb, &d.Atyb, &d.lx, &d.ux, &d.taux, &d.itaux, &d.ex, &d.xst, &d.Atybar};
    for (T **p : nv) PDNQP_TRY(dalloc(p, n_));
    T **mv[] = {&d.qs, &d.qr, &d.hp, &d.h, &d.Bwb, &d.ls, &d.us, &d.eta, &d.taus, &d.taur, &d.ieta, &d.itaus,
                &d.itaur, &d.es, &d.er, &d.dy, &d.yst, &d.sst, &d.rst, &d.Bwbar};
    for (T **p : mv) {
      PDNQP_TRY(dalloc(p, m_));
      PDNQP_CK(cudaMemsetAsync(*p, 0, sizeof(T) * std::max(m_, 1), s_));
    }
    PDNQP_TRY(dalloc(&x64_, n_));
    PDNQP_TRY(dalloc(&y64_, m_));
    PDNQP_TRY(dalloc(&sb64_, m_));
    PDNQP_TRY(dalloc(&rb64_, m_));
    PDNQP_CK(cudaMemsetAsync(sb64_, 0, sizeof(double) * std::max(m_, 1), s_));
    PDNQP_CK(cudaMemsetAsync(rb64_, 0, sizeof(double) * std::max(m_, 1), s_));
    PDNQP_CK(cudaMemsetAsync(y64_, 0, sizeof(double) * std::max(m_, 1), s_));
    d.xb = x64_;
    d.yb = y64_;
    d.sb = sb64_;
    d.rb = rb64_;
    d.lam = lam_;
    d.sig = sig_;
    d.part = part_;
    d.st = st_;
    PDNQP_TRY(dalloc(&d.ctr, kCtrWords));
    PDNQP_CK(cudaMemsetAsync(d.ctr, 0, kCtrWords * sizeof(unsigned), s_));
    PDNQP_TRY(dalloc(&d.ptime, 8));
    PDNQP_CK(cudaMemsetAsync(d.ptime, 0, 8 * sizeof(unsigned long long), s_));
    d.hw = 0;
    d.hc = 0;
    PDNQP_CK(cudaGetLastError());
    return 0;
  }

  // Dense coupling rows of A (more than kLongRowMin entries; the kMaxLong
  // longest when there are more): copies of their entries in row order for
  // the split products, and As = A with those rows emptied for the row-wise
  // passes of the trial.  Device-to-device copies of contiguous runs, after
  // the values were scaled and converted.
  int split_long_rows(const std::vector<int> &arp) {
    Dev<T> &d = d_;
    d.nlr = 0;
    d.lr_nnz = 0;
    d.As = d.A;
    d.lr_row = d.lr_ptr = d.lr_ci = nullptr;
    d.lr_val = nullptr;
    d.lr_flag = nullptr;
    d.lr_part = d.lr_acc = nullptr;
    auto len = [&](int j) { return arp[j + 1] - arp[j]; };
    std::vector<int> lr;
    for (int j = 0; j < m_; ++j)
      if (len(j) > kLongRowMin) lr.push_back(j);
    if (lr.empty()) return 0;
    if ((int)lr.size() > kMaxLong) {
      std::stable_sort(lr.begin(), lr.end(), [&](int a, int b) { return len(a) > len(b); });
      lr.resize(kMaxLong);
      std::sort(lr.begin(), lr.end());
    }
    const int nl = (int)lr.size();
    std::vector<int> lptr(nl + 1, 0), srp(m_ + 1, 0);
    std::vector<unsigned char> flag(m_, 0);
    for (int k = 0; k < nl; ++k) {
      lptr[k + 1] = lptr[k] + len(lr[k]);
      flag[lr[k]] = 1;
    }
    for (int j = 0; j < m_; ++j) srp[j + 1] = srp[j] + (flag[j] ? 0 : len(j));
    int *lrow, *lp, *lci, *srpd, *sci;
    unsigned char *lflag;
    T *lval, *sval;
    PDNQP_TRY(upload(&lrow, lr));
    PDNQP_TRY(upload(&lp, lptr));
    PDNQP_TRY(upload(&lflag, flag));
    PDNQP_TRY(upload(&srpd, srp));
    PDNQP_TRY(dalloc(&lci, lptr[nl]));
    PDNQP_TRY(dalloc(&lval, lptr[nl]));
    PDNQP_TRY(dalloc(&sci, srp[m_]));
    PDNQP_TRY(dalloc(&sval, srp[m_]));
    for (int k = 0; k < nl; ++k) {
      const size_t c = (size_t)len(lr[k]);
      PDNQP_CK(cudaMemcpyAsync(lci + lptr[k], d.A.ci + arp[lr[k]], c * sizeof(int), cudaMemcpyDeviceToDevice, s_));
      PDNQP_CK(cudaMemcpyAsync(lval + lptr[k], d.A.val + arp[lr[k]], c * sizeof(T), cudaMemcpyDeviceToDevice, s_));
    }
    // Runs of ordinary rows between the long ones.
    for (int j0 = 0, k = 0; j0 < m_; ++k) {
      const int j1 = k < nl ? lr[k] : m_;
      const size_t c = (size_t)(arp[j1] - arp[j0]);
      if (c) {
        PDNQP_CK(cudaMemcpyAsync(sci + srp[j0], d.A.ci + arp[j0], c * sizeof(int), cudaMemcpyDeviceToDevice, s_));
        PDNQP_CK(cudaMemcpyAsync(sval + srp[j0], d.A.val + arp[j0], c * sizeof(T), cudaMemcpyDeviceToDevice, s_));
      }
      j0 = j1 + 1;
    }
    PDNQP_TRY(dalloc(&d.lr_part, (size_t)kMaxLong * kMaxBlocks));
    PDNQP_TRY(dalloc(&d.lr_acc, 4));
    PDNQP_CK(cudaMemsetAsync(d.lr_acc, 0, 4 * sizeof(double), s_));
    d.nlr = nl;
    d.lr_nnz = lptr[nl];
    d.lr_row = lrow;
    d.lr_ptr = lp;
    d.lr_ci = lci;
    d.lr_val = lval;
    d.lr_flag = lflag;
    d.As = {m_, srpd, sci, sval};
    return 0;
  }

  // ------------------------------------------------------- launchers
  // Tile kernels: one warp per 32 rows and trip, kBlock / 32 warps per block.
  int nb_rows() const { return grid_for(std::max(m_, 1), kBlock); }
  int nb_cols() const { return grid_for(n_, kBlock); }
  void launch_primal() { k_primal<T><<<grid_n(), kBlock, 0, s_>>>(d_); }
  void launch_rows() {
    with_G(gA_, [&](auto GG) { k_rows<T, decltype(GG)::value><<<nb_rows(), kBlock, 0, s_>>>(d_); });
  }
  void launch_cols() {
    with_G(gN_, [&](auto GG) {
      if (d_.hw)
        k_cols<T, decltype(GG)::value, true><<<nb_cols(), kBlock, 0, s_>>>(d_, nb_rows());
      else
        k_cols<T, decltype(GG)::value, false><<<nb_cols(), kBlock, 0, s_>>>(d_, nb_rows());
    });
  }
  // Trial: primal, rows, cols (+ decision in its last block).  Check: rows,
  // cols (+ check decisions in its last block), apply.  The conditional
  // handles travel in the kernels' Dev argument (captured per graph).
  static constexpr int kSlotKernels = 6;
  void launch_trial() {
    launch_primal();
    launch_rows();
    launch_cols();
  }
  void launch_check_group() {
    launch_check(0);
    k_check_apply<T><<<grid_nm(), kBlock, 0, s_>>>(d_);
  }
  void launch_slot() {
    launch_trial();
    launch_check_group();
  }
  // The persistent loop with or without the dense-coupling-row split.
  void (*trials_fn() const)(Dev<T>) { return d_.nlr ? k_trials<T, true> : k_trials<T, false>; }
  // Persistent trial loop: one cooperative launch per slot, grid = the
  // co-resident block count (capped by the work), each launch bracketed by a
  // pair of events so the loop's device time is measured on its own stream.
  int coop_grid(int bps) {
    if (coop_key_ == bps) return coop_nb_;
    coop_key_ = bps;
    coop_nb_ = 0;
    int dev = 0, sms = 0, can = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&can, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !can) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const int smem = (int)stream_smem_bytes<T>();
    if (cudaFuncSetAttribute(trials_fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, trials_fn(), kBlock, smem) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    if (bps > 0) per_sm = std::min(per_sm, bps);
    const int work = std::max(nb_rows(), nb_cols());
    coop_nb_ = std::max(0, std::min(std::min(per_sm * sms, kMaxBlocks), work));
    return coop_nb_;
  }
  int launch_trials_persistent(int nb, int slot) {
    if (!loop_ev_[2 * slot]) {
      PDNQP_CK(cudaEventCreate(&loop_ev_[2 * slot]));
      PDNQP_CK(cudaEventCreate(&loop_ev_[2 * slot + 1]));
    }
    PDNQP_CK(cudaEventRecord(loop_ev_[2 * slot], s_));
    void *args[] = {(void *)&d_};
    PDNQP_CK(cudaLaunchCooperativeKernel((const void *)trials_fn(), dim3(nb), dim3(kBlock), args,
                                         stream_smem_bytes<T>(), s_));
    PDNQP_CK(cudaEventRecord(loop_ev_[2 * slot + 1], s_));
    return 0;
  }
  void launch_check(int mode) {
    with_G(gA_, [&](auto GG) { k_check_rows<T, decltype(GG)::value><<<nb_rows(), kBlock, 0, s_>>>(d_, mode); });
    with_G(gN_, [&](auto GG) {
      if (d_.hw)
        k_check_cols<T, decltype(GG)::value, true><<<nb_cols(), kBlock, 0, s_>>>(d_, mode, nb_rows());
      else
        k_check_cols<T, decltype(GG)::value, false><<<nb_cols(), kBlock, 0, s_>>>(d_, mode, nb_rows());
    });
  }

  // Row-binning autotuner of the graph form: replays the row kernel and the
  // column kernel (each captured as a graph of kTuneReps launches, on the
  // state of the first inner solve) for every lanes-per-row choice, and makes
  // the fastest the default of this handle.  Replays write trial buffers only
  // and restore the device state.
  int autotune_g() {
    static constexpr int kTuneReps = 20;
    const int cand[3] = {4, 8, 16};
    const int gA = gA_, gN = gN_;
    double best[2] = {INFINITY, INFINITY};
    int pick[2] = {gA, gN};
    for (int which = 0; which < 2; ++which)
      for (int g : cand) {
        if (which == 0) gN_ = g; else gA_ = g;
        PDNQP_TRY(replay(which | 8, 1));  // first capture and launch (not timed)
        PDNQP_TRY(replay(which | 8, kTuneReps));
        if (last_replay_ms_ < best[which]) {
          best[which] = last_replay_ms_;
          pick[which] = g;
        }
        gA_ = gA;
        gN_ = gN;
      }
    gN0_ = pick[0];
    gA0_ = pick[1];
    tuned_ = true;
    return 0;
  }
  int tuned_g(int which) const override { return which == 0 ? gN0_ : gA0_; }

  // Lanes per CSR row: parameter override, else the mean-row-length choice of setup.
  void apply_g(const Params &prm) {
    gA_ = prm.g_rows > 0 ? prm.g_rows : gA0_;
    gN_ = prm.g_cols > 0 ? prm.g_cols : gN0_;
  }

  int build_graph(int chunk, int cond) {
    if (gexec_ && chunk == graph_chunk_ && gA_ == graph_gA_ && gN_ == graph_gN_ && cond == graph_cond_) return 0;
    graph_cond_ = cond;
    use_cond_ = cond != 0;
    graph_gA_ = gA_;
    graph_gN_ = gN_;
    if (gexec_) {
      cudaGraphExecDestroy(gexec_);
      gexec_ = nullptr;
    }
    graph_chunk_ = chunk;
    if (use_cond_ && build_graph_cond(chunk) == 0) return 0;
    use_cond_ = false;  // conditional nodes unavailable: unrolled slots
    cudaGetLastError();
    cudaGraph_t g;
    PDNQP_CK(cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < chunk; ++k) launch_slot();
    PDNQP_CK(cudaStreamEndCapture(s_, &g));
    cudaError_t e = cudaGraphInstantiate(&gexec_, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      last_err_ = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e);
      return PDNQP_ERR_CUDA;
    }
    return 0;
  }

  // Device-driven loop: [begin] -> WHILE(hw) { primal, rows, cols, decide,
  // IF(hc) { check-rows, check-cols, check-final, check-apply } }.  decide
  // sets hw (continue while running and fewer than `chunk` trials ran in this
  // launch) and hc (a check is due); check-final updates hw.  Every launch
  // therefore ends after at most `chunk` trials.
  int build_graph_cond(int chunk) {
    cudaGraph_t g = nullptr;
    if (cudaGraphCreate(&g, 0) != cudaSuccess) return -1;
    auto fail = [&]() {
      d_.hw = 0;
      d_.hc = 0;
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(s_, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t junk;
        cudaStreamEndCapture(s_, &junk);
        if (junk) cudaGraphDestroy(junk);
      }
      cudaGraphDestroy(g);
      cudaGetLastError();
      return -1;
    };
    cudaGraphConditionalHandle hw, hc;
    if (cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return fail();
    if (cudaGraphConditionalHandleCreate(&hc, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) return fail();
    if (cudaStreamBeginCaptureToGraph(s_, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fail();
    k_loop_begin<<<1, 1, 0, s_>>>(st_, (long long)chunk);
    if (cudaStreamEndCapture(s_, &g) != cudaSuccess) return fail();
    cudaGraphNode_t begin;
    size_t nn = 1;
    if (cudaGraphGetNodes(g, &begin, &nn) != cudaSuccess || nn != 1) return fail();
    cudaGraphNodeParams wp = {};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = hw;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    if (cudaGraphAddNode(&wnode, g, &begin, nullptr, 1, &wp) != cudaSuccess) return fail();
    cudaGraph_t body = wp.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(s_, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fail();
    d_.hw = hw;
    d_.hc = hc;
    launch_trial();
    cudaStreamCaptureStatus cst;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    if (cudaStreamGetCaptureInfo(s_, &cst, nullptr, nullptr, &deps, nullptr, &ndeps) != cudaSuccess) return fail();
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hc;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    if (cudaGraphAddNode(&inode, body, deps, nullptr, ndeps, &ip) != cudaSuccess) return fail();
    if (cudaStreamUpdateCaptureDependencies(s_, &inode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
      return fail();
    cudaGraph_t body_out = nullptr;
    if (cudaStreamEndCapture(s_, &body_out) != cudaSuccess) return fail();
    cudaGraph_t cbody = ip.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(s_, cbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fail();
    launch_check_group();
    d_.hw = 0;
    d_.hc = 0;
    cudaGraph_t cbody_out = nullptr;
    if (cudaStreamEndCapture(s_, &cbody_out) != cudaSuccess) return fail();
    if (cudaGraphInstantiate(&gexec_, g, 0) != cudaSuccess) return fail();
    cudaGraphDestroy(g);
    return 0;
  }

  // ----------------------------------------------------- solve state
  // Initial point, multipliers, penalties (Sec. 3.2.1 and the QPALM rule).
  int start_point(const Params &prm) {
    DevState S;
    memset(&S, 0, sizeof(S));
    S.status = ST_IDLE;
    S.cur = 0;
    PDNQP_CK(cudaMemcpyAsync(st_, &S, sizeof(S), cudaMemcpyHostToDevice, s_));
    if (has_x0_) PDNQP_CK(cudaMemcpyAsync(dx0_, h_x0_.data(), sizeof(double) * n_, cudaMemcpyHostToDevice, s_));
    if (has_l0_) PDNQP_CK(cudaMemcpyAsync(dl0_, h_l0_.data(), sizeof(double) * m_, cudaMemcpyHostToDevice, s_));
    k_init_x<<<grid_n(), kBlock, 0, s_>>>(n_, has_x0_ ? dx0_ : nullptr, Dx_, lxd_, uxd_, x64_, z_);
    if (m_) k_init_lambda<<<grid_m(), kBlock, 0, s_>>>(m_, lam_, has_l0_ ? dl0_ : nullptr, Dc_, cs_, y64_);
    // f(x0) and the constraint violation for sigma0
    double ob[2];
    {
      const int nb = nb_cols();
      with_G(gN_, [&](auto GG) {
        k_objective<T, decltype(GG)::value><<<nb, kBlock, 0, s_>>>(d_, Hd_, c_, 1.0 / gamma_);
      });
      PDNQP_TRY(reduce_to_host(2, nb, 0u, ob));
    }
    double dist2 = 0.0;
    if (m_) {
      const int nb = nb_rows();
      with_G(gA_, [&](auto GG) {
        k_init_rows<T, decltype(GG)::value><<<nb, kBlock, 0, s_>>>(d_, Ad_, lcd_, ucd_, lam_, sig_, rprev_, 0);
      });
      PDNQP_TRY(reduce_to_host(1, nb, 0u, &dist2));
    }
    const double f0 = 0.5 * ob[0] + ob[1];
    double s0 = prm.sigma_init * std::max(1.0, std::fabs(f0)) / std::max(1.0, 0.5 * dist2);
    s0 = std::min(1e4, std::max(1e-4, s0));
    sigma0_ = s0;
    if (m_) {
      k_fill_d<<<grid_m(), kBlock, 0, s_>>>(sig_, m_, s0);
      with_G(gA_, [&](auto GG) {
        k_init_rows<T, decltype(GG)::value><<<nb_rows(), kBlock, 0, s_>>>(d_, Ad_, lcd_, ucd_, lam_, sig_, rprev_, 1);
      });
    }
    PDNQP_CK(cudaGetLastError());
    omega_ = 1.0;
    trials_ = accepted_ = restarts_ = rebases_ = 0;
    return 0;
  }

  // a0: setup of one inner solve (Algorithm 4 lines "warm start" and "inner scaling").
  int inner_setup(const Params &prm, double dta, double dtr, long long k_in, long long pause_at, int ignore) {
    const double ginv = 1.0 / gamma_;
    // Base point of this solve (FP64) and zero corrections.
    if (m_) k_base_rows<T><<<grid_m(), kBlock, 0, s_>>>(d_, Ad_, lcd_, ucd_, sb64_, rb64_);
    with_G(gN_, [&](auto GG) {
      k_base_cols<T, decltype(GG)::value><<<nb_cols(), kBlock, 0, s_>>>(d_, Hd_, Atd_, c_, z_, lxd_, uxd_, ginv);
    });
    k_iscale_init<T><<<grid_nm(), kBlock, 0, s_>>>(d_);
    for (int sw = 0; sw < prm.ruiz_inner; ++sw) {
      with_G(gN_, [&](auto GG) {
        k_iruiz_cols<T, decltype(GG)::value><<<nb_cols(), kBlock, 0, s_>>>(d_, scn_[0]);
      });
      if (m_)
        with_G(gA_, [&](auto GG) {
          k_iruiz_rows<T, decltype(GG)::value><<<nb_rows(), kBlock, 0, s_>>>(d_, scm_[0], scm_[1], scm_[2]);
        });
      k_iruiz_update<T><<<grid_nm(), kBlock, 0, s_>>>(d_, scn_[0], scm_[0], scm_[1], scm_[2]);
    }
    with_G(gN_, [&](auto GG) { k_mw_cols<T, decltype(GG)::value><<<nb_cols(), kBlock, 0, s_>>>(d_, scn_[0]); });
    if (m_) with_G(gA_, [&](auto GG) { k_my_rows<T, decltype(GG)::value><<<nb_rows(), kBlock, 0, s_>>>(d_, scn_[0]); });
    k_inner_init<T><<<grid_nm(), kBlock, 0, s_>>>(d_);
    // Device state of this solve (the host holds every field it needs; the
    // iterates sit in buffer 0 between inner solves).
    DevState &S = *hst_;
    memset(&S, 0, sizeof(S));
    S.cur = 0;
    S.status = ST_IDLE;
    S.accepted = 0;
    S.acur = 0;
    S.check_due = 0;
    S.restart_flag = 0;
    S.ret_avg = 0;
    S.ignore_conv = ignore;
    S.start_status = batch_ ? ST_READY : ST_RUNNING;
    S.t = 0;
    S.t_total = 0;
    S.trials = trials_;
    S.accepted_all = accepted_;
    S.restarts = restarts_;
    S.rej = 0;
    S.k_in = k_in;
    S.pause_at = pause_at;
    S.k_chk = prm.k_chk;
    S.rej_limit = prm.rej_limit;
    S.kappa = 1.0;
    S.omega = omega_;
    S.alpha_acc = 1.0;
    S.dta = dta;
    S.dtr = dtr;
    S.shrink = prm.kappa_shrink;
    S.beta_suff = prm.beta_suff;
    S.beta_nec = prm.beta_nec;
    S.beta_art = prm.beta_art;
    PDNQP_CK(cudaMemcpyAsync(st_, &S, sizeof(S), cudaMemcpyHostToDevice, s_));
    launch_check(1);  // its last block sets the restart metric of the start and the running status
    launches_ += 9 + 3LL * prm.ruiz_inner;
    PDNQP_CK(cudaGetLastError());
    return 0;
  }

  int read_state(DevState *S) {
    PDNQP_CK(cudaMemcpyAsync(hst_, st_, sizeof(DevState), cudaMemcpyDeviceToHost, s_));
    PDNQP_CK(cudaMemcpyAsync(hfault_, d_.ctr + kCtrBar + kBarFault, sizeof(unsigned), cudaMemcpyDeviceToHost, s_));
    PDNQP_CK(cudaStreamSynchronize(s_));
    *S = *hst_;
    if (*hfault_) {
      // A grid barrier of the persistent loop gave up waiting: the launch ended
      // early and the iterates are not usable.
      cudaMemsetAsync(d_.ctr, 0, kCtrWords * sizeof(unsigned), s_);
      cudaStreamSynchronize(s_);
      last_err_ = "persistent trial loop: grid barrier timed out";
      return PDNQP_ERR_CUDA;
    }
    return 0;
  }

  // Runs graph chunks until the device status leaves RUNNING.
  int run_until_stop(const Params &prm, DevState *S, double t0) {
    if (batch_) {
      PDNQP_CK(cudaStreamSynchronize(s_));  // the setup of this inner solve is complete
      const int r = batch_->run_inner(batch_idx_, S, t0 + prm.time_limit);
      if (r < 0) {
        last_err_ = "batched form: the scheduler stopped";
        return r;
      }
      *hst_ = *S;
      return r;
    }
    const int nbp = prm.persistent ? coop_grid(prm.loop_blocks_per_sm) : 0;
    if (nbp > 0) {
      // Persistent loop: batches of slots [trial loop, check rows, check cols
      // (+ decisions), check apply]; a batch runs at most `per` trials, after
      // which the host reads the state once.
      const long long kc = std::max<long long>(1, prm.k_chk);
      const long long per = std::max<long long>(prm.chunk, 8 * kc);
      const int R = (int)std::min<long long>(kMaxLoopSlots, per / kc + 1);
      for (;;) {
        k_loop_begin<<<1, 1, 0, s_>>>(st_, per);
        for (int r = 0; r < R; ++r) {
          PDNQP_TRY(launch_trials_persistent(nbp, r));
          launch_check_group();
        }
        PDNQP_CK(cudaGetLastError());
        launches_ += 1 + 4LL * R;
        loop_launches_ += R;
        const long long tr_before = hst_->trials;
        PDNQP_TRY(read_state(S));
        for (int r = 0; r < R; ++r) {
          float ms = 0.f;
          PDNQP_CK(cudaEventElapsedTime(&ms, loop_ev_[2 * r], loop_ev_[2 * r + 1]));
          loop_seconds_ += 1e-3 * ms;
        }
        loop_trials_ += S->trials - tr_before;
        if (S->status != ST_RUNNING) return 0;
        if (seconds_since(t0) > prm.time_limit) return 1;
      }
    }
    PDNQP_TRY(build_graph(prm.chunk, prm.cond_graph));
    long long tr0 = -1, ac0 = 0;
    for (;;) {
      PDNQP_CK(cudaGraphLaunch(gexec_, s_));
      PDNQP_TRY(read_state(S));
      if (use_cond_) {
        // 3 kernels per trial, 3 more per check, 1 loop-begin kernel per launch.
        if (tr0 < 0) tr0 = trials_, ac0 = accepted_;
        launches_ += 1;
        launches_ += 3 * (S->trials - tr0) + 3 * ((S->accepted_all / std::max<long long>(1, prm.k_chk)) -
                                                  (ac0 / std::max<long long>(1, prm.k_chk)));
        tr0 = S->trials;
        ac0 = S->accepted_all;
      } else {
        launches_ += (long long)prm.chunk * kSlotKernels;
      }
      if (S->status != ST_RUNNING) return 0;
      if (seconds_since(t0) > prm.time_limit) return 1;
    }
  }

  static double now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
  }
  static double seconds_since(double t0) { return now() - t0; }

  int finish_inner(const DevState &S) {
    trials_ = S.trials;
    accepted_ = S.accepted_all;
    restarts_ = S.restarts;
    omega_ = S.omega;
    // Outer x and inner y = base + correction (current point or converged average).
    k_finish<T><<<grid_nm(), kBlock, 0, s_>>>(d_, x64_, y64_, (S.status == ST_CONVERGED && S.ret_avg) ? 1 : 0);
    PDNQP_CK(cudaGetLastError());
    DevState Z = S;
    Z.cur = 0;
    Z.status = ST_IDLE;
    PDNQP_CK(cudaMemcpyAsync(st_, &Z, sizeof(Z), cudaMemcpyHostToDevice, s_));
    return 0;
  }

  // Outer residuals; update = 1 also applies the multiplier update first.
  int outer_residuals(int update, double *q) {
    const double ginv = 1.0 / gamma_;
    launches_ += 4;
    double a[12] = {0}, b[12] = {0};
    const int nbr = nb_rows(), nbc = nb_cols();
    if (m_) {
      with_G(gA_, [&](auto GG) {
        k_outer_rows<T, decltype(GG)::value><<<nbr, kBlock, 0, s_>>>(d_, Ad_, lcd_, ucd_, Dc_, lam_, sig_, rcur_,
                                                                      update);
      });
      k_reduce_rows<<<12, 32, 0, s_>>>(part_, 12, nbr, OUT_MAXMASK, dred_);
    }
    // A' lambda uses the updated multipliers: launched after the row kernel.
    with_G(gN_, [&](auto GG) {
      k_outer_cols<T, decltype(GG)::value><<<nbc, kBlock, 0, s_>>>(d_, Hd_, Atd_, c_, lxd_, uxd_, Dx_, lam_, z_,
                                                                    ginv, cs_);
    });
    k_reduce_rows<<<12, 32, 0, s_>>>(part_ + 12 * kMaxBlocks, 12, nbc, OUT_MAXMASK, dred_ + 12);
    PDNQP_CK(cudaGetLastError());
    PDNQP_CK(cudaMemcpyAsync(hred_.data(), dred_, sizeof(double) * 24, cudaMemcpyDeviceToHost, s_));
    PDNQP_CK(cudaStreamSynchronize(s_));
    if (m_)
      for (int k = 0; k < 12; ++k) a[k] = hred_[k];
    for (int k = 0; k < 12; ++k) b[k] = hred_[12 + k];
    for (int k = 0; k < 12; ++k) q[k] = ((OUT_MAXMASK >> k) & 1u) ? std::max(a[k], b[k]) : a[k] + b[k];
    return 0;
  }

  int solve_impl(double ea, double er, Params &prm) {
    if (!ready_) return PDNQP_ERR_STATE;
    const double t0 = now();
    if (gamma_pending_ > 0) {
      PDNQP_TRY(regamma(gamma_pending_));
      gamma_pending_ = 0;
    }
    launches_ = 0;
    loop_seconds_ = 0.0;
    loop_trials_ = 0;
    loop_launches_ = 0;
    PDNQP_CK(cudaMemsetAsync(d_.ptime, 0, 8 * sizeof(unsigned long long), s_));
    double t_setup = 0.0, t_inner = 0.0;
    apply_g(prm);
    PDNQP_TRY(start_point(prm));
    double dta = 1.0, dtr = 1.0, eak = 1.0, erk = 1.0;
    int status = PDNQP_ITER_LIMIT;
    long long k;
    double q[12];
    trace_.clear();
    ctrl_used_ = ctrl_fallbacks_ = 0;
    // Anderson state of this solve.
    aa_cap_ = std::max(2, std::min(5, prm.anderson_mem));
    aa_len_ = aa_head_ = 0;
    bool aa_applied = false, aa_off = false, aa_pok_prev = false;
    double aa_rel_prev = INFINITY;
    if (prm.anderson && !aa_u_) {
      const size_t D = (size_t)m_ + n_;
      PDNQP_TRY(dalloc(&aa_u_, kAaRing * D));
      PDNQP_TRY(dalloc(&aa_g_, kAaRing * D));
      PDNQP_TRY(dalloc(&aa_out_, D));
    }
    bool ctrl_last = false;
    double rel_prev = 0.0, f0_prev = 0.0, f1_prev = 0.0;
    unsigned long long rng = (unsigned long long)prm.ctrl_seed * 0x9E3779B97F4A7C15ULL + 0x1234567ULL;
    for (k = 0; k < prm.k_out; ++k) {
      const long long acc_before = accepted_, rst_before = restarts_;
      if (seconds_since(t0) > prm.time_limit) {
        status = PDNQP_TIME_LIMIT;
        break;
      }
      const long long left = prm.iter_budget - accepted_;
      if (left <= 0) {
        status = PDNQP_ITER_LIMIT;
        break;
      }
      const double ts0 = now();
      PDNQP_CK(cudaMemcpyAsync(xprev_, x64_, sizeof(double) * n_, cudaMemcpyDeviceToDevice, s_));
      if (prm.anderson) PDNQP_TRY(aa_stage_u());
      PDNQP_TRY(inner_setup(prm, dta, dtr, std::min(prm.k_in, left), -1, 0));
      if (prm.autotune && !tuned_ && (!prm.persistent || !coop_grid(prm.loop_blocks_per_sm))) {
        PDNQP_TRY(autotune_g());
        apply_g(prm);
      }
      PDNQP_CK(cudaStreamSynchronize(s_));
      const double ts1 = now();
      t_setup += ts1 - ts0;
      DevState S;
      int tl = 0;
      PDNQP_TRY(tl = run_until_stop(prm, &S, t0));
      t_inner += now() - ts1;
      if (tl == 1) {
        // time limit inside the inner solve: stop the device loop
        PDNQP_TRY(read_state(&S));
        PDNQP_TRY(finish_inner(S));
        status = PDNQP_TIME_LIMIT;
        ++k;
        break;
      }
      PDNQP_TRY(finish_inner(S));
      if (S.status == ST_NUMERICAL_ERROR) {
        // FP32-bulk: a run of rejections down to the limit means that the
        // FP32 products H x_tr, A'y_tr (rounded to about 6e-8 of |H||dx|)
        // no longer resolve the step differences of Eq. adaptive-condition.
        // finish_inner has folded the last accepted point into the FP64 base,
        // so the next outer iteration re-warm-starts there (as after the
        // inner iteration limit) with zero corrections, which restores the
        // FP32 resolution; a rebase that follows one without any accepted
        // iteration in between is a true numerical error.  Non-finite sums
        // (rej below the limit) are always a numerical error.
        const bool floor = sizeof(T) == 4 && S.rej >= S.rej_limit && S.t_total > 0;
        if (floor) {
          ++rebases_;
          continue;
        }
        status = PDNQP_NUMERICAL_ERROR;
        ++k;
        break;
      }
      if (S.status == ST_ITER_LIMIT) continue;
      // Multiplier update + outer residuals (Eqs. practical-multiplier-update, outer-residuals).
      if (m_) PDNQP_CK(cudaMemcpyAsync(lamprev_, lam_, sizeof(double) * m_, cudaMemcpyDeviceToDevice, s_));
      PDNQP_TRY(outer_residuals(1, q));
      const double rps = q[0], sps = std::max(1.0, q[1]), rpu = q[2], spu = std::max(1.0, q[3]), rn = q[4];
      const double rds = q[5], rdu = q[7], sdu = std::max(1.0, q[8]), dxz = q[9];
      if (rpu <= ea + er * spu && rdu <= ea + er * sdu) {
        status = PDNQP_SOLVED;
        ++k;
        break;
      }
      {
        int inf = 0;
        PDNQP_TRY(inf = infeasibility(prm.eps_inf > 0.0 ? prm.eps_inf : 1e-5));
        if (inf) {
          status = inf;
          ++k;
          break;
        }
      }
      // Eq. penalty-trigger-eq; penalties grow only while the primal part of
      // Eq. outer-termination fails (scaled or original data).
      const int grow = !(rpu <= ea + er * spu && rps <= ea + er * sps);
      if (m_)
        k_sigma_update<<<grid_m(), kBlock, 0, s_>>>(m_, mE_, sig_, lam_, rcur_, rprev_, prm.theta_sigma, grow, rn,
                                                    prm.delta_sigma, prm.sigma_max);
      // Eq. inner-tolerance-factor.
      const double ratio = rds > 0.0 ? std::min(1.0, (dxz / gamma_) / rds) : 1.0;
      double rho = prm.rho_in_max - (prm.rho_in_max - prm.rho_in_min) * ratio;
      {
        // Learned controller (with the rules as fallback and judge) and the
        // trace of this outer iteration.
        const double rel_now = std::max(rpu / (1.0 + spu), rdu / (1.0 + sdu));
        auto lg = [](double v) { return std::log10(std::max(v, 1e-300)); };
        double f[16];
        f[0] = lg(rpu / (1.0 + spu));
        f[1] = lg(rdu / (1.0 + sdu));
        f[2] = lg(rps / sps);
        f[3] = lg(rds);
        f[4] = trace_.empty() ? 0.0 : f[0] - f0_prev;
        f[5] = trace_.empty() ? 0.0 : f[1] - f1_prev;
        f[6] = lg(dta);
        f[7] = std::log10(1.0 + (double)(accepted_ - acc_before));
        f[8] = std::log10(1.0 + (double)(restarts_ - rst_before));
        f[9] = lg(omega_);
        f[10] = lg(gamma_);
        f[11] = lg(dxz / gamma_);
        f[12] = rho;
        f[13] = ratio;
        f[14] = std::log10(1.0 + (double)k);
        f[15] = grow ? 1.0 : 0.0;
        for (double &v : f) v = std::min(30.0, std::max(-30.0, v));
        const double span = prm.rho_in_max - prm.rho_in_min;
        double fr = span > 0.0 ? (rho - prm.rho_in_min) / span : 0.5;
        fr = std::min(1.0 - 1e-3, std::max(1e-3, fr));
        const double ar[2] = {std::log(fr / (1.0 - fr)), 0.0};
        double a[2] = {ar[0], ar[1]};
        bool used = false, moved = false;
        if (prm.controller && has_ctrl_) {
          if (ctrl_last && rel_now > rel_prev) {
            ++ctrl_fallbacks_;  // the last proposal made the KKT residual worse: the rules decide
          } else {
            float fx[16], fy[2] = {0.f, 0.f};
            for (int i = 0; i < 16; ++i) fx[i] = (float)f[i];
            PDNQP_CK(cudaMemcpyAsync(ctrl_x_, fx, sizeof(fx), cudaMemcpyHostToDevice, s_));
            if (pdnqp_mlp_forward(ctrl_w_, ctrl_x_, 1, ctrl_y_, nullptr, s_) != 0) {
              last_err_ = std::string("controller: ") + pdnqp_mlp_last_error();
              return PDNQP_ERR_CUDA;
            }
            PDNQP_CK(cudaMemcpyAsync(fy, ctrl_y_, sizeof(fy), cudaMemcpyDeviceToHost, s_));
            PDNQP_CK(cudaStreamSynchronize(s_));
            if (std::isfinite(fy[0]) && std::isfinite(fy[1])) {
              // The network proposes corrections to the rules' actions.
              a[0] = ar[0] + fy[0];
              a[1] = ar[1] + fy[1];
              used = moved = true;
              ++ctrl_used_;
            } else {
              ++ctrl_fallbacks_;
            }
          }
        }
        if (prm.ctrl_explore > 0.0) {
          for (double &v : a) v += prm.ctrl_explore * gauss(rng);
          moved = true;
        }
        if (moved) {
          rho = prm.rho_in_min + span / (1.0 + std::exp(-a[0]));
          omega_ *= std::exp(std::min(1.0, std::max(-1.0, a[1])));
        }
        trace_.push_back((double)k);
        trace_.push_back(rel_now);
        trace_.push_back((double)(accepted_ - acc_before));
        for (double v : f) trace_.push_back(v);
        trace_.push_back(ar[0]);
        trace_.push_back(ar[1]);
        trace_.push_back(a[0]);
        trace_.push_back(a[1]);
        trace_.push_back(used ? 1.0 : 0.0);
        ctrl_last = used;
        rel_prev = rel_now;
        f0_prev = f[0];
        f1_prev = f[1];
      }
      dta = std::max(dta * rho, prm.tol_floor * ea);
      dtr = std::max(dtr * rho, prm.tol_floor * er);
      // FP32-bulk: the inner residuals are formed from FP32 iterates and
      // cached products, whose rounding is about 2^-24 of the terms that
      // make up the scales of Eq. inner-scales; a relative inner tolerance
      // below a few units of it cannot be certified (the inner solve would
      // run to K_in on rounding noise), so delta_r stops at 8 units.
      if (sizeof(T) == 4) dtr = std::max(dtr, kFp32RelTolFloor);
      // Eq. center-update / center-tolerance-update.
      if (rps <= eak + erk * sps) {
        PDNQP_CK(cudaMemcpyAsync(z_, x64_, sizeof(double) * n_, cudaMemcpyDeviceToDevice, s_));
        eak = std::max(eak * prm.rho_z, ea);
        erk = std::max(erk * prm.rho_z, er);
      }
      // Anderson step (active while the primal termination test holds on this
      // and the previous outer iteration; a step that raised the relative KKT
      // residual or lost primal feasibility switches it off for the solve).
      if (prm.anderson) {
        const double rel = std::max(rpu / (1.0 + spu), rdu / (1.0 + sdu));
        const int primal_ok = !grow;
        if (aa_applied && (rel > aa_rel_prev || !primal_ok)) aa_off = true;
        const bool active = primal_ok && aa_pok_prev && !aa_off;
        aa_applied = false;
        if (!active) {
          aa_len_ = 0;
        } else {
          PDNQP_TRY(aa_push_g());
          int stepped = 0;
          PDNQP_TRY(stepped = aa_try_step());
          aa_applied = stepped != 0;
        }
        aa_rel_prev = rel;
        aa_pok_prev = primal_ok;
      }
      PDNQP_CK(cudaGetLastError());
    }
    // Result in the original coordinates.
    PDNQP_TRY(outer_residuals(0, q));
    k_unscale<double><<<grid_nm(), kBlock, 0, s_>>>(x64_, Dx_, n_, lam_, Dc_, m_, cs_, xo_, lo_);
    PDNQP_CK(cudaGetLastError());
    PDNQP_CK(cudaStreamSynchronize(s_));
    res_.status = status;
    res_.rp = q[2];
    res_.sp = std::max(1.0, q[3]);
    res_.rd = q[7];
    res_.sd = std::max(1.0, q[8]);
    res_.rel_kkt = std::max(res_.rp / (1.0 + res_.sp), res_.rd / (1.0 + res_.sd));
    res_.obj = (0.5 * q[10] + q[11]) / cs_;
    res_.outer = k;
    res_.inner = accepted_;
    res_.trials = trials_;
    res_.restarts = restarts_;
    res_.rebases = rebases_;
    res_.passes = 3 * trials_ + 2 * (accepted_ / std::max(1, prm.k_chk));
    res_.seconds = seconds_since(t0);
    res_.launches = launches_;
    res_.inner_seconds = t_inner;
    res_.setup_seconds = t_setup;
    res_.loop_seconds = loop_seconds_;
    res_.loop_trials = loop_trials_;
    res_.loop_blocks = coop_nb_;
    res_.loop_launches = loop_launches_;
    res_.ctrl_used = ctrl_used_;
    res_.ctrl_fallbacks = ctrl_fallbacks_;
    {
      unsigned long long pt[8];
      PDNQP_CK(cudaMemcpy(pt, d_.ptime, sizeof(pt), cudaMemcpyDeviceToHost));
      for (int k = 0; k < 6; ++k) res_.loop_phase_seconds[k] = 1e-9 * (double)pt[k];
    }
    solved_once_ = true;
    return status;
  }

  // Anderson acceleration (Sec. "Anderson acceleration"), Type-II on u =
  // (lambda, z) with the last anderson_mem pairs (u_k, G(u_k)) in a ring on
  // the device: the sums go through k_aa_dots, the small normal equations
  // (dF'dF + 1e-12 tr I) g = dF'f_k are solved here by Gaussian elimination,
  // and the step is skipped when it would move G(u_k) by more than
  // 10 ||f_k||_2.  Returns 1 when (lambda, z) were replaced.
  int aa_try_step() {
    const int L = aa_len_, nc = L - 1;
    if (nc < 1) return 0;
    const long long D = (long long)m_ + n_;
    const int nb = grid_for(D, kBlock);
    const int nq = nc * nc + nc + 1;
    switch (nc) {
      case 1: k_aa_dots<1><<<nb, kBlock, 0, s_>>>(aa_u_, aa_g_, aa_head_, kAaRing, D, part_); break;
      case 2: k_aa_dots<2><<<nb, kBlock, 0, s_>>>(aa_u_, aa_g_, aa_head_, kAaRing, D, part_); break;
      case 3: k_aa_dots<3><<<nb, kBlock, 0, s_>>>(aa_u_, aa_g_, aa_head_, kAaRing, D, part_); break;
      default: k_aa_dots<4><<<nb, kBlock, 0, s_>>>(aa_u_, aa_g_, aa_head_, kAaRing, D, part_); break;
    }
    double q[21];
    PDNQP_TRY(reduce_to_host(nq, nb, 0u, q));
    double M[16], r[4], g[4] = {0.0, 0.0, 0.0, 0.0};
    double tr = 0.0;
    for (int a = 0; a < nc; ++a) {
      for (int b = 0; b < nc; ++b) M[a * nc + b] = q[a * nc + b];
      r[a] = q[nc * nc + a];
      tr += M[a * nc + a];
    }
    const double fn = q[nc * nc + nc];
    if (!(tr > 0.0) || !std::isfinite(tr)) return 0;
    for (int a = 0; a < nc; ++a) M[a * nc + a] += 1e-12 * tr;
    for (int c = 0; c < nc; ++c) {
      const double piv = M[c * nc + c];
      if (!(piv > 0.0)) return 0;
      for (int rr = c + 1; rr < nc; ++rr) {
        const double f = M[rr * nc + c] / piv;
        for (int k = c; k < nc; ++k) M[rr * nc + k] -= f * M[c * nc + k];
        r[rr] -= f * r[c];
      }
    }
    for (int c = nc - 1; c >= 0; --c) {
      double v = r[c];
      for (int k = c + 1; k < nc; ++k) v -= M[c * nc + k] * g[k];
      g[c] = v / M[c * nc + c];
    }
    k_aa_apply<<<nb, kBlock, 0, s_>>>(aa_g_, aa_head_, kAaRing, nc, D, g[0], g[1], g[2], g[3], aa_out_, part_);
    double sn = 0.0;
    PDNQP_TRY(reduce_to_host(1, nb, 0u, &sn));
    launches_ += 2;
    if (!(sn <= 100.0 * fn)) return 0;
    if (m_) PDNQP_CK(cudaMemcpyAsync(lam_, aa_out_, sizeof(double) * m_, cudaMemcpyDeviceToDevice, s_));
    PDNQP_CK(cudaMemcpyAsync(z_, aa_out_ + m_, sizeof(double) * n_, cudaMemcpyDeviceToDevice, s_));
    return 1;
  }
  // Ring of kAaRing = 6 slots (logical pair a at (head + a) % 6, at most
  // aa_cap_ <= 5 pairs), so the slot after the last pair is always free: it
  // receives u, the point this outer iteration starts from.
  int aa_stage_u() {
    const long long D = (long long)m_ + n_;
    const int slot = (aa_head_ + aa_len_) % kAaRing;
    double *u = aa_u_ + (size_t)slot * D;
    if (m_) PDNQP_CK(cudaMemcpyAsync(u, lam_, sizeof(double) * m_, cudaMemcpyDeviceToDevice, s_));
    PDNQP_CK(cudaMemcpyAsync(u + m_, z_, sizeof(double) * n_, cudaMemcpyDeviceToDevice, s_));
    return 0;
  }
  // Appends G(u) = (lambda, z) to the staged slot (dropping the oldest pair when full).
  int aa_push_g() {
    const long long D = (long long)m_ + n_;
    const int slot = (aa_head_ + aa_len_) % kAaRing;
    double *g = aa_g_ + (size_t)slot * D;
    if (m_) PDNQP_CK(cudaMemcpyAsync(g, lam_, sizeof(double) * m_, cudaMemcpyDeviceToDevice, s_));
    PDNQP_CK(cudaMemcpyAsync(g + m_, z_, sizeof(double) * n_, cudaMemcpyDeviceToDevice, s_));
    if (aa_len_ == aa_cap_) {
      aa_head_ = (aa_head_ + 1) % kAaRing;
    } else {
      ++aa_len_;
    }
    return 0;
  }

  // Sec. "Infeasibility detection" on the scaled problem (see k_inf_rows /
  // k_inf_cols): PDNQP_PRIMAL_INFEASIBLE when lambda^{k+1} - lambda^k is an
  // approximate Farkas certificate, PDNQP_DUAL_INFEASIBLE when x^{k+1} - x^k
  // is an approximate recession direction of descent, else 0.
  int infeasibility(double eps) {
    const double ginv = 1.0 / gamma_;
    k_sub<<<grid_n(), kBlock, 0, s_>>>(n_, x64_, xprev_, dxv_);
    double a[4] = {0.0, 0.0, 0.0, 0.0}, b[7];
    if (m_) {
      const int nb = nb_rows();
      with_G(gA_, [&](auto GG) {
        k_inf_rows<T, decltype(GG)::value><<<nb, kBlock, 0, s_>>>(d_, Ad_, lcd_, ucd_, lam_, lamprev_, dxv_);
      });
      PDNQP_TRY(reduce_to_host(4, nb, INF_R_MAXMASK, a));
    }
    {
      const int nb = nb_cols();
      with_G(gN_, [&](auto GG) {
        k_inf_cols<T, decltype(GG)::value><<<nb, kBlock, 0, s_>>>(d_, Hd_, Atd_, c_, lxd_, uxd_, lam_,
                                                                  m_ ? lamprev_ : lam_, dxv_, ginv);
      });
      PDNQP_TRY(reduce_to_host(7, nb, INF_C_MAXMASK, b));
    }
    launches_ += m_ ? 3 : 2;
    const double nl = a[3], nx = b[6];
    if (nl > 0.0 && std::max(a[0], b[0]) <= eps * nl && a[1] + b[1] < -eps * nl) return PDNQP_PRIMAL_INFEASIBLE;
    if (nx > 0.0 && std::max(a[2], b[2]) <= eps * nx &&
        (b[3] < -eps * nx * nx || (b[5] <= eps * nx && b[4] < -eps * nx)))
      return PDNQP_DUAL_INFEASIBLE;
    return 0;
  }

  int regamma(double g) {
    // Replace gamma: H = Qbar + g^-1 I (undo the previous shift).
    k_add_diag<<<grid_n(), kBlock, 0, s_>>>(n_, qdiag_, qv_, 1.0 / g - 1.0 / gamma_);
    gamma_ = g;
    if (!std::is_same<T, double>::value)
      k_to_T<T><<<grid_for(nnzH_, kBlock), kBlock, 0, s_>>>((T *)d_.H.val, qv_, nnzH_);
    PDNQP_CK(cudaGetLastError());
    return 0;
  }

  int snapshot(const DevState &S, double *o) {
    const long long n = n_, m = m_, mI = m_ - mE_, dw = n + mI + m;
    if (!snapbuf_) PDNQP_TRY(dalloc(&snapbuf_, (size_t)(2 * (dw + m))));
    k_totals<T><<<grid_nm(), kBlock, 0, s_>>>(d_, snapbuf_);
    PDNQP_CK(cudaGetLastError());
    PDNQP_CK(cudaMemcpyAsync(o, snapbuf_, sizeof(double) * 2 * (dw + m), cudaMemcpyDeviceToHost, s_));
    PDNQP_CK(cudaStreamSynchronize(s_));
    double *sc = o + 2 * (dw + m);
    sc[0] = S.omega;
    sc[1] = S.kappa;
    sc[2] = (double)S.t;
    sc[3] = (double)S.t_total;
    sc[4] = (double)S.trials;
    sc[5] = (double)S.restarts;
    sc[6] = S.k_restart;
    sc[7] = S.k_last;
    return 0;
  }

  int debug_impl(Params &prm, int nck, const int64_t *ck, double *snap) {
    if (!ready_) return PDNQP_ERR_STATE;
    if (gamma_pending_ > 0) {
      PDNQP_TRY(regamma(gamma_pending_));
      gamma_pending_ = 0;
    }
    apply_g(prm);
    PDNQP_TRY(start_point(prm));
    const long long len = 2 * ((long long)n_ + (m_ - mE_) + m_ + m_) + 8;
    int got = 0;
    PDNQP_TRY(inner_setup(prm, 1.0, 1.0, (long long)4e18, nck > 0 ? ck[0] : -1, 1));
    const double t0 = now();
    while (got < nck) {
      DevState S;
      int tl = 0;
      PDNQP_TRY(tl = run_until_stop(prm, &S, t0));
      if (tl == 1 || S.status != ST_PAUSED) break;
      if (S.accepted) {  // materialise the pending running averages before reading them
        k_average<T><<<grid_nm(), kBlock, 0, s_>>>(d_);
        PDNQP_CK(cudaGetLastError());
      }
      PDNQP_TRY(snapshot(S, snap + (long long)got * len));
      ++got;
      S.status = ST_RUNNING;
      S.pause_at = got < nck ? ck[got] : -1;
      PDNQP_CK(cudaMemcpyAsync(st_, &S, sizeof(S), cudaMemcpyHostToDevice, s_));
    }
    DevState S;
    PDNQP_TRY(read_state(&S));
    (void)S;
    return got;
  }

 public:
  // members
  cudaStream_t s_;
  std::string last_err_;
  std::vector<void *> allocs_;
  int n_ = 0, m_ = 0, mE_ = 0;
  long long nnzA_ = 0, nnzH_ = 0;
  int gA_ = 8, gN_ = 8, gA0_ = 8, gN0_ = 8, graph_gA_ = 0, graph_gN_ = 0;
  Mat<double> Hd_{}, Ad_{}, Atd_{};
  double *qv_ = nullptr, *av_ = nullptr, *atv_ = nullptr;
  int *qdiag_ = nullptr;
  double *c_ = nullptr, *lxd_ = nullptr, *uxd_ = nullptr, *lcd_ = nullptr, *ucd_ = nullptr;
  double *Dc_ = nullptr, *Dx_ = nullptr, *lam_ = nullptr, *sig_ = nullptr, *rprev_ = nullptr, *rcur_ = nullptr;
  double *z_ = nullptr, *xo_ = nullptr, *lo_ = nullptr, *dx0_ = nullptr, *dl0_ = nullptr;
  double *x64_ = nullptr, *y64_ = nullptr, *sb64_ = nullptr, *rb64_ = nullptr, *snapbuf_ = nullptr;
  double *scn_[2] = {nullptr, nullptr}, *scm_[3] = {nullptr, nullptr, nullptr};
  double *V_ = nullptr, *hdev_ = nullptr, *lzpart_ = nullptr;
  double *part_ = nullptr, *dred_ = nullptr;
  std::vector<double> hred_;
  DevState *st_ = nullptr, *hst_ = nullptr;
  Dev<T> d_{};
  cudaGraphExec_t gexec_ = nullptr;
  cudaEvent_t replay_ev_[2] = {nullptr, nullptr};
  static constexpr int kMaxLoopSlots = 32;
  cudaEvent_t loop_ev_[2 * kMaxLoopSlots] = {};
  double loop_seconds_ = 0.0;  // device time of the persistent trial-loop launches
  long long loop_launches_ = 0;
  long long loop_trials_ = 0;  // trials they ran
  int coop_key_ = -1, coop_nb_ = 0;
  unsigned *hfault_ = nullptr;
  // learned controller
  double *xprev_ = nullptr, *lamprev_ = nullptr, *dxv_ = nullptr;  // infeasibility tests
  double *aa_u_ = nullptr, *aa_g_ = nullptr, *aa_out_ = nullptr;    // Anderson ring and step
  static constexpr int kAaRing = 6;
  int aa_cap_ = 5, aa_len_ = 0, aa_head_ = 0;
  uint16_t *ctrl_w_ = nullptr;
  float *ctrl_w32_ = nullptr, *ctrl_x_ = nullptr, *ctrl_y_ = nullptr;
  bool has_ctrl_ = false;
  std::vector<double> trace_;
  long long ctrl_used_ = 0, ctrl_fallbacks_ = 0;
  // Standard normal draw (splitmix64 counter stream, Box-Muller).
  static double gauss(unsigned long long &s) {
    auto next = [&s]() {
      unsigned long long z = (s += 0x9E3779B97F4A7C15ULL);
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
      z ^= z >> 31;
      return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    const double u1 = next(), u2 = next();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
  float last_replay_ms_ = 0.f;
  int graph_chunk_ = 0;
  bool use_cond_ = true;  // device-driven WHILE/IF graph (else unrolled slots)
  int graph_cond_ = -1;
  double cs_ = 1.0, qnorm_ = 0.0, gamma_ = 1.0, lam_min_ = 0.0, sigma0_ = 1.0, omega_ = 1.0;
  double gamma_pending_ = 0.0;
  long long trials_ = 0, accepted_ = 0, restarts_ = 0, launches_ = 0;
  long long rebases_ = 0;  // FP32-bulk inner solves ended at the rejection limit and re-based
  BatchHook *batch_ = nullptr;  // batched form: the scheduler that runs this solver's inner solves
  int batch_idx_ = -1;
  bool ready_ = false, solved_once_ = false, has_x0_ = false, has_l0_ = false, own_stream_ = false;
  bool tuned_ = false;
  std::vector<double> h_x0_, h_l0_;
  Result res_;
};

}  // namespace pdq
