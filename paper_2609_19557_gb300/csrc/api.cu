// C ABI of the PDNQP solver (include/pdnqp.h): input validation, row
// classification (equality rows first), CSR construction on the host (Q with
// an explicit diagonal, A^T by counting sort), and dispatch to the FP64 or
// FP32-bulk device solver.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <numeric>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/pdnqp.h"
#include "solver.cuh"

using pdq::HostProblem;
using pdq::Params;
using pdq::Result;
using pdq::SolverBase;

struct pdnqp {
  SolverBase *solver = nullptr;
  int n = 0, m = 0, mE = 0;
  std::vector<int> perm;
  Params prm;
  std::string err;
  cudaStream_t stream = nullptr;
  int device = 0;
  int precision = PDNQP_FP64;
  int64_t nnzq = 0;
  double t_prepare = 0.0, t_setup = 0.0;  // wall time of pdnqp_create's host preparation and device setup
  // FP32-bulk handles keep the prepared host problem, from which an FP64
  // solver is built the first time a solve has to continue in FP64.
  std::unique_ptr<HostProblem> host;
  SolverBase *solver64 = nullptr;
  bool escalated = false;  // the last solve finished in the FP64 solver
  Result r32;              // counters of that solve's FP32 phase
  std::vector<double> start_x, start_l;  // the start point given by pdnqp_set_start (internal row order)
  // Fused batched form: totals of the last pdnqp_solve_batch over this handle's precision group.
  double batch_graph_seconds = 0.0;
  long long batch_graph_launches = 0, batch_kernel_launches = 0;
  int batch_size = 0;
};

static thread_local std::string g_err;

static int fail(pdnqp_t *h, int code, const std::string &msg) {
  if (h) h->err = msg;
  g_err = msg;
  return code;
}

static double clean_bound(double v) {
  if (v >= 1e20) return INFINITY;
  if (v <= -1e20) return -INFINITY;
  return v;
}

// ---------------------------------------------------------------------------
// Host preparation, parallel over row ranges (std::thread; the results do
// not depend on the number of threads).
// ---------------------------------------------------------------------------
static int host_threads() {
  const unsigned hc = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(hc == 0 ? 1u : hc, 32u));
}

// Runs f(lo, hi, t) on [0, n) split into contiguous ranges, one per thread.
template <typename F>
static void parallel_for(long long n, F f) {
  const int T = (int)std::min<long long>(host_threads(), std::max<long long>(1, n / 4096));
  if (T <= 1) {
    f(0LL, n, 0);
    return;
  }
  std::vector<std::thread> th;
  th.reserve(T);
  for (int t = 0; t < T; ++t) {
    const long long lo = n * t / T, hi = n * (t + 1) / T;
    th.emplace_back([=, &f] { f(lo, hi, t); });
  }
  for (auto &x : th) x.join();
}

// First error found by any thread (the one on the lowest row wins, so the
// message does not depend on the thread count).
struct ErrSlot {
  std::mutex mu;
  long long row = -1;
  int code = 0;
  std::string msg;
  void set(long long r, int c, std::string m) {
    std::lock_guard<std::mutex> g(mu);
    if (row < 0 || r < row) {
      row = r;
      code = c;
      msg = std::move(m);
    }
  }
};

// Validates a host CSR matrix; returns its rows with columns sorted.
static int read_csr(const pdnqp_csr *M, int rows, int cols, const char *name, std::vector<int> &rp,
                    std::vector<int> &ci, std::vector<double> &v, std::string &msg) {
  if (!M) {
    msg = std::string(name) + " is NULL";
    return PDNQP_ERR_ARG;
  }
  if (M->n_rows != rows || M->n_cols != cols) {
    msg = std::string(name) + " has the wrong shape";
    return PDNQP_ERR_ARG;
  }
  if (M->nnz < 0 || M->nnz > 2147483647LL || (M->nnz > 0 && (!M->col_idx || !M->val)) || !M->row_ptr) {
    msg = std::string(name) + ": bad nnz or NULL arrays";
    return PDNQP_ERR_ARG;
  }
  if (M->row_ptr[0] != 0 || M->row_ptr[rows] != M->nnz) {
    msg = std::string(name) + ": row_ptr[0] must be 0 and row_ptr[n_rows] == nnz";
    return PDNQP_ERR_ARG;
  }
  for (int i = 0; i < rows; ++i)
    if (M->row_ptr[i + 1] < M->row_ptr[i]) {
      msg = std::string(name) + ": row_ptr not monotone";
      return PDNQP_ERR_ARG;
    }
  rp.assign(M->row_ptr, M->row_ptr + rows + 1);
  ci.resize(M->nnz);
  v.resize(M->nnz);
  ErrSlot err;
  parallel_for(rows, [&](long long lo, long long hi, int) {
    std::vector<std::pair<int, double>> tmp;
    for (long long i = lo; i < hi; ++i) {
      const int b = M->row_ptr[i], e = M->row_ptr[i + 1];
      bool sorted = true;
      for (int k = b; k < e; ++k) {
        const int c = M->col_idx[k];
        if (c < 0 || c >= cols) {
          err.set(i, PDNQP_ERR_ARG, std::string(name) + ": column index out of range");
          return;
        }
        if (!std::isfinite(M->val[k])) {
          err.set(i, PDNQP_ERR_BOUNDS, std::string(name) + ": non-finite value");
          return;
        }
        if (k > b && c <= M->col_idx[k - 1]) sorted = false;
      }
      if (sorted) {  // strictly increasing: no sort, no duplicates
        std::copy(M->col_idx + b, M->col_idx + e, ci.begin() + b);
        std::copy(M->val + b, M->val + e, v.begin() + b);
        continue;
      }
      tmp.clear();
      for (int k = b; k < e; ++k) tmp.push_back({M->col_idx[k], M->val[k]});
      std::sort(tmp.begin(), tmp.end(), [](const std::pair<int, double> &x, const std::pair<int, double> &y) {
        return x.first < y.first;
      });
      for (size_t k = 1; k < tmp.size(); ++k)
        if (tmp[k].first == tmp[k - 1].first) {
          err.set(i, PDNQP_ERR_ARG, std::string(name) + ": duplicate entry");
          return;
        }
      for (size_t k = 0; k < tmp.size(); ++k) {
        ci[b + k] = tmp[k].first;
        v[b + k] = tmp[k].second;
      }
    }
  });
  if (err.code) {
    msg = err.msg;
    return err.code;
  }
  return 0;
}

// Symmetry of a square CSR with sorted rows: every entry (i, j, v) has the
// entry (j, i, v) (binary search in row j).
static bool symmetric(int n, const std::vector<int> &rp, const std::vector<int> &ci, const std::vector<double> &v) {
  std::atomic<bool> ok(true);
  parallel_for(n, [&](long long lo, long long hi, int) {
    for (long long i = lo; i < hi && ok.load(std::memory_order_relaxed); ++i)
      for (int k = rp[i]; k < rp[i + 1]; ++k) {
        const int j = ci[k];
        const int *b = ci.data() + rp[j], *e = ci.data() + rp[j + 1];
        const int *f = std::lower_bound(b, e, (int)i);
        if (f == e || *f != (int)i || v[f - ci.data()] != v[k]) {
          ok = false;
          return;
        }
      }
  });
  return ok;
}

// Transpose of a CSR (rows sorted by column in the result): per-thread
// column counts over contiguous row ranges, offsets thread by thread within
// each column, then each thread scatters its rows in order.
static void transpose(int rows, int cols, const std::vector<int> &rp, const std::vector<int> &ci,
                      const std::vector<double> &v, std::vector<int> &trp, std::vector<int> &tci,
                      std::vector<double> &tv) {
  trp.assign(cols + 1, 0);
  tci.resize(ci.size());
  tv.resize(v.size());
  const int T = (int)std::min<long long>(host_threads(), std::max<long long>(1, rows / 4096));
  std::vector<std::vector<int>> cnt(T, std::vector<int>(cols, 0));
  auto range = [&](int t, long long &lo, long long &hi) {
    lo = (long long)rows * t / T;
    hi = (long long)rows * (t + 1) / T;
  };
  {
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t)
      th.emplace_back([&, t] {
        long long lo, hi;
        range(t, lo, hi);
        for (long long i = lo; i < hi; ++i)
          for (int k = rp[i]; k < rp[i + 1]; ++k) cnt[t][ci[k]]++;
      });
    for (auto &x : th) x.join();
  }
  // offsets: column c starts at trp[c]; within it, thread t's entries follow
  // thread t-1's (column totals and per-thread offsets in parallel over
  // column ranges, the prefix over columns in between)
  std::vector<int> tot(cols, 0);
  parallel_for(cols, [&](long long c0, long long c1, int) {
    for (long long c = c0; c < c1; ++c) {
      int a = 0;
      for (int t = 0; t < T; ++t) a += cnt[t][c];
      tot[c] = a;
    }
  });
  for (int c = 0; c < cols; ++c) trp[c + 1] = trp[c] + tot[c];
  parallel_for(cols, [&](long long c0, long long c1, int) {
    for (long long c = c0; c < c1; ++c) {
      int acc = trp[c];
      for (int t = 0; t < T; ++t) {
        const int k = cnt[t][c];
        cnt[t][c] = acc;
        acc += k;
      }
    }
  });
  {
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t)
      th.emplace_back([&, t] {
        long long lo, hi;
        range(t, lo, hi);
        std::vector<int> &pos = cnt[t];
        for (long long i = lo; i < hi; ++i)
          for (int k = rp[i]; k < rp[i + 1]; ++k) {
            const int d = pos[ci[k]]++;
            tci[d] = (int)i;
            tv[d] = v[k];
          }
      });
    for (auto &x : th) x.join();
  }
}

static int prepare(const pdnqp_csr *Q, const double *c, const pdnqp_csr *A, const double *l_c, const double *u_c,
                   const double *l_x, const double *u_x, HostProblem &P, std::string &msg) {
  if (!Q || !c || !l_x || !u_x) {
    msg = "NULL argument";
    return PDNQP_ERR_ARG;
  }
  const int n = Q->n_rows;
  const int m = A ? A->n_rows : 0;
  if (n <= 0 || Q->n_cols != n) {
    msg = "Q must be square with n >= 1";
    return PDNQP_ERR_NOT_SYMMETRIC;
  }
  if (m < 0 || (m > 0 && (!l_c || !u_c))) {
    msg = "row bounds missing";
    return PDNQP_ERR_ARG;
  }
  P.n = n;
  P.m = m;
  std::vector<int> qrp, qci;
  std::vector<double> qv;
  int rc = read_csr(Q, n, n, "Q", qrp, qci, qv, msg);
  if (rc) return rc;
  if (!symmetric(n, qrp, qci, qv)) {
    msg = "Q is not symmetric with both triangles stored";
    return PDNQP_ERR_NOT_SYMMETRIC;
  }
  // Q with an explicit diagonal entry in every row: new row lengths, offsets,
  // then a parallel fill.
  P.q_rp.assign(n + 1, 0);
  P.q_diag.assign(n, 0);
  {
    std::vector<char> has(n, 0);
    parallel_for(n, [&](long long lo, long long hi, int) {
      for (long long i = lo; i < hi; ++i) {
        const int *b = qci.data() + qrp[i], *e = qci.data() + qrp[i + 1];
        const int *f = std::lower_bound(b, e, (int)i);
        has[i] = (f != e && *f == (int)i) ? 1 : 0;
      }
    });
    for (int i = 0; i < n; ++i) P.q_rp[i + 1] = P.q_rp[i] + (qrp[i + 1] - qrp[i]) + (has[i] ? 0 : 1);
    P.q_ci.resize(P.q_rp[n]);
    P.q_v.resize(P.q_rp[n]);
    parallel_for(n, [&](long long lo, long long hi, int) {
      for (long long i = lo; i < hi; ++i) {
        int o = P.q_rp[i];
        bool done = false;
        for (int k = qrp[i]; k < qrp[i + 1]; ++k) {
          if (!done && qci[k] >= (int)i) {
            P.q_diag[i] = o;
            if (qci[k] != (int)i) {
              P.q_ci[o] = (int)i;
              P.q_v[o] = 0.0;
              ++o;
            }
            done = true;
          }
          P.q_ci[o] = qci[k];
          P.q_v[o] = qv[k];
          ++o;
        }
        if (!done) {
          P.q_diag[i] = o;
          P.q_ci[o] = (int)i;
          P.q_v[o] = 0.0;
        }
      }
    });
  }
  P.c.assign(c, c + n);
  P.lx.resize(n);
  P.ux.resize(n);
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(c[i])) {
      msg = "c has a non-finite entry";
      return PDNQP_ERR_BOUNDS;
    }
    const double lo = clean_bound(l_x[i]), hi = clean_bound(u_x[i]);
    if (std::isnan(lo) || std::isnan(hi) || lo > hi || lo == INFINITY || hi == -INFINITY) {
      msg = "variable bounds: need l_x <= u_x (no NaN)";
      return PDNQP_ERR_BOUNDS;
    }
    P.lx[i] = lo;
    P.ux[i] = hi;
  }
  // Rows: classify and order equality rows first (stable).
  std::vector<int> arp, aci;
  std::vector<double> av;
  if (m > 0) {
    rc = read_csr(A, m, n, "A", arp, aci, av, msg);
    if (rc) return rc;
  }
  P.perm.clear();
  std::vector<double> lo(m), hi(m);
  for (int j = 0; j < m; ++j) {
    lo[j] = clean_bound(l_c[j]);
    hi[j] = clean_bound(u_c[j]);
    if (std::isnan(lo[j]) || std::isnan(hi[j]) || lo[j] > hi[j] || lo[j] == INFINITY || hi[j] == -INFINITY) {
      msg = "row bounds: need l_c <= u_c (no NaN, no infinite equality)";
      return PDNQP_ERR_BOUNDS;
    }
  }
  for (int j = 0; j < m; ++j)
    if (lo[j] == hi[j]) P.perm.push_back(j);
  P.mE = (int)P.perm.size();
  for (int j = 0; j < m; ++j)
    if (lo[j] != hi[j]) P.perm.push_back(j);
  P.a_rp.assign(m + 1, 0);
  P.lc.resize(m);
  P.uc.resize(m);
  for (int r = 0; r < m; ++r) {
    const int j = P.perm[r];
    P.a_rp[r + 1] = P.a_rp[r] + (arp[j + 1] - arp[j]);
    P.lc[r] = lo[j];
    P.uc[r] = hi[j];
  }
  P.a_ci.resize(P.a_rp[m]);
  P.a_v.resize(P.a_rp[m]);
  parallel_for(m, [&](long long r0, long long r1, int) {
    for (long long r = r0; r < r1; ++r) {
      const int j = P.perm[r];
      std::copy(aci.begin() + arp[j], aci.begin() + arp[j + 1], P.a_ci.begin() + P.a_rp[r]);
      std::copy(av.begin() + arp[j], av.begin() + arp[j + 1], P.a_v.begin() + P.a_rp[r]);
    }
  });
  transpose(m, n, P.a_rp, P.a_ci, P.a_v, P.at_rp, P.at_ci, P.at_v);
  return 0;
}

extern "C" {

int pdnqp_create_ex(pdnqp_t **out, const pdnqp_csr *Q, const double *c, const pdnqp_csr *A, const double *l_c,
                    const double *u_c, const double *l_x, const double *u_x, const pdnqp_options *opt) {
  if (!out) return fail(nullptr, PDNQP_ERR_ARG, "out is NULL");
  *out = nullptr;
  pdnqp_options o = {PDNQP_FP64, -1, nullptr};
  if (opt) o = *opt;
  if (o.precision != PDNQP_FP64 && o.precision != PDNQP_FP32_BULK)
    return fail(nullptr, PDNQP_ERR_ARG, "precision must be PDNQP_FP64 or PDNQP_FP32_BULK");
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0)
    return fail(nullptr, PDNQP_ERR_CUDA,
                std::string("no usable CUDA device: ") + (e != cudaSuccess ? cudaGetErrorString(e) : "0 devices"));
  if (o.device >= 0) {
    e = cudaSetDevice(o.device);
    if (e != cudaSuccess) return fail(nullptr, PDNQP_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
  }
  HostProblem P;
  std::string msg;
  const auto t0 = std::chrono::steady_clock::now();
  int rc = prepare(Q, c, A, l_c, u_c, l_x, u_x, P, msg);
  if (rc) return fail(nullptr, rc, msg);
  const auto t1 = std::chrono::steady_clock::now();
  pdnqp_t *h = new (std::nothrow) pdnqp_t();
  if (!h) return fail(nullptr, PDNQP_ERR_OOM, "host allocation failed");
  h->n = P.n;
  h->m = P.m;
  h->mE = P.mE;
  h->perm = P.perm;
  h->stream = (cudaStream_t)o.stream;
  cudaGetDevice(&h->device);
  h->precision = o.precision;
  h->nnzq = (int64_t)P.q_ci.size();
  h->solver = o.precision == PDNQP_FP64 ? pdq::make_solver_f64(h->stream) : pdq::make_solver_f32(h->stream);
  rc = h->solver->setup(P, h->prm, &msg);
  if (rc < 0) {
    fail(nullptr, rc, msg);
    delete h->solver;
    delete h;
    return rc;
  }
  if (o.precision == PDNQP_FP32_BULK) h->host.reset(new (std::nothrow) HostProblem(std::move(P)));
  const auto t2 = std::chrono::steady_clock::now();
  h->t_prepare = std::chrono::duration<double>(t1 - t0).count();
  h->t_setup = std::chrono::duration<double>(t2 - t1).count();
  *out = h;
  return 0;
}

int pdnqp_create(pdnqp_t **out, const pdnqp_csr *Q, const double *c, const pdnqp_csr *A, const double *l_c,
                 const double *u_c, const double *l_x, const double *u_x) {
  return pdnqp_create_ex(out, Q, c, A, l_c, u_c, l_x, u_x, nullptr);
}

void pdnqp_destroy(pdnqp_t *h) {
  if (!h) return;
  cudaSetDevice(h->device);
  delete h->solver;
  delete h->solver64;
  delete h;
}

int pdnqp_solve(pdnqp_t *h, double eps_abs, double eps_rel) {
  if (!h) return fail(nullptr, PDNQP_ERR_ARG, "handle is NULL");
  if (!(eps_abs >= 0) || !(eps_rel >= 0)) return fail(h, PDNQP_ERR_ARG, "tolerances must be >= 0");
  cudaSetDevice(h->device);
  h->escalated = false;
  std::string msg;
  const auto t0 = std::chrono::steady_clock::now();
  int rc = h->solver->solve(eps_abs, eps_rel, h->prm, &msg);
  if (rc < 0) return fail(h, rc, msg);
  const double used = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rc == PDNQP_NUMERICAL_ERROR && h->precision == PDNQP_FP32_BULK && h->prm.escalate && h->host &&
      used < h->prm.time_limit) {
    // FP32 rounding stalls the acceptance test near a tight tolerance: the
    // solve continues in the plain FP64 form from the FP32 form's last point.
    if (!h->solver64) {
      h->solver64 = pdq::make_solver_f64(h->stream);
      const int rs = h->solver64->setup(*h->host, h->prm, &msg);
      if (rs < 0) {
        delete h->solver64;
        h->solver64 = nullptr;
        return fail(h, rs, msg);
      }
    }
    // The FP64 solve starts from the handle's start point, not from the FP32
    // point: it then returns exactly what the plain FP64 form returns (on the
    // n = 50,000 workload at 1e-6 a warm start from the FP32 point was also
    // slower, as the penalties and steps start over).
    Result r32;
    const int rg = h->solver->get(nullptr, nullptr, &r32);
    if (rg < 0) return fail(h, rg, "escalation: reading the FP32 counters failed");
    const int rst = h->solver64->set_start(h->start_x.empty() ? nullptr : h->start_x.data(),
                                           h->start_l.empty() ? nullptr : h->start_l.data());
    if (rst < 0) return fail(h, rst, "escalation: set_start failed");
    Params p64 = h->prm;
    p64.time_limit = h->prm.time_limit - used;
    p64.controller = 0;  // the network's weights belong to the FP32 solver
    rc = h->solver64->solve(eps_abs, eps_rel, p64, &msg);
    if (rc < 0) return fail(h, rc, msg);
    h->escalated = true;
    h->r32 = r32;
  }
  return rc;
}

// The fused batched form: the problems of each precision get one scheduler
// (pdq::BatchBase) that runs all their inner iterations in one launch per
// phase of a captured CUDA graph; every problem's outer iteration runs on a
// host thread of its own (pdnqp_solve, escalation included), which sleeps
// while its inner solve is on the device.  Returns PDNQP_ERR_STATE without
// solving anything when the handles are not all on one device.
static int solve_batch_fused(pdnqp_t *const *hs, int count, double eps_abs, double eps_rel, int *status) {
  const int dev = hs[0]->device;
  for (int i = 0; i < count; ++i)
    if (hs[i]->device != dev) return PDNQP_ERR_STATE;
  cudaSetDevice(dev);
  std::vector<int> keep(count), keep_tune(count);
  for (int i = 0; i < count; ++i) {
    keep[i] = hs[i]->prm.persistent;
    keep_tune[i] = hs[i]->prm.autotune;
    hs[i]->prm.persistent = 0;  // escalated FP64 solves run the graph form: no cooperative launch beside the batch
    hs[i]->prm.autotune = 0;    // the per-handle tuner replays kernels on a running state: not beside the batch
  }
  struct Group {
    std::vector<int> idx;
    std::unique_ptr<pdq::BatchBase> batch;
  };
  Group groups[2];  // FP64, FP32-bulk
  for (int i = 0; i < count; ++i) groups[hs[i]->precision == PDNQP_FP32_BULK ? 1 : 0].idx.push_back(i);
  std::string err;
  int rc = 0;
  for (int g = 0; g < 2 && rc == 0; ++g) {
    Group &G = groups[g];
    if (G.idx.empty()) continue;
    std::vector<SolverBase *> sv;
    std::vector<int> gr, gc;
    for (int i : G.idx) {
      pdnqp_t *h = hs[i];
      sv.push_back(h->solver);
      gr.push_back(h->prm.g_rows > 0 ? h->prm.g_rows : h->solver->tuned_g(1));
      gc.push_back(h->prm.g_cols > 0 ? h->prm.g_cols : h->solver->tuned_g(0));
    }
    const int chunk = hs[G.idx[0]]->prm.batch_chunk;
    G.batch.reset(g ? pdq::make_batch_f32(sv, gr, gc, chunk, &err) : pdq::make_batch_f64(sv, gr, gc, chunk, &err));
    if (!G.batch) rc = PDNQP_ERR_CUDA;
  }
  std::vector<int> rcs(count, 0);
  std::vector<std::string> errs(count);
  if (rc == 0) {
    std::vector<std::thread> workers, schedulers;
    int sched_rc[2] = {0, 0};
    for (int g = 0; g < 2; ++g) {
      Group &G = groups[g];
      if (!G.batch) continue;
      schedulers.emplace_back([&, g, dev] {
        cudaSetDevice(dev);
        sched_rc[g] = groups[g].batch->schedule();
      });
      for (int k = 0; k < (int)G.idx.size(); ++k)
        workers.emplace_back([&, g, k] {
          const int i = groups[g].idx[k];
          rcs[i] = pdnqp_solve(hs[i], eps_abs, eps_rel);
          if (rcs[i] < 0) errs[i] = g_err;
          groups[g].batch->finished(k);
        });
    }
    for (auto &t : workers) t.join();
    for (auto &t : schedulers) t.join();
    for (int g = 0; g < 2; ++g)
      if (groups[g].batch)
        for (int i : groups[g].idx) {
          hs[i]->batch_graph_seconds = groups[g].batch->graph_seconds();
          hs[i]->batch_graph_launches = groups[g].batch->graph_launches();
          hs[i]->batch_kernel_launches = groups[g].batch->kernel_launches();
          hs[i]->batch_size = (int)groups[g].idx.size();
        }
    for (int g = 0; g < 2; ++g)
      if (sched_rc[g] < 0 && rc == 0) {
        rc = sched_rc[g];
        err = groups[g].batch->error();
      }
  }
  for (int g = 0; g < 2; ++g) groups[g].batch.reset();
  for (int i = 0; i < count; ++i) {
    hs[i]->prm.persistent = keep[i];
    hs[i]->prm.autotune = keep_tune[i];
  }
  if (rc < 0) return fail(nullptr, rc, "batch: " + err);
  int worst = 0;
  std::string first;
  for (int i = 0; i < count; ++i) {
    status[i] = rcs[i];
    if (rcs[i] < 0 && worst == 0) {
      worst = rcs[i];
      first = errs[i];
    }
  }
  if (worst < 0) return fail(nullptr, worst, "batch: " + first);
  return 0;
}

int pdnqp_solve_batch(pdnqp_t *const *hs, int count, double eps_abs, double eps_rel, int threads, int *status) {
  if (count < 0 || (count > 0 && (!hs || !status))) return fail(nullptr, PDNQP_ERR_ARG, "bad batch arguments");
  if (!(eps_abs >= 0) || !(eps_rel >= 0)) return fail(nullptr, PDNQP_ERR_ARG, "tolerances must be >= 0");
  for (int i = 0; i < count; ++i) {
    if (!hs[i]) return fail(nullptr, PDNQP_ERR_ARG, "batch handle is NULL");
    for (int k = 0; k < i; ++k)
      if (hs[k] == hs[i]) return fail(nullptr, PDNQP_ERR_ARG, "batch handles must be distinct");
  }
  if (count == 0) return 0;
  if (hs[0]->prm.batch_fused) {
    const int rf = solve_batch_fused(hs, count, eps_abs, eps_rel, status);
    if (rf != PDNQP_ERR_STATE) return rf;  // else: the batch does not fit the fused form
  }
  // Largest problems first, so that the long solves start early.
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long long)hs[a]->n + hs[a]->m > (long long)hs[b]->n + hs[b]->m;
  });
  const int nt = std::max(1, std::min(count, threads > 0 ? threads : 16));
  std::atomic<int> next{0};
  std::vector<int> rcs(count, 0);
  std::mutex err_mu;
  std::string first_err;
  auto work = [&]() {
    for (int k; (k = next.fetch_add(1)) < count;) {
      pdnqp_t *h = hs[order[k]];
      const int keep = h->prm.persistent;
      h->prm.persistent = 0;  // graph form: no concurrent cooperative launches
      const int rc = pdnqp_solve(h, eps_abs, eps_rel);
      h->prm.persistent = keep;
      rcs[order[k]] = rc;
      if (rc < 0) {
        std::lock_guard<std::mutex> lk(err_mu);
        if (first_err.empty()) first_err = g_err;
      }
    }
  };
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(work);
  work();
  for (auto &t : pool) t.join();
  int worst = 0;
  for (int i = 0; i < count; ++i) {
    status[i] = rcs[i];
    if (rcs[i] < 0 && worst == 0) worst = rcs[i];
  }
  if (worst < 0) return fail(nullptr, worst, "batch: " + first_err);
  return 0;
}

int pdnqp_get(const pdnqp_t *h, double *x, double *y, pdnqp_residuals *r) {
  if (!h) return fail(nullptr, PDNQP_ERR_ARG, "handle is NULL");
  cudaSetDevice(h->device);
  Result R;
  std::vector<double> lam_int(y ? h->m : 0);
  SolverBase *sv = h->escalated ? h->solver64 : h->solver;
  int rc = sv->get(x, y ? lam_int.data() : nullptr, &R);
  if (rc >= 0 && h->escalated) {  // counters cover both phases of the solve
    R.outer += h->r32.outer;
    R.inner += h->r32.inner;
    R.trials += h->r32.trials;
    R.restarts += h->r32.restarts;
    R.passes += h->r32.passes;
    R.seconds += h->r32.seconds;
    R.launches += h->r32.launches;
    R.inner_seconds += h->r32.inner_seconds;
    R.setup_seconds += h->r32.setup_seconds;
  }
  if (rc < 0) return fail(const_cast<pdnqp_t *>(h), rc, "pdnqp_get: no solution yet or CUDA failure");
  if (y)
    for (int k = 0; k < h->m; ++k) y[h->perm[k]] = lam_int[k];
  if (r) {
    r->r_p = R.rp;
    r->r_d = R.rd;
    r->s_p = R.sp;
    r->s_d = R.sd;
    r->rel_kkt = R.rel_kkt;
    r->outer_iters = R.outer;
    r->inner_iters = R.inner;
    r->trials = R.trials;
    r->restarts = R.restarts;
    r->kkt_passes = R.passes;
    r->solve_seconds = R.seconds;
    r->gamma = sv->gamma();
    r->lambda_min = sv->lambda_min();
    r->obj = R.obj;
    r->kernel_launches = R.launches;
    r->inner_seconds = R.inner_seconds;
    r->setup_seconds = R.setup_seconds;
    r->loop_seconds = R.loop_seconds;
    r->loop_trials = R.loop_trials;
    r->loop_blocks = R.loop_blocks;
    r->loop_launches = R.loop_launches;
    r->ctrl_used = R.ctrl_used;
    r->ctrl_fallbacks = R.ctrl_fallbacks;
    for (int k = 0; k < 6; ++k) r->loop_phase_seconds[k] = R.loop_phase_seconds[k];
  }
  return 0;
}

int pdnqp_set_start(pdnqp_t *h, const double *x0, const double *y0) {
  if (!h) return fail(nullptr, PDNQP_ERR_ARG, "handle is NULL");
  std::vector<double> l0;
  if (y0) {
    l0.resize(h->m);
    for (int k = 0; k < h->m; ++k) l0[k] = y0[h->perm[k]];
    for (double v : l0)
      if (!std::isfinite(v)) return fail(h, PDNQP_ERR_BOUNDS, "y0 has a non-finite entry");
  }
  if (x0)
    for (int i = 0; i < h->n; ++i)
      if (!std::isfinite(x0[i])) return fail(h, PDNQP_ERR_BOUNDS, "x0 has a non-finite entry");
  const int rc = h->solver->set_start(x0, y0 ? l0.data() : nullptr);
  if (rc == 0) {
    h->start_x.assign(x0 ? x0 : nullptr, x0 ? x0 + h->n : nullptr);
    h->start_l = l0;
  }
  return rc;
}

#define PDNQP_PARAMS(X)                                                                           \
  X(time_limit, d, 0.0, 1e300) X(k_out, ll, 1.0, 9.2e18) X(k_in, ll, 1.0, 9.2e18)                 \
  X(sigma_init, d, 1e-300, 1e300) X(theta_sigma, d, 0.0, 1.0) X(delta_gamma, d, 1e-300, 1e300)    \
  X(rho_in_min, d, 0.0, 1.0) X(rho_in_max, d, 0.0, 1.0) X(rho_z, d, 0.0, 1.0)                      \
  X(ruiz_inner, i, 0.0, 1000.0) X(lanczos_steps, i, 1.0, 100000.0) X(k_chk, i, 1.0, 1e9)           \
  X(beta_suff, d, 0.0, 1.0) X(beta_nec, d, 0.0, 1.0) X(beta_art, d, 0.0, 1.0)                      \
  X(rej_limit, i, 1.0, 1e9) X(kappa_shrink, d, 1e-6, 0.999999) X(delta_sigma, d, 1.0, 1e300)       \
  X(sigma_max, d, 1e-300, 1e300) X(tol_floor, d, 0.0, 1.0) X(chunk, i, 1.0, 65536.0)               \
  X(g_rows, i, 0.0, 16.0) X(g_cols, i, 0.0, 16.0) X(iter_budget, ll, 1.0, 4e18) X(cond_graph, i, 0.0, 1.0) \
  X(persistent, i, 0.0, 1.0) X(loop_blocks_per_sm, i, 0.0, 32.0) X(controller, i, 0.0, 1.0)             \
  X(ctrl_explore, d, 0.0, 10.0) X(ctrl_seed, ll, 0.0, 9.2e18) X(eps_inf, d, 0.0, 1.0) \
  X(anderson, i, 0.0, 1.0) X(anderson_mem, i, 2.0, 5.0) X(autotune, i, 0.0, 1.0) X(escalate, i, 0.0, 1.0) \
  X(batch_fused, i, 0.0, 1.0) X(batch_chunk, i, 1.0, 4096.0)

int pdnqp_set_param(pdnqp_t *h, const char *name, double value) {
  if (!h || !name) return fail(h, PDNQP_ERR_ARG, "NULL handle or name");
  const std::string s(name);
  if (s == "gamma") {
    if (!(value > 0) || !std::isfinite(value)) return fail(h, PDNQP_ERR_ARG, "gamma must be > 0");
    h->solver->set_gamma(value);
    return 0;
  }
#define X(nm, kind, lo, hi)                                                              \
  if (s == #nm) {                                                                        \
    if (!(value >= (lo) && value <= (hi))) return fail(h, PDNQP_ERR_ARG, "out of range: " #nm); \
    h->prm.nm = (decltype(h->prm.nm))value;                                              \
    return 0;                                                                            \
  }
  PDNQP_PARAMS(X)
#undef X
  return fail(h, PDNQP_ERR_ARG, "unknown parameter: " + s);
}

int pdnqp_get_param(const pdnqp_t *h, const char *name, double *value) {
  if (!h || !name || !value) return fail(nullptr, PDNQP_ERR_ARG, "NULL argument");
  const std::string s(name);
  if (s == "gamma") {
    *value = h->solver->gamma();
    return 0;
  }
  if (s == "ruiz_outer") {
    *value = h->prm.ruiz_outer;
    return 0;
  }
  if (s == "precision") {
    *value = h->precision;
    return 0;
  }
  if (s == "create_prepare_seconds") {
    *value = h->t_prepare;
    return 0;
  }
  if (s == "create_setup_seconds") {
    *value = h->t_setup;
    return 0;
  }
  if (s == "escalated") {
    *value = h->escalated ? 1.0 : 0.0;
    return 0;
  }
  if (s == "batch_graph_seconds") {
    *value = h->batch_graph_seconds;
    return 0;
  }
  if (s == "batch_graph_launches" || s == "batch_kernel_launches" || s == "batch_size") {
    *value = (double)(s == "batch_size" ? h->batch_size
                      : s == "batch_graph_launches" ? h->batch_graph_launches : h->batch_kernel_launches);
    return 0;
  }
  if (s == "rebases") {
    pdq::Result R;
    (h->escalated ? h->solver64 : h->solver)->get(nullptr, nullptr, &R);
    *value = (double)R.rebases;
    return 0;
  }
  if (s == "lanes_rows" || s == "lanes_cols") {
    *value = h->solver->tuned_g(s == "lanes_cols" ? 0 : 1);
    return 0;
  }
#define X(nm, kind, lo, hi) \
  if (s == #nm) {           \
    *value = (double)h->prm.nm; \
    return 0;               \
  }
  PDNQP_PARAMS(X)
#undef X
  return fail(const_cast<pdnqp_t *>(h), PDNQP_ERR_ARG, "unknown parameter: " + s);
}

int pdnqp_dims(const pdnqp_t *h, int64_t *out5) {
  if (!h || !out5) return fail(nullptr, PDNQP_ERR_ARG, "NULL argument");
  out5[0] = h->n;
  out5[1] = h->m;
  out5[2] = h->mE;
  out5[3] = h->m - h->mE;
  out5[4] = h->nnzq;
  return 0;
}

const char *pdnqp_last_error(const pdnqp_t *h) { return h ? h->err.c_str() : g_err.c_str(); }

int pdnqp_debug_inner(pdnqp_t *h, int n_ckpt, const int64_t *ckpt, double *snap) {
  if (!h || n_ckpt < 0 || (n_ckpt > 0 && (!ckpt || !snap))) return fail(h, PDNQP_ERR_ARG, "bad arguments");
  for (int k = 0; k < n_ckpt; ++k)
    if (ckpt[k] < 1 || (k > 0 && ckpt[k] <= ckpt[k - 1]))
      return fail(h, PDNQP_ERR_ARG, "checkpoints must be strictly increasing and >= 1");
  cudaSetDevice(h->device);
  std::string msg;
  int rc = h->solver->debug_inner(h->prm, n_ckpt, ckpt, snap, &msg);
  if (rc < 0) return fail(h, rc, msg);
  return rc;
}

int pdnqp_replay_kernel(pdnqp_t *h, int which, int reps) {
  const int kind = which & 7;
  if (!h || kind > 2 || (which & ~15) || reps < 0) return fail(h, PDNQP_ERR_ARG, "bad arguments");
  cudaSetDevice(h->device);
  int rc = h->solver->replay(which, reps);
  if (rc < 0) return fail(h, rc, "replay failed (solve first)");
  return 0;
}

double pdnqp_replay_last_ms(const pdnqp_t *h) { return h ? h->solver->last_replay_ms() : -1.0; }

int pdnqp_kernel_bytes(const pdnqp_t *h, int which, double *bytes) {
  if (!h || !bytes || which < -1 || which > 5 || which == 4) return fail(nullptr, PDNQP_ERR_ARG, "bad arguments");
  *bytes = h->solver->kernel_bytes(which);
  return 0;
}

int pdnqp_set_controller(pdnqp_t *h, const float *weights, int count) {
  if (!h) return fail(nullptr, PDNQP_ERR_ARG, "NULL handle");
  if (weights && count != pdnqp_mlp_param_count())
    return fail(h, PDNQP_ERR_ARG, "controller weights must have pdnqp_mlp_param_count() entries");
  cudaSetDevice(h->device);
  int rc = h->solver->set_controller(weights, weights ? count : 0);
  if (rc < 0) return fail(h, rc, "pdnqp_set_controller: device error");
  return 0;
}

int pdnqp_get_trace(const pdnqp_t *h, double *rows, int64_t max_rows, int64_t *n_rows) {
  if (!h || !n_rows || max_rows < 0 || (max_rows > 0 && !rows)) return fail(nullptr, PDNQP_ERR_ARG, "bad arguments");
  const std::vector<double> &t = h->solver->trace();
  const int64_t n = (int64_t)(t.size() / PDNQP_TRACE_COLS);
  *n_rows = n;
  const int64_t k = n < max_rows ? n : max_rows;
  for (int64_t i = 0; i < k * PDNQP_TRACE_COLS; ++i) rows[i] = t[(size_t)i];
  return 0;
}

}  // extern "C"
