// Batched form, fused: the scheduler that runs the inner iterations
// (Algorithm 4) of many problems of one precision together.  Each problem
// keeps its own solver, device state and host thread for the outer
// iteration (Algorithm 3, on the CPU as in Sec. 3.4); when its inner solve
// is set up, its thread hands it here and sleeps.  The scheduler launches one
// captured CUDA graph of `chunk` trial slots over the whole batch, one launch
// per phase (kernels.cuh, "Batched form"): every running problem takes its
// trial, its acceptance decision, its periodic check, restart and inner
// termination on the device, and problems that are not running skip.  After
// each graph launch one gather of all device states tells the scheduler
// which inner solves stopped; their threads resume.  Included by each solver
// translation unit after solver_impl.cuh.
#pragma once
#include <algorithm>
#include <condition_variable>
#include <mutex>
#include <numeric>

namespace pdq {

#define BK(expr)                                                                              \
  do {                                                                                        \
    cudaError_t _e = (expr);                                                                  \
    if (_e != cudaSuccess) return fail(std::string(#expr) + ": " + cudaGetErrorString(_e));   \
  } while (0)
#define BTRY(x)            \
  do {                     \
    int _r = (x);          \
    if (_r < 0) return _r; \
  } while (0)

template <typename T>
class BatchRunner : public BatchBase, public BatchHook {
 public:
  BatchRunner(std::vector<Solver<T> *> sv, std::vector<int> g_rows, std::vector<int> g_cols, int chunk)
      : sv_(std::move(sv)), g_rows_(std::move(g_rows)), g_cols_(std::move(g_cols)),
        chunk_(std::max(1, chunk)) {}

  ~BatchRunner() override {
    for (Solver<T> *s : sv_) {
      s->batch_ = nullptr;
      s->batch_idx_ = -1;
    }
    if (bs_) cudaStreamSynchronize(bs_);
    if (gexec_) cudaGraphExecDestroy(gexec_);
    for (void *p : dmem_) cudaFree(p);
    if (hstates_) cudaFreeHost(hstates_);
    if (hlist_) cudaFreeHost(hlist_);
    for (cudaEvent_t e : ev_)
      if (e) cudaEventDestroy(e);
    if (bs_) cudaStreamDestroy(bs_);
  }

  int build() {
    const int P = (int)sv_.size();
    hs_.assign(P, H_HOST);
    deadline_.assign(P, INFINITY);
    got_.assign(P, DevState{});
    tl_.assign(P, 0);
    stop_sent_.assign(P, 0);
    BK(cudaStreamCreateWithFlags(&bs_, cudaStreamNonBlocking));
    BK(cudaEventCreate(&ev_[0]));
    BK(cudaEventCreate(&ev_[1]));
    // Blocks of the largest problems first.
    std::vector<int> order(P);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return (long long)sv_[a]->n_ + sv_[a]->m_ > (long long)sv_[b]->n_ + sv_[b]->m_;
    });
    std::vector<Dev<T>> devs(P);
    std::vector<int> nbr(P);
    for (int i = 0; i < P; ++i) {
      devs[i] = sv_[i]->d_;
      devs[i].hw = 0;
      devs[i].hc = 0;
      nbr[i] = sv_[i]->nb_rows();
    }
    BTRY(upload(&devs_, devs));
    BTRY(upload(&nbr_, nbr));
    // One block map per launch: the problem's solo partition.
    auto map_of = [&](auto nb_of, auto keep) {
      std::vector<BatchBlk> m;
      for (int i : order)
        if (keep(i))
          for (int b = 0, nb = nb_of(i); b < nb; ++b) m.push_back(BatchBlk{i, b, nb});
      return m;
    };
    auto all = [](int) { return true; };
    BTRY(add_map(&primal_, map_of([&](int i) { return sv_[i]->grid_n(); }, all)));
    BTRY(add_map(&apply_, map_of([&](int i) { return sv_[i]->grid_nm(); }, all)));
    for (int g : {4, 8, 16}) {
      Launch r, c;
      r.g = c.g = g;
      BTRY(add_map(&r, map_of([&](int i) { return sv_[i]->nb_rows(); }, [&](int i) { return g_rows_[i] == g; })));
      BTRY(add_map(&c, map_of([&](int i) { return sv_[i]->nb_cols(); }, [&](int i) { return g_cols_[i] == g; })));
      if (r.nblk) rows_.push_back(r);
      if (c.nblk) cols_.push_back(c);
    }
    BTRY(dalloc(&dstates_, (size_t)P));
    BTRY(dalloc(&dlist_, (size_t)2 * P));
    BK(cudaMallocHost(&hstates_, sizeof(DevState) * (size_t)P));
    BK(cudaMallocHost(&hlist_, sizeof(int) * (size_t)2 * P));
    // The graph: chunk slots of [primal, rows, cols (+ decisions), check rows,
    // check cols (+ check decisions), check apply] over the whole batch.
    cudaGraph_t g;
    BK(cudaStreamBeginCapture(bs_, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < chunk_; ++k) launch_slot();
    BK(cudaStreamEndCapture(bs_, &g));
    cudaError_t e = cudaGraphInstantiate(&gexec_, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    BK(cudaGraphUpload(gexec_, bs_));
    BK(cudaStreamSynchronize(bs_));
    for (int i = 0; i < P; ++i) {
      sv_[i]->batch_ = this;
      sv_[i]->batch_idx_ = i;
    }
    return 0;
  }

  // ---- BatchHook (worker threads)
  int run_inner(int idx, DevState *S, double deadline) override {
    std::unique_lock<std::mutex> lk(mu_);
    if (failed_) return PDNQP_ERR_CUDA;
    hs_[idx] = H_READY;
    deadline_[idx] = deadline;
    cv_.notify_all();
    cv_.wait(lk, [&] { return hs_[idx] == H_STOPPED || failed_; });
    if (failed_) return PDNQP_ERR_CUDA;
    *S = got_[idx];
    hs_[idx] = H_HOST;
    return tl_[idx];
  }

  // ---- BatchBase
  void finished(int idx) override {
    std::lock_guard<std::mutex> lk(mu_);
    hs_[idx] = H_DONE;
    cv_.notify_all();
  }

  int schedule() override {
    const int P = (int)sv_.size();
    std::vector<int> go, stop;
    for (;;) {
      go.clear();
      stop.clear();
      bool any_run = false;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] {
          int done = 0;
          for (int h : hs_) {
            if (h == H_READY || h == H_RUN) return true;
            done += h == H_DONE;
          }
          return done == P;
        });
        const double now = Solver<T>::now();
        for (int i = 0; i < P; ++i) {
          if (hs_[i] == H_READY) {
            hs_[i] = H_RUN;
            go.push_back(i);
          } else if (hs_[i] == H_RUN && !stop_sent_[i] && now > deadline_[i]) {
            stop_sent_[i] = 1;
            stop.push_back(i);
          }
          any_run |= hs_[i] == H_RUN;
        }
        if (!any_run) return 0;  // every problem has finished
      }
      int rc = step(go, stop);
      std::lock_guard<std::mutex> lk(mu_);
      if (rc < 0) {
        failed_ = true;
        cv_.notify_all();
        return rc;
      }
      for (int i = 0; i < P; ++i) {
        if (hs_[i] != H_RUN) continue;
        const DevState &S = hstates_[i];
        if (S.status == ST_RUNNING || S.status == ST_READY) continue;
        got_[i] = S;
        tl_[i] = (S.status == ST_PAUSED && stop_sent_[i]) ? 1 : 0;
        stop_sent_[i] = 0;
        hs_[i] = H_STOPPED;
      }
      cv_.notify_all();
    }
  }

  const std::string &error() const override { return err_; }
  long long graph_launches() const override { return graph_launches_; }
  double graph_seconds() const override { return graph_seconds_; }
  long long kernel_launches() const override { return kernel_launches_; }

 private:
  enum { H_HOST = 0, H_READY = 1, H_RUN = 2, H_STOPPED = 3, H_DONE = 4 };
  struct Launch {
    int g = 0;
    int nblk = 0;
    BatchBlk *map = nullptr;
  };

  int fail(const std::string &m) {
    err_ = m;
    return PDNQP_ERR_CUDA;
  }
  template <typename V>
  int dalloc(V **p, size_t count) {
    void *q = nullptr;
    BK(cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(V)));
    dmem_.push_back(q);
    *p = (V *)q;
    return 0;
  }
  template <typename V>
  int upload(V **p, const std::vector<V> &h) {
    BTRY(dalloc(p, h.size()));
    if (!h.empty()) BK(cudaMemcpy(*p, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
    return 0;
  }
  int add_map(Launch *L, const std::vector<BatchBlk> &m) {
    L->nblk = (int)m.size();
    if (L->nblk) BTRY(upload(&L->map, m));
    return 0;
  }

  // One trial slot over the batch (captured into the graph).
  void launch_slot() {
    kb_primal<T><<<primal_.nblk, kBlock, 0, bs_>>>(devs_, primal_.map);
    for (const Launch &L : rows_)
      with_G(L.g, [&](auto GG) { kb_rows<T, decltype(GG)::value><<<L.nblk, kBlock, 0, bs_>>>(devs_, L.map); });
    for (const Launch &L : cols_)
      with_G(L.g, [&](auto GG) { kb_cols<T, decltype(GG)::value><<<L.nblk, kBlock, 0, bs_>>>(devs_, L.map, nbr_); });
    for (const Launch &L : rows_)
      with_G(L.g, [&](auto GG) {
        kb_check_rows<T, decltype(GG)::value><<<L.nblk, kBlock, 0, bs_>>>(devs_, L.map);
      });
    for (const Launch &L : cols_)
      with_G(L.g, [&](auto GG) {
        kb_check_cols<T, decltype(GG)::value><<<L.nblk, kBlock, 0, bs_>>>(devs_, L.map, nbr_);
      });
    kb_check_apply<T><<<apply_.nblk, kBlock, 0, bs_>>>(devs_, apply_.map);
  }
  long long kernels_per_slot() const { return 2 + 2 * (long long)(rows_.size() + cols_.size()); }

  // Scheduler edits, one graph launch, one read-back of all states.
  int step(const std::vector<int> &go, const std::vector<int> &stop) {
    const int P = (int)sv_.size();
    const int ng = (int)go.size(), ns = (int)stop.size();
    if (ng + ns) {
      std::copy(go.begin(), go.end(), hlist_);
      std::copy(stop.begin(), stop.end(), hlist_ + ng);
      BK(cudaMemcpyAsync(dlist_, hlist_, sizeof(int) * (size_t)(ng + ns), cudaMemcpyHostToDevice, bs_));
      kb_control<T><<<(ng + ns + 255) / 256, 256, 0, bs_>>>(devs_, dlist_, ng, dlist_ + ng, ns);
      ++kernel_launches_;
    }
    BK(cudaEventRecord(ev_[0], bs_));
    BK(cudaGraphLaunch(gexec_, bs_));
    BK(cudaEventRecord(ev_[1], bs_));
    ++graph_launches_;
    kernel_launches_ += chunk_ * kernels_per_slot();
    kb_gather_states<T><<<(P * (int)(sizeof(DevState) / 4) + 255) / 256, 256, 0, bs_>>>(devs_, P, dstates_);
    ++kernel_launches_;
    BK(cudaGetLastError());
    BK(cudaMemcpyAsync(hstates_, dstates_, sizeof(DevState) * (size_t)P, cudaMemcpyDeviceToHost, bs_));
    BK(cudaStreamSynchronize(bs_));
    float ms = 0.f;
    BK(cudaEventElapsedTime(&ms, ev_[0], ev_[1]));
    graph_seconds_ += 1e-3 * ms;
    return 0;
  }

  std::vector<Solver<T> *> sv_;
  std::vector<int> g_rows_, g_cols_;
  int chunk_;
  cudaStream_t bs_ = nullptr;
  cudaGraphExec_t gexec_ = nullptr;
  std::vector<void *> dmem_;
  Dev<T> *devs_ = nullptr;
  int *nbr_ = nullptr;
  Launch primal_, apply_;
  std::vector<Launch> rows_, cols_;
  DevState *dstates_ = nullptr, *hstates_ = nullptr;
  int *dlist_ = nullptr, *hlist_ = nullptr;
  std::mutex mu_;
  std::condition_variable cv_;
  std::vector<int> hs_, tl_, stop_sent_;
  std::vector<double> deadline_;
  std::vector<DevState> got_;
  bool failed_ = false;
  std::string err_;
  long long graph_launches_ = 0, kernel_launches_ = 0;
  double graph_seconds_ = 0.0;
  cudaEvent_t ev_[2] = {nullptr, nullptr};
};

template <typename T>
BatchBase *make_batch_impl(const std::vector<SolverBase *> &sv, const std::vector<int> &g_rows,
                           const std::vector<int> &g_cols, int chunk, std::string *err) {
  std::vector<Solver<T> *> s;
  for (SolverBase *b : sv) {
    Solver<T> *p = dynamic_cast<Solver<T> *>(b);
    if (!p || !p->ready_) {
      if (err) *err = "batched form: every solver must be set up and of the batch's precision";
      return nullptr;
    }
    s.push_back(p);
  }
  BatchRunner<T> *r = new BatchRunner<T>(std::move(s), g_rows, g_cols, chunk);
  if (r->build() < 0) {
    if (err) *err = r->error();
    delete r;
    return nullptr;
  }
  return r;
}

#undef BK
#undef BTRY

}  // namespace pdq
