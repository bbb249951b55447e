// Device helpers shared by the PDNQP kernels: sub-warp row groups for CSR
// SpMV, deterministic block reductions, and the device-resident scalar state
// of the inner solver.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pdq {

constexpr int kBlock = 256;        // threads per block of every vector/SpMV kernel
constexpr int kMaxBlocks = 152 * 8;  // grid cap: 8 resident 256-thread blocks on each of 152 SMs
constexpr int kRedThreads = 1024;  // threads of the single-block final reductions
constexpr int kMaxPartials = 48;   // quantities reduced per launch (rows of the partials array)

// Inner-solver status kept on the device (Algorithm 4 return paths).
enum InnerStatus : int {
  ST_RUNNING = 0,
  ST_CONVERGED = 1,
  ST_ITER_LIMIT = 2,
  ST_NUMERICAL_ERROR = 3,
  ST_PAUSED = 4,
  ST_IDLE = 5,
  ST_READY = 6,  // batched form: set up, waiting for the batch scheduler to let it run
};

// Scalar state of one inner solve.  Written by the host before the solve,
// updated only by single-block kernels (decide / check-final), read by all.
struct DevState {
  int status;
  int cur;             // index (0/1) of the current iterate buffers; the trial goes to 1 - cur
  int accepted;        // the last trial was accepted: the new averages are in buffer acur ^ 1
  int acur;            // index (0/1) of the committed running averages
  int check_due;       // a stopping/restart check follows this trial
  int restart_flag;    // the last check restarts the epoch
  int restart_use_avg; // ... from the averaged candidate
  int ret_avg;         // converged candidate is the average
  int ignore_conv;     // debug: never stop on the inner termination test
  int start_status;    // status the inner-solve setup ends in: ST_RUNNING, or ST_READY in the batched form
  long long t;         // accepted steps in the current epoch (N_p = N_d, Eq. pdqp-trial)
  long long t_total;   // accepted steps in this inner solve
  long long trials;    // all trials, all solves
  long long accepted_all;
  long long restarts;
  long long rej;       // consecutive rejections
  long long k_in;      // accepted-iteration limit (Table tab:parameters)
  long long pause_at;  // debug: pause after this many accepted steps (-1: never)
  long long k_chk;     // check period
  long long rej_limit;
  long long slot_left; // trials left in the current graph launch (bounds each device loop)
  double kappa;        // common step factor of the rejection rule
  double omega;        // primal weight (Eq. primal-weight-update)
  double alpha_acc;    // alpha of the last accepted trial
  double k_restart;    // restart metric at the start of the epoch
  double k_last;       // restart metric of the candidate at the previous check
  double dta, dtr;     // inner tolerances delta_a, delta_r
  double shrink;       // kappa factor on rejection
  double beta_suff, beta_nec, beta_art;
  double chk[16];      // reductions of the last check (diagnostics)
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <int G, typename A>
__device__ __forceinline__ A group_sum(A v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <int G, typename A>
__device__ __forceinline__ A group_max(A v) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// The blocks a kernel's work is spread over: the hardware grid, or, in the
// batched form, the contiguous run of blocks of one launch that one problem
// of the batch owns (block b of nb).  Reductions and grid-stride loops use
// it instead of blockIdx / gridDim, so a problem sees the same partition
// (and the same rounding) whether it runs alone or in a batch.
struct GridCtx {
  int b, nb;
};
__device__ __forceinline__ GridCtx hw_grid() { return GridCtx{(int)blockIdx.x, (int)gridDim.x}; }

// Block reduction of NQ doubles; bit q of kind_mask: 0 sum, 1 max (all maxima
// are of non-negative values).  Thread 0... of the block writes
// part[q * kMaxBlocks + blockIdx.x].  Must be called by every thread of the
// block (kBlock threads).  On this GPU the FP64 pipe is narrow and its cost is
// per active lane, so the reduction avoids FP64 shuffle trees: values go to
// shared memory and 8 threads per quantity sum 32 values each serially, then
// one thread sums the 8.  Fixed order: deterministic for a fixed grid.
template <int NQ>
__device__ __forceinline__ void block_reduce_store(double (&v)[NQ], const unsigned kind_mask, double *part,
                                                   int blk = -1) {
  if (blk < 0) blk = blockIdx.x;
  constexpr int NW = kBlock / 32;
  constexpr int WIN = 4;  // quantities staged at a time (8 KB of shared memory)
  __shared__ double sm[WIN][kBlock];
  __shared__ double s2[WIN][NW];
  const int t = threadIdx.x;
#pragma unroll
  for (int q0 = 0; q0 < NQ; q0 += WIN) {
#pragma unroll
    for (int k = 0; k < WIN; ++k)
      if (q0 + k < NQ) sm[k][t] = v[q0 + k];
    __syncthreads();
    if (t < WIN * NW) {
      const int k = t / NW, c = t % NW, q = q0 + k;
      if (q < NQ) {
        const bool mx = (kind_mask >> q) & 1u;
        const double *src = &sm[k][c * 32];
        double a = src[0];
        if (mx) {
          for (int i = 1; i < 32; ++i) a = fmax(a, src[i]);
        } else {
          for (int i = 1; i < 32; ++i) a += src[i];
        }
        s2[k][c] = a;
      }
    }
    __syncthreads();
    if (t < WIN && q0 + t < NQ) {
      const int q = q0 + t;
      const bool mx = (kind_mask >> q) & 1u;
      double a = s2[t][0];
      for (int c = 1; c < NW; ++c) a = mx ? fmax(a, s2[t][c]) : a + s2[t][c];
      part[q * kMaxBlocks + blk] = a;
    }
    __syncthreads();
  }
}

// Grid barrier of a cooperative (co-resident) launch.  bar[0] counts the
// arrivals, bar[kBarGen] is the generation, bar[kBarFault] the fault flag.  The last block to
// arrive runs lead() with all its threads before it releases the others, so
// lead() sees every block's writes from before the barrier and every block
// sees lead()'s writes after it.  The wait is bounded: a block that polls
// kSpinLimit times without a release (about a second or more), or that sees
// the fault flag, sets the flag and the call returns false; the caller then
// leaves the kernel, so a barrier that can never complete ends the launch
// instead of hanging it.
constexpr unsigned kSpinLimit = 1u << 22;
constexpr unsigned kSpinLimitTx = 1u << 24;  // polls of a bulk-copy barrier (with a 32 ns sleep)

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// Shared-memory mbarriers and bulk (TMA) copies global -> shared.  One thread
// arms a barrier with the byte count it expects and issues the copies; the
// barrier's phase completes when the bytes have landed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Makes barrier initialisation visible to the copy engine (async proxy).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier shared-memory accesses before later bulk copies.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// L2 policy for data read once per pass (the CSR streams): evict first, so
// that it does not push the iterate vectors, re-read every pass, out of L2.
__device__ __forceinline__ unsigned long long l2_evict_first_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, unsigned bytes, unsigned long long *bar,
                                              unsigned long long policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Bounded wait of one warp for the phase with the given parity: lane 0 polls
// (and every 64 polls looks at the fault flag), the result is warp-uniform,
// and on success every lane observes the completed phase itself, which makes
// the copied bytes visible to it.  Returns false on a timeout (the fault flag
// is then set) or when another warp has already set the fault flag.
__device__ __forceinline__ bool mbar_wait_warp(unsigned long long *bar, unsigned parity, unsigned *fault) {
  int r = 0;
  if ((threadIdx.x & 31) == 0) {
    for (unsigned it = 0; it <= kSpinLimitTx; ++it) {
      if (mbar_test(bar, parity)) {
        r = 1;
        break;
      }
      if ((it & 63u) == 63u && ld_acquire_gpu(fault) != 0u) break;
      __nanosleep(32);
    }
    if (!r) atomicExch(fault, 1u);
  }
  r = __shfl_sync(0xffffffffu, r, 0);
  if (r)
    for (unsigned it = 0; it <= kSpinLimitTx && !mbar_test(bar, parity); ++it) {
    }
  __syncwarp();
  return r != 0;
}

// Device-wide nanosecond timer (phase timing of the persistent loop).
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Word offsets of the barrier's generation and fault flag from its arrival
// counter: each on its own 128-byte line, so that the polls of the
// generation do not queue behind the arrival atomics.
constexpr int kBarGen = 32, kBarFault = 64, kBarWords = 96;

template <typename F>
__device__ __forceinline__ bool grid_sync(unsigned *bar, F lead) {
  __shared__ int role;  // 0 released, 1 leader, 2 fault
  unsigned gen = 0;
  __syncthreads();
  if (threadIdx.x == 0) {
    gen = ld_acquire_gpu(bar + kBarGen);
    __threadfence();
    role = (atomicAdd(bar, 1u) == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  if (role == 1) {
    __threadfence();
    lead();
    __syncthreads();
    if (threadIdx.x == 0) {
      atomicExch(bar, 0u);
      __threadfence();
      st_release_gpu(bar + kBarGen, gen + 1);
    }
  } else if (threadIdx.x == 0) {
    unsigned it = 0;
    while (ld_acquire_gpu(bar + kBarGen) == gen) {
      if (ld_acquire_gpu(bar + kBarFault) != 0u || ++it > kSpinLimit) {
        atomicExch(bar + kBarFault, 1u);
        role = 2;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
  }
  __syncthreads();
  return role != 2;
}
__device__ __forceinline__ bool grid_sync(unsigned *bar) {
  return grid_sync(bar, [] {});
}

// Single-block final reduction of NQ quantities over nb partials (fixed order):
// warp w handles quantities w, w + nwarps, ...; lane l sums partials l, l + 32,
// ... serially, then a fixed butterfly combines the 32 lane sums.  Every thread
// of the block gets out[].  blockDim.x must be a multiple of 32.
// Terms of the termination-test maxima (Eqs. outer-residuals / outer-scales).
// fmax drops a NaN operand, so a residual term that is not finite counts as
// +inf (a point with NaN or infinite entries never passes), and a scale term
// that is not finite is left out (an infinite scale would excuse any residual).
__device__ __forceinline__ double res_term(double v) { return isfinite(v) ? v : INFINITY; }
__device__ __forceinline__ double scale_term(double v) { return isfinite(v) ? v : 0.0; }

template <int NQ>
__device__ __forceinline__ void final_reduce(const double *part, int nb, const unsigned kind_mask, double (&out)[NQ]) {
  __shared__ double res[NQ];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = wid; q < NQ; q += nw) {
    const bool mx = (kind_mask >> q) & 1u;
    double a = 0.0;
    for (int b = lane; b < nb; b += 32) {
      const double p = __ldcg(part + q * kMaxBlocks + b);
      a = mx ? fmax(a, p) : a + p;
    }
    a = mx ? warp_max(a) : warp_sum(a);  // fixed butterfly: deterministic
    if (lane == 0) res[q] = a;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q) out[q] = res[q];
  __syncthreads();
}

// Rows of a CSR matrix are processed by groups of G lanes (G divides 32).
// Iteration is warp-uniform: every lane of a warp runs the same trips
// (base is the same for the whole warp), with row >= nrows marking idle
// groups, so group shuffles are always executed by the full warp.
template <int G>
struct GroupIter {
  int lane_g, sub;
  long long first, step;
  __device__ __forceinline__ GroupIter() {
    lane_g = threadIdx.x & (G - 1);
    sub = (threadIdx.x & 31) / G;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    first = gw * (32 / G);
    step = nw * (32 / G);
  }
};

// Sum over the entries of one row of f(col, val), reduced over the group; every
// lane of the group gets the result.
template <int G, typename Acc, typename T, typename F>
__device__ __forceinline__ Acc row_sum(const int *__restrict__ rp, const int *__restrict__ ci,
                                       const T *__restrict__ val, long long row, bool valid, int lane_g, F f) {
  Acc a = Acc(0);
  if (valid) {
    const int b = rp[row], e = rp[row + 1];
    for (int k = b + lane_g; k < e; k += G) a += f(ci[k], val[k]);
  }
  return group_sum<G, Acc>(a);
}
template <int G, typename Acc, typename T, typename F>
__device__ __forceinline__ Acc row_max(const int *__restrict__ rp, const int *__restrict__ ci,
                                       const T *__restrict__ val, long long row, bool valid, int lane_g, F f) {
  Acc a = Acc(0);
  if (valid) {
    const int b = rp[row], e = rp[row + 1];
    for (int k = b + lane_g; k < e; k += G) a = fmax(a, f(ci[k], val[k]));
  }
  return group_max<G, Acc>(a);
}


// Warp tiles of 32 consecutive rows: lane l owns row tile + l for the
// epilogue (all lanes active, coalesced per-row loads and stores), while the
// row dot products are computed by groups of G lanes in G passes of 32/G rows
// each, and the result of each row is shuffled to the lane that owns it.
struct TileIter {
  int lane;
  long long first, step;
  __device__ __forceinline__ TileIter(GridCtx g = hw_grid()) {
    lane = threadIdx.x & 31;
    const long long gw = ((long long)g.b * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)g.nb * blockDim.x) >> 5;
    first = gw * 32;
    step = nw * 32;
  }
};

template <typename Acc>
__device__ __forceinline__ Acc shfl_any(Acc v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}

// Per-warp staging buffer of one CSR-stream chunk: 32 * K entries.
template <int K, typename Acc>
__device__ __forceinline__ Acc *warp_stage_buffer() {
  __shared__ Acc buf[kBlock / 32][32 * K];
  return buf[threadIdx.x >> 5];
}

// CSR-stream row reduction over a warp tile of 32 consecutive rows: the
// tile's contiguous nonzero range is streamed in chunks of 32 * K entries;
// each lane loads K entries with coalesced, independent loads, evaluates
// f(col, val) (including its gather) and stores it in the warp's staging
// buffer; then lane l reduces the slice of the chunk that belongs to row
// tile + l.  Rows of any length are handled (a long row spans several
// chunks).  Lane l returns the result of row tile + l (0 past nrows).
template <int K, bool IsMax, typename Acc, typename T, typename F>
__device__ __forceinline__ Acc tile_stream(const int *__restrict__ rp, const int *__restrict__ ci,
                                           const T *__restrict__ val, long long tile, long long nrows, F f) {
  const int lane = threadIdx.x & 31;
  Acc *sb = warp_stage_buffer<K, Acc>();
  const long long my = tile + lane;
  const long long last = (nrows - 1 - tile) < 31 ? (nrows - 1 - tile) : 31;  // last valid lane (>= 0)
  int rb = 0, re = 0;
  if (my < nrows) {
    rb = rp[my];
    re = rp[my + 1];
  }
  const int base = __shfl_sync(0xffffffffu, rb, 0);
  const int end = __shfl_sync(0xffffffffu, re, (int)last);
  if (my >= nrows) rb = re = end;
  Acc acc = Acc(0);
  for (int c0 = base; c0 < end; c0 += 32 * K) {
    Acc p[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int k = c0 + j * 32 + lane;
      p[j] = k < end ? f(ci[k], val[k]) : Acc(0);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) sb[j * 32 + lane] = p[j];
    __syncwarp();
    const int lo = rb > c0 ? rb : c0;
    const int hi = re < c0 + 32 * K ? re : c0 + 32 * K;
    for (int k = lo; k < hi; ++k) acc = IsMax ? fmax(acc, sb[k - c0]) : acc + sb[k - c0];
    __syncwarp();
  }
  return acc;
}

// Two CSR matrices with the same rows streamed together over one warp tile
// (the column pass: Q and A^T): both row-pointer pairs, then in every trip
// one chunk of each matrix, so the two dependent load chains (row pointers ->
// entries -> gathers) overlap instead of running one after the other.  Lane l
// gets the sums of row tile + l of both matrices in o1, o2.
template <int K1, int K2, typename Acc, typename T, typename F1, typename F2>
__device__ __forceinline__ void tile_pair_sum(const int *__restrict__ rp1, const int *__restrict__ ci1,
                                              const T *__restrict__ v1, const int *__restrict__ rp2,
                                              const int *__restrict__ ci2, const T *__restrict__ v2, long long tile,
                                              long long nrows, F1 f1, F2 f2, Acc &o1, Acc &o2) {
  const int lane = threadIdx.x & 31;
  Acc *sb1 = warp_stage_buffer<K1, Acc>();
  __shared__ Acc buf2[kBlock / 32][32 * K2];
  Acc *sb2 = buf2[threadIdx.x >> 5];
  const long long my = tile + lane;
  const long long last = (nrows - 1 - tile) < 31 ? (nrows - 1 - tile) : 31;
  int rb1 = 0, re1 = 0, rb2 = 0, re2 = 0;
  if (my < nrows) {
    rb1 = rp1[my];
    re1 = rp1[my + 1];
    rb2 = rp2[my];
    re2 = rp2[my + 1];
  }
  const int base1 = __shfl_sync(0xffffffffu, rb1, 0), end1 = __shfl_sync(0xffffffffu, re1, (int)last);
  const int base2 = __shfl_sync(0xffffffffu, rb2, 0), end2 = __shfl_sync(0xffffffffu, re2, (int)last);
  if (my >= nrows) {
    rb1 = re1 = end1;
    rb2 = re2 = end2;
  }
  Acc a1 = Acc(0), a2 = Acc(0);
  for (int c1 = base1, c2 = base2; c1 < end1 || c2 < end2; c1 += 32 * K1, c2 += 32 * K2) {
    Acc p1[K1], p2[K2];
#pragma unroll
    for (int j = 0; j < K1; ++j) {
      const int k = c1 + j * 32 + lane;
      p1[j] = k < end1 ? f1(ci1[k], v1[k]) : Acc(0);
    }
#pragma unroll
    for (int j = 0; j < K2; ++j) {
      const int k = c2 + j * 32 + lane;
      p2[j] = k < end2 ? f2(ci2[k], v2[k]) : Acc(0);
    }
#pragma unroll
    for (int j = 0; j < K1; ++j) sb1[j * 32 + lane] = p1[j];
#pragma unroll
    for (int j = 0; j < K2; ++j) sb2[j * 32 + lane] = p2[j];
    __syncwarp();
    {
      const int lo = rb1 > c1 ? rb1 : c1, hi = re1 < c1 + 32 * K1 ? re1 : c1 + 32 * K1;
      for (int k = lo; k < hi; ++k) a1 += sb1[k - c1];
    }
    {
      const int lo = rb2 > c2 ? rb2 : c2, hi = re2 < c2 + 32 * K2 ? re2 : c2 + 32 * K2;
      for (int k = lo; k < hi; ++k) a2 += sb2[k - c2];
    }
    __syncwarp();
  }
  o1 = a1;
  o2 = a2;
}

template <int K, typename Acc, typename T, typename F>
__device__ __forceinline__ Acc tile_row_sum(const int *__restrict__ rp, const int *__restrict__ ci,
                                            const T *__restrict__ val, long long tile, long long nrows, F f) {
  return tile_stream<K, false, Acc>(rp, ci, val, tile, nrows, f);
}
template <int K, typename Acc, typename T, typename F>
__device__ __forceinline__ Acc tile_row_max(const int *__restrict__ rp, const int *__restrict__ ci,
                                            const T *__restrict__ val, long long tile, long long nrows, F f) {
  return tile_stream<K, true, Acc>(rp, ci, val, tile, nrows, f);
}

inline int grid_for(long long work_items, int per_block) {
  long long b = (work_items + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > kMaxBlocks) b = kMaxBlocks;
  return (int)b;
}

}  // namespace pdq
