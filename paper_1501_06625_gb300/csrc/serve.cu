// serve.cu -- ph_server_*: a continuous-batching request loop for path-tracking
// jobs of different sizes and precisions.
//
// The paper tracks one path at a time from the host (Section 3.1).  A service
// receives jobs while others run, so here:
//  * every job gets its own workspace (its point, history, step size, Jacobian)
//    carved from one device pool; the host admits a job only when its
//    footprint fits in the free pool (first fit), otherwise it waits on the host
//    in arrival order; a finished job's region returns to the pool;
//  * admitted jobs go to a queue in host-mapped pinned memory (coherent with the
//    GPU on Grace-Blackwell): a descriptor per table slot, then the queue
//    position, then the tail index, each published after the previous with a
//    release fence;
//  * one persistent kernel works the queue: each block claims the next
//    published position with a compare-and-swap (a block that finds nothing
//    holds no claim), tracks that job with pathblock.cuh in the job's precision
//    (double-double or quad-double), writes the end point and statistics to
//    mapped memory, sets the slot's completion word and claims the next job --
//    so new jobs start as soon as any block is free, and they overlap the jobs
//    already running on the other blocks;
//  * the kernel stays whole while there is work: a block that finds nothing to
//    claim keeps polling as long as another block holds a job or a job was
//    claimed or finished in the last 20 ms; only then does one block close the
//    kernel (a flag bit on the claim counter, set by compare-and-swap while no
//    block holds or is claiming a job), and every block leaves.  So a long job
//    never leaves the kernel with fewer blocks than the GPU holds;
//  * a host thread reaps completions (timestamps, pool space), admits waiting
//    jobs and, when a published job is unclaimed and no kernel runs, reopens
//    the claim counter and launches the kernel again.
// A job's result does not depend on what runs beside it: a block runs one job
// at a time and the tracking code takes no value from other blocks.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "pathblock.cuh"

using namespace ph;

long ph_lda(int N);
ph_status ph_track_path_exec(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                             const double *gamma, const double *x0,
                             const ph_track_params *params, double *x_out,
                             ph_path_stats *stats, ph_step_record *log, int log_cap);
void ph_job_fill_system(Job &j, const ph_system *f, const ph_system *g);
long ph_job_ws_doubles(const Job &j);

namespace {

constexpr unsigned long long kIdleNs = 20000000ull;   // an idle block waits 20 ms

// one table slot, in mapped pinned memory
struct Slot {
  Job job;                        // x0/x_out/stats point into this slot's mapped buffers
  volatile unsigned long long seq;      // published job number (0: empty)
  volatile unsigned long long claimed;  // set to seq by the block that claims the job
  volatile unsigned long long done;     // set to seq when the job's results are written
};

struct Queue {                    // mapped pinned memory
  volatile unsigned long long tail;     // positions [0, tail) are published (host)
  volatile int shutdown;
  int pad;
};

// device memory: the claim counter (positions [0, head) are claimed; the top
// bit closes the kernel), the blocks holding or claiming a job, and the
// globaltimer of the last claim or completion
struct Ctl {
  unsigned long long head;
  unsigned long long busy;
  unsigned long long last;
};
constexpr unsigned long long kClosed = 1ull << 63;

PHD unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// copy of a slot's job descriptor through loads that do not trust cached lines
__device__ void load_job(const Slot *s, Job *out) {
  const unsigned long long *src = (const unsigned long long *)&s->job;
  unsigned long long *dst = (unsigned long long *)out;
  for (int i = 0; i < (int)(sizeof(Job) / 8); ++i) dst[i] = __ldcv(src + i);
}

// Claim protocol (thread 0 of a block).  A block that wants a job first counts
// itself busy, then reads the counter and, if a published position is
// unclaimed, takes it by compare-and-swap.  A block that closes the kernel
// sees busy == 0 and then swaps the counter to its closed form: a claim that
// raced with it either landed first (the close fails: the counter moved) or
// fails itself and finds the counter closed.  So a job is never claimed by a
// kernel that is closing, and a kernel never closes while a job runs.
__device__ int claim_job(const int *queue, const Queue *q, Ctl *c, int cap) {
  volatile unsigned long long *head = &c->head, *busy = &c->busy, *last = &c->last;
  for (;;) {
    if (q->shutdown) return -1;
    const unsigned long long h = *head;
    if (h & kClosed) return -1;
    if (h < q->tail) {
      atomicAdd(&c->busy, 1ull);
      __threadfence();
      const unsigned long long h2 = *head;
      if (!(h2 & kClosed) && h2 < q->tail && atomicCAS(&c->head, h2, h2 + 1) == h2) {
        *last = gtimer();
        return __ldcv(queue + (h2 % cap));   // stays busy until the job is done
      }
      atomicAdd(&c->busy, ~0ull);
      continue;
    }
    __threadfence();
    if (gtimer() - *last > kIdleNs && *busy == 0) {
      __threadfence();
      if (atomicCAS(&c->head, h, h | kClosed) == h) return -1;
      continue;
    }
    __nanosleep(2000);
  }
}

__global__ void k_reopen(Ctl *c) {
  c->head &= ~kClosed;
  c->busy = 0;
  c->last = gtimer();
}

__global__ void __launch_bounds__(kBT, 1) k_serve(Slot *slots, const int *queue, Queue *q, Ctl *ctl,
                                               int cap) {
  extern __shared__ double smem[];
  __shared__ Job s_job;
  __shared__ int s_slot;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) {
      const int claimed = claim_job(queue, q, ctl, cap);
      s_slot = claimed;
      if (claimed >= 0) {
        // the descriptor was published before the position: wait for its sequence
        // word (bounded), then copy it
        Slot *s = slots + claimed;
        unsigned long long w0 = gtimer();
        while (s->seq == 0 && gtimer() - w0 < kIdleNs) __nanosleep(100);
        __threadfence_system();
        load_job(s, &s_job);
        s->claimed = s->seq;
      }
    }
    __syncthreads();
    const int slot = s_slot;
    if (slot < 0) return;
    Job j = s_job;
    // the start point and gamma: from mapped memory into the job's workspace
    const long pt = 2L * j.L * j.n;
    double *x0d = j.ws + j.o_dx;                 // dx is free until the first solve
    double *gd = j.ws + j.o_g;
    for (long e = tid; e < pt; e += kBT) x0d[e] = __ldcv(j.x0 + e);
    for (int e = tid; e < 2 * j.L; e += kBT) gd[e] = __ldcv(j.gamma + e);
    __syncthreads();
    j.x0 = x0d;
    j.gamma = gd;
    if (j.L == 1) track_job<F64>(j, smem);
    else if (j.L == 2) track_job<DD>(j, smem);
    else track_job<QD>(j, smem);
    __threadfence_system();
    __syncthreads();
    if (tid == 0) {
      slots[slot].done = slots[slot].seq;
      *(volatile unsigned long long *)&ctl->last = gtimer();
      __threadfence();
      atomicAdd(&ctl->busy, ~0ull);
    }
    __syncthreads();
  }
}

struct PoolAlloc {                // first fit over [0, size) in bytes, 256-byte units
  size_t size = 0;
  std::map<size_t, size_t> free_;  // offset -> length
  void init(size_t s) {
    size = s;
    free_.clear();
    free_[0] = s;
  }
  bool alloc(size_t len, size_t *off) {
    len = (len + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= len) {
        *off = it->first;
        size_t rest = it->second - len, o = it->first + len;
        free_.erase(it);
        if (rest) free_[o] = rest;
        return true;
      }
    return false;
  }
  void release(size_t off, size_t len) {
    len = (len + 255) / 256 * 256;
    auto it = free_.emplace(off, len).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

using clk = std::chrono::steady_clock;

struct JobRec {
  Job job;                         // system, parameters, layout (pointers filled on admission)
  std::vector<double> x0, gamma;
  size_t bytes = 0, off = 0;
  int slot = -1;
  int state = 0;                   // 0 waiting, 1 on the device, 2 done
  clk::time_point t_submit, t_done;
  std::vector<double> x_out;
  ph_path_stats stats;
  // the large-job route: the homotopy, run by the single-path tracker
  bool big = false;
  const ph_system *f = nullptr, *g = nullptr;
  ph_track_params p;
};

}  // namespace

struct ph_server {
  ph_ctx *ctx = nullptr;
  ph_server_config cfg;
  cudaStream_t stream = nullptr;
  int cap = 0, grid = 0;
  size_t smem = 0, slot_doubles = 0;
  // mapped pinned memory
  Slot *slots = nullptr;           // [cap]
  int *queue = nullptr;            // [cap]
  Queue *q = nullptr;
  double *bufs = nullptr;          // per slot: x0 [2*4*max_n], x_out [2*4*max_n], gamma [8]
  ph_path_stats *stats = nullptr;  // [cap]
  // device pool
  DevBuf pool, ctl;
  PoolAlloc palloc;
  // host state
  std::mutex mu;
  std::condition_variable cv;
  std::thread worker;
  bool stop = false, launched = false;
  std::string err;
  int64_t next_id = 1;
  std::map<int64_t, JobRec> jobs;
  std::deque<int64_t> waiting;     // not yet admitted, in arrival order
  std::vector<int> free_slots;
  std::vector<int64_t> slot_job;   // slot -> job id
  unsigned long long published = 0;
  long long launches = 0;
  // the large-job route: a context and stream of the server's own
  ph_ctx *big_ctx = nullptr;
  cudaStream_t big_stream = nullptr;
  long long big_done = 0;
};

static void server_loop(ph_server *s);

static void admit_locked(ph_server *s) {
  while (!s->waiting.empty() && !s->free_slots.empty()) {
    JobRec &r = s->jobs[s->waiting.front()];
    if (r.big) break;                             // the GPU is drained for it first
    size_t off;
    if (!s->palloc.alloc(r.bytes, &off)) break;   // the oldest waiting job does not fit yet
    const int64_t id = s->waiting.front();
    s->waiting.pop_front();
    const int slot = s->free_slots.back();
    s->free_slots.pop_back();
    r.off = off;
    r.slot = slot;
    r.state = 1;
    s->slot_job[slot] = id;
    double *b = s->bufs + (size_t)slot * s->slot_doubles;
    const size_t pt = r.x0.size();
    double *x0m = b, *xom = b + 8 * s->cfg.max_n, *gm = b + 16 * s->cfg.max_n;
    memcpy(x0m, r.x0.data(), sizeof(double) * pt);
    memcpy(gm, r.gamma.data(), sizeof(double) * r.gamma.size());
    Job j = r.job;
    j.ws = (double *)((char *)s->pool.p + off);
    j.gamma = gm;                 // read by the block's first thread through L2 (mapped)
    j.x0 = x0m;
    j.x_out = xom;
    j.stats = s->stats + slot;
    j.log = nullptr;
    j.log_cap = 0;
    Slot *sl = s->slots + slot;
    sl->done = 0;
    sl->claimed = 0;
    sl->seq = 0;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    memcpy((void *)&sl->job, &j, sizeof(Job));
    std::atomic_thread_fence(std::memory_order_seq_cst);
    sl->seq = (unsigned long long)id;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    s->queue[s->published % s->cap] = slot;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    s->published += 1;
    s->q->tail = s->published;
    std::atomic_thread_fence(std::memory_order_seq_cst);
  }
}

static void reap_locked(ph_server *s) {
  for (int slot = 0; slot < s->cap; ++slot) {
    const int64_t id = s->slot_job[slot];
    if (id == 0) continue;
    Slot *sl = s->slots + slot;
    if (sl->done != (unsigned long long)id) continue;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    JobRec &r = s->jobs[id];
    r.t_done = clk::now();
    const size_t pt = r.x0.size();
    const double *xom = s->bufs + (size_t)slot * s->slot_doubles + 8 * s->cfg.max_n;
    r.x_out.assign(xom, xom + pt);
    r.stats = s->stats[slot];
    r.state = 2;
    s->palloc.release(r.off, r.bytes);
    s->slot_job[slot] = 0;
    sl->seq = 0;
    s->free_slots.push_back(slot);
  }
}

// The large job at the head of the arrival order, once no small job is on the
// device and the persistent kernel has closed: tracked by the single-path
// tracker on the whole GPU (the lock is released meanwhile).
static bool run_big_locked(ph_server *s, std::unique_lock<std::mutex> &lk) {
  if (s->waiting.empty()) return false;
  const int64_t id = s->waiting.front();
  JobRec &r = s->jobs[id];
  if (!r.big) return false;
  for (int64_t sj : s->slot_job)
    if (sj != 0) return false;
  if (s->launched && cudaStreamQuery(s->stream) == cudaErrorNotReady) return false;
  cudaGetLastError();
  s->waiting.pop_front();
  r.state = 1;
  std::vector<double> xo(r.x0.size());
  ph_path_stats st;
  memset(&st, 0, sizeof st);
  lk.unlock();
  ph_status status = ph_track_path_exec(s->big_ctx, r.f, r.g, r.gamma.data(), r.x0.data(), &r.p,
                                        xo.data(), &st, nullptr, 0);
  lk.lock();
  if (status != PH_OK && st.status == PH_OK) st.status = status;
  r.x_out = std::move(xo);
  r.stats = st;
  r.t_done = clk::now();
  r.state = 2;
  s->big_done += 1;
  return true;
}

static void server_loop(ph_server *s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    reap_locked(s);
    if (run_big_locked(s, lk)) continue;
    admit_locked(s);
    // a kernel is needed while a published job is unclaimed
    bool pending = false;
    for (int slot = 0; slot < s->cap && !pending; ++slot) {
      const int64_t id = s->slot_job[slot];
      pending = id != 0 && s->slots[slot].claimed != (unsigned long long)id;
    }
    if (pending) {
      bool running = s->launched && cudaStreamQuery(s->stream) == cudaErrorNotReady;
      if (!running) {
        cudaGetLastError();
        Ctl *c = s->ctl.as<Ctl>();
        k_reopen<<<1, 1, 0, s->stream>>>(c);
        k_serve<<<s->grid, kBT, s->smem, s->stream>>>(s->slots, s->queue, s->q, c, s->cap);
        if (cudaGetLastError() != cudaSuccess) s->err = "k_serve launch failed";
        s->launched = true;
        s->launches += 1;
      }
    }
    s->cv.notify_all();
    s->cv.wait_for(lk, std::chrono::microseconds(20));
  }
}

extern "C" ph_status ph_server_create(ph_ctx *ctx, const ph_server_config *cfg, ph_server **out) {
  if (!ctx) return PH_EINVAL;
  if (!cfg || !out || cfg->max_n < 1 || cfg->max_n > 4096 || cfg->pool_bytes <= 0 ||
      cfg->queue_cap < 1 || cfg->queue_cap > 65536)
    return ph_fail(ctx, PH_EINVAL, "ph_server_create: invalid configuration");
  cudaSetDevice(ctx->device);
  ph_server *s = new (std::nothrow) ph_server();
  if (!s) return ph_fail(ctx, PH_ENOMEM, "ph_server_create: out of host memory");
  s->ctx = ctx;
  s->cfg = *cfg;
  s->cap = cfg->queue_cap;
  s->slot_doubles = (size_t)16 * cfg->max_n + 8;
  s->smem = job_smem_bytes(4, cfg->max_n);
  cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess && s->smem > 48 * 1024)
    e = cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem);
  int bps = 1;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_serve, kBT, s->smem);
  if (bps < 1) bps = 1;
  if (bps > 2) bps = 2;
  s->grid = cfg->max_blocks > 0 ? cfg->max_blocks : ctx->sm_count * bps;
  if (s->grid > ctx->sm_count * bps) s->grid = ctx->sm_count * bps;
  unsigned flags = cudaHostAllocMapped;
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->slots, sizeof(Slot) * s->cap, flags);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->queue, sizeof(int) * s->cap, flags);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->q, sizeof(Queue), flags);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->bufs, sizeof(double) * s->slot_doubles * s->cap, flags);
  if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->stats, sizeof(ph_path_stats) * s->cap, flags);
  if (e == cudaSuccess) e = s->pool.ensure((size_t)cfg->pool_bytes);
  if (e == cudaSuccess) e = s->ctl.ensure(sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMemset(s->ctl.p, 0, sizeof(Ctl));
  if (e == cudaSuccess && cfg->big_n > 0) {
    e = cudaStreamCreateWithFlags(&s->big_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && ph_init(&s->big_ctx, ctx->device, s->big_stream) != PH_OK)
      e = cudaErrorInitializationError;
  }
  if (e != cudaSuccess) {
    ph_status st = ph_cuda_fail(ctx, e, "ph_server_create");
    ph_server_destroy(s);
    return st;
  }
  memset((void *)s->slots, 0, sizeof(Slot) * s->cap);
  memset((void *)s->q, 0, sizeof(Queue));
  s->palloc.init((size_t)cfg->pool_bytes);
  s->slot_job.assign(s->cap, 0);
  for (int i = s->cap - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->worker = std::thread(server_loop, s);
  *out = s;
  return PH_OK;
}

extern "C" ph_status ph_server_submit(ph_server *s, const ph_system *f, const ph_system *g,
                                      const double *gamma, const double *x0,
                                      const ph_track_params *params, int64_t *job_id) {
  if (!s) return PH_EINVAL;
  ph_ctx *ctx = s->ctx;
  if (!f || f->ctx != ctx || !gamma || !x0 || !params || !job_id)
    return ph_fail(ctx, PH_EINVAL, "ph_server_submit: invalid argument");
  if (g && (g->ctx != ctx || g->L != f->L || g->N != f->N || g->n != f->n))
    return ph_fail(ctx, PH_EINVAL, "ph_server_submit: g does not match f");
  const bool big = s->cfg.big_n > 0 && f->n > s->cfg.big_n;
  if (!big && f->n > s->cfg.max_n)
    return ph_fail(ctx, PH_EINVAL, "ph_server_submit: more variables than max_n");
  if (big && params->lin_prec != 0 && params->lin_prec != 1)
    return ph_fail(ctx, PH_EINVAL, "ph_server_submit: a large job takes lin_prec 0 or 1");
  const ph_track_params &p = *params;
  if (p.max_newton < 1 || p.max_newton > 64 || p.pred_order < 0 || p.pred_order > 8 ||
      p.relax_k < 1 || p.relax_k > 64 || p.max_steps < 0 || p.lin_prec < 0 || p.lin_prec > 3 ||
      p.fixed_rows < 0 || p.fixed_rows > 1 || (p.fixed_rows && !g) ||
      (p.fixed_steps <= 0 && !(p.max_dt > 0.0 && p.min_dt > 0.0 && p.min_dt <= p.max_dt)))
    return ph_fail(ctx, PH_EINVAL, "ph_server_submit: invalid parameters");
  if (!g) {
    if (f->N != f->n) return ph_fail(ctx, PH_EINVAL, "ph_server_submit: the total-degree start system needs N == n");
    for (int d : f->h_deg)
      if (d < 1) return ph_fail(ctx, PH_EINVAL, "ph_server_submit: f has a constant polynomial");
  }
  cudaSetDevice(ctx->device);
  JobRec r;
  memset(&r.job, 0, sizeof r.job);
  ph_job_fill_system(r.job, f, g);
  r.job.p = p;
  r.bytes = sizeof(double) * (size_t)ph_job_ws_doubles(r.job);
  r.big = big;
  r.f = f;
  r.g = g;
  r.p = p;
  if (!big && r.bytes > (size_t)s->cfg.pool_bytes)
    return ph_fail(ctx, PH_ENOMEM, "ph_server_submit: the job's workspace exceeds the pool");
  const int L = f->L;
  r.x0.resize((size_t)2 * L * f->n);
  r.gamma.resize((size_t)2 * L);
  PH_CUDA(ctx, cudaMemcpy(r.x0.data(), x0, sizeof(double) * r.x0.size(), cudaMemcpyDefault));
  PH_CUDA(ctx, cudaMemcpy(r.gamma.data(), gamma, sizeof(double) * r.gamma.size(), cudaMemcpyDefault));
  memset(&r.stats, 0, sizeof r.stats);
  r.t_submit = clk::now();
  std::lock_guard<std::mutex> lk(s->mu);
  const int64_t id = s->next_id++;
  s->jobs.emplace(id, std::move(r));
  s->waiting.push_back(id);
  admit_locked(s);
  *job_id = id;
  return PH_OK;
}

static ph_status take_result(ph_server *s, JobRec &r, double *x_out, ph_path_stats *stats,
                             double *latency_ms) {
  if (x_out) {
    cudaError_t e = cudaMemcpy(x_out, r.x_out.data(), sizeof(double) * r.x_out.size(), cudaMemcpyDefault);
    if (e != cudaSuccess) return ph_cuda_fail(s->ctx, e, "ph_server result copy");
  }
  if (stats) *stats = r.stats;
  if (latency_ms)
    *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
  return PH_OK;
}

extern "C" ph_status ph_server_poll(ph_server *s, int64_t job_id, int *done, double *x_out,
                                    ph_path_stats *stats, double *latency_ms) {
  if (!s || !done) return PH_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return ph_fail(s->ctx, PH_EINVAL, "ph_server_poll: unknown job");
  *done = it->second.state == 2;
  if (!*done) return PH_OK;
  ph_status st = take_result(s, it->second, x_out, stats, latency_ms);
  s->jobs.erase(it);
  return st;
}

extern "C" ph_status ph_server_wait(ph_server *s, int64_t job_id, int timeout_ms, double *x_out,
                                    ph_path_stats *stats, double *latency_ms) {
  if (!s) return PH_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto deadline = clk::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return ph_fail(s->ctx, PH_EINVAL, "ph_server_wait: unknown job");
    if (it->second.state == 2) {
      ph_status st = take_result(s, it->second, x_out, stats, latency_ms);
      s->jobs.erase(it);
      return st;
    }
    if (clk::now() >= deadline) return ph_fail(s->ctx, PH_TIMEOUT, "ph_server_wait: not done yet");
    s->cv.wait_for(lk, std::chrono::milliseconds(1));
  }
}

extern "C" ph_status ph_server_info(ph_server *s, int64_t *waiting, int64_t *on_device,
                                    int64_t *kernel_launches, int64_t *pool_free_bytes) {
  if (!s) return PH_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t w = 0, d = 0;
  for (auto &kv : s->jobs) {
    if (kv.second.state == 0) ++w;
    if (kv.second.state == 1) ++d;
  }
  if (waiting) *waiting = w;
  if (on_device) *on_device = d;
  if (kernel_launches) *kernel_launches = s->launches;
  if (pool_free_bytes) {
    size_t fr = 0;
    for (auto &kv : s->palloc.free_) fr += kv.second;
    *pool_free_bytes = (int64_t)fr;
  }
  return PH_OK;
}

extern "C" ph_status ph_server_job_bytes(ph_server *s, const ph_system *f, const ph_system *g,
                                         int64_t *bytes) {
  if (!s || !f || !bytes) return PH_EINVAL;
  Job j;
  memset(&j, 0, sizeof j);
  ph_job_fill_system(j, f, g);
  *bytes = (int64_t)((sizeof(double) * (size_t)ph_job_ws_doubles(j) + 255) / 256 * 256);
  return PH_OK;
}

extern "C" ph_status ph_server_destroy(ph_server *s) {
  if (!s) return PH_EINVAL;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
      if (s->q) s->q->shutdown = 1;
    }
    s->worker.join();
  }
  if (s->stream) {
    cudaStreamSynchronize(s->stream);
    cudaStreamDestroy(s->stream);
  }
  if (s->big_ctx) ph_destroy(s->big_ctx);
  if (s->big_stream) cudaStreamDestroy(s->big_stream);
  if (s->slots) cudaFreeHost(s->slots);
  if (s->queue) cudaFreeHost(s->queue);
  if (s->q) cudaFreeHost(s->q);
  if (s->bufs) cudaFreeHost(s->bufs);
  if (s->stats) cudaFreeHost(s->stats);
  s->pool.release();
  s->ctl.release();
  delete s;
  return PH_OK;
}
