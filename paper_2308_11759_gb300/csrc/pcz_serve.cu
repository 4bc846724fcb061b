// pcz_serve.cu -- progressive-query server over device-resident component
// streams (Sec. 6.1: keep the components compressed and decode and add blocks
// on demand to form the requested pieces of x~; Sec. 6.2: a query consults the
// per-component tolerances for the number of components, and more precision
// is more components added to the current approximation).
//
// Per field the server keeps a cache of partial sums x~ and, per brick, the k
// the cache holds.  A batch of queries is one launch of the retrieval kernel
// over a list of box jobs; a brick whose cached k is at most the query's k
// starts from the cache and decodes only the components above it, every other
// brick decodes from its first component.  Both give the same bits, because
// Algorithm 2's partial sums are formed in one fixed order.  After the batch,
// bricks that a query produced in full at a k above their cached one are
// written back into the cache (one winner per brick).
//
// Scheduling (continuous batching): a dispatcher thread owned by the server
// admits queries in submission order as long as their output boxes fit in an
// arena sized by the device memory budget, and launches the admitted queries
// of one type as one batch into a free slot.  Each slot has its own CUDA
// stream, so batches launched while others are still running execute
// concurrently on the device.  A batch that reads or writes back cache bricks
// of a field region that an in-flight batch also touches waits for that
// batch first (both the cache reads and the write-back of a brick are then
// ordered); batches on disjoint regions do not wait.  A host function queued
// behind each batch tells the dispatcher when it has completed, so nothing
// polls: the dispatcher sleeps on a condition variable until a query arrives
// or a batch completes.  Queries arrive through pc_server_submit (online) or
// pc_server_replay (a recorded stream with arrival times).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "pcz_host.h"

namespace pcz {

// Where a job's cache writes go: the field's cache, its per-brick levels and
// claims, the job's first brick among all bricks of the batch, and the job's
// claim key (k above the job's index in the batch, so that the largest k
// wins and ties go to one job).
struct CacheAux {
  void* cache;
  uint8_t* level;
  uint32_t* pend;
  int64_t brick_begin;
  uint32_t key;
  int pad_;
};

__device__ __forceinline__ int find_job(const CacheAux* aux, int njobs, int64_t item) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (aux[mid].brick_begin <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Brick g of job J (box order, x fastest): coordinates, and whether all of
// its in-field values lie inside the box (so the job's output holds it whole).
__device__ __forceinline__ bool brick_covered(const BoxJob& J, int64_t g, int64_t bc[3]) {
  bc[0] = J.bl[0] + g % J.bn[0];
  const int64_t r = g / J.bn[0];
  bc[1] = J.bl[1] + r % J.bn[1];
  bc[2] = J.bl[2] + r / J.bn[1];
  bool in = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int64_t e0 = 4 * bc[a], e1 = min(4 * bc[a] + 4, J.dims[a]);
    in = in && J.lo[a] <= e0 && e1 <= J.hi[a];
  }
  return in;
}

__global__ void __launch_bounds__(256) k_cache_claim(const BoxJob* __restrict__ jobs,
                                                     const CacheAux* __restrict__ aux, int njobs, int64_t nitems) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nitems; i += stride) {
    const int j = find_job(aux, njobs, i);
    const BoxJob& J = jobs[j];
    int64_t bc[3];
    if (!brick_covered(J, i - aux[j].brick_begin, bc)) continue;
    const int64_t b = bc[0] + J.nb[0] * (bc[1] + J.nb[1] * bc[2]);
    if (J.k > (int)aux[j].level[b]) atomicMax(aux[j].pend + b, aux[j].key);
  }
}

// 16 threads per brick, one x-line each.  A claim key carries k in its top
// bits and the cached level only grows, so a stale key from an earlier batch
// never equals a new winner's key: claims need no reset.
template <typename T>
__global__ void __launch_bounds__(256) k_cache_fill(const BoxJob* __restrict__ jobs,
                                                    const CacheAux* __restrict__ aux, int njobs, int64_t nitems) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nitems * 16; i += stride) {
    const int64_t item = i >> 4;
    const int t = (int)(i & 15);
    const int j = find_job(aux, njobs, item);
    const BoxJob& J = jobs[j];
    int64_t bc[3];
    if (!brick_covered(J, item - aux[j].brick_begin, bc)) continue;
    const int64_t b = bc[0] + J.nb[0] * (bc[1] + J.nb[1] * bc[2]);
    if (aux[j].pend[b] != aux[j].key) continue;
    const int64_t y = 4 * bc[1] + (t & 3), z = 4 * bc[2] + (t >> 2);
    if (y < J.dims[1] && z < J.dims[2]) {
      T* cache = reinterpret_cast<T*>(aux[j].cache);
      const T* out = reinterpret_cast<const T*>(J.out);
      const int64_t ext0 = J.hi[0] - J.lo[0], ext1 = J.hi[1] - J.lo[1];
      const int64_t orow = ((z - J.lo[2]) * ext1 + (y - J.lo[1])) * ext0 - J.lo[0];
      const int64_t frow = (z * J.dims[1] + y) * J.dims[0];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int64_t x = 4 * bc[0] + m;
        if (x < J.dims[0]) cache[frow + x] = out[orow + x];
      }
    }
    if (t == 0) aux[j].level[b] = (uint8_t)J.k;
  }
}

static cudaError_t launch_cache_update(int dtype, const BoxJob* jobs, const CacheAux* aux, int njobs,
                                       int64_t nitems, cudaStream_t s) {
  if (nitems == 0) return cudaSuccess;
  auto blocks = [](int64_t work) {
    int64_t b = (work + 255) / 256;
    return (unsigned)(b > 152 * 16 ? 152 * 16 : b);
  };
  k_cache_claim<<<blocks(nitems), 256, 0, s>>>(jobs, aux, njobs, nitems);
  if (dtype == 1)
    k_cache_fill<float><<<blocks(nitems * 16), 256, 0, s>>>(jobs, aux, njobs, nitems);
  else
    k_cache_fill<double><<<blocks(nitems * 16), 256, 0, s>>>(jobs, aux, njobs, nitems);
  return cudaGetLastError();
}

}  // namespace pcz

using namespace pcz;

namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxSlots = 4;  // batches in flight at once

struct ServeField {
  const pc_streams* s = nullptr;
  void* cache = nullptr;      // x~ at the cached level, whole field
  uint8_t* level = nullptr;   // per brick
  uint32_t* pend = nullptr;   // per brick: claim of the batch being written back
  uint64_t bytes = 0;         // device bytes counted against the budget
};

struct Query {
  int field, k;
  int64_t lo[3], hi[3];
  uint64_t bytes;
  pc_dtype dtype;
};

// One submitted query and its progress.
struct Request {
  Query q;
  void* d_out = nullptr;   // caller's buffer for a copy of the result (may be null)
  uint64_t off = 0;        // its box in the arena while it runs
  uint64_t arena_seq = 0;  // its arena entry
  double t_arrive = 0.0;   // seconds since the server's clock origin
  double t_done = -1.0;
  bool done = false;
};

// The brick region of one field that a batch reads (and may write back).
struct FieldRegion {
  int field;
  int64_t lo[3], hi[3];  // brick units, half-open
};

}  // namespace

struct pc_server;

namespace {

struct Slot {
  pc_server* S = nullptr;
  int index = 0;
  BoxJob* h_jobs = nullptr;  // pinned
  CacheAux* h_aux = nullptr;
  BoxJob* d_jobs = nullptr;
  CacheAux* d_aux = nullptr;
  uint64_t* spill = nullptr;  // the retrieval kernel's per-CTA spill, one area per slot
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<uint64_t> reqs;  // request ids of the batch
  std::vector<Query> qs;       // their queries (copies)
  std::vector<uint64_t> offs;
  std::vector<void*> outs;
  std::vector<FieldRegion> regions;
  bool busy = false;
  double t_done = 0.0;  // set by the completion callback
};

// FIFO arena for output boxes: entries are allocated in submission order and
// released when their batch completes (in any order); the space of a released
// entry returns once every older entry is released too, so the live region
// stays one contiguous run, possibly wrapped.
struct Arena {
  uint64_t cap = 0;
  struct Entry {
    uint64_t lo, hi;
    bool freed;
  };
  std::deque<Entry> live;
  uint64_t base_seq = 0;  // sequence number of live.front()
  uint64_t in_use = 0;
  bool alloc(uint64_t n, uint64_t* off, uint64_t* seq) {
    n = (n + 255) & ~255ull;
    uint64_t o;
    if (live.empty()) {
      if (n > cap) return false;
      o = 0;
    } else {
      const uint64_t tail = live.front().lo, head = live.back().hi;
      if (live.back().lo >= tail) {  // live = [tail, head)
        if (cap - head >= n)
          o = head;
        else if (tail >= n)
          o = 0;
        else
          return false;
      } else {  // live = [tail, cap) + [0, head)
        if (tail - head >= n)
          o = head;
        else
          return false;
      }
    }
    live.push_back({o, o + n, false});
    in_use += n;
    *off = o;
    *seq = base_seq + live.size() - 1;
    return true;
  }
  void release(uint64_t seq) {
    live[(size_t)(seq - base_seq)].freed = true;
    while (!live.empty() && live.front().freed) {
      in_use -= live.front().hi - live.front().lo;
      live.pop_front();
      ++base_seq;
    }
  }
  void clear() {
    base_seq += live.size();
    live.clear();
    in_use = 0;
  }
};

}  // namespace

struct pc_server {
  int device = 0;
  cudaStream_t user_st = nullptr;  // the caller's stream at creation (fields were made on it)
  uint64_t budget = 0;
  int max_batch = 1;
  int flags = 0;
  std::vector<ServeField> fields;
  uint64_t fixed = 0;  // fields, caches, job buffers, spill
  char* arena_mem = nullptr;
  Arena arena;
  size_t spill_words = 0;  // per slot
  unsigned int* d_err = nullptr;
  Slot slots[kMaxSlots];
  int nslots = 2;
  // dispatcher state, guarded by mu
  std::mutex mu;
  std::condition_variable cv;       // wakes the dispatcher
  std::condition_variable cv_done;  // wakes callers waiting for results
  std::thread worker;
  bool running = false, stopping = false;
  bool mem_blocked = false;      // the oldest pending query waits for arena space
  std::deque<uint64_t> pending;  // submitted, not yet admitted
  std::deque<int> completed;     // slots whose batch has completed
  std::vector<Request> reqs;
  uint64_t done_count = 0;
  Clock::time_point t0;
  pc_status err = PC_OK;
  std::string err_msg;
  // counters since creation
  uint64_t batches = 0, launched = 0, bytes_out = 0, peak_arena = 0, max_seen = 0;
  int inflight = 0, max_inflight = 0;
};

namespace {

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

void CUDART_CB batch_done(void* p) {  // runs on a CUDA-internal thread: no CUDA calls here
  Slot* sl = static_cast<Slot*>(p);
  pc_server* S = sl->S;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    sl->t_done = seconds_since(S->t0);
    S->completed.push_back(sl->index);
  }
  S->cv.notify_one();
}

bool regions_overlap(const std::vector<FieldRegion>& a, const std::vector<FieldRegion>& b) {
  for (const FieldRegion& x : a)
    for (const FieldRegion& y : b) {
      if (x.field != y.field) continue;
      bool ov = true;
      for (int d = 0; d < 3; ++d) ov = ov && x.lo[d] < y.hi[d] && y.lo[d] < x.hi[d];
      if (ov) return true;
    }
  return false;
}

// Issues one batch on its slot's stream: waits for in-flight batches whose
// cache regions overlap, the box jobs, the retrieval kernel, the cache
// write-back, the copies into the callers' buffers, then the completion
// callback.  Called by the dispatcher without the lock held; `others` are the
// slots in flight when it was admitted.
cudaError_t issue_batch(pc_server* S, Slot& sl, const std::vector<int>& others) {
  TraceRange trace_("pc_server batch");
  const bool cache = !(S->flags & PC_SERVE_NO_CACHE);
  const int nj = (int)sl.qs.size();
  const pc_dtype dt = sl.qs[0].dtype;
  cudaError_t e = cudaSuccess;
  if (cache)
    for (int o : others)
      if (regions_overlap(sl.regions, S->slots[o].regions)) {
        e = cudaStreamWaitEvent(sl.st, S->slots[o].done, 0);
        if (e != cudaSuccess) return e;
      }
  int64_t nunits = 0, nitems = 0;
  for (int j = 0; j < nj; ++j) {
    const Query& q = sl.qs[j];
    const ServeField& F = S->fields[q.field];
    BoxJob J = make_box_job(F.s, 0, q.k, q.lo, q.hi, S->arena_mem + sl.offs[j]);
    J.unit_begin = nunits;
    if (cache) {
      J.cache = F.cache;
      J.level = F.level;
    }
    nunits += box_job_units(J);
    sl.h_jobs[j] = J;
    CacheAux A;
    A.cache = F.cache;
    A.level = F.level;
    A.pend = F.pend;
    A.brick_begin = nitems;
    A.key = ((uint32_t)q.k << 16) | (uint32_t)j;
    A.pad_ = 0;
    sl.h_aux[j] = A;
    nitems += J.nbox;
  }
  e = cudaMemcpyAsync(sl.d_jobs, sl.h_jobs, sizeof(BoxJob) * nj, cudaMemcpyHostToDevice, sl.st);
  if (e == cudaSuccess && cache)
    e = cudaMemcpyAsync(sl.d_aux, sl.h_aux, sizeof(CacheAux) * nj, cudaMemcpyHostToDevice, sl.st);
  if (e != cudaSuccess) return e;
  RetrieveParams R;
  std::memset(&R, 0, sizeof(R));
  R.jobs = sl.d_jobs;
  R.njobs = nj;
  R.nunits = nunits;
  R.write = 1;
  R.err = S->d_err;
  R.spill = sl.spill;
  R.grid = retrieve_grid(dt, 3, nunits);
  e = launch_retrieve(dt, 3, R, sl.st);
  if (e == cudaSuccess && cache) e = launch_cache_update(dt, sl.d_jobs, sl.d_aux, nj, nitems, sl.st);
  for (int j = 0; j < nj && e == cudaSuccess; ++j)
    if (sl.outs[j])
      e = cudaMemcpyAsync(sl.outs[j], S->arena_mem + sl.offs[j], sl.qs[j].bytes, cudaMemcpyDeviceToDevice, sl.st);
  if (e == cudaSuccess) e = cudaEventRecord(sl.done, sl.st);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(sl.st, batch_done, &sl);
  return e;
}

// The dispatcher: completions, then admission and launch, until stopped with
// nothing left to do.
void dispatch(pc_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    auto free_slot = [&]() {
      for (int i = 0; i < S->nslots; ++i)
        if (!S->slots[i].busy) return i;
      return -1;
    };
    S->cv.wait(lk, [&] {
      return !S->completed.empty() || (S->stopping && S->pending.empty() && S->inflight == 0) ||
             (!S->pending.empty() && !S->mem_blocked && free_slot() >= 0);
    });
    // completions: the batch's results are in the callers' buffers
    bool finished = false;
    while (!S->completed.empty()) {
      Slot& sl = S->slots[S->completed.front()];
      S->completed.pop_front();
      for (uint64_t id : sl.reqs) {
        Request& r = S->reqs[id];
        r.t_done = sl.t_done;
        r.done = true;
        S->arena.release(r.arena_seq);
        ++S->done_count;
      }
      sl.reqs.clear();
      sl.busy = false;
      --S->inflight;
      finished = true;
      S->mem_blocked = false;
    }
    if (finished) S->cv_done.notify_all();
    if (S->stopping && S->pending.empty() && S->inflight == 0) break;
    // admission and launch while a slot is free and the arena has room
    int si;
    while (!S->pending.empty() && (si = free_slot()) >= 0) {
      Slot& sl = S->slots[si];
      sl.qs.clear();
      sl.offs.clear();
      sl.outs.clear();
      sl.regions.clear();
      const pc_dtype dt = S->reqs[S->pending.front()].q.dtype;
      while (!S->pending.empty() && (int)sl.reqs.size() < S->max_batch) {
        Request& r = S->reqs[S->pending.front()];
        if (r.q.dtype != dt) break;
        if (!S->arena.alloc(r.q.bytes, &r.off, &r.arena_seq)) break;  // admission by memory
        sl.reqs.push_back(S->pending.front());
        sl.qs.push_back(r.q);
        sl.offs.push_back(r.off);
        sl.outs.push_back(r.d_out);
        bool merged = false;  // the batch's brick region per field (a bounding box)
        for (FieldRegion& g : sl.regions)
          if (g.field == r.q.field) {
            for (int d = 0; d < 3; ++d) {
              g.lo[d] = std::min(g.lo[d], r.q.lo[d] / 4);
              g.hi[d] = std::max(g.hi[d], (r.q.hi[d] + 3) / 4);
            }
            merged = true;
          }
        if (!merged) {
          FieldRegion g;
          g.field = r.q.field;
          for (int d = 0; d < 3; ++d) {
            g.lo[d] = r.q.lo[d] / 4;
            g.hi[d] = (r.q.hi[d] + 3) / 4;
          }
          sl.regions.push_back(g);
        }
        S->pending.pop_front();
      }
      if (sl.reqs.empty()) {  // the oldest query waits for memory: until a batch completes
        S->mem_blocked = true;
        break;
      }
      std::vector<int> others;
      for (int i = 0; i < S->nslots; ++i)
        if (S->slots[i].busy) others.push_back(i);
      sl.busy = true;
      ++S->inflight;
      S->max_inflight = std::max(S->max_inflight, S->inflight);
      S->peak_arena = std::max(S->peak_arena, S->arena.in_use);
      ++S->batches;
      S->launched += sl.reqs.size();
      S->max_seen = std::max(S->max_seen, (uint64_t)sl.reqs.size());
      for (const Query& q : sl.qs) S->bytes_out += q.bytes;
      lk.unlock();
      const cudaError_t e = issue_batch(S, sl, others);
      lk.lock();
      if (e != cudaSuccess && S->err == PC_OK) {
        S->err = api_cuda_fail(e, "server batch");
        S->err_msg = pc_last_error();
      }
      if (e != cudaSuccess) {  // nothing will complete this batch: finish it here
        cudaGetLastError();
        for (uint64_t id : sl.reqs) {
          S->reqs[id].done = true;
          S->arena.release(S->reqs[id].arena_seq);
          ++S->done_count;
        }
        sl.reqs.clear();
        sl.busy = false;
        --S->inflight;
        S->cv_done.notify_all();
      }
    }
  }
}

// Starts the dispatcher (and allocates the arena from what the budget leaves)
// on first use; the caller holds no lock.
pc_status ensure_started(pc_server* S) {
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->running) return PC_OK;
  if (S->fields.empty()) return api_fail(PC_ERR_ARG, "no fields");
  if (!S->arena_mem) {
    const uint64_t room = S->budget - S->fixed;
    S->arena.cap = room & ~255ull;
    cudaError_t e = S->arena.cap ? cudaMalloc((void**)&S->arena_mem, S->arena.cap) : cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
      S->arena.cap = 0;
      return api_cuda_fail(e, "arena allocation");
    }
  }
  // batches start after the work queued so far on the caller's stream
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, S->user_st);
  for (int i = 0; i < S->nslots && e == cudaSuccess; ++i) e = cudaStreamWaitEvent(S->slots[i].st, ev, 0);
  if (e == cudaSuccess) e = cudaEventDestroy(ev);
  if (e != cudaSuccess) return api_cuda_fail(e, "server start");
  S->t0 = Clock::now();
  S->stopping = false;
  S->running = true;
  S->worker = std::thread(dispatch, S);
  return PC_OK;
}

// Drains and joins the dispatcher.
void stop_worker(pc_server* S) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->running) return;
    S->stopping = true;
  }
  S->cv.notify_one();
  S->worker.join();
  std::lock_guard<std::mutex> lk(S->mu);
  S->running = false;
  S->stopping = false;
}

void server_release(pc_server* S) {
  if (!S) return;
  stop_worker(S);
  for (Slot& sl : S->slots)
    if (sl.st) cudaStreamSynchronize(sl.st);
  for (ServeField& f : S->fields) {
    cudaFree(f.cache);
    cudaFree(f.level);
    cudaFree(f.pend);
  }
  for (Slot& sl : S->slots) {
    cudaFreeHost(sl.h_jobs);
    cudaFreeHost(sl.h_aux);
    cudaFree(sl.d_jobs);
    cudaFree(sl.d_aux);
    cudaFree(sl.spill);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.st) cudaStreamDestroy(sl.st);
  }
  cudaFree(S->arena_mem);
  cudaFree(S->d_err);
  delete S;
}

#define SK(call)                                                    \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return api_cuda_fail(e_, #call);         \
  } while (0)

// Resolves and checks one query (PC_ERR_ARG, PC_ERR_TOL_UNREACHABLE).
pc_status resolve(const pc_server* S, const pc_query& in, Query* q) {
  if (in.field < 0 || in.field >= (int)S->fields.size()) return api_fail(PC_ERR_ARG, "bad field index");
  const pc_streams* s = S->fields[in.field].s;
  q->field = in.field;
  q->dtype = s->dtype;
  if (in.k > 0) {
    if (in.k > s->n) return api_fail(PC_ERR_ARG, "k out of range");
    q->k = in.k;
  } else {
    pc_status r = pc_query_k(s, in.tau, &q->k);
    if (r != PC_OK) return r;
  }
  pc_status r = check_box(s, &in.box, q->lo, q->hi);
  if (r != PC_OK) return r;
  q->bytes = (uint64_t)((q->hi[0] - q->lo[0]) * (q->hi[1] - q->lo[1]) * (q->hi[2] - q->lo[2])) * dtype_size(q->dtype);
  return PC_OK;
}

// Queues a resolved query arriving at t_arrive (seconds on the server clock).
uint64_t enqueue(pc_server* S, const Query& q, void* d_out, double t_arrive) {
  uint64_t id;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    id = S->reqs.size();
    Request r;
    r.q = q;
    r.d_out = d_out;
    r.t_arrive = t_arrive;
    S->reqs.push_back(r);
    S->pending.push_back(id);
  }
  S->cv.notify_one();
  return id;
}

void fill_stats(pc_server* S, pc_serve_stats* st, double wall, uint64_t b0, uint64_t q0, uint64_t o0) {
  std::memset(st, 0, sizeof(*st));
  st->wall_s = wall;
  st->batches = S->batches - b0;
  st->queries = S->launched - q0;
  st->bytes_out = S->bytes_out - o0;
  st->max_batch = S->max_seen;
  st->peak_device_bytes = S->fixed + S->peak_arena;
  st->arena_bytes = S->arena.cap;
  st->max_inflight = (uint64_t)S->max_inflight;
}

}  // namespace

extern "C" {

pc_status pc_server_create(uint64_t hbm_budget_bytes, int max_batch, int flags, void* cuda_stream,
                           pc_server** out) {
  if (!out) return api_fail(PC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (max_batch < 1 || max_batch > 65535) return api_fail(PC_ERR_ARG, "max_batch must be in [1, 65535]");
  if (flags & ~(PC_SERVE_NO_CACHE | PC_SERVE_SERIAL)) return api_fail(PC_ERR_ARG, "unknown flags");
  pc_server* S = new pc_server();
  S->budget = hbm_budget_bytes;
  S->max_batch = (flags & PC_SERVE_SERIAL) ? 1 : max_batch;
  S->flags = flags;
  S->nslots = (flags & PC_SERVE_SERIAL) ? 1 : kMaxSlots;
  S->user_st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&S->device);
  for (int i = 0; i < kMaxSlots; ++i) {
    Slot& sl = S->slots[i];
    sl.S = S;
    sl.index = i;
    if (i >= S->nslots) continue;
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_jobs, sizeof(BoxJob) * S->max_batch);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_aux, sizeof(CacheAux) * S->max_batch);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_jobs, sizeof(BoxJob) * S->max_batch);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_aux, sizeof(CacheAux) * S->max_batch);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_err, 16);
  if (e == cudaSuccess) e = cudaMemset(S->d_err, 0, 16);
  if (e != cudaSuccess) {
    server_release(S);
    return api_cuda_fail(e, "server allocation");
  }
  S->fixed = (uint64_t)S->nslots * (sizeof(BoxJob) + sizeof(CacheAux)) * (uint64_t)S->max_batch + 16;
  if (S->fixed > S->budget) {
    server_release(S);
    return api_fail(PC_ERR_OOM, "budget below the server's own buffers");
  }
  *out = S;
  return PC_OK;
}

pc_status pc_server_add_field(pc_server* S, const pc_streams* s, int* field) {
  if (!S || !s || !field) return api_fail(PC_ERR_ARG, "NULL argument");
  if (s->ndims != 3) return api_fail(PC_ERR_ARG, "the server takes 3D fields");
  if (s->device != S->device) return api_fail(PC_ERR_ARG, "streams live on another device");
  if (S->arena_mem) return api_fail(PC_ERR_ARG, "fields must be added before the first query");
  ServeField F;
  F.s = s;
  const uint64_t vals = (uint64_t)(s->dims[0] * s->dims[1] * s->dims[2]);
  uint64_t stream_bytes = 0;
  for (int i = 0; i < s->n; ++i) stream_bytes += 8 * s->words[i];
  stream_bytes += (uint64_t)s->n * (8 * s->nchunks + 6 * s->nbricks) + sizeof(CompDesc) * s->n;
  const bool cache = !(S->flags & PC_SERVE_NO_CACHE);
  F.bytes = stream_bytes + (cache ? vals * dtype_size(s->dtype) + 5 * (uint64_t)s->nbricks : 0);
  if (S->fixed + F.bytes > S->budget) return api_fail(PC_ERR_OOM, "the field does not fit in the budget");
  if (cache) {
    cudaError_t e = cudaMalloc(&F.cache, vals * dtype_size(s->dtype));
    if (e == cudaSuccess) e = cudaMalloc((void**)&F.level, s->nbricks);
    if (e == cudaSuccess) e = cudaMalloc((void**)&F.pend, 4 * s->nbricks);
    if (e == cudaSuccess) e = cudaMemset(F.level, 0, s->nbricks);
    if (e == cudaSuccess) e = cudaMemset(F.pend, 0, 4 * s->nbricks);
    if (e != cudaSuccess) {
      cudaFree(F.cache);
      cudaFree(F.level);
      cudaFree(F.pend);
      return api_cuda_fail(e, "cache allocation");
    }
  }
  // per-CTA spill of the retrieval kernel at its largest grid, one area per slot
  const size_t sw = retrieve_spill_words(s->dtype, 3, retrieve_grid(s->dtype, 3, (int64_t)1 << 40));
  if (sw > S->spill_words) {
    const uint64_t grow = 8 * (uint64_t)(sw - S->spill_words) * (uint64_t)S->nslots;
    if (S->fixed + F.bytes + grow > S->budget) {
      cudaFree(F.cache);
      cudaFree(F.level);
      cudaFree(F.pend);
      return api_fail(PC_ERR_OOM, "the field does not fit in the budget");
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < S->nslots; ++i) {
      cudaFree(S->slots[i].spill);
      S->slots[i].spill = nullptr;
      if (e == cudaSuccess) e = cudaMalloc((void**)&S->slots[i].spill, 8 * sw);
    }
    if (e != cudaSuccess) {
      for (int i = 0; i < S->nslots; ++i) {
        cudaFree(S->slots[i].spill);
        S->slots[i].spill = nullptr;
      }
      S->fixed -= 8 * (uint64_t)S->spill_words * (uint64_t)S->nslots;
      S->spill_words = 0;
      cudaFree(F.cache);
      cudaFree(F.level);
      cudaFree(F.pend);
      return api_cuda_fail(e, "spill allocation");
    }
    S->fixed += grow;
    S->spill_words = sw;
  }
  S->fixed += F.bytes;
  S->fields.push_back(F);
  *field = (int)S->fields.size() - 1;
  return PC_OK;
}

pc_status pc_server_reset_cache(pc_server* S) {
  if (!S) return api_fail(PC_ERR_ARG, "NULL server");
  {
    std::unique_lock<std::mutex> lk(S->mu);  // no batch may run while the levels change
    S->cv_done.wait(lk, [&] { return S->pending.empty() && S->inflight == 0; });
  }
  for (int i = 0; i < S->nslots; ++i) SK(cudaStreamSynchronize(S->slots[i].st));
  for (ServeField& f : S->fields)
    if (f.level) SK(cudaMemset(f.level, 0, f.s->nbricks));
  SK(cudaDeviceSynchronize());
  return PC_OK;
}

pc_status pc_server_submit(pc_server* S, const pc_query* query, void* d_out, uint64_t* ticket) {
  if (!S || !query || !ticket) return api_fail(PC_ERR_ARG, "NULL argument");
  Query q;
  pc_status r = resolve(S, *query, &q);
  if (r != PC_OK) return r;
  if (d_out && !device_pointer(d_out)) return api_fail(PC_ERR_ARG, "d_out must be device memory");
  r = ensure_started(S);
  if (r != PC_OK) return r;
  if (((q.bytes + 255) & ~255ull) > S->arena.cap)
    return api_fail(PC_ERR_OOM, "the query's box exceeds the budget left for results");
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->err != PC_OK) return api_fail(S->err, S->err_msg);
  }
  *ticket = enqueue(S, q, d_out, seconds_since(S->t0));
  return PC_OK;
}

pc_status pc_server_poll(pc_server* S, uint64_t ticket, int* done, double* latency_s) {
  if (!S || !done) return api_fail(PC_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (ticket >= S->reqs.size()) return api_fail(PC_ERR_ARG, "unknown ticket");
  const Request& r = S->reqs[ticket];
  *done = r.done ? 1 : 0;
  if (latency_s) *latency_s = r.done ? r.t_done - r.t_arrive : -1.0;
  if (r.done && S->err != PC_OK) return api_fail(S->err, S->err_msg);
  return PC_OK;
}

pc_status pc_server_wait(pc_server* S, uint64_t ticket, double timeout_s, int* done, double* latency_s) {
  if (!S || !done) return api_fail(PC_ERR_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  if (ticket >= S->reqs.size()) return api_fail(PC_ERR_ARG, "unknown ticket");
  auto ready = [&] { return S->reqs[ticket].done; };
  if (timeout_s < 0)
    S->cv_done.wait(lk, ready);
  else
    S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
  const Request& r = S->reqs[ticket];
  *done = r.done ? 1 : 0;
  if (latency_s) *latency_s = r.done ? r.t_done - r.t_arrive : -1.0;
  if (r.done && S->err != PC_OK) return api_fail(S->err, S->err_msg);
  return PC_OK;
}

pc_status pc_server_stats(pc_server* S, pc_serve_stats* stats) {
  if (!S || !stats) return api_fail(PC_ERR_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  fill_stats(S, stats, S->running ? seconds_since(S->t0) : 0.0, 0, 0, 0);
  return PC_OK;
}

pc_status pc_server_replay(pc_server* S, const pc_query* queries, const double* arrival_s, int nq,
                           void* const* d_out, double* latency_s, pc_serve_stats* stats) {
  TraceRange trace_("pc_server_replay");
  if (!S || (nq > 0 && (!queries || !arrival_s || !latency_s))) return api_fail(PC_ERR_ARG, "NULL argument");
  if (nq < 0) return api_fail(PC_ERR_ARG, "nq < 0");
  if (S->fields.empty() && nq > 0) return api_fail(PC_ERR_ARG, "no fields");
  // resolve and check every query before any GPU work
  std::vector<Query> qs(nq);
  uint64_t largest = 0;
  for (int i = 0; i < nq; ++i) {
    if (i && !(arrival_s[i] >= arrival_s[i - 1])) return api_fail(PC_ERR_ARG, "arrival times must not decrease");
    pc_status r = resolve(S, queries[i], &qs[i]);
    if (r != PC_OK) return r;
    largest = std::max(largest, qs[i].bytes);
  }
  pc_status r = ensure_started(S);
  if (r != PC_OK) return r;
  if (((largest + 255) & ~255ull) > S->arena.cap)
    return api_fail(PC_ERR_OOM, "a query's box exceeds the budget left for results");
  uint64_t b0, q0, o0;
  double origin;
  {
    std::unique_lock<std::mutex> lk(S->mu);  // start from an idle server
    S->cv_done.wait(lk, [&] { return S->pending.empty() && S->inflight == 0; });
    if (S->err != PC_OK) return api_fail(S->err, S->err_msg);
    b0 = S->batches;
    q0 = S->launched;
    o0 = S->bytes_out;
    S->max_seen = 0;
    S->max_inflight = 0;
    S->peak_arena = 0;
    origin = seconds_since(S->t0);
  }
  SK(cudaMemsetAsync(S->d_err, 0, 4, S->slots[0].st));
  SK(cudaStreamSynchronize(S->slots[0].st));
  std::vector<uint64_t> ids(nq);
  const Clock::time_point start = Clock::now();
  for (int i = 0; i < nq; ++i) {
    // sleep until shortly before the arrival, then yield until it
    const auto due = start + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(arrival_s[i]));
    if (due - Clock::now() > std::chrono::microseconds(200)) std::this_thread::sleep_until(due - std::chrono::microseconds(100));
    while (Clock::now() < due) std::this_thread::yield();
    ids[i] = enqueue(S, qs[i], d_out ? d_out[i] : nullptr, origin + arrival_s[i]);
  }
  double last = origin;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_done.wait(lk, [&] { return S->pending.empty() && S->inflight == 0; });
    for (int i = 0; i < nq; ++i) {
      const Request& q = S->reqs[ids[i]];
      latency_s[i] = q.t_done - q.t_arrive;
      last = std::max(last, q.t_done);
    }
    if (stats) fill_stats(S, stats, last - origin, b0, q0, o0);
    if (S->err != PC_OK) return api_fail(S->err, S->err_msg);
  }
  unsigned int h_err = 0;
  SK(cudaMemcpy(&h_err, S->d_err, 4, cudaMemcpyDeviceToHost));
  if (h_err) return api_fail(PC_ERR_CORRUPT_STREAM, "a component stream failed to parse");
  return PC_OK;
}

pc_status pc_server_free(pc_server* S) {
  if (!S) return PC_OK;
  server_release(S);
  return PC_OK;
}

}  // extern "C"
