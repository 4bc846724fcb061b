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
// Scheduling (continuous batching): the host loop admits queries in arrival
// order as long as their output boxes fit in an arena sized by the device
// memory budget, launches every admitted query of one type as one batch while
// the previous batch is still running (two batches in flight on one stream),
// and frees a batch's boxes when its completion event has fired.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
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

struct ServeField {
  const pc_streams* s = nullptr;
  void* cache = nullptr;      // x~ at the cached level, whole field
  uint8_t* level = nullptr;   // per brick
  uint32_t* pend = nullptr;   // per brick: claim of the batch being written back
  uint64_t bytes = 0;         // device bytes counted against the budget
};

struct Slot {
  BoxJob* h_jobs = nullptr;  // pinned
  CacheAux* h_aux = nullptr;
  BoxJob* d_jobs = nullptr;
  CacheAux* d_aux = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<int> queries;
};

// FIFO arena for output boxes: queries are freed in the order they were
// admitted, so the live region is one contiguous run, possibly wrapped.
struct Arena {
  uint64_t cap = 0;
  std::deque<std::pair<uint64_t, uint64_t>> live;  // [lo, hi) per query, oldest first
  uint64_t in_use = 0;
  bool alloc(uint64_t n, uint64_t* off) {
    n = (n + 255) & ~255ull;
    uint64_t o;
    if (live.empty()) {
      if (n > cap) return false;
      o = 0;
    } else {
      const uint64_t tail = live.front().first, head = live.back().second;
      if (live.back().first >= tail) {  // live = [tail, head)
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
    live.emplace_back(o, o + n);
    in_use += n;
    *off = o;
    return true;
  }
  void pop() {
    in_use -= live.front().second - live.front().first;
    live.pop_front();
  }
};

struct Query {
  int field, k;
  int64_t lo[3], hi[3];
  uint64_t bytes;
  pc_dtype dtype;
};

}  // namespace

struct pc_server {
  int device = 0;
  cudaStream_t st = nullptr;
  uint64_t budget = 0;
  int max_batch = 1;
  int flags = 0;
  std::vector<ServeField> fields;
  uint64_t fixed = 0;  // fields, caches, job buffers, spill
  char* arena_mem = nullptr;
  Arena arena;
  uint64_t* spill = nullptr;
  size_t spill_words = 0;
  unsigned int* d_err = nullptr;
  Slot slots[2];
  int nslots = 2;
};

namespace {

void server_release(pc_server* S) {
  if (!S) return;
  cudaStreamSynchronize(S->st);
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
    if (sl.done) cudaEventDestroy(sl.done);
  }
  cudaFree(S->arena_mem);
  cudaFree(S->spill);
  cudaFree(S->d_err);
  delete S;
}

#define SK(call)                                                    \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return api_cuda_fail(e_, #call);         \
  } while (0)

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

// One batch: the queries' box jobs, the write-back into the caches and the
// copies into the callers' buffers, then the slot's completion event.
pc_status launch_batch(pc_server* S, Slot& sl, const std::vector<Query>& qs, const std::vector<uint64_t>& off,
                       void* const* d_out) {
  TraceRange trace_("pc_server batch");
  const bool cache = !(S->flags & PC_SERVE_NO_CACHE);
  const int nj = (int)sl.queries.size();
  const pc_dtype dt = qs[sl.queries[0]].dtype;
  int64_t nunits = 0, nitems = 0;
  for (int j = 0; j < nj; ++j) {
    const Query& q = qs[sl.queries[j]];
    const ServeField& F = S->fields[q.field];
    BoxJob J = make_box_job(F.s, 0, q.k, q.lo, q.hi, S->arena_mem + off[sl.queries[j]]);
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
  SK(cudaMemcpyAsync(sl.d_jobs, sl.h_jobs, sizeof(BoxJob) * nj, cudaMemcpyHostToDevice, S->st));
  if (cache) SK(cudaMemcpyAsync(sl.d_aux, sl.h_aux, sizeof(CacheAux) * nj, cudaMemcpyHostToDevice, S->st));
  RetrieveParams R;
  std::memset(&R, 0, sizeof(R));
  R.jobs = sl.d_jobs;
  R.njobs = nj;
  R.nunits = nunits;
  R.write = 1;
  R.err = S->d_err;
  R.spill = S->spill;
  R.grid = retrieve_grid(dt, 3, nunits);
  SK(launch_retrieve(dt, 3, R, S->st));
  if (cache) SK(launch_cache_update(dt, sl.d_jobs, sl.d_aux, nj, nitems, S->st));
  if (d_out) {
    for (int qi : sl.queries)
      if (d_out[qi])
        SK(cudaMemcpyAsync(d_out[qi], S->arena_mem + off[qi], qs[qi].bytes, cudaMemcpyDeviceToDevice, S->st));
  }
  SK(cudaEventRecord(sl.done, S->st));
  return PC_OK;
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
  S->nslots = (flags & PC_SERVE_SERIAL) ? 1 : 2;
  S->st = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaGetDevice(&S->device);
  for (Slot& sl : S->slots) {
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_jobs, sizeof(BoxJob) * S->max_batch);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&sl.h_aux, sizeof(CacheAux) * S->max_batch);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_jobs, sizeof(BoxJob) * S->max_batch);
    if (e == cudaSuccess) e = cudaMalloc((void**)&sl.d_aux, sizeof(CacheAux) * S->max_batch);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&S->d_err, 16);
  if (e == cudaSuccess) e = cudaMemset(S->d_err, 0, 16);
  if (e != cudaSuccess) {
    server_release(S);
    return api_cuda_fail(e, "server allocation");
  }
  S->fixed = 2 * (sizeof(BoxJob) + sizeof(CacheAux)) * (uint64_t)S->max_batch + 16;
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
  if (S->arena_mem) return api_fail(PC_ERR_ARG, "fields must be added before the first replay");
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
  // per-CTA spill of the retrieval kernel at its largest grid
  const size_t sw = retrieve_spill_words(s->dtype, 3, retrieve_grid(s->dtype, 3, (int64_t)1 << 40));
  if (sw > S->spill_words) {
    const uint64_t grow = 8 * (uint64_t)(sw - S->spill_words);
    if (S->fixed + F.bytes + grow > S->budget) {
      cudaFree(F.cache);
      cudaFree(F.level);
      cudaFree(F.pend);
      return api_fail(PC_ERR_OOM, "the field does not fit in the budget");
    }
    cudaFree(S->spill);
    S->spill = nullptr;
    cudaError_t e = cudaMalloc((void**)&S->spill, 8 * sw);
    if (e != cudaSuccess) {
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
  SK(cudaStreamSynchronize(S->st));
  for (ServeField& f : S->fields)
    if (f.level) SK(cudaMemset(f.level, 0, f.s->nbricks));
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
    const pc_query& in = queries[i];
    if (in.field < 0 || in.field >= (int)S->fields.size()) return api_fail(PC_ERR_ARG, "bad field index");
    if (i && !(arrival_s[i] >= arrival_s[i - 1])) return api_fail(PC_ERR_ARG, "arrival times must not decrease");
    const pc_streams* s = S->fields[in.field].s;
    Query& q = qs[i];
    q.field = in.field;
    q.dtype = s->dtype;
    if (in.k > 0) {
      if (in.k > s->n) return api_fail(PC_ERR_ARG, "k out of range");
      q.k = in.k;
    } else {
      pc_status r = pc_query_k(s, in.tau, &q.k);
      if (r != PC_OK) return r;
    }
    pc_status r = check_box(s, &in.box, q.lo, q.hi);
    if (r != PC_OK) return r;
    q.bytes = (uint64_t)((q.hi[0] - q.lo[0]) * (q.hi[1] - q.lo[1]) * (q.hi[2] - q.lo[2])) * dtype_size(q.dtype);
    largest = std::max(largest, q.bytes);
  }
  if (!S->arena_mem && nq > 0) {  // the arena takes what the budget leaves
    const uint64_t room = S->budget - S->fixed;
    S->arena.cap = room & ~255ull;
    cudaError_t e = S->arena.cap ? cudaMalloc((void**)&S->arena_mem, S->arena.cap) : cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
      S->arena.cap = 0;
      return api_cuda_fail(e, "arena allocation");
    }
  }
  if (((largest + 255) & ~255ull) > S->arena.cap) return api_fail(PC_ERR_OOM, "a query's box exceeds the budget left for results");
  SK(cudaMemsetAsync(S->d_err, 0, 4, S->st));
  SK(cudaStreamSynchronize(S->st));

  std::vector<uint64_t> off(nq, 0);
  std::deque<int> pending, inflight;
  uint64_t batches = 0, launched = 0, bytes_out = 0, peak_arena = 0;
  int done = 0, next = 0, max_seen = 0;
  pc_status rc = PC_OK;
  const Clock::time_point t0 = Clock::now();
  while (done < nq) {
    const double now = seconds_since(t0);
    while (next < nq && arrival_s[next] <= now) pending.push_back(next++);
    // completions, oldest batch first
    while (!inflight.empty()) {
      Slot& sl = S->slots[inflight.front()];
      const cudaError_t e = cudaEventQuery(sl.done);
      if (e == cudaErrorNotReady) break;
      if (e != cudaSuccess) {
        rc = api_cuda_fail(e, "batch");
        break;
      }
      const double tc = seconds_since(t0);
      for (int qi : sl.queries) {
        latency_s[qi] = tc - arrival_s[qi];
        S->arena.pop();
        ++done;
      }
      sl.queries.clear();
      inflight.pop_front();
    }
    if (rc != PC_OK) break;
    // admit and launch the next batch while a slot is free
    if (!pending.empty() && (int)inflight.size() < S->nslots) {
      int si = 0;
      while (!S->slots[si].queries.empty()) ++si;
      Slot& sl = S->slots[si];
      const pc_dtype dt = qs[pending.front()].dtype;
      while (!pending.empty() && (int)sl.queries.size() < S->max_batch) {
        const int qi = pending.front();
        if (qs[qi].dtype != dt) break;
        if (!S->arena.alloc(qs[qi].bytes, &off[qi])) break;  // admission by memory
        sl.queries.push_back(qi);
        pending.pop_front();
      }
      if (!sl.queries.empty()) {
        peak_arena = std::max(peak_arena, S->arena.in_use);
        rc = launch_batch(S, sl, qs, off, d_out);
        if (rc != PC_OK) break;
        inflight.push_back(si);
        ++batches;
        launched += sl.queries.size();
        max_seen = std::max(max_seen, (int)sl.queries.size());
        for (int qi : sl.queries) bytes_out += qs[qi].bytes;
      }
    }
  }
  const double wall = seconds_since(t0);
  if (rc != PC_OK) {
    cudaStreamSynchronize(S->st);
    while (!S->arena.live.empty()) S->arena.pop();
    for (Slot& sl : S->slots) sl.queries.clear();
    return rc;
  }
  unsigned int h_err = 0;
  SK(cudaMemcpyAsync(&h_err, S->d_err, 4, cudaMemcpyDeviceToHost, S->st));
  SK(cudaStreamSynchronize(S->st));
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->wall_s = wall;
    stats->batches = batches;
    stats->queries = launched;
    stats->bytes_out = bytes_out;
    stats->max_batch = (uint64_t)max_seen;
    stats->peak_device_bytes = S->fixed + peak_arena;
    stats->arena_bytes = S->arena.cap;
  }
  if (h_err) return api_fail(PC_ERR_CORRUPT_STREAM, "a component stream failed to parse");
  return PC_OK;
}

pc_status pc_server_free(pc_server* S) {
  if (!S) return PC_OK;
  server_release(S);
  return PC_OK;
}

}  // extern "C"
