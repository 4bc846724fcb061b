// pcz_api.cu -- host side of the C ABI declared in include/pcz.h: argument
// checks, the scratch pool, kernel launches on the caller's stream, the
// component streams object and its serialized form.
//
// Every step of the method runs in the kernels (pcz_compress.cu,
// pcz_retrieve.cu, pcz_misc.cu); this file only moves sizes, pointers and
// per-component metadata (tolerances, Sec. 6.2) around them.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pcz.h"
#include "pcz_host.h"

using namespace pcz;

namespace {

thread_local std::string g_err;

pc_status fail(pc_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

pc_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error so later calls can proceed
  return fail(e == cudaErrorMemoryAllocation ? PC_ERR_OOM : PC_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);       \
  } while (0)

constexpr uint32_t kMagic = 0x315a4350u;  // "PCZ1"
constexpr uint32_t kFormatVersion = 2;
constexpr size_t kCompRecord = 64;  // serialized bytes per component record

size_t dsize(pc_dtype t) { return t == PC_F32 ? 4 : 8; }

// Scratch pool per device, grown on demand and kept for later calls.
struct DevCtx {
  uint64_t* pool = nullptr;
  uint64_t pool_words = 0;
  bool pool_cfg = false;
};
std::mutex g_mu;
DevCtx g_ctx[128];

std::mutex g_pool_mu;
// [0]: scratch and the streams' index arrays; [1]: the streams' payloads.
// Payloads have a pool of their own so that the smaller arrays never split
// a freed payload block: a payload of the size freed before is then served
// from that block without mapping new memory.
cudaMemPool_t g_pools[2][128] = {};

// The library's stream-ordered memory pool `which` on the current device.  It
// keeps freed memory for later calls: the device's default pool hands it back
// to the driver at every synchronisation, so that the next call would pay
// for fresh allocations again.
cudaError_t pool_alloc(int which, void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    cudaMemPool_t& slot = g_pools[which][dev & 127];
    if (!slot) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      e = cudaMemPoolCreate(&slot, &props);
      if (e != cudaSuccess) return e;
      uint64_t keep = ~0ull;
      cudaMemPoolSetAttribute(slot, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    pool = slot;
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

}  // namespace

cudaError_t pcz::scratch_alloc(void** p, size_t bytes, cudaStream_t st) { return pool_alloc(0, p, bytes, st); }

namespace {

// Stream-ordered device allocation; freed on the same stream.
struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t s;
  explicit Scratch(cudaStream_t st) : s(st) {}
  cudaError_t get(void** p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = scratch_alloc(p, bytes ? bytes : 16, s);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, s);
  }
};

// Makes the current device's primary context current on this host thread
// (once per thread): a thread whose first CUDA call is a pointer query would
// otherwise see pinned host memory as unregistered.
void bind_context() {
  thread_local bool bound = false;
  if (bound) return;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) {
    cudaGetLastError();  // this call's own failure; the query below reports what it finds
    return;
  }
  bound = true;
}

// Where a caller's pointer lives.
bool is_device_ptr(const void* p) {
  bind_context();
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Address under which the kernels can use caller memory directly: device or
// managed memory as is, pinned host memory through its device mapping (on a
// Grace-Blackwell node the kernels then read and write it over the C2C link,
// so the transfer overlaps the computation).  False for pageable memory.
bool kernel_pointer(const void* p, const void** dptr, bool* host) {
  bind_context();
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *host = false;
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    *dptr = p;
    return true;
  }
  if (a.type == cudaMemoryTypeHost && a.devicePointer) {
    *dptr = a.devicePointer;
    *host = true;
    return true;
  }
  return false;
}

// floor(log2 tau) from the bit pattern of a positive finite double.
int floor_log2_bits(double tau) {
  uint64_t b;
  std::memcpy(&b, &tau, 8);
  const int be = (int)((b >> 52) & 0x7ff);
  if (be) return be - 1023;
  const uint64_t f = b & ((1ull << 52) - 1);
  int hb = 63;
  while (!((f >> hb) & 1ull)) --hb;
  return hb - 1074;
}

// Bit pattern of the largest T value not above tau (so |e| <= tau is an
// exact comparison of bit patterns on the device).
uint64_t tau_threshold_bits(double tau, pc_dtype dt) {
  if (dt == PC_F64) {
    uint64_t b;
    std::memcpy(&b, &tau, 8);
    return b;
  }
  float f = (float)tau;
  if ((double)f > tau) f = std::nextafterf(f, 0.0f);
  uint32_t b;
  std::memcpy(&b, &f, 4);
  return b;
}

// The T value of a bit pattern, as a double (exact).
double bits_to_double(uint64_t b, pc_dtype dt) {
  if (dt == PC_F64) {
    double d;
    std::memcpy(&d, &b, 8);
    return d;
  }
  const uint32_t u = (uint32_t)b;
  float f;
  std::memcpy(&f, &u, 4);
  return (double)f;
}

bool tau_valid(const double* tau, int n) {
  for (int i = 0; i < n; ++i) {
    if (!std::isfinite(tau[i]) || !(tau[i] > 0)) return false;
    if (i && !(tau[i] < tau[i - 1])) return false;
  }
  return true;
}

void make_geometry(int ndims, const int64_t* dims, int64_t d3[3], int64_t nb[3], int64_t* nbricks, int64_t* nchunks) {
  for (int a = 0; a < 3; ++a) {
    d3[a] = a < ndims ? dims[a] : 1;
    nb[a] = a < ndims ? (d3[a] + 3) / 4 : 1;
  }
  *nbricks = nb[0] * nb[1] * nb[2];
  *nchunks = (*nbricks + kChunk - 1) / kChunk;
}

// Optional per-kernel timing: events around each launch, summed on read.
struct Timing {
  std::mutex mu;
  bool on = false;
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  double ms[PC_KERNEL_KINDS] = {};
  uint64_t launches[PC_KERNEL_KINDS] = {};
} g_timing;

struct TimedLaunch {
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  TimedLaunch(int k, cudaStream_t s) : kind(k), st(s) {
    if (!g_timing.on) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      a = b = nullptr;
      return;
    }
    cudaEventRecord(a, st);
  }
  ~TimedLaunch() {
    if (!a) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(g_timing.mu);
    g_timing.pending.push_back({kind, a, b});
  }
};

}  // namespace

void pcz::set_last_error(const char* msg) { g_err = msg; }

namespace {

// A stream of the library's own on the current device (non-blocking, made
// once): 0 for the copies of retrievals into pinned memory, 1 for releases.
cudaStream_t lib_stream(int which) {
  static std::mutex mu;
  static cudaStream_t streams[2][128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  cudaStream_t& cs = streams[which][dev & 127];
  if (!cs && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    cs = nullptr;
  }
  return cs;
}

// The device arrays of a pc_streams come from the library's memory pools (on
// the stream of the call that makes them, which synchronises before it
// returns), so that neither making nor releasing streams maps or unmaps device
// memory.  Release waits for the library's launches that read the arrays --
// on whatever streams they were queued -- and not for the rest of the device,
// so that a thread freeing its streams does not stall work other threads have
// queued; the memory is back in the pool when it returns.  sync_device (the
// error paths of the calls that make streams, whose allocations may still be
// pending on their stream) waits for the device first.
void streams_release(pc_streams* s, bool sync_device = false) {
  if (!s) return;
  if (s->backing) {  // a batch's streams share device arenas, freed with the last of them
    cudaDeviceSynchronize();
    delete s;
    return;
  }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != s->device) cudaSetDevice(s->device);
  cudaStream_t rs = lib_stream(1);
  {
    std::lock_guard<std::mutex> lk(s->use_mu);
    if (sync_device || s->sync_device || !rs) cudaDeviceSynchronize();
    for (auto& u : s->uses) {
      if (rs) cudaStreamWaitEvent(rs, u.second, 0);
      cudaEventDestroy(u.second);  // released once the wait is resolved
    }
    s->uses.clear();
  }
  void* arrays[] = {s->d_payload, s->d_index};
  for (void* a : arrays)
    if (a) cudaFreeAsync(a, rs);  // rs null: the legacy stream, after the device synchronisation
  if (rs) cudaStreamSynchronize(rs);
  if (cur >= 0 && cur != s->device) cudaSetDevice(cur);
  delete s;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// A small pinned host buffer per host thread for the results a call reads
// back and the parameters it uploads (grown on demand; one copy each way).
struct PinnedStage {
  void* p = nullptr;
  size_t cap = 0;
  ~PinnedStage() {
    if (p) cudaFreeHost(p);
  }
  void* get(size_t bytes) {
    if (bytes > cap) {
      if (p) cudaFreeHost(p);
      p = nullptr;
      cap = 0;
      const size_t want = std::max(bytes, size_t(16) << 10);
      if (cudaMallocHost(&p, want) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        return nullptr;
      }
      cap = want;
    }
    return p;
  }
};
thread_local PinnedStage t_stage;

// One device array of a pc_streams, from the library's pool on stream st.
cudaError_t streams_alloc(void** p, size_t bytes, cudaStream_t st) { return pool_alloc(0, p, bytes, st); }
cudaError_t payload_alloc(void** p, size_t bytes, cudaStream_t st) { return pool_alloc(1, p, bytes, st); }

// The index arrays of s in one allocation (from the index pool): chunk word
// offsets [n][nchunks] (u64), brick lengths [n][nbricks] (u16), brick bit
// offsets [n][nbricks] (u32), the component descriptors and the error word,
// which is cleared on st.
cudaError_t alloc_index(pc_streams* s, cudaStream_t st) {
  const size_t n = (size_t)s->n, nbr = (size_t)s->nbricks, nch = (size_t)s->nchunks;
  const size_t o_cw = 0, o_bl = align256(o_cw + 8 * n * nch + 16), o_bo = align256(o_bl + 2 * n * nbr + 16);
  const size_t o_desc = align256(o_bo + 4 * n * nbr + 16), o_err = align256(o_desc + sizeof(CompDesc) * n);
  char* p = nullptr;
  cudaError_t e = streams_alloc((void**)&p, o_err + 16, st);
  if (e != cudaSuccess) return e;
  s->d_index = p;
  s->d_chunk_word = (uint64_t*)(p + o_cw);
  s->d_brick_len = (uint16_t*)(p + o_bl);
  s->d_brick_off = (uint32_t*)(p + o_bo);
  s->d_desc = (CompDesc*)(p + o_desc);
  s->d_err = (unsigned int*)(p + o_err);
  return cudaMemsetAsync(s->d_err, 0, 16, st);
}

// The per-component descriptors the retrieval kernel reads.
void fill_desc(const pc_streams* s, CompDesc* d) {
  for (int i = 0; i < s->n; ++i) {
    d[i].payload = s->d_payload + s->word_base[i];
    d[i].nwords = s->words[i];
    d[i].chunk_word = s->d_chunk_word + (int64_t)i * s->nchunks;
    d[i].brick_len = s->d_brick_len + (int64_t)i * s->nbricks;
    d[i].brick_off = s->d_brick_off + (int64_t)i * s->nbricks;
    d[i].L = s->L[i];
    d[i].pad_ = 0;
  }
}

// Uploads the descriptors and waits for them.
pc_status upload_desc(pc_streams* s, cudaStream_t st) {
  std::vector<CompDesc> d(s->n);
  fill_desc(s, d.data());
  CK(cudaMemcpyAsync(s->d_desc, d.data(), sizeof(CompDesc) * s->n, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
  return PC_OK;
}

pc_status box_of(const pc_streams* s, const pc_box* box, int64_t lo[3], int64_t hi[3]) {
  for (int a = 0; a < 3; ++a) {
    lo[a] = 0;
    hi[a] = s->dims[a];
    if (box && a < s->ndims) {
      lo[a] = box->lo[a];
      hi[a] = box->hi[a];
      if (lo[a] < 0 || hi[a] > s->dims[a] || lo[a] >= hi[a]) return fail(PC_ERR_ARG, "box outside the field or empty");
    }
  }
  return PC_OK;
}

// Magic numbers of DivMagic for divisor d (1 <= d < 2^32).
DivMagic div_magic(uint64_t d) {
  int l = 0;
  while (l < 32 && (1ull << l) < d) ++l;
  DivMagic D;
  D.m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
  D.s1 = (uint8_t)(l ? 1 : 0);
  D.s2 = (uint8_t)(l ? l - 1 : 0);
  D.pad_ = 0;
  return D;
}

// One retrieval job over the box of a stream set (units not yet placed).
BoxJob make_job(const pc_streams* s, int k0, int k, const int64_t lo[3], const int64_t hi[3], void* d_out) {
  BoxJob J;
  std::memset(&J, 0, sizeof(J));
  J.comp = s->d_desc;
  for (int a = 0; a < 3; ++a) {
    J.dims[a] = s->dims[a];
    J.nb[a] = s->nb[a];
    J.lo[a] = lo[a];
    J.hi[a] = hi[a];
    J.bl[a] = lo[a] / 4;
    J.bn[a] = (hi[a] - 1) / 4 - J.bl[a] + 1;
  }
  J.nbox = J.bn[0] * J.bn[1] * J.bn[2];
  J.k0 = k0;
  J.k = k;
  J.umult = retrieve_unit_mult(k - k0);
  if (J.nbox < (1ll << 32)) {
    J.dv_bn0 = div_magic((uint64_t)J.bn[0]);
    J.dv_bn1 = div_magic((uint64_t)J.bn[1]);
  }
  J.dv_ub = div_magic(16ull * (uint64_t)J.umult);
  J.out = d_out;
  return J;
}

int64_t job_units(const BoxJob& J) { return (J.nbox + 16 * J.umult - 1) / (16 * J.umult); }

// Runs Algorithm 2 on the box: components k0+1..k added into d_out (device).
pc_status run_retrieve(const pc_streams* s, int k0, int k, const int64_t lo[3], const int64_t hi[3], void* d_out,
                       int write, cudaStream_t st) {
  if (k == k0) {
    if (k0 == 0 && write) {
      const size_t bytes = (size_t)((hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])) * dsize(s->dtype);
      CK(cudaMemsetAsync(d_out, 0, bytes, st));
    }
    return PC_OK;
  }
  RetrieveParams R;
  std::memset(&R, 0, sizeof(R));
  R.job0 = make_job(s, k0, k, lo, hi, d_out);
  R.jobs = nullptr;
  R.njobs = 1;
  R.nunits = job_units(R.job0);
  R.write = write;
  R.err = s->d_err;
  R.grid = retrieve_grid(s->dtype, s->ndims, R.nunits);
  Scratch scr(st);  // per-CTA spill for planes below the shared-memory slots
  CK(scr.get((void**)&R.spill, 8 * retrieve_spill_words(s->dtype, s->ndims, R.grid)));
  {
    TimedLaunch tl(PC_KERNEL_RETRIEVE, st);
    CK(launch_retrieve(s->dtype, s->ndims, R, st));
  }
  note_use(s, st);
  return PC_OK;
}

}  // namespace

pc_status pcz::api_fail(pc_status st, const std::string& msg) { return fail(st, msg); }
pc_status pcz::api_cuda_fail(cudaError_t e, const char* what) { return cuda_fail(e, what); }
size_t pcz::dtype_size(pc_dtype t) { return dsize(t); }
pc_status pcz::check_box(const pc_streams* s, const pc_box* box, int64_t lo[3], int64_t hi[3]) {
  return box_of(s, box, lo, hi);
}
BoxJob pcz::make_box_job(const pc_streams* s, int k0, int k, const int64_t lo[3], const int64_t hi[3], void* out) {
  return make_job(s, k0, k, lo, hi, out);
}
int64_t pcz::box_job_units(const BoxJob& J) { return job_units(J); }
double pcz::value_of_bits(uint64_t b, pc_dtype dt) { return bits_to_double(b, dt); }
int pcz::floor_log2_of(double tau) { return floor_log2_bits(tau); }
uint64_t pcz::tau_bits_of(double tau, pc_dtype dt) { return tau_threshold_bits(tau, dt); }
bool pcz::tolerances_valid(const double* tau, int n) { return tau_valid(tau, n); }
void pcz::field_geometry(int ndims, const int64_t* dims, int64_t d3[3], int64_t nb[3], int64_t* nbricks,
                         int64_t* nchunks) {
  make_geometry(ndims, dims, d3, nb, nbricks, nchunks);
}
bool pcz::device_pointer(const void* p) { return is_device_ptr(p); }
void pcz::note_use(const pc_streams* s, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(s->use_mu);
  for (auto& u : s->uses)
    if (u.first == st) {  // the new record follows every earlier launch on st
      if (cudaEventRecord(u.second, st) != cudaSuccess) {
        cudaGetLastError();
        s->sync_device = true;
      }
      return;
    }
  cudaEvent_t ev = nullptr;
  if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(ev, st) != cudaSuccess) {
    cudaGetLastError();
    if (ev) cudaEventDestroy(ev);
    s->sync_device = true;
    return;
  }
  s->uses.emplace_back(st, ev);
}

extern "C" {

const char* pc_last_error(void) { return g_err.c_str(); }

pc_status pc_debug_status(uint32_t* word, int* enabled, int reset) {
  g_err.clear();
  if (!word) return fail(PC_ERR_ARG, "word is NULL");
  *word = check_word_compress(reset) | check_word_small(reset) | check_word_retrieve(reset) |
          check_word_batch(reset);
#ifdef PCZ_DEBUG
  if (enabled) *enabled = 1;
#else
  if (enabled) *enabled = 0;
#endif
  return PC_OK;
}

int pc_version(void) { return (int)kFormatVersion; }

pc_status pc_compress(const void* field, const int64_t* dims, int ndims, pc_dtype dtype, const double* tau, int n,
                      void* cuda_stream, pc_streams** out) {
  TraceRange trace_("pc_compress");
  g_err.clear();
  if (!out) return fail(PC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!field || !dims || !tau) return fail(PC_ERR_ARG, "NULL field, dims or tau");
  if (ndims < 1 || ndims > 3) return fail(PC_ERR_ARG, "ndims must be 1, 2 or 3");
  if (dtype != PC_F32 && dtype != PC_F64) return fail(PC_ERR_ARG, "dtype must be PC_F32 or PC_F64");
  if (n < 1 || n > PC_MAX_COMPONENTS) return fail(PC_ERR_ARG, "n out of range");
  for (int a = 0; a < ndims; ++a)
    if (dims[a] < 1) return fail(PC_ERR_ARG, "extent < 1");
  if (!tau_valid(tau, n)) return fail(PC_ERR_TAU_ORDER, "tolerances must be finite, positive, strictly decreasing");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  CK(cudaGetDevice(&dev));

  pc_streams* s = new pc_streams();
  s->device = dev;
  s->ndims = ndims;
  s->dtype = dtype;
  s->n = n;
  make_geometry(ndims, dims, s->dims, s->nb, &s->nbricks, &s->nchunks);
  const int64_t count = s->dims[0] * s->dims[1] * s->dims[2];
  const int64_t nbr = s->nbricks, nch = s->nchunks;

  CompressParams P;
  std::memset(&P, 0, sizeof(P));
  for (int a = 0; a < 3; ++a) {
    P.dims[a] = s->dims[a];
    P.nb[a] = s->nb[a];
  }
  P.nbricks = nbr;
  P.nchunks = nch;
  P.n = n;
  for (int i = 0; i < n; ++i) {
    s->tau[i] = tau[i];
    s->L[i] = floor_log2_bits(tau[i]);
    P.tau_bits[i] = tau_threshold_bits(tau[i], dtype);
    P.L[i] = s->L[i];
  }

  pc_status rc = PC_OK;
  {
    Scratch scr(st);
    cudaError_t e = cudaSuccess;
    const void* d_field = field;
    void* staged = nullptr;
    bool mapped_host = false;
    if (!kernel_pointer(field, &d_field, &mapped_host)) {  // pageable host field: copy it in on the stream
      e = scr.get(&staged, count * dsize(dtype));
      if (e == cudaSuccess) e = cudaMemcpyAsync(staged, field, count * dsize(dtype), cudaMemcpyHostToDevice, st);
      d_field = staged;
    }
    P.field = d_field;
    // one scratch block: the per-(component, chunk) arrays, then the call's
    // results back to back (read with one copy), then the payload bases
    const size_t nc = (size_t)n * nch;
    const size_t o_nwords = 0, o_maxerr_c = align256(o_nwords + 4 * nc), o_pool = align256(o_maxerr_c + 8 * nc);
    const size_t o_counts_c = align256(o_pool + 8 * nc), o_res = align256(o_counts_c + 20 * nc);
    const size_t res_bytes = 56 * (size_t)n + 16;  // totals[n], counts[5n], maxerr[n], flags (8 bytes), used
    const size_t o_base = align256(o_res + res_bytes), scratch_bytes = o_base + 8 * (size_t)n;
    char* sb = nullptr;
    if (e == cudaSuccess) e = scr.get((void**)&sb, scratch_bytes);
    if (e == cudaSuccess) e = alloc_index(s, st);
    if (e != cudaSuccess) {
      streams_release(s, true);
      return cuda_fail(e, "allocation");
    }
    uint32_t* chunk_nwords = (uint32_t*)(sb + o_nwords);
    uint64_t* chunk_maxerr = (uint64_t*)(sb + o_maxerr_c);
    uint64_t* chunk_pool = (uint64_t*)(sb + o_pool);
    uint32_t* chunk_counts = (uint32_t*)(sb + o_counts_c);
    uint64_t* totals = (uint64_t*)(sb + o_res);
    unsigned long long* counts = (unsigned long long*)(totals + n);
    unsigned long long* maxerr = counts + 5 * n;
    unsigned int* flags = (unsigned int*)(maxerr + n);
    unsigned long long* used = (unsigned long long*)(maxerr + n) + 1;
    uint64_t* comp_base = (uint64_t*)(sb + o_base);
    P.brick_off = s->d_brick_off;
    P.chunk_nwords = chunk_nwords;
    P.chunk_pool = chunk_pool;
    P.brick_len = s->d_brick_len;
    P.chunk_counts = chunk_counts;
    P.chunk_maxerr = chunk_maxerr;
    P.flags = flags;
    P.pool_used = used;

    // the results come back through this thread's pinned staging buffer
    const size_t up_bytes = 8 * (size_t)n + sizeof(CompDesc) * (size_t)n;  // payload bases, descriptors
    char* h = static_cast<char*>(t_stage.get(std::max(res_bytes, up_bytes)));
    if (!h) {
      streams_release(s, true);
      return fail(PC_ERR_OOM, "pinned staging buffer");
    }
    const uint64_t* h_tot = (const uint64_t*)h;
    const unsigned long long* h_cnt = (const unsigned long long*)(h_tot + n);
    const unsigned long long* h_merr = h_cnt + 5 * n;
    unsigned int h_flags = 0;
    unsigned long long h_used = 0;
    // the pool is shared by every call on this device: hold it until the
    // packing kernel that reads it has finished (the last synchronisation)
    std::unique_lock<std::mutex> pool_lock(g_mu);
    for (int attempt = 0; attempt < 3; ++attempt) {
      {
        DevCtx& cx = g_ctx[dev & 127];
        // first guess: two bytes of stream per input byte, plus chunk padding
        const uint64_t want = attempt == 0 ? (uint64_t)(count * dsize(dtype) * 2 / 8 + 2 * n * nch + 1024)
                                           : (uint64_t)(h_used + h_used / 8 + 1024);
        if (cx.pool_words < want) {
          if (cx.pool) cudaFree(cx.pool);
          cx.pool = nullptr;
          cx.pool_words = 0;
          e = cudaMalloc((void**)&cx.pool, want * 8);
          if (e != cudaSuccess) break;
          cx.pool_words = want;
        }
        P.pool = cx.pool;
        P.pool_words = cx.pool_words;
      }
      if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 16, st);  // flags and the pool's bump counter
      if (e == cudaSuccess) {
        TimedLaunch tl(PC_KERNEL_COMPRESS, st);
        e = launch_compress(dtype, ndims, P, st, !mapped_host);
      }
      if (e == cudaSuccess) {
        TimedLaunch tl(PC_KERNEL_SCAN, st);
        e = launch_scan_chunks(chunk_nwords, s->d_chunk_word, totals, chunk_counts, counts, chunk_maxerr, maxerr, n,
                               nch, st);
      }
      if (e == cudaSuccess) e = cudaMemcpyAsync(h, totals, res_bytes, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) break;
      h_flags = *(const unsigned int*)(h_merr + n);
      h_used = *((const unsigned long long*)(h_merr + n) + 1);
      if (!(h_flags & kFlagPoolOverflow)) break;
    }
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "compress");
    } else if (h_flags & kFlagNonFinite) {
      rc = fail(PC_ERR_NONFINITE, "the field holds a NaN or an infinity");
    } else if (h_flags & kFlagStageTimeout) {
      rc = fail(PC_ERR_CUDA, "a tile copy of the field into shared memory did not complete");
    } else if (h_flags & kFlagPoolOverflow) {
      rc = fail(PC_ERR_OOM, "scratch pool could not be sized");
    } else {
      uint64_t total = 0;
      for (int i = 0; i < n; ++i) {
        s->word_base[i] = total;
        s->words[i] = h_tot[i];
        total += h_tot[i];
        for (int k = 0; k < 5; ++k) s->counts[i][k] = h_cnt[5 * i + k];
        s->measured[i] = bits_to_double(h_merr[i], dtype);
      }
      e = payload_alloc((void**)&s->d_payload, 8 * total + 16, st);
      if (e == cudaSuccess) {
        // payload bases and the retrieval's descriptors, staged together (the results are read)
        uint64_t* h_base = (uint64_t*)h;
        CompDesc* h_desc = (CompDesc*)(h + 8 * (size_t)n);
        for (int i = 0; i < n; ++i) h_base[i] = s->word_base[i];
        fill_desc(s, h_desc);
        e = cudaMemcpyAsync(comp_base, h_base, 8 * (size_t)n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync(s->d_desc, h_desc, sizeof(CompDesc) * (size_t)n, cudaMemcpyHostToDevice, st);
      }
      if (e == cudaSuccess) {
        TimedLaunch tl(PC_KERNEL_PACK, st);
        e = launch_pack(P.pool, chunk_nwords, chunk_pool, s->d_chunk_word, comp_base, s->d_payload, n, nch, st);
      }
      // the staging buffer, the bit pool and the scratch are idle once this returns
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) rc = cuda_fail(e, "pack");
    }
  }
  if (rc != PC_OK) {
    streams_release(s, true);
    return rc;
  }
  *out = s;
  return PC_OK;
}

pc_status pc_query_k_measured(const pc_streams* s, double tau, int* k_out) {
  g_err.clear();
  if (!s || !k_out) return fail(PC_ERR_ARG, "NULL argument");
  if (!(tau >= 0) || std::isnan(tau)) return fail(PC_ERR_ARG, "tau must be a number >= 0");
  for (int i = 0; i < s->n; ++i)
    if (s->measured[i] <= tau) {
      *k_out = i + 1;
      return PC_OK;
    }
  return fail(PC_ERR_TOL_UNREACHABLE, "tolerance finer than the last component's measured error");
}

pc_status pc_stream_measured_error(const pc_streams* s, int i, double* err) {
  g_err.clear();
  if (!s || !err || i < 0 || i >= s->n) return fail(PC_ERR_ARG, "bad streams, component index or pointer");
  *err = s->measured[i];
  return PC_OK;
}

pc_status pc_query_k(const pc_streams* s, double tau, int* k_out) {
  g_err.clear();
  if (!s || !k_out) return fail(PC_ERR_ARG, "NULL argument");
  if (!(tau >= 0) || std::isnan(tau)) return fail(PC_ERR_ARG, "tau must be a number >= 0");
  for (int i = 0; i < s->n; ++i)
    if (s->tau[i] <= tau) {
      *k_out = i + 1;
      return PC_OK;
    }
  return fail(PC_ERR_TOL_UNREACHABLE, "tolerance finer than the last component's");
}

// A per-device stream of the library for copies between the device and
// pinned host memory, so that they overlap the kernels of the caller's stream.
static cudaStream_t copy_stream() { return lib_stream(0); }

// Retrieval into pinned host memory by slabs of whole brick layers along z:
// each slab is decoded into one of two device staging buffers on the caller's
// stream, and the copy engines move it to the host on the library's copy
// stream while the next slab decodes (a slab of the box is a contiguous run of
// its bytes, x fastest).  With read_in (refinement) each slab's x~_k0 is first
// copied in.  The caller's stream waits for the last copy, so the host buffer
// is complete in stream order, as after a cudaMemcpyAsync.
static pc_status retrieve_pinned_slabs(const pc_streams* s, int k0, int k, const int64_t lo[3], const int64_t hi[3],
                                       char* hbuf, int read_in, cudaStream_t st, cudaStream_t cs) {
  const size_t T = dsize(s->dtype);
  const size_t plane = (size_t)((hi[0] - lo[0]) * (hi[1] - lo[1])) * T;  // bytes of one z-plane of the box
  constexpr size_t kSlabTarget = size_t(64) << 20;
  int64_t layers = (int64_t)(kSlabTarget / (4 * plane));  // brick layers (4 planes) per slab
  if (layers < 1) layers = 1;
  // slab boundaries on brick layers (z multiple of 4), the box's own ends excepted
  std::vector<int64_t> zs{lo[2]};
  while (zs.back() < hi[2]) {
    const int64_t z = zs.back();
    const int64_t next = std::min(hi[2], (z / 4 + layers) * 4);
    zs.push_back(next);
  }
  const int nslab = (int)zs.size() - 1;
  size_t max_bytes = 0;
  for (int i = 0; i < nslab; ++i) max_bytes = std::max(max_bytes, (size_t)(zs[i + 1] - zs[i]) * plane);
  Scratch scr(st);
  void* stage[2] = {nullptr, nullptr};
  CK(scr.get(&stage[0], max_bytes));
  CK(scr.get(&stage[1], max_bytes));
  cudaEvent_t kdone[2] = {nullptr, nullptr}, cdone[2] = {nullptr, nullptr};
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
    e = cudaEventCreateWithFlags(&kdone[j], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&cdone[j], cudaEventDisableTiming);
  }
  pc_status r = PC_OK;
  for (int i = 0; i < nslab && e == cudaSuccess && r == PC_OK; ++i) {
    const int b = i & 1;
    int64_t slo[3] = {lo[0], lo[1], zs[i]}, shi[3] = {hi[0], hi[1], zs[i + 1]};
    const size_t off = (size_t)(zs[i] - lo[2]) * plane, bytes = (size_t)(zs[i + 1] - zs[i]) * plane;
    if (i >= 2) e = cudaStreamWaitEvent(st, cdone[b], 0);  // staging buffer b has been copied out
    if (e == cudaSuccess && read_in) e = cudaMemcpyAsync(stage[b], hbuf + off, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) break;
    r = run_retrieve(s, k0, k, slo, shi, stage[b], 1, st);
    if (r != PC_OK) break;
    e = cudaEventRecord(kdone[b], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, kdone[b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hbuf + off, stage[b], bytes, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess) e = cudaEventRecord(cdone[b], cs);
  }
  // the caller's stream (and the staging buffers' release on it) wait for every copy
  for (int j = 0; j < 2 && e == cudaSuccess; ++j)
    if (j < nslab) e = cudaStreamWaitEvent(st, cdone[j], 0);
  for (int j = 0; j < 2; ++j) {
    if (kdone[j]) cudaEventDestroy(kdone[j]);
    if (cdone[j]) cudaEventDestroy(cdone[j]);
  }
  if (r != PC_OK) return r;
  CK(e);
  return PC_OK;
}

static pc_status retrieve_common(const pc_streams* s, int k0, int k, const pc_box* box, void* buf, int read_in,
                                 void* cuda_stream) {
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int64_t lo[3], hi[3];
  pc_status r = box_of(s, box, lo, hi);
  if (r != PC_OK) return r;
  const size_t bytes = (size_t)((hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])) * dsize(s->dtype);
  const void* kp = nullptr;
  bool host = false;
  if (kernel_pointer(buf, &kp, &host)) {
    if (host && s->ndims == 3 && k > k0 && bytes >= (size_t(32) << 20)) {
      // a large box in pinned host memory: decoded into device slabs and copied by the copy engines
      cudaStream_t cs = copy_stream();
      if (cs) return retrieve_pinned_slabs(s, k0, k, lo, hi, static_cast<char*>(buf), read_in, st, cs);
    }
    // device memory, or pinned host memory written in place by the kernel
    return run_retrieve(s, k0, k, lo, hi, const_cast<void*>(kp), 1, st);
  }
  Scratch scr(st);
  void* d = nullptr;
  CK(scr.get(&d, bytes));
  if (read_in) CK(cudaMemcpyAsync(d, buf, bytes, cudaMemcpyHostToDevice, st));
  r = run_retrieve(s, k0, k, lo, hi, d, 1, st);
  if (r != PC_OK) return r;
  CK(cudaMemcpyAsync(buf, d, bytes, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PC_OK;
}

pc_status pc_retrieve(const pc_streams* s, double tau, int k, const pc_box* box, void* out, void* cuda_stream) {
  TraceRange trace_("pc_retrieve");
  g_err.clear();
  if (!s || !out) return fail(PC_ERR_ARG, "NULL argument");
  if (tau >= 0) {
    pc_status r = pc_query_k(s, tau, &k);
    if (r != PC_OK) return r;
  } else if (k < 0 || k > s->n) {
    return fail(PC_ERR_ARG, "k out of range");
  }
  return retrieve_common(s, 0, k, box, out, 0, cuda_stream);
}

pc_status pc_refine(const pc_streams* s, int k0, int k, const pc_box* box, void* inout, void* cuda_stream) {
  TraceRange trace_("pc_refine");
  g_err.clear();
  if (!s || !inout) return fail(PC_ERR_ARG, "NULL argument");
  if (k0 < 0 || k < k0 || k > s->n) return fail(PC_ERR_ARG, "need 0 <= k0 <= k <= n");
  return retrieve_common(s, k0, k, box, inout, 1, cuda_stream);
}

pc_status pc_stream_info(const pc_streams* s, int i, double* tau_i, uint64_t* bits, uint64_t* index_bytes) {
  g_err.clear();
  if (!s || i < 0 || i >= s->n) return fail(PC_ERR_ARG, "bad streams or component index");
  if (tau_i) *tau_i = s->tau[i];
  if (bits) *bits = s->words[i] * 64;
  if (index_bytes) *index_bytes = (uint64_t)s->nchunks * 8 + (uint64_t)s->nbricks * 2;
  return PC_OK;
}

pc_status pc_streams_shape(const pc_streams* s, int* ndims, int64_t* dims, pc_dtype* dtype, int* n) {
  g_err.clear();
  if (!s) return fail(PC_ERR_ARG, "NULL streams");
  if (ndims) *ndims = s->ndims;
  if (dims)
    for (int a = 0; a < 3; ++a) dims[a] = s->dims[a];
  if (dtype) *dtype = s->dtype;
  if (n) *n = s->n;
  return PC_OK;
}

pc_status pc_stream_counts(const pc_streams* s, int i, uint64_t counts[5]) {
  g_err.clear();
  if (!s || !counts || i < 0 || i >= s->n) return fail(PC_ERR_ARG, "bad arguments");
  for (int k = 0; k < 5; ++k) counts[k] = s->counts[i][k];
  return PC_OK;
}

pc_status pc_stream_device_ptrs(const pc_streams* s, int i, const uint64_t** payload, const uint64_t** chunk_word,
                                const uint16_t** brick_len, uint64_t* payload_words, uint64_t* nchunks,
                                uint64_t* nbricks) {
  g_err.clear();
  if (!s || i < 0 || i >= s->n) return fail(PC_ERR_ARG, "bad streams or component index");
  if (payload) *payload = s->d_payload + s->word_base[i];
  if (chunk_word) *chunk_word = s->d_chunk_word + (int64_t)i * s->nchunks;
  if (brick_len) *brick_len = s->d_brick_len + (int64_t)i * s->nbricks;
  if (payload_words) *payload_words = s->words[i];
  if (nchunks) *nchunks = (uint64_t)s->nchunks;
  if (nbricks) *nbricks = (uint64_t)s->nbricks;
  return PC_OK;
}

// Serialized layout (little endian): a 64-byte header {magic, version, dtype,
// ndims, n, 0, dims[3], nbricks, nchunks}, then per component {tau, words,
// counts[5], measured error} (64 bytes), then per component chunk_word[nchunks] (u64),
// brick_len[nbricks] (u16, padded to 8 bytes) and payload[words] (u64).
static size_t serialized_size(const pc_streams* s) {
  size_t sz = 64 + kCompRecord * (size_t)s->n;
  for (int i = 0; i < s->n; ++i)
    sz += 8 * (size_t)s->nchunks + (((size_t)s->nbricks * 2 + 7) & ~(size_t)7) + 8 * s->words[i];
  return sz;
}

pc_status pc_streams_serialize(const pc_streams* s, void* h_buf, size_t* len, void* cuda_stream) {
  TraceRange trace_("pc_streams_serialize");
  g_err.clear();
  if (!s || !len) return fail(PC_ERR_ARG, "NULL argument");
  const size_t need = serialized_size(s);
  if (!h_buf) {
    *len = need;
    return PC_OK;
  }
  if (*len < need) return fail(PC_ERR_ARG, "buffer too small");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  unsigned char* p = (unsigned char*)h_buf;
  std::memset(p, 0, 64);
  uint32_t hd[6] = {kMagic, kFormatVersion, (uint32_t)s->dtype, (uint32_t)s->ndims, (uint32_t)s->n, 0};
  std::memcpy(p, hd, 24);
  std::memcpy(p + 24, s->dims, 24);
  std::memcpy(p + 48, &s->nbricks, 8);
  std::memcpy(p + 56, &s->nchunks, 8);
  p += 64;
  for (int i = 0; i < s->n; ++i) {
    std::memcpy(p, &s->tau[i], 8);
    std::memcpy(p + 8, &s->words[i], 8);
    std::memcpy(p + 16, s->counts[i], 40);
    std::memcpy(p + 56, &s->measured[i], 8);
    p += kCompRecord;
  }
  for (int i = 0; i < s->n; ++i) {
    CK(cudaMemcpyAsync(p, s->d_chunk_word + (int64_t)i * s->nchunks, 8 * s->nchunks, cudaMemcpyDeviceToHost, st));
    p += 8 * s->nchunks;
    const size_t bl = (size_t)s->nbricks * 2;
    CK(cudaMemcpyAsync(p, s->d_brick_len + (int64_t)i * s->nbricks, bl, cudaMemcpyDeviceToHost, st));
    std::memset(p + bl, 0, ((bl + 7) & ~(size_t)7) - bl);
    p += (bl + 7) & ~(size_t)7;
    CK(cudaMemcpyAsync(p, s->d_payload + s->word_base[i], 8 * s->words[i], cudaMemcpyDeviceToHost, st));
    p += 8 * s->words[i];
  }
  CK(cudaStreamSynchronize(st));
  *len = need;
  return PC_OK;
}

pc_status pc_streams_deserialize(const void* h_buf, size_t len, void* cuda_stream, pc_streams** out) {
  TraceRange trace_("pc_streams_deserialize");
  g_err.clear();
  if (!h_buf || !out) return fail(PC_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (len < 64) return fail(PC_ERR_VERSION, "too short for a header");
  const unsigned char* p = (const unsigned char*)h_buf;
  uint32_t hd[6];
  std::memcpy(hd, p, 24);
  if (hd[0] != kMagic || hd[1] != kFormatVersion) return fail(PC_ERR_VERSION, "not a PCZ stream of this version");
  const pc_dtype dt = (pc_dtype)hd[2];
  const int ndims = (int)hd[3], n = (int)hd[4];
  if ((dt != PC_F32 && dt != PC_F64) || ndims < 1 || ndims > 3 || n < 1 || n > PC_MAX_COMPONENTS)
    return fail(PC_ERR_CORRUPT_STREAM, "bad header fields");
  int64_t dims[3], nbr, nch;
  std::memcpy(dims, p + 24, 24);
  std::memcpy(&nbr, p + 48, 8);
  std::memcpy(&nch, p + 56, 8);
  for (int a = 0; a < 3; ++a)
    if (dims[a] < 1 || dims[a] > ((int64_t)1 << 40)) return fail(PC_ERR_CORRUPT_STREAM, "bad extents");
  pc_streams* s = new pc_streams();
  s->ndims = ndims;
  s->dtype = dt;
  s->n = n;
  make_geometry(ndims, dims, s->dims, s->nb, &s->nbricks, &s->nchunks);
  bool unit_tail = true;  // extents beyond ndims are 1
  for (int a = ndims; a < 3; ++a) unit_tail = unit_tail && dims[a] == 1;
  if (s->nbricks != nbr || s->nchunks != nch || !unit_tail) {
    delete s;
    return fail(PC_ERR_CORRUPT_STREAM, "brick counts do not match the extents");
  }
  size_t off = 64;
  if (len < off + kCompRecord * (size_t)n) {
    delete s;
    return fail(PC_ERR_CORRUPT_STREAM, "truncated");
  }
  uint64_t total = 0;
  for (int i = 0; i < n; ++i) {
    std::memcpy(&s->tau[i], p + off, 8);
    std::memcpy(&s->words[i], p + off + 8, 8);
    std::memcpy(s->counts[i], p + off + 16, 40);
    std::memcpy(&s->measured[i], p + off + 56, 8);
    off += kCompRecord;
    s->word_base[i] = total;
    total += s->words[i];
  }
  if (!tau_valid(s->tau, n)) {
    delete s;
    return fail(PC_ERR_CORRUPT_STREAM, "bad tolerances");
  }
  for (int i = 0; i < n; ++i)
    if (!(s->measured[i] >= 0.0) || !std::isfinite(s->measured[i])) {
      delete s;
      return fail(PC_ERR_CORRUPT_STREAM, "bad measured errors");
    }
  for (int i = 0; i < n; ++i) s->L[i] = floor_log2_bits(s->tau[i]);
  if (len != serialized_size(s)) {
    delete s;
    return fail(PC_ERR_CORRUPT_STREAM, "length does not match the header");
  }
  // index consistency on the host: chunk word offsets follow from the brick lengths
  {
    size_t q = off;
    for (int i = 0; i < n; ++i) {
      const uint64_t* cw = (const uint64_t*)(p + q);
      const uint16_t* bl = (const uint16_t*)(p + q + 8 * nch);
      uint64_t w = 0;
      for (int64_t c = 0; c < nch; ++c) {
        uint64_t bits = 0;
        for (int64_t b = c * kChunk; b < nbr && b < (c + 1) * kChunk; ++b) bits += bl[b];
        if (cw[c] != w) {
          delete s;
          return fail(PC_ERR_CORRUPT_STREAM, "chunk offsets inconsistent with brick lengths");
        }
        w += (bits + 63) / 64;
      }
      if (w != s->words[i]) {
        delete s;
        return fail(PC_ERR_CORRUPT_STREAM, "payload size inconsistent with brick lengths");
      }
      q += 8 * nch + (((size_t)nbr * 2 + 7) & ~(size_t)7) + 8 * s->words[i];
    }
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  s->device = dev;
  if (e == cudaSuccess) e = payload_alloc((void**)&s->d_payload, 8 * total + 16, st);
  if (e == cudaSuccess) e = alloc_index(s, st);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    e = cudaMemcpyAsync(s->d_chunk_word + (int64_t)i * nch, p + off, 8 * nch, cudaMemcpyHostToDevice, st);
    off += 8 * nch;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->d_brick_len + (int64_t)i * nbr, p + off, 2 * nbr, cudaMemcpyHostToDevice, st);
    off += ((size_t)nbr * 2 + 7) & ~(size_t)7;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->d_payload + s->word_base[i], p + off, 8 * s->words[i], cudaMemcpyHostToDevice, st);
    off += 8 * s->words[i];
  }
  if (e == cudaSuccess) e = launch_brick_offsets(s->d_brick_len, s->d_brick_off, n, nbr, st);
  if (e != cudaSuccess) {
    streams_release(s, true);
    return cuda_fail(e, "deserialize upload");
  }
  pc_status r = upload_desc(s, st);
  // every block must parse: one pass of Algorithm 2 over all components, no output
  int64_t lo[3] = {0, 0, 0}, hi[3] = {s->dims[0], s->dims[1], s->dims[2]};
  if (r == PC_OK) r = run_retrieve(s, 0, n, lo, hi, nullptr, 0, st);
  unsigned int h_err = 0;
  if (r == PC_OK) {
    e = cudaMemcpyAsync(&h_err, s->d_err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) r = cuda_fail(e, "validation");
  }
  if (r == PC_OK && h_err) r = fail(PC_ERR_CORRUPT_STREAM, "a block does not parse");
  if (r != PC_OK) {
    streams_release(s, true);
    return r;
  }
  *out = s;
  return PC_OK;
}

pc_status pc_stream_read_index(const pc_streams* s, int i, uint64_t* h_chunk_word, uint16_t* h_brick_len,
                               void* cuda_stream) {
  g_err.clear();
  if (!s || i < 0 || i >= s->n) return fail(PC_ERR_ARG, "bad streams or component index");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (h_chunk_word)
    CK(cudaMemcpyAsync(h_chunk_word, s->d_chunk_word + (int64_t)i * s->nchunks, 8 * (size_t)s->nchunks,
                       cudaMemcpyDeviceToHost, st));
  if (h_brick_len)
    CK(cudaMemcpyAsync(h_brick_len, s->d_brick_len + (int64_t)i * s->nbricks, 2 * (size_t)s->nbricks,
                       cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PC_OK;
}

pc_status pc_stream_read(const pc_streams* s, int i, uint64_t word_off, uint64_t nwords, uint64_t* h_out,
                         void* cuda_stream) {
  g_err.clear();
  if (!s || i < 0 || i >= s->n || !h_out) return fail(PC_ERR_ARG, "bad arguments");
  if (word_off > s->words[i] || nwords > s->words[i] - word_off) return fail(PC_ERR_ARG, "range outside the payload");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (nwords)
    CK(cudaMemcpyAsync(h_out, s->d_payload + s->word_base[i] + word_off, 8 * nwords, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return PC_OK;
}

void pc_streams_free(pc_streams* s) { streams_release(s); }

// The extents and checks shared by the derivative calls: nx, ny, nz of a
// field of 1..3 dimensions (PC_ERR_ARG on a bad argument).
static pc_status fd_check(const int64_t* dims, int ndims, pc_dtype dtype, double h, int64_t d3[3]) {
  if (!dims || ndims < 1 || ndims > 3) return fail(PC_ERR_ARG, "ndims must be 1, 2 or 3");
  if (dtype != PC_F32 && dtype != PC_F64) return fail(PC_ERR_ARG, "bad dtype");
  if (!(h > 0.0) || !std::isfinite(h)) return fail(PC_ERR_ARG, "h must be positive and finite");
  for (int a = 0; a < 3; ++a) {
    d3[a] = a < ndims ? dims[a] : 1;
    if (d3[a] < 1) return fail(PC_ERR_ARG, "extent < 1");
  }
  if (d3[0] > (int64_t(1) << 40) / d3[1] / d3[2]) return fail(PC_ERR_ARG, "field too large");
  if (d3[0] > INT32_MAX || d3[1] > 8 * 65535 || d3[2] > INT32_MAX) return fail(PC_ERR_ARG, "an extent is too large");
  return PC_OK;
}

// True when [a, a + n) and [b, b + n) share a byte.
static bool overlaps(const void* a, const void* b, size_t n) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + n && y < x + n;
}

pc_status pc_fd_vorticity_z(const void* u, const void* v, const int64_t* dims, int ndims, pc_dtype dtype, double h,
                            void* out, void* cuda_stream) {
  TraceRange trace_("pc_fd_vorticity_z");
  g_err.clear();
  int64_t d3[3];
  pc_status r = fd_check(dims, ndims, dtype, h, d3);
  if (r != PC_OK) return r;
  if (ndims < 2 || d3[0] < 3 || d3[1] < 3) return fail(PC_ERR_ARG, "v_x - u_y needs ndims >= 2, nx >= 3 and ny >= 3");
  if (!u || !v || !out || !is_device_ptr(u) || !is_device_ptr(v) || !is_device_ptr(out))
    return fail(PC_ERR_ARG, "u, v and out must be device memory");
  const size_t bytes = (size_t)(d3[0] * d3[1] * d3[2]) * dsize(dtype);
  if (overlaps(out, u, bytes) || overlaps(out, v, bytes)) return fail(PC_ERR_ARG, "out overlaps an input");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TimedLaunch tl(PC_KERNEL_FD, st);
  CK(launch_fd_vorticity_z(dtype, u, v, out, d3[0], d3[1], d3[2], h, st));
  return PC_OK;
}

pc_status pc_fd_second(const void* w, const int64_t* dims, int ndims, pc_dtype dtype, int axis, double h, void* out,
                       void* cuda_stream) {
  TraceRange trace_("pc_fd_second");
  g_err.clear();
  int64_t d3[3];
  pc_status r = fd_check(dims, ndims, dtype, h, d3);
  if (r != PC_OK) return r;
  if (axis < 0 || axis >= ndims) return fail(PC_ERR_ARG, "axis must be below ndims");
  if (d3[axis] < 4) return fail(PC_ERR_ARG, "a second derivative needs 4 points along the axis");
  if (!w || !out || !is_device_ptr(w) || !is_device_ptr(out)) return fail(PC_ERR_ARG, "w and out must be device memory");
  const size_t bytes = (size_t)(d3[0] * d3[1] * d3[2]) * dsize(dtype);
  if (overlaps(out, w, bytes)) return fail(PC_ERR_ARG, "out overlaps the input");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  TimedLaunch tl(PC_KERNEL_FD, st);
  CK(launch_fd_second(dtype, w, out, d3[0], d3[1], d3[2], axis, h, st));
  return PC_OK;
}

pc_status pc_release_cached_memory(void) {
  g_err.clear();
  int cur = 0;
  CK(cudaGetDevice(&cur));
  cudaError_t e = cudaSuccess;
  std::lock_guard<std::mutex> lk(g_mu);  // the construction bit pools
  std::lock_guard<std::mutex> lp(g_pool_mu);
  for (int dev = 0; dev < 128; ++dev) {
    if (!g_pools[0][dev] && !g_pools[1][dev] && !g_ctx[dev].pool) continue;
    if (e == cudaSuccess) e = cudaSetDevice(dev);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) break;
    if (g_ctx[dev].pool) {
      e = cudaFree(g_ctx[dev].pool);
      g_ctx[dev].pool = nullptr;
      g_ctx[dev].pool_words = 0;
    }
    for (int w = 0; w < 2; ++w)
      if (e == cudaSuccess && g_pools[w][dev]) e = cudaMemPoolTrimTo(g_pools[w][dev], 0);
  }
  const cudaError_t e2 = cudaSetDevice(cur);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return cuda_fail(e, "pc_release_cached_memory");
  return PC_OK;
}

pc_status pc_timing_enable(int on) {
  g_err.clear();
  CK(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_timing.mu);
  for (auto& p : g_timing.pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_timing.pending.clear();
  for (int k = 0; k < PC_KERNEL_KINDS; ++k) {
    g_timing.ms[k] = 0;
    g_timing.launches[k] = 0;
  }
  g_timing.on = on != 0;
  return PC_OK;
}

pc_status pc_timing_read(double* ms, uint64_t* launches) {
  g_err.clear();
  if (!ms || !launches) return fail(PC_ERR_ARG, "NULL argument");
  CK(cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(g_timing.mu);
  for (auto& p : g_timing.pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
      g_timing.ms[p.kind] += t;
      g_timing.launches[p.kind] += 1;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_timing.pending.clear();
  for (int k = 0; k < PC_KERNEL_KINDS; ++k) {
    ms[k] = g_timing.ms[k];
    launches[k] = g_timing.launches[k];
  }
  return PC_OK;
}

pc_status pc_field_range(const void* d_field, int64_t count, pc_dtype dtype, void* cuda_stream, double* vmin,
                         double* vmax) {
  TraceRange trace_("pc_field_range");
  g_err.clear();
  if (!d_field || count < 1 || !vmin || !vmax) return fail(PC_ERR_ARG, "bad arguments");
  if (dtype != PC_F32 && dtype != PC_F64) return fail(PC_ERR_ARG, "bad dtype");
  const void* kp = nullptr;
  bool host = false;
  if (!kernel_pointer(d_field, &kp, &host)) return fail(PC_ERR_ARG, "field must be device or pinned host memory");
  d_field = kp;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  Scratch scr(st);
  unsigned long long* enc = nullptr;
  CK(scr.get((void**)&enc, 32));
  unsigned int* flags = (unsigned int*)(enc + 2);
  unsigned long long init[4] = {~0ull, 0ull, 0ull, 0ull};
  CK(cudaMemcpyAsync(enc, init, 32, cudaMemcpyHostToDevice, st));
  {
    TimedLaunch tl(PC_KERNEL_RANGE, st);
    CK(launch_range(dtype, d_field, count, enc, flags, st));
  }
  unsigned long long h[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(h, enc, 24, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if ((unsigned int)h[2] & kFlagNonFinite) return fail(PC_ERR_NONFINITE, "the field holds a NaN or an infinity");
  for (int w = 0; w < 2; ++w) {  // undo the order-preserving key
    double v;
    if (dtype == PC_F32) {
      uint32_t k = (uint32_t)h[w];
      uint32_t b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
      float f;
      std::memcpy(&f, &b, 4);
      v = f;
    } else {
      uint64_t k = h[w];
      uint64_t b = (k & 0x8000000000000000ull) ? (k & 0x7fffffffffffffffull) : ~k;
      std::memcpy(&v, &b, 8);
    }
    (w ? *vmax : *vmin) = v;
  }
  return PC_OK;
}

}  // extern "C"
