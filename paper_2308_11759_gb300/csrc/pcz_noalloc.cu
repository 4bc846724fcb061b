// pcz_noalloc.cu -- pc_compress_noalloc: the construction path of
// pc_compress with every piece of scratch memory taken from one fixed,
// file-scope device array instead of device allocations.
//
// Who needs it: callers that cannot allocate device memory while they run --
// for example a host whose memory allocator has already reserved all free
// device memory for itself (a framework's caching allocator or an
// application-level pool), or a latency-critical loop that must not make the
// implicitly synchronising cudaMalloc/cudaFree calls.  Such a caller passes
// its own output buffers; everything temporary lives in kScratch below.
//
// The scratch array is shared by every call in the process: two calls whose
// kernels overlap on the GPU (on different streams, or from different host
// threads) race on it and corrupt each other's output.  Serialise them.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include <cuda_runtime.h>

#include "../../include/pcz.h"
#include "pcz_host.h"
#include "pcz_kernels.h"

using namespace pcz;

namespace {

// 64 MiB of scratch on every GPU that loads this library, held until the
// process exits.  It bounds the fields pc_compress_noalloc accepts (see the
// size check below).
constexpr size_t kScratchBytes = size_t(64) << 20;
static __device__ __align__(256) unsigned char kScratch[kScratchBytes];

// Device address of kScratch per device, looked up once with that device
// current (the host-side name kScratch is only a stand-in for it).
std::mutex g_nomu;
void* g_scratch_addr[128] = {};

pc_status nfail(pc_status st, const std::string& m) {
  set_last_error(m.c_str());  // reported by pc_last_error()
  return st;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Largest bit string one brick and component can take (a CODED block whose
// every plane is non-empty), as in the compress kernel.
int64_t max_brick_bits(pc_dtype dt) { return dt == PC_F32 ? 2 + 3 + 8 + 32 * 129 : 2 + 3 + 11 + 64 * 129; }

// Pool words the worst chunk (32 such bricks) takes.
uint64_t worst_chunk_words(pc_dtype dt) { return (uint64_t)((kChunk * max_brick_bits(dt) + 63) / 64); }

// Byte offsets of the scratch regions for n components of nchunks chunks:
// per (component, chunk) 32 bytes of metadata (word count, pool offset, five
// counters), per component 56 bytes (total, counters, payload base), the
// flags, and then the bit pool.
struct Layout {
  size_t nwords, cpool, ccnt, tot, cnt, flags, base, pool;
};
Layout layout(int n, int64_t nchunks) {
  Layout l;
  l.nwords = 0;
  l.cpool = align256(l.nwords + 4 * (size_t)n * nchunks);
  l.ccnt = align256(l.cpool + 8 * (size_t)n * nchunks);
  l.tot = align256(l.ccnt + 20 * (size_t)n * nchunks);
  l.cnt = align256(l.tot + 8 * (size_t)n);
  l.flags = align256(l.cnt + 40 * (size_t)n);
  l.base = align256(l.flags + 16);
  l.pool = align256(l.base + 8 * (size_t)n);
  return l;
}
// True when the worst case of every chunk of every component fits the pool.
bool fits(const Layout& l, int n, int64_t nchunks, uint64_t chunk_worst_words) {
  if (l.pool > kScratchBytes) return false;
  return chunk_worst_words * (uint64_t)n * (uint64_t)nchunks <= (kScratchBytes - l.pool) / 8;
}

}  // namespace

extern "C" {

pc_status pc_compress_noalloc(const void* d_field, const int64_t* dims, int ndims, pc_dtype dtype,
                              const double* tau, int n, uint64_t* d_payload, uint64_t payload_capacity_words,
                              uint64_t* d_chunk_word, uint16_t* d_brick_len, uint64_t* h_words,
                              uint64_t* h_counts, void* cuda_stream) {
  set_last_error("");
  if (!d_field || !dims || !tau || !d_payload || !d_chunk_word || !d_brick_len || !h_words || !h_counts)
    return nfail(PC_ERR_ARG, "NULL argument");
  if (ndims != 3) return nfail(PC_ERR_ARG, "pc_compress_noalloc codes 3D fields only");
  if (dtype != PC_F32 && dtype != PC_F64) return nfail(PC_ERR_ARG, "bad dtype");
  if (n < 1 || n > PC_MAX_COMPONENTS) return nfail(PC_ERR_ARG, "n out of range");
  for (int i = 0; i < n; ++i) {
    if (!(tau[i] > 0) || tau[i] != tau[i] || tau[i] > 1.7976931348623157e308 || (i && !(tau[i] < tau[i - 1])))
      return nfail(PC_ERR_TAU_ORDER, "tolerances must be finite, positive, strictly decreasing");
  }
  int64_t d3[3], nb[3];
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1) return nfail(PC_ERR_ARG, "extent < 1");
    d3[a] = dims[a];
    nb[a] = (dims[a] + 3) / 4;
  }
  const int64_t nbricks = nb[0] * nb[1] * nb[2];
  const int64_t nchunks = (nbricks + kChunk - 1) / kChunk;

  // scratch layout: per-chunk metadata, totals, flags, then the bit pool
  const Layout lay = layout(n, nchunks);
  const uint64_t chunk_worst_words = worst_chunk_words(dtype);
  if (!fits(lay, n, nchunks, chunk_worst_words)) {
    // the largest n * ceil(bricks/32) that fits for this n, from the same layout
    int64_t lo = 0, hi = (int64_t)(kScratchBytes / 8 / chunk_worst_words) + 1;  // fits(lo), !fits(hi)
    while (hi - lo > 1) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (fits(layout(n, mid), n, mid, chunk_worst_words)) lo = mid; else hi = mid;
    }
    return nfail(PC_ERR_ARG, "field too large for the fixed 64 MiB scratch of pc_compress_noalloc: with n = " +
                                 std::to_string(n) + " it needs n * ceil(bricks/32) <= " + std::to_string((int64_t)n * lo) +
                                 " (bricks are 4x4x4 values); use pc_compress");
  }
  // outputs and the field must be device memory the kernels can write/read
  if (!device_pointer(d_field) || !device_pointer(d_payload) || !device_pointer(d_chunk_word) ||
      !device_pointer(d_brick_len))
    return nfail(PC_ERR_ARG, "d_field, d_payload, d_chunk_word and d_brick_len must be device memory");
  const size_t off_nwords = lay.nwords, off_cpool = lay.cpool, off_ccnt = lay.ccnt, off_tot = lay.tot,
               off_cnt = lay.cnt, off_flags = lay.flags, off_base = lay.base, off_pool = lay.pool;

  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return nfail(PC_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_nomu);
    if (!g_scratch_addr[dev & 127]) {  // set-up, once per device, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, kScratch);
      if (e != cudaSuccess) return nfail(PC_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[dev & 127] = p;
    }
    base = (unsigned char*)g_scratch_addr[dev & 127];
  }

  CompressParams P;
  std::memset(&P, 0, sizeof(P));
  P.field = d_field;
  for (int a = 0; a < 3; ++a) {
    P.dims[a] = d3[a];
    P.nb[a] = nb[a];
  }
  P.nbricks = nbricks;
  P.nchunks = nchunks;
  P.n = n;
  for (int i = 0; i < n; ++i) {
    uint64_t tb;
    if (dtype == PC_F64) {
      std::memcpy(&tb, &tau[i], 8);
    } else {
      float f = (float)tau[i];
      if ((double)f > tau[i]) f = std::nextafterf(f, 0.0f);
      uint32_t b32;
      std::memcpy(&b32, &f, 4);
      tb = b32;
    }
    P.tau_bits[i] = tb;
    int E;
    std::frexp(tau[i], &E);
    P.L[i] = E - 1;
  }
  uint32_t* chunk_nwords = (uint32_t*)(base + off_nwords);
  uint64_t* chunk_pool = (uint64_t*)(base + off_cpool);
  uint32_t* chunk_counts = (uint32_t*)(base + off_ccnt);
  uint64_t* totals = (uint64_t*)(base + off_tot);
  unsigned long long* counts = (unsigned long long*)(base + off_cnt);
  unsigned int* flags = (unsigned int*)(base + off_flags);
  unsigned long long* used = (unsigned long long*)(base + off_flags + 8);
  uint64_t* comp_base = (uint64_t*)(base + off_base);
  P.pool = (uint64_t*)(base + off_pool);
  P.pool_words = (kScratchBytes - off_pool) / 8;
  P.pool_used = used;
  P.chunk_nwords = chunk_nwords;
  P.chunk_pool = chunk_pool;
  P.brick_len = d_brick_len;
  P.chunk_counts = chunk_counts;
  P.flags = flags;

  // the flags and the pool's bump counter must start at zero on every call
  e = cudaMemsetAsync(flags, 0, 16, st);
  if (e == cudaSuccess) e = launch_compress(dtype, ndims, P, st);
  if (e == cudaSuccess) e = launch_scan_chunks(chunk_nwords, d_chunk_word, totals, chunk_counts, counts, nullptr, nullptr, n,
                                                nchunks, st);
  unsigned int h_flags = 0;
  unsigned long long hc[5 * PC_MAX_COMPONENTS];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_words, totals, 8 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc, counts, 40 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_flags, flags, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nfail(PC_ERR_CUDA, std::string("compress: ") + cudaGetErrorString(e));
  }
  for (int k = 0; k < 5 * n; ++k) h_counts[k] = hc[k];
  if (h_flags & kFlagNonFinite) return nfail(PC_ERR_NONFINITE, "the field holds a NaN or an infinity");
  if (h_flags & kFlagPoolOverflow) return nfail(PC_ERR_ARG, "compressed data exceeded the fixed scratch");
  uint64_t cb[PC_MAX_COMPONENTS];
  uint64_t total = 0;
  for (int i = 0; i < n; ++i) {
    cb[i] = total;
    total += h_words[i];
  }
  if (total > payload_capacity_words)
    return nfail(PC_ERR_ARG, "payload buffer too small: need " + std::to_string(total) + " words");
  e = cudaMemcpyAsync(comp_base, cb, 8 * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_pack(P.pool, chunk_nwords, chunk_pool, d_chunk_word, comp_base, d_payload, n, nchunks, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return nfail(PC_ERR_CUDA, std::string("pack: ") + cudaGetErrorString(e));
  }
  return PC_OK;
}

}  // extern "C"
