// pcz_batch.cu -- Algorithm 1 (Magri & Lindstrom, Sec. 4.1) over a batch of
// fields of uneven sizes and dimensionalities in one persistent launch, and
// Algorithm 2 (Sec. 4.2) over a batch of boxes of several fields.
//
// Construction: two kernels run side by side (two branches of one CUDA
// graph), or one kernel does both parts.  In the 3D kernel, CTAs of 512
// threads claim items from a work counter; an item is one chunk of 32 bricks of a 3D field, which the
// whole CTA codes as pcz_compress.cu does.  In the 1D/2D kernel, CTAs of a
// few warps claim items of several chunks of a 1D or 2D field from a second
// counter, and each warp codes one chunk at a time, a brick per lane, as
// pcz_small.cu does (no register cap: a 2D brick of float64 values lives in
// one thread's registers).  All fields share one scratch pool and one set of
// chunk arrays; a segmented scan (one segment per field and component) places
// every chunk in its component's stream, and a packing kernel copies the
// chunks there.  The schedule (field order, CTAs per SM of the 3D kernel,
// warps per CTA and chunks per item of the 1D/2D kernel, items per claim) is
// picked by a small autotuner that times the candidates on the plan's first
// batch.  The launches up to the scan are captured in CUDA graphs, one per
// kernel shape; the pointers and tolerances of each call reach the kernels
// through parameter blocks that the graph copies from pinned host memory, so
// one graph serves every call.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "pcz_chunk3.cuh"
#include "pcz_chunk_small.cuh"
#include "pcz_host.h"

namespace pcz {

template <typename T, int W>
__host__ __device__ constexpr size_t batch_small_smem() {  // a chunk buffer per warp, sized for 2D bricks
  return (size_t)W * chunk_words_small<T, 2>() * 4;
}

// The item of work list `bp` that `it` falls in: its slot's field, first chunk,
// chunk count and dimensionality, written to the CTA's shared copies.
__device__ __forceinline__ void find_item(const BatchParams* __restrict__ bp, int64_t it, int* f_out, int64_t* c0_out,
                                          int* nch_out, int* nd_out) {
  int lo = 0, hi = bp->nslots - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bp->slot_first[mid] <= it)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int f = bp->slot_field[lo];
  const int w = bp->slot_width[lo];
  const int64_t c0 = (it - bp->slot_first[lo]) * w;
  const int64_t nch = bp->fields[f].nchunks;
  *f_out = f;
  *c0_out = c0;
  *nch_out = (int)(nch - c0 < w ? nch - c0 : w);
  *nd_out = bp->slot_ndims[lo];
}

// 3D part of a batch: CTAs of 16 warps claim chunks of the 3D
// fields (one chunk of 32 bricks per item) and code each as pc_compress does.
// MINB = CTAs per SM the variant is compiled for: 1 (up to 128 registers per
// thread) or 2 (at most 64, two CTAs sharing an SM).
template <typename T, int MINB>
__global__ void __launch_bounds__(kCompressThreads3, MINB) k_batch3(const BatchParams* __restrict__ bp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CompressParams sP;
  __shared__ long long s_first, s_chunk0;
  __shared__ int s_field, s_nchunks, s_ndims;
  static_assert(sizeof(CompressParams) % 8 == 0, "parameter copy");
  constexpr int PW = (int)(sizeof(CompressParams) / 8);
  const int tid = threadIdx.x;
  const int64_t nitems = bp->nitems;
  const int per = bp->per_fetch;
  for (;;) {
    __syncthreads();  // every thread is done with the previous claim
    if (tid == 0) s_first = (long long)atomicAdd(bp->next, (unsigned long long)per);
    __syncthreads();
    const int64_t first = s_first;
    if (first >= nitems) break;
    const int64_t last = first + per < nitems ? first + per : nitems;
    for (int64_t it = first; it < last; ++it) {
      __syncthreads();  // the previous item is done with sP and the buffers
      if (tid == 0) {
        int f, nch, nd;
        int64_t c0;
        find_item(bp, it, &f, &c0, &nch, &nd);
        s_field = f;
        s_chunk0 = c0;
        s_nchunks = nch;
        s_ndims = nd;
      }
      __syncthreads();
      {
        const uint64_t* src = reinterpret_cast<const uint64_t*>(bp->fields + s_field);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&sP);
        for (int w = tid; w < PW; w += kCompressThreads3) dst[w] = src[w];
      }
      __syncthreads();
      compress3_chunk<T>(sP, s_chunk0, smem);
    }
  }
}

// 1D/2D part of a batch: CTAs of W warps claim items of `width`
// chunks of the 1D and 2D fields; the CTA's warps take the item's chunks one
// at a time (a brick per lane, as in pcz_small.cu).  Float32 variants are
// held to 128 registers so that 16 warps share an SM; float64 ones have no
// cap, because a 2D brick of float64 values lives in one thread's registers.
template <typename T, int W>
__global__ void __launch_bounds__(32 * W, sizeof(T) == 4 ? 16 / W : 1) k_batch_small(const BatchParams* __restrict__ bp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CompressParams sP;
  __shared__ long long s_first, s_chunk0;
  __shared__ int s_field, s_nchunks, s_ndims;
  constexpr int PW = (int)(sizeof(CompressParams) / 8);
  constexpr int NT = 32 * W;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t nitems = bp->nitems;
  const int per = bp->per_fetch;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_first = (long long)atomicAdd(bp->next, (unsigned long long)per);
    __syncthreads();
    const int64_t first = s_first;
    if (first >= nitems) break;
    const int64_t last = first + per < nitems ? first + per : nitems;
    for (int64_t it = first; it < last; ++it) {
      __syncthreads();
      if (tid == 0) {
        int f, nch, nd;
        int64_t c0;
        find_item(bp, it, &f, &c0, &nch, &nd);
        s_field = f;
        s_chunk0 = c0;
        s_nchunks = nch;
        s_ndims = nd;
      }
      __syncthreads();
      {
        const uint64_t* src = reinterpret_cast<const uint64_t*>(bp->fields + s_field);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&sP);
        for (int w = tid; w < PW; w += NT) dst[w] = src[w];
      }
      __syncthreads();
      const int64_t c0 = s_chunk0;
      const int nch = s_nchunks;
      if (s_ndims == 2) {
        uint32_t* cbuf = reinterpret_cast<uint32_t*>(smem) + (size_t)warp * chunk_words_small<T, 2>();
        for (int c = warp; c < nch; c += W) compress_small_chunk<T, 2>(sP, c0 + c, cbuf);
      } else {
        uint32_t* cbuf = reinterpret_cast<uint32_t*>(smem) + (size_t)warp * chunk_words_small<T, 1>();
        for (int c = warp; c < nch; c += W) compress_small_chunk<T, 1>(sP, c0 + c, cbuf);
      }
    }
  }
}

// Both parts in one kernel: CTAs of 16 warps (up to 128 registers per thread)
// claim items of one work list holding the 3D and the 1D/2D fields; a 3D item
// takes the whole CTA, a 1D/2D item one chunk per warp at a time.  With one
// queue the two kinds of work share the SMs to the end.
template <typename T>
__global__ void __launch_bounds__(kCompressThreads3, 1) k_batch_mixed(const BatchParams* __restrict__ bp) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ CompressParams sP;
  __shared__ long long s_first, s_chunk0;
  __shared__ int s_field, s_nchunks, s_ndims;
  constexpr int PW = (int)(sizeof(CompressParams) / 8);
  constexpr int WARPS = kCompressThreads3 / 32;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t nitems = bp->nitems;
  const int per = bp->per_fetch;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_first = (long long)atomicAdd(bp->next, (unsigned long long)per);
    __syncthreads();
    const int64_t first = s_first;
    if (first >= nitems) break;
    const int64_t last = first + per < nitems ? first + per : nitems;
    for (int64_t it = first; it < last; ++it) {
      __syncthreads();
      if (tid == 0) {
        int f, nch, nd;
        int64_t c0;
        find_item(bp, it, &f, &c0, &nch, &nd);
        s_field = f;
        s_chunk0 = c0;
        s_nchunks = nch;
        s_ndims = nd;
      }
      __syncthreads();
      {
        const uint64_t* src = reinterpret_cast<const uint64_t*>(bp->fields + s_field);
        uint64_t* dst = reinterpret_cast<uint64_t*>(&sP);
        for (int w = tid; w < PW; w += kCompressThreads3) dst[w] = src[w];
      }
      __syncthreads();
      const int64_t c0 = s_chunk0;
      const int nch = s_nchunks;
      if (s_ndims == 3) {
        compress3_chunk<T>(sP, c0, smem);
      } else if (s_ndims == 2) {
        uint32_t* cbuf = reinterpret_cast<uint32_t*>(smem) + (size_t)warp * chunk_words_small<T, 2>();
        for (int c = warp; c < nch; c += WARPS) compress_small_chunk<T, 2>(sP, c0 + c, cbuf);
      } else {
        uint32_t* cbuf = reinterpret_cast<uint32_t*>(smem) + (size_t)warp * chunk_words_small<T, 1>();
        for (int c = warp; c < nch; c += WARPS) compress_small_chunk<T, 1>(sP, c0 + c, cbuf);
      }
    }
  }
}

template <typename T>
__host__ __device__ constexpr size_t batch_mixed_smem() {
  const size_t a = compress_smem3<T>();
  const size_t b = (size_t)(kCompressThreads3 / 32) * chunk_words_small<T, 2>() * 4;
  return a > b ? a : b;
}

template <typename T>
static int batch_mixed_grid_t() {
  // CTAs that fit on the GPU at once, queried once (thread-safe initialisation);
  // also sets the kernel's shared-memory limit, which launches and graph
  // captures need
  static const int grid = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_batch_mixed<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)batch_mixed_smem<T>());
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_mixed<T>, kCompressThreads3, batch_mixed_smem<T>()) !=
        cudaSuccess) {
      cudaGetLastError();
      per = 1;
    }
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }();
  return grid;
}

// The mixed kernel exists for float32 only: its CTAs of 16 warps hold a
// thread to 128 registers, and a 2D float64 brick coded in one thread's
// registers needs more (it would spill about 2 KB per thread).
int compress_batch_mixed_grid(int dtype) { return dtype == 1 ? batch_mixed_grid_t<float>() : 0; }

cudaError_t launch_compress_batch_mixed(int dtype, const BatchParams* d_bp, int grid, cudaStream_t s) {
  if (dtype != 1) return cudaErrorNotSupported;
  k_batch_mixed<float><<<grid, kCompressThreads3, batch_mixed_smem<float>(), s>>>(d_bp);
  return cudaGetLastError();
}

template <typename T, int MINB>
static int batch3_grid_t() {
  // CTAs that fit on the GPU at once, queried once (thread-safe initialisation);
  // also sets the kernel's shared-memory limit, which launches and graph
  // captures need
  static const int grid = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_batch3<T, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)compress_smem3<T>());
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch3<T, MINB>, kCompressThreads3, compress_smem3<T>()) !=
        cudaSuccess) {
      cudaGetLastError();
      per = 1;
    }
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }();
  return grid;
}

template <typename T, int W>
static int batch_small_grid_t() {
  // CTAs that fit on the GPU at once, queried once (thread-safe initialisation);
  // also sets the kernel's shared-memory limit, which launches and graph
  // captures need
  static const int grid = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_batch_small<T, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)batch_small_smem<T, W>());
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_small<T, W>, 32 * W, batch_small_smem<T, W>()) !=
        cudaSuccess) {
      cudaGetLastError();
      per = 1;
    }
    return (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  }();
  return grid;
}

uint32_t check_word_batch(int reset) { return read_check_word(reset); }

int compress_batch_grid(int dtype, int minb) {
  if (dtype == 1) return minb == 2 ? batch3_grid_t<float, 2>() : batch3_grid_t<float, 1>();
  return minb == 2 ? batch3_grid_t<double, 2>() : batch3_grid_t<double, 1>();
}

int compress_batch_small_grid(int dtype, int warps) {
  if (dtype == 1)
    return warps == 2   ? batch_small_grid_t<float, 2>()
           : warps == 4 ? batch_small_grid_t<float, 4>()
           : warps == 8 ? batch_small_grid_t<float, 8>()
                        : batch_small_grid_t<float, 16>();
  return warps == 2   ? batch_small_grid_t<double, 2>()
         : warps == 4 ? batch_small_grid_t<double, 4>()
         : warps == 8 ? batch_small_grid_t<double, 8>()
                      : 0;  // no 16-warp float64 variant (see launch_small_t)
}

cudaError_t launch_compress_batch(int dtype, int minb, const BatchParams* d_bp, int grid, cudaStream_t s) {
  if (dtype == 1) {
    if (minb == 2)
      k_batch3<float, 2><<<grid, kCompressThreads3, compress_smem3<float>(), s>>>(d_bp);
    else
      k_batch3<float, 1><<<grid, kCompressThreads3, compress_smem3<float>(), s>>>(d_bp);
  } else {
    if (minb == 2)
      k_batch3<double, 2><<<grid, kCompressThreads3, compress_smem3<double>(), s>>>(d_bp);
    else
      k_batch3<double, 1><<<grid, kCompressThreads3, compress_smem3<double>(), s>>>(d_bp);
  }
  return cudaGetLastError();
}

// CTAs of 16 warps exist for float32 only: 512 threads leave 128 registers a
// thread, fewer than a 2D float64 brick in one thread's registers takes.
template <typename T>
static cudaError_t launch_small_t(int warps, const BatchParams* d_bp, int grid, cudaStream_t s) {
  if (warps == 2) {
    k_batch_small<T, 2><<<grid, 64, batch_small_smem<T, 2>(), s>>>(d_bp);
  } else if (warps == 4) {
    k_batch_small<T, 4><<<grid, 128, batch_small_smem<T, 4>(), s>>>(d_bp);
  } else if (warps == 8) {
    k_batch_small<T, 8><<<grid, 256, batch_small_smem<T, 8>(), s>>>(d_bp);
  } else {
    if constexpr (sizeof(T) == 4)
      k_batch_small<T, 16><<<grid, 512, batch_small_smem<T, 16>(), s>>>(d_bp);
    else
      return cudaErrorNotSupported;
  }
  return cudaGetLastError();
}

cudaError_t launch_compress_batch_small(int dtype, int warps, const BatchParams* d_bp, int grid, cudaStream_t s) {
  return dtype == 1 ? launch_small_t<float>(warps, d_bp, grid, s) : launch_small_t<double>(warps, d_bp, grid, s);
}

}  // namespace pcz

using namespace pcz;

namespace {

#define BK(call)                                                    \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return api_cuda_fail(e_, #call);         \
  } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Device arrays of one batch's streams, shared by its pc_streams objects.
struct BatchArena {
  void* index = nullptr;
  void* payload = nullptr;
  ~BatchArena() {
    cudaFree(index);
    cudaFree(payload);
  }
};

// A schedule of the batched construction: the order of the fields' work,
// the block shapes of the two persistent kernels and how much a claim takes.
// A 3D item is one chunk of 32 bricks for a whole CTA of 16 warps (two bricks
// per warp); `ctas3` such CTAs share an SM (1 at up to 128 registers per
// thread, 2 at 64).  A 1D/2D item is warps_small * chunks_per_warp chunks
// for a CTA of warps_small warps, one chunk (a brick per lane) per warp at a
// time.
struct Schedule {
  int order;            // 0: fields in the caller's order; 1: largest first
  int ctas3;            // CTAs per SM of the 3D kernel: 1 or 2; 0: one kernel for both parts, whose
                        // CTAs of 16 warps take 3D and 1D/2D items from one queue
  int warps_small;      // warps per CTA of the 1D/2D kernel: 2, 4, 8 or 16
  int chunks_per_warp;  // chunks per warp in a 1D/2D item: 1 or 2
  int per_fetch;        // items per claim
};

const Schedule kSchedules[] = {
    {1, 2, 4, 1, 1},  {1, 2, 8, 1, 1},  {1, 2, 16, 1, 1}, {1, 1, 4, 1, 1},  {1, 1, 8, 1, 1},  {1, 1, 16, 1, 1},
    {1, 2, 4, 2, 1},  {1, 2, 8, 2, 1},  {1, 2, 16, 2, 1}, {1, 2, 2, 1, 1},  {1, 2, 2, 2, 1},  {1, 0, 16, 1, 1},
    {1, 0, 16, 2, 1}, {1, 2, 8, 1, 2},  {1, 2, 16, 1, 2}, {0, 2, 16, 1, 1}};
constexpr int kNumSchedules = (int)(sizeof(kSchedules) / sizeof(kSchedules[0]));
constexpr int kSmallShapes[4] = {2, 4, 8, 16};
constexpr int kVariants = 9;  // graphs: 2 x 4 two-kernel shapes and the mixed kernel

// Graph of the kernel variants (3D CTAs per SM x 1D/2D warps per CTA: 0..7;
// the single mixed kernel: 8).
int variant_of(const Schedule& sc) {
  if (sc.ctas3 == 0) return 8;
  const int w = sc.warps_small == 2 ? 0 : sc.warps_small == 4 ? 1 : sc.warps_small == 8 ? 2 : 3;
  return (sc.ctas3 - 1) * 4 + w;
}

// Kernel variants that exist for the type: float64 has neither 16-warp 1D/2D
// CTAs nor the mixed kernel (both would hold a thread to 128 registers).
bool variant_exists(int v, pc_dtype dt) {
  return dt == PC_F32 || (v != kVariants - 1 && kSmallShapes[v % 4] != 16);
}
bool schedule_exists(const Schedule& sc, pc_dtype dt) { return variant_exists(variant_of(sc), dt); }

}  // namespace

struct pc_batch {
  int device = 0;
  cudaStream_t st = nullptr;      // the plan's own stream (graphs cannot capture the legacy stream)
  cudaStream_t caller = nullptr;  // the caller's stream, waited for before each call
  cudaEvent_t ready = nullptr;
  pc_dtype dtype = PC_F32;
  int n = 0, nfields = 0, nseg = 0;
  std::vector<int> ndims;
  std::vector<int64_t> dims;  // 3 per field
  std::vector<int64_t> d3, nb, nbricks, nchunks, cbase, bbase;
  int64_t nentries = 0, nbentries = 0;
  // plan-owned device scratch
  void* scratch = nullptr;
  CompressParams* d_fields = nullptr;
  BatchParams* d_bp = nullptr;  // [2]: the 3D work list, the 1D/2D work list
  ScanParams* d_sp = nullptr;
  int32_t* d_slot_field = nullptr;
  int32_t* d_slot_width = nullptr;
  int32_t* d_slot_ndims = nullptr;
  int64_t* d_slot_first = nullptr;
  uint32_t* d_nwords = nullptr;
  uint64_t* d_chunk_pool = nullptr;
  uint32_t* d_counts = nullptr;
  uint64_t* d_maxerr_c = nullptr;
  uint64_t* d_totals = nullptr;
  unsigned long long* d_segcounts = nullptr;
  unsigned long long* d_segmaxerr = nullptr;
  int64_t* d_seg_start = nullptr;
  int64_t* d_seg_len = nullptr;
  uint64_t* d_seg_base = nullptr;
  unsigned int* d_flags = nullptr;
  unsigned long long* d_used = nullptr;
  unsigned long long* d_next = nullptr;
  uint64_t* pool = nullptr;
  uint64_t pool_words = 0;
  // pinned host mirrors
  void* pinned = nullptr;
  CompressParams* h_fields = nullptr;
  BatchParams* h_bp = nullptr;  // [2]
  ScanParams* h_sp = nullptr;
  int32_t* h_slot_field = nullptr;
  int32_t* h_slot_width = nullptr;
  int32_t* h_slot_ndims = nullptr;
  int64_t* h_slot_first = nullptr;
  uint64_t* h_totals = nullptr;
  unsigned long long* h_segcounts = nullptr;
  unsigned long long* h_segmaxerr = nullptr;
  unsigned int* h_flags = nullptr;
  unsigned long long* h_used = nullptr;
  // graphs (one per kernel variant: 3D CTAs per SM x 1D/2D warps per CTA) and schedule
  cudaStream_t st2 = nullptr;  // the 1D/2D kernel's branch of the graph
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaGraphExec_t execs[kVariants] = {};
  int grid_mixed = 0;
  cudaGraphExec_t exec = nullptr;  // the current schedule's
  int grid3[2] = {0, 0};
  int grid_small[4] = {0, 0, 0, 0};
  int grid = 0;
  int schedule = -1;
  double tune_ms[kNumSchedules] = {};
  uint64_t calls = 0;
};

namespace {

void batch_release(pc_batch* B) {
  if (!B) return;
  if (B->st) cudaStreamSynchronize(B->st);
  for (cudaGraphExec_t x : B->execs)
    if (x) cudaGraphExecDestroy(x);
  if (B->ready) cudaEventDestroy(B->ready);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->join) cudaEventDestroy(B->join);
  if (B->st2) cudaStreamDestroy(B->st2);
  if (B->st) cudaStreamDestroy(B->st);
  cudaFree(B->scratch);
  cudaFree(B->pool);
  cudaFreeHost(B->pinned);
  delete B;
}

// The two work lists of a schedule (3D fields, then 1D/2D fields), as slots
// in the pinned mirrors: list 0 at slot arrays [0, F), list 1 at [F, 2F).
void set_schedule(pc_batch* B, const Schedule& sc) {
  std::vector<int> ord(B->nfields);
  std::iota(ord.begin(), ord.end(), 0);
  if (sc.order == 1) {
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      return B->nbricks[a] * (B->ndims[a] == 3 ? 4 : 1) > B->nbricks[b] * (B->ndims[b] == 3 ? 4 : 1);
    });
  }
  const int F = B->nfields;
  for (int list = 0; list < 2; ++list) {
    int64_t items = 0;
    int ns = 0;
    const int base = list * F;
    for (int f : ord) {
      if (sc.ctas3 == 0 ? list == 1 : (B->ndims[f] == 3) != (list == 0)) continue;
      const int w = B->ndims[f] == 3 ? 1 : sc.warps_small * sc.chunks_per_warp;
      B->h_slot_field[base + ns] = f;
      B->h_slot_width[base + ns] = w;
      B->h_slot_ndims[base + ns] = B->ndims[f];
      B->h_slot_first[base + list + ns] = items;
      items += (B->nchunks[f] + w - 1) / w;
      ++ns;
    }
    B->h_slot_first[base + list + ns] = items;
    BatchParams& bp = B->h_bp[list];
    bp.nslots = ns;
    bp.nitems = items;
    bp.per_fetch = sc.per_fetch;
  }
  B->exec = B->execs[variant_of(sc)];
  B->grid = sc.ctas3 == 0 ? B->grid_mixed : B->grid3[sc.ctas3 - 1];
}

// Captures H2D of the parameter blocks, the counters' reset, the batched
// construction (kernel variant v: the 3D kernel for v / 3 + 1 CTAs per SM and,
// on a parallel branch, the 1D/2D kernel with kSmallShapes[v % 3] warps per
// CTA), the segmented scan and the D2H of the results.
pc_status capture_graph(pc_batch* B, int v) {
  cudaStream_t st = B->st;
  cudaGraph_t g = nullptr;
  BK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaMemcpyAsync(B->d_fields, B->h_fields, sizeof(CompressParams) * B->nfields,
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_bp, B->h_bp, 2 * sizeof(BatchParams), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_sp, B->h_sp, sizeof(ScanParams), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_slot_field, B->h_slot_field, 8 * (size_t)B->nfields, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_slot_width, B->h_slot_width, 8 * (size_t)B->nfields, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_slot_ndims, B->h_slot_ndims, 8 * (size_t)B->nfields, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->d_slot_first, B->h_slot_first, 16 * (size_t)(B->nfields + 1), cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_flags, 0, 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_used, 0, 16, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->d_next, 0, 16, st);
  // fork: the 1D/2D kernel on the second stream, the 3D kernel on the first
  if (v == kVariants - 1) {
    if (e == cudaSuccess) e = launch_compress_batch_mixed(B->dtype, B->d_bp, B->grid_mixed, st);
  } else {
    if (e == cudaSuccess) e = cudaEventRecord(B->fork, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->st2, B->fork, 0);
    if (e == cudaSuccess)
      e = launch_compress_batch_small(B->dtype, kSmallShapes[v % 4], B->d_bp + 1, B->grid_small[v % 4], B->st2);
    if (e == cudaSuccess) e = cudaEventRecord(B->join, B->st2);
    if (e == cudaSuccess) e = launch_compress_batch(B->dtype, v / 4 + 1, B->d_bp, B->grid3[v / 4], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, B->join, 0);
  }
  if (e == cudaSuccess) e = launch_scan_segments(B->d_sp, B->nseg, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->h_totals, B->d_totals, 8 * (size_t)B->nseg, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->h_segcounts, B->d_segcounts, 40 * (size_t)B->nseg, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(B->h_segmaxerr, B->d_segmaxerr, 8 * (size_t)B->nseg, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->h_flags, B->d_flags, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->h_used, B->d_used, 8, cudaMemcpyDeviceToHost, st);
  const cudaError_t e2 = cudaStreamEndCapture(st, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&B->execs[v], g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) return api_cuda_fail(e, "graph capture");
  return PC_OK;
}

// Runs the graph until the pool was large enough; returns the flags.
pc_status run_graph(pc_batch* B, unsigned int* flags) {
  for (int attempt = 0; attempt < 3; ++attempt) {
    BK(cudaGraphLaunch(B->exec, B->st));
    BK(cudaStreamSynchronize(B->st));
    *flags = *B->h_flags;
    if (!(*flags & kFlagPoolOverflow)) return PC_OK;
    const uint64_t want = *B->h_used + *B->h_used / 8 + 1024;
    cudaFree(B->pool);
    B->pool = nullptr;
    B->pool_words = 0;
    BK(cudaMalloc((void**)&B->pool, want * 8));
    B->pool_words = want;
    for (int f = 0; f < B->nfields; ++f) {
      B->h_fields[f].pool = B->pool;
      B->h_fields[f].pool_words = B->pool_words;
    }
  }
  return api_fail(PC_ERR_OOM, "scratch pool could not be sized");
}

}  // namespace

extern "C" {

pc_status pc_batch_create(int nfields, const int64_t* dims, const int* ndims, pc_dtype dtype, int n,
                          void* cuda_stream, pc_batch** out) {
  TraceRange trace_("pc_batch_create");
  if (!out) return api_fail(PC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (nfields < 1 || !dims || !ndims) return api_fail(PC_ERR_ARG, "need at least one field, dims and ndims");
  if (dtype != PC_F32 && dtype != PC_F64) return api_fail(PC_ERR_ARG, "dtype must be PC_F32 or PC_F64");
  if (n < 1 || n > PC_MAX_COMPONENTS) return api_fail(PC_ERR_ARG, "n out of range");
  for (int f = 0; f < nfields; ++f) {
    if (ndims[f] < 1 || ndims[f] > 3) return api_fail(PC_ERR_ARG, "ndims must be 1, 2 or 3");
    for (int a = 0; a < ndims[f]; ++a)
      if (dims[3 * f + a] < 1) return api_fail(PC_ERR_ARG, "extent < 1");
  }
  pc_batch* B = new pc_batch();
  B->caller = (cudaStream_t)cuda_stream;
  B->dtype = dtype;
  B->n = n;
  B->nfields = nfields;
  B->nseg = nfields * n;
  B->ndims.assign(ndims, ndims + nfields);
  B->dims.assign(dims, dims + 3 * nfields);
  B->d3.resize(3 * nfields);
  B->nb.resize(3 * nfields);
  B->nbricks.resize(nfields);
  B->nchunks.resize(nfields);
  B->cbase.resize(nfields);
  B->bbase.resize(nfields);
  for (int f = 0; f < nfields; ++f) {
    field_geometry(ndims[f], dims + 3 * f, &B->d3[3 * f], &B->nb[3 * f], &B->nbricks[f], &B->nchunks[f]);
    B->cbase[f] = B->nentries;
    B->bbase[f] = B->nbentries;
    B->nentries += (int64_t)n * B->nchunks[f];
    B->nbentries += (int64_t)n * B->nbricks[f];
  }
  cudaError_t e = cudaGetDevice(&B->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->st2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&B->ready, cudaEventDisableTiming);
  // one scratch allocation, carved in 256-byte aligned pieces
  const size_t F = nfields, S = B->nseg, E = B->nentries;
  const size_t sizes[] = {sizeof(CompressParams) * F, 2 * sizeof(BatchParams), sizeof(ScanParams), 8 * F, 8 * F,
                          8 * F, 16 * (F + 1), 4 * E, 8 * E, 20 * E, 8 * E, 8 * S, 40 * S, 8 * S, 8 * S, 8 * S, 8 * S,
                          16, 16, 16};
  size_t total = 0;
  for (size_t v : sizes) total += align256(v);
  if (e == cudaSuccess) e = cudaMalloc(&B->scratch, total);
  if (e == cudaSuccess) {
    char* p = (char*)B->scratch;
    void** slots[] = {(void**)&B->d_fields,     (void**)&B->d_bp,          (void**)&B->d_sp,
                      (void**)&B->d_slot_field, (void**)&B->d_slot_width,  (void**)&B->d_slot_ndims,
                      (void**)&B->d_slot_first,
                      (void**)&B->d_nwords,     (void**)&B->d_chunk_pool,  (void**)&B->d_counts,
                      (void**)&B->d_maxerr_c,   (void**)&B->d_totals,      (void**)&B->d_segcounts,
                      (void**)&B->d_segmaxerr,  (void**)&B->d_seg_start,   (void**)&B->d_seg_len,
                      (void**)&B->d_seg_base,   (void**)&B->d_flags,       (void**)&B->d_used,
                      (void**)&B->d_next};
    for (size_t i = 0; i < sizeof(sizes) / sizeof(sizes[0]); ++i) {
      *slots[i] = p;
      p += align256(sizes[i]);
    }
  }
  const size_t hsizes[] = {sizeof(CompressParams) * F, 2 * sizeof(BatchParams), sizeof(ScanParams), 8 * F, 8 * F,
                           8 * F, 16 * (F + 1), 8 * S, 40 * S, 8 * S, 16, 16};
  size_t htotal = 0;
  for (size_t v : hsizes) htotal += align256(v);
  if (e == cudaSuccess) e = cudaMallocHost(&B->pinned, htotal);
  if (e == cudaSuccess) {
    std::memset(B->pinned, 0, htotal);
    char* p = (char*)B->pinned;
    void** slots[] = {(void**)&B->h_fields,     (void**)&B->h_bp,         (void**)&B->h_sp,
                      (void**)&B->h_slot_field, (void**)&B->h_slot_width, (void**)&B->h_slot_ndims,
                      (void**)&B->h_slot_first,
                      (void**)&B->h_totals,     (void**)&B->h_segcounts,  (void**)&B->h_segmaxerr,
                      (void**)&B->h_flags,      (void**)&B->h_used};
    for (size_t i = 0; i < sizeof(hsizes) / sizeof(hsizes[0]); ++i) {
      *slots[i] = p;
      p += align256(hsizes[i]);
    }
  }
  // segments (field, component) over the chunk arrays, fixed by the shapes
  if (e == cudaSuccess) {
    std::vector<int64_t> ss(S), sl(S);
    for (int f = 0; f < nfields; ++f)
      for (int i = 0; i < n; ++i) {
        ss[(size_t)f * n + i] = B->cbase[f] + (int64_t)i * B->nchunks[f];
        sl[(size_t)f * n + i] = B->nchunks[f];
      }
    e = cudaMemcpy(B->d_seg_start, ss.data(), 8 * S, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_seg_len, sl.data(), 8 * S, cudaMemcpyHostToDevice);
  }
  // first pool: two bytes of stream per input byte, plus chunk padding
  if (e == cudaSuccess) {
    uint64_t vals = 0;
    for (int f = 0; f < nfields; ++f) vals += (uint64_t)(B->d3[3 * f] * B->d3[3 * f + 1] * B->d3[3 * f + 2]);
    B->pool_words = vals * dtype_size(dtype) * 2 / 8 + 2 * (uint64_t)E + 1024;
    e = cudaMalloc((void**)&B->pool, B->pool_words * 8);
  }
  if (e != cudaSuccess) {
    batch_release(B);
    return api_cuda_fail(e, "batch allocation");
  }
  // Both kernels launch a CTA per work item at most (the CTAs still claim
  // items from their counters, so every schedule's item count is covered): the
  // hardware then spreads the CTAs of both kernels over the SMs as they free
  // up, and neither kernel's tail leaves SMs idle while the other has work.
  {
    int64_t items3 = 0, items_small[4] = {0, 0, 0, 0};  // 1D/2D items: at least one chunk per warp
    for (int f = 0; f < nfields; ++f) {
      if (ndims[f] == 3)
        items3 += B->nchunks[f];
      else
        for (int w = 0; w < 4; ++w) items_small[w] += (B->nchunks[f] + kSmallShapes[w] - 1) / kSmallShapes[w];
    }
    const int64_t cap = 1 << 22;
    for (int m = 0; m < 2; ++m) {
      compress_batch_grid(dtype, m + 1);  // sets the kernel's shared-memory limit
      B->grid3[m] = (int)std::max<int64_t>(std::min(items3, cap), 1);
    }
    for (int w = 0; w < 4; ++w) {
      compress_batch_small_grid(dtype, kSmallShapes[w]);
      B->grid_small[w] = (int)std::max<int64_t>(std::min(items_small[w], cap), 1);
    }
    B->grid_mixed = compress_batch_mixed_grid(dtype);  // persistent
  }
  // parameter blocks: fixed parts (list 0: 3D fields, list 1: 1D/2D fields)
  for (int list = 0; list < 2; ++list) {
    BatchParams& bp = B->h_bp[list];
    bp.fields = B->d_fields;
    bp.slot_field = B->d_slot_field + list * nfields;
    bp.slot_width = B->d_slot_width + list * nfields;
    bp.slot_ndims = B->d_slot_ndims + list * nfields;
    bp.slot_first = B->d_slot_first + list * (nfields + 1);
    bp.nslots = 0;
    bp.next = B->d_next + list;
  }
  ScanParams& sp = *B->h_sp;
  sp.nwords = B->d_nwords;
  sp.totals = B->d_totals;
  sp.chunk_counts = B->d_counts;
  sp.counts = B->d_segcounts;
  sp.chunk_maxerr = B->d_maxerr_c;
  sp.maxerr = B->d_segmaxerr;
  sp.seg_start = B->d_seg_start;
  sp.seg_len = B->d_seg_len;
  sp.nseg = B->nseg;
  pc_status r = PC_OK;
  for (int v = 0; v < kVariants && r == PC_OK; ++v)
    if (variant_exists(v, B->dtype)) r = capture_graph(B, v);
  if (r != PC_OK) {
    batch_release(B);
    return r;
  }
  set_schedule(B, kSchedules[0]);
  *out = B;
  return PC_OK;
}

pc_status pc_batch_compress(pc_batch* B, const void* const* d_fields, const double* tau, pc_streams** out) {
  TraceRange trace_("pc_batch_compress");
  if (!B || !d_fields || !tau || !out) return api_fail(PC_ERR_ARG, "NULL argument");
  const int nf = B->nfields, n = B->n;
  for (int f = 0; f < nf; ++f) {
    out[f] = nullptr;
    if (!d_fields[f] || !device_pointer(d_fields[f])) return api_fail(PC_ERR_ARG, "fields must be device pointers");
    if (!tolerances_valid(tau + (size_t)f * n, n))
      return api_fail(PC_ERR_TAU_ORDER, "tolerances must be finite, positive, strictly decreasing");
  }
  // the fields are ready once the caller's stream reaches this point
  BK(cudaEventRecord(B->ready, B->caller));
  BK(cudaStreamWaitEvent(B->st, B->ready, 0));
  // the streams' index arrays, in one allocation shared by the batch
  auto arena = std::make_shared<BatchArena>();
  const size_t cw_bytes = align256(8 * (size_t)B->nentries), bl_bytes = align256(2 * (size_t)B->nbentries + 16);
  const size_t bo_bytes = align256(4 * (size_t)B->nbentries + 16), desc_bytes = align256(sizeof(CompDesc) * nf * n);
  const size_t err_bytes = align256(16 * (size_t)nf);
  BK(cudaMalloc(&arena->index, cw_bytes + bl_bytes + bo_bytes + desc_bytes + err_bytes));
  char* ip = (char*)arena->index;
  uint64_t* cw = (uint64_t*)ip;
  uint16_t* bl = (uint16_t*)(ip + cw_bytes);
  uint32_t* bo = (uint32_t*)(ip + cw_bytes + bl_bytes);
  CompDesc* desc = (CompDesc*)(ip + cw_bytes + bl_bytes + bo_bytes);
  unsigned int* errs = (unsigned int*)(ip + cw_bytes + bl_bytes + bo_bytes + desc_bytes);
  BK(cudaMemsetAsync(errs, 0, err_bytes, B->st));
  for (int f = 0; f < nf; ++f) {
    CompressParams& P = B->h_fields[f];
    std::memset(&P, 0, sizeof(P));
    P.field = d_fields[f];
    for (int a = 0; a < 3; ++a) {
      P.dims[a] = B->d3[3 * f + a];
      P.nb[a] = B->nb[3 * f + a];
    }
    P.nbricks = B->nbricks[f];
    P.nchunks = B->nchunks[f];
    P.n = n;
    for (int i = 0; i < n; ++i) {
      P.tau_bits[i] = tau_bits_of(tau[(size_t)f * n + i], B->dtype);
      P.L[i] = floor_log2_of(tau[(size_t)f * n + i]);
    }
    P.pool = B->pool;
    P.pool_words = B->pool_words;
    P.pool_used = B->d_used;
    P.chunk_nwords = B->d_nwords + B->cbase[f];
    P.chunk_pool = B->d_chunk_pool + B->cbase[f];
    P.brick_len = bl + B->bbase[f];
    P.brick_off = bo + B->bbase[f];
    P.chunk_counts = B->d_counts + 5 * B->cbase[f];
    P.chunk_maxerr = B->d_maxerr_c + B->cbase[f];
    P.flags = B->d_flags;
  }
  B->h_sp->word_off = cw;
  unsigned int flags = 0;
  if (B->schedule < 0) {  // autotuner: time every schedule on this batch, keep the fastest
    cudaEvent_t a, b;
    BK(cudaEventCreate(&a));
    BK(cudaEventCreate(&b));
    double best = 1e30;
    for (int c = 0; c < kNumSchedules; ++c) {
      if (!schedule_exists(kSchedules[c], B->dtype)) {
        B->tune_ms[c] = -1.0;  // not a schedule of this type
        continue;
      }
      set_schedule(B, kSchedules[c]);
      pc_status r = run_graph(B, &flags);  // also sizes the pool
      if (r != PC_OK) return r;
      BK(cudaEventRecord(a, B->st));
      BK(cudaGraphLaunch(B->exec, B->st));
      BK(cudaEventRecord(b, B->st));
      BK(cudaEventSynchronize(b));
      float ms = 0.f;
      BK(cudaEventElapsedTime(&ms, a, b));
      B->tune_ms[c] = ms;
      if (ms < best) {
        best = ms;
        B->schedule = c;
      }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  set_schedule(B, kSchedules[B->schedule]);
  pc_status r = run_graph(B, &flags);
  if (r != PC_OK) return r;
  if (flags & kFlagNonFinite) return api_fail(PC_ERR_NONFINITE, "a field holds a NaN or an infinity");
  // payloads: per segment its place in one allocation
  std::vector<uint64_t> seg_base(B->nseg);
  std::vector<uint64_t> field_words(nf, 0);
  uint64_t total = 0;
  for (int f = 0; f < nf; ++f)
    for (int i = 0; i < n; ++i) {
      seg_base[(size_t)f * n + i] = total;
      total += B->h_totals[(size_t)f * n + i];
      field_words[f] += B->h_totals[(size_t)f * n + i];
    }
  BK(cudaMalloc(&arena->payload, 8 * total + 16));
  uint64_t* payload = (uint64_t*)arena->payload;
  BK(cudaMemcpyAsync(B->d_seg_base, seg_base.data(), 8 * (size_t)B->nseg, cudaMemcpyHostToDevice, B->st));
  BK(launch_pack_segments(B->pool, B->d_nwords, B->d_chunk_pool, cw, B->d_seg_start, B->d_seg_base, B->nseg,
                          B->nentries, payload, B->st));
  // the streams objects and their descriptors
  std::vector<CompDesc> hd((size_t)nf * n);
  std::vector<pc_streams*> made(nf, nullptr);
  uint64_t fbase = 0;
  for (int f = 0; f < nf; ++f) {
    pc_streams* s = new pc_streams();
    s->device = B->device;
    s->ndims = B->ndims[f];
    s->dtype = B->dtype;
    s->n = n;
    for (int a = 0; a < 3; ++a) {
      s->dims[a] = B->d3[3 * f + a];
      s->nb[a] = B->nb[3 * f + a];
    }
    s->nbricks = B->nbricks[f];
    s->nchunks = B->nchunks[f];
    s->d_payload = payload + fbase;
    s->d_chunk_word = cw + B->cbase[f];
    s->d_brick_len = bl + B->bbase[f];
    s->d_brick_off = bo + B->bbase[f];
    s->d_desc = desc + (size_t)f * n;
    s->d_err = errs + 4 * (size_t)f;
    s->backing = arena;
    uint64_t wb = 0;
    for (int i = 0; i < n; ++i) {
      const size_t sg = (size_t)f * n + i;
      s->tau[i] = tau[sg];
      s->L[i] = floor_log2_of(tau[sg]);
      s->words[i] = B->h_totals[sg];
      s->word_base[i] = wb;
      for (int k = 0; k < 5; ++k) s->counts[i][k] = B->h_segcounts[5 * sg + k];
      s->measured[i] = value_of_bits(B->h_segmaxerr[sg], B->dtype);
      CompDesc& d = hd[sg];
      d.payload = s->d_payload + wb;
      d.nwords = s->words[i];
      d.chunk_word = s->d_chunk_word + (int64_t)i * s->nchunks;
      d.brick_len = s->d_brick_len + (int64_t)i * s->nbricks;
      d.brick_off = s->d_brick_off + (int64_t)i * s->nbricks;
      d.L = s->L[i];
      d.pad_ = 0;
      wb += s->words[i];
    }
    fbase += field_words[f];
    made[f] = s;
  }
  cudaError_t e = cudaMemcpyAsync(desc, hd.data(), sizeof(CompDesc) * hd.size(), cudaMemcpyHostToDevice, B->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(B->st);
  if (e != cudaSuccess) {
    for (pc_streams* s : made) pc_streams_free(s);
    return api_cuda_fail(e, "batch streams");
  }
  for (int f = 0; f < nf; ++f) out[f] = made[f];
  ++B->calls;
  return PC_OK;
}

pc_status pc_batch_info(const pc_batch* B, pc_batch_info_t* info) {
  if (!B || !info) return api_fail(PC_ERR_ARG, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->schedule = B->schedule;
  if (B->schedule >= 0) {
    const Schedule& sc = kSchedules[B->schedule];
    info->order = sc.order;
    info->chunks_per_item = sc.warps_small * sc.chunks_per_warp;
    info->items_per_claim = sc.per_fetch;
    info->ctas_per_sm = sc.ctas3 ? sc.ctas3 : 1;
    info->warps_small = sc.warps_small;
    info->mixed = sc.ctas3 == 0;
  }
  info->candidates = kNumSchedules;
  for (int c = 0; c < kNumSchedules && c < 16; ++c) info->candidate_ms[c] = B->tune_ms[c];
  info->grid = B->grid;
  info->calls = B->calls;
  info->graph = B->exec != nullptr;
  return PC_OK;
}

pc_status pc_batch_free(pc_batch* B) {
  batch_release(B);
  return PC_OK;
}

pc_status pc_retrieve_batch(int nq, const pc_streams* const* s, const int* k, const pc_box* boxes,
                            void* const* d_out, void* cuda_stream) {
  TraceRange trace_("pc_retrieve_batch");
  if (nq < 0 || (nq > 0 && (!s || !k || !d_out))) return api_fail(PC_ERR_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // group the queries by (type, dimensionality): one launch per group
  struct Group {
    std::vector<BoxJob> jobs;
    int64_t units = 0;
  };
  Group groups[2][4];
  unsigned int* err = nullptr;
  for (int q = 0; q < nq; ++q) {
    if (!s[q] || !d_out[q]) return api_fail(PC_ERR_ARG, "NULL streams or output");
    if (k[q] < 0 || k[q] > s[q]->n) return api_fail(PC_ERR_ARG, "k out of range");
    if (!device_pointer(d_out[q])) return api_fail(PC_ERR_ARG, "outputs must be device pointers");
    int64_t lo[3], hi[3];
    pc_status r = check_box(s[q], boxes ? &boxes[q] : nullptr, lo, hi);
    if (r != PC_OK) return r;
    if (k[q] == 0) {
      BK(cudaMemsetAsync(d_out[q], 0,
                         (size_t)((hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])) * dtype_size(s[q]->dtype), st));
      continue;
    }
    Group& G = groups[s[q]->dtype == PC_F64][s[q]->ndims];
    BoxJob J = make_box_job(s[q], 0, k[q], lo, hi, d_out[q]);
    J.unit_begin = G.units;
    G.units += s[q]->ndims == 3 ? box_job_units(J) : J.nbox;  // 1D/2D units are bricks
    G.jobs.push_back(J);
    err = s[q]->d_err;
  }
  for (int t = 0; t < 2; ++t)
    for (int d = 1; d <= 3; ++d) {
      Group& G = groups[t][d];
      if (G.jobs.empty()) continue;
      const int dt = t ? PC_F64 : PC_F32;
      void* mem = nullptr;
      const size_t jb = align256(sizeof(BoxJob) * G.jobs.size());
      const size_t spill = d == 3 ? 8 * retrieve_spill_words(dt, 3, retrieve_grid(dt, 3, G.units)) : 0;
      BK(scratch_alloc(&mem, jb + spill + 16, st));
      cudaError_t e = cudaMemcpyAsync(mem, G.jobs.data(), sizeof(BoxJob) * G.jobs.size(), cudaMemcpyHostToDevice, st);
      RetrieveParams R;
      std::memset(&R, 0, sizeof(R));
      R.jobs = (const BoxJob*)mem;
      R.njobs = (int)G.jobs.size();
      R.nunits = G.units;
      R.write = 1;
      R.err = err;
      R.spill = (uint64_t*)((char*)mem + jb);
      R.grid = retrieve_grid(dt, d, G.units);
      if (e == cudaSuccess) e = launch_retrieve(dt, d, R, st);
      cudaFreeAsync(mem, st);
      if (e != cudaSuccess) return api_cuda_fail(e, "batched retrieval");
    }
  for (int q = 0; q < nq; ++q)
    if (k[q] > 0) note_use(s[q], st);
  return PC_OK;
}

}  // extern "C"
