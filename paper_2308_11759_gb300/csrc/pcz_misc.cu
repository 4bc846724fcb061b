// pcz_misc.cu -- the memory-bound kernels around the fused coder:
//  * k_scan_chunks: per component, exclusive prefix sum of the chunks' word
//    counts (their place in the packed stream) and the component totals, plus
//    the block-mode counters and the largest error (Sec. 4.3);
//  * k_pack: copies every chunk from the scratch pool to its place in the
//    component's stream (word aligned, so a plain copy);
//  * k_range: min and max of a field (Sec. 5.1: tau_0 is the value range) and
//    a check that every value is finite.
#include <cstdint>

#include "pcz_device.cuh"
#include "pcz_kernels.h"

namespace pcz {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;

// One CTA per segment (a component's chunks); tiles of 4096 chunks with a
// block-wide scan and a running carry.  in/out/cc/me point at the segment's
// first chunk.
__device__ __forceinline__ void scan_segment(const uint32_t* __restrict__ in, uint64_t* __restrict__ out,
                                             const uint32_t* __restrict__ cc, const uint64_t* __restrict__ me,
                                             int64_t nchunks, uint64_t* total_out,
                                             unsigned long long* counts_out, unsigned long long* maxerr_out) {
  __shared__ uint64_t warp_sums[32];
  __shared__ uint64_t carry_s;
  __shared__ unsigned long long cnt_s[5];
  __shared__ unsigned long long merr_s;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) carry_s = 0;
  if (tid < 5) cnt_s[tid] = 0;
  if (tid == 0) merr_s = 0;
  unsigned long long my_cnt[5] = {0, 0, 0, 0, 0};
  unsigned long long my_merr = 0;
  __syncthreads();
  for (int64_t tile = 0; tile < nchunks; tile += (int64_t)kScanThreads * kScanItems) {
    const int64_t first = tile + (int64_t)tid * kScanItems;
    uint64_t v[kScanItems];
    uint64_t local = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
      const int64_t c = first + q;
      v[q] = c < nchunks ? in[c] : 0u;
      local += v[q];
      if (c < nchunks) {
#pragma unroll
        for (int k = 0; k < 5; ++k) my_cnt[k] += cc[c * 5 + k];
        if (me) my_merr = me[c] > my_merr ? me[c] : my_merr;
      }
    }
    uint64_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint64_t ws = warp_sums[lane];
      uint64_t wi = ws;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += y;
      }
      warp_sums[lane] = wi - ws;  // exclusive over warps
    }
    __syncthreads();
    uint64_t run = carry_s + warp_sums[warp] + (incl - local);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
      const int64_t c = first + q;
      if (c < nchunks) out[c] = run;
      run += v[q];
    }
    __syncthreads();
    if (tid == kScanThreads - 1) carry_s = run;
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) atomicAdd(&cnt_s[k], my_cnt[k]);
  atomicMax(&merr_s, my_merr);
  __syncthreads();
  if (tid == 0) *total_out = carry_s;
  if (tid < 5) counts_out[tid] = cnt_s[tid];
  if (tid == 0 && maxerr_out) *maxerr_out = merr_s;
}

// Components of one field, chunk tiles side by side: CTA (t, c) scans tile t
// (4096 chunks) of component c.  Its base -- the words of the component's
// chunks before the tile -- is a block reduction over those counts (read again,
// from L2), so the tiles need no order among them; the block counters and the
// largest error are accumulated with atomics into outputs cleared before the
// launch, and the last tile writes the component's total.
__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(const uint32_t* __restrict__ nwords,
                                                               uint64_t* __restrict__ word_off,
                                                               uint64_t* __restrict__ totals,
                                                               const uint32_t* __restrict__ chunk_counts,
                                                               unsigned long long* __restrict__ counts,
                                                               const uint64_t* __restrict__ chunk_maxerr,
                                                               unsigned long long* __restrict__ maxerr,
                                                               int64_t nchunks) {
  constexpr int64_t kTile = (int64_t)kScanThreads * kScanItems;
  __shared__ uint64_t warp_sums[32];
  const int comp = blockIdx.y, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t c0 = (int64_t)comp * nchunks, t0 = (int64_t)blockIdx.x * kTile;
  const uint32_t* in = nwords + c0;
  // the base: a block sum of the counts before the tile
  uint64_t part = 0;
  for (int64_t c = tid; c < t0; c += kScanThreads) part += in[c];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if (lane == 0) warp_sums[warp] = part;
  __syncthreads();
  uint64_t base = 0;
  if (warp == 0) {
    base = warp_sums[lane];
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) base += __shfl_xor_sync(0xffffffffu, base, o);
  }
  __syncthreads();  // warp_sums is reused below
  if (tid == 0) warp_sums[0] = base;
  __syncthreads();
  base = warp_sums[0];
  __syncthreads();
  // the tile: an exclusive block scan from the base
  const int64_t first = t0 + (int64_t)tid * kScanItems;
  uint64_t v[kScanItems], local = 0;
  unsigned my_cnt[5] = {0, 0, 0, 0, 0};
  unsigned long long my_merr = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const int64_t c = first + q;
    v[q] = c < nchunks ? in[c] : 0u;
    local += v[q];
    if (c < nchunks) {
#pragma unroll
      for (int k = 0; k < 5; ++k) my_cnt[k] += chunk_counts[(c0 + c) * 5 + k];
      if (chunk_maxerr) my_merr = chunk_maxerr[c0 + c] > my_merr ? chunk_maxerr[c0 + c] : my_merr;
    }
  }
  uint64_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint64_t ws = warp_sums[lane];
    uint64_t wi = ws;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += y;
    }
    warp_sums[lane] = wi - ws;  // exclusive over warps
  }
  __syncthreads();
  uint64_t run = base + warp_sums[warp] + (incl - local);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    const int64_t c = first + q;
    if (c < nchunks) word_off[c0 + c] = run;
    run += v[q];
  }
  // counters and the largest error of the tile, then the component's total
#pragma unroll
  for (int k = 0; k < 5; ++k) {  // a warp's share fits 32 bits: at most 128 chunks of 32 bricks
    const unsigned x = __reduce_add_sync(0xffffffffu, my_cnt[k]);
    if (lane == 0 && x) atomicAdd(&counts[5 * comp + k], (unsigned long long)x);
  }
  if (maxerr) {
    const unsigned long long m = warp_max_u64(0xffffffffu, my_merr);
    if (lane == 0 && m) atomicMax(&maxerr[comp], m);
  }
  if (blockIdx.x == gridDim.x - 1 && tid == kScanThreads - 1) totals[comp] = run;
}

// Segments of a batch of fields, described in device memory (so that a
// captured graph reads the current pointers).
__global__ void __launch_bounds__(kScanThreads) k_scan_segments(const ScanParams* __restrict__ sp) {
  const int seg = blockIdx.x;
  if (seg >= sp->nseg) return;
  const int64_t c0 = sp->seg_start[seg];
  scan_segment(sp->nwords + c0, sp->word_off + c0, sp->chunk_counts + c0 * 5, sp->chunk_maxerr + c0,
               sp->seg_len[seg], sp->totals + seg, sp->counts + 5 * seg, sp->maxerr + seg);
}

// One warp per (component, chunk): word-aligned copy from the pool.
__global__ void __launch_bounds__(256) k_pack(const uint64_t* __restrict__ pool, const uint32_t* __restrict__ nwords,
                                              const uint64_t* __restrict__ chunk_pool,
                                              const uint64_t* __restrict__ word_off,
                                              const uint64_t* __restrict__ comp_base, uint64_t* __restrict__ payload,
                                              int n, int64_t nchunks) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t wi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wi < (int64_t)n * nchunks;
       wi += warps) {
    const int comp = (int)(wi / nchunks);
    const uint32_t nw = nwords[wi];
    const uint64_t* src = pool + chunk_pool[wi];
    uint64_t* dst = payload + comp_base[comp] + word_off[wi];
    for (uint32_t w = lane; w < nw; w += 32) dst[w] = src[w];
  }
}

// One warp per (component, chunk): each brick's first bit within its chunk,
// the exclusive prefix sum of the chunk's brick lengths (a derived index the
// retrieval kernel uses; the stored index holds the lengths).
__global__ void __launch_bounds__(256) k_brick_offsets(const uint16_t* __restrict__ brick_len,
                                                       uint32_t* __restrict__ brick_off, int n, int64_t nbricks) {
  const int lane = threadIdx.x & 31;
  const int64_t nchunks = (nbricks + kChunk - 1) / kChunk;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t wi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wi < (int64_t)n * nchunks;
       wi += warps) {
    const int64_t comp = wi / nchunks, c = wi % nchunks;
    const int64_t b = c * kChunk + lane;
    const uint32_t len = b < nbricks ? brick_len[comp * nbricks + b] : 0u;
    uint32_t incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (b < nbricks) brick_off[comp * nbricks + b] = incl - len;
  }
}

cudaError_t launch_brick_offsets(const uint16_t* brick_len, uint32_t* brick_off, int n, int64_t nbricks,
                                 cudaStream_t s) {
  const int64_t items = (int64_t)n * ((nbricks + kChunk - 1) / kChunk);
  if (items == 0) return cudaSuccess;
  int64_t blocks = (items + 7) / 8;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_brick_offsets<<<(unsigned)blocks, 256, 0, s>>>(brick_len, brick_off, n, nbricks);
  return cudaGetLastError();
}

// Order-preserving map of a finite T to an unsigned integer.
template <typename T>
__device__ __forceinline__ unsigned long long order_key(T v) {
  using F = Fmt<T>;
  const typename F::U b = F::bits(v);
  const typename F::U k = (b & F::SIGN) ? (typename F::U)~b : (typename F::U)(b | F::SIGN);
  return (unsigned long long)k;
}

template <typename T>
__global__ void __launch_bounds__(256) k_range(const T* __restrict__ x, int64_t count,
                                               unsigned long long* __restrict__ enc, unsigned int* __restrict__ flags) {
  unsigned long long lo = ~0ull, hi = 0ull;
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const T v = x[i];
    if (not_finite<T>(v)) {
      bad = true;
      continue;
    }
    const unsigned long long k = order_key<T>(v);
    lo = k < lo ? k : lo;
    hi = k > hi ? k : hi;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xffffffffu, lo, o), c = __shfl_xor_sync(0xffffffffu, hi, o);
    lo = a < lo ? a : lo;
    hi = c > hi ? c : hi;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagNonFinite);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(enc, lo);
    atomicMax(enc + 1, hi);
  }
}

cudaError_t launch_scan_chunks(const uint32_t* nwords, uint64_t* word_off, uint64_t* totals,
                               const uint32_t* chunk_counts, unsigned long long* counts,
                               const uint64_t* chunk_maxerr, unsigned long long* maxerr, int n, int64_t nchunks,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(unsigned long long) * 5 * (size_t)n, s);
  if (e == cudaSuccess && nchunks <= 0) return cudaMemsetAsync(totals, 0, sizeof(uint64_t) * (size_t)n, s);
  if (e == cudaSuccess && maxerr) e = cudaMemsetAsync(maxerr, 0, sizeof(unsigned long long) * (size_t)n, s);
  if (e != cudaSuccess) return e;
  const int64_t tile = (int64_t)kScanThreads * kScanItems;
  const dim3 grid((unsigned)((nchunks + tile - 1) / tile), (unsigned)n);
  k_scan_chunks<<<grid, kScanThreads, 0, s>>>(nwords, word_off, totals, chunk_counts, counts, chunk_maxerr, maxerr,
                                              nchunks);
  return cudaGetLastError();
}

// One warp per chunk entry of a batch: its segment by binary search over the
// segments' first entries, then a word-aligned copy to the segment's place.
__global__ void __launch_bounds__(256) k_pack_segments(const uint64_t* __restrict__ pool,
                                                       const uint32_t* __restrict__ nwords,
                                                       const uint64_t* __restrict__ chunk_pool,
                                                       const uint64_t* __restrict__ word_off,
                                                       const int64_t* __restrict__ seg_start,
                                                       const uint64_t* __restrict__ seg_base, int nseg,
                                                       int64_t nentries, uint64_t* __restrict__ payload) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t wi = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wi < nentries; wi += warps) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (seg_start[mid] <= wi)
        lo = mid;
      else
        hi = mid - 1;
    }
    const uint32_t nw = nwords[wi];
    const uint64_t* src = pool + chunk_pool[wi];
    uint64_t* dst = payload + seg_base[lo] + word_off[wi];
    for (uint32_t w = lane; w < nw; w += 32) dst[w] = src[w];
  }
}

cudaError_t launch_scan_segments(const ScanParams* d_sp, int nseg, cudaStream_t s) {
  if (nseg <= 0) return cudaSuccess;
  k_scan_segments<<<nseg, kScanThreads, 0, s>>>(d_sp);
  return cudaGetLastError();
}

cudaError_t launch_pack_segments(const uint64_t* pool, const uint32_t* nwords, const uint64_t* chunk_pool,
                                 const uint64_t* word_off, const int64_t* seg_start, const uint64_t* seg_base,
                                 int nseg, int64_t nentries, uint64_t* payload, cudaStream_t s) {
  if (nentries == 0) return cudaSuccess;
  int64_t blocks = (nentries + 7) / 8;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_pack_segments<<<(unsigned)blocks, 256, 0, s>>>(pool, nwords, chunk_pool, word_off, seg_start, seg_base, nseg,
                                                   nentries, payload);
  return cudaGetLastError();
}

cudaError_t launch_pack(const uint64_t* pool, const uint32_t* nwords, const uint64_t* chunk_pool,
                        const uint64_t* word_off, const uint64_t* comp_base, uint64_t* payload, int n,
                        int64_t nchunks, cudaStream_t s) {
  const int64_t items = (int64_t)n * nchunks;
  if (items == 0) return cudaSuccess;
  int64_t blocks = (items + 7) / 8;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_pack<<<(unsigned)blocks, 256, 0, s>>>(pool, nwords, chunk_pool, word_off, comp_base, payload, n, nchunks);
  return cudaGetLastError();
}

cudaError_t launch_range(int dtype, const void* x, int64_t count, unsigned long long* enc, unsigned int* flags,
                         cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (count + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (dtype == 1)
    k_range<float><<<(unsigned)blocks, 256, 0, s>>>((const float*)x, count, enc, flags);
  else
    k_range<double><<<(unsigned)blocks, 256, 0, s>>>((const double*)x, count, enc, flags);
  return cudaGetLastError();
}

}  // namespace pcz
