// pcz_chunk3.cuh -- Algorithm 1 (Magri & Lindstrom, Sec. 4.1) on one index
// chunk of 32 bricks of a 3D field, all components, by one CTA: the body of
// the construction kernel (pcz_compress.cu) and of the batched persistent
// kernel (pcz_batch.cu).  The layout and the coding steps are described in
// pcz_compress.cu.
#pragma once

#include <climits>
#include <type_traits>

#include <cuda.h>  // CUtensorMap (the type only; the library links no driver API)

#include "pcz_device.cuh"
#include "pcz_kernels.h"

namespace pcz {

static __constant__ PermTable kPerm3 = make_perm(64);

// Largest bit string of one brick and component: CODED with every plane
// non-empty (each plane at most 2N + 1 bits) plus the header.
template <typename T>
__host__ __device__ constexpr int max_brick_bits3() {
  return 2 + 3 + Fmt<T>::EBITS + Fmt<T>::P * (2 * 64 + 1);
}

template <typename T>
__host__ __device__ constexpr int chunk_buf_words3() {  // u32 words, rounded to whole u64 words
  return ((kChunk * max_brick_bits3<T>() + 63) / 64) * 2;
}

constexpr int kCompressThreads3 = 512;

// The per-plane tables of a warp's two bricks share the warp's brick buffer,
// which is free from the end of the decode-back until the next component's
// forward transform: the plane words (8 bytes per plane) for 64-bit
// coefficients, the plane offsets and counts (4 bytes) for 32-bit ones --
// whichever has the buffer's element size.
template <typename T>
__host__ __device__ constexpr bool planes_in_brick_buffer() {
  return sizeof(typename Fmt<T>::S) == 8;
}

// Bytes of the staging area in front of the rest (TMA-staged form only).
template <typename T>
__host__ __device__ constexpr size_t staging_bytes3(bool staged) {
  return staged ? (size_t)kChunk * 64 * sizeof(T) + 16 : 0;  // the chunk's field values and a barrier
}

template <typename T>
constexpr size_t compress_smem3(bool staged = false) {
  using S = typename Fmt<T>::S;
  return staging_bytes3<T>(staged)
         + (size_t)chunk_buf_words3<T>() * 4 * 2  // chunk bit buffers (two components in flight)
         + (size_t)kChunk * 64 * sizeof(S)     // brick buffers, 128 elements per warp
         + (planes_in_brick_buffer<T>() ? 0 : (size_t)kChunk * 64 * 8)  // plane words of every brick
         + (planes_in_brick_buffer<T>() ? (size_t)kChunk * 64 * 4 : 0)  // plane offsets and counts
         + 2 * 32 * 4 * 4                      // per component parity: lengths, modes, escalations, violations
         + 16                                  // pool base of the two components in flight
         + 2 * 32 * 8                          // per component parity and brick: bits of max |x - x~_i|
         + 16;                                 // chunk bits of the two components in flight
}

// R11 group-test bits of one coefficient c that turns significant in plane
// pc (its highest set bit, at or above the lowest coded plane): when n
// coefficients are significant before pc and c >= n, c is a token of that
// plane.  With k its rank among the plane's tokens (1-based), the group part
// of the plane (which follows the n verbatim bits) holds c's 1 at c - n + k,
// the next token's test bit right after it unless c is the plane's last
// token (c + 1 == hi, hi one past the plane word's highest 1), and the
// plane's first test bit at 0 (set by the token with k = 1).  Zeros (runs and
// the closing test bit) need no write.  The two bits span at most two words.
__device__ __forceinline__ void write_token(uint32_t* buf, uint32_t cap_bits, uint32_t group_base, uint64_t W,
                                            int n, int c, int hi) {
  const uint64_t before = W & low_mask64(c) & ~low_mask64(n);
  const int k = 1 + __popcll((long long)before);
  const uint32_t pos = group_base + (uint32_t)(c - n + k);
  const bool two = c + 1 != hi;
  if (PCZ_CHECK(pos + (two ? 2u : 1u) <= cap_bits, 0)) {
    atomicOr(buf + (pos >> 5), (two ? 3u : 1u) << (pos & 31));
    if (two && (pos & 31) == 31) atomicOr(buf + (pos >> 5) + 1, 1u);
  }
  if (k == 1 && PCZ_CHECK(group_base < cap_bits, 0)) atomicOr(buf + (group_base >> 5), 1u << (group_base & 31));
}

// Suffix scans of one round of 32 planes of a warp's two bricks (lane l =
// plane base + l, coded in descending order): per brick, n before each plane
// (max of the one-past-highest set position over the planes above), the
// plane's own one-past-highest position and its bit offset.  The two bricks'
// offsets share one scan in 16-bit halves (a brick's code is below 2^14 bits).
template <int N>
__device__ __forceinline__ void plane_scan2(uint64_t WA, bool actA, uint64_t WB, bool actB, int lane, int& cmaxA,
                                            int& cmaxB, uint32_t& csum, int& nA, int& nB, int& hiA, int& hiB,
                                            int& offA, int& offB) {
  constexpr unsigned FULL = 0xffffffffu;
  hiA = (actA && WA) ? 64 - __clzll((long long)WA) : 0;
  hiB = (actB && WB) ? 64 - __clzll((long long)WB) : 0;
  int vA = hiA, vB = hiB;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int yA = __shfl_down_sync(FULL, vA, o);
    const int yB = __shfl_down_sync(FULL, vB, o);
    if (lane + o < 32) {
      vA = max(vA, yA);
      vB = max(vB, yB);
    }
  }
  int exA = __shfl_down_sync(FULL, vA, 1);
  int exB = __shfl_down_sync(FULL, vB, 1);
  if (lane == 31) exA = exB = 0;
  nA = max(exA, cmaxA);
  nB = max(exB, cmaxB);
  const uint32_t len = (uint32_t)(actA ? plane_len<N>(WA, nA) : 0) | ((uint32_t)(actB ? plane_len<N>(WB, nB) : 0) << 16);
  uint32_t sum = len;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_down_sync(FULL, sum, o);
    if (lane + o < 32) sum += y;
  }
  const uint32_t off = sum - len + csum;
  offA = (int)(off & 0xffffu);
  offB = (int)(off >> 16);
  cmaxA = max(cmaxA, __shfl_sync(FULL, vA, 0));
  cmaxB = max(cmaxB, __shfl_sync(FULL, vB, 0));
  csum += __shfl_sync(FULL, sum, 0);
}

// Byte m of a register of four packed shared-memory slots.
__device__ __forceinline__ int slot_of(uint32_t packed, int m) { return (int)((packed >> (8 * m)) & 0xffu); }

// Staging of a chunk's field values in shared memory with TMA (the
// persistent construction kernel, pcz_compress.cu): when the field's rows of
// bricks are whole chunks (bricks per row a multiple of 32), a chunk is one
// 128x4x4 box of the field, copied with one TMA tile copy ("row" layout: value
// (x, y, z) of the box at xs + 512 z + 128 y + x); otherwise one tile copy per
// brick of 4x4x4 boxes ("brick" layout: brick slot j at xs + 64 j, x
// fastest).  The copies signal an mbarrier by their bytes.  Values past the
// field's end arrive as zeros and are never used: readers clamp to the last
// in-field line and value (rule R4).
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Waits for the barrier's phase with parity `parity` to complete, at most
// `limit` polls (each poll may itself suspend the thread for a while); false
// when it gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int limit) {
  const uint32_t a = smem_addr(bar);
  for (int it = 0; it < limit; ++it) {
    uint32_t done = 0;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Issued by one thread: the copies of chunk `chunk` into xs, completing the
// barrier's current phase.
template <typename T>
__device__ __forceinline__ void issue_chunk_copy(const CompressParams& P, const CUtensorMap* map, bool row_box,
                                                 int64_t chunk, T* xs, uint64_t* bar) {
  const int64_t b0 = chunk * kChunk;
  const int nb = (int)(P.nbricks - b0 < kChunk ? P.nbricks - b0 : kChunk);
  const uint32_t bytes = (uint32_t)(row_box ? kChunk : nb) * 64u * (uint32_t)sizeof(T);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  for (int j = 0; j < (row_box ? 1 : nb); ++j) {
    const int64_t b = b0 + j;
    const int64_t cx = b % P.nb[0], r = b / P.nb[0];
    const int x = (int)(4 * cx), y = (int)(4 * (r % P.nb[1])), z = (int)(4 * (r / P.nb[1]));
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
        "%4}], [%5];" ::"r"(smem_addr(xs + 64 * j)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
  }
}

// This lane's x-line of its brick from the staged values (R4: the nearest
// in-field line and, along x, the last in-field value).
template <typename T>
__device__ __forceinline__ void staged_line(const T* xs, bool row_box, int slot, int ly, int lz, int nvx, int nvy,
                                            int nvz, T* v) {
  const int y = min(ly, nvy - 1), z = min(lz, nvz - 1);
  const T* src = row_box ? xs + 512 * z + 128 * y + 4 * slot : xs + 64 * slot + 16 * z + 4 * y;
  if (nvx == 4) {
    if constexpr (sizeof(T) == 4) {
      const float4 a = *reinterpret_cast<const float4*>(src);
      v[0] = a.x;
      v[1] = a.y;
      v[2] = a.z;
      v[3] = a.w;
    } else {
      const double2 a = reinterpret_cast<const double2*>(src)[0];
      const double2 b = reinterpret_cast<const double2*>(src)[1];
      v[0] = a.x;
      v[1] = a.y;
      v[2] = b.x;
      v[3] = b.y;
    }
    return;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) v[m] = src[min(m, nvx - 1)];
}

// Algorithm 1 on every brick of index chunk `chunk` of a 3D field, all
// components, by the whole CTA (kCompressThreads3 threads); smem holds
// compress_smem3<T>(map != nullptr) bytes, 128-byte aligned.  With a tensor
// map, xs (= smem) holds the chunk's field values staged by TMA (row layout when
// row_box, brick layout otherwise): each lane reads its line from there, and
// after a CTA barrier thread 0 starts the copy of chunk `next` (if below
// nchunks) into xs on barrier `bar`, so that it lands while this chunk is
// coded.  Without a tensor map each lane loads its line from the field with
// vector loads.  Every thread of the CTA must call it.
// Copies one component's finished chunk from its shared buffer to the pool
// (base ~0: the pool was too small) and clears the buffer for reuse.
__device__ __forceinline__ void append_chunk(const CompressParams& P, uint32_t* buf, unsigned long long base,
                                             int chunk_bits, int tid) {
  const int nw = (chunk_bits + 63) >> 6;
  uint64_t* b64 = reinterpret_cast<uint64_t*>(buf);
  for (int w = tid; w < nw; w += kCompressThreads3) {
    if (base != ~0ull) P.pool[base + w] = b64[w];
    b64[w] = 0ull;
  }
}

template <typename T>
__device__ __forceinline__ void compress3_chunk(const CompressParams& P, int64_t chunk, unsigned char* smem,
                                                const CUtensorMap* map = nullptr, bool row_box = false,
                                                uint64_t* bar = nullptr, int64_t next = -1) {
  using F = Fmt<T>;
  using U = typename F::U;
  using S = typename F::S;
  constexpr int N = 64;
  constexpr int Q = F::P - 2 - Geo<3>::G;  // quantisation bits (R6)
  constexpr int C = Geo<3>::C;             // guard planes (R10)
  constexpr int HDR = 2 + 3 + F::EBITS;    // mode, escalation, block exponent
  constexpr int LEN_RAW = 2 + N * F::P;
  constexpr int BUFW = chunk_buf_words3<T>();
  constexpr uint32_t CAP = (uint32_t)BUFW * 32;  // bits of one chunk buffer
  constexpr bool WIDE = F::P == 64;
  constexpr unsigned FULL = 0xffffffffu;

  // component i's bits go to buffer i & 1; it is appended to the pool while
  // component i + 1 is written, which saves a barrier per component
  uint32_t* cbufs = reinterpret_cast<uint32_t*>(smem + staging_bytes3<T>(map != nullptr));
  S* bbuf = reinterpret_cast<S*>(cbufs + (size_t)BUFW * 2);
  // [warp][brick][plane] plane words, and offsets | n << 14 | hi << 21; one of
  // the two lives in the brick buffer
  uint64_t* s_pw = planes_in_brick_buffer<T>() ? reinterpret_cast<uint64_t*>(bbuf)
                                               : reinterpret_cast<uint64_t*>(bbuf + kChunk * 64);
  uint32_t* s_pi = planes_in_brick_buffer<T>() ? reinterpret_cast<uint32_t*>(bbuf + kChunk * 64)
                                               : reinterpret_cast<uint32_t*>(bbuf);
  // per-brick tables, one set per component parity: a warp that runs ahead
  // into component i + 1 never overwrites what slower warps still read of i
  int* s_len = reinterpret_cast<int*>(planes_in_brick_buffer<T>() ? (void*)(s_pi + kChunk * 64)
                                                                  : (void*)(s_pw + kChunk * 64));  // [2][32]
  int* s_mode = s_len + 64;
  int* s_esc = s_mode + 64;
  int* s_viol = s_esc + 64;
  unsigned long long* s_base = reinterpret_cast<unsigned long long*>(s_viol + 64);
  uint64_t* s_merr = reinterpret_cast<uint64_t*>(s_base + 2);  // [2][32]
  int* s_cbits = reinterpret_cast<int*>(s_merr + 64);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int h = lane >> 4, t = lane & 15;
  const unsigned HALF = h ? 0xffff0000u : 0x0000ffffu;
  const int slot = warp * 2 + h;
  const int64_t b = chunk * kChunk + slot;
  const bool have = b < P.nbricks;

  for (int w = tid; w < 2 * BUFW; w += kCompressThreads3) cbufs[w] = 0u;

  int64_t bx = 0, by = 0, bz = 0;
  if (have) {
    bx = b % P.nb[0];
    const int64_t r = b / P.nb[0];
    by = r % P.nb[1];
    bz = r / P.nb[1];
  }
  const int ly = t & 3, lz = t >> 2;
  int nvx = 4, nvy = 4, nvz = 4;  // in-field extent of the brick per axis
  if (have) {
    nvx = (int)(P.dims[0] - 4 * bx < 4 ? P.dims[0] - 4 * bx : 4);
    nvy = (int)(P.dims[1] - 4 * by < 4 ? P.dims[1] - 4 * by : 4);
    nvz = (int)(P.dims[2] - 4 * bz < 4 ? P.dims[2] - 4 * bz : 4);
  }
  const bool line_in = have && ly < nvy && lz < nvz;
  // R4: a lane outside the field takes the nearest in-field line's values
  const int srcl = 16 * h + min(ly, nvy - 1) + 4 * min(lz, nvz - 1);
  const bool partial = have && (nvx < 4 || nvy < 4 || nvz < 4);
  const bool any_partial = __any_sync(FULL, partial);

  T x[4], xt[4], e[4];
  T* xs = reinterpret_cast<T*>(smem);
  if (map) {
    if (have) {
      staged_line<T>(xs, row_box, slot, ly, lz, nvx, nvy, nvz, x);
    } else {
#pragma unroll
      for (int m = 0; m < 4; ++m) x[m] = T(0);
    }
    __syncthreads();  // every lane has its values: xs is free for the next chunk
    if (tid == 0 && next >= 0 && next < P.nchunks) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the reads above before the copy's writes
      issue_chunk_copy<T>(P, map, row_box, next, xs, bar);
    }
  } else if (!have) {
#pragma unroll
    for (int m = 0; m < 4; ++m) x[m] = T(0);
  } else {
    const int64_t gy = 4 * by + min(ly, nvy - 1), gz = 4 * bz + min(lz, nvz - 1);
    const T* row = reinterpret_cast<const T*>(P.field) + (gz * P.dims[1] + gy) * P.dims[0] + 4 * bx;
    load_line<T>(row, nvx, x);
  }
  {
    bool bad = false;
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (line_in && m < nvx && not_finite<T>(x[m])) bad = true;
    if (__any_sync(FULL, bad) && lane == 0) atomicOr(P.flags, kFlagNonFinite);
  }
  // Algorithm 1 starts from x~ = 0; the first residual is x - 0, which is x
  // itself in IEEE arithmetic (-0 - +0 = -0), so no subtraction is issued
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    xt[m] = T(0);
    e[m] = x[m];
  }
  S* buf = bbuf + warp * 128;
  // buffer slots (each below 128) of this lane's line in each pass and of its
  // coded coefficients, four to a register: slot m of a pass is byte m
  const int xx = t & 3, yq = t >> 2;
  uint32_t pix = 0u, piy = 0u, piz = 0u, pir = 0u;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    pix |= (uint32_t)sidx<T>(m, ly, lz, h) << (8 * m);   // x-line of (y = ly, z = lz)
    piy |= (uint32_t)sidx<T>(xx, m, yq, h) << (8 * m);   // y-line of (x = xx, z = yq)
    piz |= (uint32_t)sidx<T>(xx, yq, m, h) << (8 * m);   // z-line of (x = xx, y = yq)
    const int pos = kPerm3.pos[t + 16 * m];
    pir |= (uint32_t)sidx<T>(pos & 3, (pos >> 2) & 3, pos >> 4, h) << (8 * m);
  }
  unsigned long long pool_base = 0;  // thread 0 only
  unsigned pool_nw = 0;

  for (int i = 0; i < P.n; ++i) {  // one component per tau_i
    uint32_t* cbuf = cbufs + (i & 1) * BUFW;
    __syncwarp();  // the last component's plane tables (in the brick buffer) are read
    const U tb = (U)P.tau_bits[i];
    if (any_partial) {  // R4 padding of the residual
      const T last = nvx == 1 ? e[0] : nvx == 2 ? e[1] : nvx == 3 ? e[2] : e[3];
#pragma unroll
      for (int m = 1; m < 4; ++m)
        if (m >= nvx) e[m] = last;
#pragma unroll
      for (int m = 0; m < 4; ++m) e[m] = __shfl_sync(FULL, e[m], srcl);
    }
    // R5: a brick whose residual meets tau_i on every in-field value is ZERO.
    // (Every lane takes part in each vote: a vote behind && or || would be
    // skipped by one half of the warp and leave the other half waiting.)
    bool small = true;
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (line_in && m < nvx && !within<T>(e[m], tb)) small = false;
    const unsigned big_votes = __ballot_sync(FULL, !small);
    const bool zero_blk = !have || ((big_votes & HALF) == 0u);
    // R6: block exponent and exact quantisation.  The largest biased exponent
    // of the brick is also its finiteness test: an infinite or NaN residual
    // (all-ones exponent) forces RAW.
    int be = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) be = max(be, biased_exp<T>(F::bits(e[m])));
    {  // the maximum over each brick's 16 lanes: two warp reductions (redux)
      const unsigned lo = __reduce_max_sync(FULL, h ? 0u : (unsigned)be);
      const unsigned hi = __reduce_max_sync(FULL, h ? (unsigned)be : 0u);
      be = (int)(h ? hi : lo);
    }
    const bool raw_forced = !zero_blk && be == (1 << F::EXPW) - 1;
    const int emax = block_emax_from_be<T>(be);
    const int s = Q - emax;
    S q[4];
    bool qdone = false;
    if constexpr (sizeof(T) == 4) {
      if (s >= -126 && s <= 127) {
        // 2^s is a normal float: e * 2^s is exact whenever |q| >= 1 (at most
        // 2^Q, no overflow; a product below the normal range truncates to 0
        // either way), so truncating the product is the R6 quantisation
        const float sc = __uint_as_float((uint32_t)(127 + s) << 23);
#pragma unroll
        for (int m = 0; m < 4; ++m) q[m] = __float2int_rz(__fmul_rn(e[m], sc));
        qdone = true;
      }
    }
    if (!qdone) {
#pragma unroll
      for (int m = 0; m < 4; ++m) q[m] = quantize<T>(F::bits(e[m]), s);
    }

    // R7: lifting along x (in the lane), y and z (shared buffer)
    lift_fwd(q[0], q[1], q[2], q[3]);
#pragma unroll
    for (int m = 0; m < 4; ++m) buf[slot_of(pix, m)] = q[m];
    __syncwarp();
    {
      S a = buf[slot_of(piy, 0)], bq = buf[slot_of(piy, 1)], c = buf[slot_of(piy, 2)], d = buf[slot_of(piy, 3)];
      lift_fwd(a, bq, c, d);
      buf[slot_of(piy, 0)] = a; buf[slot_of(piy, 1)] = bq; buf[slot_of(piy, 2)] = c; buf[slot_of(piy, 3)] = d;
    }
    __syncwarp();
    {
      S a = buf[slot_of(piz, 0)], bq = buf[slot_of(piz, 1)], c = buf[slot_of(piz, 2)], d = buf[slot_of(piz, 3)];
      lift_fwd(a, bq, c, d);
      buf[slot_of(piz, 0)] = a; buf[slot_of(piz, 1)] = bq; buf[slot_of(piz, 2)] = c; buf[slot_of(piz, 3)] = d;
    }
    __syncwarp();
    // R8, R9: coded order, negabinary.  Lane t holds coefficients t + 16j.
    U u[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) u[j] = nb_fwd<T>(buf[slot_of(pir, j)]);
    __syncwarp();

    // R10, R13: lowest coded plane; lowered until Eq. 1 holds in T
    const int L = P.L[i];
    int esc = 0, p = 0;
    bool done = zero_blk || raw_forced, pass = false;
    // x~ + x_i of the passing precision; the carried residual e takes its
    // x - (x~ + x_i) at the same time (a RAW brick recomputes the residual it
    // stores from x - x~, which is the same value)
    T xtc[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) xtc[m] = xt[m];
    for (int round = 0; round < 8; ++round) {  // esc runs 0..7: at most 8 rounds
      const bool active = !done;
      const int pp = min(max(L + s - C - esc, 0), F::P);
      const U keep = pp >= F::P ? U(0) : (U)~((U(1) << pp) - 1);
#pragma unroll
      for (int j = 0; j < 4; ++j) buf[slot_of(pir, j)] = nb_inv<T>((U)(u[j] & keep));
      __syncwarp();
      {
        S a = buf[slot_of(piz, 0)], bq = buf[slot_of(piz, 1)], c = buf[slot_of(piz, 2)], d = buf[slot_of(piz, 3)];
        lift_inv(a, bq, c, d);
        buf[slot_of(piz, 0)] = a; buf[slot_of(piz, 1)] = bq; buf[slot_of(piz, 2)] = c; buf[slot_of(piz, 3)] = d;
      }
      __syncwarp();
      {
        S a = buf[slot_of(piy, 0)], bq = buf[slot_of(piy, 1)], c = buf[slot_of(piy, 2)], d = buf[slot_of(piy, 3)];
        lift_inv(a, bq, c, d);
        buf[slot_of(piy, 0)] = a; buf[slot_of(piy, 1)] = bq; buf[slot_of(piy, 2)] = c; buf[slot_of(piy, 3)] = d;
      }
      __syncwarp();
      S r[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) r[m] = buf[slot_of(pix, m)];
      __syncwarp();
      lift_inv(r[0], r[1], r[2], r[3]);
      bool ok = true;
      T xtn[4], en[4];
      if constexpr (sizeof(T) == 4) {
        T xi[4];
        dequantize_line<T, false>(r, s, xi);  // x_i = D(y_i)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          xtn[m] = F::add(xt[m], xi[m]);  // x~ + x_i (candidate)
          en[m] = F::sub(x[m], xtn[m]);   // the next residual
          if (line_in && m < nvx && !within<T>(en[m], tb)) ok = false;
        }
      } else {
        const bool normal = s >= -960 && s <= 1022;  // every result normal and finite
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const T xi = normal ? Fmt<T>::val(dequantize_f64_normal(r[m], s)) : dequantize_val<T>(r[m], s);  // x_i = D(y_i)
          // x~ + x_i (candidate); for the first component +0 + x_i, which is
          // x_i with -0 turned to +0 -- a bit test instead of an FP64 add
          const U xb = F::bits(xi);
          xtn[m] = i == 0 ? F::val(xb == F::SIGN ? U(0) : xb) : F::add(xt[m], xi);
          en[m] = F::sub(x[m], xtn[m]);             // the next residual
          if (line_in && m < nvx && !within<T>(en[m], tb)) ok = false;
        }
      }
      const bool pass_h = (__ballot_sync(FULL, !ok) & HALF) == 0u;
      if (active) {
        if (pass_h) {
          pass = true;
          done = true;
          p = pp;
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            xtc[m] = xtn[m];
            if constexpr (sizeof(T) == 8) e[m] = en[m];  // float32 recomputes it below
          }
        } else if (esc == 7 || pp == 0) {
          done = true;
        } else {
          ++esc;
        }
      }
      if (__all_sync(FULL, done)) break;
    }

    // R11: plane words by transposing the coefficient bits across the warp:
    // lane l then holds plane l (and l + 32) of both bricks.
    uint64_t WA0, WB0, WA1 = 0, WB1 = 0;
    {
      uint32_t tkeep[5];
      transpose_masks(lane, tkeep);
      uint32_t tl[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) tl[j] = transpose32((uint32_t)u[j], lane, tkeep);
      WA0 = (uint64_t)__byte_perm(tl[0], tl[1], 0x5410) | ((uint64_t)__byte_perm(tl[2], tl[3], 0x5410) << 32);
      WB0 = (uint64_t)__byte_perm(tl[0], tl[1], 0x7632) | ((uint64_t)__byte_perm(tl[2], tl[3], 0x7632) << 32);
      if constexpr (WIDE) {
        uint32_t th[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) th[j] = transpose32((uint32_t)((uint64_t)u[j] >> 32), lane, tkeep);
        WA1 = (uint64_t)__byte_perm(th[0], th[1], 0x5410) | ((uint64_t)__byte_perm(th[2], th[3], 0x5410) << 32);
        WB1 = (uint64_t)__byte_perm(th[0], th[1], 0x7632) | ((uint64_t)__byte_perm(th[2], th[3], 0x7632) << 32);
      }
    }
    const int pA = __shfl_sync(FULL, p, 0), pB = __shfl_sync(FULL, p, 16);
    const bool passA = __shfl_sync(FULL, (int)pass, 0) != 0, passB = __shfl_sync(FULL, (int)pass, 16) != 0;
    // planes P-1 .. p are coded, from the top: the high round (planes 32 + l)
    // first for 64-bit coefficients, then planes l
    int nA0 = 0, nA1 = 0, nB0 = 0, nB1 = 0, oA0 = 0, oA1 = 0, oB0 = 0, oB1 = 0;
    int hA0 = 0, hA1 = 0, hB0 = 0, hB1 = 0;
    int totA = 0, totB = 0;
    {
      int cmaxA = 0, cmaxB = 0;
      uint32_t csum = 0;
      if constexpr (WIDE)
        plane_scan2<N>(WA1, passA && lane + 32 >= pA, WB1, passB && lane + 32 >= pB, lane, cmaxA, cmaxB, csum, nA1, nB1,
                       hA1, hB1, oA1, oB1);
      plane_scan2<N>(WA0, passA && lane >= pA, WB0, passB && lane >= pB, lane, cmaxA, cmaxB, csum, nA0, nB0, hA0, hB0,
                     oA0, oB0);
      totA = (int)(csum & 0xffffu);
      totB = (int)(csum >> 16);
    }
    const int lenC = HDR + (h ? totB : totA);
    {  // plane p's word, code offset and significance count, for the coefficient lanes
      uint64_t* pw = s_pw + warp * 128;
      uint32_t* pi = s_pi + warp * 128;
      pw[lane] = WA0;
      pi[lane] = (uint32_t)oA0 | ((uint32_t)nA0 << 14) | ((uint32_t)hA0 << 21);
      pw[64 + lane] = WB0;
      pi[64 + lane] = (uint32_t)oB0 | ((uint32_t)nB0 << 14) | ((uint32_t)hB0 << 21);
      if constexpr (WIDE) {
        pw[32 + lane] = WA1;
        pi[32 + lane] = (uint32_t)oA1 | ((uint32_t)nA1 << 14) | ((uint32_t)hA1 << 21);
        pw[96 + lane] = WB1;
        pi[96 + lane] = (uint32_t)oB1 | ((uint32_t)nB1 << 14) | ((uint32_t)hB1 << 21);
      }
    }

    // the residual x - x~_{i-1} again, padded (R4), where a brick may be RAW:
    // the value the coder started from, which the loop above has replaced
    // by the next residual in passing bricks
    T eo[4];
    const bool need_eo = __any_sync(FULL, !zero_blk && (!pass || lenC > LEN_RAW));
    if (need_eo) {
#pragma unroll
      for (int m = 0; m < 4; ++m) eo[m] = F::sub(x[m], xt[m]);
      if (any_partial) {
        const T last = nvx == 1 ? eo[0] : nvx == 2 ? eo[1] : nvx == 3 ? eo[2] : eo[3];
#pragma unroll
        for (int m = 1; m < 4; ++m)
          if (m >= nvx) eo[m] = last;
#pragma unroll
        for (int m = 0; m < 4; ++m) eo[m] = __shfl_sync(FULL, eo[m], srcl);
      }
    }
    // R14: RAW replaces a longer CODED brick only if it also meets tau_i
    bool raw_ok = false;
    if (__any_sync(FULL, pass && lenC > LEN_RAW)) {
      bool ok = true;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const T a = F::add(xt[m], eo[m]);
        if (line_in && m < nvx && !within<T>(F::sub(x[m], a), tb)) ok = false;
      }
      raw_ok = (__ballot_sync(FULL, !ok) & HALF) == 0u;
    }
    const int mode = zero_blk ? kModeZero : (pass && !(lenC > LEN_RAW && raw_ok)) ? kModeCoded : kModeRaw;
    const int blen = !have ? 0 : mode == kModeZero ? 2 : mode == kModeRaw ? LEN_RAW : lenC;

    // x~_i and the next residual (a RAW brick stores the residual it started
    // from); the next residual is in e already for CODED and ZERO bricks
    int viol = 0;  // Eq. 1 failures left (only a RAW brick can have them)
    U merr = 0;    // max |x - x~_i| over this lane's in-field values, as bits (Sec. 4.3)
    if (need_eo) {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if (mode == kModeRaw) {
          xtc[m] = F::add(xt[m], eo[m]);
          if constexpr (sizeof(T) == 8) e[m] = F::sub(x[m], xtc[m]);
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      // float32: the next residual x - x~_i for every mode, recomputed here so
      // that it is not live across the escalation loop (fewer spills; the
      // same values: a passing brick's candidate residual was x - x~_i, and
      // lanes outside the field are padded again at the next component).
      // Float64 keeps the loop's value: a second FP64 subtraction costs more
      // than the spills it saves.
#pragma unroll
      for (int m = 0; m < 4; ++m) e[m] = F::sub(x[m], xtc[m]);
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      if (line_in && m < nvx) {
        U a;  // float64: |e|'s pattern doubled (mag2_bits), halved after the maximum
        if constexpr (sizeof(U) == 8)
          a = mag2_bits(e[m]);
        else
          a = F::bits(e[m]) & F::ABS;
        merr = a > merr ? a : merr;
      }
    }
    if constexpr (sizeof(U) == 4) {  // per brick half: two warp reductions (redux)
      const unsigned lo = __reduce_max_sync(FULL, h ? 0u : (unsigned)merr);
      const unsigned hi = __reduce_max_sync(FULL, h ? (unsigned)merr : 0u);
      merr = (U)(h ? hi : lo);
    } else {  // per brick half: the two halves' 64-bit maxima, four warp reductions
      const unsigned long long lo = warp_max_u64(FULL, h ? 0ull : (unsigned long long)merr);
      const unsigned long long hi = warp_max_u64(FULL, h ? (unsigned long long)merr : 0ull);
      merr = (U)(h ? hi : lo) >> 1;
    }
    // failures are counted only where a brick of the warp is RAW (a CODED or
    // ZERO brick meets tau_i on every value by construction)
    if (__any_sync(FULL, have && mode == kModeRaw)) {
#pragma unroll
      for (int m = 0; m < 4; ++m)
        if (line_in && m < nvx && !within<T>(e[m], tb)) ++viol;
#pragma unroll
      for (int o = 8; o >= 1; o >>= 1) viol += __shfl_xor_sync(FULL, viol, o);
    }

    const int par = (i & 1) * 32;
    if (t == 0) {
      s_len[par + slot] = blen;
      s_mode[par + slot] = have ? mode : -1;
      s_esc[par + slot] = (have && mode == kModeCoded) ? esc : 0;
      s_viol[par + slot] = have ? viol : 0;
      s_merr[par + slot] = have ? (uint64_t)merr : 0ull;
    }
    __syncthreads();
    // chunk layout: every warp scans the 32 brick lengths for its own bricks'
    // offsets (no second barrier); warp 0 also records the chunk
    // this warp's two bricks start after the lengths of the bricks before them:
    // one warp sum (redux) over the lanes below 2 * warp
    const int l0 = s_len[par + lane];
    const int offA = (int)__reduce_add_sync(FULL, lane < 2 * warp ? (unsigned)l0 : 0u);
    const int offB = offA + __shfl_sync(FULL, l0, 2 * warp);
    // chunk bookkeeping, spread so that no warp carries much more than the
    // others to the next barrier: warp 0 sizes the chunk and reserves its
    // pool space, warp 1 gathers the block counters, and each warp writes its
    // own bricks' index entries
    if (warp == 0) {
      const int total = (int)__reduce_add_sync(FULL, (unsigned)l0);
      const unsigned nw = (unsigned)((total + 63) >> 6);
      if (lane == 0) {
        s_cbits[i & 1] = total;
        // pool space for the chunk; the atomic's result is first needed after
        // this warp's share of the bit writes, which hides its latency
        pool_base = nw ? atomicAdd(P.pool_used, (unsigned long long)nw) : 0ull;
        pool_nw = nw;
        P.chunk_nwords[(int64_t)i * P.nchunks + chunk] = nw;
      }
    } else if (warp == 1) {
      const int md = s_mode[par + lane];
      const unsigned cz = __popc(__ballot_sync(FULL, md == kModeZero));
      const unsigned cc = __popc(__ballot_sync(FULL, md == kModeCoded));
      const unsigned cr = __popc(__ballot_sync(FULL, md == kModeRaw));
      int se = s_esc[par + lane], sv = s_viol[par + lane];
      const unsigned long long me = warp_max_u64(FULL, s_merr[par + lane]);
      if (__any_sync(FULL, se != 0 || sv != 0)) {  // escalations and failures are rare
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
          se += __shfl_xor_sync(FULL, se, o);
          sv += __shfl_xor_sync(FULL, sv, o);
        }
      }
      if (lane == 0) {
        const int64_t ci = (int64_t)i * P.nchunks + chunk;
        uint32_t* cnt = P.chunk_counts + ci * 5;
        cnt[0] = cz;
        cnt[1] = cc;
        cnt[2] = cr;
        cnt[3] = (uint32_t)se;
        cnt[4] = (uint32_t)sv;
        if (P.chunk_maxerr) P.chunk_maxerr[ci] = me;
      }
    }
    if (t == 0 && have) {
      P.brick_len[(int64_t)i * P.nbricks + b] = (uint16_t)blen;
      if (P.brick_off) P.brick_off[(int64_t)i * P.nbricks + b] = (uint32_t)(h ? offB : offA);
    }

    // this component's bits of the warp's two bricks, into the chunk buffer
    const uint32_t boff = (uint32_t)(h ? offB : offA);
    if (have && mode == kModeRaw) {
      if (t == 0) or_bits_in(cbuf, boff, (uint64_t)kModeRaw, CAP, 0);
#pragma unroll
      for (int m = 0; m < 4; ++m) or_bits_in(cbuf, boff + 2 + F::P * (4 * t + m), (uint64_t)F::bits(eo[m]), CAP, 0);
    } else if (have && mode == kModeCoded && t == 0) {
      or_bits_in(cbuf, boff, (uint64_t)kModeCoded | ((uint64_t)esc << 2) | ((uint64_t)(emax + F::EBIAS) << 5), CAP,
                 0);
    }
    const int modeA = __shfl_sync(FULL, mode, 0), modeB = __shfl_sync(FULL, mode, 16);
    const bool haveA = __shfl_sync(FULL, (int)have, 0) != 0, haveB = __shfl_sync(FULL, (int)have, 16) != 0;
    // R11: each coded plane's verbatim bits, by the plane's owner lane ...
    if (haveA && modeA == kModeCoded) {
      const uint32_t base = (uint32_t)offA + HDR;
      if (lane >= pA && nA0 > 0) or_bits_in(cbuf, base + oA0, WA0 & low_mask64(nA0), CAP, 0);
      if (WIDE && lane + 32 >= pA && nA1 > 0) or_bits_in(cbuf, base + oA1, WA1 & low_mask64(nA1), CAP, 0);
    }
    if (haveB && modeB == kModeCoded) {
      const uint32_t base = (uint32_t)offB + HDR;
      if (lane >= pB && nB0 > 0) or_bits_in(cbuf, base + oB0, WB0 & low_mask64(nB0), CAP, 0);
      if (WIDE && lane + 32 >= pB && nB1 > 0) or_bits_in(cbuf, base + oB1, WB1 & low_mask64(nB1), CAP, 0);
    }
    // ... and its group-test bits, one token per newly significant coefficient,
    // by the lane that holds the coefficient
    if (have && mode == kModeCoded && p < F::P) {
      const uint64_t* pw = s_pw + warp * 128 + 64 * h;
      const uint32_t* pi = s_pi + warp * 128 + 64 * h;
      const uint32_t base = boff + HDR;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if ((u[j] >> p) == 0) continue;  // no bit at or above the lowest coded plane
        const int pc = F::P - 1 - F::clz(u[j]);
        if (!PCZ_CHECK(pc >= 0 && pc < 64, 1)) continue;
        const uint32_t info = pi[pc];
        const int n = (int)((info >> 14) & 127u), c = t + 16 * j;
        if (c >= n) write_token(cbuf, CAP, base + (info & 0x3fffu) + (uint32_t)n, pw[pc], n, c, (int)(info >> 21));
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) xt[m] = xtc[m];
    if (tid == 0) {
      unsigned long long base = pool_base;
      if (base + pool_nw > P.pool_words) {
        atomicOr(P.flags, kFlagPoolOverflow);
        base = ~0ull;
      }
      s_base[i & 1] = base;
      P.chunk_pool[(int64_t)i * P.nchunks + chunk] = base;
    }
    if (i > 0) append_chunk(P, cbufs + ((i - 1) & 1) * BUFW, s_base[(i - 1) & 1], s_cbits[(i - 1) & 1], tid);
  }
  __syncthreads();
  append_chunk(P, cbufs + ((P.n - 1) & 1) * BUFW, s_base[(P.n - 1) & 1], s_cbits[(P.n - 1) & 1], tid);
}

}  // namespace pcz
