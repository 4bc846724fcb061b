// pcz_chunk_small.cuh -- Algorithms 1 and 2 (Magri & Lindstrom, Sec. 4.1,
// 4.2) for 1D and 2D fields, whose bricks hold 4 and 16 values: one warp
// codes an index chunk of 32 bricks (a brick per lane, entirely in
// registers), one thread retrieves a brick.  Shared by the stand-alone
// kernels (pcz_small.cu) and the batched persistent kernel (pcz_batch.cu).
#pragma once

#include <type_traits>

#include "pcz_device.cuh"
#include "pcz_kernels.h"

namespace pcz {

constexpr int kSmallWarps = 4;  // chunks per CTA
constexpr int kSmallThreads = 32 * kSmallWarps;

// Largest coded block: the header, at most one verbatim or run bit per
// coefficient and plane, and at most one test bit per coefficient plus one
// closing test bit per plane (R11); RAW is shorter still.
template <typename T, int D>
__host__ __device__ constexpr int max_brick_bits_small() {
  return 2 + 3 + Fmt<T>::EBITS + Geo<D>::N * Fmt<T>::P + Geo<D>::N + Fmt<T>::P;
}

template <typename T, int D>
__host__ __device__ constexpr int chunk_words_small() {  // u32 words of one chunk buffer
  return ((kChunk * max_brick_bits_small<T, D>() + 63) / 64) * 2;
}

template <typename T, int D>
constexpr size_t small_smem() {
  return (size_t)kSmallWarps * chunk_words_small<T, D>() * 4;
}

// R8: brick position (x + 4y) of the r-th coded coefficient.  The table is a
// compile-time constant, so with r known after unrolling the lookup folds
// away and the coefficient arrays stay in registers.
template <int D>
__device__ __forceinline__ int perm_small(int r) {
  if constexpr (D == 1) {
    return r;
  } else {
    constexpr PermTable t = make_perm(16);
    return t.pos[r];
  }
}

// lifting of the brick in registers: along x, then y (D = 2)
template <int D, typename S>
__device__ __forceinline__ void lift_fwd_brick(S* v) {
  constexpr int NY = D == 2 ? 4 : 1;
#pragma unroll
  for (int y = 0; y < NY; ++y) lift_fwd(v[4 * y], v[4 * y + 1], v[4 * y + 2], v[4 * y + 3]);
  if constexpr (D == 2) {
#pragma unroll
    for (int x = 0; x < 4; ++x) lift_fwd(v[x], v[x + 4], v[x + 8], v[x + 12]);
  }
}

template <int D, typename S>
__device__ __forceinline__ void lift_inv_brick(S* v) {
  constexpr int NY = D == 2 ? 4 : 1;
  if constexpr (D == 2) {
#pragma unroll
    for (int x = 0; x < 4; ++x) lift_inv(v[x], v[x + 4], v[x + 8], v[x + 12]);
  }
#pragma unroll
  for (int y = 0; y < NY; ++y) lift_inv(v[4 * y], v[4 * y + 1], v[4 * y + 2], v[4 * y + 3]);
}

// Appends one block's bits to a thread's view of the chunk buffer: bit
// position pos is advanced; zero bits need no write.
struct SmallWriter {
  uint32_t* buf;
  uint32_t pos;
  uint32_t cap;  // bits of the buffer
  __device__ __forceinline__ void put(uint64_t v, int nbits) {  // nbits <= 64
    if (v) or_bits_in(buf, pos, v & low_mask64(nbits), cap, 2);
    pos += (uint32_t)nbits;
  }
};

// R11 for one brick in one thread: plane words are gathered from the
// coefficients (bit r of plane pl = bit pl of coefficient r); with the
// significance count n, each plane emits n verbatim bits and then its tokens.
// Planes above the highest set bit are one 0 test bit each.
template <int N, typename U>
__device__ __forceinline__ int first_empty_plane(const U* u, int p) {
  U any = 0;
#pragma unroll
  for (int r = 0; r < N; ++r) any |= u[r];
  const int top = any ? (int)(8 * sizeof(U)) - 1 - (sizeof(U) == 8 ? __clzll((long long)any) : __clz((int)any)) : -1;
  return max(top + 1, p);  // planes from here up to P-1 are empty
}

template <int N, typename U>
__device__ __forceinline__ uint32_t plane_word(const U* u, int pl) {
  uint32_t W = 0;
#pragma unroll
  for (int r = 0; r < N; ++r) W |= (uint32_t)((u[r] >> pl) & 1u) << r;
  return W;
}

// Bit length of the planes P-1 .. p, one plane at a time in closed form
// (plane_len), without walking the tokens.
template <int N, typename U>
__device__ __forceinline__ int planes_len(const U* u, int P, int p) {
  const int first = first_empty_plane<N>(u, p);
  int len = P - first, n = 0;
  for (int pl = first - 1; pl >= p; --pl) {
    const uint64_t W = plane_word<N>(u, pl);
    len += plane_len<N>(W, n);
    if (n < N && (W >> n)) n = 64 - __clzll((long long)W);
  }
  return len;
}

// Writes the planes P-1 .. p of one brick at w.pos.
template <int N, typename U>
__device__ __forceinline__ void emit_planes(const U* u, int P, int p, SmallWriter& w) {
  const int first = first_empty_plane<N>(u, p);
  w.pos += (uint32_t)(P - first);  // empty planes: 0 test bits, nothing to write
  int n = 0;
  for (int pl = first - 1; pl >= p; --pl) {
    const uint32_t W = plane_word<N>(u, pl);
    if (n > 0) w.put(W, n);
    if (n >= N) continue;
    uint32_t rest = W >> n;
    for (int it = 0; it < N && n < N; ++it) {
      if (!rest) {  // test 0
        w.pos += 1;
        break;
      }
      const int tz = __ffs((int)rest) - 1;
      w.put(1, 1);                // test 1
      w.put(1ull << tz, tz + 1);  // run up to and including the 1
      n += tz + 1;
      rest >>= (tz + 1);
    }
  }
}

// Algorithm 1 on index chunk `chunk` of a 1D or 2D field, all components, by
// one warp: lane l codes brick 32 * chunk + l.  cbuf is the warp's own
// shared buffer of chunk_words_small<T, D>() words.  Every lane of the warp
// must call it; a chunk at or past the field's last does nothing but take
// part in the warp's collective operations.
template <typename T, int D>
__device__ __forceinline__ void compress_small_chunk(const CompressParams& P, int64_t chunk, uint32_t* cbuf) {
  using F = Fmt<T>;
  using U = typename F::U;
  using S = typename F::S;
  constexpr int N = Geo<D>::N;
  constexpr int Q = F::P - 2 - Geo<D>::G;
  constexpr int C = Geo<D>::C;
  constexpr int HDR = 2 + 3 + F::EBITS;
  constexpr int LEN_RAW = 2 + N * F::P;
  constexpr int BUFW = chunk_words_small<T, D>();
  constexpr unsigned FULL = 0xffffffffu;

  const int lane = threadIdx.x & 31;
  const int64_t b = chunk * kChunk + lane;
  const bool have = chunk < P.nchunks && b < P.nbricks;
  for (int i = lane; i < BUFW; i += 32) cbuf[i] = 0u;
  __syncwarp();

  // gather with edge replication (R4); inf = in-field lanes
  int64_t bx = 0, by = 0;
  if (have) {
    bx = b % P.nb[0];
    by = b / P.nb[0];
  }
  const int nvx = have ? (int)(P.dims[0] - 4 * bx < 4 ? P.dims[0] - 4 * bx : 4) : 4;
  const int nvy = (D == 2 && have) ? (int)(P.dims[1] - 4 * by < 4 ? P.dims[1] - 4 * by : 4) : (D == 2 ? 4 : 1);
  T x[N], xt[N];
  bool bad = false;
  {
    const T* field = reinterpret_cast<const T*>(P.field);
#pragma unroll
    for (int j = 0; j < N / 4; ++j) {  // one x-line per row, rows past the field repeat the last (R4)
      if (have)
        load_line<T>(field + (4 * by + min(j, nvy - 1)) * P.dims[0] + 4 * bx, nvx, &x[4 * j]);
      else
#pragma unroll
        for (int i = 0; i < 4; ++i) x[4 * j + i] = T(0);
    }
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (have && (k & 3) < nvx && (k >> 2) < nvy && not_finite<T>(x[k])) bad = true;
      xt[k] = T(0);  // Algorithm 1 starts from x~ = 0
    }
  }
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(P.flags, kFlagNonFinite);

  for (int i = 0; i < P.n; ++i) {  // one component per tolerance
    const U tb = (U)P.tau_bits[i];
    // residual e = x - x~ on the in-field lanes; padded lanes copy the nearest
    // in-field lane along x, then along y (R4), by compile-time indices only
    T e[N];
#pragma unroll
    for (int k = 0; k < N; ++k) e[k] = F::sub(x[k], xt[k]);
#pragma unroll
    for (int j = 0; j < N / 4; ++j)
#pragma unroll
      for (int ii = 1; ii < 4; ++ii)
        if (ii >= nvx) e[ii + 4 * j] = e[ii - 1 + 4 * j];
    if constexpr (D == 2) {
#pragma unroll
      for (int j = 1; j < 4; ++j)
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
          if (j >= nvy) e[ii + 4 * j] = e[ii + 4 * (j - 1)];
    }
    bool small = true;
    int be = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if ((k & 3) < nvx && (k >> 2) < nvy && !within<T>(e[k], tb)) small = false;
      be = max(be, biased_exp<T>(F::bits(e[k])));
    }
    const bool nf = be == (1 << F::EXPW) - 1;  // an infinite or NaN residual: all-ones exponent
    const bool zero_blk = !have || small;  // R5
    int mode = kModeZero, esc = 0, p = 0, len = 2;
    const int emax = block_emax_from_be<T>(be);
    const int s = Q - emax;
    U u[N];
    T xtn[N];
    if (!zero_blk) {
      bool pass = false;
      if (!nf) {
        S q[N];
#pragma unroll
        for (int k = 0; k < N; ++k) q[k] = quantize<T>(F::bits(e[k]), s);  // R6
        lift_fwd_brick<D>(q);                                                // R7
#pragma unroll
        for (int r = 0; r < N; ++r) u[r] = nb_fwd<T>(q[perm_small<D>(r)]);  // R8, R9
        for (esc = 0;; ++esc) {  // R10, R13
          p = min(max(P.L[i] + s - C - esc, 0), F::P);
          const U keep = p >= F::P ? U(0) : (U)~((U(1) << p) - 1);
          S r[N];
#pragma unroll
          for (int rr = 0; rr < N; ++rr) r[perm_small<D>(rr)] = nb_inv<T>((U)(u[rr] & keep));
          lift_inv_brick<D>(r);
          bool ok = true;
#pragma unroll
          for (int k = 0; k < N; ++k) {
            xtn[k] = F::add(xt[k], dequantize_val<T>(r[k], s));  // x~ + D(C(e))
            if ((k & 3) < nvx && (k >> 2) < nvy && !within<T>(F::sub(x[k], xtn[k]), tb)) ok = false;
          }
          if (ok) {
            pass = true;
            break;
          }
          if (esc == 7 || p == 0) break;
        }
      }
      if (pass) {
        const int lenC = HDR + planes_len<N>(u, F::P, p);
        bool use_raw = false;
        if (lenC > LEN_RAW) {  // R14
          use_raw = true;
#pragma unroll
          for (int k = 0; k < N; ++k)
            if ((k & 3) < nvx && (k >> 2) < nvy && !within<T>(F::sub(x[k], F::add(xt[k], e[k])), tb))
              use_raw = false;
        }
        mode = use_raw ? kModeRaw : kModeCoded;
        len = use_raw ? LEN_RAW : lenC;
      } else {
        mode = kModeRaw;
        len = LEN_RAW;
      }
    }
    if (!have) len = 0;
    // chunk layout: this brick's offset, pool space, index entries
    int incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(FULL, incl, o);
      if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    const unsigned nw = (unsigned)((total + 63) >> 6);
    unsigned long long base = 0;
    if (lane == 0 && chunk < P.nchunks) base = nw ? atomicAdd(P.pool_used, (unsigned long long)nw) : 0ull;
    // write the block
    SmallWriter w{cbuf, (uint32_t)(incl - len), (uint32_t)BUFW * 32};
    if (have && mode == kModeCoded) {
      w.put((uint64_t)kModeCoded | ((uint64_t)esc << 2) | ((uint64_t)(emax + F::EBIAS) << 5), HDR);
      emit_planes<N>(u, F::P, p, w);
    } else if (have && mode == kModeRaw) {
      w.put(kModeRaw, 2);
#pragma unroll
      for (int k = 0; k < N; ++k) w.put((uint64_t)F::bits(e[k]), F::P);
    }
    // x~ += x_i; count Eq. 1 failures left (RAW only) and the largest error
    // (Sec. 4.3: the computed tolerance)
    int viol = 0;
    unsigned long long merr = 0;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      if (mode == kModeCoded) xt[k] = xtn[k];
      if (mode == kModeRaw) xt[k] = F::add(xt[k], e[k]);
      if (have && (k & 3) < nvx && (k >> 2) < nvy) {
        const T r = F::sub(x[k], xt[k]);
        if (!within<T>(r, tb)) ++viol;
        unsigned long long a;  // float64: |r|'s pattern doubled (mag2_bits), halved after the maximum
        if constexpr (sizeof(T) == 8)
          a = mag2_bits(r);
        else
          a = (unsigned long long)(F::bits(r) & F::ABS);
        merr = a > merr ? a : merr;
      }
    }
    const unsigned cz = __popc(__ballot_sync(FULL, have && mode == kModeZero));
    const unsigned cc = __popc(__ballot_sync(FULL, have && mode == kModeCoded));
    const unsigned cr = __popc(__ballot_sync(FULL, have && mode == kModeRaw));
    int se = (have && mode == kModeCoded) ? esc : 0;
    if constexpr (sizeof(T) == 4)  // 32-bit patterns: one warp reduction (redux)
      merr = __reduce_max_sync(FULL, (unsigned)merr);
    else
      merr = warp_max_u64(FULL, merr) >> 1;
    // escalations and Eq. 1 failures (RAW bricks only) are rare: summed only
    // where a lane has some
    if (__any_sync(FULL, se != 0 || viol != 0)) {
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        se += __shfl_xor_sync(FULL, se, o);
        viol += __shfl_xor_sync(FULL, viol, o);
      }
    }
    if (have) {
      P.brick_len[(int64_t)i * P.nbricks + b] = (uint16_t)len;
      if (P.brick_off) P.brick_off[(int64_t)i * P.nbricks + b] = (uint32_t)(incl - len);
    }
    __syncwarp();
    base = __shfl_sync(FULL, base, 0);
    if (chunk < P.nchunks) {
      if (lane == 0) {
        if (base + nw > P.pool_words) {
          atomicOr(P.flags, kFlagPoolOverflow);
          base = ~0ull;
        }
        const int64_t ci = (int64_t)i * P.nchunks + chunk;
        P.chunk_nwords[ci] = nw;
        P.chunk_pool[ci] = base;
        uint32_t* cnt = P.chunk_counts + ci * 5;
        cnt[0] = cz;
        cnt[1] = cc;
        cnt[2] = cr;
        cnt[3] = (uint32_t)se;
        cnt[4] = (uint32_t)viol;
        if (P.chunk_maxerr) P.chunk_maxerr[ci] = merr;
      }
      base = __shfl_sync(FULL, base, 0);
      uint64_t* b64 = reinterpret_cast<uint64_t*>(cbuf);
      for (unsigned wd = lane; wd < nw; wd += 32) {
        if (base != ~0ull) P.pool[base + wd] = b64[wd];
        b64[wd] = 0ull;
      }
    }
    __syncwarp();
  }
}

// Retrieval of brick g (box order) of job J by one thread: components
// k0+1..k parsed and rebuilt in ascending order and summed into x~
// (Algorithm 2).  No warp-collective operations.
template <typename T, int D>
__device__ __forceinline__ void retrieve_small_brick(const BoxJob& J, int write, unsigned int* err, int64_t g) {
  using F = Fmt<T>;
  using U = typename F::U;
  using S = typename F::S;
  constexpr int N = Geo<D>::N;
  constexpr int Q = F::P - 2 - Geo<D>::G;
  constexpr int C = Geo<D>::C;
  constexpr int HDR = 2 + 3 + F::EBITS;
  constexpr int EMAXT = (1 << (F::EXPW - 1));
  const int64_t bx = J.bl[0] + g % J.bn[0];
  const int64_t by = D == 2 ? J.bl[1] + g / J.bn[0] : 0;
  const int64_t b = bx + J.nb[0] * by;
  const int64_t ext0 = J.hi[0] - J.lo[0];
  T* out = reinterpret_cast<T*>(J.out);
  bool vm[N];
  int64_t oi[N];
  T xt[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int64_t gx = 4 * bx + (k & 3), gy = 4 * by + (k >> 2);
    vm[k] = gx < J.dims[0] && gx >= J.lo[0] && gx < J.hi[0] && gy < J.dims[1] && gy >= J.lo[1] && gy < J.hi[1];
    oi[k] = (gy - J.lo[1]) * ext0 + (gx - J.lo[0]);
    xt[k] = (write && J.k0 > 0 && vm[k]) ? out[oi[k]] : T(0);  // 0, or the partial sum so far
  }
  for (int j = J.k0; j < J.k; ++j) {  // Algorithm 2: x~ += D(y_j)
    const CompDesc& cd = J.comp[j];
    const uint64_t off = cd.chunk_word[b / kChunk] * 64ull + cd.brick_off[b];
    const uint64_t end = off + cd.brick_len[b];
    BitReader br;
    br.init(cd.payload, cd.nwords, off);
    const uint64_t v = br.peek(off);
    const int mode = (int)(v & 3ull);
    T xi[N];
#pragma unroll
    for (int k = 0; k < N; ++k) xi[k] = T(0);
    bool ok = true;
    if (mode == kModeZero) {
      ok = end == off + 2;
    } else if (mode == kModeRaw) {
      ok = end == off + 2 + (uint64_t)N * F::P;
      if (ok) {
#pragma unroll
        for (int k = 0; k < N; ++k) xi[k] = F::val((U)br.peek(off + 2 + (uint64_t)F::P * k));
      }
    } else if (mode == kModeCoded) {
      const int esc = (int)((v >> 2) & 7ull);
      const int emax = (int)((v >> 5) & ((1ull << F::EBITS) - 1)) - F::EBIAS;
      ok = emax >= F::EMIN && emax <= EMAXT;
      if (ok) {
        const int s = Q - emax;
        const int p = min(max(cd.L + s - C - esc, 0), F::P);
        uint64_t pos = off + HDR;
        U u[N];
#pragma unroll
        for (int r = 0; r < N; ++r) u[r] = 0;
        int n = 0, pl = F::P - 1;
        while (pl >= p) {  // leading planes with nothing significant: one 0 test bit each
          const uint64_t t = br.peek(pos);
          if (t & 1ull) break;
          const int z = t ? __ffsll((long long)t) - 1 : 64;
          const int skip = min(z, pl - p + 1);
          pos += (uint64_t)skip;
          pl -= skip;
        }
        for (; pl >= p && ok; --pl) {  // R11, as written by emit_planes
          uint64_t W = 0;
          if (n > 0) {
            W = br.peek(pos) & low_mask64(n);
            pos += (uint64_t)n;
          }
          for (int it = 0; it < N && n < N; ++it) {
            const uint64_t t = br.peek(pos);
            if (!(t & 1ull)) {
              pos += 1;
              break;
            }
            const uint64_t rest = (t >> 1) & low_mask64(N - n);
            if (!rest) {
              ok = false;
              break;
            }
            const int tz = __ffsll((long long)rest) - 1;
            W |= 1ull << (n + tz);
            n += tz + 1;
            pos += (uint64_t)tz + 2;
          }
          if (pos > end) ok = false;
#pragma unroll
          for (int r = 0; r < N; ++r) u[r] |= (U)((W >> r) & 1ull) << pl;
        }
        if (ok && pos != end) ok = false;
        S q[N];
#pragma unroll
        for (int r = 0; r < N; ++r) q[perm_small<D>(r)] = nb_inv<T>(u[r]);
        lift_inv_brick<D>(q);
#pragma unroll
        for (int k = 0; k < N; ++k) xi[k] = dequantize_val<T>(q[k], s);
      }
    } else {
      ok = false;
    }
    if (!ok) {
      atomicOr(err, 1u);
#pragma unroll
      for (int k = 0; k < N; ++k) xi[k] = T(0);
    }
#pragma unroll
    for (int k = 0; k < N; ++k) xt[k] = F::add(xt[k], xi[k]);
  }
  if (write) {
#pragma unroll
    for (int j = 0; j < N / 4; ++j) store_line<T>(out + oi[4 * j], &xt[4 * j], &vm[4 * j]);
  }
}

}  // namespace pcz
