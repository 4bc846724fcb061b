// pcz_retrieve.cu -- fused reconstruction kernel: Algorithm 2 (Magri &
// Lindstrom, Sec. 4.2) on the 4x4x4 bricks that meet a box.
//
// For each brick the kernel decodes components k0+1..k and adds them, in
// ascending order, into the partial sum x~ held in registers; x~ starts at 0
// or, to continue a refinement (Sec. 4.2), at the caller's x~_k0.  Only the
// bricks meeting the box are touched: zfp-style blocks decode on their own
// (Sec. 6.1).
//
// A launch runs a list of box jobs (one box of one field each; a single
// retrieval is a list of one, a batch of queries a longer one), each cut into
// units of consecutive bricks of its box.  A job may carry a cache of partial
// sums with, per brick, the k it holds: a brick whose cached k is at most the
// job's k starts from the cached x~ and decodes only the components above it
// (Algorithm 2's partial sums are the same whichever way they are reached).
//
// Layout: persistent CTAs of 8 warps, each taking units of 16 * umult
// consecutive bricks of a job's box.  Components are handled in rounds of up
// to 8.  Parse phase (parse_round): an index pass loads every task's block
// position and length (a task is one block: one brick and component), a
// counting sort orders the tasks longest first, and the warps steal them 32
// at a time, one block per lane (plane parsing is sequential per block, so
// this is where the lanes' parallelism comes from); a block's plane words go
// to a shared-memory slot, counted from its top plane down, and the few
// planes that do not fit to a per-CTA spill area in global memory.  After a
// barrier, each warp rebuilds its brick pairs (16 lanes per brick, lane t
// holding the x-line y = t & 3, z = t >> 2): lane p fetches plane p (and
// p + 32) of both bricks, a 32x32 bit transpose across the warp turns planes
// back into each lane's coefficients t + 16j, and the inverse reorder,
// lifting and scaling run through a bank-conflict-free brick buffer; x_j is
// then added into x~, component by component in ascending order.  Float64
// pairs whose coded planes span fewer than 16 (most of them at tolerances a
// few decades apart) are decoded in 32-bit integers scaled to their lowest
// plane and converted to double without the FP64 pipe, which the partial-sum
// adds keep busy; this form is a second instantiation of the kernel, used
// when a brick decodes at least 3 components.
#include <type_traits>

#include "pcz_device.cuh"
#include "pcz_kernels.h"

namespace pcz {

__constant__ PermTable kPerm3r = make_perm(64);

constexpr int kRWarps = 8;
constexpr int kRThreads = 32 * kRWarps;
constexpr int kRound = 8;    // components per round
constexpr int kTasks = 512;  // parse tasks (block of one brick and component) per round
constexpr int kTokLut = 512;  // entries of the group-test byte table (2 states x 256 bytes)
constexpr int kLenBuckets = 64;  // parse tasks are handed out longest block first, by len / 16
// plane words per block kept in shared memory: as many as let 3 CTAs share an SM
template <typename T>
struct Slots {
  static constexpr int n = sizeof(T) == 4 ? 15 : 14;
};

struct BlockMeta {
  uint64_t off;   // first bit of the brick in the component's payload
  int16_t s;      // scale exponent (R6), within [-1100, 1100]
  uint16_t len;   // bits of the block from the index; 0: nothing to parse (header final)
  int8_t p;       // lowest coded plane, 0..64 (64 when the block is not CODED)
  int8_t top;     // highest non-empty plane, -1 if none
  int8_t mode;
  uint8_t comp;   // component within the round
};
static_assert(sizeof(BlockMeta) == 16, "block header size");

// n / d for an invariant d, by one high multiply (DivMagic).
__device__ __forceinline__ uint32_t div_by(uint32_t n, const DivMagic& D) {
  const uint32_t t = __umulhi(D.m, n);
  return (t + ((n - t) >> D.s1)) >> D.s2;
}

template <typename T>
__host__ __device__ constexpr size_t retrieve_smem3() {
  return (size_t)kTasks * Slots<T>::n * sizeof(uint64_t)  // plane slots
         + (size_t)kTasks * sizeof(BlockMeta)       // block headers
         + (size_t)kRWarps * 128 * sizeof(typename Fmt<T>::S)  // brick buffers
         + (size_t)kTokLut * sizeof(uint16_t)                   // group-test byte table
         + (size_t)kTasks * sizeof(uint16_t)                    // parse order of the round's tasks
         + (size_t)kLenBuckets * sizeof(int);                   // task counts per length bucket
}

template <typename T>
__host__ __device__ constexpr int spill_per_block() {  // planes below a block's slot
  return Fmt<T>::P - Slots<T>::n;
}

template <typename T>
__host__ __device__ constexpr size_t spill_words_per_cta() {
  return (size_t)kTasks * spill_per_block<T>();
}

// Sequential reader of one block's bits with 32-bit positions relative to
// the start of the word that holds the block's first bit: the two current
// words in 32-bit halves, one load per 64 bits consumed, and a 64-bit window
// at any position made of two funnel shifts.  Words at or beyond the
// payload's end read as zero.  Positions must not decrease.
struct BlockBits {
  const uint64_t* __restrict__ w;  // the payload from the block's first word
  uint32_t nw;                     // words readable from w
  uint32_t wi;                     // index of the word in a0:a1
  uint32_t a0, a1, b0, b1;         // words wi and wi + 1
  __device__ __forceinline__ uint64_t ld(uint32_t i) const { return i < nw ? __ldg(w + i) : 0ull; }
  __device__ __forceinline__ void set(uint64_t lo, uint64_t hi) {
    a0 = (uint32_t)lo;
    a1 = (uint32_t)(lo >> 32);
    b0 = (uint32_t)hi;
    b1 = (uint32_t)(hi >> 32);
  }
  // bit position of the block's first bit within the reader's frame: off & 63
  __device__ __forceinline__ void init(const uint64_t* words, uint64_t nwords, uint64_t off) {
    const uint64_t w0 = off >> 6;
    w = words + w0;
    nw = w0 < nwords ? (uint32_t)min(nwords - w0, (uint64_t)0xffffffffu) : 0u;
    wi = 0;
    set(ld(0), ld(1));
  }
  __device__ __forceinline__ uint64_t peek(uint32_t pos) {
    const uint32_t i = pos >> 6;
    if (i != wi) {
      if (i == wi + 1) {
        a0 = b0;
        a1 = b1;
        const uint64_t nb = ld(i + 1);
        b0 = (uint32_t)nb;
        b1 = (uint32_t)(nb >> 32);
      } else {
        set(ld(i), ld(i + 1));
      }
      wi = i;
    }
    const bool up = pos & 32u;  // window starts in the word's upper half
    const uint32_t x0 = up ? a1 : a0, x1 = up ? b0 : a1, x2 = up ? b1 : b0;
    return ((uint64_t)__funnelshift_r(x1, x2, pos) << 32) | __funnelshift_r(x0, x1, pos);
  }
};

// Byte table of the group-test part as a two-state machine: in state "test"
// a 0 ends the part and a 1 starts a run; in state "run" every bit is the
// next coefficient's bit and a 1 ends the run.  Entry [state][byte] (16 bits):
// bits 0-7 the 1s among the byte's coefficient bits (coefficient-relative),
// bits 8-11 their count, bit 12 set when the part ends in the byte; then
// bits 13-15 hold the bits used up to and including the closing test bit,
// minus 1; otherwise bit 13 is the state after the byte.
constexpr uint32_t kTokEnded = 1u << 12;

__device__ __forceinline__ uint16_t token_lut_entry(int idx) {
  int st = idx >> 8;
  const int byte = idx & 255;
  uint32_t out = 0, cnt = 0, e = 0;
  bool ended = false;
  for (int j = 0; j < 8 && !ended; ++j) {
    const int bit = (byte >> j) & 1;
    if (st == 0) {
      if (bit) st = 1;
      else {
        ended = true;
        e = kTokEnded | ((uint32_t)j << 13);
      }
    } else {
      out |= (uint32_t)bit << cnt;
      ++cnt;
      if (bit) st = 0;
    }
  }
  if (!ended) e = (uint32_t)st << 13;
  return (uint16_t)(out | (cnt << 8) | e);
}

// The group-test part of a plane (R11), a byte at a time through the table:
// n coefficients are significant and the part starts at bit pos.  When a
// byte would carry the count to N, the last coefficient turns significant in
// it (after which no closing test bit follows) or the block is malformed; the
// part's end then follows from the byte's entry in closed form.  A valid part
// is at most 2 (N - n) + 1 <= 129 bits, so 17 bytes bound the loop.
__device__ __forceinline__ bool parse_group(BlockBits& br, uint32_t& pos, int& n, uint64_t& W, const uint16_t* lut) {
  constexpr int N = 64;
  int c = n;
  uint32_t st = 0;  // state, pre-shifted to index the table's upper half
  uint32_t used = 0;
  for (int w = 0; w < 3; ++w) {
    const uint64_t g = br.peek(pos + used);
    const uint32_t glo = (uint32_t)g, ghi = (uint32_t)(g >> 32);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (w == 2 && j == 1) return false;  // more than 17 bytes: malformed
      const uint32_t byte = ((j < 4 ? glo : ghi) >> (8 * (j & 3))) & 0xffu;
      const uint32_t e = lut[st | byte];
      const uint32_t out = e & 0xffu;
      const int cn = c + (int)((e >> 8) & 15u);
      if (cn >= N || (e & kTokEnded)) {  // the part ends in this byte
        if (cn >= N) {
          // coefficient N - 1 is the byte's coefficient bit k; its 1 ends the
          // part, with no closing test bit.  Bits used through it: k + 1
          // coefficient bits and the test bits before them (the byte's first
          // bit in the test state, and one after each earlier 1).
          const int k = N - 1 - c;
          if (!((out >> k) & 1u)) return false;  // a run past the last coefficient
          W |= (uint64_t)(out & ((2u << k) - 1u)) << c;
          pos += used + (uint32_t)(k + 1) + (st ? 0u : 1u) + (uint32_t)__popc(out & ((1u << k) - 1u));
          n = N;
        } else {
          W |= (uint64_t)out << c;
          pos += used + ((e >> 13) & 7u) + 1;
          n = cn;
        }
        return true;
      }
      W |= (uint64_t)out << c;
      c = cn;
      st = (e >> 5) & 0x100u;
      used += 8;
    }
  }
  return false;
}

// R11 decoding of planes P-1 .. p of one block, starting at bit pos and ending
// exactly at end.  Plane pl (for pl in [p, top], top = the highest non-empty
// plane, -1 if none) goes to slot[top - pl], or to spill[top - pl - Slots<T>::n]
// below the slot.  Planes above the first significant coefficient are one 0
// test bit each and are skipped together.  Returns false on a malformed
// block; every loop is bounded.
template <typename T>
__device__ bool parse_planes(BlockBits& br, uint32_t pos, uint32_t end, int p, uint64_t* slot, uint64_t* spill,
                             int& top, const uint16_t* lut) {
  constexpr int N = 64;
  int n = 0;
  top = -1;
  int pl = Fmt<T>::P - 1;
  while (pl >= p) {
    const uint64_t v = br.peek(pos);
    if (v & 1ull) break;
    const int z = v ? __ffsll((long long)v) - 1 : 64;
    const int skip = min(z, pl - p + 1);
    pos += (uint32_t)skip;
    pl -= skip;
    if (skip == z && z < 64) break;  // the bit after the zeros is the first significant plane's test 1
  }
  for (; pl >= p; --pl) {
    uint64_t W = 0;
    if (n > 0) {
      W = br.peek(pos) & low_mask64(n);
      pos += (uint32_t)n;
    }
    if (n < N && !parse_group(br, pos, n, W, lut)) return false;
    if (pos > end) return false;
    if (W && top < 0) top = pl;
    if (top >= 0) {
      const int rel = top - pl;
      if (rel < Slots<T>::n)
        slot[rel] = W;
      else if (PCZ_CHECK(rel - Slots<T>::n < spill_per_block<T>(), 3))
        spill[rel - Slots<T>::n] = W;
    }
  }
  return pos == end;
}

// One brick of the unit as seen by this lane: where it is and which of its
// values this lane's x-line writes.
struct BrickLane {
  bool have, line_ok;
  bool vm[4];
  int64_t bx, b, orow, frow;
};

// FAST_DIV: split g by invariant-integer division (measured faster for
// float64 fields and slower for float32 ones, where the kernel's register
// allocation changes with it).
template <bool FAST_DIV>
__device__ __forceinline__ BrickLane brick_lane(const BoxJob& J, int64_t g, int t) {
  BrickLane L;
  L.have = g < J.nbox;
  int64_t bx = 0, by = 0, bz = 0;
  if (L.have) {
    if (FAST_DIV && J.nbox < (1ll << 32)) {  // 32-bit division by the box's invariant extents
      const uint32_t g32 = (uint32_t)g;
      const uint32_t r = div_by(g32, J.dv_bn0);
      const uint32_t z = div_by(r, J.dv_bn1);
      bx = J.bl[0] + (int64_t)(g32 - r * (uint32_t)J.bn[0]);
      by = J.bl[1] + (int64_t)(r - z * (uint32_t)J.bn[1]);
      bz = J.bl[2] + (int64_t)z;
    } else {
      bx = J.bl[0] + g % J.bn[0];
      const int64_t r = g / J.bn[0];
      by = J.bl[1] + r % J.bn[1];
      bz = J.bl[2] + r / J.bn[1];
    }
  }
  L.bx = bx;
  L.b = bx + J.nb[0] * (by + J.nb[1] * bz);
  const int64_t gy = 4 * by + (t & 3), gz = 4 * bz + (t >> 2);
  L.line_ok = L.have && gy < J.dims[1] && gz < J.dims[2] && gy >= J.lo[1] && gy < J.hi[1] && gz >= J.lo[2] &&
              gz < J.hi[2];
  const int64_t ext0 = J.hi[0] - J.lo[0], ext1 = J.hi[1] - J.lo[1];
  L.orow = ((gz - J.lo[2]) * ext1 + (gy - J.lo[1])) * ext0 + 4 * bx - J.lo[0];
  L.frow = (gz * J.dims[1] + gy) * J.dims[0] + 4 * bx;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int64_t gx = 4 * bx + m;
    L.vm[m] = L.line_ok && gx < J.dims[0] && gx >= J.lo[0] && gx < J.hi[0];
  }
  return L;
}

// Level of brick b's cached partial sum that a job at k may start from (0:
// none): components up to it are already summed in the cache.
__device__ __forceinline__ int cached_level(const BoxJob& J, int64_t b) {
  if (!J.level) return 0;
  const int lv = J.level[b];
  return lv <= J.k ? lv : 0;
}

// x~ of this lane's 4 values at the start of a job: 0, the caller's partial
// sum x~_k0 (refinement), or the cache.
template <typename T>
__device__ __forceinline__ void start_sum(const BoxJob& J, int write, const BrickLane& BL, T* xt) {
  const int lv = BL.have ? cached_level(J, BL.b) : 0;
  const T* cache = reinterpret_cast<const T*>(J.cache);
  const T* out = reinterpret_cast<const T*>(J.out);
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    xt[m] = T(0);
    if (lv > 0 && BL.vm[m])
      xt[m] = cache[BL.frow + m];
    else if (write && J.k0 > 0 && BL.vm[m])
      xt[m] = out[BL.orow + m];
  }
}

// Rebuilds one component of the warp's brick pair (lanes 0-15: brick A,
// 16-31: brick B) from the parsed blocks mA/mB (slots sA/sB, spill pA/pB):
// returns this lane's 4 values of x_j.  SC (float64): pairs whose coded
// planes span fewer than 16 take the 32-bit integer decoding.
template <typename T, bool SC>
__device__ __forceinline__ void rebuild_pair(const BlockMeta& mA, const BlockMeta& mB, const uint64_t* sA,
                                             const uint64_t* sB, const uint64_t* pA, const uint64_t* pB,
                                             const CompDesc* cd, typename Fmt<T>::S* buf, const int* ix,
                                             const int* iy, const int* iz, const int* ir, const uint32_t* tkeep,
                                             int lane, int h, int t, T* xi) {
  using F = Fmt<T>;
  using U = typename F::U;
  using S = typename F::S;
  constexpr bool WIDE = F::P == 64;
  const BlockMeta& my = h ? mB : mA;
#pragma unroll
  for (int m = 0; m < 4; ++m) xi[m] = T(0);
  const bool cA = mA.mode == kModeCoded, cB = mB.mode == kModeCoded;
  if (cA || cB) {
    // lane l fetches plane l (and l + 32) of both bricks; planes outside
    // [p, top] are zero
    auto fetch = [&](const BlockMeta& mX, const uint64_t* sX, const uint64_t* pX, int pl) {
      if (pl < mX.p || pl > mX.top) return (uint64_t)0;  // a block not CODED has p = 64, top = -1
      const int rel = mX.top - pl;
      if (rel < Slots<T>::n) return sX[rel];
      return PCZ_CHECK(rel - Slots<T>::n < spill_per_block<T>(), 3) ? pX[rel - Slots<T>::n] : (uint64_t)0;
    };
    const int lo = min((int)mA.p, (int)mB.p);
    const int hi = max((int)mA.top, (int)mB.top);
    S r[4];            // the coefficients after the inverse transform
    bool conv = true;  // r still to be dequantised into xi
    bool scaled = false;
    if constexpr (WIDE && SC) scaled = hi - lo < 16 && lo >= 6 && hi <= 58;
    if (scaled) {
      // 64-bit coefficients whose coded planes lie in [lo, lo + 16), lo >= 6,
      // below plane 59, decoded in 32-bit integers in units of 2^(lo - 6).  A
      // coefficient with negabinary digits v from plane lo is
      // ((v ^ M) - M) * 2^lo with M = NBM >> lo (M's bits above v's do not
      // matter).  In these units each pass of the inverse lifting turns
      // multiples of 2^a into multiples of 2^(a - 2), so from 2^6 every shift
      // divides an even number exactly; and |value| < 2^(hi - lo + 6.42) *
      // 2.75^3 < 2^26 (2.75: the largest row sum of the inverse lifting's
      // coefficients), while the unscaled value stays below 2^(hi + 4.8) <= 2^63.
      // Neither form wraps, so the result is the 64-bit decoding's exactly.
      const int pl = lo + (lane & 15);
      const uint64_t WA = fetch(mA, sA, pA, pl), WB = fetch(mB, sB, pB, pl);
      const uint32_t sel = h ? 0x7632u : 0x5410u;
      const uint32_t M = (uint32_t)(F::NBM >> min(lo, 63));  // lo = 64: no digit at all
      int32_t* b32 = reinterpret_cast<int32_t*>(buf);
#pragma unroll
      for (int t2 = 0; t2 < 2; ++t2) {
        const uint32_t row = __byte_perm((uint32_t)(WA >> (32 * t2)), (uint32_t)(WB >> (32 * t2)), sel);
        const uint32_t w = transpose32(row, lane, tkeep);
        b32[ir[2 * t2]] = (int32_t)((((w & 0xffffu) ^ M) - M) << 6);
        b32[ir[2 * t2 + 1]] = (int32_t)((((w >> 16) ^ M) - M) << 6);
      }
      __syncwarp();
      {
        int32_t a = b32[iz[0]], bq = b32[iz[1]], c = b32[iz[2]], d = b32[iz[3]];
        lift_inv(a, bq, c, d);
        b32[iz[0]] = a; b32[iz[1]] = bq; b32[iz[2]] = c; b32[iz[3]] = d;
      }
      __syncwarp();
      {
        int32_t a = b32[iy[0]], bq = b32[iy[1]], c = b32[iy[2]], d = b32[iy[3]];
        lift_inv(a, bq, c, d);
        b32[iy[0]] = a; b32[iy[1]] = bq; b32[iy[2]] = c; b32[iy[3]] = d;
      }
      __syncwarp();
      int32_t q[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) q[m] = b32[ix[m]];
      __syncwarp();
      lift_inv(q[0], q[1], q[2], q[3]);
      if (my.s >= -960 && my.s <= 1022) {  // R13 without rounding (scaled_i32_to_f64)
        if constexpr (WIDE) {
          if (my.mode == kModeCoded) {
            const uint32_t eb = (uint32_t)(1053 + (lo - 6) - my.s) << 20;
#pragma unroll
            for (int m = 0; m < 4; ++m) xi[m] = scaled_i32_to_f64(q[m], eb);
          }
        }
        conv = false;
      } else {  // the general path below, on the unscaled coefficients
#pragma unroll
        for (int m = 0; m < 4; ++m) r[m] = (S)((U)(int64_t)q[m] << (lo - 6));
      }
    } else {
      U u[4];
      if ((!WIDE || !SC) && hi - lo < 16) {
        // every coded plane of the pair lies in [lo, lo + 16): one transpose
        // carries two coefficient groups, rows 0-15 the planes of group 2t and
        // rows 16-31 those of group 2t + 1 (lane l fetches plane lo + (l & 15))
        const int pl = lo + (lane & 15);
        const uint64_t WA = fetch(mA, sA, pA, pl), WB = fetch(mB, sB, pB, pl);
        const uint32_t sel = h ? 0x7632u : 0x5410u;  // 16-bit group 2 t2 + h of both words
#pragma unroll
        for (int t2 = 0; t2 < 2; ++t2) {
          const uint32_t row = __byte_perm((uint32_t)(WA >> (32 * t2)), (uint32_t)(WB >> (32 * t2)), sel);
          const uint32_t w = transpose32(row, lane, tkeep);
          u[2 * t2] = (U)((U)(w & 0xffffu) << lo);
          u[2 * t2 + 1] = (U)((U)(w >> 16) << lo);
        }
      } else {
        // lane l fetches plane base + l (and base + 32 + l for 64-bit
        // coefficients when the coded planes of the pair span more than 32)
        int base = 0;
        bool two = WIDE;
        if constexpr (WIDE) {
          if (hi - lo < 32) {  // one 32-plane window holds every coded plane
            base = lo;
            two = false;
          }
        }
        const uint64_t WA0 = fetch(mA, sA, pA, base + lane), WB0 = fetch(mB, sB, pB, base + lane);
        {
          uint32_t tl[4];
          tl[0] = __byte_perm((uint32_t)WA0, (uint32_t)WB0, 0x5410);
          tl[1] = __byte_perm((uint32_t)WA0, (uint32_t)WB0, 0x7632);
          tl[2] = __byte_perm((uint32_t)(WA0 >> 32), (uint32_t)(WB0 >> 32), 0x5410);
          tl[3] = __byte_perm((uint32_t)(WA0 >> 32), (uint32_t)(WB0 >> 32), 0x7632);
#pragma unroll
          for (int j = 0; j < 4; ++j) u[j] = (U)transpose32(tl[j], lane, tkeep) << base;
        }
        if constexpr (WIDE) {
          if (two) {
            const uint64_t WA1 = fetch(mA, sA, pA, lane + 32), WB1 = fetch(mB, sB, pB, lane + 32);
            uint32_t th[4];
            th[0] = __byte_perm((uint32_t)WA1, (uint32_t)WB1, 0x5410);
            th[1] = __byte_perm((uint32_t)WA1, (uint32_t)WB1, 0x7632);
            th[2] = __byte_perm((uint32_t)(WA1 >> 32), (uint32_t)(WB1 >> 32), 0x5410);
            th[3] = __byte_perm((uint32_t)(WA1 >> 32), (uint32_t)(WB1 >> 32), 0x7632);
#pragma unroll
            for (int j = 0; j < 4; ++j) u[j] |= (U)((uint64_t)transpose32(th[j], lane, tkeep) << 32);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) buf[ir[j]] = nb_inv<T>(u[j]);
      __syncwarp();
      {
        S a = buf[iz[0]], bq = buf[iz[1]], c = buf[iz[2]], d = buf[iz[3]];
        lift_inv(a, bq, c, d);
        buf[iz[0]] = a; buf[iz[1]] = bq; buf[iz[2]] = c; buf[iz[3]] = d;
      }
      __syncwarp();
      {
        S a = buf[iy[0]], bq = buf[iy[1]], c = buf[iy[2]], d = buf[iy[3]];
        lift_inv(a, bq, c, d);
        buf[iy[0]] = a; buf[iy[1]] = bq; buf[iy[2]] = c; buf[iy[3]] = d;
      }
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 4; ++m) r[m] = buf[ix[m]];
      __syncwarp();
      lift_inv(r[0], r[1], r[2], r[3]);
    }
    if (conv && my.mode == kModeCoded) dequantize_line<T, true>(r, my.s, xi);
  }
  if (my.mode == kModeRaw) {
#pragma unroll
    for (int m = 0; m < 4; ++m)
      xi[m] = F::val((U)peek64(cd->payload, cd->nwords, my.off + 2 + (uint64_t)F::P * (4 * t + m)));
  }
}

// Parse task L decodes the block that the round's index pass placed in
// meta[L] (component base + comp, its first bit and length) into slot L and
// replaces meta[L] by the block's header.  An entry of length 0 (a brick past
// the box, or a component the brick takes from the cache) is final already.
template <typename T>
__device__ __forceinline__ void parse_task(const BoxJob& J, unsigned int* err, int base, int L, uint64_t* slots,
                                           BlockMeta* meta, uint64_t* spill, const uint16_t* lut) {
  using F = Fmt<T>;
  constexpr int N = 64;
  constexpr int Q = F::P - 2 - Geo<3>::G;
  constexpr int C = Geo<3>::C;
  constexpr int HDR = 2 + 3 + F::EBITS;
  constexpr int EMAXT = (1 << (F::EXPW - 1));  // frexp exponent of the largest finite T
  constexpr int SP = spill_per_block<T>();
  const BlockMeta in = meta[L];
  if (in.len == 0) return;
  const CompDesc& cd = J.comp[base + in.comp];
  BlockBits br;  // positions from the start of the block's first word
  br.init(cd.payload, cd.nwords, in.off);
  const uint32_t start = (uint32_t)(in.off & 63u), end = start + in.len;
  const uint64_t v = br.peek(start);
  int mode = (int)(v & 3ull), s = 0, p = 0, top = -1;
  bool ok;
  if (mode == kModeZero) {
    ok = in.len == 2;
  } else if (mode == kModeRaw) {
    ok = in.len == 2 + N * F::P;
  } else if (mode == kModeCoded) {
    const int esc = (int)((v >> 2) & 7ull);
    const int emax = (int)((v >> 5) & ((1ull << F::EBITS) - 1)) - F::EBIAS;
    ok = emax >= F::EMIN && emax <= EMAXT;
    if (ok) {
      s = Q - emax;
      p = min(max(cd.L + s - C - esc, 0), F::P);
      ok = parse_planes<T>(br, start + HDR, end, p, slots + L * Slots<T>::n, spill + L * SP, top, lut);
    }
  } else {
    ok = false;
  }
  if (!ok) {
    atomicOr(err, 1u);
    mode = kModeZero;
  }
  BlockMeta bm = in;
  bm.mode = (int8_t)mode;
  bm.s = (int16_t)s;
  bm.p = (int8_t)(mode == kModeCoded ? p : 64);  // no plane of a ZERO or RAW block is coded
  bm.top = (int8_t)top;
  meta[L] = bm;
}

// Parse phase of a round: task L is component base + L / ub of unit brick
// L % ub (ub = bricks per unit).
//  1. Index pass: every thread looks up the index of its tasks (first bit and
//     length of the block; the loads of the whole round are in flight
//     together) into meta[L], and counts them per length bucket.
//  2. A counting sort of the tasks by block length, longest first (each warp
//     scans the bucket counts itself), into order[].
//  3. Warp-granular work stealing over order[]: each warp takes the next 32
//     tasks until none is left.  The 32 blocks a warp parses side by side are
//     then of alike length, so lanes wait little for one another, and the
//     short blocks at the end fill the gaps before the barrier.
// Every thread of the CTA calls it; hist[] is zero on entry and on return.
template <typename T>
__device__ __forceinline__ void parse_round(const BoxJob& J, unsigned int* err, int64_t unit0, int ub, int base,
                                            int nc, int* next, uint64_t* slots, BlockMeta* meta, uint64_t* spill,
                                            const uint16_t* lut, uint16_t* order, int* hist) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int ntask = nc * ub;
  constexpr int PER = kTasks / kRThreads;  // tasks per thread in the index pass
  int key[PER], rank[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int L = threadIdx.x + q * kRThreads;
    key[q] = -1;
    if (L >= ntask) continue;
    const int jj = (int)div_by((uint32_t)L, J.dv_ub);  // ub = 16 * umult
    const int64_t g = unit0 + (L - jj * ub);
    BlockMeta bm;
    bm.off = 0;
    bm.s = 0;
    bm.len = 0;
    bm.p = 64;
    bm.top = -1;
    bm.mode = kModeZero;
    bm.comp = (uint8_t)jj;
    if (g < J.nbox) {
      int64_t bx, by, bz;
      if (J.nbox < (1ll << 32)) {  // 32-bit division by the box's invariant extents
        const uint32_t g32 = (uint32_t)g;
        const uint32_t r = div_by(g32, J.dv_bn0);
        const uint32_t z = div_by(r, J.dv_bn1);
        bx = J.bl[0] + (int64_t)(g32 - r * (uint32_t)J.bn[0]);
        by = J.bl[1] + (int64_t)(r - z * (uint32_t)J.bn[1]);
        bz = J.bl[2] + (int64_t)z;
      } else {
        bx = J.bl[0] + g % J.bn[0];
        const int64_t r = g / J.bn[0];
        by = J.bl[1] + r % J.bn[1];
        bz = J.bl[2] + r / J.bn[1];
      }
      const int64_t b = bx + J.nb[0] * (by + J.nb[1] * bz);
      if (base + jj >= cached_level(J, b)) {
        const CompDesc& cd = J.comp[base + jj];
        bm.off = cd.chunk_word[b / kChunk] * 64ull + cd.brick_off[b];
        bm.len = cd.brick_len[b];
      }
    }
    meta[L] = bm;
    key[q] = kLenBuckets - 1 - min((int)(bm.len >> 4), kLenBuckets - 1);  // longest first
    rank[q] = atomicAdd(hist + key[q], 1);
  }
  __syncthreads();
  // bucket bases: an exclusive scan of the 64 counts, two per lane, in every warp
  const int h0 = hist[2 * lane], h1 = hist[2 * lane + 1];
  int incl = h0 + h1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(FULL, incl, o);
    if (lane >= o) incl += y;
  }
  const int b0 = incl - h0 - h1, b1 = incl - h1;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int k = key[q] < 0 ? 0 : key[q];
    const int e0 = __shfl_sync(FULL, b0, k >> 1), e1 = __shfl_sync(FULL, b1, k >> 1);
    if (key[q] >= 0) order[((k & 1) ? e1 : e0) + rank[q]] = (uint16_t)(threadIdx.x + q * kRThreads);
  }
  __syncthreads();
  if (threadIdx.x < kLenBuckets) hist[threadIdx.x] = 0;  // read by every warp before the barrier
  for (;;) {
    int t0 = 0;
    if (lane == 0) t0 = atomicAdd(next, 32);
    t0 = __shfl_sync(FULL, t0, 0);
    if (t0 >= ntask) break;
    if (t0 + lane < ntask) parse_task<T>(J, err, base, order[t0 + lane], slots, meta, spill, lut);
  }
}

template <typename T, bool SC>
__global__ void __launch_bounds__(kRThreads, 3) k_retrieve3(const RetrieveParams R) {
  using F = Fmt<T>;
  using S = typename F::S;
  constexpr int SP = spill_per_block<T>();

  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* slots = reinterpret_cast<uint64_t*>(smem);                // [kTasks][Slots<T>::n]
  BlockMeta* meta = reinterpret_cast<BlockMeta*>(slots + kTasks * Slots<T>::n);  // [kTasks]
  S* bufs = reinterpret_cast<S*>(meta + kTasks);                           // [kRWarps][128]
  uint16_t* lut = reinterpret_cast<uint16_t*>(bufs + kRWarps * 128);       // [kTokLut]
  uint16_t* order = lut + kTokLut;                                         // [kTasks]
  int* hist = reinterpret_cast<int*>(order + kTasks);                      // [kLenBuckets]
  if (threadIdx.x < kLenBuckets) hist[threadIdx.x] = 0;
  for (int i = threadIdx.x; i < kTokLut; i += kRThreads) lut[i] = token_lut_entry(i);  // read after the loop's first barrier
  __shared__ int s_next;  // next parse task of the round
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, t = lane & 15;
  S* buf = bufs + warp * 128;
  uint64_t* spill = R.spill + (size_t)blockIdx.x * spill_words_per_cta<T>();

  const int xx = t & 3, yq = t >> 2, ly = t & 3, lz = t >> 2;
  int ix[4], iy[4], iz[4], ir[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    ix[m] = sidx<T>(m, ly, lz, h);
    iy[m] = sidx<T>(xx, m, yq, h);
    iz[m] = sidx<T>(xx, yq, m, h);
    const int pos = kPerm3r.pos[t + 16 * m];
    ir[m] = sidx<T>(pos & 3, (pos >> 2) & 3, pos >> 4, h);
  }
  uint32_t tkeep[5];
  transpose_masks(lane, tkeep);
  __shared__ BoxJob sJ;
  const BoxJob& J = sJ;
  constexpr int JW = (int)(sizeof(BoxJob) / 8);
  static_assert(sizeof(BoxJob) % 8 == 0 && JW <= kRThreads, "job copy");

  for (int64_t unit = blockIdx.x; unit < R.nunits; unit += gridDim.x) {
    __syncthreads();  // the previous unit is done with sJ
    if (!R.jobs) {
      if (threadIdx.x == 0) sJ = R.job0;
    } else if (threadIdx.x < JW) {  // the job whose units contain this one
      int lo = 0, hi = R.njobs - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (R.jobs[mid].unit_begin <= unit)
          lo = mid;
        else
          hi = mid - 1;
      }
      reinterpret_cast<uint64_t*>(&sJ)[threadIdx.x] = reinterpret_cast<const uint64_t*>(R.jobs + lo)[threadIdx.x];
    }
    if (threadIdx.x == kRThreads - 1) s_next = 0;
    __syncthreads();
    T* out = reinterpret_cast<T*>(J.out);
    const int umult = J.umult;
    const int ub = 16 * umult;  // bricks per unit: umult brick pairs per warp
    const int64_t unit0 = (unit - J.unit_begin) * ub;
    if (J.k - J.k0 <= kRound) {
      // one round: every warp parses, then each warp rebuilds its umult
      // brick pairs and writes them out
      const int nc = J.k - J.k0;
      parse_round<T>(J, R.err, unit0, ub, J.k0, nc, &s_next, slots, meta, spill, lut, order, hist);
      __syncthreads();
      for (int q = 0; q < umult; ++q) {
        const int uA = 2 * (umult * warp + q);  // unit-local index of the pair's first brick
        const BrickLane BL = brick_lane<sizeof(T) == 8>(J, unit0 + uA + h, t);
        T xt[4];
        start_sum<T>(J, R.write, BL, xt);
        for (int jj = 0; jj < nc; ++jj) {  // Algorithm 2, components in ascending order
          const int L = jj * ub + uA;
          const BlockMeta mA = meta[L], mB = meta[L + 1];
          T xi[4];
          rebuild_pair<T, SC>(mA, mB, slots + L * Slots<T>::n, slots + (L + 1) * Slots<T>::n, spill + L * SP, spill + (L + 1) * SP,
                          &J.comp[J.k0 + jj], buf, ix, iy, iz, ir, tkeep, lane, h, t, xi);
#pragma unroll
          for (int m = 0; m < 4; ++m) xt[m] = F::add(xt[m], xi[m]);  // x~ += x_j
        }
        if (R.write) {
          store_line<T>(out + BL.orow, xt, BL.vm);
        }
      }
    } else {
      // several rounds (umult = 2, units of 32 bricks): x~ of the warp's 4
      // bricks stays in registers across rounds
      BrickLane BL[2];
      T xt[2][4];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        BL[q] = brick_lane<sizeof(T) == 8>(J, unit0 + 4 * warp + 2 * q + h, t);
        start_sum<T>(J, R.write, BL[q], xt[q]);
      }
      for (int base = J.k0; base < J.k; base += kRound) {
        const int nc = min(kRound, J.k - base);
        parse_round<T>(J, R.err, unit0, 32, base, nc, &s_next, slots, meta, spill, lut, order, hist);
        __syncthreads();
        for (int jj = 0; jj < nc; ++jj) {
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int uA = 4 * warp + 2 * q;
            const int L = jj * 32 + uA;
            const BlockMeta mA = meta[L], mB = meta[L + 1];
            T xi[4];
            rebuild_pair<T, SC>(mA, mB, slots + L * Slots<T>::n, slots + (L + 1) * Slots<T>::n, spill + L * SP,
                            spill + (L + 1) * SP, &J.comp[base + jj], buf, ix, iy, iz, ir, tkeep, lane, h, t, xi);
#pragma unroll
            for (int m = 0; m < 4; ++m) xt[q][m] = F::add(xt[q][m], xi[m]);
          }
        }
        __syncthreads();  // the next round's parse reuses the slots and the task counter
        if (threadIdx.x == 0) s_next = 0;
        __syncthreads();
      }
      if (R.write) {
#pragma unroll
        for (int q = 0; q < 2; ++q)
          store_line<T>(out + BL[q].orow, xt[q], BL[q].vm);
      }
    }
  }
}

// Brick pairs per warp in a unit (a unit is 16 * umult bricks): as many as
// keep one round's parse tasks (bricks x components) within kTasks, two per
// thread, so that warps can steal work; several rounds use 2 pairs per warp.
int retrieve_unit_mult(int ncomp) {
  if (ncomp <= 0 || ncomp > kRound) return 2;
  const int m = (kTasks / 16) / ncomp;
  return m < 1 ? 1 : m;
}

template <typename T>
static int retrieve_grid_t(int64_t nunits) {
  // CTAs that fit on the GPU at once, queried once per type (a function-local
  // static: initialised once even when several host threads get here first)
  static const int64_t g = [] {
    int dev = 0, sms = 0, ps = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_retrieve3<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)retrieve_smem3<T>());
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, k_retrieve3<T, false>, kRThreads, retrieve_smem3<T>()) !=
        cudaSuccess) {
      cudaGetLastError();
      ps = 1;
    }
    return (int64_t)(ps < 1 ? 1 : ps) * (sms < 1 ? 1 : sms);
  }();
  return (int)(nunits < g ? (nunits > 0 ? nunits : 1) : g);
}

int retrieve_grid(int dtype, int ndims, int64_t nunits) {
  if (ndims != 3) return 1;  // the 1D/2D kernel is not persistent
  return dtype == 1 ? retrieve_grid_t<float>(nunits) : retrieve_grid_t<double>(nunits);
}

size_t retrieve_spill_words(int dtype, int ndims, int grid) {
  if (ndims != 3) return 0;
  return (dtype == 1 ? spill_words_per_cta<float>() : spill_words_per_cta<double>()) * (size_t)grid;
}

// Float64 retrieval decoding at least this many components per brick takes
// the kernel with the 32-bit decoding of narrow pairs (SC): measured 7.5 %
// faster over k = 1..8 of a 512^3 field with 8 components (11 % at k = 8), but
// 8 % slower at k = 1 and 1 % slower at k = 2, where the parse, whose
// registers the extra path crowds, dominates.  Lists of jobs (batches, served
// queries) take it too.
constexpr int kScaledMinComponents = 3;

template <typename T>
static cudaError_t launch_retrieve_t(const RetrieveParams& p, cudaStream_t s) {
  const size_t smem = retrieve_smem3<T>();
  cudaError_t e = cudaFuncSetAttribute(k_retrieve3<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if constexpr (sizeof(T) == 8)
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_retrieve3<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (p.nunits == 0) return cudaSuccess;
  bool sc = false;
  if constexpr (sizeof(T) == 8) sc = p.jobs != nullptr || p.job0.k - p.job0.k0 >= kScaledMinComponents;
  if constexpr (sizeof(T) == 8)
    if (sc) {
      k_retrieve3<T, true><<<(unsigned)p.grid, kRThreads, smem, s>>>(p);
      return cudaGetLastError();
    }
  k_retrieve3<T, false><<<(unsigned)p.grid, kRThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_retrieve(int dtype, int ndims, const RetrieveParams& p, cudaStream_t s) {
  if (ndims == 1 || ndims == 2) return launch_retrieve_small(dtype, ndims, p, s);
  if (ndims != 3) return cudaErrorNotSupported;
  return dtype == 1 ? launch_retrieve_t<float>(p, s) : launch_retrieve_t<double>(p, s);
}

uint32_t check_word_retrieve(int reset) { return read_check_word(reset); }

}  // namespace pcz
