// pcz_device.cuh -- device-side building blocks of the PCZ block coder used as
// the compressor C / decompressor D of the multi-component framework
// (Algorithm 1 and 2 of Magri & Lindstrom, Sec. 4).  GPU path only.
//
// The coder is zfp-style (Sec. 4.4, Sec. 6.1): one exponent per 4^d brick and
// component, an exactly invertible integer lifting transform, negabinary
// coefficients and group-tested bit planes (Sec. 2).  The paper does not fix
// the coder's internals; the project rules R4..R15 do, and each is restated
// where it is implemented.  All floating-point work here is IEEE
// round-to-nearest with no contraction: the only arithmetic on T values is
// one add or one subtract (explicit _rn intrinsics); scaling and conversions
// are done on the bit patterns with integer operations.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "pcz_kernels.h"

namespace pcz {
constexpr int kModeZero = 0, kModeCoded = 1, kModeRaw = 2;

// ---------------------------------------------------------------------------
// Field types.  P = integer width = bits of T.
// ---------------------------------------------------------------------------
template <typename T>
struct Fmt;

template <>
struct Fmt<float> {
  using U = uint32_t;
  using S = int32_t;
  static constexpr int P = 32;
  static constexpr int MANT = 24;    // significand bits, hidden bit included
  static constexpr int EMIN = -125;  // frexp exponent of the smallest normal
  static constexpr int EBITS = 8;    // stored block exponent width
  static constexpr int EBIAS = 126;  // stored = emax + EBIAS
  static constexpr int BIAS = 127;   // IEEE exponent bias
  static constexpr int EXPW = 8;     // IEEE exponent field width
  static constexpr U SIGN = 0x80000000u, ABS = 0x7FFFFFFFu, INF = 0x7F800000u;
  static constexpr U NBM = 0xAAAAAAAAu;
  __device__ static U bits(float v) { return __float_as_uint(v); }
  __device__ static float val(U b) { return __uint_as_float(b); }
  __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ static float sub(float a, float b) { return __fsub_rn(a, b); }
  __device__ static int clz(U a) { return __clz(a); }
};

template <>
struct Fmt<double> {
  using U = uint64_t;
  using S = int64_t;
  static constexpr int P = 64;
  static constexpr int MANT = 53;
  static constexpr int EMIN = -1021;
  static constexpr int EBITS = 11;
  static constexpr int EBIAS = 1022;
  static constexpr int BIAS = 1023;
  static constexpr int EXPW = 11;
  static constexpr U SIGN = 0x8000000000000000ull, ABS = 0x7FFFFFFFFFFFFFFFull, INF = 0x7FF0000000000000ull;
  static constexpr U NBM = 0xAAAAAAAAAAAAAAAAull;
  __device__ static U bits(double v) { return (U)__double_as_longlong(v); }
  __device__ static double val(U b) { return __longlong_as_double((long long)b); }
  __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ static double sub(double a, double b) { return __dsub_rn(a, b); }
  __device__ static int clz(U a) { return __clzll((long long)a); }
};

// Brick geometry for dimensionality D: N = 4^D coefficients, G = 2D headroom
// bits for the forward transform's growth (R6), C guard planes (R10): the
// smallest c with 2^c above (2/3) * 2.75^D, the inverse transform's worst-case
// error per unit of truncated coefficient.
template <int D>
struct Geo {
  static constexpr int N = D == 1 ? 4 : D == 2 ? 16 : 64;
  static constexpr int G = 2 * D;
  static constexpr int C = D == 1 ? 1 : D == 2 ? 3 : 4;
};

// ---------------------------------------------------------------------------
// Wrapping P-bit integer arithmetic (two's complement, modulo 2^P).
// ---------------------------------------------------------------------------
template <typename S>
__device__ __forceinline__ S wadd(S a, S b) {
  using U = typename std::make_unsigned<S>::type;
  return (S)((U)a + (U)b);
}
template <typename S>
__device__ __forceinline__ S wsub(S a, S b) {
  using U = typename std::make_unsigned<S>::type;
  return (S)((U)a - (U)b);
}

// R7: forward lifting of one 4-vector: integer Haar on the pairs, Haar on the
// pair means, then the second difference and the fine slope minus half the
// coarse slope.  a,b,c,d -> (mean, coarse slope, e1, e2).
template <typename S>
__device__ __forceinline__ void lift_fwd(S& a, S& b, S& c, S& d) {
  S d1 = wsub(b, a);
  S s1 = wadd(a, d1 >> 1);
  S d2 = wsub(d, c);
  S s2 = wadd(c, d2 >> 1);
  S d0 = wsub(s2, s1);
  S s0 = wadd(s1, d0 >> 1);
  S e2 = wsub(d2, d1);
  S e1 = wsub(d1, d0 >> 1);
  a = s0;
  b = d0;
  c = e1;
  d = e2;
}

// R7 inverse: the forward steps replayed backwards with opposite signs.
template <typename S>
__device__ __forceinline__ void lift_inv(S& a, S& b, S& c, S& d) {
  S s0 = a, d0 = b, e1 = c, e2 = d;
  S d1 = wadd(e1, d0 >> 1);
  S d2 = wadd(e2, d1);
  S s1 = wsub(s0, d0 >> 1);
  S s2 = wadd(s1, d0);
  a = wsub(s1, d1 >> 1);
  b = wadd(a, d1);
  c = wsub(s2, d2 >> 1);
  d = wadd(c, d2);
}

// R9: negabinary map and its inverse, modulo 2^P.
template <typename T>
__device__ __forceinline__ typename Fmt<T>::U nb_fwd(typename Fmt<T>::S q) {
  using F = Fmt<T>;
  return (typename F::U)(((typename F::U)q + F::NBM) ^ F::NBM);
}
template <typename T>
__device__ __forceinline__ typename Fmt<T>::S nb_inv(typename Fmt<T>::U u) {
  using F = Fmt<T>;
  return (typename F::S)((u ^ F::NBM) - F::NBM);
}

// IEEE biased exponent field of a bit pattern.
template <typename T>
__device__ __forceinline__ int biased_exp(typename Fmt<T>::U b) {
  using F = Fmt<T>;
  return (int)((b >> (F::MANT - 1)) & ((1u << F::EXPW) - 1));
}

// R6: block exponent from the largest biased exponent over the brick: emax is
// the frexp exponent of the largest magnitude, floored at the smallest normal's
// (subnormals and zeros carry biased exponent 0).
template <typename T>
__device__ __forceinline__ int block_emax_from_be(int be_max) {
  using F = Fmt<T>;
  return (be_max > 1 ? be_max : 1) - (F::BIAS - 1);
}

// R6: q = sign(e) * floor(|e| * 2^s), computed exactly on the bit pattern:
// |e| = m * 2^ex with m the integer significand.
template <typename T>
__device__ __forceinline__ typename Fmt<T>::S quantize(typename Fmt<T>::U b, int s) {
  using F = Fmt<T>;
  using U = typename F::U;
  using S = typename F::S;
  int be = biased_exp<T>(b);
  U m = b & ((U(1) << (F::MANT - 1)) - 1);
  if (be) m |= U(1) << (F::MANT - 1);
  int ex = (be ? be : 1) - F::BIAS - (F::MANT - 1);
  int sh = ex + s;
  U a;
  if (sh >= 0)
    a = sh >= F::P ? U(0) : (m << sh);
  else
    a = -sh >= F::P ? U(0) : (m >> (-sh));
  S q = (S)a;
  return (b & F::SIGN) ? (S)(0 - (U)q) : q;
}

// R13: the T value nearest to q * 2^-s (ties to even, one rounding, IEEE signed
// zero, +-inf beyond the largest finite value), as a bit pattern.
template <typename T>
__device__ __forceinline__ typename Fmt<T>::U dequantize_bits(typename Fmt<T>::S q, int s) {
  using F = Fmt<T>;
  using U = typename F::U;
  if (q == 0) return U(0);
  U a = q < 0 ? (U)(U(0) - (U)q) : (U)q;
  int nb = F::P - F::clz(a);            // bit length of |q|
  int E = nb - s;                       // frexp exponent of the exact value
  int qe = (E > F::EMIN ? E : F::EMIN) - F::MANT;  // exponent of the last place
  int sh = qe + s;                      // low bits of |q| below that place
  U r;
  if (sh <= 0) {
    r = a << (-sh);
  } else if (sh > F::P) {
    r = 0;
  } else if (sh == F::P) {
    r = a > (U(1) << (F::P - 1)) ? U(1) : U(0);
  } else {
    r = a >> sh;
    U rem = a & ((U(1) << sh) - 1);
    U half = U(1) << (sh - 1);
    if (rem > half || (rem == half && (r & 1))) r += 1;
  }
  int ef = qe - (F::EMIN - F::MANT);    // biased exponent - 1 for a normal result
  U out;
  if (ef >= (1 << F::EXPW) - 2) {
    out = F::INF;
  } else {
    out = ((U)ef << (F::MANT - 1)) + r;  // a carry out of r bumps the exponent
    if (out > F::INF) out = F::INF;
  }
  return q < 0 ? (out | F::SIGN) : out;
}

// R13 for float fields, the common case in a few instructions: when 2^-s is a
// normal float and the result is normal or overflows, int->float rounding
// followed by an exact power-of-two scaling is the single correct rounding.
// Other cases take the general path.
__device__ __forceinline__ float dequantize_f32(int32_t q, int s) {
  if (q == 0) return 0.0f;
  const uint32_t a = q < 0 ? 0u - (uint32_t)q : (uint32_t)q;
  const int nb = 32 - __clz(a);
  if (s >= -127 && s <= 126 && nb - s >= -125)
    return __fmul_rn(__int2float_rn(q), __uint_as_float((uint32_t)(127 - s) << 23));
  return __uint_as_float(dequantize_bits<float>(q, s));
}

// R13 for float64 when the result is known to be normal and finite (s in
// [-960, 1022], see dequantize_line): the 53 leading bits of |q| rounded to
// nearest, ties to even, by adding half an ulp less one plus the kept lsb
// before the shift.  A carry out of the 53 bits moves into the exponent field.
__device__ __forceinline__ uint64_t dequantize_f64_normal(int64_t q, int s) {
  if (q == 0) return 0ull;
  const uint64_t a = q < 0 ? 0ull - (uint64_t)q : (uint64_t)q;
  const int nb = 64 - __clzll((long long)a);  // |q| < 2^nb, so a + half stays below 2^64
  const int sh = nb - 53;
  uint64_t r;
  if (sh > 0)
    r = (a + ((1ull << (sh - 1)) - 1ull) + ((a >> sh) & 1ull)) >> sh;
  else
    r = a << (-sh);
  const uint64_t bits = ((uint64_t)(nb - s + 1021) << 52) + r;  // r's bit 52 completes the exponent
  return q < 0 ? (bits | Fmt<double>::SIGN) : bits;
}

template <typename T>
__device__ __forceinline__ T dequantize_val(typename Fmt<T>::S q, int s) {
  if constexpr (sizeof(T) == 4)
    return dequantize_f32(q, s);
  else
    return Fmt<T>::val(dequantize_bits<T>(q, s));
}

// R13 for the 4 values of a line that share the block's scale s.
//  float: when 2^-s is a normal float, int -> float rounding followed by the
//    exact multiplication by 2^-s is the single correct rounding for every q
//    (|q| >= 1 keeps the result normal; overflow gives +-inf as IEEE does;
//    q = 0 gives +0), so the test is made once per line.
//  double with EXP: int64 -> double rounding (one rounding), then 2^-s applied
//    by subtracting s from the exponent field.  For |q| in [1, 2^63] the
//    rounded value's biased exponent lies in [1023, 1086], so for s in
//    [-960, 1022] the scaled one lies in [1, 2046]: normal and finite, the
//    scaling exact, the field never borrows from or carries into the sign.
//    This spends one conversion instead of some 25 integer instructions, for
//    kernels whose integer pipe is the busier one.
//  Other cases take the integer path (dequantize_bits).
template <typename T, bool EXP>
__device__ __forceinline__ void dequantize_line(const typename Fmt<T>::S* q, int s, T* v) {
  if constexpr (sizeof(T) == 4) {
    if (s >= -127 && s <= 126) {
      const float sc = __uint_as_float((uint32_t)(127 - s) << 23);
#pragma unroll
      for (int m = 0; m < 4; ++m) v[m] = __fmul_rn(__int2float_rn(q[m]), sc);
      return;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) v[m] = __uint_as_float(dequantize_bits<float>(q[m], s));
  } else {
    if (EXP && s >= -960 && s <= 1022) {
      const uint32_t adj = (uint32_t)s << 20;  // s in the exponent field of the high word
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const double d = __ll2double_rn(q[m]);
        const uint32_t hi = (uint32_t)__double2hiint(d);
        v[m] = __hiloint2double((int)(hi ? hi - adj : 0u), __double2loint(d));  // q = 0 stays +0
      }
      return;
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) v[m] = Fmt<double>::val(dequantize_bits<double>(q[m], s));
  }
}

// R13 for a float64 coefficient decoded in 32-bit integers in units of 2^e:
// the coefficient is q = r * 2^e exactly, |r| < 2^31, and 1 <= |q| < 2^63 when
// r != 0.  For s in [-960, 1022] the result q * 2^-s is then normal and finite
// (the bound of dequantize_line), so no rounding is needed: with |r|'s leading
// one moved to bit 31, the 31 bits below it are the top of the 52-bit
// fraction, and the biased exponent is 1023 + (31 - clz|r|) + e - s.  Pass
// eb = (1053 + e - s) << 20 (that exponent minus 1, plus clz|r|, in the high
// word's exponent field; the leading one, added at bit 20, completes it).
// r = 0 gives +0.  Integer instructions only: no int -> double conversion,
// whose FP64 pipe the partial-sum adds keep busy.
__device__ __forceinline__ double scaled_i32_to_f64(int32_t r, uint32_t eb) {
  const uint32_t a = (uint32_t)abs(r);
  const uint32_t z = (uint32_t)__clz(a);
  const uint32_t n = __funnelshift_l(0u, a, z);  // |r| << clz; 0 for r = 0
  const uint32_t hw = ((n >> 11) + eb - (z << 20)) | ((uint32_t)r & 0x80000000u);
  return __hiloint2double(a ? (int)hw : 0, (int)(n << 21));
}

// The bit pattern of |v| shifted left by one place (the sign shifted out),
// in an integer instruction the compiler cannot see through.  Masking the
// sign bit of a float64 pattern instead is recognised as fabs and emitted as
// an add on the FP64 pipe, which on this part costs as much as a real add.
// Shifted patterns order like the magnitudes (NaN above +inf above every
// finite value).
__device__ __forceinline__ uint64_t mag2_bits(double v) {
  uint64_t r;
  asm("shl.b64 %0, %1, 1;" : "=l"(r) : "l"((uint64_t)__double_as_longlong(v)));
  return r;
}

// |e| <= tau on bit patterns: tb is the pattern of the largest T value not
// above tau, so the comparison is exact; NaN and +-inf fail it.
template <typename T>
__device__ __forceinline__ bool within(T e, typename Fmt<T>::U tb) {
  using F = Fmt<T>;
  if constexpr (sizeof(T) == 8)
    return mag2_bits(e) <= (tb << 1);
  else
    return (F::bits(e) & F::ABS) <= tb;
}

template <typename T>
__device__ __forceinline__ bool not_finite(T v) {
  using F = Fmt<T>;
  return (F::bits(v) & F::INF) == F::INF;
}

// ---------------------------------------------------------------------------
// R8: sequency order of the 4^3 coefficients, ties by brick position.
// kPerm3.pos[r] = brick position of the r-th coded coefficient.  Built at
// compile time by ranking every position.
// ---------------------------------------------------------------------------
struct PermTable {
  int8_t pos[64];
};

__host__ __device__ constexpr int seq_key(int p) { return (p & 3) + ((p >> 2) & 3) + (p >> 4); }

__host__ __device__ constexpr PermTable make_perm(int n) {
  PermTable t{};
  for (int p = 0; p < n; ++p) {
    int rank = 0;
    for (int q = 0; q < n; ++q)
      if (seq_key(q) < seq_key(p) || (seq_key(q) == seq_key(p) && q < p)) ++rank;
    t.pos[rank] = (int8_t)p;
  }
  return t;
}

// ---------------------------------------------------------------------------
// Debug builds (-DPCZ_DEBUG) check buffer accesses: a failed check sets bit
// `site` of this translation unit's check word and skips the access (no trap,
// so a bad index cannot fault the GPU), and pc_debug_status reports the word.
// Release builds compile the checks out.  Sites: 0 the 3D chunk bit buffer,
// 1 the 3D plane tables, 2 the 1D/2D chunk bit buffer, 3 the retrieval plane
// slots and spill.
// ---------------------------------------------------------------------------
#ifdef PCZ_DEBUG
static __device__ unsigned int g_pcz_check;
#define PCZ_CHECK(cond, site) ((cond) ? true : (atomicOr(&g_pcz_check, 1u << (site)), false))
#else
#define PCZ_CHECK(cond, site) true
#endif

// This translation unit's check word (0 in release builds); reset clears it.
static inline uint32_t read_check_word(int reset) {
#ifdef PCZ_DEBUG
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_pcz_check, sizeof(v)) != cudaSuccess) v = ~0u;
  if (reset) {
    const unsigned int z = 0;
    cudaMemcpyToSymbol(g_pcz_check, &z, sizeof(z));
  }
  return v;
#else
  (void)reset;
  return 0;
#endif
}

// ---------------------------------------------------------------------------
// Bit writes into a shared-memory bit buffer (bit b = bit b%32 of word b/32):
// OR v into bits [off, off + 64).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void or_bits(uint32_t* buf, uint32_t off, uint64_t v) {
  if (!v) return;
  uint32_t w = off >> 5, sh = off & 31;
  uint64_t lo = v << sh;
  uint32_t hi = sh ? (uint32_t)(v >> (64 - sh)) : 0u;
  if ((uint32_t)lo) atomicOr(buf + w, (uint32_t)lo);
  if ((uint32_t)(lo >> 32)) atomicOr(buf + w + 1, (uint32_t)(lo >> 32));
  if (hi) atomicOr(buf + w + 2, hi);
}

// or_bits into a buffer of cap_bits bits, checked in debug builds.
__device__ __forceinline__ void or_bits_in(uint32_t* buf, uint32_t off, uint64_t v, uint32_t cap_bits, int site) {
#ifdef PCZ_DEBUG
  if (v && !PCZ_CHECK(off + (uint32_t)(64 - __clzll((long long)v)) <= cap_bits, site)) return;
#endif
  or_bits(buf, off, v);
}

// 64 bits of a word stream starting at bit pos (bit b = bit b%64 of word
// b/64); words at or beyond nwords read as zero.
__device__ __forceinline__ uint64_t peek64(const uint64_t* __restrict__ w, uint64_t nwords, uint64_t pos) {
  uint64_t i = pos >> 6;
  uint32_t sh = (uint32_t)(pos & 63);
  uint64_t a = i < nwords ? __ldg(w + i) : 0ull;
  if (!sh) return a;
  uint64_t b = i + 1 < nwords ? __ldg(w + i + 1) : 0ull;
  return (a >> sh) | (b << (64 - sh));
}

// The largest 64-bit value over the lanes of `mask` (every lane of it calls):
// the largest high word, then the largest low word among the lanes that hold
// it -- two warp reductions (redux) instead of a shuffle ladder.
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned mask, unsigned long long v) {
  const unsigned hi = __reduce_max_sync(mask, (unsigned)(v >> 32));
  const unsigned lo = __reduce_max_sync(mask, (unsigned)(v >> 32) == hi ? (unsigned)v : 0u);
  return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t low_mask64(int n) { return n >= 64 ? ~0ull : ((1ull << n) - 1); }

// ---------------------------------------------------------------------------
// 32x32 bit-matrix transpose across a warp: lane l holds row l; afterwards
// lane l holds column l (bit r = bit l of row r).  Five exchange stages with
// the lane l ^ k, k = 16, 8, 4, 2, 1: a lane keeps the k-bit groups of its
// word on its own side (low groups when bit k of l is 0) and takes the
// partner's groups of the other side, shifted across by k.  Stages 16 and 8
// move whole bytes, so one byte permute does the shift and the merge; stages
// 4, 2 and 1 use a rotation (the bits it wraps around land in the kept
// groups and are masked off) and one logic op.  keep[] holds this lane's byte
// selectors for stages 16 and 8 and its kept-bit masks for stages 4, 2, 1,
// from transpose_masks().
// ---------------------------------------------------------------------------
__device__ __forceinline__ void transpose_masks(int lane, uint32_t keep[5]) {
  keep[0] = (lane & 16) ? 0x3276u : 0x5410u;  // partner's high half down / own low half kept
  keep[1] = (lane & 8) ? 0x3715u : 0x6240u;   // likewise for the bytes of each half
  const uint32_t lo[3] = {0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const int k = 4 >> st;
    keep[2 + st] = (lane & k) ? ~lo[st] : lo[st];
  }
}

__device__ __forceinline__ uint32_t transpose32(uint32_t a, int lane, const uint32_t keep[5]) {
  a = __byte_perm(a, __shfl_xor_sync(0xffffffffu, a, 16), keep[0]);
  a = __byte_perm(a, __shfl_xor_sync(0xffffffffu, a, 8), keep[1]);
#pragma unroll
  for (int st = 0; st < 3; ++st) {
    const int k = 4 >> st;
    const uint32_t b = __shfl_xor_sync(0xffffffffu, a, k);
    // rotate right by k (partner's high groups down) or by 32 - k (low groups up)
    const uint32_t moved = __funnelshift_r(b, b, (uint32_t)(2 * (lane & k) - k));
    a = (a & keep[2 + st]) | (moved & ~keep[2 + st]);
  }
  return a;
}

// Index of brick element (x, y, z) of the warp's half h in the shared brick
// buffer (two bricks, 128 elements).  The rotations make every lifting pass
// (16 lanes of a brick reading one line position each) and the x-line
// accesses free of bank conflicts for 4- and 8-byte elements.
template <typename T>
__device__ __forceinline__ int sidx(int x, int y, int z, int h) {
  if constexpr (sizeof(T) == 8)
    return 64 * h + 16 * z + 4 * ((y + z) & 3) + ((x + z) & 3);
  else
    return 32 * z + 16 * h + 4 * ((y + z) & 3) + ((x + z) & 3);
}

// One x-line of a brick (4 consecutive values) between registers and memory:
// a single 16-byte access per 16 bytes when the line is whole and aligned
// (fewer transactions, which matters most when the memory is on the host side
// of the C2C link), element by element otherwise.
template <typename T>
__device__ __forceinline__ void store_line(T* dst, const T* v, const bool* ok) {
  if (ok[0] && ok[1] && ok[2] && ok[3] && ((uintptr_t)dst & 15) == 0) {
    if constexpr (sizeof(T) == 4) {
      *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
      reinterpret_cast<double2*>(dst)[0] = make_double2(v[0], v[1]);
      reinterpret_cast<double2*>(dst)[1] = make_double2(v[2], v[3]);
    }
    return;
  }
#pragma unroll
  for (int m = 0; m < 4; ++m)
    if (ok[m]) dst[m] = v[m];
}

// Loads the line's first nv (1..4) values; lanes past them repeat the last
// (R4 edge replication along x).
template <typename T>
__device__ __forceinline__ void load_line(const T* src, int nv, T* v) {
  if (nv == 4 && ((uintptr_t)src & 15) == 0) {
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
  for (int m = 0; m < 4; ++m) v[m] = src[min(m, nv - 1)];
}

// Sequential bit reader over a word stream with the two current words in
// registers: one load per 64 bits consumed.  Positions must not decrease.
struct BitReader {
  const uint64_t* __restrict__ w;
  uint64_t nw, wi, a, b;
  __device__ __forceinline__ uint64_t ld(uint64_t i) const { return i < nw ? __ldg(w + i) : 0ull; }
  __device__ __forceinline__ void init(const uint64_t* words, uint64_t nwords, uint64_t pos) {
    w = words;
    nw = nwords;
    wi = pos >> 6;
    a = ld(wi);
    b = ld(wi + 1);
  }
  __device__ __forceinline__ uint64_t peek(uint64_t pos) {
    const uint64_t i = pos >> 6;
    if (i != wi) {
      if (i == wi + 1) {
        a = b;
        b = ld(i + 1);
      } else {
        a = ld(i);
        b = ld(i + 1);
      }
      wi = i;
    }
    const uint32_t sh = (uint32_t)(pos & 63);
    return sh ? (a >> sh) | (b << (64 - sh)) : a;
  }
};

// Bits emitted for one plane (R11) given its plane word W (bit r = bit of the
// r-th coded coefficient) and n coefficients already significant:
// n verbatim bits, then (if n < N) one test bit per newly significant
// coefficient, the run of coefficient bits up to and including it, and a
// closing 0 test bit unless the last coefficient became significant.
template <int N>
__device__ __forceinline__ int plane_len(uint64_t W, int n) {
  if (n >= N) return n;
  uint64_t rest = n >= 64 ? 0ull : (W >> n);
  if (!rest) return n + 1;
  int hi = 64 - __clzll((long long)W);  // one past the highest set position
  int m = __popcll((long long)rest);
  return n + m + (hi - n) + (hi < N ? 1 : 0);
}

}  // namespace pcz
