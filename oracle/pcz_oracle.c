/*
 * pcz_oracle.c -- plain CPU oracle of the multi-component progressive-precision
 * method of Magri & Lindstrom, "A General Framework for Progressive Data
 * Compression and Retrieval" (Sec. 4: Algorithm 1 = construction, Algorithm 2 =
 * reconstruction, Eq. 1 = error bound), with the project-defined "PCZ" block
 * coder plugged in as the compressor C and decompressor D.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle_pcz.so, which
 * only the tests, __graft_entry__.smoke() and the CPU-baseline leg of bench.py
 * load.  The product library (CUDA) never links, includes or calls it, and it
 * shares no source, header, table or helper with the CUDA path.
 *
 * It is written to be read against the paper, not to be fast: one brick at a
 * time, one bit at a time, values of the field type T held in doubles (every
 * float is exactly a double) with every arithmetic step rounded to T.
 *
 * What the paper fixes (and this file follows step by step):
 *   - Algorithm 1: x~ <- 0; for i = 1..n: e <- x - x~; y_i <- C(e, tau_i);
 *     x_i <- D(y_i); x~ <- x~ + x_i.  Sums in the precision of x (Sec. 3).
 *   - Algorithm 2: x~ <- 0; for i = 1..m: x~ <- x~ + D(y_i); continuing the loop
 *     later refines an existing x~ (Sec. 4.2).
 *   - Eq. 1: ||x - x~_i||_inf <= tau_i, which may fail by O(eps) in floating
 *     point (Sec. 4.3).  The computed tolerance of component i (Sec. 4.3:
 *     tau_i <- ||x - x~_i||_inf, kept as metadata) is recorded too.
 *   - zfp-style coding of single d-dimensional blocks of 4^d values with one
 *     exponent per block and component (Sec. 4.4, Sec. 6.1) and group-tested
 *     bit planes (Sec. 2).
 * What the paper leaves open is fixed by project rules R1..R15; each is stated
 * where it is implemented below.
 *
 * Every function here is pinned by a test under tests/ against something other
 * than itself (library routines, closed forms, hand-built streams, brute force,
 * the Eq. 1 invariant evaluated with numpy).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OC_F32 1
#define OC_F64 2
#define OC_CHUNK 32 /* bricks per index chunk (R15) */
#define OC_MAXN 64  /* coefficients per brick, 4^3 */
#define OC_MAXC 64  /* components */

enum { MODE_ZERO = 0, MODE_CODED = 1, MODE_RAW = 2 };
enum { ST_ZERO = 0, ST_CODED = 1, ST_RAW = 2, ST_ESC = 3, ST_VIOL = 4, ST_N = 5 };

/* ------------------------------------------------------------------------ */
/* Coder parameters for a field type T and dimensionality d.                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  int dtype; /* OC_F32 or OC_F64 */
  int P;     /* bits of T = bits of the integer coefficients (32 / 64) */
  int mant;  /* significand bits of T, hidden bit included (24 / 53) */
  int emin;  /* frexp exponent of the smallest normal T (-125 / -1021) */
  int emaxT; /* frexp exponent of the largest finite T (128 / 1024) */
  int ebits; /* width of the stored block exponent (8 / 11) */
  int ebias; /* stored block exponent = emax + ebias (126 / 1022) */
  int d, N;  /* dimensionality and coefficients per brick (4^d) */
  int G;     /* headroom bits for the forward transform's growth: 2d (R6) */
  int Q;     /* quantisation bits: P - 2 - G (R6) */
  int c;     /* guard planes for the inverse transform's gain (R10) */
} coder;

static coder make_coder(int dtype, int d) {
  coder k;
  k.dtype = dtype;
  if (dtype == OC_F32) {
    k.P = 32; k.mant = 24; k.emin = -125; k.emaxT = 128; k.ebits = 8; k.ebias = 126;
  } else {
    k.P = 64; k.mant = 53; k.emin = -1021; k.emaxT = 1024; k.ebits = 11; k.ebias = 1022;
  }
  k.d = d;
  k.N = d == 1 ? 4 : d == 2 ? 16 : 64;
  k.G = 2 * d;
  k.Q = k.P - 2 - k.G;
  /* R10: c is the smallest integer with 2^c > (2/3) * 2.75^d, the worst-case
   * L-inf error (in units of the lowest coded plane) that the inverse
   * transform makes from coefficients truncated below that plane:
   * d=1: 1.83 -> 1, d=2: 5.04 -> 3, d=3: 13.9 -> 4. */
  k.c = d == 1 ? 1 : d == 2 ? 3 : 4;
  return k;
}

/* ------------------------------------------------------------------------ */
/* Arithmetic in the field type T (Sec. 3: sums in the precision of x; R1).  */
/* ------------------------------------------------------------------------ */
static double sub_T(const coder *k, double a, double b) {
  if (k->dtype == OC_F32) {
    float r = (float)a - (float)b;
    return (double)r;
  }
  return a - b;
}

static double add_T(const coder *k, double a, double b) {
  if (k->dtype == OC_F32) {
    float r = (float)a + (float)b;
    return (double)r;
  }
  return a + b;
}

static uint64_t bits_of_T(const coder *k, double v) {
  if (k->dtype == OC_F32) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
  }
  uint64_t u;
  memcpy(&u, &v, 8);
  return u;
}

static double T_of_bits(const coder *k, uint64_t u) {
  if (k->dtype == OC_F32) {
    uint32_t w = (uint32_t)u;
    float f;
    memcpy(&f, &w, 4);
    return (double)f;
  }
  double v;
  memcpy(&v, &u, 8);
  return v;
}

/* ------------------------------------------------------------------------ */
/* P-bit two's-complement integers, kept sign-extended in int64_t.           */
/* Sums wrap modulo 2^P, so no input can overflow a C integer.               */
/* ------------------------------------------------------------------------ */
static int64_t wrapP(int P, uint64_t v) {
  if (P == 64) return (int64_t)v;
  return (int64_t)(int32_t)(uint32_t)v;
}
static int64_t addw(int P, int64_t a, int64_t b) { return wrapP(P, (uint64_t)a + (uint64_t)b); }
static int64_t subw(int P, int64_t a, int64_t b) { return wrapP(P, (uint64_t)a - (uint64_t)b); }
/* floor(a / 2), i.e. an arithmetic shift right by one */
static int64_t half(int64_t a) { return (a - (a & 1)) / 2; }
static uint64_t maskP(int P) { return P == 64 ? ~0ull : ((1ull << P) - 1); }

/* ------------------------------------------------------------------------ */
/* R7: exactly invertible integer lifting on a 4-vector (a, b, c, d):        */
/* two levels of the integer Haar (S) transform followed by two predict       */
/* steps that cancel linear trends.  Output order (s0, d0, e1, e2):          */
/*   s0 = floor of the mean, d0 = coarse slope, e1, e2 = curvature terms.     */
/* Every step is u += f(v) or u -= f(v), so the inverse replays the steps    */
/* backwards with the opposite sign and is exact.                            */
/* ------------------------------------------------------------------------ */
void oc_lift_fwd4(int64_t *v, int stride, int P) {
  int64_t a = v[0], b = v[stride], c = v[2 * stride], d = v[3 * stride];
  int64_t d1 = subw(P, b, a), s1 = addw(P, a, half(d1)); /* s1 = floor((a+b)/2) */
  int64_t d2 = subw(P, d, c), s2 = addw(P, c, half(d2)); /* s2 = floor((c+d)/2) */
  int64_t d0 = subw(P, s2, s1), s0 = addw(P, s1, half(d0));
  int64_t e2 = subw(P, d2, d1);       /* second difference: 0 on a linear ramp */
  int64_t e1 = subw(P, d1, half(d0)); /* fine slope minus half the coarse slope */
  v[0] = s0;
  v[stride] = d0;
  v[2 * stride] = e1;
  v[3 * stride] = e2;
}

void oc_lift_inv4(int64_t *v, int stride, int P) {
  int64_t s0 = v[0], d0 = v[stride], e1 = v[2 * stride], e2 = v[3 * stride];
  int64_t d1 = addw(P, e1, half(d0));
  int64_t d2 = addw(P, e2, d1);
  int64_t s1 = subw(P, s0, half(d0));
  int64_t s2 = addw(P, s1, d0);
  int64_t a = subw(P, s1, half(d1)), b = addw(P, a, d1);
  int64_t c = subw(P, s2, half(d2)), d = addw(P, c, d2);
  v[0] = a;
  v[stride] = b;
  v[2 * stride] = c;
  v[3 * stride] = d;
}

/* Separable transform of a 4^d brick in brick order (i + 4j + 16l, i along x):
 * forward along x, then y, then z; inverse along z, then y, then x. */
void oc_lift_fwd_block(int64_t *v, int d, int P) {
  for (int l = 0; l < (d > 2 ? 4 : 1); l++)
    for (int j = 0; j < (d > 1 ? 4 : 1); j++) oc_lift_fwd4(v + 4 * j + 16 * l, 1, P);
  if (d > 1)
    for (int l = 0; l < (d > 2 ? 4 : 1); l++)
      for (int i = 0; i < 4; i++) oc_lift_fwd4(v + i + 16 * l, 4, P);
  if (d > 2)
    for (int j = 0; j < 4; j++)
      for (int i = 0; i < 4; i++) oc_lift_fwd4(v + i + 4 * j, 16, P);
}

void oc_lift_inv_block(int64_t *v, int d, int P) {
  if (d > 2)
    for (int j = 0; j < 4; j++)
      for (int i = 0; i < 4; i++) oc_lift_inv4(v + i + 4 * j, 16, P);
  if (d > 1)
    for (int l = 0; l < (d > 2 ? 4 : 1); l++)
      for (int i = 0; i < 4; i++) oc_lift_inv4(v + i + 16 * l, 4, P);
  for (int l = 0; l < (d > 2 ? 4 : 1); l++)
    for (int j = 0; j < (d > 1 ? 4 : 1); j++) oc_lift_inv4(v + 4 * j + 16 * l, 1, P);
}

/* R8: coefficients are coded in order of total sequency i + j + l, ties broken
 * by brick position.  perm[r] = brick position of the r-th coded coefficient.
 * Built by a plain insertion sort. */
void oc_perm(int d, int *perm) {
  int N = d == 1 ? 4 : d == 2 ? 16 : 64;
  int key[OC_MAXN];
  for (int pos = 0; pos < N; pos++) {
    int i = pos & 3, j = (pos >> 2) & 3, l = pos >> 4;
    key[pos] = i + j + l;
    perm[pos] = pos;
  }
  for (int a = 1; a < N; a++) {
    int cur = perm[a], b = a;
    while (b > 0 && (key[perm[b - 1]] > key[cur] ||
                     (key[perm[b - 1]] == key[cur] && perm[b - 1] > cur))) {
      perm[b] = perm[b - 1];
      b--;
    }
    perm[b] = cur;
  }
}

/* R9: negabinary.  u = (q + M) xor M with M = 0xAA..A, modulo 2^P, so that
 * q = sum_b u_b (-2)^b; the inverse is q = (u xor M) - M. */
#define NB_M 0xAAAAAAAAAAAAAAAAull
uint64_t oc_nb_fwd(int64_t q, int P) { return (((uint64_t)q + NB_M) ^ NB_M) & maskP(P); }
int64_t oc_nb_inv(uint64_t u, int P) {
  uint64_t m = NB_M & maskP(P);
  return wrapP(P, (u ^ m) - m);
}

/* ------------------------------------------------------------------------ */
/* Bit strings: bit b of a string is bit (b mod 64) of word b/64 (R12).      */
/* ------------------------------------------------------------------------ */
typedef struct {
  uint64_t *w;
  int64_t n;   /* bits written */
  int64_t cap; /* words allocated */
} bits_t;

static void put_bit(bits_t *s, int bit) {
  if ((s->n >> 6) >= s->cap) {
    int64_t ncap = s->cap ? 2 * s->cap : 8;
    s->w = (uint64_t *)realloc(s->w, (size_t)ncap * 8);
    memset(s->w + s->cap, 0, (size_t)(ncap - s->cap) * 8);
    s->cap = ncap;
  }
  if (bit) s->w[s->n >> 6] |= 1ull << (s->n & 63);
  s->n++;
}

/* a multi-bit field is written least significant bit first */
static void put_bits(bits_t *s, uint64_t v, int width) {
  for (int b = 0; b < width; b++) put_bit(s, (int)((v >> b) & 1));
}

static void append_bits(bits_t *dst, const bits_t *src) {
  for (int64_t b = 0; b < src->n; b++) put_bit(dst, (int)((src->w[b >> 6] >> (b & 63)) & 1));
}

typedef struct {
  const uint64_t *w;
  int64_t pos, end;
  int err; /* set when a read goes past end */
} reader_t;

static int get_bit(reader_t *r) {
  if (r->pos >= r->end) {
    r->err = 1;
    return 0;
  }
  int bit = (int)((r->w[r->pos >> 6] >> (r->pos & 63)) & 1);
  r->pos++;
  return bit;
}

static uint64_t get_bits(reader_t *r, int width) {
  uint64_t v = 0;
  for (int b = 0; b < width; b++) v |= (uint64_t)get_bit(r) << b;
  return v;
}

/* ------------------------------------------------------------------------ */
/* R11: embedded group-tested bit-plane coding of N unsigned P-bit words,    */
/* planes P-1 down to pmin.  n counts the coefficients found significant so  */
/* far.  Per plane: (i) bit p of coefficients 0..n-1, verbatim; (ii) while   */
/* n < N: a test bit "some coefficient n..N-1 has bit p set"; on 0 the plane */
/* ends, on 1 the bits of coefficients n, n+1, ... follow up to and          */
/* including the first 1, and n moves past it.  No bit is ever implied.      */
/* ------------------------------------------------------------------------ */
static void encode_planes(const uint64_t *u, int N, int P, int pmin, bits_t *out) {
  int n = 0;
  for (int p = P - 1; p >= pmin; p--) {
    for (int k = 0; k < n; k++) put_bit(out, (int)((u[k] >> p) & 1));
    while (n < N) {
      int any = 0;
      for (int k = n; k < N; k++)
        if ((u[k] >> p) & 1) any = 1;
      put_bit(out, any);
      if (!any) break;
      for (;;) {
        int bit = (int)((u[n] >> p) & 1);
        put_bit(out, bit);
        n++;
        if (bit) break;
      }
    }
  }
}

/* returns 0, or -1 when the bits cannot have come from encode_planes */
static int decode_planes(reader_t *r, uint64_t *u, int N, int P, int pmin) {
  for (int k = 0; k < N; k++) u[k] = 0;
  int n = 0;
  for (int p = P - 1; p >= pmin; p--) {
    for (int k = 0; k < n; k++) u[k] |= (uint64_t)get_bit(r) << p;
    while (n < N) {
      if (!get_bit(r)) break;
      for (;;) {
        if (n >= N) return -1; /* a test bit promised a 1 that never came */
        int bit = get_bit(r);
        u[n] |= (uint64_t)bit << p;
        n++;
        if (bit) break;
      }
    }
    if (r->err) return -1;
  }
  return r->err ? -1 : 0;
}

/* exported forms for the tests: out must hold maxbits bits; returns the bit
 * count, or -1 when it would not fit */
int64_t oc_encode_planes(const uint64_t *u, int N, int P, int pmin, uint64_t *out, int64_t maxbits) {
  bits_t s = {0, 0, 0};
  encode_planes(u, N, P, pmin, &s);
  int64_t n = s.n;
  if (n > maxbits) {
    free(s.w);
    return -1;
  }
  memset(out, 0, (size_t)((maxbits + 63) / 64) * 8);
  if (n) memcpy(out, s.w, (size_t)((n + 63) / 64) * 8);
  free(s.w);
  return n;
}

/* returns the bits consumed, or -1 on a malformed string */
int64_t oc_decode_planes(const uint64_t *in, int64_t nbits, int N, int P, int pmin, uint64_t *u) {
  reader_t r = {in, 0, nbits, 0};
  if (decode_planes(&r, u, N, P, pmin)) return -1;
  return r.pos;
}

/* ------------------------------------------------------------------------ */
/* R6: block-floating-point alignment.                                       */
/* ------------------------------------------------------------------------ */
/* frexp exponent: 2^(E-1) <= |v| < 2^E */
static int frexp_exp(double v) {
  int E;
  frexp(v, &E);
  return E;
}

/* emax = the largest frexp exponent over the nonzero values, but never below
 * that of the smallest normal T (so it fits the stored field) */
int oc_block_emax(const double *e, int count, int dtype) {
  coder k = make_coder(dtype, 3);
  int emax = k.emin;
  for (int i = 0; i < count; i++)
    if (e[i] != 0.0) {
      int E = frexp_exp(e[i]);
      if (E > emax) emax = E;
    }
  return emax;
}

/* q = sign(e) * floor(|e| * 2^s); |e| * 2^s is exact in double because it is
 * below 2^Q <= 2^60, and values below 1 floor to 0 however they round */
int64_t oc_quantize(double e, int s) {
  double v = floor(ldexp(fabs(e), s));
  return e < 0 ? -(int64_t)v : (int64_t)v;
}

/* R13: x = the T value nearest to q * 2^-s, ties to even; overflow gives
 * +-inf and subnormal results are rounded once, directly. */
double oc_dequantize(int64_t q, int s, int dtype) {
  coder k = make_coder(dtype, 3);
  if (q == 0) return 0.0;
  uint64_t a = q < 0 ? (uint64_t)0 - (uint64_t)q : (uint64_t)q;
  int nb = 0; /* bit length of a */
  while (nb < 64 && (a >> nb) != 0) nb++;
  int kx = -s;                                /* value = a * 2^kx */
  int E = nb + kx;                            /* frexp exponent of the exact value */
  int qe = (E > k.emin ? E : k.emin) - k.mant; /* exponent of the result's last place */
  int sh = qe - kx;                           /* bits of a below that place */
  uint64_t r;
  if (sh <= 0) {
    r = a << (-sh);
  } else if (sh > 64) {
    r = 0; /* value below half the last place */
  } else if (sh == 64) {
    r = a > (1ull << 63) ? 1 : 0; /* a == 2^63 is the tie, rounded to the even 0 */
  } else {
    r = a >> sh;
    uint64_t rem = a - (r << sh), halfulp = 1ull << (sh - 1);
    if (rem > halfulp || (rem == halfulp && (r & 1))) r++;
  }
  double v = ldexp((double)r, qe); /* exact: r <= 2^mant; overflow gives inf */
  if (q < 0) v = -v;
  if (dtype == OC_F32) v = (double)(float)v; /* exact, or +-inf beyond FLT_MAX */
  return v;
}

/* floor(log2 tau) for a positive finite tau */
int oc_floor_log2(double tau) { return frexp_exp(tau) - 1; }

/* R2: the smallest i (1-based) with tau_i <= t; -1 when t < tau_n */
int oc_query_k(const double *tau, int n, double t) {
  for (int i = 0; i < n; i++)
    if (tau[i] <= t) return i + 1;
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Fields and bricks.  dims[0] is the fastest-varying extent; a field of    */
/* ndims < 3 has unit extents on the missing axes.  Bricks are 4^d values    */
/* in raster order of brick coordinates, bx fastest.                         */
/* ------------------------------------------------------------------------ */
typedef struct {
  coder cd;
  const void *data;
  int64_t dims[3];
  int64_t nb[3]; /* bricks per axis */
  int64_t nbricks;
} field_t;

static void make_field(field_t *f, const void *data, int dtype, int ndims, const int64_t *dims) {
  f->cd = make_coder(dtype, ndims);
  f->data = data;
  for (int a = 0; a < 3; a++) {
    f->dims[a] = a < ndims ? dims[a] : 1;
    f->nb[a] = a < ndims ? (f->dims[a] + 3) / 4 : 1;
  }
  f->nbricks = f->nb[0] * f->nb[1] * f->nb[2];
}

static double load_T(const field_t *f, int64_t idx) {
  if (f->cd.dtype == OC_F32) return (double)((const float *)f->data)[idx];
  return ((const double *)f->data)[idx];
}

/* R4: lanes outside the field take the value of the nearest in-field lane
 * along each axis (edge replication); src[k] is that lane, inf[k] is 1 for
 * in-field lanes.  Padded lanes are coded but never verified nor written. */
static void brick_lanes(const field_t *f, int64_t b, int64_t org[3], int *inf, int *src) {
  int64_t bx = b % f->nb[0], by = (b / f->nb[0]) % f->nb[1], bz = b / (f->nb[0] * f->nb[1]);
  org[0] = 4 * bx;
  org[1] = 4 * by;
  org[2] = 4 * bz;
  int d = f->cd.d;
  for (int k = 0; k < f->cd.N; k++) {
    int i = k & 3, j = d > 1 ? (k >> 2) & 3 : 0, l = d > 2 ? k >> 4 : 0;
    int64_t g[3] = {org[0] + i, org[1] + j, org[2] + l};
    int cl[3] = {i, j, l};
    inf[k] = 1;
    for (int a = 0; a < 3; a++)
      if (g[a] >= f->dims[a]) {
        inf[k] = 0;
        cl[a] = (int)(f->dims[a] - 1 - org[a]);
      }
    src[k] = cl[0] + 4 * cl[1] + 16 * cl[2];
  }
}

static int64_t lane_index(const field_t *f, const int64_t org[3], int k) {
  int64_t gx = org[0] + (k & 3), gy = org[1] + ((k >> 2) & 3), gz = org[2] + (k >> 4);
  return gx + f->dims[0] * (gy + f->dims[1] * gz);
}

/* brick values with edge replication, for the tests (out holds N doubles) */
void oc_gather_brick(const void *data, int dtype, int ndims, const int64_t *dims, int64_t b, double *out) {
  field_t f;
  make_field(&f, data, dtype, ndims, dims);
  int64_t org[3];
  int inf[OC_MAXN], src[OC_MAXN];
  brick_lanes(&f, b, org, inf, src);
  for (int k = 0; k < f.cd.N; k++) out[k] = load_T(&f, lane_index(&f, org, src[k]));
}

/* ------------------------------------------------------------------------ */
/* The PCZ block coder C and decoder D.                                      */
/* ------------------------------------------------------------------------ */

/* coefficients u (coded order) truncated below plane p, back to values:
 * inverse negabinary, inverse reorder, inverse lifting, dequantisation */
static void reconstruct(const coder *k, const int *perm, const uint64_t *u, int p, int s, double *xi) {
  int64_t q[OC_MAXN];
  uint64_t below = p >= 64 ? ~0ull : (1ull << p) - 1; /* planes not coded */
  uint64_t keep = maskP(k->P) & ~below;
  for (int r = 0; r < k->N; r++) q[perm[r]] = oc_nb_inv(u[r] & keep, k->P);
  oc_lift_inv_block(q, k->d, k->P);
  for (int pos = 0; pos < k->N; pos++) xi[pos] = oc_dequantize(q[pos], s, k->dtype);
}

/* Eq. 1 evaluated in T (R13): |fl(x - fl(x~ + x_i))| <= tau on in-field lanes */
static int verify(const coder *k, const double *x, const double *xt, const double *xi, const int *inf,
                  double tau) {
  for (int pos = 0; pos < k->N; pos++) {
    if (!inf[pos]) continue;
    double r = sub_T(k, x[pos], add_T(k, xt[pos], xi[pos]));
    if (!(fabs(r) <= tau)) return 0;
  }
  return 1;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : v > hi ? hi : v; }

/* C(e, tau): appends the block's bits to out.  x and x~ are passed so that the
 * coder can check Eq. 1 on the sum it will actually produce (R13). */
static void encode_block(const coder *k, const int *perm, const double *e, const double *x, const double *xt,
                         const int *inf, double tau, bits_t *out, int64_t *st) {
  int N = k->N;
  /* R5: a block whose residual already meets tau is a ZERO block */
  int small = 1;
  for (int pos = 0; pos < N; pos++)
    if (inf[pos] && !(fabs(e[pos]) <= tau)) small = 0;
  if (small) {
    put_bits(out, MODE_ZERO, 2);
    st[ST_ZERO]++;
    return;
  }
  int finite = 1;
  for (int pos = 0; pos < N; pos++)
    if (!isfinite(e[pos])) finite = 0;
  if (finite) {
    /* R6 */
    int emax = oc_block_emax(e, N, k->dtype);
    int s = k->Q - emax;
    int64_t q[OC_MAXN];
    for (int pos = 0; pos < N; pos++) q[pos] = oc_quantize(e[pos], s);
    /* R7, R8, R9 */
    oc_lift_fwd_block(q, k->d, k->P);
    uint64_t u[OC_MAXN];
    for (int r = 0; r < N; r++) u[r] = oc_nb_fwd(q[perm[r]], k->P);
    /* R10, R13: lowest coded plane, lowered (escalated) until Eq. 1 holds */
    int L = oc_floor_log2(tau);
    int esc = 0, p = 0, pass = 0;
    double xi[OC_MAXN];
    for (esc = 0;; esc++) {
      p = clampi(L + s - k->c - esc, 0, k->P);
      reconstruct(k, perm, u, p, s, xi);
      if (verify(k, x, xt, xi, inf, tau)) {
        pass = 1;
        break;
      }
      if (esc == 7 || p == 0) break;
    }
    if (pass) {
      bits_t planes = {0, 0, 0};
      encode_planes(u, N, k->P, p, &planes);
      int64_t lenC = 2 + 3 + k->ebits + planes.n, lenR = 2 + (int64_t)N * k->P;
      /* R14: RAW replaces a longer CODED block only if it also meets tau */
      if (!(lenC > lenR && verify(k, x, xt, e, inf, tau))) {
        put_bits(out, MODE_CODED, 2);
        put_bits(out, (uint64_t)esc, 3);
        put_bits(out, (uint64_t)(emax + k->ebias), k->ebits);
        append_bits(out, &planes);
        free(planes.w);
        st[ST_CODED]++;
        st[ST_ESC] += esc;
        return;
      }
      free(planes.w);
    }
  }
  /* RAW: the residual itself, as T bit patterns in brick order */
  put_bits(out, MODE_RAW, 2);
  for (int pos = 0; pos < N; pos++) put_bits(out, bits_of_T(k, e[pos]), k->P);
  st[ST_RAW]++;
}

/* D(y): decodes one block's bits [pos, end) of w into xi (N values).
 * Returns 0, or -1 when the bits are not a block of this format. */
static int decode_block(const coder *k, const int *perm, const uint64_t *w, int64_t pos, int64_t end,
                        double tau, double *xi) {
  reader_t r = {w, pos, end, 0};
  int mode = (int)get_bits(&r, 2);
  if (mode == MODE_ZERO) {
    for (int i = 0; i < k->N; i++) xi[i] = 0.0;
  } else if (mode == MODE_CODED) {
    int esc = (int)get_bits(&r, 3);
    int emax = (int)get_bits(&r, k->ebits) - k->ebias;
    if (r.err || emax < k->emin || emax > k->emaxT) return -1;
    int s = k->Q - emax;
    int p = clampi(oc_floor_log2(tau) + s - k->c - esc, 0, k->P);
    uint64_t u[OC_MAXN];
    if (decode_planes(&r, u, k->N, k->P, p)) return -1;
    reconstruct(k, perm, u, p, s, xi);
  } else if (mode == MODE_RAW) {
    for (int i = 0; i < k->N; i++) xi[i] = T_of_bits(k, get_bits(&r, k->P));
  } else {
    return -1;
  }
  if (r.err || r.pos != end) return -1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1 on one brick.                                                 */
/* ------------------------------------------------------------------------ */
/* y[i] receives the bits of component i+1; xt (N values) the final partial
 * sum x~_n (in-field lanes); st[i] the per-component counters.
 * Returns 0, or -1 if D(y_i) ever failed to read back C's output. */
static int code_brick(const field_t *f, const int *perm, int64_t b, const double *tau, int n, bits_t *y,
                      double *xt, int64_t (*st)[ST_N], double *maxerr) {
  const coder *k = &f->cd;
  double x[OC_MAXN], e[OC_MAXN], xi[OC_MAXN];
  int inf[OC_MAXN], src[OC_MAXN];
  int64_t org[3];
  brick_lanes(f, b, org, inf, src);
  for (int pos = 0; pos < k->N; pos++) x[pos] = load_T(f, lane_index(f, org, src[pos]));
  for (int pos = 0; pos < k->N; pos++) xt[pos] = 0.0; /* Algorithm 1 starts from x~ = 0 */
  for (int i = 0; i < n; i++) {                      /* one component per tau_i */
    for (int pos = 0; pos < k->N; pos++)             /* residual e = x - x~ */
      if (inf[pos]) e[pos] = sub_T(k, x[pos], xt[pos]);
    for (int pos = 0; pos < k->N; pos++)
      if (!inf[pos]) e[pos] = e[src[pos]];
    int64_t start = y[i].n;
    encode_block(k, perm, e, x, xt, inf, tau[i], &y[i], st[i]); /* y_i = C(e, tau_i) */
    if (decode_block(k, perm, y[i].w, start, y[i].n, tau[i], xi)) return -1; /* x_i = D(y_i) */
    for (int pos = 0; pos < k->N; pos++) /* x~ = x~ + x_i */
      if (inf[pos]) xt[pos] = add_T(k, xt[pos], xi[pos]);
    for (int pos = 0; pos < k->N; pos++) { /* Eq. 1, counted where it fails */
      if (!inf[pos]) continue;
      double r = fabs(sub_T(k, x[pos], xt[pos]));
      if (!(r <= tau[i])) st[i][ST_VIOL]++;
      if (maxerr && r > maxerr[i]) maxerr[i] = r; /* Sec. 4.3: the computed tolerance */
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Component streams (R15).  Per component: bricks concatenated in raster    */
/* order; every chunk of 32 bricks starts on a 64-bit word; the index holds  */
/* the chunk's first word (u64) and each brick's bit length (u16).           */
/* ------------------------------------------------------------------------ */
struct oc_streams {
  field_t f;
  int ndims, n;
  double tau[OC_MAXC];
  int64_t nchunks;
  uint64_t *payload[OC_MAXC];
  int64_t nwords[OC_MAXC];
  uint64_t *chunk_word[OC_MAXC];
  uint16_t *brick_len[OC_MAXC];
  int64_t stats[OC_MAXC][ST_N];
  double measured[OC_MAXC]; /* max over the field of |fl_T(x - x~_i)| (Sec. 4.3) */
  double *xt; /* x~_n of every field value, as produced by Algorithm 1 */
  int status; /* 0 ok, -1 a block failed to decode, -2 a brick exceeded 65535 bits */
};
typedef struct oc_streams oc_streams;

static int tau_ok(const double *tau, int n) {
  for (int i = 0; i < n; i++) {
    if (!(tau[i] > 0) || !isfinite(tau[i])) return 0;
    if (i && !(tau[i] < tau[i - 1])) return 0;
  }
  return 1;
}

/* Algorithm 1 over a whole field.  Returns NULL on bad arguments or a
 * non-finite input value (Sec. 6.1: NaN and infinities are not handled). */
oc_streams *oc_compress(const void *data, int dtype, int ndims, const int64_t *dims, const double *tau, int n,
                        int nthreads) {
  if ((dtype != OC_F32 && dtype != OC_F64) || ndims < 1 || ndims > 3 || n < 1 || n > OC_MAXC) return NULL;
  if (!tau_ok(tau, n)) return NULL;
  for (int a = 0; a < ndims; a++)
    if (dims[a] < 1) return NULL;
  oc_streams *s = (oc_streams *)calloc(1, sizeof(oc_streams));
  make_field(&s->f, data, dtype, ndims, dims);
  int64_t count = s->f.dims[0] * s->f.dims[1] * s->f.dims[2];
  for (int64_t i = 0; i < count; i++)
    if (!isfinite(load_T(&s->f, i))) {
      free(s);
      return NULL;
    }
  s->ndims = ndims;
  s->n = n;
  memcpy(s->tau, tau, (size_t)n * sizeof(double));
  const coder *k = &s->f.cd;
  int perm[OC_MAXN];
  oc_perm(k->d, perm);
  int64_t nb = s->f.nbricks;
  s->nchunks = (nb + OC_CHUNK - 1) / OC_CHUNK;
  s->xt = (double *)calloc((size_t)count, sizeof(double));
  for (int i = 0; i < n; i++) {
    s->chunk_word[i] = (uint64_t *)calloc((size_t)s->nchunks, 8);
    s->brick_len[i] = (uint16_t *)calloc((size_t)nb, 2);
  }
  /* chunk_bits[c * n + i]: the bits of component i+1 for the bricks of chunk c */
  bits_t *chunk_bits = (bits_t *)calloc((size_t)(s->nchunks * n), sizeof(bits_t));
  int64_t(*cst)[OC_MAXC][ST_N] = calloc((size_t)s->nchunks, sizeof(*cst));
  double(*cme)[OC_MAXC] = calloc((size_t)s->nchunks, sizeof(*cme));
  int bad = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(| : bad)
#endif
  for (int64_t c = 0; c < s->nchunks; c++) {
    double xt[OC_MAXN];
    bits_t one[OC_MAXC];
    for (int64_t b = c * OC_CHUNK; b < nb && b < (c + 1) * OC_CHUNK; b++) {
      memset(one, 0, sizeof(bits_t) * (size_t)n);
      if (code_brick(&s->f, perm, b, tau, n, one, xt, cst[c], cme[c])) bad |= 1;
      for (int i = 0; i < n; i++) {
        if (one[i].n > 65535) bad |= 2;
        s->brick_len[i][b] = (uint16_t)one[i].n;
        append_bits(&chunk_bits[c * n + i], &one[i]);
        free(one[i].w);
      }
      int inf[OC_MAXN], src[OC_MAXN];
      int64_t org[3];
      brick_lanes(&s->f, b, org, inf, src);
      for (int pos = 0; pos < k->N; pos++)
        if (inf[pos]) s->xt[lane_index(&s->f, org, pos)] = xt[pos];
    }
  }
  s->status = (bad & 1) ? -1 : (bad & 2) ? -2 : 0;
  for (int64_t c = 0; c < s->nchunks; c++)
    for (int i = 0; i < n; i++)
      for (int t = 0; t < ST_N; t++) s->stats[i][t] += cst[c][i][t];
  for (int64_t c = 0; c < s->nchunks; c++)
    for (int i = 0; i < n; i++)
      if (cme[c][i] > s->measured[i]) s->measured[i] = cme[c][i];
  free(cst);
  free(cme);
  for (int i = 0; i < n; i++) {
    int64_t words = 0;
    for (int64_t c = 0; c < s->nchunks; c++) {
      s->chunk_word[i][c] = (uint64_t)words;
      words += (chunk_bits[c * n + i].n + 63) / 64;
    }
    s->nwords[i] = words;
    s->payload[i] = (uint64_t *)calloc((size_t)(words ? words : 1), 8);
    for (int64_t c = 0; c < s->nchunks; c++) {
      bits_t *cb = &chunk_bits[c * n + i];
      if (cb->n) memcpy(s->payload[i] + s->chunk_word[i][c], cb->w, (size_t)((cb->n + 63) / 64) * 8);
      free(cb->w);
    }
  }
  free(chunk_bits);
  return s;
}

int oc_status(const oc_streams *s) { return s->status; }
int oc_n(const oc_streams *s) { return s->n; }
int64_t oc_nbricks(const oc_streams *s) { return s->f.nbricks; }
int64_t oc_nchunks(const oc_streams *s) { return s->nchunks; }
int64_t oc_payload_words(const oc_streams *s, int i) { return s->nwords[i]; }
const uint64_t *oc_payload(const oc_streams *s, int i) { return s->payload[i]; }
const uint64_t *oc_chunk_word(const oc_streams *s, int i) { return s->chunk_word[i]; }
const uint16_t *oc_brick_len(const oc_streams *s, int i) { return s->brick_len[i]; }
double oc_measured(const oc_streams *s, int i) { return s->measured[i]; }
void oc_stats(const oc_streams *s, int i, int64_t *out) {
  for (int t = 0; t < ST_N; t++) out[t] = s->stats[i][t];
}

/* x~_n from Algorithm 1, written in T */
void oc_final_xt(const oc_streams *s, void *out) {
  int64_t count = s->f.dims[0] * s->f.dims[1] * s->f.dims[2];
  for (int64_t i = 0; i < count; i++) {
    if (s->f.cd.dtype == OC_F32)
      ((float *)out)[i] = (float)s->xt[i];
    else
      ((double *)out)[i] = s->xt[i];
  }
}

/* first bit of brick b in the payload of component i */
static int64_t brick_bit(const oc_streams *s, int i, int64_t b) {
  int64_t c = b / OC_CHUNK, bit = (int64_t)s->chunk_word[i][c] * 64;
  for (int64_t t = c * OC_CHUNK; t < b; t++) bit += s->brick_len[i][t];
  return bit;
}

/* Algorithm 2, continued from k0 to k components, on the half-open box
 * [lo, hi) (element units, lo/hi NULL = whole field).  inout is the box in T,
 * x fastest; it is read when k0 > 0 (the partial sum x~_k0) and always
 * written.  Returns 0, or -1 on bad arguments or an unreadable block. */
int oc_retrieve(const oc_streams *s, int k0, int k, const int64_t *lo_in, const int64_t *hi_in, void *inout) {
  const field_t *f = &s->f;
  const coder *cd = &f->cd;
  if (k0 < 0 || k < k0 || k > s->n) return -1;
  int64_t lo[3], hi[3], ext[3];
  for (int a = 0; a < 3; a++) {
    lo[a] = lo_in ? lo_in[a] : 0;
    hi[a] = hi_in ? hi_in[a] : f->dims[a];
    if (lo[a] < 0 || hi[a] > f->dims[a] || lo[a] >= hi[a]) return -1;
    ext[a] = hi[a] - lo[a];
  }
  int perm[OC_MAXN];
  oc_perm(cd->d, perm);
  int bad = 0;
  for (int64_t b = 0; b < f->nbricks; b++) {
    int inf[OC_MAXN], src[OC_MAXN];
    int64_t org[3];
    brick_lanes(f, b, org, inf, src);
    int inbox[OC_MAXN], any = 0;
    int64_t oidx[OC_MAXN];
    for (int pos = 0; pos < cd->N; pos++) {
      int64_t g[3] = {org[0] + (pos & 3), org[1] + ((pos >> 2) & 3), org[2] + (pos >> 4)};
      inbox[pos] = inf[pos];
      for (int a = 0; a < 3; a++)
        if (g[a] < lo[a] || g[a] >= hi[a]) inbox[pos] = 0;
      oidx[pos] = (g[0] - lo[0]) + ext[0] * ((g[1] - lo[1]) + ext[1] * (g[2] - lo[2]));
      any |= inbox[pos];
    }
    if (!any) continue;
    double xt[OC_MAXN], xi[OC_MAXN];
    for (int pos = 0; pos < cd->N; pos++) { /* x~ = 0, or the partial sum so far */
      xt[pos] = 0.0;
      if (k0 > 0 && inbox[pos])
        xt[pos] = cd->dtype == OC_F32 ? (double)((float *)inout)[oidx[pos]] : ((double *)inout)[oidx[pos]];
    }
    for (int j = k0; j < k; j++) { /* Algorithm 2: x~ += D(y_j) */
      int64_t start = brick_bit(s, j, b);
      if (decode_block(cd, perm, s->payload[j], start, start + s->brick_len[j][b], s->tau[j], xi)) {
        bad = 1;
        break;
      }
      for (int pos = 0; pos < cd->N; pos++)
        if (inbox[pos]) xt[pos] = add_T(cd, xt[pos], xi[pos]);
    }
    for (int pos = 0; pos < cd->N; pos++)
      if (inbox[pos]) {
        if (cd->dtype == OC_F32)
          ((float *)inout)[oidx[pos]] = (float)xt[pos];
        else
          ((double *)inout)[oidx[pos]] = xt[pos];
      }
  }
  return bad ? -1 : 0;
}

void oc_free(oc_streams *s) {
  if (!s) return;
  for (int i = 0; i < s->n; i++) {
    free(s->payload[i]);
    free(s->chunk_word[i]);
    free(s->brick_len[i]);
  }
  free(s->xt);
  free(s);
}

/* ------------------------------------------------------------------------ */
/* One brick at a time, for sampled checks on fields too large for          */
/* oc_compress: codes brick b of the field for components 1..n.             */
/* bits holds n * maxwords words (component i at i * maxwords), nbits[i]     */
/* receives each bit length, xt (N values, brick order) the partial sum      */
/* x~_n on in-field lanes, st (n * 5) the counters.                          */
/* Returns 0, -1 on a decode failure, -2 if a string exceeds maxwords.       */
/* ------------------------------------------------------------------------ */
int oc_code_brick(const void *data, int dtype, int ndims, const int64_t *dims, const double *tau, int n,
                  int64_t b, uint64_t *bits, int64_t maxwords, int64_t *nbits, double *xt, int64_t *st) {
  field_t f;
  make_field(&f, data, dtype, ndims, dims);
  if (b < 0 || b >= f.nbricks || n < 1 || n > OC_MAXC) return -1;
  int perm[OC_MAXN];
  oc_perm(f.cd.d, perm);
  bits_t y[OC_MAXC];
  memset(y, 0, sizeof(y));
  int64_t(*stv)[ST_N] = calloc((size_t)n, sizeof(*stv));
  int rc = code_brick(&f, perm, b, tau, n, y, xt, stv, NULL);
  for (int i = 0; i < n; i++) {
    nbits[i] = y[i].n;
    if ((y[i].n + 63) / 64 > maxwords) rc = rc ? rc : -2;
    memset(bits + i * maxwords, 0, (size_t)maxwords * 8);
    if (y[i].n && (y[i].n + 63) / 64 <= maxwords) memcpy(bits + i * maxwords, y[i].w, (size_t)((y[i].n + 63) / 64) * 8);
    free(y[i].w);
    for (int t = 0; t < ST_N; t++) st[i * ST_N + t] = stv[i][t];
  }
  free(stv);
  return rc;
}

/* Algorithm 2 on one brick from bit strings laid out as by oc_code_brick:
 * sums D of components 1..k into xt (N values, all lanes).  tau gives each
 * component's tolerance.  Returns 0 or -1. */
int oc_decode_brick(int dtype, int d, const double *tau, int k, const uint64_t *bits, int64_t maxwords,
                    const int64_t *nbits, double *xt) {
  coder cd = make_coder(dtype, d);
  int perm[OC_MAXN];
  oc_perm(d, perm);
  double xi[OC_MAXN];
  for (int pos = 0; pos < cd.N; pos++) xt[pos] = 0.0;
  for (int j = 0; j < k; j++) {
    if (decode_block(&cd, perm, bits + j * maxwords, 0, nbits[j], tau[j], xi)) return -1;
    for (int pos = 0; pos < cd.N; pos++) xt[pos] = add_T(&cd, xt[pos], xi[pos]);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Sec. 3 special case: Algorithm 1 with C o D = rounding to float32 on a    */
/* double input gives the float-float (double-single) expansion.             */
/* comps[i * count + v] receives x_{i+1} of value v.                         */
/* ------------------------------------------------------------------------ */
void oc_scalar_fl32(const double *x, int64_t count, int n, double *comps) {
  for (int64_t v = 0; v < count; v++) {
    double xt = 0.0;               /* x~ = 0 */
    for (int i = 0; i < n; i++) {  /* components */
      double e = x[v] - xt;        /* residual */
      float y = (float)e;          /* C = round to float32 */
      double xi = (double)y;       /* D = widen back */
      xt = xt + xi;                /* partial sum */
      comps[i * count + v] = xi;
    }
  }
}

int oc_version(void) { return 1; }
