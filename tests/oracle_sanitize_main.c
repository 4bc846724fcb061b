/*
 * Driver for the sanitizer build of the CPU oracle (test infrastructure):
 * tests/test_oracle_sanitize.py compiles it together with oracle/pcz_oracle.c
 * under AddressSanitizer and UndefinedBehaviorSanitizer and runs it.  It codes
 * and decodes small 1D/2D/3D fields of both types (ragged edges, one-brick
 * fields, sub-boxes, incremental refinement) and the single-brick entry
 * points, and exits non-zero if any call reports a failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef struct oc_streams oc_streams;
oc_streams *oc_compress(const void *data, int dtype, int ndims, const int64_t *dims, const double *tau, int n,
                        int nthreads);
int oc_status(const oc_streams *s);
int oc_retrieve(const oc_streams *s, int k0, int k, const int64_t *lo, const int64_t *hi, void *inout);
double oc_measured(const oc_streams *s, int i);
void oc_free(oc_streams *s);
int oc_code_brick(const void *data, int dtype, int ndims, const int64_t *dims, const double *tau, int n, int64_t b,
                  uint64_t *bits, int64_t maxwords, int64_t *nbits, double *xt, int64_t *st);
int oc_decode_brick(int dtype, int d, const double *tau, int k, const uint64_t *bits, int64_t maxwords,
                    const int64_t *nbits, double *out);

static uint64_t rng = 0x9E3779B97F4A7C15ull;
static double urand(void) { /* xorshift64*, uniform in [0, 1) */
  rng ^= rng >> 12;
  rng ^= rng << 25;
  rng ^= rng >> 27;
  return (double)((rng * 0x2545F4914F6CDD1Dull) >> 11) / 9007199254740992.0;
}

static int run_field(int dtype, int ndims, const int64_t *dims, int n) {
  int64_t count = 1;
  for (int a = 0; a < ndims; a++) count *= dims[a];
  size_t esz = dtype == 1 ? 4 : 8;
  void *x = malloc((size_t)count * esz);
  double lo = 1e300, hi = -1e300;
  for (int64_t i = 0; i < count; i++) {
    double v = sin(0.37 * (double)i) + 0.05 * urand() + (i % 17 == 0 ? 3.0 : 0.0);
    if (dtype == 1) {
      ((float *)x)[i] = (float)v;
      v = (double)(float)v;
    } else {
      ((double *)x)[i] = v;
    }
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  }
  double tau[16];
  for (int i = 0; i < n; i++) tau[i] = (hi - lo + 1.0) * pow(2.0, -4.0 * (i + 1));
  oc_streams *s = oc_compress(x, dtype, ndims, dims, tau, n, 1);
  int bad = 0;
  if (!s || oc_status(s) != 0) bad = 1;
  void *out = malloc((size_t)count * esz);
  for (int k = 0; !bad && k <= n; k++) {
    if (oc_retrieve(s, 0, k, NULL, NULL, out)) bad = 2;
    if (k && !(oc_measured(s, k - 1) <= tau[k - 1])) bad = 3;
  }
  /* a sub-box, refined from k = 1 to k = n */
  int64_t blo[3] = {0, 0, 0}, bhi[3] = {1, 1, 1}, bc = 1;
  for (int a = 0; a < ndims; a++) {
    blo[a] = dims[a] / 3;
    bhi[a] = dims[a] - dims[a] / 4;
    if (bhi[a] <= blo[a]) bhi[a] = blo[a] + 1;
    bc *= bhi[a] - blo[a];
  }
  void *box = malloc((size_t)bc * esz);
  if (!bad && oc_retrieve(s, 0, 1, blo, bhi, box)) bad = 4;
  if (!bad && oc_retrieve(s, 1, n, blo, bhi, box)) bad = 5;
  /* single-brick entry points on the last brick */
  int64_t nb = 1;
  for (int a = 0; a < ndims; a++) nb *= (dims[a] + 3) / 4;
  enum { MAXW = 200 };
  uint64_t *bits = calloc((size_t)n * MAXW, 8);
  int64_t nbits[16], st[16 * 5];
  double xt[64], dec[64];
  if (!bad && oc_code_brick(x, dtype, ndims, dims, tau, n, nb - 1, bits, MAXW, nbits, xt, st)) bad = 6;
  if (!bad && oc_decode_brick(dtype, ndims, tau, n, bits, MAXW, nbits, dec)) bad = 7;
  free(bits);
  free(box);
  free(out);
  oc_free(s);
  free(x);
  if (bad) fprintf(stderr, "field dtype=%d ndims=%d failed at step %d\n", dtype, ndims, bad);
  return bad;
}

int main(void) {
  const int64_t shapes[][3] = {{1, 1, 1}, {7, 1, 1}, {33, 1, 1}, {5, 9, 1}, {17, 12, 1}, {4, 4, 4},
                               {9, 6, 5}, {13, 10, 7}, {3, 2, 19}};
  const int nd[] = {1, 1, 1, 2, 2, 3, 3, 3, 3};
  int fails = 0;
  for (int t = 1; t <= 2; t++)
    for (size_t j = 0; j < sizeof(nd) / sizeof(nd[0]); j++) fails += run_field(t, nd[j], shapes[j], 6) != 0;
  printf("sanitized oracle runs: %d failed\n", fails);
  return fails ? 1 : 0;
}
