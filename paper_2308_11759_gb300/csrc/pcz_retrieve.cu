// pcz_retrieve.cu -- fused reconstruction kernel: Algorithm 2 (Magri &
// Lindstrom, Sec. 4.2) on the 4x4x4 bricks that meet a box.
//
// For each brick the kernel decodes components k0+1..k and adds them, in
// ascending order, into the partial sum x~ held in registers; x~ starts at 0
// or, to continue a refinement (Sec. 4.2), at the caller's x~_k0.  Only the
// bricks meeting the box are touched: zfp-style blocks decode on their own
// (Sec. 6.1).
//
// Layout: 4 warps per CTA, two bricks per warp, 16 lanes per brick, lane t
// holding the x-line y = t & 3, z = t >> 2.  Parsing a component's bit planes
// is sequential (each plane's length depends on the planes before it), so the
// 16 lanes of a brick parse up to 16 components side by side; the plane words
// go to shared memory, and then the brick's lanes rebuild each component's
// coefficients in ascending order, invert the transform and accumulate.
#include <type_traits>

#include "pcz_device.cuh"
#include "pcz_kernels.h"

namespace pcz {

__constant__ PermTable kPerm3r = make_perm(64);

constexpr int kRetrieveWarps3 = 4;
constexpr int kRetrieveThreads3 = 32 * kRetrieveWarps3;
constexpr int kParseLanes = 16;  // components parsed side by side per brick

struct BlockMeta {
  uint64_t off;  // first bit of the brick in the component's payload
  int mode, s, p, top;
};

template <typename T>
constexpr size_t retrieve_smem3() {
  using F = Fmt<T>;
  return (size_t)kRetrieveWarps3 *
         (2 * kParseLanes * F::P * sizeof(uint64_t)        // plane words
          + 2 * kParseLanes * sizeof(BlockMeta)            // per-component block header
          + 2 * 64 * sizeof(typename F::S));               // brick buffer
}

// R11 decoding of planes P-1 .. p of one block, starting at bit pos and ending
// exactly at end.  planes[pl] receives plane pl's word for pl in [p, top],
// where top is the highest non-empty plane (-1 if none).  Returns false on a
// malformed block; every loop is bounded by N and P.
template <typename T>
__device__ bool parse_planes(const uint64_t* __restrict__ w, uint64_t nw, uint64_t pos, uint64_t end, int p,
                             uint64_t* planes, int& top) {
  constexpr int N = 64;
  int n = 0;
  top = -1;
  for (int pl = Fmt<T>::P - 1; pl >= p; --pl) {
    uint64_t W = 0;
    if (n > 0) {
      W = peek64(w, nw, pos) & low_mask64(n);
      pos += (uint64_t)n;
    }
    while (n < N) {
      const uint64_t v = peek64(w, nw, pos);
      if (!(v & 1ull)) {  // test 0: nothing more in this plane
        pos += 1;
        break;
      }
      const uint64_t rest = v >> 1;
      int tz;
      if (rest) {
        tz = __ffsll((long long)rest) - 1;
      } else {
        if (!(peek64(w, nw, pos + 64) & 1ull)) return false;
        tz = 63;
      }
      if (n + tz >= N) return false;  // a promised 1 that never came
      W |= 1ull << (n + tz);
      n += tz + 1;
      pos += (uint64_t)tz + 2;
    }
    if (pos > end) return false;
    if (W && top < 0) top = pl;
    if (top >= 0) planes[pl] = W;
  }
  return pos == end;
}

template <typename T>
__global__ void __launch_bounds__(kRetrieveThreads3) k_retrieve3(const RetrieveParams R) {
  using F = Fmt<T>;
  using U = typename F::U;
  using S = typename F::S;
  constexpr int N = 64;
  constexpr int Q = F::P - 2 - Geo<3>::G;
  constexpr int C = Geo<3>::C;
  constexpr int HDR = 2 + 3 + F::EBITS;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int EMAXT = (1 << (F::EXPW - 1));  // frexp exponent of the largest finite T

  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, t = lane & 15;
  unsigned char* wbase = smem + (size_t)warp * (2 * kParseLanes * F::P * sizeof(uint64_t) +
                                                2 * kParseLanes * sizeof(BlockMeta) + 2 * 64 * sizeof(S));
  uint64_t* planes = reinterpret_cast<uint64_t*>(wbase);
  BlockMeta* meta = reinterpret_cast<BlockMeta*>(planes + 2 * kParseLanes * F::P);
  S* bbuf = reinterpret_cast<S*>(meta + 2 * kParseLanes) + h * 64;

  const int64_t g = (int64_t)blockIdx.x * (2 * kRetrieveWarps3) + warp * 2 + h;
  const bool have = g < R.nbox;
  int64_t bx = 0, by = 0, bz = 0, b = 0;
  if (have) {
    bx = R.bl[0] + g % R.bn[0];
    const int64_t r = g / R.bn[0];
    by = R.bl[1] + r % R.bn[1];
    bz = R.bl[2] + r / R.bn[1];
    b = bx + R.nb[0] * (by + R.nb[1] * bz);
  }
  const int64_t chunk = b / kChunk;
  const int ly = t & 3, lz = t >> 2;
  const int64_t gy = 4 * by + ly, gz = 4 * bz + lz;
  const bool line_ok = have && gy < R.dims[1] && gz < R.dims[2] && gy >= R.lo[1] && gy < R.hi[1] &&
                       gz >= R.lo[2] && gz < R.hi[2];
  const int64_t ext0 = R.hi[0] - R.lo[0], ext1 = R.hi[1] - R.lo[1];
  const int64_t orow = ((gz - R.lo[2]) * ext1 + (gy - R.lo[1])) * ext0;
  bool vm[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int64_t gx = 4 * bx + m;
    vm[m] = line_ok && gx < R.dims[0] && gx >= R.lo[0] && gx < R.hi[0];
  }
  T* out = reinterpret_cast<T*>(R.out);
  T xt[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {  // line 1, or the partial sum so far
    xt[m] = T(0);
    if (R.write && R.k0 > 0 && vm[m]) xt[m] = out[orow + 4 * bx + m - R.lo[0]];
  }
  int pos_r[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) pos_r[j] = kPerm3r.pos[t + 16 * j];
  const int xx = t & 3, yq = t >> 2;

  for (int base = R.k0; base < R.k; base += kParseLanes) {
    const int nc = min(kParseLanes, R.k - base);
    if (have && t < nc) {  // lane t parses component base + t of this brick
      const CompDesc cd = R.comp[base + t];
      uint64_t off = cd.chunk_word[chunk] * 64ull;
      for (int64_t bb = chunk * kChunk; bb < b; ++bb) off += cd.brick_len[bb];
      const uint64_t end = off + cd.brick_len[b];
      const uint64_t v = peek64(cd.payload, cd.nwords, off);
      int mode = (int)(v & 3ull), s = 0, p = 0, top = -1;
      bool ok;
      if (mode == kModeZero) {
        ok = end == off + 2;
      } else if (mode == kModeRaw) {
        ok = end == off + 2 + (uint64_t)N * F::P;
      } else if (mode == kModeCoded) {
        const int esc = (int)((v >> 2) & 7ull);
        const int emax = (int)((v >> 5) & ((1ull << F::EBITS) - 1)) - F::EBIAS;
        ok = emax >= F::EMIN && emax <= EMAXT;
        if (ok) {
          s = Q - emax;
          p = min(max(cd.L + s - C - esc, 0), F::P);
          ok = parse_planes<T>(cd.payload, cd.nwords, off + HDR, end, p, planes + (h * kParseLanes + t) * F::P, top);
        }
      } else {
        ok = false;
      }
      if (!ok) {
        atomicOr(R.err, 1u);
        mode = kModeZero;
      }
      BlockMeta bm;
      bm.off = off;
      bm.mode = mode;
      bm.s = s;
      bm.p = p;
      bm.top = top;
      meta[h * kParseLanes + t] = bm;
    }
    __syncwarp();
    for (int jj = 0; jj < nc; ++jj) {  // lines 2-4, components in ascending order
      BlockMeta my;
      my.mode = kModeZero;
      my.s = my.p = 0;
      my.top = -1;
      my.off = 0;
      if (have) my = meta[h * kParseLanes + jj];
      T xi[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) xi[m] = T(0);
      const bool coded = my.mode == kModeCoded;
      if (__any_sync(FULL, coded)) {
        const int hi_ = coded ? my.top : -1;
        const int lo_ = coded ? my.p : 1 << 20;
        int phi = max(hi_, __shfl_xor_sync(FULL, hi_, 16));
        int plo = min(lo_, __shfl_xor_sync(FULL, lo_, 16));
        U u[4] = {0, 0, 0, 0};
        const uint64_t* pw = planes + (h * kParseLanes + jj) * F::P;
        for (int pl = phi; pl >= plo; --pl) {
          if (coded && pl <= my.top && pl >= my.p) {
            const uint64_t W = pw[pl];
#pragma unroll
            for (int j = 0; j < 4; ++j) u[j] |= (U)((W >> (t + 16 * j)) & 1ull) << pl;
          }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) bbuf[pos_r[j]] = nb_inv<T>(u[j]);
        __syncwarp();
        {
          S a = bbuf[xx + 4 * yq], bq = bbuf[xx + 4 * yq + 16], c = bbuf[xx + 4 * yq + 32], d = bbuf[xx + 4 * yq + 48];
          lift_inv(a, bq, c, d);
          bbuf[xx + 4 * yq] = a; bbuf[xx + 4 * yq + 16] = bq; bbuf[xx + 4 * yq + 32] = c; bbuf[xx + 4 * yq + 48] = d;
        }
        __syncwarp();
        {
          S a = bbuf[xx + 16 * yq], bq = bbuf[xx + 4 + 16 * yq], c = bbuf[xx + 8 + 16 * yq], d = bbuf[xx + 12 + 16 * yq];
          lift_inv(a, bq, c, d);
          bbuf[xx + 16 * yq] = a; bbuf[xx + 4 + 16 * yq] = bq; bbuf[xx + 8 + 16 * yq] = c; bbuf[xx + 12 + 16 * yq] = d;
        }
        __syncwarp();
        S r[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) r[m] = bbuf[4 * t + m];
        __syncwarp();
        lift_inv(r[0], r[1], r[2], r[3]);
        if (coded) {
#pragma unroll
          for (int m = 0; m < 4; ++m) xi[m] = F::val(dequantize_bits<T>(r[m], my.s));
        }
      }
      if (my.mode == kModeRaw) {
        const CompDesc cd = R.comp[base + jj];
#pragma unroll
        for (int m = 0; m < 4; ++m)
          xi[m] = F::val((U)peek64(cd.payload, cd.nwords, my.off + 2 + (uint64_t)F::P * (4 * t + m)));
      }
#pragma unroll
      for (int m = 0; m < 4; ++m) xt[m] = F::add(xt[m], xi[m]);  // line 4: x~ += x_j
    }
    __syncwarp();
  }
  if (R.write) {
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (vm[m]) out[orow + 4 * bx + m - R.lo[0]] = xt[m];
  }
}

int retrieve_block_threads(int ndims) { return kRetrieveThreads3; }
int retrieve_bricks_per_block(int ndims) { return 2 * kRetrieveWarps3; }

template <typename T>
static cudaError_t launch_retrieve_t(const RetrieveParams& p, cudaStream_t s) {
  const size_t smem = retrieve_smem3<T>();
  cudaError_t e = cudaFuncSetAttribute(k_retrieve3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (p.nbox == 0) return cudaSuccess;
  const int64_t per = 2 * kRetrieveWarps3;
  k_retrieve3<T><<<(unsigned)((p.nbox + per - 1) / per), kRetrieveThreads3, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_retrieve(int dtype, int ndims, const RetrieveParams& p, cudaStream_t s) {
  if (ndims != 3) return cudaErrorNotSupported;
  return dtype == 1 ? launch_retrieve_t<float>(p, s) : launch_retrieve_t<double>(p, s);
}

}  // namespace pcz
