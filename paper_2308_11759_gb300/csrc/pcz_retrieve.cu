// pcz_retrieve.cu -- fused reconstruction kernel: Algorithm 2 (Magri &
// Lindstrom, Sec. 4.2) on the 4x4x4 bricks that meet a box.
//
// For each brick the kernel decodes components k0+1..k and adds them, in
// ascending order, into the partial sum x~ held in registers; x~ starts at 0
// or, to continue a refinement (Sec. 4.2), at the caller's x~_k0.  Only the
// bricks meeting the box are touched: zfp-style blocks decode on their own
// (Sec. 6.1).
//
// Layout: 4 warps per CTA, two bricks per warp, 16 lanes per brick.  Parsing
// a component's bit planes is sequential (each plane's length depends on the
// planes above it), so lanes parse up to 8 components of their brick side by
// side with a register bit window; the bricks' bit offsets come from one
// coalesced load of the chunk's 32 brick lengths and a warp scan.  The plane
// words go to shared memory; then, per component in ascending order, lane p
// fetches plane p (and p + 32) of both bricks, a 32x32 bit transpose across
// the warp turns planes back into each lane's coefficients t + 16j, and the
// inverse reorder, lifting and scaling run through a bank-conflict-free brick
// buffer before x_j is added into x~.
#include <type_traits>

#include "pcz_device.cuh"
#include "pcz_kernels.h"

namespace pcz {

__constant__ PermTable kPerm3r = make_perm(64);

constexpr int kRetrieveWarps3 = 4;
constexpr int kRetrieveThreads3 = 32 * kRetrieveWarps3;
constexpr int kParseLanes = 8;  // components parsed side by side per brick

struct BlockMeta {
  uint64_t off;  // first bit of the brick in the component's payload
  int mode, s, p, top;
};

template <typename T>
__host__ __device__ constexpr size_t retrieve_warp_bytes3() {
  using F = Fmt<T>;
  return 2 * kParseLanes * F::P * sizeof(uint64_t)  // plane words
         + 2 * kParseLanes * sizeof(BlockMeta)      // per-component block header
         + 128 * sizeof(typename F::S);             // brick buffer of the two bricks
}

template <typename T>
constexpr size_t retrieve_smem3() {
  return (size_t)kRetrieveWarps3 * retrieve_warp_bytes3<T>();
}

// R11 decoding of planes P-1 .. p of one block, starting at bit pos and ending
// exactly at end.  planes[pl] receives plane pl's word for pl in [p, top],
// where top is the highest non-empty plane (-1 if none).  Returns false on a
// malformed block; every loop is bounded by N and P.
template <typename T>
__device__ bool parse_planes(BitReader& br, uint64_t pos, uint64_t end, int p, uint64_t* planes, int& top) {
  constexpr int N = 64;
  int n = 0;
  top = -1;
  for (int pl = Fmt<T>::P - 1; pl >= p; --pl) {
    uint64_t W = 0;
    if (n > 0) {
      W = br.peek(pos) & low_mask64(n);
      pos += (uint64_t)n;
    }
    for (int it = 0; it < N && n < N; ++it) {
      const uint64_t v = br.peek(pos);
      if (!(v & 1ull)) {  // test 0: nothing more in this plane
        pos += 1;
        break;
      }
      const uint64_t rest = v >> 1;
      int tz;
      if (rest) {
        tz = __ffsll((long long)rest) - 1;
      } else {
        if (!(br.peek(pos + 64) & 1ull)) return false;
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
  constexpr bool WIDE = F::P == 64;
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int EMAXT = (1 << (F::EXPW - 1));  // frexp exponent of the largest finite T

  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, h = lane >> 4, t = lane & 15;
  unsigned char* wbase = smem + (size_t)warp * retrieve_warp_bytes3<T>();
  uint64_t* planes = reinterpret_cast<uint64_t*>(wbase);
  BlockMeta* meta = reinterpret_cast<BlockMeta*>(planes + 2 * kParseLanes * F::P);
  S* buf = reinterpret_cast<S*>(meta + 2 * kParseLanes);

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
  const int inchunk = (int)(b - chunk * kChunk);
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
  const int xx = t & 3, yq = t >> 2;
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
  // the two bricks' chunks and places in them, known to every lane
  const int64_t chunkA = __shfl_sync(FULL, chunk, 0), chunkB = __shfl_sync(FULL, chunk, 16);
  const int posA = __shfl_sync(FULL, inchunk, 0), posB = __shfl_sync(FULL, inchunk, 16);
  const bool haveA = __shfl_sync(FULL, (int)have, 0) != 0, haveB = __shfl_sync(FULL, (int)have, 16) != 0;

  for (int base = R.k0; base < R.k; base += kParseLanes) {
    const int nc = min(kParseLanes, R.k - base);
    // bit offsets of both bricks in each component of this round: one coalesced
    // load of a chunk's 32 brick lengths and a warp scan per (component, brick)
    uint64_t my_off = 0, my_end = 0;
    for (int c = 0; c < nc; ++c) {
      const CompDesc& cd = R.comp[base + c];
#pragma unroll
      for (int hb = 0; hb < 2; ++hb) {
        const int64_t ch = hb ? chunkB : chunkA;
        const bool hv = hb ? haveB : haveA;
        const int pb = hb ? posB : posA;
        const int64_t bb = ch * kChunk + lane;
        const int len = (hv && bb < R.nbricks) ? (int)cd.brick_len[bb] : 0;
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(FULL, incl, o);
          if (lane >= o) incl += y;
        }
        const int before = __shfl_sync(FULL, incl - len, pb);
        const int mine = __shfl_sync(FULL, len, pb);
        if (lane == 16 * hb + c && hv) {
          my_off = cd.chunk_word[ch] * 64ull + (uint64_t)before;
          my_end = my_off + (uint64_t)mine;
        }
      }
    }
    if (have && t < nc) {  // lane t parses component base + t of this brick
      const CompDesc& cd = R.comp[base + t];
      BitReader br;
      br.init(cd.payload, cd.nwords, my_off);
      const uint64_t v = br.peek(my_off);
      int mode = (int)(v & 3ull), s = 0, p = 0, top = -1;
      bool ok;
      if (mode == kModeZero) {
        ok = my_end == my_off + 2;
      } else if (mode == kModeRaw) {
        ok = my_end == my_off + 2 + (uint64_t)N * F::P;
      } else if (mode == kModeCoded) {
        const int esc = (int)((v >> 2) & 7ull);
        const int emax = (int)((v >> 5) & ((1ull << F::EBITS) - 1)) - F::EBIAS;
        ok = emax >= F::EMIN && emax <= EMAXT;
        if (ok) {
          s = Q - emax;
          p = min(max(cd.L + s - C - esc, 0), F::P);
          ok = parse_planes<T>(br, my_off + HDR, my_end, p, planes + (h * kParseLanes + t) * F::P, top);
        }
      } else {
        ok = false;
      }
      if (!ok) {
        atomicOr(R.err, 1u);
        mode = kModeZero;
      }
      BlockMeta bm;
      bm.off = my_off;
      bm.mode = mode;
      bm.s = s;
      bm.p = p;
      bm.top = top;
      meta[h * kParseLanes + t] = bm;
    }
    __syncwarp();
    for (int jj = 0; jj < nc; ++jj) {  // lines 2-4, components in ascending order
      BlockMeta mA, mB;
      mA.mode = mB.mode = kModeZero;
      mA.s = mB.s = mA.p = mB.p = 0;
      mA.top = mB.top = -1;
      mA.off = mB.off = 0;
      if (haveA) mA = meta[jj];
      if (haveB) mB = meta[kParseLanes + jj];
      const BlockMeta& my = h ? mB : mA;
      T xi[4];
#pragma unroll
      for (int m = 0; m < 4; ++m) xi[m] = T(0);
      const bool cA = mA.mode == kModeCoded, cB = mB.mode == kModeCoded;
      if (cA || cB) {
        // lane l fetches plane l (and l + 32) of both bricks; planes outside
        // [p, top] are zero
        const uint64_t* pwA = planes + jj * F::P;
        const uint64_t* pwB = planes + (kParseLanes + jj) * F::P;
        const uint64_t WA0 = (cA && lane >= mA.p && lane <= mA.top) ? pwA[lane] : 0ull;
        const uint64_t WB0 = (cB && lane >= mB.p && lane <= mB.top) ? pwB[lane] : 0ull;
        U u[4];
        {
          uint32_t tl[4];
          tl[0] = __byte_perm((uint32_t)WA0, (uint32_t)WB0, 0x5410);
          tl[1] = __byte_perm((uint32_t)WA0, (uint32_t)WB0, 0x7632);
          tl[2] = __byte_perm((uint32_t)(WA0 >> 32), (uint32_t)(WB0 >> 32), 0x5410);
          tl[3] = __byte_perm((uint32_t)(WA0 >> 32), (uint32_t)(WB0 >> 32), 0x7632);
#pragma unroll
          for (int j = 0; j < 4; ++j) u[j] = (U)transpose32(tl[j], lane, tkeep);
        }
        if constexpr (WIDE) {
          const int pl = lane + 32;
          const uint64_t WA1 = (cA && pl >= mA.p && pl <= mA.top) ? pwA[pl] : 0ull;
          const uint64_t WB1 = (cB && pl >= mB.p && pl <= mB.top) ? pwB[pl] : 0ull;
          uint32_t th[4];
          th[0] = __byte_perm((uint32_t)WA1, (uint32_t)WB1, 0x5410);
          th[1] = __byte_perm((uint32_t)WA1, (uint32_t)WB1, 0x7632);
          th[2] = __byte_perm((uint32_t)(WA1 >> 32), (uint32_t)(WB1 >> 32), 0x5410);
          th[3] = __byte_perm((uint32_t)(WA1 >> 32), (uint32_t)(WB1 >> 32), 0x7632);
#pragma unroll
          for (int j = 0; j < 4; ++j) u[j] |= (U)((uint64_t)transpose32(th[j], lane, tkeep) << 32);
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
        S r[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) r[m] = buf[ix[m]];
        __syncwarp();
        lift_inv(r[0], r[1], r[2], r[3]);
        if (my.mode == kModeCoded) {
#pragma unroll
          for (int m = 0; m < 4; ++m) xi[m] = dequantize_val<T>(r[m], my.s);
        }
      }
      if (my.mode == kModeRaw) {
        const CompDesc& cd = R.comp[base + jj];
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
