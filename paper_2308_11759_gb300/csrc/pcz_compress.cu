// pcz_compress.cu -- fused construction kernel: Algorithm 1 (Magri & Lindstrom,
// Sec. 4.1) for every 4x4x4 brick of a 3D field, all n components in one pass.
//
// Per brick and component i the kernel computes the residual e = x - x~_{i-1},
// codes it with the PCZ coder at tau_i (y_i = C(e, tau_i)), reconstructs
// x_i = D(y_i) from the coded planes and adds it into x~.  x and x~ never
// leave registers, so the field is read once.
//
// Layout: one CTA per index chunk of 32 bricks (R15), 16 warps, two CTAs per
// SM; each lane loads its line of the field with 16-byte vector loads.  (A
// second form, k_compress3_tma, stages the chunks in shared memory with TMA
// tile copies in persistent CTAs; it is selected by PCZ_COMPRESS_TMA=1.)
// A warp codes two bricks, 16 lanes each; lane t of a brick holds the x-line y = t & 3,
// z = t >> 2, and after the transform the coded coefficients t + 16j.  The y
// and z lifting passes and the reorder go through a bank-conflict-free brick
// buffer in shared memory.  Bit planes come from 32x32 bit transposes across
// the warp, after which lane p owns plane p (and p + 32): each lane emits its
// plane's verbatim bits (R11), with the significance count before the plane
// and the plane's bit offset from suffix scans over lanes (planes are coded
// from the top down); the lane holding a coefficient writes the bits of the
// token that makes it significant, at positions that follow from the plane's
// offset, its significance count and the coefficient's rank among the plane's
// new coefficients.  The chunk's bits are assembled in shared memory and
// appended to a scratch pool with one atomic per chunk; pcz_misc.cu then scans
// the chunk sizes and packs the final streams.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "pcz_chunk3.cuh"

namespace pcz {

// One chunk per CTA, each lane's line loaded straight into registers.
template <typename T>
__global__ void __launch_bounds__(kCompressThreads3, 2) k_compress3(const CompressParams P) {
  extern __shared__ __align__(128) unsigned char smem[];
  compress3_chunk<T>(P, (int64_t)blockIdx.x, smem);
}

// Persistent CTAs with the chunks staged by TMA: chunk c's values are copied
// into shared memory while chunk c - grid is coded.
template <typename T>
__global__ void __launch_bounds__(kCompressThreads3, 2)
    k_compress3_tma(const CompressParams P, const __grid_constant__ CUtensorMap tmap, int row_box) {
  extern __shared__ __align__(128) unsigned char smem[];
  T* xs = reinterpret_cast<T*>(smem);
  uint64_t* bar = reinterpret_cast<uint64_t*>(xs + kChunk * 64);
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(bar);
    if ((int64_t)blockIdx.x < P.nchunks) issue_chunk_copy<T>(P, &tmap, row_box != 0, (int64_t)blockIdx.x, xs, bar);
  }
  __syncthreads();
  uint32_t parity = 0;
  for (int64_t c = blockIdx.x; c < P.nchunks; c += gridDim.x) {
    const bool ok = mbar_wait(bar, parity, 1 << 20);
    if (!__syncthreads_and(ok)) {  // the copy did not land: report, wait once more (bounded) and stop
      if (tid == 0) atomicOr(P.flags, kFlagStageTimeout);
      mbar_wait(bar, parity, 1 << 20);
      return;
    }
    parity ^= 1u;
    compress3_chunk<T>(P, c, smem, &tmap, row_box != 0, bar, c + gridDim.x);
  }
}

// cuTensorMapEncodeTiled, looked up once through the runtime (the library
// does not link the driver API).
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_tiled() {
  static std::once_flag once;
  static EncodeTiled fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

// A tensor map of the 3D field with a box of bx x 4 x 4 values (bx = 128: a
// chunk of 32 bricks along x; 4: one brick), when the rules of TMA tile copies
// hold for it: a 16-byte aligned base, rows whose byte length is a multiple of
// 16 (so every stride is), extents below 2^31.  Box origins are multiples of 4
// values along x, so every copy starts on a 16-byte boundary.
template <typename T>
static bool make_brick_map(const CompressParams& p, cuuint32_t bx, CUtensorMap* map) {
  const EncodeTiled fn = encode_tiled();
  if (!fn) return false;
  if (((uintptr_t)p.field & 15) != 0 || ((uint64_t)p.dims[0] * sizeof(T)) % 16 != 0) return false;
  for (int a = 0; a < 3; ++a)
    if (p.dims[a] < 1 || p.dims[a] >= (1ll << 31)) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)p.dims[0], (cuuint64_t)p.dims[1], (cuuint64_t)p.dims[2]};
  const cuuint64_t strides[2] = {(cuuint64_t)p.dims[0] * sizeof(T), (cuuint64_t)p.dims[0] * p.dims[1] * sizeof(T)};
  const cuuint32_t box[3] = {bx, 4, 4}, estr[3] = {1, 1, 1};
  const CUresult r = fn(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                        const_cast<void*>(p.field), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// TMA staging is measured slower than the direct loads on GB300 (by 9 % for
// float32 and 6 % for float64 on a 512^3 field; 4 % for float32 with one
// chunk per CTA and no prefetch), so it is off unless PCZ_COMPRESS_TMA=1 is in
// the environment when the library is first used.
static bool tma_staging() {
  static const bool on = [] {
    const char* v = std::getenv("PCZ_COMPRESS_TMA");
    return v && v[0] == '1' && v[1] == 0;
  }();
  return on;
}

template <typename T>
static cudaError_t launch_compress_t(const CompressParams& p, cudaStream_t s, bool device_field) {
  const size_t smem_direct = compress_smem3<T>(false), smem_tma = compress_smem3<T>(true);
  cudaError_t e = cudaFuncSetAttribute(k_compress3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_direct);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_compress3_tma<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tma);
  if (e != cudaSuccess) return e;
  if (p.nchunks == 0) return cudaSuccess;
  CUtensorMap map;
  std::memset(&map, 0, sizeof(map));
  const int row_box = p.nb[0] % kChunk == 0 ? 1 : 0;
  const int use_tma = tma_staging() && device_field && make_brick_map<T>(p, row_box ? 128 : 4, &map) ? 1 : 0;
  int64_t grid = p.nchunks;
  if (use_tma) {  // persistent: the CTAs that fit at once
    static const int64_t fit = [smem_tma] {  // once per type, thread-safe
      int dev = 0, sms = 0, per = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_compress3_tma<T>, kCompressThreads3, smem_tma) !=
          cudaSuccess) {
        cudaGetLastError();
        per = 1;
      }
      return (int64_t)std::max(per, 1) * std::max(sms, 1);
    }();
    grid = std::min<int64_t>(grid, fit);
  }
  if (use_tma)
    k_compress3_tma<T><<<(unsigned)grid, kCompressThreads3, smem_tma, s>>>(p, map, row_box);
  else
    k_compress3<T><<<(unsigned)grid, kCompressThreads3, smem_direct, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_compress(int dtype, int ndims, const CompressParams& p, cudaStream_t s, bool device_field) {
  if (ndims == 1 || ndims == 2) return launch_compress_small(dtype, ndims, p, s);
  if (ndims != 3) return cudaErrorNotSupported;
  return dtype == 1 ? launch_compress_t<float>(p, s, device_field) : launch_compress_t<double>(p, s, device_field);
}

uint32_t check_word_compress(int reset) { return read_check_word(reset); }

}  // namespace pcz
