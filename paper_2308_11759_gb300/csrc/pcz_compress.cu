// pcz_compress.cu -- fused construction kernel: Algorithm 1 (Magri & Lindstrom,
// Sec. 4.1) for every 4x4x4 brick of a 3D field, all n components in one pass.
//
// Per brick and component i the kernel computes the residual e = x - x~_{i-1},
// codes it with the PCZ coder at tau_i (y_i = C(e, tau_i)), reconstructs
// x_i = D(y_i) from the coded planes and adds it into x~.  x and x~ never
// leave registers, so the field is read once.
//
// Layout: one CTA per index chunk of 32 bricks (R15), 16 warps; a warp codes
// two bricks, 16 lanes each; lane t of a brick holds the x-line y = t & 3,
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
#include "pcz_chunk3.cuh"

namespace pcz {

template <typename T>
__global__ void __launch_bounds__(kCompressThreads3, 2) k_compress3(const CompressParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  compress3_chunk<T>(P, (int64_t)blockIdx.x, smem);
}

template <typename T>
static cudaError_t launch_compress_t(const CompressParams& p, cudaStream_t s) {
  const size_t smem = compress_smem3<T>();
  cudaError_t e = cudaFuncSetAttribute(k_compress3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (p.nchunks == 0) return cudaSuccess;
  k_compress3<T><<<(unsigned)p.nchunks, kCompressThreads3, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_compress(int dtype, int ndims, const CompressParams& p, cudaStream_t s) {
  if (ndims == 1 || ndims == 2) return launch_compress_small(dtype, ndims, p, s);
  if (ndims != 3) return cudaErrorNotSupported;
  return dtype == 1 ? launch_compress_t<float>(p, s) : launch_compress_t<double>(p, s);
}

uint32_t check_word_compress(int reset) { return read_check_word(reset); }

}  // namespace pcz
