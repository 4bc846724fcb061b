// pcz_small.cu -- Algorithms 1 and 2 (Magri & Lindstrom, Sec. 4.1, 4.2) for
// 1D and 2D fields, whose bricks hold 4 and 16 values.
//
// A brick this small fits one thread: each thread codes one brick entirely
// in registers (residual, alignment, lifting along x then y, sequency order,
// negabinary, bit planes from the top down, decode-back and verification),
// and one warp covers one index chunk of 32 bricks, so the bricks' bit
// offsets in the chunk come from a warp scan.  The bits are assembled in a
// per-warp shared buffer and appended to the scratch pool like the 3D
// kernel's chunks; retrieval mirrors this with one thread per brick and
// component parsing and rebuilding a brick.
#include "pcz_chunk_small.cuh"

namespace pcz {

template <typename T, int D>
__global__ void __launch_bounds__(kSmallThreads) k_compress_small(const CompressParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5;
  uint32_t* cbuf = reinterpret_cast<uint32_t*>(smem) + (size_t)warp * chunk_words_small<T, D>();
  compress_small_chunk<T, D>(P, (int64_t)blockIdx.x * kSmallWarps + warp, cbuf);
}

// One thread per brick: of the single job, or of a job list whose units are
// bricks (unit_begin = the job's first brick among all jobs' bricks).
template <typename T, int D>
__global__ void __launch_bounds__(kSmallThreads) k_retrieve_small(const RetrieveParams R) {
  const int64_t g = (int64_t)blockIdx.x * kSmallThreads + threadIdx.x;
  if (!R.jobs) {
    if (g < R.job0.nbox) retrieve_small_brick<T, D>(R.job0, R.write, R.err, g);
    return;
  }
  if (g >= R.nunits) return;
  int lo = 0, hi = R.njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (R.jobs[mid].unit_begin <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  const BoxJob& J = R.jobs[lo];
  retrieve_small_brick<T, D>(J, R.write, R.err, g - J.unit_begin);
}

template <typename T, int D>
static cudaError_t launch_compress_small_t(const CompressParams& p, cudaStream_t s) {
  const size_t smem = small_smem<T, D>();
  cudaError_t e = cudaFuncSetAttribute(k_compress_small<T, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (p.nchunks == 0) return cudaSuccess;
  k_compress_small<T, D><<<(unsigned)((p.nchunks + kSmallWarps - 1) / kSmallWarps), kSmallThreads, smem, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_compress_small(int dtype, int ndims, const CompressParams& p, cudaStream_t s) {
  if (ndims == 1) return dtype == 1 ? launch_compress_small_t<float, 1>(p, s) : launch_compress_small_t<double, 1>(p, s);
  return dtype == 1 ? launch_compress_small_t<float, 2>(p, s) : launch_compress_small_t<double, 2>(p, s);
}

template <typename T, int D>
static cudaError_t launch_retrieve_small_t(const RetrieveParams& p, cudaStream_t s) {
  const int64_t work = p.jobs ? p.nunits : p.job0.nbox;
  if (work == 0) return cudaSuccess;
  k_retrieve_small<T, D><<<(unsigned)((work + kSmallThreads - 1) / kSmallThreads), kSmallThreads, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_retrieve_small(int dtype, int ndims, const RetrieveParams& p, cudaStream_t s) {
  if (ndims == 1) return dtype == 1 ? launch_retrieve_small_t<float, 1>(p, s) : launch_retrieve_small_t<double, 1>(p, s);
  return dtype == 1 ? launch_retrieve_small_t<float, 2>(p, s) : launch_retrieve_small_t<double, 2>(p, s);
}

uint32_t check_word_small(int reset) { return read_check_word(reset); }

}  // namespace pcz
