// pcz_fd.cu -- finite-difference derivatives of reconstructed fields: the
// operators of the progressive use case (Magri & Lindstrom, Sec. 5.3), the
// vorticity component omega_z = v_x - u_y of a velocity field and a second
// derivative such as w_zz.  A derivative of order i magnifies the error of a
// reconstruction x~_k like h^-i, which is why each needs more components.
//
// Stencils (second order at every point): a first derivative is
// (f[i+1] - f[i-1]) / (2h) inside and ((4 f1 - 3 f0) - f2) / (2h),
// ((3 f[n-1] - 4 f[n-2]) + f[n-3]) / (2h) at the ends; a second derivative
// is ((f[i+1] - 2 f[i]) + f[i-1]) / h^2 inside and
// (((2 f0 - 5 f1) + 4 f2) - f3) / h^2 and its mirror image at the ends.  The
// arithmetic is the field's own precision, one IEEE rounding per operation
// in that order, with 2h and h^2 formed from h rounded to the type.  A
// division by a power of two is done as the exact multiplication by its
// reciprocal (the same result); other spacings divide.
//
// Layout: x fastest, rows of nx values (row r = y + ny z).  The kernels are
// bound by memory: a block takes segments of 256 consecutive values of a row
// (coalesced loads and stores); the neighbouring rows and planes a stencil
// reads come back from L1/L2, so each input is read from DRAM about once.
#include <cmath>
#include <cstdint>

#include "pcz_kernels.h"

namespace pcz {

namespace {

template <typename T>
struct Ar;
template <>
struct Ar<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
};
template <>
struct Ar<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};

// Division by the denominator d (2h or h^2 in T): by the exact reciprocal
// when d is a power of two, else a correctly rounded division.
template <typename T>
struct Den {
  T d, inv;
  int pow2;
  __device__ __forceinline__ T apply(T x) const { return pow2 ? Ar<T>::mul(x, inv) : Ar<T>::div(x, d); }
};

// First derivative at coordinate c of n along a line of stride s from p
// (p points at the value at c).
template <typename T>
__device__ __forceinline__ T first_at(const T* __restrict__ p, int64_t c, int64_t n, int64_t s, const Den<T>& h2) {
  using A = Ar<T>;
  if (c > 0 && c < n - 1) return h2.apply(A::sub(__ldg(p + s), __ldg(p - s)));
  if (c == 0)
    return h2.apply(A::sub(A::sub(A::mul(T(4), __ldg(p + s)), A::mul(T(3), __ldg(p))), __ldg(p + 2 * s)));
  return h2.apply(A::add(A::sub(A::mul(T(3), __ldg(p)), A::mul(T(4), __ldg(p - s))), __ldg(p - 2 * s)));
}

template <typename T>
__device__ __forceinline__ T second_at(const T* __restrict__ p, int64_t c, int64_t n, int64_t s, const Den<T>& hh) {
  using A = Ar<T>;
  if (c > 0 && c < n - 1) return hh.apply(A::add(A::sub(__ldg(p + s), A::mul(T(2), __ldg(p))), __ldg(p - s)));
  const int64_t d = c == 0 ? s : -s;  // towards the inside
  return hh.apply(A::sub(A::add(A::sub(A::mul(T(2), __ldg(p)), A::mul(T(5), __ldg(p + d))), A::mul(T(4), __ldg(p + 2 * d))),
                         __ldg(p + 3 * d)));
}

constexpr int kFdThreads = 256;

// omega_z = v_x - u_y over rows = ny * nz rows of nx values.
template <typename T>
__global__ void __launch_bounds__(kFdThreads) k_vorticity_z(const T* __restrict__ u, const T* __restrict__ v,
                                                            T* __restrict__ out, int64_t nx, int64_t ny,
                                                            int64_t rows, Den<T> h2) {
  const int64_t segs = (nx + kFdThreads - 1) / kFdThreads;
  for (int64_t g = blockIdx.x; g < rows * segs; g += gridDim.x) {
    const int64_t r = g / segs, x = (g - r * segs) * kFdThreads + threadIdx.x;
    if (x >= nx) continue;
    const int64_t y = r % ny, i = r * nx + x;
    const T vx = first_at<T>(v + i, x, nx, 1, h2);
    const T uy = first_at<T>(u + i, y, ny, nx, h2);
    out[i] = Ar<T>::sub(vx, uy);
  }
}

// d2w/da2 along the axis of coordinate extent n and stride s (a = 0, 1, 2:
// x, y = r % ny, z = r / ny).
template <typename T>
__global__ void __launch_bounds__(kFdThreads) k_second(const T* __restrict__ w, T* __restrict__ out, int64_t nx,
                                                       int64_t ny, int64_t rows, int axis, int64_t n, int64_t s,
                                                       Den<T> hh) {
  const int64_t segs = (nx + kFdThreads - 1) / kFdThreads;
  for (int64_t g = blockIdx.x; g < rows * segs; g += gridDim.x) {
    const int64_t r = g / segs, x = (g - r * segs) * kFdThreads + threadIdx.x;
    if (x >= nx) continue;
    const int64_t c = axis == 0 ? x : axis == 1 ? r % ny : r / ny;
    const int64_t i = r * nx + x;
    out[i] = second_at<T>(w + i, c, n, s, hh);
  }
}

template <typename T>
Den<T> make_den(double h, int twice) {
  const T ht = (T)h;
  Den<T> D;
  D.d = twice ? (T)(ht * T(2)) : (T)(ht * ht);  // 2h exactly, or h^2 rounded once in T
  int e = 0;
  const double m = std::frexp((double)D.d, &e);
  const T inv = (T)std::ldexp(1.0, 1 - e);  // 1 / d when d is a power of two
  D.pow2 = m == 0.5 && std::isfinite(inv) && inv != T(0);
  D.inv = D.pow2 ? inv : T(0);
  return D;
}

int fd_grid(int64_t work) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
  }
  const int64_t cap = (int64_t)sms * 8;  // 8 blocks of 256 threads per SM, grid-stride beyond
  return (int)(work < cap ? (work > 0 ? work : 1) : cap);
}

}  // namespace

cudaError_t launch_fd_vorticity_z(int dtype, const void* u, const void* v, void* out, int64_t nx, int64_t ny,
                                  int64_t nz, double h, cudaStream_t st) {
  const int64_t rows = ny * nz, work = rows * ((nx + kFdThreads - 1) / kFdThreads);
  const int grid = fd_grid(work);
  if (dtype == 1)
    k_vorticity_z<float><<<grid, kFdThreads, 0, st>>>((const float*)u, (const float*)v, (float*)out, nx, ny, rows,
                                                      make_den<float>(h, 1));
  else
    k_vorticity_z<double><<<grid, kFdThreads, 0, st>>>((const double*)u, (const double*)v, (double*)out, nx, ny,
                                                       rows, make_den<double>(h, 1));
  return cudaGetLastError();
}

cudaError_t launch_fd_second(int dtype, const void* w, void* out, int64_t nx, int64_t ny, int64_t nz, int axis,
                             double h, cudaStream_t st) {
  const int64_t rows = ny * nz, work = rows * ((nx + kFdThreads - 1) / kFdThreads);
  const int64_t n = axis == 0 ? nx : axis == 1 ? ny : nz;
  const int64_t s = axis == 0 ? 1 : axis == 1 ? nx : nx * ny;
  const int grid = fd_grid(work);
  if (dtype == 1)
    k_second<float><<<grid, kFdThreads, 0, st>>>((const float*)w, (float*)out, nx, ny, rows, axis, n, s,
                                                 make_den<float>(h, 0));
  else
    k_second<double><<<grid, kFdThreads, 0, st>>>((const double*)w, (double*)out, nx, ny, rows, axis, n, s,
                                                  make_den<double>(h, 0));
  return cudaGetLastError();
}

}  // namespace pcz
