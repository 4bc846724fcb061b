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
// Layout: x fastest.  A CTA is a tile of 32 x 8 grid columns (x, y); each
// thread walks its column through a slice of z, so no index is divided per
// value and a second derivative along z keeps its three-point window in
// registers (each value loaded once).  Neighbours along x and y come from
// L1/L2 (float32 rows of a multiple of 4 values: the vorticity kernel moves
// float4s, 128-value tiles, x-neighbours by shuffle).  Each input is read from
// DRAM about once and the output written
// once: the kernels are bound by memory -- for float64 on GB300, whose FP64
// rate is low, by the FP64 pipe, which is why powers of two scale the
// exponent field with integer instructions where the result stays normal
// (the same value as the multiplication).
#include <algorithm>
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
  // x * 2^k, with p = 2^k
  static __device__ __forceinline__ float mul2k(float x, int, float p) { return __fmul_rn(x, p); }
};
template <>
struct Ar<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
  // x * 2^k (p = 2^k): when x and the result are normal the product is x with
  // k added to its exponent field, exactly the value the multiplication
  // gives; zeros, subnormals, infinities, NaN and results leaving the normal
  // range take the multiplication.
  static __device__ __forceinline__ double mul2k(double x, int k, double p) {
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e != 0 && e != 0x7ff && e + k >= 1 && e + k <= 2046) return __longlong_as_double(b + ((long long)k << 52));
    return __dmul_rn(x, p);
  }
};

// Division by the denominator d (2h or h^2 in T): when d = 2^-k is a power of
// two, the exact scaling by its reciprocal 2^k; else a correctly rounded
// division.
template <typename T>
struct Den {
  T d, inv;
  int pow2, k;
  __device__ __forceinline__ T apply(T x) const { return pow2 ? Ar<T>::mul2k(x, k, inv) : Ar<T>::div(x, d); }
};

// First derivative at coordinate c of n along a line of stride s from p
// (p points at the value at c).
template <typename T>
__device__ __forceinline__ T first_at(const T* __restrict__ p, int c, int n, int64_t s, const Den<T>& h2) {
  using A = Ar<T>;
  if (c > 0 && c < n - 1) return h2.apply(A::sub(__ldg(p + s), __ldg(p - s)));
  if (c == 0)
    return h2.apply(A::sub(A::sub(A::mul2k(__ldg(p + s), 2, T(4)), A::mul(T(3), __ldg(p))), __ldg(p + 2 * s)));
  return h2.apply(A::add(A::sub(A::mul(T(3), __ldg(p)), A::mul2k(__ldg(p - s), 2, T(4))), __ldg(p - 2 * s)));
}

template <typename T>
__device__ __forceinline__ T second_inner(T fp, T f0, T fm, const Den<T>& hh) {
  using A = Ar<T>;
  return hh.apply(A::add(A::sub(fp, A::mul2k(f0, 1, T(2))), fm));
}

template <typename T>
__device__ __forceinline__ T second_at(const T* __restrict__ p, int c, int n, int64_t s, const Den<T>& hh) {
  using A = Ar<T>;
  if (c > 0 && c < n - 1) return second_inner<T>(__ldg(p + s), __ldg(p), __ldg(p - s), hh);
  const int64_t d = c == 0 ? s : -s;  // towards the inside
  return hh.apply(A::sub(A::add(A::sub(A::mul2k(__ldg(p), 1, T(2)), A::mul(T(5), __ldg(p + d))),
                                A::mul2k(__ldg(p + 2 * d), 2, T(4))),
                         __ldg(p + 3 * d)));
}

constexpr int kTileX = 32, kTileY = 8;

// Thread (x, y) of a tile: its column and slice [z0, z1) of z.
struct Column {
  int x, y, z0, z1;
  bool ok;
};
__device__ __forceinline__ Column column(int nx, int ny, int nz, int zchunk) {
  Column c;
  c.x = blockIdx.x * kTileX + threadIdx.x;
  c.y = blockIdx.y * kTileY + threadIdx.y;
  c.z0 = blockIdx.z * zchunk;
  c.z1 = min(nz, c.z0 + zchunk);
  c.ok = c.x < nx && c.y < ny;
  return c;
}

// omega_z = v_x - u_y.
template <typename T>
__global__ void __launch_bounds__(kTileX * kTileY) k_vorticity_z(const T* __restrict__ u, const T* __restrict__ v,
                                                                 T* __restrict__ out, int nx, int ny, int nz,
                                                                 int zchunk, Den<T> h2) {
  const Column c = column(nx, ny, nz, zchunk);
  if (!c.ok) return;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t i0 = ((int64_t)c.z0 * ny + c.y) * nx + c.x;
  int z = c.z0;
  if (c.x > 0 && c.x < nx - 1 && c.y > 0 && c.y < ny - 1) {
    // interior column: the loads of 4 planes are issued before any is used
    using A = Ar<T>;
    for (; z + 4 <= c.z1; z += 4) {
      const int64_t i = i0 + (int64_t)(z - c.z0) * plane;
      T vp[4], vm[4], up[4], um[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        vp[j] = __ldg(v + i + j * plane + 1);
        vm[j] = __ldg(v + i + j * plane - 1);
        up[j] = __ldg(u + i + j * plane + nx);
        um[j] = __ldg(u + i + j * plane - nx);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        out[i + j * plane] = A::sub(h2.apply(A::sub(vp[j], vm[j])), h2.apply(A::sub(up[j], um[j])));
    }
  }
  for (; z < c.z1; ++z) {
    const int64_t i = i0 + (int64_t)(z - c.z0) * plane;
    out[i] = Ar<T>::sub(first_at<T>(v + i, c.x, nx, 1, h2), first_at<T>(u + i, c.y, ny, nx, h2));
  }
}

// omega_z = v_x - u_y for float32 rows whose length is a multiple of 4 (and
// 16-byte aligned arrays): a thread owns 4 consecutive x, loaded and stored as
// one float4, a warp 128; the x-neighbours of its 4 values come from the
// adjacent lanes by shuffle (the warp's two outer ones by a load), so a value
// costs 3/4 of a vector load instead of 4 loads.  Same operations and order
// as first_at.
__global__ void __launch_bounds__(kTileX * kTileY) k_vorticity_z4(const float* __restrict__ u,
                                                                  const float* __restrict__ v, float* __restrict__ out,
                                                                  int nx, int ny, int nz, int zchunk, Den<float> h2) {
  using A = Ar<float>;
  const int lane = threadIdx.x, y = blockIdx.y * kTileY + threadIdx.y;
  const int x4 = (blockIdx.x * kTileX + lane) * 4;
  const bool act = x4 < nx && y < ny;  // every lane stays for the shuffles
  const int z0 = blockIdx.z * zchunk, z1 = min(nz, z0 + zchunk);
  // rows of the y-derivative: (y + 1, y - 1) inside; the three-point ends otherwise
  const int ya = y == 0 ? 1 : y == ny - 1 ? ny - 1 : y + 1;
  const int yb = y == 0 ? 0 : y == ny - 1 ? ny - 2 : y - 1;
  const int yc = y == 0 ? 2 : ny - 3;  // third row of an end (unused inside)
  for (int z = z0; z < z1; ++z) {
    const int64_t row = ((int64_t)z * ny) * nx;
    float4 vc = make_float4(0.f, 0.f, 0.f, 0.f), ua = vc, ub = vc, uc = vc;
    float left = 0.f, right = 0.f;
    if (act) {
      const int64_t i = row + (int64_t)y * nx + x4;
      vc = __ldg(reinterpret_cast<const float4*>(v + i));
      ua = __ldg(reinterpret_cast<const float4*>(u + row + (int64_t)ya * nx + x4));
      ub = __ldg(reinterpret_cast<const float4*>(u + row + (int64_t)yb * nx + x4));
      if (y == 0 || y == ny - 1) uc = __ldg(reinterpret_cast<const float4*>(u + row + (int64_t)yc * nx + x4));
      if (lane == 0 && x4 > 0) left = __ldg(v + i - 1);
      if (lane == kTileX - 1 && x4 + 4 < nx) right = __ldg(v + i + 4);
    }
    const float l = __shfl_up_sync(0xffffffffu, vc.w, 1), r = __shfl_down_sync(0xffffffffu, vc.x, 1);
    if (lane > 0) left = l;
    if (lane < kTileX - 1) right = r;
    if (!act) continue;
    float vx[4];
    vx[0] = x4 == 0 ? h2.apply(A::sub(A::sub(A::mul2k(vc.y, 2, 4.f), A::mul(3.f, vc.x)), vc.z))
                    : h2.apply(A::sub(vc.y, left));
    vx[1] = h2.apply(A::sub(vc.z, vc.x));
    vx[2] = h2.apply(A::sub(vc.w, vc.y));
    vx[3] = x4 + 3 == nx - 1 ? h2.apply(A::add(A::sub(A::mul(3.f, vc.w), A::mul2k(vc.z, 2, 4.f)), vc.y))
                             : h2.apply(A::sub(right, vc.z));
    const float* pa = &ua.x;
    const float* pb = &ub.x;
    const float* pc = &uc.x;
    float o[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float uy;
      if (y == 0)  // ((4 u1 - 3 u0) - u2) / 2h
        uy = h2.apply(A::sub(A::sub(A::mul2k(pa[m], 2, 4.f), A::mul(3.f, pb[m])), pc[m]));
      else if (y == ny - 1)  // ((3 u[n-1] - 4 u[n-2]) + u[n-3]) / 2h
        uy = h2.apply(A::add(A::sub(A::mul(3.f, pa[m]), A::mul2k(pb[m], 2, 4.f)), pc[m]));
      else
        uy = h2.apply(A::sub(pa[m], pb[m]));
      o[m] = A::sub(vx[m], uy);
    }
    *reinterpret_cast<float4*>(out + row + (int64_t)y * nx + x4) = make_float4(o[0], o[1], o[2], o[3]);
  }
}

// d2w/da2 along x (axis 0) or y (axis 1).
template <typename T>
__global__ void __launch_bounds__(kTileX * kTileY) k_second_xy(const T* __restrict__ w, T* __restrict__ out, int nx,
                                                               int ny, int nz, int zchunk, int axis, Den<T> hh) {
  const Column c = column(nx, ny, nz, zchunk);
  if (!c.ok) return;
  const int64_t plane = (int64_t)nx * ny;
  const int cc = axis == 0 ? c.x : c.y, n = axis == 0 ? nx : ny;
  const int64_t s = axis == 0 ? 1 : nx;
  const int64_t i0 = ((int64_t)c.z0 * ny + c.y) * nx + c.x;
  int z = c.z0;
  if (cc > 0 && cc < n - 1) {  // interior column: 4 planes' loads in flight together
    for (; z + 4 <= c.z1; z += 4) {
      const int64_t i = i0 + (int64_t)(z - c.z0) * plane;
      T fp[4], f0[4], fm[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        fp[j] = __ldg(w + i + j * plane + s);
        f0[j] = __ldg(w + i + j * plane);
        fm[j] = __ldg(w + i + j * plane - s);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) out[i + j * plane] = second_inner<T>(fp[j], f0[j], fm[j], hh);
    }
  }
  for (; z < c.z1; ++z) {
    const int64_t i = i0 + (int64_t)(z - c.z0) * plane;
    out[i] = second_at<T>(w + i, cc, n, s, hh);
  }
}

// d2w/dz2: the column's window w[z-1], w[z], w[z+1] stays in registers.
template <typename T>
__global__ void __launch_bounds__(kTileX * kTileY) k_second_z(const T* __restrict__ w, T* __restrict__ out, int nx,
                                                              int ny, int nz, int zchunk, Den<T> hh) {
  const Column c = column(nx, ny, nz, zchunk);
  if (!c.ok) return;
  const int64_t plane = (int64_t)nx * ny;
  const int64_t col = (int64_t)c.y * nx + c.x;
  int za = c.z0, zb = c.z1;  // the slice's interior planes [za, zb)
  if (za == 0) {             // the four-point ends
    out[col] = second_at<T>(w + col, 0, nz, plane, hh);
    za = 1;
  }
  if (zb == nz) {
    out[col + (int64_t)(nz - 1) * plane] = second_at<T>(w + col + (int64_t)(nz - 1) * plane, nz - 1, nz, plane, hh);
    zb = nz - 1;
  }
  if (za >= zb) return;
  const T* p = w + col + (int64_t)za * plane;
  T* q = out + col + (int64_t)za * plane;
  T wm = __ldg(p - plane), w0 = __ldg(p);
  int z = za;
  for (; z + 4 <= zb; z += 4) {  // the next 4 planes' loads in flight together
    const int64_t o = (int64_t)(z - za) * plane;
    T wp[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) wp[j] = __ldg(p + o + (j + 1) * plane);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      q[o + j * plane] = second_inner<T>(wp[j], w0, wm, hh);
      wm = w0;
      w0 = wp[j];
    }
  }
  for (; z < zb; ++z) {
    const int64_t o = (int64_t)(z - za) * plane;
    const T wp = __ldg(p + o + plane);
    q[o] = second_inner<T>(wp, w0, wm, hh);
    wm = w0;
    w0 = wp;
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
  D.k = 1 - e;
  return D;
}

// Grid of tiles, with z split so that about 16 CTAs per SM are launched.
dim3 fd_grid(int nx, int ny, int nz, int* zchunk) {
  static const int sms = [] {  // once, thread-safe
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }();
  const int64_t tiles = (int64_t)((nx + kTileX - 1) / kTileX) * ((ny + kTileY - 1) / kTileY);
  int64_t split = (16 * (int64_t)sms + tiles - 1) / tiles;
  split = std::max<int64_t>(1, std::min<int64_t>(split, nz));
  *zchunk = (int)((nz + split - 1) / split);
  const int gz = (nz + *zchunk - 1) / *zchunk;
  return dim3((unsigned)((nx + kTileX - 1) / kTileX), (unsigned)((ny + kTileY - 1) / kTileY), (unsigned)gz);
}

}  // namespace

cudaError_t launch_fd_vorticity_z(int dtype, const void* u, const void* v, void* out, int64_t nx, int64_t ny,
                                  int64_t nz, double h, cudaStream_t st) {
  int zc = 1;
  const dim3 block(kTileX, kTileY);
  const bool vec4 = dtype == 1 && nx % 4 == 0 && ((uintptr_t)u | (uintptr_t)v | (uintptr_t)out) % 16 == 0;
  if (vec4) {  // the tiles are 128 values wide
    dim3 grid = fd_grid((int)(nx / 4), (int)ny, (int)nz, &zc);
    k_vorticity_z4<<<grid, block, 0, st>>>((const float*)u, (const float*)v, (float*)out, (int)nx, (int)ny, (int)nz,
                                           zc, make_den<float>(h, 1));
    return cudaGetLastError();
  }
  const dim3 grid = fd_grid((int)nx, (int)ny, (int)nz, &zc);
  if (dtype == 1)
    k_vorticity_z<float><<<grid, block, 0, st>>>((const float*)u, (const float*)v, (float*)out, (int)nx, (int)ny,
                                                 (int)nz, zc, make_den<float>(h, 1));
  else
    k_vorticity_z<double><<<grid, block, 0, st>>>((const double*)u, (const double*)v, (double*)out, (int)nx, (int)ny,
                                                  (int)nz, zc, make_den<double>(h, 1));
  return cudaGetLastError();
}

cudaError_t launch_fd_second(int dtype, const void* w, void* out, int64_t nx, int64_t ny, int64_t nz, int axis,
                             double h, cudaStream_t st) {
  int zc = 1;
  const dim3 grid = fd_grid((int)nx, (int)ny, (int)nz, &zc);
  const dim3 block(kTileX, kTileY);
  if (dtype == 1) {
    if (axis == 2)
      k_second_z<float><<<grid, block, 0, st>>>((const float*)w, (float*)out, (int)nx, (int)ny, (int)nz, zc,
                                                make_den<float>(h, 0));
    else
      k_second_xy<float><<<grid, block, 0, st>>>((const float*)w, (float*)out, (int)nx, (int)ny, (int)nz, zc, axis,
                                                 make_den<float>(h, 0));
  } else {
    if (axis == 2)
      k_second_z<double><<<grid, block, 0, st>>>((const double*)w, (double*)out, (int)nx, (int)ny, (int)nz, zc,
                                                 make_den<double>(h, 0));
    else
      k_second_xy<double><<<grid, block, 0, st>>>((const double*)w, (double*)out, (int)nx, (int)ny, (int)nz, zc, axis,
                                                  make_den<double>(h, 0));
  }
  return cudaGetLastError();
}

}  // namespace pcz
