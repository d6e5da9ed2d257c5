// Internal declarations shared by the translation units of libh2gb.
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/h2gb.h"

namespace h2 {

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
struct Error {
  h2_status code;
  std::string msg;
};

void set_error(h2_status code, const std::string &msg);
h2_status fail(h2_status code, const std::string &msg);

#define H2_CUDA(expr)                                                              \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      throw ::h2::Error{e_ == cudaErrorMemoryAllocation ? H2_ERR_OOM : H2_ERR_CUDA, \
                        std::string(#expr) + ": " + cudaGetErrorString(e_)};       \
    }                                                                              \
  } while (0)

#define H2_CHECK_LAUNCH() H2_CUDA(cudaGetLastError())

#define H2_REQUIRE(cond, msg)                        \
  do {                                               \
    if (!(cond)) throw ::h2::Error{H2_ERR_ARG, msg}; \
  } while (0)

// Counts kernels launched through the library (reported by h2_stats).
extern thread_local int64_t g_launches;
inline void count_launch(int64_t n = 1) { g_launches += n; }

// When set, the fused-summation launches record CUDA events around the main
// kernel on its stream and accumulate their device time here.
struct KernelTimer {
  double ms = 0.0;
  int64_t launches = 0;
};
extern thread_local KernelTimer *g_ksum_timer;

// ---------------------------------------------------------------------------
// Device memory.  Blocks come from a per-device cache of size buckets (at
// most 25% rounding) so that builds do not pay cudaMalloc/cudaFree (which
// synchronises the device) for every temporary.  All work of one library call
// is enqueued on one stream, so a block returned to the cache and handed out
// again is only touched after the earlier work on that stream.
// ---------------------------------------------------------------------------
void *dev_alloc(size_t bytes);
void dev_free(void *p, size_t bytes);
void dev_trim();

// A typed buffer returned to the cache on destruction.
template <typename T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    if (count) p = static_cast<T *>(dev_alloc(count * sizeof(T)));
  }
  void alloc_zero(size_t count, cudaStream_t s) {
    alloc(count);
    if (count) H2_CUDA(cudaMemsetAsync(p, 0, count * sizeof(T), s));
  }
  void release() {
    if (p) dev_free(p, n * sizeof(T));
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
};

template <typename T>
inline void to_device(DBuf<T> &b, const std::vector<T> &h, cudaStream_t s) {
  b.alloc(h.size());
  if (!h.empty())
    H2_CUDA(cudaMemcpyAsync(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

template <typename T>
inline std::vector<T> to_host(const T *p, size_t n, cudaStream_t s) {
  std::vector<T> h(n);
  if (n) {
    H2_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
  }
  return h;
}

// ---------------------------------------------------------------------------
// Matrix entries.  One descriptor per instance; the device evaluator works on
// squared distances (or dot products for the polynomial kernel).
// ---------------------------------------------------------------------------
struct KernelDesc {
  int kid;      // h2_kernel
  int pw;       // polynomial power
  double scale; // exp: 1/l; matern: sqrt3/l; gauss: 1/(2 s^2); laplace: 1/(4 pi); poly: c;
                // helmholtz: the wave number k
  double diag;  // nugget (exp/matern/gauss) or the diagonal value (laplace, helmholtz)
};

KernelDesc make_kernel_desc(int kid, const double *params, int nparams);

template <typename T>
__device__ __forceinline__ T dev_exp(T x);
template <>
__device__ __forceinline__ double dev_exp<double>(double x) { return exp(x); }
template <>
__device__ __forceinline__ float dev_exp<float>(float x) { return __expf(x); }

template <typename T>
__device__ __forceinline__ T dev_sqrt(T x);
template <>
__device__ __forceinline__ double dev_sqrt<double>(double x) { return sqrt(x); }
template <>
__device__ __forceinline__ float dev_sqrt<float>(float x) {
  return x > 0.f ? x * rsqrtf(x) : 0.f;
}

template <typename T>
__device__ __forceinline__ T dev_rsqrt(T x);
template <>
__device__ __forceinline__ double dev_rsqrt<double>(double x) { return 1.0 / sqrt(x); }
template <>
__device__ __forceinline__ float dev_rsqrt<float>(float x) { return rsqrtf(x); }

// cos(t) in FP32 to a few units of the last place for moderate |t|:
// Cody-Waite reduction u = t - q pi/2 (pi/2 split in two, the high part
// with 8 significant bits so that q * high is exact for |q| < 2^15), then
// the Taylor series of cos and sin on |u| <= pi/4 (truncation below 2e-9)
// and the quadrant q mod 4 picks +-cos(u) or +-sin(u).  All of it runs on
// the FMA pipe.
__device__ __forceinline__ float cos_reduced(float t) {
  const float q = rintf(t * 0.636619772367581343f);
  float u = fmaf(-q, 1.5703125f, t);
  u = fmaf(-q, 4.83826794896619231e-4f, u);
  const float u2 = u * u;
  float c = fmaf(u2, -2.75573192239858907e-7f, 2.48015873015873016e-5f);
  c = fmaf(u2, c, -1.38888888888888889e-3f);
  c = fmaf(u2, c, 4.16666666666666667e-2f);
  c = fmaf(u2, c, -0.5f);
  c = fmaf(u2, c, 1.f);
  float sn = fmaf(u2, 2.75573192239858907e-6f, -1.98412698412698413e-4f);
  sn = fmaf(u2, sn, 8.33333333333333333e-3f);
  sn = fmaf(u2, sn, -1.66666666666666667e-1f);
  sn = fmaf(u2 * u, sn, u);
  const int qi = (int)q & 3;
  const float v = (qi & 1) ? sn : c;
  return (qi == 1 || qi == 2) ? -v : v;
}

template <typename T>
__device__ __forceinline__ T dev_cos(T x);
template <>
__device__ __forceinline__ double dev_cos<double>(double x) { return cos(x); }
template <>
__device__ __forceinline__ float dev_cos<float>(float x) { return cos_reduced(x); }

// Off-diagonal kernel value from r^2 (or the dot product for POLY).
template <int KID, typename T>
__device__ __forceinline__ T kval(T r2_or_dot, T scale, int pw) {
  if constexpr (KID == H2_K_EXP) {
    return dev_exp<T>(-dev_sqrt<T>(r2_or_dot) * scale);
  } else if constexpr (KID == H2_K_MATERN32) {
    T a = dev_sqrt<T>(r2_or_dot) * scale;
    return (T(1) + a) * dev_exp<T>(-a);
  } else if constexpr (KID == H2_K_GAUSS) {
    return dev_exp<T>(-r2_or_dot * scale);
  } else if constexpr (KID == H2_K_LAPLACE_IE) {
    return r2_or_dot > T(0) ? dev_rsqrt<T>(r2_or_dot) * scale : T(0);
  } else if constexpr (KID == H2_K_HELMHOLTZ_IE) {
    if (!(r2_or_dot > T(0))) return T(0);
    const T ir = dev_rsqrt<T>(r2_or_dot);
    return dev_cos<T>(scale * (r2_or_dot * ir)) * ir;
  } else {  // POLY
    T base = scale + r2_or_dot;
    T v = T(1);
    for (int q = 0; q < pw; ++q) v *= base;
    return v;
  }
}

// Value on the diagonal (same point index).
template <int KID, typename T>
__device__ __forceinline__ T kdiag(T r2_or_dot, T scale, int pw, T diag) {
  if constexpr (KID == H2_K_LAPLACE_IE || KID == H2_K_HELMHOLTZ_IE) {
    return diag;
  } else if constexpr (KID == H2_K_POLY) {
    return kval<KID, T>(r2_or_dot, scale, pw);
  } else {
    return kval<KID, T>(r2_or_dot, scale, pw) + diag;
  }
}

// Geometry term between two points in FP64.
template <int KID>
__device__ __forceinline__ double geom64(double xi, double yi, double zi, double xj, double yj,
                                         double zj) {
  if constexpr (KID == H2_K_POLY) {
    return xi * xj + yi * yj + zi * zj;
  } else {
    double dx = xi - xj, dy = yi - yj, dz = zi - zj;
    return dx * dx + dy * dy + dz * dz;
  }
}

// Geometry term in FP32 from split coordinates x = hi + lo (hi = fl32(x),
// lo = fl32(x - hi)): the difference of the high parts carries a relative
// rounding of one FP32 ulp of the difference itself, so close pairs keep
// their relative accuracy.
template <int KID>
__device__ __forceinline__ float geom32(float xhi, float yhi, float zhi, float xlo, float ylo,
                                        float zlo, float xhj, float yhj, float zhj, float xlj,
                                        float ylj, float zlj) {
  if constexpr (KID == H2_K_POLY) {
    return (xhi + xlo) * (xhj + xlj) + (yhi + ylo) * (yhj + ylj) + (zhi + zlo) * (zhj + zlj);
  } else {
    float dx = (xhi - xhj) + (xlo - xlj);
    float dy = (yhi - yhj) + (ylo - ylj);
    float dz = (zhi - zhj) + (zlo - zlj);
    return dx * dx + dy * dy + dz * dz;
  }
}

// Point sets in the library's cluster-tree order, structure of arrays.
// dim < 3 is padded with zero coordinates (which leave every distance, dot
// product, box extent and box gap unchanged bit for bit).
struct Points64 {
  const double *x, *y, *z;
};
struct Points32 {
  const float *xh, *yh, *zh, *xl, *yl, *zl;
};

// Host-side dispatch of a templated functor over the kernel id.
template <typename F>
inline void dispatch_kernel(int kid, F &&f) {
  switch (kid) {
    case H2_K_EXP: f(std::integral_constant<int, H2_K_EXP>{}); break;
    case H2_K_MATERN32: f(std::integral_constant<int, H2_K_MATERN32>{}); break;
    case H2_K_GAUSS: f(std::integral_constant<int, H2_K_GAUSS>{}); break;
    case H2_K_LAPLACE_IE: f(std::integral_constant<int, H2_K_LAPLACE_IE>{}); break;
    case H2_K_POLY: f(std::integral_constant<int, H2_K_POLY>{}); break;
    case H2_K_HELMHOLTZ_IE: f(std::integral_constant<int, H2_K_HELMHOLTZ_IE>{}); break;
    default: throw Error{H2_ERR_ARG, "unknown kernel id"};
  }
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

int device_sm_count();

}  // namespace h2
