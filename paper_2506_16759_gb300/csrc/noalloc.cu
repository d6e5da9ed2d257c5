// A variant of the batched QR convergence statistic that allocates no device
// memory.  Its working copies of the panels live in a fixed array that is part
// of the loaded library image, so callers that must not call cudaMalloc (for
// example code running inside a custom allocator callback, or a host that
// pre-reserves all device memory for itself) can still use it.
//
// Layout of the fixed array for one call with `count` panels:
//   [0, base)           per-panel start offsets (int64, count + 1 of them),
//                       base rounded up to 32 doubles (256 bytes);
//   [base, capacity)    working copies of the panels that need a QR
//                       (m > d), one after the other in panel order.
#include <cuda.h>

#include <map>
#include <mutex>

#include "h2_internal.cuh"

namespace h2 {
namespace {

// Capacity of the static workspace, in doubles (16 MiB).  Every device that
// loads the library holds this array until the process exits.
constexpr int64_t kStaticQrDoubles = int64_t(1) << 21;

static __device__ __align__(256) double g_static_qr_scratch[kStaticQrDoubles];
static __device__ int g_static_qr_flag;

// Flag bits raised by the kernels.
constexpr int kFlagOverflow = 1;   // the panels needing a QR do not fit
constexpr int kFlagShape = 2;      // some panel has m < 0 or d < 1

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum_d(double v, double *sh) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_d(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double w = lane < nw ? sh[lane] : 0.0;
    w = warp_sum_d(w);
    if (lane == 0) sh[32] = w;
  }
  __syncthreads();
  double r = sh[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ bool panel_shape_ok(int32_t mt, int32_t dt) { return mt >= 0 && dt >= 1; }

// One CTA of 1024 threads: offs[i] = base + the doubles needed by the valid
// panels before i that need a QR (m > d); offs[count] = the end.  A panel
// needing more than the whole capacity counts as capacity + 1, so the sum of
// at most 2^31 panels cannot overflow and still exceeds the capacity.
__global__ void __launch_bounds__(1024)
    k_static_offsets(int count, const int32_t *__restrict__ m, const int32_t *__restrict__ d,
                     int64_t base, int64_t cap, int64_t *offs, int *flag) {
  __shared__ int64_t warp_tot[32];
  __shared__ int64_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = base;
  __syncthreads();
  bool bad = false;
  for (int c0 = 0; c0 < count; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    int64_t need = 0;
    if (i < count) {
      const int32_t mt = m[i], dt = d[i];
      if (!panel_shape_ok(mt, dt)) bad = true;
      else if (mt > dt) need = min((int64_t)mt * dt, cap + 1);
    }
    // inclusive scan within the warp, then over the warp totals
    int64_t v = need;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += u;
    }
    if (lane == 31) warp_tot[warp] = v;
    __syncthreads();
    if (warp == 0) {
      int64_t w = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t u = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += u;
      }
      warp_tot[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    const int64_t before_warp = warp > 0 ? warp_tot[warp - 1] : 0;
    if (i < count) offs[i] = carry + before_warp + (v - need);
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[31];
    __syncthreads();
  }
  if (bad) atomicOr(flag, kFlagShape);
  if (threadIdx.x == 0) offs[count] = carry;
}

// One CTA per panel: min_j |R_jj| of the Householder QR of panel t
// (m[t] x d[t], column-major at panels + off[t], ld = m[t]); 0 if m <= d.
// Its working copy starts at offs[t]; a panel that does not fit raises the
// overflow flag and gets NaN, and so does a panel with m < 0 or d < 1 (the
// offsets kernel raised the shape flag for it).
__global__ void __launch_bounds__(256)
    k_qr_mindiag_static(int count, const int32_t *__restrict__ m, const int32_t *__restrict__ d,
                        const int64_t *__restrict__ off, const double *__restrict__ panels,
                        double *mindiag, double *scratch, const int64_t *__restrict__ offs,
                        int64_t cap, int *flag) {
  __shared__ double red[33];
  int t = blockIdx.x;
  int mt = m[t], dt = d[t];
  if (!panel_shape_ok(mt, dt)) {
    if (threadIdx.x == 0) mindiag[t] = nan("");
    return;
  }
  if (mt <= dt) {
    if (threadIdx.x == 0) mindiag[t] = 0.0;
    return;
  }
  const int64_t start = offs[t];
  const int64_t need = (int64_t)mt * dt;
  if (start < 0 || start + need > cap) {
    if (threadIdx.x == 0) {
      atomicOr(flag, kFlagOverflow);
      mindiag[t] = nan("");
    }
    return;
  }
  double *A = scratch + start;
  const double *Y = panels + off[t];
  for (int64_t q = threadIdx.x; q < need; q += blockDim.x) A[q] = Y[q];
  __syncthreads();
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double minr = INFINITY;
  for (int j = 0; j < dt; ++j) {
    double *colj = A + (int64_t)j * mt;
    double part = 0.0;
    for (int i = j + threadIdx.x; i < mt; i += blockDim.x) part += colj[i] * colj[i];
    double nrm = sqrt(block_sum_d(part, red));
    minr = fmin(minr, nrm);
    if (nrm == 0.0) continue;
    double x0 = colj[j];
    double alpha = x0 != 0.0 ? -copysign(nrm, x0) : -nrm;
    double beta = 1.0 / (nrm * (nrm + fabs(x0)));
    __syncthreads();
    if (threadIdx.x == 0) colj[j] = x0 - alpha;
    __syncthreads();
    for (int c = j + 1 + warp; c < dt; c += nw) {
      double *colc = A + (int64_t)c * mt;
      double w = 0.0;
      for (int i = j + lane; i < mt; i += 32) w += colj[i] * colc[i];
      w = warp_sum_d(w) * beta;
      for (int i = j + lane; i < mt; i += 32) colc[i] -= w * colj[i];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) mindiag[t] = minr;
}

// Device addresses of the static arrays, looked up once per device and
// context (host code must not pass the symbols themselves to a kernel: on the
// host they name host-side stand-ins).  The context's unique id keys the
// cache, so a new primary context after cudaDeviceReset gets a new lookup.
struct StaticAddr {
  double *scratch = nullptr;
  int *flag = nullptr;
};
std::mutex g_setup_mutex;
std::map<std::pair<int, unsigned long long>, StaticAddr> g_static_addr;

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context; false if the driver
// does not provide one (the caller then looks the addresses up every time).
bool current_context_id(unsigned long long *id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void *f = nullptr, *g = nullptr;
    cudaDriverEntryPointQueryResult q1{}, q2{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) ==
            cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) ==
            cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
      get_id = reinterpret_cast<CtxGetIdFn>(g);
    }
    cudaGetLastError();
  });
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

h2_status lookup_addresses(StaticAddr *a) {
  void *p = nullptr, *q = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_qr_scratch);
  if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_static_qr_flag);
  if (e != cudaSuccess)
    return fail(H2_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  a->scratch = static_cast<double *>(p);
  a->flag = static_cast<int *>(q);
  return H2_OK;
}

h2_status static_addresses(StaticAddr *out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess)
    return fail(H2_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  // makes the device's primary context current (created on first use)
  e = cudaSetDevice(dev);
  if (e != cudaSuccess)
    return fail(H2_ERR_CUDA, std::string("context set-up: ") + cudaGetErrorString(e));
  unsigned long long ctx = 0;
  if (!current_context_id(&ctx)) return lookup_addresses(out);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  auto it = g_static_addr.find({dev, ctx});
  if (it == g_static_addr.end()) {
    StaticAddr a;
    h2_status st = lookup_addresses(&a);
    if (st != H2_OK) return st;
    it = g_static_addr.emplace(std::make_pair(dev, ctx), a).first;
  }
  *out = it->second;
  return H2_OK;
}

}  // namespace
}  // namespace h2

using namespace h2;

extern "C" h2_status h2_batched_qr_mindiag_static(int count, const int32_t *m, const int32_t *d,
                                                  const int64_t *off, const double *panels,
                                                  double *mindiag, h2_stream_t s) {
  if (count < 0 || (count > 0 && (!m || !d || !off || !panels || !mindiag)))
    return fail(H2_ERR_ARG, "h2_batched_qr_mindiag_static: bad arguments");
  if (count == 0) return H2_OK;
  // the offsets table sits at the front of the workspace
  const int64_t base = ((int64_t)count + 1 + 31) / 32 * 32;
  if (base >= kStaticQrDoubles)
    return fail(H2_ERR_ARG,
                "h2_batched_qr_mindiag_static: too many panels for the static workspace of "
                "2097152 doubles (its offsets table alone would not fit)");
  StaticAddr a;
  h2_status st = static_addresses(&a);
  if (st != H2_OK) return st;
  cudaStream_t stream = (cudaStream_t)s;
  int64_t *offs = reinterpret_cast<int64_t *>(a.scratch);
  // the flag keeps the previous call's value: clear it first
  cudaError_t e = cudaMemsetAsync(a.flag, 0, sizeof(int), stream);
  if (e == cudaSuccess) {
    k_static_offsets<<<1, 1024, 0, stream>>>(count, m, d, base, kStaticQrDoubles, offs, a.flag);
    k_qr_mindiag_static<<<count, 256, 0, stream>>>(count, m, d, off, panels, mindiag, a.scratch,
                                                   offs, kStaticQrDoubles, a.flag);
    count_launch(2);
    e = cudaGetLastError();
  }
  int host_flag = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&host_flag, a.flag, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess)
    return fail(H2_ERR_CUDA, std::string("h2_batched_qr_mindiag_static: ") + cudaGetErrorString(e));
  if (host_flag & kFlagShape)
    return fail(H2_ERR_ARG,
                "h2_batched_qr_mindiag_static: a panel has m < 0 or d < 1; its result is NaN");
  if (host_flag & kFlagOverflow)
    return fail(H2_ERR_ARG,
                "h2_batched_qr_mindiag_static: the panels with m > d need more than the static "
                "workspace of 2097152 doubles (sum of m*d plus the offsets table); results for "
                "the panels that did not fit are NaN");
  return H2_OK;
}
