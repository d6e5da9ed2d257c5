// A variant of the batched QR convergence statistic that allocates no device
// memory.  Its working copies of the panels live in a fixed array that is part
// of the loaded library image, so callers that must not call cudaMalloc (for
// example code running inside a custom allocator callback, or a host that
// pre-reserves all device memory for itself) can still use it.
#include <mutex>

#include "h2_internal.cuh"

namespace h2 {
namespace {

// Capacity of the static workspace, in doubles (16 MiB).  Every device that
// loads the library holds this array until the process exits.
constexpr int64_t kStaticQrDoubles = int64_t(1) << 21;

static __device__ __align__(256) double g_static_qr_scratch[kStaticQrDoubles];
static __device__ int g_static_qr_overflow;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_addr[kMaxDevices] = {};
int *g_overflow_addr[kMaxDevices] = {};

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

// One CTA per panel: min_j |R_jj| of the Householder QR of panel t
// (m[t] x d[t], column-major at panels + off[t], ld = m[t]); 0 if m <= d.
// The working copy of panel t starts after the copies of all earlier panels
// that need a QR; a panel that does not fit raises the overflow flag and gets
// NaN.
__global__ void __launch_bounds__(256)
    k_qr_mindiag_static(int count, const int32_t *__restrict__ m, const int32_t *__restrict__ d,
                        const int64_t *__restrict__ off, const double *__restrict__ panels,
                        double *mindiag, double *scratch, int64_t cap, int *overflow) {
  __shared__ double red[33];
  int t = blockIdx.x;
  int mt = m[t], dt = d[t];
  if (mt <= dt) {
    if (threadIdx.x == 0) mindiag[t] = 0.0;
    return;
  }
  double before = 0.0;
  for (int i = threadIdx.x; i < t; i += blockDim.x)
    before += m[i] > d[i] ? (double)m[i] * (double)d[i] : 0.0;
  int64_t start = (int64_t)block_sum_d(before, red);
  int64_t need = (int64_t)mt * dt;
  if (start + need > cap) {
    if (threadIdx.x == 0) {
      atomicExch(overflow, 1);
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

// Device addresses of the static arrays for the current device, looked up
// once per device.  Host code must not pass the symbols themselves to a
// kernel: on the host they name host-side stand-ins.
h2_status static_addresses(double **scratch, int **overflow) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(H2_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(H2_ERR_ARG, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr, *q = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_qr_scratch);
    if (e != cudaSuccess)
      return fail(H2_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    e = cudaGetSymbolAddress(&q, g_static_qr_overflow);
    if (e != cudaSuccess)
      return fail(H2_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double *>(p);
    g_overflow_addr[dev] = static_cast<int *>(q);
  }
  *scratch = g_scratch_addr[dev];
  *overflow = g_overflow_addr[dev];
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
  double *scratch = nullptr;
  int *overflow = nullptr;
  h2_status st = static_addresses(&scratch, &overflow);
  if (st != H2_OK) return st;
  cudaStream_t stream = (cudaStream_t)s;
  // the flag keeps the previous call's value: clear it first
  cudaError_t e = cudaMemsetAsync(overflow, 0, sizeof(int), stream);
  if (e == cudaSuccess) {
    k_qr_mindiag_static<<<count, 256, 0, stream>>>(count, m, d, off, panels, mindiag, scratch,
                                                   kStaticQrDoubles, overflow);
    count_launch();
    e = cudaGetLastError();
  }
  int host_flag = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&host_flag, overflow, sizeof(int), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess)
    return fail(H2_ERR_CUDA, std::string("h2_batched_qr_mindiag_static: ") + cudaGetErrorString(e));
  if (host_flag)
    return fail(H2_ERR_ARG,
                "h2_batched_qr_mindiag_static: the panels with m > d need more than the static "
                "workspace of 2097152 doubles (sum of m*d); results for the panels that did not "
                "fit are NaN");
  return H2_OK;
}
