// Black-box sketch Y = K Omega (the K_blk of Algorithm 1, line 1 and the
// adaptive rounds of Sec. III-B) as a fused on-the-fly kernel summation:
// Y_i = sum_j K(x_i, x_j) Omega_j, the matrix K never stored.  Also the
// Gaussian test matrix (batchedRand), the dense-matrix sketch and single
// entry blocks (batchedGen for one block).
#include <algorithm>
#include <climits>

#include "h2_ops.h"
#include "h2_types.h"

namespace h2 {
namespace {

// ----------------------------------------------------------------------------
// Fused kernel summation, FP32 arithmetic on split hi/lo coordinates.
// Each thread owns one row and DC sample columns; the CTA streams TJ points
// (coordinates as two float4) and their Omega rows through shared memory.
// Each TJ-point tile is summed in plain FP32 and the tile sums are added with
// Kahan compensation, so the rounding of the N-term sum stays a few FP32 ulps
// instead of growing with sqrt(N).
// All-points mode sums j over [j0, j1).  Far-only mode (FAR) sums, for the
// rows of one leaf, over the leaves [lb0, lb1) that are not in its near list:
// that is Y_loc = Y - sum_b D_{t,b} Omega_b of Algorithm 1 without forming Y.
// ----------------------------------------------------------------------------
template <int KID, int DC, int NT, int TJ, bool FAR>
__global__ void __launch_bounds__(NT) k_ksum32(KsumArgs32 a, int tile_rows) {
  const KsumItem it = a.items[blockIdx.x];
  const InstDev in = a.inst[it.inst];
  const float scale = (float)in.kd.scale;
  const float diag = (float)in.kd.diag;
  const int pw = in.kd.pw;
  __shared__ float4 sh[TJ], sl[TJ];
  __shared__ __align__(16) float so[TJ][DC];

  const int lr = threadIdx.x;
  int64_t g = it.row0 + (lr < it.rows ? lr : 0);
  const float xh = a.pts.xh[g], yh = a.pts.yh[g], zh = a.pts.zh[g];
  const float xl = a.pts.xl[g], yl = a.pts.yl[g], zl = a.pts.zl[g];
  float acc[DC], cmp[DC];
#pragma unroll
  for (int c = 0; c < DC; ++c) { acc[c] = 0.f; cmp[c] = 0.f; }

  auto tile = [&](int64_t j, int nj) {
    for (int q = threadIdx.x; q < TJ; q += NT) {
      int64_t gj = j + (q < nj ? q : 0);
      sh[q] = make_float4(a.pts.xh[gj], a.pts.yh[gj], a.pts.zh[gj], 0.f);
      sl[q] = make_float4(a.pts.xl[gj], a.pts.yl[gj], a.pts.zl[gj], 0.f);
    }
    for (int q = threadIdx.x; q < TJ * DC; q += NT) {
      int jj = q % TJ, c = q / TJ;
      so[jj][c] = jj < nj ? a.om[(j + jj) + (int64_t)(it.c0 + c) * a.ld] : 0.f;
    }
    __syncthreads();
    float t[DC];
#pragma unroll
    for (int c = 0; c < DC; ++c) t[c] = 0.f;
    auto pair = [&](int jj) {
      const float4 ph = sh[jj], pl = sl[jj];
      const float gm = geom32<KID>(xh, yh, zh, xl, yl, zl, ph.x, ph.y, ph.z, pl.x, pl.y, pl.z);
      const float kv = kval<KID, float>(gm, scale, pw);
      const float4 *o4 = reinterpret_cast<const float4 *>(&so[jj][0]);
#pragma unroll
      for (int c4 = 0; c4 < DC / 4; ++c4) {
        const float4 o = o4[c4];
        t[4 * c4 + 0] = fmaf(kv, o.x, t[4 * c4 + 0]);
        t[4 * c4 + 1] = fmaf(kv, o.y, t[4 * c4 + 1]);
        t[4 * c4 + 2] = fmaf(kv, o.z, t[4 * c4 + 2]);
        t[4 * c4 + 3] = fmaf(kv, o.w, t[4 * c4 + 3]);
      }
    };
    if (nj == TJ) {
#pragma unroll 4
      for (int jj = 0; jj < TJ; ++jj) pair(jj);
    } else {
      for (int jj = 0; jj < nj; ++jj) pair(jj);
    }
#pragma unroll
    for (int c = 0; c < DC; ++c) {
      float y = t[c] - cmp[c];
      float s = acc[c] + y;
      cmp[c] = (s - acc[c]) - y;
      acc[c] = s;
    }
    __syncthreads();
  };

  if (!FAR) {
    for (int64_t j = it.j0; j < it.j1; j += TJ) tile(j, (int)(it.j1 - j < TJ ? it.j1 - j : TJ));
  } else {
    int64_t p = a.far.near_ptr[it.task];
    const int64_t pe = a.far.near_ptr[it.task + 1];
    for (int b = it.lb0; b < it.lb1; ++b) {
      while (p < pe && a.far.near_idx[p] < b) ++p;
      if (p < pe && a.far.near_idx[p] == b) continue;
      const int64_t r0 = a.far.leaf_row[b];
      const int mb = a.far.leaf_m[b];
      for (int q = 0; q < mb; q += TJ) tile(r0 + q, mb - q < TJ ? mb - q : TJ);
    }
  }
  if (lr >= it.rows) return;
  g = it.row0 + lr;
  if (!FAR && KID != H2_K_POLY && g >= it.j0 && g < it.j1 && diag != 0.f) {
#pragma unroll
    for (int c = 0; c < DC; ++c) acc[c] += diag * a.om[g + (int64_t)(it.c0 + c) * a.ld];
  }
  if (it.part < 0) {
#pragma unroll
    for (int c = 0; c < DC; ++c) a.y[g + (int64_t)(it.c0 + c) * a.ld] = acc[c];
  } else {
    float *dst = a.partial + (int64_t)it.part * tile_rows * DC;
#pragma unroll
    for (int c = 0; c < DC; ++c) dst[c * tile_rows + lr] = acc[c];
  }
}

// Same summation in FP64 (no compensation needed).
template <int KID, int DC, int NT, int TJ, bool FAR>
__global__ void __launch_bounds__(NT) k_ksum64(KsumArgs64 a, int tile_rows) {
  const KsumItem it = a.items[blockIdx.x];
  const InstDev in = a.inst[it.inst];
  const double scale = in.kd.scale;
  const double diag = in.kd.diag;
  const int pw = in.kd.pw;
  __shared__ double sp[3][TJ];
  __shared__ __align__(16) double so[TJ][DC];
  const int lr = threadIdx.x;
  int64_t g = it.row0 + (lr < it.rows ? lr : 0);
  const double xi = a.pts.x[g], yi = a.pts.y[g], zi = a.pts.z[g];
  double acc[DC];
#pragma unroll
  for (int c = 0; c < DC; ++c) acc[c] = 0.0;
  auto tile = [&](int64_t j, int nj) {
    for (int q = threadIdx.x; q < TJ; q += NT) {
      int64_t gj = j + (q < nj ? q : 0);
      sp[0][q] = a.pts.x[gj]; sp[1][q] = a.pts.y[gj]; sp[2][q] = a.pts.z[gj];
    }
    for (int q = threadIdx.x; q < TJ * DC; q += NT) {
      int jj = q % TJ, c = q / TJ;
      so[jj][c] = jj < nj ? a.om[(j + jj) + (int64_t)(it.c0 + c) * a.ld] : 0.0;
    }
    __syncthreads();
    for (int jj = 0; jj < nj; ++jj) {
      double gm = geom64<KID>(xi, yi, zi, sp[0][jj], sp[1][jj], sp[2][jj]);
      double kv = kval<KID, double>(gm, scale, pw);
      const double2 *o2 = reinterpret_cast<const double2 *>(&so[jj][0]);
#pragma unroll
      for (int c2 = 0; c2 < DC / 2; ++c2) {
        double2 o = o2[c2];
        acc[2 * c2] = fma(kv, o.x, acc[2 * c2]);
        acc[2 * c2 + 1] = fma(kv, o.y, acc[2 * c2 + 1]);
      }
    }
    __syncthreads();
  };
  if (!FAR) {
    for (int64_t j = it.j0; j < it.j1; j += TJ) tile(j, (int)(it.j1 - j < TJ ? it.j1 - j : TJ));
  } else {
    int64_t p = a.far.near_ptr[it.task];
    const int64_t pe = a.far.near_ptr[it.task + 1];
    for (int b = it.lb0; b < it.lb1; ++b) {
      while (p < pe && a.far.near_idx[p] < b) ++p;
      if (p < pe && a.far.near_idx[p] == b) continue;
      const int64_t r0 = a.far.leaf_row[b];
      const int mb = a.far.leaf_m[b];
      for (int q = 0; q < mb; q += TJ) tile(r0 + q, mb - q < TJ ? mb - q : TJ);
    }
  }
  if (lr >= it.rows) return;
  g = it.row0 + lr;
  if (!FAR && KID != H2_K_POLY && g >= it.j0 && g < it.j1 && diag != 0.0) {
#pragma unroll
    for (int c = 0; c < DC; ++c) acc[c] += diag * a.om[g + (int64_t)(it.c0 + c) * a.ld];
  }
  if (it.part < 0) {
#pragma unroll
    for (int c = 0; c < DC; ++c) a.y[g + (int64_t)(it.c0 + c) * a.ld] = acc[c];
  } else {
    double *dst = a.partial + (int64_t)it.part * tile_rows * DC;
#pragma unroll
    for (int c = 0; c < DC; ++c) dst[c * tile_rows + lr] = acc[c];
  }
}

// Sums the partial slots of each output tile in slot order (deterministic).
template <typename T>
__global__ void k_ksum_reduce(const KsumPlan::Red *reds, const T *partial, T *y, int64_t ld,
                              int tile_rows, int dc) {
  const KsumPlan::Red rd = reds[blockIdx.x];
  for (int q = threadIdx.x; q < rd.rows * dc; q += blockDim.x) {
    int lr = q % rd.rows, c = q / rd.rows;
    T s = T(0);
    for (int k = 0; k < rd.nslots; ++k)
      s += partial[(rd.slot0 + k) * tile_rows * dc + (int64_t)c * tile_rows + lr];
    y[rd.row0 + lr + (int64_t)(rd.c0 + c) * ld] = s;
  }
}

// Records events around one launch when a KernelTimer is installed.
struct KernelEvents {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  explicit KernelEvents(cudaStream_t st) : s(st) {
    if (!g_ksum_timer) return;
    H2_CUDA(cudaEventCreate(&a));
    H2_CUDA(cudaEventCreate(&b));
    H2_CUDA(cudaEventRecord(a, s));
  }
  void stop() {
    if (a) H2_CUDA(cudaEventRecord(b, s));
  }
  ~KernelEvents() {
    if (!a) return;
    float ms = 0.f;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess) {
      g_ksum_timer->ms += ms;
      g_ksum_timer->launches += 1;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

template <typename T>
struct StagedPlan {
  DBuf<KsumItem> items;
  DBuf<KsumPlan::Red> reds;
  DBuf<T> partial;
};

template <typename T>
void stage_plan(const KsumPlan &p, StagedPlan<T> &sp, cudaStream_t s) {
  to_device(sp.items, p.items, s);
  to_device(sp.reds, p.reds, s);
  sp.partial.alloc((size_t)p.n_parts * p.tile_rows * p.dc);
}

// ----------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void philox_round(uint32_t &c0, uint32_t &c1, uint32_t &c2,
                                             uint32_t &c3, uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
  uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
  uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
  c0 = n0; c1 = n1; c2 = n2; c3 = n3;
}

__device__ __forceinline__ void philox4x32_10(uint32_t ctr[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    philox_round(ctr[0], ctr[1], ctr[2], ctr[3], k0, k1);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// F32: the Box-Muller transform of 24-bit uniforms in FP32 arithmetic (the
// mixed-precision builds consume FP32 samples; GB300's FP64 logarithm and
// sine are slow), else of 53-bit uniforms in FP64.
template <bool F32>
__global__ void k_philox_gauss(double *om, int64_t ld, const int32_t *orig, int64_t n, int c0,
                               int c1, uint64_t seed) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t oi = (uint32_t)orig[i];
  for (int c = c0 & ~1; c < c1; c += 2) {
    uint32_t ctr[4] = {oi, (uint32_t)(c >> 1), 0x48324742u, 0u};
    philox4x32_10(ctr, (uint32_t)seed, (uint32_t)(seed >> 32));
    double z0, z1;
    if constexpr (F32) {
      const float u1 = ((float)(ctr[0] >> 8) + 0.5f) * 0x1.0p-24f;
      const float u2 = ((float)(ctr[2] >> 8) + 0.5f) * 0x1.0p-24f;
      const float rad = sqrtf(-2.0f * logf(u1));
      float sn, cs;
      sincospif(2.0f * u2, &sn, &cs);
      z0 = (double)(rad * cs);
      z1 = (double)(rad * sn);
    } else {
      uint64_t a = ((uint64_t)ctr[0] << 32 | ctr[1]) >> 11;
      uint64_t b = ((uint64_t)ctr[2] << 32 | ctr[3]) >> 11;
      double u1 = ((double)a + 0.5) * 0x1.0p-53;
      double u2 = ((double)b + 0.5) * 0x1.0p-53;
      double rad = sqrt(-2.0 * log(u1));
      double sn, cs;
      sincospi(2.0 * u2, &sn, &cs);
      z0 = rad * cs;
      z1 = rad * sn;
    }
    if (c >= c0) om[i + (int64_t)c * ld] = z0;
    if (c + 1 < c1) om[i + (int64_t)(c + 1) * ld] = z1;
  }
}

__global__ void k_gather_rows(const double *src, int64_t ld_src, const int32_t *orig, int64_t n,
                              int c0, int c1, double *dst, int64_t ld_dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = orig[i];
  for (int c = c0; c < c1; ++c) dst[i + c * ld_dst] = src[o + c * ld_src];
}

__global__ void k_convert_cols(const double *src, int64_t ld, int64_t row0, int64_t n, int c0,
                               int c1, float *dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int c = c0; c < c1; ++c) dst[row0 + i + c * ld] = (float)src[row0 + i + c * ld];
}

__global__ void k_split32(const double *x, const double *y, const double *z, int64_t n, float *xh,
                          float *yh, float *zh, float *xl, float *yl, float *zl) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float a = (float)x[i], b = (float)y[i], c = (float)z[i];
  xh[i] = a; yh[i] = b; zh[i] = c;
  xl[i] = (float)(x[i] - (double)a);
  yl[i] = (float)(y[i] - (double)b);
  zl[i] = (float)(z[i] - (double)c);
}

// Dense FP64 GEMM tile: 64 rows x 32 columns per CTA, k-steps of 32.
// trans: C = A^T B (the transpose of a caller's operator, for the column
// sketch of a non-symmetric construction).
__global__ void __launch_bounds__(256) k_dense_gemm64(const double *A, int64_t lda, int64_t n,
                                                      const double *B, int64_t ldb, double *C,
                                                      int64_t ldc, int d, bool trans) {
  __shared__ double sa[32][65];
  __shared__ double sb[32][33];
  int64_t r0 = blockIdx.x * 64;
  int c0 = blockIdx.y * 32;
  int tr = threadIdx.x % 64;   // row within tile
  int tc = threadIdx.x / 64;   // column group (8 columns each)
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t k0 = 0; k0 < n; k0 += 32) {
    if (!trans) {
      for (int q = threadIdx.x; q < 64 * 32; q += 256) {
        int r = q % 64, k = q / 64;
        int64_t gr = r0 + r, gk = k0 + k;
        sa[k][r] = (gr < n && gk < n) ? A[gr + gk * lda] : 0.0;
      }
    } else {   // consecutive threads read consecutive k of one column of A
      for (int q = threadIdx.x; q < 64 * 32; q += 256) {
        int k = q % 32, r = q / 32;
        int64_t gr = r0 + r, gk = k0 + k;
        sa[k][r] = (gr < n && gk < n) ? A[gk + gr * lda] : 0.0;
      }
    }
    for (int q = threadIdx.x; q < 32 * 32; q += 256) {
      int k = q % 32, c = q / 32;
      int64_t gk = k0 + k;
      sb[k][c] = (gk < n && c0 + c < d) ? B[gk + (int64_t)(c0 + c) * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      double av = sa[k][tr];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = fma(av, sb[k][tc * 8 + q], acc[q]);
    }
    __syncthreads();
  }
  int64_t gr = r0 + tr;
  if (gr < n)
    for (int q = 0; q < 8; ++q) {
      int c = c0 + tc * 8 + q;
      if (c < d) C[gr + (int64_t)c * ldc] = acc[q];
    }
}

template <int KID>
__global__ void k_entry_block64(KernelDesc kd, Points64 p, const int32_t *rows, int64_t nr,
                                const int32_t *cols, int64_t nc, double *out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nr * nc) return;
  int64_t r = e % nr, c = e / nr;
  int32_t i = rows[r], j = cols[c];
  double g = geom64<KID>(p.x[i], p.y[i], p.z[i], p.x[j], p.y[j], p.z[j]);
  out[e] = i == j ? kdiag<KID, double>(g, kd.scale, kd.pw, kd.diag)
                  : kval<KID, double>(g, kd.scale, kd.pw);
}

__global__ void k_soa(const double *pts, int64_t n, int dim, double *x, double *y, double *z) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = pts[i * dim];
  y[i] = dim > 1 ? pts[i * dim + 1] : 0.0;
  z[i] = dim > 2 ? pts[i * dim + 2] : 0.0;
}

__global__ void k_to64(const float *src, int64_t n, double *dst) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)src[i];
}

template <typename T>
__global__ void k_sumsq_partial(const T *panel, const T *panel2, int64_t ld, const int64_t *base,
                                const int64_t *nn, int d, double *part) {
  // thread = rows r (grid stride) x every column: no index division, loads
  // coalesced along the rows
  const int inst = blockIdx.y;
  const int64_t b = base[inst], n = nn[inst];
  double s = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const T *p1 = panel + b + r;
    const T *p2 = panel2 ? panel2 + b + r : nullptr;
    for (int c = 0; c < d; ++c) {
      double v = (double)p1[(int64_t)c * ld];
      if (p2) v += (double)p2[(int64_t)c * ld];
      s += v * v;
    }
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[inst * gridDim.x + blockIdx.x] = sh[0];
}

__global__ void k_sumsq_final(const double *part, int nb, int count, double *out) {
  int inst = blockIdx.x * blockDim.x + threadIdx.x;
  if (inst >= count) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[inst * nb + b];
  out[inst] = s;
}

template <int KID, int DC, bool FAR>
void launch_ksum32(const KsumPlan &p, const KsumArgs32 &a0, cudaStream_t s) {
  constexpr int NT = FAR ? 64 : 128, TJ = 64;
  StagedPlan<float> sp;
  stage_plan(p, sp, s);
  KsumArgs32 a = a0;
  a.items = sp.items.p;
  a.partial = sp.partial.p;
  KernelEvents ev(s);
  k_ksum32<KID, DC, NT, TJ, FAR><<<(int)p.items.size(), NT, 0, s>>>(a, p.tile_rows);
  ev.stop();
  count_launch();
  H2_CHECK_LAUNCH();
  if (!p.reds.empty()) {
    k_ksum_reduce<float><<<(int)p.reds.size(), 256, 0, s>>>(sp.reds.p, sp.partial.p, a.y, a.ld,
                                                             p.tile_rows, DC);
    count_launch();
    H2_CHECK_LAUNCH();
  }
  H2_CUDA(cudaStreamSynchronize(s));  // staging buffers die with this scope
}

template <int KID, int DC, bool FAR>
void launch_ksum64(const KsumPlan &p, const KsumArgs64 &a0, cudaStream_t s) {
  constexpr int NT = FAR ? 64 : 128, TJ = 32;
  StagedPlan<double> sp;
  stage_plan(p, sp, s);
  KsumArgs64 a = a0;
  a.items = sp.items.p;
  a.partial = sp.partial.p;
  KernelEvents ev(s);
  k_ksum64<KID, DC, NT, TJ, FAR><<<(int)p.items.size(), NT, 0, s>>>(a, p.tile_rows);
  ev.stop();
  count_launch();
  H2_CHECK_LAUNCH();
  if (!p.reds.empty()) {
    k_ksum_reduce<double><<<(int)p.reds.size(), 256, 0, s>>>(sp.reds.p, sp.partial.p, a.y, a.ld,
                                                              p.tile_rows, DC);
    count_launch();
    H2_CHECK_LAUNCH();
  }
  H2_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

KsumPlan plan_ksum(const std::vector<int64_t> &inst_n, const std::vector<int64_t> &inst_base,
                   const std::vector<int> &insts, const std::vector<int> &c0, int ncols,
                   bool fp64, int tile_rows_hint, int sm_count) {
  KsumPlan p;
  p.tile_rows = 128;
  (void)tile_rows_hint;
  p.dc = ncols;
  int64_t tiles = 0;
  for (int i : insts) tiles += (inst_n[i] + p.tile_rows - 1) / p.tile_rows;
  // aim for several waves of equal-cost items (4 resident CTAs per SM)
  int64_t target = (int64_t)sm_count * 4 * 6;
  struct Tmp {
    int64_t work;
    KsumItem it;
  };
  std::vector<Tmp> all;
  for (size_t q = 0; q < insts.size(); ++q) {
    int i = insts[q];
    int64_t n = inst_n[i], base = inst_base[i];
    int64_t rt = (n + p.tile_rows - 1) / p.tile_rows;
    int64_t S = tiles > 0 ? (target + tiles - 1) / tiles : 1;
    S = std::max<int64_t>(1, std::min<int64_t>(S, std::min<int64_t>(32, n / 1024)));
    for (int64_t t = 0; t < rt; ++t) {
      int rows = (int)std::min<int64_t>(p.tile_rows, n - t * p.tile_rows);
      int64_t slot0 = p.n_parts;
      for (int64_t sidx = 0; sidx < S; ++sidx) {
        KsumItem it;
        it.inst = i;
        it.rows = rows;
        it.row0 = base + t * p.tile_rows;
        it.j0 = base + (n * sidx) / S;
        it.j1 = base + (n * (sidx + 1)) / S;
        it.c0 = c0[q];
        it.part = S > 1 ? (int)(p.n_parts++) : -1;
        all.push_back({(it.j1 - it.j0) * rows, it});
      }
      if (S > 1) p.reds.push_back({i, rows, base + t * p.tile_rows, c0[q], slot0, (int)S});
    }
  }
  // heaviest items first so that the tail of the grid is short
  std::stable_sort(all.begin(), all.end(),
                   [](const Tmp &a, const Tmp &b) { return a.work > b.work; });
  p.items.reserve(all.size());
  for (auto &t : all) p.items.push_back(t.it);
  return p;
}

KsumPlan plan_ksum_far(const std::vector<int64_t> &leaf_row, const std::vector<int32_t> &leaf_m,
                       const std::vector<int> &leaf_base, const std::vector<int> &leaf_count,
                       const std::vector<int> &insts, const std::vector<int> &c0, int ncols,
                       int sm_count, bool pair_leaves, int split) {
  KsumPlan p;
  const int per = pair_leaves ? 2 : 1;
  p.tile_rows = 64 * per;
  p.dc = ncols;
  int64_t tiles = 0;
  for (int i : insts) tiles += (leaf_count[i] + per - 1) / per;
  // work items in all: `split` per SM (32 by default)
  const int64_t target = (int64_t)sm_count * (split > 0 ? split : 32);
  struct Tmp {
    int64_t work;
    KsumItem it;
  };
  std::vector<Tmp> all;
  for (size_t q = 0; q < insts.size(); ++q) {
    const int i = insts[q];
    const int nl = leaf_count[i], lb = leaf_base[i];
    int64_t S = tiles > 0 ? (target + tiles - 1) / tiles : 1;
    S = std::max<int64_t>(1, std::min<int64_t>(S, std::min<int64_t>(16, nl / 8)));
    for (int t = lb; t < lb + nl; t += per) {
      const int nt = std::min(per, lb + nl - t);
      int rows = 0;
      for (int u = 0; u < nt; ++u) {
        H2_REQUIRE(leaf_m[t + u] <= 64, "far-only summation needs leaves of at most 64 points");
        rows += leaf_m[t + u];
      }
      const int64_t slot0 = p.n_parts;
      for (int64_t sidx = 0; sidx < S; ++sidx) {
        KsumItem it{};
        it.inst = i;
        it.rows = rows;
        it.row0 = leaf_row[t];
        it.c0 = c0[q];
        it.task = t;
        it.lb0 = lb + (int)((nl * sidx) / S);
        it.lb1 = lb + (int)((nl * (sidx + 1)) / S);
        it.part = S > 1 ? (int)(p.n_parts++) : -1;
        all.push_back({(int64_t)(it.lb1 - it.lb0) * rows, it});
      }
      if (S > 1) p.reds.push_back({i, rows, leaf_row[t], c0[q], slot0, (int)S});
    }
  }
  std::stable_sort(all.begin(), all.end(),
                   [](const Tmp &a, const Tmp &b) { return a.work > b.work; });
  for (auto &t : all) p.items.push_back(t.it);
  return p;
}

void run_ksum32(int kid, const KsumPlan &plan, const KsumArgs32 &a, cudaStream_t s, bool far) {
  if (plan.items.empty()) return;
  dispatch_kernel(kid, [&](auto K) {
    constexpr int KID = decltype(K)::value;
    auto go = [&](auto F) {
      constexpr bool FAR = decltype(F)::value;
      switch (plan.dc) {
        case 32: launch_ksum32<KID, 32, FAR>(plan, a, s); break;
        case 16: launch_ksum32<KID, 16, FAR>(plan, a, s); break;
        case 8: launch_ksum32<KID, 8, FAR>(plan, a, s); break;
        default: throw Error{H2_ERR_ARG, "sketch column block must be 8, 16 or 32"};
      }
    };
    if (far) go(std::true_type{});
    else go(std::false_type{});
  });
}

void run_ksum_tc(int kid, const KsumPlan &plan, const TcArgs &a0, int mode, bool f16,
                 cudaStream_t s) {
  if (plan.items.empty()) return;
  H2_REQUIRE(plan.tile_rows == 128 && plan.dc >= 1 && plan.dc <= kTcChunk,
             "tensor-core sketch needs 128-row tiles and at most 80 columns");
  StagedPlan<float> sp;
  stage_plan(plan, sp, s);
  DBuf<int> err;
  err.alloc_zero(1, s);
  TcArgs a = a0;
  a.items = sp.items.p;
  a.partial = sp.partial.p;
  a.err = err.p;
  a.ncol = plan.dc;
  {
    KernelEvents ev(s);
    launch_ksum_tc(kid, tc_chunk_ncol(plan.dc), mode, f16, (int64_t)plan.items.size(), a, s);
    ev.stop();
  }
  if (!plan.reds.empty()) {
    k_ksum_reduce<float><<<(int)plan.reds.size(), 256, 0, s>>>(sp.reds.p, sp.partial.p, a.y, a.ld,
                                                              plan.tile_rows, plan.dc);
    count_launch();
    H2_CHECK_LAUNCH();
  }
  if (to_host(err.p, 1, s)[0])
    throw Error{H2_ERR_TIMEOUT, "tensor-core sketch: an mbarrier wait ran out"};
}

KsumPlan plan_ksum_tc_near(const std::vector<int32_t> &leaf_m, const std::vector<int64_t> &leaf_row,
                           const std::vector<int> &leaf_base, const std::vector<int> &leaf_count,
                           const std::vector<int64_t> &near_ptr,
                           const std::vector<int32_t> &near_idx, const std::vector<int> &insts,
                           const std::vector<int> &c0, int ncols, std::vector<int32_t> &ul_leaf,
                           std::vector<int32_t> &ul_flags) {
  KsumPlan p;
  p.tile_rows = 128;
  p.dc = ncols;
  ul_leaf.clear();
  ul_flags.clear();
  for (size_t q = 0; q < insts.size(); ++q) {
    const int i = insts[q];
    const int lb = leaf_base[i], nl = leaf_count[i];
    for (int t = lb; t < lb + nl; t += 2) {
      const bool two = t + 1 < lb + nl;
      H2_REQUIRE(leaf_m[t] + (two ? leaf_m[t + 1] : 0) <= 128, "leaf pair above 128 rows");
      KsumItem it{};
      it.inst = i;
      it.rows = leaf_m[t] + (two ? leaf_m[t + 1] : 0);
      it.row0 = leaf_row[t];
      it.c0 = c0[q];
      it.task = t;
      it.part = -1;
      it.lb0 = (int)ul_leaf.size();
      // merge the sorted near lists of t and t+1
      int64_t a = near_ptr[t], ae = near_ptr[t + 1];
      int64_t b = two ? near_ptr[t + 1] : 0, be = two ? near_ptr[t + 2] : 0;
      while (a < ae || b < be) {
        const int va = a < ae ? near_idx[a] : INT32_MAX, vb = b < be ? near_idx[b] : INT32_MAX;
        const int v = std::min(va, vb);
        ul_leaf.push_back(v);
        ul_flags.push_back((va == v ? 0 : 1) | (vb == v ? 0 : 2));
        if (va == v) ++a;
        if (vb == v) ++b;
      }
      it.lb1 = (int)ul_leaf.size();
      p.items.push_back(it);
    }
  }
  H2_REQUIRE(ul_leaf.size() < (1u << 31), "near lists too long");
  return p;
}

KsumPlan plan_ksum_tc_all(const std::vector<int64_t> &inst_n, const std::vector<int64_t> &inst_base,
                          const std::vector<int> &leaf_base, const std::vector<int> &leaf_count,
                          const std::vector<int> &insts, const std::vector<int> &c0, int ncols,
                          int sm_count) {
  KsumPlan p;
  p.tile_rows = 128;
  p.dc = ncols;
  int64_t tiles = 0;
  for (int i : insts) tiles += (inst_n[i] + p.tile_rows - 1) / p.tile_rows;
  const int64_t target = (int64_t)sm_count * 24;
  struct Tmp {
    int64_t work;
    KsumItem it;
  };
  std::vector<Tmp> all;
  for (size_t q = 0; q < insts.size(); ++q) {
    const int i = insts[q];
    const int64_t n = inst_n[i], base = inst_base[i];
    const int nl = leaf_count[i], lb = leaf_base[i];
    const int64_t rt = (n + p.tile_rows - 1) / p.tile_rows;
    int64_t S = tiles > 0 ? (target + tiles - 1) / tiles : 1;
    S = std::max<int64_t>(1, std::min<int64_t>(S, std::min<int64_t>(32, nl / 4)));
    for (int64_t t = 0; t < rt; ++t) {
      const int rows = (int)std::min<int64_t>(p.tile_rows, n - t * p.tile_rows);
      const int64_t slot0 = p.n_parts;
      for (int64_t sidx = 0; sidx < S; ++sidx) {
        KsumItem it{};
        it.inst = i;
        it.rows = rows;
        it.row0 = base + t * p.tile_rows;
        it.c0 = c0[q];
        it.task = -1;
        it.lb0 = lb + (int)((nl * sidx) / S);
        it.lb1 = lb + (int)((nl * (sidx + 1)) / S);
        it.part = S > 1 ? (int)(p.n_parts++) : -1;
        all.push_back({(int64_t)(it.lb1 - it.lb0) * rows, it});
      }
      if (S > 1) p.reds.push_back({i, rows, base + t * p.tile_rows, c0[q], slot0, (int)S});
    }
  }
  std::stable_sort(all.begin(), all.end(),
                   [](const Tmp &a, const Tmp &b) { return a.work > b.work; });
  for (auto &t : all) p.items.push_back(t.it);
  return p;
}

void run_ksum64(int kid, const KsumPlan &plan, const KsumArgs64 &a, cudaStream_t s, bool far) {
  if (plan.items.empty()) return;
  dispatch_kernel(kid, [&](auto K) {
    constexpr int KID = decltype(K)::value;
    auto go = [&](auto F) {
      constexpr bool FAR = decltype(F)::value;
      switch (plan.dc) {
        case 32: launch_ksum64<KID, 32, FAR>(plan, a, s); break;
        case 16: launch_ksum64<KID, 16, FAR>(plan, a, s); break;
        case 8: launch_ksum64<KID, 8, FAR>(plan, a, s); break;
        default: throw Error{H2_ERR_ARG, "sketch column block must be 8, 16 or 32"};
      }
    };
    if (far) go(std::true_type{});
    else go(std::false_type{});
  });
}

void philox_gaussian64(double *om, int64_t ld, const int32_t *orig_of_pos, int64_t n, int c0,
                       int c1, uint64_t seed, bool f32_math, cudaStream_t s) {
  if (n == 0 || c1 <= c0) return;
  if (f32_math)
    k_philox_gauss<true><<<ceil_div(n, 256), 256, 0, s>>>(om, ld, orig_of_pos, n, c0, c1, seed);
  else
    k_philox_gauss<false><<<ceil_div(n, 256), 256, 0, s>>>(om, ld, orig_of_pos, n, c0, c1, seed);
  count_launch();
  H2_CHECK_LAUNCH();
}

void gather_rows64(const double *src, int64_t ld_src, const int32_t *orig_of_pos, int64_t n,
                   int c0, int c1, double *dst, int64_t ld_dst, cudaStream_t s) {
  if (n == 0 || c1 <= c0) return;
  k_gather_rows<<<ceil_div(n, 256), 256, 0, s>>>(src, ld_src, orig_of_pos, n, c0, c1, dst, ld_dst);
  count_launch();
  H2_CHECK_LAUNCH();
}

void convert_cols_to32(const double *src, int64_t ld, int64_t row0, int64_t n, int c0, int c1,
                       float *dst, cudaStream_t s) {
  if (n == 0 || c1 <= c0) return;
  k_convert_cols<<<ceil_div(n, 256), 256, 0, s>>>(src, ld, row0, n, c0, c1, dst);
  count_launch();
  H2_CHECK_LAUNCH();
}

void dense_gemm64(const double *a, int64_t lda, int64_t n, const double *om, int64_t ldo,
                  double *y, int64_t ldy, int d, cudaStream_t s, bool trans) {
  if (n == 0 || d == 0) return;
  dim3 grid(ceil_div(n, 64), ceil_div(d, 32));
  k_dense_gemm64<<<grid, 256, 0, s>>>(a, lda, n, om, ldo, y, ldy, d, trans);
  count_launch();
  H2_CHECK_LAUNCH();
}

void entry_block64(int kid, const KernelDesc &kd, Points64 pts, const int32_t *rows, int64_t nr,
                   const int32_t *cols, int64_t nc, double *out, cudaStream_t s) {
  if (nr * nc == 0) return;
  dispatch_kernel(kid, [&](auto K) {
    constexpr int KID = decltype(K)::value;
    k_entry_block64<KID><<<ceil_div(nr * nc, 256), 256, 0, s>>>(kd, pts, rows, nr, cols, nc, out);
    count_launch();
    H2_CHECK_LAUNCH();
  });
}

void split_coords32(const double *x, const double *y, const double *z, int64_t n, float *xh,
                    float *yh, float *zh, float *xl, float *yl, float *zl, cudaStream_t s) {
  if (n == 0) return;
  k_split32<<<ceil_div(n, 256), 256, 0, s>>>(x, y, z, n, xh, yh, zh, xl, yl, zl);
  count_launch();
  H2_CHECK_LAUNCH();
}

void split_points_soa(const double *pts, int64_t n, int dim, double *x, double *y, double *z,
                      cudaStream_t s) {
  if (n == 0) return;
  k_soa<<<ceil_div(n, 256), 256, 0, s>>>(pts, n, dim, x, y, z);
  count_launch();
  H2_CHECK_LAUNCH();
}

void convert_to64(const float *src, int64_t n, double *dst, cudaStream_t s) {
  if (n == 0) return;
  k_to64<<<ceil_div(n, 256), 256, 0, s>>>(src, n, dst);
  count_launch();
  H2_CHECK_LAUNCH();
}

void instance_sumsq(const void *panel, const void *panel2, bool fp64, int64_t ld,
                    const int64_t *inst_base, const int64_t *inst_n, int count, int d,
                    double *out, cudaStream_t s) {
  // about two CTAs per SM over all instances
  const int nb = std::max(4, std::min(256, 2 * device_sm_count() / std::max(count, 1)));
  DBuf<double> part;
  part.alloc((size_t)nb * count);
  dim3 grid(nb, count);
  if (fp64)
    k_sumsq_partial<double><<<grid, 256, 0, s>>>((const double *)panel, (const double *)panel2, ld,
                                                 inst_base, inst_n, d, part.p);
  else
    k_sumsq_partial<float><<<grid, 256, 0, s>>>((const float *)panel, (const float *)panel2, ld,
                                                inst_base, inst_n, d, part.p);
  count_launch();
  H2_CHECK_LAUNCH();
  k_sumsq_final<<<ceil_div(count, 128), 128, 0, s>>>(part.p, nb, count, out);
  count_launch();
  H2_CHECK_LAUNCH();
  H2_CUDA(cudaStreamSynchronize(s));
}

}  // namespace h2
