// Low-rank term U V^T of the operator: the update problem of Sec. V-A, an
// existing H2 matrix plus a rank-r product.  The sketch of the sum gets
// U (V^T Omega) added to the sampler's output (original point order), and
// every generated block (near-field D and couplings B) gets U(I, :) V(J, :)^T
// added to its entries, so that the construction sees the entries and the
// products of the whole operator.
#include "h2_internal.cuh"
#include "h2_level.h"

namespace h2 {
namespace {

constexpr int kLrMaxRank = 64;
constexpr int kLrRows = 32;        // rows of U / V / Omega staged per step
constexpr int kLrThreads = 256;
constexpr int kLrChunk = 80;       // sample columns per pass (r * 80 <= 5120 outputs)
constexpr int kLrMaxOut = kLrMaxRank * kLrChunk / kLrThreads;   // outputs per thread

// out[p * r + k] = src[orig[p] + k * ld]: tree-order rows of an N x r
// column-major factor, one contiguous row per point.
template <typename T>
__global__ void k_lr_tree_rows(const double *src, int64_t ld, const int32_t *orig, int64_t n,
                               int r, T *out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * r) return;
  const int64_t p = t / r;
  const int k = (int)(t % r);
  out[t] = (T)src[orig[p] + (int64_t)k * ld];
}

// partial[b][k * nc + c] = sum over the rows i of slice b of V(i, k) Om(i, c).
__global__ void __launch_bounds__(kLrThreads) k_lr_vt_partial(const double *V, int64_t ldv,
                                                              const double *om, int64_t ldo,
                                                              int64_t n, int r, int nc,
                                                              int64_t rows_per_cta,
                                                              double *partial) {
  __shared__ double sV[kLrRows][kLrMaxRank + 1];
  __shared__ double sO[kLrRows][kLrChunk + 1];
  const int64_t i_begin = blockIdx.x * rows_per_cta;
  const int64_t i_end = min(n, i_begin + rows_per_cta);
  const int nout = r * nc;
  double acc[kLrMaxOut];
#pragma unroll
  for (int q = 0; q < kLrMaxOut; ++q) acc[q] = 0.0;
  for (int64_t i0 = i_begin; i0 < i_end; i0 += kLrRows) {
    const int rows = (int)min((int64_t)kLrRows, i_end - i0);
    for (int u = threadIdx.x; u < kLrRows * r; u += kLrThreads) {
      const int ii = u % kLrRows, k = u / kLrRows;
      sV[ii][k] = ii < rows ? V[i0 + ii + (int64_t)k * ldv] : 0.0;
    }
    for (int u = threadIdx.x; u < kLrRows * nc; u += kLrThreads) {
      const int ii = u % kLrRows, c = u / kLrRows;
      sO[ii][c] = ii < rows ? om[i0 + ii + (int64_t)c * ldo] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kLrMaxOut; ++q) {
      const int o = threadIdx.x + q * kLrThreads;
      if (o < nout) {
        const int k = o / nc, c = o % nc;
        double s = 0.0;
        for (int ii = 0; ii < kLrRows; ++ii) s = fma(sV[ii][k], sO[ii][c], s);
        acc[q] += s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < kLrMaxOut; ++q) {
    const int o = threadIdx.x + q * kLrThreads;
    if (o < nout) partial[blockIdx.x * (int64_t)nout + o] = acc[q];
  }
}

__global__ void k_lr_reduce(const double *partial, int nb, int nout, double *W) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= nout) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += partial[(int64_t)b * nout + o];
  W[o] = s;
}

// y(i, c) += sum_k U(i, k) W(k, c) for columns c < nc (W row-major r x nc).
__global__ void k_lr_apply(const double *U, int64_t ldu, const double *W, int64_t n, int r, int nc,
                           double *y, int64_t ldy) {
  __shared__ double sW[kLrMaxRank * kLrChunk];
  for (int u = threadIdx.x; u < r * nc; u += blockDim.x) sW[u] = W[u];
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int c0 = 0; c0 < nc; c0 += 16) {
    double acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.0;
    for (int k = 0; k < r; ++k) {
      const double u = U[i + (int64_t)k * ldu];
      const double *w = sW + k * nc + c0;
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c0 + c < nc) acc[c] = fma(u, w[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 16; ++c)
      if (c0 + c < nc) y[i + (int64_t)(c0 + c) * ldy] += acc[c];
  }
}

// Block e of row task tr (m x mb, column-major at off[e]) += U(rows) V(cols)^T,
// the rows and columns being the tasks' points (leaves) or skeleton points
// (SKEL).  64 x 64 tiles of the block; the factor rows of both sides staged
// in shared memory, rows padded to r + 1 (conflict-free reads down a column).
template <typename T, bool SKEL>
__global__ void __launch_bounds__(256) k_lr_blocks(int n_rows, const int64_t *ptr,
                                                   const int32_t *idx, const int64_t *off,
                                                   const int32_t *rows_of, const int64_t *row0,
                                                   const int64_t *krow, const int32_t *skel,
                                                   const int32_t *cols_of, const int64_t *ckrow,
                                                   const int32_t *cskel, const T *Ut, const T *Vt,
                                                   int r, T *out) {
  extern __shared__ __align__(16) unsigned char lr_smem[];
  const int rs = r + 1;                       // padded row of a staged factor
  T *sU = reinterpret_cast<T *>(lr_smem);     // [64][rs]
  T *sV = sU + 64 * rs;                       // [64][rs]
  const int tr = blockIdx.x;
  if (tr >= n_rows) return;
  const int64_t e0 = ptr[tr], e1 = ptr[tr + 1];
  const int m = rows_of[tr];
  if (m == 0 || e0 == e1) return;
  auto gpos = [&](int task, int i) -> int64_t {
    return SKEL ? (int64_t)skel[krow[task] + i] : row0[task] + i;
  };
  // columns: the column side's skeletons where given (separate row and
  // column bases), else the rows' own
  auto gpos_c = [&](int task, int j) -> int64_t {
    return SKEL && cskel ? (int64_t)cskel[ckrow[task] + j] : gpos(task, j);
  };
  const int ii = threadIdx.x & 63, jg = threadIdx.x >> 6;
  for (int64_t e = e0; e < e1; ++e) {
    const int tc = idx[e];
    const int mb = cols_of ? cols_of[tc] : rows_of[tc];
    T *blk = out + off[e];
    for (int i0 = 0; i0 < m; i0 += 64) {
      const int mi = min(64, m - i0);
      for (int j0 = 0; j0 < mb; j0 += 64) {
        const int mj = min(64, mb - j0);
        for (int u = threadIdx.x; u < 64 * r; u += blockDim.x) {
          const int a = u / r, k = u % r;
          sU[a * rs + k] = a < mi ? Ut[gpos(tr, i0 + a) * r + k] : T(0);
          sV[a * rs + k] = a < mj ? Vt[gpos_c(tc, j0 + a) * r + k] : T(0);
        }
        __syncthreads();
        if (ii < mi) {
          for (int jj = jg; jj < mj; jj += 4) {
            T s = T(0);
            for (int k = 0; k < r; ++k) s += sU[ii * rs + k] * sV[jj * rs + k];
            blk[(i0 + ii) + (int64_t)(j0 + jj) * m] += s;
          }
        }
        __syncthreads();
      }
    }
  }
}

}  // namespace

void lowrank_tree_rows(bool fp64, const double *src, int64_t ld, const int32_t *orig, int64_t n,
                       int r, void *out, cudaStream_t s) {
  if (n == 0 || r == 0) return;
  const int blocks = ceil_div(n * r, 256);
  if (fp64) k_lr_tree_rows<double><<<blocks, 256, 0, s>>>(src, ld, orig, n, r, (double *)out);
  else k_lr_tree_rows<float><<<blocks, 256, 0, s>>>(src, ld, orig, n, r, (float *)out);
  count_launch();
  H2_CHECK_LAUNCH();
}

void lowrank_sample(const double *U, const double *V, int64_t ld, int64_t n, int r,
                    const double *om, int64_t ldo, int nc, double *y, int64_t ldy,
                    cudaStream_t s) {
  if (n == 0 || r == 0 || nc == 0) return;
  H2_REQUIRE(r <= kLrMaxRank, "low-rank term of rank above 64");
  const int nb = (int)std::min<int64_t>(ceil_div(n, 256), 1216);
  const int64_t rows_per_cta = (n + nb - 1) / nb;
  DBuf<double> partial, W;
  partial.alloc((size_t)nb * r * kLrChunk);
  W.alloc((size_t)r * kLrChunk);
  for (int c0 = 0; c0 < nc; c0 += kLrChunk) {
    const int w = std::min(kLrChunk, nc - c0);
    k_lr_vt_partial<<<nb, kLrThreads, 0, s>>>(V, ld, om + (int64_t)c0 * ldo, ldo, n, r, w,
                                              rows_per_cta, partial.p);
    count_launch();
    H2_CHECK_LAUNCH();
    k_lr_reduce<<<ceil_div(r * w, 256), 256, 0, s>>>(partial.p, nb, r * w, W.p);
    count_launch();
    H2_CHECK_LAUNCH();
    k_lr_apply<<<ceil_div(n, 128), 128, 0, s>>>(U, ld, W.p, n, r, w, y + (int64_t)c0 * ldy,
                                                ldy);
    count_launch();
    H2_CHECK_LAUNCH();
  }
}

void lowrank_blocks(bool fp64, bool skel_rows, int n_rows, const int64_t *ptr, const int32_t *idx,
                    const int64_t *off, const int32_t *rows_of, const int64_t *row0,
                    const int64_t *krow, const int32_t *skel, const void *Ut, const void *Vt,
                    int r, void *out, cudaStream_t s, const int32_t *cols_of,
                    const int64_t *ckrow, const int32_t *cskel) {
  if (n_rows == 0 || r == 0) return;
  H2_REQUIRE(r <= kLrMaxRank, "low-rank term of rank above 64");
  auto go = [&](auto T0, auto S0) {
    using T = decltype(T0);
    constexpr bool SK = decltype(S0)::value;
    const size_t bytes = sizeof(T) * 2 * 64 * (size_t)(r + 1);
    auto kern = k_lr_blocks<T, SK>;
    if (bytes > 48 * 1024)
      H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    kern<<<n_rows, 256, bytes, s>>>(n_rows, ptr, idx, off, rows_of, row0, krow, skel, cols_of,
                                    ckrow, cskel, (const T *)Ut, (const T *)Vt, r, (T *)out);
  };
  if (fp64) {
    if (skel_rows) go(double{}, std::true_type{});
    else go(double{}, std::false_type{});
  } else {
    if (skel_rows) go(float{}, std::true_type{});
    else go(float{}, std::false_type{});
  }
  count_launch();
  H2_CHECK_LAUNCH();
}

}  // namespace h2
