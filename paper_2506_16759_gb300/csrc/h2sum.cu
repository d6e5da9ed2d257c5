// Entries of a sum of existing H2 matrices (the H2-update workload, Sec. V-A:
// the construction needs a function that evaluates sub-blocks of the operator
// being compressed; here the operator is sum_op H2_op on the same cluster
// tree and block partition as the matrix being built).
//
//  - Near-field blocks: D(t, b) = sum_op D_op(t, b).
//  - Couplings: for an admissible pair (s, t) at level l the operand block is
//    U_op,s B_op(s,t) U_op,t^T, so its entries at the new skeleton rows are
//    G_op,s B_op(s,t) G_op,t^T with G_op,s = U_op,s(Itil_s, :).  G follows the
//    nested bases: at a leaf G_s = U_op,s(J_s, :); above,
//    G_s = (blkdiag(G_op,nu1, G_op,nu2) E_op,s)(J_s, :), because the candidate
//    rows of s are the children's skeleton rows.
// Operands are FP64 or FP32 (built in mixed precision; their bases E are
// FP64 either way); the result is written in the target's precision.
#include <algorithm>

#include "h2_level.h"
#include "h2_types.h"

namespace h2 {
namespace {

__global__ void k_g_leaf(TasksDev t, const int32_t *kop, const int64_t *eoff_op,
                         const double *Eop, const int64_t *goff, double *G) {
  const int tau = blockIdx.x;
  const int kt = t.k[tau], ko = kop[tau], m = t.m[tau];
  const int32_t *J = t.J + t.krow[tau];
  const double *E = Eop + eoff_op[tau];
  double *out = G + goff[tau];
  for (int q = threadIdx.x; q < kt * ko; q += blockDim.x) {
    const int a = q % kt, c = q / kt;
    out[q] = E[J[a] + (int64_t)c * m];
  }
}

__global__ void k_g_inner(TasksDev t, const int32_t *child0, const int32_t *kt_child,
                          const int32_t *kop_child, const int64_t *goff_child,
                          const double *Gchild, const int32_t *kop, const int32_t *mop,
                          const int64_t *eoff_op, const double *Eop, const int64_t *goff,
                          double *G) {
  const int tau = blockIdx.x;
  const int kt = t.k[tau], ko = kop[tau], mo = mop[tau];
  const int c0 = child0[tau];
  const int kt1 = kt_child[c0];
  const int32_t *J = t.J + t.krow[tau];
  const double *E = Eop + eoff_op[tau];
  double *out = G + goff[tau];
  for (int q = threadIdx.x; q < kt * ko; q += blockDim.x) {
    const int a = q % kt, col = q / kt;
    const int j = J[a];
    const int c = j < kt1 ? 0 : 1;
    const int rho = c ? j - kt1 : j;
    const int child = c0 + c;
    const int kc = kop_child[child], ktc = kt_child[child];
    const int roff = c ? kop_child[c0] : 0;
    const double *Gc = Gchild + goff_child[child];
    double s = 0.0;
    for (int p = 0; p < kc; ++p) s += Gc[rho + (int64_t)p * ktc] * E[roff + p + (int64_t)col * mo];
    out[q] = s;
  }
}

template <typename T>
__global__ void k_b_h2sum(SumCouplingArgs a, int max_kop) {
  extern __shared__ double tmp[];   // [max_kop][kt]
  const int64_t e = blockIdx.x;
  const int s = a.erow[e], tt = a.idx[e];
  const int ks = a.t.k[s], kt = a.t.k[tt];
  if (ks == 0 || kt == 0) return;
  T *out = reinterpret_cast<T *>(a.B) + a.boff[e];
  for (int q = threadIdx.x; q < ks * kt; q += blockDim.x) out[q] = T(0);
  for (int o = 0; o < a.nops; ++o) {
    const SumOperand &op = a.ops[o];
    const int kos = op.k[s], kot = op.k[tt];
    const double *Gs = op.G + op.goff[s];
    const double *Gt = op.G + op.goff[tt];
    const double *Bo = op.B ? op.B + op.boff[e] : nullptr;
    const float *Bo32 = op.B32 ? op.B32 + op.boff[e] : nullptr;
    __syncthreads();
    // tmp = B_op G_t^T  (kos x kt)
    for (int q = threadIdx.x; q < kos * kt; q += blockDim.x) {
      const int p = q % kos, b = q / kos;
      double v = 0.0;
      if (Bo)
        for (int c = 0; c < kot; ++c) v += Bo[p + (int64_t)c * kos] * Gt[b + (int64_t)c * kt];
      else
        for (int c = 0; c < kot; ++c)
          v += (double)Bo32[p + (int64_t)c * kos] * Gt[b + (int64_t)c * kt];
      tmp[q] = v;
    }
    __syncthreads();
    // out += G_s tmp  (ks x kt)
    for (int q = threadIdx.x; q < ks * kt; q += blockDim.x) {
      const int r = q % ks, b = q / ks;
      double v = 0.0;
      for (int p = 0; p < kos; ++p) v += Gs[r + (int64_t)p * ks] * tmp[p + (int64_t)b * kos];
      out[q] = (T)((double)out[q] + v);
    }
  }
  (void)max_kop;
}

template <typename T>
__global__ void k_d_h2sum(int64_t nnz, const int32_t *erow, const int32_t *idx, const int32_t *m,
                          const int64_t *doff, T *D, const double *const *Dop,
                          const float *const *Dop32, const int64_t *const *doff_op, int nops) {
  const int64_t e = blockIdx.x;
  const int n = m[erow[e]] * m[idx[e]];
  T *out = D + doff[e];
  for (int q = threadIdx.x; q < n; q += blockDim.x) {
    double v = 0.0;
    for (int o = 0; o < nops; ++o)
      v += Dop[o] ? Dop[o][doff_op[o][e] + q] : (double)Dop32[o][doff_op[o][e] + q];
    out[q] = (T)v;
  }
}

}  // namespace

void h2sum_g_leaf(const TasksDev &t, const int32_t *kop, const int64_t *eoff_op, const double *Eop,
                  const int64_t *goff, double *G, cudaStream_t s) {
  if (t.n == 0) return;
  k_g_leaf<<<t.n, 128, 0, s>>>(t, kop, eoff_op, Eop, goff, G);
  count_launch();
  H2_CHECK_LAUNCH();
}

void h2sum_g_inner(const TasksDev &t, const int32_t *child0, const int32_t *kt_child,
                   const int32_t *kop_child, const int64_t *goff_child, const double *Gchild,
                   const int32_t *kop, const int32_t *mop, const int64_t *eoff_op,
                   const double *Eop, const int64_t *goff, double *G, cudaStream_t s) {
  if (t.n == 0) return;
  k_g_inner<<<t.n, 128, 0, s>>>(t, child0, kt_child, kop_child, goff_child, Gchild, kop, mop,
                                eoff_op, Eop, goff, G);
  count_launch();
  H2_CHECK_LAUNCH();
}

void h2sum_couplings(bool fp64, const SumCouplingArgs &a, int max_kop, int max_kt, cudaStream_t s) {
  if (a.nnz == 0) return;
  H2_REQUIRE(a.nnz < (1ll << 31), "too many coupling blocks");
  const size_t bytes = sizeof(double) * (size_t)std::max(max_kop, 1) * std::max(max_kt, 1);
  H2_REQUIRE(bytes <= 200 * 1024, "operand ranks too large for the H2-sum coupling kernel");
  if (fp64) {
    auto kern = k_b_h2sum<double>;
    if (bytes > 48 * 1024)
      H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    kern<<<(int)a.nnz, 128, bytes, s>>>(a, max_kop);
  } else {
    auto kern = k_b_h2sum<float>;
    if (bytes > 48 * 1024)
      H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    kern<<<(int)a.nnz, 128, bytes, s>>>(a, max_kop);
  }
  count_launch();
  H2_CHECK_LAUNCH();
}

void h2sum_dense(bool fp64, int64_t nnz, const int32_t *erow, const int32_t *idx, const int32_t *m,
                 const int64_t *doff, void *D, const double *const *Dop, const float *const *Dop32,
                 const int64_t *const *doff_op, int nops, cudaStream_t s) {
  if (nnz == 0) return;
  H2_REQUIRE(nnz < (1ll << 31), "too many near-field blocks");
  if (fp64)
    k_d_h2sum<double><<<(int)nnz, 256, 0, s>>>(nnz, erow, idx, m, doff, (double *)D, Dop, Dop32,
                                               doff_op, nops);
  else
    k_d_h2sum<float><<<(int)nnz, 256, 0, s>>>(nnz, erow, idx, m, doff, (float *)D, Dop, Dop32,
                                              doff_op, nops);
  count_launch();
  H2_CHECK_LAUNCH();
}

}  // namespace h2
