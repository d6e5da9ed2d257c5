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
#include "tc_ptx.cuh"

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

// Mixed-precision couplings of an H2 sum (target stored in FP32): FP32
// products on the CUDA cores, every 32-term chunk summed plainly and the
// chunks with compensation.  One CTA of 256 threads per far block (s, t);
// per pass over 64 target columns b0 .. b0+63:
//   T = B_op(s,t) G_op,t(b0.., :)^T  (kos x 64), in row passes of 128, into
//       shared memory (rows padded to 68 floats: aligned float4 reads);
//   out(r0.., b0..) += G_op,s(r0.., :) T, in row passes of 64.
// Operand ranks up to 256; target ranks of any size.
constexpr int kB32MaxKop = 256, kB32Ld = 68;
constexpr size_t kB32Smem =
    sizeof(float) * ((size_t)kB32MaxKop * kB32Ld + 32 * 128 + 32 * 64 + 32 * 64);

struct Kahan32 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

__global__ void __launch_bounds__(256, 2) k_b_h2sum32(SumCouplingArgs a) {
  extern __shared__ __align__(16) float b32_smem[];
  float *sT = b32_smem;                       // [kB32MaxKop][kB32Ld]
  float *sB = sT + kB32MaxKop * kB32Ld;       // [32][128]  B_op(p0 + pp, c0 + c)
  float *sG = sB + 32 * 128;                  // [32][64]   G_t(b0 + b, c0 + c)
  float *sS = sG + 32 * 64;                   // [32][64]   G_s(r0 + r, c0 + c)
  const int64_t e = blockIdx.x;
  const int s = a.erow[e], tt = a.idx[e];
  const int ks = a.t.k[s], kt = a.t.k[tt];
  if (ks == 0 || kt == 0) return;
  float *out = reinterpret_cast<float *>(a.B) + a.boff[e];
  const int t = threadIdx.x;
  for (int q = t; q < ks * kt; q += blockDim.x) out[q] = 0.f;
  const int tp = t & 31, tb = t >> 5;     // step 1: rows p0 + tp + 32 i, columns 8 tb + j
  const int tb2 = t & 15, tr = t >> 4;    // step 2: rows r0 + tr + 16 i, columns 4 tb2 + j
  for (int o = 0; o < a.nops; ++o) {
    const SumOperand &op = a.ops[o];
    const int kos = op.k[s], kot = op.k[tt];
    if (kos == 0 || kot == 0) continue;
    const double *Gs = op.G + op.goff[s];
    const double *Gt = op.G + op.goff[tt];
    const double *Bo = op.B ? op.B + op.boff[e] : nullptr;
    const float *Bo32 = op.B32 ? op.B32 + op.boff[e] : nullptr;
    for (int b0 = 0; b0 < kt; b0 += 64) {
      // ---- T = B_op G_t(b0.., :)^T
      for (int p0 = 0; p0 < kos; p0 += 128) {
        Kahan32 acc[4][8];
        for (int c0 = 0; c0 < kot; c0 += 32) {
          __syncthreads();
          for (int u = t; u < 32 * 128; u += 256) {
            const int c = u >> 7, pp = u & 127;
            const int p = p0 + pp, cc = c0 + c;
            float v = 0.f;
            if (p < kos && cc < kot) {
              const int64_t i = p + (int64_t)cc * kos;
              v = Bo ? (float)Bo[i] : Bo32[i];
            }
            sB[u] = v;
          }
          for (int u = t; u < 32 * 64; u += 256) {
            const int c = u >> 6, b = b0 + (u & 63);
            sG[u] = (b < kt && c0 + c < kot) ? (float)Gt[b + (int64_t)(c0 + c) * kt] : 0.f;
          }
          __syncthreads();
          float part[4][8];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) part[i][j] = 0.f;
#pragma unroll 4
          for (int c = 0; c < 32; ++c) {
            const float4 g0 = *reinterpret_cast<const float4 *>(sG + c * 64 + 8 * tb);
            const float4 g1 = *reinterpret_cast<const float4 *>(sG + c * 64 + 8 * tb + 4);
            const float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float bv = sB[c * 128 + tp + 32 * i];
#pragma unroll
              for (int j = 0; j < 8; ++j) part[i][j] = fmaf(bv, gv[j], part[i][j]);
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j].add(part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int p = p0 + tp + 32 * i;
          if (p < kos) {
#pragma unroll
            for (int j = 0; j < 8; ++j) sT[p * kB32Ld + 8 * tb + j] = acc[i][j].s;
          }
        }
      }
      // ---- out(r0.., b0..) += G_s(r0.., :) T
      for (int r0 = 0; r0 < ks; r0 += 64) {
        Kahan32 acc2[4][4];
        for (int c0 = 0; c0 < kos; c0 += 32) {
          __syncthreads();
          for (int u = t; u < 32 * 64; u += 256) {
            const int c = u >> 6, r = r0 + (u & 63);
            sS[u] = (r < ks && c0 + c < kos) ? (float)Gs[r + (int64_t)(c0 + c) * ks] : 0.f;
          }
          __syncthreads();
          float part[4][4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) part[i][j] = 0.f;
          const int cn = min(32, kos - c0);
          for (int c = 0; c < cn; ++c) {
            const float4 tv = *reinterpret_cast<const float4 *>(sT + (c0 + c) * kB32Ld + 4 * tb2);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float gv = sS[c * 64 + tr + 16 * i];
              part[i][0] = fmaf(gv, tv.x, part[i][0]);
              part[i][1] = fmaf(gv, tv.y, part[i][1]);
              part[i][2] = fmaf(gv, tv.z, part[i][2]);
              part[i][3] = fmaf(gv, tv.w, part[i][3]);
            }
          }
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc2[i][j].add(part[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int r = r0 + tr + 16 * i;
          if (r >= ks) continue;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int b = b0 + 4 * tb2 + j;
            if (b < kt) out[r + (int64_t)b * ks] += acc2[i][j].s;
          }
        }
      }
    }
  }
}

// Mixed-precision couplings of an H2 sum on the tensor cores (tcgen05,
// FP32 values carried as two TF32 parts, three part products per K step
// into an FP32 accumulator in tensor memory).  One CTA of 8 warps per far
// block (s, t); per operand and per 128-row tile p0.. of the operand's rank
// at s:
//   step 1  T = B_op(s,t)(p0.., :) G_op,t^T  (M = 128 rows p, N = k_t padded
//           to np, K = the operand's rank at t in chunks of 32): the block's
//           chunk goes into TMEM as operand A (thread = row p, 16 of the 32
//           columns per warp), G_op,t's chunk into a 128-byte-swizzled K-major
//           image in shared memory (operand B);
//   step 2  C += G_op,s(:, p0..) T  (M = 128 rows r of the target rank k_s,
//           N = np, K = the tile's rows p): T is read back from TMEM and
//           written as four K chunks of B images, G_op,s's columns go into
//           TMEM as operand A.
// C stays in TMEM across operands and is stored once.  Every product is
// waited for before its operands are overwritten (no pipelining: the
// kernel's time is the blocks' streaming and these round trips).  Target
// ranks up to 96 (k_s and k_t), operand ranks of any size.  Tensor memory:
// T and C (np columns each) and one A stage (64 columns), 256 columns, so two
// CTAs fit an SM.  Waits are bounded; a timeout sets *err.
constexpr int kHsMaxN = 96;

__device__ __forceinline__ int hs_sw(int row, int j) {   // element (row, j) of a swizzled image
  return row * 32 + (((j >> 2) ^ (row & 7)) << 2) + (j & 3);
}
__device__ __forceinline__ void hs_split(float v, uint32_t &h, uint32_t &l) {
  const float hh = tf32_rna(v);
  h = __float_as_uint(hh);
  l = __float_as_uint(v - hh);
}

__global__ void __launch_bounds__(256, 2) k_b_h2sum_tc(SumCouplingArgs a, int np, int *err) {
  extern __shared__ unsigned char hs_dyn[];
  float *img = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(hs_dyn) + 1023) &
                                         ~uintptr_t(1023));   // [4][2][np][32]
  __shared__ uint64_t done;
  __shared__ uint32_t tmem_base;
  const int64_t e = blockIdx.x;
  const int s = a.erow[e], tt = a.idx[e];
  const int ks = a.t.k[s], kt = a.t.k[tt];
  if (ks == 0 || kt == 0) return;   // uniform over the CTA
  float *out = reinterpret_cast<float *>(a.B) + a.boff[e];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int quad = warp & 3, half = warp >> 2;
  if (t == 0) {
    mbar_init(saddr(&done), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     saddr(&tmem_base)),
                 "n"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tb = tmem_base;
  const uint32_t t_col = tb, c_col = tb + np, a_col = tb + 2 * np;
  const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
  const uint32_t idesc = idesc_mma(false, 128, np);
  uint32_t phase = 0;
  bool ok = true, c_started = false;

  // operand A (16 of the chunk's 32 columns of this thread's row) into TMEM
  auto stage_a = [&](const float *v) {
    uint32_t hv[16], lv[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) hs_split(v[j], hv[j], lv[j]);
    const uint32_t at = a_col + lane_addr + 16 * half;
    tmem_st8(at, hv);
    tmem_st8(at + 8, hv + 8);
    tmem_st8(at + 32, lv);
    tmem_st8(at + 40, lv + 8);
    tmem_st_wait();
  };
  // D (+)= A * B with B = the image at bimg (hi rows, then lo rows), then
  // every thread waits for the products; false (everywhere) on a timeout.
  // `prefetch` runs between the issue and the wait (the next chunk's loads).
  auto product = [&](uint32_t d, const float *bimg, bool acc, auto &&prefetch) -> bool {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {
      const uint32_t h = saddr(bimg), l = h + (uint32_t)np * 128;
#pragma unroll
      for (int k8 = 0; k8 < 4; ++k8) {
        mma_ts<false>(d, a_col + k8 * 8, desc_sw128(h + k8 * 32), idesc, (acc || k8) ? 1u : 0u);
        mma_ts<false>(d, a_col + k8 * 8, desc_sw128(l + k8 * 32), idesc, 1u);
        mma_ts<false>(d, a_col + 32 + k8 * 8, desc_sw128(h + k8 * 32), idesc, 1u);
      }
      mma_commit(saddr(&done));
    }
    prefetch();
    const bool w = mbar_wait(saddr(&done), phase);
    phase ^= 1u;
    fence_after();
    return __syncthreads_and(w ? 1 : 0) != 0;
  };

  for (int o = 0; o < a.nops && ok; ++o) {
    const SumOperand &op = a.ops[o];
    const int kos = op.k[s], kot = op.k[tt];
    if (kos == 0 || kot == 0) continue;
    const double *Gs = op.G + op.goff[s];
    const double *Gt = op.G + op.goff[tt];
    const double *Bo = op.B ? op.B + op.boff[e] : nullptr;
    const float *Bo32 = op.B32 ? op.B32 + op.boff[e] : nullptr;
    for (int p0 = 0; p0 < kos && ok; p0 += 128) {
      const int mp = min(128, kos - p0);
      // ---- step 1: T = B_op(p0.., :) G_t^T.  This thread's share of a chunk:
      // 16 values of block row p (A) and up to 12 values of G_t's image
      // (element q = t + 256 u: image row q % np, column q / np); the next
      // chunk's share is loaded while the current chunk's products run.
      const int p = p0 + quad * 32 + lane;
      float bv[16], gv[12];
      auto load1 = [&](int c0) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int c = c0 + 16 * half + j;
          float x = 0.f;
          if (p < kos && c < kot) {
            const int64_t i = p + (int64_t)c * kos;
            x = Bo ? (float)Bo[i] : Bo32[i];
          }
          bv[j] = x;
        }
#pragma unroll
        for (int u = 0; u < 12; ++u) {
          const int q = t + 256 * u;
          const int b = q % np, j = q / np;
          gv[u] = (q < np * 32 && b < kt && c0 + j < kot) ? (float)Gt[b + (int64_t)(c0 + j) * kt]
                                                           : 0.f;
        }
      };
      load1(0);
      for (int c0 = 0; c0 < kot && ok; c0 += 32) {
        stage_a(bv);
#pragma unroll
        for (int u = 0; u < 12; ++u) {
          const int q = t + 256 * u;
          if (q < np * 32) {
            const int b = q % np, j = q / np;
            const float h = tf32_rna(gv[u]);
            img[hs_sw(b, j)] = h;
            img[np * 32 + hs_sw(b, j)] = gv[u] - h;
          }
        }
        ok = product(t_col, img, c0 > 0, [&]() {
          if (c0 + 32 < kot) load1(c0 + 32);
        });
      }
      if (!ok) break;
      // ---- T rows p0 + 32 w .. (warp quadrant w) -> the B image of step-2 chunk w
      const int nch = (mp + 31) / 32;
      if (quad < nch) {   // uniform per warp
        float *hi = img + quad * (np * 64), *lo = hi + np * 32;
        for (int b0 = 8 * half; b0 < np; b0 += 16) {
          float v[8];
          tmem_ld<8>(t_col + lane_addr + b0, v);
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const float h = tf32_rna(v[u]);
            hi[hs_sw(b0 + u, lane)] = h;
            lo[hs_sw(b0 + u, lane)] = v[u] - h;
          }
        }
      }
      // ---- step 2: C += G_s(:, p0..) T (the next chunk of G_s loaded while
      // the current products run)
      const int r = quad * 32 + lane;
      auto load2 = [&](int ch) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int pp = p0 + ch * 32 + 16 * half + j;
          bv[j] = (r < ks && pp < kos) ? (float)Gs[r + (int64_t)pp * ks] : 0.f;
        }
      };
      load2(0);
      for (int ch = 0; ch < nch && ok; ++ch) {
        stage_a(bv);
        ok = product(c_col, img + ch * (np * 64), c_started || ch > 0, [&]() {
          if (ch + 1 < nch) load2(ch + 1);
        });
        c_started = true;
      }
    }
  }
  if (ok) {
    const int r = quad * 32 + lane;
    for (int b0 = 8 * half; b0 < np; b0 += 16) {
      float v[8];
      if (c_started) {
        tmem_ld<8>(c_col + lane_addr + b0, v);
      } else {
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = 0.f;
      }
      if (r < ks) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (b0 + u < kt) out[r + (int64_t)(b0 + u) * ks] = v[u];
      }
    }
  } else if (t == 0) {
    atomicExch(err, 1);
    mbar_wait(saddr(&done), phase ^ 1u);   // once more before the memory is released
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tb), "n"(256));
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

void h2sum_couplings(bool fp64, const SumCouplingArgs &a, int max_kop, int max_kt, int engine,
                     cudaStream_t s) {
  if (a.nnz == 0) return;
  H2_REQUIRE(a.nnz < (1ll << 31), "too many coupling blocks");
  const size_t bytes = sizeof(double) * (size_t)std::max(max_kop, 1) * std::max(max_kt, 1);
  if (!fp64 && engine == 1 && max_kt <= kHsMaxN) {
    const int np = std::max(16, (max_kt + 15) / 16 * 16);
    const size_t smem = (size_t)np * 1024 + 1024;
    H2_CUDA(cudaFuncSetAttribute(k_b_h2sum_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    DBuf<int> err;
    err.alloc_zero(1, s);
    k_b_h2sum_tc<<<(int)a.nnz, 256, smem, s>>>(a, np, err.p);
    count_launch();
    H2_CHECK_LAUNCH();
    if (to_host(err.p, 1, s)[0] != 0)
      throw Error{H2_ERR_TIMEOUT, "tensor-core H2-sum couplings: a bounded wait ran out"};
    return;
  }
  if (!fp64 && max_kop <= kB32MaxKop) {
    H2_CUDA(cudaFuncSetAttribute(k_b_h2sum32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kB32Smem));
    k_b_h2sum32<<<(int)a.nnz, 256, kB32Smem, s>>>(a);
  } else if (fp64) {
    H2_REQUIRE(bytes <= 200 * 1024, "operand ranks too large for the H2-sum coupling kernel");
    auto kern = k_b_h2sum<double>;
    if (bytes > 48 * 1024)
      H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    kern<<<(int)a.nnz, 128, bytes, s>>>(a, max_kop);
  } else {
    H2_REQUIRE(bytes <= 200 * 1024, "operand ranks too large for the H2-sum coupling kernel");
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
