// Per-level batched kernels of Algorithm 1 (Sec. III-A/III-B):
//  - leaf near field: D = K(I_t, I_b) generated and stored while
//    Y_loc = Y - sum_b D Omega_b is accumulated (batchedGen + batchedBSRGemm);
//  - block-sparse products with stored D or B (adaptive re-sweeps, inner
//    far-field subtraction, matvec);
//  - the QR convergence test (min_j |R_jj| of Y_loc, FP64 Householder);
//  - the row ID by column-pivoted Householder QR of Y_loc^T/sqrt(d) (FP64);
//  - shrink (skeleton-row gather) and the Omega upsweep U^T Omega;
//  - couplings B = K(Itil_s, Itil_t).
// One CTA owns one cluster (row block), so no output is written by two CTAs.
#include <algorithm>

#include "h2_level.h"
#include "h2_types.h"

namespace h2 {
namespace {

constexpr int kNT = 256;   // threads per cluster CTA
constexpr int kMaxCols = 256;   // sample columns at most (d_max)
constexpr int kMaxRows = 256;     // rows of a block-product row task
constexpr int kMaxIdRows = 512;   // rows of a cluster in the QR test / row ID

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; every thread gets the result.  `sh` holds >= 33 doubles.
__device__ double block_sum(double v, double *sh) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double w = lane < nw ? sh[lane] : 0.0;
    w = warp_sum(w);
    if (lane == 0) sh[32] = w;
  }
  __syncthreads();
  double r = sh[32];
  __syncthreads();
  return r;
}

// Argmax over the CTA, lowest index on ties.  Every thread gets the index.
__device__ int block_argmax(double v, int idx, double *shv, int *shi) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  if (lane == 0) { shv[warp] = v; shi[warp] = idx; }
  __syncthreads();
  if (warp == 0) {
    double w = lane < nw ? shv[lane] : -1.0;
    int wi = lane < nw ? shi[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, w, o);
      int oi = __shfl_xor_sync(0xffffffffu, wi, o);
      if (ov > w || (ov == w && oi < wi)) { w = ov; wi = oi; }
    }
    if (lane == 0) shi[32] = wi;
  }
  __syncthreads();
  int r = shi[32];
  __syncthreads();
  return r;
}

// Running sum of per-chunk partial sums: FP64 adds directly, FP32 with
// Kahan compensation (the chunk sums are short, the running sum is long).
template <typename T>
struct Acc {
  T s = T(0);
  __device__ void add(T v) { s += v; }
  __device__ T value() const { return s; }
};
template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ void add(float v) {
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ float value() const { return s; }
};

template <typename T>
struct PtsOf;
template <>
struct PtsOf<double> {
  __device__ static void load(const Points64 &p, const Points32 &, int64_t g, double *c) {
    c[0] = p.x[g]; c[1] = p.y[g]; c[2] = p.z[g];
  }
  template <int KID>
  __device__ static double geom(const double *a, const double *b) {
    return geom64<KID>(a[0], a[1], a[2], b[0], b[1], b[2]);
  }
  static constexpr int NC = 3;
};
template <>
struct PtsOf<float> {
  __device__ static void load(const Points64 &, const Points32 &p, int64_t g, float *c) {
    c[0] = p.xh[g]; c[1] = p.yh[g]; c[2] = p.zh[g];
    c[3] = p.xl[g]; c[4] = p.yl[g]; c[5] = p.zl[g];
  }
  template <int KID>
  __device__ static float geom(const float *a, const float *b) {
    return geom32<KID>(a[0], a[1], a[2], a[3], a[4], a[5], b[0], b[1], b[2], b[3], b[4], b[5]);
  }
  static constexpr int NC = 6;
};

// ----------------------------------------------------------------------------
// Block-sparse row products: out(rows of t) += sign * sum_e Blk_e in(rows of b_e).
//
// One CTA owns one row block (all of its m <= 256 rows).  Its partner blocks
// are stored contiguously (column-major, 16-byte aligned offsets), so a chunk
// of JC block columns is one contiguous range; chunks stream through a
// three-slot shared-memory ring filled with cp.async (16-byte copies, L2 only)
// together with the matching JC input rows, two chunks ahead of the compute.
// Thread t owns rows t%64 + 64r (r < RPT) and DC/4 output columns
// (t/64)*DC/4 ...; each chunk is summed plainly, chunk sums are added with
// compensation in FP32.  No output is shared between threads or CTAs.
// ----------------------------------------------------------------------------
constexpr int kStages = 3;
constexpr int kSlotBytes = 16384;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
template <int B>
__device__ __forceinline__ void cp_async_small(void *smem, const void *gmem, bool valid) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  int src = valid ? B : 0;  // src-size 0 fills the destination with zeros
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(sa), "l"(gmem), "n"(B),
               "r"(src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

template <typename T, int DC, int RPT>
__global__ void __launch_bounds__(kNT, sizeof(T) == 4 ? 2 : 1) k_bsr_pipe(BsrArgs a) {
  constexpr int SLOT = kSlotBytes / sizeof(T);   // block elements per slot
  constexpr int JMAX = 64;                        // block columns per chunk at most
  constexpr int CG = DC / 4;                      // output columns per thread
  constexpr int DCP = DC + 4;                     // padded row of the input slot
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *sBlk = reinterpret_cast<T *>(smem_raw);               // [kStages][SLOT]
  T *sIn = sBlk + kStages * SLOT;                          // [kStages][JMAX][DC + 4]
  // a.seg CTAs share a row task, each a contiguous part of its CSR row
  const int tau = blockIdx.x / a.seg, part_id = blockIdx.x % a.seg;
  const int m = a.row_m[tau];
  const int inst = a.row_inst[tau];
  const int cb = a.cols.cb[inst], ce = a.cols.ce[inst];
  const int64_t r0 = a.ptr[tau], rn = a.ptr[tau + 1] - r0;
  const int64_t e0 = r0 + rn * part_id / a.seg, e1 = r0 + rn * (part_id + 1) / a.seg;
  if (m == 0 || ce <= cb || e0 == e1) return;
  // block columns per chunk: fits a slot, multiple of 4 (16-byte aligned starts)
  int jc = SLOT / m;
  jc = jc > JMAX ? JMAX : jc;
  jc &= ~3;
  const int i0 = threadIdx.x % 64, g = threadIdx.x / 64;
  const int64_t orow = a.row_off[tau];
  const T *blocks = reinterpret_cast<const T *>(a.blocks);
  const T *in = reinterpret_cast<const T *>(a.in);
  T *out = reinterpret_cast<T *>(a.out);
  for (int c0 = cb; c0 < ce; c0 += DC) {
    const int ncol = min(DC, ce - c0);
    Acc<T> acc[RPT][CG];
    // producer state (chunk to issue) and consumer state (chunk to compute)
    int64_t pe = e0;
    int pj = 0;
    int64_t ce_ = e0;
    int cj = 0;
    auto issue = [&](int slot) {
      if (pe < e1) {
        const int b = a.idx[pe];
        const int mb = a.col_m[b];
        const int nj = min(jc, mb - pj);
        const T *src = blocks + a.boff[pe] + (int64_t)pj * m;
        const int n16 = (int)(((int64_t)nj * m * sizeof(T) + 15) / 16);
        char *dst = reinterpret_cast<char *>(sBlk + slot * SLOT);
        for (int u = threadIdx.x; u < n16; u += kNT)
          cp_async16(dst + 16 * u, reinterpret_cast<const char *>(src) + 16 * u);
        const int64_t irow = a.col_off[b] + pj;
        T *di = sIn + slot * JMAX * DCP;
        // consecutive threads take consecutive rows of one column (coalesced
        // reads; the padded row keeps the shared-memory writes spread over banks)
        for (int q = threadIdx.x; q < JMAX * DC; q += kNT) {
          const int j = q % JMAX, c = q / JMAX;
          const bool ok = j < nj && c < ncol;
          const T *sp = ok ? in + irow + j + (int64_t)(c0 + c) * a.ld_in : in;
          cp_async_small<sizeof(T)>(di + j * DCP + c, sp, ok);
        }
        pj += nj;
        if (pj >= mb) { pj = 0; ++pe; }
      }
      cp_async_commit();
    };
    for (int st = 0; st < kStages - 1; ++st) issue(st);
    // plain sums over one block's chunks, compensated sums across blocks
    T part[RPT][CG];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int c = 0; c < CG; ++c) part[r][c] = T(0);
    for (int it = 0; ce_ < e1; ++it) {
      issue((it + kStages - 1) % kStages);
      cp_async_wait<kStages - 1>();
      __syncthreads();
      const int slot = it % kStages;
      const int mb = a.col_m[a.idx[ce_]];
      const int nj = min(jc, mb - cj);
      const T *sb = sBlk + slot * SLOT;
      const T *si = sIn + slot * JMAX * DCP + g * CG;
      for (int j = 0; j < nj; ++j) {
        T ov[CG];
        if constexpr (sizeof(T) == 4 && CG % 4 == 0) {
          // 16-byte rows: DCP and the group offset are multiples of 4 floats
#pragma unroll
          for (int c = 0; c < CG; c += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(si + j * DCP + c);
            ov[c] = v.x; ov[c + 1] = v.y; ov[c + 2] = v.z; ov[c + 3] = v.w;
          }
        } else {
#pragma unroll
          for (int c = 0; c < CG; ++c) ov[c] = si[j * DCP + c];
        }
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          if (64 * r >= m) break;   // row groups past the block (uniform over the CTA)
          // rows at or past m read other words of the shared buffers (at most
          // 63 past the slot) and are never stored
          const T bv = sb[j * m + i0 + 64 * r];
#pragma unroll
          for (int c = 0; c < CG; ++c) part[r][c] += bv * ov[c];
        }
      }
      cj += nj;
      if (cj >= mb) {
        cj = 0;
        ++ce_;
        const T sgn = (T)a.sign;
#pragma unroll
        for (int r = 0; r < RPT; ++r)
#pragma unroll
          for (int c = 0; c < CG; ++c) {
            acc[r][c].add(sgn * part[r][c]);
            part[r][c] = T(0);
          }
      }
      __syncthreads();
    }
    cp_async_wait<0>();
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int i = i0 + 64 * r;
      if (i >= m) continue;
#pragma unroll
      for (int c = 0; c < CG; ++c) {
        const int col = g * CG + c;
        if (col < ncol) {
          T *op = out + orow + i + (int64_t)(c0 + col) * a.ld_out;
          if (a.seg > 1) {
            atomicAdd(op, acc[r][c].value());
          } else {
            Acc<T> t = acc[r][c];
            t.add(*op);
            *op = t.value();
          }
        }
      }
    }
  }
}

// ----------------------------------------------------------------------------
// FP32 block-sparse row products with register tiles (blocks of at most 64 x
// 64).  One CTA per row block; thread (rg, cg) owns rows rg, rg+16, rg+32,
// rg+48 (a warp's 16 row groups read 16 consecutive words of a block column:
// no bank conflicts) and columns 4cg..4cg+3 of a DC-column chunk.  The partner
// blocks stream through a two-slot ring (cp.async, 16-byte copies): the block
// itself (contiguous, column-major) and its DC-column slice of the input rows,
// read from a row-major copy of the input panel so that every row slice is
// contiguous.  Rows at or past the block's height read other words of the
// slot and are never stored, so the inner loop has no bounds tests.  Each
// block's product is summed plainly, the blocks with compensation.
// ----------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16z(void *smem, const void *gmem, bool valid) {
  unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  int src = valid ? 16 : 0;   // src-size 0 fills the destination with zeros
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src));
}

template <int DC>
__global__ void __launch_bounds__(4 * DC) k_bsr_tile(BsrArgs a, const float *tin, int64_t ldt) {
  constexpr int NT = 4 * DC;          // 16 row groups x DC/4 column groups
  constexpr int SLOT_B = 64 * 64;     // floats
  constexpr int SLOT_O = 64 * DC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *sB = reinterpret_cast<float *>(smem_raw);   // [2][SLOT_B]
  float *sO = sB + 2 * SLOT_B;                         // [2][64][DC]
  // a.seg CTAs share a row task, each a contiguous part of its CSR row
  const int tau = blockIdx.x / a.seg, part_id = blockIdx.x % a.seg;
  const int m = a.row_m[tau];
  const int inst = a.row_inst[tau];
  const int cb = a.cols.cb[inst], ce = a.cols.ce[inst];
  const int64_t r0 = a.ptr[tau], rn = a.ptr[tau + 1] - r0;
  const int64_t e0 = r0 + rn * part_id / a.seg, e1 = r0 + rn * (part_id + 1) / a.seg;
  if (m == 0 || ce <= cb || e0 == e1) return;
  const int rg = threadIdx.x & 15, cg = threadIdx.x >> 4;
  // input-slice copy: NT = 16 * (DC / 4), so thread t always copies chunk
  // t % (DC / 4) of rows t / (DC / 4) + 16 q
  const int cv = threadIdx.x % (DC / 4), cj0 = threadIdx.x / (DC / 4);
  const float *blocks = reinterpret_cast<const float *>(a.blocks);
  float *out = reinterpret_cast<float *>(a.out);
  const float sgn = (float)a.sign;
  for (int c0 = cb; c0 < ce; c0 += DC) {
    const int ncol = min(DC, ce - c0);
    float acc[16], cmp[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) { acc[q] = 0.f; cmp[q] = 0.f; }
    auto issue = [&](int64_t e, int slot) {
      if (e < e1) {
        const int b = a.idx[e];
        const int mb = a.col_m[b];
        const char *src = reinterpret_cast<const char *>(blocks + a.boff[e]);
        char *dst = reinterpret_cast<char *>(sB + slot * SLOT_B);
        const int n16 = (m * mb * 4 + 15) / 16;
        for (int u = threadIdx.x; u < n16; u += NT) cp_async16(dst + 16 * u, src + 16 * u);
        const float *irow = tin + a.col_off[b] * ldt + c0 + 4 * cv;
        float *di = sO + slot * SLOT_O + 4 * cv;
        const bool ok = 4 * cv < ncol;
        for (int j = cj0; j < mb; j += 16)
          cp_async16z(di + j * DC, ok ? irow + j * ldt : irow, ok);
      }
      cp_async_commit();
    };
    issue(e0, 0);
    for (int64_t e = e0; e < e1; ++e) {
      const int slot = (int)((e - e0) & 1);
      issue(e + 1, slot ^ 1);
      cp_async_wait<1>();
      __syncthreads();
      const int mb = a.col_m[a.idx[e]];
      const float *Bs = sB + slot * SLOT_B;
      const float *Os = sO + slot * SLOT_O + 4 * cg;
      float part[16];
#pragma unroll
      for (int q = 0; q < 16; ++q) part[q] = 0.f;
      const float *Br = Bs + rg;
#pragma unroll 2
      for (int j = 0; j < mb; ++j) {
        const float4 o = *reinterpret_cast<const float4 *>(Os + j * DC);
        float bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) bv[i] = Br[j * m + 16 * i];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          part[4 * i + 0] += bv[i] * o.x;
          part[4 * i + 1] += bv[i] * o.y;
          part[4 * i + 2] += bv[i] * o.z;
          part[4 * i + 3] += bv[i] * o.w;
        }
      }
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float y = sgn * part[q] - cmp[q];
        const float t = acc[q] + y;
        cmp[q] = (t - acc[q]) - y;
        acc[q] = t;
      }
      __syncthreads();
    }
    cp_async_wait<0>();
    __syncthreads();
    const int64_t orow = a.row_off[tau];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (rg + 16 * i >= m) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = 4 * cg + c;
        if (col >= ncol) continue;
        float *op = out + orow + rg + 16 * i + (int64_t)(c0 + col) * a.ld_out;
        if (a.seg > 1) {
          atomicAdd(op, acc[4 * i + c] - cmp[4 * i + c]);
        } else {
          const float y = *op - cmp[4 * i + c];
          *op = acc[4 * i + c] + y;
        }
      }
    }
  }
}

// Block-sparse row products for row blocks of 65 to 32 RI rows (ranks above
// 64, e.g. the couplings of operands built at tight tolerances).  As
// k_bsr_tile, with 32 row groups (thread rows rg + 32 i, i < RI: a warp reads
// 32 consecutive words of a block column) and the partner blocks streamed in
// chunks of JC columns: a chunk of a column-major block is one contiguous,
// 16-byte aligned range.  Plain sums over a whole block, compensated across.
template <int DC, int RI, int JC>
__global__ void __launch_bounds__(8 * DC) k_bsr_tile_big(BsrArgs a, const float *tin,
                                                         int64_t ldt) {
  constexpr int NT = 8 * DC;          // 32 row groups x DC/4 column groups
  constexpr int NR = 4 * RI;          // accumulators per thread
  constexpr int SLOT_B = 32 * RI * JC;   // floats
  constexpr int SLOT_O = JC * DC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float *sB = reinterpret_cast<float *>(smem_raw);   // [2][SLOT_B]
  float *sO = sB + 2 * SLOT_B;                         // [2][JC][DC]
  const int tau = blockIdx.x / a.seg, part_id = blockIdx.x % a.seg;
  const int m = a.row_m[tau];
  const int inst = a.row_inst[tau];
  const int cb = a.cols.cb[inst], ce = a.cols.ce[inst];
  const int64_t r0 = a.ptr[tau], rn = a.ptr[tau + 1] - r0;
  const int64_t e0 = r0 + rn * part_id / a.seg, e1 = r0 + rn * (part_id + 1) / a.seg;
  if (m == 0 || ce <= cb || e0 == e1) return;
  const int rg = threadIdx.x & 31, cg = threadIdx.x >> 5;
  // input-slice copy: NT = 32 * (DC / 4), so thread t copies chunk t % (DC / 4)
  // of rows t / (DC / 4) + 32 q
  const int cv = threadIdx.x % (DC / 4), cj0 = threadIdx.x / (DC / 4);
  const float *blocks = reinterpret_cast<const float *>(a.blocks);
  float *out = reinterpret_cast<float *>(a.out);
  const float sgn = (float)a.sign;
  for (int c0 = cb; c0 < ce; c0 += DC) {
    const int ncol = min(DC, ce - c0);
    float acc[NR], cmp[NR], part[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) { acc[q] = 0.f; cmp[q] = 0.f; part[q] = 0.f; }
    int64_t pe = e0;   // next chunk to issue: block pe, columns from pj
    int pj = 0;
    auto issue = [&](int slot) {
      if (pe < e1) {
        const int b = a.idx[pe];
        const int mb = a.col_m[b];
        const int nj = min(JC, mb - pj);
        const char *src = reinterpret_cast<const char *>(blocks + a.boff[pe] + (int64_t)pj * m);
        char *dst = reinterpret_cast<char *>(sB + slot * SLOT_B);
        const int n16 = (m * nj * 4 + 15) / 16;
        for (int u = threadIdx.x; u < n16; u += NT) cp_async16(dst + 16 * u, src + 16 * u);
        const float *irow = tin + (a.col_off[b] + pj) * ldt + c0 + 4 * cv;
        float *di = sO + slot * SLOT_O + 4 * cv;
        const bool ok = 4 * cv < ncol;
        for (int j = cj0; j < nj; j += 32)
          cp_async16z(di + j * DC, ok ? irow + (int64_t)j * ldt : irow, ok);
        pj += nj;
        if (pj >= mb) { pj = 0; ++pe; }
      }
      cp_async_commit();
    };
    int64_t ce_ = e0;  // chunk being computed: block ce_, columns from cj
    int cj = 0;
    issue(0);
    for (int it = 0; ce_ < e1; ++it) {
      const int slot = it & 1;
      issue(slot ^ 1);
      cp_async_wait<1>();
      __syncthreads();
      const int mb = a.col_m[a.idx[ce_]];
      const int nj = min(JC, mb - cj);
      // rows at or past m read other words of the slot and are never stored
      const float *Br = sB + slot * SLOT_B + rg;
      const float *Os = sO + slot * SLOT_O + 4 * cg;
#pragma unroll 2
      for (int j = 0; j < nj; ++j) {
        const float4 o = *reinterpret_cast<const float4 *>(Os + j * DC);
        float bv[RI];
#pragma unroll
        for (int i = 0; i < RI; ++i) bv[i] = Br[j * m + 32 * i];
#pragma unroll
        for (int i = 0; i < RI; ++i) {
          part[4 * i + 0] += bv[i] * o.x;
          part[4 * i + 1] += bv[i] * o.y;
          part[4 * i + 2] += bv[i] * o.z;
          part[4 * i + 3] += bv[i] * o.w;
        }
      }
      cj += nj;
      if (cj >= mb) {
        cj = 0;
        ++ce_;
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          const float y = sgn * part[q] - cmp[q];
          const float t = acc[q] + y;
          cmp[q] = (t - acc[q]) - y;
          acc[q] = t;
          part[q] = 0.f;
        }
      }
      __syncthreads();
    }
    cp_async_wait<0>();
    __syncthreads();
    const int64_t orow = a.row_off[tau];
#pragma unroll
    for (int i = 0; i < RI; ++i) {
      if (rg + 32 * i >= m) continue;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int col = 4 * cg + c;
        if (col >= ncol) continue;
        float *op = out + orow + rg + 32 * i + (int64_t)(c0 + col) * a.ld_out;
        if (a.seg > 1) {
          atomicAdd(op, acc[4 * i + c] - cmp[4 * i + c]);
        } else {
          const float y = *op - cmp[4 * i + c];
          *op = acc[4 * i + c] + y;
        }
      }
    }
  }
}

// Row-major copy t[r * ldt + c] = in[r + c * ld] of rows [0, n), columns [0, nc).
__global__ void k_transpose_panel(const float *in, int64_t ld, int64_t n, int nc, float *t,
                                  int64_t ldt) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int64_t r = r0 + threadIdx.x;
    const int c = c0 + q;
    tile[q][threadIdx.x] = (r < n && c < nc) ? in[r + (int64_t)c * ld] : 0.f;
  }
  __syncthreads();
  for (int q = threadIdx.y; q < 32; q += blockDim.y) {
    const int64_t r = r0 + q;
    const int c = c0 + threadIdx.x;
    if (r < n && c < (int)ldt) t[r * ldt + c] = c < nc ? tile[threadIdx.x][q] : 0.f;
  }
}

// ----------------------------------------------------------------------------
// Double-float arithmetic for the mixed-precision QR test and ID.  A value is
// an unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2,
// about 48 significant bits.  Sums and products are formed with the
// error-free transformations of Knuth (two-sum: a + b = s + e exactly) and
// of the fused multiply-add (a b = p + fma(a, b, -p) exactly), Dekker's
// double-length arithmetic.  GB300 issues FP32 at about 75 times its FP64
// rate, so the 12-15 FP32 operations of one double-float multiply-add cost a
// fraction of one FP64 one.  The explicit-rounding intrinsics keep the
// compiler from fusing the steps.  The products drop lo * lo (below 2^-48
// relative), and sums renormalise once (their error is below 2^-46 of the
// operands' magnitude, the backward error Householder QR needs).
// ----------------------------------------------------------------------------
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (s, e) with |e| small against |s| -> normalised pair
__device__ __forceinline__ float2 df_norm(float s, float e) {
  const float h = __fadd_rn(s, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, s)));
}
__device__ __forceinline__ float2 df_from(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double df_val(float2 a) { return (double)a.x + (double)a.y; }
// running sum of products: s + c with c the accumulated rounding errors
struct DfAcc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_prod(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    float t;
    df_two_sum(s, p, s, t);
    c = __fadd_rn(c, __fadd_rn(t, e));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
  // s and c as one normalised pair; exact even where the sum cancelled below
  // its rounding errors (|c| > |s|)
  __device__ __forceinline__ float2 pair() const {
    float h, l;
    df_two_sum(s, c, h, l);
    return make_float2(h, l);
  }
};
// a + b (the error of the low parts' sum is below 2^-46 of |a| + |b|)
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  df_two_sum(a.x, b.x, s, e);
  return df_norm(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return df_norm(p, e);
}
// a - w v
__device__ __forceinline__ float2 df_sub_prod(float2 a, float2 w, float2 v) {
  const float p = __fmul_rn(w.x, v.x);
  float e = fmaf(w.x, v.x, -p);
  e = fmaf(w.x, v.y, e);
  e = fmaf(w.y, v.x, e);
  float h, t;
  df_two_sum(a.x, -p, h, t);
  return df_norm(h, __fadd_rn(t, __fsub_rn(a.y, e)));
}

// The sum of tot and the argmax of (best, bi) over the CTA in one pass
// (lowest index on ties); every thread gets both.  Two barriers: the caller
// keeps a barrier between two calls.
__device__ void block_sum_argmax(double &tot, double &best, int &bi, double *sh, double *shv,
                                 int *shi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tot += __shfl_xor_sync(0xffffffffu, tot, o);
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
  }
  if (lane == 0) { sh[warp] = tot; shv[warp] = best; shi[warp] = bi; }
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? sh[lane] : 0.0;
    double w = lane < nw ? shv[lane] : -1.0;
    int wi = lane < nw ? shi[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      t += __shfl_xor_sync(0xffffffffu, t, o);
      const double ov = __shfl_xor_sync(0xffffffffu, w, o);
      const int oi = __shfl_xor_sync(0xffffffffu, wi, o);
      if (ov > w || (ov == w && oi < wi)) { w = ov; wi = oi; }
    }
    if (lane == 0) { sh[32] = t; shv[32] = w; shi[32] = wi; }
  }
  __syncthreads();
  tot = sh[32];
  best = shv[32];
  bi = shi[32];
}

// Sum over a group of TPC consecutive lanes (mask: the group's lanes).
template <int TPC>
__device__ __forceinline__ double group_sum(double v, unsigned mask) {
  if constexpr (TPC >= 2) v += __shfl_xor_sync(mask, v, 1);
  if constexpr (TPC >= 4) v += __shfl_xor_sync(mask, v, 2);
  return v;
}
// The same for double-float pairs (FP32 arithmetic only).
template <int TPC>
__device__ __forceinline__ float2 group_sum_df(float2 v, unsigned mask) {
  if constexpr (TPC >= 2)
    v = df_add(v, make_float2(__shfl_xor_sync(mask, v.x, 1), __shfl_xor_sync(mask, v.y, 1)));
  if constexpr (TPC >= 4)
    v = df_add(v, make_float2(__shfl_xor_sync(mask, v.x, 2), __shfl_xor_sync(mask, v.y, 2)));
  return v;
}

// ----------------------------------------------------------------------------
// Task scheduling of the per-cluster factorizations.  Without a queue each
// CTA takes one task (task = blockIdx.x, or queue[blockIdx.x]).  With one, a
// grid of as many CTAs as fit on the device at once takes tasks in queue
// order from a device counter, one at a time, so that an ordering by cost
// (largest first) evens out the CTAs' loads.
// ----------------------------------------------------------------------------
// The CTA's next position in the queue (>= n: none left); s_j is a shared
// slot that carries thread 0's draw to the CTA.
__device__ __forceinline__ int take_task(int32_t *next, int *s_j, bool first, int n) {
  if (!next) return first ? (int)blockIdx.x : n;
  __syncthreads();   // the previous task is done with shared memory
  if (threadIdx.x == 0) *s_j = atomicAdd(next, 1);
  __syncthreads();
  return *s_j;
}

// ----------------------------------------------------------------------------
// QR convergence test (FP64 Householder, one CTA per cluster).
// ----------------------------------------------------------------------------
template <typename T, int NT>
__device__ __forceinline__ void qr_task(const QrArgs &a, int tau, unsigned char *smem_raw, double *nrm2) {
  // One thread per column of Y_loc (m x d), stored row-major in shared
  // memory (a thread's column is read with unit stride across the warp).
  // Each column's trailing norm for the next step is summed while the column
  // is updated, so a step needs no block reduction.
  int inst = a.t.inst[tau];
  if (!a.active[inst] || a.conv[tau]) return;
  int m = a.t.m[tau];
  int d = a.dcur[inst];
  if (m <= d) {
    if (threadIdx.x == 0) {
      a.conv[tau] = 1;
      if (a.mindiag) a.mindiag[tau] = 0.0;
    }
    return;
  }
  double *A = a.ws_off && a.ws_off[tau] >= 0 ? a.ws + a.ws_off[tau]
                                             : reinterpret_cast<double *>(smem_raw);
  const T *Y = reinterpret_cast<const T *>(a.Y);
  int64_t row = a.t.row[tau];
  for (int64_t q = threadIdx.x; q < (int64_t)m * d; q += NT) {
    int i = (int)(q % m), c = (int)(q / m);
    A[(int64_t)i * d + c] = (double)Y[row + i + (int64_t)c * a.ld];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += NT) {
    double s2 = 0.0;
    for (int i = 0; i < m; ++i) s2 += A[(int64_t)i * d + c] * A[(int64_t)i * d + c];
    nrm2[c] = s2;
  }
  __syncthreads();
  const double eps = a.eps[inst];
  double minr = INFINITY;
  for (int j = 0; j < d; ++j) {
    const double nrm = sqrt(nrm2[j]);
    minr = fmin(minr, nrm);
    if (minr <= eps && !a.mindiag) break;  // converged: the minimum only decreases
    if (nrm == 0.0) continue;
    const double x0 = A[(int64_t)j * d + j];
    const double alpha = x0 != 0.0 ? -copysign(nrm, x0) : -nrm;
    const double beta = 1.0 / (nrm * (nrm + fabs(x0)));   // 2 / (v^T v)
    __syncthreads();
    if (threadIdx.x == 0) A[(int64_t)j * d + j] = x0 - alpha;   // v_j
    __syncthreads();
    for (int c = j + 1 + threadIdx.x; c < d; c += NT) {
      double w0 = 0.0, w1 = 0.0;
      int i = j;
      for (; i + 1 < m; i += 2) {
        w0 += A[(int64_t)i * d + j] * A[(int64_t)i * d + c];
        w1 += A[(int64_t)(i + 1) * d + j] * A[(int64_t)(i + 1) * d + c];
      }
      if (i < m) w0 += A[(int64_t)i * d + j] * A[(int64_t)i * d + c];
      const double w = (w0 + w1) * beta;
      A[(int64_t)j * d + c] -= w * A[(int64_t)j * d + j];
      double s2 = 0.0;
      for (int r = j + 1; r < m; ++r) {
        const double x = A[(int64_t)r * d + c] - w * A[(int64_t)r * d + j];
        A[(int64_t)r * d + c] = x;
        s2 += x * x;
      }
      nrm2[c] = s2;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (a.mindiag) a.mindiag[tau] = minr;
    if (minr <= eps) a.conv[tau] = 1;
    else atomicAdd(&a.unconv[inst], 1);
  }
}

// The same test on FP32 panels (mixed precision) in double-float arithmetic:
// the panel and its Householder updates as hi/lo pairs (8 bytes, like FP64),
// the scalars of a step (norm, alpha, beta, w) in FP64.  Two (clusters of 65
// to 128 columns) or four (wider) threads share a column, rows interleaved;
// their partial dot products and norms meet in shuffles within the group.
template <int NT>
__device__ __forceinline__ void qr_task_df(const QrArgs &a, int tau, unsigned char *smem_raw,
                                           double *nrm2) {
  constexpr int kTpc = NT >= 512 ? 4 : (NT >= 256 ? 2 : 1), kSlots = NT / kTpc;
  const int inst = a.t.inst[tau];
  if (!a.active[inst] || a.conv[tau]) return;
  const int m = a.t.m[tau];
  const int d = a.dcur[inst];
  if (m <= d) {
    if (threadIdx.x == 0) {
      a.conv[tau] = 1;
      if (a.mindiag) a.mindiag[tau] = 0.0;
    }
    return;
  }
  float2 *A = reinterpret_cast<float2 *>(a.ws_off && a.ws_off[tau] >= 0
                                             ? a.ws + a.ws_off[tau]
                                             : reinterpret_cast<double *>(smem_raw));
  const float *Y = reinterpret_cast<const float *>(a.Y);
  const int64_t row = a.t.row[tau];
  const int slot = threadIdx.x / kTpc, sub = threadIdx.x % kTpc;
  const unsigned gmask = kTpc == 4   ? 0xFu << (threadIdx.x & 28)
                         : kTpc == 2 ? 0x3u << (threadIdx.x & 30)
                                     : 1u << (threadIdx.x & 31);

  for (int64_t q = threadIdx.x; q < (int64_t)m * d; q += NT) {
    const int i = (int)(q % m), c = (int)(q / m);
    A[(int64_t)i * d + c] = make_float2(Y[row + i + (int64_t)c * a.ld], 0.f);
  }
  __syncthreads();
  for (int c = slot; c < d; c += kSlots) {
    DfAcc s2;
    for (int i = sub; i < m; i += kTpc) {
      const float2 x = A[(int64_t)i * d + c];
      s2.add_prod(x, x);
    }
    const double v = group_sum<kTpc>(s2.value(), gmask);
    if (sub == 0) nrm2[c] = v;
  }
  __syncthreads();
  const double eps = a.eps[inst];
  double minr = INFINITY;
  for (int j = 0; j < d; ++j) {
    const double nrm = sqrt(nrm2[j]);
    minr = fmin(minr, nrm);
    if (minr <= eps && !a.mindiag) break;
    if (nrm == 0.0) continue;
    const double x0 = df_val(A[(int64_t)j * d + j]);
    const double alpha = x0 != 0.0 ? -copysign(nrm, x0) : -nrm;
    const double beta = 1.0 / (nrm * (nrm + fabs(x0)));
    // the reflector's first entry stays in registers (A(j, j) itself is never
    // read again), so the step needs no barrier before its updates; the
    // per-column scalars of the step stay in FP32 pairs (the FP64 pipe is slow)
    const float2 vj = df_from(x0 - alpha), beta2 = df_from(beta);
    // the group's rows: j + sub, j + sub + 4, ... (row j, the pivot row, is sub 0's)
    for (int c = j + 1 + slot; c < d; c += kSlots) {
      // independent dependency chains: four running sums for the dot
      // product, two for the trailing norm
      DfAcc w0, w1, w2, w3;
      int i = j + sub;
      if (sub == 0) {
        w0.add_prod(vj, A[(int64_t)j * d + c]);
        i += kTpc;
      }
      for (; i + 3 * kTpc < m; i += 4 * kTpc) {
        w0.add_prod(A[(int64_t)i * d + j], A[(int64_t)i * d + c]);
        w1.add_prod(A[(int64_t)(i + kTpc) * d + j], A[(int64_t)(i + kTpc) * d + c]);
        w2.add_prod(A[(int64_t)(i + 2 * kTpc) * d + j], A[(int64_t)(i + 2 * kTpc) * d + c]);
        w3.add_prod(A[(int64_t)(i + 3 * kTpc) * d + j], A[(int64_t)(i + 3 * kTpc) * d + c]);
      }
      for (; i < m; i += kTpc) w0.add_prod(A[(int64_t)i * d + j], A[(int64_t)i * d + c]);
      const float2 w = df_mul(
          group_sum_df<kTpc>(df_add(df_add(w0.pair(), w1.pair()), df_add(w2.pair(), w3.pair())),
                             gmask),
          beta2);
      DfAcc s2, s3;
      int r = j + sub;
      if (sub == 0) {
        A[(int64_t)j * d + c] = df_sub_prod(A[(int64_t)j * d + c], w, vj);
        r += kTpc;
      }
      for (; r + kTpc < m; r += 2 * kTpc) {
        const float2 x = df_sub_prod(A[(int64_t)r * d + c], w, A[(int64_t)r * d + j]);
        const float2 y =
            df_sub_prod(A[(int64_t)(r + kTpc) * d + c], w, A[(int64_t)(r + kTpc) * d + j]);
        A[(int64_t)r * d + c] = x;
        A[(int64_t)(r + kTpc) * d + c] = y;
        s2.add_prod(x, x);
        s3.add_prod(y, y);
      }
      if (r < m) {
        const float2 x = df_sub_prod(A[(int64_t)r * d + c], w, A[(int64_t)r * d + j]);
        A[(int64_t)r * d + c] = x;
        s2.add_prod(x, x);
      }
      const double v = group_sum<kTpc>(s2.value() + s3.value(), gmask);
      if (sub == 0) nrm2[c] = v;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (a.mindiag) a.mindiag[tau] = minr;
    if (minr <= eps) a.conv[tau] = 1;
    else atomicAdd(&a.unconv[inst], 1);
  }
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_qr_test(QrArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double nrm2[kMaxCols];
  __shared__ int s_j;
  const int n = a.t.n;
  for (int j = take_task(a.next, &s_j, true, n); j < n; j = take_task(a.next, &s_j, false, n)) {
    if constexpr (sizeof(T) == 4) qr_task_df<NT>(a, a.queue ? a.queue[j] : j, smem_raw, nrm2);
    else qr_task<T, NT>(a, a.queue ? a.queue[j] : j, smem_raw, nrm2);
  }
}

// ----------------------------------------------------------------------------
// Row ID by column-pivoted Householder QR of A = Y_loc^T / sqrt(d), d x m.
// ----------------------------------------------------------------------------
template <typename T, int NT>
__device__ __forceinline__ void id_task(const IdArgs &a, int tau, unsigned char *smem_raw, double *red,
                        double *redv, int *redi) {
  // One thread per column (a point of the cluster) of A = Y_loc^T / sqrt(d),
  // d x m, stored row-major in shared memory; each column's trailing norm for
  // the next step is recomputed while the column is updated (FP64 panels) or
  // downdated (FP32 panels).
  constexpr bool DOWNDATE = sizeof(T) == 4;
  int inst = a.t.inst[tau];
  int m = a.t.m[tau];
  int64_t row = a.t.row[tau];
  if (!a.active[inst] || m == 0) {
    if (threadIdx.x == 0) a.k_out[tau] = 0;
    return;
  }
  int d = a.dcur[inst];
  // shared layout: norms[m] (double), piv[m], rank[m], sig[m] (int), then A
  double *nrm2 = reinterpret_cast<double *>(smem_raw);
  int *piv = reinterpret_cast<int *>(nrm2 + a.mcap);
  int *rnk = piv + a.mcap;
  int *sig = rnk + a.mcap;
  double *A = a.ws_off && a.ws_off[tau] >= 0 ? a.ws + a.ws_off[tau]
                                             : reinterpret_cast<double *>(sig + a.mcap);
  const T *Y = reinterpret_cast<const T *>(a.Y);
  const double sd = sqrt((double)d);
  for (int64_t q = threadIdx.x; q < (int64_t)m * d; q += NT) {
    int i = (int)(q % m), c = (int)(q / m);
    A[(int64_t)c * m + i] = (double)Y[row + i + (int64_t)c * a.ld] / sd;   // A(c, i)
  }
  for (int i = threadIdx.x; i < m; i += NT) piv[i] = i;
  __syncthreads();
  for (int c = threadIdx.x; c < m; c += NT) {
    double s2 = 0.0;
    for (int r = 0; r < d; ++r) s2 += A[(int64_t)r * m + c] * A[(int64_t)r * m + c];
    nrm2[c] = s2;
  }
  __syncthreads();
  const double eps = a.eps[inst];
  int kmax = min(d, m);
  int k = 0;
  while (k < kmax) {
    double tot = 0.0, best = -1.0;
    int bi = 0x7fffffff;
    for (int c = k + threadIdx.x; c < m; c += NT) {
      double nv = sqrt(nrm2[c]);
      tot += nv * nv;
      if (nv > best) { best = nv; bi = c; }
    }
    tot = block_sum(tot, red);
    if (sqrt(tot) <= eps) break;
    int p = block_argmax(best, bi, redv, redi);
    if (p < k || p >= m) break;  // no finite pivot left
    const double nk = sqrt(nrm2[p]);
    __syncthreads();
    if (p != k) {
      for (int r = threadIdx.x; r < d; r += NT) {
        double t0 = A[(int64_t)r * m + k];
        A[(int64_t)r * m + k] = A[(int64_t)r * m + p];
        A[(int64_t)r * m + p] = t0;
      }
      if (threadIdx.x == 0) {
        int t1 = piv[k]; piv[k] = piv[p]; piv[p] = t1;
        double t2 = nrm2[k]; nrm2[k] = nrm2[p]; nrm2[p] = t2;
      }
    }
    __syncthreads();
    const double x0 = A[(int64_t)k * m + k];
    const double alpha = x0 != 0.0 ? -copysign(nk, x0) : -nk;
    const double beta = nk > 0.0 ? 1.0 / (nk * (nk + fabs(x0))) : 0.0;
    __syncthreads();
    if (threadIdx.x == 0) A[(int64_t)k * m + k] = x0 - alpha;   // v_k
    __syncthreads();
    for (int c = k + 1 + threadIdx.x; c < m; c += NT) {
      double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
      int r = k;
      for (; r + 3 < d; r += 4) {
        w0 += A[(int64_t)r * m + k] * A[(int64_t)r * m + c];
        w1 += A[(int64_t)(r + 1) * m + k] * A[(int64_t)(r + 1) * m + c];
        w2 += A[(int64_t)(r + 2) * m + k] * A[(int64_t)(r + 2) * m + c];
        w3 += A[(int64_t)(r + 3) * m + k] * A[(int64_t)(r + 3) * m + c];
      }
      for (; r < d; ++r) w0 += A[(int64_t)r * m + k] * A[(int64_t)r * m + c];
      const double w = ((w0 + w1) + (w2 + w3)) * beta;
      const double rkc = A[(int64_t)k * m + c] - w * A[(int64_t)k * m + k];
      A[(int64_t)k * m + c] = rkc;
      // FP32 panels (mixed precision): the trailing norm is downdated,
      // |A(k+1:, c)|^2 = |A(k:, c)|^2 - R(k, c)^2 (the reflection keeps the
      // norm), and recomputed only after a cancellation of four digits; FP64
      // panels recompute it every step, as the FP64 parity of the skeletons
      // with the reference construction requires
      const double down = nrm2[c] - rkc * rkc;
      if (DOWNDATE && down > 1e-4 * nrm2[c]) {
        int q = k + 1;
        for (; q + 1 < d; q += 2) {
          A[(int64_t)q * m + c] -= w * A[(int64_t)q * m + k];
          A[(int64_t)(q + 1) * m + c] -= w * A[(int64_t)(q + 1) * m + k];
        }
        if (q < d) A[(int64_t)q * m + c] -= w * A[(int64_t)q * m + k];
        nrm2[c] = down;
      } else {
        double s0 = 0.0, s1 = 0.0;
        int q = k + 1;
        for (; q + 1 < d; q += 2) {
          const double x0 = A[(int64_t)q * m + c] - w * A[(int64_t)q * m + k];
          const double x1 = A[(int64_t)(q + 1) * m + c] - w * A[(int64_t)(q + 1) * m + k];
          A[(int64_t)q * m + c] = x0;
          A[(int64_t)(q + 1) * m + c] = x1;
          s0 += x0 * x0;
          s1 += x1 * x1;
        }
        if (q < d) {
          const double x0 = A[(int64_t)q * m + c] - w * A[(int64_t)q * m + k];
          A[(int64_t)q * m + c] = x0;
          s0 += x0 * x0;
        }
        nrm2[c] = s0 + s1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) A[(int64_t)k * m + k] = alpha;
    __syncthreads();
    ++k;
  }
  // T = R11^{-1} R12 by back substitution, written over R12 (one thread per column)
  for (int c = k + threadIdx.x; c < m; c += NT) {
    for (int i = k - 1; i >= 0; --i) {
      double t = A[(int64_t)i * m + c];
      for (int j = i + 1; j < k; ++j) t -= A[(int64_t)i * m + j] * A[(int64_t)j * m + c];
      A[(int64_t)i * m + c] = t / A[(int64_t)i * m + i];
    }
  }
  // sorted skeleton order
  for (int q = threadIdx.x; q < k; q += NT) {
    int r = 0;
    for (int b = 0; b < k; ++b) r += piv[b] < piv[q];
    rnk[q] = r;
    sig[r] = q;
  }
  __syncthreads();
  double *E = a.E + a.eoff[tau];
  for (int64_t q = threadIdx.x; q < (int64_t)m * k; q += NT) E[q] = 0.0;
  __syncthreads();
  for (int q = threadIdx.x; q < k; q += NT) {
    int jr = piv[sig[q]];
    E[jr + (int64_t)q * m] = 1.0;
    a.J_tmp[row + q] = jr;
    a.skel_tmp[row + q] = a.ibar ? a.ibar[row + jr] : (int32_t)(row + jr);
  }
  for (int64_t q = threadIdx.x; q < (int64_t)(m - k) * k; q += NT) {
    int rr = (int)(q % (m - k)), ap = (int)(q / (m - k));
    E[piv[k + rr] + (int64_t)ap * m] = A[(int64_t)sig[ap] * m + (k + rr)];
  }
  if (threadIdx.x == 0) a.k_out[tau] = k;
}

// The row ID of an FP32 panel (mixed precision) in double-float arithmetic:
// the panel, its Householder updates and the back substitution as hi/lo
// pairs; norms, pivots, thresholds and the scalars of a step in FP64.  The
// pivot is the largest squared trailing norm (the same order as the norm).
// In clusters wider than 128 four threads share a column in the updates
// (rows interleaved, partial sums meeting in shuffles within the 4-lane
// group).
template <int NT>
__device__ __forceinline__ void id_task_df(const IdArgs &a, int tau, unsigned char *smem_raw,
                                           double *red, double *redv, int *redi) {
  constexpr int kTpc = NT >= 512 ? 4 : (NT >= 256 ? 2 : 1), kSlots = NT / kTpc;
  const int slot = threadIdx.x / kTpc, sub = threadIdx.x % kTpc;
  const unsigned gmask = kTpc == 4   ? 0xFu << (threadIdx.x & 28)
                         : kTpc == 2 ? 0x3u << (threadIdx.x & 30)
                                     : 1u << (threadIdx.x & 31);

  const int inst = a.t.inst[tau];
  const int m = a.t.m[tau];
  const int64_t row = a.t.row[tau];
  if (!a.active[inst] || m == 0) {
    if (threadIdx.x == 0) a.k_out[tau] = 0;
    return;
  }
  const int d = a.dcur[inst];
  // shared layout: norms[m] (double), piv[m], rank[m], sig[m] (int), then A
  double *nrm2 = reinterpret_cast<double *>(smem_raw);
  int *piv = reinterpret_cast<int *>(nrm2 + a.mcap);
  int *rnk = piv + a.mcap;
  int *sig = rnk + a.mcap;
  float2 *A = reinterpret_cast<float2 *>(a.ws_off && a.ws_off[tau] >= 0
                                             ? a.ws + a.ws_off[tau]
                                             : reinterpret_cast<double *>(sig + a.mcap));
  const float *Y = reinterpret_cast<const float *>(a.Y);
  const double rsd = 1.0 / sqrt((double)d);
  for (int64_t q = threadIdx.x; q < (int64_t)m * d; q += NT) {
    const int i = (int)(q % m), c = (int)(q / m);
    A[(int64_t)c * m + i] = df_from((double)Y[row + i + (int64_t)c * a.ld] * rsd);   // A(c, i)
  }
  for (int i = threadIdx.x; i < m; i += NT) piv[i] = i;
  __syncthreads();
  for (int c = slot; c < m; c += kSlots) {
    DfAcc s2;
    for (int r = sub; r < d; r += kTpc) {
      const float2 x = A[(int64_t)r * m + c];
      s2.add_prod(x, x);
    }
    const double v = group_sum<kTpc>(s2.value(), gmask);
    if (sub == 0) nrm2[c] = v;
  }
  __syncthreads();
  const double eps2 = a.eps[inst] * a.eps[inst];
  const int kmax = min(d, m);
  int k = 0;
  while (k < kmax) {
    double tot = 0.0, best = -1.0;
    int bi = 0x7fffffff;
    for (int c = k + threadIdx.x; c < m; c += NT) {
      const double nv = nrm2[c];
      tot += nv;
      if (nv > best) { best = nv; bi = c; }
    }
    block_sum_argmax(tot, best, bi, red, redv, redi);
    if (tot <= eps2) break;
    const int p = bi;
    if (p < k || p >= m) break;  // no finite pivot left
    const double nk = sqrt(nrm2[p]);
    __syncthreads();
    if (p != k) {
      for (int r = threadIdx.x; r < d; r += NT) {
        const float2 t0 = A[(int64_t)r * m + k];
        A[(int64_t)r * m + k] = A[(int64_t)r * m + p];
        A[(int64_t)r * m + p] = t0;
      }
      if (threadIdx.x == 0) {
        const int t1 = piv[k]; piv[k] = piv[p]; piv[p] = t1;
        const double t2 = nrm2[k]; nrm2[k] = nrm2[p]; nrm2[p] = t2;
      }
    }
    __syncthreads();
    const double x0 = df_val(A[(int64_t)k * m + k]);
    const double alpha = x0 != 0.0 ? -copysign(nk, x0) : -nk;
    const double beta = nk > 0.0 ? 1.0 / (nk * (nk + fabs(x0))) : 0.0;
    // the reflector's first entry stays in registers; A(k, k) receives R's
    // diagonal after the updates.  The per-column scalars stay in FP32 pairs.
    const float2 vk = df_from(x0 - alpha), beta2 = df_from(beta);
    for (int c = k + 1 + slot; c < m; c += kSlots) {
      const double nc2 = nrm2[c];
      // four running sums (independent dependency chains)
      DfAcc w0, w1, w2, w3;
      int r = k + sub;
      if (sub == 0) {
        w0.add_prod(vk, A[(int64_t)k * m + c]);
        r += kTpc;
      }
      for (; r + 3 * kTpc < d; r += 4 * kTpc) {
        w0.add_prod(A[(int64_t)r * m + k], A[(int64_t)r * m + c]);
        w1.add_prod(A[(int64_t)(r + kTpc) * m + k], A[(int64_t)(r + kTpc) * m + c]);
        w2.add_prod(A[(int64_t)(r + 2 * kTpc) * m + k], A[(int64_t)(r + 2 * kTpc) * m + c]);
        w3.add_prod(A[(int64_t)(r + 3 * kTpc) * m + k], A[(int64_t)(r + 3 * kTpc) * m + c]);
      }
      for (; r < d; r += kTpc) w0.add_prod(A[(int64_t)r * m + k], A[(int64_t)r * m + c]);
      const float2 w = df_mul(
          group_sum_df<kTpc>(df_add(df_add(w0.pair(), w1.pair()), df_add(w2.pair(), w3.pair())),
                             gmask),
          beta2);
      const float2 rkc = df_sub_prod(A[(int64_t)k * m + c], w, vk);
      __syncwarp(gmask);   // the group has read row k before it changes
      if (sub == 0) A[(int64_t)k * m + c] = rkc;
      // trailing norm downdated, |A(k+1:, c)|^2 = |A(k:, c)|^2 - R(k, c)^2,
      // and recomputed after a cancellation of four digits
      const double rk = df_val(rkc);
      const double down = nc2 - rk * rk;
      if (down > 1e-4 * nc2) {
        for (int q = k + 1 + sub; q < d; q += kTpc)
          A[(int64_t)q * m + c] = df_sub_prod(A[(int64_t)q * m + c], w, A[(int64_t)q * m + k]);
        if (sub == 0) nrm2[c] = down;
      } else {
        DfAcc s2;
        for (int q = k + 1 + sub; q < d; q += kTpc) {
          const float2 x = df_sub_prod(A[(int64_t)q * m + c], w, A[(int64_t)q * m + k]);
          A[(int64_t)q * m + c] = x;
          s2.add_prod(x, x);
        }
        const double v = group_sum<kTpc>(s2.value(), gmask);
        if (sub == 0) nrm2[c] = v;
      }
    }
    __syncthreads();
    // column k is not read again before the next barrier
    if (threadIdx.x == 0) A[(int64_t)k * m + k] = df_from(alpha);
    ++k;
  }
  // T = R11^{-1} R12 by back substitution, written over R12 (one thread per
  // column); the reciprocals of R's diagonal go where the norms were
  __syncthreads();
  float2 *rinv = reinterpret_cast<float2 *>(nrm2);
  for (int i = threadIdx.x; i < k; i += NT) rinv[i] = df_from(1.0 / df_val(A[(int64_t)i * m + i]));
  __syncthreads();
  if (sub == 0) {
    for (int c = k + slot; c < m; c += kSlots) {
      for (int i = k - 1; i >= 0; --i) {
        float2 t = A[(int64_t)i * m + c];
        for (int j = i + 1; j < k; ++j)
          t = df_sub_prod(t, A[(int64_t)i * m + j], A[(int64_t)j * m + c]);
        A[(int64_t)i * m + c] = df_mul(t, rinv[i]);
      }
    }
  }
  // sorted skeleton order
  for (int q = threadIdx.x; q < k; q += NT) {
    int r = 0;
    for (int b = 0; b < k; ++b) r += piv[b] < piv[q];
    rnk[q] = r;
    sig[r] = q;
  }
  __syncthreads();
  double *E = a.E + a.eoff[tau];
  for (int64_t q = threadIdx.x; q < (int64_t)m * k; q += NT) E[q] = 0.0;
  __syncthreads();
  for (int q = threadIdx.x; q < k; q += NT) {
    const int jr = piv[sig[q]];
    E[jr + (int64_t)q * m] = 1.0;
    a.J_tmp[row + q] = jr;
    a.skel_tmp[row + q] = a.ibar ? a.ibar[row + jr] : (int32_t)(row + jr);
  }
  for (int64_t q = threadIdx.x; q < (int64_t)(m - k) * k; q += NT) {
    const int rr = (int)(q % (m - k)), ap = (int)(q / (m - k));
    E[piv[k + rr] + (int64_t)ap * m] = df_val(A[(int64_t)sig[ap] * m + (k + rr)]);
  }
  if (threadIdx.x == 0) a.k_out[tau] = k;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_row_id(IdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[33];
  __shared__ double redv[33];
  __shared__ int redi[33];
  __shared__ int s_j;
  const int n = a.t.n;
  for (int j = take_task(a.next, &s_j, true, n); j < n; j = take_task(a.next, &s_j, false, n)) {
    if constexpr (sizeof(T) == 4)
      id_task_df<NT>(a, a.queue ? a.queue[j] : j, smem_raw, red, redv, redi);
    else
      id_task<T, NT>(a, a.queue ? a.queue[j] : j, smem_raw, red, redv, redi);
  }
}

__global__ void k_compact(TasksDev t, const int32_t *J_tmp, const int32_t *skel_tmp, int32_t *J,
                          int32_t *skel) {
  int tau = blockIdx.x;
  int k = t.k[tau];
  int64_t row = t.row[tau], kr = t.krow[tau];
  for (int a = threadIdx.x; a < k; a += blockDim.x) {
    J[kr + a] = J_tmp[row + a];
    skel[kr + a] = skel_tmp[row + a];
  }
}

template <typename T>
__global__ void k_gather_rows_skel(TasksDev t, const T *Y, int64_t ld, T *Yn, int64_t ldn,
                                   InstCols cols, const int32_t *active) {
  int tau = blockIdx.x;
  int inst = t.inst[tau];
  if (!active[inst]) return;
  int k = t.k[tau];
  int cb = cols.cb[inst], ce = cols.ce[inst];
  int64_t row = t.row[tau], kr = t.krow[tau];
  for (int64_t q = threadIdx.x; q < (int64_t)k * (ce - cb); q += blockDim.x) {
    int a = (int)(q % k), c = cb + (int)(q / k);
    Yn[kr + a + c * ldn] = Y[row + t.J[kr + a] + c * ld];
  }
}

// out(krow+a, c) = sum_i E(i,a) in(row+i, c)
template <typename T, typename TE>
__global__ void k_basis_t(TasksDev t, const TE *E, const T *in, int64_t ld_in, T *out,
                          int64_t ld_out, InstCols cols, const int32_t *active) {
  int tau = blockIdx.x;
  int inst = t.inst[tau];
  if (active && !active[inst]) return;
  int k = t.k[tau], m = t.m[tau];
  int cb = cols.cb[inst], ce = cols.ce[inst];
  if (k == 0 || ce <= cb) return;
  int64_t row = t.row[tau], kr = t.krow[tau];
  const TE *Et = E + t.eoff[tau];
  for (int64_t q = threadIdx.x; q < (int64_t)k * (ce - cb); q += blockDim.x) {
    int a = (int)(q % k), c = cb + (int)(q / k);
    const TE *ea = Et + (int64_t)a * m;
    const T *xc = in + row + c * ld_in;
    double s = 0.0;
    for (int i = 0; i < m; ++i) s += (double)ea[i] * (double)xc[i];
    out[kr + a + c * ld_out] = (T)s;
  }
}

// out(row+i, c) += sum_a E(i,a) in(krow+a, c)
template <typename T, typename TE>
__global__ void k_basis_n(TasksDev t, const TE *E, const T *in, int64_t ld_in, T *out,
                          int64_t ld_out, InstCols cols) {
  int tau = blockIdx.x;
  int inst = t.inst[tau];
  int k = t.k[tau], m = t.m[tau];
  int cb = cols.cb[inst], ce = cols.ce[inst];
  if (k == 0 || ce <= cb) return;
  int64_t row = t.row[tau], kr = t.krow[tau];
  const TE *Et = E + t.eoff[tau];
  for (int64_t q = threadIdx.x; q < (int64_t)m * (ce - cb); q += blockDim.x) {
    int i = (int)(q % m), c = cb + (int)(q / m);
    const T *yc = in + kr + c * ld_in;
    double s = 0.0;
    for (int aa = 0; aa < k; ++aa) s += (double)Et[i + (int64_t)aa * m] * (double)yc[aa];
    out[row + i + c * ld_out] = (T)((double)out[row + i + c * ld_out] + s);
  }
}

// FP32 forms of the two basis products (mixed precision).  A cluster's
// outputs are cut into 64 x 32 tiles (64 basis columns or rows by 32
// right-hand sides) spread over gridDim.y CTAs; each tile streams the
// contracted index through shared memory in chunks of 32, so the shared
// footprint (13 KB) does not depend on the cluster.  Thread t owns tile row
// t % 64 and the 8 consecutive columns 8 (t / 64) .. 8 (t / 64) + 7: per
// contracted index it reads one basis value (rows at an odd stride, so a
// warp's 32 reads hit 32 banks) and its 8 right-hand-side values as two
// 16-byte broadcasts (the warp shares t / 64), then does 8 FMAs.
constexpr int kTileR = 64, kTileC = 32, kTileK = 32;
constexpr int kTileXS = kTileC + 4;   // row stride of the staged right-hand sides (16-byte rows)

// out(krow+a, c) = sum_i E(i,a) in(row+i, c)
__global__ void __launch_bounds__(256) k_basis_t32_tiled(TasksDev t, const double *E,
                                                         const float *in, int64_t ld_in,
                                                         float *out, int64_t ld_out, InstCols cols,
                                                         const int32_t *active) {
  __shared__ float sE[kTileR * (kTileK + 1)];              // E(i0+ii, a0+aa) at aa*(K+1) + ii
  __shared__ __align__(16) float sX[kTileK * kTileXS];     // in(row+i0+ii, c0+c) at ii*XS + c
  const int tau = blockIdx.x;
  const int inst = t.inst[tau];
  if (active && !active[inst]) return;
  const int k = t.k[tau], m = t.m[tau];
  const int cb = cols.cb[inst], ce = cols.ce[inst];
  if (k == 0 || ce <= cb) return;
  const int64_t row = t.row[tau], kr = t.krow[tau];
  const double *Et = E + t.eoff[tau];
  const int na_t = (k + kTileR - 1) / kTileR, nc_t = (ce - cb + kTileC - 1) / kTileC;
  const int tid = threadIdx.x, aa = tid % kTileR, cq = (tid / kTileR) * 8;
  for (int w = blockIdx.y; w < na_t * nc_t; w += gridDim.y) {
    const int a0 = (w % na_t) * kTileR, c0 = cb + (w / na_t) * kTileC;
    const int na = min(kTileR, k - a0), nc = min(kTileC, ce - c0);
    float acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.f;
    for (int i0 = 0; i0 < m; i0 += kTileK) {
      const int mi = min(kTileK, m - i0);
      __syncthreads();
      for (int q = tid; q < kTileR * kTileK; q += 256) {
        const int a = q / kTileK, ii = q % kTileK;
        sE[a * (kTileK + 1) + ii] =
            (a < na && ii < mi) ? (float)Et[(int64_t)(a0 + a) * m + i0 + ii] : 0.f;
      }
      for (int q = tid; q < kTileC * kTileK; q += 256) {
        const int c = q / kTileK, ii = q % kTileK;
        sX[ii * kTileXS + c] =
            (c < nc && ii < mi) ? in[row + i0 + ii + (int64_t)(c0 + c) * ld_in] : 0.f;
      }
      __syncthreads();
#pragma unroll 4
      for (int ii = 0; ii < kTileK; ++ii) {
        const float e = sE[aa * (kTileK + 1) + ii];
        const float4 x0 = *reinterpret_cast<const float4 *>(sX + ii * kTileXS + cq);
        const float4 x1 = *reinterpret_cast<const float4 *>(sX + ii * kTileXS + cq + 4);
        acc[0] = fmaf(e, x0.x, acc[0]);
        acc[1] = fmaf(e, x0.y, acc[1]);
        acc[2] = fmaf(e, x0.z, acc[2]);
        acc[3] = fmaf(e, x0.w, acc[3]);
        acc[4] = fmaf(e, x1.x, acc[4]);
        acc[5] = fmaf(e, x1.y, acc[5]);
        acc[6] = fmaf(e, x1.z, acc[6]);
        acc[7] = fmaf(e, x1.w, acc[7]);
      }
    }
    if (aa < na) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (cq + r < nc) out[kr + a0 + aa + (int64_t)(c0 + cq + r) * ld_out] = acc[r];
    }
  }
}

// out(row+i, c) += sum_a E(i,a) in(krow+a, c)
__global__ void __launch_bounds__(256) k_basis_n32_tiled(TasksDev t, const double *E,
                                                         const float *in, int64_t ld_in,
                                                         float *out, int64_t ld_out,
                                                         InstCols cols) {
  __shared__ float sE[kTileK * kTileR];                    // E(i0+ii, a0+aa) at aa*R + ii
  __shared__ __align__(16) float sY[kTileK * kTileXS];     // in(krow+a0+aa, c0+c) at aa*XS + c
  const int tau = blockIdx.x;
  const int inst = t.inst[tau];
  const int k = t.k[tau], m = t.m[tau];
  const int cb = cols.cb[inst], ce = cols.ce[inst];
  if (k == 0 || ce <= cb) return;
  const int64_t row = t.row[tau], kr = t.krow[tau];
  const double *Et = E + t.eoff[tau];
  const int ni_t = (m + kTileR - 1) / kTileR, nc_t = (ce - cb + kTileC - 1) / kTileC;
  const int tid = threadIdx.x, ii = tid % kTileR, cq = (tid / kTileR) * 8;
  for (int w = blockIdx.y; w < ni_t * nc_t; w += gridDim.y) {
    const int i0 = (w % ni_t) * kTileR, c0 = cb + (w / ni_t) * kTileC;
    const int mi = min(kTileR, m - i0), nc = min(kTileC, ce - c0);
    float acc[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) acc[r] = 0.f;
    for (int a0 = 0; a0 < k; a0 += kTileK) {
      const int na = min(kTileK, k - a0);
      __syncthreads();
      for (int q = tid; q < kTileK * kTileR; q += 256) {
        const int a = q / kTileR, i = q % kTileR;
        sE[q] = (a < na && i < mi) ? (float)Et[(int64_t)(a0 + a) * m + i0 + i] : 0.f;
      }
      for (int q = tid; q < kTileC * kTileK; q += 256) {
        const int c = q / kTileK, a = q % kTileK;
        sY[a * kTileXS + c] =
            (c < nc && a < na) ? in[kr + a0 + a + (int64_t)(c0 + c) * ld_in] : 0.f;
      }
      __syncthreads();
#pragma unroll 4
      for (int a = 0; a < kTileK; ++a) {
        const float e = sE[a * kTileR + ii];
        const float4 y0 = *reinterpret_cast<const float4 *>(sY + a * kTileXS + cq);
        const float4 y1 = *reinterpret_cast<const float4 *>(sY + a * kTileXS + cq + 4);
        acc[0] = fmaf(e, y0.x, acc[0]);
        acc[1] = fmaf(e, y0.y, acc[1]);
        acc[2] = fmaf(e, y0.z, acc[2]);
        acc[3] = fmaf(e, y0.w, acc[3]);
        acc[4] = fmaf(e, y1.x, acc[4]);
        acc[5] = fmaf(e, y1.y, acc[5]);
        acc[6] = fmaf(e, y1.z, acc[6]);
        acc[7] = fmaf(e, y1.w, acc[7]);
      }
    }
    if (ii < mi) {
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (cq + r < nc) out[row + i0 + ii + (int64_t)(c0 + cq + r) * ld_out] += acc[r];
    }
  }
}

// CTAs per cluster for the tiled products: enough to cover the device twice
// when the level has few clusters, one when it has many.
int tiled_split(int n_tasks) {
  const int want = (2 * device_sm_count() + n_tasks - 1) / n_tasks;
  return want < 1 ? 1 : (want > 16 ? 16 : want);
}

// One CTA per row task: its points (the leaf's, or its skeleton points) are
// staged once, then every partner block of its CSR row is evaluated from a
// staged copy of the partner's points; the next partner's points are loaded
// into registers while the current block is evaluated.  Column-major block
// stores, coalesced.
template <int KID, typename T, bool SKEL>
__global__ void __launch_bounds__(256) k_gen_rows(int n_rows, const int64_t *ptr,
                                                  const int32_t *idx, const int64_t *off,
                                                  const int32_t *rows_of, const int64_t *row0,
                                                  const int64_t *krow, const int32_t *skel,
                                                  const int32_t *tinst, const InstDev *inst,
                                                  Points64 p64, Points32 p32, void *out_,
                                                  const int32_t *cols_of, const int64_t *ckrow,
                                                  const int32_t *cskel) {
  constexpr int NC = PtsOf<T>::NC;
  constexpr int NS = (NC * (int)sizeof(T) + 15) / 16 * 16 / (int)sizeof(T);   // 16-byte rows
  __shared__ __align__(16) T sa[kMaxRows * NS], sb[2][kMaxRows * NS];
  __shared__ int64_t ga[kMaxRows], gb[2][kMaxRows];
  const int tr = blockIdx.x;
  if (tr >= n_rows) return;
  const int64_t e0 = ptr[tr], e1 = ptr[tr + 1];
  if (e0 == e1) return;
  const int m = rows_of[tr];
  if (m == 0) return;
  const InstDev in = inst[tinst[tr]];
  const T scale = (T)in.kd.scale, diag = (T)in.kd.diag;
  const int pw = in.kd.pw;
  auto gpos = [&](int task, int i) -> int64_t {
    return SKEL ? (int64_t)skel[krow[task] + i] : row0[task] + i;
  };
  // partners: the column side's skeletons where given (separate row and
  // column bases), else the rows' own
  auto gpos_c = [&](int task, int j) -> int64_t {
    return SKEL && cskel ? (int64_t)cskel[ckrow[task] + j] : gpos(task, j);
  };
  auto width = [&](int task) { return cols_of ? cols_of[task] : rows_of[task]; };
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int64_t g = gpos(tr, i);
    ga[i] = g;
    PtsOf<T>::load(p64, p32, g, sa + i * NS);
  }
  // partner points of entry e into buffer slot
  auto load_partner = [&](int64_t e, int slot) {
    const int tc = idx[e];
    const int mb = width(tc);
    for (int j = threadIdx.x; j < mb; j += blockDim.x) {
      const int64_t g = gpos_c(tc, j);
      gb[slot][j] = g;
      PtsOf<T>::load(p64, p32, g, sb[slot] + j * NS);
    }
  };
  load_partner(e0, 0);
  __syncthreads();
  T *out = reinterpret_cast<T *>(out_);
  // thread = row i (of RG = 32 or 64 at a time, whichever covers m with fewer
  // idle lanes) x every (256 / RG)-th column j: a warp shares j, so the
  // partner point is a broadcast read and the stores are coalesced
  const int rg = m <= 32 ? 32 : 64, cg = 256 / rg;
  const int ig = threadIdx.x % rg, jg = threadIdx.x / rg;
  for (int64_t e = e0; e < e1; ++e) {
    const int slot = (int)((e - e0) & 1);
    if (e + 1 < e1) load_partner(e + 1, slot ^ 1);   // overlaps the evaluation below
    const int tc = idx[e];
    const int mb = width(tc);
    // only a leaf's block with itself holds coincident points (the diagonal)
    const bool self = !SKEL && tc == tr;
    T *blk = out + off[e];
    const T *pb = sb[slot];
    const int64_t *gbs = gb[slot];
    for (int i = ig; i < m; i += rg) {
      T pa[NS];
#pragma unroll
      for (int c = 0; c < NS; ++c) pa[c] = sa[i * NS + c];
      T *bp = blk + i + (int64_t)jg * m;
      const int64_t bstep = (int64_t)cg * m;
      if (self) {
        const int64_t gi = ga[i];
        for (int j = jg; j < mb; j += cg, bp += bstep) {
          const T gm = PtsOf<T>::template geom<KID>(pa, pb + j * NS);
          *bp = gi == gbs[j] ? kdiag<KID, T>(gm, scale, pw, diag) : kval<KID, T>(gm, scale, pw);
        }
      } else {
#pragma unroll 4
        for (int j = jg; j < mb; j += cg, bp += bstep)
          *bp = kval<KID, T>(PtsOf<T>::template geom<KID>(pa, pb + j * NS), scale, pw);
      }
    }
    __syncthreads();
  }
}

__global__ void k_block_sizes(int64_t nnz, const int32_t *erow, const int32_t *idx,
                              const int32_t *mrow, const int32_t *mcol, int align,
                              int64_t *out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nnz) {
    int64_t sz = (int64_t)mrow[erow[e]] * mcol[idx[e]];
    out[e] = (sz + align - 1) / align * align;
  }
}

__global__ void k_inner_tasks(int n, const int32_t *child0, const int64_t *krow_child,
                              const int32_t *k_child, int64_t *row, int32_t *m) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int c = child0[t];
  row[t] = krow_child[c];
  m[t] = k_child[c] + k_child[c + 1];
}

__global__ void k_basis_capacity(int n, const int32_t *m, const int32_t *inst,
                                 const int32_t *dcur, int64_t *cap) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  int mm = m[t];
  int d = dcur[inst[t]];
  cap[t] = (int64_t)mm * min(mm, d);
}

__global__ void k_map_csr(const int64_t *ptr, const int32_t *idx, int nrows, int first_node,
                          int task_base, int64_t nnz_base, int64_t *ptr_out, int32_t *idx_out,
                          int32_t *erow_out, int write_last) {
  // one warp per row: its entries are copied by the 32 lanes (coalesced)
  const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const int64_t b = ptr[r], e = ptr[r + 1];
  if (lane == 0) {
    ptr_out[task_base + r] = nnz_base + b;
    if (write_last && r == nrows - 1) ptr_out[task_base + nrows] = nnz_base + e;
  }
  for (int64_t q = b + lane; q < e; q += 32) {
    idx_out[nnz_base + q] = task_base + (idx[q] - first_node);
    if (erow_out) erow_out[nnz_base + q] = task_base + r;
  }
}

template <typename T>
__global__ void k_permute_in(const double *x, int64_t ldx, const int32_t *orig, int64_t n,
                             int nrhs, T *xt, int64_t ldt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = orig[i];
  for (int c = 0; c < nrhs; ++c) xt[i + c * ldt] = (T)x[o + c * ldx];
}

template <typename T>
__global__ void k_permute_out(const T *yt, int64_t ldt, const int32_t *orig, int64_t n, int nrhs,
                              double *y, int64_t ldy) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int64_t o = orig[i];
  for (int c = 0; c < nrhs; ++c) y[o + c * ldy] = (double)yt[i + c * ldt];
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

// Opt-in to `bytes` of dynamic shared memory.  Set above 32 KB, not 48 KB:
// the 48 KB default covers static and dynamic shared memory together, and the
// QR / ID kernels have static arrays of their own.
template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 32 * 1024)
    H2_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

void dense_blocks_gen(int kid, bool fp64, const DgenArgs &a, cudaStream_t s) {
  if (a.nnz == 0) return;
  H2_REQUIRE(a.nnz < (1ll << 31), "too many near-field blocks");
  dispatch_kernel(kid, [&](auto K) {
    constexpr int KID = decltype(K)::value;
    if (fp64)
      k_gen_rows<KID, double, false><<<a.n_rows, 256, 0, s>>>(
          a.n_rows, a.ptr, a.idx, a.doff, a.m, a.row, nullptr, nullptr, a.tinst, a.inst, a.p64,
          a.p32, a.D, nullptr, nullptr, nullptr);
    else
      k_gen_rows<KID, float, false><<<a.n_rows, 256, 0, s>>>(
          a.n_rows, a.ptr, a.idx, a.doff, a.m, a.row, nullptr, nullptr, a.tinst, a.inst, a.p64,
          a.p32, a.D, nullptr, nullptr, nullptr);
    count_launch();
    H2_CHECK_LAUNCH();
  });
}

template <typename T, int DC, int RPT>
void launch_bsr(const BsrArgs &a, cudaStream_t s) {
  constexpr int SLOT = kSlotBytes / sizeof(T);
  size_t bytes = sizeof(T) * ((size_t)kStages * SLOT + (size_t)kStages * 64 * (DC + 4));
  auto kern = k_bsr_pipe<T, DC, RPT>;
  set_smem(kern, bytes);
  kern<<<a.n_rows * a.seg, kNT, bytes, s>>>(a);
  count_launch();
  H2_CHECK_LAUNCH();
}

template <int DC, int RI, int JC>
void launch_bsr_tile_big(const BsrArgs &a, const float *tin, int64_t ldt, cudaStream_t s) {
  const size_t bytes = sizeof(float) * 2 * (32 * RI * JC + JC * DC);
  auto kern = k_bsr_tile_big<DC, RI, JC>;
  set_smem(kern, bytes);
  kern<<<a.n_rows * a.seg, 8 * DC, bytes, s>>>(a, tin, ldt);
  count_launch();
  H2_CHECK_LAUNCH();
}

template <int DC>
void launch_bsr_tile(const BsrArgs &a, const float *tin, int64_t ldt, cudaStream_t s) {
  const size_t bytes = sizeof(float) * 2 * (64 * 64 + 64 * DC);
  auto kern = k_bsr_tile<DC>;
  set_smem(kern, bytes);
  kern<<<a.n_rows * a.seg, 4 * DC, bytes, s>>>(a, tin, ldt);
  count_launch();
  H2_CHECK_LAUNCH();
}

void bsr_apply(bool fp64, const BsrArgs &a_in, int max_m, int max_cols, cudaStream_t s) {
  if (a_in.n_rows == 0 || max_cols <= 0) return;
  H2_REQUIRE(max_m <= kMaxRows, "block rows above 256 are not supported");
  if (!fp64 && max_m <= 256 && a_in.engine == 0) {
    // tensor cores: one CTA per SM and 128-row half of a task; a row task's
    // blocks are split over several CTAs only where the row tasks would not
    // fill the device twice
    BsrArgs t = a_in;
    const int chunks = std::max(1, (max_cols + 95) / 96) * (max_m > 128 ? 2 : 1);
    t.seg = std::max(1, std::min(16, 2 * device_sm_count() / std::max(1, a_in.n_rows * chunks)));
    if (bsr_apply_tc(t, max_m, max_cols, s)) return;
  }
  // Levels with few row tasks split each CSR row over several CTAs (FP32:
  // their partial sums meet in atomic adds; FP64 keeps one CTA per row so
  // that its sums stay in a fixed order)
  BsrArgs a = a_in;
  a.seg = fp64 ? 1 : std::max(1, std::min(16, 4 * device_sm_count() / a.n_rows));
  // register-tiled kernels: up to 128 rows at any width, 256 rows for up to 32
  // columns (wider 256-row tiles would spill registers)
  const bool tiled = max_m <= 128 || (max_m <= 256 && max_cols <= 32);
  if (!fp64 && tiled && a.col_hi > 0 && a.in_rows > 0) {
    // register-tiled path on a row-major copy of the input columns [0, col_hi)
    const int64_t ldt = (a.col_hi + 3) / 4 * 4;
    DBuf<float> tin;
    tin.alloc((size_t)a.in_rows * ldt + 4);
    dim3 grid((unsigned)ceil_div(a.in_rows, 32), (unsigned)ceil_div(ldt, 32));
    k_transpose_panel<<<grid, dim3(32, 8), 0, s>>>(reinterpret_cast<const float *>(a.in), a.ld_in,
                                                    a.in_rows, a.col_hi, tin.p, ldt);
    count_launch();
    H2_CHECK_LAUNCH();
    if (max_m > 128) {   // rows rg + 32 i, i < 8; 32-column chunks of the partners
      if (max_cols <= 16) launch_bsr_tile_big<16, 8, 32>(a, tin.p, ldt, s);
      else launch_bsr_tile_big<32, 8, 32>(a, tin.p, ldt, s);
    } else if (max_m > 64) {   // rows rg + 32 i, i < 4; 64-column chunks
      if (max_cols <= 16) launch_bsr_tile_big<16, 4, 64>(a, tin.p, ldt, s);
      else if (max_cols <= 32) launch_bsr_tile_big<32, 4, 64>(a, tin.p, ldt, s);
      else if (max_cols <= 64) launch_bsr_tile_big<64, 4, 64>(a, tin.p, ldt, s);
      else launch_bsr_tile_big<80, 4, 64>(a, tin.p, ldt, s);
    } else if (max_cols <= 16) launch_bsr_tile<16>(a, tin.p, ldt, s);
    else if (max_cols <= 32) launch_bsr_tile<32>(a, tin.p, ldt, s);
    else if (max_cols <= 64) launch_bsr_tile<64>(a, tin.p, ldt, s);
    else launch_bsr_tile<80>(a, tin.p, ldt, s);
    return;
  }
  const bool narrow = max_cols <= 16;
  if (max_m <= 64 && max_cols > 32 && !fp64) {
    launch_bsr<float, 64, 1>(a, s);   // one pass over the blocks for 64 columns
  } else if (max_m <= 64) {
    if (fp64) narrow ? launch_bsr<double, 16, 1>(a, s) : launch_bsr<double, 32, 1>(a, s);
    else narrow ? launch_bsr<float, 16, 1>(a, s) : launch_bsr<float, 32, 1>(a, s);
  } else if (max_m <= 128 && !fp64) {
    narrow ? launch_bsr<float, 16, 2>(a, s) : launch_bsr<float, 32, 2>(a, s);
  } else {
    if (fp64) narrow ? launch_bsr<double, 16, 4>(a, s) : launch_bsr<double, 32, 4>(a, s);
    else narrow ? launch_bsr<float, 16, 4>(a, s) : launch_bsr<float, 32, 4>(a, s);
  }
}

// CTA width for clusters of up to `width` columns (64, 128 or 256 threads).
template <template <typename, int> class K, int MUL128, int MUL256, typename A>
void launch_width(bool fp64, int width, const A &a, int n, size_t bytes, cudaStream_t s);

template <typename T, int NT>
struct QrKern {
  static constexpr auto f = k_qr_test<T, NT>;
};
template <typename T, int NT>
struct IdKern {
  static constexpr auto f = k_row_id<T, NT>;
};

// FP32 panels (double-float kernels) run MUL128 threads per column in
// clusters of 65 to 128 columns and MUL256 in wider ones.
template <template <typename, int> class K, int MUL128, int MUL256, typename A>
void launch_width(bool fp64, int width, const A &a, int n, size_t bytes, cudaStream_t s) {
  auto go = [&](auto kern, int nt) {
    set_smem(kern, bytes);
    int grid = n;
    if (a.next) {
      // work queue: as many CTAs as are resident at once, at most one per task
      int per_sm = 0;
      H2_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, bytes));
      grid = std::min(n, std::max(1, per_sm) * device_sm_count());
      H2_CUDA(cudaMemsetAsync(a.next, 0, sizeof(int32_t), s));
    }
    kern<<<grid, nt, bytes, s>>>(a);
  };
  const int w = width <= 0 ? 256 : width;
  if (fp64) {
    if (w <= 64) go(K<double, 64>::f, 64);
    else if (w <= 128) go(K<double, 128>::f, 128);
    else go(K<double, 256>::f, 256);
  } else {
    if (w <= 64) go(K<float, 64>::f, 64);
    else if (w <= 128) go(K<float, 128 * MUL128>::f, 128 * MUL128);
    else go(K<float, 256 * MUL256>::f, 256 * MUL256);
  }
  count_launch();
  H2_CHECK_LAUNCH();
}

void qr_test(bool fp64, const QrArgs &a, size_t smem_bytes, int width, cudaStream_t s) {
  if (a.t.n == 0) return;
  launch_width<QrKern, 2, 4>(fp64, width, a, a.t.n, smem_bytes, s);
}

size_t row_id_fixed_smem(int mcap) { return (size_t)mcap * (sizeof(double) + 3 * sizeof(int)); }

void row_id(bool fp64, const IdArgs &a, size_t smem_bytes, int width, cudaStream_t s) {
  if (a.t.n == 0) return;
  H2_REQUIRE(a.mcap >= 8 && a.mcap % 8 == 0 && a.mcap <= kMaxIdRows, "row ID capacity");
  launch_width<IdKern, 1, 4>(fp64, width, a, a.t.n, smem_bytes + row_id_fixed_smem(a.mcap), s);
}

void compact_skeletons(const TasksDev &t, const int32_t *J_tmp, const int32_t *skel_tmp,
                       int32_t *J, int32_t *skel, cudaStream_t s) {
  if (t.n == 0) return;
  k_compact<<<t.n, 128, 0, s>>>(t, J_tmp, skel_tmp, J, skel);
  count_launch();
  H2_CHECK_LAUNCH();
}

void gather_skeleton_rows(bool fp64, const TasksDev &t, const void *Y, int64_t ld, void *Yn,
                          int64_t ldn, InstCols cols, const int32_t *active, cudaStream_t s) {
  if (t.n == 0) return;
  if (fp64)
    k_gather_rows_skel<double><<<t.n, 256, 0, s>>>(t, (const double *)Y, ld, (double *)Yn, ldn,
                                                   cols, active);
  else
    k_gather_rows_skel<float><<<t.n, 256, 0, s>>>(t, (const float *)Y, ld, (float *)Yn, ldn, cols,
                                                  active);
  count_launch();
  H2_CHECK_LAUNCH();
}

void basis_t_apply(bool fp64, const TasksDev &t, const void *E, const void *in, int64_t ld_in,
                   void *out, int64_t ld_out, InstCols cols, const int32_t *active, int max_m,
                   int max_k, cudaStream_t s) {
  (void)max_m;
  (void)max_k;
  if (t.n == 0) return;
  if (fp64) {
    k_basis_t<double, double><<<t.n, 256, 0, s>>>(t, (const double *)E, (const double *)in,
                                                  ld_in, (double *)out, ld_out, cols, active);
  } else {
    const dim3 grid(t.n, tiled_split(t.n));
    k_basis_t32_tiled<<<grid, 256, 0, s>>>(t, (const double *)E, (const float *)in, ld_in,
                                           (float *)out, ld_out, cols, active);
  }
  count_launch();
  H2_CHECK_LAUNCH();
}

void basis_n_apply(bool fp64, const TasksDev &t, const void *E, const void *in, int64_t ld_in,
                   void *out, int64_t ld_out, InstCols cols, int max_m, int max_k,
                   cudaStream_t s) {
  (void)max_m;
  (void)max_k;
  if (t.n == 0) return;
  if (fp64) {
    k_basis_n<double, double><<<t.n, 256, 0, s>>>(t, (const double *)E, (const double *)in,
                                                  ld_in, (double *)out, ld_out, cols);
  } else {
    const dim3 grid(t.n, tiled_split(t.n));
    k_basis_n32_tiled<<<grid, 256, 0, s>>>(t, (const double *)E, (const float *)in, ld_in,
                                           (float *)out, ld_out, cols);
  }
  count_launch();
  H2_CHECK_LAUNCH();
}

void coupling_gen(int kid, bool fp64, const CouplingArgs &a, cudaStream_t s) {
  if (a.nnz == 0) return;
  H2_REQUIRE(a.nnz < (1ll << 31), "too many coupling blocks");
  dispatch_kernel(kid, [&](auto K) {
    constexpr int KID = decltype(K)::value;
    if (fp64)
      k_gen_rows<KID, double, true><<<a.t.n, 256, 0, s>>>(
          a.t.n, a.ptr, a.idx, a.boff, a.t.k, nullptr, a.t.krow, a.skel, a.t.inst, a.inst, a.p64,
          a.p32, a.B, a.col_k, a.col_krow, a.col_skel);
    else
      k_gen_rows<KID, float, true><<<a.t.n, 256, 0, s>>>(
          a.t.n, a.ptr, a.idx, a.boff, a.t.k, nullptr, a.t.krow, a.skel, a.t.inst, a.inst, a.p64,
          a.p32, a.B, a.col_k, a.col_krow, a.col_skel);
    count_launch();
    H2_CHECK_LAUNCH();
  });
}

void block_sizes(int64_t nnz, const int32_t *erow, const int32_t *idx, const int32_t *mrow,
                 const int32_t *mcol, int align, int64_t *out, cudaStream_t s) {
  if (nnz == 0) return;
  k_block_sizes<<<ceil_div(nnz, 256), 256, 0, s>>>(nnz, erow, idx, mrow, mcol, align, out);
  count_launch();
  H2_CHECK_LAUNCH();
}

void inner_tasks(int n, const int32_t *child0, const int64_t *krow_child, const int32_t *k_child,
                 int64_t *row, int32_t *m, cudaStream_t s) {
  if (n == 0) return;
  k_inner_tasks<<<ceil_div(n, 256), 256, 0, s>>>(n, child0, krow_child, k_child, row, m);
  count_launch();
  H2_CHECK_LAUNCH();
}

void basis_capacity(int n, const int32_t *m, const int32_t *inst, const int32_t *dcur,
                    int64_t *cap, cudaStream_t s) {
  if (n == 0) return;
  k_basis_capacity<<<ceil_div(n, 256), 256, 0, s>>>(n, m, inst, dcur, cap);
  count_launch();
  H2_CHECK_LAUNCH();
}

void map_csr(const int64_t *ptr, const int32_t *idx, int nrows, int first_node, int task_base,
             int64_t nnz_base, int64_t *ptr_out, int32_t *idx_out, int32_t *erow_out,
             bool write_last, cudaStream_t s) {
  if (nrows == 0) return;
  k_map_csr<<<ceil_div(nrows, 4), 128, 0, s>>>(ptr, idx, nrows, first_node, task_base, nnz_base,
                                               ptr_out, idx_out, erow_out, write_last ? 1 : 0);
  count_launch();
  H2_CHECK_LAUNCH();
}

void permute_in(bool fp64, const double *x, int64_t ldx, const int32_t *orig, int64_t n, int nrhs,
                void *xt, int64_t ldt, cudaStream_t s) {
  if (n == 0) return;
  if (fp64) k_permute_in<double><<<ceil_div(n, 256), 256, 0, s>>>(x, ldx, orig, n, nrhs, (double *)xt, ldt);
  else k_permute_in<float><<<ceil_div(n, 256), 256, 0, s>>>(x, ldx, orig, n, nrhs, (float *)xt, ldt);
  count_launch();
  H2_CHECK_LAUNCH();
}

void permute_out(bool fp64, const void *yt, int64_t ldt, const int32_t *orig, int64_t n, int nrhs,
                 double *y, int64_t ldy, cudaStream_t s) {
  if (n == 0) return;
  if (fp64) k_permute_out<double><<<ceil_div(n, 256), 256, 0, s>>>((const double *)yt, ldt, orig, n, nrhs, y, ldy);
  else k_permute_out<float><<<ceil_div(n, 256), 256, 0, s>>>((const float *)yt, ldt, orig, n, nrhs, y, ldy);
  count_launch();
  H2_CHECK_LAUNCH();
}

void fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t s) {
  if (n == 0) return;
  k_fill_i32<<<ceil_div(n, 256), 256, 0, s>>>(p, n, v);
  count_launch();
  H2_CHECK_LAUNCH();
}

}  // namespace h2
