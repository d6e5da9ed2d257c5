// Block-sparse row products on the 5th-generation tensor cores (mixed
// precision): out(rows of task t) += sign * sum_e Blk_e * in(rows of the
// column task of e), the far-field subtraction of Algorithm 1 (the couplings
// B times the upswept samples Omega^l), the leaf near field (D times Omega)
// and the H2 matrix-vector product's coupling and near-field products.
//
// Operands are FP32 values carried as two TF32 parts (x = hi + lo, the
// tensor core keeps the leading TF32 bits of lo); the product of a block and
// an input slice is formed from three part products, A_hi [B_hi | B_lo] and
// A_lo B_hi, into one TMEM accumulator (D = D[0:N) + D[N:2N)).
//
// CTA = one 128-row half of a row task (the MMA's M, padding rows zero; row
// tasks of up to MR = 128 or 256 rows, so one or two CTAs per task) x one
// chunk of NCOL columns, 10 warps with fixed roles:
//   warp 0      producer: per step (one 32-wide K chunk of one partner block)
//               bulk copies of the partner's input slice (from an "input
//               image") and of the chunk's columns of the block (contiguous
//               in the column-major block, all of its rows: both halves read
//               the same copy pattern) into a shared-memory ring;
//   warp 1      one thread issues the MMAs of a step and commits them;
//   warps 2-5   move the half's rows of the chunk into TMEM (operand A):
//               thread = block row, 32 values read from shared memory, split
//               into TF32 parts;
//   warps 6-9   read every partner's product back from TMEM (two or four
//               accumulators, so the next partners' products proceed), plain
//               sums over eight partners, compensated sums across in shared
//               memory, then the compensated update of the output rows.
// The input image is built per call: per column task and 32-wide K chunk,
// the hi and the lo parts of the chunk's rows of every column, one 128-byte
// row per column with the 16-byte chunk k at position k ^ (column mod 8)
// (the order of a 128-byte-swizzled K-major operand in shared memory).
// Every mbarrier wait is bounded; a timeout raises the error flag, which the
// launcher turns into H2_ERR_TIMEOUT.
#include <algorithm>
#include <type_traits>

#include "h2_level.h"
#include "h2_types.h"
#include "tc_ptx.cuh"

namespace h2 {
namespace {

constexpr int kKc = 32;                 // K values per chunk: one 128-byte TF32 row
constexpr int kR = 4;                   // step barriers (>= every stage count)
// one block chunk: up to MR rows x 32 columns
template <int MR>
__host__ __device__ constexpr uint32_t slot_a() {
  return MR * kKc * 4;
}
// Per-shape resources.  TWO: two CTAs per SM (16 columns, 128 rows: the
// narrow products of the adaptive rounds and of matvecs, whose time goes into
// streaming blocks, so two independent pipelines per SM), each with half of
// the TMEM.  SB: shared-memory stages (input slice + block chunk).  ACC:
// accumulators (partners in flight between the MMAs and the read-back).  SA:
// A stages in TMEM (steps the staging warps may run ahead of the MMAs).
template <int NCOL, int MR>
struct TcStages {
  static constexpr bool TWO = NCOL == 16 && MR == 128;
  static constexpr int SB = MR == 128 ? (NCOL >= 64 ? 3 : 4) : (NCOL >= 80 ? 2 : 3);
  static constexpr int TMEM_BUDGET = TWO ? 256 : 512;
  static constexpr int ACC = 4 * 2 * NCOL + 2 * 64 <= TMEM_BUDGET ? 4 : 2;
  static constexpr int SA = ACC * 2 * NCOL + 4 * 64 <= TMEM_BUDGET ? 4 : 2;
  static constexpr int USED = ACC * 2 * NCOL + SA * 64;
  static constexpr int TCOLS = USED <= 128 ? 128 : (USED <= 256 ? 256 : 512);
};
// A row's partner metadata (column task, block width, block offset) is read
// once into shared memory for its first kMeta partners.
constexpr int kMeta = 512;
constexpr int kWarps = 10;
constexpr int kThreadsTc = 32 * kWarps;
constexpr int kGroup = 8;               // partners summed plainly before a compensated fold

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t *v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
      "%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(
          taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]),
      "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]),
      "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

struct TcBsrArgs {
  BsrArgs a;
  const float *img;   // input image
  int64_t W;          // image rows per part (columns 0 .. W-1)
  int kcmax;          // K chunks per column task in the image
  int nchunk;         // column chunks per row task
  int *err;
};

// Input image of the call (see the file comment).  Block (b, kc).
__global__ void k_bsr_tc_image(BsrArgs a, int kcmax, int64_t W, float *img) {
  const int b = blockIdx.x / kcmax, kc = blockIdx.x % kcmax;
  const int kb = a.col_m[b];
  const int inst = a.row_inst[b];
  const int cb = a.cols.cb[inst], ce = a.cols.ce[inst];
  const float *in = reinterpret_cast<const float *>(a.in);
  const int64_t r0 = a.col_off[b] + (int64_t)kc * kKc;
  float *hi = img + ((int64_t)b * kcmax + kc) * 2 * W * kKc;
  float *lo = hi + W * kKc;
  for (int64_t q = threadIdx.x; q < W * kKc; q += blockDim.x) {
    const int c = (int)(q / kKc), j = (int)(q % kKc);
    const int k = kc * kKc + j;
    const float v = (k < kb && c >= cb && c < ce) ? in[r0 + j + (int64_t)c * a.ld_in] : 0.f;
    const float h = tf32_rna(v);
    const int64_t dst = (int64_t)c * kKc + (((j >> 2) ^ (c & 7)) << 2) + (j & 3);
    hi[dst] = h;
    lo[dst] = v - h;
  }
}

template <int NCOL, int MR>
__host__ __device__ constexpr size_t tc_bsr_smem() {
  return 1024 + (size_t)TcStages<NCOL, MR>::SB * (2 * NCOL * 128 + slot_a<MR>()) +
         (size_t)2 * NCOL * 128 * sizeof(float) + (size_t)kMeta * 16;
}

template <int NCOL, int MR>
__global__ void __launch_bounds__(kThreadsTc, TcStages<NCOL, MR>::TWO ? 2 : 1)
    k_bsr_tc(TcBsrArgs ta) {
  const BsrArgs &a = ta.a;
  constexpr uint32_t STAGE_B = 2 * NCOL * 128;        // hi rows then lo rows
  constexpr uint32_t ACC_N = 2 * NCOL;
  constexpr int kSA = TcStages<NCOL, MR>::SA;
  constexpr int kAcc = TcStages<NCOL, MR>::ACC;
  constexpr uint32_t A_COL0 = kAcc * ACC_N;           // the accumulators first
  constexpr uint32_t TCOLS = TcStages<NCOL, MR>::TCOLS;
  static_assert(A_COL0 + kSA * 64 <= TCOLS && TCOLS <= 512, "TMEM columns");
  static_assert(NCOL % 16 == 0, "MMA N");
  constexpr uint32_t IDESC2 = idesc_mma(false, 128, 2 * NCOL);
  constexpr uint32_t IDESC1 = idesc_mma(false, 128, NCOL);
  constexpr int kSB = TcStages<NCOL, MR>::SB;
  constexpr uint32_t kSlotA = slot_a<MR>();
  constexpr int kHalves = MR / 128;
  static_assert(kR >= kSB && kR >= kSA, "step barriers");
  static_assert(tc_bsr_smem<NCOL, MR>() * (TcStages<NCOL, MR>::TWO ? 2 : 1) <= 226 * 1024,
                "shared memory");
  extern __shared__ unsigned char smem_dyn[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  unsigned char *sB = base;                                            // [kSB][STAGE_B]
  float *sBlk = reinterpret_cast<float *>(sB + kSB * STAGE_B);         // [kSB][kSlotA]
  float *sAcc = sBlk + kSB * (kSlotA / 4);                             // [NCOL][128]
  float *sCmp = sAcc + NCOL * 128;
  int64_t *mBoff = reinterpret_cast<int64_t *>(sCmp + NCOL * 128);     // [kMeta]
  int32_t *mB = reinterpret_cast<int32_t *>(mBoff + kMeta);            // [kMeta]
  int32_t *mKb = mB + kMeta;                                           // [kMeta]
  __shared__ uint64_t bfull[kSB], afull[kSA], stepdone[kR], accfull[kAcc], accempty[kAcc];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;

  const int seg = a.seg;
  const int part = blockIdx.x % seg;
  int rest = blockIdx.x / seg;
  const int half = rest % kHalves;
  rest /= kHalves;
  const int chunk = rest % ta.nchunk;
  const int tau = rest / ta.nchunk;
  const int m = a.row_m[tau];        // rows of the task (the blocks' leading dimension)
  const int hr0 = half * 128;        // first row of this CTA's half
  const int mh = min(128, m - hr0);  // rows of the half (<= 0: nothing to do)
  const int inst = a.row_inst[tau];
  const int cb = a.cols.cb[inst], ce = a.cols.ce[inst];
  const int c0 = cb + chunk * NCOL;
  const int64_t r0 = a.ptr[tau], rn = a.ptr[tau + 1] - r0;
  const int64_t e0 = r0 + rn * part / seg, e1 = r0 + rn * (part + 1) / seg;
  if (mh <= 0 || c0 >= ce || e0 == e1) return;   // uniform over the CTA
  const int ncol = min(NCOL, ce - c0);

  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  auto abort_cta = [&]() {
    s_abort = 1;
    atomicExch(ta.err, 1);
  };
  const int64_t ecache = e1 - e0 < kMeta ? e1 - e0 : (int64_t)kMeta;
  for (int64_t q = t; q < ecache; q += blockDim.x) {
    const int b = a.idx[e0 + q];
    mB[q] = b;
    mKb[q] = a.col_m[b];
    mBoff[q] = a.boff[e0 + q];
  }
  // partner of entry e: (column task, block width, block offset)
  auto meta_b = [&](int64_t e) { return e - e0 < kMeta ? mB[e - e0] : a.idx[e]; };
  auto meta_kb = [&](int64_t e) {
    return e - e0 < kMeta ? mKb[e - e0] : a.col_m[a.idx[e]];
  };
  auto meta_boff = [&](int64_t e) { return e - e0 < kMeta ? mBoff[e - e0] : a.boff[e]; };
  if (t == 0) {
    for (int i = 0; i < kSB; ++i) mbar_init(saddr(&bfull[i]), 1);
    for (int i = 0; i < kSA; ++i) mbar_init(saddr(&afull[i]), 4);
    for (int i = 0; i < kR; ++i) mbar_init(saddr(&stepdone[i]), 1);
    for (int i = 0; i < kAcc; ++i) {
      mbar_init(saddr(&accfull[i]), 1);
      mbar_init(saddr(&accempty[i]), 4);
    }
    s_abort = *reinterpret_cast<volatile int *>(ta.err) != 0 ? 1 : 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     saddr(&tmem_base)),
                 "n"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = tmem_base;
  auto wait_step = [&](int64_t j) {   // the products of step j have completed
    return mbar_wait(saddr(&stepdone[j % kR]), (uint32_t)((j / kR) & 1), &s_abort);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int64_t s = 0;
      bool ok = s_abort == 0;
      for (int64_t e = e0; e < e1 && ok; ++e) {
        const int b = meta_b(e);
        const int kb = meta_kb(e);
        const int nkc = (kb + kKc - 1) / kKc;
        const int64_t boff = meta_boff(e);
        for (int kc = 0; kc < nkc; ++kc, ++s) {
          if (s >= kSB && !wait_step(s - kSB)) { ok = false; break; }
          // the chunk's columns of the block: contiguous (column-major, ld = m);
          // the copy rounds up to whole 16-byte units, within the block's
          // 16-byte padded extent
          const int nc = min(kKc, kb - kc * kKc);
          const uint32_t ablk = ((uint32_t)(m * nc) * 4u + 15u) & ~15u;
          const uint32_t bar = saddr(&bfull[s % kSB]);
          mbar_expect_tx(bar, STAGE_B + ablk);
          const float *src = ta.img + (((int64_t)b * ta.kcmax + kc) * 2 * ta.W + c0) * kKc;
          const uint32_t dst = saddr(sB + (s % kSB) * STAGE_B);
          bulk_g2s(dst, src, NCOL * 128, bar);
          bulk_g2s(dst + NCOL * 128, src + ta.W * kKc, NCOL * 128, bar);
          const float *bsrc = reinterpret_cast<const float *>(a.blocks) + boff +
                              (int64_t)kc * kKc * m;
          bulk_g2s(saddr(sBlk + (s % kSB) * (kSlotA / 4)), bsrc, ablk, bar);
        }
      }
      if (!ok) abort_cta();
      // every issued copy has landed before the CTA may end
      for (int64_t j = s > kSB ? s - kSB : 0; j < s; ++j)
        mbar_wait(saddr(&bfull[j % kSB]), (uint32_t)((j / kSB) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      int64_t s = 0;
      int64_t p = 0;   // partners with a non-empty block
      bool ok = s_abort == 0;
      for (int64_t e = e0; e < e1 && ok; ++e) {
        const int nkc = (meta_kb(e) + kKc - 1) / kKc;
        if (nkc == 0) continue;
        const int ac = (int)(p % kAcc);
        if (p >= kAcc &&
            !mbar_wait(saddr(&accempty[ac]), (uint32_t)(((p / kAcc) - 1) & 1), &s_abort)) {
          ok = false;
          break;
        }
        const uint32_t d = tbase + (uint32_t)(ac * ACC_N);
        for (int kc = 0; kc < nkc; ++kc, ++s) {
          if (!mbar_wait(saddr(&bfull[s % kSB]), (uint32_t)((s / kSB) & 1), &s_abort) ||
              !mbar_wait(saddr(&afull[s % kSA]), (uint32_t)((s / kSA) & 1), &s_abort)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t a_hi = tbase + A_COL0 + (uint32_t)((s % kSA) * 64), a_lo = a_hi + 32;
          const uint32_t bst = saddr(sB + (s % kSB) * STAGE_B);
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint64_t db = desc_sw128(bst + ks * 32);
            mma_ts<false>(d, a_hi + ks * 8, db, IDESC2, (kc | ks) ? 1u : 0u);
            mma_ts<false>(d, a_lo + ks * 8, db, IDESC1, 1u);
          }
          mma_commit(saddr(&stepdone[s % kR]));
        }
        if (!ok) break;
        mma_commit(saddr(&accfull[ac]));
        ++p;
      }
      if (!ok) abort_cta();
      // the products issued last have completed before the CTA may end
      if (s > 0) mbar_wait(saddr(&stepdone[(s - 1) % kR]), (uint32_t)(((s - 1) / kR) & 1));
    }
    __syncwarp();
  } else if (warp < 6) {
    // ------------------------------------------------------------ block staging
    const int quad = warp & 3;
    const int i = quad * 32 + lane;   // row of this thread in the half
    const bool rowok = i < mh;
    const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
    int64_t s = 0;
    bool alive = s_abort == 0;
    for (int64_t e = e0; e < e1 && alive; ++e) {
      const int kb = meta_kb(e);
      const int nkc = (kb + kKc - 1) / kKc;
      for (int kc = 0; kc < nkc; ++kc, ++s) {
        // the chunk has landed in slot s % kSB (the products' B wait, shared)
        if (!__all_sync(0xffffffffu, mbar_wait(saddr(&bfull[s % kSB]),
                                               (uint32_t)((s / kSB) & 1), &s_abort)) ||
            (s >= kSA && !__all_sync(0xffffffffu, wait_step(s - kSA)))) {
          alive = false;
          if (lane == 0) abort_cta();
          break;
        }
        const int nc = min(kKc, kb - kc * kKc);
        const float *slot = sBlk + (s % kSB) * (kSlotA / 4);
        uint32_t hv[kKc], lv[kKc];
#pragma unroll
        for (int j = 0; j < kKc; ++j) {
          const float v = (rowok && j < nc) ? slot[j * m + hr0 + i] : 0.f;
          const float h = tf32_rna(v);
          hv[j] = __float_as_uint(h);
          lv[j] = __float_as_uint(v - h);
        }
        const uint32_t at = tbase + lane_addr + A_COL0 + (uint32_t)((s % kSA) * 64);
        __syncwarp();
        tmem_st32(at, hv);
        tmem_st32(at + 32, lv);
        tmem_st_wait();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(saddr(&afull[s % kSA]));
      }
    }
  } else {
    // ------------------------------------------------------------ read-back
    const int quad = warp & 3;
    const int i = quad * 32 + lane;
    const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
    float grp[NCOL];
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
      grp[c] = 0.f;
      sAcc[c * 128 + i] = 0.f;
      sCmp[c * 128 + i] = 0.f;
    }
    auto fold = [&]() {
#pragma unroll
      for (int c = 0; c < NCOL; ++c) {
        const float ac = sAcc[c * 128 + i], cm = sCmp[c * 128 + i];
        const float y = grp[c] - cm;
        const float s2 = ac + y;
        sCmp[c * 128 + i] = (s2 - ac) - y;
        sAcc[c * 128 + i] = s2;
        grp[c] = 0.f;
      }
    };
    int64_t p = 0;
    bool alive = s_abort == 0;
    for (int64_t e = e0; e < e1 && alive; ++e) {
      if (meta_kb(e) == 0) continue;
      const int ac = (int)(p % kAcc);
      if (!__all_sync(0xffffffffu,
                      mbar_wait(saddr(&accfull[ac]), (uint32_t)((p / kAcc) & 1), &s_abort))) {
        alive = false;
        if (lane == 0) abort_cta();
        break;
      }
      fence_after();
      const uint32_t ta0 = tbase + lane_addr + (uint32_t)(ac * ACC_N);
#pragma unroll
      for (int c = 0; c < NCOL; c += 16) {
        float v[16], w[16];
        tmem_ld16(ta0 + c, v);
        tmem_ld16(ta0 + NCOL + c, w);
        tmem_ld_wait();
#pragma unroll
        for (int u = 0; u < 16; ++u) grp[c + u] += v[u] + w[u];
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(saddr(&accempty[ac]));
      ++p;
      if (p % kGroup == 0) fold();
    }
    fold();
    if (alive && i < mh) {
      float *out = reinterpret_cast<float *>(a.out);
      const float sgn = (float)a.sign;
      const int64_t orow = a.row_off[tau] + hr0 + i;
      for (int c = 0; c < ncol; ++c) {
        float *op = out + orow + (int64_t)(c0 + c) * a.ld_out;
        const float v = sgn * sAcc[c * 128 + i];
        if (seg > 1) {
          atomicAdd(op, v - sgn * sCmp[c * 128 + i]);
        } else {
          // compensated update: old + v with the sum's rounding error kept
          const float old = *op;
          const float s2 = old + v;
          const float bp = s2 - old;
          const float err = (old - (s2 - bp)) + (v - bp) - sgn * sCmp[c * 128 + i];
          *op = s2 + err;
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase),
                 "n"(TCOLS));
}

template <int NCOL, int MR>
void launch_bsr_tc(const TcBsrArgs &ta, int64_t ctas, cudaStream_t s) {
  auto kern = k_bsr_tc<NCOL, MR>;
  const size_t bytes = tc_bsr_smem<NCOL, MR>();
  H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  if (TcStages<NCOL, MR>::TWO)   // room for two CTAs per SM
    H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  kern<<<(unsigned)ctas, kThreadsTc, bytes, s>>>(ta);
  count_launch();
  H2_CHECK_LAUNCH();
}

}  // namespace

bool bsr_apply_tc(const BsrArgs &a, int max_m, int max_cols, cudaStream_t s) {
  if (max_m <= 0 || max_m > 256 || max_cols <= 0 || a.col_hi <= 0 || a.n_rows <= 0) return false;
  const int ncol = max_cols <= 16 ? 16 : (max_cols <= 32 ? 32 : (max_cols <= 64 ? 64
                                                                 : (max_cols <= 80 ? 80 : 96)));
  TcBsrArgs ta{};
  ta.a = a;
  ta.kcmax = (max_m + kKc - 1) / kKc;
  ta.W = (a.col_hi + 7) / 8 * 8;
  ta.nchunk = (max_cols + ncol - 1) / ncol;
  const int64_t img_floats = (int64_t)a.n_rows * ta.kcmax * 2 * ta.W * kKc;
  // slack past the end: the last chunk's copy may read up to ncol rows beyond
  // its column range (those products land in accumulator columns that are
  // never stored)
  const int64_t slack = (int64_t)2 * 96 * kKc;
  DBuf<float> img;
  img.alloc((size_t)(img_floats + slack));
  H2_CUDA(cudaMemsetAsync(img.p + img_floats, 0, (size_t)slack * sizeof(float), s));
  DBuf<int> err;
  err.alloc_zero(1, s);
  ta.img = img.p;
  ta.err = err.p;
  k_bsr_tc_image<<<(unsigned)((int64_t)a.n_rows * ta.kcmax), 256, 0, s>>>(a, ta.kcmax, ta.W,
                                                                            img.p);
  count_launch();
  H2_CHECK_LAUNCH();
  const int halves = max_m > 128 ? 2 : 1;
  const int64_t ctas = (int64_t)a.n_rows * halves * ta.nchunk * a.seg;
  auto go = [&](auto mr) {
    constexpr int MR = decltype(mr)::value;
    switch (ncol) {
      case 16: launch_bsr_tc<16, MR>(ta, ctas, s); break;
      case 32: launch_bsr_tc<32, MR>(ta, ctas, s); break;
      case 64: launch_bsr_tc<64, MR>(ta, ctas, s); break;
      case 80: launch_bsr_tc<80, MR>(ta, ctas, s); break;
      default: launch_bsr_tc<96, MR>(ta, ctas, s); break;
    }
  };
  if (halves == 1) go(std::integral_constant<int, 128>{});
  else go(std::integral_constant<int, 256>{});
  if (to_host(err.p, 1, s)[0] != 0)
    throw Error{H2_ERR_TIMEOUT, "tensor-core block-sparse product: a bounded wait ran out"};
  return true;
}

}  // namespace h2
