// Fused kernel summation Y = K Omega on the 5th-generation tensor cores.
//
// The sketch of Algorithm 1 is a dense contraction over the point index j
// whose left operand K(x_i, x_j) is generated on the fly.
//
// Two-part operands.  Each FP32 value x is carried as two low-precision
// parts, and the product is formed from three part products (the fourth is
// below FP32 rounding):
//   TF32 mode: x = hi + lo, hi = rna_tf32(x), lo = rna_tf32(x - hi);
//              Y = A_hi B_hi + A_hi B_lo + A_lo B_hi   (K = 8 per MMA).
//   FP16 mode: the entries are formed as x' = 2048 x; h' = rn_f16(x'),
//              t = rn_f16(h' - x') (one mixed-precision subtraction of the
//              packed h'); Omega as w = h_w + (w - h_w), its image holding
//              h_w and rn_f16(h_w - w);
//              Y = 2^-11 (A_h B_h - (A_h B_s + A_s B_h))  (K = 16 per MMA).
// FP16 halves the MMA count per point; it is used when every entry is at
// most 1 (exponential, Matern, Gaussian kernels) and |Omega| is bounded,
// so no part leaves the FP16 range (tiny entries fall to subnormals with an
// absolute error near 2^-36).  Products are always of the form
// A_1 * [B_1 | B_2] (one MMA of width 2 NCOL; the two B parts are adjacent
// in shared memory) plus A_2 * B_1 into one half of the accumulator: a
// tcgen05.mma costs about the same for any width up to this size, so fewer,
// wider products win.
//
// Layout.  Points are grouped by leaf and every leaf is padded to whole
// tiles of TJ points (32 in TF32 mode, 64 in FP16 mode: 128 bytes per row
// either way).  The build stores, per padded point, its offset from its
// leaf's reference point (FP32, already multiplied by the kernel's scale
// factor sigma; per tile the x offsets of its points, then the y and the z
// offsets, so that a thread loads its points four at a time and works on
// them in packed pairs), and per leaf that reference (sigma * x_ref as FP32
// hi/lo parts).  Every sample call stores an "Omega image": per tile and column
// the TJ values' two parts in the 128-byte-swizzled K-major order the MMA
// reads, so one bulk copy per part moves a tile's operand into shared
// memory.  Padding rows are zero.
//
// A distance is formed as (row - r_ref) + (r_ref - t_ref) - (point - t_ref):
// the first and last terms are small offsets computed in FP64 and rounded
// once, the middle one is a difference of hi/lo parts, so the FP32 result
// carries an error of a few units of 2^-24 of the distance itself.
//
// CTA = 128 rows (one or two leaves, or 128 consecutive rows) x NCOL sample
// columns, 18 warps with fixed roles:
//   warp 0     producer: walks the tile sequence (all leaves; the far
//              leaves only; or the union of the row leaves' near lists, for
//              the near-field product of the norm estimate; metadata and
//              near flags of 32 leaves are
//              loaded by the whole warp at a time), writes each tile's
//              reference shift, issues the bulk copies of its Omega parts
//              and point offsets;
//   warp 1     one thread issues the two MMAs of each of the four K-steps
//              of a tile into a fresh TMEM accumulator and commits them
//              (one commit per tile releases the B stage, the A stage and
//              the accumulator);
//   warps 2-17 evaluate the tile's 128 x TJ entries (thread = row x TJ/4
//              points), store their parts into TMEM (tcgen05.st: the MMA
//              reads operand A from tensor memory, so the entry tile never
//              passes through shared memory), and read back the
//              accumulator of an earlier tile (tcgen05.ld).
// Accumulating many products in TMEM loses precision (measured: 3.8e-6
// relative after 192 products, 3.9e-7 when every 12-product tile is read
// back), so every tile gets a fresh accumulator; the per-tile partials are
// added plainly in groups of eight and the groups with compensation.
// Rings: kSA operand-A stages (TMEM), kSB operand-B stages (shared memory),
// NA TMEM accumulators, kR completion barriers (one per tile in flight).
// Every mbarrier wait is bounded (0.2 s); a timeout raises the error flag,
// the CTA ends only after its copies and products have landed, and CTAs
// that start after the flag is raised return at once.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>

#include "h2_ops.h"
#include "h2_types.h"
#include "tc_ptx.cuh"

namespace h2 {
namespace {

constexpr int kRows = 128;     // MMA M, TMEM lanes
constexpr int kSA = 2, kSB = 5, kR = 5;
// TMEM accumulators of 2 x NCOL columns: two up to 64 columns, one for 80
// (2 x 160 + 256 operand columns would not fit in 512); the read-back of
// step k-1 always follows the operands of step k.
template <int NCOL>
struct TcAcc {
  static constexpr int NA = NCOL > 64 ? 1 : 2;
  // 18 warps put five on two sub-partitions, whose 16K registers cap a
  // thread at 96: from 64 columns on the compensated sums live in shared
  // memory (and the B ring is shorter to make room)
  static constexpr bool SMEM_SUMS = NCOL >= 64;
  static constexpr int SB = NCOL > 64 ? 3 : (NCOL == 64 ? 4 : kSB);
};
constexpr int kEvalWarps = 16;
constexpr int kThreads = 32 * (2 + kEvalWarps);
// Points per tile: 128-byte operand rows of TF32 or FP16 values.
template <bool F16>
struct TcTile {
  static constexpr int TJ = F16 ? 64 : 32;
};
constexpr float kS16 = 2048.f;          // FP16 mode: scale of the second part
constexpr float kInvS16 = 1.f / 2048.f;
constexpr float kLn2 = 0.693147180559945309f;
constexpr double kLog2e = 1.4426950408889634074;

// Scale factor sigma applied to coordinates so that the entry needs no
// further multiplication:  exp: K = 2^-r';  Matern 3/2: K = (1 + r' ln2) 2^-r'
// with r' = sigma |x - y|;  Gaussian: K = 2^-(r'^2);  Laplace, Helmholtz and
// polynomial kernels keep unscaled coordinates.
double tc_sigma(const KernelDesc &kd) {
  switch (kd.kid) {
    case H2_K_EXP:
    case H2_K_MATERN32: return kd.scale * kLog2e;
    case H2_K_GAUSS: return std::sqrt(kd.scale * kLog2e);
    default: return 1.0;
  }
}

// Entry from the scaled row coordinates (rx, ry, rz) and a scaled point
// offset p (the polynomial kernel: absolute coordinates).  `c` is the
// Laplace factor 1/(4 pi), the Helmholtz wave number or the polynomial shift.
// S (FP16 parts): the entry times 2048, the scale at which its two FP16
// parts are formed (see split_parts).
template <int KID, bool S = false>
__device__ __forceinline__ float tc_entry(float rx, float ry, float rz, float4 p, float c, int pw) {
  if constexpr (KID == H2_K_POLY) {
    const float base = c + (rx * p.x + ry * p.y + rz * p.z);
    float v = 1.f;
    for (int q = 0; q < pw; ++q) v *= base;
    return v;
  } else {
    const float dx = rx - p.x, dy = ry - p.y, dz = rz - p.z;
    const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    if constexpr (KID == H2_K_GAUSS) {
      return S ? ex2_approx(-r2) * kS16 : ex2_approx(-r2);
    } else if constexpr (KID == H2_K_LAPLACE_IE) {
      return r2 > 0.f ? rsqrtf(r2) * c : 0.f;
    } else if constexpr (KID == H2_K_HELMHOLTZ_IE) {
      if (!(r2 > 0.f)) return 0.f;
      const float ir = rsqrtf(r2);
      return cos_reduced(c * (r2 * ir)) * ir;
    } else {
      const float r = sqrt_approx(r2);
      const float e = ex2_approx(-r);
      if constexpr (KID == H2_K_EXP) return S ? e * kS16 : e;
      else if constexpr (S) return fmaf(r, kS16 * kLn2, kS16) * e;
      else return fmaf(r * kLn2, e, e);
    }
  }
}

// Packed pairs of FP32 values (f32x2 arithmetic: one instruction for two
// lanes of work, same rounding as the scalar operations).
__device__ __forceinline__ uint64_t f2(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2u(uint64_t v, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// 2048 x for two entries of the exponential, Matern or Gaussian kernel at the
// scaled offsets (dx, dy, dz) of two points from the row (packed pairs).
template <int KID>
__device__ __forceinline__ uint64_t tc_entry2_s(uint64_t rx, uint64_t ry, uint64_t rz, uint64_t px,
                                                uint64_t py, uint64_t pz) {
  const uint64_t dx = f2_sub(rx, px), dy = f2_sub(ry, py), dz = f2_sub(rz, pz);
  const uint64_t r2 = f2_fma(dz, dz, f2_fma(dy, dy, f2_mul(dx, dx)));
  const uint64_t s16 = f2(kS16, kS16);
  if constexpr (KID == H2_K_GAUSS) {
    float a, b;
    f2u(r2, a, b);
    return f2_mul(f2(ex2_approx(-a), ex2_approx(-b)), s16);
  } else {
    float a, b;
    f2u(r2, a, b);
    const float ra = sqrt_approx(a), rb = sqrt_approx(b);
    const uint64_t e = f2(ex2_approx(-ra), ex2_approx(-rb));
    if constexpr (KID == H2_K_EXP) {
      return f2_mul(e, s16);
    } else {
      const uint64_t c1 = f2(kS16 * kLn2, kS16 * kLn2);
      return f2_mul(f2_fma(f2(ra, rb), c1, s16), e);
    }
  }
}

// Per-stage control word written by the producer: one step of up to two
// tiles.
struct TcCtrl {
  float dx[2], dy[2], dz[2];   // r_ref - t_ref of each tile's leaf (scaled)
  int flags[2];                // 1: near to the first row leaf, 2: near to the second
  int64_t j0[2];               // tree position of each tile's first point
  int nt;                      // tiles in the step (0: end of the sequence)
};

template <int NCOL, bool F16>
constexpr size_t tc_smem_bytes() {
  return 1024 + (size_t)TcAcc<NCOL>::SB * 2 * (2 * NCOL * 128 + TcTile<F16>::TJ * 16) +
         (TcAcc<NCOL>::SMEM_SUMS ? (size_t)2 * kRows * NCOL * sizeof(float) : 0);
}

// The two parts of 8 (FP16 mode: 16) entries, packed as the TMEM columns of
// one thread's lane.
// FP16 mode: kv holds x' = 2048 x.  Part 1 is h' = rn_f16(x') (= 2048 h,
// h = rn_f16(x)), part 2 is t = rn_f16(h' - x') (= -2048 (x - h), the scaled
// residual with its sign flipped); h' - x' comes from one mixed-precision
// subtraction of the packed part 1, so no part is unpacked.  The Omega image
// carries (h_w, h_w - w) for each value w; the products then give
// x w = 2^-11 (D_1 - D_2) with D_1 = h' h_w and D_2 = h' (h_w - w) + t h_w
// (up to the product of the two residuals, below FP32 rounding).
template <bool F16, int EPT>
__device__ __forceinline__ void split_parts(const float *kv, uint32_t *p1, uint32_t *p2) {
  if constexpr (F16) {
#pragma unroll
    for (int u = 0; u < EPT / 2; ++u) {
      uint32_t h, r;
      float t0, t1;
      asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(h) : "f"(kv[2 * u + 1]), "f"(kv[2 * u]));
      asm("{\n.reg .b16 lo, hi;\nmov.b32 {lo, hi}, %2;\n"
          "sub.f32.f16 %0, lo, %3;\nsub.f32.f16 %1, hi, %4;\n}\n"
          : "=f"(t0), "=f"(t1)
          : "r"(h), "f"(kv[2 * u]), "f"(kv[2 * u + 1]));
      asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(t1), "f"(t0));
      p1[u] = h;
      p2[u] = r;
    }
  } else {
#pragma unroll
    for (int u = 0; u < EPT; ++u) {
      const float hv = tf32_rna(kv[u]);
      p1[u] = __float_as_uint(hv);
      p2[u] = __float_as_uint(kv[u] - hv);   // the tensor core keeps its leading TF32 bits
    }
  }
}

// MODE: 0 all points, 1 far-only (leaves not on a row leaf's near list),
// 2 near-only (the union of the row leaves' near lists, from a.ul_leaf).
template <int KID, int NCOL, int MODE, bool F16>
__global__ void __launch_bounds__(kThreads, 1) k_ksum_tc(TcArgs a) {
  constexpr bool FAR = MODE == 1;
  constexpr bool MASKED = MODE != 0;
  constexpr int TJ = TcTile<F16>::TJ;
  constexpr int EPT = TJ / 4;                         // entries per eval thread and tile
  constexpr int CPT = NCOL / 4;                       // accumulator columns per eval thread
  constexpr uint32_t B_BYTES = NCOL * 128;            // one part of an NCOL x TJ tile
  constexpr uint32_t OFF_BYTES = TJ * 16;
  constexpr uint32_t B_STAGE = 2 * (2 * B_BYTES);     // two tiles, two parts each
  // TMEM columns: kNA accumulators of 2 x NCOL, then kSA operand-A stages of
  // 128 columns: part 1 of the two tiles (32 columns each), then part 2
  constexpr int kNA = TcAcc<NCOL>::NA;
  constexpr int kSB = TcAcc<NCOL>::SB;              // B stages of this width
  constexpr bool SMEM_SUMS = TcAcc<NCOL>::SMEM_SUMS;
  constexpr uint32_t ACC_N = 2 * NCOL;
  constexpr uint32_t A_COL0 = kNA * ACC_N;
  constexpr uint32_t TCOLS = A_COL0 + kSA * 128 <= 256 ? 256 : 512;
  static_assert(A_COL0 + kSA * 128 <= 512, "TMEM columns");
  static_assert(kSA == 2, "the read-back of step k-1 releases the A stage of step k+1");
  constexpr uint32_t IDESC2 = idesc_mma(F16, kRows, 2 * NCOL);
  constexpr uint32_t IDESC1 = idesc_mma(F16, kRows, NCOL);
  // second product A_2 * B_1: TF32 adds it to the first half, FP16 to the
  // scaled second half
  constexpr uint32_t D2_OFF = F16 ? NCOL : 0;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  unsigned char *sB = base;                                          // [kSB][tile][part]
  float4 *sOff = reinterpret_cast<float4 *>(sB + kSB * B_STAGE);    // [kSB][tile][TJ]
  // compensated sums [column][row] (SMEM_SUMS only)
  float *sAcc = reinterpret_cast<float *>(sOff + kSB * 2 * TJ);
  float *sCmp = sAcc + kRows * NCOL;
  __shared__ TcCtrl ctrl[kSB];
  __shared__ uint64_t bfull[kSB], afull[kSA], done[kR], accempty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int s_abort;
  __shared__ float4 m_rh[32], m_rl[32];   // producer: metadata of 32 leaves
  __shared__ int64_t m_t0[32], m_j0[32];
  __shared__ int m_nt[32], m_fl[32];

  const KsumItem it = a.items[blockIdx.x];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  auto abort_cta = [&]() {
    s_abort = 1;
    atomicExch(a.err, 1);
  };
  // completion of the products of step j (one commit per step)
  auto wait_done = [&](int j) {
    return mbar_wait(saddr(&done[j % kR]), (uint32_t)((j / kR) & 1), &s_abort);
  };

  if (t == 0) {
    for (int i = 0; i < kSB; ++i) mbar_init(saddr(&bfull[i]), 1);
    for (int i = 0; i < kSA; ++i) mbar_init(saddr(&afull[i]), kEvalWarps);
    for (int i = 0; i < kR; ++i) mbar_init(saddr(&done[i]), 1);
    for (int i = 0; i < kNA; ++i) mbar_init(saddr(&accempty[i]), kEvalWarps);
    // a CTA that timed out earlier in this launch makes the later ones skip their work
    s_abort = *reinterpret_cast<volatile int *>(a.err) != 0 ? 1 : 0;
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
  const InstDev in = a.inst[it.inst];
  const double sg = a.sigma[it.inst];
  // reference of the row tile: its first row (the origin for the polynomial kernel)
  const double cx = KID == H2_K_POLY ? 0.0 : a.p64.x[it.row0];
  const double cy = KID == H2_K_POLY ? 0.0 : a.p64.y[it.row0];
  const double cz = KID == H2_K_POLY ? 0.0 : a.p64.z[it.row0];

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    // The warp loads the metadata and near flags of 32 leaves at a time into
    // shared memory; lane 0 then pairs their tiles into steps and issues them.
    const double sx = cx * sg, sy = cy * sg, sz = cz * sg;
    const float hx = (float)sx, hy = (float)sy, hz = (float)sz;
    const float lx = (float)(sx - hx), ly = (float)(sy - hy), lz = (float)(sz - hz);
    int k = 0;
    bool ok = true;
    // the first tile of the step being assembled
    bool pend = false;
    int64_t p_tile = 0, p_j0 = 0;
    float4 p_rh, p_rl;
    int p_flags = 0;
    auto emit = [&](int nt, int64_t t1, int64_t j1, const float4 &rh1, const float4 &rl1,
                    int f1) {
      const int sb = k % kSB;
      if (k >= kSB && !wait_done(k - kSB)) {   // the stage's last products have completed
        ok = false;
        return;
      }
      TcCtrl c;
      c.nt = nt;
      const int64_t tiles[2] = {p_tile, t1};
      const float4 rhs[2] = {p_rh, rh1}, rls[2] = {p_rl, rl1};
      c.flags[0] = p_flags;
      c.flags[1] = f1;
      c.j0[0] = p_j0;
      c.j0[1] = j1;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        c.dx[h] = (hx - rhs[h].x) + (lx - rls[h].x);
        c.dy[h] = (hy - rhs[h].y) + (ly - rls[h].y);
        c.dz[h] = (hz - rhs[h].z) + (lz - rls[h].z);
      }
      ctrl[sb] = c;
      const uint32_t bar = saddr(&bfull[sb]);
      if (nt == 0) {
        mbar_arrive(bar);
      } else {
        mbar_expect_tx(bar, (uint32_t)nt * (2 * B_BYTES + OFF_BYTES));
        for (int h = 0; h < nt; ++h) {
          const int64_t img = (tiles[h] * a.img_nc + a.img_c0) * 32;   // 128-byte rows
          const uint32_t dst = saddr(sB + sb * B_STAGE + h * 2 * B_BYTES);
          bulk_g2s(dst, a.img_hi + img, B_BYTES, bar);
          bulk_g2s(dst + B_BYTES, a.img_lo + img, B_BYTES, bar);
          bulk_g2s(saddr(sOff + (sb * 2 + h) * TJ), a.off + tiles[h] * TJ, OFF_BYTES, bar);
        }
      }
      ++k;
    };
    auto add_tile = [&](int64_t tile, int64_t j0, const float4 &rh, const float4 &rl,
                        int flags) {
      if (!pend) {
        pend = true;
        p_tile = tile;
        p_j0 = j0;
        p_rh = rh;
        p_rl = rl;
        p_flags = flags;
      } else {
        emit(2, tile, j0, rh, rl, flags);
        pend = false;
      }
    };
    int64_t p1 = 0, e1 = 0, p2 = 0, e2 = 0;
    bool two = false;
    if (FAR) {
      const int t1 = it.task;
      two = it.rows > a.leaf_m[t1];
      p1 = a.near_ptr[t1];
      e1 = a.near_ptr[t1 + 1];
      if (two) { p2 = a.near_ptr[t1 + 1]; e2 = a.near_ptr[t1 + 2]; }
    }
    // bit i: leaf b0 + i is on the sorted near list [p, e); p moves past it
    auto near_bits = [&](int64_t &p, int64_t e, int b0) -> uint32_t {
      for (;;) {   // skip entries below b0, 32 at a time
        const int v = p + lane < e ? a.near_idx[p + lane] : INT32_MAX;
        const uint32_t below = __ballot_sync(0xffffffffu, v < b0);
        p += __popc(below);
        if (below != 0xffffffffu) break;
      }
      const int v = p + lane < e ? a.near_idx[p + lane] : INT32_MAX;
      const bool in = v < b0 + 32;
      p += __popc(__ballot_sync(0xffffffffu, in));
      return __reduce_or_sync(0xffffffffu, in ? 1u << (v - b0) : 0u);
    };
    for (int b0 = a.stall ? it.lb1 : it.lb0; b0 < it.lb1; b0 += 32) {
      if (__any_sync(0xffffffffu, s_abort != 0)) ok = false;
      if (!ok) break;
      uint32_t n1 = 0, n2 = 0xffffffffu;
      if (FAR) {
        n1 = near_bits(p1, e1, b0);
        if (two) n2 = near_bits(p2, e2, b0);
      }
      const int e = b0 + lane;
      int b = e;
      if (MODE == 2 && e < it.lb1) {   // entry e of the item's near-union list
        b = a.ul_leaf[e];
        m_fl[lane] = a.ul_flags[e];
      }
      if (e < it.lb1) {
        m_rh[lane] = a.ref_hi[b];
        m_rl[lane] = a.ref_lo[b];
        m_t0[lane] = a.leaf_tile[b];
        m_j0[lane] = a.leaf_row[b];
        m_nt[lane] = (a.leaf_m[b] + TJ - 1) / TJ;
      }
      __syncwarp();
      if (lane == 0) {
        const int nb = it.lb1 - b0 < 32 ? it.lb1 - b0 : 32;
        for (int i = 0; i < nb && ok; ++i) {
          const int f1 = (n1 >> i) & 1, f2 = (n2 >> i) & 1;
          if (FAR && f1 && f2) continue;
          const int flags = FAR ? (f1 | (f2 << 1)) : (MODE == 2 ? m_fl[i] : 0);
          const float4 rh = m_rh[i], rl = m_rl[i];
          const int64_t t0 = m_t0[i], j0 = m_j0[i];
          for (int u = 0; u < m_nt[i] && ok; ++u) add_tile(t0 + u, j0 + TJ * u, rh, rl, flags);
        }
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();
    }
    if (lane == 0 && !a.stall) {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ok && pend) emit(1, 0, 0, z, z, 0);
      if (ok) emit(0, 0, 0, z, z, 0);
      if (!ok) abort_cta();
      // every issued copy has landed before the CTA may end
      for (int j = k > kSB ? k - kSB : 0; j < k; ++j)
        mbar_wait(saddr(&bfull[j % kSB]), (uint32_t)((j / kSB) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issue
    if (lane == 0) {
      int k = 0;
      for (;; ++k) {
        const int sb = k % kSB, sa = k % kSA, ac = k % kNA;
        if (!mbar_wait(saddr(&bfull[sb]), (uint32_t)((k / kSB) & 1), &s_abort)) {
          abort_cta();
          break;
        }
        const int nt = ctrl[sb].nt;
        if (nt == 0) break;
        if (!mbar_wait(saddr(&afull[sa]), (uint32_t)((k / kSA) & 1), &s_abort)) {
          abort_cta();
          break;
        }
        if (k >= kNA &&
            !mbar_wait(saddr(&accempty[ac]), (uint32_t)(((k / kNA) - 1) & 1), &s_abort)) {
          abort_cta();
          break;
        }
        fence_after();
        const uint32_t a1 = tbase + A_COL0 + (uint32_t)(sa * 128), a2 = a1 + 64;
        const uint32_t b1 = saddr(sB + sb * B_STAGE);
        const uint32_t d = tbase + (uint32_t)(ac * ACC_N);
        for (int h = 0; h < nt; ++h) {
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            // rows: B part 1 then part 2 of tile h
            const uint64_t db = desc_sw128(b1 + h * 2 * B_BYTES + ks * 32);
            const uint32_t ac_ = (h | ks) ? 1u : 0u;
            mma_ts<F16>(d, a1 + h * 32 + ks * 8, db, IDESC2, ac_);
            mma_ts<F16>(d + D2_OFF, a2 + h * 32 + ks * 8, db, IDESC1, 1u);
          }
        }
        mma_commit(saddr(&done[k % kR]));
      }
      // the products issued last have completed before the CTA may end
      if (k > 0) mbar_wait(saddr(&done[(k - 1) % kR]), (uint32_t)(((k - 1) / kR) & 1));
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ evaluation + read-back
    const int quad = warp & 3;            // TMEM lane quadrant reachable by this warp
    const int q = (warp - 2) >> 2;        // point quarter of a tile and column quarter
    const int r = quad * 32 + lane;       // row of the tile
    const bool rowok = r < it.rows;
    const int64_t g = it.row0 + (rowok ? r : 0);
    const float rx0 = (float)((a.p64.x[g] - cx) * sg);
    const float ry0 = (float)((a.p64.y[g] - cy) * sg);
    const float rz0 = (float)((a.p64.z[g] - cz) * sg);
    const int nearbit = (MASKED && r >= a.leaf_m[MASKED ? it.task : 0]) ? 2 : 1;
    const float kc = (float)in.kd.scale;
    const int pw = in.kd.pw;
    const uint32_t lane_addr = (uint32_t)(quad * 32) << 16;
    constexpr int CR = SMEM_SUMS ? 1 : CPT;   // register-resident compensated sums
    float grp[CPT], acc[CR], cmp[CR];
    float *sa = sAcc + (q * CPT) * kRows + r, *sc = sCmp + (q * CPT) * kRows + r;
#pragma unroll
    for (int c = 0; c < CPT; ++c) grp[c] = 0.f;
#pragma unroll
    for (int c = 0; c < CR; ++c) { acc[c] = 0.f; cmp[c] = 0.f; }
    if constexpr (SMEM_SUMS) {
#pragma unroll
      for (int c = 0; c < CPT; ++c) { sa[c * kRows] = 0.f; sc[c * kRows] = 0.f; }
    }
    auto fold = [&]() {
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        if constexpr (SMEM_SUMS) {
          const float ac = sa[c * kRows], cm = sc[c * kRows];
          const float y = grp[c] - cm;
          const float s2 = ac + y;
          sc[c * kRows] = (s2 - ac) - y;
          sa[c * kRows] = s2;
        } else {
          const float y = grp[c] - cmp[c % CR];
          const float s2 = acc[c % CR] + y;
          cmp[c % CR] = (s2 - acc[c % CR]) - y;
          acc[c % CR] = s2;
        }
        grp[c] = 0.f;
      }
    };
    auto total = [&](int c) -> float {
      if constexpr (SMEM_SUMS) return sa[c * kRows];
      else return acc[c % CR];
    };
    bool alive = true;
    auto fail = [&]() {
      alive = false;
      if (lane == 0) abort_cta();
    };
    // read-back of step j; it also proves the A stage of step j + kSA free
    auto drain = [&](int j) {
      const int ac = j % kNA;
      if (!__all_sync(0xffffffffu, wait_done(j))) { fail(); return; }
      fence_after();
      float v[CPT], w[CPT];
      const uint32_t ta = tbase + lane_addr + (uint32_t)(ac * ACC_N + q * CPT);
      tmem_ld<CPT>(ta, v);
      tmem_ld<CPT>(ta + NCOL, w);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(saddr(&accempty[ac]));
      if constexpr (F16) {
        const uint64_t sc2 = f2(kInvS16, kInvS16);
#pragma unroll
        for (int c = 0; c < CPT; c += 2) {
          const uint64_t d = f2_sub(f2(v[c], v[c + 1]), f2(w[c], w[c + 1]));
          f2u(f2_fma(d, sc2, f2(grp[c], grp[c + 1])), grp[c], grp[c + 1]);
        }
      } else {
#pragma unroll
        for (int c = 0; c < CPT; ++c) grp[c] += v[c] + w[c];
      }
      if ((j & 7) == 7) fold();   // plain sums over 8 steps, compensated across
    };
    int k = 0;
    for (;; ++k) {
      const int sb = k % kSB, sa = k % kSA;
      if (!__all_sync(0xffffffffu, mbar_wait(saddr(&bfull[sb]), (uint32_t)((k / kSB) & 1),
                                             &s_abort))) {
        fail();
        break;
      }
      const int nt = ctrl[sb].nt;
      if (nt == 0) break;
      const uint32_t at = tbase + lane_addr + A_COL0 + (uint32_t)(sa * 128 + 8 * q);
      for (int h = 0; h < nt; ++h) {
        const bool live = rowok && !(MASKED && (ctrl[sb].flags[h] & nearbit));
        uint32_t p1[8], p2[8];
        if (live) {
          const float rx = rx0 + ctrl[sb].dx[h], ry = ry0 + ctrl[sb].dy[h],
                      rz = rz0 + ctrl[sb].dz[h];
          // this thread's EPT points of the tile: x, y, z runs of the SoA tile
          const float *pt = reinterpret_cast<const float *>(sOff + (sb * 2 + h) * TJ) + EPT * q;
          float4 xv[EPT / 4], yv[EPT / 4], zv[EPT / 4];
#pragma unroll
          for (int v4 = 0; v4 < EPT / 4; ++v4) {
            xv[v4] = *reinterpret_cast<const float4 *>(pt + 4 * v4);
            yv[v4] = *reinterpret_cast<const float4 *>(pt + TJ + 4 * v4);
            zv[v4] = *reinterpret_cast<const float4 *>(pt + 2 * TJ + 4 * v4);
          }
          const float *xs = reinterpret_cast<const float *>(xv);
          const float *ys = reinterpret_cast<const float *>(yv);
          const float *zs = reinterpret_cast<const float *>(zv);
          float kv[EPT];
          if constexpr (F16) {
            const uint64_t rx2 = f2(rx, rx), ry2 = f2(ry, ry), rz2 = f2(rz, rz);
#pragma unroll
            for (int u = 0; u < EPT; u += 2) {
              const uint64_t e = tc_entry2_s<KID>(rx2, ry2, rz2, f2(xs[u], xs[u + 1]),
                                                  f2(ys[u], ys[u + 1]), f2(zs[u], zs[u + 1]));
              f2u(e, kv[u], kv[u + 1]);
            }
          } else {
#pragma unroll
            for (int u = 0; u < EPT; ++u) {
              kv[u] = tc_entry<KID>(rx, ry, rz, make_float4(xs[u], ys[u], zs[u], 0.f), kc, pw);
              if constexpr ((KID == H2_K_LAPLACE_IE || KID == H2_K_HELMHOLTZ_IE) && !FAR) {
                // the row's own point: the rounded offsets need not cancel exactly
                if (ctrl[sb].j0[h] + EPT * q + u == g) kv[u] = 0.f;
              }
            }
          }
          split_parts<F16, EPT>(kv, p1, p2);
        } else {   // rows outside the item or near to the tile's leaf
#pragma unroll
          for (int u = 0; u < 8; ++u) { p1[u] = 0u; p2[u] = 0u; }
        }
        // points EPT q .. EPT q + EPT - 1 of tile h: columns 32 h + 8 q .. + 7 of each part
        __syncwarp();
        tmem_st8(at + h * 32, p1);
        tmem_st8(at + 64 + h * 32, p2);
      }
      tmem_st_wait();
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(saddr(&afull[sa]));
      if (k >= 1) {
        drain(k - 1);
        if (!alive) break;
      }
    }
    if (alive && k >= 1) drain(k - 1);
    fold();
    if (alive && rowok) {
      const int64_t gr = it.row0 + r;
      const int cl = q * CPT;
      // the nugget of the row's own point, if it lies in this item's leaves
      // (near-only items cover the row's own leaf)
      bool diag = false;
      if (!FAR && KID != H2_K_POLY && in.kd.diag != 0.0) {
        const int64_t p0 = MODE == 2 ? gr : a.leaf_row[it.lb0];
        const int64_t pe = MODE == 2 ? gr + 1 : a.leaf_row[it.lb1 - 1] + a.leaf_m[it.lb1 - 1];
        diag = gr >= p0 && gr < pe;
      }
      const float dg = (float)in.kd.diag;
      float *dst = it.part < 0 ? a.y + gr + (int64_t)(it.c0 + cl) * a.ld
                               : a.partial + (int64_t)it.part * kRows * a.ncol + (int64_t)cl * kRows + r;
      const int64_t stride = it.part < 0 ? a.ld : kRows;
#pragma unroll
      for (int c = 0; c < CPT; ++c) {
        if (cl + c >= a.ncol) continue;
        float v = total(c);
        if (diag) v += dg * a.om[gr + (int64_t)(it.c0 + cl + c) * a.ld];
        dst[(int64_t)c * stride] = v;
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

template <int KID, int NCOL, int MODE, bool F16>
void launch_tc(int64_t items, const TcArgs &a, cudaStream_t s) {
  auto kern = k_ksum_tc<KID, NCOL, MODE, F16>;
  const size_t bytes = tc_smem_bytes<NCOL, F16>();
  H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  kern<<<(int)items, kThreads, bytes, s>>>(a);
  count_launch();
  H2_CHECK_LAUNCH();
}

// Per leaf (one CTA): its reference sigma * x_first as FP32 hi/lo (the
// origin for the polynomial kernel) and the scaled offsets of its points,
// zero in the padding of its last tile.
__global__ void k_tc_offsets(bool poly, int tj, int n_leaves, const int64_t *leaf_row,
                             const int32_t *leaf_m, const int32_t *leaf_inst,
                             const int64_t *leaf_tile, const double *sigma, Points64 p,
                             float4 *ref_hi, float4 *ref_lo, float4 *off) {
  const int b = blockIdx.x;
  if (b >= n_leaves) return;
  const int64_t row = leaf_row[b];
  const int m = leaf_m[b];
  const double sg = sigma[leaf_inst[b]];
  const double x0 = poly ? 0.0 : p.x[row], y0 = poly ? 0.0 : p.y[row],
               z0 = poly ? 0.0 : p.z[row];
  if (threadIdx.x == 0) {
    const double sx = x0 * sg, sy = y0 * sg, sz = z0 * sg;
    const float hx = (float)sx, hy = (float)sy, hz = (float)sz;
    ref_hi[b] = make_float4(hx, hy, hz, 0.f);
    ref_lo[b] = make_float4((float)(sx - hx), (float)(sy - hy), (float)(sz - hz), 0.f);
  }
  const int np = (m + tj - 1) / tj * tj;
  // per tile: x of its tj points, then y, then z, then tj zeros
  float *o = reinterpret_cast<float *>(off + leaf_tile[b] * tj);
  for (int u = threadIdx.x; u < np; u += blockDim.x) {
    float *t = o + (int64_t)(u / tj) * 4 * tj + u % tj;
    if (u < m) {
      const int64_t i = row + u;
      t[0] = (float)((p.x[i] - x0) * sg);
      t[tj] = (float)((p.y[i] - y0) * sg);
      t[2 * tj] = (float)((p.z[i] - z0) * sg);
    } else {
      t[0] = 0.f;
      t[tj] = 0.f;
      t[2 * tj] = 0.f;
    }
    t[3 * tj] = 0.f;
  }
}

// Omega image: per tile T and image column c (< img_nc) one 128-byte row
// per part (32 TF32 or 64 FP16 values, one per point of the tile); the
// 16-byte chunk holding points [e k, e k + e) (e = 4 or 8 values) sits at
// chunk position k ^ (c % 8).  Columns c >= nc and padding points are zero.
template <bool F16>
__global__ void k_tc_image(const float *om, int64_t ld, const int32_t *tile_leaf,
                           const int64_t *leaf_row, const int32_t *leaf_m,
                           const int64_t *leaf_tile, const int32_t *leaf_inst,
                           const int32_t *inst_c0, int nc, int img_nc, float *img_1,
                           float *img_2) {
  constexpr int TJ = TcTile<F16>::TJ;
  constexpr int E = F16 ? 8 : 4;      // values per 16-byte chunk
  const int64_t T = blockIdx.x;
  const int b = tile_leaf[T];
  const int u0 = (int)(T - leaf_tile[b]) * TJ;
  const int mv = leaf_m[b] - u0;
  const int64_t row = leaf_row[b] + u0;
  const int c0 = inst_c0[leaf_inst[b]];
  for (int q = threadIdx.x; q < img_nc * TJ; q += blockDim.x) {
    const int c = q / TJ, k = q % TJ;
    const float v = (c < nc && k < mv) ? om[row + k + (int64_t)(c0 + c) * ld] : 0.f;
    const int64_t dst = (T * img_nc + c) * TJ + (((k / E) ^ (c & 7)) * E + k % E);
    if constexpr (F16) {
      const __half h = __float2half_rn(v);
      const __half r = __float2half_rn(__half2float(h) - v);   // residual, sign flipped
      reinterpret_cast<__half *>(img_1)[dst] = h;
      reinterpret_cast<__half *>(img_2)[dst] = r;
    } else {
      const float hv = tf32_rna(v);
      img_1[dst] = hv;
      img_2[dst] = tf32_rna(v - hv);
    }
  }
}

__global__ void k_max_abs(const float *x, int64_t ld, int64_t n, int c0, int c1,
                          unsigned int *out) {
  float m = 0.f;
  for (int c = c0; c < c1; ++c)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      m = fmaxf(m, fabsf(x[i + (int64_t)c * ld]));
  // non-negative floats order like their bit patterns; NaN compares above all
  atomicMax(out, __float_as_uint(m != m ? INFINITY : m));
}
}  // namespace

int tc_chunk_ncol(int w) { return w <= 16 ? 16 : (w <= 32 ? 32 : (w <= 64 ? 64 : 80)); }

bool tc_f16_kernel(int kid) {
  return kid == H2_K_EXP || kid == H2_K_MATERN32 || kid == H2_K_GAUSS;
}

float tc_max_abs(const float *x, int64_t ld, int64_t n, int c0, int c1, cudaStream_t s) {
  if (n == 0 || c1 <= c0) return 0.f;
  DBuf<unsigned int> m;
  m.alloc_zero(1, s);
  const int blocks = std::min<int64_t>(ceil_div(n, 256), 1024);
  k_max_abs<<<blocks, 256, 0, s>>>(x, ld, n, c0, c1, m.p);
  count_launch();
  H2_CHECK_LAUNCH();
  const unsigned int bits = to_host(m.p, 1, s)[0];
  float v;
  std::memcpy(&v, &bits, sizeof(v));
  return v;
}

void tc_layout_build(int kid, bool f16, const std::vector<int64_t> &leaf_row,
                     const std::vector<int32_t> &leaf_m, const std::vector<int32_t> &leaf_inst,
                     const std::vector<KernelDesc> &inst_kd, const int64_t *d_leaf_row,
                     const int32_t *d_leaf_m, Points64 p64, TcLayout &out, cudaStream_t s) {
  const int tj = f16 ? TcTile<true>::TJ : TcTile<false>::TJ;
  const int nl = (int)leaf_row.size();
  std::vector<int64_t> lt(nl);
  std::vector<int32_t> tl;
  int64_t nt = 0;
  for (int b = 0; b < nl; ++b) {
    lt[b] = nt;
    const int tiles = (leaf_m[b] + tj - 1) / tj;
    for (int u = 0; u < tiles; ++u) tl.push_back(b);
    nt += tiles;
  }
  H2_REQUIRE(nt < (1ll << 31), "too many sketch tiles");
  std::vector<double> sg(inst_kd.size());
  for (size_t i = 0; i < inst_kd.size(); ++i) sg[i] = tc_sigma(inst_kd[i]);
  out.f16 = f16;
  out.tj = tj;
  out.n_tiles = nt;
  to_device(out.leaf_tile, lt, s);
  to_device(out.tile_leaf, tl, s);
  to_device(out.leaf_inst, leaf_inst, s);
  to_device(out.sigma, sg, s);
  out.ref_hi.alloc(nl);
  out.ref_lo.alloc(nl);
  out.off.alloc((size_t)nt * tj);
  if (nl == 0) return;
  k_tc_offsets<<<nl, 128, 0, s>>>(kid == H2_K_POLY, tj, nl, d_leaf_row, d_leaf_m,
                                  out.leaf_inst.p, out.leaf_tile.p, out.sigma.p, p64,
                                  out.ref_hi.p, out.ref_lo.p, out.off.p);
  count_launch();
  H2_CHECK_LAUNCH();
}

void tc_omega_image(const TcLayout &L, const int64_t *d_leaf_row, const int32_t *d_leaf_m,
                    const float *om, int64_t ld, const int32_t *d_inst_c0, int nc, int img_nc,
                    float *img_hi, float *img_lo, cudaStream_t s) {
  if (L.n_tiles == 0 || img_nc == 0) return;
  auto kern = L.f16 ? k_tc_image<true> : k_tc_image<false>;
  kern<<<(int)L.n_tiles, 256, 0, s>>>(om, ld, L.tile_leaf.p, d_leaf_row, d_leaf_m,
                                      L.leaf_tile.p, L.leaf_inst.p, d_inst_c0, nc, img_nc,
                                      img_hi, img_lo);
  count_launch();
  H2_CHECK_LAUNCH();
}

void launch_ksum_tc(int kid, int ncol_tmpl, int mode, bool f16, int64_t items, const TcArgs &a,
                    cudaStream_t s) {
  dispatch_kernel(kid, [&](auto K) {
    constexpr int KID = decltype(K)::value;
    auto go = [&](auto M, auto H) {
      constexpr int MODE = decltype(M)::value;
      constexpr bool F16 = decltype(H)::value;
      switch (ncol_tmpl) {
        case 80: launch_tc<KID, 80, MODE, F16>(items, a, s); break;
        case 64: launch_tc<KID, 64, MODE, F16>(items, a, s); break;
        case 32: launch_tc<KID, 32, MODE, F16>(items, a, s); break;
        case 16: launch_tc<KID, 16, MODE, F16>(items, a, s); break;
        default: throw Error{H2_ERR_ARG, "tensor-core sketch takes 16, 32, 64 or 80 columns"};
      }
    };
    auto pick = [&](auto M) {
      if constexpr (KID == H2_K_EXP || KID == H2_K_MATERN32 || KID == H2_K_GAUSS) {
        if (f16) go(M, std::true_type{});
        else go(M, std::false_type{});
      } else {
        H2_REQUIRE(!f16, "FP16 sketch parts need entries bounded by 1");
        go(M, std::false_type{});
      }
    };
    switch (mode) {
      case 0: pick(std::integral_constant<int, 0>{}); break;
      case 1: pick(std::integral_constant<int, 1>{}); break;
      case 2: pick(std::integral_constant<int, 2>{}); break;
      default: throw Error{H2_ERR_ARG, "unknown tensor-core sketch mode"};
    }
  });
}

}  // namespace h2
