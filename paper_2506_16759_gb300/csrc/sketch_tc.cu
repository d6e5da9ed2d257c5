// Fused kernel summation Y = K Omega on the 5th-generation tensor cores.
//
// The sketch of Algorithm 1 is a dense contraction over the point index j
// whose left operand K(x_i, x_j) is generated on the fly.  Here each CTA owns
// 128 rows (TMEM lanes) and NCOL sample columns; for every 32-point tile:
//   * thread i evaluates its row's 32 entries in FP32 (split hi/lo
//     coordinates), splits each into TF32 parts hi = rna(x), lo = rna(x - hi)
//     and stores both parts into two 128-byte-swizzled K-major tiles (A);
//   * the Omega tile is split the same way into two K-major tiles (B);
//   * one thread issues the three TF32 products hi*hi, hi*lo, lo*hi for the
//     four K=8 steps of the tile (tcgen05.mma, FP32 accumulation in TMEM) and
//     commits them to an mbarrier;
//   * every kDrain tiles the 128 x NCOL accumulator is read back with
//     tcgen05.ld and added to per-thread FP32 sums with Kahan compensation,
//     and the next product restarts the accumulator.
// The split keeps ~22 bits of every product, the TMEM sums stay short, and
// the running sums are compensated, so the result carries a few 1e-7 of
// relative rounding like the SIMT kernel.
// Far-only mode (two leaves per CTA) skips point leaves that are near to
// both leaves and masks, per row, those near to that row's leaf.
// Every mbarrier wait is bounded; a timeout raises the error flag.
#include <cstdint>

#include "h2_ops.h"
#include "h2_types.h"

namespace h2 {
namespace {

constexpr int kRows = 128;   // MMA M, TMEM lanes
constexpr int kTJ = 32;      // points per tile (4 K-steps of 8)
#ifndef H2_TC_DRAIN
#define H2_TC_DRAIN 2
#endif
constexpr int kDrain = H2_TC_DRAIN;   // tiles accumulated in TMEM before a drain
constexpr int kWaitLimit = 1 << 24;

__device__ __forceinline__ uint32_t saddr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups of
// 128-byte rows 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;              // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= (uint64_t)1 << 46;              // descriptor version
  d |= (uint64_t)2 << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// Waits for the phase with the given parity to complete; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (int it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <int NCOL>
__device__ __forceinline__ void tmem_ld(uint32_t taddr, float *v);

template <>
__device__ __forceinline__ void tmem_ld<32>(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

template <>
__device__ __forceinline__ void tmem_ld<16>(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

// Byte offset of element (row, k) in a K-major 128-byte-swizzled tile whose
// rows hold 32 FP32 values.
__device__ __forceinline__ uint32_t sw128_off(int row, int k) {
  return (uint32_t)row * 128u + ((uint32_t)((k >> 2) ^ (row & 7)) << 4) + (uint32_t)(k & 3) * 4u;
}

template <int KID, int NCOL, bool FAR>
__global__ void __launch_bounds__(kRows) k_ksum_tc(KsumArgs32 a, int tile_rows) {
  extern __shared__ unsigned char smem_dyn[];
  // 1024-byte aligned tiles: A hi/lo (128 x 32 FP32 each), B hi/lo (NCOL x 32)
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  unsigned char *Ahi = base;
  unsigned char *Alo = Ahi + kRows * 128;
  unsigned char *Bhi = Alo + kRows * 128;
  unsigned char *Blo = Bhi + NCOL * 128;
  float4 *sh = reinterpret_cast<float4 *>(Blo + NCOL * 128);
  float4 *sl = sh + kTJ;
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;

  const KsumItem it = a.items[blockIdx.x];
  const InstDev in = a.inst[it.inst];
  const float scale = (float)in.kd.scale;
  const float diag = (float)in.kd.diag;
  const int pw = in.kd.pw;
  const int t = threadIdx.x, warp = t >> 5;
  const uint32_t mb = saddr(&mbar);

  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(mb));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;\n" ::"r"(
        saddr(&tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_base;

  const int64_t g = it.row0 + (t < it.rows ? t : 0);
  const float xh = a.pts.xh[g], yh = a.pts.yh[g], zh = a.pts.zh[g];
  const float xl = a.pts.xl[g], yl = a.pts.yl[g], zl = a.pts.zl[g];
  float acc[NCOL], cmp[NCOL];
#pragma unroll
  for (int c = 0; c < NCOL; ++c) { acc[c] = 0.f; cmp[c] = 0.f; }

  constexpr uint32_t IDESC = idesc_tf32(kRows, NCOL);
  int ntile = 0;   // tiles issued
  int since = 0;   // tiles accumulated in TMEM since the last drain
  bool ok = true;

  auto drain = [&]() {
    if (!mbar_wait(mb, (ntile - 1) & 1)) ok = false;
    fence_after();
    float v[NCOL];
    tmem_ld<NCOL>(tmem + ((uint32_t)(warp * 32) << 16), v);
#pragma unroll
    for (int c = 0; c < NCOL; ++c) {
      float y = v[c] - cmp[c];
      float s = acc[c] + y;
      cmp[c] = (s - acc[c]) - y;
      acc[c] = s;
    }
    since = 0;
    fence_before();
    __syncthreads();
  };

  auto tile = [&](int64_t j0, int nj, float mask) {
    // the previous tile's products must be done before its operands are overwritten
    if (ntile > 0 && !mbar_wait(mb, (ntile - 1) & 1)) ok = false;
    if (t < kTJ) {
      int64_t gj = j0 + (t < nj ? t : 0);
      sh[t] = make_float4(a.pts.xh[gj], a.pts.yh[gj], a.pts.zh[gj], 0.f);
      sl[t] = make_float4(a.pts.xl[gj], a.pts.yl[gj], a.pts.zl[gj], 0.f);
    }
    for (int q = t; q < NCOL * kTJ; q += kRows) {
      const int n = q / kTJ, k = q % kTJ;
      const float x = k < nj ? a.om[j0 + k + (int64_t)(it.c0 + n) * a.ld] : 0.f;
      const float hi = tf32_rna(x);
      const float lo = tf32_rna(x - hi);
      const uint32_t off = sw128_off(n, k);
      *reinterpret_cast<float *>(Bhi + off) = hi;
      *reinterpret_cast<float *>(Blo + off) = lo;
    }
    __syncthreads();
    const float m = t < it.rows ? mask : 0.f;
#pragma unroll
    for (int k4 = 0; k4 < kTJ / 4; ++k4) {
      float h[4], l[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = 4 * k4 + u;
        const float4 ph = sh[k], pl = sl[k];
        float kv = kval<KID, float>(geom32<KID>(xh, yh, zh, xl, yl, zl, ph.x, ph.y, ph.z, pl.x,
                                                pl.y, pl.z),
                                    scale, pw);
        kv = k < nj ? kv * m : 0.f;
        h[u] = tf32_rna(kv);
        l[u] = tf32_rna(kv - h[u]);
      }
      const uint32_t off = (uint32_t)t * 128u + ((uint32_t)(k4 ^ (t & 7)) << 4);
      *reinterpret_cast<float4 *>(Ahi + off) = make_float4(h[0], h[1], h[2], h[3]);
      *reinterpret_cast<float4 *>(Alo + off) = make_float4(l[0], l[1], l[2], l[3]);
    }
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (t == 0) {
      fence_after();
      const uint32_t ah = saddr(Ahi), al = saddr(Alo), bh = saddr(Bhi), bl = saddr(Blo);
#pragma unroll
      for (int ks = 0; ks < kTJ / 8; ++ks) {
        const uint32_t koff = ks * 32;   // 8 TF32 values
        const uint64_t dah = desc_sw128(ah + koff), dal = desc_sw128(al + koff);
        const uint64_t dbh = desc_sw128(bh + koff), dbl = desc_sw128(bl + koff);
        mma_tf32(tmem, dah, dbh, IDESC, (since > 0 || ks > 0) ? 1u : 0u);
        mma_tf32(tmem, dah, dbl, IDESC, 1u);
        mma_tf32(tmem, dal, dbh, IDESC, 1u);
#ifdef H2_TC_LOLO
        mma_tf32(tmem, dal, dbl, IDESC, 1u);
#endif
      }
      mma_commit(mb);
    }
    ++ntile;
    ++since;
    if (since == kDrain) drain();
  };

  if (!FAR) {
    for (int64_t j = it.j0; j < it.j1; j += kTJ)
      tile(j, (int)(it.j1 - j < kTJ ? it.j1 - j : kTJ), 1.f);
  } else {
    const int t1 = it.task;
    const int m1 = a.far.leaf_m[t1];
    const bool two = it.rows > m1;
    int64_t p1 = a.far.near_ptr[t1], e1 = a.far.near_ptr[t1 + 1];
    int64_t p2 = two ? a.far.near_ptr[t1 + 1] : 0, e2 = two ? a.far.near_ptr[t1 + 2] : 0;
    const bool second = t >= m1;
    for (int b = it.lb0; b < it.lb1; ++b) {
      while (p1 < e1 && a.far.near_idx[p1] < b) ++p1;
      const bool n1 = p1 < e1 && a.far.near_idx[p1] == b;
      bool n2 = true;
      if (two) {
        while (p2 < e2 && a.far.near_idx[p2] < b) ++p2;
        n2 = p2 < e2 && a.far.near_idx[p2] == b;
      }
      if (n1 && n2) continue;
      const float mask = (second ? n2 : n1) ? 0.f : 1.f;
      const int64_t r0 = a.far.leaf_row[b];
      const int nb = a.far.leaf_m[b];
      for (int q = 0; q < nb; q += kTJ) tile(r0 + q, nb - q < kTJ ? nb - q : kTJ, mask);
    }
  }
  if (since > 0) drain();
  if (ntile > 0 && !mbar_wait(mb, (ntile - 1) & 1)) ok = false;
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;\n" ::"r"(tmem));
  if (!ok && t == 0) atomicExch(a.err, 1);

  if (t >= it.rows) return;
  const int64_t gr = it.row0 + t;
  if (!FAR && KID != H2_K_POLY && gr >= it.j0 && gr < it.j1 && diag != 0.f) {
#pragma unroll
    for (int c = 0; c < NCOL; ++c) acc[c] += diag * a.om[gr + (int64_t)(it.c0 + c) * a.ld];
  }
  if (it.part < 0) {
#pragma unroll
    for (int c = 0; c < NCOL; ++c) a.y[gr + (int64_t)(it.c0 + c) * a.ld] = acc[c];
  } else {
    float *dst = a.partial + (int64_t)it.part * tile_rows * NCOL;
#pragma unroll
    for (int c = 0; c < NCOL; ++c) dst[c * tile_rows + t] = acc[c];
  }
}

template <int NCOL>
constexpr size_t tc_smem_bytes() {
  return 1024 + 2 * kRows * 128 + 2 * NCOL * 128 + 2 * kTJ * sizeof(float4);
}

template <int KID, int NCOL, bool FAR>
void launch_tc(const KsumPlan &p, const KsumArgs32 &a, cudaStream_t s) {
  auto kern = k_ksum_tc<KID, NCOL, FAR>;
  const size_t bytes = tc_smem_bytes<NCOL>();
  H2_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  kern<<<(int)p.items.size(), kRows, bytes, s>>>(a, p.tile_rows);
  count_launch();
  H2_CHECK_LAUNCH();
}

}  // namespace

bool tc_sketch_supported(int ncols) { return ncols == 16 || ncols == 32; }

void launch_ksum_tc(int kid, const KsumPlan &plan, const KsumArgs32 &a, bool far,
                    cudaStream_t s) {
  dispatch_kernel(kid, [&](auto K) {
    constexpr int KID = decltype(K)::value;
    if (plan.dc == 32) {
      if (far) launch_tc<KID, 32, true>(plan, a, s);
      else launch_tc<KID, 32, false>(plan, a, s);
    } else if (plan.dc == 16) {
      if (far) launch_tc<KID, 16, true>(plan, a, s);
      else launch_tc<KID, 16, false>(plan, a, s);
    } else {
      throw Error{H2_ERR_ARG, "tensor-core sketch takes 16 or 32 columns"};
    }
  });
}

}  // namespace h2
