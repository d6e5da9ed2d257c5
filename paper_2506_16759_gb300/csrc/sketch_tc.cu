// Fused kernel summation Y = K Omega on the 5th-generation tensor cores.
//
// The sketch of Algorithm 1 is a dense contraction over the point index j
// whose left operand K(x_i, x_j) is generated on the fly.  Here each CTA owns
// 128 rows (TMEM lanes) and NCOL sample columns; for every 32-point tile:
//   * the entries are evaluated in FP32 from coordinates relative to the
//     tile's first row (offsets formed in FP64), split into TF32 parts
//     hi = rna(x), lo = x - hi, and stored into two 128-byte-swizzled
//     K-major tiles (A);
//   * the Omega tile, split the same way once when its columns are drawn,
//     is copied into two K-major tiles (B);
//   * one thread issues the three TF32 products hi*hi, hi*lo, lo*hi for the
//     four K=8 steps of the tile (tcgen05.mma, FP32 accumulation in TMEM) and
//     commits them to the tile's mbarrier;
//   * each tile's 128 x NCOL accumulator is read back with tcgen05.ld and
//     added to per-thread FP32 sums with Kahan compensation.
// Accumulating many products in TMEM loses precision (measured: 3.8e-6
// relative after 192 products, 3.9e-7 when every 12-product tile is read
// back), so every tile gets a fresh accumulator; operands and accumulators
// are double-buffered so the products overlap the next tile's evaluation.
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

template <>
__device__ __forceinline__ void tmem_ld<8>(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int c = 0; c < 8; ++c) v[c] = __uint_as_float(r[c]);
}

// Byte offset of element (row, k) in a K-major 128-byte-swizzled tile whose
// rows hold 32 FP32 values.
__device__ __forceinline__ uint32_t sw128_off(int row, int k) {
  return (uint32_t)row * 128u + ((uint32_t)((k >> 2) ^ (row & 7)) << 4) + (uint32_t)(k & 3) * 4u;
}

// Entry from coordinates relative to a reference point of the row tile:
// offsets are formed in FP64 and rounded once to FP32, so a distance carries
// an absolute error of a few 2^-24 of the offsets (well below the TF32 split
// for the far pairs summed here).  The root is taken as r2 * rsqrt(max(r2, tiny)).
template <int KID>
__device__ __forceinline__ float kval_rel(float dx, float dy, float dz, float scale, int pw,
                                          float dot) {
  if constexpr (KID == H2_K_POLY) {
    return kval<KID, float>(dot, scale, pw);
  } else {
    const float r2 = dx * dx + dy * dy + dz * dz;
    if constexpr (KID == H2_K_GAUSS) {
      return __expf(-r2 * scale);
    } else if constexpr (KID == H2_K_LAPLACE_IE) {
      return r2 > 0.f ? rsqrtf(r2) * scale : 0.f;
    } else {
      const float r = r2 * rsqrtf(fmaxf(r2, 1e-30f));
      if constexpr (KID == H2_K_EXP) {
        return __expf(-r * scale);
      } else {
        const float a2 = r * scale;
        return (1.f + a2) * __expf(-a2);
      }
    }
  }
}

// Thread groups per CTA: each group of 128 threads covers all rows and a
// 1/G share of every tile's points (evaluation) and of the columns (drain).
template <int NCOL>
struct TcShape {
  static constexpr int G = NCOL >= 64 ? 4 : 2;
  static constexpr int threads = kRows * G;
  static constexpr int HC = NCOL / G;       // accumulator columns per thread
  static constexpr int EPT = kTJ / G;       // points evaluated per thread per tile
};

// One 32-point tile of the j loop: its first point, its size, and whether its
// leaf is near to the first / second leaf of the row tile (far-only mode).
struct TileDesc {
  int64_t j0;
  int nj;
  bool near1, near2;
  bool valid;
};

// Thread t owns row r = t % 128 and group h = t / 128: it evaluates points
// [h*EPT, (h+1)*EPT) of every tile for its row, and reads back accumulator
// columns [h*HC, (h+1)*HC) of its row.  Per tile: the next tile's Omega parts
// and coordinates are loaded into registers first; the previous tile's
// products are awaited and its accumulator drained; the operands are stored;
// one barrier; one thread issues the products.  Two TMEM accumulators
// alternate, so a drain never waits for the products in flight.
template <int KID, int NCOL, bool FAR>
__global__ void __launch_bounds__(TcShape<NCOL>::threads) k_ksum_tc(KsumArgs32 a, int tile_rows) {
  constexpr int kThreads = TcShape<NCOL>::threads;
  constexpr int HC = TcShape<NCOL>::HC;
  constexpr int EPT = TcShape<NCOL>::EPT;
  constexpr int BPT = NCOL * kTJ / kThreads;   // Omega elements staged per thread
  constexpr uint32_t A_BYTES = kRows * 128, B_BYTES = NCOL * 128;
  extern __shared__ unsigned char smem_dyn[];
  unsigned char *base = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
  unsigned char *Ahi = base;
  unsigned char *Alo = Ahi + A_BYTES;
  unsigned char *Bhi = Alo + A_BYTES;
  unsigned char *Blo = Bhi + B_BYTES;
  float4 *crd = reinterpret_cast<float4 *>(Blo + B_BYTES);   // [2 slots][hi 32, lo 32]
  __shared__ uint64_t mbar[2];
  __shared__ uint32_t tmem_base;

  const KsumItem it = a.items[blockIdx.x];
  const InstDev in = a.inst[it.inst];
  const float scale = (float)in.kd.scale;
  const float diag = (float)in.kd.diag;
  const int pw = in.kd.pw;
  const int t = threadIdx.x, warp = t >> 5;
  const int r = t & (kRows - 1), h = t >> 7;

  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(saddr(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  constexpr uint32_t TCOLS = 2 * NCOL < 32 ? 32 : 2 * NCOL;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     saddr(&tmem_base)),
                 "n"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }

  // ---- tile sequence (identical in every thread)
  int64_t aj = it.j0;                      // all-points cursor
  int fb = it.lb0, fq = 0;                 // far-only cursor: leaf, offset in leaf
  int64_t p1 = 0, e1 = 0, p2 = 0, e2 = 0;
  bool two = false;
  int m1 = 0;
  if (FAR) {
    const int t1 = it.task;
    m1 = a.far.leaf_m[t1];
    two = it.rows > m1;
    p1 = a.far.near_ptr[t1];
    e1 = a.far.near_ptr[t1 + 1];
    if (two) { p2 = a.far.near_ptr[t1 + 1]; e2 = a.far.near_ptr[t1 + 2]; }
  }
  bool cn1 = false, cn2 = false;           // near flags of the far cursor's leaf
  auto next = [&]() -> TileDesc {
    TileDesc d{0, 0, false, false, false};
    if constexpr (!FAR) {
      if (aj < it.j1) {
        d.j0 = aj;
        d.nj = (int)(it.j1 - aj < kTJ ? it.j1 - aj : kTJ);
        d.valid = true;
        aj += kTJ;
      }
      return d;
    }
    while (FAR && fb < it.lb1) {
      if (fq == 0) {
        while (p1 < e1 && a.far.near_idx[p1] < fb) ++p1;
        cn1 = p1 < e1 && a.far.near_idx[p1] == fb;
        cn2 = true;
        if (two) {
          while (p2 < e2 && a.far.near_idx[p2] < fb) ++p2;
          cn2 = p2 < e2 && a.far.near_idx[p2] == fb;
        }
        if (cn1 && cn2) { ++fb; continue; }
      }
      const int nb = a.far.leaf_m[fb];
      d.j0 = a.far.leaf_row[fb] + fq;
      d.nj = nb - fq < kTJ ? nb - fq : kTJ;
      d.near1 = cn1;
      d.near2 = cn2;
      d.valid = true;
      fq += kTJ;
      if (fq >= nb) { fq = 0; ++fb; }
      return d;
    }
    return d;
  };

  // ---- prefetch of a tile's Omega parts and coordinates into registers
  float bh[BPT], bl[BPT];
  float c6[3];
  // reference point: the tile's first row (the origin for the polynomial kernel)
  const double cx = KID == H2_K_POLY ? 0.0 : a.p64.x[it.row0];
  const double cy = KID == H2_K_POLY ? 0.0 : a.p64.y[it.row0];
  const double cz = KID == H2_K_POLY ? 0.0 : a.p64.z[it.row0];
  auto fetch = [&](const TileDesc &d) {
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      const int q = t + u * kThreads;
      const int n = q / kTJ, kk = q % kTJ;
      const int64_t src = d.j0 + kk + (int64_t)(it.c0 + n) * a.ld;
      const bool ok2 = d.valid && kk < d.nj;
      bh[u] = ok2 ? a.om_hi[src] : 0.f;
      bl[u] = ok2 ? a.om_lo[src] : 0.f;
    }
    if (t < kTJ) {
      const int64_t gj = d.j0 + (d.valid && t < d.nj ? t : 0);
      c6[0] = (float)(a.p64.x[gj] - cx);
      c6[1] = (float)(a.p64.y[gj] - cy);
      c6[2] = (float)(a.p64.z[gj] - cz);
    }
  };
  auto store_coords = [&](int slot) {
    if (t < kTJ) crd[slot * kTJ + t] = make_float4(c6[0], c6[1], c6[2], 0.f);
  };

  const int64_t g = it.row0 + (r < it.rows ? r : 0);
  const float xr = (float)(a.p64.x[g] - cx), yr = (float)(a.p64.y[g] - cy),
              zr = (float)(a.p64.z[g] - cz);
  const bool second = FAR && r >= m1;
  float acc[HC], cmp[HC];
#pragma unroll
  for (int c = 0; c < HC; ++c) { acc[c] = 0.f; cmp[c] = 0.f; }
  constexpr uint32_t IDESC = idesc_tf32(kRows, NCOL);
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  bool ok = true;

  auto drain = [&](int k) {
    if (!mbar_wait(saddr(&mbar[k & 1]), (uint32_t)((k >> 1) & 1))) ok = false;
    fence_after();
    float v[HC];
    tmem_ld<HC>(tmem_base + lane_base + (uint32_t)((k & 1) * NCOL + h * HC), v);
#pragma unroll
    for (int c = 0; c < HC; ++c) {
      float y = v[c] - cmp[c];
      float s2 = acc[c] + y;
      cmp[c] = (s2 - acc[c]) - y;
      acc[c] = s2;
    }
  };

  TileDesc cur = next();
  fetch(cur);
  store_coords(0);
  float cbh[BPT], cbl[BPT];
#pragma unroll
  for (int u = 0; u < BPT; ++u) { cbh[u] = bh[u]; cbl[u] = bl[u]; }
  fence_before();
  __syncthreads();
  fence_after();
  int k = 0;
  while (cur.valid) {
    const TileDesc nxt = next();
    fetch(nxt);                          // loads in flight during this tile
    if (k > 0) drain(k - 1);             // products of tile k-1 done: operands free
#pragma unroll
    for (int u = 0; u < BPT; ++u) {
      const int q = t + u * kThreads;
      const uint32_t off = sw128_off(q / kTJ, q % kTJ);
      *reinterpret_cast<float *>(Bhi + off) = cbh[u];
      *reinterpret_cast<float *>(Blo + off) = cbl[u];
    }
    const float4 *ch = crd + (k & 1) * kTJ;
    const float m = r < it.rows ? ((FAR && (second ? cur.near2 : cur.near1)) ? 0.f : 1.f) : 0.f;
    const bool full = cur.nj == kTJ;
#pragma unroll
    for (int q = 0; q < EPT / 4; ++q) {
      const int k4 = (EPT / 4) * h + q;
      float hv[4], lv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int kk = 4 * k4 + u;
        const float4 p = ch[kk];
        float kv = kval_rel<KID>(xr - p.x, yr - p.y, zr - p.z, scale, pw,
                                 xr * p.x + yr * p.y + zr * p.z);
        kv = (full || kk < cur.nj) ? kv * m : 0.f;
        hv[u] = tf32_rna(kv);
        lv[u] = kv - hv[u];   // the tensor core keeps its leading TF32 bits
      }
      const uint32_t off = (uint32_t)r * 128u + ((uint32_t)(k4 ^ (r & 7)) << 4);
      *reinterpret_cast<float4 *>(Ahi + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
      *reinterpret_cast<float4 *>(Alo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
    }
    if (nxt.valid) store_coords((k + 1) & 1);
    fence_async_smem();
    fence_before();
    __syncthreads();
    if (t == 0) {
      fence_after();
      const uint32_t ah = saddr(Ahi), al = saddr(Alo), bhs = saddr(Bhi), bls = saddr(Blo);
      const uint32_t d = tmem_base + (uint32_t)((k & 1) * NCOL);
#pragma unroll
      for (int ks = 0; ks < kTJ / 8; ++ks) {
        const uint32_t koff = ks * 32;
        const uint64_t dah = desc_sw128(ah + koff), dal = desc_sw128(al + koff);
        const uint64_t dbh = desc_sw128(bhs + koff), dbl = desc_sw128(bls + koff);
        mma_tf32(d, dah, dbh, IDESC, ks > 0 ? 1u : 0u);
        mma_tf32(d, dah, dbl, IDESC, 1u);
        mma_tf32(d, dal, dbh, IDESC, 1u);
      }
      mma_commit(saddr(&mbar[k & 1]));
    }
#pragma unroll
    for (int u = 0; u < BPT; ++u) { cbh[u] = bh[u]; cbl[u] = bl[u]; }
    cur = nxt;
    ++k;
  }
  if (k > 0) drain(k - 1);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem_base),
                 "n"(TCOLS));
  if (!ok && t == 0) atomicExch(a.err, 1);

  if (r >= it.rows) return;
  const int64_t gr = it.row0 + r;
  const int c0 = it.c0 + h * HC;
  if (!FAR && KID != H2_K_POLY && gr >= it.j0 && gr < it.j1 && diag != 0.f) {
#pragma unroll
    for (int c = 0; c < HC; ++c) acc[c] += diag * a.om[gr + (int64_t)(c0 + c) * a.ld];
  }
  if (it.part < 0) {
#pragma unroll
    for (int c = 0; c < HC; ++c) a.y[gr + (int64_t)(c0 + c) * a.ld] = acc[c];
  } else {
    float *dst = a.partial + (int64_t)it.part * tile_rows * NCOL;
#pragma unroll
    for (int c = 0; c < HC; ++c) dst[(h * HC + c) * tile_rows + r] = acc[c];
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
  kern<<<(int)p.items.size(), TcShape<NCOL>::threads, bytes, s>>>(a, p.tile_rows);
  count_launch();
  H2_CHECK_LAUNCH();
}

__global__ void k_split_tf32(const float *x, int64_t ld, int64_t row0, int64_t n, int c0, int c1,
                             float *hi, float *lo) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int c = c0; c < c1; ++c) {
    const int64_t q = row0 + i + c * ld;
    const float v = x[q];
    const float hv = tf32_rna(v);
    hi[q] = hv;
    lo[q] = tf32_rna(v - hv);
  }
}

}  // namespace

bool tc_sketch_supported(int ncols) { return ncols == 16 || ncols == 32 || ncols == 64; }

void split_tf32(const float *x, int64_t ld, int64_t row0, int64_t n, int c0, int c1, float *hi,
                float *lo, cudaStream_t s) {
  if (n == 0 || c1 <= c0) return;
  k_split_tf32<<<ceil_div(n, 256), 256, 0, s>>>(x, ld, row0, n, c0, c1, hi, lo);
  count_launch();
  H2_CHECK_LAUNCH();
}

void launch_ksum_tc(int kid, const KsumPlan &plan, const KsumArgs32 &a, bool far,
                    cudaStream_t s) {
  dispatch_kernel(kid, [&](auto K) {
    constexpr int KID = decltype(K)::value;
    if (plan.dc == 64) {
      if (far) launch_tc<KID, 64, true>(plan, a, s);
      else launch_tc<KID, 64, false>(plan, a, s);
    } else if (plan.dc == 32) {
      if (far) launch_tc<KID, 32, true>(plan, a, s);
      else launch_tc<KID, 32, false>(plan, a, s);
    } else if (plan.dc == 16) {
      if (far) launch_tc<KID, 16, true>(plan, a, s);
      else launch_tc<KID, 16, false>(plan, a, s);
    } else {
      throw Error{H2_ERR_ARG, "tensor-core sketch takes 16, 32 or 64 columns"};
    }
  });
}

}  // namespace h2
