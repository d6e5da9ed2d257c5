// Cluster tree (KD median bisection) and dual tree traversal, Sec. II-A.
//
// Every comparison that decides the tree or the block partition is taken in
// FP64 with explicitly rounded operations (no contraction), in the same order
// as the plain definition: extent = hi - lo, D(s) = sqrt(sum_k e_k^2),
// Dist(s,t) = sqrt(sum_k max(0, lo_t - hi_s, lo_s - hi_t)^2),
// adm <=> Dist > 0 and 0.5*(D(s)+D(t)) <= eta*Dist.
#include <algorithm>

#include "h2_types.h"

namespace h2 {
namespace {

constexpr int kSortTile = 2048;  // elements sorted in shared memory per CTA

struct SortItem {
  unsigned long long key;
  unsigned int idx;
  unsigned int pad;
};

__device__ __forceinline__ bool item_less(const SortItem &a, const SortItem &b) {
  return a.key < b.key || (a.key == b.key && a.idx < b.idx);
}

// Order-preserving map of a double to an unsigned key; -0.0 is folded into
// +0.0 first so that equal coordinates tie and the point index decides.
__device__ __forceinline__ unsigned long long order_key(double v) {
  v = __dadd_rn(v, 0.0);
  unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void k_check_points(const double *pts, int64_t n, int dim, int *bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n * dim) return;
  if (!isfinite(pts[i])) atomicExch(bad, 1);
}

__global__ void k_split_coords(const double *pts, int64_t n, int dim, double *x, double *y,
                               double *z) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = pts[i * dim];
  y[i] = dim > 1 ? pts[i * dim + 1] : 0.0;
  z[i] = dim > 2 ? pts[i * dim + 2] : 0.0;
}

__global__ void k_iota(int32_t *p, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

// Box of a node from its coordinate minima a and maxima c; the extent
// argmax (lowest dimension on ties) gives its split dimension.
__device__ void box_finish(int node, const double *a, const double *c, double *lo, double *hi,
                           int n_nodes_total, int *split_dim) {
  double ext[3];
  for (int k = 0; k < 3; ++k) {
    lo[k * n_nodes_total + node] = a[k];
    hi[k * n_nodes_total + node] = c[k];
    ext[k] = __dsub_rn(c[k], a[k]);
  }
  int s = 0;
  for (int k = 1; k < 3; ++k)
    if (ext[k] > ext[s]) s = k;
  split_dim[node] = s;
}

// Tight box of each node of one depth over its points (in the current
// order `cur`).  CTA (node, part) takes the part-th of gridDim.y slices of
// the node's points; with one slice it writes the box, else its partial
// minima and maxima go to part[] for k_node_boxes_final (the top levels have
// too few nodes to fill the device with one CTA each).
__global__ void k_node_boxes(const double *__restrict__ x, const double *__restrict__ y,
                             const double *__restrict__ z, const int32_t *__restrict__ cur,
                             const int64_t *__restrict__ begin, const int64_t *__restrict__ end,
                             int first_node, double *lo, double *hi, int n_nodes_total,
                             int *split_dim, double *part) {
  int node = first_node + blockIdx.x;
  const int nsplit = gridDim.y;
  int64_t b = begin[node], e = end[node];
  if (nsplit > 1) {
    const int64_t chunk = (e - b + nsplit - 1) / nsplit;
    const int64_t pb = b + blockIdx.y * chunk;
    e = pb + chunk < e ? pb + chunk : e;
    b = pb;
  }
  double mn[3] = {INFINITY, INFINITY, INFINITY};
  double mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t p = b + threadIdx.x; p < e; p += blockDim.x) {
    int32_t q = cur[p];
    double v[3] = {x[q], y[q], z[q]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      mn[k] = fmin(mn[k], v[k]);
      mx[k] = fmax(mx[k], v[k]);
    }
  }
  __shared__ double smn[3][32], smx[3][32];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[k] = fmin(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
      mx[k] = fmax(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
    }
    if (lane == 0) { smn[k][warp] = mn[k]; smx[k][warp] = mx[k]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = blockDim.x / 32;
    double a[3], c[3];
    for (int k = 0; k < 3; ++k) {
      a[k] = smn[k][0];
      c[k] = smx[k][0];
      for (int w = 1; w < nw; ++w) { a[k] = fmin(a[k], smn[k][w]); c[k] = fmax(c[k], smx[k][w]); }
    }
    if (nsplit == 1) {
      box_finish(node, a, c, lo, hi, n_nodes_total, split_dim);
    } else {
      double *pp = part + ((int64_t)blockIdx.x * nsplit + blockIdx.y) * 6;
      for (int k = 0; k < 3; ++k) { pp[k] = a[k]; pp[3 + k] = c[k]; }
    }
  }
}

// The boxes of nodes split over several CTAs: minima and maxima of the parts.
__global__ void k_node_boxes_final(int n_at, int nsplit, int first_node, const double *part,
                                   double *lo, double *hi, int n_nodes_total, int *split_dim) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_at) return;
  double a[3] = {INFINITY, INFINITY, INFINITY}, c[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int q = 0; q < nsplit; ++q) {
    const double *pp = part + ((int64_t)i * nsplit + q) * 6;
    for (int k = 0; k < 3; ++k) { a[k] = fmin(a[k], pp[k]); c[k] = fmax(c[k], pp[3 + k]); }
  }
  box_finish(first_node + i, a, c, lo, hi, n_nodes_total, split_dim);
}

// Sort keys of every node of one depth, each segment padded to P slots.
__global__ void k_fill_keys(const double *__restrict__ x, const double *__restrict__ y,
                            const double *__restrict__ z, const int32_t *__restrict__ cur,
                            const int64_t *__restrict__ begin, const int64_t *__restrict__ end,
                            const int *__restrict__ split_dim, int first_node, int n_seg,
                            int64_t P, SortItem *items) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_seg * P) return;
  int seg = (int)(i / P);
  int64_t slot = i - (int64_t)seg * P;
  int node = first_node + seg;
  int64_t b = begin[node], e = end[node];
  SortItem it;
  it.pad = 0;
  if (b + slot < e) {
    int32_t q = cur[b + slot];
    int s = split_dim[node];
    double v = s == 0 ? x[q] : (s == 1 ? y[q] : z[q]);
    it.key = order_key(v);
    it.idx = (unsigned int)q;
  } else {
    it.key = ~0ull;
    it.idx = ~0u;
  }
  items[i] = it;
}

// Bitonic compare-exchange for one (size, stride) step over global memory.
__global__ void k_bitonic_global(SortItem *items, int64_t total, int64_t P, int64_t size,
                                 int64_t stride) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // thread t handles the pair whose lower index has bit `stride` clear
  // (stride is a power of two: the index is t with a zero bit inserted)
  int64_t i = ((t & ~(stride - 1)) << 1) | (t & (stride - 1));
  int64_t j = i + stride;
  if (j >= total) return;
  bool up = ((i & (P - 1)) & size) == 0;
  SortItem a = items[i], b = items[j];
  bool swap = up ? item_less(b, a) : item_less(a, b);
  if (swap) { items[i] = b; items[j] = a; }
}

// All steps with stride < kSortTile/2 of sizes [size_lo, size_hi] in shared
// memory; one CTA per tile of kSortTile elements.
__global__ void __launch_bounds__(kSortTile / 2) k_bitonic_smem(SortItem *items, int64_t total,
                                                               int64_t P, int64_t size_lo,
                                                               int64_t size_hi) {
  __shared__ SortItem sh[kSortTile];
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int q = threadIdx.x; q < kSortTile; q += blockDim.x) {
    int64_t g = base + q;
    if (g < total) sh[q] = items[g];
    else { sh[q].key = ~0ull; sh[q].idx = ~0u; sh[q].pad = 0; }
  }
  __syncthreads();
  for (int64_t size = size_lo; size <= size_hi; size <<= 1) {
    int64_t s0 = size / 2;
    if (s0 > kSortTile / 2) s0 = kSortTile / 2;
    for (int64_t stride = s0; stride > 0; stride >>= 1) {
      const int t = threadIdx.x, st = (int)stride;   // a power of two
      const int i = ((t & ~(st - 1)) << 1) | (t & (st - 1));
      const int j = i + st;
      int64_t gi = base + i;
      bool up = ((gi & (P - 1)) & size) == 0;
      SortItem a = sh[i], b = sh[j];
      bool swap = up ? item_less(b, a) : item_less(a, b);
      if (swap) { sh[i] = b; sh[j] = a; }
      __syncthreads();
    }
  }
  for (int q = threadIdx.x; q < kSortTile; q += blockDim.x) {
    int64_t g = base + q;
    if (g < total) items[g] = sh[q];
  }
}

__global__ void k_scatter_sorted(const SortItem *__restrict__ items,
                                 const int64_t *__restrict__ begin,
                                 const int64_t *__restrict__ end, int first_node, int n_seg,
                                 int64_t P, int32_t *cur) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= (int64_t)n_seg * P) return;
  int seg = (int)(i / P);
  int64_t slot = i - (int64_t)seg * P;
  int node = first_node + seg;
  int64_t b = begin[node], e = end[node];
  if (b + slot < e) cur[b + slot] = (int32_t)items[i].idx;
}

__global__ void k_gather_tree_coords(const double *x, const double *y, const double *z,
                                     const int32_t *perm, int64_t n, double *xt, double *yt,
                                     double *zt, int32_t *iperm) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t q = perm[i];
  xt[i] = x[q];
  yt[i] = y[q];
  zt[i] = z[q];
  iperm[q] = (int32_t)i;
}

__global__ void k_diameters(const double *lo, const double *hi, int n_nodes, double *diam) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n_nodes) return;
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double e = __dsub_rn(hi[k * n_nodes + v], lo[k * n_nodes + v]);
    acc = __dadd_rn(acc, __dmul_rn(e, e));
  }
  diam[v] = __dsqrt_rn(acc);
}

__device__ __forceinline__ bool admissible_pair(int s, int t, const double *__restrict__ lo,
                                                const double *__restrict__ hi,
                                                const double *__restrict__ diam, int n_nodes,
                                                double eta) {
  double acc = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double a = __dsub_rn(lo[k * n_nodes + t], hi[k * n_nodes + s]);
    double b = __dsub_rn(lo[k * n_nodes + s], hi[k * n_nodes + t]);
    double g = fmax(0.0, fmax(a, b));
    acc = __dadd_rn(acc, __dmul_rn(g, g));
  }
  double dist = __dsqrt_rn(acc);
  return dist > 0.0 && __dmul_rn(0.5, __dadd_rn(diam[s], diam[t])) <= __dmul_rn(eta, dist);
}

// Pass 1 of one depth of the dual traversal: every node s of depth k scans
// the children of its parent's inadmissible partners (in increasing id) and
// counts admissible (-> F) and inadmissible (-> next frontier or N) pairs.
// Pass 2 (fill = true) writes them in the same order, so rows come out sorted.
// One warp per node s of depth k: the lanes take the parent's inadmissible
// partners 32 at a time; each partner contributes its two children in order,
// so both output lists stay sorted.  Positions come from ballots (a lane adds
// 0, 1 or 2 entries to each list).
template <bool FILL>
__global__ void k_traverse(int k, int n_nodes, const double *__restrict__ lo,
                           const double *__restrict__ hi, const double *__restrict__ diam,
                           double eta, const int64_t *__restrict__ par_ptr,
                           const int32_t *__restrict__ par_idx, int64_t *cnt_far,
                           int64_t *cnt_in, const int64_t *__restrict__ far_ptr,
                           int32_t *far_idx, const int64_t *__restrict__ in_ptr,
                           int32_t *in_idx) {
  const int lane = threadIdx.x & 31;
  const int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int n_at = 1 << k;
  if (r >= n_at) return;   // whole warps leave together
  const int s = (1 << k) - 1 + r;
  const int p = (s - 1) / 2;
  const int pr = p - ((1 << (k - 1)) - 1);
  int64_t nf = 0, ni = 0;
  const int64_t of = FILL ? far_ptr[r] : 0, oi = FILL ? in_ptr[r] : 0;
  const uint32_t lt = (1u << lane) - 1u;
  for (int64_t e0 = par_ptr[pr]; e0 < par_ptr[pr + 1]; e0 += 32) {
    const int64_t e = e0 + lane;
    const bool has = e < par_ptr[pr + 1];
    int t1 = 0, t2 = 0;
    bool a1 = false, a2 = false;
    if (has) {
      const int tp = par_idx[e];
      t1 = 2 * tp + 1;
      t2 = 2 * tp + 2;
      a1 = admissible_pair(s, t1, lo, hi, diam, n_nodes, eta);
      a2 = admissible_pair(s, t2, lo, hi, diam, n_nodes, eta);
    }
    const int fc = (int)a1 + (int)a2;
    const int ic = has ? 2 - fc : 0;
    const uint32_t f1 = __ballot_sync(0xffffffffu, fc >= 1), f2 = __ballot_sync(0xffffffffu, fc == 2);
    const uint32_t i1 = __ballot_sync(0xffffffffu, ic >= 1), i2 = __ballot_sync(0xffffffffu, ic == 2);
    if (FILL && has) {
      int64_t pf = of + nf + __popc(f1 & lt) + __popc(f2 & lt);
      int64_t pi = oi + ni + __popc(i1 & lt) + __popc(i2 & lt);
      if (a1) far_idx[pf++] = t1; else in_idx[pi++] = t1;
      if (a2) far_idx[pf] = t2; else in_idx[pi] = t2;
    }
    nf += __popc(f1) + __popc(f2);
    ni += __popc(i1) + __popc(i2);
  }
  if (!FILL && lane == 0) {
    cnt_far[r] = nf;
    cnt_in[r] = ni;
  }
}

__global__ void k_scan_single(const int64_t *in, const int32_t *in32, int64_t *out, int64_t n) {
  __shared__ int64_t warp_sums[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t base = 0; base < n; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < n ? (in ? in[i] : (int64_t)in32[i]) : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int nw = blockDim.x / 32;
      int64_t w = lane < nw ? warp_sums[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nw) warp_sums[lane] = w;
    }
    __syncthreads();
    int64_t incl = x + (warp > 0 ? warp_sums[warp - 1] : 0) + carry;
    if (i < n) out[i] = incl - v;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = carry;
}

// Three-phase scan for long arrays: each CTA scans its 1024-element tile in
// place (exclusive) and writes the tile's total; the totals are scanned by one
// CTA; each tile then adds its offset.
__global__ void k_scan_tiles(const int64_t *in, const int32_t *in32, int64_t *out, int64_t n,
                             int64_t *tile_sums) {
  __shared__ int64_t warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t v = i < n ? (in ? in[i] : (int64_t)in32[i]) : 0;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x / 32;
    int64_t w = lane < nw ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) warp_sums[lane] = w;
  }
  __syncthreads();
  const int64_t incl = x + (warp > 0 ? warp_sums[warp - 1] : 0);
  if (i < n) out[i] = incl - v;
  if (threadIdx.x == blockDim.x - 1) tile_sums[blockIdx.x] = incl;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *tile_offsets) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tile_offsets[blockIdx.x];
}

int64_t next_pow2(int64_t v) {
  int64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

void sort_segments(SortItem *items, int64_t total, int64_t P, cudaStream_t s) {
  int64_t tile = kSortTile;
  int64_t first_hi = std::min<int64_t>(P, tile);
  int nblk = ceil_div(total, tile);
  k_bitonic_smem<<<nblk, kSortTile / 2, 0, s>>>(items, total, P, 2, first_hi);
  count_launch();
  H2_CHECK_LAUNCH();
  for (int64_t size = 2 * tile; size <= P; size <<= 1) {
    for (int64_t stride = size / 2; stride >= tile; stride >>= 1) {
      int64_t pairs = total / 2;
      k_bitonic_global<<<ceil_div(pairs, 256), 256, 0, s>>>(items, total, P, size, stride);
      count_launch();
      H2_CHECK_LAUNCH();
    }
    k_bitonic_smem<<<nblk, kSortTile / 2, 0, s>>>(items, total, P, size, size);
    count_launch();
    H2_CHECK_LAUNCH();
  }
}

}  // namespace

namespace {
// out[0..n] = exclusive scan of in (int64 or int32) with out[n] = the total.
void scan_any(const int64_t *in, const int32_t *in32, int64_t *out, int64_t n, cudaStream_t s) {
  constexpr int kTile = 1024;
  if (n <= 8 * kTile) {
    k_scan_single<<<1, kTile, 0, s>>>(in, in32, out, n);
    count_launch();
    H2_CHECK_LAUNCH();
    return;
  }
  const int64_t nb = (n + kTile - 1) / kTile;
  DBuf<int64_t> sums, offs;
  sums.alloc(nb);
  offs.alloc(nb + 1);
  k_scan_tiles<<<(unsigned)nb, kTile, 0, s>>>(in, in32, out, n, sums.p);
  count_launch();
  H2_CHECK_LAUNCH();
  k_scan_single<<<1, kTile, 0, s>>>(sums.p, nullptr, offs.p, nb);
  count_launch();
  H2_CHECK_LAUNCH();
  k_scan_add<<<(unsigned)nb, kTile, 0, s>>>(out, n, offs.p);
  count_launch();
  H2_CHECK_LAUNCH();
  // the total is the scan of the tile sums at nb
  H2_CUDA(cudaMemcpyAsync(out + n, offs.p + nb, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
}
}  // namespace

void scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  scan_any(in, nullptr, out, n, s);
}

void scan_exclusive_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s) {
  scan_any(nullptr, in, out, n, s);
}

int leaf_depth(int64_t n, int leaf) {
  int L = 0;
  while ((n + (1ll << L) - 1) / (1ll << L) > leaf) ++L;
  return L;
}

// Builds the tree into *t.  Throws h2::Error.
void build_tree(const double *pts, int64_t n, int dim, int leaf, double eta, cudaStream_t s,
                h2_tree *t) {
  H2_REQUIRE(pts != nullptr, "points is NULL");
  H2_REQUIRE(n >= 1 && n < (1ll << 31) - 1, "n must be in [1, 2^31-2]");
  H2_REQUIRE(dim >= 1 && dim <= 3, "dim must be 1, 2 or 3");
  H2_REQUIRE(leaf >= 2, "leaf_size must be >= 2");
  H2_REQUIRE(eta >= 0.0 && std::isfinite(eta), "eta must be finite and >= 0");
  t->n = n;
  t->dim = dim;
  t->leaf_size = leaf;
  t->eta = eta;
  int L = leaf_depth(n, leaf);
  H2_REQUIRE(L <= 30, "tree too deep");
  t->depth = L;
  int n_nodes = (1 << (L + 1)) - 1;
  t->n_nodes = n_nodes;

  DBuf<int> bad;
  bad.alloc_zero(1, s);
  k_check_points<<<ceil_div(n * dim, 256), 256, 0, s>>>(pts, n, dim, bad.p);
  count_launch();
  H2_CHECK_LAUNCH();
  if (to_host(bad.p, 1, s)[0]) throw Error{H2_ERR_INPUT, "non-finite point coordinates"};

  // node ranges follow from n alone (left child takes ceil(size/2))
  t->h_begin.assign(n_nodes, 0);
  t->h_end.assign(n_nodes, 0);
  t->h_end[0] = n;
  for (int v = 0; 2 * v + 1 < n_nodes; ++v) {
    int64_t sz = t->h_end[v] - t->h_begin[v];
    int64_t nl = (sz + 1) / 2;
    t->h_begin[2 * v + 1] = t->h_begin[v];
    t->h_end[2 * v + 1] = t->h_begin[v] + nl;
    t->h_begin[2 * v + 2] = t->h_begin[v] + nl;
    t->h_end[2 * v + 2] = t->h_end[v];
  }
  to_device(t->begin, t->h_begin, s);
  to_device(t->end, t->h_end, s);

  DBuf<double> ox, oy, oz;
  ox.alloc(n);
  oy.alloc(n);
  oz.alloc(n);
  k_split_coords<<<ceil_div(n, 256), 256, 0, s>>>(pts, n, dim, ox.p, oy.p, oz.p);
  count_launch();
  H2_CHECK_LAUNCH();

  t->perm.alloc(n);
  k_iota<<<ceil_div(n, 256), 256, 0, s>>>(t->perm.p, n);
  count_launch();
  H2_CHECK_LAUNCH();
  t->lo.alloc(3 * (size_t)n_nodes);
  t->hi.alloc(3 * (size_t)n_nodes);
  DBuf<int> split;
  split.alloc(n_nodes);
  DBuf<SortItem> items;
  DBuf<double> box_part;   // partial boxes of nodes split over several CTAs
  const int sms = device_sm_count();

  for (int k = 0; k <= L; ++k) {
    int first = (1 << k) - 1;
    int n_at = 1 << k;
    {
      // nodes of the top levels are split over several CTAs (slices of at
      // least 1024 points) so that the level fills the device
      const int64_t seg = (n + n_at - 1) / n_at;
      int nsplit = n_at >= 2 * sms ? 1 : (2 * sms + n_at - 1) / n_at;
      nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(nsplit, seg / 1024));
      if (nsplit > 1 && (int64_t)box_part.n < (int64_t)n_at * nsplit * 6)
        box_part.alloc((size_t)n_at * nsplit * 6);
      k_node_boxes<<<dim3(n_at, nsplit), 256, 0, s>>>(ox.p, oy.p, oz.p, t->perm.p, t->begin.p,
                                                      t->end.p, first, t->lo.p, t->hi.p, n_nodes,
                                                      split.p, box_part.p);
      count_launch();
      H2_CHECK_LAUNCH();
      if (nsplit > 1) {
        k_node_boxes_final<<<ceil_div(n_at, 128), 128, 0, s>>>(n_at, nsplit, first, box_part.p,
                                                                t->lo.p, t->hi.p, n_nodes,
                                                                split.p);
        count_launch();
        H2_CHECK_LAUNCH();
      }
    }
    if (k == L) break;
    int64_t maxseg = (n + n_at - 1) / n_at;
    int64_t P = next_pow2(maxseg);
    int64_t total = (int64_t)n_at * P;
    if ((int64_t)items.n < total) items.alloc(total);
    k_fill_keys<<<ceil_div(total, 256), 256, 0, s>>>(ox.p, oy.p, oz.p, t->perm.p, t->begin.p,
                                                     t->end.p, split.p, first, n_at, P,
                                                     items.p);
    count_launch();
    H2_CHECK_LAUNCH();
    sort_segments(items.p, total, P, s);
    k_scatter_sorted<<<ceil_div(total, 256), 256, 0, s>>>(items.p, t->begin.p, t->end.p, first,
                                                          n_at, P, t->perm.p);
    count_launch();
    H2_CHECK_LAUNCH();
  }

  t->x.alloc(n);
  t->y.alloc(n);
  t->z.alloc(n);
  t->iperm.alloc(n);
  k_gather_tree_coords<<<ceil_div(n, 256), 256, 0, s>>>(ox.p, oy.p, oz.p, t->perm.p, n, t->x.p,
                                                        t->y.p, t->z.p, t->iperm.p);
  count_launch();
  H2_CHECK_LAUNCH();
  t->diam.alloc(n_nodes);
  k_diameters<<<ceil_div(n_nodes, 256), 256, 0, s>>>(t->lo.p, t->hi.p, n_nodes, t->diam.p);
  count_launch();
  H2_CHECK_LAUNCH();

  // dual traversal, one depth at a time
  t->far_ptr.clear();
  t->far_idx.clear();
  t->far_nnz.assign(L + 1, 0);
  t->far_ptr.resize(L + 1);
  t->far_idx.resize(L + 1);
  // depth 0: the root pair is inadmissible (Dist = 0)
  t->far_ptr[0].alloc_zero(2, s);
  DBuf<int64_t> in_ptr;
  DBuf<int32_t> in_idx;
  if (L == 0) {
    std::vector<int64_t> p = {0, 1};
    std::vector<int32_t> c = {0};
    to_device(t->near_ptr, p, s);
    to_device(t->near_idx, c, s);
    t->near_nnz = 1;
  } else {
    std::vector<int64_t> p = {0, 1};
    std::vector<int32_t> c = {0};
    to_device(in_ptr, p, s);
    to_device(in_idx, c, s);
  }
  for (int k = 1; k <= L; ++k) {
    int n_at = 1 << k;
    DBuf<int64_t> cf, ci, pf, pi;
    cf.alloc(n_at);
    ci.alloc(n_at);
    pf.alloc(n_at + 1);
    pi.alloc(n_at + 1);
    int nb = ceil_div((int64_t)n_at * 32, 256);   // one warp per node
    k_traverse<false><<<nb, 256, 0, s>>>(k, n_nodes, t->lo.p, t->hi.p, t->diam.p, eta, in_ptr.p,
                                         in_idx.p, cf.p, ci.p, nullptr, nullptr, nullptr,
                                         nullptr);
    count_launch();
    H2_CHECK_LAUNCH();
    scan_exclusive(cf.p, pf.p, n_at, s);
    scan_exclusive(ci.p, pi.p, n_at, s);
    int64_t tot[2];
    H2_CUDA(cudaMemcpyAsync(&tot[0], pf.p + n_at, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaMemcpyAsync(&tot[1], pi.p + n_at, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    DBuf<int32_t> fidx, iidx;
    fidx.alloc(std::max<int64_t>(tot[0], 1));
    iidx.alloc(std::max<int64_t>(tot[1], 1));
    k_traverse<true><<<nb, 256, 0, s>>>(k, n_nodes, t->lo.p, t->hi.p, t->diam.p, eta, in_ptr.p,
                                        in_idx.p, nullptr, nullptr, pf.p, fidx.p, pi.p, iidx.p);
    count_launch();
    H2_CHECK_LAUNCH();
    t->far_ptr[k] = std::move(pf);
    t->far_idx[k] = std::move(fidx);
    t->far_nnz[k] = tot[0];
    if (k == L) {
      t->near_ptr = std::move(pi);
      t->near_idx = std::move(iidx);
      t->near_nnz = tot[1];
    } else {
      in_ptr = std::move(pi);
      in_idx = std::move(iidx);
    }
  }
  t->l_top = 0;
  for (int level = 1; level <= L + 1; ++level) {
    int depth = L - level + 1;
    if (t->far_nnz[depth] > 0) t->l_top = level;
  }
  H2_CUDA(cudaStreamSynchronize(s));
}

}  // namespace h2
