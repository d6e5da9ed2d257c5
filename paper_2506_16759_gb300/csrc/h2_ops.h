// Internal launch interfaces between the driver and the kernel translation
// units.  All pointers are device pointers unless stated otherwise.
#pragma once

#include "h2_internal.cuh"

namespace h2 {

// One instance of a (possibly batched) build, as seen by the kernels.
struct InstDev {
  int64_t pbase;   // first global tree position of the instance
  int64_t n;       // points
  KernelDesc kd;   // entry evaluator
};

// ---------------------------------------------------------------- sketch
// Work item of the fused kernel summation: rows [row0, row0+rows) of
// instance `inst` against its points [j0, j1), sample columns
// [c0, c0+DC) of the launch; part >= 0 selects a partial-sum slot.
struct KsumItem {
  int inst;
  int rows;
  int64_t row0;
  int64_t j0, j1;   // point range (all-points mode)
  int c0;
  int part;
  int task;         // far-only mode: the leaf task that owns the rows
  int lb0, lb1;     // far-only mode: range of leaf tasks summed over
};

// Leaf tasks and their near lists, for the far-only summation
// Y_loc(I_t) = sum over points outside the near leaves of t.
struct FarLists {
  const int64_t *leaf_row;  // first tree position of each leaf task
  const int32_t *leaf_m;    // points of each leaf task
  const int64_t *near_ptr;  // near CSR over leaf tasks (sorted)
  const int32_t *near_idx;
};

// Plan for one ksum launch (host side): items and the partial reduction.
struct KsumPlan {
  std::vector<KsumItem> items;
  int64_t n_parts = 0;      // partial slots (each tile_rows x dc values)
  int tile_rows = 0;
  int dc = 0;
  // reduction: for each output tile (inst, row0, rows, c0) the first slot and count
  struct Red {
    int inst, rows;
    int64_t row0;
    int c0;
    int64_t slot0;
    int nslots;
  };
  std::vector<Red> reds;
};

struct KsumArgs64 {
  FarLists far;
  Points64 pts;
  const double *om;  // panel, ld = ld
  double *y;         // panel, ld = ld
  int64_t ld;
  const InstDev *inst;
  const KsumItem *items;
  double *partial;
};
struct KsumArgs32 {
  FarLists far;
  Points32 pts;
  const float *om;
  float *y;
  int64_t ld;
  const InstDev *inst;
  const KsumItem *items;
  float *partial;
};

// Plans a launch covering, for every listed instance, all its rows and
// columns [c0[i], c0[i]+ncols).  `insts` are instance indices.
KsumPlan plan_ksum(const std::vector<int64_t> &inst_n, const std::vector<int64_t> &inst_base,
                   const std::vector<int> &insts, const std::vector<int> &c0, int ncols,
                   bool fp64, int tile_rows_hint, int sm_count);

// Plan of the far-only summation over the leaf tasks [t0, t1) of each listed
// instance (one item row tile = one leaf).  leaf_base/leaf_count: per
// instance, its first leaf task and number of leaves.
// pair_leaves: row tiles of two consecutive leaves (128 rows, tensor-core path).
KsumPlan plan_ksum_far(const std::vector<int64_t> &leaf_row, const std::vector<int32_t> &leaf_m,
                       const std::vector<int> &leaf_base, const std::vector<int> &leaf_count,
                       const std::vector<int> &insts, const std::vector<int> &c0, int ncols,
                       int sm_count, bool pair_leaves = false, int split = 0);

// Runs a plan (items/partials staged in `scratch`-owned buffers).  Returns the
// number of kernel launches.  `work` must hold plan.n_parts*tile_rows*dc
// values; items/reds are copied to device-side staging inside.
void run_ksum64(int kid, const KsumPlan &plan, const KsumArgs64 &a, cudaStream_t s,
                bool far = false);
void run_ksum32(int kid, const KsumPlan &plan, const KsumArgs32 &a, cudaStream_t s,
                bool far = false);

// ---- tensor-core sketch (sketch_tc.cu)
// Leaves padded to whole tiles (32 points with TF32 parts, 64 with FP16
// parts).  Per padded point: its offset from
// its leaf's reference point; per leaf: the reference (FP32 hi/lo parts);
// both multiplied by the instance's coordinate scale sigma.
struct TcLayout {
  bool f16 = false;          // FP16 parts (64-point tiles) instead of TF32 (32-point tiles)
  int tj = 32;
  int64_t n_tiles = 0;
  DBuf<int64_t> leaf_tile;   // first tile of each leaf
  DBuf<int32_t> tile_leaf;   // leaf of each tile
  DBuf<int32_t> leaf_inst;   // instance of each leaf
  DBuf<double> sigma;        // per instance
  DBuf<float4> ref_hi, ref_lo, off;
};
// Arguments of one tensor-core launch (device pointers).
struct TcArgs {
  const KsumItem *items;
  const InstDev *inst;
  Points64 p64;              // FP64 coordinates in tree order
  const int64_t *leaf_row;   // leaves (the layout's), first position and size
  const int32_t *leaf_m;
  const int64_t *leaf_tile;
  const float4 *ref_hi, *ref_lo, *off;
  const double *sigma;
  const int64_t *near_ptr;   // far-only mode: near leaves of each leaf (sorted CSR)
  const int32_t *near_idx;
  const int32_t *ul_leaf;    // near-only mode: per item entries [lb0, lb1) of the union
  const int32_t *ul_flags;   //   of its leaves' near lists; bit 1/2: not near to leaf 1/2
  const float *img_hi, *img_lo;   // Omega image: 128-byte rows [tile][img_nc]
  int img_nc, img_c0;        // image columns; first one read by this launch
  const float *om;           // Omega panel (tree order, ld) for the diagonal term
  float *y;                  // output panel, ld
  int64_t ld;
  float *partial;            // plan partial slots (kRows x ncol each)
  int *err;                  // set if an mbarrier wait timed out
  int ncol;                  // valid columns of this launch (<= the template width)
  int stall;                 // self-test: the producer issues nothing, the waits run out
};
constexpr int kTcChunk = 80;  // sample columns per tensor-core launch at most
int tc_chunk_ncol(int w);    // template width (16, 32, 64 or 80) for w <= 80 columns
// Kernels whose entries are at most 1 (FP16 parts allowed).
bool tc_f16_kernel(int kid);
// max |x| over rows [0, n) and columns [c0, c1) (synchronises the stream).
float tc_max_abs(const float *x, int64_t ld, int64_t n, int c0, int c1, cudaStream_t s);
void tc_layout_build(int kid, bool f16, const std::vector<int64_t> &leaf_row,
                     const std::vector<int32_t> &leaf_m, const std::vector<int32_t> &leaf_inst,
                     const std::vector<KernelDesc> &inst_kd, const int64_t *d_leaf_row,
                     const int32_t *d_leaf_m, Points64 p64, TcLayout &out, cudaStream_t s);
// Omega image of the columns [c0_inst, c0_inst + nc) (d_inst_c0 per instance)
// with img_nc >= nc columns per tile (extra columns zero).
void tc_omega_image(const TcLayout &L, const int64_t *d_leaf_row, const int32_t *d_leaf_m,
                    const float *om, int64_t ld, const int32_t *d_inst_c0, int nc, int img_nc,
                    float *img_hi, float *img_lo, cudaStream_t s);
// mode: 0 all points, 1 far-only, 2 near-only.
void launch_ksum_tc(int kid, int ncol_tmpl, int mode, bool f16, int64_t items, const TcArgs &a,
                    cudaStream_t s);
// Stages a plan (plan.tile_rows = 128, plan.dc = valid columns <= 64) and
// runs it on the tensor cores; a.items/partial/err are filled in here.
void run_ksum_tc(int kid, const KsumPlan &plan, const TcArgs &a, int mode, bool f16,
                 cudaStream_t s);
// Near-only plan: one item per pair of consecutive leaves of each listed
// instance, over the union of the pair's near lists (host CSR near_ptr /
// near_idx over leaf tasks); fills ul_leaf / ul_flags (host).
KsumPlan plan_ksum_tc_near(const std::vector<int32_t> &leaf_m, const std::vector<int64_t> &leaf_row,
                           const std::vector<int> &leaf_base, const std::vector<int> &leaf_count,
                           const std::vector<int64_t> &near_ptr,
                           const std::vector<int32_t> &near_idx, const std::vector<int> &insts,
                           const std::vector<int> &c0, int ncols, std::vector<int32_t> &ul_leaf,
                           std::vector<int32_t> &ul_flags);
// Y = K Omega on the tensor cores for a flat point set (the points taken as
// consecutive leaves of one tile each); stall: self-test (waits run out).
void tc_sum_points(int kernel_id, const KernelDesc &kd, const InstDev *idev, Points64 p64,
                   int64_t n, const float *om32, float *y32, int d, bool stall, cudaStream_t st);
// Plan of the all-points summation for the tensor-core kernel: 128-row
// tiles, the point range split over leaf ranges [lb0, lb1) of the layout.
KsumPlan plan_ksum_tc_all(const std::vector<int64_t> &inst_n, const std::vector<int64_t> &inst_base,
                          const std::vector<int> &leaf_base, const std::vector<int> &leaf_count,
                          const std::vector<int> &insts, const std::vector<int> &c0, int ncols,
                          int sm_count);

// Gaussian sample columns for rows in tree order: om[pos + c*ld] for
// c in [c0, c1), drawn from Philox4x32-10 keyed by (seed) at counter
// (original index of pos, column pair), Box-Muller in FP64 (53-bit
// uniforms) or, with f32_math, in FP32 (24-bit uniforms).
void philox_gaussian64(double *om, int64_t ld, const int32_t *orig_of_pos, int64_t n, int c0,
                       int c1, uint64_t seed, bool f32_math, cudaStream_t s);
// Stored Omega (original order, ld_src) gathered into tree order.
void gather_rows64(const double *src, int64_t ld_src, const int32_t *orig_of_pos, int64_t n,
                   int c0, int c1, double *dst, int64_t ld_dst, cudaStream_t s);
void convert_cols_to32(const double *src, int64_t ld, int64_t row0, int64_t n, int c0, int c1,
                       float *dst, cudaStream_t s);

// Dense GEMM Y[:, c] = A Om[:, c] (FP64), all column-major.
void dense_gemm64(const double *a, int64_t lda, int64_t n, const double *om, int64_t ldo,
                  double *y, int64_t ldy, int d, cudaStream_t s, bool trans = false);
// Entries K(rows, cols) into out (nr x nc, ld nr).
void entry_block64(int kid, const KernelDesc &kd, Points64 pts, const int32_t *rows, int64_t nr,
                   const int32_t *cols, int64_t nc, double *out, cudaStream_t s);

// Split FP64 coordinates into FP32 hi/lo parts.
void split_coords32(const double *x, const double *y, const double *z, int64_t n, float *xh,
                    float *yh, float *zh, float *xl, float *yl, float *zl, cudaStream_t s);

// Row-major n x dim points -> SoA (zero padding to 3 coordinates).
void split_points_soa(const double *pts, int64_t n, int dim, double *x, double *y, double *z,
                      cudaStream_t s);
void convert_to64(const float *src, int64_t n, double *dst, cudaStream_t s);

// Sum of squares of (panel + panel2) columns [0, d) over each instance's rows
// (FP64 result); panel2 may be NULL.
void instance_sumsq(const void *panel, const void *panel2, bool fp64, int64_t ld,
                    const int64_t *inst_base, const int64_t *inst_n, int count, int d,
                    double *out, cudaStream_t s);

}  // namespace h2
