/*
 * h2gb: bottom-up adaptive-sketching H2 matrix construction on one GB300
 * (sm_103a).  C ABI of libh2gb.so.
 *
 * Method: Boukaram, Liu, Ghysels, Li, "Adaptive Sketching Based Construction
 * of H2 Matrices on GPUs" (arXiv 2506.16759).  Algorithm 1 builds the nested
 * bases, couplings and dense near-field blocks level by level from the leaves,
 * driven by a black-box sketch Y = K Omega and an entry evaluator; Sec. III-B
 * adds samples until every cluster's local samples pass a QR-based
 * convergence test.
 *
 * Conventions for every entry point:
 *  - Pointers documented as "device" must point to memory of the current CUDA
 *    device; "host" pointers to host memory.  The caller owns every buffer it
 *    passes in; the library copies what it keeps.
 *  - Matrices are column-major.  Vectors and panels exchanged with the caller
 *    are in the caller's ORIGINAL point order; the library permutes to its
 *    cluster-tree order internally.
 *  - All GPU work is enqueued on the given stream (NULL = legacy default
 *    stream).  Calls return once the host-side decisions they need are made
 *    (level sizes, the adaptive "any cluster unconverged" flag).
 *  - Errors are returned as h2_status; h2_last_error() gives a message for the
 *    calling thread.  Nothing aborts the process.  Handles are freed only by
 *    the matching *_destroy call.
 */
#ifndef H2GB_H
#define H2GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *h2_stream_t; /* a cudaStream_t */

typedef enum {
  H2_OK = 0,
  H2_ERR_ARG = -1,            /* invalid argument (message says which) */
  H2_ERR_CUDA = -2,           /* a CUDA call failed */
  H2_ERR_OOM = -3,            /* device allocation failed */
  H2_ERR_NOT_CONVERGED = -4,  /* d_max reached before every cluster converged;
                                 the H2 matrix is still complete and usable */
  H2_ERR_TIMEOUT = -5,        /* a bounded wait inside a kernel ran out; the
                                 kernel ended without faulting and the device
                                 context stays usable */
  H2_ERR_SAMPLER = -6,        /* the user sampler returned non-zero */
  H2_ERR_INPUT = -7           /* non-finite coordinates or sketch values */
} h2_status;

/* Kernels of the workloads.  params[] per kernel:
 *   H2_K_EXP        exp(-r/l) (+ nugget on the diagonal)   {l, nugget}
 *                   -- the covariance kernel of Sec. V-A
 *   H2_K_MATERN32   (1+sqrt3 r/l) exp(-sqrt3 r/l) (+nugget) {l, nugget}
 *   H2_K_GAUSS      exp(-r^2/(2 s^2)) (+ nugget)            {s, nugget}
 *   H2_K_LAPLACE_IE 1/(4 pi r) off the diagonal, diag on it {diag}
 *   H2_K_POLY       (c + x.y)^p, p a small integer          {c, p}
 *   H2_K_H2SUM      sum of existing H2 matrices (the update workload of
 *                   Sec. V-A); operands given in h2_build_opts
 *   H2_K_HELMHOLTZ_IE cos(k r)/r off the diagonal, diag on it {k, diag}
 *                   -- the Helmholtz volume-IE operator of Sec. V-A (the
 *                   paper fixes k = 3 and defines only x != y)           */
typedef enum {
  H2_K_EXP = 0,
  H2_K_MATERN32 = 1,
  H2_K_GAUSS = 2,
  H2_K_LAPLACE_IE = 3,
  H2_K_POLY = 4,
  H2_K_H2SUM = 5,
  H2_K_HELMHOLTZ_IE = 6
} h2_kernel;

typedef enum {
  H2_PREC_FP64 = 0,       /* every step in FP64 */
  H2_PREC_MIXED = 1,      /* entries and block products in FP32, the fused
                             sketch on the tensor cores (two-part operands:
                             FP16 for the exponential, Matern and Gaussian
                             kernels with drawn Omega, TF32 otherwise; FP32
                             accumulation); QR convergence test and
                             pivoted-QR ID in FP64 */
  H2_PREC_MIXED_SIMT = 2  /* as H2_PREC_MIXED with the sketch in FP32 on the
                             CUDA cores */
} h2_prec;

typedef enum {
  H2_SKETCH_KSUM = 0,     /* built-in fused kernel summation Y = K Omega */
  H2_SKETCH_DENSE = 1,    /* Y = A Omega with a caller-supplied dense A */
  H2_SKETCH_CALLBACK = 2, /* caller's h2_sampler_fn */
  H2_SKETCH_H2SUM = 3     /* Y = sum_op H2_op Omega (batched H2 matvecs) */
} h2_sketch_kind;

typedef struct h2_tree h2_tree;
typedef struct h2_matrix h2_matrix;

/* Black-box sketch K_blk of Algorithm 1: y = K omega for an n x d block of
 * sample vectors (device, column-major, leading dimension ld, original point
 * order), enqueued on stream s.  Return 0 on success. */
typedef int (*h2_sampler_fn)(void *ctx, const double *omega, double *y, int64_t n, int d,
                             int64_t ld, h2_stream_t s);

typedef struct {
  int d0;              /* initial samples (32) */
  int d_inc;           /* samples added per adaptive round (16); 0 = fixed sampling:
                          no convergence test, every cluster compressed from
                          its d0 samples (the non-adaptive construction) */
  int d_max;           /* sample budget (256) */
  int prec;            /* h2_prec */
  int omega_mode;      /* 0: Gaussian Omega from Philox4x32-10 (seed) and the
                          Box-Muller transform (FP64 builds: in FP64 on 53-bit
                          uniforms; mixed precision: in FP32 on 24-bit ones);
                          1: stored Omega (omega_stored) */
  uint64_t seed;
  const double *omega_stored; /* device, N_total x d_max, column-major with
                                 ld = N_total, original order (instances
                                 stacked in order) */
  int sketch;                 /* h2_sketch_kind */
  const double *dense_a;      /* device N x N column-major (H2_SKETCH_DENSE) */
  h2_sampler_fn sampler;      /* H2_SKETCH_CALLBACK */
  void *sampler_ctx;
  const h2_matrix *const *operands; /* H2_SKETCH_H2SUM / H2_K_H2SUM */
  int n_operands;
  int timing;                 /* 1: record per-phase CUDA-event timers */
  int ksum_tile;              /* 0 = autotuned; else rows per sketch CTA tile */
  /* Optional low-rank term: the operator becomes (kernel or H2 sum) + U V^T,
   * the update problem of Sec. V-A (an H2 matrix plus a rank-r product).
   * U, V: device, N x lowrank_rank column-major with ld = N, original point
   * order, FP64, read during the call only.  Unless nonsym = 1, U V^T must
   * be symmetric (the symmetric construction shares row and column bases),
   * e.g. V = U S with S symmetric.  Needs a single instance and a sketch in original order
   * (dense, callback or H2 sum): the library adds U (V^T Omega) to the
   * sampler's output and U(I,:) V(J,:)^T to every generated block. */
  const double *lowrank_u;
  const double *lowrank_v;
  int lowrank_rank;           /* 0 = none, at most 64 */
  /* Launch shapes (mixed precision; 0 = the default), the knobs h2_autotune
   * tunes: */
  int bsr_engine;             /* block-sparse products: 0 tensor cores where the
                                 blocks have at most 256 rows, 1 CUDA cores */
  int tc_cols;                /* sample columns per tensor-core sketch launch:
                                 0 = 80, or 64 or 32 */
  int ksum_split;             /* far-only sketch: target work items per SM, each
                                 a contiguous range of one row tile's partner
                                 leaves (0 = 32; items run largest first) */
  /* Non-symmetric operators (Sec. II-A: admissible blocks U_s B_st V_t^T with
   * separate row and column bases; Sec. III calls the change a direct
   * modification of the symmetric algorithm).  nonsym = 1: the row side runs
   * Algorithm 1 on Y = A Omega (row IDs, bases U), the column side on
   * Z = A^T Psi (column IDs, bases V), level by level together; each side's
   * far-field subtraction goes through the other side's bases, the couplings
   * are A(row skeletons, column skeletons), and nrmK is taken from both
   * sketches, sqrt((||Y||^2 + ||Z||^2) / (2 d0)).  A node is converged when
   * both of its sides are.  Needs a single instance, a kernel (not H2_K_H2SUM)
   * and a sketch in original order: dense (Z from the transpose of dense_a),
   * callback (sampler_t gives A^T x) or H2 matvecs (symmetric operands); the
   * low-rank term U V^T may then be non-symmetric. */
  int nonsym;
  const double *psi_stored;   /* omega_mode 1: the column side's samples,
                                 device N x d_max like omega_stored */
  h2_sampler_fn sampler_t;    /* nonsym + H2_SKETCH_CALLBACK: y = A^T x */
  void *sampler_t_ctx;
  int queue_order;            /* order of the per-cluster QR tests and IDs: 0 one
                                 CTA per cluster in tree order; 1 a work queue
                                 over a device-filling grid, largest estimated
                                 cost first (m d^2 for the test, d m min(m, d)
                                 for the ID).  Results do not depend on it. */
  int sum_engine;             /* couplings of an H2 sum (H2_K_H2SUM), mixed
                                 precision: 0 CUDA cores (FP32 products with
                                 compensated sums), 1 tensor cores (two-part
                                 TF32, accumulated in tensor memory: faster,
                                 but the accumulator adds a few units of 1e-7
                                 relative error, which can cost adaptive
                                 rounds on problems whose blocks are large
                                 against eps_l); falls back to 0 for target
                                 ranks above 96 */
} h2_build_opts;

/* Fills opts with the workload defaults (32/16/256, FP64, Philox seed 0,
 * built-in kernel summation). */
void h2_default_opts(h2_build_opts *opts);

/* ---------------------------------------------------------------------------
 * Cluster tree and block partition (Sec. II-A).
 * KD median bisection to a uniform leaf depth L (smallest L with
 * ceil(n/2^L) <= leaf_size): each node splits on the longest side of its tight
 * bounding box (lowest dimension on ties), points ordered by (coordinate,
 * original index), left child = first ceil(n/2).  The dual tree traversal
 * from (root, root) with the general admissibility condition
 * (D(s)+D(t))/2 <= eta Dist(s,t), Dist > 0, yields per-depth far lists F and
 * the leaf near list N (self included), rows sorted by node id.
 *
 * points: device, n x dim row-major FP64, dim in {1,2,3}, finite values.
 * leaf_size >= 2.  On success *out owns device copies of everything it needs.
 * ------------------------------------------------------------------------- */
h2_status h2_build_cluster_tree(const double *points, int64_t n, int dim, int leaf_size,
                                double eta, h2_stream_t s, h2_tree **out);

typedef struct {
  int64_t n;
  int dim;
  int leaf_size;
  double eta;
  int depth;        /* leaf depth L; heap node ids 0 .. 2^(L+1)-2 */
  int n_nodes;
  int l_top;        /* highest paper level (1 = leaves) with an admissible pair */
  int64_t near_nnz; /* entries of the leaf near list */
  int64_t far_nnz[64]; /* entries of the far list per depth (0..depth) */
} h2_tree_info_t;

h2_status h2_tree_info(const h2_tree *t, h2_tree_info_t *info);

/* Host copies for inspection.  perm[n]: tree position -> original index.
 * begin/end[n_nodes]: each node's range of tree positions.
 * lo/hi[n_nodes*dim]: tight boxes (node-major).  Any pointer may be NULL. */
h2_status h2_tree_export(const h2_tree *t, int32_t *perm, int64_t *begin, int64_t *end,
                         double *lo, double *hi);

/* Host copy of one list in CSR form over the nodes of `depth` (row r is heap
 * node 2^depth - 1 + r); cols hold heap node ids.  which = 0: far list F at
 * `depth`; which = 1: near list N (depth must be the leaf depth).  rowptr has
 * 2^depth + 1 entries; cols has the list's nnz entries. */
h2_status h2_tree_export_list(const h2_tree *t, int which, int depth, int64_t *rowptr,
                              int32_t *cols);

void h2_tree_destroy(h2_tree *t);

/* ---------------------------------------------------------------------------
 * H2 construction: Algorithm 1 with the adaptive loop of Sec. III-B.
 * For each level l = 1 (leaves) .. l_top: local samples (leaf near-field
 * subtraction with dense blocks D = K(I_t, I_b), or at inner levels the
 * merge of the children's skeleton samples minus the coupling products
 * B Omega^l), the QR convergence test (min_j |R_jj| <= eps_l, or m <= d),
 * extra d_inc samples swept up from the leaves while any cluster is
 * unconverged, the row ID by column-pivoted QR of Y_loc^T/sqrt(d), the
 * shrink/upsweep of Y and Omega, and the couplings B = K(Itil_s, Itil_t).
 * Thresholds: nrmK = ||Y||_F/sqrt(d0), eps_abs = tol*nrmK,
 * eps_l = eps_abs/sqrt(2 * l_top * n_l) (a Frobenius budget over the levels,
 * the nodes of a level and the row and column sides of each block).
 *
 * kernel_id/params/nparams: the entry evaluator (see h2_kernel).  tol >= 0.
 * Returns H2_ERR_NOT_CONVERGED (with *out valid) if d_max was reached.
 * ------------------------------------------------------------------------- */
h2_status h2_build(const h2_tree *tree, int kernel_id, const double *params, int nparams,
                   double tol, const h2_build_opts *opts, h2_stream_t s, h2_matrix **out);

/* Independent instances of uneven size built together: every per-level step
 * runs once for the clusters of all instances.  kernel_ids[count],
 * params[count*4] (row i = params of instance i), tols[count].  The result
 * is one handle; vectors for it stack the instances' points in order. */
h2_status h2_build_batched(const h2_tree *const *trees, int count, const int *kernel_ids,
                           const double *params, const double *tols,
                           const h2_build_opts *opts, h2_stream_t s, h2_matrix **out);

/* y = K_H2 x: x, y device, N_total x nrhs column-major (ld = N_total),
 * original order.  Upsweep x^ = U^T x / E^T [x^_1; x^_2], couplings at every
 * level, downsweep, near field.  Arithmetic in the matrix's precision. */
h2_status h2_matvec(const h2_matrix *h, const double *x, double *y, int nrhs, h2_stream_t s);

typedef struct {
  int count;               /* instances */
  int64_t n_total;
  int levels;              /* max l_top over instances */
  int d_final;             /* samples used (max over instances) */
  int rank_min, rank_max;  /* over all compressed clusters */
  int converged;           /* 1 if every instance converged within d_max */
  int64_t bytes_dense;     /* stored near-field blocks */
  int64_t bytes_coupling;  /* stored coupling blocks */
  int64_t bytes_basis;     /* stored U/E */
  int64_t near_entries;    /* sum of m_t*m_b over near pairs */
  int64_t sketch_pairs;    /* kernel entries evaluated by the built-in sketch */
  int64_t sketch_columns;  /* sample columns sketched (all rounds) */
  int64_t kernel_launches; /* CUDA kernels launched by the build */
  int rounds;              /* adaptive rounds taken */
  double nrmK;             /* of instance 0 */
  /* per-phase device time (ms) when opts.timing = 1 */
  double ms_tree_unused, ms_sketch, ms_nearfield, ms_qr, ms_id, ms_upsweep, ms_coupling,
      ms_bsr, ms_total;
  double ms_sketch_launch_max;  /* longest sketch phase (one round) */
  double sketch_flops;          /* algorithmic flops of the sketch launches:
                                   pairs * (2*columns + 10) */
  double ms_sketch_kernel;      /* summed device time of the fused-summation
                                   kernel launches alone (timing = 1) */
  int64_t sketch_launches;      /* fused-summation kernel launches */
} h2_stats_t;

h2_status h2_stats(const h2_matrix *h, h2_stats_t *st);

/* Host copies of one level of instance `inst` (paper level, 1 = leaves):
 * ranks[n_l] per cluster (heap order) and skel[sum ranks], each cluster's
 * skeleton rows as ORIGINAL point indices, clusters in heap order, rows in
 * the library's skeleton order (ascending candidate position).  eps_l/d_l may
 * be NULL. */
h2_status h2_export_level(const h2_matrix *h, int inst, int level, int32_t *ranks,
                          int32_t *skel, double *eps_l, int32_t *d_l);

/* The column side of a non-symmetric build (h2_build_opts.nonsym = 1): ranks
 * and column skeletons of one level, laid out as h2_export_level lays out the
 * row side's (which h2_export_level returns for such a matrix).  H2_ERR_ARG
 * for a symmetric build, whose rows and columns share one set of bases. */
h2_status h2_export_col_level(const h2_matrix *h, int inst, int level, int32_t *ranks,
                              int32_t *skel);

void h2_matrix_destroy(h2_matrix *h);

/* Autotuner: times full builds of `tree` and writes the fastest candidate
 * that converged into *best (other fields copied from *base); best_ms
 * receives its build time.  Stage 1 searches the sample schedule (d0, d_inc
 * in {32, 64, 80, leaf size} x {16, 32}, d0 <= d_max) and, for mixed
 * precision, both sketch engines (tensor cores / CUDA cores); later stages
 * keep that choice and try, one knob at a time, the block-sparse engine, the
 * sketch's columns per launch and its work split (h2_build_opts launch
 * shapes).  Every candidate is an ordinary adaptive build at tolerance tol,
 * so the choice changes speed, not the accuracy target. */
h2_status h2_autotune(const h2_tree *tree, int kernel_id, const double *params, int nparams,
                      double tol, const h2_build_opts *base, h2_stream_t s, h2_build_opts *best,
                      double *best_ms);

/* ---------------------------------------------------------------------------
 * Batched building blocks (the paper's batchedGen, K_blk, the convergence
 * QR and batchedID), exposed for direct use and testing.
 * ------------------------------------------------------------------------- */

/* Y = K Omega by on-the-fly kernel summation (the fused sketch).
 * points: device n x dim row-major; omega: device n x d (ld = ldo);
 * y: device n x d (ld = ldy); original order.  prec selects FP64 or FP32
 * arithmetic (FP32 evaluates distances from split hi/lo coordinates). */
h2_status h2_ksum_sketch(const double *points, int64_t n, int dim, int kernel_id,
                         const double *params, int nparams, const double *omega, int64_t ldo,
                         double *y, int64_t ldy, int d, int prec, h2_stream_t s);

/* Dense block K(rows, cols) (batchedGen for one block): rows[nr], cols[nc]
 * device int32 point indices; out device nr x nc column-major (ld = nr). */
h2_status h2_entry_block(const double *points, int64_t n, int dim, int kernel_id,
                         const double *params, int nparams, const int32_t *rows, int64_t nr,
                         const int32_t *cols, int64_t nc, double *out, h2_stream_t s);

/* Dense sketch Y = A Omega, A device n x n column-major (ld = lda). */
h2_status h2_dense_sketch(const double *a, int64_t lda, int64_t n, const double *omega,
                          int64_t ldo, double *y, int64_t ldy, int d, h2_stream_t s);

/* Convergence statistic of Sec. III-B for `count` panels: mindiag[i] =
 * min_j |R_jj| of the Householder QR of panel i (m[i] x d[i], column-major at
 * panels + off[i], ld = m[i]); panels with m[i] <= d[i] get 0. Device arrays. */
h2_status h2_batched_qr_mindiag(int count, const int32_t *m, const int32_t *d, const int64_t *off,
                                const double *panels, double *mindiag, h2_stream_t s);

/* Row ID of `count` sample panels Y (m[i] x d[i], column-major at
 * panels + off[i], ld = m[i]) at absolute thresholds eps[i] (Sec. II-B):
 * column-pivoted Householder QR of Y^T/sqrt(d[i]) with norms recomputed every
 * step, stopping at the first k whose trailing block has Frobenius norm
 * <= eps[i] (or k = min(m, d)).  Outputs (device): k[i]; the sorted skeleton
 * rows J at J + i*ldj (ldj >= max m); the interpolation basis at
 * basis + eoff[i] as an m[i] x k[i] column-major matrix with E(J,:) = I and
 * E(R,:) = T^T (the caller reserves m[i]*min(m[i],d[i]) doubles). */
h2_status h2_batched_row_id(int count, const int32_t *m, const int32_t *d, const int64_t *off,
                            const double *panels, const double *eps, int32_t *k, int32_t *J,
                            int ldj, const int64_t *eoff, double *basis, h2_stream_t s);

/* Same statistic as h2_batched_qr_mindiag, for callers that cannot allocate
 * device memory: code that runs while another component owns the device's
 * memory (a custom or pre-reserving allocator, an allocation callback, a
 * memory-capped service), where a cudaMalloc would fail, deadlock or break a
 * budget.  This entry point allocates nothing; the paper has no counterpart.
 * Arguments are those of h2_batched_qr_mindiag and stay owned by the caller.
 *
 * Working copies of the panels that need a QR (m[i] > d[i]) go to one fixed
 * workspace compiled into the library: 2097152 doubles (16 MiB), present on
 * every device that loads the library until the process exits.  Its front
 * holds a table of count + 1 panel offsets (rounded up to 32 doubles).  If the
 * table and the sum of m[i]*d[i] over those panels exceed it, the call returns
 * H2_ERR_ARG and the panels that did not fit get NaN.  A panel with m[i] < 0 or
 * d[i] < 1 gets NaN and the call returns H2_ERR_ARG (checked on the device,
 * since m and d are device arrays).
 * The first call on a device looks up the workspace's device address (once
 * per device and CUDA context, with that device current).  All calls share
 * the one workspace and it keeps the last call's contents: calls that overlap
 * on the GPU (other streams, other host threads) race with each other.  The
 * call reads its status flag back and waits for its stream to finish before
 * it returns, so it cannot be recorded into a CUDA graph (stream capture). */
h2_status h2_batched_qr_mindiag_static(int count, const int32_t *m, const int32_t *d,
                                       const int64_t *off, const double *panels,
                                       double *mindiag, h2_stream_t s);

/* Measured throughput of one arithmetic pipe of the current device, for the
 * roofline fractions: which = 0 FP64 FMA (TFLOP/s), 1 FP32 FMA (TFLOP/s),
 * 2 exp2 on the special-function units (G operations/s), 3 dense tcgen05
 * products of FP16 operands with FP32 accumulation (TFLOP/s), 4 the same with
 * TF32 operands (TFLOP/s), 5 square root and 6 reciprocal square root on the
 * special-function units (G operations/s).  Each probe runs a fixed amount of independent work
 * on every SM (tens of milliseconds in all) and reports the best of five
 * timed launches.  Not part of the construction. */
h2_status h2_measure_peak(int which, h2_stream_t stream, double *value);

/* Failure-detection self-test of the tensor-core sketch: one small launch in
 * which the producer warp withholds the first tile, so the waits of the
 * other warps run out (0.2 s bound each), followed by a normal launch of the
 * same problem.  Returns H2_OK when the stalled launch reported
 * H2_ERR_TIMEOUT and the normal one then completed; otherwise the status
 * that went wrong.  Not part of the construction. */
h2_status h2_selftest_wait_timeout(h2_stream_t stream);

/* The library keeps device blocks it freed for reuse (size buckets per
 * device), so repeated builds avoid cudaMalloc/cudaFree; this synchronises
 * the devices and returns those cached blocks to CUDA.  Handles stay valid. */
void h2_trim_memory(void);

/* CUDA kernels the library has launched from the calling host thread so far
 * (all entry points); a profiling aid. */
int64_t h2_kernel_launches(void);

/* Device blocks the library has requested from its allocator so far (all
 * threads; every request counts, whether its cache or cudaMalloc served it).
 * An entry point that allocates nothing leaves it unchanged. */
int64_t h2_device_allocations(void);

const char *h2_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* H2GB_H */
