// Per-level launch interfaces of the construction (Algorithm 1) and the
// H2 matrix-vector product.  Device pointers unless stated otherwise.
#pragma once

#include "h2_ops.h"

namespace h2 {

// Clusters of one paper level across all instances ("tasks").  Rows of the
// level panel: at level 1 the global tree positions of the leaf's points; at
// level l > 1 the concatenated skeleton rows of the two children.
struct TasksDev {
  int n;                  // tasks
  const int32_t *inst;    // task -> instance
  const int32_t *m;       // rows of the task
  const int64_t *row;     // first row in the level panel
  const int32_t *k;       // rank after the ID
  const int64_t *krow;    // first row of the task's skeletons in the next level
  const int32_t *J;       // sorted local skeleton rows, at krow
  const int64_t *eoff;    // basis offset (m x k column-major)
};

// Per-instance column range [cb, ce) of the current pass and other
// per-instance scalars.
struct InstCols {
  const int32_t *cb;
  const int32_t *ce;
};

// Block-sparse row product: out(rows of task t) += sign * sum_e Blk_e * in(rows of col task)
struct BsrArgs {
  int n_rows;               // row tasks
  const int32_t *row_inst;  // row task -> instance
  const int32_t *row_m;     // rows of each row task
  const int64_t *row_off;   // output row offset of each row task
  const int32_t *col_m;     // columns of each column task (block width)
  const int64_t *col_off;   // input row offset of each column task
  const int64_t *ptr;       // CSR over row tasks
  const int32_t *idx;       // column task of each entry
  const int64_t *boff;      // block offset of each entry (row_m x col_m, column-major)
  const void *blocks;       // T
  const void *in;           // T panel
  int64_t ld_in;
  void *out;                // T panel
  int64_t ld_out;
  double sign;
  InstCols cols;
  int64_t in_rows;          // rows of the input panel (FP32 tiled path)
  int col_hi;               // max over instances of ce (0: use the row-block kernel)
  int seg = 1;              // CTAs per row task (set by bsr_apply; > 1: atomic adds)
  int engine = 0;           // FP32: 0 tensor cores where blocks have <= 256 rows, 1 CUDA cores
};
// max_cols: the widest per-instance column range of this call.
void bsr_apply(bool fp64, const BsrArgs &a, int max_m, int max_cols, cudaStream_t s);
// FP32 blocks of at most 256 rows on the tensor cores (bsr_tc.cu); false if
// the call is outside that range.
bool bsr_apply_tc(const BsrArgs &a, int max_m, int max_cols, cudaStream_t s);

// Leaf near field: every D_{t,b} = K(I_t, I_b) of the near list, stored at
// doff (16-byte aligned offsets).
struct DgenArgs {
  int64_t nnz;
  const int32_t *erow;      // row task of each near entry
  const int32_t *idx;       // column task of each near entry
  const int64_t *doff;
  const int32_t *m;         // rows of each leaf task
  const int64_t *row;       // first global tree position of each leaf task
  const int32_t *tinst;     // instance of each task
  const InstDev *inst;
  Points64 p64;
  Points32 p32;
  void *D;                  // T
  int n_rows;               // leaf tasks (rows of the near CSR)
  const int64_t *ptr;       // near CSR over the leaf tasks
};
void dense_blocks_gen(int kid, bool fp64, const DgenArgs &a, cudaStream_t s);

// QR convergence test of Sec. III-B on each active unconverged task.
struct QrArgs {
  TasksDev t;
  const void *Y;            // T panel (level l)
  int64_t ld;
  const int32_t *dcur;      // per instance: current sample count
  const double *eps;        // per instance: eps_l
  const int32_t *active;    // per instance: 1 if the level is compressed
  int32_t *conv;            // per task flag (in/out)
  int32_t *unconv;          // per instance counter (out, accumulated)
  double *ws;               // global workspace for panels too large for smem
  const int64_t *ws_off;    // per task offset into ws, -1 = shared memory
  double *mindiag;          // optional per task output (may be NULL)
  // work queue (both NULL: one CTA per task in task order): the order in which
  // the tasks are taken, and a device counter the launcher zeroes
  const int32_t *queue = nullptr;
  int32_t *next = nullptr;
};
// width: the widest cluster of the call (threads = columns), 0 = 256 threads.
void qr_test(bool fp64, const QrArgs &a, size_t smem_bytes, int width, cudaStream_t s);

// Row ID (batchedID) of each active task: CPQR of Y^T/sqrt(d).
struct IdArgs {
  TasksDev t;
  const void *Y;            // T panel
  int64_t ld;
  const int32_t *dcur;
  const double *eps;
  const int32_t *active;
  const int32_t *ibar;      // candidate rows -> global tree position (NULL at level 1)
  int32_t *k_out;           // per task rank
  int32_t *J_tmp;           // sorted skeleton rows at the task's row offset
  int32_t *skel_tmp;        // skeleton global positions at the task's row offset
  const int64_t *eoff;
  double *E;                // bases (m x k at eoff)
  double *ws;
  const int64_t *ws_off;
  int mcap;                 // rows the per-cluster index arrays hold (>= every m, <= 512)
  const int32_t *queue = nullptr;   // work queue, as in QrArgs
  int32_t *next = nullptr;
};
void row_id(bool fp64, const IdArgs &a, size_t smem_bytes, int width, cudaStream_t s);
// Shared memory the ID kernel needs besides the d x m panel (clusters of at
// most mcap rows).
size_t row_id_fixed_smem(int mcap);

// Moves the per-task skeleton arrays from row offsets to krow offsets.
void compact_skeletons(const TasksDev &t, const int32_t *J_tmp, const int32_t *skel_tmp,
                       int32_t *J, int32_t *skel, cudaStream_t s);

// Rows of the next level: Ynext(krow+a, c) = Y(row + J[a], c).
void gather_skeleton_rows(bool fp64, const TasksDev &t, const void *Y, int64_t ld, void *Ynext,
                          int64_t ldn, InstCols cols, const int32_t *active, cudaStream_t s);
// out(krow+a, c) = sum_i E(i,a) in(row+i, c)       (E^T products: upsweep)
// E is FP64 in both modes: FP64 sums, or (mixed precision) converted to FP32
// on load with FP32 sums.
void basis_t_apply(bool fp64, const TasksDev &t, const void *E, const void *in, int64_t ld_in,
                   void *out, int64_t ld_out, InstCols cols, const int32_t *active, int max_m,
                   int max_k, cudaStream_t s);
// out(row+i, c) += sum_a E(i,a) in(krow+a, c)      (E products: downsweep)
void basis_n_apply(bool fp64, const TasksDev &t, const void *E, const void *in, int64_t ld_in,
                   void *out, int64_t ld_out, InstCols cols, int max_m, int max_k,
                   cudaStream_t s);

// Couplings B(e) = K(Itil_row, Itil_col) for each far entry e.
struct CouplingArgs {
  int64_t nnz;
  const int32_t *erow;      // row task of each entry
  const int32_t *idx;       // column task of each entry
  const int64_t *boff;
  TasksDev t;
  const int32_t *skel;      // compacted skeleton global positions (at krow)
  const InstDev *inst;
  Points64 p64;
  Points32 p32;
  void *B;
  const int64_t *ptr;       // far CSR over the level's tasks (t.n rows)
  // column tasks' ranks, skeleton offsets and skeletons when they differ from
  // the rows' (separate row and column bases); NULL = the rows'
  const int32_t *col_k = nullptr;
  const int64_t *col_krow = nullptr;
  const int32_t *col_skel = nullptr;
};
void coupling_gen(int kid, bool fp64, const CouplingArgs &a, cudaStream_t s);

// Sizes of blocks for offset scans: out[e] = rows(row task) * cols(col task),
// rounded up to a multiple of `align` elements (16-byte aligned blocks).
void block_sizes(int64_t nnz, const int32_t *erow, const int32_t *idx, const int32_t *mrow,
                 const int32_t *mcol, int align, int64_t *out, cudaStream_t s);

// Inner-level task geometry: row[t] = krow_child[c0], m[t] = k[c0] + k[c0+1].
void inner_tasks(int n, const int32_t *child0, const int64_t *krow_child,
                 const int32_t *k_child, int64_t *row, int32_t *m, cudaStream_t s);

// Per-task m*min(m,d) sizes (basis capacity) and eoff scan helper.
void basis_capacity(int n, const int32_t *m, const int32_t *inst, const int32_t *dcur,
                    int64_t *cap, cudaStream_t s);

// CSR of one instance's list (rows: nodes first..first+nrows-1, cols: heap
// ids) appended to a level CSR with task indices.
void map_csr(const int64_t *ptr, const int32_t *idx, int nrows, int first_node, int task_base,
             int64_t nnz_base, int64_t *ptr_out, int32_t *idx_out, int32_t *erow_out,
             bool write_last, cudaStream_t s);

// x (original order, ld_x) -> xt (tree order, T) and back.
void permute_in(bool fp64, const double *x, int64_t ldx, const int32_t *orig_of_pos, int64_t n,
                int nrhs, void *xt, int64_t ldt, cudaStream_t s);
void permute_out(bool fp64, const void *yt, int64_t ldt, const int32_t *orig_of_pos, int64_t n,
                 int nrhs, double *y, int64_t ldy, cudaStream_t s);

void fill_i32(int32_t *p, int64_t n, int32_t v, cudaStream_t s);

// ---- entries of a sum of H2 matrices (h2sum.cu)
// One FP64 operand at one level: its ranks, G = U_op(Itil, :) blocks of the
// target's clusters (k_target x k_op at goff), its couplings.
struct SumOperand {
  const int32_t *k;      // operand ranks of the level's tasks
  const int64_t *goff;   // G offsets per task
  const double *G;
  const int64_t *boff;   // operand coupling offsets per far entry
  const double *B;       // FP64 operand couplings, or
  const float *B32;      // FP32 ones (an operand built in mixed precision)
};
struct SumCouplingArgs {
  int64_t nnz;
  const int32_t *erow;
  const int32_t *idx;
  const int64_t *boff;   // target coupling offsets
  TasksDev t;            // target tasks (ranks)
  void *B;               // target couplings (T)
  const SumOperand *ops; // device array
  int nops;
};
void h2sum_g_leaf(const TasksDev &t, const int32_t *kop, const int64_t *eoff_op, const double *Eop,
                  const int64_t *goff, double *G, cudaStream_t s);
void h2sum_g_inner(const TasksDev &t, const int32_t *child0, const int32_t *kt_child,
                   const int32_t *kop_child, const int64_t *goff_child, const double *Gchild,
                   const int32_t *kop, const int32_t *mop, const int64_t *eoff_op,
                   const double *Eop, const int64_t *goff, double *G, cudaStream_t s);
// engine (mixed precision): 0 CUDA cores, 1 tensor cores where target ranks are <= 96.
void h2sum_couplings(bool fp64, const SumCouplingArgs &a, int max_kop, int max_kt, int engine,
                     cudaStream_t s);
void h2sum_dense(bool fp64, int64_t nnz, const int32_t *erow, const int32_t *idx, const int32_t *m,
                 const int64_t *doff, void *D, const double *const *Dop, const float *const *Dop32,
                 const int64_t *const *doff_op, int nops, cudaStream_t s);

// ---- low-rank term U V^T of the operator (lowrank.cu)
// Tree-order row-major copy out[p * r + k] = src[orig[p] + k * ld] (T by fp64).
void lowrank_tree_rows(bool fp64, const double *src, int64_t ld, const int32_t *orig, int64_t n,
                       int r, void *out, cudaStream_t s);
// y(:, 0:nc) += U (V^T om(:, 0:nc)), all FP64 column-major in original order
// (U, V with leading dimension ld).
void lowrank_sample(const double *U, const double *V, int64_t ld, int64_t n, int r,
                    const double *om, int64_t ldo, int nc, double *y, int64_t ldy,
                    cudaStream_t s);
// Every block e of the CSR (rows n_rows tasks) += U(rows) V(cols)^T, the rows
// of a task being its points (row0) or its skeleton points (skel at krow).
// cols_of / ckrow / cskel: the column tasks' ranks and skeletons when they
// differ from the rows' (separate row and column bases); NULL = the rows'.
void lowrank_blocks(bool fp64, bool skel_rows, int n_rows, const int64_t *ptr, const int32_t *idx,
                    const int64_t *off, const int32_t *rows_of, const int64_t *row0,
                    const int64_t *krow, const int32_t *skel, const void *Ut, const void *Vt,
                    int r, void *out, cudaStream_t s, const int32_t *cols_of = nullptr,
                    const int64_t *ckrow = nullptr, const int32_t *cskel = nullptr);

}  // namespace h2
