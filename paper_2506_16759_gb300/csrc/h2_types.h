// Host-side handle layouts shared by the library's translation units.
#pragma once

#include <memory>
#include <vector>

#include "h2_internal.cuh"

struct h2_tree {
  int64_t n = 0;
  int dim = 0;
  int leaf_size = 0;
  double eta = 0.0;
  int depth = 0;      // leaf depth L
  int n_nodes = 0;    // 2^(L+1) - 1
  int l_top = 0;      // highest paper level with an admissible pair
  // tree-ordered coordinates (dim < 3 padded with zeros)
  h2::DBuf<double> x, y, z;
  h2::DBuf<int32_t> perm;   // tree position -> original index
  h2::DBuf<int32_t> iperm;  // original index -> tree position
  std::vector<int64_t> h_begin, h_end;  // per node, host copy
  h2::DBuf<int64_t> begin, end;         // per node, device
  h2::DBuf<double> lo, hi;              // per node boxes, [3][n_nodes]
  h2::DBuf<double> diam;                // per node box diagonal
  // far list per depth: CSR over the nodes of that depth (cols: heap ids)
  std::vector<h2::DBuf<int64_t>> far_ptr;
  std::vector<h2::DBuf<int32_t>> far_idx;
  std::vector<int64_t> far_nnz;
  // near list at the leaf depth
  h2::DBuf<int64_t> near_ptr;
  h2::DBuf<int32_t> near_idx;
  int64_t near_nnz = 0;
};

namespace h2 {

// Exclusive scan of n int64 values on the device (one CTA); writes the total
// to out[n] (out has n+1 entries).
void scan_exclusive(const int64_t *in, int64_t *out, int64_t n, cudaStream_t s);
void scan_exclusive_i32(const int32_t *in, int64_t *out, int64_t n, cudaStream_t s);

// KD tree and block lists (tree.cu); throws h2::Error.
void build_tree(const double *pts, int64_t n, int dim, int leaf, double eta, cudaStream_t s,
                h2_tree *t);

}  // namespace h2
