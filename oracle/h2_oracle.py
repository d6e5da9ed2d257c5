"""FP64 CPU oracle for bottom-up adaptive-sketching H2 construction.

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA library is checked against.  Only the tests, the smoke check and the
bench's CPU-baseline leg may import it; the library itself never does.  It
shares no code with the CUDA path.

It follows Boukaram, Liu, Ghysels, Li, "Adaptive Sketching Based
Construction of H2 Matrices on GPUs" (arXiv 2506.16759):

* cluster tree and general admissibility, Sec. II-A (the adm equation) and
  the dual tree traversal described right after it;
* the interpolative decomposition via column-pivoted QR, Sec. II-B;
* Algorithm 1 (fixed-sample form, Sec. III-A) with the adaptive convergence
  loop of Sec. III-B;
* the H2 matrix-vector product used as a sketching operator, Sec. V-A;
* the error measures of Sec. V-A.

Where the paper is silent the oracle takes these readings (each one is also
listed in the design notes of the repository):

* KD split: the longest side of the node's tight bounding box (lowest
  dimension on ties); points ordered by (coordinate, point index); the left
  child receives the first ceil(n/2) points; uniform leaf depth L, the
  smallest L with ceil(N/2^L) <= leaf size.
* Boxes are tight; D(s) is the box diagonal; Dist(s,t) is the Euclidean gap
  between boxes; a pair is admissible iff Dist>0 and (D(s)+D(t))/2 <= eta Dist.
* nrmK = ||Y||_F / sqrt(d0) from the first sketch; eps_abs = tol * nrmK;
  per-level threshold eps_l = eps_abs / sqrt(2 * l_top * n_l), a Frobenius
  budget spread over the l_top compressed levels, the n_l nodes of level l and
  the two sides of every admissible block: the same bases act on rows and
  columns, and A - P A P = (I - P) A + P A (I - P) splits into two parts that
  are orthogonal in the Frobenius inner product (the "simple error
  compensation" of Sec. V-B is left unspecified by the paper).
* Convergence of node tau: m_tau <= d, or min_j |R_jj| <= eps_l where R is the
  triangular factor of an unpivoted Householder QR of Y_loc (m x d).
* Row ID: column-pivoted Householder QR of A = Y_loc^T / sqrt(d) with column
  norms recomputed at every step, pivot = largest norm (lowest index on
  ties); stop at the first k whose trailing block has Frobenius norm <= eps_l
  (or k = min(d, m)).  T = R11^{-1} R12.  Skeleton indices J are stored in
  ascending order; U(J,:) = I and U(R,:) = T^T with columns following J.
* Samples for the adaptive rounds are the next d_inc columns of one stored
  Gaussian matrix Omega (N x d_max, original point order).
* The matrix is real and symmetric, so the column basis equals the row basis.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

K_EXP, K_MATERN32, K_GAUSS, K_LAPLACE_IE, K_POLY, K_HELMHOLTZ_IE = 0, 1, 2, 3, 4, 6

# -----------------------------------------------------------------------------
# Matrix entries  (Sec. V-A test problems: exponential covariance and the
# Helmholtz volume-IE kernel, plus the kernels of the synthetic workloads)
# -----------------------------------------------------------------------------


def kernel_block(kernel: int, params, Xa: np.ndarray, Xb: np.ndarray,
                 ia: np.ndarray, ib: np.ndarray) -> np.ndarray:
    """K(ia, ib) for points Xa = X[ia], Xb = X[ib]; ia/ib are point indices.

    The diagonal terms (nugget, IE self-integral) apply where the two point
    indices are equal.
    """
    Xa = np.asarray(Xa, dtype=np.float64)
    Xb = np.asarray(Xb, dtype=np.float64)
    same = np.asarray(ia)[:, None] == np.asarray(ib)[None, :]
    dim = Xa.shape[1]
    if kernel == K_POLY:
        c, p = float(params[0]), int(params[1])
        g = np.zeros((Xa.shape[0], Xb.shape[0]))
        for k in range(dim):
            g = g + Xa[:, k, None] * Xb[None, :, k]
        return (c + g) ** p
    r2 = np.zeros((Xa.shape[0], Xb.shape[0]))
    for k in range(dim):
        diff = Xa[:, k, None] - Xb[None, :, k]
        r2 = r2 + diff * diff
    r = np.sqrt(r2)
    if kernel == K_EXP:
        ell, nugget = params
        return np.exp(-r / ell) + nugget * same
    if kernel == K_MATERN32:
        ell, nugget = params
        a = math.sqrt(3.0) * r / ell
        return (1.0 + a) * np.exp(-a) + nugget * same
    if kernel == K_GAUSS:
        sigma, nugget = params
        return np.exp(-r2 / (2.0 * sigma * sigma)) + nugget * same
    if kernel == K_LAPLACE_IE:
        (diag,) = params
        with np.errstate(divide="ignore"):
            off = 1.0 / (4.0 * math.pi * r)
        return np.where(same, diag, off)
    if kernel == K_HELMHOLTZ_IE:
        # Sec. V-A: cos(k|x-y|)/|x-y| for x != y; the diagonal is a parameter
        wave = float(params[0])
        diag = float(params[1]) if len(params) > 1 else 0.0
        with np.errstate(divide="ignore", invalid="ignore"):
            off = np.cos(wave * r) / r
        return np.where(same, diag, off)
    raise ValueError(f"unknown kernel {kernel}")


# -----------------------------------------------------------------------------
# Cluster tree (Sec. II-A; KD-tree of Sec. V-A)
# -----------------------------------------------------------------------------


@dataclass
class ClusterTree:
    X: np.ndarray            # (N, dim) points, original order
    leaf_size: int
    depth: int               # leaf depth L (root at depth 0)
    perm: np.ndarray         # tree position -> original point index
    begin: np.ndarray        # per heap node: first tree position
    end: np.ndarray          # per heap node: one past the last tree position
    lo: np.ndarray           # per heap node: tight box lower corner (n_nodes, dim)
    hi: np.ndarray           # per heap node: tight box upper corner
    split_dim: np.ndarray    # per inner node: the dimension it was split on

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def n_nodes(self) -> int:
        return 2 ** (self.depth + 1) - 1

    def nodes_at_depth(self, k: int) -> range:
        return range(2 ** k - 1, 2 ** (k + 1) - 1)

    def level_depth(self, level: int) -> int:
        """Paper level l (1 = leaves) -> tree depth."""
        return self.depth - level + 1

    def Xt(self) -> np.ndarray:
        """Points in tree order (formed once: a per-block permutation would make
        the construction quadratic in N)."""
        xt = self.__dict__.get("_xt")
        if xt is None:
            xt = self.X[self.perm]
            self.__dict__["_xt"] = xt
        return xt


def leaf_depth(n: int, leaf_size: int) -> int:
    L = 0
    while -(-n // (2 ** L)) > leaf_size:
        L += 1
    return L


def build_cluster_tree(X: np.ndarray, leaf_size: int) -> ClusterTree:
    """KD median bisection to a uniform leaf depth."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, dim = X.shape
    if n < 1 or leaf_size < 2:
        raise ValueError("need n >= 1 and leaf_size >= 2")
    L = leaf_depth(n, leaf_size)
    n_nodes = 2 ** (L + 1) - 1
    members: list = [None] * n_nodes
    members[0] = np.arange(n, dtype=np.int64)
    lo = np.zeros((n_nodes, dim))
    hi = np.zeros((n_nodes, dim))
    split = np.full(n_nodes, -1, dtype=np.int64)
    for node in range(n_nodes):
        P = members[node]
        lo[node] = X[P].min(axis=0)
        hi[node] = X[P].max(axis=0)
        if 2 * node + 1 >= n_nodes:
            continue
        extent = hi[node] - lo[node]
        s = int(np.argmax(extent))            # first maximum: lowest dim on ties
        order = np.lexsort((P, X[P, s]))      # by coordinate, then point index
        P = P[order]
        n_left = -(-len(P) // 2)
        members[2 * node + 1] = P[:n_left]
        members[2 * node + 2] = P[n_left:]
        split[node] = s
    first_leaf = 2 ** L - 1
    perm = np.concatenate([members[v] for v in range(first_leaf, n_nodes)])
    begin = np.zeros(n_nodes, dtype=np.int64)
    end = np.zeros(n_nodes, dtype=np.int64)
    pos = 0
    for v in range(first_leaf, n_nodes):
        begin[v] = pos
        pos += len(members[v])
        end[v] = pos
    for v in range(first_leaf - 1, -1, -1):
        begin[v] = begin[2 * v + 1]
        end[v] = end[2 * v + 2]
    return ClusterTree(X, leaf_size, L, perm, begin, end, lo, hi, split)


def box_diameter(lo, hi) -> float:
    """D(s): length of the box diagonal, summed in dimension order."""
    acc = 0.0
    for k in range(len(lo)):
        e = float(hi[k]) - float(lo[k])
        acc = acc + e * e
    return math.sqrt(acc)


def box_distance(lo_s, hi_s, lo_t, hi_t) -> float:
    """Dist(s,t): Euclidean gap between two axis-aligned boxes."""
    acc = 0.0
    for k in range(len(lo_s)):
        g = max(0.0, float(lo_t[k]) - float(hi_s[k]), float(lo_s[k]) - float(hi_t[k]))
        acc = acc + g * g
    return math.sqrt(acc)


def admissible(tree: ClusterTree, s: int, t: int, eta: float) -> bool:
    """General admissibility (D(s)+D(t))/2 <= eta Dist(s,t), with Dist > 0."""
    Ds = box_diameter(tree.lo[s], tree.hi[s])
    Dt = box_diameter(tree.lo[t], tree.hi[t])
    dist = box_distance(tree.lo[s], tree.hi[s], tree.lo[t], tree.hi[t])
    return dist > 0.0 and 0.5 * (Ds + Dt) <= eta * dist


@dataclass
class BlockLists:
    far: list     # far[depth]: dict node -> sorted list of admissible partners (F)
    near: dict    # leaf -> sorted list of inadmissible partners (N), self included


def dual_traversal(tree: ClusterTree, eta: float) -> BlockLists:
    """Dual tree traversal from (root, root): admissible pairs become F
    entries, inadmissible leaf pairs become N entries, other inadmissible pairs
    recurse on their four child pairs."""
    far = [dict() for _ in range(tree.depth + 1)]
    near = {}
    frontier = [(0, 0)]
    for k in range(tree.depth + 1):
        nxt = []
        for s, t in frontier:
            if admissible(tree, s, t, eta):
                far[k].setdefault(s, []).append(t)
            elif k == tree.depth:
                near.setdefault(s, []).append(t)
            else:
                for si in (2 * s + 1, 2 * s + 2):
                    for tj in (2 * t + 1, 2 * t + 2):
                        nxt.append((si, tj))
        frontier = nxt
    for k in range(tree.depth + 1):
        for s in far[k]:
            far[k][s].sort()
    for s in near:
        near[s].sort()
    return BlockLists(far, near)


def top_level(tree: ClusterTree, lists: BlockLists) -> int:
    """l_top: the highest paper level with at least one admissible pair."""
    lt = 0
    for level in range(1, tree.depth + 2):
        if lists.far[tree.level_depth(level)]:
            lt = level
    return lt


# -----------------------------------------------------------------------------
# Dense kernels of the construction (Sec. II-B, Sec. III-B)
# -----------------------------------------------------------------------------


def qr_min_abs_diag(Y: np.ndarray) -> float:
    """min_j |R_jj| of the Householder QR of Y (m x d, m > d), Sec. III-B."""
    R = np.linalg.qr(Y, mode="r")
    return float(np.min(np.abs(np.diag(R))))


def node_converged(Yloc: np.ndarray, eps_l: float) -> bool:
    m, d = Yloc.shape
    if m <= d:
        return True
    return qr_min_abs_diag(Yloc) <= eps_l


@dataclass
class RowID:
    k: int
    J: np.ndarray        # sorted skeleton rows (local indices)
    U: np.ndarray        # (m, k) interpolation basis, U[J,:] = I
    pivots: np.ndarray   # pivot order chosen by the CPQR (local indices)
    T: np.ndarray        # (k, m-k) interpolation matrix in pivot order


def cpqr_column_id(A: np.ndarray, eps: float) -> tuple:
    """Column ID of A (Sec. II-B) by Householder QR with column pivoting.

    Norms of the remaining columns are recomputed at every step.  Stops at the
    first k with ||trailing block||_F <= eps, or k = min(rows, cols).
    Returns (k, pivots, T) with A[:, piv[k:]] ~= A[:, piv[:k]] @ T.
    """
    A = np.array(A, dtype=np.float64, copy=True)
    rows, cols = A.shape
    piv = np.arange(cols)
    kmax = min(rows, cols)
    k = 0
    while k < kmax:
        sub = A[k:, k:]
        norms = np.sqrt(np.sum(sub * sub, axis=0))
        if math.sqrt(float(np.sum(norms * norms))) <= eps:
            break
        j = k + int(np.argmax(norms))          # first maximum -> lowest index
        if j != k:
            A[:, [k, j]] = A[:, [j, k]]
            piv[[k, j]] = piv[[j, k]]
        x = A[k:, k].copy()
        alpha = -math.copysign(np.linalg.norm(x), x[0]) if x[0] != 0 else -np.linalg.norm(x)
        v = x
        v[0] = x[0] - alpha
        vnorm2 = float(v @ v)
        if vnorm2 > 0.0:
            beta = 2.0 / vnorm2
            A[k:, k:] -= beta * np.outer(v, v @ A[k:, k:])
        A[k, k] = alpha
        A[k + 1:, k] = 0.0
        k += 1
    R11 = A[:k, :k]
    R12 = A[:k, k:]
    if k > 0:
        import scipy.linalg
        T = scipy.linalg.solve_triangular(R11, R12, lower=False)
    else:
        T = np.zeros((0, cols))
    return k, piv, T


def row_id(Yloc: np.ndarray, eps_l: float) -> RowID:
    """Row ID of the samples: column ID of Y_loc^T / sqrt(d) (Sec. II-B)."""
    m, d = Yloc.shape
    A = Yloc.T / math.sqrt(d) if d > 0 else Yloc.T
    k, piv, T = cpqr_column_id(A, eps_l)
    S = piv[:k]
    Rd = piv[k:]
    order = np.argsort(S, kind="stable")
    J = S[order]
    U = np.zeros((m, k))
    U[J, np.arange(k)] = 1.0
    if k > 0 and len(Rd) > 0:
        U[Rd, :] = T[order, :].T
    return RowID(k, J, U, piv, T)


# -----------------------------------------------------------------------------
# Algorithm 1: bottom-up construction with adaptive sampling
# -----------------------------------------------------------------------------


@dataclass
class NodeData:
    m: int = 0
    Ibar: np.ndarray = None     # candidate rows as tree positions
    k: int = 0
    J: np.ndarray = None        # sorted local skeleton rows
    U: np.ndarray = None        # (m, k): leaf basis U or transfer [E_1; E_2]
    Itil: np.ndarray = None     # skeleton rows as tree positions
    Yloc: np.ndarray = None     # (m, d) local samples used by the ID
    Om: np.ndarray = None       # (m, d) Omega^l for the node
    Yhat: np.ndarray = None     # (k, d) Y^{l+1} rows of the node
    Omhat: np.ndarray = None    # (k, d) Omega^{l+1} rows of the node
    converged_d: int = 0


@dataclass
class H2Oracle:
    tree: ClusterTree
    lists: BlockLists
    kernel: int
    params: tuple
    tol: float
    l_top: int
    nodes: dict                 # heap id -> NodeData (levels 1..l_top)
    D: dict                     # (s, t) leaf pair -> dense block
    B: dict                     # (s, t) admissible pair -> coupling block
    d_final: int
    nrmK: float
    eps_abs: float
    eps_level: dict             # level -> eps_l
    d_level: dict               # level -> samples used by its ID
    converged: bool
    timings: dict = field(default_factory=dict)

    def rank(self, node: int) -> int:
        return self.nodes[node].k


def _entries(tree: ClusterTree, kernel, params, Ia, Ib) -> np.ndarray:
    """K(Ia, Ib) for tree positions Ia, Ib.  `kernel` is a kernel id, or a
    callable f(Ia, Ib) giving the entries of an operator in tree order (the
    entry function of Algorithm 1 for operators such as sums of H2 matrices)."""
    if callable(kernel):
        return np.asarray(kernel(np.asarray(Ia), np.asarray(Ib)), dtype=np.float64)
    Xt = tree.Xt()
    return kernel_block(kernel, params, Xt[Ia], Xt[Ib], np.asarray(Ia), np.asarray(Ib))


class _Builder:
    """State of one run of Algorithm 1."""

    def __init__(self, tree, lists, kernel, params, tol, omega, d0, d_inc, d_max, sampler):
        self.tree, self.lists = tree, lists
        self.kernel, self.params, self.tol = kernel, params, tol
        self.omega = np.asarray(omega, dtype=np.float64)      # (N, >= d_max), original order
        self.d0, self.d_inc, self.d_max = d0, d_inc, d_max
        self.sampler = sampler
        self.nodes = {}
        self.D = {}
        self.B = {}
        self.l_top = top_level(tree, lists)
        self.eps_level = {}
        self.d_level = {}
        self.converged = True
        self.t_sketch = 0.0

    # -- helpers -------------------------------------------------------------
    def sample(self, c0: int, c1: int):
        """Y = K Omega[:, c0:c1] in tree order, with that Omega in tree order."""
        om = np.ascontiguousarray(self.omega[:, c0:c1])
        t0 = time.perf_counter()
        Y = self.sampler(om)
        self.t_sketch += time.perf_counter() - t0
        perm = self.tree.perm
        return np.asarray(Y)[perm], om[perm]

    def level_nodes(self, level):
        return self.tree.nodes_at_depth(self.tree.level_depth(level))

    def far(self, level, node):
        return self.lists.far[self.tree.level_depth(level)].get(node, [])

    # -- one level for a block of sample columns ----------------------------
    def local_samples(self, level, Yt, Ot, below):
        """Y_loc and Omega^l of every node of `level` for one column block.

        Yt/Ot: sketch and Omega of the block in tree order.  `below` holds, per
        node of level-1, the (Yhat, Omhat) of the same block (None at leaves).
        Leaf level: Y_loc = Y(I_tau) - sum_{b in N_tau} D_{tau,b} Omega(I_b).
        Inner level: Y_loc = [Yhat_1; Yhat_2] - [sum_{F_1} B Omhat_b; sum_{F_2} ...].
        """
        tree = self.tree
        out = {}
        for tau in self.level_nodes(level):
            if level == 1:
                rows = np.arange(tree.begin[tau], tree.end[tau])
                Y = Yt[rows].copy()
                for b in self.lists.near.get(tau, []):
                    cols = np.arange(tree.begin[b], tree.end[b])
                    Y -= self.D[(tau, b)] @ Ot[cols]
                out[tau] = (Y, Ot[rows].copy())
            else:
                parts_y, parts_o = [], []
                for nu in (2 * tau + 1, 2 * tau + 2):
                    Yhat, Omhat = below[nu]
                    Ysub = Yhat.copy()
                    for b in self.far(level - 1, nu):
                        Ysub -= self.B[(nu, b)] @ below[b][1]
                    parts_y.append(Ysub)
                    parts_o.append(Omhat)
                out[tau] = (np.vstack(parts_y), np.vstack(parts_o))
        return out

    def skeleton_rows(self, nd):
        """Itil_tau = Ibar_tau(J_tau): skeleton rows as tree positions."""
        return nd.Ibar[nd.J]

    def upsweep(self, level, local):
        """Y^{l+1} = Y_loc(J,:) and Omega^{l+1} = U^T Omega^l for each node."""
        res = {}
        for tau, (Y, O) in local.items():
            nd = self.nodes[tau]
            res[tau] = (Y[nd.J, :], nd.U.T @ O)
        return res

    def sweep_new_columns(self, level, c0, c1):
        """updateSamples: push new columns c0:c1 from the leaves up to `level`."""
        Yt, Ot = self.sample(c0, c1)
        below = None
        for lv in range(1, level + 1):
            local = self.local_samples(lv, Yt, Ot, below)
            if lv == level:
                return local
            below = self.upsweep(lv, local)
        return None

    # -- the construction -------------------------------------------------------
    def run(self):
        tree = self.tree
        t_start = time.perf_counter()
        d = self.d0
        Yt, Ot = self.sample(0, d)
        # approximate ||K||_F from the first sketch (Sec. III-B)
        self.nrmK = float(np.linalg.norm(Yt) / math.sqrt(d))
        self.eps_abs = self.tol * self.nrmK
        # dense near-field blocks D_{tau,b} = K(I_tau, I_b)   (batchedGen, D)
        for tau in tree.nodes_at_depth(tree.depth):
            rows = np.arange(tree.begin[tau], tree.end[tau])
            for b in self.lists.near.get(tau, []):
                cols = np.arange(tree.begin[b], tree.end[b])
                self.D[(tau, b)] = _entries(tree, self.kernel, self.params, rows, cols)
        below = None
        for level in range(1, self.l_top + 1):
            nodes = list(self.level_nodes(level))
            eps_l = self.eps_abs / math.sqrt(2 * self.l_top * len(nodes))
            self.eps_level[level] = eps_l
            local = self.local_samples(level, Yt if level == 1 else None,
                                       Ot if level == 1 else None, below)
            for tau in nodes:
                nd = NodeData()
                Y, O = local[tau]
                nd.m = Y.shape[0]
                if level == 1:
                    nd.Ibar = np.arange(tree.begin[tau], tree.end[tau])
                else:
                    nd.Ibar = np.concatenate([self.nodes[2 * tau + 1].Itil,
                                              self.nodes[2 * tau + 2].Itil])
                nd.Yloc, nd.Om = Y, O
                self.nodes[tau] = nd
            # adaptive sampling: add d_inc columns until every node converges
            # (d_inc = 0: fixed sample count, no convergence test)
            while self.d_inc > 0:
                pending = [t for t in nodes if not node_converged(self.nodes[t].Yloc, eps_l)]
                if not pending:
                    break
                if d + self.d_inc > self.d_max:
                    self.converged = False
                    break
                new_local = self.sweep_new_columns(level, d, d + self.d_inc)
                # the lower levels keep their IDs; their panels just grow
                d += self.d_inc
                for tau in nodes:
                    Yn, On = new_local[tau]
                    nd = self.nodes[tau]
                    nd.Yloc = np.hstack([nd.Yloc, Yn])
                    nd.Om = np.hstack([nd.Om, On])
            self.d_level[level] = d
            # row ID of every node (batchedID), shrink and upsweep
            for tau in nodes:
                nd = self.nodes[tau]
                rid = row_id(nd.Yloc, eps_l)
                nd.k, nd.J, nd.U = rid.k, rid.J, rid.U
                nd.Itil = self.skeleton_rows(nd)
                nd.converged_d = d
            up = self.upsweep(level, {tau: (self.nodes[tau].Yloc, self.nodes[tau].Om)
                                      for tau in nodes})
            for tau in nodes:
                self.nodes[tau].Yhat, self.nodes[tau].Omhat = up[tau]
            # couplings B_{tau,b} = K(Itil_tau, Itil_b)   (batchedGen, B)
            for tau in nodes:
                for b in self.far(level, tau):
                    self.B[(tau, b)] = _entries(tree, self.kernel, self.params,
                                                self.nodes[tau].Itil, self.nodes[b].Itil)
            below = {tau: (self.nodes[tau].Yhat, self.nodes[tau].Omhat) for tau in nodes}
        self.d_final = d
        self.t_total = time.perf_counter() - t_start
        return self


def build_h2(tree: ClusterTree, lists: BlockLists, kernel: int, params, tol: float,
             omega: np.ndarray, sampler, d0: int = 32, d_inc: int = 16,
             d_max: int = 256) -> H2Oracle:
    """Algorithm 1 with the adaptive loop of Sec. III-B.

    `sampler(Om)` returns K @ Om for Om (N x c) in original point order;
    `omega` is the stored Gaussian matrix (N x >= d_max, original order).
    """
    bld = _Builder(tree, lists, kernel, params, tol, omega, d0, d_inc, d_max, sampler).run()
    h = H2Oracle(tree, lists, kernel, tuple(params or ()), tol, bld.l_top, bld.nodes, bld.D, bld.B,
                 bld.d_final, bld.nrmK, bld.eps_abs, bld.eps_level, bld.d_level, bld.converged)
    h.timings = {"total_s": bld.t_total, "sketch_s": bld.t_sketch,
                 "construct_s": bld.t_total - bld.t_sketch}
    return h


# -----------------------------------------------------------------------------
# Samplers (the black box K_blk of Algorithm 1)
# -----------------------------------------------------------------------------


def dense_matrix(X: np.ndarray, kernel: int, params) -> np.ndarray:
    idx = np.arange(X.shape[0])
    return kernel_block(kernel, params, X, X, idx, idx)


def dense_sampler(A: np.ndarray):
    """Y = A @ Omega with the matrix formed explicitly."""
    return lambda Om: A @ Om


def ksum_rows(X: np.ndarray, kernel: int, params, Om: np.ndarray, rows: np.ndarray,
              chunk: int = 256) -> np.ndarray:
    """Direct kernel summation Y[rows] = sum_j K(x_rows, x_j) Om[j] (original order)."""
    n = X.shape[0]
    allidx = np.arange(n)
    out = np.zeros((len(rows), Om.shape[1]))
    for a in range(0, len(rows), chunk):
        r = rows[a:a + chunk]
        out[a:a + len(r)] = kernel_block(kernel, params, X[r], X, r, allidx) @ Om
    return out


def ksum_sampler(X: np.ndarray, kernel: int, params, chunk: int = 256):
    """Y = K @ Omega by direct summation, never storing K."""
    rows = np.arange(X.shape[0])
    return lambda Om: ksum_rows(X, kernel, params, Om, rows, chunk)


# -----------------------------------------------------------------------------
# H2 matrix-vector product and dense expansion (used as K_blk in Sec. V-A)
# -----------------------------------------------------------------------------


def h2_matvec(h: H2Oracle, x: np.ndarray) -> np.ndarray:
    """y = K_H2 x for x (N x nrhs) in original point order."""
    tree = h.tree
    x = np.asarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[:, None]
    xt = x[tree.perm]
    yt = np.zeros_like(xt)
    # near field
    for (s, t), Dst in h.D.items():
        yt[tree.begin[s]:tree.end[s]] += Dst @ xt[tree.begin[t]:tree.end[t]]
    if h.l_top > 0:
        # upsweep: xhat_tau = U_tau^T x_tau, xhat_tau = E_tau^T [xhat_1; xhat_2]
        xhat = {}
        for level in range(1, h.l_top + 1):
            for tau in tree.nodes_at_depth(tree.level_depth(level)):
                nd = h.nodes[tau]
                if level == 1:
                    xin = xt[tree.begin[tau]:tree.end[tau]]
                else:
                    xin = np.vstack([xhat[2 * tau + 1], xhat[2 * tau + 2]])
                xhat[tau] = nd.U.T @ xin
        # couplings at every level
        yhat = {tau: np.zeros_like(v) for tau, v in xhat.items()}
        for (s, t), Bst in h.B.items():
            yhat[s] += Bst @ xhat[t]
        # downsweep
        for level in range(h.l_top, 0, -1):
            for tau in tree.nodes_at_depth(tree.level_depth(level)):
                nd = h.nodes[tau]
                z = nd.U @ yhat[tau]
                if level == 1:
                    yt[tree.begin[tau]:tree.end[tau]] += z
                else:
                    k1 = h.nodes[2 * tau + 1].k
                    yhat[2 * tau + 1] += z[:k1]
                    yhat[2 * tau + 2] += z[k1:]
    y = np.zeros_like(yt)
    y[tree.perm] = yt
    return y[:, 0] if squeeze else y


def expanded_basis(h: H2Oracle, tau: int, level: int) -> np.ndarray:
    """The full basis of node tau (|I_tau| x k_tau) from the nested form."""
    if level == 1:
        return h.nodes[tau].U
    U1 = expanded_basis(h, 2 * tau + 1, level - 1)
    U2 = expanded_basis(h, 2 * tau + 2, level - 1)
    blk = np.zeros((U1.shape[0] + U2.shape[0], U1.shape[1] + U2.shape[1]))
    blk[:U1.shape[0], :U1.shape[1]] = U1
    blk[U1.shape[0]:, U1.shape[1]:] = U2
    return blk @ h.nodes[tau].U


def h2_dense(h: H2Oracle) -> np.ndarray:
    """Dense N x N matrix (original order) represented by the H2 matrix."""
    tree = h.tree
    n = tree.n
    At = np.zeros((n, n))
    for (s, t), Dst in h.D.items():
        At[tree.begin[s]:tree.end[s], tree.begin[t]:tree.end[t]] = Dst
    cache = {}
    for level in range(1, h.l_top + 1):
        depth = tree.level_depth(level)
        for s, partners in h.lists.far[depth].items():
            if s not in cache:
                cache[s] = expanded_basis(h, s, level)
            for t in partners:
                if t not in cache:
                    cache[t] = expanded_basis(h, t, level)
                At[tree.begin[s]:tree.end[s], tree.begin[t]:tree.end[t]] = \
                    cache[s] @ h.B[(s, t)] @ cache[t].T
    A = np.zeros_like(At)
    A[np.ix_(tree.perm, tree.perm)] = At
    return A


def h2_sampler(h: H2Oracle):
    """The black box K_blk of the covariance and IE test problems (Sec. V-A):
    samples Y = H Omega from the matvec of an H2 matrix H prebuilt for the
    same kernel; the entries of the new matrix are still evaluated directly."""
    def sampler(Om):
        return h2_matvec(h, Om)
    return sampler


def low_rank_update(tree: ClusterTree, entries, sampler, U: np.ndarray, V: np.ndarray) -> tuple:
    """Entry function and sampler of an operator plus the product U V^T (the
    update problem of Sec. V-A: an existing H2 matrix plus a rank-32 product;
    the symmetric construction needs U V^T symmetric, the non-symmetric one
    takes any U, V).  `entries` is a kernel id
    with its parameters as a pair (kernel, params), or a callable on tree
    positions; `sampler` gives the operator's products in original order; U
    and V are (N, r) in original order."""
    Ut, Vt = U[tree.perm], V[tree.perm]

    def entries2(Ia, Ib):
        if callable(entries):
            base = np.asarray(entries(Ia, Ib), dtype=np.float64)
        else:
            base = _entries(tree, entries[0], entries[1], Ia, Ib)
        return base + Ut[Ia] @ Vt[Ib].T

    def sampler2(Om):
        return sampler(Om) + U @ (V.T @ Om)

    return entries2, sampler2


def h2_sum_operator(ops: list) -> tuple:
    """Entry function and sampler of the sum of H2 matrices `ops` on one tree
    (the H2-update operator of Sec. V-A): entries from the dense expansion of
    each representation, samples from the tree-walk matvecs."""
    tree = ops[0].tree
    At = sum(h2_dense(h) for h in ops)[np.ix_(tree.perm, tree.perm)]

    def entries(Ia, Ib):
        return At[np.ix_(Ia, Ib)]

    def sampler(Om):
        return sum(h2_matvec(h, Om) for h in ops)

    return entries, sampler


# -----------------------------------------------------------------------------
# Error measures (Sec. V-A)
# -----------------------------------------------------------------------------


def dense_rel_error(h: H2Oracle, A: np.ndarray) -> float:
    """||A - A_H2||_F / ||A||_F."""
    return float(np.linalg.norm(A - h2_dense(h)) / np.linalg.norm(A))


def sampled_rel_error(h: H2Oracle, X, kernel, params, G: np.ndarray,
                      rows: np.ndarray | None = None) -> float:
    """||(A - A_H2) G||_F / ||A G||_F, restricted to `rows` when given."""
    AG = ksum_rows(X, kernel, params, G, np.arange(X.shape[0]) if rows is None else rows)
    HG = h2_matvec(h, G)
    if rows is not None:
        HG = HG[rows]
    return float(np.linalg.norm(AG - HG) / np.linalg.norm(AG))


def power_rel_error(h: H2Oracle, sampler, n: int, iters: int = 10, seed: int = 0) -> float:
    """||A - A_H2||_2 / ||A||_2, both by power iteration (the paper's measure,
    Sec. V-A); A is symmetric so E^T E v = E (E v)."""
    rng = np.random.default_rng(seed)

    def top_singular(apply):
        v = rng.standard_normal((n, 1))
        v /= np.linalg.norm(v)
        est = 0.0
        for _ in range(iters):
            r = apply(v)
            est = float(np.linalg.norm(r))
            if est == 0.0:
                return 0.0
            v = apply(r)
            v /= np.linalg.norm(v)
        return est

    err = top_singular(lambda v: sampler(v) - h2_matvec(h, v))
    nrm = top_singular(sampler)
    return err / nrm


def storage_entries(h: H2Oracle) -> dict:
    """Stored entries of the representation (D, B, U/E), for the O(N) memory check."""
    dn = sum(v.size for v in h.D.values())
    bn = sum(v.size for v in h.B.values())
    un = sum(nd.U.size for nd in h.nodes.values())
    return {"D": dn, "B": bn, "U": un, "total": dn + bn + un}


# -----------------------------------------------------------------------------
# Non-symmetric operators.  Sec. II-A writes an admissible block as
# U_s B_st V_t^T; for a symmetric operator V = U and Algorithm 1 needs one
# sketch.  For a non-symmetric one the same bottom-up steps run twice per
# level: the row side on Y = A Omega gives U (row IDs), the column side on
# Z = A^T Psi gives V (column IDs).  The inner subtraction of each side uses
# the other side's bases: A(I_nu, I_b) Omega_b = U_nu B_nu,b (V_b^T Omega_b)
# and A(I_b, I_nu)^T Psi_b = V_nu B_b,nu^T (U_b^T Psi_b).  Couplings are
# B_st = A(Itil_row(s), Itil_col(t)).
# -----------------------------------------------------------------------------


@dataclass
class H2OracleNonSym:
    tree: ClusterTree
    lists: BlockLists
    tol: float
    l_top: int
    rows: dict                  # heap id -> NodeData of the row side (U, row skeletons)
    cols: dict                  # heap id -> NodeData of the column side (V in .U)
    D: dict
    B: dict
    d_final: int
    nrmK: float
    eps_abs: float
    eps_level: dict
    d_level: dict
    converged: bool


class _NonSymBuilder:
    """Algorithm 1 with separate row and column bases (see above)."""

    def __init__(self, tree, lists, entries, tol, omega, psi, sampler, sampler_t, d0, d_inc,
                 d_max):
        self.tree, self.lists, self.entries, self.tol = tree, lists, entries, tol
        self.omega = np.asarray(omega, dtype=np.float64)
        self.psi = np.asarray(psi, dtype=np.float64)
        self.sampler, self.sampler_t = sampler, sampler_t
        self.d0, self.d_inc, self.d_max = d0, d_inc, d_max
        self.rows, self.cols, self.D, self.B = {}, {}, {}, {}
        self.l_top = top_level(tree, lists)
        self.eps_level, self.d_level = {}, {}
        self.converged = True

    def sample(self, c0, c1):
        """(Y, Omega, Z, Psi) of columns c0:c1 in tree order."""
        perm = self.tree.perm
        om = np.ascontiguousarray(self.omega[:, c0:c1])
        ps = np.ascontiguousarray(self.psi[:, c0:c1])
        Y = np.asarray(self.sampler(om))
        Z = np.asarray(self.sampler_t(ps))
        return Y[perm], om[perm], Z[perm], ps[perm]

    def level_nodes(self, level):
        return self.tree.nodes_at_depth(self.tree.level_depth(level))

    def far(self, level, node):
        return self.lists.far[self.tree.level_depth(level)].get(node, [])

    def local_samples(self, level, S, below):
        """Per node: (Y_loc, Omega^l, Z_loc, Psi^l).  S = (Y, Om, Z, Psi) of the
        block in tree order at level 1; `below` holds per node of level - 1
        (Yhat, Omhat, Zhat, Psihat)."""
        tree = self.tree
        out = {}
        for tau in self.level_nodes(level):
            if level == 1:
                Yt, Ot, Zt, Pt = S
                r = np.arange(tree.begin[tau], tree.end[tau])
                Y, Z = Yt[r].copy(), Zt[r].copy()
                for b in self.lists.near.get(tau, []):
                    c = np.arange(tree.begin[b], tree.end[b])
                    Y -= self.D[(tau, b)] @ Ot[c]
                    Z -= self.D[(b, tau)].T @ Pt[c]
                out[tau] = (Y, Ot[r].copy(), Z, Pt[r].copy())
            else:
                py, po, pz, pp = [], [], [], []
                for nu in (2 * tau + 1, 2 * tau + 2):
                    Yh, Oh, Zh, Ph = below[nu]
                    Ys, Zs = Yh.copy(), Zh.copy()
                    for b in self.far(level - 1, nu):
                        Ys -= self.B[(nu, b)] @ below[b][1]
                        Zs -= self.B[(b, nu)].T @ below[b][3]
                    py.append(Ys)
                    po.append(Oh)
                    pz.append(Zs)
                    pp.append(Ph)
                out[tau] = (np.vstack(py), np.vstack(po), np.vstack(pz), np.vstack(pp))
        return out

    def upsweep(self, local):
        """Yhat = Y_loc(J_row), Omhat = V^T Omega^l, Zhat = Z_loc(J_col),
        Psihat = U^T Psi^l."""
        res = {}
        for tau, (Y, O, Z, P) in local.items():
            rn, cn = self.rows[tau], self.cols[tau]
            res[tau] = (Y[rn.J, :], cn.U.T @ O, Z[cn.J, :], rn.U.T @ P)
        return res

    def sweep_new_columns(self, level, c0, c1):
        S = self.sample(c0, c1)
        below = None
        for lv in range(1, level + 1):
            local = self.local_samples(lv, S, below)
            if lv == level:
                return local
            below = self.upsweep(local)
        return None

    def run(self):
        tree = self.tree
        d = self.d0
        S = self.sample(0, d)
        # ||A||_F estimated from both sketches (the same number for A and A^T)
        self.nrmK = float(math.sqrt((np.linalg.norm(S[0]) ** 2 + np.linalg.norm(S[2]) ** 2)
                                    / (2 * d)))
        self.eps_abs = self.tol * self.nrmK
        for tau in tree.nodes_at_depth(tree.depth):
            r = np.arange(tree.begin[tau], tree.end[tau])
            for b in self.lists.near.get(tau, []):
                c = np.arange(tree.begin[b], tree.end[b])
                self.D[(tau, b)] = _entries(tree, self.entries, None, r, c)
        below = None
        for level in range(1, self.l_top + 1):
            nodes = list(self.level_nodes(level))
            eps_l = self.eps_abs / math.sqrt(2 * self.l_top * len(nodes))
            self.eps_level[level] = eps_l
            local = self.local_samples(level, S if level == 1 else None, below)
            for tau in nodes:
                Y, O, Z, P = local[tau]
                rn, cn = NodeData(), NodeData()
                for nd, side in ((rn, self.rows), (cn, self.cols)):
                    nd.m = Y.shape[0]
                    if level == 1:
                        nd.Ibar = np.arange(tree.begin[tau], tree.end[tau])
                    else:
                        nd.Ibar = np.concatenate([side[2 * tau + 1].Itil, side[2 * tau + 2].Itil])
                rn.Yloc, rn.Om, cn.Yloc, cn.Om = Y, O, Z, P
                self.rows[tau], self.cols[tau] = rn, cn
            while self.d_inc > 0:
                pending = [t for t in nodes
                           if not (node_converged(self.rows[t].Yloc, eps_l)
                                   and node_converged(self.cols[t].Yloc, eps_l))]
                if not pending:
                    break
                if d + self.d_inc > self.d_max:
                    self.converged = False
                    break
                new = self.sweep_new_columns(level, d, d + self.d_inc)
                d += self.d_inc
                for tau in nodes:
                    Yn, On, Zn, Pn = new[tau]
                    rn, cn = self.rows[tau], self.cols[tau]
                    rn.Yloc, rn.Om = np.hstack([rn.Yloc, Yn]), np.hstack([rn.Om, On])
                    cn.Yloc, cn.Om = np.hstack([cn.Yloc, Zn]), np.hstack([cn.Om, Pn])
            self.d_level[level] = d
            for tau in nodes:
                for nd in (self.rows[tau], self.cols[tau]):
                    rid = row_id(nd.Yloc, eps_l)
                    nd.k, nd.J, nd.U = rid.k, rid.J, rid.U
                    nd.Itil = nd.Ibar[nd.J]
            up = self.upsweep({tau: (self.rows[tau].Yloc, self.rows[tau].Om,
                                     self.cols[tau].Yloc, self.cols[tau].Om) for tau in nodes})
            for tau in nodes:
                for b in self.far(level, tau):
                    self.B[(tau, b)] = _entries(tree, self.entries, None, self.rows[tau].Itil,
                                                self.cols[b].Itil)
            below = up
        self.d_final = d
        return self


def build_h2_nonsym(tree: ClusterTree, lists: BlockLists, entries, tol: float, omega: np.ndarray,
                    psi: np.ndarray, sampler, sampler_t, d0: int = 32, d_inc: int = 16,
                    d_max: int = 256) -> H2OracleNonSym:
    """H2 construction of a non-symmetric operator: `entries(Ia, Ib)` on tree
    positions, `sampler(Om)` = A Om and `sampler_t(Psi)` = A^T Psi in original
    order, `omega` and `psi` the stored Gaussian matrices of the two sides."""
    b = _NonSymBuilder(tree, lists, entries, tol, omega, psi, sampler, sampler_t, d0, d_inc,
                       d_max).run()
    return H2OracleNonSym(tree, lists, tol, b.l_top, b.rows, b.cols, b.D, b.B, b.d_final,
                          b.nrmK, b.eps_abs, b.eps_level, b.d_level, b.converged)


def h2_matvec_nonsym(h: H2OracleNonSym, x: np.ndarray) -> np.ndarray:
    """y = A_H2 x: near field, upsweep with the column bases V, couplings,
    downsweep with the row bases U."""
    tree = h.tree
    x = np.asarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[:, None]
    xt = x[tree.perm]
    yt = np.zeros_like(xt)
    for (s, t), Dst in h.D.items():
        yt[tree.begin[s]:tree.end[s]] += Dst @ xt[tree.begin[t]:tree.end[t]]
    if h.l_top > 0:
        xhat = {}
        for level in range(1, h.l_top + 1):
            for tau in tree.nodes_at_depth(tree.level_depth(level)):
                xin = (xt[tree.begin[tau]:tree.end[tau]] if level == 1
                       else np.vstack([xhat[2 * tau + 1], xhat[2 * tau + 2]]))
                xhat[tau] = h.cols[tau].U.T @ xin
        yhat = {tau: np.zeros((h.rows[tau].k, x.shape[1])) for tau in xhat}
        for (s, t), Bst in h.B.items():
            yhat[s] += Bst @ xhat[t]
        for level in range(h.l_top, 0, -1):
            for tau in tree.nodes_at_depth(tree.level_depth(level)):
                z = h.rows[tau].U @ yhat[tau]
                if level == 1:
                    yt[tree.begin[tau]:tree.end[tau]] += z
                else:
                    k1 = h.rows[2 * tau + 1].k
                    yhat[2 * tau + 1] += z[:k1]
                    yhat[2 * tau + 2] += z[k1:]
    y = np.zeros_like(yt)
    y[tree.perm] = yt
    return y[:, 0] if squeeze else y
