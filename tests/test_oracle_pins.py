"""Pins for the CPU oracle: each check compares it with something other than
itself (closed forms, brute force, exact low rank, dense SVD, the identities
of Sec. III-A).  CPU only."""
import math
import os

import numpy as np
import pytest

from oracle import h2_oracle as O
from paper_2506_16759_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KNAMES = {"exp": O.K_EXP, "matern32": O.K_MATERN32, "gauss": O.K_GAUSS,
          "laplace_ie": O.K_LAPLACE_IE, "poly": O.K_POLY, "helmholtz_ie": O.K_HELMHOLTZ_IE}


def _golden_kernel_rows():
    rows = []
    with open(os.path.join(GOLDEN, "kernel_values.txt")) as f:
        for line in f:
            if not line.strip() or line.startswith("#"):
                continue
            fields = [x.strip() for x in line.split("|")]
            kname, params = fields[0].split()
            rows.append((KNAMES[kname], tuple(float(v) for v in params.split(",")),
                         [float(v) for v in fields[1].split(",")],
                         [float(v) for v in fields[2].split(",")],
                         fields[3] == "1", float(fields[4])))
    return rows


@pytest.mark.parametrize("row", _golden_kernel_rows())
def test_kernel_closed_forms(row):
    kernel, params, xa, xb, same, expected = row
    if kernel == O.K_POLY:
        params = (params[0], int(params[1]))
    ia = np.array([0])
    ib = np.array([0 if same else 1])
    val = O.kernel_block(kernel, params, np.array([xa]), np.array([xb]), ia, ib)[0, 0]
    assert val == pytest.approx(expected, rel=1e-14, abs=1e-15)


# --- cluster tree ----------------------------------------------------------------


@pytest.mark.parametrize("n,dim,leaf", [(1000, 2, 64), (777, 3, 16), (64, 2, 64), (65, 3, 64),
                                        (5, 2, 2), (1, 3, 4)])
def test_tree_structure(n, dim, leaf):
    X = W.uniform_points(n, dim, 11)
    t = O.build_cluster_tree(X, leaf)
    # uniform depth: smallest L with ceil(n / 2^L) <= leaf
    L = t.depth
    assert math.ceil(n / 2 ** L) <= leaf and (L == 0 or math.ceil(n / 2 ** (L - 1)) > leaf)
    assert sorted(t.perm.tolist()) == list(range(n))
    for v in range(t.n_nodes):
        P = t.perm[t.begin[v]:t.end[v]]
        assert len(P) >= 1
        # tight box
        assert np.array_equal(t.lo[v], X[P].min(0)) and np.array_equal(t.hi[v], X[P].max(0))
        if 2 * v + 1 < t.n_nodes:
            a, b = 2 * v + 1, 2 * v + 2
            na, nb = t.end[a] - t.begin[a], t.end[b] - t.begin[b]
            assert na == (len(P) + 1) // 2 and na + nb == len(P)
            ext = t.hi[v] - t.lo[v]
            s = t.split_dim[v]
            assert ext[s] == ext.max() and all(ext[q] < ext[s] for q in range(s))
            # every left point precedes every right point in (coordinate, index) order
            left = [(X[p, s], p) for p in t.perm[t.begin[a]:t.end[a]]]
            right = [(X[p, s], p) for p in t.perm[t.begin[b]:t.end[b]]]
            assert max(left) < min(right)
    # leaf members are ordered by the parent's split key
    if L > 0:
        for v in t.nodes_at_depth(L):
            s = t.split_dim[(v - 1) // 2]
            keys = [(X[p, s], p) for p in t.perm[t.begin[v]:t.end[v]]]
            assert keys == sorted(keys)


def test_tree_duplicate_points():
    # all points identical: every extent is 0, so dimension 0 is used and the
    # point index alone orders the split
    X = np.full((100, 3), 0.25)
    t = O.build_cluster_tree(X, 8)
    assert t.perm.tolist() == list(range(100))
    lists = O.dual_traversal(t, 0.7)
    assert O.top_level(t, lists) == 0


def test_admissibility_hand_cases():
    # unit squares: D = sqrt 2 each.  Gap 2 -> (sqrt2 + sqrt2)/2 = 1.414 > 0.7*2
    t = O.ClusterTree(np.zeros((1, 2)), 2, 0, np.zeros(1, int), np.zeros(3, int), np.zeros(3, int),
                      np.array([[0, 0], [3, 0], [4, 0.]]), np.array([[1, 1], [4, 1], [5, 1.]]),
                      np.zeros(3, int))
    assert O.box_diameter(t.lo[0], t.hi[0]) == pytest.approx(math.sqrt(2))
    assert O.box_distance(t.lo[0], t.hi[0], t.lo[1], t.hi[1]) == 2.0
    assert not O.admissible(t, 0, 1, 0.7)
    assert O.box_distance(t.lo[0], t.hi[0], t.lo[2], t.hi[2]) == 3.0
    assert O.admissible(t, 0, 2, 0.7)           # 1.414 <= 2.1
    assert O.admissible(t, 2, 0, 0.7)
    assert not O.admissible(t, 0, 2, 0.47)      # 1.414 > 1.41
    # touching or overlapping boxes are never admissible (Dist = 0)
    assert not O.admissible(t, 1, 2, 1e9)
    # diagonal gap: boxes [0,1]^2 and [2,3]^2 -> Dist = sqrt(2)
    t.lo[1], t.hi[1] = [2, 2], [3, 3]
    assert O.box_distance(t.lo[0], t.hi[0], t.lo[1], t.hi[1]) == pytest.approx(math.sqrt(2))


@pytest.mark.parametrize("eta", [0.7, 1.5, 0.3])
def test_block_partition_brute_force(eta):
    n = 300
    X = W.uniform_points(n, 2, 3)
    t = O.build_cluster_tree(X, 8)
    lists = O.dual_traversal(t, eta)
    cover = np.zeros((n, n), dtype=int)
    for s, partners in lists.near.items():
        for b in partners:
            cover[t.begin[s]:t.end[s], t.begin[b]:t.end[b]] += 1
    for k in range(t.depth + 1):
        for s, partners in lists.far[k].items():
            for b in partners:
                cover[t.begin[s]:t.end[s], t.begin[b]:t.end[b]] += 1
                assert O.admissible(t, s, b, eta)
                # F_s: the parents must form an inadmissible pair
                if k > 0:
                    assert not O.admissible(t, (s - 1) // 2, (b - 1) // 2, eta)
    assert (cover == 1).all()
    # symmetry of both lists
    for s, partners in lists.near.items():
        for b in partners:
            assert s in lists.near[b]
    for k in range(t.depth + 1):
        for s, partners in lists.far[k].items():
            assert partners == sorted(partners)
            for b in partners:
                assert s in lists.far[k][b]


# --- dense kernels of the construction ---------------------------------------------


def test_qr_min_diag_known_factor():
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 12)))
    R0 = np.triu(rng.standard_normal((12, 12)))
    diag = np.array([3.0, -2.0, 1.5, 1e-3, 7.0, 0.5, -0.25, 2.0, 1.0, 4.0, -9.0, 0.75])
    R0[np.arange(12), np.arange(12)] = diag
    assert O.qr_min_abs_diag(Q @ R0) == pytest.approx(1e-3, rel=1e-9)
    assert O.node_converged(Q @ R0, 2e-3) and not O.node_converged(Q @ R0, 5e-4)
    assert O.node_converged(rng.standard_normal((8, 12)), 0.0)   # m <= d


def test_cpqr_exact_rank_and_interpolation():
    rng = np.random.default_rng(1)
    for rows, cols, k in [(30, 50, 7), (20, 20, 20), (12, 40, 1)]:
        A = rng.standard_normal((rows, k)) @ rng.standard_normal((k, cols))
        kk, piv, T = O.cpqr_column_id(A, 1e-10 * np.linalg.norm(A))
        assert kk == k
        S, R = piv[:kk], piv[kk:]
        assert np.linalg.norm(A[:, R] - A[:, S] @ T) <= 1e-12 * np.linalg.norm(A)
        if len(R):
            Tls = np.linalg.lstsq(A[:, S], A[:, R], rcond=None)[0]
            assert np.allclose(T, Tls, atol=1e-8)


def test_cpqr_pivots_follow_norms():
    # orthogonal columns: pivots in decreasing norm order, lowest index on ties
    norms = np.array([1.0, 5.0, 3.0, 5.0, 0.5])
    Q, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((8, 5)))
    A = Q * norms
    k, piv, T = O.cpqr_column_id(A, 0.0)
    assert piv.tolist() == [1, 3, 2, 0, 4] and k == 5
    k, piv, T = O.cpqr_column_id(A, math.sqrt(1.0 + 0.25) + 1e-12)
    assert k == 3


def test_row_id_basis_identity_rows():
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((30, 6)) @ rng.standard_normal((6, 40))
    rid = O.row_id(Y, 1e-9)
    assert rid.k == 6
    assert np.array_equal(rid.J, np.sort(rid.J))
    assert np.array_equal(rid.U[rid.J], np.eye(6))
    assert np.linalg.norm(Y - rid.U @ Y[rid.J]) <= 1e-11 * np.linalg.norm(Y)


# --- whole construction ------------------------------------------------------------


def _build(n, dim, kernel, params, tol, leaf=64, eta=0.7, seed=1, d0=32, d_inc=16, d_max=256):
    X = W.uniform_points(n, dim, seed)
    om = W.gaussian_omega(n, d_max, seed + 1)
    t = O.build_cluster_tree(X, leaf)
    lists = O.dual_traversal(t, eta)
    A = O.dense_matrix(X, kernel, params)
    h = O.build_h2(t, lists, kernel, params, tol, om, O.dense_sampler(A), d0, d_inc, d_max)
    return X, om, t, lists, A, h


def test_c1_dense_error_within_tolerance():
    w = W.config("c1")
    X, om = w.points(), w.omega()
    t = O.build_cluster_tree(X, w.leaf_size)
    lists = O.dual_traversal(t, w.eta)
    A = O.dense_matrix(X, w.kernel, w.params)
    h = O.build_h2(t, lists, w.kernel, w.params, w.tol, om, O.dense_sampler(A),
                   w.d0, w.d_inc, w.d_max)
    assert h.converged and h.l_top >= 2
    err = O.dense_rel_error(h, A)
    assert err <= 10 * w.tol
    # the tree-walk matvec agrees with the dense expansion of the representation
    G = W.gaussian_probe(w.n, 4, 0)
    Ad = O.h2_dense(h)
    assert np.linalg.norm(O.h2_matvec(h, G) - Ad @ G) <= 1e-13 * np.linalg.norm(Ad @ G)
    # randomized Frobenius estimate agrees with the dense error to a factor ~2
    est = O.sampled_rel_error(h, X, w.kernel, w.params, W.gaussian_probe(w.n, 16, 1))
    assert 0.3 * err <= est <= 3 * err


def test_polynomial_kernel_exact_rank():
    # (1 + x.y)^3 in 2D has rank C(2+3, 3) = 10: every compressed node whose
    # admissible block row has rank 10 gets k = 10 and the result is exact.
    X, om, t, lists, A, h = _build(2048, 2, O.K_POLY, (1.0, 3), 1e-10, leaf=32)
    assert h.l_top >= 2
    for level in range(1, h.l_top + 1):
        for tau in t.nodes_at_depth(t.level_depth(level)):
            nd = h.nodes[tau]
            assert nd.k <= 10
            if nd.m >= 10 and _far_columns(t, lists, h.l_top, tau, level).size >= 10:
                assert nd.k == 10
    assert O.dense_rel_error(h, A) <= 1e-12


def _far_columns(t, lists, l_top, tau, level):
    """Tree positions of every column block admissible to tau or an ancestor at
    levels >= level."""
    cols = []
    node, lv = tau, level
    while lv <= l_top:
        for b in lists.far[t.level_depth(lv)].get(node, []):
            cols.extend(range(t.begin[b], t.end[b]))
        node, lv = (node - 1) // 2, lv + 1
    return np.array(sorted(cols), dtype=int)


def _frobenius_rank(s, eps):
    tail = np.sqrt(np.cumsum((s ** 2)[::-1])[::-1])
    for r in range(len(s)):
        if tail[r] <= eps:
            return r
    return len(s)


def _svd_rank_violations(t, lists, h, kernel, params, slack=3):
    Xt = t.Xt()
    bad = []
    for level in range(1, h.l_top + 1):
        eps = h.eps_level[level]
        for tau in t.nodes_at_depth(t.level_depth(level)):
            nd = h.nodes[tau]
            cols = _far_columns(t, lists, h.l_top, tau, level)
            if cols.size == 0 or nd.m == 0:
                continue
            M = O.kernel_block(kernel, params, Xt[nd.Ibar], Xt[cols], nd.Ibar, cols)
            s = np.linalg.svd(M, compute_uv=False)
            if not (_frobenius_rank(s, 2 * eps) <= nd.k <= _frobenius_rank(s, eps) + slack):
                bad.append((level, tau, nd.k, _frobenius_rank(s, eps)))
    return bad


@pytest.mark.parametrize("tol", [1e-4, 1e-6, 1e-8])
def test_ranks_match_dense_svd(tol):
    # The ID rank of each node sits between the Frobenius eps_l-ranks of its
    # true admissible block row (rows: the node's candidate skeletons; columns:
    # everything admissible to it or its ancestors).
    X, om, t, lists, A, h = _build(1024, 2, O.K_EXP, (0.2, 1e-4), tol, leaf=16, seed=5)
    assert h.l_top >= 3
    assert _svd_rank_violations(t, lists, h, O.K_EXP, (0.2, 1e-4)) == []
    assert O.dense_rel_error(h, A) <= 10 * tol


def test_helmholtz_ranks_match_dense_svd():
    # the same rank pin for the oscillatory, sign-changing IE kernel cos(3r)/r
    params = (3.0, 0.0)
    X, om, t, lists, A, h = _build(2048, 3, O.K_HELMHOLTZ_IE, params, 1e-6, leaf=16, seed=6)
    assert h.l_top >= 2
    assert _svd_rank_violations(t, lists, h, O.K_HELMHOLTZ_IE, params) == []
    assert O.dense_rel_error(h, A) <= 10 * 1e-6


def test_sample_recurrence_exact_low_rank():
    # Y^l = W^l Y^{l-1} (Sec. III-A): with exact IDs (rank-10 kernel) the local
    # samples of child nu inside its parent equal the samples of the blocks
    # admissible to nu's ancestors only, restricted to nu's skeleton rows.
    X, om, t, lists, A, h = _build(2048, 2, O.K_POLY, (1.0, 3), 1e-10, leaf=32)
    Xt = t.Xt()
    omt = om[t.perm]
    d = h.d_level[2]
    checked = 0
    for tau in t.nodes_at_depth(t.level_depth(2)):
        nd = h.nodes[tau]
        row0 = 0
        cols = _far_columns(t, lists, h.l_top, tau, 2)
        for nu in (2 * tau + 1, 2 * tau + 2):
            Itil = h.nodes[nu].Itil
            expect = O.kernel_block(O.K_POLY, (1.0, 3), Xt[Itil], Xt[cols], Itil, cols) @ omt[cols, :d]
            got = nd.Yloc[row0:row0 + len(Itil)]
            assert np.linalg.norm(got - expect) <= 1e-9 * max(1.0, np.linalg.norm(expect))
            checked += int(cols.size > 0)
            row0 += len(Itil)
    assert checked > 0


def test_full_sampling_is_exact():
    # tol = 0: no node converges until d >= m, so every ID keeps all rows.
    X, om, t, lists, A, h = _build(512, 2, O.K_EXP, (0.2, 1e-4), 0.0, leaf=16, d0=8, d_inc=8,
                                   d_max=64)
    assert h.converged
    assert h.d_level[1] >= 16
    assert O.dense_rel_error(h, A) <= 1e-13


def test_nothing_admissible_is_exact():
    X, om, t, lists, A, h = _build(600, 3, O.K_MATERN32, (0.1, 1e-4), 1e-6, leaf=16, eta=1e-12)
    assert h.l_top == 0 and not h.B
    assert O.dense_rel_error(h, A) == 0.0


def test_adaptive_rounds_and_budget():
    X, om, t, lists, A, h = _build(4096, 2, O.K_EXP, (0.2, 1e-4), 1e-9, leaf=64)
    assert h.converged and max(h.d_level.values()) > 32
    assert O.dense_rel_error(h, A) <= 10 * 1e-9
    # the same problem with the sample budget capped at the first block
    X, om, t, lists, A, h2 = _build(4096, 2, O.K_EXP, (0.2, 1e-4), 1e-9, leaf=64, d_max=32)
    assert not h2.converged


def test_fixed_sampling_mode():
    # d_inc = 0: the non-adaptive construction with a fixed sample count
    # (the fixed-d runs of Sec. V-B / Table I).  With enough samples it meets
    # the tolerance and matches the adaptive run that needed no extra round;
    # with fewer samples than the ranks the truncation caps every rank at d.
    X, om, t, lists, A, ha = _build(2048, 2, O.K_EXP, (0.2, 1e-4), 1e-6, leaf=32, d0=96)
    assert ha.converged and max(ha.d_level.values()) == 96   # no adaptive round
    _, _, _, _, _, hf = _build(2048, 2, O.K_EXP, (0.2, 1e-4), 1e-6, leaf=32, d0=96, d_inc=0)
    assert O.dense_rel_error(hf, A) <= 10 * 1e-6
    for tau, nd in hf.nodes.items():
        assert np.array_equal(nd.J, ha.nodes[tau].J)
    _, _, _, _, _, hs = _build(2048, 2, O.K_EXP, (0.2, 1e-4), 1e-6, leaf=32, d0=8, d_inc=0)
    assert max(nd.k for nd in hs.nodes.values()) <= 8
    assert O.dense_rel_error(hs, A) > 10 * 1e-6


def test_power_method_matches_dense_two_norm():
    X, om, t, lists, A, h = _build(1024, 2, O.K_EXP, (0.2, 1e-4), 1e-5, leaf=16)
    Ad = O.h2_dense(h)
    exact = np.linalg.norm(A - Ad, 2) / np.linalg.norm(A, 2)
    est = O.power_rel_error(h, O.dense_sampler(A), 1024, iters=30)
    assert est == pytest.approx(exact, rel=0.05)


def test_sparsity_constant_bounded():
    # C_sp (Sec. II-A): the longest block row of any level's list does not grow
    # with N (uniform points, eta 0.7).
    csp = []
    for n in (4096, 16384, 65536):
        t = O.build_cluster_tree(W.uniform_points(n, 2, 4), 16)
        lists = O.dual_traversal(t, 0.7)
        m = max(len(v) for v in lists.near.values())
        for k in range(t.depth + 1):
            if lists.far[k]:
                m = max(m, max(len(v) for v in lists.far[k].values()))
        csp.append(m)
    assert max(csp) <= 1.25 * csp[0]


def test_storage_entries_hand_count():
    # storage_entries against a count made from the partition and the ranks
    # alone: every near pair stores an m_tau x m_b block (sizes from the tree's
    # ranges), every far pair a k_s x k_t coupling, every compressed node an
    # m x k basis with m = its leaf size or the sum of its children's ranks.
    X = W.uniform_points(300, 2, 17)
    t = O.build_cluster_tree(X, 16)
    lists = O.dual_traversal(t, 0.7)
    h = O.build_h2(t, lists, O.K_EXP, (0.2, 1e-4), 1e-6, W.gaussian_omega(300, 256, 18),
                   O.ksum_sampler(X, O.K_EXP, (0.2, 1e-4)))
    size = lambda v: int(t.end[v] - t.begin[v])
    d = sum(size(s) * size(b) for s, bs in lists.near.items() for b in bs)
    b = 0
    for level in range(1, h.l_top + 1):
        for s, ts in lists.far[t.level_depth(level)].items():
            b += sum(h.nodes[s].k * h.nodes[u].k for u in ts)
    u = 0
    for level in range(1, h.l_top + 1):
        for v in t.nodes_at_depth(t.level_depth(level)):
            m = size(v) if level == 1 else h.nodes[2 * v + 1].k + h.nodes[2 * v + 2].k
            u += m * h.nodes[v].k
    assert h.l_top >= 2 and b > 0 and u > 0
    assert O.storage_entries(h) == {"D": d, "B": b, "U": u, "total": d + b + u}


def _poly_features(X, p):
    """phi with (1 + x.y)^p = phi(x) . phi(y): sqrt of the multinomial weight
    times each monomial of degree <= p."""
    n, dim = X.shape
    cols = []

    def rec(i, alpha):
        if i == dim:
            rest = p - sum(alpha)
            w = math.factorial(p) / math.factorial(rest)
            for a in alpha:
                w /= math.factorial(a)
            cols.append(math.sqrt(w) * np.prod([X[:, j] ** a for j, a in enumerate(alpha)], 0))
            return
        for a in range(p - sum(alpha) + 1):
            rec(i + 1, alpha + [a])

    rec(0, [])
    return np.stack(cols, 1)


def _timed_poly_builds(sizes, dim, seed):
    """Construction time (sketch excluded) and stored entries of builds of
    (1 + x.y)^3, whose rank is fixed (C(dim+3, 3)), sampled through its
    feature factorisation K = Phi Phi^T."""
    out = []
    for n in sizes:
        X = W.uniform_points(n, dim, seed)
        t = O.build_cluster_tree(X, 64)
        lists = O.dual_traversal(t, 0.7)
        P = _poly_features(X, 3)
        h = O.build_h2(t, lists, O.K_POLY, (1.0, 3), 1e-8, W.gaussian_omega(n, 64, seed + 1),
                       lambda Om: P @ (P.T @ Om), 32, 16, 64)
        out.append((n, h.timings["construct_s"], O.storage_entries(h)["total"]))
    return out


def _slope(x, y):
    return float(np.polyfit(np.log(x), np.log(y), 1)[0])


def test_poly_features_factor_the_kernel():
    X = W.uniform_points(40, 3, 3)
    P = _poly_features(X, 3)
    assert P.shape[1] == math.comb(3 + 3, 3)
    A = O.dense_matrix(X, O.K_POLY, (1.0, 3))
    assert np.allclose(P @ P.T, A, rtol=1e-13, atol=1e-13)


def test_construction_time_and_memory_linear_in_n():
    # Sec. III-A: the construction takes O(N) time and memory once the sketch
    # is given; Sec. V-B measures linear memory.  In 2D the block partition of
    # a uniform cloud reaches its asymptotic sparsity already at these sizes
    # (same-parity depths, whose near lists are alike), so both log-log slopes
    # over N = 2^13, 2^15, 2^17 are close to 1.
    r = _timed_poly_builds([8192, 32768, 131072], 2, 31)
    n = [a for a, _, _ in r]
    assert 0.8 <= _slope(n, [b for _, b, _ in r]) <= 1.25, r
    assert 0.8 <= _slope(n, [c for _, _, c in r]) <= 1.25, r


def test_construction_time_follows_stored_entries_in_3d():
    # In 3D the near list of a uniform cloud (eta 0.7, leaf 64) keeps growing
    # up to about 2^17 points (59 partners per leaf at 2^12, about 200 at
    # 2^17), so storage per point is not yet flat over 2^12..2^15.  The
    # construction must still cost a fixed amount per stored entry: the slope
    # of time against stored entries over four sizes is close to 1 (a hidden
    # per-block O(N) step would make it about 2).
    r = _timed_poly_builds([4096, 8192, 16384, 32768], 3, 41)
    sl = _slope([c for _, _, c in r], [b for _, b, _ in r])
    assert 0.8 <= sl <= 1.25, r
    assert 0.8 <= _slope([a for a, _, _ in r], [b for _, b, _ in r]) <= 1.6, r


# --- sensitivity: mistakes planted in the oracle must trip a pin -------------------


def test_planted_mistake_dropped_inner_subtraction(monkeypatch):
    orig = O._Builder.local_samples

    def no_far_subtraction(self, level, Yt, Ot, below):
        saved = self.B
        if level > 1:
            self.B = {k: np.zeros_like(v) for k, v in saved.items()}
        try:
            return orig(self, level, Yt, Ot, below)
        finally:
            self.B = saved

    monkeypatch.setattr(O._Builder, "local_samples", no_far_subtraction)
    with pytest.raises(AssertionError):
        test_sample_recurrence_exact_low_rank()
    with pytest.raises(AssertionError):
        test_ranks_match_dense_svd(1e-6)


def test_planted_mistake_skeleton_indices(monkeypatch):
    # local skeleton positions used where tree positions are needed
    monkeypatch.setattr(O._Builder, "skeleton_rows", lambda self, nd: nd.J)
    with pytest.raises(AssertionError):
        test_c1_dense_error_within_tolerance()


def test_planted_mistake_wrong_threshold(monkeypatch):
    # eps_l without the per-level split of the budget
    orig = O.row_id
    monkeypatch.setattr(O, "row_id", lambda Y, eps: orig(Y, eps * 30.0))
    with pytest.raises(AssertionError):
        test_ranks_match_dense_svd(1e-6)


def test_planted_mistake_omega_upsweep(monkeypatch):
    # Omega^{l+1} taken as the skeleton rows of Omega^l instead of U^T Omega^l
    def bad(self, level, local):
        return {tau: (Y[self.nodes[tau].J, :], O_[self.nodes[tau].J, :])
                for tau, (Y, O_) in local.items()}

    monkeypatch.setattr(O._Builder, "upsweep", bad)
    with pytest.raises(AssertionError):
        test_sample_recurrence_exact_low_rank()


def test_planted_mistake_near_field_sign(monkeypatch):
    orig = O._Builder.local_samples

    def flipped(self, level, Yt, Ot, below):
        if level == 1:
            saved = self.D
            self.D = {k: -v for k, v in saved.items()}
            try:
                return orig(self, level, Yt, Ot, below)
            finally:
                self.D = saved
        return orig(self, level, Yt, Ot, below)

    monkeypatch.setattr(O._Builder, "local_samples", flipped)
    with pytest.raises(AssertionError):
        test_ranks_match_dense_svd(1e-6)


def test_h2_sum_operator_entries_and_samples():
    # the H2-update operator: its entries and samples are those of the sum of
    # the dense matrices the operands represent
    X = W.uniform_points(1024, 2, 51)
    t = O.build_cluster_tree(X, 16)
    lists = O.dual_traversal(t, 0.7)
    om = W.gaussian_omega(1024, 256, 52)
    ops = [O.build_h2(t, lists, k, p, 1e-8, om, O.ksum_sampler(X, k, p))
           for k, p in ((O.K_EXP, (0.1, 0.0)), (O.K_GAUSS, (0.05, 0.0)))]
    entries, sampler = O.h2_sum_operator(ops)
    A = O.dense_matrix(X, O.K_EXP, (0.1, 0.0)) + O.dense_matrix(X, O.K_GAUSS, (0.05, 0.0))
    At = A[np.ix_(t.perm, t.perm)]
    full = np.arange(1024)
    assert np.linalg.norm(entries(full, full) - At) <= 1e-7 * np.linalg.norm(At)
    rows, cols = np.arange(40, 90), np.arange(500, 560)
    blk = At[np.ix_(rows, cols)]
    assert np.linalg.norm(entries(rows, cols) - blk) <= 1e-6 * np.linalg.norm(blk)
    G = W.gaussian_probe(1024, 3, 0)
    assert np.linalg.norm(sampler(G) - A @ G) <= 1e-7 * np.linalg.norm(A @ G)
    # a target built from the operator meets its tolerance against the exact sum
    h = O.build_h2(t, lists, entries, None, 1e-6, W.gaussian_omega(1024, 256, 53), sampler)
    assert O.dense_rel_error(h, A) <= 10 * 1e-6


def test_helmholtz_at_zero_wave_number_is_scaled_laplace():
    # cos(0 r)/r = 4 pi * 1/(4 pi r) off the diagonal; both take the stated
    # diagonal value
    X = W.uniform_points(300, 3, 71)
    idx = np.arange(300)
    H = O.kernel_block(O.K_HELMHOLTZ_IE, (0.0, 0.5), X, X, idx, idx)
    L = O.kernel_block(O.K_LAPLACE_IE, (0.5,), X, X, idx, idx)
    off = ~np.eye(300, dtype=bool)
    assert np.allclose(H[off], 4 * math.pi * L[off], rtol=1e-14, atol=0)
    assert np.array_equal(np.diag(H), np.diag(L))
    # symmetric, and bounded by 1/r in magnitude
    H3 = O.kernel_block(O.K_HELMHOLTZ_IE, (3.0, 0.0), X, X, idx, idx)
    assert np.array_equal(H3, H3.T)
    assert np.all(np.abs(H3[off]) <= np.abs(H[off]) * (1 + 1e-15))


def test_helmholtz_build_with_h2_matvec_sampler():
    # Sec. V-A: the Helmholtz volume-IE operator cos(3r)/r sketched through
    # the matvec of an H2 matrix prebuilt for the same kernel, entries
    # evaluated directly; the result meets the tolerance against dense A.
    n, dim, leaf, tol = 4096, 3, 32, 1e-6
    params = (3.0, 0.0)
    X = W.uniform_points(n, dim, 72)
    t = O.build_cluster_tree(X, leaf)
    lists = O.dual_traversal(t, 0.7)
    A = O.dense_matrix(X, O.K_HELMHOLTZ_IE, params)
    pre = O.build_h2(t, lists, O.K_HELMHOLTZ_IE, params, tol / 10, W.gaussian_omega(n, 256, 73),
                     O.dense_sampler(A))
    assert pre.converged and O.dense_rel_error(pre, A) <= tol
    h = O.build_h2(t, lists, O.K_HELMHOLTZ_IE, params, tol, W.gaussian_omega(n, 256, 74),
                   O.h2_sampler(pre))
    assert h.converged and h.l_top >= 2
    assert O.dense_rel_error(h, A) <= 10 * tol


def test_low_rank_update_operator():
    # Sec. V-A update problem: an H2 matrix plus a symmetric rank-r product.
    # Entries and samples are those of the exact dense sum, and a target
    # built from them meets the tolerance against it (and not against the
    # operand alone: the product is not negligible).
    n = 1024
    X = W.uniform_points(n, 2, 81)
    t = O.build_cluster_tree(X, 16)
    lists = O.dual_traversal(t, 0.7)
    kp = (O.K_EXP, (0.2, 0.0))
    A = O.dense_matrix(X, *kp)
    op = O.build_h2(t, lists, *kp, 1e-8, W.gaussian_omega(n, 256, 82), O.dense_sampler(A))
    U, V = W.low_rank_factors(n, 8, 83, 0.01 * n)
    assert np.allclose(U @ V.T, V @ U.T, rtol=0, atol=1e-14 * n)
    full = A + U @ V.T
    base_entries, base_sampler = O.h2_sum_operator([op])
    entries, sampler = O.low_rank_update(t, base_entries, base_sampler, U, V)
    Ft = full[np.ix_(t.perm, t.perm)]
    idx = np.arange(n)
    assert np.linalg.norm(entries(idx, idx) - Ft) <= 1e-7 * np.linalg.norm(Ft)
    G = W.gaussian_probe(n, 3, 0)
    assert np.linalg.norm(sampler(G) - full @ G) <= 1e-7 * np.linalg.norm(full @ G)
    h = O.build_h2(t, lists, entries, None, 1e-6, W.gaussian_omega(n, 256, 84), sampler)
    assert O.dense_rel_error(h, full) <= 10 * 1e-6
    assert O.dense_rel_error(h, A) > 1e3 * 1e-6
    # the same update of the kernel itself (entries evaluated, dense samples)
    entries_k, sampler_k = O.low_rank_update(t, kp, O.dense_sampler(A), U, V)
    assert np.linalg.norm(entries_k(idx, idx) - Ft) <= 1e-13 * np.linalg.norm(Ft)
    hk = O.build_h2(t, lists, entries_k, None, 1e-6, W.gaussian_omega(n, 256, 84), sampler_k)
    assert O.dense_rel_error(hk, full) <= 10 * 1e-6


def test_update_problem_at_16384_within_tolerance():
    # the paper's update problem (Sec. V-A) at N = 2^14: the covariance H2
    # (exp(-r/0.2), 3D, built at 1e-7) plus a symmetric rank-32 product,
    # recompressed at 1e-6; dense error against the exact sum within 10 tol
    w = W.paper_problem("update", 16384)
    X = w.points()
    t = O.build_cluster_tree(X, w.leaf_size)
    lists = O.dual_traversal(t, w.eta)
    kp = w.extra["operands"][0]
    A = O.dense_matrix(X, *kp)
    op = O.build_h2(t, lists, *kp, w.extra["operand_tol"], W.gaussian_omega(w.n, 256, 101),
                    O.dense_sampler(A))
    U, V = W.low_rank_factors(w.n, w.extra["rank"], w.extra["lowrank_seed"],
                              w.extra["lowrank_scale"])
    entries, sampler = O.low_rank_update(t, *O.h2_sum_operator([op]), U, V)
    h = O.build_h2(t, lists, entries, None, w.tol, W.gaussian_omega(w.n, 256, 102), sampler)
    A += U @ V.T
    assert h.l_top >= 3
    assert O.dense_rel_error(h, A) <= 10 * w.tol


# --- non-symmetric operators (separate row and column bases) -------------------


def _nonsym_problem(n=1024, seed=101, scale=0.02):
    X = W.uniform_points(n, 2, seed)
    t = O.build_cluster_tree(X, 16)
    lists = O.dual_traversal(t, 0.7)
    K = O.dense_matrix(X, O.K_EXP, (0.2, 1e-4))
    rng = np.random.default_rng(seed + 1)
    U = rng.standard_normal((n, 6)) / math.sqrt(n)
    V = rng.standard_normal((n, 6)) / math.sqrt(n)
    A = K + scale * n * U @ V.T          # not symmetric
    At = A[np.ix_(t.perm, t.perm)]
    return X, t, lists, A, At


def test_nonsym_build_on_a_symmetric_operator_matches_the_symmetric_build():
    # with A = A^T and Psi = Omega both sides see the same samples: the row and
    # the column bases are the symmetric construction's U
    n = 1024
    X, t, lists, A, _ = _nonsym_problem(n, scale=0.0)
    om = W.gaussian_omega(n, 256, 102)
    hs = O.build_h2(t, lists, O.K_EXP, (0.2, 1e-4), 1e-6, om, O.dense_sampler(A))
    hn = O.build_h2_nonsym(t, lists, lambda Ia, Ib: O._entries(t, O.K_EXP, (0.2, 1e-4), Ia, Ib),
                           1e-6, om, om, O.dense_sampler(A), O.dense_sampler(A.T))
    for tau, nd in hs.nodes.items():
        for side in (hn.rows[tau], hn.cols[tau]):
            assert side.k == nd.k and np.array_equal(side.J, nd.J)
            assert np.allclose(side.U, nd.U, rtol=0, atol=1e-12)
    G = W.gaussian_probe(n, 3, 0)
    y1, y2 = O.h2_matvec(hs, G), O.h2_matvec_nonsym(hn, G)
    assert np.linalg.norm(y1 - y2) <= 1e-12 * np.linalg.norm(y1)


def test_nonsym_build_meets_tolerance_where_the_symmetric_one_cannot():
    n, tol = 1024, 1e-6
    X, t, lists, A, At = _nonsym_problem(n)
    assert np.linalg.norm(A - A.T) > 0.1 * np.linalg.norm(A)
    entries = lambda Ia, Ib: At[np.ix_(Ia, Ib)]
    om, ps = W.gaussian_omega(n, 256, 103), W.gaussian_omega(n, 256, 104)
    hn = O.build_h2_nonsym(t, lists, entries, tol, om, ps, O.dense_sampler(A),
                           O.dense_sampler(A.T))
    assert hn.converged and hn.l_top >= 2
    dense = O.h2_matvec_nonsym(hn, np.eye(n))
    assert np.linalg.norm(dense - A) <= 10 * tol * np.linalg.norm(A)
    # one shared basis (the symmetric construction) misses the column space
    hs = O.build_h2(t, lists, entries, None, tol, om, O.dense_sampler(A))
    assert np.linalg.norm(O.h2_matvec(hs, np.eye(n)) - A) > 1e3 * tol * np.linalg.norm(A)


def test_nonsym_build_of_the_transpose_is_the_transpose():
    # swapping the operator for its transpose swaps the two sides exactly
    n, tol = 1024, 1e-6
    X, t, lists, A, At = _nonsym_problem(n)
    om, ps = W.gaussian_omega(n, 256, 105), W.gaussian_omega(n, 256, 106)
    h = O.build_h2_nonsym(t, lists, lambda Ia, Ib: At[np.ix_(Ia, Ib)], tol, om, ps,
                          O.dense_sampler(A), O.dense_sampler(A.T))
    hT = O.build_h2_nonsym(t, lists, lambda Ia, Ib: At.T[np.ix_(Ia, Ib)], tol, ps, om,
                           O.dense_sampler(A.T), O.dense_sampler(A))
    for tau in h.rows:
        assert np.array_equal(h.rows[tau].J, hT.cols[tau].J)
        assert np.array_equal(h.cols[tau].J, hT.rows[tau].J)
    M, MT = O.h2_matvec_nonsym(h, np.eye(n)), O.h2_matvec_nonsym(hT, np.eye(n))
    assert np.linalg.norm(MT - M.T) <= 1e-12 * np.linalg.norm(M)


def test_nonsym_update_of_an_h2_matrix():
    # the update use case with a non-symmetric product: H2(exp) + U V^T, U != V
    # (LU-type updates); entries from the operand's representation plus the
    # product's, samples of A and A^T from matvecs plus the product
    n, tol = 1024, 1e-6
    X = W.uniform_points(n, 2, 111)
    t = O.build_cluster_tree(X, 16)
    lists = O.dual_traversal(t, 0.7)
    kp = (O.K_EXP, (0.2, 0.0))
    K = O.dense_matrix(X, *kp)
    op = O.build_h2(t, lists, *kp, 1e-8, W.gaussian_omega(n, 256, 112), O.dense_sampler(K))
    rng = np.random.default_rng(113)
    U = rng.standard_normal((n, 4)) / math.sqrt(n) * 0.05 * n
    V = rng.standard_normal((n, 4)) / math.sqrt(n)
    base_entries, base_sampler = O.h2_sum_operator([op])
    entries, sampler = O.low_rank_update(t, base_entries, base_sampler, U, V)
    _, sampler_t = O.low_rank_update(t, base_entries, base_sampler, V, U)   # A^T = H2 + V U^T
    A = K + U @ V.T
    h = O.build_h2_nonsym(t, lists, entries, tol, W.gaussian_omega(n, 256, 114),
                          W.gaussian_omega(n, 256, 115), sampler, sampler_t)
    assert h.converged
    assert np.linalg.norm(O.h2_matvec_nonsym(h, np.eye(n)) - A) <= 10 * tol * np.linalg.norm(A)
