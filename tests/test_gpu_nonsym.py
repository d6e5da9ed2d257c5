"""Non-symmetric operators on the GPU (separate row and column bases, Sec. II-A
and Sec. III) against the oracle's construction, through the C ABI.

Bars: row and column ranks and skeletons of every level as in the oracle
(FP64), matvec within 1e-10 (FP64) and 1e-5 (mixed precision) of the
oracle's, approximation error within 10 tol of the dense operator.
"""
import ctypes
import math

import numpy as np
import pytest
import torch

from oracle import h2_oracle as O
from paper_2506_16759_gb300 import _lib, api
from paper_2506_16759_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _problem(n, dim, seed, scale, rank=6):
    """exp(-r/0.2) + 1e-4 nugget plus scale * n * U V^T (U != V)."""
    X = W.uniform_points(n, dim, seed)
    K = O.dense_matrix(X, O.K_EXP, (0.2, 1e-4))
    rng = np.random.default_rng(seed + 1)
    U = rng.standard_normal((n, rank)) / math.sqrt(n)
    V = rng.standard_normal((n, rank)) / math.sqrt(n)
    Us = np.asfortranarray(scale * n * U)
    return X, K, Us, np.asfortranarray(V), K + Us @ V.T


def _check_sides(h, t, ho):
    for level in range(1, ho.l_top + 1):
        nodes = list(t.nodes_at_depth(t.level_depth(level)))
        ranks, skel, eps, d = h.export_level(level)
        assert ranks.tolist() == [ho.rows[v].k for v in nodes], f"row ranks, level {level}"
        want = np.concatenate([t.perm[ho.rows[v].Itil] for v in nodes])
        assert np.array_equal(skel, want), f"row skeletons, level {level}"
        assert d == ho.d_level[level]
        assert eps == pytest.approx(ho.eps_level[level], rel=1e-12)
        cranks, cskel = h.export_col_level(level)
        assert cranks.tolist() == [ho.cols[v].k for v in nodes], f"column ranks, level {level}"
        want = np.concatenate([t.perm[ho.cols[v].Itil] for v in nodes])
        assert np.array_equal(cskel, want), f"column skeletons, level {level}"


@pytest.mark.parametrize("n,dim,leaf,seed", [(2048, 2, 32, 201), (3000, 3, 32, 202)])
def test_nonsym_dense_sketch_matches_oracle(n, dim, leaf, seed):
    tol = 1e-6
    X, K, U, V, A = _problem(n, dim, seed, 0.02)
    assert np.linalg.norm(A - A.T) > 0.05 * np.linalg.norm(A)
    om, ps = W.gaussian_omega(n, 256, seed + 2), W.gaussian_omega(n, 256, seed + 3)
    t = O.build_cluster_tree(X, leaf)
    lists = O.dual_traversal(t, 0.7)
    At = A[np.ix_(t.perm, t.perm)]
    ho = O.build_h2_nonsym(t, lists, lambda Ia, Ib: At[np.ix_(Ia, Ib)], tol, om, ps,
                           O.dense_sampler(A), O.dense_sampler(A.T))
    assert ho.converged and ho.l_top >= 2
    tree = api.ClusterTree(gpu(X), leaf, 0.7)
    G = W.gaussian_probe(n, 4, 5)
    yo = O.h2_matvec_nonsym(ho, G)
    AG = A @ G
    for prec, bar in (("fp64", 1e-10), ("mixed", 1e-5)):
        # samples K Omega + U (V^T Omega) and K Psi + V (U^T Psi): the dense
        # matrix is the kernel part, the library adds the product's share
        h = api.H2Matrix.build(tree, W.K_EXP, (0.2, 1e-4), tol, omega=gpu(om), psi=gpu(ps),
                               nonsym=True, sketch="dense", dense_a=gpu(K), prec=prec,
                               lowrank=(gpu(U), gpu(V)))
        assert h.converged
        if prec == "fp64":
            _check_sides(h, t, ho)
        y = h.matvec(gpu(G)).cpu().numpy()
        assert np.linalg.norm(y - yo) <= bar * np.linalg.norm(yo), prec
        assert np.linalg.norm(y - AG) <= 10 * tol * np.linalg.norm(AG), prec


def test_nonsym_h2_matvec_sampler():
    # the paper's O(N) sampler: the matvec of an H2 matrix of the kernel
    # (prebuilt at 1e-8) plus U (V^T x); A^T x the same with U and V swapped
    n, dim, leaf, tol, seed = 2048, 3, 32, 1e-6, 203
    X, K, U, V, A = _problem(n, dim, seed, 0.02)
    om, ps = W.gaussian_omega(n, 256, seed + 2), W.gaussian_omega(n, 256, seed + 3)
    om_pre = W.gaussian_omega(n, 256, seed + 4)
    t = O.build_cluster_tree(X, leaf)
    lists = O.dual_traversal(t, 0.7)
    pre_o = O.build_h2(t, lists, O.K_EXP, (0.2, 1e-4), 1e-8, om_pre, O.dense_sampler(K))
    samp = lambda Om: O.h2_matvec(pre_o, Om) + U @ (V.T @ Om)
    samp_t = lambda Ps: O.h2_matvec(pre_o, Ps) + V @ (U.T @ Ps)
    At = A[np.ix_(t.perm, t.perm)]
    ho = O.build_h2_nonsym(t, lists, lambda Ia, Ib: At[np.ix_(Ia, Ib)], tol, om, ps, samp,
                           samp_t)
    tree = api.ClusterTree(gpu(X), leaf, 0.7)
    pre = api.H2Matrix.build(tree, W.K_EXP, (0.2, 1e-4), 1e-8, omega=gpu(om_pre))
    G = W.gaussian_probe(n, 4, 6)
    yo = O.h2_matvec_nonsym(ho, G)
    for prec, bar in (("fp64", 1e-10), ("mixed", 1e-5)):
        h = api.H2Matrix.build(tree, W.K_EXP, (0.2, 1e-4), tol, omega=gpu(om), psi=gpu(ps),
                               nonsym=True, sketch="h2sum", operands=[pre], prec=prec,
                               lowrank=(gpu(U), gpu(V)))
        if prec == "fp64":
            _check_sides(h, t, ho)
        y = h.matvec(gpu(G)).cpu().numpy()
        assert np.linalg.norm(y - yo) <= bar * np.linalg.norm(yo), prec
        assert np.linalg.norm(y - A @ G) <= 10 * tol * np.linalg.norm(A @ G), prec


def test_nonsym_callback_samplers_match_the_dense_sketch():
    # the caller's samplers: sampler gives K x, sampler_t gives K^T x (both
    # through the library's dense product); the build equals the dense-sketch
    # build bit for bit and calls both samplers
    n, leaf, tol, seed = 2048, 32, 1e-6, 206
    X, K, U, V, A = _problem(n, 2, seed, 0.02)
    om, ps = W.gaussian_omega(n, 256, seed + 2), W.gaussian_omega(n, 256, seed + 3)
    Kd = gpu(K)
    Kt = gpu(np.ascontiguousarray(K.T))
    L = _lib.lib()
    calls = {"A": 0, "At": 0}

    def make(mat, key):
        def f(ctx, x_p, y_p, nn, d, ld, stream):
            calls[key] += d
            return L.h2_dense_sketch(mat.data_ptr(), nn, nn, ctypes.cast(x_p, ctypes.c_void_p), ld,
                                     ctypes.cast(y_p, ctypes.c_void_p), ld, d, stream)
        return f

    tree = api.ClusterTree(gpu(X), leaf, 0.7)
    hc = api.H2Matrix.build(tree, W.K_EXP, (0.2, 1e-4), tol, omega=gpu(om), psi=gpu(ps),
                            nonsym=True, sketch="callback", sampler=make(Kd, "A"),
                            sampler_t=make(Kt, "At"), lowrank=(gpu(U), gpu(V)))
    hd = api.H2Matrix.build(tree, W.K_EXP, (0.2, 1e-4), tol, omega=gpu(om), psi=gpu(ps),
                            nonsym=True, sketch="dense", dense_a=Kd, lowrank=(gpu(U), gpu(V)))
    assert calls["A"] >= 32 and calls["At"] == calls["A"]
    G = gpu(W.gaussian_probe(n, 2, 8))
    assert torch.equal(hc.matvec(G), hd.matvec(G))


def test_nonsym_on_a_symmetric_operator_matches_the_symmetric_build():
    # A = A^T and Psi = Omega: both sides of the non-symmetric build equal the
    # symmetric build's bases, and the matvecs agree
    n, leaf, tol = 2048, 32, 1e-6
    X, K, _, _, _ = _problem(n, 2, 204, 0.0)
    om = W.gaussian_omega(n, 256, 205)
    tree = api.ClusterTree(gpu(X), leaf, 0.7)
    hs = api.H2Matrix.build(tree, W.K_EXP, (0.2, 1e-4), tol, omega=gpu(om), sketch="dense",
                            dense_a=gpu(K))
    hn = api.H2Matrix.build(tree, W.K_EXP, (0.2, 1e-4), tol, omega=gpu(om), psi=gpu(om),
                            nonsym=True, sketch="dense", dense_a=gpu(K))
    for level in range(1, tree.info.l_top + 1):
        r, sk, _, _ = hs.export_level(level)
        r1, sk1, _, _ = hn.export_level(level)
        r2, sk2 = hn.export_col_level(level)
        assert np.array_equal(r, r1) and np.array_equal(r, r2)
        assert np.array_equal(sk, sk1) and np.array_equal(sk, sk2)
    G = gpu(W.gaussian_probe(n, 3, 7))
    y1, y2 = hs.matvec(G), hn.matvec(G)
    assert float(torch.linalg.norm(y1 - y2) / torch.linalg.norm(y1)) <= 1e-12
