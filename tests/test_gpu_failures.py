"""Failure detection on the GPU without a GPU fault: error statuses from the
host side (sampler errors, non-finite input) and a bounded in-kernel wait that
is made to run out (the producer warp withholds its first tile), after which
the device context stays usable."""
import ctypes
import time

import numpy as np
import pytest
import torch

from paper_2506_16759_gb300 import _lib, api
from paper_2506_16759_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def test_tensor_core_wait_runs_out_and_context_survives():
    lib = _lib.lib()
    t0 = time.perf_counter()
    st = lib.h2_selftest_wait_timeout(torch.cuda.current_stream().cuda_stream)
    dt = time.perf_counter() - t0
    assert st == 0, lib.h2_last_error()
    assert dt < 30.0
    # the context still works: a normal sketch afterwards
    X = W.uniform_points(2000, 3, 7)
    om = W.gaussian_omega(2000, 16, 8)
    y = api.ksum_sketch(gpu(X), W.K_EXP, (0.2, 0.0), gpu(om), prec="mixed")
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()


def test_sampler_error_status():
    X = W.uniform_points(1024, 2, 9)
    tree = api.ClusterTree(gpu(X), 32, 0.7)

    def sampler(ctx, omega_p, y_p, n, d, ld, stream):
        return 7   # the caller's sampler fails

    with pytest.raises(_lib.H2Error) as e:
        api.H2Matrix.build(tree, W.K_EXP, (0.2, 0.0), 1e-6, sketch="callback", sampler=sampler)
    assert e.value.status == -6
    # the library keeps working on the same device
    h = api.H2Matrix.build(tree, W.K_EXP, (0.2, 0.0), 1e-6)
    assert h.stats()["converged"]


def test_sampler_non_finite_values_rejected():
    X = W.uniform_points(1024, 2, 10)
    tree = api.ClusterTree(gpu(X), 32, 0.7)
    n = 1024

    eye = torch.eye(n, dtype=torch.float64, device="cuda:0")

    def sampler(ctx, omega_p, y_p, n_, d, ld, stream):
        # y = I * (a NaN panel): a sampler that produces non-finite values
        bad = torch.full((d * ld,), float("nan"), dtype=torch.float64, device="cuda:0")
        return _lib.lib().h2_dense_sketch(eye.data_ptr(), n, n,
                                          ctypes.cast(bad.data_ptr(), ctypes.c_void_p), ld,
                                          ctypes.cast(y_p, ctypes.c_void_p), ld, d, stream)

    with pytest.raises(_lib.H2Error) as e:
        api.H2Matrix.build(tree, W.K_EXP, (0.2, 0.0), 1e-6, sketch="callback", sampler=sampler)
    assert e.value.status == -7


def test_non_finite_points_rejected():
    X = W.uniform_points(512, 3, 11)
    X[100, 1] = np.nan
    with pytest.raises(_lib.H2Error) as e:
        api.ClusterTree(gpu(X), 32, 0.7)
    assert e.value.status == -7


def test_low_rank_term_argument_errors():
    # a low-rank term needs a sketch in original order, a rank of at most
    # 64 and both factors; each violation is an H2_ERR_ARG, not a fault
    n = 1024
    X = W.uniform_points(n, 2, 13)
    tree = api.ClusterTree(gpu(X), 32, 0.7)
    U, V = (gpu(a) for a in W.low_rank_factors(n, 4, 14, 1.0))
    with pytest.raises(_lib.H2Error) as e:
        api.H2Matrix.build(tree, "exp", (0.2, 1e-4), 1e-6, sketch="ksum", lowrank=(U, V))
    assert e.value.status == _lib.H2_ERR_ARG
    from oracle import h2_oracle as O
    A = gpu(O.dense_matrix(X, O.K_EXP, (0.2, 1e-4)))
    Ub, Vb = (gpu(a) for a in W.low_rank_factors(n, 65, 14, 1.0))
    with pytest.raises(_lib.H2Error) as e:
        api.H2Matrix.build(tree, "exp", (0.2, 1e-4), 1e-6, sketch="dense", dense_a=A,
                           lowrank=(Ub, Vb))
    assert e.value.status == _lib.H2_ERR_ARG
    # the context still works afterwards
    h = api.H2Matrix.build(tree, "exp", (0.2, 1e-4), 1e-6, sketch="dense", dense_a=A,
                           lowrank=(U, V))
    assert h.converged
