"""The allocation-free QR statistic (h2_batched_qr_mindiag_static) against the
allocating entry point, through the C ABI.

Some callers cannot allocate device memory while they run (another component
owns it, or an allocation would break their memory budget); this entry point
serves them from a workspace compiled into the library.  This file is
collected last so that a failure here stops a -x run only after every other
test has run; it also passes alone in a fresh process (the first call there
does the per-device set-up).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2506_16759_gb300 import _lib, api

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _panels(seed):
    rng = np.random.default_rng(seed)
    shapes = [(64, 32), (100, 48), (33, 32), (8, 16), (300, 96), (129, 1), (64, 64), (200, 150)]
    return [rng.standard_normal((m, d)) @ np.diag(rng.uniform(1e-6, 2, d)) for m, d in shapes]


def _static_call(panels):
    m, d, off, flat, _, _ = api._pack_panels([torch.from_numpy(p).to(DEV) for p in panels])
    out = torch.full((len(panels),), -1.0, dtype=torch.float64, device=DEV)
    st = _lib.lib().h2_batched_qr_mindiag_static(
        len(panels), m.data_ptr(), d.data_ptr(), off.data_ptr(), flat.data_ptr(),
        out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return st, out.cpu().numpy()


def _raw_call(m, d, off, flat, n, out=None):
    if out is None:
        out = torch.full((n,), -1.0, dtype=torch.float64, device=DEV)
    st = _lib.lib().h2_batched_qr_mindiag_static(
        n, m.data_ptr(), d.data_ptr(), off.data_ptr(), flat.data_ptr(), out.data_ptr(),
        torch.cuda.current_stream().cuda_stream)
    return st, out.cpu().numpy()


def test_static_workspace_matches_allocating_entry_point():
    L = _lib.lib()
    for seed in (1, 2):                    # two calls in a row
        panels = _panels(seed)
        m, d, off, flat, _, _ = api._pack_panels([torch.from_numpy(p).to(DEV) for p in panels])
        out = torch.full((len(panels),), -1.0, dtype=torch.float64, device=DEV)
        torch.cuda.synchronize()
        reserved, requests = torch.cuda.memory_reserved(DEV), L.h2_device_allocations()
        st, got = _raw_call(m, d, off, flat, len(panels), out)
        # the defining property: no device memory requested, by the library
        # or through torch
        assert L.h2_device_allocations() == requests
        assert torch.cuda.memory_reserved(DEV) == reserved
        assert st == 0, L.h2_last_error()
        want = api.batched_qr_mindiag([torch.from_numpy(p).to(DEV) for p in panels]).cpu().numpy()
        for g, w, p in zip(got, want, panels):
            if p.shape[0] <= p.shape[1]:
                assert g == 0.0 and w == 0.0
            else:
                assert g == pytest.approx(w, rel=1e-11)


def test_static_workspace_rejects_oversize_requests():
    # 2 x (2048 x 600) doubles exceed the 2097152-double workspace
    big = [np.ones((2048, 600)), np.ones((2048, 600))]
    st, got = _static_call(big)
    assert st == -1
    assert b"static workspace" in _lib.lib().h2_last_error()
    assert np.isnan(got).any()
    # the next call starts clean
    st, _ = _static_call(_panels(3))
    assert st == 0


def test_static_workspace_rejects_bad_shapes():
    # d = 0 with m > 0, and a negative d ahead of a valid panel: both get NaN
    # and the call reports an argument error; the valid panel is still right
    rng = np.random.default_rng(4)
    good = rng.standard_normal((50, 20))
    want = api.batched_qr_mindiag([torch.from_numpy(good).to(DEV)]).cpu().numpy()[0]
    for shapes in ([(10, 0)], [(10, -3), (50, 20)]):
        ms = torch.tensor([a for a, _ in shapes], dtype=torch.int32, device=DEV)
        ds = torch.tensor([b for _, b in shapes], dtype=torch.int32, device=DEV)
        offs = torch.zeros(len(shapes), dtype=torch.int64, device=DEV)
        flat = torch.from_numpy(good.T.reshape(-1).copy()).to(DEV)   # column-major 50 x 20
        st, got = _raw_call(ms, ds, offs, flat, len(shapes))
        assert st == -1
        assert b"m < 0 or d < 1" in _lib.lib().h2_last_error()
        assert np.isnan(got[0])
        if len(shapes) == 2:
            assert got[1] == pytest.approx(want, rel=1e-11)
    st, _ = _static_call(_panels(5))        # and the next call starts clean
    assert st == 0
