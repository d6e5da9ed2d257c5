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


def test_static_workspace_matches_allocating_entry_point():
    for seed in (1, 2):                    # two calls in a row
        panels = _panels(seed)
        st, got = _static_call(panels)
        assert st == 0, _lib.lib().h2_last_error()
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
