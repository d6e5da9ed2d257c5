"""The pipe-throughput probes behind the roofline fractions return plausible
rates on this device (they are measurements, so only loose bounds apply)."""
import ctypes

import pytest
import torch

from paper_2506_16759_gb300 import _lib

pytestmark = pytest.mark.gpu

# which -> (low, high): FP64 and FP32 TFLOP/s, exp2 G op/s, FP16 and TF32
# tensor TFLOP/s, square root and reciprocal square root G op/s.  The bounds are generous brackets around GB300's unit
# counts and clocks, not targets.
BOUNDS = {0: (0.2, 10.0), 1: (20.0, 150.0), 2: (500.0, 20000.0), 3: (300.0, 4000.0),
          4: (150.0, 2500.0), 5: (500.0, 20000.0), 6: (500.0, 20000.0)}


@pytest.mark.parametrize("which", sorted(BOUNDS))
def test_peak_probe(which):
    v = ctypes.c_double()
    st = _lib.lib().h2_measure_peak(which, torch.cuda.current_stream().cuda_stream,
                                    ctypes.byref(v))
    assert st == 0, _lib.lib().h2_last_error()
    lo, hi = BOUNDS[which]
    assert lo <= v.value <= hi, v.value
