"""dh_conserved_totals_static: the allocation-free variant of the conserved-totals reduction.

It exists for callers that cannot allocate device memory (an embedding framework that owns the
device-memory budget, or a time-critical loop that must not pay for cudaMalloc's implicit
device synchronisation).  It keeps its partial sums in a fixed file-scope device array, so two
calls in a row reuse the same scratch; both must agree with the context-based
dh_conserved_totals.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2512_13403_b300 import _lib, inputs
from tests.gpu_util import solver, to_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,shape", [("f64", (12, 16, 20)), ("f32", (64, 64, 72))])
def test_static_scratch_totals_match_context_totals(prec, shape):
    lib = _lib.load()
    U = to_gpu(inputs.decaying_turbulence(shape, seed=4, sigma=0.5, mach=1.0, p_sigma=0.2), prec)
    s = solver(shape, prec)
    code = _lib.DH_F64 if prec == "f64" else _lib.DH_F32
    stream = torch.cuda.current_stream()
    base = U
    for call in range(2):
        # a different state on each call, through the same static scratch
        U = (base * (1.0 + call)).contiguous()
        s.init_state(U)
        ref = s.conserved_totals()
        scale = U.double().abs().sum(dim=(1, 2, 3)).cpu().tolist()
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.dh_conserved_totals_static(C.c_void_p(U.data_ptr()), code, U[0].numel(),
                                            C.c_void_p(out.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == _lib.DH_OK, lib.dh_last_error(None)
        stream.synchronize()
        got = out.cpu().tolist()
        for f in range(5):
            # same float64 sums, different blocking: agreement to round-off of the sum of |U|
            assert abs(got[f] - ref[f]) <= 1e-13 * scale[f], (call, f, got[f], ref[f])


def test_static_scratch_rejects_oversized_grid():
    lib = _lib.load()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    U = torch.zeros(5 * 8, dtype=torch.float64, device="cuda")
    st = lib.dh_conserved_totals_static(C.c_void_p(U.data_ptr()), _lib.DH_F64, 2 ** 28 + 1,
                                        C.c_void_p(out.data_ptr()), None)
    assert st == _lib.DH_ERR_ARG
    assert b"268435456" in lib.dh_last_error(None)
