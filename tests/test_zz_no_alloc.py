"""The allocation-free evaluation entry point (ot_prox_evaluate_noalloc).

It exists for callers that cannot allocate device memory when they need an
answer (code inside another framework's memory pool, or a latency-critical
loop where cudaMalloc/cudaFree would synchronise the device).  It must give
what the allocating ot_prox_evaluate gives for the same state, on repeated
calls that share its fixed scratch array.  Kept in a file collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from synth import blob_pairs, rng_for

pytestmark = pytest.mark.gpu

NAMES = ("Mx", "My", "x0", "x1", "r", "a")
FIELDS = ("res_pri", "objective", "primal_feasible", "dual_obj", "rel_gap")


@pytest.mark.parametrize("B,H,W,mode", [(3, 40, 37, "prox"), (2, 64, 64, "fixed_first"), (1, 17, 130, "eval")])
def test_noalloc_matches_evaluate_twice(lib, B, H, W, mode):
    p0, p1 = blob_pairs(rng_for(0, 21 + W), B, H, W)
    d0 = torch.from_numpy(p0).cuda()
    d1 = torch.from_numpy(p1).cuda()
    with lib.OtProx(B, H, W, mu=3.0, rho=0.01, mode=mode) as s:
        s.set_input(d0, d1)
        s.step(120)
        ref = s.evaluate()
        st = s.get_state()                      # dense [B, H, W] device tensors
        prm = s.params
    ptrs = [d0.data_ptr(), d1.data_ptr()] + [st[k].data_ptr() for k in NAMES]
    for call in range(2):
        out = lib.ot_prox_result()
        rc = lib.ot_prox_evaluate_noalloc(ctypes.byref(prm), *ptrs, ctypes.byref(out), None)
        assert rc == 0, lib.ot_last_error().decode()
        for f in FIELDS:
            a, b = getattr(out, f), ref[f]
            assert abs(a - b) <= 1e-9 * max(abs(b), 1e-12), (call, f, a, b)
    assert ref["objective"] > 0


def test_noalloc_rejects_bad_arguments(lib):
    prm = lib.default_params(B=0, H=4, W=4)
    out = lib.ot_prox_result()
    rc = lib.ot_prox_evaluate_noalloc(ctypes.byref(prm), *([None] * 8), ctypes.byref(out), None)
    assert rc == -1
    prm = lib.default_params(B=70000, H=200, W=200)
    x = torch.zeros(4, device="cuda")
    rc = lib.ot_prox_evaluate_noalloc(ctypes.byref(prm), *([x.data_ptr()] * 8), ctypes.byref(out), None)
    assert rc == -1 and "maximum" in lib.ot_last_error().decode()
