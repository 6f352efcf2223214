"""The C ABI: the library builds, loads and exports every function that
include/*.h declares; host-side validation (no GPU needed: invalid arguments
are rejected before any CUDA call)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cdll():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "otprox_build", os.path.join(ROOT, "paper_1909_00149_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = mod.build()
    return ctypes.CDLL(path)


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(ot_[a-z0-9_]+)\s*\(", src):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("ot_prox_create", "ot_prox_solve", "ot_prox_step", "ot_prox_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(cdll):
    missing = [n for n in declared_functions() if not hasattr(cdll, n)]
    assert not missing, missing


def test_binding_names_match_header():
    import paper_1909_00149_gb300 as otp
    from paper_1909_00149_gb300 import _abi
    declared = set(declared_functions())
    bound = {n for n, _, _ in _abi.PROTOTYPES}
    assert bound <= declared
    for n in bound:
        assert hasattr(otp, n)


def test_lambda_max_and_identity_blocks_match_oracle():
    import paper_1909_00149_gb300 as otp
    from oracle import grid
    from oracle import prox as P
    for H, W in ((1, 1), (1, 9), (64, 64), (256, 256), (7, 300)):
        assert abs(otp.ot_lambda_max(H, W) - grid.lambda_max(H, W)) <= 1e-12
    for mode, code in (("prox", 0), ("fixed_first", 1), ("eval", 2)):
        for bal in (False, True):
            ref = P.n_identity_blocks(P.ProxParams(mode=mode, balanced=bal))
            assert otp.ot_n_identity_blocks(code, int(bal)) == ref


def _create(**kw):
    import paper_1909_00149_gb300 as otp
    p = otp.default_params(**kw)
    h = ctypes.c_void_p()
    rc = otp.ot_prox_create(ctypes.byref(p), None, ctypes.byref(h))
    return rc, otp.ot_last_error().decode()


@pytest.mark.parametrize("kw,needle", [
    (dict(B=0, H=4, W=4), "B, H, W"),
    (dict(B=1, H=-3, W=4), "B, H, W"),
    (dict(B=1, H=4, W=4, mode=7), "mode"),
    (dict(B=1, H=4, W=4, p_exp=3), "p_exp"),
    (dict(B=1, H=4, W=4, mu=0.0), "mu"),
    (dict(B=1, H=4, W=4, rho=-1.0), "rho"),
    (dict(B=1, H=4, W=4, check_every=0), "check_every"),
    (dict(B=1, H=4, W=4, tau1=1.0, tau2=1.0), "Theorem 1"),
    (dict(B=1, H=4, W=4, tau1=0.5, tau2=0.25), "Theorem 1"),
    (dict(B=1, H=200, W=200, kernel="resident"), "resident"),
    (dict(B=1, H=4, W=4, kernel="temporal", tb_depth=5), "tb_depth"),
    (dict(B=1, H=4, W=4, kernel="temporal", tb_depth=1), "tb_depth"),
    (dict(B=1, H=4, W=4, kernel="temporal", algorithm="projection"), "TEMPORAL"),
    (dict(B=1, H=4, W=4, kernel=5), "kernel"),
])
def test_create_rejects_invalid_arguments(kw, needle):
    rc, msg = _create(**kw)
    assert rc == -1, (rc, msg)
    assert needle in msg


def test_inner_prox_rejects_the_temporal_kernel():
    """ot_rpca_* and ot_uotdf_* hold the inner prox's x planes as their z, w:
    the ping-ponged planes of temporal blocking are refused before any CUDA
    call."""
    import paper_1909_00149_gb300 as otp
    from paper_1909_00149_gb300 import _abi
    p = otp.rpca_default_params(T=4, H=8, W=8, prox_kernel=4)
    h = ctypes.c_void_p()
    assert otp.ot_rpca_create(ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert "OT_KERNEL_TEMPORAL" in otp.ot_last_error().decode()
    q = _abi.ot_uotdf_params()
    otp.ot_uotdf_default_params(ctypes.byref(q))
    q.B, q.H, q.W, q.prox_kernel = 2, 8, 8, 4
    assert otp.ot_uotdf_create(ctypes.byref(q), None, ctypes.byref(h)) == -1
    assert "OT_KERNEL_TEMPORAL" in otp.ot_last_error().decode()


def test_theorem1_boundary():
    """Steps exactly at the bound are rejected, just inside accepted by the
    validation (the accepted case then allocates, so only the rejection is
    exercised here without a GPU)."""
    import paper_1909_00149_gb300 as otp
    L = otp.ot_lambda_max(8, 8) + 3
    t = (1.0 / L) ** 0.5
    rc, msg = _create(B=1, H=8, W=8, tau1=t * 1.0000001, tau2=t)
    assert rc == -1 and "Theorem 1" in msg


def test_null_arguments():
    import paper_1909_00149_gb300 as otp
    assert otp.ot_prox_create(None, None, None) == -1
    assert otp.ot_prox_step(None, 1) == -1
    assert otp.ot_prox_solve(None, None) == -1
    assert otp.ot_prox_destroy(None) == 0
    # every handle-taking call checks its pointers before any CUDA call
    for name, args in [("ot_rpca_step", (None, 1)), ("ot_rpca_iterate_checked", (None, 1, None)),
                       ("ot_rpca_step_profiled", (None, None)), ("ot_debug_grid_barrier", (1, 0, None, None)),
                       ("ot_prox_warm_start", (None, None, 0.0)), ("ot_unet_forward", (None, None, None, 1)),
                       ("ot_unet_param_count", (None,)), ("ot_prox_batch_step", (None, 1))]:
        assert getattr(otp, name)(*args) == -1, name
        assert otp.ot_last_error().decode().startswith(name), (name, otp.ot_last_error())
    assert otp.ot_rpca_destroy(None) == 0 and otp.ot_unet_destroy(None) == 0


def test_param_structs_match_their_ctypes_mirrors(cdll):
    """The default-parameter calls write exactly the C structs: a buffer one
    ctypes-size long plus a sentinel tail keeps its tail, so the C struct is
    no larger than the binding's mirror; the fields the mirror names come back
    with the documented defaults."""
    from paper_1909_00149_gb300 import _abi
    for name, cls in (("ot_rpca_default_params", _abi.ot_rpca_params),
                      ("ot_prox_default_params", _abi.ot_prox_params)):
        n = ctypes.sizeof(cls)
        buf = (ctypes.c_ubyte * (n + 64))(*([0xA5] * (n + 64)))
        fn = getattr(cdll, name)
        fn.restype = None
        fn(ctypes.byref(buf))
        assert bytes(buf[n:]) == b"\xa5" * 64, name
        p = cls.from_buffer_copy(bytes(buf[:n]))
        if cls is _abi.ot_rpca_params:
            assert p.signed_fg == 0 and p.use_graph == 1 and p.rho == 1.0 and p.kappa == 0.005
        else:
            assert p.tb_depth == 4 and p.beta == 1.0 and p.check_every == 10


def test_committed_warm_start_weights_fit_the_network(cdll):
    """The warm-start parameters that the benchmark loads have the network's
    layout (weights [co, ci, k, k] then biases [co] per layer) and a record
    of the training run that wrote them."""
    import numpy as np
    from paper_1909_00149_gb300 import unet_layer_specs, warmstart as WS
    with np.load(WS.WEIGHTS) as d:
        n = sum(co * ci * k * k + co for _, ci, co, k in unet_layer_specs(int(d["base_channels"])))
        assert d["params"].shape == (n,) and d["params"].dtype == np.float32
        assert np.all(np.isfinite(d["params"]))
        assert int(d["pairs"]) >= 20000 and int(d["size"]) == 256
        assert float(d["mu"]) == 3.0 and float(d["rho"]) == 0.01 and float(d["tol"]) == 1e-5
