"""GB300 (sm_103a) unbalanced Beckmann-OT proximal solver -- Python binding.

Thin marshalling layer over the C ABI of include/otprox.h (libotprox.so):
every step of the computation runs in the library's CUDA kernels.  PyTorch
is used only for device memory and the current CUDA stream.  If the library
is not built, importing this package raises: there is no CPU fallback.

The raw C functions are re-exported under their C names (``ot_prox_create``
etc.); :class:`OtProx` wraps a handle with tensor arguments.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _abi
from ._abi import (KERNELS, MODES, NORMS, OT_ENONFINITE, OT_ENOTCONV, OT_OK, STATUS_NAMES, ot_prox_params,
                   ot_prox_result)

_lib = _abi.load()
LIB_PATH = _abi.LIB_PATH

for _name, _res, _args in _abi.PROTOTYPES:
    globals()[_name] = getattr(_lib, _name)


class OtError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.ot_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str, ok=(OT_OK,)) -> int:
    if code not in ok:
        raise OtError(code, where)
    return code


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class _Arrays:
    """Keeps numpy temporaries alive for the duration of a call."""

    def __init__(self, n: int):
        self.n = n
        self.keep = []

    def ptr(self, x, writable=False):
        if x is None:
            return None
        try:
            import torch
            if isinstance(x, torch.Tensor):
                if x.dtype != torch.float32 or not x.is_contiguous():
                    raise ValueError("tensors must be contiguous float32")
                if x.numel() != self.n:
                    raise ValueError(f"expected {self.n} elements, got {x.numel()}")
                return x.data_ptr()
        except ImportError:
            pass
        a = np.asarray(x)
        if writable:
            if a.dtype != np.float32 or not a.flags.c_contiguous:
                raise ValueError("output arrays must be C-contiguous float32")
        else:
            a = np.ascontiguousarray(a, dtype=np.float32)
        if a.size != self.n:
            raise ValueError(f"expected {self.n} elements, got {a.size}")
        self.keep.append(a)
        return a.ctypes.data


def default_params(**kw) -> ot_prox_params:
    p = ot_prox_params()
    _lib.ot_prox_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k == "mode":
            v = MODES[v] if isinstance(v, str) else v
        elif k == "norm":
            v = NORMS[v] if isinstance(v, str) else v
        elif k == "kernel":
            v = KERNELS[v] if isinstance(v, str) else v
        elif k == "algorithm":
            v = _abi.ALGORITHMS[v] if isinstance(v, str) else v
        elif k == "precision":
            v = _abi.PRECISIONS[v] if isinstance(v, str) else v
        elif k in ("balanced", "use_graph"):
            v = int(bool(v))
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k!r}")
        setattr(p, k, v)
    return p


class OtProx:
    """B independent prox problems of eq. (Prox_UOT) on an H x W grid."""

    def __init__(self, B: int, H: int, W: int, stream=None, **params):
        self.B, self.H, self.W = int(B), int(H), int(W)
        p = default_params(B=self.B, H=self.H, W=self.W, **params)
        h = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        check(_lib.ot_prox_create(ctypes.byref(p), self._stream, ctypes.byref(h)), "ot_prox_create")
        self.h = h
        self.params = ot_prox_params()
        check(_lib.ot_prox_get_params(self.h, ctypes.byref(self.params)), "ot_prox_get_params")

    @property
    def n(self) -> int:
        return self.B * self.H * self.W

    def close(self):
        if getattr(self, "h", None):
            _lib.ot_prox_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_input(self, p0, p1):
        A = _Arrays(self.n)
        check(_lib.ot_prox_set_input(self.h, A.ptr(p0), A.ptr(p1)), "ot_prox_set_input")

    def step(self, n_iter: int):
        check(_lib.ot_prox_step(self.h, int(n_iter)), "ot_prox_step")

    def solve(self) -> dict:
        r = ot_prox_result()
        check(_lib.ot_prox_solve(self.h, ctypes.byref(r)), "ot_prox_solve", ok=(OT_OK, OT_ENOTCONV))
        return r.as_dict()

    def check_interval(self, n_iter: int) -> dict:
        r = ot_prox_result()
        check(_lib.ot_prox_check_interval(self.h, int(n_iter), ctypes.byref(r)), "ot_prox_check_interval")
        return r.as_dict()

    def step_timed(self, n_iter: int) -> float:
        ms = ctypes.c_double()
        check(_lib.ot_prox_step_timed(self.h, int(n_iter), ctypes.byref(ms)), "ot_prox_step_timed")
        return ms.value

    def evaluate(self) -> dict:
        r = ot_prox_result()
        check(_lib.ot_prox_evaluate(self.h, ctypes.byref(r)), "ot_prox_evaluate", ok=(OT_OK, OT_ENONFINITE))
        return r.as_dict()

    def reset(self):
        check(_lib.ot_prox_reset(self.h), "ot_prox_reset")

    def get_state(self, device=None) -> dict:
        """State as float32 tensors [B, H, W] (on ``device``, default cuda)."""
        import torch
        dev = torch.device("cuda") if device is None else torch.device(device)
        names = ("Mx", "My", "x0", "x1", "r", "a")
        out = {k: torch.empty((self.B, self.H, self.W), dtype=torch.float32, device=dev,
                              pin_memory=(dev.type == "cpu" and torch.cuda.is_available()))
               for k in names}
        A = _Arrays(self.n)
        check(_lib.ot_prox_get_state(self.h, *(A.ptr(out[k], True) for k in names)), "ot_prox_get_state")
        torch.cuda.synchronize()
        return out

    def set_state(self, Mx=None, My=None, x0=None, x1=None, r=None, a=None):
        A = _Arrays(self.n)
        check(_lib.ot_prox_set_state(self.h, A.ptr(Mx), A.ptr(My), A.ptr(x0), A.ptr(x1), A.ptr(r), A.ptr(a)),
              "ot_prox_set_state")

    def warm_start(self, pred, gate: float = 0.0):
        """Warm state from a prediction [B, 4, H, W] (Mx, My, r, a) CUDA
        tensor, x from the x-step's fixed point; with gate > 0 only near
        mass (ot_prox_warm_start)."""
        import torch
        if not (isinstance(pred, torch.Tensor) and pred.is_cuda and pred.dtype == torch.float32
                and pred.is_contiguous() and pred.numel() == 4 * self.n):
            raise ValueError("pred must be a contiguous float32 CUDA tensor of B x 4 x H x W values")
        check(_lib.ot_prox_warm_start(self.h, pred.data_ptr(), float(gate)), "ot_prox_warm_start")


def rpca_default_params(**kw) -> "_abi.ot_rpca_params":
    p = _abi.ot_rpca_params()
    _lib.ot_rpca_default_params(ctypes.byref(p))
    for k, v in kw.items():
        k = "lambda_" if k in ("lam", "lambda") else k
        if k == "prox_kernel":
            v = KERNELS[v] if isinstance(v, str) else v
        elif k in ("use_graph", "signed_fg"):
            v = int(bool(v))
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k!r}")
        setattr(p, k, v)
    return p


class Rpca:
    """RPCA+UOT-DF (Algorithm 3, Phi = I) on a T-frame H x W video."""

    def __init__(self, T: int, H: int, W: int, stream=None, **params):
        self.T, self.H, self.W = int(T), int(H), int(W)
        p = rpca_default_params(T=self.T, H=self.H, W=self.W, **params)
        h = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        check(_lib.ot_rpca_create(ctypes.byref(p), self._stream, ctypes.byref(h)), "ot_rpca_create")
        self.h = h
        self.params = _abi.ot_rpca_params()
        check(_lib.ot_rpca_get_params(self.h, ctypes.byref(self.params)), "ot_rpca_get_params")

    def close(self):
        if getattr(self, "h", None):
            _lib.ot_rpca_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_input(self, Y):
        A = _Arrays(self.T * self.H * self.W)
        check(_lib.ot_rpca_set_input(self.h, A.ptr(Y)), "ot_rpca_set_input")

    def step(self, n_outer: int):
        check(_lib.ot_rpca_step(self.h, int(n_outer)), "ot_rpca_step")

    def iterate_checked(self, n_outer: int = 1) -> dict:
        r = _abi.ot_rpca_result()
        check(_lib.ot_rpca_iterate_checked(self.h, int(n_outer), ctypes.byref(r)), "ot_rpca_iterate_checked")
        return r.as_dict()

    def solve(self) -> dict:
        r = _abi.ot_rpca_result()
        check(_lib.ot_rpca_solve(self.h, ctypes.byref(r)), "ot_rpca_solve", ok=(OT_OK, OT_ENOTCONV))
        return r.as_dict()

    def step_profiled(self) -> list:
        """Two outer iterations; device ms of their eight phases (see the C
        header: pre, Gram, eigensolver, the second apply, prox, post, the
        fused pass between them (with the first apply and the second Gram for
        T <= 64), the second Gram otherwise)."""
        ms = (ctypes.c_double * 8)()
        check(_lib.ot_rpca_step_profiled(self.h, ms), "ot_rpca_step_profiled")
        return list(ms)

    def reset(self):
        check(_lib.ot_rpca_reset(self.h), "ot_rpca_reset")

    def get(self, name: str, device=None, out=None):
        """Copy of a variable ([T] or [T-1] x H x W float32) into ``out`` (host
        or device, e.g. pinned host memory) or a new tensor on ``device``."""
        import torch
        nf = self.T - 1 if name in _abi.RPCA_PAIR_VARS else self.T
        if out is None:
            dev = torch.device("cuda") if device is None else torch.device(device)
            out = torch.empty((nf, self.H, self.W), dtype=torch.float32, device=dev)
        A = _Arrays(nf * self.H * self.W)
        check(_lib.ot_rpca_get(self.h, _abi.RPCA_VARS[name], A.ptr(out, True)), "ot_rpca_get")
        return out


class ProxBatch:
    """Algorithm 1 on sequences of uneven size in one launch per iteration.
    ``sizes``: list of (B_i, H_i, W_i); ``params``: the shared ot_prox_params
    fields (mode, norm, mu, rho, tol, max_iter, check_every, use_graph, ...)."""

    def __init__(self, sizes, stream=None, **params):
        self.sizes = [(int(b), int(h), int(w)) for b, h, w in sizes]
        n = len(self.sizes)
        arr = lambda k: (ctypes.c_int32 * n)(*[s[k] for s in self.sizes])
        p = default_params(**params)
        h = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        check(_lib.ot_prox_batch_create(n, arr(0), arr(1), arr(2), ctypes.byref(p), self._stream, ctypes.byref(h)),
              "ot_prox_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            _lib.ot_prox_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_input(self, seq: int, p0, p1):
        b, hh, w = self.sizes[seq]
        A = _Arrays(b * hh * w)
        check(_lib.ot_prox_batch_set_input(self.h, int(seq), A.ptr(p0), A.ptr(p1)), "ot_prox_batch_set_input")

    def step(self, n_iter: int):
        check(_lib.ot_prox_batch_step(self.h, int(n_iter)), "ot_prox_batch_step")

    def solve(self):
        n = len(self.sizes)
        res = (_abi.ot_prox_batch_result * n)()
        launches = ctypes.c_int32()
        check(_lib.ot_prox_batch_solve(self.h, res, ctypes.byref(launches)), "ot_prox_batch_solve",
              ok=(OT_OK, OT_ENOTCONV))
        return [r.as_dict() for r in res], launches.value

    def set_config(self, kernel="tma", tile_rows: int = 16, ctas_per_sm: int = 1):
        k = KERNELS[kernel] if isinstance(kernel, str) else kernel
        check(_lib.ot_prox_batch_set_config(self.h, int(k), int(tile_rows), int(ctas_per_sm)),
              "ot_prox_batch_set_config")

    def autotune(self) -> dict:
        k, th, cp, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        check(_lib.ot_prox_batch_autotune(self.h, ctypes.byref(k), ctypes.byref(th), ctypes.byref(cp),
                                          ctypes.byref(ms)), "ot_prox_batch_autotune")
        names = {v: n for n, v in KERNELS.items()}
        return {"kernel": names.get(k.value, k.value), "tile_rows": th.value, "ctas_per_sm": cp.value,
                "ms_per_iter": ms.value}

    def reset(self):
        check(_lib.ot_prox_batch_reset(self.h), "ot_prox_batch_reset")

    def get_state(self, seq: int, device=None) -> dict:
        import torch
        b, hh, w = self.sizes[seq]
        dev = torch.device("cuda") if device is None else torch.device(device)
        names = ("Mx", "My", "x0", "x1", "r", "a")
        out = {k: torch.empty((b, hh, w), dtype=torch.float32, device=dev) for k in names}
        A = _Arrays(b * hh * w)
        check(_lib.ot_prox_batch_get_state(self.h, int(seq), *(A.ptr(out[k], True) for k in names)),
              "ot_prox_batch_get_state")
        return out


def uotdf_default_params(**kw) -> "_abi.ot_uotdf_params":
    p = _abi.ot_uotdf_params()
    _lib.ot_uotdf_default_params(ctypes.byref(p))
    for k, v in kw.items():
        k = "lambda_" if k in ("lam", "lambda") else k
        if k == "prox_kernel":
            v = KERNELS[v] if isinstance(v, str) else v
        elif k == "norm":
            v = NORMS[v] if isinstance(v, str) else v
        if not hasattr(p, k):
            raise TypeError(f"unknown parameter {k!r}")
        setattr(p, k, v)
    return p


class Uotdf:
    """UOT-DF / BPDN+UOT-DF (Algorithm 2, Phi = I) on B independent H x W frames."""

    def __init__(self, B: int, H: int, W: int, stream=None, **params):
        self.B, self.H, self.W = int(B), int(H), int(W)
        p = uotdf_default_params(B=self.B, H=self.H, W=self.W, **params)
        h = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        check(_lib.ot_uotdf_create(ctypes.byref(p), self._stream, ctypes.byref(h)), "ot_uotdf_create")
        self.h = h
        self.params = _abi.ot_uotdf_params()
        check(_lib.ot_uotdf_get_params(self.h, ctypes.byref(self.params)), "ot_uotdf_get_params")

    def close(self):
        if getattr(self, "h", None):
            _lib.ot_uotdf_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_input(self, y, s0):
        A = _Arrays(self.B * self.H * self.W)
        check(_lib.ot_uotdf_set_input(self.h, A.ptr(y), A.ptr(s0)), "ot_uotdf_set_input")

    def step(self, n: int):
        check(_lib.ot_uotdf_step(self.h, int(n)), "ot_uotdf_step")

    def iterate_checked(self, n: int = 1) -> dict:
        r = _abi.ot_uotdf_result()
        check(_lib.ot_uotdf_iterate_checked(self.h, int(n), ctypes.byref(r)), "ot_uotdf_iterate_checked")
        return r.as_dict()

    def solve(self) -> dict:
        r = _abi.ot_uotdf_result()
        check(_lib.ot_uotdf_solve(self.h, ctypes.byref(r)), "ot_uotdf_solve", ok=(OT_OK, OT_ENOTCONV))
        return r.as_dict()

    def reset(self):
        check(_lib.ot_uotdf_reset(self.h), "ot_uotdf_reset")

    def get(self, name: str, device=None):
        import torch
        dev = torch.device("cuda") if device is None else torch.device(device)
        out = torch.empty((self.B, self.H, self.W), dtype=torch.float32, device=dev)
        A = _Arrays(out.numel())
        check(_lib.ot_uotdf_get(self.h, _abi.UOTDF_VARS[name], A.ptr(out, True)), "ot_uotdf_get")
        return out


def unet_layer_specs(base: int = 32) -> list[tuple[str, int, int, int]]:
    """(name, in channels, out channels, kernel size) of the warm-start
    network's convolutions in the library's parameter order."""
    c = base
    return [("enc0a", 2, c, 3), ("enc0b", c, c, 3), ("enc1a", c, 2 * c, 3), ("enc1b", 2 * c, 2 * c, 3),
            ("enc2a", 2 * c, 4 * c, 3), ("enc2b", 4 * c, 4 * c, 3), ("botta", 4 * c, 8 * c, 3),
            ("bottb", 8 * c, 8 * c, 3), ("dec2a", 12 * c, 4 * c, 3), ("dec2b", 4 * c, 4 * c, 3),
            ("dec1a", 6 * c, 2 * c, 3), ("dec1b", 2 * c, 2 * c, 3), ("dec0a", 3 * c, c, 3), ("dec0b", c, c, 3),
            ("head", c, 4, 1)]


class UNet:
    """The learned warm start of Algorithm 1: (p0, p1) [n, 2, H, W] ->
    (Mx, My, r, a) [n, 4, H, W].  Parameters are one flat float32 array in
    the order of :func:`unet_layer_specs` (weights [co, ci, k, k], then
    biases [co], per layer)."""

    def __init__(self, H: int, W: int, max_batch: int, base_channels: int = 32, stream=None,
                 bias_free: bool = False):
        self.H, self.W, self.max_batch, self.base = int(H), int(W), int(max_batch), int(base_channels)
        h = ctypes.c_void_p()
        self._stream = _stream_handle(stream)
        check(_lib.ot_unet_create(self.H, self.W, self.max_batch, self.base, self._stream, ctypes.byref(h)),
              "ot_unet_create")
        self.h = h
        self.n_params = int(_lib.ot_unet_param_count(self.h))
        check(_lib.ot_unet_set_bias_free(self.h, int(bool(bias_free))), "ot_unet_set_bias_free")

    def close(self):
        if getattr(self, "h", None):
            _lib.ot_unet_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, seed: int = 0):
        """He-normal weights, zero biases (numpy generator ``seed``)."""
        rng = np.random.default_rng(seed)
        parts = []
        for _, ci, co, k in unet_layer_specs(self.base):
            parts.append(rng.normal(0.0, np.sqrt(2.0 / (ci * k * k)), co * ci * k * k))
            parts.append(np.zeros(co))
        self.set_params(np.concatenate(parts).astype(np.float32))

    def set_params(self, flat):
        A = _Arrays(self.n_params)
        check(_lib.ot_unet_set_params(self.h, A.ptr(flat)), "ot_unet_set_params")

    def get_params(self) -> np.ndarray:
        out = np.empty(self.n_params, dtype=np.float32)
        check(_lib.ot_unet_get_params(self.h, out.ctypes.data), "ot_unet_get_params")
        return out

    def _n(self, x) -> int:
        n = int(np.prod(x.shape)) // (2 * self.H * self.W)
        if n < 1 or n * 2 * self.H * self.W != int(np.prod(x.shape)):
            raise ValueError("input must hold n x 2 x H x W values")
        return n

    def forward(self, x, out=None):
        """Prediction for x [n, 2, H, W] (host or device); a CUDA tensor."""
        import torch
        n = self._n(x)
        y = torch.empty((n, 4, self.H, self.W), dtype=torch.float32, device="cuda") if out is None else out
        check(_lib.ot_unet_forward(self.h, _Arrays(n * 2 * self.H * self.W).ptr(x),
                                   _Arrays(n * 4 * self.H * self.W).ptr(y, True), n), "ot_unet_forward")
        return y

    def gradients(self, x, target) -> tuple[float, np.ndarray]:
        """(MSE loss, d loss / d params) for one batch; no update."""
        n = self._n(x)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        Ax = _Arrays(n * 2 * self.H * self.W)
        At = _Arrays(n * 4 * self.H * self.W)
        check(_lib.ot_unet_gradients(self.h, Ax.ptr(x), At.ptr(target), n, g.ctypes.data, ctypes.byref(loss)),
              "ot_unet_gradients")
        return loss.value, g

    def train_step(self, x, target, lr: float) -> float:
        """One Adam step on the MSE loss; returns the loss before the step."""
        n = self._n(x)
        loss = ctypes.c_double()
        Ax = _Arrays(n * 2 * self.H * self.W)
        At = _Arrays(n * 4 * self.H * self.W)
        check(_lib.ot_unet_train_step(self.h, Ax.ptr(x), At.ptr(target), n, float(lr), ctypes.byref(loss)),
              "ot_unet_train_step")
        return loss.value


def neumann_solve(X, c: float, precision="fp32", out=None, stream=None):
    """(D D* + c I)^{-1} X for X [B, H, W] float32 CUDA (DCT-II)."""
    import torch
    B, H, W = X.shape
    Y = torch.empty_like(X) if out is None else out
    prec = _abi.PRECISIONS[precision] if isinstance(precision, str) else precision
    check(_lib.ot_neumann_solve(X.data_ptr(), Y.data_ptr(), B, H, W, float(c), prec, _stream_handle(stream)),
          "ot_neumann_solve")
    return Y


def neumann_solve_timed(X, c: float, precision="fp32", n_rep: int = 10, out=None, stream=None) -> float:
    """Device milliseconds of one (D D* + c I)^{-1} X solve, averaged over
    n_rep solves on one set of tables (ot_neumann_solve_timed)."""
    import torch
    B, H, W = X.shape
    Y = torch.empty_like(X) if out is None else out
    prec = _abi.PRECISIONS[precision] if isinstance(precision, str) else precision
    ms = ctypes.c_double()
    check(_lib.ot_neumann_solve_timed(X.data_ptr(), Y.data_ptr(), B, H, W, float(c), prec, int(n_rep),
                                      ctypes.byref(ms), _stream_handle(stream)), "ot_neumann_solve_timed")
    return ms.value


def svt(X, theta: float, stream=None):
    """shrink*_theta of the N x T matrix whose T columns are X[t] (X: [T, ...]
    float32 CUDA tensor).  Returns a tensor of the same shape."""
    import torch
    T = X.shape[0]
    N = X.numel() // T
    Y = torch.empty_like(X)
    check(_lib.ot_svt(X.data_ptr(), Y.data_ptr(), N, T, float(theta), _stream_handle(stream)), "ot_svt")
    return Y


def debug_grid_barrier(ctas: int, preset_count: int = 0) -> tuple[int, int]:
    """Run the fused RPCA pass's grid barrier alone on ``ctas`` cooperative
    CTAs with its arrival count preset; returns (error flag, generation)."""
    err = ctypes.c_int32(0)
    gen = ctypes.c_uint32(0)
    check(_lib.ot_debug_grid_barrier(int(ctas), int(preset_count), ctypes.byref(err), ctypes.byref(gen)),
          "ot_debug_grid_barrier")
    return err.value, gen.value


__all__ = ["debug_grid_barrier", "ProxBatch", "Uotdf", "uotdf_default_params", "Rpca", "svt", "neumann_solve", "rpca_default_params", "OtProx", "OtError", "default_params", "check", "LIB_PATH", "ot_prox_params", "ot_prox_result"]
