"""GB300-native Landau gauge fixing (steepest descent with Fourier
acceleration) for SU(3) lattice gauge fields.

The work runs in ``liblgf.so`` (hand-written sm_103a CUDA kernels behind the C
ABI of ``include/lgf.h``).  This package is its thin Python face:
``GaugeFixer`` wraps one library handle; the raw entry points are in
``paper_1208_1186_gb300._lib`` under their C names.

Host link arrays are complex128 of shape (Lt, Lz, Ly, Lx, 4, 3, 3) (x fastest,
mu = x, y, z, t), the layout ``lgf_load_links`` takes.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import LgfError

__all__ = ["GaugeFixer", "GaugeBatch", "WarmStartNet", "LgfError", "fix_stream"]

def _as_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class GaugeFixer:
    """One liblgf handle for an (Lx, Ly, Lz, Lt) lattice.

    dtype: 'f64' (FP64, 18 reals), 'f64_r12', 'f32' (FP32 bulk with FP64 F/theta
    sums and an FP64 tail in ``fix``), 'f32_r12' (the same with 12-real links).
    """

    def __init__(self, dims, dtype: str = "f64", stream=None, torch_allocator: bool = True,
                 alpha: float = 0.08):
        self.lib = _lib.load()
        if torch_allocator:
            _lib.use_torch_allocator()
        self.dims = tuple(int(v) for v in dims)
        self.shape = (self.dims[3], self.dims[2], self.dims[1], self.dims[0])
        self.V = int(np.prod(self.dims))
        self.dtype = dtype
        h = ctypes.c_void_p()
        _lib.check(self.lib.lgf_create(*self.dims, _lib.DTYPES[dtype], ctypes.byref(h)), "lgf_create")
        self.h = h
        if stream is not None:
            self.set_stream(stream)
        self.set_param(_lib.LGF_ALPHA, alpha)

    # -- lifetime ---------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            self.lib.lgf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration ----------------------------------------------------
    def set_stream(self, stream):
        ptr = stream if isinstance(stream, int) else stream.cuda_stream
        _lib.check(self.lib.lgf_set_stream(self.h, ctypes.c_void_p(ptr)), "lgf_set_stream", self.h)

    def set_param(self, key: int, value: float):
        _lib.check(self.lib.lgf_set_param(self.h, key, float(value)), "lgf_set_param", self.h)

    # -- links --------------------------------------------------------------
    def load_links(self, U):
        """Host complex128 array (numpy) or a CUDA complex128/float64 torch tensor."""
        if isinstance(U, np.ndarray):
            a = np.ascontiguousarray(U, dtype=np.complex128)
            if a.size != self.V * 36:
                raise ValueError(f"expected {self.V * 36} complex entries, got {a.size}")
            _lib.check(self.lib.lgf_load_links(self.h, _as_ptr(a)), "lgf_load_links", self.h)
        else:  # torch tensor on the device
            if not U.is_cuda or not U.is_contiguous() or U.numel() * U.element_size() != self.V * 576:
                raise ValueError("expected a contiguous CUDA tensor of V*4*3*3 complex128")
            _lib.check(self.lib.lgf_load_links_device(self.h, ctypes.c_void_p(U.data_ptr())),
                       "lgf_load_links_device", self.h)

    def store_links(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.shape + (4, 3, 3), dtype=np.complex128)
        _lib.check(self.lib.lgf_store_links(self.h, _as_ptr(out)), "lgf_store_links", self.h)
        return out

    def store_gauge(self, out: np.ndarray | None = None) -> np.ndarray:
        """The gauge transformation G applied since the last load, complex128
        (Lt, Lz, Ly, Lx, 3, 3): links = G(x) U_loaded G(x+mu)^dagger
        (``lgf_store_gauge``; FP64 handles need LGF_TRACK_G before the load)."""
        if out is None:
            out = np.empty(self.shape + (3, 3), dtype=np.complex128)
        _lib.check(self.lib.lgf_store_gauge(self.h, _as_ptr(out)), "lgf_store_gauge", self.h)
        return out

    # -- the method -----------------------------------------------------------
    def iterate(self, n: int):
        _lib.check(self.lib.lgf_iterate(self.h, int(n)), "lgf_iterate", self.h)

    def fix(self, theta_tol: float, max_iter: int, raise_on_fail: bool = False):
        """Returns (iterations, converged)."""
        it = ctypes.c_int(0)
        st = self.lib.lgf_fix(self.h, float(theta_tol), int(max_iter), ctypes.byref(it))
        if st == _lib.LGF_ERR_NOT_CONVERGED and not raise_on_fail:
            return it.value, False
        _lib.check(st, "lgf_fix", self.h)
        return it.value, True

    def functional(self):
        F, th = ctypes.c_double(), ctypes.c_double()
        _lib.check(self.lib.lgf_functional(self.h, ctypes.byref(F), ctypes.byref(th)), "lgf_functional", self.h)
        return F.value, th.value

    def probe(self):
        """Gradient, accelerated gradient (both packed, (.., 4) complex) and g
        of the current links; the links are not changed."""
        d = np.empty(self.shape + (4,), dtype=np.complex128)
        dt = np.empty(self.shape + (4,), dtype=np.complex128)
        g = np.empty(self.shape + (3, 3), dtype=np.complex128)
        _lib.check(self.lib.lgf_probe(self.h, _as_ptr(d), _as_ptr(dt), _as_ptr(g)), "lgf_probe", self.h)
        return {"delta": d, "delta_tilde": dt, "g": g}

    def fix_split(self):
        """(FP32 updates, FP64 updates) of the last fix."""
        a, b = ctypes.c_int(0), ctypes.c_int(0)
        _lib.check(self.lib.lgf_fix_split(self.h, ctypes.byref(a), ctypes.byref(b)), "lgf_fix_split", self.h)
        return a.value, b.value

    def history(self, cap: int = 1 << 16) -> np.ndarray:
        buf = np.empty(cap, dtype=np.float64)
        n = ctypes.c_int(0)
        _lib.check(self.lib.lgf_history(self.h, _as_ptr(buf), cap, ctypes.byref(n)), "lgf_history", self.h)
        return buf[: n.value].copy()

    def launch_count(self) -> int:
        return int(self.lib.lgf_launch_count(self.h))

    def profile(self, enable: bool):
        _lib.check(self.lib.lgf_profile(self.h, int(bool(enable))), "lgf_profile", self.h)

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since profile(True)."""
        n = _lib.LGF_NUM_KERNELS
        ms = np.zeros(n, dtype=np.float64)
        cnt = np.zeros(n, dtype=np.int64)
        _lib.check(self.lib.lgf_profile_read(self.h, _as_ptr(ms), _as_ptr(cnt), n), "lgf_profile_read", self.h)
        return {self.lib.lgf_kernel_name(k).decode(): (float(ms[k]), int(cnt[k])) for k in range(n)}

    def autotune(self, reps: int = 10) -> int:
        """Time the FFT schedules that apply to this lattice (pipelines, z-t
        tile widths, radix orders) and use the fastest; returns the pipeline
        (1 Stockham planes, 2 axis passes, 3 register planes)."""
        ch = ctypes.c_int(0)
        _lib.check(self.lib.lgf_autotune(self.h, int(reps), ctypes.byref(ch)), "lgf_autotune", self.h)
        return ch.value

    def schedule(self, engine: int | None = None):
        """(pipeline, z-t tile width, radix order) of an engine (0 FP64, 1 the
        FP32 engine of a mixed handle; default: the one that iterates first)."""
        if engine is None:
            engine = 1 if self.dtype.startswith("f32") else 0
        p, b, r = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _lib.check(self.lib.lgf_tune_schedule(self.h, int(engine), ctypes.byref(p), ctypes.byref(b), ctypes.byref(r)),
                   "lgf_tune_schedule", self.h)
        return p.value, b.value, r.value

    def set_schedule(self, pipeline: int, zt_bx: int = 0, zt_ro: int = 0, engine: int | None = None):
        if engine is None:
            engine = 1 if self.dtype.startswith("f32") else 0
        _lib.check(self.lib.lgf_set_schedule(self.h, int(engine), int(pipeline), int(zt_bx), int(zt_ro)),
                   "lgf_set_schedule", self.h)


def fix_stream(fixers, inputs, outputs, theta_tol: float, max_iter: int):
    """Fix configurations inputs[k] into outputs[k] through two GaugeFixer
    handles of one lattice and dtype (``lgf_fix_stream``): while one handle
    fixes a configuration, the next is copied in and the previous copied out.
    inputs/outputs: complex128 host arrays of the link layout, ideally in
    pinned memory (e.g. views of ``torch.empty(..., pin_memory=True)``).
    Returns (per-configuration update counts, all converged)."""
    f0, f1 = fixers
    n = len(inputs)
    if len(outputs) != n:
        raise ValueError("inputs and outputs differ in length")
    for a in list(inputs) + list(outputs):
        if not isinstance(a, np.ndarray) or a.dtype != np.complex128 or not a.flags.c_contiguous \
                or a.size != f0.V * 36:
            raise ValueError(f"expected C-contiguous complex128 arrays of {f0.V * 36} entries")
    ins = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in inputs])
    outs = (ctypes.c_void_p * max(n, 1))(*[a.ctypes.data for a in outputs])
    its = (ctypes.c_int * max(n, 1))()
    st = f0.lib.lgf_fix_stream(f0.h, f1.h, n, ins, outs, float(theta_tol), int(max_iter), its)
    if st == _lib.LGF_ERR_NOT_CONVERGED:
        return list(its)[:n], False
    _lib.check(st, "lgf_fix_stream", f0.h)
    return list(its)[:n], True


class GaugeBatch:
    """Several GaugeFixer handles (any sizes) iterated together from CUDA
    graphs with one branch per lattice.  The fixers must outlive the batch."""

    def __init__(self, fixers):
        self.lib = _lib.load()
        self.fixers = list(fixers)
        arr = (ctypes.c_void_p * len(self.fixers))(*[f.h.value for f in self.fixers])
        b = ctypes.c_void_p()
        _lib.check(self.lib.lgf_batch_create(arr, len(self.fixers), ctypes.byref(b)), "lgf_batch_create")
        self.b = b

    def _check(self, st, where):
        if st != _lib.LGF_OK:
            raise LgfError(st, where, self.lib.lgf_batch_last_error(self.b).decode())

    def set_lanes(self, lanes: int):
        """Parallel graph branches: 0 one per member, n > 0 n lanes."""
        self._check(self.lib.lgf_batch_set_lanes(self.b, int(lanes)), "lgf_batch_set_lanes")

    def autotune(self, reps: int = 4) -> int:
        """Time the lane counts on reps iterations (applied to the links) and
        keep the fastest; returns it (0: one lane per member)."""
        out = ctypes.c_int(0)
        self._check(self.lib.lgf_batch_autotune(self.b, int(reps), ctypes.byref(out)), "lgf_batch_autotune")
        return out.value

    def iterate(self, n: int):
        self._check(self.lib.lgf_batch_iterate(self.b, int(n)), "lgf_batch_iterate")

    def fix(self, theta_tol: float, max_iter: int):
        """Returns (iterations per member, converged per member)."""
        n = len(self.fixers)
        it = np.zeros(n, dtype=np.int32)
        cv = np.zeros(n, dtype=np.int32)
        st = self.lib.lgf_batch_fix(self.b, float(theta_tol), int(max_iter), _as_ptr(it), _as_ptr(cv))
        if st not in (_lib.LGF_OK, _lib.LGF_ERR_NOT_CONVERGED):
            self._check(st, "lgf_batch_fix")
        return it.tolist(), [bool(c) for c in cv]

    def close(self):
        if getattr(self, "b", None):
            self.lib.lgf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class WarmStartNet:
    """The learned warm start (lgf_net_*): a small 4D convolutional network
    that predicts the initial gauge transformation of an FP32 handle."""

    def __init__(self, seed: int = 0, torch_allocator: bool = True):
        self.lib = _lib.load()
        if torch_allocator:
            _lib.use_torch_allocator()
        n = ctypes.c_void_p()
        st = self.lib.lgf_net_create(ctypes.c_ulonglong(seed), ctypes.byref(n))
        if st != _lib.LGF_OK:
            raise LgfError(st, "lgf_net_create", self.lib.lgf_net_last_error(None).decode())
        self.n = n
        self.nparams = int(self.lib.lgf_net_param_count())

    def _check(self, st, where):
        if st != _lib.LGF_OK:
            raise LgfError(st, where, self.lib.lgf_net_last_error(self.n).decode())

    def get_params(self) -> np.ndarray:
        p = np.empty(self.nparams, dtype=np.float32)
        self._check(self.lib.lgf_net_get_params(self.n, _as_ptr(p)), "lgf_net_get_params")
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        self._check(self.lib.lgf_net_set_params(self.n, _as_ptr(p)), "lgf_net_set_params")

    def forward(self, gf: "GaugeFixer") -> np.ndarray:
        c = np.empty(gf.shape + (8,), dtype=np.float32)
        self._check(self.lib.lgf_net_forward(self.n, gf.h, _as_ptr(c)), "lgf_net_forward")
        return c

    def train_step(self, gf: "GaugeFixer", lr: float, want_grad: bool = False):
        """Returns (F(U^{g0}) before the step, parameter gradient of -F or None)."""
        F = ctypes.c_double()
        g = np.empty(self.nparams, dtype=np.float32) if want_grad else None
        self._check(self.lib.lgf_net_train_step(self.n, gf.h, float(lr), ctypes.byref(F),
                                                _as_ptr(g) if want_grad else None), "lgf_net_train_step")
        return F.value, g

    def conv(self, layer: int, backward: bool, x, dims, mask=None, out_f32=None):
        """One layer on device bf16 activations (torch tensors [V][channels]);
        returns the bf16 output tensor (see lgf_net_conv)."""
        import torch
        V = int(np.prod(dims))
        nout = 32 if (backward or layer < 3) else 16
        out = torch.empty((V, nout), dtype=torch.bfloat16, device=x.device)
        st = torch.cuda.current_stream().cuda_stream
        self._check(self.lib.lgf_net_conv(self.n, int(layer), int(bool(backward)), ctypes.c_void_p(x.data_ptr()),
                                          ctypes.c_void_p(mask.data_ptr()) if mask is not None else None,
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(out_f32.data_ptr()) if out_f32 is not None else None,
                                          *[int(d) for d in dims], ctypes.c_void_p(st)), "lgf_net_conv")
        return out

    def set_wait_budget(self, polls: int):
        """Poll budget of the convolutions' stage waits (lgf_net_set_wait_budget;
        negative: the default)."""
        self._check(self.lib.lgf_net_set_wait_budget(self.n, ctypes.c_longlong(int(polls))),
                    "lgf_net_set_wait_budget")

    def warm_start(self, gf: "GaugeFixer"):
        self._check(self.lib.lgf_net_warm_start(self.n, gf.h), "lgf_net_warm_start")

    def close(self):
        if getattr(self, "n", None):
            self.lib.lgf_net_destroy(self.n)
            self.n = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
