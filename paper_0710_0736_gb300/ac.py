"""Thin Python binding of libac (include/ac.h): argument marshalling only.

Every function keeps the C name and forwards to the library; all arithmetic
runs in the library's CUDA kernels.  Buffers may be numpy arrays (host memory,
is_device = 0) or torch CUDA tensors (device memory, is_device = 1).  Importing
this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libac.so")

AC_OK, AC_ERR_ARG, AC_ERR_CUDA, AC_ERR_NOT_CONVERGED, AC_ERR_NUMERIC, AC_ERR_STATE, AC_ERR_NOMEM = 0, -1, -2, -3, -4, -5, -6
AC_FP64, AC_MIXED = 0, 1
AC_PROJ_SIMPLEX, AC_PROJ_NODE = 0, 1
AC_TILES_AUTO, AC_TILES_NEVER, AC_TILES_ALWAYS = 0, 1, 2
AC_LOOP_AUTO, AC_LOOP_HOST = 0, 1
AC_SMOOTH_GS3, AC_SMOOTH_JACOBI = 0, 1
AC_ADJ_PRECOND_F32, AC_ADJ_PRECOND_F64 = 0, 1
AC_BATCH_STREAMS, AC_BATCH_ONE_GRAPH = 0, 1
AC_MAX_PHASES = 8

EXPORTS = [
    "ac_default_params", "ac_create", "ac_set_image", "ac_set_image_f64", "ac_step", "ac_segment", "ac_destroy",
    "ac_set_phase", "ac_get_phase", "ac_get_means", "ac_get_moments", "ac_get_rhs", "ac_get_node_labels",
    "ac_get_composite", "ac_energy", "ac_residual", "ac_project_simplex", "ac_set_profiling", "ac_set_profiling_mask", "ac_get_profile", "ac_colour_means_static",
    "ac_batch_create", "ac_batch_set_image", "ac_batch_set_phase", "ac_batch_get_phase", "ac_batch_segment",
    "ac_batch_step", "ac_batch_tune", "ac_batch_destroy", "ac_adjoint_forward", "ac_adjoint_backward",
    "ac_adjoint_recompute_diff", "ac_set_coarse_tiling", "ac_set_cycle_loop", "ac_get_cycle_loop", "ac_set_coarse_smoother", "ac_set_adjoint_preconditioner",
    "ac_batch_set_launch", "ac_batch_set_cycle_loop", "ac_last_error",
]
PROF_CLASSES = ["smooth", "resid", "coarse", "transfer", "linesearch", "setup", "outer"]


class ac_params(C.Structure):
    _fields_ = [("width", C.c_int), ("height", C.c_int), ("n_phases", C.c_int),
                ("eps", C.c_double), ("lambda_", C.c_double), ("tau", C.c_double), ("tol", C.c_double),
                ("nu1", C.c_int), ("nu2", C.c_int), ("max_cycles", C.c_int), ("coarse_min", C.c_int),
                ("precision", C.c_int), ("seed", C.c_uint64), ("refine", C.c_int), ("projection", C.c_int),
                ("stream", C.c_void_p)]


class ac_stats(C.Structure):
    _fields_ = [("energy", C.c_double), ("residual", C.c_double), ("cycles", C.c_int),
                ("total_cycles", C.c_int), ("steps", C.c_int), ("converged", C.c_int),
                ("fine_sweeps", C.c_int64), ("outer", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ac_profile(C.Structure):
    _fields_ = [("ms", C.c_double * 7), ("launches", C.c_int64 * 7), ("smooth_bytes_per_launch", C.c_double),
                ("total_launches", C.c_int64), ("smooth_corr_launches", C.c_int64),
                ("smooth_corr_extra_bytes", C.c_double), ("bytes", C.c_double * 7)]

    def as_dict(self):
        return {"ms": dict(zip(PROF_CLASSES, list(self.ms))),
                "launches": dict(zip(PROF_CLASSES, list(self.launches))),
                "smooth_bytes_per_launch": self.smooth_bytes_per_launch,
                "total_launches": self.total_launches,
                "smooth_corr_launches": self.smooth_corr_launches,
                "smooth_corr_extra_bytes": self.smooth_corr_extra_bytes,
                "bytes": dict(zip(PROF_CLASSES, list(self.bytes)))}


class ac_batch_stats(C.Structure):
    _fields_ = [("images", C.c_int), ("steps", C.c_int), ("converged_images", C.c_int),
                ("total_cycles", C.c_int64), ("fine_sweeps", C.c_int64), ("nodes", C.c_int64), ("dof", C.c_int64),
                ("dof_sweeps", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libac error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"libac is not built ({_LIB_PATH} missing): run __graft_entry__.build()")
    L = C.CDLL(_LIB_PATH)
    vp, i, i64, d = C.c_void_p, C.c_int, C.c_int64, C.c_double
    P = C.POINTER
    sig = {
        "ac_default_params": ([P(ac_params)], i),
        "ac_create": ([P(vp), P(ac_params)], i),
        "ac_set_image": ([vp, vp, i], i),
        "ac_set_image_f64": ([vp, vp, i], i),
        "ac_step": ([vp, i, P(ac_stats)], i),
        "ac_segment": ([vp, i, vp, i, P(ac_stats)], i),
        "ac_destroy": ([vp], None),
        "ac_set_phase": ([vp, vp, i], i),
        "ac_get_phase": ([vp, vp, i], i),
        "ac_get_means": ([vp, vp], i),
        "ac_get_moments": ([vp, vp], i),
        "ac_get_rhs": ([vp, vp], i),
        "ac_get_node_labels": ([vp, vp, i], i),
        "ac_get_composite": ([vp, vp, i, i], i),
        "ac_energy": ([vp, P(d)], i),
        "ac_residual": ([vp, P(d)], i),
        "ac_project_simplex": ([vp, vp, i64, i, vp], i),
        "ac_set_profiling": ([vp, i], i),
        "ac_set_profiling_mask": ([vp, C.c_uint], i),
        "ac_get_profile": ([vp, P(ac_profile)], i),
        "ac_colour_means_static": ([vp, vp, i, i, i, vp, vp], i),
        "ac_batch_create": ([P(vp), P(ac_params), i, i], i),
        "ac_batch_set_image": ([vp, i, vp, i], i),
        "ac_batch_set_phase": ([vp, i, vp, i], i),
        "ac_batch_get_phase": ([vp, i, vp, i], i),
        "ac_batch_segment": ([vp, i, vp, i], i),
        "ac_batch_step": ([vp, i, P(ac_batch_stats)], i),
        "ac_batch_tune": ([vp, i, vp], i),
        "ac_batch_destroy": ([vp], None),
        "ac_adjoint_forward": ([vp, i, i], i),
        "ac_adjoint_backward": ([vp, vp, P(d), P(d), vp, vp], i),
        "ac_adjoint_recompute_diff": ([vp, P(i64)], i),
        "ac_set_coarse_tiling": ([vp, i], i),
        "ac_set_cycle_loop": ([vp, i], i),
        "ac_set_coarse_smoother": ([vp, i], i),
        "ac_set_adjoint_preconditioner": ([vp, i], i),
        "ac_get_cycle_loop": ([vp, P(i)], i),
        "ac_batch_set_launch": ([vp, i], i),
        "ac_batch_set_cycle_loop": ([vp, i], i),
        "ac_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    return L


lib = _load()


def _check(rc, ok=(AC_OK,)):
    if rc not in ok:
        raise AcError(rc, lib.ac_last_error().decode())
    return rc


def _buf(x, dtype, count, writable=False):
    """(pointer, is_device) of a numpy array or torch tensor of `count` elements."""
    if hasattr(x, "data_ptr"):  # torch tensor
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64, np.int8: torch.int8}[dtype]
        if x.dtype != want or not x.is_contiguous() or x.numel() != count:
            raise ValueError(f"expected a contiguous {want} tensor of {count} elements")
        return x.data_ptr(), int(x.is_cuda)
    if not isinstance(x, np.ndarray) or x.dtype != dtype or not x.flags.c_contiguous or x.size != count:
        raise ValueError(f"expected a C-contiguous {np.dtype(dtype)} array of {count} elements")
    if writable and not x.flags.writeable:
        raise ValueError("output array is read-only")
    return x.ctypes.data, 0


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def ac_default_params(**kw) -> ac_params:
    p = ac_params()
    _check(lib.ac_default_params(C.byref(p)))
    if "lambda" in kw:
        kw["lambda_"] = kw.pop("lambda")
    if "stream" not in kw:
        kw["stream"] = _current_stream()
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def ac_create(params: ac_params):
    ctx = C.c_void_p()
    _check(lib.ac_create(C.byref(ctx), C.byref(params)))
    return ctx


def ac_destroy(ctx):
    lib.ac_destroy(ctx)


def ac_set_image(ctx, rgb, W, H):
    """rgb: H x W x 3 float32 (numpy host array or torch CUDA tensor)."""
    ptr, dev = _buf(rgb, np.float32, W * H * 3)
    return _check(lib.ac_set_image(ctx, ptr, dev))


def ac_set_image_f64(ctx, rgb, W, H):
    ptr, dev = _buf(rgb, np.float64, W * H * 3)
    return _check(lib.ac_set_image_f64(ctx, ptr, dev))


def ac_step(ctx, n_steps, allow_not_converged=False):
    st = ac_stats()
    ok = (AC_OK, AC_ERR_NOT_CONVERGED) if allow_not_converged else (AC_OK,)
    rc = _check(lib.ac_step(ctx, n_steps, C.byref(st)), ok)
    return rc, st


def ac_segment(ctx, n_steps, labels, W, H, allow_not_converged=False, stats=True):
    """stats=False passes no statistics struct: the library then skips the
    energy evaluation of the last step (st is returned as None)."""
    ptr, dev = _buf(labels, np.int8, W * H, writable=True)
    st = ac_stats() if stats else None
    ok = (AC_OK, AC_ERR_NOT_CONVERGED) if allow_not_converged else (AC_OK,)
    rc = _check(lib.ac_segment(ctx, n_steps, ptr, dev, C.byref(st) if stats else None), ok)
    return rc, st


def ac_set_phase(ctx, u, n_nodes, N):
    ptr, dev = _buf(u, np.float64, n_nodes * N)
    return _check(lib.ac_set_phase(ctx, ptr, dev))


def ac_get_phase(ctx, u, n_nodes, N):
    ptr, dev = _buf(u, np.float64, n_nodes * N, writable=True)
    return _check(lib.ac_get_phase(ctx, ptr, dev))


def ac_get_means(ctx, N):
    c = np.zeros((N, 3))
    _check(lib.ac_get_means(ctx, c.ctypes.data))
    return c


def ac_get_moments(ctx, n_nodes):
    m = np.zeros((n_nodes, 5))
    _check(lib.ac_get_moments(ctx, m.ctypes.data))
    return m


def ac_get_rhs(ctx, n_nodes, N):
    b = np.zeros((n_nodes, N))
    _check(lib.ac_get_rhs(ctx, b.ctypes.data))
    return b


def ac_get_node_labels(ctx, labels, n_nodes):
    ptr, dev = _buf(labels, np.int8, n_nodes, writable=True)
    return _check(lib.ac_get_node_labels(ctx, ptr, dev))


def ac_get_composite(ctx, rgb, W, H, rounded=False):
    """Composite (rounded: rounded composite) into rgb, H x W x 3 float32 (numpy or CUDA tensor)."""
    ptr, dev = _buf(rgb, np.float32, W * H * 3, writable=True)
    return _check(lib.ac_get_composite(ctx, ptr, 1 if rounded else 0, dev))


def ac_energy(ctx) -> float:
    e = C.c_double()
    _check(lib.ac_energy(ctx, C.byref(e)))
    return e.value


def ac_residual(ctx) -> float:
    r = C.c_double()
    _check(lib.ac_residual(ctx, C.byref(r)))
    return r.value


def ac_project_simplex(y, x, count, N, stream=None):
    """y, x: torch CUDA float64 tensors of count*N elements."""
    py, dy = _buf(y, np.float64, count * N)
    px, dx = _buf(x, np.float64, count * N, writable=True)
    if not (dy and dx):
        raise ValueError("ac_project_simplex takes device tensors")
    return _check(lib.ac_project_simplex(py, px, count, N, stream if stream is not None else _current_stream()))


def ac_set_profiling(ctx, enable=True):
    return _check(lib.ac_set_profiling(ctx, int(bool(enable))))


def ac_set_profiling_mask(ctx, classes):
    """Profile only the named classes (see PROF_CLASSES); an empty list turns profiling off."""
    mask = 0
    for c in classes:
        mask |= 1 << PROF_CLASSES.index(c)
    return _check(lib.ac_set_profiling_mask(ctx, mask))


def ac_get_profile(ctx) -> ac_profile:
    p = ac_profile()
    _check(lib.ac_get_profile(ctx, C.byref(p)))
    return p


def ac_colour_means_static(u, rgb, W, H, N, c, stream=None):
    """Colour means without device allocation; u, rgb, c: torch CUDA tensors
    (float64 (H+1)(W+1) x N, float32 H x W x 3, float64 N x 3)."""
    pu, du = _buf(u, np.float64, (W + 1) * (H + 1) * N)
    pr, dr = _buf(rgb, np.float32, W * H * 3)
    pc, dc = _buf(c, np.float64, N * 3, writable=True)
    if not (du and dr and dc):
        raise ValueError("ac_colour_means_static takes device tensors")
    return _check(lib.ac_colour_means_static(pu, pr, W, H, N, pc, stream if stream is not None else _current_stream()))


def ac_batch_create(params_list, n_streams):
    arr = (ac_params * len(params_list))(*params_list)
    b = C.c_void_p()
    _check(lib.ac_batch_create(C.byref(b), arr, len(params_list), n_streams))
    return b


def ac_batch_step(b, n_steps, allow_not_converged=False):
    st = ac_batch_stats()
    ok = (AC_OK, AC_ERR_NOT_CONVERGED) if allow_not_converged else (AC_OK,)
    rc = _check(lib.ac_batch_step(b, n_steps, C.byref(st)), ok)
    return rc, st


def ac_batch_tune(b, count, trial_steps=2):
    """Per image: nu1, nu2, depth and the coarse smoother the tuner chose."""
    chosen = np.zeros((count, 4), np.int32)
    _check(lib.ac_batch_tune(b, trial_steps, chosen.ctypes.data))
    return chosen


def ac_adjoint_forward(ctx, n_steps, checkpoint_every, allow_not_converged=False):
    ok = (AC_OK, AC_ERR_NOT_CONVERGED) if allow_not_converged else (AC_OK,)
    return _check(lib.ac_adjoint_forward(ctx, n_steps, checkpoint_every), ok)


def ac_adjoint_backward(ctx, grad_u, grad_image, grad_u0=None, allow_not_converged=False):
    """grad_u, grad_image, grad_u0: torch CUDA float64 tensors.  Returns
    (dL/dlambda, dL/deps)."""
    gl, ge = C.c_double(), C.c_double()
    ok = (AC_OK, AC_ERR_NOT_CONVERGED) if allow_not_converged else (AC_OK,)
    for t in (grad_u, grad_image) + ((grad_u0,) if grad_u0 is not None else ()):
        if not (hasattr(t, "is_cuda") and t.is_cuda and t.is_contiguous() and str(t.dtype) == "torch.float64"):
            raise ValueError("ac_adjoint_backward takes contiguous float64 CUDA tensors")
    _check(lib.ac_adjoint_backward(ctx, grad_u.data_ptr(), C.byref(gl), C.byref(ge), grad_image.data_ptr(),
                                   None if grad_u0 is None else grad_u0.data_ptr()), ok)
    return gl.value, ge.value


def ac_adjoint_recompute_diff(ctx) -> int:
    """Components at which the last backward pass's recomputed segment ends
    differed from the forward's states (0 when the recomputation repeated the
    forward exactly)."""
    k = C.c_int64()
    _check(lib.ac_adjoint_recompute_diff(ctx, C.byref(k)))
    return k.value


def ac_set_coarse_tiling(ctx, mode):
    """AC_TILES_AUTO, AC_TILES_NEVER or AC_TILES_ALWAYS (see include/ac.h)."""
    return _check(lib.ac_set_coarse_tiling(ctx, mode))


def ac_set_cycle_loop(ctx, mode):
    """AC_LOOP_AUTO (the V-cycle loop on the device where the context allows)
    or AC_LOOP_HOST (see include/ac.h)."""
    return _check(lib.ac_set_cycle_loop(ctx, mode))


def ac_set_coarse_smoother(ctx, mode):
    """AC_SMOOTH_GS3 (default) or AC_SMOOTH_JACOBI (see include/ac.h)."""
    return _check(lib.ac_set_coarse_smoother(ctx, mode))


def ac_set_adjoint_preconditioner(ctx, precision):
    """AC_ADJ_PRECOND_F32 (default) or AC_ADJ_PRECOND_F64 (see include/ac.h)."""
    return _check(lib.ac_set_adjoint_preconditioner(ctx, precision))


def ac_get_cycle_loop(ctx) -> bool:
    """True if the next ac_step runs its cycle loop on the device."""
    k = C.c_int()
    _check(lib.ac_get_cycle_loop(ctx, C.byref(k)))
    return bool(k.value)


def ac_last_error() -> str:
    return lib.ac_last_error().decode()


class Segmenter:
    """Owns one context: image W x H, N phases.  Convenience over the C calls.
    With refine = r the phase field, node labels and moments live on the grid
    refined r times (Wr x Hr cells); images, pixel labels and composites stay
    W x H."""

    def __init__(self, W, H, N, eps, lam, tau, **kw):
        self.W, self.H, self.N = W, H, N
        r = kw.get("refine", 0)
        self.Wr, self.Hr = W << r, H << r
        self.n_nodes = (self.Wr + 1) * (self.Hr + 1)
        self.params = ac_default_params(width=W, height=H, n_phases=N, eps=eps, tau=tau, **{"lambda": lam}, **kw)
        self.ctx = ac_create(self.params)

    def close(self):
        if self.ctx is not None:
            ac_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_image(self, rgb):
        dt = getattr(rgb, "dtype", None)
        if dt == np.float64 or str(dt) == "torch.float64":
            return ac_set_image_f64(self.ctx, rgb, self.W, self.H)
        return ac_set_image(self.ctx, rgb, self.W, self.H)

    def set_phase(self, u):
        return ac_set_phase(self.ctx, u, self.n_nodes, self.N)

    def phase(self):
        u = np.zeros((self.n_nodes, self.N))
        ac_get_phase(self.ctx, u, self.n_nodes, self.N)
        return u

    def step(self, n=1, allow_not_converged=False):
        return ac_step(self.ctx, n, allow_not_converged)[1]

    def segment(self, n=0, allow_not_converged=False):
        lab = np.zeros((self.H, self.W), np.int8)
        ac_segment(self.ctx, n, lab, self.W, self.H, allow_not_converged)
        return lab

    def node_labels(self):
        lab = np.zeros((self.Hr + 1, self.Wr + 1), np.int8)
        ac_get_node_labels(self.ctx, lab, self.n_nodes)
        return lab

    def means(self):
        return ac_get_means(self.ctx, self.N)

    def moments(self):
        return ac_get_moments(self.ctx, self.n_nodes)

    def rhs(self):
        return ac_get_rhs(self.ctx, self.n_nodes, self.N)

    def composite(self, rounded=False):
        out = np.zeros((self.H, self.W, 3), np.float32)
        ac_get_composite(self.ctx, out, self.W, self.H, rounded)
        return out

    def set_cycle_loop(self, mode):
        return ac_set_cycle_loop(self.ctx, mode)

    def loop_on_device(self):
        return ac_get_cycle_loop(self.ctx)

    def energy(self):
        return ac_energy(self.ctx)

    def residual(self):
        return ac_residual(self.ctx)


class Batch:
    """Many independent images (uneven sizes and phase counts) advanced together.

    specs: list of dicts with W, H, N and optionally eps, lam, tau, tol,
    precision, seed, nu1, nu2, coarse_min, max_cycles."""

    def __init__(self, specs, n_streams=8):
        self.specs = [dict(s) for s in specs]
        plist = []
        for sp in self.specs:
            kw = {k: sp[k] for k in ("tol", "precision", "seed", "nu1", "nu2", "coarse_min", "max_cycles", "projection")
                  if k in sp}
            plist.append(ac_default_params(width=sp["W"], height=sp["H"], n_phases=sp["N"], eps=sp.get("eps", 2.0),
                                           tau=sp.get("tau", 4.0), stream=None, **{"lambda": sp.get("lam", 1.0)},
                                           **kw))
        self.b = ac_batch_create(plist, n_streams)

    def close(self):
        if self.b is not None:
            lib.ac_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_image(self, k, rgb):
        sp = self.specs[k]
        ptr, dev = _buf(rgb, np.float32, sp["W"] * sp["H"] * 3)
        return _check(lib.ac_batch_set_image(self.b, k, ptr, dev))

    def set_phase(self, k, u):
        sp = self.specs[k]
        ptr, dev = _buf(u, np.float64, (sp["W"] + 1) * (sp["H"] + 1) * sp["N"])
        return _check(lib.ac_batch_set_phase(self.b, k, ptr, dev))

    def phase(self, k):
        sp = self.specs[k]
        u = np.zeros(((sp["W"] + 1) * (sp["H"] + 1), sp["N"]))
        _check(lib.ac_batch_get_phase(self.b, k, u.ctypes.data, 0))
        return u

    def labels(self, k):
        sp = self.specs[k]
        lab = np.zeros((sp["H"], sp["W"]), np.int8)
        _check(lib.ac_batch_segment(self.b, k, lab.ctypes.data, 0))
        return lab

    def step(self, n=1, allow_not_converged=False):
        return ac_batch_step(self.b, n, allow_not_converged)[1]

    def tune(self, trial_steps=2):
        return ac_batch_tune(self.b, len(self.specs), trial_steps)

    def set_launch(self, mode):
        """AC_BATCH_STREAMS or AC_BATCH_ONE_GRAPH (see include/ac.h)."""
        return _check(lib.ac_batch_set_launch(self.b, mode))

    def set_cycle_loop(self, mode):
        return _check(lib.ac_batch_set_cycle_loop(self.b, mode))
