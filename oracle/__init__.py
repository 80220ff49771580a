"""CPU oracle for the vector-valued Allen-Cahn segmentation step.

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by
the benchmark's CPU-baseline leg, never by the product path. The arithmetic
lives in ``ac_oracle.c`` (plain sequential FP64 C); this module compiles it
with gcc and marshals numpy arrays through ctypes.

Every function follows a passage of Kay & Tomasi: the P1 matrices (Sec. 3.1),
projection by simplex and by node (Sec. 4.2), colour means and fitting terms (Eq.
VV_fidelity, Sec. 4.4), the step problem (Sec. 3.2, Eq. alpha), the Gibbs
clamp-and-redistribute loop (Sec. 3.3), SSC over all levels (Sec. 3.2) and the
rounded composite (Sec. 4.3).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ac_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "libac_oracle.so")
ROW = 7

_dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_bp = np.ctypeslib.ndpointer(np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle library in-tree (gcc -O2, portable flags only)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        i, i64, d = C.c_int, C.c_int64, C.c_double
        L.or_assemble.argtypes = [i, i, _dp, _ip, _dp, _ip]
        L.or_moments.argtypes = [i, i, _dp, _dp]
        L.or_moments_node.argtypes = [i, i, _dp, _dp]
        L.or_means.argtypes = [i, i, i, _dp, _dp, C.c_void_p, _dp, C.c_void_p]
        L.or_rhs.argtypes = [i, i, i, _dp, _dp, _dp, d, d, d, _dp]
        L.or_energy.argtypes = [i, i, i, _dp, _dp, d, d]
        L.or_energy.restype = d
        L.or_project_simplex_batch.argtypes = [i, i64, _dp, _dp, _ip]
        L.or_natural_residual.argtypes = [i, i, i, _dp, _dp, d, d]
        L.or_natural_residual.restype = d
        L.or_num_levels.argtypes = [i, i, i]
        ip = C.POINTER(C.c_int)
        dpp = C.POINTER(C.c_double)
        L.or_ssc_solve.argtypes = [i, i, i, _dp, _dp, d, d, d, i, i, i, i, ip, dpp]
        L.or_pgs_solve.argtypes = [i, i, i, _dp, _dp, d, d, d, i, ip, dpp]
        L.or_step.argtypes = [i, i, i, _dp, _dp, _dp, d, d, d, d, i, i, i, i, i, ip, dpp]
        L.or_labels.argtypes = [i, i, i, _dp, _bp, _bp]
        L.or_adjoint.argtypes = [i, i, i, _dp, _dp, i, d, d, d, _dp, dpp, dpp, _dp, C.c_void_p, d, i]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def n_nodes(W, H):
    return (W + 1) * (H + 1)


def assemble(W: int, H: int):
    """Lumped mass Mhat (n,) and stiffness A as a dense-row list: returns
    (mhat, cols (n,7), vals (n,7), cnt (n,)) assembled triangle by triangle."""
    n = n_nodes(W, H)
    mhat = np.zeros(n)
    col = np.zeros((n, ROW), np.int32)
    val = np.zeros((n, ROW))
    cnt = np.zeros(n, np.int32)
    if lib().or_assemble(W, H, mhat, col, val, cnt):
        raise ValueError("or_assemble failed")
    return mhat, col, val, cnt


PROJECTIONS = {"simplex": 0, "node": 1}


def moments(img: np.ndarray, projection: str = "simplex") -> np.ndarray:
    """Per-node image moments (n, 5): m0, m1 (RGB), m2 (Sec. 4.2).
    projection="simplex": exact integrals of the pixelwise-constant image
    against each hat function, triangle by triangle; "node": one image value
    per node (the pixel whose lower-left corner the node is, clamped to the
    last column and row) and the consistent mass matrix, m1 = M I, m2 = M |I|^2."""
    H, W, _ = img.shape
    m = np.zeros((n_nodes(W, H), 5))
    if projection == "node":
        lib().or_moments_node(W, H, _f64(img), m)
    elif projection == "simplex":
        lib().or_moments(W, H, _f64(img), m)
    else:
        raise ValueError(projection)
    return m


def means(u: np.ndarray, m: np.ndarray, W: int, H: int, c_prev=None):
    """Colour means c (N, 3) and masses (N,) of phase field u (n, N)."""
    N = u.shape[1]
    c = np.zeros((N, 3))
    mass = np.zeros(N)
    cp = None if c_prev is None else _f64(c_prev)
    lib().or_means(W, H, N, _f64(u), _f64(m), None if cp is None else cp.ctypes.data, c, mass.ctypes.data)
    return c, mass


def rhs(ut, m, c, W, H, eps, lam, tau):
    N = ut.shape[1]
    b = np.zeros_like(_f64(ut))
    lib().or_rhs(W, H, N, _f64(ut), _f64(m), _f64(c), eps, lam, tau, b)
    return b


def energy(u, m, W, H, eps, lam) -> float:
    return lib().or_energy(W, H, u.shape[1], _f64(u), _f64(m), eps, lam)


def project_simplex(y: np.ndarray):
    """Paper's clamp-and-redistribute projection of each row of y (k, N).
    Returns (x, passes)."""
    y = _f64(np.atleast_2d(y))
    x = np.zeros_like(y)
    passes = np.zeros(y.shape[0], np.int32)
    lib().or_project_simplex_batch(y.shape[1], y.shape[0], y, x, passes)
    return x, passes


def natural_residual(u, b, W, H, eps, tau) -> float:
    return lib().or_natural_residual(W, H, u.shape[1], _f64(u), _f64(b), eps, tau)


def num_levels(W, H, coarse_min=4) -> int:
    return lib().or_num_levels(W, H, coarse_min)


def ssc_solve(u0, b, W, H, eps, tau, tol=1e-13, max_iter=500, nu1=1, nu2=1, coarse_min=4):
    """Successive subspace correction over all levels. Returns (u, iters, rho, status)."""
    u = _f64(u0).copy()
    it, rho = C.c_int(0), C.c_double(0)
    st = lib().or_ssc_solve(W, H, u.shape[1], u, _f64(b), eps, tau, tol, max_iter, nu1, nu2, coarse_min,
                            C.byref(it), C.byref(rho))
    if st < 0:
        raise ValueError("or_ssc_solve: bad arguments")
    return u, it.value, rho.value, st


def pgs_solve(u0, b, W, H, eps, tau, tol=1e-13, max_sweeps=100000):
    """Plain lexicographic projected Gauss-Seidel. Returns (u, sweeps, rho, status)."""
    u = _f64(u0).copy()
    it, rho = C.c_int(0), C.c_double(0)
    st = lib().or_pgs_solve(W, H, u.shape[1], u, _f64(b), eps, tau, tol, max_sweeps, C.byref(it), C.byref(rho))
    if st < 0:
        raise ValueError("or_pgs_solve: bad arguments")
    return u, it.value, rho.value, st


def step(u, m, c, W, H, eps, lam, tau, tol=1e-13, method="ssc", max_iter=500, nu1=1, nu2=1, coarse_min=4):
    """One time step. Returns (u_next, c_t, iters, rho, status); c is the
    previous means (used for empty phases) and is not modified."""
    u = _f64(u).copy()
    c = _f64(c).copy()
    it, rho = C.c_int(0), C.c_double(0)
    meth = {"ssc": 0, "pgs": 1}[method]
    st = lib().or_step(W, H, u.shape[1], u, _f64(m), c, eps, lam, tau, tol, meth, max_iter, nu1, nu2, coarse_min,
                       C.byref(it), C.byref(rho))
    if st < 0:
        raise ValueError("or_step: bad arguments")
    return u, c, it.value, rho.value, st


def labels(u, W, H):
    """Rounded composite: (node labels (H+1, W+1), pixel labels (H, W)), int8."""
    nl = np.zeros(n_nodes(W, H), np.int8)
    pl = np.zeros(W * H, np.int8)
    lib().or_labels(W, H, u.shape[1], _f64(u), nl, pl)
    return nl.reshape(H + 1, W + 1), pl.reshape(H, W)


def _pixel_means(u, W, H, r=0):
    """Mean of each u_i over each image pixel: per cell of the right-diagonal
    split (2 u00 + u10 + u01 + 2 u11) / 6, averaged over the 4^r cells of the
    pixel when the solve grid is the W x H pixel grid refined r times.
    Returns (H, W, N)."""
    s = 1 << r
    U = np.asarray(u, dtype=np.float64).reshape(H * s + 1, W * s + 1, -1)
    cell = (2 * U[:-1, :-1] + U[:-1, 1:] + U[1:, :-1] + 2 * U[1:, 1:]) / 6.0
    return cell.reshape(H, s, W, s, -1).mean(axis=(1, 3))


def pixel_labels(u, W, H, r=0):
    """Pixel labels (Sec. 4.3): argmax_i of the pixel mean of u_i, lowest
    index on ties.  (H, W) int8."""
    return np.argmax(_pixel_means(u, W, H, r), axis=2).astype(np.int8)


def composite(u, c, W, H, rounded=False, r=0):
    """Composite image (Sec. 4.3): per pixel sum_i c_i ubar_i, ubar_i the mean
    of u_i over the pixel (both triangles of the right-diagonal split, i.e.
    (2 u00 + u10 + u01 + 2 u11) / 6 per cell); rounded: c of the pixel label
    (the rounded composite).  Returns (H, W, 3) float64."""
    ubar = _pixel_means(u, W, H, r)
    c = np.asarray(c, dtype=np.float64)
    if rounded:
        return c[np.argmax(ubar, axis=2)]
    return ubar @ c


def refine_image(img, r):
    """The pixel grid refined r times with data projection by copy (Sec. 4.1,
    4.2): every pixel becomes 2^r x 2^r cells carrying its colour (no
    interpolation, no new values)."""
    s = 1 << r
    return np.repeat(np.repeat(np.asarray(img, dtype=np.float64), s, axis=0), s, axis=1)


def refined_params(eps, lam, tau, r):
    """The step on the refined mesh in pixel units (cells of side h = 2^-r,
    eps, tau, lambda in pixel units) written on cells of side 1: the lumped
    mass and the fitting integrals scale with the cell area h^2, the 2-D P1
    stiffness does not scale, so S_px = h^2 (M + (tau eps / h^2) A) and
    b_px = h^2 (M u (1 + 2 tau/eps) - tau lambda f): the unit-cell step with
    eps' = 2^r eps, tau' = 2^r tau (tau' eps' = 4^r tau eps, tau'/eps' =
    tau/eps) and lambda' = 2^-r lambda (tau' lambda' = tau lambda).
    Returns (eps', lambda', tau')."""
    return eps * 2.0 ** r, lam * 2.0 ** -r, tau * 2.0 ** r


def run(img, u0, eps, lam, tau, steps, tol=1e-13, method="ssc", projection="simplex", **kw):
    """T steps from u0 on img (data projection by simplex or by node, Sec.
    4.2). Returns (u_T, c_last, per-step stats list)."""
    H, W, _ = img.shape
    m = moments(img, projection)
    u = _f64(u0)
    c = np.zeros((u.shape[1], 3))
    stats = []
    for _ in range(steps):
        u, c, it, rho, st = step(u, m, c, W, H, eps, lam, tau, tol=tol, method=method, **kw)
        stats.append((it, rho, st))
    return u, c, stats


def forward_states(img, u0, eps, lam, tau, steps, tol=1e-15, projection="simplex", **kw):
    """u^0..u^T of the oracle's time stepping (list of (n, N) arrays)."""
    H, W, _ = img.shape
    m = moments(img, projection)
    u = _f64(u0)
    c = np.zeros((u.shape[1], 3))
    states = [u.copy()]
    for _ in range(steps):
        u, c, it, rho, st = step(u, m, c, W, H, eps, lam, tau, tol=tol, **kw)
        states.append(u.copy())
    return states


def adjoint(img, states, eps, lam, tau, gT, cg_rtol=1e-13, projection="simplex"):
    """Gradients of a loss on u^T (gT = dL/du^T) through the steps that
    produced `states`: returns (dL/dlambda, dL/deps with tau fixed,
    dL/dI (H, W, 3), dL/du^0 (n, N)).  Each step's tangent system is solved
    by CG to cg_rtol relative residual (1e-13: above the rounding floor of
    the system, below which CG loses conjugacy)."""
    H, W, _ = img.shape
    T = len(states) - 1
    N = states[0].shape[1]
    st = np.ascontiguousarray(np.stack(states), dtype=np.float64)
    g_img = np.zeros((H, W, 3))
    g_u0 = np.zeros_like(st[0])
    gl, ge = C.c_double(0), C.c_double(0)
    if lib().or_adjoint(W, H, N, _f64(img), st, T, eps, lam, tau, _f64(gT), C.byref(gl), C.byref(ge), g_img,
                        g_u0.ctypes.data, cg_rtol, PROJECTIONS[projection]):
        raise ValueError("or_adjoint failed")
    return gl.value, ge.value, g_img, g_u0


def misfit_loss(u, m0, target):
    """L = 1/2 sum_n Mhat_n |u_n - onehot(target_n)|^2 and dL/du."""
    onehot = np.eye(u.shape[1])[target.ravel().astype(int)]
    diff = u - onehot
    return 0.5 * float((m0[:, None] * diff * diff).sum()), m0[:, None] * diff
