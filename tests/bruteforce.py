"""Independent checkers used to pin the oracle (numpy only, no oracle code).

- a generic P1 assembly that inverts each triangle's vertex matrix (a
  different computation from the oracle's closed-form gradients);
- two simplex projections that are not the paper's loop: the sort-based
  method of Held, Wolfe & Crowder (1974) and bisection on the threshold;
- FISTA with gradient restart on the step problem (Beck & Teboulle 2009);
- the KKT certificate of the step problem.
"""
from __future__ import annotations

import numpy as np


def triangles(W, H):
    """Right-diagonal split of every pixel, as lists of (x, y) vertices."""
    out = []
    for py in range(H):
        for px in range(W):
            out.append([(px, py), (px + 1, py), (px + 1, py + 1)])
            out.append([(px, py), (px, py + 1), (px + 1, py + 1)])
    return out


def assemble_dense(W, H):
    """Dense lumped mass (vector) and stiffness matrix of P1 on the pixel grid.
    Barycentric coordinates come from inverting [1 x y] at the vertices."""
    n = (W + 1) * (H + 1)
    A = np.zeros((n, n))
    mhat = np.zeros(n)
    for tri in triangles(W, H):
        V = np.array([[1.0, x, y] for x, y in tri])
        Cm = np.linalg.inv(V)           # column k: coefficients of lambda_k
        G = Cm[1:3, :]                  # gradients (2 x 3)
        area = abs(np.linalg.det(V)) / 2
        idx = [y * (W + 1) + x for x, y in tri]
        A[np.ix_(idx, idx)] += area * G.T @ G
        mhat[idx] += area / 3
    return mhat, A


def project_sort(Y):
    """Euclidean projection of each row of Y onto the unit simplex by sorting."""
    Y = np.atleast_2d(np.asarray(Y, float))
    U = -np.sort(-Y, axis=1)
    css = np.cumsum(U, axis=1) - 1.0
    j = np.arange(1, Y.shape[1] + 1)
    cond = U - css / j > 0
    r = cond.shape[1] - 1 - np.argmax(cond[:, ::-1], axis=1)
    theta = css[np.arange(Y.shape[0]), r] / (r + 1)
    return np.maximum(Y - theta[:, None], 0.0)


def project_bisect(Y, iters=200):
    """Same projection by bisection on theta in sum_i max(y_i - theta, 0) = 1."""
    Y = np.atleast_2d(np.asarray(Y, float))
    lo = Y.min(axis=1) - 1.0
    hi = Y.max(axis=1)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        s = np.maximum(Y - mid[:, None], 0).sum(axis=1)
        big = s > 1
        lo = np.where(big, mid, lo)
        hi = np.where(big, hi, mid)
    return np.maximum(Y - 0.5 * (lo + hi)[:, None], 0.0)


def fista_step(S, B, U0, tol=1e-15, max_iter=200000):
    """min_U sum_i 1/2 U[:,i]' S U[:,i] - B[:,i]' U[:,i], each row of U on the
    simplex.  Projected gradient with Nesterov momentum and gradient restart."""
    L = np.linalg.eigvalsh(S).max()
    x = project_sort(U0)
    y = x.copy()
    t = 1.0
    for it in range(max_iter):
        g = S @ y - B
        xn = project_sort(y - g / L)
        if np.abs(xn - x).max() < tol:
            return xn, it
        tn = 0.5 * (1 + np.sqrt(1 + 4 * t * t))
        if np.sum((y - xn) * (xn - x)) > 0:  # restart
            tn = 1.0
            y = xn.copy()
        else:
            y = xn + (t - 1) / tn * (xn - x)
        x, t = xn, tn
    return x, max_iter


def kkt_violation(S, B, U, act_tol=1e-12):
    """KKT certificate of the step problem.  With g = S U - B, at each node the
    phases with u > 0 share one value mu_n and the phases at 0 have g >= mu_n.
    Returns (max spread of g over the inactive phases, max amount by which an
    active phase's g falls below mu_n)."""
    G = S @ U - B
    spread, below = 0.0, 0.0
    for n in range(U.shape[0]):
        inact = U[n] > act_tol
        if not inact.any():
            continue
        mu = G[n, inact].mean()
        spread = max(spread, np.abs(G[n, inact] - mu).max())
        if (~inact).any():
            below = max(below, max(0.0, mu - G[n, ~inact].min()))
    return spread, below


def prolong_p1(u, W, H):
    """P1 interpolation of a node field (n, N) on the W x H cell grid to the
    grid refined once (nested right-diagonal meshes: new nodes on axis edges
    take the mean of the edge's ends, new nodes on the SW-NE diagonal the mean
    of the diagonal's ends).  Returns ((2W+1)(2H+1), N)."""
    U = np.asarray(u, dtype=np.float64).reshape(H + 1, W + 1, -1)
    F = np.zeros((2 * H + 1, 2 * W + 1, U.shape[2]))
    F[::2, ::2] = U
    F[::2, 1::2] = 0.5 * (U[:, :-1] + U[:, 1:])
    F[1::2, ::2] = 0.5 * (U[:-1] + U[1:])
    F[1::2, 1::2] = 0.5 * (U[:-1, :-1] + U[1:, 1:])
    return F.reshape(-1, U.shape[2])
