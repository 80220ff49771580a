"""Pins of the oracle's adjoint against central finite differences of the
oracle's own forward (no GPU).  The forward is solved to 1e-15, so the
difference quotient (h = 1e-6) is accurate to ~1e-8 relative."""
import numpy as np
import pytest

from paper_0710_0736_gb300 import synth


def _problem(oracle_mod, seed=0, W=10, H=8, N=3, T=3):
    img = synth.shapes_image(seed, W, H, n_rect=2, n_disk=1, rect_side=(2, 5), disk_r=(1, 3), sigma=0.05)
    img = img.astype(np.float64)
    u0 = synth.dirichlet_init(seed + 1, (W + 1) * (H + 1), N)
    target = synth.voronoi_labels(seed + 2, W + 1, H + 1, n_seeds=4, n_labels=N)
    m0 = oracle_mod.moments(img)[:, 0]
    return img, u0, target, m0


def _loss(oracle_mod, img, u0, target, m0, eps, lam, tau, T, projection="simplex"):
    uT = oracle_mod.forward_states(img, u0, eps, lam, tau, T, projection=projection)[-1]
    return oracle_mod.misfit_loss(uT, m0, target)[0]


@pytest.mark.parametrize("seed,projection", [(0, "simplex"), (1, "simplex"), (2, "node")])
def test_adjoint_matches_finite_differences(oracle_mod, seed, projection):
    """Data projection by simplex or by node (Sec. 4.2): the image enters
    through the moments, whose adjoint differs between the two."""
    eps, lam, tau, T = 2.0, 1.0, 4.0, 3
    img, u0, target, m0 = _problem(oracle_mod, seed)
    states = oracle_mod.forward_states(img, u0, eps, lam, tau, T, projection=projection)
    L, gT = oracle_mod.misfit_loss(states[-1], m0, target)
    g_lam, g_eps, g_img, g_u0 = oracle_mod.adjoint(img, states, eps, lam, tau, gT, projection=projection)
    P = projection
    h = 1e-6

    def fd(f):
        return (f(h) - f(-h)) / (2 * h)

    def close(a, b):
        return abs(a - b) <= 1e-5 * max(abs(b), 1e-3 * abs(L))

    assert close(g_lam, fd(lambda d: _loss(oracle_mod, img, u0, target, m0, eps, lam + d, tau, T, P)))
    assert close(g_eps, fd(lambda d: _loss(oracle_mod, img, u0, target, m0, eps + d, lam, tau, T, P)))
    rng = np.random.default_rng(seed)
    for _ in range(6):
        py, px, ch = rng.integers(0, img.shape[0]), rng.integers(0, img.shape[1]), rng.integers(0, 3)

        def f(d, py=py, px=px, ch=ch):
            im = img.copy()
            im[py, px, ch] += d
            return _loss(oracle_mod, im, u0, target, m0, eps, lam, tau, T, P)
        assert close(g_img[py, px, ch], fd(f))
    for _ in range(2):  # a random direction in image space and one in u0 (sum zero per node)
        v = rng.normal(size=img.shape)
        assert close((g_img * v).sum(), fd(lambda d: _loss(oracle_mod, img + d * v, u0, target, m0, eps, lam, tau, T, P)))
        z = rng.normal(size=u0.shape)
        z -= z.mean(1, keepdims=True)
        assert close((g_u0 * z).sum(), fd(lambda d: _loss(oracle_mod, img, u0 + d * z, target, m0, eps, lam, tau, T, P)))
