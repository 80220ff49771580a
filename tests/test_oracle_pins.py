"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-derived
golden values, closed forms, invariants, independent algorithms (sorting and
bisection projections, FISTA, a bounded least-squares library solver) or
symmetries of the triangulation.  No GPU needed.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import bruteforce as BF
from paper_0710_0736_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read_rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _img_2x2():
    I = {(0, 0): 1.0, (1, 0): 2.0, (0, 1): 4.0, (1, 1): 8.0}
    img = np.zeros((2, 2, 3))
    for (px, py), v in I.items():
        img[py, px] = (v, 2 * v, 0.0)
    return img


# --------------------------------------------------------------------------
# Triangulation and P1 matrices (Sec. 3.1)
# --------------------------------------------------------------------------

def test_golden_mass_and_moments_2x2(oracle_mod):
    m = oracle_mod.moments(_img_2x2())
    mhat, _, _, _ = oracle_mod.assemble(2, 2)
    for x, y, a, b, c, d in _read_rows("mesh_2x2.txt"):
        n = int(y) * 3 + int(x)
        m0 = Fraction(int(a), int(b))
        m1 = Fraction(int(c), int(d))
        assert m[n, 0] == pytest.approx(float(m0), abs=1e-15)
        assert mhat[n] == pytest.approx(float(m0), abs=1e-15)
        assert m[n, 1] == pytest.approx(float(m1), abs=1e-14)
        assert m[n, 2] == pytest.approx(2 * float(m1), abs=1e-14)
        assert m[n, 3] == 0.0


def test_golden_stiffness_2x2(oracle_mod):
    _, col, val, cnt = oracle_mod.assemble(2, 2)
    for x, y, dx, dy, a, b in _read_rows("stiffness_2x2.txt"):
        r = int(y) * 3 + int(x)
        c = (int(y) + int(dy)) * 3 + int(x) + int(dx)
        got = sum(val[r, k] for k in range(cnt[r]) if col[r, k] == c)
        assert got == pytest.approx(float(Fraction(int(a), int(b))), abs=1e-15)


def _dense_A(oracle_mod, W, H):
    mhat, col, val, cnt = oracle_mod.assemble(W, H)
    n = mhat.size
    A = np.zeros((n, n))
    for r in range(n):
        for k in range(cnt[r]):
            A[r, col[r, k]] += val[r, k]
    return mhat, A


def test_matrices_match_independent_assembly(oracle_mod):
    for W, H in [(3, 2), (5, 4)]:
        mhat, A = _dense_A(oracle_mod, W, H)
        mhat2, A2 = BF.assemble_dense(W, H)
        assert np.abs(mhat - mhat2).max() < 1e-14
        assert np.abs(A - A2).max() < 1e-13


@pytest.mark.parametrize("W,H", [(1, 1), (4, 3), (7, 5)])
def test_stiffness_invariants(oracle_mod, W, H):
    mhat, A = _dense_A(oracle_mod, W, H)
    assert mhat.sum() == pytest.approx(W * H, abs=1e-12)        # area of the domain
    assert np.abs(A - A.T).max() == 0.0                          # symmetric
    assert np.abs(A @ np.ones(A.shape[0])).max() < 1e-14         # constants in the kernel
    assert np.linalg.eigvalsh(A).min() > -1e-12                  # positive semi-definite
    # P1 reproduces linear functions: u'Au = int |grad u|^2 exactly.
    ys, xs = np.mgrid[0:H + 1, 0:W + 1]
    for a, b in [(1.0, 0.0), (0.0, 1.0), (0.3, -1.7)]:
        u = (a * xs + b * ys + 0.25).ravel()
        assert u @ A @ u == pytest.approx((a * a + b * b) * W * H, rel=1e-13)


# --------------------------------------------------------------------------
# Projection by simplex (Sec. 4.2)
# --------------------------------------------------------------------------

def test_moment_closed_forms(oracle_mod):
    rng = np.random.default_rng(3)
    W, H = 9, 7
    img = rng.uniform(0, 1, (H, W, 3))
    m = oracle_mod.moments(img)
    ys, xs = np.mgrid[0:H + 1, 0:W + 1]
    xs, ys = xs.ravel().astype(float), ys.ravel().astype(float)
    pys, pxs = np.mgrid[0:H, 0:W]
    # integrals of 1, I, |I|^2
    assert m[:, 0].sum() == pytest.approx(W * H, abs=1e-12)
    assert np.allclose(m[:, 1:4].sum(0), img.reshape(-1, 3).sum(0), atol=1e-12)
    assert m[:, 4].sum() == pytest.approx((img ** 2).sum(), abs=1e-12)
    # P1 is exact for x and y: sum_n x_n m1_n = int x I = sum_p I_p (px + 1/2)
    for ch in range(3):
        assert xs @ m[:, 1 + ch] == pytest.approx((img[..., ch] * (pxs + 0.5)).sum(), rel=1e-13)
        assert ys @ m[:, 1 + ch] == pytest.approx((img[..., ch] * (pys + 0.5)).sum(), rel=1e-13)
    # xy is not in P1: on pixel [a,a+1]x[c,c+1] its interpolant on the
    # right-diagonal split integrates to ac + a/2 + c/2 + 1/3 (the other
    # diagonal would give + 1/6), which pins the orientation of the split.
    want = (img[..., 0] * (pxs * pys + pxs / 2 + pys / 2 + 1 / 3)).sum()
    assert (xs * ys) @ m[:, 1] == pytest.approx(want, rel=1e-13)


def test_constant_image_moments(oracle_mod):
    img = np.empty((6, 5, 3))
    img[:] = (0.2, 0.5, 0.9)
    m = oracle_mod.moments(img)
    assert np.allclose(m[:, 1:4], m[:, :1] * np.array([0.2, 0.5, 0.9]), atol=1e-15)
    assert np.allclose(m[:, 4], m[:, 0] * (0.04 + 0.25 + 0.81), atol=1e-15)


# --------------------------------------------------------------------------
# Colour means, fitting term, energy (Eq. VV_fidelity, Eq. E, Sec. 4.4)
# --------------------------------------------------------------------------

def test_means_closed_forms(oracle_mod):
    rng = np.random.default_rng(4)
    W, H = 8, 6
    img = rng.uniform(0, 1, (H, W, 3))
    m = oracle_mod.moments(img)
    n = (W + 1) * (H + 1)
    # spatially uniform u: every phase's mean is the image mean
    u = np.tile([0.1, 0.6, 0.3], (n, 1))
    c, mass = oracle_mod.means(u, m, W, H)
    assert np.allclose(c, img.reshape(-1, 3).mean(0), atol=1e-14)
    assert np.allclose(mass, np.array([0.1, 0.6, 0.3]) * W * H, atol=1e-12)
    # u_1 = x/W, u_2 = 1 - x/W: int u_1 I = sum_p I_p (px + 1/2)/W, int u_1 = WH/2
    ys, xs = np.mgrid[0:H + 1, 0:W + 1]
    u1 = (xs / W).ravel()
    u = np.stack([u1, 1 - u1], 1)
    c, mass = oracle_mod.means(u, m, W, H)
    pys, pxs = np.mgrid[0:H, 0:W]
    w1 = (pxs + 0.5) / W
    assert np.allclose(c[0], (img * w1[..., None]).sum((0, 1)) / (W * H / 2), atol=1e-14)
    assert np.allclose(c[1], (img * (1 - w1)[..., None]).sum((0, 1)) / (W * H / 2), atol=1e-14)
    # an empty phase keeps the previous mean
    u = np.stack([np.ones(n), np.zeros(n)], 1)
    c, mass = oracle_mod.means(u, m, W, H, c_prev=np.array([[0, 0, 0], [0.7, 0.1, 0.2]]))
    assert mass[1] == 0.0 and np.allclose(c[1], [0.7, 0.1, 0.2])


def test_fitting_term_integrates_to_squared_error(oracle_mod):
    rng = np.random.default_rng(5)
    W, H = 7, 5
    img = rng.uniform(0, 1, (H, W, 3))
    m = oracle_mod.moments(img)
    n = (W + 1) * (H + 1)
    c = rng.uniform(0, 1, (3, 3))
    # with tau*lambda = 1 and u^t = 0, b = -f: sum_n f_n,i = int |I - c_i|^2
    b = oracle_mod.rhs(np.zeros((n, 3)), m, c, W, H, 1.0, 1.0, 1.0)
    for i in range(3):
        assert -b[:, i].sum() == pytest.approx(((img - c[i]) ** 2).sum(), rel=1e-13)


def test_energy_closed_forms(oracle_mod):
    rng = np.random.default_rng(6)
    W, H = 8, 5
    img = rng.uniform(0, 1, (H, W, 3))
    m = oracle_mod.moments(img)
    n = (W + 1) * (H + 1)
    eps, lam = 1.7, 0.6
    # a single pure phase: only the fitting term is left, lambda * int |I - mean I|^2
    u = np.zeros((n, 3))
    u[:, 1] = 1.0
    E = oracle_mod.energy(u, m, W, H, eps, lam)
    assert E == pytest.approx(lam * ((img - img.reshape(-1, 3).mean(0)) ** 2).sum(), rel=1e-13)
    # u_1 = x/W on a constant image: fitting term 0 (c_i = I); gradient term
    # eps/2 * 2 * (1/W^2) * W H; lumped potential (1/eps) sum_n Mhat_n * 2 s(1-s), s = x/W
    img[:] = (0.3, 0.3, 0.3)
    m = oracle_mod.moments(img)
    ys, xs = np.mgrid[0:H + 1, 0:W + 1]
    s = (xs / W).ravel()
    u = np.stack([s, 1 - s], 1)
    mhat, _ = BF.assemble_dense(W, H)
    want = eps * H / W + (2.0 / eps) * (mhat * s * (1 - s)).sum()
    assert oracle_mod.energy(u, m, W, H, eps, lam) == pytest.approx(want, rel=1e-13)


def test_rhs_is_energy_gradient(oracle_mod):
    """(S u - b(u))/tau equals the gradient of Eq. (E) minus the constant
    (1/eps) Mhat 1 (c enters only through means, whose own derivative
    vanishes at the mean); checked by central differences along directions
    that sum to zero at every node, where that constant drops out."""
    rng = np.random.default_rng(7)
    W, H = 6, 5
    img = rng.uniform(0, 1, (H, W, 3))
    m = oracle_mod.moments(img)
    n = (W + 1) * (H + 1)
    N, eps, lam, tau = 3, 1.3, 0.8, 0.7
    u = synth.dirichlet_init(1, n, N)
    c, _ = oracle_mod.means(u, m, W, H)
    b = oracle_mod.rhs(u, m, c, W, H, eps, lam, tau)
    mhat, A = BF.assemble_dense(W, H)
    S = np.diag(mhat) + tau * eps * A
    grad = (S @ u - b) / tau
    for k in range(4):
        v = rng.normal(size=(n, N))
        v -= v.mean(1, keepdims=True)
        h = 1e-5
        fd = (oracle_mod.energy(u + h * v, m, W, H, eps, lam) - oracle_mod.energy(u - h * v, m, W, H, eps, lam)) / (2 * h)
        assert fd == pytest.approx((grad * v).sum(), rel=1e-8, abs=1e-9)


# --------------------------------------------------------------------------
# Gibbs constraint (Sec. 3.3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_projection_matches_independent_methods(oracle_mod, N):
    rng = np.random.default_rng(N)
    Y = rng.normal(0, 1, (20000, N)) * rng.choice([0.01, 1, 10], size=(20000, 1))
    X, passes = oracle_mod.project_simplex(Y)
    scale = 1.0 + np.abs(Y).max(1, keepdims=True)   # rounding grows with |y|
    assert (np.abs(X - BF.project_sort(Y)) / scale).max() < 1e-15 * N
    assert (np.abs(X - BF.project_bisect(Y)) / scale).max() < 1e-14
    assert passes.max() <= N  # at most N repetitions (Sec. 3.3)
    assert X.min() >= 0 and (np.abs(X.sum(1, keepdims=True) - 1) / scale).max() < 1e-15 * N


def test_projection_special_cases(oracle_mod):
    rng = np.random.default_rng(1)
    F = synth.dirichlet_init(2, 1000, 5)          # feasible points are fixed
    X, passes = oracle_mod.project_simplex(F)
    assert np.abs(X - F).max() < 1e-15 and passes.max() == 1
    D = rng.uniform(0, 0.1, (100, 4))
    D[np.arange(100), rng.integers(0, 4, 100)] += 5.0  # a dominant component gives a vertex
    X, _ = oracle_mod.project_simplex(D)
    vert = (D == D.max(1, keepdims=True)).astype(float)
    assert np.array_equal(X > 0, vert > 0) and np.abs(X - vert).max() < 4e-15  # inputs ~5: a few ulps
    X, _ = oracle_mod.project_simplex(np.full((1, 4), 7.0))  # symmetric input -> barycentre
    assert np.allclose(X, 0.25, atol=1e-16)


# --------------------------------------------------------------------------
# The step problem (Sec. 3.2, Eq. alpha) and its solvers
# --------------------------------------------------------------------------

def _small_problem(oracle_mod, W=8, H=8, N=4, seed=0, eps=2.0, lam=1.0, tau=4.0):
    img = synth.shapes_image(seed, W, H, n_rect=2, n_disk=1, rect_side=(2, 5), disk_r=(1, 3), sigma=0.05)
    m = oracle_mod.moments(img)
    u = synth.dirichlet_init(seed + 10, (W + 1) * (H + 1), N)
    c, _ = oracle_mod.means(u, m, W, H)
    b = oracle_mod.rhs(u, m, c, W, H, eps, lam, tau)
    return img, m, u, b


@pytest.mark.parametrize("N,seed", [(2, 0), (4, 1), (8, 2)])
def test_step_matches_bruteforce_fista(oracle_mod, N, seed):
    W = H = 8
    eps, tau = 2.0, 4.0
    img, m, u, b = _small_problem(oracle_mod, W, H, N, seed)
    mhat, A = BF.assemble_dense(W, H)
    S = np.diag(mhat) + tau * eps * A
    xf, _ = BF.fista_step(S, b, u)
    us, _, rho_s, st_s = oracle_mod.ssc_solve(u, b, W, H, eps, tau, tol=1e-15, max_iter=5000)
    ug, _, rho_g, st_g = oracle_mod.pgs_solve(u, b, W, H, eps, tau, tol=1e-15)
    assert st_s == 0 and st_g == 0
    assert np.abs(us - xf).max() < 1e-12
    assert np.abs(ug - xf).max() < 1e-12
    spread, below = BF.kkt_violation(S, b, us)
    assert spread < 1e-12 and below < 1e-12


def test_two_phases_reduce_to_box_qp(oracle_mod):
    """N = 2: u_2 = 1 - u_1 turns the step into the scalar double-obstacle
    problem min u'(2S)u/2 - (b_1 - b_2 + S 1)'u over [0,1]^n, solved here with
    scipy's bounded-variable least squares (S = L L')."""
    scipy_opt = pytest.importorskip("scipy.optimize")
    W = H = 6
    eps, tau = 2.0, 4.0
    _, m, u, b = _small_problem(oracle_mod, W, H, 2, 5)
    mhat, A = BF.assemble_dense(W, H)
    S = np.diag(mhat) + tau * eps * A
    q = b[:, 0] - b[:, 1] + S @ np.ones(S.shape[0])
    Lc = np.linalg.cholesky(2 * S)
    # 1/2 u'(2S)u - q'u = 1/2 ||L'u - L^{-1} q||^2 + const
    res = scipy_opt.lsq_linear(Lc.T, np.linalg.solve(Lc, q), bounds=(0, 1), method="bvls", tol=1e-15)
    us, _, _, st = oracle_mod.ssc_solve(u, b, W, H, eps, tau, tol=1e-15, max_iter=5000)
    assert st == 0
    assert np.abs(us[:, 0] - res.x).max() < 1e-10


def test_constant_state_closed_form(oracle_mod):
    """Uniform u on a constant image: f = 0 and A u = 0, so the KKT
    conditions give u^{t+1} = P_G((1 + 2 tau/eps) u^t) at every node."""
    W, H, N = 16, 8, 4
    eps, lam, tau = 2.0, 1.0, 4.0
    img = np.empty((H, W, 3))
    img[:] = (0.4, 0.1, 0.7)
    m = oracle_mod.moments(img)
    n = (W + 1) * (H + 1)
    for w in ([0.4, 0.3, 0.2, 0.1], [0.26, 0.25, 0.25, 0.24]):
        u = np.tile(w, (n, 1))
        want, _ = BF.project_sort(np.array(w) * (1 + 2 * tau / eps)), None
        for method in ("ssc", "pgs"):
            u1, _, _, _, st = oracle_mod.step(u, m, np.zeros((N, 3)), W, H, eps, lam, tau, tol=1e-15, method=method)
            assert st == 0
            # error <= rho / (1 - q) with q ~ 1 - 1/(1 + 4 tau eps) the Jacobi factor
            assert np.abs(u1 - want).max() < 33 * 1.5e-15


def test_ssc_and_pgs_same_fixed_point_c1(oracle_mod):
    img = synth.config_image("c1_64_n4_fp64", 0)
    H, W, _ = img.shape
    m = oracle_mod.moments(img)
    u = synth.dirichlet_init(1, (W + 1) * (H + 1), 4)
    c, _ = oracle_mod.means(u, m, W, H)
    b = oracle_mod.rhs(u, m, c, W, H, 2.0, 1.0, 4.0)
    us, it, rho, st = oracle_mod.ssc_solve(u, b, W, H, 2.0, 4.0, tol=3e-15, nu1=2, nu2=2)
    ug, sw, rho2, st2 = oracle_mod.pgs_solve(u, b, W, H, 2.0, 4.0, tol=3e-15)
    assert st == 0 and st2 == 0
    assert it < sw  # the coarse levels do help
    assert np.abs(us - ug).max() < 1e-12


def test_invariants_and_energy_decrease(oracle_mod):
    """After every step: sum_i u_i = 1, 0 <= u <= 1, and the energy does not
    increase (convex-concave splitting, plus c being the minimiser over c)."""
    W = H = 32
    img = synth.config_image("c1_64_n4_fp64", 2, W, H)
    m = oracle_mod.moments(img)
    u = synth.dirichlet_init(3, (W + 1) * (H + 1), 4)
    c = np.zeros((4, 3))
    E = oracle_mod.energy(u, m, W, H, 2.0, 1.0)
    for _ in range(6):
        u, c, _, _, st = oracle_mod.step(u, m, c, W, H, 2.0, 1.0, 4.0, tol=1e-14, nu1=2, nu2=2)
        assert st == 0
        assert np.abs(u.sum(1) - 1).max() < 1e-14
        assert u.min() >= 0 and u.max() <= 1 + 4 * 2.0 ** -52   # a vertex is y - theta, rounded
        E1 = oracle_mod.energy(u, m, W, H, 2.0, 1.0)
        assert E1 <= E + 1e-9
        E = E1


def test_symmetries(oracle_mod):
    """The right-diagonal mesh is invariant under the 180-degree rotation and
    under transposition; the step commutes with both and with a permutation
    of the phases."""
    W, H, N = 24, 16, 3
    img = synth.shapes_image(7, W, H, rect_side=(3, 10), disk_r=(2, 6))
    u0 = synth.dirichlet_init(8, (W + 1) * (H + 1), N).reshape(H + 1, W + 1, N)

    def run(img, u0):
        Hh, Ww, _ = img.shape
        u, _, _ = oracle_mod.run(img, u0.reshape(-1, N), 2.0, 1.0, 4.0, 3, tol=1e-15, nu1=2, nu2=2)
        return u.reshape(Hh + 1, Ww + 1, N)

    base = run(img, u0)
    rot = run(img[::-1, ::-1].copy(), u0[::-1, ::-1].copy())
    assert np.abs(rot[::-1, ::-1] - base).max() < 1e-11
    tr = run(img.transpose(1, 0, 2).copy(), u0.transpose(1, 0, 2).copy())
    assert np.abs(tr.transpose(1, 0, 2) - base).max() < 1e-11
    perm = [2, 0, 1]
    pm = run(img, u0[..., perm].copy())
    assert np.abs(pm - base[..., perm]).max() < 1e-11


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_exact_segmentation_of_stripes(oracle_mod, seed):
    """A noise-free two-colour image of full-length straight stripes is
    segmented exactly: the pixel labels equal the stripe labels up to a swap."""
    W, H = 48, 24
    img = synth.stripes_image(W, H, [8, 12, 10, 18], [(0.9, 0.2, 0.1), (0.1, 0.3, 0.8)])
    truth = np.broadcast_to(((np.arange(W) >= 8) & (np.arange(W) < 20) | (np.arange(W) >= 30)).astype(np.int8), (H, W))
    u0 = synth.dirichlet_init(seed, (W + 1) * (H + 1), 2)
    u, _, _ = oracle_mod.run(img, u0, 2.0, 1.0, 4.0, 30, tol=1e-12)
    _, pl = oracle_mod.labels(u, W, H)
    assert np.array_equal(pl, truth) or np.array_equal(pl, 1 - truth)


def test_labels_golden(oracle_mod):
    rows = _read_rows("labels_1x1.txt")
    u = np.zeros((4, 2))
    for r in rows[:4]:
        x, y = int(r[0]), int(r[1])
        u[y * 2 + x] = (float(r[2]), float(r[3]))
    nl, pl = oracle_mod.labels(u, 1, 1)
    assert pl[0, 0] == int(rows[4][1])
    assert nl.ravel().tolist() == [int(v) for v in rows[5][1:]]
    # ties go to the lowest index
    nl, pl = oracle_mod.labels(np.full((4, 3), 1 / 3), 1, 1)
    assert nl.max() == 0 and pl[0, 0] == 0


def test_levels(oracle_mod):
    assert oracle_mod.num_levels(64, 64) == 5       # 64 -> 4 cells
    assert oracle_mod.num_levels(1024, 1024) == 9
    assert oracle_mod.num_levels(4096, 4096) == 11
    assert oracle_mod.num_levels(768, 512) == 8     # coarsest 6 x 4 cells
    assert oracle_mod.num_levels(37, 64) == 1       # odd cell count: no coarsening


# ---------------------------------------------------------------------------
# Composite image (Sec. 4.3)
# ---------------------------------------------------------------------------

def test_composite_of_constant_image_is_the_image(oracle_mod):
    """Every non-empty phase's mean is the constant colour and the pixel means
    of u sum to 1, so the composite (and the rounded composite) is the image."""
    W, H, N = 16, 12, 3
    u = synth.dirichlet_init(0, (W + 1) * (H + 1), N)
    img = np.full((H, W, 3), [0.3, 0.6, 0.1])
    c, _ = oracle_mod.means(u, oracle_mod.moments(img), W, H)
    assert np.abs(oracle_mod.composite(u, c, W, H) - img).max() < 1e-15
    assert np.abs(oracle_mod.composite(u, c, W, H, rounded=True) - img).max() < 1e-15


def test_composite_of_pure_phases_is_the_label_colour(oracle_mod):
    """A one-hot phase field (node labels) gives, at pixels whose four corners
    share a label, exactly that label's colour; rounded and plain agree there."""
    W, H, N = 20, 14, 4
    lab = synth.voronoi_labels(3, W + 1, H + 1, n_seeds=5, n_labels=N).reshape(-1)
    u = np.eye(N)[lab]
    c = np.random.default_rng(1).uniform(size=(N, 3))
    comp = oracle_mod.composite(u, c, W, H)
    rnd = oracle_mod.composite(u, c, W, H, rounded=True)
    L = lab.reshape(H + 1, W + 1)
    same = (L[:-1, :-1] == L[:-1, 1:]) & (L[:-1, :-1] == L[1:, :-1]) & (L[:-1, :-1] == L[1:, 1:])
    assert same.sum() > 100
    np.testing.assert_array_equal(comp[same], c[L[:-1, :-1][same]])
    np.testing.assert_array_equal(rnd[same], c[L[:-1, :-1][same]])


def test_composite_pixel_mean_is_exact_for_linear_fields(oracle_mod):
    """The pixel mean of a P1 function linear in x and y is its value at the
    pixel centre (x + 1/2, y + 1/2): pins the weights (2, 1, 1, 2)/6 and the
    orientation of the diagonal."""
    W, H = 9, 7
    y, x = np.meshgrid(np.arange(H + 1), np.arange(W + 1), indexing="ij")
    t = (0.1 + 0.03 * x + 0.05 * y) / (0.1 + 0.03 * W + 0.05 * H)
    u = np.stack([t.ravel(), 1 - t.ravel()], axis=1)
    c = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    comp = oracle_mod.composite(u, c, W, H)
    yc, xc = np.meshgrid(np.arange(H) + 0.5, np.arange(W) + 0.5, indexing="ij")
    tc = (0.1 + 0.03 * xc + 0.05 * yc) / (0.1 + 0.03 * W + 0.05 * H)
    assert np.abs(comp[..., 0] - tc).max() < 1e-15
    assert np.abs(comp[..., 1] - (1 - tc)).max() < 1e-15


# ---------------------------------------------------------------------------
# Pixel-grid refinement with data projection by copy (Sec. 4.1, 4.2)
# ---------------------------------------------------------------------------

def test_refined_step_is_the_pixel_unit_step(oracle_mod):
    """On the pixel grid refined r times (cells of side h = 2^-r in pixel
    units) the P1 lumped mass and the fitting integrals scale with the cell
    area h^2 and the 2-D stiffness does not scale.  The pixel-unit system
    (S_px, b_px) built from those facts equals 4^-r times the unit-cell system
    with refined_params(): same minimiser."""
    W0, H0, N, r = 6, 4, 3, 1
    eps, lam, tau = 2.0, 1.5, 4.0
    s = 1 << r
    W, H = W0 * s, H0 * s
    img = np.random.default_rng(0).uniform(size=(H0, W0, 3))
    fine = oracle_mod.refine_image(img, r)
    assert fine.shape == (H, W, 3) and np.array_equal(fine[::s, ::s], img)
    u = synth.dirichlet_init(1, (W + 1) * (H + 1), N)
    mhat, col, val, cnt = oracle_mod.assemble(W, H)
    m_unit = oracle_mod.moments(fine)
    c, _ = oracle_mod.means(u, m_unit, W, H)

    def A_times(v):
        out = np.zeros_like(v)
        for k in range(v.shape[0]):
            for j in range(cnt[k]):
                out[k] += val[k, j] * v[col[k, j]]
        return out

    h2 = 4.0 ** -r
    f_unit = (m_unit[:, 4:5] - 2 * m_unit[:, 1:4] @ c.T + m_unit[:, 0:1] * (c * c).sum(1)[None, :])
    S_px = h2 * mhat[:, None] * u + tau * eps * A_times(u)
    b_px = h2 * mhat[:, None] * u * (1 + 2 * tau / eps) - tau * lam * h2 * f_unit
    e2, l2, t2 = oracle_mod.refined_params(eps, lam, tau, r)
    S_unit = mhat[:, None] * u + t2 * e2 * A_times(u)
    b_unit = oracle_mod.rhs(u, m_unit, c, W, H, e2, l2, t2)
    assert np.abs(S_unit - S_px / h2).max() <= 1e-13 * np.abs(S_unit).max()
    assert np.abs(b_unit - b_px / h2).max() <= 1e-13 * np.abs(b_unit).max()


def test_refined_labels_reduce_to_the_plain_ones(oracle_mod):
    """r = 0: the pixel-mean labels are the oracle's pixel labels."""
    W, H, N = 15, 11, 4
    u = synth.dirichlet_init(3, (W + 1) * (H + 1), N)
    _, pl = oracle_mod.labels(u, W, H)
    np.testing.assert_array_equal(oracle_mod.pixel_labels(u, W, H, 0), pl)


@pytest.mark.parametrize("seed", [0, 1])
def test_refined_exact_segmentation_of_stripes(oracle_mod, seed):
    """The noise-free stripes of the exact-segmentation pin, solved on the
    pixel grid refined once (eps, tau, lambda in pixel units) from the P1
    interpolation of the unrefined start: the pixel labels are the stripe
    labels up to a swap, and at the unrefined grid's nodes the phase field is
    within the discretisation difference (0.1) of the unrefined solution.  (A
    random start drawn on the refined grid itself coarsens differently and may
    settle in another local minimum of the non-convex evolution.)"""
    W, H, r = 48, 24, 1
    img = synth.stripes_image(W, H, [8, 12, 10, 18], [(0.9, 0.2, 0.1), (0.1, 0.3, 0.8)])
    truth = np.broadcast_to(((np.arange(W) >= 8) & (np.arange(W) < 20) | (np.arange(W) >= 30)).astype(np.int8), (H, W))
    u0 = synth.dirichlet_init(seed, (W + 1) * (H + 1), 2)
    e2, l2, t2 = oracle_mod.refined_params(2.0, 1.0, 4.0, r)
    u, _, _ = oracle_mod.run(oracle_mod.refine_image(img, r), BF.prolong_p1(u0, W, H), e2, l2, t2, 30, tol=1e-12)
    pl = oracle_mod.pixel_labels(u, W, H, r)
    assert np.array_equal(pl, truth) or np.array_equal(pl, 1 - truth)
    uc, _, _ = oracle_mod.run(img, u0, 2.0, 1.0, 4.0, 30, tol=1e-12)
    assert np.abs(u.reshape(2 * H + 1, 2 * W + 1, 2)[::2, ::2] - uc.reshape(H + 1, W + 1, 2)).max() < 0.1


# --------------------------------------------------------------------------
# Data projection by node (Sec. 4.2): one image value per node, the
# consistent mass matrix
# --------------------------------------------------------------------------

def test_golden_node_moments_2x1(oracle_mod):
    img = np.zeros((1, 2, 3))
    img[0, 0] = (1.0, 2.0, 0.0)
    img[0, 1] = (4.0, 8.0, 2.0)
    m = oracle_mod.moments(img, "node")
    rows = _read_rows("node_moments_2x1.txt")
    assert len(rows) == 6
    for x, y, *vals in rows:
        n = int(y) * 3 + int(x)
        for k, v in enumerate(vals):
            assert m[n, k] == pytest.approx(int(v) / 24.0, abs=1e-14)


def test_node_moments_of_a_constant_image(oracle_mod):
    """The consistent mass matrix's rows sum to <eta_n, 1>: a constant image
    gives m1 = m0 I and m2 = m0 |I|^2, with the lumped mass as m0."""
    W, H = 7, 5
    img = np.empty((H, W, 3))
    img[:] = (0.2, 0.7, 0.4)
    m = oracle_mod.moments(img, "node")
    mhat, _, _, _ = oracle_mod.assemble(W, H)
    assert np.abs(m[:, 0] - mhat).max() < 1e-15
    assert np.abs(m[:, 1:4] - m[:, :1] * img[0, 0]).max() < 1e-15
    assert np.abs(m[:, 4] - m[:, 0] * (img[0, 0] ** 2).sum()).max() < 1e-15


def _node_values(img):
    """The copy rule: node (x, y) takes pixel (min(x, W-1), min(y, H-1))."""
    H, W, _ = img.shape
    ys = np.minimum(np.arange(H + 1), H - 1)
    xs = np.minimum(np.arange(W + 1), W - 1)
    return img[ys][:, xs]


def test_node_moments_integrate_the_interpolant(oracle_mod):
    """sum_n m1_n = sum_n (M I)_n = int I_h, the integral of the P1
    interpolant of the nodal values: on each triangle (area 1/2) the mean of
    its three vertex values; likewise sum_n m2_n for |I|^2."""
    W, H = 9, 6
    img = synth.shapes_image(4, W, H, rect_side=(1, 4), disk_r=(1, 3), sigma=0.1).astype(np.float64)
    m = oracle_mod.moments(img, "node")
    V = _node_values(img)
    V2 = (V ** 2).sum(axis=2)
    lo = (V[:-1, :-1] + V[:-1, 1:] + V[1:, 1:]) / 3.0      # (px,py), (px+1,py), (px+1,py+1)
    up = (V[:-1, :-1] + V[1:, :-1] + V[1:, 1:]) / 3.0      # (px,py), (px,py+1), (px+1,py+1)
    lo2 = (V2[:-1, :-1] + V2[:-1, 1:] + V2[1:, 1:]) / 3.0
    up2 = (V2[:-1, :-1] + V2[1:, :-1] + V2[1:, 1:]) / 3.0
    assert np.abs(m[:, 1:4].sum(0) - 0.5 * (lo + up).sum(axis=(0, 1))).max() < 1e-12
    assert abs(m[:, 4].sum() - 0.5 * (lo2 + up2).sum()) < 1e-12


def test_node_moments_of_a_linear_field(oracle_mod):
    """Pixel values linear in the pixel index give nodal values linear in
    (x, y) away from the last column and row; an interior node's hat function
    is point-symmetric, so its m1 is its own value (m0 = 1) exactly."""
    W, H = 8, 7
    py, px = np.mgrid[0:H, 0:W]
    img = np.stack([0.1 + 0.03 * px + 0.05 * py, 0.9 - 0.02 * px, 0.4 + 0.07 * py], axis=2)
    m = oracle_mod.moments(img, "node").reshape(H + 1, W + 1, 5)
    V = _node_values(img)
    inner = (slice(1, H - 1), slice(1, W - 1))
    assert np.abs(m[inner][..., 0] - 1.0).max() < 1e-15
    assert np.abs(m[inner][..., 1:4] - V[inner]).max() < 1e-14


def test_node_and_simplex_projections_converge_under_refinement(oracle_mod):
    """The paper notes that the errors of both projections decrease with
    every mesh refinement: on the pixel grid refined r times by copy, the two
    projections differ only in the cells along pixel edges, a band whose area
    halves with each r: the relative error of the by-node integral of I
    (against the exact one, sum_n m1 of the projection by simplex) halves, and the
    node-by-node difference of m1 shrinks towards the same rate."""
    W, H = 6, 5
    img = synth.shapes_image(9, W, H, rect_side=(1, 3), disk_r=(1, 2), sigma=0.2).astype(np.float64)
    total, nodewise = [], []
    for r in range(5):
        fine = oracle_mod.refine_image(img, r)
        a, b = oracle_mod.moments(fine, "node"), oracle_mod.moments(fine, "simplex")
        total.append(np.abs(a[:, 1:4].sum(0) - b[:, 1:4].sum(0)).sum() / np.abs(b[:, 1:4].sum(0)).sum())
        nodewise.append(np.abs(a[:, 1:4] - b[:, 1:4]).sum() / np.abs(b[:, 1:4]).sum())
    for e0, e1 in zip(total, total[1:]):
        assert 0.45 * e0 < e1 < 0.55 * e0
    for e0, e1 in zip(nodewise, nodewise[1:]):
        assert e1 < 0.8 * e0
    assert 0.45 * nodewise[-2] < nodewise[-1] < 0.55 * nodewise[-2]


def test_node_projection_step_kkt_and_fixed_point(oracle_mod):
    """A step with the by-node fitting terms: SSC and plain projected
    Gauss-Seidel reach the same minimiser, and it satisfies the KKT
    conditions of the step problem (Sec. 3.2) to 1e-12."""
    W, H, N = 12, 10, 3
    img = synth.shapes_image(5, W, H, rect_side=(2, 6), disk_r=(1, 3), sigma=0.05).astype(np.float64)
    u0 = synth.dirichlet_init(6, (W + 1) * (H + 1), N)
    m = oracle_mod.moments(img, "node")
    c, _ = oracle_mod.means(u0, m, W, H)
    b = oracle_mod.rhs(u0, m, c, W, H, 2.0, 1.0, 4.0)
    u1, _, rho1, st1 = oracle_mod.ssc_solve(u0, b, W, H, 2.0, 4.0, tol=1e-14, nu1=2, nu2=2)
    u2, _, rho2, st2 = oracle_mod.pgs_solve(u0, b, W, H, 2.0, 4.0, tol=1e-14)
    assert st1 == 0 and st2 == 0
    assert np.abs(u1 - u2).max() < 1e-11
    mhat, A = BF.assemble_dense(W, H)
    spread, below = BF.kkt_violation(np.diag(mhat) + 4.0 * 2.0 * A, b, u1)
    assert spread < 1e-12 and below < 1e-12
