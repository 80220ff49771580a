"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64 form: phase fields within 1e-10 max-abs of the oracle, labels equal
except where the oracle's top-two margin is below 1e-8 (both answers are then
valid).  Both sides solve each step to a natural residual of 3e-15 so that the
comparison measures the method, not the stopping point: the error of a step
is about 20x its residual, and the explicit 1 + 2 tau/eps factor amplifies
differences ~1000x over the first 20 steps of a random start.
"""
import numpy as np
import pytest

import oracle
from paper_0710_0736_gb300 import synth

pytestmark = pytest.mark.gpu

TIGHT = 3e-15


@pytest.fixture(scope="module")
def ac():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0710_0736_gb300 import build
    build.build()
    from paper_0710_0736_gb300 import ac as mod
    oracle.build()
    return mod


def _seg(ac, W, H, N, eps=2.0, lam=1.0, tau=4.0, **kw):
    kw.setdefault("tol", TIGHT)
    kw.setdefault("max_cycles", 2000)
    return ac.Segmenter(W, H, N, eps, lam, tau, **kw)


def _label_mismatch_ok(u_ref, lab_gpu, lab_ref, W, H, margin=1e-8):
    """Pixels whose labels differ must be near-ties of the oracle's field."""
    diff = np.argwhere(lab_gpu != lab_ref)
    if diff.size == 0:
        return True
    N = u_ref.shape[1]
    U = u_ref.reshape(H + 1, W + 1, N)
    for py, px in diff:
        v = 2 * U[py, px] + U[py, px + 1] + U[py + 1, px] + 2 * U[py + 1, px + 1]
        s = np.sort(v)
        if s[-1] - s[-2] > 6 * margin:
            return False
    return True


def _node_mismatch_ok(u_ref, nl_gpu, nl_ref, margin=1e-8):
    """Nodes whose labels differ must be near-ties of the oracle's field: its
    top two phase values there differ by less than `margin` (both answers
    are then valid)."""
    diff = np.flatnonzero(nl_gpu.ravel() != nl_ref.ravel())
    if diff.size == 0:
        return True
    s = np.sort(u_ref[diff], axis=1)
    return bool((s[:, -1] - s[:, -2] < margin).all())


def _check_labels(seg, u_gpu, u_ref, W, H, margin=1e-8):
    """Node and pixel labels (Sec. 4.3): bit-exact against the oracle's rule
    applied to the GPU's own field, and equal to the oracle's labels of its
    own field except at near-ties."""
    nl, lab = seg.node_labels(), seg.segment(0)
    nl_own, lab_own = oracle.labels(u_gpu, W, H)
    assert np.array_equal(nl, nl_own) and np.array_equal(lab, lab_own)
    nl_ref, lab_ref = oracle.labels(u_ref, W, H)
    assert _node_mismatch_ok(u_ref, nl, nl_ref, margin)
    assert _label_mismatch_ok(u_ref, lab, lab_ref, W, H, margin)
    return int((nl != nl_ref).sum()), int((lab != lab_ref).sum())


# --------------------------------------------------------------------------
# a1, a2, a3, a5: moments, means, right-hand side, energy, projection
# --------------------------------------------------------------------------

def test_moments_golden_and_c1(ac):
    img = np.zeros((2, 2, 3))
    for (px, py), v in {(0, 0): 1.0, (1, 0): 2.0, (0, 1): 4.0, (1, 1): 8.0}.items():
        img[py, px] = (v, 2 * v, 0)
    def close(a, b):  # ~9 ulps: six-term sums in another order, with FMA contraction on the GPU
        return (np.abs(a - b) <= 2e-15 * np.maximum(1.0, np.abs(b))).all()

    seg = _seg(ac, 2, 2, 2)
    seg.set_image(img)
    assert close(seg.moments(), oracle.moments(img))
    img = synth.config_image("c1_64_n4_fp64", 0).astype(np.float64)
    seg = _seg(ac, 64, 64, 4)
    seg.set_image(img)
    assert close(seg.moments(), oracle.moments(img))
    seg32 = _seg(ac, 64, 64, 4)
    seg32.set_image(img.astype(np.float32))          # float32 input path, same values
    assert close(seg32.moments(), oracle.moments(img))


@pytest.mark.parametrize("N", [2, 3, 4, 5, 6, 7, 8])
def test_projection_kernel(ac, N):
    import torch
    rng = np.random.default_rng(N)
    Y = rng.normal(0, 1, (50001, N)) * rng.choice([0.01, 1, 10], size=(50001, 1))
    y = torch.tensor(Y, device="cuda")
    x = torch.empty_like(y)
    ac.ac_project_simplex(y, x, Y.shape[0], N)
    torch.cuda.synchronize()
    X = x.cpu().numpy()
    ref, _ = oracle.project_simplex(Y)
    scale = 1 + np.abs(Y).max(1, keepdims=True)
    assert (np.abs(X - ref) / scale).max() < 1e-15 * N
    assert X.min() >= 0


def test_means_rhs_energy(ac):
    W = H = 64
    img = synth.config_image("c1_64_n4_fp64", 1).astype(np.float64)
    u0 = synth.dirichlet_init(2, (W + 1) * (H + 1), 4)
    m = oracle.moments(img)
    seg = _seg(ac, W, H, 4)
    seg.set_image(img)
    seg.set_phase(u0)
    E_gpu = seg.energy()
    assert E_gpu == pytest.approx(oracle.energy(u0, m, W, H, 2.0, 1.0), rel=1e-13)
    seg.step(1)
    c_ref, _ = oracle.means(u0, m, W, H)
    assert np.abs(seg.means() - c_ref).max() < 1e-14
    b_ref = oracle.rhs(u0, m, c_ref, W, H, 2.0, 1.0, 4.0)
    assert np.abs(seg.rhs() - b_ref).max() < 1e-13


@pytest.mark.parametrize("W,H,N", [(64, 64, 4), (37, 23, 3), (96, 64, 8)])
def test_mixed_means_rhs_energy_double_float(ac, W, H, N):
    """The mixed form forms the colour means, the energy and the right-hand
    side in double-float arithmetic (about 2^-46 of the terms' magnitudes):
    against the FP64 oracle on the BF16-rounded image, with and without the
    energy terms in the same pass."""
    img = synth.shapes_image(W * 7 + H, W, H, rect_side=(1, max(1, W // 2)), disk_r=(1, max(1.5, W / 4)))
    m = oracle.moments(synth.round_bf16(img).astype(np.float64))
    u0 = synth.dirichlet_init(W + H, (W + 1) * (H + 1), N)
    c_ref, _ = oracle.means(u0, m, W, H)
    b_ref = oracle.rhs(u0, m, c_ref, W, H, 2.0, 1.0, 4.0)
    E_ref = oracle.energy(u0, m, W, H, 2.0, 1.0)
    for with_energy in (False, True):
        seg = _mixed(ac, W, H, N, 1e-6)
        seg.set_image(img)
        seg.set_phase(u0)
        if with_energy:
            st = seg.step(1)
            assert st.energy == pytest.approx(E_ref, rel=1e-12)
        else:
            assert ac.lib.ac_step(seg.ctx, 1, None) == ac.AC_OK
        assert np.abs(seg.means() - c_ref).max() < 1e-13
        assert np.abs(seg.rhs() - b_ref).max() < 2e-12 * max(1.0, np.abs(b_ref).max())


# --------------------------------------------------------------------------
# a4-a9: the step solve
# --------------------------------------------------------------------------

def test_one_step_c1(ac):
    W = H = 64
    img = synth.config_image("c1_64_n4_fp64", 0).astype(np.float64)
    u0 = synth.dirichlet_init(1, (W + 1) * (H + 1), 4)
    seg = _seg(ac, W, H, 4)
    seg.set_image(img)
    seg.set_phase(u0)
    st = seg.step(1)
    assert st.converged and st.residual <= TIGHT
    u_ref, _, it, rho, stt = oracle.step(u0, oracle.moments(img), np.zeros((4, 3)), W, H, 2.0, 1.0, 4.0, tol=TIGHT,
                                         nu1=2, nu2=2)
    assert stt == 0
    assert np.abs(seg.phase() - u_ref).max() < 1e-12
    assert seg.residual() <= TIGHT


def test_trajectory_c1_20_steps(ac):
    W = H = 64
    img = synth.config_image("c1_64_n4_fp64", 0).astype(np.float64)
    u0 = synth.dirichlet_init(1, (W + 1) * (H + 1), 4)
    seg = _seg(ac, W, H, 4)
    seg.set_image(img)
    seg.set_phase(u0)
    lab = seg.segment(20)
    u = seg.phase()
    u_ref, c_ref, stats = oracle.run(img, u0, 2.0, 1.0, 4.0, 20, tol=TIGHT, nu1=2, nu2=2)
    assert all(s[2] == 0 for s in stats)
    assert np.abs(u - u_ref).max() < 1e-10
    assert np.abs(seg.means() - c_ref).max() < 1e-10
    assert np.array_equal(lab, seg.segment(0))
    _check_labels(seg, u, u_ref, W, H)


@pytest.fixture(scope="module")
def tiled_coarse_cases():
    """Grids whose first coarse level is too large for the one-launch coarse
    tail (7 arrays per node of 4 or 8 bytes, 200 KB cap), so that the tiled
    coarse kernels (fused Jacobi pairs with the level's residual, restriction,
    Galerkin products, prolongation) run on it: 256^2 with N = 8 (level 1:
    129^2 nodes, 466 KB in float) and 320 x 192 with N = 5 (161 x 97 nodes,
    437 KB, rows that are not a multiple of the 32-node tile).  The oracle
    (SSC, Sec. 3.2) takes one step from the random start to reach a
    phase-separated state u1, then the step from u1 is compared, on the
    float image (FP64 form) and on its bfloat16 rounding (mixed form)."""
    out = {}
    for (W, H, N) in [(256, 256, 8), (320, 192, 5)]:
        assert 7 * 4 * (W // 2 + 1) * (H // 2 + 1) > 200 * 1024
        img = synth.shapes_image(W + H, W, H, rect_side=(8, W // 3), disk_r=(4, W / 6))
        u0 = synth.dirichlet_init(W * H, (W + 1) * (H + 1), N)
        for form, im in (("fp64", img.astype(np.float64)), ("mixed", synth.round_bf16(img).astype(np.float64))):
            m = oracle.moments(im)
            u1, c1, _, _, st1 = oracle.step(u0, m, np.zeros((N, 3)), W, H, 2.0, 1.0, 4.0, tol=TIGHT)
            u2, _, _, rho2, st2 = oracle.step(u1, m, c1, W, H, 2.0, 1.0, 4.0, tol=TIGHT)
            assert st1 == 0 and st2 == 0
            out[(W, H, N, form)] = dict(img=img, u1=u1, u2=u2)
    return out


@pytest.mark.parametrize("W,H,N", [(256, 256, 8), (320, 192, 5)])
@pytest.mark.parametrize("form,tol,bound", [("fp64", TIGHT, 1e-10), ("mixed", 1e-6, 25e-6), ("mixed", 1e-12, 1e-10)])
def test_one_step_tiled_coarse_levels(ac, tiled_coarse_cases, W, H, N, form, tol, bound):
    """One step from the oracle's phase-separated u1, element by element
    against the oracle's u2, where the first coarse level runs through the
    tiled kernels: the FP64 form to 1e-10 (both solved to 3e-15), the mixed
    form to 25 tol at tol 1e-6 and to 1e-10 at tol 1e-12; node and pixel
    labels bit-exact from the GPU's own field and equal to the oracle's except
    at near-ties."""
    case = tiled_coarse_cases[(W, H, N, form)]
    prec = ac.AC_MIXED if form == "mixed" else ac.AC_FP64
    seg = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=tol, max_cycles=3000, precision=prec)
    seg.set_image(case["img"] if form == "mixed" else case["img"].astype(np.float64))
    seg.set_phase(case["u1"])
    st = seg.step(1)
    assert st.converged and st.total_cycles > 1
    u = seg.phase()
    assert np.abs(u - case["u2"]).max() < bound
    assert np.abs(u.sum(1) - 1).max() < 1e-13 and u.min() >= 0
    # the first step's colour means are those of u1 on the oracle's side; the
    # labels of the new field
    _check_labels(seg, u, case["u2"], W, H, margin=max(1e-8, 10 * bound))
    seg.close()


@pytest.mark.parametrize("W,H,N", [(37, 23, 3), (1, 1, 2), (2, 1, 4), (1, 5, 8), (48, 40, 2), (96, 64, 8),
                                   (34, 66, 5), (24, 24, 7), (40, 24, 6)])
def test_ragged_sizes(ac, W, H, N):
    """Single-level grids, odd sizes, degenerate 1-pixel-wide images, and grids
    that coarsen a few times, for every phase count."""
    img = synth.shapes_image(W * 7 + H, W, H, rect_side=(1, max(1, W // 2)), disk_r=(1, max(1.5, W / 4))).astype(np.float64)
    u0 = synth.dirichlet_init(W + H, (W + 1) * (H + 1), N)
    seg = _seg(ac, W, H, N)
    seg.set_image(img)
    seg.set_phase(u0)
    seg.step(3)
    u_ref, _, stats = oracle.run(img, u0, 2.0, 1.0, 4.0, 3, tol=TIGHT, nu1=2, nu2=2)
    assert np.abs(seg.phase() - u_ref).max() < 1e-11


def test_pixel_labels_at_near_ties(ac):
    """Pixel labels (Sec. 4.3) on a field built of near-ties: phases 0 and 1
    at 0.4 + e and 0.4 - e per node with e >= 0 drawn from 0 to 1e-5, so the
    two pixel sums differ by 0 (an exact tie: the lowest index) to about
    1e-4, on both sides of the float filter's 4e-6 margin.  The labels must
    be the oracle's rule on the same field, bit for bit, and the node labels
    too."""
    W, H, N = 64, 48, 4
    rng = np.random.default_rng(5)
    levels = np.array([0.0, 0.0, 1e-9, 1e-8, 1e-7, 3e-7, 6e-7, 1e-6, 2e-6, 3e-6, 1e-5])
    e = levels[rng.integers(0, levels.size, (H + 1) * (W + 1))]
    e[: 5 * (W + 1)] = 0.0  # pixel rows 0..3: exact ties
    u = np.empty(((H + 1) * (W + 1), N))
    u[:, 0] = 0.4 + e
    u[:, 1] = 0.4 - e
    u[:, 2:] = 0.1
    seg = _seg(ac, W, H, N)
    seg.set_image(np.zeros((H, W, 3), np.float32))
    seg.set_phase(u)
    u_gpu = seg.phase()
    assert np.array_equal(u_gpu, u)
    nl_own, lab_own = oracle.labels(u, W, H)
    lab = seg.segment(0)
    assert np.array_equal(lab, lab_own)
    assert np.array_equal(seg.node_labels(), nl_own)
    # the field holds exact ties and margins around the filter's threshold
    U = u.reshape(H + 1, W + 1, N)
    v = 2 * U[:-1, :-1] + U[:-1, 1:] + U[1:, :-1] + 2 * U[1:, 1:]
    m = v[..., 0] - v[..., 1]
    assert (m == 0).any() and ((m > 0) & (m < 4e-6)).any() and (m > 1e-5).any()
    seg.close()


def test_empty_phase_and_constant_state(ac):
    W, H, N = 32, 16, 4
    img = synth.config_image("c1_64_n4_fp64", 3, W, H).astype(np.float64)
    u0 = synth.dirichlet_init(5, (W + 1) * (H + 1), N)
    u0[:, 2] = 0
    u0 /= u0.sum(1, keepdims=True)
    seg = _seg(ac, W, H, N)
    seg.set_image(img)
    seg.set_phase(u0)
    seg.step(2)
    u_ref, _, _ = oracle.run(img, u0, 2.0, 1.0, 4.0, 2, tol=TIGHT, nu1=2, nu2=2)
    assert np.abs(seg.phase() - u_ref).max() < 1e-11
    # constant image, uniform u: closed form u1 = P_G((1 + 2 tau/eps) u0) at every node
    img = np.empty((H, W, 3))
    img[:] = (0.3, 0.6, 0.1)
    w = np.array([0.26, 0.25, 0.25, 0.24])
    seg.set_image(img)
    seg.set_phase(np.tile(w, ((W + 1) * (H + 1), 1)))
    seg.step(1)
    want, _ = oracle.project_simplex(w * (1 + 2 * 4.0 / 2.0))
    assert np.abs(seg.phase() - want).max() < 5e-14


@pytest.mark.parametrize("seed", [0, 1])
def test_exact_segmentation_of_stripes(ac, seed):
    W, H = 48, 24
    img = synth.stripes_image(W, H, [8, 12, 10, 18], [(0.9, 0.2, 0.1), (0.1, 0.3, 0.8)])
    truth = np.broadcast_to(((np.arange(W) >= 8) & (np.arange(W) < 20) | (np.arange(W) >= 30)).astype(np.int8), (H, W))
    seg = _seg(ac, W, H, 2, tol=1e-12, seed=seed)
    seg.set_image(img)                      # float32 path + the library's own seeded start
    lab = seg.segment(30)
    assert np.array_equal(lab, truth) or np.array_equal(lab, 1 - truth)


def test_seeded_init_on_simplex(ac):
    W, H, N = 64, 48, 6
    seg = _seg(ac, W, H, N, seed=123)
    seg.set_image(np.zeros((H, W, 3), np.float32))
    u = seg.phase()
    assert np.abs(u.sum(1) - 1).max() < 1e-14 and u.min() > 0
    assert np.abs(u.mean(0) - 1 / N).max() < 0.01          # Dirichlet(1..1) mean
    seg2 = _seg(ac, W, H, N, seed=123)
    seg2.set_image(np.zeros((H, W, 3), np.float32))
    assert np.array_equal(u, seg2.phase())


def test_deterministic_and_device_buffers(ac):
    import torch
    W = H = 64
    img = synth.config_image("c1_64_n4_fp64", 4)
    outs = []
    for _ in range(2):
        seg = _seg(ac, W, H, 4, tol=1e-10, seed=9)
        seg.set_image(torch.tensor(img, device="cuda"))
        lab = torch.empty((H, W), dtype=torch.int8, device="cuda")
        ac.ac_segment(seg.ctx, 5, lab, W, H)
        torch.cuda.synchronize()
        outs.append((seg.phase(), lab.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_graphs_match_direct_launches(ac, precision):
    """On a capturable stream the V-cycle halves run as CUDA graphs; on the
    legacy default stream they are launched one by one.  Same arithmetic,
    same order: the results must be bit-identical, profiling on or off."""
    W, H, N = 96, 64, 5
    img = synth.shapes_image(11, W, H, rect_side=(4, 30), disk_r=(3, 12))
    u0 = synth.dirichlet_init(12, (W + 1) * (H + 1), N)
    import torch
    prec = ac.AC_MIXED if precision == "mixed" else ac.AC_FP64
    outs = []
    side = torch.cuda.Stream()
    for stream, prof in [(None, False), ("side", False), ("side", True)]:
        kw = {"stream": side.cuda_stream if stream == "side" else None}
        seg = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=1e-9, precision=prec, **kw)
        seg.set_image(img)
        seg.set_phase(u0)
        ac.ac_set_profiling(seg.ctx, prof)
        # the V-cycle halves as graphs, with the host loop (the device-side
        # loop has its own test)
        ac.ac_set_cycle_loop(seg.ctx, ac.AC_LOOP_HOST)
        assert not seg.loop_on_device()
        st = seg.step(4)
        outs.append(seg.phase())
        if prof:
            p = ac.ac_get_profile(seg.ctx).as_dict()
            assert p["launches"]["smooth"] > 0 and p["ms"]["smooth"] > 0 and st.fine_sweeps > 0
        seg.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def _stream_seg(ac, W, H, N, stream, **kw):
    return ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, stream=stream.cuda_stream, **kw)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("W,H,N,nu1,nu2,max_cycles", [(96, 64, 5, 2, 1, 200), (37, 23, 3, 2, 2, 200),
                                                      (1, 1, 2, 1, 1, 200), (64, 48, 4, 0, 2, 200),
                                                      (128, 128, 8, 2, 1, 3)])
def test_device_loop_matches_host_loop(ac, precision, W, H, N, nu1, nu2, max_cycles):
    """The V-cycle loop run on the device (graph WHILE nodes, conditions set
    from rho by one-thread kernels) takes the decisions of the host loop:
    bit-identical fields, the same statistics and return codes -- also with
    no coarse level (1 x 1), no pre-smoothing (no warm start), and a cycle
    cap that stops every step unconverged."""
    import torch
    prec = ac.AC_MIXED if precision == "mixed" else ac.AC_FP64
    img = synth.shapes_image(21, W, H, rect_side=(1, max(1, W // 3)), disk_r=(1, max(1.5, W / 5)))
    u0 = synth.dirichlet_init(22, (W + 1) * (H + 1), N)
    st = torch.cuda.Stream()
    res = []
    for mode in (ac.AC_LOOP_HOST, ac.AC_LOOP_AUTO):
        seg = _stream_seg(ac, W, H, N, st, tol=1e-9, precision=prec, nu1=nu1, nu2=nu2, max_cycles=max_cycles)
        seg.set_cycle_loop(mode)
        assert seg.loop_on_device() == (mode == ac.AC_LOOP_AUTO)
        seg.set_image(img)
        seg.set_phase(u0)
        stats = []
        for n in (1, 3, 2):  # several calls: the warm start carries across them
            rc, s = ac.ac_step(seg.ctx, n, allow_not_converged=True)
            stats.append((rc, s.as_dict()))
        # a capture failure would drop the context to the host loop silently
        assert seg.loop_on_device() == (mode == ac.AC_LOOP_AUTO)
        res.append((seg.phase(), stats, seg.node_labels()))
        seg.close()
    (u_h, st_h, nl_h), (u_d, st_d, nl_d) = res
    assert np.array_equal(u_h, u_d)
    assert np.array_equal(nl_h, nl_d)
    assert st_h == st_d
    if max_cycles == 3:
        assert all(rc == ac.AC_ERR_NOT_CONVERGED and s["converged"] == 0 for rc, s in st_d)


@pytest.mark.parametrize("W,H,N", [(256, 256, 8), (320, 192, 5)])
@pytest.mark.parametrize("form,tol,bound", [("fp64", TIGHT, 1e-10), ("mixed", 1e-12, 1e-10)])
@pytest.mark.parametrize("tiling", ["auto", "always"])
def test_coarse_smoothers_reach_the_same_minimiser(ac, tiled_coarse_cases, W, H, N, form, tol, bound, tiling):
    """The coarse levels' 3-colour Gauss-Seidel and l1-Jacobi take different
    cycles to the same step minimiser (Sec. 3.2): one step from the oracle's
    phase-separated u1 matches the oracle's u2 element by element with either
    smoother, with dense coarse levels and with AC_TILES_ALWAYS (the live-tile
    lists), and Gauss-Seidel needs no more V-cycles than Jacobi."""
    import torch
    case = tiled_coarse_cases[(W, H, N, form)]
    prec = ac.AC_MIXED if form == "mixed" else ac.AC_FP64
    st = torch.cuda.Stream()
    cyc = {}
    for mode in (ac.AC_SMOOTH_GS3, ac.AC_SMOOTH_JACOBI):
        seg = _stream_seg(ac, W, H, N, st, tol=tol, precision=prec, max_cycles=3000)
        ac.ac_set_coarse_smoother(seg.ctx, mode)
        if tiling == "always":
            ac.ac_set_coarse_tiling(seg.ctx, ac.AC_TILES_ALWAYS)
        seg.set_image(case["img"] if form == "mixed" else case["img"].astype(np.float64))
        seg.set_phase(case["u1"])
        cyc[mode] = seg.step(1).total_cycles
        err = np.abs(seg.phase() - case["u2"]).max()
        assert err < bound, f"smoother {mode}: {err:.3e}"
        seg.close()
    assert cyc[ac.AC_SMOOTH_GS3] <= cyc[ac.AC_SMOOTH_JACOBI]
    with pytest.raises(ac.AcError):
        ac.ac_set_coarse_smoother(None, ac.AC_SMOOTH_GS3)


def test_device_loop_eligibility(ac):
    """The loop runs on the device only with a stream, profiling off and no
    coarse level that can run tiled; the legacy default stream, profiling and
    a tiled hierarchy keep it on the host."""
    import torch
    st = torch.cuda.Stream()
    seg = _stream_seg(ac, 64, 64, 4, st)
    assert seg.loop_on_device()
    ac.ac_set_profiling(seg.ctx, True)
    assert not seg.loop_on_device()
    ac.ac_set_profiling(seg.ctx, False)
    assert seg.loop_on_device()
    seg.close()
    seg = ac.Segmenter(64, 64, 4, 2.0, 1.0, 4.0, stream=None)
    assert not seg.loop_on_device()
    seg.close()
    seg = _stream_seg(ac, 256, 256, 8, st)
    assert seg.loop_on_device()  # AUTO: level 1 too small for tiles
    ac.ac_set_coarse_tiling(seg.ctx, ac.AC_TILES_ALWAYS)
    assert not seg.loop_on_device()
    seg.close()
    with pytest.raises(ac.AcError):
        ac.ac_set_cycle_loop(None, ac.AC_LOOP_AUTO)


def test_profiling_mask(ac):
    """ac_set_profiling_mask: events (time) only around the chosen classes,
    every class's launches still counted; switching back to all classes
    re-captures the graphs with every event.  The arithmetic is unchanged."""
    W, H, N = 96, 64, 5
    img = synth.shapes_image(11, W, H, rect_side=(4, 30), disk_r=(3, 12))
    u0 = synth.dirichlet_init(12, (W + 1) * (H + 1), N)
    outs = []
    for mode in ("all", "smooth", "off"):
        seg = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=1e-9, precision=ac.AC_MIXED)
        seg.set_image(img)
        seg.set_phase(u0)
        if mode == "all":
            ac.ac_set_profiling(seg.ctx, True)
        elif mode == "smooth":
            ac.ac_set_profiling_mask(seg.ctx, ["smooth"])
        seg.step(3)
        outs.append(seg.phase())
        if mode == "smooth":
            p = ac.ac_get_profile(seg.ctx).as_dict()
            assert p["ms"]["smooth"] > 0 and p["launches"]["smooth"] > 0
            assert all(p["ms"][c] == 0 for c in ac.PROF_CLASSES if c != "smooth")
            assert p["launches"]["resid"] > 0 and p["launches"]["coarse"] > 0
            ac.ac_set_profiling(seg.ctx, True)
            seg.step(1)
            p = ac.ac_get_profile(seg.ctx).as_dict()
            assert p["ms"]["smooth"] > 0 and p["ms"]["resid"] > 0 and p["ms"]["coarse"] > 0
        seg.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


# --------------------------------------------------------------------------
# coarse-level tiling: the tiled and the dense forms compute the same numbers
# --------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("W,H,N", [(256, 256, 8), (1024, 1024, 4)])
def test_coarse_tiling_is_bit_identical(ac, precision, W, H, N):
    """The tiled coarse levels (live flags, work lists, zeros written once per
    dying tile) against the dense levels: the same fields bit for bit, also
    when a run switches between the forms every two steps (each switch into
    the tiled form must rewrite every tile)."""
    img = synth.shapes_image(W + N, W, H, rect_side=(8, W // 4), disk_r=(4, W / 8))
    u0 = synth.dirichlet_init(W - N, (W + 1) * (H + 1), N)
    prec = ac.AC_MIXED if precision == "mixed" else ac.AC_FP64
    tol = 1e-6 if precision == "mixed" else 1e-8

    def run(modes):
        seg = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=tol, max_cycles=2000, precision=prec)
        seg.set_image(img)
        seg.set_phase(u0)
        cycles = 0
        for m in modes:
            ac.ac_set_coarse_tiling(seg.ctx, m)
            cycles += seg.step(2).total_cycles
        u = seg.phase()
        seg.close()
        return u, cycles

    NEVER, ALWAYS, AUTO = ac.AC_TILES_NEVER, ac.AC_TILES_ALWAYS, ac.AC_TILES_AUTO
    u_ref, c_ref = run([NEVER] * 4)
    for modes in ([ALWAYS] * 4, [ALWAYS, NEVER, ALWAYS, NEVER], [AUTO] * 4):
        u, c = run(modes)
        assert c == c_ref and np.array_equal(u, u_ref), modes


def test_coarse_tiling_adjoint_is_bit_identical(ac):
    """The adjoint's tangent solve (FP64) runs the same coarse levels: tiled
    and dense give the same gradients bit for bit."""
    import torch
    W, H, N, T, every = 256, 256, 4, 4, 2
    img = synth.shapes_image(91, W, H, rect_side=(8, 64), disk_r=(4, 32)).astype(np.float64)
    u0 = synth.dirichlet_init(92, (W + 1) * (H + 1), N)
    target = synth.voronoi_labels(93, W + 1, H + 1, n_seeds=6, n_labels=N)
    m0 = oracle.moments(img)[:, 0]
    out = []
    for mode in (ac.AC_TILES_NEVER, ac.AC_TILES_ALWAYS):
        seg = _seg(ac, W, H, N, tol=1e-10)
        ac.ac_set_coarse_tiling(seg.ctx, mode)
        seg.set_image(img)
        seg.set_phase(u0)
        ac.ac_adjoint_forward(seg.ctx, T, every)
        _, gT = oracle.misfit_loss(seg.phase(), m0, target)
        g_img = torch.zeros((H, W, 3), dtype=torch.float64, device="cuda")
        gl, ge = ac.ac_adjoint_backward(seg.ctx, torch.tensor(gT, device="cuda"), g_img)
        out.append((gl, ge, g_img.cpu().numpy()))
        seg.close()
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1] and np.array_equal(out[0][2], out[1][2])


# --------------------------------------------------------------------------
# full sizes: properties that hold at any size, checked by the oracle
# --------------------------------------------------------------------------

@pytest.mark.parametrize("name,W,steps,prec,tol", [("c2_1024_n4", 1024, 2, "fp64", 1e-8),
                                                   ("c2_1024_n4", 1024, 2, "mixed", 1e-6),
                                                   ("c3_4096_n8_mixed", 4096, 1, "fp64", 1e-8),
                                                   ("c3_4096_n8_mixed", 4096, 2, "mixed", 1e-6)])
def test_full_size_invariants_and_kkt(ac, name, W, steps, prec, tol):
    """At the benchmark sizes and in the benchmark's launch configuration:
    after each step sum_i u = 1, 0 <= u <= 1, the energy does not increase, and
    the oracle's natural residual of the GPU's u^{t+1} against the oracle's
    b(u^t) is within the step tolerance."""
    cfg = synth.CONFIGS[name]
    H = W
    N, eps, lam, tau = cfg["N"], cfg["eps"], cfg["lam"], cfg["tau"]
    img = synth.config_image(name, 0, W, H)
    precision = ac.AC_MIXED if prec == "mixed" else ac.AC_FP64
    seg = ac.Segmenter(W, H, N, eps, lam, tau, tol=tol, max_cycles=500, seed=1, precision=precision)
    seg.set_image(img)
    img_used = synth.round_bf16(img) if prec == "mixed" else img
    m = oracle.moments(img_used.astype(np.float64))
    u = seg.phase()
    c = np.zeros((N, 3))
    E = oracle.energy(u, m, W, H, eps, lam)
    for _ in range(steps):
        st = seg.step(1)
        assert st.converged
        u1 = seg.phase()
        assert np.abs(u1.sum(1) - 1).max() < 1e-13
        assert u1.min() >= 0 and u1.max() <= 1 + 1e-15
        c, _ = oracle.means(u, m, W, H, c)
        b = oracle.rhs(u, m, c, W, H, eps, lam, tau)
        rho = oracle.natural_residual(u1, b, W, H, eps, tau)
        assert rho <= 2 * tol
        E1 = oracle.energy(u1, m, W, H, eps, lam)
        assert E1 <= E + 1e-6 * abs(E)
        u, E = u1, E1


# --------------------------------------------------------------------------
# error paths
# --------------------------------------------------------------------------

def test_error_paths(ac):
    import ctypes as C
    seg = _seg(ac, 16, 16, 3)
    assert ac.lib.ac_step(seg.ctx, 1, None) == ac.AC_ERR_STATE
    img = np.full((16, 16, 3), 0.5, np.float32)
    img[3, 4, 1] = np.nan
    seg.set_image(img)
    assert ac.lib.ac_step(seg.ctx, 1, None) == ac.AC_ERR_NUMERIC
    seg2 = _seg(ac, 16, 16, 3, tol=1e-300, max_cycles=2)
    seg2.set_image(np.full((16, 16, 3), 0.5, np.float32))
    st = ac.ac_stats()
    assert ac.lib.ac_step(seg2.ctx, 2, C.byref(st)) == ac.AC_ERR_NOT_CONVERGED
    assert st.steps == 2 and st.converged == 0
    u = seg2.phase()
    assert np.abs(u.sum(1) - 1).max() < 1e-14 and u.min() >= 0  # still feasible


# --------------------------------------------------------------------------
# a11: mixed precision (FP32 correction multigrid, FP64 defect correction)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nu1,nu2", [(0, 2), (1, 0), (3, 3)])
def test_smoothing_schedules(ac, precision, nu1, nu2):
    """Other V(nu1, nu2) schedules reach the same step.  nu1 = 0 makes the
    first cycle take the every-node residual; later cycles let the last
    smoothing pass store its colour's mask and residual and the residual
    kernel visit the other colour only."""
    W, H, N = 96, 64, 5
    img = synth.shapes_image(21, W, H, rect_side=(4, 30), disk_r=(3, 12))
    u0 = synth.dirichlet_init(22, (W + 1) * (H + 1), N)
    tol = 1e-12
    prec = ac.AC_MIXED if precision == "mixed" else ac.AC_FP64
    seg = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=tol, max_cycles=3000, precision=prec, nu1=nu1, nu2=nu2)
    seg.set_image(img)
    seg.set_phase(u0)
    st = seg.step(2)
    assert st.converged
    img_used = synth.round_bf16(img).astype(np.float64) if precision == "mixed" else img.astype(np.float64)
    u_ref, _, _ = oracle.run(img_used, u0, 2.0, 1.0, 4.0, 2, tol=TIGHT)
    assert np.abs(seg.phase() - u_ref).max() < 1e-9
    seg.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_composite_matches_oracle(ac, precision):
    """ac_get_composite (Sec. 4.3) against the oracle's composite of the GPU's
    own phase field, with the colour means of that field: float output within
    2 float ulps of values <= 1; the rounded composite uses the same labels as
    ac_segment."""
    W, H, N = 96, 64, 5
    img = synth.shapes_image(31, W, H, rect_side=(4, 30), disk_r=(3, 12))
    prec = ac.AC_MIXED if precision == "mixed" else ac.AC_FP64
    seg = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=1e-8, max_cycles=3000, precision=prec, seed=7)
    seg.set_image(img)
    seg.step(5)
    u = seg.phase()
    img_used = synth.round_bf16(img).astype(np.float64) if precision == "mixed" else img.astype(np.float64)
    c, _ = oracle.means(u, oracle.moments(img_used), W, H, seg.means())
    for rounded in (False, True):
        got = seg.composite(rounded)
        ref = oracle.composite(u, c, W, H, rounded)
        assert np.abs(got - ref).max() <= 2.4e-7
    lab = seg.segment(0)
    assert np.abs(seg.composite(True) - c[lab.astype(int)]).max() <= 1.2e-7
    seg.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("r", [1, 2])
def test_refine_matches_oracle(ac, precision, r):
    """refine = r (Sec. 4.1): the context takes the W x H image and
    eps, lambda, tau in pixel units; the oracle runs the copy-refined image
    (refine_image) with refined_params on the same start.  Phase fields
    within 1e-10 (FP64, both solved to 3e-15) or 1e-7 (mixed, tol 1e-12);
    pixel labels and composites aggregated over each pixel's cells; the
    energy in pixel units."""
    W0, H0, N = 24, 16, 4
    s = 1 << r
    img = synth.shapes_image(41 + r, W0, H0, rect_side=(3, 10), disk_r=(2, 6))
    prec = ac.AC_MIXED if precision == "mixed" else ac.AC_FP64
    tol = TIGHT if precision == "fp64" else 1e-12
    u0 = synth.dirichlet_init(43, (W0 * s + 1) * (H0 * s + 1), N)
    seg = ac.Segmenter(W0, H0, N, 2.0, 1.0, 4.0, tol=tol, max_cycles=3000, precision=prec, refine=r)
    seg.set_image(img)
    seg.set_phase(u0)
    st = seg.step(3)
    assert st.converged
    img_used = synth.round_bf16(img).astype(np.float64) if precision == "mixed" else img.astype(np.float64)
    fine = oracle.refine_image(img_used, r)
    e2, l2, t2 = oracle.refined_params(2.0, 1.0, 4.0, r)
    u_ref, _, _ = oracle.run(fine, u0, e2, l2, t2, 3, tol=TIGHT)
    u = seg.phase()
    assert np.abs(u - u_ref).max() < (1e-10 if precision == "fp64" else 1e-7)
    # pixel labels of the W0 x H0 image: equal except at near ties
    lab = seg.segment(0)
    ref_lab = oracle.pixel_labels(u, W0, H0, r)
    diff = lab != ref_lab
    if diff.any():
        pm = np.sort(oracle._pixel_means(u, W0, H0, r), axis=2)
        assert (pm[..., -1] - pm[..., -2])[diff].max() < 1e-12
    m = oracle.moments(fine)
    c, _ = oracle.means(u, m, W0 * s, H0 * s, seg.means())
    for rounded in (False, True):
        assert np.abs(seg.composite(rounded) - oracle.composite(u, c, W0, H0, rounded, r)).max() <= 2.4e-7
    E = oracle.energy(u, m, W0 * s, H0 * s, e2, l2) * 2.0 ** -r
    assert seg.energy() == pytest.approx(E, rel=1e-12)
    seg.close()


def test_refine_adjoint_matches_oracle(ac):
    """Gradients through T steps on the refined grid, mapped back to the
    pixel-unit lambda (x 2^-r), eps (x 2^r, tau held fixed) and the W x H
    image (sum over each pixel's cells, the adjoint of the copy), against the
    FP64 oracle adjoint of the refined problem: 1e-6 relative."""
    W0, H0, N, r, T, every = 12, 8, 3, 1, 4, 2
    s = 1 << r
    img = synth.shapes_image(51, W0, H0, rect_side=(2, 6), disk_r=(1.5, 4), sigma=0.08).astype(np.float64)
    u0 = synth.dirichlet_init(52, (W0 * s + 1) * (H0 * s + 1), N)
    target = synth.voronoi_labels(53, W0 * s + 1, H0 * s + 1, n_seeds=4, n_labels=N)
    import torch
    seg = ac.Segmenter(W0, H0, N, 2.0, 1.0, 4.0, tol=1e-14, max_cycles=3000, refine=r)
    seg.set_image(img)
    seg.set_phase(u0)
    ac.ac_adjoint_forward(seg.ctx, T, every)
    uT = seg.phase()
    fine = oracle.refine_image(img, r)
    m0 = oracle.moments(fine)[:, 0]
    _, gT = oracle.misfit_loss(uT, m0, target)
    g_img = torch.zeros((H0, W0, 3), dtype=torch.float64, device="cuda")
    g_u0 = torch.zeros((seg.n_nodes, N), dtype=torch.float64, device="cuda")
    gl, ge = ac.ac_adjoint_backward(seg.ctx, torch.tensor(gT, device="cuda"), g_img, g_u0)
    seg.close()
    e2, l2, t2 = oracle.refined_params(2.0, 1.0, 4.0, r)
    states = oracle.forward_states(fine, u0, e2, l2, t2, T)
    rl, re_, rimg, ru0 = oracle.adjoint(fine, states, e2, l2, t2, gT)
    assert gl == pytest.approx(rl * 2.0 ** -r, rel=1e-6)
    assert ge == pytest.approx(re_ * 2.0 ** r, rel=1e-6)
    rimg0 = rimg.reshape(H0, s, W0, s, 3).sum(axis=(1, 3))
    gi = g_img.cpu().numpy()
    assert np.abs(gi - rimg0).max() <= 1e-6 * np.abs(rimg0).max()
    assert np.abs(g_u0.cpu().numpy() - ru0).max() <= 1e-6 * np.abs(ru0).max()


def _mixed(ac, W, H, N, tol, **kw):
    return ac.Segmenter(W, H, N, kw.pop("eps", 2.0), kw.pop("lam", 1.0), kw.pop("tau", 4.0), tol=tol,
                        max_cycles=kw.pop("max_cycles", 2000), precision=ac.AC_MIXED, **kw)


def test_mixed_image_is_bf16(ac):
    img = synth.config_image("c1_64_n4_fp64", 0)
    seg = _mixed(ac, 64, 64, 4, 1e-6)
    seg.set_image(img)
    ref = oracle.moments(synth.round_bf16(img).astype(np.float64))
    got = seg.moments()
    assert (np.abs(got - ref) <= 2e-15 * np.maximum(1.0, np.abs(ref))).all()
    # and it is not the unrounded image's moments
    assert np.abs(got - oracle.moments(img.astype(np.float64))).max() > 1e-6


@pytest.mark.parametrize("tol,bound", [(1e-6, 25e-6), (1e-12, 1e-10)])
def test_mixed_one_step_c1(ac, tol, bound):
    """One step from identical u^t.  The error of a step is at most ~20 times
    its natural residual, so the mixed form must land within 25 tol of the
    oracle, and with a tight tol the FP64 defect correction must reach FP64
    accuracy although every sweep runs in FP32."""
    W = H = 64
    img = synth.config_image("c1_64_n4_fp64", 0)
    u0 = synth.dirichlet_init(1, (W + 1) * (H + 1), 4)
    seg = _mixed(ac, W, H, 4, tol)
    seg.set_image(img)
    seg.set_phase(u0)
    st = seg.step(1)
    assert st.converged and st.residual <= tol and st.outer >= 1
    img16 = synth.round_bf16(img).astype(np.float64)
    u_ref, _, _, _, stt = oracle.step(u0, oracle.moments(img16), np.zeros((4, 3)), W, H, 2.0, 1.0, 4.0, tol=TIGHT,
                                      nu1=2, nu2=2)
    u = seg.phase()
    assert np.abs(u - u_ref).max() < bound
    assert np.abs(u.sum(1) - 1).max() < 1e-14 and u.min() >= 0


def test_mixed_trajectory_c1(ac):
    """20 steps at tol 1e-12: within 1e-7 of the FP64 oracle (per-step error
    ~2e-11, amplified ~1000x by the first steps of a random start); labels
    equal except at near-ties."""
    W = H = 64
    img = synth.config_image("c1_64_n4_fp64", 0)
    u0 = synth.dirichlet_init(1, (W + 1) * (H + 1), 4)
    seg = _mixed(ac, W, H, 4, 1e-12)
    seg.set_image(img)
    seg.set_phase(u0)
    lab = seg.segment(20)
    img16 = synth.round_bf16(img).astype(np.float64)
    u_ref, _, _ = oracle.run(img16, u0, 2.0, 1.0, 4.0, 20, tol=TIGHT, nu1=2, nu2=2)
    u = seg.phase()
    assert np.abs(u - u_ref).max() < 1e-7
    assert np.array_equal(lab, seg.segment(0))
    _check_labels(seg, u, u_ref, W, H, margin=1e-6)


def test_set_phase_restarts_the_correction(ac):
    """The mixed form starts a step's first correction from the previous
    step's; a new state (ac_set_phase) starts it from zero, so a reused
    context and a fresh one give bit-identical fields from the same state."""
    W, H, N = 96, 64, 5
    img = synth.shapes_image(61, W, H, rect_side=(4, 30), disk_r=(3, 12))
    u0 = synth.dirichlet_init(62, (W + 1) * (H + 1), N)
    a = _mixed(ac, W, H, N, 1e-8)
    a.set_image(img)
    a.set_phase(u0)
    a.step(3)
    u3 = a.phase()
    a.set_phase(u3)
    a.step(2)
    b = _mixed(ac, W, H, N, 1e-8)
    b.set_image(img)
    b.set_phase(u3)
    b.step(2)
    assert np.array_equal(a.phase(), b.phase())
    a.close()
    b.close()


@pytest.mark.parametrize("W,H,N", [(37, 23, 3), (2, 1, 4), (48, 40, 2), (96, 64, 8), (40, 24, 6)])
def test_mixed_ragged(ac, W, H, N):
    img = synth.shapes_image(W * 5 + H, W, H, rect_side=(1, max(1, W // 2)), disk_r=(1, max(1.5, W / 4)))
    u0 = synth.dirichlet_init(W * H, (W + 1) * (H + 1), N)
    seg = _mixed(ac, W, H, N, 1e-11)
    seg.set_image(img)
    seg.set_phase(u0)
    seg.step(2)
    u_ref, _, _ = oracle.run(synth.round_bf16(img).astype(np.float64), u0, 2.0, 1.0, 4.0, 2, tol=TIGHT, nu1=2, nu2=2)
    assert np.abs(seg.phase() - u_ref).max() < 1e-9


# --------------------------------------------------------------------------
# data projection by node (Sec. 4.2)
# --------------------------------------------------------------------------

def test_node_projection_moments(ac):
    """The by-node moments (nodal image values by the copy rule, consistent
    mass matrix) against the oracle: the hand-derived 2x1 case, a 64x64
    image through the float and FP64 inputs, a 1-pixel-wide image, and the
    mixed form's bfloat16 image."""
    def close(a, b):
        return (np.abs(a - b) <= 2e-15 * np.maximum(1.0, np.abs(b))).all()

    img = np.zeros((1, 2, 3))
    img[0, 0] = (1.0, 2.0, 0.0)
    img[0, 1] = (4.0, 8.0, 2.0)
    seg = _seg(ac, 2, 1, 2, projection=ac.AC_PROJ_NODE)
    seg.set_image(img)
    assert close(seg.moments(), oracle.moments(img, "node"))
    for (W, H) in [(64, 64), (1, 7), (37, 23)]:
        img = synth.shapes_image(W + 3 * H, W, H, rect_side=(1, max(1, W // 2)), disk_r=(1, max(1.5, W / 4)))
        ref = oracle.moments(img.astype(np.float64), "node")
        for im in (img, img.astype(np.float64)):
            seg = _seg(ac, W, H, 3, projection=ac.AC_PROJ_NODE)
            seg.set_image(im)
            assert close(seg.moments(), ref)
        segm = _mixed(ac, W, H, 3, 1e-6, projection=ac.AC_PROJ_NODE)
        segm.set_image(img)
        assert close(segm.moments(), oracle.moments(synth.round_bf16(img).astype(np.float64), "node"))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("W,H,N,steps", [(64, 64, 4, 20), (96, 64, 5, 3), (256, 256, 8, 1)])
def test_node_projection_steps(ac, precision, W, H, N, steps):
    """Time steps with the by-node fitting terms against the oracle's:
    phase fields to 1e-10 (FP64, both solved to 3e-15) or 1e-7 (mixed at tol
    1e-12, against the oracle on the bfloat16-rounded image), labels bit-exact
    from the GPU's own field and equal to the oracle's except at near-ties.
    256^2 runs the tiled coarse kernels."""
    img = synth.shapes_image(W * 3 + N, W, H, rect_side=(4, W // 3), disk_r=(3, W / 6))
    u0 = synth.dirichlet_init(W + N, (W + 1) * (H + 1), N)
    if precision == "fp64":
        seg = _seg(ac, W, H, N, projection=ac.AC_PROJ_NODE)
        seg.set_image(img.astype(np.float64))
        img_used, bound = img.astype(np.float64), 1e-10
    else:
        seg = _mixed(ac, W, H, N, 1e-12, max_cycles=3000, projection=ac.AC_PROJ_NODE)
        seg.set_image(img)
        img_used, bound = synth.round_bf16(img).astype(np.float64), 1e-7
    seg.set_phase(u0)
    st = seg.step(steps)
    assert st.converged
    u_ref, c_ref, _ = oracle.run(img_used, u0, 2.0, 1.0, 4.0, steps, tol=TIGHT, nu1=2, nu2=2, projection="node")
    u = seg.phase()
    assert np.abs(u - u_ref).max() < bound
    assert np.abs(seg.means() - c_ref).max() < 10 * bound
    _check_labels(seg, u, u_ref, W, H, margin=max(1e-8, 10 * bound))
    seg.close()


def test_node_projection_refined(ac):
    """Projection by node on the pixel grid refined once (Sec. 4.1): the
    nodes of the refined grid copy the cells, which copy the pixels."""
    W0, H0, N, r = 24, 16, 4, 1
    s_ = 1 << r
    img = synth.shapes_image(71, W0, H0, rect_side=(3, 10), disk_r=(2, 6)).astype(np.float64)
    u0 = synth.dirichlet_init(72, (W0 * s_ + 1) * (H0 * s_ + 1), N)
    seg = _seg(ac, W0, H0, N, refine=r, projection=ac.AC_PROJ_NODE)
    seg.set_image(img)
    seg.set_phase(u0)
    seg.step(3)
    fine = oracle.refine_image(img, r)
    assert np.abs(seg.moments() - oracle.moments(fine, "node")).max() < 1e-14
    e2, l2, t2 = oracle.refined_params(2.0, 1.0, 4.0, r)
    u_ref, _, _ = oracle.run(fine, u0, e2, l2, t2, 3, tol=TIGHT, projection="node")
    assert np.abs(seg.phase() - u_ref).max() < 1e-10
    seg.close()


@pytest.mark.parametrize("r", [0, 1])
def test_node_projection_adjoint(ac, r):
    """Gradients through T steps with the by-node fitting terms against the
    FP64 oracle adjoint of the same projection: 1e-6 relative (the image
    gradient goes through the copy rule and the consistent mass matrix)."""
    import torch
    W0, H0, N, T, every = (20, 14, 3, 5, 2) if r == 0 else (12, 8, 3, 4, 2)
    s_ = 1 << r
    img = synth.shapes_image(81 + r, W0, H0, rect_side=(2, 6), disk_r=(1.5, 4), sigma=0.08).astype(np.float64)
    u0 = synth.dirichlet_init(82, (W0 * s_ + 1) * (H0 * s_ + 1), N)
    target = synth.voronoi_labels(83, W0 * s_ + 1, H0 * s_ + 1, n_seeds=4, n_labels=N)
    seg = _seg(ac, W0, H0, N, tol=1e-14, refine=r, projection=ac.AC_PROJ_NODE)
    seg.set_image(img)
    seg.set_phase(u0)
    ac.ac_adjoint_forward(seg.ctx, T, every)
    uT = seg.phase()
    fine = oracle.refine_image(img, r)
    m0 = oracle.moments(fine)[:, 0]
    _, gT = oracle.misfit_loss(uT, m0, target)
    g_img = torch.zeros((H0, W0, 3), dtype=torch.float64, device="cuda")
    gl, ge = ac.ac_adjoint_backward(seg.ctx, torch.tensor(gT, device="cuda"), g_img)
    seg.close()
    e2, l2, t2 = oracle.refined_params(2.0, 1.0, 4.0, r)
    states = oracle.forward_states(fine, u0, e2, l2, t2, T, projection="node")
    rl, re_, rimg, _ = oracle.adjoint(fine, states, e2, l2, t2, gT, projection="node")
    assert gl == pytest.approx(rl * 2.0 ** -r, rel=1e-6)
    assert ge == pytest.approx(re_ * 2.0 ** r, rel=1e-6)
    rimg0 = rimg.reshape(H0, s_, W0, s_, 3).sum(axis=(1, 3))
    assert np.abs(g_img.cpu().numpy() - rimg0).max() <= 1e-6 * np.abs(rimg0).max()


# --------------------------------------------------------------------------
# a12: batches of uneven images
# --------------------------------------------------------------------------

def _batch_specs():
    return [dict(W=64, H=64, N=4), dict(W=37, H=23, N=3), dict(W=96, H=64, N=6), dict(W=48, H=40, N=2),
            dict(W=128, H=128, N=4), dict(W=64, H=32, N=8), dict(W=40, H=24, N=6)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_single_images(ac, precision):
    """Every image of a batch (uneven sizes and phase counts, 3 streams) ends
    bit-identical to the same image solved alone."""
    specs = _batch_specs()
    prec = ac.AC_MIXED if precision == "mixed" else ac.AC_FP64
    for sp in specs:
        sp.update(tol=1e-9, precision=prec)
    imgs = [synth.shapes_image(7 + k, sp["W"], sp["H"], rect_side=(2, max(2, sp["W"] // 3)),
                               disk_r=(1, max(1.5, sp["W"] / 5))) for k, sp in enumerate(specs)]
    u0s = [synth.dirichlet_init(50 + k, (sp["W"] + 1) * (sp["H"] + 1), sp["N"]) for k, sp in enumerate(specs)]
    b = ac.Batch(specs, n_streams=3)
    for k in range(len(specs)):
        b.set_image(k, imgs[k])
        b.set_phase(k, u0s[k])
    st = b.step(3)
    assert st.images == len(specs) and st.converged_images == len(specs)
    for k, sp in enumerate(specs):
        seg = ac.Segmenter(sp["W"], sp["H"], sp["N"], 2.0, 1.0, 4.0, tol=1e-9, precision=prec)
        seg.set_image(imgs[k])
        seg.set_phase(u0s[k])
        seg.step(3)
        assert np.array_equal(b.phase(k), seg.phase()), f"image {k}"
        assert np.array_equal(b.labels(k), seg.segment(0))
        seg.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_one_graph_matches_single_images(ac, precision):
    """AC_BATCH_ONE_GRAPH: one graph launch per time step runs every image's
    step with its cycle loop on the device.  Every image ends bit-identical to
    the same image solved alone with the host loop, over two calls (the second
    replays the captured graph and carries the warm start), after a retune
    (the graph is captured again), and the statistics agree with the stream
    pool's."""
    specs = _batch_specs()
    prec = ac.AC_MIXED if precision == "mixed" else ac.AC_FP64
    for sp in specs:
        sp.update(tol=1e-9, precision=prec)
    imgs = [synth.shapes_image(7 + k, sp["W"], sp["H"], rect_side=(2, max(2, sp["W"] // 3)),
                               disk_r=(1, max(1.5, sp["W"] / 5))) for k, sp in enumerate(specs)]
    u0s = [synth.dirichlet_init(50 + k, (sp["W"] + 1) * (sp["H"] + 1), sp["N"]) for k, sp in enumerate(specs)]
    runs = {}
    for mode, loop in [("pool_host", ac.AC_LOOP_HOST), ("pool_dev", ac.AC_LOOP_AUTO), ("graph", ac.AC_LOOP_AUTO)]:
        b = ac.Batch(specs, n_streams=3)
        b.set_cycle_loop(loop)
        if mode == "graph":
            b.set_launch(ac.AC_BATCH_ONE_GRAPH)
        for k in range(len(specs)):
            b.set_image(k, imgs[k])
            b.set_phase(k, u0s[k])
        s1 = b.step(2).as_dict()
        s2 = b.step(1).as_dict()
        runs[mode] = ([b.phase(k) for k in range(len(specs))], s1, s2)
        if mode == "graph":
            b.tune(trial_steps=1)
            assert b.step(1).converged_images == len(specs)
        b.close()
    for k, sp in enumerate(specs):
        seg = ac.Segmenter(sp["W"], sp["H"], sp["N"], 2.0, 1.0, 4.0, tol=1e-9, precision=prec)
        seg.set_image(imgs[k])
        seg.set_phase(u0s[k])
        seg.step(2)
        seg.step(1)
        for mode in runs:
            assert np.array_equal(runs[mode][0][k], seg.phase()), f"{mode}, image {k}"
        seg.close()
    assert runs["graph"][1] == runs["pool_host"][1] == runs["pool_dev"][1]
    assert runs["graph"][2] == runs["pool_host"][2] == runs["pool_dev"][2]
    assert runs["graph"][1]["converged_images"] == len(specs)


def test_batch_one_graph_rejects_tiled_images(ac):
    """A 2048 x 1024, N = 8 image has a first coarse level large enough for
    tiles, so its loop stays on the host and the one-graph launch refuses the
    batch with AC_ERR_STATE; the stream pool still runs it."""
    specs = [dict(W=64, H=64, N=4, tol=1e-6, precision=ac.AC_MIXED),
             dict(W=2048, H=1024, N=8, tol=1e-6, precision=ac.AC_MIXED)]
    b = ac.Batch(specs, n_streams=2)
    for k, sp in enumerate(specs):
        b.set_image(k, synth.shapes_image(k, sp["W"], sp["H"]))
    b.set_launch(ac.AC_BATCH_ONE_GRAPH)
    with pytest.raises(ac.AcError) as e:
        b.step(1)
    assert "-5" in str(e.value)
    b.set_launch(ac.AC_BATCH_STREAMS)
    assert b.step(1).converged_images == 2
    b.close()


def test_batch_autotuner(ac):
    """The autotuner picks a valid schedule per group; the tuned batch still
    solves every step to tol (checked by the oracle's natural residual)."""
    specs = _batch_specs()[:4]
    for sp in specs:
        sp.update(tol=1e-8, precision=ac.AC_MIXED)
    imgs = [synth.shapes_image(3 + k, sp["W"], sp["H"], rect_side=(2, max(2, sp["W"] // 3)),
                               disk_r=(1, max(1.5, sp["W"] / 5))) for k, sp in enumerate(specs)]
    b = ac.Batch(specs, n_streams=2)
    for k in range(len(specs)):
        b.set_image(k, imgs[k])
    u_before = [b.phase(k) for k in range(len(specs))]
    chosen = b.tune(trial_steps=2)
    for k in range(len(specs)):  # tuning restores the state
        assert np.array_equal(b.phase(k), u_before[k])
    assert ((chosen[:, 0] >= 1) & (chosen[:, 0] <= 2) & (chosen[:, 1] >= 1) & (chosen[:, 1] <= 2)).all()
    assert (chosen[:, 2] >= 1).all()
    assert np.isin(chosen[:, 3], [ac.AC_SMOOTH_GS3, ac.AC_SMOOTH_JACOBI]).all()
    assert b.step(1).converged_images == len(specs)
    u_prev = [b.phase(k) for k in range(len(specs))]
    assert b.step(1).converged_images == len(specs)
    for k, sp in enumerate(specs):
        W, H = sp["W"], sp["H"]
        m = oracle.moments(synth.round_bf16(imgs[k]).astype(np.float64))
        u1 = b.phase(k)
        assert np.abs(u1.sum(1) - 1).max() < 1e-13 and u1.min() >= 0
        c, _ = oracle.means(u_prev[k], m, W, H)
        rhs = oracle.rhs(u_prev[k], m, c, W, H, 2.0, 1.0, 4.0)
        assert oracle.natural_residual(u1, rhs, W, H, 2.0, 4.0) <= 2e-8
    b.close()


# --------------------------------------------------------------------------
# a13: adjoint
# --------------------------------------------------------------------------

def _adj_problem(seed, W, H, N, n_disk=3):
    img = synth.shapes_image(seed, W, H, n_rect=1, n_disk=n_disk, rect_side=(2, max(2, W // 3)),
                             disk_r=(1.5, max(2.0, W / 5)), sigma=0.08).astype(np.float64)
    u0 = synth.dirichlet_init(seed + 1, (W + 1) * (H + 1), N)
    target = synth.voronoi_labels(seed + 2, W + 1, H + 1, n_seeds=6, n_labels=N)
    return img, u0, target


def _gpu_grads(ac, img, u0, target, eps, lam, tau, T, every, tol, precision):
    import torch
    from paper_0710_0736_gb300.adjoint import SegmentationSteps, misfit_loss
    image = torch.tensor(img, device="cuda", requires_grad=True)
    lam_t = torch.tensor(lam, dtype=torch.float64, device="cuda", requires_grad=True)
    eps_t = torch.tensor(eps, dtype=torch.float64, device="cuda", requires_grad=True)
    u0_t = torch.tensor(u0, device="cuda", requires_grad=True)
    uT = SegmentationSteps.apply(image, lam_t, eps_t, u0_t, tau, T, every, tol, precision)
    m0 = torch.tensor(oracle.moments(img)[:, 0], device="cuda")
    L = misfit_loss(uT, m0, torch.tensor(target, device="cuda"))
    L.backward()
    return (float(L.detach()), float(lam_t.grad), float(eps_t.grad), image.grad.cpu().numpy(), u0_t.grad.cpu().numpy())


def _gpu_loss(ac, img, u0, target, eps, lam, tau, T, tol, precision):
    H, W, _ = img.shape
    seg = ac.Segmenter(W, H, u0.shape[1], eps, lam, tau, tol=tol, precision=precision, max_cycles=2000)
    seg.set_image(img.astype(np.float32) if precision == ac.AC_MIXED else img)
    seg.set_phase(u0)
    seg.step(T)
    L, _ = oracle.misfit_loss(seg.phase(), oracle.moments(img)[:, 0], target)
    seg.close()
    return L


def test_adjoint_matches_oracle_gradient(ac):
    """FP64 forward and adjoint on the GPU against the FP64 oracle adjoint (on
    the oracle's own forward states): 1e-6 relative."""
    W, H, N, T, every = 24, 16, 3, 6, 2
    eps, lam, tau = 2.0, 1.0, 4.0
    img, u0, target = _adj_problem(0, W, H, N)
    L, gl, ge, gimg, gu0 = _gpu_grads(ac, img, u0, target, eps, lam, tau, T, every, 1e-14, ac.AC_FP64)
    states = oracle.forward_states(img, u0, eps, lam, tau, T)
    m0 = oracle.moments(img)[:, 0]
    L_ref, gT = oracle.misfit_loss(states[-1], m0, target)
    rl, re_, rimg, ru0 = oracle.adjoint(img, states, eps, lam, tau, gT)
    assert L == pytest.approx(L_ref, rel=1e-9)
    assert gl == pytest.approx(rl, rel=1e-6, abs=1e-9)
    assert ge == pytest.approx(re_, rel=1e-6, abs=1e-9)
    assert np.abs(gimg - rimg).max() <= 1e-6 * np.abs(rimg).max()
    assert np.abs(gu0 - ru0).max() <= 1e-6 * np.abs(ru0).max()


def test_adjoint_matches_finite_differences(ac):
    """Central differences (h = 1e-6) of the GPU forward itself, solved to
    1e-14: lambda, eps, two image directions and one u0 direction."""
    W, H, N, T, every = 32, 24, 4, 8, 3
    eps, lam, tau, tol, prec = 2.0, 1.0, 4.0, 1e-14, ac.AC_FP64
    img, u0, target = _adj_problem(1, W, H, N)
    L, gl, ge, gimg, gu0 = _gpu_grads(ac, img, u0, target, eps, lam, tau, T, every, tol, prec)
    h = 1e-6

    def fd(f):
        return (f(h) - f(-h)) / (2 * h)

    assert gl == pytest.approx(fd(lambda d: _gpu_loss(ac, img, u0, target, eps, lam + d, tau, T, tol, prec)),
                               rel=1e-6, abs=1e-9)
    assert ge == pytest.approx(fd(lambda d: _gpu_loss(ac, img, u0, target, eps + d, lam, tau, T, tol, prec)),
                               rel=1e-6, abs=1e-9)
    rng = np.random.default_rng(2)
    for _ in range(2):
        v = rng.normal(size=img.shape)
        assert (gimg * v).sum() == pytest.approx(
            fd(lambda d: _gpu_loss(ac, img + d * v, u0, target, eps, lam, tau, T, tol, prec)), rel=1e-6)
    z = rng.normal(size=u0.shape)
    z -= z.mean(1, keepdims=True)
    assert (gu0 * z).sum() == pytest.approx(
        fd(lambda d: _gpu_loss(ac, img, u0 + d * z, target, eps, lam, tau, T, tol, prec)), rel=1e-6, abs=1e-9)


def test_adjoint_mixed_forward(ac):
    """The mixed-precision forward (FP32 sweeps, FP64 defect correction to
    1e-12) with the FP64 adjoint, against the FP64 oracle gradient on the
    same bfloat16-rounded image: relative 1e-6."""
    W, H, N, T, every = 32, 24, 4, 8, 3
    eps, lam, tau = 2.0, 1.0, 4.0
    img, u0, target = _adj_problem(1, W, H, N)
    img = synth.round_bf16(img.astype(np.float32)).astype(np.float64)
    L, gl, ge, gimg, gu0 = _gpu_grads(ac, img, u0, target, eps, lam, tau, T, every, 1e-12, ac.AC_MIXED)
    states = oracle.forward_states(img, u0, eps, lam, tau, T)
    L_ref, gT = oracle.misfit_loss(states[-1], oracle.moments(img)[:, 0], target)
    rl, re_, rimg, ru0 = oracle.adjoint(img, states, eps, lam, tau, gT)
    assert L == pytest.approx(L_ref, rel=1e-9)
    assert gl == pytest.approx(rl, rel=1e-6)
    assert ge == pytest.approx(re_, rel=1e-6)
    assert np.abs(gimg - rimg).max() <= 1e-6 * np.abs(rimg).max()
    assert np.abs(gu0 - ru0).max() <= 1e-6 * np.abs(ru0).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_recomputation_repeats_the_forward(ac, precision):
    """Checkpointing: ac_adjoint_forward's u^T equals plain steps restarted
    at every checkpoint (each segment starts its first correction from zero),
    and every segment that ac_adjoint_backward recomputes ends bit for bit on
    the forward's own state (ac_adjoint_recompute_diff = 0)."""
    import torch
    W, H, N, T, every = 48, 32, 4, 7, 3
    img, u0, target = _adj_problem(3, W, H, N)
    prec = ac.AC_MIXED if precision == "mixed" else ac.AC_FP64
    tol = 1e-10
    seg = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=tol, max_cycles=2000, precision=prec)
    seg.set_image(img.astype(np.float32))
    seg.set_phase(u0)
    ac.ac_adjoint_forward(seg.ctx, T, every)
    uT = seg.phase()
    ref = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=tol, max_cycles=2000, precision=prec)
    ref.set_image(img.astype(np.float32))
    ref.set_phase(u0)
    for t0 in range(0, T, every):
        ref.set_phase(ref.phase())
        ref.step(min(every, T - t0))
    assert np.array_equal(ref.phase(), uT)
    ref.close()
    m0 = oracle.moments(img)[:, 0]
    _, gT = oracle.misfit_loss(uT, m0, target)
    g_img = torch.zeros((H, W, 3), dtype=torch.float64, device="cuda")
    ac.ac_adjoint_backward(seg.ctx, torch.tensor(gT, device="cuda"), g_img)
    assert ac.ac_adjoint_recompute_diff(seg.ctx) == 0
    assert np.array_equal(seg.phase(), uT)
    seg.close()


@pytest.mark.parametrize("stream", ["legacy", "side"])
def test_adjoint_preconditioners_agree(ac, stream):
    """The adjoint's flexible CG preconditioned by FP32 V-cycles (the default)
    and by FP64 ones reach the same tangent solutions (both stop at 1e-13 of
    max |Pi g|): gradients to 1e-9 relative, on the legacy stream (direct
    launches) and on a stream of its own (graphs)."""
    import torch
    W, H, N, T, every = 48, 32, 4, 6, 3
    img, u0, target = _adj_problem(4, W, H, N)
    m0 = oracle.moments(img)[:, 0]
    side = torch.cuda.Stream()
    out = {}
    for pre in (ac.AC_ADJ_PRECOND_F32, ac.AC_ADJ_PRECOND_F64):
        kw = {"stream": side.cuda_stream} if stream == "side" else {"stream": None}
        seg = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=1e-12, max_cycles=2000, **kw)
        ac.ac_set_adjoint_preconditioner(seg.ctx, pre)
        seg.set_image(img)
        seg.set_phase(u0)
        ac.ac_adjoint_forward(seg.ctx, T, every)
        _, gT = oracle.misfit_loss(seg.phase(), m0, target)
        g_img = torch.zeros((H, W, 3), dtype=torch.float64, device="cuda")
        g_u = torch.tensor(gT, device="cuda")
        torch.cuda.synchronize()  # torch's stream and the library's are not ordered with "side"
        gl, ge = ac.ac_adjoint_backward(seg.ctx, g_u, g_img)
        torch.cuda.synchronize()
        assert ac.ac_adjoint_recompute_diff(seg.ctx) == 0
        out[pre] = (gl, ge, g_img.cpu().numpy())
        seg.close()
    (l32, e32, i32), (l64, e64, i64) = out[ac.AC_ADJ_PRECOND_F32], out[ac.AC_ADJ_PRECOND_F64]
    assert l32 == pytest.approx(l64, rel=1e-9) and e32 == pytest.approx(e64, rel=1e-9)
    assert np.abs(i32 - i64).max() <= 1e-9 * np.abs(i64).max()
    with pytest.raises(ac.AcError):
        ac.ac_set_adjoint_preconditioner(None, ac.AC_ADJ_PRECOND_F32)


@pytest.fixture(scope="module")
def c5_problem(ac):
    """The 512x512, N = 4 workload (12 disks, noise 0.08, Voronoi target of 6
    seeds) over 16 steps with checkpoints every 4, every step solved to 1e-14,
    and its GPU gradients."""
    W = H = 512
    cfg = synth.CONFIGS["c5_512_n4_adjoint"]
    N, eps, lam, tau, T = cfg["N"], cfg["eps"], cfg["lam"], cfg["tau"], 16
    img = synth.config_image("c5_512_n4_adjoint", 0).astype(np.float64)
    u0 = synth.dirichlet_init(1, (W + 1) * (H + 1), N)
    target = synth.voronoi_labels(2, W + 1, H + 1, n_seeds=6, n_labels=4)
    tol = 1e-14
    grads = _gpu_grads(ac, img, u0, target, eps, lam, tau, T, 4, tol, ac.AC_FP64)
    return dict(img=img, u0=u0, target=target, eps=eps, lam=lam, tau=tau, T=T, tol=tol, grads=grads)


def test_adjoint_full_size_c5(ac, c5_problem):
    """lambda, eps and 8 random image directions against central differences
    (h = 1e-7) of the GPU forward.

    Rounding noise of the forward, amplified by the first steps of a random
    start, leaves ~5e-11 of noise in L, i.e. ~2.5e-4 in a difference quotient
    at h = 1e-7; larger h meets kinks (active-set changes; h = 1e-6 is off by
    1e-5 relative).  lambda and eps are held to 1e-6 relative, the random image
    directions (derivatives ~300-3000) to 1e-6 relative or 1e-3 absolute, that
    noise floor, whichever is larger.  (A
    direction aligned with the gradient's signs moves every interface at once
    and meets kinks within +-h: its quotient is off by ~1e-3 relative.)  Over
    the full 64 steps the quotients wander by ~0.5% with h."""
    P = c5_problem
    img, u0, target, eps, lam, tau, T, tol = (P[k] for k in ("img", "u0", "target", "eps", "lam", "tau", "T", "tol"))
    L, gl, ge, gimg, gu0 = P["grads"]
    h = 1e-7

    def fd(f):
        return (f(h) - f(-h)) / (2 * h)

    assert gl == pytest.approx(fd(lambda d: _gpu_loss(ac, img, u0, target, eps, lam + d, tau, T, tol, ac.AC_FP64)),
                               rel=1e-6)
    assert ge == pytest.approx(fd(lambda d: _gpu_loss(ac, img, u0, target, eps + d, lam, tau, T, tol, ac.AC_FP64)),
                               rel=1e-6)
    rng = np.random.default_rng(3)
    for _ in range(8):
        v = rng.normal(size=img.shape)
        assert (gimg * v).sum() == pytest.approx(
            fd(lambda d: _gpu_loss(ac, img + d * v, u0, target, eps, lam, tau, T, tol, ac.AC_FP64)), rel=1e-6, abs=1e-3)


def test_adjoint_full_size_c5_pixels(ac, c5_problem):
    """64 random pixel-channels of dL/dI against central differences at
    h = 1e-4.  A single pixel moves its own neighbourhood only, so kinks are
    rare there and the quotient's truncation and noise stay near 1e-6 (24
    channels measured: at most 1.2e-6 off, entries up to 33); at h = 1e-6
    rounding noise dominates (~1e-4).  Bound: 1e-6 |g| + 4e-6."""
    P = c5_problem
    img, u0, target, eps, lam, tau, T, tol = (P[k] for k in ("img", "u0", "target", "eps", "lam", "tau", "T", "tol"))
    gimg = P["grads"][3]
    H, W, _ = img.shape
    rng = np.random.default_rng(5)
    h = 1e-4
    for _ in range(64):
        py, px, ch = int(rng.integers(H)), int(rng.integers(W)), int(rng.integers(3))
        e = np.zeros_like(img)
        e[py, px, ch] = 1.0
        q = (_gpu_loss(ac, img + h * e, u0, target, eps, lam, tau, T, tol, ac.AC_FP64) -
             _gpu_loss(ac, img - h * e, u0, target, eps, lam, tau, T, tol, ac.AC_FP64)) / (2 * h)
        g = gimg[py, px, ch]
        assert abs(q - g) <= 1e-6 * abs(g) + 4e-6, (py, px, ch, g, q)
