"""ac_colour_means_static: colour means for callers that cannot allocate.

Real-time pipelines that forbid device allocation once running, and code under
a framework's fixed device-memory budget, cannot let a library call
cudaMalloc.  This entry point keeps its reduction scratch in a file-scope
__device__ array instead.  Its output must match the colour means that the
ordinary path (ac_step, then ac_get_means) computes, and the CPU oracle's
colour means, on two calls in a row (the second call reuses the scratch the
first one left behind).  Kept in a
file that is collected last.
"""
import numpy as np
import pytest

from paper_0710_0736_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ac():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0710_0736_gb300 import build
    build.build()
    from paper_0710_0736_gb300 import ac as mod
    return mod


@pytest.mark.parametrize("W,H,N,empty", [(64, 48, 4, None), (37, 23, 8, None), (300, 200, 3, None),
                                         (96, 64, 5, 2), (512, 512, 8, None)])
def test_static_means_match_allocating_path(ac, W, H, N, empty):
    """(96, 64, 5) has phase 2 at zero everywhere: a phase of zero mass gets
    c_i = 0 on both paths.  512 x 512 (263 169 nodes) needs more than the
    scratch's 512 blocks of 256 threads, so each block sums several strides."""
    import torch
    import oracle
    img = synth.shapes_image(W + H, W, H, rect_side=(2, max(2, W // 3)), disk_r=(1, max(1.5, W / 5)))
    u0 = synth.dirichlet_init(W * H, (W + 1) * (H + 1), N)
    if empty is not None:
        u0[:, empty] = 0.0
        u0 /= u0.sum(1, keepdims=True)
    # the colour means by their definition (Sec. 4.4), from the CPU oracle
    c_def, mass = oracle.means(u0, oracle.moments(img.astype(np.float64)), W, H, np.zeros((N, 3)))
    if empty is not None:
        assert mass[empty] == 0 and not c_def[empty].any()
    # the ordinary path: c^t of u0 is what the first step uses
    seg = ac.Segmenter(W, H, N, 2.0, 1.0, 4.0, tol=1e-8)
    seg.set_image(img)
    seg.set_phase(u0)
    seg.step(1)
    c_ref = seg.means()
    seg.close()
    u = torch.tensor(u0, device="cuda")
    rgb = torch.tensor(img, device="cuda")
    for _ in range(2):
        c = torch.full((N, 3), float("nan"), dtype=torch.float64, device="cuda")
        ac.ac_colour_means_static(u, rgb, W, H, N, c)
        torch.cuda.synchronize()
        got = c.cpu().numpy()
        assert np.abs(got - c_ref).max() < 1e-14
        assert np.abs(got - c_def).max() < 1e-13
        if empty is not None:
            assert not got[empty].any()


def test_static_means_rejects_beyond_limit(ac):
    import torch
    u = torch.zeros(9 * 9 * 9, dtype=torch.float64, device="cuda")
    rgb = torch.zeros(8 * 8 * 3, dtype=torch.float32, device="cuda")
    c = torch.zeros(9 * 3, dtype=torch.float64, device="cuda")
    rc = ac.lib.ac_colour_means_static(u.data_ptr(), rgb.data_ptr(), 8, 8, 9, c.data_ptr(), None)
    assert rc == ac.AC_ERR_ARG and "n_phases" in ac.ac_last_error()
