"""Union over non-binary material levels (App. B, Alg. 1) through the C ABI
(adg_levels_eps, adg_levels_grad) against the FP64 oracle (oracle/levels.py).

eps: every sample within 2e-6 K eps^K + 1e-6 |eps| -- each set's fill is
within 1e-6 of the oracle's and Alg. 1's result moves by at most eps^K per
unit change of one set's fill.  g: 1e-4 ||g||_2 + 1e-5 ||g||_inf.  Cases
cover both logic families, 2D and 3D, the 16-byte path (component plane a
multiple of 4) and the scalar path (an odd plane), K = 1 and K = 8."""
import numpy as np
import pytest

from paper_2311_05646_gb300 import inputs as I

from . import _gpu as H
from .conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

CASES = {
    "2d_product": dict(n=(200, 200, 1), d=(20.0, 20.0, 20.0), logic="product"),
    "2d_clamp": dict(n=(200, 200, 1), d=(20.0, 20.0, 20.0), logic="clamp"),
    "3d_product_odd": dict(n=(97, 45, 19), d=(40.0, 40.0, 40.0), logic="product",
                           levels=(0.5, 1.3, 2.0), eps_bg=2.085),
    "3d_clamp_vec": dict(n=(128, 64, 24), d=(30.0, 30.0, 30.0), logic="clamp", per_level=4),
    "one_level": dict(n=(150, 120, 1), d=(20.0, 20.0, 20.0), levels=(0.9,), eps_bg=1.0),
    "eight_levels": dict(n=(160, 150, 1), d=(20.0, 20.0, 20.0), per_level=2,
                         levels=(0.1, 0.2, 0.3, 0.45, 0.6, 0.62, 0.8, 1.0)),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_2311_05646_gb300 import adg
    return adg.Context(0)


def _run(ctx, m, ef, ea, w):
    import torch
    from paper_2311_05646_gb300 import adg
    sets = [adg.Design(ctx, d) for d in m["sets"]]
    p = m["sets"][0]["params"]
    eps = torch.full(sets[0].shape, float("nan"), dtype=torch.float32, device="cuda")
    adg.adg_levels_eps(sets, m["levels"], m["eps_bg"], p, eps)
    g = torch.full((sets[0].n_params,), float("nan"), dtype=torch.float32, device="cuda")
    adg.adg_levels_grad(sets, m["levels"], p, torch.from_numpy(ef).cuda(),
                        torch.from_numpy(ea).cuda(), w, g)
    adg.adg_sync(ctx)
    return sets, eps.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", sorted(CASES))
def test_levels_match_oracle(ctx, case):
    from oracle import levels as LV
    m = I.nonbinary_circles(**CASES[case])
    s0 = m["sets"][0]
    ef, ea, w = I.plane_wave_field(s0, 81), I.plane_wave_field(s0, 82), I.seeded_w(
        s0["grid"]["ncomp"], 83)
    _, eps, g = _run(ctx, m, ef, ea, w)
    want = LV.eps(m["sets"], m["levels"], m["eps_bg"])
    K, top = len(m["sets"]), float(m["levels"][-1])
    tol = 2e-6 * K * top + 1e-6 * np.abs(want)
    bad = np.abs(eps - want) > tol
    assert not bad.any(), (int(bad.sum()), float(np.abs(eps - want).max()))
    gref = LV.grad(m["sets"], m["levels"], ef, ea, w)
    ok, err, bound = H.grad_ok(g, gref)
    assert ok, (err, bound)


def test_levels_are_deterministic_and_reuse_scratch(ctx):
    """Two calls agree bit for bit; a smaller call after a larger one reuses
    the first set's scratch."""
    m = I.nonbinary_circles(n=(128, 64, 24), d=(30.0, 30.0, 30.0), logic="product")
    s0 = m["sets"][0]
    ef, ea, w = I.plane_wave_field(s0, 1), I.plane_wave_field(s0, 2), I.seeded_w(3, 3)
    sets, e1, g1 = _run(ctx, m, ef, ea, w)
    _, e2, g2 = _run(ctx, m, ef, ea, w)
    assert np.array_equal(e1, e2) and np.array_equal(g1, g2)


def test_levels_reject_bad_inputs(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    m = I.nonbinary_circles(n=(64, 48, 1), d=(20.0, 20.0, 20.0))
    sets = [adg.Design(ctx, d) for d in m["sets"]]
    p = m["sets"][0]["params"]
    eps = torch.zeros(sets[0].shape, dtype=torch.float32, device="cuda")
    with pytest.raises(adg.AdgError):  # unsorted levels
        adg.adg_levels_eps(sets, m["levels"][::-1].copy(), 0.0, p, eps)
    with pytest.raises(adg.AdgError):  # a level of zero
        adg.adg_levels_eps(sets, np.r_[0.0, m["levels"][1:]], 0.0, p, eps)
    bad = dict(m["sets"][1])
    bad["eps_fg"] = 2.0  # material slots must be 0 / 1
    with pytest.raises(adg.AdgError):
        adg.adg_levels_eps([sets[0], adg.Design(ctx, bad)], m["levels"][:2], 0.0, p, eps)
    other = I.nonbinary_circles(n=(64, 48, 1), d=(20.0, 20.0, 20.0), per_level=1)
    with pytest.raises(adg.AdgError):  # different parameter vectors
        adg.adg_levels_eps([sets[0], adg.Design(ctx, other["sets"][1])], m["levels"][:2], 0.0,
                           p, eps)
    nine = I.nonbinary_circles(n=(64, 48, 1), d=(20.0, 20.0, 20.0), per_level=1,
                               levels=tuple(0.1 * (k + 1) for k in range(9)))
    with pytest.raises(adg.AdgError):  # more than 8 sets
        adg.adg_levels_eps([adg.Design(ctx, d) for d in nine["sets"]], nine["levels"], 0.0,
                           nine["sets"][0]["params"], eps)
