"""The finite-difference baseline on the GPU (adg_grad_fd: two builds per
parameter and a fixed-order dot product) against the FP64 oracle's own
central differences at the same step, and against the AutoDiff gradient
(adg_grad), which it approximates to O(h^2) -- exactly for exact-overlap box
edges whose +-h stays inside one cell."""
import numpy as np
import pytest

from paper_2311_05646_gb300 import inputs as I

from . import _gpu as H
from .conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def ctx():
    from paper_2311_05646_gb300 import adg
    return adg.Context(0)


def _fd(ctx, desc, ef, ea, w, h):
    import torch
    from paper_2311_05646_gb300 import adg
    d = adg.Design(ctx, desc)
    g = torch.zeros(d.n_params, dtype=torch.float32, device="cuda")
    adg.adg_grad_fd(d, desc["params"], torch.from_numpy(ef).cuda(), torch.from_numpy(ea).cuda(), w,
                    h, g)
    adg.adg_sync(ctx)
    return d, g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", ["grating2d", "grating3d_small", "holes_2d"])
def test_fd_matches_oracle_fd_and_ad(ctx, oracle_mod, case):
    desc = {"grating2d": lambda: I.grating_2d("fit"),
            "grating3d_small": lambda: I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0),
            "holes_2d": lambda: I.hole_lattice(n=(96, 80, 1), d=(40.0, 40.0, 40.0), holes=4,
                                               ncomp=1)}[case]()
    ef, ea = I.plane_wave_field(desc, 31), I.plane_wave_field(desc, 32)
    w = I.seeded_w(desc["grid"]["ncomp"], 33)
    h = 0.5  # nm: fill in fp32 resolves the differences; the step stays inside a cell
    d, g = _fd(ctx, desc, ef, ea, w, h)
    gref = oracle_mod.grad_fd(desc, ef, ea, w, h)
    # fp32 fills differenced: the error scales with |Re(w E E)| |deps| eps32 / h per cell
    ok, err, bound = H.grad_ok(g, gref)
    assert err <= 10 * bound, (err, bound)
    g_ad = H.run_grad(d, desc, ef, ea, w)
    assert np.linalg.norm(g - g_ad) <= 1e-2 * np.linalg.norm(g_ad) + 1e-3 * np.abs(g_ad).max()


def test_fd_is_deterministic_and_rejects_bad_steps(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    desc = I.grating_2d("fit")
    ef, ea = I.plane_wave_field(desc, 1), I.plane_wave_field(desc, 2)
    w = I.seeded_w(1, 3)
    _, g1 = _fd(ctx, desc, ef, ea, w, 0.5)
    d, g2 = _fd(ctx, desc, ef, ea, w, 0.5)
    assert np.array_equal(g1, g2)
    g = torch.zeros(d.n_params, dtype=torch.float32, device="cuda")
    with pytest.raises(adg.AdgError):
        adg.adg_grad_fd(d, desc["params"], torch.from_numpy(ef).cuda(), torch.from_numpy(ea).cuda(),
                        w, 0.0, g)
