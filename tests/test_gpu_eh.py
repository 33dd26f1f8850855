"""Both terms of Eq. 1 through the C ABI (adg_grad_eh): the permittivity
sweep over E plus the permeability sweep (Eqs. mu, jacmu) over H, two
compositions of the same parameters at the E and H sample offsets, against
the FP64 oracle's sum within 1e-4 ||g||_2 + 1e-5 ||g||_inf."""
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


def _run(ctx, desc, dmu, ef, ea, we, hf, ha, wh):
    import torch
    from paper_2311_05646_gb300 import adg
    de, dm = adg.Design(ctx, desc), adg.Design(ctx, dmu)
    g = torch.full((de.n_params,), float("nan"), dtype=torch.float32, device="cuda")
    cu = lambda a: torch.from_numpy(a).cuda()
    adg.adg_grad_eh(de, dm, desc["params"], cu(ef), cu(ea), we, cu(hf), cu(ha), wh, g)
    adg.adg_sync(ctx)
    return de, dm, g.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", ["grating2d", "grating3d_small", "random3d"])
def test_eh_gradient_matches_oracle(ctx, oracle_mod, case):
    desc = {"grating2d": lambda: I.grating_2d("fit"),
            "grating3d_small": lambda: I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0),
            "random3d": lambda: I.random_design(17, n=(70, 45, 19), nprims=16)}[case]()
    dmu = I.mu_design(desc, mu_bg=1.0, mu_fg=1.8)
    ef, ea, we = I.plane_wave_field(desc, 61), I.plane_wave_field(desc, 62), I.seeded_w(
        desc["grid"]["ncomp"], 63)
    hf, ha, wh = I.plane_wave_field(dmu, 64), I.plane_wave_field(dmu, 65), I.seeded_w(
        dmu["grid"]["ncomp"], 66)
    de, dm, g = _run(ctx, desc, dmu, ef, ea, we, hf, ha, wh)
    gref = oracle_mod.grad_eh(desc, dmu, ef, ea, we, hf, ha, wh)
    ok, err, bound = H.grad_ok(g, gref)
    assert ok, (err, bound)
    # the sum is the two single-term sweeps added (the same kernels run)
    g_e = H.run_grad(de, desc, ef, ea, we)
    g_h = H.run_grad(dm, dmu, hf, ha, wh)
    assert np.allclose(g, g_e + g_h, rtol=1e-6, atol=1e-6 * np.abs(g).max())


def test_eh_rejects_designs_with_different_parameters(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    desc = I.grating_2d("fit")
    other = I.random_design(3, n=(40, 30, 1), nprims=6)
    other["grid"]["ncomp"] = 1
    other["grid"]["off"] = other["grid"]["off"][:1]
    de = adg.Design(ctx, desc)
    do = adg.Design(ctx, I.mu_design(other))
    g = torch.zeros(de.n_params, dtype=torch.float32, device="cuda")
    f = torch.zeros(I.field_shape(desc), dtype=torch.complex64, device="cuda")
    fo = torch.zeros(I.field_shape(other), dtype=torch.complex64, device="cuda")
    assert de.n_params != do.n_params
    with pytest.raises(ValueError):
        adg.adg_grad_eh(de, do, desc["params"], f, f, 1.0, fo, fo, 1.0, g)
