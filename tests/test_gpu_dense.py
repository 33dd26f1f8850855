"""adg_grad_dense against the FP64 oracle: the material-level derivatives
dL/d eps_bg, dL/d eps_fg (every cell's fields streamed) and the parameter
gradient, which must equal adg_grad's bit for bit.  Grids with a ragged plane
(nx ny nz not a multiple of 4) take the scalar path of the field stream."""
import numpy as np
import pytest

from paper_2311_05646_gb300 import inputs as I

from . import _gpu as H
from .conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

CASES = {
    "grating3d_small": lambda: I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0),
    "random_mix": lambda: I.random_design(41, n=(150, 70, 36), nprims=40),
    "ragged_2d": lambda: I.hole_lattice(n=(97, 81, 1), d=(40.0, 40.0, 40.0), holes=4, ncomp=1),
    "ragged_3d": lambda: I.random_design(47, n=(61, 37, 13), nprims=9),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_2311_05646_gb300 import adg
    return adg.Context(0)


def _dense(design, desc, ef, ea, w):
    import torch
    from paper_2311_05646_gb300 import adg
    p = desc["params"]
    fill = torch.empty(design.shape, dtype=torch.float32, device="cuda")
    eps = torch.empty_like(fill)
    adg.adg_build_eps(design, p, eps, fill=fill)
    g = torch.zeros(max(design.n_params, 1), dtype=torch.float32, device="cuda")[: design.n_params]
    gm = torch.zeros(2, dtype=torch.float64, device="cuda")
    adg.adg_grad_dense(design, p, torch.from_numpy(ef).cuda(), torch.from_numpy(ea).cuda(), w,
                       fill, g, gm)
    adg.adg_sync(design.ctx)
    return g.cpu().numpy().astype(np.float64), gm.cpu().numpy()


@pytest.mark.parametrize("case", sorted(CASES))
def test_dense_matches_oracle(ctx, oracle_mod, case):
    from paper_2311_05646_gb300 import adg
    desc = CASES[case]()
    d = adg.Design(ctx, desc)
    ef, ea = I.plane_wave_field(desc, 12), I.plane_wave_field(desc, 13)
    w = I.seeded_w(desc["grid"]["ncomp"], 5)
    g, gm = _dense(d, desc, ef, ea, w)
    gm_ref = oracle_mod.grad_material(desc, ef, ea, w)
    # bound: fp32 products and compensated fp32 partial sums, relative to the
    # sum of |Re(w E_adj E)| over all samples
    C = desc["grid"]["ncomp"]
    wc = np.broadcast_to(np.asarray(w, np.complex128).reshape(-1), (C,))
    zabs = sum(np.abs((wc[c] * ea[c].astype(np.complex128) * ef[c].astype(np.complex128)).real).sum()
               for c in range(C))
    assert np.abs(gm - gm_ref).max() <= 1e-6 * zabs, (gm, gm_ref, zabs)
    # the parameter gradient is the band path's, bit for bit
    g_plain = H.run_grad(d, desc, ef, ea, w)
    assert np.array_equal(g, g_plain)
    ok, err, bound = H.grad_ok(g, oracle_mod.grad(desc, ef, ea, w))
    assert ok, (err, bound)


def test_dense_is_deterministic(ctx):
    from paper_2311_05646_gb300 import adg
    desc = CASES["grating3d_small"]()
    d = adg.Design(ctx, desc)
    ef, ea = I.plane_wave_field(desc, 1), I.plane_wave_field(desc, 2)
    w = I.seeded_w(3, 3)
    r1 = _dense(d, desc, ef, ea, w)
    r2 = _dense(d, desc, ef, ea, w)
    assert np.array_equal(r1[0], r2[0]) and np.array_equal(r1[1], r2[1])
