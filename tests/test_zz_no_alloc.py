"""adg_grad_noalloc -- the gradient for callers that cannot allocate device
memory (their device memory belongs to another runtime's fixed arena, or
they must not grow their footprint after start-up) -- against the regular
adg_grad, through the C ABI, on two calls in a row.

This file is collected last on purpose, and it also passes alone in a fresh
process."""
import numpy as np
import pytest

from paper_2311_05646_gb300 import inputs as I

from . import _gpu as H
from .conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def test_noalloc_gradient_matches_adg_grad_on_two_calls():
    import torch

    from paper_2311_05646_gb300 import adg

    ctx = adg.Context(0)
    desc = I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0)
    design = adg.Design(ctx, desc)
    efd = torch.from_numpy(I.plane_wave_field(desc, 31)).cuda()
    ead = torch.from_numpy(I.plane_wave_field(desc, 32)).cuda()
    w = I.seeded_w(3, 33)
    p1 = desc["params"].copy()
    p2 = p1 + np.random.default_rng(5).uniform(-20.0, 20.0, p1.size)
    for p in (p1, p2):  # the second call must not see the first call's scratch
        g_ref = torch.zeros(design.n_params, dtype=torch.float32, device="cuda")
        adg.adg_grad(design, p, efd, ead, w, g_ref)
        adg.adg_sync(ctx)
        g_na = torch.full((design.n_params,), float("nan"), dtype=torch.float32, device="cuda")
        adg.adg_grad_noalloc(desc, p, efd, ead, w, g_na)
        a = g_na.cpu().numpy().astype(np.float64)
        b = g_ref.cpu().numpy().astype(np.float64)
        ok, err, bound = H.grad_ok(a, b)
        assert ok, (err, bound)
    # a design whose per-tile programs alone exceed the 32 MiB static scratch
    # (8192 x 4096 cells in 32 x 4 x 1 tiles = 262144 tiles) is refused
    big = I.grating_2d(n=(8192, 4096))
    shape = I.field_shape(big)
    ef_big = torch.zeros(shape, dtype=torch.complex64, device="cuda")
    g_big = torch.zeros(big["params"].size, dtype=torch.float32, device="cuda")
    with pytest.raises(adg.AdgError) as e:
        adg.adg_grad_noalloc(big, big["params"], ef_big, ef_big, 1.0, g_big, tile=(32, 4, 1))
    assert e.value.status == adg.ADG_EINVAL
    assert "static scratch" in str(e.value)


@pytest.mark.parametrize("case", ["polar", "mixed"])
def test_noalloc_gradient_of_polar_and_polygon_designs(case, oracle_mod):
    """Designs whose primitive records carry auxiliary tables (Polar2D Fourier
    coefficients; polygon edges, circles and boxes) through the no-allocation
    entry point: against the FP64 oracle at the stated tolerance and against
    adg_grad, on two calls in a row."""
    import torch

    from paper_2311_05646_gb300 import adg

    ctx = adg.Context(0)
    if case == "polar":
        desc = I.psgc_lattice(n=(64, 56, 12), rows=2, cols=3, harmonics=6, centres=True)
    else:
        desc = I.random_design(44, n=(70, 52, 14), nprims=18)
    design = adg.Design(ctx, desc)
    ef, ea = I.plane_wave_field(desc, 41), I.plane_wave_field(desc, 42)
    w = I.seeded_w(desc["grid"]["ncomp"], 43)
    efd, ead = torch.from_numpy(ef).cuda(), torch.from_numpy(ea).cuda()
    p1 = desc["params"].copy()
    p2 = p1 + np.random.default_rng(6).uniform(-3.0, 3.0, p1.size)
    for p in (p1, p2):
        g_ref = torch.zeros(design.n_params, dtype=torch.float32, device="cuda")
        adg.adg_grad(design, p, efd, ead, w, g_ref)
        adg.adg_sync(ctx)
        g_na = torch.full((design.n_params,), float("nan"), dtype=torch.float32, device="cuda")
        adg.adg_grad_noalloc(desc, p, efd, ead, w, g_na)
        a = g_na.cpu().numpy().astype(np.float64)
        ok, err, bound = H.grad_ok(a, g_ref.cpu().numpy().astype(np.float64))
        assert ok, ("vs adg_grad", err, bound)
        ok, err, bound = H.grad_ok(a, oracle_mod.grad(desc, ef, ea, w, params=p))
        assert ok, ("vs oracle", err, bound)


@pytest.mark.parametrize("tile", [(32, 16, 4), (32, 8, 8)])
def test_noalloc_gradient_at_2048_cell_tiles(tile, oracle_mod):
    """The largest tile shapes (2048 cells, whose VJP blocks hold a longer
    active-sample list) through the no-allocation entry point: against
    adg_grad at the same tile and against the FP64 oracle."""
    import torch

    from paper_2311_05646_gb300 import adg

    ctx = adg.Context(0)
    desc = I.random_design(4107, n=(75, 53, 27), nprims=14)
    design = adg.Design(ctx, desc, tile=tile)
    ef, ea = I.plane_wave_field(desc, 51), I.plane_wave_field(desc, 52)
    w = I.seeded_w(desc["grid"]["ncomp"], 53)
    efd, ead = torch.from_numpy(ef).cuda(), torch.from_numpy(ea).cuda()
    g_ref = torch.zeros(design.n_params, dtype=torch.float32, device="cuda")
    adg.adg_grad(design, desc["params"], efd, ead, w, g_ref)
    adg.adg_sync(ctx)
    g_na = torch.full((design.n_params,), float("nan"), dtype=torch.float32, device="cuda")
    adg.adg_grad_noalloc(desc, desc["params"], efd, ead, w, g_na, tile=tile)
    a = g_na.cpu().numpy().astype(np.float64)
    ok, err, bound = H.grad_ok(a, g_ref.cpu().numpy().astype(np.float64))
    assert ok, ("vs adg_grad", err, bound)
    ok, err, bound = H.grad_ok(a, oracle_mod.grad(desc, ef, ea, w))
    assert ok, ("vs oracle", err, bound)
