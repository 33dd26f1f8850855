"""Failure paths, none of which faults or hangs the GPU.

* A device-side capacity check: a tile crossed by more edge bands than a tile
  may hold is reported by adg_sync as ADG_EDEVICE, nothing is written outside
  the caller's buffers, and the context stays usable.
* Host-side fault injection (adg_debug_alloc): an allocation made to fail, in
  design creation or in the first gradient's scratch, is reported as
  ADG_ENOMEM, the failed call releases what it had taken, and a retry works.
"""
import numpy as np
import pytest

from paper_2311_05646_gb300 import inputs as I
from paper_2311_05646_gb300.inputs import P

from . import _gpu as H
from .conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def ctx():
    from paper_2311_05646_gb300 import adg
    return adg.Context(0)


def _crowded(n_boxes=70):
    """n_boxes thin boxes whose edges all fall inside the first 32 x-cells:
    with the default 32 x 4 x 4 tile, one tile column is crossed by more
    edge bands than a tile may hold (64)."""
    D = I.Design((64, 8, 1), (1.0, 1.0, 1.0), ncomp=1, eps_bg=1.0, eps_fg=2.0)
    for i in range(n_boxes):
        x0 = 0.37 + 0.4 * i
        D.box(x=(P(D.param(x0)), x0 + 0.61))
    return D.to_desc()


def _guarded(shape, fill_value=float("nan")):
    """A tensor of `shape` at the front of a larger buffer whose tail is a
    guard that nothing may write."""
    import torch
    n = int(np.prod(shape))
    buf = torch.full((n + 4096,), fill_value, dtype=torch.float32, device="cuda")
    return buf, buf[:n].view(shape)


def test_tile_capacity_overflow_is_reported_and_stays_in_bounds(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    desc = _crowded()
    d = adg.Design(ctx, desc)
    ebuf, eps = _guarded(d.shape)
    fbuf, fill = _guarded(d.shape)
    adg.adg_build_eps(d, desc["params"], eps, fill=fill)
    with pytest.raises(adg.AdgError) as e:
        adg.adg_sync(ctx)
    assert e.value.status == adg.ADG_EDEVICE
    assert "smaller tile" in str(e.value)
    n = eps.numel()
    assert torch.isnan(ebuf[n:]).all() and torch.isnan(fbuf[n:]).all()
    # every sample of the buffer was written (the overflowed tiles as constants)
    assert not torch.isnan(eps).any()
    gbuf, g = _guarded((d.n_params,))
    ef = torch.zeros(d.shape, dtype=torch.complex64, device="cuda")
    adg.adg_grad(d, desc["params"] + 1e-3, ef, ef, 1.0, g)  # new parameters: a new binning
    with pytest.raises(adg.AdgError) as e:
        adg.adg_sync(ctx)
    assert e.value.status == adg.ADG_EDEVICE
    assert torch.isnan(gbuf[d.n_params:]).all()
    d.close()
    # the context still works, and reports no stale error
    ok = I.grating_2d("fit")
    d2 = adg.Design(ctx, ok)
    fill2, _ = H.run_build(d2, ok)
    adg.adg_sync(ctx)
    assert np.isfinite(fill2).all()
    d2.close()


def test_smaller_tiles_clear_the_capacity_error(ctx, oracle_mod):
    """The message's remedy: 70 boxes with edges in x < 60 overflow a 64-wide
    tile and fit 32-wide ones (about 38 per tile), where the fill matches
    the oracle."""
    from paper_2311_05646_gb300 import adg
    D = I.Design((128, 8, 1), (1.0, 1.0, 1.0), ncomp=1, eps_bg=1.0, eps_fg=2.0)
    for i in range(70):
        x0 = 0.37 + 0.85 * i
        D.box(x=(P(D.param(x0)), x0 + 0.61))
    desc = D.to_desc()
    wide = adg.Design(ctx, desc, tile=(64, 2, 1))
    _, eps = _guarded(wide.shape)
    adg.adg_build_eps(wide, desc["params"], eps)
    with pytest.raises(adg.AdgError) as e:
        adg.adg_sync(ctx)
    assert e.value.status == adg.ADG_EDEVICE
    wide.close()
    narrow = adg.Design(ctx, desc, tile=(32, 4, 1))
    fill, _ = H.run_build(narrow, desc)
    assert np.abs(fill - oracle_mod.fill(desc)).max() <= H.FILL_TOL
    narrow.close()


def test_allocation_failure_in_design_create_leaks_nothing(ctx, oracle_mod):
    from paper_2311_05646_gb300 import adg
    desc = I.grating_3d(n=(96, 24, 40), teeth=5, pitch=500.0)
    live0 = adg.adg_debug_alloc(-1)
    try:
        for k in (0, 1, 5, 11, 14):  # the first, an early table, a late one, the bins
            adg.adg_debug_alloc(k)
            with pytest.raises(adg.AdgError) as e:
                adg.Design(ctx, desc)
            assert e.value.status == adg.ADG_ENOMEM, k
            assert adg.adg_debug_alloc(-1) == live0, k  # injection is off again, nothing held
    finally:
        adg.adg_debug_alloc(-1)
    d = adg.Design(ctx, desc)  # the retry works
    fill, _ = H.run_build(d, desc)
    assert np.abs(fill - oracle_mod.fill(desc)).max() <= H.FILL_TOL
    d.close()
    assert adg.adg_debug_alloc(-2) == live0


def test_allocation_failure_of_first_gradient_scratch(ctx, oracle_mod):
    import torch
    from paper_2311_05646_gb300 import adg
    desc = I.grating_3d(n=(96, 24, 40), teeth=5, pitch=500.0)
    before = adg.adg_debug_alloc(-1)
    d = adg.Design(ctx, desc)
    ef, ea = I.plane_wave_field(desc, 1), I.plane_wave_field(desc, 2)
    w = I.seeded_w(3, 3)
    efd, ead = torch.from_numpy(ef).cuda(), torch.from_numpy(ea).cuda()
    g = torch.zeros(d.n_params, dtype=torch.float32, device="cuda")
    live0 = adg.adg_debug_alloc(-1)
    try:
        adg.adg_debug_alloc(0)  # the partial buffer, allocated on the first gradient
        with pytest.raises(adg.AdgError) as e:
            adg.adg_grad(d, desc["params"], efd, ead, w, g)
        assert e.value.status == adg.ADG_ENOMEM
        assert adg.adg_debug_alloc(-1) == live0
    finally:
        adg.adg_debug_alloc(-1)
    adg.adg_sync(ctx)
    gg = H.run_grad(d, desc, ef, ea, w)  # the retry allocates and computes
    ok, err, bound = H.grad_ok(gg, oracle_mod.grad(desc, ef, ea, w))
    assert ok, (err, bound)
    d.close()
    assert adg.adg_debug_alloc(-2) == before


def test_allocation_failure_inside_a_batch_submit(ctx, oracle_mod):
    """A batch whose second design cannot get its gradient scratch: ADG_ENOMEM,
    nothing held, and the designs already prepared for the batch are binned
    afresh by the retry, whose gradients match the oracle."""
    import torch
    from paper_2311_05646_gb300 import adg
    descs = [I.grating_3d(n=(96, 24, 40), teeth=5, pitch=500.0),
             I.random_design(7, n=(60, 40, 16), nprims=12)]
    designs = [adg.Design(ctx, d) for d in descs]
    fields = [(I.plane_wave_field(d, 5 + k), I.plane_wave_field(d, 9 + k)) for k, d in enumerate(descs)]
    w = I.seeded_w(3, 4)
    grads = [torch.zeros(d.n_params, dtype=torch.float32, device="cuda") for d in designs]
    items = [adg.BatchItem(d, desc["params"], efwd=torch.from_numpy(f[0]).cuda(),
                           eadj=torch.from_numpy(f[1]).cuda(), w=w[: d.ncomp], grad=g)
             for d, desc, f, g in zip(designs, descs, fields, grads)]
    live0 = adg.adg_debug_alloc(-1)
    try:
        adg.adg_debug_alloc(1)  # the first design's partials succeed, the second's fail
        with pytest.raises(adg.AdgError) as e:
            adg.adg_batch_submit(ctx, items)
        assert e.value.status == adg.ADG_ENOMEM
        assert adg.adg_debug_alloc(-1) == live0 + 1  # only the first design's partials
    finally:
        adg.adg_debug_alloc(-1)
    adg.adg_batch_wait(ctx, adg.adg_batch_submit(ctx, items), 60.0)
    adg.adg_sync(ctx)
    for desc, f, g in zip(descs, fields, grads):
        gref = oracle_mod.grad(desc, f[0], f[1], w[: desc["grid"]["ncomp"]])
        ok, err, bound = H.grad_ok(g.cpu().numpy().astype(np.float64), gref)
        assert ok, (err, bound)
    for d in designs:
        d.close()
