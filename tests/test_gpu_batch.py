"""Batched persistent launch: many designs of uneven size and primitive count
in one job table, at one tile shape or each at its own.  Every item's eps and
gradient equal, bit for bit, what the same design gives alone; graph replay
equals direct launch; waits are bounded."""
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


def _mix():
    descs = [I.random_design(100 + k, n=(int(40 + 23 * k), int(30 + 11 * k), int(12 + 5 * k)),
                             nprims=8 + 7 * k) for k in range(5)]
    descs.append(I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0))
    descs.append(I.taper_3d(n=(160, 60, 20), nverts=12))
    descs.append(I.hole_lattice(n=(96, 80, 1), d=(40.0, 40.0, 40.0), holes=4, ncomp=1))
    return descs


def _alloc(d, desc, rng):
    import torch
    sh = I.field_shape(desc)
    ef = torch.from_numpy(I.plane_wave_field(desc, int(rng.integers(1 << 30)))).cuda()
    ea = torch.from_numpy(I.plane_wave_field(desc, int(rng.integers(1 << 30)))).cuda()
    eps = torch.empty(sh, dtype=torch.float32, device="cuda")
    fill = torch.empty_like(eps)
    g = torch.zeros(d.n_params, dtype=torch.float32, device="cuda")
    return ef, ea, eps, fill, g


# per-design tile shapes of the mixed table: the VJP's shared memory and grid
# follow the largest tile among the gradient items (2048 cells here)
MIXED_TILES = [(32, 8, 8), None, (64, 8, 4), (32, 4, 2), (32, 16, 4), (32, 8, 4), (64, 4, 4), None]


@pytest.mark.parametrize("graph,mixed", [(False, False), (True, False), (False, True), (True, True)])
def test_batch_equals_alone(ctx, graph, mixed):
    import torch
    from paper_2311_05646_gb300 import adg
    rng = np.random.default_rng(0)
    descs = _mix()
    tiles = MIXED_TILES if mixed else [None] * len(descs)
    designs = [adg.Design(ctx, d, tile=t) for d, t in zip(descs, tiles)]
    bufs = [_alloc(d, desc, rng) for d, desc in zip(designs, descs)]
    w = I.seeded_w(3, 9)
    for rep in range(2):  # the second submit replays the captured graph
        params = [desc["params"] + (0.3 * rep) for desc in descs]
        items = []
        for k, (d, desc) in enumerate(zip(designs, descs)):
            ef, ea, eps, fill, g = bufs[k]
            wk = w[: d.ncomp]
            items.append(adg.BatchItem(d, params[k], eps=eps, fill=fill, efwd=ef, eadj=ea, w=wk, grad=g))
        t = adg.adg_batch_submit(ctx, items, graph=graph)
        adg.adg_batch_wait(ctx, t, 60.0)
        adg.adg_sync(ctx)
        for k, (d, desc) in enumerate(zip(designs, descs)):
            ef, ea, eps, fill, g = bufs[k]
            eps_b, fill_b, g_b = eps.clone(), fill.clone(), g.clone()
            adg.adg_build_eps(d, params[k], eps, fill=fill)
            adg.adg_grad(d, params[k], ef, ea, w[: d.ncomp], g)
            adg.adg_sync(ctx)
            assert torch.equal(eps_b, eps) and torch.equal(fill_b, fill), k
            assert torch.equal(g_b, g), (k, (g_b - g).abs().max().item())


def test_batch_matches_oracle_real_seed(ctx, oracle_mod):
    import torch
    from paper_2311_05646_gb300 import adg
    descs = _mix()[:4]
    designs = [adg.Design(ctx, d) for d in descs]
    Gs = [np.random.default_rng(k).normal(size=I.field_shape(d)).astype(np.float32)
          for k, d in enumerate(descs)]
    grads = [torch.zeros(d.n_params, dtype=torch.float32, device="cuda") for d in designs]
    items = [adg.BatchItem(d, desc["params"], G=torch.from_numpy(G).cuda(), grad=g)
             for d, desc, G, g in zip(designs, descs, Gs, grads)]
    adg.adg_batch_wait(ctx, adg.adg_batch_submit(ctx, items), 60.0)
    for desc, G, g in zip(descs, Gs, grads):
        ok, err, bound = H.grad_ok(g.cpu().numpy().astype(np.float64), oracle_mod.grad_real(desc, G))
        assert ok, (err, bound)


def test_batch_rejects_duplicate_designs_and_bad_ops(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    desc = I.grating_2d()
    d = adg.Design(ctx, desc)
    eps = torch.empty(d.shape, dtype=torch.float32, device="cuda")
    it = adg.BatchItem(d, desc["params"], eps=eps)
    with pytest.raises(adg.AdgError) as e:
        adg.adg_batch_submit(ctx, [it, it])
    assert e.value.status == adg.ADG_EINVAL
    with pytest.raises(adg.AdgError):
        adg.adg_batch_submit(ctx, [adg.BatchItem(d, desc["params"])])  # no operation


def test_batch_wait_is_bounded(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    desc = I.grating_3d(n=(300, 100, 60), teeth=12)
    d = adg.Design(ctx, desc)
    eps = torch.empty(d.shape, dtype=torch.float32, device="cuda")
    t = adg.adg_batch_submit(ctx, [adg.BatchItem(d, desc["params"], eps=eps)])
    try:
        adg.adg_batch_wait(ctx, t, 0.0)  # may already be done
    except adg.AdgError as e:
        assert e.status == adg.ADG_ETIMEOUT
    adg.adg_batch_wait(ctx, t, 60.0)
    assert adg.adg_batch_poll(ctx, t)


def test_large_design_between_single_calls_and_batches(ctx):
    """A grid large enough (3.6 M samples) that single calls copy their primitive
    records on the context's upload stream into the record buffer the kernels
    ahead are not reading, interleaved with batch submits that re-bin the
    design with their own records, without synchronising in between: every
    result equals that of a design used only by single calls, bit for bit."""
    import torch
    from paper_2311_05646_gb300 import adg
    desc = I.grating_3d(n=(200, 100, 60), teeth=8, pitch=600.0)
    mixed = adg.Design(ctx, desc)
    plain = adg.Design(ctx, desc)
    ef = torch.from_numpy(I.plane_wave_field(desc, 41)).cuda()
    ea = torch.from_numpy(I.plane_wave_field(desc, 42)).cuda()
    w = I.seeded_w(3, 43)
    ps = [desc["params"] + 0.2 * k for k in range(6)]
    outs, tickets = [], []
    for k, p in enumerate(ps):
        eps = torch.empty(mixed.shape, dtype=torch.float32, device="cuda")
        g = torch.zeros(mixed.n_params, dtype=torch.float32, device="cuda")
        if k % 3 == 1:
            tickets.append(adg.adg_batch_submit(
                ctx, [adg.BatchItem(mixed, p, eps=eps, efwd=ef, eadj=ea, w=w, grad=g)]))
        else:
            adg.adg_build_eps(mixed, p, eps)
            adg.adg_grad(mixed, p, ef, ea, w, g)
        outs.append((eps, g))
    for t in tickets:
        adg.adg_batch_wait(ctx, t, 60.0)
    adg.adg_sync(ctx)
    for p, (eps, g) in zip(ps, outs):
        e2 = torch.empty_like(eps)
        g2 = torch.zeros_like(g)
        adg.adg_build_eps(plain, p, e2)
        adg.adg_grad(plain, p, ef, ea, w, g2)
        adg.adg_sync(ctx)
        assert torch.equal(eps, e2)
        assert torch.equal(g, g2)
    mixed.close()
    plain.close()
