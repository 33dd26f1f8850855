"""Rotation and aspect-ratio transforms of primitives (Sec. 4, item iii) on
the GPU against the FP64 oracle: fill element by element (1e-6) and the
gradient (1e-4 relative L2 + 1e-5 of the infinity norm) with the primitives'
own scalars and the pivot, angle and aspect driven by parameters, for every
sigma kind, both logic families, 2D and 3D, ragged grids over several tiles."""
import math

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


def tilted_grating(sigma="sigmoid", kr=4.0, logic="product", n=(150, 44, 30), teeth=6):
    """A slab minus teeth that are boxes (the paper's Rect form) tilted by a
    shared angle about their own centres, each with two driven edges; a
    rotated elliptical hole with driven centre, radius, angle and aspect; a
    rotated quadrilateral and a rotated Fourier-boundary scatterer."""
    d = (40.0, 40.0, 20.0)
    D = I.Design(n, d, ncomp=3, eps_bg=2.085, eps_fg=12.11, logic=logic)
    zc = 0.5 * n[2] * d[2]
    slab = D.box(z=(zc - 110.0, zc + 110.0))
    tilt = D.param(0.21)
    ext_y = n[1] * d[1]
    etches = []
    for t in range(teeth):
        xa = 700.0 + 780.0 * t
        xb = xa + 260.0
        cx = 0.5 * (xa + xb)
        etches.append(D.box(x=(P(D.param(xa)), P(D.param(xb))), y=(-400.0, ext_y + 400.0),
                            z=(zc - 60.0, zc + 160.0), mode="sigma", sigma=sigma, kr=kr,
                            xform=(cx, 0.5 * ext_y, P(tilt), 1.0, 1.0)))
    hx, hy = D.param(2100.0), D.param(860.0)
    ell = D.circle(P(hx), P(hy), P(D.param(230.0)), z=(zc - 110.0, zc + 110.0), sigma=sigma, kr=kr,
                   xform=(P(hx), P(hy), P(D.param(0.5)), P(D.param(1.6)), P(D.param(0.7))))
    quad = [(3300.0, 420.0), (3900.0, 520.0), (3780.0, 1260.0), (3240.0, 1100.0)]
    poly = D.polygon([(P(D.param(x)), P(D.param(y))) for x, y in quad], z=(zc - 110.0, zc + 110.0),
                     sigma=sigma, kr=kr,
                     xform=(3550.0, 830.0, P(D.param(-0.35)), P(D.param(1.2)), 0.9))
    pol = D.polar(4700.0, 900.0, P(D.param(260.0)), [(P(D.param(40.0)), P(D.param(-25.0)))],
                  z=(zc - 110.0, zc + 110.0), sigma=sigma, kr=kr,
                  xform=(P(D.param(4650.0)), 880.0, P(D.param(0.8)), 1.3, P(D.param(0.8))))
    D.set_program(("diff", slab, ("union",) + tuple(etches) + (ell, poly, pol)))
    return D.to_desc()


def _check(ctx, desc, oracle_mod, tile=None):
    from paper_2311_05646_gb300 import adg
    d = adg.Design(ctx, desc, tile=tile)
    fill, eps = H.run_build(d, desc)
    fref = oracle_mod.fill(desc)
    err = np.abs(fill - fref).max()
    assert err <= H.FILL_TOL, ("fill", err)
    eref = desc["eps_bg"] + (desc["eps_fg"] - desc["eps_bg"]) * fref
    assert np.abs(eps - eref).max() <= H.eps_tol(desc)
    ef, ea = I.plane_wave_field(desc, 12), I.plane_wave_field(desc, 13)
    w = I.seeded_w(desc["grid"]["ncomp"], 5)
    g = H.run_grad(d, desc, ef, ea, w)
    gref = oracle_mod.grad(desc, ef, ea, w)
    ok, e, bound = H.grad_ok(g, gref)
    assert ok, ("grad", e, bound)
    return d, g, gref


@pytest.mark.parametrize("sigma,kr", [("sigmoid", 4.0), ("linear", 1.0), ("quadratic", 1.0),
                                      ("sin", 1.0), ("erf", 2.0)])
def test_transformed_primitives_match_the_oracle(ctx, oracle_mod, sigma, kr):
    desc = tilted_grating(sigma, kr)
    d, g, gref = _check(ctx, desc, oracle_mod)
    # the shared tilt and every transform scalar carry gradient; the tilt's
    # (radians) dominates the norm, so the rest is checked on its own too
    assert abs(gref[0]) > 0 and np.count_nonzero(gref) > 0.8 * gref.size
    ok, e, bound = H.grad_ok(g[1:], gref[1:])
    assert ok, ("grad without the tilt", e, bound)
    d.close()


@pytest.mark.parametrize("tile", [(32, 4, 4), (32, 8, 2), (64, 2, 2)])
def test_transformed_primitives_clamped_logic_and_tiles(ctx, oracle_mod, tile):
    _check(ctx, tilted_grating("sigmoid", 4.0, logic="clamp"), oracle_mod, tile=tile)[0].close()


def test_transformed_2d_single_component(ctx, oracle_mod):
    D = I.Design((97, 83, 1), (30.0, 30.0, 30.0), ncomp=1, eps_bg=1.0, eps_fg=4.0)
    th = D.param(0.37)
    D.box(x=(P(D.param(600.0)), P(D.param(1500.0))), y=(P(D.param(700.0)), P(D.param(1200.0))),
          mode="sigma", sigma="sigmoid", kr=4.0, xform=(1050.0, 950.0, P(th), 1.0, 1.0))
    D.circle(2100.0, 1600.0, P(D.param(300.0)), sigma="erf", kr=2.0,
             xform=(2100.0, 1600.0, P(th), P(D.param(1.7)), 0.6))
    _check(ctx, D.to_desc(), oracle_mod)[0].close()


def test_quarter_turn_equals_the_turned_box_on_the_gpu(ctx, oracle_mod):
    """The GPU's transformed box at 90 degrees equals the GPU's plain box with
    turned extents (up to the fill tolerance: the transformed path runs in
    FP64 local coordinates, the plain one in fp32 anchors)."""
    from paper_2311_05646_gb300 import adg
    x0, x1, y0, y1, px, py = 412.0, 1013.0, 377.0, 821.0, 700.0, 640.0
    D = I.Design((64, 60, 1), (20.0, 20.0, 20.0), ncomp=1)
    D.box(x=(x0, x1), y=(y0, y1), mode="sigma", sigma="sigmoid", kr=4.0,
          xform=(px, py, math.pi / 2, 1.0, 1.0))
    E = I.Design((64, 60, 1), (20.0, 20.0, 20.0), ncomp=1)
    E.box(x=(px - (y1 - py), px - (y0 - py)), y=(py + (x0 - px), py + (x1 - px)), mode="sigma",
          sigma="sigmoid", kr=4.0)
    a = H.run_build(adg.Design(ctx, D.to_desc()), D.to_desc())[0]
    b = H.run_build(adg.Design(ctx, E.to_desc()), E.to_desc())[0]
    assert np.abs(a - b).max() <= 2 * H.FILL_TOL


def test_transformed_design_in_a_batch_equals_alone(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    descs = [tilted_grating(), I.grating_3d(n=(96, 24, 40), teeth=5, pitch=500.0)]
    designs = [adg.Design(ctx, d) for d in descs]
    w = I.seeded_w(3, 9)
    bufs = []
    for d, desc in zip(designs, descs):
        ef = torch.from_numpy(I.plane_wave_field(desc, 3)).cuda()
        ea = torch.from_numpy(I.plane_wave_field(desc, 4)).cuda()
        eps = torch.empty(d.shape, dtype=torch.float32, device="cuda")
        g = torch.zeros(d.n_params, dtype=torch.float32, device="cuda")
        bufs.append((ef, ea, eps, g))
    items = [adg.BatchItem(d, desc["params"], eps=b[2], efwd=b[0], eadj=b[1], w=w, grad=b[3])
             for d, desc, b in zip(designs, descs, bufs)]
    adg.adg_batch_wait(ctx, adg.adg_batch_submit(ctx, items), 60.0)
    adg.adg_sync(ctx)
    for d, desc, (ef, ea, eps, g) in zip(designs, descs, bufs):
        eb, gb = eps.clone(), g.clone()
        adg.adg_build_eps(d, desc["params"] + 1e-9, eps)  # fresh binning, same values
        adg.adg_build_eps(d, desc["params"], eps)
        adg.adg_grad(d, desc["params"], ef, ea, w, g)
        adg.adg_sync(ctx)
        assert torch.equal(eb, eps)
        assert torch.equal(gb, g)


def test_bad_transforms_are_refused(ctx):
    from paper_2311_05646_gb300 import adg
    D = I.Design((40, 40, 1), (10.0, 10.0, 10.0), ncomp=1)
    D.box(x=(100.0, 200.0), y=(100.0, 300.0), xform=(150.0, 200.0, 0.3, 1.0, 1.0))  # exact form
    with pytest.raises(adg.AdgError):
        adg.Design(ctx, D.to_desc())
    D = I.Design((40, 40, 1), (10.0, 10.0, 10.0), ncomp=1)
    D.circle(200.0, 200.0, 80.0, xform=(200.0, 200.0, 0.3, 1.0, P(D.param(0.0))))  # sy = 0
    desc = D.to_desc()
    with pytest.raises(adg.AdgError) as e:  # refused once the parameters are known
        H.run_build(adg.Design(ctx, desc), desc)
    assert e.value.status == adg.ADG_EINVAL
    D = I.Design((40, 40, 1), (10.0, 20.0, 10.0), ncomp=1)  # dx != dy
    D.box(x=(100.0, 200.0), y=(100.0, 300.0), mode="sigma", xform=(150.0, 200.0, 0.3, 1.0, 1.0))
    with pytest.raises(adg.AdgError):
        adg.Design(ctx, D.to_desc())
