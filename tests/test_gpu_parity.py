"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

fill: max abs <= 1e-6; eps: 1e-6 |deps| plus fp32 rounding of eps;
gradients: ||g - g_ref||_2 <= 1e-4 ||g_ref||_2 + 1e-5 ||g_ref||_inf.
Sizes span several tiles with ragged tails; the full-size 3D grating is
checked in full (every fill and eps value, the whole gradient) at the tile
shapes the benchmark launches."""
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


def _design(ctx, desc, tile=None):
    from paper_2311_05646_gb300 import adg
    return adg.Design(ctx, desc, tile=tile)


def _check_build(ctx, desc, O, tile=None):
    d = _design(ctx, desc, tile)
    fill, eps = H.run_build(d, desc)
    fref = O.fill(desc)
    err = np.abs(fill - fref).max()
    assert err <= H.FILL_TOL, err
    eref = desc["eps_bg"] + (desc["eps_fg"] - desc["eps_bg"]) * fref
    assert np.abs(eps - eref).max() <= H.eps_tol(desc)
    return d


def _check_grad(ctx, desc, O, seeds=(12, 13), tile=None, d=None):
    d = d or _design(ctx, desc, tile)
    ef, ea = I.plane_wave_field(desc, seeds[0]), I.plane_wave_field(desc, seeds[1])
    w = I.seeded_w(desc["grid"]["ncomp"], 5)
    g = H.run_grad(d, desc, ef, ea, w)
    gref = O.grad(desc, ef, ea, w)
    ok, err, bound = H.grad_ok(g, gref)
    assert ok, (err, bound)
    return d, g


CASES = {
    "grating2d_fit": lambda: I.grating_2d("fit"),
    "grating2d_literal": lambda: I.grating_2d("literal"),
    "grating3d_small": lambda: I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0),
    "taper_small": lambda: I.taper_3d(n=(200, 75, 25), nverts=16),
    "holes_small": lambda: I.hole_lattice(n=(130, 100, 20), holes=5),
    "holes_2d": lambda: I.hole_lattice(n=(96, 80, 1), d=(40.0, 40.0, 40.0), holes=4, ncomp=1),
    "random_mix": lambda: I.random_design(41, n=(150, 70, 36), nprims=40),
    "random_mix2": lambda: I.random_design(43, n=(97, 130, 33), nprims=25),
}


def _polygon_design(per_vertex: bool, sigma="sigmoid", kr=4.0):
    """Convex polygons (Poly2D): a translated 40-gon and a hexagon whose
    every vertex coordinate is its own parameter, extruded in z."""
    D = I.Design((96, 80, 24), (40.0, 40.0, 20.0), ncomp=3, eps_bg=2.0, eps_fg=11.0)
    rng = np.random.default_rng(17)
    tx, ty = D.param(3.7), D.param(-2.2)
    import math
    big = [(I.P(tx, 1500 + 700 * math.cos(a)), I.P(ty, 1600 + 500 * math.sin(a)))
           for a in np.linspace(0, 2 * math.pi, 40, endpoint=False)]
    hexa = []
    for a in np.linspace(0, 2 * math.pi, 6, endpoint=False):
        # centre and radius off the sample lattice: no sample sits on a kink
        # of the piecewise sigmas, where fp32 and fp64 may pick either side
        x, y = 2900.37 + 301.3 * math.cos(a + 0.1), 1500.61 + 301.3 * math.sin(a + 0.1)
        hexa.append((I.P(D.param(x)), I.P(D.param(y))) if per_vertex else (x, y))
    z0 = D.param(150.0)
    p1 = D.polygon(big, z=(I.P(z0), 330.0), sigma=sigma, kr=kr)
    p2 = D.polygon(hexa[::-1], z=(120.0, 300.0), sigma=sigma, kr=kr)  # clockwise winding
    D.set_program(("union", p1, p2))
    return D.to_desc()


@pytest.mark.parametrize("per_vertex", [False, True])
@pytest.mark.parametrize("sigma", ["sigmoid", "quadratic", "linear"])
def test_polygons_match_oracle(ctx, oracle_mod, per_vertex, sigma):
    kr = {"sigmoid": 4.0, "quadratic": 1.0, "linear": 1.0}[sigma]
    desc = _polygon_design(per_vertex, sigma, kr)
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)


@pytest.mark.parametrize("case", sorted(CASES))
def test_fill_and_eps_match_oracle(ctx, oracle_mod, case):
    _check_build(ctx, CASES[case](), oracle_mod)


@pytest.mark.parametrize("case", sorted(CASES))
def test_gradient_matches_oracle(ctx, oracle_mod, case):
    _check_grad(ctx, CASES[case](), oracle_mod)


@pytest.mark.parametrize("tile", [(32, 4, 4), (64, 2, 1), (32, 1, 8), (64, 4, 4), (32, 8, 4),
                                  (32, 8, 8), (64, 8, 4), (32, 16, 4)])
def test_tile_shapes_agree(ctx, oracle_mod, tile):
    desc = I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0)
    d = _check_build(ctx, desc, oracle_mod, tile=tile)
    _check_grad(ctx, desc, oracle_mod, d=d)


@pytest.mark.parametrize("logic", ["product", "clamp"])
def test_primitive_pushed_twice(ctx, oracle_mod, logic):
    """A program that uses primitives more than once (a disc cut by a smaller
    disc, the same disc intersected with a box, and the box again): the
    binner's fold gives each repeated push the leaf it already has."""
    D = I.Design((70, 50, 20), (40.0, 40.0, 40.0), ncomp=3, logic=logic)
    a = D.circle(P(D.param(1400.0)), P(D.param(1000.0)), P(D.param(600.0)), sigma="sigmoid", kr=4.0)
    b = D.box(x=(P(D.param(900.0)), P(D.param(1900.0))), y=(700.0, 1300.0), mode="sigma",
              sigma="sigmoid", kr=4.0)
    c = D.circle(1400.0, 1000.0, P(D.param(300.0)), sigma="sigmoid", kr=4.0)
    D.set_program(("union", ("diff", a, c), ("intersect", b, a), b))
    desc = D.to_desc()
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)


@pytest.mark.parametrize("tile", [(32, 16, 4), (32, 8, 8), (64, 16, 2), (64, 4, 8)])
def test_largest_tiles_without_collapse(ctx, oracle_mod, tile):
    """2048-cell tiles on a design that collapses neither y nor z (boxes,
    circles and polygons at random places): up to 3 x 16 x 4 = 192 x-rows per
    tile, so the VJP's row scan runs its warps' rows in several rounds of 32;
    ragged in every axis."""
    desc = I.random_design(4107, n=(75, 53, 27), nprims=14)
    d = _check_build(ctx, desc, oracle_mod, tile=tile)
    _check_grad(ctx, desc, oracle_mod, d=d)


def _crowded_design(nbox: int, nested: bool, logic: str = "product"):
    """`nbox` parameterised boxes whose x and z edges all fall in the first
    tile column: a band tile there folds to 2 nbox - 1 ops.  nested: the
    program's stack is nbox deep (right-nested unions around one difference);
    else one n-ary union."""
    D = I.Design((64, 12, 6), (20.0, 20.0, 20.0), ncomp=3, eps_bg=1.5, eps_fg=4.0)
    rng = np.random.default_rng(23 + nbox)
    kids = []
    for _ in range(nbox):
        x0 = rng.uniform(10.0, 500.0)
        pa = D.param(x0)
        kids.append(D.box(x=(I.P(pa), x0 + rng.uniform(30.0, 120.0)),
                          z=(rng.uniform(3.0, 40.0), rng.uniform(70.0, 110.0))))
    if nested:
        prog = ("diff", kids[-1], kids[-2])
        for b in reversed(kids[:-2]):
            prog = ("union", b, prog)
    else:
        prog = ("union",) + tuple(kids)
    D.set_program(prog)
    desc = D.to_desc()
    desc["logic"] = logic
    return desc


@pytest.mark.parametrize("logic", ["product", "clamp"])
@pytest.mark.parametrize("nbox", [24, 40, 60])
def test_long_programs_use_the_global_tape(ctx, oracle_mod, logic, nbox):
    # 60 boxes: 119 ops and 60 leaves in one tile, next to the limits of 120 and 64
    from paper_2311_05646_gb300 import adg
    desc = _crowded_design(nbox, nested=False, logic=logic)
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)
    st = adg.adg_design_stats(d)
    # beyond the shared-memory tape (16 ops); up to 119 ops in 7-bit operand fields
    assert st["max_ops"] == 2 * nbox - 1, st


@pytest.mark.parametrize("logic", ["product", "clamp"])
def test_deep_programs_use_the_stack_fallback(ctx, oracle_mod, logic):
    desc = _crowded_design(20, nested=True, logic=logic)
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)


def test_clamp_logic_family(ctx, oracle_mod):
    desc = I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0)
    desc["logic"] = "clamp"
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)


@pytest.mark.parametrize("sigma", ["linear", "sigmoid", "quadratic", "sin", "erf"])
def test_sigma_kinds_on_graph_boundaries(ctx, oracle_mod, sigma):
    kr = {"linear": 1.0, "sigmoid": 4.0, "quadratic": 1.0, "sin": 1.5, "erf": 1.2}[sigma]
    desc = I.taper_3d(n=(160, 60, 20), nverts=12, sigma=sigma, kr=kr)
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)


def test_paper_form_rect_sigma_product(ctx, oracle_mod):
    D = I.Design((70, 50, 1), (20.0, 20.0, 20.0), ncomp=1, eps_bg=1.0, eps_fg=3.0)
    rng = np.random.default_rng(8)
    kids = []
    for _ in range(6):
        x0, y0 = rng.uniform(0, 900), rng.uniform(0, 600)
        px, py = D.param(x0), D.param(y0)
        kids.append(D.box(x=(I.P(px), x0 + rng.uniform(30, 300)), y=(I.P(py), y0 + rng.uniform(30, 300)),
                          mode="sigma", sigma=["linear", "sigmoid", "sin"][len(kids) % 3],
                          kr=[1.0, 3.0, 1.2][len(kids) % 3]))
    D.set_program(("union",) + tuple(kids))
    desc = D.to_desc()
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)


def test_real_seed_matches_oracle(ctx, oracle_mod):
    desc = I.taper_3d(n=(200, 75, 25), nverts=16)
    d = _design(ctx, desc)
    G = np.random.default_rng(3).normal(size=I.field_shape(desc)).astype(np.float32)
    g = H.run_grad_real(d, desc, G)
    gref = oracle_mod.grad_real(desc, G)
    ok, err, bound = H.grad_ok(g, gref)
    assert ok, (err, bound)


def test_gradient_is_deterministic(ctx):
    desc = I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0)
    d = _design(ctx, desc)
    ef, ea = I.plane_wave_field(desc, 1), I.plane_wave_field(desc, 2)
    w = I.seeded_w(3, 3)
    g1 = H.run_grad(d, desc, ef, ea, w)
    p2 = desc["params"] + 1.0  # force a rebin in between
    H.run_grad(d, desc, ef, ea, w, params=p2)
    g2 = H.run_grad(d, desc, ef, ea, w)
    assert np.array_equal(g1, g2)


def test_long_chains_span_binner_segments(ctx, oracle_mod):
    """A 48 x 48 hole lattice: 2306 primitives, a chained program of 4611
    words, so the binner compacts and walks it in two segments and in many
    512-word slabs.  The tile programs it writes are what the build and the
    VJP run; they are checked through the fill, on sampled cells of a 3D grid
    and in full on a 2D one (the oracle gradient of 6912 parameters on this
    design takes minutes)."""
    desc = I.hole_lattice(n=(192, 192, 8), d=(40.0, 40.0, 20.0), holes=48)
    assert len(desc["prims"]["kind"]) == 2306
    d = _design(ctx, desc)
    fill, _ = H.run_build(d, desc)
    idx = np.random.default_rng(9).choice(fill.size, 20000, replace=False)
    fref = oracle_mod.fill_at(desc, idx)
    assert np.abs(fill.reshape(-1)[idx] - fref).max() <= H.FILL_TOL
    desc2 = I.hole_lattice(n=(192, 192, 1), d=(40.0, 40.0, 40.0), holes=48, ncomp=1)
    _check_build(ctx, desc2, oracle_mod)


def test_build_fill_warps_agree(ctx, oracle_mod):
    """The build's second fill warp (tile option) changes who writes the
    constant tiles, not what is written: fill and eps equal bit for bit, and
    the fill matches the oracle.  Other counts are rejected."""
    from paper_2311_05646_gb300 import adg
    desc = I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0)
    f1, e1 = H.run_build(_design(ctx, desc, (32, 8, 4)), desc)
    f2, e2 = H.run_build(_design(ctx, desc, (32, 8, 4, 2)), desc)
    assert np.array_equal(f1, f2) and np.array_equal(e1, e2)
    assert np.abs(f2 - oracle_mod.fill(desc)).max() <= H.FILL_TOL
    with pytest.raises(adg.AdgError):
        _design(ctx, desc, (32, 8, 4, 3))


def test_partials_and_counts_reset_between_calls(ctx):
    """The finalize clears the partials it sums and moves the active-sample
    count, so a call after others (same bins, or a rebin with another partial
    layout) equals the first call on a fresh design."""
    from paper_2311_05646_gb300 import adg
    desc = I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0)
    ef, ea = I.plane_wave_field(desc, 4), I.plane_wave_field(desc, 5)
    w = I.seeded_w(3, 6)
    d = _design(ctx, desc)
    g0 = H.run_grad(d, desc, ef, ea, w)
    n0 = adg.adg_design_stats(d)["active_samples"]
    H.run_grad(d, desc, ef, ea, w)
    assert adg.adg_design_stats(d)["active_samples"] == n0 > 0
    p2 = desc["params"] + 40.0  # other partial boxes
    H.run_grad(d, desc, ef, ea, w, params=p2)
    g1 = H.run_grad(d, desc, ef, ea, w)
    assert np.array_equal(g0, g1)
    assert adg.adg_design_stats(d)["active_samples"] == n0
    fresh = _design(ctx, desc)
    assert np.array_equal(H.run_grad(fresh, desc, ef, ea, w), g0)


def test_param_change_rebins(ctx, oracle_mod):
    desc = I.grating_2d()
    d = _design(ctx, desc)
    p2 = desc["params"] + np.random.default_rng(2).uniform(-30, 30, desc["params"].size)
    fill, _ = H.run_build(d, desc, params=p2)
    assert np.abs(fill - oracle_mod.fill(desc, p2)).max() <= H.FILL_TOL


def test_degenerate_designs(ctx, oracle_mod):
    # design entirely outside the grid: fill 0 everywhere, zero gradient
    D = I.Design((40, 30, 1), (10.0, 10.0, 10.0), ncomp=1, eps_bg=1.0, eps_fg=2.0)
    p = D.param(-500.0)
    D.box(x=(I.P(p), -400.0), y=(0.0, 100.0))
    desc = D.to_desc()
    d = _design(ctx, desc)
    fill, eps = H.run_build(d, desc)
    assert fill.max() == 0.0 and np.all(eps == 1.0)
    ef, ea = I.plane_wave_field(desc, 1), I.plane_wave_field(desc, 2)
    assert np.all(H.run_grad(d, desc, ef, ea, 1.0) == 0.0)
    # covering everything: constant 1, no parameters at all
    D = I.Design((40, 30, 1), (10.0, 10.0, 10.0), ncomp=1, eps_bg=1.0, eps_fg=2.0)
    D.box(x=(-100.0, 1000.0))
    desc = D.to_desc()
    d = _design(ctx, desc)
    fill, eps = H.run_build(d, desc)
    assert np.all(fill == 1.0) and np.all(eps == 2.0)
    # a single-cell-thin feature and a box thinner than one cell
    D = I.Design((33, 9, 1), (1.0, 1.0, 1.0), ncomp=1, eps_bg=1.0, eps_fg=2.0)
    a = D.param(10.3)
    D.set_program(("union", D.box(x=(I.P(a), 10.55)), D.box(x=(20.1, 20.2), y=(2.0, 7.0))))
    desc = D.to_desc()
    _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod)


def _degenerate_geometry(logic):
    """Parameterised shapes at the edges of their definitions: a box that its
    parameters turn inside out (x1 < x0: empty, zero gradient), edges exactly
    on cell faces, two boxes sharing one edge parameter, a circle of radius 0
    and one of negative radius, and a triangle a few cells across."""
    D = I.Design((48, 40, 6), (10.0, 10.0, 10.0), ncomp=3, eps_bg=1.0, eps_fg=3.0, logic=logic)
    inv = D.box(x=(P(D.param(260.0)), P(D.param(200.0))), y=(50.0, 300.0))
    face = D.box(x=(P(D.param(100.0)), P(D.param(150.0))), y=(P(D.param(40.0)), 90.0))
    e = D.param(330.0)
    b1 = D.box(x=(300.0, P(e)), y=(200.0, 300.0))
    b2 = D.box(x=(P(e), 360.0), y=(200.0, 300.0))
    c0 = D.circle(150.0, 300.0, P(D.param(0.0)), sigma="sigmoid", kr=4.0)
    cn = D.circle(250.0, 320.0, P(D.param(-20.0)), sigma="sigmoid", kr=4.0)
    tri = D.polygon([(P(D.param(400.0)), 100.0), (420.0, 100.0), (410.0, P(D.param(115.0)))],
                    sigma="sigmoid", kr=4.0)
    D.set_program(("union", inv, face, b1, b2, c0, cn, tri))
    return D.to_desc()


@pytest.mark.parametrize("logic,tile", [("product", None), ("clamp", None), ("product", (32, 16, 4))])
def test_degenerate_geometry_matches_the_oracle(ctx, oracle_mod, logic, tile):
    desc = _degenerate_geometry(logic)
    d = _check_build(ctx, desc, oracle_mod, tile=tile)
    _, g = _check_grad(ctx, desc, oracle_mod, d=d)
    assert np.all(g[:2] == 0.0)  # the inverted box drives nothing


def test_invalid_descriptions_rejected(ctx):
    from paper_2311_05646_gb300 import adg
    desc = I.grating_2d()
    bad = dict(desc)
    bad["ops"] = np.asarray(list(desc["ops"]) + [(1 << 24) | 2], dtype=np.int32)  # stack underflow
    with pytest.raises(adg.AdgError) as e:
        adg.Design(ctx, bad)
    assert e.value.status == adg.ADG_EINVAL
    bad = dict(desc)
    bad["q_param"] = desc["q_param"].copy()
    bad["q_param"][5] = 999
    with pytest.raises(adg.AdgError):
        adg.Design(ctx, bad)
    with pytest.raises(adg.AdgError):
        adg.Design(ctx, desc, tile=(48, 4, 4))
    with pytest.raises(adg.AdgError):
        adg.Design(ctx, desc, tile=(64, 16, 8))  # more cells than a tile may hold
    with pytest.raises(adg.AdgError):
        adg.Design(ctx, desc, tile=(64, 8, 8))  # 4096 cells


@pytest.mark.slow
def test_full_size_grating3d(ctx, oracle_mod):
    """600 x 200 x 120 x 3 components, 60 etches, 120 parameters, in the
    launch configurations the benchmark times -- the library's default tile
    and the autotuner's choice for this design (32x16x4 with two build fill
    warps, and with one; 32x8x4, the best 1024-cell shape): every fill and
    eps value against the oracle's full
    fill, the full gradient against the oracle's full reverse sweep (the
    oracle runs once for both)."""
    import torch
    from paper_2311_05646_gb300 import adg
    desc = I.grating_3d()
    ef, ea = I.plane_wave_field(desc, 22), I.plane_wave_field(desc, 23)
    w = I.seeded_w(3, 24)
    fref = oracle_mod.fill(desc)
    eref = desc["eps_bg"] + (desc["eps_fg"] - desc["eps_bg"]) * fref
    gref = oracle_mod.grad(desc, ef, ea, w)
    for tile in (None, (32, 16, 4, 2), (32, 16, 4, 1), (32, 8, 4, 2)):
        d = _design(ctx, desc, tile)
        fill = torch.empty(d.shape, dtype=torch.float32, device="cuda")
        eps = torch.empty_like(fill)
        adg.adg_build_eps(d, desc["params"], eps, fill=fill)
        adg.adg_sync(ctx)
        ferr = float(np.abs(fill.cpu().numpy().astype(np.float64) - fref).max())
        eerr = float(np.abs(eps.cpu().numpy().astype(np.float64) - eref).max())
        assert ferr <= H.FILL_TOL, ("fill max abs err", tile, ferr)
        assert eerr <= H.eps_tol(desc), ("eps max abs err", tile, eerr)
        g = H.run_grad(d, desc, ef, ea, w)
        ok, err, bound = H.grad_ok(g, gref)
        assert ok, (tile, err, bound)
        d.close()
