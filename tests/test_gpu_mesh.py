"""The exact polygon mesher (Prop. 2's standard representation) and the
finite-difference gradient built on it (Sec. 6.3's FD baseline), through the
C ABI (adg_mesh_fill, adg_mesh_grad_fd), against the FP64 oracle
(oracle/mesh.py, Sutherland-Hodgman clipping): fills within 1e-6 per sample
(FP64 in the kernel, rounded to float once), gradients within
1e-4 ||g||_2 + 1e-5 ||g||_inf.  Cases: concave polygons in 2D, hexagonal holes
through a slab in 3D with Yee offsets and a z range, ragged regions."""
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


def _stars(seed, n, d):
    rng = np.random.default_rng(seed)
    ex, ey = n[0] * d[0], n[1] * d[1]
    polys = []
    for cx, cy in ((0.25, 0.3), (0.7, 0.35), (0.45, 0.75), (0.85, 0.8)):
        nv = int(rng.integers(5, 15))
        t = np.sort(rng.uniform(0, 2 * np.pi, nv))
        r = 0.12 * min(ex, ey) * np.where(np.arange(nv) % 2 == 0, 1.0, 0.5) * rng.uniform(0.8, 1, nv)
        p = np.stack([cx * ex + r * np.cos(t), cy * ey + r * np.sin(t)], axis=1)
        polys.append(p if rng.uniform() < 0.5 else p[::-1])
    return polys


def _fill(ctx, grid, layer, region=None):
    import torch
    from paper_2311_05646_gb300 import adg
    nx, ny, nz = grid["n"]
    f = torch.full((grid["ncomp"], nz, ny, nx), float("nan"), dtype=torch.float32, device="cuda")
    adg.adg_mesh_fill(ctx, grid, layer, f, region=region)
    torch.cuda.synchronize()
    return f.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", ["stars2d", "stars2d_corner", "hex3d", "hex3d_region"])
def test_mesh_fill_matches_oracle(ctx, case):
    from oracle import mesh as M
    if case.startswith("stars2d"):
        off = [[0.5, 0.5, 0.0]] if case == "stars2d" else [[0.0, 0.0, 0.0]]
        grid = {"n": (83, 61, 1), "ncomp": 1, "d": (10.0, 7.0, 10.0), "o": (-13.0, 4.5, 0.0),
                "off": off}
        layer = {"polys": _stars(5, grid["n"], grid["d"]), "z": None}
        region = None
    else:
        spec = I.hex_hole_lattice(n=(97, 45, 19), d=(40.0, 40.0, 20.0), holes=(5, 3), R=230.0)
        grid = spec["desc"]["grid"]
        layer = I.hex_layer(spec, spec["desc"]["params"])
        region = (13, 7, 61, 29, 3, 17) if case == "hex3d_region" else None
    got = _fill(ctx, grid, layer, region)
    want = M.fill(grid, layer)
    if region is None:
        assert np.abs(got - want).max() <= 1e-6
    else:
        x0, y0, rx, ry, z0, z1 = region
        sl = (slice(None), slice(z0, z1), slice(y0, y0 + ry), slice(x0, x0 + rx))
        assert np.abs(got[sl] - want[sl]).max() <= 1e-6
        outside = np.ones(got.shape, dtype=bool)
        outside[sl] = False
        assert np.isnan(got[outside]).all()  # not written
    assert want.max() > 0.99


def test_mesh_fd_gradient_matches_oracle(ctx):
    import torch
    from oracle import mesh as M
    from paper_2311_05646_gb300 import adg
    spec = I.hex_hole_lattice(n=(60, 40, 10), d=(40.0, 40.0, 40.0), holes=(3, 2), R=200.0)
    desc = spec["desc"]
    grid = desc["grid"]
    p0 = desc["params"]
    h = 0.5
    plus, minus, regions = I.hex_fd_layers(spec, p0, h)
    ef, ea, w = I.plane_wave_field(desc, 41), I.plane_wave_field(desc, 42), I.seeded_w(3, 43)
    deps = -(desc["eps_fg"] - desc["eps_bg"])  # the layer holds the holes
    efd, ead = torch.from_numpy(ef).cuda(), torch.from_numpy(ea).cuda()
    g = torch.full((p0.size,), float("nan"), dtype=torch.float32, device="cuda")
    adg.adg_mesh_grad_fd(ctx, grid, plus, minus, regions, h, deps, efd, ead, w, g)
    g2 = torch.zeros_like(g)
    adg.adg_mesh_grad_fd(ctx, grid, plus, minus, None, h, deps, efd, ead, w, g2)  # whole grid
    torch.cuda.synchronize()
    gref = M.grad_fd(grid, plus, minus, ef, ea, w, h, deps)
    gg = g.cpu().numpy().astype(np.float64)
    ok, err, bound = H.grad_ok(gg, gref)
    assert ok, (err, bound)
    ok2, err2, bound2 = H.grad_ok(g2.cpu().numpy().astype(np.float64), gref)
    assert ok2, (err2, bound2)
    g3 = torch.zeros_like(g)
    adg.adg_mesh_grad_fd(ctx, grid, plus, minus, regions, h, deps, efd, ead, w, g3)
    torch.cuda.synchronize()
    assert torch.equal(g, g3)  # fixed-order sums


def test_mesh_rejects_bad_inputs(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    grid = {"n": (16, 12, 1), "ncomp": 1, "d": (10.0, 10.0, 10.0), "o": (0.0, 0.0, 0.0),
            "off": [[0.5, 0.5, 0.0]]}
    f = torch.zeros((1, 1, 12, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(adg.AdgError):  # two vertices
        adg.adg_mesh_fill(ctx, grid, {"polys": [np.array([[0.0, 0.0], [5.0, 5.0]])], "z": None}, f)
    with pytest.raises(adg.AdgError):  # region outside the grid
        adg.adg_mesh_fill(ctx, grid, {"polys": [], "z": None}, f, region=(10, 0, 8, 4, 0, 1))
    with pytest.raises(adg.AdgError):  # reversed z range
        adg.adg_mesh_fill(ctx, grid, {"polys": [], "z": (5.0, 1.0)}, f)
    fields = torch.zeros((1, 1, 12, 16), dtype=torch.complex64, device="cuda")
    g = torch.zeros(1, dtype=torch.float32, device="cuda")
    lay = {"polys": [np.array([[10.0, 10.0], [50.0, 10.0], [30.0, 40.0]])], "z": None}
    with pytest.raises(adg.AdgError):  # step must be positive
        adg.adg_mesh_grad_fd(ctx, grid, [lay], [lay], None, 0.0, 1.0, fields, fields, 1.0, g)
