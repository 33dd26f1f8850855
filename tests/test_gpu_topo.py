"""The bi-level topology special case (Sec. 3.1, Eqs. TO_example and top_AD)
through the C ABI against the FP64 oracle (oracle/topology.py), element by
element: eps within 1e-6 |deps| plus fp32 rounding; the gradient within
1e-4 ||g||_2 + 1e-5 ||g||_inf.  Regions are ragged (not multiples of a warp),
touch the grid's edges, and cover 2D and 3D grids."""
import numpy as np
import pytest

from . import _gpu as H
from .conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

CASES = {
    # grid (nx, ny, nz), ncomp, region (x0, y0, nx, ny, z0, z1)
    "slab3d": ((150, 70, 24), 3, (5, 3, 131, 61, 9, 20)),
    "edges3d": ((97, 33, 9), 3, (0, 0, 97, 33, 0, 9)),
    "one_cell_z": ((64, 40, 5), 2, (10, 7, 37, 29, 2, 3)),
    "grid2d": ((200, 100, 1), 1, (20, 10, 157, 83, 0, 1)),
}


@pytest.fixture(scope="module")
def ctx():
    from paper_2311_05646_gb300 import adg
    return adg.Context(0)


def _inputs(n, C, region, seed):
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, 2.0, region[2] * region[3]).astype(np.float32)
    shape = (C, n[2], n[1], n[0])
    ef = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    ea = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    w = rng.normal(size=C) + 1j * rng.normal(size=C)
    return v, ef, ea, w


@pytest.mark.parametrize("case", sorted(CASES))
def test_topology_matches_oracle(ctx, case):
    import torch
    from oracle import topology as T
    from paper_2311_05646_gb300 import adg
    n, C, region = CASES[case]
    v, ef, ea, w = _inputs(n, C, region, 17)
    eps_l, deps = 2.085, 12.11 - 2.085
    vd = torch.from_numpy(v).cuda()
    eps = torch.full((C, n[2], n[1], n[0]), -1.0, dtype=torch.float32, device="cuda")
    adg.adg_topo_eps(ctx, n, C, region, vd, eps_l, deps, eps)
    g = torch.zeros(v.size, dtype=torch.float32, device="cuda")
    adg.adg_topo_grad(ctx, n, C, region, vd, deps, torch.from_numpy(ef).cuda(),
                      torch.from_numpy(ea).cuda(), w, g)
    torch.cuda.synchronize()
    # the oracle with the same fp32 parameters
    eref = T.eps(n, C, region, v.astype(np.float64), eps_l, deps, eps_out=-1.0)
    tol = 1e-6 * deps + 2 * np.finfo(np.float32).eps * (eps_l + deps)
    assert np.abs(eps.cpu().numpy() - eref).max() <= tol
    gref = T.grad(n, C, region, v.astype(np.float64), deps, ef, ea, w)
    ok, err, bound = H.grad_ok(g.cpu().numpy().astype(np.float64), gref)
    assert ok, (err, bound)


def test_topology_gradient_is_deterministic(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    n, C, region = CASES["slab3d"]
    v, ef, ea, w = _inputs(n, C, region, 5)
    vd, efd, ead = torch.from_numpy(v).cuda(), torch.from_numpy(ef).cuda(), torch.from_numpy(ea).cuda()
    out = []
    for _ in range(2):
        g = torch.zeros(v.size, dtype=torch.float32, device="cuda")
        adg.adg_topo_grad(ctx, n, C, region, vd, 3.0, efd, ead, w, g)
        out.append(g.cpu().numpy())
    assert np.array_equal(out[0], out[1])


def test_topology_rejects_bad_regions(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    n, C = (32, 16, 4), 3
    eps = torch.zeros((C, 4, 16, 32), dtype=torch.float32, device="cuda")
    for region in [(0, 0, 33, 16, 0, 4), (0, 0, 8, 8, 2, 2), (-1, 0, 8, 8, 0, 4), (0, 10, 8, 8, 0, 4)]:
        v = torch.zeros(max(region[2] * region[3], 1), dtype=torch.float32, device="cuda")
        with pytest.raises((adg.AdgError, ValueError)):
            adg.adg_topo_eps(ctx, n, C, region, v[: region[2] * region[3]], 1.0, 2.0, eps)
