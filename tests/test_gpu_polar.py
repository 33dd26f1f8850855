"""Polar2D with a Fourier boundary (Table 4; the PSGC scatterers' R(theta))
through the C ABI against the FP64 oracle: fill within 1e-6, eps within
1e-6 |deps| plus fp32 rounding, gradients within 1e-4 ||g||_2 + 1e-5
||g||_inf.  Cases: PSGC-like lattices in 3D (Yee offsets, z range) and 2D,
scatterer centres as parameters or fixed, up to 8 harmonics, every sigma
kind, both logic families, ragged grids over several tiles."""
import numpy as np
import pytest

from paper_2311_05646_gb300 import inputs as I

from . import _gpu as H
from .conftest import cuda_ok
from .test_gpu_parity import _check_build, _check_grad

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def ctx():
    from paper_2311_05646_gb300 import adg
    return adg.Context(0)


CASES = {
    "psgc3d_centres": lambda: I.psgc_lattice(n=(150, 97, 21), rows=3, cols=4, harmonics=3,
                                             centres=True),
    "psgc3d_six": lambda: I.psgc_lattice(n=(131, 110, 19), rows=3, cols=3, harmonics=6),
    "psgc2d_eight": lambda: I.psgc_lattice(n=(203, 161, 1), rows=3, cols=4, harmonics=8,
                                           centres=True),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_polar_fill_and_gradient_match_oracle(ctx, oracle_mod, case):
    desc = CASES[case]()
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)


@pytest.mark.parametrize("sigma", ["linear", "quadratic", "sin", "erf"])
def test_polar_sigma_kinds(ctx, oracle_mod, sigma):
    desc = I.psgc_lattice(n=(96, 80, 1), rows=2, cols=3, harmonics=4, centres=True, sigma=sigma,
                          kr=2.0)
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)


def test_polar_clamp_logic(ctx, oracle_mod):
    desc = I.psgc_lattice(n=(120, 90, 12), rows=2, cols=3, harmonics=5, centres=True)
    desc["logic"] = "clamp"
    d = _check_build(ctx, desc, oracle_mod)
    _check_grad(ctx, desc, oracle_mod, d=d)


def test_polar_rejects_bad_scalar_counts(ctx):
    from paper_2311_05646_gb300 import adg
    desc = I.psgc_lattice(n=(64, 48, 1), rows=1, cols=1, harmonics=2)
    bad = dict(desc)
    bad["prims"] = {k: v.copy() for k, v in desc["prims"].items()}
    bad["prims"]["nq"][1] -= 1  # 5 + 2N - 1 scalars
    with pytest.raises(adg.AdgError):
        adg.Design(ctx, bad)
