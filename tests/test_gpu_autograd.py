"""The differentiable taper through torch.autograd: backward recomputes fill
(adg_grad_real), matches the FP64 oracle gradient, which matches central FD of
the oracle's loss at h = 1e-3 nm; the graph saves no grid-sized tensor."""
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


def _loss_and_grad(design, desc, G):
    import torch
    from paper_2311_05646_gb300.autograd import eps_of
    p = torch.tensor(desc["params"], dtype=torch.float64, requires_grad=True)
    eps = eps_of(design, p)
    Gt = torch.from_numpy(G).cuda()
    L = (eps * Gt).sum()
    L.backward()
    return eps, p.grad.numpy().copy()


def test_autograd_backward_matches_oracle_and_fd(ctx, oracle_mod):
    from paper_2311_05646_gb300 import adg
    desc = I.taper_3d(n=(160, 60, 20), nverts=12)
    design = adg.Design(ctx, desc)
    G = np.random.default_rng(11).normal(size=I.field_shape(desc)).astype(np.float32)
    eps, g = _loss_and_grad(design, desc, G)
    gref = oracle_mod.grad_real(desc, G)
    ok, err, bound = H.grad_ok(g, gref)
    assert ok, (err, bound)
    # the FP64 chain: the oracle's analytic gradient against central FD of
    # L = sum G eps (fields G + 0i, ones, w = 1) at h = 1e-3 nm
    Gc = G.astype(np.complex64)
    ones = np.ones_like(Gc)
    gfd = oracle_mod.grad_fd(desc, Gc, ones, 1.0, 1e-3)
    assert np.linalg.norm(gfd - gref) <= 1e-6 * np.linalg.norm(gref)
    # and the fp32 GPU gradient against FD directly, at the parity tolerance
    ok, err, bound = H.grad_ok(g, gfd)
    assert ok, (err, bound)


def test_backward_saves_only_parameters(ctx):
    import torch
    from paper_2311_05646_gb300 import adg
    from paper_2311_05646_gb300.autograd import eps_of
    desc = I.taper_3d(n=(200, 75, 25), nverts=16)
    design = adg.Design(ctx, desc)
    p = torch.tensor(desc["params"], dtype=torch.float64, requires_grad=True)
    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    eps = eps_of(design, p)
    torch.cuda.synchronize()
    m1 = torch.cuda.memory_allocated()
    saved = eps.grad_fn.saved_tensors
    assert len(saved) == 1 and saved[0].numel() == desc["params"].size
    # forward keeps exactly the output (no fill, no Jacobian, no tape)
    assert m1 - m0 <= eps.numel() * 4 + (1 << 20)
    (eps.sum()).backward()
    assert p.grad is not None and p.grad.shape == p.shape


@pytest.mark.slow
def test_full_size_taper_autograd(ctx, oracle_mod):
    """The 800 x 300 x 100 taper, 128 vertex-offset parameters, sigmoid k = 4/dx."""
    from paper_2311_05646_gb300 import adg
    desc = I.taper_3d()
    design = adg.Design(ctx, desc)
    G = np.random.default_rng(12).normal(size=I.field_shape(desc)).astype(np.float32)
    eps, g = _loss_and_grad(design, desc, G)
    gref = oracle_mod.grad_real(desc, G)
    ok, err, bound = H.grad_ok(g, gref)
    assert ok, (err, bound)
    fref = oracle_mod.fill(desc)
    eref = desc["eps_bg"] + (desc["eps_fg"] - desc["eps_bg"]) * fref
    err = float(np.abs(eps.detach().cpu().numpy().astype(np.float64) - eref).max())
    assert err <= H.eps_tol(desc), ("eps max abs err", err)
