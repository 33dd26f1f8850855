"""Helpers for the GPU tests: run the CUDA path through the C ABI on torch
tensors and compare with the oracle at the stated tolerances."""
import numpy as np

FILL_TOL = 1e-6          # max abs on fill
G_REL, G_INF = 1e-4, 1e-5  # ||g - g_ref||_2 <= G_REL ||g_ref||_2 + G_INF ||g_ref||_inf


def eps_tol(desc):
    return FILL_TOL * abs(desc["eps_fg"] - desc["eps_bg"]) + 2e-6 * max(abs(desc["eps_fg"]), 1.0)


def grad_ok(g, gref):
    err = float(np.linalg.norm(np.asarray(g, np.float64) - gref))
    bound = G_REL * float(np.linalg.norm(gref)) + G_INF * float(np.abs(gref).max() if gref.size else 0)
    return err <= bound + 1e-30, err, bound


def run_build(design, desc, params=None):
    import torch
    from paper_2311_05646_gb300 import adg
    p = desc["params"] if params is None else params
    fill = torch.empty(design.shape, dtype=torch.float32, device="cuda")
    eps = torch.empty_like(fill)
    adg.adg_build_eps(design, p, eps, fill=fill)
    adg.adg_sync(design.ctx)
    return fill.cpu().numpy().astype(np.float64), eps.cpu().numpy().astype(np.float64)


def run_grad(design, desc, ef, ea, w, params=None):
    import torch
    from paper_2311_05646_gb300 import adg
    p = desc["params"] if params is None else params
    g = torch.zeros(max(design.n_params, 1), dtype=torch.float32, device="cuda")[: design.n_params]
    efd = torch.from_numpy(ef).cuda()
    ead = torch.from_numpy(ea).cuda()
    adg.adg_grad(design, p, efd, ead, w, g)
    adg.adg_sync(design.ctx)
    return g.cpu().numpy().astype(np.float64)


def run_grad_real(design, desc, G, params=None):
    import torch
    from paper_2311_05646_gb300 import adg
    p = desc["params"] if params is None else params
    g = torch.zeros(design.n_params, dtype=torch.float32, device="cuda")
    adg.adg_grad_real(design, p, torch.from_numpy(G).cuda(), g)
    adg.adg_sync(design.ctx)
    return g.cpu().numpy().astype(np.float64)
