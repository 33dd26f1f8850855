"""Serving: continuous batching with memory-gated admission.  Each request's
gradient matches the FP64 oracle at the same parameters (the stated
tolerance) and equals what the same design gives alone (bitwise), admission
respects the memory budget counted from the bytes libadg reports, and every
client completes its iterations."""
import numpy as np
import pytest

from paper_2311_05646_gb300 import inputs as I

from . import _gpu as H
from .conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


def test_served_results_match_the_oracle_and_admission_is_gated(oracle_mod):
    import torch
    from paper_2311_05646_gb300 import adg
    from paper_2311_05646_gb300 import serve as S

    ctx = adg.Context(0)
    descs = [I.hole_lattice(n=(96, 80, 1), d=(40.0, 40.0, 40.0), holes=4, ncomp=1, seed=60 + k)
             for k in range(3)]
    descs += [I.random_design(70 + k, n=(64 + 16 * k, 48, 24), nprims=12 + 4 * k) for k in range(3)]
    clients = []
    for k, desc in enumerate(descs):
        ef = torch.from_numpy(I.plane_wave_field(desc, 500 + k)).cuda()
        ea = torch.from_numpy(I.plane_wave_field(desc, 600 + k)).cuda()
        clients.append(S.Client(cid=k, desc=desc, efwd=ef, eadj=ea,
                                w=I.seeded_w(desc["grid"]["ncomp"], 700 + k), iterations=4))
    # a budget that holds about two clients at a time, from the bytes libadg
    # reports for each compiled design plus its buffers
    feet = [S.footprint(ctx, c) for c in clients]
    assert all(f > c.buffer_bytes() for f, c in zip(feet, clients))
    budget = 2 * max(feet) + 1
    seen = []

    def record(r):
        if r.op == "grad":
            seen.append((r.client.cid, r.params.copy(), r.client.grad.clone()))

    srv = S.Server(ctx, mem_budget_bytes=budget, max_inflight=2, on_result=record)
    peak = 0
    for c in clients:
        srv.arrive(c, 0.0)
        peak = max(peak, srv.used)
    t_end = 0
    while not srv.idle():
        if not srv.poll():
            pass
        peak = max(peak, srv.used)
        t_end += 1
        assert t_end < 10_000_000
    assert peak <= budget
    assert len(srv.finished_clients) == len(clients)
    assert all(c.done_iters == 4 for c in clients)
    # every gradient seen in the mix equals the one the design gives alone
    alone = {}
    for cid, p, g_mix in seen:
        c = clients[cid]
        d = alone.get(cid) or adg.Design(ctx, c.desc)
        alone[cid] = d
        ef = torch.from_numpy(I.plane_wave_field(c.desc, 500 + cid)).cuda()
        ea = torch.from_numpy(I.plane_wave_field(c.desc, 600 + cid)).cuda()
        g = torch.zeros(d.n_params, dtype=torch.float32, device="cuda")
        adg.adg_grad(d, p, ef, ea, c.w, g)
        adg.adg_sync(ctx)
        a = g_mix.cpu().numpy().astype(np.float64)
        b = g.cpu().numpy().astype(np.float64)
        ok, err, bound = H.grad_ok(a, b)
        assert ok, (cid, err, bound)
        assert np.array_equal(a, b), cid
        gref = oracle_mod.grad(c.desc, I.plane_wave_field(c.desc, 500 + cid),
                               I.plane_wave_field(c.desc, 600 + cid), c.w, params=p)
        ok, err, bound = H.grad_ok(a, gref)
        assert ok, ("served vs oracle", cid, err, bound)
    assert len(seen) == 4 * len(clients)
