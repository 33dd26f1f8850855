"""The ADG_DEBUG build (-DADG_DEBUG): bound checks in the kernels that record
an error bit (reported by adg_sync as ADG_EDEVICE, bit 0x80) and skip the
access instead of touching memory out of range.  Its checks stay silent on
valid work, whose results still match the FP64 oracle; and a fault planted on
the host (the debug build's ADG_DEBUG_PLANT hook moves one primitive's partial
sums one entry past the design's range -- still inside the allocated buffer,
so nothing can fault even if a check were missing) is caught and reported.
Each case runs in a child process that loads libadg_debug.so."""
import json
import os
import subprocess
import sys

import pytest

from .conftest import ROOT, cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]

CHILD = r"""
import json, sys
sys.path.insert(0, %r)
import numpy as np
from oracle import oracle as O
from paper_2311_05646_gb300 import adg, inputs as I
from tests import _gpu as H
O.build()
ctx = adg.Context(0)
cases = (("grating", I.grating_3d(n=(150, 36, 60), teeth=8, pitch=600.0)),
         ("random", I.random_design(41, n=(150, 70, 36), nprims=40)),
         ("polar", I.psgc_lattice(n=(64, 56, 12), rows=2, cols=3, harmonics=3, centres=True)))
out = {"library": adg.LIB_PATH}
for name, desc in cases:
    d = adg.Design(ctx, desc)
    try:
        fill, eps = H.run_build(d, desc)
        ef, ea = I.plane_wave_field(desc, 12), I.plane_wave_field(desc, 13)
        w = I.seeded_w(desc["grid"]["ncomp"], 5)
        g = H.run_grad(d, desc, ef, ea, w)
        out[name] = {"ok": True, "fill_err": float(np.abs(fill - O.fill(desc)).max()),
                     "grad_ok": bool(H.grad_ok(g, O.grad(desc, ef, ea, w))[0])}
    except adg.AdgError as e:
        out[name] = {"ok": False, "status": int(e.status), "msg": str(e)}
    d.close()
print(json.dumps(out))
""" % ROOT


def _run(extra_env):
    from paper_2311_05646_gb300 import build as B
    lib = B.build(debug=True)
    env = dict(os.environ, ADG_LIBRARY=lib, **extra_env)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out.pop("library").endswith("libadg_debug.so")
    return out


def test_debug_build_is_silent_on_valid_work():
    for name, v in _run({}).items():
        assert v["ok"], (name, v)
        assert v["fill_err"] <= 1e-6 and v["grad_ok"], (name, v)


def test_debug_build_catches_a_planted_partial_index():
    for name, v in _run({"ADG_DEBUG_PLANT": "partials"}).items():
        assert not v["ok"] and v["status"] == 6, (name, v)  # ADG_EDEVICE
        assert "bits 0x80" in v["msg"], (name, v)
