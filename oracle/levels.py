"""FP64 CPU oracle for the union over non-binary material levels (App. B,
Alg. 1 of arXiv 2311.05646).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product library
never loads it and shares no code with it.

K sets of shape primitives, set k carrying the material level eps^k above the
background (0 < eps^1 <= ... <= eps^K).  Each set is one design description
whose program is that set's union and whose material slots are eps_bg = 0,
eps_fg = 1, so its fill (``oracle.fill``) is s^k = union(s^k_1, ..., s^k_Nk).
All sets share one parameter vector.

* :func:`eps`  -- Alg. 1 in its order: s <- s^1; for k = 2..K,
  s <- union((eps^{k-1} / eps^k) s, s^k); the result is eps_bg + eps^K s.
  union is the designs' own logic family (Eq. union, clamped; or the product
  form of App. B.2).
* :func:`grad` -- Eq. 1 (eps term) through Alg. 1: the reverse of the loop
  turns the seed Re(w E_adj E) into one real cotangent per set, and each
  set's reverse sweep (``oracle.grad_real``) maps its cotangent to the
  parameters; the K results add.
* :func:`loss` -- L = Re sum_c sum_samples w_c E_adj,c E_fwd,c eps_c (the
  scalar whose gradient :func:`grad` is; used by the finite-difference pin).

Readings: the clamped union passes its derivative through at a + b = 1
(inclusive), as everywhere else in this package; the per-set cotangent goes
to ``oracle.grad_real`` rounded to float32 (that entry takes float32, as the
library's does), a relative rounding of 6e-8 per sample.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def _check(sets, eps_levels):
    lv = np.asarray(eps_levels, dtype=np.float64).reshape(-1)
    if len(sets) != lv.size or lv.size < 1:
        raise ValueError("one material level per set")
    if not (lv[0] > 0 and np.all(np.diff(lv) >= 0)):
        raise ValueError("levels must be positive and sorted ascending")
    logic = sets[0]["logic"]
    for d in sets:
        if d["logic"] != logic or d["eps_bg"] != 0.0 or d["eps_fg"] != 1.0:
            raise ValueError("every set needs the same logic and material slots 0 / 1")
    return lv, logic


def union(logic: str, a, b):
    """Eq. union for two operands (clamped), or App. B.2's product form."""
    if logic == "clamp":
        return np.minimum(1.0, a + b)
    return a + b - a * b


def _union_partials(logic: str, a, b):
    """(d union / d a, d union / d b)."""
    if logic == "clamp":
        t = (a + b <= 1.0).astype(np.float64)
        return t, t
    return 1.0 - b, 1.0 - a


def eps(sets, eps_levels, eps_bg: float, params=None) -> np.ndarray:
    lv, logic = _check(sets, eps_levels)
    s = O.fill(sets[0], params)
    for k in range(1, lv.size):
        sk = O.fill(sets[k], params)
        s = union(logic, (lv[k - 1] / lv[k]) * s, sk)
    return eps_bg + lv[-1] * s


def _seed(desc, efwd, eadj, w):
    C = int(desc["grid"]["ncomp"])
    wc = np.asarray(w, dtype=np.complex128).reshape(-1)
    if wc.size == 1:
        wc = np.repeat(wc, C)
    ef = np.asarray(efwd).astype(np.complex128)
    ea = np.asarray(eadj).astype(np.complex128)
    return np.real(wc[:C, None, None, None] * ea * ef)


def loss(sets, eps_levels, eps_bg, efwd, eadj, w, params=None) -> float:
    return float(np.sum(_seed(sets[0], efwd, eadj, w) * eps(sets, eps_levels, eps_bg, params)))


def grad(sets, eps_levels, efwd, eadj, w, params=None) -> np.ndarray:
    lv, logic = _check(sets, eps_levels)
    K = lv.size
    # forward, keeping the scaled operand a_k and the set fill s^k of every step
    S = [O.fill(d, params) for d in sets]
    s = S[0]
    a = [None] * K
    for k in range(1, K):
        a[k] = (lv[k - 1] / lv[k]) * s
        s = union(logic, a[k], S[k])
    # reverse: d L / d s starts at eps^K times the seed
    sbar = lv[-1] * _seed(sets[0], efwd, eadj, w)
    cot = [None] * K
    for k in range(K - 1, 0, -1):
        da, db = _union_partials(logic, a[k], S[k])
        cot[k] = sbar * db
        sbar = sbar * da * (lv[k - 1] / lv[k])
    cot[0] = sbar
    g = None
    for k in range(K):
        gk = O.grad_real(sets[k], cot[k].astype(np.float32), params)
        g = gk if g is None else g + gk
    return g
