"""FP64 CPU oracle for the bi-level topology special case (Sec. 3.1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product library
never loads it and shares no code with it.

Plain numpy in double precision, written from the paper's composition
eps(v) = p3 o p2 o p1 (v):

* :func:`eps`  -- Eq. TO_example: eps = B (deps sigma(v) + eps_l 1), with the
  logistic sigmoid sigma and B the planarity broadcast of the region's pixels
  along z (every component's sample at the pixel's (x, y) and each z of the
  region takes the pixel's value; samples outside keep eps_out).
* :func:`grad` -- Eq. top_AD: deps sigma(v) (1 - sigma(v)) B^T Re(w E_adj E),
  the eps term of Eq. 1 with the complex weight w per component (w = -2 i
  omega gives the paper's 2 omega Im(E E_adj); no complex conjugate).
* :func:`loss` -- L = Re sum_c sum_samples w_c E_adj,c E_fwd,c eps_c, the
  scalar whose gradient Eq. top_AD is (used by the finite-difference pin).

A region is (x0, y0, nx, ny, z0, z1): pixels [x0, x0 + nx) x [y0, y0 + ny) of
the grid, broadcast to the cells [z0, z1); v has ny x nx entries, x fastest.
"""
from __future__ import annotations

import numpy as np


def sigmoid(v):
    return 1.0 / (1.0 + np.exp(-np.asarray(v, dtype=np.float64)))


def eps(n, ncomp, region, v, eps_l, deps, eps_out=0.0):
    """[ncomp][nz][ny][nx] permittivity of Eq. TO_example (p1: sigmoid, p2:
    affine map to [eps_l, eps_l + deps], p3: the broadcast B)."""
    nx, ny, nz = n
    x0, y0, rx, ry, z0, z1 = region
    e = np.full((ncomp, nz, ny, nx), float(eps_out))
    a1 = sigmoid(np.asarray(v, dtype=np.float64).reshape(ry, rx))   # p1
    a2 = deps * a1 + eps_l                                           # p2
    for c in range(ncomp):                                           # p3 = B
        for k in range(z0, z1):
            e[c, k, y0:y0 + ry, x0:x0 + rx] = a2
    return e


def loss(n, ncomp, region, v, eps_l, deps, efwd, eadj, w):
    """L = Re sum w_c E_adj,c E_fwd,c eps_c over every sample."""
    e = eps(n, ncomp, region, v, eps_l, deps)
    wc = np.broadcast_to(np.asarray(w, np.complex128).reshape(-1), (ncomp,))
    L = 0.0
    for c in range(ncomp):
        z = (wc[c] * eadj[c].astype(np.complex128) * efwd[c].astype(np.complex128)).real
        L += float((z * e[c]).sum())
    return L


def grad(n, ncomp, region, v, deps, efwd, eadj, w):
    """Eq. top_AD: the reverse sweep of the three maps, one Jacobian at a
    time: seed Re(w E_adj E) per sample, B^T (sum over the components and the
    region's z cells), times deps (p2), times sigma (1 - sigma) (p1)."""
    x0, y0, rx, ry, z0, z1 = region
    wc = np.broadcast_to(np.asarray(w, np.complex128).reshape(-1), (ncomp,))
    bt = np.zeros((ry, rx))
    for c in range(ncomp):
        z = (wc[c] * eadj[c].astype(np.complex128) * efwd[c].astype(np.complex128)).real
        bt += z[z0:z1, y0:y0 + ry, x0:x0 + rx].sum(axis=0)        # B^T
    s = sigmoid(np.asarray(v, dtype=np.float64).reshape(ry, rx))
    return (s * (1.0 - s) * deps * bt).reshape(-1)               # p1' p2' B^T
