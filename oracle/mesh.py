"""FP64 CPU oracle of the exact polygon mesher and of the finite-difference
gradient built on it (arXiv 2311.05646: Prop. 2's "standard, exact shape
representation" for the simulation grid; Sec. 6.3's FD baseline, which
re-meshes the layout once per parameter perturbation).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.  The product library
never loads it and shares no code with it.

A layer is {"polys": [array (N, 2) of x, y vertices], "z": (z0, z1) or None}:
simple polygons (convex or concave, either winding, not overlapping one
another) extruded over [z0, z1] (None: every z).  The fill of the sample of
component c at cell (i, j, k) is the exact volume average of the layer over
the averaging cell centred at the sample, [x_s - dx/2, x_s + dx/2] x
[y_s - dy/2, y_s + dy/2] x [z_s - dz/2, z_s + dz/2], x_s = o_x + (i +
off[c][0]) dx and so on:

    fill = min(1, sum_p area(P_p n cell_xy) / (dx dy)) * |[z0, z1] n cell_z| / dz

* :func:`clip_area` -- area of one polygon inside one axis-aligned rectangle:
  Sutherland-Hodgman clipping against the rectangle's four half-planes, then
  the shoelace formula.
* :func:`fill`      -- the layer's fill on the grid (plain loops).
* :func:`grad_fd`   -- dL/dp_k = deps sum_c sum_samples Re(w E_adj E)
  (fill(layer_k^+) - fill(layer_k^-)) / 2h, the layers at p +- h e_k given.
"""
from __future__ import annotations

import numpy as np


def _clip(poly, keep, cut):
    """One Sutherland-Hodgman stage: keep(p) tells the inside of the
    half-plane, cut(p, q) the crossing of segment pq with its boundary."""
    out = []
    n = len(poly)
    for a in range(n):
        p, q = poly[a], poly[(a + 1) % n]
        ip, iq = keep(p), keep(q)
        if ip:
            out.append(p)
            if not iq:
                out.append(cut(p, q))
        elif iq:
            out.append(cut(p, q))
    return out


def _at_x(x):
    return lambda p, q: (x, p[1] + (q[1] - p[1]) * (x - p[0]) / (q[0] - p[0]))


def _at_y(y):
    return lambda p, q: (p[0] + (q[0] - p[0]) * (y - p[1]) / (q[1] - p[1]), y)


def shoelace(poly) -> float:
    """Signed area (positive counter-clockwise)."""
    s = 0.0
    n = len(poly)
    for a in range(n):
        (x0, y0), (x1, y1) = poly[a], poly[(a + 1) % n]
        s += x0 * y1 - x1 * y0
    return 0.5 * s


def clip_area(xy, x0, x1, y0, y1) -> float:
    poly = [(float(x), float(y)) for x, y in np.asarray(xy, dtype=np.float64)]
    for keep, cut in ((lambda p: p[0] >= x0, _at_x(x0)), (lambda p: p[0] <= x1, _at_x(x1)),
                      (lambda p: p[1] >= y0, _at_y(y0)), (lambda p: p[1] <= y1, _at_y(y1))):
        poly = _clip(poly, keep, cut)
        if len(poly) < 3:
            return 0.0
    return abs(shoelace(poly))


def fill(grid: dict, layer: dict) -> np.ndarray:
    nx, ny, nz = grid["n"]
    C = int(grid["ncomp"])
    dx, dy, dz = grid["d"]
    ox, oy, oz = grid["o"]
    polys = [np.asarray(p, dtype=np.float64) for p in layer["polys"]]
    boxes = [(p[:, 0].min(), p[:, 0].max(), p[:, 1].min(), p[:, 1].max()) for p in polys]
    out = np.zeros((C, nz, ny, nx))
    for c in range(C):
        offx, offy, offz = grid["off"][c]
        zf = np.ones(nz)
        if layer.get("z") is not None:
            z0, z1 = layer["z"]
            for k in range(nz):
                zs = oz + (k + offz) * dz
                zf[k] = max(0.0, min(zs + 0.5 * dz, z1) - max(zs - 0.5 * dz, z0)) / dz
        for j in range(ny):
            ys = oy + (j + offy) * dy
            cy0, cy1 = ys - 0.5 * dy, ys + 0.5 * dy
            for i in range(nx):
                xs = ox + (i + offx) * dx
                cx0, cx1 = xs - 0.5 * dx, xs + 0.5 * dx
                a = 0.0
                for p, (bx0, bx1, by0, by1) in zip(polys, boxes):
                    if bx1 <= cx0 or bx0 >= cx1 or by1 <= cy0 or by0 >= cy1:
                        continue
                    a += clip_area(p, cx0, cx1, cy0, cy1)
                out[c, :, j, i] = min(1.0, a / (dx * dy)) * zf
    return out


def _seed(grid, efwd, eadj, w):
    C = int(grid["ncomp"])
    wc = np.asarray(w, dtype=np.complex128).reshape(-1)
    if wc.size == 1:
        wc = np.repeat(wc, C)
    return np.real(wc[:C, None, None, None] * np.asarray(eadj).astype(np.complex128) *
                   np.asarray(efwd).astype(np.complex128))


def grad_fd(grid: dict, plus, minus, efwd, eadj, w, h: float, deps: float) -> np.ndarray:
    z = _seed(grid, efwd, eadj, w)
    g = np.zeros(len(plus))
    for k, (lp, lm) in enumerate(zip(plus, minus)):
        g[k] = deps * np.sum(z * (fill(grid, lp) - fill(grid, lm))) / (2.0 * h)
    return g
