"""Independent exact 2D geometry for pinning the oracle: convex polygon
clipping (Sutherland-Hodgman) and shoelace areas.  Shares nothing with the
oracle's formulas; it is a different algorithm for the same areas."""
import numpy as np


def clip_halfplane(poly, a, b, c):
    """Keep the part of `poly` with a*x + b*y <= c."""
    out = []
    n = len(poly)
    for i in range(n):
        p, q = poly[i], poly[(i + 1) % n]
        fp, fq = a * p[0] + b * p[1] - c, a * q[0] + b * q[1] - c
        if fp <= 0:
            out.append(p)
        if (fp < 0 < fq) or (fq < 0 < fp):
            t = fp / (fp - fq)
            out.append((p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1])))
    return out


def area(poly):
    if len(poly) < 3:
        return 0.0
    s = 0.0
    for i in range(len(poly)):
        x0, y0 = poly[i]
        x1, y1 = poly[(i + 1) % len(poly)]
        s += x0 * y1 - x1 * y0
    return 0.5 * abs(s)


def square(cx, cy, h):
    return [(cx - h / 2, cy - h / 2), (cx + h / 2, cy - h / 2), (cx + h / 2, cy + h / 2),
            (cx - h / 2, cy + h / 2)]


def clip_convex(poly, convex):
    """Intersect `poly` with a convex polygon given by its vertices (any winding)."""
    v = np.asarray(convex, dtype=float)
    s = 0.0
    for i in range(len(v)):
        s += v[i, 0] * v[(i + 1) % len(v), 1] - v[(i + 1) % len(v), 0] * v[i, 1]
    ccw = s > 0
    out = list(poly)
    for i in range(len(v)):
        p, q = v[i], v[(i + 1) % len(v)]
        ex, ey = q[0] - p[0], q[1] - p[1]
        # inside is to the left of p->q for ccw polygons: cross(e, r - p) >= 0
        if ccw:
            a, b = ey, -ex
        else:
            a, b = -ey, ex
        c = a * p[0] + b * p[1]
        out = clip_halfplane(out, a, b, c)
        if not out:
            break
    return out


def cell_fraction(convex, cx, cy, h):
    return area(clip_convex(square(cx, cy, h), convex)) / (h * h)
