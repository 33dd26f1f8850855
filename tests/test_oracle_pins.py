"""Pins of the FP64 oracle against what arXiv 2311.05646 and geometry fix.

No test here compares the oracle with itself or retypes one of its formulas:
each check uses an independent algorithm (polygon clipping, lattice
supersampling, brute-force finite differences), a closed form printed in the
paper, the paper's truth table, or an invariant of the mathematics.
"""
import math

import numpy as np
import pytest

from paper_2311_05646_gb300 import inputs as I
from paper_2311_05646_gb300.inputs import P

from . import _geom as G

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _grid2d(nx, ny, h=1.0, off=(0.5, 0.5, 0.0), logic="product", eps=(1.0, 2.0)):
    return I.Design((nx, ny, 1), (h, h, h), ncomp=1, off=[list(off)], eps_bg=eps[0],
                    eps_fg=eps[1], logic=logic)


def _centres(desc):
    g = desc["grid"]
    nx, ny, nz = g["n"]
    off = g["off"][0]
    xs = g["o"][0] + (np.arange(nx) + off[0]) * g["d"][0]
    ys = g["o"][1] + (np.arange(ny) + off[1]) * g["d"][1]
    return xs, ys


# ---------------------------------------------------------------- P1 --------
def test_p1_box_exact_on_lattice_supersampling(oracle_mod):
    """Cuboid fill equals the exact volume average (Sec. 5.1, zero-error claim
    of Sec. 5.2).  Edges on a 1/16-cell lattice make 16-point-per-axis midpoint
    supersampling exact, an algorithm independent of the overlap formula."""
    O = oracle_mod
    rng = np.random.default_rng(1)
    for trial in range(20):
        D = I.Design((7, 5, 4), (1.0, 1.0, 1.0), ncomp=3)
        lo = rng.integers(0, 48, size=3) / 16.0
        ext = rng.integers(1, 64, size=3) / 16.0
        D.box(x=(lo[0], lo[0] + ext[0]), y=(lo[1], lo[1] + ext[1]), z=(lo[2], lo[2] + ext[2]))
        desc = D.to_desc()
        f = O.fill(desc)
        N = 16
        sub = (np.arange(N) + 0.5) / N - 0.5
        for c in range(3):
            off = desc["grid"]["off"][c]
            for k in range(4):
                for j in range(5):
                    for i in range(7):
                        cx, cy, cz = i + off[0], j + off[1], k + off[2]
                        ix = ((cx + sub >= lo[0]) & (cx + sub <= lo[0] + ext[0])).mean()
                        iy = ((cy + sub >= lo[1]) & (cy + sub <= lo[1] + ext[1])).mean()
                        iz = ((cz + sub >= lo[2]) & (cz + sub <= lo[2] + ext[2])).mean()
                        assert abs(f[c, k, j, i] - ix * iy * iz) <= 1e-14


def test_p1_box_exact_by_clipping_random_edges(oracle_mod):
    """2D cuboids with arbitrary edges against exact square clipping."""
    O = oracle_mod
    rng = np.random.default_rng(2)
    for trial in range(30):
        h = float(rng.uniform(0.5, 2.0))
        D = _grid2d(9, 7, h)
        x0, y0 = rng.uniform(0, 4 * h), rng.uniform(0, 3 * h)
        x1, y1 = x0 + rng.uniform(0.1, 5) * h, y0 + rng.uniform(0.1, 4) * h
        D.box(x=(x0, x1), y=(y0, y1))
        desc = D.to_desc()
        f = O.fill(desc)[0, 0]
        xs, ys = _centres(desc)
        rect = [(x0, y0), (x1, y0), (x1, y1), (x0, y1)]
        for j, cy in enumerate(ys):
            for i, cx in enumerate(xs):
                assert abs(f[j, i] - G.cell_fraction(rect, cx, cy, h)) <= 1e-12


def test_p1_supersampling_converges_first_order(oracle_mod):
    """Quadrature with N sub-samples converges to the oracle's fill as O(1/N)
    (Sec. 5.2: exact averaging is the many-sample limit)."""
    O = oracle_mod
    D = _grid2d(6, 6)
    D.box(x=(1.2345, 4.6789), y=(0.777, 3.3333))
    desc = D.to_desc()
    f = O.fill(desc)[0, 0]
    xs, ys = _centres(desc)
    errs = []
    for N in (8, 32, 128, 512):
        sub = (np.arange(N) + 0.5) / N - 0.5
        e = 0.0
        for j, cy in enumerate(ys):
            for i, cx in enumerate(xs):
                ix = ((cx + sub >= 1.2345) & (cx + sub <= 4.6789)).mean()
                iy = ((cy + sub >= 0.777) & (cy + sub <= 3.3333)).mean()
                e = max(e, abs(ix * iy - f[j, i]))
        errs.append(e)
        assert e <= 2.0 / N
    assert errs[-1] < errs[0] / 16


# ---------------------------------------------------------------- P2 --------
def test_p2_linear_sigma_rect_is_eq_linear(oracle_mod):
    """Paper-form Rect1D with linear sigma and k = 1/dx reproduces Eq. linear,
    a_o = x/dx + 1/2 for an axis-parallel edge, x the signed distance."""
    O = oracle_mod
    h = 0.08
    for a in (0.0123, 0.1, 0.2777, 0.333):
        D = _grid2d(12, 1, h)
        D.box(x=(a, 10.0), mode="sigma", sigma="linear", kr=1.0)
        desc = D.to_desc()
        f = O.fill(desc)[0, 0, 0]
        xs, _ = _centres(desc)
        for i, cx in enumerate(xs):
            x = cx - a
            if -0.5 <= x / h <= 0.5:
                assert abs(f[i] - (x / h + 0.5)) <= 1e-13
            else:
                assert f[i] == (1.0 if x > 0 else 0.0)


def test_p2_rect_forms_agree_for_wide_boxes_and_differ_for_thin(oracle_mod):
    """The sigma-product Rect and the exact overlap agree whenever the box is
    at least one cell wide; a 0.2-cell bar centred in a cell gives 0.36 vs 0.2."""
    O = oracle_mod
    rng = np.random.default_rng(3)
    for _ in range(20):
        D1, D2 = _grid2d(10, 8), _grid2d(10, 8)
        x0, y0 = rng.uniform(0, 4), rng.uniform(0, 3)
        x1, y1 = x0 + rng.uniform(1.0, 5), y0 + rng.uniform(1.0, 4)
        D1.box(x=(x0, x1), y=(y0, y1), mode="exact")
        D2.box(x=(x0, x1), y=(y0, y1), mode="sigma", sigma="linear", kr=1.0)
        assert np.abs(O.fill(D1.to_desc()) - O.fill(D2.to_desc())).max() <= 1e-13
    D1, D2 = _grid2d(3, 1), _grid2d(3, 1)
    D1.box(x=(1.4, 1.6), mode="exact")
    D2.box(x=(1.4, 1.6), mode="sigma", sigma="linear", kr=1.0)
    assert abs(O.fill(D1.to_desc())[0, 0, 0, 1] - 0.2) < 1e-12
    assert abs(O.fill(D2.to_desc())[0, 0, 0, 1] - 0.36) < 1e-12


# ---------------------------------------------------------------- P3 --------
def _diamond(R, cx=0.0, cy=0.0):
    return [(cx + R, cy), (cx, cy + R), (cx - R, cy), (cx, cy - R)]


def _edges_cutting(poly, cx, cy, h):
    """How many polygon edge lines cross a cell that the polygon partly covers
    (brute force: sign change of each edge's line function over the cell's
    corners; 0 for cells the polygon misses or covers)."""
    sq = G.square(cx, cy, h)
    a = G.cell_fraction(poly, cx, cy, h)
    if not (0.0 < a < 1.0):
        return 0
    n = 0
    for i in range(len(poly)):
        p, q = np.array(poly[i]), np.array(poly[(i + 1) % len(poly)])
        e = q - p
        vals = [e[0] * (y - p[1]) - e[1] * (x - p[0]) for x, y in sq]
        if min(vals) < 0 < max(vals):
            n += 1
    return n


def test_p3_quadratic_sigma_exact_for_45_degree_edges(oracle_mod):
    """Quadratic sigma with k = 1/dx gives the exact area of a cell cut by one
    45-degree edge (Eq. quadratic; Sec. 5.2).  Checked against clipping."""
    O = oracle_mod
    h = 0.08
    R = 0.61
    D = _grid2d(24, 24, h, logic="product")
    D.grid["o"] = (-12 * h, -12 * h, 0.0)
    verts = _diamond(R, 0.0123, -0.0071)
    D.polygon(verts, sigma="quadratic", kr=1.0)
    desc = D.to_desc()
    f = O.fill(desc)[0, 0]
    xs, ys = _centres(desc)
    checked = 0
    for j, cy in enumerate(ys):
        for i, cx in enumerate(xs):
            if _edges_cutting(verts, cx, cy, h) == 1:
                assert abs(f[j, i] - G.cell_fraction(verts, cx, cy, h)) <= 1e-12
                checked += 1
    assert checked > 20


def test_p3_linear_sigma_axis_aligned_polygon_is_exact(oracle_mod):
    """An axis-aligned rectangle as a Poly2D with linear sigma, k = 1/dx: the
    product of edge factors is the exact area in every cell (Eq. linear)."""
    O = oracle_mod
    h = 0.5
    D = _grid2d(14, 12, h)
    rect = [(1.13, 0.87), (5.41, 0.87), (5.41, 4.02), (1.13, 4.02)]
    D.polygon(rect, sigma="linear", kr=1.0)
    desc = D.to_desc()
    f = O.fill(desc)[0, 0]
    xs, ys = _centres(desc)
    for j, cy in enumerate(ys):
        for i, cx in enumerate(xs):
            assert abs(f[j, i] - G.cell_fraction(rect, cx, cy, h)) <= 1e-12


# ---------------------------------------------------------------- P4 --------
def _dfill_dp(O, desc, flat_cell):
    G_ = np.zeros(I.field_shape(desc), dtype=np.float32)
    G_.reshape(-1)[flat_cell] = 1.0
    g = O.grad_real(desc, G_)
    return g / (desc["eps_fg"] - desc["eps_bg"])


def test_p4_edge_derivative_eq_dlinear(oracle_mod):
    """d a_o / dx = 1/dx for an axis-parallel edge (Eq. dlinear)."""
    O = oracle_mod
    h = 0.25
    D = _grid2d(8, 1, h)
    p = D.param(0.93)
    D.box(x=(I.P(p), 5.0))
    desc = D.to_desc()
    # the cell whose window [i h, (i+1) h] contains 0.93 is i = 3
    d = _dfill_dp(O, desc, 3)
    assert abs(d[0] - (-1.0 / h)) <= 1e-12  # moving the left edge right removes material
    for i in (0, 1, 2, 4, 5):
        assert _dfill_dp(O, desc, i)[0] == 0.0


def test_p4_45_degree_derivative_eq_dquadratic(oracle_mod):
    """Translating a 45-degree edge: d fill / dt equals Eq. dquadratic times the
    normal's x component, and the numerical derivative of the clipped area."""
    O = oracle_mod
    h = 0.08
    D = _grid2d(24, 24, h)
    D.grid["o"] = (-12 * h, -12 * h, 0.0)
    t = D.param(0.0)
    R = 0.61
    base = _diamond(R, 0.0123, -0.0071)
    D.polygon([(I.P(t, vx), vy) for vx, vy in base], sigma="quadratic", kr=1.0)
    desc = D.to_desc()
    xs, ys = _centres(desc)
    checked = 0
    for j, cy in enumerate(ys):
        for i, cx in enumerate(xs):
            if _edges_cutting(base, cx, cy, h) != 1:
                continue
            # the one edge: find its inward unit normal and signed distance
            best = None
            for e in range(4):
                p, q = np.array(base[e]), np.array(base[(e + 1) % 4])
                ev = q - p
                n_in = np.array([-ev[1], ev[0]]) / np.linalg.norm(ev)  # ccw diamond
                dist = n_in @ (np.array([cx, cy]) - p)
                if best is None or abs(dist) < abs(best[1]):
                    best = (n_in, dist)
            n_in, x = best
            if abs(x / h) < 1e-6:
                continue
            dq = (math.sqrt(2) * h + 2 * x) / h ** 2 if x < 0 else (math.sqrt(2) * h - 2 * x) / h ** 2
            expect = dq * (-n_in[0])  # shifting the shape by +t moves the edge by n_x t
            got = _dfill_dp(O, desc, j * 24 + i)[0]
            assert abs(got - expect) <= 1e-9 * max(1.0, abs(expect))
            eps_ = 1e-7
            fd = (G.cell_fraction([(vx + eps_, vy) for vx, vy in base], cx, cy, h)
                  - G.cell_fraction([(vx - eps_, vy) for vx, vy in base], cx, cy, h)) / (2 * eps_)
            assert abs(got - fd) <= 1e-5 * max(1.0, abs(fd))
            checked += 1
    assert checked > 20


# ---------------------------------------------------------------- P5 --------
def _truth_table():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "union_truth_table.txt")
    rows = []
    for line in open(path):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(tuple(int(v) for v in line.split()))
    return rows


@pytest.mark.parametrize("logic", ["product", "clamp"])
def test_p5_logic_on_binary_inputs(oracle_mod, logic):
    """On binary inputs the union reproduces logical OR (Table 'Logical union
    truth table'), intersection AND, difference AND-NOT, in both families."""
    O = oracle_mod
    table = _truth_table()
    assert len(table) == 4

    def run(prog):
        D = _grid2d(2, 2, 1.0, logic=logic)
        a = D.box(x=(0.0, 1.0))   # cells (i=0, j=*)
        b = D.box(y=(0.0, 1.0))   # cells (i=*, j=0)
        D.set_program(prog(a, b))
        return O.fill(D.to_desc())[0, 0]

    fu = run(lambda a, b: ("union", a, b))
    fi = run(lambda a, b: ("intersect", a, b))
    fd = run(lambda a, b: ("diff", a, b))
    for b1, b2, orv in table:
        # (a, b) = (b1, b2) at cell i = 1 - b1, j = 1 - b2
        i, j = 1 - b1, 1 - b2
        assert fu[j, i] == orv
        assert fi[j, i] == (b1 & b2)
        assert fd[j, i] == (b1 & (1 - b2))


def test_p5_half_half_union(oracle_mod):
    """Two shapes sharing a boundary inside a cell (0.5, 0.5): the clamped union
    gives 1 (Appendix B.2), the product form 0.75."""
    O = oracle_mod
    out = {}
    for logic in ("product", "clamp"):
        D = _grid2d(1, 1, 1.0, logic=logic)
        a = D.box(x=(-1.0, 0.5))
        b = D.box(x=(0.5, 2.0))
        D.set_program(("union", a, b))
        out[logic] = O.fill(D.to_desc())[0, 0, 0, 0]
    assert out["clamp"] == 1.0
    assert abs(out["product"] - 0.75) < 1e-15


def _lattice_pairs():
    # values on the 1/16 lattice: products and sums of them are exact in FP64
    return [(a / 16.0, b / 16.0) for a in (1, 3, 6, 11, 13, 15) for b in (2, 5, 8, 9, 14)]


@pytest.mark.parametrize("logic", ["product", "clamp"])
def test_p5_logic_on_fractional_inputs(oracle_mod, logic):
    """Away from {0, 1} the two families differ, and each must take its own
    closed form (App. B.2 for the product family; Eqs. union / intersection
    for the clamped one; difference = intersection(a, 1 - b)).  Box A covers
    the window [0, 1] of the single sample by a fraction a along x, box B by b
    along y, box C by c along x again: each leaf value is exact, so so is the
    expected result.  The three-input forms fix the n-ary definitions too."""
    O = oracle_mod

    def run(prog, a, b, c=0.5):
        D = _grid2d(1, 1, 1.0, logic=logic)
        A = D.box(x=(-1.0, a))
        B = D.box(y=(1.0 - b, 2.0))
        C = D.box(x=(1.0 - c, 3.0))
        D.set_program(prog(A, B, C))
        return O.fill(D.to_desc())[0, 0, 0, 0]

    for a, b in _lattice_pairs():
        c = (a + b) / 2.0 if (a + b) < 1.0 else 0.5
        fi = run(lambda A, B, C: ("intersect", A, B), a, b)
        fd = run(lambda A, B, C: ("diff", A, B), a, b)
        fu = run(lambda A, B, C: ("union", A, B), a, b)
        fi3 = run(lambda A, B, C: ("intersect", A, B, C), a, b, c)
        fu3 = run(lambda A, B, C: ("union", A, B, C), a, b, c)
        if logic == "product":
            want = (a * b, a * (1.0 - b), a + b - a * b, a * b * c,
                    1.0 - (1.0 - a) * (1.0 - b) * (1.0 - c))
        else:
            want = (max(0.0, a + b - 1.0), max(0.0, a - b), min(1.0, a + b),
                    max(2.0, a + b + c) - 2.0, min(1.0, a + b + c))
        got = (fi, fd, fu, fi3, fu3)
        for g_, w_ in zip(got, want):
            assert abs(g_ - w_) <= 1e-15, (logic, a, b, c, got, want)


# ---------------------------------------------------------------- P6 --------
KINKS = {0: [-0.5, 0.5], 1: [], 2: [-1 / math.sqrt(2), 0.0, 1 / math.sqrt(2)],
         3: [-math.pi / 2, math.pi / 2], 4: []}


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_p6_sigma_table_properties(oracle_mod, kind):
    """Table 'Nonlinear function definitions': sigma(0) = 1/2, [0,1]-bounded,
    monotone, sigma(-u) = 1 - sigma(u), and d sigma/du equals a central
    finite difference of sigma away from kinks."""
    O = oracle_mod
    assert abs(O.sigma(kind, 0.0)[0] - 0.5) < 1e-15
    us = np.linspace(-6, 6, 2401)
    vals = np.array([O.sigma(kind, u)[0] for u in us])
    assert vals.min() >= 0.0 and vals.max() <= 1.0
    assert np.all(np.diff(vals) >= -1e-15)
    for u in us[::7]:
        assert abs(O.sigma(kind, -u)[0] - (1.0 - O.sigma(kind, u)[0])) < 1e-14
        if any(abs(u - k) < 1e-4 for k in KINKS[kind]):
            continue
        hh = 1e-6
        fd = (O.sigma(kind, u + hh)[0] - O.sigma(kind, u - hh)[0]) / (2 * hh)
        assert abs(O.sigma(kind, u)[1] - fd) < 1e-7


def test_p6_sigma_saturation_points(oracle_mod):
    """Each piecewise function reaches exactly 0 and 1 at the ends of its
    transition (linear +-1/2, quadratic +-1/sqrt 2, sin +-pi/2)."""
    O = oracle_mod
    assert O.sigma(0, 0.5)[0] == 1.0 and O.sigma(0, -0.5)[0] == 0.0
    assert abs(O.sigma(2, 1 / math.sqrt(2))[0] - 1.0) < 1e-15
    assert abs(O.sigma(2, -1 / math.sqrt(2))[0]) < 1e-15
    assert abs(O.sigma(3, math.pi / 2)[0] - 1.0) < 1e-15 and O.sigma(3, -math.pi / 2)[0] == 0.0
    # the sigmoid's slope at 0 is 1/4 of the unit scale (so k/4 = 1/dx for k = 4/dx)
    assert abs(O.sigma(1, 0.0)[1] - 0.25) < 1e-15


def test_p6_erf_sigma_is_the_table_form(oracle_mod):
    """Table 'Nonlinear function definitions' prints erf(k, x) = (1 + Erf(k x))/2
    with Erf the error function (not the normal CDF (1 + Erf(u / sqrt 2))/2).
    Values against the standard library's erf; slope 1/sqrt(pi) at 0 (the
    error function's derivative 2/sqrt(pi) e^(-u^2), halved) and against
    central differences of math.erf elsewhere."""
    O = oracle_mod
    assert abs(O.sigma(4, 1.0)[0] - 0.5 * (1.0 + math.erf(1.0))) < 1e-15
    assert abs(O.sigma(4, 0.0)[1] - 1.0 / math.sqrt(math.pi)) < 1e-15
    hh = 1e-5
    for u in np.linspace(-3.0, 3.0, 61):
        u = float(u)
        assert abs(O.sigma(4, u)[0] - 0.5 * (1.0 + math.erf(u))) < 2e-16
        fd = 0.5 * (math.erf(u + hh) - math.erf(u - hh)) / (2 * hh)
        assert abs(O.sigma(4, u)[1] - fd) < 1e-9


def test_p6_erf_circle_uses_the_grid_scale(oracle_mod):
    """sigma_k(x) = sigma(k x) with k = kr / dx (Sec. 4): an erf circle of
    radius R at kr = 2 on a dx = 0.5 grid is (1 + Erf(4 (R - r)))/2 at every
    sample, r the sample's distance from the centre."""
    O = oracle_mod
    h, R, cx, cy = 0.5, 2.3, 3.1, 2.7
    D = _grid2d(13, 11, h)
    D.circle(cx, cy, R, sigma="erf", kr=2.0)
    desc = D.to_desc()
    f = O.fill(desc)[0, 0]
    xs, ys = _centres(desc)
    for j, y in enumerate(ys):
        for i, x in enumerate(xs):
            r = math.hypot(x - cx, y - cy)
            assert abs(f[j, i] - 0.5 * (1.0 + math.erf(4.0 * (R - r)))) < 1e-15


# ---------------------------------------------------------------- P7 --------
def test_p7_single_edge_gradient_closed_form(oracle_mod):
    """For one exact-overlap edge at x = a, dL/da = -(deps/dx) * sum over the
    cells whose window holds a of Re(w E_adj E) (Eq. 1 with Eq. dlinear)."""
    O = oracle_mod
    h = 20.0
    D = I.Design((30, 12, 1), (h, h, h), ncomp=1, eps_bg=2.085, eps_fg=12.11)
    pa = D.param(211.7)
    D.box(x=(I.P(pa), 480.3))
    desc = D.to_desc()
    ef = I.plane_wave_field(desc, 1)
    ea = I.plane_wave_field(desc, 2)
    w = np.complex64(0.3 - 1.7j)
    g = O.grad(desc, ef, ea, w)
    i = int(math.floor(211.7 / h - 0.5 + 0.5))  # window [ (i) h, (i+1) h ] with offset 0.5
    z = (w * ea[0, 0, :, i].astype(np.complex128) * ef[0, 0, :, i].astype(np.complex128)).real
    expect = -(desc["eps_fg"] - desc["eps_bg"]) / h * z.sum()
    assert abs(g[0] - expect) <= 1e-12 * abs(expect)


# ------------------------------------------------- GeneralCartesian2D ------
def _graph_case(above, rng):
    """A linear-sigma graph boundary with k = 1/dy on a dx != dy grid: knots
    at irregular, off-lattice x (some columns lie beyond the end knots), knot
    heights inside the grid with at least two cells of margin."""
    nx, ny, dx, dy = 40, 30, 1.0, 0.5
    D = I.Design((nx, ny, 1), (dx, dy, 1.0), ncomp=1, eps_bg=0.0, eps_fg=1.0)
    M = 7
    X = np.sort(rng.uniform(4.0, 36.0, size=M)) + 0.137
    Y = rng.uniform(1.5, 13.5, size=M)
    ids = [D.param(float(v)) for v in Y]
    D.graph([float(v) for v in X], [P(i) for i in ids], above=above, sigma="linear", kr=1.0)
    return D.to_desc(), X, Y, dy, ny


@pytest.mark.parametrize("above", [False, True])
def test_graph_column_sums_follow_the_interpolant(oracle_mod, above):
    """GeneralCartesian2D (Table 4; Eq. taper_eps of Sec. 6.2) is
    sigma_k(+-(f(x) - y)), f the piecewise-linear curve through the knots,
    constant beyond the end knots.  With the linear sigma and k = 1/dy each
    cell holds exactly the covered fraction of its y window (Eq. linear), so
    the fill of a column sums to (f(x_i) - y_lo)/dy, or (y_hi - f(x_i))/dy for
    the region above, and each cell is the covered fraction of its y window.
    f(x_i) comes from numpy's interp, an independent implementation of the
    same curve.  The derivatives of that column sum
    w.r.t. the knot heights are numpy's hat weights over dy (interp of a unit
    vector), taken from the oracle's reverse sweep with a one-column cotangent."""
    O = oracle_mod
    rng = np.random.default_rng(17 + int(above))
    desc, X, Y, dy, ny = _graph_case(above, rng)
    f = O.fill(desc)[0, 0]
    xs, _ = _centres(desc)
    fx = np.interp(xs, X, Y)
    want = (ny * dy - fx) / dy if above else fx / dy
    assert np.abs(f.sum(axis=0) - want).max() <= 1e-12
    # cell by cell: the covered fraction of each y window [j dy, (j + 1) dy]
    lo = np.arange(ny)[:, None] * dy
    cover = np.clip((fx[None, :] - lo) / dy, 0.0, 1.0)
    assert np.abs(f - ((1.0 - cover) if above else cover)).max() <= 1e-12
    nx = len(xs)
    sgn = -1.0 if above else 1.0
    for i in range(0, nx, 3):
        G = np.zeros((1, 1, ny, nx), dtype=np.float32)
        G[0, 0, :, i] = 1.0
        g = O.grad_real(desc, G)
        hat = np.array([np.interp(xs[i], X, np.eye(len(X))[j]) for j in range(len(X))])
        assert np.abs(g - sgn * hat / dy).max() <= 1e-12, (i, g, hat)


def test_graph_knot_position_derivatives_follow_the_interpolant(oracle_mod):
    """The same column sums as functions of the knots' x positions: their
    derivatives are central differences of numpy's interp (exact for a curve
    that is linear between knots, with every sample away from a knot)."""
    O = oracle_mod
    rng = np.random.default_rng(23)
    nx, ny, dx, dy = 40, 30, 1.0, 0.5
    D = I.Design((nx, ny, 1), (dx, dy, 1.0), ncomp=1, eps_bg=0.0, eps_fg=1.0)
    M = 6
    X = np.sort(rng.uniform(4.0, 36.0, size=M)) + 0.137
    Y = rng.uniform(1.5, 13.5, size=M)
    idx = [D.param(float(v)) for v in X]
    D.graph([P(i) for i in idx], [float(v) for v in Y], sigma="linear", kr=1.0)
    desc = D.to_desc()
    xs, _ = _centres(desc)
    hh = 1e-6
    for i in range(0, nx, 3):
        G = np.zeros((1, 1, ny, nx), dtype=np.float32)
        G[0, 0, :, i] = 1.0
        g = O.grad_real(desc, G)
        for j in range(M):
            Xp, Xm = X.copy(), X.copy()
            Xp[j] += hh
            Xm[j] -= hh
            fd = (np.interp(xs[i], Xp, Y) - np.interp(xs[i], Xm, Y)) / (2 * hh) / dy
            assert abs(g[j] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, j, g[j], fd)


# ----------------------------------------------- rotation / aspect ---------
# The paper notes that its primitives support rotation and aspect-ratio
# transforms (Sec. 4, item iii) without a formula; the reading pinned here: a
# primitive with transform (px, py, theta, sx, sy) is the untransformed one
# stretched by (sx, sy) along its own axes and rotated by theta about (px, py).
def _xbase(kind, xform=None, sigma="sigmoid", kr=4.0, D=None):
    D = D or _grid2d(40, 36, 1.0)
    if kind == "box":
        D.box(x=(P(D.param(12.3)), P(D.param(25.6))), y=(P(D.param(9.2)), P(D.param(20.7))),
              mode="sigma", sigma=sigma, kr=kr, xform=xform)
    elif kind == "circle":
        D.circle(P(D.param(19.4)), P(D.param(17.1)), P(D.param(7.3)), sigma=sigma, kr=kr,
                 xform=xform)
    elif kind == "polygon":
        verts = [(11.2, 10.1), (27.3, 12.4), (24.6, 25.2), (13.1, 22.8)]
        D.polygon([(P(D.param(x)), P(D.param(y))) for x, y in verts], sigma=sigma, kr=kr,
                  xform=xform)
    else:
        D.polar(P(D.param(19.6)), P(D.param(17.7)), P(D.param(7.1)),
                [(P(D.param(0.9)), P(D.param(-0.6))), (P(D.param(0.4)), P(D.param(0.2)))],
                sigma=sigma, kr=kr, xform=xform)
    return D


@pytest.mark.parametrize("kind", ["box", "circle", "polygon", "polar"])
def test_xform_identity_is_the_primitive(oracle_mod, kind):
    """theta = 0 and sx = sy = 1 leave the primitive as it is, at any pivot:
    fill and the derivatives w.r.t. its own scalars."""
    O = oracle_mod
    plain = _xbase(kind).to_desc()
    xd = _xbase(kind, xform=(7.7, 31.1, 0.0, 1.0, 1.0)).to_desc()
    assert np.abs(O.fill(xd) - O.fill(plain)).max() <= 1e-14
    ef, ea = I.plane_wave_field(plain, 3), I.plane_wave_field(plain, 4)
    w = I.seeded_w(1, 2)
    g0, g1 = O.grad(plain, ef, ea, w), O.grad(xd, ef, ea, w)
    assert np.abs(g1 - g0).max() <= 1e-12 * max(1.0, np.abs(g0).max())


@pytest.mark.parametrize("turn", [1, 2, 3])
def test_xform_quarter_turns_of_a_box(oracle_mod, turn):
    """A sigma-box [x0, x1] x [y0, y1] turned by a multiple of 90 degrees
    about a pivot is the untransformed box with the turned extents (the
    sigma product is symmetric in its two edges): counter-clockwise,
    (x, y) - p -> (-(y - py), x - px) per quarter turn."""
    O = oracle_mod
    x0, x1, y0, y1, px, py = 12.3, 25.6, 9.2, 20.7, 17.4, 16.1
    D = _grid2d(44, 40, 1.0)
    D.box(x=(x0, x1), y=(y0, y1), mode="sigma", sigma="sigmoid", kr=4.0,
          xform=(px, py, turn * math.pi / 2, 1.0, 1.0))
    corners = np.array([[x0, y0], [x1, y1]]) - [px, py]
    for _ in range(turn):
        corners = np.stack([-corners[:, 1], corners[:, 0]], axis=1)
    corners += [px, py]
    E = _grid2d(44, 40, 1.0)
    E.box(x=tuple(sorted(corners[:, 0])), y=tuple(sorted(corners[:, 1])), mode="sigma",
          sigma="sigmoid", kr=4.0)
    assert np.abs(O.fill(D.to_desc()) - O.fill(E.to_desc())).max() <= 1e-12


@pytest.mark.parametrize("axis", [0, 1])
def test_xform_aspect_stretches_about_the_pivot(oracle_mod, axis):
    """Aspect s along one local axis (theta = 0): a box bounded only along
    that axis, [a, b], becomes [p + s (a - p), p + s (b - p)] with its sigma
    transition s times wider, i.e. the untransformed box with those edges and
    kr / s.  A box bounded along the other axis is untouched."""
    O = oracle_mod
    a, b, pv, sc, kr = 8.3, 17.9, 11.2, 2.5, 1.0
    xf = (pv, 0.0, 0.0, sc, 1.0) if axis == 0 else (0.0, pv, 0.0, 1.0, sc)
    D = _grid2d(60, 60, 1.0)
    kw = {"x": (a, b)} if axis == 0 else {"y": (a, b)}
    D.box(mode="sigma", sigma="linear", kr=kr, xform=xf, **kw)
    E = _grid2d(60, 60, 1.0)
    kw2 = {("x" if axis == 0 else "y"): (pv + sc * (a - pv), pv + sc * (b - pv))}
    E.box(mode="sigma", sigma="linear", kr=kr / sc, **kw2)
    assert np.abs(O.fill(D.to_desc()) - O.fill(E.to_desc())).max() <= 1e-12
    F = _grid2d(60, 60, 1.0)
    kw3 = {("y" if axis == 0 else "x"): (a, b)}
    F.box(mode="sigma", sigma="linear", kr=kr, xform=xf, **kw3)
    G_ = _grid2d(60, 60, 1.0)
    G_.box(mode="sigma", sigma="linear", kr=kr, **kw3)
    assert np.abs(O.fill(F.to_desc()) - O.fill(G_.to_desc())).max() <= 1e-12


def test_xform_45_degree_box_is_exact_with_the_quadratic_sigma(oracle_mod):
    """A square turned by 45 degrees with the quadratic sigma at k = 1/dx:
    every cell cut by one edge holds exactly the clipped area of the turned
    square (Eq. quadratic, Sec. 5.2), checked against polygon clipping."""
    O = oracle_mod
    h = 1.0
    px, py, half = 20.37, 19.81, 9.6
    D = _grid2d(40, 40, h)
    D.box(x=(px - half, px + half), y=(py - half, py + half), mode="sigma", sigma="quadratic",
          kr=1.0, xform=(px, py, math.pi / 4, 1.0, 1.0))
    desc = D.to_desc()
    f = O.fill(desc)[0, 0]
    c, s_ = math.cos(math.pi / 4), math.sin(math.pi / 4)
    verts = [(px + c * dx - s_ * dy, py + s_ * dx + c * dy)
             for dx, dy in ((-half, -half), (half, -half), (half, half), (-half, half))]
    xs, ys = _centres(desc)
    checked = 0
    for j, cy in enumerate(ys):
        for i, cx in enumerate(xs):
            if _edges_cutting(verts, cx, cy, h) == 1:
                assert abs(f[j, i] - G.cell_fraction(verts, cx, cy, h)) <= 1e-12
                checked += 1
    assert checked > 40


def test_xform_ellipse_area(oracle_mod):
    """A circle of radius R with aspect (sx, sy) is an ellipse: with the
    smooth sigmoid its fill sums (unit cells) to sx sy times the radial
    integral 2 pi int rho sigma(k (R - rho)) d rho, whatever the rotation and
    pivot.  The integral comes from scipy's quadrature and expit, the sum of
    a smooth profile over the lattice matches it to ~1e-6."""
    from scipy import integrate, special
    O = oracle_mod
    R, sx, sy, kr = 10.0, 2.2, 0.7, 1.0
    radial, _ = integrate.quad(lambda r: 2 * math.pi * r * special.expit(kr * (R - r)), 0.0, R + 60.0,
                               epsabs=1e-12, epsrel=1e-12, limit=200)
    want = sx * sy * radial
    for th, pv in ((0.3, (60.0, 59.0)), (1.1, (61.5, 57.2))):
        D = _grid2d(120, 120, 1.0)
        D.circle(60.3, 59.6, R, sigma="sigmoid", kr=kr, xform=(pv[0], pv[1], th, sx, sy))
        v = O.fill(D.to_desc()).sum()
        assert abs(v - want) <= 1e-5 * want, (v, want)


@pytest.mark.parametrize("kind", ["box", "circle", "polygon", "polar"])
def test_xform_gradient_matches_central_fd(oracle_mod, kind):
    """The reverse sweep through the transform -- the primitive's own scalars
    and the pivot, angle and aspect, each driven by a parameter -- equals
    central finite differences of L."""
    O = oracle_mod
    D = _grid2d(40, 36, 1.0)
    xf = (P(D.param(18.7)), P(D.param(16.2)), P(D.param(0.41)), P(D.param(1.3)), P(D.param(0.8)))
    D = _xbase(kind, xform=xf, D=D)
    desc = D.to_desc()
    ef, ea, w = _fields(desc, 7, 8)
    g = O.grad(desc, ef, ea, w)
    gfd = O.grad_fd(desc, ef, ea, w, 1e-5)
    assert np.linalg.norm(g - gfd) <= 1e-6 * np.linalg.norm(g) + 1e-9 * np.abs(g).max()
    assert np.abs(g[:5]).min() > 0  # every transform scalar moves the loss


# ---------------------------------------------------------------- P8 --------
def _fields(desc, s1, s2, wseed=5):
    return (I.plane_wave_field(desc, s1), I.plane_wave_field(desc, s2),
            I.seeded_w(desc["grid"]["ncomp"], wseed))


@pytest.mark.parametrize("case", ["grating2d", "grating3d", "taper", "random", "clamp", "polar"])
def test_p8_analytic_gradient_matches_central_fd(oracle_mod, case):
    """The reverse sweep (Eqs. AD/jaceps) equals brute-force central finite
    differences of L, the paper's baseline method, at h = 1e-3 nm."""
    O = oracle_mod
    if case == "grating2d":
        desc = I.grating_2d()
    elif case == "grating3d":
        desc = I.grating_3d(n=(48, 6, 24), teeth=3, pitch=300.0)
    elif case == "taper":
        desc = I.taper_3d(n=(60, 30, 12), nverts=8)
    elif case == "random":
        desc = I.random_design(7, n=(40, 30, 12), nprims=14)
    elif case == "polar":
        desc = I.psgc_lattice(n=(48, 40, 10), rows=2, cols=2, harmonics=3, centres=True)
    else:
        desc = I.grating_2d()
        desc["logic"] = "clamp"
    ef, ea, w = _fields(desc, 12, 13)
    g = O.grad(desc, ef, ea, w)
    gfd = O.grad_fd(desc, ef, ea, w, 1e-3)
    err = np.linalg.norm(g - gfd)
    assert err <= 1e-6 * np.linalg.norm(g) + 1e-9 * np.abs(g).max()


def test_p8_fd_converges_second_order(oracle_mod):
    """Central FD error against the analytic gradient falls as O(h^2) on a
    smooth (sigmoid) design."""
    O = oracle_mod
    desc = I.taper_3d(n=(60, 30, 12), nverts=6)
    ef, ea, w = _fields(desc, 32, 33)
    g = O.grad(desc, ef, ea, w)
    errs = []
    for h in (8.0, 4.0, 2.0):
        errs.append(np.linalg.norm(O.grad_fd(desc, ef, ea, w, h) - g))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.0 and 3.0 < r2 < 5.0


# ------------------------------------------------ both terms of Eq. 1 -------
@pytest.mark.parametrize("case", ["grating2d", "random3d"])
def test_eh_gradient_matches_fd_of_the_total_loss(oracle_mod, case):
    """Eq. 1 with both terms: L = Re sum w_e E_adj E eps + Re sum w_h H_adj H
    mu, eps and mu two compositions (Eqs. eps, mu) of the same parameters
    sampled at the E and H offsets.  Central differences of L itself (loss
    evaluations only, no reverse sweep) fix the sum of the two sweeps."""
    O = oracle_mod
    desc = I.grating_2d() if case == "grating2d" else I.random_design(5, n=(30, 24, 10), nprims=10)
    dmu = I.mu_design(desc, mu_bg=1.0, mu_fg=1.7)
    ef, ea, we = _fields(desc, 41, 42, 43)
    hf, ha, wh = _fields(dmu, 44, 45, 46)
    g = O.grad_eh(desc, dmu, ef, ea, we, hf, ha, wh)
    p0 = np.asarray(desc["params"], dtype=np.float64)
    h = 1e-3
    fd = np.zeros_like(p0)
    for k in range(p0.size):
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        Lp = O.loss(desc, ef, ea, we, pp) + O.loss(dmu, hf, ha, wh, pp)
        Lm = O.loss(desc, ef, ea, we, pm) + O.loss(dmu, hf, ha, wh, pm)
        fd[k] = (Lp - Lm) / (2 * h)
    assert np.linalg.norm(g - fd) <= 1e-6 * np.linalg.norm(g) + 1e-9 * np.abs(g).max()
    # the H term is really there: it moves the gradient
    g_e = O.grad(desc, ef, ea, we)
    assert np.linalg.norm(g - g_e) > 1e-3 * np.linalg.norm(g_e)


def test_eh_gradient_of_a_nonmagnetic_design_is_the_eps_term(oracle_mod):
    """mu_fg = mu_bg: mu does not depend on the parameters, so Eq. 1's H term
    vanishes identically (every d mu / dp is a multiple of mu_fg - mu_bg)."""
    O = oracle_mod
    desc = I.random_design(9, n=(30, 24, 10), nprims=10)
    dmu = I.mu_design(desc, mu_bg=1.0, mu_fg=1.0)
    ef, ea, we = _fields(desc, 51, 52, 53)
    hf, ha, wh = _fields(dmu, 54, 55, 56)
    assert np.array_equal(O.grad_eh(desc, dmu, ef, ea, we, hf, ha, wh), O.grad(desc, ef, ea, we))


# ------------------------------------------------------------ Polar2D ------
def test_polar_without_harmonics_is_the_circle(oracle_mod):
    """Polar2D with R(theta) = R0 (no harmonics) is Circ2D (Table 4): same
    fill and same gradient, for every sigma kind."""
    O = oracle_mod
    for sk in ("linear", "sigmoid", "sin"):
        a = I.Design((40, 36, 1), (10.0, 10.0, 10.0), ncomp=1)
        b = I.Design((40, 36, 1), (10.0, 10.0, 10.0), ncomp=1)
        for D in (a, b):
            ix, iy, ir = D.param(191.3), D.param(173.8), D.param(97.6)
        a.circle(P(ix), P(iy), P(ir), sigma=sk, kr=2.0)
        b.polar(P(ix), P(iy), P(ir), (), sigma=sk, kr=2.0)
        da, db = a.to_desc(), b.to_desc()
        assert np.array_equal(O.fill(da), O.fill(db))
        ef, ea, w = _fields(da, 61, 62, 63)
        assert np.allclose(O.grad(da, ef, ea, w), O.grad(db, ef, ea, w), rtol=1e-13, atol=0)


@pytest.mark.parametrize("phase", ["cos", "sin"])
def test_polar_table_example_lobes(oracle_mod, phase):
    """Table 4's Polar2D example, R(1 + delta cos(alpha theta)) with alpha = 4,
    delta = 0.2: four lobes of radius R(1 + delta) on the axes and waists of
    R(1 - delta) on the diagonals (with sin, all turned by pi/8).  A sharp
    sigmoid puts samples just inside / outside those radii at ~1 / ~0."""
    O = oracle_mod
    R, delta, h = 50.0, 0.2, 1.0
    D = I.Design((200, 200, 1), (h, h, h), ncomp=1, off=[[0.0, 0.0, 0.0]])
    c = (D.param(100.0), D.param(100.0))
    coef = [(0.0, 0.0)] * 3 + ([(R * delta, 0.0)] if phase == "cos" else [(0.0, R * delta)])
    D.polar(P(c[0]), P(c[1]), R, coef, sigma="sigmoid", kr=200.0)
    f = O.fill(D.to_desc())[0, 0]
    rot = 0.0 if phase == "cos" else np.pi / 8
    for k in range(8):
        th = rot + k * np.pi / 4
        Rt = R * (1 + delta) if k % 2 == 0 else R * (1 - delta)
        for rr, want in ((Rt - 1.5, 1.0), (Rt + 1.5, 0.0)):
            x, y = 100.0 + rr * np.cos(th), 100.0 + rr * np.sin(th)
            i, j = int(round(x)), int(round(y))
            # the sample nearest the point: its radius differs by < 0.71 cells
            assert abs(f[j, i] - want) < 1e-6, (phase, k, rr, f[j, i])


def test_polar_area_of_the_fourier_boundary(oracle_mod):
    """The area inside r < R(theta) is the integral of R(theta)^2 / 2:
    pi R0^2 + (pi / 2) sum_n (c_n^2 + s_n^2).  With the linear sigma at k = 1
    / dx the fill sums to it up to the boundary's curvature (< 0.2% here)."""
    O = oracle_mod
    D = I.Design((160, 160, 1), (1.0, 1.0, 1.0), ncomp=1)
    D.param(0.0)
    coef = [(3.0, -2.0), (0.0, 4.5), (2.5, 1.0)]
    D.polar(80.3, 79.6, 50.0, coef, sigma="linear", kr=1.0)
    f = O.fill(D.to_desc())
    want = np.pi * 50.0 ** 2 + 0.5 * np.pi * sum(a * a + b * b for a, b in coef)
    assert abs(f.sum() - want) < 2e-3 * want


def _table4():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table4_examples.txt")
    out = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        name, *kv = line.split()
        out[name] = {k: [float(v) for v in val.split(",")] if "," in val else float(val)
                     for k, val in (t.split("=") for t in kv)}
    return out


@pytest.mark.parametrize("name", ["Rect2D", "Poly2D", "Circ2D", "Polar2D"])
def test_table4_examples_have_their_closed_form_areas(oracle_mod, name):
    """Table 4's printed examples, built on [-1, 1]^2 at dx = 0.005 with the
    linear sigma at k = 1 / dx: the fills add up to each shape's area
    (rectangle exactly; the paper's clockwise triangle, whose area is its
    shoelace value in either winding; the circle; Polar2D with
    R(theta) = R (1 + delta cos(alpha theta)), area pi R^2 (1 + delta^2 / 2))."""
    O = oracle_mod
    ex = _table4()[name]
    h, n = 0.005, 400
    D = I.Design((n, n, 1), (h, h, h), o=(-1.0, -1.0, 0.0), ncomp=1, off=[[0.5, 0.5, 0.0]])
    D.param(0.0)
    if name == "Rect2D":
        D.box(x=(ex["x0"], ex["x1"]), y=(ex["y0"], ex["y1"]))
        want, tol = (ex["x1"] - ex["x0"]) * (ex["y1"] - ex["y0"]), 1e-12
    elif name == "Poly2D":
        verts = list(zip(ex["x"], ex["y"]))
        D.polygon(verts, sigma="linear", kr=1.0)
        want, tol = G.area(verts), 2e-4
        signed = 0.5 * sum(x0 * y1 - x1 * y0 for (x0, y0), (x1, y1) in zip(verts, verts[1:] + verts[:1]))
        assert signed < 0  # the printed example winds clockwise
    elif name == "Circ2D":
        D.circle(ex["x0"], ex["y0"], ex["R"], sigma="linear", kr=1.0)
        want, tol = np.pi * ex["R"] ** 2, 2e-4
    else:
        R, dl, a = ex["R"], ex["delta"], int(ex["alpha"])
        coef = [(0.0, 0.0)] * (a - 1) + [(R * dl, 0.0)]
        D.polar(ex["x0"], ex["y0"], R, coef, sigma="linear", kr=1.0)
        want, tol = np.pi * R * R * (1 + 0.5 * dl * dl), 2e-4
    got = O.fill(D.to_desc()).sum() * h * h
    assert abs(got - want) <= tol * want, (got, want)


# ------------------------------------- non-binary union (App. B, Alg. 1) ----
@pytest.mark.parametrize("logic", ["product", "clamp"])
@pytest.mark.parametrize("dims", ["2d", "3d"])
def test_levels_gradient_matches_fd_of_the_loss(logic, dims):
    """The reverse of Alg. 1 (one cotangent per set, each set's sweep) equals
    central differences of the loss of Alg. 1's forward result."""
    from oracle import levels as LV
    if dims == "2d":
        m = I.nonbinary_circles(n=(90, 80, 1), d=(40.0, 40.0, 40.0), logic=logic, per_level=2)
    else:
        m = I.nonbinary_circles(n=(40, 36, 10), d=(80.0, 80.0, 40.0), logic=logic, per_level=2,
                                levels=(0.5, 1.3, 2.0))
    sets, lv, eb = m["sets"], m["levels"], m["eps_bg"]
    ef, ea, w = _fields(sets[0], 71, 72, 73)
    g = LV.grad(sets, lv, ef, ea, w)
    p0 = np.asarray(sets[0]["params"], dtype=np.float64)
    h = 1e-3
    fd = np.zeros_like(p0)
    for k in range(p0.size):
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        fd[k] = (LV.loss(sets, lv, eb, ef, ea, w, pp) - LV.loss(sets, lv, eb, ef, ea, w, pm)) / (2 * h)
    # the set cotangents pass through float32 (6e-8 relative) on their way in
    assert np.linalg.norm(g - fd) <= 1e-5 * np.linalg.norm(g) + 1e-9 * np.abs(g).max()
    assert np.abs(g).max() > 0


def test_levels_one_set_is_the_binary_design():
    """K = 1: Alg. 1 returns eps_bg + eps^1 s^1, the two-level map of Sec. 5.1."""
    from oracle import levels as LV
    from oracle import oracle as O
    m = I.nonbinary_circles(levels=(0.7,), eps_bg=1.5)
    desc = dict(m["sets"][0])
    desc["eps_bg"], desc["eps_fg"] = 1.5, 1.5 + 0.7
    assert np.allclose(LV.eps(m["sets"], m["levels"], 1.5), O.eps(desc), rtol=0, atol=1e-15)


def test_levels_product_closed_form():
    """Unrolling Alg. 1 with the product union gives front-to-back compositing:
    eps - eps_bg = sum_k eps^k s^k prod_{j > k} (1 - s^j)."""
    from oracle import levels as LV
    from oracle import oracle as O
    m = I.nonbinary_circles(n=(120, 100, 1), d=(30.0, 30.0, 30.0), logic="product")
    S = [O.fill(d) for d in m["sets"]]
    lv = m["levels"]
    want = np.zeros_like(S[0])
    for k in range(len(S)):
        term = lv[k] * S[k]
        for j in range(k + 1, len(S)):
            term = term * (1.0 - S[j])
        want += term
    got = LV.eps(m["sets"], lv, m["eps_bg"]) - m["eps_bg"]
    assert np.abs(got - want).max() <= 1e-14
    assert np.abs(want).max() > 0.9


@pytest.mark.parametrize("logic", ["product", "clamp"])
def test_levels_highest_covering_level_wins(logic):
    """App. B: the algorithm gives priority to the set with the largest level.
    Lattice-aligned boxes (exact 0 / 1 fills) of four levels, overlapping in a
    staircase: every cell takes the largest level among the boxes covering it,
    and the background where none does."""
    from oracle import levels as LV
    lv = np.array([0.1, 0.34, 0.62, 1.0])
    nx, ny = 24, 20
    sets, cover = [], np.zeros((len(lv), ny, nx), dtype=bool)
    for k in range(len(lv)):
        D = I.Design((nx, ny, 1), (1.0, 1.0, 1.0), ncomp=1, off=[[0.5, 0.5, 0.0]], eps_bg=0.0,
                     eps_fg=1.0, logic=logic)
        x0, y0 = 2 + 4 * k, 1 + 3 * k
        D.param(0.0)
        D.box(x=(float(x0), float(x0 + 9)), y=(float(y0), float(y0 + 8)), sigma="linear")
        sets.append(D.to_desc())
        cover[k, y0:y0 + 8, x0:x0 + 9] = True
    e = LV.eps(sets, lv, 2.0)[0, 0]
    want = np.full((ny, nx), 2.0)
    for k in range(len(lv)):
        want[cover[k]] = 2.0 + lv[k]
    assert np.abs(e - want).max() <= 1e-15


@pytest.mark.parametrize("logic", ["product", "clamp"])
def test_levels_equal_levels_are_the_binary_union(logic):
    """eps^1 = ... = eps^K: Alg. 1 is the plain union of all sets (Eq. union or
    its product form) at that one level."""
    from oracle import levels as LV
    from oracle import oracle as O
    m = I.nonbinary_circles(n=(100, 90, 1), d=(40.0, 40.0, 40.0), levels=(0.8, 0.8, 0.8, 0.8),
                            logic=logic)
    sets = m["sets"]
    D = I.Design((100, 90, 1), (40.0, 40.0, 40.0), ncomp=1, eps_bg=0.0, eps_fg=1.0, logic=logic)
    for _ in range(sets[0]["params"].size):
        D.param(0.0)
    # every set's primitives, in set order, as one union
    one = dict(sets[0])
    kinds = {k: np.concatenate([s["prims"][k] for s in sets]) for k in sets[0]["prims"]}
    nq = [s["q_base"].size for s in sets]
    q0 = np.concatenate([s["prims"]["q0"] + sum(nq[:i]) for i, s in enumerate(sets)])
    kinds["q0"] = q0.astype(np.int32)
    one["prims"] = kinds
    for key in ("q_base", "q_coeff", "q_param"):
        one[key] = np.concatenate([s[key] for s in sets])
    npr = kinds["kind"].size
    one["ops"] = np.asarray([(I.OP_PUSH << 24) | i for i in range(npr)] + [(I.OP_UNION << 24) | npr],
                            dtype=np.int32)
    one["eps_bg"], one["eps_fg"] = 1.0, 1.8
    got = LV.eps(sets, m["levels"], 1.0)
    assert np.abs(got - O.eps(one)).max() <= 1e-13


# ----------------------------------- the exact polygon mesher (Prop. 2) -----
def _star(rng, cx, cy, r, nv=9):
    """A concave star-shaped polygon (radii alternate), counter-clockwise."""
    t = np.sort(rng.uniform(0, 2 * np.pi, nv))
    rad = r * np.where(np.arange(nv) % 2 == 0, 1.0, 0.45) * rng.uniform(0.8, 1.0, nv)
    return np.stack([cx + rad * np.cos(t), cy + rad * np.sin(t)], axis=1)


def _inside(poly, x, y):
    """Even-odd ray casting (vectorised over points)."""
    inside = np.zeros(np.broadcast(x, y).shape, dtype=bool)
    n = len(poly)
    for a in range(n):
        (x0, y0), (x1, y1) = poly[a], poly[(a + 1) % n]
        cross = (y0 > y) != (y1 > y)
        with np.errstate(divide="ignore", invalid="ignore"):
            xi = x0 + (y - y0) * (x1 - x0) / (y1 - y0)
        inside ^= cross & (x < xi)
    return inside


def _grid(n, d=(10.0, 10.0, 10.0), off=((0.5, 0.5, 0.0),), o=(0.0, 0.0, 0.0)):
    return {"n": n, "ncomp": len(off), "d": d, "o": o, "off": [list(r) for r in off]}


def test_mesh_total_area_is_the_polygons_area():
    """Non-overlapping concave polygons inside the grid: the fills, times the
    cell area, add up to the shoelace areas, for any sample offset."""
    from oracle import mesh as M
    rng = np.random.default_rng(3)
    polys = [_star(rng, 120.0, 110.0, 60.0), _star(rng, 330.0, 200.0, 80.0, nv=12),
             _star(rng, 260.0, 60.0, 35.0, nv=7)[::-1]]
    want = sum(abs(G.area([tuple(v) for v in p])) for p in polys)
    for off in ((0.5, 0.5, 0.0), (0.0, 0.0, 0.0), (0.25, 0.8, 0.0)):
        f = M.fill(_grid((50, 52, 1), d=(10.0, 7.0, 10.0), off=(off,)), {"polys": polys, "z": None})
        assert abs(f.sum() * 70.0 - want) <= 1e-9 * want


def test_mesh_rectangle_is_the_product_of_overlaps():
    from oracle import mesh as M
    grid = _grid((20, 16, 1), off=((0.5, 0.5, 0.0), (0.0, 0.5, 0.0)))
    x0, x1, y0, y1 = 23.7, 141.2, 38.05, 97.9
    rect = np.array([[x0, y0], [x1, y0], [x1, y1], [x0, y1]])
    f = M.fill(grid, {"polys": [rect], "z": None})
    for c, off in enumerate(grid["off"]):
        xs = (np.arange(20) + off[0]) * 10.0
        ys = (np.arange(16) + off[1]) * 10.0
        ox = np.clip(np.minimum(xs + 5, x1) - np.maximum(xs - 5, x0), 0, None) / 10.0
        oy = np.clip(np.minimum(ys + 5, y1) - np.maximum(ys - 5, y0), 0, None) / 10.0
        assert np.abs(f[c, 0] - oy[:, None] * ox[None, :]).max() <= 1e-13


def test_mesh_box_matches_the_exact_autodiffgeo_box(oracle_mod):
    """An axis-aligned box: the mesher and the AutoDiffGeo box with its exact
    edge form (Eq. linear, zero error against volume averaging) agree, in 3D
    with Yee offsets and a z range."""
    from oracle import mesh as M
    D = I.Design((24, 18, 12), (10.0, 10.0, 10.0), ncomp=3, eps_bg=0.0, eps_fg=1.0)
    D.box(x=(31.3, 177.8), y=(12.6, 141.05), z=(22.2, 87.5))
    desc = D.to_desc()
    rect = np.array([[31.3, 12.6], [177.8, 12.6], [177.8, 141.05], [31.3, 141.05]])
    f = M.fill(desc["grid"], {"polys": [rect], "z": (22.2, 87.5)})
    assert np.abs(f - oracle_mod.fill(desc)).max() <= 1e-12


def test_mesh_converges_to_supersampling():
    """Lattice supersampling of a concave polygon's indicator converges to the
    mesher's fill (first order in the sub-lattice step)."""
    from oracle import mesh as M
    rng = np.random.default_rng(8)
    poly = _star(rng, 100.0, 90.0, 70.0, nv=11)
    grid = _grid((20, 18, 1))
    f = M.fill(grid, {"polys": [poly], "z": None})[0, 0]
    errs = []
    for s in (16, 64):
        u = (np.arange(s) + 0.5) / s
        X = (np.arange(20)[:, None] + u[None, :]).reshape(-1) * 10.0
        Y = (np.arange(18)[:, None] + u[None, :]).reshape(-1) * 10.0
        ins = _inside(poly, X[None, :], Y[:, None]).astype(np.float64)
        ss = ins.reshape(18, s, 20, s).mean(axis=(1, 3))
        errs.append(np.abs(ss - f).max())
    assert errs[1] < 0.4 * errs[0] and errs[1] < 0.03


def test_mesh_special_values():
    """Half a cell cut along its diagonal is 0.5 in either winding; a polygon
    covering everything gives the exact z overlap of the layer."""
    from oracle import mesh as M
    grid = _grid((4, 3, 1))
    tri = np.array([[10.0, 10.0], [20.0, 10.0], [20.0, 20.0]])
    for p in (tri, tri[::-1]):
        f = M.fill(grid, {"polys": [p], "z": None})[0, 0]
        assert f[1, 1] == 0.5 and f.sum() == 0.5
    g3 = _grid((3, 2, 6), off=((0.5, 0.5, 0.5),))
    big = np.array([[-100.0, -100.0], [100.0, -100.0], [100.0, 100.0], [-100.0, 100.0]])
    f = M.fill(g3, {"polys": [big], "z": (13.0, 38.5)})
    zs = (np.arange(6) + 0.5) * 10.0
    want = np.clip(np.minimum(zs + 5, 38.5) - np.maximum(zs - 5, 13.0), 0, None) / 10.0
    assert np.abs(f[0, :, 1, 1] - want).max() <= 1e-15


def test_mesh_fd_on_boxes_is_the_exact_gradient(oracle_mod):
    """Central differences of exactly meshed rectangles, with the step inside
    a cell, equal the AutoDiffGeo gradient of the same boxes in their exact
    edge form (both are the exact derivative of the volume average there)."""
    from oracle import mesh as M
    D = I.Design((40, 20, 1), (10.0, 10.0, 10.0), ncomp=1, eps_bg=1.0, eps_fg=3.5)
    edges = [(33.2, 96.7), (151.4, 233.9), (288.1, 351.35)]
    boxes = []
    for a, b in edges:
        ia, ib = D.param(a), D.param(b)
        boxes.append(D.box(x=(P(ia), P(ib)), y=(41.3, 122.6)))
    desc = D.to_desc()
    ef, ea, w = _fields(desc, 91, 92, 93)

    def layer(p):
        return {"polys": [np.array([[p[2 * k], 41.3], [p[2 * k + 1], 41.3], [p[2 * k + 1], 122.6],
                                    [p[2 * k], 122.6]]) for k in range(3)], "z": None}
    p0 = desc["params"]
    h = 0.01
    plus = [layer(p0 + h * np.eye(p0.size)[k]) for k in range(p0.size)]
    minus = [layer(p0 - h * np.eye(p0.size)[k]) for k in range(p0.size)]
    g = M.grad_fd(desc["grid"], plus, minus, ef, ea, w, h, 2.5)
    gad = oracle_mod.grad(desc, ef, ea, w)
    assert np.abs(g - gad).max() <= 1e-9 * np.abs(gad).max()


# ------------------------------------------- material levels (dense form) ---
def test_material_level_derivatives_match_fd_of_the_loss(oracle_mod):
    """dL/d eps_bg and dL/d eps_fg (Sec. 5.1's eps = eps_bg + deps fill): L is
    linear in both, so central differences of the loss are exact up to
    rounding."""
    O = oracle_mod
    desc = I.random_design(13, n=(36, 28, 10), nprims=12)
    ef, ea, w = _fields(desc, 21, 22)
    gm = O.grad_material(desc, ef, ea, w)
    h = 0.25
    fd = []
    for key in ("eps_bg", "eps_fg"):
        dp, dm = dict(desc), dict(desc)
        dp[key] = desc[key] + h
        dm[key] = desc[key] - h
        fd.append((O.loss(dp, ef, ea, w) - O.loss(dm, ef, ea, w)) / (2 * h))
    scale = abs(O.loss(desc, ef, ea, w)) + np.abs(gm).sum()
    assert np.abs(gm - np.array(fd)).max() <= 1e-11 * scale


def test_material_level_derivatives_count_cells(oracle_mod):
    """Unit fields and w = 1 make every sample's Re(w E_adj E) = 1: the two
    derivatives count the samples outside and inside a lattice-aligned box."""
    O = oracle_mod
    D = I.Design((20, 12, 6), (10.0, 10.0, 10.0), ncomp=3, eps_bg=1.0, eps_fg=3.0)
    D.box(x=(-100.0, 1000.0), y=(-100.0, 1000.0), z=(-100.0, 1000.0))
    D.box(x=(-50.0, -10.0))  # entirely off the grid: adds nothing
    desc = D.to_desc()
    ones = np.ones(I.field_shape(desc), dtype=np.complex64)
    gm = O.grad_material(desc, ones, ones, 1.0)
    total = ones.size
    assert gm[1] == total and gm[0] == 0.0
    D = I.Design((20, 12, 6), (10.0, 10.0, 10.0), ncomp=3, eps_bg=1.0, eps_fg=3.0)
    D.box(x=(-100.0, 1000.0), y=(-100.0, 1000.0), z=(-1000.0, -500.0))  # below the grid
    desc = D.to_desc()
    gm = O.grad_material(desc, ones, ones, 1.0)
    assert gm[0] == total and gm[1] == 0.0


# ---------------------------------------------------------------- P9 --------
def test_p9_invariants(oracle_mod):
    O = oracle_mod
    desc = I.random_design(9, n=(40, 32, 16), nprims=20)
    f = O.fill(desc)
    assert f.min() >= 0.0 and f.max() <= 1.0
    e = O.eps(desc)
    assert e.min() >= desc["eps_bg"] - 1e-12 and e.max() <= desc["eps_fg"] + 1e-12
    # translating the grid by one cell shifts the fill by one cell
    d2 = dict(desc)
    g = dict(desc["grid"])
    g["o"] = (g["o"][0] - g["d"][0], g["o"][1], g["o"][2])
    d2["grid"] = g
    f2 = O.fill(d2)
    assert np.abs(f2[..., 1:] - f[..., :-1]).max() <= 1e-12
    # g is linear in w; the complex seed equals the real seed G = Re(w E_adj E)
    ef, ea, _ = _fields(desc, 3, 4)
    w1 = np.array([0.3 + 0.1j, -1.0 + 0.5j, 0.2 - 0.9j], dtype=np.complex64)
    w2 = np.array([1.1 - 0.4j, 0.0 + 1.0j, -0.5 + 0.5j], dtype=np.complex64)
    g1, g2 = O.grad(desc, ef, ea, w1), O.grad(desc, ef, ea, w2)
    g12 = O.grad(desc, ef, ea, w1.astype(np.complex128) + w2.astype(np.complex128))
    assert np.linalg.norm(g12 - g1 - g2) <= 1e-9 * np.linalg.norm(g12)
    Gr = np.empty(I.field_shape(desc), dtype=np.float64)
    for c in range(3):
        Gr[c] = (w1[c].astype(np.complex128) * ea[c].astype(np.complex128)
                 * ef[c].astype(np.complex128)).real
    # the real-seed form takes float32 cotangents; compare at that precision
    gr = O.grad_real(desc, Gr.astype(np.float32))
    assert np.linalg.norm(gr - g1) <= 1e-5 * np.linalg.norm(g1)


# ---------------------------------------------------------------- P10 -------
def test_p10_topology_special_case(oracle_mod):
    """Independent one-cell boxes (B = I): each parameter moves one box's edge
    inside its own cell, so g_i = deps * Re(w E E_adj)_i / dx (Eq. top_AD with
    the exact pixel map)."""
    O = oracle_mod
    h = 1.0
    nx, ny = 6, 5
    D = I.Design((nx, ny, 1), (h, h, h), ncomp=1, off=[[0.5, 0.5, 0.0]], eps_bg=1.5, eps_fg=4.0)
    rng = np.random.default_rng(4)
    kids = []
    for j in range(ny):
        for i in range(nx):
            p = D.param(i + rng.uniform(0.2, 0.8))
            kids.append(D.box(x=(float(i), I.P(p)), y=(float(j), float(j + 1))))
    D.set_program(("union",) + tuple(kids))
    desc = D.to_desc()
    ef, ea, _ = _fields(desc, 5, 6)
    w = np.complex64(-2j)
    g = O.grad(desc, ef, ea, w)
    z = (w * ea[0, 0].astype(np.complex128) * ef[0, 0].astype(np.complex128)).real
    # PRODUCT union of disjoint boxes: other children are 0 in the cell -> factor 1
    expect = (desc["eps_fg"] - desc["eps_bg"]) * z.reshape(-1) / h
    assert np.abs(g - expect).max() <= 1e-12 * np.abs(expect).max()


# ------------------------------------------------ paper fixtures (Table 4) ---
def test_fixture_circ2d_area(oracle_mod):
    """Circ2D example (R = 0.5 at (0, -0.5), dx = 0.08): the grid sum of a
    symmetric sigmoid edge integrates to pi R^2 + pi^3 / (3 k^2)."""
    O = oracle_mod
    h = 0.08
    D = _grid2d(40, 40, h)
    D.grid["o"] = (-1.6, -2.1, 0.0)
    kr = 2.0
    D.circle(0.0, -0.5, 0.5, sigma="sigmoid", kr=kr)
    f = O.fill(D.to_desc())
    k = kr / h
    expect = math.pi * 0.25 + math.pi ** 3 / (3 * k * k)
    assert abs(f.sum() * h * h - expect) <= 2e-4 * expect


def test_fixture_poly2d_winding_independent(oracle_mod):
    """Poly2D example vertices (-0.7,0.6), (0.7,0.5), (0,-0.5) are clockwise;
    the inward normal reading makes the fill independent of winding, and
    with a steep sigma the fill is 1/0 at cells well inside/outside."""
    O = oracle_mod
    h = 0.08
    verts = [(-0.7, 0.6), (0.7, 0.5), (0.0, -0.5)]
    out = []
    for vv in (verts, verts[::-1]):
        D = _grid2d(25, 20, h)
        D.grid["o"] = (-1.0, -0.8, 0.0)
        D.polygon(vv, sigma="sigmoid", kr=200.0)
        out.append(O.fill(D.to_desc())[0, 0])
        desc = D.to_desc()
    assert np.abs(out[0] - out[1]).max() <= 1e-13  # edge order changes rounding only
    xs, ys = _centres(desc)
    for j, cy in enumerate(ys):
        for i, cx in enumerate(xs):
            a = G.cell_fraction(verts, cx, cy, h)
            if a == 1.0:
                assert out[0][j, i] > 1 - 1e-6
            elif a == 0.0:
                assert out[0][j, i] < 1e-6


# ------------------------------------- topology special case (Sec. 3.1) ------
def _topo_case(seed=3):
    from oracle import topology as T
    rng = np.random.default_rng(seed)
    n, C = (7, 6, 5), 3
    region = (1, 2, 4, 3, 1, 4)       # 4 x 3 pixels, broadcast to z = 1, 2, 3
    v = rng.normal(0.0, 1.5, 12)
    shape = (C, n[2], n[1], n[0])
    ef = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    ea = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    w = rng.normal(size=C) + 1j * rng.normal(size=C)
    return T, n, C, region, v, ef, ea, w


def test_topology_gradient_matches_central_differences():
    """Eq. top_AD against central differences of the loss whose gradient it
    is (L is smooth in v; h = 1e-5 in FP64)."""
    T, n, C, region, v, ef, ea, w = _topo_case()
    g = T.grad(n, C, region, v, 8.0, ef, ea, w)
    h = 1e-5
    fd = np.zeros_like(g)
    for i in range(v.size):
        vp, vm = v.copy(), v.copy()
        vp[i] += h
        vm[i] -= h
        fd[i] = (T.loss(n, C, region, vp, 2.0, 8.0, ef, ea, w) -
                 T.loss(n, C, region, vm, 2.0, 8.0, ef, ea, w)) / (2 * h)
    assert np.abs(g - fd).max() <= 1e-6 * np.abs(fd).max()


def test_topology_forward_special_values():
    """Eq. TO_example: sigma(0) = 1/2 puts every region sample halfway between
    the bounds, saturated v reaches the bounds, and samples outside the
    region (or outside its z cells) keep their value."""
    T, n, C, region, v, ef, ea, w = _topo_case()
    x0, y0, rx, ry, z0, z1 = region
    e = T.eps(n, C, region, np.zeros(rx * ry), 2.0, 8.0, eps_out=-1.0)
    assert np.all(e[:, z0:z1, y0:y0 + ry, x0:x0 + rx] == 6.0)
    inside = np.zeros(e.shape, bool)
    inside[:, z0:z1, y0:y0 + ry, x0:x0 + rx] = True
    assert np.all(e[~inside] == -1.0)
    hi = T.eps(n, C, region, np.full(rx * ry, 60.0), 2.0, 8.0)
    lo = T.eps(n, C, region, np.full(rx * ry, -60.0), 2.0, 8.0)
    assert np.allclose(hi[inside], 10.0, atol=1e-12) and np.allclose(lo[inside], 2.0, atol=1e-12)


def test_topology_reduces_to_the_im_form():
    """With w = -2 i omega (Eq. 1), one component and a one-cell z range, the
    gradient at v = 0 (sigma (1 - sigma) = 1/4) is 2 omega deps Im(E E_adj) / 4
    at each pixel: the paper's unconstrained form times the sigmoid slope."""
    from oracle import topology as T
    rng = np.random.default_rng(8)
    n, region = (5, 4, 1), (0, 0, 5, 4, 0, 1)
    shape = (1, 1, 4, 5)
    ef = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    ea = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    omega, deps = 1.7, 3.0
    g = T.grad(n, 1, region, np.zeros(20), deps, ef, ea, -2j * omega)
    z = ef[0, 0].astype(np.complex128) * ea[0, 0].astype(np.complex128)
    assert np.allclose(g, (2 * omega * deps * z.imag / 4).reshape(-1), rtol=1e-12, atol=0)
