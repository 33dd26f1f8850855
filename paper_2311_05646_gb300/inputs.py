"""Seeded synthetic inputs: design descriptions and complex64 fields.

This module holds none of the method's arithmetic.  It only builds the plain
design description (grid, materials, parameter map, primitive table, postfix
logic program) and seeded complex fields, with the shapes and sizes of the
paper's workloads (a grating coupler, a waveguide taper, a hole lattice; see
Sec. 6 of arXiv 2311.05646).  Both the CUDA library binding and the CPU
oracle consume what it produces, each through its own marshalling code.

The description format (integer codes, array meanings) is documented in
``include/adg.h``; this module writes the same codes by value.
"""
from __future__ import annotations

import math

import numpy as np

# ---- format codes (values fixed by the description format) -----------------
BOX, CIRCLE, POLYGON, GRAPH, POLAR = 0, 1, 2, 3, 4
SIGMA = {"linear": 0, "sigmoid": 1, "quadratic": 2, "sin": 3, "erf": 4}
BOUND_X, BOUND_Y, BOUND_Z, RECT_SIGMA, GRAPH_ABOVE, XFORM = 1, 2, 4, 8, 16, 64
OP_PUSH, OP_UNION, OP_INTERSECT, OP_DIFF = 0, 1, 2, 3

# Yee sample offsets (in cells) used by default: 2D single component at the
# cell centre; 3D edge-centred E components Ex, Ey, Ez.
OFF_2D = [[0.5, 0.5, 0.0]]
OFF_3D = [[0.5, 0.0, 0.0], [0.0, 0.5, 0.0], [0.0, 0.0, 0.5]]
# H sample offsets: 2D single component at the cell corner; 3D face-centred
# H components Hx, Hy, Hz.
OFF_H_2D = [[0.0, 0.0, 0.0]]
OFF_H_3D = [[0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]


class P:
    """A geometric scalar driven by a parameter: q = base + coeff * p[idx]."""

    __slots__ = ("idx", "base", "coeff")

    def __init__(self, idx: int, base: float = 0.0, coeff: float = 1.0):
        self.idx, self.base, self.coeff = int(idx), float(base), float(coeff)


class Design:
    """Builder for one design description."""

    def __init__(self, n, d, o=(0.0, 0.0, 0.0), ncomp=1, off=None, eps_bg=1.0, eps_fg=2.0,
                 logic="product"):
        n = tuple(int(v) for v in n)
        if len(n) == 2:
            n = (n[0], n[1], 1)
        d = tuple(float(v) for v in d)
        if len(d) == 2:
            d = (d[0], d[1], 1.0)
        if off is None:
            off = OFF_2D if ncomp == 1 else OFF_3D
        self.grid = {"n": n, "ncomp": int(ncomp), "d": d, "o": tuple(float(v) for v in o),
                     "off": [list(map(float, r)) for r in off][:ncomp]}
        self.eps_bg, self.eps_fg, self.logic = float(eps_bg), float(eps_fg), logic
        self.params: list[float] = []
        self.q_base: list[float] = []
        self.q_coeff: list[float] = []
        self.q_param: list[int] = []
        self.prims = {"kind": [], "sigma": [], "flags": [], "q0": [], "nq": [], "kr": []}
        self.program = None

    # parameters and geometric scalars
    def param(self, value: float) -> int:
        self.params.append(float(value))
        return len(self.params) - 1

    def _q(self, spec) -> int:
        if isinstance(spec, P):
            self.q_base.append(spec.base)
            self.q_coeff.append(spec.coeff)
            self.q_param.append(spec.idx)
        else:
            self.q_base.append(float(spec))
            self.q_coeff.append(0.0)
            self.q_param.append(-1)
        return len(self.q_base) - 1

    def _prim(self, kind, sigma, kr, flags, specs, xform=None) -> int:
        """xform = (px, py, theta, sx, sy): the in-plane rotation (radians) and
        aspect transform about the pivot (px, py), appended as five scalars."""
        if xform is not None:
            if len(xform) != 5:
                raise ValueError("xform = (px, py, theta, sx, sy)")
            flags |= XFORM
            specs = list(specs) + list(xform)
        q0 = len(self.q_base)
        for s in specs:
            self._q(s)
        pr = self.prims
        pr["kind"].append(kind)
        pr["sigma"].append(SIGMA[sigma] if isinstance(sigma, str) else int(sigma))
        pr["flags"].append(int(flags))
        pr["q0"].append(q0)
        pr["nq"].append(len(specs))
        pr["kr"].append(float(kr))
        return len(pr["kind"]) - 1

    # primitives (Table "AutoDiffGeo definitions")
    def box(self, x=None, y=None, z=None, mode="exact", sigma="linear", kr=1.0, xform=None) -> int:
        flags, specs = 0, []
        for ax, iv in enumerate((x, y, z)):
            if iv is None:
                specs += [0.0, 0.0]
            else:
                flags |= 1 << ax
                specs += [iv[0], iv[1]]
        if mode == "sigma":
            flags |= RECT_SIGMA
        return self._prim(BOX, sigma, kr, flags, specs, xform)

    def circle(self, cx, cy, r, z=None, sigma="sigmoid", kr=4.0, xform=None) -> int:
        flags = BOUND_Z if z is not None else 0
        zz = z if z is not None else (0.0, 0.0)
        return self._prim(CIRCLE, sigma, kr, flags, [cx, cy, r, zz[0], zz[1]], xform)

    def polar(self, cx, cy, R0, coeffs=(), z=None, sigma="sigmoid", kr=4.0, xform=None) -> int:
        """Polar2D with the Fourier boundary R(theta) = R0 + sum_n c_n cos(n
        theta) + s_n sin(n theta); coeffs = [(c_1, s_1), ..., (c_N, s_N)]."""
        flags = BOUND_Z if z is not None else 0
        zz = z if z is not None else (0.0, 0.0)
        specs = [cx, cy, R0, zz[0], zz[1]]
        for c, s in coeffs:
            specs += [c, s]
        return self._prim(POLAR, sigma, kr, flags, specs, xform)

    def polygon(self, verts, z=None, sigma="sigmoid", kr=4.0, xform=None) -> int:
        flags = BOUND_Z if z is not None else 0
        zz = z if z is not None else (0.0, 0.0)
        specs = [zz[0], zz[1]]
        for vx, vy in verts:
            specs += [vx, vy]
        return self._prim(POLYGON, sigma, kr, flags, specs, xform)

    def graph(self, X, Y, above=False, z=None, sigma="sigmoid", kr=4.0) -> int:
        flags = (BOUND_Z if z is not None else 0) | (GRAPH_ABOVE if above else 0)
        zz = z if z is not None else (0.0, 0.0)
        return self._prim(GRAPH, sigma, kr, flags, [zz[0], zz[1]] + list(X) + list(Y))

    # logic program: nested tuples ('union', ...), ('intersect', ...), ('diff', a, b)
    def set_program(self, tree) -> None:
        self.program = tree

    def _emit(self, node, out):
        if isinstance(node, (int, np.integer)):
            out.append((OP_PUSH << 24) | int(node))
            return
        op = node[0]
        kids = node[1:]
        for k in kids:
            self._emit(k, out)
        if op == "union":
            out.append((OP_UNION << 24) | len(kids))
        elif op == "intersect":
            out.append((OP_INTERSECT << 24) | len(kids))
        elif op == "diff":
            assert len(kids) == 2
            out.append(OP_DIFF << 24)
        else:
            raise ValueError(op)

    def to_desc(self) -> dict:
        ops: list[int] = []
        tree = self.program if self.program is not None else ("union",) + tuple(
            range(len(self.prims["kind"])))
        self._emit(tree, ops)
        return {
            "grid": self.grid,
            "eps_bg": self.eps_bg,
            "eps_fg": self.eps_fg,
            "logic": self.logic,
            "params": np.asarray(self.params, dtype=np.float64),
            "q_base": np.asarray(self.q_base, dtype=np.float64),
            "q_coeff": np.asarray(self.q_coeff, dtype=np.float64),
            "q_param": np.asarray(self.q_param, dtype=np.int32),
            "prims": {k: np.asarray(v, dtype=np.float64 if k == "kr" else np.int32)
                      for k, v in self.prims.items()},
            "ops": np.asarray(ops, dtype=np.int32),
        }


def mu_design(desc: dict, mu_bg: float = 1.0, mu_fg: float = 1.5, off=None) -> dict:
    """The permeability composition of a design (Eq. mu): the same shapes,
    program and parameters, sampled at the H offsets, with the two material
    levels mu_bg / mu_fg in the eps_bg / eps_fg slots of the description."""
    C = int(desc["grid"]["ncomp"])
    if off is None:
        off = OFF_H_2D if C == 1 else OFF_H_3D
    out = dict(desc)
    out["grid"] = dict(desc["grid"])
    out["grid"]["off"] = [list(map(float, r)) for r in off][:C]
    out["eps_bg"], out["eps_fg"] = float(mu_bg), float(mu_fg)
    return out


def field_shape(desc: dict):
    g = desc["grid"]
    nx, ny, nz = g["n"]
    return (g["ncomp"], nz, ny, nx)


def n_cells(desc: dict) -> int:
    nx, ny, nz = desc["grid"]["n"]
    return nx * ny * nz


# ---- fields ---------------------------------------------------------------
def plane_wave_field(desc: dict, seed: int, nwaves: int = 8, wavelength: float = 1550.0,
                     n_eff: float = 2.85, waist_frac: float = 1.0 / 3.0) -> np.ndarray:
    """Sum of seeded random plane waves times a Gaussian envelope, complex64.

    Each component gets its own waves; sample points follow the grid's
    per-component offsets.  Separable in x, y, z, so it is built from outer
    products (cheap even for large grids)."""
    g = desc["grid"]
    nx, ny, nz = g["n"]
    C = g["ncomp"]
    dx, dy, dz = g["d"]
    ox, oy, oz = g["o"]
    rng = np.random.default_rng(seed)
    kmag = 2.0 * math.pi * n_eff / wavelength
    out = np.zeros((C, nz, ny, nx), dtype=np.complex64)
    ext = (nx * dx, ny * dy, nz * dz)
    cen = (ox + 0.5 * ext[0], oy + 0.5 * ext[1], oz + 0.5 * ext[2])
    for c in range(C):
        off = g["off"][c]
        xs = ox + (np.arange(nx) + off[0]) * dx
        ys = oy + (np.arange(ny) + off[1]) * dy
        zs = oz + (np.arange(nz) + off[2]) * dz
        env = []
        for a, v in enumerate((xs, ys, zs)):
            wst = max(ext[a] * waist_frac, 1e-9)
            env.append(np.exp(-(((v - cen[a]) / wst) ** 2)))
        acc = np.zeros((nz, ny, nx), dtype=np.complex128)
        for _ in range(nwaves):
            if nz > 1:
                v = rng.normal(size=3)
            else:
                v = np.array([*rng.normal(size=2), 0.0])
            v /= np.linalg.norm(v)
            ph = rng.uniform(0, 2 * math.pi)
            amp = (rng.normal() + 1j * rng.normal()) / math.sqrt(2.0)
            fx = env[0] * np.exp(1j * kmag * v[0] * xs)
            fy = env[1] * np.exp(1j * kmag * v[1] * ys)
            fz = env[2] * np.exp(1j * (kmag * v[2] * zs + ph))
            acc += amp * (fz[:, None, None] * fy[None, :, None] * fx[None, None, :])
        out[c] = acc.astype(np.complex64)
    return out


def seeded_w(ncomp: int, seed: int) -> np.ndarray:
    """Per-component complex weights (Eq. 1 uses w = -2 i omega; tests use
    random complex w so that real/imaginary mix-ups cannot cancel)."""
    rng = np.random.default_rng(seed)
    return (rng.normal(size=ncomp) + 1j * rng.normal(size=ncomp)).astype(np.complex64)


# ---- workloads ------------------------------------------------------------
def grating_2d(variant: str = "fit", seed: int = 11, n=(200, 100), d: float = 20.0) -> dict:
    """2D TE single design: an input waveguide with a 20-tooth etched grating
    (Sec. 6.1 blazed-grating recipe: rectangles, union, difference).

    variant 'fit': 180 +- 15 nm pitch so all 20 teeth lie on the 4 um grid;
    variant 'literal': 600 +- 50 nm pitch, most teeth fall off the grid.
    40 parameters: the two x edges of every tooth."""
    rng = np.random.default_rng(seed)
    nx, ny = n
    D = Design((nx, ny, 1), (d, d, d), ncomp=1, eps_bg=2.085, eps_fg=12.11)
    y_top = 0.5 * ny * d + 110.0
    wg = D.box(x=(-10.0 * d, (nx + 10) * d), y=(y_top - 220.0, y_top))
    pitch, jit, width = (180.0, 15.0, 90.0) if variant == "fit" else (600.0, 50.0, 300.0)
    x = 300.0 if variant == "fit" else 200.0
    teeth = []
    for _ in range(20):
        x0 = x + rng.uniform(-0.1, 0.1) * jit
        x1 = x0 + width + rng.uniform(-0.1, 0.1) * jit
        p0, p1 = D.param(x0), D.param(x1)
        teeth.append(D.box(x=(P(p0), P(p1)), y=(y_top - 110.0, y_top + 60.0)))
        x += pitch + rng.uniform(-1.0, 1.0) * jit
    D.set_program(("diff", wg, ("union",) + tuple(teeth)))
    return D.to_desc()


def grating_3d(n=(600, 200, 120), d=(40.0, 40.0, 20.0), teeth: int = 30, seed: int = 21,
               pitch: float = 600.0) -> dict:
    """3D two-etch grating: a 220 nm slab with `teeth` periods, each a deep
    (150 nm) and a shallow (70 nm) full-width etched rectangle; 4 edge
    parameters per period.  eps = slab - union(etches)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    D = Design(n, d, ncomp=3, eps_bg=2.085, eps_fg=12.11)
    zc = 0.5 * nz * d[2]
    z_bot, z_top = zc - 110.0, zc + 110.0
    slab = D.box(z=(z_bot, z_top))
    x0 = 0.5 * (nx * d[0] - teeth * pitch) + 0.25 * pitch
    etches = []
    for t in range(teeth):
        xa = x0 + t * pitch + rng.uniform(-20, 20)
        xb = xa + 150.0 + rng.uniform(-20, 20)
        xc = xb + 30.0 + rng.uniform(-10, 10)
        xd = xc + 150.0 + rng.uniform(-20, 20)
        pa, pb, pc, pd = (D.param(v) for v in (xa, xb, xc, xd))
        etches.append(D.box(x=(P(pa), P(pb)), z=(z_top - 150.0, z_top + 60.0)))
        etches.append(D.box(x=(P(pc), P(pd)), z=(z_top - 70.0, z_top + 60.0)))
    D.set_program(("diff", slab, ("union",) + tuple(etches)))
    return D.to_desc()


def taper_3d(n=(800, 300, 100), d: float = 40.0, nverts: int = 64, seed: int = 31,
             kr: float = 4.0, sigma: str = "sigmoid") -> dict:
    """Non-adiabatic taper (Sec. 6.2): input waveguide 0.5 um, output 10.5 um,
    taper length 23 um starting at x0 = 1 um; each side of the taper is a
    graph boundary through `nverts` vertices whose y offsets (0-300 nm,
    seeded) are the parameters.  A 300 nm slab, extruded along z."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    D = Design(n, (d, d, d), ncomp=3, eps_bg=1.444 ** 2, eps_fg=3.4757 ** 2)
    ext_x, ext_y = nx * d, ny * d
    scale = ext_x / 32000.0
    x0, L = 1000.0 * scale, 23000.0 * scale
    w_in, w_out = 500.0 * min(1.0, ext_y / 12000.0), 10500.0 * min(1.0, ext_y / 12000.0)
    yc = 0.5 * ext_y
    zc = 0.5 * nz * d
    zr = (zc - 150.0, zc + 150.0)
    X = np.linspace(x0, x0 + L, nverts)
    half = 0.5 * (w_in + (w_out - w_in) * (X - x0) / L)
    up_p = [D.param(v) for v in rng.uniform(0.0, 300.0, nverts)]
    lo_p = [D.param(v) for v in rng.uniform(0.0, 300.0, nverts)]
    wg_in = D.box(x=(-10 * d, x0), y=(yc - 0.5 * w_in, yc + 0.5 * w_in), z=zr)
    wg_out = D.box(x=(x0 + L, ext_x + 10 * d), y=(yc - 0.5 * w_out, yc + 0.5 * w_out), z=zr)
    g_up = D.graph(list(X), [P(up_p[j], yc + half[j], 1.0) for j in range(nverts)], above=False,
                   z=zr, sigma=sigma, kr=kr)
    g_lo = D.graph(list(X), [P(lo_p[j], yc - half[j], -1.0) for j in range(nverts)], above=True,
                   z=zr, sigma=sigma, kr=kr)
    xr = D.box(x=(x0, x0 + L))
    D.set_program(("union", wg_in, wg_out, ("intersect", g_up, g_lo, xr)))
    return D.to_desc()


def _convex_polygon(rng, cx, cy, r, nv):
    """Vertices of a perturbed circle that stays convex (radial jitter only
    on every other vertex, small)."""
    th = np.linspace(0, 2 * math.pi, nv, endpoint=False) + rng.uniform(0, 2 * math.pi)
    rr = r * (1.0 + 0.02 * np.cos(th * 2))
    return [(cx + rr[i] * math.cos(th[i]), cy + rr[i] * math.sin(th[i])) for i in range(nv)]


def random_design(seed: int, n=None, nprims=None, d: float = 40.0) -> dict:
    """One design of the batched mix: a slab plus `nprims` features (50% boxes,
    30% circles r 80-200 nm, 20% convex 16-64-gons) combined by a random tree
    of unions and differences.  Parameters: box x edges, circle (x, y, r),
    polygon centre (x, y)."""
    rng = np.random.default_rng(seed)
    if n is None:
        n = (int(rng.integers(128, 513)), int(rng.integers(64, 257)), int(rng.integers(32, 97)))
    nx, ny, nz = n
    if nprims is None:
        nprims = int(rng.integers(10, 401))
    D = Design(n, (d, d, d), ncomp=3, eps_bg=2.085, eps_fg=12.11)
    ex, ey, ez = nx * d, ny * d, nz * d
    zc = 0.5 * ez
    slab = D.box(z=(zc - 110.0, zc + 110.0))
    feats = []
    for _ in range(nprims - 1):
        u = rng.uniform()
        z0 = zc - 110.0 - rng.uniform(0, 60)
        zr = (z0, z0 + rng.uniform(100, 260))
        if u < 0.5:
            cx, cy = rng.uniform(0, ex), rng.uniform(0, ey)
            wx, wy = rng.uniform(80, 600), rng.uniform(80, 600)
            pa, pb = D.param(cx - wx / 2), D.param(cx + wx / 2)
            feats.append(D.box(x=(P(pa), P(pb)), y=(cy - wy / 2, cy + wy / 2), z=zr))
        elif u < 0.8:
            px, py, pr = D.param(rng.uniform(0, ex)), D.param(rng.uniform(0, ey)), D.param(
                rng.uniform(80, 200))
            feats.append(D.circle(P(px), P(py), P(pr), z=zr, sigma="sigmoid", kr=4.0))
        else:
            nv = int(rng.integers(16, 65))
            cx, cy, r = rng.uniform(0, ex), rng.uniform(0, ey), rng.uniform(120, 300)
            px, py = D.param(0.0), D.param(0.0)
            verts = _convex_polygon(rng, cx, cy, r, nv)
            feats.append(D.polygon([(P(px, vx), P(py, vy)) for vx, vy in verts], z=zr,
                                   sigma="sigmoid", kr=4.0))

    def tree(items):
        if len(items) == 1:
            return items[0]
        if len(items) <= 4 or rng.uniform() < 0.3:
            return ("union",) + tuple(items)
        cut = int(rng.integers(1, len(items)))
        a, b = tree(items[:cut]), tree(items[cut:])
        return ("diff", a, b) if rng.uniform() < 0.5 else ("union", a, b)

    D.set_program(("union", slab, tree(feats)) if feats else slab)
    return D.to_desc()


def hole_lattice(n=(1000, 1000, 80), d=(40.0, 40.0, 20.0), holes: int = 20, seed: int = 51,
                 ncomp: int = 3) -> dict:
    """The largest served design: a `holes` x `holes` lattice of circular holes
    (x, y, r parameters each) etched through a 220 nm slab, united with a
    fixed shallow-etch rectangle layer; eps = slab - union(holes, shallow)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    D = Design(n, d, ncomp=ncomp, eps_bg=2.085, eps_fg=12.11)
    ex, ey = nx * d[0], ny * d[1]
    zc = 0.5 * nz * d[2] if nz > 1 else 0.0
    zr = (zc - 110.0, zc + 110.0) if nz > 1 else None
    slab = D.box(z=zr) if nz > 1 else D.box(x=(-1e3, ex + 1e3))
    pitch_x, pitch_y = ex / holes, ey / holes
    hs = []
    for a in range(holes):
        for b in range(holes):
            cx = (a + 0.5) * pitch_x + rng.uniform(-0.05, 0.05) * pitch_x
            cy = (b + 0.5) * pitch_y + rng.uniform(-0.05, 0.05) * pitch_y
            r = rng.uniform(0.2, 0.3) * min(pitch_x, pitch_y)
            px, py, pr = D.param(cx), D.param(cy), D.param(r)
            hz = (zr[0] - 40.0, zr[1] + 40.0) if zr else None
            hs.append(D.circle(P(px), P(py), P(pr), z=hz, sigma="sigmoid", kr=4.0))
    if zr:
        shallow = D.box(x=(0.1 * ex, 0.3 * ex), y=(0.0 - 1e3, ey + 1e3),
                        z=(zr[1] - 70.0, zr[1] + 40.0))
    else:
        shallow = D.box(x=(0.1 * ex, 0.3 * ex), y=(0.4 * ey, 0.45 * ey))
    D.set_program(("diff", slab, ("union",) + tuple(hs) + (shallow,)))
    return D.to_desc()


def nonbinary_circles(n=(200, 200, 1), d=(20.0, 20.0, 20.0), levels=(0.1, 0.34, 0.62, 1.0),
                      per_level: int = 3, t: float = 0.55, eps_bg: float = 0.0, seed: int = 61,
                      ncomp=None, logic: str = "product", boxes: bool = True) -> dict:
    """Overlapping shapes of several material levels (App. B, Alg. 1; its
    example: circles of levels 0.1, 0.34, 0.62 and 1.0 over a background of 0,
    brought in from the four quadrants towards the centre).

    Level k's set is `per_level` circles (cx, cy, r parameters each) placed
    around its quadrant's centre and moved a fraction `t` of the way to the
    grid's centre, plus one fixed-size box (two x-edge parameters) when
    `boxes`; in 3D the shapes are slabs of the middle half of z.  Every set is
    one description with material slots 0 / 1 and its own union program; all
    sets carry the same parameter vector, in the same order.  Returns
    {"sets": [desc, ...], "levels": array of K, "eps_bg": float}."""
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    if len(n) == 2:
        n = (n[0], n[1], 1)
    nx, ny, nz = n
    d = tuple(float(v) for v in d)
    if ncomp is None:
        ncomp = 1 if nz == 1 else 3
    K = len(levels)
    ex, ey = nx * d[0], ny * d[1]
    zc = 0.5 * nz * d[2]
    zr = (zc - 0.25 * nz * d[2], zc + 0.25 * nz * d[2]) if nz > 1 else None
    sets = [Design(n, d, ncomp=ncomp, eps_bg=0.0, eps_fg=1.0, logic=logic) for _ in range(K)]
    owned = [[] for _ in range(K)]
    quad = [(0.25, 0.25), (0.75, 0.25), (0.25, 0.75), (0.75, 0.75)]
    rmax = 0.2 * min(ex, ey)
    for k in range(K):
        qx, qy = quad[k % 4]
        cx0 = ex * (qx + t * (0.5 - qx))
        cy0 = ey * (qy + t * (0.5 - qy))
        for _ in range(per_level):
            vals = (cx0 + rng.uniform(-0.3, 0.3) * rmax, cy0 + rng.uniform(-0.3, 0.3) * rmax,
                    rng.uniform(0.35, 0.7) * rmax)
            idx = [[D.param(v) for v in vals] for D in sets][k]
            owned[k].append(("circle", idx))
        if boxes:
            x0 = cx0 - rng.uniform(0.5, 1.0) * rmax
            vals = (x0, x0 + rng.uniform(0.6, 1.2) * rmax)
            idx = [[D.param(v) for v in vals] for D in sets][k]
            y0 = cy0 + rng.uniform(-0.6, 0.2) * rmax
            owned[k].append(("box", idx, (y0, y0 + 0.4 * rmax)))
    for k, D in enumerate(sets):
        prims = []
        for item in owned[k]:
            if item[0] == "circle":
                i = item[1]
                prims.append(D.circle(P(i[0]), P(i[1]), P(i[2]), z=zr, sigma="sigmoid", kr=4.0))
            else:
                i = item[1]
                prims.append(D.box(x=(P(i[0]), P(i[1])), y=item[2], z=zr, sigma="linear"))
        D.set_program(("union",) + tuple(prims))
    return {"sets": [D.to_desc() for D in sets],
            "levels": np.asarray(levels, dtype=np.float64), "eps_bg": float(eps_bg)}


def hex_hole_lattice(n=(300, 200, 40), d=(40.0, 40.0, 20.0), holes=(10, 6), R: float = 260.0,
                     seed: int = 71, ncomp=None, sigma: str = "sigmoid", kr: float = 4.0) -> dict:
    """Prop. 2's setting on a small scale: hexagonal holes (centre x, y
    parameters each) etched through a 220 nm slab.  Returns the AutoDiffGeo
    description ("desc": slab - union of Poly2D hexagons, eps 2.085 / 12.11)
    and, for the exact mesher, the hole geometry ("R", "z", "centres": the
    (x, y) parameter indices of each hole) from which `hex_layer` builds the
    polygon layer at any parameter vector."""
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    nx, ny, nz = n
    if ncomp is None:
        ncomp = 1 if nz == 1 else 3
    D = Design(n, d, ncomp=ncomp, eps_bg=2.085, eps_fg=12.11)
    ex, ey = nx * d[0], ny * d[1]
    zc = 0.5 * nz * d[2]
    zr = (zc - 110.0, zc + 110.0) if nz > 1 else None
    slab = D.box(z=zr) if nz > 1 else D.box(x=(-1e3, ex + 1e3))
    hx, hy = holes
    px, py = ex / hx, ey / hy
    centres, hs = [], []
    for a in range(hx):
        for b in range(hy):
            ix = D.param((a + 0.5) * px + rng.uniform(-0.1, 0.1) * px)
            iy = D.param((b + 0.5) * py + rng.uniform(-0.1, 0.1) * py)
            ang = [math.pi * m / 3.0 + math.pi / 6.0 for m in range(6)]
            verts = [(P(ix, R * math.cos(t)), P(iy, R * math.sin(t))) for t in ang]
            hs.append(D.polygon(verts, z=zr, sigma=sigma, kr=kr))
            centres.append((ix, iy))
    D.set_program(("diff", slab, ("union",) + tuple(hs)))
    return {"desc": D.to_desc(), "R": float(R), "z": zr, "centres": centres}


def hex_layer(spec: dict, params) -> dict:
    """The holes of `hex_hole_lattice` at `params` as a polygon layer for the
    exact mesher: {"polys": [(6, 2) vertices], "z": (z0, z1) or None}."""
    p = np.asarray(params, dtype=np.float64)
    R = spec["R"]
    ang = np.array([math.pi * m / 3.0 + math.pi / 6.0 for m in range(6)])
    polys = [np.stack([p[ix] + R * np.cos(ang), p[iy] + R * np.sin(ang)], axis=1)
             for ix, iy in spec["centres"]]
    return {"polys": polys, "z": spec["z"]}


def hex_fd_layers(spec: dict, params, h: float):
    """Per parameter: the layer at p + h e_k, at p - h e_k, and a cell region
    (x0, y0, nx, ny, z0, z1) holding every sample whose fill the step moves
    (the moved hole's box, two cells of margin, every z)."""
    grid = spec["desc"]["grid"]
    nx, ny, nz = grid["n"]
    dx, dy, _ = grid["d"]
    ox, oy, _ = grid["o"]
    p0 = np.asarray(params, dtype=np.float64)
    owner = {}
    for hidx, (ix, iy) in enumerate(spec["centres"]):
        owner[ix] = owner[iy] = hidx
    plus, minus, regions = [], [], []
    R = spec["R"]
    for k in range(p0.size):
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        plus.append(hex_layer(spec, pp))
        minus.append(hex_layer(spec, pm))
        ix, iy = spec["centres"][owner[k]]
        x0 = int(math.floor((p0[ix] - R - h - ox) / dx)) - 2
        x1 = int(math.ceil((p0[ix] + R + h - ox) / dx)) + 2
        y0 = int(math.floor((p0[iy] - R - h - oy) / dy)) - 2
        y1 = int(math.ceil((p0[iy] + R + h - oy) / dy)) + 2
        x0, y0, x1, y1 = max(x0, 0), max(y0, 0), min(x1, nx), min(y1, ny)
        regions.append((x0, y0, x1 - x0, y1 - y0, 0, nz))
    return plus, minus, regions


def psgc_lattice(n=(200, 160, 40), d=(30.0, 30.0, 30.0), rows: int = 4, cols: int = 5,
                 harmonics: int = 6, seed: int = 81, centres: bool = False, ncomp=None,
                 sigma: str = "sigmoid", kr: float = 4.0) -> dict:
    """A polarisation-splitting-grating-like layout (Sec. 5.3 / 6.3): a
    `rows` x `cols` array of Polar2D scatterers with Fourier boundaries
    R(theta) = R0 + sum_{n <= harmonics} c_n cos(n theta) + s_n sin(n theta),
    etched through a 220 nm slab (eps = slab - union(scatterers)).  Each
    scatterer's R0 is a parameter; the Fourier coefficients are parameters
    shared by the scatterers of a row; with `centres`, each scatterer's
    (cx, cy) are parameters too."""
    rng = np.random.default_rng(seed)
    n = tuple(int(v) for v in n)
    nx, ny, nz = n
    if ncomp is None:
        ncomp = 1 if nz == 1 else 3
    D = Design(n, d, ncomp=ncomp, eps_bg=2.085, eps_fg=12.11)
    ex, ey = nx * d[0], ny * d[1]
    zc = 0.5 * nz * d[2]
    zr = (zc - 110.0, zc + 110.0) if nz > 1 else None
    slab = D.box(z=zr) if nz > 1 else D.box(x=(-1e3, ex + 1e3))
    px, py = ex / cols, ey / rows
    base = 0.28 * min(px, py)
    scat = []
    for r in range(rows):
        amp = base * 0.25 / max(harmonics, 1)
        coef = [(D.param(rng.uniform(-amp, amp)), D.param(rng.uniform(-amp, amp)))
                for _ in range(harmonics)]
        for c in range(cols):
            cx = (c + 0.5) * px + rng.uniform(-0.05, 0.05) * px
            cy = (r + 0.5) * py + rng.uniform(-0.05, 0.05) * py
            if centres:
                cx, cy = P(D.param(cx)), P(D.param(cy))
            R0 = P(D.param(base * rng.uniform(0.85, 1.0)))
            scat.append(D.polar(cx, cy, R0, [(P(a), P(b)) for a, b in coef], z=zr, sigma=sigma,
                                kr=kr))
    D.set_program(("diff", slab, ("union",) + tuple(scat)))
    return D.to_desc()
