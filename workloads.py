"""Seeded synthetic inputs for the 2D-FC hot path: domains, grids, parameters, functions.

This module is shared by the tests, the benchmark and the oracle.  It holds no
2D-FC arithmetic: only workload definitions (literal numbers), closed-form test
functions and a counter-based random generator.

Random numbers: splitmix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) on the counter seed*2^32 + i, the top 53 bits
giving a uniform double in [0, 1), and Box-Muller for normals.  Everything is
generated on the host, so every consumer sees identical bits.

Domains are closed curves given by trigonometric polynomials
    x(theta) = sum_k cx[k] cos(k theta) + sx[k] sin(k theta)
    y(theta) = sum_k cy[k] cos(k theta) + sy[k] sin(k theta),
counter-clockwise.  The Cartesian grid is x_i = a0 + i h, y_j = b0 + j h with
0 <= i < nx, 0 <= j < ny, stored row-major as [ny][nx].

The box, h and the normal step k1 of each workload are literals.  They were chosen
once by this rule: the grid must contain the domain and its outer strip, whose
width is C*k1, with a margin of a few h.  k1 is h unless that would let the strip
leave the box, or pass half the smallest concave radius of curvature of the curve.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

_MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)


# --------------------------------------------------------------------------- #
# Counter-based generator
# --------------------------------------------------------------------------- #
def splitmix64(seed: int, n: int) -> np.ndarray:
    """n outputs of splitmix64 applied to the counters seed*2^32 + i (uint64)."""
    with np.errstate(over="ignore"):
        z = (np.uint64(seed) << np.uint64(32)) + np.arange(n, dtype=np.uint64)
        z = z * np.uint64(0x9E3779B97F4A7C15) + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of splitmix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms."""
    m = (n + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    return z[:n]


# --------------------------------------------------------------------------- #
# Domains, grids, parameters
# --------------------------------------------------------------------------- #
@dataclass(frozen=True)
class Boundary:
    cx: tuple
    sx: tuple
    cy: tuple
    sy: tuple

    def arrays(self):
        k = max(len(self.cx), len(self.sx), len(self.cy), len(self.sy))
        pad = lambda t: np.array(list(t) + [0.0] * (k - len(t)), dtype=np.float64)
        return pad(self.cx), pad(self.sx), pad(self.cy), pad(self.sy)

    def polygon(self, n: int = 4096):
        """Dense polygon of the curve (input generation only)."""
        cx, sx, cy, sy = self.arrays()
        th = 2 * np.pi * np.arange(n) / n
        k = np.arange(len(cx))[:, None]
        c, s = np.cos(k * th), np.sin(k * th)
        return cx @ c + sx @ s, cy @ c + sy @ s


def disk(radius: float = 1.0) -> Boundary:
    return Boundary(cx=(0.0, radius), sx=(0.0, 0.0), cy=(0.0, 0.0), sy=(0.0, radius))


def star(a: float, k: int) -> Boundary:
    """r(theta) = 1 + a cos(k theta) written as a trigonometric polynomial."""
    n = k + 2
    cx = [0.0] * n
    sy = [0.0] * n
    cx[1] += 1.0
    sy[1] += 1.0
    cx[k + 1] += a / 2
    cx[k - 1] += a / 2
    sy[k + 1] += a / 2
    sy[k - 1] -= a / 2
    return Boundary(cx=tuple(cx), sx=(0.0,) * n, cy=(0.0,) * n, sy=tuple(sy))


def kite(a: float, b: float) -> Boundary:
    """x = cos t + a cos 2t - a, y = b sin t."""
    return Boundary(cx=(-a, 1.0, a), sx=(0.0, 0.0, 0.0), cy=(0.0, 0.0, 0.0), sy=(0.0, b, 0.0))


@dataclass(frozen=True)
class Grid:
    a0: float
    b0: float
    h: float
    nx: int
    ny: int

    def coords(self):
        x = self.a0 + self.h * np.arange(self.nx)
        y = self.b0 + self.h * np.arange(self.ny)
        return x, y


@dataclass(frozen=True)
class Params:
    d: int = 5
    C: int = 27
    Z: int = 12
    n_os: int = 20
    n_r: int = 6
    M: int = 8
    B: int = 256
    m_F: int = 20
    k1: float = 0.0


@dataclass(frozen=True)
class Workload:
    name: str
    boundary: Boundary
    grid: Grid
    params: Params
    note: str = ""


def _sq(a0, b0, side, n):
    return Grid(a0=a0, b0=b0, h=side / n, nx=n, ny=n)


WORKLOADS = {
    # FP64 plain 2D-FC: unit disk in [-1.5, 1.5)^2 at 128^2 with 256 normals.  The
    # strip 27*k1 must stay inside the box: k1 = 0.015 < h = 0.0234.
    "disk128": Workload("disk128", disk(), _sq(-1.5, -1.5, 3.0, 128),
                        Params(B=256, k1=0.015)),
    # Star r = 1 + 0.3 cos 5 theta at 1024^2, 2048 normals.  Concave radius 0.0721,
    # so k1 = 0.0013 (half of it over C) < h = 0.00254.
    "star1024": Workload("star1024", star(0.3, 5), _sq(-1.1955, -1.3, 2.6, 1024),
                         Params(B=2048, k1=0.0013)),
    # Kite x = cos t + 0.65 cos 2t - 0.65, y = 1.5 sin t at 4096^2, 8192 normals;
    # concave radius 1.41, so k1 = h.
    "kite4096": Workload("kite4096", kite(0.65, 1.5), _sq(-1.776, -1.53, 3.06, 4096),
                         Params(B=8192, k1=3.06 / 4096)),
    # The same kite at 2048^2 (the Fourier Forwarding workload) and 1024^2: square
    # grids fitted to the curve's box plus the strip (h = 1.51e-3 and 3.12e-3; the
    # 3.06-wide box of the 4096^2 grid leaves 0.03 in y, less than C h at these steps).
    "kite2048": None,
    "kite1024": None,
    # Small cases for CPU tests and quick parity: several tiles and ragged sizes.
    "disk64": Workload("disk64", disk(), _sq(-2.0, -2.0, 4.0, 64), Params(B=128, k1=0.03)),
    "kite160x144": Workload("kite160x144", kite(0.65, 1.5),
                            Grid(a0=-3.17, b0=-2.63, h=0.0366, nx=160, ny=144),
                            Params(B=320, k1=0.0366)),
    "star200": Workload("star200", star(0.15, 3), Grid(a0=-1.5167, b0=-1.6667, h=1 / 60,
                                                      nx=200, ny=200),
                        Params(B=400, k1=1 / 60)),
}


def fit_grid(xmin, xmax, ymin, ymax, h, C=27, k1=None, margin=4) -> Grid:
    """Smallest grid of step h (plus a margin of cells) holding the box
    [xmin, xmax] x [ymin, ymax] widened by the strip width C*k1 on every side."""
    k1 = h if k1 is None else k1
    nx = int(math.ceil((xmax - xmin + 2 * C * k1) / h)) + 2 * margin
    ny = int(math.ceil((ymax - ymin + 2 * C * k1) / h)) + 2 * margin
    return Grid(a0=0.5 * (xmin + xmax) - 0.5 * nx * h, b0=0.5 * (ymin + ymax) - 0.5 * ny * h,
                h=h, nx=nx, ny=ny)


def next_smooth_even(n: int) -> int:
    """Smallest even m >= n of the form 2^a 3^b 5^c (a DFT-friendly length)."""
    m = n + (n & 1)
    while True:
        r = m
        for q in (2, 3, 5):
            while r % q == 0:
                r //= q
        if r == 1:
            return m
        m += 2


def fit_grid_smooth(xmin, xmax, ymin, ymax, h, C=27, margin=4) -> Grid:
    """fit_grid with both sizes raised to the next even 2^a 3^b 5^c, same centre."""
    g = fit_grid(xmin, xmax, ymin, ymax, h, C=C, margin=margin)
    nx, ny = next_smooth_even(g.nx), next_smooth_even(g.ny)
    return Grid(a0=0.5 * (xmin + xmax) - 0.5 * nx * h, b0=0.5 * (ymin + ymax) - 0.5 * ny * h,
                h=h, nx=nx, ny=ny)


def far_inside(boundary: Boundary, xs, ys, dmin: float, n: int = 20000) -> np.ndarray:
    """Mask [len(ys)][len(xs)] of the grid points inside the curve at a distance
    greater than dmin from it (where errors are measured away from the boundary).  The
    curve is sampled at n points (spacing ~2.5e-4 on the test domains, so distances are
    overestimated by at most about half of that): the distance test is a
    nearest-neighbour search among the samples, the inside test an even-odd count of
    polygon crossings along each row."""
    from scipy.spatial import cKDTree
    cx, cy = boundary.polygon(n)
    X, Y = np.meshgrid(xs, ys)
    d, _ = cKDTree(np.column_stack([cx, cy])).query(
        np.column_stack([X.ravel(), Y.ravel()]), distance_upper_bound=dmin, workers=-1)
    far = np.isinf(d).reshape(X.shape)
    x2, y2 = np.roll(cx, -1), np.roll(cy, -1)
    inside = np.zeros(X.shape, bool)
    for r, y in enumerate(ys):
        e = (cy > y) != (y2 > y)
        xc = np.sort(cx[e] + (y - cy[e]) * (x2[e] - cx[e]) / (y2[e] - cy[e]))
        for a, b in zip(xc[0::2], xc[1::2]):
            inside[r] |= (xs > a) & (xs < b)
    return far & inside


def star_min_radius(a: float, k: int, n: int = 8192) -> float:
    """Smallest radius of curvature of r = 1 + a cos(k theta) (sampled): 1/max kappa with
    kappa = |r^2 + 2 r'^2 - r r''| / (r^2 + r'^2)^(3/2)."""
    th = 2 * np.pi * np.arange(n) / n
    r = 1 + a * np.cos(k * th)
    r1 = -a * k * np.sin(k * th)
    r2 = -a * k * k * np.cos(k * th)
    kappa = np.abs(r * r + 2 * r1 * r1 - r * r2) / (r * r + r1 * r1) ** 1.5
    return float(1.0 / kappa.max())


def square_grid_for(boundary: Boundary, N: int, rho_min: float, C: int = 27,
                    margin: int = 4) -> tuple:
    """An N x N grid centred on the curve's bounding box, and k1.  The strip step is
    k1 = min(h, rho_min / (2C)) (the strip C k1 stays within half the smallest radius of
    curvature), and h = (W + 2 C k1) / (N - 2 margin) with W the larger side of the
    bounding box, so the strip ends `margin` cells inside the grid on every side."""
    px, py = boundary.polygon(8192)
    xmin, xmax, ymin, ymax = px.min(), px.max(), py.min(), py.max()
    W = max(xmax - xmin, ymax - ymin)
    cap = rho_min / (2 * C)
    h = W / (N - 2 * margin - 2 * C)           # k1 = h
    k1 = h
    if h > cap:
        k1 = cap
        h = (W + 2 * C * k1) / (N - 2 * margin)
    xc, yc = 0.5 * (xmin + xmax), 0.5 * (ymin + ymax)
    return Grid(a0=xc - 0.5 * N * h, b0=yc - 0.5 * N * h, h=h, nx=N, ny=N), k1


STAR_SIZES = (256, 384, 512, 640, 768, 1024, 1536, 2048)


def stars8(seed: int = 4, sizes=STAR_SIZES) -> list:
    """Eight stars r = 1 + a cos(k theta), a ~ U[0.1, 0.3], k ~ U{3..7} (seeded), each on
    a square grid: the more concave a star (smaller radius of curvature), the larger its
    grid.  B: the multiple of 32 at or above the perimeter over h."""
    u = uniform(seed, 16)
    shapes = [(0.1 + 0.2 * u[2 * i], 3 + int(5 * u[2 * i + 1])) for i in range(8)]
    rho = [star_min_radius(a, k) for a, k in shapes]
    order = np.argsort(rho)[::-1]              # least concave first -> smallest grid
    out = [None] * 8
    for rank, i in enumerate(order):
        a, k = shapes[i]
        bd = star(a, k)
        N = sorted(sizes)[rank]
        grid, k1 = square_grid_for(bd, N, rho[i])
        px, py = bd.polygon(8192)
        L = float(np.sum(np.hypot(np.diff(np.append(px, px[0])), np.diff(np.append(py, py[0])))))
        B = int(math.ceil(L / grid.h / 32.0)) * 32
        out[i] = Workload(f"star{i}_{N}", bd, grid, Params(B=B, k1=k1),
                          note=f"a={a:.4f} k={k} rho_min={rho[i]:.4f}")
    return out


def _fitted_kite(name: str, N: int, B: int) -> Workload:
    b = kite(0.65, 1.5)
    g, k1 = square_grid_for(b, N, 1.41)
    return Workload(name, b, g, Params(B=B, k1=float(k1)))


WORKLOADS["kite2048"] = _fitted_kite("kite2048", 2048, 4096)
WORKLOADS["kite1024"] = _fitted_kite("kite1024", 1024, 2048)


def workload(name: str, **overrides) -> Workload:
    w = WORKLOADS[name]
    if overrides:
        w = replace(w, params=replace(w.params, **overrides))
    return w


# --------------------------------------------------------------------------- #
# Closed-form test functions (vectorised over numpy arrays)
# --------------------------------------------------------------------------- #
def f_expsincos(x, y):
    """exp(sin 3x + cos 2y)."""
    return np.exp(np.sin(3 * x) + np.cos(2 * y))


def f_sin5pi(x, y):
    """-sin(5 pi x) sin(5 pi y)."""
    return -np.sin(5 * np.pi * x) * np.sin(5 * np.pi * y)


def f_kite_paper(x, y):
    """-(x^6 + y^6) sin(10 pi x) sin(10 pi y)."""
    return -(x ** 6 + y ** 6) * np.sin(10 * np.pi * x) * np.sin(10 * np.pi * y)


def u_manufactured(x, y):
    """u = sin(2x) e^y; its Laplacian is -3 sin(2x) e^y."""
    return np.sin(2 * x) * np.exp(y)


def lap_u_manufactured(x, y):
    return -3.0 * np.sin(2 * x) * np.exp(y)


def polynomial(px: int, py: int):
    """x^px y^py."""
    return lambda x, y: (x ** px) * (y ** py)


def _inside_polygon(px, py, vx, vy):
    """Even-odd crossing test of points (px, py) against a polygon (input sampling)."""
    inside = np.zeros(px.shape, dtype=bool)
    n = len(vx)
    for k in range(n):
        x1, y1, x2, y2 = vx[k], vy[k], vx[(k + 1) % n], vy[(k + 1) % n]
        cond = (y1 > py) != (y2 > py)
        xint = x1 + (py - y1) * (x2 - x1) / (y2 - y1 + (y2 == y1))
        inside ^= cond & (px < xint)
    return inside


@dataclass
class GaussianSum:
    """sum_i a_i exp(-|r - c_i|^2 / (2 w_i^2))."""
    a: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    w: np.ndarray

    def __call__(self, x, y):
        out = np.zeros(np.broadcast(x, y).shape)
        for a, cx, cy, w in zip(self.a, self.cx, self.cy, self.w):
            out = out + a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * w * w))
        return out


def gaussian_sum(boundary: Boundary, n: int, seed: int, wmin=0.1, wmax=0.3,
                 margin: float = 0.0) -> GaussianSum:
    """n Gaussians with centres uniform in the domain (rejection; with `margin`, only
    centres at least that far from the curve), widths U[wmin, wmax] and amplitudes
    N(0, 1)."""
    vx, vy = boundary.polygon()
    x0, x1, y0, y1 = vx.min(), vx.max(), vy.min(), vy.max()
    cx, cy = [], []
    ctr = 0
    while len(cx) < n:
        u = uniform(seed * 7919 + 1 + ctr, 64)
        ctr += 1
        px = x0 + (x1 - x0) * u[0::2]
        py = y0 + (y1 - y0) * u[1::2]
        ok = _inside_polygon(px, py, vx, vy)
        if margin > 0:
            dist = np.sqrt(((px[:, None] - vx[None, :]) ** 2 +
                            (py[:, None] - vy[None, :]) ** 2).min(axis=1))
            ok &= dist >= margin
        for a, b, o in zip(px, py, ok):
            if o and len(cx) < n:
                cx.append(a)
                cy.append(b)
    w = wmin + (wmax - wmin) * uniform(seed * 7919, n)
    a = normal(seed * 7919 + 100003, n)
    return GaussianSum(a=a, cx=np.array(cx), cy=np.array(cy), w=w)


@dataclass
class TrigSum:
    """T^{-1/2} sum over (p, q) with |p|+|q| <= deg in a half-plane of
    alpha cos(p x + q y) + beta sin(p x + q y), alpha, beta ~ N(0, 1)."""
    p: np.ndarray
    q: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray

    def __call__(self, x, y):
        out = np.zeros(np.broadcast(x, y).shape)
        s = 1.0 / math.sqrt(len(self.p))
        for p, q, al, be in zip(self.p, self.q, self.alpha, self.beta):
            ph = p * x + q * y
            out = out + s * (al * np.cos(ph) + be * np.sin(ph))
        return out


def trig_grid(t: TrigSum, xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    """t on the tensor grid (ys x xs), shape [len(ys)][len(xs)], evaluated separably:
    cos(px + qy) = cos px cos qy - sin px sin qy, sin(px + qy) = sin px cos qy +
    cos px sin qy, so the sum is Y^T G X with X = [cos px; sin px], Y = [cos qy; sin qy]."""
    ps = np.unique(t.p)
    qs = np.unique(t.q)
    pi = {v: i for i, v in enumerate(ps)}
    qi = {v: i for i, v in enumerate(qs)}
    npx, nqy = len(ps), len(qs)
    G = np.zeros((2 * nqy, 2 * npx))
    s = 1.0 / math.sqrt(len(t.p))
    for p, q, al, be in zip(t.p, t.q, t.alpha, t.beta):
        a, b = pi[p], qi[q]
        G[b, a] += s * al               # cos qy cos px
        G[nqy + b, npx + a] -= s * al   # sin qy sin px
        G[b, npx + a] += s * be         # cos qy sin px
        G[nqy + b, a] += s * be         # sin qy cos px
    X = np.concatenate([np.cos(np.outer(ps, xs)), np.sin(np.outer(ps, xs))])
    Y = np.concatenate([np.cos(np.outer(qs, ys)), np.sin(np.outer(qs, ys))])
    return Y.T @ (G @ X)


def star_functions(w: Workload, index: int, n: int = 32) -> list:
    """The n trigonometric sums (degree 12) of star `index` of the batched workload."""
    return [trig_sum(12, 4 * 1000 + 32 * index + m) for m in range(n)]


def trig_sum(deg: int, seed: int) -> TrigSum:
    pq = [(p, q) for p in range(0, deg + 1) for q in range(-deg, deg + 1)
          if abs(p) + abs(q) <= deg and (p > 0 or q >= 0)]
    p = np.array([t[0] for t in pq], dtype=np.float64)
    q = np.array([t[1] for t in pq], dtype=np.float64)
    al = normal(seed * 104729, len(pq))
    be = normal(seed * 104729 + 1, len(pq))
    return TrigSum(p=p, q=q, alpha=al, beta=be)


def grid_values(w: Workload, f, n_f: int = 1) -> np.ndarray:
    """f on every grid point, shape [ny][nx] (values outside the domain are garbage
    the method must ignore: here simply f itself)."""
    x, y = w.grid.coords()
    X, Y = np.meshgrid(x, y)
    return f(X, Y)
