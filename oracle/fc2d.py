"""Oracle: the 2D-FC Cartesian evaluation (Sections 3.2, 3.4, 3.5 steps 5-7).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

extension(geo, mats, f_grid, f_bdry) -> f^c on the grid H   (steps 5 and 6)
coefficients(ext)                    -> hat f^c, eq. (3.1)  (step 7)
extension_complex, coefficients_complex: the same for complex f (full spectrum)

Matching values (Section 3.2, "two-step polynomial interpolation"), reading:
* Normal p with foot b = q(theta_p), outward normal n.  If |n_x| >= |n_y| (with a
  relative tie margin of 2^-30 in favour of the vertical case, so that an exact 45
  degree normal is treated the same by every implementation) the red stars lie on
  vertical grid lines, else on horizontal ones; below, the vertical case (the other
  swaps x and y).
* sigma = sign(n_x).  The M-1 lines are i_k = i_0 - sigma*k, k = 0..M-2, where i_0 is
  the first grid line at least h/2 inside b along the normal: i_0 =
  floor((b_x - h n_x/2 - a0)/h) if sigma > 0 else ceil(...).  Line k meets the normal
  at t_k = (x_{i_k} - b_x)/n_x <= -h/2 (the red star R_k = b + t_k n).  Starting half
  a cell in keeps the first line away from tangency with the curve at b, where its
  inside chord would hold no grid node.
* The value at R_k is the degree <= M-1 Lagrange interpolant along line i_k of the
  candidates, in increasing y: the lower "square" (the crossing Y_lo of the line with
  the curve that bounds the inside interval containing R_k), the grid nodes in
  [Y_lo, Y_hi] (the first and last are dropped when closer than h/2 to the square),
  and the upper square Y_hi.  Of these, the M consecutive candidates with ceil(M/2)
  at or below R_k are used (the window is clamped to the list; a list shorter than M
  is used whole).  Square values are boundary data.
* The matching value at r_{p,q} (eq. (3.5); t = (q-d+1) k1) is the degree M-1 Lagrange
  interpolant in t over M nodes: t = 0 with the boundary datum f(b) and the M-1 red
  stars, q = 0..d-2; r_{p,d-1} = b takes the boundary datum itself.
Interior data only (Remark 3.2 II: no boundary values given), reading: the same lines
  and red stars, each star interpolated from the grid nodes of its inside interval
  alone (no squares, no node dropped), the M consecutive nodes with ceil(M/2) at or
  below R_k; along the normal the degree M-2 Lagrange interpolant over the M-1 red
  stars, evaluated at every matching point r_{p,q}, q = 0..d-1, including the foot b
  itself (q = d-1, an extrapolation), whose value also serves as F_{p,0}.
Blending (eq. (2.6) with A_r of Remark 2.2): F_{p,0} = f(b) and
F_{p,q} = (A_r (Q^T f_{D_p}))_q for q = 1..C_r, evaluated right to left.
Interpolation onto H cap V+ (Section 3.4), reading:
* p0 = floor(theta^Q/k2); the re-centred set S_{theta^Q} is p0-K_l .. p0+K_r (mod B),
  K_l = ceil(M/2)-1, K_r = floor(M/2) (eq. (3.8) with K_r = K_l + 1 for even M).
* Along each of these normals the value at distance eta_Q is the degree M-1 Lagrange
  interpolant over the fine nodes q = s..s+M-1 (spacing k1/n_r),
  s = clamp(floor(u) - K_l, 0, C_r + 1 - M), u = eta_Q n_r/k1.
* The final value is the degree M-1 Lagrange interpolant in theta over S_{theta^Q}.
Grid points inside keep f; strip points get the interpolant; all others are 0.

Parity of the extension digits is unpinned by the paper (they depend on the
readings above); it is pinned by polynomial reproduction, linearity, exactness inside
and zero beyond the strip, and convergence orders (tests/test_oracle_fc2d.py).
"""
from __future__ import annotations

import math

import numpy as np

TIE = 2.0 ** -30  # relative tie margin for |n_x| >= |n_y|
DROP = 0.5        # grid nodes closer than DROP*h to a square are not used


def lagrange_weights(nodes, t):
    """L_k(t) = prod_{m != k} (t - x_m)/(x_k - x_m)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    n = len(nodes)
    w = np.ones(n)
    for k in range(n):
        for m in range(n):
            if m != k:
                w[k] *= (t - nodes[m]) / (nodes[k] - nodes[m])
    return w


def _line_candidates(coord_nodes, cross, star, h, drop=DROP, squares=True):
    """Candidates (coordinate, kind, index) on one grid line around the red star.

    coord_nodes: coordinates of the grid nodes along the line; cross: sorted crossings
    of the line with the curve.  kind 0 = grid node (index along the line), kind 1 =
    square (index into ``cross``).  squares=False (interior data only): the grid nodes
    of the inside interval alone, none dropped."""
    m = np.searchsorted(cross, star, side="right") - 1
    if m < 0 or m % 2 == 1 or m + 1 >= len(cross):
        raise ValueError("red star outside the domain along its grid line")
    lo, hi = cross[m], cross[m + 1]
    o, step = coord_nodes[0], coord_nodes[1] - coord_nodes[0]
    jl = int(math.ceil((lo - o) / step))
    jh = int(math.floor((hi - o) / step))
    jl = max(jl, 0)
    jh = min(jh, len(coord_nodes) - 1)
    while jl <= jh and coord_nodes[jl] < lo:
        jl += 1
    while jh >= jl and coord_nodes[jh] > hi:
        jh -= 1
    if not squares:
        return [(coord_nodes[j], 0, j) for j in range(jl, jh + 1)]
    if jl <= jh and coord_nodes[jl] - lo < drop * h:
        jl += 1
    if jl <= jh and hi - coord_nodes[jh] < drop * h:
        jh -= 1
    cands = [(lo, 1, m)] + [(coord_nodes[j], 0, j) for j in range(jl, jh + 1)] + [(hi, 1, m + 1)]
    return cands


def _choose_window(cands, star, M):
    n = len(cands)
    if n <= M:
        return cands
    c = sum(1 for v in cands if v[0] <= star)
    s = min(max(c - (M + 1) // 2, 0), n - M)
    return cands[s:s + M]


def matching_stencils(geo, interior=False):
    """Per normal p: the red-star parameters t_k, for each red star a dict
    {("g", lin) or ("b", idx): weight} over grid values and boundary data, and the
    along-normal weights giving f(r_{p,q}), q = 0..d-2, from the boundary datum and
    the red stars (Section 3.2).  interior: interior data only (Remark 3.2 II), the
    weights give f(r_{p,q}), q = 0..d-1, from the red stars alone."""
    g, p = geo.grid, geo.params
    M, d, h = p.M, p.d, g.h
    out = []
    for k in range(p.B):
        bxk, byk, nxk, nyk = geo.bx[k], geo.by[k], geo.nx_[k], geo.ny_[k]
        vertical = abs(nxk) >= abs(nyk) * (1.0 - TIE)
        if vertical:
            base, nb, other_b, other_n = bxk, nxk, byk, nyk
            o0, nlines = g.a0, g.nx
            line_coord, node_coords, crosses = geo.xs, geo.ys, geo.col_cross
            offs = geo.col_offset
        else:
            base, nb, other_b, other_n = byk, nyk, bxk, nxk
            o0, nlines = g.b0, g.ny
            line_coord, node_coords, crosses = geo.ys, geo.xs, geo.row_cross
            offs = geo.row_offset
        sigma = 1 if nb > 0 else -1
        xi = (base - 0.5 * h * nb - o0) / h
        i0 = math.floor(xi) if sigma > 0 else math.ceil(xi)
        tk = [] if interior else [0.0]
        star_terms = [] if interior else [{("b", k): 1.0}]
        for kk in range(M - 1):
            li = i0 - sigma * kk
            if li < 0 or li >= nlines:
                raise ValueError("matching stencil leaves the grid")
            t = (line_coord[li] - base) / nb
            star = other_b + t * other_n
            cands = _choose_window(_line_candidates(node_coords, crosses[li], star, h,
                                                    squares=not interior), star, M)
            wv = lagrange_weights([c[0] for c in cands], star)
            terms = {}
            for (coord, kind, idx), wgt in zip(cands, wv):
                if kind == 0:
                    lin = (idx * g.nx + li) if vertical else (li * g.nx + idx)
                    key = ("g", lin)
                else:
                    key = ("b", int(offs[li] + idx))
                terms[key] = terms.get(key, 0.0) + wgt
            tk.append(t)
            star_terms.append(terms)
        nq = d if interior else d - 1
        wns = [lagrange_weights(tk, (q - d + 1) * p.k1) for q in range(nq)]
        out.append({"t": tk, "stars": star_terms, "wn": wns, "interior": interior})
    return out


def matching_values(geo, stencils, f_grid, f_bdry):
    """f_{D_p}: [B][d] matching values (q = d-1 is the boundary datum at the node; with
    interior stencils and f_bdry None, its extrapolation from the red stars)."""
    p = geo.params
    fg = np.asarray(f_grid, dtype=np.float64).ravel()
    fb = None if f_bdry is None else np.asarray(f_bdry, dtype=np.float64)
    fD = np.zeros((p.B, p.d))
    for k, st in enumerate(stencils):
        stars = np.array([sum(wgt * (fg[key[1]] if key[0] == "g" else fb[key[1]])
                              for key, wgt in terms.items()) for terms in st["stars"]])
        for q in range(len(st["wn"])):
            fD[k, q] = float(np.dot(st["wn"][q], stars))
        if not st.get("interior", False):
            fD[k, p.d - 1] = fb[k]
    return fD


def blend(mats, fD):
    """Strip values F[p][q], q = 0..C_r: F[p][0] = boundary datum,
    F[p][1:] = A_r (Q^T f_{D_p}) (eq. (2.6), Remark 2.2)."""
    c = fD @ mats["Q"]              # row p holds (Q^T f_{D_p})^T
    Fr = c @ mats["Ar"].T           # row p holds (A_r c)^T
    return np.concatenate([fD[:, -1:], Fr], axis=1)


def interpolate_strip(geo, F):
    """Continuation values at the strip points (Section 3.4)."""
    p = geo.params
    M, B, Cr = p.M, p.B, p.C * p.n_r
    Kl = (M + 1) // 2 - 1
    k2 = 2 * np.pi / B
    n = len(geo.strip_lin)
    tt = geo.strip_theta / k2
    p0 = np.floor(tt).astype(np.int64)
    u = geo.strip_eta * p.n_r / p.k1
    s = np.clip(np.floor(u).astype(np.int64) - Kl, 0, Cr + 1 - M)
    wth = _lagrange_equispaced(M, tt - (p0 - Kl))     # [n][M]
    weta = _lagrange_equispaced(M, u - s)              # [n][M]
    rows = np.mod(p0[:, None] - Kl + np.arange(M)[None, :], B)    # [n][M]
    cols = s[:, None] + np.arange(M)[None, :]                      # [n][M]
    vals = F[rows[:, :, None], cols[:, None, :]]                   # [n][M][M]
    return np.einsum("na,nab,nb->n", wth, vals, weta)


def _lagrange_equispaced(M, t):
    """Lagrange weights of the nodes 0..M-1 at each t (vector): [len(t)][M]."""
    t = np.asarray(t, dtype=np.float64)
    w = np.ones((len(t), M))
    for k in range(M):
        for m in range(M):
            if m != k:
                w[:, k] *= (t - m) / (k - m)
    return w


def extension(geo, mats, f_grid, f_bdry, stencils=None):
    """f^c on H: f inside, interpolated continuation on H cap V+, 0 elsewhere.
    f_bdry None: interior data only (Remark 3.2 II)."""
    if stencils is None:
        stencils = matching_stencils(geo, interior=f_bdry is None)
    fD = matching_values(geo, stencils, f_grid, f_bdry)
    F = blend(mats, fD)
    vals = interpolate_strip(geo, F)
    ext = np.where(geo.inside, np.asarray(f_grid, dtype=np.float64), 0.0)
    flat = ext.ravel()
    flat[geo.strip_lin] = vals
    return flat.reshape(ext.shape)


def coefficients(ext):
    """hat f^c_{l,m} = (1/(Nx Ny)) sum_{i,j} f^c_{ij} exp(-2 pi i (l i/Nx + m j/Ny)),
    the R2C half spectrum [Ny][Nx/2+1] in DFT index order (eq. (3.1), step 7).
    numpy's FFT serves as the library primitive for the DFT."""
    ny, nx = ext.shape
    return np.fft.rfft2(ext) / (nx * ny)


def extension_complex(geo, mats, f_grid, f_bdry, stencils=None):
    """f^c of a complex f (Section 3: f maps the domain to C): every step is linear and
    real, so f^c = (Re f)^c + i (Im f)^c.  f_grid complex [ny][nx]; f_bdry complex or None."""
    fg = np.asarray(f_grid)
    fb = None if f_bdry is None else np.asarray(f_bdry)
    re = extension(geo, mats, fg.real, None if fb is None else fb.real, stencils)
    im = extension(geo, mats, fg.imag, None if fb is None else fb.imag, stencils)
    return re + 1j * im


def coefficients_complex(ext):
    """hat f^c_{l,m} of eq. (3.1) for complex data: the full spectrum [Ny][Nx] in DFT
    index order (l > Nx/2 and m > Ny/2 stand for l - Nx and m - Ny).  numpy's FFT
    serves as the library primitive for the DFT."""
    ny, nx = ext.shape
    return np.fft.fft2(ext) / (nx * ny)


def dft_bruteforce_complex(ext):
    """The full spectrum by the O(N^4) definition (small grids only)."""
    ny, nx = ext.shape
    i = np.arange(nx)
    j = np.arange(ny)
    out = np.zeros((ny, nx), dtype=np.complex128)
    for m in range(ny):
        for l in range(nx):
            ph = np.exp(-2j * np.pi * (l * i[None, :] / nx + m * j[:, None] / ny))
            out[m, l] = np.sum(ext * ph) / (nx * ny)
    return out


def dft_bruteforce(ext):
    """The same half spectrum by the O(N^4) definition (small grids only)."""
    ny, nx = ext.shape
    out = np.zeros((ny, nx // 2 + 1), dtype=np.complex128)
    i = np.arange(nx)
    j = np.arange(ny)
    for m in range(ny):
        for l in range(nx // 2 + 1):
            ph = np.exp(-2j * np.pi * (l * i[None, :] / nx + m * j[:, None] / ny))
            out[m, l] = np.sum(ext * ph) / (nx * ny)
    return out


def boundary_values(geo, f):
    """f at every boundary data point (B nodes, column crossings, row crossings)."""
    return f(geo.bdry_x, geo.bdry_y)
