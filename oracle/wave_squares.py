"""Oracle: the Fourier Forwarding small-square interface procedure (Section 4.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper gives U_B's values at the inner edge of the near-boundary region not by
evaluating the full 2D-FC expansion U_FC at every small step but from solutions "similar
to (4.8), without boundary conditions, over some small square regions contained in
Omega and centred at points on the interior boundary of Omega minus Omega_Delta T",
detailed in the authors' FF paper.  Reading (the steps the library follows):

* Squares.  A square is the (2a+1) x (2a+1) block of grid points around a centre grid
  point c, all of them inside the domain; a = (P - C - 1)/2 with the periodic length
  P = 64 and the 1D-FC continuation length C = 27 (the 2D-FC's), so a = 18.
* Validity.  The solution at an interface point q is U_FC's domain-of-dependence value
  for t - T_j <= Delta T = n_c h / c when the disk of radius n_c h around q lies in the
  square: |q - c|_inf <= R = a - n_c (grid units).  For a straight boundary at 45
  degrees a square inside the domain can serve q only if q is at least sqrt(2) n_c h
  from the curve, so the near-boundary band in this mode reaches
  (ceil(sqrt(2) n_c) + 2) h from the curve (instead of (n_c + 2) h).
* Placement (deterministic).  Interface points in increasing linear index; for the first
  one q not yet served, every centre c with |c - q|_inf <= R whose square is inside is a
  candidate; the one serving the most unserved interface points (|p - c|_inf <= R) wins,
  ties to the smaller (row, column); it serves all of them.  No candidate: an error.
* Expansion, once per large step.  The square's values of u(T_j) and u_t(T_j): each of
  its 2a+1 rows continued by the 1D-FC of eq. (2.7) (the d = 4 matching values at each
  end, A Q^T with the coarse continuation matrix A, C values) to P = 2a+1+C values, then
  each of the P columns the same way; the normalised 2D DFT gives hat f and hat g on the
  P x P box of period P h.
* Evaluation, every small step s < S.  a(s Delta t) of eq. (4.12) with the box's
  frequencies w = 2 pi c sqrt((l/(P h))^2 + (m/(P h))^2) (signed l, m), inverse DFT, the
  real value at each served interface point.  At T_{j+1} (the merge and the extra step
  for u_t) the full U_FC is used as in the exact mode.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from oracle import fc1d

P_BOX = 64   # periodic length of a square's expansion (grid points)


def band_reach_cells(n_c: int) -> int:
    """The band's reach from the curve in the small-square mode, in grid units."""
    return int(math.ceil(math.sqrt(2.0) * n_c)) + 2


def half_width(C: int = 27, P: int = P_BOX) -> int:
    return (P - C - 1) // 2


@dataclass
class Squares:
    a: int                       # half-width (grid units)
    R: int                       # service radius a - n_c
    centres: np.ndarray          # [n_sq][2] (j, i) grid indices of the centres
    served: list                 # per square: array of interface indices it serves
    owner: np.ndarray            # per interface point: its square


def place(geo, iface_lin, n_c: int, C: int = 27, P: int = P_BOX) -> Squares:
    """Square placement of the reading above."""
    ny, nx = geo.inside.shape
    a = half_width(C, P)
    R = a - n_c
    if R < 0:
        raise ValueError("n_c too large for the square size")
    ins = geo.inside.astype(np.int64)
    S = np.zeros((ny + 1, nx + 1), np.int64)  # summed-area table of the inside mask
    S[1:, 1:] = np.cumsum(np.cumsum(ins, axis=0), axis=1)

    def square_inside(j, i):
        j0, j1, i0, i1 = j - a, j + a + 1, i - a, i + a + 1
        if j0 < 0 or i0 < 0 or j1 > ny or i1 > nx:
            return False
        return S[j1, i1] - S[j0, i1] - S[j1, i0] + S[j0, i0] == (2 * a + 1) ** 2

    qj, qi = np.divmod(np.asarray(iface_lin, dtype=np.int64), nx)
    n = len(iface_lin)
    owner = -np.ones(n, np.int64)
    centres, served = [], []
    for t in np.argsort(np.asarray(iface_lin), kind="stable"):
        if owner[t] >= 0:
            continue
        # only interface points within 2R of q can be served by a candidate
        loc = np.nonzero((np.abs(qj - qj[t]) <= 2 * R) & (np.abs(qi - qi[t]) <= 2 * R))[0]
        best = None
        for dj in range(-R, R + 1):
            for di in range(-R, R + 1):
                cj, ci = qj[t] + dj, qi[t] + di
                if not square_inside(cj, ci):
                    continue
                near = loc[(np.abs(qj[loc] - cj) <= R) & (np.abs(qi[loc] - ci) <= R) &
                           (owner[loc] < 0)]
                key = (-len(near), cj, ci)
                if best is None or key < best[0]:
                    best = (key, cj, ci, near)
        if best is None:
            raise ValueError(f"no square inside the domain serves interface point {iface_lin[t]}")
        _, cj, ci, near = best
        k = len(centres)
        owner[near] = k
        centres.append((cj, ci))
        served.append(np.sort(near))
    return Squares(a=a, R=R, centres=np.array(centres, dtype=np.int64).reshape(-1, 2),
                   served=served, owner=owner)


def continue_2d(mats, block, P: int = P_BOX):
    """1D-FC (eq. (2.7)) of every row, then of every column: the P x P periodic values
    (the square's 2a+1 points plus the C continuation points fill P exactly)."""
    rows = np.array([fc1d.fc1d_values(mats, r) for r in block])      # [n][n + C]
    if rows.shape[1] != P:
        raise ValueError("square side + C must equal the periodic length")
    return np.array([fc1d.fc1d_values(mats, c) for c in rows.T]).T   # [P][P]


def square_spectra(geo, mats, sq: Squares, u, ut, P: int = P_BOX):
    """Normalised 2D DFTs (hat f, hat g) of every square's continued u and u_t."""
    a = sq.a
    out = []
    for (cj, ci) in sq.centres:
        bu = u[cj - a:cj + a + 1, ci - a:ci + a + 1]
        bt = ut[cj - a:cj + a + 1, ci - a:ci + a + 1]
        Fh = np.fft.fft2(continue_2d(mats, bu, P)) / (P * P)
        Gh = np.fft.fft2(continue_2d(mats, bt, P)) / (P * P)
        out.append((Fh, Gh))
    return out


def box_frequencies(h, c, P: int = P_BOX):
    k = np.fft.fftfreq(P, 1.0 / P)
    L = P * h
    return 2 * np.pi * c * np.sqrt((k[None, :] / L) ** 2 + (k[:, None] / L) ** 2)


def evaluate(geo, sq: Squares, spectra, iface_lin, h, c, tau, P: int = P_BOX):
    """U at every interface point at time tau after the expansion, from its square."""
    nx = geo.inside.shape[1]
    w = box_frequencies(h, c, P)
    wz = np.where(w == 0, 1.0, w)
    out = np.zeros(len(iface_lin))
    a = sq.a
    for k, ((cj, ci), (Fh, Gh)) in enumerate(zip(sq.centres, spectra)):
        A = Fh * np.cos(w * tau) + Gh * np.where(w == 0, tau, np.sin(w * tau) / wz)
        U = np.real(np.fft.ifft2(A * P * P))
        idx = sq.served[k]
        qj, qi = np.divmod(np.asarray(iface_lin)[idx], nx)
        out[idx] = U[qj - (cj - a), qi - (ci - a)]
    return out
