"""Oracle: the 1D blending-to-zero matrices Q, A and A_r (Section 2.2, Remark 2.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Steps, in the paper's order and notation (Section 2.2, eqs. (2.1)-(2.6), Remark 2.2):

1. Matching points x_i = i*k, 0 <= i <= d-1, with k = 1 (A and Q do not depend on k,
   end of Section 2.3).  P = (x_i^j) and P = QR by the stabilised (modified)
   Gram-Schmidt process, eq. (2.2).  Column j of Q holds the Gram polynomial g_j on D.
2. Oversampled Gram values Q_os = P_os R^{-1} on the n_os(d-1)+1 points j/n_os,
   eq. (2.3).
3. For each j the band-limited trigonometric polynomial g^c_j of eq. (2.4), period
   (d+2C+Z-1), modes -m_F..m_F, is the least-squares solution of eq. (2.5): it matches
   Q_os[:, j] on D_os and 0 on the (Z-1)n_os+1 points of [(d+C), (d+C+Z-1)] spaced
   1/n_os.  The minimiser is taken from the SVD of B_os.  Real data make the complex
   coefficients Hermitian, so the real basis {1, cos(2 pi m x/P), sin(2 pi m x/P)}
   is used; it spans the same functions.
4. A[q, j] = g^c_j(d + q), q = 0..C-1 (points dk..(d+C-1)k) and the refined
   A_r[q-1, j] = g^c_j((d-1) + q/n_r), q = 1..C_r = C n_r (Remark 2.2).

Readings (the paper does not state these):
* m_F, the number of modes, is a parameter (default 20).  With m_F = 20 the matrix
  B_os (302 x 41 for d=5, C=27, Z=12, n_os=20) has sigma_min/sigma_max ~ 4e-16: full
  numerical rank at 50 digits, so the SVD least-squares solution is the unique
  minimiser and no truncation threshold is involved.
* All arithmetic is 50-significant-digit ``decimal``; results are rounded to double
  once, at the end.

The SVD is Chan's R-SVD: Householder QR of B_os, then one-sided (Hestenes) Jacobi
on the triangular factor.  The result is cached in tests/golden by
``oracle/make_fc_matrices.py``; ``load_fc_matrices`` reads the cache or computes.
"""
from __future__ import annotations

import decimal
import os
from decimal import Decimal as D

import numpy as np

DIGITS = 50
_GOLDEN = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "tests", "golden")


def _ctx():
    c = decimal.Context(prec=DIGITS + 10)
    return c


# --------------------------------------------------------------------------- #
# Elementary functions in Decimal (own code: Machin's formula and Taylor series)
# --------------------------------------------------------------------------- #
def _arctan_inv(n: int) -> D:
    """arctan(1/n) by its Taylor series (n >= 2)."""
    x = D(1) / n
    x2 = x * x
    term = x
    s = x
    k = 1
    eps = D(10) ** (-(DIGITS + 8))
    while abs(term) > eps:
        term = -term * x2
        k += 2
        s += term / k
    return s


def decimal_pi() -> D:
    """pi from Machin's formula pi = 16 atan(1/5) - 4 atan(1/239)."""
    with decimal.localcontext(_ctx()):
        return 16 * _arctan_inv(5) - 4 * _arctan_inv(239)


def _cos_sin_small(x: D) -> tuple[D, D]:
    """cos and sin of |x| <= pi/4 by Taylor series."""
    eps = D(10) ** (-(DIGITS + 8))
    x2 = x * x
    c = D(1)
    s = x
    tc = D(1)
    ts = x
    k = 0
    while True:
        k += 2
        tc = -tc * x2 / ((k - 1) * k)
        ts = -ts * x2 / (k * (k + 1))
        c += tc
        s += ts
        if abs(tc) < eps and abs(ts) < eps:
            break
    return c, s


def cos_sin_turn(num: int, den: int, pi: D) -> tuple[D, D]:
    """cos and sin of 2*pi*num/den (an exact rational turn).

    The angle is split as o*pi/4 + phi with integer octant o and 0 <= phi < pi/4;
    phi goes through the Taylor series and the octant is a rotation.
    """
    with decimal.localcontext(_ctx()):
        r = num % den
        o = (8 * r) // den
        phi = 2 * pi * (D(8 * r - o * den) / D(8 * den))
        cp, sp = _cos_sin_small(phi)
        cb, sb = _octant(o)
        return cb * cp - sb * sp, sb * cp + cb * sp


def _octant(o: int) -> tuple[D, D]:
    """cos and sin of o*pi/4 for integer o."""
    with decimal.localcontext(_ctx()):
        h = D(2).sqrt() / 2
        table = [(D(1), D(0)), (h, h), (D(0), D(1)), (-h, h),
                 (D(-1), D(0)), (-h, -h), (D(0), D(-1)), (h, -h)]
        return table[o % 8]


# --------------------------------------------------------------------------- #
# Dense linear algebra in Decimal
# --------------------------------------------------------------------------- #
def gram_qr(d: int):
    """Modified Gram-Schmidt QR of P = (x_i^j), x_i = i (eq. (2.2))."""
    with decimal.localcontext(_ctx()):
        P = [[D(i) ** j if j > 0 else D(1) for j in range(d)] for i in range(d)]
        V = [[P[i][j] for i in range(d)] for j in range(d)]  # columns
        R = [[D(0)] * d for _ in range(d)]
        Qc = []
        for j in range(d):
            v = V[j][:]
            for k in range(j):
                r = sum(Qc[k][i] * v[i] for i in range(d))
                R[k][j] = r
                v = [v[i] - r * Qc[k][i] for i in range(d)]
            nrm = sum(t * t for t in v).sqrt()
            R[j][j] = nrm
            Qc.append([t / nrm for t in v])
        Q = [[Qc[j][i] for j in range(d)] for i in range(d)]
        return Q, R


def _householder_qr(A):
    """Householder QR of an m x n list-of-rows matrix, m >= n.

    Returns (vs, betas, R) where the reflectors H_k = I - beta_k v_k v_k^T map A to R.
    """
    m = len(A)
    n = len(A[0])
    R = [row[:] for row in A]
    vs, betas = [], []
    for k in range(n):
        x = [R[i][k] for i in range(k, m)]
        alpha = sum(t * t for t in x).sqrt()
        if x[0] > 0:
            alpha = -alpha
        v = x[:]
        v[0] -= alpha
        vv = sum(t * t for t in v)
        beta = D(2) / vv if vv != 0 else D(0)
        for j in range(k, n):
            s = sum(v[i - k] * R[i][j] for i in range(k, m)) * beta
            for i in range(k, m):
                R[i][j] -= s * v[i - k]
        vs.append(v)
        betas.append(beta)
    return vs, betas, [R[i][:] for i in range(n)]


def _apply_qt(vs, betas, b):
    """Q^T b for the Householder factorisation (b is a list of length m)."""
    b = b[:]
    m = len(b)
    for k, (v, beta) in enumerate(zip(vs, betas)):
        s = sum(v[i - k] * b[i] for i in range(k, m)) * beta
        for i in range(k, m):
            b[i] -= s * v[i - k]
    return b


def _jacobi_svd(R, tol_exp: int = DIGITS - 5, max_sweeps: int = 60):
    """One-sided Jacobi SVD of a square matrix R = U S V^T (Hestenes' method)."""
    n = len(R)
    # work on columns of R
    cols = [[R[i][j] for i in range(n)] for j in range(n)]
    Vc = [[D(1) if i == j else D(0) for i in range(n)] for j in range(n)]
    tol = D(10) ** (-tol_exp)
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                a = sum(t * t for t in cols[p])
                b = sum(t * t for t in cols[q])
                g = sum(s * t for s, t in zip(cols[p], cols[q]))
                if g == 0 or abs(g) <= tol * (a * b).sqrt():
                    continue
                rotated = True
                zeta = (b - a) / (2 * g)
                sgn = D(1) if zeta >= 0 else D(-1)
                t = sgn / (abs(zeta) + (1 + zeta * zeta).sqrt())
                c = 1 / (1 + t * t).sqrt()
                s = c * t
                cp, cq = cols[p], cols[q]
                cols[p] = [c * x - s * y for x, y in zip(cp, cq)]
                cols[q] = [s * x + c * y for x, y in zip(cp, cq)]
                vp, vq = Vc[p], Vc[q]
                Vc[p] = [c * x - s * y for x, y in zip(vp, vq)]
                Vc[q] = [s * x + c * y for x, y in zip(vp, vq)]
        if not rotated:
            break
    S = [sum(t * t for t in col).sqrt() for col in cols]
    U = [[cols[j][i] / S[j] for j in range(n)] for i in range(n)]
    V = [[Vc[j][i] for j in range(n)] for i in range(n)]
    return U, S, V


# --------------------------------------------------------------------------- #
# The FC matrices
# --------------------------------------------------------------------------- #
def compute_fc_matrices(d=5, C=27, Z=12, n_os=20, n_r=6, m_F=20):
    """Q (d x d), A (C x d), A_r (C n_r x d) in 50-digit arithmetic, rounded to double.

    Also returns diagnostics: singular values of B_os, LS residual per column.
    """
    with decimal.localcontext(_ctx()):
        pi = decimal_pi()
        Per = d + 2 * C + Z - 1
        Q, R = gram_qr(d)
        # Q_os = P_os R^{-1} on x = i/n_os (eq. (2.3)); back-substitution row by row
        n_fine = n_os * (d - 1) + 1
        Qos = []
        for i in range(n_fine):
            x = D(i) / n_os
            prow = [x ** j if j > 0 else D(1) for j in range(d)]
            # solve q R = prow for the row vector q (R upper triangular)
            qrow = [D(0)] * d
            for j in range(d):
                s = prow[j] - sum(qrow[k] * R[k][j] for k in range(j))
                qrow[j] = s / R[j][j]
            Qos.append(qrow)
        # fit points in units of 1/n_os: matching 0..n_os(d-1), zeros n_os(d+C)..n_os(d+C+Z-1)
        fit_num = list(range(0, n_os * (d - 1) + 1)) + \
            list(range(n_os * (d + C), n_os * (d + C + Z - 1) + 1))
        den = n_os * Per  # x/Per = num/den

        def basis_row(num, dn):
            row = [D(1)]
            for m in range(1, m_F + 1):
                c, s = cos_sin_turn(m * num, dn, pi)
                row += [c, s]
            return row

        Bos = [basis_row(num, den) for num in fit_num]
        m = len(Bos)
        nb = len(Bos[0])
        vs, betas, Rb = _householder_qr(Bos)
        U, S, V = _jacobi_svd(Rb)
        coefs = []
        resid = []
        for j in range(d):
            b = [Qos[i][j] for i in range(n_fine)] + [D(0)] * (m - n_fine)
            qtb = _apply_qt(vs, betas, b)[:nb]
            # a = V S^{-1} U^T (Q_B^T b)
            utb = [sum(U[i][k] * qtb[i] for i in range(nb)) for k in range(nb)]
            y = [utb[k] / S[k] for k in range(nb)]
            a = [sum(V[i][k] * y[k] for k in range(nb)) for i in range(nb)]
            coefs.append(a)
            r = max(abs(sum(Bos[i][l] * a[l] for l in range(nb)) - b[i]) for i in range(m))
            resid.append(float(r))

        def g_at(num, dn, j):
            row = basis_row(num, dn)
            return sum(row[l] * coefs[j][l] for l in range(nb))

        A = np.zeros((C, d))
        for q in range(C):
            for j in range(d):
                A[q, j] = float(g_at(d + q, Per, j))
        Cr = C * n_r
        Ar = np.zeros((Cr, d))
        for q in range(1, Cr + 1):
            num = (d - 1) * n_r + q  # x = num / n_r
            for j in range(d):
                Ar[q - 1, j] = float(g_at(num, n_r * Per, j))
        Qd = np.array([[float(Q[i][j]) for j in range(d)] for i in range(d)])
        Rd = np.array([[float(R[i][j]) for j in range(d)] for i in range(d)])
        sv = sorted((float(s) for s in S), reverse=True)
        return {"Q": Qd, "R": Rd, "A": A, "Ar": Ar, "sv": np.array(sv),
                "resid": np.array(resid),
                "params": dict(d=d, C=C, Z=Z, n_os=n_os, n_r=n_r, m_F=m_F)}


def golden_path(d=5, C=27, Z=12, n_os=20, n_r=6, m_F=20) -> str:
    return os.path.join(_GOLDEN, f"fc_matrices_d{d}_C{C}_Z{Z}_os{n_os}_r{n_r}_m{m_F}.txt")


def save_fc_matrices(mats, path):
    """Text format: one 'name rows cols' header line, then hex doubles row by row."""
    with open(path, "w") as fh:
        p = mats["params"]
        fh.write("# oracle FC matrices (50-digit decimal, rounded once to double)\n")
        fh.write("# written by oracle/make_fc_matrices.py\n")
        fh.write("# params " + " ".join(f"{k}={v}" for k, v in p.items()) + "\n")
        for name in ("Q", "R", "A", "Ar", "sv", "resid"):
            arr = np.atleast_2d(mats[name])
            fh.write(f"{name} {arr.shape[0]} {arr.shape[1]}\n")
            for row in arr:
                fh.write(" ".join(float(v).hex() for v in row) + "\n")


def read_fc_matrices(path):
    out = {}
    with open(path) as fh:
        lines = [ln for ln in fh.read().splitlines() if ln and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        name, r, c = lines[i].split()
        r, c = int(r), int(c)
        arr = np.array([[float.fromhex(t) for t in lines[i + 1 + k].split()] for k in range(r)])
        out[name] = arr[0] if name in ("sv", "resid") else arr
        i += 1 + r
    return out


def load_fc_matrices(d=5, C=27, Z=12, n_os=20, n_r=6, m_F=20):
    """Cached FC matrices (computed and cached on first use if absent)."""
    path = golden_path(d, C, Z, n_os, n_r, m_F)
    if os.path.exists(path):
        m = read_fc_matrices(path)
    else:
        m = compute_fc_matrices(d, C, Z, n_os, n_r, m_F)
        try:
            save_fc_matrices(m, path)
        except OSError:
            pass
    m["params"] = dict(d=d, C=C, Z=Z, n_os=n_os, n_r=n_r, m_F=m_F)
    return m
