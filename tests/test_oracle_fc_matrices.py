"""Pins for the oracle's 1D blending-to-zero matrices (Section 2.2, Remark 2.2)."""
import numpy as np
import pytest

from oracle.fc_matrices import compute_fc_matrices, load_fc_matrices
from oracle.fc1d import fc1d_eval


@pytest.fixture(scope="module")
def mats():
    return load_fc_matrices()


def test_gram_qr_is_a_qr_of_the_vandermonde(mats):
    """Eq. (2.2): P = QR with Q orthonormal and R upper triangular, positive diagonal."""
    Q, R = mats["Q"], mats["R"]
    d = Q.shape[0]
    x = np.arange(d, dtype=float)
    P = x[:, None] ** np.arange(d)[None, :]
    assert np.allclose(Q.T @ Q, np.eye(d), atol=1e-14)
    assert np.allclose(np.tril(R, -1), 0)
    assert np.all(np.diag(R) > 0)
    assert np.allclose(Q @ R, P, rtol=0, atol=1e-12 * np.abs(P).max())


def test_gram_columns_are_polynomials_of_increasing_degree(mats):
    """Column j of Q is the j-th Gram polynomial: degree exactly j on the nodes."""
    Q = mats["Q"]
    d = Q.shape[0]
    x = np.arange(d, dtype=float)
    for j in range(d):
        c = np.polyfit(x, Q[:, j], d - 1)[::-1]  # exact interpolation, ascending
        assert np.all(np.abs(c[j + 1:]) < 1e-10)
        assert abs(c[j]) > 1e-6


def test_least_squares_fit_is_tight(mats):
    """Eq. (2.5) with m_F = 20 modes matches the oversampled Gram values and the zero
    interval to <= 1.2e-12 (full-rank minimiser, sigma_min/sigma_max ~ 2e-16)."""
    assert mats["resid"].max() < 1.2e-12
    sv = mats["sv"]
    assert sv[-1] / sv[0] > 1e-17


def test_refined_matrix_agrees_with_unrefined_on_common_points(mats):
    """A (points d..d+C-1) and A_r (points (d-1)+q/n_r) evaluate the same g^c_j: every
    n_r-th row of A_r, starting at q = n_r, equals a row of A."""
    A, Ar = mats["A"], mats["Ar"]
    n_r = mats["params"]["n_r"]
    C = A.shape[0]
    for q in range(C):
        assert np.allclose(Ar[(q + 1) * n_r - 1], A[q], rtol=1e-15, atol=1e-13)


def test_continuation_decays_toward_the_zero_interval(mats):
    """g^c_j nearly vanishes one step before the zero-matching interval."""
    Ar = mats["Ar"]
    assert np.abs(Ar[-1]).max() < 3e-7


def test_fc1d_converges_at_order_d(mats):
    """Section 2.3: 1D-FC of Figure 1's phi converges as O(k^d), d = 5."""
    phi = lambda x: np.exp(np.sin(5.4 * np.pi * x - 2.7 * np.pi) - np.cos(2 * np.pi * x)) \
        - np.sin(2.5 * np.pi * x) + 1
    xe = np.linspace(0, 1, 1501)
    errs = []
    for N in (101, 201, 401):
        x = np.linspace(0, 1, N)
        errs.append(np.abs(fc1d_eval(mats, phi(x), xe) - phi(xe)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > 4.5), (errs, orders)
    assert errs[-1] < 1e-7


@pytest.mark.parametrize("d,order", [(10, 8.0), (12, 9.5)])
def test_fc1d_converges_at_high_order(d, order):
    """Section 2.3 at the paper's higher orders (d = 10, 12; same C, Z, n_os, n_r and
    m_F = 20): the 1D-FC of Figure 1's phi converges faster than O(k^order) from
    N = 51 to 201 and reaches 1e-9.  The least-squares misfit of the highest Gram
    columns is 5e-7 (d = 10) and 2e-5 (d = 12), but smooth data carry almost nothing
    in those columns."""
    m = load_fc_matrices(d)
    phi = lambda x: np.exp(np.sin(5.4 * np.pi * x - 2.7 * np.pi) - np.cos(2 * np.pi * x)) \
        - np.sin(2.5 * np.pi * x) + 1
    errs = []
    for N in (51, 101, 201):
        x = np.linspace(0, 1, N)
        xe = np.linspace(0, 1, 4 * N + 1)
        errs.append(np.abs(fc1d_eval(m, phi(x), xe) - phi(xe)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > order), (errs, orders)
    assert errs[-1] < 1e-9


@pytest.mark.parametrize("d", [10, 12])
def test_high_order_gram_qr(d):
    """Eq. (2.2) at d = 10, 12: Q orthonormal, R upper triangular with a positive
    diagonal, QR = P, and Q R^{-1} reproduces the oversampled Vandermonde rows."""
    m = load_fc_matrices(d)
    Q, R = m["Q"], m["R"]
    x = np.arange(d, dtype=float)
    P = x[:, None] ** np.arange(d)[None, :]
    assert np.allclose(Q.T @ Q, np.eye(d), atol=1e-13)
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R) > 0)
    assert np.abs(Q @ R - P).max() <= 1e-12 * np.abs(P).max()


@pytest.mark.slow
def test_golden_matrices_regenerate_bit_for_bit():
    """The cached matrices are what the 50-digit computation gives."""
    fresh = compute_fc_matrices()
    cached = load_fc_matrices()
    for k in ("Q", "A", "Ar"):
        assert np.array_equal(fresh[k], cached[k]), k


@pytest.mark.parametrize("d", [5, 10])
def test_matrices_agree_with_an_independent_multiprecision_qr(d):
    """Re-derive A_r by mpmath's QR least squares at 40 digits (a different
    algorithm and library): every entry agrees after rounding to double."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    mats = load_fc_matrices(d)
    C, Z, n_os, n_r, m_F = 27, 12, 20, 6, 20
    Per = d + 2 * C + Z - 1
    x = [mp.mpf(i) for i in range(d)]
    P = mp.matrix([[x[i] ** j if j else mp.mpf(1) for j in range(d)] for i in range(d)])
    Qm, Rm = mp.qr(P)
    sgn = [1 if Rm[j, j] > 0 else -1 for j in range(d)]
    Rm = mp.matrix([[Rm[i, j] * sgn[i] for j in range(d)] for i in range(d)])
    xos = [mp.mpf(i) / n_os for i in range(n_os * (d - 1) + 1)]
    Pos = mp.matrix([[t ** j if j else mp.mpf(1) for j in range(d)] for t in xos])
    Qos = Pos * mp.inverse(Rm)
    pts = xos + [mp.mpf(d + C) + mp.mpf(i) / n_os for i in range(n_os * (Z - 1) + 1)]

    def row(t):
        r = [mp.mpf(1)]
        for m in range(1, m_F + 1):
            a = 2 * mp.pi * m * t / Per
            r += [mp.cos(a), mp.sin(a)]
        return r

    Bm = mp.matrix([row(t) for t in pts])
    Ar = np.zeros((C * n_r, d))
    for j in range(d):
        b = mp.matrix([Qos[i, j] if i < len(xos) else 0 for i in range(len(pts))])
        a = mp.qr_solve(Bm, b)[0]
        for q in range(1, C * n_r + 1):
            t = mp.mpf(d - 1) + mp.mpf(q) / n_r
            Ar[q - 1, j] = float(sum(a[l] * v for l, v in enumerate(row(t))))
    assert np.abs(Ar - mats["Ar"]).max() <= 1e-13 * np.abs(Ar).max()
