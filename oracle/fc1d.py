"""Oracle: the 1D-FC continuation of Section 2.3, eqs. (2.7)-(2.8).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

phi_r^r = A Q^T phi_r and phi_l^l = R^C A Q^T R^d phi_l (R^e reverses order); the
N given values followed by phi_l^l + phi_r^r form phi^c, whose DFT is the
continuation (eq. (2.8)), with period b = (N + C) k.
"""
from __future__ import annotations

import numpy as np


def fc1d_values(mats, phi):
    """phi^c of eq. (2.7) for the samples phi_0..phi_{N-1}."""
    Q, A = mats["Q"], mats["A"]
    d = Q.shape[0]
    right = A @ (Q.T @ phi[-d:])
    left = (A @ (Q.T @ phi[:d][::-1]))[::-1]
    return np.concatenate([phi, left + right])


def fc1d_eval(mats, phi, x_eval):
    """Evaluate the continuation (eq. (2.8)) at points of [0, 1]; phi sampled at
    x_j = j/(N-1)."""
    N = len(phi)
    k = 1.0 / (N - 1)
    v = fc1d_values(mats, phi)
    L = len(v)
    c = np.fft.fft(v) / L
    freq = np.fft.fftfreq(L, 1.0 / L)
    b = L * k
    return np.real(np.exp(2j * np.pi * np.outer(x_eval, freq) / b) @ c)
