"""Test helpers: error of a 2D-FC extension on the h/2 grid inside the domain
(Section 3.6: errors are measured on a grid of step h/2 within the domain)."""
import math

import numpy as np

import workloads as W
from oracle import fc2d as F
from oracle import geometry as G


def upsample2(ext):
    """Trigonometric interpolant of the grid values on the grid of step h/2."""
    ny, nx = ext.shape
    c = np.fft.fft2(ext)
    big = np.zeros((2 * ny, 2 * nx), complex)
    ky = np.fft.fftfreq(ny, 1.0 / ny).astype(int)
    kx = np.fft.fftfreq(nx, 1.0 / nx).astype(int)
    big[np.ix_(ky % (2 * ny), kx % (2 * nx))] = c
    return np.real(np.fft.ifft2(big)) * 4


def inside_fine(curve, xf, yf):
    out = np.zeros((len(yf), len(xf)), bool)
    for r, y in enumerate(yf):
        X = G.crossings(curve, "row", y, 20000)
        for m in range(0, len(X) - 1, 2):
            out[r] |= (xf >= X[m]) & (xf <= X[m + 1])
    return out


def paper_setup(boundary, h, d=5, M=None, B=None, smooth=False):
    """Grid and parameters of the paper's experiments: k1 = k2 = h (Remark 3.3).
    smooth: grid sizes raised to even 2^a 3^b 5^c (what the library's DFT takes)."""
    cv = G.make_curve(boundary)
    th = np.linspace(0, 2 * np.pi, 20001)
    xx, yy = cv.point(th)
    fit = W.fit_grid_smooth if smooth else W.fit_grid
    grid = fit(xx.min(), xx.max(), yy.min(), yy.max(), h)
    B = B or int(round(2 * math.pi / h))
    return W.Workload("paper", boundary, grid, W.Params(d=d, M=M or d + 3, B=B, k1=h))


def fine_error(w, mats, f, relative=True):
    geo = G.build_geometry(w)
    fg = W.grid_values(w, f)
    fb = F.boundary_values(geo, f)
    ext = F.extension(geo, mats, fg, fb)
    fine = upsample2(ext)
    g = w.grid
    xf = g.a0 + (g.h / 2) * np.arange(2 * g.nx)
    yf = g.b0 + (g.h / 2) * np.arange(2 * g.ny)
    X, Y = np.meshgrid(xf, yf)
    ins = inside_fine(geo.curve, xf, yf)
    err = np.abs(fine - f(X, Y))[ins].max()
    if relative:
        err /= np.abs(f(X, Y)[ins]).max()
    return err

