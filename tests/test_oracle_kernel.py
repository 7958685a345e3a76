"""Pins for the oracle's volume operator V (Sec. 4.2 Eq. eq:green, Sec. 5.1
Eq. e:volume_integral) and its self term.

Independent checks: 2-D quadrature of ln r over the cell, a numpy brute-force dense
matrix, an FFT lattice convolution, and the symmetry G_ij = G_ji.
"""
import numpy as np
from scipy import integrate

import oracle as O
import synth_inputs as S
from conftest import rel_l2


def test_self_constant_is_cell_mean_of_log():
    # mean of ln|x| over [-1/2,1/2]^2 = 4 * int_0^{1/2} int_0^{1/2} ln sqrt(x^2+y^2)
    val, err = integrate.dblquad(lambda y, x: 0.5 * np.log(x * x + y * y), 0, 0.5, 0, 0.5,
                                 epsabs=1e-13, epsrel=1e-13)
    assert abs(4 * val - O.self_constant()) < 1e-9


def _dense_G(n, h):
    X, Y, _ = S.grid_coords(n)
    D2 = (X[:, None] - X[None, :]) ** 2 + (Y[:, None] - Y[None, :]) ** 2
    np.fill_diagonal(D2, 1.0)
    G = -0.5 * np.log(D2) / (2 * np.pi)
    np.fill_diagonal(G, -(np.log(h) + O.self_constant()) / (2 * np.pi))
    return G


def test_direct_V_bruteforce():
    n = 10
    h = 1 / 11
    r = S.random_field(n, 5)
    assert rel_l2(O.direct_V(n, 0, 0, 1, r), _dense_G(n, h) @ (h * h * r)) < 1e-13


def test_direct_V_equals_fft_lattice_convolution():
    n = 40
    h = 1.0 / (n + 1)
    r = S.random_field(n, 7)
    di = np.arange(-(n - 1), n)
    DX, DY = np.meshgrid(di, di)
    with np.errstate(divide="ignore"):
        K = -(np.log(h) + 0.5 * np.log(DX ** 2 + DY ** 2)) / (2 * np.pi)
    K[n - 1, n - 1] = -(np.log(h) + O.self_constant()) / (2 * np.pi)
    M = 2 * n
    Kp = np.zeros((M, M))
    Kp[: 2 * n - 1, : 2 * n - 1] = K
    Rp = np.zeros((M, M))
    Rp[:n, :n] = (h * h * r).reshape(n, n)
    full = np.real(np.fft.ifft2(np.fft.fft2(Kp) * np.fft.fft2(Rp)))
    conv = full[n - 1: 2 * n - 1, n - 1: 2 * n - 1]
    assert rel_l2(O.direct_V(n, 0, 0, 1, r), conv.ravel()) < 1e-12


def test_direct_V_is_symmetric():
    n = 20
    a, b = S.random_field(n, 1), S.random_field(n, 2)
    lhs = a @ O.direct_V(n, 0, 0, 1, b)
    rhs = b @ O.direct_V(n, 0, 0, 1, a)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_direct_V_nodes_matches_full():
    n = 16
    r = S.random_field(n, 9)
    idx = np.array([0, 5, 100, 255], np.int32)
    assert rel_l2(O.direct_V_nodes(n, 0, 0, 1, r, idx), O.direct_V(n, 0, 0, 1, r)[idx]) < 1e-15
