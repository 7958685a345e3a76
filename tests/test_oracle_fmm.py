"""Pins for the oracle's FMM (Sec. 5.3: P2M, M2M, M2L, L2L, L2P; Sec. 5.1 flow).

Independent checks: exact identities (M2M and L2L are exact under truncation), direct
summation of the free-space potential at far points, geometric decay of the error in p,
and the FMM preconditioner against the direct one.
"""
import numpy as np
import pytest

import oracle as O
import synth_inputs as S
from conftest import rel_l2


def _cluster(rng, c, r, k=40):
    ang = rng.uniform(0, 2 * np.pi, k)
    rad = r * np.sqrt(rng.uniform(0, 1, k))
    return c.real + rad * np.cos(ang), c.imag + rad * np.sin(ang), rng.standard_normal(k)


def test_m2m_is_exact():
    rng = np.random.default_rng(0)
    p = 12
    zM = 0.3 + 0.2j
    Mp = np.zeros(p, complex)
    xs, ys, fs = [], [], []
    for ch in (0.05 + 0.05j, -0.05 + 0.05j, 0.05 - 0.05j, -0.05 - 0.05j):
        x, y, f = _cluster(rng, zM + ch, 0.04)
        Mp += O.m2m(O.p2m(p, x, y, f, zM + ch), zM - (zM + ch))
        xs.append(x); ys.append(y); fs.append(f)
    direct = O.p2m(p, np.concatenate(xs), np.concatenate(ys), np.concatenate(fs), zM)
    assert np.max(np.abs(Mp - direct)) <= 1e-14 * np.max(np.abs(direct))


def test_l2l_is_exact_recentring():
    rng = np.random.default_rng(1)
    p = 10
    Lp = rng.standard_normal(p) + 1j * rng.standard_normal(p)
    zL, zl = 0.1 + 0.1j, 0.13 + 0.07j
    Lc = O.l2l(Lp, zl - zL)
    for _ in range(5):
        zi = zl + 0.02 * (rng.standard_normal() + 1j * rng.standard_normal())
        assert abs(O.l2p(Lc, zi - zl) - O.l2p(Lp, zi - zL)) < 1e-13


def _direct_log(x, y, f, z):
    return float(np.sum(f * np.log(np.abs(z - (x + 1j * y)))))


def test_p2m_converges_geometrically():
    rng = np.random.default_rng(2)
    x, y, f = _cluster(rng, 0j, 0.1)
    z = 0.5 + 0.2j  # |z| / r ~ 5.4
    errs = [abs(O.m2p(O.p2m(p, x, y, f, 0j), z) - _direct_log(x, y, f, z)) for p in (2, 4, 6, 8, 10)]
    for a, b in zip(errs, errs[1:]):
        assert b < a * 0.15
    assert errs[-1] < 1e-7 * np.sum(np.abs(f))


def test_m2l_converges_geometrically():
    rng = np.random.default_rng(3)
    x, y, f = _cluster(rng, 0j, 0.1)
    zL = 0.6 + 0.1j
    pts = zL + 0.1 * (rng.standard_normal(8) + 1j * rng.standard_normal(8)) / 3
    errs = []
    for p in (4, 8, 12, 16):
        Lc = O.m2l(O.p2m(p, x, y, f, 0j), zL - 0j)
        errs.append(max(abs(O.l2p(Lc, z - zL) - _direct_log(x, y, f, z)) for z in pts))
    for a, b in zip(errs, errs[1:]):
        assert b < a * 0.1
    assert errs[-1] < 1e-10


def test_fmm_volume_error_decays_in_p():
    n = 64
    r = S.gaussian_mixture(n, 0)
    ref = O.direct_V(n, 0, 0, 1, r)
    errs = []
    for p in (2, 4, 6, 8, 10):
        out = O.Problem(n, p=p).apply(r, "fmm", stages=True)
        errs.append(rel_l2(out["vr"], ref))
    for a, b in zip(errs, errs[1:]):
        assert b < a * 0.3
    # Sec. 7.1: p = 6, theta = 0.4 gives about six significant digits
    assert errs[2] < 1e-6
    assert errs[4] < 1e-8


def test_fmm_near_plus_far_is_vr():
    n = 32
    out = O.Problem(n, p=8).apply(S.random_field(n, 1), "fmm", stages=True)
    assert rel_l2(out["near"] + out["far"], out["vr"]) < 1e-14


@pytest.mark.parametrize("n", [32, 64])
def test_fmm_preconditioner_matches_direct(n):
    r = S.random_field(n, 11)
    P = O.Problem(n, p=10)
    d = P.apply(r, "direct", stages=True)
    f = P.apply(r, "fmm", stages=True)
    for k in ("vr", "vr_col", "q", "z"):
        assert rel_l2(f[k], d[k]) < 1e-7, k
