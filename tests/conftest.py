"""Shared pytest set-up: the ``gpu`` marker and small helpers.

Tests marked ``gpu`` need a CUDA device and the compiled library; everything else
runs on the CPU (oracle pins, host logic, ABI export checks, gloo multi-process).
"""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled fmmpc library")
    config.addinivalue_line("markers", "slow: long CPU test")


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def grid_xy(n, x0=0.0, y0=0.0, side=1.0):
    h = side / (n + 1)
    x = x0 + (np.arange(n) + 1) * h
    y = y0 + (np.arange(n) + 1) * h
    X, Y = np.meshgrid(x, y)  # natural order: row j (y), column i (x)
    return X.ravel(), Y.ravel(), h


def max_rel(a, b):
    """Largest element-wise difference over the largest reference magnitude,
    max|a - b| / max|b|: bounds the worst node, where a relative L2 norm could hide a
    localised error (the boundary band is 0.4% of the nodes at 1024^2)."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def check_close(name, a, b, l2, mx):
    """Relative L2 error below l2 and element-wise error (max_rel) below mx; prints both
    measured figures so a run with -s records them next to their gates."""
    e2, em = rel_l2(a, b), max_rel(a, b)
    print(f"PARITY {name}: rel_l2 {e2:.3e} (gate {l2:.1e}) max_rel {em:.3e} (gate {mx:.1e})", flush=True)
    assert e2 < l2, f"{name}: relative L2 error {e2:.3e} >= {l2:.1e}"
    assert em < mx, f"{name}: element-wise error {em:.3e} >= {mx:.1e}"
    return e2, em
