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
