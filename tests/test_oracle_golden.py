"""Regression pin: the oracle still reproduces the fixture written by
tests/golden/make_golden.py (which calls only the oracle)."""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

import make_golden  # noqa: E402


def test_tiny_sweep_fixture():
    ref = np.loadtxt(os.path.join(HERE, "golden", "sweep2d_tiny.txt"))
    I, mom = make_golden.tiny_case()
    got = np.r_[I.ravel(), mom.ravel()]
    assert got.shape == ref.shape
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-300)
