"""Shared fixtures: repo root on sys.path, the `gpu` marker, statistics helpers."""

import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def binned(x, n_bins=20, cut=0.2):
    """Mean and standard error of a Monte Carlo time series: drop the first `cut` fraction,
    split the rest into n_bins equal bins, and use the spread of the bin means."""
    x = np.asarray(x, dtype=np.float64)
    x = x[int(len(x) * cut):]
    m = (len(x) // n_bins) * n_bins
    b = x[len(x) - m:].reshape(n_bins, -1).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(n_bins))


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle
