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


def noalloc_device_layout(torch, s, spins_by_replica):
    """A sample in the library's device format, for the allocation-free entry point:
    colour-major renumbering (greedy colouring, caller ids ascending inside a class), links as
    (neighbour, J float32 bits), spins as [site][replica][4] float32, on the current device."""
    import paper_1803_07030_gb300 as vg

    n = s.n_sites
    colour, nc = vg.vegas_greedy_colour(s.row_ptr, s.col)
    order = np.lexsort((np.arange(n), colour))  # new index -> caller id
    inv = np.empty(n, dtype=np.int64)
    inv[order] = np.arange(n)
    cstart = np.concatenate([[0], np.cumsum(np.bincount(colour, minlength=nc))]).astype(np.int32)
    deg = np.diff(s.row_ptr)[order]
    row_ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int64)
    first = np.repeat(s.row_ptr[order] - row_ptr[:-1], deg) + np.arange(row_ptr[-1])
    links = np.empty((row_ptr[-1], 2), dtype=np.int32)
    links[:, 0] = inv[s.col[first]]
    links[:, 1] = s.J[first].astype(np.float32).view(np.int32)
    R = len(spins_by_replica)
    spins = np.zeros((n, R, 4), dtype=np.float32)
    for r, S in enumerate(spins_by_replica):
        spins[:, r, :3] = S[order]
    dev = "cuda"
    return {
        "spins": torch.from_numpy(spins).to(dev),
        "links": torch.from_numpy(links).to(dev),
        "row_ptr": torch.from_numpy(row_ptr).to(dev),
        "site_id": torch.from_numpy(order.astype(np.int32)).to(dev),
        "colour_start": cstart,
        "order": order,
        "links_host": links,
    }
