"""The allocation-free sweep (vegas_sweep_noalloc) against the context API.

vegas_sweep_noalloc serves callers that cannot let the library call cudaMalloc (programs
that own all device memory in their own pool, or cannot afford an allocation's implicit
synchronisation); it takes device buffers from the caller and keeps its scratch in a
static device array. This test lays a sample out in the library's device format with
torch, runs two MCS through the C-ABI entry point, and checks energy and magnetization
of both against vegas_run on a context with the same seed, instances and temperatures.
This file is collected last on purpose.
"""

import numpy as np
import pytest

from conftest import noalloc_device_layout

import paper_1803_07030_gb300 as vg
from paper_1803_07030_gb300 import vegas as vb
from lattices import sc_periodic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    vg.build()
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


def test_no_alloc_sweep_matches_context_two_calls(torch):
    s = sc_periodic(12, bimodal_seed=3)
    R, seed, inst0 = 4, 5, 8
    T = np.array([0.3, 0.8, 1.5, 2.5])
    B = np.array([0.0, 0.2, -0.1, 0.4])
    with vg.Context([s], precision=32, replicas=R, seed=seed, inst_base=inst0, stream=None) as c:
        start = [c.spins(r) for r in range(R)]
        c.run(T[:, None], B[:, None], 2)  # one step of two MCS: records 0 and 1
        H = c.history()
        final = [c.spins(r) for r in range(R)]
    lay = noalloc_device_layout(torch, s, start)
    out = torch.zeros((R, 4), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    got = []
    for t in (0, 1):  # two calls in a row share (and rewrite) the static scratch
        vg.vegas_sweep_noalloc(lay["spins"].data_ptr(), lay["links"].data_ptr(), lay["row_ptr"].data_ptr(),
                               lay["site_id"].data_ptr(), s.n_sites, lay["colour_start"], R, 1.0 / T, B,
                               seed=seed, inst0=inst0, t=t, out_ptr=out.data_ptr(), stream=stream)
        got.append(out.cpu().numpy().copy())
    N = s.n_sites
    for t in (0, 1):
        # same tolerance as the other FP32 history comparisons: sums grouped differently
        assert np.all(np.abs(got[t] - H[:, t, :]) <= 1e-6 * N), (t, got[t], H[:, t, :])
    spins = lay["spins"].cpu().numpy()
    for r in range(R):
        mine = np.empty((N, 3))
        mine[lay["order"]] = spins[:, r, :3]
        # the context renormalises at the end of its step; the allocation-free call does not
        assert np.max(np.abs(mine - final[r])) < 1e-6


def test_no_alloc_rejects_sizes_beyond_its_scratch(torch):
    s = sc_periodic(4)
    lay = noalloc_device_layout(torch, s, [np.tile([0, 0, 1.0], (s.n_sites, 1))])
    out = torch.zeros((64, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(vb.VegasError) as e:
        vg.vegas_sweep_noalloc(lay["spins"].data_ptr(), lay["links"].data_ptr(), lay["row_ptr"].data_ptr(),
                               lay["site_id"].data_ptr(), s.n_sites, lay["colour_start"], 64, np.ones(64),
                               np.zeros(64), out_ptr=out.data_ptr())
    assert e.value.status == vb.EINVAL and "32" in str(e.value)
