"""The serving loop on the GPU: each stream's tracked boxes are the same
whether it is served alone or in a mix of streams (continuous batching
changes only which frames share a step, never a stream's result), and
admission keeps the device memory in use under the budget."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06017_b300 import omt, serve, synth
    sizes = ((320, 240), (480, 272), (640, 360))
    specs, frames, det = serve.build_workload(6, 1.0, workload=15, sizes=sizes, boxes=(4, 24),
                                              max_corners=20)
    params = omt.default_params(levels=3, win=15, max_corners=20, storage=omt.F16)
    return omt, serve, specs, frames, det, params


def _trajectories(stats):
    out = {}
    for f in stats.frames:
        if f.boxes is not None:
            out[(f.sid, f.index)] = f.boxes
    return out


def test_alone_equals_in_the_mix(setup):
    omt, serve, specs, frames, det, params = setup
    stats, _ = serve.serve(specs, frames, det, params, 1 << 34, keep_boxes=True)
    s = stats.summary()
    assert s["frames_done"] == sum(len(sp.arrivals) for sp in specs)
    mix = _trajectories(stats)
    assert len(mix) > 20
    for sp in specs[:3]:
        st1, _ = serve.serve([sp], frames, det, params, 1 << 34, keep_boxes=True)
        alone = _trajectories(st1)
        assert set(alone) == {k for k in mix if k[0] == sp.sid}
        for k, v in alone.items():
            np.testing.assert_array_equal(v, mix[k])


def test_budget_admission_on_device(setup):
    omt, serve, specs, frames, det, params = setup
    from paper_1910_06017_b300.serve import GpuBackend
    be = GpuBackend(params, len(specs), 1000, 640, 360, 20, frames, det)
    need = sorted(be.bytes_for(sp) for sp in specs)
    budget = need[-1] + need[-2]          # about two streams at a time
    stats, _ = serve.serve(specs, frames, det, params, budget)
    s = stats.summary()
    assert s["frames_done"] == sum(len(sp.arrivals) for sp in specs)
    assert s["max_bytes_in_use"] <= budget
    assert s["latency_ms_p99"] > 0
