"""Detection beside tracking (Section V-B runs the motion field and the
detector concurrently): with a stub detector -- bf16 GEMMs through torch
(cuBLAS) on a CUDA stream of its own, issued every step so that its kernels
share the GPU with the tracking step's -- the batched step's points,
statuses, iteration counts and boxes are the same bit for bit as without it.
Nothing a step computes depends on which SMs its work lands on or in what
order (each point is one warp's fixed computation, each box one CTA's)."""
import math

import numpy as np
import pytest

from paper_1910_06017_b300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def omt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_06017_b300 import omt as m
    m.lib()
    return m


def _run(omt, sps, params, detector, steps=4, graph=True):
    caps = [int(math.ceil(sp.n_target / 64)) for sp in sps]
    B = omt.BatchTracker([sp.size for sp in sps], params, max_boxes=[len(sp.boxes) for sp in sps],
                         max_corners=caps)
    for s, sp in enumerate(sps):
        B.prime(s, torch.from_numpy(sp.frame0).cuda())
        B.frame[s][0].copy_(torch.from_numpy(sp.frame1))
        B.frame[s][1].copy_(torch.from_numpy(sp.frame0))
        B.set_boxes(s, torch.from_numpy(sp.boxes))
    B.pack()
    B.step()
    if graph:
        B.capture()
    torch.cuda.synchronize()
    out = []
    for _ in range(steps):
        if detector is not None:
            detector()
        B.step()
        torch.cuda.synchronize()
        rec = []
        for s, sp in enumerate(sps):
            n = B.count(s)
            rec.append((B.pts_out[s][:n].cpu().numpy(), B.status[s][:n].cpu().numpy(),
                        B.iters[s][:n].cpu().numpy(), B.boxes_out[s][:len(sp.boxes)].cpu().numpy()))
        out.append(rec)
    return out


@pytest.mark.parametrize("graph", [True, False])
def test_tracking_unchanged_beside_a_detector_stream(omt, graph):
    sps = [synth.stream_pair(s, workload=13, n_range=(2000, 6000)) for s in range(6)]
    caps = [int(math.ceil(sp.n_target / 64)) for sp in sps]
    params = omt.default_params(levels=4, win=21, min_dist=3.0, storage=1, max_corners=max(caps))
    alone = _run(omt, sps, params, None, graph=graph)

    det = torch.cuda.Stream()
    a = torch.randn(4096, 1024, dtype=torch.bfloat16, device="cuda")
    w = torch.randn(1024, 1024, dtype=torch.bfloat16, device="cuda")
    o = torch.empty(4096, 1024, dtype=torch.bfloat16, device="cuda")
    main = torch.cuda.current_stream()

    def detector():
        # issued just before the step, on its own stream: the GEMMs run while
        # the step's kernels run
        det.wait_stream(main)
        with torch.cuda.stream(det):
            for _ in range(24):
                torch.matmul(a, w, out=o)

    beside = _run(omt, sps, params, detector, graph=graph)
    torch.cuda.synchronize()
    for k, (x, y) in enumerate(zip(alone, beside)):
        for s, (p, q) in enumerate(zip(x, y)):
            for name, u, v in zip(("pts_out", "status", "iters", "boxes"), p, q):
                np.testing.assert_array_equal(u, v, err_msg=f"step {k} stream {s} {name}")
    assert sum(len(r[0]) for r in alone[0]) > 10000
