"""Matching and update phases on the GPU (Section V-A): the device IoU
matrix equals the FP64 oracle's bit for bit (same operations, no fused
multiply-add), and matching + update from the device matrix equal the
oracle's on tracked boxes against detections."""
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


def _boxes(rng, n, w=1920, h=1080):
    x0 = rng.uniform(-50, w, n)
    y0 = rng.uniform(-50, h, n)
    bw = rng.uniform(0, 300, n)
    bh = rng.uniform(0, 300, n)
    b = np.stack([x0, y0, x0 + bw, y0 + bh], 1).astype(np.float32)
    b[::17, 2] = b[::17, 0]          # some zero-area boxes
    b[5::23] = b[3::23][:len(b[5::23])]   # some identical pairs
    return b


@pytest.mark.parametrize("na,nb", [(1, 1), (7, 300), (300, 7), (257, 129), (0, 4)])
def test_iou_matrix_bit_exact(omt, oracle, na, nb):
    rng = np.random.default_rng(20191006 + na + 1000 * nb)
    a, b = _boxes(rng, na), _boxes(rng, nb)
    # shift b near a so that many pairs overlap
    if na and nb:
        b[: min(na, nb)] = a[: min(na, nb)] + rng.uniform(-20, 20, (min(na, nb), 4)).astype(np.float32)
    out = torch.full((max(na, 1), max(nb, 1)), -1.0, dtype=torch.float64, device="cuda")
    ad = torch.from_numpy(a).cuda() if na else torch.zeros((0, 4), device="cuda")
    bd = torch.from_numpy(b).cuda() if nb else torch.zeros((0, 4), device="cuda")
    omt.iou_matrix(ad, bd, out)
    torch.cuda.synchronize()
    want = oracle.iou_matrix(a, b)
    np.testing.assert_array_equal(out.cpu().numpy()[:na, :nb], want)


def test_match_and_update_equals_oracle(omt, oracle):
    # boxes tracked one step on a synthetic clip, matched against the next
    # ground-truth boxes with some detections dropped and some added
    sp = synth.stream_pair(3, workload=13, n_range=(300, 600))
    rng = np.random.default_rng(5)
    pred = sp.boxes + rng.normal(0, 3, sp.boxes.shape).astype(np.float32)
    active = (rng.uniform(0, 1, len(pred)) < 0.9).astype(np.uint8)
    dets = np.concatenate([sp.boxes[rng.uniform(0, 1, len(sp.boxes)) < 0.8],
                           _boxes(rng, 5, *sp.size)]).astype(np.float32)
    for iou_min in (0.0, 0.3):
        boxes, act, ms, md = omt.match_and_update(torch.from_numpy(pred).cuda(), active,
                                                  torch.from_numpy(dets).cuda(), iou_min)
        iou = oracle.iou_matrix(pred, dets)
        oms, omd = oracle.assign(iou, active, iou_min)
        np.testing.assert_array_equal(ms, oms)
        np.testing.assert_array_equal(md, omd)
        ob, oa = oracle.update_tracks(pred, active, dets, oms, omd)
        np.testing.assert_array_equal(boxes, ob)
        np.testing.assert_array_equal(act, oa)
        assert (ms >= 0).sum() >= 0.7 * active.sum()
