"""GPU parity of the dense flow engine (structure-texture, Huber-TV-L1,
mean-in-box prediction; Sections IV and V-A) against the FP64 oracle,
through the C-ABI.

Bars.  The u8 texture: FP32 and FP64 ROF structures differ by rounding, so
a texel whose scaled texture sits within that rounding of a .5 boundary may
round the other way: at most 0.5 % of the texels, by one level.  The flow
is compared on identical u8 inputs (the oracle's texture frames); the
primal-dual map is continuous and non-expansive, so FP32 rounding stays of
the order of the iterations times the FP32 epsilon of the flow (a few px):
the bar is 2e-3 px at every pixel and 1e-4 px on average.  Identical frames
give exactly zero flow on both.  The box means are compared within 1e-4 px.
"""
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


def _t(a, dt=None):
    return torch.from_numpy(np.ascontiguousarray(a if dt is None else a.astype(dt))).cuda()


def _pyr(omt, frame, levels):
    h, w = frame.shape
    P = omt.Pyramid(w, h, levels, 0)
    omt.build_pyramid(_t(frame, np.uint8), P, omt.default_params(levels=levels))
    return P


def _scene(w, h, shift, seed=3):
    rng = np.random.default_rng(seed)
    tex = synth.Texture.draw(rng, w, h)
    return synth.render_shift(tex, w, h, 0, 0), synth.render_shift(tex, w, h, *shift)


@pytest.mark.parametrize("size", [(160, 120), (720, 576), (37, 23)])
def test_structure_texture_matches_oracle(omt, oracle, size):
    w, h = size
    f0, _ = _scene(w, h, (0, 0), seed=w)
    want = oracle.structure_texture(f0)
    fp = omt.default_flow_params()
    out = torch.zeros((h, w), dtype=torch.uint8, device="cuda")
    omt.structure_texture(_t(f0, np.uint8), fp, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(int)
    d = np.abs(got - want.astype(int))
    assert d.max() <= 1 and (d > 0).mean() <= 0.005, (d.max(), (d > 0).mean())


def _flows(omt, oracle, T0, T1, levels, fp=None):
    h, w = T0.shape
    fp = fp or omt.default_flow_params()
    P0, P1 = _pyr(omt, T0, levels), _pyr(omt, T1, levels)
    flow = torch.zeros((h, w, 2), device="cuda")
    omt.tvl1_flow(P0, P1, fp, flow)
    torch.cuda.synchronize()
    want = oracle.tvl1(oracle.Pyramid(T0, levels), oracle.Pyramid(T1, levels), fp.lambda_, fp.eps,
                       fp.warps, fp.iters)
    return flow.cpu().numpy(), want


@pytest.mark.parametrize("size,shift,levels", [((160, 120), (1.37, -0.62), 3),
                                               ((320, 240), (5.5, 3.25), 4),
                                               ((61, 47), (-2.0, 0.75), 2)])
def test_tvl1_matches_oracle(omt, oracle, size, shift, levels):
    w, h = size
    f0, f1 = _scene(w, h, shift, seed=w + h)
    T0, T1 = oracle.structure_texture(f0), oracle.structure_texture(f1)
    got, want = _flows(omt, oracle, T0, T1, levels)
    err = np.abs(got - want)
    print(f"tvl1 {size} {shift}: |gpu - oracle| max {err.max():.2e} mean {err.mean():.2e}")
    assert err.max() <= 2e-3 and err.mean() <= 1e-4, (err.max(), err.mean())
    # and the field is the motion: the interior recovers the shift (frames
    # large enough to have an interior away from the borders)
    if min(w, h) >= 100:
        inner = got[h // 6:-h // 6, w // 6:-w // 6].reshape(-1, 2)
        assert np.allclose(np.median(inner, 0), shift, atol=0.05)


@pytest.mark.parametrize("size,st_iters", [((37, 23), 7), ((333, 250), 100), ((1, 1), 3)])
def test_structure_texture_two_steps_per_launch_same_bits(omt, size, st_iters):
    # one projection step per launch and two per launch (the last one alone
    # when the count is odd) give the same texture bit for bit
    w, h = size
    f0, _ = _scene(w, h, (0, 0), seed=w * 3)
    outs = []
    for block in (1, 2):
        fp = omt.default_flow_params(st_iters=st_iters, block=block)
        out = torch.zeros((h, w), dtype=torch.uint8, device="cuda")
        omt.structure_texture(_t(f0, np.uint8), fp, out)
        outs.append(out.cpu().numpy())
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("size,shift,levels,warps,iters", [((333, 250), (3.3, -1.7), 3, 3, 5),
                                                           ((97, 61), (1.25, 0.5), 1, 1, 30),
                                                           ((160, 120), (0.6, 2.2), 2, 2, 1),
                                                           ((65, 33), (-1.0, 1.0), 2, 3, 4),
                                                           ((200, 150), (1.5, -2.0), 3, 3, 2)])
def test_tvl1_two_iterations_per_launch_same_bits(omt, oracle, size, shift, levels, warps, iters):
    # pairs of iterations per launch (with the flow ping-ponged, an odd count
    # of swaps per level, a single iteration left over) equal one iteration
    # per launch bit for bit, on ragged tiles
    w, h = size
    f0, f1 = _scene(w, h, shift, seed=w + 2 * h)
    T0, T1 = oracle.structure_texture(f0), oracle.structure_texture(f1)
    P0, P1 = _pyr(omt, T0, levels), _pyr(omt, T1, levels)
    flows = []
    for block in (1, 2):
        fp = omt.default_flow_params(warps=warps, iters=iters, block=block)
        flow = torch.full((h, w, 2), float("nan"), device="cuda")
        omt.tvl1_flow(P0, P1, fp, flow)
        flows.append(flow.cpu().numpy())
    assert np.all(np.isfinite(flows[1]))
    np.testing.assert_array_equal(flows[0], flows[1])


def test_tvl1_identical_frames_zero(omt, oracle):
    f0, _ = _scene(96, 80, (0, 0), seed=9)
    T = oracle.structure_texture(f0)
    got, want = _flows(omt, oracle, T, T, 3)
    assert np.all(got == 0.0) and np.all(want == 0.0)


def test_box_mean_flow_matches_oracle(omt, oracle):
    rng = np.random.default_rng(12)
    h, w = 120, 160
    flow = rng.normal(0, 3, (h, w, 2)).astype(np.float32)
    boxes = np.concatenate([rng.uniform(-20, 180, (60, 2)), rng.uniform(0, 60, (60, 2))], 1)
    boxes[:, 2:] += boxes[:, :2]
    boxes = np.concatenate([boxes, [[200, 200, 300, 300], [10.5, 10.5, 11.0, 11.0],
                                    [0, 0, w, h]]]).astype(np.float32)
    out = torch.zeros((len(boxes), 4), device="cuda")
    omt.box_mean_flow(_t(flow), _t(boxes), out)
    torch.cuda.synchronize()
    want = oracle.box_mean_flow(flow.astype(np.float64), boxes)
    np.testing.assert_allclose(out.cpu().numpy(), want, atol=1e-4)


def test_end_to_end_translation(omt, oracle):
    # u8 frames -> GPU textures -> GPU pyramids -> GPU flow -> box means
    w, h = 320, 240
    f0, f1 = _scene(w, h, (2.25, -1.5), seed=31)
    fp = omt.default_flow_params()
    T = [torch.zeros((h, w), dtype=torch.uint8, device="cuda") for _ in range(2)]
    for f, t in zip((f0, f1), T):
        omt.structure_texture(_t(f, np.uint8), fp, t)
    P = []
    for t in T:
        p = omt.Pyramid(w, h, 3, 0)
        omt.build_pyramid(t, p, omt.default_params(levels=3))
        P.append(p)
    flow = torch.zeros((h, w, 2), device="cuda")
    omt.tvl1_flow(P[0], P[1], fp, flow)
    boxes = _t(np.array([[60, 40, 260, 200], [100, 80, 140, 120]], np.float32))
    out = torch.zeros((2, 4), device="cuda")
    omt.box_mean_flow(flow, boxes, out)
    torch.cuda.synchronize()
    moved = out.cpu().numpy() - boxes.cpu().numpy()
    np.testing.assert_allclose(moved[:, :2], [[2.25, -1.5]] * 2, atol=0.05)


def test_flow_step_captured_in_a_cuda_graph(omt):
    # the whole flow step (texture, pyramid, flow, box means; kernels chained
    # by programmatic dependent launch) captured once and replayed equals
    # the eager calls bit for bit, and a replay reads the frame it is given
    w, h = 160, 120
    f0, f1 = _scene(w, h, (1.75, -0.5), seed=44)
    fp = omt.default_flow_params()
    prm = omt.default_params(levels=3)
    frames = [_t(f, np.uint8) for f in (f0, f1)]
    tex = [torch.zeros((h, w), dtype=torch.uint8, device="cuda") for _ in range(2)]
    pyr = [omt.Pyramid(w, h, 3, 0) for _ in range(2)]
    st_scr = torch.empty(omt.lib().omt_structure_texture_scratch_bytes(w, h), dtype=torch.uint8,
                         device="cuda")
    tv_scr = torch.empty(omt.lib().omt_tvl1_scratch_bytes(w, h), dtype=torch.uint8, device="cuda")
    flow = torch.zeros((h, w, 2), device="cuda")
    boxes = _t(np.array([[20, 10, 120, 90], [50, 40, 70, 60]], np.float32))
    out = torch.zeros((2, 4), device="cuda")
    src = torch.zeros((h, w), dtype=torch.uint8, device="cuda")

    def prime(k):
        omt.structure_texture(frames[k], fp, tex[k], st_scr)
        omt.build_pyramid(tex[k], pyr[k], prm)

    def step():
        # src holds frame 1 of the pair; its texture and pyramid, then the flow
        omt.structure_texture(src, fp, tex[1], st_scr)
        omt.build_pyramid(tex[1], pyr[1], prm)
        omt.tvl1_flow(pyr[0], pyr[1], fp, flow, tv_scr)
        omt.box_mean_flow(flow, boxes, out)

    prime(0)
    src.copy_(frames[1])
    step()
    torch.cuda.synchronize()
    want_flow, want_out = flow.clone(), out.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            step()
    torch.cuda.synchronize()
    flow.zero_()
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(flow, want_flow) and torch.equal(out, want_out)
    # the replay reads the new frame: frame 0 again gives exactly zero flow
    src.copy_(frames[0])
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(flow == 0) and torch.equal(out, boxes)
