"""The serving scheduler on the host, against a fake device backend.

The fake backend records every call and completes each step a fixed time
after submission on a simulated clock, so these checks are exact and fast:
admission under an HBM budget, per-stream frame order, one frame per stream
per step, continuous batching (frames that arrive while a step runs join
the next one), and failures injected on the host (allocation failure,
malformed frames, a stream that stops sending, a delayed producer).
"""
import math

import numpy as np
import pytest

from paper_1910_06017_b300.serve import Backend, Scheduler, StreamSpec


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeBackend(Backend):
    def __init__(self, clock, step_time=0.004, fail_alloc=()):
        self.clock = clock
        self.step_time = step_time
        self.fail_alloc = dict(fail_alloc)   # sid -> failures left
        self.calls = []
        self.live = {}
        self.last_index = {}
        self.busy_until = 0.0      # the device runs one step at a time
        self.handles = []

    def bytes_for(self, spec):
        return spec.size[0] * spec.size[1]

    def alloc(self, spec):
        if self.fail_alloc.get(spec.sid, 0) > 0:
            self.fail_alloc[spec.sid] -= 1
            self.calls.append(("alloc_fail", spec.sid))
            raise MemoryError("injected")
        slot = {"sid": spec.sid}
        self.live[spec.sid] = slot
        self.calls.append(("alloc", spec.sid))
        return slot

    def free(self, slot):
        self.calls.append(("free", slot["sid"]))
        del self.live[slot["sid"]]

    def submit(self, items):
        sids = [slot["sid"] for slot, _ in items]
        assert len(sids) == len(set(sids)), "two frames of one stream in a step"
        for slot, idx in items:
            assert slot["sid"] in self.live, "step for a released stream"
            assert idx > self.last_index.get(slot["sid"], -1), "frames out of order"
            self.last_index[slot["sid"]] = idx
        pending = sum(1 for h in self.handles if not self.done(h))
        self.calls.append(("submit", [(slot["sid"], idx) for slot, idx in items], self.clock(), pending))
        self.busy_until = max(self.clock(), self.busy_until) + self.step_time
        h = {"t": self.busy_until, "items": items}
        self.handles.append(h)
        return h

    def done(self, handle):
        return self.clock() >= handle["t"]


def _specs(n, fps=30.0, frames=20, size=(100, 100), start=0.0, stagger=0.001):
    return [StreamSpec(s, size, 10, 5, start + s * stagger + np.arange(frames) / fps) for s in range(n)]


def _run(specs, budget, **kw):
    clk = FakeClock()
    be = FakeBackend(clk, **{k: v for k, v in kw.items() if k in ("step_time", "fail_alloc")})
    sch = Scheduler(be, budget, clock=clk, **{k: v for k, v in kw.items()
                                              if k in ("max_in_flight", "idle_timeout", "frame_ok")})
    stats = sch.run(specs, deadline=60.0, sleep=clk.sleep)
    return stats, be


def test_every_frame_in_order_and_once():
    specs = _specs(6)
    stats, be = _run(specs, budget=10 ** 9)
    s = stats.summary()
    assert s["frames_done"] == 6 * 20 and s["frames_rejected"] == 0
    done = {(f.sid, f.index) for f in stats.frames if not math.isnan(f.done)}
    assert done == {(sid, i) for sid in range(6) for i in range(20)}
    assert all(f.latency >= 0 for f in stats.frames)
    assert [c[0] for c in be.calls].count("free") == 6 and not be.live


def test_budget_admission_queues_streams():
    specs = _specs(5, frames=10)
    budget = 2 * 100 * 100            # two streams fit at a time
    stats, be = _run(specs, budget)
    assert stats.summary()["frames_done"] == 50
    assert stats.max_bytes_in_use <= budget
    # never more than two streams resident at once
    live = peak = 0
    for c in be.calls:
        if c[0] == "alloc":
            live += 1
            peak = max(peak, live)
        elif c[0] == "free":
            live -= 1
    assert peak == 2
    # admitted in order of first arrival
    assert [c[1] for c in be.calls if c[0] == "alloc"] == [0, 1, 2, 3, 4]


def test_continuous_batching_joins_running_work():
    # 8 streams at 60 fps with a step of 10 ms: frames arriving during a
    # running step must join the next step rather than wait for a queue slot
    specs = _specs(8, fps=60.0, frames=30, stagger=0.0007)
    stats, be = _run(specs, budget=10 ** 9, step_time=0.010, max_in_flight=2)
    s = stats.summary()
    assert s["frames_done"] == 240
    assert s["mean_batch"] > 2.0
    submits = [c for c in be.calls if c[0] == "submit"]
    # never more than two steps outstanding: at most one unfinished at a submit
    assert max(c[3] for c in submits) <= 1
    assert s["latency_ms_p99"] < 40.0


def test_injected_allocation_failure_is_retried():
    specs = _specs(3, frames=8)
    stats, be = _run(specs, budget=10 ** 9, fail_alloc={1: 3})
    assert stats.summary()["frames_done"] == 24
    assert [c[1] for c in be.calls if c[0] == "alloc_fail"] == [1, 1, 1]
    assert sum(1 for c in be.calls if c[0] == "alloc") == 3


def test_malformed_frames_are_dropped_not_fatal():
    specs = _specs(3, frames=12)
    bad = {(1, 4), (1, 5), (2, 0)}
    stats, be = _run(specs, budget=10 ** 9, frame_ok=lambda sid, i: (sid, i) not in bad)
    s = stats.summary()
    assert s["frames_rejected"] == 3 and s["frames_done"] == 36 - 3
    submitted = {(sid, i) for c in be.calls if c[0] == "submit" for sid, i in c[1]}
    assert not (submitted & bad)


def test_stream_that_stops_sending_is_released():
    # stream 0 sends 5 frames then goes silent for 5 s (a disconnect); with
    # room for one stream only, stream 1 must get in after the idle timeout
    s0 = StreamSpec(0, (100, 100), 10, 5, np.concatenate([np.arange(5) / 30.0, [5.0]]))
    s1 = StreamSpec(1, (100, 100), 10, 5, 0.01 + np.arange(10) / 30.0)
    stats, be = _run([s0, s1], budget=100 * 100, idle_timeout=0.5)
    allocs = [c for c in be.calls if c[0] in ("alloc", "free")]
    assert allocs[:3] == [("alloc", 0), ("free", 0), ("alloc", 1)]
    done = {(f.sid, f.index) for f in stats.frames if not math.isnan(f.done)}
    assert {(1, i) for i in range(10)} <= done
    assert (0, 5) not in done        # the disconnected stream's late frame is not served


def test_delayed_producer_latency_counts_from_arrival():
    # frames of stream 0 are produced 0.2 s late in a burst: latency is
    # measured from each frame's arrival time, and frames stay in order
    arr = np.concatenate([np.arange(5) / 30.0, 0.4 + np.arange(5) * 1e-4])
    specs = [StreamSpec(0, (100, 100), 10, 5, arr)]
    stats, be = _run(specs, budget=10 ** 9, step_time=0.004)
    fr = sorted(stats.frames, key=lambda f: f.index)
    assert all(not math.isnan(f.done) for f in fr)
    assert all(f.done >= f.arrival for f in fr)
    # the burst is served one frame per step
    assert fr[-1].latency >= 4 * 0.004


@pytest.mark.parametrize("threshold", [0.3, 1.0, 5.0, 40.0])
def test_capacity_search_brackets_the_threshold(threshold):
    from paper_1910_06017_b300.serve import search_scale
    seen = []

    def probe(scale):
        seen.append(scale)
        return scale <= threshold, scale

    best = search_scale(probe, bisect=4)
    assert best is not None and best <= threshold
    # four geometric bisections of a factor-2 bracket leave < 2^(1/16) of slack
    assert best > threshold / 2 ** (1 / 16) - 1e-12
    assert len(seen) <= 2 + int(math.ceil(abs(math.log2(threshold)))) + 4


def test_capacity_search_none_passes():
    from paper_1910_06017_b300.serve import search_scale
    assert search_scale(lambda s: (False, s), limit=8.0) is None
