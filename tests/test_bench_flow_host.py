"""Host-side arithmetic of bench.py's dense-flow line: the kernel launches
one frame takes (the figure reported as gpu_launches; the launch list of one
step under ncu counts 252 for the default parameters) and the algorithmic
bytes of the primal-dual launches behind the roofline."""
import os
import sys
from types import SimpleNamespace

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _fp(**kw):
    base = dict(st_iters=100, iters=30, warps=3, block=2)
    base.update(kw)
    return SimpleNamespace(**base)


def test_default_step_launches_match_the_launch_list():
    # 50 two-step projection launches + texture, 4 pyramid levels, per level
    # the upsampling and per warp the warp kernel and 15 pair launches, box means
    assert bench.FLOW_LEVELS == 4
    assert bench.flow_launches_per_step(_fp()) == 50 + 1 + 4 + 4 * (1 + 3 * (1 + 15)) + 1 == 252


@pytest.mark.parametrize("st_iters,iters,warps,block,want", [
    (100, 30, 3, 1, 100 + 1 + 4 + 4 * (1 + 3 * 31) + 1),
    (7, 5, 3, 2, 4 + 1 + 4 + 4 * (1 + 3 * (1 + 3)) + 1),   # odd counts: one single launch each
    (0, 1, 1, 2, 0 + 1 + 4 + 4 * (1 + 1 * (1 + 1)) + 1),
])
def test_launch_count_follows_the_parameters(st_iters, iters, warps, block, want):
    assert bench.flow_launches_per_step(_fp(st_iters=st_iters, iters=iters, warps=warps,
                                            block=block)) == want


def test_bytes_per_launch_count_each_launch_once():
    area = sum(4.0 ** -L for L in range(bench.FLOW_LEVELS))
    # two iterations per launch move the 76-byte state once
    assert bench.flow_bytes_per_l0px(None, _fp()) == pytest.approx(76 * 3 * 15 * area)
    assert bench.flow_bytes_per_l0px(None, _fp(block=1)) == pytest.approx(76 * 3 * 30 * area)
    assert bench.flow_bytes_per_l0px(None, _fp(iters=5)) == pytest.approx(76 * 3 * 3 * area)
