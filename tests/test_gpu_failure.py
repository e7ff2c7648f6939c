"""Failure detection without a GPU fault: a bounded device wait that nothing satisfies gives
up, the call reports DAGRT_E_TIMEOUT and the context stays usable."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2602_20826_gb300 import workloads as wl
from tests.gpu_helpers import context

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as g
    g.build()
    return context()


def test_bounded_wait_gives_up_and_context_survives(ctx):
    from paper_2602_20826_gb300.dagrt import E_TIMEOUT, dagrt_selftest_wait
    for limit in (1, 1000):
        assert dagrt_selftest_wait(ctx.h, limit) == E_TIMEOUT
    assert "gave up" in ctx.last_error()
    b = wl.small_config(2, 6, 5, 40, seed=3)
    lb = ctx.load(b)
    res = lb.schedule(0)
    want, st = oracle.schedule_batch(b)
    assert np.array_equal(res["bound"], want) and (res["status"] == 0).all()
    ctx.sync()
    lb.free()
