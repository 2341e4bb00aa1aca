"""Failure handling on the GPU without a fault: a bounded device wait that nothing satisfies
gives up, the handle's error word reports it as PID_ERR_TIMEOUT at the next pid_sync, the
word is cleared, and the context keeps computing correct results."""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import FP32_TOL, assert_close, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2512_15187_gb300 import binding, build
    build.build()
    h = binding.Handle(0)
    yield h
    h.close()


def test_bounded_wait_times_out_and_the_context_survives(H):
    import torch
    from paper_2512_15187_gb300 import binding as B
    lib = B.load()
    assert lib.pid_selftest_wait_timeout(H.h, 0.2, None) == B.PID_OK
    assert lib.pid_sync(H.h, None) == B.PID_ERR_TIMEOUT
    assert lib.pid_sync(H.h, None) == B.PID_OK          # the word was cleared
    U = synth.random_soft(20, 5000, seed=4)
    o = H.mean(torch.from_numpy(U).cuda())
    H.sync()
    assert_close(to_np(o["depth"]), O.pid_mean(U)[2], FP32_TOL, "after the timeout")


def test_selftest_rejects_long_waits(H):
    from paper_2512_15187_gb300 import binding as B
    lib = B.load()
    for s in (0.0, -1.0, 2.5):
        assert lib.pid_selftest_wait_timeout(H.h, s, None) == B.PID_ERR_INVALID_ARG
