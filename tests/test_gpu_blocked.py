"""GPU parity of PID-mean and the exact full PID for ensembles larger than the fused
kernel's tile (N > 512: member-blocked column sums, then per-member sums), against the FP64
oracle: soft masks, weighted cells and fields, ranks across the CTA-sized finalisation
(N > 1024), up to N = 40 000 members."""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import FP32_TOL, assert_close, assert_rank_valid, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2512_15187_gb300 import binding, build
    build.build()
    h = binding.Handle(0)
    yield h
    h.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(o, ref, what):
    a, b, d = ref
    assert_close(to_np(o["in_in"]), a, FP32_TOL, what + " in_in")
    assert_close(to_np(o["in_out"]), b, FP32_TOL, what + " in_out")
    assert_close(to_np(o["depth"]), d, FP32_TOL, what + " depth")
    assert_rank_valid(to_np(o["rank"]), to_np(o["depth"]))


@pytest.mark.parametrize("N,M", [(513, 777), (1000, 20000), (1025, 4096), (3000, 2001)])
@pytest.mark.parametrize("weighted", [False, True])
def test_blocked_mean_and_linear(H, N, M, weighted):
    U = synth.random_soft(N, M, seed=N + M, binary_frac=0.2)
    w = np.random.default_rng(M).uniform(0.2, 5, M).astype(np.float32) if weighted else None
    Ud, wd = _dev(U), (None if w is None else _dev(w))
    o = H.mean(Ud, wd)
    H.sync()
    _check(o, O.pid_mean(U, w), f"mean N={N}")
    o = H.full(Ud, wd, mode="linear")
    H.sync()
    _check(o, O.pid(U, w), f"linear N={N}")


def test_blocked_fields(H):
    N, Hh, W = 700, 40, 50
    F = synth.rbf_fields_2d(N=N, H=Hh, W=W, n_rbf=6)
    F = (F - np.median(F, axis=1, keepdims=True) + 0.5).astype(np.float32)
    o = H.from_fields(_dev(F), 0.5, 0.1, mode="linear")
    H.sync()
    _check(o, O.pid(O.iso_soft_mask(F, 0.5, 0.1)), "fields linear N=700")


def test_blocked_forty_thousand_members(H):
    N, M = 40000, 1000
    U = synth.random_soft(N, M, seed=40000)
    o = H.mean(_dev(U))
    H.sync()
    _check(o, O.pid_mean(U), "mean N=40000")


def test_blocked_rejections(H):
    import torch
    from paper_2512_15187_gb300 import binding as B
    U = torch.rand((600, 300), device="cuda")
    with pytest.raises(B.PidError) as e:
        H.full(U, mode="full", precision="bf16")
    assert e.value.status == B.PID_ERR_UNSUPPORTED
    with pytest.raises(B.PidError) as e:
        H.batch([dict(data=U, mode="mean")])
    assert e.value.status == B.PID_ERR_UNSUPPORTED
