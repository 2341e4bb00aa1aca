"""GPU tests of the tile-shape autotuner (pid_autotune_shapes).

A tuned shape (streaming tile class, Gram cell chunk) changes the launch, and so the order
of the FP32 sums, but the results stay within the bars against the FP64 oracle, and a batch
stays bitwise equal to its single calls on the same handle.
"""
import os

import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import FP32_TOL, GRAM_TOL, assert_close, to_np

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture()
def forced_handle(tmp_path, monkeypatch):
    """A handle whose tune cache pins N = 100, M = 2^16 soft masks to the 192-row streaming
    class (index 8; the default for 100 members is the 128-row class, index 7) and doubles
    the BF16 Gram's chunk."""
    from paper_2512_15187_gb300 import binding, build
    build.build()
    cache = tmp_path / "tune.txt"
    cache.write_text("shape stream n100 m16 iso0 w0|8\nshape gram n100 m16 p1 iso0 w0|1\n")
    monkeypatch.setenv("PID_AUTOTUNE_CACHE", str(cache))
    h = binding.Handle(0)
    yield h
    h.close()


def test_a_tuned_shape_changes_the_launch_and_stays_exact(forced_handle, monkeypatch):
    import torch
    from paper_2512_15187_gb300 import binding
    H = forced_handle
    desc = H.autotune_describe()
    assert "shape stream n100 m16 iso0 w0 -> 8" in desc, desc
    Un = synth.random_soft(100, 1 << 16, seed=41)
    U = _dev(Un)
    tuned = H.mean(U)
    lin = H.full(U, mode="linear")
    gram = H.full(U, mode="full", precision="bf16")
    H.sync()
    ref_mean, ref_full = O.pid_mean(Un), O.pid(Un)
    assert_close(to_np(tuned["depth"]), ref_mean[2], FP32_TOL, "tuned class PID-mean")
    assert_close(to_np(lin["depth"]), ref_full[2], FP32_TOL, "tuned class exact full PID")
    assert_close(to_np(gram["depth"]), ref_full[2], GRAM_TOL, "tuned chunk BF16 Gram")
    # a handle without the cache runs the 128-row class: a different order of the FP32 sums
    monkeypatch.delenv("PID_AUTOTUNE_CACHE")
    d = binding.Handle(0)
    assert "shape" not in d.autotune_describe()
    dflt = d.mean(U)
    d.sync()
    d.close()
    assert not torch.equal(tuned["in_in"], dflt["in_in"]) or not torch.equal(tuned["in_out"], dflt["in_out"])
    # batch and single calls plan with the same tuned shape: bitwise equal (the Gram item is
    # batched without a PID-mean item of the same masks, whose sums it would take)
    U2 = _dev(synth.random_soft(100, 1 << 16, seed=42))
    outs = H.batch([dict(data=U, mode="mean"), dict(data=U2, mode="mean")])
    gouts = H.batch([dict(data=U, mode="full", precision="bf16"), dict(data=U2, mode="mean")])
    H.sync()
    for k in ("depth", "in_in", "in_out", "rank"):
        assert torch.equal(outs[0][k], tuned[k]), k
        assert torch.equal(gouts[0][k], gram[k]), k


def test_autotune_shapes_records_winners_and_results_match(tmp_path, monkeypatch):
    import torch
    from paper_2512_15187_gb300 import binding, build
    build.build()
    monkeypatch.setenv("PID_AUTOTUNE_CACHE", str(tmp_path / "tune.txt"))
    h = binding.Handle(0)
    Un = synth.random_soft(150, 300000, seed=5)
    U = _dev(Un)
    items = [dict(data=U, mode="mean"), dict(data=U, mode="full", precision="split_bf16")]
    h.autotune_shapes(items)
    desc = h.autotune_describe()
    assert "shape stream n150 m18 iso0 w0" in desc and "shape gram n150 m18 p2 iso0 w0" in desc, desc
    assert "shape stream n150" in open(tmp_path / "tune.txt").read()
    outs = h.batch(items)
    single = h.mean(U)
    h.sync()
    assert_close(to_np(outs[0]["depth"]), O.pid_mean(Un)[2], FP32_TOL, "tuned PID-mean")
    assert_close(to_np(outs[1]["depth"]), O.pid(Un)[2], GRAM_TOL, "tuned split Gram")
    for k in ("depth", "in_in", "in_out", "rank"):
        assert torch.equal(outs[0][k], single[k]), k
    # a second handle loads the winners from the cache file
    h2 = binding.Handle(0)
    assert "shape stream n150 m18 iso0 w0" in h2.autotune_describe()
    h2.close()
    h.close()
