"""GPU parity of 4D space-time PID (pid_spacetime: time as one more cell axis) with the
FP64 oracle on the concatenated cells (x, t): PID-mean, exact linear full PID and the
tensor-core Gram with its inclusion matrix, soft masks and fields, cell measures, steps as
separate allocations and as strided views, one step against the single call bit for bit,
graph replay with new contents, and the host checks."""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import (FP32_TOL, GRAM_TOL, assert_close, assert_rank_agrees_outside_ties,
                           assert_rank_valid, to_np)

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


def _steps(T, N, M, seed):
    return [synth.random_soft(N, M, seed=seed + 31 * t, binary_frac=0.2) for t in range(T)]


@pytest.mark.parametrize("T,N,M", [(1, 5, 300), (3, 24, 5003), (17, 64, 1024), (4, 200, 2500),
                                   (2, 300, 1500), (40, 9, 129)])
@pytest.mark.parametrize("mode", ["mean", "linear"])
@pytest.mark.parametrize("cellw", [False, True])
def test_spacetime_soft_masks(H, T, N, M, mode, cellw):
    S = _steps(T, N, M, seed=T + N)
    w = np.random.default_rng(M).uniform(0.2, 4.0, M).astype(np.float32) if cellw else None
    o = H.spacetime([_dev(x) for x in S], w=None if w is None else _dev(w), mode=mode)
    H.sync()
    U, wt = O.spacetime_cells(S, w)
    ref = O.pid_mean(U, wt) if mode == "mean" else O.pid(U, wt)
    for k, r in zip(("in_in", "in_out", "depth"), ref):
        assert_close(to_np(o[k]), r, FP32_TOL, f"T={T} N={N} {mode} {k}")
    assert_rank_valid(to_np(o["rank"]), to_np(o["depth"]))


@pytest.mark.parametrize("T,N,precision", [(3, 64, "bf16"), (5, 150, "bf16"), (2, 40, "fp8"),
                                           (3, 33, "split_bf16")])
def test_spacetime_gram_and_inclusion_matrix(H, T, N, precision):
    M = 4100
    S = _steps(T, N, M, seed=N)
    w = np.random.default_rng(5).uniform(0.5, 2.0, M).astype(np.float32)
    o = H.spacetime([_dev(x) for x in S], w=_dev(w), mode="full", precision=precision,
                    want_P=True)
    H.sync()
    U, wt = O.spacetime_cells(S, w)
    ref = O.pid(U, wt)
    for k, r in zip(("in_in", "in_out", "depth"), ref):
        assert_close(to_np(o[k]), r, GRAM_TOL, f"gram T={T} {precision} {k}")
    assert_rank_agrees_outside_ties(to_np(o["rank"]), ref[2], GRAM_TOL)
    assert_close(to_np(o["P"]), O.inclusion_matrix(U, wt), GRAM_TOL, "P")


@pytest.mark.parametrize("iso", [(0.5, 0.05, 0), (0.5, 0.0, 1), (0.5, 0.1, 0, "level"),
                                 (0.5, 0.1, 1, "uniform")])
@pytest.mark.parametrize("mode", ["mean", "linear"])
def test_spacetime_fields(H, iso, mode):
    T, N = 4, 30
    S = []
    for t in range(T):
        F = synth.rbf_fields_2d(N=N, H=40, W=50, n_rbf=8, seed=synth.DEFAULT_SEED + 60 + t)
        S.append((F - np.median(F, axis=1, keepdims=True) + 0.5).astype(np.float32))
    o = H.spacetime([_dev(x) for x in S], iso=iso, mode=mode)
    H.sync()
    kind = iso[3] if len(iso) > 3 else "normal"
    if kind == "normal":
        masks = [O.iso_soft_mask(F, iso[0], iso[1], bool(iso[2])) for F in S]
    elif kind == "level":
        masks = [O.level_soft_mask(F, iso[0], iso[1]) for F in S]
    else:
        masks = [O.iso_soft_mask_uniform(F, iso[0], iso[1], bool(iso[2])) for F in S]
    U, _ = O.spacetime_cells(masks)
    ref = O.pid_mean(U) if mode == "mean" else O.pid(U)
    for k, r in zip(("in_in", "in_out", "depth"), ref):
        assert_close(to_np(o[k]), r, FP32_TOL, f"fields {iso} {mode} {k}")


def test_strided_views_of_one_array_and_replay(H):
    """Steps as views [t] of one [T][N][ld] tensor with ld > M; a second call with the same
    layout replays the recorded graph and must read the new contents."""
    import torch
    T, N, M = 6, 20, 777
    big = torch.zeros((T, N, M + 5), dtype=torch.float32, device="cuda")
    S = _steps(T, N, M, seed=3)
    for t in range(T):
        big[t, :, :M] = _dev(S[t])
    views = [big[t, :, :M] for t in range(T)]
    for rep in range(3):
        if rep == 2:
            big.mul_(0.5).add_(torch.rand_like(big) * 0.5)
            S = [to_np(big[t, :, :M]) for t in range(T)]
        o = H.spacetime(views, mode="linear")
        H.sync()
        ref = O.pid(O.spacetime_cells(S)[0])
        assert_close(to_np(o["depth"]), ref[2], FP32_TOL, f"rep {rep}")


def test_one_step_equals_the_single_call_bitwise(H):
    U = _dev(synth.random_soft(50, 6000, seed=4))
    for mode in ("mean", "linear"):
        a = H.spacetime([U], mode=mode)
        b = H.full(U, mode=mode) if mode != "mean" else H.mean(U)
        H.sync()
        for k in ("in_in", "in_out", "depth", "rank"):
            assert np.array_equal(to_np(a[k]), to_np(b[k])), (mode, k)


def test_host_checks(H):
    import torch
    from paper_2512_15187_gb300 import binding as B
    a = torch.rand((8, 100), device="cuda")
    with pytest.raises(ValueError):
        H.spacetime([])
    with pytest.raises(ValueError):
        H.spacetime([a, torch.rand((8, 101), device="cuda")])
    with pytest.raises(B.PidError):
        H.spacetime([torch.rand((513, 64), device="cuda")] * 2)       # N beyond one tile
    with pytest.raises(B.PidError):
        H.spacetime([torch.rand((513, 64), device="cuda")] * 2, mode="full", precision="bf16")
    o = H.spacetime([a, a], mode="mean")                               # still usable
    H.sync()
    assert_close(to_np(o["depth"]), O.pid_mean(to_np(a))[2], FP32_TOL, "after errors")
