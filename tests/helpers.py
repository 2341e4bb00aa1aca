"""Shared test helpers: comparison of library outputs with oracle outputs."""
import numpy as np

FP32_TOL = 1e-6      # FP32 paths vs the FP64 oracle (absolute, on depths and fractions)
ISO_TOL = 3e-7       # the FP32 isovalue map (soft-mask values) vs FP64 erfc
GRAM_TOL = 1e-3      # BF16 / split-BF16 / FP8 tensor-core Gram vs the FP64 oracle


def to_np(t):
    return t.detach().cpu().numpy()


def assert_close(got, want, tol, what=""):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    err = np.max(np.abs(got - want)) if got.size else 0.0
    assert err <= tol, f"{what}: max abs error {err:.3e} > {tol:.1e}"
    return err


def assert_rank_valid(rank, depth):
    """rank must be the ranking of `depth` (descending, ties to the lower index)."""
    rank = np.asarray(rank)
    depth = np.asarray(depth, dtype=np.float64)
    N = depth.shape[0]
    assert sorted(rank.tolist()) == list(range(N)), "rank is not a permutation"
    order = sorted(range(N), key=lambda i: (-depth[i], i))
    expect = np.empty(N, dtype=np.int64)
    expect[order] = np.arange(N)
    assert np.array_equal(rank, expect), "rank does not follow the returned depths"


def assert_rank_agrees_outside_ties(rank, oracle_depth, tol):
    """Pairs whose oracle depths differ by more than 2*tol must be ordered the same way."""
    rank = np.asarray(rank, dtype=np.int64)
    d = np.asarray(oracle_depth, dtype=np.float64)
    diff = d[:, None] - d[None, :]
    firm = np.abs(diff) > 2 * tol
    wrong = firm & (np.sign(diff) != -np.sign(rank[:, None] - rank[None, :]))
    assert not wrong.any(), f"{int(wrong.sum())} member pairs ranked against the oracle order"
