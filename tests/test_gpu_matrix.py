"""GPU parity of PID from an inclusion matrix (pid_depth_from_matrix): the FP64 oracle's
exact matrix in, depths within groups of members (multimodal ensembles, Sec. 2.2) against
the oracle's PID of each group's own sub-ensemble; ranks within groups exactly; the
tensor-core Gram's matrix in, the same depths pid_full returns; and the host checks."""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import GRAM_TOL, assert_close, assert_rank_agrees_outside_ties, to_np

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


@pytest.mark.parametrize("N,M,n_groups", [(1, 50, 1), (7, 300, 1), (40, 1000, 3), (300, 500, 7),
                                          (257, 200, 257), (700, 100, 2)])
def test_groups_against_the_oracle_subensembles(H, N, M, n_groups):
    rng = np.random.default_rng(N)
    U = synth.random_soft(N, M, seed=N + 1, binary_frac=0.2)
    U[rng.integers(0, N)] = 0.0                      # an empty member: inclusions 0
    labels = rng.integers(0, n_groups, N).astype(np.int32) * 7 - 3
    w = rng.uniform(0.5, 2.0, M)
    P = O.inclusion_matrix(U, w)
    o = H.depth_from_matrix(_dev(P), _dev(labels))
    ref = O.pid_grouped(U, labels, w)
    for k, r in zip(("in_in", "in_out", "depth"), ref[:3]):
        assert_close(to_np(o[k]), r, 1e-12, f"N={N} groups={n_groups} {k}")
    assert np.array_equal(to_np(o["rank"]), ref[3])


def test_no_labels_reproduces_the_gram_depths(H):
    U = _dev(synth.random_soft(100, 20000, seed=5))
    full = H.full(U, mode="full", precision="bf16", want_P=True)
    o = H.depth_from_matrix(full["P"])
    # pid_full takes IN_in from the exact PID-mean identity and sums the calibrated FP32
    # Gram in its own order; the means of the P it returns agree to the calibration's
    # FP32 tolerance
    for k in ("in_in", "in_out", "depth"):
        assert_close(to_np(o[k]), to_np(full[k]), 2e-6, k)
    assert_rank_agrees_outside_ties(to_np(o["rank"]), to_np(full["depth"]), 2e-6)
    ref = O.pid(to_np(U))
    assert_close(to_np(o["depth"]), ref[2], GRAM_TOL, "vs oracle")


def test_strided_matrix_and_host_checks(H):
    import torch
    from paper_2512_15187_gb300 import binding as B
    U = synth.random_soft(33, 400, seed=2)
    P = O.inclusion_matrix(U)
    big = torch.zeros((33, 40), dtype=torch.float64, device="cuda")
    big[:, :33] = _dev(P)
    o = H.depth_from_matrix(big[:, :33])
    assert_close(to_np(o["depth"]), O.pid(U)[2], 1e-12, "strided P")
    with pytest.raises(ValueError):
        H.depth_from_matrix(big)                                        # not square
    with pytest.raises(ValueError):
        H.depth_from_matrix(_dev(P), torch.zeros(32, dtype=torch.int32, device="cuda"))
    with pytest.raises(B.PidError):
        B.pid_depth_from_matrix(H.h, big.data_ptr(), 33, 20, None, None, None, None, None)
