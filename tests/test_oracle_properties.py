"""Randomised properties of the FP64 oracle (hypothesis): for arbitrary small ensembles,
the invariants the paper states or its definitions imply hold. CPU only; skipped where
hypothesis is not installed."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

from oracle import pid_oracle as O  # noqa: E402

SETTINGS = settings(max_examples=40, deadline=None)


@st.composite
def ensembles(draw, binary=False):
    N = draw(st.integers(1, 7))
    M = draw(st.integers(1, 40))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    U = rng.uniform(0, 1, (N, M))
    U[rng.uniform(size=(N, M)) < 0.3] = 0.0            # exact zeros, sometimes empty members
    if binary:
        U = (U > 0.5).astype(np.float64)
    w = rng.uniform(0.1, 5.0, M) if draw(st.booleans()) else None
    return U, w, rng


@SETTINGS
@given(ensembles())
def test_range_and_min(e):
    # every fraction and depth lies in [0, 1]; depth is the min of the two fractions (Eq. 10).
    # The oracle's inclusion matrix uses the penalty form of Eq. 14, 1 - sum w u_i (1 - u_j) /
    # m_i: for an empty u_j the two sums are the same numbers added in different orders, so
    # P_ij may round to a few 1e-17 below 0; the range is checked to 1e-12 on both sides.
    U, w, _ = e
    for a, b, d in (O.pid(U, w), O.pid_mean(U, w)):
        assert np.all((a >= -1e-12) & (a <= 1 + 1e-12)) and np.all((b >= -1e-12) & (b <= 1 + 1e-12))
        np.testing.assert_array_equal(d, np.minimum(a, b))


@SETTINGS
@given(ensembles())
def test_cell_permutation_and_split(e):
    # coordinate-agnostic: permuting cells (with their measures) or splitting a cell into
    # two halves of its measure changes nothing
    U, w, rng = e
    M = U.shape[1]
    w1 = np.ones(M) if w is None else w
    perm = rng.permutation(M)
    ref = np.array(O.pid(U, w1))
    np.testing.assert_allclose(np.array(O.pid(U[:, perm], w1[perm])), ref, atol=1e-12)
    k = int(rng.integers(0, M))
    U2 = np.concatenate([U, U[:, k:k + 1]], axis=1)
    w2 = np.concatenate([w1, [w1[k] / 2]])
    w2[k] = w1[k] / 2
    np.testing.assert_allclose(np.array(O.pid(U2, w2)), ref, atol=1e-12)


@SETTINGS
@given(ensembles(), st.floats(0.01, 1.0))
def test_scale_invariance_of_the_first_argument(e, alpha):
    # (alpha u) subset_p v = u subset_p v for alpha in (0, 1] (a property stated in Sec. 3.3)
    U, w, _ = e
    N = U.shape[0]
    for i in range(N):
        for j in range(N):
            assert abs(O.inclusion(alpha * U[i], U[j], w) - O.inclusion(U[i], U[j], w)) < 1e-12


@SETTINGS
@given(ensembles(binary=True))
def test_binary_members_are_eid(e):
    # u in {0, 1}: PID is eID over the sets of cells (Sec. 3.3), with PID's zero-mass
    # convention for an empty reference mask (the eps-subset of an empty set is 1, Eq. 1)
    U, _, _ = e
    N = U.shape[0]
    sets = [set(np.nonzero(U[i])[0].tolist()) for i in range(N)]
    if not all(sets):
        return
    np.testing.assert_allclose(np.array(O.pid(U)), np.array(O.eid(sets)), atol=1e-12)


@SETTINGS
@given(ensembles(), st.integers(1, 9))
def test_block_accumulated_forms(e, nblocks):
    # the block-accumulated forms equal the direct definitions for any block split
    U, w, rng = e
    M = U.shape[1]
    edges = np.unique(np.r_[0, np.sort(rng.integers(0, M + 1, nblocks)), M])
    blocks = [(U[:, a:b], None if w is None else w[a:b]) for a, b in zip(edges[:-1], edges[1:])]
    np.testing.assert_allclose(np.array(O.pid_chunked(iter(blocks))), np.array(O.pid(U, w)),
                               atol=1e-12)
    np.testing.assert_allclose(np.array(O.pid_mean_chunked(iter(blocks))),
                               np.array(O.pid_mean(U, w)), atol=1e-12)


@SETTINGS
@given(ensembles())
def test_recall_identity_and_cv_bound(e):
    # IN_in of full PID equals PID-mean's (Eq. 17); |PID - PID-mean| <= CV of the masses
    U, w, _ = e
    a, b, d = O.pid(U, w)
    am, bm, dm = O.pid_mean(U, w)
    np.testing.assert_allclose(a, am, atol=1e-12)
    m = O.mass(U, w)
    if m.mean() > 0:
        cv = m.std() / m.mean()
        assert np.all(np.abs(d - dm) <= cv + 1e-12)
