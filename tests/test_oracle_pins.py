"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

No test here re-types an oracle formula: each checks the oracle against a
hand-worked example, a closed form, brute-force set counts, an invariant the
paper states, or a textbook/library value. CPU only.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import ndtr

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --- hand-worked examples (tests/golden) -------------------------------------------

def test_hand_weighted_example():
    g = _load("hand_weighted_2x3.json")
    U, w = np.array(g["U"]), np.array(g["w"])
    np.testing.assert_allclose(O.mass(U, w), g["mass"], rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.inclusion_matrix(U, w), g["P"], rtol=0, atol=1e-15)
    a, b, d = O.pid(U, w)
    np.testing.assert_allclose(a, g["pid_in_in"], atol=1e-15)
    np.testing.assert_allclose(b, g["pid_in_out"], atol=1e-15)
    np.testing.assert_allclose(d, g["pid_depth"], atol=1e-15)
    a, b, d = O.pid_mean(U, w)
    np.testing.assert_allclose(a, g["mean_in_in"], atol=1e-15)
    np.testing.assert_allclose(b, g["mean_in_out"], atol=1e-15)
    np.testing.assert_allclose(d, g["mean_depth"], atol=1e-15)
    assert list(O.rank_by_depth(O.pid(U, w)[2])) == g["rank"]


def test_hand_binary_with_empty_member():
    g = _load("hand_binary_empty_3x4.json")
    U = np.array(g["U"], dtype=np.float64)
    a, b, d = O.pid(U)
    np.testing.assert_allclose(a, g["pid_in_in"], atol=1e-15)
    np.testing.assert_allclose(b, g["pid_in_out"], atol=1e-15)
    np.testing.assert_allclose(d, g["pid_depth"], atol=1e-15)
    sets = [set(np.nonzero(r)[0].tolist()) for r in U]
    a, b, d = O.eid(sets)
    np.testing.assert_allclose(a, g["eid_in_in"], atol=1e-15)
    np.testing.assert_allclose(b, g["eid_in_out"], atol=1e-15)
    np.testing.assert_allclose(d, g["eid_depth"], atol=1e-15)
    assert list(O.rank_by_depth(O.pid(U)[2])) == g["rank"]


# --- binary reduction to eID by set counts (Eq. 5, Sec. 3.3) -------------------------

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_binary_masks_reduce_to_eid(seed):
    rng = np.random.default_rng(seed)
    N, M = 7, 40
    U = (rng.uniform(size=(N, M)) < 0.5).astype(np.float64)
    U[:, 0] = 1.0  # every set non-empty: eID and PID then agree exactly (Eq. 5)
    sets = [set(np.nonzero(r)[0].tolist()) for r in U]
    for got, want in zip(O.pid(U), O.eid(sets)):
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-14)
    # the per-pair operator is |A cap B| / |A| by brute-force counting
    P = O.inclusion_matrix(U)
    for i in range(N):
        for j in range(N):
            assert P[i, j] == pytest.approx(len(sets[i] & sets[j]) / len(sets[i]), abs=1e-15)


def test_thresholded_ellipses_reduce_to_eid():
    Ub = synth.ellipses_2d(N=6, H=48, W=48, binary=True)
    sets = [set(np.nonzero(r)[0].tolist()) for r in Ub]
    assert all(len(s) > 0 for s in sets)
    for got, want in zip(O.pid(Ub), O.eid(sets)):
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


# --- closed forms ----------------------------------------------------------------------

def test_constant_masks_closed_form():
    # u_i = c_i everywhere: u_i subset_p u_j = c_j, so IN_in = mean(c), IN_out(i) = c_i
    c = np.array([0.2, 0.9, 0.5, 0.7, 0.05])
    M = 11
    U = np.repeat(c[:, None], M, axis=1)
    w = np.linspace(0.5, 3.0, M)
    a, b, d = O.pid(U, w)
    np.testing.assert_allclose(a, np.full(5, c.mean()), atol=1e-15)
    np.testing.assert_allclose(b, c, atol=1e-15)
    np.testing.assert_allclose(d, np.minimum(c.mean(), c), atol=1e-15)
    a, b, d = O.pid_mean(U, w)
    np.testing.assert_allclose(a, np.full(5, c.mean()), atol=1e-15)
    np.testing.assert_allclose(b, c, atol=1e-15)


def test_nested_binary_disks_closed_form():
    radii = [4, 7, 10, 13, 16, 20]
    U = synth.nested_disks(radii, 48, 48).astype(np.float64)
    a_area = U.sum(axis=1)
    N = len(radii)
    # members are nested: A_1 subset A_2 subset ... (index k = 0..N-1 here)
    in_in = np.array([((N - k) + sum(a_area[j] / a_area[k] for j in range(k))) / N
                      for k in range(N)])
    in_out = np.array([((k + 1) + sum(a_area[k] / a_area[j] for j in range(k + 1, N))) / N
                       for k in range(N)])
    a, b, d = O.pid(U)
    np.testing.assert_allclose(a, in_in, atol=1e-14)
    np.testing.assert_allclose(b, in_out, atol=1e-14)
    # centre-outward order: depth rises then falls (unimodal)
    peak = int(np.argmax(d))
    assert np.all(np.diff(d[: peak + 1]) > 0) and np.all(np.diff(d[peak:]) < 0)


def test_soft_nested_disks_unimodal():
    radii = [5, 8, 11, 14, 17, 21, 24]
    H = 64
    yy, xx = np.meshgrid(np.arange(H) + 0.5 - H / 2, np.arange(H) + 0.5 - H / 2, indexing="ij")
    dist = np.sqrt(yy ** 2 + xx ** 2).reshape(-1)
    U = np.stack([0.5 * (1 + np.tanh((r - dist) / 1.5)) for r in radii])
    d = O.pid(U)[2]
    peak = int(np.argmax(d))
    assert 0 < peak < len(radii) - 1
    assert np.all(np.diff(d[: peak + 1]) > 0) and np.all(np.diff(d[peak:]) < 0)


def test_identical_members_tie():
    base = synth.random_soft(1, 50, seed=3)[0].astype(np.float64)
    U = np.stack([base, base, base, 0.5 * base + 0.1])
    d = O.pid(U)[2]
    assert d[0] == d[1] == d[2]
    # all-identical: binary masks give depth 1, soft masks give sum w u^2 / sum w u
    ub = (base > 0.5).astype(np.float64)
    assert np.all(O.pid(np.stack([ub] * 5))[2] == 1.0)
    w = np.linspace(1, 2, 50)
    expect = np.sum(w * base * base) / np.sum(w * base)
    np.testing.assert_allclose(O.pid(np.stack([base] * 4), w)[2], expect, atol=1e-15)
    np.testing.assert_allclose(O.pid_mean(np.stack([base] * 4), w)[2], expect, atol=1e-15)


# --- identities and bounds of Sec. 4.1 -------------------------------------------------

@pytest.mark.parametrize("seed", [0, 1])
def test_recall_identity(seed):
    U = synth.random_soft(9, 77, seed=seed, binary_frac=0.3)
    w = np.random.default_rng(seed).uniform(0.1, 5, 77)
    np.testing.assert_allclose(O.pid(U, w)[0], O.pid_mean(U, w)[0], atol=1e-14)


def test_linear_identity_for_in_out():
    # IN_out(i) = (1/N) sum_j G_ij / m_j = sum_x w u_i u_tilde,  u_tilde = (1/N) sum_j u_j / m_j
    U = synth.random_soft(12, 90, seed=5).astype(np.float64)
    w = np.random.default_rng(5).uniform(0.5, 2, 90)
    m = U @ w
    u_tilde = (U / m[:, None]).mean(axis=0)
    np.testing.assert_allclose(O.pid(U, w)[1], (U * w) @ u_tilde, atol=1e-14)


def test_equal_masses_make_pid_and_pid_mean_agree():
    rng = np.random.default_rng(11)
    values = rng.uniform(0, 1, 64)
    U = np.stack([rng.permutation(values) for _ in range(10)])  # equal masses, unit cells
    for a, b in zip(O.pid(U), O.pid_mean(U)):
        np.testing.assert_allclose(a, b, atol=1e-14)


@pytest.mark.parametrize("seed", range(5))
def test_cv_error_bound(seed):
    rng = np.random.default_rng(seed)
    N, M = 15, 60
    U = rng.uniform(0, 1, (N, M)) * rng.uniform(0.05, 1.0, (N, 1))  # varied masses
    w = rng.uniform(0.2, 3, M)
    m = U @ w
    cv = m.std() / m.mean()  # population CV of member masses
    err = np.abs(O.pid(U, w)[2] - O.pid_mean(U, w)[2])
    assert np.all(err <= cv + 1e-12)


# --- invariants of Sec. 3.3 ------------------------------------------------------------

def test_range_zero_one():
    rng = np.random.default_rng(4)
    U = rng.uniform(0, 1, (8, 30))
    U[3] = 0.0
    for arr in (*O.pid(U), *O.pid_mean(U), O.inclusion_matrix(U)):
        # the penalty form 1 - D/m may round a few ulp past the ends
        assert np.all(arr >= -1e-14) and np.all(arr <= 1 + 1e-14)


def test_coordinate_agnostic_permutation_split_scale():
    rng = np.random.default_rng(9)
    N, M = 6, 40
    U = rng.uniform(0, 1, (N, M))
    w = rng.uniform(0.5, 2, M)
    ref = O.pid(U, w)
    perm = rng.permutation(M)
    for a, b in zip(ref, O.pid(U[:, perm], w[perm])):
        np.testing.assert_allclose(a, b, atol=1e-14)
    # split every cell into two copies carrying half the measure each
    for a, b in zip(ref, O.pid(np.repeat(U, 2, axis=1), np.repeat(w / 2, 2))):
        np.testing.assert_allclose(a, b, atol=1e-14)
    for a, b in zip(ref, O.pid(U, 7.5 * w)):
        np.testing.assert_allclose(a, b, atol=1e-14)
    refm = O.pid_mean(U, w)
    for a, b in zip(refm, O.pid_mean(np.repeat(U, 2, axis=1), np.repeat(w / 2, 2))):
        np.testing.assert_allclose(a, b, atol=1e-14)


def test_cell_measure_counts_like_repeated_cells():
    # an integer cell measure k behaves exactly like k unit cells (Sec. 3.4)
    rng = np.random.default_rng(2)
    U = rng.uniform(0, 1, (5, 12))
    k = rng.integers(1, 4, 12)
    for a, b in zip(O.pid(U, k.astype(float)), O.pid(np.repeat(U, k, axis=1))):
        np.testing.assert_allclose(a, b, atol=1e-14)


def test_scale_invariance_first_argument_and_linearity():
    rng = np.random.default_rng(8)
    u, v, v2 = rng.uniform(0, 1, (3, 25))
    w = rng.uniform(0.5, 2, 25)
    assert O.inclusion(0.3 * u, v, w) == pytest.approx(O.inclusion(u, v, w), abs=1e-15)
    lin = O.inclusion(u, 0.25 * v + 0.75 * v2, w)
    assert lin == pytest.approx(0.25 * O.inclusion(u, v, w) + 0.75 * O.inclusion(u, v2, w),
                                abs=1e-15)
    assert O.inclusion(u, np.ones(25), w) == pytest.approx(1.0, abs=1e-15)
    assert O.inclusion(u, np.zeros(25), w) == 0.0
    assert O.inclusion(np.zeros(25), v, w) == 0.0  # zero-mass convention


# --- isovalue map (Sec. 3.5) -------------------------------------------------------------

def test_iso_map_textbook_values():
    mu, sigma = 0.5, 0.05
    # F = mu - k sigma lies inside (F < q) with probability Phi(k)
    F = np.array([mu, mu - sigma, mu - 1.96 * sigma, mu + 2 * sigma])
    u = O.iso_soft_mask(F, mu, sigma)
    np.testing.assert_allclose(u, [0.5, 0.8413447460685429, 0.9750021048517795,
                                   0.022750131948179195], atol=1e-15)
    F = np.linspace(0, 1, 101)
    np.testing.assert_allclose(O.iso_soft_mask(F, mu, sigma), ndtr((mu - F) / sigma), atol=1e-15)
    np.testing.assert_allclose(O.iso_soft_mask(F, mu, sigma, superlevel=True),
                               ndtr((F - mu) / sigma), atol=1e-15)


def test_iso_map_sigma_zero_is_threshold():
    F = np.array([0.1, 0.49, 0.5, 0.51, 0.9])
    np.testing.assert_array_equal(O.iso_soft_mask(F, 0.5, 0.0), [1, 1, 0, 0, 0])
    np.testing.assert_array_equal(O.iso_soft_mask(F, 0.5, 0.0, superlevel=True), [0, 0, 0, 1, 1])
    # a very narrow distribution converges to the threshold masks, so eID applies (Eq. 5)
    F = synth.rbf_fields_2d(N=4, H=32, W=32, n_rbf=4)
    Fd = F.astype(np.float64)
    soft = O.iso_soft_mask(Fd, 0.5, 1e-9)
    hard = O.iso_soft_mask(Fd, 0.5, 0.0)
    near = np.abs(Fd - 0.5) < 1e-7
    assert np.all((soft == hard) | near)


# --- ranking (Sec. 5.1) -------------------------------------------------------------------

def test_rank_matches_sorted_with_ties():
    d = np.array([0.3, 0.7, 0.3, 0.9, 0.7, 0.1])
    order = sorted(range(6), key=lambda i: (-d[i], i))
    r = O.rank_by_depth(d)
    assert [int(np.where(r == k)[0][0]) for k in range(6)] == order
    assert list(r) == [3, 1, 4, 0, 2, 5]


def test_eid_is_strictly_pinned_by_counts():
    A = [{0, 1, 2, 3}, {1, 2}, {2, 3, 4}]
    assert O.eps_subset(A[1], A[0]) == 1.0
    assert O.eps_subset(A[0], A[1]) == 0.5
    assert O.eps_subset(A[2], A[0]) == pytest.approx(2 / 3)
    assert O.eps_subset(set(), A[0]) == 1.0
    a, b, d = O.eid(A)
    assert a[0] == pytest.approx((1 + 0.5 + 0.5) / 3)
    assert b[0] == pytest.approx((1 + 1 + 2 / 3) / 3)


# --- the block-accumulated forms used at full workload sizes --------------------------

def _blocks(U, w, edges):
    return ((U[:, a:b], None if w is None else w[a:b]) for a, b in zip(edges[:-1], edges[1:]))


def test_chunked_forms_match_closed_forms_and_set_counts():
    # nested binary disks: the closed form above, through uneven blocks
    radii = [4, 7, 10, 13, 16, 20]
    U = synth.nested_disks(radii, 48, 48).astype(np.float64)
    a_area = U.sum(axis=1)
    N = len(radii)
    in_in = np.array([((N - k) + sum(a_area[j] / a_area[k] for j in range(k))) / N
                      for k in range(N)])
    in_out = np.array([((k + 1) + sum(a_area[k] / a_area[j] for j in range(k + 1, N))) / N
                       for k in range(N)])
    edges = [0, 1, 700, 701, 1500, 48 * 48]
    a, b, _ = O.pid_chunked(_blocks(U, None, edges))
    np.testing.assert_allclose(a, in_in, atol=1e-14)
    np.testing.assert_allclose(b, in_out, atol=1e-14)
    # binary masks with an empty member: eID by set counts (zero-mass reading: P_i. = 0)
    rng = np.random.default_rng(4)
    Ub = (rng.uniform(0, 1, (6, 300)) < 0.4).astype(np.float64)
    sets = [set(np.nonzero(r)[0].tolist()) for r in Ub]
    a, b, d = O.pid_chunked(_blocks(Ub, None, [0, 77, 78, 300]))
    ea, eb, ed = O.eid(sets)
    np.testing.assert_allclose(a, ea, atol=1e-14)
    np.testing.assert_allclose(b, eb, atol=1e-14)
    # constant masks: PID-mean closed form min(mean c, c_i), weighted, uneven blocks
    c = np.array([0.2, 0.9, 0.5, 0.7, 0.05])
    Uc = np.repeat(c[:, None], 40, axis=1)
    w = np.linspace(0.5, 3.0, 40)
    a, b, d = O.pid_mean_chunked(_blocks(Uc, w, [0, 3, 39, 40]))
    np.testing.assert_allclose(a, np.full(5, c.mean()), atol=1e-15)
    np.testing.assert_allclose(b, c, atol=1e-15)


@pytest.mark.parametrize("seed", [0, 1])
def test_chunked_forms_do_not_depend_on_the_blocks(seed):
    rng = np.random.default_rng(seed)
    U = synth.random_soft(9, 2000, seed=seed, binary_frac=0.3).astype(np.float64)
    U[3] = 0.0                                            # a zero-mass member
    w = rng.uniform(0.1, 5, 2000)
    full = np.array(O.pid(U, w))
    mean = np.array(O.pid_mean(U, w))
    for edges in ([0, 2000], [0, 1, 2, 1999, 2000], list(range(0, 2001, 250))):
        np.testing.assert_allclose(np.array(O.pid_chunked(_blocks(U, w, edges))), full, atol=1e-13)
        np.testing.assert_allclose(np.array(O.pid_mean_chunked(_blocks(U, w, edges))), mean,
                                   atol=1e-13)


# --- contour boxplot bands (Sec. 6) -------------------------------------------------

def test_bands_hand_example():
    g = _load("hand_bands_3x6.json")
    got = O.contour_bands(np.array(g["U"]), np.array(g["rank"]), g["tau"], g["inner_fraction"])
    assert got.tolist() == g["bands"]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bands_nesting_invariants(seed):
    rng = np.random.default_rng(seed)
    N, M = int(rng.integers(1, 12)), 500
    U = synth.random_soft(N, M, seed=seed, binary_frac=0.3).astype(np.float64)
    rank = rng.permutation(N)
    for frac in (0.25, 0.5, 1.0):
        b = O.contour_bands(U, rank, 0.5, frac)
        iu, ii = (b & 1) > 0, (b & 2) > 0
        au, ai = (b & 4) > 0, (b & 8) > 0
        med = (b & 16) > 0
        assert np.all(ii <= iu) and np.all(ai <= ai & iu) and np.all(iu <= au)
        assert np.all(ai <= ii) and np.all(ii <= med) and np.all(med <= iu)
        if frac == 1.0:
            assert np.array_equal(iu, au) and np.array_equal(ii, ai)
    if N == 1:
        b = O.contour_bands(U, rank, 0.5)
        assert np.array_equal(b, (U[0] > 0.5).astype(np.uint8) * 31)


def test_bands_of_nested_disks_are_the_extreme_disks():
    # PID orders nested disks centre-outward; the deepest half is a run of consecutive
    # radii, whose union is its largest disk and whose intersection its smallest
    radii = [3, 5, 7, 9, 11, 13, 15, 17, 19]
    U = synth.nested_disks(radii, 48, 48).astype(np.float64)
    depth = O.pid(U)[2]
    rank = O.rank_by_depth(depth)
    inner = np.nonzero(rank < 5)[0]
    assert np.all(np.diff(inner) == 1)                 # a contiguous run of radii
    b = O.contour_bands(U, rank, 0.5, 0.5)
    assert np.array_equal((b & 1) > 0, U[inner.max()] > 0.5)
    assert np.array_equal((b & 2) > 0, U[inner.min()] > 0.5)
    assert np.array_equal((b & 4) > 0, U[-1] > 0.5)
    assert np.array_equal((b & 8) > 0, U[0] > 0.5)
    assert np.array_equal((b & 16) > 0, U[int(np.argmin(rank))] > 0.5)


# --- other mask models and the weighted mean contour ---------------------------------

def test_uniform_isovalue_mask_closed_form():
    # q ~ U[0.4, 0.6]: P(F < q) is 1 below 0.4, 0 above 0.6, and linear in between
    F = np.array([0.0, 0.4, 0.45, 0.5, 0.55, 0.6, 1.0])
    np.testing.assert_allclose(O.iso_soft_mask_uniform(F, 0.5, 0.1),
                               [1.0, 1.0, 0.75, 0.5, 0.25, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(O.iso_soft_mask_uniform(F, 0.5, 0.1, superlevel=True),
                               [0.0, 0.0, 0.25, 0.5, 0.75, 1.0, 1.0], atol=1e-15)
    # the mean of the uniform mask over a linear ramp equals the normal one's by symmetry
    F = np.linspace(0, 1, 100001)
    assert abs(O.iso_soft_mask_uniform(F, 0.5, 0.2).mean() - O.iso_soft_mask(F, 0.5, 0.1).mean()) < 1e-4


def test_level_mask_closed_form():
    F = np.array([0.2, 0.35, 0.5, 0.6, 0.7, 0.9])
    np.testing.assert_allclose(O.level_soft_mask(F, 0.5, 0.2), [0.0, 0.25, 1.0, 0.5, 0.0, 0.0],
                               atol=1e-15)


def test_weighted_mean_contour_special_cases():
    rng = np.random.default_rng(8)
    U = synth.random_soft(6, 400, seed=8).astype(np.float64)
    w = rng.uniform(0.5, 2, 400)
    # equal reliabilities: plain PID-mean
    np.testing.assert_allclose(np.array(O.pid_mean_weighted(U, np.full(6, 3.0), w)),
                               np.array(O.pid_mean(U, w)), atol=1e-14)
    # all reliability on member k: u_bar = u_k, the pairwise inclusions of Eq. 9
    k = 2
    r = np.zeros(6)
    r[k] = 1.0
    a, b, _ = O.pid_mean_weighted(U, r, w)
    np.testing.assert_allclose(a, [O.inclusion(U[i], U[k], w) for i in range(6)], atol=1e-14)
    np.testing.assert_allclose(b, [O.inclusion(U[k], U[i], w) for i in range(6)], atol=1e-14)


# --- 4D space-time PID: time as one more cell axis -------------------------------------

def test_spacetime_binary_members_are_eid_over_space_time_cells():
    # binary members over 2 steps x 5 cells; the sets of (x, t) cells are built by hand
    rng = np.random.default_rng(12)
    steps = [(rng.uniform(size=(4, 5)) < 0.6).astype(np.float64) for _ in range(2)]
    sets = [{(x, t) for t in range(2) for x in range(5) if steps[t][i, x] == 1.0}
            for i in range(4)]
    assert all(sets)
    U, w = O.spacetime_cells(steps)
    a, b, d = O.pid(U, w)
    ea, eb, ed = O.eid(sets)
    np.testing.assert_allclose(np.c_[a, b, d], np.c_[ea, eb, ed], atol=1e-14)


def test_spacetime_invariants():
    rng = np.random.default_rng(13)
    S = [synth.random_soft(7, 300, seed=20 + t).astype(np.float64) for t in range(3)]
    w = rng.uniform(0.5, 2.0, 300)
    base = np.array(O.pid(*O.spacetime_cells(S, w)))
    # one step: the plain ensemble
    U1, w1 = O.spacetime_cells(S[:1], w)
    np.testing.assert_allclose(np.array(O.pid(U1, w1)), np.array(O.pid(S[0], w)), atol=1e-14)
    # the order of the time steps does not matter
    np.testing.assert_allclose(np.array(O.pid(*O.spacetime_cells(S[::-1], w))), base, atol=1e-13)
    # T identical steps: every sum scales by T, the depths of one step remain
    np.testing.assert_allclose(np.array(O.pid_mean(*O.spacetime_cells([S[1]] * 4, w))),
                               np.array(O.pid_mean(S[1], w)), atol=1e-13)
    # a step whose members are all empty adds nothing
    Z = np.zeros_like(S[0])
    np.testing.assert_allclose(np.array(O.pid(*O.spacetime_cells(S + [Z], w))), base, atol=1e-13)


# --- PID within groups of members (multimodal ensembles) -------------------------------

def test_grouped_pid_special_cases():
    U = synth.random_soft(9, 200, seed=31).astype(np.float64)
    a, b, d = O.pid(U)
    # one group: plain PID, ranks of Sec. 5.1
    ga, gb, gd, gr = O.pid_grouped(U, np.zeros(9, dtype=int))
    np.testing.assert_allclose(np.c_[ga, gb, gd], np.c_[a, b, d], atol=1e-15)
    assert list(gr) == list(O.rank_by_depth(d))
    # singletons: a member against itself only, u subset_p u = sum u^2 / sum u (Eq. 9)
    sa, sb, sd, sr = O.pid_grouped(U, np.arange(9))
    self_inc = (U * U).sum(axis=1) / U.sum(axis=1)
    np.testing.assert_allclose(sd, self_inc, rtol=1e-14)
    assert np.all(sr == 0)
    B = (U > 0.5).astype(np.float64)       # binary members: fully included in themselves
    assert np.all(O.pid_grouped(B, np.arange(9))[2] == 1.0)
    # label values do not matter, only which members share one
    lab = np.array([3, 3, 7, 7, 7, 3, -1, -1, 7])
    ref = O.pid_grouped(U, lab)
    for x, y in zip(ref, O.pid_grouped(U, np.where(lab == 3, 100, np.where(lab == 7, 5, 0)))):
        np.testing.assert_array_equal(x, y)


def test_grouped_pid_of_two_disk_families_is_each_familys_order():
    # two families of nested binary disks far apart; within a family the inclusion of disk
    # i in disk j is |D_i & D_j| / |D_i| = min(|D_i|, |D_j|) / |D_i| from pixel counts, and
    # the other family never enters
    yy, xx = np.mgrid[0:64, 0:128]
    masks, labels = [], []
    for fam, cx in ((0, 32), (1, 96)):
        for r in (6, 10, 14, 18, 22):
            masks.append(((xx - cx) ** 2 + (yy - 32) ** 2 <= r * r).astype(np.float64).ravel())
            labels.append(fam)
    U = np.array(masks)
    a, b, d, r = O.pid_grouped(U, np.array(labels))
    for fam in (0, 1):
        idx = np.arange(5) + 5 * fam
        area = U[idx].sum(axis=1)
        want_in = np.array([np.mean([min(ai, aj) / ai for aj in area]) for ai in area])
        want_out = np.array([np.mean([min(ai, aj) / aj for aj in area]) for ai in area])
        np.testing.assert_allclose(a[idx], want_in, rtol=1e-14)
        np.testing.assert_allclose(b[idx], want_out, rtol=1e-14)
        assert r[idx[2]] == 0 and sorted(r[idx]) == [0, 1, 2, 3, 4]
