"""GPU parity of full PID on tensor cores (BF16, split BF16, E4M3 Gram) vs the FP64 oracle.

Bar: depths, IN_in, IN_out and the inclusion matrix within 1e-3 absolute, the same ranking
outside ties, for every precision; split BF16 much tighter; binary masks exact (integer
counts in FP32). A PID_FP8 request below 4096 cells, or asking for P, computes its Gram
from BF16 operands (pid_gram_operands says which); the E4M3 operand path itself is checked
on requests that use it, including members whose values are all small (per-member scales).
"""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import (FP32_TOL, GRAM_TOL, assert_close, assert_rank_agrees_outside_ties,
                           assert_rank_valid, to_np)

pytestmark = pytest.mark.gpu
PRECS = ["bf16", "split_bf16", "fp8"]
# Raw (pre-calibration) Gram error err_est = max_i |mean_j G'_ij / m_i - A_i / m_i| that each
# operand precision reaches, before the calibration fixes the row sums: BF16 within the
# 1e-3 bar, split BF16 within 2e-5; E4M3's per-element rounding (up to 2^-4 of a value)
# does not average over j for member i's own values, so its raw error falls as ~0.1/sqrt(M)
# (measured 1.1e-3 to 1.4e-3 at 4000 to 9000 weighted cells) and meets the bar from about
# 2^14 cells on.
def raw_err_bound(ops, M):
    return {"bf16": 1e-3, "split_bf16": 2e-5}.get(ops) or max(1e-3, 0.15 / np.sqrt(M))


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


def _operands(prec, M, want_P):
    from paper_2512_15187_gb300 import binding as B
    return {B.PID_BF16: "bf16", B.PID_SPLIT_BF16: "split_bf16", B.PID_FP8: "fp8"}[
        B.pid_gram_operands(prec, M, want_P)]


def _check(o, U, w, tol, what, raw_bound=None):
    a, b, d = O.pid(U, w)
    # IN_in comes from the exact FP32 arithmetic of the same pass (Eq. 17)
    assert_close(to_np(o["in_in"]), a, FP32_TOL, what + " in_in")
    assert_close(to_np(o["in_out"]), b, tol, what + " in_out")
    assert_close(to_np(o["depth"]), d, tol, what + " depth")
    assert_rank_valid(to_np(o["rank"]), to_np(o["depth"]))
    assert_rank_agrees_outside_ties(to_np(o["rank"]), d, tol)
    if "err_est" in o:
        # err_est: the raw Gram's |mean_j G'_ij / m_i - A_i / m_i| before calibration
        err = float(to_np(o["err_est"])[0])
        assert 0.0 <= err <= (raw_bound if raw_bound is not None else tol), (what, err)
    if "P" in o:
        assert_close(to_np(o["P"]), O.inclusion_matrix(U, w), tol, what + " P")
        # the calibrated inclusion matrix reproduces the exact IN_in row means
        assert_close(to_np(o["P"]).mean(axis=1), a, 1e-6, what + " P row means")


def test_gram_first_small_case(H):
    U = synth.ellipses_2d(N=20, H=64, W=64)
    o = H.full(_dev(U), mode="full", precision="bf16", want_P=True)
    H.sync()
    _check(o, U, None, GRAM_TOL, "bf16 N=20")


@pytest.mark.parametrize("prec", PRECS)
# every tile: 48 rows (N <= 48), 64, 96 (64 < N <= 96), 128, and the wide 192- and 256-row
# tiles
@pytest.mark.parametrize("N,M", [(1, 64), (2, 1000), (16, 4097), (33, 3000), (48, 5000),
                                 (49, 3001), (64, 65543), (65, 4100), (96, 6000), (100, 5000),
                                 (128, 20000), (129, 777), (192, 5003), (193, 2000),
                                 (200, 20011), (256, 9000)])
@pytest.mark.parametrize("weighted", [False, True])
def test_gram_parity(H, prec, N, M, weighted):
    U = synth.random_soft(N, M, seed=N * 131 + M, binary_frac=0.2)
    w = np.random.default_rng(M).uniform(0.2, 5, M).astype(np.float32) if weighted else None
    o = H.full(_dev(U), None if w is None else _dev(w), mode="full", precision=prec, want_P=True)
    H.sync()
    # asking for P: an E4M3 request computes from BF16 operands, every precision meets 1e-3
    ops = _operands(prec, M, True)
    assert ops == ("bf16" if prec == "fp8" else prec)
    _check(o, U, w, GRAM_TOL, f"{prec} N={N} M={M} w={weighted}", raw_err_bound(ops, M))


# E4M3 operands proper: no P, at least 4096 cells; every tile (48, 64, 96, 128, 192, 256
# rows) and the row-block-tiled Gram above 256 members
@pytest.mark.parametrize("N,M", [(16, 4097), (48, 5000), (64, 65543), (65, 4100), (96, 6000),
                                 (128, 20000), (192, 5003), (200, 20011), (256, 9000),
                                 (300, 8191), (512, 4096)])
@pytest.mark.parametrize("weighted", [False, True])
def test_e4m3_operands_parity(H, N, M, weighted):
    U = synth.random_soft(N, M, seed=N * 7 + M, binary_frac=0.2)
    w = np.random.default_rng(M + 1).uniform(0.2, 5, M).astype(np.float32) if weighted else None
    assert _operands("fp8", M, False) == "fp8"
    o = H.full(_dev(U), None if w is None else _dev(w), mode="full", precision="fp8",
               want_err=True)
    H.sync()
    _check(o, U, w, GRAM_TOL, f"e4m3 N={N} M={M} w={weighted}", raw_err_bound("fp8", M))


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("N,small", [(24, 1e-4), (200, 1e-4), (64, 3e-7), (300, 1e-4)])
def test_e4m3_member_with_small_values(H, N, small, weighted):
    """A member whose values are all below `small` (its largest u is `small`): with one
    scale for the whole ensemble its E4M3 operands would be subnormal or zero; its own
    power-of-two scale keeps 3 significant bits, and its inclusions G_ij / m_i (Eq. 9 is
    invariant to its scale) stay within the bar."""
    M = 30011
    U = synth.random_soft(N, M, seed=N + 5, binary_frac=0.1)
    U[3] *= np.float32(small)
    U[N - 1] = np.float32(small) * synth.random_soft(1, M, seed=99)[0]
    w = np.random.default_rng(7).uniform(0.2, 5, M).astype(np.float32) if weighted else None
    for prec in ("fp8", "bf16"):
        o = H.full(_dev(U), None if w is None else _dev(w), mode="full", precision=prec,
                   want_err=True)
        H.sync()
        _check(o, U, w, GRAM_TOL, f"{prec} small member {small} N={N} w={weighted}",
               raw_err_bound(prec, M))


def test_raw_gram_error_per_precision(H):
    """The raw tensor-core Gram (before the calibration that fixes its row sums) is itself
    within the bar: err_est per precision on one fields ensemble."""
    F = synth.rbf_fields_2d(N=64, H=256, W=256, n_rbf=16)
    F = (F - np.median(F, axis=1, keepdims=True)).astype(np.float32)
    Ud = H.soft_masks(_dev(F), 0.0, 0.05)
    U = to_np(Ud)
    errs = {}
    for prec in PRECS:
        o = H.full(Ud, mode="full", precision=prec, want_err=True)
        H.sync()
        errs[prec] = float(to_np(o["err_est"])[0])
        _check(o, U, None, GRAM_TOL, f"raw {prec}", raw_err_bound(prec, U.shape[1]))
    print("raw Gram err_est per precision:", errs)
    assert errs["split_bf16"] < errs["bf16"]


def test_split_bf16_is_much_tighter(H):
    U = synth.radial_disk(N=64, M=1 << 16)[0]
    ref = O.pid(U)
    errs = {}
    for prec in PRECS:
        o = H.full(_dev(U), mode="full", precision=prec)
        H.sync()
        errs[prec] = float(np.max(np.abs(to_np(o["depth"]) - ref[2])))
    assert errs["split_bf16"] <= 2e-5, errs
    assert errs["bf16"] <= GRAM_TOL and errs["fp8"] <= GRAM_TOL, errs


@pytest.mark.parametrize("N,weighted", [(150, False), (200, True), (208, False), (256, True)])
def test_split_bf16_wide_tile_is_much_tighter(H, N, weighted):
    """The wide tile (128 < N <= 256: two row blocks, the second against the columns from
    128 on, mirrored by the drain) keeps split BF16's accuracy: depths, IN_out, P and the
    raw Gram within 2e-5, with and without cell measures, on TMA and cp.async rows."""
    M = 30011 if weighted else 30016   # rows staged by cp.async, and by TMA
    U = synth.random_soft(N, M, seed=N + 17, binary_frac=0.1)
    w = np.random.default_rng(N).uniform(0.2, 5, M).astype(np.float32) if weighted else None
    o = H.full(_dev(U), None if w is None else _dev(w), mode="full", precision="split_bf16",
               want_P=True, want_err=True)
    H.sync()
    _check(o, U, w, 2e-5, f"split wide N={N} w={weighted}", raw_bound=2e-5)


@pytest.mark.parametrize("prec", PRECS)
def test_gram_binary_masks_are_exact(H, prec):
    # {0,1} operands are exact in BF16 and E4M3 and the Gram sums are integer counts; what
    # remains is the FP32 rounding of the exact mean-contour arithmetic (about 1e-8)
    Ub = synth.ellipses_2d(N=20, binary=True)
    sets = [set(np.nonzero(r)[0].tolist()) for r in Ub]
    o = H.full(_dev(Ub), mode="full", precision=prec, want_P=True)
    H.sync()
    for k, r in zip(("in_in", "in_out", "depth"), O.eid(sets)):
        assert_close(to_np(o[k]), r, 1e-7, f"{prec} binary {k}")
    assert float(to_np(o["err_est"])[0]) <= 1e-7


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("superlevel", [False, True])
@pytest.mark.parametrize("N", [64, 200])
def test_gram_from_fields(H, prec, superlevel, N):
    F = synth.rbf_fields_2d(N=N, H=128, W=96, n_rbf=8)
    F = (F - np.median(F, axis=1, keepdims=True)).astype(np.float32)
    w = np.random.default_rng(3).uniform(0.5, 2, F.shape[1]).astype(np.float32)
    o = H.from_fields(_dev(F), 0.01, 0.05, superlevel=superlevel, w=_dev(w), mode="full",
                      precision=prec)
    H.sync()
    _check(o, O.iso_soft_mask(F, 0.01, 0.05, superlevel), w, GRAM_TOL, f"fields {prec}")


def test_gram_in_batch_with_exact_mean(H):
    rng = np.random.default_rng(5)
    items, refs = [], []
    for k, prec in enumerate(["bf16", "split_bf16", "fp8", "bf16", "fp8"]):
        N = int(rng.integers(3, 257))
        M = int(rng.integers(500, 20000))
        U = synth.random_soft(N, M, seed=900 + k)
        w = rng.uniform(0.5, 3, M).astype(np.float32) if k % 2 else None
        items.append(dict(data=_dev(U), w=None if w is None else _dev(w), mode="full",
                          precision=prec, want_P=True))
        refs.append((U, w, prec))
    outs = H.batch(items)
    H.sync()
    for o, (U, w, prec) in zip(outs, refs):
        _check(o, U, w, GRAM_TOL, f"batch {prec}",
               raw_err_bound(_operands(prec, U.shape[1], True), U.shape[1]))
        assert_close(to_np(o["mean_depth"]), O.pid_mean(U, w)[2], FP32_TOL, "exact PID-mean by-product")


def test_gram_rejects_too_many_members(H):
    import torch
    from paper_2512_15187_gb300 import binding as B
    U = torch.rand((513, 256), device="cuda")
    with pytest.raises(B.PidError) as e:
        H.full(U, mode="full", precision="bf16")
    assert e.value.status == B.PID_ERR_UNSUPPORTED


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [24, 150])
def test_gram_unaligned_rows_read_directly(H, prec, N):
    import torch
    M = 9001
    U = synth.random_soft(N, M, seed=11)
    big = torch.zeros((N, M + 3), dtype=torch.float32, device="cuda")
    big[:, :M] = _dev(U)
    for want_P in (True, False):   # E4M3 operands when P is not asked for
        o = H.full(big[:, :M], mode="full", precision=prec, want_P=want_P, want_err=True)  # ld = M + 3
        H.sync()
        _check(o, U, None, GRAM_TOL, f"{prec} ld=M+3 P={want_P}",
               raw_err_bound(_operands(prec, M, want_P), M))


@pytest.mark.parametrize("N", [96, 200, 300])
@pytest.mark.parametrize("weighted", [False, True])
def test_e4m3_scales_from_the_streaming_pass_in_a_batch(H, N, weighted):
    """In a batch that also runs PID-mean of the same soft masks, the E4M3 Gram takes its
    per-member scales from that streaming pass (no pass of its own); the maxima are those
    of the same operands, so the results are bitwise those of a single E4M3 call."""
    import torch
    M = 50021
    U = _dev(synth.random_soft(N, M, seed=N + 77, binary_frac=0.1))
    U[5] *= 1e-4
    w = _dev(np.random.default_rng(2).uniform(0.3, 3, M).astype(np.float32)) if weighted else None
    H.profile(True)
    outs = H.batch([dict(data=U, w=w, mode="mean"), dict(data=U, w=w, mode="full", precision="fp8")])
    H.sync()
    prof = H.profile_read()
    H.profile(False)
    # only the scale finalisation ran (N keys read), no read of the ensemble for its maxima
    assert prof["scale"]["launches"] == 1 and prof["scale"]["bytes"] == 4.0 * N, prof["scale"]
    single = H.full(U, w, mode="full", precision="fp8")
    H.sync()
    for k in ("depth", "in_in", "in_out", "rank"):
        assert torch.equal(outs[1][k], single[k]), k
    Un = to_np(U)
    _check(outs[1], Un, None if w is None else to_np(w), GRAM_TOL, f"batch e4m3 N={N}")


@pytest.mark.parametrize("N", [40, 130, 256])
def test_gram_takes_exact_sums_from_a_sibling_pass(H, N):
    """Gram items of a batch that also runs PID-mean of the same soft masks take the exact
    (m, A) partials from that streaming pass and skip them in the Gram pass: the results stay
    within the bar, and IN_in equals the sibling PID-mean's IN_in (recall identity, Eq. 17)."""
    M = 30011
    Un = synth.random_soft(N, M, seed=N + 3, binary_frac=0.2)
    U = _dev(Un)
    items = [dict(data=U, mode="mean")]
    items += [dict(data=U, mode="full", precision=p) for p in PRECS]
    outs = H.batch(items)
    H.sync()
    ref_mean = O.pid_mean(Un)
    assert_close(to_np(outs[0]["depth"]), ref_mean[2], FP32_TOL, "sibling PID-mean")
    for o, p in zip(outs[1:], PRECS):
        _check(o, Un, None, GRAM_TOL, f"lean {p} N={N}")
        assert_close(to_np(o["in_in"]), to_np(outs[0]["in_in"]), 1e-12, f"lean {p} IN_in")
        single = H.full(U, mode="full", precision=p)
        H.sync()
        assert_close(to_np(o["depth"]), to_np(single["depth"]), 2e-6 if p == "split_bf16" else 2e-4,
                     f"lean {p} vs single call")
