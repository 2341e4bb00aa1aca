"""GPU parity of the other mask models with the FP64 oracle: the isovalue uniform on
[mu - h, mu + h] (Sec. 3.5 with another isovalue distribution, both level sets), the
level-centred map of the weather example (Sec. 3.6), and PID-mean against a
reliability-weighted mean contour (Sec. 4.1). Soft masks, every depth path (PID-mean,
exact linear full PID, tensor-core Gram, the member-blocked path beyond 512 members,
batches), contour bands bit for bit, and the host and device checks of the new inputs."""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import (FP32_TOL, GRAM_TOL, assert_close, assert_rank_agrees_outside_ties,
                           assert_rank_valid, to_np)

pytestmark = pytest.mark.gpu

MU, HW = 0.5, 0.1
KINDS = [("uniform", 0), ("uniform", 1), ("level", 0)]
# FP32 map vs FP64: mu' = mu +- h and 1/(2h) (or 1/h) are rounded once to float
# (|d mu'| inv <= 0.6 * 2^-24 * 10 < 4e-7 for the level map's inv = 10, 1.8e-7 for the
# uniform map's inv = 5), plus one rounding of the product (< 6e-8).
MAP_TOL = 5e-7


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


def _fields(N, Hh, W, seed=0):
    F = synth.rbf_fields_2d(N=N, H=Hh, W=W, n_rbf=8, seed=synth.DEFAULT_SEED + 40 + seed)
    return (F - np.median(F, axis=1, keepdims=True) + MU).astype(np.float32)


def _masks(F, kind, sup, mu=MU, h=HW):
    if kind == "uniform":
        return O.iso_soft_mask_uniform(F, mu, h, bool(sup))
    return O.level_soft_mask(F, mu, h)


@pytest.mark.parametrize("kind,sup", KINDS)
@pytest.mark.parametrize("N,Hh,W", [(1, 9, 7), (5, 40, 25), (33, 96, 75)])
def test_soft_masks(H, kind, sup, N, Hh, W):
    F = _fields(N, Hh, W)
    got = to_np(H.soft_masks(_dev(F), MU, HW, sup, kind=kind))
    assert_close(got, _masks(F, kind, sup), MAP_TOL, f"{kind} soft masks")
    assert got.min() >= 0.0 and got.max() <= 1.0


@pytest.mark.parametrize("kind,sup", KINDS)
@pytest.mark.parametrize("N,Hh,W,mode", [(24, 64, 80, "mean"), (24, 64, 80, "linear"),
                                         (7, 33, 31, "linear"), (130, 48, 50, "mean"),
                                         (300, 40, 41, "linear")])
def test_depths_from_fields(H, kind, sup, N, Hh, W, mode):
    F = _fields(N, Hh, W, seed=N)
    U = _masks(F, kind, sup)
    o = H.from_fields(_dev(F), MU, HW, sup, mode=mode, kind=kind)
    ref = O.pid_mean(U) if mode == "mean" else O.pid(U)
    for k, r in zip(("in_in", "in_out", "depth"), ref):
        assert_close(to_np(o[k]), r, FP32_TOL, f"{kind} {mode} N={N} {k}")
    assert_rank_valid(to_np(o["rank"]), to_np(o["depth"]))


@pytest.mark.parametrize("kind,sup", KINDS)
@pytest.mark.parametrize("N,precision", [(64, "bf16"), (200, "bf16"), (24, "fp8")])
def test_gram_from_fields(H, kind, sup, N, precision):
    F = _fields(N, 64, 72, seed=N + 1)
    U = _masks(F, kind, sup)
    o = H.from_fields(_dev(F), MU, HW, sup, mode="full", precision=precision, kind=kind)
    ref = O.pid(U)
    for k, r in zip(("in_in", "in_out", "depth"), ref):
        assert_close(to_np(o[k]), r, GRAM_TOL, f"{kind} gram {precision} N={N} {k}")
    assert_rank_agrees_outside_ties(to_np(o["rank"]), ref[2], GRAM_TOL)


def test_blocked_path_level_map(H):
    F = _fields(700, 30, 70, seed=3)
    U = _masks(F, "level", 0)
    for mode, ref in (("mean", O.pid_mean(U)), ("linear", O.pid(U))):
        o = H.from_fields(_dev(F), MU, HW, mode=mode, kind="level")
        for k, r in zip(("in_in", "in_out", "depth"), ref):
            assert_close(to_np(o[k]), r, FP32_TOL, f"blocked {mode} {k}")
        assert_rank_valid(to_np(o["rank"]), to_np(o["depth"]))


def test_batch_mixes_kinds(H):
    items, refs = [], []
    for k, (kind, sup) in enumerate(KINDS + [("normal", 0), ("normal", 1)]):
        F = _fields(9 + 10 * k, 30 + k, 41, seed=k)
        mode = ["mean", "linear"][k % 2]
        items.append(dict(data=_dev(F), iso=(MU, HW, sup, kind), mode=mode))
        U = _masks(F, kind, sup) if kind != "normal" else O.iso_soft_mask(F, MU, HW, bool(sup))
        refs.append((U, mode))
    outs = H.batch(items)
    H.sync()
    for o, (U, mode) in zip(outs, refs):
        ref = O.pid_mean(U) if mode == "mean" else O.pid(U)
        for k, r in zip(("in_in", "in_out", "depth"), ref):
            assert_close(to_np(o[k]), r, FP32_TOL, f"batch {mode} {k}")


@pytest.mark.parametrize("kind,sup", KINDS)
@pytest.mark.parametrize("tau", [0.5, 0.02, 0.9])
def test_bands(H, kind, sup, tau):
    import torch
    F = _fields(33, 96, 75, seed=5)
    perm = np.random.default_rng(4).permutation(33).astype(np.int32)
    got = to_np(H.contour_bands(_dev(F), torch.from_numpy(perm).cuda(), tau, 0.5,
                                iso=(MU, HW, sup, kind)))
    assert np.array_equal(got, O.contour_bands(_masks(F, kind, sup), perm, tau, 0.5))


def test_bands_at_exact_thresholds(H):
    """Field values where u = tau exactly (all of mu, h, tau and the thresholds are binary
    fractions, so the FP64 oracle meets them exactly) are not above tau; their float
    neighbours fall on either side."""
    import torch
    mu, h, tau = 0.5, 0.125, 0.75
    # uniform below: u = tau at 0.4375; uniform above: at 0.5625; level: at 0.46875, 0.53125
    edges = np.array([0.4375, 0.5625, 0.46875, 0.53125], np.float32)
    cols = np.concatenate([edges, np.nextafter(edges, np.float32(-1)),
                           np.nextafter(edges, np.float32(2)), [mu, 0.0, 1.0]]).astype(np.float32)
    F = np.tile(cols, (3, 1))
    r = torch.arange(3, dtype=torch.int32, device="cuda")
    for kind, sup in KINDS:
        got = to_np(H.contour_bands(_dev(F), r, tau, 1.0, iso=(mu, h, sup, kind)))
        U = _masks(F, kind, sup, mu, h)
        assert np.any(U == tau)
        want = O.contour_bands(U, np.arange(3), tau, 1.0)
        assert np.array_equal(got, want), (kind, sup, got, want)


def test_host_checks(H):
    from paper_2512_15187_gb300 import binding as B
    F = _dev(_fields(4, 10, 10))
    with pytest.raises(B.PidError):
        H.soft_masks(F, MU, 0.0, kind="uniform")        # a uniform map needs h > 0
    with pytest.raises(B.PidError):
        H.soft_masks(F, MU, HW, 1, kind="level")        # no super-level form
    with pytest.raises(B.PidError):
        H.soft_masks(F, MU, 1e-300, kind="level")       # 1/h beyond the float range
    with pytest.raises(KeyError):
        H.soft_masks(F, MU, HW, kind="triangle")


# --------------------------------------------------------------------------------------
# Reliability-weighted mean contour (Sec. 4.1)
# --------------------------------------------------------------------------------------

def _weights(N, seed, zeros=True):
    r = np.random.default_rng(seed).uniform(0.0, 3.0, N)
    if zeros and N > 3:
        r[::4] = 0.0
    return r


@pytest.mark.parametrize("N,M,cellw", [(1, 100, False), (40, 5000, False), (40, 5000, True),
                                       (257, 3001, True), (600, 2100, False),
                                       (1100, 1500, True)])
def test_weighted_mean_soft_masks(H, N, M, cellw):
    import torch
    U = synth.random_soft(N, M, seed=N + 7, binary_frac=0.2)
    w = np.random.default_rng(M).uniform(0.2, 4.0, M).astype(np.float32) if cellw else None
    r = _weights(N, N)
    if not r.sum() > 0:
        r[0] = 1.0
    o = H.mean_weighted(_dev(U), torch.from_numpy(r).cuda(), w=None if w is None else _dev(w))
    ref = O.pid_mean_weighted(U, r, w)
    for k, v in zip(("in_in", "in_out", "depth"), ref):
        assert_close(to_np(o[k]), v, FP32_TOL, f"weighted N={N} {k}")
    assert_rank_valid(to_np(o["rank"]), to_np(o["depth"]))


@pytest.mark.parametrize("kind,sup", KINDS + [("normal", 0)])
def test_weighted_mean_fields(H, kind, sup):
    import torch
    F = _fields(30, 50, 60, seed=9)
    U = _masks(F, kind, sup) if kind != "normal" else O.iso_soft_mask(F, MU, HW, False)
    r = _weights(30, 2)
    o = H.mean_weighted(_dev(F), torch.from_numpy(r).cuda(), iso=(MU, HW, sup, kind))
    ref = O.pid_mean_weighted(U, r)
    for k, v in zip(("in_in", "in_out", "depth"), ref):
        assert_close(to_np(o[k]), v, FP32_TOL, f"weighted {kind} {k}")


def test_equal_weights_give_pid_mean(H):
    import torch
    U = synth.random_soft(50, 4000, seed=3)
    o = H.mean_weighted(_dev(U), torch.full((50,), 2.5, dtype=torch.float64, device="cuda"))
    ref = O.pid_mean(U)
    for k, v in zip(("in_in", "in_out", "depth"), ref):
        assert_close(to_np(o[k]), v, FP32_TOL, f"equal weights {k}")


def test_invalid_member_weights_report_a_domain_error(H):
    import torch
    from paper_2512_15187_gb300 import binding as B
    U = _dev(synth.random_soft(20, 500, seed=1))
    for bad in (np.r_[np.ones(19), -1.0], np.zeros(20), np.r_[np.ones(19), np.nan]):
        o = H.mean_weighted(U, torch.from_numpy(bad).cuda())
        with pytest.raises(B.PidError) as e:
            H.sync()
        assert e.value.status == B.PID_ERR_DOMAIN
        assert np.all(to_np(o["depth"]) == 0.0)
    H.sync()                                   # the word was cleared; the handle still works
    o = H.mean_weighted(U, torch.ones(20, dtype=torch.float64, device="cuda"))
    H.sync()
    assert_close(to_np(o["depth"]), O.pid_mean(to_np(U))[2], FP32_TOL, "after the error")
    with pytest.raises(ValueError):
        H.mean_weighted(U, torch.ones(19, dtype=torch.float64, device="cuda"))


# --------------------------------------------------------------------------------------
# bfloat16 output of the isovalue map
# --------------------------------------------------------------------------------------

@pytest.mark.parametrize("kind,sup,sigma", [("normal", 0, 0.05), ("normal", 1, 0.05),
                                            ("normal", 0, 0.0), ("uniform", 1, HW),
                                            ("level", 0, HW)])
@pytest.mark.parametrize("N,Hh,W", [(3, 17, 11), (12, 64, 80)])
def test_soft_masks_bf16(H, kind, sup, sigma, N, Hh, W):
    import torch
    F = _fields(N, Hh, W, seed=11)
    Fd = _dev(F)
    a = H.soft_masks(Fd, MU, sigma, sup, kind=kind)
    b = H.soft_masks(Fd, MU, sigma, sup, kind=kind, dtype=torch.bfloat16)
    H.sync()
    assert b.dtype == torch.bfloat16
    # the float32 masks rounded to nearest even, element for element
    assert torch.equal(b, a.to(torch.bfloat16))
    if kind == "normal":
        ref = O.iso_soft_mask(F, MU, sigma, bool(sup))
    else:
        ref = _masks(F, kind, sup)
    # bfloat16 keeps 8 significant bits (7 stored): half an ulp is at most 2^-8 of the value
    err = np.abs(b.float().cpu().numpy() - ref)
    assert np.all(err <= np.abs(ref) * 2.0 ** -8 + 1e-6)
