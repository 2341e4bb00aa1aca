"""GPU parity of the streaming path (PID-mean, exact full PID, isovalue map) vs the oracle.

Every call goes through the C ABI (ctypes binding). Sizes span several tiles and
chunks with ragged tails; N covers every tile class of the streaming kernel.
"""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import (FP32_TOL, ISO_TOL, assert_close, assert_rank_agrees_outside_ties,
                           assert_rank_valid, to_np)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import torch  # noqa: F401
    from paper_2512_15187_gb300 import build, binding
    build.build()
    h = binding.Handle(0)
    yield h
    h.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(o, ref, tol=FP32_TOL, what=""):
    a, b, d = ref
    assert_close(to_np(o["in_in"]), a, tol, what + " in_in")
    assert_close(to_np(o["in_out"]), b, tol, what + " in_out")
    assert_close(to_np(o["depth"]), d, tol, what + " depth")
    assert_rank_valid(to_np(o["rank"]), to_np(o["depth"]))
    assert_rank_agrees_outside_ties(to_np(o["rank"]), d, tol)


# every tile class (members <= 8, 16, 24, 32, 48, 64, 96, 128, 192, 208, 256, 320, 384, 448,
# 512), filled and partly filled, with ragged cell counts
SHAPES = [(1, 1), (1, 300), (2, 7), (3, 129), (7, 1000), (8, 4099), (9, 513), (16, 2000),
          (17, 3001), (24, 2500), (31, 777), (33, 5000), (48, 3000), (64, 4097), (65, 2049),
          (96, 1000), (128, 1025), (129, 999), (192, 800), (193, 777), (200, 1500), (208, 1001),
          (256, 640), (257, 333),
          (350, 300), (384, 257), (420, 260), (448, 130), (500, 450), (512, 257)]


@pytest.mark.parametrize("N,M", SHAPES)
@pytest.mark.parametrize("weighted", [False, True])
def test_pid_mean_parity(H, N, M, weighted):
    U = synth.random_soft(N, M, seed=N * 7919 + M, binary_frac=0.2)
    w = np.random.default_rng(M).uniform(0.1, 10, M).astype(np.float32) if weighted else None
    H.sync()
    o = H.mean(_dev(U), None if w is None else _dev(w))
    H.sync()
    _check(o, O.pid_mean(U, w), what=f"mean N={N} M={M}")


@pytest.mark.parametrize("N,M", [(1, 50), (2, 7), (5, 1000), (20, 16384), (33, 5000), (64, 4097),
                                 (90, 700), (129, 999), (257, 333), (350, 300), (420, 260),
                                 (500, 450)])
@pytest.mark.parametrize("weighted", [False, True])
def test_full_linear_parity(H, N, M, weighted):
    U = synth.random_soft(N, M, seed=N * 31 + M, binary_frac=0.3)
    w = np.random.default_rng(M + 1).uniform(0.1, 10, M).astype(np.float32) if weighted else None
    o = H.full(_dev(U), None if w is None else _dev(w), mode="linear")
    H.sync()
    _check(o, O.pid(U, w), what=f"full-linear N={N} M={M}")


def test_unaligned_stride_uses_generic_loads(H):
    import torch
    N, M = 37, 1001
    U = synth.random_soft(N, M, seed=5)
    big = torch.zeros((N, M + 3), dtype=torch.float32, device="cuda")
    big[:, :M] = _dev(U)
    view = big[:, :M]                      # ld = M + 3 (not a multiple of 4 floats)
    _check(H.mean(view), O.pid_mean(U), what="mean ld=M+3")
    _check(H.full(view, mode="linear"), O.pid(U), what="full ld=M+3")
    H.sync()
    off = torch.zeros(N * M + 1, dtype=torch.float32, device="cuda")
    off[1:] = _dev(U).reshape(-1)
    view2 = off[1:].view(N, M)            # base not 16-byte aligned
    _check(H.mean(view2), O.pid_mean(U), what="mean misaligned base")
    H.sync()


@pytest.mark.parametrize("N", [37, 200, 300, 500])      # one, two and one cell per lane classes
@pytest.mark.parametrize("boff,pad", [(1, 1), (2, 2), (3, 5)])
def test_unaligned_spans_every_class(H, N, boff, pad):
    """Rows staged as 16-byte-aligned spans: a base `boff` floats past an aligned address
    (row 0's first span would start before the data), row strides of M + pad floats (every
    row at another offset in its span), a ragged last stage, cell measures, PID-mean and
    the exact full PID (which also streams the rows a second time)."""
    import torch
    M = 1003
    U = synth.random_soft(N, M, seed=N + 17 * boff, binary_frac=0.2)
    w = np.random.default_rng(N + boff).uniform(0.1, 10, M).astype(np.float32)
    ld = M + pad
    buf = torch.zeros(boff + N * ld, dtype=torch.float32, device="cuda")
    view = buf[boff:].view(N, ld)[:, :M]
    view.copy_(_dev(U))
    _check(H.mean(view, _dev(w)), O.pid_mean(U, w), what=f"mean N={N} boff={boff} ld=M+{pad}")
    _check(H.full(view, mode="linear"), O.pid(U), what=f"linear N={N} boff={boff} ld=M+{pad}")
    H.sync()


@pytest.mark.parametrize("N", [3, 4, 13, 37, 200, 300, 500])
@pytest.mark.parametrize("boff,pad", [(0, 0), (0, 1), (1, 3), (2, 2), (3, 1)])
def test_unaligned_rows_match_aligned_rows_bitwise(H, N, boff, pad):
    """Rows that are not 16-byte aligned are staged by TMA through residue-class tensor maps
    (odd ld: four classes of members i mod 4; ld = 2 mod 4: two; a base alone off the
    16-byte boundary: one), or by cp.async spans where a class map does not apply (fewer
    members than classes, a warp whose members straddle classes, cell measures off the
    boundary). Either way each row's cells reach the same arithmetic: PID-mean and the
    exact full PID equal, bit for bit, those of an aligned copy of the ensemble."""
    import torch
    M = 1001
    ld = M + pad                       # 1001, 1002, 1004, 1003, 1002
    U = synth.random_soft(N, M, seed=N * 7 + pad, binary_frac=0.2)
    w = np.random.default_rng(N + pad).uniform(0.1, 10, M).astype(np.float32)
    buf = torch.zeros(boff + N * ld, dtype=torch.float32, device="cuda")
    view = buf[boff:].view(N, ld)[:, :M]
    view.copy_(_dev(U))
    ref_buf = torch.zeros((N, (M + 3) // 4 * 4), dtype=torch.float32, device="cuda")
    ref_view = ref_buf[:, :M]
    ref_view.copy_(_dev(U))
    wd = _dev(w)
    wbuf = torch.zeros(M + 1, dtype=torch.float32, device="cuda")
    w_off = wbuf[1:]                   # cell measures 4 bytes past the boundary
    w_off.copy_(wd)
    for got_w, what in ((wd, "measures aligned"), (w_off, "measures unaligned"), (None, "unit measures")):
        ref_w = None if got_w is None else wd
        a = H.mean(view, got_w)
        b = H.mean(ref_view, ref_w)
        c = H.full(view, got_w, mode="linear")
        d = H.full(ref_view, ref_w, mode="linear")
        H.sync()
        for x, y, mode in ((a, b, "mean"), (c, d, "linear")):
            for k in ("in_in", "in_out", "depth", "rank"):
                assert torch.equal(x[k], y[k]), (N, boff, pad, what, mode, k)
    _check(a, O.pid_mean(U), what=f"mean N={N} boff={boff} ld={ld}")


def test_zero_mass_and_binary_members(H):
    N, M = 6, 900
    U = synth.random_soft(N, M, seed=2)
    U[2] = 0.0                             # zero-mass member: inclusions with it as reference = 0
    U[4] = (U[4] > 0.5)
    for o, ref in ((H.mean(_dev(U)), O.pid_mean(U)), (H.full(_dev(U)), O.pid(U))):
        H.sync()
        _check(o, ref, what="zero-mass")


def test_binary_ellipses_match_eid(H):
    Ub = synth.ellipses_2d(N=20, binary=True)
    sets = [set(np.nonzero(r)[0].tolist()) for r in Ub]
    o = H.full(_dev(Ub), mode="linear")
    H.sync()
    _check(o, O.eid(sets), what="binary ellipses vs eID")


def test_identical_members_bitwise_tie(H):
    base = synth.random_soft(1, 5000, seed=9)[0]
    U = np.stack([base, base, base, base * 0.5, base])
    for o in (H.mean(_dev(U)), H.full(_dev(U))):
        H.sync()
        d = to_np(o["depth"])
        assert d[0] == d[1] == d[2] == d[4]


def test_all_identical_binary_depth_one(H):
    ub = (synth.random_soft(1, 3000, seed=4)[0] > 0.3).astype(np.float32)
    o = H.full(_dev(np.stack([ub] * 9)))
    H.sync()
    assert np.all(np.abs(to_np(o["depth"]) - 1.0) <= 1e-7)


# ---- isovalue map -----------------------------------------------------------------------

@pytest.mark.parametrize("sigma,superlevel", [(0.05, False), (0.05, True), (0.0, False), (0.0, True)])
def test_soft_masks_parity(H, sigma, superlevel):
    F = synth.rbf_fields_2d(N=5, H=96, W=80, n_rbf=6)
    out = H.soft_masks(_dev(F), 0.5, sigma, superlevel)
    H.sync()
    ref = O.iso_soft_mask(F, 0.5, sigma, superlevel)
    assert_close(to_np(out), ref, ISO_TOL, "iso map")


def test_soft_masks_threshold_not_float_representable(H):
    F = np.array([[0.1, 0.3, np.nextafter(np.float32(0.3), np.float32(1)), 0.31]], np.float32)
    for sup in (False, True):
        out = H.soft_masks(_dev(F), 0.3, 0.0, sup)
        H.sync()
        np.testing.assert_array_equal(to_np(out), O.iso_soft_mask(F, 0.3, 0.0, sup))


@pytest.mark.parametrize("mode", ["mean", "linear"])
@pytest.mark.parametrize("superlevel", [False, True])
@pytest.mark.parametrize("N,H_,W_", [(9, 64, 70), (64, 128, 128), (130, 40, 50)])
def test_from_fields_parity(H, mode, superlevel, N, H_, W_):
    F = synth.rbf_fields_2d(N=N, H=H_, W=W_, n_rbf=8)
    # centre every member on its median so that both level sets of mu = 0.01 are non-empty
    F = (F - np.median(F, axis=1, keepdims=True)).astype(np.float32)
    mu = 0.01
    w = np.random.default_rng(N).uniform(0.5, 2, H_ * W_).astype(np.float32)
    U = O.iso_soft_mask(F, mu, 0.05, superlevel)
    # precondition of the FP32 guarantee: every mask reaches well inside FP32's normal range
    assert np.all(U.max(axis=1) > 1e-20)
    o = H.from_fields(_dev(F), mu, 0.05, superlevel=superlevel, w=_dev(w), mode=mode)
    H.sync()
    ref = O.pid_mean(U, w) if mode == "mean" else O.pid(U, w)
    _check(o, ref, what=f"fields {mode}")


def test_vanishing_member_outside_fp32_range(H):
    # Member 3's field lies more than 1 above mu everywhere: with sigma = 0.05 its mask is
    # about 1e-88 in every cell. The fused path evaluates u in FP32, where that is exactly 0,
    # so the member has zero mass and falls under the zero-mass convention (Sec. 3.2). The
    # reference is the oracle applied to the masks rounded to FP32.
    N, H_, W_ = 12, 48, 48
    F = synth.rbf_fields_2d(N=N, H=H_, W=W_, n_rbf=4)
    mu = float(np.median(F))
    F[3] = mu + 1.0 + np.abs(F[3])
    U32 = O.iso_soft_mask(F, mu, 0.05).astype(np.float32)
    assert U32[3].max() == 0.0
    for mode, ref in (("mean", O.pid_mean(U32)), ("linear", O.pid(U32))):
        o = H.from_fields(_dev(F), mu, 0.05, mode=mode)
        H.sync()
        _check(o, ref, what=f"vanishing member {mode}")
        assert to_np(o["in_in"])[3] == 0.0


# ---- validation and argument errors -------------------------------------------------------

def test_validate_flags_out_of_range(H):
    from paper_2512_15187_gb300 import binding as B
    U = synth.random_soft(4, 500, seed=1)
    U[1, 17] = 1.5
    H.full(_dev(U), mode="linear", validate=True)
    with pytest.raises(B.PidError) as e:
        H.sync()
    assert e.value.status == B.PID_ERR_DOMAIN
    U[1, 17] = 0.5
    H.full(_dev(U), mode="linear", validate=True)
    H.sync()  # clean again


def test_invalid_arguments(H):
    import torch
    from paper_2512_15187_gb300 import binding as B
    U = torch.rand((4, 100), device="cuda")
    d = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PidError) as e:
        B.pid_mean(H.h, U.data_ptr(), 4, 100, 99, None, d.data_ptr(), None, None, None)
    assert e.value.status == B.PID_ERR_INVALID_ARG
    with pytest.raises(B.PidError) as e:
        B.pid_mean(H.h, U.data_ptr(), 0, 100, 100, None, d.data_ptr(), None, None, None)
    assert e.value.status == B.PID_ERR_INVALID_ARG
    big = torch.zeros(((1 << 22) + 1, 8), device="cuda")     # above the member limit
    with pytest.raises(B.PidError) as e:
        H.mean(big)
    assert e.value.status == B.PID_ERR_UNSUPPORTED


def test_autotuned_launch_is_bitwise_identical(H):
    from paper_2512_15187_gb300 import binding
    U = _dev(synth.random_soft(100, 70000, seed=77))     # G = 16 class: both exchange schemes
    ref = H.mean(U)
    H.sync()
    h2 = binding.Handle(0)
    n0 = h2.autotune(True)
    tuned = h2.mean(U)
    h2.sync()
    assert h2.autotune(False) >= n0 + 1
    again = h2.mean(U)
    h2.sync()
    for k in ("in_in", "in_out", "depth", "rank"):
        assert np.array_equal(to_np(ref[k]), to_np(tuned[k]))
        assert np.array_equal(to_np(ref[k]), to_np(again[k]))
    h2.close()
