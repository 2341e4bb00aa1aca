"""Parity at the full sizes of the benchmark workloads, through pid_batch (the launch the
benchmark times), element by element against the FP64 oracle:

  2D ellipses     20 x 128^2, soft and binary: PID-mean, exact full PID, the three Gram
                  precisions with the inclusion matrix; binary masks against eID counts
  2D fields       64 x 512^2, isovalue ~ Normal(0.5, 0.05): PID-mean, exact full PID and
                  the BF16 Gram, batched with three more ensembles of the same workload
  non-Cartesian   128 x 2^20 points with lumped-area weights: PID-mean, exact full PID and
                  the split-BF16 / E4M3 Gram
  3D plume        one time step, 200 x 256^3 (13.4 GB): PID-mean, exact full PID and the
                  E4M3 / split-BF16 Gram, the oracle accumulated over blocks of 2^20 cells;
                  two time steps batched against single calls, bitwise
"""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import (FP32_TOL, GRAM_TOL, assert_close, assert_rank_agrees_outside_ties,
                           assert_rank_valid, to_np)

pytestmark = pytest.mark.gpu
PRECS = ["bf16", "split_bf16", "fp8"]


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


def _check(o, ref, tol, what, P_ref=None, p_tol=None):
    a, b, d = ref
    assert_close(to_np(o["in_in"]), a, FP32_TOL if tol > FP32_TOL else tol, what + " in_in")
    assert_close(to_np(o["in_out"]), b, tol, what + " in_out")
    assert_close(to_np(o["depth"]), d, tol, what + " depth")
    assert_rank_valid(to_np(o["rank"]), to_np(o["depth"]))
    assert_rank_agrees_outside_ties(to_np(o["rank"]), d, tol)
    if P_ref is not None and "P" in o:
        assert_close(to_np(o["P"]), P_ref, p_tol or tol, what + " P")


def _cv_bound_holds(o_full, o_mean, mass):
    # |PID - PID-mean| <= CV_pop(m) (the bound derived from Eq. 16 and 0 <= G_ij/m_j <= 1)
    m = np.asarray(mass, dtype=np.float64)
    cv = m.std() / m.mean()
    gap = np.abs(to_np(o_full["depth"]) - to_np(o_mean["depth"]))
    assert gap.max() <= cv + 1e-9, (gap.max(), cv)


def test_ellipses_20x128x128(H):
    U = synth.ellipses_2d()
    Ub = synth.ellipses_2d(binary=True)
    items = [dict(data=_dev(U), mode="mean"), dict(data=_dev(U), mode="linear")]
    items += [dict(data=_dev(U), mode="full", precision=p, want_P=True) for p in PRECS]
    items += [dict(data=_dev(Ub), mode="linear")]
    items += [dict(data=_dev(Ub), mode="full", precision=p) for p in PRECS]
    outs = H.batch(items)
    H.sync()
    ref_mean, ref_full, P = O.pid_mean(U), O.pid(U), O.inclusion_matrix(U)
    _check(outs[0], ref_mean, FP32_TOL, "ellipses mean")
    _check(outs[1], ref_full, FP32_TOL, "ellipses linear")
    for o, p in zip(outs[2:5], PRECS):
        _check(o, ref_full, GRAM_TOL, f"ellipses {p}", P, GRAM_TOL)
    sets = [set(np.nonzero(r)[0].tolist()) for r in Ub]
    ref_eid = O.eid(sets)
    for o in outs[5:]:
        _check(o, ref_eid, 1e-7, "binary ellipses vs eID")
    _cv_bound_holds(outs[1], outs[0], to_np(outs[0]["mass"]))


def test_fields_64x512x512(H):
    import torch
    F = torch.empty((4, 64, 512 * 512), device="cuda")
    for e in range(4):
        synth.rbf_fields_2d_torch(64, 512, 512, 32, seed=synth.DEFAULT_SEED + 2 + 7919 * e,
                                  device="cuda", out=F[e])
    iso = (0.5, 0.05, 0)
    items = [dict(data=F[0], iso=iso, mode="mean"), dict(data=F[0], iso=iso, mode="linear"),
             dict(data=F[0], iso=iso, mode="full", precision="bf16", want_P=True)]
    items += [dict(data=F[e], iso=iso, mode="linear") for e in (1, 2, 3)]
    outs = H.batch(items)
    H.sync()
    U = O.iso_soft_mask(to_np(F[0]), 0.5, 0.05)
    _check(outs[0], O.pid_mean(U), FP32_TOL, "fields mean")
    ref_full = O.pid(U)
    _check(outs[1], ref_full, FP32_TOL, "fields linear")
    _check(outs[2], ref_full, GRAM_TOL, "fields bf16", O.inclusion_matrix(U))
    _cv_bound_holds(outs[1], outs[0], to_np(outs[0]["mass"]))
    # a batched neighbour of the same workload, against the oracle too
    U3 = O.iso_soft_mask(to_np(F[3]), 0.5, 0.05)
    _check(outs[5], O.pid(U3), FP32_TOL, "fields linear (4th ensemble)")


def test_noncartesian_128x1M_weighted(H):
    U, w = synth.radial_disk(N=128, M=1 << 20)
    Ud, wd = _dev(U), _dev(w)
    items = [dict(data=Ud, w=wd, mode="mean"), dict(data=Ud, w=wd, mode="linear"),
             dict(data=Ud, w=wd, mode="full", precision="split_bf16"),
             dict(data=Ud, w=wd, mode="full", precision="fp8")]
    outs = H.batch(items)
    H.sync()
    ref_mean, ref_full = O.pid_mean(U, w), O.pid(U, w)
    _check(outs[0], ref_mean, FP32_TOL, "disk mean")
    _check(outs[1], ref_full, FP32_TOL, "disk linear")
    _check(outs[2], ref_full, GRAM_TOL, "disk split_bf16")
    _check(outs[3], ref_full, GRAM_TOL, "disk fp8")
    _cv_bound_holds(outs[1], outs[0], to_np(outs[0]["mass"]))


def _host_blocks(Ud, block=1 << 20):
    M = Ud.shape[1]
    for x0 in range(0, M, block):
        yield to_np(Ud[:, x0:x0 + block]), None


def test_plume_one_step_200x256cubed(H):
    import torch
    U = synth.plume_3d(200, 256, t=8)                    # [200, 256^3] on the device
    items = [dict(data=U, mode="mean"), dict(data=U, mode="linear"),
             dict(data=U, mode="full", precision="fp8"),
             dict(data=U, mode="full", precision="split_bf16")]
    outs = H.batch(items)
    H.sync()
    ref_full = O.pid_chunked(_host_blocks(U))
    _check(outs[0], O.pid_mean_chunked(_host_blocks(U)), FP32_TOL, "plume mean")
    _check(outs[1], ref_full, FP32_TOL, "plume linear")
    _check(outs[2], ref_full, GRAM_TOL, "plume fp8")
    _check(outs[3], ref_full, GRAM_TOL, "plume split_bf16")
    _cv_bound_holds(outs[1], outs[0], to_np(outs[0]["mass"]))
    del U
    torch.cuda.empty_cache()


def test_plume_time_steps_batched_equal_single_calls(H):
    import torch
    steps = [synth.plume_3d(200, 256, t=t) for t in (3, 12)]
    outs = H.batch([dict(data=U, mode=m) for U in steps for m in ("mean", "linear")])
    H.sync()
    for k, U in enumerate(steps):
        single_mean = H.mean(U)
        single_full = H.full(U, mode="linear")
        H.sync()
        for f in ("depth", "in_in", "in_out", "rank"):
            assert torch.equal(outs[2 * k][f], single_mean[f]), f"step {k} mean {f}"
            assert torch.equal(outs[2 * k + 1][f], single_full[f]), f"step {k} linear {f}"
    del steps
    torch.cuda.empty_cache()
