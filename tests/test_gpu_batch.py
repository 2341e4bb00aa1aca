"""GPU tests of pid_batch: uneven ensembles in one persistent launch per tile class.

Each ensemble's results must be bitwise identical to the single-ensemble call (same tile
class, same chunking, same reduction order) and match the FP64 oracle; a replayed graph
must pick up new data written in place.
"""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import FP32_TOL, assert_close, assert_rank_valid, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    from paper_2512_15187_gb300 import build, binding
    build.build()
    h = binding.Handle(0)
    yield h
    h.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _mixed_batch(seed=0, n=14):
    rng = np.random.default_rng(seed)
    items, refs = [], []
    Ns = [1, 5, 8, 13, 20, 33, 64, 70, 128, 150, 256, 300, 500, 3][:n]
    for k, N in enumerate(Ns):
        M = int(rng.integers(50, 6000))
        weighted = bool(k % 3 == 1)
        field = bool(k % 4 in (2, 3))   # fields in both modes (linear stores the masks)
        mode = ["mean", "linear"][k % 2]
        w = rng.uniform(0.2, 4, M).astype(np.float32) if weighted else None
        if field:
            F = (rng.normal(0, 1, (N, M))).astype(np.float32)
            U = O.iso_soft_mask(F, 0.1, 0.5)
            data = F
            iso = (0.1, 0.5, 0)
        else:
            U = synth.random_soft(N, M, seed=seed * 100 + k, binary_frac=0.2)
            data = U
            iso = None
        items.append(dict(data=_dev(data), w=None if w is None else _dev(w), iso=iso, mode=mode))
        refs.append((U, w, mode))
    return items, refs


def test_batch_matches_oracle_and_single_calls_bitwise(H):
    items, refs = _mixed_batch()
    outs = H.batch(items)
    H.sync()
    for it, o, (U, w, mode) in zip(items, outs, refs):
        ref = O.pid_mean(U, w) if mode == "mean" else O.pid(U, w)
        for k, r in zip(("in_in", "in_out", "depth"), ref):
            assert_close(to_np(o[k]), r, FP32_TOL, f"batch N={U.shape[0]} {mode} {k}")
        assert_rank_valid(to_np(o["rank"]), to_np(o["depth"]))
        # PID-mean depth and masses are by-products of every mode
        assert_close(to_np(o["mean_depth"]), O.pid_mean(U, w)[2], FP32_TOL, "mean_depth")
        assert_close(to_np(o["mass"]) / max(1.0, float(O.mass(U, w).max())),
                     O.mass(U, w) / max(1.0, float(O.mass(U, w).max())), 1e-6, "mass")
        if it["iso"] is None:
            single = H.mean(it["data"], it["w"]) if mode == "mean" else \
                H.full(it["data"], it["w"], mode="linear")
        else:
            mu, sg, sup = it["iso"]
            single = H.from_fields(it["data"], mu, sg, superlevel=bool(sup), w=it["w"], mode=mode)
        H.sync()
        for k in ("in_in", "in_out", "depth", "rank"):
            assert np.array_equal(to_np(o[k]), to_np(single[k])), f"batch != single for {k}"


def test_batch_graph_replay_sees_new_data(H):
    import torch
    from paper_2512_15187_gb300 import binding as B
    rng = np.random.default_rng(3)
    datas, ws, modes, outs, ens = [], [], [], [], []
    for k, N in enumerate([4, 20, 70, 200, 9]):
        M = int(rng.integers(300, 3000))
        U = _dev(synth.random_soft(N, M, seed=40 + k))
        w = _dev(rng.uniform(0.5, 2, M).astype(np.float32)) if k % 2 else None
        mode = "linear" if k % 2 == 0 else "mean"
        o = H._outputs(N, extras=True)
        e = B.pid_ensemble()
        e.data, e.N, e.M, e.ld = U.data_ptr(), N, M, U.stride(0)
        e.w = None if w is None else w.data_ptr()
        e.opt = B.pid_options(B.MODES[mode], 0, 0, 0)
        for key in ("depth", "in_in", "in_out", "rank", "mass", "mean_depth"):
            setattr(e, key, o[key].data_ptr())
        datas.append(U); ws.append(w); modes.append(mode); outs.append(o); ens.append(e)
    stream = B.c_void_p(torch.cuda.current_stream().cuda_stream)
    for rep in range(4):
        if rep >= 2:  # same layout, new contents: the replayed graph must read them
            for U in datas:
                U.copy_(torch.flip(U, dims=[1]) * 0.9)
        B.pid_batch(H.h, ens, stream)
        H.sync()
        for U, w, mode, o in zip(datas, ws, modes, outs):
            Un = to_np(U)
            wn = None if w is None else to_np(w)
            ref = O.pid_mean(Un, wn) if mode == "mean" else O.pid(Un, wn)
            assert_close(to_np(o["depth"]), ref[2], FP32_TOL, f"replay {rep} {mode}")


def test_batch_of_many_uneven_ensembles(H):
    rng = np.random.default_rng(7)
    items, refs = [], []
    for k in range(48):
        N = int(rng.integers(10, 501))
        M = int(np.exp(rng.uniform(np.log(64 * 64), np.log(24 * 24 * 24))))
        U = synth.random_soft(N, M, seed=k)
        items.append(dict(data=_dev(U), mode="mean"))
        refs.append(U)
    outs = H.batch(items)
    H.sync()
    for o, U in zip(outs, refs):
        assert_close(to_np(o["depth"]), O.pid_mean(U)[2], FP32_TOL, "48-ensemble batch")


def test_empty_batch_and_bad_entries(H):
    from paper_2512_15187_gb300 import binding as B
    B.pid_batch(H.h, [], None)
    U = _dev(synth.random_soft(4, 100, seed=1))
    with pytest.raises(B.PidError) as e:
        H.batch([dict(data=U, mode="mean"), dict(data=U[:, :0], mode="mean")])
    assert e.value.status == B.PID_ERR_INVALID_ARG


def test_profiled_graph_replays_time_every_launch(H):
    """With profiling on, the batch is recorded with timing nodes around every kernel and
    replayed as a graph: every replay's launches are counted and timed, and the results
    are bitwise those of the unprofiled graph."""
    import torch
    from paper_2512_15187_gb300 import binding
    h = binding.Handle(0)
    U = [torch.rand((64, 40000 + 4 * k), device="cuda") for k in range(3)]
    items = [dict(data=X, mode="mean") for X in U]       # one streaming class: 1 launch
    items += [dict(data=U[0], mode="full", precision="fp8")]   # scale pass + E4M3 Gram
    ref = h.batch(items)
    h.sync()
    h.profile(True)
    outs = h.batch(items)                                  # records the profiled graph
    for _ in range(3):
        h.batch(items, outs=outs)                          # replays
    h.sync()
    prof = h.profile_read()
    h.profile(False)
    assert prof["stream"]["launches"] == 4, prof["stream"]
    assert prof["gram_fp8"]["launches"] == 4, prof["gram_fp8"]
    assert prof["scale"]["launches"] == 4, prof["scale"]
    assert prof["finalize"]["launches"] == 4, prof["finalize"]
    for k in ("stream", "gram_fp8", "scale", "finalize"):
        assert prof[k]["total_ms"] > 0.0, (k, prof[k])
    assert prof["stream"]["bytes"] == 4 * 4.0 * sum(X.numel() for X in U)
    for a, b in zip(ref, outs):
        for k in ("depth", "in_in", "in_out", "rank"):
            assert torch.equal(a[k], b[k]), k
    h.close()


def test_pid_mean_shares_the_exact_items_first_pass():
    """A PID-mean item and an exact full-PID item over the same data run one first pass
    between them (both sum m_i and A_i, Eq. 6, 16, 17): every result stays bitwise that of
    its single call, and the streaming kernels read such an ensemble twice (pass 1 and
    pass 2), not three times. A PID-mean item under another isovalue map runs its own pass."""
    import torch
    from paper_2512_15187_gb300 import binding
    h = binding.Handle(0)
    g = torch.Generator(device="cuda").manual_seed(7)
    items, expect = [], 0.0
    # 16-byte aligned rows, rows that are not (odd M), weighted cells
    for N, M, weighted in [(64, 40000, False), (37, 9001, True), (200, 30003, False)]:
        U = torch.rand((N, M), generator=g, device="cuda")
        w = torch.rand(M, generator=g, device="cuda") + 0.5 if weighted else None
        items += [dict(data=U, w=w, mode="mean"), dict(data=U, w=w, mode="linear")]
        expect += 2 * (4.0 * N * M + (4.0 * M if weighted else 0.0))
    F = torch.randn((20, 5000), generator=g, device="cuda")
    items += [dict(data=F, iso=(0.1, 0.5, 0), mode="mean"),
              dict(data=F, iso=(0.1, 0.5, 0), mode="linear"),
              dict(data=F, iso=(0.2, 0.5, 0), mode="mean")]
    expect += 3 * 4.0 * F.numel()
    h.profile(True)
    outs = h.batch(items)
    h.sync()
    prof = h.profile_read()
    h.profile(False)
    assert prof["stream"]["bytes"] == expect, (prof["stream"]["bytes"], expect)
    for it, o in zip(items, outs):
        if it.get("iso") is None:
            single = h.mean(it["data"], it["w"]) if it["mode"] == "mean" else \
                h.full(it["data"], it["w"], mode="linear")
        else:
            mu, sg, sup = it["iso"]
            single = h.from_fields(it["data"], mu, sg, superlevel=bool(sup), mode=it["mode"])
        h.sync()
        for k in ("in_in", "in_out", "depth", "rank"):
            assert torch.equal(o[k], single[k]), (it["mode"], tuple(it["data"].shape), k)
    h.close()
