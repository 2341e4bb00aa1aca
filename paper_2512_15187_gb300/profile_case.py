"""Run one small, fixed case of one path of the library, for a profiler to capture.

    python -m paper_2512_15187_gb300.profile_case fields        # isovalue map + PID-mean
    python -m paper_2512_15187_gb300.profile_case fields-full   # isovalue map + exact full PID
    python -m paper_2512_15187_gb300.profile_case mean          # PID-mean of soft masks
    python -m paper_2512_15187_gb300.profile_case linear        # exact full PID, O(N M)
    python -m paper_2512_15187_gb300.profile_case gram --precision bf16 --ensembles 4
    python -m paper_2512_15187_gb300.profile_case plume --side 128   # one 3D plume step:
        # PID-mean, E4M3 Gram and split-BF16 Gram of 200 members on side^3 cells, one batch
    python -m paper_2512_15187_gb300.profile_case bands --members 64 --cells 4194304
        # contour boxplot bands of 64 fields on 2048^2 cells

Each case builds its inputs on the device (seeded), makes one call (planning, tuning and
graph capture), then `--repeat` timed calls, and prints the best call time (CUDA events,
host work included) and each kernel's time per launch from the library's own profiler.
Sizes default to N = 64 members and M = 2^20 cells (256 MiB of FP32 masks, larger than
the 129 MB L2, so DRAM counters stay meaningful); `--max-gb` bounds the input.
"""
from __future__ import annotations

import argparse


def main(argv=None) -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["fields", "fields-full", "mean", "linear", "gram", "plume",
                                     "bands"])
    ap.add_argument("--side", type=int, default=128, help="plume: cells per axis")
    ap.add_argument("--members", type=int, default=64)
    ap.add_argument("--cells", type=int, default=1 << 20)
    ap.add_argument("--ensembles", type=int, default=1,
                    help="ensembles per call (more than one goes through pid_batch)")
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "split_bf16", "fp8"])
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default tiles (no timing of candidate tiles on the first call)")
    ap.add_argument("--max-gb", type=float, default=4.0,
                    help="refuse inputs above this size (profilers save and restore memory)")
    a = ap.parse_args(argv)

    import torch

    from . import binding, build, synth
    build.build()
    N, M, E = a.members, a.cells, a.ensembles
    if a.case == "plume":
        N, M, E = 200, a.side ** 3, 1
    if 4.0 * N * M * E > a.max_gb * 1e9:
        raise SystemExit(f"input above --max-gb {a.max_gb}")
    h = binding.Handle(0)
    if a.no_autotune:
        h.autotune(False)
    if a.case == "plume":
        U = synth.plume_3d(N, a.side, t=8, T=16)
        items = [dict(data=U, mode="mean"), dict(data=U, mode="full", precision="fp8"),
                 dict(data=U, mode="full", precision="split_bf16")]
        _run(h, items, a, f"plume N={N} M={M} (mean, fp8, split_bf16)")
        return
    if a.case == "bands":
        _run_bands(h, N, M, a)
        return
    X = torch.empty((E, N, M), device="cuda")
    side = int(round(M ** 0.5))
    for e in range(E):
        if a.case in ("fields", "fields-full", "gram") and side * side == M:
            synth.rbf_fields_2d_torch(N, side, side, 32, seed=7 + e, device="cuda", out=X[e])
        else:
            g = torch.Generator(device="cuda").manual_seed(7 + e)
            X[e].uniform_(0.0, 1.0, generator=g)
    is_field = a.case in ("fields", "fields-full", "gram") and side * side == M
    mode = {"fields": "mean", "fields-full": "linear", "mean": "mean", "linear": "linear",
            "gram": "full"}[a.case]
    prec = a.precision if mode == "full" else "fp32"
    items = [dict(data=X[e], iso=(0.5, 0.05, 0) if is_field else None, mode=mode, precision=prec)
             for e in range(E)]
    _run(h, items, a, f"{a.case} {mode} {prec} N={N} M={M} E={E}")


def _run_bands(h, N, M, a) -> None:
    """Contour boxplot bands of one ensemble of N fields on M = side^2 cells (Sec. 6), from
    the ranks of its exact full PID: one bands launch per call."""
    import torch
    from . import synth
    side = int(round(M ** 0.5))
    F = torch.empty((N, side * side), device="cuda")
    synth.rbf_fields_2d_torch(N, side, side, 32, seed=7, device="cuda", out=F)
    iso = (0.5, 0.05, 0)
    rank = h.from_fields(F, *iso[:2], mode="linear")["rank"]
    out = h.contour_bands(F, rank, 0.5, 0.5, iso=iso)
    h.sync()
    h.profile(True)
    ms = []
    for _ in range(a.repeat):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        h.contour_bands(F, rank, 0.5, 0.5, iso=iso, out=out)
        t1.record()
        t1.synchronize()
        ms.append(t0.elapsed_time(t1))
    h.sync()
    st = h.profile_read()["bands"]
    h.profile(False)
    per = st["total_ms"] / st["launches"]
    print("ok bands", f"N={N} M={side * side}", int(out.sum()), f"call best {min(ms):.3f} ms")
    print(f"  bands     {st['launches']:4d} launches  {per:8.3f} ms/launch  "
          f"{st['bytes'] / st['launches'] / per / 1e6:8.1f} GB/s algorithmic")
    h.close()


def _run(h, items, a, label) -> None:
    import torch
    outs = h.batch(items)          # first call: plans, tunes and records the graph
    h.sync()
    h.profile(True)
    ms = []
    for _ in range(a.repeat):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        outs = h.batch(items)
        t1.record()
        t1.synchronize()
        ms.append(t0.elapsed_time(t1))
    h.sync()
    prof = h.profile_read()
    h.profile(False)
    print("ok", label, float(outs[0]["depth"].sum()), f"call best {min(ms):.3f} ms")
    for kind, st in prof.items():
        if st["launches"]:
            per = st["total_ms"] / st["launches"]
            print(f"  {kind:9s} {st['launches']:4d} launches  {per:8.3f} ms/launch  "
                  f"{st['bytes'] / st['launches'] / per / 1e6:8.1f} GB/s algorithmic")
    h.close()


if __name__ == "__main__":
    main()
