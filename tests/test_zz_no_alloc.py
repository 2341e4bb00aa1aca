"""pid_mean_noalloc: PID-mean for callers that cannot allocate device memory.

Real-time loops in which a cudaMalloc would synchronise the device, and host applications
whose own allocator owns all device memory, cannot let the library allocate workspace.
pid_mean_noalloc keeps its scratch in a fixed array inside the library instead; it must
return bit for bit what pid_mean returns, call after call (the scratch keeps the previous
call's partial sums, so a leak of them into the next call would show as a changed bit).
"""
import pytest


pytestmark = pytest.mark.gpu


def _noalloc(U, w):
    import torch
    from paper_2512_15187_gb300 import binding as B
    N, M = U.shape
    dev = U.device
    out = {k: torch.empty(N, dtype=torch.float64, device=dev) for k in ("depth", "in_in", "in_out")}
    out["rank"] = torch.empty(N, dtype=torch.int32, device=dev)
    status = torch.full((1,), 0xFFFF, dtype=torch.int32, device=dev)
    B.pid_mean_noalloc(U.data_ptr(), N, M, U.stride(0), None if w is None else w.data_ptr(),
                       out["depth"].data_ptr(), out["in_in"].data_ptr(), out["in_out"].data_ptr(),
                       out["rank"].data_ptr(), status.data_ptr(),
                       B.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return out


@pytest.mark.parametrize("N,M,weighted", [(64, 50000, False), (20, 16384, True), (200, 9001, True)])
def test_noalloc_matches_pid_mean_on_two_calls(N, M, weighted):
    import torch
    from paper_2512_15187_gb300 import binding, build
    build.build()
    g = torch.Generator(device="cuda").manual_seed(N * 1000 + M)
    U = torch.rand((N, M), generator=g, device="cuda")
    w = torch.rand(M, generator=g, device="cuda") + 0.5 if weighted else None
    h = binding.Handle(0)
    ref = h.mean(U, w)
    h.sync()
    for _ in range(2):   # the shared scratch keeps the previous call's contents
        got = _noalloc(U, w)
        for k in ("in_in", "in_out", "depth", "rank"):
            assert torch.equal(got[k], ref[k]), f"noalloc {k} differs from pid_mean"
    # a smaller problem after a larger one: fewer chunks, stale partials left behind
    U2 = U[: max(1, N // 3), : M // 2]
    ref2 = h.mean(U2, None if w is None else w[: M // 2].contiguous())
    h.sync()
    got2 = _noalloc(U2, None if w is None else w[: M // 2].contiguous())
    for k in ("in_in", "in_out", "depth", "rank"):
        assert torch.equal(got2[k], ref2[k]), f"noalloc {k} differs after a larger call"
    h.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    from paper_2512_15187_gb300 import binding as B, build
    build.build()
    N, M = 512, 4_400_000          # needs more than the 4 MiB of per-chunk partials
    # the size check rejects the call before any kernel could read U: a small real buffer
    # stands in for the 9 GB a problem of this size would occupy
    U = torch.empty(16, dtype=torch.float32, device="cuda")
    d = torch.empty(N, dtype=torch.float64, device="cuda")
    with pytest.raises(B.PidError) as e:
        B.pid_mean_noalloc(U.data_ptr(), N, M, M, None, d.data_ptr(), None, None, None, None, None)
    assert e.value.status == B.PID_ERR_UNSUPPORTED
    assert "scratch" in str(e.value)
