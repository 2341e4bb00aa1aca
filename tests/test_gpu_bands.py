"""GPU parity of the contour boxplot bands (pid_contour_bands, Sec. 6) with the FP64
oracle, bit for bit: soft masks and fields (normal isovalue, both level sets, sigma = 0),
ragged and unaligned rows, any N, several thresholds and inner fractions, ranks from a
permutation and from the library's own depths, and the 2D field workload at full size."""
import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth
from tests.helpers import to_np

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


def _rank(N, seed):
    import torch
    perm = np.random.default_rng(seed).permutation(N).astype(np.int32)
    return perm, torch.from_numpy(perm).cuda()


@pytest.mark.parametrize("N,M", [(1, 37), (7, 1001), (64, 65536), (300, 5003), (1000, 2050)])
@pytest.mark.parametrize("tau,frac", [(0.5, 0.5), (0.02, 0.25), (0.9, 1.0)])
def test_bands_soft_masks(H, N, M, tau, frac):
    U = synth.random_soft(N, M, seed=N + M, binary_frac=0.3)
    U[:, ::7] = np.float32(tau)          # exactly at the threshold: not above it
    perm, r = _rank(N, M)
    got = to_np(H.contour_bands(_dev(U), r, tau, frac))
    assert np.array_equal(got, O.contour_bands(U, perm, tau, frac))


@pytest.mark.parametrize("sigma,superlevel", [(0.05, False), (0.05, True), (0.0, False), (0.0, True)])
@pytest.mark.parametrize("tau", [0.5, 0.02])
def test_bands_fields(H, sigma, superlevel, tau):
    F = synth.rbf_fields_2d(N=33, H=96, W=75, n_rbf=8)
    F = (F - np.median(F, axis=1, keepdims=True) + 0.5).astype(np.float32)
    perm, r = _rank(33, 3)
    got = to_np(H.contour_bands(_dev(F), r, tau, 0.5, iso=(0.5, sigma, int(superlevel))))
    U = O.iso_soft_mask(F, 0.5, sigma, superlevel)
    assert np.array_equal(got, O.contour_bands(U, perm, tau, 0.5))


def test_bands_unaligned_rows(H):
    import torch
    N, M = 21, 4097
    U = synth.random_soft(N, M, seed=9)
    big = torch.zeros((N, M + 3), dtype=torch.float32, device="cuda")
    big[:, :M] = _dev(U)
    perm, r = _rank(N, 1)
    got = to_np(H.contour_bands(big[:, :M], r, 0.5, 0.5))
    assert np.array_equal(got, O.contour_bands(U, perm, 0.5, 0.5))


def test_bands_from_library_depths_full_size(H):
    import torch
    F = torch.empty((64, 512 * 512), device="cuda")
    synth.rbf_fields_2d_torch(64, 512, 512, 32, seed=synth.DEFAULT_SEED + 2, device="cuda", out=F)
    o = H.from_fields(F, 0.5, 0.05, mode="mean")
    got = to_np(H.contour_bands(F, o["rank"], 0.5, 0.5, iso=(0.5, 0.05, 0)))
    U = O.iso_soft_mask(to_np(F), 0.5, 0.05)
    assert np.array_equal(got, O.contour_bands(U, to_np(o["rank"]), 0.5, 0.5))
    # the deepest half's band lies inside the all-member band, the median inside both
    b = got
    assert np.all(((b & 2) > 0) <= ((b & 16) > 0)) and np.all(((b & 16) > 0) <= ((b & 1) > 0))
    assert np.all(((b & 1) > 0) <= ((b & 4) > 0)) and np.all(((b & 8) > 0) <= ((b & 2) > 0))


def test_bands_rejects_bad_arguments(H):
    import torch
    from paper_2512_15187_gb300 import binding as B
    U = torch.rand((4, 100), device="cuda")
    r = torch.arange(4, dtype=torch.int32, device="cuda")
    for tau, frac in [(0.0, 0.5), (1.0, 0.5), (0.5, 0.0), (0.5, 1.5)]:
        with pytest.raises(B.PidError) as e:
            H.contour_bands(U, r, tau, frac)
        assert e.value.status == B.PID_ERR_INVALID_ARG
