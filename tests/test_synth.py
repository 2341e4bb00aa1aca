"""CPU checks of the seeded input generators (no GPU): every ensemble is reproducible from
its seed, soft masks lie in [0, 1], the shapes are those asked for, and the slab generator
that feeds the host-side samples gives the planes of the full 3D plume volume."""
import numpy as np
import pytest

from paper_2512_15187_gb300 import synth


@pytest.mark.parametrize("make", [
    lambda s: synth.ellipses_2d(N=5, H=24, W=20, seed=s),
    lambda s: synth.ellipses_2d(N=5, H=128, W=128, seed=s, binary=True),
    lambda s: synth.rbf_fields_2d(N=3, H=16, W=16, n_rbf=4, seed=s),
    lambda s: synth.radial_disk(N=4, M=500, seed=s)[0],
    lambda s: synth.random_soft(6, 300, seed=s, binary_frac=0.3),
])
def test_generators_are_reproducible_from_their_seed(make):
    a, b, c = make(11), make(11), make(12)
    assert a.dtype == np.float32
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)


def test_soft_masks_lie_in_the_unit_interval_and_binary_copies_are_binary():
    for U in (synth.ellipses_2d(N=6, H=32, W=32), synth.random_soft(5, 400, seed=3, binary_frac=0.5),
              synth.radial_disk(N=3, M=1000)[0]):
        assert U.min() >= 0.0 and U.max() <= 1.0
    B = synth.ellipses_2d(N=6, H=32, W=32, binary=True)
    assert set(np.unique(B).tolist()) <= {0.0, 1.0}
    R = synth.random_soft(5, 2000, seed=4, binary_frac=1.0)
    assert set(np.unique(R).tolist()) <= {0.0, 1.0}


def test_radial_disk_points_and_measures():
    U, w = synth.radial_disk(N=3, M=5000)
    assert U.shape == (3, 5000) and w.shape == (5000,)
    assert np.all(w > 0)
    # lumped areas of points scattered in the unit disk sum to its area
    assert float(w.astype(np.float64).sum()) == pytest.approx(np.pi, rel=1e-5)


def test_nested_disks_are_nested():
    U = synth.nested_disks([3, 6, 9], 32, 32)
    assert np.all(U[0] <= U[1]) and np.all(U[1] <= U[2])
    assert U[0].sum() < U[1].sum() < U[2].sum()


def test_plume_slab_is_the_planes_of_the_full_volume():
    torch = pytest.importorskip("torch")
    N, R, z0, nz = 3, 24, 7, 5
    full = synth.plume_3d(N, R, t=5, T=16, device="cpu")
    slab = synth.plume_3d_slab(N, R, z0, nz, t=5, T=16, device="cpu")
    assert slab.shape == (N, nz * R * R)
    want = full[:, z0 * R * R:(z0 + nz) * R * R]
    assert torch.allclose(slab, want, atol=2e-5)
    assert float(full.min()) >= 0.0 and float(full.max()) <= 1.0
    # the plume front rises with the time step: more of the volume is inside later
    early = synth.plume_3d(N, R, t=0, T=16, device="cpu")
    assert float(early.sum()) < float(full.sum())


def test_ellipsoids_are_reproducible_and_outliers_last():
    torch = pytest.importorskip("torch")
    a = synth.ellipsoids_3d(10, 12, device="cpu")
    b = synth.ellipsoids_3d(10, 12, device="cpu")
    assert torch.equal(a, b)
    assert a.shape == (10, 12 ** 3)
    assert float(a.min()) >= 0.0 and float(a.max()) <= 1.0
