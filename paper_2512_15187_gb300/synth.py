"""Seeded synthetic ensembles shaped like the paper's workloads.

This module holds no depth arithmetic: it only draws inputs (soft masks, scalar
fields, cell measures). Both the FP64 oracle tests and the CUDA path consume
the arrays it returns, so the two sides always see the same float32 values.

Every ensemble is reproducible from a 64-bit seed; member i draws from the
sub-stream (seed, i) so that members can be regenerated independently.

Workloads (sizes of the benchmark configurations):
  ellipses_2d     N = 20 soft ellipses on 128 x 128 (plus their binary copies)
  rbf_fields_2d   N = 64 scalar fields on 512 x 512, 32 Gaussian bumps + noise,
                  used with an isovalue ~ Normal(0.5, 0.05)
  radial_disk     N = 128 perturbed radial masks on 2^20 scattered points in the
                  unit disk with log-uniform lumped-area weights (non-Cartesian)
  plume_3d        smoke-plume-like 3D soft masks (sigmoid of a noise-displaced
                  cone, 5-octave fBm), generated on the device with torch;
                  plume_3d_slab gives a slab of z-planes of the same recipe
  ellipsoids_3d   3D ellipsoid soft masks, 80% normal members and 20% outliers (the
                  scalability study's ensembles), generated on the device with torch
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_SEED = 2512015187


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed) & 0xFFFFFFFFFFFFFFFF, *[int(s) for s in stream]])


def _sigmoid(z: np.ndarray) -> np.ndarray:
    return 0.5 * (1.0 + np.tanh(0.5 * z))


# ---------------------------------------------------------------------------
# 2D ellipses (128 x 128): soft masks sigmoid((r_i - d(x, c_i)) / w_i)
# ---------------------------------------------------------------------------

def ellipses_2d(N: int = 20, H: int = 128, W: int = 128, seed: int = DEFAULT_SEED + 1,
                binary: bool = False) -> np.ndarray:
    """Random soft ellipses; returns float32 [N, H*W].

    Member i: centre = (H/2, W/2) + U[-10, 10]^2 px, semi-axes a, b ~ U[25, 45] px,
    rotation ~ U[0, pi), edge width w ~ U[1, 4] px. With s the ellipse-normalised
    radius of pixel x (s = 1 on the boundary) and r = sqrt(a b), the signed
    distance is approximated by d - r = (s - 1) r and u(x) = sigmoid((1 - s) r / w).
    `binary` returns the thresholded copies 1[s <= 1].
    """
    yy, xx = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64),
                         indexing="ij")
    out = np.empty((N, H * W), dtype=np.float32)
    for i in range(N):
        g = _rng(seed, i)
        cy, cx = H / 2 + g.uniform(-10, 10), W / 2 + g.uniform(-10, 10)
        a, b = g.uniform(25, 45, size=2)
        th = g.uniform(0, math.pi)
        wd = g.uniform(1, 4)
        dx, dy = xx - cx, yy - cy
        xr = math.cos(th) * dx + math.sin(th) * dy
        yr = -math.sin(th) * dx + math.cos(th) * dy
        s = np.sqrt((xr / a) ** 2 + (yr / b) ** 2)
        if binary:
            out[i] = (s <= 1.0).reshape(-1)
        else:
            out[i] = _sigmoid((1.0 - s) * math.sqrt(a * b) / wd).reshape(-1)
    return out


# ---------------------------------------------------------------------------
# 2D scalar fields (512 x 512): sum of 32 Gaussian RBFs + i.i.d. noise
# ---------------------------------------------------------------------------

def rbf_fields_2d(N: int = 64, H: int = 512, W: int = 512, n_rbf: int = 32,
                  seed: int = DEFAULT_SEED + 2) -> np.ndarray:
    """Scalar fields F_i = sum_k A_k exp(-|x - c_k|^2 / (2 s_k^2)) + N(0, 0.05).

    Centres uniform on the grid, amplitudes ~ N(1, 0.3), widths s_k ~ U[20, 60] px.
    Returns float32 [N, H*W]. Pair with the isovalue distribution Normal(0.5, 0.05).
    """
    y = np.arange(H, dtype=np.float64)
    x = np.arange(W, dtype=np.float64)
    out = np.empty((N, H * W), dtype=np.float32)
    for i in range(N):
        g = _rng(seed, i)
        cy = g.uniform(0, H, n_rbf)
        cx = g.uniform(0, W, n_rbf)
        amp = g.normal(1.0, 0.3, n_rbf)
        sd = g.uniform(20, 60, n_rbf)
        F = np.zeros((H, W), dtype=np.float64)
        for k in range(n_rbf):  # separable Gaussian bump
            gy = np.exp(-((y - cy[k]) ** 2) / (2 * sd[k] ** 2))
            gx = np.exp(-((x - cx[k]) ** 2) / (2 * sd[k] ** 2))
            F += amp[k] * np.outer(gy, gx)
        F += g.normal(0.0, 0.05, size=(H, W))
        out[i] = F.reshape(-1)
    return out


# ---------------------------------------------------------------------------
# Non-Cartesian: scattered points in the unit disk with lumped-area weights
# ---------------------------------------------------------------------------

def disk_points(M: int = 1 << 20, seed: int = DEFAULT_SEED + 3):
    """M random points in the unit disk and positive per-point cell measures.

    Returns (r, theta, w): float64 radius and angle, float32 weights drawn
    log-uniformly over two decades (10^U[0, 2]) and scaled to sum to pi (the disk area).
    """
    g = _rng(seed, 1 << 30)
    r = np.sqrt(g.uniform(0, 1, M))
    th = g.uniform(0, 2 * math.pi, M)
    w = 10.0 ** g.uniform(0, 2, M)
    w = (w * (math.pi / w.sum())).astype(np.float32)
    return r, th, w


def radial_disk(N: int = 128, M: int = 1 << 20, seed: int = DEFAULT_SEED + 3):
    """Perturbed radial soft masks u_i = (1 + tanh((0.5 + 0.1 xi_i(theta) - r) / 0.02)) / 2.

    xi_i is an 8-term Fourier series with a_k, b_k ~ N(0, 1/k^2), divided by its
    maximum magnitude over the points so that max |xi_i| = 1.
    Returns (U float32 [N, M], w float32 [M]).
    """
    r, th, w = disk_points(M, seed)
    K = 8
    basis = np.empty((M, 2 * K), dtype=np.float64)
    for k in range(1, K + 1):
        basis[:, 2 * (k - 1)] = np.cos(k * th)
        basis[:, 2 * (k - 1) + 1] = np.sin(k * th)
    U = np.empty((N, M), dtype=np.float32)
    for i in range(N):
        g = _rng(seed, i)
        coef = g.normal(0.0, 1.0, 2 * K) / np.repeat(np.arange(1, K + 1), 2)
        xi = basis @ coef
        xi /= max(np.abs(xi).max(), 1e-12)
        U[i] = 0.5 * (1.0 + np.tanh((0.5 + 0.1 * xi - r) / 0.02))
    return U, w


# ---------------------------------------------------------------------------
# Binary / nested shapes used by the closed-form tests
# ---------------------------------------------------------------------------

def nested_disks(radii, H: int = 64, W: int = 64) -> np.ndarray:
    """Concentric binary disks (pixel centres within radius r of the grid centre)."""
    yy, xx = np.meshgrid(np.arange(H) + 0.5 - H / 2, np.arange(W) + 0.5 - W / 2, indexing="ij")
    d = np.sqrt(yy ** 2 + xx ** 2).reshape(-1)
    return np.stack([(d <= r).astype(np.float32) for r in radii])


def random_soft(N: int, M: int, seed: int, binary_frac: float = 0.0) -> np.ndarray:
    """Unstructured random masks in [0, 1] (some exact 0/1 entries when binary_frac > 0)."""
    g = _rng(seed, 0)
    U = g.uniform(0, 1, size=(N, M))
    if binary_frac > 0:
        sel = g.uniform(0, 1, size=(N, M)) < binary_frac
        U[sel] = np.round(U[sel])
    return U.astype(np.float32)


# ---------------------------------------------------------------------------
# 3D smoke-plume-like soft masks (device generator, torch)
# ---------------------------------------------------------------------------

def plume_3d(N: int, R: int, t: int = 0, T: int = 16, seed: int = DEFAULT_SEED + 4,
             device: str = "cuda", out=None, octaves: int = 5):
    """Soft masks u = sigmoid((R(z, t) - rho + A fBm(x)) / w) of a noise-displaced cone.

    rho is the horizontal distance to the vertical axis, R(z, t) a cone radius that
    widens with height and is cut off above the plume front h(t) = 0.3 + 0.65 t / (T-1).
    fBm: `octaves` octaves of trilinearly interpolated value noise, lattice 4 * 2^o,
    amplitude 2^-o, member-specific seed (seed, t, i). Constants: A = 0.08, w = 0.02.
    Returns a float32 torch tensor [N, R^3] on `device` (written into `out` if given).
    """
    import torch
    import torch.nn.functional as Fnn

    if out is None:
        out = torch.empty((N, R ** 3), dtype=torch.float32, device=device)
    z = torch.linspace(0, 1, R, device=device).view(R, 1, 1)
    yy = torch.linspace(-0.5, 0.5, R, device=device).view(1, R, 1)
    xx = torch.linspace(-0.5, 0.5, R, device=device).view(1, 1, R)
    rho = torch.sqrt(yy ** 2 + xx ** 2)
    h = 0.3 + 0.65 * t / max(T - 1, 1)
    cone = (0.04 + 0.25 * z) * torch.clamp((h - z) / 0.08, 0.0, 1.0)
    base = cone - rho  # [R, R, R]
    for i in range(N):
        g = torch.Generator(device=device)
        g.manual_seed((int(seed) * 1_000_003 + t * 10_007 + i) & 0x7FFFFFFFFFFFFFFF)
        noise = torch.zeros((R, R, R), device=device)
        amp = 1.0
        for o in range(octaves):
            L = 4 * (2 ** o) + 1
            lat = torch.rand((1, 1, L, L, L), generator=g, device=device) * 2.0 - 1.0
            noise += amp * Fnn.interpolate(lat, size=(R, R, R), mode="trilinear",
                                          align_corners=True)[0, 0]
            amp *= 0.5
        out[i] = torch.sigmoid((base + 0.08 * noise) / 0.02).reshape(-1)
    return out


def plume_3d_slab(N: int, R: int, z0: int, nz: int, t: int = 0, T: int = 16,
                  seed: int = DEFAULT_SEED + 4, device: str = "cpu", octaves: int = 5):
    """Planes z0 .. z0 + nz - 1 of plume_3d(N, R, t, T, seed) on `device`: [N, nz * R^2].

    The same recipe restricted to a slab of the volume, for samples that a host can afford
    (the whole 256^3 volume of 200 members takes minutes on host cores). Trilinear
    interpolation with aligned corners is separable, so each octave's lattice is
    interpolated along z at the slab's planes first, then bilinearly in (y, x). On a given
    device the lattices are the draws of plume_3d, so the slab matches the corresponding
    planes of the full volume up to rounding; on the host the generator's stream differs from
    the GPU's, so a host slab is another member of the same ensemble distribution.
    """
    import torch
    import torch.nn.functional as Fnn

    zs = torch.arange(z0, z0 + nz, dtype=torch.float32, device=device)
    z = (zs / (R - 1)).view(nz, 1, 1)
    yy = torch.linspace(-0.5, 0.5, R, device=device).view(1, R, 1)
    xx = torch.linspace(-0.5, 0.5, R, device=device).view(1, 1, R)
    rho = torch.sqrt(yy ** 2 + xx ** 2)
    h = 0.3 + 0.65 * t / max(T - 1, 1)
    cone = (0.04 + 0.25 * z) * torch.clamp((h - z) / 0.08, 0.0, 1.0)
    base = cone - rho  # [nz, R, R]
    out = torch.empty((N, nz * R * R), dtype=torch.float32, device=device)
    for i in range(N):
        g = torch.Generator(device=device)
        g.manual_seed((int(seed) * 1_000_003 + t * 10_007 + i) & 0x7FFFFFFFFFFFFFFF)
        noise = torch.zeros((nz, R, R), device=device)
        amp = 1.0
        for o in range(octaves):
            L = 4 * (2 ** o) + 1
            lat = torch.rand((L, L, L), generator=g, device=device) * 2.0 - 1.0
            # along z: lattice coordinate of each slab plane, linear weights
            pz = zs * (L - 1) / (R - 1)
            k0 = torch.clamp(pz.floor().long(), 0, L - 2)
            fz = (pz - k0.to(pz.dtype)).view(nz, 1, 1)
            planes = lat[k0] * (1.0 - fz) + lat[k0 + 1] * fz          # [nz, L, L]
            noise += amp * Fnn.interpolate(planes.unsqueeze(1), size=(R, R), mode="bilinear",
                                           align_corners=True)[:, 0]
            amp *= 0.5
        out[i] = torch.sigmoid((base + 0.08 * noise) / 0.02).reshape(-1)
    return out


def ellipses_2d_torch(N: int, H: int, W: int, seed: int = DEFAULT_SEED + 1, device: str = "cuda"):
    """The recipe of ellipses_2d on the device (torch's generator: other draws, the same
    distribution): float32 [N, H*W] soft ellipses of semi-axes U[25, 45] px around the grid
    centre +- 10 px, rotation U[0, pi), edge width U[1, 4] px."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    p = torch.rand((N, 6), generator=g, device=device, dtype=torch.float64)
    cy = H / 2 + (p[:, 0] * 20 - 10)
    cx = W / 2 + (p[:, 1] * 20 - 10)
    a = 25 + 20 * p[:, 2]
    b = 25 + 20 * p[:, 3]
    th = math.pi * p[:, 4]
    wd = 1 + 3 * p[:, 5]
    yy = torch.arange(H, device=device, dtype=torch.float64).view(1, H, 1)
    xx = torch.arange(W, device=device, dtype=torch.float64).view(1, 1, W)
    out = torch.empty((N, H * W), dtype=torch.float32, device=device)
    for i0 in range(0, N, 16):
        sl = slice(i0, min(N, i0 + 16))
        v = lambda t: t[sl].view(-1, 1, 1)
        dx, dy = xx - v(cx), yy - v(cy)
        xr = torch.cos(v(th)) * dx + torch.sin(v(th)) * dy
        yr = -torch.sin(v(th)) * dx + torch.cos(v(th)) * dy
        sdist = torch.sqrt((xr / v(a)) ** 2 + (yr / v(b)) ** 2)
        out[sl] = torch.sigmoid((1.0 - sdist) * torch.sqrt(v(a) * v(b)) / v(wd)).reshape(-1, H * W).float()
    return out


def radial_disk_torch(N: int, M: int, seed: int = DEFAULT_SEED + 3, device: str = "cuda"):
    """The recipe of radial_disk on the device (torch's generator: other draws, the same
    distribution): points uniform in the unit disk with cell measures 10^U[0, 2] scaled to sum
    to pi, masks (1 + tanh((0.5 + 0.1 xi_i(theta) - r) / 0.02)) / 2 with xi_i an 8-term Fourier
    series (a_k, b_k ~ N(0, 1/k^2)) normalised to max |xi_i| = 1. Returns (U [N, M], w [M])."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    r = torch.sqrt(torch.rand(M, generator=g, device=device, dtype=torch.float64))
    th = 2 * math.pi * torch.rand(M, generator=g, device=device, dtype=torch.float64)
    w = 10.0 ** (2 * torch.rand(M, generator=g, device=device, dtype=torch.float64))
    w = (w * (math.pi / w.sum())).float()
    K = 8
    ks = torch.arange(1, K + 1, device=device, dtype=torch.float64)
    basis = torch.cat([torch.cos(th[:, None] * ks), torch.sin(th[:, None] * ks)], dim=1)  # [M, 2K]
    coef = torch.randn((N, 2 * K), generator=g, device=device, dtype=torch.float64) / torch.cat([ks, ks])
    U = torch.empty((N, M), dtype=torch.float32, device=device)
    for i0 in range(0, N, 32):
        xi = coef[i0:i0 + 32] @ basis.T
        xi = xi / xi.abs().amax(dim=1, keepdim=True).clamp_min(1e-12)
        U[i0:i0 + 32] = (0.5 * (1.0 + torch.tanh((0.5 + 0.1 * xi - r) / 0.02))).float()
    return U, w


def rbf_fields_2d_torch(N: int = 64, H: int = 512, W: int = 512, n_rbf: int = 32,
                        seed: int = DEFAULT_SEED + 2, device: str = "cuda", out=None,
                        chunk: int = 256):
    """Device twin of rbf_fields_2d (same recipe, torch Philox stream instead of numpy's).

    F_i = sum_k A_k gy_k(y) gx_k(x) + N(0, 0.05): each Gaussian bump is separable, so a
    member is the product of a [H, n_rbf] and an [n_rbf, W] factor. Returns float32 [N, H*W].
    """
    import torch

    if out is None:
        out = torch.empty((N, H * W), dtype=torch.float32, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    y = torch.arange(H, dtype=torch.float32, device=device).view(1, H, 1)
    x = torch.arange(W, dtype=torch.float32, device=device).view(1, 1, W)
    for s in range(0, N, chunk):
        n = min(chunk, N - s)
        cy = torch.rand((n, 1, n_rbf), generator=g, device=device) * H
        cx = torch.rand((n, n_rbf, 1), generator=g, device=device) * W
        amp = 1.0 + 0.3 * torch.randn((n, 1, n_rbf), generator=g, device=device)
        sd = 20.0 + 40.0 * torch.rand((n, 1, n_rbf), generator=g, device=device)
        gy = torch.exp(-((y - cy) ** 2) / (2 * sd ** 2)) * amp          # [n, H, K]
        gx = torch.exp(-((x - cx) ** 2) / (2 * sd.transpose(1, 2) ** 2))  # [n, K, W]
        F = torch.bmm(gy, gx).view(n, H * W)
        F += 0.05 * torch.randn((n, H * W), generator=g, device=device)
        out[s:s + n] = F
    return out


# ---------------------------------------------------------------------------
# Scalability study: 3D ellipsoids with controlled contamination
# ---------------------------------------------------------------------------

def ellipsoids_3d(N: int, R: int, seed: int = DEFAULT_SEED + 5, outlier_frac: float = 0.2,
                  device: str = "cuda", out=None, chunk: int = 64):
    """Soft 3D ellipsoid masks on an R^3 grid over the unit cube, float32 [N, R^3].

    Member i is an axis-aligned ellipsoid with centre c_i and semi-axes a_i, and soft mask
    u = sigmoid((1 - s) / 0.05) with s the ellipsoid-normalised radius (s = 1 on the
    surface). Normal members (the first 80%): c = 0.5 + N(0, 0.02) per axis, semi-axes
    0.25 + N(0, 0.015). Outliers (the last 20%): c = 0.5 + N(0, 0.08), semi-axes drawn
    from U[0.12, 0.38] independently per axis. These constants are this generator's own
    choice (the paper does not print them).
    """
    import torch

    if out is None:
        out = torch.empty((N, R ** 3), dtype=torch.float32, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) & 0x7FFFFFFFFFFFFFFF)
    n_out = int(round(outlier_frac * N))
    n_norm = N - n_out
    c = 0.5 + 0.02 * torch.randn((N, 3), generator=g, device=device)
    a = 0.25 + 0.015 * torch.randn((N, 3), generator=g, device=device)
    if n_out:
        c[n_norm:] = 0.5 + 0.08 * torch.randn((n_out, 3), generator=g, device=device)
        a[n_norm:] = 0.12 + 0.26 * torch.rand((n_out, 3), generator=g, device=device)
    t = (torch.arange(R, dtype=torch.float32, device=device) + 0.5) / R
    chunk = max(1, min(chunk, (1 << 27) // (R ** 3)))   # bounded temporaries
    for s0 in range(0, N, chunk):
        n = min(chunk, N - s0)
        cz, cy, cx = (c[s0:s0 + n, k].view(n, 1, 1, 1) for k in range(3))
        az, ay, ax = (a[s0:s0 + n, k].view(n, 1, 1, 1) for k in range(3))
        s2 = (((t.view(1, R, 1, 1) - cz) / az) ** 2 + ((t.view(1, 1, R, 1) - cy) / ay) ** 2 +
              ((t.view(1, 1, 1, R) - cx) / ax) ** 2)
        out[s0:s0 + n] = torch.sigmoid((1.0 - torch.sqrt(s2)) / 0.05).view(n, -1)
    return out
