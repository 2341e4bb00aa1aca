"""Plain FP64 CPU oracle for Probabilistic Inclusion Depth (PID).

TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the CPU-baseline leg of
the benchmark call this module; the library and its Python binding never do.
It shares no code with the CUDA path: it is a direct transcription of the
paper's definitions, slow and obviously correct, computed in float64 from the
same float32 inputs the GPU receives.

Every function cites the passage it follows:
  Eq. 1            epsilon-subset operator (Sec. 3.1)
  Eq. 2            inside region of a contour, F_i(x) < q_i (Sec. 3.1)
  Eq. 3, Eq. 4     eID inclusion fractions and their minimum (Sec. 3.1)
  Eq. 6            mass of a probabilistic mask (Sec. 3.2)
  Eq. 9            probabilistic inclusion operator, ratio form (Sec. 3.2)
  Eq. 10           PID (Sec. 3.2)
  Eq. 12, 13, 14   uniform and non-uniform (cell-measure weighted) grids (Sec. 3.4)
  Eq. 15, Eq. 16   mean contour and PID-mean (Sec. 4.1)
  Sec. 3.5         probabilistic mask from a scalar field and an isovalue distribution
  Sec. 5.1         ranking: higher rank = lower depth
  (pid_chunked / pid_mean_chunked restate Eq. 6, 9, 10, 15, 16 with their sums over
  cells accumulated block by block, for ensembles larger than host memory in float64)
  Sec. 6           contour boxplots: unions and intersections of the binarised members
                   of a depth-ordered population, and the median member
  Sec. 3.5, 3.6    other mask models: a uniform isovalue distribution, the level-centred
                   map of the weather example
  Sec. 4.1         the reliability-weighted mean contour
  Sec. 6.3         4D (space-time) PID: time as one more cell axis

Readings where the paper is silent (Sec. 3.2, Sec. 3.5, Sec. 5.1 leave these open):
  * Zero-mass reference mask: u subset_p v = 0 (Sec. 3.2), unlike eID's 1 (Eq. 1).
  * The sums over j in Eq. 10 / Eq. 14 include j = i and are normalised by 1/N.
  * Isovalue distribution q ~ Normal(mu, sigma): u(x) = P(F(x) < q) =
    Phi((mu - F(x)) / sigma) (inside = sub-level set, Eq. 2); sigma = 0 gives the
    strict indicator 1[F < mu]; `superlevel` swaps to P(F(x) > q).
  * Ranking ties: depth descending, then member index ascending.

Parity pins: every function here is pinned by the CPU tests (closed forms,
brute-force set counts, invariants, textbook values); none is "parity unpinned".
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc as _erfc

__all__ = [
    "cell_measure",
    "mass",
    "inclusion",
    "inclusion_matrix",
    "pid",
    "mean_contour",
    "pid_mean",
    "iso_soft_mask",
    "rank_by_depth",
    "eps_subset",
    "eid",
    "pid_chunked",
    "pid_mean_chunked",
    "contour_bands",
    "iso_soft_mask_uniform",
    "level_soft_mask",
    "pid_mean_weighted",
]


def _f64(a) -> np.ndarray:
    return np.asarray(a, dtype=np.float64)


def cell_measure(M: int, w=None) -> np.ndarray:
    """Cell measure w_x of Eq. 13; a uniform grid (Eq. 12) is w_x = 1."""
    if w is None:
        return np.ones(M, dtype=np.float64)
    w = _f64(w).reshape(-1)
    if w.shape[0] != M:
        raise ValueError("weights must have one entry per cell")
    if not np.all(w > 0):
        raise ValueError("cell measures must be positive (Sec. 3.4, w_x > 0)")
    return w


def mass(U, w=None) -> np.ndarray:
    """m(u_i) = sum_x w_x u_i(x): Eq. 6 with the cell-wise constant measure of Eq. 13."""
    U = np.atleast_2d(_f64(U))
    w = cell_measure(U.shape[1], w)
    return U @ w


def inclusion(u, v, w=None) -> float:
    """u subset_p v = sum_x w u v / sum_x w u (Eq. 9 with Eq. 13); 0 if m(u) = 0."""
    u = _f64(u).reshape(-1)
    v = _f64(v).reshape(-1)
    w = cell_measure(u.shape[0], w)
    m = float(np.dot(w, u))
    if m == 0.0:
        return 0.0
    return float(np.dot(w * u, v) / m)


def inclusion_matrix(U, w=None) -> np.ndarray:
    """P[i, j] = u_i subset_p u_j for every ordered pair, in the penalty form of Eq. 14:

        P[i, j] = 1 - sum_x w_x u_i(x) (1 - u_j(x)) / sum_x w_x u_i(x),

    with P[i, :] = 0 when m(u_i) = 0 (zero-mass convention of Sec. 3.2).
    """
    U = np.atleast_2d(_f64(U))
    w = cell_measure(U.shape[1], w)
    m = U @ w                                   # Eq. 6
    penalty = (U * w) @ (1.0 - U).T             # sum_x w u_i (1 - u_j)
    P = np.zeros_like(penalty)
    nz = m > 0
    P[nz, :] = 1.0 - penalty[nz, :] / m[nz, None]
    return P


def pid(U, w=None):
    """Full PID over all N^2 ordered pairs (Eq. 10, weighted sums of Eq. 14).

    IN_in(i)  = (1/N) sum_j u_i subset_p u_j
    IN_out(i) = (1/N) sum_j u_j subset_p u_i
    PID(i)    = min(IN_in(i), IN_out(i))
    Returns (in_in, in_out, depth) as float64 arrays of length N.
    """
    P = inclusion_matrix(U, w)
    N = P.shape[0]
    in_in = P.sum(axis=1) / N
    in_out = P.sum(axis=0) / N
    return in_in, in_out, np.minimum(in_in, in_out)


def mean_contour(U) -> np.ndarray:
    """u_bar(x) = (1/N) sum_i u_i(x) (Eq. 15)."""
    U = np.atleast_2d(_f64(U))
    return U.mean(axis=0)


def pid_mean(U, w=None):
    """PID-mean (Eq. 16): each member against the mean contour only.

    IN_in^mean(i)  = u_i subset_p u_bar
    IN_out^mean(i) = u_bar subset_p u_i
    Returns (in_in, in_out, depth).
    """
    U = np.atleast_2d(_f64(U))
    ubar = mean_contour(U)
    N = U.shape[0]
    in_in = np.array([inclusion(U[i], ubar, w) for i in range(N)])
    in_out = np.array([inclusion(ubar, U[i], w) for i in range(N)])
    return in_in, in_out, np.minimum(in_in, in_out)


# ---------------------------------------------------------------------------
# The same definitions for ensembles too large to hold in float64 at once: every sum over
# cells in Eq. 6, Eq. 9 and Eq. 15/16 is a sum of per-cell terms, so it can be accumulated
# over consecutive blocks of cells. `chunks` yields (U_block [N, m], w_block [m] or None);
# the blocks must cover the cells once.
# ---------------------------------------------------------------------------

def pid_chunked(chunks):
    """Full PID (Eq. 10 with Eq. 14) from G_ij = sum_x w u_i u_j and m_i = sum_x w u_i,
    both accumulated block by block; P_ij = G_ij / m_i (ratio form of Eq. 9, 0 if m_i = 0).
    Returns (in_in, in_out, depth)."""
    G = None
    m = None
    for Ub, wb in chunks:
        Ub = np.atleast_2d(_f64(Ub))
        wb = cell_measure(Ub.shape[1], wb)
        if G is None:
            G = np.zeros((Ub.shape[0], Ub.shape[0]))
            m = np.zeros(Ub.shape[0])
        G += (Ub * wb) @ Ub.T
        m += Ub @ wb
    N = G.shape[0]
    P = np.zeros_like(G)
    nz = m > 0
    P[nz, :] = G[nz, :] / m[nz, None]
    in_in = P.sum(axis=1) / N
    in_out = P.sum(axis=0) / N
    return in_in, in_out, np.minimum(in_in, in_out)


def pid_mean_chunked(chunks):
    """PID-mean (Eq. 16) with u_bar of Eq. 15 formed per block (it is cell-local):
    IN_in(i) = sum_x w u_i u_bar / sum_x w u_i, IN_out(i) = sum_x w u_bar u_i / sum_x w u_bar,
    each sum accumulated block by block. Returns (in_in, in_out, depth)."""
    num = None
    for Ub, wb in chunks:
        Ub = np.atleast_2d(_f64(Ub))
        wb = cell_measure(Ub.shape[1], wb)
        ubar = mean_contour(Ub)
        if num is None:
            num = np.zeros(Ub.shape[0])
            m = np.zeros(Ub.shape[0])
            mbar = 0.0
        num += Ub @ (wb * ubar)
        m += Ub @ wb
        mbar += float(wb @ ubar)
    in_in = np.where(m > 0, num / np.where(m > 0, m, 1.0), 0.0)
    in_out = num / mbar if mbar > 0 else np.zeros_like(num)
    return in_in, in_out, np.minimum(in_in, in_out)


def iso_soft_mask(F, mu: float, sigma: float, superlevel: bool = False) -> np.ndarray:
    """Probabilistic mask from a scalar field and a Normal isovalue distribution (Sec. 3.5).

    The inside of a contour is the sub-level set F(x) < q (Eq. 2). With the isovalue
    q ~ Normal(mu, sigma) the membership probability is
        u(x) = P(F(x) < q) = Phi((mu - F(x)) / sigma) = erfc((F(x) - mu) / (sigma sqrt 2)) / 2.
    sigma = 0 degenerates to the strict indicator 1[F(x) < mu]. `superlevel` takes the
    super-level set F(x) > q instead: u(x) = Phi((F(x) - mu) / sigma), or 1[F(x) > mu].
    """
    F = _f64(F)
    if sigma < 0:
        raise ValueError("sigma must be >= 0")
    if sigma == 0.0:
        return (F > mu).astype(np.float64) if superlevel else (F < mu).astype(np.float64)
    z = (F - mu) / (sigma * math.sqrt(2.0))
    if superlevel:
        z = -z
    return 0.5 * _erfc(z)


def iso_soft_mask_uniform(F, mu: float, half_width: float, superlevel: bool = False) -> np.ndarray:
    """Soft mask for an isovalue uniform on [mu - h, mu + h] (Sec. 3.5 with another
    isovalue distribution): u(x) = P(F(x) < q) = clamp((mu + h - F) / (2 h), 0, 1), or
    P(F(x) > q) = clamp((F - (mu - h)) / (2 h), 0, 1) for the super-level set."""
    F = _f64(F)
    if not half_width > 0:
        raise ValueError("half_width must be > 0")
    if superlevel:
        return np.clip((F - (mu - half_width)) / (2.0 * half_width), 0.0, 1.0)
    return np.clip((mu + half_width - F) / (2.0 * half_width), 0.0, 1.0)


def level_soft_mask(F, level: float, half_width: float) -> np.ndarray:
    """Level-centred soft mask (the weather example of Sec. 3.6): probability 1 at the level,
    falling linearly to 0 at distance `half_width`: u = max(0, 1 - |F - level| / h)."""
    F = _f64(F)
    if not half_width > 0:
        raise ValueError("half_width must be > 0")
    return np.maximum(0.0, 1.0 - np.abs(F - level) / half_width)


def pid_mean_weighted(U, member_weights, w=None):
    """PID-mean against a reliability-weighted mean contour (Sec. 4.1):
    u_bar = sum_j r_j u_j / sum_j r_j, then IN_in(i) = u_i subset_p u_bar and
    IN_out(i) = u_bar subset_p u_i (Eq. 16). Returns (in_in, in_out, depth)."""
    U = np.atleast_2d(_f64(U))
    r = _f64(member_weights).reshape(-1)
    if r.shape[0] != U.shape[0] or not np.all(r >= 0) or not r.sum() > 0:
        raise ValueError("one non-negative member weight per member, not all zero")
    ubar = (r[:, None] * U).sum(axis=0) / r.sum()
    N = U.shape[0]
    in_in = np.array([inclusion(U[i], ubar, w) for i in range(N)])
    in_out = np.array([inclusion(ubar, U[i], w) for i in range(N)])
    return in_in, in_out, np.minimum(in_in, in_out)


def pid_grouped(U, labels, w=None):
    """Full PID (Eq. 10) of each member within its group: member i is compared only with
    the members j that share its label (the depth of i within its mode of a multimodal
    ensemble, Sec. 2.2). Returns (in_in, in_out, depth, rank), rank within the group
    (Sec. 5.1 ordering, ties to the lower member index)."""
    U = np.atleast_2d(_f64(U))
    labels = np.asarray(labels).reshape(-1)
    N = U.shape[0]
    if labels.shape[0] != N:
        raise ValueError("one label per member")
    in_in, in_out, depth = np.zeros(N), np.zeros(N), np.zeros(N)
    rank = np.zeros(N, dtype=np.int64)
    for g in np.unique(labels):
        idx = np.nonzero(labels == g)[0]
        a, b, d = pid(U[idx], w)
        in_in[idx], in_out[idx], depth[idx] = a, b, d
        rank[idx] = rank_by_depth(d)
    return in_in, in_out, depth, rank


def spacetime_cells(steps, w=None):
    """4D PID (time as one more cell axis): the cells (x, t) of T time steps, each [N][M],
    concatenated into one ensemble [N][T*M]; the cell measure w_x repeats at every step (a
    uniform time step is a common factor of every sum and cancels in Eq. 9). Returns
    (U, w) to pass to pid / pid_mean."""
    steps = [np.atleast_2d(_f64(S)) for S in steps]
    U = np.concatenate(steps, axis=1)
    return U, (None if w is None else np.tile(_f64(w), len(steps)))


def rank_by_depth(depth) -> np.ndarray:
    """Rank 0 = deepest member; higher rank = lower depth (Sec. 5.1).

    Ties are broken by the lower member index (a stable sort on descending depth).
    Returns rank[i] for every member i (int32).
    """
    depth = _f64(depth).reshape(-1)
    order = sorted(range(depth.shape[0]), key=lambda i: (-depth[i], i))
    rank = np.empty(depth.shape[0], dtype=np.int32)
    for r, i in enumerate(order):
        rank[i] = r
    return rank


# ---------------------------------------------------------------------------
# Epsilon Inclusion Depth on binary masks (Sec. 3.1), by set counts.
# Used by the tests as the binary specialisation of PID (Eq. 5).
# ---------------------------------------------------------------------------

def eps_subset(A: set, B: set) -> float:
    """A subset_eps B = 1 - |A minus B| / |A|, and 1 if |A| = 0 (Eq. 1)."""
    if len(A) == 0:
        return 1.0
    return 1.0 - len(A - B) / len(A)


def eid(sets):
    """eID over a list of cell-index sets (Eq. 3 and Eq. 4), counting measure.

    Returns (in_in, in_out, depth); the sums over j include j = i (Eq. 3).
    """
    N = len(sets)
    in_in = np.array([sum(eps_subset(sets[i], sets[j]) for j in range(N)) / N for i in range(N)])
    in_out = np.array([sum(eps_subset(sets[j], sets[i]) for j in range(N)) / N for i in range(N)])
    return in_in, in_out, np.minimum(in_in, in_out)


# ---------------------------------------------------------------------------
# Contour boxplot bands (Sec. 6): binarise each soft mask at a probability threshold,
# then take the union and the intersection over the deepest fraction of the members and
# over all members; the median member is the deepest one.
# ---------------------------------------------------------------------------

BAND_INNER_UNION, BAND_INNER_INTERSECTION = 1, 2
BAND_ALL_UNION, BAND_ALL_INTERSECTION = 4, 8
BAND_MEDIAN = 16


def contour_bands(U, rank, tau: float, inner_fraction: float = 0.5) -> np.ndarray:
    """Per cell, a byte of band flags for the contour boxplot of Sec. 6.

    b_i(x) = [u_i(x) > tau]; the inner population is the ceil(inner_fraction N) members of
    lowest rank (rank 0 = deepest, Sec. 5.1), the outer population all N members.
    bit 0: union over the inner population      bit 1: intersection over it
    bit 2: union over all members               bit 3: intersection over all members
    bit 4: b of the median (rank-0) member
    """
    U = np.atleast_2d(_f64(U))
    rank = np.asarray(rank).reshape(-1)
    N, M = U.shape
    if rank.shape[0] != N:
        raise ValueError("one rank per member")
    n_inner = int(math.ceil(inner_fraction * N))
    B = U > tau
    inner = B[rank < n_inner]
    out = np.zeros(M, dtype=np.uint8)
    if inner.shape[0] > 0:
        out |= inner.any(axis=0).astype(np.uint8) * BAND_INNER_UNION
        out |= inner.all(axis=0).astype(np.uint8) * BAND_INNER_INTERSECTION
    out |= B.any(axis=0).astype(np.uint8) * BAND_ALL_UNION
    out |= B.all(axis=0).astype(np.uint8) * BAND_ALL_INTERSECTION
    med = np.nonzero(rank == 0)[0]
    if med.size:
        out |= B[med[0]].astype(np.uint8) * BAND_MEDIAN
    return out
