"""The pins catch plausible oracle mistakes.

Each mutant below is a deliberately broken copy of an oracle routine (a dropped
term, a wrong normalisation, a swapped index, a transposed operand, a wrong
zero-mass convention). The test asserts that at least one pin check rejects
each mutant, so a mistake of that kind in the real oracle could not pass.
CPU only; nothing here touches the GPU.
"""
import json
import os

import numpy as np
import pytest

from oracle import pid_oracle as O
from paper_2512_15187_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _P(U, w, *, weights=True, zero_mass=0.0, transpose=False, norm_by_j=False):
    U = np.atleast_2d(np.asarray(U, np.float64))
    w = np.ones(U.shape[1]) if (w is None or not weights) else np.asarray(w, np.float64)
    m = U @ w
    G = (U * w) @ U.T
    den = m[None, :] if norm_by_j else m[:, None]
    with np.errstate(divide="ignore", invalid="ignore"):
        P = np.where(den > 0, G / den, zero_mass)
    return P.T if transpose else P


def _pid_from(P, exclude_self=False):
    N = P.shape[0]
    if exclude_self:
        P = P - np.diag(np.diag(P))
        a, b = P.sum(1) / max(N - 1, 1), P.sum(0) / max(N - 1, 1)
    else:
        a, b = P.sum(1) / N, P.sum(0) / N
    return a, b, np.minimum(a, b)


MUTANTS = {
    "exclude_self_pair": lambda U, w=None: _pid_from(_P(U, w), exclude_self=True),
    "dropped_cell_measure": lambda U, w=None: _pid_from(_P(U, w, weights=False)),
    "eid_zero_mass_convention": lambda U, w=None: _pid_from(_P(U, w, zero_mass=1.0)),
    "transposed_pairs": lambda U, w=None: _pid_from(_P(U, w, transpose=True)),
    "normalised_by_wrong_member": lambda U, w=None: _pid_from(_P(U, w, norm_by_j=True)),
    "max_instead_of_min": lambda U, w=None: (lambda a, b, d: (a, b, np.maximum(a, b)))(
        *_pid_from(_P(U, w))),
}


def _pin_checks(pid):
    """Return the names of the pin checks that `pid` fails."""
    failed = []

    g = json.load(open(os.path.join(GOLDEN, "hand_weighted_2x3.json")))
    got = pid(np.array(g["U"]), np.array(g["w"]))
    if not np.allclose(got[2], g["pid_depth"], atol=1e-12):
        failed.append("hand_weighted")

    g = json.load(open(os.path.join(GOLDEN, "hand_binary_empty_3x4.json")))
    got = pid(np.array(g["U"], np.float64))
    if not np.allclose(got[2], g["pid_depth"], atol=1e-12):
        failed.append("hand_binary_empty")

    c = np.array([0.2, 0.9, 0.5, 0.7, 0.05])
    U = np.repeat(c[:, None], 9, axis=1)
    got = pid(U, np.linspace(0.5, 3, 9))
    if not (np.allclose(got[0], c.mean()) and np.allclose(got[1], c)):
        failed.append("constant_masks")

    radii = [4, 7, 10, 13, 16]
    U = synth.nested_disks(radii, 40, 40).astype(np.float64)
    area, N = U.sum(1), len(radii)
    in_in = [((N - k) + sum(area[j] / area[k] for j in range(k))) / N for k in range(N)]
    got = pid(U)
    if not np.allclose(got[0], in_in):
        failed.append("nested_disks")

    rng = np.random.default_rng(0)
    U = rng.uniform(0, 1, (5, 20))
    w = rng.uniform(0.5, 2, 20)
    a = pid(U, w)
    b = pid(np.repeat(U, 2, axis=1), np.repeat(w / 2, 2))
    c2 = pid(np.repeat(U, 3, axis=1))
    d = pid(U)
    if not np.allclose(a[2], b[2]) or np.allclose(a[2], d[2]) and not np.allclose(c2[2], d[2]):
        failed.append("cell_splitting")
    return failed


def test_real_oracle_passes_the_checks():
    assert _pin_checks(O.pid) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_mutant_is_caught(name):
    assert _pin_checks(MUTANTS[name]), f"mutant {name} slipped through every pin"


def test_pid_mean_mutants_are_caught():
    g = json.load(open(os.path.join(GOLDEN, "hand_weighted_2x3.json")))
    U, w = np.array(g["U"]), np.array(g["w"])

    def sum_not_mean(U, w):  # u_bar without the 1/N of Eq. 15
        ub = U.sum(0)
        a = np.array([O.inclusion(u, ub, w) for u in U])
        b = np.array([O.inclusion(ub, u, w) for u in U])
        return a, b, np.minimum(a, b)

    def swapped(U, w):
        ub = U.mean(0)
        a = np.array([O.inclusion(ub, u, w) for u in U])
        b = np.array([O.inclusion(u, ub, w) for u in U])
        return a, b, np.minimum(a, b)

    for mut in (sum_not_mean, swapped):
        got = mut(U, w)
        assert not (np.allclose(got[0], g["mean_in_in"]) and np.allclose(got[1], g["mean_in_out"]))
