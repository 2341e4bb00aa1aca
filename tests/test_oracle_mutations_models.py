"""The pins of the oracle's other routines catch plausible mistakes in them.

Each mutant is a deliberately broken version of one oracle routine (a non-strict
threshold, a floor for a ceiling, a reversed order, swapped flags, a dropped sqrt 2, a
wrong normalisation, groups or time steps ignored, blocks of the accumulated forms lost).
The oracle module's routine is replaced by the mutant and the routine's pin tests run
against it; at least one of them must fail, so a mistake of that kind in the real oracle
could not pass. CPU only.
"""
import math

import numpy as np
import pytest

from oracle import pid_oracle as O
from tests import test_oracle_pins as P

REAL = {name: getattr(O, name) for name in (
    "contour_bands", "iso_soft_mask", "iso_soft_mask_uniform", "level_soft_mask",
    "rank_by_depth", "pid_grouped", "spacetime_cells", "pid_mean_weighted", "pid_chunked",
    "pid_mean_chunked")}


# --- mutants ------------------------------------------------------------------------------

def _bands_swap_bits(U, rank, tau, inner_fraction=0.5):
    b = REAL["contour_bands"](U, rank, tau, inner_fraction)
    swap = ((b & 1) << 1) | ((b & 2) >> 1) | ((b & 4) << 1) | ((b & 8) >> 1)
    return (b & 16) | swap


def _bands_median_last(U, rank, tau, inner_fraction=0.5):
    b = REAL["contour_bands"](U, rank, tau, inner_fraction) & ~np.uint8(16)
    last = int(np.argmax(np.asarray(rank)))
    return b | ((np.atleast_2d(U)[last] > tau).astype(np.uint8) * 16)


def _bands_floor(U, rank, tau, inner_fraction=0.5):
    N = np.atleast_2d(U).shape[0]
    return REAL["contour_bands"](U, rank, tau, math.floor(inner_fraction * N) / N)


def _bands_deepest_is_last(U, rank, tau, inner_fraction=0.5):
    r = np.asarray(rank)
    return REAL["contour_bands"](U, r.max() - r, tau, inner_fraction)


def _iso_threshold_non_strict(F, mu, sigma, superlevel=False):
    if sigma == 0.0:
        F = np.asarray(F, np.float64)
        return (F >= mu).astype(np.float64) if superlevel else (F <= mu).astype(np.float64)
    return REAL["iso_soft_mask"](F, mu, sigma, superlevel)


def _rank_ties_to_higher_index(depth):
    d = np.asarray(depth, np.float64).reshape(-1)
    order = sorted(range(d.shape[0]), key=lambda i: (-d[i], -i))
    r = np.empty(d.shape[0], dtype=np.int32)
    for k, i in enumerate(order):
        r[i] = k
    return r


def _rank_ascending(depth):
    return REAL["rank_by_depth"](-np.asarray(depth, np.float64))


def _grouped_ignoring_groups(U, labels, w=None):
    a, b, d = O.pid(U, w)
    return a, b, d, O.rank_by_depth(d)


def _grouped_normalised_by_n(U, labels, w=None):
    a, b, d, r = REAL["pid_grouped"](U, labels, w)
    labels = np.asarray(labels).reshape(-1)
    size = np.array([np.count_nonzero(labels == g) for g in labels], np.float64)
    f = size / labels.shape[0]
    return a * f, b * f, np.minimum(a * f, b * f), r


def _grouped_global_rank(U, labels, w=None):
    a, b, d, _ = REAL["pid_grouped"](U, labels, w)
    return a, b, d, O.rank_by_depth(d)


def _spacetime_averaged(steps, w=None):
    U = np.mean([np.atleast_2d(np.asarray(S, np.float64)) for S in steps], axis=0)
    return U, (None if w is None else np.asarray(w, np.float64))


def _spacetime_first_step(steps, w=None):
    return np.atleast_2d(np.asarray(steps[0], np.float64)), (None if w is None else np.asarray(w, np.float64))


def _wmean_by_n(U, member_weights, w=None):
    U = np.atleast_2d(np.asarray(U, np.float64))
    r = np.asarray(member_weights, np.float64).reshape(-1)
    ubar = (r[:, None] * U).sum(axis=0) / U.shape[0]
    a = np.array([O.inclusion(u, ubar, w) for u in U])
    b = np.array([O.inclusion(ubar, u, w) for u in U])
    return a, b, np.minimum(a, b)


def _chunked_last_block_only(chunks):
    last = list(chunks)[-1:]
    return REAL["pid_chunked"](iter(last))


def _chunked_mass_of_first_block(chunks):
    chunks = list(chunks)
    a, b, d = REAL["pid_chunked"](iter(chunks))
    # the pairs' ratios formed with the first block's masses instead of the totals
    U0, w0 = chunks[0]
    m0 = np.atleast_2d(U0) @ O.cell_measure(np.atleast_2d(U0).shape[1], w0)
    m = sum(np.atleast_2d(Ub) @ O.cell_measure(np.atleast_2d(Ub).shape[1], wb) for Ub, wb in chunks)
    f = np.where(m0 > 0, m / np.where(m0 > 0, m0, 1.0), 0.0)
    return a * f, b, np.minimum(a * f, b)


def _mean_chunked_without_measures(chunks):
    # every sum over cells taken without the cell measures
    chunks = list(chunks)
    a, b, d = REAL["pid_mean_chunked"](iter([(Ub, None) for Ub, _ in chunks]))
    return a, b, d


def _mean_chunked_sum_not_mean(chunks):
    num, m, mbar = None, None, 0.0
    for Ub, wb in chunks:
        Ub = np.atleast_2d(np.asarray(Ub, np.float64))
        wb = O.cell_measure(Ub.shape[1], wb)
        ubar = Ub.sum(axis=0)                    # without the 1/N of Eq. 15
        num = (0 if num is None else num) + Ub @ (wb * ubar)
        m = (0 if m is None else m) + Ub @ wb
        mbar += float(wb @ ubar)
    a = np.where(m > 0, num / np.where(m > 0, m, 1.0), 0.0)
    b = num / mbar
    return a, b, np.minimum(a, b)


MUTANTS = {
    "pid_chunked": {
        "last_block_only": _chunked_last_block_only,
        "masses_of_the_first_block": _chunked_mass_of_first_block,
    },
    "pid_mean_chunked": {
        "cell_measures_dropped": _mean_chunked_without_measures,
        "sum_not_mean": _mean_chunked_sum_not_mean,
    },
    "contour_bands": {
        "non_strict_threshold": lambda U, rank, tau, f=0.5:
            REAL["contour_bands"](U, rank, np.nextafter(tau, -np.inf), f),
        "floor_inner_count": _bands_floor,
        "deepest_is_last_rank": _bands_deepest_is_last,
        "union_intersection_swapped": _bands_swap_bits,
        "median_is_last_rank": _bands_median_last,
    },
    "iso_soft_mask": {
        "sigma_without_sqrt2": lambda F, mu, s, sup=False:
            REAL["iso_soft_mask"](F, mu, s / math.sqrt(2.0), sup),
        "superlevel_ignored": lambda F, mu, s, sup=False: REAL["iso_soft_mask"](F, mu, s, False),
        "inside_is_the_superlevel_set": lambda F, mu, s, sup=False:
            REAL["iso_soft_mask"](F, mu, s, not sup),
        "threshold_non_strict": _iso_threshold_non_strict,
    },
    "iso_soft_mask_uniform": {
        "half_width_as_width": lambda F, mu, h, sup=False:
            REAL["iso_soft_mask_uniform"](F, mu, h / 2.0, sup),
        "no_clamp": lambda F, mu, h, sup=False:
            ((np.asarray(F, np.float64) - (mu - h)) if sup else (mu + h - np.asarray(F, np.float64)))
            / (2.0 * h),
    },
    "level_soft_mask": {
        "no_absolute_value": lambda F, level, h:
            np.maximum(0.0, 1.0 - (np.asarray(F, np.float64) - level) / h).clip(0.0, 1.0),
        "width_doubled": lambda F, level, h: REAL["level_soft_mask"](F, level, 2.0 * h),
    },
    "rank_by_depth": {
        "ties_to_higher_index": _rank_ties_to_higher_index,
        "ascending_depth": _rank_ascending,
    },
    "pid_grouped": {
        "groups_ignored": _grouped_ignoring_groups,
        "normalised_by_ensemble_size": _grouped_normalised_by_n,
        "ranked_over_the_ensemble": _grouped_global_rank,
    },
    "spacetime_cells": {
        "steps_averaged": _spacetime_averaged,
        "first_step_only": _spacetime_first_step,
    },
    "pid_mean_weighted": {
        "reliabilities_ignored": lambda U, r, w=None: O.pid_mean(U, w),
        "normalised_by_n": _wmean_by_n,
    },
}

# the pins that hold each routine
PINS = {
    "pid_chunked": [(P.test_chunked_forms_match_closed_forms_and_set_counts, ()),
                    (P.test_chunked_forms_do_not_depend_on_the_blocks, (0,)),
                    (P.test_chunked_forms_do_not_depend_on_the_blocks, (1,))],
    "pid_mean_chunked": [(P.test_chunked_forms_match_closed_forms_and_set_counts, ()),
                         (P.test_chunked_forms_do_not_depend_on_the_blocks, (0,)),
                         (P.test_chunked_forms_do_not_depend_on_the_blocks, (1,))],
    "contour_bands": [(P.test_bands_hand_example, ()), (P.test_bands_nesting_invariants, (0,)),
                      (P.test_bands_nesting_invariants, (1,)), (P.test_bands_nesting_invariants, (2,)),
                      (P.test_bands_of_nested_disks_are_the_extreme_disks, ())],
    "iso_soft_mask": [(P.test_iso_map_textbook_values, ()), (P.test_iso_map_sigma_zero_is_threshold, ())],
    "iso_soft_mask_uniform": [(P.test_uniform_isovalue_mask_closed_form, ())],
    "level_soft_mask": [(P.test_level_mask_closed_form, ())],
    "rank_by_depth": [(P.test_rank_matches_sorted_with_ties, ())],
    "pid_grouped": [(P.test_grouped_pid_special_cases, ()),
                    (P.test_grouped_pid_of_two_disk_families_is_each_familys_order, ())],
    "spacetime_cells": [(P.test_spacetime_binary_members_are_eid_over_space_time_cells, ()),
                        (P.test_spacetime_invariants, ())],
    "pid_mean_weighted": [(P.test_weighted_mean_contour_special_cases, ())],
}


def _failing_pins(name, fn, monkeypatch):
    failed = []
    with monkeypatch.context() as m:
        m.setattr(O, name, fn)
        for pin, args in PINS[name]:
            try:
                pin(*args)
            except Exception:     # an assertion, or a shape the mutant gets wrong
                failed.append(pin.__name__)
    return failed


@pytest.mark.parametrize("name", sorted(PINS))
def test_real_routines_pass_their_pins(name, monkeypatch):
    assert _failing_pins(name, REAL[name], monkeypatch) == []


@pytest.mark.parametrize("name,mutant", [(n, k) for n in sorted(MUTANTS) for k in sorted(MUTANTS[n])])
def test_each_mutant_is_caught(name, mutant, monkeypatch):
    assert _failing_pins(name, MUTANTS[name][mutant], monkeypatch), \
        f"mutant {mutant} of {name} slipped through every pin"
