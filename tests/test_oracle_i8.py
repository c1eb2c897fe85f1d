"""Pins of the oracle's 8-bit fixed-point mode (i8: 2 fractional bits, messages within +-127).

The paper names 8-bit integer LLRs as an option without a quantization scheme; i8 is the reading
used here (the i16 mode with 2 fractional bits and a +-127 clamp).  Pinned by hand-worked updates
(including the clamp), the Eq. (1) closed-form recurrence on the quarter grid, tree codes that are
exact on the quarter grid while nothing saturates, and the layered schedule's agreement with
flooding where the schedule cannot matter.
"""
import numpy as np
import pytest

import oracle
from helpers import brute_force_min_marginals, csr, load_matrix, random_tree_pcm, syndrome_dense
from paper_2508_07879_gb300 import workloads as w
from test_oracle_pins import eq1_closed_form, eq1_closed_form_fixed


def run(h, syn, prior, max_iter, alpha, precision="i8", early_stop=True, schedule="flooding"):
    c = csr(h)
    return oracle.msa(c.row_ptr, c.col_idx, c.m, c.n, np.atleast_2d(syn), prior, max_iter, alpha, precision,
                      early_stop, schedule=schedule)


@pytest.mark.parametrize("schedule", ["flooding", "layered"])
def test_single_check_hand_example(schedule):
    # gamma = [2, -3, 5, 1] -> q = 4 gamma = [8, -12, 20, 4]; s = 1, alpha_q = 24576:
    # |r| = floor(min_others * 24576 / 2^15) = [3, 3, 3, 6], signs [+, -, +, +]
    h = np.ones((1, 4), dtype=np.uint8)
    res = run(h, [1], np.array([2.0, -3.0, 5.0, 1.0]), 1, 0.75, early_stop=False, schedule=schedule)
    np.testing.assert_array_equal(res["post"][0], [8 + 3, -12 - 3, 20 + 3, 4 + 6])


def test_prior_and_message_clamp():
    # prior 40 -> 160 clamps to 127; a prior decision needs no iteration
    h = np.ones((1, 3), dtype=np.uint8)
    res = run(h, [0], np.array([40.0, -40.0, 1.0]), 0, 0.75)
    np.testing.assert_array_equal(res["post"][0], [127, -127, 4])
    # chain c0 = {0,1}, c1 = {1,2}, gamma = 31 (124), s = 0, alpha = 1 (worked by hand):
    # iteration 1: every r = 124; q_{c0,1} = q_{c1,1} = clamp(124 + 124) = 127
    # iteration 2: r_{c0->0} = r_{c1->2} = 127, r_{c0->1} = r_{c1->1} = 124 -> Q = [251, 372, 251]
    h = np.array([[1, 1, 0], [0, 1, 1]], dtype=np.uint8)
    one = run(h, [0, 0], np.full(3, 31.0), 1, 1.0, early_stop=False)
    np.testing.assert_array_equal(one["post"][0], [248, 372, 248])
    two = run(h, [0, 0], np.full(3, 31.0), 2, 1.0, early_stop=False)
    np.testing.assert_array_equal(two["post"][0], [251, 372, 251])


def test_eq1_trace_on_the_quarter_grid():
    h = load_matrix("eq1_pcm.txt")
    s = syndrome_dense(h, np.array([1, 0, 0, 0, 0, 0]))
    for k in range(1, 25):
        res = run(h, s, np.ones(6), k, 0.75, early_stop=False)
        np.testing.assert_array_equal(res["post"][0], eq1_closed_form_fixed(k, gamma_q=4))
    # while the recurrence stays on the quarter grid the fixed point equals the exact value
    np.testing.assert_array_equal(np.array(eq1_closed_form_fixed(1, gamma_q=4)) / 4.0,
                                  [float(x) for x in eq1_closed_form(1)])


@pytest.mark.parametrize("seed", range(8))
def test_tree_codes_exact_on_quarter_grid(seed):
    rng = np.random.default_rng(3000 + seed)
    h = random_tree_pcm(rng, n_checks=3, max_deg=3)
    n = h.shape[1]
    gamma = rng.integers(-6, 20, n) / 4.0
    e = (rng.random(n) < 0.3).astype(np.uint8)
    s = syndrome_dense(h, e)
    L, *_ = brute_force_min_marginals(h, s, gamma)
    for schedule in ("flooding", "layered"):
        res = run(h, s, gamma, 2 * h.shape[0] + 2, 1.0, early_stop=False, schedule=schedule)
        np.testing.assert_array_equal(res["post"][0] / 4.0, L)


def test_i8_decodes_like_f64_on_most_converged_shots():
    code = w.lp_code(1054)
    h = code.hz_csr
    e = w.iid_x_errors(h.n, 0.03, 300, seed=17)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.03))
    a = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, 50, 0.75, "i8", threads=8)
    b = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, 50, 0.75, "f64", threads=8)
    both = (a["ok"] == 1) & (b["ok"] == 1)
    assert both.mean() > 0.9
    same = (a["err"][both] == b["err"][both]).all(axis=1)
    assert same.mean() > 0.95
