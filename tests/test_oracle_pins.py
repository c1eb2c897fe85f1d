"""Pins of the CPU oracle (Algorithm 1, Sec. 2) to facts outside the oracle itself.

Each test checks the oracle against something it cannot agree with by construction: a hand-worked
check-node update, the closed-form recurrence of the Eq. (1) example, exact max-product marginals
by enumeration on tree graphs, minimum-weight decoding by enumeration on loopy graphs, and exact
symmetries of min-sum.  A dropped syndrome sign, a wrong exclusion index, a transposed H, a
misplaced alpha or a wrong stop rule each fails at least one of them.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from helpers import (brute_force_min_marginals, csr, load_matrix, random_tree_pcm,
                     syndrome_dense)
from paper_2508_07879_gb300 import workloads as w

PRECISIONS = ["f64", "f32", "i16"]


def run(h, syn, prior, max_iter, alpha, precision="f64", early_stop=True):
    c = csr(h)
    return oracle.msa(c.row_ptr, c.col_idx, c.m, c.n, np.atleast_2d(syn), prior, max_iter, alpha,
                      precision, early_stop)


def llr(res, precision):
    return res["post"] / 256.0 if precision == "i16" else res["post"].astype(np.float64)


# ---------------------------------------------------------------------------------------------
# Hand-worked single check-node update (Alg. 1, CN step, syndrome bit 1)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", PRECISIONS)
def test_single_check_hand_example(precision):
    # One check over four variables, s = 1, q = gamma = [2, -3, 5, 1], alpha = 0.75.
    # r_n = (-1)^{s} * prod_{j != n} sign(q_j) * 0.75 * min_{j != n} |q_j|:
    #   n=0: others [-3, 5, 1] -> sign (-1)(-1) = +, min 1 -> +0.75
    #   n=1: others [ 2, 5, 1] -> sign (-1)(+1) = -, min 1 -> -0.75
    #   n=2: others [ 2,-3, 1] -> +, min 1 -> +0.75
    #   n=3: others [ 2,-3, 5] -> +, min 2 -> +1.5
    # After one iteration Q_n = gamma_n + r_n.  (Early stop off: the prior already meets s.)
    h = np.array([[1, 1, 1, 1]], dtype=np.uint8)
    gamma = np.array([2.0, -3.0, 5.0, 1.0])
    res = run(h, [1], gamma, 1, 0.75, precision, early_stop=False)
    r = llr(res, precision)[0] - gamma
    np.testing.assert_array_equal(r, [0.75, -0.75, 0.75, 1.5])
    if precision == "i16":   # fixed point: gamma_q = 256 gamma, |r| = floor(min * 24576 / 2^15)
        np.testing.assert_array_equal(res["post"][0], [512 + 192, -768 - 192, 1280 + 192, 256 + 384])


def test_single_check_syndrome_zero_flips_signs():
    h = np.array([[1, 1, 1, 1]], dtype=np.uint8)
    gamma = np.array([2.0, -3.0, 5.0, 1.0])
    res = run(h, [0], gamma, 1, 0.75, "f64", early_stop=False)
    np.testing.assert_array_equal(res["post"][0] - gamma, [-0.75, 0.75, -0.75, -1.5])


# ---------------------------------------------------------------------------------------------
# Eq. (1) example: closed-form recurrence
# ---------------------------------------------------------------------------------------------
def eq1_closed_form(k, gamma=Fraction(1), alpha=Fraction(3, 4)):
    """Q^(k) for H of Eq. (1), s = [1, 1, 0], uniform prior gamma.

    By the code's symmetry every check-to-variable magnitude at iteration k equals a_k, with
    a_1 = alpha*gamma and a_{k+1} = alpha*(gamma - a_k): each check's other inputs all carry
    gamma - a_k (one opposing message removed).  Checks 0 and 1 (s = 1) send -a_k, check 2 sends
    +a_k, so variables 0 and 3 (in checks 0 and 1) get Q = gamma - 2 a_k and the rest Q = gamma.
    """
    a = alpha * gamma
    for _ in range(k - 1):
        a = alpha * (gamma - a)
    q0 = gamma - 2 * a
    return [q0, gamma, gamma, q0, gamma, gamma]


def eq1_closed_form_fixed(k, gamma_q=256, alpha_q=24576):
    """The same recurrence in the 16-bit mode: a_{k+1} = floor((gamma_q - a_k) * alpha_q / 2^15)."""
    a = (gamma_q * alpha_q) >> 15
    for _ in range(k - 1):
        a = ((gamma_q - a) * alpha_q) >> 15
    q0 = gamma_q - 2 * a
    return [q0, gamma_q, gamma_q, q0, gamma_q, gamma_q]


def test_eq1_fixture_is_the_papers_matrix():
    h = load_matrix("eq1_pcm.txt")
    np.testing.assert_array_equal(h, w.eq1_pcm())
    assert (h.sum(axis=1) == 4).all() and (h.sum(axis=0) == 2).all()


@pytest.mark.parametrize("precision,kmax", [("f64", 20), ("f32", 10), ("i16", 30)])
def test_eq1_trace(precision, kmax):
    h = load_matrix("eq1_pcm.txt")
    e = np.array([1, 0, 0, 0, 0, 0])
    s = syndrome_dense(h, e)
    np.testing.assert_array_equal(s, [1, 1, 0])
    for k in range(1, kmax + 1):
        res = run(h, s, np.ones(6), k, 0.75, precision, early_stop=False)
        if precision == "i16":
            np.testing.assert_array_equal(res["post"][0], eq1_closed_form_fixed(k))
        else:
            np.testing.assert_array_equal(res["post"][0], [float(x) for x in eq1_closed_form(k)])
        q0 = res["post"][0][0]
        np.testing.assert_array_equal(res["err"][0], [int(q0 < 0), 0, 0, int(q0 < 0), 0, 0])
        assert res["ok"][0] == 0 and res["iters"][0] == k
    # the first four iterations are dyadic and short: all precisions agree exactly
    for k in range(1, 5):
        exact = [float(x) for x in eq1_closed_form(k)]
        np.testing.assert_array_equal(np.array(eq1_closed_form_fixed(k)) / 256.0, exact)


def test_eq1_with_early_stop_never_converges():
    h = load_matrix("eq1_pcm.txt")
    for precision in PRECISIONS:
        res = run(h, [1, 1, 0], np.ones(6), 25, 0.75, precision)
        assert res["ok"][0] == 0 and res["iters"][0] == 25


# ---------------------------------------------------------------------------------------------
# Tree graphs: min-sum with alpha = 1 is exact max-product
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(12))
def test_tree_codes_equal_bruteforce_max_product(seed):
    rng = np.random.default_rng(1000 + seed)
    h = random_tree_pcm(rng, n_checks=int(rng.integers(2, 6)), max_deg=4)
    n = h.shape[1]
    if n > 14:
        h = h[:, :14][:, h[:, :14].any(axis=0)]
        h = h[(h.sum(axis=1) >= 2)]
        n = h.shape[1]
    e = (rng.random(n) < 0.3).astype(np.uint8)
    s = syndrome_dense(h, e)
    gamma = rng.uniform(0.5, 3.0, n) * rng.choice([-1.0, 1.0], n, p=[0.2, 0.8])
    L, best, n_min, e_star = brute_force_min_marginals(h, s, gamma)
    iters = h.shape[0] + 2                       # more than the diameter (in checks) of the tree
    res = run(h, s, gamma, iters, 1.0, "f64", early_stop=False)
    np.testing.assert_allclose(res["post"][0], L, rtol=1e-12, atol=1e-12)
    if n_min == 1:
        np.testing.assert_array_equal(res["err"][0], e_star)
        assert res["ok"][0] == 1


@pytest.mark.parametrize("seed", range(6))
def test_tree_codes_fixed_point_exact_on_integer_llrs(seed):
    # gamma on the 2^-8 grid and alpha = 1: the fixed-point mode is exact while nothing saturates
    rng = np.random.default_rng(2000 + seed)
    h = random_tree_pcm(rng, n_checks=4, max_deg=3)
    n = h.shape[1]
    gamma = rng.integers(-200, 800, n) / 256.0
    e = (rng.random(n) < 0.3).astype(np.uint8)
    s = syndrome_dense(h, e)
    L, *_ = brute_force_min_marginals(h, s, gamma)
    res = run(h, s, gamma, h.shape[0] + 2, 1.0, "i16", early_stop=False)
    np.testing.assert_array_equal(res["post"][0] / 256.0, L)


# ---------------------------------------------------------------------------------------------
# Loopy tiny codes: any converged output satisfies H e = s and cannot beat the minimum weight
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", PRECISIONS)
def test_loopy_converged_outputs_vs_bruteforce(precision):
    code = w.bb_code(3, 3)          # 9 checks, 18 qubits: small enough to enumerate 2^18
    h = code.hz
    rng = np.random.default_rng(7)
    gamma = np.full(h.shape[1], w.prior_llr(0.1))
    from helpers import all_errors
    es = all_errors(h.shape[1])
    synd_all = syndrome_dense(h, es)
    weights = es.sum(axis=1)
    for _ in range(40):
        e = (rng.random(h.shape[1]) < 0.1).astype(np.uint8)
        s = syndrome_dense(h, e)
        res = run(h, s, gamma, 30, 0.75, precision)
        e_hat = res["err"][0]
        met = (syndrome_dense(h, e_hat) == s).all()
        assert res["ok"][0] == int(met)
        if met:
            feasible = (synd_all == s[None, :]).all(axis=1)
            assert e_hat.sum() >= weights[feasible].min()


# ---------------------------------------------------------------------------------------------
# Stop rule: iteration 0 test, first-success stop, ok <=> H e_hat = s
# ---------------------------------------------------------------------------------------------
def test_zero_syndrome_stops_before_first_iteration():
    code = w.hgp_code(400)
    h = code.hz
    for precision in PRECISIONS:
        res = run(h, np.zeros(h.shape[0], np.uint8), np.full(h.shape[1], 2.0), 10, 0.75, precision)
        assert res["iters"][0] == 0 and res["ok"][0] == 1 and not res["err"].any()


def test_max_iter_zero_returns_prior_decision():
    h = w.eq1_pcm()
    gamma = np.array([-1.0, 2, 3, -0.5, 1, 1])
    res = run(h, [1, 1, 0], gamma, 0, 0.75, "f64", early_stop=False)
    np.testing.assert_array_equal(res["err"][0], [1, 0, 0, 1, 0, 0])
    assert res["iters"][0] == 0
    assert res["ok"][0] == int((syndrome_dense(h, res["err"][0]) == [1, 1, 0]).all())


@pytest.mark.parametrize("precision", PRECISIONS)
def test_early_stop_is_first_success(precision):
    code = w.hgp_code(400)
    b = w.x_error_batch(code, 0.06, 60, seed=11)
    h = b.h
    full = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes, b.prior, 32, 0.75, precision)
    hz = h.dense()
    for i in range(len(full["iters"])):
        k = int(full["iters"][i])
        met = (syndrome_dense(hz, full["err"][i]) == b.syndromes[i]).all()
        assert full["ok"][i] == int(met)
        if full["ok"][i]:
            # no earlier iteration met the syndrome; iteration k's decisions equal the fixed run
            for kk in range(k):
                r = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes[i:i + 1], b.prior, kk,
                               0.75, precision, early_stop=False)
                assert r["ok"][0] == 0
            r = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes[i:i + 1], b.prior, k, 0.75,
                           precision, early_stop=False)
            np.testing.assert_array_equal(r["err"][0], full["err"][i])
            np.testing.assert_array_equal(r["post"][0], full["post"][i])
        else:
            assert k == 32


# ---------------------------------------------------------------------------------------------
# Exact symmetries of min-sum
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_positive_homogeneity(precision):
    # gamma -> 2 gamma scales every message by exactly 2 (power of two, no rounding change)
    code = w.lp_code(1054)
    b = w.x_error_batch(code, 0.04, 40, seed=5)
    h = b.h
    r1 = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes, b.prior, 50, 0.75, precision)
    r2 = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes, 2 * b.prior, 50, 0.75, precision)
    np.testing.assert_array_equal(r2["post"], 2 * r1["post"])
    np.testing.assert_array_equal(r2["err"], r1["err"])
    np.testing.assert_array_equal(r2["iters"], r1["iters"])


@pytest.mark.parametrize("precision", PRECISIONS)
def test_gauge_symmetry(precision):
    # decoding (s + H e0, gamma * (1 - 2 e0)) returns e_hat + e0 (negation is exact)
    code = w.hgp_code(400)
    b = w.x_error_batch(code, 0.05, 40, seed=9)
    h = b.h
    hz = h.dense()
    rng = np.random.default_rng(3)
    base = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes, b.prior, 32, 0.75, precision)
    for i in range(len(b.errors)):
        if base["margin"][i] == 0:
            continue            # exact zeros break the sign symmetry (sign(0) = +1 both ways)
        e0 = (rng.random(h.n) < 0.5).astype(np.uint8)
        s2 = (b.syndromes[i] + syndrome_dense(hz, e0)) % 2
        g2 = b.prior * (1 - 2 * e0.astype(np.float32))
        r = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s2[None, :], g2, 32, 0.75, precision)
        np.testing.assert_array_equal(r["err"][0], base["err"][i] ^ e0)
        assert r["iters"][0] == base["iters"][i] and r["ok"][0] == base["ok"][i]
        sign = 1 - 2 * e0.astype(np.int64)
        np.testing.assert_array_equal(r["post"][0], base["post"][i] * sign)


def test_permutation_invariance_fixed_point():
    # relabelling checks and variables permutes the outputs; integer sums make it exact
    code = w.lp_code(1054)
    b = w.x_error_batch(code, 0.04, 30, seed=21)
    hz = b.h.dense()
    rng = np.random.default_rng(5)
    pr, pc = rng.permutation(hz.shape[0]), rng.permutation(hz.shape[1])
    hp = hz[pr][:, pc]
    cp = csr(hp)
    base = oracle.msa(b.h.row_ptr, b.h.col_idx, b.h.m, b.h.n, b.syndromes, b.prior, 50, 0.75, "i16")
    perm = oracle.msa(cp.row_ptr, cp.col_idx, cp.m, cp.n, b.syndromes[:, pr], b.prior[pc], 50,
                      0.75, "i16")
    np.testing.assert_array_equal(perm["err"], base["err"][:, pc])
    np.testing.assert_array_equal(perm["post"], base["post"][:, pc])
    np.testing.assert_array_equal(perm["iters"], base["iters"])


def test_permutation_invariance_fp64_close():
    code = w.hgp_code(400)
    b = w.x_error_batch(code, 0.05, 30, seed=22)
    hz = b.h.dense()
    rng = np.random.default_rng(6)
    pr, pc = rng.permutation(hz.shape[0]), rng.permutation(hz.shape[1])
    cp = csr(hz[pr][:, pc])
    base = oracle.msa(b.h.row_ptr, b.h.col_idx, b.h.m, b.h.n, b.syndromes, b.prior, 32, 0.75, "f64")
    perm = oracle.msa(cp.row_ptr, cp.col_idx, cp.m, cp.n, b.syndromes[:, pr], b.prior[pc], 32, 0.75, "f64")
    keep = base["margin"] > 1e-6
    np.testing.assert_array_equal(perm["err"][keep], base["err"][keep][:, pc])
    np.testing.assert_allclose(perm["post"][keep], base["post"][keep][:, pc], rtol=1e-9, atol=1e-9)


# ---------------------------------------------------------------------------------------------
# Precision modes agree in distribution
# ---------------------------------------------------------------------------------------------
def test_fixed_point_tracks_fp64_decisions():
    code = w.hgp_code(400)
    b = w.x_error_batch(code, 0.05, 300, seed=1)
    h = b.h
    r64 = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes, b.prior, 32, 0.75, "f64", threads=4)
    r16 = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes, b.prior, 32, 0.75, "i16", threads=4)
    same = (r64["err"] == r16["err"]).all(axis=1)
    conv = r64["ok"] == 1
    assert conv.sum() > 100
    assert same[conv].mean() > 0.95          # converged shots: the same estimate
    assert abs(int(r64["ok"].sum()) - int(r16["ok"].sum())) <= 15


def test_alpha_fixed_point_scale():
    assert oracle.alpha_q(0.75) == 24576
    assert oracle.alpha_q(1.0) == 32768
    assert oracle.alpha_q(1.5) == -1 and oracle.alpha_q(0.0) == -1


def test_rejects_malformed_graph():
    with pytest.raises(ValueError):
        oracle.msa(np.array([0, 2]), np.array([0, 5]), 1, 3, np.zeros((1, 1)), np.ones(3), 5, 0.75)
