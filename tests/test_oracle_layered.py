"""Pins of the oracle's layered (row-serial) min-sum schedule.

The layered schedule applies the check update of Algorithm 1 (Sec. 2) one check at a time, each
check reading the a-posteriori LLRs the checks before it already refreshed.  Pinned by:
  * codes whose variables each touch one check: the schedule cannot matter, so it equals flooding
    at every iteration (exact in fixed point);
  * tree codes with alpha = 1: the fixed point is exact max-product, equal to brute-force
    min-marginals;
  * reordering checks without reordering any two that share a variable leaves every result
    bit-identical (the property a parallel implementation of the schedule relies on), while
    reordering two that share one changes the trajectory;
  * loopy tiny codes: converged outputs meet the syndrome and weigh at least the brute-force minimum;
  * stop rule and positive homogeneity as for flooding.
"""
import numpy as np
import pytest

import oracle
from helpers import brute_force_min_marginals, csr, random_tree_pcm, syndrome_dense
from paper_2508_07879_gb300 import workloads as w


def run(h, syn, prior, max_iter, alpha, precision="f64", early_stop=True, schedule="layered"):
    c = csr(h) if isinstance(h, np.ndarray) else h
    return oracle.msa(c.row_ptr, c.col_idx, c.m, c.n, np.atleast_2d(syn), prior, max_iter, alpha, precision,
                      early_stop, schedule=schedule)


def llr(res, precision):
    return res["post"] / 256.0 if precision == "i16" else res["post"].astype(np.float64)


@pytest.mark.parametrize("precision", ["f64", "f32", "i16"])
def test_single_check_one_iteration_equals_flooding(precision):
    h = np.ones((1, 4), dtype=np.uint8)
    prior = np.array([2.0, -3.0, 5.0, 1.0])
    for s in (0, 1):
        a = run(h, [s], prior, 1, 0.75, precision, early_stop=False)
        b = run(h, [s], prior, 1, 0.75, precision, early_stop=False, schedule="flooding")
        np.testing.assert_array_equal(a["post"], b["post"])
    # hand example of the single-check update (s = 1): r = [0.75, -0.75, 0.75, 1.5]
    a = run(h, [1], prior, 1, 0.75, precision, early_stop=False)
    np.testing.assert_allclose(llr(a, precision)[0], prior + np.array([0.75, -0.75, 0.75, 1.5]))


@pytest.mark.parametrize("precision", ["f64", "f32", "i16"])
def test_two_check_hand_example(precision):
    """Checks c0 = {0, 1}, c1 = {1, 2}, gamma = [2, 3, 1], s = 0, alpha = 1 (worked by hand).
    Iteration 1, c0 first: q = (2, 3) -> r = (3, 2), Q = [5, 5, 1]; then c1 sees Q_1 = 5:
    q = (5, 1) -> r = (1, 5), Q = [5, 6, 6].  (c1 first would give [6, 6, 4].)
    Iteration 2: c0: q = (5-3, 6-2) = (2, 4) -> r = (4, 2), Q_0 = 6, Q_1 = 6; c1: q = (6-1, 6-5) =
    (5, 1) -> r = (1, 5): Q = [6, 6, 6], the exact max-product LLRs (errors 000 or 111)."""
    h = np.array([[1, 1, 0], [0, 1, 1]], dtype=np.uint8)
    gamma = np.array([2.0, 3.0, 1.0])
    one = run(h, [0, 0], gamma, 1, 1.0, precision, early_stop=False)
    np.testing.assert_array_equal(llr(one, precision)[0], [5.0, 6.0, 6.0])
    two = run(h, [0, 0], gamma, 2, 1.0, precision, early_stop=False)
    np.testing.assert_array_equal(llr(two, precision)[0], [6.0, 6.0, 6.0])


@pytest.mark.parametrize("precision,gamma,lim", [("i8", 31.0, 127), ("i16", 120.0, 32767)])
def test_fixed_point_clamp_feeds_only_the_check(precision, gamma, lim):
    """Chain c0 = {0, 1}, c1 = {1, 2}, s = 0, alpha = 1, every prior gamma_q = g (i8: 4 * 31 = 124,
    i16: 256 * 120 = 30720), worked by hand with the messages' clamp L (127, 32767) active.
    The a-posteriori LLR stays the exact sum gamma + sum r (Algorithm 1's APP step); only the
    check's input q = clamp(Q - r_old) is clamped.
    Iteration 1: c0: q = (g, g) -> r = (g, g), Q_0 = Q_1 = 2g; c1: q = (clamp(2g) = L, g) ->
    r = (g, L), Q_1 = 2g + g = 3g, Q_2 = g + L.
    Iteration 2: c0: q = (clamp(2g - g) = g, clamp(3g - g) = L) -> r = (L, g): Q_0 = 2g - g + L,
    Q_1 = 3g - g + g; c1: q = (clamp(3g - g) = L, clamp(g + L - L) = g) -> r = (g, L): Q_1 = 3g,
    Q_2 = g + L.  So Q = [g + L, 3g, g + L], what flooding gives on this chain, where rebuilding Q
    from the clamped q would cap the middle variable at L + g."""
    h = np.array([[1, 1, 0], [0, 1, 1]], dtype=np.uint8)
    g = int(gamma * (4 if precision == "i8" else 256))
    assert 2 * g > lim >= g
    one = run(h, [0, 0], np.full(3, gamma), 1, 1.0, precision, early_stop=False)
    np.testing.assert_array_equal(one["post"][0], [2 * g, 3 * g, g + lim])
    two = run(h, [0, 0], np.full(3, gamma), 2, 1.0, precision, early_stop=False)
    np.testing.assert_array_equal(two["post"][0], [g + lim, 3 * g, g + lim])
    flood = run(h, [0, 0], np.full(3, gamma), 2, 1.0, precision, early_stop=False, schedule="flooding")
    np.testing.assert_array_equal(two["post"][0], flood["post"][0])


def test_degree_one_variables_make_the_schedule_irrelevant():
    """Every variable in exactly one check: flooding and layered coincide at every iteration (i16:
    (Q - r) + r' is exact integer arithmetic)."""
    rng = np.random.default_rng(4)
    h = np.zeros((6, 24), dtype=np.uint8)
    perm = rng.permutation(24)
    for i in range(6):
        h[i, perm[4 * i:4 * i + 4]] = 1
    prior = rng.uniform(-2, 4, 24).astype(np.float32)
    e = (rng.random((20, 24)) < 0.2).astype(np.uint8)
    s = syndrome_dense(h, e)
    for k in (1, 2, 5):
        a = run(h, s, prior, k, 0.75, "i16", early_stop=False)
        b = run(h, s, prior, k, 0.75, "i16", early_stop=False, schedule="flooding")
        np.testing.assert_array_equal(a["post"], b["post"])
        np.testing.assert_array_equal(a["err"], b["err"])


@pytest.mark.parametrize("seed", range(6))
def test_tree_codes_reach_bruteforce_max_product(seed):
    rng = np.random.default_rng(2000 + seed)
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
    res = run(h, s, gamma, 2 * h.shape[0] + 2, 1.0, "f64", early_stop=False)
    np.testing.assert_allclose(res["post"][0], L, rtol=1e-12, atol=1e-12)
    if n_min == 1:
        np.testing.assert_array_equal(res["err"][0], e_star)


def asap_layers(h):
    """Layer of each check: one more than the largest layer of an earlier check sharing a variable."""
    last = np.full(h.shape[1], -1)
    layer = np.zeros(h.shape[0], dtype=int)
    for i in range(h.shape[0]):
        cols = np.nonzero(h[i])[0]
        layer[i] = last[cols].max() + 1
        last[cols] = layer[i]
    return layer


@pytest.mark.parametrize("precision", ["f32", "i16"])
def test_reordering_independent_checks_is_exact(precision):
    code = w.hgp_code(400)
    hd = code.hz_csr.dense()
    rng = np.random.default_rng(8)
    e = w.iid_x_errors(code.n, 0.06, 40, seed=12)
    s = syndrome_dense(hd, e)
    prior = np.full(code.n, w.prior_llr(0.05), dtype=np.float32)
    base = run(hd, s, prior, 25, 0.75, precision)
    layer = asap_layers(hd)
    # any order that sorts by layer keeps every pair of checks sharing a variable in place
    order = np.lexsort((rng.random(hd.shape[0]), layer))
    assert (order != np.arange(hd.shape[0])).any()
    other = run(hd[order], s[:, order], prior, 25, 0.75, precision)
    for k in ("err", "iters", "ok", "post"):
        np.testing.assert_array_equal(other[k], base[k])
    # swapping the first pair of checks that share a variable changes some trajectory
    for i in range(hd.shape[0] - 1):
        if (hd[i] & hd[i + 1]).any():
            break
    swap = np.arange(hd.shape[0])
    swap[[i, i + 1]] = swap[[i + 1, i]]
    moved = run(hd[swap], s[:, swap], prior, 3, 0.75, precision, early_stop=False)
    fixed = run(hd, s, prior, 3, 0.75, precision, early_stop=False)
    assert (moved["post"] != fixed["post"]).any()


@pytest.mark.parametrize("precision", ["f64", "i16"])
def test_loopy_converged_outputs_vs_bruteforce(precision):
    code = w.bb_code(3, 3)          # 9 checks, 18 qubits: small enough to enumerate 2^18
    h = code.hz
    rng = np.random.default_rng(7)
    gamma = np.full(h.shape[1], w.prior_llr(0.1))
    from helpers import all_errors
    es = all_errors(h.shape[1])
    synd_all = syndrome_dense(h, es)
    weights = es.sum(axis=1)
    converged = 0
    for _ in range(60):
        e = (rng.random(h.shape[1]) < 0.08).astype(np.uint8)
        s = syndrome_dense(h, e)
        res = run(h, s, gamma, 30, 0.75, precision)
        e_hat = res["err"][0]
        met = (syndrome_dense(h, e_hat) == s).all()
        assert res["ok"][0] == int(met)
        if met:
            converged += 1
            feasible = (synd_all == s[None, :]).all(axis=1)
            assert e_hat.sum() >= weights[feasible].min()
    assert converged >= 5


def test_stop_rule_and_homogeneity():
    code = w.lp_code(1054)
    h = code.hz_csr
    zero = np.zeros((1, h.m), dtype=np.uint8)
    res = run(h, zero, np.full(h.n, 3.0), 20, 0.75)
    assert res["iters"][0] == 0 and res["ok"][0] == 1
    e = w.iid_x_errors(h.n, 0.04, 30, seed=5)
    s = w.syndromes(h, e)
    a = run(h, s, np.full(h.n, 1.5), 12, 0.75, early_stop=False)
    b = run(h, s, np.full(h.n, 3.0), 12, 0.75, early_stop=False)
    np.testing.assert_array_equal(b["post"], 2 * a["post"])
    # early stop: the first iteration whose decisions meet the syndrome
    full = run(h, s, np.full(h.n, 3.0), 12, 0.75)
    for bidx in range(30):
        k = int(full["iters"][bidx])
        if full["ok"][bidx] and k > 1:
            prev = run(h, s[bidx:bidx + 1], np.full(h.n, 3.0), k - 1, 0.75, early_stop=False)
            assert (syndrome_dense(h.dense(), prev["err"]) != s[bidx]).any()


def test_layered_needs_fewer_iterations_than_flooding():
    code = w.lp_code(1054)
    h = code.hz_csr
    e = w.iid_x_errors(h.n, 0.04, 400, seed=77)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.04), dtype=np.float32)
    lay = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, 50, 0.75, "f32", threads=8, schedule="layered")
    fl = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, 50, 0.75, "f32", threads=8)
    both = (lay["ok"] == 1) & (fl["ok"] == 1)
    assert lay["iters"][both].mean() < 0.7 * fl["iters"][both].mean()
