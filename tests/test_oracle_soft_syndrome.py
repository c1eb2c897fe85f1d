"""Soft-syndrome decoding: Algorithm 1 (Sec. 2) on the data-syndrome Tanner graph [H | I_m].

A syndrome bit read with error probability q becomes a degree-1 variable of its check with prior
LLR ln((1 - q)/q); the measured bits s~ = H e + e' are the syndrome of (e, e') on that graph.  The
decoder itself is unchanged, so these tests pin the construction, not new arithmetic:
  * infinitely reliable syndrome bits reproduce the hard-syndrome decoder on H exactly;
  * on tree codes the augmented graph is still a tree, and the a-posteriori LLRs of data and
    syndrome bits equal brute-force max-product marginals over (e, e');
  * a lone syndrome read error is explained as one, not as data errors.
"""
import numpy as np
import pytest

import oracle
from helpers import brute_force_min_marginals, csr, random_tree_pcm, syndrome_dense
from paper_2508_07879_gb300 import workloads as w


def run(h, syn, prior, max_iter, alpha, precision="f64", early_stop=True):
    return oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, np.atleast_2d(syn), prior, max_iter, alpha, precision,
                      early_stop)


def test_data_syndrome_graph():
    h = w.lp_code(1054).hz_csr
    a = w.data_syndrome_csr(h)
    d, da = h.dense(), a.dense()
    assert a.m == h.m and a.n == h.n + h.m
    np.testing.assert_array_equal(da[:, :h.n], d)
    np.testing.assert_array_equal(da[:, h.n:], np.eye(h.m, dtype=np.uint8))
    e, es, s = w.noisy_syndrome_batch(h, 0.03, 0.01, 64, seed=9)
    np.testing.assert_array_equal(s, w.syndromes(a, np.concatenate([e, es], axis=1)))
    assert es.any() and (s != w.syndromes(h, e)).any()


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_reliable_syndrome_bits_reproduce_the_hard_decoder(precision):
    h = w.lp_code(1054).hz_csr
    a = w.data_syndrome_csr(h)
    e, es, s = w.noisy_syndrome_batch(h, 0.03, 0.02, 40, seed=4)
    gamma = np.full(h.n, w.prior_llr(0.03))
    hard = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, gamma, 30, 0.75, precision, threads=8)
    soft = oracle.msa(a.row_ptr, a.col_idx, a.m, a.n, s, np.concatenate([gamma, np.full(h.m, 1e30)]), 30, 0.75,
                      precision, threads=8)
    np.testing.assert_array_equal(soft["err"][:, :h.n], hard["err"])
    assert not soft["err"][:, h.n:].any()
    np.testing.assert_array_equal(soft["iters"], hard["iters"])
    np.testing.assert_array_equal(soft["ok"], hard["ok"])
    np.testing.assert_array_equal(soft["post"][:, :h.n], hard["post"])


@pytest.mark.parametrize("seed", range(8))
def test_tree_codes_match_brute_force_marginals(seed):
    rng = np.random.default_rng(500 + seed)
    hd = random_tree_pcm(rng, n_checks=3, max_deg=3)
    m, n = hd.shape
    ad = np.concatenate([hd, np.eye(m, dtype=np.uint8)], axis=1)   # still a tree: one leaf per check
    gamma = np.concatenate([rng.uniform(0.5, 3.0, n), rng.uniform(0.3, 2.5, m)])
    e = (rng.random(n + m) < 0.3).astype(np.uint8)
    s = syndrome_dense(ad, e)
    L, *_ = brute_force_min_marginals(ad, s, gamma)
    res = run(csr(ad), s, gamma, 2 * m + 2, 1.0, early_stop=False)
    np.testing.assert_allclose(res["post"][0], L, rtol=1e-12, atol=1e-12)


def test_lone_read_error_is_explained_as_one():
    h = w.lp_code(1054).hz_csr
    a = w.data_syndrome_csr(h)
    gamma = np.full(h.n, w.prior_llr(0.03))
    lam = np.full(h.m, w.prior_llr(0.01))
    for i in (0, 100, 464):
        s = np.zeros((1, h.m), np.uint8)
        s[0, i] = 1                                  # no data error, one misread bit
        res = run(a, s, np.concatenate([gamma, lam]), 30, 0.75)
        assert res["ok"][0] == 1
        assert not res["err"][0, :h.n].any()
        np.testing.assert_array_equal(np.nonzero(res["err"][0, h.n:])[0], [i])
        hard = run(h, s, gamma, 30, 0.75)         # the hard decoder must invent data errors
        assert hard["err"][0].any() or hard["ok"][0] == 0
