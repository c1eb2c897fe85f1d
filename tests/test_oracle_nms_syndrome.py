"""Pins of the oracle's syndrome loss for the neural min-sum decoder (loss="syndrome").

The unrolled decoder is scored on the soft syndrome: with independent bits of P(e_n = 1) =
sigma(-Q_n), P_m is the probability that row m's parity equals s_m, and the loss is the mean over
checks (and iterations, weighted by lambda_t) of -log P_m.  Nothing here compares the oracle with
itself:
  * P_m by brute force: the probability of every one of the 2^d bit patterns of a row, summed over
    the patterns of parity s_m, from the a-posteriori LLRs the oracle reports;
  * the loss ignores the sampled error and is unchanged by a stabilizer-equivalent target;
  * the reverse-mode gradient equals central finite differences of the forward loss;
  * one check: the loss and its gradient in closed form from the definition of sigma.
"""
import itertools

import numpy as np
import pytest

import oracle
from helpers import csr, random_tree_pcm, syndrome_dense
from paper_2508_07879_gb300 import workloads as w


def train(c, syn, y, prior, weights, **kw):
    return oracle.nms_train(c.row_ptr, c.col_idx, c.m, c.n, syn, y, prior, weights, loss="syndrome", **kw)


def parity_prob_brute_force(q_row, s_bit):
    """P(parity of independent bits = s_bit) with P(bit = 1) = sigma(-Q), by enumeration."""
    p1 = 1.0 / (1.0 + np.exp(q_row))                 # sigma(-Q)
    total = 0.0
    for bits in itertools.product((0, 1), repeat=len(q_row)):
        if sum(bits) % 2 != s_bit:
            continue
        pr = 1.0
        for b, p in zip(bits, p1):
            pr *= p if b else 1.0 - p
        total += pr
    return total


@pytest.mark.parametrize("which", ["eq1", "tree", "regular"])
def test_loss_equals_brute_force_parity_probabilities(which):
    rng = np.random.default_rng(21)
    hd = {"eq1": w.eq1_pcm(), "tree": random_tree_pcm(rng, 4),
          "regular": w.random_regular_ldpc(6, 8, 3, 4, seed=9)}[which]
    c = csr(hd)
    T = 3
    prior = rng.uniform(0.3, 2.5, c.n) * rng.choice([1, 1, -1], c.n)
    weights = rng.uniform(0.5, 1.0, (T, c.nnz))
    e, s = (lambda e: (e, syndrome_dense(hd, e)))((rng.random((5, c.n)) < 0.3).astype(np.uint8))
    lam = rng.uniform(0.2, 1.0, T)
    out = train(c, s, e, prior, weights, post=True, loss_weights=lam)
    for b in range(5):
        want = 0.0
        for t in range(T):
            q = out["post"][b, t]
            terms = [-np.log(max(parity_prob_brute_force(q[c.col_idx[c.row_ptr[i]:c.row_ptr[i + 1]]], int(s[b, i])),
                                 1e-7)) for i in range(c.m)]
            want += lam[t] * np.mean(terms)
        np.testing.assert_allclose(out["loss"][b], want, rtol=1e-12)


def test_loss_ignores_the_sampled_error():
    code = w.bb_code(12, 6)
    c = code.hz_csr
    rng = np.random.default_rng(4)
    T = 4
    e = w.iid_x_errors(c.n, 0.05, 6, seed=3)
    s = w.syndromes(c, e)
    prior = np.full(c.n, w.prior_llr(0.05))
    weights = rng.uniform(0.6, 0.9, (T, c.nnz))
    a = train(c, s, e, prior, weights)["loss"]
    b = train(c, s, np.zeros_like(e), prior, weights)["loss"]
    np.testing.assert_array_equal(a, b)
    # a stabilizer-equivalent error (e + a row of H_X) has the same syndrome and the same loss,
    # while the error loss tells the two apart
    e2 = e ^ code.hx_csr.dense()[0][None, :]
    np.testing.assert_array_equal(w.syndromes(c, e2), s)
    np.testing.assert_array_equal(train(c, s, e2, prior, weights)["loss"], a)
    err = oracle.nms_train(c.row_ptr, c.col_idx, c.m, c.n, s, e, prior, weights)["loss"]
    err2 = oracle.nms_train(c.row_ptr, c.col_idx, c.m, c.n, s, e2, prior, weights)["loss"]
    assert not np.allclose(err, err2)


def test_single_check_closed_form():
    """One check of degree 3, T = 1, weights w: r_j = (-1)^s sign-product * w_j * min of the other
    two magnitudes, Q_j = gamma_j + r_j; loss = -log P, P = (1 + (-1)^s prod tanh(Q_j/2)) / 2."""
    hd = np.ones((1, 3), dtype=np.uint8)
    c = csr(hd)
    gamma = np.array([1.5, -0.7, 2.2])
    wts = np.array([[0.8, 0.6, 0.9]])
    for s_bit in (0, 1):
        out = train(c, np.array([[s_bit]], np.uint8), np.zeros((1, 3), np.uint8), gamma, wts, grad_loss=np.ones(1),
                    post=True)
        sg = -1.0 if s_bit else 1.0
        r = np.empty(3)
        for j in range(3):
            o = [k for k in range(3) if k != j]
            r[j] = sg * np.prod(np.sign(gamma[o])) * wts[0, j] * np.abs(gamma[o]).min()
        Q = gamma + r
        np.testing.assert_allclose(out["post"][0, 0], Q, rtol=1e-15)
        P = 0.5 * (1 + sg * np.prod(np.tanh(Q / 2)))
        np.testing.assert_allclose(out["loss"][0], -np.log(P), rtol=1e-12)
        # d loss / d w_j = d loss / d Q_j * d r_j / d w_j (r_j enters only Q_j at T = 1)
        dQ = np.array([-(1 / P) * 0.5 * sg * np.prod(np.tanh(np.delete(Q, j) / 2)) * 0.5 * (1 - np.tanh(Q[j] / 2) ** 2)
                       for j in range(3)])
        np.testing.assert_allclose(out["grad"][0], dQ * r / wts[0], rtol=1e-10)


def finite_difference(c, s, e, prior, weights, entries, eps=1e-6, lam=None):
    fd = []
    for t, k in entries:
        wp, wm = weights.copy(), weights.copy()
        wp[t, k] += eps
        wm[t, k] -= eps
        lp = train(c, s, e, prior, wp, loss_weights=lam)["loss"].sum()
        lm = train(c, s, e, prior, wm, loss_weights=lam)["loss"].sum()
        fd.append((lp - lm) / (2 * eps))
    return np.array(fd)


@pytest.mark.parametrize("which", ["eq1", "tree", "regular"])
def test_gradient_equals_finite_differences_everywhere(which):
    rng = np.random.default_rng(17)
    hd = {"eq1": w.eq1_pcm(), "tree": random_tree_pcm(rng, 5),
          "regular": w.random_regular_ldpc(6, 8, 3, 4, seed=5)}[which]
    c = csr(hd)
    T = 4
    prior = rng.uniform(0.4, 3.0, c.n) * rng.choice([1, 1, 1, -1], c.n)   # distinct magnitudes: no ties
    weights = rng.uniform(0.4, 1.1, (T, c.nnz))
    e = (rng.random((6, c.n)) < 0.25).astype(np.uint8)
    s = syndrome_dense(hd, e)
    g = rng.uniform(0.5, 2.0, 6)
    lam = None if which != "regular" else rng.uniform(0.0, 1.0, T)
    out = train(c, s, e, prior, weights, grad_loss=g, loss_weights=lam)
    entries = [(t, k) for t in range(T) for k in range(c.nnz)]
    fd = np.zeros(len(entries))
    for b in range(6):
        fd += g[b] * finite_difference(c, s[b:b + 1], e[b:b + 1], prior, weights, entries, lam=lam)
    np.testing.assert_allclose(out["grad"].reshape(-1), fd, rtol=1e-6, atol=1e-8)
    assert np.abs(out["grad"]).max() > 1e-3


def test_gradient_equals_finite_differences_lp1054_sampled():
    h = w.lp_code(1054).hz_csr
    rng = np.random.default_rng(6)
    T = 5
    e = w.iid_x_errors(h.n, 0.04, 3, seed=78)
    s = w.syndromes(h, e)
    prior = w.prior_llr(0.04) * rng.uniform(0.8, 1.2, h.n)
    weights = rng.uniform(0.5, 1.0, (T, h.nnz))
    out = train(h, s, e, prior, weights, grad_loss=np.ones(3))
    flat = np.abs(out["grad"])
    entries = [(T - 1, int(np.argmax(flat[T - 1]))), (0, int(np.argmax(flat[0]))), (2, int(np.argmax(flat[2])))]
    entries += [(int(rng.integers(T)), int(rng.integers(h.nnz))) for _ in range(12)]
    fd = finite_difference(h, s, e, prior, weights, entries, eps=1e-6)
    got = np.array([out["grad"][t, k] for t, k in entries])
    np.testing.assert_allclose(got, fd, rtol=1e-5, atol=1e-10)
    assert np.abs(got[:3]).min() > 0


def test_f32_forward_matches_f64_and_rejects_unknown_loss():
    h = w.hgp_code(400).hz_csr
    rng = np.random.default_rng(2)
    e = w.iid_x_errors(h.n, 0.05, 4, seed=5)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.05))
    weights = rng.uniform(0.6, 0.9, (6, h.nnz))
    a = train(h, s, e, prior, weights, precision="f64")["loss"]
    b = train(h, s, e, prior, weights, precision="f32")["loss"]
    np.testing.assert_allclose(a, b, rtol=1e-5)
    with pytest.raises(KeyError):
        oracle.nms_train(h.row_ptr, h.col_idx, h.m, h.n, s, e, prior, weights, loss="other")
