"""Pins of the oracle's neural normalized min-sum (learned per-edge, per-iteration weights).

The learned decoder replaces the scale alpha of Algorithm 1 (Sec. 2) by a weight w[t][e]; it is
trained on the BCE of its soft outputs sigma(-Q).  Nothing here compares the oracle with itself:
  * constant weights w = alpha reduce every iteration to the plain decoder, pinned on its own;
  * one iteration on any code has a closed form, evaluated here with dense numpy arrays;
  * weights zero except one (t, e) switch on exactly one message, which pins the weight index;
  * the reverse-mode gradient equals central finite differences of the forward loss, and the
    one-check gradient has a closed form;
  * the learned decoder with constant weights is the plain decoder, and its fallback re-decodes
    exactly the unconverged shots with plain min-sum.
"""
import numpy as np
import pytest

import oracle
from helpers import csr, random_tree_pcm, syndrome_dense
from paper_2508_07879_gb300 import workloads as w


def softplus(x):
    return np.logaddexp(0.0, x)


def bce_of_posts(post, y):
    """Mean over iterations and variables of BCE(sigma(-Q), y) for Q of shape [B, T, n]."""
    yb = y[:, None, :].astype(np.float64)
    return (yb * softplus(post) + (1 - yb) * softplus(-post)).mean(axis=(1, 2))


def train(h, syn, y, prior, weights, **kw):
    c = csr(h) if isinstance(h, np.ndarray) else h
    return oracle.nms_train(c.row_ptr, c.col_idx, c.m, c.n, syn, y, prior, weights, **kw)


def sample(h, p, shots, seed):
    rng = np.random.default_rng(seed)
    e = (rng.random((shots, h.shape[1])) < p).astype(np.uint8)
    return e, syndrome_dense(h, e)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_constant_weights_reduce_to_plain_decoder(precision):
    code = w.hgp_code(400)
    h = code.hz_csr
    e = w.iid_x_errors(h.n, 0.05, 6, seed=31)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.05))
    T, alpha = 6, 0.75
    real = np.float64 if precision == "f64" else np.float32
    weights = np.full((T, h.nnz), real(alpha), dtype=real)
    out = train(h, s, e, prior, weights, precision=precision, post=True)
    for t in range(T):
        ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, t + 1, alpha, precision, early_stop=False)
        np.testing.assert_array_equal(out["post"][:, t, :], ref["post"])
    np.testing.assert_allclose(out["loss"], bce_of_posts(out["post"].astype(np.float64), e), rtol=1e-12)


def test_loss_weights_select_iterations():
    """lambda one-hot at iteration t: the loss is the mean BCE of the plain decoder's Q after t
    iterations (constant weights); a general lambda is the lambda-weighted sum of those."""
    code = w.hgp_code(400)
    h = code.hz_csr
    e = w.iid_x_errors(h.n, 0.05, 5, seed=12)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.05))
    T = 5
    weights = np.full((T, h.nnz), 0.75)
    per_iter = []
    for t in range(T):
        ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, t + 1, 0.75, "f64", early_stop=False)
        per_iter.append(bce_of_posts(ref["post"][:, None, :], e))
        lam = np.zeros(T)
        lam[t] = 1.0
        np.testing.assert_allclose(train(h, s, e, prior, weights, loss_weights=lam)["loss"], per_iter[-1],
                                   rtol=1e-12)
    lam = np.array([0.1, 0.0, 0.5, 0.2, 2.0])
    np.testing.assert_allclose(train(h, s, e, prior, weights, loss_weights=lam)["loss"],
                               np.sum([l * p for l, p in zip(lam, per_iter)], axis=0), rtol=1e-12)


def first_iteration_dense(hd, s, prior, w0):
    """Q after one iteration, straight from the definitions with dense arrays."""
    m, n = hd.shape
    Q = prior.astype(np.float64).copy()
    rows, cols = np.nonzero(hd)              # CSR edge order
    for e_id, (c, v) in enumerate(zip(rows, cols)):
        others = [j for j in np.nonzero(hd[c])[0] if j != v]
        sign = (-1) ** (int(s[c]) + sum(int(prior[j] < 0) for j in others))
        Q[v] += sign * w0[e_id] * min(abs(prior[j]) for j in others)
    return Q


@pytest.mark.parametrize("seed", range(4))
def test_first_iteration_closed_form(seed):
    rng = np.random.default_rng(seed)
    hd = w.random_regular_ldpc(12, 16, 3, 4, seed=100 + seed)
    c = csr(hd)
    prior = rng.normal(1.0, 1.5, c.n)
    weights = rng.uniform(0.2, 1.2, (1, c.nnz))
    e, s = sample(hd, 0.2, 5, seed)
    out = train(c, s, e, prior, weights, post=True)
    for b in range(5):
        np.testing.assert_allclose(out["post"][b, 0], first_iteration_dense(hd, s[b], prior, weights[0]),
                                   rtol=1e-13, atol=1e-13)


def test_single_weight_switches_on_single_message():
    """w = 0 except at (t*, e*): messages are zero before t*, so Q^(t*) differs from the prior only
    at the variable of e*, by the CN message of that one edge."""
    hd = w.random_regular_ldpc(12, 16, 3, 4, seed=7)
    c = csr(hd)
    rng = np.random.default_rng(3)
    prior = rng.normal(1.0, 1.0, c.n)
    e, s = sample(hd, 0.2, 3, 8)
    rows, cols = np.nonzero(hd)
    T = 4
    for t_star, e_star in ((0, 0), (2, 17), (3, c.nnz - 1)):
        weights = np.zeros((T, c.nnz))
        weights[t_star, e_star] = 0.9
        out = train(c, s, e, prior, weights, post=True)
        chk, var = rows[e_star], cols[e_star]
        others = [j for j in np.nonzero(hd[chk])[0] if j != var]
        for b in range(3):
            for t in range(t_star):
                np.testing.assert_array_equal(out["post"][b, t], prior)
            sign = (-1) ** (int(s[b, chk]) + sum(int(prior[j] < 0) for j in others))
            expect = prior.copy()
            expect[var] += sign * 0.9 * min(abs(prior[j]) for j in others)
            np.testing.assert_allclose(out["post"][b, t_star], expect, rtol=1e-15, atol=1e-15)


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
    rng = np.random.default_rng(11)
    if which == "eq1":
        hd = w.eq1_pcm()
    elif which == "tree":
        hd = random_tree_pcm(rng, 5)
    else:
        hd = w.random_regular_ldpc(6, 8, 3, 4, seed=5)
    c = csr(hd)
    T = 4
    prior = rng.uniform(0.4, 3.0, c.n) * rng.choice([1, 1, 1, -1], c.n)   # distinct magnitudes: no ties
    weights = rng.uniform(0.4, 1.1, (T, c.nnz))
    e, s = sample(hd, 0.25, 6, 12)
    g = rng.uniform(0.5, 2.0, 6)
    lam = None if which != "regular" else rng.uniform(0.0, 1.0, T)   # also non-uniform loss weights
    out = train(c, s, e, prior, weights, grad_loss=g, loss_weights=lam)
    entries = [(t, k) for t in range(T) for k in range(c.nnz)]
    fd = np.zeros(len(entries))
    for b in range(6):   # weight each shot's loss by g[b]
        fd += g[b] * finite_difference(c, s[b:b + 1], e[b:b + 1], prior, weights, entries, lam=lam)
    np.testing.assert_allclose(out["grad"].reshape(-1), fd, rtol=1e-6, atol=1e-8)
    assert np.abs(out["grad"]).max() > 1e-3


def test_gradient_equals_finite_differences_lp1054_sampled():
    code = w.lp_code(1054)
    h = code.hz_csr
    rng = np.random.default_rng(5)
    T = 5
    e = w.iid_x_errors(h.n, 0.04, 3, seed=77)
    s = w.syndromes(h, e)
    prior = w.prior_llr(0.04) * rng.uniform(0.8, 1.2, h.n)            # no exact ties
    weights = rng.uniform(0.5, 1.0, (T, h.nnz))
    out = train(h, s, e, prior, weights, grad_loss=np.ones(3))
    # the largest gradients of the last and the first iteration, plus random entries
    flat = np.abs(out["grad"])
    entries = [(T - 1, int(np.argmax(flat[T - 1]))), (0, int(np.argmax(flat[0]))), (2, int(np.argmax(flat[2])))]
    entries += [(int(rng.integers(T)), int(rng.integers(h.nnz))) for _ in range(12)]
    fd = finite_difference(h, s, e, prior, weights, entries, eps=1e-6)
    got = np.array([out["grad"][t, k] for t, k in entries])
    np.testing.assert_allclose(got, fd, rtol=1e-5, atol=1e-10)
    assert np.abs(got[:3]).min() > 0


def test_gradient_single_check_closed_form():
    """H = one check on d variables, T = 1: dL/dw_n = (y_n - sigma(-Q_n)) sgn_n mu_n / N."""
    d = 6
    hd = np.ones((1, d), dtype=np.uint8)
    c = csr(hd)
    rng = np.random.default_rng(2)
    prior = rng.uniform(0.5, 2.5, d) * np.array([1, -1, 1, 1, -1, 1])
    weights = rng.uniform(0.5, 1.0, (1, d))
    for s_bit, y in ((0, [0, 1, 0, 0, 1, 0]), (1, [1, 0, 0, 0, 0, 0])):
        y = np.array([y], dtype=np.uint8)
        out = train(c, np.array([[s_bit]], dtype=np.uint8), y, prior, weights, grad_loss=np.ones(1), post=True)
        for n in range(d):
            others = [j for j in range(d) if j != n]
            sgn = (-1) ** (s_bit + sum(int(prior[j] < 0) for j in others))
            mu = min(abs(prior[j]) for j in others)
            Q = prior[n] + sgn * weights[0, n] * mu
            assert out["post"][0, 0, n] == pytest.approx(Q, rel=1e-15)
            expect = (y[0, n] - 1.0 / (1.0 + np.exp(Q))) * sgn * mu / d
            assert out["grad"][0, n] == pytest.approx(expect, rel=1e-12)


def test_f32_forward_tracks_f64():
    code = w.hgp_code(400)
    h = code.hz_csr
    rng = np.random.default_rng(9)
    e = w.iid_x_errors(h.n, 0.05, 8, seed=41)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.05))
    weights = rng.uniform(0.6, 0.9, (8, h.nnz))
    a = train(h, s, e, prior, weights, grad_loss=np.full(8, 0.125), precision="f64")
    b = train(h, s, e, prior, weights.astype(np.float32), grad_loss=np.full(8, 0.125), precision="f32")
    np.testing.assert_allclose(b["loss"], a["loss"], rtol=1e-5)
    scale = np.abs(a["grad"]).max()
    assert np.abs(b["grad"] - a["grad"]).max() < 1e-3 * scale


def decode(h, s, prior, weights, max_iter_plain, alpha=0.75):
    return oracle.nms_decode(h.row_ptr, h.col_idx, h.m, h.n, s, prior, weights, max_iter_plain, alpha)


def test_learned_decode_with_constant_weights_is_plain_decode():
    code = w.lp_code(1054)
    h = code.hz_csr
    e = w.iid_x_errors(h.n, 0.06, 40, seed=3)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.06), dtype=np.float32)
    K, L = 12, 30
    weights = np.full((K, h.nnz), 0.75, dtype=np.float32)
    got = decode(h, s, prior, weights, L)
    short = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, K, 0.75, "f32")
    plain = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, L, 0.75, "f32")
    conv = short["ok"] == 1
    assert conv.any() and (~conv).any()
    np.testing.assert_array_equal(got["fallback"], (~conv).astype(np.uint8))
    np.testing.assert_array_equal(got["err"][conv], short["err"][conv])
    np.testing.assert_array_equal(got["iters"][conv], short["iters"][conv])
    np.testing.assert_array_equal(got["post"][conv], short["post"][conv])
    # unconverged shots: plain min-sum from the prior, its iterations added to the K learned ones
    np.testing.assert_array_equal(got["err"][~conv], plain["err"][~conv])
    np.testing.assert_array_equal(got["iters"][~conv], K + plain["iters"][~conv])
    np.testing.assert_array_equal(got["ok"], np.where(conv, 1, plain["ok"]))
    # no learned iterations at all: exactly the plain decoder
    none = decode(h, s, prior, np.zeros((0, h.nnz), dtype=np.float32), L)
    np.testing.assert_array_equal(none["err"], plain["err"])
    np.testing.assert_array_equal(none["iters"], plain["iters"])


def test_learned_decode_follows_training_forward():
    """With arbitrary weights, the decode's learned phase is the training forward stopped at the
    first iteration whose decisions meet the syndrome."""
    code = w.hgp_code(400)
    h = code.hz_csr
    rng = np.random.default_rng(4)
    e = w.iid_x_errors(h.n, 0.04, 30, seed=90)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.04), dtype=np.float32)
    T = 10
    weights = rng.uniform(0.5, 1.0, (T, h.nnz)).astype(np.float32)
    got = decode(h, s, prior, weights, 20)
    fwd = train(h, s, e, prior, weights, precision="f32", post=True)["post"]
    hd = h.dense()
    for b in range(30):
        if got["fallback"][b]:
            continue
        k = int(got["iters"][b])
        if k == 0:
            continue
        np.testing.assert_array_equal(got["post"][b], fwd[b, k - 1])
        for t in range(k - 1):   # no earlier iteration met the syndrome
            dec = (fwd[b, t] < 0).astype(np.uint8)
            assert (syndrome_dense(hd, dec) != s[b]).any()
        assert (syndrome_dense(hd, got["err"][b]) == s[b]).all()


def test_rejects_bad_arguments():
    hd = w.eq1_pcm()
    c = csr(hd)
    s = np.zeros((1, 3), dtype=np.uint8)
    y = np.zeros((1, 6), dtype=np.uint8)
    with pytest.raises(ValueError):
        train(c, s, y, np.ones(6), np.zeros((0, c.nnz)))
