"""Layered (row-serial) schedule on the GPU against the oracle: bit-exact in FP32 and INT16.

The kernel runs the checks of each layer in parallel and the layers in order; the oracle visits
the checks strictly one after another.  Equality of e_hat, iterations, ok and the a-posteriori
LLRs on every shot checks both the layering and the arithmetic.
"""
import numpy as np
import pytest

import oracle
from paper_2508_07879_gb300 import workloads as w

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    from paper_2508_07879_gb300 import build
    build.build()
    from paper_2508_07879_gb300 import qldpc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qldpc


def irregular_code(seed=3, m=60, n=120):
    rng = np.random.default_rng(seed)
    h = np.zeros((m, n), dtype=np.uint8)
    for i in range(m):
        h[i, rng.choice(n, size=int(rng.integers(3, 10)), replace=False)] = 1
    for v in np.nonzero(h.sum(0) == 0)[0]:
        h[rng.integers(m), v] = 1
    return w.csr_from_dense(h)


def device_layered(q, h, s, prior, max_iter, precision, early_stop=True):
    g = q.Graph.from_csr(h)
    st = torch.from_numpy(np.ascontiguousarray(s, dtype=np.uint8)).cuda()
    pt = torch.from_numpy(np.ascontiguousarray(prior, dtype=np.float32)).cuda()
    err, iters, ok, post = q.decode(g, st, pt, max_iter, 0.75, precision, early_stop, want_post=True, layered=True)
    torch.cuda.synchronize()
    return err.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy(), post.cpu().numpy()


def oracle_layered(h, s, prior, max_iter, precision, early_stop=True):
    prec = {"fp32": "f32", "int16": "i16", "int8": "i8"}[precision]
    return oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, max_iter, 0.75, prec, early_stop, threads=16,
                      schedule="layered")


def check_equal(q, h, s, prior, max_iter, precision, early_stop=True):
    err, iters, ok, post = device_layered(q, h, s, prior, max_iter, precision, early_stop)
    ref = oracle_layered(h, s, prior, max_iter, precision, early_stop)
    np.testing.assert_array_equal(err, ref["err"])
    np.testing.assert_array_equal(iters, ref["iters"])
    np.testing.assert_array_equal(ok, ref["ok"])
    want = ref["post"] / {"fp32": 1.0, "int16": 256.0, "int8": 4.0}[precision]
    np.testing.assert_array_equal(post, want.astype(np.float32))
    return iters, ok


@pytest.mark.parametrize("precision", ["fp32", "int16"])
def test_lp1054_mixed_rates(q, precision):
    h = w.lp_code(1054).hz_csr
    s = np.concatenate([w.x_error_batch(w.lp_code(1054), p, 400, seed=700 + i).syndromes
                        for i, p in enumerate((0.01, 0.02, 0.03, 0.04, 0.05))])
    prior = np.full(h.n, w.prior_llr(0.03), dtype=np.float32)
    iters, ok = check_equal(q, h, s, prior, 50, precision)
    assert (ok == 0).any() and (iters > 3).any()


@pytest.mark.parametrize("precision", ["fp32", "int16"])
@pytest.mark.parametrize("code", ["hgp400", "bb144", "bb288"])
def test_other_codes(q, precision, code):
    c = w.CONFIG_CODES[code]()
    for h in (c.hz_csr, c.hx_csr):
        e = w.iid_x_errors(h.n, 0.05, 500, seed=31)
        s = w.syndromes(h, e)
        prior = np.full(h.n, w.prior_llr(0.05), dtype=np.float32)
        check_equal(q, h, s, prior, 40, precision)


@pytest.mark.parametrize("precision", ["fp32", "int16"])
def test_irregular_and_paper_mode(q, precision):
    h = irregular_code()
    rng = np.random.default_rng(2)
    e = (rng.random((300, h.n)) < 0.06).astype(np.uint8)
    s = w.syndromes(h, e)
    prior = rng.uniform(1.0, 4.0, h.n).astype(np.float32)
    check_equal(q, h, s, prior, 30, precision)
    iters, _ = check_equal(q, h, s, prior, 10, precision, early_stop=False)
    assert (iters == 10).all()


def test_edge_cases(q):
    h = w.hgp_code(400).hz_csr
    g = q.Graph.from_csr(h)
    prior = np.full(h.n, 2.5, dtype=np.float32)
    e = w.iid_x_errors(h.n, 0.05, 20, seed=4)
    s = w.syndromes(h, e)
    check_equal(q, h, s, prior, 0, "fp32")                       # max_iter = 0: prior decision
    check_equal(q, h, np.zeros((5, h.m), np.uint8), prior, 20, "fp32")   # met before iteration 1
    st = torch.from_numpy(s).cuda()
    empty = torch.zeros((0, h.m), dtype=torch.uint8, device="cuda")
    err, iters, ok, _ = q.decode(g, empty, torch.from_numpy(prior).cuda(), 20, layered=True)
    assert err.shape == (0, h.n)
    bad = prior.copy()
    bad[7] = np.nan
    err, iters, ok, _ = q.decode(g, st, torch.from_numpy(bad).cuda(), 20, layered=True)
    assert (iters.cpu().numpy() == -1).all() and (ok.cpu().numpy() == 0).all()
    g.set_weights(np.full((4, h.nnz), 0.75, np.float32))
    with pytest.raises(q.QldpcError) as ei:
        q.decode(g, st, torch.from_numpy(prior).cuda(), 20, learned=True, layered=True)
    assert ei.value.status == q.QLDPC_ERR_INVALID_ARG


def test_pair_and_host_path(q):
    c = w.bb_code(12, 6)
    gz, gx = q.Graph.from_csr(c.hz_csr), q.Graph.from_csr(c.hx_csr)
    ex, ez = w.depolarizing_errors(c.n, 0.04, 200, seed=9)
    sx, sz = w.syndromes(c.hz_csr, ex), w.syndromes(c.hx_csr, ez)
    prior = np.full(c.n, w.prior_llr(2 * 0.04 / 3), dtype=np.float32)
    pt = torch.from_numpy(prior).cuda()
    (a, ia, oa, _), (b, ib, ob, _) = q.decode_pair(gz, gx, torch.from_numpy(sx).cuda(), torch.from_numpy(sz).cuda(),
                                                   pt, pt, 64, layered=True)
    ra = oracle_layered(c.hz_csr, sx, prior, 64, "fp32")
    rb = oracle_layered(c.hx_csr, sz, prior, 64, "fp32")
    np.testing.assert_array_equal(a.cpu().numpy(), ra["err"])
    np.testing.assert_array_equal(ib.cpu().numpy(), rb["iters"])
    np.testing.assert_array_equal(b.cpu().numpy(), rb["err"])
    # end-to-end host path (pageable and page-locked buffers)
    h = w.lp_code(1054).hz_csr
    g = q.Graph.from_csr(h)
    e = w.iid_x_errors(h.n, 0.04, 64, seed=3)
    s = w.syndromes(h, e)
    pr = np.full(h.n, w.prior_llr(0.04), dtype=np.float32)
    ref = oracle_layered(h, s, pr, 50, "fp32")
    err, iters, ok = q.decode_host(g, s, pr, 50, layered=True)
    np.testing.assert_array_equal(err, ref["err"])
    np.testing.assert_array_equal(iters, ref["iters"])
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    out = (pin(np.zeros((64, h.n), np.uint8)), pin(np.zeros(64, np.int32)), pin(np.zeros(64, np.uint8)))
    q.decode_host(g, pin(s), pr, 50, out=out, layered=True)
    np.testing.assert_array_equal(out[0], ref["err"])
    np.testing.assert_array_equal(out[1], ref["iters"])


def test_batch_invariance(q):
    h = w.lp_code(1054).hz_csr
    e = w.iid_x_errors(h.n, 0.05, 4096, seed=21)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.05), dtype=np.float32)
    full = device_layered(q, h, s, prior, 50, "fp32")
    for lo, hi in ((0, 1), (100, 164), (4000, 4096)):
        part = device_layered(q, h, s[lo:hi], prior, 50, "fp32")
        for a, b in zip(part, full):
            np.testing.assert_array_equal(a, b[lo:hi])


@pytest.mark.parametrize("precision", ["fp32", "int16", "int8"])
def test_single_shot_register_kernel(q, precision):
    """Batches no larger than the SM count run the register-resident layered kernel (LP-1054: 7
    layers of degree-8 rows): bit-exact against the oracle as well."""
    h = w.lp_code(1054).hz_csr
    e = w.iid_x_errors(h.n, 0.05, 100, seed=88)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.05), dtype=np.float32)
    iters, ok = check_equal(q, h, s, prior, 50, precision)
    assert (iters > 3).any()
    check_equal(q, h, s[:1], prior, 50, precision)
    check_equal(q, h, s[:7], prior, 12, precision, early_stop=False)


def block_layered_code(seed, degree=None, n=168, blocks=6):
    """Rows in `blocks` groups, each group a random partition of the columns into rows of `degree`
    (or of 8 with 0-5 entries then dropped per row: degrees 3..8).  Row order by group, so the
    as-soon-as-possible layering gives at most `blocks` layers: the register-resident regime."""
    rng = np.random.default_rng(seed)
    d = degree or 8
    rows = []
    for _ in range(blocks):
        for r in rng.permutation(n).reshape(n // d, d):
            rows.append(r if degree else r[:d - int(rng.integers(0, 6))])
    h = np.zeros((len(rows), n), dtype=np.uint8)
    for i, r in enumerate(rows):
        h[i, r] = 1
    return w.csr_from_dense(h)


@pytest.mark.parametrize("precision", ["fp32", "int16", "int8"])
@pytest.mark.parametrize("degree", [6, 7, None])
def test_single_shot_kernel_on_few_layer_codes(q, precision, degree):
    """Rows of exact degree 6 and 7 and of varying degree 3..8 in the register-resident kernel
    (six layers), where a check's edges do not fill its lanes evenly."""
    h = block_layered_code(40 + (degree or 0), degree)
    e = w.iid_x_errors(h.n, 0.06, 120, seed=89)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.06), dtype=np.float32)
    iters, ok = check_equal(q, h, s, prior, 30, precision)
    assert (iters > 2).any()
