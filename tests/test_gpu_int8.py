"""INT8 fixed-point decoding on the GPU (2 fractional bits, messages within +-127): bit-exact
against the oracle's i8 mode in the batch and single-shot kernels, the pair decode and the layered
schedule, including priors and sums that saturate."""
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


def check(q, h, s, prior, max_iter, kernel="auto", layered=False, early_stop=True, alpha=0.75):
    g = q.Graph.from_csr(h)
    if kernel != "auto":
        g.set_launch(kernel)
    st = torch.from_numpy(np.ascontiguousarray(s, dtype=np.uint8)).cuda()
    pt = torch.from_numpy(np.ascontiguousarray(prior, dtype=np.float32)).cuda()
    err, iters, ok, post = q.decode(g, st, pt, max_iter, alpha, "int8", early_stop, want_post=True, layered=layered)
    torch.cuda.synchronize()
    ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, max_iter, alpha, "i8", early_stop, threads=16,
                     schedule="layered" if layered else "flooding")
    np.testing.assert_array_equal(err.cpu().numpy(), ref["err"])
    np.testing.assert_array_equal(iters.cpu().numpy(), ref["iters"])
    np.testing.assert_array_equal(ok.cpu().numpy(), ref["ok"])
    np.testing.assert_array_equal(post.cpu().numpy(), (ref["post"] / 4.0).astype(np.float32))
    return ref


@pytest.mark.parametrize("kernel", ["batch", "latency"])
@pytest.mark.parametrize("code", ["lp1054", "hgp400", "bb288"])
def test_int8_flooding_bit_exact(q, kernel, code):
    c = w.CONFIG_CODES[code]()
    h = c.hz_csr
    s = np.concatenate([w.x_error_batch(c, p, 150, seed=900 + i).syndromes for i, p in enumerate((0.01, 0.03, 0.05))])
    prior = np.full(h.n, w.prior_llr(0.03), dtype=np.float32)
    ref = check(q, h, s, prior, 50, kernel)
    assert (ref["ok"] == 0).any() and (ref["iters"] > 3).any()


@pytest.mark.parametrize("code", ["lp1054", "hgp400"])
def test_int8_layered_bit_exact(q, code):
    c = w.CONFIG_CODES[code]()
    h = c.hz_csr
    e = w.iid_x_errors(h.n, 0.04, 400, seed=41)
    s = w.syndromes(h, e)
    check(q, h, s, np.full(h.n, w.prior_llr(0.04), dtype=np.float32), 50, layered=True)


def test_int8_saturation_and_paper_mode(q):
    h = w.hgp_code(400).hz_csr
    rng = np.random.default_rng(5)
    e = w.iid_x_errors(h.n, 0.05, 200, seed=6)
    s = w.syndromes(h, e)
    prior = rng.uniform(5.0, 45.0, h.n).astype(np.float32)     # many priors clamp to 127
    check(q, h, s, prior, 30)
    check(q, h, s, prior, 10, early_stop=False)
    check(q, h, s, prior, 10, kernel="latency", early_stop=False)


def test_int8_pair_equals_single_decodes(q):
    c = w.bb_code(12, 6)
    gz, gx = q.Graph.from_csr(c.hz_csr), q.Graph.from_csr(c.hx_csr)
    ex, ez = w.depolarizing_errors(c.n, 0.04, 300, seed=2)
    sx = torch.from_numpy(w.syndromes(c.hz_csr, ex)).cuda()
    sz = torch.from_numpy(w.syndromes(c.hx_csr, ez)).cuda()
    pr = torch.full((c.n,), w.prior_llr(2 * 0.04 / 3), device="cuda")
    (a, ia, oa, _), (b, ib, ob, _) = q.decode_pair(gz, gx, sx, sz, pr, pr, 64, precision="int8")
    ra = q.decode(gz, sx, pr, 64, precision="int8")
    rb = q.decode(gx, sz, pr, 64, precision="int8")
    assert torch.equal(a, ra[0]) and torch.equal(ia, ra[1]) and torch.equal(b, rb[0]) and torch.equal(ib, rb[1])


@pytest.mark.parametrize("dv", [8, 12])
def test_int8_pairs_at_large_column_degree(q, dv):
    """The two-shots-per-block INT8 kernel where its sums are largest: every column of degree dv and
    priors that saturate to 127, so a variable's sum reaches 127 (1 + dv).  Column degree 8 is the
    largest the half-precision lanes take (|sum| <= 1143, every integer exact in FP16); 12 runs the
    16-bit integer lanes."""
    rng = np.random.default_rng(70 + dv)
    m, n = 96, 128
    hd = np.zeros((m, n), dtype=np.uint8)
    for v in range(n):
        hd[rng.choice(m, dv, replace=False), v] = 1
    keep = hd.sum(axis=1) >= 2
    from helpers import csr
    h = csr(hd[keep])
    assert h.col_degrees().max() == dv
    e = (rng.random((301, n)) < 0.08).astype(np.uint8)
    s = w.syndromes(h, e)
    for prior in (np.full(n, 40.0, dtype=np.float32), rng.uniform(-45.0, 45.0, n).astype(np.float32)):
        ref = check(q, h, s, prior, 25, kernel="packed")
        if prior.min() > 0:   # saturated prior 127 plus dv messages of floor(127 * 0.75) = 95
            assert np.abs(ref["post"]).max() >= 127 + (dv - 1) * 95
        check(q, h, s, prior, 8, kernel="packed", early_stop=False)
        # alpha = 1: messages reach 127 themselves, and a sum 127 (1 + dv) (1143 at column degree 8)
        ref = check(q, h, s, prior, 12, kernel="packed", early_stop=False, alpha=1.0)
        if prior.min() > 0:
            assert np.abs(ref["post"]).max() >= 127 + (dv - 2) * 127
