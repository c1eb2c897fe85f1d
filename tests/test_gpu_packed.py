"""The two-shots-per-block kernel (QLDPC_KERNEL_PACKED; the default throughput kernel of INT16)
against the oracle, element by element: decisions, iterations, ok and a-posteriori LLRs, bit-exact,
in INT16 and INT8 (two 16-bit lanes per message word) and FP32 (float2 slots, paired additions).

The kernel decodes two shots per block and refills each lane with the next shot as soon as its own
shot stops, so the cases below mix shots that stop at very different iterations (met syndromes at
iteration 0 beside shots that run to the limit), odd batch sizes (a lane idle at the end), the pair
decode, paper mode, max_iter = 0, block sizes, a non-finite prior and codes of irregular degree."""
import numpy as np
import pytest

import oracle
from helpers import csr
from paper_2508_07879_gb300 import workloads as w

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
OPREC = {"int16": "i16", "int8": "i8", "fp32": "f32"}
SCALE = {"int16": 256.0, "int8": 4.0, "fp32": 1.0}


@pytest.fixture(scope="module")
def q():
    from paper_2508_07879_gb300 import build
    build.build()
    from paper_2508_07879_gb300 import qldpc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qldpc


def run_packed(q, g, s, prior, max_iter, precision, early_stop=True, threads=0):
    g.set_launch("packed", threads, 0)
    try:
        st = torch.from_numpy(np.ascontiguousarray(s, dtype=np.uint8)).cuda()
        pt = torch.from_numpy(np.ascontiguousarray(prior, dtype=np.float32)).cuda()
        res = q.decode(g, st, pt, max_iter, 0.75, precision, early_stop, want_post=True)
        torch.cuda.synchronize()
    finally:
        g.set_launch("auto")
    return [t.cpu().numpy() for t in res]


def assert_oracle(got, h, s, prior, max_iter, precision, early_stop=True):
    ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, np.ascontiguousarray(s, dtype=np.uint8), prior, max_iter,
                     0.75, OPREC[precision], early_stop, threads=16)
    err, iters, ok, post = got
    np.testing.assert_array_equal(iters, ref["iters"])
    np.testing.assert_array_equal(ok, ref["ok"])
    np.testing.assert_array_equal(err, ref["err"])
    np.testing.assert_array_equal(post.astype(np.float64) * SCALE[precision], ref["post"].astype(np.float64))
    return ref


def mixed_batch(code, shots, seed):
    """Shots at p = 0.01..0.06 interleaved with all-zero syndromes (met before iteration 1)."""
    parts = [w.x_error_batch(code, p, shots // 6 + 1, seed=seed + i).syndromes
             for i, p in enumerate((0.01, 0.02, 0.03, 0.04, 0.05, 0.06))]
    s = np.concatenate(parts)[:shots]
    rng = np.random.default_rng(seed)
    s = s[rng.permutation(len(s))]
    s[::7] = 0
    return s


@pytest.mark.parametrize("precision", ["int16", "int8", "fp32"])
@pytest.mark.parametrize("name", ["lp1054", "hgp400", "bb288"])
def test_packed_matches_oracle(q, name, precision):
    code = w.CONFIG_CODES[name]()
    h = code.hz_csr
    g = q.Graph.from_csr(h)
    s = mixed_batch(code, 2001, seed=700)
    prior = np.full(h.n, w.prior_llr(0.03), dtype=np.float32)
    ref = assert_oracle(run_packed(q, g, s, prior, 50, precision), h, s, prior, 50, precision)
    assert (ref["iters"] == 0).any() and (ref["iters"] > 10).any() and (ref["ok"] == 0).any()


@pytest.mark.parametrize("precision", ["int16", "int8", "fp32"])
def test_packed_batch_sizes_and_block_shapes(q, precision):
    """B = 1, 2, 3 (a lane idle from the start or at the end), 257, and 64 / 256 / 512 threads."""
    code = w.lp_code(1054)
    h = code.hz_csr
    g = q.Graph.from_csr(h)
    s = mixed_batch(code, 600, seed=710)
    prior = np.full(h.n, w.prior_llr(0.04), dtype=np.float32)
    for lo, hi in ((0, 1), (1, 3), (3, 6), (6, 263)):
        assert_oracle(run_packed(q, g, s[lo:hi], prior, 50, precision), h, s[lo:hi], prior, 50, precision)
    for threads in (64, 256, 512):
        assert_oracle(run_packed(q, g, s, prior, 50, precision, threads=threads), h, s, prior, 50, precision)
    # the decisions-only layout (no a-posteriori LLRs requested) gives the same decisions
    g.set_launch("packed")
    try:
        st = torch.from_numpy(np.ascontiguousarray(s, dtype=np.uint8)).cuda()
        pt = torch.from_numpy(np.ascontiguousarray(prior, dtype=np.float32)).cuda()
        err, iters, ok, _ = q.decode(g, st, pt, 50, 0.75, precision, True, want_post=False)
        torch.cuda.synchronize()
    finally:
        g.set_launch("auto")
    ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, 50, 0.75, OPREC[precision], True, threads=16)
    np.testing.assert_array_equal(err.cpu().numpy(), ref["err"])
    np.testing.assert_array_equal(iters.cpu().numpy(), ref["iters"])
    np.testing.assert_array_equal(ok.cpu().numpy(), ref["ok"])


@pytest.mark.parametrize("precision", ["int16", "int8", "fp32"])
def test_packed_paper_mode_and_zero_iterations(q, precision):
    code = w.hgp_code(400)
    h = code.hz_csr
    g = q.Graph.from_csr(h)
    s = mixed_batch(code, 500, seed=720)
    prior = np.full(h.n, w.prior_llr(0.05), dtype=np.float32)
    ref = assert_oracle(run_packed(q, g, s, prior, 10, precision, early_stop=False), h, s, prior, 10, precision,
                        early_stop=False)
    assert (ref["iters"] == 10).all()
    assert_oracle(run_packed(q, g, s, prior, 0, precision), h, s, prior, 0, precision)


@pytest.mark.parametrize("precision", ["int16", "int8", "fp32"])
def test_packed_saturating_priors_and_irregular_rows(q, precision):
    """Priors that saturate the message range, and a code with rows of degree 3..8 and columns of
    degree 1..5 (the non-uniform kernel variant)."""
    rng = np.random.default_rng(730)
    dense = np.zeros((60, 130), dtype=np.uint8)
    for i in range(60):
        dense[i, rng.choice(130, size=int(rng.integers(3, 9)), replace=False)] = 1
    h = csr(dense)
    g = q.Graph.from_csr(h)
    e = (rng.random((700, 130)) < 0.04).astype(np.uint8)
    s = w.syndromes(h, e)
    for prior in (np.full(130, w.prior_llr(0.04), dtype=np.float32),
                  rng.uniform(-3.0, 200.0, 130).astype(np.float32)):
        assert_oracle(run_packed(q, g, s, prior, 40, precision), h, s, prior, 40, precision)


@pytest.mark.parametrize("precision", ["int16", "int8", "fp32"])
def test_packed_pair_decode(q, precision):
    """The X+Z pair in one launch (blockIdx.y selects the half) equals the oracle on each half."""
    code = w.bb_code(12, 12)
    gz, gx = q.Graph.from_csr(code.hz_csr), q.Graph.from_csr(code.hx_csr)
    ex, ez = w.depolarizing_errors(code.n, 0.04, 901, seed=740)
    sx, sz = w.syndromes(code.hz_csr, ex), w.syndromes(code.hx_csr, ez)
    prior = np.full(code.n, w.prior_llr(2 * 0.04 / 3), dtype=np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    gz.set_launch("packed")
    try:
        rx, rz = q.decode_pair(gz, gx, dev(sx), dev(sz), dev(prior), dev(prior), 64, 0.75, precision, True,
                               want_post=True)
        torch.cuda.synchronize()
    finally:
        gz.set_launch("auto")
    assert_oracle([t.cpu().numpy() for t in rx], code.hz_csr, sx, prior, 64, precision)
    assert_oracle([t.cpu().numpy() for t in rz], code.hx_csr, sz, prior, 64, precision)


@pytest.mark.parametrize("precision", ["int16", "fp32"])
def test_packed_non_finite_prior(q, precision):
    code = w.hgp_code(400)
    h = code.hz_csr
    g = q.Graph.from_csr(h)
    s = mixed_batch(code, 300, seed=750)
    prior = np.full(h.n, 2.0, dtype=np.float32)
    prior[17] = np.nan
    err, iters, ok, post = run_packed(q, g, s, prior, 20, precision)
    assert (iters == -1).all() and (ok == 0).all() and (err == 0).all() and np.isnan(post).all()


@pytest.mark.parametrize("precision", ["int16", "fp32"])
def test_packed_large_batch_sampled_against_oracle(q, precision):
    """The benchmark's launch shape (LP-1054, 65536 shots): 1500 sampled shots against the oracle,
    and every reported success meets its syndrome."""
    code = w.lp_code(1054)
    h = code.hz_csr
    g = q.Graph.from_csr(h)
    b = w.x_error_batch(code, 0.03, 65536, seed=2003)
    g.set_launch("packed")
    try:           # the benchmark's form: no a-posteriori LLRs requested (the decisions-only layout)
        res = q.decode(g, torch.from_numpy(b.syndromes).cuda(), torch.from_numpy(b.prior).cuda(), 50, 0.75, precision)
        err, iters, ok = (t.cpu().numpy() for t in res[:3])
    finally:
        g.set_launch("auto")
    idx = np.random.default_rng(3).choice(65536, 1500, replace=False)
    ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes[idx], b.prior, 50, 0.75, OPREC[precision], True,
                     threads=16)
    np.testing.assert_array_equal(err[idx], ref["err"])
    np.testing.assert_array_equal(iters[idx], ref["iters"])
    np.testing.assert_array_equal(ok[idx], ref["ok"])
    met = (w.syndromes(h, err) == b.syndromes).all(axis=1)
    assert (met[ok == 1]).all() and not met[ok == 0].any()


def shifted_code(m, seed):
    """A (4, 8)-regular parity-check matrix, m x 2m: check i meets variables (i + a_t) mod m for four
    distinct seeded shifts a_t, and m + (i + b_t) mod m for four more."""
    rng = np.random.default_rng(seed)
    a, b = rng.choice(m, 4, replace=False), rng.choice(m, 4, replace=False)
    dense = np.zeros((m, 2 * m), dtype=np.uint8)
    i = np.arange(m)
    for t in range(4):
        dense[i, (i + a[t]) % m] = 1
        dense[i, m + (i + b[t]) % m] = 1
    return csr(dense)


@pytest.mark.parametrize("m", [1100, 2100])
def test_packed_large_graphs(q, m):
    """The pair kernel on graphs far larger than the benchmark's: 1100 and 2100 checks of degree 8
    (8800 and 16800 slots; two FP32 shots take 97 and 193 KB of shared memory), every precision,
    against the oracle."""
    h = shifted_code(m, seed=m)
    g = q.Graph.from_csr(h)
    rng = np.random.default_rng(m + 1)
    e = (rng.random((97, h.n)) < 0.02).astype(np.uint8)
    s = w.syndromes(h, e)
    s[::9] = 0
    prior = np.full(h.n, w.prior_llr(0.02), dtype=np.float32)
    for precision in ("fp32", "int16", "int8"):
        assert_oracle(run_packed(q, g, s, prior, 30, precision), h, s, prior, 30, precision)
