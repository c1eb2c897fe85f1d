"""CUDA decoder vs the CPU oracle, element by element, through the C ABI.

Both precisions are bit-exact by construction (the FP32 kernel performs the oracle's additions and
multiplications in the same order with explicit round-to-nearest intrinsics; the INT16 kernel is
integer arithmetic), so every comparison below is exact equality of e_hat, iterations, ok and the
a-posteriori LLRs.  Exact equality implies the looser FP32 requirement (1e-5 relative, identical
decisions and iteration counts outside |LLR| < 1e-4 ties).
"""
import os

import numpy as np
import pytest

import oracle
from helpers import csr, random_tree_pcm, syndrome_dense
from paper_2508_07879_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ORACLE_PREC = {"fp32": "f32", "int16": "i16"}
THREADS = os.cpu_count() or 4


@pytest.fixture(scope="module")
def q():
    from paper_2508_07879_gb300 import build
    build.build()
    from paper_2508_07879_gb300 import qldpc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qldpc


def set_kernel(graph, kernel):
    """"auto", "batch", "latency" or "latencyT" (the latency kernel with T threads per block)."""
    if kernel.startswith("latency") and kernel != "latency":
        graph.set_launch("latency", int(kernel[len("latency"):]))
    else:
        graph.set_launch(kernel)


def gpu_decode(q, graph, syn, prior, max_iter, alpha, precision, early_stop=True, kernel="auto"):
    """kernel: "auto" (the library's choice), "batch", "latency" or "latencyT" (forced for the
    whole batch; see set_kernel)."""
    syn = np.ascontiguousarray(syn, dtype=np.uint8)
    p = torch.from_numpy(np.ascontiguousarray(prior, dtype=np.float32)).cuda()
    s = torch.from_numpy(syn).cuda()
    if kernel != "auto":
        set_kernel(graph, kernel)
    try:
        err, iters, ok, post = q.decode(graph, s, p, max_iter, alpha, precision, early_stop, want_post=True)
        torch.cuda.synchronize()
    finally:
        if kernel != "auto":
            graph.set_launch("auto")
    return {"err": err.cpu().numpy(), "iters": iters.cpu().numpy(), "ok": ok.cpu().numpy(),
            "post": post.cpu().numpy()}


def oracle_decode(h, syn, prior, max_iter, alpha, precision, early_stop=True):
    return oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, syn, prior, max_iter, alpha,
                      ORACLE_PREC[precision], early_stop, threads=THREADS)


def assert_parity(g, o, precision, where=""):
    np.testing.assert_array_equal(g["iters"], o["iters"], err_msg=f"iters {where}")
    np.testing.assert_array_equal(g["ok"], o["ok"], err_msg=f"ok {where}")
    np.testing.assert_array_equal(g["err"], o["err"], err_msg=f"err {where}")
    if precision == "int16":
        np.testing.assert_array_equal(g["post"] * 256.0, o["post"].astype(np.float64), err_msg=f"post {where}")
    else:
        np.testing.assert_array_equal(g["post"], o["post"], err_msg=f"post {where}")


def check(q, h, syn, prior, max_iter, alpha=0.75, precision="fp32", early_stop=True, graph=None,
          kernels=("batch", "latency")):
    """Decode on every kernel in `kernels` and compare each with the oracle."""
    graph = graph or q.Graph.from_csr(h)
    o = oracle_decode(h, syn, prior, max_iter, alpha, precision, early_stop)
    g = None
    for kernel in kernels:
        g = gpu_decode(q, graph, syn, prior, max_iter, alpha, precision, early_stop, kernel)
        assert_parity(g, o, precision, f"{kernel} {precision} early={early_stop} max_iter={max_iter}")
    return g, o


PRECS = ["fp32", "int16"]


# ---------------------------------------------------------------------------------------------
# Tiny graphs: every syndrome, several iteration limits, both stop modes
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", PRECS)
def test_eq1_all_syndromes(q, precision):
    h = csr(w.eq1_pcm())
    syn = np.array([[(i >> b) & 1 for b in range(3)] for i in range(8)], dtype=np.uint8)
    for gamma in (np.ones(6), np.array([1.5, -0.25, 2.0, 0.5, -1.0, 3.0])):
        for max_iter in (0, 1, 2, 7, 25):
            for early in (True, False):
                check(q, h, syn, gamma, max_iter, 0.75, precision, early)


@pytest.mark.parametrize("precision", PRECS)
def test_single_check_hand_example_on_gpu(q, precision):
    h = csr(np.array([[1, 1, 1, 1]], dtype=np.uint8))
    g, _ = check(q, h, np.array([[1]]), np.array([2.0, -3.0, 5.0, 1.0]), 1, 0.75, precision, False)
    np.testing.assert_array_equal(g["post"][0] - np.array([2.0, -3.0, 5.0, 1.0]), [0.75, -0.75, 0.75, 1.5])


@pytest.mark.parametrize("precision", PRECS)
def test_tree_graphs(q, precision):
    rng = np.random.default_rng(77)
    for _ in range(8):
        hd = random_tree_pcm(rng, n_checks=int(rng.integers(2, 8)), max_deg=5)
        h = csr(hd)
        e = (rng.random((64, h.n)) < 0.2).astype(np.uint8)
        gamma = (rng.integers(50, 700, h.n) / 256.0) * rng.choice([-1, 1], h.n, p=[0.2, 0.8])
        check(q, h, w.syndromes(h, e), gamma, h.m + 2, 1.0, precision, False)
        check(q, h, w.syndromes(h, e), gamma, h.m + 2, 0.75, precision, True)


# ---------------------------------------------------------------------------------------------
# Workload configurations
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("precision", PRECS)
def test_hgp400_config(q, precision):
    """Hypergraph-product N=400, 1000 shots of i.i.d. X errors at p = 0.05, max 32 iterations."""
    code = w.hgp_code(400)
    b = w.x_error_batch(code, 0.05, 1000, seed=1)
    g, o = check(q, b.h, b.syndromes, b.prior, 32, 0.75, precision)
    assert 0.3 < o["ok"].mean() < 0.8


@pytest.mark.parametrize("precision", PRECS)
def test_lp1054_config_mixed_p(q, precision):
    """Lifted-product N=1054, p in {0.01..0.05}, max 50 iterations, ragged batch of 2503 shots."""
    code = w.lp_code(1054)
    h = code.hz_csr
    graph = q.Graph.from_csr(h)
    for i, p in enumerate((0.01, 0.02, 0.03, 0.04, 0.05)):
        b = w.x_error_batch(code, p, 2503 if i == 2 else 500, seed=2001 + i)
        check(q, h, b.syndromes, b.prior, 50, 0.75, precision, graph=graph, kernels=("batch",))
        check(q, h, b.syndromes[:300], b.prior, 50, 0.75, precision, graph=graph,
              kernels=("latency", "latency544", "latency640"))


@pytest.mark.parametrize("precision", PRECS)
def test_lp1054_full_batch_sampled(q, precision):
    """B = 65536 in the automatic (benchmark) launch shape; 1200 sampled shots vs the oracle and
    properties that hold for every shot."""
    code = w.lp_code(1054)
    h = code.hz_csr
    graph = q.Graph.from_csr(h)
    B = 65536
    b = w.x_error_batch(code, 0.03, B, seed=2003)
    g = gpu_decode(q, graph, b.syndromes, b.prior, 50, 0.75, precision)
    rng = np.random.default_rng(4)
    idx = np.unique(np.concatenate([[0, 1, B - 2, B - 1], rng.choice(B, 1200, replace=False)]))
    o = oracle_decode(h, b.syndromes[idx], b.prior, 50, 0.75, precision)
    assert_parity({k: v[idx] for k, v in g.items()}, o, precision, "sampled")
    met = (w.syndromes(h, g["err"]) == b.syndromes).all(axis=1)
    np.testing.assert_array_equal(g["ok"], met.astype(np.uint8))
    assert ((g["iters"] >= 0) & (g["iters"] <= 50)).all()
    assert (g["iters"][g["ok"] == 0] == 50).all()
    assert g["ok"].mean() > 0.98


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("name", ["bb144", "bb288"])
def test_bb_pair_decode(q, name, precision):
    """X and Z halves in one launch equal two separate decodes and the oracle (depolarizing noise)."""
    code = w.CONFIG_CODES[name]()
    gz, gx = q.Graph.from_csr(code.hz_csr), q.Graph.from_csr(code.hx_csr)
    for i, p in enumerate((0.01, 0.03, 0.05)):
        ex, ez = w.depolarizing_errors(code.n, p, 700, seed=3001 + i)
        sx, sz = w.syndromes(code.hz_csr, ex), w.syndromes(code.hx_csr, ez)
        prior = np.full(code.n, w.prior_llr(2 * p / 3), dtype=np.float32)
        for max_iter, early in ((64, True), (10, False)):      # plain mode and the paper's mode
            dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
            ox = oracle_decode(code.hz_csr, sx, prior, max_iter, 0.75, precision, early)
            oz = oracle_decode(code.hx_csr, sz, prior, max_iter, 0.75, precision, early)
            for chunk in (len(sx), 50):          # one batch-kernel launch / latency-kernel launches
                parts_x, parts_z = [], []
                for lo in range(0, len(sx), chunk):
                    hi = min(lo + chunk, len(sx))
                    (rx, rz) = q.decode_pair(gz, gx, dev(sx[lo:hi]), dev(sz[lo:hi]), dev(prior), dev(prior),
                                             max_iter, 0.75, precision, early, want_post=True)
                    torch.cuda.synchronize()
                    parts_x.append([t.cpu().numpy() for t in rx])
                    parts_z.append([t.cpu().numpy() for t in rz])
                keys = ("err", "iters", "ok", "post")
                pair_x = {k: np.concatenate([p[i] for p in parts_x]) for i, k in enumerate(keys)}
                pair_z = {k: np.concatenate([p[i] for p in parts_z]) for i, k in enumerate(keys)}
                assert_parity(pair_x, ox, precision, f"pair x chunk {chunk}")
                assert_parity(pair_z, oz, precision, f"pair z chunk {chunk}")
            # the pair on the latency kernel for the whole batch (the launch shape follows the first graph)
            gz.set_launch("latency")
            try:
                (rx, rz) = q.decode_pair(gz, gx, dev(sx), dev(sz), dev(prior), dev(prior), max_iter, 0.75,
                                         precision, early, want_post=True)
                torch.cuda.synchronize()
            finally:
                gz.set_launch("auto")
            assert_parity(dict(zip(("err", "iters", "ok", "post"), [t.cpu().numpy() for t in rx])), ox,
                          precision, "pair x latency")
            assert_parity(dict(zip(("err", "iters", "ok", "post"), [t.cpu().numpy() for t in rz])), oz,
                          precision, "pair z latency")
            sep_x = gpu_decode(q, gz, sx, prior, max_iter, 0.75, precision, early)
            sep_z = gpu_decode(q, gx, sz, prior, max_iter, 0.75, precision, early)
            for k in pair_x:
                np.testing.assert_array_equal(pair_x[k], sep_x[k])
                np.testing.assert_array_equal(pair_z[k], sep_z[k])


# ---------------------------------------------------------------------------------------------
# Invariances of the launch
# ---------------------------------------------------------------------------------------------
def test_batch_invariance(q):
    code = w.lp_code(1054)
    graph = q.Graph.from_csr(code.hz_csr)
    b = w.x_error_batch(code, 0.04, 4096, seed=8)
    for precision in PRECS:
        ref = gpu_decode(q, graph, b.syndromes, b.prior, 50, 0.75, precision)
        for B in (1, 64):
            for start in (0, 1000, 4096 - B):
                part = gpu_decode(q, graph, b.syndromes[start:start + B], b.prior, 50, 0.75, precision)
                for k in ref:
                    np.testing.assert_array_equal(part[k], ref[k][start:start + B])


def test_launch_shapes_give_identical_results(q):
    code = w.lp_code(1054)
    graph = q.Graph.from_csr(code.hz_csr)
    b = w.x_error_batch(code, 0.05, 700, seed=12)
    ref = {p: gpu_decode(q, graph, b.syndromes, b.prior, 50, 0.75, p) for p in PRECS}
    shapes = [("batch", 32, 0), ("batch", 96, 2), ("batch", 128, 0), ("batch", 256, 1),
              ("batch", 544, 0), ("batch", 1024, 1), ("latency", 544, 0), ("latency", 640, 0),
              ("latency", 0, 0), ("latency", 0, 1), ("latency", 576, 1)]
    for kernel, threads, per_sm in shapes:
        graph.set_launch(kernel, threads, per_sm)
        for p in PRECS:
            got = gpu_decode(q, graph, b.syndromes, b.prior, 50, 0.75, p)
            for k in got:
                np.testing.assert_array_equal(got[k], ref[p][k], err_msg=f"{kernel} {threads}x{per_sm} {p} {k}")
    graph.set_launch("auto")
    # the latency kernel needs m <= 2*threads and n <= 2*threads, threads <= 640
    for bad_threads in (256, 1024):
        with pytest.raises(q.QldpcError) as ei:
            graph.set_launch("latency", bad_threads, 0)
        assert ei.value.status == q.QLDPC_ERR_UNSUPPORTED
    with pytest.raises(q.QldpcError) as ei:      # two 576-thread latency blocks do not fit an SM
        graph.set_launch("latency", 576, 2)
    assert ei.value.status == q.QLDPC_ERR_UNSUPPORTED
    with pytest.raises(q.QldpcError) as ei:
        graph.set_launch("latency", 256, 0)
    assert ei.value.status == q.QLDPC_ERR_UNSUPPORTED
    with pytest.raises(q.QldpcError) as ei:
        graph.set_launch("auto", 256, 0)
    assert ei.value.status == q.QLDPC_ERR_INVALID_ARG


# ---------------------------------------------------------------------------------------------
# Edge cases
# ---------------------------------------------------------------------------------------------
def test_empty_batch_is_a_noop(q):
    h = csr(w.eq1_pcm())
    graph = q.Graph.from_csr(h)
    s = torch.zeros((0, 3), dtype=torch.uint8, device="cuda")
    p = torch.ones(6, dtype=torch.float32, device="cuda")
    err, iters, ok, _ = q.decode(graph, s, p, 10)
    assert err.shape == (0, 6) and iters.shape == (0,)


def test_irregular_graph_with_isolated_variables(q):
    rng = np.random.default_rng(5)
    hd = (rng.random((40, 90)) < 0.06).astype(np.uint8)
    hd[:, 80:] = 0                                       # ten variables in no check
    for r in range(40):                                  # every row degree >= 2, varied
        while hd[r].sum() < 2:
            hd[r, rng.integers(0, 80)] = 1
    h = csr(hd)
    assert len(set(h.row_degrees().tolist())) > 2
    e = (rng.random((300, 90)) < 0.05).astype(np.uint8)
    gamma = rng.uniform(-1, 4, 90)
    for precision in PRECS:
        for early in (True, False):
            check(q, h, w.syndromes(h, e), gamma, 20, 0.625, precision, early)


def test_maximum_degrees(q):
    """Row degree 32 and column degree 16, the largest the kernels support."""
    rng = np.random.default_rng(9)
    m, n = 16, 40
    hd = np.zeros((m, n), dtype=np.uint8)
    hd[0, :32] = 1                                       # one row of degree 32
    hd[:, 0] = 1                                         # column 0 of degree 16
    for r in range(1, m):
        hd[r, rng.choice(np.arange(1, n), 3, replace=False)] = 1
    h = csr(hd)
    assert h.row_degrees().max() == 32 and h.col_degrees().max() == 16
    e = (rng.random((200, n)) < 0.1).astype(np.uint8)
    gamma = rng.uniform(0.2, 3, n)
    for precision in PRECS:
        check(q, h, w.syndromes(h, e), gamma, 30, 0.75, precision)


def test_zero_syndrome_and_prior_decision(q):
    code = w.hgp_code(400)
    h = code.hz_csr
    syn = np.zeros((5, h.m), dtype=np.uint8)
    for precision in PRECS:
        g, _ = check(q, h, syn, np.full(h.n, 2.0), 30, 0.75, precision)
        assert (g["iters"] == 0).all() and (g["ok"] == 1).all() and not g["err"].any()
        b = w.x_error_batch(code, 0.05, 50, seed=4)
        check(q, h, b.syndromes, b.prior, 0, 0.75, precision)              # max_iter = 0


def test_nonfinite_prior_reported_per_shot(q):
    code = w.bb_code(12, 6)
    h = code.hz_csr
    graph = q.Graph.from_csr(h)
    prior = np.full(h.n, 3.0, dtype=np.float32)
    prior[17] = np.nan
    for precision in PRECS:
        g = gpu_decode(q, graph, np.ones((9, h.m), np.uint8), prior, 10, 0.75, precision)
        assert (g["iters"] == -1).all() and (g["ok"] == 0).all() and not g["err"].any()


def test_host_buffer_path_matches_device_path(q):
    code = w.lp_code(1054)
    graph = q.Graph.from_csr(code.hz_csr)
    for precision in PRECS:
        for p in (0.02, 0.05):
            b = w.x_error_batch(code, p, 333, seed=31)
            dev = gpu_decode(q, graph, b.syndromes, b.prior, 50, 0.75, precision)
            err, iters, ok = q.decode_host(graph, b.syndromes, b.prior, 50, 0.75, precision)
            np.testing.assert_array_equal(err, dev["err"])
            np.testing.assert_array_equal(iters, dev["iters"])
            np.testing.assert_array_equal(ok, dev["ok"])


def test_host_path_with_pinned_buffers(q):
    """Page-locked buffers take the no-copy path (the kernel reads/writes host memory); pageable
    ones the staged path; both equal the device path, for single shots and a large batch."""
    code = w.lp_code(1054)
    graph = q.Graph.from_csr(code.hz_csr)
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()
    for precision in PRECS:
        for shots in (1, 3, 5000):
            b = w.x_error_batch(code, 0.04, shots, seed=41 + shots)
            dev = gpu_decode(q, graph, b.syndromes, b.prior, 50, 0.75, precision)
            syn = pin((shots, graph.m), torch.uint8)
            syn[:] = b.syndromes
            outs = (pin((shots, graph.n), torch.uint8), pin((shots,), torch.int32), pin((shots,), torch.uint8))
            for o in outs:
                o.fill(0x5A if o.dtype == np.uint8 else -3)
            err, iters, ok = q.decode_host(graph, syn, b.prior, 50, 0.75, precision, out=outs)
            np.testing.assert_array_equal(err, dev["err"])
            np.testing.assert_array_equal(iters, dev["iters"])
            np.testing.assert_array_equal(ok, dev["ok"])
            # mixed: pinned syndromes, pageable outputs -> staged copies
            err2, iters2, ok2 = q.decode_host(graph, syn, b.prior, 50, 0.75, precision)
            np.testing.assert_array_equal(err2, dev["err"])
            np.testing.assert_array_equal(iters2, dev["iters"])


@pytest.mark.parametrize("name", ["bb144", "bb288"])
def test_pair_host_path_matches_oracle(q, name):
    """The X+Z pair end to end with host buffers (qldpc_decode_pair_host): page-locked buffers (no
    copies) and pageable ones (staged), in plain and the paper's mode, against the oracle's two
    separate decodes; single shots (the latency sweep) and a batch."""
    code = w.CONFIG_CODES[name]()
    gz, gx = q.Graph.from_csr(code.hz_csr), q.Graph.from_csr(code.hx_csr)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    ex, ez = w.depolarizing_errors(code.n, 0.04, 300, seed=3301)
    sx, sz = w.syndromes(code.hz_csr, ex), w.syndromes(code.hx_csr, ez)
    prior = np.full(code.n, w.prior_llr(2 * 0.04 / 3), dtype=np.float32)
    for max_iter, early in ((64, True), (10, False)):
        ox = oracle_decode(code.hz_csr, sx, prior, max_iter, 0.75, "fp32", early)
        oz = oracle_decode(code.hx_csr, sz, prior, max_iter, 0.75, "fp32", early)
        for pinned in (True, False):
            for lo, hi in ((0, 1), (1, 2), (2, 300)):
                a, b = (pin(sx[lo:hi]), pin(sz[lo:hi])) if pinned else (sx[lo:hi].copy(), sz[lo:hi].copy())
                outs = None
                if pinned:
                    outs = tuple((pin(np.zeros((hi - lo, code.n), np.uint8)), pin(np.zeros(hi - lo, np.int32)),
                                  pin(np.zeros(hi - lo, np.uint8))) for _ in range(2))
                (rx, rz) = q.decode_pair_host(gz, gx, a, b, prior, prior, max_iter, 0.75, "fp32", early, out=outs)
                for got, ref in ((rx, ox), (rz, oz)):
                    np.testing.assert_array_equal(got[0], ref["err"][lo:hi])
                    np.testing.assert_array_equal(got[1], ref["iters"][lo:hi])
                    np.testing.assert_array_equal(got[2], ref["ok"][lo:hi])
    with pytest.raises(q.QldpcError):
        q.decode_pair_host(gz, gz, sx[:1], sx[:1], prior, prior, 10)      # one graph for both halves


def test_side_stream(q):
    code = w.hgp_code(400)
    graph = q.Graph.from_csr(code.hz_csr)
    b = w.x_error_batch(code, 0.05, 400, seed=2)
    ref = gpu_decode(q, graph, b.syndromes, b.prior, 32, 0.75, "fp32")
    st = torch.cuda.Stream()
    s = torch.from_numpy(b.syndromes).cuda()
    p = torch.from_numpy(b.prior).cuda()
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        err, iters, ok, _ = q.decode(graph, s, p, 32)
    st.synchronize()
    np.testing.assert_array_equal(err.cpu().numpy(), ref["err"])
    np.testing.assert_array_equal(iters.cpu().numpy(), ref["iters"])


def test_invalid_decode_arguments(q):
    code = w.bb_code(12, 6)
    graph = q.Graph.from_csr(code.hz_csr)
    s = torch.zeros((4, graph.m), dtype=torch.uint8, device="cuda")
    p = torch.ones(graph.n, dtype=torch.float32, device="cuda")
    for kwargs in (dict(alpha=1.5, precision="int16"), dict(alpha=float("nan")), dict(alpha=0.0),
                   dict(alpha=-0.5), dict(max_iter=-1)):
        args = dict(max_iter=10, alpha=0.75, precision="fp32")
        args.update(kwargs)
        with pytest.raises(q.QldpcError) as ei:
            q.decode(graph, s, p, **args)
        assert ei.value.status == q.QLDPC_ERR_INVALID_ARG
    ptr = lambda t: t.data_ptr()
    rc = q.qldpc_decode_ex(graph.handle, ptr(s), 4, ptr(p), 10, 0.75, None, None, None, None, 0, 0, None)
    assert rc == q.QLDPC_ERR_INVALID_ARG
    rc = q.qldpc_decode_ex(graph.handle, ptr(s), 0, ptr(p), 10, 0.75, None, None, None, None, 7, 0, None)
    assert rc == q.QLDPC_ERR_INVALID_ARG                                  # unknown precision
    rc = q.qldpc_decode_ex(graph.handle, ptr(s), 0, ptr(p), 10, 0.75, None, None, None, None, 0, 6, None)
    assert rc == q.QLDPC_ERR_INVALID_ARG                                  # unknown flag bits


def test_pair_with_different_row_widths(q):
    """A pair whose graphs have different row-degree buckets (8 and 16) shares one kernel variant:
    each half must still decode as it does alone and as the oracle does."""
    rng = np.random.default_rng(12)
    n = 150

    def random_code(m, lo, hi):
        h = np.zeros((m, n), dtype=np.uint8)
        for i in range(m):
            h[i, rng.choice(n, size=int(rng.integers(lo, hi)), replace=False)] = 1
        for v in np.nonzero(h.sum(0) == 0)[0]:   # cover every column without exceeding degree hi
            rows = np.nonzero(h.sum(1) < hi)[0]
            h[rng.choice(rows), v] = 1
        return w.csr_from_dense(h)

    ha, hb = random_code(70, 3, 8), random_code(60, 9, 13)
    assert np.diff(ha.row_ptr).max() <= 8 < np.diff(hb.row_ptr).max()
    ga, gb = q.Graph.from_csr(ha), q.Graph.from_csr(hb)
    B = 400
    ea = (rng.random((B, n)) < 0.05).astype(np.uint8)
    eb = (rng.random((B, n)) < 0.05).astype(np.uint8)
    sa, sb = w.syndromes(ha, ea), w.syndromes(hb, eb)
    prior = rng.uniform(1.5, 3.5, n).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    (xa, ia, oa, pa), (xb, ib, ob, pb) = q.decode_pair(ga, gb, dev(sa), dev(sb), dev(prior), dev(prior), 40,
                                                       want_post=True)
    for h, s, got in ((ha, sa, (xa, ia, oa, pa)), (hb, sb, (xb, ib, ob, pb))):
        ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, 40, 0.75, "f32", threads=8)
        np.testing.assert_array_equal(got[0].cpu().numpy(), ref["err"])
        np.testing.assert_array_equal(got[1].cpu().numpy(), ref["iters"])
        np.testing.assert_array_equal(got[2].cpu().numpy(), ref["ok"])
        np.testing.assert_array_equal(got[3].cpu().numpy(), ref["post"])
