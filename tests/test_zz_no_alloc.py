"""qldpc_decode_host_noalloc: the host-buffer decode that allocates no device memory.

It serves callers that cannot call cudaMalloc once running (a real-time control loop whose device
memory is fixed at start-up, a plug-in whose host owns all device memory): the staging lives in a
static device array inside the library instead of graph-owned allocations.  Its results must equal
those of qldpc_decode_host, which stages through memory it allocates, on consecutive calls (the
array keeps the previous call's contents).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

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


def ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def noalloc(q, graph, syn, prior, max_iter, alpha, precision, flags=0):
    syn = np.ascontiguousarray(syn, dtype=np.uint8)
    prior = np.ascontiguousarray(prior, dtype=np.float32)
    batch = syn.shape[0]
    err = np.full((batch, graph.n), 0xAB, dtype=np.uint8)
    iters = np.full(batch, -7, dtype=np.int32)
    ok = np.full(batch, 0xCD, dtype=np.uint8)
    rc = q.qldpc_decode_host_noalloc(graph.handle, ptr(syn), batch, ptr(prior), max_iter, alpha,
                                     ptr(err), ptr(iters), ptr(ok), q.PRECISIONS[precision], flags, None)
    return rc, err, iters, ok


@pytest.mark.parametrize("precision", ["fp32", "int16"])
def test_noalloc_matches_allocating_host_path_on_consecutive_calls(q, precision):
    code = w.lp_code(1054)
    graph = q.Graph.from_csr(code.hz_csr)
    # two calls in a row with different sizes and noise, so the second reads over the first's leftovers
    for p, shots, seed in ((0.05, 1500, 71), (0.02, 257, 72), (0.04, 1, 73)):
        b = w.x_error_batch(code, p, shots, seed=seed)
        rc, err, iters, ok = noalloc(q, graph, b.syndromes, b.prior, 50, 0.75, precision)
        assert rc == q.QLDPC_OK, q.qldpc_status_string(rc)
        ref_err, ref_iters, ref_ok = q.decode_host(graph, b.syndromes, b.prior, 50, 0.75, precision)
        np.testing.assert_array_equal(err, ref_err)
        np.testing.assert_array_equal(iters, ref_iters)
        np.testing.assert_array_equal(ok, ref_ok)


def test_noalloc_pair_of_graphs_and_paper_mode(q):
    code = w.bb_code(12, 6)
    gz, gx = q.Graph.from_csr(code.hz_csr), q.Graph.from_csr(code.hx_csr)
    ex, ez = w.depolarizing_errors(code.n, 0.03, 400, seed=74)
    prior = np.full(code.n, w.prior_llr(0.02), dtype=np.float32)
    for graph, e in ((gz, ex), (gx, ez)):
        s = w.syndromes(code.hz_csr if graph is gz else code.hx_csr, e)
        rc, err, iters, ok = noalloc(q, graph, s, prior, 10, 0.75, "fp32", q.QLDPC_NO_EARLY_STOP)
        assert rc == q.QLDPC_OK
        ref = q.decode_host(graph, s, prior, 10, 0.75, "fp32", early_stop=False)
        np.testing.assert_array_equal(err, ref[0])
        np.testing.assert_array_equal(iters, ref[1])
        np.testing.assert_array_equal(ok, ref[2])


def test_noalloc_rejects_batches_beyond_the_scratch(q):
    code = w.lp_code(1054)
    graph = q.Graph.from_csr(code.hz_csr)
    r = lambda x: (x + 255) // 256 * 256
    fits = lambda b: r(4 * graph.n) + r(b * graph.m) + r(b * graph.n) + r(4 * b) + r(b) \
        <= q.QLDPC_NOALLOC_SCRATCH_BYTES
    biggest = max(b for b in range(1, 5000) if fits(b))
    syn = np.zeros((biggest + 1, graph.m), dtype=np.uint8)
    prior = np.full(graph.n, 3.0, dtype=np.float32)
    rc, err, iters, ok = noalloc(q, graph, syn, prior, 10, 0.75, "fp32")
    assert rc == q.QLDPC_ERR_UNSUPPORTED
    assert (iters == -7).all()                           # nothing written
    rc, err, iters, ok = noalloc(q, graph, syn[:biggest], prior, 10, 0.75, "fp32")
    assert rc == q.QLDPC_OK and (iters == 0).all() and (ok == 1).all()


def test_noalloc_allocates_nothing_once_warm(q):
    """After the start-up zero-shot call and one call of each kind (which may load kernel code), a
    series of further calls of every kind and size leaves the device's free memory unchanged, and
    the scratch size the binding uses is the one compiled into the library."""
    assert q.qldpc_noalloc_scratch_bytes() == q.QLDPC_NOALLOC_SCRATCH_BYTES
    code = w.lp_code(1054)
    graph = q.Graph.from_csr(code.hz_csr)
    graph.set_weights(np.random.default_rng(5).uniform(0.6, 0.9, (6, code.hz_csr.nnz)).astype(np.float32))
    b = w.x_error_batch(code, 0.04, 2000, seed=75)
    kinds = [("fp32", 0), ("int16", 0), ("int8", 0), ("fp32", q.QLDPC_LAYERED),
             ("int16", q.QLDPC_LAYERED | q.QLDPC_NO_EARLY_STOP), ("int8", q.QLDPC_NO_EARLY_STOP),
             ("fp32", q.QLDPC_LEARNED)]
    sizes = (1, 97, 2000)                       # single-shot and batch kernels
    assert q.qldpc_decode_host_noalloc(graph.handle, None, 0, None, 50, 0.75, None, None, None,
                                       q.QLDPC_FP32, 0, None) == q.QLDPC_OK
    for prec, flags in kinds:
        for shots in sizes:
            rc, *_ = noalloc(q, graph, b.syndromes[:shots], b.prior, 50, 0.75, prec, flags)
            assert rc == q.QLDPC_OK, (prec, flags, shots)
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for rep in range(2):
        for prec, flags in kinds:
            for shots in sizes:
                rc, err, iters, ok = noalloc(q, graph, b.syndromes[:shots], b.prior, 50, 0.75, prec, flags)
                assert rc == q.QLDPC_OK and (iters >= 0).all()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_validates_before_enqueueing(q):
    code = w.bb_code(12, 6)
    graph = q.Graph.from_csr(code.hz_csr)
    syn = np.zeros((4, graph.m), dtype=np.uint8)
    prior = np.ones(graph.n, dtype=np.float32)
    rc, *_ = noalloc(q, graph, syn, prior, 10, 1.5, "int16")      # alpha > 1 in fixed point
    assert rc == q.QLDPC_ERR_INVALID_ARG
    rc, *_ = noalloc(q, graph, syn, prior, -1, 0.75, "fp32")
    assert rc == q.QLDPC_ERR_INVALID_ARG
    assert q.qldpc_decode_host_noalloc(None, None, 0, None, 10, 0.75, None, None, None, 0, 0, None) \
        == q.QLDPC_ERR_INVALID_ARG
