"""Persistent decoding server: continuous batching of single syndrome rounds across codes.

Every request decodes to the same result alone (qldpc_decode_ex on the device path) and in a
mixed stream of three codes served concurrently; the ring refuses requests while full; a worker
whose wait runs out (no request arrives: the tail word nothing writes) leaves with a status bit
and the library restarts the workers on the next request.
"""
import time

import numpy as np
import pytest

from paper_2508_07879_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
CODES = ("hgp400", "lp1054", "bb288")


@pytest.fixture(scope="module")
def q():
    from paper_2508_07879_gb300 import build
    build.build()
    from paper_2508_07879_gb300 import qldpc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qldpc


def device_reference(q, graph, syn, prior, max_iter, precision, early_stop=True, layered=False):
    s = torch.from_numpy(np.ascontiguousarray(syn, dtype=np.uint8)).cuda()
    p = torch.from_numpy(np.ascontiguousarray(prior, dtype=np.float32)).cuda()
    err, iters, ok, _ = q.decode(graph, s, p, max_iter, 0.75, precision, early_stop, layered=layered)
    torch.cuda.synchronize()
    return err.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy()


def mixed_stream(n_req, seed, p=0.03):
    """Request mix 40/40/20 over the three codes (H_Z, i.i.d. X noise), Poisson arrivals 20 us apart."""
    rng = np.random.default_rng(seed)
    codes = rng.choice(3, size=n_req, p=[0.4, 0.4, 0.2]).astype(np.int32)
    arrival = np.cumsum(rng.exponential(20e3, size=n_req)).astype(np.int64)
    return codes, arrival


@pytest.mark.parametrize("precision", ["fp32", "int16", "int8"])
def test_mixed_stream_equals_alone(q, precision):
    graphs, priors, batches = [], [], []
    codes, arrival = mixed_stream(600, seed=5)
    for ci, name in enumerate(CODES):
        code = w.CONFIG_CODES[name]()
        count = int((codes == ci).sum())
        b = w.x_error_batch(code, 0.03, count, seed=6001 + ci)
        graphs.append(q.Graph.from_csr(b.h))
        priors.append(b.prior)
        batches.append(b)
    refs = [device_reference(q, graphs[i], batches[i].syndromes, priors[i], 50, precision) for i in range(3)]
    cursor = [0, 0, 0]
    syn, ref_index = [], []
    for c in codes:
        syn.append(batches[c].syndromes[cursor[c]])
        ref_index.append(cursor[c])
        cursor[c] += 1
    with q.Server(graphs, priors, 50, 0.75, precision, blocks=[12, 12, 8], idle_timeout_s=2.0) as srv:
        errs, iters, ok, lat = srv.replay(codes, syn, arrival)
    for i, c in enumerate(codes):
        j = ref_index[i]
        np.testing.assert_array_equal(errs[i], refs[c][0][j])
        assert iters[i] == refs[c][1][j] and ok[i] == refs[c][2][j]
    assert (lat > 0).all()


def test_paper_mode_and_saturated_replay(q):
    """Ten fixed iterations without early stop (the paper's timed mode), all requests at t = 0."""
    code = w.bb_code(12, 6)
    graphs = [q.Graph.from_csr(code.hz_csr), q.Graph.from_csr(code.hx_csr)]
    ex, ez = w.depolarizing_errors(code.n, 0.03, 300, seed=71)
    prior = np.full(code.n, w.prior_llr(0.02), dtype=np.float32)
    sx, sz = w.syndromes(code.hz_csr, ex), w.syndromes(code.hx_csr, ez)
    ref_x = device_reference(q, graphs[0], sx, prior, 10, "fp32", early_stop=False)
    ref_z = device_reference(q, graphs[1], sz, prior, 10, "fp32", early_stop=False)
    codes = np.array([0, 1] * 300, dtype=np.int32)
    syn = [r for pair in zip(sx, sz) for r in pair]
    with q.Server(graphs, [prior, prior], 10, 0.75, "fp32", early_stop=False, blocks=[16, 16],
                  ring_capacity=64) as srv:
        errs, iters, ok, lat = srv.replay(codes, syn, np.zeros(600, dtype=np.int64))
    for i in range(300):
        np.testing.assert_array_equal(errs[2 * i], ref_x[0][i])
        np.testing.assert_array_equal(errs[2 * i + 1], ref_z[0][i])
    assert (iters == 10).all()


def test_submit_poll_ring_full(q):
    code = w.hgp_code(400)
    b = w.x_error_batch(code, 0.05, 6, seed=9)
    g = q.Graph.from_csr(b.h)
    ref = device_reference(q, g, b.syndromes, b.prior, 32, "fp32")
    with q.Server([g], [b.prior], 32, 0.75, "fp32", ring_capacity=4, blocks=[2]) as srv:
        tickets = [srv.submit(0, b.syndromes[i]) for i in range(4)]
        assert tickets == [0, 1, 2, 3]
        assert srv.submit(0, b.syndromes[4]) is None           # all four slots hold uncollected results
        for i, t in enumerate(tickets):
            res = None
            deadline = time.time() + 10
            while res is None and time.time() < deadline:
                res = srv.poll(0, t)
            assert res is not None
            np.testing.assert_array_equal(res[0], ref[0][i])
            assert res[1] == ref[1][i] and res[2] == ref[2][i]
        with pytest.raises(q.QldpcError):
            srv.poll(0, tickets[0])                            # already collected
        t4 = srv.submit(0, b.syndromes[4])
        assert t4 == 4


def test_idle_wait_runs_out_and_workers_restart(q):
    """No request arrives: the workers' bounded wait on the ring tail runs out, they leave with the
    idle status bit, and the next request starts them again."""
    code = w.bb_code(12, 6)
    b = w.x_error_batch(code, 0.05, 2, seed=3)
    g = q.Graph.from_csr(b.h)
    ref = device_reference(q, g, b.syndromes, b.prior, 20, "fp32")
    with q.Server([g], [b.prior], 20, 0.75, "fp32", blocks=[2], idle_timeout_s=0.02) as srv:
        for i in range(2):
            t = srv.submit(0, b.syndromes[i])
            res = None
            deadline = time.time() + 10
            while res is None and time.time() < deadline:
                res = srv.poll(0, t)
            assert res is not None
            np.testing.assert_array_equal(res[0], ref[0][i])
            time.sleep(0.2)                                    # > idle timeout: the workers leave
            assert srv.status() & 1                            # idle-exit bit


def test_server_rejects_bad_arguments(q):
    code = w.bb_code(12, 6)
    g = q.Graph.from_csr(code.hz_csr)
    prior = np.full(code.n, 2.0, dtype=np.float32)
    bad = prior.copy()
    bad[3] = np.inf
    with pytest.raises(q.QldpcError) as ei:
        q.Server([g], [bad], 10)
    assert ei.value.status == q.QLDPC_ERR_INVALID_ARG
    for kwargs in (dict(ring_capacity=3), dict(alpha=1.5, precision="int16"), dict(max_iter=-1)):
        args = dict(max_iter=10)
        args.update(kwargs)
        mi = args.pop("max_iter")
        with pytest.raises(q.QldpcError) as ei:
            q.Server([g], [prior], mi, **args)
        assert ei.value.status == q.QLDPC_ERR_INVALID_ARG
    with pytest.raises(q.QldpcError) as ei:
        q.Server([g], [prior], 10, blocks=[100000])            # more workers than can be resident
    assert ei.value.status == q.QLDPC_ERR_UNSUPPORTED


@pytest.mark.parametrize("precision", ["fp32", "int16", "int8"])
def test_layered_server_equals_layered_decode(q, precision):
    """Layered-schedule workers (QLDPC_LAYERED) over LP-1054's H_Z and H_X (7 layers each), a mixed
    stream: every request decodes as the layered batch decode does."""
    code = w.lp_code(1054)
    ex, ez = w.depolarizing_errors(code.n, 0.03, 400, seed=72)
    prior = np.full(code.n, w.prior_llr(0.02), dtype=np.float32)
    hs = [code.hz_csr, code.hx_csr]
    syns = [w.syndromes(code.hz_csr, ex), w.syndromes(code.hx_csr, ez)]
    graphs = [q.Graph.from_csr(h) for h in hs]
    refs = [device_reference(q, graphs[i], syns[i], prior, 50, precision, layered=True) for i in range(2)]
    rng = np.random.default_rng(9)
    codes = rng.integers(0, 2, 400).astype(np.int32)
    arrival = np.cumsum(rng.exponential(20e3, size=400)).astype(np.int64)
    cursor = [0, 0]
    syn, ref_index = [], []
    for c in codes:
        syn.append(syns[c][cursor[c]])
        ref_index.append(cursor[c])
        cursor[c] += 1
    with q.Server(graphs, [prior, prior], 50, 0.75, precision, blocks=[8, 8], idle_timeout_s=2.0,
                  layered=True) as srv:
        errs, iters, ok, lat = srv.replay(codes, syn, arrival)
    for i, c in enumerate(codes):
        j = ref_index[i]
        np.testing.assert_array_equal(errs[i], refs[c][0][j])
        assert iters[i] == refs[c][1][j] and ok[i] == refs[c][2][j]
    assert (lat > 0).all() and np.asarray(ok).mean() > 0.9


def test_layered_server_limits(q):
    hgp = w.hgp_code(400)
    prior = np.full(hgp.n, 2.0, dtype=np.float32)
    with pytest.raises(q.QldpcError) as ei:                    # 15 layers: above the register-resident 8
        q.Server([q.Graph.from_csr(hgp.hz_csr)], [prior], 10, layered=True)
    assert ei.value.status == q.QLDPC_ERR_UNSUPPORTED
    lp = w.lp_code(1054)
    g = q.Graph.from_csr(lp.hz_csr)
    g.set_weights(np.full((4, lp.hz_csr.nnz), 0.75, dtype=np.float32))
    with pytest.raises(q.QldpcError) as ei:
        q.Server([g], [np.full(lp.n, 2.0, dtype=np.float32)], 10, learned=True, layered=True)
    assert ei.value.status == q.QLDPC_ERR_INVALID_ARG
    with pytest.raises(q.QldpcError) as ei:                    # fewer threads than the widest layer (93)
        q.Server([g], [np.full(lp.n, 2.0, dtype=np.float32)], 10, layered=True, threads_per_block=64)
    assert ei.value.status == q.QLDPC_ERR_UNSUPPORTED
