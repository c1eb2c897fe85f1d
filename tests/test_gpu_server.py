"""Persistent decoding server: continuous batching of single syndrome rounds across codes.

Every request of a mixed stream (40/40/20 over the N=400, 1054 and 288 codes, Poisson arrivals)
decodes exactly as the CPU oracle decodes it alone: flooding and layered schedule, FP32, INT16 and
INT8, and with per-code learned or plain weights.  Workers serve every code: a burst of one code
is taken up by more workers than an equal per-code share of the pool.  The ring refuses requests
while full; a worker whose wait runs out (no request arrives: the queue entry nothing writes)
leaves with a status bit and the library restarts the workers on the next request.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2508_07879_gb300 import workloads as w

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
CODES = ("hgp400", "lp1054", "bb288")
OPREC = {"fp32": "f32", "int16": "i16", "int8": "i8"}


@pytest.fixture(scope="module")
def q():
    from paper_2508_07879_gb300 import build
    build.build()
    from paper_2508_07879_gb300 import qldpc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return qldpc


def oracle_reference(h, syn, prior, max_iter, precision, early_stop=True, layered=False):
    r = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, np.ascontiguousarray(syn, dtype=np.uint8), prior, max_iter,
                   0.75, OPREC[precision], early_stop, threads=8, schedule="layered" if layered else "flooding")
    return r["err"], r["iters"], r["ok"]


def mixed_stream(n_req, seed, p=0.03):
    """Request mix 40/40/20 over the three codes (H_Z, i.i.d. X noise), Poisson arrivals 20 us apart."""
    rng = np.random.default_rng(seed)
    codes = rng.choice(3, size=n_req, p=[0.4, 0.4, 0.2]).astype(np.int32)
    arrival = np.cumsum(rng.exponential(20e3, size=n_req)).astype(np.int64)
    return codes, arrival


def interleave(codes, per_code_rows):
    cursor = [0] * len(per_code_rows)
    syn, ref_index = [], []
    for c in codes:
        syn.append(per_code_rows[c][cursor[c]])
        ref_index.append(cursor[c])
        cursor[c] += 1
    return syn, ref_index


def three_codes(n_req, seed, p=0.03):
    codes, arrival = mixed_stream(n_req, seed, p)
    batches = []
    for ci, name in enumerate(CODES):
        batches.append(w.x_error_batch(w.CONFIG_CODES[name](), p, int((codes == ci).sum()), seed=6001 + ci))
    return codes, arrival, batches


def assert_matches(codes, ref_index, refs, errs, iters, ok):
    for i, c in enumerate(codes):
        j = ref_index[i]
        np.testing.assert_array_equal(errs[i], refs[c][0][j])
        assert iters[i] == refs[c][1][j] and ok[i] == refs[c][2][j], (i, c, j)


@pytest.mark.parametrize("precision", ["fp32", "int16", "int8"])
def test_mixed_stream_matches_oracle(q, precision):
    codes, arrival, batches = three_codes(600, seed=5)
    graphs = [q.Graph.from_csr(b.h) for b in batches]
    refs = [oracle_reference(b.h, b.syndromes, b.prior, 50, precision) for b in batches]
    syn, ref_index = interleave(codes, [b.syndromes for b in batches])
    with q.Server(graphs, [b.prior for b in batches], 50, 0.75, precision, blocks=[12, 12, 8],
                  idle_timeout_s=2.0) as srv:
        assert srv.info()["workers"] == 32
        errs, iters, ok, lat = srv.replay(codes, syn, arrival)
    assert_matches(codes, ref_index, refs, errs, iters, ok)
    assert (lat > 0).all()


@pytest.mark.parametrize("precision", ["fp32", "int16", "int8"])
def test_layered_mixed_stream_matches_oracle(q, precision):
    """Layered-schedule workers over the three serving codes: LP-1054 (7 layers) keeps its checks in
    registers, HGP-400 (15 layers) and BB-288 (56 layers in its natural row order) their messages
    in shared memory, in one worker pool."""
    codes, arrival, batches = three_codes(450, seed=15)
    graphs = [q.Graph.from_csr(b.h) for b in batches]
    refs = [oracle_reference(b.h, b.syndromes, b.prior, 50, precision, layered=True) for b in batches]
    syn, ref_index = interleave(codes, [b.syndromes for b in batches])
    with q.Server(graphs, [b.prior for b in batches], 50, 0.75, precision, blocks=[10, 10, 4],
                  idle_timeout_s=2.0, layered=True) as srv:
        errs, iters, ok, lat = srv.replay(codes, syn, arrival, timeout_s=30.0)
    assert_matches(codes, ref_index, refs, errs, iters, ok)
    assert np.asarray(ok).mean() > 0.9


def test_layered_reordered_rows_match_oracle(q):
    """The BB-288 matrix with its rows in a greedy layer order (a different, shorter layered
    schedule: the row order of H is the schedule) on the register-resident path, against the oracle
    run on the same reordered matrix."""
    code = w.bb_code(12, 12)
    h = w.csr_rows(code.hz_csr, w.layer_order(code.hz_csr))
    b = w.x_error_batch(code, 0.03, 200, seed=77)
    syn = b.syndromes[:, w.layer_order(code.hz_csr)]
    g = q.Graph.from_csr(h)
    assert 1 <= g.layers() <= 8
    ref = oracle_reference(h, syn, b.prior, 64, "fp32", layered=True)
    arrival = (np.arange(200) * 30000).astype(np.int64)
    with q.Server([g], [b.prior], 64, 0.75, "fp32", blocks=[8], layered=True) as srv:
        errs, iters, ok, _ = srv.replay(np.zeros(200, np.int32), list(syn), arrival)
    assert_matches(np.zeros(200, np.int32), list(range(200)), [ref], errs, iters, ok)


def test_learned_and_plain_codes_match_oracle(q):
    """Per-code weights: LP-1054 decodes with learned weights (then the plain fallback), HGP-400 and
    BB-288 plainly, all in one worker pool."""
    codes, arrival, batches = three_codes(450, seed=25)
    graphs = [q.Graph.from_csr(b.h) for b in batches]
    h = batches[1].h
    weights = np.random.default_rng(11).uniform(0.55, 0.95, (12, h.nnz)).astype(np.float32)
    graphs[1].set_weights(weights)
    refs = []
    for ci, b in enumerate(batches):
        if ci == 1:
            r = oracle.nms_decode(h.row_ptr, h.col_idx, h.m, h.n, b.syndromes, b.prior, weights, 50, 0.75, threads=8)
            refs.append((r["err"], r["iters"], r["ok"]))
        else:
            refs.append(oracle_reference(b.h, b.syndromes, b.prior, 50, "fp32"))
    syn, ref_index = interleave(codes, [b.syndromes for b in batches])
    with q.Server(graphs, [b.prior for b in batches], 50, 0.75, "fp32", blocks=[12, 12, 8], learned=True,
                  idle_timeout_s=2.0) as srv:
        errs, iters, ok, _ = srv.replay(codes, syn, arrival)
    assert_matches(codes, ref_index, refs, errs, iters, ok)


def test_burst_of_one_code_takes_most_workers(q):
    """A burst of LP-1054 requests at t = 0 between sparse requests of the other two codes: the
    burst is decoded by more distinct workers than a third of the pool (what a static equal share
    per code would give it), and every result equals the oracle's."""
    batches = [w.x_error_batch(w.CONFIG_CODES[name](), 0.03, cnt, seed=6101 + i)
               for i, (name, cnt) in enumerate(zip(CODES, (40, 1200, 40)))]
    graphs = [q.Graph.from_csr(b.h) for b in batches]
    refs = [oracle_reference(b.h, b.syndromes, b.prior, 50, "fp32") for b in batches]
    codes = np.array([0] * 20 + [1] * 1200 + [2] * 40 + [0] * 20, dtype=np.int32)
    arrival = np.concatenate([np.arange(20) * 1000, np.full(1200, 20000), 20000 + np.arange(40) * 1000,
                              60000 + np.arange(20) * 1000]).astype(np.int64)
    syn, ref_index = interleave(codes, [b.syndromes for b in batches])
    with q.Server(graphs, [b.prior for b in batches], 50, 0.75, "fp32", ring_capacity=2048,
                  idle_timeout_s=2.0) as srv:
        pool = srv.info()["workers"]
        errs, iters, ok, lat, workers = srv.replay(codes, syn, arrival, timeout_s=30.0, want_workers=True)
    assert_matches(codes, ref_index, refs, errs, iters, ok)
    assert ((workers >= 0) & (workers < pool)).all()
    used = len(set(workers[codes == 1].tolist()))
    assert used > pool // 3, (used, pool)


def test_paper_mode_and_saturated_replay(q):
    """Ten fixed iterations without early stop (the paper's timed mode), all requests at t = 0."""
    code = w.bb_code(12, 6)
    graphs = [q.Graph.from_csr(code.hz_csr), q.Graph.from_csr(code.hx_csr)]
    ex, ez = w.depolarizing_errors(code.n, 0.03, 300, seed=71)
    prior = np.full(code.n, w.prior_llr(0.02), dtype=np.float32)
    sx, sz = w.syndromes(code.hz_csr, ex), w.syndromes(code.hx_csr, ez)
    ref_x = oracle_reference(code.hz_csr, sx, prior, 10, "fp32", early_stop=False)
    ref_z = oracle_reference(code.hx_csr, sz, prior, 10, "fp32", early_stop=False)
    codes = np.array([0, 1] * 300, dtype=np.int32)
    syn = [r for pair in zip(sx, sz) for r in pair]
    with q.Server(graphs, [prior, prior], 10, 0.75, "fp32", early_stop=False, blocks=[16, 16],
                  ring_capacity=64) as srv:
        errs, iters, ok, lat = srv.replay(codes, syn, np.zeros(600, dtype=np.int64))
    for i in range(300):
        np.testing.assert_array_equal(errs[2 * i], ref_x[0][i])
        np.testing.assert_array_equal(errs[2 * i + 1], ref_z[0][i])
        assert ok[2 * i] == ref_x[2][i] and ok[2 * i + 1] == ref_z[2][i]
    assert (iters == 10).all()


def test_submit_poll_ring_full(q):
    code = w.hgp_code(400)
    b = w.x_error_batch(code, 0.05, 6, seed=9)
    g = q.Graph.from_csr(b.h)
    ref = oracle_reference(b.h, b.syndromes, b.prior, 32, "fp32")
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
    """No request arrives: the workers' bounded wait on the queue runs out, they leave with the
    idle status bit, and the next request starts them again."""
    code = w.bb_code(12, 6)
    b = w.x_error_batch(code, 0.05, 2, seed=3)
    g = q.Graph.from_csr(b.h)
    ref = oracle_reference(b.h, b.syndromes, b.prior, 20, "fp32")
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


def test_layered_server_limits(q):
    lp = w.lp_code(1054)
    g = q.Graph.from_csr(lp.hz_csr)
    g.set_weights(np.full((4, lp.hz_csr.nnz), 0.75, dtype=np.float32))
    with pytest.raises(q.QldpcError) as ei:
        q.Server([g], [np.full(lp.n, 2.0, dtype=np.float32)], 10, learned=True, layered=True)
    assert ei.value.status == q.QLDPC_ERR_INVALID_ARG
    with pytest.raises(q.QldpcError) as ei:                    # fewer threads than the widest layer (93)
        q.Server([g], [np.full(lp.n, 2.0, dtype=np.float32)], 10, layered=True, threads_per_block=64)
    assert ei.value.status == q.QLDPC_ERR_UNSUPPORTED
    # rows of degree 9 (LP-1054's data-syndrome graph) exceed the layered workers' degree 8
    ds = w.data_syndrome_csr(lp.hz_csr)
    with pytest.raises(q.QldpcError) as ei:
        q.Server([q.Graph.from_csr(ds)], [np.full(ds.n, 2.0, dtype=np.float32)], 10, layered=True)
    assert ei.value.status == q.QLDPC_ERR_UNSUPPORTED
