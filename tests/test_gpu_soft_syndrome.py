"""Soft-syndrome decoding on the GPU: the decoder on the data-syndrome graph [H | I_m] against the
oracle on the same graph, bit-exact (data and syndrome-error decisions, iterations, ok, LLRs) in
FP32, INT16 and INT8 and with the layered schedule; infinitely reliable syndrome bits reproduce the
device's hard-syndrome decode on H."""
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


SCALE = {"fp32": 1.0, "int16": 256.0, "int8": 4.0}
ORACLE = {"fp32": "f32", "int16": "i16", "int8": "i8"}


@pytest.mark.parametrize("precision,layered", [("fp32", False), ("int16", False), ("int8", False), ("fp32", True),
                                               ("int16", True)])
def test_lp1054_noisy_syndromes_match_oracle(q, precision, layered):
    h = w.lp_code(1054).hz_csr
    a = w.data_syndrome_csr(h)
    g = q.Graph.from_csr(a)
    e, es, s = w.noisy_syndrome_batch(h, 0.03, 0.01, 1500, seed=77)
    gamma = np.full(h.n, w.prior_llr(0.03), np.float32)
    lam = np.full(h.m, w.prior_llr(0.01), np.float32)
    st = torch.from_numpy(s).cuda()
    ed, esd, iters, ok, post = q.decode_soft(g, st, torch.from_numpy(gamma).cuda(), torch.from_numpy(lam).cuda(), 50,
                                             precision=precision, want_post=True, layered=layered)
    torch.cuda.synchronize()
    ref = oracle.msa(a.row_ptr, a.col_idx, a.m, a.n, s, np.concatenate([gamma, lam]), 50, 0.75, ORACLE[precision],
                     threads=16, schedule="layered" if layered else "flooding")
    np.testing.assert_array_equal(ed.cpu().numpy(), ref["err"][:, :h.n])
    np.testing.assert_array_equal(esd.cpu().numpy(), ref["err"][:, h.n:])
    np.testing.assert_array_equal(iters.cpu().numpy(), ref["iters"])
    np.testing.assert_array_equal(ok.cpu().numpy(), ref["ok"])
    np.testing.assert_array_equal(post.cpu().numpy().astype(np.float64) * SCALE[precision],
                                  ref["post"].astype(np.float64))
    assert 0.25 < ref["ok"].mean() < 0.6 and esd.cpu().numpy().any()   # the oracle: 36 % of these shots decode


@pytest.mark.parametrize("precision", ["fp32", "int16", "int8"])
def test_single_shot_kernel_matches_oracle(q, precision):
    """A (4, 8)-regular code with 60 checks: its data-syndrome rows have exact degree 9, and a batch
    of at most one shot per SM takes the single-shot kernel."""
    h = w.csr_from_dense(w.random_regular_ldpc(60, 120, 4, 8, seed=5))
    a = w.data_syndrome_csr(h)
    g = q.Graph.from_csr(a)
    e, es, s = w.noisy_syndrome_batch(h, 0.03, 0.02, 100, seed=79)
    gamma = np.full(h.n, w.prior_llr(0.03), np.float32)
    lam = np.full(h.m, w.prior_llr(0.02), np.float32)
    ed, esd, iters, ok, post = q.decode_soft(g, torch.from_numpy(s).cuda(), torch.from_numpy(gamma).cuda(),
                                             torch.from_numpy(lam).cuda(), 50, precision=precision,
                                             want_post=True)
    torch.cuda.synchronize()
    ref = oracle.msa(a.row_ptr, a.col_idx, a.m, a.n, s, np.concatenate([gamma, lam]), 50, 0.75, ORACLE[precision],
                     threads=16)
    np.testing.assert_array_equal(ed.cpu().numpy(), ref["err"][:, :h.n])
    np.testing.assert_array_equal(esd.cpu().numpy(), ref["err"][:, h.n:])
    np.testing.assert_array_equal(iters.cpu().numpy(), ref["iters"])
    np.testing.assert_array_equal(ok.cpu().numpy(), ref["ok"])
    np.testing.assert_array_equal(post.cpu().numpy().astype(np.float64) * SCALE[precision],
                                  ref["post"].astype(np.float64))
    assert ref["iters"].max() > 5 and esd.cpu().numpy().any()


def test_reliable_bits_reproduce_the_hard_decode(q):
    h = w.lp_code(1054).hz_csr
    a = w.data_syndrome_csr(h)
    e, es, s = w.noisy_syndrome_batch(h, 0.03, 0.01, 500, seed=78)
    st = torch.from_numpy(s).cuda()
    gamma = torch.full((h.n,), w.prior_llr(0.03), device="cuda")
    soft = q.decode_soft(q.Graph.from_csr(a), st, gamma, torch.full((h.m,), 1e30, device="cuda"), 50, want_post=True)
    hard = q.decode(q.Graph.from_csr(h), st, gamma, 50, want_post=True)
    torch.cuda.synchronize()
    assert torch.equal(soft[0], hard[0]) and not soft[1].any()
    assert torch.equal(soft[2], hard[1]) and torch.equal(soft[3], hard[2])
    assert torch.equal(soft[4][:, :h.n], hard[3])


def test_served_soft_syndromes_equal_the_batch_decode(q):
    """The persistent server on a data-syndrome graph (rows of exact degree 9) decodes every request
    as the batch decode does."""
    h = w.csr_from_dense(w.random_regular_ldpc(60, 120, 4, 8, seed=5))
    a = w.data_syndrome_csr(h)
    g = q.Graph.from_csr(a)
    e, es, s = w.noisy_syndrome_batch(h, 0.03, 0.02, 200, seed=80)
    prior = np.concatenate([np.full(h.n, w.prior_llr(0.03)), np.full(h.m, w.prior_llr(0.02))]).astype(np.float32)
    err, iters, ok, _ = q.decode(g, torch.from_numpy(s).cuda(), torch.from_numpy(prior).cuda(), 50)
    torch.cuda.synchronize()
    codes = np.zeros(len(s), np.int32)
    arrival = np.arange(len(s), dtype=np.int64) * 20000
    with q.Server([g], [prior], 50, 0.75, "fp32", blocks=[16], idle_timeout_s=2.0) as srv:
        errs, it, okk, _ = srv.replay(codes, list(s), arrival)
    np.testing.assert_array_equal(np.stack(errs), err.cpu().numpy())
    np.testing.assert_array_equal(np.asarray(it), iters.cpu().numpy())
    np.testing.assert_array_equal(np.asarray(okk), ok.cpu().numpy())
