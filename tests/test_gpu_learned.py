"""Learned (neural) normalized min-sum on the GPU against the oracle.

* learned decoding (weights, then the plain fallback) is bit-exact against the oracle's FP32
  learned decoder, in the batch and the latency kernel, on uniform and irregular codes, and
  through the server;
* the training forward is bit-exact on the last iteration's a-posteriori LLRs and matches the
  oracle's loss to FP32 accumulation error;
* the backward's weight gradient matches the oracle's reverse sweep (taken over the same FP32
  forward) within the tolerance derived in the test, and is deterministic up to the order of the
  FP32 additions over shots (global reductions): two calls agree to 1e-5 of each iteration's
  largest gradient;
* the device sampler draws exactly the workloads module's errors, Adam matches torch.optim.Adam,
  and the logical-failure kernel matches the GF(2) check on the host.
"""
import numpy as np
import pytest

import oracle
from paper_2508_07879_gb300 import gf2
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
    """Rows of degree 3..9 (non-uniform: the generic row-degree kernels), columns of degree >= 1."""
    rng = np.random.default_rng(seed)
    h = np.zeros((m, n), dtype=np.uint8)
    for i in range(m):
        h[i, rng.choice(n, size=int(rng.integers(3, 10)), replace=False)] = 1
    for v in np.nonzero(h.sum(0) == 0)[0]:
        h[rng.integers(m), v] = 1
    return w.csr_from_dense(h)


CODES = {
    "lp1054": lambda: w.lp_code(1054).hz_csr,
    "hgp400": lambda: w.hgp_code(400).hz_csr,
    "irregular": irregular_code,
}


def run_learned(q, h, s, prior, weights, max_iter, kernel):
    g = q.Graph.from_csr(h)
    g.set_weights(weights)
    g.set_launch(kernel)
    st = torch.from_numpy(np.ascontiguousarray(s)).cuda()
    pt = torch.from_numpy(np.ascontiguousarray(prior, dtype=np.float32)).cuda()
    err, iters, ok, post = q.decode(g, st, pt, max_iter, 0.75, learned=True, want_post=True)
    torch.cuda.synchronize()
    return err.cpu().numpy(), iters.cpu().numpy(), ok.cpu().numpy(), post.cpu().numpy()


@pytest.mark.parametrize("code", list(CODES))
@pytest.mark.parametrize("kernel", ["batch", "latency"])
def test_learned_decode_bit_exact(q, code, kernel):
    h = CODES[code]()
    rng = np.random.default_rng(17)
    T, L = 12, 25
    e = w.iid_x_errors(h.n, 0.05, 200, seed=44)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.05), dtype=np.float32)
    weights = rng.uniform(0.55, 0.95, (T, h.nnz)).astype(np.float32)
    ref = oracle.nms_decode(h.row_ptr, h.col_idx, h.m, h.n, s, prior, weights, L, 0.75, threads=8)
    err, iters, ok, post = run_learned(q, h, s, prior, weights, L, kernel)
    assert ref["fallback"].any() and (~ref["fallback"].astype(bool)).any()
    np.testing.assert_array_equal(err, ref["err"])
    np.testing.assert_array_equal(iters, ref["iters"])
    np.testing.assert_array_equal(ok, ref["ok"])
    np.testing.assert_array_equal(post.view(np.uint32), ref["post"].view(np.uint32))


def test_learned_decode_constant_weights_equal_plain(q):
    """alpha everywhere: the learned phase is plain min-sum, the fallback adds plain iterations."""
    h = w.lp_code(1054).hz_csr
    e = w.iid_x_errors(h.n, 0.05, 500, seed=5)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.05), dtype=np.float32)
    err, iters, ok, _ = run_learned(q, h, s, prior, np.full((20, h.nnz), 0.75, np.float32), 30, "batch")
    ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, 20, 0.75, "f32", threads=8)
    conv = ref["ok"] == 1
    np.testing.assert_array_equal(err[conv], ref["err"][conv])
    np.testing.assert_array_equal(iters[conv], ref["iters"][conv])
    assert (iters[~conv] > 20).all() or (~conv).sum() == 0


def test_learned_flag_validation(q):
    h = w.bb_code(12, 6).hz_csr
    g = q.Graph.from_csr(h)
    st = torch.zeros((4, h.m), dtype=torch.uint8, device="cuda")
    pt = torch.full((h.n,), 2.0, device="cuda")
    with pytest.raises(q.QldpcError) as ei:                    # no weights set
        q.decode(g, st, pt, 10, learned=True)
    assert ei.value.status == q.QLDPC_ERR_INVALID_ARG
    g.set_weights(np.full((5, h.nnz), 0.8, np.float32))
    for kw in (dict(precision="int16"), dict(early_stop=False)):
        with pytest.raises(q.QldpcError) as ei:
            q.decode(g, st, pt, 10, learned=True, **kw)
        assert ei.value.status == q.QLDPC_ERR_INVALID_ARG
    bad = np.full((5, h.nnz), 0.8, np.float32)
    bad[2, 7] = np.nan
    with pytest.raises(q.QldpcError):
        g.set_weights(bad)
    g.set_weights(None)
    with pytest.raises(q.QldpcError):
        q.decode(g, st, pt, 10, learned=True)


def test_learned_pair_and_server_equal_device_decode(q):
    """Per-code learned or plain weights in the persistent server: each request decodes as the
    device decode of its code does, in a mixed stream."""
    codes = [w.hgp_code(400).hz_csr, w.lp_code(1054).hz_csr, w.bb_code(12, 12).hz_csr]
    rng = np.random.default_rng(2)
    graphs, priors, syns, refs = [], [], [], []
    for i, h in enumerate(codes):
        g = q.Graph.from_csr(h)
        if i < 2:   # the third code stays plain
            g.set_weights(rng.uniform(0.5, 1.0, (10, h.nnz)).astype(np.float32))
        prior = np.full(h.n, w.prior_llr(0.03), dtype=np.float32)
        e = w.iid_x_errors(h.n, 0.05, 100, seed=300 + i)
        s = w.syndromes(h, e)
        st = torch.from_numpy(s).cuda()
        pt = torch.from_numpy(prior).cuda()
        dec, it, ok, _ = q.decode(g, st, pt, 30, 0.75, learned=(i < 2))
        refs.append((dec.cpu().numpy(), it.cpu().numpy(), ok.cpu().numpy()))
        graphs.append(g)
        priors.append(prior)
        syns.append(s)
    order = np.array([c for c in range(3) for _ in range(100)], dtype=np.int32)
    rng.shuffle(order)
    cursor = [0, 0, 0]
    req_syn, idx = [], []
    for c in order:
        req_syn.append(syns[c][cursor[c]])
        idx.append(cursor[c])
        cursor[c] += 1
    with q.Server(graphs, priors, 30, 0.75, "fp32", blocks=[8, 8, 8], learned=True, idle_timeout_s=2.0) as srv:
        errs, iters, ok, _ = srv.replay(order, req_syn, np.arange(300, dtype=np.int64) * 5000)
    for r, c in enumerate(order):
        j = idx[r]
        np.testing.assert_array_equal(errs[r], refs[c][0][j])
        assert iters[r] == refs[c][1][j] and ok[r] == refs[c][2][j]
    # pair decode with learned weights on both halves equals two single decodes
    hz, hx = w.hgp_code(400).hz_csr, w.hgp_code(400).hx_csr
    gz, gx = q.Graph.from_csr(hz), q.Graph.from_csr(hx)
    wz = rng.uniform(0.5, 1.0, (8, hz.nnz)).astype(np.float32)
    wx = rng.uniform(0.5, 1.0, (8, hx.nnz)).astype(np.float32)
    gz.set_weights(wz)
    gx.set_weights(wx)
    ex, ez = w.depolarizing_errors(hz.n, 0.05, 64, seed=8)
    sx = torch.from_numpy(w.syndromes(hz, ex)).cuda()
    sz = torch.from_numpy(w.syndromes(hx, ez)).cuda()
    pr = torch.full((hz.n,), w.prior_llr(0.04), device="cuda")
    (a, ia, oa, _), (b, ib, ob, _) = q.decode_pair(gz, gx, sx, sz, pr, pr, 20, learned=True)
    ra = q.decode(gz, sx, pr, 20, learned=True)
    rb = q.decode(gx, sz, pr, 20, learned=True)
    assert torch.equal(a, ra[0]) and torch.equal(ia, ra[1]) and torch.equal(b, rb[0]) and torch.equal(ib, rb[1])


def train_case(q, h, B, T, seed, p=0.05):
    rng = np.random.default_rng(seed)
    e = w.iid_x_errors(h.n, p, B, seed=seed)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.04), dtype=np.float32)
    weights = rng.uniform(0.5, 1.0, (T, h.nnz)).astype(np.float32)
    gl = rng.uniform(0.5, 1.5, B).astype(np.float32)
    g = q.Graph.from_csr(h)
    ws = torch.empty(q.nms_workspace_bytes(g, B, T), dtype=torch.uint8, device="cuda")
    dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (s, e, prior, weights, gl)]
    return g, ws, (e, s, prior, weights, gl), dev


@pytest.mark.parametrize("code,B,T", [("lp1054", 48, 20), ("hgp400", 300, 8), ("irregular", 40, 6)])
def test_training_forward_matches_oracle(q, code, B, T):
    h = CODES[code]()
    g, ws, (e, s, prior, weights, gl), (sd, ed, pd, wd, _) = train_case(q, h, B, T, 21)
    loss, post = q.nms_forward(g, sd, ed, pd, wd, ws, want_post=True)
    torch.cuda.synchronize()
    ref = oracle.nms_train(h.row_ptr, h.col_idx, h.m, h.n, s, e, prior, weights, precision="f32", post=True,
                           threads=8)
    np.testing.assert_array_equal(post.cpu().numpy().view(np.uint32), ref["post"][:, T - 1].view(np.uint32))
    # FP32 sum of T*n non-negative terms against the oracle's FP64 sum of the same FP32-derived terms
    np.testing.assert_allclose(loss.cpu().numpy(), ref["loss"], rtol=2e-5)


def grad_tolerance(ref):
    """Per-iteration bound: the GPU sums each gradient entry in FP32 over the shots and the reverse
    chain (terms of both signs), the oracle in FP64 from the same FP32 forward.  The error of an
    FP32 sum is below (terms) * 2^-24 * sum |term|; with at most a few hundred effective terms per
    entry this stays under 1e-4 of the iteration's largest gradient, plus 1e-3 relative."""
    scale = np.abs(ref).max(axis=1, keepdims=True)
    return 1e-4 * scale + 1e-3 * np.abs(ref)


@pytest.mark.parametrize("code,B,T", [("lp1054", 64, 20), ("hgp400", 2000, 6), ("irregular", 50, 5)])
def test_training_backward_matches_oracle(q, code, B, T):
    h = CODES[code]()
    g, ws, (e, s, prior, weights, gl), (sd, ed, pd, wd, gd) = train_case(q, h, B, T, 33)
    q.nms_forward(g, sd, ed, pd, wd, ws)
    grad = q.nms_backward(g, sd, ed, pd, T, gd, ws).cpu().numpy()
    grad2 = q.nms_backward(g, sd, ed, pd, T, gd, ws).cpu().numpy()
    assert (np.abs(grad - grad2) <= 1e-5 * np.abs(grad).max(axis=1, keepdims=True)).all()   # reduction order only
    ref = oracle.nms_train(h.row_ptr, h.col_idx, h.m, h.n, s, e, prior, weights, grad_loss=gl.astype(np.float64),
                           precision="f32", threads=16)["grad"]
    assert np.abs(ref).max() > 0
    assert (np.abs(grad - ref) <= grad_tolerance(ref)).all(), np.abs(grad - ref).max()


def test_training_loss_weights_match_oracle(q):
    """Non-uniform per-iteration loss weights lambda_t in both the loss and the gradient."""
    h = w.hgp_code(400).hz_csr
    B, T = 200, 8
    g, ws, (e, s, prior, weights, gl), (sd, ed, pd, wd, gd) = train_case(q, h, B, T, 51)
    lam = np.random.default_rng(3).uniform(0.0, 1.0, T).astype(np.float32)
    ld = torch.from_numpy(lam).cuda()
    loss, _ = q.nms_forward(g, sd, ed, pd, wd, ws, loss_weights=ld)
    grad = q.nms_backward(g, sd, ed, pd, T, gd, ws, loss_weights=ld).cpu().numpy()
    ref = oracle.nms_train(h.row_ptr, h.col_idx, h.m, h.n, s, e, prior, weights, grad_loss=gl.astype(np.float64),
                           precision="f32", threads=16, loss_weights=lam.astype(np.float64))
    np.testing.assert_allclose(loss.cpu().numpy(), ref["loss"], rtol=2e-5)
    assert (np.abs(grad - ref["grad"]) <= grad_tolerance(ref["grad"])).all()


def test_autograd_function_and_training_step(q):
    from paper_2508_07879_gb300 import learned
    h = w.hgp_code(400).hz_csr
    model = learned.NeuralMinSum(h, np.full(h.n, w.prior_llr(0.04)), T=6, max_batch=512)
    err, syn = q.sample_errors(model.graph, 5, 0, 512, 0.02, 0.06)
    loss = model.loss(syn, err)
    loss.mean().backward()
    direct = q.nms_backward(model.graph, syn, err, model.prior, 6,
                            torch.full((512,), 1.0 / 512, device="cuda"), model.workspace)
    assert torch.allclose(model.weights.grad, direct, rtol=1e-6, atol=1e-9)
    model.weights.grad = None
    e_fix, s_fix = q.sample_errors(model.graph, 77, 0, 512, 0.02, 0.06)   # held-out batch
    with torch.no_grad():
        before = model.loss(s_fix, e_fix).mean().item()
    hist = model.train(shots=512 * 40, batch=512, lr=3e-3, record_every=1)
    with torch.no_grad():
        after = model.loss(s_fix, e_fix).mean().item()
    assert len(hist) == 40 and np.isfinite(hist).all()
    assert after < before
    # checkpoint round trip
    import tempfile, os
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "w.qnms")
        model.save(path)
        other = learned.NeuralMinSum(h, np.full(h.n, w.prior_llr(0.04)), T=6, max_batch=64)
        other.load(path)
        assert torch.equal(other.weights, model.weights) and other.step == model.step
        assert torch.equal(other.exp_avg_sq, model.exp_avg_sq)


def test_device_sampler_matches_workloads(q):
    h = w.lp_code(1054).hz_csr
    g = q.Graph.from_csr(h)
    err, syn = q.sample_errors(g, 1234, 777, 300, 0.02, 0.06)
    e_ref, _ = w.iid_x_errors_prange(h.n, 0.02, 0.06, 300, seed=1234, first_shot=777)
    np.testing.assert_array_equal(err.cpu().numpy(), e_ref)
    np.testing.assert_array_equal(syn.cpu().numpy(), w.syndromes(h, e_ref))
    err2, _ = q.sample_errors(g, 99, 0, 200, 0.05)
    np.testing.assert_array_equal(err2.cpu().numpy(), w.iid_x_errors(h.n, 0.05, 200, seed=99))


def test_adam_matches_torch(q):
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=(7, 333)).astype(np.float32)
    ref = torch.nn.Parameter(torch.from_numpy(p0.copy()))
    opt = torch.optim.Adam([ref], lr=1e-2, betas=(0.9, 0.999), eps=1e-8, foreach=False)
    p = torch.from_numpy(p0.copy()).cuda()
    m1, m2 = torch.zeros_like(p), torch.zeros_like(p)
    for step in range(1, 6):
        g = rng.normal(size=p0.shape).astype(np.float32)
        ref.grad = torch.from_numpy(g)
        opt.step()
        q.adam_step(p, torch.from_numpy(g).cuda(), m1, m2, step, 1e-2)
    torch.testing.assert_close(p.cpu(), ref.detach(), rtol=2e-6, atol=2e-7)


def test_logical_failures_match_host(q):
    code = w.lp_code(1054)
    L = gf2.logical_basis(code.hx_csr.dense(), code.hz_csr.dense())       # detect X residuals
    Lx = gf2.logical_basis(code.hz_csr.dense(), code.hx_csr.dense())      # X logical operators
    rng = np.random.default_rng(1)
    B = 500
    e = (rng.random((B, code.n)) < 0.05).astype(np.uint8)
    d = e.copy()
    # residuals: stabilizers (rows of H_X), logicals, random, and nothing
    hx = code.hx_csr.dense()
    for b in range(B):
        kind = b % 4
        if kind == 0:
            d[b] ^= hx[rng.integers(hx.shape[0])]
        elif kind == 1:
            d[b] ^= Lx[rng.integers(Lx.shape[0])]
        elif kind == 2:
            d[b] ^= (rng.random(code.n) < 0.01).astype(np.uint8)
    ok = (rng.random(B) < 0.9).astype(np.uint8)
    fail = q.logical_failures(torch.from_numpy(L).cuda(), torch.from_numpy(e).cuda(), torch.from_numpy(d).cuda(),
                              torch.from_numpy(ok).cuda()).cpu().numpy()
    expect = (ok == 0) | gf2.logical_failures(e ^ d, L)
    np.testing.assert_array_equal(fail, expect.astype(np.uint8))
    assert fail[1::4].all()


@pytest.mark.parametrize("kernel", ["batch", "latency"])
def test_learned_alone_without_fallback(q, kernel):
    """max_iter = 0 after the learned iterations: unconverged shots keep the prior's decisions (the
    plain decoder with no iterations), as the oracle's learned decoder specifies."""
    h = w.lp_code(1054).hz_csr
    rng = np.random.default_rng(9)
    e = w.iid_x_errors(h.n, 0.05, 200, seed=45)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.05), dtype=np.float32)
    weights = rng.uniform(0.55, 0.95, (10, h.nnz)).astype(np.float32)
    ref = oracle.nms_decode(h.row_ptr, h.col_idx, h.m, h.n, s, prior, weights, 0, 0.75, threads=8)
    err, iters, ok, post = run_learned(q, h, s, prior, weights, 0, kernel)
    assert ref["fallback"].any()
    np.testing.assert_array_equal(err, ref["err"])
    np.testing.assert_array_equal(iters, ref["iters"])
    np.testing.assert_array_equal(ok, ref["ok"])
    np.testing.assert_array_equal(post.view(np.uint32), ref["post"].view(np.uint32))
