"""Syndrome loss of the learned min-sum decoder on the GPU against the oracle.

The training forward runs the same unrolled decoder as with the error loss (its last a-posteriori
LLRs stay bit-exact); the loss is the mean over checks and iterations of -log P_c, the soft
syndrome's BCE, and the backward's weight gradient is compared with the oracle's reverse sweep
over the same FP32 forward.
"""
import numpy as np
import pytest

import oracle
from paper_2508_07879_gb300 import workloads as w
from test_gpu_learned import CODES, grad_tolerance, train_case

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def q():
    from paper_2508_07879_gb300 import build
    build.build()
    from paper_2508_07879_gb300 import qldpc
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return qldpc


def oracle_syn(h, s, e, prior, weights, **kw):
    return oracle.nms_train(h.row_ptr, h.col_idx, h.m, h.n, s, e, prior, weights, precision="f32", loss="syndrome",
                            threads=16, **kw)


# Loss tolerance: each term is -log P with P from a product of up to 8 FP32 tanh values (a few ulp
# each) in FP32; near P -> 0 the relative error of P grows as 1/P, which the floor bounds, and the
# terms are averaged over m checks.  1e-4 relative plus 1e-6 absolute covers that with margin.
LOSS_RTOL, LOSS_ATOL = 1e-4, 1e-6


@pytest.mark.parametrize("code,B,T", [("lp1054", 48, 20), ("hgp400", 300, 8), ("irregular", 40, 6)])
def test_forward_matches_oracle(q, code, B, T):
    h = CODES[code]()
    g, ws, (e, s, prior, weights, gl), (sd, ed, pd, wd, _) = train_case(q, h, B, T, 23)
    loss, post = q.nms_forward(g, sd, None, pd, wd, ws, want_post=True, loss="syndrome")
    torch.cuda.synchronize()
    ref = oracle_syn(h, s, e, prior, weights, post=True)
    np.testing.assert_array_equal(post.cpu().numpy().view(np.uint32), ref["post"][:, T - 1].view(np.uint32))
    np.testing.assert_allclose(loss.cpu().numpy(), ref["loss"], rtol=LOSS_RTOL, atol=LOSS_ATOL)
    # targets are not read: passing them changes nothing
    loss2, _ = q.nms_forward(g, sd, ed, pd, wd, ws, loss="syndrome")
    assert torch.equal(loss, loss2)


@pytest.mark.parametrize("code,B,T", [("lp1054", 64, 20), ("hgp400", 500, 6), ("irregular", 50, 5)])
def test_backward_matches_oracle(q, code, B, T):
    h = CODES[code]()
    g, ws, (e, s, prior, weights, gl), (sd, ed, pd, wd, gd) = train_case(q, h, B, T, 35)
    q.nms_forward(g, sd, None, pd, wd, ws, loss="syndrome")
    grad = q.nms_backward(g, sd, None, pd, T, gd, ws, loss="syndrome").cpu().numpy()
    ref = oracle_syn(h, s, e, prior, weights, grad_loss=gl.astype(np.float64))["grad"]
    assert np.abs(ref).max() > 0
    assert (np.abs(grad - ref) <= grad_tolerance(ref)).all(), np.abs(grad - ref).max()


def test_loss_weights_match_oracle(q):
    h = w.hgp_code(400).hz_csr
    B, T = 200, 8
    g, ws, (e, s, prior, weights, gl), (sd, ed, pd, wd, gd) = train_case(q, h, B, T, 52)
    lam = np.random.default_rng(4).uniform(0.0, 1.0, T).astype(np.float32)
    ld = torch.from_numpy(lam).cuda()
    loss, _ = q.nms_forward(g, sd, ed, pd, wd, ws, loss_weights=ld, loss="syndrome")
    grad = q.nms_backward(g, sd, ed, pd, T, gd, ws, loss_weights=ld, loss="syndrome").cpu().numpy()
    ref = oracle_syn(h, s, e, prior, weights, grad_loss=gl.astype(np.float64), loss_weights=lam.astype(np.float64))
    np.testing.assert_allclose(loss.cpu().numpy(), ref["loss"], rtol=LOSS_RTOL, atol=LOSS_ATOL)
    assert (np.abs(grad - ref["grad"]) <= grad_tolerance(ref["grad"])).all()


def test_training_lowers_held_out_syndrome_loss(q):
    from paper_2508_07879_gb300 import learned
    h = w.hgp_code(400).hz_csr
    model = learned.NeuralMinSum(h, np.full(h.n, w.prior_llr(0.04)), T=6, max_batch=512, loss="syndrome")
    err, syn = q.sample_errors(model.graph, 5, 0, 512, 0.02, 0.06)
    loss = model.loss(syn, None)
    loss.mean().backward()
    direct = q.nms_backward(model.graph, syn, None, model.prior, 6, torch.full((512,), 1.0 / 512, device="cuda"),
                            model.workspace, loss="syndrome")
    assert torch.allclose(model.weights.grad, direct, rtol=1e-6, atol=1e-9)
    model.weights.grad = None
    e_fix, s_fix = q.sample_errors(model.graph, 78, 0, 512, 0.02, 0.06)
    with torch.no_grad():
        before = model.loss(s_fix, None).mean().item()
    hist = model.train(shots=512 * 40, batch=512, lr=3e-3, record_every=1)
    with torch.no_grad():
        after = model.loss(s_fix, None).mean().item()
    assert len(hist) == 40 and np.isfinite(hist).all()
    assert after < before
