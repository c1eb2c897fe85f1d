"""Maximum sizes on the GPU: the largest graph whose FP32 shot fits the device's shared memory, the
next size up (rejected before any launch), and a 2^21-shot batch in one call."""
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


def qc_code(L, seed=1):
    """Quasi-cyclic (3,6)-regular H: a 3 x 6 array of L x L circulant permutations."""
    rng = np.random.default_rng(seed)
    shifts = rng.integers(0, L, size=(3, 6))
    h = np.zeros((3 * L, 6 * L), dtype=np.uint8)
    eye = np.eye(L, dtype=np.uint8)
    for r in range(3):
        for c in range(6):
            h[r * L:(r + 1) * L, c * L:(c + 1) * L] = np.roll(eye, shifts[r, c], axis=1)
    return w.csr_from_dense(h)


def fp32_shot_bytes(m, lanes, dc):
    """Shared memory of one FP32 shot of the batch kernel: Q and gamma [lanes], parity words [m],
    messages [dc * m + 32] (32 scratch slots for idle lanes), each section 16-byte aligned."""
    a16 = lambda x: (x + 15) // 16 * 16
    return a16(a16(a16(a16(4 * lanes) + 4 * lanes) + 4 * m) + 4 * (dc * m + 32))


def test_footprint_formula_and_lanes(q):
    """The reported footprint follows the layout above; the lift-31 code packs 31 variables and
    one idle lane per warp (34 warps), the 144- and 288-qubit codes need no idle lane."""
    for code, lanes_want in ((w.lp_code(1054), 1088), (w.bb_code(12, 6), 144), (w.bb_code(12, 12), 288)):
        h = code.hz_csr
        g = q.Graph.from_csr(h)
        lanes, nbytes = g.footprint("fp32")
        assert lanes == lanes_want
        assert nbytes == fp32_shot_bytes(h.m, lanes, int(h.row_degrees().max()))
        l16, b16 = g.footprint("int16")
        assert l16 == lanes and b16 < nbytes
        g.close()


def test_largest_graph_that_fits(q):
    optin = getattr(torch.cuda.get_device_properties(0), "shared_memory_per_block_optin", 232448)

    def fp32_bytes(L):
        g = q.Graph.from_csr(qc_code(L))
        try:
            return g.footprint("fp32")[1]
        finally:
            g.close()

    def boundary(limit):
        # largest L (step 8) whose shot fits `limit` bytes: bracket, then bisect
        lo, hi = 16, 16
        while fp32_bytes(hi) <= limit:
            lo, hi = hi, hi * 2
        while hi - lo > 8:
            mid = (lo + hi) // 16 * 8
            lo, hi = (mid, hi) if fp32_bytes(mid) <= limit else (lo, mid)
        return lo

    # the kernel adds a few bytes of static shared memory: leave it 256 bytes
    L = boundary(optin - 256)
    assert fp32_bytes(L) <= optin - 256 < fp32_bytes(L + 8)
    h = qc_code(L)
    g = q.Graph.from_csr(h)
    e = w.iid_x_errors(h.n, 0.02, 200, seed=5)
    s = w.syndromes(h, e)
    prior = np.full(h.n, w.prior_llr(0.02), dtype=np.float32)
    st, pt = torch.from_numpy(s).cuda(), torch.from_numpy(prior).cuda()
    err, iters, ok, post = q.decode(g, st, pt, 30, 0.75, "fp32", want_post=True)
    torch.cuda.synchronize()
    ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s, prior, 30, 0.75, "f32", threads=16)
    np.testing.assert_array_equal(err.cpu().numpy(), ref["err"])
    np.testing.assert_array_equal(iters.cpu().numpy(), ref["iters"])
    np.testing.assert_array_equal(post.cpu().numpy(), ref["post"])
    assert ref["ok"].mean() > 0.5
    # sizes up to the first whose shot exceeds the limit itself: decoded or refused, never a
    # launch failure; that first size is refused and still decodes in INT16
    Lx = boundary(optin) + 8
    for Lm in range(L + 8, Lx, 8):
        hm = qc_code(Lm)
        gm = q.Graph.from_csr(hm)
        try:
            q.decode(gm, torch.zeros((4, hm.m), dtype=torch.uint8, device="cuda"),
                     torch.full((hm.n,), 3.0, device="cuda"), 10, precision="fp32")
        except q.QldpcError as ex:
            assert ex.status == q.QLDPC_ERR_UNSUPPORTED
        gm.close()
    big = qc_code(Lx)
    gb = q.Graph.from_csr(big)            # INT16 still fits, so the graph itself is accepted
    assert gb.footprint("fp32")[1] > optin >= gb.footprint("int16")[1]
    sb = torch.zeros((4, big.m), dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QldpcError) as ei:
        q.decode(gb, sb, torch.full((big.n,), 3.0, device="cuda"), 10, precision="fp32")
    assert ei.value.status == q.QLDPC_ERR_UNSUPPORTED
    q.decode(gb, sb, torch.full((big.n,), 3.0, device="cuda"), 10, precision="int16")
    torch.cuda.synchronize()


def test_two_million_shots_in_one_call(q):
    h = w.hgp_code(400).hz_csr
    g = q.Graph.from_csr(h)
    B = 1 << 21
    err_true, syn = q.sample_errors(g, 2024, 0, B, 0.05)
    prior = torch.full((h.n,), w.prior_llr(0.05), device="cuda")
    err, iters, ok, _ = q.decode(g, syn, prior, 32, 0.75, "fp32")
    torch.cuda.synchronize()
    # every shot that reports success meets its syndrome (checked on the device, in chunks)
    hd = torch.from_numpy(h.dense().astype(np.float32)).cuda()
    for lo in range(0, B, 1 << 18):
        okm = ok[lo:lo + (1 << 18)].bool()
        s_hat = (err[lo:lo + (1 << 18)][okm].float() @ hd.T).remainder(2).to(torch.uint8)
        assert torch.equal(s_hat, syn[lo:lo + (1 << 18)][okm])
    assert 0.4 < ok.float().mean().item() < 0.6      # the oracle decodes 48 % of HGP-400 shots at p = 0.05
    # sampled shots across the whole range against the oracle
    idx = np.unique(np.random.default_rng(0).integers(0, B, 400))
    idx = np.concatenate([idx, [0, B - 1]])
    s_host = syn[torch.from_numpy(idx).cuda()].cpu().numpy()
    ref = oracle.msa(h.row_ptr, h.col_idx, h.m, h.n, s_host, np.full(h.n, w.prior_llr(0.05), np.float32), 32, 0.75,
                     "f32", threads=16)
    sel = torch.from_numpy(idx).cuda()
    np.testing.assert_array_equal(err[sel].cpu().numpy(), ref["err"])
    np.testing.assert_array_equal(iters[sel].cpu().numpy(), ref["iters"])
    np.testing.assert_array_equal(ok[sel].cpu().numpy(), ref["ok"])
