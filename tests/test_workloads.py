"""Input generators: code invariants (Sec. 2 CSS condition, degrees, k) and sampler behaviour."""
import numpy as np
import pytest

from paper_2508_07879_gb300 import gf2
from paper_2508_07879_gb300 import workloads as w

SHAPES = {   # name: (checks per H, N, row degree, column degrees, edges per H)
    "hgp400": (192, 400, {7}, {3, 4}, 1344),
    "lp1054": (465, 1054, {8}, {3, 5}, 3720),
    "bb144": (72, 144, {6}, {3}, 432),
    "bb288": (144, 288, {6}, {3}, 864),
}


@pytest.mark.parametrize("name", sorted(SHAPES))
def test_css_code_shapes_and_commutativity(name):
    code = w.CONFIG_CODES[name]()
    m, n, dc, dv, e = SHAPES[name]
    for h in (code.hx, code.hz):
        assert h.shape == (m, n)
        assert set(h.sum(axis=1).tolist()) == dc
        assert set(h.sum(axis=0).tolist()) == dv
        assert int(h.sum()) == e
    # CSS commutativity condition H_X H_Z^T = 0 over GF(2) (Sec. 2)
    assert not ((code.hx.astype(np.int64) @ code.hz.T.astype(np.int64)) % 2).any()


def test_bb144_is_the_papers_144_12_code():
    # [[144,12,12]] of Bravyi et al. (the paper's Sec. 3 code list): k = 12
    code = w.bb_code(12, 6)
    assert code.n == 144 and gf2.css_dimension(code.hx, code.hz) == 12


def test_bb288_sibling_dimension():
    # the same polynomials on the 12 x 12 torus give k = 16 (not the paper's [[288,12,18]])
    code = w.bb_code(12, 12)
    assert gf2.css_dimension(code.hx, code.hz) == 16


def test_hgp_dimension_formula():
    # k(HGP(H, H)) = (n_c - r)^2 + (m_c - r)^2 for an m_c x n_c classical H of rank r
    h = w.random_regular_ldpc(12, 16, 3, 4, 400)
    r = gf2.rank(h)
    code = w.hgp_code(400)
    assert gf2.css_dimension(code.hx, code.hz) == (16 - r) ** 2 + (12 - r) ** 2


def test_random_regular_is_seeded_and_regular():
    a = w.random_regular_ldpc(12, 16, 3, 4, 400)
    b = w.random_regular_ldpc(12, 16, 3, 4, 400)
    c = w.random_regular_ldpc(12, 16, 3, 4, 401)
    np.testing.assert_array_equal(a, b)
    assert (a != c).any()
    assert (a.sum(0) == 3).all() and (a.sum(1) == 4).all()


def test_logical_basis_properties():
    code = w.bb_code(12, 6)
    L = gf2.logical_basis(code.hx, code.hz)
    assert L.shape == (12, 144)
    assert not ((code.hx.astype(np.int64) @ L.T.astype(np.int64)) % 2).any()
    assert gf2.rank(np.vstack([code.hz, L])) == gf2.rank(code.hz) + 12
    # stabilizers (rows of H_X) are never flagged as logical failures
    assert not gf2.logical_failures(code.hx, L).any()
    # and each logical of the dual type (in ker H_Z, outside rowspace H_X) is flagged
    assert gf2.logical_failures(gf2.logical_basis(code.hz, code.hx), L).all()


def test_splitmix64_reference_values():
    # SplitMix64 from state 0 (Steele, Lea, Flood 2014; the widely published first outputs)
    assert int(w.splitmix64(np.uint64(0))) == 0xE220A8397B1DCDAF
    s = w._Stream(0)
    assert [s.next() for _ in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_sampler_is_counter_based():
    full = w.iid_x_errors(300, 0.05, 40, seed=7)
    part = w.iid_x_errors(300, 0.05, 10, seed=7, first_shot=25)
    np.testing.assert_array_equal(full[25:35], part)
    assert (w.iid_x_errors(300, 0.05, 40, seed=8) != full).any()


def test_sampler_rates():
    e = w.iid_x_errors(1000, 0.03, 400, seed=1)
    rate = e.mean()
    assert abs(rate - 0.03) < 5 * np.sqrt(0.03 * 0.97 / e.size)
    ex, ez = w.depolarizing_errors(1000, 0.06, 400, seed=2)
    for part in (ex, ez):
        assert abs(part.mean() - 0.04) < 5 * np.sqrt(0.04 * 0.96 / part.size)
    both = (ex & ez).mean()            # Y errors: p/3
    assert abs(both - 0.02) < 5 * np.sqrt(0.02 * 0.98 / ex.size)


def test_syndromes_match_dense_product():
    code = w.lp_code(1054)
    h = code.hz_csr
    e = w.iid_x_errors(code.n, 0.05, 20, seed=3)
    s = w.syndromes(h, e)
    np.testing.assert_array_equal(s, (e.astype(np.int64) @ code.hz.T.astype(np.int64)) % 2)


def test_csr_roundtrip():
    code = w.hgp_code(400)
    h = code.hz_csr
    np.testing.assert_array_equal(h.dense(), code.hz)
    assert h.nnz == 1344


def test_prange_sampler_rates_and_keying():
    e, p = w.iid_x_errors_prange(200, 0.02, 0.06, 5000, seed=8)
    assert e.shape == (5000, 200) and p.shape == (5000,)
    assert 0.02 <= p.min() and p.max() < 0.06
    assert abs(p.mean() - 0.04) < 1e-3
    # flips follow each shot's own rate: binned error density tracks the bin's mean rate
    order = np.argsort(p)
    for chunk in np.array_split(order, 5):
        assert abs(e[chunk].mean() - p[chunk].mean()) < 3e-3
    # the rate uses counter n and the flips counters 0..n-1 of the same key
    u = w.uniform01(8, np.arange(3), np.arange(201))
    np.testing.assert_array_equal(p[:3], 0.02 + (0.06 - 0.02) * u[:, 200])
    np.testing.assert_array_equal(e[:3], (u[:, :200] < p[:3, None]).astype(np.uint8))
    e2, p2 = w.iid_x_errors_prange(200, 0.02, 0.06, 10, seed=8, first_shot=4990)
    np.testing.assert_array_equal(e2, e[4990:])
