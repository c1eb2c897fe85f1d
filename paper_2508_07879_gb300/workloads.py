"""Seeded synthetic inputs for syndrome decoding: parity-check matrices and error samples.

This module builds the codes and the noise that both the CUDA decoder and the CPU oracle are
fed. It holds none of the decoder's arithmetic (no message passing, no decisions); it only
produces H matrices in CSR form, error vectors and their syndromes s = H e^T mod 2.

Codes
-----
* ``eq1_pcm()``: the 3x6 example parity-check matrix printed as Eq. (1) of the paper (Sec. 2).
* ``hgp_code(seed)``: hypergraph product of a seeded random (3,4)-regular 12x16 classical H,
  H_X = [H (x) I16 | I12 (x) H^T], H_Z = [I16 (x) H | H^T (x) I12]  (N = 400, 192 checks each).
* ``lp_code(seed)``: quasi-cyclic lifted product over F2[x]/(x^31 - 1) of a seeded 3x5 base matrix
  of monomials, H_X = [A (x) I5 | I3 (x) A*], H_Z = [I5 (x) A | A* (x) I3]  (N = 1054, 465 checks).
* ``bb_code(l, m)``: bivariate-bicycle code with A = x^3 + y + y^2, B = y^3 + x + x^2,
  H_X = [A | B], H_Z = [B^T | A^T]  (l=12, m=6 gives the [[144,12,12]] code of the paper's Sec. 3).

Every CSS pair satisfies H_X H_Z^T = 0 (the commutativity condition of Sec. 2).

Noise
-----
A counter-based SplitMix64 generator (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) keyed by (seed, shot, qubit) draws every random number, so a shot's error
does not depend on the batch it is drawn in.  ``iid_x_errors`` draws Bernoulli(p) bit flips (``iid_x_errors_prange`` at a rate drawn per shot);
``depolarizing_errors`` draws X, Y, Z with probability p/3 each and splits them into the X part
(X or Y) and the Z part (Z or Y).  Per Sec. 2, s_X = H_Z e_X^T is decoded with H_Z and
s_Z = H_X e_Z^T with H_X.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


# --------------------------------------------------------------------------------------------
# SplitMix64 (Steele, Lea, Flood 2014), counter-based use
# --------------------------------------------------------------------------------------------
def splitmix64(x):
    """SplitMix64 output function applied to state ``x`` (uint64, scalar or array).

    Returns the generator's output for the state x + golden gamma, i.e. one step of
    SplitMix64 started from state ``x``.  Arithmetic wraps modulo 2^64.
    """
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        return z ^ (z >> np.uint64(31))


def uniform01(seed: int, shots, qubits) -> np.ndarray:
    """Counter-based uniforms in [0, 1): u[b, q] = top 53 bits of mix(mix(mix(seed)+shot)+qubit) / 2^53.

    ``shots`` and ``qubits`` are 1-D integer arrays; the result has shape (len(shots), len(qubits)).
    """
    shots = np.asarray(shots, dtype=np.uint64)
    qubits = np.asarray(qubits, dtype=np.uint64)
    with np.errstate(over="ignore"):
        k_seed = splitmix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF))
        k_shot = splitmix64(k_seed + shots)                      # (B,)
        x = splitmix64(k_shot[:, None] + qubits[None, :])        # (B, Q)
    return (x >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class _Stream:
    """Sequential SplitMix64 stream used only to build seeded random codes."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next(self) -> int:
        out = int(splitmix64(self.state))
        with np.errstate(over="ignore"):
            self.state = self.state + _GOLDEN
        return out

    def below(self, k: int) -> int:
        """Integer in [0, k) (plain modulo reduction; the bias is < 2^-58 for k < 64)."""
        return self.next() % k


# --------------------------------------------------------------------------------------------
# Sparse helpers
# --------------------------------------------------------------------------------------------
@dataclass(frozen=True)
class CSR:
    """Parity-check matrix in CSR form: row m holds the columns col_idx[row_ptr[m]:row_ptr[m+1]]."""

    row_ptr: np.ndarray   # int32 [m+1]
    col_idx: np.ndarray   # int32 [nnz], ascending within each row
    m: int
    n: int

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        h = np.zeros((self.m, self.n), dtype=np.uint8)
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        h[rows, self.col_idx] = 1
        return h

    def row_degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def col_degrees(self) -> np.ndarray:
        return np.bincount(self.col_idx, minlength=self.n)


def csr_from_dense(h) -> CSR:
    h = np.asarray(h, dtype=np.uint8) & 1
    m, n = h.shape
    rows, cols = np.nonzero(h)            # row-major order: columns ascend within a row
    row_ptr = np.zeros(m + 1, dtype=np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr).astype(np.int32)
    return CSR(row_ptr=row_ptr, col_idx=cols.astype(np.int32), m=m, n=n)


def syndromes(h: CSR, errors: np.ndarray) -> np.ndarray:
    """s[b, m] = XOR over n in row m of errors[b, n]  (s = H e^T over GF(2), Sec. 2)."""
    errors = np.asarray(errors, dtype=np.uint8)
    if errors.ndim == 1:
        errors = errors[None, :]
    out = np.zeros((errors.shape[0], h.m), dtype=np.uint8)
    deg = h.row_degrees()
    for d in np.unique(deg):
        rows = np.nonzero(deg == d)[0]
        if d == 0:
            continue
        cols = h.col_idx[h.row_ptr[rows][:, None] + np.arange(d)[None, :]]   # (R, d)
        out[:, rows] = np.bitwise_xor.reduce(errors[:, cols], axis=2)
    return out


# --------------------------------------------------------------------------------------------
# Codes
# --------------------------------------------------------------------------------------------
def eq1_pcm() -> np.ndarray:
    """The 3x6 parity-check matrix of Eq. (1) (Sec. 2): d_c = 4, d_v = 2."""
    return np.array([[1, 0, 1, 1, 0, 1],
                     [1, 1, 0, 1, 1, 0],
                     [0, 1, 1, 0, 1, 1]], dtype=np.uint8)


def random_regular_ldpc(rows: int, cols: int, dv: int, dc: int, seed: int) -> np.ndarray:
    """Seeded (dv, dc)-regular rows x cols binary matrix by the configuration model.

    Each column contributes dv sockets; the rows*dc sockets are shuffled by Fisher-Yates with
    a SplitMix64 stream and dealt dc per row.  A draw that puts the same column twice in a row
    is rejected and the shuffle repeated on the continuing stream.
    """
    assert rows * dc == cols * dv
    rng = _Stream(seed)
    sockets = np.repeat(np.arange(cols), dv)
    while True:
        s = sockets.copy()
        for i in range(len(s) - 1, 0, -1):
            j = rng.below(i + 1)
            s[i], s[j] = s[j], s[i]
        dealt = s.reshape(rows, dc)
        if all(len(set(r.tolist())) == dc for r in dealt):
            h = np.zeros((rows, cols), dtype=np.uint8)
            for r, cs in enumerate(dealt):
                h[r, cs] = 1
            return h


@dataclass(frozen=True)
class CSSCode:
    name: str
    hx: np.ndarray     # dense uint8 [mx, n]
    hz: np.ndarray     # dense uint8 [mz, n]

    @property
    def n(self) -> int:
        return self.hx.shape[1]

    @property
    def hx_csr(self) -> CSR:
        return csr_from_dense(self.hx)

    @property
    def hz_csr(self) -> CSR:
        return csr_from_dense(self.hz)


def hgp_code(seed: int = 400, rows: int = 12, cols: int = 16) -> CSSCode:
    """Hypergraph-product code of a seeded (3,4)-regular rows x cols H (N = cols^2 + rows^2)."""
    h = random_regular_ldpc(rows, cols, 3, 4, seed)
    i_r = np.eye(rows, dtype=np.uint8)
    i_c = np.eye(cols, dtype=np.uint8)
    hx = np.hstack([np.kron(h, i_c), np.kron(i_r, h.T)]) & 1
    hz = np.hstack([np.kron(i_c, h), np.kron(h.T, i_r)]) & 1
    return CSSCode(f"hgp{hx.shape[1]}", hx.astype(np.uint8), hz.astype(np.uint8))


def _circulant(a: int, L: int) -> np.ndarray:
    """L x L permutation matrix of the monomial x^a: P[i, (i + a) mod L] = 1."""
    p = np.zeros((L, L), dtype=np.uint8)
    p[np.arange(L), (np.arange(L) + a) % L] = 1
    return p


def _ring_kron(a, b):
    """Kronecker product of two matrices over F2[x]/(x^L - 1).

    An entry is a tuple of exponents (the polynomial with those monomials, () being 0); the
    product of two entries is the tuple of all pairwise exponent sums (reduced mod L and
    cancelled in pairs when the matrix is expanded).
    """
    ra, ca = len(a), len(a[0])
    rb, cb = len(b), len(b[0])
    out = [[() for _ in range(ca * cb)] for _ in range(ra * rb)]
    for i in range(ra):
        for j in range(ca):
            for k in range(rb):
                for l in range(cb):
                    out[i * rb + k][j * cb + l] = tuple(x + y for x in a[i][j] for y in b[k][l])
    return out


def _ring_expand(mat, L: int) -> np.ndarray:
    """Replace each polynomial entry by the sum over F2 of its L x L circulant permutations."""
    rows, cols = len(mat), len(mat[0])
    out = np.zeros((rows * L, cols * L), dtype=np.uint8)
    for i in range(rows):
        for j in range(cols):
            block = np.zeros((L, L), dtype=np.uint8)
            for e in mat[i][j]:
                block ^= _circulant(e % L, L)
            out[i * L:(i + 1) * L, j * L:(j + 1) * L] = block
    return out


def lp_code(seed: int = 1054, L: int = 31, base_rows: int = 3, base_cols: int = 5) -> CSSCode:
    """Quasi-cyclic lifted-product code of a seeded base matrix of monomials.

    A[i][j] = x^{a_ij} with a_ij drawn row-major from a SplitMix64 stream in [0, L).
    A* is the block transpose with exponents negated mod L (the transpose of the lifted matrix).
    H_X = [A (x) I_c | I_r (x) A*],  H_Z = [I_c (x) A | A* (x) I_r]  with r = base_rows, c = base_cols.
    """
    rng = _Stream(seed)
    a = [[(rng.below(L),) for _ in range(base_cols)] for _ in range(base_rows)]
    a_star = [[((-a[i][j][0]) % L,) for i in range(base_rows)] for j in range(base_cols)]
    eye = lambda k: [[(0,) if i == j else () for j in range(k)] for i in range(k)]
    hx = np.hstack([_ring_expand(_ring_kron(a, eye(base_cols)), L),
                    _ring_expand(_ring_kron(eye(base_rows), a_star), L)])
    hz = np.hstack([_ring_expand(_ring_kron(eye(base_cols), a), L),
                    _ring_expand(_ring_kron(a_star, eye(base_rows)), L)])
    return CSSCode(f"lp{hx.shape[1]}", hx & 1, hz & 1)


def bb_code(l: int = 12, m: int = 6) -> CSSCode:
    """Bivariate-bicycle code: x = S_l (x) I_m, y = I_l (x) S_m, A = x^3 + y + y^2, B = y^3 + x + x^2."""
    s_l = _circulant(1, l)
    s_m = _circulant(1, m)
    x = np.kron(s_l, np.eye(m, dtype=np.uint8))
    y = np.kron(np.eye(l, dtype=np.uint8), s_m)
    mp = np.linalg.matrix_power
    a = (mp(x, 3) + y + mp(y, 2)) % 2
    b = (mp(y, 3) + x + mp(x, 2)) % 2
    hx = np.hstack([a, b]).astype(np.uint8)
    hz = np.hstack([b.T, a.T]).astype(np.uint8)
    return CSSCode(f"bb{2 * l * m}", hx, hz)


# --------------------------------------------------------------------------------------------
# Noise
# --------------------------------------------------------------------------------------------
def prior_llr(p: float) -> float:
    """Channel log-likelihood ratio ln((1 - p) / p) used as the decoder prior gamma_n."""
    return math.log((1.0 - p) / p)


def _chunked(fn, shots: int, first_shot: int, chunk: int = 4096):
    """Evaluate fn(first, count) over shot chunks on a thread pool (numpy releases the GIL);
    chunking does not change the result because every draw is keyed by its absolute shot index."""
    from concurrent.futures import ThreadPoolExecutor
    starts = list(range(0, shots, chunk))
    if len(starts) <= 1:
        return fn(first_shot, shots)
    workers = min(len(starts), os.cpu_count() or 1)
    with ThreadPoolExecutor(workers) as ex:
        parts = list(ex.map(lambda s0: fn(first_shot + s0, min(chunk, shots - s0)), starts))
    if isinstance(parts[0], tuple):
        return tuple(np.concatenate([p[i] for p in parts]) for i in range(len(parts[0])))
    return np.concatenate(parts)


def iid_x_errors(n: int, p: float, shots: int, seed: int, first_shot: int = 0) -> np.ndarray:
    """Bernoulli(p) bit flips, e[b, q] = [u(seed, first_shot + b, q) < p]  (uint8 [shots, n])."""
    def draw(s0, count):
        u = uniform01(seed, np.arange(s0, s0 + count), np.arange(n))
        return (u < p).astype(np.uint8)
    return _chunked(draw, shots, first_shot)


def iid_x_errors_prange(n: int, p_lo: float, p_hi: float, shots: int, seed: int, first_shot: int = 0):
    """Bernoulli flips at a per-shot rate drawn uniformly from [p_lo, p_hi).

    p_b = p_lo + (p_hi - p_lo) * u(seed, b, n)   (counter n: one past the last qubit)
    e[b, q] = [u(seed, b, q) < p_b]              for q < n
    Returns (uint8 errors [shots, n], float64 rates [shots]).  The same definition drives the
    device sampler used for training the learned decoder.
    """
    def draw(s0, count):
        u = uniform01(seed, np.arange(s0, s0 + count), np.arange(n + 1))
        p = p_lo + (p_hi - p_lo) * u[:, n]
        return (u[:, :n] < p[:, None]).astype(np.uint8), p
    return _chunked(draw, shots, first_shot)


def depolarizing_errors(n: int, p: float, shots: int, seed: int, first_shot: int = 0):
    """Depolarizing noise split into (e_X, e_Z): u < p/3 -> X, < 2p/3 -> Y, < p -> Z.

    e_X marks X or Y, e_Z marks Z or Y.  Each part has marginal probability 2p/3.
    """
    def draw(s0, count):
        u = uniform01(seed, np.arange(s0, s0 + count), np.arange(n))
        x = u < p / 3.0
        y = (u >= p / 3.0) & (u < 2.0 * p / 3.0)
        z = (u >= 2.0 * p / 3.0) & (u < p)
        return (x | y).astype(np.uint8), (z | y).astype(np.uint8)
    return _chunked(draw, shots, first_shot)


def data_syndrome_csr(h: CSR) -> CSR:
    """The data-syndrome Tanner graph [H | I_m]: column n + i is the measurement error of syndrome
    bit i (one edge, to check i).  A syndrome read with errors, s~ = H e + e', is the syndrome of
    the combined error (e, e') on this graph."""
    rp = np.asarray(h.row_ptr, dtype=np.int64)
    cols = []
    for i in range(h.m):
        cols.append(np.asarray(h.col_idx[rp[i]:rp[i + 1]], dtype=np.int32))
        cols.append(np.array([h.n + i], dtype=np.int32))
    row_ptr = (rp + np.arange(h.m + 1)).astype(np.int32)
    return CSR(row_ptr, np.concatenate(cols) if cols else np.zeros(0, np.int32), h.m, h.n + h.m)


def csr_rows(h: CSR, order) -> CSR:
    """H with its rows permuted: row i of the result is row order[i] of h (same columns).  The
    syndrome of the result is s[:, order]."""
    order = np.asarray(order, dtype=np.int64)
    rp = np.asarray(h.row_ptr, dtype=np.int64)
    deg = rp[order + 1] - rp[order]
    row_ptr = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    cols = [np.asarray(h.col_idx[rp[i]:rp[i + 1]], dtype=np.int32) for i in order]
    return CSR(row_ptr, np.concatenate(cols) if cols else np.zeros(0, np.int32), h.m, h.n)


def layer_order(h: CSR) -> np.ndarray:
    """A row order for the layered schedule with few layers: rows that share a variable get
    different colours (greedy colouring, most-constrained row first), and rows are listed colour by
    colour in ascending index.  In that order every colour class is a set of rows without a common
    variable, so the as-soon-as-possible layering of the reordered matrix needs at most as many
    layers as there are colours.  (A different row order is a different layered schedule.)"""
    rp = np.asarray(h.row_ptr, dtype=np.int64)
    rows_of = [[] for _ in range(h.n)]
    for i in range(h.m):
        for v in h.col_idx[rp[i]:rp[i + 1]]:
            rows_of[int(v)].append(i)
    nbrs = [set() for _ in range(h.m)]
    for rows in rows_of:
        for a in rows:
            nbrs[a].update(rows)
    for i in range(h.m):
        nbrs[i].discard(i)
    colour = np.full(h.m, -1, dtype=np.int64)
    seen = [set() for _ in range(h.m)]          # colours of the coloured neighbours
    for _ in range(h.m):
        cand = [i for i in range(h.m) if colour[i] < 0]
        i = max(cand, key=lambda r: (len(seen[r]), len(nbrs[r]), -r))
        c = 0
        while c in seen[i]:
            c += 1
        colour[i] = c
        for j in nbrs[i]:
            seen[j].add(c)
    return np.lexsort((np.arange(h.m), colour))


def noisy_syndrome_batch(h: CSR, p: float, q: float, shots: int, seed: int, first_shot: int = 0):
    """Data errors at rate p and syndrome measurement errors at rate q, one draw per shot:
    e[b, j] = [u(seed, b, j) < p] for the n data bits, e'[b, i] = [u(seed, b, n + i) < q] for the m
    syndrome bits; returns (e uint8 [shots, n], e' uint8 [shots, m], s~ = H e + e' uint8 [shots, m])."""
    def draw(s0, count):
        u = uniform01(seed, np.arange(s0, s0 + count), np.arange(h.n + h.m))
        return (u[:, :h.n] < p).astype(np.uint8), (u[:, h.n:] < q).astype(np.uint8)
    e, es = _chunked(draw, shots, first_shot)
    return e, es, syndromes(h, e) ^ es


@dataclass(frozen=True)
class Batch:
    """One batch of synthetic decoding problems for a single parity-check matrix."""

    h: CSR
    errors: np.ndarray      # uint8 [B, n]
    syndromes: np.ndarray   # uint8 [B, m]
    prior: np.ndarray       # float32 [n]
    p: float


def x_error_batch(code: CSSCode, p: float, shots: int, seed: int, first_shot: int = 0) -> Batch:
    """i.i.d. X errors decoded with H_Z from s_X = H_Z e_X^T (Sec. 2), prior ln((1-p)/p)."""
    h = code.hz_csr
    e = iid_x_errors(code.n, p, shots, seed, first_shot)
    s = syndromes(h, e)
    prior = np.full(code.n, prior_llr(p), dtype=np.float32)
    return Batch(h, e, s, prior, p)


CONFIG_CODES = {
    "hgp400": lambda: hgp_code(400),
    "lp1054": lambda: lp_code(1054),
    "bb144": lambda: bb_code(12, 6),
    "bb288": lambda: bb_code(12, 12),
}
