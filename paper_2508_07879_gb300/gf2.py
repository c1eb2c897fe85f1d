"""GF(2) linear algebra for the evaluation harness: rank, code dimension and logical failures.

Decoding itself never calls this module.  It answers two questions about decoder *outputs*:

* the number of logical qubits k = N - rank(H_X) - rank(H_Z) of a CSS code (Sec. 3 names codes
  by [[n, k, d]]);
* whether a residual r = e XOR e_hat of a converged X-error decode (H_Z r^T = 0) is a stabilizer
  (harmless: r in rowspace(H_X)) or a logical operator (a decoding failure).

Rows are bit-packed into uint64 words so elimination on the 465 x 1054 lifted-product matrices
takes milliseconds.
"""
from __future__ import annotations

import numpy as np


def _pack(mat: np.ndarray) -> np.ndarray:
    mat = np.asarray(mat, dtype=np.uint8) & 1
    r, c = mat.shape
    words = (c + 63) // 64
    padded = np.zeros((r, words * 64), dtype=np.uint8)
    padded[:, :c] = mat
    bits = padded.reshape(r, words, 64)
    weights = (np.uint64(1) << np.arange(64, dtype=np.uint64))
    return (bits.astype(np.uint64) * weights).sum(axis=2, dtype=np.uint64)


def _unpack(words: np.ndarray, c: int) -> np.ndarray:
    r = words.shape[0]
    bits = (words[:, :, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
    return bits.reshape(r, -1)[:, :c].astype(np.uint8)


def row_echelon(mat: np.ndarray):
    """Reduced row echelon form over GF(2).  Returns (packed rows, pivot columns)."""
    a = _pack(mat).copy()
    r, _ = a.shape
    c = np.asarray(mat).shape[1]
    pivots = []
    row = 0
    for col in range(c):
        if row >= r:
            break
        w, b = divmod(col, 64)
        bit = np.uint64(1) << np.uint64(b)
        hits = np.nonzero(a[row:, w] & bit)[0]
        if hits.size == 0:
            continue
        p = row + hits[0]
        if p != row:
            a[[row, p]] = a[[p, row]]
        others = np.nonzero(a[:, w] & bit)[0]
        others = others[others != row]
        a[others] ^= a[row]
        pivots.append(col)
        row += 1
    return a[:row], pivots


def rank(mat: np.ndarray) -> int:
    return len(row_echelon(mat)[1])


def css_dimension(hx: np.ndarray, hz: np.ndarray) -> int:
    """k = N - rank(H_X) - rank(H_Z)."""
    return hx.shape[1] - rank(hx) - rank(hz)


def nullspace(mat: np.ndarray) -> np.ndarray:
    """Basis (rows) of {v : mat v^T = 0} over GF(2)."""
    mat = np.asarray(mat, dtype=np.uint8) & 1
    c = mat.shape[1]
    red, piv = row_echelon(mat)
    red = _unpack(red, c)
    free = [j for j in range(c) if j not in set(piv)]
    basis = np.zeros((len(free), c), dtype=np.uint8)
    for i, f in enumerate(free):
        basis[i, f] = 1
        for r, p in enumerate(piv):
            if red[r, f]:
                basis[i, p] = 1
    return basis


def logical_basis(h_same: np.ndarray, h_other: np.ndarray) -> np.ndarray:
    """Logical operators that detect residuals of the type h_same's rowspace stabilizes.

    For X errors decoded with H_Z (residual r in ker H_Z), pass h_same = H_X, h_other = H_Z:
    returns k rows L in ker(H_X) independent modulo rowspace(H_Z).  A residual r with H_Z r = 0 is
    a stabilizer iff L r^T = 0 for every row L.
    """
    ker = nullspace(h_same)
    c = ker.shape[1]
    red, piv = row_echelon(h_other)
    basis = [row for row in red]          # packed rows, each with a leading pivot bit
    lead = list(piv)
    out = []
    for v in ker:
        x = _pack(v[None, :])[0].copy()
        for row, p in zip(basis, lead):
            w, b = divmod(p, 64)
            if (x[w] >> np.uint64(b)) & np.uint64(1):
                x ^= row
        nz = np.nonzero(x)[0]
        if nz.size == 0:
            continue
        w = nz[0]
        low = (int(x[w]) & -int(x[w])).bit_length() - 1
        p = w * 64 + low
        # keep the basis reduced: clear the new pivot bit from every earlier row
        pw, pb = divmod(p, 64)
        for i, row in enumerate(basis):
            if (row[pw] >> np.uint64(pb)) & np.uint64(1):
                basis[i] = row ^ x
        basis.append(x)
        lead.append(p)
        out.append(v)
    return np.array(out, dtype=np.uint8).reshape(-1, c)


def logical_failures(residual: np.ndarray, logicals: np.ndarray) -> np.ndarray:
    """failure[b] = any over L of <L, residual[b]> mod 2  (residuals assumed in ker of the decoder's H)."""
    residual = np.asarray(residual, dtype=np.uint8)
    prod = residual.astype(np.int64) @ logicals.T.astype(np.int64)
    return (prod % 2).any(axis=1)
