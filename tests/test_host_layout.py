"""The library's host-side graph layout, checked on the CPU (no GPU needed).

tests/host_layout_probe.cpp runs validate_and_layout from qldpc_host.cpp on a CSR matrix and
prints what it builds; this file checks it against the matrix:
  * variable lanes: a permutation of the variables plus idle lanes, degrees non-increasing, each
    lane's slots the slots j*m + i of its edges in ascending check order, idle lanes on scratch slots
    in free banks and at their warp's degree;
  * the magic number: floor(slot / m) exact for every slot;
  * bank packing: no conflicts in the variable step for the lift-31 code, fewer than the plain
    order for the others; each warp's halves chosen for 8-byte slots;
  * layers: checks of a layer share no variable, and each check sits one above the highest
    earlier check it shares a variable with.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2508_07879_gb300 import workloads as w

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path_factory.mktemp("probe") / "host_layout_probe")
    subprocess.check_call([nvcc, "-std=c++17", "-O1", "-I" + os.path.join(ROOT, "include"),
                           os.path.join(HERE, "host_layout_probe.cpp"), "-o", exe])
    return exe


def layout(exe, h):
    inp = f"{h.m} {h.n} {h.nnz}\n" + " ".join(map(str, h.row_ptr)) + "\n" + " ".join(map(str, h.col_idx)) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    d = {}
    for line in out.splitlines():
        k, *v = line.split()
        d[k] = np.array([int(x) for x in v], dtype=np.int64)
    return d


def wavefronts(words):
    banks = {}
    for a in words:
        banks.setdefault(a % 32, set()).add(a)
    return max(len(s) for s in banks.values())


def vn_wavefronts(vslot, vdeg, nv, lanes_real):
    total = 0
    for w0 in range(0, nv, 32):
        lanes = range(w0, min(nv, w0 + 32))
        for k in range(int(vdeg[w0:w0 + 32].max())):
            words = [int(vslot[k * nv + u]) for u in lanes if k < vdeg[u] and lanes_real[u]]
            if words:
                total += wavefronts(words)
    return total


CODES = {
    "lp1054": lambda: w.lp_code(1054).hz_csr,
    "lp1054x": lambda: w.lp_code(1054).hx_csr,
    "hgp400": lambda: w.hgp_code(400).hz_csr,
    "bb144": lambda: w.bb_code(12, 6).hz_csr,
    "bb288": lambda: w.bb_code(12, 12).hx_csr,
    "eq1": lambda: w.csr_from_dense(w.eq1_pcm()),
}


@pytest.mark.parametrize("name", list(CODES))
def test_variable_lanes(probe, name):
    h = CODES[name]()
    d = layout(probe, h)
    assert d["rc"][0] == 0
    dc, dv, nv, _ = (int(x) for x in d["dims"])
    m, n = h.m, h.n
    vorder, vdeg, vslot = d["vorder"], d["vdeg"], d["vslot"].reshape(max(dv, 1), nv)
    real = vorder < n
    assert sorted(vorder[real].tolist()) == list(range(n))          # each variable in exactly one lane
    assert (vorder[~real] == n).all()
    if (~real).any():
        assert nv % 32 == 0                                          # packed warps are whole
    assert (np.diff(vdeg) <= 0).all()                                # non-increasing degrees
    # each real lane's slots: j*m + i over its edges in ascending check order
    want = [[] for _ in range(n)]
    for i in range(m):
        for j, v in enumerate(h.col_idx[h.row_ptr[i]:h.row_ptr[i + 1]]):
            want[v].append(j * m + i)
    for u in np.nonzero(real)[0]:
        v = int(vorder[u])
        assert vdeg[u] == len(want[v])
        assert vslot[:vdeg[u], u].tolist() == want[v]
    # idle lanes: scratch slots in free banks, their warp's degree
    for u in np.nonzero(~real)[0]:
        w0 = u - u % 32
        warp = [x for x in range(w0, min(nv, w0 + 32)) if real[x]]
        assert vdeg[u] == max(vdeg[x] for x in warp)
        for k in range(vdeg[u]):
            s = int(vslot[k, u])
            assert dc * m <= s < dc * m + 32
            assert s % 32 not in {int(vslot[k, x]) % 32 for x in warp if k < vdeg[x]}
    # the CSR edge -> slot map
    for i in range(m):
        for j, e in enumerate(range(h.row_ptr[i], h.row_ptr[i + 1])):
            assert d["eslot"][e] == j * m + i


@pytest.mark.parametrize("name", list(CODES))
def test_magic_division_is_exact(probe, name):
    h = CODES[name]()
    d = layout(probe, h)
    dc = int(d["dims"][0])
    magic, shift = (int(x) for x in d["magic"])
    if h.m == 1:
        return
    x = np.arange(dc * h.m + 32, dtype=np.uint64)
    np.testing.assert_array_equal((x * np.uint64(magic)) >> np.uint64(32 + shift), x // np.uint64(h.m))


def test_bank_packing(probe):
    h = w.lp_code(1054).hz_csr
    d = layout(probe, h)
    dc, dv, nv, _ = (int(x) for x in d["dims"])
    real = d["vorder"] < h.n
    got = vn_wavefronts(d["vslot"], d["vdeg"], nv, real)
    accesses = sum(int(d["vdeg"][w0:w0 + 32].max()) for w0 in range(0, nv, 32))
    assert nv == 1088 and got == accesses                           # conflict-free: one wavefront each
    # the plain degree order of the same code (what the packing replaced) needs more
    deg = np.bincount(h.col_idx, minlength=h.n)
    order = sorted(range(h.n), key=lambda v: -deg[v])
    slots = [[] for _ in range(h.n)]
    for i in range(h.m):
        for j, v in enumerate(h.col_idx[h.row_ptr[i]:h.row_ptr[i + 1]]):
            slots[v].append(j * h.m + i)
    plain = 0
    for w0 in range(0, h.n, 32):
        lanes = order[w0:w0 + 32]
        for k in range(max(deg[v] for v in lanes)):
            plain += wavefronts([slots[v][k] for v in lanes if k < deg[v]])
    assert plain > 1.5 * got


def half_wavefronts(vslot, vdeg, nv):
    """Wavefronts of the variable step with 8-byte slot words (the paired FP32 messages): a half-warp
    per wavefront over 16 bank pairs; idle lanes included (their scratch slots are accessed too)."""
    total = 0
    for w0 in range(0, nv, 32):
        for k in range(int(vdeg[w0:w0 + 32].max())):
            for h0 in (w0, w0 + 16):
                words = [int(vslot[k * nv + u]) for u in range(h0, min(nv, h0 + 16)) if k < vdeg[u]]
                if words:
                    banks = {}
                    for a in words:
                        banks.setdefault(a % 16, set()).add(a)
                    total += max(len(x) for x in banks.values())
    return total


def test_half_warp_split_for_8_byte_slots(probe):
    """Each warp's lanes are split into halves that suit 8-byte slots without changing the warp's
    4-byte banks: LP-1054's variable step takes 298 half-warp wavefronts (the 4-byte packing in its
    own lane order: 366; conflict-free would be 240), and the 4-byte accesses stay conflict-free."""
    h = w.lp_code(1054).hz_csr
    d = layout(probe, h)
    nv = int(d["dims"][2])
    assert half_wavefronts(d["vslot"], d["vdeg"], nv) <= 300
    assert vn_wavefronts(d["vslot"], d["vdeg"], nv, np.ones(nv, dtype=bool)) == \
        sum(int(d["vdeg"][w0:w0 + 32].max()) for w0 in range(0, nv, 32))   # idle lanes included


@pytest.mark.parametrize("name", list(CODES))
def test_layers(probe, name):
    h = CODES[name]()
    d = layout(probe, h)
    ptr, chk = d["layer_ptr"], d["layer_chk"]
    assert sorted(chk.tolist()) == list(range(h.m))
    layer = np.empty(h.m, dtype=np.int64)
    for l in range(len(ptr) - 1):
        cs = chk[ptr[l]:ptr[l + 1]]
        assert (np.diff(cs) > 0).all()
        layer[cs] = l
        vs = np.concatenate([h.col_idx[h.row_ptr[c]:h.row_ptr[c + 1]] for c in cs])
        assert len(np.unique(vs)) == len(vs)                         # no shared variable in a layer
    last = np.full(h.n, -1)
    for i in range(h.m):
        cols = h.col_idx[h.row_ptr[i]:h.row_ptr[i + 1]]
        assert layer[i] == last[cols].max() + 1                      # as soon as possible
        last[cols] = layer[i]


def test_rejects_malformed(probe):
    bad = w.CSR(np.array([0, 1], dtype=np.int32), np.array([0], dtype=np.int32), 1, 3)   # a row of degree 1
    assert layout(probe, bad)["rc"][0] == -1
