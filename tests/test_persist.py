"""Saved plans (sptrsv_plan_save / sptrsv_plan_load) on the host (device = -1).

A loaded plan must export exactly the schedule that was saved, and a damaged
or mismatched file must be refused with an error, never accepted: a schedule
that breaks Def. 2.1, or a block-local partition out of (wavefront, id) order,
could make a polled solve wait on a row that never arrives."""
import os
import struct

import numpy as np
import pytest

import oracle
import workloads as W

sp = pytest.importorskip("paper_2503_05408_gb300")

HEADER = 56


@pytest.fixture(scope="module", autouse=True)
def _lib():
    try:
        sp.lib()
    except RuntimeError as e:
        pytest.skip(str(e))


def _same(p, q):
    a, b = p.export(), q.export()
    for f in ("level", "sigma", "pi", "perm"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f


CASES = [
    ("levels", dict(mode="levels"), lambda: W.laplace2d_lower(4096, 64), "lower"),
    ("growlocal", dict(mode="growlocal", k=22), lambda: W.erdos_renyi_lower(5000, 1e-3, 1), "lower"),
    ("blocks", dict(mode="growlocal", k=16, sched_blocks=5), lambda: W.random_window_lower(20000, 5, 3000, 4),
     "lower"),
    ("upper", dict(mode="growlocal", k=8), lambda: W.transpose(W.narrow_band_lower(8000, 0.05, 20, 2)), "upper"),
    ("transposed", dict(mode="levels"), lambda: W.laplace3d_lower(12 ** 3, 12), "lower_transposed"),
    ("empty", dict(mode="levels"), lambda: W.from_pattern(0, []), "lower"),
]


@pytest.mark.parametrize("name,kw,make,tri", CASES, ids=[c[0] for c in CASES])
def test_round_trip(tmp_path, name, kw, make, tri):
    A = make()
    p = sp.Plan(A, device=-1, triangle=tri, **kw)
    path = tmp_path / "f.plan"
    p.save(A, path)
    q = sp.Plan.load(path, device=-1)
    _same(p, q)
    sp_, sq = p.stats(), q.stats()
    for f in ("n", "nnz", "levels", "supersteps", "k", "phases", "sched_blocks"):
        assert sp_[f] == sq[f], f
    # the loaded plan's schedule still matches the oracle's
    if tri == "lower" and kw["mode"] == "growlocal" and A.n:
        s, pi, S = oracle.growlocal_blocks(A, kw["k"], kw.get("sched_blocks", 1))
        ex = q.export()
        assert np.array_equal(ex.sigma, s) and np.array_equal(ex.pi, pi)


def test_save_refuses_another_pattern(tmp_path):
    A = W.random_window_lower(3000, 4, 500, 1)
    p = sp.Plan(A, mode="growlocal", k=8, device=-1)
    B = W.random_window_lower(3000, 4, 500, 2)               # same size, other pattern
    if B.nnz == A.nnz:
        with pytest.raises(sp.SptrsvError) as e:
            p.save(B, tmp_path / "x.plan")
        assert e.value.status == sp.ERR_ARG
    C = W.random_window_lower(3001, 4, 500, 1)
    with pytest.raises(sp.SptrsvError) as e:
        p.save(C, tmp_path / "y.plan")
    assert e.value.status == sp.ERR_ARG
    # same pattern, other values: saved as given, the schedule still holds
    D = W.CSR(A.n, A.rowptr, A.col, A.val * 2.0, "scaled")
    p.save(D, tmp_path / "z.plan")
    _same(p, sp.Plan.load(tmp_path / "z.plan", device=-1))


def _saved(tmp_path, mode="growlocal"):
    A = W.erdos_renyi_lower(2000, 2e-3, 5)
    p = sp.Plan(A, mode=mode, k=6, device=-1)
    path = tmp_path / "g.plan"
    p.save(A, path)
    return A, path, bytearray(path.read_bytes())


def _refused(tmp_path, data, status):
    bad = tmp_path / "bad.plan"
    bad.write_bytes(bytes(data))
    with pytest.raises(sp.SptrsvError) as e:
        sp.Plan.load(bad, device=-1)
    assert e.value.status == status


def _fix_checksum(data):
    # recompute the trailing checksum the way the file format defines it
    h = 0x9e3779b97f4a7c15
    M = (1 << 64) - 1
    payload = bytes(data[HEADER:-8])
    n, tri, nnz = struct.unpack_from("<iiq", data, 16)
    mode, k, S, sb, loc_nb, _ = struct.unpack_from("<6i", data, 32)
    sizes = [(n + 1) * 4, nnz * 4, nnz * 8, n * 4, n * 4] + ([n * 4, n * 4] if loc_nb else [])
    off = 0
    for size in sizes:
        if size == 0:
            continue
        chunk = payload[off:off + size]
        off += size
        i = 0
        while i + 8 <= size:
            h = ((h ^ int.from_bytes(chunk[i:i + 8], "little")) * 0x100000001b3) & M
            i += 8
        w = int.from_bytes(chunk[i:] + b"\0" * (8 - (size - i)), "little")
        h = ((h ^ w ^ (size << 56)) * 0x100000001b3) & M
    z = h
    z = ((z ^ (z >> 30)) * 0xbf58476d1ce4e5b9) & M
    z = ((z ^ (z >> 27)) * 0x94d049bb133111eb) & M
    z ^= z >> 31
    data[-8:] = z.to_bytes(8, "little")
    return data


def test_checksum_reimplementation_matches(tmp_path):
    _, _, data = _saved(tmp_path)
    assert bytes(_fix_checksum(bytearray(data))) == bytes(data)


def test_load_refuses_damage(tmp_path):
    A, path, data = _saved(tmp_path)
    n = A.n
    sig_off = HEADER + (n + 1) * 4 + A.nnz * 12
    _refused(tmp_path, data[:-1], sp.ERR_IO)                          # truncated
    _refused(tmp_path, data + b"\0", sp.ERR_IO)                       # trailing bytes
    d = bytearray(data); d[0:8] = b"NOTAPLAN"
    _refused(tmp_path, d, sp.ERR_ARG)                                 # magic
    d = bytearray(data); struct.pack_into("<I", d, 8, 2)
    _refused(tmp_path, d, sp.ERR_ARG)                                 # version
    d = bytearray(data); struct.pack_into("<I", d, 12, 0x04030201)
    _refused(tmp_path, d, sp.ERR_ARG)                                 # byte order
    d = bytearray(data); d[sig_off + 5] ^= 0x40
    _refused(tmp_path, d, sp.ERR_ARG)                                 # flipped bit: checksum
    with pytest.raises(sp.SptrsvError) as e:
        sp.Plan.load(tmp_path / "missing.plan", device=-1)
    assert e.value.status == sp.ERR_IO


def test_load_refuses_invalid_schedule_with_valid_checksum(tmp_path):
    A, path, data = _saved(tmp_path)
    n = A.n
    sig_off = HEADER + (n + 1) * 4 + A.nnz * 12
    pi_off = sig_off + 4 * n
    sigma = np.frombuffer(bytes(data[sig_off:sig_off + 4 * n]), dtype="<i4").copy()
    pi = np.frombuffer(bytes(data[pi_off:pi_off + 4 * n]), dtype="<i4").copy()
    u, v = oracle.edges(A)
    # an edge whose endpoints sit in different supersteps: pull the child before its parent
    e = int(np.nonzero(sigma[u] < sigma[v])[0][0])
    d = bytearray(data)
    bad = sigma.copy(); bad[v[e]] = sigma[u[e]] - 1 if sigma[u[e]] > 0 else 0
    if bad[v[e]] == sigma[u[e]]:
        bad_pi = pi.copy(); bad_pi[v[e]] = (pi[u[e]] + 1) % 6
        d[pi_off:pi_off + 4 * n] = bad_pi.astype("<i4").tobytes()
    d[sig_off:sig_off + 4 * n] = bad.astype("<i4").tobytes()
    _refused(tmp_path, _fix_checksum(d), sp.ERR_ARG)
    d = bytearray(data)                                               # core out of range
    bad_pi = pi.copy(); bad_pi[0] = 6
    d[pi_off:pi_off + 4 * n] = bad_pi.astype("<i4").tobytes()
    _refused(tmp_path, _fix_checksum(d), sp.ERR_ARG)
    d = bytearray(data)                                               # superstep gap
    gap = sigma.copy(); gap[gap == gap.max()] += 1
    struct.pack_into("<i", d, 40, int(gap.max()) + 1)
    d[sig_off:sig_off + 4 * n] = gap.astype("<i4").tobytes()
    _refused(tmp_path, _fix_checksum(d), sp.ERR_ARG)


def test_load_refuses_wavefront_schedule_that_is_not_the_wavefronts(tmp_path):
    A, path, data = _saved(tmp_path, mode="levels")
    n = A.n
    sig_off = HEADER + (n + 1) * 4 + A.nnz * 12
    sigma = np.frombuffer(bytes(data[sig_off:sig_off + 4 * n]), dtype="<i4").copy()
    # shift a sink row one wavefront later: still valid by Def. 2.1, not the wavefronts
    has_child = np.zeros(n, bool)
    u, v = oracle.edges(A)
    has_child[u] = True
    r = int(np.nonzero(~has_child & (sigma < sigma.max()))[0][0])
    sigma[r] += 1
    d = bytearray(data)
    d[sig_off:sig_off + 4 * n] = sigma.astype("<i4").tobytes()
    _refused(tmp_path, _fix_checksum(d), sp.ERR_ARG)


def test_load_refuses_factor_damage_with_valid_checksum(tmp_path):
    A, path, data = _saved(tmp_path)
    d = bytearray(data)
    # make a row's columns unsorted: validation of the stored factor must catch it
    row = int(np.nonzero(np.diff(A.rowptr) >= 3)[0][0])
    q = HEADER + (A.n + 1) * 4 + int(A.rowptr[row]) * 4
    a, b = struct.unpack_from("<ii", d, q)
    struct.pack_into("<ii", d, q, b, a)
    _refused(tmp_path, _fix_checksum(d), sp.ERR_UNSORTED_OR_DUP)


def test_load_refuses_out_of_range_header_fields(tmp_path):
    A, path, data = _saved(tmp_path)
    n = A.n
    for off, value in ((36, (1 << 20) + 1),      # k
                       (40, n + 1),              # supersteps
                       (32, 7),                  # mode
                       (52, n + 1)):             # coarsened vertices
        d = bytearray(data)
        struct.pack_into("<i", d, off, value)
        _refused(tmp_path, d, sp.ERR_ARG)
