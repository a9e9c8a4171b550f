"""Forest files (gf_forest_save / gf_forest_load).

The layout include/gf.h documents is written and read here with numpy alone, so the format is
pinned by a second, independent implementation: a file the library writes must parse here into the
forest the library exports, and a file written here from an oracle-built forest must load into a
forest that answers as the oracle does.  Every malformed file must be rejected with GF_EIO before
the device is touched, which the CPU tests check without a GPU.
"""
import os

import numpy as np
import pytest
import torch

import oracle
import synth

MAGIC = b"GFFOREST"
HEADER = 128
DEFAULT_TUNING = [[8, 8, 8], [0, 0, 0], [0, 64, 128], [0, 0, 0]]


def checksum(payload: bytes):
    w = np.frombuffer(payload, dtype="<u4").astype(np.uint64)
    i = np.arange(1, w.size + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return int(w.sum(dtype=np.uint64)), int((w * i).sum(dtype=np.uint64))


def encode(n, d, T, leaf_size, L, split_dim, split_val, perm, X, U=None, flags=0, tuning=DEFAULT_TUNING,
           version=1, payload_bytes=None, checks=None):
    nodes = np.empty((T, (1 << L) - 1, 2), dtype="<i4")
    nodes[..., 0] = split_dim
    nodes[..., 1] = np.ascontiguousarray(split_val, dtype="<f4").view("<i4")
    parts = [nodes.tobytes(), np.ascontiguousarray(perm, dtype="<i4").tobytes()]
    if U is not None:
        flags |= 1
        parts.append(np.ascontiguousarray(U, dtype="<f4").tobytes())
    parts.append(np.ascontiguousarray(X, dtype="<f4").tobytes())
    payload = b"".join(parts)
    h = bytearray(HEADER)
    h[0:8] = MAGIC
    h[8:16] = np.array([version, 0x01020304], dtype="<u4").tobytes()
    h[16:24] = np.array([n], dtype="<i8").tobytes()
    h[24:44] = np.array([d, T, leaf_size, L, flags], dtype="<u4").tobytes()
    h[44:92] = np.array(tuning, dtype="<i4").reshape(-1).tobytes()
    s1, s2 = checksum(bytes(h[:96]) + payload) if checks is None else checks
    h[96:120] = np.array([len(payload) if payload_bytes is None else payload_bytes, s1, s2],
                         dtype="<u8").tobytes()
    return bytes(h) + payload


def decode(blob: bytes):
    assert blob[:8] == MAGIC
    version, bom = np.frombuffer(blob, "<u4", 2, 8)
    assert version == 1 and bom == 0x01020304
    n = int(np.frombuffer(blob, "<i8", 1, 16)[0])
    d, T, leaf_size, L, flags = (int(v) for v in np.frombuffer(blob, "<i4", 5, 24))
    tuning = np.frombuffer(blob, "<i4", 12, 44).reshape(4, 3)
    payload_bytes, s1, s2 = (int(v) for v in np.frombuffer(blob, "<u8", 3, 96))
    payload = blob[HEADER:]
    assert len(payload) == payload_bytes
    assert checksum(blob[:96] + payload) == (s1, s2)
    nn = (1 << L) - 1
    off = 0

    def take(dtype, count, shape):
        nonlocal off
        a = np.frombuffer(payload, dtype, count, off).reshape(shape)
        off += a.nbytes
        return a

    nodes = take("<i4", T * nn * 2, (T, nn, 2))
    perm = take("<i4", T * n, (T, n))
    U = take("<f4", T * d, (T, d)) if flags & 1 else None
    X = take("<f4", n * d, (n, d))
    assert off == len(payload)
    return dict(n=n, d=d, T=T, leaf_size=leaf_size, L=L, flags=flags, tuning=tuning,
                split_dim=nodes[..., 0].copy(), split_val=nodes[..., 1].copy().view("<f4"), perm=perm, U=U, X=X)


@pytest.fixture(scope="module")
def gf():
    import paper_1603_09596_gb300 as g
    g.lib()
    return g


@pytest.fixture(scope="module")
def small():
    X, Q = synth.mixture(3001, 37, 50, "B", seed=0, qseed=1)
    F = oracle.build_forest(X, 5, 9, t=5, seed=3)
    return X, Q, F


def forest_blob(small, **kw):
    X, _, F = small
    return encode(F.n, F.d, F.T, F.leaf_size, F.L, F.split_dim, F.split_val, F.perm, X, **kw)


def load_code(gf, path):
    import ctypes
    h = ctypes.c_void_p()
    return gf.lib().gf_forest_load(os.fsencode(path), ctypes.byref(h)), h


# ------------------------------------------------------------------ CPU: the format is checked on the host

def test_writer_matches_the_documented_header(small):
    blob = forest_blob(small)
    d = decode(blob)
    X, _, F = small
    assert (d["n"], d["d"], d["T"], d["leaf_size"], d["L"]) == (F.n, F.d, F.T, F.leaf_size, F.L)
    assert np.array_equal(d["split_dim"], F.split_dim) and np.array_equal(d["split_val"], F.split_val)
    assert np.array_equal(d["perm"], F.perm) and np.array_equal(d["X"], X)


def test_checksum_pins():
    # s1 = sum w_i, s2 = sum (i + 1) w_i over u32 words, by hand on three words
    p = np.array([5, 7, 0xffffffff], dtype="<u4").tobytes()
    assert checksum(p) == (5 + 7 + 0xffffffff, 5 + 2 * 7 + 3 * 0xffffffff)
    # the position weight catches a swap the plain sum misses
    q = np.array([7, 5, 0xffffffff], dtype="<u4").tobytes()
    assert checksum(q)[0] == checksum(p)[0] and checksum(q)[1] != checksum(p)[1]


def test_load_rejects_null_arguments(gf):
    import ctypes
    h = ctypes.c_void_p()
    assert gf.lib().gf_forest_load(None, ctypes.byref(h)) == gf.GF_EINVAL
    assert gf.lib().gf_forest_load(b"x", None) == gf.GF_EINVAL
    assert gf.lib().gf_forest_save(None, b"x") == gf.GF_EINVAL


def test_missing_file_is_eio(gf, tmp_path):
    code, h = load_code(gf, tmp_path / "absent.gff")
    assert code == gf.GF_EIO and not h.value
    assert b"cannot open" in gf.lib().gf_last_error()


def _mutations(small):
    X, _, F = small
    good = forest_blob(small)
    nn = (1 << F.L) - 1
    bad_tuning = [row[:] for row in DEFAULT_TUNING]
    bad_tuning[3][1] = 3   # rows in flight must be 0, 2 or 4
    many_ctas = [row[:] for row in DEFAULT_TUNING]
    many_ctas[1][0] = 33   # an SM runs at most 32 CTAs
    long_list = [row[:] for row in DEFAULT_TUNING]
    long_list[2][2] = 2049  # the streaming kernel keeps at most 2048 keys per query
    flip = bytearray(good)
    flip[HEADER + len(good[HEADER:]) // 2] ^= 0x10
    w = np.frombuffer(good[HEADER:], "<u4").copy()
    w[[0, 1]] = w[[1, 0]]
    swapped = good[:HEADER] + w.tobytes()
    retuned = bytearray(good)
    retuned[44:48] = np.array([4], "<i4").tobytes()  # a valid tuning value, but not the one summed
    return {
        "empty": b"",
        "short_header": good[:100],
        "magic": b"GFFORESX" + good[8:],
        "version": forest_blob(small, version=2),
        "byte_order": good[:12] + np.array([0x04030201], "<u4").tobytes() + good[16:],
        "depth": encode(F.n, F.d, F.T, F.leaf_size + 100, F.L, F.split_dim, F.split_val, F.perm, X),
        "flags": forest_blob(small, flags=8),
        "tuning": forest_blob(small, tuning=bad_tuning),
        "tuning_ctas": forest_blob(small, tuning=many_ctas),
        "tuning_shortlist": forest_blob(small, tuning=long_list),
        "payload_size": forest_blob(small, payload_bytes=len(good) - HEADER + 4),
        "truncated": good[:-4],
        "trailing": good + b"\0\0\0\0",
        "bit_flip": bytes(flip),
        "swapped_words": swapped,
        "checksum": forest_blob(small, checks=(1, 2)),
        "header_field": bytes(retuned),
        "zero_trees": encode(F.n, F.d, 0, F.leaf_size, F.L, np.zeros((0, nn)), np.zeros((0, nn)),
                             np.zeros((0, F.n)), X),
    }


@pytest.mark.parametrize("kind", ["empty", "short_header", "magic", "version", "byte_order", "depth", "flags",
                                  "tuning", "tuning_ctas", "tuning_shortlist", "payload_size", "truncated", "trailing", "bit_flip",
                                  "swapped_words", "checksum", "header_field", "zero_trees"])
def test_malformed_file_is_eio(gf, small, tmp_path, kind):
    p = tmp_path / f"{kind}.gff"
    p.write_bytes(_mutations(small)[kind])
    code, h = load_code(gf, p)
    assert code == gf.GF_EIO, gf.lib().gf_last_error()
    assert not h.value


def test_well_formed_file_passes_the_host_checks(gf, small, tmp_path):
    """Without a GPU a good file gets past every format check and fails only at the device."""
    p = tmp_path / "good.gff"
    p.write_bytes(forest_blob(small))
    code, h = load_code(gf, p)
    if torch.cuda.is_available():
        assert code == gf.GF_OK
        gf.Forest(h).free()
    else:
        assert code in (gf.GF_ENOMEM, gf.GF_ECUDA), gf.lib().gf_last_error()


# ------------------------------------------------------------------ GPU: round trips

def _same_structure(gf, A, B):
    for a, b in zip(gf.gf_forest_export(A), gf.gf_forest_export(B)):
        assert np.array_equal(a, b)


@pytest.mark.gpu
def test_save_load_round_trip(gf, tmp_path):
    X, Q = synth.mixture(20_000, 960, 300, "B", seed=0, qseed=1)
    T = 8
    rng = np.random.default_rng(5)
    U = rng.standard_normal((T, 960)).astype(np.float32)
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    Xg, Qg = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = gf.gf_build(Xg, T, 64, seed=11, U=U)
    gf.gf_forest_add_screen(G, gf.GF_BF16_RERANK)
    gf.gf_forest_set_tuning(G, gf.GF_BF16_RERANK, 4, 2, 24, 2)
    path = tmp_path / "f.gff"
    gf.gf_forest_save(G, path)
    assert not os.path.exists(str(path) + ".tmp")

    # the file parses with the independent reader into exactly what the library holds
    f = decode(path.read_bytes())
    sd, sv, pm = gf.gf_forest_export(G)
    inf = G.info
    assert (f["n"], f["d"], f["T"], f["leaf_size"], f["L"]) == (inf.n, inf.d, inf.T, inf.leaf_size, inf.L)
    assert f["flags"] == 1 | 2
    assert np.array_equal(f["split_dim"], sd) and np.array_equal(f["split_val"].view(np.int32), sv.view(np.int32))
    assert np.array_equal(f["perm"], pm) and np.array_equal(f["X"], X) and np.array_equal(f["U"], U)
    assert list(f["tuning"][:, gf.GF_BF16_RERANK]) == [4, 2, 24, 2]

    H = gf.gf_forest_load(path)
    _same_structure(gf, G, H)
    hi = H.info
    assert hi.screens == inf.screens and hi.device_bytes == inf.device_bytes
    # every path answers bit for bit as before: the tuned shortlist (R = 24) comes back too
    for kw in (dict(), dict(precision=gf.GF_BF16_RERANK, algo=gf.GF_ALGO_LEAF),
               dict(precision=gf.GF_BF16_RERANK, algo=gf.GF_ALGO_STREAM), dict(checks=24),
               dict(precision=gf.GF_BF16_RERANK, checks=24, algo=gf.GF_ALGO_LEAF)):
        a = gf.gf_query(G, Qg, 10, **kw)
        b = gf.gf_query(H, Qg, 10, **kw)
        torch.cuda.synchronize()
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), kw

    # saving the loaded forest gives the same bytes
    path2 = tmp_path / "g.gff"
    gf.gf_forest_save(H, path2)
    assert path.read_bytes() == path2.read_bytes()


@pytest.mark.gpu
def test_oracle_forest_through_a_file_answers_as_the_oracle(gf, small, tmp_path):
    from parity import assert_topk_close, candidate_sets
    X, Q, F = small
    p = tmp_path / "oracle.gff"
    p.write_bytes(forest_blob(small))
    G = gf.gf_forest_load(p)
    ids, dists = gf.gf_query(G, torch.from_numpy(Q).cuda(), 7)
    oi, od = oracle.search(F, X, Q, 7)
    offs, cids = oracle.candidates(F, oracle.descend(F, Q))
    assert_topk_close(X, Q, ids.cpu().numpy(), dists.cpu().numpy(), oi, od, candidate_sets(offs, cids))


@pytest.mark.gpu
def test_file_with_an_invalid_forest_is_eio(gf, small, tmp_path):
    X, _, F = small
    bad_dim = F.split_dim.copy()
    bad_dim[1, 3] = F.d
    bad_perm = F.perm.copy()
    bad_perm[2, 0] = bad_perm[2, 1]
    Xnan = X.copy()
    Xnan[17, 5] = np.nan
    Unan = np.ones((F.T, F.d), np.float32)
    Unan[0, 0] = np.inf
    blobs = {
        "split_dim": encode(F.n, F.d, F.T, F.leaf_size, F.L, bad_dim, F.split_val, F.perm, X),
        "perm": encode(F.n, F.d, F.T, F.leaf_size, F.L, F.split_dim, F.split_val, bad_perm, X),
        "nan_x": encode(F.n, F.d, F.T, F.leaf_size, F.L, F.split_dim, F.split_val, F.perm, Xnan),
        "inf_u": encode(F.n, F.d, F.T, F.leaf_size, F.L, F.split_dim, F.split_val, F.perm, X, U=Unan),
    }
    for kind, blob in blobs.items():
        p = tmp_path / f"{kind}.gff"
        p.write_bytes(blob)
        code, h = load_code(gf, p)
        assert code == gf.GF_EIO and not h.value, (kind, gf.lib().gf_last_error())


@pytest.mark.gpu
def test_save_failures_leave_no_file(gf, small, tmp_path):
    X, _, F = small
    G = gf.gf_forest_import(torch.from_numpy(X).cuda(), F.T, F.leaf_size, F.split_dim, F.split_val, F.perm)
    bad = tmp_path / "no_such_dir" / "f.gff"
    with pytest.raises(gf.GFError) as e:
        gf.gf_forest_save(G, bad)
    assert e.value.code == gf.GF_EIO
    assert not os.path.exists(bad.parent)
    # an existing file is replaced whole
    p = tmp_path / "f.gff"
    p.write_bytes(b"old contents")
    gf.gf_forest_save(G, p)
    H = gf.gf_forest_load(p)
    _same_structure(gf, G, H)


@pytest.mark.gpu
def test_single_leaf_forest_round_trip(gf, tmp_path):
    """leaf_size >= n: no internal node (L = 0), every query scans all points; the file still
    round-trips and the loaded forest is exact."""
    X, Q = synth.mixture(500, 24, 20, "A", seed=2, qseed=3)
    G = gf.gf_build(torch.from_numpy(X).cuda(), 3, 500, seed=1)
    assert G.info.L == 0
    p = tmp_path / "one_leaf.gff"
    gf.gf_forest_save(G, p)
    f = decode(p.read_bytes())
    assert f["L"] == 0 and f["split_dim"].size == 0 and np.array_equal(f["X"], X)
    H = gf.gf_forest_load(p)
    _same_structure(gf, G, H)
    ids, dists = gf.gf_query(H, torch.from_numpy(Q).cuda(), 5)
    oi, od = oracle.bruteforce(X, Q, 5)
    from parity import assert_topk_close
    assert_topk_close(X, Q, ids.cpu().numpy(), dists.cpu().numpy(), oi, od)
