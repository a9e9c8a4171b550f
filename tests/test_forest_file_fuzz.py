"""The forest-file parser under AddressSanitizer and UndefinedBehaviorSanitizer (CPU, no GPU).

csrc/gf_io.cu is built on its own with the host sanitizers, with stand-ins for the storage calls it
makes once a file has passed every host check (tests/native/io_stubs.cu: they report GF_ENOMEM and
touch no device).  A child process that preloads the sanitizer runtime then loads a good file and
several hundred damaged copies: random byte flips anywhere, truncations at random lengths, bytes
appended, and header fields set to random values.  Every load must return GF_EIO, or GF_ENOMEM
from the stand-in when the damage left a valid file; any out-of-bounds access, overflow or other
undefined behaviour aborts the child.
"""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth
from test_forest_file import HEADER, encode

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GF_EIO, GF_ENOMEM = -6, -2

CHILD = r"""
import ctypes, json, os, sys
lib = ctypes.CDLL(sys.argv[1])
lib.gf_forest_load.argtypes = [ctypes.c_char_p, ctypes.c_void_p]
lib.gf_forest_load.restype = ctypes.c_int32
out = {}
for name in sorted(os.listdir(sys.argv[2])):
    h = ctypes.c_void_p()
    out[name] = lib.gf_forest_load(os.path.join(sys.argv[2], name).encode(), ctypes.byref(h))
print(json.dumps(out))
"""


def _runtime(name):
    p = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return p if os.path.isabs(p) and os.path.exists(p) else None


def _nvcc():
    for c in ("/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def test_parser_survives_damaged_files_under_sanitizers(tmp_path):
    asan, nvcc = _runtime("libasan.so"), _nvcc()
    if asan is None or nvcc is None:
        pytest.skip("needs gcc's AddressSanitizer runtime and nvcc")
    so = str(tmp_path / "libgfio_san.so")
    r = subprocess.run([nvcc, "-std=c++17", "-g", "-O1", "--expt-relaxed-constexpr",
                        "-Xcompiler", "-fPIC,-fsanitize=address,-fsanitize=undefined,-fno-omit-frame-pointer,"
                                      "-fno-sanitize-recover=all",
                        "-I", os.path.join(ROOT, "include"), "-I", os.path.join(ROOT, "paper_1603_09596_gb300", "csrc"),
                        "-shared", "-o", so, os.path.join(ROOT, "paper_1603_09596_gb300", "csrc", "gf_io.cu"),
                        os.path.join(ROOT, "tests", "native", "io_stubs.cu"), "-Xlinker", "-lasan", "-Xlinker",
                        "-lubsan"], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip(f"sanitizer build unavailable: {r.stderr[-300:]}")

    X, _ = synth.mixture(400, 9, 1, "B", seed=1, qseed=2)
    F = oracle.build_forest(X, 3, 7, t=5, seed=4)
    U = np.eye(3, 9, dtype=np.float32)
    good = encode(F.n, F.d, F.T, F.leaf_size, F.L, F.split_dim, F.split_val, F.perm, X, U=U)
    files = tmp_path / "files"
    files.mkdir()
    (files / "good").write_bytes(good)
    rng = np.random.default_rng(0)
    for i in range(300):
        b = bytearray(good)
        kind = i % 4
        if kind == 0:    # flip 1..8 random bytes anywhere
            for pos in rng.integers(0, len(b), rng.integers(1, 9)):
                b[pos] ^= int(rng.integers(1, 256))
        elif kind == 1:  # truncate
            b = b[:int(rng.integers(0, len(b)))]
        elif kind == 2:  # append
            b += bytes(rng.integers(0, 256, int(rng.integers(1, 64)), dtype=np.uint8))
        else:            # one header word set at random (the checksum then fails, or the field check)
            w = int(rng.integers(0, HEADER // 4))
            b[4 * w:4 * w + 4] = rng.integers(0, 2 ** 32, dtype=np.uint64).astype("<u4").tobytes()
        (files / f"bad{i:03d}").write_bytes(bytes(b))

    env = dict(os.environ, LD_PRELOAD=asan, ASAN_OPTIONS="detect_leaks=0:abort_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    p = subprocess.run([sys.executable, "-c", CHILD, so, str(files)], capture_output=True, text=True, env=env,
                       timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    assert "AddressSanitizer" not in p.stderr and "runtime error" not in p.stderr, p.stderr[-3000:]
    import json
    codes = json.loads(p.stdout.strip().splitlines()[-1])
    assert codes["good"] == GF_ENOMEM  # every host check passed; the stand-in allocator refuses
    bad = {k: v for k, v in codes.items() if k != "good" and v not in (GF_EIO, GF_ENOMEM)}
    assert not bad, bad
    assert sum(v == GF_EIO for k, v in codes.items() if k != "good") >= 290
