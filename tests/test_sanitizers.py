"""Memory-safety evidence on the host (compute-sanitizer is closed on the GPU
pool): the oracle and the CUDA library's host-side card expansion are built
with AddressSanitizer and UndefinedBehaviorSanitizer and run over real and
malformed inputs; any report makes the run fail.

* the oracle (oracle/oracle.c): every event of a tiny and a batched sample
  and of hand-made degenerate events, with marginal-decision flips, all
  clustering algorithms with a forced step, impact parameters, the threaded
  batch form, and pile-up draws with forced truncation decisions;
* the card expansion (pdr_card.h, pdr_hot.h): the three stock cards and
  thousands of mutated copies (out-of-range counts, non-finite or negative
  values), each accepted or rejected cleanly.
"""
import ctypes
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import oracle
from paper_2606_26089_b300 import binding as B
from paper_2606_26089_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.join(ROOT, "tests", "sanitize")
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=all", "-fno-omit-frame-pointer", "-g", "-O1"]
ENV = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0:exitcode=23",
           UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1:exitcode=24")

pytestmark = pytest.mark.skipif(shutil.which("gcc") is None or shutil.which("g++") is None, reason="no gcc")


def _batch_file(path, card_name, batch):
    card = oracle.load_card(card_name)
    with open(path, "wb") as f:
        f.write(b"PDRS")
        f.write(struct.pack("<QQI", batch.n_events, batch.n_particles, 0 if batch.vz is None else 1))
        f.write(ctypes.string_at(ctypes.addressof(card), ctypes.sizeof(card)))
        f.write(np.ascontiguousarray(batch.offsets, np.uint64).tobytes())
        for k, dt in (("pt", np.float32), ("eta", np.float32), ("phi", np.float32), ("mass", np.float32),
                      ("pdg", np.int32), ("charge", np.int8)):
            f.write(np.ascontiguousarray(getattr(batch, k), dt).tobytes())
        if batch.vz is not None:
            f.write(np.ascontiguousarray(batch.vz, np.float32).tobytes())


def _run(exe, arg):
    p = subprocess.run([exe, arg], capture_output=True, text=True, env=ENV, timeout=900)
    assert p.returncode == 0 and "ERROR" not in p.stderr and "runtime error" not in p.stderr, p.stderr[-4000:]
    return p.stdout


def test_oracle_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    exe = str(tmp_path / "oracle_driver")
    subprocess.check_call(["gcc", "-std=c11", "-D_GNU_SOURCE", *SAN, "-I", os.path.join(ROOT, "oracle"),
                           os.path.join(HERE, "oracle_driver.c"), os.path.join(ROOT, "oracle", "oracle.c"),
                           "-lm", "-lpthread", "-o", exe])
    M = 0.13957039
    hand = synth.from_particles([
        [], [(10.0, 0.3, 1.0, 0.497611, 130, 0)],
        [(0.0, 1.0, 0.0, M, 211, 1), (5.0, 0.0, 0.0, 0.0, 22, 0), (1e-4, -7.0, 3.14, M, -211, -1),
         (20.0, 0.4, 1.0, 0.0, 12, 0), (500.0, 4.89, -3.1415925, M, 211, 1), (30.0, 0.1, 0.1, 0.000511, 11, -1)],
        [(50.0, 0.1, 0.1, 0.1056583755, 13, -1)] + [(3.0, 0.1 + 0.01 * k, 0.1, M, 211, 1) for k in range(40)],
        [(0.7, 0.2, 0.5, M, 211, 2, 0.1), (2.0, 3.5, -1.0, M, -211, -1, -0.2)],
    ])
    for name, card, b in (("tiny", "cms_like", synth.make("tiny", n_events=30)),
                          ("batched", "cms_like", synth.make("batched", n_events=6)),
                          ("ee", "ee_like", synth.make("ee", n_events=40)),
                          ("pileup", "atlas_like", synth.make("pileup", n_events=1).slice_events(0, 1)),
                          ("hand", "cms_like", hand)):
        path = str(tmp_path / f"{name}.bin")
        _batch_file(path, card, b)
        out = _run(exe, path)
        assert out.startswith("ok"), out


def test_card_expansion_under_address_and_undefined_behaviour_sanitizers(tmp_path):
    exe = str(tmp_path / "card_driver")
    csrc = os.path.join(ROOT, "paper_2606_26089_b300", "csrc")
    subprocess.check_call(["g++", "-std=c++17", *SAN, "-I", os.path.join(ROOT, "include"), "-I", csrc,
                           "-I", "/usr/local/cuda/include", os.path.join(HERE, "card_driver.cpp"), "-o", exe])
    path = str(tmp_path / "cards.bin")
    with open(path, "wb") as f:
        for name in ("cms_like", "atlas_like", "ee_like"):
            c = B.card_from_json(name)
            f.write(ctypes.string_at(ctypes.addressof(c), ctypes.sizeof(c)))
    out = _run(exe, path)
    assert out.startswith("ok"), out
    acc, rej = (int(x) for x in out.split()[1:4:2])
    assert acc > 0 and rej > 0
