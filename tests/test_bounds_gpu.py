"""The bounds-checking debug build (libpdr_bounds.so, -DPDR_BOUNDS): every
index the response kernel uses into a batch array, an event array or its
tower table is checked, and an index out of range raises ERR_BOUNDS in the
error word instead of being used.  The parity tests of the response run
against this build in a child process (the binding loads it when
PDR_LIB_VARIANT=bounds) and must pass with the error word clear: no access of
the kernel left its arrays on any of those workloads and launch shapes."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_suite_under_the_bounds_checking_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26089_b300 import build
    lib = build.build(bounds=True)
    assert lib.endswith("libpdr_bounds.so")
    env = dict(os.environ, PDR_LIB_VARIANT="bounds")
    sel = ("tiny or several_chunks or ee_parity or pileup_parity or atlas_card or every_launch or global_table "
           "or empty_and or charges or larger_than or offset_past or malformed or rerun or concurrent")
    p = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_parity_gpu.py"),
                        "-q", "-x", "-m", "gpu", "-k", sel, "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    assert p.returncode == 0, p.stdout[-3000:] + p.stderr[-2000:]
    assert "passed" in p.stdout
    # the child really used the debug build
    q = subprocess.run([sys.executable, "-c", "from paper_2606_26089_b300 import binding as b; print(b.LIB_PATH)"],
                       cwd=ROOT, env=env, capture_output=True, text=True)
    assert q.stdout.strip().endswith("libpdr_bounds.so")
