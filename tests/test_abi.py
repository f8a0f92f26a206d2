"""The C-ABI library loads on the CPU host and exports every entry point that
include/pdr.h declares (no compute calls: there may be no GPU here)."""
import ctypes
import os
import re

import pytest

from paper_2606_26089_b300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pdr.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(pdr_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def libpdr():
    build.build()
    return binding.lib()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("pdr_create", "pdr_destroy", "pdr_card_load", "pdr_card_unload", "pdr_run",
              "pdr_run_per_event", "pdr_run_host", "pdr_autotune", "pdr_submit", "pdr_wait",
              "pdr_fetch", "pdr_release", "pdr_check", "pdr_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(libpdr):
    for name in declared_symbols():
        assert hasattr(libpdr, name), name
        assert isinstance(getattr(libpdr, name), ctypes._CFuncPtr)


def test_abi_version(libpdr):
    assert libpdr.pdr_abi_version() == 1


STRUCTS = ("pdr_card", "pdr_batch", "pdr_outputs", "pdr_launch", "pdr_options", "pdr_result",
           "pdr_serve_options", "pdr_serve_stats", "pdr_pileup", "pdr_particles", "pdr_condition",
           "pdr_filter", "pdr_features", "pdr_ip_params", "pdr_jet_params")


def test_binding_structs_match_header_layout(tmp_path):
    """Compile a probe against include/pdr.h and compare sizeof/offsetof with ctypes."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdr.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} %zu\\n", sizeof({s}));')
        for f, _ in getattr(binding, s)._fields_:
            lines.append(f'  printf("{s}.{f} %zu\\n", offsetof({s}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    import subprocess
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for s in STRUCTS:
        cls = getattr(binding, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for f, _ in cls._fields_:
            assert int(got[f"{s}.{f}"]) == getattr(cls, f).offset, (s, f)
    # record layouts the binding views as float32 columns
    for rec, size in (("pdr_track", 16), ("pdr_tower", 12), ("pdr_eflow", 12), ("pdr_cand", 16),
                      ("pdr_iso", 8), ("pdr_debug", 16), ("pdr_ip", 16), ("pdr_jet", 32)):
        probe = tmp_path / f"{rec}.c"
        probe.write_text(f'#include "pdr.h"\nint x[sizeof({rec}) == {size} ? 1 : -1];\n')
        subprocess.check_call(["gcc", "-c", "-I", os.path.join(ROOT, "include"), str(probe), "-o",
                               str(tmp_path / f"{rec}.o")])


def test_cards_parse():
    for name in ("cms_like", "atlas_like", "ee_like"):
        c = binding.card_from_json(name)
        assert c.R > 0 and c.L > 0 and c.nseg[0] >= 1 and c.nseg[1] >= 1
