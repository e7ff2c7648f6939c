"""CPU-side checks of the C ABI: the library builds, loads and exports every function
that include/dagrt.h declares; host-side argument checks need no GPU."""
from __future__ import annotations

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dagrt.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dagrt_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    import __graft_entry__ as g
    g.build()
    from paper_2602_20826_gb300 import build
    return build.LIB


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("dagrt_create", "dagrt_destroy", "dagrt_last_error", "dagrt_load_csr",
                     "dagrt_schedule", "dagrt_bound", "dagrt_batch_free"):
        assert required in names


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(dagrt_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_loads_and_names_match(libpath):
    from paper_2602_20826_gb300 import dagrt
    for n in _declared():
        assert hasattr(dagrt.lib, n)
        assert hasattr(dagrt, n), f"binding lacks {n}"


def test_null_arguments_are_rejected_without_a_device(libpath):
    from paper_2602_20826_gb300 import dagrt
    assert dagrt.dagrt_create(None, 0, None) == dagrt.E_INVAL
    assert dagrt.dagrt_sync(None) == dagrt.E_INVAL
    assert dagrt.dagrt_schedule(None, 0, None, 0) == dagrt.E_INVAL
    assert dagrt.dagrt_bound(None, 1, None, 1, None, 16, None, None, None, 0) == dagrt.E_INVAL
    dagrt.dagrt_destroy(None)
    dagrt.dagrt_batch_free(None)
    assert dagrt.dagrt_batch_n_dags(None) == -1


def test_status_codes_match_the_oracle_codes(libpath):
    import oracle
    from paper_2602_20826_gb300 import dagrt
    assert (dagrt.E_INVAL, dagrt.E_CYCLE, dagrt.E_RANGE, dagrt.E_CAP) == \
        (oracle.E_INVAL, oracle.E_CYCLE, oracle.E_RANGE, oracle.E_CAP)
    hdr = open(os.path.join(ROOT, "include", "dagrt.h")).read()
    for name in ("OK", "E_INVAL", "E_CYCLE", "E_RANGE", "E_OOM", "E_DEVICE", "E_TIMEOUT", "E_CAP",
                 "E_INTERNAL"):
        m = re.search(rf"#define DAGRT_{name} \(?(-?\d+)\)?", hdr)
        assert m and int(m.group(1)) == getattr(dagrt, name)
