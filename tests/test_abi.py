"""CPU-only checks of the C-ABI library: it loads, exports every function that
include/amb.h declares, and its host-side threshold tables (no GPU involved)
equal the oracle's independently computed tables."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2601_16292_gb300 import amb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INCLUDE = os.path.join(ROOT, "include")


def declared_functions():
    names = set()
    for f in os.listdir(INCLUDE):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(INCLUDE, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**\s*(amb_[a-z0-9_]+)\s*\(", text,
                             flags=re.M):
            names.add(m.group(1))
    return names


def test_library_loads_and_exports_all_declared_symbols():
    lib = amb.lib()
    names = declared_functions()
    assert len(names) >= 16
    for name in sorted(names):
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_version_string():
    assert "sm_103a" in amb.amb_version()


@pytest.mark.parametrize("beta,gamma", [(0.05, 0.02), (0.01, 0.005), (0.2, 0.05), (0.123456789, 0.0333),
                                        (0.0, 0.0), (1.0, 1.0), (1e-6, 0.5), (0.5, 1e-9)])
def test_threshold_tables_match_oracle(beta, gamma):
    for cap in (1, 7, 1000, 10_000_000):
        a, ta = amb.amb_sir_thresholds(beta, gamma, cap)
        b, tb = oracle.sir_thresholds(beta, gamma, cap)
        assert ta == tb
        assert np.array_equal(a, b)


def test_threshold_rejects_bad_probabilities():
    with pytest.raises(amb.AmbError) as e:
        amb.amb_sir_thresholds(1.5, 0.1, 10)
    assert e.value.status == amb.AMB_EINVAL
    with pytest.raises(amb.AmbError):
        amb.amb_sir_thresholds(0.1, float("nan"), 10)


def test_params_struct_layout():
    assert ctypes.sizeof(amb.amb_params) == 40
    assert ctypes.sizeof(amb.amb_invariant_report) == 40
    assert amb.amb_stats.max_occupancy.offset == 96


def _c_layout(tmp_path, structs):
    """sizeof and field offsets of the header's structs, as gcc lays them out."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "amb.h"', "int main(void) {"]
    for name, cls in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def test_binding_structs_match_header_layout(tmp_path):
    structs = [(n, getattr(amb, n)) for n in ("amb_params", "amb_cparams", "amb_invariant_report", "amb_stats", "amb_job", "amb_tune",
                                              "amb_batch_report")]
    structs += [(n, getattr(amb, n)) for n in ("amb_server_config", "amb_result", "amb_server_report")
                if hasattr(amb, n)]
    c = _c_layout(tmp_path, structs)
    for name, cls in structs:
        assert c[name] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert c["%s.%s" % (name, f)] == getattr(cls, f).offset, (name, f)


def test_job_bytes_host_only():
    job = amb.make_job("sir", 100_000, seed=1, steps=100, L=408, beta=0.1, gamma=0.02, n0=100)
    r, t = amb.amb_job_bytes(job)
    C = 408 * 408
    # records, cell index and thresholds at least; creation scratch: columns + counters
    assert r >= 16 * 100_000 + 4 * C + 4 * 100_000
    assert t == 13 * 100_000 + 8 * C
    r2, _ = amb.amb_job_bytes(amb.make_job("sir", 200_000, seed=1, steps=100, L=408, beta=0.1, gamma=0.02, n0=100))
    assert r2 > r
    rw, tw = amb.amb_job_bytes(amb.make_job("walk", 100_000, seed=1, steps=100, L=408))
    assert tw == 0 and 8 * 100_000 <= rw < r
    small, _ = amb.amb_job_bytes(amb.make_job("wealth", 1000, seed=1, steps=100))
    large, _ = amb.amb_job_bytes(amb.make_job("wealth", 100_000, seed=1, steps=100))
    assert large - small >= 8 * 99_000  # large wealth populations keep a credit column
    # the per-step count rows grow with the steps
    a, _ = amb.amb_job_bytes(amb.make_job("walk", 1000, seed=1, steps=10, L=40))
    b, _ = amb.amb_job_bytes(amb.make_job("walk", 1000, seed=1, steps=10_000, L=40))
    assert b - a >= 32 * (10_000 - 64)


def test_job_bytes_rejects_what_create_rejects():
    with pytest.raises(amb.AmbError) as e:
        amb.amb_job_bytes(amb.make_job("sir", 10, seed=1, steps=1, L=4, beta=1.5, gamma=0.1, n0=1))
    assert e.value.status == amb.AMB_EINVAL
    with pytest.raises(amb.AmbError):
        amb.amb_job_bytes(amb.make_job("sir", 10, seed=1, steps=1, L=4, beta=0.5, gamma=0.1, n0=11))
    with pytest.raises(amb.AmbError):
        amb.amb_job_bytes(amb.make_job("walk", 10, seed=1 << 33, steps=1, L=4))
    # continuous-space models are not batched or served
    for model in ("cwalk", "csir"):
        with pytest.raises(amb.AmbError) as e:
            amb.amb_job_bytes(amb.make_job(model, 10, seed=1, steps=1))
        assert e.value.status == amb.AMB_EINVAL


def test_injected_creation_failures_on_the_host():
    """The fault-injection hook fails creations before any device call."""
    amb.amb_debug_fail_creates(2)
    try:
        for _ in range(2):
            with pytest.raises(amb.AmbError) as e:
                amb.amb_create("wealth", amb.amb_params(n=10, grid_side=1, w_init=1), 0)
            assert e.value.status == amb.AMB_ENOMEM
            assert "injected" in str(e.value)
        # the hook is spent: the next call is checked as usual (continuous
        # models are refused by amb_create before any device call)
        with pytest.raises(amb.AmbError) as e:
            amb.amb_create("csir", amb.amb_params(n=10), 0)
        assert e.value.status == amb.AMB_EINVAL
    finally:
        amb.amb_debug_fail_creates(0)


def test_sir_variant_constants_match_header():
    """The binding's SIR path constants are the header's enum values."""
    with open(os.path.join(os.path.dirname(__file__), "..", "include", "amb.h")) as f:
        text = f.read()
    for name in ("AMB_SIR_AUTO", "AMB_SIR_GENERIC", "AMB_SIR_BAND", "AMB_SIR_BAND32", "AMB_SIR_BAND16"):
        m = re.search(r"\b%s\s*=\s*(\d+)" % name, text)
        assert m is not None, name
        assert int(m.group(1)) == getattr(amb, name), name


def test_job_bytes_rejects_bad_band16_grids():
    """16-bit band counters need rows of a multiple of 8 cells, at most 8192."""
    for L, ok in ((12, False), (8200, False), (16, True), (8192, True)):
        job = amb.make_job("sir", 10, seed=1, steps=1, L=L, beta=0.5, gamma=0.1, n0=1)
        job.params.variant = amb.AMB_SIR_BAND16
        if ok:
            amb.amb_job_bytes(job)
        else:
            with pytest.raises(amb.AmbError) as e:
                amb.amb_job_bytes(job)
            assert e.value.status == amb.AMB_EINVAL
