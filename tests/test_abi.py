"""The C ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/lpa.h declares; the Python binding covers the same names."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lpa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lpa_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2312_08140_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lpa_graph_create", "lpa_graph_destroy", "lpa_run", "lpa_modularity",
                     "lpa_batch_create", "lpa_batch_run", "lpa_batch_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(lib_path):
    import paper_2312_08140_gb300 as lpa
    assert set(lpa.exported_symbols()) == set(_declared())
    lpa.load(lib_path)
    for n in _declared():
        assert callable(getattr(lpa, n))


def test_pure_host_entry_points(lib_path):
    import paper_2312_08140_gb300 as lpa
    lpa.load(lib_path)
    assert lpa.lpa_version().startswith("lpa-gb300")
    assert lpa.lpa_status_string(lpa.LPA_ERR_INVALID_GRAPH) == "invalid graph"
    lpa.lpa_autotune_cache_clear()                      # host only
    # argument checks happen before any CUDA call
    with pytest.raises(lpa.LpaError) as e:
        lpa.lpa_graph_create(-5, 0, None, None)
    assert e.value.status == lpa.LPA_ERR_INVALID_ARG
    with pytest.raises(lpa.LpaError):
        lpa.lpa_graph_destroy(None)
    # the server takes plain modes only: the non-strict and FLPA flags are refused
    for mode in ("async+prune_other", "sync+nonstrict"):
        with pytest.raises(lpa.LpaError) as e:
            lpa.lpa_serve_create(1 << 30, 1000, 10000, mode=mode)
        assert e.value.status == lpa.LPA_ERR_INVALID_ARG
    # mode strings: flags combine with "+", unknown ones are refused in the binding
    assert lpa._mode("async+nonstrict+prune_other") == lpa.MODES["async"] | lpa.LPA_NONSTRICT | lpa.LPA_PRUNE_OTHER
    with pytest.raises(ValueError):
        lpa._mode("async+bogus")


def test_tolerance_threshold_is_one_integer_on_both_sides(lib_path):
    """The tolerance test of Algorithm 1 (Section 4.1.3), dN / N <= tau, is
    one integer threshold per graph, floor(tau * N): the library's helper
    (the same inline function the device's loop control calls) equals the
    exact floor of the decimal tolerance times N and agrees with the oracle's
    test on both sides of it.  At N = 100,000,019 and tau = 0.05 (0.05 N =
    5,000,000.95) dN = 5,000,001 must not stop a run; the fp32 value of 0.05
    would have stopped it."""
    from fractions import Fraction

    import numpy as np

    import oracle as O
    import paper_2312_08140_gb300 as lpa
    lpa.load(lib_path)
    n = 100_000_019
    assert lpa.lpa_tolerance_threshold(0.05, n) == 5_000_000
    assert O.converged(5_000_000, n, 0.05) and not O.converged(5_000_001, n, 0.05)
    assert int(np.floor(float(np.float32(0.05)) * n)) == 5_000_001
    assert lpa.lpa_tolerance_threshold(0.0, 12) == 0 and lpa.lpa_tolerance_threshold(1.0, 12) == 12
    assert lpa.lpa_tolerance_threshold(0.05, 0) == 0
    rng = np.random.default_rng(12)
    for text in ("0.05", "0.1", "0.01", "0.00001", "0.3"):
        tau = float(text)
        for N in [1, 19, 20, 21, 2**31 - 1] + rng.integers(1, 2**31 - 1, size=300).tolist():
            thr = lpa.lpa_tolerance_threshold(tau, int(N))
            assert thr == int(Fraction(text) * int(N)), (text, N)
            assert O.converged(thr, int(N), tau) and (thr + 1 > N or not O.converged(thr + 1, int(N), tau))
    for bad in ((-0.1, 5), (1.5, 5), (float("nan"), 5), (0.05, -1), (0.05, 2**31)):
        with pytest.raises(lpa.LpaError) as e:
            lpa.lpa_tolerance_threshold(*bad)
        assert e.value.status == lpa.LPA_ERR_INVALID_ARG


def test_struct_layouts_match_c(lib_path):
    import paper_2312_08140_gb300 as lpa
    H = lpa.LPA_MAX_RECORDED_ITERS
    assert ctypes.sizeof(lpa.LpaRunInfo) == 8 + 3 * 8 * H + 8
    assert ctypes.sizeof(lpa.LpaGraphProps) == 8 * 2 + 4 * 4 + 8 * 5 + 4 * 2
    assert ctypes.sizeof(lpa.LpaConfig) == 20
    B = lpa.LPA_BINS
    assert ctypes.sizeof(lpa.LpaProfile) == 16 + 4 * H + 4 * B * H + 4 * B * 8 * H


_C_STRUCTS = {"LpaRunInfo": "lpa_run_info", "LpaGraphProps": "lpa_graph_props", "LpaConfig": "lpa_config",
              "LpaProfile": "lpa_profile", "LpaServeConfig": "lpa_serve_config",
              "LpaServeStats": "lpa_serve_stats_t", "LpaAutotuneInfo": "lpa_autotune_info"}


def test_header_is_plain_c_and_layouts_match_the_binding(lib_path, tmp_path):
    """A C11 program (no C++) includes lpa.h, links liblpa.so, prints every
    struct's size and field offsets, and calls the host-only entry points: the
    binding's ctypes layouts must agree field by field."""
    import paper_2312_08140_gb300 as lpa
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include <string.h>', '#include "lpa.h"',
             'int main(void) {']
    for py, c in _C_STRUCTS.items():
        lines.append(f'    printf("{py} . %zu\\n", sizeof({c}));')
        for f, _ in getattr(lpa, py)._fields_:
            lines.append(f'    printf("{py} {f} %zu\\n", offsetof({c}, {f}));')
    lines += ['    lpa_graph_t g = 0;',
              '    if (lpa_graph_create(-1, 0, 0, 0, 0, LPA_HOST_PTRS, 0, &g) != LPA_ERR_INVALID_ARG) return 2;',
              '    if (strcmp(lpa_status_string(LPA_ERR_INVALID_GRAPH), "invalid graph") != 0) return 3;',
              '    printf("version %s\\n", lpa_version());',
              '    return 0;', '}']
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "abi"
    libdir = os.path.dirname(lib_path)
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe),
                           "-L", libdir, "-l:" + os.path.basename(lib_path), "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    *layout, version = out.stdout.rstrip().splitlines()
    assert version.startswith("version lpa-gb300")
    got = {}
    for ln in layout:
        a, b, v = ln.split(" ")
        got[(a, b)] = v
    for py in _C_STRUCTS:
        cls = getattr(lpa, py)
        assert int(got[(py, ".")]) == ctypes.sizeof(cls), py
        for f, _ in cls._fields_:
            assert int(got[(py, f)]) == getattr(cls, f).offset, (py, f)
