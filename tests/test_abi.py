"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/enuf.h declares, and validates plan parameters."""
import ctypes
import os
import re

import pytest

import paper_2004_12484_b300 as P

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "enuf.h")


def declared_functions():
    text = open(HDR).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(enuf_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = P.lib()
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_checked_build_exports_the_same_symbols():
    """libenuf_check.so (bounds checks in every kernel) has the same entry
    points as libenuf.so and says that it is the checked build; libenuf.so
    says that it is not."""
    chk = ctypes.CDLL(os.path.join(os.path.dirname(P.LIB_PATH), "libenuf_check.so"))
    for n in declared_functions():
        assert hasattr(chk, n), n
    rel = ctypes.CDLL(os.path.join(os.path.dirname(P.LIB_PATH), "libenuf.so"))
    assert chk.enuf_bounds_checked() == 1
    assert rel.enuf_bounds_checked() == 0
    # without a GPU the release library still answers: no checks, no failures
    fails = ctypes.c_ulonglong(5)
    assert rel.enuf_bounds_status(ctypes.byref(fails), None, 0, 0) == 0
    assert fails.value == 0
    assert rel.enuf_bounds_selftest() == -1  # ENUF_EINVAL: not the checked build


def test_probe_library_is_separate_and_exports_its_header():
    """The benchmark's FMA probe lives in its own library, not in libenuf.so."""
    lib = P.lib()
    assert not hasattr(lib, "enuf_fma_peak_tflops")
    phdr = os.path.join(os.path.dirname(HDR), "enuf_probe.h")
    text = re.sub(r"/\*.*?\*/", "", open(phdr).read(), flags=re.S)
    names = sorted(set(re.findall(r"\b(enuf_[a-z0-9_]+)\s*\(", text)))
    probe = ctypes.CDLL(os.path.join(os.path.dirname(P.LIB_PATH), "libenuf_probe.so"))
    assert names == ["enuf_fma_peak_tflops", "enuf_probe_last_error"]
    for n in names:
        assert hasattr(probe, n), n


def test_params_struct_matches_header_layout(tmp_path):
    """The binding's ctypes structure has the size and field offsets that
    a C compiler gives enuf_params from the header."""
    import subprocess
    fields = [f[0] for f in P.EnufParams._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "enuf.h"\nint main(void) {\n'
                   + '    printf("%zu\\n", sizeof(enuf_params));\n'
                   + "".join(f'    printf("%zu\\n", offsetof(enuf_params, {f}));\n' for f in fields)
                   + "    return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HDR), "-o", str(exe), str(src)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert got[0] == ctypes.sizeof(P.EnufParams)
    for f, off in zip(fields, got[1:]):
        assert getattr(P.EnufParams, f).offset == off, f


def base(**kw):
    d = dict(L=(20.0, 20.0, 20.0), N=100, alpha=0.3, r_c=9.0, M=32, p=4, n_c=0, precision="mixed")
    d.update(kw)
    return d


def test_workspace_bytes_scales_with_grid():
    a = P.workspace_bytes(**base(M=32))
    b = P.workspace_bytes(**base(M=64))
    assert b > 6 * a


@pytest.mark.parametrize("bad", [dict(M=48), dict(M=4), dict(M=1024), dict(p=5), dict(p=14), dict(p=0),
                                 dict(n_c=16), dict(n_c=-1), dict(r_c=11.0), dict(r_c=0.0), dict(alpha=0.0),
                                 dict(N=0), dict(L=(20.0, -1.0, 20.0)), dict(precision=7),
                                 dict(slater_lambda=-1.0), dict(slater_lambda=float("inf"))])
def test_invalid_parameters_are_rejected(bad):
    with pytest.raises(P.EnufError):
        P.workspace_bytes(**base(**bad))


def test_error_message_is_reported():
    with pytest.raises(P.EnufError, match="power of two"):
        P.workspace_bytes(**base(M=48))


def test_entry_points_reject_a_missing_plan():
    """Every call that takes a plan reports ENUF_EINVAL for NULL instead of
    touching the device."""
    L = P.lib()
    v = ctypes.c_void_p
    assert L.enuf_compute(None, v(1), v(1), None, None, None, 0) == -1
    assert L.enuf_backward_flags(None, v(1), v(1), None, v(1), v(1), 0) == -1
    assert L.enuf_md_run(None, v(1), v(1), v(1), v(1), v(1), 0, 0.1, 1, 0, v(1)) == -1


def test_slater_decay_length_is_accepted():
    assert P.workspace_bytes(**base(slater_lambda=0.889)) == P.workspace_bytes(**base())

