"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/mpdiv.h declares, and rejects bad arguments before any
GPU work (no compute call is made here)."""

import ctypes
import os
import re
import subprocess

import pytest

import paper_2606_06386_gb300 as mp

HEADER = mp.HEADER


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpdiv_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    mp.build()
    return mp.lib()


def test_every_declared_function_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", mp.SO_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mpdiv_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_binding_covers_the_header(lib):
    for n in _declared():
        assert n in mp._SIGS, f"{n} has no binding"


def test_null_context_and_bad_arguments_are_rejected(lib):
    assert lib.mpdiv_batch(None, 1, None, 1, 1, None, 1, 1, None, 1, 1, None, 1, 1, None, None, None, None) == mp.MPDIV_EINVAL
    assert lib.mpdiv_init(None, 0, None) == mp.MPDIV_EINVAL
    assert lib.mpdiv_serve_submit(None, None, 1, None, 1, None) == mp.MPDIV_EINVAL
    assert lib.mpdiv_last_error(None) == b"null context"
    # the allocation-free entry checks sizes before touching the GPU
    one = (ctypes.c_int32 * 1)(1)
    assert lib.mpdiv_batch_ragged_noalloc(-1, *([None] * 14), None) == mp.MPDIV_EINVAL
    assert lib.mpdiv_batch_ragged_noalloc(mp.MPDIV_NOALLOC_MAX_ITEMS + 1, *([None] * 13), one, None) == mp.MPDIV_EUNSUPPORTED


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(mp, "SO_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(mp, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        mp.lib()


def test_config_structs_match_the_header(tmp_path):
    # the binding's ctypes structures against the C compiler's layout of the
    # header's structs (size and every field offset)
    import ctypes
    import subprocess

    import paper_2606_06386_gb300 as mp

    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = {"mpdiv_config": mp.mpdiv_config, "mpdiv_serve_config": mp.mpdiv_serve_config}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mpdiv.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = str(tmp_path / "layout")
    subprocess.run(["gcc", "-I", inc, str(src), "-o", exe], check=True)
    got = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    want = []
    for name, cls in structs.items():
        want.append(f"{name} size {ctypes.sizeof(cls)}")
        want += [f"{name} {f} {getattr(cls, f).offset}" for f, _ in cls._fields_]
    assert [g for g in got if g] == want
