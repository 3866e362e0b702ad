"""The C-ABI library builds, loads and exports every symbol include/*.h declares
(CPU only: no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(dos_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1308_5467_gb300.build import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dos_ctx_create", "dos_ctx_destroy", "dos_bounds", "dos_kpm_moments",
                     "dos_kpm_moments_batched", "dos_reconstruct", "dos_smoothed_error",
                     "dos_start_vectors", "dos_tune"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_status_strings(lib):
    lib.dos_status_string.restype = ctypes.c_char_p
    assert lib.dos_status_string(0) == b"DOS_OK"
    assert lib.dos_status_string(4) == b"DOS_ESPECTRUM"
    assert lib.dos_status_string(99) == b"DOS_UNKNOWN"


def test_binding_loads_and_null_context_is_rejected(lib):
    from paper_1308_5467_gb300 import dos
    assert dos._lib.dos_ctx_destroy(None) == dos.DOS_OK
    assert dos._lib.dos_bounds(None, None, 0, 0, 0, 0.0, None, None, None) == dos.DOS_EINVAL


def test_struct_layouts_match_the_binding(tmp_path):
    """The ctypes mirrors of dos_csr, dos_launch and dos_kpm_opts have the C header's
    size and field offsets (a field added on one side only would shift every later
    field the library reads)."""
    import shutil
    import subprocess
    from paper_1308_5467_gb300 import dos
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"dos_csr": dos.dos_csr, "dos_launch": dos.dos_launch,
               "dos_kpm_opts": dos.dos_kpm_opts}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dos.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ['return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        name, field, value = line.split()
        got[(name, field)] = int(value)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
