"""The C-ABI library loads and exports every symbol the header declares (CPU only)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "galario_gb300.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gal_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_06999_gb300 import _native
    return _native.load()


def test_header_declares_entry_points():
    names = _declared()
    for op in ("sweep", "sample_image", "sample_profile", "chi2_image", "chi2_profile"):
        for p in ("f32", "f64"):
            assert f"gal_{op}_{p}" in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_1709_06999_gb300 import _native
    assert sorted(_native.EXPORTED) == _declared()


def test_nm_lists_symbols_as_c(lib):
    from paper_1709_06999_gb300 import _native
    out = subprocess.run(["nm", "-D", "--defined-only", _native.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (gal_\w+)", out))
    assert set(_declared()) <= exported


def test_status_strings(lib):
    assert lib.gal_strerror(0) == b"ok"
    assert lib.gal_strerror(-1) == b"invalid argument"


def test_create_without_gpu_fails_cleanly(lib):
    import ctypes as ct
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ct.c_void_p()
    assert lib.gal_create(ct.byref(h), 0) == -5


def test_options_struct_layout():
    """struct gal_opts { double pb_fwhm; int full_plane; }: the binding's
    ctypes mirror has the C layout (8-byte double, int at offset 8, size 16)."""
    import ctypes as ct
    from paper_1709_06999_gb300._native import GalOpts
    assert ct.sizeof(GalOpts) == 16
    assert GalOpts.pb_fwhm.offset == 0 and GalOpts.full_plane.offset == 8
    text = open(HEADER).read()
    assert re.search(r"typedef struct gal_opts \{\s*double pb_fwhm;\s*int full_plane;\s*\} gal_opts;",
                     text)


def test_struct_layouts_match_c(tmp_path):
    """sizeof and field offsets of the header's structs, compiled by the C
    compiler, equal those of the binding's ctypes mirrors."""
    import ctypes as ct
    import shutil
    from paper_1709_06999_gb300 import _native
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"gal_opts": _native.GalOpts, "gal_request": _native.GalRequest,
               "gal_server_stats": _native.GalServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "galario_gb300.h"',
             'int main(void) {']
    for name, cls in mirrors.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                 check=True).stdout.splitlines())
    for name, cls in mirrors.items():
        assert int(got[name]) == ct.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_fft_radix_plan_validation():
    """The FFT plan calls are host-side: the set of valid radices per side and
    precision, and that a plan set is read back (no GPU needed)."""
    from paper_1709_06999_gb300 import GalError, get_fft_radix, set_fft_radix
    set_fft_radix(5, "float32", 256, 8, 16)
    assert get_fft_radix(5, "float32", 256) == (8, 16)
    set_fft_radix(5, "float32", 256, 16, 8)
    assert get_fft_radix(5, "float32", 256) == (16, 8)
    assert get_fft_radix(5, "float32", 128) == (0, 0)          # not fixed yet
    assert get_fft_radix(5, "float32", 4096) == (16, 16)       # one radix only
    assert get_fft_radix(5, "float64", 256) == (8, 8)
    for bad in ((5, "float32", 1024, 8, 16),    # radix 8 only up to 512
                (5, "float32", 256, 4, 16),     # no radix 4
                (5, "float32", 16, 8, 8),       # below 32
                (5, "float32", 300, 16, 16),    # not a power of two
                (5, "float64", 256, 16, 8),     # float64 runs at 8
                (-1, "float32", 256, 16, 16)):
        with pytest.raises(GalError):
            set_fft_radix(*bad)
