"""The C ABI library without a GPU: it builds, loads, exports every symbol that include/egh.h
declares, its structs have the header's layout, and argument checks answer before any device
call."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2512_16642_gb300 import build, egh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "egh.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return egh.load()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(egh_\w+)\s*\(", text, re.M)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", egh.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(egh_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(egh.EXPORTS) == set(names)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "egh.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(egh_config),'
                   ' offsetof(egh_config, freq_hz), offsetof(egh_config, reserved), sizeof(egh_stats),'
                   ' offsetof(egh_stats, mu), offsetof(egh_stats, gram_splits), offsetof(egh_config, fd_rows),'
                   ' offsetof(egh_stats, fd_rows), offsetof(egh_stats, gram_ms), offsetof(egh_config, fd_kernel),'
                   ' offsetof(egh_stats, fd_tiles));return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()))
    ref = [ctypes.sizeof(egh.egh_config), egh.egh_config.freq_hz.offset, egh.egh_config.reserved.offset,
           ctypes.sizeof(egh.egh_stats), egh.egh_stats.mu.offset, egh.egh_stats.gram_splits.offset,
           egh.egh_config.fd_rows.offset, egh.egh_stats.fd_rows.offset, egh.egh_stats.gram_ms.offset,
           egh.egh_config.fd_kernel.offset, egh.egh_stats.fd_tiles.offset]
    assert got == ref


def test_version_and_status_strings(lib):
    assert egh.egh_version() == 10000
    assert egh.status_string(egh.EGH_ENOTPD) == "EGH_ENOTPD"
    assert egh.status_string(99) == "EGH_UNKNOWN"


@pytest.mark.parametrize("bad", [
    dict(nz=0), dict(dx=0.0), dict(dt=-1.0), dict(nt=0), dict(rec_ix=[0, 200]),
    dict(freq_hz=[600.0]), dict(freq_hz=[0.0]), dict(sponge_R=1.5), dict(dft_chunk=7), dict(dft_chunk=16),
    dict(freq_hz=np.arange(1, 66) * 1.0),
])
def test_create_rejects_bad_config(lib, bad):
    args = dict(nz=20, nx=30, dz=10.0, dx=10.0, nsponge=5, sponge_R=1e-3, dt=1e-3, nt=50,
                rec_iz=[0, 0], rec_ix=[0, 5], freq_hz=[5.0, 6.0])
    args.update(bad)
    if "rec_ix" in bad:
        args["rec_iz"] = [0] * len(bad["rec_ix"])
    with pytest.raises(egh.EghError) as ei:
        egh.egh_create(**args)
    assert ei.value.status == egh.EGH_EINVAL


def test_null_context_is_rejected(lib):
    assert lib.egh_green(None, None, None) == egh.EGH_EINVAL
    assert lib.egh_factor(None, None, None) == egh.EGH_EINVAL
    lib.egh_destroy(None)


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: without the compiled library every entry point raises (a fresh process, so
    that no library is loaded yet)."""
    import sys

    code = ("import sys; sys.path.insert(0, %r)\n"
            "from paper_2512_16642_gb300 import egh\n"
            "egh.LIB_PATH = %r\n"
            "egh.load.__defaults__ = (egh.LIB_PATH,)\n"
            "try:\n"
            "    egh.Context(4, 4, 10.0, 10.0, 1, 1e-3, 1e-3, 4, [0], [0], [10.0])\n"
            "except RuntimeError as e:\n"
            "    print('raised:', e)\n"
            "else:\n"
            "    print('no error')\n") % (ROOT, str(tmp_path / "libegh.so"))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert "raised: libegh.so not built" in out.stdout, out.stdout + out.stderr
