"""The boundary is a C ABI: include/fastalign.h compiles as strict C99 on
its own, and a plain C program links the in-tree library and gets the
expected answers from its host-only entries (CPU only; no device work)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2607_11952_gb300")


def test_plain_c_program_uses_the_abi(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_2607_11952_gb300 import _lib as L
    L.lib()                                       # the library is built and loads
    exe = str(tmp_path / "abi_check")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", os.path.join(ROOT, "include"),
                        os.path.join(ROOT, "tests", "c", "abi_check.c"),
                        "-L", PKG, "-lfastalign", f"-Wl,-rpath,{PKG}", "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    lines = dict(l.split(" ", 1) for l in r.stdout.strip().splitlines())
    assert lines["params"] == "10 1 0.05 0.50"
    assert lines["plan"] == "0 5 10016 5 1 5 256"
    # rows 0..2 each see the other two, node 3 is isolated
    assert lines["csr"] == "0 6 0 2 4 6 6 1 0.50"
    assert lines["error"] == "1 1"
    assert "bad edge arrays" in lines["message"]
