"""The product path and the oracle stay apart, and the product path has no
fallback (CPU only).

* No module of the package, nor bench.py outside its CPU-baseline and
  reference legs, imports the oracle; the oracle imports nothing from the
  package.
* Without the compiled library every entry point raises at once instead of
  computing anything another way.
"""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2607_11952_gb300")


def _imports(path):
    tree = ast.parse(open(path).read(), filename=path)
    out = []
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            out += [(a.name, node) for a in node.names]
        elif isinstance(node, ast.ImportFrom):
            out.append((("." * node.level) + (node.module or ""), node))
    return tree, out


def test_package_never_imports_the_oracle():
    for name in sorted(os.listdir(PKG)):
        if name.endswith(".py"):
            _, imps = _imports(os.path.join(PKG, name))
            assert not any(m.split(".")[0] == "oracle" for m, _ in imps), name


def test_oracle_never_imports_the_package():
    odir = os.path.join(ROOT, "oracle")
    for name in sorted(os.listdir(odir)):
        if name.endswith(".py"):
            _, imps = _imports(os.path.join(odir, name))
            assert not any("paper_2607_11952_gb300" in m or m.startswith("..")
                           for m, _ in imps), name


def test_bench_uses_the_oracle_only_in_its_cpu_legs():
    tree, imps = _imports(os.path.join(ROOT, "bench.py"))
    allowed = {"_oracle_run"}          # shared by the cpu_baseline leg and --impl reference
    funcs = [f for f in ast.walk(tree) if isinstance(f, ast.FunctionDef)]
    for m, node in imps:
        if m.split(".")[0] != "oracle":
            continue
        owner = [f.name for f in funcs
                 if f.lineno <= node.lineno <= max(getattr(n, "lineno", 0) for n in ast.walk(f))]
        assert owner and set(owner) <= allowed, (m, owner)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2607_11952_gb300 import _lib as L
    monkeypatch.setattr(L, "LIB_PATH", str(tmp_path / "libfastalign.so"))
    monkeypatch.setattr(L, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        L.fa_params_default()
    with pytest.raises(RuntimeError, match="missing"):
        L.fa_sweep_plan(10, 128, L.FA_BF16)
