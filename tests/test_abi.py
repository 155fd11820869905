"""The C-ABI library builds, loads and exports every symbol include/*.h
declares; host-side argument checks answer without touching the GPU."""
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fa_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_11952_gb300 import _lib
    return _lib


def test_every_declared_symbol_is_exported(lib):
    L = lib.lib()
    names = _declared_symbols()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"
    assert set(lib.SIGNATURES) <= set(names) | {"fa_params_default"}


def test_param_defaults_match_oracle(lib):
    from oracle import fastalign_ref as R
    p = lib.fa_params_default()
    o = R.Params()
    for f in ("eps", "eps_anc", "alpha", "beta", "lam_e", "lam_n", "lam_a", "lam_p"):
        assert getattr(p, f) == pytest.approx(getattr(o, f), rel=1e-7), f
    assert p.k_rwr == o.k_rwr and p.k_prop == o.k_prop
    assert p.delta == pytest.approx(o.delta, rel=1e-6)
    assert p.normalize_features == 1 and p.dtype == lib.FA_F32


def test_build_graph_rejects_bad_arguments_on_host(lib):
    with pytest.raises(lib.FastAlignError) as e:
        lib.fa_build_graph(0, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert e.value.status == lib.FA_ERR_ARG
    with pytest.raises(lib.FastAlignError) as e:
        lib.fa_build_graph(5, np.array([0, 1]), np.array([1, 7]))
    assert e.value.status == lib.FA_ERR_ARG
    assert "outside" in lib.fa_last_error_string()
    with pytest.raises(lib.FastAlignError) as e:
        lib.fa_build_graph(5, np.array([0, -1]), np.array([1, 2]))
    assert e.value.status == lib.FA_ERR_ARG


def test_null_handles_are_argument_errors(lib):
    L = lib.lib()
    assert L.fa_ctx_create(None, None, None, None) == lib.FA_ERR_ARG
    assert L.fa_sinkhorn(None, None, None, None, None, 1, -1.0, 1, None, None, None) == lib.FA_ERR_ARG
    assert L.fa_topk(None, None, None, 1, None, None, None) == lib.FA_ERR_ARG
    assert L.fa_graph_info(None, None, None) == lib.FA_ERR_ARG
    assert L.fa_ctx_ld(None) == -1
    assert L.fa_graph_destroy(None) == lib.FA_OK
    assert L.fa_ctx_destroy(None) == lib.FA_OK
