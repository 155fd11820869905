"""ctypes binding of libfastalign.so (include/fastalign.h).

Argument marshalling only: every function here has the name and argument
order of its C counterpart, converts torch tensors / numpy arrays to raw
pointers, and raises ``FastAlignError`` on a non-OK status.  There is no
fallback: if the library is missing or the GPU is absent the calls fail.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfastalign.so")

FA_OK, FA_ERR_ARG, FA_ERR_OOM, FA_ERR_CUDA, FA_ERR_NOT_CONVERGED, \
    FA_ERR_NUMERIC, FA_ERR_UNSUPPORTED, FA_ERR_TIMEOUT = range(8)
STATUS_NAMES = ["FA_OK", "FA_ERR_ARG", "FA_ERR_OOM", "FA_ERR_CUDA",
                "FA_ERR_NOT_CONVERGED", "FA_ERR_NUMERIC", "FA_ERR_UNSUPPORTED",
                "FA_ERR_TIMEOUT"]
FA_F32, FA_BF16 = 0, 1
FA_GEMM_AUTO, FA_GEMM_TCGEN05, FA_GEMM_SIMT = 0, 1, 2


class FastAlignError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {detail}")


class fa_params(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int32),
        ("eps", ctypes.c_float),
        ("eps_anc", ctypes.c_float),
        ("alpha", ctypes.c_float),
        ("beta", ctypes.c_float),
        ("k_rwr", ctypes.c_int32),
        ("k_prop", ctypes.c_int32),
        ("lam_e", ctypes.c_float),
        ("lam_n", ctypes.c_float),
        ("lam_a", ctypes.c_float),
        ("lam_p", ctypes.c_float),
        ("delta", ctypes.c_float),
        ("normalize_features", ctypes.c_int32),
        ("gemm_mode", ctypes.c_int32),
    ]


_c = ctypes
_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f64 = ctypes.c_double

# name -> (restype, argtypes); mirrors include/fastalign.h
SIGNATURES = {
    "fa_params_default": (None, [ctypes.POINTER(fa_params)]),
    "fa_build_graph": (_i32, [_i32, _i64, _p, _p, ctypes.POINTER(_p)]),
    "fa_graph_destroy": (_i32, [_p]),
    "fa_graph_info": (_i32, [_p, ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "fa_ctx_create": (_i32, [_p, _p, ctypes.POINTER(fa_params), ctypes.POINTER(_p)]),
    "fa_ctx_destroy": (_i32, [_p]),
    "fa_ctx_ld": (_i64, [_p]),
    "fa_ctx_workspace_bytes": (_i64, [_p]),
    "fa_node_cost": (_i32, [_p, _p, _p, _i32, _p, _i32, _p, _p]),
    "fa_plan_init": (_i32, [_p, _p, _p, _p, _p]),
    "fa_align_iter": (_i32, [_p, _p, _p, _p, _p, _p]),
    "fa_sinkhorn": (_i32, [_p, _p, _p, _p, _p, _i32, _f64, _i32,
                           ctypes.POINTER(_i32), ctypes.POINTER(_f64), _p]),
    "fa_topk": (_i32, [_p, _p, _p, _i32, _p, _p, _p]),
    "fa_rank": (_i32, [_p, _p, _p, _i32, _p, _p, _p, _p]),
    "fa_ctx_set_timing": (_i32, [_p, _i32]),
    "fa_ctx_last_sweep_ms": (_i32, [_p, ctypes.POINTER(_f64), ctypes.POINTER(_i32)]),
    "fa_last_error_string": (ctypes.c_char_p, []),
    "fa_kernel_launch_count": (_i64, []),
    "fa_gnn_create": (_i32, [ctypes.POINTER(_p)]),
    "fa_gnn_destroy": (_i32, [_p]),
    "fa_gnn_set_params": (_i32, [_p, _p]),
    "fa_gnn_get_params": (_i32, [_p, _p]),
    "fa_gnn_workspace_floats": (_i64, [_i32]),
    "fa_gnn_features": (_i32, [_p, _p, _p, _p, _p, _i32, _p, _p, _p]),
    "fa_gnn_forward": (_i32, [_p, _p, _p, _p, _p, _p]),
    "fa_gnn_backward": (_i32, [_p, _p, _p, _p, _p, _p, _p, _p]),
    "fa_gnn_adam_step": (_i32, [_p, _p, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                ctypes.c_float, _p]),
    "fa_vec_axpby": (_i32, [_i32, ctypes.c_float, _p, ctypes.c_float, _p, _p, _p]),
    "fa_gnn_warm_start": (_i32, [_i32, _p, _p, ctypes.c_float, _p, _p, _p]),
    "fa_gnn_fit_scale": (_i32, [_i32, _p, _p, ctypes.c_float, _i32, _p, _p]),
    "fa_sinkhorn_step_static": (_i32, [_p, _i32, _i32, _i32, _i64, _p, _p, _p, _p, _p, _p]),
    "fa_plan_change": (_i32, [_p, _p, _p, _p, _p, _p, _p, _p, _p]),
    "fa_ctx_selftest_wait": (_i32, [_p, _p]),
    "fa_graph_csr_host": (_i32, [_i32, _i64, _p, _p, ctypes.POINTER(_i64), _p, _p, _p, _p,
                                 _i64]),
    "fa_sweep_plan": (_i32, [_i32, _i64, _i32, _p]),
    "fa_shard_blocks": (_i64, [_i64]),
    "fa_sinkhorn_shard_rows": (_i32, [_p, _p, _p, _i64, _i64, _p, _p]),
    "fa_sinkhorn_shard_combine": (_i32, [_p, _p, _p, _p]),
    "fa_sinkhorn_shard_cols": (_i32, [_p, _p, _p, _p, _i64, _i64, _p, _p, _p]),
}

FA_SHARD_BLOCK = 2048
FA_GNN_FIN, FA_GNN_HIDDEN = 6, 64
FA_GNN_NPARAMS = FA_GNN_FIN * FA_GNN_HIDDEN + 2 * FA_GNN_HIDDEN + 1

_lib = None


def lib() -> ctypes.CDLL:
    """Load the in-tree library (fails loudly if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                "(or python -m paper_2607_11952_gb300._build)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status: int, where: str) -> int:
    if status != FA_OK:
        detail = lib().fa_last_error_string()
        raise FastAlignError(status, where, detail.decode() if detail else "")
    return status


def ptr(x) -> int | None:
    """Raw address of a torch tensor or numpy array (None passes NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x)


def stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ------------------------------------------------------------ entry points

def fa_params_default() -> fa_params:
    p = fa_params()
    lib().fa_params_default(ctypes.byref(p))
    return p


def fa_build_graph(n: int, src: np.ndarray, dst: np.ndarray) -> int:
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    out = _p()
    _check(lib().fa_build_graph(n, src.shape[0], ptr(src), ptr(dst), ctypes.byref(out)),
           "fa_build_graph")
    return out.value


def fa_graph_destroy(g: int) -> None:
    _check(lib().fa_graph_destroy(g), "fa_graph_destroy")


def fa_graph_info(g: int):
    n = _i32()
    nnz = _i64()
    _check(lib().fa_graph_info(g, ctypes.byref(n), ctypes.byref(nnz)), "fa_graph_info")
    return n.value, nnz.value


def fa_ctx_create(g1: int, g2: int, params: fa_params) -> int:
    out = _p()
    _check(lib().fa_ctx_create(g1, g2, ctypes.byref(params), ctypes.byref(out)),
           "fa_ctx_create")
    return out.value


def fa_ctx_destroy(ctx: int) -> None:
    _check(lib().fa_ctx_destroy(ctx), "fa_ctx_destroy")


def fa_ctx_ld(ctx: int) -> int:
    return lib().fa_ctx_ld(ctx)


def fa_ctx_workspace_bytes(ctx: int) -> int:
    return lib().fa_ctx_workspace_bytes(ctx)


def fa_node_cost(ctx, X1, X2, d, anchors: np.ndarray, C_node, stream=None) -> None:
    a = np.ascontiguousarray(anchors, dtype=np.int32).reshape(-1, 2)
    _check(lib().fa_node_cost(ctx, ptr(X1), ptr(X2), d, ptr(a) if a.size else None,
                              a.shape[0], ptr(C_node), stream_ptr(stream)),
           "fa_node_cost")


def fa_plan_init(ctx, K, log_u, log_v, stream=None) -> None:
    _check(lib().fa_plan_init(ctx, ptr(K), ptr(log_u), ptr(log_v), stream_ptr(stream)),
           "fa_plan_init")


def fa_align_iter(ctx, K, log_u, log_v, C_node, stream=None) -> None:
    _check(lib().fa_align_iter(ctx, ptr(K), ptr(log_u), ptr(log_v), ptr(C_node),
                               stream_ptr(stream)), "fa_align_iter")


def fa_sinkhorn(ctx, K, log_u, log_v, warm_log_v, max_iter, tol, check_every,
                stream=None, allow_not_converged: bool = True):
    it = _i32()
    err = _f64()
    st = lib().fa_sinkhorn(ctx, ptr(K), ptr(log_u), ptr(log_v), ptr(warm_log_v),
                           int(max_iter), float(tol), int(check_every),
                           ctypes.byref(it), ctypes.byref(err), stream_ptr(stream))
    if not (allow_not_converged and st == FA_ERR_NOT_CONVERGED):
        _check(st, "fa_sinkhorn")
    return it.value, err.value, st


def fa_graph_csr_host(n: int, src: np.ndarray, dst: np.ndarray):
    """Host CSR of fa_build_graph: (row_ptr, col, val_row, val_col) as
    NumPy arrays (int32, int32, float32, float32)."""
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = int(src.shape[0])
    nnz = _i64()
    _check(lib().fa_graph_csr_host(int(n), m, src.ctypes.data, dst.ctypes.data,
                                   ctypes.byref(nnz), None, None, None, None, 0),
           "fa_graph_csr_host")
    k = int(nnz.value)
    rp = np.empty(int(n) + 1, np.int32)
    col = np.empty(max(k, 1), np.int32)
    vr = np.empty(max(k, 1), np.float32)
    vc = np.empty(max(k, 1), np.float32)
    _check(lib().fa_graph_csr_host(int(n), m, src.ctypes.data, dst.ctypes.data,
                                   ctypes.byref(nnz), rp.ctypes.data, col.ctypes.data,
                                   vr.ctypes.data, vc.ctypes.data, max(k, 1)),
           "fa_graph_csr_host")
    return rp, col[:k], vr[:k], vc[:k]


SWEEP_PLAN_FIELDS = ("Q", "W", "S", "R", "NS", "NT", "kind", "G")


def fa_sweep_plan(n1: int, ld: int, dtype: int) -> dict:
    out = (_i32 * 8)()
    _check(lib().fa_sweep_plan(int(n1), int(ld), int(dtype), out), "fa_sweep_plan")
    return dict(zip(SWEEP_PLAN_FIELDS, list(out)))


def fa_ctx_selftest_wait(ctx, stream=None) -> None:
    _check(lib().fa_ctx_selftest_wait(ctx, stream_ptr(stream)), "fa_ctx_selftest_wait")


def fa_topk(ctx, K, log_v, k, idx, score, stream=None) -> None:
    _check(lib().fa_topk(ctx, ptr(K), ptr(log_v), int(k), ptr(idx), ptr(score),
                         stream_ptr(stream)), "fa_topk")


def fa_rank(ctx, K, log_v, rows, cols, rank_out, stream=None) -> None:
    n = 0 if rows is None else int(rows.numel() if hasattr(rows, "numel") else len(rows))
    _check(lib().fa_rank(ctx, ptr(K), ptr(log_v), n, ptr(rows), ptr(cols), ptr(rank_out),
                         stream_ptr(stream)), "fa_rank")


def fa_ctx_set_timing(ctx, on: bool) -> None:
    _check(lib().fa_ctx_set_timing(ctx, 1 if on else 0), "fa_ctx_set_timing")


def fa_ctx_last_sweep_ms(ctx):
    ms = _f64()
    n = _i32()
    _check(lib().fa_ctx_last_sweep_ms(ctx, ctypes.byref(ms), ctypes.byref(n)),
           "fa_ctx_last_sweep_ms")
    return ms.value, n.value


def fa_last_error_string() -> str:
    s = lib().fa_last_error_string()
    return s.decode() if s else ""


def fa_kernel_launch_count() -> int:
    return lib().fa_kernel_launch_count()


# ------------------------------------------------------------ learned warm start

def fa_gnn_create() -> int:
    out = _p()
    _check(lib().fa_gnn_create(ctypes.byref(out)), "fa_gnn_create")
    return out.value


def fa_gnn_destroy(m: int) -> None:
    _check(lib().fa_gnn_destroy(m), "fa_gnn_destroy")


def fa_gnn_set_params(m: int, theta: np.ndarray) -> None:
    t = np.ascontiguousarray(theta, dtype=np.float32)
    if t.size != FA_GNN_NPARAMS:
        raise ValueError(f"expected {FA_GNN_NPARAMS} parameters")
    _check(lib().fa_gnn_set_params(m, ptr(t)), "fa_gnn_set_params")


def fa_gnn_get_params(m: int) -> np.ndarray:
    t = np.empty(FA_GNN_NPARAMS, np.float32)
    _check(lib().fa_gnn_get_params(m, ptr(t)), "fa_gnn_get_params")
    return t


def fa_gnn_workspace_floats(n: int) -> int:
    return lib().fa_gnn_workspace_floats(n)


def fa_gnn_features(g2, log_v1, corr_prev, pot_prev, anchor_mask, outer_index, F, ws,
                    stream=None) -> None:
    _check(lib().fa_gnn_features(g2, ptr(log_v1), ptr(corr_prev), ptr(pot_prev),
                                 ptr(anchor_mask), int(outer_index), ptr(F), ptr(ws),
                                 stream_ptr(stream)), "fa_gnn_features")


def fa_gnn_forward(m, g, F, ws, a_out, stream=None) -> None:
    _check(lib().fa_gnn_forward(m, g, ptr(F), ptr(ws), ptr(a_out), stream_ptr(stream)),
           "fa_gnn_forward")


def fa_gnn_backward(m, g, ws, a_pred, target, grad, loss, stream=None) -> None:
    _check(lib().fa_gnn_backward(m, g, ptr(ws), ptr(a_pred), ptr(target), ptr(grad),
                                 ptr(loss), stream_ptr(stream)), "fa_gnn_backward")


def fa_gnn_adam_step(m, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None) -> None:
    _check(lib().fa_gnn_adam_step(m, ptr(grad), float(lr), float(beta1), float(beta2),
                                  float(eps), stream_ptr(stream)), "fa_gnn_adam_step")


def fa_vec_axpby(n, a, x, b, y, out, stream=None) -> None:
    _check(lib().fa_vec_axpby(int(n), float(a), ptr(x), float(b), ptr(y), ptr(out),
                              stream_ptr(stream)), "fa_vec_axpby")


def fa_gnn_warm_start(n, log_v1, pred, max_abs, out, scale=None, stream=None) -> None:
    _check(lib().fa_gnn_warm_start(int(n), ptr(log_v1), ptr(pred), float(max_abs), ptr(scale),
                                   ptr(out), stream_ptr(stream)), "fa_gnn_warm_start")


def fa_gnn_fit_scale(n, pred, y, max_abs, scale, shrink=0, stream=None) -> None:
    _check(lib().fa_gnn_fit_scale(int(n), ptr(pred), ptr(y), float(max_abs), int(shrink),
                                  ptr(scale), stream_ptr(stream)), "fa_gnn_fit_scale")


def fa_sinkhorn_step_static(K, dtype, n1, n2, ld, log_v, log_u, log_v_next, err, status=None,
                            stream=None) -> None:
    _check(lib().fa_sinkhorn_step_static(ptr(K), int(dtype), int(n1), int(n2), int(ld),
                                         ptr(log_v), ptr(log_u), ptr(log_v_next), ptr(err),
                                         ptr(status), stream_ptr(stream)),
           "fa_sinkhorn_step_static")


def fa_plan_change(ctx, K_a, log_u_a, log_v_a, K_b, log_u_b, log_v_b, stream=None) -> float:
    out = _f64()
    _check(lib().fa_plan_change(ctx, ptr(K_a), ptr(log_u_a), ptr(log_v_a), ptr(K_b),
                                ptr(log_u_b), ptr(log_v_b), ctypes.byref(out),
                                stream_ptr(stream)), "fa_plan_change")
    return out.value


def fa_shard_blocks(ld: int) -> int:
    return int(lib().fa_shard_blocks(int(ld)))


def fa_sinkhorn_shard_rows(ctx, K, log_v, j0, j1, row_partials, stream=None) -> None:
    _check(lib().fa_sinkhorn_shard_rows(ctx, ptr(K), ptr(log_v), int(j0), int(j1),
                                        ptr(row_partials), stream_ptr(stream)),
           "fa_sinkhorn_shard_rows")


def fa_sinkhorn_shard_combine(ctx, row_partials, log_u, stream=None) -> None:
    _check(lib().fa_sinkhorn_shard_combine(ctx, ptr(row_partials), ptr(log_u),
                                           stream_ptr(stream)), "fa_sinkhorn_shard_combine")


def fa_sinkhorn_shard_cols(ctx, K, log_u, log_v, j0, j1, log_v_next, err=None,
                           stream=None) -> None:
    _check(lib().fa_sinkhorn_shard_cols(ctx, ptr(K), ptr(log_u), ptr(log_v), int(j0), int(j1),
                                        ptr(log_v_next), ptr(err), stream_ptr(stream)),
           "fa_sinkhorn_shard_cols")
