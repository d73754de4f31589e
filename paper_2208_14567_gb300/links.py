"""Thin ctypes binding of the C ABI in include/links.h (same names, argument marshalling only).

Device buffers are torch CUDA tensors (PyTorch provides memory and streams); every
step of the computation runs in the library's CUDA kernels.  Importing this module
does not load the library; the first call does, and raises if the library has not
been built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblinks.so")

# Mirrors of the #defines in include/links.h.
OK, EINVAL, ECUDA, ENOMEM, ECAPACITY, EBUSY, ETIMEDOUT, ESTATE, EDEVICE = range(9)
MECH_OK, MECH_BAD_SIZE, MECH_BAD_TYPE, MECH_BAD_ADJ, MECH_NO_MOTOR, MECH_NO_PIVOT, \
    MECH_NOT_DYAD_SOLVABLE, MECH_OVERCONSTRAINED = range(8)
F32, F64 = 0, 1
PLAIN_F64, MIXED = 0, 1
OUT_FULL, OUT_VALID_ONLY = 0, 1
MAX_JOINTS, MAX_T = 32, 32767

_lib = None


class Request(ctypes.Structure):
    """Mirror of links_request (host buffers)."""
    _fields_ = [("count", ctypes.c_int64), ("n_joints", ctypes.c_void_p), ("adj", ctypes.c_void_p),
                ("type", ctypes.c_void_p), ("pos0", ctypes.c_void_p), ("valid", ctypes.c_void_p),
                ("lock_step", ctypes.c_void_p), ("min_disc", ctypes.c_void_p), ("out_capacity", ctypes.c_int64),
                ("valid_index", ctypes.c_void_p), ("paths", ctypes.c_void_p), ("traj", ctypes.c_void_p)]


class Result(ctypes.Structure):
    """Mirror of links_result."""
    _fields_ = [("status", ctypes.c_int), ("n_valid", ctypes.c_int64), ("submit_ms", ctypes.c_double),
                ("admit_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


class LinksError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str):
        super().__init__(f"{what} failed: {strerror(status)}: {detail}")
        self.status = status


def lib():
    """The loaded CUDA library (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built ({LIB_PATH} missing): run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        sig = {
            "links_last_error": ([], ctypes.c_char_p),
            "links_strerror": ([i32], ctypes.c_char_p),
            "links_create": ([P, i32, P], i32),
            "links_destroy": ([P], i32),
            "links_set_stream": ([P, P], i32),
            "links_sync": ([P], i32),
            "links_prepare": ([P, i32], i32),
            "links_plan_create": ([P, i64, i32, P], i32),
            "links_plan_free": ([P], i32),
            "links_plan_build": ([P, P, i64, P, P, P, P, i32, P], i32),
            "links_plan_build_host": ([P, P, i64, P, P, P, P, i32, P], i32),
            "links_plan_build_masks": ([P, P, i64, P, P, P, P, i32, P], i32),
            "links_plan_info": ([P, P, P, P], i32),
            "links_plan_export": ([P, i64, i64, P, P], i32),
            "links_simulate": ([P, P, i32, i32, i32, P, P, P, P, P, P, i64, P], i32),
            "links_emit_census": ([P, P, i32, i32, P, P, i64, P], i32),
            "links_simulate_two_stage": ([P, P, i32, i32, P, P, P, P, P, P, i64, P, P], i32),
            "links_simulate_packed": ([P, P, i32, i32, P, i64, P, P, P, P, P, P, i64, P], i32),
            "links_normalize": ([P, i64, i32, P, P], i32),
            "links_normalize_maxline": ([P, i64, i32, P, P, P, P], i32),
            "links_chamfer_topk": ([P, i32, i64, i32, P, P, i32, P, P], i32),
            "links_curate_paths": ([P, i64, i32, i32, P, P, i64, P, P, P, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_uint64, P, P, P, P, P, i64, P], i32),
            "links_topo_create": ([P, i32, i32, P, P, i32, P], i32),
            "links_topo_info": ([P, P, P, P], i32),
            "links_topo_source": ([i32, i32, P, P, P, ctypes.c_size_t, P], i32),
            "links_topo_free": ([P], i32),
            "links_simulate_topology": ([P, P, P, i32, i32, P, P, P, P, P, P, i64, P, P], i32),
            "links_chamfer_first_under": ([P, i32, i64, i32, P, P, i64, P, ctypes.c_double, i32, P, P], i32),
            "links_workspace_reserve": ([P, ctypes.c_size_t], i32),
            "links_serve_start": ([P, ctypes.c_size_t, i32, i32, i32, i32], i32),
            "links_serve_submit": ([P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)], i32),
            "links_serve_poll": ([P, ctypes.c_uint64, i32, ctypes.POINTER(Result)], i32),
            "links_serve_pause": ([P, i32], i32),
            "links_serve_stop": ([P], i32),
            "links_serve_inject_stall": ([P, i32], i32),
            "links_serve_stats": ([P, P], i32),
            "links_profile": ([P, i32], i32),
            "links_profile_read": ([P, i32, P, P, P, P], i32),
            "links_launch_count": ([P, P], i32),
            "links_compact_valid_static": ([P, i64, P, i64, P, P], i32),
            "links_autotune": ([P, P, i32, P], i32),
            "links_set_screen_lanes": ([P, i32, i32], i32),
            "links_set_tuning": ([P, i32, i32, i32], i32),
            "links_get_tuning": ([P, i32, i32, P], i32),
            "links_tuning_save": ([P, ctypes.c_char_p], i32),
            "links_tuning_load": ([P, ctypes.c_char_p], i32),
            "links_set_chamfer_prune": ([P, i32], i32),
            "links_capture_begin": ([P], i32),
            "links_capture_end": ([P, P], i32),
            "links_graph_launch": ([P, P], i32),
            "links_graph_free": ([P], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes, f.restype = args, res
        _lib = L
    return _lib


def strerror(status: int) -> str:
    return lib().links_strerror(int(status)).decode()


def links_last_error() -> str:
    return lib().links_last_error().decode()


def _check(status: int, what: str):
    if status != OK:
        raise LinksError(status, what, links_last_error())


def _dev(t, dtype=None, name="tensor"):
    """Device pointer of a contiguous CUDA tensor (or None)."""
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _host(a, dtype=None, name="array"):
    """Host pointer of a C-contiguous numpy array (or None)."""
    import numpy as np
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.flags.c_contiguous):
        raise ValueError(f"{name} must be a C-contiguous numpy array")
    if dtype is not None and a.dtype != dtype:
        raise ValueError(f"{name} must be {np.dtype(dtype)}, got {a.dtype}")
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ----------------------------------------------------------------------- C-ABI calls

def links_create(device: int = 0, stream=None):
    out = ctypes.c_void_p()
    _check(lib().links_create(ctypes.byref(out), int(device), _stream_handle(stream)), "links_create")
    return out


def links_destroy(ctx):
    _check(lib().links_destroy(ctx), "links_destroy")


def links_set_stream(ctx, stream):
    _check(lib().links_set_stream(ctx, _stream_handle(stream)), "links_set_stream")


def links_sync(ctx):
    _check(lib().links_sync(ctx), "links_sync")


def links_prepare(ctx, T: int):
    _check(lib().links_prepare(ctx, int(T)), "links_prepare")


def links_plan_create(ctx, capacity: int, n_max: int):
    out = ctypes.c_void_p()
    _check(lib().links_plan_create(ctx, int(capacity), int(n_max), ctypes.byref(out)), "links_plan_create")
    return out


def links_plan_free(plan):
    _check(lib().links_plan_free(plan), "links_plan_free")


def _pos_dtype(t):
    import torch
    import numpy as np
    if t.dtype in (torch.float32, np.float32):
        return F32
    if t.dtype in (torch.float64, np.float64):
        return F64
    raise ValueError("pos0 must be float32 or float64")


def links_plan_build(ctx, plan, n_joints, adj, jtype, pos0, status_out=None):
    """Device build: torch CUDA tensors int32 [B], uint8 [B,n,n], int8 [B,n], float32|64 [B,n,2]."""
    import torch
    B = n_joints.shape[0]
    _check(lib().links_plan_build(ctx, plan, int(B), _dev(n_joints, torch.int32, "n_joints"),
                                  _dev(adj, torch.uint8, "adj"), _dev(jtype, torch.int8, "type"),
                                  _dev(pos0, None, "pos0"), _pos_dtype(pos0),
                                  _dev(status_out, torch.int32, "status_out")), "links_plan_build")


def links_plan_build_masks(ctx, plan, n_joints, nbr, jtype, pos0, status_out=None):
    """Device build from neighbour bit masks: nbr int32 [B, n] (bit c of row a: joints a
    and c linked; the uint32 words viewed as int32), the rest as links_plan_build."""
    import torch
    B = n_joints.shape[0]
    _check(lib().links_plan_build_masks(ctx, plan, int(B), _dev(n_joints, torch.int32, "n_joints"),
                                        _dev(nbr, torch.int32, "nbr"), _dev(jtype, torch.int8, "type"),
                                        _dev(pos0, None, "pos0"), _pos_dtype(pos0),
                                        _dev(status_out, torch.int32, "status_out")), "links_plan_build_masks")


def links_plan_build_host(ctx, plan, n_joints, adj, jtype, pos0, status_out=None):
    """Host build: numpy arrays with the dtypes of links_plan_build."""
    import numpy as np
    B = n_joints.shape[0]
    _check(lib().links_plan_build_host(ctx, plan, int(B), _host(n_joints, np.int32, "n_joints"),
                                       _host(adj, np.uint8, "adj"), _host(jtype, np.int8, "type"),
                                       _host(pos0, None, "pos0"), _pos_dtype(pos0),
                                       _host(status_out, np.int32, "status_out")), "links_plan_build_host")


def links_plan_info(plan):
    B, nm, cap = ctypes.c_int64(), ctypes.c_int(), ctypes.c_int64()
    _check(lib().links_plan_info(plan, ctypes.byref(B), ctypes.byref(nm), ctypes.byref(cap)), "links_plan_info")
    return B.value, nm.value, cap.value


def links_plan_export(plan, b0: int, count: int, with_lengths: bool = True):
    """-> (topo int32 [count, 6 + 3 (n_max-2)], lengths float64 [count, 2 (n_max-2)] or None)."""
    import numpy as np
    _, nm, _ = links_plan_info(plan)
    md = max(nm - 2, 0)
    topo = np.empty((count, 6 + 3 * md), np.int32)
    lengths = np.empty((count, 2 * md), np.float64) if with_lengths else None
    _check(lib().links_plan_export(plan, int(b0), int(count), _host(topo), _host(lengths)), "links_plan_export")
    return topo, lengths


def links_simulate(ctx, plan, T: int, precision: int, out_mode: int, traj, path, valid, lock_step, min_disc,
                   out_index=None, out_capacity: int = 0, n_out=None):
    import torch
    fdt = torch.float64 if precision == PLAIN_F64 else torch.float32
    _check(lib().links_simulate(ctx, plan, int(T), int(precision), int(out_mode), _dev(traj, fdt, "traj"),
                                _dev(path, fdt, "path"), _dev(valid, torch.uint8, "valid"),
                                _dev(lock_step, torch.int16, "lock_step"), _dev(min_disc, torch.float32, "min_disc"),
                                _dev(out_index, torch.int32, "out_index"), int(out_capacity),
                                _dev(n_out, torch.int32, "n_out")), "links_simulate")


def links_simulate_packed(ctx, plan, T: int, precision: int, traj, traj_capacity: int, path, valid, lock_step,
                          min_disc, out_index, row_offset, out_capacity: int, n_out=None):
    import torch
    fdt = torch.float64 if precision == PLAIN_F64 else torch.float32
    _check(lib().links_simulate_packed(ctx, plan, int(T), int(precision), _dev(traj, fdt, "traj"), int(traj_capacity),
                                       _dev(path, fdt, "path"), _dev(valid, torch.uint8, "valid"),
                                       _dev(lock_step, torch.int16, "lock_step"),
                                       _dev(min_disc, torch.float32, "min_disc"),
                                       _dev(out_index, torch.int32, "out_index"),
                                       _dev(row_offset, torch.int64, "row_offset"), int(out_capacity),
                                       _dev(n_out, torch.int32, "n_out")), "links_simulate_packed")


def links_topo_create(ctx, n: int, adj, jtype, lanes: int = 0):
    """Compile the screen specialised to one topology: adj [n_max, n_max] uint8 and jtype [n_max]
    int8 of one mechanism with n joints (numpy, host).  Returns the handle."""
    import numpy as np
    a = np.ascontiguousarray(adj, dtype=np.uint8)
    t = np.ascontiguousarray(jtype, dtype=np.int8)
    h = ctypes.c_void_p()
    _check(lib().links_topo_create(ctx, int(n), int(a.shape[0]), a.ctypes.data_as(ctypes.c_void_p),
                                   t.ctypes.data_as(ctypes.c_void_p), int(lanes), ctypes.byref(h)),
           "links_topo_create")
    return h


def links_topo_source(n: int, adj, jtype) -> str:
    """The CUDA source links_topo_create compiles for this topology (host only)."""
    import numpy as np
    a = np.ascontiguousarray(adj, dtype=np.uint8)
    t = np.ascontiguousarray(jtype, dtype=np.int8)
    need = ctypes.c_size_t()
    args = (int(n), int(a.shape[0]), a.ctypes.data_as(ctypes.c_void_p), t.ctypes.data_as(ctypes.c_void_p))
    _check(lib().links_topo_source(*args, None, 0, ctypes.byref(need)), "links_topo_source")
    buf = ctypes.create_string_buffer(need.value)
    _check(lib().links_topo_source(*args, buf, need.value, None), "links_topo_source")
    return buf.value.decode()


def links_topo_info(topo) -> dict:
    nf, nd, ms = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().links_topo_info(topo, ctypes.byref(nf), ctypes.byref(nd), ctypes.byref(ms)), "links_topo_info")
    return {"fixed": nf.value, "dyads": nd.value, "compile_ms": ms.value}


def links_topo_free(topo):
    _check(lib().links_topo_free(topo), "links_topo_free")


def links_simulate_topology(ctx, plan, topo, T: int, out_mode: int, traj, path, valid, lock_step, min_disc,
                            out_index=None, out_capacity: int = 0, n_out=None, n_escaped=None):
    import torch
    _check(lib().links_simulate_topology(ctx, plan, topo, int(T), int(out_mode), _dev(traj, torch.float32, "traj"),
                                         _dev(path, torch.float32, "path"), _dev(valid, torch.uint8, "valid"),
                                         _dev(lock_step, torch.int16, "lock_step"),
                                         _dev(min_disc, torch.float32, "min_disc"),
                                         _dev(out_index, torch.int32, "out_index"), int(out_capacity),
                                         _dev(n_out, torch.int32, "n_out"), _dev(n_escaped, torch.int32, "n_escaped")),
           "links_simulate_topology")


def links_simulate_two_stage(ctx, plan, T: int, T_low: int, traj, path, valid, lock_step, min_disc,
                             out_index=None, out_capacity: int = 0, n_out=None, n_low_valid=None):
    import torch
    _check(lib().links_simulate_two_stage(ctx, plan, int(T), int(T_low), _dev(traj, torch.float32, "traj"),
                                          _dev(path, torch.float32, "path"), _dev(valid, torch.uint8, "valid"),
                                          _dev(lock_step, torch.int16, "lock_step"),
                                          _dev(min_disc, torch.float32, "min_disc"),
                                          _dev(out_index, torch.int32, "out_index"), int(out_capacity),
                                          _dev(n_out, torch.int32, "n_out"), _dev(n_low_valid, torch.int32, "n_low_valid")),
           "links_simulate_two_stage")


def links_emit_census(ctx, plan, T: int, out_mode: int, lock_step=None, out_index=None, out_capacity: int = 0):
    """-> dict(steps, double_word_steps, double_word_dyads): what the mixed emit does for
    the rows links_simulate wrote (FULL: from lock_step; VALID_ONLY: out_index rows)."""
    import torch
    out = (ctypes.c_int64 * 3)()
    _check(lib().links_emit_census(ctx, plan, int(T), int(out_mode), _dev(lock_step, torch.int16, "lock_step"),
                                   _dev(out_index, torch.int32, "out_index"), int(out_capacity), out),
           "links_emit_census")
    return dict(zip(("steps", "double_word_steps", "double_word_dyads"), (int(v) for v in out)))


def links_normalize(ctx, curves, out):
    """curves, out: float32 CUDA tensors [M, T, 2] (may be the same tensor)."""
    import torch
    M, T = curves.shape[0], curves.shape[1]
    _check(lib().links_normalize(ctx, int(M), int(T), _dev(curves, torch.float32, "curves"),
                                 _dev(out, torch.float32, "out")), "links_normalize")


def links_normalize_maxline(ctx, curves, out, pair=None, circ_var=None):
    """curves, out: float32 CUDA tensors [M, T, 2]; pair int32 [M, 2] and circ_var float32 [M] optional."""
    import torch
    M, T = curves.shape[0], curves.shape[1]
    _check(lib().links_normalize_maxline(ctx, int(M), int(T), _dev(curves, torch.float32, "curves"),
                                         _dev(out, torch.float32, "out"), _dev(pair, torch.int32, "pair"),
                                         _dev(circ_var, torch.float32, "circ_var")), "links_normalize_maxline")


def links_chamfer_topk(ctx, queries, db, k: int, idx, dist):
    """queries [Q,T,2], db [M,T,2] float32; idx [Q,k] int32 and dist [Q,k] float32 outputs (CUDA)."""
    import torch
    Q, T = queries.shape[0], queries.shape[1]
    M = db.shape[0]
    _check(lib().links_chamfer_topk(ctx, int(Q), int(M), int(T), _dev(queries, torch.float32, "queries"),
                                    _dev(db, torch.float32, "db"), int(k), _dev(idx, torch.int32, "idx"),
                                    _dev(dist, torch.float32, "dist")), "links_chamfer_topk")


def links_chamfer_first_under(ctx, queries, db, order, threshold: float, k: int, idx, dist):
    """queries [Q,T,2], db [M,T,2] float32, order [L] int32 scan order; idx [Q,k] int32 and
    dist [Q,k] float32 outputs: the first k curves of the scan with CD < threshold (CUDA)."""
    import torch
    Q, T = queries.shape[0], queries.shape[1]
    _check(lib().links_chamfer_first_under(ctx, int(Q), int(db.shape[0]), int(T),
                                           _dev(queries, torch.float32, "queries"), _dev(db, torch.float32, "db"),
                                           int(order.shape[0]), _dev(order, torch.int32, "order"),
                                           float(threshold), int(k), _dev(idx, torch.int32, "idx"),
                                           _dev(dist, torch.float32, "dist")), "links_chamfer_first_under")


def links_curate_paths(ctx, traj, row_index, n_joints, adj, jtype, flags, n_kept, *, circle_var: float = 5e-4,
                       keep_rate: float = 0.005, seed: int = 0, circ_var=None, pair=None, kept_index=None,
                       kept_paths=None):
    """traj [R, n_max, T, 2] float32, row_index [R] int32 (or None), n_joints [B] int32, adj
    [B, n_max, n_max] uint8, jtype [B, n_max] int8; outputs flags [R, n_max] uint8, n_kept [1]
    int32, optional circ_var [R, n_max] float32, pair [R, n_max, 2] int32, kept_index [cap]
    int32 and kept_paths [cap, T, 2] float32 (all CUDA)."""
    import torch
    R, n_max, T = traj.shape[0], traj.shape[1], traj.shape[2]
    cap = 0 if kept_index is None else int(kept_index.shape[0])
    if kept_paths is not None and kept_paths.shape[0] < cap:
        raise ValueError("kept_paths holds fewer rows than kept_index")
    _check(lib().links_curate_paths(ctx, int(R), int(n_max), int(T), _dev(traj, torch.float32, "traj"),
                                    _dev(row_index, torch.int32, "row_index"), int(n_joints.shape[0]),
                                    _dev(n_joints, torch.int32, "n_joints"), _dev(adj, torch.uint8, "adj"),
                                    _dev(jtype, torch.int8, "jtype"), float(circle_var), float(keep_rate),
                                    int(seed) & 0xFFFFFFFFFFFFFFFF, _dev(flags, torch.uint8, "flags"),
                                    _dev(circ_var, torch.float32, "circ_var"), _dev(pair, torch.int32, "pair"),
                                    _dev(kept_index, torch.int32, "kept_index"),
                                    _dev(kept_paths, torch.float32, "kept_paths"), cap,
                                    _dev(n_kept, torch.int32, "n_kept")), "links_curate_paths")


def links_workspace_reserve(ctx, nbytes: int):
    _check(lib().links_workspace_reserve(ctx, int(nbytes)), "links_workspace_reserve")


def links_serve_start(ctx, mem_budget_bytes: int, max_pending: int, n_max: int, T: int, with_traj: bool = False):
    _check(lib().links_serve_start(ctx, int(mem_budget_bytes), int(max_pending), int(n_max), int(T),
                                   1 if with_traj else 0), "links_serve_start")


def links_serve_submit(ctx, req: Request) -> int:
    """Returns the ticket; raises LinksError (status EBUSY / ECAPACITY / EINVAL) on refusal."""
    t = ctypes.c_uint64()
    _check(lib().links_serve_submit(ctx, ctypes.byref(req), ctypes.byref(t)), "links_serve_submit")
    return t.value


def links_serve_poll(ctx, ticket: int, timeout_us: int):
    """-> Result, or None if the ticket did not finish within timeout_us."""
    res = Result()
    st = lib().links_serve_poll(ctx, ctypes.c_uint64(ticket), int(timeout_us), ctypes.byref(res))
    if st == ETIMEDOUT:
        return None
    _check(st, "links_serve_poll")
    return res


def links_serve_pause(ctx, paused: bool):
    _check(lib().links_serve_pause(ctx, 1 if paused else 0), "links_serve_pause")


def links_serve_inject_stall(ctx, wait_ms: int):
    _check(lib().links_serve_inject_stall(ctx, int(wait_ms)), "links_serve_inject_stall")


def links_serve_stats(ctx) -> dict:
    out = (ctypes.c_int64 * 6)()
    _check(lib().links_serve_stats(ctx, out), "links_serve_stats")
    return dict(zip(("passes", "kernel_launches", "blocks", "capacity", "last_error_word", "passes_done"),
                    (int(v) for v in out)))


def links_serve_stop(ctx):
    _check(lib().links_serve_stop(ctx), "links_serve_stop")


def make_request(n_joints, adj, jtype, pos0, valid, lock_step, min_disc=None, valid_index=None, paths=None,
                 traj=None) -> Request:
    """A Request over numpy host arrays (kept alive by the caller until completion)."""
    import numpy as np
    cap = 0 if valid_index is None else valid_index.shape[0]
    return Request(int(n_joints.shape[0]), _host(n_joints, np.int32), _host(adj, np.uint8), _host(jtype, np.int8),
                   _host(pos0, np.float32), _host(valid, np.uint8), _host(lock_step, np.int16),
                   _host(min_disc, np.float32), cap, _host(valid_index, np.int32), _host(paths, np.float32),
                   _host(traj, np.float32))


def links_profile(ctx, enable: bool):
    _check(lib().links_profile(ctx, 1 if enable else 0), "links_profile")


def links_profile_read(ctx, max_entries: int = 64):
    """-> {kernel name: (total milliseconds, launches)}."""
    import numpy as np
    names = ctypes.create_string_buffer(32 * max_entries)
    ms = np.zeros(max_entries, np.float64)
    nl = np.zeros(max_entries, np.int64)
    cnt = ctypes.c_int()
    _check(lib().links_profile_read(ctx, max_entries, names, _host(ms), _host(nl), ctypes.byref(cnt)),
           "links_profile_read")
    raw = names.raw
    return {raw[32 * i: 32 * i + 32].split(b"\0")[0].decode(): (float(ms[i]), int(nl[i])) for i in range(cnt.value)}


def links_launch_count(ctx) -> int:
    out = ctypes.c_int64()
    _check(lib().links_launch_count(ctx, ctypes.byref(out)), "links_launch_count")
    return out.value


def links_compact_valid_static(valid, out_index, n_out, stream=None):
    """Allocation-free valid-row compaction on the current device (see include/links.h)."""
    import torch
    cap = 0 if out_index is None else out_index.shape[0]
    _check(lib().links_compact_valid_static(_dev(valid, torch.uint8, "valid"), int(valid.shape[0]),
                                            _dev(out_index, torch.int32, "out_index"), int(cap),
                                            _dev(n_out, torch.int32, "n_out"), _stream_handle(stream)),
           "links_compact_valid_static")


def links_autotune(ctx, plan, T: int) -> int:
    """Tunes the screen's lanes per mechanism on the built plan; returns the choice."""
    lanes = ctypes.c_int()
    _check(lib().links_autotune(ctx, plan, int(T), ctypes.byref(lanes)), "links_autotune")
    return lanes.value


def links_set_chamfer_prune(ctx, on: bool):
    _check(lib().links_set_chamfer_prune(ctx, 1 if on else 0), "links_set_chamfer_prune")


(TUNE_BUILDER, TUNE_SCREEN_LANES, TUNE_SCREEN_STEPS, TUNE_SCREEN_CTAS, TUNE_EMIT_DWS, TUNE_EMIT_CTAS,
 TUNE_SCREEN_DEFER) = range(7)
TUNE_KEYS = {"builder": TUNE_BUILDER, "screen_lanes": TUNE_SCREEN_LANES, "screen_steps": TUNE_SCREEN_STEPS,
             "screen_ctas": TUNE_SCREEN_CTAS, "emit_dws": TUNE_EMIT_DWS, "emit_ctas": TUNE_EMIT_CTAS,
             "screen_defer": TUNE_SCREEN_DEFER}


def links_set_tuning(ctx, n_max: int, key: int, value: int):
    _check(lib().links_set_tuning(ctx, int(n_max), int(key), int(value)), "links_set_tuning")


def links_get_tuning(ctx, n_max: int, key: int) -> int:
    v = ctypes.c_int()
    _check(lib().links_get_tuning(ctx, int(n_max), int(key), ctypes.byref(v)), "links_get_tuning")
    return v.value


def tuning_table(ctx, n_max: int) -> dict:
    """The context's kernel shapes for plans of n_max joints, by key name."""
    return {name: links_get_tuning(ctx, n_max, k) for name, k in TUNE_KEYS.items()}


def links_tuning_save(ctx, path: str):
    _check(lib().links_tuning_save(ctx, os.fsencode(path)), "links_tuning_save")


def links_tuning_load(ctx, path: str):
    _check(lib().links_tuning_load(ctx, os.fsencode(path)), "links_tuning_load")


def links_set_screen_lanes(ctx, n_max: int, lanes: int):
    _check(lib().links_set_screen_lanes(ctx, int(n_max), int(lanes)), "links_set_screen_lanes")


def links_capture_begin(ctx):
    _check(lib().links_capture_begin(ctx), "links_capture_begin")


def links_capture_end(ctx):
    out = ctypes.c_void_p()
    _check(lib().links_capture_end(ctx, ctypes.byref(out)), "links_capture_end")
    return out


def links_graph_launch(ctx, graph):
    _check(lib().links_graph_launch(ctx, graph), "links_graph_launch")


def links_graph_free(graph):
    _check(lib().links_graph_free(graph), "links_graph_free")
