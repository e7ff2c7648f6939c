"""Thin Python binding of libdagrt's C ABI (include/dagrt.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels. The raw entry points keep their C names (`dagrt_create`, `dagrt_load_csr`,
`dagrt_schedule`, `dagrt_bound`, ...); `Context` and `LoadedBatch` wrap them for numpy
(host) arrays and torch CUDA tensors (device pointers, used in place).

Importing this module loads `libdagrt.so` built in-tree by `build.py`; it raises
ImportError when the library is missing. There is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libdagrt.so is not built ({_LIB_PATH}); run "
                      "`python -c 'import __graft_entry__ as g; g.build()'` first")
lib = C.CDLL(_LIB_PATH)

OK, E_INVAL, E_CYCLE, E_RANGE, E_OOM, E_DEVICE, E_TIMEOUT, E_CAP, E_INTERNAL = 0, -1, -2, -3, -4, -5, -6, -7, -8
PTR_DEVICE = 1
VAR_PAPER, VAR_NOPARA, VAR_NOSEG, VAR_LITERAL, VAR_NOREPAIR = 0, 1, 2, 3, 4
MAX_M, MAX_V = 4096, 65535

_vp = C.c_void_p


class dagrt_schedule_out(C.Structure):
    _fields_ = [(n, _vp) for n in (
        "bound", "status", "n_groups", "n_seg", "n_rows", "n_extra", "level", "wanc", "block_of",
        "group_of", "exec_group", "m", "group_R", "seg_parent", "seg_load", "seg_m", "seg_group",
        "row_id", "row_group", "row_m0", "row_load", "extra_off", "extra_src", "extra_dst",
        "greedy", "greedy_unaware", "graham_para", "crit_path")]


def _sig(name, res, args):
    f = getattr(lib, name)
    f.restype = res
    f.argtypes = args
    return f


dagrt_create = _sig("dagrt_create", C.c_int, [C.POINTER(_vp), C.c_int, _vp])
dagrt_set_stream = _sig("dagrt_set_stream", C.c_int, [_vp, _vp])
dagrt_sync = _sig("dagrt_sync", C.c_int, [_vp])
dagrt_destroy = _sig("dagrt_destroy", None, [_vp])
dagrt_last_error = _sig("dagrt_last_error", C.c_char_p, [_vp])
dagrt_launch_count = _sig("dagrt_launch_count", C.c_int64, [_vp])
dagrt_load_csr = _sig("dagrt_load_csr", C.c_int,
                      [_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int32, C.c_uint32, C.POINTER(_vp)])
dagrt_batch_free = _sig("dagrt_batch_free", None, [_vp])
dagrt_batch_n_dags = _sig("dagrt_batch_n_dags", C.c_int32, [_vp])
dagrt_batch_total_nodes = _sig("dagrt_batch_total_nodes", C.c_int64, [_vp])
dagrt_schedule = _sig("dagrt_schedule", C.c_int, [_vp, C.c_int32, C.POINTER(dagrt_schedule_out), C.c_uint32])
dagrt_schedulable = _sig("dagrt_schedulable", C.c_int, [_vp, C.c_int32, _vp, _vp, C.POINTER(C.c_int64), C.c_uint32])
dagrt_bound = _sig("dagrt_bound", C.c_int,
                   [_vp, C.c_int32, C.POINTER(C.c_int32), C.c_int32, _vp, C.c_int64, _vp, _vp, _vp, C.c_uint32])
SEARCH_RANDOM, SEARCH_EXHAUSTIVE, SEARCH_PERTURB = 0, 1, 2


class dagrt_search_cfg(C.Structure):
    _fields_ = [("n_variants", C.c_int32), ("variant_ids", C.POINTER(C.c_int32)), ("n_alloc", C.c_int32),
                ("n_levels", C.c_int32), ("levels", C.POINTER(C.c_uint8)), ("seed", C.c_uint64),
                ("mode", C.c_int32)]


dagrt_search = _sig("dagrt_search", C.c_int, [_vp, C.POINTER(dagrt_search_cfg), _vp, _vp, _vp, _vp, C.c_uint32])
dagrt_schedule_noalloc = _sig("dagrt_schedule_noalloc", C.c_int,
                              [C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int64, C.c_int64, C.c_int32,
                               C.c_int32, _vp, _vp, _vp])

dagrt_cond_bound = _sig("dagrt_cond_bound", C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_int32,
                                                      C.c_int32, C.c_int32, _vp, _vp, _vp, _vp])
REALISE_BARRIER, REALISE_EDGES, REALISE_GREEDY = 0, 1, 2
dagrt_realise = _sig("dagrt_realise", C.c_int, [_vp, C.c_int32, _vp, _vp, _vp, _vp, C.c_int32, C.c_int32, C.c_int32,
                                                C.c_float, C.c_int32, _vp, C.POINTER(C.c_int64)])
dagrt_model_n_params = _sig("dagrt_model_n_params", C.c_int64, [])
dagrt_model_create = _sig("dagrt_model_create", C.c_int, [_vp, C.c_int32, _vp, C.c_uint64, C.POINTER(_vp)])
dagrt_model_free = _sig("dagrt_model_free", None, [_vp])
dagrt_model_params = _sig("dagrt_model_params", C.c_int, [_vp, _vp, _vp])
dagrt_model_state = _sig("dagrt_model_state", C.c_int, [_vp, _vp, C.POINTER(C.c_int32), _vp, C.c_int32])
dagrt_selftest_wait = _sig("dagrt_selftest_wait", C.c_int, [_vp, C.c_uint32])
dagrt_model_logits = _sig("dagrt_model_logits", C.c_int, [_vp, _vp, _vp, C.c_uint32])
dagrt_model_grad = _sig("dagrt_model_grad", C.c_int, [_vp, _vp, _vp, _vp, _vp])
dagrt_train_step = _sig("dagrt_train_step", C.c_int, [_vp, _vp, _vp, C.c_float, _vp])
dagrt_propose = _sig("dagrt_propose", C.c_int, [_vp, _vp, C.c_int32, _vp, _vp, _vp, _vp, _vp, C.c_uint32])


class dagrt_tuning(C.Structure):
    _fields_ = [("warp_max_v", C.c_int32), ("chunk_rows", C.c_int32), ("item_warps", C.c_int32),
                ("cta_smem", C.c_int32)]


dagrt_get_tuning = _sig("dagrt_get_tuning", C.c_int, [_vp, C.POINTER(dagrt_tuning)])
dagrt_set_tuning = _sig("dagrt_set_tuning", C.c_int, [_vp, C.POINTER(dagrt_tuning)])
dagrt_autotune_schedule = _sig("dagrt_autotune_schedule", C.c_int,
                               [_vp, C.c_int32, C.c_int32, C.POINTER(dagrt_tuning), C.POINTER(C.c_float)])
dagrt_autotune_bound = _sig("dagrt_autotune_bound", C.c_int,
                            [_vp, C.c_int32, C.POINTER(C.c_int32), C.c_int32, _vp, C.c_int64, C.c_int32,
                             C.POINTER(dagrt_tuning), C.POINTER(C.c_float)])
dagrt_graph_begin = _sig("dagrt_graph_begin", C.c_int, [_vp])
dagrt_graph_end = _sig("dagrt_graph_end", C.c_int, [_vp, C.POINTER(_vp)])
dagrt_graph_launch = _sig("dagrt_graph_launch", C.c_int, [_vp])
dagrt_graph_free = _sig("dagrt_graph_free", None, [_vp])


def _tdict(t):
    return {"warp_max_v": t.warp_max_v, "chunk_rows": t.chunk_rows, "item_warps": t.item_warps,
            "cta_smem": t.cta_smem}


class DagrtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dagrt error {code}: {msg}")
        self.code = code


def _ptr(x):
    """Address of a numpy array or a torch tensor (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"]
        return x.ctypes.data
    return x.data_ptr()  # torch tensor


def _is_device(x):
    return x is not None and not isinstance(x, np.ndarray) and getattr(x, "is_cuda", False)


# per-node / per-DAG output fields and their dtypes
_DAG_FIELDS = {"bound": np.int64, "status": np.int32, "n_groups": np.int32, "n_seg": np.int32,
               "n_rows": np.int32, "n_extra": np.int64, "greedy": np.int64, "greedy_unaware": np.int64,
               "graham_para": np.int64, "crit_path": np.int64}
_NODE_FIELDS = {"level": np.int32, "wanc": np.int64, "block_of": np.int32, "group_of": np.int32,
                "exec_group": np.int32, "m": np.int32, "group_R": np.int64, "seg_parent": np.int32,
                "seg_load": np.int64, "seg_m": np.int32, "seg_group": np.int32}
_ROW_FIELDS = {"row_id": np.int32, "row_group": np.int32, "row_m0": np.int32, "row_load": np.int64}
ALL_FIELDS = tuple(_DAG_FIELDS) + tuple(_NODE_FIELDS) + tuple(_ROW_FIELDS)


class Context:
    def __init__(self, device: int = 0, stream=None):
        h = _vp()
        rc = dagrt_create(C.byref(h), int(device), stream)
        if rc != OK:
            raise DagrtError(rc, "dagrt_create failed (no usable CUDA device?)")
        self.h = h
        self.device = device

    def check(self, rc):
        if rc != OK:
            raise DagrtError(rc, dagrt_last_error(self.h).decode())
        return rc

    def set_stream(self, stream):
        self.check(dagrt_set_stream(self.h, stream))

    def last_error(self) -> str:
        return dagrt_last_error(self.h).decode()

    def sync(self):
        self.check(dagrt_sync(self.h))

    def launches(self) -> int:
        return int(dagrt_launch_count(self.h))

    def close(self):
        if self.h:
            dagrt_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cond_bound(self, batch, cond, variant: int = VAR_PAPER, max_real: int = 4096, M: int | None = None):
        """dagrt_cond_bound on a workloads.Batch (host arrays) with per-node conditional
        flags: dict of adaptive, fixed, worst_real, n_real (numpy, one entry per DAG)."""
        a = {k: np.ascontiguousarray(getattr(batch, k)) for k in ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")}
        cd = np.ascontiguousarray(cond, np.uint8)
        n = batch.n_dags
        out = {"adaptive": np.zeros(max(n, 1), np.int64), "fixed": np.zeros(max(n, 1), np.int64),
               "worst_real": np.zeros(max(n, 1), np.int32), "n_real": np.zeros(max(n, 1), np.int32)}
        self.check(dagrt_cond_bound(self.h, n, _ptr(a["node_off"]), _ptr(a["edge_off"]), _ptr(a["row_ptr"]),
                                    _ptr(a["col"]) if len(a["col"]) else None, _ptr(a["wcet"]), _ptr(a["k64"]),
                                    _ptr(cd), int(batch.M if M is None else M), int(variant), int(max_real),
                                    _ptr(out["adaptive"]), _ptr(out["fixed"]), _ptr(out["worst_real"]),
                                    _ptr(out["n_real"])))
        return {k: v[:n] for k, v in out.items()}

    def realise(self, row_ptr, col, wcet, k64, M: int, mode: int = REALISE_BARRIER, variant: int = VAR_PAPER,
                tick_us: float = 20.0, reps: int = 10):
        """dagrt_realise on one DAG (host arrays): (makespans in us [reps], bound in ticks)."""
        rp = np.ascontiguousarray(row_ptr, np.int32)
        cl = np.ascontiguousarray(col, np.int32)
        w = np.ascontiguousarray(wcet, np.int64)
        k = np.ascontiguousarray(k64, np.uint8)
        out = np.zeros(reps, np.float32)
        bnd = C.c_int64(0)
        self.check(dagrt_realise(self.h, len(w), _ptr(rp), _ptr(cl) if len(cl) else None, _ptr(w), _ptr(k), int(M),
                                 int(variant), int(mode), C.c_float(tick_us), int(reps), _ptr(out), C.byref(bnd)))
        return out, int(bnd.value)

    def graph_begin(self):
        self.check(dagrt_graph_begin(self.h))

    def graph_end(self) -> "Graph":
        g = _vp()
        self.check(dagrt_graph_end(self.h, C.byref(g)))
        return Graph(self, g)

    def load(self, arrays, M: int | None = None) -> "LoadedBatch":
        """Load a batch: a workloads.Batch (host numpy arrays, copied) or a dict of torch
        CUDA tensors with keys node_off, edge_off, row_ptr, col, wcet, k64 (used in place)."""
        if isinstance(arrays, dict):
            a = arrays
            if M is None:
                M = int(a["M"])
            flags = PTR_DEVICE if _is_device(a["wcet"]) else 0
            n = int(a["node_off"].shape[0]) - 1
        else:
            a = {k: np.ascontiguousarray(getattr(arrays, k)) for k in
                 ("node_off", "edge_off", "row_ptr", "col", "wcet", "k64")}
            M = arrays.M if M is None else M
            flags = 0
            n = arrays.n_dags
        h = _vp()
        rc = dagrt_load_csr(self.h, n, _ptr(a["node_off"]), _ptr(a["edge_off"]), _ptr(a["row_ptr"]),
                            _ptr(a["col"]), _ptr(a["wcet"]), _ptr(a["k64"]), int(M), flags, C.byref(h))
        self.check(rc)
        return LoadedBatch(self, h, n, M, keep=a)


class Graph:
    """A recorded sequence of device-side library calls (dagrt_graph_*)."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h

    def launch(self):
        self.ctx.check(dagrt_graph_launch(self.h))

    def free(self):
        if self.h:
            dagrt_graph_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class LoadedBatch:
    def __init__(self, ctx: Context, h, n_dags: int, M: int, keep=None):
        self.ctx, self.h, self.n_dags, self.M = ctx, h, n_dags, M
        self._keep = keep  # device inputs must outlive the batch
        self.total_nodes = int(dagrt_batch_total_nodes(h))

    def free(self):
        if self.h:
            dagrt_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def tuning(self) -> dict:
        t = dagrt_tuning()
        self.ctx.check(dagrt_get_tuning(self.h, C.byref(t)))
        return _tdict(t)

    def set_tuning(self, **kw):
        cur = self.tuning()
        cur.update(kw)
        t = dagrt_tuning(int(cur["warp_max_v"]), int(cur["chunk_rows"]), int(cur["item_warps"]),
                         int(cur["cta_smem"]))
        self.ctx.check(dagrt_set_tuning(self.h, C.byref(t)))

    def autotune_schedule(self, variant: int = VAR_PAPER, reps: int = 3):
        t, ms = dagrt_tuning(), C.c_float(0)
        self.ctx.check(dagrt_autotune_schedule(self.h, int(variant), int(reps), C.byref(t), C.byref(ms)))
        return _tdict(t), ms.value

    def autotune_bound(self, variant_ids, n_alloc: int, m_alloc, cand_stride: int, reps: int = 3):
        """m_alloc: a torch CUDA tensor (device candidates)."""
        vids = (C.c_int32 * len(variant_ids))(*[int(v) for v in variant_ids])
        t, ms = dagrt_tuning(), C.c_float(0)
        self.ctx.check(dagrt_autotune_bound(self.h, len(variant_ids), vids, int(n_alloc), _ptr(m_alloc),
                                            int(cand_stride), int(reps), C.byref(t), C.byref(ms)))
        return _tdict(t), ms.value

    def schedule(self, variant: int = VAR_PAPER, fields=("bound", "status"), extra_cap=None,
                 out=None, check: bool = True):
        """Run the scheduler. With `out` (a dict of torch CUDA tensors) the call enqueues
        device work only and returns `out`; otherwise the requested fields come back as
        numpy arrays. extra_cap: per-DAG capacities of the extra-edge buffer (host)."""
        o = dagrt_schedule_out()
        if out is not None:
            for k, t in out.items():
                setattr(o, k, _ptr(t))
            rc = dagrt_schedule(self.h, int(variant), C.byref(o), PTR_DEVICE)
            if check:
                self.ctx.check(rc)
            return out
        res = {}
        nd, nn = self.n_dags, self.total_nodes
        for f in fields:
            if f in _DAG_FIELDS:
                res[f] = np.zeros(max(nd, 1), _DAG_FIELDS[f])
            elif f in _NODE_FIELDS:
                res[f] = np.zeros(max(nn, 1), _NODE_FIELDS[f])
            elif f in _ROW_FIELDS:
                res[f] = np.zeros(max(2 * nn, 1), _ROW_FIELDS[f])
            else:
                raise KeyError(f)
            setattr(o, f, _ptr(res[f]))
        if extra_cap is not None:
            cap = np.asarray(extra_cap, np.int64)
            eo = np.zeros(nd + 1, np.int64)
            eo[1:] = np.cumsum(cap)
            res["extra_off"] = eo
            res["extra_src"] = np.zeros(max(int(eo[-1]), 1), np.int32)
            res["extra_dst"] = np.zeros(max(int(eo[-1]), 1), np.int32)
            for f in ("extra_off", "extra_src", "extra_dst"):
                setattr(o, f, _ptr(res[f]))
        rc = dagrt_schedule(self.h, int(variant), C.byref(o), 0)
        res["rc"] = rc
        if check and rc not in (OK, E_INVAL, E_RANGE, E_CYCLE, E_CAP):
            self.ctx.check(rc)
        for f in list(res):
            if f in _DAG_FIELDS:
                res[f] = res[f][:nd]
        return res

    def schedulable(self, variant: int, deadline):
        """dagrt_schedulable with host arrays: (ok flags int32 [n_dags], number schedulable)."""
        dl = np.ascontiguousarray(deadline, np.int64)
        assert dl.shape == (self.n_dags,)
        ok = np.zeros(max(self.n_dags, 1), np.int32)
        n = C.c_int64(0)
        self.ctx.check(dagrt_schedulable(self.h, int(variant), _ptr(dl), _ptr(ok), C.byref(n), 0))
        return ok[:self.n_dags], int(n.value)

    def bound(self, variant_ids, n_alloc: int, m_alloc, cand_stride: int, out_bound=None,
              best_bound=None, best_cand=None, want_all: bool = True):
        """Bounds of candidate allocations (see dagrt_bound). Host numpy inputs return
        numpy outputs; torch CUDA inputs need torch CUDA outputs and only enqueue."""
        vids = (C.c_int32 * len(variant_ids))(*[int(v) for v in variant_ids])
        n_cand = len(variant_ids) * n_alloc
        if _is_device(m_alloc):
            rc = dagrt_bound(self.h, len(variant_ids), vids, int(n_alloc), _ptr(m_alloc), int(cand_stride),
                             _ptr(out_bound), _ptr(best_bound), _ptr(best_cand), PTR_DEVICE)
            self.ctx.check(rc)
            return out_bound, best_bound, best_cand
        m_alloc = np.ascontiguousarray(m_alloc, np.uint8)
        ob = np.zeros(max(self.n_dags * n_cand, 1), np.int64) if want_all else None
        bb = np.zeros(max(self.n_dags, 1), np.int64)
        bc = np.zeros(max(self.n_dags, 1), np.int32)
        rc = dagrt_bound(self.h, len(variant_ids), vids, int(n_alloc), _ptr(m_alloc), int(cand_stride),
                         _ptr(ob), _ptr(bb), _ptr(bc), 0)
        self.ctx.check(rc)
        return (ob[:self.n_dags * n_cand].reshape(self.n_dags, n_cand) if want_all else None,
                bb[:self.n_dags], bc[:self.n_dags])

    def search(self, variant_ids, n_alloc: int, levels, seed: int = 0, want_all: bool = False,
               want_m: bool = False, out=None, mode: int = SEARCH_RANDOM):
        """dagrt_search over generated candidates (mode: SEARCH_RANDOM, SEARCH_EXHAUSTIVE or
        SEARCH_PERTURB). Host outputs (numpy) by default; with `out` (dict of torch CUDA
        tensors: out_bound/best_bound/best_cand/best_m, any subset) the call only enqueues
        device work."""
        vids = (C.c_int32 * len(variant_ids))(*[int(v) for v in variant_ids])
        lev = (C.c_uint8 * len(levels))(*[int(x) for x in levels])
        cfg = dagrt_search_cfg(len(variant_ids), vids, int(n_alloc), len(levels), lev, C.c_uint64(seed & (2**64 - 1)),
                               int(mode))
        if out is not None:
            rc = dagrt_search(self.h, C.byref(cfg), _ptr(out.get("out_bound")), _ptr(out.get("best_bound")),
                              _ptr(out.get("best_cand")), _ptr(out.get("best_m")), PTR_DEVICE)
            self.ctx.check(rc)
            return out
        n_cand = len(variant_ids) * n_alloc
        ob = np.zeros(max(self.n_dags * n_cand, 1), np.int64) if want_all else None
        bb = np.zeros(max(self.n_dags, 1), np.int64)
        bc = np.zeros(max(self.n_dags, 1), np.int32)
        bm = np.zeros(max(2 * self.total_nodes, 1), np.uint8) if want_m else None
        rc = dagrt_search(self.h, C.byref(cfg), _ptr(ob), _ptr(bb), _ptr(bc), _ptr(bm), 0)
        self.ctx.check(rc)
        return {"out_bound": ob[:self.n_dags * n_cand].reshape(self.n_dags, n_cand) if want_all else None,
                "best_bound": bb[:self.n_dags], "best_cand": bc[:self.n_dags], "best_m": bm}


_BATCH_DTYPES = {"node_off": "int64", "edge_off": "int64", "row_ptr": "int32", "col": "int32",
                 "wcet": "int64", "k64": "uint8"}


def _check_device_array(name, t, dtype, min_len):
    """A contiguous torch CUDA tensor of `dtype` with at least min_len elements."""
    if t is None or not getattr(t, "is_cuda", False):
        raise ValueError(f"{name}: a torch CUDA tensor is required")
    if str(t.dtype) != f"torch.{dtype}":
        raise ValueError(f"{name}: dtype {t.dtype}, expected torch.{dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if t.numel() < min_len:
        raise ValueError(f"{name}: {t.numel()} elements, at least {min_len} needed")


def schedule_noalloc(dev: dict, M: int, variant: int, bound, status, stream=None) -> int:
    """dagrt_schedule_noalloc on a batch held in torch CUDA tensors (keys as for
    Context.load); bound (int64) and status (int32) are torch CUDA tensors of n_dags
    entries. The array lengths passed to the library are the tensors' own lengths, so the
    kernel rejects offsets that reach outside them. Enqueues only; returns the C status."""
    n = int(dev["node_off"].shape[0]) - 1
    for k, dt in _BATCH_DTYPES.items():
        _check_device_array(k, dev[k], dt, 0)
    _check_device_array("bound", bound, "int64", n)
    _check_device_array("status", status, "int32", n)
    tot_nodes = min(int(dev["wcet"].numel()), int(dev["k64"].numel()), int(dev["row_ptr"].numel()) - max(n, 0))
    tot_edges = int(dev["col"].numel())
    return int(dagrt_schedule_noalloc(n, _ptr(dev["node_off"]), _ptr(dev["edge_off"]), _ptr(dev["row_ptr"]),
                                      _ptr(dev["col"]) if tot_edges else None, _ptr(dev["wcet"]), _ptr(dev["k64"]),
                                      max(tot_nodes, 0), tot_edges, int(M), int(variant), _ptr(bound),
                                      _ptr(status), stream))


class Model:
    """Learned proposer (dagrt_model_*): per-kernel SM-level scores from a message-passing
    network; `propose` evaluates the paper's allocation and the k best assignments exactly."""

    def __init__(self, ctx: Context, levels, seed: int = 0):
        self.ctx = ctx
        self.levels = np.ascontiguousarray(levels, np.uint8)
        h = _vp()
        ctx.check(dagrt_model_create(ctx.h, len(self.levels), _ptr(self.levels),
                                     C.c_uint64(seed & (2**64 - 1)), C.byref(h)))
        self.h = h
        self.n_params = int(dagrt_model_n_params())

    def free(self):
        if getattr(self, "h", None):
            dagrt_model_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def params(self, set_to=None) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        st = None if set_to is None else np.ascontiguousarray(set_to, np.float32)
        self.ctx.check(dagrt_model_params(self.h, _ptr(out), _ptr(st)))
        return out

    def state(self):
        """(parameters, Adam m, Adam v) as one float32 array of 3 * n_params, and the step."""
        buf = np.zeros(3 * self.n_params, np.float32)
        step = C.c_int32(0)
        self.ctx.check(dagrt_model_state(self.h, _ptr(buf), C.byref(step), None, 0))
        return buf, int(step.value)

    def set_state(self, buf, step: int):
        buf = np.ascontiguousarray(buf, np.float32)
        assert buf.size == 3 * self.n_params
        self.ctx.check(dagrt_model_state(self.h, None, None, _ptr(buf), int(step)))

    def logits(self, batch: "LoadedBatch", out=None) -> np.ndarray:
        L = len(self.levels)
        if out is not None:  # torch CUDA tensor [total_nodes * L]
            self.ctx.check(dagrt_model_logits(batch.h, self.h, _ptr(out), PTR_DEVICE))
            return out
        z = np.zeros(max(batch.total_nodes * L, 1), np.float32)
        self.ctx.check(dagrt_model_logits(batch.h, self.h, _ptr(z), 0))
        return z[:batch.total_nodes * L].reshape(batch.total_nodes, L)

    def grad(self, batch: "LoadedBatch", labels):
        lab = np.ascontiguousarray(labels, np.int8)
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_float(0)
        self.ctx.check(dagrt_model_grad(batch.h, self.h, _ptr(lab), _ptr(g), C.byref(loss)))
        return float(loss.value), g

    def train_step(self, batch: "LoadedBatch", labels, lr: float) -> float:
        lab = np.ascontiguousarray(labels, np.int8)
        loss = C.c_float(0)
        self.ctx.check(dagrt_train_step(batch.h, self.h, _ptr(lab), C.c_float(lr), C.byref(loss)))
        return float(loss.value)

    def propose(self, batch: "LoadedBatch", k: int = 16, want_all: bool = False, want_m: bool = False, out=None):
        """dagrt_propose. Host outputs (numpy) by default; with `out` (dict of torch CUDA
        tensors: out_bound/cand_m/best_bound/best_cand/best_m, any subset) the call only
        enqueues device work."""
        if out is not None:
            self.ctx.check(dagrt_propose(batch.h, self.h, int(k), _ptr(out.get("out_bound")), _ptr(out.get("cand_m")),
                                         _ptr(out.get("best_bound")), _ptr(out.get("best_cand")),
                                         _ptr(out.get("best_m")), PTR_DEVICE))
            return out
        nd, nr, nc = batch.n_dags, 2 * batch.total_nodes, int(k) + 1
        ob = np.zeros(max(nd * nc, 1), np.int64) if want_all else None
        cm = np.zeros(max(nr * nc, 1), np.uint8) if want_all else None
        bb = np.zeros(max(nd, 1), np.int64)
        bc = np.zeros(max(nd, 1), np.int32)
        bm = np.zeros(max(nr, 1), np.uint8) if want_m else None
        self.ctx.check(dagrt_propose(batch.h, self.h, int(k), _ptr(ob), _ptr(cm), _ptr(bb), _ptr(bc), _ptr(bm), 0))
        return {"out_bound": ob[:nd * nc].reshape(nd, nc) if want_all else None,
                "cand_m": cm[:nr * nc].reshape(nr, nc) if want_all else None,
                "best_bound": bb[:nd], "best_cand": bc[:nd], "best_m": bm}
