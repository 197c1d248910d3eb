"""GB300-native JABBA symbolization (arXiv 2401.00109): Python binding.

Every step runs in the CUDA library `libjabba.so` (hand-written sm_103a
kernels behind the C ABI of include/jabba.h).  This module only marshals
torch tensors (device memory and the current stream) into those calls; it has
no compute path of its own and refuses to run without the library and a GPU.

    import paper_2401_00109_gb300 as jb
    ctx = jb.Context()
    out = ctx.symbolize(x, series_off, jb.Params(tol=0.1, alpha=0.1))
    out["symbol"], out["dict_len"], out["dict_inc"]
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import _build

__all__ = ["Params", "Context", "JabbaError", "load", "build", "JabbaMSE", "EQUAL_COUNT", "FIXED_LEN"]

EQUAL_COUNT = 0
FIXED_LEN = 1

STATUS = {
    0: "ok", 1: "invalid argument", 2: "capacity exceeded", 3: "non-finite input value", 4: "CUDA runtime error",
    5: "bounded device wait timed out", 6: "call out of order / allocation during graph capture",
    7: "input value out of range",
}
ERR_CAPACITY = 2


class JabbaError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {STATUS.get(code, 'unknown')} (status {code})")
        self.code = code


class _Params(C.Structure):
    _fields_ = [("tol", C.c_double), ("alpha", C.c_double), ("scl", C.c_double), ("domain_mode", C.c_int32),
                ("round_mode", C.c_int32), ("domain_value", C.c_int64), ("key_mode", C.c_int32),
                ("reserved", C.c_int32)]


@dataclass
class Params:
    """Method parameters (Eq. 1 tol; Sec. 3.2 alpha, scl; Sec. 4.1.1 domains;
    Sec. 3.3 rounding of the quantization; Sec. 5 sort key: 0 = norm,
    1 = PCA projection)."""
    tol: float = 0.1
    alpha: float = 0.1
    scl: float = 1.0
    domain_mode: int = EQUAL_COUNT
    domain_value: int = 4
    round_mode: int = 0
    key_mode: int = 0

    def c(self) -> _Params:
        return _Params(float(self.tol), float(self.alpha), float(self.scl), int(self.domain_mode),
                       int(self.round_mode), int(self.domain_value), int(self.key_mode), 0)


class _Tuning(C.Structure):
    _fields_ = [("compress_ctas_per_sm", C.c_int32), ("compress_pack", C.c_int32), ("local_mid_warps", C.c_int32),
                ("local_big_warps", C.c_int32), ("merge_ctas_per_sm", C.c_int32), ("per_domain_launch", C.c_int32),
                ("local_k_warps", C.c_int32), ("local_ctas_cap", C.c_int32), ("merge_form", C.c_int32),
                ("merge_warps", C.c_int32)]


TUNING_FIELDS = ("compress_ctas_per_sm", "compress_pack", "local_mid_warps", "local_big_warps", "merge_ctas_per_sm",
                 "per_domain_launch", "local_k_warps", "local_ctas_cap", "merge_form", "merge_warps")

JABBA_GROUP_BYTES = 48
PIECE_STATS_BYTES = 256

_lib = None
_lock = threading.Lock()
V = C.c_void_p
I64 = C.c_int64


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load():
    """Load libjabba.so (building it first if needed).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            sig = {
                "jabba_create": (C.c_int, [C.POINTER(V), C.c_int]),
                "jabba_destroy": (None, [V]),
                "jabba_status_string": (C.c_char_p, [C.c_int]),
                "jabba_version": (C.c_char_p, []),
                "jabba_sync_status": (C.c_int, [V, V]),
                "jabba_plan": (C.c_int, [V, I64, C.POINTER(_Params), C.POINTER(I64), C.POINTER(I64),
                                         C.POINTER(I64)]),
                "jabba_reserve": (C.c_int, [V, I64, I64, I64, I64, I64, I64]),
                "jabba_compress": (C.c_int, [V, V, I64, V, I64, C.POINTER(_Params), I64, I64, V, V, V, V, V, V, V,
                                             V, V, V, V]),
                "jabba_digitize_local": (C.c_int, [V, V, V, V, V, I64, V, C.POINTER(_Params), V, V, V, V, V, I64,
                                                   V, V]),
                "jabba_merge_global": (C.c_int, [V, V, V, I64, V, V, C.POINTER(_Params), V, V, V, V, I64, V, V]),
                "jabba_symbolize": (C.c_int, [V, V, V, V, V, V, I64, V, V, V]),
                "jabba_merge_global_points": (C.c_int, [V, V, V, V, V, I64, V, V, C.POINTER(_Params), V, V, V, V,
                                                        I64, V, V]),
                "jabba_block_order": (C.c_int, [V, V, V, V, V, V, I64, I64, V, C.POINTER(_Params), I64, V, V, V, V,
                                                V, V, V]),
                "jabba_block_items": (C.c_int, [V, V, V, V, V, I64, V, V, V, V, I64, V, C.POINTER(_Params), V, V,
                                                V]),
                "jabba_block_scatter": (C.c_int, [V, V, V, I64, V, V]),
                "jabba_reconstruct": (C.c_int, [V, V, I64, V, I64, V, V, V, V, V, C.POINTER(_Params), V, V, V]),
                "jabba_reconstruct_backward": (C.c_int, [V, V, I64, V, I64, V, V, V, V, V, I64, V, V]),
                "jabba_mse": (C.c_int, [V, V, V, I64, V, V]),
                "jabba_check_division": (C.c_int, [V, V, V, I64, C.c_int, V, V]),
                "jabba_profile_slot": (C.c_int, [V, C.c_int]),
                "jabba_diagnostics": (C.c_int, [V, C.POINTER(C.c_int64), C.c_int]),
                "jabba_reconstruct_noalloc": (C.c_int, [V, I64, V, I64, V, V, I64, V, V, V, C.c_int32, V, V, V]),
                "jabba_reconstruct_noalloc_status": (C.c_int, [V]),
                "jabba_profile_elapsed": (C.c_int, [V, C.c_int, C.c_int, C.POINTER(C.c_float)]),
                "jabba_autotune": (C.c_int, [V, C.c_int]),
                "jabba_reassign": (C.c_int, [V, V, V, V, V, V, I64, V, V, V, V, I64, C.POINTER(_Params), V, V]),
                "jabba_sse": (C.c_int, [V, V, V, V, V, V, I64, V, V, V, V, C.POINTER(_Params), V, V]),
                "jabba_get_tuning": (C.c_int, [V, C.POINTER(_Tuning)]),
                "jabba_set_tuning": (C.c_int, [V, C.POINTER(_Tuning)]),
                "jabba_set_spin_limit": (C.c_int, [V, C.c_uint32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _torch():
    import torch
    return torch


def _ptr(t) -> int:
    return 0 if t is None else t.data_ptr()


def _check(code: int, where: str):
    if code != 0:
        raise JabbaError(code, where)


class Context:
    """A device context of the library (its scratch space and status word)."""

    def __init__(self, device: int | None = None):
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2401_00109_gb300 needs a CUDA GPU; there is no CPU path")
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.lib = load()
        h = V()
        _check(self.lib.jabba_create(C.byref(h), self.device), "jabba_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.jabba_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- helpers
    def _stream(self, stream=None):
        torch = _torch()
        s = torch.cuda.current_stream(self.device) if stream is None else stream
        return V(s.cuda_stream)

    def sync_status(self, stream=None, where: str = "device"):
        _check(self.lib.jabba_sync_status(self.h, self._stream(stream)), where)

    def status(self, stream=None) -> int:
        """Synchronize and return (and clear) the device status code."""
        return int(self.lib.jabba_sync_status(self.h, self._stream(stream)))

    def set_spin_limit(self, polls: int):
        """Poll limit of the bounded device waits (0 = the default)."""
        _check(self.lib.jabba_set_spin_limit(self.h, int(polls)), "jabba_set_spin_limit")

    @staticmethod
    def plan(series_off_host: np.ndarray, p: Params, with_max: bool = False):
        off = np.ascontiguousarray(series_off_host, dtype=np.int64)
        nd, ns, mx = I64(), I64(), I64()
        _check(load().jabba_plan(off.ctypes.data_as(V), len(off) - 1, C.byref(p.c()), C.byref(nd), C.byref(ns),
                                 C.byref(mx)), "jabba_plan")
        return (nd.value, ns.value, mx.value) if with_max else (nd.value, ns.value)

    def reserve(self, n_points, n_series, n_domains, n_slots, group_capacity, max_dom_intervals=0):
        _check(self.lib.jabba_reserve(self.h, n_points, n_series, n_domains, n_slots, group_capacity,
                                      max_dom_intervals), "jabba_reserve")

    # -------------------------------------------------------------- steps
    def compress(self, x, series_off, p: Params, series_off_host=None, stream=None):
        """Domains + Eq. 1 compression.  Returns a dict of device tensors."""
        torch = _torch()
        dev = x.device
        if series_off_host is None:
            series_off_host = series_off.cpu().numpy()
        D, slots, mx = self.plan(series_off_host, p, with_max=True)
        S = len(series_off_host) - 1
        self.reserve(x.numel(), S, D, slots, 0, mx)
        o = dict(
            dom_begin=torch.empty(D, dtype=torch.int64, device=dev),
            dom_end=torch.empty(D, dtype=torch.int64, device=dev),
            dom_series=torch.empty(D, dtype=torch.int32, device=dev),
            series_dom_off=torch.empty(S + 1, dtype=torch.int64, device=dev),
            dom_slot_off=torch.empty(D + 1, dtype=torch.int64, device=dev),
            piece_len=torch.empty(max(slots, 1), dtype=torch.int32, device=dev),
            piece_inc=torch.empty(max(slots, 1), dtype=torch.float64, device=dev),
            dom_piece_cnt=torch.empty(max(D, 1), dtype=torch.int32, device=dev),
            dom_piece_off=torch.empty(D + 1, dtype=torch.int64, device=dev),
            piece_stats=torch.empty(PIECE_STATS_BYTES // 8, dtype=torch.int64, device=dev),
        )
        _check(self.lib.jabba_compress(
            self.h, _ptr(x), x.numel(), _ptr(series_off), S, C.byref(p.c()), D, slots, _ptr(o["dom_begin"]),
            _ptr(o["dom_end"]), _ptr(o["dom_series"]), _ptr(o["series_dom_off"]), _ptr(o["dom_slot_off"]),
            _ptr(o["piece_len"]), _ptr(o["piece_inc"]), _ptr(o["dom_piece_cnt"]), _ptr(o["dom_piece_off"]),
            _ptr(o["piece_stats"]), self._stream(stream)), "jabba_compress")
        o.update(n_domains=D, n_slots=slots, n_series=S)
        return o

    def digitize_local(self, c: dict, p: Params, group_capacity: int | None = None, stream=None):
        torch = _torch()
        dev = c["piece_len"].device
        D = c["n_domains"]
        if group_capacity is None:
            group_capacity = max(1, min(c["n_slots"], max(1 << 16, c["n_slots"] // 4)))
        while True:
            o = dict(
                sigma=torch.empty(4, dtype=torch.float64, device=dev),   # sigma_len, sigma_inc (+ PCA axis)
                local_label=torch.empty(max(c["n_slots"], 1), dtype=torch.int32, device=dev),
                dom_group_cnt=torch.empty(max(D, 1), dtype=torch.int32, device=dev),
                dom_group_off=torch.empty(D + 1, dtype=torch.int64, device=dev),
                groups=torch.empty(group_capacity * JABBA_GROUP_BYTES // 8, dtype=torch.int64, device=dev),
                n_groups=torch.zeros(1, dtype=torch.int64, device=dev),
            )
            _check(self.lib.jabba_digitize_local(
                self.h, _ptr(c["piece_len"]), _ptr(c["piece_inc"]), _ptr(c["dom_slot_off"]), _ptr(c["dom_piece_cnt"]),
                D, _ptr(c["piece_stats"]), C.byref(p.c()), _ptr(o["sigma"]), _ptr(o["local_label"]),
                _ptr(o["dom_group_cnt"]), _ptr(o["dom_group_off"]), _ptr(o["groups"]), group_capacity,
                _ptr(o["n_groups"]), self._stream(stream)), "jabba_digitize_local")
            code = self.lib.jabba_sync_status(self.h, self._stream(stream))
            if code == ERR_CAPACITY:
                need = int(o["n_groups"].item())
                if need > group_capacity:
                    group_capacity = need
                    continue
            _check(code, "jabba_digitize_local")
            break
        o["group_capacity"] = group_capacity
        return o

    def merge_global(self, l: dict, p: Params, dict_capacity: int | None = None, stream=None, items=None):
        """Stage II.  items = (item_X, item_Y): binary64 points of the group
        records to merge (the block form's starting points); None merges the
        records' centres."""
        torch = _torch()
        dev = l["groups"].device
        cap = l["group_capacity"]
        if dict_capacity is None:
            dict_capacity = cap
        o = dict(
            l2g=torch.empty(max(cap, 1), dtype=torch.int32, device=dev),
            dict_len=torch.empty(max(dict_capacity, 1), dtype=torch.float64, device=dev),
            dict_inc=torch.empty(max(dict_capacity, 1), dtype=torch.float64, device=dev),
            dict_count=torch.empty(max(dict_capacity, 1), dtype=torch.int64, device=dev),
            k=torch.zeros(1, dtype=torch.int64, device=dev),
        )
        if items is None:
            _check(self.lib.jabba_merge_global(
                self.h, _ptr(l["groups"]), _ptr(l["n_groups"]), cap, _ptr(l["dom_group_off"]), _ptr(l["sigma"]),
                C.byref(p.c()), _ptr(o["l2g"]), _ptr(o["dict_len"]), _ptr(o["dict_inc"]), _ptr(o["dict_count"]),
                dict_capacity, _ptr(o["k"]), self._stream(stream)), "jabba_merge_global")
        else:
            _check(self.lib.jabba_merge_global_points(
                self.h, _ptr(l["groups"]), _ptr(items[0]), _ptr(items[1]), _ptr(l["n_groups"]), cap,
                _ptr(l["dom_group_off"]), _ptr(l["sigma"]), C.byref(p.c()), _ptr(o["l2g"]), _ptr(o["dict_len"]),
                _ptr(o["dict_inc"]), _ptr(o["dict_count"]), dict_capacity, _ptr(o["k"]), self._stream(stream)),
                "jabba_merge_global_points")
        return o

    def symbolize_step(self, c: dict, l: dict, m: dict, n_pieces: int, stream=None):
        torch = _torch()
        sym = torch.empty(max(n_pieces, 1), dtype=torch.int32, device=c["piece_len"].device)
        _check(self.lib.jabba_symbolize(
            self.h, _ptr(l["local_label"]), _ptr(c["dom_slot_off"]), _ptr(c["dom_piece_cnt"]), _ptr(c["dom_piece_off"]),
            _ptr(l["dom_group_off"]), c["n_domains"], _ptr(m["l2g"]), _ptr(sym), self._stream(stream)),
            "jabba_symbolize")
        return sym[:n_pieces]

    def symbolize(self, x, series_off, p: Params, series_off_host=None, stream=None):
        """The whole forward path: compress, local digitization, merge, symbols."""
        c = self.compress(x, series_off, p, series_off_host, stream)
        self.sync_status(stream, "jabba_compress")
        l = self.digitize_local(c, p, stream=stream)
        m = self.merge_global(l, p, stream=stream)
        self.sync_status(stream, "jabba_merge_global")
        N = int(c["dom_piece_off"][-1].item())
        k = int(m["k"].item())
        G = int(l["n_groups"].item())
        sym = self.symbolize_step(c, l, m, N, stream)
        self.sync_status(stream, "jabba_symbolize")
        out = dict(c)
        out.update(l)
        out.update(m)
        out.update(symbol=sym, n_pieces=N, n_groups_host=G, k_host=k, dict_len=m["dict_len"][:k],
                   dict_inc=m["dict_inc"][:k], dict_count=m["dict_count"][:k])
        return out

    def symbolize_blocks(self, x, series_off, p: Params, n_blocks: int | None = None, series_off_host=None,
                         stream=None):
        """The two-stage digitization in the block form of Sec. 5: one global
        sort of the pieces by rho, n_blocks contiguous sorted blocks (default:
        as many as the collection has domains) aggregated by Stage I, and
        Stage II over the local groups' starting points.  Returns the
        compression outputs, the dictionary and the symbols in compact-piece
        order (plus the block arrays)."""
        torch = _torch()
        c = self.compress(x, series_off, p, series_off_host, stream)
        self.sync_status(stream, "jabba_compress")
        N = int(c["dom_piece_off"][-1].item())
        M = int(n_blocks) if n_blocks else max(1, c["n_domains"])
        dev = x.device
        b = dict(
            sigma=torch.empty(2, dtype=torch.float64, device=dev),
            order=torch.empty(max(N, 1), dtype=torch.int32, device=dev),
            piece_len=torch.empty(max(N, 1), dtype=torch.int32, device=dev),
            piece_inc=torch.empty(max(N, 1), dtype=torch.float64, device=dev),
            dom_slot_off=torch.empty(M + 1, dtype=torch.int64, device=dev),
            dom_piece_cnt=torch.empty(M, dtype=torch.int32, device=dev),
        )
        _check(self.lib.jabba_block_order(
            self.h, _ptr(c["piece_len"]), _ptr(c["piece_inc"]), _ptr(c["dom_slot_off"]), _ptr(c["dom_piece_cnt"]),
            _ptr(c["dom_piece_off"]), c["n_domains"], N, _ptr(c["piece_stats"]), C.byref(p.c()), M,
            _ptr(b["sigma"]), _ptr(b["order"]), _ptr(b["piece_len"]), _ptr(b["piece_inc"]), _ptr(b["dom_slot_off"]),
            _ptr(b["dom_piece_cnt"]), self._stream(stream)), "jabba_block_order")
        b.update(dom_piece_off=b["dom_slot_off"], n_domains=M, n_slots=max(N, 1), piece_stats=c["piece_stats"])
        l = self.digitize_local(b, p, stream=stream)
        cap = l["group_capacity"]
        iX = torch.empty(max(cap, 1), dtype=torch.float64, device=dev)
        iY = torch.empty(max(cap, 1), dtype=torch.float64, device=dev)
        _check(self.lib.jabba_block_items(
            self.h, _ptr(l["local_label"]), _ptr(b["dom_slot_off"]), _ptr(b["dom_piece_cnt"]), _ptr(l["dom_group_off"]),
            M, _ptr(b["piece_len"]), _ptr(b["piece_inc"]), _ptr(l["groups"]), _ptr(l["n_groups"]), cap,
            _ptr(l["sigma"]), C.byref(p.c()), _ptr(iX), _ptr(iY), self._stream(stream)), "jabba_block_items")
        m = self.merge_global(l, p, stream=stream, items=(iX, iY))
        self.sync_status(stream, "jabba_merge_global_points")
        k = int(m["k"].item())
        sym_b = self.symbolize_step(b, l, m, N, stream)
        sym = torch.empty(max(N, 1), dtype=torch.int32, device=dev)
        _check(self.lib.jabba_block_scatter(self.h, _ptr(b["order"]), _ptr(sym_b), N, _ptr(sym),
                                            self._stream(stream)), "jabba_block_scatter")
        self.sync_status(stream, "jabba_block_scatter")
        out = dict(c)
        out.update(blocks=b, local=l, n_blocks=M, l2g=m["l2g"], symbol=sym[:N], n_pieces=N, k_host=k,
                   n_groups_host=int(l["n_groups"].item()), sigma=l["sigma"], dict_len=m["dict_len"][:k],
                   dict_inc=m["dict_inc"][:k], dict_count=m["dict_count"][:k], k=m["k"])
        return out

    def reconstruct(self, x, series_off, out: dict, p: Params, dict_inc=None, stream=None):
        torch = _torch()
        dev = x.device
        di = out["dict_inc"] if dict_inc is None else dict_inc
        qlen = torch.empty(max(out["n_pieces"], 1), dtype=torch.int32, device=dev)
        xhat = torch.empty_like(x)
        _check(self.lib.jabba_reconstruct(
            self.h, _ptr(x), x.numel(), _ptr(series_off), out["n_series"], _ptr(out["series_dom_off"]),
            _ptr(out["dom_piece_off"]), _ptr(out["symbol"]), _ptr(out["dict_len"]), _ptr(di), C.byref(p.c()),
            _ptr(qlen), _ptr(xhat), self._stream(stream)), "jabba_reconstruct")
        return qlen[:out["n_pieces"]], xhat

    def reconstruct_backward(self, x, series_off, out: dict, qlen, dict_inc, stream=None):
        torch = _torch()
        k = dict_inc.numel()
        grad = torch.empty(max(k, 1), dtype=torch.float64, device=x.device)
        _check(self.lib.jabba_reconstruct_backward(
            self.h, _ptr(x), x.numel(), _ptr(series_off), out["n_series"], _ptr(out["series_dom_off"]),
            _ptr(out["dom_piece_off"]), _ptr(out["symbol"]), _ptr(qlen), _ptr(dict_inc), k, _ptr(grad),
            self._stream(stream)), "jabba_reconstruct_backward")
        return grad[:k]

    def reassign(self, out: dict, p: Params, stream=None):
        """Full-reassignment digitization (Alg. 1 Digitize; Sec. 3.2 argmin):
        the nearest dictionary entry of every piece of a symbolize() result,
        ties to the smaller entry index.  Returns the compact symbols."""
        torch = _torch()
        N = int(out["n_pieces"])
        sym = torch.empty(max(N, 1), dtype=torch.int32, device=out["piece_len"].device)
        cap = max(int(out["k_host"]), 1)
        _check(self.lib.jabba_reassign(
            self.h, _ptr(out["piece_len"]), _ptr(out["piece_inc"]), _ptr(out["dom_slot_off"]),
            _ptr(out["dom_piece_cnt"]), _ptr(out["dom_piece_off"]), out["n_domains"], _ptr(out["sigma"]),
            _ptr(out["dict_len"]), _ptr(out["dict_inc"]), _ptr(out["k"]), cap, C.byref(p.c()), _ptr(sym),
            self._stream(stream)), "jabba_reassign")
        return sym[:N]

    def sse(self, out: dict, p: Params, symbol, stream=None):
        """Exact sum of squared normalised errors of an assignment (device scalar)."""
        torch = _torch()
        res = torch.empty(1, dtype=torch.float64, device=out["piece_len"].device)
        _check(self.lib.jabba_sse(
            self.h, _ptr(out["piece_len"]), _ptr(out["piece_inc"]), _ptr(out["dom_slot_off"]),
            _ptr(out["dom_piece_cnt"]), _ptr(out["dom_piece_off"]), out["n_domains"], _ptr(out["sigma"]),
            _ptr(out["dict_len"]), _ptr(out["dict_inc"]), _ptr(symbol), C.byref(p.c()), _ptr(res),
            self._stream(stream)), "jabba_sse")
        return res

    def autotune(self, enable: bool):
        """Autotuning mode: while on, every compress / local digitization /
        merge call times each candidate launch configuration on its own
        inputs and keeps the fastest (jabba_autotune)."""
        _check(self.lib.jabba_autotune(self.h, 1 if enable else 0), "jabba_autotune")

    def tuning(self) -> dict:
        t = _Tuning()
        _check(self.lib.jabba_get_tuning(self.h, C.byref(t)), "jabba_get_tuning")
        return {f: int(getattr(t, f)) for f in TUNING_FIELDS}

    def set_tuning(self, cfg: dict):
        t = _Tuning()
        cur = self.tuning()
        cur.update(cfg)
        for f in TUNING_FIELDS:
            setattr(t, f, int(cur[f]))
        _check(self.lib.jabba_set_tuning(self.h, C.byref(t)), "jabba_set_tuning")

    def diagnostics(self):
        """Counters of the last calls: exact compression decisions, merge rounds."""
        out = (C.c_int64 * 2)()
        _check(self.lib.jabba_diagnostics(self.h, out, 2), "jabba_diagnostics")
        return dict(exact_decisions=int(out[0]), merge_rounds=int(out[1]))

    def profile_slot(self, slot: int):
        _check(self.lib.jabba_profile_slot(self.h, int(slot)), "jabba_profile_slot")

    def profile_elapsed(self, slot: int, stage: int) -> float:
        ms = C.c_float()
        _check(self.lib.jabba_profile_elapsed(self.h, int(slot), int(stage), C.byref(ms)), "jabba_profile_elapsed")
        return ms.value

    def check_division(self, a, b, mode: int = 0, stream=None):
        """Self-check of the merge's integer-unit binary64 division (device
        float64 tensors a, b of one size): returns (quotients the path
        handled, quotients that differ from the binary64 division)."""
        torch = _torch()
        counts = torch.zeros(2, dtype=torch.int64, device=a.device)
        _check(self.lib.jabba_check_division(self.h, _ptr(a), _ptr(b), a.numel(), int(mode), _ptr(counts),
                                             self._stream(stream)), "jabba_check_division")
        c = counts.cpu().numpy()
        return int(c[0]), int(c[1])

    def mse(self, x, xhat, stream=None):
        torch = _torch()
        out = torch.empty(1, dtype=torch.float64, device=x.device)
        _check(self.lib.jabba_mse(self.h, _ptr(x), _ptr(xhat), x.numel(), _ptr(out), self._stream(stream)),
               "jabba_mse")
        return out


NOALLOC_MAX_PIECES = 1 << 18
NOALLOC_MAX_SERIES = 1 << 14


def reconstruct_noalloc(x, series_off, out: dict, p: Params, qlen=None, xhat=None, dict_inc=None, stream=None,
                        n_pieces=None):
    """jabba_reconstruct_noalloc: the reconstruction without a context and
    without any device allocation by the library (fixed internal scratch;
    at most NOALLOC_MAX_PIECES pieces and NOALLOC_MAX_SERIES series).  The
    output buffers may be passed in (qlen, xhat) so that nothing is
    allocated on this path at all.  n_pieces overrides the piece count passed
    to the library (the device-side bounds check is tested with it)."""
    torch = _torch()
    L = load()
    N = int(out["n_pieces"]) if n_pieces is None else int(n_pieces)
    # the C call works on the current device: make it the inputs' device
    with torch.cuda.device(x.device):
        s = torch.cuda.current_stream(x.device) if stream is None else stream
        if qlen is None:
            qlen = torch.empty(max(N, 1), dtype=torch.int32, device=x.device)
        if xhat is None:
            xhat = torch.empty_like(x)
        di = out["dict_inc"] if dict_inc is None else dict_inc
        _check(L.jabba_reconstruct_noalloc(
            _ptr(x), x.numel(), _ptr(series_off), out["n_series"], _ptr(out["series_dom_off"]),
            _ptr(out["dom_piece_off"]), N, _ptr(out["symbol"]), _ptr(out["dict_len"]), _ptr(di), int(p.round_mode),
            _ptr(qlen), _ptr(xhat), V(s.cuda_stream)), "jabba_reconstruct_noalloc")
    return qlen[:N], xhat


def reconstruct_noalloc_status(device=None, stream=None) -> int:
    """Synchronize and return (and clear) the status word of the
    allocation-free reconstruction on `device` (0 or ERR_CAPACITY)."""
    torch = _torch()
    dev = torch.cuda.current_device() if device is None else device
    with torch.cuda.device(dev):
        s = torch.cuda.current_stream(dev) if stream is None else stream
        return int(load().jabba_reconstruct_noalloc_status(V(s.cuda_stream)))


def _autograd_function():
    torch = _torch()

    class JabbaMSE(torch.autograd.Function):
        """Reconstruction MSE as a function of the dictionary increments, with
        the symbols and the quantized lengths held fixed (Sec. 3.3).  The
        backward pass is the library's adjoint kernel, which recomputes the
        reconstruction instead of storing it."""

        @staticmethod
        def forward(ctx_, dict_inc, jctx: Context, x, series_off, out: dict, qlen, p: Params):
            _, xhat = _reconstruct_fixed(jctx, x, series_off, out, qlen, dict_inc, p)
            loss = jctx.mse(x, xhat)
            ctx_.save_for_backward(dict_inc.detach())
            ctx_.jabba = (jctx, x, series_off, out, qlen)
            return loss[0]

        @staticmethod
        def backward(ctx_, g):
            (dict_inc,) = ctx_.saved_tensors
            jctx, x, series_off, out, qlen = ctx_.jabba
            grad = jctx.reconstruct_backward(x, series_off, out, qlen, dict_inc)
            return grad * g, None, None, None, None, None, None

    return JabbaMSE


def _reconstruct_fixed(jctx: Context, x, series_off, out, qlen, dict_inc, p: Params):
    """Reconstruction with the quantized lengths given (the dictionary lengths
    are replaced by exactly those integers, which the carry then reproduces)."""
    return jctx.reconstruct(x, series_off, out, p, dict_inc=dict_inc)


_JabbaMSE = None


def JabbaMSE():
    global _JabbaMSE
    if _JabbaMSE is None:
        _JabbaMSE = _autograd_function()
    return _JabbaMSE


class Pipeline:
    """Preallocated forward path for one collection shape: the four C-ABI
    steps (compress, local digitization, merge, label propagation) enqueued on
    one stream with no host synchronization, so that a whole step can be
    captured once in a CUDA graph and replayed (the batched form).  Output
    capacities are fixed at construction; a run that needs more reports
    JABBA_ERR_CAPACITY through sync_status()."""

    def __init__(self, ctx: Context, series_off_host, n_points: int, p: Params, group_capacity: int,
                 dict_capacity: int | None = None, device=None):
        torch = _torch()
        self.ctx, self.p = ctx, p
        self.pc = p.c()
        dev = torch.device("cuda", ctx.device) if device is None else device
        off = np.ascontiguousarray(series_off_host, dtype=np.int64)
        self.S = len(off) - 1
        self.n_points = int(n_points)
        D, slots, mx = Context.plan(off, p, with_max=True)
        self.D, self.slots = D, slots
        self.gcap = int(max(1, group_capacity))
        self.kcap = int(self.gcap if dict_capacity is None else max(1, dict_capacity))
        ctx.reserve(self.n_points, self.S, D, slots, self.gcap, mx)
        e = lambda n, dt: torch.empty(max(int(n), 1), dtype=dt, device=dev)
        i64, i32, f64 = torch.int64, torch.int32, torch.float64
        self.x = e(self.n_points, f64)
        self.series_off = e(self.S + 1, i64)
        self.series_off.copy_(torch.from_numpy(off))
        self.b = dict(dom_begin=e(D, i64), dom_end=e(D, i64), dom_series=e(D, i32), series_dom_off=e(self.S + 1, i64),
                      dom_slot_off=e(D + 1, i64), piece_len=e(slots, i32), piece_inc=e(slots, f64),
                      dom_piece_cnt=e(D, i32), dom_piece_off=e(D + 1, i64), piece_stats=e(PIECE_STATS_BYTES // 8, i64),
                      sigma=e(4, f64), local_label=e(slots, i32), dom_group_cnt=e(D, i32), dom_group_off=e(D + 1, i64),
                      groups=e(self.gcap * JABBA_GROUP_BYTES // 8, i64), n_groups=e(1, i64), l2g=e(self.gcap, i32),
                      dict_len=e(self.kcap, f64), dict_inc=e(self.kcap, f64), dict_count=e(self.kcap, i64),
                      k=e(1, i64), symbol=e(slots, i32))
        self.graph = None

    def enqueue(self, stream=None):
        """Enqueue one forward step on `stream` (default: current stream)."""
        self.enqueue_front(stream)
        self.enqueue_back(stream)

    def enqueue_front(self, stream=None):
        """The per-domain half of a step: compression and Stage I."""
        L, h, b, pc = self.ctx.lib, self.ctx.h, self.b, self.pc
        st = self.ctx._stream(stream)
        P = _ptr
        _check(L.jabba_compress(h, P(self.x), self.n_points, P(self.series_off), self.S, C.byref(pc), self.D,
                                self.slots, P(b["dom_begin"]), P(b["dom_end"]), P(b["dom_series"]),
                                P(b["series_dom_off"]), P(b["dom_slot_off"]), P(b["piece_len"]), P(b["piece_inc"]),
                                P(b["dom_piece_cnt"]), P(b["dom_piece_off"]), P(b["piece_stats"]), st),
               "jabba_compress")
        _check(L.jabba_digitize_local(h, P(b["piece_len"]), P(b["piece_inc"]), P(b["dom_slot_off"]),
                                      P(b["dom_piece_cnt"]), self.D, P(b["piece_stats"]), C.byref(pc), P(b["sigma"]),
                                      P(b["local_label"]), P(b["dom_group_cnt"]), P(b["dom_group_off"]),
                                      P(b["groups"]), self.gcap, P(b["n_groups"]), st), "jabba_digitize_local")

    def enqueue_back(self, stream=None):
        """The global half of a step: Stage II merge and label propagation."""
        L, h, b, pc = self.ctx.lib, self.ctx.h, self.b, self.pc
        st = self.ctx._stream(stream)
        P = _ptr
        _check(L.jabba_merge_global(h, P(b["groups"]), P(b["n_groups"]), self.gcap, P(b["dom_group_off"]),
                                    P(b["sigma"]), C.byref(pc), P(b["l2g"]), P(b["dict_len"]), P(b["dict_inc"]),
                                    P(b["dict_count"]), self.kcap, P(b["k"]), st), "jabba_merge_global")
        _check(L.jabba_symbolize(h, P(b["local_label"]), P(b["dom_slot_off"]), P(b["dom_piece_cnt"]),
                                 P(b["dom_piece_off"]), P(b["dom_group_off"]), self.D, P(b["l2g"]), P(b["symbol"]), st),
               "jabba_symbolize")

    def tune(self, stream=None) -> dict:
        """Autotune the launch configuration on this collection: one eager
        step in tuning mode (each stage times its candidates on its own
        inputs).  Returns the configuration chosen."""
        self.ctx.autotune(True)
        try:
            self.enqueue(stream)
            self.ctx.sync_status(stream, "autotuning step")
        finally:
            self.ctx.autotune(False)
        return self.ctx.tuning()

    def capture(self, keep_graph: bool = False):
        """Capture one step into a CUDA graph (call after one eager step).
        keep_graph=True keeps the graph for inspection (graph_kernel_nodes)."""
        torch = _torch()
        g = torch.cuda.CUDAGraph(keep_graph=keep_graph) if keep_graph else torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(device=self.x.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.enqueue(s)
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def capture_halves(self, stream):
        """Capture the two halves of a step (front: compression + Stage I;
        back: merge + label propagation) as two CUDA graphs on `stream`, so
        that consecutive steps of two pipelines can overlap (see
        InFlight)."""
        torch = _torch()
        graphs = []
        for fn in (self.enqueue_front, self.enqueue_back):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(stream):
                with torch.cuda.graph(g, stream=stream):
                    fn(stream)
            graphs.append(g)
        return graphs

    def as_result(self) -> dict:
        """The last step's outputs in the layout Context.symbolize() returns
        (device tensors; reads the piece and dictionary counts)."""
        b = self.b
        N = int(b["dom_piece_off"][self.D].item())
        k = int(b["k"][0].item())
        out = {key: b[key] for key in ("piece_len", "piece_inc", "dom_slot_off", "dom_piece_cnt", "dom_piece_off",
                                       "sigma", "k")}
        out.update(n_domains=self.D, n_pieces=N, k_host=k, dict_len=b["dict_len"][:k], dict_inc=b["dict_inc"][:k],
                   symbol=b["symbol"][:N])
        return out

    def results(self):
        """Host copies of the symbols and dictionary of the last step."""
        b = self.b
        N = int(b["dom_piece_off"][self.D].item())
        k = int(b["k"][0].item())
        return dict(symbol=b["symbol"][:N].cpu().numpy(), dict_len=b["dict_len"][:k].cpu().numpy(),
                    dict_inc=b["dict_inc"][:k].cpu().numpy(), dict_count=b["dict_count"][:k].cpu().numpy(),
                    n_pieces=N, k=k, n_groups=int(b["n_groups"][0].item()))


class InFlight:
    """Two batches in flight: two pipelines (each with its own context and
    buffers) on two streams.  Step i runs on pipeline i % 2: its front half
    (compression, Stage I) may overlap the other pipeline's back half, whose
    merge-rounds kernel leaves most of the GPU idle; the back halves of the
    two pipelines are ordered one after the other (the merge's cooperative
    kernels never run concurrently)."""

    def __init__(self, pipelines):
        torch = _torch()
        self.pl = list(pipelines)
        self.streams = [torch.cuda.Stream(device=p.x.device) for p in self.pl]
        for s in self.streams:
            s.wait_stream(torch.cuda.current_stream())
        self.halves = [p.capture_halves(s) for p, s in zip(self.pl, self.streams)]
        self.back_done = [torch.cuda.Event() for _ in self.pl]
        # recorded after each front half: the pipeline's input series are no
        # longer read, so the next batch may be copied into them
        self.front_done = [torch.cuda.Event() for _ in self.pl]
        self.count = 0

    def next_index(self) -> int:
        """Pipeline that the next step() runs on."""
        return self.count % len(self.pl)

    def step(self, before=None, after=None):
        """Issue one step on the next pipeline.  before(i, stream) and
        after(i, stream), if given, enqueue work on that pipeline's stream
        around the step (e.g. a wait for the host->device copy of its input
        and the device->host copy of its symbols)."""
        torch = _torch()
        i = self.count % len(self.pl)
        j = (i + len(self.pl) - 1) % len(self.pl)
        s = self.streams[i]
        front, back = self.halves[i]
        with torch.cuda.stream(s):
            if before is not None:
                before(i, s)
            front.replay()
            self.front_done[i].record(s)
            s.wait_event(self.back_done[j])
            back.replay()
            self.back_done[i].record(s)
            if after is not None:
                after(i, s)
        self.count += 1

    def join(self, stream=None):
        """Make `stream` (default: current) wait for every step issued so far."""
        torch = _torch()
        cur = torch.cuda.current_stream() if stream is None else stream
        for s in self.streams:
            cur.wait_stream(s)

    def fork(self, stream=None):
        """Make the pipelines' streams wait for `stream` (default: current)."""
        torch = _torch()
        cur = torch.cuda.current_stream() if stream is None else stream
        for s in self.streams:
            s.wait_stream(cur)


def tune_inflight(pipelines, base: dict, steps: int = 4, finalists: int = 4, final_steps: int = 20):
    """Pick the launch configuration of two batches in flight: the front
    half's kernels must leave room on every SM for the other batch's
    cooperative merge, so the resident CTAs per SM of compression, of the
    local-aggregation kernels and of the merge rounds (and its warps per CTA)
    are searched around `base` (the single-batch autotuned configuration),
    timing a few steps of each candidate with CUDA events; the `finalists`
    fastest are timed again over `final_steps` steps (step times vary from
    run to run by a few percent).  Returns (best configuration, its ms per
    step, an InFlight runner captured with it)."""
    torch = _torch()

    def timed(cfg, n):
        for pl in pipelines:
            pl.ctx.set_tuning(cfg)
        fl = InFlight(pipelines)
        for _ in range(2):
            fl.step()
        fl.join()
        torch.cuda.synchronize()
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fl.fork(st)
        for _ in range(n):
            fl.step()
        fl.join(st)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n, fl

    m_opts = [(1, 8), (2, 8), (1, 4), (2, 4)] if base.get("merge_form", 1) == 1 else [(1, 8), (2, 8)]
    first = []
    for c_sm in (1, 2):
        for cap in (2, 3, 4, 6):
            for m_sm, m_w in m_opts:
                cfg = dict(base, compress_ctas_per_sm=c_sm, local_ctas_cap=cap, merge_ctas_per_sm=m_sm,
                           merge_warps=m_w)
                first.append((timed(cfg, steps)[0], cfg))
    first.sort(key=lambda r: r[0])
    best = None
    for _, cfg in first[:max(1, finalists)]:
        ms, fl = timed(cfg, final_steps)
        if best is None or ms < best[1]:
            best = (cfg, ms, fl)
    for pl in pipelines:
        pl.ctx.set_tuning(best[0])
        pl.ctx.sync_status(where="in-flight tuning")
    return best


def graph_kernel_nodes(graph) -> int:
    """Number of kernel nodes of a captured torch CUDA graph (driver API)."""
    import ctypes.util
    raw = graph.raw_cuda_graph()
    cuda = C.CDLL(ctypes.util.find_library("cuda") or "libcuda.so.1")
    n = C.c_size_t(0)
    if cuda.cuGraphGetNodes(C.c_void_p(raw), None, C.byref(n)) != 0:
        raise RuntimeError("cuGraphGetNodes failed")
    nodes = (C.c_void_p * n.value)()
    cuda.cuGraphGetNodes(C.c_void_p(raw), nodes, C.byref(n))
    k = 0
    for i in range(n.value):
        t = C.c_int(-1)
        cuda.cuGraphNodeGetType(C.c_void_p(nodes[i]), C.byref(t))
        k += int(t.value == 0)  # CU_GRAPH_NODE_TYPE_KERNEL
    return k
