"""CPU oracle for bulk transaction execution -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it.

The arithmetic lives in ``gputx_oracle.c`` (plain single-threaded C, built with
gcc); this module marshals numpy arrays into it and adds a few numpy-only
statistics.  Each function cites the part of the paper it follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gputx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MODE_PAPER = 0
MODE_ADD = 1
CLS_R, CLS_W, CLS_A = 0, 1, 2
MAX_OPS = 17
OE_DIST_PER_WH = 10
OE_CUST_PER_DIST = 3000


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 (plain C, no vector intrinsics)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        i64, i32, p = C.c_int64, C.c_int32, C.c_void_p
        _lib.orc_num_objects.restype = i64
        _lib.orc_num_objects.argtypes = [p]
        _lib.orc_extract.restype = C.c_int
        _lib.orc_extract.argtypes = [p, i64, p, p, C.c_int, C.c_int, C.c_int, p, p, p]
        _lib.orc_levels.restype = None
        _lib.orc_levels.argtypes = [i64, C.c_int, p, p, i64, p]
        _lib.orc_onepass_levels.restype = None
        _lib.orc_onepass_levels.argtypes = [i64, C.c_int, p, p, p, p]
        _lib.orc_appb_edges.restype = i64
        _lib.orc_appb_edges.argtypes = [i64, C.c_int, p, p, i64, p, i64]
        _lib.orc_topo_levels.restype = None
        _lib.orc_topo_levels.argtypes = [i64, p, i64, p]
        _lib.orc_execute.restype = C.c_int
        _lib.orc_execute.argtypes = [p, i64, p, p, p, C.c_int, C.c_int, p, p, p]
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


_P = C.c_void_p
_I = C.c_int64


class _OrcDB(C.Structure):
    _fields_ = [
        ("n_branch", _I), ("n_teller", _I), ("n_account", _I),
        ("br_bal", _P), ("tel_bal", _P), ("acc_bal", _P),
        ("hist_cap", _I), ("hist_n", _I), ("hist", _P),
        ("n_sub", _I), ("sub", _P), ("ai_present", _P), ("ai_data", _P),
        ("sf_present", _P), ("sf_active", _P), ("sf_err", _P), ("sf_data_a", _P),
        ("sf_data_b", _P), ("cf_present", _P), ("cf_end", _P), ("cf_numberx", _P),
        ("n_wh", _I), ("n_items", _I),
        ("w_tax", _P), ("w_ytd", _P), ("d_tax", _P), ("d_ytd", _P), ("d_next_o_id", _P),
        ("c_discount", _P), ("c_balance", _P), ("c_ytd", _P), ("c_payment_cnt", _P),
        ("c_last_o_id", _P), ("i_price", _P), ("s_quantity", _P), ("s_ytd", _P),
        ("s_order_cnt", _P),
        ("ord_cap", _I), ("ord_n", _I), ("ord", _P),
        ("ol_cap", _I), ("ol_n", _I), ("ol", _P),
        ("oid_cap", _I), ("ord_idx", _P),
    ]


class OracleDB:
    """The database state the serial executor mutates, as numpy arrays.

    ``dc``/``sub``/``oe`` take the dicts produced by ``workloads.dc_tables``,
    ``workloads.sub_tables`` and ``workloads.oe_tables`` (copied).  History,
    order and order-line tables are append-only arrays with the given
    capacities.
    """

    def __init__(self, dc=None, sub=None, oe=None, hist_cap=0, ord_cap=0,
                 ol_cap=0, oid_cap=0):
        s = _OrcDB()
        self.a = {}

        def keep(name, arr, dtype):
            arr = np.ascontiguousarray(np.array(arr, dtype=dtype, copy=True))
            self.a[name] = arr
            return _ptr(arr)

        if dc is not None:
            s.n_branch = len(dc["branch_balance"])
            s.n_teller = len(dc["teller_balance"])
            s.n_account = len(dc["account_balance"])
            s.br_bal = keep("br_bal", dc["branch_balance"], np.int64)
            s.tel_bal = keep("tel_bal", dc["teller_balance"], np.int64)
            s.acc_bal = keep("acc_bal", dc["account_balance"], np.int64)
            s.hist_cap = hist_cap
            s.hist = keep("hist", np.zeros((max(hist_cap, 1), 5)), np.int64)
        if sub is not None:
            s.n_sub = sub["sub"].shape[0]
            s.sub = keep("sub", sub["sub"], np.int32)
            s.ai_present = keep("ai_present", sub["ai_present"], np.uint8)
            s.ai_data = keep("ai_data", sub["ai_data"], np.int32)
            s.sf_present = keep("sf_present", sub["sf_present"], np.uint8)
            s.sf_active = keep("sf_active", sub["sf_active"], np.int32)
            s.sf_err = keep("sf_err", sub["sf_err"], np.int32)
            s.sf_data_a = keep("sf_data_a", sub["sf_data_a"], np.int32)
            s.sf_data_b = keep("sf_data_b", sub["sf_data_b"], np.int32)
            s.cf_present = keep("cf_present", sub["cf_present"], np.uint8)
            s.cf_end = keep("cf_end", sub["cf_end"], np.int32)
            s.cf_numberx = keep("cf_numberx", sub["cf_numberx"], np.int32)
        if oe is not None:
            s.n_wh = len(oe["w_tax"])
            s.n_items = len(oe["i_price"])
            for name, dt in (("w_tax", np.int64), ("w_ytd", np.int64), ("d_tax", np.int64),
                             ("d_ytd", np.int64), ("d_next_o_id", np.int64),
                             ("c_discount", np.int64), ("c_balance", np.int64),
                             ("c_ytd", np.int64), ("c_payment_cnt", np.int64),
                             ("c_last_o_id", np.int64), ("i_price", np.int64),
                             ("s_quantity", np.int32), ("s_ytd", np.int64),
                             ("s_order_cnt", np.int32)):
                setattr(s, name, keep(name, oe[name], dt))
            s.ord_cap, s.ol_cap, s.oid_cap = ord_cap, ol_cap, oid_cap
            s.ord = keep("ord", np.zeros((max(ord_cap, 1), 6)), np.int64)
            s.ol = keep("ol", np.zeros((max(ol_cap, 1), 5)), np.int64)
            n_d = s.n_wh * OE_DIST_PER_WH
            s.ord_idx = keep("ord_idx", np.full((n_d, max(oid_cap, 1)), -1), np.int64)
        self.s = s

    # -- views ------------------------------------------------------------
    def __getitem__(self, name):
        return self.a[name]

    @property
    def hist_n(self):
        return self.s.hist_n

    def history(self):
        return self.a["hist"][: self.s.hist_n]

    def orders(self):
        return self.a["ord"][: self.s.ord_n]

    def order_lines(self):
        return self.a["ol"][: self.s.ol_n]

    def num_objects(self) -> int:
        return _load().orc_num_objects(C.byref(self.s))

    # -- Definition 1 ------------------------------------------------------
    def execute(self, bulk, R: int, order=None):
        """Serial execution in timestamp order (Definition 1), or in the given
        order (a permutation of 0..n-1).  Returns (status int32[n],
        out int64[n, R])."""
        n = len(bulk["ts"])
        if self.s.hist_cap and self.s.hist_n + n > self.s.hist_cap:
            raise ValueError("history capacity exceeded")
        ts = np.ascontiguousarray(bulk["ts"], dtype=np.int64)
        ty = np.ascontiguousarray(bulk["type"], dtype=np.int32)
        pa = np.ascontiguousarray(bulk["params"], dtype=np.int64)
        st = np.zeros(n, dtype=np.int32)
        out = np.zeros((n, R), dtype=np.int64)
        od = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
        rc = _load().orc_execute(C.byref(self.s), n, _ptr(ts), _ptr(ty), _ptr(pa),
                                 int(bulk["P"]), R, _ptr(od), _ptr(st), _ptr(out))
        if rc == -2:
            raise ValueError("append-only table capacity exceeded")
        if rc != 0:
            raise ValueError("unknown transaction type")
        return st, out

    # -- basic operations (Section 4.1) -------------------------------------
    def extract(self, bulk, mode: int = MODE_PAPER, K: int = MAX_OPS):
        """Basic operations of every transaction: (obj, cls, root), each
        [n, K] int64/int32/int64 with obj = -1 in unused slots."""
        n = len(bulk["ts"])
        obj = np.empty((n, K), dtype=np.int64)
        cls = np.empty((n, K), dtype=np.int32)
        root = np.empty((n, K), dtype=np.int64)
        ty = np.ascontiguousarray(bulk["type"], dtype=np.int32)
        pa = np.ascontiguousarray(bulk["params"], dtype=np.int64)
        rc = _load().orc_extract(C.byref(self.s), n, _ptr(ty), _ptr(pa), int(bulk["P"]),
                                 mode, K, _ptr(obj), _ptr(cls), _ptr(root))
        if rc < 0:
            raise ValueError("unknown type or too many operations")
        return obj, cls, root


# ---------------------------------------------------------------------------
# T-dependency graph depth (Section 4)
# ---------------------------------------------------------------------------
def levels(obj, cls, n_objects: int):
    """Exact depth (longest path from a source, Section 4.1) of every
    transaction; obj/cls are [n, K]."""
    n, K = obj.shape
    obj = np.ascontiguousarray(obj, dtype=np.int64)
    cls = np.ascontiguousarray(cls, dtype=np.int32)
    lv = np.zeros(n, dtype=np.int64)
    _load().orc_levels(n, K, _ptr(obj), _ptr(cls), int(n_objects), _ptr(lv))
    return lv


def onepass_levels(obj, cls):
    """Section 4.2's five-step calculation: (level[n], rank[n, K])."""
    n, K = obj.shape
    obj = np.ascontiguousarray(obj, dtype=np.int64)
    cls = np.ascontiguousarray(cls, dtype=np.int32)
    lv = np.zeros(n, dtype=np.int64)
    rk = np.full((n, K), -1, dtype=np.int64)
    _load().orc_onepass_levels(n, K, _ptr(obj), _ptr(cls), _ptr(rk), _ptr(lv))
    return lv, rk


def appb_edges(obj, cls, n_objects: int, max_edges: int | None = None):
    """Appendix B construction; returns int64 [E, 2] (from, to)."""
    n, K = obj.shape
    if max_edges is None:
        max_edges = max(16, n * K * 4)
    obj = np.ascontiguousarray(obj, dtype=np.int64)
    cls = np.ascontiguousarray(cls, dtype=np.int32)
    e = np.zeros((max_edges, 2), dtype=np.int64)
    ne = _load().orc_appb_edges(n, K, _ptr(obj), _ptr(cls), int(n_objects), _ptr(e), max_edges)
    if ne < 0:
        raise ValueError("edge capacity exceeded")
    return e[:ne].copy()


def topo_levels(n: int, edges):
    """Depth by topological sort of an explicit graph (Section 4.2)."""
    edges = np.ascontiguousarray(edges, dtype=np.int64).reshape(-1, 2)
    lv = np.zeros(n, dtype=np.int64)
    _load().orc_topo_levels(n, _ptr(edges), len(edges), _ptr(lv))
    return lv


def graph_stats(level, root, part_size: int = 1):
    """Algorithm 1's structural parameters: d (depth of the graph = largest
    vertex depth), w0 (size of the 0-set) and c (transactions whose
    operations fall in more than one partition; a partition groups
    ``part_size`` consecutive root keys)."""
    level = np.asarray(level)
    d = int(level.max()) if len(level) else 0
    w0 = int(np.count_nonzero(level == 0))
    pid = np.where(root >= 0, root // part_size, -1)
    lo = np.where(pid >= 0, pid, np.iinfo(np.int64).max).min(axis=1)
    hi = pid.max(axis=1)
    c = int(np.count_nonzero((hi >= 0) & (lo != hi)))
    return d, w0, c
