"""Python binding of the GB300 bulk transaction engine (libgputx.so).

Argument marshalling only: every step of bulk execution runs in the CUDA
library behind the C ABI declared in ``include/gputx.h``.  Functions named
``gputx_*`` mirror the C entry points one to one; ``Database`` and ``Bulk``
are thin conveniences over them.  Importing works without a GPU; any call that
needs the library raises ``GputxError`` if ``libgputx.so`` has not been built
(``__graft_entry__.build()``) -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# GPUTX_DEBUG=1 loads the bounds-checked build (``_build.build(debug=True)``)
LIB_PATH = os.path.join(_HERE, "libgputx_debug.so" if os.environ.get("GPUTX_DEBUG") == "1" else "libgputx.so")

# --- constants mirrored from include/gputx.h --------------------------------
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBOUNDS, ESTATE, ECAPACITY = range(8)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ETIMEOUT", "EBOUNDS", "ESTATE", "ECAPACITY"]
KSET, PART, TPL, AUTO, SCAN, PART_RELAXED, TPL_RELAXED = range(7)
STRATEGIES = {"kset": KSET, "part": PART, "tpl": TPL, "auto": AUTO, "scan": SCAN,
              "part_relaxed": PART_RELAXED, "tpl_relaxed": TPL_RELAXED}
CONFLICT_PAPER, CONFLICT_ADD = 0, 1
MEM_HOST, MEM_DEVICE = 0, 1

(T_DC_DEBIT_CREDIT, T_SUB_GET_SUBSCRIBER, T_SUB_GET_ACCESS, T_SUB_GET_NEW_DEST,
 T_SUB_UPDATE_LOCATION, T_SUB_UPDATE_FACILITY, T_SUB_INSERT_CF, T_SUB_DELETE_CF,
 T_OE_NEW_ORDER, T_OE_PAYMENT, T_OE_ORDER_STATUS) = range(11)
NUM_TYPES = 11
DC_TYPES = (T_DC_DEBIT_CREDIT,)
SUB_TYPES = tuple(range(1, 8))
OE_TYPES = (8, 9, 10)

(TBL_DC_BRANCH, TBL_DC_TELLER, TBL_DC_ACCOUNT, TBL_DC_HISTORY, TBL_SUB_SUBSCRIBER,
 TBL_SUB_ACCESS_INFO, TBL_SUB_SPECIAL_FACILITY, TBL_SUB_CALL_FORWARDING, TBL_OE_WAREHOUSE,
 TBL_OE_DISTRICT, TBL_OE_CUSTOMER, TBL_OE_ITEM, TBL_OE_STOCK, TBL_OE_ORDER,
 TBL_OE_ORDER_LINE) = range(15)
TABLE_FIELDS = (1, 1, 1, 5, 16, 6, 6, 5, 2, 3, 5, 1, 3, 5, 7)

EXPORTED = ("gputx_create_db", "gputx_destroy_db", "gputx_last_error", "gputx_register_types",
            "gputx_load_table", "gputx_read_table", "gputx_read_index", "gputx_read_slots",
            "gputx_submit_bulk", "gputx_execute",
            "gputx_sync_bulk", "gputx_read_results", "gputx_bulk_results_device",
            "gputx_output_width", "gputx_free_bulk", "gputx_version", "gputx_launch_count",
            "gputx_execute_kset_noalloc", "gputx_clock_ns", "gputx_server_create", "gputx_server_submit",
            "gputx_server_results", "gputx_server_drain", "gputx_server_stats",
            "gputx_server_last_error", "gputx_server_destroy", "gputx_batcher_create",
            "gputx_batcher_run", "gputx_batcher_run_bulks", "gputx_batcher_choice", "gputx_batcher_destroy",
            "gputx_pool_create", "gputx_pool_add", "gputx_pool_step", "gputx_pool_results",
            "gputx_pool_pending", "gputx_pool_destroy", "gputx_bulk_order", "gputx_probe_level_chain",
            "gputx_probe_atomics")


class GputxError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class SchemaDesc(C.Structure):
    _fields_ = [("dc_branches", C.c_int64), ("dc_tellers", C.c_int64), ("dc_accounts", C.c_int64),
                ("dc_history_capacity", C.c_int64), ("sub_subscribers", C.c_int64),
                ("sub_child_capacity", C.c_int64), ("oe_warehouses", C.c_int64),
                ("oe_items", C.c_int64), ("oe_order_capacity", C.c_int64),
                ("oe_orderline_capacity", C.c_int64)]


class Config(C.Structure):
    _fields_ = [("max_bulk", C.c_int64), ("block_threads", C.c_int32), ("part_size", C.c_int32),
                ("spin_limit_ns", C.c_int64), ("kset_w0_min", C.c_int64),
                ("part_c_max", C.c_int64), ("part_d_min", C.c_int64)]


class ExecStats(C.Structure):
    _fields_ = [("strategy", C.c_int32), ("fallback", C.c_int32), ("n", C.c_int64),
                ("n_ops", C.c_int64), ("depth", C.c_int64), ("w0", C.c_int64),
                ("cross", C.c_int64), ("fixpoint_rounds", C.c_int64),
                ("ms_h2d", C.c_float), ("ms_analysis", C.c_float), ("ms_sort", C.c_float),
                ("ms_execute", C.c_float), ("ms_d2h", C.c_float), ("ms_total", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServeConfig(C.Structure):
    _fields_ = [("deadline_us", C.c_int64), ("max_bulk", C.c_int64), ("max_inflight", C.c_int32),
                ("strategy", C.c_int32), ("conflict_mode", C.c_int32), ("params_per_txn", C.c_int32),
                ("queue_capacity", C.c_int64), ("min_free_bytes", C.c_int64), ("zero_set", C.c_int32),
                ("reserved", C.c_int32)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("bulks", C.c_int64),
                ("max_bulk_seen", C.c_int64), ("refused", C.c_int64), ("p50_us", C.c_double),
                ("p99_us", C.c_double), ("mean_us", C.c_double), ("txn_per_s", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchConfig(C.Structure):
    _fields_ = [("tune", C.c_int32), ("strategy", C.c_int32), ("block_threads", C.c_int32),
                ("conflict_mode", C.c_int32), ("bulk_size", C.c_int64), ("bulk_size_max", C.c_int64),
                ("params_per_txn", C.c_int32), ("reserved", C.c_int32)]


class BatchChoice(C.Structure):
    _fields_ = [("tuned", C.c_int32), ("strategy", C.c_int32), ("block_threads", C.c_int32),
                ("n_measured", C.c_int32), ("bulk_size", C.c_int64), ("bulks_run", C.c_int64),
                ("measured_strategy", C.c_int32 * 16), ("measured_block", C.c_int32 * 16),
                ("measured_bulk", C.c_int64 * 16), ("measured_ns_per_txn", C.c_double * 16),
                ("p50_us", C.c_double), ("p99_us", C.c_double)]

    def as_dict(self):
        k = self.n_measured
        return {"tuned": bool(self.tuned), "strategy": self.strategy, "block_threads": self.block_threads,
                "bulk_size": self.bulk_size, "bulks_run": self.bulks_run,
                "measured": [{"strategy": self.measured_strategy[i], "block": self.measured_block[i],
                              "bulk": self.measured_bulk[i], "ns_per_txn": self.measured_ns_per_txn[i]}
                             for i in range(k)],
                "p50_us": self.p50_us, "p99_us": self.p99_us}


class PoolConfig(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("params_per_txn", C.c_int32), ("conflict_mode", C.c_int32),
                ("reserved", C.c_int64 * 2)]


class ExecOpts(C.Structure):
    _fields_ = [("conflict_mode", C.c_int32), ("block_threads", C.c_int32),
                ("part_size", C.c_int32), ("timing", C.c_int32), ("kset_launch", C.c_int32),
                ("narrow_max", C.c_int32)]


_lib = None


def signatures() -> dict:
    """ctypes (argument types, result type) of every entry point of
    include/gputx.h, by name."""
    p, sz = C.c_void_p, C.c_size_t
    return {
        "gputx_create_db": ([C.POINTER(SchemaDesc), C.POINTER(Config), p, C.POINTER(p)], C.c_int),
        "gputx_destroy_db": ([p], None),
        "gputx_last_error": ([p], C.c_char_p),
        "gputx_register_types": ([p, p, C.c_int], C.c_int),
        "gputx_load_table": ([p, C.c_int, p, sz], C.c_int),
        "gputx_read_table": ([p, C.c_int, p, sz, C.POINTER(sz)], C.c_int),
        "gputx_read_index": ([p, C.c_int, p, p, sz, C.POINTER(sz)], C.c_int),
        "gputx_read_slots": ([p, C.c_int, p, sz, C.POINTER(sz)], C.c_int),
        "gputx_submit_bulk": ([p, p, p, p, C.c_int, sz, C.c_int, C.POINTER(p)], C.c_int),
        "gputx_execute": ([p, p, C.c_int, C.POINTER(ExecOpts)], C.c_int),
        "gputx_sync_bulk": ([p, C.POINTER(ExecStats)], C.c_int),
        "gputx_read_results": ([p, p, p, sz, C.c_int], C.c_int),
        "gputx_bulk_results_device": ([p, C.POINTER(p), C.POINTER(p)], C.c_int),
        "gputx_bulk_order": ([p, p, sz], C.c_int),
        "gputx_probe_level_chain": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                     C.POINTER(C.c_double)], C.c_int),
        "gputx_probe_atomics": ([C.c_int64, C.c_int, C.POINTER(C.c_double)], C.c_int),
        "gputx_output_width": ([p], C.c_int),
        "gputx_free_bulk": ([p], None),
        "gputx_version": ([], C.c_char_p),
        "gputx_launch_count": ([], C.c_ulonglong),
        "gputx_execute_kset_noalloc": ([p, p, p, p, C.c_int, sz, C.c_int, p, p], C.c_int),
        "gputx_clock_ns": ([], C.c_int64),
        "gputx_server_create": ([p, C.POINTER(ServeConfig), C.POINTER(p)], C.c_int),
        "gputx_server_submit": ([p, p, p, sz, p, C.POINTER(C.c_int64)], C.c_int),
        "gputx_server_results": ([p, C.c_int64, sz, p, p, p, C.POINTER(sz)], C.c_int),
        "gputx_server_drain": ([p], C.c_int),
        "gputx_server_stats": ([p, C.POINTER(ServeStats)], C.c_int),
        "gputx_server_last_error": ([p], C.c_char_p),
        "gputx_server_destroy": ([p], None),
        "gputx_batcher_create": ([p, C.POINTER(BatchConfig), C.POINTER(p)], C.c_int),
        "gputx_batcher_run": ([p, p, p, p, sz, p, p], C.c_int),
        "gputx_batcher_run_bulks": ([p, p, p, p, p, sz, p, p], C.c_int),
        "gputx_batcher_choice": ([p, C.POINTER(BatchChoice)], C.c_int),
        "gputx_batcher_destroy": ([p], None),
        "gputx_pool_create": ([p, C.POINTER(PoolConfig), C.POINTER(p)], C.c_int),
        "gputx_pool_add": ([p, p, p, p, sz], C.c_int),
        "gputx_pool_step": ([p, C.POINTER(sz)], C.c_int),
        "gputx_pool_results": ([p, p, p, p, sz, C.POINTER(sz)], C.c_int),
        "gputx_pool_pending": ([p], sz),
        "gputx_pool_destroy": ([p], None),
    }


def lib():
    """The loaded CUDA library; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GputxError(ECUDA, f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH, mode=C.RTLD_GLOBAL)
        sig = signatures()
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(a):
    """Address of a numpy array, a torch tensor (host or device) or None."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


# --- one-to-one wrappers of the C entry points -------------------------------
def _check(db, st):
    if st != OK:
        msg = lib().gputx_last_error(db).decode() if db else ""
        raise GputxError(st, msg)


def gputx_version() -> str:
    return lib().gputx_version().decode()


def gputx_launch_count() -> int:
    return int(lib().gputx_launch_count())


def gputx_create_db(schema: SchemaDesc, cfg: Config | None = None, stream: int | None = None):
    out = C.c_void_p()
    st = lib().gputx_create_db(C.byref(schema), C.byref(cfg) if cfg else None,
                               C.c_void_p(stream) if stream else None, C.byref(out))
    if st != OK:
        raise GputxError(st, "create_db")
    return out


def gputx_destroy_db(db):
    lib().gputx_destroy_db(db)


def gputx_last_error(db) -> str:
    return lib().gputx_last_error(db).decode()


def gputx_register_types(db, type_ids):
    arr = np.ascontiguousarray(type_ids, dtype=np.int32)
    _check(db, lib().gputx_register_types(db, _ptr(arr), len(arr)))


def gputx_load_table(db, table: int, rows):
    rows = np.ascontiguousarray(rows, dtype=np.int64).reshape(-1, TABLE_FIELDS[table])
    _check(db, lib().gputx_load_table(db, table, _ptr(rows), rows.shape[0]))


def gputx_read_table(db, table: int) -> np.ndarray:
    n = C.c_size_t()
    _check(db, lib().gputx_read_table(db, table, None, 0, C.byref(n)))
    rows = np.zeros((n.value, TABLE_FIELDS[table]), dtype=np.int64)
    _check(db, lib().gputx_read_table(db, table, _ptr(rows), n.value, C.byref(n)))
    return rows[: n.value]


INDEX_ACCESS_INFO, INDEX_SPECIAL_FACILITY, INDEX_CALL_FORWARDING, INDEX_ORDER = range(4)
HKEY_EMPTY, HKEY_TOMB = (1 << 64) - 1, (1 << 64) - 2


def gputx_read_index(db, index: int):
    """(keys uint64[size], rows uint32[size]): the raw open-addressing arrays."""
    n = C.c_size_t()
    _check(db, lib().gputx_read_index(db, index, None, None, 0, C.byref(n)))
    keys = np.zeros(n.value, dtype=np.uint64)
    rows = np.zeros(n.value, dtype=np.uint32)
    _check(db, lib().gputx_read_index(db, index, _ptr(keys), _ptr(rows), n.value, C.byref(n)))
    return keys, rows


def gputx_read_slots(db, table: int) -> np.ndarray:
    """Every storage slot of a child or order table: fields + a live flag."""
    n = C.c_size_t()
    _check(db, lib().gputx_read_slots(db, table, None, 0, C.byref(n)))
    rows = np.zeros((n.value, TABLE_FIELDS[table] + 1), dtype=np.int64)
    _check(db, lib().gputx_read_slots(db, table, _ptr(rows), n.value, C.byref(n)))
    return rows


def gputx_submit_bulk(db, ts, type_, params, params_per_txn: int, n: int, mem: int = MEM_HOST):
    out = C.c_void_p()
    _check(db, lib().gputx_submit_bulk(db, _ptr(ts), _ptr(type_), _ptr(params), params_per_txn,
                                       n, mem, C.byref(out)))
    return out


def gputx_execute(db, bulk, strategy: int, opts: ExecOpts | None = None):
    _check(db, lib().gputx_execute(db, bulk, strategy, C.byref(opts) if opts else None))


def gputx_sync_bulk(db, bulk) -> ExecStats:
    stats = ExecStats()
    _check(db, lib().gputx_sync_bulk(bulk, C.byref(stats)))
    return stats


def gputx_read_results(db, bulk, n: int, width: int, status=None, values=None):
    if status is None:
        status = np.zeros(n, dtype=np.int32)
    if values is None:
        values = np.zeros((n, width), dtype=np.int64)
    _check(db, lib().gputx_read_results(bulk, _ptr(status), _ptr(values), n, width))
    return status, values


def gputx_probe_level_chain(levels: int, cluster_size: int, threads: int, loads: int, stores: int,
                            stores_after: int = 0, rmw: int = 0) -> float:
    """ns per level of the bare level chain (see gputx.h)."""
    ns = C.c_double()
    st = lib().gputx_probe_level_chain(levels, cluster_size, threads, loads, stores, stores_after, rmw,
                                       C.byref(ns))
    if st != OK:
        raise GputxError(st, "probe_level_chain")
    return ns.value


def gputx_probe_atomics(n_cells: int, fetch: int = 0) -> float:
    """G atomic 64-bit additions per second on random cells of a table of
    n_cells (see gputx.h)."""
    g = C.c_double()
    st = lib().gputx_probe_atomics(n_cells, fetch, C.byref(g))
    if st != OK:
        raise GputxError(st, "probe_atomics")
    return g.value


def gputx_bulk_order(db, bulk, n: int) -> np.ndarray:
    order = np.zeros(n, dtype=np.uint32)
    _check(db, lib().gputx_bulk_order(bulk, _ptr(order), n))
    return order


def gputx_bulk_results_device(bulk):
    s, v = C.c_void_p(), C.c_void_p()
    lib().gputx_bulk_results_device(bulk, C.byref(s), C.byref(v))
    return s.value, v.value


def gputx_output_width(db) -> int:
    return lib().gputx_output_width(db)


def gputx_free_bulk(bulk):
    lib().gputx_free_bulk(bulk)


NOALLOC_SCRATCH_BYTES = 48 << 20


def gputx_execute_kset_noalloc(db, ts, type_, params, params_per_txn: int, n: int, conflict_mode: int,
                               status, values):
    """All arrays are CUDA tensors (or device addresses); see gputx.h."""
    _check(db, lib().gputx_execute_kset_noalloc(db, _ptr(ts), _ptr(type_), _ptr(params), params_per_txn,
                                                n, conflict_mode, _ptr(status), _ptr(values)))


# --- conveniences --------------------------------------------------------------
class Bulk:
    def __init__(self, db: "Database", handle, n: int, keep=()):
        self.db, self.h, self.n = db, handle, n
        self._keep = keep   # device inputs referenced in place stay alive

    def execute(self, strategy="kset", conflict_mode=CONFLICT_PAPER, block_threads=0, part_size=0,
                timing=False, kset_launch=0, narrow_max=0):
        s = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        gputx_execute(self.db.h, self.h, s, ExecOpts(conflict_mode, block_threads, part_size, int(timing),
                                                     kset_launch, narrow_max))
        return self

    def sync(self) -> dict:
        return gputx_sync_bulk(self.db.h, self.h).as_dict()

    def results(self, status=None, values=None):
        return gputx_read_results(self.db.h, self.h, self.n, self.db.width, status, values)

    def order(self) -> np.ndarray:
        """A serial order with this bulk's results (timestamp order unless a
        relaxed strategy ran)."""
        return gputx_bulk_order(self.db.h, self.h, self.n)

    def free(self):
        if self.h:
            gputx_free_bulk(self.h)
            self.h = None
            self._keep = ()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Database:
    """A device-resident database of the built-in schemas."""

    def __init__(self, dc=None, sub=None, oe=None, history_capacity=0, sub_child_capacity=0,
                 order_capacity=0, orderline_capacity=0, max_bulk=1 << 22, block_threads=256,
                 part_size=0, spin_limit_ns=0, stream=None, **alg1):
        sch = SchemaDesc()
        if dc is not None:
            sch.dc_branches, sch.dc_tellers, sch.dc_accounts = dc
            sch.dc_history_capacity = history_capacity
        if sub is not None:
            sch.sub_subscribers = sub
            sch.sub_child_capacity = sub_child_capacity
        if oe is not None:
            sch.oe_warehouses, sch.oe_items = oe
            sch.oe_order_capacity = order_capacity
            sch.oe_orderline_capacity = orderline_capacity
        cfg = Config(max_bulk, block_threads, part_size, spin_limit_ns,
                     alg1.get("kset_w0_min", 0), alg1.get("part_c_max", 0), alg1.get("part_d_min", 0))
        self.h = gputx_create_db(sch, cfg, stream)
        self.width = gputx_output_width(self.h)
        # servers, batchers and pools over this database: closed before it
        self._dependents = weakref.WeakSet()

    def _adopt(self, obj):
        self._dependents.add(obj)

    def register(self, types):
        gputx_register_types(self.h, list(types))

    def load(self, table: int, rows):
        gputx_load_table(self.h, table, rows)

    def read(self, table: int) -> np.ndarray:
        return gputx_read_table(self.h, table)

    def read_index(self, index: int):
        return gputx_read_index(self.h, index)

    def read_slots(self, table: int) -> np.ndarray:
        return gputx_read_slots(self.h, table)

    def submit(self, ts, type_, params, mem=None) -> Bulk:
        """Host numpy arrays or CUDA tensors (mem inferred from the first)."""
        n = len(ts)
        if mem is None:
            mem = MEM_DEVICE if getattr(ts, "is_cuda", False) else MEM_HOST
        if mem == MEM_HOST:
            ts = np.ascontiguousarray(ts, dtype=np.int64)
            type_ = np.ascontiguousarray(type_, dtype=np.int32)
            params = np.ascontiguousarray(params, dtype=np.int64)
        P = params.shape[1] if params.ndim == 2 else 1
        h = gputx_submit_bulk(self.h, ts, type_, params, P, n, mem)
        return Bulk(self, h, n, keep=(ts, type_, params) if mem == MEM_DEVICE else ())

    def submit_dict(self, bulk: dict, mem=None) -> Bulk:
        return self.submit(bulk["ts"], bulk["type"], bulk["params"], mem)

    def close(self):
        if self.h:
            for d in list(self._dependents):
                d.close()
            gputx_destroy_db(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- serving -------------------------------------------------------------------
def gputx_clock_ns() -> int:
    return int(lib().gputx_clock_ns())


def _scheck(srv, st):
    if st != OK:
        raise GputxError(st, lib().gputx_server_last_error(srv).decode() if srv else "")


def gputx_server_create(db, cfg: ServeConfig):
    out = C.c_void_p()
    st = lib().gputx_server_create(db, C.byref(cfg), C.byref(out))
    if st != OK:
        raise GputxError(st, "server_create")
    return out


def gputx_server_submit(srv, type_, params, arrival_ns=None) -> int:
    type_ = np.ascontiguousarray(type_, dtype=np.int32)
    params = np.ascontiguousarray(params, dtype=np.int64)
    arr = None if arrival_ns is None else np.ascontiguousarray(arrival_ns, dtype=np.int64)
    first = C.c_int64()
    _scheck(srv, lib().gputx_server_submit(srv, _ptr(type_), _ptr(params), len(type_), _ptr(arr),
                                           C.byref(first)))
    return first.value


def gputx_server_results(srv, first_id: int, n: int, width: int):
    st = np.zeros(n, dtype=np.int32)
    vals = np.zeros((n, width), dtype=np.int64)
    done_ns = np.zeros(n, dtype=np.int64)
    nd = C.c_size_t()
    _scheck(srv, lib().gputx_server_results(srv, first_id, n, _ptr(st), _ptr(vals), _ptr(done_ns),
                                            C.byref(nd)))
    return st, vals, done_ns, nd.value


def gputx_server_drain(srv):
    _scheck(srv, lib().gputx_server_drain(srv))


def gputx_server_stats(srv) -> dict:
    st = ServeStats()
    _scheck(srv, lib().gputx_server_stats(srv, C.byref(st)))
    return st.as_dict()


def gputx_server_destroy(srv):
    lib().gputx_server_destroy(srv)


class Server:
    """Transaction pool + bulk generator over a Database (see gputx.h)."""

    def __init__(self, db: Database, deadline_us=1000, max_bulk=0, max_inflight=2, strategy="kset",
                 conflict_mode=CONFLICT_PAPER, params_per_txn=2, queue_capacity=0, min_free_bytes=0,
                 zero_set=False):
        s = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        cfg = ServeConfig(deadline_us, max_bulk, max_inflight, s, conflict_mode, params_per_txn,
                          queue_capacity, min_free_bytes, int(bool(zero_set)), 0)
        self.db = db
        self.h = gputx_server_create(db.h, cfg)
        db._adopt(self)

    def submit(self, type_, params, arrival_ns=None) -> int:
        return gputx_server_submit(self.h, type_, params, arrival_ns)

    def results(self, first_id, n):
        return gputx_server_results(self.h, first_id, n, self.db.width)

    def drain(self):
        gputx_server_drain(self.h)

    def stats(self) -> dict:
        return gputx_server_stats(self.h)

    def close(self):
        if self.h:
            gputx_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- batched execution through captured graphs -----------------------------------
def gputx_batcher_create(db, cfg: BatchConfig):
    out = C.c_void_p()
    _check(db, lib().gputx_batcher_create(db, C.byref(cfg), C.byref(out)))
    return out


def gputx_batcher_run(db, bt, ts, type_, params, status, values):
    _check(db, lib().gputx_batcher_run(bt, _ptr(ts), _ptr(type_), _ptr(params), len(ts), _ptr(status),
                                       _ptr(values)))


def gputx_batcher_run_bulks(db, bt, ts, type_, params, bulk_off, status, values):
    _check(db, lib().gputx_batcher_run_bulks(bt, _ptr(ts), _ptr(type_), _ptr(params), _ptr(bulk_off),
                                             len(bulk_off) - 1, _ptr(status), _ptr(values)))


def gputx_batcher_choice(bt) -> dict:
    c = BatchChoice()
    lib().gputx_batcher_choice(bt, C.byref(c))
    return c.as_dict()


def gputx_batcher_destroy(bt):
    lib().gputx_batcher_destroy(bt)


class Batcher:
    """Consecutive graph-captured bulks with an optional online autotuner."""

    def __init__(self, db: Database, tune=True, strategy="kset", block_threads=256,
                 conflict_mode=CONFLICT_PAPER, bulk_size=0, bulk_size_max=0, params_per_txn=2):
        s = STRATEGIES[strategy] if isinstance(strategy, str) else int(strategy)
        cfg = BatchConfig(int(tune), s, block_threads, conflict_mode, bulk_size, bulk_size_max,
                          params_per_txn, 0)
        self.db = db
        self.h = gputx_batcher_create(db.h, cfg)
        db._adopt(self)

    def run(self, ts, type_, params):
        ts = np.ascontiguousarray(ts, dtype=np.int64)
        type_ = np.ascontiguousarray(type_, dtype=np.int32)
        params = np.ascontiguousarray(params, dtype=np.int64)
        st = np.zeros(len(ts), dtype=np.int32)
        vals = np.zeros((len(ts), self.db.width), dtype=np.int64)
        gputx_batcher_run(self.db.h, self.h, ts, type_, params, st, vals)
        return st, vals

    def run_bulks(self, ts, type_, params, sizes):
        """A stream of bulks of the given (uneven) sizes, in order."""
        ts = np.ascontiguousarray(ts, dtype=np.int64)
        type_ = np.ascontiguousarray(type_, dtype=np.int32)
        params = np.ascontiguousarray(params, dtype=np.int64)
        off = np.zeros(len(sizes) + 1, dtype=np.int64)
        off[1:] = np.cumsum(np.asarray(sizes, dtype=np.int64))
        st = np.zeros(len(ts), dtype=np.int32)
        vals = np.zeros((len(ts), self.db.width), dtype=np.int64)
        gputx_batcher_run_bulks(self.db.h, self.h, ts, type_, params, off, st, vals)
        return st, vals

    def choice(self) -> dict:
        return gputx_batcher_choice(self.h)

    def close(self):
        if self.h:
            gputx_batcher_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --- incremental 0-set execution (Section 5.3) -------------------------------
def gputx_pool_create(db, cfg: PoolConfig):
    out = C.c_void_p()
    _check(db, lib().gputx_pool_create(db, C.byref(cfg), C.byref(out)))
    return out


def gputx_pool_add(db, pool, ts, type_, params):
    ts = np.ascontiguousarray(ts, dtype=np.int64)
    type_ = np.ascontiguousarray(type_, dtype=np.int32)
    params = np.ascontiguousarray(params, dtype=np.int64)
    _check(db, lib().gputx_pool_add(pool, _ptr(ts), _ptr(type_), _ptr(params), len(ts)))


def gputx_pool_step(db, pool) -> int:
    n = C.c_size_t()
    _check(db, lib().gputx_pool_step(pool, C.byref(n)))
    return n.value


def gputx_pool_results(db, pool, width: int):
    n = C.c_size_t()
    _check(db, lib().gputx_pool_results(pool, None, None, None, 0, C.byref(n)))
    ts = np.zeros(n.value, dtype=np.int64)
    st = np.zeros(n.value, dtype=np.int32)
    vals = np.zeros((n.value, width), dtype=np.int64)
    _check(db, lib().gputx_pool_results(pool, _ptr(ts), _ptr(st), _ptr(vals), n.value, C.byref(n)))
    return ts, st, vals


def gputx_pool_pending(pool) -> int:
    return int(lib().gputx_pool_pending(pool))


def gputx_pool_destroy(pool):
    lib().gputx_pool_destroy(pool)


class Pool:
    """Device-resident transaction pool executed 0-set by 0-set (gputx.h)."""

    def __init__(self, db: Database, capacity: int, params_per_txn: int = 2, conflict_mode=CONFLICT_PAPER):
        self.db = db
        self.h = gputx_pool_create(db.h, PoolConfig(capacity, params_per_txn, conflict_mode))
        db._adopt(self)

    def add(self, ts, type_, params):
        gputx_pool_add(self.db.h, self.h, ts, type_, params)

    def step(self) -> int:
        return gputx_pool_step(self.db.h, self.h)

    def results(self):
        """(ts, status, values) of the last step, in timestamp order."""
        return gputx_pool_results(self.db.h, self.h, self.db.width)

    @property
    def pending(self) -> int:
        return gputx_pool_pending(self.h)

    def close(self):
        if self.h:
            gputx_pool_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
