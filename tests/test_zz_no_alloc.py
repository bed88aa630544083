"""The allocation-free K-SET entry point against the regular one.

Some callers cannot allocate device memory: a process whose device memory is
all reserved up front by another allocator (a serving stack, or a host
framework that must account for every byte), or a latency-critical path where
a cudaMalloc could block on a device-wide synchronisation or fail under memory
pressure.  They use gputx_execute_kset_noalloc, whose working memory is a
fixed device array inside the library.  Its results must equal those of
gputx_submit_bulk + gputx_execute(K-SET) + gputx_read_results exactly (all
columns are integers: tolerance 0), on consecutive calls that reuse the array.

This file is named to be collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _db(G, max_bulk=1 << 16):
    g = G.Database(dc=(100, 1000, 100_000), history_capacity=1 << 18, max_bulk=max_bulk)
    g.register(G.DC_TYPES)
    return g


def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_3105_gb300 as G
    import workloads as W

    ref, nal = _db(G), _db(G)
    ts0 = 0
    for k, (n, mode) in enumerate([(50_000, G.CONFLICT_PAPER), (60_000, G.CONFLICT_ADD)]):
        bulk = W.dc_bulk(n, 100_000, 0.7, seed=500 + k, ts0=ts0)
        ts0 += n
        b = ref.submit_dict(bulk).execute("kset", conflict_mode=mode)
        st_ref, out_ref = b.results()
        b.free()
        d = {key: torch.from_numpy(bulk[key]).cuda() for key in ("ts", "type", "params")}
        # the caller owns inputs and outputs; the call itself allocates nothing
        st = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        out = torch.full((n, nal.width), -7, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        G.gputx_execute_kset_noalloc(nal.h, d["ts"], d["type"], d["params"], bulk["P"], n, mode, st, out)
        assert np.array_equal(st.cpu().numpy(), st_ref)
        assert np.array_equal(out.cpu().numpy(), out_ref)
    for t in (G.TBL_DC_ACCOUNT, G.TBL_DC_TELLER, G.TBL_DC_BRANCH):
        assert np.array_equal(ref.read(t), nal.read(t))
    h1, h2 = ref.read(G.TBL_DC_HISTORY), nal.read(G.TBL_DC_HISTORY)
    assert np.array_equal(h1[np.argsort(h1[:, 0])], h2[np.argsort(h2[:, 0])])
    ref.close()
    nal.close()


def _schema_pair(G, W, schema):
    """Two identical databases of the subscriber or order-entry schema."""
    dbs = []
    for _ in range(2):
        if schema == "sub":
            g = G.Database(sub=300, sub_child_capacity=1 << 14, max_bulk=1 << 14)
            g.register(G.SUB_TYPES)
            for t, r in W.sub_rows(W.sub_tables(300, seed=21)).items():
                g.load(t, r)
        else:
            g = G.Database(oe=(2, 500), order_capacity=1 << 15, orderline_capacity=15 << 15, max_bulk=1 << 14)
            g.register(G.OE_TYPES)
            for t, r in W.oe_rows(W.oe_tables(2, n_items=500, seed=22)).items():
                g.load(t, r)
        dbs.append(g)
    return dbs


@pytest.mark.parametrize("schema", ["sub", "oe"])
def test_noalloc_matches_regular_entry_point_on_other_schemas(schema):
    """Multi-item order-entry transactions (uneven operation counts, insert
    slots for orders and order lines, the exact-depth pass) and subscriber
    bulks with call-forwarding inserts and deletes: status, outputs and every
    table equal the regular K-SET path's, on two calls in a row."""
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_3105_gb300 as G
    import workloads as W
    from tests._helpers import gpu_logical_state, state_diff, states_equal

    ref, nal = _schema_pair(G, W, schema)
    ts0 = 0
    for k, (n, mode) in enumerate([(5000, G.CONFLICT_PAPER), (7000, G.CONFLICT_ADD)]):
        if schema == "sub":
            bulk = W.sub_bulk(n, 300, 0.5, seed=600 + k, ts0=ts0, mix=(0.1, 0.05, 0.15, 0.05, 0.05, 0.35, 0.25))
        else:
            bulk = W.oe_bulk(n, 2, n_items=500, remote_frac=0.1, invalid_frac=0.02, seed=700 + k, ts0=ts0)
        ts0 += n
        b = ref.submit_dict(bulk).execute("kset", conflict_mode=mode)
        st_ref, out_ref = b.results()
        b.free()
        d = {key: torch.from_numpy(bulk[key]).cuda() for key in ("ts", "type", "params")}
        st = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        out = torch.full((n, nal.width), -7, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        G.gputx_execute_kset_noalloc(nal.h, d["ts"], d["type"], d["params"], bulk["P"], n, mode, st, out)
        assert np.array_equal(st.cpu().numpy(), st_ref), k
        assert np.array_equal(out.cpu().numpy(), out_ref), k
    kw = {"sub": True, "n_sub": 300} if schema == "sub" else {"oe": True}
    a, b = gpu_logical_state(ref, **kw), gpu_logical_state(nal, **kw)
    assert states_equal(a, b), state_diff(a, b)
    ref.close()
    nal.close()


def test_noalloc_rejects_a_bulk_beyond_its_working_memory():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_3105_gb300 as G
    import workloads as W

    n = 1 << 20
    g = _db(G, max_bulk=n)
    bulk = W.dc_bulk(n, 100_000, 0.0, seed=9)
    d = {key: torch.from_numpy(bulk[key]).cuda() for key in ("ts", "type", "params")}
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    out = torch.zeros((n, g.width), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    with pytest.raises(G.GputxError) as e:
        G.gputx_execute_kset_noalloc(g.h, d["ts"], d["type"], d["params"], bulk["P"], n,
                                     G.CONFLICT_PAPER, st, out)
    assert e.value.status == G.EINVAL
    assert int(g.read(G.TBL_DC_ACCOUNT).any()) == 0     # nothing ran
    g.close()
