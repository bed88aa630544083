// batch.cu -- batched execution through captured CUDA graphs, with an online
// autotuner.
//
// A stream of bulks of uneven sizes and mixed types runs in segments: a
// segment is a run of consecutive bulks (at most kSegMax, their total at
// most the segment capacity; a bulk larger than that is cut into pieces)
// that goes through ONE replay of a captured CUDA graph.  The graph holds
// the whole pipeline for a fixed capacity -- extraction, grouping sort,
// ranks, the device-side exact-depth pass, (level, type) regrouping and one
// persistent executor launch -- and reads the segment's bulk boundaries from
// a device descriptor array, so no host synchronisation happens inside it.
// For K-SET every bulk keeps its own dependency graph: the bulk's index sits
// above the object id in the grouping key, each bulk's levels are numbered
// after those of the bulks before it, and the persistent executor walks the
// levels of the whole segment in that order with per-level counters (bulk
// by bulk, level by level).  TPL and PART need no boundary: their order is
// the timestamp order, which runs across bulks.  Shorter segments are padded
// with inactive transactions.
//
// The autotuner runs the stream's own first segments under different
// configurations (every transaction still executes exactly once, in order,
// so the results are unaffected) and keeps the fastest per transaction.  Its
// first guess follows Algorithm 1 (Appendix D) on the structural parameters
// of the first segment: a wide 0-set favours K-SET, otherwise TPL; PART is
// tried when that segment had no cross-partition transaction, and a PART
// segment that turns out to have one runs nothing and is re-run with TPL
// (Section 5.2's fallback, decided on the device).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "engine.h"

namespace {

struct GraphBulk {
    int64_t cap = 0;
    int strategy = GPUTX_KSET, block = 256, mode = 0, P = 0, part_size = 1, slot = 0;
    gputx_bulk *b = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, done = nullptr;
};

// pinned host staging of one segment in flight: inputs copied in by the host,
// results and the control block copied back by the device
struct Staging {
    int64_t cap = 0;
    int P = 0, R = 0;
    int64_t *ts = nullptr, *params = nullptr, *values = nullptr;
    int32_t *type = nullptr, *status = nullptr;
    uint32_t *ctl_words = nullptr;   // n_live, n_seg, seg_off[kSegMax]
    gtx::BulkCtl *ctl = nullptr;
};

struct Candidate {
    int strategy;
    int block;
    int64_t bulk;
    double ns_per_txn;   // measured (0 = not yet)
};

gputx_status fail_bt(gputx_db *db, gputx_status st, const char *msg)
{
    db->last_error = msg;
    return st;
}

#define CKB(call, what)                                                            \
    do {                                                                           \
        cudaError_t e_ = (call);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            db->last_error = std::string(what) + ": " + cudaGetErrorString(e_);    \
            return e_ == cudaErrorMemoryAllocation ? GPUTX_ENOMEM : GPUTX_ECUDA;   \
        }                                                                          \
    } while (0)

// the capturable pipeline of one fixed-capacity bulk (stream = b->stream)
cudaError_t enqueue_pipeline(GraphBulk *g)
{
    gputx_bulk *b = g->b;
    gputx_db *db = b->db;
    const bool add = g->mode == GPUTX_CONFLICT_ADD;
    cudaError_t e;
    if ((e = gtx::launch_insert_slots(b))) return e;
    if ((e = cudaMemsetAsync(&b->ctl->cross, 0, 4, b->stream))) return e;
    if (g->strategy == GPUTX_PART) {
        // partition ids (Section 5.2 step 1); a segment with a
        // cross-partition transaction is flagged and runs nothing
        uint32_t *pk = b->sc.pid_key, *pv = b->sc.pid_val, *pk2 = b->sc.pid_key2, *pv2 = b->sc.pid_val2;
        if ((e = gtx::launch_extract(b, g->mode, g->part_size, pk, pv, false))) return e;
        if ((e = gtx::launch_part_fallback_check(b))) return e;
        const int64_t roots = std::max<int64_t>({db->dev.n_br, db->dev.n_sub, db->dev.n_wh, 1});
        const int64_t parts = (roots + g->part_size - 1) / g->part_size;   // the padding's id
        if ((e = gtx::launch_sort(b, pk, pv, pk2, pv2, b->n, gtx::bits_for((uint64_t)parts)))) return e;
        if ((e = gtx::launch_part_heads(b, pk, b->n))) return e;
        if (gtx::part_dc_applies(db, g->part_size)) e = gtx::launch_gather_dc(b, pv);
        else e = gtx::launch_gather(b, pv);
        if (e) return e;
        if ((e = gtx::launch_begin(b))) return e;
        if ((e = gtx::launch_part(b, pk, 128, parts, g->part_size))) return e;
        return gtx::launch_finish(b);
    }
    const bool seg = g->strategy == GPUTX_KSET && gtx::seg_bits(db) > 0;
    if (seg && (e = gtx::launch_seg_index(b))) return e;
    if ((e = gtx::launch_extract(b, g->mode, 1, nullptr, nullptr, true, seg))) return e;
    const int64_t m = b->n * db->kmax;
    uint32_t *sk = b->sc.keys_a, *sv = b->sc.vals_a, *ak = b->sc.keys_b, *av = b->sc.vals_b;
    const int kbits = db->obj_bits + (seg ? gtx::seg_bits(db) : 0);
    if ((e = gtx::launch_sort(b, sk, sv, ak, av, m, kbits))) return e;
    if (g->strategy == GPUTX_KSET) {
        if ((e = gtx::launch_rank_scan(b, sk, sv, m, db->need_fixpoint))) return e;
        if (db->need_fixpoint && (e = gtx::launch_exact_depth(b, sv, m))) return e;
        if ((e = gtx::launch_level_stats(b))) return e;
        if (seg && (e = gtx::launch_seg_levels(b))) return e;
        uint32_t *rk = ak, *rv = av, *rk2 = sk, *rv2 = sv;
        if ((e = gtx::launch_regroup_keys(b, rk, rv))) return e;
        // global levels < capacity, and the padding key is the capacity itself
        if ((e = gtx::launch_sort(b, rk, rv, rk2, rv2, b->n, gtx::bits_for((uint64_t)b->n) + db->tbits))) return e;
        if ((e = gtx::launch_level_tables(b, rk, 0, g->block, true))) return e;
        if ((e = gtx::launch_gather(b, rv))) return e;
        if ((e = gtx::launch_begin(b))) return e;
        if ((e = gtx::launch_kset(b, rv, b->sc.chunk_cap, g->block, add))) return e;
    } else {
        if ((e = gtx::launch_ticket_scan(b, sk, sv, m))) return e;
        if ((e = gtx::launch_begin(b))) return e;
        if ((e = gtx::launch_tpl(b, g->block, add))) return e;
        if ((e = gtx::launch_tpl_reset(b, sk, m))) return e;
    }
    return gtx::launch_finish(b);
}

}  // namespace

size_t gtx_carve_bulk(gputx_bulk *b, char *base, bool device_inputs);   // api.cu

struct gputx_batcher {
    gputx_db *db = nullptr;
    gputx_batch_config cfg{};
    std::vector<GraphBulk *> graphs;
    std::vector<Candidate> cands;
    size_t next_cand = 0;
    bool tuned = false;
    bool part_ok = false;              // the first segment had no cross-partition transaction
    Candidate best{GPUTX_KSET, 256, 1 << 16, 0};
    int64_t bulks_run = 0;             // segments (graph replays) run
    int part_size = 1;
    // per-transaction latency of the last run call: (transactions, ms from
    // the call's start to their segment's results on the host)
    std::vector<std::pair<double, int64_t>> lat;
    Staging stage[2];                  // double buffer: one segment runs while the next is staged
};

namespace {

void free_staging(Staging &st)
{
    cudaFreeHost(st.ts);
    cudaFreeHost(st.params);
    cudaFreeHost(st.values);
    cudaFreeHost(st.type);
    cudaFreeHost(st.status);
    cudaFreeHost(st.ctl_words);
    cudaFreeHost(st.ctl);
    st = Staging{};
}

// pinned buffers for segments of up to cap transactions
gputx_status ensure_staging(gputx_batcher *bt, Staging &st, int64_t cap)
{
    gputx_db *db = bt->db;
    const int P = bt->cfg.params_per_txn, R = db->dev.out_width;
    if (st.cap >= cap && st.P == P && st.R == R) return GPUTX_OK;
    free_staging(st);
    CKB(cudaMallocHost(&st.ts, sizeof(int64_t) * cap), "staging");
    CKB(cudaMallocHost(&st.params, sizeof(int64_t) * cap * P), "staging");
    CKB(cudaMallocHost(&st.values, sizeof(int64_t) * cap * R), "staging");
    CKB(cudaMallocHost(&st.type, sizeof(int32_t) * cap), "staging");
    CKB(cudaMallocHost(&st.status, sizeof(int32_t) * cap), "staging");
    CKB(cudaMallocHost(&st.ctl_words, sizeof(uint32_t) * (gtx::kSegMax + 2)), "staging");
    CKB(cudaMallocHost(&st.ctl, sizeof(gtx::BulkCtl)), "staging");
    st.cap = cap;
    st.P = P;
    st.R = R;
    return GPUTX_OK;
}

void destroy_graph(GraphBulk *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->e0) cudaEventDestroy(g->e0);
    if (g->e1) cudaEventDestroy(g->e1);
    if (g->done) cudaEventDestroy(g->done);
    if (g->b) gputx_free_bulk(g->b);
    delete g;
}

// the fixed-capacity bulk and captured graph for a shape (created on first use)
gputx_status get_graph(gputx_batcher *bt, int64_t cap, int strategy, int block, int slot, GraphBulk **out)
{
    gputx_db *db = bt->db;
    for (GraphBulk *g : bt->graphs)
        if (g->cap == cap && g->strategy == strategy && g->block == block && g->slot == slot) {
            *out = g;
            return GPUTX_OK;
        }
    GraphBulk *g = new GraphBulk();
    g->cap = cap;
    g->strategy = strategy;
    g->block = block;
    g->slot = slot;
    g->mode = bt->cfg.conflict_mode;
    g->P = bt->cfg.params_per_txn;
    g->part_size = bt->part_size;
    gputx_bulk *b = new gputx_bulk();
    g->b = b;
    b->db = db;
    b->n = cap;
    b->P = g->P;
    b->R = db->dev.out_width;
    b->graph = true;
    b->stream = db->pool[db->next_pool];
    db->next_pool = (db->next_pool + 1) % gputx_db::kPool;
    b->arena_bytes = gtx_carve_bulk(b, nullptr, false);
    CKB(cudaMallocAsync(&b->arena, b->arena_bytes, b->stream), "batch bulk allocation");
    CKB(cudaStreamSynchronize(b->stream), "batch bulk allocation");
    gtx_carve_bulk(b, (char *)b->arena, false);
    CKB(cudaEventCreate(&b->ev[7]), "event");
    CKB(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming), "event");
    CKB(cudaEventCreate(&g->e0), "event");
    CKB(cudaEventCreate(&g->e1), "event");
    CKB(cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming), "event");
    b->executed = true;
    // one uncaptured run sets up per-kernel attributes; its inputs are all
    // padding, so it changes nothing
    CKB(cudaMemsetAsync(b->ctl, 0, sizeof(gtx::BulkCtl), b->stream), "init");
    CKB(cudaMemsetAsync(b->type, 0xff, sizeof(int32_t) * cap, b->stream), "init");
    CKB(cudaMemsetAsync(b->params, 0, sizeof(int64_t) * cap * g->P, b->stream), "init");
    CKB(cudaMemsetAsync(b->ts, 0, sizeof(int64_t) * cap, b->stream), "init");
    CKB(cudaMemsetAsync(b->sc.seg_off, 0, sizeof(uint32_t) * (gtx::kSegMax + 1), b->stream), "init");
    CKB(cudaStreamWaitEvent(b->stream, db->last_done, 0), "order");
    CKB(enqueue_pipeline(g), "warm-up");
    CKB(cudaStreamSynchronize(b->stream), "warm-up");
    cudaGraph_t graph = nullptr;
    CKB(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "capture");
    cudaError_t ce = enqueue_pipeline(g);
    cudaError_t ee = cudaStreamEndCapture(b->stream, &graph);
    if (ce || ee) {
        if (graph) cudaGraphDestroy(graph);
        destroy_graph(g);
        db->last_error = std::string("capture: ") + cudaGetErrorString(ce ? ce : ee);
        return GPUTX_ECUDA;
    }
    cudaError_t ie = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie) {
        destroy_graph(g);
        return fail_bt(db, GPUTX_ECUDA, "graph instantiate failed");
    }
    bt->graphs.push_back(g);
    *out = g;
    return GPUTX_OK;
}

// One segment of n <= cap transactions through a graph: n_seg bulks whose
// first transactions (relative to the segment) are seg_off[0..n_seg-1].  The
// host copies the inputs into the pinned staging `st`; the device copies them
// in, replays the graph and copies the results and the control block back
// into `st`, then records g->done.  Nothing here waits for the device.
gputx_status enqueue_segment(gputx_batcher *bt, GraphBulk *g, Staging &st, const int64_t *ts, const int32_t *type,
                             const int64_t *params, int64_t n, const uint32_t *seg_off, uint32_t n_seg)
{
    gputx_db *db = bt->db;
    gputx_bulk *b = g->b;
    cudaStream_t s = b->stream;
    const int64_t cap = g->cap;
    std::memcpy(st.ts, ts, sizeof(int64_t) * n);
    std::memcpy(st.type, type, sizeof(int32_t) * n);
    std::memcpy(st.params, params, sizeof(int64_t) * n * g->P);
    st.ctl_words[0] = (uint32_t)n;
    st.ctl_words[1] = n_seg;
    std::memcpy(st.ctl_words + 2, seg_off, sizeof(uint32_t) * n_seg);
    // earlier work on the database stream (loads, other bulks) comes first
    CKB(cudaEventRecord(b->ev_in, db->stream), "order");
    CKB(cudaStreamWaitEvent(s, b->ev_in, 0), "order");
    CKB(cudaStreamWaitEvent(s, db->last_done, 0), "order");
    CKB(cudaMemsetAsync(b->ctl, 0, sizeof(gtx::BulkCtl), s), "reset");
    CKB(cudaMemcpyAsync(&b->ctl->n_live, &st.ctl_words[0], sizeof(uint32_t), cudaMemcpyHostToDevice, s), "inputs");
    CKB(cudaMemcpyAsync(&b->ctl->n_seg, &st.ctl_words[1], sizeof(uint32_t), cudaMemcpyHostToDevice, s), "inputs");
    CKB(cudaMemcpyAsync(b->sc.seg_off, st.ctl_words + 2, sizeof(uint32_t) * n_seg, cudaMemcpyHostToDevice, s),
        "inputs");
    CKB(cudaMemcpyAsync(b->ts, st.ts, sizeof(int64_t) * n, cudaMemcpyHostToDevice, s), "inputs");
    CKB(cudaMemcpyAsync(b->type, st.type, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s), "inputs");
    CKB(cudaMemcpyAsync(b->params, st.params, sizeof(int64_t) * n * g->P, cudaMemcpyHostToDevice, s), "inputs");
    if (n < cap) CKB(cudaMemsetAsync(b->type + n, 0xff, sizeof(int32_t) * (cap - n), s), "inputs");
    CKB(cudaMemsetAsync(b->out, 0, sizeof(int64_t) * cap * b->R, s), "inputs");
    CKB(cudaEventRecord(g->e0, s), "event");
    CKB(cudaGraphLaunch(g->exec, s), "graph launch");
    CKB(cudaEventRecord(g->e1, s), "event");
    CKB(cudaEventRecord(db->last_done, s), "order");
    CKB(cudaStreamWaitEvent(db->stream, db->last_done, 0), "order");
    CKB(cudaMemcpyAsync(st.status, b->status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s), "results");
    CKB(cudaMemcpyAsync(st.values, b->out, sizeof(int64_t) * n * b->R, cudaMemcpyDeviceToHost, s), "results");
    CKB(cudaMemcpyAsync(st.ctl, b->ctl, sizeof(gtx::BulkCtl), cudaMemcpyDeviceToHost, s), "results");
    CKB(cudaEventRecord(g->done, s), "event");
    return GPUTX_OK;
}

// Waits for a segment enqueued by enqueue_segment, copies its results to the
// caller's arrays and returns its device time.  *fallback is set when a PART
// segment held a cross-partition transaction (nothing ran).
gputx_status finish_segment(gputx_batcher *bt, GraphBulk *g, Staging &st, int64_t n, int32_t *status,
                            int64_t *values, double *ms, gtx::BulkCtl *ctl_out, bool *fallback)
{
    gputx_db *db = bt->db;
    *fallback = false;
    CKB(cudaEventSynchronize(g->done), "results");
    float t = 0;
    cudaEventElapsedTime(&t, g->e0, g->e1);
    *ms = t;
    const gtx::BulkCtl ctl = *st.ctl;
    if (ctl_out) *ctl_out = ctl;
    if (ctl.err == gtx::ERR_FALLBACK) {
        *fallback = true;
        return GPUTX_OK;
    }
    if (ctl.err & gtx::ERR_INVAL) return fail_bt(db, GPUTX_EINVAL, "invalid bulk contents");
    if (ctl.err & gtx::ERR_TIMEOUT) return fail_bt(db, GPUTX_ETIMEOUT, "a bounded device wait ran out");
    if (ctl.err & gtx::ERR_CAPACITY) return fail_bt(db, GPUTX_ECAPACITY, "an insert area is full");
    if (ctl.err) return fail_bt(db, GPUTX_EBOUNDS, "device bounds check failed");
    std::memcpy(status, st.status, sizeof(int32_t) * n);
    std::memcpy(values, st.values, sizeof(int64_t) * n * st.R);
    return GPUTX_OK;
}

void plan_candidates(gputx_batcher *bt, int first_strategy)
{
    bt->cands.clear();
    for (int64_t sz : {int64_t(1) << 14, int64_t(1) << 16, int64_t(1) << 18, int64_t(1) << 20})
        if (sz <= bt->cfg.bulk_size_max) bt->cands.push_back({first_strategy, 256, sz, 0});
    if (bt->cands.empty()) bt->cands.push_back({first_strategy, 256, bt->cfg.bulk_size_max, 0});
    // block shapes and the other strategies are tried at the best size found
    // so far (filled in when the sizes are measured)
}

// The next segment of the caller's bulks: starting at bulk `bi`, offset
// `off` into it, consecutive bulks (pieces of at most cap) until cap
// transactions or `seg_limit` bulks.  Fills seg_off (relative starts) and
// returns the segment's transaction count; advances bi/off.
int64_t next_segment(const int64_t *bulk_off, size_t n_bulks, size_t &bi, int64_t &off, int64_t cap, int seg_limit,
                     std::vector<uint32_t> &seg_off)
{
    seg_off.clear();
    int64_t total = 0;
    while (bi < n_bulks && (int)seg_off.size() < seg_limit && total < cap) {
        const int64_t left = bulk_off[bi + 1] - bulk_off[bi] - off;
        if (left <= 0) {   // an empty bulk (or a finished one)
            bi++;
            off = 0;
            continue;
        }
        const int64_t take = std::min<int64_t>(left, cap - total);
        seg_off.push_back((uint32_t)total);
        total += take;
        off += take;
        if (off >= bulk_off[bi + 1] - bulk_off[bi]) {
            bi++;
            off = 0;
        }
    }
    return total;
}

}  // namespace

extern "C" {

gputx_status gputx_batcher_create(gputx_db *db, const gputx_batch_config *cfg, gputx_batcher **out)
{
    if (!db || !out) return GPUTX_EINVAL;
    *out = nullptr;
    if (!db->dev.registered) return GPUTX_ESTATE;
    gputx_batcher *bt = new gputx_batcher();
    bt->db = db;
    if (cfg) bt->cfg = *cfg;
    gputx_batch_config &c = bt->cfg;
    if (c.params_per_txn <= 0) c.params_per_txn = 2;
    if (c.bulk_size_max <= 0 || c.bulk_size_max > db->cfg.max_bulk) c.bulk_size_max = db->cfg.max_bulk;
    if (c.bulk_size <= 0 || c.bulk_size > c.bulk_size_max) c.bulk_size = std::min<int64_t>(1 << 16, c.bulk_size_max);
    if (c.block_threads <= 0) c.block_threads = 256;
    if (c.strategy != GPUTX_KSET && c.strategy != GPUTX_TPL && c.strategy != GPUTX_PART) c.strategy = GPUTX_KSET;
    bt->part_size = db->cfg.part_size > 0 ? db->cfg.part_size
                                          : ((db->dev.n_sub > 0 && db->dev.n_acc == 0 && db->dev.n_wh == 0) ? 128 : 1);
    bt->best = {c.strategy, c.block_threads, c.bulk_size, 0};
    bt->tuned = !c.tune;
    *out = bt;
    return GPUTX_OK;
}

gputx_status gputx_batcher_run_bulks(gputx_batcher *bt, const int64_t *ts, const int32_t *type,
                                     const int64_t *params, const int64_t *bulk_off, size_t n_bulks,
                                     int32_t *status, int64_t *values)
{
    if (!bt || (n_bulks && !bulk_off)) return GPUTX_EINVAL;
    gputx_db *db = bt->db;
    const size_t n = n_bulks ? (size_t)bulk_off[n_bulks] : 0;
    if (n && (!ts || !type || !params || !status || !values)) return fail_bt(db, GPUTX_EINVAL, "null array");
    if (n_bulks && bulk_off[0] != 0) return fail_bt(db, GPUTX_EINVAL, "bulk_off[0] must be 0");
    for (size_t k = 0; k < n_bulks; k++)
        if (bulk_off[k + 1] < bulk_off[k]) return fail_bt(db, GPUTX_EINVAL, "bulk offsets must not decrease");
    const int P = bt->cfg.params_per_txn, R = db->dev.out_width;
    // bulks in one segment: the bulk index must fit above the object id
    const int sb = gtx::seg_bits(db);
    const int seg_kset = sb > 0 ? std::min(gtx::kSegMax, (1 << sb) - 1) : 1;
    const auto t_start = std::chrono::steady_clock::now();
    bt->lat.clear();
    // a segment enqueued and not yet finished
    struct InFlight {
        bool valid = false, first = false;
        GraphBulk *g = nullptr;
        int buf = 0, strategy = GPUTX_KSET, block = 256;
        int64_t first_txn = 0, k = 0, size = 0;
        Candidate *cand = nullptr;
        std::vector<uint32_t> seg_off;
    };
    auto finish = [&](InFlight &f) -> gputx_status {
        f.valid = false;
        double ms = 0;
        gtx::BulkCtl ctl{};
        bool fb = false;
        Staging &stg = bt->stage[f.buf];
        gputx_status st = finish_segment(bt, f.g, stg, f.k, status + f.first_txn, values + f.first_txn * R, &ms, &ctl,
                                         &fb);
        if (st) return st;
        if (fb) {
            // Section 5.2: a PART segment with a cross-partition transaction
            // runs with TPL (nothing of it ran)
            GraphBulk *gt = nullptr;
            if ((st = get_graph(bt, f.size, GPUTX_TPL, f.block, f.g->slot, &gt))) return st;
            if ((st = enqueue_segment(bt, gt, stg, ts + f.first_txn, type + f.first_txn, params + f.first_txn * P, f.k,
                                      f.seg_off.data(), (uint32_t)f.seg_off.size())))
                return st;
            double ms2 = 0;
            if ((st = finish_segment(bt, gt, stg, f.k, status + f.first_txn, values + f.first_txn * R, &ms2, nullptr,
                                     &fb)))
                return st;
            ms += ms2;
        }
        bt->lat.push_back(
            {std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count(), f.k});
        if (f.first) {
            const bool wide = (int64_t)ctl.w0 >= std::min<int64_t>(db->cfg.kset_w0_min, f.k / 4);
            bt->part_ok = ctl.cross == 0;
            plan_candidates(bt, wide ? GPUTX_KSET : GPUTX_TPL);
        } else if (f.cand) {
            // a short segment is padded: charge it at least half its capacity
            f.cand->ns_per_txn = ms * 1e6 / (double)std::max<int64_t>(f.k, f.size / 2);
            bt->next_cand++;
        }
        bt->bulks_run++;
        return GPUTX_OK;
    };
    InFlight prev;
    int buf = 0;
    size_t bi = 0;
    int64_t boff = 0;
    std::vector<uint32_t> seg_off;
    gputx_status st = GPUTX_OK;
    while (bi < n_bulks) {
        Candidate *cand = nullptr;
        int strategy, block;
        int64_t size;
        bool first = false;
        if (!bt->tuned && bt->cands.empty()) {
            // first segment: K-SET at 2^16 gives d, w0, c; Algorithm 1 orders
            // the strategies to try
            strategy = GPUTX_KSET;
            block = 256;
            size = std::min<int64_t>(1 << 16, bt->cfg.bulk_size_max);
            first = true;
        } else {
            if (!bt->tuned) {
                if (bt->next_cand >= bt->cands.size()) {
                    // the sizes are measured: then block shapes and the other
                    // strategies at the best size, once each
                    auto best = std::min_element(bt->cands.begin(), bt->cands.end(),
                                                 [](const Candidate &a, const Candidate &b) {
                                                     return a.ns_per_txn < b.ns_per_txn;
                                                 });
                    const Candidate bc = *best;
                    const size_t before = bt->cands.size();
                    auto have = [&](int s_, int blk, int64_t sz) {
                        for (auto &c : bt->cands)
                            if (c.strategy == s_ && c.block == blk && c.bulk == sz) return true;
                        return false;
                    };
                    for (int blk : {128, 512})
                        if (!have(bc.strategy, blk, bc.bulk)) bt->cands.push_back({bc.strategy, blk, bc.bulk, 0});
                    for (int other : {GPUTX_KSET, GPUTX_TPL, GPUTX_PART}) {
                        if (other == GPUTX_PART && !bt->part_ok) continue;
                        if (other != bc.strategy && !have(other, 256, bc.bulk))
                            bt->cands.push_back({other, 256, bc.bulk, 0});
                    }
                    if (bt->cands.size() == before) {
                        bt->best = bc;
                        bt->tuned = true;
                    }
                }
                if (!bt->tuned) cand = &bt->cands[bt->next_cand];
            }
            strategy = cand ? cand->strategy : bt->best.strategy;
            block = cand ? cand->block : bt->best.block;
            size = cand ? cand->bulk : bt->best.bulk;
        }
        // tuning segments and PART segments (whose fallback must run before
        // any later segment) complete before the next is enqueued; a tuned
        // K-SET or TPL stream keeps two segments in flight, so the host's
        // copies of one overlap the other's execution
        const bool sync = !bt->tuned || strategy == GPUTX_PART;
        const int first_limit = strategy == GPUTX_KSET ? seg_kset : gtx::kSegMax;
        const int64_t first_txn = bulk_off[bi] + boff;
        const int64_t k = next_segment(bulk_off, n_bulks, bi, boff, size, first_limit, seg_off);
        if (k == 0) continue;   // only empty bulks were left
        GraphBulk *g = nullptr;
        if ((st = get_graph(bt, size, strategy, block, sync ? 0 : buf, &g))) break;
        if ((st = ensure_staging(bt, bt->stage[buf], size))) break;
        if ((st = enqueue_segment(bt, g, bt->stage[buf], ts + first_txn, type + first_txn, params + first_txn * P, k,
                                  seg_off.data(), (uint32_t)seg_off.size())))
            break;
        InFlight cur;
        cur.valid = true;
        cur.first = first;
        cur.g = g;
        cur.buf = buf;
        cur.strategy = strategy;
        cur.block = block;
        cur.first_txn = first_txn;
        cur.k = k;
        cur.size = size;
        cur.cand = cand;
        cur.seg_off = seg_off;
        if (prev.valid && (st = finish(prev))) {
            cudaEventSynchronize(g->done);   // nothing left in flight
            return st;
        }
        if (sync) {
            if ((st = finish(cur))) return st;
        } else {
            prev = cur;
        }
        buf ^= 1;
    }
    if (prev.valid) {
        gputx_status st2 = finish(prev);
        if (!st) st = st2;
    }
    return st;
}

gputx_status gputx_batcher_run(gputx_batcher *bt, const int64_t *ts, const int32_t *type, const int64_t *params,
                               size_t n, int32_t *status, int64_t *values)
{
    if (!bt || (n && (!ts || !type || !params || !status || !values))) return GPUTX_EINVAL;
    const int64_t off[2] = {0, (int64_t)n};   // one bulk: cut into segments of the tuned capacity
    return gputx_batcher_run_bulks(bt, ts, type, params, off, n ? 1 : 0, status, values);
}

gputx_status gputx_batcher_choice(const gputx_batcher *bt, gputx_batch_choice *out)
{
    if (!bt || !out) return GPUTX_EINVAL;
    std::memset(out, 0, sizeof *out);
    out->tuned = bt->tuned;
    Candidate cur = bt->best;
    if (!bt->tuned) {   // still tuning: the fastest measured so far
        double best_ns = 0;
        for (const Candidate &c : bt->cands)
            if (c.ns_per_txn > 0 && (best_ns == 0 || c.ns_per_txn < best_ns)) {
                best_ns = c.ns_per_txn;
                cur = c;
            }
    }
    out->strategy = cur.strategy;
    out->block_threads = cur.block;
    out->bulk_size = cur.bulk;
    out->bulks_run = bt->bulks_run;
    out->n_measured = 0;
    for (const Candidate &c : bt->cands) {
        if (out->n_measured >= 16) break;
        if (c.ns_per_txn <= 0) continue;
        out->measured_strategy[out->n_measured] = c.strategy;
        out->measured_block[out->n_measured] = c.block;
        out->measured_bulk[out->n_measured] = c.bulk;
        out->measured_ns_per_txn[out->n_measured] = c.ns_per_txn;
        out->n_measured++;
    }
    // per-transaction latency of the last run call
    std::vector<std::pair<double, int64_t>> v = bt->lat;
    std::sort(v.begin(), v.end());
    int64_t total = 0;
    for (auto &x : v) total += x.second;
    auto pct = [&](double q) {
        const int64_t want = (int64_t)(q * (double)total);
        int64_t acc = 0;
        for (auto &x : v) {
            acc += x.second;
            if (acc > want) return x.first * 1e3;
        }
        return v.empty() ? 0.0 : v.back().first * 1e3;
    };
    out->p50_us = pct(0.50);
    out->p99_us = pct(0.99);
    return GPUTX_OK;
}

void gputx_batcher_destroy(gputx_batcher *bt)
{
    if (!bt) return;
    for (GraphBulk *g : bt->graphs) destroy_graph(g);
    for (Staging &st : bt->stage) free_staging(st);
    delete bt;
}

}  // extern "C"
