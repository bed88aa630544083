// batch.cu -- batched execution through captured CUDA graphs, with an online
// autotuner.
//
// A stream of transactions (uneven sizes, mixed types) runs as consecutive
// bulks of a chosen size.  Each bulk size, strategy and block shape has one
// fixed-capacity bulk whose whole pipeline -- extraction, grouping sort,
// ranks, device-side refinement rounds, (level, type) regrouping, and one
// persistent K-SET launch (or the TPL kernel) -- is captured once in a CUDA
// graph and replayed for every bulk of that shape: no host synchronisation
// inside the pipeline, one graph launch per bulk.  Bulks shorter than the
// capacity are padded with inactive transactions.
//
// The autotuner runs the stream's own first bulks under different
// configurations (every bulk still executes exactly once, in order, so the
// results are unaffected) and keeps the fastest per transaction.  Its first
// guess follows Algorithm 1 (Appendix D) on the structural parameters of the
// first bulk: a wide 0-set favours K-SET, otherwise TPL.
#include <algorithm>
#include <cstring>
#include <vector>

#include "engine.h"

namespace {

struct GraphBulk {
    int64_t cap = 0;
    int strategy = GPUTX_KSET, block = 256, mode = 0, P = 0;
    gputx_bulk *b = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
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
    if ((e = gtx::launch_extract(b, g->mode, 1, nullptr, nullptr, true))) return e;
    const int64_t m = b->n * db->kmax;
    uint32_t *sk = b->sc.keys_a, *sv = b->sc.vals_a, *ak = b->sc.keys_b, *av = b->sc.vals_b;
    if ((e = gtx::launch_sort(b, sk, sv, ak, av, m, db->obj_bits))) return e;
    if (g->strategy == GPUTX_KSET) {
        if ((e = gtx::launch_rank_scan(b, sk, sv, m, db->need_fixpoint))) return e;
        if (db->need_fixpoint && (e = gtx::launch_fixpoint_device(b, sv, m))) return e;
        if ((e = gtx::launch_level_stats(b))) return e;
        uint32_t *rk = ak, *rv = av, *rk2 = sk, *rv2 = sv;
        if ((e = gtx::launch_regroup_keys(b, rk, rv))) return e;
        // depth < capacity, and the padding key is the capacity itself
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
    Candidate best{GPUTX_KSET, 256, 1 << 16, 0};
    int64_t bulks_run = 0;
};

namespace {

void destroy_graph(GraphBulk *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->e0) cudaEventDestroy(g->e0);
    if (g->e1) cudaEventDestroy(g->e1);
    if (g->b) gputx_free_bulk(g->b);
    delete g;
}

// the fixed-capacity bulk and captured graph for a shape (created on first use)
gputx_status get_graph(gputx_batcher *bt, int64_t cap, int strategy, int block, GraphBulk **out)
{
    gputx_db *db = bt->db;
    for (GraphBulk *g : bt->graphs)
        if (g->cap == cap && g->strategy == strategy && g->block == block) {
            *out = g;
            return GPUTX_OK;
        }
    GraphBulk *g = new GraphBulk();
    g->cap = cap;
    g->strategy = strategy;
    g->block = block;
    g->mode = bt->cfg.conflict_mode;
    g->P = bt->cfg.params_per_txn;
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
    b->executed = true;
    // one uncaptured run sets up per-kernel attributes; its inputs are all
    // padding, so it changes nothing
    CKB(cudaMemsetAsync(b->ctl, 0, sizeof(gtx::BulkCtl), b->stream), "init");
    CKB(cudaMemsetAsync(b->type, 0xff, sizeof(int32_t) * cap, b->stream), "init");
    CKB(cudaMemsetAsync(b->params, 0, sizeof(int64_t) * cap * g->P, b->stream), "init");
    CKB(cudaMemsetAsync(b->ts, 0, sizeof(int64_t) * cap, b->stream), "init");
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

// one bulk of n <= cap transactions through a graph; returns its time
gputx_status run_bulk(gputx_batcher *bt, GraphBulk *g, const int64_t *ts, const int32_t *type,
                      const int64_t *params, int64_t n, int32_t *status, int64_t *values, double *ms,
                      gtx::BulkCtl *ctl_out)
{
    gputx_db *db = bt->db;
    gputx_bulk *b = g->b;
    cudaStream_t s = b->stream;
    const int64_t cap = g->cap;
    // earlier work on the database stream (loads, other bulks) comes first
    CKB(cudaEventRecord(b->ev_in, db->stream), "order");
    CKB(cudaStreamWaitEvent(s, b->ev_in, 0), "order");
    CKB(cudaStreamWaitEvent(s, db->last_done, 0), "order");
    CKB(cudaMemsetAsync(b->ctl, 0, sizeof(gtx::BulkCtl), s), "reset");
    const uint32_t nl = (uint32_t)n;
    CKB(cudaMemcpyAsync(&b->ctl->n_live, &nl, sizeof nl, cudaMemcpyHostToDevice, s), "inputs");
    CKB(cudaMemcpyAsync(b->ts, ts, sizeof(int64_t) * n, cudaMemcpyHostToDevice, s), "inputs");
    CKB(cudaMemcpyAsync(b->type, type, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s), "inputs");
    CKB(cudaMemcpyAsync(b->params, params, sizeof(int64_t) * n * g->P, cudaMemcpyHostToDevice, s), "inputs");
    if (n < cap) CKB(cudaMemsetAsync(b->type + n, 0xff, sizeof(int32_t) * (cap - n), s), "inputs");
    CKB(cudaMemsetAsync(b->out, 0, sizeof(int64_t) * cap * b->R, s), "inputs");
    CKB(cudaEventRecord(g->e0, s), "event");
    CKB(cudaGraphLaunch(g->exec, s), "graph launch");
    CKB(cudaEventRecord(g->e1, s), "event");
    CKB(cudaEventRecord(db->last_done, s), "order");
    CKB(cudaStreamWaitEvent(db->stream, db->last_done, 0), "order");
    CKB(cudaMemcpyAsync(status, b->status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s), "results");
    CKB(cudaMemcpyAsync(values, b->out, sizeof(int64_t) * n * b->R, cudaMemcpyDeviceToHost, s), "results");
    gtx::BulkCtl ctl{};
    CKB(cudaMemcpyAsync(&ctl, b->ctl, sizeof ctl, cudaMemcpyDeviceToHost, s), "results");
    CKB(cudaStreamSynchronize(s), "results");
    float t = 0;
    cudaEventElapsedTime(&t, g->e0, g->e1);
    *ms = t;
    if (ctl_out) *ctl_out = ctl;
    if (ctl.err & gtx::ERR_INVAL) return fail_bt(db, GPUTX_EINVAL, "invalid bulk contents");
    if (ctl.err & gtx::ERR_TIMEOUT) return fail_bt(db, GPUTX_ETIMEOUT, "a bounded device wait ran out");
    if (ctl.err & gtx::ERR_CAPACITY) return fail_bt(db, GPUTX_ECAPACITY, "an insert area is full");
    if (ctl.err) return fail_bt(db, GPUTX_EBOUNDS, "device bounds check failed");
    return GPUTX_OK;
}

void plan_candidates(gputx_batcher *bt, int first_strategy)
{
    bt->cands.clear();
    for (int64_t sz : {int64_t(1) << 14, int64_t(1) << 16, int64_t(1) << 18, int64_t(1) << 20})
        if (sz <= bt->cfg.bulk_size_max) bt->cands.push_back({first_strategy, 256, sz, 0});
    if (bt->cands.empty()) bt->cands.push_back({first_strategy, 256, bt->cfg.bulk_size_max, 0});
    // block shapes and the other strategy are tried at the best size found so
    // far (filled in when the sizes are measured)
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
    if (c.strategy != GPUTX_KSET && c.strategy != GPUTX_TPL) c.strategy = GPUTX_KSET;
    bt->best = {c.strategy, c.block_threads, c.bulk_size, 0};
    bt->tuned = !c.tune;
    *out = bt;
    return GPUTX_OK;
}

gputx_status gputx_batcher_run(gputx_batcher *bt, const int64_t *ts, const int32_t *type, const int64_t *params,
                               size_t n, int32_t *status, int64_t *values)
{
    if (!bt || (n && (!ts || !type || !params || !status || !values))) return GPUTX_EINVAL;
    gputx_db *db = bt->db;
    const int P = bt->cfg.params_per_txn, R = db->dev.out_width;
    size_t i = 0;
    while (i < n) {
        Candidate *cand = nullptr;
        if (!bt->tuned) {
            if (bt->cands.empty()) {
                // first bulk: K-SET at 2^16 gives d, w0, c; Algorithm 1 orders
                // the strategies to try
                GraphBulk *g = nullptr;
                const int64_t sz = std::min<int64_t>(1 << 16, bt->cfg.bulk_size_max);
                gputx_status st = get_graph(bt, sz, GPUTX_KSET, 256, &g);
                if (st) return st;
                const int64_t k = std::min<int64_t>(sz, (int64_t)(n - i));
                double ms = 0;
                gtx::BulkCtl ctl{};
                st = run_bulk(bt, g, ts + i, type + i, params + i * P, k, status + i, values + i * R, &ms, &ctl);
                if (st) return st;
                i += (size_t)k;
                const bool wide = (int64_t)ctl.w0 >= std::min<int64_t>(db->cfg.kset_w0_min, k / 4);
                plan_candidates(bt, wide ? GPUTX_KSET : GPUTX_TPL);
                bt->bulks_run++;
                continue;
            }
            if (bt->next_cand < bt->cands.size()) {
                cand = &bt->cands[bt->next_cand];
            } else {
                // the sizes are measured: then block shapes and the other
                // strategy at the best size, once each
                auto best = std::min_element(bt->cands.begin(), bt->cands.end(),
                                             [](const Candidate &a, const Candidate &b) {
                                                 return a.ns_per_txn < b.ns_per_txn;
                                             });
                const Candidate bc = *best;
                const size_t before = bt->cands.size();
                auto have = [&](int s, int blk, int64_t sz) {
                    for (auto &c : bt->cands)
                        if (c.strategy == s && c.block == blk && c.bulk == sz) return true;
                    return false;
                };
                for (int blk : {128, 512})
                    if (!have(bc.strategy, blk, bc.bulk)) bt->cands.push_back({bc.strategy, blk, bc.bulk, 0});
                const int other = bc.strategy == GPUTX_KSET ? GPUTX_TPL : GPUTX_KSET;
                if (!have(other, 256, bc.bulk)) bt->cands.push_back({other, 256, bc.bulk, 0});
                if (bt->cands.size() == before) {
                    bt->best = bc;
                    bt->tuned = true;
                    continue;
                }
                cand = &bt->cands[bt->next_cand];
            }
        }
        const int strategy = cand ? cand->strategy : bt->best.strategy;
        const int block = cand ? cand->block : bt->best.block;
        const int64_t size = cand ? cand->bulk : bt->best.bulk;
        GraphBulk *g = nullptr;
        gputx_status st = get_graph(bt, size, strategy, block, &g);
        if (st) return st;
        const int64_t k = std::min<int64_t>(size, (int64_t)(n - i));
        double ms = 0;
        st = run_bulk(bt, g, ts + i, type + i, params + i * P, k, status + i, values + i * R, &ms, nullptr);
        if (st) return st;
        if (cand) {
            // a short tail bulk is padded: charge it its full capacity
            cand->ns_per_txn = ms * 1e6 / (double)std::max<int64_t>(k, size / 2);
            bt->next_cand++;
        }
        i += (size_t)k;
        bt->bulks_run++;
    }
    return GPUTX_OK;
}

gputx_status gputx_batcher_choice(const gputx_batcher *bt, gputx_batch_choice *out)
{
    if (!bt || !out) return GPUTX_EINVAL;
    std::memset(out, 0, sizeof *out);
    out->tuned = bt->tuned;
    out->strategy = bt->best.strategy;
    out->block_threads = bt->best.block;
    out->bulk_size = bt->best.bulk;
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
    return GPUTX_OK;
}

void gputx_batcher_destroy(gputx_batcher *bt)
{
    if (!bt) return;
    for (GraphBulk *g : bt->graphs) destroy_graph(g);
    delete bt;
}

}  // extern "C"
