/*
 * gputx_oracle.c -- plain, single-threaded CPU oracle for bulk transaction
 * execution ("High-Throughput Transaction Executions on Graphics Processors",
 * He & Yu).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code with the
 * CUDA path.
 *
 * What it computes, each part following the paper:
 *   orc_execute        Definition 1 (Section 3.1): the result database is that
 *                      of executing the bulk serially in increasing timestamp
 *                      order.  Procedures are the two-phase stored procedures
 *                      of Appendix D (read phase may abort, write phase never
 *                      does) for the three stand-in schemas.
 *   orc_access_set     The basic operations (Section 4.1) of one transaction:
 *                      reads/writes on data items at field granularity
 *                      (Section 3.2).  A third class ADD (blind commutative
 *                      increment) is an optional refinement beyond the paper.
 *   orc_levels         Depth of every vertex of the T-dependency graph
 *                      (Section 4.1): length of the longest path from a
 *                      source, computed by a single walk in timestamp order.
 *   orc_onepass_levels The data-oriented k-set calculation of Section 4.2:
 *                      group operations by item, order by timestamp, apply the
 *                      rank rule, take the maximum rank per transaction.
 *   orc_appb_edges     The incremental T-dependency graph construction of
 *                      Appendix B.
 *   orc_topo_levels    Depth by topological sort of an explicit graph
 *                      (Section 4.2, first paragraph).
 *
 * Parity pins for each function live in the tests (closed forms, the paper's
 * Figure 1 example, Properties 1-2, brute force over linear extensions).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { CLS_R = 0, CLS_W = 1, CLS_A = 2 };
enum { MODE_PAPER = 0, MODE_ADD = 1 };

enum {
    T_DC = 0,
    T_SUB_GET_SUBSCRIBER = 1, T_SUB_GET_ACCESS = 2, T_SUB_GET_NEW_DEST = 3,
    T_SUB_UPDATE_LOCATION = 4, T_SUB_UPDATE_FACILITY = 5,
    T_SUB_INSERT_CF = 6, T_SUB_DELETE_CF = 7,
    T_OE_NEW_ORDER = 8, T_OE_PAYMENT = 9, T_OE_ORDER_STATUS = 10
};

#define OE_DIST_PER_WH 10
#define OE_CUST_PER_DIST 3000

typedef struct orc_db {
    /* debit-credit */
    int64_t n_branch, n_teller, n_account;
    int64_t *br_bal, *tel_bal, *acc_bal;
    int64_t hist_cap, hist_n;
    int64_t *hist;              /* hist_cap x 5: ts, account, teller, branch, delta */
    /* subscriber, dense logical form */
    int64_t n_sub;
    int32_t *sub;               /* n_sub x 16 */
    uint8_t *ai_present;        /* n_sub x 4 */
    int32_t *ai_data;           /* n_sub x 4 x 4 */
    uint8_t *sf_present;        /* n_sub x 4 */
    int32_t *sf_active, *sf_err, *sf_data_a, *sf_data_b;  /* n_sub x 4 */
    uint8_t *cf_present;        /* n_sub x 4 x 3 */
    int32_t *cf_end, *cf_numberx;                         /* n_sub x 4 x 3 */
    /* order-entry */
    int64_t n_wh, n_items;
    int64_t *w_tax, *w_ytd;
    int64_t *d_tax, *d_ytd, *d_next_o_id;
    int64_t *c_discount, *c_balance, *c_ytd, *c_payment_cnt, *c_last_o_id;
    int64_t *i_price;
    int32_t *s_quantity;
    int64_t *s_ytd;
    int32_t *s_order_cnt;
    int64_t ord_cap, ord_n;
    int64_t *ord;               /* ord_cap x 6: w, d, o_id, c, ol_cnt, first ol row */
    int64_t ol_cap, ol_n;
    int64_t *ol;                /* ol_cap x 5: order row, item, supply_w, qty, amount */
    int64_t oid_cap;            /* o_id capacity per district */
    int64_t *ord_idx;           /* n_dist x oid_cap: order row of (district, o_id) or -1 */
} orc_db;

/* ------------------------------------------------------------------------- */
/* object numbering: one contiguous range per (table, field group)           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int64_t acc, tel, br, sub, wytd, dytd, dnext, cpay, clast, stock, total;
} orc_layout;

static orc_layout layout_of(const orc_db *db)
{
    orc_layout L;
    int64_t n_d = db->n_wh * OE_DIST_PER_WH;
    int64_t n_c = n_d * OE_CUST_PER_DIST;
    L.acc = 0;
    L.tel = L.acc + db->n_account;
    L.br = L.tel + db->n_teller;
    L.sub = L.br + db->n_branch;
    L.wytd = L.sub + db->n_sub;
    L.dytd = L.wytd + db->n_wh;
    L.dnext = L.dytd + n_d;
    L.cpay = L.dnext + n_d;
    L.clast = L.cpay + n_c;
    L.stock = L.clast + n_c;
    L.total = L.stock + db->n_wh * db->n_items;
    return L;
}

int64_t orc_num_objects(const orc_db *db) { return layout_of(db).total; }

/* ------------------------------------------------------------------------- */
/* basic operations of one transaction (Section 4.1)                          */
/* ------------------------------------------------------------------------- */
#define ORC_MAX_OPS 17

/* Writes up to ORC_MAX_OPS (object, class, root key) triples; returns the
 * count.  Root keys name the root relation's primary key (Section 5.1):
 * branch for debit-credit, subscriber for the subscriber schema, warehouse
 * for order-entry. */
int orc_access_set(const orc_db *db, int32_t type, const int64_t *p, int mode,
                   int64_t *obj, int32_t *cls, int64_t *root)
{
    orc_layout L = layout_of(db);
    int blind = (mode == MODE_ADD) ? CLS_A : CLS_W;
    int k = 0;
    switch (type) {
    case T_DC: {
        int64_t a = p[0];
        int64_t t = a / (db->n_account / db->n_teller);
        int64_t b = a / (db->n_account / db->n_branch);
        obj[k] = L.acc + a; cls[k] = CLS_W; root[k] = b; k++;
        obj[k] = L.tel + t; cls[k] = blind; root[k] = b; k++;
        obj[k] = L.br + b;  cls[k] = blind; root[k] = b; k++;
        break;
    }
    case T_SUB_GET_SUBSCRIBER: case T_SUB_GET_ACCESS: case T_SUB_GET_NEW_DEST:
        obj[k] = L.sub + p[0]; cls[k] = CLS_R; root[k] = p[0]; k++;
        break;
    case T_SUB_UPDATE_LOCATION: case T_SUB_UPDATE_FACILITY:
    case T_SUB_INSERT_CF: case T_SUB_DELETE_CF:
        obj[k] = L.sub + p[0]; cls[k] = CLS_W; root[k] = p[0]; k++;
        break;
    case T_OE_NEW_ORDER: {
        int64_t w = p[0], d = w * OE_DIST_PER_WH + p[1];
        int64_t c = d * OE_CUST_PER_DIST + p[2];
        int64_t cnt = p[3];
        obj[k] = L.dnext + d; cls[k] = CLS_W; root[k] = w; k++;
        obj[k] = L.clast + c; cls[k] = CLS_W; root[k] = w; k++;
        for (int64_t j = 0; j < cnt; j++) {
            int64_t line = p[4 + j];
            int64_t item = line & 0xFFFFFF;
            int64_t sw = (line >> 24) & 0xFFFF;
            if (item >= db->n_items) continue;   /* no such stock row */
            obj[k] = L.stock + sw * db->n_items + item; cls[k] = CLS_W; root[k] = sw; k++;
        }
        break;
    }
    case T_OE_PAYMENT: {
        int64_t w = p[0], d = w * OE_DIST_PER_WH + p[1];
        int64_t c = d * OE_CUST_PER_DIST + p[2];
        obj[k] = L.wytd + w; cls[k] = blind; root[k] = w; k++;
        obj[k] = L.dytd + d; cls[k] = blind; root[k] = w; k++;
        obj[k] = L.cpay + c; cls[k] = CLS_W; root[k] = w; k++;
        break;
    }
    case T_OE_ORDER_STATUS: {
        int64_t w = p[0], d = w * OE_DIST_PER_WH + p[1];
        int64_t c = d * OE_CUST_PER_DIST + p[2];
        obj[k] = L.cpay + c;  cls[k] = CLS_R; root[k] = w; k++;
        obj[k] = L.clast + c; cls[k] = CLS_R; root[k] = w; k++;
        break;
    }
    default:
        return -1;
    }
    return k;
}

/* Fills obj/cls/root for a whole bulk, K slots per transaction; unused
 * slots get obj = -1.  Returns the largest per-transaction count, or -1 on an
 * unknown type or a count above K. */
int orc_extract(const orc_db *db, int64_t n, const int32_t *type,
                const int64_t *params, int P, int mode, int K,
                int64_t *obj, int32_t *cls, int64_t *root)
{
    int maxk = 0;
    int64_t o[ORC_MAX_OPS], r[ORC_MAX_OPS];
    int32_t c[ORC_MAX_OPS];
    for (int64_t i = 0; i < n; i++) {
        int k = orc_access_set(db, type[i], params + i * P, mode, o, c, r);
        if (k < 0 || k > K) return -1;
        if (k > maxk) maxk = k;
        for (int j = 0; j < K; j++) {
            obj[i * K + j] = j < k ? o[j] : -1;
            cls[i * K + j] = j < k ? c[j] : 0;
            root[i * K + j] = j < k ? r[j] : -1;
        }
    }
    return maxk;
}

/* ------------------------------------------------------------------------- */
/* depth of every transaction: longest path from a source (Section 4.1)       */
/* ------------------------------------------------------------------------- */
/* Two basic operations conflict when they touch the same item and at least
 * one writes (Section 4.1); ADD conflicts with R and W but not with ADD.
 * Walking the bulk in timestamp order, each item remembers the largest depth
 * of an earlier reader, writer and adder.  A transaction's depth is one more
 * than the largest depth among earlier transactions it conflicts with (0 if
 * none), which is the longest path ending at it. */
void orc_levels(int64_t n, int K, const int64_t *obj, const int32_t *cls,
                int64_t n_objects, int64_t *level)
{
    int64_t *mr = malloc(sizeof(int64_t) * n_objects);
    int64_t *mw = malloc(sizeof(int64_t) * n_objects);
    int64_t *ma = malloc(sizeof(int64_t) * n_objects);
    for (int64_t o = 0; o < n_objects; o++) mr[o] = mw[o] = ma[o] = -1;
    for (int64_t i = 0; i < n; i++) {
        int64_t lv = 0;
        for (int j = 0; j < K; j++) {
            int64_t o = obj[i * K + j];
            if (o < 0) continue;
            int64_t dep = -1;
            switch (cls[i * K + j]) {
            case CLS_W: dep = mr[o] > mw[o] ? mr[o] : mw[o]; if (ma[o] > dep) dep = ma[o]; break;
            case CLS_R: dep = mw[o] > ma[o] ? mw[o] : ma[o]; break;
            case CLS_A: dep = mw[o] > mr[o] ? mw[o] : mr[o]; break;
            }
            if (dep + 1 > lv) lv = dep + 1;
        }
        level[i] = lv;
        for (int j = 0; j < K; j++) {
            int64_t o = obj[i * K + j];
            if (o < 0) continue;
            int64_t *m = cls[i * K + j] == CLS_W ? mw : cls[i * K + j] == CLS_R ? mr : ma;
            if (lv > m[o]) m[o] = lv;
        }
    }
    free(mr); free(mw); free(ma);
}

/* ------------------------------------------------------------------------- */
/* the one-pass k-set calculation of Section 4.2                              */
/* ------------------------------------------------------------------------- */
typedef struct { int64_t v, id; int32_t cls; int64_t op; } orc_op;

static int cmp_op(const void *a, const void *b)
{
    const orc_op *x = a, *y = b;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;      /* first on the item */
    if (x->id != y->id) return x->id < y->id ? -1 : 1;  /* then on the id   */
    return 0;
}

/* Step 1 sorts the (v, id) tuples by item then id; step 2 marks group
 * boundaries; step 3 ranks inside each group: the first operation gets 0, a
 * write gets the previous rank + 1, a read after a read keeps the previous
 * rank, a read after a write gets + 1.  ADD after ADD keeps the rank like
 * read after read.  Steps 4-5 take the maximum rank of each transaction.
 * rank_out (per operation, indexed like obj) may be NULL. */
void orc_onepass_levels(int64_t n, int K, const int64_t *obj, const int32_t *cls,
                        int64_t *rank_out, int64_t *level)
{
    int64_t m = 0;
    orc_op *ops = malloc(sizeof(orc_op) * (size_t)(n * K + 1));
    for (int64_t i = 0; i < n; i++)
        for (int j = 0; j < K; j++)
            if (obj[i * K + j] >= 0) {
                ops[m].v = obj[i * K + j]; ops[m].id = i;
                ops[m].cls = cls[i * K + j]; ops[m].op = i * K + j; m++;
            }
    qsort(ops, (size_t)m, sizeof(orc_op), cmp_op);
    for (int64_t i = 0; i < n; i++) level[i] = 0;
    int64_t r = 0;
    for (int64_t x = 0; x < m; x++) {
        if (x == 0 || ops[x].v != ops[x - 1].v) {
            r = 0;
        } else {
            int same_shared = ops[x].cls == ops[x - 1].cls && ops[x].cls != CLS_W;
            if (!same_shared) r = r + 1;
        }
        if (rank_out) rank_out[ops[x].op] = r;
        if (r > level[ops[x].id]) level[ops[x].id] = r;
    }
    free(ops);
}

/* ------------------------------------------------------------------------- */
/* Appendix B: incremental T-dependency graph construction                    */
/* ------------------------------------------------------------------------- */
/* Per item, the list of transactions that touched it (ascending).  A new
 * write scans back from the tail to the most recent writer t_w: if t_w is the
 * tail the edge is t_w -> t, otherwise every reader after t_w gets an edge to
 * t (reading "t'" as each of them).  A new read gets the edge t_w -> t.  ADD
 * behaves like a read against writes and like a write against reads.
 * Duplicate edges are kept out.  Returns the number of edges, or -1 when
 * max_edges is exceeded.  edges is [max_edges x 2] (from, to). */
int64_t orc_appb_edges(int64_t n, int K, const int64_t *obj, const int32_t *cls,
                       int64_t n_objects, int64_t *edges, int64_t max_edges)
{
    /* per-item access list stored as a linked list over operation slots */
    int64_t *tail = malloc(sizeof(int64_t) * n_objects);
    int64_t *prev = malloc(sizeof(int64_t) * (size_t)(n * K + 1));
    for (int64_t o = 0; o < n_objects; o++) tail[o] = -1;
    int64_t ne = 0;
#define ADD_EDGE(f, t_)                                                        \
    do {                                                                       \
        int64_t f_ = (f), tt_ = (t_), dup_ = 0;                                \
        if (f_ == tt_) break;                                                  \
        for (int64_t e_ = ne - 1; e_ >= 0 && edges[2 * e_ + 1] == tt_; e_--)    \
            if (edges[2 * e_] == f_) { dup_ = 1; break; }                       \
        if (dup_) break;                                                       \
        if (ne >= max_edges) { ne = -1; goto out; }                            \
        edges[2 * ne] = f_; edges[2 * ne + 1] = tt_; ne++;                     \
    } while (0)
    for (int64_t i = 0; i < n; i++) {
        for (int j = 0; j < K; j++) {
            int64_t o = obj[i * K + j];
            if (o < 0) continue;
            int32_t c = cls[i * K + j];
            int64_t s = tail[o];
            if (c == CLS_W) {
                /* every earlier access up to and including the last writer */
                int first = 1;
                while (s >= 0) {
                    int32_t cs = cls[s];
                    if (cs == CLS_W) {
                        if (first) ADD_EDGE(s / K, i);
                        break;
                    }
                    ADD_EDGE(s / K, i);
                    first = 0;
                    s = prev[s];
                }
            } else {
                /* the most recent access of the conflicting kind(s) */
                int32_t other = (c == CLS_R) ? CLS_A : CLS_R;
                while (s >= 0) {
                    int32_t cs = cls[s];
                    if (cs == CLS_W) { ADD_EDGE(s / K, i); break; }
                    if (cs == other) {
                        /* the run of the other shared class right before */
                        while (s >= 0 && cls[s] == other) { ADD_EDGE(s / K, i); s = prev[s]; }
                        break;
                    }
                    s = prev[s];
                }
            }
            int64_t slot = i * K + j;
            prev[slot] = tail[o];
            tail[o] = slot;
        }
    }
out:
#undef ADD_EDGE
    free(tail); free(prev);
    return ne;
}

/* Topological-sort depth: depth(v) = 1 + max depth of its predecessors, 0
 * for a source.  Vertices are numbered in timestamp order and every edge goes
 * forward, so increasing index is a topological order. */
void orc_topo_levels(int64_t n, const int64_t *edges, int64_t n_edges, int64_t *level)
{
    int64_t *indeg = calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *start = calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *adj = malloc(sizeof(int64_t) * (size_t)(n_edges + 1));
    for (int64_t e = 0; e < n_edges; e++) start[edges[2 * e + 1] + 1]++;
    for (int64_t v = 0; v < n; v++) start[v + 1] += start[v];
    for (int64_t e = 0; e < n_edges; e++) {
        int64_t to = edges[2 * e + 1];
        adj[start[to] + indeg[to]++] = edges[2 * e];
    }
    for (int64_t v = 0; v < n; v++) {
        int64_t d = 0;
        for (int64_t x = start[v]; x < start[v + 1]; x++)
            if (level[adj[x]] + 1 > d) d = level[adj[x]] + 1;
        level[v] = d;
    }
    free(indeg); free(start); free(adj);
}

/* ------------------------------------------------------------------------- */
/* serial execution (Definition 1) with the two-phase procedures              */
/* ------------------------------------------------------------------------- */
static int64_t pack2(int32_t lo, int32_t hi)
{
    return (int64_t)((uint64_t)(uint32_t)lo | ((uint64_t)(uint32_t)hi << 32));
}

static int64_t wrap_add(int64_t a, int64_t b)
{
    return (int64_t)((uint64_t)a + (uint64_t)b);
}

static int32_t run_dc(orc_db *db, int64_t ts, const int64_t *p, int64_t *out)
{
    int64_t a = p[0], delta = p[1];
    int64_t t = a / (db->n_account / db->n_teller);
    int64_t b = a / (db->n_account / db->n_branch);
    if (db->hist_n >= db->hist_cap) return -2;        /* capacity, not a result */
    db->acc_bal[a] = wrap_add(db->acc_bal[a], delta);
    db->tel_bal[t] = wrap_add(db->tel_bal[t], delta);
    db->br_bal[b] = wrap_add(db->br_bal[b], delta);
    int64_t *h = db->hist + db->hist_n * 5;
    h[0] = ts; h[1] = a; h[2] = t; h[3] = b; h[4] = delta;
    db->hist_n++;
    out[0] = db->acc_bal[a];
    return 0;
}

static int32_t run_sub(orc_db *db, int32_t type, const int64_t *p, int64_t *out)
{
    int64_t s = p[0];
    int32_t *row = db->sub + s * 16;
    switch (type) {
    case T_SUB_GET_SUBSCRIBER:
        for (int j = 0; j < 8; j++) out[j] = pack2(row[2 * j], row[2 * j + 1]);
        return 0;
    case T_SUB_GET_ACCESS: {
        int64_t ai = s * 4 + (p[1] - 1);
        if (!db->ai_present[ai]) return 1;
        const int32_t *d = db->ai_data + ai * 4;
        out[0] = pack2(d[0], d[1]);
        out[1] = pack2(d[2], d[3]);
        return 0;
    }
    case T_SUB_GET_NEW_DEST: {
        int64_t sf = s * 4 + (p[1] - 1);
        if (!db->sf_present[sf] || db->sf_active[sf] != 1) return 1;
        int64_t cnt = 0;
        for (int k = 0; k < 3; k++) {
            int64_t st = 8 * k;
            int64_t cf = sf * 3 + k;
            if (st <= p[2] && db->cf_present[cf] && db->cf_end[cf] > p[3])
                out[1 + cnt++] = db->cf_numberx[cf];
        }
        out[0] = cnt;
        return cnt ? 0 : 1;
    }
    case T_SUB_UPDATE_LOCATION:
        out[0] = row[15];
        row[15] = (int32_t)p[1];
        return 0;
    case T_SUB_UPDATE_FACILITY: {
        int64_t sf = s * 4 + (p[1] - 1);
        if (!db->sf_present[sf]) return 1;       /* read phase: abort */
        row[0] = (int32_t)p[2];
        db->sf_data_a[sf] = (int32_t)p[3];
        return 0;
    }
    case T_SUB_INSERT_CF: {
        int64_t sf = s * 4 + (p[1] - 1);
        if (!db->sf_present[sf]) return 1;
        int64_t cf = sf * 3 + p[2] / 8;
        if (db->cf_present[cf]) return 2;         /* duplicate key */
        db->cf_present[cf] = 1;
        db->cf_end[cf] = (int32_t)p[3];
        db->cf_numberx[cf] = (int32_t)p[4];
        return 0;
    }
    case T_SUB_DELETE_CF: {
        int64_t cf = (s * 4 + (p[1] - 1)) * 3 + p[2] / 8;
        if (!db->cf_present[cf]) return 1;
        db->cf_present[cf] = 0;
        return 0;
    }
    }
    return -1;
}

static int32_t run_oe(orc_db *db, int32_t type, const int64_t *p, int64_t *out)
{
    int64_t w = p[0], d = w * OE_DIST_PER_WH + p[1];
    int64_t c = d * OE_CUST_PER_DIST + p[2];
    switch (type) {
    case T_OE_NEW_ORDER: {
        int64_t cnt = p[3];
        for (int64_t j = 0; j < cnt; j++)                /* read phase */
            if ((p[4 + j] & 0xFFFFFF) >= db->n_items) return 1;
        int64_t o_id = db->d_next_o_id[d];
        if (db->ord_n >= db->ord_cap || db->ol_n + cnt > db->ol_cap || o_id >= db->oid_cap)
            return -2;                                   /* capacity, not a result */
        db->d_next_o_id[d] = o_id + 1;
        int64_t row = db->ord_n++;
        int64_t total = 0;
        for (int64_t j = 0; j < cnt; j++) {
            int64_t line = p[4 + j];
            int64_t item = line & 0xFFFFFF, sw = (line >> 24) & 0xFFFF;
            int64_t qty = (line >> 40) & 0xFF;
            int64_t amount = qty * db->i_price[item];
            total += amount;
            int64_t s = sw * db->n_items + item;
            if (db->s_quantity[s] >= qty + 10) db->s_quantity[s] -= (int32_t)qty;
            else db->s_quantity[s] = (int32_t)(db->s_quantity[s] - qty + 91);
            db->s_ytd[s] += qty;
            db->s_order_cnt[s] += 1;
            int64_t *l = db->ol + (db->ol_n++) * 5;
            l[0] = row; l[1] = item; l[2] = sw; l[3] = qty; l[4] = amount;
        }
        int64_t *o = db->ord + row * 6;
        o[0] = w; o[1] = p[1]; o[2] = o_id; o[3] = p[2]; o[4] = cnt; o[5] = db->ol_n - cnt;
        db->ord_idx[d * db->oid_cap + o_id] = row;
        db->c_last_o_id[c] = o_id;
        out[0] = o_id;
        out[1] = total * (10000 - db->c_discount[c]) * (10000 + db->w_tax[w] + db->d_tax[d])
                 / 100000000;
        out[2] = cnt;
        return 0;
    }
    case T_OE_PAYMENT: {
        int64_t amount = p[3];
        db->w_ytd[w] += amount;
        db->d_ytd[d] += amount;
        db->c_balance[c] -= amount;
        db->c_ytd[c] += amount;
        db->c_payment_cnt[c] += 1;
        out[0] = db->c_balance[c];
        return 0;
    }
    case T_OE_ORDER_STATUS: {
        int64_t o_id = db->c_last_o_id[c];
        out[0] = db->c_balance[c];
        out[1] = o_id;
        if (o_id == 0) return 1;                       /* no order yet */
        int64_t row = db->ord_idx[d * db->oid_cap + o_id];
        const int64_t *o = db->ord + row * 6;
        int64_t sum = 0;
        for (int64_t j = 0; j < o[4]; j++) sum += db->ol[(o[5] + j) * 5 + 4];
        out[2] = o[4];
        out[3] = sum;
        return 0;
    }
    }
    return -1;
}

/* Executes the bulk one transaction at a time.  order == NULL means
 * increasing timestamp (index) order, which is Definition 1; a permutation
 * lets tests execute other linear extensions of the dependency graph.
 * Output row i (R int64 values, zero-filled) and status[i] belong to
 * transaction i whatever the order.  Returns 0, -1 on an unknown type, or -2
 * when an append-only table is full. */
int orc_execute(orc_db *db, int64_t n, const int64_t *ts, const int32_t *type,
                const int64_t *params, int P, int R, const int64_t *order,
                int32_t *status, int64_t *out)
{
    int64_t tmp[16];
    for (int64_t x = 0; x < n; x++) {
        int64_t i = order ? order[x] : x;
        const int64_t *p = params + i * P;
        for (int j = 0; j < 16; j++) tmp[j] = 0;
        int32_t st;
        if (type[i] == T_DC) st = run_dc(db, ts[i], p, tmp);
        else if (type[i] >= T_SUB_GET_SUBSCRIBER && type[i] <= T_SUB_DELETE_CF)
            st = run_sub(db, type[i], p, tmp);
        else if (type[i] >= T_OE_NEW_ORDER && type[i] <= T_OE_ORDER_STATUS)
            st = run_oe(db, type[i], p, tmp);
        else return -1;
        if (st < 0) return st;
        status[i] = st;
        for (int j = 0; j < R; j++) out[i * R + j] = tmp[j];
    }
    return 0;
}
