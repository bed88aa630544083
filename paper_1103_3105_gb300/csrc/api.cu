// api.cu -- the C ABI (include/gputx.h): database creation and loading, bulk
// submission, strategy dispatch (Section 5 / Algorithm 1), synchronisation
// and result read-back.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_set>
#include <vector>

#include "engine.h"

using namespace gtx;

namespace {

constexpr int64_t HIST_HOLE = INT64_MIN;

gputx_status fail(gputx_db *db, gputx_status st, const char *fmt, ...)
    __attribute__((format(printf, 3, 4)));

gputx_status fail(gputx_db *db, gputx_status st, const char *fmt, ...)
{
    if (db) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        db->last_error = buf;
    }
    return st;
}

gputx_status cuda_fail(gputx_db *db, cudaError_t e, const char *what)
{
    return fail(db, e == cudaErrorMemoryAllocation ? GPUTX_ENOMEM : GPUTX_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(db, e_, what); \
    } while (0)

template <class T> gputx_status dalloc(gputx_db *db, T **p, int64_t count, const char *what)
{
    *p = nullptr;
    if (count <= 0) return GPUTX_OK;
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, (size_t)count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(db, e, what);
    db->allocs.push_back(q);
    e = cudaMemsetAsync(q, 0, (size_t)count * sizeof(T), db->stream);
    if (e != cudaSuccess) return cuda_fail(db, e, what);
    *p = (T *)q;
    return GPUTX_OK;
}

uint64_t next_pow2(uint64_t v)
{
    uint64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// host replica of the device hash (MurmurHash3 64-bit finaliser) for bulk loads
uint64_t hmix_host(unsigned long long k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

gputx_status alloc_hash(gputx_db *db, HashIndex &h, int64_t rows, const char *what)
{
    const uint64_t cap = next_pow2((uint64_t)std::max<int64_t>(rows, 1) * 2);
    gputx_status st = dalloc(db, &h.keys, (int64_t)cap, what);
    if (st) return st;
    st = dalloc(db, &h.rows, (int64_t)cap, what);
    if (st) return st;
    h.mask = cap - 1;
    cudaError_t e = launch_fill_u64(h.keys, (int64_t)cap, HKEY_EMPTY, db->stream);
    if (e) return cuda_fail(db, e, what);
    return GPUTX_OK;
}

// builds a hash index for rows 0..n-1 with the given keys on the host and
// uploads it; false on a duplicate key
gputx_status upload_hash(gputx_db *db, const HashIndex &h, const std::vector<unsigned long long> &keys)
{
    const uint64_t cap = h.mask + 1;
    if ((uint64_t)keys.size() * 2 > cap) return fail(db, GPUTX_ECAPACITY, "hash index too small");
    std::vector<unsigned long long> hk(cap, HKEY_EMPTY);
    std::vector<uint32_t> hr(cap, 0);
    for (size_t r = 0; r < keys.size(); r++) {
        uint64_t i = hmix_host(keys[r]) & h.mask;
        while (hk[i] != HKEY_EMPTY) {
            if (hk[i] == keys[r]) return fail(db, GPUTX_EINVAL, "duplicate key in loaded rows");
            i = (i + 1) & h.mask;
        }
        hk[i] = keys[r];
        hr[i] = (uint32_t)r;
    }
    CK(cudaMemcpy(h.keys, hk.data(), cap * sizeof(unsigned long long), cudaMemcpyHostToDevice), "hash upload");
    CK(cudaMemcpy(h.rows, hr.data(), cap * sizeof(uint32_t), cudaMemcpyHostToDevice), "hash upload");
    return GPUTX_OK;
}

int table_fields(int table)
{
    static const int f[GPUTX_NUM_TABLES] = {1, 1, 1, 5, 16, 6, 6, 5, 2, 3, 5, 1, 3, 5, 7};
    return (table >= 0 && table < GPUTX_NUM_TABLES) ? f[table] : 0;
}

template <class T> gputx_status put_col(gputx_db *db, T *dst, const std::vector<T> &v)
{
    if (v.empty()) return GPUTX_OK;
    CK(cudaMemcpyAsync(dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, db->stream), "load");
    CK(cudaStreamSynchronize(db->stream), "load");
    return GPUTX_OK;
}

template <class T> gputx_status get_col(gputx_db *db, std::vector<T> &v, const T *src, int64_t n)
{
    v.resize((size_t)std::max<int64_t>(n, 0));
    if (n <= 0) return GPUTX_OK;
    CK(cudaMemcpyAsync(v.data(), src, (size_t)n * sizeof(T), cudaMemcpyDeviceToHost, db->stream), "read");
    CK(cudaStreamSynchronize(db->stream), "read");
    return GPUTX_OK;
}

int type_schema(int t)
{
    if (t == GPUTX_T_DC_DEBIT_CREDIT) return 0;
    if (t >= GPUTX_T_SUB_GET_SUBSCRIBER && t <= GPUTX_T_SUB_DELETE_CF) return 1;
    if (t >= GPUTX_T_OE_NEW_ORDER && t <= GPUTX_T_OE_ORDER_STATUS) return 2;
    return -1;
}

// operations per type: fixed count, or -1 when it depends on the parameters
int type_ops(int t, int *maxk)
{
    switch (t) {
    case GPUTX_T_DC_DEBIT_CREDIT: *maxk = 1; return 1;
    case GPUTX_T_OE_NEW_ORDER: *maxk = 2 + 15; return -1;
    case GPUTX_T_OE_PAYMENT: *maxk = 3; return 3;
    case GPUTX_T_OE_ORDER_STATUS: *maxk = 2; return 2;
    default: *maxk = 1; return 1;
    }
}

struct Carver {
    char *base;
    size_t off = 0;
    template <class T> T *take(int64_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T *p = (T *)(base ? base + off : nullptr);
        off += (size_t)std::max<int64_t>(count, 0) * sizeof(T);
        return p;
    }
};

// lays out (or sizes, with base == nullptr) a bulk's arena
size_t carve_bulk(gputx_bulk *b, char *base, bool device_inputs)
{
    gputx_db *db = b->db;
    const int64_t n = b->n, m = n * std::max(db->kmax, 1);
    const int64_t nn = std::max<int64_t>(n, 1), mm = std::max<int64_t>(m, 1);
    Carver c{base};
    if (!device_inputs) {
        b->ts = c.take<int64_t>(nn);
        b->type = c.take<int32_t>(nn);
        b->params = c.take<int64_t>(nn * b->P);
    }
    b->status = c.take<int32_t>(nn);
    b->out = c.take<int64_t>(nn * b->R);
    b->ctl = c.take<BulkCtl>(1);
    Scratch &s = b->sc;
    s.m_cap = m;
    s.keys_a = c.take<uint32_t>(mm);
    s.vals_a = c.take<uint32_t>(mm);
    s.keys_b = c.take<uint32_t>(mm);
    s.vals_b = c.take<uint32_t>(mm);
    s.op_off = c.take<uint32_t>(nn + 1);
    s.level = c.take<uint32_t>(nn);
    s.rid = db->need_fixpoint ? c.take<uint32_t>(mm) : nullptr;
    s.runmax = db->need_fixpoint ? c.take<uint32_t>(2 * mm) : nullptr;
    s.lock_key = c.take<uint32_t>(mm);
    s.lock_ticket = c.take<uint32_t>(mm);
    s.level_off = c.take<uint32_t>(nn + 2);
    s.type_cut = db->group_oe ? c.take<uint32_t>(3 * (nn + 2)) : nullptr;
    s.chunk_off = c.take<uint32_t>(nn + 2);
    // chunks count lanes: at most lanes / block + levels, and order-entry
    // groups take up to 16 lanes a transaction (+ half-warp padding)
    s.chunk_cap = db->group_oe ? 2 * nn + 2 : nn + nn / 32 + 2;
    s.chunk_level = c.take<uint32_t>(s.chunk_cap);
    s.done = c.take<uint32_t>(nn + 1);
    s.part_start = c.take<uint32_t>(nn + 1);
    s.pid_key = c.take<uint32_t>(nn);
    s.pid_val = c.take<uint32_t>(nn);
    s.pid_key2 = c.take<uint32_t>(nn);
    s.pid_val2 = c.take<uint32_t>(nn);
    s.rec_params = c.take<int64_t>(nn * b->P);
    s.rec_ts = c.take<int64_t>(nn);
    s.rec_type = c.take<int32_t>(nn);
    s.rec_t = c.take<uint32_t>(nn);
    const bool slots = (db->dev.registered >> GPUTX_T_SUB_INSERT_CF & 1u) ||
                       (db->dev.registered >> GPUTX_T_OE_NEW_ORDER & 1u);
    s.slot_cf = slots ? c.take<uint32_t>(nn) : nullptr;
    s.slot_ord = slots ? c.take<uint32_t>(nn) : nullptr;
    s.slot_ol = slots ? c.take<uint32_t>(nn) : nullptr;
    s.slot_hist = db->hist_by_type ? c.take<uint32_t>(nn) : nullptr;
    s.sort_hist = c.take<uint32_t>(4 * 256);
    s.sort_offs = c.take<uint32_t>(4 * 256);
    const int64_t big = std::max(mm, nn + 2);
    s.sort_tiles = (big + 8191) / 8192;
    s.sort_status = c.take<uint32_t>(4 * s.sort_tiles * 256);
    s.tile_ctr = c.take<uint32_t>(16);
    s.scan_tiles = (big + 2047) / 2048;
    s.scan_status = c.take<uint64_t>(s.scan_tiles);
    s.scan_vals = c.take<uint64_t>(2 * s.scan_tiles);
    s.rec_dc = db->dev.registered == (1u << GPUTX_T_DC_DEBIT_CREDIT) ? c.take<DcRecord>(nn) : nullptr;
    s.seg_off = b->graph ? c.take<uint32_t>(kSegMax + 1) : nullptr;
    s.bulk_of = b->graph ? c.take<uint32_t>(nn) : nullptr;
    s.seg_depth = b->graph ? c.take<uint32_t>(kSegMax) : nullptr;
    s.seg_base = b->graph ? c.take<uint32_t>(kSegMax + 1) : nullptr;
    return c.off + 256;
}

gputx_status bulk_error(gputx_db *db, uint32_t err)
{
    if (err & ERR_INVAL) return fail(db, GPUTX_EINVAL, "invalid bulk: unknown or unregistered type, "
                                                       "parameter out of range or timestamps not increasing");
    if (err & ERR_TIMEOUT) return fail(db, GPUTX_ETIMEOUT, "a bounded device wait ran out");
    if (err & ERR_CAPACITY) return fail(db, GPUTX_ECAPACITY, "an insert area or hash index is full");
    if (err & ERR_BOUNDS) return fail(db, GPUTX_EBOUNDS, "device bounds check failed");
    return GPUTX_OK;
}

gputx_status read_ctl(gputx_bulk *b)
{
    gputx_db *db = b->db;
    CK(cudaMemcpyAsync(&b->host_ctl, b->ctl, sizeof(BulkCtl), cudaMemcpyDeviceToHost, b->stream), "sync");
    CK(cudaStreamSynchronize(b->stream), "sync");
    return GPUTX_OK;
}

}  // namespace

size_t gtx_carve_bulk(gputx_bulk *b, char *base, bool device_inputs) { return carve_bulk(b, base, device_inputs); }

extern "C" {

const char *gputx_version(void) { return "gputx-gb300 0.1 (sm_103a)"; }

const char *gputx_last_error(const gputx_db *db) { return db ? db->last_error.c_str() : "null database"; }

int gputx_output_width(const gputx_db *db) { return db ? db->dev.out_width : 0; }

void gputx_destroy_db(gputx_db *db)
{
    if (!db) return;
    if (db->last_done) cudaStreamWaitEvent(db->stream, db->last_done, 0);
    cudaStreamSynchronize(db->stream);
    for (cudaStream_t ps : db->pool)
        if (ps) {
            cudaStreamSynchronize(ps);
            cudaStreamDestroy(ps);
        }
    if (db->last_done) cudaEventDestroy(db->last_done);
    for (void *p : db->allocs) cudaFree(p);
    if (db->own_stream) cudaStreamDestroy(db->stream);
    delete db;
}

gputx_status gputx_create_db(const gputx_schema_desc *schema, const gputx_config *cfg, void *cuda_stream,
                             gputx_db **out)
{
    if (!schema || !out) return GPUTX_EINVAL;
    *out = nullptr;
    gputx_db *db = new (std::nothrow) gputx_db();
    if (!db) return GPUTX_ENOMEM;
    db->schema = *schema;
    if (cfg) db->cfg = *cfg;
    gputx_config &c = db->cfg;
    if (c.max_bulk <= 0) c.max_bulk = 1 << 22;
    if (c.block_threads <= 0) c.block_threads = 256;
    if (c.spin_limit_ns <= 0) c.spin_limit_ns = 2000000000LL;
    if (c.kset_w0_min <= 0) c.kset_w0_min = 152 * 256;
    if (c.part_c_max <= 0) c.part_c_max = 0;
    if (c.part_d_min <= 0) c.part_d_min = 4096;
    const gputx_schema_desc &s = db->schema;
    auto bad = [&](const char *m) {
        gputx_status st = fail(db, GPUTX_EINVAL, "%s", m);
        std::string msg = db->last_error;
        delete db;
        (void)msg;
        return st;
    };
    if (c.block_threads < 32 || c.block_threads > 1024 || c.block_threads % 32) return bad("block_threads");
    if (c.max_bulk > (1 << 25)) return bad("max_bulk above 2^25");
    if (s.dc_branches < 0 || s.dc_tellers < 0 || s.dc_accounts < 0 || s.sub_subscribers < 0 ||
        s.oe_warehouses < 0 || s.oe_items < 0)
        return bad("negative size");
    if (s.dc_branches > 0) {
        if (s.dc_tellers <= 0 || s.dc_accounts <= 0 || s.dc_tellers % s.dc_branches ||
            s.dc_accounts % s.dc_tellers)
            return bad("debit-credit: tellers must be a multiple of branches and accounts of tellers");
    }
    if (s.oe_warehouses > 0 && (s.oe_items <= 0 || s.oe_items >= (1 << 24) || s.oe_warehouses >= (1 << 16)))
        return bad("order-entry sizes");
    int dev = 0;
    cudaGetDevice(&dev);
    db->device = dev;
    cudaDeviceGetAttribute(&db->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (cuda_stream) {
        db->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&db->stream, cudaStreamNonBlocking) != cudaSuccess) return bad("stream");
        db->own_stream = true;
    }
    for (int i = 0; i < gputx_db::kPool; i++)
        if (cudaStreamCreateWithFlags(&db->pool[i], cudaStreamNonBlocking) != cudaSuccess) {
            gputx_destroy_db(db);
            return GPUTX_ECUDA;
        }
    if (cudaEventCreateWithFlags(&db->last_done, cudaEventDisableTiming) != cudaSuccess) {
        gputx_destroy_db(db);
        return GPUTX_ECUDA;
    }
    // keep freed stream-ordered allocations for reuse by later bulks
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }

    DevDB &d = db->dev;
    // object ids: one range per (table, field group)
    uint64_t o = 0;
    const int64_t n_d = s.oe_warehouses * OE_DIST, n_c = n_d * OE_CUST;
    // small root tables first, so a bulk whose keys are only root keys sorts
    // on few bits
    d.o_br = (uint32_t)o; o += s.dc_branches;
    d.o_tel = (uint32_t)o; o += s.dc_tellers;
    d.o_wytd = (uint32_t)o; o += s.oe_warehouses;
    d.o_dytd = (uint32_t)o; o += n_d;
    d.o_dnext = (uint32_t)o; o += n_d;
    d.o_acc = (uint32_t)o; o += s.dc_accounts;
    d.o_sub = (uint32_t)o; o += s.sub_subscribers;
    d.o_cpay = (uint32_t)o; o += n_c;
    d.o_clast = (uint32_t)o; o += n_c;
    d.o_stock = (uint32_t)o; o += s.oe_warehouses * s.oe_items;
    if (o >= 0xffffffffull) {
        gputx_destroy_db(db);
        return GPUTX_EINVAL;
    }
    d.n_objects = (uint32_t)o;
    db->obj_bits = std::max(1, bits_for(o));   // covers the padding key o as well

    gputx_status st = GPUTX_OK;
#define TRY(x)                         \
    do {                               \
        st = (x);                      \
        if (st) {                      \
            std::string m = db->last_error; \
            gputx_destroy_db(db);      \
            (void)m;                   \
            return st;                 \
        }                              \
    } while (0)
    if (s.dc_branches > 0) {
        d.n_br = s.dc_branches;
        d.n_tel = s.dc_tellers;
        d.n_acc = s.dc_accounts;
        d.acc_per_tel = s.dc_accounts / s.dc_tellers;
        d.acc_per_br = s.dc_accounts / s.dc_branches;
        d.div_tel = FastDiv::make((uint32_t)d.acc_per_tel);
        d.div_br = FastDiv::make((uint32_t)d.acc_per_br);
        TRY(dalloc(db, &d.br_bal, d.n_br, "branch"));
        TRY(dalloc(db, &d.tel_bal, d.n_tel, "teller"));
        TRY(dalloc(db, &d.acc_bal, d.n_acc, "account"));
        d.hist_cap = s.dc_history_capacity > 0 ? s.dc_history_capacity : 4 * c.max_bulk;
        TRY(dalloc(db, &d.h_ts, d.hist_cap, "history"));
        TRY(dalloc(db, &d.h_acc, d.hist_cap, "history"));
        TRY(dalloc(db, &d.h_tel, d.hist_cap, "history"));
        TRY(dalloc(db, &d.h_br, d.hist_cap, "history"));
        TRY(dalloc(db, &d.h_delta, d.hist_cap, "history"));
        if (launch_fill_i64(d.h_ts, d.hist_cap, HIST_HOLE, db->stream)) TRY(fail(db, GPUTX_ECUDA, "fill"));
    }
    if (s.sub_subscribers > 0) {
        d.n_sub = s.sub_subscribers;
        TRY(dalloc(db, &d.sub_rows, d.n_sub * SUB_FIELDS, "subscriber"));
        const int64_t cap4 = 4 * d.n_sub;
        d.child_cap = s.sub_child_capacity > 0 ? s.sub_child_capacity : 6 * d.n_sub;
        TRY(dalloc(db, &d.ai_data, cap4 * 4, "access_info"));
        TRY(dalloc(db, &d.ai_sid, cap4, "access_info"));
        TRY(dalloc(db, &d.ai_type, cap4, "access_info"));
        TRY(alloc_hash(db, d.ai_idx, cap4, "access_info index"));
        TRY(dalloc(db, &d.sf_sid, cap4, "special_facility"));
        TRY(dalloc(db, &d.sf_type, cap4, "special_facility"));
        TRY(dalloc(db, &d.sf_active, cap4, "special_facility"));
        TRY(dalloc(db, &d.sf_err, cap4, "special_facility"));
        TRY(dalloc(db, &d.sf_data_a, cap4, "special_facility"));
        TRY(dalloc(db, &d.sf_data_b, cap4, "special_facility"));
        TRY(alloc_hash(db, d.sf_idx, cap4, "special_facility index"));
        const int64_t cc = d.child_cap;
        TRY(dalloc(db, &d.cf_sid, cc, "call_forwarding"));
        TRY(dalloc(db, &d.cf_type, cc, "call_forwarding"));
        TRY(dalloc(db, &d.cf_start, cc, "call_forwarding"));
        TRY(dalloc(db, &d.cf_end, cc, "call_forwarding"));
        TRY(dalloc(db, &d.cf_numberx, cc, "call_forwarding"));
        TRY(dalloc(db, &d.cf_live, cc, "call_forwarding"));
        TRY(alloc_hash(db, d.cf_idx, cc, "call_forwarding index"));
    }
    if (s.oe_warehouses > 0) {
        d.n_wh = s.oe_warehouses;
        d.n_items = s.oe_items;
        TRY(dalloc(db, &d.w_tax, d.n_wh, "warehouse"));
        TRY(dalloc(db, &d.w_ytd, d.n_wh, "warehouse"));
        TRY(dalloc(db, &d.d_tax, n_d, "district"));
        TRY(dalloc(db, &d.d_ytd, n_d, "district"));
        TRY(dalloc(db, &d.d_next_o_id, n_d, "district"));
        TRY(dalloc(db, &d.c_discount, n_c, "customer"));
        TRY(dalloc(db, &d.c_balance, n_c, "customer"));
        TRY(dalloc(db, &d.c_ytd, n_c, "customer"));
        TRY(dalloc(db, &d.c_payment_cnt, n_c, "customer"));
        TRY(dalloc(db, &d.c_last_o_id, n_c, "customer"));
        TRY(dalloc(db, &d.i_price, d.n_items, "item"));
        const int64_t ns = d.n_wh * d.n_items;
        TRY(dalloc(db, &d.s_quantity, ns, "stock"));
        TRY(dalloc(db, &d.s_order_cnt, ns, "stock"));
        TRY(dalloc(db, &d.s_ytd, ns, "stock"));
        d.ord_cap = s.oe_order_capacity > 0 ? s.oe_order_capacity : 2 * c.max_bulk;
        d.ol_cap = s.oe_orderline_capacity > 0 ? s.oe_orderline_capacity : 16 * d.ord_cap;
        TRY(dalloc(db, &d.o_w, d.ord_cap, "order"));
        TRY(dalloc(db, &d.o_d, d.ord_cap, "order"));
        TRY(dalloc(db, &d.o_c, d.ord_cap, "order"));
        TRY(dalloc(db, &d.o_cnt, d.ord_cap, "order"));
        TRY(dalloc(db, &d.o_id, d.ord_cap, "order"));
        TRY(dalloc(db, &d.o_first, d.ord_cap, "order"));
        TRY(dalloc(db, &d.o_live, d.ord_cap, "order"));
        TRY(dalloc(db, &d.ol_item, d.ol_cap, "order_line"));
        TRY(dalloc(db, &d.ol_sw, d.ol_cap, "order_line"));
        TRY(dalloc(db, &d.ol_qty, d.ol_cap, "order_line"));
        TRY(dalloc(db, &d.ol_amount, d.ol_cap, "order_line"));
        TRY(alloc_hash(db, d.ord_idx, d.ord_cap, "order index"));
    }
    TRY(dalloc(db, &db->d_cursor, 1, "cursor"));
    {
        const uint32_t lines = (uint32_t)((std::max<int64_t>(d.n_objects, 1) + 31) / 32);
        db->lock_slots.lines = FastDiv::make(lines);
        TRY(dalloc(db, &db->d_done, (int64_t)lines * 32, "lock counters"));
    }
#undef TRY
    d.out_width = s.sub_subscribers > 0 ? 8 : s.oe_warehouses > 0 ? 4 : 1;
    if (cudaStreamSynchronize(db->stream) != cudaSuccess) {
        gputx_destroy_db(db);
        return GPUTX_ECUDA;
    }
    *out = db;
    return GPUTX_OK;
}

gputx_status gputx_register_types(gputx_db *db, const int32_t *type_ids, int n)
{
    if (!db || (n > 0 && !type_ids) || n < 0) return fail(db, GPUTX_EINVAL, "bad arguments");
    uint32_t reg = db->dev.registered;
    for (int i = 0; i < n; i++) {
        const int t = type_ids[i];
        const int sc = type_schema(t);
        if (sc < 0) return fail(db, GPUTX_EINVAL, "unknown type id %d", t);
        const bool have = (sc == 0 && db->dev.n_acc > 0) || (sc == 1 && db->dev.n_sub > 0) ||
                          (sc == 2 && db->dev.n_wh > 0);
        if (!have) return fail(db, GPUTX_EINVAL, "type %d needs a schema this database lacks", t);
        reg |= 1u << t;
    }
    db->dev.registered = reg;
    int kmax = 0, uniform = -2, ntypes = 0, maxid = 0;
    bool fix = false;
    for (int t = 0; t < GPUTX_NUM_TYPES; t++) {
        if (!((reg >> t) & 1u)) continue;
        ntypes++;
        maxid = t;
        int mk = 0;
        const int k = type_ops(t, &mk);
        kmax = std::max(kmax, mk);
        if (uniform == -2) uniform = k;
        else if (uniform != k) uniform = -1;
        // one-pass ranks are exact when every transaction's items nest under
        // one item it writes (debit-credit: account within teller within
        // branch) or it touches one item (subscriber); order-entry's
        // multi-item transactions need the exact-depth pass
        if (t >= GPUTX_T_OE_NEW_ORDER) fix = true;
    }
    db->kmax = kmax;
    db->uniform_k = uniform > 0 ? uniform : 0;
    db->need_fixpoint = fix;
    db->tbits = ntypes > 1 ? bits_for((uint64_t)maxid) : 0;
    // a bulk that mixes debit-credit with other types takes history rows
    // for its debit-credit transactions only
    db->hist_by_type = (db->dev.registered & 1u) && db->dev.registered != 1u;
    // levels sorted by (level, type) know where each order-entry type starts
    db->group_oe = db->tbits > 0 && (db->dev.registered & ((1u << GPUTX_T_OE_NEW_ORDER) |
                                                           (1u << GPUTX_T_OE_ORDER_STATUS)));
    return GPUTX_OK;
}

gputx_status gputx_load_table(gputx_db *db, int table, const int64_t *rows, size_t n_rows)
{
    if (!db || (!rows && n_rows)) return fail(db, GPUTX_EINVAL, "bad arguments");
    DevDB &d = db->dev;
    const int f = table_fields(table);
    if (!f) return fail(db, GPUTX_EINVAL, "unknown table %d", table);
    const int64_t n = (int64_t)n_rows;
    auto col64 = [&](int j) {
        std::vector<int64_t> v((size_t)n);
        for (int64_t i = 0; i < n; i++) v[i] = rows[i * f + j];
        return v;
    };
    auto col32 = [&](int j) {
        std::vector<int32_t> v((size_t)n);
        for (int64_t i = 0; i < n; i++) v[i] = (int32_t)rows[i * f + j];
        return v;
    };
    auto need = [&](int64_t want, const char *what) -> gputx_status {
        if (want <= 0) return fail(db, GPUTX_EINVAL, "%s: schema not created", what);
        if (n != want) return fail(db, GPUTX_EINVAL, "%s: expected %lld rows, got %lld", what, (long long)want,
                                   (long long)n);
        return GPUTX_OK;
    };
    gputx_status st;
    switch (table) {
    case GPUTX_TBL_DC_BRANCH:
        if ((st = need(d.n_br, "branch"))) return st;
        return put_col(db, d.br_bal, col64(0));
    case GPUTX_TBL_DC_TELLER:
        if ((st = need(d.n_tel, "teller"))) return st;
        return put_col(db, d.tel_bal, col64(0));
    case GPUTX_TBL_DC_ACCOUNT:
        if ((st = need(d.n_acc, "account"))) return st;
        return put_col(db, d.acc_bal, col64(0));
    case GPUTX_TBL_SUB_SUBSCRIBER: {
        if ((st = need(d.n_sub, "subscriber"))) return st;
        std::vector<int32_t> v((size_t)n * SUB_FIELDS);
        for (int64_t i = 0; i < n * SUB_FIELDS; i++) v[i] = (int32_t)rows[i];
        return put_col(db, d.sub_rows, v);
    }
    case GPUTX_TBL_SUB_ACCESS_INFO:
    case GPUTX_TBL_SUB_SPECIAL_FACILITY:
    case GPUTX_TBL_SUB_CALL_FORWARDING: {
        if (d.n_sub <= 0) return fail(db, GPUTX_EINVAL, "subscriber schema not created");
        InsertBase cur{};
        CK(cudaMemcpy(&cur, db->d_cursor, sizeof cur, cudaMemcpyDeviceToHost), "cursor");
        const bool is_cf = table == GPUTX_TBL_SUB_CALL_FORWARDING;
        const int64_t cap = is_cf ? d.child_cap : 4 * d.n_sub;
        if (n > cap) return fail(db, GPUTX_ECAPACITY, "too many child rows");
        std::vector<unsigned long long> keys((size_t)n);
        for (int64_t i = 0; i < n; i++) {
            const int64_t *r = rows + i * f;
            if (r[0] < 0 || r[0] >= d.n_sub || r[1] < 1 || r[1] > 4)
                return fail(db, GPUTX_EINVAL, "child row %lld: key out of range", (long long)i);
            if (is_cf && !(r[2] == 0 || r[2] == 8 || r[2] == 16))
                return fail(db, GPUTX_EINVAL, "call_forwarding row %lld: start_time", (long long)i);
            keys[i] = is_cf ? (unsigned long long)((r[0] * 4 + (r[1] - 1)) * 3 + r[2] / 8)
                            : (unsigned long long)(r[0] * 4 + (r[1] - 1));
        }
        if (table == GPUTX_TBL_SUB_ACCESS_INFO) {
            if ((st = upload_hash(db, d.ai_idx, keys))) return st;
            std::vector<int32_t> data((size_t)n * 4);
            for (int64_t i = 0; i < n; i++)
                for (int j = 0; j < 4; j++) data[i * 4 + j] = (int32_t)rows[i * f + 2 + j];
            if ((st = put_col(db, d.ai_data, data))) return st;
            if ((st = put_col(db, d.ai_sid, col32(0)))) return st;
            return put_col(db, d.ai_type, col32(1));
        }
        if (table == GPUTX_TBL_SUB_SPECIAL_FACILITY) {
            if ((st = upload_hash(db, d.sf_idx, keys))) return st;
            if ((st = put_col(db, d.sf_sid, col32(0)))) return st;
            if ((st = put_col(db, d.sf_type, col32(1)))) return st;
            if ((st = put_col(db, d.sf_active, col32(2)))) return st;
            if ((st = put_col(db, d.sf_err, col32(3)))) return st;
            if ((st = put_col(db, d.sf_data_a, col32(4)))) return st;
            return put_col(db, d.sf_data_b, col32(5));
        }
        if (cur.cf != 0) return fail(db, GPUTX_ESTATE, "call_forwarding already holds rows");
        if ((st = upload_hash(db, d.cf_idx, keys))) return st;
        if ((st = put_col(db, d.cf_sid, col32(0)))) return st;
        if ((st = put_col(db, d.cf_type, col32(1)))) return st;
        if ((st = put_col(db, d.cf_start, col32(2)))) return st;
        if ((st = put_col(db, d.cf_end, col32(3)))) return st;
        if ((st = put_col(db, d.cf_numberx, col32(4)))) return st;
        if ((st = put_col(db, d.cf_live, std::vector<uint8_t>((size_t)n, 1)))) return st;
        cur.cf = n;
        CK(cudaMemcpy(db->d_cursor, &cur, sizeof cur, cudaMemcpyHostToDevice), "cursor");
        return GPUTX_OK;
    }
    case GPUTX_TBL_OE_WAREHOUSE:
        if ((st = need(d.n_wh, "warehouse"))) return st;
        if ((st = put_col(db, d.w_tax, col64(0)))) return st;
        return put_col(db, d.w_ytd, col64(1));
    case GPUTX_TBL_OE_DISTRICT:
        if ((st = need(d.n_wh * OE_DIST, "district"))) return st;
        if ((st = put_col(db, d.d_tax, col64(0)))) return st;
        if ((st = put_col(db, d.d_ytd, col64(1)))) return st;
        return put_col(db, d.d_next_o_id, col64(2));
    case GPUTX_TBL_OE_CUSTOMER:
        if ((st = need(d.n_wh * OE_DIST * OE_CUST, "customer"))) return st;
        if ((st = put_col(db, d.c_discount, col64(0)))) return st;
        if ((st = put_col(db, d.c_balance, col64(1)))) return st;
        if ((st = put_col(db, d.c_ytd, col64(2)))) return st;
        if ((st = put_col(db, d.c_payment_cnt, col64(3)))) return st;
        return put_col(db, d.c_last_o_id, col64(4));
    case GPUTX_TBL_OE_ITEM:
        if ((st = need(d.n_items, "item"))) return st;
        return put_col(db, d.i_price, col64(0));
    case GPUTX_TBL_OE_STOCK:
        if ((st = need(d.n_wh * d.n_items, "stock"))) return st;
        if ((st = put_col(db, d.s_quantity, col32(0)))) return st;
        if ((st = put_col(db, d.s_ytd, col64(1)))) return st;
        return put_col(db, d.s_order_cnt, col32(2));
    }
    return fail(db, GPUTX_EINVAL, "table %d is read only", table);
}

gputx_status gputx_read_index(gputx_db *db, int index, uint64_t *keys, uint32_t *rows, size_t capacity,
                              size_t *size)
{
    if (!db || !size) return fail(db, GPUTX_EINVAL, "bad arguments");
    const DevDB &d = db->dev;
    const HashIndex *h = nullptr;
    switch (index) {
    case 0: h = d.n_sub > 0 ? &d.ai_idx : nullptr; break;
    case 1: h = d.n_sub > 0 ? &d.sf_idx : nullptr; break;
    case 2: h = d.n_sub > 0 ? &d.cf_idx : nullptr; break;
    case 3: h = d.n_wh > 0 ? &d.ord_idx : nullptr; break;
    default: break;
    }
    if (!h || !h->keys) return fail(db, GPUTX_EINVAL, "index %d does not exist", index);
    const size_t n = (size_t)h->mask + 1;
    *size = n;
    if (!keys && !rows) return GPUTX_OK;
    if (!keys || !rows || capacity < n) return fail(db, GPUTX_EINVAL, "capacity %zu < index size %zu", capacity, n);
    CK(cudaStreamWaitEvent(db->stream, db->last_done, 0), "sync");
    CK(cudaMemcpyAsync(keys, h->keys, n * sizeof(uint64_t), cudaMemcpyDeviceToHost, db->stream), "read index");
    CK(cudaMemcpyAsync(rows, h->rows, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, db->stream), "read index");
    CK(cudaStreamSynchronize(db->stream), "read index");
    return GPUTX_OK;
}

gputx_status gputx_read_slots(gputx_db *db, int table, int64_t *rows, size_t capacity_rows, size_t *n_rows)
{
    if (!db || !n_rows) return fail(db, GPUTX_EINVAL, "bad arguments");
    const DevDB &d = db->dev;
    const int f = table_fields(table);
    CK(cudaStreamWaitEvent(db->stream, db->last_done, 0), "sync");
    CK(cudaStreamSynchronize(db->stream), "sync");
    InsertBase cur{};
    CK(cudaMemcpy(&cur, db->d_cursor, sizeof cur, cudaMemcpyDeviceToHost), "cursor");
    std::vector<std::vector<int64_t>> cols;
    gputx_status st = GPUTX_OK;
    auto add32 = [&](const int32_t *src, int64_t n) {
        std::vector<int32_t> v;
        if (!st) st = get_col(db, v, src, n);
        cols.emplace_back(v.begin(), v.end());
    };
    auto add64 = [&](const int64_t *src, int64_t n) {
        std::vector<int64_t> v;
        if (!st) st = get_col(db, v, src, n);
        cols.push_back(std::move(v));
    };
    auto add8 = [&](const uint8_t *src, int64_t n) {
        std::vector<uint8_t> v;
        if (!st) st = get_col(db, v, src, n);
        cols.emplace_back(v.begin(), v.end());
    };
    int64_t n = 0;
    switch (table) {
    case GPUTX_TBL_SUB_ACCESS_INFO: {
        if (d.n_sub <= 0) return fail(db, GPUTX_EINVAL, "subscriber schema not created");
        n = 4 * d.n_sub;
        add32(d.ai_sid, n); add32(d.ai_type, n);
        std::vector<int32_t> data;
        if (!st) st = get_col(db, data, d.ai_data, n * 4);
        if (st) return st;
        for (int j = 0; j < 4; j++) {
            std::vector<int64_t> c((size_t)n);
            for (int64_t i = 0; i < n; i++) c[i] = data[(size_t)i * 4 + j];
            cols.push_back(std::move(c));
        }
        std::vector<int64_t> live((size_t)n);
        for (int64_t i = 0; i < n; i++) live[i] = cols[1][i] >= 1;
        cols.push_back(std::move(live));
        break;
    }
    case GPUTX_TBL_SUB_SPECIAL_FACILITY: {
        if (d.n_sub <= 0) return fail(db, GPUTX_EINVAL, "subscriber schema not created");
        n = 4 * d.n_sub;
        add32(d.sf_sid, n); add32(d.sf_type, n); add32(d.sf_active, n);
        add32(d.sf_err, n); add32(d.sf_data_a, n); add32(d.sf_data_b, n);
        if (st) return st;
        std::vector<int64_t> live((size_t)n);
        for (int64_t i = 0; i < n; i++) live[i] = cols[1][i] >= 1;
        cols.push_back(std::move(live));
        break;
    }
    case GPUTX_TBL_SUB_CALL_FORWARDING:
        if (d.n_sub <= 0) return fail(db, GPUTX_EINVAL, "subscriber schema not created");
        n = std::min<int64_t>(cur.cf, d.child_cap);
        add32(d.cf_sid, n); add32(d.cf_type, n); add32(d.cf_start, n); add32(d.cf_end, n);
        add32(d.cf_numberx, n); add8(d.cf_live, n);
        break;
    case GPUTX_TBL_OE_ORDER: {
        if (d.n_wh <= 0) return fail(db, GPUTX_EINVAL, "order-entry schema not created");
        n = std::min<int64_t>(cur.ord, d.ord_cap);
        add32(d.o_w, n); add32(d.o_d, n); add64(d.o_id, n); add32(d.o_c, n); add32(d.o_cnt, n);
        add8(d.o_live, n);
        break;
    }
    default:
        return fail(db, GPUTX_EINVAL, "table %d has no slot storage to read", table);
    }
    if (st) return st;
    if ((int)cols.size() != f + 1) return fail(db, GPUTX_EINVAL, "table %d layout", table);
    *n_rows = (size_t)n;
    if (!rows) return GPUTX_OK;
    if (capacity_rows < (size_t)n) return fail(db, GPUTX_EINVAL, "capacity %zu < %lld slots", capacity_rows,
                                               (long long)n);
    for (int64_t i = 0; i < n; i++)
        for (int j = 0; j <= f; j++) rows[i * (f + 1) + j] = cols[j][i];
    return GPUTX_OK;
}

gputx_status gputx_read_table(gputx_db *db, int table, int64_t *rows, size_t capacity_rows, size_t *n_rows)
{
    if (!db || !n_rows) return fail(db, GPUTX_EINVAL, "bad arguments");
    const DevDB &d = db->dev;
    const int f = table_fields(table);
    if (!f) return fail(db, GPUTX_EINVAL, "unknown table %d", table);
    CK(cudaStreamWaitEvent(db->stream, db->last_done, 0), "sync");
    CK(cudaStreamSynchronize(db->stream), "sync");
    InsertBase cur{};
    CK(cudaMemcpy(&cur, db->d_cursor, sizeof cur, cudaMemcpyDeviceToHost), "cursor");
    std::vector<std::vector<int64_t>> cols;   // output columns
    gputx_status st = GPUTX_OK;
    auto add64 = [&](const int64_t *src, int64_t n) {
        std::vector<int64_t> v;
        if (!st) st = get_col(db, v, src, n);
        cols.push_back(std::move(v));
    };
    auto add32 = [&](const int32_t *src, int64_t n) {
        std::vector<int32_t> v;
        if (!st) st = get_col(db, v, src, n);
        cols.emplace_back(v.begin(), v.end());
    };
    std::vector<uint8_t> keep;   // live-row filter (empty = all)
    switch (table) {
    case GPUTX_TBL_DC_BRANCH: add64(d.br_bal, d.n_br); break;
    case GPUTX_TBL_DC_TELLER: add64(d.tel_bal, d.n_tel); break;
    case GPUTX_TBL_DC_ACCOUNT: add64(d.acc_bal, d.n_acc); break;
    case GPUTX_TBL_DC_HISTORY: {
        const int64_t n = std::min<int64_t>(cur.hist, d.hist_cap);
        add64(d.h_ts, n); add64(d.h_acc, n); add64(d.h_tel, n); add64(d.h_br, n); add64(d.h_delta, n);
        if (!st) {
            keep.resize((size_t)n);
            for (int64_t i = 0; i < n; i++) keep[i] = cols[0][i] != HIST_HOLE;
        }
        break;
    }
    case GPUTX_TBL_SUB_SUBSCRIBER: {
        std::vector<int32_t> v;
        st = get_col(db, v, d.sub_rows, d.n_sub * SUB_FIELDS);
        if (st) return st;
        const int64_t n = d.n_sub;
        *n_rows = (size_t)n;
        if (!rows) return GPUTX_OK;
        if ((int64_t)capacity_rows < n) return fail(db, GPUTX_EINVAL, "capacity");
        for (int64_t i = 0; i < n * SUB_FIELDS; i++) rows[i] = v[i];
        return GPUTX_OK;
    }
    case GPUTX_TBL_SUB_ACCESS_INFO: {
        // rows live = those indexed; read index to find them
        std::vector<unsigned long long> hk;
        std::vector<uint32_t> hr;
        st = get_col(db, hk, d.ai_idx.keys, (int64_t)d.ai_idx.mask + 1);
        if (!st) st = get_col(db, hr, d.ai_idx.rows, (int64_t)d.ai_idx.mask + 1);
        if (st) return st;
        std::vector<int32_t> data, sid, ty;
        const int64_t cap = 4 * d.n_sub;
        st = get_col(db, data, d.ai_data, cap * 4);
        if (!st) st = get_col(db, sid, d.ai_sid, cap);
        if (!st) st = get_col(db, ty, d.ai_type, cap);
        if (st) return st;
        std::vector<uint32_t> live;
        for (size_t i = 0; i < hk.size(); i++)
            if (hk[i] != HKEY_EMPTY && hk[i] != HKEY_TOMB) live.push_back(hr[i]);
        std::sort(live.begin(), live.end());
        *n_rows = live.size();
        if (!rows) return GPUTX_OK;
        if (capacity_rows < live.size()) return fail(db, GPUTX_EINVAL, "capacity");
        for (size_t i = 0; i < live.size(); i++) {
            const uint32_t r = live[i];
            int64_t *o = rows + i * f;
            o[0] = sid[r]; o[1] = ty[r];
            for (int j = 0; j < 4; j++) o[2 + j] = data[(size_t)r * 4 + j];
        }
        return GPUTX_OK;
    }
    case GPUTX_TBL_SUB_SPECIAL_FACILITY: {
        std::vector<unsigned long long> hk;
        std::vector<uint32_t> hr;
        st = get_col(db, hk, d.sf_idx.keys, (int64_t)d.sf_idx.mask + 1);
        if (!st) st = get_col(db, hr, d.sf_idx.rows, (int64_t)d.sf_idx.mask + 1);
        if (st) return st;
        const int64_t cap = 4 * d.n_sub;
        add32(d.sf_sid, cap); add32(d.sf_type, cap); add32(d.sf_active, cap);
        add32(d.sf_err, cap); add32(d.sf_data_a, cap); add32(d.sf_data_b, cap);
        if (st) return st;
        keep.assign((size_t)cap, 0);
        for (size_t i = 0; i < hk.size(); i++)
            if (hk[i] != HKEY_EMPTY && hk[i] != HKEY_TOMB) keep[hr[i]] = 1;
        break;
    }
    case GPUTX_TBL_SUB_CALL_FORWARDING: {
        const int64_t n = std::min<int64_t>(cur.cf, d.child_cap);
        add32(d.cf_sid, n); add32(d.cf_type, n); add32(d.cf_start, n); add32(d.cf_end, n);
        add32(d.cf_numberx, n);
        if (!st) st = get_col(db, keep, d.cf_live, n);
        break;
    }
    case GPUTX_TBL_OE_WAREHOUSE: add64(d.w_tax, d.n_wh); add64(d.w_ytd, d.n_wh); break;
    case GPUTX_TBL_OE_DISTRICT: {
        const int64_t n = d.n_wh * OE_DIST;
        add64(d.d_tax, n); add64(d.d_ytd, n); add64(d.d_next_o_id, n);
        break;
    }
    case GPUTX_TBL_OE_CUSTOMER: {
        const int64_t n = d.n_wh * OE_DIST * OE_CUST;
        add64(d.c_discount, n); add64(d.c_balance, n); add64(d.c_ytd, n); add64(d.c_payment_cnt, n);
        add64(d.c_last_o_id, n);
        break;
    }
    case GPUTX_TBL_OE_ITEM: add64(d.i_price, d.n_items); break;
    case GPUTX_TBL_OE_STOCK: {
        const int64_t n = d.n_wh * d.n_items;
        add32(d.s_quantity, n); add64(d.s_ytd, n); add32(d.s_order_cnt, n);
        break;
    }
    case GPUTX_TBL_OE_ORDER:
    case GPUTX_TBL_OE_ORDER_LINE: {
        const int64_t n = std::min<int64_t>(cur.ord, d.ord_cap);
        std::vector<int32_t> ow, od, oc, ocnt;
        std::vector<int64_t> oid, ofirst;
        std::vector<uint8_t> olive;
        st = get_col(db, ow, d.o_w, n);
        if (!st) st = get_col(db, od, d.o_d, n);
        if (!st) st = get_col(db, oc, d.o_c, n);
        if (!st) st = get_col(db, ocnt, d.o_cnt, n);
        if (!st) st = get_col(db, oid, d.o_id, n);
        if (!st) st = get_col(db, ofirst, d.o_first, n);
        if (!st) st = get_col(db, olive, d.o_live, n);
        if (st) return st;
        if (table == GPUTX_TBL_OE_ORDER) {
            cols = {std::vector<int64_t>(ow.begin(), ow.end()), std::vector<int64_t>(od.begin(), od.end()),
                    oid, std::vector<int64_t>(oc.begin(), oc.end()),
                    std::vector<int64_t>(ocnt.begin(), ocnt.end())};
            keep = olive;
            break;
        }
        const int64_t nl = std::min<int64_t>(cur.ol, d.ol_cap);
        std::vector<int32_t> li, ls, lq;
        std::vector<int64_t> la;
        st = get_col(db, li, d.ol_item, nl);
        if (!st) st = get_col(db, ls, d.ol_sw, nl);
        if (!st) st = get_col(db, lq, d.ol_qty, nl);
        if (!st) st = get_col(db, la, d.ol_amount, nl);
        if (st) return st;
        size_t total = 0;
        for (int64_t i = 0; i < n; i++)
            if (olive[i]) total += (size_t)ocnt[i];
        *n_rows = total;
        if (!rows) return GPUTX_OK;
        if (capacity_rows < total) return fail(db, GPUTX_EINVAL, "capacity");
        size_t r = 0;
        for (int64_t i = 0; i < n; i++) {
            if (!olive[i]) continue;
            for (int j = 0; j < ocnt[i]; j++, r++) {
                const int64_t l = ofirst[i] + j;
                int64_t *o = rows + r * f;
                o[0] = ow[i]; o[1] = od[i]; o[2] = oid[i];
                o[3] = li[l]; o[4] = ls[l]; o[5] = lq[l]; o[6] = la[l];
            }
        }
        return GPUTX_OK;
    }
    default:
        return fail(db, GPUTX_EINVAL, "table %d", table);
    }
    if (st) return st;
    if ((int)cols.size() != f) return fail(db, GPUTX_EINVAL, "table %d has no schema", table);
    const int64_t n = cols.empty() ? 0 : (int64_t)cols[0].size();
    size_t live = 0;
    for (int64_t i = 0; i < n; i++) live += keep.empty() || keep[i];
    *n_rows = live;
    if (!rows) return GPUTX_OK;
    if (capacity_rows < live) return fail(db, GPUTX_EINVAL, "capacity %zu < %zu rows", capacity_rows, live);
    size_t r = 0;
    for (int64_t i = 0; i < n; i++) {
        if (!keep.empty() && !keep[i]) continue;
        for (int j = 0; j < f; j++) rows[r * f + j] = cols[j][i];
        r++;
    }
    return GPUTX_OK;
}

gputx_status gputx_submit_bulk(gputx_db *db, const int64_t *ts, const int32_t *type, const int64_t *params,
                               int params_per_txn, size_t n, int mem, gputx_bulk **out)
{
    if (!db || !out) return fail(db, GPUTX_EINVAL, "bad arguments");
    *out = nullptr;
    if (n > 0 && (!ts || !type || !params)) return fail(db, GPUTX_EINVAL, "null bulk array");
    if ((int64_t)n > db->cfg.max_bulk) return fail(db, GPUTX_EINVAL, "bulk of %zu above max_bulk", n);
    if (params_per_txn < 1 || params_per_txn > 64) return fail(db, GPUTX_EINVAL, "params_per_txn");
    if (mem != GPUTX_MEM_HOST && mem != GPUTX_MEM_DEVICE) return fail(db, GPUTX_EINVAL, "mem");
    if (!db->dev.registered) return fail(db, GPUTX_ESTATE, "no registered types");
    gputx_bulk *b = new (std::nothrow) gputx_bulk();
    if (!b) return fail(db, GPUTX_ENOMEM, "host allocation");
    b->db = db;
    b->n = (int64_t)n;
    b->P = params_per_txn;
    b->R = db->dev.out_width;
    b->stream = db->pool[db->next_pool];
    db->next_pool = (db->next_pool + 1) % gputx_db::kPool;
    // the bulk's stream starts after what the caller queued on the database
    // stream (device inputs may be produced there)
    cudaError_t e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (!e) e = cudaEventRecord(b->ev_in, db->stream);
    if (!e) e = cudaStreamWaitEvent(b->stream, b->ev_in, 0);
    if (e) {
        if (b->ev_in) cudaEventDestroy(b->ev_in);
        delete b;
        return cuda_fail(db, e, "bulk stream");
    }
    const bool dev_in = mem == GPUTX_MEM_DEVICE;
    b->arena_bytes = carve_bulk(b, nullptr, dev_in);
    e = cudaMallocAsync(&b->arena, b->arena_bytes, b->stream);
    if (e != cudaSuccess) {
        cudaEventDestroy(b->ev_in);
        delete b;
        return cuda_fail(db, e, "bulk allocation");
    }
    carve_bulk(b, (char *)b->arena, dev_in);
    if (dev_in) {
        // referenced in place: the caller keeps them unchanged until the sync
        b->ts = const_cast<int64_t *>(ts);
        b->type = const_cast<int32_t *>(type);
        b->params = const_cast<int64_t *>(params);
    } else if (n > 0) {
        e = cudaMemcpyAsync(b->ts, ts, n * sizeof(int64_t), cudaMemcpyHostToDevice, b->stream);
        if (!e) e = cudaMemcpyAsync(b->type, type, n * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream);
        if (!e) e = cudaMemcpyAsync(b->params, params, n * params_per_txn * sizeof(int64_t),
                                    cudaMemcpyHostToDevice, b->stream);
    }
    if (!e) e = cudaMemsetAsync(b->ctl, 0, sizeof(BulkCtl), b->stream);
    if (!e && n > 0) e = cudaMemsetAsync(b->out, 0, n * b->R * sizeof(int64_t), b->stream);
    if (!e && n > 0) e = cudaMemsetAsync(b->status, 0, n * sizeof(int32_t), b->stream);
    if (!e) e = cudaEventCreate(&b->ev[7]);
    if (e) {
        cudaFreeAsync(b->arena, b->stream);
        cudaEventDestroy(b->ev_in);
        delete b;
        return cuda_fail(db, e, "bulk upload");
    }
    *out = b;
    return GPUTX_OK;
}

namespace {

// key bits of the largest object id the registered types can extract under
// `mode` (objects are numbered small root tables first)
int key_bits(const gputx_db *db, int mode)
{
    const DevDB &d = db->dev;
    const uint32_t reg = d.registered;
    uint64_t top = 1;
    if (reg & 1u) top = std::max<uint64_t>(top, mode == GPUTX_CONFLICT_ADD ? (uint64_t)d.o_acc + d.n_acc
                                                                           : (uint64_t)d.o_br + d.n_br);
    if (reg & 0xFEu) top = std::max<uint64_t>(top, (uint64_t)d.o_sub + d.n_sub);
    if (reg & 0x700u) top = std::max<uint64_t>(top, (uint64_t)d.n_objects);
    return std::max(1, bits_for(top - 1));
}

gputx_status run_kset_analysis(gputx_bulk *b, int mode, int part_size, uint32_t *&sk, uint32_t *&sv,
                               uint32_t *&ak, uint32_t *&av, int64_t &m)
{
    gputx_db *db = b->db;
    CK(cudaMemsetAsync(&b->ctl->cross, 0, 4, b->stream), "extract");
    CK(launch_extract(b, mode, part_size, nullptr, nullptr, true), "extract");
    m = b->n * db->uniform_k;
    if (!db->uniform_k) {
        uint32_t mm = 0;
        CK(cudaMemcpyAsync(&mm, b->sc.op_off + b->n, sizeof mm, cudaMemcpyDeviceToHost, b->stream), "ops");
        CK(cudaStreamSynchronize(b->stream), "ops");
        m = mm;
        if (m > b->sc.m_cap) m = b->sc.m_cap;
    }
    if (b->timing) cudaEventRecord(b->ev[1], b->stream);
    sk = b->sc.keys_a; sv = b->sc.vals_a; ak = b->sc.keys_b; av = b->sc.vals_b;
    CK(launch_sort(b, sk, sv, ak, av, m, key_bits(db, mode)), "sort");
    if (b->timing) cudaEventRecord(b->ev[2], b->stream);
    return GPUTX_OK;
}

// The database-touching tail of a bulk starts after the previous bulk's tail
// (bulks apply in gputx_execute order); the analysis before it overlaps.
cudaError_t begin_tail(gputx_bulk *b)
{
    cudaError_t e = cudaStreamWaitEvent(b->stream, b->db->last_done, 0);
    if (e) return e;
    return launch_begin(b);
}

cudaError_t end_tail(gputx_bulk *b)
{
    gputx_db *db = b->db;
    cudaError_t e = launch_finish(b);
    if (!e) e = cudaEventRecord(db->last_done, b->stream);
    if (!e) e = cudaEventRecord(b->ev[7], b->stream);
    // callers that order work on the database stream see the bulk as done
    if (!e) e = cudaStreamWaitEvent(db->stream, db->last_done, 0);
    return e;
}

// relaxed PART's counters: allocated once, for every possible partition
gputx_status part_scratch(gputx_db *db, int64_t roots)
{
    if (db->part_cnt) return GPUTX_OK;
    const int64_t tiles = (roots + 2047) / 2048;   // scan tiles of 2,048 counters
    gputx_status st = dalloc(db, &db->part_cnt, roots, "part counters");
    if (!st) st = dalloc(db, &db->part_off, roots + 1, "part counters");
    if (!st) st = dalloc(db, &db->part_scan_status, tiles, "part counters");
    if (!st) st = dalloc(db, &db->part_tile_ctr, 1, "part counters");
    if (st) return st;
    CK(cudaStreamSynchronize(db->stream), "part counters");
    db->part_cnt_n = roots;
    return GPUTX_OK;
}

}  // namespace

gputx_status gputx_execute(gputx_db *db, gputx_bulk *b, int strategy, const gputx_exec_opts *opts)
{
    if (!db || !b || b->db != db) return fail(db, GPUTX_EINVAL, "bad arguments");
    if (b->executed) return fail(db, GPUTX_ESTATE, "bulk already executed");
    if (strategy < GPUTX_KSET || strategy > GPUTX_TPL_RELAXED) return fail(db, GPUTX_EINVAL, "strategy %d", strategy);
    if (strategy == GPUTX_SCAN && db->dev.registered != (1u << GPUTX_T_DC_DEBIT_CREDIT))
        return fail(db, GPUTX_EINVAL, "SCAN needs a database whose only registered type is debit-credit");
    const int mode = opts ? opts->conflict_mode : GPUTX_CONFLICT_PAPER;
    if (mode != GPUTX_CONFLICT_PAPER && mode != GPUTX_CONFLICT_ADD) return fail(db, GPUTX_EINVAL, "conflict mode");
    int block = (opts && opts->block_threads) ? opts->block_threads : db->cfg.block_threads;
    if (block < 32 || block > 1024 || block % 32) return fail(db, GPUTX_EINVAL, "block_threads");
    int part_size = (opts && opts->part_size) ? opts->part_size : db->cfg.part_size;
    if (part_size <= 0) part_size = (db->dev.n_sub > 0 && db->dev.n_acc == 0 && db->dev.n_wh == 0) ? 128 : 1;
    b->executed = true;
    b->timing = opts && opts->timing;
    if (b->timing)
        for (int i = 0; i < 7; i++)
            if (!b->ev[i]) cudaEventCreate(&b->ev[i]);
    cudaStream_t s = b->stream;
    if (b->timing) cudaEventRecord(b->ev[0], s);
    CK(launch_insert_slots(b), "insert slots");
    const bool add = mode == GPUTX_CONFLICT_ADD;
    gputx_status st = GPUTX_OK;
    uint32_t *sk = nullptr, *sv = nullptr, *ak = nullptr, *av = nullptr;
    int64_t m = 0;
    int run = strategy;

    // AUTO on a database whose only registered type is debit-credit: the
    // segmented-sum strategy gives Definition 1's results bit for bit and
    // moves each transaction once, whatever the depth of its graph
    if (strategy == GPUTX_AUTO && db->dev.registered == (1u << GPUTX_T_DC_DEBIT_CREDIT)) run = GPUTX_SCAN;
    if (strategy == GPUTX_KSET || (strategy == GPUTX_AUTO && run == GPUTX_AUTO)) {
        if ((st = run_kset_analysis(b, mode, part_size, sk, sv, ak, av, m))) return st;
        CK(launch_rank_scan(b, sk, sv, m, db->need_fixpoint), "rank");
        // AUTO decides on the one-pass ranks first: w0 and c are exact there
        // (a transaction is a source exactly when all its operations have
        // rank 0), and the one-pass depth bounds the exact one from below.
        // The exact-depth pass runs only once K-SET is chosen.
        if (db->need_fixpoint && strategy == GPUTX_KSET) CK(launch_exact_depth(b, sv, m), "exact depth");
        CK(launch_level_stats(b), "stats");
        if ((st = read_ctl(b))) return st;
        if (b->host_ctl.err) {
            CK(cudaEventRecord(b->ev[7], s), "event");
            return GPUTX_OK;     // reported by the sync
        }
        if (strategy == GPUTX_AUTO) {
            // Algorithm 1 (Appendix D): wide 0-set -> K-SET; else few
            // cross-partition transactions or a deep graph -> PART; else TPL
            const int64_t w0 = b->host_ctl.w0, d = b->host_ctl.depth, c = b->host_ctl.cross;
            if (w0 >= db->cfg.kset_w0_min) run = GPUTX_KSET;
            else if (c <= db->cfg.part_c_max || d >= db->cfg.part_d_min) run = c ? GPUTX_TPL : GPUTX_PART;
            else run = GPUTX_TPL;
            // a PART pick with cross-partition transactions runs as TPL
            // (Section 5.2); the sorted operations are reused for tickets
            if (run == GPUTX_TPL && c && (c <= db->cfg.part_c_max || d >= db->cfg.part_d_min))
                b->fallback = 1;
            if (run == GPUTX_KSET && db->need_fixpoint) {
                // exact depths for the level schedule (Property 1)
                CK(launch_exact_depth(b, sv, m), "exact depth");
                CK(cudaMemsetAsync(&b->ctl->depth, 0, 2 * sizeof(uint32_t), s), "stats");
                CK(launch_level_stats(b), "stats");
                if ((st = read_ctl(b))) return st;
                if (b->host_ctl.err) {
                    CK(cudaEventRecord(b->ev[7], s), "event");
                    return GPUTX_OK;
                }
            }
        }
    }
    if (run == GPUTX_KSET) {
        const int64_t depth = b->host_ctl.depth;
        const bool persistent = opts && opts->kset_launch == 1;
        // regroup by (level, type): reuse the free op buffers
        uint32_t *rk = ak, *rv = av, *rk2 = sk, *rv2 = sv;
        CK(launch_regroup_keys(b, rk, rv), "regroup");
        CK(launch_sort(b, rk, rv, rk2, rv2, b->n, bits_for((uint64_t)depth) + db->tbits), "regroup sort");
        CK(launch_level_tables(b, rk, depth, block, persistent), "level tables");
        if (persistent) {
            CK(launch_gather(b, rv), "gather");
            CK(begin_tail(b), "order");
            if (b->timing) cudaEventRecord(b->ev[3], s);
            CK(launch_kset(b, rv, b->sc.chunk_cap, block, add), "k-set execute");
        } else if (b->n > 0) {
            // plan launches from the level widths
            b->level_off_host.resize((size_t)depth + 2);
            CK(cudaMemcpyAsync(b->level_off_host.data(), b->sc.level_off, (depth + 2) * sizeof(uint32_t),
                               cudaMemcpyDeviceToHost, s), "level plan");
            if (b->sc.type_cut) {
                b->type_cut_host.resize(3 * ((size_t)depth + 1));
                CK(cudaMemcpyAsync(b->type_cut_host.data(), b->sc.type_cut, 3 * (depth + 1) * sizeof(uint32_t),
                                   cudaMemcpyDeviceToHost, s), "level plan");
            }
            CK(cudaMemcpyAsync(&b->host_ctl.err, &b->ctl->err, 4, cudaMemcpyDeviceToHost, s), "level plan");
            CK(cudaStreamSynchronize(s), "level plan");
            if (!b->host_ctl.err) {
                const int narrow = (opts && opts->narrow_max > 0) ? opts->narrow_max : 8192;
                // debit-credit-only bulks run from packed records
                const bool dc_only = b->sc.rec_dc != nullptr;
                if (dc_only) CK(launch_gather_dc(b, rv), "gather");
                else CK(launch_gather(b, rv), "gather");
                CK(begin_tail(b), "order");
                if (b->timing) cudaEventRecord(b->ev[3], s);
                CK(launch_kset_levels(b, b->level_off_host.data(), depth, narrow, add,
                                      dc_only ? b->sc.rec_dc : nullptr,
                                      b->sc.type_cut ? b->type_cut_host.data() : nullptr),
                   "k-set execute");
            }
        } else {
            CK(begin_tail(b), "order");   // empty bulk
        }
    } else if (run == GPUTX_PART) {
        // partition ids by root key (Section 5.2 step 1), stable sort (step 2)
        uint32_t *pk = b->sc.pid_key, *pv = b->sc.pid_val, *pk2 = b->sc.pid_key2, *pv2 = b->sc.pid_val2;
        CK(cudaMemsetAsync(&b->ctl->cross, 0, 4, s), "part");
        CK(launch_extract(b, mode, part_size, pk, pv, false), "extract");
        if (b->timing) cudaEventRecord(b->ev[1], s);
        if ((st = read_ctl(b))) return st;
        if (b->host_ctl.err) {
            CK(cudaEventRecord(b->ev[7], s), "event");
            return GPUTX_OK;
        }
        if (b->host_ctl.cross > 0) {
            // Section 5.2: cross-partition transactions run with TPL
            b->fallback = 1;
            run = GPUTX_TPL;
            CK(cudaMemsetAsync(&b->ctl->cross, 0, 4, s), "part");
        } else {
            const int64_t roots = std::max<int64_t>({db->dev.n_br, db->dev.n_sub, db->dev.n_wh, 1});
            const int bits = bits_for((uint64_t)((roots - 1) / part_size));
            CK(launch_sort(b, pk, pv, pk2, pv2, b->n, bits), "partition sort");
            if (b->timing) cudaEventRecord(b->ev[2], s);
            CK(launch_part_heads(b, pk, b->n), "partition heads");
            if (part_dc_applies(db, part_size)) CK(launch_gather_dc(b, pv), "gather");
            else CK(launch_gather(b, pv), "gather");
            CK(begin_tail(b), "order");
            if (b->timing) cudaEventRecord(b->ev[3], s);
            CK(launch_part(b, pk, 128, (roots + part_size - 1) / part_size, part_size), "part execute");
        }
    }
    if (run == GPUTX_PART_RELAXED) {
        // Appendix G: counters instead of the sort.  The counters are the
        // database's, so all of it runs in the bulk's ordered tail.
        const int64_t roots = std::max<int64_t>({db->dev.n_br, db->dev.n_sub, db->dev.n_wh, 1});
        const int64_t parts = (roots + part_size - 1) / part_size;
        if ((st = part_scratch(db, roots))) return st;
        CK(begin_tail(b), "order");
        CK(cudaMemsetAsync(db->part_cnt, 0, parts * sizeof(uint32_t), s), "part counters");
        uint32_t *pid_of = b->sc.pid_key, *key_of = b->sc.pid_val, *pk = b->sc.pid_key2, *order = b->sc.pid_val2;
        CK(launch_part_count(b, mode, part_size, db->part_cnt, parts, pid_of, key_of), "part count");
        if (b->timing) cudaEventRecord(b->ev[1], s);
        if ((st = read_ctl(b))) return st;
        if (b->host_ctl.err) {
            CK(end_tail(b), "finish");
            b->strategy_run = run;
            return GPUTX_OK;   // reported by the sync
        }
        if (b->host_ctl.cross > 0) {
            b->fallback = 1;   // cross-partition transactions: spin-lock TPL
            run = GPUTX_TPL_RELAXED;
        } else {
            CK(launch_part_offsets(b, db->part_cnt, db->part_off, parts, db->part_scan_status, db->part_tile_ctr),
               "part offsets");
            CK(launch_part_scatter(b, db->part_off, pid_of, key_of, pk, order), "part scatter");
            if (b->timing) cudaEventRecord(b->ev[2], s);
            CK(launch_part_heads(b, pk, b->n), "partition heads");
            if (part_dc_applies(db, part_size)) CK(launch_gather_dc(b, order), "gather");
            else CK(launch_gather(b, order), "gather");
            if (b->timing) cudaEventRecord(b->ev[3], s);
            CK(launch_part(b, pk, 128, parts, part_size), "part execute");
            b->serial_order = order;
        }
    }
    if (run == GPUTX_TPL_RELAXED) {
        if (strategy == GPUTX_TPL_RELAXED) {
            if (b->timing) cudaEventRecord(b->ev[1], s);
            CK(launch_validate(b), "validate");
            if (b->timing) cudaEventRecord(b->ev[2], s);
            CK(begin_tail(b), "order");
        }
        if (b->timing) cudaEventRecord(b->ev[3], s);
        CK(launch_tpl_relaxed(b, b->sc.level, add), "tpl execute");
        b->serial_order = b->sc.level;
    }
    if (run == GPUTX_SCAN) {
        if ((st = run_kset_analysis(b, GPUTX_CONFLICT_ADD, part_size, sk, sv, ak, av, m))) return st;
        CK(begin_tail(b), "order");
        if (b->timing) cudaEventRecord(b->ev[3], s);
        CK(launch_scan_exec(b, sk, sv, m), "scan execute");
    }
    if (run == GPUTX_TPL) {
        if (!sk) {
            if ((st = run_kset_analysis(b, mode, part_size, sk, sv, ak, av, m))) return st;
        }
        CK(launch_ticket_scan(b, sk, sv, m), "tickets");
        CK(begin_tail(b), "order");
        if (b->timing) cudaEventRecord(b->ev[3], s);
        CK(launch_tpl(b, block, add), "tpl execute");
        if (b->timing) cudaEventRecord(b->ev[4], s);
        CK(launch_tpl_reset(b, sk, m), "tpl reset");
    }
    if (b->timing && run != GPUTX_TPL) cudaEventRecord(b->ev[4], s);
    CK(end_tail(b), "finish");
    b->strategy_run = run;
    return GPUTX_OK;
}

gputx_status gputx_sync_bulk(gputx_bulk *b, gputx_exec_stats *stats)
{
    if (!b) return GPUTX_EINVAL;
    gputx_db *db = b->db;
    if (!b->executed) return fail(db, GPUTX_ESTATE, "bulk not executed");
    CK(cudaEventSynchronize(b->ev[7]), "sync");
    CK(cudaMemcpy(&b->host_ctl, b->ctl, sizeof(BulkCtl), cudaMemcpyDeviceToHost), "sync");
    b->synced = true;
    if (stats) {
        memset(stats, 0, sizeof *stats);
        stats->strategy = b->strategy_run;
        stats->fallback = b->fallback;
        stats->n = b->n;
        stats->n_ops = b->sc.m_cap;
        stats->depth = b->host_ctl.depth;
        stats->w0 = b->host_ctl.w0;
        stats->cross = b->host_ctl.cross;
        stats->fixpoint_rounds = b->host_ctl.rounds;
        if (b->timing) {
            float ms = 0;
            if (!cudaEventElapsedTime(&ms, b->ev[0], b->ev[3])) stats->ms_analysis = ms;
            if (!cudaEventElapsedTime(&ms, b->ev[1], b->ev[2])) stats->ms_sort = ms;
            if (!cudaEventElapsedTime(&ms, b->ev[3], b->ev[4])) stats->ms_execute = ms;
            if (!cudaEventElapsedTime(&ms, b->ev[0], b->ev[7])) stats->ms_total = ms;
            cudaGetLastError();   // a phase this strategy does not have leaves its events unrecorded
        }
    }
    return bulk_error(db, b->host_ctl.err);
}

gputx_status gputx_bulk_order(gputx_bulk *b, uint32_t *order, size_t n)
{
    if (!b) return GPUTX_EINVAL;
    gputx_db *db = b->db;
    if ((int64_t)n != b->n) return fail(db, GPUTX_EINVAL, "n %zu != bulk size %lld", n, (long long)b->n);
    if (n && !order) return fail(db, GPUTX_EINVAL, "null order");
    gputx_status st = gputx_sync_bulk(b, nullptr);
    if (st) return st;
    if (!b->serial_order) {
        for (size_t i = 0; i < n; i++) order[i] = (uint32_t)i;   // timestamp order (Definition 1)
        return GPUTX_OK;
    }
    CK(cudaMemcpy(order, b->serial_order, n * sizeof(uint32_t), cudaMemcpyDeviceToHost), "d2h");
    return GPUTX_OK;
}

gputx_status gputx_read_results(gputx_bulk *b, int32_t *status, int64_t *values, size_t n, int n_values)
{
    if (!b) return GPUTX_EINVAL;
    gputx_db *db = b->db;
    if ((int64_t)n != b->n) return fail(db, GPUTX_EINVAL, "n %zu != bulk size %lld", n, (long long)b->n);
    if (values && n_values != b->R) return fail(db, GPUTX_EINVAL, "output width is %d", b->R);
    gputx_status st = gputx_sync_bulk(b, nullptr);
    if (st) return st;
    if (n == 0) return GPUTX_OK;
    if (status) CK(cudaMemcpyAsync(status, b->status, n * sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream), "d2h");
    if (values)
        CK(cudaMemcpyAsync(values, b->out, n * b->R * sizeof(int64_t), cudaMemcpyDeviceToHost, b->stream), "d2h");
    CK(cudaStreamSynchronize(b->stream), "d2h");
    return GPUTX_OK;
}

gputx_status gputx_bulk_results_device(gputx_bulk *b, const int32_t **status, const int64_t **values)
{
    if (!b) return GPUTX_EINVAL;
    if (status) *status = b->status;
    if (values) *values = b->out;
    return GPUTX_OK;
}

void gputx_free_bulk(gputx_bulk *b)
{
    if (!b) return;
    if (b->arena) cudaFreeAsync(b->arena, b->stream);
    for (int i = 0; i < 8; i++)
        if (b->ev[i]) cudaEventDestroy(b->ev[i]);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    delete b;
}

// ---------------------------------------------------------------------------
// allocation-free K-SET execution (see gputx_execute_kset_noalloc)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

// The working memory of gputx_execute_kset_noalloc: one array per device,
// resident for the life of the process.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GPUTX_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// device address of the scratch array for the current device (set-up once per
// device, with that device current)
gputx_status noalloc_scratch(gputx_db *db, void **out)
{
    int dev = 0;
    CK(cudaGetDevice(&dev), "get device");
    if (dev < 0 || dev >= kMaxDevices) return fail(db, GPUTX_ECUDA, "device index %d", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(db, e ? e : cudaErrorInvalidSymbol, "scratch address");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return GPUTX_OK;
}

}  // namespace

extern "C" gputx_status gputx_execute_kset_noalloc(gputx_db *db, const int64_t *ts, const int32_t *type,
                                                   const int64_t *params, int params_per_txn, size_t n,
                                                   int conflict_mode, int32_t *status, int64_t *values)
{
    if (!db) return GPUTX_EINVAL;
    if (n > 0 && (!ts || !type || !params || !status || !values)) return fail(db, GPUTX_EINVAL, "null array");
    if (params_per_txn < 1 || params_per_txn > 64) return fail(db, GPUTX_EINVAL, "params_per_txn");
    if ((int64_t)n > db->cfg.max_bulk) return fail(db, GPUTX_EINVAL, "bulk above max_bulk");
    if (conflict_mode != GPUTX_CONFLICT_PAPER && conflict_mode != GPUTX_CONFLICT_ADD)
        return fail(db, GPUTX_EINVAL, "conflict mode");
    if (!db->dev.registered) return fail(db, GPUTX_ESTATE, "no registered types");
    void *scratch = nullptr;
    gputx_status st = noalloc_scratch(db, &scratch);
    if (st) return st;

    // a bulk whose arrays all live in the scratch array (inputs and outputs
    // stay in the caller's buffers)
    gputx_bulk b;
    b.db = db;
    b.n = (int64_t)n;
    b.P = params_per_txn;
    b.R = db->dev.out_width;
    const size_t need = carve_bulk(&b, nullptr, true);
    if (need > GPUTX_NOALLOC_SCRATCH_BYTES)
        return fail(db, GPUTX_EINVAL, "bulk needs %zu bytes of working memory, the no-allocation area has %u",
                    need, (unsigned)GPUTX_NOALLOC_SCRATCH_BYTES);
    carve_bulk(&b, (char *)scratch, true);
    b.stream = db->stream;
    b.ts = const_cast<int64_t *>(ts);
    b.type = const_cast<int32_t *>(type);
    b.params = const_cast<int64_t *>(params);
    b.status = status;
    b.out = values;
    cudaStream_t s = db->stream;
    // the array keeps the previous call's contents: clear what starts at zero
    CK(cudaMemsetAsync(b.ctl, 0, sizeof(BulkCtl), s), "clear");
    if (n > 0) {
        CK(cudaMemsetAsync(values, 0, n * b.R * sizeof(int64_t), s), "clear");
        CK(cudaMemsetAsync(status, 0, n * sizeof(int32_t), s), "clear");
    }
    const bool add = conflict_mode == GPUTX_CONFLICT_ADD;
    const int block = db->cfg.block_threads;
    CK(cudaStreamWaitEvent(s, db->last_done, 0), "order");
    CK(launch_begin(&b), "begin");
    CK(launch_insert_slots(&b), "insert slots");
    CK(cudaMemsetAsync(&b.ctl->cross, 0, 4, s), "extract");
    CK(launch_extract(&b, conflict_mode, 1, nullptr, nullptr, true), "extract");
    int64_t m = b.n * db->uniform_k;
    if (!db->uniform_k) {
        uint32_t mm = 0;
        CK(cudaMemcpyAsync(&mm, b.sc.op_off + b.n, sizeof mm, cudaMemcpyDeviceToHost, s), "ops");
        CK(cudaStreamSynchronize(s), "ops");
        m = mm > (uint32_t)b.sc.m_cap ? b.sc.m_cap : mm;
    }
    uint32_t *sk = b.sc.keys_a, *sv = b.sc.vals_a, *ak = b.sc.keys_b, *av = b.sc.vals_b;
    CK(launch_sort(&b, sk, sv, ak, av, m, key_bits(db, conflict_mode)), "sort");
    CK(launch_rank_scan(&b, sk, sv, m, db->need_fixpoint), "rank");
    if (db->need_fixpoint) CK(launch_exact_depth(&b, sv, m), "exact depth");
    CK(launch_level_stats(&b), "stats");
    if ((st = read_ctl(&b))) return st;
    if (b.host_ctl.err) return bulk_error(db, b.host_ctl.err);
    const int64_t depth = b.host_ctl.depth;
    uint32_t *rk = ak, *rv = av, *rk2 = sk, *rv2 = sv;
    CK(launch_regroup_keys(&b, rk, rv), "regroup");
    CK(launch_sort(&b, rk, rv, rk2, rv2, b.n, bits_for((uint64_t)depth) + db->tbits), "regroup sort");
    CK(launch_level_tables(&b, rk, depth, block, true), "level tables");
    CK(launch_gather(&b, rv), "gather");
    CK(launch_kset(&b, rv, b.sc.chunk_cap, block, add), "k-set execute");
    CK(launch_finish(&b), "finish");
    CK(cudaEventRecord(db->last_done, s), "order");
    if ((st = read_ctl(&b))) return st;
    return bulk_error(db, b.host_ctl.err);
}
