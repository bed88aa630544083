// serve.cu -- a serving loop over the bulk engine (Section 3.2's transaction
// pool and bulk generator, Section 6.3's response time vs throughput).
//
// Clients submit transactions into a pool; the pool assigns each one the next
// id, which is its timestamp (Section 3.2).  A worker thread closes a bulk
// when the oldest pending transaction has waited `deadline_us` or `max_bulk`
// are pending, and hands it to gputx_execute.  Up to `max_inflight` bulks are
// on the device at once: the analysis of a new bulk runs while earlier bulks
// execute, and the database applies bulks in id order, so the served stream
// equals serial execution in id order (Definition 1 over the whole stream).
// Admission refuses work the pool, the insert areas or free device memory
// cannot hold.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// latency histogram: 1 us bins up to 1 s, then one overflow bin
struct LatencyHist {
    static constexpr int kBins = 1000000;
    std::vector<uint64_t> bins = std::vector<uint64_t>(kBins + 1, 0);
    uint64_t count = 0;
    double sum_us = 0;
    void add(int64_t ns)
    {
        int64_t us = ns / 1000;
        if (us < 0) us = 0;
        bins[us < kBins ? us : kBins]++;
        count++;
        sum_us += (double)ns / 1000.0;
    }
    double quantile(double q) const
    {
        if (!count) return 0;
        const uint64_t target = (uint64_t)(q * (double)(count - 1)) + 1;
        uint64_t acc = 0;
        for (int i = 0; i <= kBins; i++) {
            acc += bins[i];
            if (acc >= target) return (double)i + 0.5;
        }
        return (double)kBins;
    }
};

// memcpy of a large block split over a few threads: one host core copies
// well below what the memory system moves, and a served bulk of 2^20
// transactions moves tens of MB through these copies
void par_memcpy(void *dst, const void *src, size_t bytes)
{
    constexpr size_t kPart = size_t(4) << 20;
    constexpr int kMaxThreads = 8;
    const int parts = (int)std::min<size_t>(kMaxThreads, bytes / kPart);
    if (parts < 2) {
        std::memcpy(dst, src, bytes);
        return;
    }
    const size_t per = (bytes + parts - 1) / parts;
    std::thread th[kMaxThreads];
    for (int i = 1; i < parts; i++) {
        const size_t o = per * (size_t)i, k = std::min(per, bytes - o);
        try {
            th[i] = std::thread([=] { std::memcpy((char *)dst + o, (const char *)src + o, k); });
        } catch (...) {   // no thread to spare: this part on the caller
            std::memcpy((char *)dst + o, (const char *)src + o, k);
        }
    }
    std::memcpy(dst, src, std::min(per, bytes));
    for (int i = 1; i < parts; i++)
        if (th[i].joinable()) th[i].join();
}

// An append-only array stored in fixed-size chunks and indexed by absolute
// position: appending never moves what is already there (no reallocation
// copies while the server lock is held), and whole chunks below a position
// can be released.
template <class T> class Chunked {
    static constexpr int64_t kShift = 20, kChunk = int64_t(1) << kShift, kMask = kChunk - 1;
    std::vector<std::unique_ptr<T[]>> chunks_;   // chunks_[c - first_] holds [c * kChunk, (c + 1) * kChunk)
    int64_t first_ = 0;                          // chunks before this one were released
    int64_t size_ = 0;

    T *at(int64_t i) { return &chunks_[(i >> kShift) - first_][i & kMask]; }
    const T *at(int64_t i) const { return &chunks_[(i >> kShift) - first_][i & kMask]; }
    // calls f(pointer, count) for the pieces of [i, i + n) chunk by chunk
    template <class F> void pieces(int64_t i, int64_t n, F f)
    {
        while (n > 0) {
            const int64_t k = std::min(n, kChunk - (i & kMask));
            f(at(i), k);
            i += k;
            n -= k;
        }
    }

  public:
    int64_t size() const { return size_; }
    T &operator[](int64_t i) { return *at(i); }
    const T &operator[](int64_t i) const { return *at(i); }
    // n more elements, left unwritten: for arrays each element of which is
    // written before it is read
    void grow_uninit(int64_t n)
    {
        const int64_t end = size_ + n;
        while ((int64_t)(chunks_.size() + first_) * kChunk < end) chunks_.emplace_back(new T[kChunk]);
        size_ = end;
    }
    // n more elements, each `v`
    void grow(int64_t n, T v)
    {
        const int64_t at0 = size_;
        grow_uninit(n);
        fill(at0, n, v);
    }
    void append(const T *src, int64_t n)
    {
        const int64_t at0 = size_;
        grow(n, T());
        copy_in(at0, src, n);
    }
    void copy_in(int64_t i, const T *src, int64_t n)
    {
        pieces(i, n, [&](T *p, int64_t k) {
            par_memcpy(p, src, sizeof(T) * k);
            src += k;
        });
    }
    void copy_out(int64_t i, int64_t n, T *dst)
    {
        pieces(i, n, [&](T *p, int64_t k) {
            par_memcpy(dst, p, sizeof(T) * k);
            dst += k;
        });
    }
    void fill(int64_t i, int64_t n, T v)
    {
        pieces(i, n, [&](T *p, int64_t k) { std::fill(p, p + k, v); });
    }
    // frees the chunks that lie wholly below position i
    void release_before(int64_t i)
    {
        const int64_t c = std::min(i, size_) >> kShift;
        if (c <= first_) return;
        chunks_.erase(chunks_.begin(), chunks_.begin() + (c - first_));
        first_ = c;
    }
};

struct Slot {
    gputx_bulk *bulk = nullptr;
    int64_t first_id = 0;
    int64_t n = 0;
    int32_t *h_type = nullptr;
    int64_t *h_ts = nullptr, *h_params = nullptr, *h_values = nullptr;
    int32_t *h_status = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    int64_t inserts[4] = {0, 0, 0, 0};   // hist, cf, ord, ol reserved by this bulk
};

}  // namespace

struct gputx_server {
    gputx_db *db = nullptr;
    gputx_serve_config cfg{};
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    bool flush = false;               // drain: close bulks without waiting for deadlines
    gputx_status worker_status = GPUTX_OK;
    std::string worker_error;
    // the pool: pending transactions, ids next_consume .. next_id-1
    Chunked<int32_t> p_type;          // all indexed by id (params by id x P)
    Chunked<int64_t> p_params;
    Chunked<int64_t> p_arrival;
    Chunked<uint8_t> p_need;          // insert rows per transaction (packed, see pack_need)
    int64_t next_consume = 0;         // first id not yet in a bulk
    int64_t next_id = 0;              // next id to assign
    int64_t inflight_txns = 0;
    // insert accounting (rows reserved by pending + in-flight work, and used)
    int64_t ins_reserved[4] = {0, 0, 0, 0};
    int64_t ins_used[4] = {0, 0, 0, 0};
    int64_t ins_cap[4] = {0, 0, 0, 0};
    // results, indexed by id
    Chunked<int32_t> r_status;
    Chunked<int64_t> r_values;
    Chunked<int64_t> r_complete;
    Chunked<uint8_t> r_done;
    int64_t completed = 0, bulks = 0, max_bulk_seen = 0, refused = 0;
    int64_t first_arrival = -1, last_complete = 0;
    LatencyHist hist;
    std::vector<Slot> slots;
    std::deque<int> order;            // in-flight slots in execution order
    int R = 1, P = 1;
    // incremental 0-set mode: the device pool, and the oldest id not yet done
    gputx_pool *zpool = nullptr;
    int64_t oldest_open = 0;
};

namespace {

// rows of each append area one transaction takes (a history row per
// debit-credit transaction)
void insert_need(const gputx_server *s, int32_t type, const int64_t *p, int64_t need[4])
{
    (void)s;
    need[0] = type == GPUTX_T_DC_DEBIT_CREDIT ? 1 : 0;
    need[1] = type == GPUTX_T_SUB_INSERT_CF ? 1 : 0;
    need[2] = type == GPUTX_T_OE_NEW_ORDER ? 1 : 0;
    need[3] = type == GPUTX_T_OE_NEW_ORDER ? (p[3] > 0 && p[3] <= 15 ? p[3] : 0) : 0;
}

// call-forwarding (bit 0), order (bit 1), order-line rows (bits 2-5) and
// history (bit 6) of one transaction, packed at submission so a bulk's
// totals are a byte sum
inline uint8_t pack_need(const int64_t need[4])
{
    return (uint8_t)(need[1] | (need[2] << 1) | (need[3] << 2) | (need[0] << 6));
}

void sum_needs(gputx_server *s, int64_t first_id, int64_t n, int64_t out[4])
{
    int64_t cf = 0, ord = 0, ol = 0, hist = 0;
    for (int64_t i = first_id; i < first_id + n; i++) {
        const uint8_t q = s->p_need[i];
        cf += q & 1u;
        ord += (q >> 1) & 1u;
        ol += (q >> 2) & 15u;
        hist += q >> 6;
    }
    // a debit-credit-only database takes a row per bulk position
    out[0] = s->db->dev.registered == 1u ? n : hist;
    out[1] = cf;
    out[2] = ord;
    out[3] = ol;
}

gputx_status set_worker_error(gputx_server *s, gputx_status st, const char *what)
{
    s->worker_status = st;
    s->worker_error = std::string(what) + ": " + gputx_last_error(s->db);
    return st;
}

// frees the pool's chunks below id `keep_from` (no bulk needs them any more)
void release_pool_before(gputx_server *s, int64_t keep_from)
{
    s->p_type.release_before(keep_from);
    s->p_params.release_before(keep_from * s->P);
    s->p_arrival.release_before(keep_from);
    s->p_need.release_before(keep_from);
}

// reaps finished bulks in order (lock held)
void reap(gputx_server *s, bool block)
{
    while (!s->order.empty()) {
        Slot &sl = s->slots[s->order.front()];
        if (block) {
            s->mu.unlock();
            cudaEventSynchronize(sl.done);
            s->mu.lock();
        } else if (cudaEventQuery(sl.done) == cudaErrorNotReady) {
            return;
        }
        const int64_t t = now_ns();
        if (sl.bulk) {
            gputx_status st = gputx_sync_bulk(sl.bulk, nullptr);
            if (st != GPUTX_OK) set_worker_error(s, st, "bulk");
        }
        // a bulk is a contiguous id range: results move in block copies
        s->r_status.copy_in(sl.first_id, sl.h_status, sl.n);
        s->r_values.copy_in(sl.first_id * s->R, sl.h_values, sl.n * s->R);
        s->r_complete.fill(sl.first_id, sl.n, t);
        s->r_done.fill(sl.first_id, sl.n, (uint8_t)1);
        for (int64_t i = sl.first_id; i < sl.first_id + sl.n; i++) s->hist.add(t - s->p_arrival[i]);
        s->completed += sl.n;
        s->last_complete = t;
        s->inflight_txns -= sl.n;
        for (int k = 0; k < 4; k++) {
            s->ins_reserved[k] -= sl.inserts[k];
            s->ins_used[k] += sl.inserts[k];
        }
        if (sl.bulk) gputx_free_bulk(sl.bulk);
        sl.bulk = nullptr;
        sl.busy = false;
        s->order.pop_front();
        s->cv.notify_all();
    }
    // drop the pool's prefix no bulk still needs (arrivals of finished ids)
    const int64_t keep_from = s->order.empty() ? s->next_consume : s->slots[s->order.front()].first_id;
    release_pool_before(s, keep_from);
}

// cuts the next bulk [next_consume, next_consume + n) and launches it (lock
// held on entry and exit; released while the engine works)
void launch(gputx_server *s, int slot_idx, int64_t n)
{
    Slot &sl = s->slots[slot_idx];
    sl.first_id = s->next_consume;
    sl.n = n;
    sl.busy = true;
    s->p_type.copy_out(sl.first_id, n, sl.h_type);
    s->p_params.copy_out(sl.first_id * s->P, n * s->P, sl.h_params);
    sum_needs(s, sl.first_id, n, sl.inserts);
    for (int64_t i = 0; i < n; i++) sl.h_ts[i] = sl.first_id + i;
    s->next_consume += n;
    s->inflight_txns += n;
    s->bulks++;
    s->max_bulk_seen = std::max(s->max_bulk_seen, n);
    s->order.push_back(slot_idx);
    s->mu.unlock();
    gputx_bulk *b = nullptr;
    gputx_status st = gputx_submit_bulk(s->db, sl.h_ts, sl.h_type, sl.h_params, s->P, (size_t)n,
                                        GPUTX_MEM_HOST, &b);
    if (st == GPUTX_OK) {
        gputx_exec_opts o{};
        o.conflict_mode = s->cfg.conflict_mode;
        st = gputx_execute(s->db, b, s->cfg.strategy, &o);
    }
    if (st == GPUTX_OK) {
        // results come back asynchronously into this slot's pinned buffers
        const int32_t *ds = nullptr;
        const int64_t *dv = nullptr;
        gputx_bulk_results_device(b, &ds, &dv);
        cudaMemcpyAsync(sl.h_status, ds, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream);
        cudaMemcpyAsync(sl.h_values, dv, sizeof(int64_t) * n * s->R, cudaMemcpyDeviceToHost, b->stream);
        cudaEventRecord(sl.done, b->stream);
    }
    s->mu.lock();
    sl.bulk = b;
    if (st != GPUTX_OK) {
        set_worker_error(s, st, "launch");
        if (!b) cudaEventRecord(sl.done, s->db->stream);
        else cudaEventRecord(sl.done, b->stream);
        // no results were queued: complete the bulk with its error status
        for (int64_t i = 0; i < n; i++) sl.h_status[i] = -(int32_t)st;
        std::memset(sl.h_values, 0, sizeof(int64_t) * n * s->R);
    }
}

void worker_main(gputx_server *s)
{
    int dev = s->db->device;
    cudaSetDevice(dev);
    std::unique_lock<std::mutex> lk(s->mu);
    const int64_t deadline = s->cfg.deadline_us * 1000;
    while (true) {
        reap(s, false);
        const int64_t pending = s->next_id - s->next_consume;
        if (s->stop && pending == 0 && s->order.empty()) break;
        int free_slot = -1;
        for (int i = 0; i < (int)s->slots.size(); i++)
            if (!s->slots[i].busy) { free_slot = i; break; }
        bool ready = false;
        if (pending > 0) {
            const int64_t oldest = s->p_arrival[s->next_consume];
            ready = pending >= s->cfg.max_bulk || now_ns() - oldest >= deadline || s->stop || s->flush;
        }
        if (ready && free_slot >= 0) {
            launch(s, free_slot, std::min<int64_t>(pending, s->cfg.max_bulk));
            continue;
        }
        if (ready && free_slot < 0) {
            reap(s, true);   // every slot busy: wait for the oldest bulk
            continue;
        }
        // sleep until the oldest pending transaction reaches its deadline, a
        // submit arrives, or a bulk may have finished
        int64_t wait_ns = 200000;
        if (pending > 0) {
            const int64_t oldest = s->p_arrival[s->next_consume];
            wait_ns = std::max<int64_t>(0, oldest + deadline - now_ns());
        }
        if (!s->order.empty()) wait_ns = std::min<int64_t>(wait_ns, 20000);
        if (wait_ns > 0) s->cv.wait_for(lk, std::chrono::nanoseconds(wait_ns));
    }
}

// Incremental 0-set serving (Section 5.3): arrivals join the device pool as
// they come (at once while the pool holds work, else when the oldest waited
// deadline_us or max_bulk are waiting), and every step executes the pool's
// current 0-set.  Results complete per transaction.
void worker_zero_set(gputx_server *s)
{
    cudaSetDevice(s->db->device);
    std::unique_lock<std::mutex> lk(s->mu);
    const int64_t deadline = s->cfg.deadline_us * 1000;
    std::vector<int64_t> a_ts, r_ts, r_vals;
    std::vector<int32_t> a_type, r_st;
    std::vector<int64_t> a_params;
    while (s->worker_status == GPUTX_OK) {
        const int64_t queued = s->next_id - s->next_consume;
        const size_t in_pool = gputx_pool_pending(s->zpool);
        if (s->stop && queued == 0 && in_pool == 0) break;
        bool take = false;
        if (queued > 0) {
            const int64_t oldest = s->p_arrival[s->next_consume];
            take = in_pool > 0 || queued >= s->cfg.max_bulk || now_ns() - oldest >= deadline || s->stop || s->flush;
        }
        if (take) {
            // as many as the pool's capacity takes (halving on ECAPACITY)
            int64_t n = std::min<int64_t>(queued, s->cfg.max_bulk);
            a_ts.resize(n);
            a_type.resize(n);
            a_params.resize(n * s->P);
            s->p_type.copy_out(s->next_consume, n, a_type.data());
            s->p_params.copy_out(s->next_consume * s->P, n * s->P, a_params.data());
            for (int64_t i = 0; i < n; i++) a_ts[i] = s->next_consume + i;
            lk.unlock();
            gputx_status st = GPUTX_ECAPACITY;
            while (n > 0 && (st = gputx_pool_add(s->zpool, a_ts.data(), a_type.data(), a_params.data(), (size_t)n)) ==
                                GPUTX_ECAPACITY)
                n /= 2;
            lk.lock();
            if (st == GPUTX_OK) {
                s->next_consume += n;
                s->inflight_txns += n;
            } else if (st != GPUTX_ECAPACITY) {
                set_worker_error(s, st, "pool add");
                break;
            }
        }
        if (gputx_pool_pending(s->zpool) > 0) {
            lk.unlock();
            size_t k = 0, got = 0;
            gputx_status st = gputx_pool_step(s->zpool, &k);
            if (st == GPUTX_OK && k) {
                r_ts.resize(k);
                r_st.resize(k);
                r_vals.resize(k * s->R);
                st = gputx_pool_results(s->zpool, r_ts.data(), r_st.data(), r_vals.data(), k, &got);
            }
            const int64_t t = now_ns();
            lk.lock();
            if (st != GPUTX_OK) {
                set_worker_error(s, st, "pool step");
                break;
            }
            for (size_t i = 0; i < got; i++) {
                const int64_t id = r_ts[i];
                s->r_status[id] = r_st[i];
                s->r_values.copy_in(id * s->R, &r_vals[i * s->R], s->R);
                s->r_complete[id] = t;
                s->r_done[id] = 1;
                s->hist.add(t - s->p_arrival[id]);
                int64_t need[4];
                sum_needs(s, id, 1, need);
                for (int q = 0; q < 4; q++) {
                    s->ins_reserved[q] -= need[q];
                    s->ins_used[q] += need[q];
                }
            }
            s->completed += (int64_t)got;
            s->inflight_txns -= (int64_t)got;
            s->last_complete = t;
            s->bulks++;
            s->max_bulk_seen = std::max<int64_t>(s->max_bulk_seen, (int64_t)got);
            while (s->oldest_open < s->next_id && s->r_done[s->oldest_open]) s->oldest_open++;
            release_pool_before(s, std::min(s->oldest_open, s->next_consume));
            s->cv.notify_all();
            continue;
        }
        int64_t wait_ns = 200000;
        if (queued > 0) {
            const int64_t oldest = s->p_arrival[s->next_consume];
            wait_ns = std::max<int64_t>(0, oldest + deadline - now_ns());
        }
        if (wait_ns > 0) s->cv.wait_for(lk, std::chrono::nanoseconds(wait_ns));
    }
    s->cv.notify_all();
}

}  // namespace

extern "C" {

int64_t gputx_clock_ns(void) { return now_ns(); }

gputx_status gputx_server_create(gputx_db *db, const gputx_serve_config *cfg, gputx_server **out)
{
    if (!db || !out) return GPUTX_EINVAL;
    *out = nullptr;
    if (!db->dev.registered) return GPUTX_ESTATE;
    gputx_server *s = new (std::nothrow) gputx_server();
    if (!s) return GPUTX_ENOMEM;
    s->db = db;
    if (cfg) s->cfg = *cfg;
    gputx_serve_config &c = s->cfg;
    if (c.deadline_us <= 0) c.deadline_us = 1000;
    if (c.max_bulk <= 0 || c.max_bulk > db->cfg.max_bulk) c.max_bulk = db->cfg.max_bulk;
    if (c.max_inflight <= 0) c.max_inflight = 2;
    if (c.max_inflight > 8) c.max_inflight = 8;
    if (c.params_per_txn <= 0) c.params_per_txn = 2;
    if (c.queue_capacity <= 0) c.queue_capacity = 1ll << 30;
    if (c.strategy < GPUTX_KSET || c.strategy > GPUTX_SCAN) {
        delete s;
        return GPUTX_EINVAL;
    }
    s->P = c.params_per_txn;
    s->R = db->dev.out_width;
    s->ins_cap[0] = db->dev.hist_cap;
    s->ins_cap[1] = db->dev.child_cap;
    s->ins_cap[2] = db->dev.ord_cap;
    s->ins_cap[3] = db->dev.ol_cap;
    // rows already used by earlier bulks of this database
    gtx::InsertBase cur{};
    cudaStreamWaitEvent(db->stream, db->last_done, 0);
    if (cudaMemcpyAsync(&cur, db->d_cursor, sizeof cur, cudaMemcpyDeviceToHost, db->stream) != cudaSuccess ||
        cudaStreamSynchronize(db->stream) != cudaSuccess) {
        delete s;
        return GPUTX_ECUDA;
    }
    s->ins_used[0] = cur.hist;
    s->ins_used[1] = cur.cf;
    s->ins_used[2] = cur.ord;
    s->ins_used[3] = cur.ol;
    if (c.zero_set) {
        gputx_pool_config pc{};
        pc.capacity = std::min<int64_t>(1 << 25, std::max<int64_t>(2 * c.max_bulk, 1 << 12));
        pc.params_per_txn = c.params_per_txn;
        pc.conflict_mode = c.conflict_mode;
        const gputx_status pst = gputx_pool_create(db, &pc, &s->zpool);
        if (pst != GPUTX_OK) {
            delete s;
            return pst;
        }
        s->worker = std::thread(worker_zero_set, s);
        *out = s;
        return GPUTX_OK;
    }
    s->slots.resize(c.max_inflight);
    for (Slot &sl : s->slots) {
        const int64_t n = c.max_bulk;
        bool ok = cudaHostAlloc((void **)&sl.h_type, sizeof(int32_t) * n, cudaHostAllocDefault) == cudaSuccess &&
                  cudaHostAlloc((void **)&sl.h_ts, sizeof(int64_t) * n, cudaHostAllocDefault) == cudaSuccess &&
                  cudaHostAlloc((void **)&sl.h_params, sizeof(int64_t) * n * s->P, cudaHostAllocDefault) ==
                      cudaSuccess &&
                  cudaHostAlloc((void **)&sl.h_status, sizeof(int32_t) * n, cudaHostAllocDefault) == cudaSuccess &&
                  cudaHostAlloc((void **)&sl.h_values, sizeof(int64_t) * n * s->R, cudaHostAllocDefault) ==
                      cudaSuccess &&
                  cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            gputx_server_destroy(s);
            return GPUTX_ENOMEM;
        }
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return GPUTX_OK;
}

gputx_status gputx_server_submit(gputx_server *s, const int32_t *type, const int64_t *params, size_t n,
                                 const int64_t *arrival_ns, int64_t *first_id)
{
    if (!s || (n && (!type || !params))) return GPUTX_EINVAL;
    const int64_t t = now_ns();
    // insert rows of each transaction, before taking the lock
    int64_t need[4] = {0, 0, 0, 0};
    std::vector<uint8_t> packed(n);
    for (size_t i = 0; i < n; i++) {
        int64_t q[4];
        insert_need(s, type[i], params + i * s->P, q);
        for (int k = 0; k < 4; k++) need[k] += q[k];
        packed[i] = pack_need(q);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->worker_status != GPUTX_OK) return s->worker_status;
    // admission: the pool, the insert areas and free device memory
    const int64_t queued = s->next_id - s->next_consume + s->inflight_txns;
    if (queued + (int64_t)n > s->cfg.queue_capacity) {
        s->refused += (int64_t)n;
        return GPUTX_ENOMEM;
    }
    for (int k = 0; k < 4; k++)
        if (need[k] && s->ins_used[k] + s->ins_reserved[k] + need[k] > s->ins_cap[k]) {
            s->refused += (int64_t)n;
            return GPUTX_ENOMEM;
        }
    if (s->cfg.min_free_bytes > 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && (int64_t)fr < s->cfg.min_free_bytes) {
            s->refused += (int64_t)n;
            return GPUTX_ENOMEM;
        }
    }
    for (int k = 0; k < 4; k++) s->ins_reserved[k] += need[k];
    const int64_t id0 = s->next_id;
    s->p_type.append(type, (int64_t)n);
    s->p_params.append(params, (int64_t)n * s->P);
    s->p_need.append(packed.data(), (int64_t)n);
    if (arrival_ns) s->p_arrival.append(arrival_ns, (int64_t)n);
    else s->p_arrival.grow((int64_t)n, t);
    if (s->first_arrival < 0 && n) s->first_arrival = arrival_ns ? arrival_ns[0] : t;
    s->next_id += (int64_t)n;
    // results are read only once r_done marks them written
    s->r_status.grow_uninit((int64_t)n);
    s->r_values.grow_uninit((int64_t)n * s->R);
    s->r_complete.grow_uninit((int64_t)n);
    s->r_done.grow((int64_t)n, 0);
    if (first_id) *first_id = id0;
    s->cv.notify_all();
    return GPUTX_OK;
}

gputx_status gputx_server_results(gputx_server *s, int64_t first_id, size_t n, int32_t *status, int64_t *values,
                                  int64_t *complete_ns, size_t *n_done)
{
    if (!s || first_id < 0) return GPUTX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (first_id + (int64_t)n > s->next_id) return GPUTX_EINVAL;
    size_t done = 0;
    for (size_t i = 0; i < n; i++) {
        const int64_t id = first_id + (int64_t)i;
        if (!s->r_done[id]) continue;
        done++;
        if (status) status[i] = s->r_status[id];
        if (values) s->r_values.copy_out(id * s->R, s->R, values + i * s->R);
        if (complete_ns) complete_ns[i] = s->r_complete[id];
    }
    if (n_done) *n_done = done;
    return GPUTX_OK;
}

gputx_status gputx_server_drain(gputx_server *s)
{
    if (!s) return GPUTX_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv.notify_all();
    s->flush = true;   // the pending tail goes out without waiting for its deadline
    s->cv.notify_all();
    while (s->completed < s->next_id && s->worker_status == GPUTX_OK) s->cv.wait_for(lk, std::chrono::milliseconds(1));
    s->flush = false;
    return s->worker_status;
}

gputx_status gputx_server_stats(gputx_server *s, gputx_serve_stats *st)
{
    if (!s || !st) return GPUTX_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(st, 0, sizeof *st);
    st->submitted = s->next_id;
    st->completed = s->completed;
    st->bulks = s->bulks;
    st->max_bulk_seen = s->max_bulk_seen;
    st->refused = s->refused;
    st->p50_us = s->hist.quantile(0.50);
    st->p99_us = s->hist.quantile(0.99);
    st->mean_us = s->hist.count ? s->hist.sum_us / (double)s->hist.count : 0;
    if (s->completed && s->last_complete > s->first_arrival)
        st->txn_per_s = (double)s->completed / ((double)(s->last_complete - s->first_arrival) * 1e-9);
    return GPUTX_OK;
}

const char *gputx_server_last_error(const gputx_server *s)
{
    return s ? s->worker_error.c_str() : "null server";
}

void gputx_server_destroy(gputx_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    if (s->zpool) gputx_pool_destroy(s->zpool);
    for (Slot &sl : s->slots) {
        if (sl.bulk) gputx_free_bulk(sl.bulk);
        if (sl.h_type) cudaFreeHost(sl.h_type);
        if (sl.h_ts) cudaFreeHost(sl.h_ts);
        if (sl.h_params) cudaFreeHost(sl.h_params);
        if (sl.h_status) cudaFreeHost(sl.h_status);
        if (sl.h_values) cudaFreeHost(sl.h_values);
        if (sl.done) cudaEventDestroy(sl.done);
    }
    delete s;
}

}  // extern "C"
