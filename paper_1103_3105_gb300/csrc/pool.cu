// pool.cu -- incremental 0-set execution (Section 5.3).
//
// The transaction pool lives on the device: a ring of signatures indexed by
// arrival sequence and the pending transactions' basic operations, kept
// sorted by item (timestamp order inside an item: the sort is stable and the
// pool's operations always precede newer ones).
//
//   add   validate the new signatures, extract their operations
//         (Section 4.2 step 1), sort them, merge them into the pool's sorted
//         array ("their basic operations are merged into the sorted array");
//   step  rank the operations of each item (Section 4.2 steps 2-3): a
//         transaction is in the 0-set when every one of its operations has
//         rank 0, i.e. no earlier pending operation conflicts with it.  The
//         0-set, in timestamp order, becomes an ordinary bulk that runs in one
//         launch (Property 1); its transactions leave the ring and their
//         operations leave the sorted array, so the former 1-set is the next
//         0-set.
//
// A 0-set transaction conflicts with no earlier pending transaction, so
// moving it ahead of them changes no result: every step's outputs and the
// final database equal serial execution of the stream in timestamp order.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"
#include "procs.cuh"
#include "scan.cuh"

using namespace gtx;

size_t gtx_carve_bulk(gputx_bulk *b, char *base, bool device_inputs);   // api.cu

struct gputx_pool {
    gputx_db *db = nullptr;
    gputx_pool_config cfg{};
    int P = 1, R = 1, K = 1;
    int64_t cap = 0;
    // ring of pending signatures, index = arrival sequence % cap
    int64_t *r_ts = nullptr;
    int32_t *r_type = nullptr;
    int64_t *r_params = nullptr;
    uint8_t *r_pending = nullptr;
    uint32_t *r_blocked = nullptr;   // step id of the last step that found the transaction blocked
    // the pending operations sorted by item (a) and the merge target (c)
    uint32_t *a_key = nullptr, *a_val = nullptr, *c_key = nullptr, *c_val = nullptr;
    uint32_t *sel = nullptr;         // a step's 0-set: ring indices in timestamp order
    uint32_t *cnt = nullptr;         // device counters (kCnt)
    uint32_t *h_cnt = nullptr;       // pinned copy
    int64_t head = 0, tail = 0;      // sequence of the oldest pending transaction, of the next added
    int64_t m_pool = 0, pending = 0;
    int64_t last_ts = 0;
    bool any = false;
    uint32_t step = 0;
    gputx_bulk *carrier = nullptr;   // sort/scan scratch, and each step's 0-set bulk
    std::vector<void *> allocs;
    std::vector<int64_t> res_ts, res_values;
    std::vector<int32_t> res_status;
    size_t res_n = 0;
};

namespace gtx {
namespace {

enum { C_NEW_OPS = 0, C_ZERO = 1, C_KEPT = 2, C_INVALID = 3, C_HEAD = 4, kCnt = 8 };

// validation, ring copy and operation extraction of n new transactions
__global__ void pool_ingest_kernel(DevDB db, const int64_t *in_ts, const int32_t *in_type, const int64_t *in_params,
                                   int64_t n, int P, int64_t tail, int64_t cap, int64_t prev_ts, bool has_prev,
                                   int mode, int K, int64_t *r_ts, int32_t *r_type, int64_t *r_params,
                                   uint32_t *okey, uint32_t *oval, uint32_t *cnt)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t *p = in_params + i * P;
    const int32_t type = in_type[i];
    const int64_t ts = in_ts[i];
    bool ok = valid_txn(db, type, p, P);
    if (i > 0) ok = ok && ts > in_ts[i - 1];
    else if (has_prev) ok = ok && ts > prev_ts;
    const uint32_t r = (uint32_t)((tail + i) % cap);
    r_ts[r] = ts;
    r_type[r] = type;
    for (int j = 0; j < P; j++) r_params[(int64_t)r * P + j] = p[j];
    uint32_t obj[MAX_OPS], root[MAX_OPS];
    uint8_t cls[MAX_OPS];
    int k = 0;
    if (ok) k = access_set(db, type, p, mode, obj, cls, root);
    else atomicOr(&cnt[C_INVALID], 1u);
    if (k > K) {                       // cannot happen for a valid registered type
        atomicOr(&cnt[C_INVALID], 1u);
        k = 0;
    }
    for (int j = 0; j < K; j++) {
        okey[i * K + j] = j < k ? obj[j] : db.n_objects;   // padding sorts past every item
        oval[i * K + j] = j < k ? ((r << 7) | ((uint32_t)j << 2) | cls[j]) : OP_SENTINEL;
    }
    if (k) atomicAdd(&cnt[C_NEW_OPS], (uint32_t)k);
}

__global__ void pool_commit_kernel(int64_t n, int64_t tail, int64_t cap, uint8_t *r_pending)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) r_pending[(tail + i) % cap] = 1;
}

// stable merge of sorted a[0, ma) and b[0, mb) into c (a first on equal keys:
// the pool's operations are older than the new ones).  Each thread finds its
// start on the merge path by binary search, then merges kItems outputs.
constexpr int kMergeItems = 8;
__global__ void pool_merge_kernel(const uint32_t *ak, const uint32_t *av, int64_t ma, const uint32_t *bk,
                                  const uint32_t *bv, int64_t mb, uint32_t *ck, uint32_t *cv)
{
    const int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * kMergeItems;
    const int64_t total = ma + mb;
    if (d >= total) return;
    int64_t lo = d > mb ? d - mb : 0, hi = d < ma ? d : ma;
    while (lo < hi) {   // i = how many of the first d outputs come from a
        const int64_t mid = (lo + hi) >> 1;
        if (ak[mid] <= bk[d - mid - 1]) lo = mid + 1;
        else hi = mid;
    }
    int64_t ia = lo, ib = d - lo;
    const int64_t end = d + kMergeItems < total ? d + kMergeItems : total;
    for (int64_t o = d; o < end; o++) {
        const bool take_a = ia < ma && (ib >= mb || ak[ia] <= bk[ib]);
        if (take_a) {
            ck[o] = ak[ia];
            cv[o] = av[ia];
            ia++;
        } else {
            ck[o] = bk[ib];
            cv[o] = bv[ib];
            ib++;
        }
    }
}

// ranks within each item's group as in the K-SET analysis; an operation with
// rank > 0 blocks its transaction for this step
struct ZeroMode {
    const uint32_t *sk, *sv;
    uint32_t *blocked;
    uint32_t step;
    __device__ uint64_t element(int64_t i) const
    {
        const uint32_t k = sk[i];
        const bool head = (i == 0) || sk[i - 1] != k;
        uint32_t runhead = 0;
        if (!head) {
            const uint32_t c = sv[i] & 3u, pc = sv[i - 1] & 3u;
            runhead = !(c == pc && c != CLS_W);
        }
        return DualSeg::make(head, runhead, 0, 0);
    }
    __device__ void output(int64_t i, uint64_t s) const
    {
        if (DualSeg::v1(s) > 0) blocked[sv[i] >> 7] = step;
    }
};

// the 0-set in timestamp order: pending and not blocked, over the ring window
struct SelectMode {
    const uint8_t *pending;
    const uint32_t *blocked;
    uint32_t *sel, *cnt;
    int64_t head, cap, span;
    uint32_t step;
    __device__ bool in(int64_t j) const
    {
        const uint32_t r = (uint32_t)((head + j) % cap);
        return pending[r] && blocked[r] != step;
    }
    __device__ uint64_t element(int64_t j) const { return DualSeg::make(0, 0, 0, in(j) ? 1u : 0u); }
    __device__ void output(int64_t j, uint64_t s) const
    {
        const uint32_t c = DualSeg::v2(s);
        if (in(j)) sel[c - 1] = (uint32_t)((head + j) % cap);
        if (j == span - 1) cnt[C_ZERO] = c;
    }
};

// the 0-set's signatures into the step's bulk; they leave the ring
__global__ void pool_gather_kernel(const uint32_t *sel, const uint32_t *cnt, const int64_t *r_ts,
                                   const int32_t *r_type, const int64_t *r_params, int P, uint8_t *r_pending,
                                   int64_t *b_ts, int32_t *b_type, int64_t *b_params)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= (int64_t)cnt[C_ZERO]) return;
    const uint32_t r = sel[k];
    b_ts[k] = r_ts[r];
    b_type[k] = r_type[r];
    for (int j = 0; j < P; j++) b_params[k * P + j] = r_params[(int64_t)r * P + j];
    r_pending[r] = 0;
}

// the operations of transactions still pending, order kept
struct KeepMode {
    const uint32_t *ck, *cv;
    uint32_t *ak, *av, *cnt;
    const uint8_t *pending;
    int64_t m;
    __device__ bool keep(int64_t i) const { return pending[cv[i] >> 7] != 0; }
    __device__ uint64_t element(int64_t i) const { return DualSeg::make(0, 0, 0, keep(i) ? 1u : 0u); }
    __device__ void output(int64_t i, uint64_t s) const
    {
        const uint32_t c = DualSeg::v2(s);
        if (keep(i)) {
            ak[c - 1] = ck[i];
            av[c - 1] = cv[i];
        }
        if (i == m - 1) cnt[C_KEPT] = c;
    }
};

// offset of the oldest pending transaction in the ring window
__global__ void pool_head_kernel(const uint8_t *pending, int64_t head, int64_t cap, int64_t span, uint32_t *cnt)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j < span && pending[(head + j) % cap]) atomicMin(&cnt[C_HEAD], (uint32_t)j);
}

inline unsigned blocks_for(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

template <class Mode>
cudaError_t pool_scan(gputx_bulk *b, const Mode &mode, int64_t count, int ctr_slot)
{
    if (count <= 0) return cudaSuccess;
    const int64_t tiles = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles > b->sc.scan_tiles) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(b->sc.scan_status, 0, tiles * sizeof(uint64_t), b->stream);
    if (!e) e = cudaMemsetAsync(b->sc.tile_ctr + ctr_slot, 0, sizeof(uint32_t), b->stream);
    if (e) return e;
    dualseg_scan_kernel<Mode><<<(unsigned)tiles, SCAN_THREADS, 0, b->stream>>>(
        mode, count, b->sc.scan_status, b->sc.tile_ctr + ctr_slot, &b->ctl->err,
        (uint64_t)b->db->cfg.spin_limit_ns);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace
}  // namespace gtx

namespace {

gputx_status pool_fail(gputx_pool *p, gputx_status st, const std::string &what)
{
    p->db->last_error = "pool: " + what;
    return st;
}

gputx_status pool_cuda(gputx_pool *p, cudaError_t e, const char *what)
{
    return pool_fail(p, e == cudaErrorMemoryAllocation ? GPUTX_ENOMEM : GPUTX_ECUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

#define PCK(call, what)                                   \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return pool_cuda(p, e_, what); \
    } while (0)

template <class T> cudaError_t palloc(gputx_pool *p, T **ptr, int64_t count)
{
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, (size_t)std::max<int64_t>(count, 1) * sizeof(T));
    if (e) return e;
    p->allocs.push_back(q);
    *ptr = (T *)q;
    return cudaMemset(q, 0, (size_t)std::max<int64_t>(count, 1) * sizeof(T));
}

void pool_free(gputx_pool *p)
{
    if (p->carrier) {
        if (p->carrier->stream) {
            cudaStreamSynchronize(p->carrier->stream);
            cudaStreamDestroy(p->carrier->stream);
        }
        if (p->carrier->arena) cudaFree(p->carrier->arena);
        if (p->carrier->ev[7]) cudaEventDestroy(p->carrier->ev[7]);
        delete p->carrier;
    }
    for (void *q : p->allocs) cudaFree(q);
    if (p->h_cnt) cudaFreeHost(p->h_cnt);
    delete p;
}

gputx_status read_counters(gputx_pool *p)
{
    PCK(cudaMemcpyAsync(p->h_cnt, p->cnt, kCnt * sizeof(uint32_t), cudaMemcpyDeviceToHost, p->carrier->stream),
        "counters");
    PCK(cudaMemcpyAsync(&p->carrier->host_ctl, p->carrier->ctl, sizeof(BulkCtl), cudaMemcpyDeviceToHost,
                        p->carrier->stream),
        "counters");
    PCK(cudaStreamSynchronize(p->carrier->stream), "counters");
    if (p->carrier->host_ctl.err & ERR_TIMEOUT) return pool_fail(p, GPUTX_ETIMEOUT, "a bounded device wait ran out");
    return GPUTX_OK;
}

}  // namespace

extern "C" {

gputx_status gputx_pool_create(gputx_db *db, const gputx_pool_config *cfg, gputx_pool **out)
{
    if (!db || !cfg || !out) return GPUTX_EINVAL;
    *out = nullptr;
    if (!db->dev.registered) return GPUTX_ESTATE;
    if (cfg->capacity < 1 || cfg->capacity > (1 << 25) || cfg->params_per_txn < 1 || cfg->params_per_txn > 64 ||
        (cfg->conflict_mode != GPUTX_CONFLICT_PAPER && cfg->conflict_mode != GPUTX_CONFLICT_ADD)) {
        db->last_error = "pool: bad configuration";
        return GPUTX_EINVAL;
    }
    gputx_pool *p = new (std::nothrow) gputx_pool();
    if (!p) return GPUTX_ENOMEM;
    p->db = db;
    p->cfg = *cfg;
    p->P = cfg->params_per_txn;
    p->R = db->dev.out_width;
    p->K = std::max(db->kmax, 1);
    p->cap = cfg->capacity;
    const int64_t ops = p->cap * p->K;
    cudaError_t e = cudaSuccess;
    if (!e) e = palloc(p, &p->r_ts, p->cap);
    if (!e) e = palloc(p, &p->r_type, p->cap);
    if (!e) e = palloc(p, &p->r_params, p->cap * p->P);
    if (!e) e = palloc(p, &p->r_pending, p->cap);
    if (!e) e = palloc(p, &p->r_blocked, p->cap);
    if (!e) e = palloc(p, &p->a_key, ops);
    if (!e) e = palloc(p, &p->a_val, ops);
    if (!e) e = palloc(p, &p->c_key, ops);
    if (!e) e = palloc(p, &p->c_val, ops);
    if (!e) e = palloc(p, &p->sel, p->cap);
    if (!e) e = palloc(p, &p->cnt, kCnt);
    if (!e) e = cudaMallocHost(&p->h_cnt, kCnt * sizeof(uint32_t));
    if (e) {
        gputx_status st = pool_cuda(p, e, "allocation");
        pool_free(p);
        return st;
    }
    // the carrier: a bulk of capacity `cap` whose arena holds the sort and
    // scan scratch and, at each step, the 0-set's signatures and results
    gputx_bulk *b = new (std::nothrow) gputx_bulk();
    if (!b) {
        pool_free(p);
        return GPUTX_ENOMEM;
    }
    p->carrier = b;
    b->db = db;
    b->n = p->cap;
    b->P = p->P;
    b->R = p->R;
    // its own stream: the pool may outlive nothing of the database's but
    // memory, so destroying it never touches the database's streams
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e) {
        b->stream = nullptr;
        gputx_status st = pool_cuda(p, e, "stream");
        pool_free(p);
        return st;
    }
    b->executed = true;
    b->arena_bytes = gtx_carve_bulk(b, nullptr, false);
    e = cudaMalloc(&b->arena, b->arena_bytes);
    if (!e) e = cudaEventCreate(&b->ev[7]);
    if (e) {
        gputx_status st = pool_cuda(p, e, "allocation");
        pool_free(p);
        return st;
    }
    gtx_carve_bulk(b, (char *)b->arena, false);
    e = cudaDeviceSynchronize();
    if (e) {
        gputx_status st = pool_cuda(p, e, "allocation");
        pool_free(p);
        return st;
    }
    *out = p;
    return GPUTX_OK;
}

gputx_status gputx_pool_add(gputx_pool *p, const int64_t *ts, const int32_t *type, const int64_t *params, size_t n)
{
    if (!p) return GPUTX_EINVAL;
    if (n == 0) return GPUTX_OK;
    if (!ts || !type || !params) return pool_fail(p, GPUTX_EINVAL, "null array");
    if (p->tail + (int64_t)n - p->head > p->cap) return pool_fail(p, GPUTX_ECAPACITY, "pending span above capacity");
    gputx_bulk *b = p->carrier;
    gputx_db *db = p->db;
    cudaStream_t s = b->stream;
    const int64_t nn = (int64_t)n;
    // the carrier's input arrays stage the upload
    PCK(cudaMemcpyAsync(b->ts, ts, nn * sizeof(int64_t), cudaMemcpyHostToDevice, s), "upload");
    PCK(cudaMemcpyAsync(b->type, type, nn * sizeof(int32_t), cudaMemcpyHostToDevice, s), "upload");
    PCK(cudaMemcpyAsync(b->params, params, nn * p->P * sizeof(int64_t), cudaMemcpyHostToDevice, s), "upload");
    PCK(cudaMemsetAsync(p->cnt, 0, kCnt * sizeof(uint32_t), s), "add");
    PCK(cudaMemsetAsync(b->ctl, 0, sizeof(BulkCtl), s), "add");
    uint32_t *nk = b->sc.keys_a, *nv = b->sc.vals_a, *xk = b->sc.keys_b, *xv = b->sc.vals_b;
    pool_ingest_kernel<<<blocks_for(nn), 256, 0, s>>>(db->dev, b->ts, b->type, b->params, nn, p->P, p->tail, p->cap,
                                                       p->last_ts, p->any, p->cfg.conflict_mode, p->K, p->r_ts,
                                                       p->r_type, p->r_params, nk, nv, p->cnt);
    count_launches(1);
    PCK(cudaGetLastError(), "ingest");
    gputx_status st = read_counters(p);
    if (st) return st;
    if (p->h_cnt[C_INVALID])
        return pool_fail(p, GPUTX_EINVAL, "invalid signature, unregistered type or timestamps not increasing");
    const int64_t m_new = p->h_cnt[C_NEW_OPS];
    // the new operations by item (stable: timestamp order within an item),
    // padding last, then merged behind the pool's own
    PCK(launch_sort(b, nk, nv, xk, xv, nn * p->K, db->obj_bits), "sort");
    const int64_t total = p->m_pool + m_new;
    if (m_new > 0) {
        const int64_t threads = (total + kMergeItems - 1) / kMergeItems;
        pool_merge_kernel<<<blocks_for(threads), 256, 0, s>>>(p->a_key, p->a_val, p->m_pool, nk, nv, m_new, p->c_key,
                                                              p->c_val);
        count_launches(1);
        PCK(cudaGetLastError(), "merge");
        std::swap(p->a_key, p->c_key);
        std::swap(p->a_val, p->c_val);
    }
    pool_commit_kernel<<<blocks_for(nn), 256, 0, s>>>(nn, p->tail, p->cap, p->r_pending);
    count_launches(1);
    PCK(cudaGetLastError(), "commit");
    st = read_counters(p);
    if (st) return st;
    p->m_pool = total;
    p->tail += nn;
    p->pending += nn;
    p->last_ts = ts[n - 1];
    p->any = true;
    return GPUTX_OK;
}

gputx_status gputx_pool_step(gputx_pool *p, size_t *executed)
{
    if (!p) return GPUTX_EINVAL;
    if (executed) *executed = 0;
    p->res_n = 0;
    if (p->pending == 0) return GPUTX_OK;
    gputx_bulk *b = p->carrier;
    gputx_db *db = p->db;
    cudaStream_t s = b->stream;
    const uint32_t step = ++p->step == 0 ? ++p->step : p->step;   // 0 marks "never blocked"
    const int64_t span = p->tail - p->head;
    PCK(cudaMemsetAsync(p->cnt, 0, kCnt * sizeof(uint32_t), s), "step");
    PCK(cudaMemsetAsync(b->ctl, 0, sizeof(BulkCtl), s), "step");
    // ranks over the pool's sorted operations: rank > 0 blocks the transaction
    ZeroMode zm{p->a_key, p->a_val, p->r_blocked, step};
    PCK(pool_scan(b, zm, p->m_pool, 13), "ranks");
    SelectMode sm{p->r_pending, p->r_blocked, p->sel, p->cnt, p->head, p->cap, span, step};
    PCK(pool_scan(b, sm, span, 14), "select");
    gputx_status st = read_counters(p);
    if (st) return st;
    const int64_t n0 = p->h_cnt[C_ZERO];
    if (n0 <= 0) return pool_fail(p, GPUTX_EBOUNDS, "empty 0-set with pending transactions");
    // the 0-set as the carrier's bulk, executed in one launch after every
    // bulk queued before it on this database
    pool_gather_kernel<<<blocks_for(n0), 256, 0, s>>>(p->sel, p->cnt, p->r_ts, p->r_type, p->r_params, p->P,
                                                      p->r_pending, b->ts, b->type, b->params);
    count_launches(1);
    PCK(cudaGetLastError(), "gather");
    b->n = n0;
    PCK(cudaMemsetAsync(b->status, 0, n0 * sizeof(int32_t), s), "step");
    PCK(cudaMemsetAsync(b->out, 0, n0 * p->R * sizeof(int64_t), s), "step");
    PCK(launch_insert_slots(b), "insert slots");
    PCK(cudaStreamWaitEvent(s, db->last_done, 0), "order");
    PCK(launch_begin(b), "begin");
    PCK(launch_independent(b, p->cfg.conflict_mode == GPUTX_CONFLICT_ADD), "execute");
    PCK(launch_finish(b), "finish");
    PCK(cudaEventRecord(db->last_done, s), "order");
    PCK(cudaStreamWaitEvent(db->stream, db->last_done, 0), "order");
    // the executed transactions' operations leave the sorted array
    if (p->m_pool > 0) {
        KeepMode km{p->a_key, p->a_val, p->c_key, p->c_val, p->cnt, p->r_pending, p->m_pool};
        PCK(pool_scan(b, km, p->m_pool, 15), "compact");
    }
    PCK(cudaMemsetAsync(p->cnt + C_HEAD, 0xff, sizeof(uint32_t), s), "head");
    pool_head_kernel<<<blocks_for(span), 256, 0, s>>>(p->r_pending, p->head, p->cap, span, p->cnt);
    count_launches(1);
    PCK(cudaGetLastError(), "head");
    p->res_ts.resize(n0);
    p->res_status.resize(n0);
    p->res_values.resize(n0 * p->R);
    PCK(cudaMemcpyAsync(p->res_ts.data(), b->ts, n0 * sizeof(int64_t), cudaMemcpyDeviceToHost, s), "results");
    PCK(cudaMemcpyAsync(p->res_status.data(), b->status, n0 * sizeof(int32_t), cudaMemcpyDeviceToHost, s), "results");
    PCK(cudaMemcpyAsync(p->res_values.data(), b->out, n0 * p->R * sizeof(int64_t), cudaMemcpyDeviceToHost, s),
        "results");
    st = read_counters(p);
    if (st) return st;
    if (b->host_ctl.err & ERR_CAPACITY) return pool_fail(p, GPUTX_ECAPACITY, "an insert area or hash index is full");
    if (b->host_ctl.err) return pool_fail(p, GPUTX_EBOUNDS, "device check failed");
    if (p->m_pool > 0) {
        std::swap(p->a_key, p->c_key);
        std::swap(p->a_val, p->c_val);
        p->m_pool = p->h_cnt[C_KEPT];
    }
    p->pending -= n0;
    const uint32_t off = p->h_cnt[C_HEAD];
    p->head = (p->pending == 0 || off == 0xffffffffu) ? p->tail : p->head + off;
    p->res_n = (size_t)n0;
    if (executed) *executed = (size_t)n0;
    return GPUTX_OK;
}

gputx_status gputx_pool_results(const gputx_pool *p, int64_t *ts, int32_t *status, int64_t *values, size_t capacity,
                                size_t *n)
{
    if (!p || !n) return GPUTX_EINVAL;
    *n = p->res_n;
    if (!ts && !status && !values) return GPUTX_OK;
    if (capacity < p->res_n) return GPUTX_EINVAL;
    if (ts) std::memcpy(ts, p->res_ts.data(), p->res_n * sizeof(int64_t));
    if (status) std::memcpy(status, p->res_status.data(), p->res_n * sizeof(int32_t));
    if (values) std::memcpy(values, p->res_values.data(), p->res_n * p->R * sizeof(int64_t));
    return GPUTX_OK;
}

size_t gputx_pool_pending(const gputx_pool *p) { return p ? (size_t)p->pending : 0; }

void gputx_pool_destroy(gputx_pool *p)
{
    if (!p) return;
    pool_free(p);
}

}  // extern "C"
