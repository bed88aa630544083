// analysis.cu -- bulk generation on the device (Section 4.2, Section 5.2 step
// 1-2, Appendix D): basic-operation extraction, grouping by data item with a
// radix sort, per-group ranks, transaction depths (k-set levels), regrouping
// by (level, type), insert slots, partition ids.
#include <algorithm>
#include <cooperative_groups.h>
#include <cstdio>

#include "engine.h"
#include "procs.cuh"
#include "scan.cuh"

namespace gtx {

namespace {

constexpr int TB = 256;  // threads per block of the simple map kernels

inline unsigned grid_for(int64_t n, int block = TB)
{
    int64_t g = (n + block - 1) / block;
    return (unsigned)(g < 1 ? 1 : g);
}

// ---------------------------------------------------------------------------
// bulk begin / finish: insert bases from the device cursors
// ---------------------------------------------------------------------------
// hist_rows < 0: the history rows were counted by the insert-slot scan
__global__ void begin_kernel(const InsertBase *cursor, BulkCtl *ctl, int64_t hist_rows, bool live_rows)
{
    ctl->base = *cursor;
    if (hist_rows >= 0) ctl->total.hist = live_rows ? (int64_t)ctl->n_live : hist_rows;
}

__global__ void finish_kernel(InsertBase *cursor, const BulkCtl *ctl)
{
    if (ctl->err) return;
    cursor->hist += ctl->total.hist;
    cursor->cf += ctl->total.cf;
    cursor->ord += ctl->total.ord;
    cursor->ol += ctl->total.ol;
}

// ---------------------------------------------------------------------------
// a2: basic-operation extraction (map), with validation and partition ids
// ---------------------------------------------------------------------------
struct ExtractArgs {
    DevDB db;
    DevBulk b;
    BulkCtl *ctl;
    uint32_t *keys, *vals;         // op keys / payloads
    const uint32_t *op_off;        // exclusive op offsets or null (uniform)
    int uniform_k;
    int mode;
    int part_size;
    uint32_t *pid_key, *pid_val;   // PART: partition id and txn per transaction (or null)
    bool write_ops;
    bool sentinel_fill;            // fill unused slots with padding operations
    uint32_t sentinel_key;         // object id above every real one
    const uint32_t *bulk_of;       // segmented graph bulks: the bulk above the object id (or null)
    int obj_shift;                 // bits of the object id under the bulk
    uint32_t pad_pid;              // PART: partition id of a padding transaction (after every real one)
};

__device__ __forceinline__ bool txn_padding(const DevBulk &b, int64_t t)
{
    return b.n_live && t >= (int64_t)*b.n_live;
}

__device__ __forceinline__ bool txn_valid(const DevDB &db, const DevBulk &b, int64_t t)
{
    const int64_t *p = b.params + t * b.P;
    if (!valid_txn(db, b.type[t], p, b.P)) return false;
    if (t > 0 && !(b.ts[t] > b.ts[t - 1])) return false;   // ids strictly increase
    return true;
}

__global__ void count_ops_kernel(DevDB db, DevBulk b, BulkCtl *ctl, uint32_t *cnt)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= b.n) return;
    int c = 0;
    if (txn_valid(db, b, t)) c = op_count(db, b.type[t], b.params + t * b.P);
    else set_err(&ctl->err, ERR_INVAL);
    cnt[t] = (uint32_t)c;
}

__global__ void extract_kernel(ExtractArgs a)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool cross = false;
    if (t < a.b.n) {
        const int64_t *p = a.b.params + t * a.b.P;
        const int64_t off = a.op_off ? (int64_t)a.op_off[t] : t * a.uniform_k;   // used when writing
        const bool pad = txn_padding(a.b, t);
        const bool ok = pad || txn_valid(a.db, a.b, t);
        uint32_t obj[MAX_OPS], root[MAX_OPS];
        uint8_t cls[MAX_OPS];
        int k = 0;
        if (ok && !pad) {
            k = access_set(a.db, a.b.type[t], p, a.mode, obj, cls, root);
        } else if (!ok) {
            set_err(&a.ctl->err, ERR_INVAL);
        }
        if (a.write_ops && a.sentinel_fill) {
            // padding operations after the real ones: they sort past every
            // real group and every consumer skips their payload
            for (int j = k; j < a.uniform_k; j++) {
                a.keys[off + j] = a.sentinel_key;
                a.vals[off + j] = OP_SENTINEL;
            }
        } else if (a.write_ops && a.op_off == nullptr) {
            // uniform layout: always fill K slots (dummy reads on object 0 for
            // an invalid transaction; the bulk will not execute)
            for (int j = k; j < a.uniform_k; j++) { obj[j] = 0; cls[j] = CLS_R; root[j] = 0; }
            k = a.uniform_k;
        }
        const uint32_t pid = pad ? a.pad_pid : (k ? root[0] / (uint32_t)a.part_size : 0);
        const uint32_t seg = (a.bulk_of && !pad) ? (a.bulk_of[t] << a.obj_shift) : 0u;
        for (int j = 0; j < k; j++) {
            if (a.write_ops) {
                a.keys[off + j] = obj[j] | seg;
                a.vals[off + j] = ((uint32_t)t << 7) | ((uint32_t)j << 2) | cls[j];
            }
            cross |= (root[j] / (uint32_t)a.part_size) != pid;
        }
        if (a.pid_key) {
            a.pid_key[t] = pid;
            a.pid_val[t] = (uint32_t)t;
        }
    }
    const uint32_t cross_mask = __ballot_sync(0xffffffffu, cross);
    if ((threadIdx.x & 31) == 0 && cross_mask) atomicAdd(&a.ctl->cross, (uint32_t)__popc(cross_mask));
}

// exclusive op offsets from per-transaction counts
struct OffsetMode {
    const uint32_t *cnt;
    uint32_t *off;
    int64_t n;
    __device__ uint64_t element(int64_t i) const { return DualSeg::make(0, 0, 0, cnt[i]); }
    __device__ void output(int64_t i, uint64_t s) const
    {
        off[i + 1] = DualSeg::v2(s);
        if (i == 0) off[0] = 0;
    }
};

// ---------------------------------------------------------------------------
// a4/a5: ranks in each group and transaction depth (Section 4.2 steps 2-5)
// ---------------------------------------------------------------------------
// Within a group (one data item, operations in timestamp order) an operation
// starts a new run unless it and its predecessor are both reads or both ADDs.
// rank = run index within the group; depth(t) = max rank over t's operations.
struct RankMode {
    const uint32_t *sk, *sv;
    uint32_t *level;
    uint32_t *rid;   // optional: global run id, bit 31 = first run of its group
    __device__ uint64_t element(int64_t i) const
    {
        const uint32_t k = sk[i], v = sv[i];
        const bool head = (i == 0) || sk[i - 1] != k;
        uint32_t runhead = 1;
        if (!head) {
            const uint32_t c = v & 3u, pc = sv[i - 1] & 3u;
            runhead = !(c == pc && c != CLS_W);
        }
        return DualSeg::make(head, head ? 0u : runhead, 0, runhead);
    }
    __device__ void output(int64_t i, uint64_t s) const
    {
        if (sv[i] == OP_SENTINEL) return;
        const uint32_t rank = DualSeg::v1(s);
        const uint32_t txn = sv[i] >> 7;
        atomicMax(&level[txn], rank);
        if (rid) rid[i] = (DualSeg::v2(s) - 1u) | (rank == 0 ? 0x80000000u : 0u);
    }
};

// TPL tickets: number of operations of the group before this operation's run
// (Section 5.1 key values, read with ticket semantics).  A ticket of at least
// `hot_ticket` raises `hot`: some counter carries a chain that long, which
// picks the executor (the flag is written once, by the first such ticket seen).
struct TicketMode {
    const uint32_t *sk, *sv;
    uint32_t *lock_key, *lock_ticket;
    const uint32_t *op_off;
    int uniform_k;
    uint32_t *hot;
    uint32_t hot_ticket;
    uint32_t n_objects;   // a debug build checks every lock key against it
    uint32_t *err;
    __device__ uint64_t element(int64_t i) const
    {
        const uint32_t k = sk[i], v = sv[i];
        const bool head = (i == 0) || sk[i - 1] != k;
        uint32_t runhead = 1;
        if (!head) {
            const uint32_t c = v & 3u, pc = sv[i - 1] & 3u;
            runhead = !(c == pc && c != CLS_W);
        }
        return DualSeg::make(head, 1, runhead, 1);
    }
    __device__ void output(int64_t i, uint64_t s) const
    {
        const uint32_t v = sv[i];
        if (v == OP_SENTINEL) return;
        const uint32_t txn = v >> 7, j = (v >> 2) & 31u;
        const int64_t slot = (op_off ? (int64_t)op_off[txn] : (int64_t)txn * uniform_k) + j;
        const uint32_t tk = DualSeg::v1(s) - DualSeg::v2(s);
        if (!dbg_in(sk[i], n_objects, err)) return;
        lock_key[slot] = sk[i];
        lock_ticket[slot] = tk;
        if (tk >= hot_ticket && !*(volatile uint32_t *)hot) *hot = 1u;
    }
};

// Exact depths by dataflow (one pass, no rounds).
//
// Within a group (one item, operations in timestamp order) the runs follow
// one another: every operation of run q conflicts with every operation of run
// q-1, and transitively with all earlier runs.  So a transaction's depth is
// the largest, over its operations outside their group's first run, of one
// more than the deepest transaction of the run before -- the longest path of
// the conflict graph, the depth the Jacobi refinement converges to.  Here each
// transaction computes it once the runs before its operations are complete.
// Run q keeps one 64-bit word: the number of its operations still to finish
// (high half) and the largest depth among the finished ones (low half).  A
// finishing operation replaces both at once by compare-and-swap, so a waiter
// that reads a count of zero reads the run's maximum in the same word: no
// fence and no second read.  Transactions run in timestamp order, a CTA's
// chunk of consecutive ones at a time, so every run a transaction waits for
// belongs to earlier transactions already running: the chain of waits always
// ends.

// per operation: its run id into the transaction's slot, its run counted
__global__ void depth_prep_kernel(const uint32_t *sv, const uint32_t *rid, int64_t m, const uint32_t *op_off,
                                  int kslots, uint32_t *txn_rid, unsigned long long *runword, const BulkCtl *ctl)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m || ctl->err) return;
    const uint32_t v = sv[i];
    if (v == OP_SENTINEL) return;
    const uint32_t rr = rid[i];
    const uint32_t txn = v >> 7, j = (v >> 2) & 31u;
    const int64_t slot = (op_off ? (int64_t)op_off[txn] : (int64_t)txn * kslots) + j;
    txn_rid[slot] = rr;
    atomicAdd(&runword[rr & 0x7fffffffu], 1ull << 32);
}

constexpr uint32_t kNoRun = 0xffffffffu;   // an operation slot with no operation
constexpr uint32_t kFlowSleepMax = 512;     // longest back-off between polls, ns
constexpr int kFlowBlocksPerSm = 1;         // resident CTAs of the pass per SM (fewer waiters poll less)

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__global__ void __launch_bounds__(256) depth_flow_kernel(const uint32_t *txn_rid, const uint32_t *op_off, int kslots,
                                                        unsigned long long *runword, uint32_t *level, BulkCtl *ctl,
                                                        int64_t n, uint64_t limit_ns)
{
    __shared__ uint32_t s_c, s_stop;
    if (ctl->err) return;   // set before this launch only: every block returns
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->rounds = 1;
    while (true) {
        if (threadIdx.x == 0) {
            s_stop = *(volatile uint32_t *)&ctl->err ? 1u : 0u;
            s_c = atomicAdd(&ctl->claim, 1u);
        }
        __syncthreads();
        const int64_t start = (int64_t)s_c * blockDim.x;
        if (s_stop || start >= n) break;
        const int64_t t = start + threadIdx.x;
        if (t < n) {
            const int64_t s0 = op_off ? (int64_t)op_off[t] : t * kslots;
            const int k = op_off ? (int)(op_off[t + 1] - op_off[t]) : kslots;
            // every per-operation array below is indexed by unrolled loop
            // counters only, so it lives in registers
            uint32_t rr[MAX_OPS];
            uint32_t waits = 0, own = 0;   // bit j: operation j follows an earlier run / has a run
#pragma unroll
            for (int j = 0; j < MAX_OPS; j++) {
                rr[j] = j < k ? txn_rid[s0 + j] : kNoRun;
                if (rr[j] != kNoRun) {
                    own |= 1u << j;
                    if (!(rr[j] & 0x80000000u)) waits |= 1u << j;
                }
            }
            // the preceding runs: all polled at once (first, and after any of
            // them completes), else only the first incomplete one, so that
            // waiters far down a chain do not flood L2 with polls
            uint32_t pending = waits, lv = 0;
            uint64_t t_prog = globaltimer();
            uint32_t ns = 64;
            bool all = true;
            while (pending) {
                // this look's runs: every pending one, or the first
                const uint32_t look = all ? pending : pending & (0u - pending);
                unsigned long long w[MAX_OPS];
#pragma unroll
                for (int j = 0; j < MAX_OPS; j++)   // all loads in flight at once
                    w[j] = (look >> j & 1u) ? ld_relaxed_u64(&runword[(rr[j] & 0x7fffffffu) - 1u]) : 0ull;
                uint32_t still = pending;
#pragma unroll
                for (int j = 0; j < MAX_OPS; j++) {
                    if ((look >> j & 1u) && !(w[j] >> 32)) {   // complete: its maximum is final
                        still &= ~(1u << j);
                        if ((uint32_t)w[j] + 1u > lv) lv = (uint32_t)w[j] + 1u;
                    }
                }
                if (still != pending) {
                    pending = still;
                    t_prog = globaltimer();
                    ns = 64;
                    all = true;
                    continue;
                }
                all = false;
                if (globaltimer() - t_prog > limit_ns) {
                    set_err(&ctl->err, ERR_TIMEOUT);
                    break;
                }
                __nanosleep(ns);
                if (ns < kFlowSleepMax) ns <<= 1;
            }
            level[t] = lv;
            // this transaction's depth into each of its runs, counted off in
            // the same compare-and-swap
            unsigned long long cur[MAX_OPS];
#pragma unroll
            for (int j = 0; j < MAX_OPS; j++) cur[j] = 1ull << 32;   // a guess: the run's only operation
            uint32_t todo = own;
            for (int attempt = 0; todo && attempt < (1 << 20); attempt++) {
                unsigned long long prev[MAX_OPS];
#pragma unroll
                for (int j = 0; j < MAX_OPS; j++) {   // every swap in flight at once
                    prev[j] = cur[j];
                    if (!(todo >> j & 1u)) continue;
                    const uint32_t mx = (uint32_t)cur[j] > lv ? (uint32_t)cur[j] : lv;
                    const unsigned long long nv = (((cur[j] >> 32) - 1ull) << 32) | mx;
                    prev[j] = atomicCAS(&runword[rr[j] & 0x7fffffffu], cur[j], nv);
                }
#pragma unroll
                for (int j = 0; j < MAX_OPS; j++) {
                    if (!(todo >> j & 1u)) continue;
                    if (prev[j] == cur[j]) todo &= ~(1u << j);
                    else cur[j] = prev[j];
                }
            }
            if (todo) set_err(&ctl->err, ERR_TIMEOUT);
        }
        __syncthreads();
    }
}


// d and w0 (Appendix D structural parameters)
__global__ void level_stats_kernel(const uint32_t *level, int64_t n, BulkCtl *ctl)
{
    __shared__ uint32_t s_max, s_zero;
    if (threadIdx.x == 0) { s_max = 0; s_zero = 0; }
    __syncthreads();
    uint32_t mx = 0, zero = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t l = level[i];
        mx = l > mx ? l : mx;
        zero += (l == 0);
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    zero = __reduce_add_sync(0xffffffffu, zero);
    if ((threadIdx.x & 31) == 0) { atomicMax(&s_max, mx); atomicAdd(&s_zero, zero); }
    __syncthreads();
    if (threadIdx.x == 0) { atomicMax(&ctl->depth, s_max); atomicAdd(&ctl->w0, s_zero); }
}

// ---------------------------------------------------------------------------
// a6: regroup by (level, type) -- Appendix D's grouping by type, per level
// ---------------------------------------------------------------------------
__global__ void regroup_keys_kernel(const uint32_t *level, const int32_t *type, int64_t n, int tbits,
                                    uint32_t *keys, uint32_t *vals, const uint32_t *n_live,
                                    const uint32_t *bulk_of, const uint32_t *seg_base)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (n_live && t >= (int64_t)*n_live) {
        keys[t] = (uint32_t)n << tbits;   // padding: past every real level
    } else {
        const int32_t ty = type[t];
        // a segment's levels run bulk after bulk: global level = the bulk's
        // first global level + the level within the bulk
        const uint32_t lv = level[t] + (bulk_of ? seg_base[bulk_of[t]] : 0u);
        keys[t] = (lv << tbits) | (tbits && ty > 0 ? (uint32_t)ty : 0u);
    }
    vals[t] = (uint32_t)t;
}

// the bulk of each live transaction of a segment (seg_off: first
// transaction of each of its n_seg bulks, ascending from 0)
__global__ void seg_index_kernel(const uint32_t *seg_off, const BulkCtl *ctl, uint32_t *bulk_of, int64_t cap)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= cap) return;
    const uint32_t nseg = ctl->n_seg < 1 ? 1u : (ctl->n_seg > (uint32_t)kSegMax ? (uint32_t)kSegMax : ctl->n_seg);
    uint32_t lo = 0, hi = nseg - 1;   // last bulk whose start is <= t
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= (uint32_t)t) lo = mid;
        else hi = mid - 1;
    }
    bulk_of[t] = lo;
}

__global__ void seg_depth_kernel(const uint32_t *level, const uint32_t *bulk_of, const BulkCtl *ctl,
                                 uint32_t *seg_depth, int64_t cap)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= cap || t >= (int64_t)ctl->n_live) return;
    atomicMax(&seg_depth[bulk_of[t]], level[t]);
}

// first global level of each bulk; the segment's depth becomes the last
// global level
__global__ void seg_base_kernel(const uint32_t *seg_depth, BulkCtl *ctl, uint32_t *seg_base)
{
    if (threadIdx.x != 0) return;
    const uint32_t nseg = ctl->n_seg < 1 ? 1u : (ctl->n_seg > (uint32_t)kSegMax ? (uint32_t)kSegMax : ctl->n_seg);
    uint32_t acc = 0;
    for (uint32_t i = 0; i < nseg; i++) {
        seg_base[i] = acc;
        acc += seg_depth[i] + 1;
    }
    seg_base[nseg] = acc;
    ctl->depth = acc - 1;
}

__global__ void part_fallback_kernel(BulkCtl *ctl)
{
    if (ctl->cross) ctl->err |= ERR_FALLBACK;
}

// Level boundaries from the keys sorted by (level << tbits | type); with
// type_cut, also where each level's new-order, payment and order-status
// transactions start (type_cut[3 k + j] = first position of level k whose
// type is >= 8 + j), so the executors can give order-entry's line-parallel
// types their lane groups.  A cut (k, type) lands on the first key at or
// above k << tbits | type; levels are contiguous, so between two adjacent
// keys at most two levels' cuts fall.
// a debug build's check of the level table the executors index by: the
// bounds of levels 0..depth rise and stay within the bulk (an executor whose
// bulk carries an error returns before its first gather)
__global__ void check_level_off_kernel(const uint32_t *level_off, int64_t n, BulkCtl *ctl)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ctl->err || k > (int64_t)ctl->depth || k >= n) return;
    const uint32_t lo = level_off[k], hi = level_off[k + 1];
    if (lo > hi || !dbg_in(hi, n + 1, &ctl->err)) set_err(&ctl->err, ERR_BOUNDS);
}

__global__ void level_off_kernel(const uint32_t *skeys, int64_t n, int tbits, uint32_t *level_off,
                                 uint32_t *type_cut, const BulkCtl *ctl, const uint32_t *err)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n || *err) return;
    // real levels are 0..depth; a graph bulk's padding sorts after them as
    // level n, whose boundary is the only one needed past depth
    const uint32_t top = ctl->depth + 1;
    const uint32_t key = skeys[i];
    const uint32_t lv = key >> tbits;
    const uint32_t lvc = lv < top ? lv : top;
    const uint32_t prev = i ? (skeys[i - 1] >> tbits) : 0u;
    if (i == 0) {
        for (uint32_t k = 0; k <= lvc; k++) level_off[k] = 0;
    } else if (lv != prev) {
        for (uint32_t k = prev + 1; k <= lvc; k++) level_off[k] = (uint32_t)i;
    }
    if (i == n - 1 && lv < top) level_off[lv + 1] = (uint32_t)n;
    if (type_cut && (i == 0 || skeys[i - 1] != key)) {
        const uint64_t below = i ? (uint64_t)skeys[i - 1] + 1 : 0;   // cuts in (key[i-1], key[i]]
        const uint32_t kmax = lv < top ? lv : top - 1;
        for (uint32_t k = i ? prev : 0; k <= kmax; k++)
            for (uint32_t j = 0; j < 3; j++) {
                const uint64_t cut = ((uint64_t)k << tbits) | (GPUTX_T_OE_NEW_ORDER + j);
                if (cut >= below && cut <= key) type_cut[3 * k + j] = (uint32_t)i;
            }
    }
    if (type_cut && i == n - 1 && lv < top)
        for (uint32_t j = 0; j < 3; j++) {
            const uint64_t cut = ((uint64_t)lv << tbits) | (GPUTX_T_OE_NEW_ORDER + j);
            if (cut > key) type_cut[3 * lv + j] = (uint32_t)n;
        }
}

struct ChunkMode {
    const uint32_t *level_off;
    uint32_t *chunk_off;
    uint32_t block;
    const BulkCtl *ctl;   // levels = depth + 1, read on the device
    const uint32_t *type_cut;   // chunks count lanes (order-entry groups) when set
    __device__ uint64_t element(int64_t k) const
    {
        if (k > (int64_t)ctl->depth) return 0;
        const uint32_t w = level_lane_count(level_off[k], level_off[k + 1], type_cut ? type_cut + 3 * k : nullptr);
        return DualSeg::make(0, 0, 0, (w + block - 1) / block);
    }
    __device__ void output(int64_t k, uint64_t s) const
    {
        chunk_off[k + 1] = DualSeg::v2(s);
        if (k == 0) chunk_off[0] = 0;
    }
};

__global__ void chunk_level_kernel(const uint32_t *chunk_off, const BulkCtl *ctl, uint32_t *chunk_level,
                                   int64_t cap, const uint32_t *err)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (*err) return;
    const int64_t levels = (int64_t)ctl->depth + 1;
    const uint32_t nchunks = chunk_off[levels];
    if (c >= cap || c >= nchunks) return;
    // largest k with chunk_off[k] <= c
    int64_t lo = 0, hi = levels - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (chunk_off[mid] <= (uint32_t)c) lo = mid;
        else hi = mid - 1;
    }
    chunk_level[c] = (uint32_t)lo;
}

// ---------------------------------------------------------------------------
// a7: deterministic insert slots: exclusive counts in timestamp order
// ---------------------------------------------------------------------------
struct SlotMode {
    const int32_t *type;
    const int64_t *params;
    int P;
    int64_t n;
    uint32_t *slot_a, *slot_b;
    BulkCtl *ctl;
    int which;   // 0: (call-forwarding inserts, orders) 1: (-, order lines)
    __device__ uint32_t a(int64_t t) const
    {
        return which == 0 ? (type[t] == GPUTX_T_SUB_INSERT_CF) : 0u;
    }
    __device__ uint32_t bv(int64_t t) const
    {
        if (type[t] != GPUTX_T_OE_NEW_ORDER) return 0u;
        if (which == 0) return 1u;
        const int64_t c = params[t * P + 3];
        return (c >= 1 && c <= OE_MAX_LINES) ? (uint32_t)c : 0u;
    }
    __device__ uint64_t element(int64_t t) const { return DualSeg::make(0, a(t), 0, bv(t)); }
    __device__ void output(int64_t t, uint64_t s) const
    {
        const uint32_t ia = DualSeg::v1(s), ib = DualSeg::v2(s);
        if (which == 0) {
            slot_a[t] = ia - a(t);
            slot_b[t] = ib - bv(t);
            if (t == n - 1) { ctl->total.cf = ia; ctl->total.ord = ib; }
        } else {
            slot_b[t] = ib - bv(t);
            if (t == n - 1) ctl->total.ol = ib;
        }
    }
};

// ---------------------------------------------------------------------------
// PART: partition starts; TPL: counter reset
// ---------------------------------------------------------------------------
// partition heads in sorted order: part_start[p] = first position of the
// p-th partition, part_start[npart] = n (a compaction by prefix count)
struct HeadMode {
    const uint32_t *skeys;
    uint32_t *part_start;
    BulkCtl *ctl;
    int64_t n;
    const uint32_t *n_live;   // graph bulks: padding (sorted last) forms no partition
    __device__ int64_t live() const { return n_live ? (int64_t)*n_live : n; }
    __device__ bool head(int64_t i) const { return i < live() && (i == 0 || skeys[i] != skeys[i - 1]); }
    __device__ uint64_t element(int64_t i) const { return DualSeg::make(0, 0, 0, head(i) ? 1u : 0u); }
    __device__ void output(int64_t i, uint64_t s) const
    {
        const uint32_t c = DualSeg::v2(s);
        if (head(i)) part_start[c - 1] = (uint32_t)i;
        if (i == live() - 1) {
            part_start[c] = (uint32_t)live();
            ctl->npart = c;
        }
    }
};

// records of a debit-credit bulk packed in execution order (32 B: two
// 16-byte loads), teller and branch precomputed
__global__ void gather_dc_kernel(DevDB db, DevBulk b, const uint32_t *order, DcRecord *rec, const uint32_t *err)
{
    const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= b.n || *err) return;
    const uint32_t t = order[pos];
    if (!dbg_in(t, b.n, b.err)) return;
    const uint32_t a = (uint32_t)b.params[(int64_t)t * b.P];
    DcRecord r;
    r.delta = b.params[(int64_t)t * b.P + 1];
    r.ts = b.ts[t];
    r.a = a;
    r.t = t;
    r.tl = db.div_tel.div(a);
    r.br = db.div_br.div(a);
    rec[pos] = r;
}

__global__ void tpl_reset_kernel(const uint32_t *skeys, int64_t m, uint32_t *done, uint32_t n_objects,
                                 LockSlots slot)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    const uint32_t k = skeys[i];
    if ((i == 0 || skeys[i - 1] != k) && k < n_objects) done[slot(k)] = 0;
}

template <class Mode>
cudaError_t run_scan(gputx_bulk *b, const Mode &mode, int64_t count, int ctr_slot)
{
    if (count <= 0) return cudaSuccess;
    const int64_t tiles = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles > b->sc.scan_tiles) return cudaErrorInvalidValue;
    cudaStream_t s = b->stream;
    cudaError_t e = cudaMemsetAsync(b->sc.scan_status, 0, tiles * sizeof(uint64_t), s);
    if (e) return e;
    e = cudaMemsetAsync(b->sc.tile_ctr + ctr_slot, 0, sizeof(uint32_t), s);
    if (e) return e;
    dualseg_scan_kernel<Mode><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(
        mode, count, b->sc.scan_status, b->sc.tile_ctr + ctr_slot, &b->ctl->err,
        (uint64_t)b->db->cfg.spin_limit_ns);
    count_launches(1);
    return cudaGetLastError();
}

inline DevBulk dev_bulk(gputx_bulk *b, int mode)
{
    DevBulk d{};
    d.n = b->n;
    d.P = b->P;
    d.R = b->R;
    d.ts = b->ts;
    d.type = b->type;
    d.params = b->params;
    d.status = b->status;
    d.out = b->out;
    d.err = &b->ctl->err;
    d.base = &b->ctl->base;
    d.slot_cf = b->sc.slot_cf;
    d.slot_ord = b->sc.slot_ord;
    d.slot_ol = b->sc.slot_ol;
    d.slot_hist = b->sc.slot_hist;
    d.rec_params = b->sc.rec_params;
    d.rec_ts = b->sc.rec_ts;
    d.rec_type = b->sc.rec_type;
    d.rec_t = b->sc.rec_t;
    d.n_live = b->graph ? &b->ctl->n_live : nullptr;
    d.conflict_mode = mode;
    return d;
}

// the bulk's signatures permuted into execution order: executors then read
// them sequentially instead of chasing order[] into random rows
__global__ void gather_kernel(DevBulk b, const uint32_t *order, int64_t *r_params, int64_t *r_ts,
                              int32_t *r_type, uint32_t *r_t, const uint32_t *err)
{
    const int64_t pos = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (pos >= b.n || *err) return;
    const uint32_t t = order[pos];
    if (!dbg_in(t, b.n, b.err)) return;
    r_t[pos] = t;
    r_ts[pos] = b.ts[t];
    r_type[pos] = b.type[t];
    const int64_t *src = b.params + (int64_t)t * b.P;
    int64_t *dst = r_params + pos * b.P;
    for (int j = 0; j < b.P; j++) dst[j] = src[j];
}

// ---------------------------------------------------------------------------
// relaxed timestamps (Appendix G): validation and counter-based grouping
// ---------------------------------------------------------------------------
__global__ void validate_kernel(DevDB db, DevBulk b, BulkCtl *ctl)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < b.n && !txn_valid(db, b, t)) set_err(&ctl->err, ERR_INVAL);
}

// each transaction takes the next counter value of its partition as its
// position in the partition (the order of the atomics is the relaxation).
// With few partitions a block first counts in shared memory, then takes one
// global range per partition it saw (kPartCountItems transactions a thread),
// so 4 M transactions over 1,000 counters do not serialise on the counters.
constexpr int kPartCountThreads = 1024, kPartCountItems = 8, kPartLocalMax = 4096;

__device__ __forceinline__ bool part_of(const DevDB &db, const DevBulk &b, int64_t t, int mode, int part_size,
                                        uint32_t &pid, bool &cross)
{
    if (!txn_valid(db, b, t)) return false;
    uint32_t obj[MAX_OPS], root[MAX_OPS];
    uint8_t cls[MAX_OPS];
    const int k = access_set(db, b.type[t], b.params + t * b.P, mode, obj, cls, root);
    pid = k ? root[0] / (uint32_t)part_size : 0;
    for (int j = 1; j < k; j++) cross |= (root[j] / (uint32_t)part_size) != pid;
    return true;
}

template <bool LOCAL>
__global__ void __launch_bounds__(kPartCountThreads) part_count_kernel(DevDB db, DevBulk b, BulkCtl *ctl, int mode,
                                                                       int part_size, uint32_t *cnt, int64_t parts,
                                                                       uint32_t *pid_of, uint32_t *key_of)
{
    __shared__ uint32_t scnt[LOCAL ? kPartLocalMax : 1], sbase[LOCAL ? kPartLocalMax : 1];
    if (LOCAL) {
        for (int64_t p = threadIdx.x; p < parts; p += blockDim.x) scnt[p] = 0;
        __syncthreads();
    }
    const int64_t base = (int64_t)blockIdx.x * kPartCountThreads * kPartCountItems + threadIdx.x;
    uint32_t pid[kPartCountItems], local[kPartCountItems];
    bool ok[kPartCountItems];
    bool cross = false;
#pragma unroll
    for (int j = 0; j < kPartCountItems; j++) {
        const int64_t t = base + (int64_t)j * kPartCountThreads;
        pid[j] = 0;
        local[j] = 0;
        ok[j] = false;
        if (t < b.n) {
            ok[j] = part_of(db, b, t, mode, part_size, pid[j], cross);
            if (!ok[j]) set_err(&ctl->err, ERR_INVAL);
            else local[j] = LOCAL ? atomicAdd(&scnt[pid[j]], 1u) : atomicAdd(&cnt[pid[j]], 1u);
        }
    }
    if (LOCAL) {
        __syncthreads();
        // the block's first transaction of each partition takes the range
#pragma unroll
        for (int j = 0; j < kPartCountItems; j++)
            if (ok[j] && local[j] == 0) sbase[pid[j]] = atomicAdd(&cnt[pid[j]], scnt[pid[j]]);
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kPartCountItems; j++) {
        const int64_t t = base + (int64_t)j * kPartCountThreads;
        if (t < b.n) {
            pid_of[t] = pid[j];
            key_of[t] = ok[j] ? (LOCAL ? sbase[pid[j]] + local[j] : local[j]) : 0;
        }
    }
    const uint32_t cross_mask = __ballot_sync(0xffffffffu, cross);
    if ((threadIdx.x & 31) == 0 && cross_mask) atomicAdd(&ctl->cross, (uint32_t)__popc(cross_mask));
}

// position = start of the partition (prefix sum of the counters) + counter value
__global__ void part_scatter_kernel(int64_t n, const uint32_t *off, const uint32_t *pid_of, const uint32_t *key_of,
                                    uint32_t *pkeys, uint32_t *order, const uint32_t *err)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n || *err) return;
    const uint32_t pid = pid_of[t];
    const uint32_t pos = off[pid] + key_of[t];
    pkeys[pos] = pid;
    order[pos] = (uint32_t)t;
}

// ---------------------------------------------------------------------------
// SCAN executor for bulks of debit-credit transactions (blind increments,
// the ADD refinement taken to its end).  Under Definition 1 the output of
// transaction t is its account's balance before the bulk plus the deltas of
// the bulk's transactions on that account up to and including t, in
// timestamp order: a segmented prefix sum over the operations grouped by
// account (the stable grouping sort keeps timestamp order inside a group).
// Teller and branch balances only receive sums, and wrapping addition is
// associative and commutative, so atomic adds give the serial result.
// ---------------------------------------------------------------------------
struct ScanExecMode {
    const uint32_t *sk, *sv;     // operations grouped by account object id
    const int64_t *params;
    int64_t *acc_bal, *out;
    int32_t *status;
    int64_t m;
    int P, R;
    uint32_t o_acc;
    __device__ Seg64 element(int64_t i) const
    {
        const uint32_t k = sk[i], t = sv[i] >> 7;
        const bool head = i == 0 || sk[i - 1] != k;
        const uint64_t d = (uint64_t)__ldg(&params[(int64_t)t * P + 1]);
        // the balance before the bulk matters only at the first operation on
        // the account; loading it for every operation keeps the loads free of
        // branches, so the tile's loads all overlap
        const uint64_t bal = (uint64_t)__ldcg(&acc_bal[k - o_acc]);
        return Seg64::make(head ? 1u : 0u, head ? bal + d : d);
    }
    __device__ void output(int64_t i, const Seg64 &s) const
    {
        const uint32_t k = sk[i], t = sv[i] >> 7;
        out[(int64_t)t * R] = (int64_t)s.v;
        // last operation on the account: its balance after the bulk (every
        // tile reading this account's balance published its aggregate
        // before this tile finished its look-back)
        if (i == m - 1 || sk[i + 1] != k) __stcg(&acc_bal[k - o_acc], (int64_t)s.v);
    }
};

// the whole bulk's history rows fit, or nothing of it runs
__global__ void scan_capacity_kernel(BulkCtl *ctl, int64_t n, int64_t hist_cap)
{
    if (ctl->base.hist + n > hist_cap) set_err(&ctl->err, ERR_CAPACITY);
}

// history rows in timestamp order (slot = base + t) and the teller and branch
// sums; reads the signatures sequentially.  With `local` the sums gather in
// shared memory first (one slot per teller and branch) and each block adds
// its non-zero sums once: the same-address atomics on the few branch rows
// would otherwise serialise in L2.
__global__ void scan_dc_rows_kernel(DevDB db, DevBulk b, const BulkCtl *ctl, bool local)
{
    extern __shared__ unsigned long long sums[];   // [n_tel] tellers, then [n_br] branches
    const bool stop = ctl->err != 0;               // uniform: set before this launch
    if (stop) return;
    const uint32_t n_tel = (uint32_t)db.n_tel, n_br = (uint32_t)db.n_br;
    if (local) {
        for (uint32_t i = threadIdx.x; i < n_tel + n_br; i += blockDim.x) sums[i] = 0;
        __syncthreads();
    }
    const int64_t hb = ctl->base.hist;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < b.n;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t a = (uint32_t)b.params[t * b.P];
        const int64_t d = b.params[t * b.P + 1];
        const uint32_t tl = db.div_tel.div(a), br = db.div_br.div(a);
        const int64_t slot = hb + t;
        db.h_ts[slot] = b.ts[t];
        db.h_acc[slot] = a;
        db.h_tel[slot] = tl;
        db.h_br[slot] = br;
        db.h_delta[slot] = d;
        b.status[t] = 0;   // here, in timestamp order, rather than scattered by the scan
        if (local) {
            atomicAdd(&sums[tl], (unsigned long long)d);
            atomicAdd(&sums[n_tel + br], (unsigned long long)d);
        } else {
            atomicAdd((unsigned long long *)&db.tel_bal[tl], (unsigned long long)d);
            atomicAdd((unsigned long long *)&db.br_bal[br], (unsigned long long)d);
        }
    }
    if (local) {
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n_tel + n_br; i += blockDim.x) {
            const unsigned long long v = sums[i];
            if (!v) continue;
            unsigned long long *dst = i < n_tel ? (unsigned long long *)&db.tel_bal[i]
                                                : (unsigned long long *)&db.br_bal[i - n_tel];
            atomicAdd(dst, v);
        }
    }
}

}  // namespace

DevBulk make_dev_bulk(gputx_bulk *b, int mode) { return dev_bulk(b, mode); }

cudaError_t launch_scan_exec(gputx_bulk *b, const uint32_t *sk, const uint32_t *sv, int64_t m)
{
    gputx_db *db = b->db;
    cudaStream_t s = b->stream;
    scan_capacity_kernel<<<1, 1, 0, s>>>(b->ctl, b->n, db->dev.hist_cap);
    count_launches(1);
    if (m > 0) {
        const int64_t tiles = (m + SCAN_TILE - 1) / SCAN_TILE;
        if (tiles > b->sc.scan_tiles) return cudaErrorInvalidValue;
        ScanExecMode mode;
        mode.sk = sk;
        mode.sv = sv;
        mode.params = b->params;
        mode.acc_bal = db->dev.acc_bal;
        mode.out = b->out;
        mode.status = b->status;
        mode.m = m;
        mode.P = b->P;
        mode.R = b->R;
        mode.o_acc = db->dev.o_acc;
        Seg64Status st;
        st.word = (uint32_t *)b->sc.scan_status;
        st.agg = b->sc.scan_vals;
        st.inc = b->sc.scan_vals + tiles;
        cudaError_t e = cudaMemsetAsync(st.word, 0, tiles * sizeof(uint32_t), s);
        if (!e) e = cudaMemsetAsync(b->sc.tile_ctr + 12, 0, sizeof(uint32_t), s);
        if (e) return e;
        seg64_scan_kernel<ScanExecMode><<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(
            mode, m, st, b->sc.tile_ctr + 12, &b->ctl->err, (uint64_t)db->cfg.spin_limit_ns);
        count_launches(1);
    }
    if (b->n > 0) {
        // teller and branch sums in shared memory when they fit, one block per SM
        const size_t smem = (size_t)(db->dev.n_tel + db->dev.n_br) * sizeof(unsigned long long);
        const bool local = smem <= (200u << 10);
        const int threads = 1024;
        int64_t grid = (b->n + threads - 1) / threads;
        if (grid > (int64_t)db->num_sms) grid = db->num_sms;
        if (local && smem > (48u << 10)) {
            const cudaError_t e = cudaFuncSetAttribute(scan_dc_rows_kernel,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e) return e;
        }
        scan_dc_rows_kernel<<<(unsigned)grid, threads, local ? smem : 0, s>>>(
            db->dev, dev_bulk(b, GPUTX_CONFLICT_ADD), b->ctl, local);
        count_launches(1);
    }
    return cudaGetLastError();
}

cudaError_t launch_gather(gputx_bulk *b, const uint32_t *order)
{
    if (b->n == 0) return cudaSuccess;
    const DevBulk d = dev_bulk(b, 0);
    gather_kernel<<<grid_for(b->n), TB, 0, b->stream>>>(d, order, b->sc.rec_params, b->sc.rec_ts,
                                                             b->sc.rec_type, b->sc.rec_t, &b->ctl->err);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_gather_dc(gputx_bulk *b, const uint32_t *order)
{
    if (b->n == 0) return cudaSuccess;
    if (!b->sc.rec_dc) return cudaErrorInvalidValue;
    gather_dc_kernel<<<grid_for(b->n), TB, 0, b->stream>>>(b->db->dev, dev_bulk(b, 0), order, b->sc.rec_dc,
                                                                &b->ctl->err);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_validate(gputx_bulk *b)
{
    if (b->n == 0) return cudaSuccess;
    validate_kernel<<<grid_for(b->n), TB, 0, b->stream>>>(b->db->dev, dev_bulk(b, 0), b->ctl);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_part_count(gputx_bulk *b, int mode, int part_size, uint32_t *cnt, int64_t parts,
                              uint32_t *pid_of, uint32_t *key_of)
{
    if (b->n == 0) return cudaSuccess;
    const int64_t per_block = (int64_t)kPartCountThreads * kPartCountItems;
    const unsigned grid = (unsigned)((b->n + per_block - 1) / per_block);
    const int ps = part_size < 1 ? 1 : part_size;
    if (parts <= kPartLocalMax)
        part_count_kernel<true><<<grid, kPartCountThreads, 0, b->stream>>>(b->db->dev, dev_bulk(b, mode), b->ctl,
                                                                          mode, ps, cnt, parts, pid_of, key_of);
    else
        part_count_kernel<false><<<grid, kPartCountThreads, 0, b->stream>>>(b->db->dev, dev_bulk(b, mode), b->ctl,
                                                                           mode, ps, cnt, parts, pid_of, key_of);
    count_launches(1);
    return cudaGetLastError();
}

// exclusive offsets of `parts` counters: off[p] = start of partition p,
// off[parts] = total (scan scratch supplied by the caller)
cudaError_t launch_part_offsets(gputx_bulk *b, const uint32_t *cnt, uint32_t *off, int64_t parts, uint64_t *status,
                                uint32_t *tile_ctr)
{
    if (parts <= 0) return cudaSuccess;
    OffsetMode om{cnt, off, parts};
    const int64_t tiles = (parts + SCAN_TILE - 1) / SCAN_TILE;
    cudaError_t e = cudaMemsetAsync(status, 0, tiles * sizeof(uint64_t), b->stream);
    if (!e) e = cudaMemsetAsync(tile_ctr, 0, sizeof(uint32_t), b->stream);
    if (e) return e;
    dualseg_scan_kernel<OffsetMode><<<(unsigned)tiles, SCAN_THREADS, 0, b->stream>>>(
        om, parts, status, tile_ctr, &b->ctl->err, (uint64_t)b->db->cfg.spin_limit_ns);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_part_scatter(gputx_bulk *b, const uint32_t *off, const uint32_t *pid_of, const uint32_t *key_of,
                                uint32_t *pkeys, uint32_t *order)
{
    if (b->n == 0) return cudaSuccess;
    part_scatter_kernel<<<grid_for(b->n), TB, 0, b->stream>>>(b->n, off, pid_of, key_of, pkeys, order,
                                                                &b->ctl->err);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_begin(gputx_bulk *b)
{
    const bool dc = (b->db->dev.registered & 1u) != 0;
    const int64_t rows = b->sc.slot_hist ? -1 : (dc ? b->n : 0);
    begin_kernel<<<1, 1, 0, b->stream>>>(b->db->d_cursor, b->ctl, rows, dc && b->graph);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_finish(gputx_bulk *b)
{
    finish_kernel<<<1, 1, 0, b->stream>>>(b->db->d_cursor, b->ctl);
    count_launches(1);
    return cudaGetLastError();
}

int seg_bits(const gputx_db *db)
{
    // segment bulk ids sit above the object id in a 32-bit key
    const int room = 32 - db->obj_bits;
    return room < 1 ? 0 : (room > 6 ? 6 : room);
}

cudaError_t launch_seg_index(gputx_bulk *b)
{
    if (b->n == 0 || !b->sc.bulk_of) return cudaSuccess;
    seg_index_kernel<<<grid_for(b->n), TB, 0, b->stream>>>(b->sc.seg_off, b->ctl, b->sc.bulk_of, b->n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_seg_levels(gputx_bulk *b)
{
    if (b->n == 0 || !b->sc.bulk_of) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(b->sc.seg_depth, 0, kSegMax * sizeof(uint32_t), b->stream);
    if (e) return e;
    seg_depth_kernel<<<grid_for(b->n), TB, 0, b->stream>>>(b->sc.level, b->sc.bulk_of, b->ctl, b->sc.seg_depth, b->n);
    seg_base_kernel<<<1, 32, 0, b->stream>>>(b->sc.seg_depth, b->ctl, b->sc.seg_base);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_part_fallback_check(gputx_bulk *b)
{
    part_fallback_kernel<<<1, 1, 0, b->stream>>>(b->ctl);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_extract(gputx_bulk *b, int mode, int part_size, uint32_t *pid_key, uint32_t *pid_val,
                           bool write_ops, bool segmented)
{
    gputx_db *db = b->db;
    cudaStream_t s = b->stream;
    if (b->n == 0) return cudaSuccess;
    ExtractArgs a{};
    a.db = db->dev;
    a.b = dev_bulk(b, mode);
    a.ctl = b->ctl;
    a.keys = b->sc.keys_a;
    a.vals = b->sc.vals_a;
    a.uniform_k = db->uniform_k;
    a.mode = mode;
    a.part_size = part_size < 1 ? 1 : part_size;
    a.pid_key = pid_key;
    a.pid_val = pid_val;
    a.write_ops = write_ops;
    a.sentinel_fill = b->graph;
    a.sentinel_key = db->dev.n_objects;
    if (b->graph) a.uniform_k = db->kmax;
    if (segmented && b->graph && b->sc.bulk_of && seg_bits(db) > 0) {
        a.bulk_of = b->sc.bulk_of;
        a.obj_shift = db->obj_bits;
        a.sentinel_key = (uint32_t)(((1ull << seg_bits(db)) - 1) << db->obj_bits);   // after every bulk
    }
    {
        const int64_t roots = std::max<int64_t>({db->dev.n_br, db->dev.n_sub, db->dev.n_wh, 1});
        a.pad_pid = (uint32_t)((roots + a.part_size - 1) / a.part_size);
    }
    if (!db->uniform_k && write_ops && !b->graph) {
        // counts into level[] (free until the rank scan), then offsets
        count_ops_kernel<<<grid_for(b->n), TB, 0, s>>>(db->dev, a.b, b->ctl, b->sc.level);
        count_launches(1);
        cudaError_t e = cudaGetLastError();
        if (e) return e;
        OffsetMode om{b->sc.level, b->sc.op_off, b->n};
        e = run_scan(b, om, b->n, 0);
        if (e) return e;
        a.op_off = b->sc.op_off;
    }
    extract_kernel<<<grid_for(b->n), TB, 0, s>>>(a);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_sort(gputx_bulk *b, uint32_t *&keys, uint32_t *&vals, uint32_t *&keys_alt, uint32_t *&vals_alt,
                        int64_t count, int bits)
{
    if (count <= 1 || bits <= 0) return cudaSuccess;
    cudaStream_t s = b->stream;
    const int passes = (bits + 7) / 8;
    const int64_t tiles = (count + SORT_TILE - 1) / SORT_TILE;
    if (tiles > b->sc.sort_tiles || passes > 4) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(b->sc.sort_hist, 0, 4 * RADIX * sizeof(uint32_t), s);
    if (e) return e;
    e = cudaMemsetAsync(b->sc.sort_status, 0, (size_t)passes * tiles * RADIX * sizeof(uint32_t), s);
    if (e) return e;
    e = cudaMemsetAsync(b->sc.tile_ctr + 8, 0, 4 * sizeof(uint32_t), s);
    if (e) return e;
    static bool smem_set = false;
    if (!smem_set) {
        e = cudaFuncSetAttribute(radix_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SORT_SMEM);
        if (e) return e;
        smem_set = true;
    }
    int hist_blocks = b->db->num_sms * 4;
    const int64_t need = (count + 255) / 256;
    if (hist_blocks > need) hist_blocks = (int)need;
    radix_hist_kernel<<<hist_blocks, 256, 0, s>>>(keys, count, passes, b->sc.sort_hist, &b->ctl->err);
    count_launches(1);
    radix_offsets_kernel<<<passes, RADIX, 0, s>>>(b->sc.sort_hist, b->sc.sort_offs);
    count_launches(1);
    for (int p = 0; p < passes; p++) {
        radix_pass_kernel<<<(unsigned)tiles, SORT_THREADS, SORT_SMEM, s>>>(
            keys, vals, keys_alt, vals_alt, count, 8 * p, b->sc.sort_offs + p * RADIX,
            b->sc.sort_status + (size_t)p * tiles * RADIX, b->sc.tile_ctr + 8 + p, &b->ctl->err,
            (uint64_t)b->db->cfg.spin_limit_ns);
        count_launches(1);
        e = cudaGetLastError();
        if (e) return e;
        uint32_t *t = keys; keys = keys_alt; keys_alt = t;
        t = vals; vals = vals_alt; vals_alt = t;
    }
    return cudaSuccess;
}

cudaError_t launch_rank_scan(gputx_bulk *b, const uint32_t *sk, const uint32_t *sv, int64_t m, bool want_rid)
{
    cudaError_t e = cudaMemsetAsync(b->sc.level, 0, b->n * sizeof(uint32_t), b->stream);
    if (e) return e;
    RankMode rm{sk, sv, b->sc.level, want_rid ? b->sc.rid : nullptr};
    return run_scan(b, rm, m, 1);
}

cudaError_t launch_ticket_scan(gputx_bulk *b, const uint32_t *sk, const uint32_t *sv, int64_t m)
{
    const bool fixed = b->db->uniform_k || b->graph;
    // CTA-wide lock groups pay off once a counter's chain reaches about
    // n/512 operations: on debit-credit under R/W (one lock per branch) they
    // run Zipf 0.7 accounts (a branch chain of about n/300) 15 % faster than
    // warp groups, and uniform ones (1,000 chains of about n/1,000) 13 %
    // slower
    const int64_t hot = b->n / 512 > 32 ? b->n / 512 : 32;
    TicketMode tm{sk, sv, b->sc.lock_key, b->sc.lock_ticket, fixed ? nullptr : b->sc.op_off,
                  b->graph ? b->db->kmax : b->db->uniform_k, &b->ctl->hot,
                  (uint32_t)(hot > 0xffffffffll ? 0xffffffffll : hot), b->db->dev.n_objects, &b->ctl->err};
    cudaError_t e = cudaMemsetAsync(&b->ctl->hot, 0, sizeof(uint32_t), b->stream);
    if (e) return e;
    return run_scan(b, tm, m, 2);
}

cudaError_t launch_depth_flow(gputx_bulk *b, const uint32_t *sv, int64_t m)
{
    if (m == 0 || b->n == 0) return cudaSuccess;
    cudaStream_t s = b->stream;
    const bool fixed = b->db->uniform_k || b->graph;
    const uint32_t *op_off = fixed ? nullptr : b->sc.op_off;
    const int kslots = b->graph ? b->db->kmax : b->db->uniform_k;
    // the per-slot run ids reuse a TPL buffer (free during the analysis)
    uint32_t *txn_rid = b->sc.lock_key;
    unsigned long long *runword = reinterpret_cast<unsigned long long *>(b->sc.runmax);
    cudaError_t e;
    if ((e = cudaMemsetAsync(txn_rid, 0xff, (size_t)m * sizeof(uint32_t), s))) return e;
    if ((e = cudaMemsetAsync(runword, 0, (size_t)m * sizeof(unsigned long long), s))) return e;
    if ((e = cudaMemsetAsync(&b->ctl->claim, 0, sizeof(uint32_t), s))) return e;
    depth_prep_kernel<<<grid_for(m), TB, 0, s>>>(sv, b->sc.rid, m, op_off, kslots, txn_rid, runword, b->ctl);
    static int per_sm = 0;
    if (!per_sm) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, depth_flow_kernel, 256, 0);
        if (per_sm > kFlowBlocksPerSm) per_sm = kFlowBlocksPerSm;
        if (per_sm < 1) per_sm = 1;
    }
    int64_t grid = (int64_t)b->db->num_sms * per_sm;
    const int64_t chunks = (b->n + 255) / 256;
    if (grid > chunks) grid = chunks;
    depth_flow_kernel<<<(unsigned)grid, 256, 0, s>>>(txn_rid, op_off, kslots, runword, b->sc.level, b->ctl, b->n,
                                                     (uint64_t)b->db->cfg.spin_limit_ns);
    count_launches(2);
    return cudaGetLastError();
}

// exact depths after the one-pass ranks (A1): the dataflow pass
cudaError_t launch_exact_depth(gputx_bulk *b, const uint32_t *sv, int64_t m)
{
    return launch_depth_flow(b, sv, m);
}

cudaError_t launch_level_stats(gputx_bulk *b)
{
    if (b->n == 0) return cudaSuccess;
    int blocks = b->db->num_sms * 2;
    const int64_t need = (b->n + 255) / 256;
    if (blocks > need) blocks = (int)need;
    level_stats_kernel<<<blocks, 256, 0, b->stream>>>(b->sc.level, b->n, b->ctl);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_regroup_keys(gputx_bulk *b, uint32_t *keys, uint32_t *vals)
{
    if (b->n == 0) return cudaSuccess;
    const bool seg = b->graph && b->sc.bulk_of;
    regroup_keys_kernel<<<grid_for(b->n), TB, 0, b->stream>>>(b->sc.level, b->type, b->n, b->db->tbits,
                                                               keys, vals, b->graph ? &b->ctl->n_live : nullptr,
                                                               seg ? b->sc.bulk_of : nullptr,
                                                               seg ? b->sc.seg_base : nullptr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_level_tables(gputx_bulk *b, const uint32_t *skeys, int64_t depth, int block, bool chunks)
{
    cudaStream_t s = b->stream;
    if (b->n == 0) return cudaSuccess;
    level_off_kernel<<<grid_for(b->n), TB, 0, s>>>(skeys, b->n, b->db->tbits, b->sc.level_off, b->sc.type_cut,
                                                   b->ctl, &b->ctl->err);
    count_launches(1);
    if (kDebug) {
        check_level_off_kernel<<<grid_for(b->n + 1), TB, 0, s>>>(b->sc.level_off, b->n, b->ctl);
        count_launches(1);
    }
    if (!chunks) return cudaGetLastError();
    // graph bulks do not know their depth on the host: scan every possible level
    const int64_t levels = b->graph ? b->n : depth + 1;
    ChunkMode cm{b->sc.level_off, b->sc.chunk_off, (uint32_t)block, b->ctl, b->sc.type_cut};
    cudaError_t e = run_scan(b, cm, levels, 3);
    if (e) return e;
    chunk_level_kernel<<<grid_for(b->sc.chunk_cap), TB, 0, s>>>(b->sc.chunk_off, b->ctl, b->sc.chunk_level,
                                                                b->sc.chunk_cap, &b->ctl->err);
    count_launches(1);
    return cudaGetLastError();
}

// history rows of a mixed bulk: exclusive count of debit-credit transactions
// in timestamp order
struct HistSlotMode {
    const int32_t *type;
    int64_t n;
    uint32_t *slot;
    BulkCtl *ctl;
    __device__ uint32_t a(int64_t t) const { return type[t] == GPUTX_T_DC_DEBIT_CREDIT ? 1u : 0u; }
    __device__ uint64_t element(int64_t t) const { return DualSeg::make(0, 0, 0, a(t)); }
    __device__ void output(int64_t t, uint64_t s) const
    {
        const uint32_t v = DualSeg::v2(s);
        slot[t] = v - a(t);
        if (t == n - 1) ctl->total.hist = v;
    }
};

cudaError_t launch_insert_slots(gputx_bulk *b)
{
    if (b->n == 0) return cudaSuccess;
    if (b->sc.slot_hist) {
        HistSlotMode hm{b->type, b->n, b->sc.slot_hist, b->ctl};
        cudaError_t e = run_scan(b, hm, b->n, 7);
        if (e) return e;
    }
    const uint32_t reg = b->db->dev.registered;
    const bool sub_ins = (reg >> GPUTX_T_SUB_INSERT_CF) & 1u;
    const bool oe_no = (reg >> GPUTX_T_OE_NEW_ORDER) & 1u;
    if (!sub_ins && !oe_no) return cudaSuccess;
    SlotMode m0{b->type, b->params, b->P, b->n, b->sc.slot_cf, b->sc.slot_ord, b->ctl, 0};
    cudaError_t e = run_scan(b, m0, b->n, 5);
    if (e || !oe_no) return e;
    SlotMode m1{b->type, b->params, b->P, b->n, nullptr, b->sc.slot_ol, b->ctl, 1};
    return run_scan(b, m1, b->n, 6);
}

cudaError_t launch_part_heads(gputx_bulk *b, const uint32_t *skeys, int64_t n)
{
    if (n <= 0) return cudaSuccess;
    HeadMode hm;
    hm.skeys = skeys;
    hm.part_start = b->sc.part_start;
    hm.ctl = b->ctl;
    hm.n = n;
    hm.n_live = b->graph ? &b->ctl->n_live : nullptr;
    return run_scan(b, hm, n, 4);
}

cudaError_t launch_tpl_reset(gputx_bulk *b, const uint32_t *skeys, int64_t m)
{
    if (m == 0) return cudaSuccess;
    tpl_reset_kernel<<<grid_for(m), TB, 0, b->stream>>>(skeys, m, b->db->d_done, b->db->dev.n_objects,
                                                        b->db->lock_slots);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace gtx
