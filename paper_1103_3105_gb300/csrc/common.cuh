// common.cuh -- device-side layout of the database and a bulk, shared by the
// engine's translation units.
//
// HBM layout (all arrays cudaMalloc'd by the database):
//   debit-credit   balance columns int64[branches|tellers|accounts];
//                  history SoA int64[capacity] x 5 (ts, account, teller,
//                  branch, delta) written at deterministic slots.
//   subscriber     16 x int32 fields per row, 64 B rows (two 32 B sectors per
//                  full-row read); child tables are SoA slot pools reached
//                  through open-addressing hash indexes on the composite key.
//   order-entry    SoA columns per table; order / order-line slot pools with a
//                  hash index on (district, o_id).
// Every item that can conflict (Section 4.1) has a dense 32-bit object id:
// one contiguous range per (table, field group).
#pragma once
#include "fastdiv.h"
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gputx.h"

namespace gtx {

enum : uint32_t { CLS_R = 0, CLS_W = 1, CLS_A = 2 };

// device error word bits
enum : uint32_t {
    ERR_INVAL = 1u << 0,
    ERR_TIMEOUT = 1u << 1,
    ERR_BOUNDS = 1u << 2,
    ERR_CAPACITY = 1u << 3,
    ERR_FALLBACK = 1u << 4,   // a graph bulk's PART segment has cross-partition transactions: not run
};

constexpr int MAX_OPS = 17;       // largest access set (new-order, 15 lines)
constexpr int MAX_OUT = 8;        // widest output row (subscriber read)
constexpr int OE_DIST = 10;
constexpr int OE_CUST = 3000;
constexpr int OE_MAX_LINES = 15;
constexpr int SUB_FIELDS = 16;

// open-addressing hash index: key -> row slot; empty = ~0ull, deleted = ~1ull
struct HashIndex {
    unsigned long long *keys;
    uint32_t *rows;
    uint64_t mask;                 // capacity - 1 (power of two)
};
constexpr unsigned long long HKEY_EMPTY = ~0ull;
constexpr unsigned long long HKEY_TOMB = ~1ull;

struct DevDB {
    // object id layout
    uint32_t o_acc, o_tel, o_br, o_sub, o_wytd, o_dytd, o_dnext, o_cpay, o_clast, o_stock;
    uint32_t n_objects;

    // debit-credit
    int64_t n_br, n_tel, n_acc, acc_per_tel, acc_per_br;
    FastDiv div_tel, div_br;   // account -> teller, account -> branch
    int64_t *br_bal, *tel_bal, *acc_bal;
    int64_t hist_cap;
    int64_t *h_ts, *h_acc, *h_tel, *h_br, *h_delta;

    // subscriber
    int64_t n_sub;
    int32_t *sub_rows;             // n_sub x 16, 64 B aligned rows
    int64_t child_cap;
    // access_info pool
    int32_t *ai_data;              // child_cap x 4
    int32_t *ai_sid, *ai_type;
    HashIndex ai_idx;
    // special_facility pool
    int32_t *sf_sid, *sf_type, *sf_active, *sf_err, *sf_data_a, *sf_data_b;
    HashIndex sf_idx;
    // call_forwarding pool
    int32_t *cf_sid, *cf_type, *cf_start, *cf_end, *cf_numberx;
    uint8_t *cf_live;
    HashIndex cf_idx;

    // order-entry
    int64_t n_wh, n_items;
    int64_t *w_tax, *w_ytd;
    int64_t *d_tax, *d_ytd, *d_next_o_id;
    int64_t *c_discount, *c_balance, *c_ytd, *c_payment_cnt, *c_last_o_id;
    int64_t *i_price;
    int32_t *s_quantity, *s_order_cnt;
    int64_t *s_ytd;
    int64_t ord_cap, ol_cap;
    int32_t *o_w, *o_d, *o_c, *o_cnt;
    int64_t *o_id, *o_first;       // o_first: first order-line slot
    int32_t *ol_item, *ol_sw, *ol_qty;
    int64_t *ol_amount;
    uint8_t *o_live;
    HashIndex ord_idx;             // key (district << 32 | o_id) -> order slot

    // which types are enabled (bit per type id)
    uint32_t registered;
    int out_width;
};

// a debit-credit transaction packed for the executors (32 B, 16-byte
// aligned: two vector loads), with its teller and branch precomputed
struct __align__(16) DcRecord {
    int64_t delta, ts;
    uint32_t a, t, tl, br;
};

// insert bases of one bulk: where its new rows start in each append area
struct InsertBase {
    int64_t hist, cf, ord, ol;
};

struct DevBulk {
    int64_t n;
    int P, R;
    const int64_t *ts;
    const int32_t *type;
    const int64_t *params;
    int32_t *status;
    int64_t *out;
    uint32_t *err;                 // device error word of this bulk
    const InsertBase *base;        // device: where this bulk's inserts start
    // per-transaction insert slots (exclusive prefix counts in ts order)
    const uint32_t *slot_cf, *slot_ord, *slot_ol;
    // history row of each debit-credit transaction when other types share
    // the bulk (null: the row is the transaction's position)
    const uint32_t *slot_hist;
    // signatures gathered into this strategy's execution order
    const int64_t *rec_params, *rec_ts;
    const int32_t *rec_type;
    const uint32_t *rec_t;
    // fixed-capacity (graph) bulks: transactions at t >= *n_live are padding
    // (no operations, never executed); null = every transaction is live
    const uint32_t *n_live;
    int conflict_mode;
};

constexpr uint32_t OP_SENTINEL = 0xffffffffu;   // payload of a padding operation

// ---------------------------------------------------------------------------
// memory-model helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add(uint32_t *p, uint32_t v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
// a relaxed poll of a counter: several can be in flight at once (an acquire
// load would order each behind the one before); one acquire fence follows
// once every polled counter has reached its value
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acquire_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t *p)
{
    return *(const volatile uint64_t *)p;
}
__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %lanemask_lt;" : "=r"(m));
    return m;
}

// loads/stores of mutable table cells bypass L1 (L2 is the coherence point)
template <class T> __device__ __forceinline__ T ldg_cg(const T *p) { return __ldcg(p); }
template <class T> __device__ __forceinline__ void stg_cg(T *p, T v) { __stcg(p, v); }

__device__ __forceinline__ int64_t wrap_add(int64_t a, int64_t b)
{
    return (int64_t)((unsigned long long)a + (unsigned long long)b);
}

__device__ __forceinline__ void set_err(uint32_t *err, uint32_t bit) { atomicOr(err, bit); }

// Debug builds (compiled with -DGPUTX_DEBUG into libgputx_debug.so) check,
// inside the executors, every index that a gather or scatter takes: positions
// in the bulk and in its execution order, the rows a transaction's parameters
// name, the rows an index probe returns, lock counters, level bounds.  A
// failed check records ERR_BOUNDS in the bulk's error word and the access is
// skipped (its transaction is not executed), so the bulk fails at its sync
// with GPUTX_EBOUNDS instead of touching memory it does not own.  In release
// builds every check compiles away.
#ifdef GPUTX_DEBUG
constexpr bool kDebug = true;
#else
constexpr bool kDebug = false;
#endif

// i in [0, n): a debug build's check (always true in a release build)
__device__ __forceinline__ bool dbg_in(int64_t i, int64_t n, uint32_t *err)
{
    if (!kDebug || (i >= 0 && i < n)) return true;
    set_err(err, ERR_BOUNDS);
    return false;
}

// Where the counter (TPL) or lock (relaxed TPL) of item k lives: slot
// (k mod L) * 32 + k / L of an array of 32 L words, a 32-column transposition
// of the item order.  Consecutive items -- the branches of debit-credit, the
// few hot items of a skewed bulk -- each get their own 128-byte line instead
// of sharing one, so the waiters' polls spread over the L2 slices.
struct LockSlots {
    FastDiv lines;   // L
    __device__ __forceinline__ uint32_t operator()(uint32_t k) const
    {
        const uint32_t q = lines.div(k);
        return (k - q * lines.d) * 32u + q;
    }
};

// L2 prefetch of a row a transaction will touch (a hint: it returns no data,
// so it can run before the transaction is allowed to execute)
__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

}  // namespace gtx
