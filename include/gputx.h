/*
 * gputx.h -- C ABI of the GB300 bulk transaction engine.
 *
 * Implements the bulk execution model of "High-Throughput Transaction
 * Executions on Graphics Processors" (He & Yu):
 *   - transactions are instances of registered stored procedures, each with a
 *     signature <id, type, parameter list> whose id is its timestamp
 *     (Section 3.2);
 *   - a bulk of transactions executes on the GPU as one task, and the result
 *     database and per-transaction outputs equal serial execution in
 *     increasing timestamp order (Definition 1, Section 3.1);
 *   - three strategies: K-SET (Section 5.3), PART (Section 5.2) and TPL
 *     (Section 5.1), all driven by the sort-based dependency analysis of
 *     Section 4.2; AUTO picks one by Algorithm 1 (Appendix D).
 *
 * Conventions (every function):
 *   - Returns a gputx_status; never aborts the process.  The text of the last
 *     failure of a database is available from gputx_last_error().
 *   - Host arrays belong to the caller.  The library copies what it needs
 *     and keeps no host pointer after a call returns.
 *   - All device memory belongs to the database or bulk that allocated it and
 *     is released by gputx_destroy_db / gputx_free_bulk.
 *   - Work is enqueued on the database's CUDA stream.  gputx_execute returns
 *     once the work is enqueued; failures detected on the device (invalid
 *     bulk contents, a bounded wait that ran out, a full insert area) are
 *     returned by the next synchronising call on that bulk:
 *     gputx_sync_bulk or gputx_read_results.
 *   - Integer columns wrap on overflow (two's complement).
 */
#ifndef GPUTX_H
#define GPUTX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPUTX_OK = 0,
    GPUTX_EINVAL = 1,     /* bad argument or bulk contents (type, key, ts order) */
    GPUTX_ENOMEM = 2,     /* device allocation failed or admission refused */
    GPUTX_ECUDA = 3,      /* a CUDA runtime call failed */
    GPUTX_ETIMEOUT = 4,   /* a bounded device wait ran out (no forward progress) */
    GPUTX_EBOUNDS = 5,    /* a device-side bounds check failed */
    GPUTX_ESTATE = 6,     /* call out of order (e.g. executing a bulk twice) */
    GPUTX_ECAPACITY = 7   /* an append-only table or hash index is full */
} gputx_status;

typedef enum {
    GPUTX_KSET = 0,       /* Section 5.3: k-sets level by level */
    GPUTX_PART = 1,       /* Section 5.2: one thread per partition */
    GPUTX_TPL = 2,        /* Section 5.1: ordered counter locks */
    GPUTX_AUTO = 3,       /* Algorithm 1 over the measured d, w0, c.  The
                           * decision reads the one-pass ranks of Section 4.2
                           * (w0 and c exact there, d a lower bound); the
                           * exact-depth pass runs only when
                           * K-SET is chosen, so the reported depth of a PART
                           * or TPL pick is the one-pass depth.  On a database
                           * whose only registered type is debit-credit, AUTO
                           * runs GPUTX_SCAN (same results, one pass). */
    /* Debit-credit bulks only (every registered type is
     * GPUTX_T_DC_DEBIT_CREDIT, else EINVAL): the blind-increment refinement
     * (GPUTX_CONFLICT_ADD) carried to the end.  Operations are grouped by
     * account with the stable sort of Section 4.2. Each output is then the
     * account's balance before the bulk plus a segmented prefix sum of the
     * deltas in timestamp order. Teller and branch balances receive wrapping
     * sums. History rows take slots base + t (timestamp order).  The work
     * does not depend on the depth of the dependency graph; the results are
     * those of Definition 1.  If the bulk's history rows do not all fit, the
     * bulk fails with ECAPACITY and writes nothing. */
    GPUTX_SCAN = 4,
    /* Appendix G, timestamp constraint relaxed: the results equal serial
     * execution in SOME order (serializability), the one gputx_bulk_order
     * reports, instead of timestamp order.
     * PART_RELAXED groups transactions by partition with per-partition
     * counters and a prefix sum (no sort); each partition runs in counter
     * order.  A bulk with a cross-partition transaction runs as TPL_RELAXED.
     * TPL_RELAXED: every transaction takes a spin lock on each of its items in
     * increasing item order (no deadlock), executes, takes a commit ticket
     * while holding the locks and releases them; the ticket order is the
     * serial order.  With GPUTX_CONFLICT_ADD, ADD-class items are updated with
     * atomics instead of locked.  Waits are bounded (ETIMEOUT). */
    GPUTX_PART_RELAXED = 5,
    GPUTX_TPL_RELAXED = 6
} gputx_strategy;

typedef enum {
    /* Section 4.1: every basic operation is a read or a write. */
    GPUTX_CONFLICT_PAPER = 0,
    /* Refinement beyond the paper: increments whose old value is never read
     * (debit-credit teller/branch, order-entry warehouse/district ytd) are a
     * third class ADD that conflicts with reads and writes but not with other
     * ADDs, and execute as atomic additions.  Results are identical because
     * wrapping integer addition is commutative and associative. */
    GPUTX_CONFLICT_ADD = 1
} gputx_conflict_mode;

typedef enum { GPUTX_MEM_HOST = 0, GPUTX_MEM_DEVICE = 1 } gputx_mem;

/* Registered transaction types (the combined kernel's switch, Section 3.2). */
enum {
    GPUTX_T_DC_DEBIT_CREDIT = 0,      /* params: account, delta */
    GPUTX_T_SUB_GET_SUBSCRIBER = 1,   /* params: s_id */
    GPUTX_T_SUB_GET_ACCESS = 2,       /* params: s_id, ai_type */
    GPUTX_T_SUB_GET_NEW_DEST = 3,     /* params: s_id, sf_type, start_time, end_time */
    GPUTX_T_SUB_UPDATE_LOCATION = 4,  /* params: s_id, location */
    GPUTX_T_SUB_UPDATE_FACILITY = 5,  /* params: s_id, sf_type, bit, data_a */
    GPUTX_T_SUB_INSERT_CF = 6,        /* params: s_id, sf_type, start_time, end_time, numberx */
    GPUTX_T_SUB_DELETE_CF = 7,        /* params: s_id, sf_type, start_time */
    GPUTX_T_OE_NEW_ORDER = 8,         /* params: w, d, c, ol_cnt, ol_cnt packed lines */
    GPUTX_T_OE_PAYMENT = 9,           /* params: w, d, c, amount */
    GPUTX_T_OE_ORDER_STATUS = 10,     /* params: w, d, c */
    GPUTX_NUM_TYPES = 11
};

/* Tables, addressed for loading and reading back.  Row transfer format is a
 * fixed number of int64 fields per row (listed beside each table). */
typedef enum {
    GPUTX_TBL_DC_BRANCH = 0,          /* 1: balance (row = branch id) */
    GPUTX_TBL_DC_TELLER = 1,          /* 1: balance (row = teller id) */
    GPUTX_TBL_DC_ACCOUNT = 2,         /* 1: balance (row = account id) */
    GPUTX_TBL_DC_HISTORY = 3,         /* 5: ts, account, teller, branch, delta (read only) */
    GPUTX_TBL_SUB_SUBSCRIBER = 4,     /* 16: int32 fields f0..f15 (row = s_id) */
    GPUTX_TBL_SUB_ACCESS_INFO = 5,    /* 6: s_id, ai_type, data1..data4 */
    GPUTX_TBL_SUB_SPECIAL_FACILITY = 6, /* 6: s_id, sf_type, is_active, error_cntrl, data_a, data_b */
    GPUTX_TBL_SUB_CALL_FORWARDING = 7,  /* 5: s_id, sf_type, start_time, end_time, numberx */
    GPUTX_TBL_OE_WAREHOUSE = 8,       /* 2: tax, ytd (row = w) */
    GPUTX_TBL_OE_DISTRICT = 9,        /* 3: tax, ytd, next_o_id (row = w*10+d) */
    GPUTX_TBL_OE_CUSTOMER = 10,       /* 5: discount, balance, ytd_payment, payment_cnt, last_o_id */
    GPUTX_TBL_OE_ITEM = 11,           /* 1: price */
    GPUTX_TBL_OE_STOCK = 12,          /* 3: quantity, ytd, order_cnt (row = w*n_items+item) */
    GPUTX_TBL_OE_ORDER = 13,          /* 5: w, d, o_id, c, ol_cnt (read only) */
    GPUTX_TBL_OE_ORDER_LINE = 14,     /* 7: w, d, o_id, item, supply_w, qty, amount (read only) */
    GPUTX_NUM_TABLES = 15
} gputx_table;

/* Sizes of the three built-in schemas; a zero count leaves a schema out. */
typedef struct {
    int64_t dc_branches, dc_tellers, dc_accounts;   /* tellers and accounts are
                                                       multiples of branches */
    int64_t dc_history_capacity;                    /* rows */
    int64_t sub_subscribers;
    int64_t sub_child_capacity;  /* rows per child table (0 = 4 per subscriber
                                    + room for inserts) */
    int64_t oe_warehouses, oe_items;
    int64_t oe_order_capacity, oe_orderline_capacity;
} gputx_schema_desc;

/* Engine configuration; zero fields take the documented defaults. */
typedef struct {
    int64_t max_bulk;         /* largest bulk (transactions); default 1<<22 */
    int32_t block_threads;    /* executor CTA size: 128..1024, default 256 */
    int32_t part_size;        /* root keys per PART partition; default 1 for
                                 debit-credit and order-entry, 128 for the
                                 subscriber schema (Appendix E) */
    int64_t spin_limit_ns;    /* bound on every device-side wait; default 2 s */
    int64_t kset_w0_min;      /* Algorithm 1 thresholds; defaults below */
    int64_t part_c_max;
    int64_t part_d_min;
} gputx_config;

/* Filled by gputx_sync_bulk / gputx_read_results when requested. */
typedef struct {
    int32_t strategy;         /* strategy actually run */
    int32_t fallback;         /* 1 when PART fell back to TPL (Section 5.2) */
    int64_t n;                /* transactions */
    int64_t n_ops;            /* basic operations extracted */
    int64_t depth;            /* d: depth of the T-dependency graph */
    int64_t w0;               /* size of the 0-set */
    int64_t cross;            /* c: cross-partition transactions */
    int64_t fixpoint_rounds;  /* exact-depth passes after the one-pass ranks
                               * (1 when they ran, 0 when skipped) */
    float ms_h2d, ms_analysis, ms_sort, ms_execute, ms_d2h, ms_total;
} gputx_exec_stats;

typedef struct {
    int32_t conflict_mode;    /* gputx_conflict_mode */
    int32_t block_threads;    /* 0 = database default */
    int32_t part_size;        /* 0 = database default */
    int32_t timing;           /* 1 = record per-phase CUDA events in stats */
    int32_t kset_launch;      /* K-SET launch shape: 0 = per-level plan (wide
                                 levels on the whole grid, runs of narrow levels
                                 on one thread-block cluster), 1 = one persistent
                                 launch with per-level counters (no host sync
                                 after the analysis) */
    int32_t narrow_max;       /* widest level run on one cluster; 0 = 16384 */
} gputx_exec_opts;

typedef struct gputx_db gputx_db;
typedef struct gputx_bulk gputx_bulk;

/* Creates a database on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = a new non-blocking stream owned by the database).
 * Allocates every table of the schemas whose sizes are non-zero, zeroed, and
 * the dependency-analysis state.  EINVAL on inconsistent sizes, ENOMEM when
 * device memory is short. */
gputx_status gputx_create_db(const gputx_schema_desc *schema, const gputx_config *cfg,
                             void *cuda_stream, gputx_db **out);
void gputx_destroy_db(gputx_db *db);
const char *gputx_last_error(const gputx_db *db);

/* Selects which compiled-in procedures this database accepts (Section 3.2:
 * registering a type = adding its procedure to the combined kernel, which
 * here is compiled in; registration enables it).  EINVAL on an unknown id or
 * a type whose schema was not created. */
gputx_status gputx_register_types(gputx_db *db, const int32_t *type_ids, int n);

/* Bulk loading (initialisation, excluded from throughput by Appendix E):
 * `rows` is n_rows x fields int64 on the host in the table's transfer format.
 * Keyed tables (row = id) take exactly their row count; child tables
 * (access_info, special_facility, call_forwarding) take any number of rows
 * with distinct keys and build their hash index.  EINVAL on a read-only
 * table, a wrong row count, an out-of-range or duplicate key. */
gputx_status gputx_load_table(gputx_db *db, int table, const int64_t *rows, size_t n_rows);

/* Reads the live rows of a table into `rows` (host, capacity_rows x fields
 * int64).  *n_rows receives the live row count; rows == NULL only counts.
 * Child, order and history tables return rows in storage order.
 * Synchronises the database stream. */
gputx_status gputx_read_table(gputx_db *db, int table, int64_t *rows, size_t capacity_rows,
                              size_t *n_rows);

/* The primary indexes of the child and order tables (Section 3.2: tables
 * are reached through their index), for checking them from outside.
 *   index  0 access_info, 1 special_facility, 2 call_forwarding, 3 order.
 *   keys   host uint64[capacity]: the raw open-addressing key array, in slot
 *          order.  ~0 marks an empty slot, ~1 a deleted one (tombstone);
 *          every other value is a live key:
 *            access_info, special_facility   s_id * 4 + (type - 1)
 *            call_forwarding                 (s_id * 4 + (sf_type - 1)) * 3 + start_time / 8
 *            order                           (w * 10 + d) << 32 | o_id
 *          A key sits at the first free slot at or after
 *          mix(key) & (size - 1), probing linearly (mix = the 64-bit
 *          finaliser of MurmurHash3), so a lookup finds it before any empty
 *          slot.
 *   rows   host uint32[capacity]: the table slot each key points to
 *          (meaningful for live keys only; slots as gputx_read_slots numbers
 *          them).
 *   *size  receives the index size (a power of two); keys/rows == NULL only
 *          query it.  EINVAL on an unknown index, one whose schema was not
 *          created, or capacity < size.  Synchronises the database stream. */
gputx_status gputx_read_index(gputx_db *db, int index, uint64_t *keys, uint32_t *rows, size_t capacity,
                              size_t *size);

/* The storage of a child or order table slot by slot, dead slots included,
 * so that gputx_read_index's row numbers can be resolved.  `rows` (host,
 * capacity_rows x (fields + 1) int64) receives for slot i the table's
 * transfer-format fields (as gputx_read_table) followed by a live flag:
 *   access_info, special_facility   slots 0 .. 4 * subscribers - 1, rows in
 *       load order; the flag is 1 when the slot holds a loaded row (these
 *       tables have no inserts or deletions after loading);
 *   call_forwarding                  slots 0 .. rows ever inserted - 1; the
 *       flag is 0 once the row was deleted;
 *   order                            slots 0 .. order slots handed out - 1;
 *       the flag is 0 for the slot of a new-order that aborted.
 * *n_rows receives the slot count; rows == NULL only counts.  EINVAL on
 * another table or capacity_rows < slots.  Synchronises the database
 * stream. */
gputx_status gputx_read_slots(gputx_db *db, int table, int64_t *rows, size_t capacity_rows, size_t *n_rows);

/* Submits a bulk: n transactions as structure-of-arrays, ts[n] strictly
 * increasing int64 timestamps (the ids of Section 3.2), type[n] registered
 * type ids, params[n x params_per_txn] int64.  `mem` says whether the three
 * arrays are host or device memory; host arrays are copied (asynchronously
 * when pinned), device arrays are copied on the device.  Contents are
 * validated on the device; an invalid bulk executes nothing and reports
 * EINVAL at its sync.  EINVAL here for null pointers, n > max_bulk or too few
 * parameters for the registered types; ENOMEM when the bulk's buffers cannot
 * be allocated. */
gputx_status gputx_submit_bulk(gputx_db *db, const int64_t *ts, const int32_t *type,
                               const int64_t *params, int params_per_txn, size_t n, int mem,
                               gputx_bulk **out);

/* Executes a submitted bulk with the given strategy (gputx_strategy).  `opts`
 * may be NULL.  Bulks execute in the order they are passed to this call, so
 * the database after several bulks equals serial execution of them in call
 * order.  ESTATE if the bulk already executed. */
gputx_status gputx_execute(gputx_db *db, gputx_bulk *bulk, int strategy,
                           const gputx_exec_opts *opts);

/* Waits for the bulk and returns its device-side status (OK, EINVAL,
 * ETIMEOUT, EBOUNDS, ECAPACITY); fills *stats when non-NULL. */
gputx_status gputx_sync_bulk(gputx_bulk *bulk, gputx_exec_stats *stats);

/* Copies per-transaction results to host memory after synchronising:
 * status[n] int32 (0 = committed, 1 = not found / aborted in the read phase,
 * 2 = duplicate key on insert) and values[n x n_values] int64 (the
 * procedure's outputs, zero-filled).  Either pointer may be NULL.  EINVAL if
 * n differs from the bulk size or n_values is not the database's output
 * width (gputx_output_width). */
gputx_status gputx_read_results(gputx_bulk *bulk, int32_t *status, int64_t *values, size_t n,
                                int n_values);

/* After a sync: order[k] = the index (0..n-1) of the transaction at position
 * k of a serial order whose execution gives exactly this bulk's results.  For
 * the timestamp-order strategies that is 0, 1, ..., n-1 (Definition 1); for
 * the relaxed strategies it is the order they executed in.  EINVAL if n
 * differs from the bulk size or the bulk has not been executed. */
gputx_status gputx_bulk_order(gputx_bulk *bulk, uint32_t *order, size_t n);

/* Device pointers of the result arrays (status int32[n], values int64[n x
 * width]) for callers that keep results on the device. */
gputx_status gputx_bulk_results_device(gputx_bulk *bulk, const int32_t **status,
                                       const int64_t **values);

/* Number of int64 outputs per transaction: 1 for debit-credit, 8 when the
 * subscriber schema exists, 4 for order-entry (the maximum over schemas). */
int gputx_output_width(const gputx_db *db);

void gputx_free_bulk(gputx_bulk *bulk);

/* Library version string. */
const char *gputx_version(void);

/* Number of CUDA kernels this library has launched since it was loaded, all
 * databases together (for tracing and launch accounting). */
unsigned long long gputx_launch_count(void);

/* Allocation-free K-SET execution of one bulk.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory,
 * such as a process whose device memory is all reserved up front by another
 * allocator (a serving stack or a host framework that must account for every
 * byte), or a latency-critical path where a cudaMalloc could block on a
 * device-wide synchronisation or fail under memory pressure.
 *
 * ts[n], type[n], params[n x params_per_txn] are DEVICE arrays; status[n]
 * (int32) and values[n x gputx_output_width(db)] (int64) are DEVICE arrays
 * the caller owns and the call fills.  The bulk runs with K-SET (one
 * persistent launch per level run) under conflict_mode on the database's
 * stream, and the call returns after it finished.  Results and the database
 * are the same as gputx_submit_bulk + gputx_execute(GPUTX_KSET) +
 * gputx_read_results would produce.
 *
 * Working memory comes from one file-scope device array of
 * GPUTX_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds
 * until the process exits; the call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  A bulk whose working set does
 * not fit returns EINVAL before any work is enqueued (for debit-credit
 * about 300,000 transactions fit; multi-item order-entry bulks fewer).
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture.  Every
 * call shares the one array and each clears what must start at zero, so
 * calls that overlap on the GPU (two databases on different streams, or two
 * host threads) race: serialise them.
 * Errors: EINVAL (null pointer, bad width, unregistered type found on the
 * device, bulk too large), ETIMEOUT/ECAPACITY/EBOUNDS as for gputx_sync_bulk,
 * ECUDA when the device address cannot be obtained. */
#define GPUTX_NOALLOC_SCRATCH_BYTES (48u << 20)
gputx_status gputx_execute_kset_noalloc(gputx_db *db, const int64_t *ts, const int32_t *type,
                                        const int64_t *params, int params_per_txn, size_t n,
                                        int conflict_mode, int32_t *status, int64_t *values);

/* ------------------------------------------------------------------------ */
/* Batched execution through captured CUDA graphs, with an online autotuner   */
/* ------------------------------------------------------------------------ */
/* A stream of transactions (uneven sizes, mixed types) runs as consecutive
 * bulks of one size.  For each (bulk size, strategy, block shape) a
 * fixed-capacity bulk's whole pipeline -- extraction, grouping sort, ranks,
 * the exact-depth pass on the device, regrouping and one persistent K-SET launch
 * (or the TPL kernel) -- is captured once in a CUDA graph and replayed for
 * every bulk of that shape, shorter bulks padded with inactive transactions.
 * With tune = 1 the stream's own first bulks run under different
 * configurations, seeded by Algorithm 1 (Appendix D) on the first bulk's
 * depth, 0-set and cross-partition count, and the fastest per transaction is
 * kept.  Every transaction executes exactly once, in timestamp order, so
 * tuning never changes results.  History rows are consumed per live
 * transaction. */
typedef struct gputx_batcher gputx_batcher;

typedef struct {
    int32_t tune;             /* 1 = choose strategy, bulk size, block shape */
    int32_t strategy;         /* GPUTX_KSET, GPUTX_TPL or GPUTX_PART when not tuning */
    int32_t block_threads;    /* when not tuning (default 256) */
    int32_t conflict_mode;    /* gputx_conflict_mode */
    int64_t bulk_size;        /* segment capacity when not tuning (default 2^16) */
    int64_t bulk_size_max;    /* largest segment capacity the tuner may pick (default: db max_bulk) */
    int32_t params_per_txn;   /* parameter row width (default 2) */
    int32_t reserved;
} gputx_batch_config;

typedef struct {
    int32_t tuned;            /* 1 once the tuner settled */
    int32_t strategy, block_threads, n_measured;
    int64_t bulk_size;        /* segment capacity (transactions per graph replay) */
    int64_t bulks_run;        /* segments run (graph replays) */
    int32_t measured_strategy[16], measured_block[16];
    int64_t measured_bulk[16];
    double measured_ns_per_txn[16];
    double p50_us, p99_us;    /* last run call: per-transaction time from the call's start to its
                                 segment's results on the host */
} gputx_batch_choice;

/* ESTATE without registered types. */
gputx_status gputx_batcher_create(gputx_db *db, const gputx_batch_config *cfg, gputx_batcher **out);

/* Executes a stream of n_bulks bulks of uneven sizes: bulk k is transactions
 * [bulk_off[k], bulk_off[k+1]) of the host arrays ts, type, params (ts
 * strictly increasing over the whole stream; bulk_off[0] = 0, offsets
 * non-decreasing, n = bulk_off[n_bulks]).  Results go to the host arrays
 * status[n], values[n x output width]; returns after the last segment
 * finished.  Consecutive bulks share a segment (one graph replay) up to the
 * segment capacity the tuner chose (or cfg.bulk_size) and at most 63 bulks;
 * a bulk above the capacity is cut into pieces, each its own bulk.  Under
 * K-SET each bulk (piece) keeps its own dependency graph and k-sets
 * (Definition 1 per bulk, bulks in order); TPL and PART run a segment in
 * timestamp order.  EINVAL on bad offsets; device errors as for
 * gputx_sync_bulk. */
gputx_status gputx_batcher_run_bulks(gputx_batcher *bt, const int64_t *ts, const int32_t *type,
                                     const int64_t *params, const int64_t *bulk_off, size_t n_bulks,
                                     int32_t *status, int64_t *values);

/* gputx_batcher_run_bulks over one bulk of n transactions (cut into
 * segments of the chosen capacity). */
gputx_status gputx_batcher_run(gputx_batcher *bt, const int64_t *ts, const int32_t *type, const int64_t *params,
                               size_t n, int32_t *status, int64_t *values);

/* The configuration in use and the tuner's measurements. */
gputx_status gputx_batcher_choice(const gputx_batcher *bt, gputx_batch_choice *out);

void gputx_batcher_destroy(gputx_batcher *bt);

/* ------------------------------------------------------------------------ */
/* Serving: a transaction pool and bulk generator over one database          */
/* ------------------------------------------------------------------------ */
/* Section 3.2: submitted transactions wait in a pool; the system periodically
 * generates a bulk from it and returns the results.  Here a worker thread
 * closes a bulk when its oldest transaction has waited deadline_us or max_bulk
 * transactions are pending, and keeps up to max_inflight bulks on the GPU:
 * the analysis of a new bulk overlaps the execution of earlier ones, and bulks
 * apply in id order.  Every submitted transaction gets the next id, which is
 * its timestamp, so the served stream equals serial execution in id order.
 * While a server runs, only the server may submit or execute bulks on its
 * database. */
typedef struct gputx_server gputx_server;

typedef struct {
    int64_t deadline_us;      /* bulk closes when its oldest transaction waited
                                 this long (default 1000) */
    int64_t max_bulk;         /* ... or holds this many (default: db max_bulk) */
    int32_t max_inflight;     /* bulks on the device at once, 1..8 (default 2);
                                 1 = one bulk at a time, no overlap */
    int32_t strategy;         /* gputx_strategy of every bulk (default K-SET) */
    int32_t conflict_mode;    /* gputx_conflict_mode */
    int32_t params_per_txn;   /* parameter row width of submissions (default 2) */
    int64_t queue_capacity;   /* pending + in-flight transactions admitted
                                 (default 2^30) */
    int64_t min_free_bytes;   /* refuse submissions while free device memory is
                                 below this (0 = no check) */
    int32_t zero_set;         /* 1: incremental 0-set execution (Section 5.3):
                                 arrivals join a device-resident pool
                                 (gputx_pool, capacity 2 x max_bulk) and
                                 every step executes the pool's 0-set, so a
                                 long dependency chain never holds back the
                                 transactions that do not depend on it;
                                 strategy and max_inflight are unused */
    int32_t reserved;         /* zero */
} gputx_serve_config;

typedef struct {
    int64_t submitted, completed, bulks, max_bulk_seen, refused;
    double p50_us, p99_us, mean_us;   /* arrival -> result available on the host */
    double txn_per_s;                 /* completed / (last completion - first arrival) */
} gputx_serve_stats;

/* Monotonic clock (ns) that arrival times passed to gputx_server_submit use. */
int64_t gputx_clock_ns(void);

/* Starts a server on a database with registered types.  ESTATE if none are
 * registered, EINVAL on a bad strategy, ENOMEM if its pinned staging buffers
 * cannot be allocated. */
gputx_status gputx_server_create(gputx_db *db, const gputx_serve_config *cfg, gputx_server **out);

/* Adds n transactions (host arrays: type[n], params[n x params_per_txn]) to
 * the pool; arrival_ns[n] (gputx_clock_ns timebase) or NULL for now.  *first_id
 * receives the id (timestamp) of the first; the rest follow consecutively.
 * Admission: ENOMEM, with nothing added, when the pool would exceed
 * queue_capacity, an insert area (history, call forwarding, orders, order
 * lines) could not hold the inserts already admitted plus these, or free
 * device memory is below min_free_bytes.  A device error of an earlier bulk
 * is returned here too. */
gputx_status gputx_server_submit(gputx_server *s, const int32_t *type, const int64_t *params, size_t n,
                                 const int64_t *arrival_ns, int64_t *first_id);

/* Copies the results of ids [first_id, first_id + n) that have completed
 * into status[n] / values[n x output width] / complete_ns[n] (any may be
 * NULL); entries of unfinished ids are left as they are.  *n_done counts the
 * finished ones.  EINVAL for ids never submitted. */
gputx_status gputx_server_results(gputx_server *s, int64_t first_id, size_t n, int32_t *status, int64_t *values,
                                  int64_t *complete_ns, size_t *n_done);

/* Waits until every submitted transaction completed (closing the last bulk
 * without waiting for its deadline); returns the first device error. */
gputx_status gputx_server_drain(gputx_server *s);

gputx_status gputx_server_stats(gputx_server *s, gputx_serve_stats *stats);
const char *gputx_server_last_error(const gputx_server *s);

/* Stops the worker after the pending transactions complete, frees buffers. */
void gputx_server_destroy(gputx_server *s);

/* Latency floor of a chain of levels on one thread-block cluster: the
 * skeleton of the K-SET narrow-level runner (Section 5.3) with no transaction
 * logic.  At each of `levels` levels, each of cluster_size x threads threads
 * loads `loads` (0..8) values that the previous level wrote on another CTA,
 * updates `stores` (>= 1) values, arrives at the cluster barrier (release),
 * stores `stores_after` (>= 0) more values, and waits (acquire);
 * stores + stores_after <= 16.  rmw = 0: the updates are plain stores;
 * rmw = 1: they are 64-bit atomic additions to cells that the previous level
 * updated on another CTA, one a fetch-and-add whose old value feeds the
 * stores after the arrival and the rest reductions (the shape of a runner
 * applying its balance updates at L2); rmw = 2: as 1, but the fetch-and-add
 * goes to a cell drawn uniformly from a table of 10,000,000 8-byte cells (the
 * debit-credit accounts' footprint) and the cell of two levels ahead is
 * prefetched into L2 before the barrier, as the debit-credit runner does.
 * *ns_per_level = the time of one timed launch (after a warm-up launch)
 * divided by `levels`.  Allocates and frees its own device memory
 * ((levels + 17) x cluster_size x threads x 128 bytes, and 80 MB for rmw = 2).
 * EINVAL on a parameter out of range (rmw other than 0, 1 or 2 included),
 * ECUDA if the cluster shape cannot launch. */
gputx_status gputx_probe_level_chain(int levels, int cluster_size, int threads, int loads, int stores,
                                     int stores_after, int rmw, double *ns_per_level);

/* Throughput of 64-bit atomic additions performed at L2, the operation TPL's
 * counters, the ADD class's blind increments (Section 5.1's workload under
 * the blind-increment refinement) and the debit-credit level runners rely on.
 * A grid of (SMs x 8) CTAs of 256 threads each adds 1 to 64 cells drawn
 * uniformly from a table of n_cells (1 .. 2^32) 8-byte cells: reductions
 * (fetch = 0) or fetch-and-adds whose results are used (fetch = 1).  The
 * table is zeroed and touched by one warm-up launch, so a table that fits in
 * L2 is L2-resident.  *gops = atomic operations per nanosecond (G/s) of one
 * timed launch.  Allocates and frees n_cells x 8 bytes.  EINVAL on a
 * parameter out of range, ENOMEM, ECUDA. */
gputx_status gputx_probe_atomics(int64_t n_cells, int fetch, double *gops);

/* ---------------------------------------------------------------------------
 * Incremental 0-set execution (Section 5.3).  A device-resident pool of
 * pending transactions keeps their basic operations sorted by item.  New
 * transactions' operations are sorted and merged into that array.  Each step
 * executes the pool's 0-set as one bulk and removes it, so the former 1-set
 * becomes the next 0-set.  The 0-set holds the sources of the T-dependency
 * graph (Section 4.1): transactions with no earlier conflicting pending
 * operation, so each commutes with every earlier transaction still pending.  The results of all steps therefore
 * equal serial execution of the whole stream in timestamp order
 * (Definition 1).  A step always executes the oldest pending transaction, so
 * a pool with pending work always makes progress.
 * ------------------------------------------------------------------------- */
typedef struct gputx_pool gputx_pool;

typedef struct {
    int64_t capacity;       /* ring slots: the timestamp span pending at once
                               (oldest pending to newest added), >= 1 */
    int32_t params_per_txn; /* P of every added transaction */
    int32_t conflict_mode;  /* gputx_conflict_mode of the 0-set */
    int64_t reserved[2];    /* zero */
} gputx_pool_config;

/* The pool's device memory is about capacity x (56 + 8 P + 40 K) bytes, where
 * K is the largest number of basic operations of a registered type. */
gputx_status gputx_pool_create(gputx_db *db, const gputx_pool_config *cfg, gputx_pool **out);

/* Appends n transactions from host arrays (ts[n], type[n], params[n x P]);
 * timestamps continue the stream strictly increasing.  Returns ECAPACITY when
 * the pending span would exceed the capacity and EINVAL for an invalid
 * signature or timestamp.  In both cases nothing is added. */
gputx_status gputx_pool_add(gputx_pool *p, const int64_t *ts, const int32_t *type, const int64_t *params,
                            size_t n);

/* Executes the pool's current 0-set; *executed = its size (0 only when the
 * pool is empty).  Synchronous: the results are ready on return. */
gputx_status gputx_pool_step(gputx_pool *p, size_t *executed);

/* The last step's transactions in timestamp order: ts[k], status[k],
 * values[k x R] (R = gputx_output_width).  *n = how many; capacity too small
 * -> EINVAL. */
gputx_status gputx_pool_results(const gputx_pool *p, int64_t *ts, int32_t *status, int64_t *values,
                                size_t capacity, size_t *n);

/* Transactions added and not yet executed. */
size_t gputx_pool_pending(const gputx_pool *p);

void gputx_pool_destroy(gputx_pool *p);

#ifdef __cplusplus
}
#endif
#endif /* GPUTX_H */
