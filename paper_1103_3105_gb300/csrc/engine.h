// engine.h -- host-side state of a database and a bulk, and the launchers each
// translation unit provides.  Internal to the library.
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace gtx {

// Per-bulk control block in device memory (zeroed at submit).
struct BulkCtl {
    uint32_t err;          // ERR_* bits
    uint32_t depth;        // d: largest level
    uint32_t w0;           // 0-set size
    uint32_t cross;        // cross-partition transactions
    uint32_t npart;        // PART: non-empty partitions
    uint32_t claim;        // executors: next chunk to claim
    uint32_t n_live;       // fixed-capacity bulks: live transactions (the rest pad)
    InsertBase base;       // where this bulk's inserts start (copied from the cursor)
    InsertBase total;      // inserts this bulk reserves
    uint32_t rounds;       // exact-depth passes run (the dataflow pass: 1)
    uint32_t n_seg;        // segmented graph bulks: bulks in this segment (0 = one)
    uint32_t hot;          // TPL: some counter has a chain of at least the hot ticket
    uint32_t chunk;        // relaxed TPL: next chunk to claim (claim counts commit tickets)
};

constexpr int kSegMax = 64;        // bulks in one segment of a graph bulk, at most

// Scratch carved from one per-bulk allocation.
struct Scratch {
    uint32_t *keys_a, *vals_a, *keys_b, *vals_b;  // sort ping-pong, m entries each
    uint32_t *op_off;      // n+1 exclusive op offsets (non-uniform op counts)
    uint32_t *level;       // n
    uint32_t *rid;         // m: global run id per sorted op (exact depth)
    uint32_t *runmax;      // m: deepest finished transaction of each run (exact depth)
    uint32_t *lock_key;    // m: TPL per-op object, indexed by op slot
    uint32_t *lock_ticket; // m
    uint32_t *level_off;   // n+2
    uint32_t *type_cut;    // 3 (n+2): per level, where types >= new-order, payment, order-status start
    uint32_t *chunk_off;   // n+2
    uint32_t *chunk_level; // n + n/min_block + 2
    uint32_t *done;        // n+1 per-level completion counters
    uint32_t *part_start;  // n
    uint32_t *pid_key, *pid_val, *pid_key2, *pid_val2;  // PART sort, n each
    int64_t *rec_params, *rec_ts;  // signatures gathered into execution order
    int32_t *rec_type;
    uint32_t *rec_t;
    uint32_t *slot_cf, *slot_ord, *slot_ol;   // n each
    uint32_t *slot_hist;   // n: history rows of debit-credit transactions in mixed databases
    uint32_t *sort_hist;   // 4 x 256
    uint32_t *sort_offs;   // 4 x 256
    uint32_t *sort_status; // 4 x tiles x 256
    uint32_t *tile_ctr;    // 16 counters
    uint64_t *scan_status; // tiles
    uint64_t *scan_vals;   // 2 x tiles: per-tile values of 64-bit scans
    DcRecord *rec_dc;      // n packed debit-credit records (debit-credit-only databases)
    // graph bulks that carry a segment of several bulks
    uint32_t *seg_off;     // kSegMax + 1: first transaction of each bulk
    uint32_t *bulk_of;     // n: bulk of each transaction
    uint32_t *seg_depth;   // kSegMax: largest level of each bulk
    uint32_t *seg_base;    // kSegMax + 1: first global level of each bulk
    int64_t m_cap;         // op capacity
    int64_t sort_tiles, scan_tiles, chunk_cap;
};

}  // namespace gtx

struct gputx_db {
    gtx::DevDB dev{};
    gputx_schema_desc schema{};
    gputx_config cfg{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    int num_sms = 0;
    std::string last_error;
    std::vector<void *> allocs;
    gtx::InsertBase *d_cursor = nullptr;   // device insert cursors
    uint32_t *d_done = nullptr;            // TPL per-object counters, kept zero between bulks
    gtx::LockSlots lock_slots{};           // item -> slot of d_done (32 x lines words)
    int kmax = 0;                          // largest op count of a registered type
    int uniform_k = 0;                     // every registered type has exactly this many ops (0 = no)
    bool need_fixpoint = false;            // a registered type's ops may leave one-pass ranks inexact
    int tbits = 0;                         // type bits in the level/type regroup key
    bool group_oe = false;                 // K-SET runs new-order and order-status on 16-lane groups
    bool hist_by_type = false;             // debit-credit and other types: history rows for debit-credit only
    int obj_bits = 1;                      // key bits of object ids
    // Each bulk runs on a stream of this pool, so the analysis of one bulk
    // overlaps the execution of the one before; `last_done` orders the
    // database-touching tail of every bulk after that of its predecessor.
    static constexpr int kPool = 4;
    cudaStream_t pool[kPool] = {};
    int next_pool = 0;
    cudaEvent_t last_done = nullptr;
    // relaxed PART: per-partition counters and their prefix-scan scratch,
    // allocated at first use (used only inside a bulk's ordered tail)
    uint32_t *part_cnt = nullptr;          // part_cnt_n counters, zero between bulks
    uint32_t *part_off = nullptr;          // part_cnt_n + 1 offsets
    int64_t part_cnt_n = 0;
    uint64_t *part_scan_status = nullptr;
    uint32_t *part_tile_ctr = nullptr;
};

struct gputx_bulk {
    gputx_db *db = nullptr;
    cudaStream_t stream = nullptr;          // this bulk's stream (from the database's pool)
    cudaEvent_t ev_in = nullptr;            // inputs ready on the database stream
    int64_t n = 0;
    int P = 0, R = 0;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    int64_t *ts = nullptr;
    int32_t *type = nullptr;
    int64_t *params = nullptr;
    int32_t *status = nullptr;
    int64_t *out = nullptr;
    gtx::BulkCtl *ctl = nullptr;
    gtx::Scratch sc{};
    bool executed = false;
    bool synced = false;
    const uint32_t *serial_order = nullptr;   // relaxed strategies: the serial order executed
    bool graph = false;    // fixed capacity, padded with inactive transactions,
                           // no host synchronisation (capturable in a CUDA graph)
    int strategy_run = -1;
    int fallback = 0;
    int64_t fixpoint_rounds = 0;
    bool timing = false;
    cudaEvent_t ev[8] = {};
    gtx::BulkCtl host_ctl{};
    std::vector<uint32_t> level_off_host;   // K-SET level boundaries read back for launch planning
    std::vector<uint32_t> type_cut_host;    // and where each order-entry type starts in each level
};

namespace gtx {

// analysis.cu
DevBulk make_dev_bulk(gputx_bulk *b, int mode);
cudaError_t launch_extract(gputx_bulk *b, int mode, int part_size, uint32_t *pid_key, uint32_t *pid_val,
                           bool write_ops, bool segmented = false);
// segmented graph bulks: bulk of each transaction; per-bulk depths and the
// global level numbering (bulk by bulk, levels in order)
int seg_bits(const gputx_db *db);
cudaError_t launch_seg_index(gputx_bulk *b);
cudaError_t launch_seg_levels(gputx_bulk *b);
// PART in a graph: flags a segment with cross-partition transactions (it
// then runs nothing and is re-run with TPL)
cudaError_t launch_part_fallback_check(gputx_bulk *b);
cudaError_t launch_sort(gputx_bulk *b, uint32_t *&keys, uint32_t *&vals, uint32_t *&keys_alt,
                        uint32_t *&vals_alt, int64_t count, int bits);
cudaError_t launch_rank_scan(gputx_bulk *b, const uint32_t *sk, const uint32_t *sv, int64_t m, bool want_rid);
cudaError_t launch_ticket_scan(gputx_bulk *b, const uint32_t *sk, const uint32_t *sv, int64_t m);
cudaError_t launch_depth_flow(gputx_bulk *b, const uint32_t *sv, int64_t m);
cudaError_t launch_exact_depth(gputx_bulk *b, const uint32_t *sv, int64_t m);
cudaError_t launch_level_stats(gputx_bulk *b);
cudaError_t launch_regroup_keys(gputx_bulk *b, uint32_t *keys, uint32_t *vals);
cudaError_t launch_level_tables(gputx_bulk *b, const uint32_t *skeys, int64_t depth, int block, bool chunks);
cudaError_t launch_insert_slots(gputx_bulk *b);
cudaError_t launch_part_heads(gputx_bulk *b, const uint32_t *skeys, int64_t n);
cudaError_t launch_tpl_reset(gputx_bulk *b, const uint32_t *skeys, int64_t m);
cudaError_t launch_gather(gputx_bulk *b, const uint32_t *order);
cudaError_t launch_gather_dc(gputx_bulk *b, const uint32_t *order);
bool part_dc_applies(const gputx_db *db, int part_size);
cudaError_t launch_begin(gputx_bulk *b);
cudaError_t launch_finish(gputx_bulk *b);

// exec.cu
cudaError_t launch_kset(gputx_bulk *b, const uint32_t *order, int64_t nchunks, int block, bool atomic_add);
cudaError_t launch_kset_levels(gputx_bulk *b, const uint32_t *level_off_host, int64_t depth, int narrow_max,
                               bool atomic_add, const DcRecord *dc_records = nullptr,
                               const uint32_t *type_cut_host = nullptr);
cudaError_t launch_part(gputx_bulk *b, const uint32_t *pkeys, int block, int64_t max_parts, int part_size);
cudaError_t launch_tpl(gputx_bulk *b, int block, bool atomic_add);
// a conflict-free bulk (a 0-set) in one launch
cudaError_t launch_independent(gputx_bulk *b, bool atomic_add);
// relaxed timestamps (Appendix G)
cudaError_t launch_tpl_relaxed(gputx_bulk *b, uint32_t *order, bool atomic_add);
cudaError_t launch_validate(gputx_bulk *b);
cudaError_t launch_part_count(gputx_bulk *b, int mode, int part_size, uint32_t *cnt, int64_t parts,
                              uint32_t *pid_of, uint32_t *key_of);
cudaError_t launch_part_offsets(gputx_bulk *b, const uint32_t *cnt, uint32_t *off, int64_t parts, uint64_t *status,
                                uint32_t *tile_ctr);
cudaError_t launch_part_scatter(gputx_bulk *b, const uint32_t *off, const uint32_t *pid_of, const uint32_t *key_of,
                                uint32_t *pkeys, uint32_t *order);
// SCAN: segmented prefix sums over operations grouped by account
cudaError_t launch_scan_exec(gputx_bulk *b, const uint32_t *sk, const uint32_t *sv, int64_t m);
int exec_blocks_per_sm(int kind, int block);

// tables.cu
cudaError_t launch_fill_i64(int64_t *p, int64_t n, int64_t v, cudaStream_t s);
cudaError_t launch_fill_u64(unsigned long long *p, int64_t n, unsigned long long v, cudaStream_t s);

// kernels launched by this library since load (tracing)
void count_launches(int k);

inline int bits_for(uint64_t maxval)
{
    int b = 0;
    while (b < 32 && (maxval >> b) != 0) b++;
    return b;
}

}  // namespace gtx
