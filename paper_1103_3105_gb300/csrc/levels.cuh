// levels.cuh -- the arguments of the K-SET level runners (Section 5.3) and
// the launcher of the debit-credit narrow-level runner, which lives in its
// own translation unit (exec_dc.cu).
#pragma once
#include "engine.h"

namespace gtx {

struct LevelArgs {
    DevDB db;
    DevBulk b;
    const BulkCtl *ctl;
    const uint32_t *level_off;
    const DcRecord *rec_dc;   // debit-credit-only bulks: packed records in execution order
    const uint32_t *type_cut; // per level, where new-order, payment, order-status start (or null)
    uint32_t k0, k1;          // levels [k0, k1)
    bool atomic_add;
};

// the run of narrow levels [a.k0, a.k1) from debit-credit records, on one
// cluster of csize CTAs (one plain CTA when csize <= 1) of `threads` threads
cudaError_t launch_narrow_dc(const LevelArgs &a, int csize, int threads, cudaStream_t s);

}  // namespace gtx
