// cta_groups.cuh -- lock groups over a whole CTA, shared by the debit-credit
// TPL executors (ordered counters in exec.cu, relaxed spin locks in
// relaxed.cu).
//
// A CTA holds a chunk of up to 256 consecutive transactions of the bulk.
// Those that need the same lock form one group: a shared-memory hash table
// maps the lock's key to a slot with a 256-bit member mask.  The group's first
// member (lowest thread) deals with the lock for all of them; the members
// run, in thread order, inside that one critical section.  Members on the
// same account combine their deltas: the account's first member performs one
// fetch-and-add of their sum and publishes the old value, and each member's
// new balance is that old value plus the inclusive prefix of the deltas in
// thread order -- the serial result bit for bit.  Every wait in shared memory
// is bounded.
#pragma once
#include "common.cuh"

namespace gtx {

constexpr int kCtaTab = 512;                 // hash slots (2 x the largest chunk)
constexpr int kCtaMax = 256;                 // threads of a CTA that groups
constexpr uint32_t kCtaEmpty = 0xffffffffu;  // a free slot's key

struct CtaGroupTables {
    uint32_t key[kCtaTab];
    uint32_t state[kCtaTab];   // 0 waiting, 1 granted, 2 failed (set by the group's first member)
    uint32_t fin[kCtaTab];     // members done with their account update
    uint32_t base[kCtaTab];    // relaxed TPL: the group's first commit ticket
    uint32_t mask[kCtaTab][8];
    int64_t delta[kCtaMax];    // each member's delta (0 if it does not run)
    int64_t old[kCtaMax];      // an account's balance before its first member's addition
    uint32_t acct[kCtaMax];
    uint32_t aflag[kCtaMax];   // old[] is valid
};

// spin on a shared-memory flag until it is non-zero, at most limit_ns
__device__ __forceinline__ bool wait_smem(volatile uint32_t *f, uint64_t limit_ns)
{
    if (*f) return true;
    const uint64_t t0 = globaltimer();
    uint32_t spins = 0;
    while (!*f) {
        if (++spins > 32) __nanosleep(64);
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return true;
}

// empty every slot (the whole CTA, at the start of each chunk; a barrier
// must follow before any join)
__device__ __forceinline__ void cta_groups_reset(CtaGroupTables &g, uint32_t tid, uint32_t nt)
{
    for (uint32_t i = tid; i < (uint32_t)kCtaTab; i += nt) {
        g.key[i] = kCtaEmpty;
        g.state[i] = 0;
        g.fin[i] = 0;
#pragma unroll
        for (int w = 0; w < 8; w++) g.mask[i][w] = 0;
    }
}

// thread tid joins the group of `key` (linear probing); returns its slot
__device__ __forceinline__ uint32_t cta_group_join(CtaGroupTables &g, uint32_t key, uint32_t tid)
{
    uint32_t e = (key * 2654435761u) & (kCtaTab - 1);
    while (true) {
        const uint32_t prev = atomicCAS(&g.key[e], kCtaEmpty, key);
        if (prev == kCtaEmpty || prev == key) break;
        e = (e + 1) & (kCtaTab - 1);
    }
    atomicOr(&g.mask[e][tid >> 5], 1u << (tid & 31));
    return e;
}

// a member's view of its group, read after the barrier that ends the joins
struct CtaMember {
    uint32_t m[8];             // the member mask
    uint32_t leader, size, rank;   // first member, members, members before this one
    uint32_t afirst;           // first member on this member's account
    int64_t pre, tot;          // inclusive prefix and sum of the deltas on the account
};

__device__ __forceinline__ void cta_member(const CtaGroupTables &g, uint32_t e, uint32_t tid, uint32_t acct,
                                           CtaMember &c)
{
    bool found = false;
    c.leader = 0;
    c.size = 0;
    c.rank = 0;
#pragma unroll
    for (int w = 0; w < 8; w++) {
        c.m[w] = g.mask[e][w];
        if (!found && c.m[w]) {
            c.leader = 32u * w + (uint32_t)(__ffs(c.m[w]) - 1);
            found = true;
        }
        c.size += __popc(c.m[w]);
        const uint32_t tw = tid >> 5;
        if ((uint32_t)w < tw) c.rank += __popc(c.m[w]);
        else if ((uint32_t)w == tw) c.rank += __popc(c.m[w] & ((1u << (tid & 31)) - 1u));
    }
    c.afirst = tid;
    if (c.size == 1) {             // alone on its lock, so alone on its account
        c.pre = c.tot = g.delta[tid];
        return;
    }
    c.pre = 0;
    c.tot = 0;
    for (int w = 0; w < 8; w++) {
        for (uint32_t bits = c.m[w]; bits; bits &= bits - 1) {
            const uint32_t j = 32u * w + (uint32_t)(__ffs(bits) - 1);
            if (g.acct[j] != acct) continue;
            const int64_t d = g.delta[j];
            c.tot = wrap_add(c.tot, d);
            if (j <= tid) c.pre = wrap_add(c.pre, d);
            if (j < c.afirst) c.afirst = j;
        }
    }
}

// The account update of a member that runs: its account's first member adds
// the sum and publishes the old value, the others read it.  False (and
// ERR_TIMEOUT) if the old value never came within the limit.
__device__ __forceinline__ bool cta_account_update(CtaGroupTables &g, const CtaMember &c, uint32_t tid,
                                                   int64_t *cell, uint64_t limit_ns, uint32_t *err, int64_t &old)
{
    if (c.afirst == tid) {
        old = (int64_t)atomicAdd((unsigned long long *)cell, (unsigned long long)c.tot);
        g.old[tid] = old;
        __threadfence_block();
        *(volatile uint32_t *)&g.aflag[tid] = 1u;
        return true;
    }
    if (wait_smem(&g.aflag[c.afirst], limit_ns)) {
        old = *(volatile int64_t *)&g.old[c.afirst];
        return true;
    }
    set_err(err, ERR_TIMEOUT);
    return false;
}

// the group's first member waits until all `size` members counted themselves
// done (bounded); false if the limit ran out
__device__ __forceinline__ bool cta_wait_members(const CtaGroupTables &g, uint32_t e, uint32_t size,
                                                 uint64_t limit_ns)
{
    volatile const uint32_t *fin = &g.fin[e];
    const uint64_t t0 = globaltimer();
    while (*fin < size) {
        __nanosleep(32);
        if (globaltimer() - t0 > limit_ns) return false;
    }
    return true;
}

}  // namespace gtx
