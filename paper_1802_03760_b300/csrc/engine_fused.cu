// Fused engine: one persistent launch evaluates one or many queries.
//
// Each warp runs the BiGJoin schedule on its own bounded buffers (Section
// 3.2 with the batching rule of Section 3.1.2, B' = 32 proposals per step):
// level j holds at most 2B' = 64 prefixes of length j in shared memory (the
// invariant of Appendix B). When a level has at least B' prefixes, or its
// parent has no proposals left, the warp extends it: Count gives each
// prefix its smallest binding list (min-c, min-i), a warp scan lays their
// candidates on one line, and every step proposes the next 32 candidates
// (one per lane, several prefixes per step when lists are short), tests
// each against the other binding lists (hash sets for long lists, binary
// search for short ones), and ballots the survivors into the next level
// (or counts and hashes them at the last level, two candidates per lane
// while one prefix's list lasts). The warp always works on the deepest
// level with pending work, so memory stays O(k * B') per warp.
//
// Balance (Section 3.4 at warp granularity): warps take seed chunks (32
// seed edges by default) from one counter shared by every query of the
// launch; a warp that fills a level while others are idle hands the batch
// to a ring of bundles, and a warp with a long remaining candidate range
// hands over its upper half.
#include "gj_internal.cuh"

namespace {

constexpr int FC = 64;          // frontier capacity per level per warp (2 B')
constexpr int FT = 32;          // B': descend once a level holds this many prefixes
constexpr int FW = 8;           // warps per block
constexpr int SEED_CHUNK = 32;  // default seeds per grab (a multiple of 8; tunable per launch)
constexpr uint32_t DELTA_CHUNK = 8;  // most seeds per grab in delta launches

// A batch of up to FC prefixes of one plan and level that a busy warp hands
// to idle warps (the balance step of Section 3.4 at warp granularity).
struct Bundle {
    uint32_t plan, level, n, pad;
    unsigned long long c_lo, c_hi;  // candidate range of the batch to extend (all: 0, ~0)
    uint32_t tup[GJ_MAX_K][FC];
    uint64_t hp[FC];  // a factorised last level's hash factors (the count weights are in tup)
    int8_t sg[FC];
};

constexpr uint64_t RANGE_SPLIT_MIN = 4096;  // remaining candidates worth splitting off

// Shared state of the donation queue, a bounded ring of bundles in which
// every slot carries a sequence number (free for ticket t when seq == t,
// holding ticket t's bundle when seq == t + 1). A giver reserves ticket
// tail only if its slot is free and never waits; a taker takes ticket head
// only once it is published and frees the slot for ticket head + cap.
// busy counts the warps that hold work: a warp counts itself from its start
// until it runs out of seeds, and again from just before it claims a bundle
// until it has finished it. A warp without work leaves once busy == 0 and
// head == tail: only busy warps give, so nothing can arrive after that. The
// rule waits only on warps that have started, so the launch needs no
// co-resident grid and can share the GPU with other launches. idle counts
// the waiting warps (a hint for givers).
struct DonationQueue {
    Bundle* b = nullptr;  // null: donation off
    uint32_t cap = 0;     // power of two
    unsigned long long* head = nullptr;
    unsigned long long* tail = nullptr;
    unsigned long long* seq = nullptr;  // [cap]
    unsigned int* idle = nullptr;
    unsigned int* busy = nullptr;
    unsigned long long* err = nullptr;  // set when the bounded wait gives up
    unsigned int always = 0;  // 1: give whenever a slot is free (stress setting)
};

struct FusedArgs {
    GraphView G;
    const Plan* plans;
    uint32_t nq;
    uint32_t kmax;
    const uint64_t* qbase;      // [nq + 1] start of each query's seed space (multiples of chunk)
    const int64_t* seed_lo;     // [nq] first seed slot of each query's seed index
    const int64_t* seed_n;      // [nq] number of seeds
    unsigned long long* next;   // work counter over the concatenated seed spaces
    unsigned long long* counts; // [nq]
    unsigned long long* chks;   // [nq]
    unsigned long long* stats;  // [5 * 9] extended, nbind, proposals, produced, seeds; may be null
    unsigned long long* ovf;    // set when a static count passes 2^63 - 1 (may be null)
    DeltaView D;                // delta plans: the batch's per-direction insert/delete arrays
    DeltaBatch B;               // delta plans: the batch's signed changes (the seeds)
    uint32_t chunk = SEED_CHUNK;  // seeds a warp takes per grab (multiple of 8)
    DonationQueue Q;
    uint64_t wait_ns = 0;       // bound of the end-of-launch wait without progress
};

// Counter block of a launch after the per-query counts and checksums: the
// shared work counter, the work units (5 x 9) and the overflow flag.
constexpr size_t NSTAT = 5 * 9 + 1;

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Shared-memory layout of one warp (identical on host and device): the
// plan, 4 x 8 scalars (n, cursor, total, cursor's prefix per level), then
// per level j >= 2 the prefix tuples [j][FC] (column-major), the min-list
// pointers [FC], the candidate offsets [FC + 1] and the min-i bytes [FC]
// (delta plans add the new-version parts of each min list and the seed's
// sign), then one block that only the query's last level uses: the hash
// factor of each prefix [FC] and, in EXT launches, the other binding list
// of a two-binding last level [FC] (pointer, hash set, length) and the size
// of each aggregated group [FC]. A warp finishes a last-level batch before
// it activates another one, so one block serves every query. Offsets are
// closed forms so that no per-level table sits in local memory. The
// footprint is kept small on purpose: the CUDA driver gives an SM's L1 /
// shared memory the smallest shared-memory size that holds the resident
// blocks, and the rest is L1 for the probed lists and hash sets (four
// extended k = 4 blocks fit 196 KB, leaving about 60 KB of L1).
constexpr uint32_t ALIGN16(uint32_t b) { return (b + 15u) & ~15u; }
constexpr uint32_t PLAN_BYTES = ALIGN16(sizeof(Plan));
constexpr uint32_t SCAL_BYTES = 4 * GJ_MAX_K * 8;
constexpr uint32_t LVL_FIXED = FC * 8 + ALIGN16((FC + 1) * 8) + ALIGN16(FC);  // mptr + cs + minb
// Delta plans also keep, per prefix, the new-version parts of the min list
// (where its inserts and deletes start in the batch's arrays of the min
// binding's direction, committed length, number of deletes) and the seed's
// sign.
constexpr uint32_t LVL_DELTA = FC * 4 + FC * 4 + FC * 4 + FC * 4 + FC;  // ins, del, base len, ndel, sign
__host__ __device__ __forceinline__ uint32_t lvl_size_fixed(bool d) { return LVL_FIXED + (d ? ALIGN16(LVL_DELTA) : 0); }
__host__ __device__ __forceinline__ uint32_t lvl_base(uint32_t j, bool d) {
    // sum over i = 2..j-1 of (FC * i * 4 + fixed part)
    return PLAN_BYTES + SCAL_BYTES + (uint32_t)(FC * 4) * ((j * (j - 1)) / 2 - 1) + lvl_size_fixed(d) * (j - 2);
}
__host__ __device__ __forceinline__ uint32_t off_tup(uint32_t j, bool d, bool) { return lvl_base(j, d); }
__host__ __device__ __forceinline__ uint32_t off_mptr(uint32_t j, bool d, bool) { return lvl_base(j, d) + FC * 4 * j; }
__host__ __device__ __forceinline__ uint32_t off_cs(uint32_t j, bool d, bool x) { return off_mptr(j, d, x) + FC * 8; }
__host__ __device__ __forceinline__ uint32_t off_minb(uint32_t j, bool d, bool x) {
    return off_cs(j, d, x) + ALIGN16((FC + 1) * 8);
}
__host__ __device__ __forceinline__ uint32_t off_dins(uint32_t j, bool x) { return off_minb(j, true, x) + ALIGN16(FC); }
__host__ __device__ __forceinline__ uint32_t off_ddel(uint32_t j, bool x) { return off_dins(j, x) + FC * 4; }
__host__ __device__ __forceinline__ uint32_t off_dblen(uint32_t j, bool x) { return off_ddel(j, x) + FC * 4; }

// The batch's insert and delete arrays of one direction (delta plans).
__device__ __forceinline__ const uint32_t* dins_base(const DeltaView& D, uint32_t dir) {
    return dir ? D.rev.ins_nbr : D.fwd.ins_nbr;
}
__device__ __forceinline__ const uint32_t* ddel_base(const DeltaView& D, uint32_t dir) {
    return dir ? D.rev.del_nbr : D.fwd.del_nbr;
}
__host__ __device__ __forceinline__ uint32_t off_dndel(uint32_t j, bool x) { return off_dblen(j, x) + FC * 4; }
__host__ __device__ __forceinline__ uint32_t off_dsg(uint32_t j, bool x) { return off_dndel(j, x) + FC * 4; }
// the last-level block, after the levels of the launch's longest query
__host__ __device__ __forceinline__ uint32_t off_hpre(uint32_t kmax, bool d, bool) { return lvl_base(kmax, d); }
// the kept second list: its hash set when it has one (length >= GJ_HASH_MIN_DEG), else the sorted list
__host__ __device__ __forceinline__ uint32_t off_olp(uint32_t kmax, bool d, bool x) { return off_hpre(kmax, d, x) + FC * 8; }
__host__ __device__ __forceinline__ uint32_t off_oll(uint32_t kmax, bool d, bool x) { return off_olp(kmax, d, x) + FC * 8; }
__host__ __device__ __forceinline__ uint32_t off_grp(uint32_t kmax, bool d, bool x) { return off_oll(kmax, d, x) + FC * 4; }
// Delta plans: the other bindings' views of the prefix that a run of
// single-prefix steps extends (committed list or hash set, and the batch's
// inserts and deletes of its vertex), computed once for the run.
struct DViewCache {
    const uint32_t* cp[2];  // committed list, or its hash set when cbits > 0
    const uint32_t* ins[2];
    const uint32_t* del[2];
    uint32_t cl[2], cbits[2], nins[2], ndel[2];
};
__host__ __device__ __forceinline__ uint32_t off_dvc(uint32_t kmax, bool d, bool x) {
    return off_hpre(kmax, d, x) + FC * 8 + (x ? ALIGN16(FC * 8 + FC * 4 + FC) : 0);
}
__host__ __device__ __forceinline__ uint32_t warp_bytes(uint32_t kmax, bool d, bool x) {
    return kmax <= 2 ? PLAN_BYTES + SCAL_BYTES : off_dvc(kmax, d, x) + (d ? ALIGN16(sizeof(DViewCache)) : 0);
}

__device__ __forceinline__ void stat_add(unsigned long long* s, int which, int j, unsigned long long v) {
    if (s && v) atomicAdd(s + which * 9 + j, v);
}


// Membership of e in the sorted list a[0, len), len < 2^32: branch-free
// binary search over power-of-two steps (1 + floor(log2 len) probes). The
// first probe decides whether the answer lies in the top S = 2^floor(log2
// len) elements; every later probe halves a power-of-two range.
__device__ __forceinline__ bool member32(const uint32_t* __restrict__ a, uint32_t len, uint32_t e) {
    if (len == 0) return false;
    uint32_t step = 1u << (31 - __clz(len));
    uint32_t pos = (__ldg(a + (len - step)) <= e) ? len - step : 0u;
    for (step >>= 1; step; step >>= 1) {
        const uint32_t q = pos + step;
        pos = (__ldg(a + q) <= e) ? q : pos;
    }
    return __ldg(a + pos) == e;
}

// Two membership tests against the same sorted list, interleaved so that
// the two chains of dependent loads overlap (same list: same step count).
__device__ __forceinline__ void member32x2(const uint32_t* __restrict__ a, uint32_t len, uint32_t e0, bool& k0,
                                           uint32_t e1, bool& k1) {
    if (len == 0) {
        k0 = k1 = false;
        return;
    }
    uint32_t step = 1u << (31 - __clz(len));
    const uint32_t x = __ldg(a + (len - step));
    uint32_t p0 = (x <= e0) ? len - step : 0u;
    uint32_t p1 = (x <= e1) ? len - step : 0u;
    for (step >>= 1; step; step >>= 1) {
        const uint32_t q0 = p0 + step, q1 = p1 + step;
        const uint32_t v0 = __ldg(a + q0), v1 = __ldg(a + q1);
        p0 = (v0 <= e0) ? q0 : p0;
        p1 = (v1 <= e1) ? q1 : p1;
    }
    const uint32_t f0 = __ldg(a + p0), f1 = __ldg(a + p1);
    k0 = k0 && f0 == e0;
    k1 = k1 && f1 == e1;
}

// Membership of e0 and e1 in two different lists, each given as a hash set
// (t != null, len >= GJ_HASH_MIN_DEG) or a short sorted list p[0, len) with
// len < GJ_HASH_MIN_DEG; the two tests' loads are interleaved. k0 / k1 enter
// as "test this one" and leave as the answers.
__device__ __forceinline__ void member_pair(const uint32_t* t0, const uint32_t* p0, uint32_t len0, uint32_t e0,
                                            bool& k0, const uint32_t* t1, const uint32_t* p1, uint32_t len1,
                                            uint32_t e1, bool& k1) {
    bool r0 = false, r1 = false;
    // hash sets: group by group from each key's home group
    bool a0 = k0 && t0, a1 = k1 && t1;
    const uint32_t b0 = a0 ? gj_tab_bits(len0) : 0u, b1 = a1 ? gj_tab_bits(len1) : 0u;
    uint32_t g0 = a0 ? gj_tab_start(e0, b0) : 0u, g1 = a1 ? gj_tab_start(e1, b1) : 0u;
    while (a0 || a1) {
        bool hit0 = false, emp0 = false, hit1 = false, emp1 = false;
        if (a0) gj_tab_group(t0, g0, e0, hit0, emp0);
        if (a1) gj_tab_group(t1, g1, e1, hit1, emp1);
        r0 |= hit0;
        r1 |= hit1;
        a0 = a0 && !hit0 && !emp0;
        a1 = a1 && !hit1 && !emp1;
        g0 = (g0 + 8u) & ((1u << b0) - 1u);
        g1 = (g1 + 8u) & ((1u << b1) - 1u);
    }
    // short sorted lists: four halving steps over [0, len < 16) (lower bound), then one compare
    const bool s0 = k0 && !t0 && len0, s1 = k1 && !t1 && len1;
    if (s0 || s1) {
        uint32_t q0 = 0, q1 = 0;
#pragma unroll
        for (uint32_t st = 8; st; st >>= 1) {
            const bool c0 = s0 && q0 + st <= len0, c1 = s1 && q1 + st <= len1;
            const uint32_t v0 = c0 ? __ldg(p0 + q0 + st - 1) : 0u, v1 = c1 ? __ldg(p1 + q1 + st - 1) : 0u;
            if (c0 && v0 < e0) q0 += st;
            if (c1 && v1 < e1) q1 += st;
        }
        if (s0) r0 = q0 < len0 && __ldg(p0 + q0) == e0;
        if (s1) r1 = q1 < len1 && __ldg(p1 + q1) == e1;
    }
    k0 = r0;
    k1 = r1;
}

// Two membership tests against the same hash set (groups of eight slots,
// as in gj_tab_member), their loads interleaved.
__device__ __forceinline__ void tab_member2(const uint32_t* __restrict__ tab, uint32_t bits, uint32_t e0, bool& k0,
                                            uint32_t e1, bool& k1) {
    const uint32_t mask = (1u << bits) - 1u;
    uint32_t g0 = gj_tab_start(e0, bits), g1 = gj_tab_start(e1, bits);
    bool a0 = k0, a1 = k1, r0 = false, r1 = false;
    while (a0 || a1) {
        bool hit0 = false, emp0 = false, hit1 = false, emp1 = false;
        if (a0) gj_tab_group(tab, g0, e0, hit0, emp0);
        if (a1) gj_tab_group(tab, g1, e1, hit1, emp1);
        r0 |= hit0;
        r1 |= hit1;
        a0 = a0 && !hit0 && !emp0;
        a1 = a1 && !hit1 && !emp1;
        g0 = (g0 + 8u) & mask;
        g1 = (g1 + 8u) & mask;
    }
    k0 = r0;
    k1 = r1;
}

__device__ __forceinline__ unsigned int vload(const unsigned int* p) {
    return *reinterpret_cast<const volatile unsigned int*>(p);
}

__device__ __forceinline__ unsigned long long vload64(const unsigned long long* p) {
    return *reinterpret_cast<const volatile unsigned long long*>(p);
}

__global__ void k_queue_init(unsigned long long* seq, uint32_t cap) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += gridDim.x * blockDim.x) seq[i] = i;
}

// DELTA: every plan is a delta query dQ_i (Section 3.3.1): seeds are the
// batch's signed changes, atoms read the old or the new version, and each
// prefix carries its seed's sign into the counts and checksums.
// EXT: some plan of the launch has tri atoms, inequality filters or an
// aggregated last level (Section 5.4, Section 3.4.2); without them those
// paths are compiled out.
template <bool DELTA, bool EXT>
__global__ void __launch_bounds__(FW * 32, 4) k_fused(FusedArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const uint32_t lt = gj_lanemask_lt();
    unsigned char* ws = smem_raw + (size_t)warp * warp_bytes(A.kmax, DELTA, EXT);
    Plan& P = *reinterpret_cast<Plan*>(ws);
    uint64_t* n_ = reinterpret_cast<uint64_t*>(ws + PLAN_BYTES);
    uint64_t* cur_ = n_ + GJ_MAX_K;
    uint64_t* tot_ = cur_ + GJ_MAX_K;
    uint64_t* ip_ = tot_ + GJ_MAX_K;  // prefix that owns candidate cur_ (advances monotonically)
    const GraphView& G = A.G;
    const uint64_t space = A.qbase[A.nq];

    if (lane < GJ_MAX_K) { n_[lane] = 0; cur_[lane] = 0; tot_[lane] = 0; ip_[lane] = 0; }
    if (lane == 0 && A.Q.b) atomicAdd(A.Q.busy, 1u);  // before the first grab of seeds
    __syncwarp();
    const DeltaView* Dv = DELTA ? &A.D : nullptr;

    int cur_q = -1;
    uint32_t k = 0;
    unsigned long long cnt = 0, chk = 0;  // cnt is kept warp-uniform (ballot counts); chk per lane
    uint64_t gpos = 0, gend = 0;  // the warp's grabbed, not yet read part of the seed space
    int depth = 1;             // deepest level being extended; 1 = none (take seeds)

    auto flush_q = [&]() {
        unsigned long long h = chk;
        for (int o = 16; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
        if (lane == 0 && cur_q >= 0) {
            if (cnt) {
                const unsigned long long old = atomicAdd(A.counts + cur_q, cnt);
                // a static count is exact below 2^63 (it is reported as int64)
                if (!DELTA && A.ovf && (old + cnt < old || ((old + cnt) >> 63))) atomicOr(A.ovf, 1ull);
            }
            if (h) atomicAdd(A.chks + cur_q, h);
        }
        cnt = 0;
        chk = 0;
    };

    // Count step for level j: min-c / min-i per prefix, scan of min-c. At
    // the last level also each prefix's factor of the match hash (the
    // query's factor times those of its k - 1 values), and in EXT launches
    // the other list of a two-binding level, kept for the extension step.
    auto activate = [&](int j, bool count_stats = true) {
        const uint32_t nj = (uint32_t)n_[j];
        uint32_t* tup = reinterpret_cast<uint32_t*>(ws + off_tup(j, DELTA, EXT));
        const uint32_t** mptr = reinterpret_cast<const uint32_t**>(ws + off_mptr(j, DELTA, EXT));
        uint64_t* cs = reinterpret_cast<uint64_t*>(ws + off_cs(j, DELTA, EXT));
        uint64_t* hpre = reinterpret_cast<uint64_t*>(ws + off_hpre(A.kmax, DELTA, EXT));
        uint8_t* minb = ws + off_minb(j, DELTA, EXT);
        const bool last = (j == (int)k - 1);
        // aggregation: a prefix that agrees with the one before it on every
        // position the last level reads has the same extensions; it joins
        // that prefix's group and proposes nothing itself
        const uint32_t aggm = (EXT && !DELTA && last) ? P.agg : 0u;
        // factorised output: at level k-2 the per-parent counters start at
        // zero; at the last level row i stands for w_i prefixes (its weight,
        // in the unread column k-2) and hpre already holds its factor sum
        const bool factl = EXT && !DELTA && last && P.fact;
        if (EXT && !DELTA && P.fact && j == (int)k - 2) {
            uint32_t* acc_n = reinterpret_cast<uint32_t*>(ws + off_tup(j + 1, DELTA, EXT)) + j * FC;
            acc_n[lane] = 0;
            acc_n[lane + 32] = 0;
            hpre[lane] = 0;
            hpre[lane + 32] = 0;
            __syncwarp();
        }
        uint64_t wsum = 0;  // factorised last level: the prefixes the rows stand for
        uint64_t len2[2];
        uint64_t all2 = 0;  // the min counts of every prefix, members of groups included
        bool lead2[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            uint32_t i = lane + 32 * h;
            uint64_t best = 0;
            bool lead = i < nj;
            if (aggm && i > 0 && i < nj) {
                lead = false;
                for (uint32_t p = 0; p < (uint32_t)j; p++)
                    if (((aggm >> p) & 1u) && tup[p * FC + i] != tup[p * FC + i - 1]) lead = true;
            }
            lead2[h] = lead;
            if (i < nj) {
                best = ~0ull;
                uint32_t bi = 0;
                const uint32_t* bp = nullptr;
                if (DELTA) {
                    // min by the degree in each atom's version; the list's
                    // enumeration space also holds the batch's deletions
                    uint32_t bdeg = 0xffffffffu;
                    ViewList bl{};
                    for (uint32_t b = 0; b < P.nb[j]; b++) {
                        const uint32_t v = tup[P.bpos[j][b] * FC + i];
                        const ViewList L = gj_view_list(G, Dv, P.bdir[j][b], P.bview[j][b], v);
                        if (L.degree() < bdeg) {
                            bdeg = L.degree();
                            bl = L;
                            bi = b;
                        }
                    }
                    best = bl.space();
                    bp = bl.base;
                    const uint32_t bdir = P.bdir[j][bi];
                    reinterpret_cast<uint32_t*>(ws + off_dins(j, EXT))[i] =
                        bl.nins ? (uint32_t)(bl.ins - dins_base(A.D, bdir)) : 0u;
                    reinterpret_cast<uint32_t*>(ws + off_ddel(j, EXT))[i] =
                        bl.ndel ? (uint32_t)(bl.del - ddel_base(A.D, bdir)) : 0u;
                    reinterpret_cast<uint32_t*>(ws + off_dblen(j, EXT))[i] = bl.base_len;
                    reinterpret_cast<uint32_t*>(ws + off_dndel(j, EXT))[i] = bl.ndel;
                } else {
                    // EXT, last level with two bindings: keep the other list
                    const bool keep_other = EXT && last && P.nb[j] == 2;
                    BindList other{G.fn, 0u, nullptr, 0u}, bestL{G.fn, 0u, nullptr, 0u};
                    for (uint32_t b = 0; b < P.nb[j]; b++) {
                        uint32_t v = tup[P.bpos[j][b] * FC + i];
                        const uint32_t dir = P.bdir[j][b];
                        uint64_t len;
                        const uint32_t* lp;
                        if (EXT && (dir == GJ_BIND_TRI || keep_other)) {
                            const BindList L = gj_bind_list(G, dir, v, tup[P.bpos2[j][b] * FC + i]);
                            len = L.len;
                            lp = L.p;
                            if (keep_other) {
                                if (len < best) {
                                    other = bestL;
                                    bestL = L;
                                } else {
                                    other = L;
                                }
                            }
                        } else if (GJ_CHECK(G.chk, v < G.n, GJ_SITE_VERTEX, v)) {
                            const int64_t* off = dir ? G.ro : G.fo;
                            int64_t s = __ldg(off + v);
                            len = (uint64_t)(__ldg(off + v + 1) - s);
                            lp = (dir ? G.rn : G.fn) + s;
                            if (!GJ_CHECK(G.chk, (uint64_t)s + len <= G.m, GJ_SITE_LIST, v)) len = 0;
                        } else {
                            len = 0;
                            lp = G.fn;
                        }
                        if (len < best) {
                            best = len;
                            bi = b;
                            bp = lp;
                        }
                    }
                    if (keep_other) {
                        reinterpret_cast<const uint32_t**>(ws + off_olp(A.kmax, DELTA, EXT))[i] = other.bits ? other.tab : other.p;
                        reinterpret_cast<uint32_t*>(ws + off_oll(A.kmax, DELTA, EXT))[i] = other.len;
                    }
                    all2 += best;
                    if (!lead) best = 0;
                }
                mptr[i] = bp;
                minb[i] = (uint8_t)bi;
                if (factl) {
                    const uint32_t w = tup[(j - 1) * FC + i];
                    wsum += w;
                    all2 += (uint64_t)w * best - best;  // the row counted once above
                } else if (last) {
                    uint64_t hh = gj_hq(k);
                    for (uint32_t p = 0; p < (uint32_t)j; p++) hh *= gj_hf(P.order[p], tup[p * FC + i]);
                    hpre[i] = hh;
                }
            }
            len2[h] = best;
        }
        if (aggm || factl)
            for (int o = 16; o > 0; o >>= 1) all2 += __shfl_xor_sync(0xffffffffu, all2, o);
        if (factl)
            for (int o = 16; o > 0; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
        if (aggm) {
            const uint32_t l0 = __ballot_sync(0xffffffffu, lead2[0]), l1 = __ballot_sync(0xffffffffu, lead2[1]);
            const uint64_t L = (uint64_t)l0 | ((uint64_t)l1 << 32);
            uint8_t* grp = ws + off_grp(A.kmax, DELTA, EXT);
            uint32_t gend[2] = {0, 0};
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t i = lane + 32 * h;
                if (lead2[h]) {
                    const uint64_t rest = i + 1 < 64 ? (L >> (i + 1)) : 0ull;
                    const uint32_t next = rest ? i + 1 + (uint32_t)__ffsll((long long)rest) - 1 : nj;
                    grp[i] = (uint8_t)(next - i);
                    gend[h] = next;
                }
            }
            __syncwarp();
            // a group's matches are its members' prefixes times the leader's
            // extensions: the sum of their hashes is (sum of the members'
            // factors) x (the extension's factor), so the leader keeps the sum
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t i = lane + 32 * h;
                if (lead2[h]) {
                    uint64_t sum = hpre[i];
                    for (uint32_t m = i + 1; m < gend[h]; m++) sum += hpre[m];
                    hpre[i] = sum;
                }
            }
        }
        // inclusive scans of the two halves, then exclusive offsets
        uint64_t a = len2[0], b = len2[1];
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t ta = __shfl_up_sync(0xffffffffu, a, o);
            uint64_t tb = __shfl_up_sync(0xffffffffu, b, o);
            if (lane >= o) { a += ta; b += tb; }
        }
        uint64_t tot_a = __shfl_sync(0xffffffffu, a, 31);
        b += tot_a;
        uint64_t total = __shfl_sync(0xffffffffu, b, 31);
        cs[lane] = a - len2[0];
        cs[lane + 32] = b - len2[1];
        if (lane == 0) {
            cs[FC] = total;
            cur_[j] = 0;
            tot_[j] = total;
            ip_[j] = 0;
        }
        __syncwarp();
        // work units of the cost model count every prefix, also those whose
        // extensions an aggregated group shares
        if (lane == 0 && count_stats) {
            const uint64_t rows = factl ? wsum : nj;
            stat_add(A.stats, 0, j, rows);
            stat_add(A.stats, 1, j, (unsigned long long)rows * P.nb[j]);
            stat_add(A.stats, 2, j, (aggm || factl) ? all2 : total);
        }
    };

    // The count step runs from one place (one inlined copy of its code): the
    // branches that descend to a level set act (and, for a donated candidate
    // range, its bounds) and loop back here.
    int act = -1;
    bool act_stats = true, act_ranged = false;
    unsigned long long act_lo = 0, act_hi = 0;
    while (true) {
        if (act >= 0) {
            activate(act, act_stats);
            if (act_ranged) {
                if (lane == 0) {
                    cur_[act] = act_lo;
                    if (act_hi < tot_[act]) tot_[act] = act_hi;
                }
                __syncwarp();
            }
            depth = act;
            act = -1;
            act_stats = true;
            act_ranged = false;
            continue;
        }
        if (depth == 1) {
            // ---------------- take seeds, 32 at a time from the grabbed range
            if (gpos >= gend) {
                unsigned long long t = 0;
                if (lane == 0) t = atomicAdd(A.next, (unsigned long long)A.chunk);
                gpos = __shfl_sync(0xffffffffu, t, 0);
                gend = gpos + A.chunk;
            }
            const uint64_t g = gpos;
            if (g >= space) {
                if (k > 2 && n_[2] > 0) {
                    act = 2;
                    continue;
                }
                if (!A.Q.b) break;
                // No seeds left: take a donated bundle, or wait until no warp
                // holds work and none is left. The wait is bounded: it gives
                // up once the queue (head, tail, idle and busy counts) has not
                // changed for A.wait_ns, or once another warp has given up.
                const unsigned long long mask = A.Q.cap - 1;
                long long took = -1;
                bool idle_marked = false, give_up = false;
                uint32_t backoff = 64;  // ns; doubles while nothing is published (less polling traffic)
                unsigned long long seen_h = ~0ull, seen_t = ~0ull;
                unsigned int seen_i = ~0u, seen_b = ~0u;
                uint64_t since = globaltimer_ns();
                if (lane == 0) atomicSub(A.Q.busy, 1u);
                while (true) {
                    long long b = -1;
                    if (lane == 0) {
                        const unsigned long long h = vload64(A.Q.head);
                        if (vload64(A.Q.seq + (h & mask)) == h + 1) {  // published
                            if (idle_marked) atomicSub(A.Q.idle, 1u);
                            idle_marked = false;
                            atomicAdd(A.Q.busy, 1u);  // before the claim, so that busy == 0 never hides it
                            if (atomicCAS(A.Q.head, h, h + 1) == h) b = (long long)h;
                            else atomicSub(A.Q.busy, 1u);
                        } else if (h == vload64(A.Q.tail)) {  // empty
                            if (!idle_marked) atomicAdd(A.Q.idle, 1u);
                            idle_marked = true;
                            if (vload(A.Q.busy) == 0u) {
                                // a giver fences between its reservation and its
                                // leaving busy: read busy first, then the queue
                                __threadfence();
                                if (vload64(A.Q.head) == vload64(A.Q.tail)) b = -2;
                            }
                        }
                        if (b == -1) {
                            const unsigned long long t = vload64(A.Q.tail);
                            const unsigned int iw = vload(A.Q.idle), bw = vload(A.Q.busy);
                            const uint64_t now = globaltimer_ns();
                            if (h != seen_h || t != seen_t || iw != seen_i || bw != seen_b) {
                                seen_h = h;
                                seen_t = t;
                                seen_i = iw;
                                seen_b = bw;
                                since = now;
                            } else if (now - since > A.wait_ns || vload64(A.Q.err)) {
                                b = -3;
                            }
                        }
                    }
                    b = __shfl_sync(0xffffffffu, b, 0);
                    idle_marked = __shfl_sync(0xffffffffu, idle_marked, 0);
                    if (b >= 0) {
                        took = b;
                        break;
                    }
                    if (b == -2) break;
                    if (b == -3) {
                        give_up = true;
                        break;
                    }
                    __nanosleep(backoff);
                    if (backoff < 16384) backoff <<= 1;
                }
                if (give_up) {
                    if (lane == 0) atomicExch(A.Q.err, 1ull);
                    break;
                }
                if (took < 0) break;
                __threadfence();
                const Bundle& Bd = A.Q.b[took & mask];
                const int q2 = (int)Bd.plan;
                if (q2 != cur_q) {
                    flush_q();
                    cur_q = q2;
                    const uint32_t* srcw = reinterpret_cast<const uint32_t*>(A.plans + q2);
                    uint32_t* dstw = reinterpret_cast<uint32_t*>(&P);
                    for (uint32_t w = lane; w < sizeof(Plan) / 4; w += 32) dstw[w] = srcw[w];
                    __syncwarp();
                    k = P.k;
                }
                const uint32_t L = Bd.level, nb_ = Bd.n;
                if (!GJ_CHECK(G.chk, nb_ <= FC && L >= 2 && L < k, GJ_SITE_BUNDLE, ((uint64_t)L << 32) | nb_)) {
                    if (lane == 0) atomicExch(A.Q.seq + (took & mask), (unsigned long long)took + A.Q.cap);
                    __syncwarp();
                    continue;
                }
                uint32_t* tupL = reinterpret_cast<uint32_t*>(ws + off_tup(L, DELTA, EXT));
                for (uint32_t c = 0; c < L; c++)
                    for (uint32_t i = lane; i < nb_; i += 32) tupL[c * FC + i] = Bd.tup[c][i];
                if (DELTA)
                    for (uint32_t i = lane; i < nb_; i += 32) reinterpret_cast<int8_t*>(ws + off_dsg(L, EXT))[i] = Bd.sg[i];
                if (EXT && !DELTA && P.fact && L == k - 1)
                    for (uint32_t i = lane; i < nb_; i += 32)
                        reinterpret_cast<uint64_t*>(ws + off_hpre(A.kmax, DELTA, EXT))[i] = Bd.hp[i];
                const unsigned long long c_lo = Bd.c_lo, c_hi = Bd.c_hi;
                __syncwarp();
                if (lane == 0) {
                    n_[L] = nb_;
                    __threadfence();
                    atomicExch(A.Q.seq + (took & mask), (unsigned long long)took + A.Q.cap);  // free the slot
                }
                __syncwarp();
                // a candidate range of a batch already counted by its giver is not counted again
                act = (int)L;
                act_ranged = c_hi != ~0ull;
                act_stats = !act_ranged;
                act_lo = c_lo;
                act_hi = c_hi;
                continue;
            }
            // query owning this chunk: last q with qbase[q] <= g
            uint32_t lo = 0, hi = A.nq;
            while (hi - lo > 1) {
                uint32_t mid = (lo + hi) >> 1;
                if (A.qbase[mid] <= g) lo = mid; else hi = mid;
            }
            const int q = (int)lo;
            if (q != cur_q) {
                if (k > 2 && n_[2] > 0) {  // finish the other query's prefixes first (g is read later)
                    act = 2;
                    continue;
                }
                flush_q();
                cur_q = q;
                const uint32_t* srcw = reinterpret_cast<const uint32_t*>(A.plans + q);
                uint32_t* dstw = reinterpret_cast<uint32_t*>(&P);
                for (uint32_t w = lane; w < sizeof(Plan) / 4; w += 32) dstw[w] = srcw[w];
                __syncwarp();
                k = P.k;
            }
            // up to 32 seeds of the grabbed range (fewer when a grab is smaller)
            const uint64_t span = gend - g < 32 ? gend - g : 32;
            const uint64_t s = g - A.qbase[q] + lane;
            bool keep = (int64_t)s < A.seed_n[q] && (uint64_t)lane < span;
            gpos = g + span;
            if (lane == 0) {
                int64_t left = A.seed_n[q] - (int64_t)(g - A.qbase[q]);
                if (left > 0) stat_add(A.stats, 4, 0, (unsigned long long)((uint64_t)left < span ? left : span));
            }
            uint32_t x0 = 0, x1 = 0;
            int8_t sg = 1;
            if (keep) {
                const int64_t e = A.seed_lo[q] + (int64_t)s;
                if (DELTA) {
                    x0 = A.B.chg_src[e];
                    x1 = A.B.chg_dst[e];
                    sg = A.B.chg_sign[e];
                } else {
                    x0 = __ldg((P.seed_dir ? G.rk : G.fk) + e);
                    x1 = __ldg((P.seed_dir ? G.rn : G.fn) + e);
                }
                for (uint32_t f = 0; f < P.nsf && keep; f++) {
                    uint32_t u = P.sf_dir[f] ? x1 : x0, w = P.sf_dir[f] ? x0 : x1;
                    keep = DELTA ? gj_view_member(G, Dv, 0, P.sf_view[f], u, w)
                                 : gj_list_member(G.fo, G.fn, G.fto, G.ft, u, w);
                }
                if (EXT) keep = keep && gj_lt_ok(P, 1, x1, [&](uint32_t) { return x0; });
            }
            if (k == 2) {
                if (keep) {
                    const uint64_t h = gj_hq(2) * gj_hf(P.order[0], x0) * gj_hf(P.order[1], x1);
                    chk += sg > 0 ? h : 0ull - h;
                }
                cnt += __popc(__ballot_sync(0xffffffffu, keep && sg > 0)) -
                       __popc(__ballot_sync(0xffffffffu, keep && sg < 0));
                continue;
            }
            uint32_t mask = __ballot_sync(0xffffffffu, keep);
            uint32_t n2 = (uint32_t)n_[2];
            if (keep) {
                uint32_t slot = n2 + __popc(mask & lt);
                uint32_t* tup = reinterpret_cast<uint32_t*>(ws + off_tup(2, DELTA, EXT));
                tup[0 * FC + slot] = x0;
                tup[1 * FC + slot] = x1;
                if (DELTA) reinterpret_cast<int8_t*>(ws + off_dsg(2, EXT))[slot] = sg;
            }
            __syncwarp();
            if (lane == 0) {
                n_[2] = n2 + __popc(mask);
                stat_add(A.stats, 3, 2, __popc(mask));
            }
            __syncwarp();
            if (n_[2] >= FT) act = 2;
            continue;
        }

        // ---------------- extend level j = depth
        // Proposals of the level's batch are taken 32 at a time (one per
        // lane) in a local loop; a mid level leaves the loop as soon as the
        // next level holds B' prefixes (deepest level first), the last
        // level runs to the end. When all 32 candidates of a step belong to
        // one prefix (long lists), that prefix's other binding lists stay
        // cached in registers across steps.
        const int j = depth;
        if (cur_[j] < tot_[j]) {
            uint64_t tot = tot_[j];
            const uint32_t nj = (uint32_t)n_[j];
            const uint32_t* tup = reinterpret_cast<const uint32_t*>(ws + off_tup(j, DELTA, EXT));
            const uint32_t* const* mptr = reinterpret_cast<const uint32_t* const*>(ws + off_mptr(j, DELTA, EXT));
            const uint64_t* cs = reinterpret_cast<const uint64_t*>(ws + off_cs(j, DELTA, EXT));
            uint64_t* hpre = reinterpret_cast<uint64_t*>(ws + off_hpre(A.kmax, DELTA, EXT));
            const uint8_t* minb = ws + off_minb(j, DELTA, EXT);
            const bool last = (j == (int)k - 1);
            // factorised output: level k-2 only counts and sums the factors of
            // each parent's extensions (into the last level's weight column
            // and hpre); the last level weighs each row by its weight
            const bool factj = EXT && !DELTA && P.fact && j == (int)k - 2;
            const bool factl = EXT && !DELTA && P.fact && last;
            uint32_t* acc_n = reinterpret_cast<uint32_t*>(ws + off_tup(j + 1, DELTA, EXT)) + j * FC;
            const uint32_t nb = P.nb[j];
            const uint32_t a_new = P.order[j];
            uint32_t* nt = reinterpret_cast<uint32_t*>(ws + off_tup(last ? j : j + 1, DELTA, EXT));
            const uint8_t* grp = ws + off_grp(A.kmax, DELTA, EXT);
            const bool agg = EXT && !DELTA && last && P.agg;
            // other binding lists cached in registers for a step-uniform prefix:
            // two for plain edge queries (up to 4-cliques), one in the extended
            // variant (its code size and registers cost more than the cache saves)
            constexpr int MAXO = EXT ? 1 : 2;
            const uint32_t* ob[MAXO];  // the list, or its hash set when obits > 0
            uint32_t ol[MAXO], obits[MAXO];
            uint32_t cached = 0xffffffffu;
            uint32_t dcached = 0xffffffffu;  // delta plans: the prefix whose views the cache holds
            DViewCache* dvc = reinterpret_cast<DViewCache*>(ws + off_dvc(A.kmax, DELTA, EXT));
            // delta plans: the other views of prefix pi, lane q taking the q-th one
            auto dcache = [&](uint32_t pi) {
                const uint32_t b0 = minb[pi];
                if (lane + 1 < (int)nb) {
                    const uint32_t b = (uint32_t)lane < b0 ? (uint32_t)lane : (uint32_t)lane + 1;
                    const uint32_t dir = P.bdir[j][b];
                    const uint32_t v = tup[P.bpos[j][b] * FC + pi];
                    const ViewList L = gj_view_list(G, Dv, dir, P.bview[j][b], v);
                    const bool hs = L.base_len >= GJ_HASH_MIN_DEG;
                    dvc->cp[lane] = hs ? (dir ? G.rt : G.ft) + __ldg((dir ? G.rto : G.fto) + v) : L.base;
                    dvc->cbits[lane] = hs ? gj_tab_bits(L.base_len) : 0u;
                    dvc->cl[lane] = L.base_len;
                    dvc->ins[lane] = L.ins;
                    dvc->nins[lane] = L.nins;
                    dvc->del[lane] = L.del;
                    dvc->ndel[lane] = L.ndel;
                }
                __syncwarp();
                dcached = pi;
            };
            uint32_t lo_in = 0;         // the cached prefix's inequality bounds: lo_in <= e < hi_ex
            uint64_t hi_ex = 1ull << 32;
            // the other binding lists and the inequality bounds of prefix pi, in registers
            auto cache_prefix = [&](uint32_t pi) {
                if (EXT && last && nb == 2) {  // the other list, kept by the count step
                    ol[0] = reinterpret_cast<const uint32_t*>(ws + off_oll(A.kmax, DELTA, EXT))[pi];
                    ob[0] = reinterpret_cast<const uint32_t* const*>(ws + off_olp(A.kmax, DELTA, EXT))[pi];
                    obits[0] = ol[0] >= GJ_HASH_MIN_DEG ? gj_tab_bits(ol[0]) : 0u;
                } else {
                    const uint32_t b0 = minb[pi];
                    uint32_t o = 0;
                    for (uint32_t b = 0; b < nb; b++) {
                        if (b == b0) continue;
                        const uint32_t dir = EXT ? P.bdir[j][b] : (P.bdir[j][b] & 1u);
                        const BindList L =
                            gj_bind_list(G, dir, tup[P.bpos[j][b] * FC + pi], tup[P.bpos2[j][b] * FC + pi]);
#pragma unroll
                        for (int q = 0; q < MAXO; q++)
                            if (q == (int)o) {
                                ob[q] = L.bits ? L.tab : L.p;
                                ol[q] = L.len;
                                obits[q] = L.bits;
                            }
                        o++;
                    }
                }
                lo_in = 0;
                hi_ex = 1ull << 32;
                for (uint32_t c = 0; EXT && c < P.nlt[j]; c++) {
                    const uint32_t v = tup[P.lt_pos[j][c] * FC + pi];
                    if (P.lt_less[j][c]) hi_ex = v < hi_ex ? v : hi_ex;
                    else lo_in = v + 1 > lo_in ? v + 1 : lo_in;
                }
                cached = pi;
            };
            uint64_t cur = cur_[j];
            uint32_t ip = (uint32_t)ip_[j];
            uint32_t nn = last ? 0u : (uint32_t)n_[j + 1];
            bool descend = false;
            uint64_t chk_at = cur;  // the next cursor at which the shared idle counter is read
            while (cur < tot) {
                // give the upper half of a long remaining range to an idle warp
                // (the shared idle counter is read once per 1024 candidates)
                if (A.Q.b && tot - cur >= RANGE_SPLIT_MIN && cur >= chk_at) {
                    chk_at = cur + 1024;
                    bool give = false;
                    unsigned long long slot = 0;
                    const uint64_t mid = cur + (((tot - cur) / 2 + 31) & ~31ull);
                    if (lane == 0 && (A.Q.always || vload(A.Q.idle) > 0u)) {
                        const unsigned long long t = vload64(A.Q.tail);
                        if (vload64(A.Q.seq + (t & (A.Q.cap - 1))) == t && atomicCAS(A.Q.tail, t, t + 1) == t) {
                            slot = t;
                            give = true;
                        }
                    }
                    give = __shfl_sync(0xffffffffu, give, 0);
                    if (give) {
                        slot = __shfl_sync(0xffffffffu, slot, 0);
                        Bundle& Bd = A.Q.b[slot & (A.Q.cap - 1)];
                        for (int c = 0; c < j; c++)
                            for (uint32_t i2 = lane; i2 < nj; i2 += 32) Bd.tup[c][i2] = tup[c * FC + i2];
                        if (DELTA)
                            for (uint32_t i2 = lane; i2 < nj; i2 += 32)
                                Bd.sg[i2] = reinterpret_cast<const int8_t*>(ws + off_dsg(j, EXT))[i2];
                        if (factl)
                            for (uint32_t i2 = lane; i2 < nj; i2 += 32) Bd.hp[i2] = hpre[i2];
                        if (lane == 0) {
                            Bd.plan = (uint32_t)cur_q;
                            Bd.level = (uint32_t)j;
                            Bd.n = nj;
                            Bd.c_lo = mid;
                            Bd.c_hi = tot;
                        }
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) atomicExch(A.Q.seq + (slot & (A.Q.cap - 1)), slot + 1);  // publish
                        tot = mid;
                    }
                }
                while (ip + 1 < nj && cs[ip + 1] <= cur) ip++;
                if (!DELTA && (last || factj) && nb - 1 <= (uint32_t)MAXO && !(ip + 1 < nj && cs[ip + 1] < cur + 64)) {
                    // Last level (or a factorised level k-2), next 64
                    // candidates all in prefix ip: two per lane, with their
                    // probes interleaved.
                    if (ip != cached) cache_prefix(ip);
                    // prefixes whose matches these candidates make (hp is then
                    // the sum of their hash factors)
                    const uint32_t gsz = (EXT && agg) ? grp[ip] : (factl ? tup[(j - 1) * FC + ip] : 1u);
                    // Up to 16 steps on prefix ip alone, its invariants in
                    // registers and 32-bit offsets r into its min list. When
                    // the warp's range [cur, tot) ends inside prefix ip (its
                    // batch's last prefix, or a range split off by a
                    // donation), the last step may be partial.
                    const uint64_t c0 = cs[ip];
                    const uint64_t pend = ip + 1 < nj ? cs[ip + 1] : tot;
                    const bool tail_ok = tot <= pend;
                    const uint32_t rend = (uint32_t)((tail_ok ? tot : pend) - c0);
                    const uint32_t* ml = mptr[ip];
                    const uint64_t hp = hpre[ip];
                    uint32_t r = (uint32_t)(cur - c0);
                    uint32_t steps = 0;
                    uint64_t sacc = 0;  // factorised level k-2: the step's factor sum and count
                    uint32_t nacc = 0;
                    do {
                        const uint32_t q0 = r + lane, q1 = r + 32 + lane;
                        bool k0 = q0 < rend, k1 = q1 < rend;
                        const uint32_t e0 = k0 ? __ldg(ml + q0) : 0u;
                        const uint32_t e1 = k1 ? __ldg(ml + q1) : 0u;
                        if (EXT) {
                            k0 = k0 && e0 >= lo_in && (uint64_t)e0 < hi_ex;
                            k1 = k1 && e1 >= lo_in && (uint64_t)e1 < hi_ex;
                        }
#pragma unroll
                        for (int q = 0; q < MAXO; q++) {
                            if (q + 1 < (int)nb) {
                                if (obits[q]) tab_member2(ob[q], obits[q], e0, k0, e1, k1);
                                else member32x2(ob[q], ol[q], e0, k0, e1, k1);
                            }
                        }
                        const uint32_t c2 = __popc(__ballot_sync(0xffffffffu, k0)) + __popc(__ballot_sync(0xffffffffu, k1));
                        if (EXT && factj) {
                            if (k0) sacc += gj_hf(a_new, e0);
                            if (k1) sacc += gj_hf(a_new, e1);
                            nacc += c2;
                        } else {
                            if (k0) chk += hp * gj_hf(a_new, e0);
                            if (k1) chk += hp * gj_hf(a_new, e1);
                            cnt += EXT ? (unsigned long long)c2 * gsz : (unsigned long long)c2;
                        }
                        r += 64;
                    } while (++steps < 16 && r < rend && (tail_ok || rend - r >= 64));
                    if (EXT && factj) {
                        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                        if (lane == 0 && nacc) {
                            acc_n[ip] += nacc;
                            hpre[ip] += sacc;
                            stat_add(A.stats, 3, j + 1, nacc);
                        }
                        __syncwarp();
                    }
                    cur = c0 + r;
                    continue;
                }
                if (DELTA && last && nb <= 3 && !(ip + 1 < nj && cs[ip + 1] < cur + 64)) {
                    // Delta plans, last level, next 64 candidates all in prefix ip:
                    // two per lane, the other views cached once for the run, the
                    // committed-list probes of the two candidates interleaved.
                    if (ip != dcached) dcache(ip);
                    const uint64_t c0 = cs[ip];
                    const uint32_t r0 = (uint32_t)(cur - c0) + lane, r1 = r0 + 32;
                    bool k0 = cur + lane < tot, k1 = cur + 32 + lane < tot;
                    const uint32_t blen = reinterpret_cast<const uint32_t*>(ws + off_dblen(j, EXT))[ip];
                    const uint32_t mdel = reinterpret_cast<const uint32_t*>(ws + off_dndel(j, EXT))[ip];
                    const uint32_t mdir = P.bdir[j][minb[ip]];
                    const uint32_t* mins = dins_base(A.D, mdir) + reinterpret_cast<const uint32_t*>(ws + off_dins(j, EXT))[ip];
                    const uint32_t* mdl = ddel_base(A.D, mdir) + reinterpret_cast<const uint32_t*>(ws + off_ddel(j, EXT))[ip];
                    const uint32_t* ml = mptr[ip];
                    uint32_t e0 = 0, e1 = 0;
                    if (k0) e0 = r0 < blen ? __ldg(ml + r0) : __ldg(mins + (r0 - blen));
                    if (k1) e1 = r1 < blen ? __ldg(ml + r1) : __ldg(mins + (r1 - blen));
                    if (mdel) {  // committed entries deleted in the min list's view
                        if (k0 && r0 < blen) k0 = !gj_contains(mdl, mdel, e0);
                        if (k1 && r1 < blen) k1 = !gj_contains(mdl, mdel, e1);
                    }
                    if (EXT && P.nlt[j]) {
                        k0 = k0 && gj_lt_ok(P, j, e0, [&](uint32_t p) { return tup[p * FC + ip]; });
                        k1 = k1 && gj_lt_ok(P, j, e1, [&](uint32_t p) { return tup[p * FC + ip]; });
                    }
                    for (uint32_t q = 0; q + 1 < nb; q++) {
                        // inserted in this view: a member; deleted: not; else the committed list
                        const bool in0 = k0 && dvc->nins[q] && gj_contains(dvc->ins[q], dvc->nins[q], e0);
                        const bool in1 = k1 && dvc->nins[q] && gj_contains(dvc->ins[q], dvc->nins[q], e1);
                        const bool de0 = k0 && !in0 && dvc->ndel[q] && gj_contains(dvc->del[q], dvc->ndel[q], e0);
                        const bool de1 = k1 && !in1 && dvc->ndel[q] && gj_contains(dvc->del[q], dvc->ndel[q], e1);
                        bool c0 = k0 && !in0 && !de0, c1 = k1 && !in1 && !de1;
                        const uint32_t* tb = dvc->cbits[q] ? dvc->cp[q] : nullptr;
                        member_pair(tb, dvc->cp[q], dvc->cl[q], e0, c0, tb, dvc->cp[q], dvc->cl[q], e1, c1);
                        k0 = in0 || c0;
                        k1 = in1 || c1;
                    }
                    const int8_t sg = reinterpret_cast<const int8_t*>(ws + off_dsg(j, EXT))[ip];
                    const uint64_t hp = hpre[ip];
                    uint64_t h = (k0 ? hp * gj_hf(a_new, e0) : 0ull) + (k1 ? hp * gj_hf(a_new, e1) : 0ull);
                    chk += sg > 0 ? h : 0ull - h;
                    const int c2 = __popc(__ballot_sync(0xffffffffu, k0)) + __popc(__ballot_sync(0xffffffffu, k1));
                    cnt += sg > 0 ? (unsigned long long)c2 : 0ull - (unsigned long long)c2;
                    cur += 64;
                    continue;
                }
                if (EXT && !DELTA && last && nb == 2) {
                    // Last level with the kept second list, candidates of several
                    // short prefixes: two per lane (t and t + 32), each resolved to
                    // its prefix by binary search, their probes interleaved.
                    const uint64_t t0 = cur + lane, t1 = cur + 32 + lane;
                    bool k0 = t0 < tot, k1 = t1 < tot;
                    uint32_t lo0 = ip, hi0 = nj, lo1 = ip, hi1 = nj;  // last i with cs[i] <= t
                    while (hi0 - lo0 > 1 || hi1 - lo1 > 1) {
                        if (hi0 - lo0 > 1) {
                            const uint32_t mid = (lo0 + hi0) >> 1;
                            if (cs[mid] <= t0) lo0 = mid; else hi0 = mid;
                        }
                        if (hi1 - lo1 > 1) {
                            const uint32_t mid = (lo1 + hi1) >> 1;
                            if (cs[mid] <= t1) lo1 = mid; else hi1 = mid;
                        }
                    }
                    const uint32_t i0 = lo0, i1 = lo1;
                    ip = __shfl_sync(0xffffffffu, i1, 31);  // the next step starts in or after it
                    const uint32_t e0 = k0 ? __ldg(mptr[i0] + (t0 - cs[i0])) : 0u;
                    const uint32_t e1 = k1 ? __ldg(mptr[i1] + (t1 - cs[i1])) : 0u;
                    if (P.nlt[j]) {
                        k0 = k0 && gj_lt_ok(P, j, e0, [&](uint32_t p) { return tup[p * FC + i0]; });
                        k1 = k1 && gj_lt_ok(P, j, e1, [&](uint32_t p) { return tup[p * FC + i1]; });
                    }
                    const uint32_t* const* olp = reinterpret_cast<const uint32_t* const*>(ws + off_olp(A.kmax, DELTA, EXT));
                    const uint32_t* oll = reinterpret_cast<const uint32_t*>(ws + off_oll(A.kmax, DELTA, EXT));
                    const uint32_t l0 = oll[i0], l1 = oll[i1];
                    member_pair(l0 >= GJ_HASH_MIN_DEG ? olp[i0] : nullptr, olp[i0], l0, e0, k0,
                                l1 >= GJ_HASH_MIN_DEG ? olp[i1] : nullptr, olp[i1], l1, e1, k1);
                    if (k0) chk += hpre[i0] * gj_hf(a_new, e0);
                    if (k1) chk += hpre[i1] * gj_hf(a_new, e1);
                    if (agg || factl) {
                        // weighted rows: aggregated groups, or factorised parents
                        const uint32_t w0 = k0 ? (agg ? grp[i0] : tup[(j - 1) * FC + i0]) : 0u;
                        const uint32_t w1 = k1 ? (agg ? grp[i1] : tup[(j - 1) * FC + i1]) : 0u;
                        unsigned long long w = (unsigned long long)w0 + w1;
                        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                        cnt += w;
                    } else {
                        cnt += __popc(__ballot_sync(0xffffffffu, k0)) + __popc(__ballot_sync(0xffffffffu, k1));
                    }
                    cur += 64;
                    continue;
                }
                const uint64_t t = cur + lane;
                bool keep = t < tot;
                const bool uni = !(ip + 1 < nj && cs[ip + 1] < cur + 32);
                uint32_t i = ip;
                if (!uni) {
                    // this step spans several prefixes: last i with cs[i] <= t
                    uint32_t lo = ip, hi = nj;
                    while (hi - lo > 1) {
                        uint32_t mid = (lo + hi) >> 1;
                        if (cs[mid] <= t) lo = mid; else hi = mid;
                    }
                    i = lo;
                    // the next step starts at or after the last lane's prefix
                    ip = __shfl_sync(0xffffffffu, i, 31);
                }
                uint32_t e = 0;
                int8_t sg = 1;
                if (DELTA) {
                    if (keep) {
                        // element r of the min list's new-version enumeration space
                        const uint32_t r = (uint32_t)(t - cs[i]);
                        const uint32_t blen = reinterpret_cast<const uint32_t*>(ws + off_dblen(j, EXT))[i];
                        const uint32_t ndel = reinterpret_cast<const uint32_t*>(ws + off_dndel(j, EXT))[i];
                        if (r < blen) {
                            e = __ldg(mptr[i] + r);
                            if (ndel)
                                keep = !gj_contains(ddel_base(A.D, P.bdir[j][minb[i]]) +
                                                        reinterpret_cast<const uint32_t*>(ws + off_ddel(j, EXT))[i],
                                                    ndel, e);
                        } else {
                            e = __ldg(dins_base(A.D, P.bdir[j][minb[i]]) +
                                      reinterpret_cast<const uint32_t*>(ws + off_dins(j, EXT))[i] + (r - blen));
                        }
                        sg = reinterpret_cast<const int8_t*>(ws + off_dsg(j, EXT))[i];
                    }
                    if (uni && nb <= 3) {
                        // every candidate of the step is prefix ip's: its other views
                        // are looked up once per run (lane q takes the q-th one)
                        if (ip != dcached) dcache(ip);
                        for (uint32_t q = 0; q + 1 < nb && keep; q++) {
                            // committed member unless deleted; otherwise only if inserted
                            const bool c = dvc->cbits[q] ? gj_tab_member(dvc->cp[q], dvc->cbits[q], e)
                                                         : gj_contains(dvc->cp[q], dvc->cl[q], e);
                            keep = c ? !(dvc->ndel[q] && gj_contains(dvc->del[q], dvc->ndel[q], e))
                                     : (dvc->nins[q] && gj_contains(dvc->ins[q], dvc->nins[q], e));
                        }
                    } else if (keep) {
                        const uint32_t b0 = minb[i];
                        for (uint32_t b = 0; b < nb && keep; b++) {
                            if (b == b0) continue;
                            const uint32_t v = tup[P.bpos[j][b] * FC + i];
                            keep = gj_view_member(G, Dv, P.bdir[j][b], P.bview[j][b], v, e);
                        }
                    }
                } else if (keep) {
                    e = __ldg(mptr[i] + (t - cs[i]));
                }
                if (EXT && keep && P.nlt[j]) keep = gj_lt_ok(P, j, e, [&](uint32_t p) { return tup[p * FC + i]; });
                if (DELTA) {
                } else if (uni && nb - 1 <= (uint32_t)MAXO) {
                    if (ip != cached) cache_prefix(ip);
#pragma unroll
                    for (int q = 0; q < MAXO; q++)
                        if (q + 1 < (int)nb && keep)
                            keep = obits[q] ? gj_tab_member(ob[q], obits[q], e) : member32(ob[q], ol[q], e);
                } else if (EXT && last && nb == 2) {
                    // the other list, kept by the count step
                    if (keep) {
                        const uint32_t len = reinterpret_cast<const uint32_t*>(ws + off_oll(A.kmax, DELTA, EXT))[i];
                        const uint32_t* t = len >= GJ_HASH_MIN_DEG
                                                ? reinterpret_cast<const uint32_t* const*>(ws + off_olp(A.kmax, DELTA, EXT))[i]
                                                : nullptr;
                        keep = t ? gj_tab_member(t, gj_tab_bits(len), e)
                                 : gj_contains(reinterpret_cast<const uint32_t* const*>(ws + off_olp(A.kmax, DELTA, EXT))[i],
                                               len, e);
                    }
                } else if (EXT) {
                    // The lanes of one prefix look its lists up once: the first
                    // lane of each run of equal prefixes resolves them and the
                    // others read the result (aggregation of identical lookups).
                    const uint32_t b0 = minb[i];
                    const uint32_t prev = __shfl_up_sync(0xffffffffu, i, 1);
                    const bool head = lane == 0 || prev != i;
                    const int src = 31 - __clz(__ballot_sync(0xffffffffu, head) & (lt | (1u << lane)));
                    for (uint32_t b = 0; b < nb; b++) {
                        BindList L{nullptr, 0u, nullptr, 0u};
                        if (head && b != b0)
                            L = gj_bind_list(G, P.bdir[j][b], tup[P.bpos[j][b] * FC + i], tup[P.bpos2[j][b] * FC + i]);
                        L.p = reinterpret_cast<const uint32_t*>(
                            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(L.p), src));
                        L.tab = reinterpret_cast<const uint32_t*>(
                            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(L.tab), src));
                        L.len = __shfl_sync(0xffffffffu, L.len, src);
                        L.bits = __shfl_sync(0xffffffffu, L.bits, src);
                        if (keep && b != b0) keep = gj_bind_member(L, e);
                    }
                } else if (keep) {
                    const uint32_t b0 = minb[i];
                    for (uint32_t b = 0; b < nb && keep; b++) {
                        if (b == b0) continue;
                        const uint32_t v = tup[P.bpos[j][b] * FC + i];
                        keep = GJ_CHECK(G.chk, v < G.n, GJ_SITE_VERTEX, v) &&
                               (P.bdir[j][b] ? gj_list_member(G.ro, G.rn, G.rto, G.rt, v, e)
                                             : gj_list_member(G.fo, G.fn, G.fto, G.ft, v, e));
                    }
                }
                cur += 32;
                if (last) {
                    // members of an aggregated group, or the prefixes a
                    // factorised row stands for (hpre[i] sums their factors)
                    const uint32_t gsz = (EXT && agg && keep) ? grp[i] : 1u;
                    if (keep) {
                        const uint64_t h = hpre[i] * gj_hf(a_new, e);
                        chk += (!DELTA || sg > 0) ? h : 0ull - h;
                    }
                    if (DELTA) {
                        cnt += __popc(__ballot_sync(0xffffffffu, keep && sg > 0)) -
                               __popc(__ballot_sync(0xffffffffu, keep && sg < 0));
                    } else if (EXT && factl) {
                        unsigned long long w = keep ? tup[(j - 1) * FC + i] : 0u;
                        for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                        cnt += w;
                    } else if (EXT && agg) {
                        cnt += __reduce_add_sync(0xffffffffu, keep ? gsz : 0u);
                    } else {
                        cnt += __popc(__ballot_sync(0xffffffffu, keep));
                    }
                    continue;
                }
                if (EXT && factj) {
                    // count the extension and add its factor to its parent's sum
                    if (keep) {
                        atomicAdd(acc_n + i, 1u);
                        atomicAdd(reinterpret_cast<unsigned long long*>(hpre + i),
                                  (unsigned long long)gj_hf(a_new, e));
                    }
                    const uint32_t c1 = __popc(__ballot_sync(0xffffffffu, keep));
                    if (lane == 0) stat_add(A.stats, 3, j + 1, c1);
                    continue;
                }
                const uint32_t mask = __ballot_sync(0xffffffffu, keep);
                if (keep && GJ_CHECK(G.chk, nn + __popc(mask & lt) < FC, GJ_SITE_PREFIX, nn + __popc(mask & lt))) {
                    const uint32_t slot = nn + __popc(mask & lt);
                    for (int p = 0; p < j; p++) nt[p * FC + slot] = tup[p * FC + i];
                    nt[j * FC + slot] = e;
                    if (DELTA) reinterpret_cast<int8_t*>(ws + off_dsg(j + 1, EXT))[slot] = sg;
                }
                nn += __popc(mask);
                if (lane == 0) stat_add(A.stats, 3, j + 1, __popc(mask));
                if (nn >= FT) {
                    // hand the batch to an idle warp when one is waiting
                    bool donate = false;
                    unsigned long long slot = 0;
                    if (A.Q.b && lane == 0 && (A.Q.always || vload(A.Q.idle) > 0u)) {
                        const unsigned long long t = vload64(A.Q.tail);
                        if (vload64(A.Q.seq + (t & (A.Q.cap - 1))) == t && atomicCAS(A.Q.tail, t, t + 1) == t) {
                            slot = t;
                            donate = true;
                        }
                    }
                    donate = __shfl_sync(0xffffffffu, donate, 0);
                    if (donate) {
                        slot = __shfl_sync(0xffffffffu, slot, 0);
                        Bundle& Bd = A.Q.b[slot & (A.Q.cap - 1)];
                        for (int c = 0; c <= j; c++)
                            for (uint32_t i = lane; i < nn; i += 32) Bd.tup[c][i] = nt[c * FC + i];
                        if (DELTA)
                            for (uint32_t i = lane; i < nn; i += 32)
                                Bd.sg[i] = reinterpret_cast<const int8_t*>(ws + off_dsg(j + 1, EXT))[i];
                        if (lane == 0) {
                            Bd.plan = (uint32_t)cur_q;
                            Bd.level = (uint32_t)(j + 1);
                            Bd.n = nn;
                            Bd.c_lo = 0;
                            Bd.c_hi = ~0ull;
                        }
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) atomicExch(A.Q.seq + (slot & (A.Q.cap - 1)), slot + 1);  // publish
                        nn = 0;
                        continue;
                    }
                    descend = true;
                    break;
                }
            }
            __syncwarp();
            if (lane == 0) {
                cur_[j] = cur;
                tot_[j] = tot;
                ip_[j] = ip;
                if (!last) n_[j + 1] = nn;
            }
            __syncwarp();
            if (EXT && factj) {
                // The level-(k-2) batch (or this warp's range of it) is done:
                // every parent with extensions becomes one row of the last
                // level's batch, with its weight (extension count) in the
                // unread column k-2 and its factor sum (the parent's factors
                // times the sum of its extensions' factors) in hpre.
                uint32_t* tK = acc_n - j * FC;
                uint32_t w[2];
                uint64_t f[2];
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t i = lane + 32 * h;
                    w[h] = i < nj ? acc_n[i] : 0u;
                    f[h] = 0;
                    if (w[h]) {
                        uint64_t hh = gj_hq(k);
                        for (uint32_t p = 0; p < (uint32_t)j; p++) hh *= gj_hf(P.order[p], tup[p * FC + i]);
                        f[h] = hh * hpre[i];
                    }
                }
                const uint32_t m0 = __ballot_sync(0xffffffffu, w[0] != 0), m1 = __ballot_sync(0xffffffffu, w[1] != 0);
                __syncwarp();
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const uint32_t i = lane + 32 * h;
                    if (w[h]) {
                        const uint32_t d = h ? __popc(m0) + __popc(m1 & lt) : __popc(m0 & lt);
                        for (uint32_t p = 0; p < (uint32_t)j; p++) tK[p * FC + d] = tup[p * FC + i];
                        tK[j * FC + d] = w[h];
                        hpre[d] = f[h];
                    }
                }
                __syncwarp();
                const uint32_t rows = __popc(m0) + __popc(m1);
                if (lane == 0) n_[j + 1] = rows;
                __syncwarp();
                if (rows) act = j + 1;
                continue;
            }
            if (descend) act = j + 1;
            continue;
        }
        // level j has no proposals left
        if (j + 1 < (int)k && n_[j + 1] > 0) {
            act = j + 1;
            continue;
        }
        if (lane == 0) n_[j] = 0;
        __syncwarp();
        depth = j - 1;
    }
    flush_q();
}

// Seed ranges of each query: slots of the seed index keyed by x0 in [v_lo, v_hi).
__global__ void k_seed_ranges(const Plan* plans, uint32_t nq, GraphView G, uint32_t v_lo, uint32_t v_hi,
                              int64_t* seed_lo, int64_t* seed_n, uint64_t* qbase, uint64_t n_changes = 0,
                              uint32_t chunk = SEED_CHUNK) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    uint64_t base = 0;
    for (uint32_t q = 0; q < nq; q++) {
        int64_t a, b;
        if (plans[q].delta) {
            a = 0;
            b = (int64_t)n_changes;
        } else {
            const int64_t* off = plans[q].seed_dir ? G.ro : G.fo;
            a = off[v_lo];
            b = off[v_hi];
        }
        seed_lo[q] = a;
        seed_n[q] = b - a;
        qbase[q] = base;
        base += ((uint64_t)(b - a) + chunk - 1) / chunk * chunk;
    }
    qbase[nq] = base;
}

}  // namespace

namespace {

// Launch settings of one fused launch: dynamic shared memory, resident
// blocks per SM (the context's cap applied) and the kernel variant.
struct FusedCfg {
    int smem = 0;
    int per_sm = 1;
    bool ext = false;
};

template <bool DELTA, bool EXT>
int fused_cfg_t(gj_ctx* ctx, uint32_t kmax, bool cap, FusedCfg* c) {
    c->smem = (int)(warp_bytes(kmax, DELTA, EXT) * FW);
    if (c->smem > 48 * 1024)  // a per-device attribute: set on every call, as the context's device is current
        GJ_CUDA_TRY(ctx, cudaFuncSetAttribute(k_fused<DELTA, EXT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              c->smem));
    GJ_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->per_sm, k_fused<DELTA, EXT>, FW * 32, c->smem));
    if (cap && ctx->blocks_per_sm && (int)ctx->blocks_per_sm < c->per_sm) c->per_sm = (int)ctx->blocks_per_sm;
    if (c->per_sm < 1) c->per_sm = 1;
    c->ext = EXT;
    return GJ_OK;
}

// The variant for plans[0..n): the extended one if any plan needs it.
template <bool DELTA>
int fused_cfg(gj_ctx* ctx, uint32_t kmax, const Plan* plans, uint32_t n, FusedCfg* c) {
    bool ext = false;
    for (uint32_t q = 0; q < n; q++) ext = ext || gj_plan_ext(plans[q]);
    return ext ? fused_cfg_t<DELTA, true>(ctx, kmax, true, c) : fused_cfg_t<DELTA, false>(ctx, kmax, true, c);
}

// An ordinary launch: the end-of-launch wait of the donation queue waits
// only on warps that have started, so blocks need not be co-resident (the
// grid is one persistent wave on an idle GPU; on a shared one, as in
// serving, later blocks start as earlier launches leave room).
template <bool DELTA, bool EXT>
int launch_t(gj_ctx* ctx, FusedArgs& A, unsigned grid, int smem, cudaStream_t st) {
    k_fused<DELTA, EXT><<<grid, FW * 32, smem, st>>>(A);
    GJ_CUDA_TRY(ctx, cudaGetLastError());
    GJ_LAUNCHED(ctx);
    return GJ_OK;
}

template <bool DELTA>
int launch_fused(gj_ctx* ctx, FusedArgs& A, const FusedCfg& c, cudaStream_t st) {
    const unsigned grid = (unsigned)(ctx->sm_count * c.per_sm);
    return c.ext ? launch_t<DELTA, true>(ctx, A, grid, c.smem, st) : launch_t<DELTA, false>(ctx, A, grid, c.smem, st);
}

}  // namespace

constexpr uint32_t DONATION_CAP = 16384;  // ring slots of a context's queue (power of two)
constexpr uint32_t WAVE_DONATION_CAP = 2048;  // ring slots of a served wave's own queue

// Bytes of a donation queue of cap slots: the bundles, their sequence
// numbers and the counters head, tail, idle and busy, each on its own
// 256-byte line.
static size_t queue_bytes(uint32_t cap) {
    return ((sizeof(Bundle) * (size_t)cap + 255) & ~(size_t)255) +
           ((sizeof(unsigned long long) * (size_t)cap + 255) & ~(size_t)255) + 4 * 256;
}

// Lays a queue of cap slots out at base (256-byte aligned) and enqueues on
// st the reset of its counters and slot sequence numbers; err is the
// launch's give-up flag (a zeroed device word).
static int queue_init(gj_ctx* ctx, char* base, uint32_t cap, unsigned long long* err, cudaStream_t st,
                      DonationQueue* Q) {
    char* p = base + ((sizeof(Bundle) * (size_t)cap + 255) & ~(size_t)255);
    unsigned long long* seq = (unsigned long long*)p;
    unsigned long long* ctr = (unsigned long long*)(p + ((sizeof(unsigned long long) * (size_t)cap + 255) & ~(size_t)255));
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(ctr, 0, 4 * 256, st));
    // failure injection for tests: the queue starts with one busy warp that
    // never leaves, so the end-of-launch wait can only end by its time bound
    // (GJ_E_TIMEOUT)
    if (ctx->fault == GJ_FAULT_WAIT) GJ_CUDA_TRY(ctx, cudaMemsetAsync(ctr + 96, 1, 1, st));
    k_queue_init<<<64, 256, 0, st>>>(seq, cap);
    GJ_LAUNCHED(ctx);
    Q->b = (Bundle*)base;
    Q->cap = cap;
    Q->head = ctr;
    Q->tail = ctr + 32;
    Q->idle = (unsigned int*)(ctr + 64);
    Q->busy = (unsigned int*)(ctr + 96);
    Q->err = err;
    Q->seq = seq;
    Q->always = ctx->donation == 1 ? 1u : 0u;
    if (ctx->donation == 2) Q->b = nullptr;  // off
    return GJ_OK;
}

// Donation queue of a synchronous launch, in scratch slot 4; its give-up
// flag sits on a line of its own after the counters.
static int donation_queue(gj_ctx* ctx, DonationQueue* Q) {
    char* base = nullptr;
    GJ_TRY(gj_scratch(ctx, 4, queue_bytes(DONATION_CAP) + 256, (void**)&base));
    unsigned long long* err = (unsigned long long*)(base + queue_bytes(DONATION_CAP));
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(err, 0, sizeof(*err), ctx->stream));
    return queue_init(ctx, base, DONATION_CAP, err, ctx->stream, Q);
}

static int donation_check(gj_ctx* ctx, const DonationQueue& Q) {
    if (!Q.b) return GJ_OK;
    unsigned long long err = 0;
    GJ_CUDA_TRY(ctx, cudaMemcpy(&err, Q.err, sizeof(err), cudaMemcpyDeviceToHost));
    if (err) {
        gj_set_error(ctx, GJ_E_TIMEOUT, "fused engine: a bounded wait of the work-donation queue expired");
        return GJ_E_TIMEOUT;
    }
    return GJ_OK;
}

int gj_fused_occupancy(gj_ctx* ctx, uint32_t kmax, bool ext) {
    FusedCfg c;
    const int rc = ext ? fused_cfg_t<false, true>(ctx, kmax, false, &c) : fused_cfg_t<false, false>(ctx, kmax, false, &c);
    if (rc != GJ_OK) {
        cudaGetLastError();
        return 1;
    }
    return c.per_sm;
}

size_t gj_fused_async_bytes(uint32_t nq) {
    const size_t plan_bytes = ((sizeof(Plan) * nq) + 255) & ~(size_t)255;
    return plan_bytes + 8 * (4 * (size_t)nq + 2) + 8 * (2 * (size_t)nq) + 8 * 64 + 1024;
}

size_t gj_fused_wave_bytes(uint32_t nq) {
    return ((gj_fused_async_bytes(nq) + 255) & ~(size_t)255) + queue_bytes(WAVE_DONATION_CAP);
}

// Enqueues one fused launch over nq plans on stream st, with all device
// state, its own donation queue included, in dscratch
// (gj_fused_wave_bytes(nq) bytes); nothing waits. On completion *results
// holds nq counts, nq checksums and two flags: the donation queue's bounded
// wait gave up (GJ_E_TIMEOUT), a count passed 2^63 - 1 (GJ_E_OVERFLOW).
int gj_fused_enqueue(gj_ctx* ctx, const GraphView& G, const Plan* hp, uint32_t nq, cudaStream_t st, void* dscratch,
                     unsigned long long** results) {
    const size_t plan_bytes = ((sizeof(Plan) * nq) + 255) & ~(size_t)255;
    char* base = (char*)dscratch;
    Plan* d_plans = (Plan*)base;
    int64_t* seed_lo = (int64_t*)(base + plan_bytes);
    int64_t* seed_n = seed_lo + nq;
    uint64_t* qbase = (uint64_t*)(seed_n + nq);
    unsigned long long* counts_d = (unsigned long long*)(qbase + nq + 1);
    unsigned long long* chks_d = counts_d + nq;
    unsigned long long* flags = chks_d + nq;  // [2] give-up, overflow
    unsigned long long* next = flags + 2;
    unsigned long long* stats = next + 1;
    uint32_t kmax = 2;
    for (uint32_t q = 0; q < nq; q++) kmax = hp[q].k > kmax ? hp[q].k : kmax;
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(d_plans, hp, sizeof(Plan) * nq, cudaMemcpyHostToDevice, st));
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(counts_d, 0, 8 * (2 * (size_t)nq + 3 + NSTAT), st));
    k_seed_ranges<<<1, 1, 0, st>>>(d_plans, nq, G, 0, G.n, seed_lo, seed_n, qbase, 0, ctx->seed_chunk);
    GJ_LAUNCHED(ctx);
    FusedCfg cfg;
    GJ_TRY(fused_cfg<false>(ctx, kmax, hp, nq, &cfg));
    FusedArgs A{G, d_plans, nq, kmax, qbase, seed_lo, seed_n, next, counts_d, chks_d, stats, flags + 1};
    A.chunk = ctx->seed_chunk;
    A.wait_ns = gj_wait_ns(ctx);
    char* qmem = base + ((gj_fused_async_bytes(nq) + 255) & ~(size_t)255);
    GJ_TRY(queue_init(ctx, qmem, WAVE_DONATION_CAP, flags, st, &A.Q));
    GJ_TRY(launch_fused<false>(ctx, A, cfg, st));
    *results = counts_d;
    return GJ_OK;
}

int gj_engine_fused(gj_ctx* ctx, const gj_graph* g, const gj_query* const* qs, uint32_t nq, uint32_t v_lo,
                    uint32_t v_hi, int64_t* counts, uint64_t* checksums) {
    if (nq == 0) return GJ_OK;
    GJ_RANGE("fused launch (%u queries)", nq);
    cudaStream_t st = ctx->stream;
    if (v_hi > g->n) v_hi = g->n;
    if (v_lo > v_hi) v_lo = v_hi;
    uint32_t kmax = 2;
    for (uint32_t q = 0; q < nq; q++) kmax = qs[q]->k > kmax ? qs[q]->k : kmax;
    // device-side arguments in scratch slot 1
    size_t plan_bytes = ((sizeof(Plan) * nq) + 255) & ~(size_t)255;
    size_t need = plan_bytes + 8 * (4 * (size_t)nq + 2) + 8 * (2 * (size_t)nq) + 8 * 64 + 1024;
    char* base = nullptr;
    GJ_TRY(gj_scratch(ctx, 1, need, (void**)&base));
    Plan* d_plans = (Plan*)base;
    int64_t* seed_lo = (int64_t*)(base + plan_bytes);
    int64_t* seed_n = seed_lo + nq;
    uint64_t* qbase = (uint64_t*)(seed_n + nq);
    unsigned long long* counts_d = (unsigned long long*)(qbase + nq + 1);
    unsigned long long* chks_d = counts_d + nq;
    unsigned long long* next = chks_d + nq;
    unsigned long long* stats = next + 1;
    std::vector<Plan> hp(nq);
    for (uint32_t q = 0; q < nq; q++) hp[q] = qs[q]->plan;
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(d_plans, hp.data(), sizeof(Plan) * nq, cudaMemcpyHostToDevice, st));
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(counts_d, 0, 8 * (2 * (size_t)nq + 1 + NSTAT), st));
    GraphView G = g->view();
    k_seed_ranges<<<1, 1, 0, st>>>(d_plans, nq, G, v_lo, v_hi, seed_lo, seed_n, qbase, 0, ctx->seed_chunk);
    GJ_LAUNCHED(ctx);
    // failure injection for tests: counts start just below 2^63
    const uint64_t cbase = ctx->fault == GJ_FAULT_COUNT ? (1ull << 63) - 1024 : 0;
    std::vector<unsigned long long> hbase(nq, cbase);
    if (cbase) GJ_CUDA_TRY(ctx, cudaMemcpyAsync(counts_d, hbase.data(), 8 * (size_t)nq, cudaMemcpyHostToDevice, st));

    FusedCfg cfg;
    GJ_TRY(fused_cfg<false>(ctx, kmax, hp.data(), nq, &cfg));
    FusedArgs A{G, d_plans, nq, kmax, qbase, seed_lo, seed_n, next, counts_d, chks_d, stats, stats + 45};
    A.chunk = ctx->seed_chunk;
    A.wait_ns = gj_wait_ns(ctx);
    GJ_TRY(donation_queue(ctx, &A.Q));
    gj_timer_begin(ctx);
    GJ_TRY(launch_fused<false>(ctx, A, cfg, st));
    gj_timer_end(ctx);
    std::vector<unsigned long long> h(2 * (size_t)nq + 1 + NSTAT);
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), counts_d, 8 * h.size(), cudaMemcpyDeviceToHost, st));
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    GJ_TRY(donation_check(ctx, A.Q));
    GJ_TRY(gj_timer_collect(ctx));
    if (h[2 * (size_t)nq + 1 + 45]) {
        gj_set_error(ctx, GJ_E_OVERFLOW, "fused engine: a match count passed 2^63 - 1");
        return GJ_E_OVERFLOW;
    }
    for (uint32_t q = 0; q < nq; q++) {
        counts[q] = (int64_t)(h[q] - cbase);
        checksums[q] = h[nq + q];
    }
    gj_work_stats& W = ctx->work;
    memset(&W, 0, sizeof(W));
    const unsigned long long* s = h.data() + 2 * nq + 1;
    for (int j = 0; j < 9; j++) {
        W.extended[j] = (int64_t)s[0 * 9 + j];
        W.nbind[j] = (int64_t)s[1 * 9 + j];
        W.proposals[j] = (int64_t)s[2 * 9 + j];
        W.produced[j] = (int64_t)s[3 * 9 + j];
    }
    W.seeds = (int64_t)s[4 * 9 + 0];
    int64_t total = 0;
    for (uint32_t q = 0; q < nq; q++) total += counts[q];
    if (kmax > 0) W.produced[kmax] = total;
    return GJ_OK;
}

// ---------------------------------------------------------------------------
// Variant of the fused launch that allocates nothing (gj_count_noalloc).
//
// The launch's scratch (query plans, seed ranges, per-query counters, the
// shared work counter and the work units) lives in one file-scope device
// array instead of cudaMalloc'd memory. Host code cannot use the array's
// name as a device address, so the address is fetched once per device with
// cudaGetSymbolAddress and cached. All calls on a device share the array.

namespace {

constexpr uint32_t NOALLOC_MAX_QUERIES = 64;
constexpr size_t NOALLOC_SCRATCH_BYTES = 64 * 1024;
constexpr size_t NA_PLANS = 0;
constexpr size_t NA_SEED_LO = ((sizeof(Plan) * NOALLOC_MAX_QUERIES) + 255) & ~(size_t)255;
constexpr size_t NA_SEED_N = NA_SEED_LO + 8 * NOALLOC_MAX_QUERIES;
constexpr size_t NA_QBASE = NA_SEED_N + 8 * NOALLOC_MAX_QUERIES;
constexpr size_t NA_COUNTS = NA_QBASE + 8 * (NOALLOC_MAX_QUERIES + 1);    // zeroed per call from here on
constexpr size_t NA_CHKS = NA_COUNTS + 8 * NOALLOC_MAX_QUERIES;
constexpr size_t NA_NEXT = NA_CHKS + 8 * NOALLOC_MAX_QUERIES;
constexpr size_t NA_STATS = NA_NEXT + 8;
constexpr size_t NA_END = NA_STATS + 8 * NSTAT;
static_assert(NA_END <= NOALLOC_SCRATCH_BYTES, "no-allocation scratch too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on `dev` (which must be current).
int noalloc_scratch(gj_ctx* ctx, int dev, unsigned char** out) {
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        gj_set_error(ctx, GJ_E_INVALID, "gj_count_noalloc: device id out of range");
        return GJ_E_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_addr[dev]) {
        // still this device's memory? (not after the process reset the device)
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, g_noalloc_addr[dev]) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
            at.device != dev) {
            cudaGetLastError();
            g_noalloc_addr[dev] = nullptr;
        }
    }
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            gj_set_error(ctx, GJ_E_CUDA, std::string("gj_count_noalloc: cudaGetSymbolAddress: ") +
                                             cudaGetErrorString(e));
            return GJ_E_CUDA;
        }
        g_noalloc_addr[dev] = p;
    }
    *out = (unsigned char*)g_noalloc_addr[dev];
    return GJ_OK;
}

int count_noalloc(gj_ctx* ctx, const gj_graph* g, const gj_query* const* qs, uint32_t nq, int64_t* counts,
                  uint64_t* checksums) {
    cudaStream_t st = ctx->stream;
    unsigned char* base = nullptr;
    GJ_TRY(noalloc_scratch(ctx, ctx->device, &base));
    Plan* d_plans = (Plan*)(base + NA_PLANS);
    int64_t* seed_lo = (int64_t*)(base + NA_SEED_LO);
    int64_t* seed_n = (int64_t*)(base + NA_SEED_N);
    uint64_t* qbase = (uint64_t*)(base + NA_QBASE);
    unsigned long long* counts_d = (unsigned long long*)(base + NA_COUNTS);
    unsigned long long* chks_d = (unsigned long long*)(base + NA_CHKS);
    unsigned long long* next = (unsigned long long*)(base + NA_NEXT);
    unsigned long long* stats = (unsigned long long*)(base + NA_STATS);
    uint32_t kmax = 2;
    for (uint32_t q = 0; q < nq; q++) {
        kmax = qs[q]->k > kmax ? qs[q]->k : kmax;
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(d_plans + q, &qs[q]->plan, sizeof(Plan), cudaMemcpyHostToDevice, st));
    }
    // the array keeps the previous call's contents: clear the counters this launch adds into
    GJ_CUDA_TRY(ctx, cudaMemsetAsync(base + NA_COUNTS, 0, NA_END - NA_COUNTS, st));
    GraphView G = g->view();
    k_seed_ranges<<<1, 1, 0, st>>>(d_plans, nq, G, 0, g->n, seed_lo, seed_n, qbase, 0, ctx->seed_chunk);
    GJ_LAUNCHED(ctx);
    std::vector<Plan> hp(nq);
    for (uint32_t q = 0; q < nq; q++) hp[q] = qs[q]->plan;
    FusedCfg cfg;
    GJ_TRY(fused_cfg<false>(ctx, kmax, hp.data(), nq, &cfg));
    FusedArgs A{G, d_plans, nq, kmax, qbase, seed_lo, seed_n, next, counts_d, chks_d, stats, stats + 45};
    A.chunk = ctx->seed_chunk;
    A.wait_ns = gj_wait_ns(ctx);
    GJ_TRY(launch_fused<false>(ctx, A, cfg, st));
    static_assert(sizeof(int64_t) == sizeof(unsigned long long), "count width");
    unsigned long long hs[NSTAT];
    std::vector<unsigned long long> hc(2 * (size_t)nq);
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(hc.data(), counts_d, 8 * (size_t)nq, cudaMemcpyDeviceToHost, st));
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(hc.data() + nq, chks_d, 8 * (size_t)nq, cudaMemcpyDeviceToHost, st));
    GJ_CUDA_TRY(ctx, cudaMemcpyAsync(hs, stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
    GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (hs[45]) {
        gj_set_error(ctx, GJ_E_OVERFLOW, "gj_count_noalloc: a match count passed 2^63 - 1");
        return GJ_E_OVERFLOW;
    }
    for (uint32_t q = 0; q < nq; q++) {
        counts[q] = (int64_t)hc[q];
        checksums[q] = hc[nq + q];
    }
    gj_work_stats& W = ctx->work;
    memset(&W, 0, sizeof(W));
    for (int j = 0; j < 9; j++) {
        W.extended[j] = (int64_t)hs[0 * 9 + j];
        W.nbind[j] = (int64_t)hs[1 * 9 + j];
        W.proposals[j] = (int64_t)hs[2 * 9 + j];
        W.produced[j] = (int64_t)hs[3 * 9 + j];
    }
    W.seeds = (int64_t)hs[4 * 9 + 0];
    int64_t total = 0;
    for (uint32_t q = 0; q < nq; q++) total += counts[q];
    W.produced[kmax] = total;
    return GJ_OK;
}

}  // namespace

extern "C" int gj_count_noalloc(gj_graph* g, const gj_query* const* qs, uint32_t nq, int64_t* counts,
                                uint64_t* checksums) {
    if (!g || !qs || !counts || !checksums || nq == 0) return GJ_E_INVALID;
    gj_ctx* ctx = g->ctx;
    if (ctx->server) return GJ_E_INVALID;
    if (nq > NOALLOC_MAX_QUERIES) {
        gj_set_error(ctx, GJ_E_INVALID, "gj_count_noalloc: at most 64 queries per call");
        return GJ_E_INVALID;
    }
    for (uint32_t i = 0; i < nq; i++) {
        if (!qs[i] || qs[i]->ctx != ctx) return GJ_E_INVALID;
        if (qs[i]->ntri && !g->tri.off) {  // building the triangle index would allocate
            gj_set_error(ctx, GJ_E_INVALID, "gj_count_noalloc: build the triangle index first");
            return GJ_E_INVALID;
        }
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) cudaSetDevice(ctx->device);
    int rc = count_noalloc(ctx, g, qs, nq, counts, checksums);
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}

// Delta queries of one batch on the fused engine: all plans (the dQ_i of
// every query) share persistent launches of up to 64 plans; warps take 32
// signed changes at a time from one counter across all plans.
int gj_engine_fused_delta(gj_ctx* ctx, const gj_graph* g, const DeltaBatch& batch, const Plan* plans, uint32_t np,
                          int64_t* counts, uint64_t* checksums) {
    cudaStream_t st = ctx->stream;
    gj_work_stats& W = ctx->work;
    memset(&W, 0, sizeof(W));
    const GraphView G = g->view();
    for (uint32_t c0 = 0; c0 < np; c0 += 64) {
        const uint32_t nc = (np - c0) < 64 ? (np - c0) : 64u;
        char* base = nullptr;
        GJ_TRY(gj_scratch(ctx, 1, gj_fused_async_bytes(nc), (void**)&base));
        const size_t plan_bytes = ((sizeof(Plan) * nc) + 255) & ~(size_t)255;
        Plan* d_plans = (Plan*)base;
        int64_t* seed_lo = (int64_t*)(base + plan_bytes);
        int64_t* seed_n = seed_lo + nc;
        uint64_t* qbase = (uint64_t*)(seed_n + nc);
        unsigned long long* counts_d = (unsigned long long*)(qbase + nc + 1);
        unsigned long long* chks_d = counts_d + nc;
        unsigned long long* next = chks_d + nc;
        unsigned long long* stats = next + 1;
        uint32_t kmax = 2;
        for (uint32_t q = 0; q < nc; q++) kmax = plans[c0 + q].k > kmax ? plans[c0 + q].k : kmax;
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(d_plans, plans + c0, sizeof(Plan) * nc, cudaMemcpyHostToDevice, st));
        GJ_CUDA_TRY(ctx, cudaMemsetAsync(counts_d, 0, 8 * (2 * (size_t)nc + 1 + NSTAT), st));
        // a batch's signed seeds are few and each fans out through hub lists:
        // warps take at most DELTA_CHUNK of them per grab, so more warps start
        const uint32_t chunk = ctx->seed_chunk < DELTA_CHUNK ? ctx->seed_chunk : DELTA_CHUNK;
        k_seed_ranges<<<1, 1, 0, st>>>(d_plans, nc, G, 0, 0, seed_lo, seed_n, qbase, batch.n, chunk);
        GJ_LAUNCHED(ctx);
        FusedCfg cfg;
        GJ_TRY(fused_cfg<true>(ctx, kmax, plans + c0, nc, &cfg));
        FusedArgs A{G, d_plans, nc, kmax, qbase, seed_lo, seed_n, next, counts_d, chks_d, stats, nullptr};
        A.chunk = chunk;
        A.wait_ns = gj_wait_ns(ctx);
        A.D = batch.view;
        A.B = batch;
        GJ_TRY(donation_queue(ctx, &A.Q));
        gj_timer_begin(ctx);
        GJ_TRY(launch_fused<true>(ctx, A, cfg, st));
        gj_timer_end(ctx);
        unsigned long long h[2 * 64 + 1 + NSTAT];
        GJ_CUDA_TRY(ctx, cudaMemcpyAsync(h, counts_d, 8 * (2 * (size_t)nc + 1 + NSTAT), cudaMemcpyDeviceToHost, st));
        GJ_CUDA_TRY(ctx, cudaStreamSynchronize(st));
        GJ_TRY(donation_check(ctx, A.Q));
        for (uint32_t q = 0; q < nc; q++) {
            counts[c0 + q] = (int64_t)h[q];
            checksums[c0 + q] = h[nc + q];
        }
        const unsigned long long* s = h + 2 * nc + 1;
        for (int j = 0; j < 9; j++) {
            W.extended[j] += (int64_t)s[0 * 9 + j];
            W.nbind[j] += (int64_t)s[1 * 9 + j];
            W.proposals[j] += (int64_t)s[2 * 9 + j];
            W.produced[j] += (int64_t)s[3 * 9 + j];
        }
        W.seeds += (int64_t)s[4 * 9 + 0];
    }
    GJ_TRY(gj_timer_collect(ctx));
    return GJ_OK;
}
