// Batched joins: many independent equi-joins in one persistent launch.
//
// Each join j gets a global open-addressing multiset of slots_j = 2^ceil(log2
// (nb_j / load)) slots in the workspace (packed 8-byte slots for int32 keys,
// 16-byte {key, row} slots for int64 keys, the layouts of the non-partitioned
// join). Its work is cut into items: clear items (kClearSlots slots of its
// table each), build items and probe items (`chunk` rows each). The items of
// all joins form one sequence, pulled by a persistent grid with an atomic
// counter, in stages: stage s holds the clear items of join s, then the build
// items of join s-1, then the probe items of join s-2. A build item waits
// (bounded) until all clear items of its join are done, a probe item until
// all build rows of its join are in. So a table is cleared just before it is
// filled (its lines are still in L2), and a join's probes start one stage
// after its builds, with the next join's builds in between to absorb the
// wait. No wait can deadlock: every item waits only on items earlier in the
// sequence, items are claimed in order, waiting items never hold anything an
// earlier item needs, and the grid is no larger than what is resident at once.
// Matches go through the CTA stage to join j's own outputs, reserved on its
// own cursor (d_counts[j]).
//
// Small joins (at most knobs.small_rows build rows) take no global table and
// no items of that sequence: each of their items is one probe chunk that a
// single CTA runs whole, building the join's table in its own shared memory
// from all nb build rows and probing the chunk against it. These items wait
// on nothing and run in a kernel of their own after the persistent one, so
// that kernel keeps its shared-memory footprint (reserving the small joins'
// table in it took L1 from every CTA and made the large joins 1.8x slower).
//
// Launches, all asynchronous and graph-capturable: a one-block setup
// (per-join tables and the stage prefix sums), the persistent join kernel,
// the small joins' kernel (when the knobs allow small joins) and a one-thread
// status fold.
#include "eiger.h"
#include "emit.cuh"
#include "kernels.cuh"

namespace eiger {

namespace {

struct BatchMeta {
    unsigned long long table_off;  // first slot of the join's table
    uint32_t slots;                // power of two (0: no global table)
    uint32_t nci;                  // clear items
    uint32_t nbi;                  // build items
    uint32_t npi;                  // probe items
    uint32_t solo;                 // small join: slots of its shared-memory table (0: none)
};

constexpr int kSoloBytes = 32768;  // shared-memory table of a small join

constexpr unsigned long long kClearSlots = 16384;  // table slots per clear item

struct BatchCtrl {
    unsigned long long next_item;
    unsigned long long total_items;
    unsigned long long total_slots;
    unsigned long long next_solo;   // small joins' items (probe chunks)
    unsigned long long total_solo;
    unsigned int err;
    unsigned int pad;
};

constexpr int kSetupThreads = 1024;
constexpr uint32_t kWaitLimit = 1u << 22;  // polls (with back-off) before giving up

struct alignas(16) WideSlot {
    unsigned long long key;
    unsigned long long row;
};

// One block. Pass 1: per-join slots, item counts and table offsets (prefix
// sum of slots). Pass 2: item counts of the stages (clear items of join s,
// build items of join s-1, probe items of join s-2) and their prefix sums.
__device__ __forceinline__ unsigned long long block_excl_scan64(unsigned long long v, unsigned long long* s_w,
                                                                unsigned long long* total) {
    const unsigned lane = lane_id();
    const int warp = threadIdx.x / kWarp;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    if ((int)lane == kWarp - 1) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = s_w[lane];
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if ((int)lane >= o) t += y;
        }
        s_w[lane] = t;
    }
    __syncthreads();
    const unsigned long long r = (warp ? s_w[warp - 1] : 0ull) + x - v;
    *total = s_w[kWarp - 1];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kSetupThreads)
    batch_setup_kernel(const eiger_join_desc* __restrict__ descs, int k, int chunk, float load,
                       long long small_rows, uint32_t solo_max, unsigned long long max_slots,
                       BatchMeta* __restrict__ meta,
                       unsigned long long* __restrict__ stage_prefix, unsigned* __restrict__ built,
                       unsigned* __restrict__ cleared, unsigned* __restrict__ dup, long long* __restrict__ counts,
                       unsigned long long* __restrict__ solo_prefix, BatchCtrl* __restrict__ bc, int* status) {
    __shared__ unsigned long long s_w[kSetupThreads / kWarp];
    unsigned long long slot_carry = 0, item_carry = 0, solo_carry = 0, total;
    for (int base = 0; base < k; base += kSetupThreads) {
        const int j = base + threadIdx.x;
        unsigned long long slots = 0, solo_items = 0;
        if (j < k) {
            const long long nb = descs[j].nb, np = descs[j].np;
            BatchMeta m{};
            if (nb > 0 && np > 0) {
                const double want = (double)nb / (double)load;
                unsigned long long sl = 64;
                while ((double)sl < want) sl <<= 1;
                if (nb <= small_rows) {
                    // whole per probe chunk, table in shared memory (load at
                    // most 1/2 at the cap: small_rows <= solo_max / 2)
                    m.solo = (uint32_t)(sl < solo_max ? sl : solo_max);
                    solo_items = (unsigned long long)((np + chunk - 1) / chunk);
                } else {
                    slots = sl;
                    m.slots = (uint32_t)sl;
                    m.nci = (uint32_t)((sl + kClearSlots - 1) / kClearSlots);
                    m.nbi = (uint32_t)((nb + chunk - 1) / chunk);
                    m.npi = (uint32_t)((np + chunk - 1) / chunk);
                }
            }
            meta[j] = m;
            built[j] = 0;
            cleared[j] = 0;
            dup[j] = 0;
            counts[j] = 0;
        }
        const unsigned long long off = slot_carry + block_excl_scan64(slots, s_w, &total);
        if (j < k) meta[j].table_off = off;
        slot_carry += total;
        const unsigned long long soff = solo_carry + block_excl_scan64(solo_items, s_w, &total);
        if (j < k) solo_prefix[j] = soff;
        solo_carry += total;
    }
    __syncthreads();
    __threadfence_block();
    const int nstages = k + 2;
    for (int base = 0; base < nstages; base += kSetupThreads) {
        const int st = base + threadIdx.x;
        unsigned long long items = 0;
        if (st < nstages) {
            if (st < k) items += meta[st].nci;
            if (st >= 1 && st - 1 < k) items += meta[st - 1].nbi;
            if (st >= 2) items += meta[st - 2].npi;
        }
        const unsigned long long off = item_carry + block_excl_scan64(items, s_w, &total);
        if (st < nstages) stage_prefix[st] = off;
        item_carry += total;
    }
    if (threadIdx.x == 0) {
        stage_prefix[nstages] = item_carry;
        solo_prefix[k] = solo_carry;
        bc->next_item = 0;
        bc->next_solo = 0;
        bc->err = 0;
        bc->total_slots = slot_carry;
        if (slot_carry > max_slots) {  // tables do not fit: run nothing, report
            bc->total_items = 0;
            bc->total_solo = 0;
            *status = EIGER_ERR_WORKSPACE;
        } else {
            bc->total_items = item_carry;
            bc->total_solo = solo_carry;
            *status = EIGER_OK;
        }
    }
}

// Warp-collective: the stage whose items contain `item` (last s with prefix[s] <= item).
__device__ __forceinline__ int find_join(const unsigned long long* __restrict__ prefix, int k,
                                         unsigned long long item) {
    const unsigned lane = lane_id();
    int lo = 0, hi = k;
    while (hi - lo > 1) {
        const int step = (hi - lo + kWarp - 1) / kWarp;
        const int piv = lo + (int)lane * step;
        const bool le = piv < hi && prefix[piv] <= item;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        const int last = 31 - __clz(m);
        lo = lo + last * step;
        hi = lo + step < hi ? lo + step : hi;
    }
    return lo;
}

// Table words: a global table is read through L2 (other CTAs wrote it), a
// shared-memory one directly.
template <bool SMEM>
__device__ __forceinline__ unsigned long long tab_word(const unsigned long long* p) {
    if constexpr (SMEM)
        return *p;
    else
        return __ldcg(p);
}
template <bool SMEM>
__device__ __forceinline__ ulonglong2 tab_pair(const void* p) {
    if constexpr (SMEM)
        return *static_cast<const ulonglong2*>(p);
    else
        return __ldcg(static_cast<const ulonglong2*>(p));
}

// Inserts build rows [r0, r1) of one join into its table of mask + 1 slots at
// `tab` (global or shared memory): packed (key << 32 | row) words for 32-bit
// keys, chains starting at even slots; {key, row} slots claimed on the row
// word for 64-bit keys. An insert that meets its own key on the path sets
// *dup (32-bit keys; 64-bit joins always walk whole chains).
template <typename InKey, int THREADS>
__device__ __forceinline__ void build_rows(unsigned char* tab, uint32_t mask, const InKey* __restrict__ keys,
                                           long long r0, long long r1, unsigned* dup, unsigned* err) {
    constexpr bool kWide = sizeof(InKey) == 8;
    // the next row's key is loaded before this row's inserts
    InKey knext = r0 + threadIdx.x < r1 ? __ldcs(keys + r0 + threadIdx.x) : InKey(0);
    for (long long r = r0 + threadIdx.x; r < r1; r += THREADS) {
        const InKey key = knext;
        if (r + THREADS < r1) knext = __ldcs(keys + r + THREADS);
        if constexpr (kWide) {
            WideSlot* t = reinterpret_cast<WideSlot*>(tab);
            uint32_t s = (uint32_t)mix64((uint64_t)key) & mask;
            for (uint32_t step = 0;; ++step) {
                if (atomicCAS(&t[s].row, kEmptySlot, (unsigned long long)r) == kEmptySlot) {
                    t[s].key = (unsigned long long)key;
                    break;
                }
                if (step == mask) {
                    atomicOr(err, kErrTableFull);
                    break;
                }
                s = (s + 1) & mask;
            }
        } else {
            unsigned long long* t = reinterpret_cast<unsigned long long*>(tab);
            const uint32_t k32 = (uint32_t)key;
            const unsigned long long v = ((unsigned long long)k32 << 32) | (uint32_t)r;
            uint32_t s = mix32(k32) & mask & ~1u;  // chains start at even slots (pair loads)
            for (uint32_t step = 0;; ++step) {
                const unsigned long long prev = atomicCAS(t + s, kEmptySlot, v);
                if (prev == kEmptySlot) break;
                if ((uint32_t)(prev >> 32) == k32) *dup = 1u;  // an equal key lies on the path
                if (step == mask) {
                    atomicOr(err, kErrTableFull);
                    break;
                }
                s = (s + 1) & mask;
            }
        }
    }
}

// Block-collective: probes rows [r0, r1) of one join against its table (as
// build_rows lays it out) and emits every match through the CTA stage to the
// join's outputs. `first`: no build key repeats (32-bit keys), so each row
// stops at its first match.
template <typename InKey, int THREADS, bool SMEM, int kStage>
__device__ __forceinline__ void probe_rows(const unsigned char* tab, uint32_t mask, bool first,
                                           const InKey* __restrict__ keys, long long r0, long long r1,
                                           Stage<kStage>& st, AggState& agg, const JoinOut& out,
                                           unsigned long long* cursor, unsigned* err) {
    constexpr bool kWide = sizeof(InKey) == 8;
    constexpr int kRows = kStage / (THREADS * 2);  // probe rows per thread per round
    const long long round = (long long)THREADS * kRows;
    // each row's key is loaded one row ahead of its chain walk
    long long rn = r0 + threadIdx.x;
    InKey knext = rn < r1 ? __ldcs(keys + rn) : InKey(0);
    for (long long base = r0; base < r1; base += round) {
#pragma unroll 1
        for (int it = 0; it < kRows; ++it) {
            const long long r = base + (long long)it * THREADS + threadIdx.x;
            const InKey kraw = knext;
            rn = r + THREADS;
            if (rn < r1) knext = __ldcs(keys + rn);
            bool active = r < r1;
            InKey key = 0;
            uint32_t s = 0, steps = 0;
            if (active) {
                key = kraw;
                s = kWide ? (uint32_t)mix64((uint64_t)key) & mask : mix32((uint32_t)key) & mask & ~1u;
            }
            if (first) {
                const unsigned long long* t = reinterpret_cast<const unsigned long long*>(tab);
                bool hit = false;
                uint32_t bi = 0;
                if (active) {
                    for (uint32_t step = 0;; step += 2) {
                        const ulonglong2 v = tab_pair<SMEM>(t + s);
                        if (v.x == kEmptySlot) break;
                        if ((uint32_t)(v.x >> 32) == (uint32_t)key) {
                            hit = true;
                            bi = (uint32_t)v.x;
                            break;
                        }
                        if (v.y == kEmptySlot) break;
                        if ((uint32_t)(v.y >> 32) == (uint32_t)key) {
                            hit = true;
                            bi = (uint32_t)v.y;
                            break;
                        }
                        if (step + 2 > mask) {
                            atomicOr(err, kErrTableFull);
                            break;
                        }
                        s = (s + 2) & mask;
                    }
                }
                emit<false, kStage>(st, agg, hit, bi, (uint32_t)r, out, cursor);
                continue;
            }
            while (__any_sync(0xffffffffu, active)) {
                bool hit = false;
                uint32_t bi = 0;
                if (active) {
                    if constexpr (kWide) {
                        const WideSlot* t = reinterpret_cast<const WideSlot*>(tab);
                        const ulonglong2 v = tab_pair<SMEM>(t + s);
                        if (v.y == kEmptySlot) {
                            active = false;
                        } else {
                            hit = v.x == (unsigned long long)key;
                            bi = (uint32_t)v.y;
                        }
                    } else {
                        const unsigned long long* t = reinterpret_cast<const unsigned long long*>(tab);
                        const unsigned long long v = tab_word<SMEM>(t + s);
                        if (v == kEmptySlot) {
                            active = false;
                        } else {
                            hit = (uint32_t)(v >> 32) == (uint32_t)key;
                            bi = (uint32_t)v;
                        }
                    }
                    if (active) {
                        s = (s + 1) & mask;
                        if (++steps > mask) {
                            atomicOr(err, kErrTableFull);
                            active = false;
                        }
                    }
                }
                emit<false, kStage>(st, agg, hit, bi, (uint32_t)r, out, cursor);
            }
        }
        if (stage_nearly_full(st, (unsigned)round)) stage_flush<false, kStage>(st, out, cursor);
    }
    stage_flush<false, kStage>(st, out, cursor);
}

template <typename InKey, int THREADS>
__global__ void __launch_bounds__(THREADS)
    batch_join_kernel(const eiger_join_desc* __restrict__ descs, int k, const BatchMeta* __restrict__ meta,
                      const unsigned long long* __restrict__ stage_prefix, unsigned char* __restrict__ tables,
                      unsigned* __restrict__ built, unsigned* __restrict__ cleared, unsigned* __restrict__ dup,
                      long long* __restrict__ counts, BatchCtrl* bc, int chunk, int* status) {
    constexpr bool kWide = sizeof(InKey) == 8;
    constexpr int kSlotBytes = kWide ? 16 : 8;
    constexpr int kRows = 2;                   // probe rows per thread per round
    constexpr int kStage = THREADS * kRows * 2;
    __shared__ Stage<kStage> st;
    __shared__ unsigned long long s_item;
    __shared__ int s_stage;
    __shared__ int s_ready;
    const unsigned lane = lane_id();
    AggState agg{0ull, 0ull};
    if (threadIdx.x == 0) st.count = 0;
    const unsigned long long total = bc->total_items;

    for (;;) {
        if (threadIdx.x < kWarp) {
            unsigned long long it = 0;
            if (lane == 0) it = atomicAdd(&bc->next_item, 1ull);
            it = __shfl_sync(0xffffffffu, it, 0);
            const int sg = it < total ? find_join(stage_prefix, k + 2, it) : 0;
            if (lane == 0) {
                s_item = it;
                s_stage = sg;
            }
        }
        __syncthreads();
        const unsigned long long item = s_item;
        const int sg = s_stage;
        if (item >= total) break;
        // decode: the clear items of join sg, then the build items of join
        // sg - 1, then the probe items of join sg - 2
        unsigned long long local = item - stage_prefix[sg];
        int kind = 0, j = sg;
        if (sg < k && local < meta[sg].nci) {
            kind = 0;
        } else {
            if (sg < k) local -= meta[sg].nci;
            j = sg - 1;
            kind = 1;
            if (!(j >= 0 && j < k && local < meta[j].nbi)) {
                if (j >= 0 && j < k) local -= meta[j].nbi;
                j = sg - 2;
                kind = 2;
            }
        }
        const eiger_join_desc d = descs[j];
        const BatchMeta m = meta[j];
        const uint32_t mask = m.slots - 1;
        unsigned char* gtab = tables + m.table_off * kSlotBytes;
        JoinOut out{};
        out.bidx = d.out_bidx;
        out.pidx = d.out_pidx;
        out.capacity = d.capacity > 0 ? (unsigned long long)d.capacity : 0ull;
        unsigned long long* cursor = reinterpret_cast<unsigned long long*>(counts + j);

        if (kind == 0) {
            // ---- clear chunk: kClearSlots slots of the join's table to the empty word
            constexpr int kWords = kWide ? 2 : 1;
            unsigned long long* w = reinterpret_cast<unsigned long long*>(gtab);
            const unsigned long long lo = local * kClearSlots * kWords;
            const unsigned long long hi0 = (local + 1) * kClearSlots * kWords;
            const unsigned long long hi = hi0 < (unsigned long long)m.slots * kWords ? hi0 : (unsigned long long)m.slots * kWords;
            for (unsigned long long i = lo + threadIdx.x; i < hi; i += THREADS) w[i] = kEmptySlot;
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&cleared[j], 1u);
            }
        } else if (kind == 1) {
            // ---- build chunk: wait until the join's table is cleared
            if (threadIdx.x == 0) {
                const volatile unsigned* cp = cleared + j;
                int ok = 0;
                for (uint32_t i = 0; i < kWaitLimit; ++i) {
                    if (*cp >= m.nci) {
                        ok = 1;
                        break;
                    }
                    __nanosleep(i < 64 ? 32 : 256);
                }
                __threadfence();
                if (!ok) atomicOr(&bc->err, kErrInternal);
                s_ready = ok;
            }
            __syncthreads();
            if (!s_ready) continue;
            const long long r0 = (long long)local * chunk;
            const long long r1 = r0 + chunk < d.nb ? r0 + chunk : d.nb;
            build_rows<InKey, THREADS>(gtab, mask, static_cast<const InKey*>(d.build_keys), r0, r1, dup + j,
                                       &bc->err);
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(&built[j], (unsigned)(r1 - r0));
            }
        } else {
            // ---- probe chunk: wait until every build row of join j is in
            if (threadIdx.x == 0) {
                const volatile unsigned* bp = built + j;
                int ok = 0;
                for (uint32_t i = 0; i < kWaitLimit; ++i) {
                    if ((long long)*bp >= d.nb) {
                        ok = 1;
                        break;
                    }
                    __nanosleep(i < 64 ? 32 : 256);
                }
                __threadfence();
                if (!ok) atomicOr(&bc->err, kErrInternal);
                s_ready = ok;
            }
            __syncthreads();
            if (s_ready) {
                const long long r0 = (long long)local * chunk;
                const long long r1 = r0 + chunk < d.np ? r0 + chunk : d.np;
                // a join without duplicate build keys: each lane stops at its first match
                const bool first = !kWide && __ldcg(dup + j) == 0u;
                probe_rows<InKey, THREADS, false, kStage>(gtab, mask, first, static_cast<const InKey*>(d.probe_keys),
                                                          r0, r1, st, agg, out, cursor, &bc->err);
            }
        }
        __syncthreads();
    }
    (void)status;  // device errors are folded in by batch_status_kernel
}

// The small joins: a grid of CTAs pulls their items (join j, probe chunk c)
// from a counter; per item the CTA clears its shared-memory table, inserts all
// of join j's build rows, and probes chunk c against it. No item waits on
// another, so the grid may be any size.
template <typename InKey, int THREADS>
__global__ void __launch_bounds__(THREADS)
    batch_small_kernel(const eiger_join_desc* __restrict__ descs, int k, const BatchMeta* __restrict__ meta,
                       const unsigned long long* __restrict__ solo_prefix, long long* __restrict__ counts,
                       BatchCtrl* bc, int chunk) {
    constexpr bool kWide = sizeof(InKey) == 8;
    constexpr int kSlotBytes = kWide ? 16 : 8;
    constexpr int kStage = THREADS * 4;
    extern __shared__ __align__(16) unsigned char s_tab[];  // kSoloBytes
    __shared__ Stage<kStage> st;
    __shared__ unsigned long long s_item;
    __shared__ int s_join;
    __shared__ unsigned s_dup;
    AggState agg{0ull, 0ull};
    if (threadIdx.x == 0) st.count = 0;
    const unsigned long long total = bc->total_solo;
    for (;;) {
        if (threadIdx.x < kWarp) {
            unsigned long long it = 0;
            if (threadIdx.x == 0) it = atomicAdd(&bc->next_solo, 1ull);
            it = __shfl_sync(0xffffffffu, it, 0);
            const int j = it < total ? find_join(solo_prefix, k, it) : 0;
            if (threadIdx.x == 0) {
                s_item = it;
                s_join = j;
                s_dup = 0;
            }
        }
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= total) break;
        const int j = s_join;
        const eiger_join_desc d = descs[j];
        const uint32_t slots = meta[j].solo;  // power of two, at most kSoloBytes / kSlotBytes
        unsigned long long* w = reinterpret_cast<unsigned long long*>(s_tab);
        for (uint32_t i = threadIdx.x; i < slots * (kSlotBytes / 8); i += THREADS) w[i] = kEmptySlot;
        __syncthreads();
        build_rows<InKey, THREADS>(s_tab, slots - 1, static_cast<const InKey*>(d.build_keys), 0, d.nb, &s_dup,
                                   &bc->err);
        __syncthreads();
        const bool first = !kWide && s_dup == 0;
        const long long r0 = (long long)(item - solo_prefix[j]) * chunk;
        const long long r1 = r0 + chunk < d.np ? r0 + chunk : d.np;
        JoinOut out{};
        out.bidx = d.out_bidx;
        out.pidx = d.out_pidx;
        out.capacity = d.capacity > 0 ? (unsigned long long)d.capacity : 0ull;
        probe_rows<InKey, THREADS, true, kStage>(s_tab, slots - 1, first, static_cast<const InKey*>(d.probe_keys),
                                                 r0, r1, st, agg, out,
                                                 reinterpret_cast<unsigned long long*>(counts + j), &bc->err);
        __syncthreads();
    }
}

// Folds the device error flags into the caller's status word.
__global__ void batch_status_kernel(const BatchCtrl* __restrict__ bc, int* status) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *status == EIGER_OK) {
        if (bc->err & kErrTableFull)
            *status = EIGER_ERR_TABLE_FULL;
        else if (bc->err)
            *status = EIGER_ERR_INTERNAL;
    }
}

template <typename Kern>
int resident_grid(Kern kern, int threads, size_t smem, const DevInfo& di) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return di.sms * per_sm;
}

template <typename InKey, int THREADS>
cudaError_t launch_batch(const eiger_join_desc* d_descs, int k, const BatchLayout& L, long long* d_counts,
                         int chunk, bool small, int* d_status, const DevInfo& di, cudaStream_t stream) {
    auto kern = batch_join_kernel<InKey, THREADS>;
    // Persistent grid no larger than what is resident at once (probe items may
    // wait for build items held by other CTAs).
    const int grid = resident_grid(kern, THREADS, 0, di);
    {
        ProfScope ps("batch_join", 0.0, stream);
        kern<<<grid, THREADS, 0, stream>>>(d_descs, k, reinterpret_cast<const BatchMeta*>(L.meta), L.item_prefix,
                                           L.tables, L.built, L.cleared, L.dup, d_counts,
                                           reinterpret_cast<BatchCtrl*>(L.ctrl), chunk, d_status);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess || !small) return e;
    }
    auto skern = batch_small_kernel<InKey, THREADS>;
    // kSoloBytes plus the static stage: more than the 48 KB a launch gets
    // without opting in. Set once per device, so that later calls, which may
    // be recorded into a CUDA graph, make no attribute call.
    constexpr int kDevSlots = 64;
    static bool opted_in[kDevSlots] = {};
    const bool cached = di.dev >= 0 && di.dev < kDevSlots;
    cudaError_t e;
    if (!(cached && opted_in[di.dev])) {
        if ((e = cudaFuncSetAttribute(skern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSoloBytes)) !=
            cudaSuccess)
            return e;
        if (cached) opted_in[di.dev] = true;
    }
    ProfScope ps("batch_small", 0.0, stream);
    skern<<<resident_grid(skern, THREADS, kSoloBytes, di), THREADS, kSoloBytes, stream>>>(
        d_descs, k, reinterpret_cast<const BatchMeta*>(L.meta), L.solo_prefix, d_counts,
        reinterpret_cast<BatchCtrl*>(L.ctrl), chunk);
    return cudaGetLastError();
}

}  // namespace

BatchLayout batch_layout(Carve& c, int k, unsigned long long total_slots, int slot_bytes) {
    BatchLayout L;
    L.ctrl = c.take<unsigned char>(sizeof(BatchCtrl));
    L.meta = c.take<unsigned char>(sizeof(BatchMeta) * (size_t)(k > 0 ? k : 1));
    L.item_prefix = c.take<unsigned long long>((size_t)k + 3);  // stage prefix sums
    L.solo_prefix = c.take<unsigned long long>((size_t)k + 1);  // small joins' item prefix sums
    L.built = c.take<unsigned>((size_t)(k > 0 ? k : 1));
    L.cleared = c.take<unsigned>((size_t)(k > 0 ? k : 1));
    L.dup = c.take<unsigned>((size_t)(k > 0 ? k : 1));
    L.tables = c.take<unsigned char>((size_t)total_slots * slot_bytes);
    L.table_slots = total_slots;
    return L;
}

cudaError_t batch_run(const eiger_join_desc* d_descs, int k, int dtype, const eiger_batch_knobs& knobs,
                      const BatchLayout& L, long long* d_counts, int* d_status, cudaStream_t stream) {
    DevInfo di;
    cudaError_t e = current_device_info(&di);
    if (e != cudaSuccess) return e;
    BatchCtrl* bc = reinterpret_cast<BatchCtrl*>(L.ctrl);
    BatchMeta* meta = reinterpret_cast<BatchMeta*>(L.meta);
    {
        ProfScope ps("batch_setup", 0.0, stream);
        batch_setup_kernel<<<1, kSetupThreads, 0, stream>>>(d_descs, k, knobs.chunk_rows, knobs.load_factor,
                                                            (long long)knobs.small_rows,
                                                            (uint32_t)(kSoloBytes / (dtype == EIGER_I32 ? 8 : 16)),
                                                            L.table_slots, meta, L.item_prefix, L.built,
                                                            L.cleared, L.dup, d_counts, L.solo_prefix, bc,
                                                            d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const bool small = knobs.small_rows > 0;
    switch (knobs.block_threads) {
        case 128:
            e = dtype == EIGER_I32 ? launch_batch<int32_t, 128>(d_descs, k, L, d_counts, knobs.chunk_rows, small, d_status, di, stream)
                                   : launch_batch<int64_t, 128>(d_descs, k, L, d_counts, knobs.chunk_rows, small, d_status, di, stream);
            break;
        case 256:
            e = dtype == EIGER_I32 ? launch_batch<int32_t, 256>(d_descs, k, L, d_counts, knobs.chunk_rows, small, d_status, di, stream)
                                   : launch_batch<int64_t, 256>(d_descs, k, L, d_counts, knobs.chunk_rows, small, d_status, di, stream);
            break;
        default:
            e = dtype == EIGER_I32 ? launch_batch<int32_t, 512>(d_descs, k, L, d_counts, knobs.chunk_rows, small, d_status, di, stream)
                                   : launch_batch<int64_t, 512>(d_descs, k, L, d_counts, knobs.chunk_rows, small, d_status, di, stream);
            break;
    }
    if (e != cudaSuccess) return e;
    batch_status_kernel<<<1, 32, 0, stream>>>(bc, d_status);
    return cudaGetLastError();
}

}  // namespace eiger
