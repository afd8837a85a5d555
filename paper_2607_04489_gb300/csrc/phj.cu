// Partitioned hash join (Sec. 3.2): after both sides are radix-partitioned on
// the same hash bits, partition p of R can only match partition p of S. Each
// build partition fits a hash table in shared memory, so every probe is a
// shared-memory access instead of a random global one.
//
// Work item = (partition p, build chunk c_R, probe chunk c_S). A build
// partition larger than one shared-memory table (duplicate-heavy keys) is cut
// into chunks of at most kBuildCap rows, each joined with the whole probe
// partition; a large probe partition (skew) is cut into chunks of at most
// kProbeChunk rows so that hot partitions spread over many CTAs. The chunks of
// a partition are balanced in size. A persistent grid pulls
// items from a global counter. Per item a CTA clears a table of about three
// slots per build row (load factor <= 1/3), inserts the build chunk with
// shared-memory CAS, then streams the probe chunk, walking linear-probe chains.
// Index pairs leave through per-warp output runs (chunks.cuh), so the probe
// loop has no CTA barrier; payloads, GFTR positions and aggregates go through
// the CTA stage (emit.cuh).
#include "chunks.cuh"
#include "emit.cuh"
#include "kernels.cuh"

namespace eiger {

size_t part_counts_len(int64_t n, int b1, int b2, int passes);
size_t part_scan_blocks(size_t counts_len);

namespace {

constexpr int kJoinThreads = EIGER_JOIN_THREADS;
constexpr int kMaxRows = 8;                       // rows per thread per round (at most)
constexpr int kJoinStage = kJoinThreads * kMaxRows;  // a unique-key round never spills
constexpr uint32_t kBuildCap = EIGER_BUILD_CAP;   // build rows per shared-memory table

// Rows each thread keeps in flight per round (the current round and the next
// one's loads) and CTAs per SM. Index pairs of 32-bit keys: 4 rows, three
// 512-thread CTAs per SM (40 registers), so that while one CTA clears or builds
// its table the others probe theirs (measured on GB300: 16 % faster than two
// CTAs of 8 rows). Payload, position and aggregate outputs keep more live
// state per match and 64-bit keys larger tables: two CTAs per SM, 8 rows for
// 32-bit keys and 4 for 64-bit keys (64 registers).
template <typename KeyT, bool PAIRS>
struct Rows {
    static constexpr bool kLean = sizeof(KeyT) == 4 && PAIRS;
    static constexpr int kN = kLean || sizeof(KeyT) != 4 ? 4 : 8;
    static constexpr int kMinBlocks = (kLean ? 1536 : 1024) / kJoinThreads;
    static constexpr uint32_t kRound = kJoinThreads * kN;
};
#ifndef EIGER_PROBE_CHUNK
#define EIGER_PROBE_CHUNK 32768
#endif
constexpr uint32_t kProbeChunk = EIGER_PROBE_CHUNK;  // probe rows per work item, at most
constexpr uint32_t kTableMax = 2 * kBuildCap;
constexpr uint32_t kEmptyRow = 0xFFFFFFFFu;

template <typename KeyT>
struct JoinIn {
    const KeyT* bkey;
    const uint32_t* bidx;
    const uint32_t* bstart;
    const KeyT* pkey;
    const uint32_t* pidx;
    const uint32_t* pstart;
    const unsigned long long* item_prefix;
    uint32_t P;
};

// Work items of partition p: build chunks x probe chunks (none if a side is empty).
__global__ void items_count_kernel(const uint32_t* __restrict__ bstart, const uint32_t* __restrict__ pstart,
                                   uint32_t P, unsigned long long* __restrict__ count) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const uint32_t bs = bstart[p + 1] - bstart[p];
        const uint32_t ps = pstart[p + 1] - pstart[p];
        count[p] = (bs && ps) ? (unsigned long long)((bs + kBuildCap - 1) / kBuildCap) *
                                    ((ps + kProbeChunk - 1) / kProbeChunk)
                              : 0ull;
    }
}

// One block: exclusive scan of the item counts in place, 4096 per chunk with
// coalesced loads and stores; prefix[P] and ctrl->nitems get the total.
__global__ void __launch_bounds__(1024)
    items_scan_kernel(unsigned long long* __restrict__ prefix, uint32_t P, Ctrl* ctrl) {
    constexpr int kPer = 4;
    constexpr uint32_t kChunk = 1024 * kPer;
    __shared__ unsigned long long s_buf[kChunk];
    __shared__ unsigned long long s_warp[1024 / kWarp];
    const unsigned lane = lane_id();
    const int warp = threadIdx.x / kWarp;
    unsigned long long carry = 0;
    for (uint32_t base = 0; base < P; base += kChunk) {
        for (uint32_t i = threadIdx.x; i < kChunk; i += blockDim.x)
            s_buf[i] = base + i < P ? prefix[base + i] : 0ull;
        __syncthreads();
        unsigned long long local = 0;
#pragma unroll
        for (int j = 0; j < kPer; ++j) local += s_buf[threadIdx.x * kPer + j];
        unsigned long long x = local;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if ((int)lane == kWarp - 1) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long v = s_warp[lane];
#pragma unroll
            for (int o = 1; o < kWarp; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
                if ((int)lane >= o) v += y;
            }
            s_warp[lane] = v;
        }
        __syncthreads();
        unsigned long long run = carry + (warp ? s_warp[warp - 1] : 0ull) + x - local;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const unsigned long long c = s_buf[threadIdx.x * kPer + j];
            s_buf[threadIdx.x * kPer + j] = run;
            run += c;
        }
        carry += s_warp[kWarp - 1];
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < kChunk && base + i < P; i += blockDim.x) prefix[base + i] = s_buf[i];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        prefix[P] = carry;
        ctrl->nitems = carry;
    }
}

template <typename KeyT>
struct SmemTable;

// Home slot of a key in a table of `tsize` slots. The partition was chosen by
// the top bits of a mixed key, so the keys of one partition are a scattered
// subset of the key space; a Fibonacci (multiplicative) hash of the key itself
// spreads them over the table, and a multiply-shift range reduction maps its
// top bits onto [0, tsize).
// Slots come in aligned pairs: the home slot is even, so a probe reads its
// first two candidates with one 16-byte shared load (inserts are ordinary
// linear probing from the same home slot, filling a pair's first slot first).
__device__ __forceinline__ uint32_t slot_hash(uint32_t k) { return k * 0x9E3779B1u; }
__device__ __forceinline__ uint32_t slot_hash(uint64_t k) {
    return (uint32_t)((k * 0x9E3779B97F4A7C15ull) >> 32);
}

template <typename KeyT>
__device__ __forceinline__ uint32_t home_slot(KeyT k, uint32_t tsize) {
    return 2u * (uint32_t)(((unsigned long long)slot_hash(k) * (tsize >> 1)) >> 32);
}

__device__ __forceinline__ uint32_t next_slot(uint32_t s, uint32_t tsize) {
    return s + 1 == tsize ? 0u : s + 1;
}

// 32-bit keys: one packed 64-bit word per slot, claimed by CAS.
template <>
struct SmemTable<uint32_t> {
    static constexpr size_t kSlotBytes = 8;
    unsigned long long* slot;
    __device__ void bind(unsigned char* smem) { slot = reinterpret_cast<unsigned long long*>(smem); }
    // every slot of a table of tsize (a multiple of 2) slots, two per 16-byte store
    __device__ void clear_all(uint32_t tsize) {
        ulonglong2* p = reinterpret_cast<ulonglong2*>(slot);
        for (uint32_t i = threadIdx.x; i < tsize / 2; i += blockDim.x) p[i] = make_ulonglong2(kEmptySlot, kEmptySlot);
    }
    // 1: inserted; 0: slot taken by another key; -1: slot taken by the same key
    __device__ int insert(uint32_t s, uint32_t k, uint32_t row) {
        const unsigned long long prev = atomicCAS(slot + s, kEmptySlot, ((unsigned long long)k << 32) | row);
        if (prev == kEmptySlot) return 1;
        return (uint32_t)(prev >> 32) == k ? -1 : 0;
    }
    // the aligned pair of slots starting at even slot s
    __device__ ulonglong2 pair(uint32_t s) const { return *reinterpret_cast<const ulonglong2*>(slot + s); }
    // 0: empty (chain ends), 1: occupied, other key, 2: match
    __device__ int probe(uint32_t s, uint32_t k, uint32_t& row) const {
        const unsigned long long v = slot[s];
        if (v == kEmptySlot) return 0;
        row = (uint32_t)v;
        return (uint32_t)(v >> 32) == k ? 2 : 1;
    }
};

// 64-bit keys: key array plus row array; the row word is claimed by CAS.
template <>
struct SmemTable<uint64_t> {
    static constexpr size_t kSlotBytes = 12;
    unsigned long long* key;
    uint32_t* row;
    __device__ void bind(unsigned char* smem) {
        key = reinterpret_cast<unsigned long long*>(smem);
        row = reinterpret_cast<uint32_t*>(smem + (size_t)kTableMax * 8);
    }
    __device__ void clear_all(uint32_t tsize) {
        for (uint32_t i = threadIdx.x; i < tsize; i += blockDim.x) row[i] = kEmptyRow;
    }
    // 1: inserted; 0: slot taken (its key may still be in flight, so equal
    // keys are not detected here but by has_equal_keys after the build)
    __device__ int insert(uint32_t s, uint64_t k, uint32_t r) {
        if (atomicCAS(row + s, kEmptyRow, r) != kEmptyRow) return 0;
        key[s] = k;
        return 1;
    }
    // After every insert has completed: 1 when an occupied slot of this
    // thread's share finds its own key earlier in its probe chain, i.e. the
    // table holds a key twice. Linear probing leaves no empty slot between a
    // key's home slot and its slot, so each walk is short and bounded.
    __device__ int has_equal_keys(uint32_t tsize) const;
    __device__ int probe(uint32_t s, uint64_t k, uint32_t& r) const {
        const uint32_t v = row[s];
        if (v == kEmptyRow) return 0;
        r = v;
        return key[s] == k ? 2 : 1;
    }
};

__device__ int SmemTable<uint64_t>::has_equal_keys(uint32_t tsize) const {
    for (uint32_t s = threadIdx.x; s < tsize; s += blockDim.x) {
        if (row[s] == kEmptyRow) continue;
        const uint64_t k = key[s];
        uint32_t t = home_slot(k, tsize);
        for (uint32_t n = 0; t != s && n < tsize; ++n, t = next_slot(t, tsize))
            if (key[t] == k) return 1;
    }
    return 0;
}

// Rows of a probe round: kRows per thread, strided by the block size so every
// load instruction of a warp reads 32 consecutive rows.
template <typename KeyT, int N>
struct RoundRegs {
    KeyT k[N];
    uint32_t id[N];
};

// POS (GFTR): a row is identified by its position in the partitioned arrays
// (pos0 + i), not by the tuple ID stored beside its key.
template <bool POS, typename KeyT, int N>
__device__ __forceinline__ void load_round(RoundRegs<KeyT, N>& r, const KeyT* __restrict__ key,
                                           const uint32_t* __restrict__ idx, uint32_t base,
                                           uint32_t n, uint32_t pos0) {
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const uint32_t i = base + j * kJoinThreads + threadIdx.x;
        if (i < n) {
            r.k[j] = __ldcs(key + i);
            r.id[j] = POS ? pos0 + i : __ldcs(idx + i);
        }
    }
}

// The 128-byte lines of rows [0, n) of a partitioned side (keys, then tuple
// IDs unless rows are identified by position) asked into L2, one line per
// participating thread and step (thread t of `threads`). A hint: no register
// waits on it.
template <bool POS, typename KeyT>
__device__ __forceinline__ void prefetch_rows_l2(const KeyT* key, const uint32_t* idx, uint32_t n, uint32_t t,
                                                 uint32_t threads) {
    const uint32_t klines = (uint32_t)((n * sizeof(KeyT) + 127) / 128);
    const uint32_t ilines = POS ? 0u : (n * 4u + 127) / 128;
    for (uint32_t l = t; l < klines + ilines; l += threads) {
        const char* p = l < klines ? reinterpret_cast<const char*>(key) + (size_t)l * 128
                                   : reinterpret_cast<const char*>(idx) + (size_t)(l - klines) * 128;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
    }
}

constexpr uint32_t kHole = 0xFFFFFFFFu;  // stage position without a match

// Warp-collective: the last partition p in [0, P) with prefix[p] <= item
// (prefix is non-decreasing, prefix[0] = 0). Each step tests 32 evenly spaced
// pivots at once, so 2^15 partitions take three dependent loads.
__device__ __forceinline__ uint32_t find_partition(const unsigned long long* __restrict__ prefix,
                                                   uint32_t P, unsigned long long item) {
    const unsigned lane = lane_id();
    uint32_t lo = 0, hi = P;
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + kWarp - 1) / kWarp;
        const uint32_t piv = lo + lane * step;
        const bool le = piv < hi && prefix[piv] <= item;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        const uint32_t last = 31 - __clz(m);  // lane 0 always qualifies
        lo = lo + last * step;
        hi = lo + step < hi ? lo + step : hi;
    }
    return lo;
}
constexpr int kJoinWarps = kJoinThreads / kWarp;

// Block-collective flush of a positional stage: position j * kJoinThreads + t
// holds the match of thread t's row j, or kHole. Ballots give every match its
// rank within its (row j, warp) group, one scan over the kN x warps group
// counts places the groups, one global atomic reserves the round's output,
// and each warp then writes its group to consecutive output positions.
// Thread t reads back only its own stage entries, so no barrier precedes the
// ballots: the previous round's closing barrier already orders every read of
// s_grp before the new counts are written.
template <int kN>
__device__ __forceinline__ void flush_positional(Stage<kJoinStage>& st, uint32_t* s_grp,
                                                 const JoinOut& out, Ctrl* ctrl) {
    const unsigned lane = lane_id();
    const int w = threadIdx.x / kWarp;
    unsigned ball[kN];
#pragma unroll
    for (int j = 0; j < kN; ++j) {
        ball[j] = __ballot_sync(0xffffffffu, st.b[j * kJoinThreads + threadIdx.x] != kHole);
        if (lane == 0) s_grp[j * kJoinWarps + w] = __popc(ball[j]);
    }
    __syncthreads();
    if (w == 0) {
        // exclusive scan of kN * kJoinWarps group counts, kN * 16 / 32 per lane
        constexpr int kPer = (kN * kJoinWarps + kWarp - 1) / kWarp;
        uint32_t v[kPer], local = 0;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int e = lane * kPer + i;
            v[i] = e < kN * kJoinWarps ? s_grp[e] : 0u;
            local += v[i];
        }
        uint32_t x = local;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        uint32_t run = x - local;
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int e = lane * kPer + i;
            if (e < kN * kJoinWarps) s_grp[e] = run;
            run += v[i];
        }
        const uint32_t total = __shfl_sync(0xffffffffu, x, kWarp - 1);
        if (lane == 0) {
            st.base = total ? atomicAdd(&ctrl->cursor, (unsigned long long)total) : 0ull;
            st.count = (unsigned)(st.base + total <= out.capacity);  // whole round fits
        }
    }
    __syncthreads();
    const unsigned long long base = st.base;
    const bool fits = st.count != 0;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < kN; ++j) {
        const uint32_t i = j * kJoinThreads + threadIdx.x;
        if (ball[j] & (1u << lane)) {
            const unsigned long long pos = base + s_grp[j * kJoinWarps + w] + __popc(ball[j] & lt);
            (void)fits;
            write_match(out, pos, st.b[i], st.p[i]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) st.count = 0;
}

// PAIRS: index pairs only, written through per-warp output runs (chunks.cuh)
// without any CTA barrier in the probe loop; otherwise matches go through the
// CTA stage (emit.cuh), which also gathers payloads, maps positions back to
// tuple IDs (GFTR) or aggregates.
template <typename KeyT, bool AGG, bool PAIRS, bool POS>
__global__ void __launch_bounds__(kJoinThreads, (Rows<KeyT, PAIRS>::kMinBlocks))
    phj_join_kernel(JoinIn<KeyT> a, JoinOut out, PairSink sink, Ctrl* ctrl) {
    extern __shared__ __align__(16) unsigned char smem[];
    // the stage follows the table in dynamic shared memory; index pairs and
    // aggregates use none, so none is allocated for them (shared memory left
    // unreserved serves as L1 cache, which the payload gathers of the
    // aggregate need)
    constexpr bool kStage = !PAIRS && !AGG;
    Stage<kJoinStage>& st = *reinterpret_cast<Stage<kJoinStage>*>(smem + (size_t)kTableMax * SmemTable<KeyT>::kSlotBytes);
    __shared__ uint32_t s_grp[kMaxRows * kJoinWarps];
    __shared__ unsigned long long s_next_item;
    __shared__ uint32_t s_next_part;
    constexpr int kN = Rows<KeyT, PAIRS>::kN;
    constexpr uint32_t kRound = Rows<KeyT, PAIRS>::kRound;
    SmemTable<KeyT> tab;
    tab.bind(smem);
    if (kStage && threadIdx.x == 0) st.count = 0;
    AggState agg{0ull, 0ull};
    WarpChunk wc;
    wc.init();
    const unsigned long long nitems = ctrl->nitems;

    // Work items are claimed one ahead: the claim for the next item is issued
    // when an item starts, and its partition is looked up by warp 0 after the
    // build, so neither round trip sits between two items.
    if (threadIdx.x < kWarp) {
        unsigned long long it0 = 0;
        if (threadIdx.x == 0) it0 = atomicAdd(&ctrl->next_item, 1ull);
        it0 = __shfl_sync(0xffffffffu, it0, 0);
        const uint32_t p0 = it0 < nitems ? find_partition(a.item_prefix, a.P, it0) : 0u;
        if (threadIdx.x == 0) {
            s_next_item = it0;
            s_next_part = p0;
        }
    }
    __syncthreads();

    for (;;) {
        const unsigned long long item = s_next_item;
        const uint32_t p = s_next_part;
        if (item >= nitems) break;
        unsigned long long claim = 0;
        if (threadIdx.x == 0) claim = atomicAdd(&ctrl->next_item, 1ull);

        const uint32_t bs0 = a.bstart[p], bsz = a.bstart[p + 1] - bs0;
        const uint32_t ps0 = a.pstart[p], psz = a.pstart[p + 1] - ps0;
        const uint32_t npc = (psz + kProbeChunk - 1) / kProbeChunk;
        const uint32_t local = (uint32_t)(item - a.item_prefix[p]);  // < items of one partition
        const uint32_t bc = local / npc, pc = local - bc * npc;
        // chunks of a partition are balanced (sizes differ by at most one
        // row), so no item joins a full table with a sliver of probe rows
        const uint32_t nbc = (bsz + kBuildCap - 1) / kBuildCap;
        const uint32_t b_lo = (uint32_t)((unsigned long long)bc * bsz / nbc);
        const uint32_t bn = (uint32_t)((unsigned long long)(bc + 1) * bsz / nbc) - b_lo;
        const uint32_t p_lo = (uint32_t)((unsigned long long)pc * psz / npc);
        const uint32_t pn = (uint32_t)((unsigned long long)(pc + 1) * psz / npc) - p_lo;
        const KeyT* bkey = a.bkey + bs0 + b_lo;
        const uint32_t* bidx = a.bidx + bs0 + b_lo;
        const KeyT* pkey = a.pkey + ps0 + p_lo;
        const uint32_t* pidx = a.pidx + ps0 + p_lo;
        // about three slots per build row (load <= 1/3), at most kTableMax
        uint32_t tsize = (3 * bn + 31) & ~31u;
        if (tsize < 64) tsize = 64;
        if (tsize > kTableMax) tsize = kTableMax;

        // Issue the first build and probe loads before clearing the table, so
        // their latency overlaps the clear.
        RoundRegs<KeyT, kN> cur, nxt;
        const uint32_t bpos0 = bs0 + b_lo, ppos0 = ps0 + p_lo;
        load_round<POS>(nxt, bkey, bidx, 0, bn, bpos0);
        load_round<POS>(cur, pkey, pidx, 0, pn, ppos0);
        tab.clear_all(tsize);
        __syncthreads();
        // Build. An insert that meets its own key proves a duplicate in this
        // chunk; without one, every probe key has at most one match here.
        int dup = 0;
        for (uint32_t bb = 0; bb < bn; bb += kRound) {
            if (bb) load_round<POS>(nxt, bkey, bidx, bb, bn, bpos0);
#pragma unroll
            for (int j = 0; j < kN; ++j) {
                if (bb + j * kJoinThreads + threadIdx.x >= bn) continue;
                uint32_t s = home_slot(nxt.k[j], tsize);
                for (uint32_t step = 0;; ++step) {
                    const int r = tab.insert(s, nxt.k[j], nxt.id[j]);
                    if (r > 0) break;
                    if (r < 0) dup = 1;
                    if (step + 1 == tsize) {
                        atomicOr(&ctrl->err, kErrTableFull);
                        break;
                    }
                    s = next_slot(s, tsize);
                }
            }
        }
        if constexpr (sizeof(KeyT) != 4) {
            __syncthreads();  // every key of the table is written
            dup = tab.has_equal_keys(tsize);
        }
        const bool unique = __syncthreads_or(dup) == 0;
        if (threadIdx.x < kWarp) {  // look up the next item while the probes run
            claim = __shfl_sync(0xffffffffu, claim, 0);
            const uint32_t pn2 = claim < nitems ? find_partition(a.item_prefix, a.P, claim) : 0u;
            if (threadIdx.x == 0) {
                s_next_item = claim;
                s_next_part = pn2;
            }
            // ask L2 for the start of the next partition's build rows and its
            // first probe round, so that item starts on cache hits
            if (claim < nitems) {
                const uint32_t nb0 = a.bstart[pn2], nbn = min(a.bstart[pn2 + 1] - nb0, kBuildCap);
                const uint32_t np0 = a.pstart[pn2], npn = min(a.pstart[pn2 + 1] - np0, kRound);
                prefetch_rows_l2<POS>(a.bkey + nb0, a.bidx + nb0, nbn, threadIdx.x, kWarp);
                prefetch_rows_l2<POS>(a.pkey + np0, a.pidx + np0, npn, threadIdx.x, kWarp);
            }
        }

        for (uint32_t base = 0; base < pn; base += kRound) {
            // the next round's loads are in flight while this round probes,
            // and the round after it is on its way into L2
            if (base + kRound < pn) load_round<POS>(nxt, pkey, pidx, base + kRound, pn, ppos0);
            if (base + 2 * kRound < pn)
                prefetch_rows_l2<POS>(pkey + base + 2 * kRound, pidx + base + 2 * kRound,
                                      min(pn - (base + 2 * kRound), kRound), threadIdx.x, kJoinThreads);
            if (unique) {
                // Fast path: stop at the first match, no collectives per step.
#pragma unroll
                for (int j = 0; j < kN; ++j) {
                    uint32_t brow = kHole;
                    if (base + j * kJoinThreads + threadIdx.x < pn) {
                        const KeyT k = cur.k[j];
                        uint32_t s = home_slot(k, tsize);
                        if constexpr (sizeof(KeyT) == 4) {
                            for (uint32_t step = 0; step < tsize; step += 2) {
                                const ulonglong2 v = tab.pair(s);
                                if (v.x == kEmptySlot) break;
                                if ((uint32_t)(v.x >> 32) == (uint32_t)k) {
                                    brow = (uint32_t)v.x;
                                    break;
                                }
                                if (v.y == kEmptySlot) break;
                                if ((uint32_t)(v.y >> 32) == (uint32_t)k) {
                                    brow = (uint32_t)v.y;
                                    break;
                                }
                                s = s + 2 == tsize ? 0u : s + 2;
                            }
                        } else {
                            for (uint32_t step = 0; step < tsize; ++step) {
                                uint32_t r;
                                const int q = tab.probe(s, k, r);
                                if (q == 0) break;
                                if (q == 2) {
                                    brow = r;
                                    break;
                                }
                                s = next_slot(s, tsize);
                            }
                        }
                    }
                    if constexpr (PAIRS) {
                        warp_emit(wc, sink, brow != kHole, brow, cur.id[j]);
                    } else if constexpr (AGG) {
                        if (brow != kHole) {
                            agg.sum += (unsigned long long)read_pay(out.b.src[0], out.b.bytes[0], brow) +
                                       (unsigned long long)read_pay(out.p.src[0], out.p.bytes[0], cur.id[j]);
                            agg.count += 1;
                        }
                    } else {
                        st.b[j * kJoinThreads + threadIdx.x] = brow;
                        st.p[j * kJoinThreads + threadIdx.x] = cur.id[j];
                    }
                }
                if constexpr (!AGG && !PAIRS) flush_positional<kN>(st, s_grp, out, ctrl);
            } else {
                // General path (duplicate keys): every match of every chain,
                // emitted through the warp-aggregated stage.
#pragma unroll 1
                for (int j = 0; j < kN; ++j) {
                    bool active = base + j * kJoinThreads + threadIdx.x < pn;
                    const KeyT k = cur.k[j];
                    const uint32_t id = cur.id[j];
                    uint32_t s = active ? home_slot(k, tsize) : 0u;
                    uint32_t steps = 0;
                    while (__any_sync(0xffffffffu, active)) {
                        bool hit = false;
                        uint32_t brow = 0;
                        if (active) {
                            const int r = tab.probe(s, k, brow);
                            if (r == 0) {
                                active = false;
                            } else {
                                hit = r == 2;
                                s = next_slot(s, tsize);
                                if (++steps == tsize) active = false;
                            }
                        }
                        if constexpr (PAIRS)
                            warp_emit(wc, sink, hit, brow, id);
                        else
                            emit<AGG, kJoinStage>(st, agg, hit, brow, id, out, &ctrl->cursor);
                    }
                }
                if constexpr (!PAIRS) stage_flush<AGG, kJoinStage>(st, out, &ctrl->cursor);
            }
            cur = nxt;
        }
        __syncthreads();
    }
    if (AGG) agg_commit(agg, ctrl);
    if constexpr (PAIRS) warp_chunk_commit(wc, sink, blockIdx.x * kJoinWarps + threadIdx.x / kWarp);
}

template <typename KeyT>
size_t join_smem(bool stage) {
    return (size_t)kTableMax * SmemTable<KeyT>::kSlotBytes + (stage ? sizeof(Stage<kJoinStage>) : 0);
}

template <typename KeyT>
cudaError_t launch_join(const PhjScratch& s, const PlanDev& plan, const JoinOut& out, Ctrl* ctrl,
                        const DevInfo& di, cudaStream_t stream, int64_t nb, int64_t np) {
    const int passes = plan.variant == 3 ? 2 : 1;
    const int buf = passes - 1;
    JoinIn<KeyT> a;
    a.bkey = static_cast<const KeyT*>(s.side[0].key[buf]);
    a.bidx = s.side[0].idx[buf];
    a.bstart = s.side[0].part_start;
    a.pkey = static_cast<const KeyT*>(s.side[1].key[buf]);
    a.pidx = s.side[1].idx[buf];
    a.pstart = s.side[1].part_start;
    a.item_prefix = s.item_prefix;
    a.P = 1u << (plan.bits1 + (passes == 2 ? plan.bits2 : 0));
    const bool pairs = !out.aggregate && out.bidx && out.pidx && out.b.n == 0 && out.p.n == 0 && !out.b.rowmap &&
                       !out.p.rowmap;
    auto kern = out.aggregate ? (plan.gftr ? phj_join_kernel<KeyT, true, false, true>
                                           : phj_join_kernel<KeyT, true, false, false>)
                : pairs       ? phj_join_kernel<KeyT, false, true, false>
                : plan.gftr   ? phj_join_kernel<KeyT, false, false, true>
                              : phj_join_kernel<KeyT, false, false, false>;
    // reads every partitioned (key', row) of both sides once, writes the matches;
    // the positional aggregate reads keys only, each carried build payload at
    // most once and the probe payload of every match
    const double tuple = (double)(sizeof(KeyT) + sizeof(uint32_t));
    const bool pos_agg = out.aggregate && plan.gftr;
    ProfScope ps("phj_join",
                 pos_agg ? (double)sizeof(KeyT) * (double)(nb + np) + (double)out.b.bytes[0] * (double)nb
                         : tuple * (double)(nb + np),
                 stream, pos_agg ? (double)out.p.bytes[0] : match_bytes(out));
    const size_t smem = join_smem<KeyT>(!pairs && !out.aggregate);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kJoinThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    uint32_t grid = (uint32_t)(di.sms * per_sm);
    if (grid > kMaxOutWarps / kJoinWarps) grid = kMaxOutWarps / kJoinWarps;  // warp records of the pairs sink
    PairSink sink{};
    if (pairs) {
        sink.bidx = out.bidx;
        sink.pidx = out.pidx;
        sink.capacity = out.capacity;
        sink.ovf_b = s.ovf[0];
        sink.ovf_p = s.ovf[1];
        sink.cursor = &ctrl->cursor;
        sink.rec = static_cast<ChunkRec*>(s.rec);
    }
    kern<<<grid, kJoinThreads, smem, stream>>>(a, out, sink, ctrl);
    if ((e = cudaGetLastError()) != cudaSuccess || !pairs) return e;
    return chunk_fix_run(sink, grid * kJoinWarps, s.fix, &ctrl->err, di, stream);
}

}  // namespace

PhjScratch phj_layout(Carve& c, int64_t nb, int64_t np, const PlanDev& plan) {
    PhjScratch s;
    const int passes = plan.variant == 3 ? 2 : 1;
    const int b1 = plan.bits1, b2 = passes == 2 ? plan.bits2 : 0;
    const size_t kb = plan.key32 ? 4 : 8;
    const size_t P = (size_t)1 << (b1 + b2);
    part_side_layout(c, s.side[0], nb, b1, b2, passes, false, kb, plan, 0);
    part_side_layout(c, s.side[1], np, b1, b2, passes, false, kb, plan, 1);
    s.item_prefix = c.take<unsigned long long>(P + 1);
    s.rec = c.take<ChunkRec>(kMaxOutWarps);
    s.ovf[0] = c.take<uint32_t>((size_t)kMaxOutWarps * kOutChunk);
    s.ovf[1] = c.take<uint32_t>((size_t)kMaxOutWarps * kOutChunk);
    s.fix = chunk_fix_layout(c);
    return s;
}

cudaError_t phj_run(const JoinArgs& a, const PlanDev& plan, const PhjScratch& s, const JoinOut& out,
                    Ctrl* ctrl, cudaStream_t stream) {
    if (a.nb == 0 || a.np == 0) return cudaSuccess;  // no partition pair can match
    DevInfo di;
    cudaError_t e = current_device_info(&di);
    if (e != cudaSuccess) return e;
    // the two sides are partitioned concurrently: build on a second stream
    cudaStream_t side;
    if ((e = fork_side(stream, &side)) != cudaSuccess) return e;
    if ((e = partition_side(a.bkeys, a.nb, 0, plan, s.side[0], &out.b, &ctrl->err, side)) != cudaSuccess)
        return e;
    if ((e = partition_side(a.pkeys, a.np, 1, plan, s.side[1], &out.p, &ctrl->err, stream)) != cudaSuccess)
        return e;
    if ((e = join_side(stream, side)) != cudaSuccess) return e;
    const int passes = plan.variant == 3 ? 2 : 1;
    // GFTR: gather from the partitioned copies at the positions the join emits
    const JoinOut o = plan.gftr ? gftr_out(out, s.side[0], s.side[1], passes - 1) : out;
    const uint32_t P = 1u << (plan.bits1 + (passes == 2 ? plan.bits2 : 0));
    {
        ProfScope ps("phj_items", 32.0 * P, stream, 0.0, 2);
        items_count_kernel<<<(P + 255) / 256, 256, 0, stream>>>(s.side[0].part_start, s.side[1].part_start,
                                                               P, s.item_prefix);
        items_scan_kernel<<<1, 1024, 0, stream>>>(s.item_prefix, P, ctrl);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return plan.key32 ? launch_join<uint32_t>(s, plan, o, ctrl, di, stream, a.nb, a.np)
                      : launch_join<uint64_t>(s, plan, o, ctrl, di, stream, a.nb, a.np);
}

}  // namespace eiger
