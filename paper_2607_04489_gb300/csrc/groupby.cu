// Group-by with aggregates (Sec. 3.3), chosen and sized from the HyperLogLog++
// estimate of the number of groups (Sec. 4.2: the group cardinality picks the
// algorithm and sizes the hash table).
//
// Keys travel as 32- or 64-bit offsets from the key minimum (frame of
// reference, Sec. 4.3). Aggregates are 64-bit: SUM modulo 2^64, COUNT, signed
// MIN and MAX, so every result is exact and independent of the order rows
// arrive in.
//
// HASH: one global open-addressing table (linear probing, slots a power of two
// sized from the estimate), keys claimed by CAS and aggregates updated by
// global atomics. While the table is small enough, every CTA first aggregates
// its rows in a private shared-memory copy of the same table (lanes of a warp
// that hit the same slot are combined by their lowest lane before one shared
// atomic), then merges its occupied slots into the global table; compaction
// writes the occupied slots out.
//
// PARTITION: the keys are radix-partitioned on hash bits (Sec. 3.3 hashes
// before partitioning so partitions are even) with the value columns carried
// along (gather from transformed relations), so that each partition's groups
// fit one shared-memory table; a persistent grid takes partitions from a
// global counter, aggregates each in shared memory and writes its groups out.
//
// A key whose offset equals the empty-slot pattern (all ones: only possible
// when the key span is the whole 32- or 64-bit range) is aggregated in one
// extra slot past the table.
#include "kernels.cuh"

namespace eiger {

namespace {

constexpr int kGbThreads = 512;
constexpr uint32_t kPartSlots = 4096;      // shared-memory table of the partition variant
constexpr int kProbeCap = 1 << 20;         // probe steps before a global insert gives up

template <typename KeyT>
struct Empty;
template <>
struct Empty<uint32_t> {
    static constexpr uint32_t v = 0xFFFFFFFFu;
};
template <>
struct Empty<uint64_t> {
    static constexpr unsigned long long v = ~0ull;
};

__device__ __forceinline__ long long agg_init(int op) {
    return op == EIGER_AGG_MIN ? (long long)INT64_MAX : op == EIGER_AGG_MAX ? (long long)INT64_MIN : 0ll;
}

__device__ __forceinline__ long long agg_combine(int op, long long a, long long b) {
    switch (op) {
        case EIGER_AGG_SUM:
        case EIGER_AGG_COUNT:
            return (long long)((unsigned long long)a + (unsigned long long)b);
        case EIGER_AGG_MIN:
            return a < b ? a : b;
        default:
            return a > b ? a : b;
    }
}

// Adds v into *p under op (works on global and shared memory).
__device__ __forceinline__ void agg_atomic(int op, long long* p, long long v) {
    switch (op) {
        case EIGER_AGG_SUM:
        case EIGER_AGG_COUNT:
            atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
            break;
        case EIGER_AGG_MIN:
            atomicMin(p, v);
            break;
        default:
            atomicMax(p, v);
    }
}

// The aggregates of a group-by: per aggregate its op, value column (of the
// caller, or carried through the partitioning) and width.
struct AggSpec {
    int n;
    int op[kMaxCols];
    const void* vals[kMaxCols];
    int bytes[kMaxCols];
};

__device__ __forceinline__ long long agg_value(const AggSpec& s, int a, uint32_t row) {
    if (s.op[a] == EIGER_AGG_COUNT) return 1;
    return s.bytes[a] == 4 ? (long long)__ldcs(static_cast<const int*>(s.vals[a]) + row)
                           : __ldcs(static_cast<const long long*>(s.vals[a]) + row);
}

template <typename KeyT>
__device__ __forceinline__ uint32_t gb_hash(KeyT k) {
    return (uint32_t)KeyCodec<KeyT>::hash(k);
}

__device__ __forceinline__ uint32_t cas_key(uint32_t* p, uint32_t expect, uint32_t v) { return atomicCAS(p, expect, v); }
__device__ __forceinline__ uint64_t cas_key(uint64_t* p, uint64_t expect, uint64_t v) {
    return atomicCAS(reinterpret_cast<unsigned long long*>(p), (unsigned long long)expect, (unsigned long long)v);
}

// ------------------------------------------------------------------ hash variant

template <typename KeyT>
struct GbTable {
    KeyT* keys;         // [slots + 1]; keys[slots] unused (the special slot is flagged below)
    long long* aggs;    // [naggs][stride]
    unsigned* special;  // 1 when the all-ones key has been seen
    unsigned long long slots;
    unsigned long long stride;                // >= slots + 1
    const unsigned long long* slots_dev;      // when set, kernels read the slot count here
};

// Kernels that get a table whose size was decided on the device read it first.
template <typename KeyT>
__device__ __forceinline__ void resolve_slots(GbTable<KeyT>& t) {
    if (t.slots_dev) t.slots = *t.slots_dev;
}

template <typename KeyT>
__global__ void gb_init_kernel(GbTable<KeyT> t, AggSpec s) {
    resolve_slots(t);
    const unsigned long long total = t.slots + 1;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < total;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        t.keys[i] = Empty<KeyT>::v;
        for (int a = 0; a < s.n; ++a) t.aggs[(size_t)a * t.stride + i] = agg_init(s.op[a]);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *t.special = 0;
}

// Global slot of key k (claimed if new); t.slots for the all-ones key; or
// ~0ull when the probe cap is exhausted (error flagged).
template <typename KeyT>
__device__ __forceinline__ unsigned long long gb_global_slot(const GbTable<KeyT>& t, KeyT k, unsigned* err) {
    if (k == Empty<KeyT>::v) {
        atomicOr(t.special, 1u);
        return t.slots;
    }
    const unsigned long long mask = t.slots - 1;
    unsigned long long s = (unsigned long long)KeyCodec<KeyT>::hash(k) & mask;
    for (int step = 0; step < kProbeCap && (unsigned long long)step <= mask; ++step) {
        KeyT cur = t.keys[s];
        if (cur == k) return s;
        if (cur == Empty<KeyT>::v) {
            const KeyT prev = cas_key(t.keys + s, Empty<KeyT>::v, k);
            if (prev == Empty<KeyT>::v || prev == k) return s;
        }
        s = (s + 1) & mask;
    }
    atomicOr(err, kErrTableFull);
    return ~0ull;
}

template <typename InKey, typename KeyT>
__global__ void __launch_bounds__(kGbThreads)
    gb_hash_global_kernel(const InKey* __restrict__ keys, uint32_t n, uint64_t offset, GbTable<KeyT> t, AggSpec s,
                          unsigned* err) {
    const unsigned long long total = t.stride;
    for (unsigned long long rr = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; rr < n;
         rr += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)rr;
        const KeyT k = KeyCodec<KeyT>::encode((int64_t)__ldcs(keys + r), offset);
        const unsigned long long slot = gb_global_slot(t, k, err);
        if (slot == ~0ull) continue;
        for (int a = 0; a < s.n; ++a) agg_atomic(s.op[a], t.aggs + (size_t)a * total + slot, agg_value(s, a, r));
    }
}

// Shared-memory table of one CTA: tsize slots (power of two) plus the special
// slot at index tsize. Layout: keys[tsize + 1], then aggs[naggs][tsize + 1].
template <typename KeyT>
struct SmemGb {
    KeyT* keys;
    long long* aggs;
    uint32_t tsize;
    __device__ void bind(unsigned char* smem, uint32_t ts) {
        tsize = ts;
        keys = reinterpret_cast<KeyT*>(smem);
        aggs = reinterpret_cast<long long*>(smem + align_up((size_t)(ts + 1) * sizeof(KeyT), 8));
    }
    __device__ long long* agg(int a, uint32_t slot) const { return aggs + (size_t)a * (tsize + 1) + slot; }
    __device__ void clear(const AggSpec& s) {
        for (uint32_t i = threadIdx.x; i <= tsize; i += blockDim.x) {
            keys[i] = Empty<KeyT>::v;
            for (int a = 0; a < s.n; ++a) *agg(a, i) = agg_init(s.op[a]);
        }
    }
    // Slot of k (claimed if new), tsize for the all-ones key, or 0xFFFFFFFF
    // when the table is full.
    __device__ uint32_t slot_of(KeyT k) {
        if (k == Empty<KeyT>::v) return tsize;
        const uint32_t mask = tsize - 1;
        uint32_t sl = gb_hash(k) & mask;
        for (uint32_t step = 0; step < tsize; ++step) {
            const KeyT cur = keys[sl];
            if (cur == k) return sl;
            if (cur == Empty<KeyT>::v) {
                const KeyT prev = cas_key(keys + sl, Empty<KeyT>::v, k);
                if (prev == Empty<KeyT>::v || prev == k) return sl;
            }
            sl = (sl + 1) & mask;
        }
        return 0xFFFFFFFFu;
    }
};

template <typename KeyT>
__host__ __device__ constexpr size_t smem_gb_bytes(uint32_t tsize, int naggs) {
    return align_up((size_t)(tsize + 1) * sizeof(KeyT), 8) + (size_t)naggs * (tsize + 1) * 8;
}

// Every aggregate's value of row `row` (0 where !ok), loaded together so that
// the row costs one global-load round trip, not one per aggregate.
__device__ __forceinline__ void agg_values(const AggSpec& s, bool ok, uint32_t row, long long (&v)[kMaxCols]) {
#pragma unroll
    for (int a = 0; a < kMaxCols; ++a) v[a] = (ok && a < s.n) ? agg_value(s, a, row) : 0;
}

// Warp-collective: the lanes with `ok` add their row's aggregates `v` into
// slot `slot` of the CTA table; lanes sharing a slot are first combined by the
// lowest of them (values staged in the warp's scratch), so a hot group costs
// one shared atomic per warp instead of 32.
template <typename KeyT>
__device__ __forceinline__ void warp_aggregate_vals(SmemGb<KeyT>& tab, const AggSpec& s, bool ok, uint32_t slot,
                                                    const long long (&v)[kMaxCols], long long* scratch) {
    const unsigned lane = lane_id();
    const unsigned peers = __match_any_sync(0xffffffffu, ok ? slot : 0xFFFFFFFFu);
    const bool leader = ok && (int)lane == __ffs(peers) - 1;
#pragma unroll
    for (int a = 0; a < kMaxCols; ++a) {
        if (a >= s.n) break;
        scratch[lane] = v[a];
        __syncwarp();
        if (leader) {
            long long acc = v[a];
            unsigned m = peers & ~(1u << lane);
            while (m) {
                const int l = __ffs(m) - 1;
                acc = agg_combine(s.op[a], acc, scratch[l]);
                m &= m - 1;
            }
            agg_atomic(s.op[a], tab.agg(a, slot), acc);
        }
        __syncwarp();
    }
}

template <typename KeyT>
__device__ __forceinline__ void warp_aggregate(SmemGb<KeyT>& tab, const AggSpec& s, bool ok, uint32_t slot,
                                               uint32_t row, long long* scratch) {
    long long v[kMaxCols];
    agg_values(s, ok, row, v);
    warp_aggregate_vals(tab, s, ok, slot, v, scratch);
}

template <typename InKey, typename KeyT>
__global__ void __launch_bounds__(kGbThreads)
    gb_hash_smem_kernel(const InKey* __restrict__ keys, uint32_t n, uint64_t offset, GbTable<KeyT> t, AggSpec s,
                        unsigned* err) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_scratch[kGbThreads];
    __shared__ unsigned s_special;
    SmemGb<KeyT> tab;
    tab.bind(smem, (uint32_t)t.slots);
    tab.clear(s);
    if (threadIdx.x == 0) s_special = 0;
    __syncthreads();
    long long* scratch = s_scratch + (threadIdx.x & ~(kWarp - 1));
    // contiguous row range per CTA, rounds of blockDim rows
    const unsigned long long per = ((unsigned long long)n + gridDim.x - 1) / gridDim.x;
    const unsigned long long lo64 = blockIdx.x * per;
    const uint32_t lo = (uint32_t)(lo64 < n ? lo64 : n);
    const uint32_t hi = (uint32_t)(lo64 + per < n ? lo64 + per : n);
    bool full = false;
    for (unsigned long long base = lo; base < hi; base += kGbThreads) {
        const uint32_t r = (uint32_t)(base + threadIdx.x);
        bool ok = base + threadIdx.x < hi;
        uint32_t slot = 0;
        if (ok) {
            const KeyT k = KeyCodec<KeyT>::encode((int64_t)__ldcs(keys + r), offset);
            slot = tab.slot_of(k);
            if (slot == tab.tsize) s_special = 1;
            if (slot == 0xFFFFFFFFu) {  // cannot happen with the table sized from the estimate; go global
                full = true;
                const unsigned long long g = gb_global_slot(t, k, err);
                if (g != ~0ull)
                    for (int a = 0; a < s.n; ++a)
                        agg_atomic(s.op[a], t.aggs + (size_t)a * t.stride + g, agg_value(s, a, r));
                ok = false;
            }
        }
        warp_aggregate(tab, s, ok, slot, r, scratch);
    }
    (void)full;
    __syncthreads();
    // merge the CTA's groups into the global table
    const unsigned long long total = t.stride;
    for (uint32_t i = threadIdx.x; i <= tab.tsize; i += blockDim.x) {
        unsigned long long g;
        if (i == tab.tsize) {
            if (!s_special) continue;
            atomicOr(t.special, 1u);
            g = t.slots;
        } else {
            const KeyT k = tab.keys[i];
            if (k == Empty<KeyT>::v) continue;
            g = gb_global_slot(t, k, err);
            if (g == ~0ull) continue;
        }
        for (int a = 0; a < s.n; ++a) agg_atomic(s.op[a], t.aggs + (size_t)a * total + g, *tab.agg(a, i));
    }
}

// Output of a group-by: keys in the caller's dtype and one int64 column per aggregate.
struct GbOut {
    void* keys;
    int key_bytes;
    long long* aggs[kMaxCols];
    unsigned long long capacity;
};

__device__ __forceinline__ void write_group(const GbOut& o, unsigned long long pos, int64_t key, const long long* v,
                                            int naggs) {
    if (pos >= o.capacity) return;
    if (o.key_bytes == 4)
        static_cast<int32_t*>(o.keys)[pos] = (int32_t)key;
    else
        static_cast<int64_t*>(o.keys)[pos] = key;
    for (int a = 0; a < naggs; ++a) o.aggs[a][pos] = v[a];
}

// Occupied slots of the global table -> output, reserved per warp.
template <typename KeyT>
__global__ void gb_compact_kernel(GbTable<KeyT> t, AggSpec s, uint64_t offset, GbOut o, Ctrl* ctrl) {
    resolve_slots(t);
    const unsigned long long total = t.slots + 1;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long start = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
    const unsigned long long rounds = (total + stride - 1) / stride;
    for (unsigned long long it = 0; it < rounds; ++it) {
        const unsigned long long i = start + it * stride;
        bool has = false;
        if (i < t.slots)
            has = t.keys[i] != Empty<KeyT>::v;
        else if (i == t.slots)
            has = *t.special != 0;
        const unsigned m = __ballot_sync(0xffffffffu, has);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if ((int)lane_id() == leader) base = atomicAdd(&ctrl->cursor, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (has) {
            const KeyT k = i == t.slots ? Empty<KeyT>::v : t.keys[i];
            long long v[kMaxCols];
            for (int a = 0; a < s.n; ++a) v[a] = t.aggs[(size_t)a * t.stride + i];
            write_group(o, base + __popc(m & lanemask_lt()), (int64_t)((uint64_t)k + offset), v, s.n);
        }
    }
}

// ------------------------------------------------------------------ partition variant

constexpr uint32_t kGbChunk = 65536;  // rows per work item of the partition variant

template <typename KeyT>
struct GbPartIn {
    const KeyT* key;                          // partitioned keys
    const uint32_t* start;                    // [P + 1]
    const unsigned long long* item_prefix;    // [P + 1] work items before each partition
    uint32_t P;
    AggSpec s;                                // value columns: the partitioned copies
};

// One block: work items per partition (row chunks of kGbChunk), their
// exclusive prefix, the item total (ctrl->nitems) and the slots of the spill
// table for the groups of partitions that span several items: at most
// kPartSlots groups each, at load <= 1/2, capped at spill_max.
__global__ void __launch_bounds__(1024)
    gb_items_kernel(const uint32_t* __restrict__ start, uint32_t P, unsigned long long* __restrict__ prefix,
                    Ctrl* ctrl, unsigned long long* spill_slots, unsigned long long spill_max) {
    __shared__ unsigned long long s_w[1024 / kWarp];
    __shared__ unsigned long long s_m[1024 / kWarp];
    const unsigned lane = lane_id();
    const int w = threadIdx.x / kWarp;
    unsigned long long carry = 0, multi = 0;
    for (uint32_t base = 0; base < P; base += blockDim.x) {
        const uint32_t p = base + threadIdx.x;
        unsigned long long items = 0;
        if (p < P) {
            const uint32_t rows = start[p + 1] - start[p];
            items = (rows + kGbChunk - 1) / kGbChunk;
        }
        unsigned long long x = items, m = items > 1;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            const unsigned long long z = __shfl_up_sync(0xffffffffu, m, o);
            if ((int)lane >= o) {
                x += y;
                m += z;
            }
        }
        if ((int)lane == kWarp - 1) {
            s_w[w] = x;
            s_m[w] = m;
        }
        __syncthreads();
        if (w == 0) {
            unsigned long long t = s_w[lane], u = s_m[lane];
#pragma unroll
            for (int o = 1; o < kWarp; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
                const unsigned long long z = __shfl_up_sync(0xffffffffu, u, o);
                if ((int)lane >= o) {
                    t += y;
                    u += z;
                }
            }
            s_w[lane] = t;
            s_m[lane] = u;
        }
        __syncthreads();
        if (p < P) prefix[p] = carry + (w ? s_w[w - 1] : 0ull) + x - items;
        carry += s_w[kWarp - 1];
        multi += s_m[kWarp - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        prefix[P] = carry;
        ctrl->nitems = carry;
        unsigned long long sl = 64;
        while (sl < 2ull * kPartSlots * multi && sl < spill_max) sl <<= 1;
        *spill_slots = multi ? (sl < spill_max ? sl : spill_max) : 0ull;
    }
}

// Warp-collective: the partition of work item `item` (last p with prefix[p] <= item).
__device__ __forceinline__ uint32_t find_item_part(const unsigned long long* __restrict__ prefix, uint32_t P,
                                                   unsigned long long item) {
    const unsigned lane = lane_id();
    uint32_t lo = 0, hi = P;
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + kWarp - 1) / kWarp;
        const uint32_t piv = lo + lane * step;
        const bool le = piv < hi && prefix[piv] <= item;
        const unsigned m = __ballot_sync(0xffffffffu, le);
        lo = lo + (31 - __clz(m)) * step;
        hi = lo + step < hi ? lo + step : hi;
    }
    return lo;
}

// A persistent grid takes work items (a partition's chunk of kGbChunk rows)
// from a global counter and aggregates each in a shared-memory table. A
// partition that is one item writes its groups out directly; the items of a
// larger partition (few groups, many rows) merge their groups into the spill
// table, which is compacted afterwards.
template <typename KeyT>
__global__ void __launch_bounds__(kGbThreads)
    gb_part_kernel(GbPartIn<KeyT> a, GbTable<KeyT> spill, uint64_t offset, GbOut o, Ctrl* ctrl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_scratch[kGbThreads];
    __shared__ uint32_t s_warp[kGbThreads / kWarp];
    __shared__ unsigned s_special;
    __shared__ unsigned long long s_item;
    __shared__ uint32_t s_part;
    __shared__ unsigned long long s_base;
    __shared__ int s_full;
    resolve_slots(spill);
    SmemGb<KeyT> tab;
    tab.bind(smem, kPartSlots);
    long long* scratch = s_scratch + (threadIdx.x & ~(kWarp - 1));
    const unsigned long long nitems = ctrl->nitems;
    for (;;) {
        if (threadIdx.x < kWarp) {
            unsigned long long it = 0;
            if (threadIdx.x == 0) it = atomicAdd(&ctrl->next_item, 1ull);
            it = __shfl_sync(0xffffffffu, it, 0);
            const uint32_t p = it < nitems ? find_item_part(a.item_prefix, a.P, it) : 0u;
            if (threadIdx.x == 0) {
                s_item = it;
                s_part = p;
                s_special = 0;
                s_full = 0;
            }
        }
        tab.clear(a.s);
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= nitems) break;
        const uint32_t p = s_part;
        const unsigned long long c = item - a.item_prefix[p];
        const bool multi = a.item_prefix[p + 1] - a.item_prefix[p] > 1;
        const uint32_t pend = a.start[p + 1];
        const unsigned long long beg = (unsigned long long)a.start[p] + c * kGbChunk;
        const unsigned long long end = beg + kGbChunk < pend ? beg + kGbChunk : pend;
        // each round's key and values are loaded one round ahead, so their
        // round trip overlaps the previous round's table updates
        KeyT kn{};
        long long vn[kMaxCols];
        {
            const bool okn = beg + threadIdx.x < end;
            if (okn) kn = __ldcs(a.key + (uint32_t)(beg + threadIdx.x));
            agg_values(a.s, okn, (uint32_t)(beg + threadIdx.x), vn);
        }
        for (unsigned long long base = beg; base < end; base += kGbThreads) {
            bool ok = base + threadIdx.x < end;
            const KeyT k = kn;
            long long v[kMaxCols];
#pragma unroll
            for (int q = 0; q < kMaxCols; ++q) v[q] = vn[q];
            const unsigned long long nx = base + kGbThreads + threadIdx.x;
            const bool okn = nx < end;
            if (okn) kn = __ldcs(a.key + (uint32_t)nx);
            agg_values(a.s, okn, (uint32_t)nx, vn);
            uint32_t slot = 0;
            if (ok) {
                slot = tab.slot_of(k);
                if (slot == tab.tsize) s_special = 1;
                if (slot == 0xFFFFFFFFu) {
                    s_full = 1;
                    ok = false;
                }
            }
            warp_aggregate_vals(tab, a.s, ok, slot, v, scratch);
        }
        __syncthreads();
        if (s_full) {  // more groups than one table: the host repartitions with more bits
            if (threadIdx.x == 0) atomicOr(&ctrl->err, kErrTableFull);
            __syncthreads();
            continue;
        }
        if (multi) {
            // merge this item's groups into the spill table
            for (uint32_t i = threadIdx.x; i <= kPartSlots; i += blockDim.x) {
                KeyT k;
                if (i == kPartSlots) {
                    if (!s_special) continue;
                    k = Empty<KeyT>::v;
                } else {
                    k = tab.keys[i];
                    if (k == Empty<KeyT>::v) continue;
                }
                const unsigned long long g = gb_global_slot(spill, k, &ctrl->err);
                if (g == ~0ull) continue;
                for (int b = 0; b < a.s.n; ++b)
                    agg_atomic(a.s.op[b], spill.aggs + (size_t)b * spill.stride + g, *tab.agg(b, i));
            }
            __syncthreads();
            continue;
        }
        // compact: block scan of occupancy, one global reservation
        const uint32_t per = (kPartSlots + 1 + kGbThreads - 1) / kGbThreads;
        uint32_t cnt = 0;
        for (uint32_t q = 0; q < per; ++q) {
            const uint32_t i = threadIdx.x * per + q;
            if (i < kPartSlots) cnt += tab.keys[i] != Empty<KeyT>::v;
            else if (i == kPartSlots) cnt += s_special != 0;
        }
        uint32_t x = cnt;
        const unsigned lane = lane_id();
        const int w = threadIdx.x / kWarp;
#pragma unroll
        for (int off = 1; off < kWarp; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, off);
            if ((int)lane >= off) x += y;
        }
        if ((int)lane == kWarp - 1) s_warp[w] = x;
        __syncthreads();
        if (w == 0) {
            uint32_t v = (int)lane < kGbThreads / kWarp ? s_warp[lane] : 0u;
#pragma unroll
            for (int off = 1; off < kWarp; off <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, v, off);
                if ((int)lane >= off) v += y;
            }
            if ((int)lane < kGbThreads / kWarp) s_warp[lane] = v;
            if (lane == kGbThreads / kWarp - 1) s_base = v ? atomicAdd(&ctrl->cursor, (unsigned long long)v) : 0ull;
        }
        __syncthreads();
        unsigned long long pos = s_base + (w ? s_warp[w - 1] : 0u) + (x - cnt);
        for (uint32_t q = 0; q < per; ++q) {
            const uint32_t i = threadIdx.x * per + q;
            bool has = false;
            KeyT k = Empty<KeyT>::v;
            if (i < kPartSlots) {
                k = tab.keys[i];
                has = k != Empty<KeyT>::v;
            } else if (i == kPartSlots) {
                has = s_special != 0;
            }
            if (has) {
                long long v[kMaxCols];
                for (int b = 0; b < a.s.n; ++b) v[b] = *tab.agg(b, i);
                write_group(o, pos++, (int64_t)((uint64_t)k + offset), v, a.s.n);
            }
        }
        __syncthreads();
    }
}

template <typename KeyT>
size_t gb_global_bytes(unsigned long long slots, int naggs) {
    return align_up((size_t)(slots + 1) * sizeof(KeyT), 256) + (size_t)naggs * (slots + 1) * 8 + 256;
}

template <typename InKey, typename KeyT>
cudaError_t gb_hash_run(const GbArgs& g, const GbPlanDev& plan, const GbScratch& sc, const AggSpec& s,
                        const GbOut& o, Ctrl* ctrl, const DevInfo& di, cudaStream_t stream) {
    GbTable<KeyT> t;
    Carve c{static_cast<char*>(sc.table), 0};
    t.keys = c.take<KeyT>(plan.slots + 1);
    t.aggs = c.take<long long>((size_t)s.n * (plan.slots + 1));
    t.special = c.take<unsigned>(1);
    t.slots = plan.slots;
    t.stride = plan.slots + 1;
    t.slots_dev = nullptr;
    cudaError_t e;
    const double kb = (double)sizeof(KeyT);
    {
        ProfScope ps("gb_init", (kb + 8.0 * s.n) * (double)(plan.slots + 1), stream);
        const unsigned long long blocks = (plan.slots + 1 + 255) / 256;
        gb_init_kernel<KeyT><<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, stream>>>(t, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    double vbytes = 0;
    for (int a = 0; a < s.n; ++a) vbytes += s.op[a] == EIGER_AGG_COUNT ? 0 : s.bytes[a];
    const uint32_t n = (uint32_t)g.n;
    const size_t smem = smem_gb_bytes<KeyT>((uint32_t)plan.slots, s.n);
    if (plan.smem) {
        auto kern = gb_hash_smem_kernel<InKey, KeyT>;
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return e;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGbThreads, smem) != cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
        ProfScope ps("gb_hash_smem", ((double)sizeof(InKey) + vbytes) * (double)n, stream);
        kern<<<di.sms * per_sm, kGbThreads, smem, stream>>>(static_cast<const InKey*>(g.keys), n, plan.offset, t, s,
                                                            &ctrl->err);
    } else {
        ProfScope ps("gb_hash_global", ((double)sizeof(InKey) + vbytes) * (double)n, stream);
        gb_hash_global_kernel<InKey, KeyT><<<di.sms * 4, kGbThreads, 0, stream>>>(
            static_cast<const InKey*>(g.keys), n, plan.offset, t, s, &ctrl->err);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ProfScope ps("gb_compact", (kb + 8.0 * s.n) * (double)(plan.slots + 1), stream,
                 (double)sizeof(InKey) + 8.0 * s.n);
    const unsigned long long blocks = (plan.slots + 1 + 255) / 256;
    gb_compact_kernel<KeyT><<<(int)(blocks < 8192 ? blocks : 8192), 256, 0, stream>>>(t, s, plan.offset, o, ctrl);
    return cudaGetLastError();
}

template <typename InKey, typename KeyT>
cudaError_t gb_part_run(const GbArgs& g, const GbPlanDev& plan, const GbScratch& sc, const AggSpec& s,
                        const GbOut& o, Ctrl* ctrl, const DevInfo& di, cudaStream_t stream) {
    // partition the keys with the value columns carried along
    PlanDev pd{};
    pd.variant = plan.bits2 ? EIGER_PHJ2 : EIGER_PHJ1;
    pd.bits1 = plan.bits1;
    pd.bits2 = plan.bits2;
    pd.narrow = sizeof(KeyT) == 4;
    pd.key32 = sizeof(KeyT) == 4;
    pd.dtype = sizeof(InKey) == 4 ? EIGER_I32 : EIGER_I64;
    pd.range.lo = INT64_MIN;
    pd.range.hi = INT64_MAX;
    pd.range.offset = plan.offset;
    pd.check_range = 0;
    pd.no_rows = 1;  // groups are aggregated from the carried columns by position
    ColSide carry{};
    int nc = 0;
    int col_of[kMaxCols];
    for (int a = 0; a < s.n; ++a) {
        col_of[a] = -1;
        if (s.op[a] == EIGER_AGG_COUNT) continue;
        carry.src[nc] = s.vals[a];
        carry.bytes[nc] = s.bytes[a];
        col_of[a] = nc++;
    }
    carry.n = nc;
    pd.gftr = nc > 0;
    pd.ncols[0] = nc;
    for (int q = 0; q < nc; ++q) pd.col_bytes[0][q] = carry.bytes[q];
    cudaError_t e = partition_side(g.keys, g.n, 0, pd, sc.part, &carry, &ctrl->err, stream);
    if (e != cudaSuccess) return e;
    const int buf = plan.bits2 ? 1 : 0;
    const uint32_t P = 1u << (plan.bits1 + plan.bits2);
    GbTable<KeyT> spill;
    {
        Carve c{static_cast<char*>(sc.spill), 0};
        spill.keys = c.take<KeyT>(sc.spill_max + 1);
        spill.aggs = c.take<long long>((size_t)s.n * (sc.spill_max + 1));
        spill.special = c.take<unsigned>(1);
        spill.slots = sc.spill_max;
        spill.stride = sc.spill_max + 1;
        spill.slots_dev = sc.spill_slots;
    }
    {
        ProfScope ps("gb_items", 8.0 * P, stream, 0.0, 2);
        gb_items_kernel<<<1, 1024, 0, stream>>>(sc.part.part_start, P, sc.item_prefix, ctrl, sc.spill_slots,
                                                sc.spill_max);
        gb_init_kernel<KeyT><<<di.sms * 2, 256, 0, stream>>>(spill, s);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    GbPartIn<KeyT> in;
    in.key = static_cast<const KeyT*>(sc.part.key[buf]);
    in.start = sc.part.part_start;
    in.item_prefix = sc.item_prefix;
    in.P = P;
    in.s = s;
    for (int a = 0; a < s.n; ++a)
        if (col_of[a] >= 0) in.s.vals[a] = sc.part.col[buf][col_of[a]];
    auto kern = gb_part_kernel<KeyT>;
    const size_t smem = smem_gb_bytes<KeyT>(kPartSlots, s.n);
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGbThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    double vbytes = 0;
    for (int a = 0; a < s.n; ++a) vbytes += s.op[a] == EIGER_AGG_COUNT ? 0 : s.bytes[a];
    {
        ProfScope ps("gb_part", ((double)sizeof(KeyT) + vbytes) * (double)g.n, stream,
                     (double)sizeof(InKey) + 8.0 * s.n);
        kern<<<di.sms * per_sm, kGbThreads, smem, stream>>>(in, spill, plan.offset, o, ctrl);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    // the groups of multi-item partitions (an empty spill table when there are none)
    ProfScope ps("gb_spill_compact", 0.0, stream);
    gb_compact_kernel<KeyT><<<di.sms * 2, 256, 0, stream>>>(spill, s, plan.offset, o, ctrl);
    return cudaGetLastError();
}

}  // namespace

size_t gb_smem_table_bytes(unsigned long long slots, int naggs, bool key32) {
    if (slots > (1ull << 16)) return ~(size_t)0;  // far beyond any shared-memory budget
    return key32 ? smem_gb_bytes<uint32_t>((uint32_t)slots, naggs) : smem_gb_bytes<uint64_t>((uint32_t)slots, naggs);
}

GbScratch gb_layout(Carve& c, int64_t n, const GbPlanDev& plan, const int* col_bytes, int ncols) {
    GbScratch s{};
    if (plan.variant == EIGER_GB_HASH) {
        const size_t b = plan.key32 ? gb_global_bytes<uint32_t>(plan.slots, plan.naggs)
                                    : gb_global_bytes<uint64_t>(plan.slots, plan.naggs);
        s.table = c.take<unsigned char>(b);
    } else {
        PlanDev pd{};
        pd.gftr = ncols > 0;
        pd.ncols[0] = ncols;
        for (int q = 0; q < ncols; ++q) pd.col_bytes[0][q] = col_bytes[q];
        const int passes = plan.bits2 ? 2 : 1;
        part_side_layout(c, s.part, n, plan.bits1, plan.bits2, passes, false, plan.key32 ? 4 : 8, pd, 0);
        // spill table: each multi-item partition has more than kGbChunk rows and at
        // most kPartSlots groups; load <= 1/2
        const unsigned long long nn = n > 0 ? (unsigned long long)n : 1ull;
        unsigned long long groups = (nn / kGbChunk + 1) * kPartSlots;
        if (groups > nn) groups = nn;
        unsigned long long sl = 64;
        while (sl < 2 * groups) sl <<= 1;
        s.spill_max = sl;
        s.spill = c.take<unsigned char>(plan.key32 ? gb_global_bytes<uint32_t>(sl, plan.naggs)
                                                   : gb_global_bytes<uint64_t>(sl, plan.naggs));
        s.spill_slots = c.take<unsigned long long>(1);
        s.item_prefix = c.take<unsigned long long>(((size_t)1 << (plan.bits1 + plan.bits2)) + 1);
    }
    return s;
}

cudaError_t gb_run(const GbArgs& g, const GbPlanDev& plan, const GbScratch& sc, const GbAggs& aggs, void* out_keys,
                   unsigned long long capacity, Ctrl* ctrl, cudaStream_t stream) {
    if (g.n == 0) return cudaSuccess;
    DevInfo di;
    cudaError_t e = current_device_info(&di);
    if (e != cudaSuccess) return e;
    AggSpec s{};
    s.n = aggs.n;
    GbOut o{};
    o.keys = out_keys;
    o.key_bytes = g.dtype == EIGER_I32 ? 4 : 8;
    o.capacity = capacity;
    for (int a = 0; a < aggs.n; ++a) {
        s.op[a] = aggs.op[a];
        s.vals[a] = aggs.vals[a];
        s.bytes[a] = aggs.bytes[a];
        o.aggs[a] = aggs.out[a];
    }
    const bool i32 = g.dtype == EIGER_I32;
    if (plan.variant == EIGER_GB_HASH) {
        if (plan.key32)
            return i32 ? gb_hash_run<int32_t, uint32_t>(g, plan, sc, s, o, ctrl, di, stream)
                       : gb_hash_run<int64_t, uint32_t>(g, plan, sc, s, o, ctrl, di, stream);
        return gb_hash_run<int64_t, uint64_t>(g, plan, sc, s, o, ctrl, di, stream);
    }
    if (plan.key32)
        return i32 ? gb_part_run<int32_t, uint32_t>(g, plan, sc, s, o, ctrl, di, stream)
                   : gb_part_run<int64_t, uint32_t>(g, plan, sc, s, o, ctrl, di, stream);
    return gb_part_run<int64_t, uint64_t>(g, plan, sc, s, o, ctrl, di, stream);
}

}  // namespace eiger
