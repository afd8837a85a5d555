// Partitioned hash join (Sec. 3.2): after both sides are radix-partitioned on
// the same hash bits, partition p of R can only match partition p of S. Each
// build partition fits a hash table in shared memory, so every probe is a
// shared-memory access instead of a random global one.
//
// Work item = (partition p, build chunk c_R, probe chunk c_S). A build
// partition larger than one shared-memory table (duplicate-heavy keys) is cut
// into chunks of at most kBuildCap rows, each joined with the whole probe
// partition; a large probe partition (skew) is cut into chunks of kProbeChunk
// rows so that hot partitions spread over many CTAs. A persistent grid pulls
// items from a global counter. Per item a CTA clears a table of the next power
// of two >= 2 x rows (load factor <= 0.5), inserts the build chunk with
// shared-memory CAS, then streams the probe chunk, walking linear-probe chains
// and emitting matches through the CTA stage (emit.cuh).
//
// Table slots use the low bits of the same mix(key') whose top bits chose the
// partition, so slots are uniform within a partition.
#include "emit.cuh"
#include "kernels.cuh"

namespace eiger {

size_t part_counts_len(int64_t n, int b1, int b2, int passes);
size_t part_scan_blocks(size_t counts_len);

namespace {

constexpr int kJoinThreads = 512;
constexpr int kJoinItems = 2;
constexpr int kJoinStage = 2048;  // >= kJoinThreads * kJoinItems
constexpr uint32_t kBuildCap = 4096;
constexpr uint32_t kProbeChunk = 16384;
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

// One block: item counts per partition, exclusive prefix, total.
__global__ void __launch_bounds__(1024)
    items_kernel(const uint32_t* __restrict__ bstart, const uint32_t* __restrict__ pstart, uint32_t P,
                 unsigned long long* __restrict__ prefix, Ctrl* ctrl) {
    __shared__ unsigned long long s_warp[1024 / kWarp];
    const uint32_t per = (P + blockDim.x - 1) / blockDim.x;
    uint32_t beg = threadIdx.x * per;
    if (beg > P) beg = P;
    uint32_t end = beg + per;
    if (end > P) end = P;
    unsigned long long local = 0;
    for (uint32_t p = beg; p < end; ++p) {
        const uint32_t bs = bstart[p + 1] - bstart[p];
        const uint32_t ps = pstart[p + 1] - pstart[p];
        const unsigned long long c =
            (bs && ps) ? (unsigned long long)((bs + kBuildCap - 1) / kBuildCap) *
                             ((ps + kProbeChunk - 1) / kProbeChunk)
                       : 0ull;
        prefix[p] = c;
        local += c;
    }
    unsigned long long x = local;
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    const int warp = threadIdx.x / kWarp;
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
    unsigned long long run = (warp ? s_warp[warp - 1] : 0ull) + x - local;
    for (uint32_t p = beg; p < end; ++p) {
        const unsigned long long c = prefix[p];
        prefix[p] = run;
        run += c;
    }
    if (threadIdx.x == blockDim.x - 1) {
        prefix[P] = s_warp[kWarp - 1];
        ctrl->nitems = s_warp[kWarp - 1];
    }
}

template <typename KeyT>
struct SmemTable;

// 32-bit keys: one packed 64-bit word per slot, claimed by CAS.
template <>
struct SmemTable<uint32_t> {
    static constexpr size_t kSlotBytes = 8;
    unsigned long long* slot;
    __device__ void bind(unsigned char* smem) { slot = reinterpret_cast<unsigned long long*>(smem); }
    __device__ void clear(uint32_t i) { slot[i] = kEmptySlot; }
    __device__ bool insert(uint32_t s, uint32_t k, uint32_t row) {
        return atomicCAS(slot + s, kEmptySlot, ((unsigned long long)k << 32) | row) == kEmptySlot;
    }
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
    __device__ void clear(uint32_t i) { row[i] = kEmptyRow; }
    __device__ bool insert(uint32_t s, uint64_t k, uint32_t r) {
        if (atomicCAS(row + s, kEmptyRow, r) != kEmptyRow) return false;
        key[s] = k;
        return true;
    }
    __device__ int probe(uint32_t s, uint64_t k, uint32_t& r) const {
        const uint32_t v = row[s];
        if (v == kEmptyRow) return 0;
        r = v;
        return key[s] == k ? 2 : 1;
    }
};

template <typename KeyT, bool AGG>
__global__ void __launch_bounds__(kJoinThreads)
    phj_join_kernel(JoinIn<KeyT> a, JoinOut out, Ctrl* ctrl) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ Stage<kJoinStage> st;
    __shared__ unsigned long long s_item;
    SmemTable<KeyT> tab;
    tab.bind(smem);
    if (threadIdx.x == 0) st.count = 0;
    AggState agg{0ull, 0ull};
    const unsigned long long nitems = ctrl->nitems;

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctrl->next_item, 1ull);
        __syncthreads();
        const unsigned long long item = s_item;
        if (item >= nitems) break;

        // partition p: the last p with prefix[p] <= item
        uint32_t lo = 0, hi = a.P;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (a.item_prefix[mid] <= item) lo = mid; else hi = mid;
        }
        const uint32_t p = lo;
        const uint32_t bs0 = a.bstart[p], bsz = a.bstart[p + 1] - bs0;
        const uint32_t ps0 = a.pstart[p], psz = a.pstart[p + 1] - ps0;
        const uint32_t npc = (psz + kProbeChunk - 1) / kProbeChunk;
        const unsigned long long local = item - a.item_prefix[p];
        const uint32_t bc = (uint32_t)(local / npc), pc = (uint32_t)(local % npc);
        const uint32_t b0 = bs0 + bc * kBuildCap;
        const uint32_t bn = bsz - bc * kBuildCap < kBuildCap ? bsz - bc * kBuildCap : kBuildCap;
        const uint32_t p0 = ps0 + pc * kProbeChunk;
        const uint32_t pn = psz - pc * kProbeChunk < kProbeChunk ? psz - pc * kProbeChunk : kProbeChunk;
        uint32_t tsize = 64;
        while (tsize < 2 * bn) tsize <<= 1;
        const uint32_t tmask = tsize - 1;

        for (uint32_t i = threadIdx.x; i < tsize; i += blockDim.x) tab.clear(i);
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < bn; i += blockDim.x) {
            const KeyT k = a.bkey[b0 + i];
            const uint32_t r = a.bidx[b0 + i];
            uint32_t s = (uint32_t)KeyCodec<KeyT>::hash(k) & tmask;
            for (uint32_t step = 0;; ++step) {
                if (tab.insert(s, k, r)) break;
                if (step == tmask) {
                    atomicOr(&ctrl->err, kErrTableFull);
                    break;
                }
                s = (s + 1) & tmask;
            }
        }
        __syncthreads();

        const uint32_t round = kJoinThreads * kJoinItems;
        for (uint32_t base = 0; base < pn; base += round) {
#pragma unroll 1
            for (int it = 0; it < kJoinItems; ++it) {
                const uint32_t i = base + it * kJoinThreads + threadIdx.x;
                bool active = i < pn;
                KeyT k = 0;
                uint32_t id = 0, s = 0, steps = 0;
                if (active) {
                    k = __ldcs(a.pkey + p0 + i);
                    id = __ldcs(a.pidx + p0 + i);
                    s = (uint32_t)KeyCodec<KeyT>::hash(k) & tmask;
                }
                while (__any_sync(0xffffffffu, active)) {
                    bool hit = false;
                    uint32_t brow = 0;
                    if (active) {
                        const int r = tab.probe(s, k, brow);
                        if (r == 0) {
                            active = false;
                        } else {
                            hit = r == 2;
                            s = (s + 1) & tmask;
                            if (++steps > tmask) active = false;
                        }
                    }
                    emit<AGG, kJoinStage>(st, agg, hit, brow, id, out, ctrl);
                }
            }
            if (!AGG && stage_nearly_full(st, round)) stage_flush<AGG, kJoinStage>(st, out, ctrl);
        }
        __syncthreads();
    }
    if (AGG)
        agg_commit(agg, ctrl);
    else
        stage_flush<AGG, kJoinStage>(st, out, ctrl);
}

template <typename KeyT>
size_t join_smem() {
    return (size_t)kTableMax * SmemTable<KeyT>::kSlotBytes;
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
    auto kern = out.aggregate ? phj_join_kernel<KeyT, true> : phj_join_kernel<KeyT, false>;
    // reads every partitioned (key', row) of both sides once, writes the matches
    const double tuple = (double)(sizeof(KeyT) + sizeof(uint32_t));
    ProfScope ps("phj_join", tuple * (double)(nb + np), stream, match_bytes(out));
    const size_t smem = join_smem<KeyT>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kJoinThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    kern<<<di.sms * per_sm, kJoinThreads, smem, stream>>>(a, out, ctrl);
    return cudaGetLastError();
}

}  // namespace

PhjScratch phj_layout(Carve& c, int64_t nb, int64_t np, const PlanDev& plan) {
    PhjScratch s;
    const int passes = plan.variant == 3 ? 2 : 1;
    const int b1 = plan.bits1, b2 = passes == 2 ? plan.bits2 : 0;
    const size_t kb = plan.key32 ? 4 : 8;
    const size_t P = (size_t)1 << (b1 + b2);
    for (int side = 0; side < 2; ++side) {
        const int64_t n = side == 0 ? nb : np;
        PartSide& ps = s.side[side];
        for (int k = 0; k < 2; ++k) {
            if (k < passes) {
                ps.key[k] = c.take<unsigned char>((size_t)n * kb);
                ps.idx[k] = c.take<uint32_t>((size_t)n);
            } else {
                ps.key[k] = nullptr;
                ps.idx[k] = nullptr;
            }
        }
        ps.counts_len = part_counts_len(n, b1, b2, passes);
        ps.counts = c.take<uint32_t>(ps.counts_len);
        ps.block_sums = c.take<uint32_t>(part_scan_blocks(ps.counts_len));
        ps.total = c.take<uint32_t>(4);
        ps.segs = c.take<SegInfo>((size_t)1 << b1);
        ps.tiles = c.take<Tile>(passes == 2 ? (size_t)((n + kPartTile - 1) / kPartTile) + ((size_t)1 << b1) : 1);
        ps.part_start = c.take<uint32_t>(P + 1);
    }
    s.item_prefix = c.take<unsigned long long>(P + 1);
    return s;
}

cudaError_t phj_run(const JoinArgs& a, const PlanDev& plan, const PhjScratch& s, const JoinOut& out,
                    Ctrl* ctrl, cudaStream_t stream) {
    if (a.nb == 0 || a.np == 0) return cudaSuccess;  // no partition pair can match
    DevInfo di;
    cudaError_t e = current_device_info(&di);
    if (e != cudaSuccess) return e;
    if ((e = partition_side(a.bkeys, a.nb, 0, plan, s.side[0], stream)) != cudaSuccess) return e;
    if ((e = partition_side(a.pkeys, a.np, 1, plan, s.side[1], stream)) != cudaSuccess) return e;
    const int passes = plan.variant == 3 ? 2 : 1;
    const uint32_t P = 1u << (plan.bits1 + (passes == 2 ? plan.bits2 : 0));
    {
        ProfScope ps("phj_items", 24.0 * P, stream);
        items_kernel<<<1, 1024, 0, stream>>>(s.side[0].part_start, s.side[1].part_start, P, s.item_prefix,
                                             ctrl);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return plan.key32 ? launch_join<uint32_t>(s, plan, out, ctrl, di, stream, a.nb, a.np)
                      : launch_join<uint64_t>(s, plan, out, ctrl, di, stream, a.nb, a.np);
}

}  // namespace eiger
