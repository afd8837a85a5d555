// Non-partitioned hash join (Sec. 3.2): one open-addressing multiset in global
// memory holding every build row, probed by every probe row.
//
// Two slot layouts:
//  - packed, 8 bytes: (key' << 32) | build_row, with key' the 32-bit key
//    (narrowed int64 offset or raw int32). Claimed by one 64-bit CAS; the
//    all-ones word is the empty slot (build_row never reaches 2^32 - 1).
//  - wide, 16 bytes: {int64 key, build_row}: the row word is claimed by CAS,
//    the key stored after it; build and probe are separate launches, so the
//    probe never sees a half-written slot.
// Linear probing from mix(key') & (slots - 1). The static baseline is the same
// machinery without statistics: raw keys, wide slots for int64, no probe range
// test, load factor 0.5.
//
// Packed tables start every chain at an even slot, so a probe reads its slots
// two at a time with one 16-byte load. The build records whether any key was
// inserted twice: with packed slots an equal key always lies on the later
// insert's path and is seen by its failed CAS. Without duplicates every probe
// key has at most one match, so (outside the static baseline) each lane walks
// its chain alone, stops at its first match and emits once.
#include "emit.cuh"
#include "kernels.cuh"

namespace eiger {

namespace {

constexpr int kBuildThreads = 512;
constexpr int kProbeThreads = 512;
constexpr int kProbeItems = 2;  // rows per thread between stage checks
constexpr int kStage = 2048;    // >= kProbeThreads * kProbeItems

struct alignas(16) WideSlot {
    unsigned long long key;
    unsigned long long row;
};

template <typename InKey>
__global__ void __launch_bounds__(kBuildThreads)
    nphj_build_packed(const InKey* __restrict__ keys, int64_t n, uint64_t offset,
                      unsigned long long* __restrict__ table, uint32_t mask, Ctrl* ctrl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // the next row's key is loaded before this row's inserts (off the critical path)
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    InKey knext = r < n ? __ldcs(keys + r) : InKey(0);
    for (; r < n; r += stride) {
        const InKey kraw = knext;
        if (r + stride < n) knext = __ldcs(keys + r + stride);
        const uint32_t k = KeyCodec<uint32_t>::encode((int64_t)kraw, offset);
        const unsigned long long v = ((unsigned long long)k << 32) | (uint32_t)r;
        uint32_t slot = mix32(k) & mask & ~1u;
        for (uint32_t step = 0;; ++step) {
            const unsigned long long prev = atomicCAS(table + slot, kEmptySlot, v);
            if (prev == kEmptySlot) break;
            if ((uint32_t)(prev >> 32) == k) ctrl->dup = 1u;
            if (step == mask) {
                atomicOr(&ctrl->err, kErrTableFull);
                break;
            }
            slot = (slot + 1) & mask;
        }
    }
}

__global__ void __launch_bounds__(kBuildThreads)
    nphj_build_wide(const int64_t* __restrict__ keys, int64_t n, WideSlot* __restrict__ table,
                    unsigned long long mask, Ctrl* ctrl) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t knext = r < n ? __ldcs(keys + r) : 0;
    for (; r < n; r += stride) {
        const uint64_t k = (uint64_t)knext;
        if (r + stride < n) knext = __ldcs(keys + r + stride);
        unsigned long long slot = mix64(k) & mask;
        for (unsigned long long step = 0;; ++step) {
            if (atomicCAS(&table[slot].row, kEmptySlot, (unsigned long long)r) == kEmptySlot) {
                table[slot].key = k;
                break;
            }
            if (step == mask) {
                atomicOr(&ctrl->err, kErrTableFull);
                break;
            }
            slot = (slot + 1) & mask;
        }
    }
}

template <typename InKey, bool AGG>
__global__ void __launch_bounds__(kProbeThreads)
    nphj_probe_packed(const InKey* __restrict__ keys, int64_t n, KeyRange rng, int check_range,
                      const unsigned long long* __restrict__ table, uint32_t mask, JoinOut out,
                      Ctrl* ctrl, int allow_first_match) {
    __shared__ Stage<kStage> st;
    if (threadIdx.x == 0) st.count = 0;
    __syncthreads();
    AggState agg{0ull, 0ull};
    const uint64_t keep = l2_keep_policy();  // the table stays in L2 while keys and pairs stream
    const bool first_match = allow_first_match && ctrl->dup == 0u;
    const int64_t round = (int64_t)kProbeThreads * kProbeItems;
    const int64_t grid_round = (int64_t)gridDim.x * round;
    // each row's key is loaded one row ahead, so a chain walk waits only on its slots
    int64_t rn = (int64_t)blockIdx.x * round + threadIdx.x;
    InKey knext = rn < n ? __ldcs(keys + rn) : InKey(0);
    for (int64_t base = (int64_t)blockIdx.x * round; base < n; base += grid_round) {
#pragma unroll 1
        for (int it = 0; it < kProbeItems; ++it) {
            const int64_t r = base + (int64_t)it * kProbeThreads + threadIdx.x;
            const InKey kraw = knext;
            rn = it + 1 < kProbeItems ? r + kProbeThreads : base + grid_round + threadIdx.x;
            if (rn < n) knext = __ldcs(keys + rn);
            bool active = r < n;
            uint32_t k = 0, slot = 0, steps = 0;
            if (active) {
                const int64_t key = (int64_t)kraw;
                if (check_range && (key < rng.lo || key > rng.hi)) active = false;
                k = KeyCodec<uint32_t>::encode(key, rng.offset);
                slot = mix32(k) & mask & ~1u;
            }
            if (first_match) {
                // unique build keys: walk the chain alone, two slots per load
                uint32_t bi = 0;
                bool hit = false;
                if (active) {
                    for (uint32_t step = 0;; step += 2) {
                        const ulonglong2 v = ld_keep2(reinterpret_cast<const ulonglong2*>(table + slot), keep);
                        if (v.x == kEmptySlot) break;
                        if ((uint32_t)(v.x >> 32) == k) {
                            hit = true;
                            bi = (uint32_t)v.x;
                            break;
                        }
                        if (v.y == kEmptySlot) break;
                        if ((uint32_t)(v.y >> 32) == k) {
                            hit = true;
                            bi = (uint32_t)v.y;
                            break;
                        }
                        if (step + 2 > mask) {
                            atomicOr(&ctrl->err, kErrTableFull);
                            break;
                        }
                        slot = (slot + 2) & mask;
                    }
                }
                emit<AGG, kStage>(st, agg, hit, bi, (uint32_t)r, out, &ctrl->cursor);
                continue;
            }
            while (__any_sync(0xffffffffu, active)) {
                bool hit = false;
                uint32_t bi = 0;
                if (active) {
                    const unsigned long long s = ld_keep(table + slot, keep);
                    if (s == kEmptySlot) {
                        active = false;
                    } else {
                        if ((uint32_t)(s >> 32) == k) {
                            hit = true;
                            bi = (uint32_t)s;
                        }
                        slot = (slot + 1) & mask;
                        if (++steps > mask) {
                            atomicOr(&ctrl->err, kErrTableFull);
                            active = false;
                        }
                    }
                }
                emit<AGG, kStage>(st, agg, hit, bi, (uint32_t)r, out, &ctrl->cursor);
            }
        }
        if (!AGG && stage_nearly_full(st, (unsigned)round)) stage_flush<AGG, kStage>(st, out, &ctrl->cursor);
    }
    if (AGG)
        agg_commit(agg, ctrl);
    else
        stage_flush<AGG, kStage>(st, out, &ctrl->cursor);
}

template <bool AGG>
__global__ void __launch_bounds__(kProbeThreads)
    nphj_probe_wide(const int64_t* __restrict__ keys, int64_t n, KeyRange rng, int check_range,
                    const WideSlot* __restrict__ table, unsigned long long mask, JoinOut out,
                    Ctrl* ctrl) {
    __shared__ Stage<kStage> st;
    if (threadIdx.x == 0) st.count = 0;
    __syncthreads();
    AggState agg{0ull, 0ull};
    const uint64_t keep = l2_keep_policy();  // the table stays in L2 while keys and pairs stream
    const int64_t round = (int64_t)kProbeThreads * kProbeItems;
    const int64_t grid_round = (int64_t)gridDim.x * round;
    int64_t rn = (int64_t)blockIdx.x * round + threadIdx.x;
    int64_t knext = rn < n ? __ldcs(keys + rn) : 0;
    for (int64_t base = (int64_t)blockIdx.x * round; base < n; base += grid_round) {
#pragma unroll 1
        for (int it = 0; it < kProbeItems; ++it) {
            const int64_t r = base + (int64_t)it * kProbeThreads + threadIdx.x;
            const int64_t kraw = knext;
            rn = it + 1 < kProbeItems ? r + kProbeThreads : base + grid_round + threadIdx.x;
            if (rn < n) knext = __ldcs(keys + rn);
            bool active = r < n;
            uint64_t k = 0;
            unsigned long long slot = 0, steps = 0;
            if (active) {
                const int64_t key = kraw;
                if (check_range && (key < rng.lo || key > rng.hi)) active = false;
                k = (uint64_t)key;
                slot = mix64(k) & mask;
            }
            while (__any_sync(0xffffffffu, active)) {
                bool hit = false;
                uint32_t bi = 0;
                if (active) {
                    const ulonglong2 s = ld_keep2(reinterpret_cast<const ulonglong2*>(table + slot), keep);
                    if (s.y == kEmptySlot) {
                        active = false;
                    } else {
                        if (s.x == k) {
                            hit = true;
                            bi = (uint32_t)s.y;
                        }
                        slot = (slot + 1) & mask;
                        if (++steps > mask) {
                            atomicOr(&ctrl->err, kErrTableFull);
                            active = false;
                        }
                    }
                }
                emit<AGG, kStage>(st, agg, hit, bi, (uint32_t)r, out, &ctrl->cursor);
            }
        }
        if (!AGG && stage_nearly_full(st, (unsigned)round)) stage_flush<AGG, kStage>(st, out, &ctrl->cursor);
    }
    if (AGG)
        agg_commit(agg, ctrl);
    else
        stage_flush<AGG, kStage>(st, out, &ctrl->cursor);
}

template <typename Kern>
int probe_grid(Kern k, int64_t n, const DevInfo& di) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kProbeThreads, 0) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int64_t round = (int64_t)kProbeThreads * kProbeItems;
    int64_t want = (n + round - 1) / round;
    int64_t g = (int64_t)di.sms * per_sm;
    if (want < g) g = want;
    return (int)(g < 1 ? 1 : g);
}

int build_grid(int64_t n, const DevInfo& di) {
    int64_t want = (n + kBuildThreads - 1) / kBuildThreads;
    int64_t cap = (int64_t)di.sms * 4;
    if (want > cap) want = cap;
    return (int)(want < 1 ? 1 : want);
}

}  // namespace

unsigned long long nphj_slots(int64_t nb, float load_factor) {
    double want = (double)(nb > 0 ? nb : 1) / (double)load_factor;
    unsigned long long s = 64;
    while ((double)s < want) s <<= 1;
    return s;
}

NphjScratch nphj_layout(Carve& c, int64_t nb, const PlanDev& plan) {
    NphjScratch s;
    s.slots = nphj_slots(nb, plan.load_factor);
    s.slot_bytes = plan.key32 ? 8 : 16;
    s.table = c.take<unsigned char>(s.slots * (size_t)s.slot_bytes);
    return s;
}

cudaError_t nphj_run(const JoinArgs& a, const PlanDev& plan, const NphjScratch& s,
                     const JoinOut& out, Ctrl* ctrl, cudaStream_t stream) {
    DevInfo di;
    cudaError_t e = current_device_info(&di);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(s.table, 0xFF, s.slots * (size_t)s.slot_bytes, stream);
    if (e != cudaSuccess) return e;
    const bool agg = out.aggregate != 0;
    const double kb = plan.dtype == 0 ? 4.0 : 8.0;
    const double build_bytes = (kb + s.slot_bytes) * (double)a.nb;  // read keys, write slots
    const double probe_bytes = (kb + s.slot_bytes) * (double)a.np;  // read keys, >= one slot each
    const double per_match = match_bytes(out);
    if (s.slot_bytes == 8) {
        const uint32_t mask = (uint32_t)(s.slots - 1);
        auto* table = static_cast<unsigned long long*>(s.table);
        if (a.nb > 0) {
            ProfScope ps("nphj_build", build_bytes, stream);
            if (plan.dtype == 0)
                nphj_build_packed<int32_t><<<build_grid(a.nb, di), kBuildThreads, 0, stream>>>(
                    static_cast<const int32_t*>(a.bkeys), a.nb, plan.range.offset, table, mask, ctrl);
            else
                nphj_build_packed<int64_t><<<build_grid(a.nb, di), kBuildThreads, 0, stream>>>(
                    static_cast<const int64_t*>(a.bkeys), a.nb, plan.range.offset, table, mask, ctrl);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (a.np > 0) {
            ProfScope ps("nphj_probe", probe_bytes, stream, per_match);
            if (plan.dtype == 0) {
                auto kern = agg ? nphj_probe_packed<int32_t, true> : nphj_probe_packed<int32_t, false>;
                kern<<<probe_grid(kern, a.np, di), kProbeThreads, 0, stream>>>(
                    static_cast<const int32_t*>(a.pkeys), a.np, plan.range, plan.check_range, table,
                    mask, out, ctrl, plan.variant != EIGER_STATIC);
            } else {
                auto kern = agg ? nphj_probe_packed<int64_t, true> : nphj_probe_packed<int64_t, false>;
                kern<<<probe_grid(kern, a.np, di), kProbeThreads, 0, stream>>>(
                    static_cast<const int64_t*>(a.pkeys), a.np, plan.range, plan.check_range, table,
                    mask, out, ctrl, plan.variant != EIGER_STATIC);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    } else {
        const unsigned long long mask = s.slots - 1;
        auto* table = static_cast<WideSlot*>(s.table);
        if (a.nb > 0) {
            ProfScope ps("nphj_build", build_bytes, stream);
            nphj_build_wide<<<build_grid(a.nb, di), kBuildThreads, 0, stream>>>(
                static_cast<const int64_t*>(a.bkeys), a.nb, table, mask, ctrl);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (a.np > 0) {
            ProfScope ps("nphj_probe", probe_bytes, stream, per_match);
            auto kern = agg ? nphj_probe_wide<true> : nphj_probe_wide<false>;
            kern<<<probe_grid(kern, a.np, di), kProbeThreads, 0, stream>>>(
                static_cast<const int64_t*>(a.pkeys), a.np, plan.range, plan.check_range, table, mask,
                out, ctrl);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

}  // namespace eiger
