// Batched joins: many independent equi-joins in one persistent launch.
//
// Each join j gets a global open-addressing multiset of slots_j = 2^ceil(log2
// (nb_j / load)) slots in the workspace (packed 8-byte slots for int32 keys,
// 16-byte {key, row} slots for int64 keys, the layouts of the non-partitioned
// join). The work of all joins is cut into items of `chunk` rows: join j
// contributes its build chunks followed by its probe chunks, and the items of
// all joins form one sequence that a persistent grid pulls with an atomic
// counter. A build item inserts its rows and then adds them to built[j]; a
// probe item first waits (bounded) until built[j] == nb_j. The wait cannot
// deadlock: items are claimed in order, every build item of join j precedes
// its probe items, the grid is no larger than what is resident at once, and
// build items never wait. Matches go through the CTA stage to join j's own
// outputs, reserved on its own cursor (d_counts[j]).
//
// Three launches, all asynchronous and graph-capturable: a one-block setup
// (per-join table and item offsets by prefix sums), a table clear, and the
// persistent join kernel.
#include "eiger.h"
#include "emit.cuh"
#include "kernels.cuh"

namespace eiger {

namespace {

struct BatchMeta {
    unsigned long long table_off;  // first slot of the join's table
    uint32_t slots;                // power of two (0: no work)
    uint32_t nbi;                  // build items
};

struct BatchCtrl {
    unsigned long long next_item;
    unsigned long long total_items;
    unsigned long long total_slots;
    unsigned int err;
    unsigned int pad;
};

constexpr int kSetupThreads = 1024;
constexpr uint32_t kWaitLimit = 1u << 22;  // polls (with back-off) before giving up

struct alignas(16) WideSlot {
    unsigned long long key;
    unsigned long long row;
};

// One block: per-join slots, items and their exclusive prefix sums.
__global__ void __launch_bounds__(kSetupThreads)
    batch_setup_kernel(const eiger_join_desc* __restrict__ descs, int k, int chunk, float load,
                       unsigned long long max_slots, BatchMeta* __restrict__ meta,
                       unsigned long long* __restrict__ item_prefix, unsigned* __restrict__ built,
                       long long* __restrict__ counts, BatchCtrl* __restrict__ bc, int* status) {
    __shared__ unsigned long long s_w[2][kSetupThreads / kWarp];
    const unsigned lane = lane_id();
    const int warp = threadIdx.x / kWarp;
    unsigned long long slot_carry = 0, item_carry = 0;
    for (int base = 0; base < k; base += kSetupThreads) {
        const int j = base + threadIdx.x;
        unsigned long long slots = 0, items = 0, nbi = 0;
        if (j < k) {
            const long long nb = descs[j].nb, np = descs[j].np;
            if (nb > 0 && np > 0) {
                const double want = (double)nb / (double)load;
                unsigned long long s = 64;
                while ((double)s < want) s <<= 1;
                slots = s;
                nbi = (unsigned long long)((nb + chunk - 1) / chunk);
                items = nbi + (unsigned long long)((np + chunk - 1) / chunk);
            }
            built[j] = 0;
            counts[j] = 0;
        }
        // block exclusive scans of slots and items
        unsigned long long xs = slots, xi = items;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const unsigned long long ys = __shfl_up_sync(0xffffffffu, xs, o);
            const unsigned long long yi = __shfl_up_sync(0xffffffffu, xi, o);
            if ((int)lane >= o) {
                xs += ys;
                xi += yi;
            }
        }
        if ((int)lane == kWarp - 1) {
            s_w[0][warp] = xs;
            s_w[1][warp] = xi;
        }
        __syncthreads();
        if (warp == 0) {
            unsigned long long vs = s_w[0][lane], vi = s_w[1][lane];
#pragma unroll
            for (int o = 1; o < kWarp; o <<= 1) {
                const unsigned long long ys = __shfl_up_sync(0xffffffffu, vs, o);
                const unsigned long long yi = __shfl_up_sync(0xffffffffu, vi, o);
                if ((int)lane >= o) {
                    vs += ys;
                    vi += yi;
                }
            }
            s_w[0][lane] = vs;
            s_w[1][lane] = vi;
        }
        __syncthreads();
        const unsigned long long off_s = slot_carry + (warp ? s_w[0][warp - 1] : 0ull) + xs - slots;
        const unsigned long long off_i = item_carry + (warp ? s_w[1][warp - 1] : 0ull) + xi - items;
        if (j < k) {
            meta[j].table_off = off_s;
            meta[j].slots = (uint32_t)slots;
            meta[j].nbi = (uint32_t)nbi;
            item_prefix[j] = off_i;
        }
        slot_carry += s_w[0][kWarp - 1];
        item_carry += s_w[1][kWarp - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        item_prefix[k] = item_carry;
        bc->next_item = 0;
        bc->err = 0;
        bc->total_slots = slot_carry;
        if (slot_carry > max_slots) {  // tables do not fit: run nothing, report
            bc->total_items = 0;
            *status = EIGER_ERR_WORKSPACE;
        } else {
            bc->total_items = item_carry;
            *status = EIGER_OK;
        }
    }
}

// Fills the table region with all-ones words (the empty slot of both layouts).
__global__ void batch_clear_kernel(unsigned long long* __restrict__ words, const BatchCtrl* __restrict__ bc,
                                   int words_per_slot) {
    const unsigned long long n = bc->total_items ? bc->total_slots * (unsigned long long)words_per_slot : 0ull;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        words[i] = kEmptySlot;
}

// Warp-collective: the join j whose items contain `item` (last j with prefix[j] <= item).
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

template <typename InKey, int THREADS>
__global__ void __launch_bounds__(THREADS)
    batch_join_kernel(const eiger_join_desc* __restrict__ descs, int k, const BatchMeta* __restrict__ meta,
                      const unsigned long long* __restrict__ item_prefix, unsigned char* __restrict__ tables,
                      unsigned* __restrict__ built, long long* __restrict__ counts, BatchCtrl* bc, int chunk,
                      int* status) {
    constexpr bool kWide = sizeof(InKey) == 8;
    constexpr int kRows = 2;                   // probe rows per thread per round
    constexpr int kStage = THREADS * kRows * 2;
    __shared__ Stage<kStage> st;
    __shared__ unsigned long long s_item;
    __shared__ int s_join;
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
            const int j = it < total ? find_join(item_prefix, k, it) : 0;
            if (lane == 0) {
                s_item = it;
                s_join = j;
            }
        }
        __syncthreads();
        const unsigned long long item = s_item;
        const int j = s_join;
        if (item >= total) break;
        const eiger_join_desc d = descs[j];
        const BatchMeta m = meta[j];
        const unsigned long long local = item - item_prefix[j];
        const uint32_t mask = m.slots - 1;

        if (local < m.nbi) {
            // ---- build chunk
            const long long r0 = (long long)local * chunk;
            const long long r1 = r0 + chunk < d.nb ? r0 + chunk : d.nb;
            const InKey* keys = static_cast<const InKey*>(d.build_keys);
            for (long long r = r0 + threadIdx.x; r < r1; r += THREADS) {
                const InKey key = keys[r];
                if constexpr (kWide) {
                    WideSlot* t = reinterpret_cast<WideSlot*>(tables) + m.table_off;
                    uint32_t s = (uint32_t)mix64((uint64_t)key) & mask;
                    for (uint32_t step = 0;; ++step) {
                        if (atomicCAS(&t[s].row, kEmptySlot, (unsigned long long)r) == kEmptySlot) {
                            t[s].key = (unsigned long long)key;
                            break;
                        }
                        if (step == mask) {
                            atomicOr(&bc->err, kErrTableFull);
                            break;
                        }
                        s = (s + 1) & mask;
                    }
                } else {
                    unsigned long long* t = reinterpret_cast<unsigned long long*>(tables) + m.table_off;
                    const uint32_t k32 = (uint32_t)key;
                    const unsigned long long v = ((unsigned long long)k32 << 32) | (uint32_t)r;
                    uint32_t s = mix32(k32) & mask;
                    for (uint32_t step = 0;; ++step) {
                        if (atomicCAS(t + s, kEmptySlot, v) == kEmptySlot) break;
                        if (step == mask) {
                            atomicOr(&bc->err, kErrTableFull);
                            break;
                        }
                        s = (s + 1) & mask;
                    }
                }
            }
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
                const long long c = (long long)(local - m.nbi);
                const long long r0 = c * chunk;
                const long long r1 = r0 + chunk < d.np ? r0 + chunk : d.np;
                const InKey* keys = static_cast<const InKey*>(d.probe_keys);
                JoinOut out{};
                out.bidx = d.out_bidx;
                out.pidx = d.out_pidx;
                out.capacity = d.capacity > 0 ? (unsigned long long)d.capacity : 0ull;
                unsigned long long* cursor = reinterpret_cast<unsigned long long*>(counts + j);
                const long long round = (long long)THREADS * kRows;
                for (long long base = r0; base < r1; base += round) {
#pragma unroll 1
                    for (int it = 0; it < kRows; ++it) {
                        const long long r = base + (long long)it * THREADS + threadIdx.x;
                        bool active = r < r1;
                        InKey key = 0;
                        uint32_t s = 0, steps = 0;
                        if (active) {
                            key = __ldcs(keys + r);
                            s = kWide ? (uint32_t)mix64((uint64_t)key) & mask : mix32((uint32_t)key) & mask;
                        }
                        while (__any_sync(0xffffffffu, active)) {
                            bool hit = false;
                            uint32_t bi = 0;
                            if (active) {
                                if constexpr (kWide) {
                                    const WideSlot* t = reinterpret_cast<const WideSlot*>(tables) + m.table_off;
                                    const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(t + s));
                                    if (v.y == kEmptySlot) {
                                        active = false;
                                    } else {
                                        hit = v.x == (unsigned long long)key;
                                        bi = (uint32_t)v.y;
                                    }
                                } else {
                                    const unsigned long long* t =
                                        reinterpret_cast<const unsigned long long*>(tables) + m.table_off;
                                    const unsigned long long v = __ldcg(t + s);
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
                                        atomicOr(&bc->err, kErrTableFull);
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
        }
        __syncthreads();
    }
    (void)status;  // device errors are folded in by batch_status_kernel
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
int resident_grid(Kern kern, int threads, const DevInfo& di) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return di.sms * per_sm;
}

template <typename InKey, int THREADS>
cudaError_t launch_batch(const eiger_join_desc* d_descs, int k, const BatchLayout& L, long long* d_counts,
                         int chunk, int* d_status, const DevInfo& di, cudaStream_t stream) {
    auto kern = batch_join_kernel<InKey, THREADS>;
    // Persistent grid no larger than what is resident at once (probe items may
    // wait for build items held by other CTAs).
    const int grid = resident_grid(kern, THREADS, di);
    ProfScope ps("batch_join", 0.0, stream);
    kern<<<grid, THREADS, 0, stream>>>(d_descs, k, reinterpret_cast<const BatchMeta*>(L.meta), L.item_prefix,
                                       L.tables, L.built, d_counts, reinterpret_cast<BatchCtrl*>(L.ctrl), chunk,
                                       d_status);
    return cudaGetLastError();
}

}  // namespace

BatchLayout batch_layout(Carve& c, int k, unsigned long long total_slots, int slot_bytes) {
    BatchLayout L;
    L.ctrl = c.take<unsigned char>(sizeof(BatchCtrl));
    L.meta = c.take<unsigned char>(sizeof(BatchMeta) * (size_t)(k > 0 ? k : 1));
    L.item_prefix = c.take<unsigned long long>((size_t)k + 1);
    L.built = c.take<unsigned>((size_t)(k > 0 ? k : 1));
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
                                                            L.table_slots, meta, L.item_prefix, L.built,
                                                            d_counts, bc, d_status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int wps = dtype == EIGER_I32 ? 1 : 2;
    {
        ProfScope ps("batch_clear", 8.0 * wps * (double)L.table_slots, stream);
        batch_clear_kernel<<<di.sms * 4, 512, 0, stream>>>(reinterpret_cast<unsigned long long*>(L.tables), bc,
                                                           wps);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    switch (knobs.block_threads) {
        case 128:
            e = dtype == EIGER_I32 ? launch_batch<int32_t, 128>(d_descs, k, L, d_counts, knobs.chunk_rows, d_status, di, stream)
                                   : launch_batch<int64_t, 128>(d_descs, k, L, d_counts, knobs.chunk_rows, d_status, di, stream);
            break;
        case 256:
            e = dtype == EIGER_I32 ? launch_batch<int32_t, 256>(d_descs, k, L, d_counts, knobs.chunk_rows, d_status, di, stream)
                                   : launch_batch<int64_t, 256>(d_descs, k, L, d_counts, knobs.chunk_rows, d_status, di, stream);
            break;
        default:
            e = dtype == EIGER_I32 ? launch_batch<int32_t, 512>(d_descs, k, L, d_counts, knobs.chunk_rows, d_status, di, stream)
                                   : launch_batch<int64_t, 512>(d_descs, k, L, d_counts, knobs.chunk_rows, d_status, di, stream);
            break;
    }
    if (e != cudaSuccess) return e;
    batch_status_kernel<<<1, 32, 0, stream>>>(bc, d_status);
    return cudaGetLastError();
}

}  // namespace eiger
