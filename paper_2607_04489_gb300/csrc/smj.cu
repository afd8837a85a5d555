// Sort-merge join (Sec. 3.2, the third join algorithm the paper adopts; Sec.
// 5.3 compares it with the hash joins). Both sides are sorted on the encoded
// key by the stable LSD radix sort of partition.cu; equal keys are then
// adjacent and in the same order on both sides, and the join is a merge.
//
// Merge: the sorted probe side is cut into chunks of kSmjChunk rows. A first
// kernel finds, for every chunk, the window of sorted build rows that can
// match it: [lower_bound(first key), upper_bound(last key)). The join kernel
// takes chunks from a global counter, stages the chunk's keys in shared
// memory, and walks its build window in segments of kSmjWin rows staged the
// same way. For each probe row a binary search over the segment gives its run
// of equal build keys; a block scan of the run lengths places the matches,
// one global atomic reserves them, and they are written either directly (short
// runs) or, when some run is long (duplicate keys), by a load-balanced
// expansion in which every thread writes consecutive output slots and finds
// its probe row by a search over the scanned run starts.
//
// GFTR: the payload columns were sorted with the keys, and matches carry
// positions in the sorted arrays, so the gathers read nearby rows; GFUR:
// matches carry tuple IDs and gather from the caller's columns.
#include "emit.cuh"
#include "kernels.cuh"

namespace eiger {

namespace {

constexpr int kSmjThreads = 512;
constexpr int kSmjRows = 4;                               // probe rows per thread per chunk
constexpr uint32_t kSmjChunk = kSmjThreads * kSmjRows;    // probe rows per chunk
constexpr uint32_t kSmjWin = 4096;                        // build rows per staged segment
constexpr uint32_t kLinear = 8;                           // run scan before a binary search
constexpr uint32_t kDirectMax = 4;                        // longest run written directly

template <typename KeyT>
struct SmjIn {
    const KeyT* bkey;
    const uint32_t* bidx;
    const uint32_t* nb_dev;  // sorted build rows
    const KeyT* pkey;
    const uint32_t* pidx;
    const uint32_t* np_dev;  // sorted probe rows (after the range test)
    const uint32_t* window;  // [chunk][2]
};

template <typename KeyT>
__device__ __forceinline__ uint32_t lower_bound(const KeyT* a, uint32_t lo, uint32_t hi, KeyT k) {
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

template <typename KeyT>
__device__ __forceinline__ uint32_t upper_bound(const KeyT* a, uint32_t lo, uint32_t hi, KeyT k) {
    while (lo < hi) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= k)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

template <typename KeyT>
__global__ void smj_window_kernel(SmjIn<KeyT> a, uint32_t* __restrict__ window) {
    const uint32_t nb = *a.nb_dev, np = *a.np_dev;
    const uint32_t nch = (np + kSmjChunk - 1) / kSmjChunk;
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += gridDim.x * blockDim.x) {
        const uint32_t s = c * kSmjChunk;
        const uint32_t e = np - s < kSmjChunk ? np : s + kSmjChunk;
        window[2 * c] = lower_bound(a.bkey, 0u, nb, a.pkey[s]);
        window[2 * c + 1] = upper_bound(a.bkey, 0u, nb, a.pkey[e - 1]);
    }
}

// Block-collective exclusive scan of one value per thread; returns the total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t& excl, uint32_t* s_warp) {
    const unsigned lane = lane_id();
    const int w = threadIdx.x / kWarp;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    if ((int)lane == kWarp - 1) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t t = (int)lane < kSmjThreads / kWarp ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if ((int)lane >= o) t += y;
        }
        if ((int)lane < kSmjThreads / kWarp) s_warp[lane] = t;
    }
    __syncthreads();
    excl = (w ? s_warp[w - 1] : 0u) + x - v;
    const uint32_t total = s_warp[kSmjThreads / kWarp - 1];
    __syncthreads();
    return total;
}

template <typename KeyT>
constexpr size_t smj_smem() {
    return (size_t)kSmjChunk * (sizeof(KeyT) + 3 * sizeof(uint32_t)) + (size_t)kSmjWin * (sizeof(KeyT) + 4);
}

template <typename KeyT, bool AGG, bool POS>
__global__ void __launch_bounds__(kSmjThreads, 2) smj_join_kernel(SmjIn<KeyT> a, JoinOut out, Ctrl* ctrl) {
    extern __shared__ __align__(16) unsigned char smem[];
    KeyT* s_pk = reinterpret_cast<KeyT*>(smem);
    KeyT* s_bk = s_pk + kSmjChunk;
    uint32_t* s_pid = reinterpret_cast<uint32_t*>(s_bk + kSmjWin);
    uint32_t* s_bid = s_pid + kSmjChunk;
    uint32_t* s_off = s_bid + kSmjWin;
    uint32_t* s_lo = s_off + kSmjChunk;
    __shared__ uint32_t s_warp[kSmjThreads / kWarp];
    __shared__ unsigned long long s_base;
    __shared__ unsigned long long s_chunk;

    const uint32_t np = *a.np_dev;
    const uint32_t nch = (np + kSmjChunk - 1) / kSmjChunk;
    AggState agg{0ull, 0ull};
    for (;;) {
        if (threadIdx.x == 0) s_chunk = atomicAdd(&ctrl->next_item, 1ull);
        __syncthreads();
        const unsigned long long c = s_chunk;
        if (c >= nch) break;
        const uint32_t s0 = (uint32_t)c * kSmjChunk;
        const uint32_t pn = np - s0 < kSmjChunk ? np - s0 : kSmjChunk;
        for (uint32_t i = threadIdx.x; i < pn; i += kSmjThreads) {
            s_pk[i] = __ldcs(a.pkey + s0 + i);
            s_pid[i] = POS ? s0 + i : __ldcs(a.pidx + s0 + i);
        }
        const uint32_t wlo = a.window[2 * c], whi = a.window[2 * c + 1];
        for (unsigned long long seg64 = wlo; seg64 < whi; seg64 += kSmjWin) {
            const uint32_t seg = (uint32_t)seg64;
            const uint32_t bn = whi - seg < kSmjWin ? whi - seg : kSmjWin;
            __syncthreads();  // previous segment consumed; chunk staged
            for (uint32_t i = threadIdx.x; i < bn; i += kSmjThreads) {
                s_bk[i] = a.bkey[seg + i];
                s_bid[i] = POS ? seg + i : a.bidx[seg + i];
            }
            __syncthreads();
            uint32_t lo[kSmjRows], cnt[kSmjRows], tot = 0, mx = 0;
#pragma unroll
            for (int q = 0; q < kSmjRows; ++q) {
                const uint32_t j = threadIdx.x * kSmjRows + q;
                lo[q] = 0;
                cnt[q] = 0;
                if (j < pn) {
                    const KeyT k = s_pk[j];
                    const uint32_t l = lower_bound(s_bk, 0u, bn, k);
                    uint32_t h = l;
                    while (h < bn && h - l < kLinear && s_bk[h] == k) ++h;
                    if (h - l == kLinear) h = upper_bound(s_bk, h, bn, k);
                    lo[q] = l;
                    cnt[q] = h - l;
                }
                tot += cnt[q];
                mx = cnt[q] > mx ? cnt[q] : mx;
            }
            if (AGG) {
#pragma unroll
                for (int q = 0; q < kSmjRows; ++q) {
                    const uint32_t j = threadIdx.x * kSmjRows + q;
                    for (uint32_t x = 0; x < cnt[q]; ++x)
                        agg.sum += (unsigned long long)read_pay(out.b.src[0], out.b.bytes[0], s_bid[lo[q] + x]) +
                                   (unsigned long long)read_pay(out.p.src[0], out.p.bytes[0], s_pid[j]);
                    agg.count += cnt[q];
                }
                continue;
            }
            uint32_t off;
            const uint32_t T = block_excl_scan(tot, off, s_warp);
            if (T == 0) continue;
            const bool expand = __syncthreads_or(mx > kDirectMax) != 0;
            if (threadIdx.x == 0) s_base = atomicAdd(&ctrl->cursor, (unsigned long long)T);
            if (expand) {
                uint32_t run = off;
#pragma unroll
                for (int q = 0; q < kSmjRows; ++q) {
                    const uint32_t j = threadIdx.x * kSmjRows + q;
                    s_off[j] = run;  // rows past pn get runs of length 0
                    s_lo[j] = lo[q];
                    run += cnt[q];
                }
            }
            __syncthreads();
            const unsigned long long base = s_base;
            if (!expand) {
                unsigned long long pos = base + off;
#pragma unroll
                for (int q = 0; q < kSmjRows; ++q) {
                    const uint32_t j = threadIdx.x * kSmjRows + q;
                    for (uint32_t x = 0; x < cnt[q]; ++x) write_match(out, pos++, s_bid[lo[q] + x], s_pid[j]);
                }
            } else {
                for (uint32_t t = threadIdx.x; t < T; t += kSmjThreads) {
                    // probe row of output slot t: the last row whose run starts at or before t
                    const uint32_t j = upper_bound(s_off, 0u, kSmjChunk, t) - 1;
                    write_match(out, base + t, s_bid[s_lo[j] + (t - s_off[j])], s_pid[j]);
                }
            }
        }
        __syncthreads();
    }
    if (AGG) agg_commit(agg, ctrl);
}

template <typename KeyT>
cudaError_t launch_smj(const SmjScratch& s, const PlanDev& plan, const JoinOut& out, Ctrl* ctrl, const DevInfo& di,
                       cudaStream_t stream, int64_t nb, int64_t np) {
    const int buf = (plan.bits2 - 1) & 1;
    SmjIn<KeyT> a;
    a.bkey = static_cast<const KeyT*>(s.side[0].key[buf]);
    a.bidx = s.side[0].idx[buf];
    a.nb_dev = s.side[0].total;
    a.pkey = static_cast<const KeyT*>(s.side[1].key[buf]);
    a.pidx = s.side[1].idx[buf];
    a.np_dev = s.side[1].total;
    a.window = s.window;
    cudaError_t e;
    {
        const uint32_t nch = (uint32_t)((np + kSmjChunk - 1) / kSmjChunk);
        ProfScope ps("smj_window", 8.0 * nch, stream);
        smj_window_kernel<KeyT><<<(nch + 255) / 256, 256, 0, stream>>>(a, s.window);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    auto kern = out.aggregate ? (plan.gftr ? smj_join_kernel<KeyT, true, true> : smj_join_kernel<KeyT, true, false>)
                : plan.gftr   ? smj_join_kernel<KeyT, false, true>
                              : smj_join_kernel<KeyT, false, false>;
    const size_t smem = smj_smem<KeyT>();
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSmjThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    // reads every sorted (key', row) of both sides once, writes the matches
    const double tuple = (double)(sizeof(KeyT) + sizeof(uint32_t));
    ProfScope ps("smj_merge", tuple * (double)(nb + np), stream, match_bytes(out));
    kern<<<di.sms * per_sm, kSmjThreads, smem, stream>>>(a, out, ctrl);
    return cudaGetLastError();
}

}  // namespace

SmjScratch smj_layout(Carve& c, int64_t nb, int64_t np, const PlanDev& plan) {
    SmjScratch s;
    const size_t kb = plan.key32 ? 4 : 8;
    part_side_layout(c, s.side[0], nb, plan.bits1, 0, plan.bits2, true, kb, plan, 0);
    part_side_layout(c, s.side[1], np, plan.bits1, 0, plan.bits2, true, kb, plan, 1);
    s.window = c.take<uint32_t>(2 * ((size_t)(np + kSmjChunk - 1) / kSmjChunk + 1));
    return s;
}

cudaError_t smj_run(const JoinArgs& a, const PlanDev& plan, const SmjScratch& s, const JoinOut& out, Ctrl* ctrl,
                    cudaStream_t stream) {
    if (a.nb == 0 || a.np == 0) return cudaSuccess;
    DevInfo di;
    cudaError_t e = current_device_info(&di);
    if (e != cudaSuccess) return e;
    // the two sides are sorted concurrently: build on a second stream
    cudaStream_t side;
    if ((e = fork_side(stream, &side)) != cudaSuccess) return e;
    if ((e = sort_side(a.bkeys, a.nb, 0, plan, s.side[0], &out.b, &ctrl->err, side)) != cudaSuccess) return e;
    if ((e = sort_side(a.pkeys, a.np, 1, plan, s.side[1], &out.p, &ctrl->err, stream)) != cudaSuccess) return e;
    if ((e = join_side(stream, side)) != cudaSuccess) return e;
    const JoinOut o = plan.gftr ? gftr_out(out, s.side[0], s.side[1], (plan.bits2 - 1) & 1) : out;
    return plan.key32 ? launch_smj<uint32_t>(s, plan, o, ctrl, di, stream, a.nb, a.np)
                      : launch_smj<uint64_t>(s, plan, o, ctrl, di, stream, a.nb, a.np);
}

}  // namespace eiger
