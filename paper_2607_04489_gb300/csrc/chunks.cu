// Compaction of the per-warp output runs of a chunked join launch (the pairs
// of the partitioned join): see chunks.cuh.
//
// With R positions reserved (the cursor, a multiple of kOutChunk) and H holes
// (the unfilled tails of the warps' last runs), the match count is C = R - H.
// Every hole below C is matched with one filled position at or above C, and
// the pair stored there moves into the hole:
//   plan (one CTA)  H, C; the fill of every run at or above C; exclusive
//                   prefixes of the holes below C per warp record and of the
//                   filled positions at or above C per run; cursor := C;
//   move (grid)     one warp per record walks its holes below C; the k-th
//                   hole takes the k-th filled position at or above C.
// Holes lie below C and sources at or above it, so no move overwrites the
// source of another.
#include "chunks.cuh"
#include "kernels.cuh"

namespace eiger {

namespace {

constexpr int kFixThreads = 1024;

// Block-collective exclusive scan of v(i), i in [0, n), into out[0, n];
// out[n] = total, which is also returned. 1024 entries per step.
template <typename F>
__device__ unsigned long long block_exscan(uint32_t n, F v, uint32_t* out, unsigned long long* s_warp) {
    const unsigned lane = lane_id();
    const int warp = threadIdx.x / kWarp;
    unsigned long long carry = 0;
    for (uint32_t base = 0; base < n; base += kFixThreads) {
        const uint32_t i = base + threadIdx.x;
        const unsigned long long x0 = i < n ? v(i) : 0ull;
        unsigned long long x = x0;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if ((int)lane >= o) x += y;
        }
        if ((int)lane == kWarp - 1) s_warp[warp] = x;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = s_warp[lane];
#pragma unroll
            for (int o = 1; o < kWarp; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, w, o);
                if ((int)lane >= o) w += y;
            }
            s_warp[lane] = w;
        }
        __syncthreads();
        if (i < n) out[i] = (uint32_t)(carry + (warp ? s_warp[warp - 1] : 0ull) + x - x0);
        carry += s_warp[kWarp - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = (uint32_t)carry;
    return carry;
}

__global__ void __launch_bounds__(kFixThreads) chunk_fix_plan_kernel(PairSink s, uint32_t W, ChunkFix f,
                                                                   unsigned* err) {
    __shared__ unsigned long long s_warp[kWarp];
    const unsigned long long R = *s.cursor;
    unsigned long long h = 0;
    for (uint32_t w = threadIdx.x; w < W; w += kFixThreads) {
        const ChunkRec r = s.rec[w];
        if (r.base != ~0ull) h += kOutChunk - r.used;
    }
#pragma unroll
    for (int o = kWarp / 2; o > 0; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    if (lane_id() == 0) s_warp[threadIdx.x / kWarp] = h;
    __syncthreads();
    unsigned long long H = 0;
    for (int w = 0; w < kFixThreads / kWarp; ++w) H += s_warp[w];
    __syncthreads();  // every thread has read R and s_warp
    const unsigned long long C = R - H;
    if (H > R || C > s.capacity || H == 0) {
        // nothing to move (no holes), or the count alone is reported
        if (threadIdx.x == 0) {
            if (H > R) atomicOr(err, kErrInternal);
            f.hdr[0] = 0;
            *s.cursor = H > R ? R : C;
        }
        return;
    }
    const unsigned long long c0 = C / kOutChunk;
    const uint32_t nab = (uint32_t)(R / kOutChunk - c0);  // runs at or above C: at most W
    if (nab > W + 1) {
        if (threadIdx.x == 0) {
            atomicOr(err, kErrInternal);
            f.hdr[0] = 0;
        }
        return;
    }
    for (uint32_t i = threadIdx.x; i < nab; i += kFixThreads) f.used_above[i] = kOutChunk;
    __syncthreads();
    for (uint32_t w = threadIdx.x; w < W; w += kFixThreads) {
        const ChunkRec r = s.rec[w];
        if (r.base != ~0ull && r.base >= c0 * kOutChunk) f.used_above[r.base / kOutChunk - c0] = r.used;
    }
    __syncthreads();
    // filled positions of run i inside [C, R): a run's filled part is its prefix
    const unsigned long long va = block_exscan(
        nab,
        [&](uint32_t i) -> unsigned long long {
            const unsigned long long st = (c0 + i) * kOutChunk;
            const unsigned long long lo = st > C ? st : C;
            const unsigned long long hi = st + f.used_above[i];
            return hi > lo ? hi - lo : 0ull;
        },
        f.va_pref, s_warp);
    // holes of record w below C
    const unsigned long long hb = block_exscan(
        W,
        [&](uint32_t w) -> unsigned long long {
            const ChunkRec r = s.rec[w];
            if (r.base == ~0ull || r.base >= C) return 0ull;
            const unsigned long long hs = r.base + r.used;
            const unsigned long long he = r.base + kOutChunk < C ? r.base + kOutChunk : C;
            return he > hs ? he - hs : 0ull;
        },
        f.hb_pref, s_warp);
    if (threadIdx.x == 0) {
        if (va != hb) {
            atomicOr(err, kErrInternal);
            f.hdr[0] = 0;
        } else {
            f.hdr[0] = va;
        }
        f.hdr[1] = C;
        f.hdr[2] = c0;
        f.hdr[3] = nab;
        *s.cursor = C;
    }
}

__global__ void __launch_bounds__(256) chunk_fix_move_kernel(PairSink s, uint32_t W, ChunkFix f) {
    const unsigned long long V = f.hdr[0];
    if (V == 0) return;
    const unsigned long long C = f.hdr[1], c0 = f.hdr[2];
    const uint32_t nab = (uint32_t)f.hdr[3];
    const unsigned lane = lane_id();
    const uint32_t warps = blockDim.x / kWarp;
    for (uint32_t w = blockIdx.x * warps + threadIdx.x / kWarp; w < W; w += gridDim.x * warps) {
        const uint32_t k0 = f.hb_pref[w], k1 = f.hb_pref[w + 1];
        if (k0 == k1) continue;
        const ChunkRec r = s.rec[w];
        uint32_t run = 0;  // warp-uniform: the run holding filled position kb (below)
        for (uint32_t kb = k0; kb < k1; kb += kWarp) {
            // one binary search per 32 positions (lane 0), then each lane
            // steps forward from there: 32 consecutive positions span at most
            // a few runs, as a full run holds kOutChunk of them
            if (lane == 0) {
                uint32_t lo = run, hi = nab;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (f.va_pref[mid] <= kb) lo = mid; else hi = mid;
                }
                run = lo;
            }
            run = __shfl_sync(0xffffffffu, run, 0);
            const uint32_t k = kb + lane;
            if (k >= k1) continue;
            uint32_t lo = run;
            while (lo + 1 < nab && f.va_pref[lo + 1] <= k) ++lo;
            const unsigned long long st = (c0 + lo) * kOutChunk;
            const unsigned long long src = (st > C ? st : C) + (k - f.va_pref[lo]);
            const unsigned long long dst = r.base + r.used + (k - k0);
            uint32_t b, p;
            if (src < s.capacity) {
                b = s.bidx[src];
                p = s.pidx[src];
            } else {
                b = s.ovf_b[src - s.capacity];
                p = s.ovf_p[src - s.capacity];
            }
            s.bidx[dst] = b;
            s.pidx[dst] = p;
        }
    }
}

}  // namespace

ChunkFix chunk_fix_layout(Carve& c) {
    ChunkFix f;
    f.hdr = c.take<unsigned long long>(4);
    f.hb_pref = c.take<uint32_t>(kMaxOutWarps + 1);
    f.va_pref = c.take<uint32_t>(kMaxOutWarps + 2);
    f.used_above = c.take<uint32_t>(kMaxOutWarps + 2);
    return f;
}

cudaError_t chunk_fix_run(const PairSink& s, uint32_t W, const ChunkFix& f, unsigned* err, const DevInfo& di,
                          cudaStream_t stream) {
    ProfScope ps("chunk_fix", 16.0 * W, stream, 0.0, 2);
    chunk_fix_plan_kernel<<<1, kFixThreads, 0, stream>>>(s, W, f, err);
    chunk_fix_move_kernel<<<di.sms * 2, 256, 0, stream>>>(s, W, f);
    return cudaGetLastError();
}

}  // namespace eiger
