// Radix partitioning for the partitioned hash join (Sec. 3.2, the PHJ the
// paper adopts; partitions are taken on bits of a hash of the key so their
// sizes are even, as Sec. 3.3 does before partitioning).
//
// Each pass splits every input segment by `bits` further bits of mix(key'):
// pass 1 by the top b1 bits, pass 2 by the next b2 bits within each pass-1
// partition. A pass runs three steps over fixed tiles of kPartTile rows:
//   hist    per tile, a shared-memory histogram of the digits, written to a
//           counts array laid out [segment][digit][tile-in-segment];
//   scan    one device-wide exclusive scan of that array, which turns every
//           (tile, digit) count into the global output offset of that tile's
//           run of the digit (segments stay contiguous and in order);
//   scatter per tile, rank each row within its digit with a shared-memory
//           atomic, stage the tile in shared memory grouped by digit, then
//           write each digit run to its global offset with consecutive
//           threads on consecutive addresses (coalesced runs instead of one
//           scattered 8-byte store per row).
// The first pass reads the raw key column (row ids are implicit), applies the
// probe-side range test (a probe key outside [min_R, max_R] cannot match and
// is dropped here) and the frame-of-reference narrowing; later passes read the
// (key', row) pairs of the previous pass.
#include <cstdio>
#include <type_traits>

#include "kernels.cuh"

namespace eiger {

namespace {

#ifndef EIGER_PART_THREADS
#define EIGER_PART_THREADS 512
#endif
constexpr int kPartThreads = EIGER_PART_THREADS;
constexpr int kPartItems = kPartTile / kPartThreads;  // rows per thread per tile
constexpr uint32_t kNoDigit = 0xFFFFFFFFu;

constexpr int kScanThreads = 512;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

// Payload columns that travel with the keys (GFTR): read at the tile rows of
// `in`, written to the same output positions as the keys.
struct ColCarry {
    const void* in[kMaxCols];
    void* out[kMaxCols];
    int bytes[kMaxCols];
    int n;
};

template <typename InKey, typename KeyT>
struct PartPass {
    const InKey* raw;        // pass 1 input: raw key column
    const KeyT* in_key;      // later passes: previous pass output
    const uint32_t* in_idx;
    KeyT* out_key;
    uint32_t* out_idx;
    uint32_t n;              // pass 1: rows
    KeyRange rng;
    int check_range;
    int dshift;              // digit = (hash >> dshift) & dmask
    uint32_t dmask;
    int bits;
    uint32_t* counts;
    const Tile* tiles;       // nullptr: pass-1 tiling of [0, n)
    const uint32_t* ntiles_dev;
    uint32_t ntiles_fixed;
    ColCarry cc;
    // Exclusive ends of the memory a tile load may read around its rows (key
    // source, tuple-ID source); the arrays' bases are the starts. A tile whose
    // 16-byte aligned cover [align_down(first), align_up(last + 1)) lies
    // inside is loaded by one bulk copy of the cover; nullptr: never.
    const void* src_end[2];
};

template <typename InKey, typename KeyT>
__device__ __forceinline__ Tile get_tile(const PartPass<InKey, KeyT>& a, uint32_t t) {
    if (a.tiles) return a.tiles[t];
    Tile tl;
    tl.start = t * (uint32_t)kPartTile;
    const uint32_t rest = a.n - tl.start;
    tl.len = rest < (uint32_t)kPartTile ? rest : (uint32_t)kPartTile;
    tl.seg = 0;
    tl.tile_base = 0;
    tl.ntiles_seg = a.ntiles_fixed;
    return tl;
}

__device__ __forceinline__ size_t count_index(const Tile& tl, uint32_t t, uint32_t d, int bits) {
    return ((size_t)tl.tile_base << bits) + (size_t)d * tl.ntiles_seg + (t - tl.tile_base);
}

// Partition digit: bits of the mixed key (hash partitioning) or, for the
// sort, bits of the encoded key itself.
template <bool SORTM, typename KeyT>
__device__ __forceinline__ uint32_t digit_of(KeyT k, int dshift, uint32_t dmask) {
    if constexpr (SORTM)
        return (uint32_t)(k >> dshift) & dmask;
    else
        return (uint32_t)(KeyCodec<KeyT>::hash(k) >> dshift) & dmask;
}

// Exclusive scan of in[0, n) into out[0, n), n <= kPartItems * blockDim.x.
// Block-collective; returns the total. s_warp: blockDim.x / 32 words. With
// `rebase`, also rebase[i] -= out[i] for every i (by the thread that wrote
// out[i], so no barrier is needed in between).
__device__ uint32_t block_scan_smem(const uint32_t* in, uint32_t* out, uint32_t n, uint32_t* s_warp,
                                    uint32_t* rebase = nullptr) {
    const uint32_t per = (n + blockDim.x - 1) / blockDim.x;
    uint32_t beg = threadIdx.x * per;
    if (beg > n) beg = n;
    uint32_t end = beg + per;
    if (end > n) end = n;
    uint32_t local = 0;
    for (uint32_t i = beg; i < end; ++i) local += in[i];
    uint32_t x = local;
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    const int warp = threadIdx.x / kWarp;
    const int nw = blockDim.x / kWarp;
    __syncthreads();
    if ((int)lane == kWarp - 1) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = (int)lane < nw ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if ((int)lane >= o) v += y;
        }
        if ((int)lane < nw) s_warp[lane] = v;
    }
    __syncthreads();
    uint32_t prefix = (warp ? s_warp[warp - 1] : 0u) + x - local;
    const uint32_t total = s_warp[nw - 1];
    for (uint32_t i = beg; i < end; ++i) {
        out[i] = prefix;
        if (rebase) rebase[i] -= prefix;
        prefix += in[i];
    }
    return total;
}

// Input element type of a pass: raw keys in pass 1, (key', row) later.
template <typename InKey, typename KeyT, bool FIRST>
struct PassIn {
    using E = typename std::conditional<FIRST, InKey, KeyT>::type;
    static constexpr uint32_t kPad = 32 / sizeof(E);  // room for the 16-byte lead and tail of a cover copy
    static constexpr size_t kKeyBytes = align_up((kPartTile + kPad) * sizeof(E), 16);
    static constexpr size_t kIdxBytes = FIRST ? 0 : align_up((kPartTile + 8) * sizeof(uint32_t), 16);
    static constexpr size_t kBufBytes = kKeyBytes + kIdxBytes;
};

// Shared-memory tile ring: two input buffers, each filled by TMA bulk copies
// one tile ahead of the one being processed, each with its mbarrier.
template <typename InKey, typename KeyT, bool FIRST>
struct TileRing {
    using P = PassIn<InKey, KeyT, FIRST>;
    using E = typename P::E;
    uint64_t* bar;          // [2]
    unsigned char* buf[2];  // keys, then (later passes) rows

    __device__ E* keys(int b) const { return reinterpret_cast<E*>(buf[b]); }
    __device__ uint32_t* rows(int b) const { return reinterpret_cast<uint32_t*>(buf[b] + P::kKeyBytes); }

    __device__ static const E* key_src(const PartPass<InKey, KeyT>& a, uint32_t start) {
        if constexpr (FIRST)
            return a.raw + start;
        else
            return a.in_key + start;
    }

    // Warp 0 only: start loading tile `tl` into buffer b (with its tuple IDs
    // when ROWS). Lane 0 declares the bulk bytes on the buffer's barrier and
    // issues the bulk copies first; the lanes then copy the few unaligned
    // head and tail elements in parallel while the bulk copies are in flight,
    // and lane 0 arrives once they are written, so waiters see both.
    template <bool ROWS>
    __device__ void issue(const PartPass<InKey, KeyT>& a, const Tile& tl, int b) const {
        const unsigned lane = lane_id();
        const E* kf = key_src(a, tl.start);
        {
            // The aligned cover of the tile inside the source arrays: one bulk
            // copy per array, no element copies, no wait in this warp.
            const E* kbase = FIRST ? reinterpret_cast<const E*>(a.raw) : reinterpret_cast<const E*>(a.in_key);
            uint32_t kb = 0, ib = 0;
            const char* kc = cover(kf, tl.len, kbase, a.src_end[0], kb);
            const char* ic = nullptr;
            bool ok = kc != nullptr;
            if constexpr (ROWS) {
                ic = cover(a.in_idx + tl.start, tl.len, a.in_idx, a.src_end[1], ib);
                ok = ok && ic != nullptr;
            }
            if (ok) {
                if (lane == 0) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(&bar[b], kb + ib);
                    bulk_load(keys(b), kc, kb, &bar[b]);
                    if constexpr (ROWS) bulk_load(rows(b), ic, ib, &bar[b]);
                }
                return;
            }
        }
        uint32_t klead, klo, khi;
        uint32_t bytes = tile_copy_plan(kf, tl.len, klead, klo, khi);
        uint32_t ilead = 0, ilo = 0, ihi = 0;
        const uint32_t* rf = nullptr;
        if constexpr (ROWS) {
            rf = a.in_idx + tl.start;
            bytes += tile_copy_plan(rf, tl.len, ilead, ilo, ihi);
        }
        if (lane == 0) {
            fence_proxy_async_smem();
            mbar_expect_tx(&bar[b], bytes);
            tile_copy_body(keys(b), kf, klead, klo, khi, &bar[b]);
            if constexpr (ROWS) tile_copy_body(rows(b), rf, ilead, ilo, ihi, &bar[b]);
        }
        edges_warp(keys(b), kf, tl.len, klead, klo, khi, lane);
        if constexpr (ROWS) edges_warp(rows(b), rf, tl.len, ilead, ilo, ihi, lane);
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar[b]);
    }

    // Start of the 16-byte aligned cover of [first, first + len) and its bytes
    // (a multiple of 16), or nullptr when the cover leaves [base, end).
    template <typename T>
    __device__ static const char* cover(const T* first, uint32_t len, const T* base, const void* end,
                                        uint32_t& bytes) {
        if (!end) return nullptr;
        const uintptr_t lo = reinterpret_cast<uintptr_t>(first) & ~(uintptr_t)15;
        const uintptr_t hi = (reinterpret_cast<uintptr_t>(first + len) + 15) & ~(uintptr_t)15;
        if (lo < reinterpret_cast<uintptr_t>(base) || hi > reinterpret_cast<uintptr_t>(end)) return nullptr;
        bytes = (uint32_t)(hi - lo);
        return reinterpret_cast<const char*>(lo);
    }

    // Lane l of the issuing warp copies head element l and tail element l.
    template <typename T>
    __device__ static void edges_warp(T* dst, const T* first, uint32_t len, uint32_t lead, uint32_t lo,
                                      uint32_t hi, unsigned lane) {
        if (lane < lo) dst[lead + lane] = first[lane];
        if (hi + lane < len) dst[lead + hi + lane] = first[hi + lane];
    }
};

template <typename E>
__device__ __forceinline__ uint32_t lead_of(const E* first) {
    return (uint32_t)((reinterpret_cast<uintptr_t>(first) & 15u) / sizeof(E));
}

// Warp 0: start loading tile `tl` of a scatter pass into buffer b. Later passes
// load the tile's tuple IDs too, unless the side keeps none (in_idx == nullptr:
// its consumer reads rows by position only).
template <typename InKey, typename KeyT, bool FIRST>
__device__ __forceinline__ void issue_tile(const TileRing<InKey, KeyT, FIRST>& ring,
                                           const PartPass<InKey, KeyT>& a, const Tile& tl, int b) {
    if constexpr (FIRST) {
        ring.template issue<false>(a, tl, b);
    } else {
        if (a.in_idx)
            ring.template issue<true>(a, tl, b);
        else
            ring.template issue<false>(a, tl, b);
    }
}

// Decodes element e of the current tile: applies the range test and the
// narrowing in pass 1. Returns false for a dropped row.
template <typename InKey, typename KeyT, bool FIRST>
__device__ __forceinline__ bool tile_key(const PartPass<InKey, KeyT>& a,
                                         const typename PassIn<InKey, KeyT, FIRST>::E* kbuf, uint32_t e,
                                         KeyT& k) {
    if constexpr (FIRST) {
        const int64_t key = (int64_t)kbuf[e];
        if (a.check_range && (key < a.rng.lo || key > a.rng.hi)) return false;
        k = KeyCodec<KeyT>::encode(key, a.rng.offset);
    } else {
        k = kbuf[e];
    }
    return true;
}

template <typename InKey, typename KeyT, bool FIRST>
__device__ __forceinline__ TileRing<InKey, KeyT, FIRST> ring_setup(unsigned char* smem, size_t off) {
    using P = PassIn<InKey, KeyT, FIRST>;
    TileRing<InKey, KeyT, FIRST> r;
    r.bar = reinterpret_cast<uint64_t*>(smem);
    r.buf[0] = smem + off;
    r.buf[1] = smem + off + P::kBufBytes;
    if (threadIdx.x == 0) {
        mbar_init(&r.bar[0], 1);
        mbar_init(&r.bar[1], 1);
        fence_mbar_init();
    }
    return r;
}

// After a failed bounded wait: record the error and wait (bounded) for the
// copy into the other buffer, so no TMA write lands after the CTA exits.
template <typename InKey, typename KeyT, bool FIRST>
__device__ void ring_abort(const TileRing<InKey, KeyT, FIRST>& r, int other, uint32_t parity,
                           bool other_pending, unsigned* err) {
    if (threadIdx.x == 0) {
        atomicOr(err, kErrInternal);
        if (other_pending) mbar_wait(&r.bar[other], parity);
    }
}

template <typename InKey, typename KeyT, bool FIRST>
__host__ __device__ constexpr size_t hist_smem_bytes(int bits) {
    return align_up(16 + 2 * ((size_t)1 << bits) * sizeof(uint32_t), 16) +
           2 * PassIn<InKey, KeyT, FIRST>::kBufBytes;
}

// Two CTA barriers per tile: the digit counters are double-buffered by tile
// parity, so the next tile's counting starts while slower threads still store
// this tile's counts.
template <typename InKey, typename KeyT, bool FIRST, bool SORTM>
__global__ void __launch_bounds__(kPartThreads) part_hist_kernel(PartPass<InKey, KeyT> a, unsigned* err) {
    using Ring = TileRing<InKey, KeyT, FIRST>;
    extern __shared__ __align__(16) unsigned char smem[];
    const uint32_t nd = 1u << a.bits;
    uint32_t* s_cnt2 = reinterpret_cast<uint32_t*>(smem + 16);  // [2][nd]
    const Ring ring = ring_setup<InKey, KeyT, FIRST>(smem, align_up(16 + 2 * (size_t)nd * 4, 16));
    __syncthreads();
    const uint32_t ntiles = a.tiles ? *a.ntiles_dev : a.ntiles_fixed;
    uint32_t t = blockIdx.x;
    Tile d_next{};  // warp 0: descriptor of the next tile to issue, loaded one tile early
    if (threadIdx.x < kWarp) {
        if (t < ntiles) ring.template issue<false>(a, get_tile(a, t), 0);
        if (t + gridDim.x < ntiles) d_next = get_tile(a, t + gridDim.x);
    }
    for (uint32_t it = 0; t < ntiles; t += gridDim.x, ++it) {
        const int b = it & 1;
        const uint32_t tn = t + gridDim.x;
        if (threadIdx.x < kWarp && tn < ntiles) {
            ring.template issue<false>(a, d_next, b ^ 1);
            if (tn + gridDim.x < ntiles) d_next = get_tile(a, tn + gridDim.x);
        }
        uint32_t* s_cnt = s_cnt2 + b * nd;
        for (uint32_t d = threadIdx.x; d < nd; d += blockDim.x) s_cnt[d] = 0;
        const Tile tl = get_tile(a, t);
        const bool ok = mbar_wait(&ring.bar[b], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            ring_abort(ring, b ^ 1, ((it + 1) >> 1) & 1, tn < ntiles, err);
            return;
        }
        const auto* kbuf = ring.keys(b) + lead_of(Ring::key_src(a, tl.start));
#pragma unroll 4
        for (uint32_t e = threadIdx.x; e < tl.len; e += kPartThreads) {
            KeyT k;
            if (tile_key<InKey, KeyT, FIRST>(a, kbuf, e, k))
                atomicAdd(&s_cnt[digit_of<SORTM>(k, a.dshift, a.dmask)], 1u);
        }
        __syncthreads();
        for (uint32_t d = threadIdx.x; d < nd; d += blockDim.x)
            a.counts[count_index(tl, t, d, a.bits)] = s_cnt[d];
    }
}

template <typename InKey, typename KeyT, bool FIRST>
__host__ __device__ constexpr size_t scatter_smem_bytes(int bits) {
    return align_up(16 + 4 * ((size_t)1 << bits) * sizeof(uint32_t), 16) +
           2 * PassIn<InKey, KeyT, FIRST>::kBufBytes + align_up((size_t)kPartTile * sizeof(KeyT), 16) +
           (size_t)kPartTile * sizeof(uint32_t) + (size_t)kPartTile * sizeof(uint16_t);
}

// Digits a thread owns in the per-tile offset table (prefetched one tile ahead).
constexpr int kGoffPerThread = (1 << kMaxBits) / kPartThreads;

constexpr int kPartWarps = kPartThreads / kWarp;
constexpr int kWarpRows = kPartTile / kPartWarps;  // sort scatter: consecutive rows per warp
static_assert(kWarpRows == kPartItems * kWarp, "sort tiles are warp-blocked");

// Block-collective: moves one carried column of the current tile to the
// output positions of its rows. Row j of this thread (tile element e_j, digit
// and rank in dr[j]) is staged at its tile position, then every digit run is
// written out with consecutive threads on consecutive addresses, like the
// keys. Hash mode: e_j = j * threads + t, position = start[d] + rank. Sort
// mode: e_j = warp * kWarpRows + j * 32 + lane, position = start[d] +
// (rows of digit d in earlier warps) + rank.
template <bool SORTM, typename V, typename DigT>
__device__ __forceinline__ void carry_column(const V* __restrict__ src, V* __restrict__ dst,
                                             const uint32_t (&dr)[kPartItems], const uint16_t* s_wc, uint32_t nd,
                                             const uint32_t* s_start, const uint32_t* s_goff, const DigT* s_dig,
                                             uint32_t nk, V* s_col) {
    const unsigned lane = lane_id();
    const uint32_t w = threadIdx.x / kWarp;
#pragma unroll
    for (int j = 0; j < kPartItems; ++j) {
        if (dr[j] != kNoDigit) {
            const uint32_t d = dr[j] & 0xFFFu;
            uint32_t e, pos;
            if constexpr (SORTM) {
                e = w * kWarpRows + j * kWarp + lane;
                pos = s_start[d] + s_wc[w * nd + d] + (dr[j] >> 12);
            } else {
                e = j * kPartThreads + threadIdx.x;
                pos = s_start[d] + (dr[j] >> 12);
            }
            s_col[pos] = __ldcs(src + e);
        }
    }
    __syncthreads();
    for (uint32_t q = threadIdx.x; q < nk; q += blockDim.x) {
        const uint32_t d = s_dig[q];
        dst[s_goff[d] + q] = s_col[q];
    }
    __syncthreads();
}

// Every thread: asks L2 to fetch the carried columns of tile `tl` (one
// 128-byte line per thread and step), a tile ahead of carry_columns reading
// them, so the carry does not wait on DRAM. Addresses stay inside the tile.
// Used in later passes only: measured on GB300, it cut the pass-2 scatters by
// 0.1-0.3 ms but slowed the pass-1 scatters (which stream the caller's
// columns beside the TMA key loads) by 0.7-1.0 ms on the wide, group-by and
// star workloads.
__device__ __forceinline__ void prefetch_columns(const ColCarry& cc, const Tile& tl) {
#pragma unroll 1
    for (int c = 0; c < cc.n; ++c) {
        const char* base = static_cast<const char*>(cc.in[c]) + (size_t)tl.start * cc.bytes[c];
        const uint32_t bytes = tl.len * (uint32_t)cc.bytes[c];
        for (uint32_t off = threadIdx.x * 128u; off < bytes; off += blockDim.x * 128u)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
    }
}

template <bool SORTM, typename DigT>
__device__ __forceinline__ void carry_columns(const ColCarry& cc, uint32_t tstart, const uint32_t (&dr)[kPartItems],
                                              const uint16_t* s_wc, uint32_t nd, const uint32_t* s_start,
                                              const uint32_t* s_goff, const DigT* s_dig, uint32_t nk,
                                              void* s_stage) {
#pragma unroll 1
    for (int c = 0; c < cc.n; ++c) {
        if (cc.bytes[c] == 4)
            carry_column<SORTM>(static_cast<const uint32_t*>(cc.in[c]) + tstart, static_cast<uint32_t*>(cc.out[c]),
                                dr, s_wc, nd, s_start, s_goff, s_dig, nk, static_cast<uint32_t*>(s_stage));
        else
            carry_column<SORTM>(static_cast<const unsigned long long*>(cc.in[c]) + tstart,
                                static_cast<unsigned long long*>(cc.out[c]), dr, s_wc, nd, s_start, s_goff, s_dig,
                                nk, static_cast<unsigned long long*>(s_stage));
    }
}

// The global digit offsets are double-buffered by tile parity, so no barrier
// follows the write-out: the next tile stores its offsets into the other
// buffer while slower threads still write the current tile out.
// At most 64 registers (two CTAs per SM wherever shared memory allows; 64-bit
// keys otherwise take ~100).
template <typename InKey, typename KeyT, bool FIRST>
__global__ void __launch_bounds__(kPartThreads, 2) part_scatter_kernel(PartPass<InKey, KeyT> a, unsigned* err) {
    using Ring = TileRing<InKey, KeyT, FIRST>;
    using P = PassIn<InKey, KeyT, FIRST>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_warp[kPartThreads / kWarp];
    __shared__ uint32_t s_kept;
    const uint32_t nd = 1u << a.bits;
    const bool rows = a.out_idx != nullptr;  // tuple IDs travel with the keys
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + 16);
    uint32_t* s_start = s_cnt + nd;
    uint32_t* s_goff2 = s_start + nd;  // [2][nd]
    const size_t ring_off = align_up(16 + 4 * (size_t)nd * 4, 16);
    const Ring ring = ring_setup<InKey, KeyT, FIRST>(smem, ring_off);
    KeyT* s_key = reinterpret_cast<KeyT*>(smem + ring_off + 2 * P::kBufBytes);
    uint32_t* s_idx = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(s_key) +
                                                  align_up((size_t)kPartTile * sizeof(KeyT), 16));
    uint16_t* s_dig = reinterpret_cast<uint16_t*>(s_idx + kPartTile);
    __syncthreads();

    const uint32_t ntiles = a.tiles ? *a.ntiles_dev : a.ntiles_fixed;
    uint32_t t = blockIdx.x;
    // Global offsets of this CTA's first tile; later ones are loaded one tile
    // ahead into registers (thread i owns digits i, i + blockDim, ...).
    uint32_t goff[kGoffPerThread] = {};
    Tile tl_cur;
    if (t < ntiles) {
        tl_cur = get_tile(a, t);
#pragma unroll
        for (int q = 0; q < kGoffPerThread; ++q) {
            const uint32_t d = threadIdx.x + q * kPartThreads;
            if (d < nd) goff[q] = a.counts[count_index(tl_cur, t, d, a.bits)];
        }
    }
    Tile d_next{};  // warp 0: descriptor of the next tile to issue, loaded one tile early
    if (threadIdx.x < kWarp) {
        if (t < ntiles) issue_tile(ring, a, tl_cur, 0);
        if (t + gridDim.x < ntiles) d_next = get_tile(a, t + gridDim.x);
    }
    for (uint32_t it = 0; t < ntiles; t += gridDim.x, ++it) {
        const int b = it & 1;
        const uint32_t tn = t + gridDim.x;
        if (threadIdx.x < kWarp && tn < ntiles) {
            issue_tile(ring, a, d_next, b ^ 1);
            if (tn + gridDim.x < ntiles) d_next = get_tile(a, tn + gridDim.x);
        }
        uint32_t* s_goff = s_goff2 + b * nd;
        for (uint32_t d = threadIdx.x; d < nd; d += blockDim.x) s_cnt[d] = 0;
#pragma unroll
        for (int q = 0; q < kGoffPerThread; ++q) {
            const uint32_t d = threadIdx.x + q * kPartThreads;
            if (d < nd) s_goff[d] = goff[q];
        }
        const bool ok = mbar_wait(&ring.bar[b], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            ring_abort(ring, b ^ 1, ((it + 1) >> 1) & 1, tn < ntiles, err);
            return;
        }
        const Tile tl = tl_cur;
        if (tn < ntiles) {  // next tile's offsets, consumed next iteration
            tl_cur = get_tile(a, tn);
            if constexpr (!FIRST)
                if (a.cc.n) prefetch_columns(a.cc, tl_cur);
#pragma unroll
            for (int q = 0; q < kGoffPerThread; ++q) {
                const uint32_t d = threadIdx.x + q * kPartThreads;
                if (d < nd) goff[q] = a.counts[count_index(tl_cur, tn, d, a.bits)];
            }
        }
        const auto* kbuf = ring.keys(b) + lead_of(Ring::key_src(a, tl.start));
        const uint32_t* rbuf = nullptr;
        if constexpr (!FIRST)
            if (rows) rbuf = ring.rows(b) + lead_of(a.in_idx + tl.start);

        KeyT kk[kPartItems];
        uint32_t dr[kPartItems];  // (rank << 12) | digit, or kNoDigit
#pragma unroll
        for (int j = 0; j < kPartItems; ++j) {
            const uint32_t e = j * kPartThreads + threadIdx.x;
            dr[j] = kNoDigit;
            if (e < tl.len && tile_key<InKey, KeyT, FIRST>(a, kbuf, e, kk[j]))
                dr[j] = digit_of<false>(kk[j], a.dshift, a.dmask);
        }
#pragma unroll
        for (int j = 0; j < kPartItems; ++j)
            if (dr[j] != kNoDigit) dr[j] |= atomicAdd(&s_cnt[dr[j]], 1u) << 12;
        __syncthreads();

        // s_goff becomes (global offset - tile offset) of each digit
        const uint32_t kept = block_scan_smem(s_cnt, s_start, nd, s_warp, s_goff);
        if (threadIdx.x == 0) s_kept = kept;
        __syncthreads();

#pragma unroll
        for (int j = 0; j < kPartItems; ++j) {
            if (dr[j] != kNoDigit) {
                const uint32_t e = j * kPartThreads + threadIdx.x;
                const uint32_t d = dr[j] & 0xFFFu;
                const uint32_t pos = s_start[d] + (dr[j] >> 12);
                s_key[pos] = kk[j];
                s_dig[pos] = (uint16_t)d;
                if (rows) s_idx[pos] = FIRST ? tl.start + e : rbuf[e];
            }
        }
        __syncthreads();

        // No barrier after the write-out: the next tile stores its offsets
        // into the other s_goff buffer, and its staging writes come after
        // three more barriers, which every thread reaches only once done here.
        const uint32_t nk = s_kept;
        for (uint32_t pos = threadIdx.x; pos < nk; pos += blockDim.x) {
            const uint32_t d = s_dig[pos];
            const uint32_t g = s_goff[d] + pos;
            a.out_key[g] = s_key[pos];
            if (rows) a.out_idx[g] = s_idx[pos];
        }
        // carried columns reuse the key and row staging (contiguous, >= 8 bytes per row)
        if (a.cc.n) {
            __syncthreads();
            carry_columns<false>(a.cc, tl.start, dr, nullptr, nd, s_start, s_goff, s_dig, nk, s_key);
        }
    }
}

// ------------------------------------------------------------ stable sort scatter

template <typename InKey, typename KeyT, bool FIRST>
__host__ __device__ constexpr size_t sort_scatter_smem_bytes(int bits) {
    return align_up(16 + 3 * ((size_t)1 << bits) * sizeof(uint32_t), 16) +
           2 * PassIn<InKey, KeyT, FIRST>::kBufBytes + align_up((size_t)kPartTile * sizeof(KeyT), 16) +
           (size_t)kPartTile * sizeof(uint32_t) + (size_t)kPartTile * sizeof(uint8_t) +
           (size_t)kPartWarps * ((size_t)1 << bits) * sizeof(uint16_t);
}

// One pass of the stable LSD radix sort (the sort of the sort-merge join,
// Sec. 3.2). Same three steps as a partitioning pass, but the digit is taken
// from the key itself and the scatter is stable: every warp owns kWarpRows
// consecutive rows of the tile and ranks them in order, 32 at a time, with
// __match_any_sync against its own per-digit counters; the counters of the
// warps are then scanned in warp order, so rows of equal digit keep their
// input order within the tile, and the [digit][tile] scan keeps tile order.
template <typename InKey, typename KeyT, bool FIRST>
__global__ void __launch_bounds__(kPartThreads, 2) sort_scatter_kernel(PartPass<InKey, KeyT> a, unsigned* err) {
    using Ring = TileRing<InKey, KeyT, FIRST>;
    using P = PassIn<InKey, KeyT, FIRST>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_warp[kPartThreads / kWarp];
    __shared__ uint32_t s_kept;
    const uint32_t nd = 1u << a.bits;
    const bool rows = a.out_idx != nullptr;  // tuple IDs travel with the keys
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem + 16);
    uint32_t* s_start = s_cnt + nd;
    uint32_t* s_goff = s_start + nd;
    const size_t ring_off = align_up(16 + 3 * (size_t)nd * 4, 16);
    const Ring ring = ring_setup<InKey, KeyT, FIRST>(smem, ring_off);
    KeyT* s_key = reinterpret_cast<KeyT*>(smem + ring_off + 2 * P::kBufBytes);
    uint32_t* s_idx = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned char*>(s_key) +
                                                  align_up((size_t)kPartTile * sizeof(KeyT), 16));
    uint8_t* s_dig = reinterpret_cast<uint8_t*>(s_idx + kPartTile);
    uint16_t* s_wc = reinterpret_cast<uint16_t*>(s_dig + kPartTile);  // [warp][digit]
    __syncthreads();

    const unsigned lane = lane_id();
    const uint32_t w = threadIdx.x / kWarp;
    const uint32_t ntiles = a.tiles ? *a.ntiles_dev : a.ntiles_fixed;
    uint32_t t = blockIdx.x;
    uint32_t goff[kGoffPerThread] = {};
    Tile tl_cur;
    if (t < ntiles) {
        tl_cur = get_tile(a, t);
#pragma unroll
        for (int q = 0; q < kGoffPerThread; ++q) {
            const uint32_t d = threadIdx.x + q * kPartThreads;
            if (d < nd) goff[q] = a.counts[count_index(tl_cur, t, d, a.bits)];
        }
    }
    Tile d_next{};  // warp 0: descriptor of the next tile to issue, loaded one tile early
    if (threadIdx.x < kWarp) {
        if (t < ntiles) issue_tile(ring, a, tl_cur, 0);
        if (t + gridDim.x < ntiles) d_next = get_tile(a, t + gridDim.x);
    }
    for (uint32_t it = 0; t < ntiles; t += gridDim.x, ++it) {
        const int b = it & 1;
        const uint32_t tn = t + gridDim.x;
        if (threadIdx.x < kWarp && tn < ntiles) {
            issue_tile(ring, a, d_next, b ^ 1);
            if (tn + gridDim.x < ntiles) d_next = get_tile(a, tn + gridDim.x);
        }
        for (uint32_t d = lane; d < nd; d += kWarp) s_wc[w * nd + d] = 0;
#pragma unroll
        for (int q = 0; q < kGoffPerThread; ++q) {
            const uint32_t d = threadIdx.x + q * kPartThreads;
            if (d < nd) s_goff[d] = goff[q];
        }
        const bool ok = mbar_wait(&ring.bar[b], (it >> 1) & 1);
        if (__syncthreads_or(!ok)) {
            ring_abort(ring, b ^ 1, ((it + 1) >> 1) & 1, tn < ntiles, err);
            return;
        }
        const Tile tl = tl_cur;
        if (tn < ntiles) {
            tl_cur = get_tile(a, tn);
            if constexpr (!FIRST)
                if (a.cc.n) prefetch_columns(a.cc, tl_cur);
#pragma unroll
            for (int q = 0; q < kGoffPerThread; ++q) {
                const uint32_t d = threadIdx.x + q * kPartThreads;
                if (d < nd) goff[q] = a.counts[count_index(tl_cur, tn, d, a.bits)];
            }
        }
        const auto* kbuf = ring.keys(b) + lead_of(Ring::key_src(a, tl.start));
        const uint32_t* rbuf = nullptr;
        if constexpr (!FIRST)
            if (rows) rbuf = ring.rows(b) + lead_of(a.in_idx + tl.start);

        KeyT kk[kPartItems];
        uint32_t dr[kPartItems];  // (rank within this warp's rows << 12) | digit, or kNoDigit
#pragma unroll
        for (int j = 0; j < kPartItems; ++j) {
            const uint32_t e = w * kWarpRows + j * kWarp + lane;
            const bool v = e < tl.len && tile_key<InKey, KeyT, FIRST>(a, kbuf, e, kk[j]);
            const uint32_t d = v ? digit_of<true>(kk[j], a.dshift, a.dmask) : kNoDigit;
            const unsigned peers = __match_any_sync(0xffffffffu, d);
            const uint32_t before = v ? s_wc[w * nd + d] : 0u;
            __syncwarp();
            if (v && (int)lane == __ffs(peers) - 1) s_wc[w * nd + d] = (uint16_t)(before + __popc(peers));
            __syncwarp();
            dr[j] = v ? ((before + __popc(peers & lanemask_lt())) << 12) | d : kNoDigit;
        }
        __syncthreads();
        // per digit: exclusive prefix over the warps in order, and the tile count
        for (uint32_t d = threadIdx.x; d < nd; d += blockDim.x) {
            uint32_t run = 0;
#pragma unroll
            for (int q = 0; q < kPartWarps; ++q) {
                const uint32_t c = s_wc[q * nd + d];
                s_wc[q * nd + d] = (uint16_t)run;
                run += c;
            }
            s_cnt[d] = run;
        }
        __syncthreads();
        // s_goff becomes (global offset - tile offset) of each digit
        const uint32_t kept = block_scan_smem(s_cnt, s_start, nd, s_warp, s_goff);
        if (threadIdx.x == 0) s_kept = kept;
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kPartItems; ++j) {
            if (dr[j] != kNoDigit) {
                const uint32_t e = w * kWarpRows + j * kWarp + lane;
                const uint32_t d = dr[j] & 0xFFFu;
                const uint32_t pos = s_start[d] + s_wc[w * nd + d] + (dr[j] >> 12);
                s_key[pos] = kk[j];
                s_dig[pos] = (uint8_t)d;
                if (rows) s_idx[pos] = FIRST ? tl.start + e : rbuf[e];
            }
        }
        __syncthreads();
        const uint32_t nk = s_kept;
        for (uint32_t pos = threadIdx.x; pos < nk; pos += blockDim.x) {
            const uint32_t d = s_dig[pos];
            const uint32_t g = s_goff[d] + pos;
            a.out_key[g] = s_key[pos];
            if (rows) a.out_idx[g] = s_idx[pos];
        }
        __syncthreads();
        if (a.cc.n) carry_columns<true>(a.cc, tl.start, dr, s_wc, nd, s_start, s_goff, s_dig, nk, s_key);
    }
}

// ------------------------------------------------------------ device-wide scan

struct ScanLen {
    size_t fixed;
    const uint32_t* ntiles_dev;  // when set: length = *ntiles_dev << bits
    int bits;
    __device__ __forceinline__ size_t get() const {
        return ntiles_dev ? ((size_t)*ntiles_dev << bits) : fixed;
    }
};

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* s_warp) {
#pragma unroll
    for (int o = kWarp / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane_id() == 0) s_warp[threadIdx.x / kWarp] = v;
    __syncthreads();
    uint32_t t = 0;
    for (int w = 0; w < (int)(blockDim.x / kWarp); ++w) t += s_warp[w];
    return t;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_reduce_kernel(const uint32_t* __restrict__ data, ScanLen L, uint32_t* __restrict__ block_sums) {
    __shared__ uint32_t s_warp[kScanThreads / kWarp];
    const size_t len = L.get();
    const size_t beg = (size_t)blockIdx.x * kScanChunk;
    uint32_t v = 0;
    for (size_t i = beg + threadIdx.x; i < beg + kScanChunk && i < len; i += blockDim.x) v += data[i];
    v = block_sum(v, s_warp);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = v;
}

// One block: exclusive scan of block_sums[0, nblocks) in place; *total = sum.
__global__ void __launch_bounds__(1024)
    scan_blocksums_kernel(uint32_t* __restrict__ block_sums, uint32_t nblocks, uint32_t* total) {
    __shared__ uint32_t s_in[1024];
    __shared__ uint32_t s_out[1024];
    __shared__ uint32_t s_warp[1024 / kWarp];
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nblocks; base += 1024) {
        const uint32_t i = base + threadIdx.x;
        s_in[threadIdx.x] = i < nblocks ? block_sums[i] : 0u;
        __syncthreads();
        const uint32_t m = nblocks - base < 1024u ? nblocks - base : 1024u;
        const uint32_t t = block_scan_smem(s_in, s_out, m, s_warp);
        __syncthreads();
        if (i < nblocks) block_sums[i] = s_out[threadIdx.x] + carry;
        carry += t;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads)
    scan_apply_kernel(uint32_t* __restrict__ data, ScanLen L, const uint32_t* __restrict__ block_sums) {
    __shared__ uint32_t s_buf[kScanChunk];
    __shared__ uint32_t s_warp[kScanThreads / kWarp];
    const size_t len = L.get();
    const size_t beg = (size_t)blockIdx.x * kScanChunk;
    if (beg >= len) return;
    const uint32_t m = (uint32_t)(len - beg < (size_t)kScanChunk ? len - beg : (size_t)kScanChunk);
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) s_buf[i] = data[beg + i];
    __syncthreads();
    // per-thread run of kScanItems consecutive entries
    const uint32_t lo = threadIdx.x * kScanItems;
    uint32_t local = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (lo + j < m) local += s_buf[lo + j];
    uint32_t x = local;
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < kWarp; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    const int warp = threadIdx.x / kWarp;
    if ((int)lane == kWarp - 1) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = s_warp[lane < kScanThreads / kWarp ? lane : 0];
        if (lane >= kScanThreads / kWarp) v = 0;
#pragma unroll
        for (int o = 1; o < kWarp; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
            if ((int)lane >= o) v += y;
        }
        if (lane < kScanThreads / kWarp) s_warp[lane] = v;
    }
    __syncthreads();
    uint32_t prefix = block_sums[blockIdx.x] + (warp ? s_warp[warp - 1] : 0u) + x - local;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (lo + j < m) {
            const uint32_t v = s_buf[lo + j];
            s_buf[lo + j] = prefix;
            prefix += v;
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) data[beg + i] = s_buf[i];
}

// ------------------------------------------------------------ pass-2 tiling

// From the scanned pass-1 counts, the pass-1 partitions become the pass-2
// segments; each is cut into tiles of kPartTile rows. Every block scans the
// (at most 2^kMaxBits) segment tile counts in shared memory itself; block 0
// writes the segments and the tile count, and the blocks fill the tiles
// grid-stride.
__global__ void __launch_bounds__(1024)
    seg_tiles_kernel(const uint32_t* __restrict__ counts1, uint32_t ntiles1, int b1,
                     const uint32_t* __restrict__ total1, SegInfo* __restrict__ segs,
                     Tile* __restrict__ tiles, uint32_t* __restrict__ ntiles2) {
    __shared__ uint32_t s_nt[1u << kMaxBits];
    __shared__ uint32_t s_base[1u << kMaxBits];
    __shared__ uint32_t s_warp[1024 / kWarp];
    const uint32_t nseg = 1u << b1;
    for (uint32_t s = threadIdx.x; s < nseg; s += blockDim.x) {
        const uint32_t st = ntiles1 ? counts1[(size_t)s * ntiles1] : 0u;
        const uint32_t en = s + 1 < nseg ? (ntiles1 ? counts1[(size_t)(s + 1) * ntiles1] : 0u) : *total1;
        const uint32_t sz = en - st;
        if (blockIdx.x == 0) {
            segs[s].start = st;
            segs[s].size = sz;
        }
        s_nt[s] = (sz + kPartTile - 1) / kPartTile;
    }
    __syncthreads();
    const uint32_t total = block_scan_smem(s_nt, s_base, nseg, s_warp);
    __syncthreads();
    if (blockIdx.x == 0)
        for (uint32_t s = threadIdx.x; s < nseg; s += blockDim.x) {
            segs[s].tile_base = s_base[s];
            segs[s].ntiles = s_nt[s];
        }
    // the segment of tile k is the last s with s_base[s] <= k among segments
    // that have tiles (binary search in shared memory)
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        uint32_t lo = 0, hi = nseg;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (s_base[mid] <= k) lo = mid; else hi = mid;
        }
        // (an empty segment shares its base with the next one, so the last
        // segment whose base is <= k always has tiles)
        const uint32_t j = k - s_base[lo];
        const uint32_t st = ntiles1 ? counts1[(size_t)lo * ntiles1] : 0u;
        const uint32_t sz = (lo + 1 < nseg ? (ntiles1 ? counts1[(size_t)(lo + 1) * ntiles1] : 0u) : *total1) - st;
        Tile tl;
        tl.start = st + j * kPartTile;
        const uint32_t rest = sz - j * kPartTile;
        tl.len = rest < (uint32_t)kPartTile ? rest : (uint32_t)kPartTile;
        tl.seg = lo;
        tl.tile_base = s_base[lo];
        tl.ntiles_seg = s_nt[lo];
        tiles[k] = tl;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *ntiles2 = total;
}

// Blocks of seg_tiles_kernel for at most `max_tiles` pass-2 tiles.
inline int seg_tiles_grid(size_t max_tiles, const DevInfo& di) {
    const size_t g = (max_tiles + 4095) / 4096;
    const size_t cap = (size_t)di.sms * 2;
    return (int)(g < 1 ? 1 : g > cap ? cap : g);
}

// Start of every final partition, plus part_start[P] = rows kept.
__global__ void part_start_kernel(const uint32_t* __restrict__ counts, int passes, uint32_t ntiles1,
                                  int b1, int b2, const SegInfo* __restrict__ segs,
                                  const uint32_t* __restrict__ total, uint32_t* __restrict__ part_start) {
    const uint32_t P = 1u << (b1 + b2);
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p <= P; p += gridDim.x * blockDim.x) {
        uint32_t v;
        if (p == P) {
            v = *total;
        } else if (passes == 1) {
            v = ntiles1 ? counts[(size_t)p * ntiles1] : 0u;
        } else {
            const SegInfo sg = segs[p >> b2];
            const uint32_t d2 = p & ((1u << b2) - 1u);
            v = sg.ntiles ? counts[((size_t)sg.tile_base << b2) + (size_t)d2 * sg.ntiles] : sg.start;
        }
        part_start[p] = v;
    }
}

template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename K>
int occupancy_grid(K kern, int threads, size_t smem, const DevInfo& di, size_t work) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    size_t g = (size_t)di.sms * per_sm;
    if (work < g) g = work;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t scan_counts(uint32_t* counts, ScanLen L, size_t max_len, uint32_t* block_sums,
                        uint32_t* total, cudaStream_t stream) {
    const uint32_t nblocks = (uint32_t)((max_len + kScanChunk - 1) / kScanChunk);
    const uint32_t g = nblocks ? nblocks : 1;
    scan_reduce_kernel<<<g, kScanThreads, 0, stream>>>(counts, L, block_sums);
    scan_blocksums_kernel<<<1, 1024, 0, stream>>>(block_sums, g, total);
    scan_apply_kernel<<<g, kScanThreads, 0, stream>>>(counts, L, block_sums);
    return cudaGetLastError();
}

// Carried-column bytes per row (each is read once and written once per pass).
inline double carry_bytes(const ColCarry& cc) {
    double b = 0;
    for (int c = 0; c < cc.n; ++c) b += cc.bytes[c];
    return b;
}

// One partitioning (or sort) pass over n rows. Algorithmic bytes per launch:
// the histogram reads each key once; the scatter reads each (key, row) once
// and writes each kept (key', row) once (keys alone when the side keeps no
// tuple IDs), plus the carried columns; the scan reads and writes the counts.
template <typename InKey, typename KeyT, bool FIRST, bool SORTM>
cudaError_t run_pass(PartPass<InKey, KeyT> a, size_t max_tiles, const PartSide& s, uint32_t* total,
                     unsigned* err, const DevInfo& di, cudaStream_t stream, const char* side_name, int pass_no) {
    cudaError_t e;
    const size_t hsmem = hist_smem_bytes<InKey, KeyT, FIRST>(a.bits);
    const size_t ssmem = SORTM ? sort_scatter_smem_bytes<InKey, KeyT, FIRST>(a.bits)
                               : scatter_smem_bytes<InKey, KeyT, FIRST>(a.bits);
    auto hist = part_hist_kernel<InKey, KeyT, FIRST, SORTM>;
    auto scat = SORTM ? sort_scatter_kernel<InKey, KeyT, FIRST> : part_scatter_kernel<InKey, KeyT, FIRST>;
    if ((e = set_smem(hist, hsmem)) != cudaSuccess) return e;
    if ((e = set_smem(scat, ssmem)) != cudaSuccess) return e;
    const double n = (double)a.n;
    const double in_key = FIRST ? (double)sizeof(InKey) : (double)sizeof(KeyT);
    const double row = a.out_idx ? (double)sizeof(uint32_t) : 0.0;  // tuple IDs, when the side keeps them
    const double tuple = (double)sizeof(KeyT) + row;
    const double in_tuple = FIRST ? (double)sizeof(InKey) : tuple;
    const char* kind = SORTM ? "sort" : "part";
    char name[32];
    {
        snprintf(name, sizeof name, "%s_hist.p%d.%s", kind, pass_no, side_name);
        ProfScope ps(name, n * in_key, stream);
        hist<<<occupancy_grid(hist, kPartThreads, hsmem, di, max_tiles), kPartThreads, hsmem, stream>>>(a, err);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    ScanLen L{max_tiles << a.bits, a.tiles ? a.ntiles_dev : nullptr, a.bits};
    {
        snprintf(name, sizeof name, "%s_scan.p%d.%s", kind, pass_no, side_name);
        ProfScope ps(name, 12.0 * (double)(max_tiles << a.bits), stream, 0.0, 3);
        if ((e = scan_counts(a.counts, L, max_tiles << a.bits, s.block_sums, total, stream)) != cudaSuccess)
            return e;
    }
    snprintf(name, sizeof name, "%s_scatter.p%d.%s", kind, pass_no, side_name);
    ProfScope ps(name, n * (in_tuple + tuple + 2.0 * carry_bytes(a.cc)), stream);
    scat<<<occupancy_grid(scat, kPartThreads, ssmem, di, max_tiles), kPartThreads, ssmem, stream>>>(a, err);
    return cudaGetLastError();
}

// Carried columns of pass `pass` (0-based) of one side: pass 0 reads the
// caller's columns, later passes the previous pass's copies.
ColCarry carry_for(const PlanDev& plan, int side, const ColSide* carry, const PartSide& s, int pass) {
    ColCarry cc{};
    cc.n = plan.gftr && carry ? plan.ncols[side] : 0;
    for (int c = 0; c < cc.n; ++c) {
        cc.in[c] = pass == 0 ? carry->src[c] : s.col[(pass - 1) & 1][c];
        cc.out[c] = s.col[pass & 1][c];
        cc.bytes[c] = plan.col_bytes[side][c];
    }
    return cc;
}

template <typename InKey, typename KeyT>
cudaError_t partition_typed(const InKey* keys, uint32_t n, int side, const PlanDev& plan, const PartSide& s,
                            const ColSide* carry, unsigned* err, const DevInfo& di, cudaStream_t stream) {
    const int passes = plan.variant == 3 ? 2 : 1;
    const int b1 = plan.bits1, b2 = passes == 2 ? plan.bits2 : 0;
    const uint32_t ntiles1 = (n + kPartTile - 1) / kPartTile;
    cudaError_t e;

    PartPass<InKey, KeyT> a{};
    a.raw = keys;
    a.src_end[0] = keys + n;
    a.out_key = static_cast<KeyT*>(s.key[0]);
    a.out_idx = plan.no_rows ? nullptr : s.idx[0];
    a.n = n;
    a.rng = plan.range;
    a.check_range = side == 1 ? plan.check_range : 0;
    a.dshift = KeyCodec<KeyT>::kBits - b1;
    a.dmask = (1u << b1) - 1u;
    a.bits = b1;
    a.counts = s.counts;
    a.tiles = nullptr;
    a.ntiles_fixed = ntiles1;
    a.cc = carry_for(plan, side, carry, s, 0);
    const char* sn = side == 0 ? "build" : "probe";
    if ((e = run_pass<InKey, KeyT, true, false>(a, ntiles1, s, s.total, err, di, stream, sn, 1)) != cudaSuccess)
        return e;

    if (passes == 2) {
        {
            ProfScope ps("seg_tiles", 0.0, stream);
            const size_t max_tiles2 = (size_t)ntiles1 + ((size_t)1 << b1);
            seg_tiles_kernel<<<seg_tiles_grid(max_tiles2, di), 1024, 0, stream>>>(s.counts, ntiles1, b1, s.total,
                                                                                 s.segs, s.tiles, s.total + 2);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        PartPass<InKey, KeyT> b{};
        b.in_key = static_cast<const KeyT*>(s.key[0]);
        b.in_idx = plan.no_rows ? nullptr : s.idx[0];
        b.src_end[0] = static_cast<const char*>(s.key[0]) + (size_t)n * sizeof(KeyT) + 16;
        b.src_end[1] = s.idx[0] + (size_t)n + 4;
        b.out_key = static_cast<KeyT*>(s.key[1]);
        b.out_idx = plan.no_rows ? nullptr : s.idx[1];
        b.n = n;
        b.rng = plan.range;
        b.check_range = 0;
        b.dshift = KeyCodec<KeyT>::kBits - b1 - b2;
        b.dmask = (1u << b2) - 1u;
        b.bits = b2;
        b.counts = s.counts;
        b.tiles = s.tiles;
        b.ntiles_dev = s.total + 2;
        b.cc = carry_for(plan, side, carry, s, 1);
        const size_t max_tiles2 = (size_t)ntiles1 + ((size_t)1 << b1);
        if ((e = run_pass<InKey, KeyT, false, false>(b, max_tiles2, s, s.total + 1, err, di, stream, sn, 2)) !=
            cudaSuccess)
            return e;
    }
    const uint32_t P = 1u << (b1 + b2);
    const int threads = 256;
    const int blocks = (int)((P + 1 + threads - 1) / threads);
    ProfScope ps("part_start", 8.0 * (P + 1), stream);
    part_start_kernel<<<blocks, threads, 0, stream>>>(s.counts, passes, ntiles1, b1, b2, s.segs, s.total,
                                                      s.part_start);
    return cudaGetLastError();
}

// Stable LSD radix sort of one side (see sort_scatter_kernel): pass 1 reads
// the raw keys (range test and narrowing as in partitioning) with a fixed
// tiling; the kept rows then form one segment, tiled once, which every later
// pass re-reads from the previous pass's buffer.
template <typename InKey, typename KeyT>
cudaError_t sort_typed(const InKey* keys, uint32_t n, int side, const PlanDev& plan, const PartSide& s,
                       const ColSide* carry, unsigned* err, const DevInfo& di, cudaStream_t stream) {
    const int D = plan.bits1, passes = plan.bits2;
    const uint32_t ntiles1 = (n + kPartTile - 1) / kPartTile;
    const char* sn = side == 0 ? "build" : "probe";
    cudaError_t e;
    PartPass<InKey, KeyT> a{};
    a.raw = keys;
    a.src_end[0] = keys + n;
    a.out_key = static_cast<KeyT*>(s.key[0]);
    a.out_idx = plan.no_rows ? nullptr : s.idx[0];
    a.n = n;
    a.rng = plan.range;
    a.check_range = side == 1 ? plan.check_range : 0;
    a.dshift = 0;
    a.dmask = (1u << D) - 1u;
    a.bits = D;
    a.counts = s.counts;
    a.tiles = nullptr;
    a.ntiles_fixed = ntiles1;
    a.cc = carry_for(plan, side, carry, s, 0);
    if ((e = run_pass<InKey, KeyT, true, true>(a, ntiles1, s, s.total, err, di, stream, sn, 1)) != cudaSuccess)
        return e;
    if (passes < 2) return cudaSuccess;
    {
        ProfScope ps("seg_tiles", 0.0, stream);
        seg_tiles_kernel<<<seg_tiles_grid((size_t)ntiles1 + 1, di), 1024, 0, stream>>>(s.counts, ntiles1, 0, s.total,
                                                                                     s.segs, s.tiles, s.total + 2);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int i = 1; i < passes; ++i) {
        PartPass<InKey, KeyT> b{};
        b.in_key = static_cast<const KeyT*>(s.key[(i - 1) & 1]);
        b.in_idx = plan.no_rows ? nullptr : s.idx[(i - 1) & 1];
        b.src_end[0] = static_cast<const char*>(s.key[(i - 1) & 1]) + (size_t)n * sizeof(KeyT) + 16;
        b.src_end[1] = s.idx[(i - 1) & 1] + (size_t)n + 4;
        b.out_key = static_cast<KeyT*>(s.key[i & 1]);
        b.out_idx = plan.no_rows ? nullptr : s.idx[i & 1];
        b.n = n;
        b.rng = plan.range;
        b.check_range = 0;
        b.dshift = i * D;
        b.dmask = (1u << D) - 1u;
        b.bits = D;
        b.counts = s.counts;
        b.tiles = s.tiles;
        b.ntiles_dev = s.total + 2;
        b.cc = carry_for(plan, side, carry, s, i);
        if ((e = run_pass<InKey, KeyT, false, true>(b, ntiles1, s, s.total + 1, err, di, stream, sn, i + 1)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace

size_t part_counts_len(int64_t n, int b1, int b2, int passes) {
    const size_t ntiles1 = (size_t)((n + kPartTile - 1) / kPartTile);
    size_t l1 = ntiles1 << b1;
    size_t l2 = passes == 2 ? (ntiles1 + ((size_t)1 << b1)) << b2 : 0;
    return l1 > l2 ? l1 : l2;
}

size_t part_scan_blocks(size_t counts_len) { return (counts_len + kScanChunk - 1) / kScanChunk + 1; }

void part_side_layout(Carve& c, PartSide& ps, int64_t n, int b1, int b2, int passes, bool sort, size_t kb,
                      const PlanDev& plan, int side) {
    const int nbuf = passes < 2 ? passes : 2;
    const int ncols = plan.gftr ? plan.ncols[side] : 0;
    for (int k = 0; k < 2; ++k) {
        // 16 bytes of slack after each buffer: a later pass's tile loads may
        // read the aligned cover of the last rows (see PartPass::src_end)
        ps.key[k] = k < nbuf ? c.take<unsigned char>((size_t)n * kb + 16) : nullptr;
        ps.idx[k] = k < nbuf ? c.take<uint32_t>((size_t)n + 4) : nullptr;
        for (int q = 0; q < kMaxCols; ++q)
            ps.col[k][q] = (k < nbuf && q < ncols) ? c.take<unsigned char>((size_t)n * plan.col_bytes[side][q])
                                                  : nullptr;
    }
    const size_t ntiles1 = (size_t)((n + kPartTile - 1) / kPartTile);
    ps.counts_len = sort ? ntiles1 << b1 : part_counts_len(n, b1, b2, passes);
    ps.counts = c.take<uint32_t>(ps.counts_len);
    ps.block_sums = c.take<uint32_t>(part_scan_blocks(ps.counts_len));
    ps.total = c.take<uint32_t>(4);
    ps.segs = c.take<SegInfo>(sort ? 1 : (size_t)1 << b1);
    ps.tiles = c.take<Tile>(passes >= 2 ? ntiles1 + (sort ? 1 : ((size_t)1 << b1)) : 1);
    ps.part_start = sort ? nullptr : c.take<uint32_t>(((size_t)1 << (b1 + b2)) + 1);
}

int sort_key_bits(const PlanDev& plan) {
    const uint64_t span = (uint64_t)plan.range.hi - (uint64_t)plan.range.lo;
    int b = 0;
    while (b < 64 && (span >> b) != 0) ++b;
    return b;
}

cudaError_t partition_side(const void* keys, int64_t n, int side, const PlanDev& plan, const PartSide& s,
                           const ColSide* carry, unsigned* err, cudaStream_t stream) {
    DevInfo di;
    cudaError_t e = current_device_info(&di);
    if (e != cudaSuccess) return e;
    const uint32_t nn = (uint32_t)n;
    if (plan.key32) {
        if (plan.dtype == 0)
            return partition_typed<int32_t, uint32_t>(static_cast<const int32_t*>(keys), nn, side, plan, s, carry,
                                                      err, di, stream);
        return partition_typed<int64_t, uint32_t>(static_cast<const int64_t*>(keys), nn, side, plan, s, carry,
                                                  err, di, stream);
    }
    return partition_typed<int64_t, uint64_t>(static_cast<const int64_t*>(keys), nn, side, plan, s, carry, err,
                                              di, stream);
}

cudaError_t sort_side(const void* keys, int64_t n, int side, const PlanDev& plan, const PartSide& s,
                      const ColSide* carry, unsigned* err, cudaStream_t stream) {
    DevInfo di;
    cudaError_t e = current_device_info(&di);
    if (e != cudaSuccess) return e;
    const uint32_t nn = (uint32_t)n;
    if (plan.key32) {
        if (plan.dtype == 0)
            return sort_typed<int32_t, uint32_t>(static_cast<const int32_t*>(keys), nn, side, plan, s, carry, err,
                                                 di, stream);
        return sort_typed<int64_t, uint32_t>(static_cast<const int64_t*>(keys), nn, side, plan, s, carry, err, di,
                                             stream);
    }
    return sort_typed<int64_t, uint64_t>(static_cast<const int64_t*>(keys), nn, side, plan, s, carry, err, di,
                                         stream);
}

}  // namespace eiger
