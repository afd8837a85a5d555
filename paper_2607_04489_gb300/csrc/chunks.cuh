// Barrier-free output of index pairs through per-warp chunks.
//
// Every warp owns a run of kOutChunk consecutive output positions, reserved
// with one global atomic on the output cursor, and fills it in order with its
// matches (ballot, rank, store: no shared memory, no CTA barrier). When the
// run is used up the warp reserves the next one. At kernel end every warp
// records its last run (start, used); the other runs it reserved are full.
//
// The positions a warp reserved but did not fill are holes. After the kernel,
// chunks_fix moves the matches stored at or above the final match count C into
// the holes below C, so the pairs are dense in [0, C) again and the cursor
// holds C. Reserved positions at or above the caller's capacity go to an
// overflow area of the workspace (kMaxOutWarps x kOutChunk pairs), never to
// the caller's arrays; when C exceeds the capacity the call reports the count
// only and nothing is moved.
#pragma once

#include "common.cuh"

namespace eiger {

constexpr uint32_t kOutChunk = 512;       // positions per warp reservation
constexpr uint32_t kMaxOutWarps = 10240;  // warps of one chunked launch (grid x warps per CTA)

struct ChunkRec {
    unsigned long long base;  // start of the warp's last run, ~0 when it reserved none
    uint32_t used;            // positions filled in it
    uint32_t pad;
};

// Destination of the pairs: the caller's arrays below `capacity`, the
// workspace overflow above it.
struct PairSink {
    uint32_t* bidx;
    uint32_t* pidx;
    unsigned long long capacity;
    uint32_t* ovf_b;  // [kMaxOutWarps * kOutChunk]
    uint32_t* ovf_p;
    unsigned long long* cursor;  // positions reserved so far (a multiple of kOutChunk)
    ChunkRec* rec;               // [kMaxOutWarps]
};

// Warp-uniform state of a warp's current run.
struct WarpChunk {
    unsigned long long base;
    uint32_t used;
    __device__ __forceinline__ void init() {
        base = ~0ull;
        used = kOutChunk;
    }
};

__device__ __forceinline__ void sink_store(const PairSink& s, unsigned long long pos, uint32_t b, uint32_t p) {
    if (pos < s.capacity) {
        __stcs(s.bidx + pos, b);
        __stcs(s.pidx + pos, p);
    } else if (pos - s.capacity < (unsigned long long)kMaxOutWarps * kOutChunk) {
        s.ovf_b[pos - s.capacity] = b;
        s.ovf_p[pos - s.capacity] = p;
    }
}

// Warp-collective (all 32 lanes): lanes with `has` emit the pair (b, p).
__device__ __forceinline__ void warp_emit(WarpChunk& wc, const PairSink& s, bool has, uint32_t b, uint32_t p) {
    const unsigned mask = __ballot_sync(0xffffffffu, has);
    if (mask == 0) return;
    const uint32_t n = __popc(mask);
    const uint32_t rank = __popc(mask & lanemask_lt());
    const uint32_t room = kOutChunk - wc.used;
    unsigned long long pos = wc.base + wc.used + rank;
    if (n > room) {  // warp-uniform: the run is used up, reserve the next one
        unsigned long long nb = 0;
        if (lane_id() == 0) nb = atomicAdd(s.cursor, (unsigned long long)kOutChunk);
        nb = __shfl_sync(0xffffffffu, nb, 0);
        if (rank >= room) pos = nb + (rank - room);
        wc.base = nb;
        wc.used = n - room;
    } else {
        wc.used += n;
    }
    if (has) sink_store(s, pos, b, p);
}

// Lane 0 records the warp's last run; `gwarp` < kMaxOutWarps.
__device__ __forceinline__ void warp_chunk_commit(const WarpChunk& wc, const PairSink& s, uint32_t gwarp) {
    if (lane_id() == 0) {
        ChunkRec r;
        r.base = wc.base;
        r.used = wc.base == ~0ull ? 0u : wc.used;
        r.pad = 0;
        s.rec[gwarp] = r;
    }
}

}  // namespace eiger
