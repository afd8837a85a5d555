// Match emission shared by the join kernels.
//
// Matches are staged per CTA in shared memory: a warp reserves room for all of
// its matching lanes with one shared-memory atomic (ballot + popc), and the CTA
// reserves room in the global output with one global atomic per flush. That
// keeps the output writes coalesced and the single global cursor cold (one
// atomic per ~thousand matches instead of one per warp). If a CTA produces more
// matches between two flushes than the stage holds (duplicate-heavy keys), the
// lanes that do not fit write straight to global memory with a warp-aggregated
// atomic, so no match is ever lost and no stage size bounds the multiplicity.
//
// In aggregate mode nothing is written: each thread accumulates the payload
// sum and the match count, reduced once per CTA at the end.
#pragma once

#include "common.cuh"

namespace eiger {

template <int STAGE>
struct Stage {
    uint32_t b[STAGE];
    uint32_t p[STAGE];
    unsigned int count;
    unsigned long long base;
};

__device__ __forceinline__ void copy_cols(const ColSide& cs, unsigned long long pos, uint32_t i) {
#pragma unroll 1
    for (int c = 0; c < cs.n; ++c) {
        if (cs.bytes[c] == 4)
            static_cast<uint32_t*>(cs.dst[c])[pos] = __ldg(static_cast<const uint32_t*>(cs.src[c]) + i);
        else
            static_cast<unsigned long long*>(cs.dst[c])[pos] =
                __ldg(static_cast<const unsigned long long*>(cs.src[c]) + i);
    }
}

// Writes match `pos` of the output: b and p are tuple IDs, or positions in
// the transformed relations when the side has a rowmap (GFTR).
__device__ __forceinline__ void write_match(const JoinOut& out, unsigned long long pos, uint32_t b,
                                            uint32_t p) {
    if (pos >= out.capacity) return;
    // outputs are written once and not read back here: streaming stores
    if (out.bidx) __stcs(out.bidx + pos, out.b.rowmap ? __ldg(out.b.rowmap + b) : b);
    if (out.pidx) __stcs(out.pidx + pos, out.p.rowmap ? __ldg(out.p.rowmap + p) : p);
    copy_cols(out.b, pos, b);
    copy_cols(out.p, pos, p);
}

struct AggState {
    unsigned long long sum;
    unsigned long long count;
};

// Warp-collective: all 32 lanes call it; lanes with `has` emit the pair (b, p).
template <bool AGG, int STAGE>
__device__ __forceinline__ void emit(Stage<STAGE>& st, AggState& agg, bool has, uint32_t b,
                                     uint32_t p, const JoinOut& out, unsigned long long* cursor) {
    if (AGG) {
        if (has) {
            agg.sum += (unsigned long long)read_pay(out.b.src[0], out.b.bytes[0], b) +
                       (unsigned long long)read_pay(out.p.src[0], out.p.bytes[0], p);
            agg.count += 1;
        }
        return;
    }
    const unsigned mask = __ballot_sync(0xffffffffu, has);
    if (mask == 0) return;
    const unsigned lane = lane_id();
    const int leader = __ffs(mask) - 1;
    unsigned pos0 = 0;
    if ((int)lane == leader) pos0 = atomicAdd(&st.count, (unsigned)__popc(mask));
    pos0 = __shfl_sync(0xffffffffu, pos0, leader);
    const unsigned pos = pos0 + __popc(mask & lanemask_lt());
    const bool spill = has && pos >= (unsigned)STAGE;
    if (has && !spill) {
        st.b[pos] = b;
        st.p[pos] = p;
    }
    const unsigned smask = __ballot_sync(0xffffffffu, spill);
    if (smask) {
        const int sl = __ffs(smask) - 1;
        unsigned long long g0 = 0;
        if ((int)lane == sl) g0 = atomicAdd(cursor, (unsigned long long)__popc(smask));
        g0 = __shfl_sync(0xffffffffu, g0, sl);
        if (spill) write_match(out, g0 + __popc(smask & lanemask_lt()), b, p);
    }
}

// Block-collective: writes the staged matches out and empties the stage.
template <bool AGG, int STAGE>
__device__ __forceinline__ void stage_flush(Stage<STAGE>& st, const JoinOut& out, unsigned long long* cursor) {
    if (AGG) return;
    __syncthreads();
    const unsigned n = st.count < (unsigned)STAGE ? st.count : (unsigned)STAGE;
    if (threadIdx.x == 0) st.base = n ? atomicAdd(cursor, (unsigned long long)n) : 0ull;
    __syncthreads();
    const unsigned long long base = st.base;
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) write_match(out, base + i, st.b[i], st.p[i]);
    __syncthreads();
    if (threadIdx.x == 0) st.count = 0;
    __syncthreads();
}

// Block-collective: true when the stage may not hold another `room` matches.
// The first barrier orders every emit before the read; the second keeps the
// count unchanged until thread 0 has read it.
template <int STAGE>
__device__ __forceinline__ bool stage_nearly_full(Stage<STAGE>& st, unsigned room) {
    __syncthreads();
    return __syncthreads_or(threadIdx.x == 0 && st.count + room > (unsigned)STAGE) != 0;
}

// Once per thread at kernel end (aggregate mode): warp-reduce, one atomic pair.
__device__ __forceinline__ void agg_commit(AggState& agg, Ctrl* ctrl) {
#pragma unroll
    for (int o = kWarp / 2; o > 0; o >>= 1) {
        agg.sum += __shfl_xor_sync(0xffffffffu, agg.sum, o);
        agg.count += __shfl_xor_sync(0xffffffffu, agg.count, o);
    }
    if (lane_id() == 0 && agg.count) {
        atomicAdd(&ctrl->sum, agg.sum);
        atomicAdd(&ctrl->cursor, agg.count);
    }
}

}  // namespace eiger
