// Internal definitions shared by the CUDA translation units of libeiger.
// Nothing here is part of the public ABI (see include/eiger.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

// Shape of the partitioned join: threads per CTA and build rows per
// shared-memory table (the planner aims at 2048-4096 rows per partition; the
// cap leaves room for the spread of hashed partition sizes around 4096, and
// its table of 2 x 4608 slots of 8 bytes still lets three CTAs share an SM).
#ifndef EIGER_JOIN_THREADS
#define EIGER_JOIN_THREADS 512
#endif
#ifndef EIGER_BUILD_CAP
#define EIGER_BUILD_CAP 4608
#endif

namespace eiger {

// ---------------------------------------------------------------- constants

constexpr int kHllP = 14;              // HyperLogLog precision p (Sec. 4.1)
constexpr int kHllM = 1 << kHllP;      // m = 2^p registers
constexpr int kRhoMax = 64 - kHllP + 1;  // rank when the 50 low hash bits are zero

constexpr unsigned long long kEmptySlot = ~0ull;  // empty hash-table slot / idx word

// Device-side error flags, OR-ed into Ctrl::err and mapped to statuses on the host.
constexpr unsigned kErrTableFull = 1u;  // a probe sequence walked the whole table
constexpr unsigned kErrInternal = 2u;   // a consistency check failed

constexpr int kWarp = 32;

// ---------------------------------------------------------------- hashes

// SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014): the 64-bit
// hash of the HyperLogLog sketch. Applied to the key's 64-bit two's-complement
// pattern, so int32 keys are sign-extended first.
__host__ __device__ __forceinline__ uint64_t sketch_hash(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// MurmurHash3 finalisers (Appleby): bijective avalanche mixers used to place
// keys in hash tables and radix partitions. Partitions take the top bits of the
// mixed key, table slots the low bits, so the two never overlap.
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85EBCA6Bu;
    h ^= h >> 13;
    h *= 0xC2B2AE35u;
    h ^= h >> 16;
    return h;
}

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xFF51AFD7ED558CCDull;
    k ^= k >> 33;
    k *= 0xC4CEB9FE1A85EC53ull;
    k ^= k >> 33;
    return k;
}

// Key encodings carried through the join.
//  - 32-bit: key' = (uint32)(key - offset). offset = build minimum when the
//    build span fits 32 bits (range-offset narrowing, Sec. 4.3 frame of
//    reference), or 0 for raw int32 keys (their bit pattern).
//  - 64-bit: key' = the int64 bit pattern minus offset (mod 2^64): offset 0
//    for hashing; the build minimum for the sort-merge join, which then
//    orders only the span's significant bits.
template <typename KeyT>
struct KeyCodec;

template <>
struct KeyCodec<uint32_t> {
    static constexpr int kBits = 32;
    __device__ __forceinline__ static uint32_t encode(int64_t k, uint64_t offset) {
        return (uint32_t)((uint64_t)k - offset);
    }
    __device__ __forceinline__ static uint32_t hash(uint32_t k) { return mix32(k); }
};

template <>
struct KeyCodec<uint64_t> {
    static constexpr int kBits = 64;
    __device__ __forceinline__ static uint64_t encode(int64_t k, uint64_t offset) { return (uint64_t)k - offset; }
    __device__ __forceinline__ static uint64_t hash(uint64_t k) { return mix64(k); }
};

// Probe-side range test: a key outside [lo, hi] of the build side cannot match.
struct KeyRange {
    int64_t lo, hi;
    uint64_t offset;  // encoding offset (see KeyCodec)
};

// ---------------------------------------------------------------- control

// Small control block at the start of every join workspace.
struct Ctrl {
    unsigned long long cursor;     // matches found (output cursor)
    unsigned long long sum;        // aggregate mode: sum of payload pairs mod 2^64
    unsigned long long next_item;  // PHJ work-item dispenser
    unsigned long long nitems;     // PHJ work items
    unsigned int err;              // kErr* flags
    unsigned int ntiles2[2];       // pass-2 tile count per side (build, probe)
    unsigned int kept[2];          // rows kept by the range test per side
    unsigned int dup;              // non-partitioned build: a key was inserted twice
    unsigned int pad[2];
};

// Payload columns per side a wide join can materialise.
constexpr int kMaxCols = 4;

// The payload columns of one side gathered for every match (Sec. 3.2, payload
// materialisation). With GFUR the sources are the caller's columns and the
// match carries tuple IDs; with GFTR the sources are the partitioned or
// sorted copies of the columns and the match carries positions in them, which
// `rowmap` turns back into tuple IDs for the index outputs.
struct ColSide {
    const void* src[kMaxCols];
    void* dst[kMaxCols];    // outputs, `capacity` rows each
    int bytes[kMaxCols];    // 4 or 8
    int n;                  // columns materialised
    const uint32_t* rowmap; // GFTR: position -> tuple ID; nullptr: matches carry tuple IDs
};

// Output of one join: materialised arrays or a fused aggregate.
struct JoinOut {
    uint32_t* bidx;
    uint32_t* pidx;
    ColSide b, p;
    int aggregate;  // 1: accumulate the sum of b.src[0] + p.src[0] and the count only
    unsigned long long capacity;
};

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & (kWarp - 1); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int64_t read_pay(const void* p, int bytes, uint32_t i) {
    return bytes == 4 ? (int64_t)((const int32_t*)p)[i] : ((const int64_t*)p)[i];
}

__device__ __forceinline__ void write_pay(void* p, int bytes, unsigned long long i, int64_t v) {
    if (bytes == 4)
        ((int32_t*)p)[i] = (int32_t)v;
    else
        ((int64_t*)p)[i] = v;
}

// ---------------------------------------------------------------- cache policies

// An L2 policy that keeps lines resident ahead of normally cached ones: for
// hash tables probed while other data streams through the cache.
__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ unsigned long long ld_keep(const unsigned long long* a, uint64_t pol) {
    unsigned long long v;
    asm volatile("ld.global.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ ulonglong2 ld_keep2(const ulonglong2* a, uint64_t pol) {
    ulonglong2 v;
    asm volatile("ld.global.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;" : "=l"(v.x), "=l"(v.y) : "l"(a), "l"(pol));
    return v;
}

// ---------------------------------------------------------------- TMA bulk copies

// Shared-memory address of a generic pointer into shared memory.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes mbarrier initialisation visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) writes to the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Raises the barrier's expected transaction bytes without arriving.
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// One arrival on the barrier (release: this thread's earlier shared-memory
// writes are visible to threads that then observe the phase complete).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// One-dimensional bulk copy global -> shared, completing on `bar`. Both
// addresses and `bytes` must be multiples of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `bar` with the given parity; false after
// kSpinLimit polls (the caller reports kErrInternal and stops).
constexpr uint32_t kSpinLimit = 1u << 24;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Tile copies: the elements [first, first + len) of a global array go to a
// shared buffer so that element e lands at dst[lead + e], with
// lead = (address of first mod 16) / sizeof(E). The 16-byte aligned body
// [body_lo, body_hi) moves by one bulk copy; the few head and tail elements
// outside it are copied with plain loads by the issuing thread before it
// arrives on the barrier, so waiters see both. Nothing outside the array is
// read. tile_copy_plan returns the bulk bytes for arrive.expect_tx.
template <typename E>
__device__ __forceinline__ uint32_t tile_copy_plan(const E* first, uint32_t len, uint32_t& lead,
                                                   uint32_t& body_lo, uint32_t& body_hi) {
    constexpr uint32_t V = 16 / sizeof(E);
    const uintptr_t a = reinterpret_cast<uintptr_t>(first);
    lead = (uint32_t)((a & 15u) / sizeof(E));
    uint32_t lo = lead ? V - lead : 0u;  // first element index of the aligned body
    if (lo > len) lo = len;
    uint32_t hi = lo + (len - lo) / V * V;
    body_lo = lo;
    body_hi = hi;
    return (hi - lo) * (uint32_t)sizeof(E);
}

template <typename E>
__device__ __forceinline__ void tile_copy_edges(E* dst, const E* first, uint32_t len, uint32_t lead,
                                                uint32_t body_lo, uint32_t body_hi) {
    for (uint32_t e = 0; e < body_lo; ++e) dst[lead + e] = first[e];
    for (uint32_t e = body_hi; e < len; ++e) dst[lead + e] = first[e];
}

template <typename E>
__device__ __forceinline__ void tile_copy_body(E* dst, const E* first, uint32_t lead, uint32_t body_lo,
                                               uint32_t body_hi, uint64_t* bar) {
    if (body_hi > body_lo)
        bulk_load(dst + lead + body_lo, first + body_lo, (body_hi - body_lo) * (uint32_t)sizeof(E), bar);
}

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) {
    return (x + a - 1) / a * a;
}

// Bump allocator over a caller-provided workspace; with base == nullptr it only
// measures, so one layout function serves both the size query and the carving.
struct Carve {
    char* base;
    size_t off;
    template <typename T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

inline int ceil_log2_u64(unsigned long long x) {
    int b = 0;
    while ((1ull << b) < x) ++b;
    return b;
}

// ---------------------------------------------------------------- device info

struct DevInfo {
    int dev;
    int sms;
    int smem_optin;   // max dynamic shared memory per block (opt-in)
    int l2_bytes;
    int max_threads_sm;
};

// Cached properties of the current device; returns cudaSuccess or the error.
cudaError_t current_device_info(DevInfo* out);

}  // namespace eiger
