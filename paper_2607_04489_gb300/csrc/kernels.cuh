// Internal launcher declarations and workspace layouts of libeiger.
#pragma once

#include "common.cuh"
#include "eiger.h"

namespace eiger {

// ------------------------------------------------------------------ profiling

// Optional per-launch timing (eiger_profile): when enabled on the calling host
// thread, every kernel launch of a call is bracketed by CUDA events on its
// stream, tagged with a name and the launch's algorithmic bytes. Disabled, a
// scope costs one thread-local branch.
struct ProfScope {
    // bytes: fixed algorithmic bytes; per_match: bytes added for every match of
    // the call (output writes), resolved once the match count is known.
    ProfScope(const char* name, double bytes, cudaStream_t stream, double per_match = 0.0,
              int launches = 1);
    ~ProfScope();
    cudaStream_t stream;
    int slot;
};
void prof_reset();
void prof_set_matches(unsigned long long m);
bool prof_set_enabled(bool on);  // returns the previous setting
bool prof_enabled();
double match_bytes(const JoinOut& out);

// ------------------------------------------------------------------ streams

// A second stream of the calling host thread on the current device, for work
// of a call that can run beside the main stream (the build and probe sides'
// partitioning). fork_side makes it wait for everything enqueued on `main`;
// join_side makes `main` wait for everything enqueued on it. Created once per
// host thread and device; no device memory is allocated. While per-launch
// profiling is on, fork_side returns `main` itself, so every timed launch runs
// alone and its events time that kernel only.
cudaError_t fork_side(cudaStream_t main, cudaStream_t* side);
cudaError_t join_side(cudaStream_t main, cudaStream_t side);

// ------------------------------------------------------------------ stats

constexpr int kStatsMaxGrid = 512;

struct StatsDev {
    int64_t mn;
    int64_t mx;
    uint32_t regs[kHllM / 4];  // register bytes, 4 per word, little-endian order
};

struct StatsScratch {
    uint32_t* part_regs;  // [kStatsMaxGrid][kHllM/4]
    int64_t* part_mm;     // [kStatsMaxGrid][2]
    StatsDev* out;
};

StatsScratch stats_layout(Carve& c);
cudaError_t stats_launch(const void* keys, int64_t n, int dtype, const StatsScratch& s,
                         cudaStream_t stream);

// ------------------------------------------------------------------ plans

// Resolved plan handed to the variant launchers.
struct PlanDev {
    int variant;      // EIGER_NPHJ / PHJ1 / PHJ2 / STATIC / SMJ
    int bits1, bits2; // PHJ: radix bits per pass; SMJ: digit bits per sort pass, sort passes
    int narrow;       // frame-of-reference narrowing applied (offset = build min)
    int key32;        // keys carried as 32-bit values (int32, or int64 narrowed)
    float load_factor;
    int dtype;        // 0 int32, 1 int64
    KeyRange range;   // build range (probe range test) and encoding offset
    int check_range;  // 1 when `range` holds real statistics
    int gftr;         // payload columns travel with the keys (GFTR) instead of being gathered by tuple ID
    int ncols[2];     // GFTR: columns carried per side (build, probe)
    int col_bytes[2][kMaxCols];
    int no_rows;      // the consumer reads rows by position only: the passes keep no tuple IDs
};

// Inputs of one join, as given to eiger_join.
struct JoinArgs {
    const void* bkeys;
    int64_t nb;
    const void* pkeys;
    int64_t np;
};

// ------------------------------------------------------------------ NPHJ

struct NphjScratch {
    void* table;
    unsigned long long slots;  // power of two
    int slot_bytes;            // 8 (packed 32-bit key + idx) or 16 (64-bit key, idx)
};

unsigned long long nphj_slots(int64_t nb, float load_factor);
NphjScratch nphj_layout(Carve& c, int64_t nb, const PlanDev& plan);
cudaError_t nphj_run(const JoinArgs& a, const PlanDev& plan, const NphjScratch& s,
                     const JoinOut& out, Ctrl* ctrl, cudaStream_t stream);

// ------------------------------------------------------------------ PHJ

#ifndef EIGER_PART_TILE
#define EIGER_PART_TILE 4096
#endif
constexpr int kPartTile = EIGER_PART_TILE;  // rows per partitioning tile
constexpr int kMaxBits = 12;     // radix bits per pass

struct Tile {
    uint32_t start, len, seg, tile_base, ntiles_seg;
};

struct SegInfo {
    uint32_t start, size, tile_base, ntiles;
};

// Buffers of one side (build or probe) of the partitioned join or of the
// sort of the sort-merge join.
struct PartSide {
    void* key[2];        // ping-pong key buffers (uint32 or uint64 per row)
    uint32_t* idx[2];    // matching tuple-ID buffers
    void* col[2][kMaxCols];  // GFTR: ping-pong copies of the carried payload columns
    uint32_t* counts;    // per-(tile, digit) counts, scanned in place
    uint32_t* block_sums;
    uint32_t* total;     // [2] kept rows after pass 1 / pass 2
    SegInfo* segs;       // pass-2 segments (pass-1 partitions)
    Tile* tiles;         // pass-2 tiles
    uint32_t* part_start;  // [P + 1] final partition starts
    size_t counts_len;
};

// Scratch of the compaction that follows a chunked pairs launch (chunks.cu).
struct ChunkFix {
    unsigned long long* hdr;  // [4]: moves, match count C, first run index at or above C, runs at or above C
    uint32_t* hb_pref;        // [kMaxOutWarps + 1] holes below C per warp record, exclusive prefix
    uint32_t* va_pref;        // [kMaxOutWarps + 2] filled positions at or above C per run, exclusive prefix
    uint32_t* used_above;     // [kMaxOutWarps + 2] fill of every run at or above C
};

struct PairSink;
ChunkFix chunk_fix_layout(Carve& c);
// Makes the pairs of a chunked launch of W warps dense in [0, C) and sets the
// cursor to C (two launches on `stream`).
cudaError_t chunk_fix_run(const PairSink& s, uint32_t W, const ChunkFix& f, unsigned* err, const DevInfo& di,
                          cudaStream_t stream);

struct PhjScratch {
    PartSide side[2];
    unsigned long long* item_prefix;  // [P + 1]
    // pairs output (chunks.cuh): warp records, overflow above the capacity, compaction scratch
    void* rec;
    uint32_t* ovf[2];
    ChunkFix fix;
};

PhjScratch phj_layout(Carve& c, int64_t nb, int64_t np, const PlanDev& plan);

// Radix-partitions one side into s.key/idx[passes - 1] and fills
// s.part_start. side: 0 build, 1 probe (only the probe side is range-tested).
// With plan.gftr the columns `carry->src[0, plan.ncols[side])` travel along
// into s.col[passes - 1].
cudaError_t partition_side(const void* keys, int64_t n, int side, const PlanDev& plan,
                           const PartSide& s, const ColSide* carry, unsigned* err, cudaStream_t stream);
// Carves the buffers of one side: ping-pong keys, tuple IDs and carried
// columns for `passes` passes, the counts of b1 (+ b2) radix bits, segments,
// tiles and partition starts (none for a sort, whose passes all take b1 bits).
void part_side_layout(Carve& c, PartSide& ps, int64_t n, int b1, int b2, int passes, bool sort, size_t kb,
                      const PlanDev& plan, int side);

// The output of a GFTR join: the payload sources become the transformed
// copies in buffer `buf` of each side, and the tuple IDs of the index outputs
// are looked up at the emitted positions.
inline JoinOut gftr_out(const JoinOut& out, const PartSide& b, const PartSide& p, int buf) {
    JoinOut o = out;
    for (int c = 0; c < o.b.n; ++c) o.b.src[c] = b.col[buf][c];
    for (int c = 0; c < o.p.n; ++c) o.p.src[c] = p.col[buf][c];
    o.b.rowmap = b.idx[buf];
    o.p.rowmap = p.idx[buf];
    return o;
}

// ------------------------------------------------------------------ SMJ

constexpr int kSortMaxBits = 8;  // digit bits per sort pass

// Significant bits of the encoded build keys (their span), the number of
// bits a sort must order.
int sort_key_bits(const PlanDev& plan);

// Stable LSD radix sort of one side on the encoded keys: plan.bits2 passes of
// plan.bits1 bits from the least significant end; the result (with tuple IDs
// and carried columns) is in buffer (passes - 1) & 1; s.total[0] = rows kept.
cudaError_t sort_side(const void* keys, int64_t n, int side, const PlanDev& plan, const PartSide& s,
                      const ColSide* carry, unsigned* err, cudaStream_t stream);

struct SmjScratch {
    PartSide side[2];
    uint32_t* window;  // [chunks][2] build window of every probe chunk
};
SmjScratch smj_layout(Carve& c, int64_t nb, int64_t np, const PlanDev& plan);
cudaError_t smj_run(const JoinArgs& a, const PlanDev& plan, const SmjScratch& s, const JoinOut& out,
                    Ctrl* ctrl, cudaStream_t stream);
cudaError_t phj_run(const JoinArgs& a, const PlanDev& plan, const PhjScratch& s, const JoinOut& out,
                    Ctrl* ctrl, cudaStream_t stream);

// ------------------------------------------------------------------ group-by

struct GbArgs {
    const void* keys;
    int64_t n;
    int dtype;
};

// Resolved group-by plan.
struct GbPlanDev {
    int variant;               // EIGER_GB_HASH or EIGER_GB_PARTITION
    int bits1, bits2;          // partition: radix bits per pass (bits2 = 0: one pass)
    int key32;                 // keys carried as 32-bit offsets
    uint64_t offset;           // key minimum (frame of reference)
    unsigned long long slots;  // hash: global table slots (power of two)
    int smem;                  // hash: aggregate in a CTA-private shared-memory copy first
    int naggs;
};

struct GbAggs {
    int n;
    int op[kMaxCols];
    const void* vals[kMaxCols];
    int bytes[kMaxCols];
    long long* out[kMaxCols];
};

struct GbScratch {
    void* table;   // hash: keys, aggregates, special flag
    PartSide part; // partition: the partitioned keys and carried value columns
    void* spill;                       // partition: table of the groups of multi-item partitions
    unsigned long long spill_max;      // its capacity in slots
    unsigned long long* spill_slots;   // its size, decided on the device
    unsigned long long* item_prefix;   // [P + 1] work items per partition, prefix
};

// Shared-memory bytes of a CTA-private table of `slots` slots.
size_t gb_smem_table_bytes(unsigned long long slots, int naggs, bool key32);
GbScratch gb_layout(Carve& c, int64_t n, const GbPlanDev& plan, const int* col_bytes, int ncols);
cudaError_t gb_run(const GbArgs& g, const GbPlanDev& plan, const GbScratch& s, const GbAggs& aggs, void* out_keys,
                   unsigned long long capacity, Ctrl* ctrl, cudaStream_t stream);

// ------------------------------------------------------------------ selector network

int mlp_param_count();
size_t mlp_grad_ws_bytes(int n);
cudaError_t mlp_forward(const float* P, const float* X, int n, float* Z, cudaStream_t s);
cudaError_t mlp_grad(const float* P, const float* X, const float* C, int n, float tau, float* grad, float* loss,
                     void* ws, cudaStream_t s);
cudaError_t mlp_adam(float* P, const float* grad, float* M, float* V, int step, float lr, cudaStream_t s);

// Learned selector state and helpers (selector.cu).
bool selector_get(const float** params, float* mean, float* scale);
void compute_features(const eiger_stats_t* b, const eiger_stats_t* ps, int64_t nb, int64_t np, int dtype,
                      size_t l2, float* f);
eiger_plan_t class_plan(int cls);

// ------------------------------------------------------------------ batches

struct BatchLayout {
    unsigned char* ctrl;
    unsigned char* meta;
    unsigned long long* item_prefix;  // [k + 3] item prefix of the k + 2 stages
    unsigned long long* solo_prefix;  // [k + 1] item prefix of the small joins
    unsigned* built;                  // [k] build rows inserted per join
    unsigned* cleared;                // [k] clear items done per join
    unsigned* dup;                    // [k] 1 when a join's build keys repeat
    unsigned char* tables;
    unsigned long long table_slots;   // capacity of `tables` in slots
};

BatchLayout batch_layout(Carve& c, int k, unsigned long long total_slots, int slot_bytes);
cudaError_t batch_run(const eiger_join_desc* d_descs, int k, int dtype, const eiger_batch_knobs& knobs,
                      const BatchLayout& L, long long* d_counts, int* d_status, cudaStream_t stream);

}  // namespace eiger
