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
double match_bytes(const JoinOut& out);

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
    int variant;      // EIGER_NPHJ / PHJ1 / PHJ2 / STATIC
    int bits1, bits2;
    int narrow;       // frame-of-reference narrowing applied (offset = build min)
    int key32;        // keys carried as 32-bit values (int32, or int64 narrowed)
    float load_factor;
    int dtype;        // 0 int32, 1 int64
    KeyRange range;   // build range (probe range test) and encoding offset
    int check_range;  // 1 when `range` holds real statistics
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

// Buffers of one side (build or probe) of the partitioned join.
struct PartSide {
    void* key[2];        // ping-pong key buffers (uint32 or uint64 per row)
    uint32_t* idx[2];    // matching tuple-ID buffers
    uint32_t* counts;    // per-(tile, digit) counts, scanned in place
    uint32_t* block_sums;
    uint32_t* total;     // [2] kept rows after pass 1 / pass 2
    SegInfo* segs;       // pass-2 segments (pass-1 partitions)
    Tile* tiles;         // pass-2 tiles
    uint32_t* part_start;  // [P + 1] final partition starts
    size_t counts_len;
};

struct PhjScratch {
    PartSide side[2];
    unsigned long long* item_prefix;  // [P + 1]
};

PhjScratch phj_layout(Carve& c, int64_t nb, int64_t np, const PlanDev& plan);

// Radix-partitions one side into s.key/idx[passes - 1] and fills
// s.part_start. side: 0 build, 1 probe (only the probe side is range-tested).
cudaError_t partition_side(const void* keys, int64_t n, int side, const PlanDev& plan,
                           const PartSide& s, unsigned* err, cudaStream_t stream);
cudaError_t phj_run(const JoinArgs& a, const PlanDev& plan, const PhjScratch& s, const JoinOut& out,
                    Ctrl* ctrl, cudaStream_t stream);

// ------------------------------------------------------------------ selector network

int mlp_param_count();
size_t mlp_grad_ws_bytes(int n);
cudaError_t mlp_forward(const float* P, const float* X, int n, float* Z, cudaStream_t s);
cudaError_t mlp_grad(const float* P, const float* X, const float* C, int n, float* grad, float* loss, void* ws,
                     cudaStream_t s);
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
    unsigned long long* item_prefix;  // [k + 1]
    unsigned* built;                  // [k]
    unsigned char* tables;
    unsigned long long table_slots;   // capacity of `tables` in slots
};

BatchLayout batch_layout(Carve& c, int k, unsigned long long total_slots, int slot_bytes);
cudaError_t batch_run(const eiger_join_desc* d_descs, int k, int dtype, const eiger_batch_knobs& knobs,
                      const BatchLayout& L, long long* d_counts, int* d_status, cudaStream_t stream);

}  // namespace eiger
