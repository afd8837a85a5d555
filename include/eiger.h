/*
 * eiger.h -- C ABI of the GB300 runtime-adaptive equi-join library.
 *
 * The library implements the join path of "Eiger: An Efficient Library for
 * GPU-based Data Analytics": it profiles the join keys while the query runs
 * (min/max and a HyperLogLog++ sketch, Sec. 4 and Sec. 4.1), uses those
 * statistics to choose between a non-partitioned global-memory hash join and a
 * radix-partitioned shared-memory hash join and to set their knobs (fanout,
 * passes, table load factor; Sec. 1, Table 1, Sec. 3.2), and compresses int64
 * keys on the fly to uint32 offsets from the build-side minimum when the value
 * range allows (frame-of-reference encoding, Sec. 4.3). The result is the list
 * of matching tuple-ID pairs (Sec. 2.2, late materialisation via TIDs).
 *
 * Names: the paper's R is the build side (the smaller relation), S the probe
 * side; the join throughput is (|R| + |S|) / time (Sec. 5.2).
 *
 * Conventions shared by every entry point
 *  - Pointers prefixed d_ are device memory owned by the caller. The library
 *    never allocates, frees or retains them beyond the call.
 *  - Scratch memory ("workspace") is supplied by the caller; its size comes
 *    from the matching *_workspace query. Contents need not be initialised and
 *    are garbage after the call. The library allocates no device memory; it
 *    keeps one 32 KB page-locked host buffer per calling host thread, made on
 *    first use, for reading small results back (eiger_join_static_noalloc
 *    uses none).
 *  - `stream` is a CUDA stream handle (cudaStream_t / CUstream) passed as
 *    void*; NULL means the legacy default stream. Work is enqueued on it.
 *    Calls that return host-side results (statistics, match counts)
 *    synchronise that stream before returning.
 *  - Row counts are int64. Build and probe sizes must each be < 2^32 (the
 *    output tuple IDs are uint32); larger inputs return EIGER_ERR_INVALID_ARG.
 *  - No CPU fallback exists: every step runs in the library's CUDA kernels. A
 *    CUDA failure returns EIGER_ERR_CUDA with the message in
 *    eiger_last_error().
 *  - Errors leave caller buffers in an unspecified state but never write past
 *    the sizes given. The library stays usable after any error status.
 */
#ifndef EIGER_H
#define EIGER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EIGER_OK = 0,
    EIGER_ERR_INVALID_ARG = 1, /* bad pointer/size/dtype/knob combination          */
    EIGER_ERR_CAPACITY = 2,    /* more matches than `capacity`; *out_count = needed  */
    EIGER_ERR_WORKSPACE = 3,   /* workspace smaller than the *_workspace query says */
    EIGER_ERR_TABLE_FULL = 4,  /* a hash-table probe sequence hit its iteration cap  */
    EIGER_ERR_CUDA = 5,        /* a CUDA runtime call or kernel launch failed        */
    EIGER_ERR_INTERNAL = 6     /* a device-side consistency check failed             */
} eiger_status;

typedef enum { EIGER_I32 = 0, EIGER_I64 = 1 } eiger_dtype;

/* Join variants (Sec. 3.2; Table 1 lists the runtime properties that choose). */
typedef enum {
    EIGER_AUTO = 0,   /* statistics -> planner -> one of NPHJ / PHJ1 / PHJ2           */
    EIGER_NPHJ = 1,   /* non-partitioned hash join, global-memory open addressing    */
    EIGER_PHJ1 = 2,   /* radix-partitioned hash join, 1 partitioning pass            */
    EIGER_PHJ2 = 3,   /* radix-partitioned hash join, 2 partitioning passes          */
    EIGER_STATIC = 4, /* the plain static method: NPHJ with no statistics, no
                         narrowing, load factor 0.5 (the single fixed choice the
                         paper contrasts with adaptivity, Sec. 1 and Sec. 3.2)      */
    EIGER_SMJ = 5     /* sort-merge join: stable LSD radix sort of both sides on
                         the (narrowed) key, then a merge (Sec. 3.2, Sec. 5.3).
                         Chosen only when asked for; the planner never picks it. */
} eiger_variant;

/* Payload materialisation (Sec. 3.2, after Wu et al.): gather the payload
 * columns from the untransformed relations by tuple ID (GFUR), or let them go
 * through the same partitioning / sort as the keys and gather from the
 * transformed relations by position (GFTR; PHJ and SMJ only). */
typedef enum { EIGER_GFUR = 0, EIGER_GFTR = 1, EIGER_MAT_AUTO = 2 } eiger_materialize;

#define EIGER_HLL_P 14
#define EIGER_HLL_M 16384 /* 2^EIGER_HLL_P registers */

/* Column statistics (Sec. 4: min/max; Sec. 4.1: HyperLogLog++ NDV estimate). */
typedef struct {
    int64_t n;        /* rows profiled                                          */
    int64_t min;      /* signed minimum; INT64_MAX when n == 0                   */
    int64_t max;      /* signed maximum; INT64_MIN when n == 0                   */
    double estimate;  /* distinct-value estimate from the registers; 0 when n==0 */
    uint8_t hll[EIGER_HLL_M]; /* dense registers, each the max rank seen (0..51) */
} eiger_stats_t;

/* A join plan: the variant and its knobs (Sec. 1 "knob tuning"). */
typedef struct {
    int32_t variant;     /* EIGER_NPHJ, EIGER_PHJ1, EIGER_PHJ2, EIGER_STATIC or
                            EIGER_SMJ                                                */
    int32_t bits1;       /* PHJ: radix bits of pass 1 (1..12); SMJ: radix bits per
                            sort pass (1..8, 0 on input = 8)                         */
    int32_t bits2;       /* PHJ2: radix bits of pass 2 (1..12); 0 for PHJ1; SMJ:
                            sort passes (set by the library from the key span)       */
    int32_t narrow;      /* 1: keys stored as uint32 offsets from key_min            */
    float load_factor;   /* NPHJ: build rows / table slots, in (0, 0.9]              */
    int32_t selector;    /* who chose: 0 rules, 1 learned model, 2 caller knobs,
                            3 static                                                 */
    int64_t key_min;     /* build-side min/max the plan was made from (filled in by  */
    int64_t key_max;     /* the library; ignored on input)                           */
    int32_t materialize; /* EIGER_GFUR or EIGER_GFTR: how payloads were gathered
                            (filled in by the library; ignored on input)             */
    int32_t reserved;
} eiger_plan_t;

/*
 * Scratch bytes eiger_stats needs for a column of n rows of `dtype`.
 * Errors: INVALID_ARG for n < 0, a bad dtype or bytes == NULL.
 */
eiger_status eiger_stats_workspace(int64_t n, eiger_dtype dtype, size_t* bytes);

/*
 * eiger_stats -- profile one key column (Sec. 4, Sec. 4.1).
 * d_keys:  n keys of `dtype` (int32 or int64), contiguous, any alignment.
 *          An int32 key and the same value as int64 hash identically.
 * out:     host struct; receives n, min, max, the 2^14 HyperLogLog registers and
 *          the estimate. Register update: h = SplitMix64 output function of the
 *          64-bit key; index = top 14 bits of h; rank = 1 + leading zeros of the
 *          remaining 50 bits (51 when they are all zero); register = max rank.
 *          Estimate: the HyperLogLog raw estimate alpha_m m^2 / sum 2^-reg with
 *          linear counting m ln(m/V) when V zero registers remain and the raw
 *          estimate is <= 2.5 m; no bias tables (64-bit hash, no large-range
 *          correction).
 * Synchronises `stream`. n == 0 is legal (see eiger_stats_t).
 * Errors: INVALID_ARG (NULL out, NULL keys with n > 0, n < 0, bad dtype),
 *         WORKSPACE, CUDA.
 */
eiger_status eiger_stats(const void* d_keys, int64_t n, eiger_dtype dtype, eiger_stats_t* out,
                         void* d_workspace, size_t ws_bytes, void* stream);

/*
 * eiger_plan -- the rule-based selector and knob tuner (Sec. 1: statistics drive
 * algorithm selection and knob tuning; Table 1: relation cardinalities and the
 * key distribution decide). Host-only; launches nothing, needs no GPU.
 * build/probe: statistics of the build key column and of a probe sample
 *          (probe may be NULL: only the probe size np is then used; eiger_join
 *          profiles the first 2^20 probe rows when the rules would partition
 *          32-bit keys and np >= 2 nb).
 * out:     the chosen plan (variant never EIGER_AUTO; selector = 0): NPHJ
 *          while its table (load factor 0.5) fits half the L2 cache, or, for
 *          32-bit keys with np >= 2 nb, when the probe sample is heavily
 *          skewed (probe->estimate / probe->n < 0.1, or < 0.5 with the table
 *          within 4x the L2 cache); else PHJ with the fewest radix bits that
 *          keep an average build partition at or below 2048 rows (3072 when
 *          build->estimate >= 0.9 nb, i.e. the keys are distinct; 4096 for
 *          distinct keys from 2^27 rows up), in one pass up to 8 bits, else in
 *          two passes with an odd count's extra bit in the second; narrow = 1
 *          when the build range spans < 2^32.
 * Errors: INVALID_ARG.
 */
eiger_status eiger_plan(const eiger_stats_t* build, const eiger_stats_t* probe, int64_t nb,
                        int64_t np, eiger_dtype dtype, eiger_plan_t* out);

/*
 * Scratch bytes eiger_join needs (and eiger_join_sum with EIGER_GFUR).
 * `variant` and `knobs` as passed to the join; for EIGER_AUTO (or knobs ==
 * NULL with a non-static variant) the result covers every plan the selector
 * can return. Errors: INVALID_ARG.
 */
eiger_status eiger_join_workspace(int64_t nb, int64_t np, eiger_dtype dtype, eiger_variant variant,
                                  const eiger_plan_t* knobs, size_t* bytes);

/*
 * eiger_join -- equi-join R (build) with S (probe) on one key column
 * (Sec. 3.2), emitting every matching pair of tuple IDs.
 * d_bkeys, nb:  build keys (dtype), nb rows.  d_pkeys, np: probe keys.
 * d_bpay, d_ppay, payload_bytes: optional payload columns (4 or 8 bytes per
 *          row; NULL when absent). They are read only when the matching
 *          d_out_*pay output is requested (gather by tuple ID, Sec. 3.2 GFUR).
 * variant: EIGER_AUTO runs eiger_stats on the build keys, then eiger_plan,
 *          then the chosen variant. NPHJ/PHJ1/PHJ2 also profile the build keys
 *          (narrowing and the probe range test need min/max) and take their
 *          knobs from `knobs` when non-NULL (bits1/bits2/narrow/load_factor),
 *          else from the planner. EIGER_STATIC profiles nothing.
 * Outputs (each NULL or an array of `capacity` elements, at least one given):
 *          d_out_bidx / d_out_pidx: uint32 build / probe row of each match;
 *          d_out_bpay / d_out_ppay: the matching rows' payloads (payload_bytes
 *          wide). Match k is entry k of every given array. Order unspecified.
 * out_count: host; receives |J|, the number of matches.
 * capacity: entries available per output array. If |J| > capacity the call
 *          returns EIGER_ERR_CAPACITY, *out_count = |J|, and at most capacity
 *          entries are written (capacity = 0 is a count-only query).
 * plan_used: host, nullable; receives the plan that ran (with key_min/max).
 * Synchronises `stream` (statistics readback and the final count).
 * Errors: INVALID_ARG, CAPACITY, WORKSPACE, TABLE_FULL, CUDA, INTERNAL.
 */
eiger_status eiger_join(eiger_dtype dtype, const void* d_bkeys, const void* d_bpay, int64_t nb,
                        const void* d_pkeys, const void* d_ppay, int64_t np, int32_t payload_bytes,
                        eiger_variant variant, const eiger_plan_t* knobs, uint32_t* d_out_bidx,
                        uint32_t* d_out_pidx, void* d_out_bpay, void* d_out_ppay,
                        int64_t capacity, int64_t* out_count, void* d_workspace, size_t ws_bytes,
                        eiger_plan_t* plan_used, void* stream);

/*
 * Scratch bytes eiger_join_sum needs: arguments as passed to it (the
 * materialisation decides whether the two payload columns are carried).
 * Errors: INVALID_ARG.
 */
eiger_status eiger_join_sum_workspace(int64_t nb, int64_t np, eiger_dtype dtype, int32_t payload_bytes,
                                      eiger_variant variant, eiger_materialize materialize,
                                      const eiger_plan_t* knobs, size_t* bytes);

/*
 * eiger_join_sum -- the join fused with an exact aggregate instead of
 * materialised pairs: sum over matches (i, j) of build_pay[i] + probe_pay[j]
 * (payloads sign-extended to 64 bits), accumulated modulo 2^64 and returned as
 * int64; addition modulo 2^64 is exact and order-independent. This is the
 * foreign-key join whose matched payloads are summed (the star-schema workload
 * shape of the TPC-H joins, Sec. 5.7). Payloads are required.
 * materialize: how the payloads reach the sum (Sec. 3.2). EIGER_GFUR reads
 *          both payloads of every match by tuple ID from the caller's
 *          columns (any variant). EIGER_GFTR carries both columns through the
 *          partitioning (PHJ1/PHJ2) or sort (SMJ) passes and reads them by
 *          position, so the probe side's reads are sequential; rejected for
 *          NPHJ/STATIC. EIGER_MAT_AUTO decides as in eiger_join_wide.
 *          plan_used.materialize reports the strategy that ran.
 * Workspace: eiger_join_sum_workspace. Arguments otherwise as eiger_join.
 * out_sum, out_count: host.
 * Errors: as eiger_join except CAPACITY.
 */
eiger_status eiger_join_sum(eiger_dtype dtype, const void* d_bkeys, const void* d_bpay, int64_t nb,
                            const void* d_pkeys, const void* d_ppay, int64_t np,
                            int32_t payload_bytes, eiger_variant variant, eiger_materialize materialize,
                            const eiger_plan_t* knobs, int64_t* out_sum, int64_t* out_count,
                            void* d_workspace, size_t ws_bytes, eiger_plan_t* plan_used, void* stream);

/* ------------------------------------------------------------------------
 * Wide joins: several payload columns per side (Sec. 3.2 materialisation;
 * Sec. 5.2 "wide join", four columns per relation).
 * ------------------------------------------------------------------------ */
#define EIGER_MAX_COLS 4

/* Payload columns of one side. cols[c]: device, the side's rows; bytes[c]: 4
 * or 8; out[c]: device, `capacity` entries, receives column c of each match's
 * row. Only the first n entries are read. */
typedef struct {
    int32_t n;
    int32_t bytes[EIGER_MAX_COLS];
    const void* cols[EIGER_MAX_COLS];
    void* out[EIGER_MAX_COLS];
} eiger_columns;

/*
 * Scratch bytes eiger_join_wide needs. build/probe: host structs; only n and
 * bytes are read (NULL = no columns). variant, materialize, knobs as passed to
 * the join. Errors: INVALID_ARG.
 */
eiger_status eiger_join_wide_workspace(int64_t nb, int64_t np, eiger_dtype dtype, const eiger_columns* build,
                                       const eiger_columns* probe, eiger_variant variant,
                                       eiger_materialize materialize, const eiger_plan_t* knobs,
                                       size_t* bytes);

/*
 * eiger_join_wide -- eiger_join with up to EIGER_MAX_COLS payload columns per
 * side materialised for every match (Sec. 3.2). Match k is entry k of every
 * output array: out_bidx / out_pidx (nullable) and each column's out[c].
 * variant: as eiger_join, plus EIGER_SMJ.
 * materialize: EIGER_GFUR gathers from the caller's columns by tuple ID (any
 *          variant). EIGER_GFTR carries the columns through the partitioning
 *          passes (PHJ1/PHJ2) or the sort passes (SMJ) and gathers them from
 *          those copies by position; it is rejected for NPHJ/STATIC.
 *          EIGER_MAT_AUTO takes GFTR for a PHJ or SMJ plan when carrying
 *          should move fewer DRAM bytes than gathering (every pass reads and
 *          writes each carried column, against one 32-byte sector per match
 *          and column gathered; matches estimated from the build keys'
 *          distinct count), else GFUR.
 * build, probe: host structs (NULL = no columns); both sides' matched rows
 *          are gathered for every given column.
 * plan_used.materialize reports the strategy that ran.
 * Capacity, counting, synchronisation and errors as eiger_join.
 */
eiger_status eiger_join_wide(eiger_dtype dtype, const void* d_bkeys, int64_t nb, const eiger_columns* build,
                             const void* d_pkeys, int64_t np, const eiger_columns* probe,
                             eiger_variant variant, eiger_materialize materialize, const eiger_plan_t* knobs,
                             uint32_t* d_out_bidx, uint32_t* d_out_pidx, int64_t capacity, int64_t* out_count,
                             void* d_workspace, size_t ws_bytes, eiger_plan_t* plan_used, void* stream);

/* ------------------------------------------------------------------------
 * Group-by (Sec. 3.3), with the algorithm chosen and the hash table sized
 * from the HyperLogLog++ estimate of the number of groups (Sec. 4.2).
 * ------------------------------------------------------------------------ */
typedef enum {
    EIGER_GB_AUTO = 0,      /* estimate the groups, then HASH or PARTITION           */
    EIGER_GB_HASH = 1,      /* one global hash table (CTA-private shared-memory
                               copies first while it is small)                      */
    EIGER_GB_PARTITION = 2  /* radix-partition on hashed keys with the value columns
                               carried along, one shared-memory table per partition */
} eiger_groupby_variant;

typedef enum { EIGER_AGG_SUM = 0, EIGER_AGG_COUNT = 1, EIGER_AGG_MIN = 2, EIGER_AGG_MAX = 3 } eiger_agg_op;

#define EIGER_MAX_AGGS 4

/* Aggregates of a group-by. Aggregate a applies op[a] to value column vals[a]
 * (device, n rows of bytes[a] = 4 or 8, signed; unused for COUNT) and writes
 * one int64 per group to out[a] (device, `capacity` entries). SUM is taken
 * modulo 2^64; MIN and MAX are signed. */
typedef struct {
    int32_t n;
    int32_t op[EIGER_MAX_AGGS];
    int32_t bytes[EIGER_MAX_AGGS];
    const void* vals[EIGER_MAX_AGGS];
    int64_t* out[EIGER_MAX_AGGS];
} eiger_aggs;

/* A group-by plan. */
typedef struct {
    int32_t variant;      /* EIGER_GB_HASH or EIGER_GB_PARTITION                       */
    int32_t bits1;        /* PARTITION: radix bits of pass 1 (1..12)                    */
    int32_t bits2;        /* PARTITION: radix bits of pass 2 (0: one pass; 1..12)      */
    int32_t narrow;       /* 1: keys carried as uint32 offsets from the minimum         */
    int64_t table_slots;  /* HASH: slots of the global table (a power of two)           */
    double estimate;      /* the HyperLogLog++ estimate of the groups (filled in)       */
    int32_t selector;     /* 0 rules, 2 caller knobs                                    */
    int32_t attempts;     /* runs needed: 1, or more when a table overflowed because the
                             estimate was low and the plan was enlarged (filled in)    */
} eiger_groupby_plan_t;

/*
 * Scratch bytes eiger_groupby needs for n keys (aggs: host struct; only n,
 * op and bytes are read). Covers every plan `variant` may take, including the
 * enlarged plans of a retry. Errors: INVALID_ARG.
 */
eiger_status eiger_groupby_workspace(int64_t n, eiger_dtype dtype, const eiger_aggs* aggs, int32_t variant,
                                     size_t* bytes);

/*
 * eiger_groupby -- for every distinct key of d_keys[0, n) its aggregates.
 * Profiles the keys (min/max, HyperLogLog++; Sec. 4.1), narrows them to
 * uint32 offsets when their span allows (Sec. 4.3), then runs:
 *   EIGER_GB_AUTO: HASH when a table of 2.5x the estimated groups fits in half
 *          of the L2 cache, else PARTITION;
 *   EIGER_GB_HASH: slots = the power of two >= 2.5x the estimate (knobs may
 *          set table_slots);
 *   EIGER_GB_PARTITION: 2^B partitions with B = ceil(log2(estimate / 1024)),
 *          one pass up to 10 bits, else two (knobs may set bits1/bits2).
 * If a table overflows (an estimate far too low, or caller knobs too small)
 * the plan is enlarged and the group-by re-run; plan_used->attempts counts the
 * runs. Groups are written in unspecified order: d_out_keys (dtype, nullable
 * when capacity is 0) and aggs->out[a]; *out_groups receives the number of
 * groups. Capacity rules as eiger_join (EIGER_ERR_CAPACITY with the required
 * count). Synchronises `stream`.
 * Errors: INVALID_ARG, CAPACITY, WORKSPACE, TABLE_FULL (the largest plan
 *         still overflowed), CUDA, INTERNAL.
 */
eiger_status eiger_groupby(eiger_dtype dtype, const void* d_keys, int64_t n, const eiger_aggs* aggs,
                           int32_t variant, const eiger_groupby_plan_t* knobs, void* d_out_keys, int64_t capacity,
                           int64_t* out_groups, void* d_workspace, size_t ws_bytes, eiger_groupby_plan_t* plan_used,
                           void* stream);

/* One join of a batch (eiger_join_batched). All pointers are device memory. */
typedef struct {
    const void* build_keys;  /* nb keys of the batch's dtype                 */
    const void* probe_keys;  /* np keys                                      */
    int64_t nb;
    int64_t np;
    uint32_t* out_bidx;      /* capacity entries, or NULL                     */
    uint32_t* out_pidx;      /* capacity entries, or NULL                     */
    int64_t capacity;
} eiger_join_desc;

/* Launch shape of the batched join, chosen by the autotuner. */
typedef struct {
    int32_t block_threads;   /* 128, 256 or 512                               */
    int32_t chunk_rows;      /* rows per work item: 4096, 16384 or 65536      */
    float load_factor;       /* per-join table load, in (0, 0.9]               */
    int32_t small_rows;      /* joins with at most this many build rows run   */
                             /* one CTA per probe chunk, each building the    */
                             /* join's table in its own shared memory; 0:     */
                             /* none; at most EIGER_BATCH_SMALL_MAX_I32 (int32 */
                             /* keys) or EIGER_BATCH_SMALL_MAX_I64 (int64)    */
} eiger_batch_knobs;

#define EIGER_BATCH_SMALL_MAX_I32 2048
#define EIGER_BATCH_SMALL_MAX_I64 1024

/*
 * Scratch bytes eiger_join_batched needs for these joins (host copy of the
 * descriptors; only nb, np are read). knobs NULL = defaults.
 * Errors: INVALID_ARG.
 */
eiger_status eiger_join_batched_workspace(const eiger_join_desc* h_descs, int32_t k, eiger_dtype dtype,
                                          const eiger_batch_knobs* knobs, size_t* bytes);

/*
 * eiger_join_batched -- k independent equi-joins (Sec. 3.2) in one persistent
 * launch. Each join gets its own global open-addressing multiset in the
 * workspace (no statistics: the batch targets many small joins whose tables
 * fit the L2 cache, Sec. 5.2.2 "medium and small joins"); work items are
 * build chunks and probe chunks of every join, interleaved per join and pulled
 * by a persistent grid, a probe chunk waiting (bounded) until its join's build
 * chunks are in. A join with at most knobs.small_rows build rows takes no
 * global table: each of its probe chunks is one item that a single CTA runs
 * whole, with the join's table built in that CTA's shared memory. Join j's matches go to its own outputs in unspecified order;
 * d_counts[j] receives |J_j| (entries beyond capacity are not written).
 * d_descs: k descriptors in device memory. d_counts: k int64, device.
 * d_status: one int32, device: 0 on success, else an eiger_status value
 * (EIGER_ERR_TABLE_FULL, EIGER_ERR_INTERNAL, EIGER_ERR_WORKSPACE).
 * Nothing is synchronised or copied to the host, so the call can be captured
 * in a CUDA graph and replayed; the descriptors and workspace must then stay
 * valid. Host-side errors: INVALID_ARG (bad k, dtype, knobs, NULL pointers),
 * CUDA.
 */
eiger_status eiger_join_batched(eiger_dtype dtype, const eiger_join_desc* d_descs, int32_t k,
                                int64_t* d_counts, int32_t* d_status,
                                const eiger_batch_knobs* knobs, void* d_workspace, size_t ws_bytes,
                                void* stream);

/* ------------------------------------------------------------------------
 * Learned variant selector: a small FP32 network over the runtime statistics
 * (the paper defers algorithm choice to run time and bases it on statistics,
 * Sec. 1 and Sec. 4; here the rule is learned from timings). It changes only
 * which plan runs, never the join result.
 * ------------------------------------------------------------------------ */
#define EIGER_MLP_IN 12      /* features, see eiger_features               */
#define EIGER_MLP_HIDDEN 64
#define EIGER_MLP_OUT 15     /* plan classes, see eiger_class_plan          */

/* Number of float parameters: W1[64][12] b1[64] W2[64][64] b2[64] W3[15][64] b3[15]. */
int32_t eiger_mlp_param_count(void);

/* Logits d_logits[n][15] of the network for features d_x[n][12]. Device arrays. */
eiger_status eiger_mlp_forward(const float* d_params, const float* d_x, int32_t n, float* d_logits,
                               void* stream);

/* Scratch bytes of eiger_mlp_grad for n samples. */
eiger_status eiger_mlp_grad_workspace(int32_t n, size_t* bytes);

/*
 * A training loss over the relative slowdowns d_cost[i][c] of plan class c on
 * sample i (0 for the fastest class), and its gradient with respect to the
 * parameters (d_grad, eiger_mlp_param_count() floats); d_loss (one float,
 * nullable) receives the loss.
 *   tau == 0: the expected regret of the softmax choice,
 *             mean_i sum_c softmax(z_i)_c d_cost[i][c];
 *   tau > 0:  the cross-entropy toward the soft target softmax(-d_cost[i] / tau),
 *             mean_i -sum_c target_ic log softmax(z_i)_c.
 * Deterministic: per-sample gradients are summed in sample order.
 * Errors: INVALID_ARG (NULL arrays with n > 0, tau < 0 or NaN), WORKSPACE, CUDA.
 */
eiger_status eiger_mlp_grad(const float* d_params, const float* d_x, const float* d_cost, int32_t n,
                            float tau, float* d_grad, float* d_loss, void* d_workspace, size_t ws_bytes,
                            void* stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8); step counts from 1. */
eiger_status eiger_mlp_adam(float* d_params, const float* d_grad, float* d_m, float* d_v, int32_t step,
                            float lr, void* stream);

/*
 * The 12 selector features of a join (host only): log2 nb, log2 np,
 * log2(np/nb), key bytes, narrowable, log2(build span + 1),
 * log2(build NDV estimate + 1), build NDV estimate / nb, log2(probe-sample NDV
 * estimate + 1), probe-sample NDV estimate / probe-sample rows, fraction of the
 * probe sample's range inside the build range, log2(non-partitioned table
 * bytes / L2 bytes). probe_sample: statistics of the first min(np, 2^20) probe
 * keys (NULL: treated as empty). l2_bytes 0 = the current device's.
 */
eiger_status eiger_features(const eiger_stats_t* build, const eiger_stats_t* probe_sample, int64_t nb,
                            int64_t np, eiger_dtype dtype, size_t l2_bytes, float out[EIGER_MLP_IN]);

/*
 * Plan of selector class cls (0..14): 0 non-partitioned (load 0.5);
 * 1..5 one radix pass of 8..12 bits; 6..14 two passes of 10..18 bits in total,
 * split ceil/floor. narrow is left 0 (the join decides it from the statistics).
 */
eiger_status eiger_class_plan(int32_t cls, eiger_plan_t* out);

/*
 * Makes EIGER_AUTO (with knobs == NULL) choose the plan with the network:
 * d_params (device, caller-owned, kept until the next call) and per-feature
 * normalisation x' = (x - mean) / scale (host arrays of 12, copied). The join
 * then also profiles a probe sample. d_params == NULL restores the rules.
 * Process-wide setting. Errors: INVALID_ARG.
 */
eiger_status eiger_selector_set(const float* d_params, const float* h_feature_mean,
                                const float* h_feature_scale);

/*
 * eiger_join_static_noalloc -- the static non-partitioned join for callers that
 * cannot allocate device memory. The paper has no counterpart; this entry
 * point exists for code that may not call cudaMalloc or any allocator where it
 * joins (a component whose device memory is owned by someone else's pool, a
 * plug-in host that forbids allocation on its execution path), but can pass
 * arrays it already owns.
 * It computes exactly what eiger_join(..., EIGER_STATIC, ...) computes into
 * d_out_bidx / d_out_pidx (uint32, `capacity` entries each, either may be NULL;
 * same capacity and *out_count rules), without statistics, payloads or a
 * workspace argument, and allocates nothing: its hash table and control block
 * live in one file-scope device array of 8 MiB + 256 bytes that every GPU
 * loading the library holds until the process exits.
 * Limit: build sides up to 2^19 rows for int32 keys, 2^18 rows for int64 keys;
 * larger ones return EIGER_ERR_INVALID_ARG before any GPU work.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before any stream
 * capture begins. Call it under the device's primary context (the CUDA
 * runtime's). All calls on a device share the array and each clears it on
 * its stream first, so consecutive calls are independent, but calls whose
 * work overlaps on the GPU (other streams, other threads) race on it.
 * Synchronises `stream`. Errors: INVALID_ARG, CAPACITY, TABLE_FULL, CUDA,
 * INTERNAL.
 */
eiger_status eiger_join_static_noalloc(eiger_dtype dtype, const void* d_bkeys, int64_t nb,
                                       const void* d_pkeys, int64_t np, uint32_t* d_out_bidx,
                                       uint32_t* d_out_pidx, int64_t capacity, int64_t* out_count,
                                       void* stream);

/* One timed stage (one kernel launch, or the three of a scan) of the last
   call (see eiger_profile). */
typedef struct {
    char name[32];    /* stage name, e.g. "part_scatter.p1.probe"              */
    float ms;         /* device time between CUDA events around the stage     */
    int32_t launches; /* kernels the stage launched (1, or 3 for a scan)      */
    double bytes;     /* algorithmic bytes the stage must move (reads of its
                         inputs plus writes of its outputs, no re-reads)      */
} eiger_stage_t;

/*
 * eiger_profile -- per-launch timing for the calling host thread (the
 * paper's per-kernel breakdowns, Tables of Sec. 5.5-5.6, are this kind of
 * measurement). When enabled, every kernel launch of the following calls is
 * bracketed by CUDA events recorded on the call's stream; the records of the
 * most recent call are kept until the next call. Never fails.
 */
eiger_status eiger_profile(int enable);

/*
 * eiger_profile_read -- copies up to max_stages records of the most recent
 * call on this thread into `out` (host array) and returns how many the call
 * made (out == NULL: only the count). The call's stream must have completed
 * (every join/stats call synchronises it before returning).
 */
int eiger_profile_read(eiger_stage_t* out, int max_stages);

/* Message of the last non-OK status returned on the calling host thread. */
const char* eiger_last_error(void);

/* Version string of the library build. */
const char* eiger_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EIGER_H */
