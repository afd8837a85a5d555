// C ABI of libeiger (declared in include/eiger.h): argument validation,
// workspace carving, the statistics -> plan -> variant pipeline, and the
// mapping of CUDA and device-side errors to statuses.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>

#include "kernels.cuh"
#include "planner.h"

namespace eiger {

cudaError_t current_device_info(DevInfo* out) {
    static std::mutex mu;
    static DevInfo cache[64];
    static bool have[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    if (dev >= 0 && dev < 64 && have[dev]) {
        *out = cache[dev];
        return cudaSuccess;
    }
    DevInfo d;
    d.dev = dev;
    if ((e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
        cudaSuccess)
        return e;
    if ((e = cudaDeviceGetAttribute(&d.l2_bytes, cudaDevAttrL2CacheSize, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&d.max_threads_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev)) !=
        cudaSuccess)
        return e;
    if (dev >= 0 && dev < 64) {
        cache[dev] = d;
        have[dev] = true;
    }
    *out = d;
    return cudaSuccess;
}

namespace {

struct SideStreams {
    cudaStream_t side[64] = {};
    cudaEvent_t fork[64] = {};
    cudaEvent_t join[64] = {};
};
thread_local SideStreams g_side;

// Page-locked, device-mapped host staging for the small results a call reads
// back (the statistics, the control block). A kernel stores them straight
// into host memory, so the readback never waits in a copy engine's queue
// behind the caller's bulk transfers (a 16 KB copy queued behind a multi-GB
// download of a previous batch's pairs waits for all of it). One buffer per
// host thread, allocated on first use and kept until exit; when it cannot be
// had, the result is copied into the caller's destination by cudaMemcpyAsync.
constexpr size_t kStageBytes = 32 << 10;
thread_local void* g_host_stage = nullptr;
thread_local bool g_host_stage_failed = false;

void* host_stage(size_t bytes) {
    if (bytes > kStageBytes || g_host_stage_failed) return nullptr;
    if (!g_host_stage) {
        if (cudaHostAlloc(&g_host_stage, kStageBytes, cudaHostAllocPortable | cudaHostAllocMapped) != cudaSuccess) {
            cudaGetLastError();
            g_host_stage = nullptr;
            g_host_stage_failed = true;
        }
    }
    return g_host_stage;
}

// One CTA stores `words` 32-bit words of device memory into mapped host memory.
__global__ void __launch_bounds__(256) store_to_host_kernel(uint32_t* __restrict__ dst,
                                                            const uint32_t* __restrict__ src, uint32_t words) {
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
}

}  // namespace

// Small result from device memory to `dst` on `stream`, then a synchronisation
// of the stream: stored by a kernel into the mapped staging buffer when it
// exists (bytes a multiple of 4), else copied by cudaMemcpyAsync.
cudaError_t readback_sync(void* dst, const void* src, size_t bytes, cudaStream_t stream) {
    void* st = bytes % 4 == 0 ? host_stage(bytes) : nullptr;
    void* st_dev = nullptr;
    if (st && cudaHostGetDevicePointer(&st_dev, st, 0) != cudaSuccess) {
        cudaGetLastError();
        st_dev = nullptr;
    }
    cudaError_t e;
    if (st_dev) {
        store_to_host_kernel<<<1, 256, 0, stream>>>(static_cast<uint32_t*>(st_dev), static_cast<const uint32_t*>(src),
                                                   (uint32_t)(bytes / 4));
        e = cudaGetLastError();
    } else {
        e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess && st_dev) std::memcpy(dst, st, bytes);
    return e;
}

cudaError_t fork_side(cudaStream_t main, cudaStream_t* side) {
    if (prof_enabled()) {
        *side = main;
        return cudaSuccess;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_side.side[dev]) {
        if ((e = cudaStreamCreateWithFlags(&g_side.side[dev], cudaStreamNonBlocking)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&g_side.fork[dev], cudaEventDisableTiming)) != cudaSuccess) return e;
        if ((e = cudaEventCreateWithFlags(&g_side.join[dev], cudaEventDisableTiming)) != cudaSuccess) return e;
    }
    if ((e = cudaEventRecord(g_side.fork[dev], main)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(g_side.side[dev], g_side.fork[dev], 0)) != cudaSuccess) return e;
    *side = g_side.side[dev];
    return cudaSuccess;
}

cudaError_t join_side(cudaStream_t main, cudaStream_t side) {
    if (side == main) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || side != g_side.side[dev]) return cudaErrorInvalidValue;
    if ((e = cudaEventRecord(g_side.join[dev], side)) != cudaSuccess) return e;
    return cudaStreamWaitEvent(main, g_side.join[dev], 0);
}

}  // namespace eiger

using namespace eiger;

namespace {

thread_local std::string g_last_error;

eiger_status fail(eiger_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

eiger_status cuda_fail(cudaError_t e, const char* where) {
    return fail(EIGER_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define EIGER_CUDA(call, where)                          \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

constexpr int64_t kMaxRows = 0xFFFFFFFFll;  // rows < 2^32: tuple IDs are uint32
static_assert(EIGER_MAX_COLS == kMaxCols, "column limit of the ABI and the kernels");

size_t l2_bytes_or_default() {
    DevInfo di;
    if (current_device_info(&di) == cudaSuccess && di.l2_bytes > 0) return (size_t)di.l2_bytes;
    cudaGetLastError();
    return (size_t)126 << 20;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

eiger_status run_stats(const void* keys, int64_t n, int dtype, const StatsScratch& ss,
                       cudaStream_t stream, eiger_stats_t* out) {
    out->n = n;
    if (n == 0) {
        out->min = INT64_MAX;
        out->max = INT64_MIN;
        std::memset(out->hll, 0, sizeof out->hll);
        out->estimate = 0.0;
        return EIGER_OK;
    }
    EIGER_CUDA(stats_launch(keys, n, dtype, ss, stream), "statistics kernels");
    static thread_local StatsDev host;
    EIGER_CUDA(readback_sync(&host, ss.out, sizeof(StatsDev), stream), "statistics readback");
    out->min = host.mn;
    out->max = host.mx;
    std::memcpy(out->hll, host.regs, sizeof out->hll);
    for (int j = 0; j < kHllM; ++j)
        if (out->hll[j] > kRhoMax) return fail(EIGER_ERR_INTERNAL, "register %d holds %d", j, out->hll[j]);
    out->estimate = hll_estimate(out->hll);
    return EIGER_OK;
}

bool narrowable(int dtype, int64_t nb, int64_t mn, int64_t mx) {
    if (nb == 0) return false;
    if (dtype == EIGER_I32) return true;
    return (uint64_t)mx - (uint64_t)mn <= 0xFFFFFFFFull;
}

eiger_plan_t static_plan() {
    eiger_plan_t p{};
    p.variant = EIGER_STATIC;
    p.load_factor = 0.5f;
    p.narrow = 0;
    p.selector = 3;
    return p;
}

PlanDev to_dev(const eiger_plan_t& p, int dtype, const eiger_stats_t* bst) {
    PlanDev d{};
    d.variant = p.variant;
    d.bits1 = p.bits1;
    d.bits2 = p.bits2;
    d.narrow = p.narrow;
    d.key32 = dtype == EIGER_I32 || p.narrow;
    d.load_factor = p.load_factor;
    d.dtype = dtype;
    if (bst) {
        d.range.lo = bst->min;
        d.range.hi = bst->max;
        // 32-bit keys are offsets from the build minimum; the sort of the
        // sort-merge join offsets 64-bit keys too, so it orders only the span
        d.range.offset = (d.key32 || p.variant == EIGER_SMJ) ? (uint64_t)bst->min : 0ull;
        d.check_range = 1;
    } else {
        d.range.lo = INT64_MIN;
        d.range.hi = INT64_MAX;
        d.range.offset = 0;
        d.check_range = 0;
    }
    return d;
}

// Checks a plan's knobs; `narrow_ok` says whether the build keys allow it.
eiger_status check_plan(const eiger_plan_t& p, int64_t nb, int dtype, bool narrow_ok) {
    switch (p.variant) {
        case EIGER_NPHJ:
        case EIGER_STATIC: {
            if (!(p.load_factor > 0.0f && p.load_factor <= 0.9f))
                return fail(EIGER_ERR_INVALID_ARG, "load_factor %g outside (0, 0.9]", p.load_factor);
            const bool key32 = dtype == EIGER_I32 || p.narrow;
            if (key32 && table_slots(nb, p.load_factor) > (1ull << 32))
                return fail(EIGER_ERR_INVALID_ARG, "hash table of %lld rows needs more than 2^32 slots",
                            (long long)nb);
            break;
        }
        case EIGER_PHJ1:
            if (p.bits1 < 1 || p.bits1 > kMaxBits)
                return fail(EIGER_ERR_INVALID_ARG, "bits1 %d outside [1, %d]", p.bits1, kMaxBits);
            break;
        case EIGER_PHJ2:
            if (p.bits1 < 1 || p.bits1 > kMaxBits || p.bits2 < 1 || p.bits2 > kMaxBits ||
                p.bits1 + p.bits2 > 20)
                return fail(EIGER_ERR_INVALID_ARG, "bits (%d, %d) outside [1, %d] each, sum <= 20",
                            p.bits1, p.bits2, kMaxBits);
            break;
        case EIGER_SMJ:
            if (p.bits1 < 0 || p.bits1 > kSortMaxBits)
                return fail(EIGER_ERR_INVALID_ARG, "SMJ bits1 %d outside [1, %d] (0 = %d)", p.bits1, kSortMaxBits,
                            kSortMaxBits);
            break;
        default:
            return fail(EIGER_ERR_INVALID_ARG, "plan variant %d is not NPHJ/PHJ1/PHJ2/STATIC/SMJ", p.variant);
    }
    if (p.narrow != 0 && p.narrow != 1) return fail(EIGER_ERR_INVALID_ARG, "narrow must be 0 or 1");
    if (p.narrow && !narrow_ok)
        return fail(EIGER_ERR_INVALID_ARG, "narrow = 1 but the build key range spans >= 2^32");
    return EIGER_OK;
}

struct Layout {
    Ctrl* ctrl;
    StatsScratch stats;
    float* sel_x;  // selector features (one sample)
    float* sel_z;  // selector logits
    size_t fixed_end;
};

Layout fixed_layout(Carve& c) {
    Layout l;
    l.ctrl = c.take<Ctrl>(1);
    l.stats = stats_layout(c);
    l.sel_x = c.take<float>(EIGER_MLP_IN);
    l.sel_z = c.take<float>(EIGER_MLP_OUT);
    l.fixed_end = c.off;
    return l;
}

size_t variant_bytes(Carve c, int64_t nb, int64_t np, const PlanDev& pd, NphjScratch* ns,
                     PhjScratch* ps, SmjScratch* ms = nullptr) {
    if (pd.variant == EIGER_NPHJ || pd.variant == EIGER_STATIC) {
        NphjScratch s = nphj_layout(c, nb, pd);
        if (ns) *ns = s;
    } else if (pd.variant == EIGER_SMJ) {
        SmjScratch s = smj_layout(c, nb, np, pd);
        if (ms) *ms = s;
    } else {
        PhjScratch s = phj_layout(c, nb, np, pd);
        if (ps) *ps = s;
    }
    return c.off;
}

struct JoinCall {
    int dtype;
    const void* bkeys;
    const void* bpay;
    int64_t nb;
    const void* pkeys;
    const void* ppay;
    int64_t np;
    int pay_bytes;
    int variant;
    int materialize;  // eiger_materialize requested (the narrow calls ask for GFUR)
    int wide;         // columns come from eiger_columns (bpay/ppay/pay_bytes unused)
    const eiger_plan_t* knobs;
    JoinOut out;
    int64_t* out_count;
    int64_t* out_sum;
    void* ws;
    size_t ws_bytes;
    eiger_plan_t* plan_used;
    cudaStream_t stream;
};

eiger_status validate_common(const JoinCall& c) {
    if (c.dtype != EIGER_I32 && c.dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype %d", c.dtype);
    if (c.nb < 0 || c.np < 0 || c.nb > kMaxRows || c.np > kMaxRows)
        return fail(EIGER_ERR_INVALID_ARG, "row counts must be in [0, 2^32): nb=%lld np=%lld",
                    (long long)c.nb, (long long)c.np);
    const size_t kb = c.dtype == EIGER_I32 ? 4 : 8;
    if ((c.nb > 0 && !c.bkeys) || (c.np > 0 && !c.pkeys))
        return fail(EIGER_ERR_INVALID_ARG, "NULL key column with rows");
    if ((c.bkeys && !aligned(c.bkeys, kb)) || (c.pkeys && !aligned(c.pkeys, kb)))
        return fail(EIGER_ERR_INVALID_ARG, "key columns must be aligned to their element size");
    const void* bpay_out = !c.wide && c.out.b.n ? c.out.b.dst[0] : nullptr;
    const void* ppay_out = !c.wide && c.out.p.n ? c.out.p.dst[0] : nullptr;
    const bool pay_used = c.bpay || c.ppay || bpay_out || ppay_out || c.out.aggregate;
    if (pay_used && c.pay_bytes != 4 && c.pay_bytes != 8)
        return fail(EIGER_ERR_INVALID_ARG, "payload_bytes must be 4 or 8, got %d", c.pay_bytes);
    if (pay_used) {
        const size_t pb = (size_t)c.pay_bytes;
        if ((c.bpay && !aligned(c.bpay, pb)) || (c.ppay && !aligned(c.ppay, pb)) ||
            (bpay_out && !aligned(bpay_out, pb)) || (ppay_out && !aligned(ppay_out, pb)))
            return fail(EIGER_ERR_INVALID_ARG, "payload arrays must be aligned to payload_bytes");
    }
    if ((bpay_out && !c.bpay) || (ppay_out && !c.ppay))
        return fail(EIGER_ERR_INVALID_ARG, "payload output requested without its payload column");
    if ((c.out.bidx && !aligned(c.out.bidx, 4)) || (c.out.pidx && !aligned(c.out.pidx, 4)))
        return fail(EIGER_ERR_INVALID_ARG, "index outputs must be 4-byte aligned");
    if (c.variant < EIGER_AUTO || c.variant > EIGER_SMJ)
        return fail(EIGER_ERR_INVALID_ARG, "bad variant %d", c.variant);
    if (c.materialize < EIGER_GFUR || c.materialize > EIGER_MAT_AUTO)
        return fail(EIGER_ERR_INVALID_ARG, "bad materialize %d", c.materialize);
    if (!c.out_count) return fail(EIGER_ERR_INVALID_ARG, "out_count is NULL");
    if (!c.ws && c.ws_bytes) return fail(EIGER_ERR_INVALID_ARG, "NULL workspace with nonzero size");
    return EIGER_OK;
}

void sort_passes(eiger_plan_t* p);

// Resolves the plan. `bst` holds the build statistics (NULL for STATIC).
eiger_status resolve_plan(const JoinCall& c, const eiger_stats_t* bst, eiger_plan_t* pub,
                          double probe_distinct = -1.0) {
    if (c.variant == EIGER_STATIC) {
        *pub = static_plan();
        return check_plan(*pub, c.nb, c.dtype, false);
    }
    const bool nok = narrowable(c.dtype, c.nb, bst->min, bst->max);
    if (c.knobs) {
        *pub = *c.knobs;
        if (c.variant != EIGER_AUTO) pub->variant = c.variant;
        if (pub->variant == EIGER_STATIC)
            return fail(EIGER_ERR_INVALID_ARG, "use variant EIGER_STATIC, not a STATIC knob plan");
        pub->selector = 2;
    } else {
        *pub = plan_rules(c.variant, c.nb, c.np, c.dtype, nok, distinct_keys(bst->estimate, c.nb),
                          l2_bytes_or_default(), probe_distinct);
    }
    if (c.dtype == EIGER_I32) pub->narrow = 1;  // int32 keys always travel as 32-bit offsets
    eiger_status s = check_plan(*pub, c.nb, c.dtype, nok);
    if (s != EIGER_OK) return s;
    pub->key_min = bst->min;
    pub->key_max = bst->max;
    if (pub->variant == EIGER_SMJ) sort_passes(pub);
    return EIGER_OK;
}

// SMJ knobs from the build span: the sort orders the span's significant bits
// (the keys are offsets from the build minimum) in the fewest passes of at
// most bits1 bits, with the bits spread evenly over the passes.
void sort_passes(eiger_plan_t* p) {
    const int want = p->bits1 ? p->bits1 : kSortMaxBits;
    PlanDev d{};
    d.range.lo = p->key_min;
    d.range.hi = p->key_max;
    const int sb = sort_key_bits(d);
    const int passes = sb == 0 ? 1 : (sb + want - 1) / want;
    p->bits2 = passes;
    p->bits1 = sb == 0 ? 1 : (sb + passes - 1) / passes;
}

// Whether carrying the payload columns through the passes (GFTR) should move
// fewer DRAM bytes than gathering them by tuple ID (GFUR), the trade-off
// Sec. 5.2.3 measures as a switch-over by match ratio. Carrying reads and
// writes every carried column of both sides once per pass; gathering reads,
// per match and column, at least one 32-byte sector at a random position
// (columns far larger than L2). Matches are estimated as np times the average
// build multiplicity nb / distinct build keys (every probe row assumed to
// match). For |R| = 2^16, |S| = 2^28 and three 4-byte columns per side this
// puts the switch at a quarter of the probe rows matching.
bool carry_pays(const JoinCall& c, const eiger_plan_t& p, const eiger_stats_t* bst) {
    const double passes = p.variant == EIGER_PHJ2 ? 2.0 : p.variant == EIGER_SMJ ? (double)p.bits2 : 1.0;
    double wb = 0, wp = 0;
    for (int q = 0; q < c.out.b.n; ++q) wb += c.out.b.bytes[q];
    for (int q = 0; q < c.out.p.n; ++q) wp += c.out.p.bytes[q];
    const double carried = 2.0 * passes * ((double)c.nb * wb + (double)c.np * wp);
    const double distinct = bst && bst->estimate >= 1.0 ? std::min(bst->estimate, (double)c.nb) : (double)c.nb;
    const double matches = (double)c.np * (double)c.nb / (distinct > 0 ? distinct : 1.0);
    const double gathered = matches * 32.0 * (double)(c.out.b.n + c.out.p.n);
    return carried < gathered;
}

// Materialisation that runs: GFTR needs a transformation (partitioning or
// sorting) and at least one column to carry (the aggregate carries the two
// summed payload columns); AUTO takes it when carry_pays says so.
eiger_status resolve_materialize(const JoinCall& c, const eiger_stats_t* bst, eiger_plan_t* pub) {
    const bool transformed = pub->variant == EIGER_PHJ1 || pub->variant == EIGER_PHJ2 || pub->variant == EIGER_SMJ;
    const bool cols = c.out.b.n + c.out.p.n > 0;
    int m = c.materialize;
    if (m == EIGER_GFTR && !transformed)
        return fail(EIGER_ERR_INVALID_ARG, "GFTR needs a partitioned or sort-merge plan (got variant %d)",
                    pub->variant);
    if (m == EIGER_MAT_AUTO) m = transformed && carry_pays(c, *pub, bst) ? EIGER_GFTR : EIGER_GFUR;
    if (!cols) m = EIGER_GFUR;
    pub->materialize = m;
    return EIGER_OK;
}

void set_carry(PlanDev& d, const JoinOut& out, int materialize) {
    d.gftr = materialize == EIGER_GFTR;
    d.no_rows = d.gftr && out.aggregate;  // the positional sum needs no tuple IDs
    d.ncols[0] = d.gftr ? out.b.n : 0;
    d.ncols[1] = d.gftr ? out.p.n : 0;
    for (int q = 0; q < kMaxCols; ++q) {
        d.col_bytes[0][q] = q < out.b.n ? out.b.bytes[q] : 0;
        d.col_bytes[1][q] = q < out.p.n ? out.p.bytes[q] : 0;
    }
}

constexpr int64_t kProbeSample = 1 << 20;  // probe rows profiled for the selector features

// The learned selector's plan for an AUTO join: profile a probe sample,
// compute and normalise the features, run the network on the device and take
// the best-scoring class. *chosen stays false when the class's plan is not
// valid for these keys (the rules then decide).
eiger_status learned_plan(const JoinCall& c, const eiger_stats_t& bst, const Layout& lay, const float* params,
                          const float* mean, const float* scale, eiger_plan_t* pub, bool* chosen) {
    *chosen = false;
    static thread_local eiger_stats_t pst;
    const int64_t nps = c.np < kProbeSample ? c.np : kProbeSample;
    eiger_status s = run_stats(c.pkeys, nps, c.dtype, lay.stats, c.stream, &pst);
    if (s != EIGER_OK) return s;
    float f[EIGER_MLP_IN];
    compute_features(&bst, &pst, c.nb, c.np, c.dtype, l2_bytes_or_default(), f);
    for (int i = 0; i < EIGER_MLP_IN; ++i) f[i] = (f[i] - mean[i]) / scale[i];
    EIGER_CUDA(cudaMemcpyAsync(lay.sel_x, f, sizeof f, cudaMemcpyHostToDevice, c.stream), "selector features");
    EIGER_CUDA(mlp_forward(params, lay.sel_x, 1, lay.sel_z, c.stream), "selector network");
    float z[EIGER_MLP_OUT];
    EIGER_CUDA(cudaMemcpyAsync(z, lay.sel_z, sizeof z, cudaMemcpyDeviceToHost, c.stream), "selector logits");
    EIGER_CUDA(cudaStreamSynchronize(c.stream), "selector synchronise");
    int best = 0;
    for (int k = 1; k < EIGER_MLP_OUT; ++k)
        if (z[k] > z[best]) best = k;
    eiger_plan_t p = class_plan(best);
    const bool nok = narrowable(c.dtype, c.nb, bst.min, bst.max);
    p.narrow = (c.dtype == EIGER_I32 || nok) ? 1 : 0;
    const std::string saved = g_last_error;
    if (check_plan(p, c.nb, c.dtype, nok) != EIGER_OK) {
        g_last_error = saved;  // an unusable class is not an error: fall back
        return EIGER_OK;
    }
    p.key_min = bst.min;
    p.key_max = bst.max;
    *pub = p;
    *chosen = true;
    return EIGER_OK;
}

eiger_status run_join(const JoinCall& c) {
    eiger_status s = validate_common(c);
    if (s != EIGER_OK) return s;
    prof_reset();
    Carve carve{static_cast<char*>(c.ws), 0};
    Layout lay = fixed_layout(carve);
    if (lay.fixed_end > c.ws_bytes)
        return fail(EIGER_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", c.ws_bytes, lay.fixed_end);

    static thread_local eiger_stats_t bst;
    const bool adaptive = c.variant != EIGER_STATIC;
    if (adaptive) {
        s = run_stats(c.bkeys, c.nb, c.dtype, lay.stats, c.stream, &bst);
        if (s != EIGER_OK) return s;
    }
    eiger_plan_t pub;
    bool chosen = false;
    const float* sel_params;
    float sel_mean[EIGER_MLP_IN], sel_scale[EIGER_MLP_IN];
    if (adaptive && c.variant == EIGER_AUTO && !c.knobs && c.nb > 0 && c.np > 0 &&
        selector_get(&sel_params, sel_mean, sel_scale)) {
        s = learned_plan(c, bst, lay, sel_params, sel_mean, sel_scale, &pub, &chosen);
        if (s != EIGER_OK) return s;
    }
    if (!chosen) {
        s = resolve_plan(c, adaptive ? &bst : nullptr, &pub);
        if (s != EIGER_OK) return s;
        // a partitioned plan for a probe side at least twice the build side
        // looks at a probe sample first: heavy skew favours the NPHJ
        if (c.variant == EIGER_AUTO && !c.knobs &&
            wants_probe_sample(pub, c.nb, c.np, c.dtype, narrowable(c.dtype, c.nb, bst.min, bst.max))) {
            static thread_local eiger_stats_t pst;
            const int64_t ns = c.np < kProbeSampleRows ? c.np : kProbeSampleRows;
            s = run_stats(c.pkeys, ns, c.dtype, lay.stats, c.stream, &pst);
            if (s != EIGER_OK) return s;
            s = resolve_plan(c, &bst, &pub, pst.estimate / (double)ns);
            if (s != EIGER_OK) return s;
        }
    }
    s = resolve_materialize(c, adaptive ? &bst : nullptr, &pub);
    if (s != EIGER_OK) return s;
    if (c.plan_used) *c.plan_used = pub;

    *c.out_count = 0;
    if (c.out_sum) *c.out_sum = 0;
    if (c.nb == 0 || c.np == 0) return EIGER_OK;

    PlanDev pd = to_dev(pub, c.dtype, adaptive ? &bst : nullptr);
    set_carry(pd, c.out, pub.materialize);
    NphjScratch ns{};
    PhjScratch ps{};
    SmjScratch ms{};
    const size_t need = variant_bytes(carve, c.nb, c.np, pd, &ns, &ps, &ms);
    if (need > c.ws_bytes)
        return fail(EIGER_ERR_WORKSPACE, "workspace %zu bytes < %zu needed for this plan", c.ws_bytes, need);
    // Host-side fault injection for tests: EIGER_FAULT=table_full shrinks the
    // non-partitioned table to 64 slots, so inserts and probes exhaust their
    // bounded probe sequences and the device error flag path is exercised.
    const char* fault = std::getenv("EIGER_FAULT");
    if (fault && std::strcmp(fault, "table_full") == 0 &&
        (pd.variant == EIGER_NPHJ || pd.variant == EIGER_STATIC))
        ns.slots = 64;

    EIGER_CUDA(cudaMemsetAsync(lay.ctrl, 0, sizeof(Ctrl), c.stream), "control block reset");
    const JoinArgs a{c.bkeys, c.nb, c.pkeys, c.np};
    if (pd.variant == EIGER_NPHJ || pd.variant == EIGER_STATIC)
        EIGER_CUDA(nphj_run(a, pd, ns, c.out, lay.ctrl, c.stream), "non-partitioned join");
    else if (pd.variant == EIGER_SMJ)
        EIGER_CUDA(smj_run(a, pd, ms, c.out, lay.ctrl, c.stream), "sort-merge join");
    else
        EIGER_CUDA(phj_run(a, pd, ps, c.out, lay.ctrl, c.stream), "partitioned join");

    Ctrl h;
    EIGER_CUDA(readback_sync(&h, lay.ctrl, sizeof(Ctrl), c.stream), "result readback");
    if (h.err & kErrTableFull) return fail(EIGER_ERR_TABLE_FULL, "a hash-table probe sequence hit its cap");
    if (h.err & kErrInternal) return fail(EIGER_ERR_INTERNAL, "device consistency check failed");
    prof_set_matches(h.cursor);
    *c.out_count = (int64_t)h.cursor;
    if (c.out_sum) *c.out_sum = (int64_t)h.sum;
    if (!c.out.aggregate && h.cursor > c.out.capacity)
        return fail(EIGER_ERR_CAPACITY, "%llu matches exceed capacity %llu", h.cursor, c.out.capacity);
    return EIGER_OK;
}

// Columns a join may carry (GFTR) and the requested materialisation.
struct ColSpec {
    int n[2];
    int bytes[2][kMaxCols];
    int materialize;
};

size_t join_workspace_bytes(int64_t nb, int64_t np, int dtype, int variant, const eiger_plan_t* knobs,
                            const ColSpec& cs) {
    Carve c{nullptr, 0};
    fixed_layout(c);
    size_t best = c.off;
    auto consider = [&](const eiger_plan_t& p) {
        PlanDev pd{};
        pd.variant = p.variant;
        pd.bits1 = p.bits1;
        pd.bits2 = p.bits2;
        pd.narrow = p.narrow;
        pd.key32 = dtype == EIGER_I32 || p.narrow;
        pd.load_factor = p.load_factor;
        pd.dtype = dtype;
        if (p.variant == EIGER_SMJ) {  // the most buffers and counts any key span needs
            pd.bits1 = p.bits1 ? p.bits1 : kSortMaxBits;
            pd.bits2 = 2;
        }
        const bool transformed = p.variant == EIGER_PHJ1 || p.variant == EIGER_PHJ2 || p.variant == EIGER_SMJ;
        pd.gftr = transformed && cs.materialize != EIGER_GFUR && cs.n[0] + cs.n[1] > 0;
        for (int side = 0; side < 2; ++side) {
            pd.ncols[side] = pd.gftr ? cs.n[side] : 0;
            for (int q = 0; q < kMaxCols; ++q) pd.col_bytes[side][q] = cs.bytes[side][q];
        }
        const size_t b = variant_bytes(c, nb, np, pd, nullptr, nullptr);
        if (b > best) best = b;
    };
    if (variant == EIGER_STATIC) {
        consider(static_plan());
    } else if (knobs) {
        eiger_plan_t p = *knobs;
        if (variant != EIGER_AUTO) p.variant = variant;
        if (dtype == EIGER_I32) p.narrow = 1;
        consider(p);
    } else {
        const size_t l2 = l2_bytes_or_default();
        for (int nok = 0; nok < 2; ++nok) {
            for (int distinct = 0; distinct < 2; ++distinct) {  // the statistics decide both later
                eiger_plan_t p = plan_rules(variant, nb, np, dtype, nok != 0, distinct != 0, l2);
                p.narrow = (dtype == EIGER_I32 || nok) ? 1 : 0;
                consider(p);
            }
            if (variant == EIGER_AUTO)  // a learned selector may pick any class
                for (int cls = 0; cls < EIGER_MLP_OUT; ++cls) {
                    eiger_plan_t q = class_plan(cls);
                    q.narrow = (dtype == EIGER_I32 || nok) ? 1 : 0;
                    consider(q);
                }
        }
    }
    return best;
}

ColSpec no_columns() {
    ColSpec cs{};
    cs.materialize = EIGER_GFUR;
    return cs;
}

eiger_status check_columns(const eiger_columns* cols, const char* side, bool need_data, int* n) {
    *n = 0;
    if (!cols) return EIGER_OK;
    if (cols->n < 0 || cols->n > EIGER_MAX_COLS)
        return fail(EIGER_ERR_INVALID_ARG, "%s: column count %d outside [0, %d]", side, cols->n, EIGER_MAX_COLS);
    for (int q = 0; q < cols->n; ++q) {
        const int b = cols->bytes[q];
        if (b != 4 && b != 8) return fail(EIGER_ERR_INVALID_ARG, "%s column %d: bytes must be 4 or 8", side, q);
        if (need_data) {
            if (!cols->cols[q] || !cols->out[q])
                return fail(EIGER_ERR_INVALID_ARG, "%s column %d: NULL input or output", side, q);
            if (!aligned(cols->cols[q], b) || !aligned(cols->out[q], b))
                return fail(EIGER_ERR_INVALID_ARG, "%s column %d: arrays must be aligned to %d bytes", side, q, b);
        }
    }
    *n = cols->n;
    return EIGER_OK;
}

}  // namespace

namespace eiger {
// Records `msg` as the calling thread's last error and returns `s`.
eiger_status report_error(eiger_status s, const char* msg) { return fail(s, "%s", msg); }
}  // namespace eiger

extern "C" {

const char* eiger_last_error(void) { return g_last_error.c_str(); }

const char* eiger_version(void) { return "eiger-gb300 0.1 (sm_103a)"; }

eiger_status eiger_stats_workspace(int64_t n, eiger_dtype dtype, size_t* bytes) {
    if (!bytes) return fail(EIGER_ERR_INVALID_ARG, "bytes is NULL");
    if (n < 0) return fail(EIGER_ERR_INVALID_ARG, "n < 0");
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype");
    Carve c{nullptr, 0};
    stats_layout(c);
    *bytes = c.off;
    return EIGER_OK;
}

eiger_status eiger_stats(const void* d_keys, int64_t n, eiger_dtype dtype, eiger_stats_t* out,
                         void* d_workspace, size_t ws_bytes, void* stream) {
    if (!out) return fail(EIGER_ERR_INVALID_ARG, "out is NULL");
    if (n < 0) return fail(EIGER_ERR_INVALID_ARG, "n < 0");
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype");
    if (n > 0 && !d_keys) return fail(EIGER_ERR_INVALID_ARG, "NULL keys with n > 0");
    if (d_keys && !aligned(d_keys, dtype == EIGER_I32 ? 4 : 8))
        return fail(EIGER_ERR_INVALID_ARG, "keys must be aligned to their element size");
    prof_reset();
    Carve c{static_cast<char*>(d_workspace), 0};
    StatsScratch ss = stats_layout(c);
    if (n > 0 && (c.off > ws_bytes || !d_workspace))
        return fail(EIGER_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, c.off);
    return run_stats(d_keys, n, dtype, ss, static_cast<cudaStream_t>(stream), out);
}

eiger_status eiger_plan(const eiger_stats_t* build, const eiger_stats_t* probe, int64_t nb, int64_t np,
                        eiger_dtype dtype, eiger_plan_t* out) {
    if (!out || !build) return fail(EIGER_ERR_INVALID_ARG, "NULL build statistics or output");
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype");
    if (nb < 0 || np < 0 || nb > kMaxRows || np > kMaxRows)
        return fail(EIGER_ERR_INVALID_ARG, "row counts must be in [0, 2^32)");
    const bool nok = narrowable(dtype, nb, build->min, build->max);
    const double pd = probe && probe->n > 0 ? probe->estimate / (double)probe->n : -1.0;
    *out = plan_rules(EIGER_AUTO, nb, np, dtype, nok, distinct_keys(build->estimate, nb), l2_bytes_or_default(),
                      pd);
    if (dtype == EIGER_I32) out->narrow = 1;
    out->key_min = build->min;
    out->key_max = build->max;
    return EIGER_OK;
}

eiger_status eiger_join_workspace(int64_t nb, int64_t np, eiger_dtype dtype, eiger_variant variant,
                                  const eiger_plan_t* knobs, size_t* bytes) {
    if (!bytes) return fail(EIGER_ERR_INVALID_ARG, "bytes is NULL");
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype");
    if (nb < 0 || np < 0 || nb > kMaxRows || np > kMaxRows)
        return fail(EIGER_ERR_INVALID_ARG, "row counts must be in [0, 2^32)");
    if (variant < EIGER_AUTO || variant > EIGER_SMJ) return fail(EIGER_ERR_INVALID_ARG, "bad variant");
    *bytes = join_workspace_bytes(nb, np, dtype, variant, knobs, no_columns());
    return EIGER_OK;
}

eiger_status eiger_join(eiger_dtype dtype, const void* d_bkeys, const void* d_bpay, int64_t nb,
                        const void* d_pkeys, const void* d_ppay, int64_t np, int32_t payload_bytes,
                        eiger_variant variant, const eiger_plan_t* knobs, uint32_t* d_out_bidx,
                        uint32_t* d_out_pidx, void* d_out_bpay, void* d_out_ppay, int64_t capacity,
                        int64_t* out_count, void* d_workspace, size_t ws_bytes, eiger_plan_t* plan_used,
                        void* stream) {
    if (capacity < 0) return fail(EIGER_ERR_INVALID_ARG, "capacity < 0");
    if (capacity > 0 && !d_out_bidx && !d_out_pidx && !d_out_bpay && !d_out_ppay)
        return fail(EIGER_ERR_INVALID_ARG, "capacity > 0 but no output array");
    JoinCall c{};
    c.dtype = dtype;
    c.bkeys = d_bkeys;
    c.bpay = d_bpay;
    c.nb = nb;
    c.pkeys = d_pkeys;
    c.ppay = d_ppay;
    c.np = np;
    c.pay_bytes = payload_bytes;
    c.variant = variant;
    c.knobs = knobs;
    c.out.bidx = d_out_bidx;
    c.out.pidx = d_out_pidx;
    c.out.b.src[0] = d_bpay;
    c.out.b.dst[0] = d_out_bpay;
    c.out.b.bytes[0] = payload_bytes;
    c.out.b.n = d_out_bpay ? 1 : 0;
    c.out.p.src[0] = d_ppay;
    c.out.p.dst[0] = d_out_ppay;
    c.out.p.bytes[0] = payload_bytes;
    c.out.p.n = d_out_ppay ? 1 : 0;
    c.out.aggregate = 0;
    c.out.capacity = (unsigned long long)capacity;
    c.out_count = out_count;
    c.out_sum = nullptr;
    c.ws = d_workspace;
    c.ws_bytes = ws_bytes;
    c.plan_used = plan_used;
    c.stream = static_cast<cudaStream_t>(stream);
    return run_join(c);
}

eiger_status eiger_join_wide_workspace(int64_t nb, int64_t np, eiger_dtype dtype, const eiger_columns* build,
                                       const eiger_columns* probe, eiger_variant variant,
                                       eiger_materialize materialize, const eiger_plan_t* knobs,
                                       size_t* bytes) {
    if (!bytes) return fail(EIGER_ERR_INVALID_ARG, "bytes is NULL");
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype");
    if (nb < 0 || np < 0 || nb > kMaxRows || np > kMaxRows)
        return fail(EIGER_ERR_INVALID_ARG, "row counts must be in [0, 2^32)");
    if (variant < EIGER_AUTO || variant > EIGER_SMJ) return fail(EIGER_ERR_INVALID_ARG, "bad variant");
    if (materialize < EIGER_GFUR || materialize > EIGER_MAT_AUTO)
        return fail(EIGER_ERR_INVALID_ARG, "bad materialize");
    ColSpec cs{};
    cs.materialize = materialize;
    eiger_status s = check_columns(build, "build", false, &cs.n[0]);
    if (s == EIGER_OK) s = check_columns(probe, "probe", false, &cs.n[1]);
    if (s != EIGER_OK) return s;
    for (int q = 0; q < cs.n[0]; ++q) cs.bytes[0][q] = build->bytes[q];
    for (int q = 0; q < cs.n[1]; ++q) cs.bytes[1][q] = probe->bytes[q];
    *bytes = join_workspace_bytes(nb, np, dtype, variant, knobs, cs);
    return EIGER_OK;
}

eiger_status eiger_join_wide(eiger_dtype dtype, const void* d_bkeys, int64_t nb, const eiger_columns* build,
                             const void* d_pkeys, int64_t np, const eiger_columns* probe,
                             eiger_variant variant, eiger_materialize materialize, const eiger_plan_t* knobs,
                             uint32_t* d_out_bidx, uint32_t* d_out_pidx, int64_t capacity, int64_t* out_count,
                             void* d_workspace, size_t ws_bytes, eiger_plan_t* plan_used, void* stream) {
    if (capacity < 0) return fail(EIGER_ERR_INVALID_ARG, "capacity < 0");
    int nbc = 0, npc = 0;
    eiger_status s = check_columns(build, "build", true, &nbc);
    if (s == EIGER_OK) s = check_columns(probe, "probe", true, &npc);
    if (s != EIGER_OK) return s;
    if (capacity > 0 && !d_out_bidx && !d_out_pidx && nbc + npc == 0)
        return fail(EIGER_ERR_INVALID_ARG, "capacity > 0 but no output array");
    JoinCall c{};
    c.dtype = dtype;
    c.bkeys = d_bkeys;
    c.nb = nb;
    c.pkeys = d_pkeys;
    c.np = np;
    c.variant = variant;
    c.materialize = materialize;
    c.wide = 1;
    c.knobs = knobs;
    c.out.bidx = d_out_bidx;
    c.out.pidx = d_out_pidx;
    for (int q = 0; q < nbc; ++q) {
        c.out.b.src[q] = build->cols[q];
        c.out.b.dst[q] = build->out[q];
        c.out.b.bytes[q] = build->bytes[q];
    }
    c.out.b.n = nbc;
    for (int q = 0; q < npc; ++q) {
        c.out.p.src[q] = probe->cols[q];
        c.out.p.dst[q] = probe->out[q];
        c.out.p.bytes[q] = probe->bytes[q];
    }
    c.out.p.n = npc;
    c.out.aggregate = 0;
    c.out.capacity = (unsigned long long)capacity;
    c.out_count = out_count;
    c.ws = d_workspace;
    c.ws_bytes = ws_bytes;
    c.plan_used = plan_used;
    c.stream = static_cast<cudaStream_t>(stream);
    return run_join(c);
}

}  // extern "C"

namespace {

constexpr int kGbTargetGroups = 1024;          // groups per partition the PARTITION plan aims at
constexpr int kGbMaxBits = 20;                  // most partition bits a retry grows to
constexpr size_t kGbSmemBudget = 96 * 1024;     // CTA-private hash table limit

unsigned long long pow2_at_least(double x) {
    unsigned long long s = 64;
    while ((double)s < x) s <<= 1;
    return s;
}

// The most slots a HASH plan (or its retries) may take: a load of 1/2 with
// every row its own group.
unsigned long long gb_max_slots(int64_t n) { return pow2_at_least(2.0 * (double)(n > 0 ? n : 1)); }

void gb_split_bits(int B, int32_t* b1, int32_t* b2) {
    if (B <= 10) {
        *b1 = B;
        *b2 = 0;
    } else {
        *b1 = (B + 1) / 2;
        *b2 = B / 2;
    }
}

eiger_status check_aggs(const eiger_aggs* aggs, bool need_data) {
    if (!aggs) return fail(EIGER_ERR_INVALID_ARG, "aggs is NULL");
    if (aggs->n < 0 || aggs->n > EIGER_MAX_AGGS)
        return fail(EIGER_ERR_INVALID_ARG, "aggregate count %d outside [0, %d]", aggs->n, EIGER_MAX_AGGS);
    for (int a = 0; a < aggs->n; ++a) {
        const int op = aggs->op[a];
        if (op < EIGER_AGG_SUM || op > EIGER_AGG_MAX)
            return fail(EIGER_ERR_INVALID_ARG, "aggregate %d: bad op %d", a, op);
        if (op != EIGER_AGG_COUNT && aggs->bytes[a] != 4 && aggs->bytes[a] != 8)
            return fail(EIGER_ERR_INVALID_ARG, "aggregate %d: value bytes must be 4 or 8", a);
        if (need_data) {
            if (op != EIGER_AGG_COUNT && (!aggs->vals[a] || !aligned(aggs->vals[a], (size_t)aggs->bytes[a])))
                return fail(EIGER_ERR_INVALID_ARG, "aggregate %d: NULL or misaligned value column", a);
        }
    }
    return EIGER_OK;
}

// Value-column widths a PARTITION plan carries (COUNT carries none).
int gb_carried(const eiger_aggs* aggs, int* bytes) {
    int nc = 0;
    for (int a = 0; a < aggs->n; ++a)
        if (aggs->op[a] != EIGER_AGG_COUNT) bytes[nc++] = aggs->bytes[a];
    return nc;
}

size_t gb_workspace_bytes(int64_t n, int dtype, const eiger_aggs* aggs, int variant) {
    Carve c{nullptr, 0};
    fixed_layout(c);
    size_t best = c.off;
    int cb[kMaxCols];
    const int nc = gb_carried(aggs, cb);
    for (int key32 = 0; key32 < 2; ++key32) {
        if (dtype == EIGER_I32 && !key32) continue;
        GbPlanDev pd{};
        pd.key32 = key32;
        pd.naggs = aggs->n;
        if (variant != EIGER_GB_PARTITION) {
            pd.variant = EIGER_GB_HASH;
            pd.slots = gb_max_slots(n);
            Carve d = c;
            gb_layout(d, n, pd, cb, nc);
            if (d.off > best) best = d.off;
        }
        if (variant != EIGER_GB_HASH) {
            pd.variant = EIGER_GB_PARTITION;
            for (int B = 1; B <= kGbMaxBits; ++B) {
                gb_split_bits(B, &pd.bits1, &pd.bits2);
                Carve d = c;
                gb_layout(d, n, pd, cb, nc);
                if (d.off > best) best = d.off;
            }
        }
    }
    return best;
}

}  // namespace

extern "C" {

eiger_status eiger_groupby_workspace(int64_t n, eiger_dtype dtype, const eiger_aggs* aggs, int32_t variant,
                                     size_t* bytes) {
    if (!bytes) return fail(EIGER_ERR_INVALID_ARG, "bytes is NULL");
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype");
    if (n < 0 || n > kMaxRows) return fail(EIGER_ERR_INVALID_ARG, "n must be in [0, 2^32)");
    if (variant < EIGER_GB_AUTO || variant > EIGER_GB_PARTITION) return fail(EIGER_ERR_INVALID_ARG, "bad variant");
    eiger_status s = check_aggs(aggs, false);
    if (s != EIGER_OK) return s;
    *bytes = gb_workspace_bytes(n, dtype, aggs, variant);
    return EIGER_OK;
}

eiger_status eiger_groupby(eiger_dtype dtype, const void* d_keys, int64_t n, const eiger_aggs* aggs,
                           int32_t variant, const eiger_groupby_plan_t* knobs, void* d_out_keys, int64_t capacity,
                           int64_t* out_groups, void* d_workspace, size_t ws_bytes, eiger_groupby_plan_t* plan_used,
                           void* stream) {
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype %d", dtype);
    if (n < 0 || n > kMaxRows) return fail(EIGER_ERR_INVALID_ARG, "n must be in [0, 2^32)");
    if (n > 0 && !d_keys) return fail(EIGER_ERR_INVALID_ARG, "NULL keys with n > 0");
    const size_t kb = dtype == EIGER_I32 ? 4 : 8;
    if (d_keys && !aligned(d_keys, kb)) return fail(EIGER_ERR_INVALID_ARG, "keys must be aligned to their size");
    if (variant < EIGER_GB_AUTO || variant > EIGER_GB_PARTITION)
        return fail(EIGER_ERR_INVALID_ARG, "bad group-by variant %d", variant);
    if (!out_groups) return fail(EIGER_ERR_INVALID_ARG, "out_groups is NULL");
    if (capacity < 0) return fail(EIGER_ERR_INVALID_ARG, "capacity < 0");
    eiger_status s = check_aggs(aggs, n > 0);
    if (s != EIGER_OK) return s;
    if (capacity > 0) {
        if (!d_out_keys || !aligned(d_out_keys, kb))
            return fail(EIGER_ERR_INVALID_ARG, "capacity > 0 needs an aligned key output");
        for (int a = 0; a < aggs->n; ++a)
            if (!aggs->out[a] || !aligned(aggs->out[a], 8))
                return fail(EIGER_ERR_INVALID_ARG, "aggregate %d: NULL or misaligned output", a);
    }
    if (!d_workspace && ws_bytes) return fail(EIGER_ERR_INVALID_ARG, "NULL workspace with nonzero size");
    if (knobs && variant == EIGER_GB_AUTO) return fail(EIGER_ERR_INVALID_ARG, "knobs need a HASH or PARTITION variant");
    prof_reset();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Carve carve{static_cast<char*>(d_workspace), 0};
    Layout lay = fixed_layout(carve);
    if (lay.fixed_end > ws_bytes)
        return fail(EIGER_ERR_WORKSPACE, "workspace %zu bytes < %zu needed", ws_bytes, lay.fixed_end);
    static thread_local eiger_stats_t kst;
    s = run_stats(d_keys, n, dtype, lay.stats, st, &kst);
    if (s != EIGER_OK) return s;

    eiger_groupby_plan_t pub{};
    pub.estimate = kst.estimate;
    pub.narrow = narrowable(dtype, n, kst.min, kst.max) ? 1 : 0;
    const double est = kst.estimate > 1.0 ? kst.estimate : 1.0;
    const int keyb = pub.narrow ? 4 : 8;
    const unsigned long long hash_slots = pow2_at_least(2.5 * est);
    int v = variant;
    if (v == EIGER_GB_AUTO) {
        const double table = (double)hash_slots * (keyb + 8.0 * aggs->n);
        v = table <= (double)l2_bytes_or_default() / 2 ? EIGER_GB_HASH : EIGER_GB_PARTITION;
    }
    pub.variant = v;
    pub.selector = knobs ? 2 : 0;
    const unsigned long long max_slots = gb_max_slots(n);
    if (v == EIGER_GB_HASH) {
        unsigned long long sl = knobs && knobs->table_slots > 0 ? (unsigned long long)knobs->table_slots : hash_slots;
        if (sl & (sl - 1)) return fail(EIGER_ERR_INVALID_ARG, "table_slots must be a power of two");
        pub.table_slots = (int64_t)(sl < max_slots ? sl : max_slots);
    } else {
        int B = 1;
        while (B < kGbMaxBits && est / (double)(1ll << B) > kGbTargetGroups) ++B;
        if (knobs) {
            if (knobs->bits1 < 1 || knobs->bits1 > kMaxBits || knobs->bits2 < 0 || knobs->bits2 > kMaxBits ||
                knobs->bits1 + knobs->bits2 > kGbMaxBits)
                return fail(EIGER_ERR_INVALID_ARG, "partition bits (%d, %d) outside [1, %d] + [0, %d], sum <= %d",
                            knobs->bits1, knobs->bits2, kMaxBits, kMaxBits, kGbMaxBits);
            pub.bits1 = knobs->bits1;
            pub.bits2 = knobs->bits2;
        } else {
            gb_split_bits(B, &pub.bits1, &pub.bits2);
        }
    }
    GbAggs ga{};
    ga.n = aggs->n;
    for (int a = 0; a < aggs->n; ++a) {
        ga.op[a] = aggs->op[a];
        ga.vals[a] = aggs->vals[a];
        ga.bytes[a] = aggs->bytes[a];
        ga.out[a] = reinterpret_cast<long long*>(aggs->out[a]);
    }
    int cb[kMaxCols];
    const int nc = gb_carried(aggs, cb);
    *out_groups = 0;
    Ctrl h{};
    for (int attempt = 1;; ++attempt) {
        pub.attempts = attempt;
        GbPlanDev pd{};
        pd.variant = pub.variant;
        pd.bits1 = pub.bits1;
        pd.bits2 = pub.bits2;
        pd.key32 = pub.narrow;
        pd.offset = (uint64_t)kst.min;
        pd.slots = (unsigned long long)pub.table_slots;
        pd.naggs = aggs->n;
        pd.smem = pd.variant == EIGER_GB_HASH && gb_smem_table_bytes(pd.slots, aggs->n, pd.key32) <= kGbSmemBudget;
        Carve c = carve;
        const GbScratch sc = gb_layout(c, n, pd, cb, nc);
        if (c.off > ws_bytes)
            return fail(EIGER_ERR_WORKSPACE, "workspace %zu bytes < %zu needed for this plan", ws_bytes, c.off);
        if (n == 0) break;
        EIGER_CUDA(cudaMemsetAsync(lay.ctrl, 0, sizeof(Ctrl), st), "control block reset");
        EIGER_CUDA(gb_run(GbArgs{d_keys, n, dtype}, pd, sc, ga, d_out_keys, (unsigned long long)capacity, lay.ctrl, st),
                   "group-by");
        EIGER_CUDA(readback_sync(&h, lay.ctrl, sizeof(Ctrl), st), "result readback");
        if (h.err & kErrInternal) return fail(EIGER_ERR_INTERNAL, "device consistency check failed");
        if (!(h.err & kErrTableFull)) break;
        // a table overflowed: enlarge the plan and run again
        if (pub.variant == EIGER_GB_HASH && (unsigned long long)pub.table_slots < max_slots) {
            const unsigned long long sl = (unsigned long long)pub.table_slots * 4;
            pub.table_slots = (int64_t)(sl < max_slots ? sl : max_slots);
        } else if (pub.variant == EIGER_GB_PARTITION && pub.bits1 + pub.bits2 < kGbMaxBits) {
            int B = pub.bits1 + pub.bits2 + 2;
            gb_split_bits(B < kGbMaxBits ? B : kGbMaxBits, &pub.bits1, &pub.bits2);
        } else {
            if (plan_used) *plan_used = pub;
            return fail(EIGER_ERR_TABLE_FULL, "group-by tables overflowed at the largest plan");
        }
    }
    if (plan_used) *plan_used = pub;
    prof_set_matches(h.cursor);
    *out_groups = (int64_t)h.cursor;
    if (h.cursor > (unsigned long long)capacity)
        return fail(EIGER_ERR_CAPACITY, "%llu groups exceed capacity %lld", h.cursor, (long long)capacity);
    return EIGER_OK;
}

namespace {

eiger_batch_knobs batch_defaults() {
    eiger_batch_knobs k;
    k.block_threads = 256;
    k.chunk_rows = 16384;
    k.load_factor = 0.5f;
    k.small_rows = 1024;
    return k;
}

eiger_status check_batch_knobs(const eiger_batch_knobs& k, eiger_dtype dtype) {
    if (k.block_threads != 128 && k.block_threads != 256 && k.block_threads != 512)
        return fail(EIGER_ERR_INVALID_ARG, "block_threads must be 128, 256 or 512");
    if (k.chunk_rows < 1024 || k.chunk_rows > (1 << 20))
        return fail(EIGER_ERR_INVALID_ARG, "chunk_rows must be in [1024, 2^20]");
    if (!(k.load_factor > 0.0f && k.load_factor <= 0.9f))
        return fail(EIGER_ERR_INVALID_ARG, "load_factor outside (0, 0.9]");
    const int small_max = dtype == EIGER_I32 ? EIGER_BATCH_SMALL_MAX_I32 : EIGER_BATCH_SMALL_MAX_I64;
    if (k.small_rows < 0 || k.small_rows > small_max)
        return fail(EIGER_ERR_INVALID_ARG, "small_rows outside [0, %d] for this dtype", small_max);
    return EIGER_OK;
}

}  // namespace

extern "C" eiger_status eiger_join_batched_workspace(const eiger_join_desc* h_descs, int32_t k,
                                                     eiger_dtype dtype, const eiger_batch_knobs* knobs,
                                                     size_t* bytes) {
    if (!bytes) return fail(EIGER_ERR_INVALID_ARG, "bytes is NULL");
    if (k < 0 || (k > 0 && !h_descs)) return fail(EIGER_ERR_INVALID_ARG, "bad descriptor list");
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype");
    const eiger_batch_knobs kn = knobs ? *knobs : batch_defaults();
    eiger_status s = check_batch_knobs(kn, dtype);
    if (s != EIGER_OK) return s;
    unsigned long long slots = 0;
    for (int j = 0; j < k; ++j) {
        const int64_t nb = h_descs[j].nb, np = h_descs[j].np;
        if (nb < 0 || np < 0 || nb > kMaxRows || np > kMaxRows)
            return fail(EIGER_ERR_INVALID_ARG, "join %d: row counts must be in [0, 2^32)", j);
        // small joins build their tables in shared memory
        if (nb > 0 && np > 0 && nb > kn.small_rows) slots += table_slots(nb, (double)kn.load_factor);
    }
    Carve c{nullptr, 0};
    batch_layout(c, k, slots, dtype == EIGER_I32 ? 8 : 16);
    *bytes = c.off;
    return EIGER_OK;
}

extern "C" eiger_status eiger_join_batched(eiger_dtype dtype, const eiger_join_desc* d_descs, int32_t k,
                                           int64_t* d_counts, int32_t* d_status,
                                           const eiger_batch_knobs* knobs, void* d_workspace,
                                           size_t ws_bytes, void* stream) {
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype");
    if (k < 0) return fail(EIGER_ERR_INVALID_ARG, "k < 0");
    if (!d_status) return fail(EIGER_ERR_INVALID_ARG, "d_status is NULL");
    if (k > 0 && (!d_descs || !d_counts || !d_workspace))
        return fail(EIGER_ERR_INVALID_ARG, "NULL descriptors, counts or workspace");
    const eiger_batch_knobs kn = knobs ? *knobs : batch_defaults();
    eiger_status s = check_batch_knobs(kn, dtype);
    if (s != EIGER_OK) return s;
    const int slot_bytes = dtype == EIGER_I32 ? 8 : 16;
    Carve probe{nullptr, 0};
    batch_layout(probe, k, 0, slot_bytes);
    if (probe.off > ws_bytes) return fail(EIGER_ERR_WORKSPACE, "workspace smaller than the batch bookkeeping");
    // whatever follows the bookkeeping holds the tables
    const unsigned long long cap_slots = (ws_bytes - probe.off) / (size_t)slot_bytes;
    Carve c{static_cast<char*>(d_workspace), 0};
    const BatchLayout L = batch_layout(c, k, cap_slots, slot_bytes);
    if (k == 0) return EIGER_OK;
    EIGER_CUDA(batch_run(d_descs, k, dtype, kn, L, reinterpret_cast<long long*>(d_counts), d_status,
                         static_cast<cudaStream_t>(stream)),
               "batched join");
    return EIGER_OK;
}

eiger_status eiger_join_sum_workspace(int64_t nb, int64_t np, eiger_dtype dtype, int32_t payload_bytes,
                                      eiger_variant variant, eiger_materialize materialize,
                                      const eiger_plan_t* knobs, size_t* bytes) {
    if (!bytes) return fail(EIGER_ERR_INVALID_ARG, "bytes is NULL");
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return fail(EIGER_ERR_INVALID_ARG, "bad dtype");
    if (nb < 0 || np < 0 || nb > kMaxRows || np > kMaxRows)
        return fail(EIGER_ERR_INVALID_ARG, "row counts must be in [0, 2^32)");
    if (variant < EIGER_AUTO || variant > EIGER_SMJ) return fail(EIGER_ERR_INVALID_ARG, "bad variant");
    if (materialize < EIGER_GFUR || materialize > EIGER_MAT_AUTO)
        return fail(EIGER_ERR_INVALID_ARG, "bad materialize");
    if (payload_bytes != 4 && payload_bytes != 8)
        return fail(EIGER_ERR_INVALID_ARG, "payload_bytes must be 4 or 8, got %d", payload_bytes);
    ColSpec cs{};
    cs.materialize = materialize;
    cs.n[0] = cs.n[1] = 1;
    cs.bytes[0][0] = cs.bytes[1][0] = payload_bytes;
    *bytes = join_workspace_bytes(nb, np, dtype, variant, knobs, cs);
    return EIGER_OK;
}

eiger_status eiger_join_sum(eiger_dtype dtype, const void* d_bkeys, const void* d_bpay, int64_t nb,
                            const void* d_pkeys, const void* d_ppay, int64_t np, int32_t payload_bytes,
                            eiger_variant variant, eiger_materialize materialize, const eiger_plan_t* knobs,
                            int64_t* out_sum, int64_t* out_count, void* d_workspace, size_t ws_bytes,
                            eiger_plan_t* plan_used, void* stream) {
    if (!out_sum) return fail(EIGER_ERR_INVALID_ARG, "out_sum is NULL");
    if ((nb > 0 && !d_bpay) || (np > 0 && !d_ppay))
        return fail(EIGER_ERR_INVALID_ARG, "eiger_join_sum needs both payload columns");
    JoinCall c{};
    c.dtype = dtype;
    c.bkeys = d_bkeys;
    c.bpay = d_bpay;
    c.nb = nb;
    c.pkeys = d_pkeys;
    c.ppay = d_ppay;
    c.np = np;
    c.pay_bytes = payload_bytes;
    c.variant = variant;
    c.knobs = knobs;
    c.materialize = materialize;
    // one summed column per side: read by tuple ID (GFUR) or carried (GFTR)
    c.out.b.src[0] = d_bpay;
    c.out.b.bytes[0] = payload_bytes;
    c.out.b.n = 1;
    c.out.p.src[0] = d_ppay;
    c.out.p.bytes[0] = payload_bytes;
    c.out.p.n = 1;
    c.out.aggregate = 1;
    c.out.capacity = 0;
    c.out_count = out_count;
    c.out_sum = out_sum;
    c.ws = d_workspace;
    c.ws_bytes = ws_bytes;
    c.plan_used = plan_used;
    c.stream = static_cast<cudaStream_t>(stream);
    return run_join(c);
}

}  // extern "C"
