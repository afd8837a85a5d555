// eiger_join_static_noalloc: the static non-partitioned hash join for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) at the point where
// they need a join: code that runs while another component owns all device
// memory through its own pool, plug-in hosts that forbid allocation on their
// execution path, or code that must not change the device-memory footprint
// between two measurements. They can still pass input and output arrays they
// already own. For them this entry point keeps its only scratch, the hash
// table and a small control block, in one file-scope device array of fixed
// size. Every GPU that loads the library holds this array until the process
// exits.
//
// Limits and sharing:
//  - The table takes at most kTableBytes (8 MiB): build sides up to 2^19 rows
//    for int32 keys (8-byte slots) or 2^18 rows for int64 keys (16-byte
//    slots) at load factor 0.5. Larger build sides are rejected with
//    EIGER_ERR_INVALID_ARG before any GPU work.
//  - All calls on a device share the one array. Each call clears the table and
//    the control block on its stream before use, so a call never sees the
//    previous call's contents; but two calls whose work overlaps on the GPU
//    (different streams, or different host threads) race on the array.
//  - The host needs the array's device address, which is not the address of
//    the symbol in host code. The first call on each device looks it up with
//    cudaGetSymbolAddress (that device current) and caches it per device
//    ordinal; make that first call before any stream capture begins. The
//    cached address belongs to the device's primary context (the one the CUDA
//    runtime uses): call this entry point under that context, not under a
//    context pushed through the driver API.
#include <mutex>

#include "eiger.h"
#include "kernels.cuh"

namespace eiger {
eiger_status report_error(eiger_status s, const char* msg);
}  // namespace eiger

using namespace eiger;

namespace {

constexpr size_t kCtrlBytes = 256;
constexpr size_t kTableBytes = (size_t)8 << 20;

__device__ __align__(256) unsigned char g_noalloc_scratch[kCtrlBytes + kTableBytes];

// The control block sits in the first kCtrlBytes; the table starts right
// after it, on a 256-byte boundary.
static_assert(sizeof(Ctrl) <= kCtrlBytes, "control block overflows its slot of the scratch array");
static_assert(kCtrlBytes % 256 == 0, "table offset must keep 256-byte alignment");

std::mutex g_addr_mu;
void* g_addr[64];

eiger_status scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return report_error(EIGER_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= 64) return report_error(EIGER_ERR_INTERNAL, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return report_error(EIGER_ERR_CUDA, "cudaGetSymbolAddress of the join scratch failed");
        }
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return EIGER_OK;
}

eiger_status cuda_error(cudaError_t e) {
    cudaGetLastError();
    return report_error(EIGER_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace

extern "C" eiger_status eiger_join_static_noalloc(eiger_dtype dtype, const void* d_bkeys, int64_t nb,
                                                  const void* d_pkeys, int64_t np,
                                                  uint32_t* d_out_bidx, uint32_t* d_out_pidx,
                                                  int64_t capacity, int64_t* out_count,
                                                  void* stream) {
    if (dtype != EIGER_I32 && dtype != EIGER_I64) return report_error(EIGER_ERR_INVALID_ARG, "bad dtype");
    if (!out_count) return report_error(EIGER_ERR_INVALID_ARG, "out_count is NULL");
    if (nb < 0 || np < 0 || nb > 0xFFFFFFFFll || np > 0xFFFFFFFFll)
        return report_error(EIGER_ERR_INVALID_ARG, "row counts must be in [0, 2^32)");
    if ((nb > 0 && !d_bkeys) || (np > 0 && !d_pkeys))
        return report_error(EIGER_ERR_INVALID_ARG, "NULL key column with rows");
    const size_t kb = dtype == EIGER_I32 ? 4 : 8;
    if ((d_bkeys && reinterpret_cast<uintptr_t>(d_bkeys) % kb) ||
        (d_pkeys && reinterpret_cast<uintptr_t>(d_pkeys) % kb))
        return report_error(EIGER_ERR_INVALID_ARG, "key columns must be aligned to their element size");
    if (capacity < 0) return report_error(EIGER_ERR_INVALID_ARG, "capacity < 0");
    if (capacity > 0 && !d_out_bidx && !d_out_pidx)
        return report_error(EIGER_ERR_INVALID_ARG, "capacity > 0 but no output array");
    if ((d_out_bidx && reinterpret_cast<uintptr_t>(d_out_bidx) % 4) ||
        (d_out_pidx && reinterpret_cast<uintptr_t>(d_out_pidx) % 4))
        return report_error(EIGER_ERR_INVALID_ARG, "index outputs must be 4-byte aligned");

    const int slot_bytes = dtype == EIGER_I32 ? 8 : 16;
    const unsigned long long slots = nphj_slots(nb, 0.5f);
    if (slots * (unsigned long long)slot_bytes > kTableBytes)
        return report_error(EIGER_ERR_INVALID_ARG,
                            dtype == EIGER_I32
                                ? "build side exceeds the no-allocation limit of 2^19 int32 rows"
                                : "build side exceeds the no-allocation limit of 2^18 int64 rows");
    *out_count = 0;
    if (nb == 0 || np == 0) return EIGER_OK;

    void* base = nullptr;
    eiger_status s = scratch_address(&base);
    if (s != EIGER_OK) return s;
    Ctrl* ctrl = static_cast<Ctrl*>(base);
    NphjScratch ns;
    ns.table = static_cast<unsigned char*>(base) + kCtrlBytes;
    ns.slots = slots;
    ns.slot_bytes = slot_bytes;

    PlanDev pd{};
    pd.variant = EIGER_STATIC;
    pd.key32 = dtype == EIGER_I32;
    pd.load_factor = 0.5f;
    pd.dtype = dtype;
    pd.range.lo = INT64_MIN;
    pd.range.hi = INT64_MAX;
    pd.range.offset = 0;
    pd.check_range = 0;

    JoinOut out{};
    out.bidx = d_out_bidx;
    out.pidx = d_out_pidx;
    out.capacity = (unsigned long long)capacity;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool prof = prof_set_enabled(false);  // no profiling events from this path
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
    if (e == cudaSuccess) e = nphj_run(JoinArgs{d_bkeys, nb, d_pkeys, np}, pd, ns, out, ctrl, st);
    prof_set_enabled(prof);
    if (e != cudaSuccess) return cuda_error(e);
    Ctrl h;
    if ((e = cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
        return cuda_error(e);
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_error(e);
    if (h.err & kErrTableFull) return report_error(EIGER_ERR_TABLE_FULL, "probe sequence hit its cap");
    if (h.err) return report_error(EIGER_ERR_INTERNAL, "device consistency check failed");
    *out_count = (int64_t)h.cursor;
    if (h.cursor > (unsigned long long)capacity)
        return report_error(EIGER_ERR_CAPACITY, "more matches than capacity; *out_count holds |J|");
    return EIGER_OK;
}
