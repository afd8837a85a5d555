// Column statistics on the GPU: signed min/max and the dense HyperLogLog++
// registers of one key column (Sec. 4 "runtime profiling"; Sec. 4.1 HLL++).
//
// One streaming pass. Each CTA keeps a private copy of the 2^14 registers in
// shared memory (as 32-bit words so it can use the native shared-memory
// atomicMax), reads its share of the column with 16-byte vector loads, and
// raises a register only when the new rank exceeds it: after the first few
// thousand keys almost every update is a plain shared-memory read. A second,
// tiny kernel takes the byte-wise max of the per-CTA register arrays with
// __vmaxu4 and reduces min/max. The host turns the registers into the estimate.
#include "kernels.cuh"

namespace eiger {

namespace {

constexpr int kThreads = 512;

__device__ __forceinline__ void sketch_visit(int64_t k, int64_t& mn, int64_t& mx,
                                             uint32_t* sreg) {
    mn = k < mn ? k : mn;
    mx = k > mx ? k : mx;
    const uint64_t h = sketch_hash((uint64_t)k);
    const uint32_t idx = (uint32_t)(h >> (64 - kHllP));
    const uint64_t w = h << kHllP;
    const uint32_t rho = w ? (uint32_t)__clzll((long long)w) + 1u : (uint32_t)kRhoMax;
    if (rho > sreg[idx]) atomicMax(&sreg[idx], rho);
}

template <typename K>
struct Vec16;
template <>
struct Vec16<int32_t> {
    using T = int4;
    static constexpr int kN = 4;
    __device__ __forceinline__ static int64_t at(const int4& v, int i) {
        return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
    }
};
template <>
struct Vec16<int64_t> {
    using T = longlong2;
    static constexpr int kN = 2;
    __device__ __forceinline__ static int64_t at(const longlong2& v, int i) {
        return i == 0 ? v.x : v.y;
    }
};

template <typename K>
__global__ void __launch_bounds__(kThreads)
    stats_partial_kernel(const K* __restrict__ keys, int64_t n, uint32_t* __restrict__ part_regs,
                         int64_t* __restrict__ part_mm) {
    using V = Vec16<K>;
    extern __shared__ uint32_t sreg[];
    __shared__ int64_t s_mn[kThreads / kWarp], s_mx[kThreads / kWarp];

    for (int i = threadIdx.x; i < kHllM; i += blockDim.x) sreg[i] = 0;
    __syncthreads();

    int64_t mn = INT64_MAX, mx = INT64_MIN;

    // Elements before the first 16-byte boundary, then the aligned body with
    // vector loads (four in flight per thread), then the ragged tail.
    const uintptr_t addr = reinterpret_cast<uintptr_t>(keys);
    int64_t head = (int64_t)(((16u - (addr & 15u)) & 15u) / sizeof(K));
    if (head > n) head = n;
    if (blockIdx.x == 0 && (int64_t)threadIdx.x < head) sketch_visit(keys[threadIdx.x], mn, mx, sreg);

    const int64_t nvec = (n - head) / V::kN;
    const typename V::T* vp = reinterpret_cast<const typename V::T*>(keys + head);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < nvec; i += 4 * stride) {
        typename V::T a = __ldcs(vp + i);
        typename V::T b = __ldcs(vp + i + stride);
        typename V::T c = __ldcs(vp + i + 2 * stride);
        typename V::T d = __ldcs(vp + i + 3 * stride);
#pragma unroll
        for (int j = 0; j < V::kN; ++j) sketch_visit(V::at(a, j), mn, mx, sreg);
#pragma unroll
        for (int j = 0; j < V::kN; ++j) sketch_visit(V::at(b, j), mn, mx, sreg);
#pragma unroll
        for (int j = 0; j < V::kN; ++j) sketch_visit(V::at(c, j), mn, mx, sreg);
#pragma unroll
        for (int j = 0; j < V::kN; ++j) sketch_visit(V::at(d, j), mn, mx, sreg);
    }
    for (; i < nvec; i += stride) {
        typename V::T a = __ldcs(vp + i);
#pragma unroll
        for (int j = 0; j < V::kN; ++j) sketch_visit(V::at(a, j), mn, mx, sreg);
    }
    const int64_t tail = head + nvec * V::kN;
    if (blockIdx.x == gridDim.x - 1)
        for (int64_t t = tail + threadIdx.x; t < n; t += blockDim.x) sketch_visit(keys[t], mn, mx, sreg);

    // CTA min/max.
#pragma unroll
    for (int o = kWarp / 2; o > 0; o >>= 1) {
        int64_t a = __shfl_xor_sync(0xffffffffu, mn, o);
        int64_t b = __shfl_xor_sync(0xffffffffu, mx, o);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
    }
    const int warp = threadIdx.x / kWarp;
    if (lane_id() == 0) {
        s_mn[warp] = mn;
        s_mx[warp] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x / kWarp); ++w) {
            mn = s_mn[w] < mn ? s_mn[w] : mn;
            mx = s_mx[w] > mx ? s_mx[w] : mx;
        }
        part_mm[2 * blockIdx.x] = mn;
        part_mm[2 * blockIdx.x + 1] = mx;
    }
    // Registers as bytes, four per 32-bit word (little-endian register order).
    for (int w = threadIdx.x; w < kHllM / 4; w += blockDim.x) {
        const uint32_t* r = sreg + 4 * w;
        part_regs[(size_t)blockIdx.x * (kHllM / 4) + w] =
            r[0] | (r[1] << 8) | (r[2] << 16) | (r[3] << 24);
    }
}

__global__ void __launch_bounds__(256)
    stats_merge_kernel(const uint32_t* __restrict__ part_regs, const int64_t* __restrict__ part_mm,
                       int grid, StatsDev* __restrict__ out) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w < kHllM / 4) {
        // four independent running maxima, so 16 loads are in flight per
        // thread instead of one dependent load per partial array
        uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
        const uint32_t* p = part_regs + w;
        constexpr size_t W = kHllM / 4;
        int g = 0;
#pragma unroll 4
        for (; g + 4 <= grid; g += 4) {
            m0 = __vmaxu4(m0, p[(size_t)(g + 0) * W]);
            m1 = __vmaxu4(m1, p[(size_t)(g + 1) * W]);
            m2 = __vmaxu4(m2, p[(size_t)(g + 2) * W]);
            m3 = __vmaxu4(m3, p[(size_t)(g + 3) * W]);
        }
        for (; g < grid; ++g) m0 = __vmaxu4(m0, p[(size_t)g * W]);
        out->regs[w] = __vmaxu4(__vmaxu4(m0, m1), __vmaxu4(m2, m3));
    }
    if (blockIdx.x == 0) {
        __shared__ int64_t s_mn[256 / kWarp], s_mx[256 / kWarp];
        int64_t mn = INT64_MAX, mx = INT64_MIN;
        for (int g = threadIdx.x; g < grid; g += blockDim.x) {
            int64_t a = part_mm[2 * g], b = part_mm[2 * g + 1];
            mn = a < mn ? a : mn;
            mx = b > mx ? b : mx;
        }
#pragma unroll
        for (int o = kWarp / 2; o > 0; o >>= 1) {
            int64_t a = __shfl_xor_sync(0xffffffffu, mn, o);
            int64_t b = __shfl_xor_sync(0xffffffffu, mx, o);
            mn = a < mn ? a : mn;
            mx = b > mx ? b : mx;
        }
        if (lane_id() == 0) {
            s_mn[threadIdx.x / kWarp] = mn;
            s_mx[threadIdx.x / kWarp] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int i = 1; i < (int)(blockDim.x / kWarp); ++i) {
                mn = s_mn[i] < mn ? s_mn[i] : mn;
                mx = s_mx[i] > mx ? s_mx[i] : mx;
            }
            out->mn = mn;
            out->mx = mx;
        }
    }
}

template <typename K>
cudaError_t configure_partial(int dev) {
    static bool done[64] = {};
    if (dev >= 0 && dev < 64 && done[dev]) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(stats_partial_kernel<K>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kHllM * (int)sizeof(uint32_t));
    if (e == cudaSuccess && dev >= 0 && dev < 64) done[dev] = true;
    return e;
}

}  // namespace

StatsScratch stats_layout(Carve& c) {
    StatsScratch s;
    s.part_regs = c.take<uint32_t>((size_t)kStatsMaxGrid * (kHllM / 4));
    s.part_mm = c.take<int64_t>(2 * (size_t)kStatsMaxGrid);
    s.out = c.take<StatsDev>(1);
    return s;
}

cudaError_t stats_launch(const void* keys, int64_t n, int dtype, const StatsScratch& s,
                         cudaStream_t stream) {
    DevInfo di;
    cudaError_t e = current_device_info(&di);
    if (e != cudaSuccess) return e;
    const int64_t per_cta = (int64_t)kThreads * 64;  // at least 64 keys per thread
    int64_t want = (n + per_cta - 1) / per_cta;
    int grid = (int)(want < 1 ? 1 : want);
    const int cap = di.sms * 3 < kStatsMaxGrid ? di.sms * 3 : kStatsMaxGrid;
    if (grid > cap) grid = cap;
    const size_t smem = kHllM * sizeof(uint32_t);
    const double kb = dtype == 0 ? 4.0 : 8.0;
    if (dtype == 0) {
        if ((e = configure_partial<int32_t>(di.dev)) != cudaSuccess) return e;
        ProfScope ps("stats_partial", kb * n, stream);
        stats_partial_kernel<int32_t><<<grid, kThreads, smem, stream>>>(
            static_cast<const int32_t*>(keys), n, s.part_regs, s.part_mm);
    } else {
        if ((e = configure_partial<int64_t>(di.dev)) != cudaSuccess) return e;
        ProfScope ps("stats_partial", kb * n, stream);
        stats_partial_kernel<int64_t><<<grid, kThreads, smem, stream>>>(
            static_cast<const int64_t*>(keys), n, s.part_regs, s.part_mm);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    ProfScope ps("stats_merge", (double)grid * (kHllM + 16) + kHllM + 16, stream);
    stats_merge_kernel<<<(kHllM / 4 + 255) / 256, 256, 0, stream>>>(s.part_regs, s.part_mm, grid,
                                                                     s.out);
    return cudaGetLastError();
}

}  // namespace eiger
