// CPU oracle for the runtime-adaptive equi-join path of "Eiger: An Efficient
// Library for GPU-based Data Analytics".
//
// TEST INFRASTRUCTURE ONLY. Nothing in the product library links, includes or
// calls this file; only the test suite, the smoke check and the CPU-baseline
// leg of the benchmark load it. It shares no code, header, table or constant
// generator with the CUDA path. Every function is the plain definition of what
// the GPU path computes, written for a reader who checks it against the paper:
// no blocking, no fusion, fp64 where floating point occurs. Single-threaded,
// except the "-t N" entry points (oracle_join_mt, oracle_join_fingerprint),
// which split only the probe loop over host threads.
//
// Pins (checked by the CPU tests, independent of this file):
//   join            nested-loop brute force; |J| = sum_k cnt_R(k) * cnt_S(k);
//                   closed forms of the permutation workloads.
//   join (-t N)     identical output to the one-thread join.
//   fingerprint     the sum / xor of h64 over brute-force pairs, in Python.
//   join sum        direct addressing over dense dimension keys.
//   h64             published SplitMix64 output sequence; bijectivity.
//   hll registers   multiset/set invariance, union = register-wise max.
//   hll estimate    closed forms for constant registers and for linear
//                   counting; statistical accuracy vs 1.04/sqrt(m).
//   exact ndv       Python set() on small inputs.
//   min/max         numpy min/max.
//   group-by        Python dict brute force; sum of counts = rows; sum of
//                   group sums = column sum; closed forms of i mod g keys.
//
// Build: g++ -O2 -std=c++17 -ffp-contract=off -pthread -shared -fPIC oracle.cpp
// (-ffp-contract=off keeps the estimate formula evaluated exactly as written.)

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

// Key columns arrive as int32 (dtype 0) or int64 (dtype 1). Both are widened
// to int64 by sign extension, so an int32 key and the same value stored as
// int64 are the same join key and hash identically (Sec. 3.1: typed columns).
int64_t key_at(int dtype, const void* keys, int64_t i) {
    if (dtype == 0) return (int64_t)((const int32_t*)keys)[i];
    return ((const int64_t*)keys)[i];
}

// Payload columns are 4 or 8 bytes wide, widened by sign extension.
int64_t pay_at(int pay_bytes, const void* pay, int64_t i) {
    if (pay_bytes == 4) return (int64_t)((const int32_t*)pay)[i];
    return ((const int64_t*)pay)[i];
}

// 64-bit hash feeding the HyperLogLog sketch: the output function of
// SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014), applied to the key's 64-bit two's-complement
// pattern. The sketch itself (Sec. 4.1, HyperLogLog++) only needs a 64-bit
// hash with uniform bits; this bijective mixer is the reading taken here.
uint64_t h64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

const int kP = 14;                 // HLL precision p
const int64_t kM = 1LL << kP;      // m = 2^p registers
const int kRhoMax = 64 - kP + 1;   // largest rank, taken when the low 50 bits are all zero

int clz64(uint64_t w) {
    int n = 0;
    for (int b = 63; b >= 0; --b) {
        if ((w >> b) & 1ULL) break;
        ++n;
    }
    return n;
}

}  // namespace

extern "C" {

uint64_t oracle_h64(uint64_t x) { return h64(x); }

// Join result as a multiset of index pairs (Sec. 3.2 "Joins"; Sec. 2.2: the
// join emits tuple IDs, payloads are materialised from them later):
//   J = { (i, j) : R.key[i] == S.key[j] }.
// Built with std::unordered_multimap over R, probed with every row of S in
// order. Pairs are returned sorted by (probe index, build index): the
// canonical order the GPU output is sorted into before comparison.
// Returns |J|. At most `cap` pairs are written; the rest are only counted.
int64_t oracle_join(int dtype, const void* bkeys, int64_t nb, const void* pkeys, int64_t np,
                    uint32_t* out_b, uint32_t* out_p, int64_t cap) {
    std::unordered_multimap<int64_t, uint32_t> table;
    table.reserve((size_t)nb);
    for (int64_t i = 0; i < nb; ++i) table.emplace(key_at(dtype, bkeys, i), (uint32_t)i);

    std::vector<std::pair<uint32_t, uint32_t>> pairs;  // (probe, build)
    int64_t count = 0;
    for (int64_t j = 0; j < np; ++j) {
        auto range = table.equal_range(key_at(dtype, pkeys, j));
        for (auto it = range.first; it != range.second; ++it) {
            if (count < cap) pairs.emplace_back((uint32_t)j, it->second);
            ++count;
        }
    }
    std::sort(pairs.begin(), pairs.end());
    for (size_t k = 0; k < pairs.size(); ++k) {
        out_p[k] = pairs[k].first;
        out_b[k] = pairs[k].second;
    }
    return count;
}

// The same join with the probe loop split over `threads` host threads (the
// oracle's "-t N" mode, for timing on a many-core host). The multimap is built
// by one thread as above; thread t probes the contiguous probe rows
// [t*np/threads, (t+1)*np/threads) in order and keeps its pairs; the lists are
// concatenated in thread order and sorted canonically, so the output is
// identical to oracle_join's. Returns |J|; writes at most `cap` pairs.
int64_t oracle_join_mt(int dtype, const void* bkeys, int64_t nb, const void* pkeys, int64_t np,
                       uint32_t* out_b, uint32_t* out_p, int64_t cap, int threads) {
    if (threads < 1) threads = 1;
    std::unordered_multimap<int64_t, uint32_t> table;
    table.reserve((size_t)nb);
    for (int64_t i = 0; i < nb; ++i) table.emplace(key_at(dtype, bkeys, i), (uint32_t)i);

    std::vector<std::vector<std::pair<uint32_t, uint32_t>>> part((size_t)threads);
    auto probe_range = [&](int t) {
        const int64_t lo = np * t / threads, hi = np * (t + 1) / threads;
        for (int64_t j = lo; j < hi; ++j) {
            auto range = table.equal_range(key_at(dtype, pkeys, j));
            for (auto it = range.first; it != range.second; ++it) {
                part[(size_t)t].emplace_back((uint32_t)j, it->second);
            }
        }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(probe_range, t);
    probe_range(0);
    for (auto& th : pool) th.join();

    std::vector<std::pair<uint32_t, uint32_t>> pairs;  // (probe, build)
    int64_t count = 0;
    for (int t = 0; t < threads; ++t) {
        for (const auto& pr : part[(size_t)t]) {
            if (count < cap) pairs.push_back(pr);
            ++count;
        }
        std::vector<std::pair<uint32_t, uint32_t>>().swap(part[(size_t)t]);
    }
    std::sort(pairs.begin(), pairs.end());
    for (size_t k = 0; k < pairs.size(); ++k) {
        out_p[k] = pairs[k].first;
        out_b[k] = pairs[k].second;
    }
    return count;
}

// Order-independent summary of a join result too large to sort on the host:
// |J| and two 64-bit fingerprints of the pair multiset, with the pair (i, j)
// read as the 64-bit word w = i * 2^32 + j:
//   fp_sum = sum over J of h64(w)              (mod 2^64)
//   fp_xor = xor over J of h64(w + 0x9E3779B97F4A7C15)
// (the second is h64 at SplitMix64's next state, a different mixing of the
// same word). Equal multisets give equal summaries; a missing, extra or
// altered pair changes both fingerprints except with probability ~2^-64. The
// pairs are produced by the same multimap definition as oracle_join and
// streamed, never stored; the probe loop is split over `threads` host threads
// (modular sums and xors of the per-thread parts do not depend on the split).
int64_t oracle_join_fingerprint(int dtype, const void* bkeys, int64_t nb, const void* pkeys, int64_t np,
                                int threads, uint64_t* fp_sum, uint64_t* fp_xor) {
    if (threads < 1) threads = 1;
    std::unordered_multimap<int64_t, uint32_t> table;
    table.reserve((size_t)nb);
    for (int64_t i = 0; i < nb; ++i) table.emplace(key_at(dtype, bkeys, i), (uint32_t)i);
    std::vector<uint64_t> s((size_t)threads, 0), x((size_t)threads, 0);
    std::vector<int64_t> c((size_t)threads, 0);
    auto probe_range = [&](int t) {
        const int64_t lo = np * t / threads, hi = np * (t + 1) / threads;
        uint64_t ss = 0, xx = 0;
        int64_t cc = 0;
        for (int64_t j = lo; j < hi; ++j) {
            auto range = table.equal_range(key_at(dtype, pkeys, j));
            for (auto it = range.first; it != range.second; ++it) {
                const uint64_t w = ((uint64_t)it->second << 32) | (uint64_t)(uint32_t)j;
                ss += h64(w);
                xx ^= h64(w + 0x9E3779B97F4A7C15ULL);
                ++cc;
            }
        }
        s[(size_t)t] = ss;
        x[(size_t)t] = xx;
        c[(size_t)t] = cc;
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < threads; ++t) pool.emplace_back(probe_range, t);
    probe_range(0);
    for (auto& th : pool) th.join();
    uint64_t ss = 0, xx = 0;
    int64_t cc = 0;
    for (int t = 0; t < threads; ++t) {
        ss += s[(size_t)t];
        xx ^= x[(size_t)t];
        cc += c[(size_t)t];
    }
    *fp_sum = ss;
    *fp_xor = xx;
    return cc;
}

// |J| only, with no pair storage (same multimap definition as above).
int64_t oracle_join_count(int dtype, const void* bkeys, int64_t nb, const void* pkeys, int64_t np) {
    std::unordered_multimap<int64_t, uint32_t> table;
    table.reserve((size_t)nb);
    for (int64_t i = 0; i < nb; ++i) table.emplace(key_at(dtype, bkeys, i), (uint32_t)i);
    int64_t count = 0;
    for (int64_t j = 0; j < np; ++j) count += (int64_t)table.count(key_at(dtype, pkeys, j));
    return count;
}

// Aggregate over the join result: sum over (i, j) in J of (R.pay[i] + S.pay[j]),
// in 64-bit wrap-around arithmetic, i.e. exact modulo 2^64. This is the
// "payload summed per match" of the foreign-key join (a dimension table joined
// with a fact table, the shape of the TPC-H joins of Sec. 5.7). Modular addition is associative
// and commutative, so the value does not depend on the order of the matches.
// Returns the sum; *count receives |J|.
int64_t oracle_join_sum(int dtype, const void* bkeys, const void* bpay, int64_t nb,
                        const void* pkeys, const void* ppay, int64_t np, int pay_bytes,
                        int64_t* count) {
    std::unordered_multimap<int64_t, uint32_t> table;
    table.reserve((size_t)nb);
    for (int64_t i = 0; i < nb; ++i) table.emplace(key_at(dtype, bkeys, i), (uint32_t)i);
    uint64_t sum = 0;
    int64_t c = 0;
    for (int64_t j = 0; j < np; ++j) {
        auto range = table.equal_range(key_at(dtype, pkeys, j));
        for (auto it = range.first; it != range.second; ++it) {
            sum += (uint64_t)pay_at(pay_bytes, bpay, it->second);
            sum += (uint64_t)pay_at(pay_bytes, ppay, j);
            ++c;
        }
    }
    *count = c;
    return (int64_t)sum;
}

// Column statistics of Sec. 4 ("runtime profiling"): signed minimum, signed
// maximum and the dense HyperLogLog++ register array (Sec. 4.1), computed by
// one sequential pass in row order.
//   h      = h64(key as 64-bit two's complement)
//   idx    = the top p bits of h
//   w      = h shifted left by p (the remaining 64 - p bits, left-aligned)
//   rho    = position of the leftmost 1 bit of w, counting from 1; 64 - p + 1
//            when those bits are all zero
//   reg[idx] = max(reg[idx], rho)
// Empty input: min = INT64_MAX, max = INT64_MIN, all registers 0.
void oracle_stats(int dtype, const void* keys, int64_t n, int64_t* out_min, int64_t* out_max,
                  uint8_t* regs) {
    int64_t mn = INT64_MAX, mx = INT64_MIN;
    for (int64_t r = 0; r < kM; ++r) regs[r] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t k = key_at(dtype, keys, i);
        if (k < mn) mn = k;
        if (k > mx) mx = k;
        uint64_t h = h64((uint64_t)k);
        uint64_t idx = h >> (64 - kP);
        uint64_t w = h << kP;
        int rho = (w == 0) ? kRhoMax : clz64(w) + 1;
        if (rho > regs[idx]) regs[idx] = (uint8_t)rho;
    }
    *out_min = mn;
    *out_max = mx;
}

// HyperLogLog cardinality estimate from the dense registers (Flajolet, Fusy,
// Gandouet & Meunier 2007, as used by HyperLogLog++ with a 64-bit hash, so no
// large-range correction). Evaluated in this order, in fp64:
//   c[r]  = number of registers equal to r, r = 0 .. 64 - p + 1
//   Z     = sum_r c[r] * 2^(51 - r), exact in 128-bit integers
//           (= 2^51 * sum_j 2^-reg[j])
//   alpha = 0.7213 / (1 + 1.079 / m)
//   E     = alpha * m * m * 2^51 / Z
//   if c[0] > 0 and E <= 2.5 m:  E = m * ln(m / c[0])      (linear counting)
// HyperLogLog++'s empirical bias tables are not applied.
double oracle_hll_estimate(const uint8_t* regs) {
    int64_t c[kRhoMax + 1];
    for (int r = 0; r <= kRhoMax; ++r) c[r] = 0;
    for (int64_t j = 0; j < kM; ++j) c[regs[j]] += 1;
    unsigned __int128 z = 0;
    for (int r = 0; r <= kRhoMax; ++r) z += (unsigned __int128)c[r] << (kRhoMax - r);
    const double m = (double)kM;
    const double alpha = 0.7213 / (1.0 + 1.079 / m);
    double e = alpha * m * m * 0x1p51 / (double)z;
    if (c[0] > 0 && e <= 2.5 * m) e = m * std::log(m / (double)c[0]);
    return e;
}

// Exact number of distinct values: sort, then count the runs.
int64_t oracle_exact_ndv(int dtype, const void* keys, int64_t n) {
    std::vector<int64_t> v((size_t)n);
    for (int64_t i = 0; i < n; ++i) v[(size_t)i] = key_at(dtype, keys, i);
    std::sort(v.begin(), v.end());
    return (int64_t)(std::unique(v.begin(), v.end()) - v.begin());
}

// Group-by with aggregates (Sec. 3.3 group-by; Sec. 4.2: the number of groups
// decides the algorithm). For every distinct key of keys[0, n), in ascending
// key order: the key and, for each aggregate a, op[a] over the rows of that
// key of value column vals[a] (vbytes[a] = 4 or 8, sign-extended):
//   op 0 SUM   (modulo 2^64, returned as int64: exact and order-independent),
//   op 1 COUNT (rows; vals[a] unused),
//   op 2 MIN, op 3 MAX (signed).
// Writes min(groups, cap) groups: out_keys[g], out_aggs[a * cap + g].
// Returns the number of groups.
int64_t oracle_groupby(int dtype, const void* keys, int64_t n, int nagg, const int* op, const int* vbytes,
                       const void* const* vals, int64_t* out_keys, int64_t* out_aggs, int64_t cap) {
    std::map<int64_t, std::vector<int64_t>> groups;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t k = key_at(dtype, keys, i);
        auto it = groups.find(k);
        if (it == groups.end()) {
            std::vector<int64_t> init(nagg);
            for (int a = 0; a < nagg; ++a)
                init[a] = op[a] == 2 ? INT64_MAX : op[a] == 3 ? INT64_MIN : 0;
            it = groups.emplace(k, init).first;
        }
        for (int a = 0; a < nagg; ++a) {
            int64_t v = 0;
            if (op[a] != 1) v = vbytes[a] == 4 ? (int64_t)((const int32_t*)vals[a])[i] : ((const int64_t*)vals[a])[i];
            int64_t& acc = it->second[a];
            if (op[a] == 0)
                acc = (int64_t)((uint64_t)acc + (uint64_t)v);
            else if (op[a] == 1)
                acc += 1;
            else if (op[a] == 2)
                acc = std::min(acc, v);
            else
                acc = std::max(acc, v);
        }
    }
    int64_t g = 0;
    for (const auto& kv : groups) {
        if (g < cap) {
            out_keys[g] = kv.first;
            for (int a = 0; a < nagg; ++a) out_aggs[(int64_t)a * cap + g] = kv.second[a];
        }
        ++g;
    }
    return g;
}

}  // extern "C"
