// Rule-based variant selector and knob tuner (host only).
//
// The paper defers the join algorithm and its knobs to run time and decides
// them from cheap statistics (Sec. 1 "algorithm selection" and "knob tuning";
// Table 1: relation cardinalities, key distribution and data types decide the
// join; Sec. 5.2.1-5.2.2: the non-partitioned hash join wins while its table
// stays cache-resident, the partitioned join wins beyond). The rules below
// encode that on a GB300:
//  - keys are narrowed to 32 bits whenever the build range spans < 2^32
//    (frame of reference, Sec. 4.3), which halves table slots and partition
//    tuples;
//  - NPHJ while its table (load factor 0.5) fits half of the L2 cache;
//  - otherwise PHJ with enough radix bits that an average build partition
//    holds at most kTargetRows rows, or kTargetRowsDistinct when the
//    HyperLogLog estimate says the build keys are all distinct
//    (kTargetRowsDistinctLarge from kLargeBuild rows up), in one pass up to
//    kOnePassBits bits and in two balanced passes beyond (pass 2 takes an odd
//    count's extra bit). Measured on GB300: with unique build keys,
//    partitions of 2300-3000 rows beat 1100-1500 rows by 2-16 % (pairs and the
//    fused sum alike, 4.7M to 150M build rows); with duplicate build keys the
//    smaller partitions win by 11-16 % (3000 timed joins). From 2^27 unique
//    rows up, 4096-row partitions win (2^27 x 2^29: 13.7 against 14.1 ms;
//    2^28 x 2^30: 31.1 against 34.8 ms): they keep the second pass at 256
//    digits where 2048-3072-row partitions need 512, whose 8-row digit runs
//    and doubled count arrays slow that pass by a third; below 2^27 they lose
//    (2^24: 1.81 against 1.72 ms);
//  - except under heavy probe skew: when a probe sample of 2^20 rows holds
//    fewer than kSkewHeavy distinct keys per row (Zipf theta ~1.5 gives
//    0.014), or fewer than kSkewModerate with the NPHJ table within 4x the
//    L2 cache (theta ~1 gives 0.22-0.45), and the probe side is at least
//    twice the build side, 32-bit keys go to the NPHJ: hot keys keep their
//    slots in cache, while the partitioned join funnels them through one
//    partition. Measured on the GB300 variant-sweep grid (ms, NPHJ against
//    the rules' PHJ): 2^24 x 4, theta 1.5: 1.40 / 1.90; 2^24 x 16, theta 1:
//    3.73 / 5.13; 2^26 x 16, theta 1.5: 12.95 / 25.1; 2^28 x 4, theta 1.5:
//    28.4 / 33.5; without skew the PHJ wins (2^28 x 4: 49.6 / 31.1). With
//    16-byte slots (64-bit keys) the skewed NPHJ loses from 2^26 up.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "planner.h"

namespace eiger {

namespace {
constexpr int64_t kTargetRows = 2048;           // average build rows per partition
constexpr int64_t kTargetRowsDistinct = 3072;   // ... when the build keys are distinct
constexpr int64_t kTargetRowsDistinctLarge = 4096;  // ... from kLargeBuild build rows up
constexpr int64_t kLargeBuild = 1ll << 27;
static_assert(kTargetRowsDistinctLarge < EIGER_BUILD_CAP, "an average partition fits one table");
constexpr double kDistinctFraction = 0.9;  // estimate / rows above which the keys count as distinct
constexpr int kOnePassBits = 8;
constexpr double kSkewHeavy = 0.1;     // probe sample distinct fraction: heavy skew
constexpr double kSkewModerate = 0.5;  // ... moderate skew
constexpr int kMaxTotalBits = 20;
}  // namespace

bool distinct_keys(double estimate, int64_t nb) {
    return nb > 0 && estimate >= kDistinctFraction * (double)nb;
}

int phj_total_bits(int64_t nb, bool distinct) {
    const int64_t target = !distinct ? kTargetRows : nb >= kLargeBuild ? kTargetRowsDistinctLarge : kTargetRowsDistinct;
    const int64_t parts = (nb + target - 1) / target;
    int b = 0;
    while ((1ll << b) < parts) ++b;
    if (b < 2) b = 2;
    if (b > kMaxTotalBits) b = kMaxTotalBits;
    return b;
}

unsigned long long table_slots(int64_t nb, double load_factor) {
    const double want = (double)(nb > 0 ? nb : 1) / load_factor;
    unsigned long long s = 64;
    while ((double)s < want) s <<= 1;
    return s;
}

bool wants_probe_sample(const eiger_plan_t& rules_plan, int64_t nb, int64_t np, int dtype, bool narrowable) {
    const bool key32 = dtype == EIGER_I32 || narrowable;
    return key32 && np >= 2 * nb && (rules_plan.variant == EIGER_PHJ1 || rules_plan.variant == EIGER_PHJ2);
}

eiger_plan_t plan_rules(int variant, int64_t nb, int64_t np, int dtype, bool narrowable, bool distinct,
                        size_t l2_bytes, double probe_distinct) {
    eiger_plan_t p{};
    p.selector = 0;
    p.load_factor = 0.5f;
    p.narrow = narrowable ? 1 : 0;
    const bool key32 = dtype == EIGER_I32 || narrowable;
    const int B = phj_total_bits(nb, distinct);
    int v = variant;
    if (v == EIGER_AUTO) {
        const unsigned long long bytes = table_slots(nb, 0.5) * (key32 ? 8ull : 16ull);
        const bool skewed = key32 && np >= 2 * nb && probe_distinct >= 0.0 &&
                            (probe_distinct < kSkewHeavy ||
                             (probe_distinct < kSkewModerate && bytes <= 4ull * l2_bytes));
        if (bytes <= l2_bytes / 2 || skewed)
            v = EIGER_NPHJ;
        else
            v = B <= kOnePassBits ? EIGER_PHJ1 : EIGER_PHJ2;
    }
    p.variant = v;
    if (v == EIGER_PHJ1) {
        p.bits1 = std::min(B, 12);
        p.bits2 = 0;
    } else if (v == EIGER_PHJ2) {
        // an odd count's extra bit goes to pass 2: measured on GB300, 7 + 8
        // bits beat 8 + 7 on 2^26 x 2^28 (7.48 against 7.65 ms), while 7 + 9
        // lost to 8 + 8 on the 150M x 600M sum (22.0 against 20.95 ms)
        p.bits1 = B / 2;
        p.bits2 = B - p.bits1;
        if (p.bits2 < 1) {
            p.bits1 = 1;
            p.bits2 = 1;
        }
    } else if (v == EIGER_SMJ) {
        p.bits1 = 8;  // digit bits per sort pass; the passes follow from the key span
        p.bits2 = 0;
    }
    return p;
}

// HyperLogLog estimate (Flajolet et al. 2007, with HyperLogLog++'s 64-bit hash:
// no large-range correction) from the dense registers: the raw estimate
// alpha_m m^2 / sum_j 2^-reg[j], replaced by linear counting m ln(m / V) when V
// registers are still zero and the raw estimate is at most 2.5 m. The harmonic
// sum is accumulated exactly as an integer count of 2^-kRhoMax units, so the
// only rounding is the final fp64 expression, evaluated in a fixed order.
double hll_estimate(const uint8_t* regs) {
    constexpr int kRho = 64 - EIGER_HLL_P + 1;  // largest rank
    uint32_t hist[kRho + 1] = {0};
    for (int j = 0; j < EIGER_HLL_M; ++j) hist[regs[j] <= kRho ? regs[j] : kRho] += 1;
    unsigned __int128 units = 0;
    for (int r = 0; r <= kRho; ++r) units += (unsigned __int128)hist[r] << (kRho - r);
    const double m = (double)EIGER_HLL_M;
    const double alpha = 0.7213 / (1.0 + 1.079 / m);
    double est = alpha * m * m * std::ldexp(1.0, kRho) / (double)units;
    if (hist[0] != 0 && est <= 2.5 * m) est = m * std::log(m / (double)hist[0]);
    return est;
}

}  // namespace eiger
