// Host-side planner interface (internal).
#pragma once

#include <stddef.h>
#include <stdint.h>

#include "eiger.h"

namespace eiger {

// Whether a HyperLogLog estimate says nb build keys are (nearly) all distinct.
bool distinct_keys(double estimate, int64_t nb);

// Radix bits the partitioned join uses for nb build rows (distinct: the build
// keys are all distinct, which allows larger partitions).
int phj_total_bits(int64_t nb, bool distinct);

// Power-of-two slot count of a hash table holding nb rows at load_factor.
unsigned long long table_slots(int64_t nb, double load_factor);

// Plan for `variant` (EIGER_AUTO lets the rules choose) from sizes, whether
// the build keys narrow to 32 bits and whether they are distinct, and the
// distinct fraction of a probe sample (estimate / sample rows; < 0 when not
// profiled), which flags a skewed probe side.
eiger_plan_t plan_rules(int variant, int64_t nb, int64_t np, int dtype, bool narrowable, bool distinct,
                        size_t l2_bytes, double probe_distinct = -1.0);

// Whether the rules would consult a probe sample for this join: AUTO would
// partition 32-bit keys and the probe side is at least twice the build side.
bool wants_probe_sample(const eiger_plan_t& rules_plan, int64_t nb, int64_t np, int dtype, bool narrowable);

// Rows of the probe sample the rules profile (the first rows of the column).
constexpr int64_t kProbeSampleRows = 1 << 20;

// HyperLogLog estimate from 2^14 dense registers (Sec. 4.1).
double hll_estimate(const uint8_t* regs);

}  // namespace eiger
