// Test hooks of the planner (host only; no kernel includes this header).
#pragma once

#include <cstdint>

namespace msadp {

// A nonzero seed makes later plans permute the tickets inside every wave
// (seeded, reproducible), so tests can run the kernels under other topological
// orders of the same dependency graph; 0 (the default) keeps the canonical order.
void set_wave_shuffle_seed(uint64_t seed);
uint64_t wave_shuffle_seed();

}  // namespace msadp
