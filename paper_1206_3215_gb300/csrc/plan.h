// Launch plans shared by the pass launchers and the engine.
#pragma once
#include <atomic>

namespace pss {

// Plans: each pass kernel instance (equation op, length, precision) has a
// process-wide slot holding the launch-shape variant it runs in (-1: not
// chosen, variant 0).  The autotuner times the variants on a grid's own step
// and writes the winner into the slots that step used, so every grid of the
// same equation, size and precision then runs the same kernels (a batch stays
// equal to its fields run alone).  Only lean FP32 ops of length >= 512 whose
// tiling the caller does not depend on are compiled in both variants.
struct PlanSlot {
    std::atomic<int> var{-1};
};
struct PlanTuning {
    int force = -1;             // >= 0: every tunable launch runs this variant
    int open_kind = -1;         // pass being timed (0 row, 1 column), -1: none
    PlanSlot *used[2][8] = {};  // slots launched inside timed row / column passes
    int nused[2] = {0, 0};
};
PlanTuning *plan_tuning();   // this thread's tuning state (engine.cu)
std::atomic<int> &plan_epoch();  // bumped whenever a slot changes (cached graphs are stale)

}  // namespace pss
