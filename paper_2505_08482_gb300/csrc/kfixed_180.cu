// Fixed-size passes for the grid side Ng = 180 = 12 x 15 (tile variants: rows x columns per CTA).
#include "kfixed.cuh"

namespace pat {

const FixedOps* fixed_ops_180(int v) {
    static const FixedOps ops[] = {FixedImpl<12, 15, 4, 4>::ops(), FixedImpl<12, 15, 8, 2>::ops()};
    return (v >= 0 && v < 2) ? &ops[v] : nullptr;
}

}  // namespace pat
