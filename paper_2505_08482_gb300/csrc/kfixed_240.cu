// Fixed-size passes for the grid side Ng = 240 = 16 x 15 (tile variants: rows x columns per CTA).
#include "kfixed.cuh"

namespace pat {

const FixedOps* fixed_ops_240(int v) {
    static const FixedOps ops[] = {FixedImpl<16, 15, 4, 4>::ops(), FixedImpl<16, 15, 8, 2>::ops()};
    return (v >= 0 && v < 2) ? &ops[v] : nullptr;
}

}  // namespace pat
