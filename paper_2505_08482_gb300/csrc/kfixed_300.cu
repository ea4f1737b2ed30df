// Fixed-size passes for the grid side Ng = 300 = 20 x 15 (tile variants: rows x columns per CTA).
#include "kfixed.cuh"

namespace pat {

const FixedOps* fixed_ops_300(int v) {
    static const FixedOps ops[] = {FixedImpl<20, 15, 4, 4>::ops(), FixedImpl<20, 15, 8, 2>::ops()};
    return (v >= 0 && v < 2) ? &ops[v] : nullptr;
}

}  // namespace pat
