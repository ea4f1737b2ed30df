// Fixed-size passes for the grid side Ng = 200 = 20 x 10 (tile variants: rows x columns per CTA).
#include "kfixed.cuh"

namespace pat {

const FixedOps* fixed_ops_200(int v) {
    static const FixedOps ops[] = {FixedImpl<20, 10, 4, 4>::ops(), FixedImpl<20, 10, 8, 2>::ops()};
    return (v >= 0 && v < 2) ? &ops[v] : nullptr;
}

}  // namespace pat
