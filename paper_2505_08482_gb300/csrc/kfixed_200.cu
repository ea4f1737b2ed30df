// Fixed-size passes for the grid side Ng = 200 = 20 x 10.  Variants: 0 column and velocity
// passes on the 20 x 10 factorisation, density passes on 10 x 20 (fewer registers where the
// state is preloaded), and 8-column tiles for the column passes of the forward sweep, which
// runs alone on the GPU; 1 all 20 x 10, 4 rows / 4 columns per CTA; 2 the same with 8 rows /
// 2 columns; 3 state staged in shared memory by TMA bulk copies; 4 all 10 x 20; 5 as 0 with 8 rows per CTA in the row passes; 6 as 0 with the segment recompute's row passes staged by TMA (fewer registers beside the adjoint).
// Variant 7: as 5 with column passes that form their multipliers where they use them (less
// shared memory: for launches of many waves).
#include "kfixed.cuh"

namespace pat {

namespace {
using A4 = FixedImpl<20, 10, 4, 4, false>;
using A8 = FixedImpl<20, 10, 8, 2, false>;
using S4 = FixedImpl<20, 10, 4, 4, true>;
using B4 = FixedImpl<10, 20, 4, 4, false>;
using C8 = FixedImpl<20, 10, 4, 8, false>;
using B8 = FixedImpl<10, 20, 8, 2, false>;   // density rows, 8 rows per CTA
using SB = FixedImpl<10, 20, 4, 4, true>;    // density rows staged by TMA (segment recompute)
using PA = FixedImpl<20, 10, 8, 4, false>;   // persistent sweep: columns and velocity rows
using L4 = ColLeanImpl<20, 10, 4>;   // column passes, multipliers formed where used
using L8 = ColLeanImpl<20, 10, 8>;
using PB = FixedImpl<10, 20, 8, 4, false>;   // persistent sweep: density rows
}  // namespace

const FixedOps* fixed_ops_200(int v) {
    static const FixedOps ops[] = {MixedImpl<A4, A4, B4, B4, C8>::ops(), A4::ops(), A8::ops(), S4::ops(), B4::ops(),
                                   MixedImpl<A4, A8, B8, B8, C8>::ops(),
                                   MixedImpl<A4, A4, B4, B4, C8, S4, SB>::ops(), MixedImpl<L4, A8, B8, B8, L8>::ops()};
    return (v >= 0 && v < int(sizeof(ops) / sizeof(ops[0]))) ? &ops[v] : nullptr;
}

const SweepOps* sweep_ops_200() {
    static const SweepOps ops = SweepImpl<PersistentImpl<PA, PA, PB>>::ops();
    return &ops;
}

}  // namespace pat
