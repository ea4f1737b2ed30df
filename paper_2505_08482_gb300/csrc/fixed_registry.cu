// Registry of the fixed-size passes: grid sides with compiled register FFTs.
#include "kcluster.cuh"

namespace pat {

const FixedOps* fixed_ops_108(int v);
const FixedOps* fixed_ops_144(int v);
const FixedOps* fixed_ops_180(int v);
const FixedOps* fixed_ops_200(int v);
const FixedOps* fixed_ops_240(int v);
const FixedOps* fixed_ops_300(int v);
const SweepOps* sweep_ops_108();
const SweepOps* sweep_ops_144();
const SweepOps* sweep_ops_180();
const SweepOps* sweep_ops_200();
const SweepOps* sweep_ops_240();
const SweepOps* sweep_ops_300();
const ClusterOps* cluster_ops_300();

const ClusterOps* cluster_ops_for(int ng) { return ng == 300 ? cluster_ops_300() : nullptr; }

const FixedOps* fixed_ops_for(int ng, int v) {
    switch (ng) {
        case 108: return fixed_ops_108(v);
        case 144: return fixed_ops_144(v);
        case 180: return fixed_ops_180(v);
        case 200: return fixed_ops_200(v);
        case 240: return fixed_ops_240(v);
        case 300: return fixed_ops_300(v);
        default: return nullptr;
    }
}

const SweepOps* sweep_ops_for(int ng) {
    switch (ng) {
        case 108: return sweep_ops_108();
        case 144: return sweep_ops_144();
        case 180: return sweep_ops_180();
        case 200: return sweep_ops_200();
        case 240: return sweep_ops_240();
        case 300: return sweep_ops_300();
        default: return nullptr;
    }
}

int fixed_variants(int ng) {
    int v = 0;
    while (fixed_ops_for(ng, v)) ++v;
    return v;
}

}  // namespace pat
