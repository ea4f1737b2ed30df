// Cluster-resident stepping for the grid side Ng = 300: clusters of 16 CTAs (19 or 18 rows and
// 10 or 9 half-spectrum columns each), rows on the 15 x 20 factorisation (the state of a row
// thread: 15 cells of each field), columns on 20 x 15.
#include "kcluster.cuh"

namespace pat {

const ClusterOps* cluster_ops_300() {
    static const ClusterOps ops = ClusterLaunch<ClusterImpl<300, 16, 15, 20, 20, 15>>::ops();
    return &ops;
}

}  // namespace pat
