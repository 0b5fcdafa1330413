// DP kernel instantiations for d = 6.
#include "dp.cuh"
#include "dp_variants.h"

namespace knn {

namespace {
template <int DD, int PP>
bool try_launch(const DpArgs &a, int P, int kind, int grid, cudaStream_t st)
{
    if constexpr (DD == 6) {
        if (P == PP)
            return dp_launch_tpl<DD, PP>(a, kind, grid, st);
    }
    return false;
}
template <int DD, int PP>
int try_occ(int P, int kind)
{
    if constexpr (DD == 6) {
        if (P == PP)
            return dp_occupancy_tpl<DD, PP>(kind);
    }
    return 0;
}
}  // namespace

bool dp_launch_d6(const DpArgs &a, int P, int kind, int grid, cudaStream_t st)
{
#define KNN_X(DD, PP) if (try_launch<DD, PP>(a, P, kind, grid, st)) return true;
    KNN_DP_VARIANTS(KNN_X)
#undef KNN_X
    return false;
}

int dp_occ_d6(int P, int kind)
{
    int v = 0;
#define KNN_X(DD, PP) v += try_occ<DD, PP>(P, kind);
    KNN_DP_VARIANTS(KNN_X)
#undef KNN_X
    return v;
}

}  // namespace knn
