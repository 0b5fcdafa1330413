// Dispatch over the compiled (D, P) variants of the DP kernel (one unit per
// width, generated by build.py).
#include "dp.cuh"
#include "dp_variants.h"

namespace knn {

#define KNN_DECL(D)                                                                  \
    bool dp_launch_d##D(const DpArgs &a, int P, int kind, int n_sm, cudaStream_t st); \
    int dp_occ_d##D(int P, int kind);
KNN_DECL(1) KNN_DECL(2) KNN_DECL(3) KNN_DECL(4) KNN_DECL(5) KNN_DECL(6) KNN_DECL(7) KNN_DECL(8)
KNN_DECL(16)
#undef KNN_DECL

bool launch_dp(const DpArgs &a, int d, int P, int kind, int n_sm, cudaStream_t st)
{
    switch (d) {
    case 1: return dp_launch_d1(a, P, kind, n_sm, st);
    case 2: return dp_launch_d2(a, P, kind, n_sm, st);
    case 3: return dp_launch_d3(a, P, kind, n_sm, st);
    case 4: return dp_launch_d4(a, P, kind, n_sm, st);
    case 5: return dp_launch_d5(a, P, kind, n_sm, st);
    case 6: return dp_launch_d6(a, P, kind, n_sm, st);
    case 7: return dp_launch_d7(a, P, kind, n_sm, st);
    case 8: return dp_launch_d8(a, P, kind, n_sm, st);
    case 16: return dp_launch_d16(a, P, kind, n_sm, st);
    default: return false;
    }
}

int dp_max_blocks_per_sm(int d, int P, int kind)
{
    switch (d) {
    case 1: return dp_occ_d1(P, kind);
    case 2: return dp_occ_d2(P, kind);
    case 3: return dp_occ_d3(P, kind);
    case 4: return dp_occ_d4(P, kind);
    case 5: return dp_occ_d5(P, kind);
    case 6: return dp_occ_d6(P, kind);
    case 7: return dp_occ_d7(P, kind);
    case 8: return dp_occ_d8(P, kind);
    case 16: return dp_occ_d16(P, kind);
    default: return 0;
    }
}

int dp_block_threads() { return DP_THREADS; }

static const int kVariants[][2] = {
#define KNN_X(DD, PP) {DD, PP},
    KNN_DP_VARIANTS(KNN_X)
#undef KNN_X
};

int dp_num_variants(int d)
{
    int c = 0;
    for (auto &v : kVariants)
        c += v[0] == d;
    return c;
}

int dp_variant_P(int d, int idx)
{
    for (auto &v : kVariants)
        if (v[0] == d && idx-- == 0)
            return v[1];
    return 0;
}

}  // namespace knn
