// npcf_pairs_d2.cu -- instantiations of the pair kernel for D=2.
#include "npcf_pairs.cuh"

namespace npcf {

// lmax values compiled for D=2; a plan runs the smallest one >= its lmax
static const int kLf[] = {2, 4, 6, 8, 10, 12};
static const int kLd[] = {2, 4, 6, 8, 10, 12};

int pair_compiled_lmax_d2(int fp64, int lmax)
{
    const int* L = fp64 ? kLd : kLf;
    const int n = fp64 ? (int)(sizeof(kLd) / sizeof(int)) : (int)(sizeof(kLf) / sizeof(int));
    for (int i = 0; i < n; ++i)
        if (L[i] >= lmax) return L[i];
    return -1;
}

int pair_threads_d2(int fp64, int L)
{
    switch (L * 2 + (fp64 ? 1 : 0)) {
        case 4: return PairCfg<2, 2, float>::kThreads;
        case 8: return PairCfg<2, 4, float>::kThreads;
        case 12: return PairCfg<2, 6, float>::kThreads;
        case 16: return PairCfg<2, 8, float>::kThreads;
        case 20: return PairCfg<2, 10, float>::kThreads;
        case 24: return PairCfg<2, 12, float>::kThreads;
        case 5: return PairCfg<2, 2, double>::kThreads;
        case 9: return PairCfg<2, 4, double>::kThreads;
        case 13: return PairCfg<2, 6, double>::kThreads;
        case 17: return PairCfg<2, 8, double>::kThreads;
        case 21: return PairCfg<2, 10, double>::kThreads;
        case 25: return PairCfg<2, 12, double>::kThreads;
        default: return -1;
    }
}

cudaError_t launch_pairs_d2(const PairParams& p, int fp64, int L, int grid, int smem, cudaStream_t s)
{
    switch (L * 2 + (fp64 ? 1 : 0)) {
        case 4: return launch_pairs_t<2, 2, float>(p, grid, smem, s);
        case 8: return launch_pairs_t<2, 4, float>(p, grid, smem, s);
        case 12: return launch_pairs_t<2, 6, float>(p, grid, smem, s);
        case 16: return launch_pairs_t<2, 8, float>(p, grid, smem, s);
        case 20: return launch_pairs_t<2, 10, float>(p, grid, smem, s);
        case 24: return launch_pairs_t<2, 12, float>(p, grid, smem, s);
        case 5: return launch_pairs_t<2, 2, double>(p, grid, smem, s);
        case 9: return launch_pairs_t<2, 4, double>(p, grid, smem, s);
        case 13: return launch_pairs_t<2, 6, double>(p, grid, smem, s);
        case 17: return launch_pairs_t<2, 8, double>(p, grid, smem, s);
        case 21: return launch_pairs_t<2, 10, double>(p, grid, smem, s);
        case 25: return launch_pairs_t<2, 12, double>(p, grid, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npcf
