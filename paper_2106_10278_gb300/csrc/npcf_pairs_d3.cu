// npcf_pairs_d3.cu -- instantiations of the pair kernel for D=3.
#include "npcf_pairs.cuh"

namespace npcf {

// lmax values compiled for D=3; a plan runs the smallest one >= its lmax
static const int kLf[] = {1, 2, 3, 4, 5, 6, 8, 10};
static const int kLd[] = {1, 2, 3, 4, 5, 6};

int pair_compiled_lmax_d3(int fp64, int lmax)
{
    const int* L = fp64 ? kLd : kLf;
    const int n = fp64 ? (int)(sizeof(kLd) / sizeof(int)) : (int)(sizeof(kLf) / sizeof(int));
    for (int i = 0; i < n; ++i)
        if (L[i] >= lmax) return L[i];
    return -1;
}

int pair_threads_d3(int fp64, int L)
{
    switch (L * 2 + (fp64 ? 1 : 0)) {
        case 2: return PairCfg<3, 1, float>::kThreads;
        case 4: return PairCfg<3, 2, float>::kThreads;
        case 6: return PairCfg<3, 3, float>::kThreads;
        case 8: return PairCfg<3, 4, float>::kThreads;
        case 10: return PairCfg<3, 5, float>::kThreads;
        case 12: return PairCfg<3, 6, float>::kThreads;
        case 16: return PairCfg<3, 8, float>::kThreads;
        case 20: return PairCfg<3, 10, float>::kThreads;
        case 3: return PairCfg<3, 1, double>::kThreads;
        case 5: return PairCfg<3, 2, double>::kThreads;
        case 7: return PairCfg<3, 3, double>::kThreads;
        case 9: return PairCfg<3, 4, double>::kThreads;
        case 11: return PairCfg<3, 5, double>::kThreads;
        case 13: return PairCfg<3, 6, double>::kThreads;
        default: return -1;
    }
}

cudaError_t launch_pairs_d3(const PairParams& p, int fp64, int L, int grid, int smem, cudaStream_t s)
{
    switch (L * 2 + (fp64 ? 1 : 0)) {
        case 2: return launch_pairs_t<3, 1, float>(p, grid, smem, s);
        case 4: return launch_pairs_t<3, 2, float>(p, grid, smem, s);
        case 6: return launch_pairs_t<3, 3, float>(p, grid, smem, s);
        case 8: return launch_pairs_t<3, 4, float>(p, grid, smem, s);
        case 10: return launch_pairs_t<3, 5, float>(p, grid, smem, s);
        case 12: return launch_pairs_t<3, 6, float>(p, grid, smem, s);
        case 16: return launch_pairs_t<3, 8, float>(p, grid, smem, s);
        case 20: return launch_pairs_t<3, 10, float>(p, grid, smem, s);
        case 3: return launch_pairs_t<3, 1, double>(p, grid, smem, s);
        case 5: return launch_pairs_t<3, 2, double>(p, grid, smem, s);
        case 7: return launch_pairs_t<3, 3, double>(p, grid, smem, s);
        case 9: return launch_pairs_t<3, 4, double>(p, grid, smem, s);
        case 11: return launch_pairs_t<3, 5, double>(p, grid, smem, s);
        case 13: return launch_pairs_t<3, 6, double>(p, grid, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npcf
