// npcf_pairs_sph.cu -- instantiations of the pair kernel for points on the unit 2-sphere
// (Sec. "Cosmic Microwave Background"): D = 2 harmonics of the azimuth about each primary,
// neighbours found in 3-D.
#include "npcf_pairs.cuh"

namespace npcf {

// lmax values compiled for the sphere; a plan runs the smallest one >= its lmax
static const int kLsf[] = {4, 8, 12};
static const int kLsd[] = {4, 8};

int pair_compiled_lmax_sph(int fp64, int lmax)
{
    const int* L = fp64 ? kLsd : kLsf;
    const int n = fp64 ? (int)(sizeof(kLsd) / sizeof(int)) : (int)(sizeof(kLsf) / sizeof(int));
    for (int i = 0; i < n; ++i)
        if (L[i] >= lmax) return L[i];
    return -1;
}

cudaError_t launch_pairs_sph(const PairParams& p, int fp64, int L, int grid, int smem, cudaStream_t s)
{
    switch (L * 2 + (fp64 ? 1 : 0)) {
        case 8: return launch_pairs_t<2, 4, float, true>(p, grid, smem, s);
        case 16: return launch_pairs_t<2, 8, float, true>(p, grid, smem, s);
        case 24: return launch_pairs_t<2, 12, float, true>(p, grid, smem, s);
        case 9: return launch_pairs_t<2, 4, double, true>(p, grid, smem, s);
        case 17: return launch_pairs_t<2, 8, double, true>(p, grid, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npcf
