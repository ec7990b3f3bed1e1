// npcf_couple_los.cu -- the coupling of the basis about a fixed line of sight (the x_3 axis),
// D = 3 (Sec. "Large-Scale Structure": the redshift-space 3PCF and its extension to N = 4).
// The basis keeps the total angular momentum's projection on the line of sight at zero but lets
// the total L be any value the labels allow (L = 0 is the isotropic basis):
//     N=3: zeta^{b1 b2}_{l1 l2 L} += w_j sum_m <l1 m l2 -m|L 0> a^{b1}_{l1 m} a^{b2}_{l2,-m}
//     N=4: zeta^{b1 b2 b3}_{l1 l2 l12 l3 L} += w_j sum_{m1 m2} <l1 m1 l2 m2|l12 m12><l12 m12 l3 -m12|L 0>
//                                             a^{b1}_{l1 m1} a^{b2}_{l2 m2} a^{b3}_{l3,-m12}
// (the CG chain of eq. Coupling-C with the final state (L, 0)).  The terms of every label set
// (states and CG products) are tabulated on the host.
//
// A thread owns one item: a bin pair and one label set (label-major, so a warp's threads share
// the term list).  For every primary of a group held in shared memory (a^b for all signed m) it
// adds the label set's terms; for N = 4 the product of the first two a's is formed once per term
// and multiplied into a register accumulator for every b3 > b2.  Once per group the sums go into
// the CTA's FP64 partial row.
#include <cuda_runtime.h>

#include <algorithm>

#include "npcf_device.cuh"
#include "npcf_internal.h"

namespace npcf {

namespace {

template <typename T>
struct CxL {
    T r, i;
};

constexpr int kLosThreads = 256;

template <typename T, int N, int NB>
__global__ void __launch_bounds__(kLosThreads) k_couple_los(const CoupleParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nb = p.nbins, S = (p.lmax + 1) * (p.lmax + 1), G = p.group;
    CxL<T>* A = reinterpret_cast<CxL<T>*>(smem);           // [G][nb][S], all signed m
    T* W = reinterpret_cast<T*>(A + (size_t)G * nb * S);   // [G]
    const int cat = blockIdx.z;
    const int nprim = p.cat_count ? p.cat_count[cat] : *p.nprim;
    const size_t first = p.cat_first ? (size_t)p.cat_first[cat] : 0;
    const int stride = nb * p.nq;
    const T* aglob = static_cast<const T*>(p.a) + first * stride;
    const T* wglob = static_cast<const T*>(p.wprim) + first;
    const T* coef = static_cast<const T*>(p.los_coef);
    double* prow = p.partial + ((size_t)cat * gridDim.x + blockIdx.x) * 2 * p.ncoeff;
    const int npair = (int)(p.kblocks[0].y - p.kblocks[0].x);
    const int nitems = npair * p.nlam;
    const int ngroup = (nprim + G - 1) / G;
    for (int gi = blockIdx.x; gi < ngroup; gi += gridDim.x) {
        const int g0 = gi * G, gn = min(G, nprim - g0);
        __syncthreads();
        // the group's a^b for all signed m: a_{l,-m} = (-1)^m conj(a_{l m})
        for (int i = threadIdx.x; i < G * nb * S; i += blockDim.x) {
            const int g = i / (nb * S), r = i - g * (nb * S), b = r / S, s = r - b * S;
            T re = T(0), im = T(0);
            if (g < gn) {
                int l = 0;
                while ((l + 1) * (l + 1) <= s) ++l;
                const int m = s - l * l - l, am = m < 0 ? -m : m;
                const T* ap = aglob + (size_t)(g0 + g) * stride + b * p.nq + q_index_d3(l, am);
                re = ap[0];
                im = am > 0 ? ap[1] : T(0);
                if (m < 0) {
                    im = -im;
                    if (am & 1) {
                        re = -re;
                        im = -im;
                    }
                }
            }
            A[i] = CxL<T>{re, im};
        }
        for (int g = threadIdx.x; g < G; g += blockDim.x) W[g] = g < gn ? wglob[g0 + g] : T(0);
        __syncthreads();
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int il = it / npair, pr = it - il * npair;
            const int2 bb = p.pairs[p.kblocks[0].x + pr];
            const int2 tl = p.los_lam[il];  // term begin, end
            const int nk = N == 4 ? nb - bb.y - 1 : 1;
            T ar[NB], ai[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) ar[k] = ai[k] = T(0);
            for (int g = 0; g < gn; ++g) {
                const CxL<T>* u1 = A + ((size_t)g * nb + bb.x) * S;
                const CxL<T>* u2 = A + ((size_t)g * nb + bb.y) * S;
                const T w = W[g];
                for (int t = tl.x; t < tl.y; ++t) {
                    const int st = p.los_terms[t];
                    const CxL<T> x = u1[st & 0xff], y = u2[(st >> 8) & 0xff];
                    const T c = w * coef[t];
                    const T pr_ = c * (x.r * y.r - x.i * y.i), pi_ = c * (x.r * y.i + x.i * y.r);
                    if constexpr (N == 3) {
                        ar[0] += pr_;
                        ai[0] += pi_;
                    } else {
                        const int s3 = (st >> 16) & 0xff;
#pragma unroll
                        for (int k = 0; k < NB; ++k) {
                            if (k < nk) {
                                const CxL<T> z = A[((size_t)g * nb + bb.y + 1 + k) * S + s3];
                                ar[k] = fma(pr_, z.r, fma(-pi_, z.i, ar[k]));
                                ai[k] = fma(pr_, z.i, fma(pi_, z.r, ai[k]));
                            }
                        }
                    }
                }
            }
            const int key0 = p.pair_key[p.kblocks[0].x + pr] + il;
#pragma unroll
            for (int k = 0; k < NB; ++k) {
                if (k < nk) {
                    double* d = prow + 2 * (key0 + k * p.nlam);
                    d[0] += (double)ar[k];
                    d[1] += (double)ai[k];
                }
            }
        }
    }
}

template <typename T, int N, int NB>
cudaError_t launch_los_t(const CoupleParams& p, int grid, int smem, cudaStream_t s)
{
    auto kern = k_couple_los<T, N, NB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(grid, 1, p.ncat > 1 ? p.ncat : 1), kLosThreads, smem, s>>>(p);
    ++launch_counter();
    return cudaGetLastError();
}

}  // namespace

// primaries per shared-memory group of the line-of-sight coupling (at most 32, within ~160 KB)
int los_group(int nbins, int lmax, int fp64)
{
    const int per = nbins * (lmax + 1) * (lmax + 1) * 2 * (fp64 ? 8 : 4) + 8;
    return std::max(1, std::min(32, (160 * 1024) / per));
}

int couple_los_smem(const CoupleParams& p, int fp64)
{
    const int tb = fp64 ? 8 : 4;
    return p.group * p.nbins * (p.lmax + 1) * (p.lmax + 1) * 2 * tb + p.group * tb;
}

cudaError_t launch_couple_los(const CoupleParams& p, int fp64, int grid, int smem, cudaStream_t s)
{
    if (p.N == 3) return fp64 ? launch_los_t<double, 3, 1>(p, grid, smem, s) : launch_los_t<float, 3, 1>(p, grid, smem, s);
    const int nbmax = p.nbins - 2;  // b3 values per bin pair
    if (fp64) {
        if (nbmax <= 8) return launch_los_t<double, 4, 8>(p, grid, smem, s);
        if (nbmax <= 16) return launch_los_t<double, 4, 16>(p, grid, smem, s);
        return launch_los_t<double, 4, 32>(p, grid, smem, s);
    }
    if (nbmax <= 8) return launch_los_t<float, 4, 8>(p, grid, smem, s);
    if (nbmax <= 16) return launch_los_t<float, 4, 16>(p, grid, smem, s);
    return launch_los_t<float, 4, 32>(p, grid, smem, s);
}

}  // namespace npcf
