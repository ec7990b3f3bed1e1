// npcf_couple_d3n5.cu -- the coupling kernel of the D=3 isotropic 5PCF
// (eq. D=3-NPCF with the intermediate label l12):
//     zeta^{b1 b2 b3 b4}_{l1 l2 l12 l3 l4} += w_j sum_{m1 m2 m3 m4} C(m1, m2, m3, m4)
//                                             a^{b1}_{l1 m1} a^{b2}_{l2 m2} a^{b3}_{l3 m3} a^{b4}_{l4 m4}
// with C the chain <l1 m1 l2 m2|l12 m12><l12 m12 l3 m3|l4 M><l4 M l4 m4|0 0> of
// eq. Coupling-C (the CGs of eq. CG-examples), tabulated on the host per label
// set as terms (m1, m2, m3, m4, C) sorted by m4.
//
// A thread owns one item: a bin triple b1 < b2 < b3 and one label set.  The
// items are ordered label-major, so the threads of a warp share the label set
// and walk the same term list.  For every primary of a group held in shared
// memory it forms, for each m4, Q(m4) = sum over that m4's terms of
// C u_{m1}(b1) u_{m2}(b2) u_{m3}(b3), and adds w Q(m4) a^{b4}_{l4 m4} into a
// register accumulator per b4 > b3; once per group the accumulators go into
// the CTA's FP64 partial row.
#include <cuda_runtime.h>

#include <algorithm>

#include "npcf_device.cuh"
#include "npcf_internal.h"

namespace npcf {

namespace {

template <typename T>
struct Cx5 {
    T r, i;
};

template <typename T, int NB>
__global__ void __launch_bounds__(256) k_couple_d3n5(const CoupleParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nb = p.nbins, L = p.lmax, S = (p.lmax + 1) * (p.lmax + 1), G = p.group;
    Cx5<T>* A = reinterpret_cast<Cx5<T>*>(smem);                  // [G][nb][S], all signed m
    T* W = reinterpret_cast<T*>(A + (size_t)G * nb * S);           // [G]
    const int cat = blockIdx.z;
    const int nprim = p.cat_count ? p.cat_count[cat] : *p.nprim;
    const size_t first = p.cat_first ? (size_t)p.cat_first[cat] : 0;
    const int stride = nb * p.nq;
    const T* aglob = static_cast<const T*>(p.a) + first * stride;
    const T* wglob = static_cast<const T*>(p.wprim) + first;
    double* prow = p.partial + ((size_t)cat * gridDim.x + blockIdx.x) * 2 * p.ncoeff;
    const int nitems = p.ntriple * p.nlam;
    const int ngroup = (nprim + G - 1) / G;
    (void)L;
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
            A[i] = Cx5<T>{re, im};
        }
        for (int g = threadIdx.x; g < G; g += blockDim.x) W[g] = g < gn ? wglob[g0 + g] : T(0);
        __syncthreads();
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int il = it / p.ntriple, t = it - (it / p.ntriple) * p.ntriple;
            const int4 tr = p.triples[t];  // b1, b2, b3, first key of the triple
            const int4 lm = p.lam5[il];    // first term, end term, l4, -
            const int nk = nb - tr.z - 1;
            T ar[NB], ai[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) ar[k] = ai[k] = T(0);
            for (int g = 0; g < gn; ++g) {
                const Cx5<T>* u1 = A + ((size_t)g * nb + tr.x) * S;
                const Cx5<T>* u2 = A + ((size_t)g * nb + tr.y) * S;
                const Cx5<T>* u3 = A + ((size_t)g * nb + tr.z) * S;
                const Cx5<T>* u4 = A + ((size_t)g * nb + tr.z + 1) * S;
                const T w = W[g];
                int e = lm.x;
                while (e < lm.y) {
                    const int m4 = (signed char)((p.terms5[e] >> 24) & 0xff);
                    T qr = T(0), qi = T(0);
                    // the terms of this m4 (sorted by m4)
                    for (; e < lm.y; ++e) {
                        const int pk = p.terms5[e];
                        if ((signed char)((pk >> 24) & 0xff) != m4) break;
                        const Cx5<T> x = u1[pk & 0xff], y = u2[(pk >> 8) & 0xff], z = u3[(pk >> 16) & 0xff];
                        T c;
                        if constexpr (sizeof(T) == 4) c = p.coef5f[e];
                        else c = p.coef5[e];
                        const T xyr = x.r * y.r - x.i * y.i, xyi = x.r * y.i + x.i * y.r;
                        qr = fma(c, xyr * z.r - xyi * z.i, qr);
                        qi = fma(c, xyr * z.i + xyi * z.r, qi);
                    }
                    qr *= w;
                    qi *= w;
                    const int s4 = lm.z * lm.z + lm.z + m4;  // state (l4, m4)
#pragma unroll
                    for (int k = 0; k < NB; ++k) {
                        if (k < nk) {
                            const Cx5<T> v = u4[(size_t)k * S + s4];
                            ar[k] = fma(qr, v.r, fma(-qi, v.i, ar[k]));
                            ai[k] = fma(qr, v.i, fma(qi, v.r, ai[k]));
                        }
                    }
                }
            }
            const int key0 = tr.w + il;
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

template <typename T, int NB>
cudaError_t launch_t5(const CoupleParams& p, int grid, int smem, cudaStream_t s)
{
    auto kern = k_couple_d3n5<T, NB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(grid, 1, p.ncat > 1 ? p.ncat : 1), 256, smem, s>>>(p);
    ++launch_counter();
    return cudaGetLastError();
}

}  // namespace

// primaries per shared-memory group (at most 32, within ~160 KB)
int d3n5_group(int nbins, int lmax, int fp64)
{
    const int per = nbins * (lmax + 1) * (lmax + 1) * 2 * (fp64 ? 8 : 4) + 8;
    return std::max(1, std::min(32, (160 * 1024) / per));
}

int couple_d3n5_smem(const CoupleParams& p, int fp64)
{
    const int tb = fp64 ? 8 : 4;
    return p.group * p.nbins * (p.lmax + 1) * (p.lmax + 1) * 2 * tb + p.group * tb;
}

cudaError_t launch_couple_d3n5(const CoupleParams& p, int fp64, int grid, int smem, cudaStream_t s)
{
    const int nbmax = p.nbins - 3;  // b4 values per bin triple
    if (fp64) {
        if (nbmax <= 8) return launch_t5<double, 8>(p, grid, smem, s);
        if (nbmax <= 16) return launch_t5<double, 16>(p, grid, smem, s);
        return launch_t5<double, 32>(p, grid, smem, s);
    }
    if (nbmax <= 8) return launch_t5<float, 8>(p, grid, smem, s);
    if (nbmax <= 16) return launch_t5<float, 16>(p, grid, smem, s);
    return launch_t5<float, 32>(p, grid, smem, s);
}

}  // namespace npcf
