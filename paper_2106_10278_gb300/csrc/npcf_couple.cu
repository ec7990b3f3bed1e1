// npcf_couple.cu -- the coupling kernel: the outer sum of
// eq. NPCF-estimator-discrete,
//     zeta^{0,b}_Lambda = (1/V_D) sum_j w_j sum_[l] C^{Lambda;0} prod_i a^{b_i}_{l^i}(y_j),
// over the a-array written by the pair kernel.
//
// Grid: blockIdx.y picks a block of output keys (its accumulators live in
// shared memory), blockIdx.x a persistent row: CTA x handles primary chunks
// x, x + gridDim.x, ... in a fixed order.  Each primary's a^b is loaded (and,
// for N=4, expanded to all signed m) into shared memory; the per-primary
// coupling runs in registers in T and is added into the shared accumulators;
// after every chunk the accumulators are added into the CTA's FP64 row of
// the partial buffer, which a fixed-order reduction sums (launch_reduce).
//
// Couplings (all real; derived from eq. Coupling-C with eq. CG-examples):
//   N=3, D=2: zeta_l = w a_l(b1) a_{-l}(b2), a_{-l} = conj(a_l)           (complex)
//   N=3, D>=3: zeta_l = w (-1)^l/sqrt(dim_l) sum_[l] a(b1) conj(a(b2))     (real)
//   N=4, D=2: zeta_{l1 l2 l3} = w a_l1(b1) a_l2(b2) a_l3(b3), l1+l2+l3=0   (complex)
//   N=4, D=3: zeta = w sum_{m1 m2} (-1)^{l1+l2+l3} (l1 l2 l3; m1 m2 m3) a a a
//             real for even l1+l2+l3, imaginary for odd (eq. basis-parity-conj);
//             the m3 < 0 half equals (-1)^{l1+l2+l3} times the conjugate of the
//             m3 > 0 half, so only m3 >= 0 is evaluated (with weight 2 for m3 > 0).
#include <cuda_runtime.h>

#include "npcf_device.cuh"
#include "npcf_internal.h"

namespace npcf {

namespace {

constexpr int kCoupleThreads = 256;

template <typename T>
struct Cx {
    T r, i;
};

enum { MODE_N3 = 0, MODE_D2N4 = 1, MODE_D3N4 = 2 };

// ------------------------------------------------------------------ N = 3
template <int D, typename T, typename AccT>
__device__ __forceinline__ void body_n3(const CoupleParams& p, const T* a, T w, AccT* acc, int4 blk)
{
    const int L1 = p.lmax + 1;
    const int nq = p.nq;
    const int nitems = (blk.y - blk.x) * L1;
    const T* pref = static_cast<const T*>(p.pref);
    for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
        const int pr = blk.x + i / L1;
        const int l = i - (i / L1) * L1;
        const int2 bb = p.pairs[pr];
        const T* u = a + bb.x * nq;
        const T* v = a + bb.y * nq;
        const int key = p.pair_key[pr] + l - blk.z;
        if constexpr (D == 2) {
            T re, im;
            if (l == 0) {
                re = u[0] * v[0];
                im = T(0);
            } else {
                const int q = 2 * l - 1;
                re = fma(u[q], v[q], u[q + 1] * v[q + 1]);
                im = fma(u[q + 1], v[q], -(u[q] * v[q + 1]));
            }
            acc[2 * key] += w * re;
            acc[2 * key + 1] += w * im;
        } else if constexpr (D == 3) {
            const int b0 = l * l;
            T s0 = u[b0] * v[b0];
            T s1 = T(0);
            for (int m = 1; m <= l; ++m) {
                const int q = b0 + 2 * m - 1;
                s1 = fma(u[q], v[q], fma(u[q + 1], v[q + 1], s1));
            }
            acc[key] += w * pref[l] * fma(T(2), s1, s0);
        } else {
            T s0 = T(0), s1 = T(0);
            for (int l2 = 0; l2 <= l; ++l2) {
                const int b0 = q_index_d4(l, l2, 0);
                s0 = fma(u[b0], v[b0], s0);
                for (int l1 = 1; l1 <= l2; ++l1) {
                    const int q = b0 + 2 * l1 - 1;
                    s1 = fma(u[q], v[q], fma(u[q + 1], v[q + 1], s1));
                }
            }
            acc[key] += w * pref[l] * fma(T(2), s1, s0);
        }
    }
}

// --------------------------------------------------------------- D=2, N=4
template <typename T, typename AccT>
__device__ __forceinline__ void body_d2n4(const CoupleParams& p, const Cx<T>* A, T w, AccT* acc, int4 blk)
{
    const int nlam = p.nlam;
    const int S = 2 * p.lmax + 1;  // signed l in [-lmax, lmax]
    const int nitems = (blk.y - blk.x) * nlam;
    for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
        const int pr = blk.x + i / nlam;
        const int lam = i - (i / nlam) * nlam;
        const int2 bb = p.pairs[pr];
        const int2 ll = p.lam2[lam];
        const int l3 = -(ll.x + ll.y);
        const Cx<T> u = A[bb.x * S + ll.x + p.lmax];
        const Cx<T> v = A[bb.y * S + ll.y + p.lmax];
        const T tr = fma(u.r, v.r, -(u.i * v.i)), ti = fma(u.r, v.i, u.i * v.r);
        int key = p.pair_key[pr] + lam - blk.z;
        for (int b3 = bb.y + 1; b3 < p.nbins; ++b3, key += nlam) {
            const Cx<T> x = A[b3 * S + l3 + p.lmax];
            acc[2 * key] += w * fma(tr, x.r, -(ti * x.i));
            acc[2 * key + 1] += w * fma(tr, x.i, ti * x.r);
        }
    }
}

// --------------------------------------------------------------- D=3, N=4
template <int L1, int L2, int LMAX, typename T, typename AccT>
__device__ __forceinline__ void item_d3n4(const Cx<T>* A, int b1, int b2, int nbins, T w, AccT* acc, int key0)
{
    constexpr int S = (LMAX + 1) * (LMAX + 1);
    constexpr int NLAM = cx::num_lambda_d3n4(LMAX);
    constexpr int L3lo = L1 > L2 ? L1 - L2 : L2 - L1;
    constexpr int L3hi = (L1 + L2 < LMAX) ? L1 + L2 : LMAX;
    if constexpr (L3lo <= L3hi) {
        const Cx<T>* u = A + b1 * S + L1 * L1 + L1;  // u[m], m in [-L1, L1]
        const Cx<T>* v = A + b2 * S + L2 * L2 + L2;
        T Pr[L3hi + 1][L3hi + 1];
        T Pi[L3hi + 1][L3hi + 1];
        static_for<0, L3hi + 1>([&](auto I) {
            static_for<0, L3hi + 1>([&](auto J) {
                Pr[decltype(I)::value][decltype(J)::value] = T(0);
                Pi[decltype(I)::value][decltype(J)::value] = T(0);
            });
        });
        // P(l3, m3) = sum_{m1 + m2 = -m3} c u_{m1} v_{m2}, m3 >= 0
        static_for<0, 2 * L1 + 1>([&](auto I1) {
            constexpr int m1 = decltype(I1)::value - L1;
            const Cx<T> uu = u[m1];
            static_for<0, 2 * L2 + 1>([&](auto I2) {
                constexpr int m2 = decltype(I2)::value - L2;
                constexpr int m3 = -(m1 + m2);
                if constexpr (m3 >= 0 && m3 <= L3hi) {
                    const Cx<T> vv = v[m2];
                    const T tr = fma(uu.r, vv.r, -(uu.i * vv.i));
                    const T ti = fma(uu.r, vv.i, uu.i * vv.r);
                    static_for<(L3lo > m3 ? L3lo : m3), L3hi + 1>([&](auto I3) {
                        constexpr int l3 = decltype(I3)::value;
                        constexpr double cd = cx::coupling_d3n4(L1, L2, l3, m1, m2, m3) * (m3 > 0 ? 2.0 : 1.0);
                        if constexpr (cd != 0.0) {
                            Pr[l3][m3] = fma(T(cd), tr, Pr[l3][m3]);
                            Pi[l3][m3] = fma(T(cd), ti, Pi[l3][m3]);
                        }
                    });
                }
            });
        });
        // contract with the third shell, b3 > b2
        for (int b3 = b2 + 1; b3 < nbins; ++b3) {
            const Cx<T>* x = A + b3 * S;
            static_for<L3lo, L3hi + 1>([&](auto I3) {
                constexpr int l3 = decltype(I3)::value;
                constexpr bool odd = ((L1 + L2 + l3) & 1) != 0;
                constexpr int lam = cx::lambda_index_d3n4(LMAX, L1, L2, l3);
                T s = T(0);
                static_for<0, l3 + 1>([&](auto M3) {
                    constexpr int m3 = decltype(M3)::value;
                    const Cx<T> xx = x[l3 * l3 + l3 + m3];
                    if constexpr (!odd) s = fma(Pr[l3][m3], xx.r, fma(-Pi[l3][m3], xx.i, s));
                    else s = fma(Pr[l3][m3], xx.i, fma(Pi[l3][m3], xx.r, s));
                });
                acc[key0 + (b3 - b2 - 1) * NLAM + lam] += w * s;
            });
        }
    }
}

template <int LMAX, typename T, typename AccT>
__device__ __forceinline__ void body_d3n4(const CoupleParams& p, const Cx<T>* A, T w, AccT* acc, int4 blk)
{
    constexpr int NC = (LMAX + 1) * (LMAX + 1);
    const int npair = blk.y - blk.x;
    const int nchunks = (npair + 31) / 32;
    const int ntask = NC * nchunks;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int t = warp; t < ntask; t += nw) {
        const int combo = t / nchunks;
        const int pr = blk.x + (t - combo * nchunks) * 32 + lane;
        if (pr >= blk.y) continue;
        const int2 bb = p.pairs[pr];
        const int key0 = p.pair_key[pr] - blk.z;
        static_for<0, NC>([&](auto K) {
            constexpr int k = decltype(K)::value;
            if (combo == k) item_d3n4<k / (LMAX + 1), k % (LMAX + 1), LMAX, T, AccT>(A, bb.x, bb.y, p.nbins, w, acc, key0);
        });
    }
}

template <int MODE, int D, int LMAX, typename T>
__global__ void __launch_bounds__(kCoupleThreads) k_couple(const CoupleParams p)
{
    using AccT = T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 blk = p.kblocks[blockIdx.y];
    const int comps = (MODE == MODE_N3 && D != 2) || MODE == MODE_D3N4 ? 1 : 2;
    int a_elems;  // T elements of the per-primary copy
    if constexpr (MODE == MODE_D3N4) a_elems = p.nbins * (LMAX + 1) * (LMAX + 1) * 2;
    else if constexpr (MODE == MODE_D2N4) a_elems = p.nbins * (2 * p.lmax + 1) * 2;
    else a_elems = p.nbins * p.nq;
    T* A = reinterpret_cast<T*>(smem);
    AccT* acc = reinterpret_cast<AccT*>(smem + ((a_elems * (int)sizeof(T) + 15) / 16) * 16);
    const int nacc = (blk.w - blk.z) * comps;
    for (int k = threadIdx.x; k < nacc; k += blockDim.x) acc[k] = AccT(0);

    const int nprim = *p.nprim;
    const int nchunk = (nprim + p.chunk - 1) / p.chunk;
    double* prow = p.partial + (size_t)blockIdx.x * 2 * p.ncoeff;
    const T* aglob = static_cast<const T*>(p.a);
    const T* wglob = static_cast<const T*>(p.wprim);
    const int stride = p.nbins * p.nq;

    for (int ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const int p0 = ch * p.chunk;
        const int p1 = min(nprim, p0 + p.chunk);
        for (int pi = p0; pi < p1; ++pi) {
            __syncthreads();
            const T* ap = aglob + (size_t)pi * stride;
            if constexpr (MODE == MODE_D3N4) {
                constexpr int S = (LMAX + 1) * (LMAX + 1);
                for (int i = threadIdx.x; i < p.nbins * S; i += blockDim.x) {
                    const int b = i / S, s = i - (i / S) * S;
                    int l = 0;
                    while ((l + 1) * (l + 1) <= s) ++l;
                    const int m = s - l * l - l;
                    const int am = m < 0 ? -m : m;
                    const int q = q_index_d3(l, am);
                    T re = ap[b * p.nq + q];
                    T im = am > 0 ? ap[b * p.nq + q + 1] : T(0);
                    if (m < 0) {  // a_{l,-m} = (-1)^m conj(a_{l m})
                        im = -im;
                        if (am & 1) {
                            re = -re;
                            im = -im;
                        }
                    }
                    A[2 * i] = re;
                    A[2 * i + 1] = im;
                }
            } else if constexpr (MODE == MODE_D2N4) {
                const int S = 2 * p.lmax + 1;
                for (int i = threadIdx.x; i < p.nbins * S; i += blockDim.x) {
                    const int b = i / S, l = i - (i / S) * S - p.lmax;
                    const int al = l < 0 ? -l : l;
                    T re = ap[b * p.nq + q_index_d2(al)];
                    T im = al > 0 ? ap[b * p.nq + q_index_d2(al) + 1] : T(0);
                    if (l < 0) im = -im;  // a_{-l} = conj(a_l)
                    A[2 * i] = re;
                    A[2 * i + 1] = im;
                }
            } else {
                for (int i = threadIdx.x; i < stride; i += blockDim.x) A[i] = ap[i];
            }
            const T w = wglob[pi];
            __syncthreads();
            if constexpr (MODE == MODE_N3) body_n3<D, T, AccT>(p, A, w, acc, blk);
            else if constexpr (MODE == MODE_D2N4) body_d2n4<T, AccT>(p, reinterpret_cast<const Cx<T>*>(A), w, acc, blk);
            else body_d3n4<LMAX, T, AccT>(p, reinterpret_cast<const Cx<T>*>(A), w, acc, blk);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nacc; k += blockDim.x) {
            const int key = blk.z + k / comps;
            int col;
            if constexpr (MODE == MODE_D3N4) col = 2 * key + p.lam_odd[key % p.nlam];
            else col = comps == 1 ? 2 * key : 2 * key + (k % comps);
            prow[col] += (double)acc[k];
            acc[k] = AccT(0);
        }
    }
}

template <int MODE, int D, int LMAX, typename T>
cudaError_t launch_t(const CoupleParams& p, int grid, int smem, cudaStream_t s)
{
    auto kern = k_couple<MODE, D, LMAX, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(grid, p.nkb), kCoupleThreads, smem, s>>>(p); ++launch_counter();
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_d3n4(const CoupleParams& p, int grid, int smem, cudaStream_t s)
{
    switch (p.lmax) {
        case 1: return launch_t<MODE_D3N4, 3, 1, T>(p, grid, smem, s);
        case 2: return launch_t<MODE_D3N4, 3, 2, T>(p, grid, smem, s);
        case 3: return launch_t<MODE_D3N4, 3, 3, T>(p, grid, smem, s);
        case 4: return launch_t<MODE_D3N4, 3, 4, T>(p, grid, smem, s);
        case 5: return launch_t<MODE_D3N4, 3, 5, T>(p, grid, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int couple_max_lmax_d3n4() { return 5; }

int couple_smem(const CoupleParams& p, int fp64)
{
    const int tb = fp64 ? 8 : 4;
    int a_elems;
    int comps;
    if (p.N == 4 && p.D == 3) {
        a_elems = p.nbins * (p.lmax + 1) * (p.lmax + 1) * 2;
        comps = 1;
    } else if (p.N == 4) {
        a_elems = p.nbins * (2 * p.lmax + 1) * 2;
        comps = 2;
    } else {
        a_elems = p.nbins * p.nq;
        comps = p.D == 2 ? 2 : 1;
    }
    return (a_elems * tb + 15) / 16 * 16 + p.max_block_keys * comps * tb;
}

cudaError_t launch_couple(const CoupleParams& p, int fp64, int grid, int smem, cudaStream_t s)
{
    if (p.N == 3) {
        switch (p.D * 2 + (fp64 ? 1 : 0)) {
            case 4: return launch_t<MODE_N3, 2, 0, float>(p, grid, smem, s);
            case 5: return launch_t<MODE_N3, 2, 0, double>(p, grid, smem, s);
            case 6: return launch_t<MODE_N3, 3, 0, float>(p, grid, smem, s);
            case 7: return launch_t<MODE_N3, 3, 0, double>(p, grid, smem, s);
            case 8: return launch_t<MODE_N3, 4, 0, float>(p, grid, smem, s);
            case 9: return launch_t<MODE_N3, 4, 0, double>(p, grid, smem, s);
            default: return cudaErrorInvalidValue;
        }
    }
    if (p.D == 2) {
        return fp64 ? launch_t<MODE_D2N4, 2, 0, double>(p, grid, smem, s)
                    : launch_t<MODE_D2N4, 2, 0, float>(p, grid, smem, s);
    }
    return fp64 ? launch_d3n4<double>(p, grid, smem, s) : launch_d3n4<float>(p, grid, smem, s);
}

}  // namespace npcf
