// npcf_couple_d3n4.cu -- the coupling kernel of the D=3 isotropic 4PCF:
//     zeta^{b1 b2 b3}_{l1 l2 l3} += w_j sum_{m1 m2} (-1)^{l1+l2+l3} (l1 l2 l3; m1 m2 m3)
//                                    a^{b1}_{l1 m1} a^{b2}_{l2 m2} a^{b3}_{l3 m3},  m3 = -m1-m2
// (eq. NPCF-estimator-discrete with the coupling of eq. Coupling-C; the two CGs
// of eq. CG-examples, the second coupling to zero, collapse to the signed 3j).
//
// Layout of the work: a CTA holds 16 primaries' a^b (all signed m) in shared
// memory and walks the (l1, l2) label pairs with a fully unrolled body.  A lane
// owns (bin pair b1 < b2, primary); a warp task is two bin pairs x 16 primaries.
// The lane forms
//     P(l3, m3) = sum_{m1} c u_{m1} v_{-m1-m3},  m3 >= 0,
// (the m3 < 0 half is (-1)^{l1+l2+l3} times the conjugate), contracts P with
// a^{b3}_{l3 m3} for every b3 > b2, and the 16 primaries' terms of one output
// are summed with four shuffles before one lane adds them to the CTA's FP32
// shared accumulator.  All warps run one label body at a time, with a barrier
// after each (at lmax 5 this ran 1.7x faster than letting the warps drift
// apart across the 36 unrolled bodies); within a body, tasks are
// ordered by b2 (long b3 loops first) and dealt to the warps in snake order
// (w, 2W - 1 - w, 2W + w, ...), so every warp gets long and short tasks alike
// before the barrier.  Every 128 primaries the accumulators go into the CTA's
// FP64 row of the partial buffer.
#include <cuda_runtime.h>

#include "npcf_device.cuh"
#include "npcf_internal.h"

namespace npcf {

namespace {

constexpr int kGP = 16;  // primaries held at once (lanes per bin pair)

template <typename T>
struct Cx {
    T r, i;
};

// complex stride of one primary's a^b in shared memory: padded so that the 8
// primaries' copies start on different banks
__host__ __device__ inline int d3n4_astride(int nbins, int lmax)
{
    const int s = nbins * (lmax + 1) * (lmax + 1);
    return s + ((1 - s) % 16 + 16) % 16;
}

template <int L1, int L2, int LMAX, typename T>
__device__ __forceinline__ void couple_item(const Cx<T>* Ap, int b1, int b2, int b3min, int nbins, T w, bool valid,
                                            int prim, T* acc, int key0)
{
    constexpr int S = (LMAX + 1) * (LMAX + 1);
    constexpr int NLAM = cx::num_lambda_d3n4(LMAX);
    constexpr int L3lo = L1 > L2 ? L1 - L2 : L2 - L1;
    constexpr int L3hi = (L1 + L2 < LMAX) ? L1 + L2 : LMAX;
    if constexpr (L3lo <= L3hi) {
        const Cx<T>* u = Ap + b1 * S + L1 * L1 + L1;
        const Cx<T>* v = Ap + b2 * S + L2 * L2 + L2;
        Cx<T> vv[2 * L2 + 1];
        static_for<0, 2 * L2 + 1>([&](auto I) { vv[decltype(I)::value] = v[decltype(I)::value - L2]; });
        T Pr[L3hi + 1][L3hi + 1];
        T Pi[L3hi + 1][L3hi + 1];
        static_for<0, L3hi + 1>([&](auto I) {
            static_for<0, L3hi + 1>([&](auto J) {
                Pr[decltype(I)::value][decltype(J)::value] = T(0);
                Pi[decltype(I)::value][decltype(J)::value] = T(0);
            });
        });
        static_for<0, 2 * L1 + 1>([&](auto I1) {
            constexpr int m1 = decltype(I1)::value - L1;
            const Cx<T> uu = u[m1];
            static_for<0, 2 * L2 + 1>([&](auto I2) {
                constexpr int m2 = decltype(I2)::value - L2;
                constexpr int m3 = -(m1 + m2);
                if constexpr (m3 >= 0 && m3 <= L3hi) {
                    const Cx<T> v2 = vv[decltype(I2)::value];
                    const T tr = fma(uu.r, v2.r, -(uu.i * v2.i));
                    const T ti = fma(uu.r, v2.i, uu.i * v2.r);
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
        for (int b3 = b3min; b3 < nbins; ++b3) {  // warp-uniform bounds
            const bool on = valid && b3 > b2;
            const Cx<T>* x = Ap + b3 * S;
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
                s = on ? w * s : T(0);
                s += __shfl_xor_sync(0xffffffffu, s, 1);
                s += __shfl_xor_sync(0xffffffffu, s, 2);
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                s += __shfl_xor_sync(0xffffffffu, s, 8);
                if (on && prim == 0) acc[key0 + (b3 - b2 - 1) * NLAM + lam] += s;
            });
        }
    }
}

template <int LMAX, typename T>
__global__ void __launch_bounds__(320, 2) k_couple_d3n4(const CoupleParams p)
{
    constexpr int S = (LMAX + 1) * (LMAX + 1);
    constexpr int NC = (LMAX + 1) * (LMAX + 1);
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 blk = p.kblocks[blockIdx.y];
    const int nbins = p.nbins;
    const int astride = d3n4_astride(nbins, LMAX);
    Cx<T>* A = reinterpret_cast<Cx<T>*>(smem);  // [kGP][astride]
    T* wsm = reinterpret_cast<T*>(smem + sizeof(Cx<T>) * kGP * astride);
    T* acc = reinterpret_cast<T*>(smem + ((sizeof(Cx<T>) * kGP * astride + sizeof(T) * kGP + 15) / 16) * 16);
    const int nacc = blk.w - blk.z;
    for (int k = threadIdx.x; k < nacc; k += blockDim.x) acc[k] = T(0);

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int prim = lane & (kGP - 1);
    const int npair = blk.y - blk.x;
    const int ntask = (npair + 1) / 2;

    // catalogue blockIdx.z: its primaries' rows of the a-array and its own partial rows
    const int cat = blockIdx.z;
    const int nprim = p.cat_count ? p.cat_count[cat] : *p.nprim;
    const size_t first = p.cat_first ? (size_t)p.cat_first[cat] : 0;
    const int nchunk = (nprim + p.chunk - 1) / p.chunk;
    double* prow = p.partial + ((size_t)cat * gridDim.x + blockIdx.x) * 2 * p.ncoeff;
    const int gstride = nbins * p.nq;
    const T* aglob = static_cast<const T*>(p.a) + first * gstride;
    const T* wglob = static_cast<const T*>(p.wprim) + first;

    for (int ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const int p0 = ch * p.chunk;
        const int p1 = min(nprim, p0 + p.chunk);
        for (int g0 = p0; g0 < p1; g0 += kGP) {
            const int gn = min(kGP, p1 - g0);
            __syncthreads();
            // the group's a^b, all signed m: a_{l,-m} = (-1)^m conj(a_{l m})
            for (int i = threadIdx.x; i < kGP * nbins * S; i += blockDim.x) {
                const int g = i / (nbins * S);
                const int r = i - g * (nbins * S);
                const int b = r / S, s = r - (r / S) * S;
                T re = T(0), im = T(0);
                if (g < gn) {
                    int l = 0;
                    while ((l + 1) * (l + 1) <= s) ++l;
                    const int m = s - l * l - l;
                    const int am = m < 0 ? -m : m;
                    const T* ap = aglob + (size_t)(g0 + g) * gstride + b * p.nq + q_index_d3(l, am);
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
                A[g * astride + r] = Cx<T>{re, im};
            }
            if (threadIdx.x < kGP) wsm[threadIdx.x] = threadIdx.x < gn ? wglob[g0 + threadIdx.x] : T(0);
            __syncthreads();
            const T w = wsm[prim];
            const Cx<T>* Ap = A + prim * astride;
            // label bodies in turn, every warp on the same body between two barriers (one body's
            // instructions in the instruction cache at a time); within a body each warp takes its
            // tasks in snake order
            static_for<0, NC>([&](auto K) {
                constexpr int k = decltype(K)::value;
                for (int r = 0; r * nwarps < ntask; ++r) {
                    const int t = (r & 1) ? (r + 1) * nwarps - 1 - warp : r * nwarps + warp;
                    if (t >= ntask) continue;
                    const int pi = t * 2 + (lane >> 4);
                    const bool valid = pi < npair;
                    const int pr = p.task_pairs[blk.x + (valid ? pi : 0)];
                    const int2 bb = p.pairs[pr];
                    const int key0 = p.pair_key[pr] - blk.z;
                    const int b3min = __reduce_min_sync(0xffffffffu, valid ? bb.y : nbins) + 1;
                    couple_item<k / (LMAX + 1), k % (LMAX + 1), LMAX, T>(Ap, bb.x, bb.y, b3min, nbins, w, valid, prim,
                                                                     acc, key0);
                }
                __syncthreads();
            });
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nacc; k += blockDim.x) {
            const int key = blk.z + k;
            prow[2 * key + p.lam_odd[key % p.nlam]] += (double)acc[k];
            acc[k] = T(0);
        }
    }
}

template <int LMAX, typename T>
cudaError_t launch_t(const CoupleParams& p, int grid, int threads, int smem, cudaStream_t s)
{
    auto kern = k_couple_d3n4<LMAX, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // prefer the largest shared-memory carveout: two CTAs per SM fit (registers and shared
    // memory) and hide each other's per-group barriers; the default leaves room for one
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    kern<<<dim3(grid, p.nkb, p.ncat > 1 ? p.ncat : 1), threads, smem, s>>>(p); ++launch_counter();
    return cudaGetLastError();
}

}  // namespace

int couple_d3n4_smem(const CoupleParams& p, int fp64)
{
    const int tb = fp64 ? 8 : 4;
    const int a = 2 * tb * kGP * d3n4_astride(p.nbins, p.lmax) + tb * kGP;
    return (a + 15) / 16 * 16 + p.max_block_keys * tb;
}

int couple_d3n4_threads(int max_block_pairs)
{
    const int ntask = (max_block_pairs + 1) / 2;
    // about two tasks per warp (snake order balances a long and a short one), at most 10 warps:
    // with __launch_bounds__(320, 2) two CTAs share an SM
    const int nw = (ntask + 1) / 2;
    return 32 * (nw < 10 ? (nw < 1 ? 1 : nw) : 10);
}

cudaError_t launch_couple_d3n4(const CoupleParams& p, int fp64, int grid, int threads, int smem, cudaStream_t s)
{
    if (fp64) {
        switch (p.lmax) {
            case 1: return launch_t<1, double>(p, grid, threads, smem, s);
            case 2: return launch_t<2, double>(p, grid, threads, smem, s);
            case 3: return launch_t<3, double>(p, grid, threads, smem, s);
            case 4: return launch_t<4, double>(p, grid, threads, smem, s);
            case 5: return launch_t<5, double>(p, grid, threads, smem, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (p.lmax) {
        case 1: return launch_t<1, float>(p, grid, threads, smem, s);
        case 2: return launch_t<2, float>(p, grid, threads, smem, s);
        case 3: return launch_t<3, float>(p, grid, threads, smem, s);
        case 4: return launch_t<4, float>(p, grid, threads, smem, s);
        case 5: return launch_t<5, float>(p, grid, threads, smem, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace npcf
