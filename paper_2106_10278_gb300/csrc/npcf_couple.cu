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
//   N=4, D=3: in npcf_couple_d3n4.cu.
#include <cuda_runtime.h>

#include <algorithm>

#include "npcf_device.cuh"
#include "npcf_internal.h"

namespace npcf {

int couple_d3n4_smem(const CoupleParams& p, int fp64);
int couple_d3n4_threads(int max_block_pairs);
cudaError_t launch_couple_d3n4(const CoupleParams& p, int fp64, int grid, int threads, int smem, cudaStream_t s);

namespace {

constexpr int kCoupleThreads = 256;

template <typename T>
struct Cx {
    T r, i;
};

enum { MODE_N3 = 0, MODE_D2N4 = 1 };

// ------------------------------------------------------------------ N = 3
// `self` (NULL unless the remove_self option is on): the primary's sums of w_k^2 per bin; for
// keys with b1 = b2 the tuples with coinciding secondaries, w_k^2 c_l / v_b^2 per secondary
// (c_l the basis value at coinciding directions), are subtracted.
template <int D, typename T, typename AccT>
__device__ __forceinline__ void body_n3(const CoupleParams& p, const T* a, const T* self, T w, AccT* acc, int4 blk)
{
    const int L1 = p.lmax + 1;
    const int nq = p.nq;
    const int nitems = (blk.y - blk.x) * L1;
    const T* pref = static_cast<const T*>(p.pref);
    const T* selfc = static_cast<const T*>(p.selfc);
    for (int i = threadIdx.x; i < nitems; i += blockDim.x) {
        const int pr = blk.x + i / L1;
        const int l = i - (i / L1) * L1;
        const int2 bb = p.pairs[pr];
        const T* u = a + bb.x * nq;
        const T* v = a + bb.y * nq;
        const int key = p.pair_key[pr] + l - blk.z;
        const T dself = (self && bb.x == bb.y) ? selfc[bb.x * L1 + l] * self[bb.x] : T(0);
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
            acc[2 * key] += w * (re - dself);
            acc[2 * key + 1] += w * im;
        } else if constexpr (D == 3) {
            const int b0 = l * l;
            T s0 = u[b0] * v[b0];
            T s1 = T(0);
            for (int m = 1; m <= l; ++m) {
                const int q = b0 + 2 * m - 1;
                s1 = fma(u[q], v[q], fma(u[q + 1], v[q + 1], s1));
            }
            acc[key] += w * fma(pref[l], fma(T(2), s1, s0), -dself);
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
            acc[key] += w * fma(pref[l], fma(T(2), s1, s0), -dself);
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

template <int MODE, int D, int LMAX, typename T>
__global__ void __launch_bounds__(kCoupleThreads) k_couple(const CoupleParams p)
{
    using AccT = T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 blk = p.kblocks[blockIdx.y];
    const int comps = (MODE == MODE_N3 && D != 2) ? 1 : 2;
    int a_elems;  // T elements of the per-primary copy (N=3: a-row, then the nbins sums of w^2)
    if constexpr (MODE == MODE_D2N4) a_elems = p.nbins * (2 * p.lmax + 1) * 2;
    else a_elems = p.nbins * p.nq + p.nbins;
    T* A = reinterpret_cast<T*>(smem);
    AccT* acc = reinterpret_cast<AccT*>(smem + ((a_elems * (int)sizeof(T) + 15) / 16) * 16);
    const int nacc = (blk.w - blk.z) * comps;
    for (int k = threadIdx.x; k < nacc; k += blockDim.x) acc[k] = AccT(0);

    // catalogue blockIdx.z: its primaries' rows of the a-array and its own partial rows
    const int cat = blockIdx.z;
    const int nprim = p.cat_count ? p.cat_count[cat] : *p.nprim;
    const size_t first = p.cat_first ? (size_t)p.cat_first[cat] : 0;
    const int nchunk = (nprim + p.chunk - 1) / p.chunk;
    double* prow = p.partial + ((size_t)cat * gridDim.x + blockIdx.x) * 2 * p.ncoeff;
    const int stride = p.nbins * p.nq;
    const T* aglob = static_cast<const T*>(p.a) + first * stride;
    const T* wglob = static_cast<const T*>(p.wprim) + first;
    const T* sglob = p.self ? static_cast<const T*>(p.self) + first * p.nbins : nullptr;

    for (int ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const int p0 = ch * p.chunk;
        const int p1 = min(nprim, p0 + p.chunk);
        for (int pi = p0; pi < p1; ++pi) {
            __syncthreads();
            const T* ap = aglob + (size_t)pi * stride;
            if constexpr (MODE == MODE_D2N4) {
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
                if (sglob)
                    for (int i = threadIdx.x; i < p.nbins; i += blockDim.x) A[stride + i] = sglob[(size_t)pi * p.nbins + i];
            }
            const T w = wglob[pi];
            __syncthreads();
            if constexpr (MODE == MODE_N3) body_n3<D, T, AccT>(p, A, sglob ? A + stride : nullptr, w, acc, blk);
            else body_d2n4<T, AccT>(p, reinterpret_cast<const Cx<T>*>(A), w, acc, blk);
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nacc; k += blockDim.x) {
            const int key = blk.z + k / comps;
            const int col = comps == 1 ? 2 * key : 2 * key + (k % comps);
            prow[col] += (double)acc[k];
            acc[k] = AccT(0);
        }
    }
}

// --------------------------------------------------- D=2, N=4, FP32, registers
// A thread owns one item (bin pair b1 < b2, label pair (l1, l2)) and keeps the
// complex sums for every b3 > b2 in registers while it walks a group of G
// primaries held in shared memory:
//     acc[b3] += w u_{l1}(b1) u_{l2}(b2) u_{l3}(b3),   l3 = -(l1 + l2),
// then adds them once into the CTA's FP64 partial row.  Shared memory is read,
// never written, inside the group, so the terms cost FMAs and broadcast loads.
template <int NB, int THREADS>
__global__ void __launch_bounds__(THREADS) k_couple_d2n4_reg(const CoupleParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int nb = p.nbins, L = p.lmax, S = 2 * p.lmax + 1, G = p.group;
    float2* A = reinterpret_cast<float2*>(smem);                  // [G][nb][S], signed l
    float* W = reinterpret_cast<float*>(A + (size_t)G * nb * S);  // [G]
    const int cat = blockIdx.z;
    const int nprim = p.cat_count ? p.cat_count[cat] : *p.nprim;
    const size_t first = p.cat_first ? (size_t)p.cat_first[cat] : 0;
    const int stride = nb * p.nq;
    const float* aglob = static_cast<const float*>(p.a) + first * stride;
    const float* wglob = static_cast<const float*>(p.wprim) + first;
    double* prow = p.partial + ((size_t)cat * gridDim.x + blockIdx.x) * 2 * p.ncoeff;
    const int npair = p.kblocks[0].y - p.kblocks[0].x;
    const int nitems = npair * p.nlam;
    const int ngroup = (nprim + G - 1) / G;
    for (int gi = blockIdx.x; gi < ngroup; gi += gridDim.x) {
        const int g0 = gi * G, gn = min(G, nprim - g0);
        __syncthreads();
        for (int i = threadIdx.x; i < G * nb * S; i += blockDim.x) {
            const int g = i / (nb * S), r = i - g * (nb * S), b = r / S, l = r - b * S - L;
            float re = 0.f, im = 0.f;
            if (g < gn) {
                const int al = l < 0 ? -l : l;
                const float* ap = aglob + (size_t)(g0 + g) * stride + b * p.nq + q_index_d2(al);
                re = ap[0];
                im = al > 0 ? (l < 0 ? -ap[1] : ap[1]) : 0.f;  // a_{-l} = conj(a_l)
            }
            A[i] = make_float2(re, im);
        }
        for (int g = threadIdx.x; g < G; g += blockDim.x) W[g] = g < gn ? wglob[g0 + g] : 0.f;
        __syncthreads();
        for (int it = threadIdx.x; it < nitems; it += blockDim.x) {
            const int pr = it / p.nlam, il = it - (it / p.nlam) * p.nlam;
            const int2 bb = p.pairs[p.kblocks[0].x + pr];
            const int2 ll = p.lam2[il];
            const int l3 = -(ll.x + ll.y);
            const int nk = nb - bb.y - 1;
            float ar[NB], ai[NB];
#pragma unroll
            for (int k = 0; k < NB; ++k) ar[k] = ai[k] = 0.f;
            const float2* ub = A + bb.x * S + ll.x + L;
            const float2* vb = A + bb.y * S + ll.y + L;
            const float2* xb = A + (bb.y + 1) * S + l3 + L;
            for (int g = 0; g < gn; ++g) {
                const float w = W[g];
                const float2 u = ub[g * nb * S], v = vb[g * nb * S];
                const float tr = w * fmaf(u.x, v.x, -u.y * v.y), ti = w * fmaf(u.x, v.y, u.y * v.x);
                const float2* x = xb + g * nb * S;
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    if (k < nk) {
                        const float2 xx = x[k * S];
                        ar[k] = fmaf(tr, xx.x, fmaf(-ti, xx.y, ar[k]));
                        ai[k] = fmaf(tr, xx.y, fmaf(ti, xx.x, ai[k]));
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

template <int MODE, int D, int LMAX, typename T>
cudaError_t launch_t(const CoupleParams& p, int grid, int smem, cudaStream_t s)
{
    auto kern = k_couple<MODE, D, LMAX, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(grid, p.nkb, p.ncat > 1 ? p.ncat : 1), kCoupleThreads, smem, s>>>(p); ++launch_counter();
    return cudaGetLastError();
}

}  // namespace

int couple_max_lmax_d3n4() { return 5; }

// primaries per shared-memory group of the FP32 D=2 N=4 kernel (at most 64, within ~200 KB)
int d2n4_group(int nbins, int lmax)
{
    const int per = nbins * (2 * lmax + 1) * 8 + 4;
    return std::max(1, std::min(64, (200 * 1024) / per));
}

int couple_smem(const CoupleParams& p, int fp64)
{
    if (p.N == 4 && p.D == 3) return couple_d3n4_smem(p, fp64);
    if (p.N == 4 && p.D == 2 && !fp64) {
        const int G = d2n4_group(p.nbins, p.lmax);
        return G * p.nbins * (2 * p.lmax + 1) * 8 + G * 4;
    }
    const int tb = fp64 ? 8 : 4;
    int a_elems;
    int comps;
    if (p.N == 4) {
        a_elems = p.nbins * (2 * p.lmax + 1) * 2;
        comps = 2;
    } else {
        a_elems = p.nbins * p.nq + p.nbins;
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
        if (fp64) return launch_t<MODE_D2N4, 2, 0, double>(p, grid, smem, s);
        const int nbmax = p.nbins - 2;  // b3 values per bin pair
        auto go = [&](auto kern, int threads) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            kern<<<dim3(grid, 1, p.ncat > 1 ? p.ncat : 1), threads, smem, s>>>(p);
            ++launch_counter();
            return cudaGetLastError();
        };
        // one CTA per SM (its group of a-rows fills shared memory): as many warps as registers allow
        if (nbmax <= 8) return go(k_couple_d2n4_reg<8, 512>, 512);
        if (nbmax <= 16) return go(k_couple_d2n4_reg<16, 512>, 512);
        return go(k_couple_d2n4_reg<32, 256>, 256);
    }
    return launch_couple_d3n4(p, fp64, grid, couple_d3n4_threads(p.max_block_pairs), smem, s);
}

}  // namespace npcf
