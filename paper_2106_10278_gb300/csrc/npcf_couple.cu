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

template <int MODE, int D, int LMAX, typename T>
__global__ void __launch_bounds__(kCoupleThreads) k_couple(const CoupleParams p)
{
    using AccT = T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 blk = p.kblocks[blockIdx.y];
    const int comps = (MODE == MODE_N3 && D != 2) ? 1 : 2;
    int a_elems;  // T elements of the per-primary copy
    if constexpr (MODE == MODE_D2N4) a_elems = p.nbins * (2 * p.lmax + 1) * 2;
    else a_elems = p.nbins * p.nq;
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
            }
            const T w = wglob[pi];
            __syncthreads();
            if constexpr (MODE == MODE_N3) body_n3<D, T, AccT>(p, A, w, acc, blk);
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

int couple_smem(const CoupleParams& p, int fp64)
{
    if (p.N == 4 && p.D == 3) return couple_d3n4_smem(p, fp64);
    const int tb = fp64 ? 8 : 4;
    int a_elems;
    int comps;
    if (p.N == 4) {
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
    return launch_couple_d3n4(p, fp64, grid, couple_d3n4_threads(p.max_block_pairs), smem, s);
}

}  // namespace npcf
