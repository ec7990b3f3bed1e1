// npcf_pairs.cuh -- the pair kernel: for every primary y_j, the radially
// binned harmonic coefficients
//     a^b_l(y_j) = (1/v_b) sum_k w_k Y*_l(unit(y_k - y_j)) Theta^b(|y_k - y_j|)
// of eq. NPCF-estimator-discrete (the inner sum), written to an a-array in HBM.
//
// Design (GB300, sm_103a):
//  * One CTA takes one work item = up to W primaries of one cell; warp w owns
//    primary w.  The CTA walks the cell stencil (neighbour cells within r_max
//    of the primary cell) and stages each neighbour cell through shared
//    memory; every warp scans the staged candidates against its primary.
//  * Lanes own radial bins: lane l accumulates only bin lane_bin[l] (the host
//    gives big shells more lanes).  A candidate that falls in bin b is
//    appended to a per-(warp, bin) queue in shared memory; when enough are
//    queued, every lane pops one pair of its own bin and adds w Y* for all
//    (l, m) into registers.  No cross-lane reduction happens until the
//    primary is finished.
//  * The bin of a pair is decided exactly as the FP64 definition decides it:
//    FP32 distances pick the bin, and any pair within a few FP32 ulps of an
//    edge is re-decided from the original coordinates in FP64.
#pragma once

#include <cuda_runtime.h>

#include "npcf_device.cuh"
#include "npcf_internal.h"

namespace npcf {

template <int D, int LMAX, typename T>
struct PairCfg {
    static constexpr int NQ = num_q(D, LMAX);
    static constexpr int kThreads = (sizeof(T) == 4) ? (NQ <= 64 ? 512 : 256) : (NQ <= 40 ? 256 : 128);
};

// shared-memory bytes of one CTA (must match the carve-up in k_pairs)
__host__ __device__ inline int pair_warp_bytes(int rec_bytes, int t_bytes, int nbins, int nq_compiled)
{
    int stage = nbins * kStageCap * rec_bytes;
    int scratch = 32 * (nq_compiled + 1) * t_bytes;
    int body = stage > scratch ? stage : scratch;
    return ((128 + body) + 15) / 16 * 16;
}

__host__ __device__ inline int pair_fixed_bytes(int rec_bytes, int threads)
{
    return threads * rec_bytes + kTab + 576;
}

template <int D, int LMAX, typename T>
__device__ __forceinline__ void accum_pair(T* acc, const Rec<D, T>& e)
{
    if constexpr (D == 2) accum_d2<LMAX, T>(acc, e.x(0), e.x(1), e.w());
    else if constexpr (D == 3) accum_d3<LMAX, T>(acc, e.x(0), e.x(1), e.x(2), e.w());
    else accum_d4<LMAX, T>(acc, e.x(0), e.x(1), e.x(2), e.x(3), e.w());
}

__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return rsqrt(x); }

template <int D, int LMAX, typename T>
__global__ void __launch_bounds__(PairCfg<D, LMAX, T>::kThreads, 1) k_pairs(const PairParams p)
{
    using R = Rec<D, T>;
    constexpr int NQ = PairCfg<D, LMAX, T>::NQ;
    constexpr bool kFP32 = sizeof(T) == 4;
    const unsigned full = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem[];
    const int nthreads = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nbins = p.nbins;
    R* tile = reinterpret_cast<R*>(smem);
    unsigned char* tab = smem + nthreads * sizeof(R);
    float* s_edge = reinterpret_cast<float*>(tab + kTab);        // nbins + 1
    double* s_edge2 = reinterpret_cast<double*>(tab + kTab + 192); // nbins + 1
    signed char* s_first = reinterpret_cast<signed char*>(tab + kTab + 192 + 272);
    signed char* s_nl = s_first + 32;
    unsigned char* wbase = smem + pair_fixed_bytes(sizeof(R), nthreads) +
                           warp * pair_warp_bytes(sizeof(R), sizeof(T), nbins, NQ);
    int* cnt = reinterpret_cast<int*>(wbase);
    R* stage = reinterpret_cast<R*>(wbase + 128);
    T* scratch = reinterpret_cast<T*>(wbase + 128);

    for (int i = threadIdx.x; i < kTab / 4; i += nthreads)
        reinterpret_cast<int*>(tab)[i] = reinterpret_cast<const int*>(p.tab)[i];
    if (threadIdx.x <= nbins) {
        s_edge[threadIdx.x] = p.edgef[threadIdx.x];
        s_edge2[threadIdx.x] = p.edge2[threadIdx.x];
    }
    if (threadIdx.x < nbins) {
        s_first[threadIdx.x] = p.bin_first[threadIdx.x];
        s_nl[threadIdx.x] = p.bin_nlanes[threadIdx.x];
    }
    const int mybin = p.lane_bin[lane];
    const int myrank = p.lane_rank[lane];
    const int mynl = p.bin_nlanes[mybin];
    const T* qnorm = static_cast<const T*>(p.qnorm);
    const T* inv_vb = static_cast<const T*>(p.inv_vb);
    const R* rec = static_cast<const R*>(p.rec);
    const int nq = p.nq;
    const float tol = p.tol;

    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(p.ticket, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= *p.nitems) break;
        const int4 it = p.items[item];
        const bool active = warp < it.z;
        const int jslot = it.y + (active ? warp : 0);
        const int pidx = it.w + warp;

        int cc[D];
        {
#pragma unroll
            for (int d = 0; d < D; ++d) cc[d] = (it.x / p.stride[d]) % p.nc[d];
        }
        const R pj = rec[jslot];
        T xj[D];
#pragma unroll
        for (int d = 0; d < D; ++d) xj[d] = pj.x(d);
        const T wj = pj.w();

        T acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = T(0);
        if (lane < nbins) cnt[lane] = 0;
        __syncwarp();
        unsigned npairs = 0;
        unsigned long long ncand = 0;

        // one consumption round: every lane pops one pair of its own bin
        auto round = [&]() {
            const int q = cnt[mybin];
            if (myrank < q) {
                const R e = stage[mybin * kStageCap + (q - 1 - myrank)];
                accum_pair<D, LMAX, T>(acc, e);
            }
            __syncwarp();
            if (myrank == 0) cnt[mybin] = q > mynl ? q - mynl : 0;
            __syncwarp();
        };

        for (int s = 0; s < p.nstencil; ++s) {
            const int packed = p.stencil[s];
            int ncell = 0;
            bool cell_ok = true;
            T xjs[D];
            double shd[D];
            T dmin2 = T(0), dmax2 = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int o = (int)(signed char)((packed >> (8 * d)) & 0xff);
                int c = cc[d] + o;
                const T lo = T((double)c * p.side[d]);
                const T hi = T((double)(c + 1) * p.side[d]);
                double sh = 0.0;
                if (c < 0) {
                    cell_ok = cell_ok && p.periodic;
                    c += p.nc[d];
                    sh = -p.box[d];
                } else if (c >= p.nc[d]) {
                    cell_ok = cell_ok && p.periodic;
                    c -= p.nc[d];
                    sh = p.box[d];
                }
                ncell += c * p.stride[d];
                shd[d] = sh;
                xjs[d] = T((double)xj[d] - sh);
                const T a = fmax(fmax(lo - xj[d], xj[d] - hi), T(0));
                dmin2 = fma(a, a, dmin2);
                const T b = fmax(fabs(xj[d] - lo), fabs(xj[d] - hi));
                dmax2 = fma(b, b, dmax2);
            }
            if (!cell_ok) continue;  // CTA-uniform
            const bool skip = !active || dmin2 >= T(p.rmax2f) || dmax2 < T(p.rmin2f);
            const int start = p.cell_start[ncell], end = p.cell_start[ncell + 1];
            for (int t0 = start; t0 < end; t0 += nthreads) {
                const int tn = min(nthreads, end - t0);
                __syncthreads();
                if (threadIdx.x < tn) tile[threadIdx.x] = rec[t0 + threadIdx.x];
                __syncthreads();
                if (skip) continue;
                ncand += tn;
                for (int c0 = 0; c0 < tn; c0 += 32) {
                    const int k = c0 + lane;
                    const bool valid = k < tn;
                    R pk = tile[valid ? k : 0];
                    T dx[D];
                    T r2 = T(0);
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        if constexpr (kFP32) dx[d] = pk.x(d) - xjs[d];
                        else dx[d] = (pk.x(d) - xj[d]) + T(shd[d]);
                        r2 = fma(dx[d], dx[d], r2);
                    }
                    int bin = -1;
                    T rinv = T(0);
                    if (valid && r2 > T(0) && r2 < T(p.rmax2f) && r2 >= T(p.rmin2f)) {
                        rinv = rsqrt_t(r2);
                        const float r = (float)(r2 * rinv);
                        int b;
                        if (r < s_edge[0]) {
                            b = -1;
                        } else {
                            int kk = (int)((r - p.tab_lo) * p.tab_inv);
                            kk = kk < 0 ? 0 : (kk >= kTab ? kTab - 1 : kk);
                            b = tab[kk];
                            while (b < nbins && r >= s_edge[b + 1]) ++b;
                        }
                        const int blo = b < 0 ? 0 : b;
                        const int bhi = b + 1 > nbins ? nbins : (b + 1 < 0 ? 0 : b + 1);
                        const bool near = !kFP32 || fabsf(r - s_edge[blo]) < tol || fabsf(r - s_edge[bhi]) < tol;
                        if (near) {
                            // exact decision from the original coordinates, as the definition makes it
                            double sd = 0.0;
#pragma unroll
                            for (int d = 0; d < D; ++d) {
                                const double dd = __dadd_rn(__dadd_rn((double)pk.x(d), -(double)xj[d]), shd[d]);
                                sd = (d == 0) ? __dmul_rn(dd, dd) : __dadd_rn(sd, __dmul_rn(dd, dd));
                            }
                            b = -1;
                            if (sd > 0.0 && sd >= s_edge2[0]) {
                                for (int e = 0; e < nbins; ++e)
                                    if (sd < s_edge2[e + 1]) {
                                        b = e;
                                        break;
                                    }
                            }
                        } else if (b >= nbins) {
                            b = -1;
                        }
                        bin = b;
                    }
                    // append to the per-bin queues (warp-aggregated)
                    const bool take = bin >= 0;
                    const unsigned peers = __match_any_sync(full, take ? bin : 64 + lane);
                    const int rank = __popc(peers & ((1u << lane) - 1u));
                    const int base = take ? cnt[bin] : 0;
                    __syncwarp();
                    if (take) {
                        R e;
                        T* f = reinterpret_cast<T*>(e.v);
#pragma unroll
                        for (int d = 0; d < D; ++d) f[d] = dx[d] * rinv;
                        f[D] = pk.w();
                        stage[bin * kStageCap + base + rank] = e;
                        if (rank == 0) cnt[bin] = base + __popc(peers);
                        ++npairs;
                    }
                    __syncwarp();
                    // consume while enough is queued or a queue nears capacity
                    for (;;) {
                        const int qv = lane < nbins ? cnt[lane] : 0;
                        const int tot = __reduce_add_sync(full, qv);
                        const bool over = __any_sync(full, qv > kStageCap - 32);
                        if (tot < 64 && !over) break;
                        round();
                    }
                }
            }
        }
        // drain
        for (;;) {
            const int qv = lane < nbins ? cnt[lane] : 0;
            if (__reduce_add_sync(full, qv) == 0) break;
            round();
        }
        // statistics
        {
            unsigned tot = __reduce_add_sync(full, npairs);
            if (lane == 0 && active) {
                atomicAdd(&p.stats[0], (unsigned long long)tot);
                atomicAdd(&p.stats[1], ncand);
            }
        }
        // reduce the lanes of each bin and write a^b (normalised)
#pragma unroll
        for (int q = 0; q < NQ; ++q) scratch[lane * (NQ + 1) + q] = acc[q];
        __syncwarp();
        if (active) {
            T* aout = static_cast<T*>(p.a_out) + (size_t)pidx * nbins * nq;
            for (int i = lane; i < nbins * nq; i += 32) {
                const int b = i / nq, q = i - b * nq;
                const int f0 = s_first[b], nl = s_nl[b];
                T sum = T(0);
                for (int r = 0; r < nl; ++r) sum += scratch[(f0 + r) * (NQ + 1) + q];
                aout[i] = sum * qnorm[q] * inv_vb[b];
            }
            if (lane == 0) static_cast<T*>(p.w_out)[pidx] = wj;
        }
        __syncwarp();
    }
}

template <int D, int LMAX, typename T>
cudaError_t launch_pairs_t(const PairParams& p, int grid, int smem, cudaStream_t s)
{
    auto kern = k_pairs<D, LMAX, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, p.warps * 32, smem, s>>>(p); ++launch_counter();
    return cudaGetLastError();
}

}  // namespace npcf
