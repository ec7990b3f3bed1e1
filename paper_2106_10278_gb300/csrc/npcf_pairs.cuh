// npcf_pairs.cuh -- the pair kernel: for every primary y_j, the radially
// binned harmonic coefficients
//     a^b_l(y_j) = (1/v_b) sum_k w_k Y*_l(unit(y_k - y_j)) Theta^b(|y_k - y_j|)
// of eq. NPCF-estimator-discrete (the inner sum), written to an a-array in HBM.
//
// Design (GB300, sm_103a):
//  * One CTA takes one work item = up to W primaries of one cell; warp w owns
//    primary w.  The CTA lists the item's neighbour cells (the stencil cells
//    within r_max of the primary cell that are non-empty) in shared memory
//    once; then every warp walks that list on its own, skips the cells its
//    primary cannot reach, and streams the candidates from global memory
//    (L1/L2 resident) with a two-deep register prefetch -- no block barriers
//    while scanning.
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

// staged pairs per warp (shared by all bins): 416 16-byte records (D <= 3, FP32) keep the
// CTA within the 196 KB shared-memory carveout; larger records get 320
__host__ __device__ constexpr int pool_slots(int rec_bytes) { return rec_bytes <= 16 ? 416 : 320; }
constexpr int kQCap = 192;      // entries of one bin's index queue

// Shared-memory carve-up of one CTA (host and device must agree):
//   radial table + edges + lane map | job lists + scan scratch | the item's CatGeom
//   | per warp: [fstack[slots] u16 | binq[nbins][kQCap] u16 | pool of `slots` records]
// where the pool region also holds the final cross-lane reduction scratch.  Queue
// lengths and the free-stack top live in registers (lane b keeps bin b's length).
__host__ __device__ inline int pair_pool_bytes(int rec_bytes, int t_bytes, int nq_compiled)
{
    const int pool = pool_slots(rec_bytes) * rec_bytes;
    const int scratch = 32 * (nq_compiled + 1) * t_bytes;
    return pool > scratch ? pool : scratch;
}

__host__ __device__ inline int pair_warp_bytes(int rec_bytes, int t_bytes, int nbins, int nq_compiled)
{
    const int head = pool_slots(rec_bytes) * 2 + nbins * kQCap * 2;
    return ((head + 15) / 16) * 16 + ((pair_pool_bytes(rec_bytes, t_bytes, nq_compiled) + 15) / 16) * 16;
}

constexpr int kMaxJobs = 640;   // neighbour cells of one item (the largest stencil used: 613 cells, D=3 c=4)

// fixed part: radial table | edges + lane map (576) | job lists + scan scratch | the item's CatGeom
constexpr int kGeomOffset = kTab + 576 + (3 * kMaxJobs + 4 + 72) * 4;
__host__ __device__ inline int pair_fixed_bytes(int rec_bytes, int threads)
{
    (void)rec_bytes;
    (void)threads;
    return kGeomOffset + ((int)sizeof(CatGeom) + 15) / 16 * 16;
}

// Thread-block-wide: copy catalogue `cat`'s grid into shared memory (the
// caller synchronises before anyone reads it).
__device__ __forceinline__ void load_geom(CatGeom* dst, const CatGeom* geo, int cat)
{
    if (threadIdx.x < kGeomWords)
        reinterpret_cast<int*>(dst)[threadIdx.x] = reinterpret_cast<const int*>(geo + cat)[threadIdx.x];
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

// Exclusive block-wide scan of two ints per thread (deterministic), totals
// returned to every thread.  `ws` holds 2 * 32 ints of shared scratch.
__device__ __forceinline__ void block_scan2(int a, int b, int* ea, int* eb, int* ta, int* tb, int* ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int ia = a, ib = b;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int xa = __shfl_up_sync(0xffffffffu, ia, o);
        const int xb = __shfl_up_sync(0xffffffffu, ib, o);
        if (lane >= o) {
            ia += xa;
            ib += xb;
        }
    }
    if (lane == 31) {
        ws[warp] = ia;
        ws[32 + warp] = ib;
    }
    __syncthreads();
    if (warp == 0) {
        const int va = lane < nw ? ws[lane] : 0, vb = lane < nw ? ws[32 + lane] : 0;
        int sa = va, sb = vb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int xa = __shfl_up_sync(0xffffffffu, sa, o);
            const int xb = __shfl_up_sync(0xffffffffu, sb, o);
            if (lane >= o) {
                sa += xa;
                sb += xb;
            }
        }
        ws[lane] = sa - va;  // exclusive warp offsets
        ws[32 + lane] = sb - vb;
        if (lane == 31) {
            ws[64] = sa;
            ws[65] = sb;
        }
    }
    __syncthreads();
    *ea = ws[warp] + ia - a;
    *eb = ws[32 + warp] + ib - b;
    *ta = ws[64];
    *tb = ws[65];
    __syncthreads();
}


// The radial bin of one candidate pair, decided exactly as the FP64 definition
// decides it ([e_b, e_{b+1}) on the FP64 r^2 of the original coordinates):
// the FP32 r^2 indexes a table over r^2 (bits 0-5 the bin, 63 = none; bit 6:
// an edge lies within the FP32 error window of the bucket); flagged buckets
// are re-decided in FP32 unless the pair sits within that window, and those
// few pairs in FP64.  Returns -1 outside the bins.  Shared by the forward and
// adjoint pair kernels so that both see the same pair set.
template <int D, typename T>
__device__ __forceinline__ int decide_bin(const PairParams& p, const CatGeom& g, const unsigned char* tab,
                                          const float* s_edge, const double* s_edge2, const int* cc, int packed,
                                          const T* xj, const Rec<D, T>& pk, T r2, bool* flagged, bool* exact_out)
{
    constexpr bool kFP32 = sizeof(T) == 4;
    if (!(r2 > T(0) && r2 < T(p.rmax2f) && r2 >= T(p.rmin2f))) return -1;
    int kk = (int)(((float)r2 - p.tab_lo) * p.tab_inv);
    kk = kk < 0 ? 0 : (kk >= kTab ? kTab - 1 : kk);
    const int code = tab[kk];
    int b = (code & 63) == 63 ? -1 : (code & 63);
    bool exact = !kFP32;
    if (kFP32 && (code & 64)) {
        *flagged = true;
        const float r = (float)r2 * rsqrtf((float)r2);
        // bb = number of edges <= r, walked from the bucket's own count (0-1 steps)
        int bb = (code & 63) == 63 ? (r >= s_edge[p.nbins >> 1] ? p.nbins + 1 : 0) : (code & 63) + 1;
        while (bb <= p.nbins && r >= s_edge[bb]) ++bb;
        while (bb > 0 && r < s_edge[bb - 1]) --bb;
        b = (bb >= 1 && bb <= p.nbins) ? bb - 1 : -1;
        exact = (bb >= 1 && r - s_edge[bb - 1] < p.tol) || (bb <= p.nbins && s_edge[bb] - r < p.tol);
    }
    if (exact) {
        *exact_out = true;
        double sd = 0.0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
            const int c = cc[d] + (int)(signed char)((packed >> (8 * d)) & 0xff);
            const double shd = c < 0 ? -g.box[d] : (c >= g.nc[d] ? g.box[d] : 0.0);
            const double dd = __dadd_rn(__dadd_rn((double)pk.x(d), -(double)xj[d]), shd);
            sd = (d == 0) ? __dmul_rn(dd, dd) : __dadd_rn(sd, __dmul_rn(dd, dd));
        }
        b = -1;
        if (sd > 0.0 && sd >= s_edge2[0]) {
            for (int e = 0; e < p.nbins; ++e)
                if (sd < s_edge2[e + 1]) {
                    b = e;
                    break;
                }
        }
    }
    return b;
}

// Cell geometry of one stencil cell for one primary: the shifted primary
// position (so that pk - xjs is the minimum-image separation) and whether the
// cell can hold a pair in [e_0, e_nb) of that primary.
template <int D, typename T>
__device__ __forceinline__ bool cell_geometry(const PairParams& p, const CatGeom& g, const int* cc, int packed,
                                              const T* xj, T* xjs)
{
    constexpr bool kFP32 = sizeof(T) == 4;
    T dmin2 = T(0), dmax2 = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int c = cc[d] + (int)(signed char)((packed >> (8 * d)) & 0xff);
        T side, box;
        if constexpr (kFP32) {
            side = g.sidef[d];
            box = g.boxf[d];
        } else {
            side = g.side[d];
            box = g.box[d];
        }
        const T lo = T(c) * side;
        const T hi = lo + side;
        const T sh = c < 0 ? -box : (c >= g.nc[d] ? box : T(0));
        xjs[d] = xj[d] - sh;
        const T a = fmax(fmax(lo - xj[d], xj[d] - hi), T(0));
        dmin2 = fma(a, a, dmin2);
        const T b = fmax(fabs(xj[d] - lo), fabs(xj[d] - hi));
        dmax2 = fma(b, b, dmax2);
    }
    return !(dmin2 >= T(p.rmax2f) || dmax2 < T(p.rmin2f));
}

template <int D, typename T>
__device__ __forceinline__ Rec<D, T> ldg_rec(const Rec<D, T>* src, int i)
{
    // read-only path, 16 bytes at a time
    constexpr int kChunks = sizeof(Rec<D, T>) / 16;
    const float4* s = reinterpret_cast<const float4*>(src + i);
    union {
        float4 f[kChunks];
        Rec<D, T> r;
    } u;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) u.f[c] = __ldg(s + c);
    return u.r;
}

template <int D, int LMAX, typename T>
__global__ void __launch_bounds__(PairCfg<D, LMAX, T>::kThreads, 1) k_pairs(const PairParams p)
{
    using R = Rec<D, T>;
    constexpr int NQ = PairCfg<D, LMAX, T>::NQ;
    constexpr bool kFP32 = sizeof(T) == 4;
    constexpr int kPool = pool_slots((int)sizeof(R));
    const unsigned full = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem[];
    const int nthreads = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int nbins = p.nbins;
    unsigned char* tab = smem;
    float* s_edge = reinterpret_cast<float*>(tab + kTab);          // nbins + 1
    double* s_edge2 = reinterpret_cast<double*>(tab + kTab + 192);  // nbins + 1
    signed char* s_first = reinterpret_cast<signed char*>(tab + kTab + 192 + 272);
    signed char* s_nl = s_first + 32;
    int* job_a = reinterpret_cast<int*>(tab + kTab + 576);  // kMaxJobs: first slot of the cell
    int* job_pk = job_a + kMaxJobs;                          // kMaxJobs: packed stencil offset
    int* job_pre = job_pk + kMaxJobs;                        // kMaxJobs + 1: record prefix
    int* ws = job_pre + kMaxJobs + 4;                        // 68 ints of scan scratch
    CatGeom* s_geo = reinterpret_cast<CatGeom*>(smem + kGeomOffset);
    unsigned char* wbase = smem + pair_fixed_bytes(sizeof(R), nthreads) +
                           warp * pair_warp_bytes(sizeof(R), sizeof(T), nbins, NQ);
    unsigned short* fstack = reinterpret_cast<unsigned short*>(wbase);
    unsigned short* binq = fstack + kPool;
    R* pool = reinterpret_cast<R*>(wbase + ((kPool * 2 + nbins * kQCap * 2 + 15) / 16) * 16);  // as pair_warp_bytes
    T* scratch = reinterpret_cast<T*>(pool);

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
    const int lane_nl = lane < nbins ? p.bin_nlanes[lane] : 0;
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
        load_geom(s_geo, p.geo, it.z >> 8);
        __syncthreads();
        const CatGeom& g = *s_geo;
        const bool active = warp < (it.z & 0xff);
        const int jslot = it.y + (active ? warp : 0);
        const int pidx = it.w + warp;

        int cc[D];
#pragma unroll
        for (int d = 0; d < D; ++d) cc[d] = ((it.x - g.base) / g.stride[d]) % g.nc[d];

        // the item's neighbour cells: valid (periodic or inside the grid) and non-empty,
        // in stencil order, with the prefix of their record counts
        int njobs = 0, V = 0;
        for (int base = 0; base < p.nstencil; base += nthreads) {
            const int sidx = base + threadIdx.x;
            int keep = 0, len = 0, a = 0, pk = 0;
            if (sidx < p.nstencil) {
                pk = p.stencil[sidx];
                int cell = g.base;
                bool ok = true;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    int c = cc[d] + (int)(signed char)((pk >> (8 * d)) & 0xff);
                    if (c < 0) {
                        ok = ok && p.periodic;
                        c += g.nc[d];
                    } else if (c >= g.nc[d]) {
                        ok = ok && p.periodic;
                        c -= g.nc[d];
                    }
                    cell += c * g.stride[d];
                }
                if (ok) {
                    a = p.cell_start[cell];
                    len = p.cell_start[cell + 1] - a;
                    keep = len > 0;
                }
            }
            int pos, off, tcount, tlen;
            block_scan2(keep, keep ? len : 0, &pos, &off, &tcount, &tlen, ws);
            if (keep) {
                job_a[njobs + pos] = a;
                job_pk[njobs + pos] = pk;
                job_pre[njobs + pos] = V + off;
            }
            njobs += tcount;
            V += tlen;
        }
        if (threadIdx.x == 0) job_pre[njobs] = V;
        __syncthreads();

        const R pj = rec[jslot];
        T xj[D];
#pragma unroll
        for (int d = 0; d < D; ++d) xj[d] = pj.x(d);
        const T wj = pj.w();

        T acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = T(0);
        int qlen = 0;                   // lane b < nbins: length of bin b's queue
        int ftop_r = kPool, tot_r = 0;  // warp-uniform: free-stack top, staged pairs
        for (int i = lane; i < kPool; i += 32) fstack[i] = (unsigned short)i;
        __syncwarp();
        unsigned npairs = 0;
        unsigned long long ncand = 0;
        unsigned nrounds = 0, nbusy = 0, nchunks = 0, nforced = 0, nflag = 0, nexact = 0;

        // one consumption round: every lane pops one staged pair of its own bin
        auto round = [&]() {
            const int q = __shfl_sync(full, qlen, mybin);
            const bool has = myrank < q;
            ++nrounds;
            nbusy += has ? 1u : 0u;
            int idx = 0;
            if (has) {
                idx = binq[mybin * kQCap + (q - 1 - myrank)];
                const R e = pool[idx];
                accum_pair<D, LMAX, T>(acc, e);
            }
            const unsigned fm = __ballot_sync(full, has);
            if (has) fstack[ftop_r + __popc(fm & lt_mask)] = (unsigned short)idx;
            ftop_r += __popc(fm);
            tot_r -= __popc(fm);
            qlen = qlen > lane_nl ? qlen - lane_nl : 0;
            __syncwarp();
        };
        auto consume = [&](bool drain) {
            for (;;) {
                const int tot = tot_r;
                if (tot == 0) break;
                const int busy = __reduce_add_sync(full, qlen < lane_nl ? qlen : lane_nl);
                const bool over = __any_sync(full, qlen > kQCap - 32) || tot > kPool - 32;
                const bool want = busy >= p.busy_round || tot >= p.tot_round;
                if (!drain && !want && !over) break;
                if (!drain && !want) ++nforced;
                round();
            }
        };

        // every warp walks the item's cells on its own, streaming candidates from
        // global memory (L1/L2) with a two-deep register prefetch: no block barriers
        if (active) {
            for (int j = 0; j < njobs; ++j) {
                const int seg_a = job_a[j];
                const int seg_n = job_pre[j + 1] - job_pre[j];
                const int packed = job_pk[j];
                T xjs[D];
                if (!cell_geometry<D, T>(p, g, cc, packed, xj, xjs)) continue;
                ncand += seg_n;
                const R* src = rec + seg_a;
                R nxt0 = ldg_rec(src, lane < seg_n ? lane : 0);
                R nxt1 = ldg_rec(src, 32 + lane < seg_n ? 32 + lane : 0);
                for (int c0 = 0; c0 < seg_n; c0 += 32) {
                    const int k = c0 + lane;
                    const bool valid = k < seg_n;
                    const R pk = nxt0;
                    nxt0 = nxt1;
                    if (c0 + 64 < seg_n) nxt1 = ldg_rec(src, c0 + 64 + lane < seg_n ? c0 + 64 + lane : 0);
                    T dx[D];
                    T r2 = T(0);
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        if constexpr (kFP32) dx[d] = pk.x(d) - xjs[d];
                        else dx[d] = (pk.x(d) - xj[d]) + (xj[d] - xjs[d]);
                        r2 = fma(dx[d], dx[d], r2);
                    }
                    bool anyflag = false, anyexact = false;
                    const int bin = valid ? decide_bin<D, T>(p, g, tab, s_edge, s_edge2, cc, packed, xj, pk, r2, &anyflag,
                                                             &anyexact)
                                          : -1;
                    ++nchunks;
                    nflag += __any_sync(full, anyflag) ? 1u : 0u;
                    nexact += __any_sync(full, anyexact) ? 1u : 0u;
                    // stage the pair: a pool slot from the free stack, its index on the bin queue
                    const bool take = bin >= 0;
                    const unsigned tm = __ballot_sync(full, take);
                    if (tm == 0u) continue;
                    // lanes staging into the same bin: AND of the ballots of the bin's bits
                    unsigned peers = tm, mine = tm;  // mine: lanes staging into bin `lane`
#pragma unroll
                    for (int kb = 0; kb < 5; ++kb) {
                        const unsigned bk = __ballot_sync(full, (bin >> kb) & 1);
                        peers &= ((bin >> kb) & 1) ? bk : ~bk;
                        mine &= ((lane >> kb) & 1) ? bk : ~bk;
                    }
                    const int rank = __popc(peers & lt_mask);
                    const int base = __shfl_sync(full, qlen, take ? bin : 0);
                    if (take) {
                        const int slot = fstack[ftop_r - 1 - __popc(tm & lt_mask)];
                        R e;
                        T* f = reinterpret_cast<T*>(e.v);
                        const T rinv = rsqrt_t(r2);
#pragma unroll
                        for (int d = 0; d < D; ++d) f[d] = dx[d] * rinv;
                        f[D] = pk.w();
                        pool[slot] = e;
                        binq[bin * kQCap + base + rank] = (unsigned short)slot;
                        ++npairs;
                    }
                    if (lane < nbins) qlen += __popc(mine);
                    ftop_r -= __popc(tm);
                    tot_r += __popc(tm);
                    __syncwarp();
                    consume(false);
                }
            }
        }
        consume(true);
        // statistics
        {
            const unsigned tot = __reduce_add_sync(full, npairs);
            const unsigned busy = __reduce_add_sync(full, nbusy);
            if (lane == 0 && active) {
                atomicAdd(&p.stats[0], (unsigned long long)tot);
                atomicAdd(&p.stats[1], ncand);
                atomicAdd(&p.stats[2], (unsigned long long)nrounds);
                atomicAdd(&p.stats[3], (unsigned long long)busy);
                atomicAdd(&p.stats[4], (unsigned long long)nchunks);
                atomicAdd(&p.stats[5], (unsigned long long)nforced);
                atomicAdd(&p.stats[6], (unsigned long long)nflag);
                atomicAdd(&p.stats[7], (unsigned long long)nexact);
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
