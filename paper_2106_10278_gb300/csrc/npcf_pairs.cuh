// npcf_pairs.cuh -- the pair kernel: for every primary y_j, the radially
// binned harmonic coefficients
//     a^b_l(y_j) = (1/v_b) sum_k w_k Y*_l(unit(y_k - y_j)) Theta^b(|y_k - y_j|)
// of eq. NPCF-estimator-discrete (the inner sum), written to an a-array in HBM.
//
// Design (GB300, sm_103a):
//  * One CTA takes one work item = up to W primaries of one cell; warp w owns
//    primary w.  The stencil is walked by rows: the cells that differ only in
//    their axis-0 offset are consecutive in the sorted records, so each row is
//    one run of candidates.  The CTA tabulates the item's rows once; every
//    warp trims each row to the cells its primary can reach (the x range that
//    the row's distance across the other axes leaves within r_max, split where
//    it wraps) and streams the run from global memory (L1/L2 resident) with a
//    two-chunk register prefetch -- no block barriers while scanning.
//  * Accepted pairs (unit separation, weight, bin) are compacted into a
//    per-warp batch in shared memory.  A full batch is counting-sorted by bin
//    (arrival order kept inside a bin), the 32 lanes are shared out among the
//    bins in proportion to this batch's own counts (a lane accumulates pairs
//    of one bin), every lane adds w Y* for all components of its pairs into
//    registers, and the lanes' sums are merged into the warp's per-bin
//    accumulators in shared memory.  Every sum runs in a fixed order, so the
//    results are bitwise reproducible.
//  * The bin of a pair is decided exactly as the FP64 definition decides it:
//    the FP32 r^2 indexes a table of bins (guard entries catch r^2 outside
//    the bins); the few table buckets that an edge's FP32 error window
//    touches are re-decided in FP32, and pairs within that window from the
//    original coordinates in FP64 -- a warp-uniform branch taken only when a
//    lane needs it.
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

constexpr int kMaxJobs = 640;   // neighbour cells of one item (the largest stencil used: 613 cells, D=3 c=4)
constexpr int kJobWords = kMaxJobs / 32;

// Pairs per warp batch (a multiple of 32, at most 1024): by default 512 records of 16 bytes
// (FP32, D <= 3), 256 of the larger records; the plan may choose others (autotuning).
__host__ __device__ constexpr int pair_batch(int rec_bytes) { return rec_bytes <= 16 ? 512 : 256; }

// Shared-memory carve-up of one CTA (host and device must agree):
//   radial table + edges | job lists + scan scratch | the item's CatGeom
//   | per warp: [records (also the merge scratch) | acc[nbins][nq] | bins u8 | idx u16 | 4 x 32 ints
//                | sum of w^2 per bin (32)]
__host__ __device__ inline int pair_rec_region(int rec_bytes, int t_bytes, int nq_compiled, int B)
{
    const int recs = B * rec_bytes;
    const int scratch = 32 * (nq_compiled + 1) * t_bytes;
    return ((recs > scratch ? recs : scratch) + 15) / 16 * 16;
}

__host__ __device__ inline int pair_warp_bytes(int rec_bytes, int t_bytes, int nbins, int nq_compiled, int B)
{
    return pair_rec_region(rec_bytes, t_bytes, nq_compiled, B) + (nbins * nq_compiled * t_bytes + 15) / 16 * 16 +
           (3 * B + 15) / 16 * 16 + 4 * 32 * 4 + 32 * t_bytes;
}

// fixed part: radial table | edges (576) | job lists + scan scratch | the item's CatGeom
constexpr int kGeomOffset = kTabBytes + 576 + (3 * kMaxJobs + 4 + 72) * 4;
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
// decides it ([e_b, e_{b+1}) on the FP64 r^2 of the original coordinates).
// `code` is the table entry of the pair's FP32 r^2 (bits 0-5 the bin, 63 = none;
// bit 6: an edge lies within the FP32 error window of the bucket): a flagged
// bucket is re-decided in FP32 unless the pair sits within that window, and
// those few pairs in FP64 (FP64 plans: every pair in FP64).  Returns -1
// outside the bins.
template <int D, typename T>
__device__ __forceinline__ int bin_refine(const PairParams& p, const CatGeom& g, const float* s_edge,
                                          const double* s_edge2, const int* cc, int packed, const T* xj,
                                          const Rec<D, T>& pk, T r2, int code, bool* exact_out)
{
    constexpr bool kFP32 = sizeof(T) == 4;
    if (!(r2 > T(0))) return -1;
    int b = (code & 63) == 63 ? -1 : (code & 63);
    bool exact = !kFP32;
    if (kFP32 && (code & 64)) {
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

// The same decision from r^2 alone (range check, table, refinement); shared by
// the adjoint pair kernel and the FP64 forward path so that all see one pair set.
// tab: the guarded table (bucket k at tab[k + 1]).
template <int D, typename T>
__device__ __forceinline__ int decide_bin(const PairParams& p, const CatGeom& g, const unsigned char* tab,
                                          const float* s_edge, const double* s_edge2, const int* cc, int packed,
                                          const T* xj, const Rec<D, T>& pk, T r2, bool* flagged, bool* exact_out)
{
    constexpr bool kFP32 = sizeof(T) == 4;
    if (!(r2 > T(0) && r2 < T(p.rmax2f) && r2 >= T(p.rmin2f))) return -1;
    int kk = (int)(((float)r2 - p.tab_lo) * p.tab_inv);
    kk = kk < 0 ? 0 : (kk >= kTab ? kTab - 1 : kk);
    const int code = tab[kk + 1];
    if (kFP32 && (code & 64)) *flagged = true;
    return bin_refine<D, T>(p, g, s_edge, s_edge2, cc, packed, xj, pk, r2, code, exact_out);
}

// ceil(a / b) for 0 <= a < 2^20, 1 <= b < 2^20, without an integer division: the FP32
// quotient is within one of the true one and is corrected with exact integer products.
__device__ __forceinline__ int ceil_div_small(int a, int b)
{
    int q = (int)((float)a * __frcp_rn((float)b));
    q -= (q * b > a) ? 1 : 0;
    q += ((q + 1) * b <= a) ? 1 : 0;
    return q + ((q * b < a) ? 1 : 0);
}

// The 2-sphere (Sec. "Cosmic Microwave Background"): the bin of the pair (original input j, sorted
// slot k) decided as the FP64 definition decides it -- both directions normalised from the
// caller's coordinates (sqrt of the squares summed in axis order, then a division), cos theta
// summed in axis order, half-open bins [c_b, c_{b+1}) held in edge2; identical directions have no
// azimuth and are no pair (as r = 0 in a box).  Returns -1 outside.  For a pair in a bin it also
// gives the tangent vector n_k - cos(theta) n_j in FP64, projected on the frame (e1, e2) -- the
// direction of the pairs so close that the FP32 chord loses it.
template <typename T>
__device__ __forceinline__ void unit3_fp64(const T* x, double* u)
{
    const double x0 = (double)x[0], x1 = (double)x[1], x2 = (double)x[2];
    const double r = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(x0, x0), __dmul_rn(x1, x1)), __dmul_rn(x2, x2)));
    u[0] = __ddiv_rn(x0, r);
    u[1] = __ddiv_rn(x1, r);
    u[2] = __ddiv_rn(x2, r);
}

template <typename T>
__device__ __forceinline__ int bin_refine_sph(const PairParams& p, int jorig, int kslot, const T* e1, const T* e2,
                                              T* d0, T* d1)
{
    const T* o = static_cast<const T*>(p.orig);
    double uk[3], uj[3];
    unit3_fp64<T>(o + 3 * (size_t)p.perm[kslot], uk);
    unit3_fp64<T>(o + 3 * (size_t)jorig, uj);
    if (uk[0] == uj[0] && uk[1] == uj[1] && uk[2] == uj[2]) return -1;
    const double c = __dadd_rn(__dadd_rn(__dmul_rn(uk[0], uj[0]), __dmul_rn(uk[1], uj[1])), __dmul_rn(uk[2], uj[2]));
    if (!(c >= p.edge2[0])) return -1;
    int b = -1;
    for (int e = 0; e < p.nbins; ++e)
        if (c < p.edge2[e + 1]) {
            b = e;
            break;
        }
    if (b >= 0) {
        double t[3];
        for (int a = 0; a < 3; ++a) t[a] = uk[a] - c * uj[a];
        *d0 = (T)(t[0] * (double)e1[0] + t[1] * (double)e1[1] + t[2] * (double)e1[2]);
        *d1 = (T)(t[0] * (double)e2[0] + t[1] * (double)e2[1] + t[2] * (double)e2[2]);
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

// One batch of a warp's accepted pairs: sort by bin, share the lanes out, accumulate, merge.
// recs/bins hold nbuf entries; acc_s[nbins][NQ] receives the sums of w Y* and w2_s[nbins] those
// of w^2 (the coincident-secondary terms that the remove_self option subtracts); acc is the
// lane's register accumulator (zero on entry and on exit).  hist, cursor, segf, segn, segbin:
// 32 ints each.
template <int D, int LMAX, typename T>
__device__ __forceinline__ void pair_batch_flush(Rec<D, T>* recs, const unsigned char* bins, unsigned short* idx,
                                                 T* acc_s, T* w2_s, int* hist, int* cursor, int* seg, int nbuf,
                                                 int nbins, unsigned& nrounds)
{
    constexpr int NQ = PairCfg<D, LMAX, T>::NQ;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    int* segf = seg;        // first lane of bin b's segment
    int* segn = seg + 32;   // its lanes (0: the bin has no pair in this batch)
    int* segbin = hist;     // reused after the histogram: bin of the k-th segment
    // 1. histogram of the batch's bins
    hist[lane] = 0;
    __syncwarp();
    for (int i = lane; i < nbuf; i += 32) atomicAdd(&hist[bins[i]], 1);
    __syncwarp();
    const int cnt = lane < nbins ? hist[lane] : 0;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += v;
    }
    const int start = incl - cnt;
    // 2. rounds R: the fewest with sum_b ceil(n_b / R) <= 32 lanes.  R = ceil(nbuf / 32) is a lower
    // bound and ceil(nbuf / (32 - nonempty bins)) satisfies it (sum ceil <= nbuf / R + nonempty);
    // bisect between them
    const int nne = __popc(__ballot_sync(full, cnt > 0));
    int R = (nbuf + 31) >> 5;
    int Rhi = nne < 32 ? ceil_div_small(nbuf, 32 - nne) : nbuf;
    while (R < Rhi) {
        const int mid = (R + Rhi) >> 1;
        if (__reduce_add_sync(full, ceil_div_small(cnt, mid)) <= 32) Rhi = mid;
        else R = mid + 1;
    }
    const int nl = ceil_div_small(cnt, R);
    nrounds += (unsigned)R;
    int ninc = nl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(full, ninc, o);
        if (lane >= o) ninc += v;
    }
    const int first = ninc - nl;
    const unsigned E = __ballot_sync(full, nl > 0);
    __syncwarp();
    segf[lane] = first;
    segn[lane] = nl;
    if (nl > 0) segbin[__popc(E & lt_mask)] = lane;
    cursor[lane] = start;
    // 3. this lane's segment: the one that starts at or below it
    const unsigned S = __reduce_or_sync(full, nl > 0 ? (1u << (first & 31)) : 0u);
    const unsigned below = S & (0xffffffffu >> (31 - lane));
    const int s0 = 31 - __clz(below);
    __syncwarp();
    const int my_bin = segbin[__popc(S & ((1u << s0) - 1u))];
    const int my_rank = lane - s0;
    const int my_nl = __shfl_sync(full, nl, my_bin);
    const int my_start = __shfl_sync(full, start, my_bin);
    const int my_cnt = __shfl_sync(full, cnt, my_bin);
    // 4. indices sorted by bin, arrival order kept within a bin
    for (int i0 = 0; i0 < nbuf; i0 += 32) {
        const int i = i0 + lane;
        const bool v = i < nbuf;
        const int b = v ? (int)bins[i] : 64 + lane;
        const unsigned peers = __match_any_sync(full, b);
        const int rank = __popc(peers & lt_mask);
        const int base = v ? cursor[b] : 0;
        __syncwarp();
        if (v) {
            idx[base + rank] = (unsigned short)i;
            if (rank == 0) cursor[b] = base + __popc(peers);
        }
        __syncwarp();
    }
    // 5. every lane accumulates the pairs of its bin, lanes of one bin taking every my_nl-th
    // (the next record is loaded before the current one is accumulated; the index is clamped into
    // the batch, so the extra load at the end is harmless)
    // 6 (first half). The lanes' sums go through the record space (32 x (NQ + 1) scratch), so each
    // lane's accumulators live only inside this function.
    T w2 = T(0);
    T* scr = reinterpret_cast<T*>(recs);
    if constexpr (D == 2 && sizeof(T) == 4) {
        // FP32 D = 2: the complex powers accumulated as packed pairs
        float acc0 = 0.f;
        float2 accC[LMAX > 0 ? LMAX : 1];
#pragma unroll
        for (int c = 0; c < LMAX; ++c) accC[c] = make_float2(0.f, 0.f);
        if (my_rank < my_nl && my_rank < my_cnt) {
            const int last = nbuf - 1;
            Rec<D, T> e = recs[idx[my_start + my_rank]];
            for (int k = my_rank; k < my_cnt; k += my_nl) {
                const Rec<D, T> en = recs[idx[min(my_start + k + my_nl, last)]];
                accum_d2_x2<LMAX>(acc0, accC, e.x(0), e.x(1), e.w());
                w2 = fma(e.w(), e.w(), w2);
                e = en;
            }
        }
        __syncwarp();
        scr[lane * (NQ + 1)] = acc0;
#pragma unroll
        for (int l = 1; l <= LMAX; ++l) {
            scr[lane * (NQ + 1) + q_index_d2(l)] = accC[l - 1].x;
            scr[lane * (NQ + 1) + q_index_d2(l) + 1] = accC[l - 1].y;
        }
    } else if constexpr (D == 3 && sizeof(T) == 4) {
        // FP32 D = 3: the complex columns accumulated as packed pairs
        constexpr int NC = LMAX * (LMAX + 1) / 2;
        float accR[LMAX + 1];
        float2 accC[NC > 0 ? NC : 1];
#pragma unroll
        for (int l = 0; l <= LMAX; ++l) accR[l] = 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c) accC[c] = make_float2(0.f, 0.f);
        if (my_rank < my_nl && my_rank < my_cnt) {
            const int last = nbuf - 1;
            Rec<D, T> e = recs[idx[my_start + my_rank]];
            for (int k = my_rank; k < my_cnt; k += my_nl) {
                const Rec<D, T> en = recs[idx[min(my_start + k + my_nl, last)]];
                accum_d3_x2<LMAX>(accR, accC, e.x(0), e.x(1), e.x(2), e.w());
                w2 = fma(e.w(), e.w(), w2);
                e = en;
            }
        }
        __syncwarp();
        static_for<0, LMAX + 1>([&](auto L) {
            constexpr int l = decltype(L)::value;
            scr[lane * (NQ + 1) + q_index_d3(l, 0)] = accR[l];
            static_for<1, l + 1>([&](auto M) {
                constexpr int m = decltype(M)::value;
                scr[lane * (NQ + 1) + q_index_d3(l, m)] = accC[d3_cidx(l, m)].x;
                scr[lane * (NQ + 1) + q_index_d3(l, m) + 1] = accC[d3_cidx(l, m)].y;
            });
        });
    } else {
        T acc[NQ];
#pragma unroll
        for (int q = 0; q < NQ; ++q) acc[q] = T(0);
        if (my_rank < my_nl && my_rank < my_cnt) {
            const int last = nbuf - 1;
            Rec<D, T> e = recs[idx[my_start + my_rank]];
            for (int k = my_rank; k < my_cnt; k += my_nl) {
                const Rec<D, T> en = recs[idx[min(my_start + k + my_nl, last)]];
                if constexpr (D == 2) accum_d2<LMAX, T>(acc, e.x(0), e.x(1), e.w());
                else if constexpr (D == 3) accum_d3<LMAX, T>(acc, e.x(0), e.x(1), e.x(2), e.w());
                else accum_d4<LMAX, T>(acc, e.x(0), e.x(1), e.x(2), e.x(3), e.w());
                w2 = fma(e.w(), e.w(), w2);
                e = en;
            }
        }
        __syncwarp();
#pragma unroll
        for (int q = 0; q < NQ; ++q) scr[lane * (NQ + 1) + q] = acc[q];
    }
    scr[lane * (NQ + 1) + NQ] = w2;
    __syncwarp();
    // 6 (second half). Merge into acc_s (segments in lane order): components 0..31 go lane =
    // component over the bins in turn (the segment length is the same for the whole warp); the
    // last NQ - 32 components and the w^2 sums are shared out over (bin, component).
    constexpr int QA = NQ < 32 ? NQ : 32;  // components merged lane-parallel
    constexpr int QB = NQ + 1 - QA;         // the rest (w^2 last)
    // two bins per step, so that their dependent shared-memory sums overlap (each bin's sum keeps
    // its lane order)
    unsigned bm = E;                        // bins with a segment
    while (bm) {
        const int b0 = __ffs(bm) - 1;
        bm &= bm - 1;
        const int b1 = bm ? __ffs(bm) - 1 : b0;
        const bool two = bm != 0;
        bm &= bm - 1;
        const int f0 = __shfl_sync(full, first, b0), n0 = __shfl_sync(full, nl, b0);
        const int f1 = __shfl_sync(full, first, b1), n1 = two ? __shfl_sync(full, nl, b1) : 0;
        if (lane < QA) {
            const T* c0 = scr + f0 * (NQ + 1) + lane;
            const T* c1 = scr + f1 * (NQ + 1) + lane;
            T s0 = c0[0], s1 = c1[0];
            const int nmax = n0 > n1 ? n0 : n1;
            for (int l = 1; l < nmax; ++l) {
                if (l < n0) s0 += c0[l * (NQ + 1)];
                if (l < n1) s1 += c1[l * (NQ + 1)];
            }
            acc_s[b0 * NQ + lane] += s0;
            if (two) acc_s[b1 * NQ + lane] += s1;
        }
    }
    for (int o = lane; o < nbins * QB; o += 32) {
        const int b = o / QB, q = QA + (o - b * QB);
        const int f = segf[b], n = segn[b];
        T sum = T(0);
        for (int l = 0; l < n; ++l) sum += scr[(f + l) * (NQ + 1) + q];
        if (q < NQ) acc_s[b * NQ + q] += sum;
        else w2_s[b] += sum;
    }
    __syncwarp();
}

// SPH: points on the unit 2-sphere, stored as n + 1 (a cube [0, 2] of 3-vectors for the cell
// search); the separation is the chord, binned through the table on its square, and the
// direction handed to the D = 2 harmonics is the tangent vector's azimuth in the primary's frame.
template <int D, int LMAX, typename T, bool SPH = false>
__global__ void __launch_bounds__(PairCfg<D, LMAX, T>::kThreads, 1) k_pairs(const PairParams p)
{
    static_assert(!SPH || D == 2, "the 2-sphere uses the D = 2 basis");
    constexpr int DP = SPH ? 3 : D;  // components of a position
    using R = Rec<D, T>;              // a staged pair
    using RP = Rec<DP, T>;            // a sorted particle
    constexpr int NQ = PairCfg<D, LMAX, T>::NQ;
    constexpr bool kFP32 = sizeof(T) == 4;
    const int kB = p.batch;
    const unsigned full = 0xffffffffu;

    extern __shared__ __align__(16) unsigned char smem[];
    const int nthreads = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int nbins = p.nbins;
    unsigned char* tab = smem;                                          // guarded table (kTabBytes)
    float* s_edge = reinterpret_cast<float*>(tab + kTabBytes);          // nbins + 1
    double* s_edge2 = reinterpret_cast<double*>(tab + kTabBytes + 192);  // nbins + 1
    int* job_a = reinterpret_cast<int*>(tab + kTabBytes + 576);  // kMaxJobs: first slot of the cell
    int* job_pk = job_a + kMaxJobs;                          // kMaxJobs: packed stencil offset
    int* job_pre = job_pk + kMaxJobs;                        // kMaxJobs + 1: record prefix
    int* ws = job_pre + kMaxJobs + 4;                        // 68 ints of scan scratch
    CatGeom* s_geo = reinterpret_cast<CatGeom*>(smem + kGeomOffset);
    unsigned char* wbase = smem + pair_fixed_bytes(sizeof(R), nthreads) +
                           warp * pair_warp_bytes(sizeof(R), sizeof(T), nbins, NQ, kB);
    R* recs = reinterpret_cast<R*>(wbase);
    T* acc_s = reinterpret_cast<T*>(wbase + pair_rec_region(sizeof(R), sizeof(T), NQ, kB));
    unsigned char* bins = reinterpret_cast<unsigned char*>(acc_s) + (nbins * NQ * (int)sizeof(T) + 15) / 16 * 16;
    unsigned short* idx = reinterpret_cast<unsigned short*>(bins + kB);
    int* hist = reinterpret_cast<int*>(bins + (3 * kB + 15) / 16 * 16);
    int* cursor = hist + 32;
    int* seg = cursor + 32;  // 64 ints
    T* w2_s = reinterpret_cast<T*>(seg + 64);  // 32

    for (int i = threadIdx.x; i < kTabBytes / 4; i += nthreads)
        reinterpret_cast<int*>(tab)[i] = reinterpret_cast<const int*>(p.tab)[i];
    if (threadIdx.x <= nbins) {
        s_edge[threadIdx.x] = p.edgef[threadIdx.x];
        s_edge2[threadIdx.x] = p.edge2[threadIdx.x];
    }
    const T* qnorm = static_cast<const T*>(p.qnorm);
    const T* inv_vb = static_cast<const T*>(p.inv_vb);
    const RP* rec = static_cast<const RP*>(p.rec);
    const int nq = p.nq;

    // work counters of this warp, added to the statistics once at the end
    unsigned long long ncand = 0, npairs_w = 0;
    unsigned nrounds = 0, nbatch = 0, nchunks = 0, nflag = 0, nexact = 0;

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
        const int nprim_item = it.z & 0xff;

        int cc[DP];
#pragma unroll
        for (int d = 0; d < DP; ++d) cc[d] = ((it.x - g.base) / g.stride[d]) % g.nc[d];

        // the item's stencil rows (runs of cells along axis 0, contiguous in the sorted records):
        // the global index of the row's cell at x = 0 (-1: the row leaves a non-periodic grid), its
        // offsets along the other axes and its x range
        const int nrows = p.nrows;
        for (int r = threadIdx.x; r < nrows; r += nthreads) {
            const int2 rw = p.rows[r];
            int base = g.base;
            bool ok = true;
#pragma unroll
            for (int d = 1; d < DP; ++d) {
                int c = cc[d] + (int)(signed char)((rw.x >> (8 * (d - 1))) & 0xff);
                if (c < 0) {
                    ok = ok && p.periodic;
                    c += g.nc[d];
                } else if (c >= g.nc[d]) {
                    ok = ok && p.periodic;
                    c -= g.nc[d];
                }
                base += c * g.stride[d];
            }
            job_a[r] = ok ? base : -1;
            job_pk[r] = rw.x;
            job_pre[r] = rw.y;
        }
        __syncthreads();

        // warp w takes the item's primary w
        if (warp < nprim_item) {
            const int jslot = it.y + warp;
            const int pidx = it.w + warp;
            const RP pj = rec[jslot];
            T xj[DP];
#pragma unroll
            for (int d = 0; d < DP; ++d) xj[d] = pj.x(d);
            const T wj = pj.w();
            // the sphere: the primary's direction and a right-handed tangent frame (e1, e2, n_j),
            // e1 from the coordinate axis least aligned with n_j (any frame gives the same
            // isotropic coefficients)
            T uj[3], e1[3], e2[3];
            int jorig = 0;
            if constexpr (SPH) {
                jorig = p.perm[jslot];
#pragma unroll
                for (int a = 0; a < 3; ++a) uj[a] = xj[a] - T(1);
                int a0 = 0;
                if (fabs(uj[1]) < fabs(uj[a0])) a0 = 1;
                if (fabs(uj[2]) < fabs(uj[a0])) a0 = 2;
                const T c = uj[a0];
                T nu = T(0);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    e1[a] = (a == a0 ? T(1) : T(0)) - c * uj[a];
                    nu = fma(e1[a], e1[a], nu);
                }
                const T inu = rsqrt_t(nu);
#pragma unroll
                for (int a = 0; a < 3; ++a) e1[a] *= inu;
                e2[0] = uj[1] * e1[2] - uj[2] * e1[1];
                e2[1] = uj[2] * e1[0] - uj[0] * e1[2];
                e2[2] = uj[0] * e1[1] - uj[1] * e1[0];
            }

            for (int i = lane; i < nbins * NQ; i += 32) acc_s[i] = T(0);
            w2_s[lane] = T(0);

            // the stencil rows, each trimmed to the cells this primary can reach: the x range left
            // by the row's distance across the other axes, split where it wraps (at most one wrap,
            // since a row spans at most the grid)
            int nbuf = 0;  // warp-uniform: staged pairs of the current batch
            T side0, box0;
            if constexpr (kFP32) {
                side0 = g.sidef[0];
                box0 = g.boxf[0];
            } else {
                side0 = g.side[0];
                box0 = g.box[0];
            }
            const int nc0 = g.nc[0];
            for (int r = 0; r < nrows; ++r) {
                const int base = job_a[r];
                if (base < 0) continue;
                const int rest = job_pk[r], lohi = job_pre[r];
                T xjs[DP];
                T a2 = T(0);
#pragma unroll
                for (int d = 1; d < DP; ++d) {
                    const int u = cc[d] + (int)(signed char)((rest >> (8 * (d - 1))) & 0xff);
                    T side, box;
                    if constexpr (kFP32) {
                        side = g.sidef[d];
                        box = g.boxf[d];
                    } else {
                        side = g.side[d];
                        box = g.box[d];
                    }
                    const T lo = T(u) * side, hi = lo + side;
                    const T a = fmax(fmax(lo - xj[d], xj[d] - hi), T(0));
                    a2 = fma(a, a, a2);
                    xjs[d] = xj[d] - (u < 0 ? -box : (u >= g.nc[d] ? box : T(0)));
                }
                const T rx2 = T(p.rmax2f) - a2;
                if (!(rx2 >= T(0))) continue;
                const T rx = sqrt(rx2);
                // cells whose x interval meets [x_j - rx, x_j + rx] (a margin of 1e-3 cells)
                int ulo = (int)floor((xj[0] - rx) / side0 - T(1e-3));
                int uhi = (int)floor((xj[0] + rx) / side0 + T(1e-3));
                ulo = max(ulo, cc[0] + (int)(signed char)(lohi & 0xff));
                uhi = min(uhi, cc[0] + (int)(signed char)((lohi >> 8) & 0xff));
                if (!p.periodic) {
                    ulo = max(ulo, 0);
                    uhi = min(uhi, nc0 - 1);
                }
                for (int piece = 0; piece < 3; ++piece) {  // x < 0 (wrapped), inside, x >= nc (wrapped)
                    const int qa = piece == 0 ? ulo : (piece == 1 ? max(ulo, 0) : max(ulo, nc0));
                    const int qb = piece == 0 ? min(uhi, -1) : (piece == 1 ? min(uhi, nc0 - 1) : uhi);
                    if (qa > qb) continue;
                    const int wrap = piece == 0 ? nc0 : (piece == 2 ? -nc0 : 0);
                    const int seg_a = p.cell_start[base + qa + wrap];
                    const int seg_n = p.cell_start[base + qb + wrap + 1] - seg_a;
                    if (seg_n <= 0) continue;
                    // the run's image shift is that of its first cell (offset qa - cc[0] along x)
                    const int packed = ((qa - cc[0]) & 0xff) | (rest << 8);
                    xjs[0] = xj[0] - (piece == 0 ? -box0 : (piece == 2 ? box0 : T(0)));
                    ncand += seg_n;
                    nchunks += (unsigned)((seg_n + 31) >> 5);
                    // candidates in chunks of 32, two chunks per trip; each buffer is refilled two
                    // chunks ahead right after it is consumed (the record array is padded, so the
                    // loads past the run's end are harmless and masked)
                    const RP* src = rec + seg_a;
                    RP buf0 = ldg_rec(src, lane);
                    RP buf1 = ldg_rec(src, 32 + lane);
                    auto chunk = [&](const RP& pk, int c0) {
                        const bool valid = c0 + lane < seg_n;
                        T dx[DP];
                        T r2 = T(0);
#pragma unroll
                        for (int d = 0; d < DP; ++d) {
                            if constexpr (kFP32) dx[d] = pk.x(d) - xjs[d];
                            else dx[d] = (pk.x(d) - xj[d]) + (xj[d] - xjs[d]);
                            r2 = fma(dx[d], dx[d], r2);
                        }
                        int bin;
                        bool refined = false;  // the sphere: direction from the FP64 path
                        T rd0 = T(0), rd1 = T(0);
                        if constexpr (SPH) {
                            // the table on the squared chord (2 - 2 cos theta); flagged buckets (FP32)
                            // or every candidate inside the table (FP64 plans) decided in FP64
                            int kk = __float2int_rd(((float)r2 - p.tab_lo) * p.tab_inv);
                            kk = max(-1, min(kk, kTab));
                            const int code = valid ? (int)tab[kk + 1] : 63;
                            bin = code & 63;
                            const bool flg = kFP32 ? (code & 64) != 0 : code != 63;
                            if (__any_sync(full, flg)) {
                                if (flg) {
                                    ++nflag;
                                    // FP32 plans: the squared chord against the edges' (2 - 2 c_e); only a
                                    // pair within tol of one (above the FP32 error of both) goes to FP64
                                    bool nearE = !kFP32;
                                    int bb = 0;
                                    if constexpr (kFP32) {
                                        for (int e = 0; e <= nbins; ++e) {
                                            const float se = 2.f - 2.f * s_edge[e];
                                            bb += se >= (float)r2 ? 1 : 0;
                                            nearE = nearE || fabsf((float)r2 - se) < p.tol;
                                        }
                                    }
                                    if (nearE) {
                                        const int b = bin_refine_sph<T>(p, jorig, seg_a + c0 + lane, e1, e2, &rd0,
                                                                        &rd1);
                                        bin = b < 0 ? 63 : b;
                                        refined = true;
                                        ++nexact;
                                    } else {
                                        bin = (bb >= 1 && bb <= nbins) ? bb - 1 : 63;
                                    }
                                }
                            }
                        } else if constexpr (kFP32) {
                            // table lookup on the FP32 r^2 (floor; the guards at -1 and kTab catch r^2
                            // outside the table), then the warp-uniform refinement of flagged buckets
                            int kk = __float2int_rd(((float)r2 - p.tab_lo) * p.tab_inv);
                            kk = max(-1, min(kk, kTab));
                            const int code = valid ? (int)tab[kk + 1] : 63;
                            bin = code & 63;
                            const bool flg = (code & 64) != 0;
                            if (__any_sync(full, flg)) {
                                if (flg) {
                                    bool ex = false;
                                    const int b = bin_refine<D, T>(p, g, s_edge, s_edge2, cc, packed, xj, pk, r2,
                                                                   code, &ex);
                                    bin = b < 0 ? 63 : b;
                                    ++nflag;
                                    nexact += ex ? 1u : 0u;
                                }
                            }
                        } else {
                            bool flagged = false, exact = false;
                            const int b = valid ? decide_bin<D, T>(p, g, tab, s_edge, s_edge2, cc, packed, xj, pk,
                                                                   r2, &flagged, &exact)
                                                : -1;
                            bin = b < 0 ? 63 : b;
                            nexact += exact ? 1u : 0u;
                        }
                        // compact the accepted pairs into the batch: unit separation, weight, bin
                        const bool take = bin != 63;
                        const unsigned tm = __ballot_sync(full, take);
                        if (take) {
                            const int slot = nbuf + __popc(tm & lt_mask);
                            R e;
                            T* f = reinterpret_cast<T*>(e.v);
                            if constexpr (SPH) {
                                // tangent vector n_k - cos(theta) n_j = chord + (chord^2 / 2) n_j
                                const T h = T(0.5) * r2;
                                T t[3];
#pragma unroll
                                for (int a = 0; a < 3; ++a) t[a] = fma(h, uj[a], dx[a]);
                                const T d0 = refined ? rd0 : fma(t[0], e1[0], fma(t[1], e1[1], t[2] * e1[2]));
                                const T d1 = refined ? rd1 : fma(t[0], e2[0], fma(t[1], e2[1], t[2] * e2[2]));
                                const T rinv = rsqrt_t(fma(d0, d0, d1 * d1));
                                f[0] = d0 * rinv;
                                f[1] = d1 * rinv;
                            } else {
                                const T rinv = rsqrt_t(r2);
#pragma unroll
                                for (int d = 0; d < D; ++d) f[d] = dx[d] * rinv;
                            }
                            f[D] = pk.w();
                            recs[slot] = e;
                            bins[slot] = (unsigned char)bin;
                        }
                        nbuf += __popc(tm);
                        npairs_w += __popc(tm);
                    };
                    for (int c0 = 0;; c0 += 64) {
                        if (nbuf > kB - 64) {  // room for the trip's two chunks
                            __syncwarp();
                            pair_batch_flush<D, LMAX, T>(recs, bins, idx, acc_s, w2_s, hist, cursor, seg, nbuf,
                                                         nbins, nrounds);
                            nbuf = 0;
                            ++nbatch;
                        }
                        chunk(buf0, c0);
                        buf0 = ldg_rec(src, c0 + 64 + lane);
                        if (c0 + 32 >= seg_n) break;
                        chunk(buf1, c0 + 32);
                        buf1 = ldg_rec(src, c0 + 96 + lane);
                        if (c0 + 64 >= seg_n) break;
                    }
                }
            }
            if (nbuf > 0) {
                __syncwarp();
                pair_batch_flush<D, LMAX, T>(recs, bins, idx, acc_s, w2_s, hist, cursor, seg, nbuf, nbins,
                                             nrounds);
                ++nbatch;
            }
            // write a^b (normalised)
            __syncwarp();
            T* aout = static_cast<T*>(p.a_out) + (size_t)pidx * nbins * nq;
            for (int i = lane; i < nbins * nq; i += 32) {
                const int b = i / nq, q = i - b * nq;
                aout[i] = acc_s[b * NQ + q] * qnorm[q] * inv_vb[b];
            }
            if (lane == 0) static_cast<T*>(p.w_out)[pidx] = wj;
            if (p.self_out && lane < nbins) static_cast<T*>(p.self_out)[(size_t)pidx * nbins + lane] = w2_s[lane];
            __syncwarp();
        }
    }
    // statistics (the candidate counts are warp-uniform; the flags are per lane)
    nflag = __reduce_add_sync(full, nflag);
    nexact = __reduce_add_sync(full, nexact);
    if (lane == 0) {
        atomicAdd(&p.stats[0], npairs_w);
        atomicAdd(&p.stats[1], ncand);
        atomicAdd(&p.stats[2], (unsigned long long)nrounds);
        atomicAdd(&p.stats[3], npairs_w);
        atomicAdd(&p.stats[4], (unsigned long long)nchunks);
        atomicAdd(&p.stats[5], (unsigned long long)nbatch);
        atomicAdd(&p.stats[6], (unsigned long long)nflag);
        atomicAdd(&p.stats[7], (unsigned long long)nexact);
    }
}

template <int D, int LMAX, typename T, bool SPH = false>
cudaError_t launch_pairs_t(const PairParams& p, int grid, int smem, cudaStream_t s)
{
    auto kern = k_pairs<D, LMAX, T, SPH>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, p.warps * 32, smem, s>>>(p); ++launch_counter();
    return cudaGetLastError();
}

}  // namespace npcf
