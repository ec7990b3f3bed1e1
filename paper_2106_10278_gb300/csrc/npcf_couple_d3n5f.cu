// npcf_couple_d3n5f.cu -- the D=3 isotropic 5PCF coupling (eq. D=3-NPCF) factored
// through the intermediate label l12.  The CG chain of eq. Coupling-C,
//     <l1 m1 l2 m2|l12 m12><l12 m12 l3 m3|l4 M><l4 M l4 m4|0 0>,  M = m12 + m3 = -m4,
// splits the sum over (m1, m2, m3, m4) of one primary into
//     zeta^{b1 b2 b3 b4}_{l1 l2 l12 l3 l4} += w_j sum_{m12} X_j(b1 b2; l1 l2 l12; m12) Z_j(b3 b4; l12 l3 l4; m12),
//     X_j = sum_{m1} <l1 m1 l2 m12-m1|l12 m12> a^{b1}_{l1 m1} a^{b2}_{l2, m12-m1},
//     Z_j = sum_{m3} <l12 m12 l3 m3|l4 M><l4 M l4 -M|0 0> a^{b3}_{l3 m3} a^{b4}_{l4, -M}.
// For one l12 the sum over (j, m12) is a matrix product: rows (b1 < b2, l1, l2), columns
// (b3 < b4, l3, l4), K = (m12, primary).  Only blocks with b2 < b3 and l1 + l2 + l3 + l4 even
// are keys, so rows are ordered by (parity, b2) and columns by (parity, b3), and only tiles that
// hold keys are computed.
//
// Per chunk of primaries: k_d3n5_form writes X (times w_j) and Z of each primary into a scratch
// laid out K-contiguous per row (the chunk's X and Z stay in L2 for the contraction), as complex
// T or, for the tensor-core contraction (npcf_couple_d3n5tc.cu), as four BF16 planes;
// k_d3n5_contract runs the tiles on the CUDA cores, a 64 x 64 complex block of one parity per
// CTA with 4 x 4 per thread (rows ty + 16 a, columns tx + 16 b), K staged through shared memory,
// FP32 (or FP64) sums over the CTA's slice of K added into its FP64 partial row.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "npcf_device.cuh"
#include "npcf_internal.h"

namespace npcf {

namespace {

template <typename T>
struct C5 {
    T r, i;
};

constexpr int kFormWarps = 8;
constexpr int kTile = 64;   // rows and columns of a contraction tile
constexpr int kKc = 16;     // K entries per shared-memory stage
constexpr int kConThreads = 256;

// Where one X (or Z) entry of primary jj of the chunk goes.  Within the block of label l12 the
// rows are K = npc (2 l12 + 1) long and K is ordered (m12, primary), so the lanes of a warp
// (consecutive primaries) write consecutive elements.  MODE 0: complex T; MODE 1: four BF16
// planes (Re hi, Re lo, Im hi, Im lo) of the split-precision tensor-core contraction, where
// v = hi + lo with hi = v rounded to BF16 and lo the rounded remainder.
template <typename T, int MODE>
__device__ __forceinline__ void d5_store(void* base, size_t block, size_t plane, size_t at, T re, T im)
{
    if constexpr (MODE == 0) {
        static_cast<C5<T>*>(base)[block + at] = C5<T>{re, im};
    } else {
        __nv_bfloat16* o = static_cast<__nv_bfloat16*>(base) + 4 * block + at;
        const float r = (float)re, i = (float)im;
        const __nv_bfloat16 rh = __float2bfloat16_rn(r), ih = __float2bfloat16_rn(i);
        o[0] = rh;
        o[plane] = __float2bfloat16_rn(r - __bfloat162float(rh));
        o[2 * plane] = ih;
        o[3 * plane] = __float2bfloat16_rn(i - __bfloat162float(ih));
    }
}

// X and Z of PL primaries per CTA (blockIdx.x), primary = lane % PL: their a^b for all signed m
// in shared memory ([bin, state][PL], so the lanes of one term read consecutive words), then the
// CTA's slice (blockIdx.y of gridDim.y) of the X and Z entries, one entry per group of PL lanes,
// its CG terms walked together by those lanes.
template <typename T, int MODE, int PL>
__global__ void __launch_bounds__(kFormWarps * 32) k_d3n5_form(const D3n5Params q, int chunk0, int nchunk_prim)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NSUB = 32 / PL;
    const int nb = q.nbins, S = (q.lmax + 1) * (q.lmax + 1);
    C5<T>* A = reinterpret_cast<C5<T>*>(smem);  // [nb * S][PL]
    const int cat = blockIdx.z;
    const int nprim = q.cat_count ? q.cat_count[cat] : *q.nprim;
    const size_t first = q.cat_first ? (size_t)q.cat_first[cat] : 0;
    const int jj0 = blockIdx.x * PL;
    const int nx = q.ngx * q.np12, nz = q.ngz * q.np34;
    const int per = (nx + nz + gridDim.y - 1) / gridDim.y;
    const int e0 = blockIdx.y * per, e1 = min(nx + nz, e0 + per);  // entries: X then Z
    const T* abase = static_cast<const T*>(q.a);
    // state s = l^2 + l + m -> its stored component q (m >= 0) and the signs of a_{l,-m} =
    // (-1)^m conj(a_{l m}): bit 16 m != 0, bit 17 the real part flips, bit 18 the imaginary part
    __shared__ int s_state[128];
    for (int st = threadIdx.x; st < S; st += blockDim.x) {
        int l = 0;
        while ((l + 1) * (l + 1) <= st) ++l;
        const int m = st - l * l - l, am = m < 0 ? -m : m;
        const bool flip_re = m < 0 && (am & 1), flip_im = m < 0 && !(am & 1);
        s_state[st] = q_index_d3(l, am) | (am > 0 ? 1 << 16 : 0) | (flip_re ? 1 << 17 : 0) | (flip_im ? 1 << 18 : 0);
    }
    __syncthreads();
    // the a^b of the CTA's primaries, primary fastest (conflict-free stores); eight elements per
    // thread and trip, their loads issued before any is used
    constexpr int kU = 8;
    const int ntot = nb * S * PL;
    for (int i0 = threadIdx.x; i0 < ntot; i0 += kU * blockDim.x) {
        T re[kU], im[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = i0 + u * blockDim.x;
            re[u] = im[u] = T(0);
            const int pj = i % PL, bs = i / PL;
            const int jj = jj0 + pj, j = chunk0 + jj;
            if (i < ntot && jj < nchunk_prim && j < nprim) {
                const int b = bs / S, st = s_state[bs - b * S];
                const T* x = abase + (first + j) * (size_t)nb * q.nq + b * q.nq + (st & 0xffff);
                re[u] = x[0];
                if (st & (1 << 16)) im[u] = x[1];
            }
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i >= ntot) break;
            const int bs = i / PL, st = s_state[bs % S];
            A[i] = C5<T>{(st & (1 << 17)) ? -re[u] : re[u], (st & (1 << 18)) ? -im[u] : im[u]};
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pj = lane % PL, sub = lane / PL;
    const int jj = jj0 + pj, j = chunk0 + jj;
    const bool live = jj < nchunk_prim && j < nprim;
    const bool mine = jj < q.npc;  // a column of the scratch (the chunk's last CTA may overhang it)
    const T w = live ? static_cast<const T*>(q.wprim)[first + j] : T(0);
    __syncthreads();
    const T* coef = static_cast<const T*>(q.coef);
    const size_t npc = (size_t)q.npc;
    void* X = MODE == 0 ? (void*)(static_cast<C5<T>*>(q.xs) + (size_t)cat * q.xs_cat)
                        : (void*)(static_cast<__nv_bfloat16*>(q.xs) + (size_t)cat * 4 * q.xs_cat);
    void* Z = MODE == 0 ? (void*)(static_cast<C5<T>*>(q.zs) + (size_t)cat * q.zs_cat)
                        : (void*)(static_cast<__nv_bfloat16*>(q.zs) + (size_t)cat * 4 * q.zs_cat);
    // X entries: (group, bin pair); group = (l12, (l1, l2), m12) with its term list
    for (int e = e0 + warp * NSUB + sub; e < min(e1, nx); e += kFormWarps * NSUB) {
        const int g = e / q.np12, pr = e - g * q.np12;
        const int4 G = q.gx[g];  // term begin, term end, l12, row-in-pair (ix) | m12 index << 16
        const int2 bb = q.p12[pr];
        const C5<T>* u = A + bb.x * S * PL + pj;
        const C5<T>* v = A + bb.y * S * PL + pj;
        T sr = T(0), si = T(0);
        for (int t = G.x; t < G.y; ++t) {
            const int st = q.terms[t];
            const C5<T> x = u[(st & 0xff) * PL], y = v[((st >> 8) & 0xff) * PL];
            const T pr_ = x.r * y.r - x.i * y.i, pi_ = x.r * y.i + x.i * y.r;
            sr = fma(coef[t], pr_, sr);
            si = fma(coef[t], pi_, si);
        }
        const int l12 = G.z, ix = G.w & 0xffff, mi = G.w >> 16, K = 2 * l12 + 1;
        const int row = q.xrow[q.row0[l12] + pr * q.nlx[l12] + ix];  // position in the (parity, b2) order
        if (mine)
            d5_store<T, MODE>(X, (size_t)q.xoff[l12] * npc, (size_t)q.np12 * q.nlx[l12] * K * npc,
                              ((size_t)row * K + mi) * npc + jj, w * sr, w * si);
    }
    for (int e = max(e0, nx) - nx + warp * NSUB + sub; e < e1 - nx; e += kFormWarps * NSUB) {
        const int g = e / q.np34, pr = e - g * q.np34;
        const int4 G = q.gz[g];
        const int2 bb = q.p34[pr];
        const C5<T>* u = A + bb.x * S * PL + pj;
        const C5<T>* v = A + bb.y * S * PL + pj;
        T sr = T(0), si = T(0);
        for (int t = G.x; t < G.y; ++t) {
            const int st = q.terms[t];
            const C5<T> x = u[(st & 0xff) * PL], y = v[((st >> 8) & 0xff) * PL];
            const T pr_ = x.r * y.r - x.i * y.i, pi_ = x.r * y.i + x.i * y.r;
            sr = fma(coef[t], pr_, sr);
            si = fma(coef[t], pi_, si);
        }
        const int l12 = G.z, iz = G.w & 0xffff, mi = G.w >> 16, K = 2 * l12 + 1;
        const int col = q.zcol[q.col0[l12] + pr * q.nlz[l12] + iz];  // position in the (parity, b3) order
        if (mine)
            d5_store<T, MODE>(Z, (size_t)q.zoff[l12] * npc, (size_t)q.np34 * q.nlz[l12] * K * npc,
                              ((size_t)col * K + mi) * npc + jj, sr, si);
    }
}

// One tile (l12, 64 rows, 64 columns) per blockIdx.x, one slice of the chunk's primaries per
// blockIdx.y (its own partial row), catalogue blockIdx.z.
template <typename T>
__global__ void __launch_bounds__(kConThreads) k_d3n5_contract(const D3n5Params q)
{
    __shared__ C5<T> Xs[kKc][kTile + 1];
    __shared__ C5<T> Zs[kKc][kTile + 1];
    const int4 tile = q.tiles[blockIdx.x];  // l12, first row, first column, rows | columns << 16
    const int l12 = tile.x, K1 = 2 * l12 + 1;
    const int nrows = tile.w & 0xffff, ncols = tile.w >> 16;
    // rows and columns of one parity, in (parity, b2) and (parity, b3) order: row r and column c
    // meet in a key when b2 < b3
    const int cat = blockIdx.z;
    const C5<T>* X = static_cast<const C5<T>*>(q.xs) + (size_t)cat * q.xs_cat + (size_t)q.xoff[l12] * q.npc;
    const C5<T>* Z = static_cast<const C5<T>*>(q.zs) + (size_t)cat * q.zs_cat + (size_t)q.zoff[l12] * q.npc;
    // this CTA's slice of K = (m12, primary of the chunk)
    const int Kr = q.npc * K1;
    const int per = (Kr + gridDim.y - 1) / gridDim.y;
    const int k0 = min(Kr, (int)blockIdx.y * per), k1 = min(Kr, k0 + per);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    T ar[4][4], ai[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) ar[a][b] = ai[a][b] = T(0);
    for (int kb = k0; kb < k1; kb += kKc) {
        __syncthreads();
        for (int i = threadIdx.x; i < kKc * kTile; i += kConThreads) {
            const int r = i / kKc, k = i - r * kKc;  // K fastest: coalesced along a row
            const int kk = kb + k;
            const bool ok = kk < k1;
            Xs[k][r] = (ok && r < nrows) ? X[(size_t)(tile.y + r) * q.npc * K1 + kk] : C5<T>{T(0), T(0)};
            Zs[k][r] = (ok && r < ncols) ? Z[(size_t)(tile.z + r) * q.npc * K1 + kk] : C5<T>{T(0), T(0)};
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kKc; ++k) {
            C5<T> x[4], z[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {  // rows ty + 16 a, columns tx + 16 b: conflict-free reads
                x[a] = Xs[k][ty + 16 * a];
                z[a] = Zs[k][tx + 16 * a];
            }
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    ar[a][b] = fma(x[a].r, z[b].r, fma(-x[a].i, z[b].i, ar[a][b]));
                    ai[a][b] = fma(x[a].r, z[b].i, fma(x[a].i, z[b].r, ai[a][b]));
                }
        }
    }
    double* prow = q.partial + ((size_t)cat * gridDim.y + blockIdx.y) * 2 * q.ncoeff;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = ty + 16 * a;
        if (r >= nrows) continue;
        const int4 R = q.rowinfo[q.row0[l12] + tile.y + r];  // b1, b2, parity, l1 | l2 << 8
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = tx + 16 * b;
            if (c >= ncols) continue;
            const int4 C = q.colinfo[q.col0[l12] + tile.z + c];  // b3, b4, parity, l3 | l4 << 8
            if (R.y >= C.x) continue;
            const int L1 = q.lmax + 1;
            const int l1 = R.w & 0xff, l2 = R.w >> 8, l3 = C.w & 0xff, l4 = C.w >> 8;
            const int lam = q.lamidx[(((l1 * L1 + l2) * (2 * L1 - 1) + l12) * L1 + l3) * L1 + l4];
            const int key = q.trikey[(R.x * q.nbins + R.y) * q.nbins + C.x] + (C.y - C.x - 1) * q.nlam + lam;
            prow[2 * key] += (double)ar[a][b];
            prow[2 * key + 1] += (double)ai[a][b];
        }
    }
}

}  // namespace

// Primaries per CTA of the formation kernel (32, 16 or 8: the most whose a-values fit in shared
// memory), or 0 when even 8 do not fit.
int d3n5f_form_lanes(int nbins, int lmax, int fp64, int smem_optin)
{
    for (int pl = 32; pl >= 8; pl /= 2)
        if (d3n5f_form_smem(nbins, lmax, fp64, pl) <= smem_optin) return pl;
    return 0;
}

int d3n5f_form_smem(int nbins, int lmax, int fp64, int lanes)
{
    return nbins * (lmax + 1) * (lmax + 1) * lanes * 2 * (fp64 ? 8 : 4);
}

namespace {

template <typename T, int MODE, int PL>
cudaError_t launch_form(const D3n5Params& q, int nchunk_prim, int chunk0, int ncat, cudaStream_t s)
{
    auto kern = k_d3n5_form<T, MODE, PL>;
    const int fs = d3n5f_form_smem(q.nbins, q.lmax, sizeof(T) == 8, PL);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, fs);
    if (e != cudaSuccess) return e;
    // entry slices: about four CTAs per SM over the chunk's groups of PL primaries
    const int ngrp = (q.npc + PL - 1) / PL;
    const int nent = q.ngx * q.np12 + q.ngz * q.np34;
    const int slices = std::max(1, std::min((4 * q.nsm + ngrp - 1) / ngrp, (nent + 255) / 256));
    kern<<<dim3(ngrp, slices, ncat > 1 ? ncat : 1), kFormWarps * 32, fs, s>>>(q, chunk0, nchunk_prim);
    ++launch_counter();
    return cudaGetLastError();
}

template <typename T, int MODE>
cudaError_t launch_form_pl(const D3n5Params& q, int nchunk_prim, int chunk0, int ncat, cudaStream_t s)
{
    switch (q.form_lanes) {
        case 32: return launch_form<T, MODE, 32>(q, nchunk_prim, chunk0, ncat, s);
        case 16: return launch_form<T, MODE, 16>(q, nchunk_prim, chunk0, ncat, s);
        case 8: return launch_form<T, MODE, 8>(q, nchunk_prim, chunk0, ncat, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

// mode 0: FP32, 1: FP64 (CUDA-core contraction); 2: split BF16 (tensor-core contraction, FP32 inputs)
cudaError_t launch_d3n5f(const D3n5Params& q, int mode, int nchunk_prim, int chunk0, int ksplit, int ncat,
                         cudaStream_t s)
{
    cudaError_t e;
    const dim3 cgrid(q.ntiles, ksplit, ncat > 1 ? ncat : 1);
    if (mode == 1) {
        if ((e = launch_form_pl<double, 0>(q, nchunk_prim, chunk0, ncat, s)) != cudaSuccess) return e;
        k_d3n5_contract<double><<<cgrid, kConThreads, 0, s>>>(q);
    } else if (mode == 0) {
        if ((e = launch_form_pl<float, 0>(q, nchunk_prim, chunk0, ncat, s)) != cudaSuccess) return e;
        k_d3n5_contract<float><<<cgrid, kConThreads, 0, s>>>(q);
    } else {
        if ((e = launch_form_pl<float, 1>(q, nchunk_prim, chunk0, ncat, s)) != cudaSuccess) return e;
        return launch_d3n5_contract_tc(q, ksplit, ncat, s);
    }
    ++launch_counter();
    return cudaGetLastError();
}

}  // namespace npcf
