// npcf_couple_tc.cu -- the split-precision tensor-core coupling of the D=2
// 4PCF (eq. NPCF-estimator-discrete with the D=2 coupling of the applications
// section: l1 + l2 + l3 = 0), and a self-test of the tensor-core contraction.
//
// For one label set Lambda = (l1, l2), l3 = -(l1 + l2), the coupling summed
// over the primaries j of a span is a matrix product over j:
//     G[(b1, b2)][b3] = sum_j X_j(b1, b2) Y_j(b3),
//     X_j(b1, b2) = w_j a^{b1}_{l1}(y_j) a^{b2}_{l2}(y_j),   Y_j(b3) = a^{b3}_{l3}(y_j),
// all complex.  With K = (j, re/im) it is the real product D = A B^T of
//     A[(b1 b2)][(j, 0)] = Re X,  A[(b1 b2)][(j, 1)] = -Im X,
//     B[(b3, re)][(j, 0)] = Re Y, B[(b3, re)][(j, 1)] = Im Y,
//     B[(b3, im)][(j, 0)] = Im Y, B[(b3, im)][(j, 1)] = -Re Y,
// whose columns (b3, re) and (b3, im) are Re and Im of G (the weight w_j is
// carried by the B operand).  A CTA holds the M = 128 (bin pair) x N (2 nbins,
// rounded up to 16) accumulators of up to 512 / N label sets in tensor memory
// and walks its primaries in chunks: the chunk's a^b_l (l >= 0; negative l by
// conjugation) are laid out primary-fastest in shared memory once, then CUDA
// cores form A and B of one label set after another into a double-buffered
// stage, one thread issues the MMAs, and every `span` chunks the accumulators
// are added into the CTA's FP64 row of partial sums (keys with b3 > b2 only).
//
// Precision: A = Ah + Al and B = Bh + Bl (BF16 or TF32 pairs); the product
// keeps Ah Bh + Ah Bl + Al Bh in FP32 (the dropped Al Bl and the split errors
// are O(2^-16) relative for BF16, O(2^-21) for TF32); spans are summed in FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "npcf_device.cuh"
#include "npcf_internal.h"
#include "npcf_tc.cuh"

namespace npcf {

namespace {

constexpr int kTcThreads = 512;
constexpr int kTcKB = 128;                  // bytes of K per operand row per chunk
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // bounded waits on MMA completion: 2 s
constexpr int kErrTimeout = 4;              // bit in the error word: a bounded wait ran out

__host__ __device__ constexpr int tc_chunk(bool tf32) { return tf32 ? 16 : 32; }  // primaries per chunk
__host__ __device__ constexpr int tc_n(int nbins) { return ((2 * nbins + 15) / 16) * 16; }
// complex stride of one (bin, l) row of the expanded a-values: KP + 2 keeps 16-byte alignment and
// puts consecutive bins 4 banks apart
__host__ __device__ constexpr int tc_apad(bool tf32) { return tc_chunk(tf32) + 2; }

struct TcSmem {
    int a_off, a_bytes, w_off, p_off, x_off, stage_off, stage_bytes, a_tile, b_tile, total;
};

// a_off: two buffers of a chunk's raw a-rows [KP][nb * nq + 1] (padded; the next chunk's rows
// arrive by cp.async while the current one is processed); w_off: two buffers of the weights;
// p_off: the bin pairs (128 int2); x_off: a^b_l (l >= 0) as [nb][L+1][KP + 2] complex; then two
// stages of (A hi, A lo, B hi, B lo).
__host__ __device__ inline TcSmem tc_layout(int nbins, int nq, bool tf32)
{
    TcSmem s{};
    const int KP = tc_chunk(tf32), N = tc_n(nbins), L1 = (nq + 1) / 2;
    int off = 64;  // mbarriers, TMEM slot, flags
    s.a_off = off;
    s.a_bytes = ((KP * (nbins * nq + 1) * 4 + 15) / 16) * 16;
    off += 2 * s.a_bytes;
    s.w_off = off;
    off += 2 * ((KP * 4 + 15) / 16) * 16;
    s.p_off = off;
    off += 128 * 8;
    s.x_off = off;
    off += nbins * L1 * tc_apad(tf32) * 8;
    off = ((off + 127) / 128) * 128;
    s.stage_off = off;
    s.a_tile = 128 * kTcKB;
    s.b_tile = N * kTcKB;
    s.stage_bytes = 2 * s.a_tile + 2 * s.b_tile;
    off += 2 * s.stage_bytes;
    s.total = off;
    return s;
}

__device__ __forceinline__ float2 cmul(float2 u, float2 v)
{
    return make_float2(fmaf(u.x, v.x, -u.y * v.y), fmaf(u.x, v.y, u.y * v.x));
}

// Store four K-consecutive complex values (x0..x3 for four primaries) of one operand row as
// (v.x, s * v.y) pairs, split into hi and lo tiles.
template <bool TF32>
__device__ __forceinline__ void store_quad(unsigned char* hi, unsigned char* lo, int row, int quad, const float2* x,
                                           float s)
{
    if constexpr (TF32) {
        uint32_t h[8], l[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            tc::split_tf32(x[i].x, h[2 * i], l[2 * i]);
            tc::split_tf32(s * x[i].y, h[2 * i + 1], l[2 * i + 1]);
        }
        const uint32_t o0 = tc::tile_offset(row, quad * 32, kTcKB), o1 = tc::tile_offset(row, quad * 32 + 16, kTcKB);
        *reinterpret_cast<uint4*>(hi + o0) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(hi + o1) = make_uint4(h[4], h[5], h[6], h[7]);
        *reinterpret_cast<uint4*>(lo + o0) = make_uint4(l[0], l[1], l[2], l[3]);
        *reinterpret_cast<uint4*>(lo + o1) = make_uint4(l[4], l[5], l[6], l[7]);
    } else {
        uint32_t h[4], l[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) tc::split_bf16x2(x[i].x, s * x[i].y, h[i], l[i]);
        const uint32_t o = tc::tile_offset(row, quad * 16, kTcKB);
        *reinterpret_cast<uint4*>(hi + o) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(lo + o) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

// Three MMAs per K step (hi hi, hi lo, lo hi) over the chunk's 128 bytes of K.
template <bool TF32>
__device__ __forceinline__ void issue_split(uint32_t tmem, const unsigned char* ah, const unsigned char* al,
                                            const unsigned char* bh, const unsigned char* bl, uint32_t id,
                                            bool fresh)
{
    constexpr uint32_t sbo = (kTcKB / 16) * 128;
#pragma unroll
    for (int ks = 0; ks < kTcKB / 32; ++ks) {
        const uint64_t dah = tc::sdesc(tc::smem_u32(ah) + 256 * ks, 128, sbo);
        const uint64_t dal = tc::sdesc(tc::smem_u32(al) + 256 * ks, 128, sbo);
        const uint64_t dbh = tc::sdesc(tc::smem_u32(bh) + 256 * ks, 128, sbo);
        const uint64_t dbl = tc::sdesc(tc::smem_u32(bl) + 256 * ks, 128, sbo);
        tc::mma<TF32>(tmem, dah, dbh, id, (fresh && ks == 0) ? 0u : 1u);
        tc::mma<TF32>(tmem, dah, dbl, id, 1u);
        tc::mma<TF32>(tmem, dal, dbh, id, 1u);
    }
}

// grid: (rows, label-set groups, catalogues); one CTA per SM (shared memory and 512 TMEM columns)
template <bool TF32>
__global__ void __launch_bounds__(kTcThreads, 1) k_couple_d2n4_tc(const CoupleParams p)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int nb = p.nbins, nq = p.nq;
    constexpr int KP = tc_chunk(TF32);
    const int NN = tc_n(nb);
    const TcSmem lay = tc_layout(nb, nq, TF32);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);  // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 16);
    int* s_ok = reinterpret_cast<int*>(smem + 20);
    const int L1 = (nq + 1) / 2;  // l = 0..lmax
    const int astr = nb * nq + 1;   // padded raw a-row: the expansion below reads without bank conflicts
    constexpr int AP = tc_apad(TF32);
    int2* Ps = reinterpret_cast<int2*>(smem + lay.p_off);             // [128] bin pairs
    float2* AX = reinterpret_cast<float2*>(smem + lay.x_off);         // [nb][L1][AP]: a^b_l
    unsigned char* stage0 = smem + lay.stage_off;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int npair = p.tc_npairs;
    const int G = p.tc_glam;
    const int lam0 = blockIdx.y * G;
    const int nlg = min(G, p.nlam - lam0);
    const uint32_t id = tc::idesc(TF32, 128, NN);
    const uint32_t ncols = p.tc_tmem_cols;

    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_fence_init();
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, ncols);
    for (int r = tid; r < 128; r += kTcThreads) Ps[r] = r < npair ? p.pairs[r] : make_int2(0, 0);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    const int cat = blockIdx.z;
    const int nprim = p.cat_count ? p.cat_count[cat] : *p.nprim;
    const size_t first = p.cat_first ? (size_t)p.cat_first[cat] : 0;
    const int stride = nb * nq;
    const float* aglob = static_cast<const float*>(p.a) + first * stride;
    const float* wglob = static_cast<const float*>(p.wprim) + first;
    double* prow = p.partial + ((size_t)cat * gridDim.x + blockIdx.x) * 2 * p.ncoeff;
    const int nchunk = (nprim + KP - 1) / KP;

    // a chunk's raw a-rows and weights, copied asynchronously (zero-filled past the last primary)
    auto fetch = [&](int ch, int buf) {
        float* As = reinterpret_cast<float*>(smem + lay.a_off + buf * lay.a_bytes);
        float* Ws = reinterpret_cast<float*>(smem + lay.w_off) + buf * ((KP + 3) / 4 * 4);
        const int p0 = ch * KP, pn = min(KP, nprim - p0);
        const float* src = aglob + (size_t)p0 * stride;
        for (int j = warp; j < KP; j += kTcThreads / 32)
            for (int r = lane; r < stride; r += 32)
                tc::cp_async4(As + j * astr + r, j < pn ? src + (size_t)j * stride + r : aglob, j < pn);
        for (int i = tid; i < KP; i += kTcThreads) tc::cp_async4(Ws + i, i < pn ? wglob + p0 + i : wglob, i < pn);
        tc::cp_async_commit();
    };
    uint32_t committed[2] = {0u, 0u}, waited[2] = {0u, 0u};
    int it = 0, span_pos = 0, cb = 0;
    bool aborted = false;
    if (blockIdx.x < nchunk) fetch(blockIdx.x, 0);
    for (int ch = blockIdx.x; ch < nchunk && !aborted; ch += gridDim.x, cb ^= 1) {
        // the next chunk's rows go to the other buffer (read by the last expansion, long done)
        if (ch + (int)gridDim.x < nchunk) {
            fetch(ch + gridDim.x, cb ^ 1);
            tc::cp_async_wait<1>();
        } else {
            tc::cp_async_wait<0>();
        }
        __syncthreads();  // this chunk's rows are in; (also: the previous chunk's operands are formed)
        const float* As = reinterpret_cast<const float*>(smem + lay.a_off + cb * lay.a_bytes);
        const float* Ws = reinterpret_cast<const float*>(smem + lay.w_off) + cb * ((KP + 3) / 4 * 4);
        // primary-fastest complex a^b_l, l >= 0 (Re a_0; Re, Im of a_l): lanes walk the primaries
        // (32 / KP rows of (b, l) per warp step)
        for (int bl0 = warp * (32 / KP); bl0 < nb * L1; bl0 += (kTcThreads / 32) * (32 / KP)) {
            const int bl = bl0 + lane / KP, j = lane % KP;
            if (bl >= nb * L1) continue;
            const int b = bl / L1, l = bl - b * L1;
            const float* ab = As + j * astr + b * nq;
            AX[bl * AP + j] = l == 0 ? make_float2(ab[0], 0.f) : make_float2(ab[2 * l - 1], ab[2 * l]);
        }
        const bool fresh = span_pos == 0;
        for (int g = 0; g < nlg; ++g, ++it) {
            const int s = it & 1;
            unsigned char* ah = stage0 + s * lay.stage_bytes;
            unsigned char* al = ah + lay.a_tile;
            unsigned char* bh = al + lay.a_tile;
            unsigned char* bl = bh + lay.b_tile;
            if (tid == 0 && waited[s] < committed[s]) {
                // the MMAs that last read this stage must be done before it is overwritten
                if (!tc::mbar_wait_bounded(&mbar[s], waited[s] & 1u, kWaitLimitNs)) *s_ok = 0;
            }
            if (waited[s] < committed[s]) waited[s]++;
            __syncthreads();  // the stage is free; (first label set) the expansion is complete
            if (!*s_ok) {
                aborted = true;
                break;
            }
            const int2 ll = p.lam2[lam0 + g];
            const int l1 = ll.x, l2 = ll.y, l3 = -(l1 + l2);
            // a_{-l} = conj(a_l): the imaginary parts of V (l2 < 0) and Y (l3 < 0) change sign
            const float s2 = l2 < 0 ? -1.f : 1.f, s3 = l3 < 0 ? -1.f : 1.f;
            const int al2 = l2 < 0 ? -l2 : l2, al3 = l3 < 0 ? -l3 : l3;
            // A: 128 rows (bin pairs; rows past the pair list are zero) x KP primaries, four per task
            for (int t = tid; t < 128 * (KP / 4); t += kTcThreads) {
                const int r = t & 127, quad = t >> 7;
                float2 x[4];
                if (r < npair) {
                    const int2 bb = Ps[r];
                    const float4* u = reinterpret_cast<const float4*>(AX + (bb.x * L1 + l1) * AP + quad * 4);
                    const float4* v = reinterpret_cast<const float4*>(AX + (bb.y * L1 + al2) * AP + quad * 4);
                    const float4 u01 = u[0], u23 = u[1], v01 = v[0], v23 = v[1];
                    x[0] = cmul(make_float2(u01.x, u01.y), make_float2(v01.x, s2 * v01.y));
                    x[1] = cmul(make_float2(u01.z, u01.w), make_float2(v01.z, s2 * v01.w));
                    x[2] = cmul(make_float2(u23.x, u23.y), make_float2(v23.x, s2 * v23.y));
                    x[3] = cmul(make_float2(u23.z, u23.w), make_float2(v23.z, s2 * v23.w));
                } else {
#pragma unroll
                    for (int i = 0; i < 4; ++i) x[i] = make_float2(0.f, 0.f);
                }
                store_quad<TF32>(ah, al, r, quad, x, -1.f);
            }
            // B: rows (b3, re) = (Re Y, Im Y) and (b3, im) = (Im Y, -Re Y) per primary, Y = w a^{b3}_{l3}
            for (int t = tid; t < NN * (KP / 4); t += kTcThreads) {
                const int quad = t / NN, n = t - quad * NN, b3 = n >> 1;  // NN: a multiple of 16
                float2 x[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float wj = Ws[quad * 4 + i];
                    float2 y = b3 < nb ? AX[(b3 * L1 + al3) * AP + quad * 4 + i] : make_float2(0.f, 0.f);
                    y = make_float2(wj * y.x, s3 * wj * y.y);
                    x[i] = (n & 1) ? make_float2(y.y, y.x) : y;
                }
                store_quad<TF32>(bh, bl, n, quad, x, (n & 1) ? -1.f : 1.f);
            }
            tc::fence_smem_to_async();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                issue_split<TF32>(tmem + (uint32_t)(g * NN), ah, al, bh, bl, id, fresh);
                tc::commit(&mbar[s]);
            }
            committed[s]++;
        }
        if (aborted) break;
        span_pos++;
        const bool last = ch + (int)gridDim.x >= nchunk;
        if (span_pos < p.tc_span && !last) continue;
        span_pos = 0;
        // flush: every MMA done, then the accumulators into the FP64 partial row
        if (tid == 0) {
            for (int s = 0; s < 2; ++s)
                while (waited[s] < committed[s]) {
                    if (!tc::mbar_wait_bounded(&mbar[s], waited[s] & 1u, kWaitLimitNs)) {
                        *s_ok = 0;
                        break;
                    }
                    waited[s]++;
                }
        }
        for (int s = 0; s < 2; ++s) waited[s] = committed[s];
        __syncthreads();
        if (!*s_ok) {
            aborted = true;
            break;
        }
        tc::fence_after_sync();
        {
            const int r = 32 * (warp & 3) + lane;
            const bool rv = r < npair;
            int b2 = 0, key0 = 0;
            if (rv) {
                b2 = Ps[r].y;
                key0 = p.pair_key[r];
            }
            for (int g = warp >> 2; g < nlg; g += kTcThreads / 128) {
                for (int c0 = 0; c0 < NN; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(g * NN + c0), v);
                    if (!rv) continue;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int n = c0 + i, b3 = n >> 1;
                        if (b3 > b2 && b3 < nb) {
                            const int key = key0 + (b3 - b2 - 1) * p.nlam + lam0 + g;
                            prow[2 * key + (n & 1)] += (double)v[i];
                        }
                    }
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    if (aborted && tid == 0) {
        atomicOr(p.err, kErrTimeout);
        // wait (bounded) for what is still in flight before the tensor memory is released
        for (int s = 0; s < 2; ++s)
            while (waited[s] < committed[s]) {
                if (!tc::mbar_wait_bounded(&mbar[s], waited[s] & 1u, kWaitLimitNs)) break;
                waited[s]++;
            }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

// ---------------------------------------------------------------- self-test
// D[128][N] = A[128][K] B[N][K]^T with the split-precision MMAs above: the
// operands are split, staged in the K-major core-matrix layout, multiplied in
// one CTA and read back from tensor memory (K a multiple of 64 BF16 / 32 TF32
// elements, i.e. whole 128-byte chunks; N a multiple of 16, at most 256).
template <bool TF32>
__global__ void __launch_bounds__(128, 1) k_tc_selftest(const float* A, const float* B, float* D, int N, int K,
                                                        int* err)
{
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 16);
    int* s_ok = reinterpret_cast<int*>(smem + 20);
    unsigned char* ah = smem + 128;
    unsigned char* al = ah + 128 * kTcKB;
    unsigned char* bh = al + 128 * kTcKB;
    unsigned char* bl = bh + 256 * kTcKB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int EPC = TF32 ? 32 : 64;  // elements per 128-byte chunk of K
    const uint32_t id = tc::idesc(TF32, 128, N);
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_fence_init();
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    for (int k0 = 0; k0 < K; k0 += EPC) {
        for (int t = tid; t < (128 + N) * (EPC / 2); t += 128) {
            const int row = t / (EPC / 2), kk = 2 * (t % (EPC / 2));
            const bool isA = row < 128;
            const float* src = isA ? A + (size_t)row * K : B + (size_t)(row - 128) * K;
            const float x0 = src[k0 + kk], x1 = src[k0 + kk + 1];
            unsigned char* hi = isA ? ah : bh;
            unsigned char* lo = isA ? al : bl;
            const int r = isA ? row : row - 128;
            if constexpr (TF32) {
                uint32_t h0, l0, h1, l1;
                tc::split_tf32(x0, h0, l0);
                tc::split_tf32(x1, h1, l1);
                *reinterpret_cast<uint2*>(hi + tc::tile_offset(r, kk * 4, kTcKB)) = make_uint2(h0, h1);
                *reinterpret_cast<uint2*>(lo + tc::tile_offset(r, kk * 4, kTcKB)) = make_uint2(l0, l1);
            } else {
                uint32_t h, l;
                tc::split_bf16x2(x0, x1, h, l);
                *reinterpret_cast<uint32_t*>(hi + tc::tile_offset(r, kk * 2, kTcKB)) = h;
                *reinterpret_cast<uint32_t*>(lo + tc::tile_offset(r, kk * 2, kTcKB)) = l;
            }
        }
        tc::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_split<TF32>(tmem, ah, al, bh, bl, id, k0 == 0);
            tc::commit(&mbar[0]);
            if (!tc::mbar_wait_bounded(&mbar[0], phase, kWaitLimitNs)) *s_ok = 0;
        }
        phase ^= 1u;
        __syncthreads();
        if (!*s_ok) break;
    }
    tc::fence_after_sync();
    if (*s_ok) {
        const int r = 32 * warp + lane;
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) D[(size_t)r * N + c0 + i] = v[i];
        }
    } else if (tid == 0) {
        atomicOr(err, kErrTimeout);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace

int couple_tc_smem(int nbins, int nq, int tf32) { return tc_layout(nbins, nq, tf32 != 0).total; }
int couple_tc_n(int nbins) { return tc_n(nbins); }
int couple_tc_chunk(int tf32) { return tc_chunk(tf32 != 0); }

cudaError_t launch_couple_d2n4_tc(const CoupleParams& p, int tf32, int rows, int groups, int smem, cudaStream_t s)
{
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        kern<<<dim3(rows, groups, p.ncat > 1 ? p.ncat : 1), kTcThreads, smem, s>>>(p);
        ++launch_counter();
        return cudaGetLastError();
    };
    return tf32 ? go(k_couple_d2n4_tc<true>) : go(k_couple_d2n4_tc<false>);
}

int tc_selftest_smem() { return 128 + 2 * 128 * kTcKB + 2 * 256 * kTcKB; }

cudaError_t launch_tc_selftest(int tf32, const float* A, const float* B, float* D, int N, int K, int* err,
                               cudaStream_t s)
{
    const int smem = tc_selftest_smem();
    auto go = [&](auto kern) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        kern<<<1, 128, smem, s>>>(A, B, D, N, K, err);
        ++launch_counter();
        return cudaGetLastError();
    };
    return tf32 ? go(k_tc_selftest<true>) : go(k_tc_selftest<false>);
}

}  // namespace npcf
