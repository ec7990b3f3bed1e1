// npcf_couple_d3n5tc.cu -- the contraction of the factored D=3 5PCF coupling (eq. D=3-NPCF
// with the CG chain of eq. Coupling-C split at the intermediate label l12) on the tensor cores,
// in split BF16.
//
// For one l12 and one parity the chunk's contribution is the complex product C = X Z^T over
// K = (m12, primary), rows (b1 < b2, l1, l2) and columns (b3 < b4, l3, l4).  With X = Xr + i Xi,
// Z = Zr + i Zi and the 64 columns of a tile stacked as 128 real operand rows B = [Zr; Zi]:
//     D1 = Xr B^T = [Xr Zr^T | Xr Zi^T],   D2 = Xi B^T = [Xi Zr^T | Xi Zi^T],
//     Re C = D1[:, :64] - D2[:, 64:],      Im C = D1[:, 64:] + D2[:, :64].
// Every operand value is a pair hi + lo of BF16 (the formation kernel writes the four planes
// Re hi, Re lo, Im hi, Im lo); a product keeps hi*hi + hi*lo + lo*hi, accumulated in FP32 in
// tensor memory (D1 and D2: 256 columns).  The dropped lo*lo and the split leave O(2^-16) of each
// product.
//
// A CTA takes one tile (up to 128 rows x 64 columns of one parity that hold keys) and one piece of
// its K (kpiece elements).  K goes through shared memory 64 elements at a time in the K-major
// core-matrix layout (six 16 KB operand tiles per stage), copied with 16-byte cp.async from the
// chunk's scratch in L2; two stages, the next one loading while the tensor core works on the
// current.  One thread issues the 24 MMAs of a stage (M = 128, N = 128, K = 16 each) and commits
// them to the stage's mbarrier; every wait on an mbarrier is bounded (error bit 2, then the CTA
// waits for its MMAs in flight, frees its tensor memory and returns).  The epilogue reads D1 and
// D2 back and adds the keys (b2 < b3) into the CTA's FP64 partial row (one row per K piece).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "npcf_internal.h"
#include "npcf_tc.cuh"

namespace npcf {

namespace {

constexpr int kThreads = 256;
constexpr int kKs = 64;                             // K elements per stage
constexpr int kTileBytes = 128 * kKs * 2;           // one operand tile: 128 rows x 64 BF16
constexpr int kStageBytes = 6 * kTileBytes;         // Re hi, Re lo, Im hi, Im lo of X; hi, lo of [Zr; Zi]
constexpr int kHeader = 1024;
constexpr int kSmem = kHeader + 2 * kStageBytes;
constexpr uint64_t kWaitLimitNs = 2000000000ull;    // 2 s
constexpr int kErrTimeout = 4;

__global__ void __launch_bounds__(kThreads, 1) k_d3n5_contract_tc(const D3n5Params q, int npieces)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const int4 tile = q.tc_tiles[blockIdx.x];
    const int l12 = tile.x, r0 = tile.y, c0 = tile.z, nr = tile.w & 0xffff, nc = tile.w >> 16;
    const int K1 = 2 * l12 + 1;
    const int Kr = q.npc * K1;  // a multiple of 64 (npc is)
    const int piece = blockIdx.y;
    const int k0 = piece * q.kpiece;
    if (k0 >= Kr) return;  // this tile has fewer pieces (uniform over the CTA: before any allocation)
    const int k1 = min(Kr, k0 + q.kpiece);
    const int nst = (k1 - k0) / kKs;

    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 16);
    int* s_ok = reinterpret_cast<int*>(smem + 20);
    unsigned char* stage0 = smem + kHeader;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&mbar[0], 1);
        tc::mbar_init(&mbar[1], 1);
        tc::mbar_fence_init();
        *s_ok = 1;
    }
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    const int cat = blockIdx.z;
    const size_t npc = (size_t)q.npc;
    const __nv_bfloat16* X = static_cast<const __nv_bfloat16*>(q.xs) + (size_t)cat * 4 * q.xs_cat +
                             4 * (size_t)q.xoff[l12] * npc;
    const __nv_bfloat16* Z = static_cast<const __nv_bfloat16*>(q.zs) + (size_t)cat * 4 * q.zs_cat +
                             4 * (size_t)q.zoff[l12] * npc;
    const size_t xplane = (size_t)q.np12 * q.nlx[l12] * Kr, zplane = (size_t)q.np34 * q.nlz[l12] * Kr;

    // 6 x 1024 16-byte pieces per stage: in each 32-piece group, 8 rows x 4 K chunks (the 8 rows
    // of a core matrix fill all banks; the global side reads 64 contiguous bytes per row)
    auto load = [&](int buf, int kk) {
        unsigned char* st = stage0 + buf * kStageBytes;
        for (int i = tid; i < 6 * 1024; i += kThreads) {
            const int t = i >> 10, pc = i & 1023;
            const int rest = pc >> 5;
            const int row = (rest >> 1) * 8 + (pc & 7), ch = (rest & 1) * 4 + ((pc >> 3) & 3);
            unsigned char* dst = st + t * kTileBytes + tc::tile_offset(row, ch * 16, kKs * 2);
            const __nv_bfloat16* src;
            bool valid;
            if (t < 4) {  // X plane t, row r0 + row
                valid = row < nr;
                src = X + t * xplane + (size_t)(r0 + (valid ? row : 0)) * Kr + kk + ch * 8;
            } else {      // [Zr; Zi] hi (t = 4) or lo (t = 5): operand row = part * 64 + column
                const int part = row >> 6, col = row & 63;
                valid = col < nc;
                src = Z + (part * 2 + (t - 4)) * zplane + (size_t)(c0 + (valid ? col : 0)) * Kr + kk + ch * 8;
            }
            tc::cp_async16(dst, src, valid);
        }
        tc::cp_async_commit();
    };

    const uint32_t id = tc::idesc(false, 128, 128);
    constexpr uint32_t sbo = (kKs * 2 / 16) * 128;
    uint32_t committed[2] = {0u, 0u}, waited[2] = {0u, 0u};
    bool aborted = false;
    load(0, k0);
    for (int it = 0; it < nst; ++it) {
        const int b = it & 1;
        tc::cp_async_wait<0>();
        tc::fence_smem_to_async();
        __syncthreads();  // stage `it` is in shared memory
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t base = tc::smem_u32(stage0 + b * kStageBytes);
#pragma unroll
            for (int ks = 0; ks < kKs / 16; ++ks) {
                const uint32_t o = base + 256 * ks;
                const uint64_t xrh = tc::sdesc(o, 128, sbo), xrl = tc::sdesc(o + kTileBytes, 128, sbo);
                const uint64_t xih = tc::sdesc(o + 2 * kTileBytes, 128, sbo);
                const uint64_t xil = tc::sdesc(o + 3 * kTileBytes, 128, sbo);
                const uint64_t bh = tc::sdesc(o + 4 * kTileBytes, 128, sbo);
                const uint64_t bl = tc::sdesc(o + 5 * kTileBytes, 128, sbo);
                const uint32_t acc = (it > 0 || ks > 0) ? 1u : 0u;
                tc::mma<false>(tmem, xrh, bh, id, acc);
                tc::mma<false>(tmem, xrh, bl, id, 1u);
                tc::mma<false>(tmem, xrl, bh, id, 1u);
                tc::mma<false>(tmem + 128, xih, bh, id, acc);
                tc::mma<false>(tmem + 128, xih, bl, id, 1u);
                tc::mma<false>(tmem + 128, xil, bh, id, 1u);
            }
            tc::commit(&mbar[b]);
            // the MMAs of the previous stage read the other buffer: done before it is refilled
            if (waited[b ^ 1] < committed[b ^ 1]) {
                if (tc::mbar_wait_bounded(&mbar[b ^ 1], waited[b ^ 1] & 1u, kWaitLimitNs)) waited[b ^ 1]++;
                else *s_ok = 0;
            }
        }
        committed[b]++;
        __syncthreads();
        if (!*s_ok) {
            aborted = true;
            break;
        }
        if (it + 1 < nst) load(b ^ 1, k0 + (it + 1) * kKs);
    }
    if (tid == 0) {  // every MMA done (after a timeout: bounded, then give up)
        for (int s = 0; s < 2; ++s)
            while (waited[s] < committed[s]) {
                if (!tc::mbar_wait_bounded(&mbar[s], waited[s] & 1u, kWaitLimitNs)) {
                    *s_ok = 0;
                    break;
                }
                waited[s]++;
            }
        if (!*s_ok) atomicOr(q.err, kErrTimeout);
    }
    tc::cp_async_wait<0>();
    __syncthreads();
    tc::fence_after_sync();
    if (!aborted && *s_ok) {
        // warps w and w + 4 read TMEM lanes 32 (w % 4) ..: rows; columns 0..31 or 32..63 of the tile
        const int wq = warp & 3, half = warp >> 2;
        const int r = 32 * wq + lane;
        const bool rv = r < nr;
        int4 R = make_int4(0, 0, 0, 0);
        if (rv) R = q.rowinfo[q.row0[l12] + r0 + r];  // b1, b2, parity, l1 | l2 << 8
        const int L1 = q.lmax + 1;
        const int l1 = R.w & 0xff, l2 = R.w >> 8;
        double* prow = q.partial + ((size_t)cat * npieces + piece) * 2 * q.ncoeff;
        const uint32_t ta = tmem + ((uint32_t)(32 * wq) << 16);
        for (int cc = 0; cc < 2; ++cc) {
            const int cb = half * 32 + cc * 16;
            float xrzr[16], xrzi[16], xizr[16], xizi[16];
            tc::tmem_ld16(ta + cb, xrzr);
            tc::tmem_ld16(ta + 64 + cb, xrzi);
            tc::tmem_ld16(ta + 128 + cb, xizr);
            tc::tmem_ld16(ta + 192 + cb, xizi);
            if (!rv) continue;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = cb + i;
                if (c >= nc) break;
                const int4 C = q.colinfo[q.col0[l12] + c0 + c];  // b3, b4, parity, l3 | l4 << 8
                if (R.y >= C.x) continue;
                const int l3 = C.w & 0xff, l4 = C.w >> 8;
                const int lam = q.lamidx[(((l1 * L1 + l2) * (2 * L1 - 1) + l12) * L1 + l3) * L1 + l4];
                const int key =
                    q.trikey[(R.x * q.nbins + R.y) * q.nbins + C.x] + (C.y - C.x - 1) * q.nlam + lam;
                prow[2 * key] += (double)(xrzr[i] - xizi[i]);
                prow[2 * key + 1] += (double)(xrzi[i] + xizr[i]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

}  // namespace

int d3n5_tc_smem() { return kSmem; }

cudaError_t launch_d3n5_contract_tc(const D3n5Params& q, int npieces, int ncat, cudaStream_t s)
{
    if (q.ntc == 0 || npieces < 1) return cudaSuccess;  // no keys
    cudaError_t e = cudaFuncSetAttribute(k_d3n5_contract_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
    if (e != cudaSuccess) return e;
    k_d3n5_contract_tc<<<dim3(q.ntc, npieces, ncat > 1 ? ncat : 1), kThreads, kSmem, s>>>(q, npieces);
    ++launch_counter();
    return cudaGetLastError();
}

}  // namespace npcf
