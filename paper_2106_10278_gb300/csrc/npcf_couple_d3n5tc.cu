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
// its K (kpiece elements).  K goes through shared memory 16 elements at a time in the K-major
// core-matrix layout (six 4 KB operand tiles per stage), copied with 16-byte cp.async from the
// chunk's scratch in L2; four stages, the loads running three stages ahead of the tensor core,
// 97 KB of shared memory and 256 TMEM columns, so two CTAs share an SM (one's loads and
// epilogue overlap the other's MMAs).
// One thread issues the 6 MMAs of a stage (M = 128, N = 128, K = 16 each) and commits them to
// the stage's mbarrier; every wait on an mbarrier is bounded (error bit 2, then the CTA waits for
// its MMAs in flight, frees its tensor memory and returns).  The epilogue reads D1 and D2 back
// and adds every (row, column) that is a key (b2 < b3; its index from the plan's table) into
// the CTA's FP64 partial row (one row per K piece).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "npcf_internal.h"
#include "npcf_tc.cuh"

namespace npcf {

namespace {

constexpr int kThreads = 256;
constexpr int kKs = 16;                             // K elements per stage (one MMA K step)
constexpr int kStages = 4;                          // stages in flight: loads run three ahead of the MMAs
constexpr int kTileBytes = 128 * kKs * 2;           // one operand tile: 128 rows x 16 BF16
constexpr int kStageBytes = 6 * kTileBytes;         // Re hi, Re lo, Im hi, Im lo of X; hi, lo of [Zr; Zi]
constexpr int kHeader = 1024;
constexpr int kSmem = kHeader + kStages * kStageBytes;
constexpr uint64_t kWaitLimitNs = 2000000000ull;    // 2 s
constexpr int kErrTimeout = 4;

__global__ void __launch_bounds__(kThreads, 2) k_d3n5_contract_tc(const D3n5Params q, int npieces)
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

    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem);  // [kStages]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 64);
    int* s_ok = reinterpret_cast<int*>(smem + 68);
    unsigned char* stage0 = smem + kHeader;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int i = 0; i < kStages; ++i) tc::mbar_init(&mbar[i], 1);
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

    // one stage: 6 tiles x 256 16-byte pieces; in each 32-piece group 2 x 8 rows x 2 K chunks (the
    // 8 rows of a core matrix fill all banks; the global side reads 32 contiguous bytes per row).
    // Every call commits one cp.async group, empty past the last stage, so that the group count
    // stays in step with the stage count.
    auto load = [&](int it) {
        if (it < nst) {
            unsigned char* st = stage0 + (it % kStages) * kStageBytes;
            const int kk = k0 + it * kKs;
            for (int i = tid; i < 6 * 256; i += kThreads) {
                const int t = i >> 8, pc = i & 255;
                const int row = (pc >> 4) * 8 + (pc & 7), ch = (pc >> 3) & 1;
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
        }
        tc::cp_async_commit();
    };

    const uint32_t id = tc::idesc(false, 128, 128);
    constexpr uint32_t sbo = (kKs * 2 / 16) * 128;
    int issued = 0, done = 0;  // MMA stages issued / known complete (thread 0)
    bool aborted = false;
    for (int s = 0; s < kStages - 1; ++s) load(s);
    for (int it = 0; it < nst; ++it) {
        const int b = it % kStages;
        tc::cp_async_wait<kStages - 2>();  // this thread's copies of stage `it` have landed
        tc::fence_smem_to_async();
        __syncthreads();                   // everyone's have
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
            issued = it + 1;
            // the buffer the next load refills was read by the previous stage's MMAs
            if (it >= 1) {
                const int pv = it - 1;
                if (tc::mbar_wait_bounded(&mbar[pv % kStages], (uint32_t)(pv / kStages) & 1u, kWaitLimitNs))
                    done = it;
                else
                    *s_ok = 0;
            }
        }
        __syncthreads();
        if (!*s_ok) {
            aborted = true;
            break;
        }
        load(it + kStages - 1);
    }
    if (tid == 0 && issued > done) {  // the last stage's MMAs (in order: all before it too)
        const int pv = issued - 1;
        if (!tc::mbar_wait_bounded(&mbar[pv % kStages], (uint32_t)(pv / kStages) & 1u, kWaitLimitNs)) *s_ok = 0;
        if (!*s_ok) atomicOr(q.err, kErrTimeout);
    }
    tc::cp_async_wait<0>();
    __syncthreads();
    tc::fence_after_sync();
    if (!aborted && *s_ok) {
        // warps w and w + 4 read TMEM lanes 32 (w % 4) ..: rows; columns 0..31 or 32..63 of the tile;
        // the key of every (row, column) comes from the plan's table (-1: b2 >= b3)
        const int wq = warp & 3, half = warp >> 2;
        const int r = 32 * wq + lane;
        const int* tk = q.tc_keys + (size_t)blockIdx.x * 64 * 128 + r;
        double* prow = q.partial + ((size_t)cat * npieces + piece) * 2 * q.ncoeff;
        const uint32_t ta = tmem + ((uint32_t)(32 * wq) << 16);
        for (int cc = 0; cc < 2; ++cc) {
            const int cb = half * 32 + cc * 16;
            float xrzr[16], xrzi[16], xizr[16], xizi[16];
            tc::tmem_ld16(ta + cb, xrzr);
            tc::tmem_ld16(ta + 64 + cb, xrzi);
            tc::tmem_ld16(ta + 128 + cb, xizr);
            tc::tmem_ld16(ta + 192 + cb, xizi);
            int key[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) key[i] = tk[(cb + i) * 128];  // coalesced over the rows
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                if (key[i] < 0) continue;
                prow[2 * key[i]] += (double)(xrzr[i] - xizi[i]);
                prow[2 * key[i] + 1] += (double)(xrzi[i] + xizr[i]);
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
