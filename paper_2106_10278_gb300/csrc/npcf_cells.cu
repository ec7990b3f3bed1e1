// npcf_cells.cu -- cell-list construction (counting sort of particles by
// cell), the per-cell work items of the pair kernel, a two-level exclusive
// scan and the fixed-order FP64 reduction of the coupling partial sums.
//
// The cell list is not in the paper (its estimator is written as a plain sum
// over all pairs, eq. NPCF-estimator-discrete); it only restricts that sum to
// the secondaries that can lie within r_max of a primary.
#include <cuda_runtime.h>

#include <cstdint>

#include "npcf_device.cuh"
#include "npcf_internal.h"

namespace npcf {

namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;  // elements per thread
constexpr int kScanTile = kScanThreads * kScanPer;

template <typename T>
__global__ void k_cell_ids(const CellParams p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const T* pos = static_cast<const T*>(p.pos) + i * p.D;
    const T w = static_cast<const T*>(p.w)[i];
    int cat = 0;
    if (p.ncat > 1) {  // the catalogue holding particle i: offsets[cat] <= i < offsets[cat + 1]
        int lo = 0, hi = p.ncat;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (p.offsets[mid] <= i) lo = mid;
            else hi = mid;
        }
        cat = lo;
    }
    const CatGeom& g = p.geo[cat];
    int bad = isfinite((double)w) ? 0 : 1;
    int cell = g.base;
    for (int d = 0; d < p.D; ++d) {
        const double x = (double)pos[d];
        if (!isfinite(x)) bad |= 1;
        else if (!(x >= 0.0 && x < g.box[d])) bad |= 2;
        int c = isfinite(x) ? (int)floor(x * g.inv_side[d]) : 0;
        c = c < 0 ? 0 : (c >= g.nc[d] ? g.nc[d] - 1 : c);
        cell += c * g.stride[d];
    }
    if (bad) atomicOr(p.err, bad);
    p.cid[i] = cell;
    atomicAdd(&p.cell_count[cell], 1);
}

// Points on the unit 2-sphere: each 3-vector normalised and shifted by +1 per axis, so that the
// cell search runs in the cube [0, 2]^3 (a zero or non-finite vector gives NaN, which the cell
// stage flags).
template <typename T>
__global__ void k_sphere_prep(const T* pos, int64_t n, T* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T x0 = pos[3 * i], x1 = pos[3 * i + 1], x2 = pos[3 * i + 2];
    const T r2 = (x0 * x0 + x1 * x1) + x2 * x2;
    const T ir = T(1) / sqrt(r2);
    out[3 * i] = x0 * ir + T(1);
    out[3 * i + 1] = x1 * ir + T(1);
    out[3 * i + 2] = x2 * ir + T(1);
}

__global__ void k_cell_scatter(const CellParams p)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const int c = p.cid[i];
    const int slot = p.cell_start[c] + atomicAdd(&p.cell_fill[c], 1);
    p.perm[slot] = (int)i;
}

// Order each cell's slots by original index (the atomic scatter above leaves
// them in arrival order), so that every later sum runs in a fixed order.
// One block per cell; ranks by counting smaller indices.
__global__ void k_cell_order(const CellParams p, int* perm_out)
{
    __shared__ int s_idx[2048];
    const int c = blockIdx.x;
    const int start = p.cell_start[c], end = p.cell_start[c + 1];
    const int m = end - start;
    if (m <= 0) return;
    if (m <= 2048) {
        for (int e = threadIdx.x; e < m; e += blockDim.x) s_idx[e] = p.perm[start + e];
        __syncthreads();
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const int v = s_idx[e];
            int r = 0;
            for (int f = 0; f < m; ++f) r += (s_idx[f] < v) ? 1 : 0;
            perm_out[start + r] = v;
        }
    } else {
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const int v = p.perm[start + e];
            int r = 0;
            for (int f = 0; f < m; ++f) r += (p.perm[start + f] < v) ? 1 : 0;
            perm_out[start + r] = v;
        }
    }
}

template <int D, typename T>
__global__ void k_gather(const CellParams p, const int* perm)
{
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= p.n) return;
    const int i = perm[s];
    const T* pos = static_cast<const T*>(p.pos) + (int64_t)i * D;
    Rec<D, T> r;
    T* f = reinterpret_cast<T*>(r.v);
#pragma unroll
    for (int k = 0; k < 4 * Rec<D, T>::NV; ++k) f[k] = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) f[d] = pos[d];
    f[D] = static_cast<const T*>(p.w)[i];
    static_cast<Rec<D, T>*>(p.rec)[s] = r;
}

// ------------------------------------------------------------------ scan
__global__ void k_scan_tiles(const int* in, int* out, int n, int* tile_sums)
{
    __shared__ int s_warp[32];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    int v[kScanPer];
    int local = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        local += v[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int ws = s_warp[lane];
        int wi = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += t;
        }
        s_warp[lane] = wi - ws;  // exclusive warp offsets
        if (lane == 31 && tile_sums) tile_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    int run = s_warp[warp] + incl - local;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}

__global__ void k_scan_add(int* out, int n, const int* tile_offsets)
{
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    const int add = tile_offsets[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanPer; ++k)
        if (base + k < n) out[base + k] += add;
}

// --------------------------------------------------------- work items
__device__ __forceinline__ int lower_bound_i(const int* a, int lo, int hi, int64_t key)
{
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int64_t)a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Per cell: the slots whose original index lies in [pb, pe) form one
// contiguous run (slots are ordered by original index within a cell).
__global__ void k_cell_select(const int* cell_start, const int* perm, int ncells, int64_t pb, int64_t pe, int warps,
                              int* cell_lo, int* cell_prims, int* cell_items)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int s = cell_start[c], e = cell_start[c + 1];
    const int lo = lower_bound_i(perm, s, e, pb);
    const int hi = lower_bound_i(perm, s, e, pe);
    cell_lo[c] = lo;
    cell_prims[c] = hi - lo;
    cell_items[c] = (hi - lo + warps - 1) / warps;
}

// item = (global cell, first slot, primaries | catalogue << 8, first primary)
__global__ void k_write_items(int ncells, int warps, const int* cell_lo, const int* cell_prims,
                              const int* prim_start, const int* item_start, int ncat, const int* cat_cells,
                              int4* items)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncells) return;
    const int np = cell_prims[c];
    const int lo = cell_lo[c];
    const int pbase = prim_start[c];
    const int ibase = item_start[c];
    int cat = 0;
    if (ncat > 1) {
        int a = 0, b = ncat;
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (cat_cells[mid] <= c) a = mid;
            else b = mid;
        }
        cat = a;
    }
    for (int k = 0; k * warps < np; ++k) {
        const int cnt = min(warps, np - k * warps);
        items[ibase + k] = make_int4(c, lo + k * warps, cnt | (cat << 8), pbase + k * warps);
    }
}

__global__ void k_totals(int ncells, const int* cell_prims, const int* prim_start, const int* cell_items,
                         const int* item_start, int* nprim, int* nitems)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *nprim = ncells > 0 ? prim_start[ncells - 1] + cell_prims[ncells - 1] : 0;
        *nitems = ncells > 0 ? item_start[ncells - 1] + cell_items[ncells - 1] : 0;
    }
}

// out[k] = scale * sum_r partial[r][col(k)], k < nout, rows of ncols; col = colmap (the plan's
// selected keys, e.g. one parity) or the identity
__global__ void k_reduce_rows(const double* partial, int rows, int ncols, const int* colmap, int nout, double scale,
                              double* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nout) return;
    const int col = colmap ? colmap[k] : k;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += partial[(size_t)r * ncols + col];
    out[k] = s * scale;
}

__global__ void k_reduce_cats(const double* partial, int rows, int ncols, const int* colmap, int nout,
                              const double* scales, double* out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nout) return;
    const int c = blockIdx.y;
    const int col = colmap ? colmap[k] : k;
    const double* pc = partial + (size_t)c * rows * ncols;
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s += pc[(size_t)r * ncols + col];
    out[(size_t)c * nout + k] = s * scales[c];
}

inline int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_cell_ids(const CellParams& p, int fp64, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    const int t = 256;
    if (fp64) k_cell_ids<double><<<blocks_for(p.n, t), t, 0, s>>>(p);
    else k_cell_ids<float><<<blocks_for(p.n, t), t, 0, s>>>(p); ++launch_counter();
    return cudaGetLastError();
}

cudaError_t launch_sphere_prep(const void* pos, int64_t n, int fp64, void* out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int t = 256;
    if (fp64) k_sphere_prep<double><<<blocks_for(n, t), t, 0, s>>>(static_cast<const double*>(pos), n, static_cast<double*>(out));
    else k_sphere_prep<float><<<blocks_for(n, t), t, 0, s>>>(static_cast<const float*>(pos), n, static_cast<float*>(out));
    ++launch_counter();
    return cudaGetLastError();
}

cudaError_t launch_cell_scatter(const CellParams& p, int fp64, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    const int t = 256;
    k_cell_scatter<<<blocks_for(p.n, t), t, 0, s>>>(p); ++launch_counter();
    // order each cell's run, writing into cid (free by now) as scratch
    int* ordered = p.cid;
    k_cell_order<<<p.ncells, 256, 0, s>>>(p, ordered); ++launch_counter();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(p.perm, ordered, sizeof(int) * p.n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    const int gb = blocks_for(p.n, t);
    switch (p.D * 2 + (fp64 ? 1 : 0)) {
        case 4: k_gather<2, float><<<gb, t, 0, s>>>(p, p.perm); ++launch_counter(); break;
        case 5: k_gather<2, double><<<gb, t, 0, s>>>(p, p.perm); ++launch_counter(); break;
        case 6: k_gather<3, float><<<gb, t, 0, s>>>(p, p.perm); ++launch_counter(); break;
        case 7: k_gather<3, double><<<gb, t, 0, s>>>(p, p.perm); ++launch_counter(); break;
        case 8: k_gather<4, float><<<gb, t, 0, s>>>(p, p.perm); ++launch_counter(); break;
        case 9: k_gather<4, double><<<gb, t, 0, s>>>(p, p.perm); ++launch_counter(); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Exclusive scan of n ints (n <= kScanTile^2); scratch needs 2*kScanTile ints.
cudaError_t launch_exclusive_scan(const int* in, int* out, int n, int* scratch, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles > kScanTile) return cudaErrorInvalidValue;
    if (tiles == 1) {
        k_scan_tiles<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr); ++launch_counter();
        return cudaGetLastError();
    }
    int* sums = scratch;
    int* offs = scratch + kScanTile;
    k_scan_tiles<<<tiles, kScanThreads, 0, s>>>(in, out, n, sums); ++launch_counter();
    k_scan_tiles<<<1, kScanThreads, 0, s>>>(sums, offs, tiles, nullptr); ++launch_counter();
    k_scan_add<<<tiles, kScanThreads, 0, s>>>(out, n, offs); ++launch_counter();
    return cudaGetLastError();
}

// scan_scratch: 2*kScanTile ints; every cell_* array holds ncells ints.
cudaError_t launch_make_items(const ItemBuffers& b, const int* cell_start, const int* perm, int ncells, int64_t pb,
                              int64_t pe, int warps, cudaStream_t s)
{
    const int t = 256;
    k_cell_select<<<blocks_for(ncells, t), t, 0, s>>>(cell_start, perm, ncells, pb, pe, warps, b.cell_lo,
                                                      b.cell_prims, b.cell_items); ++launch_counter();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_exclusive_scan(b.cell_prims, b.prim_start, ncells, b.scan_scratch, s);
    if (e != cudaSuccess) return e;
    e = launch_exclusive_scan(b.cell_items, b.item_start, ncells, b.scan_scratch, s);
    if (e != cudaSuccess) return e;
    k_write_items<<<blocks_for(ncells, t), t, 0, s>>>(ncells, warps, b.cell_lo, b.cell_prims, b.prim_start,
                                                      b.item_start, b.ncat, b.cat_cells, b.items); ++launch_counter();
    k_totals<<<1, 32, 0, s>>>(ncells, b.cell_prims, b.prim_start, b.cell_items, b.item_start, b.nprim, b.nitems); ++launch_counter();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(b.ticket, 0, sizeof(int), s);
}

cudaError_t launch_reduce(const double* partial, int rows, int ncols, const int* colmap, int nout, double scale,
                          double* out, cudaStream_t s)
{
    if (nout <= 0) return cudaSuccess;
    const int t = 256;
    k_reduce_rows<<<blocks_for(nout, t), t, 0, s>>>(partial, rows, ncols, colmap, nout, scale, out);
    ++launch_counter();
    return cudaGetLastError();
}

cudaError_t launch_reduce_cats(const double* partial, int rows, int ncols, const int* colmap, int nout, int ncat,
                               const double* scales, double* out, cudaStream_t s)
{
    if (nout <= 0 || ncat <= 0) return cudaSuccess;
    const int t = 256;
    k_reduce_cats<<<dim3(blocks_for(nout, t), ncat), t, 0, s>>>(partial, rows, ncols, colmap, nout, scales, out);
    ++launch_counter();
    return cudaGetLastError();
}

}  // namespace npcf
