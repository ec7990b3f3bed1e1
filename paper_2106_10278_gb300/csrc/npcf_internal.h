// npcf_internal.h -- structures shared by the host plan code and the CUDA
// translation units of libnpcf.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace npcf {

constexpr int kMaxBins = 32;   // lanes own bins in the pair kernel: at most one warp's worth
constexpr int kMaxD = 4;
constexpr int kTab = 4096;     // radial lookup-table entries

// ------------------------------------------------------- catalogue geometry
// The cell grid of one catalogue.  A call covers one or more catalogues; their
// cells are numbered consecutively (catalogue c owns global cells
// [base, base + ncells)), so one cell list and one pair launch serve them all.
struct CatGeom {
    int nc[4];           // cells per axis
    int stride[4];       // local cell index = sum c[d] * stride[d]
    int base;            // first global cell
    int ncells;
    int64_t first;       // first particle (input index)
    float boxf[4];
    float sidef[4];
    double box[4];
    double side[4];
    double inv_side[4];  // nc[d] / box[d]
};
constexpr int kGeomWords = (int)(sizeof(CatGeom) / 4);

// ---------------------------------------------------------------- cell list
struct CellParams {
    int D;
    int64_t n;
    int ncells;              // all catalogues
    int ncat;
    const CatGeom* geo;      // ncat (device)
    const int64_t* offsets;  // ncat + 1 particle offsets (device; used when ncat > 1)
    int periodic;
    const void* pos;    // n x D (float or double)
    const void* w;      // n
    int* cid;           // n
    int* cell_count;    // ncells (+1 scratch)
    int* cell_start;    // ncells + 1
    int* cell_fill;     // ncells
    int* perm;          // n: slot -> original index
    void* rec;          // n records (see Rec in npcf_device.cuh)
    int* err;           // bit 0: non-finite value, bit 1: position outside the box
};

// --------------------------------------------------------------- pair kernel
struct PairParams {
    int D, nbins, lmax, nq;
    int periodic;
    const CatGeom* geo;    // per-catalogue grids (device)
    float rmax2f, rmin2f;  // squared outer / inner radius (FP32, widened by the tolerance)
    float tol;             // absolute half-width of the near-edge window (FP32 path)
    float edgef[kMaxBins + 1];
    double edge2[kMaxBins + 1];  // FP64 squares, the exact bin decision
    float tab_lo, tab_inv;       // radial table: bucket k covers [tab_lo + k/tab_inv, ...)
    signed char lane_bin[32];
    signed char lane_rank[32];
    signed char bin_nlanes[kMaxBins];
    signed char bin_first[kMaxBins];
    int warps;                   // primaries per item (= warps per CTA)
    int busy_round;              // run a consumption round when this many lanes have work
    int tot_round;               // ... or when this many pairs are staged in total
    int nstencil;
    const int* stencil;          // packed offsets, 8 bits per axis (signed)
    const unsigned char* tab;    // kTab entries
    const void* rec;             // sorted records
    const int* cell_start;
    const int4* items;           // (global cell, slot_lo, count | catalogue << 8, primary_base)
    const int* nitems;
    int* ticket;
    const void* qnorm;           // nq normalisation constants (T)
    const void* inv_vb;          // nbins (T)
    void* a_out;                 // nprim x nbins x nq (T)
    void* w_out;                 // nprim (T)
    unsigned long long* stats;   // [0] pairs, [1] candidates, [2] rounds, [3] busy lanes, [4] chunks, [5] forced rounds, [6] flagged-bucket iterations, [7] exact-FP64 iterations
};

// ----------------------------------------------------------- coupling kernel
struct CoupleParams {
    int D, N, nbins, lmax, nq, nlam;
    const void* a;             // nprim x nbins x nq (T)
    const void* wprim;         // nprim (T)
    const int* nprim;
    int chunk;                 // primaries per chunk (FP32 shared accumulation span)
    int ncoeff;
    double* partial;           // gridDim.x rows x 2*ncoeff
    const int2* pairs;         // (b1, b2) pairs of the items
    const int* pair_key;       // first key of each pair's outputs
    const int4* kblocks;       // (pair_lo, pair_hi, key_lo, key_hi) per blockIdx.y
    int nkb;
    int max_block_keys;        // largest key_hi - key_lo
    int max_block_pairs;       // largest pair_hi - pair_lo
    const int* task_pairs;     // D=3, N=4: the pairs of each block ordered by (b2, b1)
    const int2* lam2;          // D=2, N=4: (l1, l2) per Lambda index
    const signed char* lam_odd;// D=3, N=4: 1 if l1+l2+l3 is odd (coefficient imaginary)
    const void* pref;          // N=3: per-l factor of the zero coupling (T)
    int group;                 // D=2 N=4 FP32 and N=5: primaries per shared-memory group
    int ntriple;               // N=5: bin triples b1 < b2 < b3 < nbins - 1
    const int4* triples;       // N=5: (b1, b2, b3, first key) per triple
    const int4* lam5;          // N=5: (first term, end term, l4, 0) per label set
    const int* terms5;         // N=5: state(l1,m1) | state(l2,m2) << 8 | state(l3,m3) << 16 | m4 << 24
    const double* coef5;       // N=5: the coupling coefficient of each term
    const float* coef5f;       // N=5: the same in FP32 (FP32 plans)
    int ncat;                  // catalogues (blockIdx.z); 0 or 1 for a single one
    const int* cat_first;      // ncat: first primary of each catalogue in the a-array (NULL: one catalogue)
    const int* cat_count;      // ncat: its primaries
};

// ------------------------------------------------------------- launchers
// Each returns cudaSuccess or the launch error, and adds the kernels it
// launched to launch_counter() (per host thread).
inline int& launch_counter()
{
    static thread_local int n = 0;
    return n;
}
cudaError_t launch_cell_ids(const CellParams& p, int fp64, cudaStream_t s);
cudaError_t launch_cell_scatter(const CellParams& p, int fp64, cudaStream_t s);
cudaError_t launch_exclusive_scan(const int* in, int* out, int n, int* scratch, cudaStream_t s);
struct ItemBuffers {
    int* cell_lo;      // ncells
    int* cell_prims;   // ncells
    int* prim_start;   // ncells
    int* cell_items;   // ncells
    int* item_start;   // ncells
    int* scan_scratch; // 2 * 4096
    int4* items;       // up to n items
    int* nitems;       // 1
    int* nprim;        // 1
    int* ticket;       // 1
    int ncat = 1;
    const int* cat_cells = nullptr;  // ncat + 1 first global cells (used when ncat > 1)
};
cudaError_t launch_make_items(const ItemBuffers& b, const int* cell_start, const int* perm, int ncells, int64_t pb,
                              int64_t pe, int warps, cudaStream_t s);
cudaError_t launch_couple(const CoupleParams& p, int fp64, int grid, int smem, cudaStream_t s);
int couple_smem(const CoupleParams& p, int fp64);
int d2n4_group(int nbins, int lmax);
int d3n5_group(int nbins, int lmax, int fp64);
int couple_d3n5_smem(const CoupleParams& p, int fp64);
cudaError_t launch_couple_d3n5(const CoupleParams& p, int fp64, int grid, int smem, cudaStream_t s);
cudaError_t launch_reduce(const double* partial, int rows, int ncols, double scale, double* out, cudaStream_t s);
// per catalogue c: out[c][k] = scales[c] * sum_r partial[c][r][k]
cudaError_t launch_reduce_cats(const double* partial, int rows, int ncols, int ncat, const double* scales, double* out,
                               cudaStream_t s);

// adjoint of the N=3 estimator (npcf_backward.cu)
int adjoint_compiled_lmax(int D, int lmax);
int adjoint_pair_warps();
int adjoint_pair_smem(int D, int Lc, int fp64, int nbins);
cudaError_t launch_couple_adjoint(int D, int fp64, int nbins, int nq, int lmax, int64_t nprim, const void* a,
                                  const void* wprim, const double* g, int ncoeff, const int* key_base, const void* pref,
                                  const void* qnorm, const void* inv_vb, double inv_V, void* cbuf, double* gwp,
                                  int nsm, cudaStream_t s);
cudaError_t launch_pairs_adjoint(const PairParams& p, int fp64, int Lc, const void* cbuf, const double* gwp,
                                 const int* perm, double* gpos, double* gw, int nsm, cudaStream_t s);
cudaError_t launch_finalize_grads(int64_t n, int D, int fp64, const double* gpos, const double* gw, void* grad_pos,
                                  void* grad_w, cudaStream_t s);

}  // namespace npcf
