// npcf_internal.h -- structures shared by the host plan code and the CUDA
// translation units of libnpcf.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace npcf {

constexpr int kMaxBins = 32;   // the pair kernel shares a warp's 32 lanes out among the bins
constexpr int kMaxD = 4;
constexpr int kTab = 4096;     // radial lookup-table buckets
constexpr int kTabBytes = kTab + 16;  // the table: a guard entry, the buckets, a guard entry, padding
constexpr int kRecPad = 128;   // records readable past the last one (the pair kernel's prefetch runs ahead)

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
    int warps;                   // primaries per item (= warps per CTA)
    int batch;                   // pairs per warp batch (multiple of 32, <= 1024)
    int nstencil;
    const int* stencil;          // packed offsets, 8 bits per axis (signed)
    int nrows;
    const int2* rows;            // stencil rows: (offsets of axes 1..3, 8 bits each; x range lo | hi << 8)
    const unsigned char* tab;    // kTabBytes entries: [0] and [kTab + 1] "no bin", bucket k at [k + 1]
    const void* rec;             // sorted records
    const int* cell_start;
    const int4* items;           // (global cell, slot_lo, count | catalogue << 8, primary_base)
    const int* nitems;
    int* ticket;
    const void* qnorm;           // nq normalisation constants (T)
    const void* inv_vb;          // nbins (T)
    void* a_out;                 // nprim x nbins x nq (T)
    void* w_out;                 // nprim (T)
    void* self_out;              // nprim x nbins (T): sum of w_k^2 per bin, or NULL
    const int* perm;             // sorted slot -> input index (the 2-sphere's exact path)
    const void* orig;            // the caller's positions, n x 3 (the 2-sphere's exact path)
    unsigned long long* stats;   // [0] pairs, [1] candidates, [2] accumulation rounds, [3] busy lane-rounds, [4] chunks, [5] batches, [6] candidates in flagged buckets, [7] candidates decided in FP64
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
    int group;                 // D=2 N=4 FP32: primaries per shared-memory group
    int ncat;                  // catalogues (blockIdx.z); 0 or 1 for a single one
    const int* cat_first;      // ncat: first primary of each catalogue in the a-array (NULL: one catalogue)
    const int* cat_count;      // ncat: its primaries
    // split-precision tensor-core coupling (npcf_couple_tc.cu)
    int tc_npairs;             // bin pairs = MMA rows (at most 128)
    int tc_glam;               // label sets per CTA (their accumulators share the CTA's TMEM)
    int tc_tmem_cols;          // TMEM columns each CTA allocates (a power of two, <= 512)
    int tc_span;               // chunks of primaries summed in FP32 before each FP64 flush
    int* err;                  // error word: bit 2 = a bounded wait on the tensor core ran out
    const void* self;          // N=3 remove_self: nprim x nbins sums of w_k^2 (T), or NULL
    const void* selfc;         // nbins x (lmax + 1): coincident-direction value c_l / v_b^2 (T)
    // line-of-sight basis (npcf_couple_los.cu)
    const int2* los_lam;       // per label set: (first term, end term)
    const int* los_terms;      // state(l1,m1) | state(l2,m2) << 8 | state(l3,m3) << 16 (all signed m)
    const void* los_coef;      // the CG product of each term (T)
};

// --------------------------------------------------------- gridded field
// The FFT form of the gridded estimator (npcf_grid.cu).
struct GridParams {
    int dims[4];
    int64_t ncell;            // nodes = prod dims
    double spacing[4];        // box / dims
    double dV;                // node volume
    int nbins, nq;
    double edge2[kMaxBins + 1];
    double inv_vb[kMaxBins];
    int ncs;                  // complex harmonic states kept (m >= 0): components (re, im or -1) each
    const int2* cstate;       // ncs (device)
    const void* qnorm;        // nq normalisation constants (T)
    void* khat;               // nbins x ncs x ncell complex: the kernels, then their transforms
    void* xhat;               // ncell complex: the field, then its transform
    void* work;               // a batch of spectral products / inverse transforms
    void* a;                  // ncell x nbins x nq (T): the a-array
    void* wprim;              // ncell (T): dV X
};

int grid_max_lmax();
cudaError_t launch_grid_kernels(const GridParams& g, int D, int fp64, int L, cudaStream_t s);
cudaError_t launch_grid_field(const GridParams& g, int fp64, const void* X, cudaStream_t s);
cudaError_t launch_grid_product(const GridParams& g, int fp64, int bs0, int nbs, cudaStream_t s);
cudaError_t launch_grid_scatter(const GridParams& g, int fp64, int bs0, int nbs, cudaStream_t s);

// ------------------------------------------------- factored 5PCF coupling
// Tables and scratch of npcf_couple_d3n5f.cu (D=3, N=5, through the intermediate label l12).
struct D3n5Params {
    int nbins, lmax, nq, nlam, ncoeff;
    int npc;                     // primaries per chunk: K = npc (2 l12 + 1) per row and column
    const void* a;               // nprim x nbins x nq (T)
    const void* wprim;           // nprim (T)
    const int* nprim;
    const int* cat_first;        // NULL: one catalogue
    const int* cat_count;
    int np12, np34;              // bin pairs (b1 < b2) with b2 <= nbins - 3; (b3 < b4) with b3 >= 2
    const int2* p12;
    const int2* p34;
    int ngx, ngz;                // term groups of X and Z
    const int4* gx;              // (term begin, term end, l12, ix | m12 index << 16)
    const int4* gz;              // (term begin, term end, l12, iz | m12 index << 16)
    const int* terms;            // state of the first a | state of the second a << 8
    const void* coef;            // CG product of each term (T)
    const int* nlx;              // per l12: (l1, l2) label pairs
    const int* nlz;              // per l12: (l3, l4) label pairs
    const int* row0;             // per l12: first row (and X row map entry)
    const int* col0;             // per l12: first column (and Z column map entry)
    const int* xrow;             // [row0 + pair * nlx + ix]: row position in (parity, b2) order
    const int* zcol;             // [col0 + pair * nlz + iz]: column position in (parity, b3) order
    const int4* rowinfo;         // by position: b1, b2, parity, l1 | l2 << 8
    const int4* colinfo;         // by position: b3, b4, parity, l3 | l4 << 8
    const long long* xoff;       // per l12: first element of its X block in the scratch, per primary of a
    const long long* zoff;       //   chunk (complex elements; the block starts at xoff[l12] * npc)
    int ntiles;
    const int4* tiles;           // (l12, first row, first column, rows | columns << 16): the 64 x 64
                                 //   blocks of one parity that hold keys (CUDA-core contraction)
    const int* lamidx;           // [l1][l2][l12][l3][l4] -> label-set index (or -1)
    const int* trikey;           // [b1][b2][b3] -> first key of the bin triple
    int ntc;
    const int4* tc_tiles;        // (l12, first row, first column, rows | columns << 16): the 128-row x
                                 //   64-column blocks of one parity that hold keys (tensor-core path)
    const int* tc_keys;          // [tile][64 columns][128 rows]: the key of each entry, -1 if none
    int kpiece;                  // tensor-core path: K elements per CTA (a multiple of 64)
    int form_lanes;              // primaries per CTA of the formation kernel (32, 16 or 8)
    int nsm;                     // SMs of the device (launch shapes)
    void* xs;                    // scratch: X of the chunk (complex T, or four BF16 planes)
    void* zs;                    // scratch: Z of the chunk
    size_t xs_cat, zs_cat;       // complex elements per catalogue
    double* partial;             // (catalogue, ksplit) rows x 2 ncoeff
    int* err;                    // error word: bit 2 = a bounded wait on the tensor core ran out
};

int d3n5f_form_smem(int nbins, int lmax, int fp64, int lanes);
int d3n5f_form_lanes(int nbins, int lmax, int fp64, int smem_optin);
// mode 0: FP32, 1: FP64, 2: split-BF16 tensor-core contraction (FP32 a-array)
cudaError_t launch_d3n5f(const D3n5Params& q, int mode, int nchunk_prim, int chunk0, int ksplit, int ncat,
                         cudaStream_t s);
cudaError_t launch_d3n5_contract_tc(const D3n5Params& q, int npieces, int ncat, cudaStream_t s);
int d3n5_tc_smem();

// ------------------------------------------------------------- launchers
// Each returns cudaSuccess or the launch error, and adds the kernels it
// launched to launch_counter() (per host thread).
inline int& launch_counter()
{
    static thread_local int n = 0;
    return n;
}
cudaError_t launch_cell_ids(const CellParams& p, int fp64, cudaStream_t s);
// the 2-sphere: positions normalised and shifted by +1 per axis into out (n x 3)
cudaError_t launch_sphere_prep(const void* pos, int64_t n, int fp64, void* out, cudaStream_t s);
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
// out[k] = scale * sum_r partial[r][colmap[k]] (colmap NULL: the identity), k < nout
cudaError_t launch_reduce(const double* partial, int rows, int ncols, const int* colmap, int nout, double scale,
                          double* out, cudaStream_t s);
// per catalogue c: out[c][k] = scales[c] * sum_r partial[c][r][colmap[k]]
cudaError_t launch_reduce_cats(const double* partial, int rows, int ncols, const int* colmap, int nout, int ncat,
                               const double* scales, double* out, cudaStream_t s);

// the line-of-sight basis (npcf_couple_los.cu)
int los_group(int nbins, int lmax, int fp64);
int couple_los_smem(const CoupleParams& p, int fp64);
cudaError_t launch_couple_los(const CoupleParams& p, int fp64, int grid, int smem, cudaStream_t s);

// split-precision tensor-core couplings (npcf_couple_tc.cu)
int couple_tc_smem(int nbins, int nq, int tf32);
int couple_tc_n(int nbins);
int couple_tc_chunk(int tf32);
cudaError_t launch_couple_d2n4_tc(const CoupleParams& p, int tf32, int rows, int groups, int smem, cudaStream_t s);
int tc_selftest_smem();
cudaError_t launch_tc_selftest(int tf32, const float* A, const float* B, float* D, int N, int K, int* err,
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
