// npcf_plan.cu -- host side of libnpcf: plans (keys, coupling and
// normalisation tables, lane map), the cell grid, the device workspace, the
// launch sequence and the C ABI declared in include/npcf.h.
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <tuple>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "npcf.h"
#include "npcf_device.cuh"
#include "npcf_internal.h"
#include "npcf_pairs.cuh"

namespace npcf {
int pair_compiled_lmax_d2(int fp64, int lmax);
int pair_compiled_lmax_d3(int fp64, int lmax);
int pair_compiled_lmax_d4(int fp64, int lmax);
int pair_threads_d2(int fp64, int L);
int pair_threads_d3(int fp64, int L);
int pair_threads_d4(int fp64, int L);
cudaError_t launch_pairs_d2(const PairParams& p, int fp64, int L, int grid, int smem, cudaStream_t s);
cudaError_t launch_pairs_d3(const PairParams& p, int fp64, int L, int grid, int smem, cudaStream_t s);
cudaError_t launch_pairs_d4(const PairParams& p, int fp64, int L, int grid, int smem, cudaStream_t s);
int pair_compiled_lmax_sph(int fp64, int lmax);
cudaError_t launch_pairs_sph(const PairParams& p, int fp64, int L, int grid, int smem, cudaStream_t s);
int couple_max_lmax_d3n4();
}  // namespace npcf

using namespace npcf;

namespace {

thread_local std::string g_err;

npcf_status fail(npcf_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(expr)                                                                           \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) return fail(NPCF_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// A grow-only device buffer.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t reserve(size_t b)
    {
        if (b <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        size_t nb = b + b / 8 + 256;
        cudaError_t e = cudaMalloc(&p, nb);
        if (e == cudaSuccess) bytes = nb;
        return e;
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename U> U* as() const { return static_cast<U*>(p); }
};

double sphere_area(int D) { return 2.0 * std::pow(M_PI, 0.5 * D) / std::tgamma(0.5 * D); }

}  // namespace

// A batched in-place complex FFT of nf fields on a D-dimensional grid (row-major, fields
// contiguous).  cuFFT plans cover ranks 1-3; D = 4 runs as a 3-D transform over the last three
// axes (batched over the first axis and the fields) followed by a 1-D transform along the first
// axis (stride = the 3-D block, batched over the block, once per field).
struct GridFFT {
    cufftHandle a = 0, b = 0;
    int D = 0, nf = 0;
    int64_t ncell = 0, block = 0;
    void destroy()
    {
        if (a) cufftDestroy(a);
        if (b) cufftDestroy(b);
        a = b = 0;
    }
    cufftResult make(int D_, const int* dims, int nf_, bool fp64)
    {
        destroy();
        D = D_;
        nf = nf_;
        const cufftType ty = fp64 ? CUFFT_Z2Z : CUFFT_C2C;
        ncell = 1;
        for (int i = 0; i < D; ++i) ncell *= dims[i];
        int n[3];
        if (D <= 3) {
            for (int i = 0; i < D; ++i) n[i] = dims[i];
            return cufftPlanMany(&a, D, n, nullptr, 1, (int)ncell, nullptr, 1, (int)ncell, ty, nf);
        }
        block = ncell / dims[0];
        for (int i = 0; i < 3; ++i) n[i] = dims[i + 1];
        cufftResult r = cufftPlanMany(&a, 3, n, nullptr, 1, (int)block, nullptr, 1, (int)block, ty, dims[0] * nf);
        if (r != CUFFT_SUCCESS) return r;
        int n0[1] = {dims[0]};
        return cufftPlanMany(&b, 1, n0, n0, (int)block, 1, n0, (int)block, 1, ty, (int)block);
    }
    cufftResult stream(cudaStream_t s)
    {
        cufftResult r = cufftSetStream(a, s);
        if (r == CUFFT_SUCCESS && b) r = cufftSetStream(b, s);
        return r;
    }
    // data: nf fields of `ncell` complex values (complex<float> or complex<double>)
    cufftResult exec(void* data, bool fp64, int dir) const
    {
        auto run = [&](cufftHandle h, void* d) {
            return fp64 ? cufftExecZ2Z(h, (cufftDoubleComplex*)d, (cufftDoubleComplex*)d, dir)
                        : cufftExecC2C(h, (cufftComplex*)d, (cufftComplex*)d, dir);
        };
        cufftResult r = run(a, data);
        if (r != CUFFT_SUCCESS || !b) return r;
        const size_t csz = fp64 ? 16 : 8;
        for (int f = 0; f < nf && r == CUFFT_SUCCESS; ++f) r = run(b, static_cast<unsigned char*>(data) + csz * ncell * f);
        return r;
    }
};

struct npcf_plan_s {
    int D = 3, N = 3, lmax = 0, nbins = 0;
    npcf_opts opts{};
    int fp64 = 0;
    int mixed = 0;  // split-precision tensor-core coupling: 0 none, 1 BF16x3, 2 TF32x3
    std::vector<double> edges;
    double box[4] = {1, 1, 1, 1};
    double V = 1.0;
    int Dp = 3;         // components of a position (D; 3 on the 2-sphere)
    int sphere = 0;     // NPCF_GEOMETRY_SPHERE
    double rcut = 0.0;  // reach of the cell search (r_max; the largest chord on the sphere)
    // keys
    int nlam = 0;
    std::vector<int> lam;       // nlam x 3
    int64_t ncoeff = 0;         // keys the kernels compute
    std::vector<int> key_bins;  // ncoeff x 4
    std::vector<int> key_lam;   // ncoeff
    int64_t nvis = 0;           // keys the caller sees (the opts.parity selection of the computed keys)
    std::vector<int64_t> vis;   // nvis: computed key of each visible key
    // coupling structure
    std::vector<int2> pairs;
    std::vector<int> pair_key;
    std::vector<int4> kblocks;
    std::vector<int4> triples;  // N=5: (b1, b2, b3, first key) of the bin triples that have a b4
    int max_block_keys = 0;
    int max_block_pairs = 0;
    std::vector<int> task_pairs;
    // pair kernel configuration
    int Lc = 0;        // compiled lmax of the pair kernel
    int nq = 0;        // components written per bin (plan lmax)
    int nq_c = 0;      // components of the compiled kernel
    int threads = 0, warps = 0, pair_smem = 0, batch = 0, max_warps = 0;
    // launch shapes the autotuner may change (npcf_autotune); 0 = the built-in choice
    int rows_mult = 0;   // CUDA-core coupling CTAs per SM (rows = rows_mult * nsm / key blocks)
    int tc_span_t = 0;   // tensor-core coupling: chunks per FP32 span
    int d5_npc = 0;      // factored 5PCF: primaries per chunk
    int tuned = 0;       // 1 once npcf_autotune chose (or loaded) the shapes
    PairParams pp{};
    // device tables
    DevBuf d_tab, d_qnorm, d_invvb, d_pairs, d_pair_key, d_kblocks, d_lam2, d_lamodd, d_pref, d_stencil, d_task;
    // N=5: the factored coupling's tables (npcf_couple_d3n5f.cu) and its per-chunk scratch
    DevBuf d5_p12, d5_p34, d5_gx, d5_gz, d5_terms, d5_coef, d5_nlx, d5_nlz, d5_row0, d5_col0, d5_xrow, d5_zcol;
    DevBuf d5_rowinfo, d5_colinfo, d5_xoff, d5_zoff, d5_tiles, d5_tctiles, d5_tckeys, d5_lamidx, d5_trikey, w_x5, w_z5;
    std::vector<int> d5_tc_k1;  // K per primary (2 l12 + 1) of each tensor-core tile
    D3n5Params d5{};           // host copy with the device table pointers (scratch set per call)
    int64_t d5_unit_x = 0, d5_unit_z = 0;  // complex scratch elements per primary of a chunk
    DevBuf d_los_lam, d_los_terms, d_los_coef;  // line-of-sight basis: term lists per label set
    // gridded fields (npcf_compute_grid): the kernels' transforms for the last grid shape
    DevBuf g_khat, g_xhat, g_work, g_cstate, g_small;
    int g_dims[4] = {0, 0, 0, 0};
    int g_nbs = 0;
    GridFFT g_fft_k, g_fft_x, g_fft_w;  // kernels (batched), field, products (batched)
    bool g_ready = false;
    DevBuf d_colmap;  // 2*nvis computed columns of the visible outputs (when a parity is selected)
    DevBuf d_selfc;   // remove_self (N=3): c_l / v_b^2 per (bin, l)
    DevBuf w_self;    // remove_self (N=3): sum of w_k^2 per (primary, bin)
    // workspace
    DevBuf w_cid, w_perm, w_rec, w_cells, w_items, w_a, w_wprim, w_partial, w_small, w_hpos, w_hw, w_hout;
    DevBuf w_upos;  // the 2-sphere: normalised, shifted positions
    // adjoint (npcf_backward)
    DevBuf d_keybase, w_cbuf, w_gpos, w_gw, w_gwp;
    // the single-catalogue grid (one CatGeom) and the last batched layout
    DevBuf d_geo;
    DevBuf b_geo, b_cells, b_offsets, b_first, b_count, b_scales, b_stencil;
    std::vector<int64_t> b_key_off;
    std::vector<double> b_key_box;
    int b_ncat = 0, b_ncells = 0, b_nstencil = 0, b_nrows = 0;
    // cached cell grid
    int grid_c = -1;
    int grid_adj = 0;  // the cached grid was chosen for the adjoint (cells capped at kMaxJobs)
    int nc[4] = {1, 1, 1, 1};
    int ncells = 0;
    int nstencil = 0;
    int nrows = 0;  // stencil rows (after the cells in d_stencil)
    int64_t grid_n = -1;
    // device facts
    int device = -1, nsm = 0, smem_optin = 0;
    // stats of the last run (host copies)
    unsigned long long* h_stats = nullptr;  // pinned, 8 entries
    int* h_small = nullptr;                 // pinned, 4 entries
    int64_t last_nprim = 0;
    cudaStream_t last_stream = nullptr;
    // stage timing (opts.timing)
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int last_launches = 0;
    int timed = 0;
};

namespace {

enum SmallIdx { S_ERR = 0, S_TICKET = 1, S_NITEMS = 2, S_NPRIM = 3 };  // ints; stats follow at byte 16

// ----------------------------------------------------------------- keys
void build_keys(npcf_plan_s* P)
{
    const int nb = P->nbins, L = P->lmax;
    P->lam.clear();
    // labels: 5 ints per set (unused entries 0): N=3 (l); N=4 (l1, l2, l3); N=5 (l1, l2, l12, l3, l4)
    if (P->opts.basis == NPCF_BASIS_LOS) {
        // the line-of-sight basis: N=3 (l1, l2, L), N=4 (l1, l2, l12, l3, L), every L allowed
        for (int l1 = 0; l1 <= L; ++l1)
            for (int l2 = 0; l2 <= L; ++l2) {
                if (P->N == 3) {
                    for (int LL = std::abs(l1 - l2); LL <= l1 + l2; ++LL) P->lam.insert(P->lam.end(), {l1, l2, LL, 0, 0});
                    continue;
                }
                for (int l12 = std::abs(l1 - l2); l12 <= l1 + l2; ++l12)
                    for (int l3 = 0; l3 <= L; ++l3)
                        for (int LL = std::abs(l12 - l3); LL <= l12 + l3; ++LL)
                            P->lam.insert(P->lam.end(), {l1, l2, l12, l3, LL});
            }
    } else if (P->N == 3) {
        for (int l = 0; l <= L; ++l) P->lam.insert(P->lam.end(), {l, 0, 0, 0, 0});
    } else if (P->N == 5) {
        // even parity (l1 + l2 + l3 + l4), the components counted for the paper's 5PCF
        for (int l1 = 0; l1 <= L; ++l1)
            for (int l2 = 0; l2 <= L; ++l2)
                for (int l12 = std::abs(l1 - l2); l12 <= l1 + l2; ++l12)
                    for (int l3 = 0; l3 <= L; ++l3)
                        for (int l4 = 0; l4 <= L; ++l4)
                            if (l4 >= std::abs(l12 - l3) && l4 <= l12 + l3 && (l1 + l2 + l3 + l4) % 2 == 0)
                                P->lam.insert(P->lam.end(), {l1, l2, l12, l3, l4});
    } else if (P->D == 3) {
        for (int a = 0; a <= L; ++a)
            for (int b = 0; b <= L; ++b)
                for (int c = 0; c <= L; ++c)
                    if (c >= std::abs(a - b) && c <= a + b) P->lam.insert(P->lam.end(), {a, b, c, 0, 0});
    } else {
        for (int a = 0; a <= L; ++a)
            for (int b = -L; b <= L; ++b) {
                const int c = -a - b;
                if (std::abs(c) <= L) P->lam.insert(P->lam.end(), {a, b, c, 0, 0});
            }
    }
    P->nlam = (int)P->lam.size() / 5;
    P->key_bins.clear();
    P->key_lam.clear();
    P->pairs.clear();
    P->pair_key.clear();
    if (P->N == 3) {
        const int lt = P->opts.bin_order == NPCF_BINS_LT ? 1 : 0;
        for (int b1 = 0; b1 < nb; ++b1)
            for (int b2 = b1 + lt; b2 < nb; ++b2) {
                P->pairs.push_back(make_int2(b1, b2));
                P->pair_key.push_back((int)P->key_lam.size());
                for (int il = 0; il < P->nlam; ++il) {
                    P->key_bins.insert(P->key_bins.end(), {b1, b2, -1, -1});
                    P->key_lam.push_back(il);
                }
            }
    } else if (P->N == 5) {
        // keys ordered (b1, b2, b3, b4, labels); work items are the triples that have a b4
        for (int b1 = 0; b1 < nb; ++b1)
            for (int b2 = b1 + 1; b2 < nb; ++b2)
                for (int b3 = b2 + 1; b3 < nb; ++b3) {
                    if (b3 + 1 < nb) P->triples.push_back(make_int4(b1, b2, b3, (int)P->key_lam.size()));
                    for (int b4 = b3 + 1; b4 < nb; ++b4)
                        for (int il = 0; il < P->nlam; ++il) {
                            P->key_bins.insert(P->key_bins.end(), {b1, b2, b3, b4});
                            P->key_lam.push_back(il);
                        }
                }
    } else {
        for (int b1 = 0; b1 < nb; ++b1)
            for (int b2 = b1 + 1; b2 < nb; ++b2) {
                if (b2 + 1 < nb) {
                    P->pairs.push_back(make_int2(b1, b2));
                    P->pair_key.push_back((int)P->key_lam.size());
                }
                for (int b3 = b2 + 1; b3 < nb; ++b3)
                    for (int il = 0; il < P->nlam; ++il) {
                        P->key_bins.insert(P->key_bins.end(), {b1, b2, b3, -1});
                        P->key_lam.push_back(il);
                    }
            }
    }
    P->ncoeff = (int64_t)P->key_lam.size();
    // the caller's keys: all, or one parity of (-1)^(l1+l2+l3) (only the D=3 4PCF has both)
    P->vis.clear();
    for (int64_t i = 0; i < P->ncoeff; ++i) {
        const int* l = &P->lam[5 * P->key_lam[i]];
        const int odd = (P->N == 4 && P->D == 3) ? ((l[0] + l[1] + l[2]) & 1) : 0;
        if (P->opts.parity == NPCF_PARITY_ALL || odd == (P->opts.parity == NPCF_PARITY_ODD ? 1 : 0))
            P->vis.push_back(i);
    }
    P->nvis = (int64_t)P->vis.size();
}

// Split the pair list into blocks whose keys fit the shared accumulators.
void build_key_blocks(npcf_plan_s* P, int max_keys)
{
    P->kblocks.clear();
    const int np = (int)P->pairs.size();
    int lo = 0;
    P->max_block_keys = 0;
    P->max_block_pairs = 0;
    while (lo < np) {
        int hi = lo + 1;
        auto key_end = [&](int h) { return h < np ? P->pair_key[h] : (int)P->ncoeff; };
        while (hi < np && key_end(hi + 1) - P->pair_key[lo] <= max_keys) ++hi;
        const int k0 = P->pair_key[lo], k1 = key_end(hi);
        P->kblocks.push_back(make_int4(lo, hi, k0, k1));
        P->max_block_keys = std::max(P->max_block_keys, k1 - k0);
        P->max_block_pairs = std::max(P->max_block_pairs, hi - lo);
        lo = hi;
    }
    // work order of the pairs inside each block: by (b2, b1), so that the bin
    // pairs sharing a warp in the D=3, N=4 coupling have similar b2
    P->task_pairs.clear();
    for (const int4& kb : P->kblocks) {
        std::vector<int> v;
        for (int i = kb.x; i < kb.y; ++i) v.push_back(i);
        std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
            return P->pairs[a].y != P->pairs[b].y ? P->pairs[a].y < P->pairs[b].y : P->pairs[a].x < P->pairs[b].x;
        });
        P->task_pairs.insert(P->task_pairs.end(), v.begin(), v.end());
    }
}

// ------------------------------------------------------- normalisation
// Per real component of the a-array, the constant that turns the scaled
// recurrence sums of the pair kernel into sum_k w_k Y*(r^).
std::vector<double> component_norms(int D, int lmax)
{
    std::vector<double> q(num_q(D, lmax), 0.0);
    if (D == 2) {
        for (auto& v : q) v = 1.0 / std::sqrt(2.0 * M_PI);
    } else if (D == 3) {
        for (int l = 0; l <= lmax; ++l)
            for (int m = 0; m <= l; ++m) {
                const double N = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * cx::fact(l - m) / cx::fact(l + m));
                const double F = N * cx::leg_scale(l, m);
                q[q_index_d3(l, m)] = F;
                if (m > 0) q[q_index_d3(l, m) + 1] = F;
            }
    } else {
        for (int l3 = 0; l3 <= lmax; ++l3)
            for (int l2 = 0; l2 <= l3; ++l2) {
                const int n = l3 - l2, lam = l2 + 1;
                // norm of C^{(lam)}_n with weight (1-x^2)^{lam-1/2}
                const double h = M_PI * std::pow(2.0, 1.0 - 2.0 * lam) * std::tgamma(n + 2.0 * lam) /
                                 (cx::fact(n) * (n + lam) * std::tgamma((double)lam) * std::tgamma((double)lam));
                const double c = 1.0 / std::sqrt(h);
                for (int l1 = 0; l1 <= l2; ++l1) {
                    const double N3 =
                        std::sqrt((2.0 * l2 + 1.0) / (4.0 * M_PI) * cx::fact(l2 - l1) / cx::fact(l2 + l1));
                    const double F = N3 * cx::leg_scale(l2, l1) * c * cx::geg_scale(n, lam);
                    q[q_index_d4(l3, l2, l1)] = F;
                    if (l1 > 0) q[q_index_d4(l3, l2, l1) + 1] = F;
                }
            }
    }
    return q;
}

template <typename T>
cudaError_t upload(DevBuf& b, const std::vector<T>& v)
{
    cudaError_t e = b.reserve(std::max<size_t>(sizeof(T) * v.size(), 16));
    if (e != cudaSuccess || v.empty()) return e;
    return cudaMemcpy(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
}

template <typename T>
std::vector<T> cast_vec(const std::vector<double>& v)
{
    return std::vector<T>(v.begin(), v.end());
}

// ------------------------------------------------------------ cell grid
struct GridChoice {
    int c = 0;
    int nc[4] = {1, 1, 1, 1};
    int ncells = 0;
    std::vector<int> stencil;
};

std::vector<int> make_stencil(int D, int c, const double* side, double reach)
{
    std::vector<int> out;
    int o[4] = {0, 0, 0, 0};
    const int span = 2 * c + 1;
    int total = 1;
    for (int d = 0; d < D; ++d) total *= span;
    for (int idx = 0; idx < total; ++idx) {
        int r = idx;
        double m2 = 0.0;
        int packed = 0;
        for (int d = 0; d < D; ++d) {
            o[d] = r % span - c;
            r /= span;
            const double g = std::max(std::abs(o[d]) - 1, 0) * side[d];
            m2 += g * g;
            packed |= (o[d] & 0xff) << (8 * d);
        }
        if (m2 < reach * reach) out.push_back(packed);
    }
    // Visit the neighbour cells in a fixed pseudo-random order: consecutive
    // cells then lie at unrelated distances, so the pairs a warp stages spread
    // over all radial bins instead of arriving in bursts of 3-4 bins.
    const char* order = std::getenv("NPCF_STENCIL_ORDER");
    if (!(order && std::strcmp(order, "natural") == 0)) {
        std::mt19937 rng(0x5eed1234u);
        std::shuffle(out.begin(), out.end(), rng);
    }
    return out;
}

// The stencil's rows for the pair kernel: the cells that differ only in their axis-0 offset form a
// run of consecutive cell indices (axis 0 has stride 1), so of sorted records.  A row is (offsets
// along axes 1..3, 8 bits each from the lowest; x range lo | hi << 8), in a fixed pseudo-random
// order.  They follow the cell list, which is padded to an even length (the rows are read as int2);
// *nrows receives their count.
std::vector<int> stencil_with_rows(const std::vector<int>& cells, int* nrows)
{
    std::vector<int> keys;
    std::vector<int2> rows;
    for (int pk : cells) {
        const int dx = (int)(signed char)(pk & 0xff);
        const int rest = (int)((unsigned)pk >> 8);
        size_t i = 0;
        while (i < keys.size() && keys[i] != rest) ++i;
        if (i == keys.size()) {
            keys.push_back(rest);
            rows.push_back(make_int2(dx, dx));
        } else {
            rows[i].x = std::min(rows[i].x, dx);
            rows[i].y = std::max(rows[i].y, dx);
        }
    }
    std::vector<int> order(keys.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::mt19937 rng(0x5eed4321u);
    std::shuffle(order.begin(), order.end(), rng);
    std::vector<int> out(cells);
    if (out.size() & 1) out.push_back(0);
    for (int i : order) {
        out.push_back(keys[i]);
        out.push_back((rows[i].x & 0xff) | ((rows[i].y & 0xff) << 8));
    }
    *nrows = (int)keys.size();
    return out;
}

GridChoice choose_grid(const npcf_plan_s* P, int64_t n, bool adjoint)
{
    // Preferred: the cheapest grid with >= 4 particles per cell on average;
    // otherwise (very sparse inputs) the cheapest valid grid of any density.  Cells of side
    // r_max / c, c <= 4: finer cells (c up to 8, 20% fewer candidates at the D=3 4PCF workload)
    // made the forward pair kernel 1.9x slower -- many short runs, each starting with a wait for
    // its first records.  The adjoint pair kernel lists an item's cells, at most kMaxJobs.
    GridChoice best, any;
    double best_cost = 1e300, any_cost = 1e300;
    const double rmax = P->rcut;
    const double reach = rmax * (1.0 + 1e-6) + 1e-12;
    for (int c = 1; c <= 4; ++c) {
        GridChoice g;
        g.c = c;
        bool ok = true;
        double side[4];
        int64_t ncells = 1;
        for (int d = 0; d < P->Dp; ++d) {
            int k = (int)std::floor(P->box[d] * c / rmax);
            if (k < 1) k = 1;
            if (P->opts.periodic && k < 2 * c + 1) ok = false;
            if (k > 4096) k = 4096;
            g.nc[d] = k;
            side[d] = P->box[d] / k;
            ncells *= k;
        }
        if (!ok || ncells >= (1 << 24)) continue;
        g.ncells = (int)ncells;
        const double npc = (double)std::max<int64_t>(n, 1) / (double)ncells;
        g.stencil = make_stencil(P->Dp, c, side, reach);
        if (adjoint && (int)g.stencil.size() > kMaxJobs) continue;  // the adjoint lists an item's cells in smem
        // candidates examined, plus a fixed cost per stencil row (the pair kernel walks rows)
        int nrows = 0;
        stencil_with_rows(g.stencil, &nrows);
        if (nrows > kMaxJobs) continue;  // the pair kernel tabulates an item's rows in smem
        const double cost = g.stencil.size() * npc + 40.0 * nrows;
        if (cost < any_cost) {
            any_cost = cost;
            any = g;
        }
        if (npc >= 4.0 && cost < best_cost) {
            best_cost = cost;
            best = g;
        }
    }
    return best.c > 0 ? best : any;
}

CatGeom make_geom(int D, const int* nc, const double* box, int base, int64_t first)
{
    CatGeom g{};
    int stride = 1, ncells = 1;
    for (int d = 0; d < 4; ++d) {
        const bool on = d < D;
        g.nc[d] = on ? nc[d] : 1;
        g.stride[d] = stride;
        g.box[d] = on ? box[d] : 1.0;
        g.boxf[d] = (float)g.box[d];
        g.side[d] = g.box[d] / g.nc[d];
        g.sidef[d] = (float)g.side[d];
        g.inv_side[d] = g.nc[d] / g.box[d];
        if (on) {
            stride *= nc[d];
            ncells *= nc[d];
        }
    }
    g.base = base;
    g.ncells = ncells;
    g.first = first;
    return g;
}

int pair_compiled_lmax(int D, int fp64, int lmax)
{
    if (D == 2) return pair_compiled_lmax_d2(fp64, lmax);
    if (D == 3) return pair_compiled_lmax_d3(fp64, lmax);
    return pair_compiled_lmax_d4(fp64, lmax);
}

int pair_threads(int D, int fp64, int L)
{
    if (D == 2) return pair_threads_d2(fp64, L);
    if (D == 3) return pair_threads_d3(fp64, L);
    return pair_threads_d4(fp64, L);
}

int rec_bytes(int D, int fp64) { return (fp64 ? 8 : 4) * 4 * (D <= 3 ? 1 : 2); }

// The pair kernel's launch shape: up to `warps` warps per CTA (fewer if shared memory runs out)
// and `batch` pairs per warp batch.  Returns false if not even one warp fits.
bool set_pair_config(npcf_plan_s* P, int warps, int batch)
{
    const int rb = rec_bytes(P->D, P->fp64), tb = P->fp64 ? 8 : 4, nb = P->nbins;
    batch = std::max(64, std::min(1024, batch / 32 * 32));
    warps = std::max(1, std::min(P->max_warps, warps));
    while (warps > 1 && pair_fixed_bytes(rb, warps * 32) + warps * pair_warp_bytes(rb, tb, nb, P->nq_c, batch) >
                            P->smem_optin)
        --warps;
    const int smem = pair_fixed_bytes(rb, warps * 32) + warps * pair_warp_bytes(rb, tb, nb, P->nq_c, batch);
    if (smem > P->smem_optin) return false;
    P->warps = warps;
    P->threads = warps * 32;
    P->batch = batch;
    P->pair_smem = smem;
    P->pp.warps = warps;
    P->pp.batch = batch;
    return true;
}

npcf_status ensure_device(npcf_plan_s* P)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (P->device == dev) return NPCF_OK;
    if (P->device >= 0) return fail(NPCF_ERR_ARG, "plan was created on device %d, current device is %d", P->device, dev);
    P->device = dev;
    CUDA_TRY(cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&P->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    void* pinned = nullptr;
    CUDA_TRY(cudaMallocHost(&pinned, 128));
    std::memset(pinned, 0, 128);
    P->h_small = static_cast<int*>(pinned);
    P->h_stats = reinterpret_cast<unsigned long long*>(static_cast<char*>(pinned) + 16);
    return NPCF_OK;
}

// The FP32 D=2 4PCF coupling accumulates in registers over groups of primaries
// (one CTA per SM: its group of a-rows fills shared memory).
bool d2n4_registers(const npcf_plan_s* P) { return P->N == 4 && P->D == 2 && !P->fp64; }

// Plans whose coupling runs on the tensor cores in split precision (BF16x3 or TF32x3).
bool tc_coupling(const npcf_plan_s* P) { return P->mixed != 0 && P->D == 2 && P->N == 4; }

// label sets per CTA of the tensor-core coupling: as many MMA accumulators (128 x N FP32) as
// fit the 512 TMEM columns of an SM
int tc_glam(const npcf_plan_s* P) { return std::max(1, 512 / couple_tc_n(P->nbins)); }
int tc_groups(const npcf_plan_s* P) { return (P->nlam + tc_glam(P) - 1) / tc_glam(P); }

// chunks of primaries summed in FP32 (in TMEM) before each FP64 flush; NPCF_TC_SPAN overrides
int tc_span()
{
    if (const char* e = std::getenv("NPCF_TC_SPAN")) {
        const int v = std::atoi(e);
        if (v > 0 && v <= 1024) return v;
    }
    return 16;
}

// ----------------------------------------------------- factored 5PCF tables
// The tables of the 5PCF coupling through the intermediate label (npcf_couple_d3n5f.cu): bin
// pairs, the (l1, l2) and (l3, l4) label pairs of every l12, the CG terms of X and Z, the rows
// (columns) of every l12 in (parity, b2) ((parity, b3)) order, the tiles that hold keys, and
// the key maps.  The CG chain is the one of eq. Coupling-C with the CGs of eq. CG-examples.
npcf_status build_d3n5f_tables(npcf_plan_s* P)
{
    const int L = P->lmax, nb = P->nbins, NL = 2 * L + 1;
    auto cg = [](int j1, int m1, int j2, int m2, int J, int M) {
        return cx::neg1_pow(j1 - j2 + M) * std::sqrt(2.0 * J + 1.0) * cx::wigner3j(j1, j2, J, m1, m2, -M);
    };
    auto st = [](int l, int m) { return l * l + l + m; };
    std::vector<int2> p12, p34;
    for (int b2 = 1; b2 <= nb - 3; ++b2)
        for (int b1 = 0; b1 < b2; ++b1) p12.push_back(make_int2(b1, b2));
    for (int b3 = 2; b3 <= nb - 2; ++b3)
        for (int b4 = b3 + 1; b4 < nb; ++b4) p34.push_back(make_int2(b3, b4));
    std::vector<std::vector<int2>> lx(NL), lz(NL);
    for (int l12 = 0; l12 < NL; ++l12)
        for (int a = 0; a <= L; ++a)
            for (int b = 0; b <= L; ++b) {
                if (std::abs(a - b) <= l12 && l12 <= a + b) lx[l12].push_back(make_int2(a, b));
                if (std::abs(l12 - a) <= b && b <= l12 + a) lz[l12].push_back(make_int2(a, b));
            }
    std::vector<int4> gx, gz;
    std::vector<int> terms;
    std::vector<double> coef;
    for (int l12 = 0; l12 < NL; ++l12) {
        for (int ix = 0; ix < (int)lx[l12].size(); ++ix) {
            const int l1 = lx[l12][ix].x, l2 = lx[l12][ix].y;
            for (int m12 = -l12; m12 <= l12; ++m12) {
                const int t0 = (int)terms.size();
                for (int m1 = -l1; m1 <= l1; ++m1) {
                    const int m2 = m12 - m1;
                    if (std::abs(m2) > l2) continue;
                    const double c = cg(l1, m1, l2, m2, l12, m12);
                    if (c == 0.0) continue;
                    terms.push_back(st(l1, m1) | (st(l2, m2) << 8));
                    coef.push_back(c);
                }
                gx.push_back(make_int4(t0, (int)terms.size(), l12, ix | ((m12 + l12) << 16)));
            }
        }
        for (int iz = 0; iz < (int)lz[l12].size(); ++iz) {
            const int l3 = lz[l12][iz].x, l4 = lz[l12][iz].y;
            for (int m12 = -l12; m12 <= l12; ++m12) {
                const int t0 = (int)terms.size();
                for (int m3 = -l3; m3 <= l3; ++m3) {
                    const int M = m12 + m3;
                    if (std::abs(M) > l4) continue;
                    const double c = cg(l12, m12, l3, m3, l4, M) * cg(l4, M, l4, -M, 0, 0);
                    if (c == 0.0) continue;
                    terms.push_back(st(l3, m3) | (st(l4, -M) << 8));
                    coef.push_back(c);
                }
                gz.push_back(make_int4(t0, (int)terms.size(), l12, iz | ((m12 + l12) << 16)));
            }
        }
    }
    // rows (columns) of each l12 in (parity, b2, b1, ix) ((parity, b3, b4, iz)) order
    std::vector<int> nlx(NL), nlz(NL), row0(NL + 1), col0(NL + 1), xrow, zcol;
    std::vector<int4> rowinfo, colinfo, tiles, tc_tiles;
    std::vector<long long> xoff(NL), zoff(NL);
    long long ux = 0, uz = 0;
    for (int l12 = 0; l12 < NL; ++l12) {
        nlx[l12] = (int)lx[l12].size();
        nlz[l12] = (int)lz[l12].size();
        row0[l12] = (int)rowinfo.size();
        col0[l12] = (int)colinfo.size();
        const int nr = (int)p12.size() * nlx[l12], nc = (int)p34.size() * nlz[l12];
        std::vector<int> ro(nr), co(nc);
        for (int i = 0; i < nr; ++i) ro[i] = i;
        for (int i = 0; i < nc; ++i) co[i] = i;
        auto rkey = [&](int i) {
            const int pr = i / nlx[l12], ix = i % nlx[l12];
            const int par = (lx[l12][ix].x + lx[l12][ix].y) & 1;
            return std::make_tuple(par, p12[pr].y, p12[pr].x, ix);
        };
        auto ckey = [&](int i) {
            const int pr = i / nlz[l12], iz = i % nlz[l12];
            const int par = (lz[l12][iz].x + lz[l12][iz].y) & 1;
            return std::make_tuple(par, p34[pr].x, p34[pr].y, iz);
        };
        std::stable_sort(ro.begin(), ro.end(), [&](int a, int b) { return rkey(a) < rkey(b); });
        std::stable_sort(co.begin(), co.end(), [&](int a, int b) { return ckey(a) < ckey(b); });
        std::vector<int> rpos(nr), cpos(nc);
        for (int k = 0; k < nr; ++k) {
            rpos[ro[k]] = k;
            const int pr = ro[k] / nlx[l12], ix = ro[k] % nlx[l12];
            const int2 l = lx[l12][ix];
            rowinfo.push_back(make_int4(p12[pr].x, p12[pr].y, (l.x + l.y) & 1, l.x | (l.y << 8)));
        }
        for (int k = 0; k < nc; ++k) {
            cpos[co[k]] = k;
            const int pr = co[k] / nlz[l12], iz = co[k] % nlz[l12];
            const int2 l = lz[l12][iz];
            colinfo.push_back(make_int4(p34[pr].x, p34[pr].y, (l.x + l.y) & 1, l.x | (l.y << 8)));
        }
        xrow.insert(xrow.end(), rpos.begin(), rpos.end());
        zcol.insert(zcol.end(), cpos.begin(), cpos.end());
        xoff[l12] = ux;
        zoff[l12] = uz;
        ux += (long long)nr * (2 * l12 + 1);
        uz += (long long)nc * (2 * l12 + 1);
        // blocks within one parity (rows and columns of a parity are contiguous in this order)
        // that hold a key: 64 x 64 for the CUDA-core contraction, 128 rows x 64 columns for the
        // tensor-core path
        for (int par = 0; par < 2; ++par) {
            int ra = 0, rb = 0, ca = 0, cb = 0;
            while (ra < nr && rowinfo[row0[l12] + ra].z != par) ++ra;
            for (rb = ra; rb < nr && rowinfo[row0[l12] + rb].z == par;) ++rb;
            while (ca < nc && colinfo[col0[l12] + ca].z != par) ++ca;
            for (cb = ca; cb < nc && colinfo[col0[l12] + cb].z == par;) ++cb;
            for (int r0 = ra; r0 < rb; r0 += 64)
                for (int c0 = ca; c0 < cb; c0 += 64) {
                    const int tr = std::min(64, rb - r0), tcn = std::min(64, cb - c0);
                    // rows ascend in b2 and columns in b3: a key iff the first row's b2 < the last column's b3
                    if (rowinfo[row0[l12] + r0].y < colinfo[col0[l12] + c0 + tcn - 1].x)
                        tiles.push_back(make_int4(l12, r0, c0, tr | (tcn << 16)));
                }
            for (int r0 = ra; r0 < rb; r0 += 128)
                for (int c0 = ca; c0 < cb; c0 += 64) {
                    const int tr = std::min(128, rb - r0), tcn = std::min(64, cb - c0);
                    // rows ascend in b2 and columns in b3: a key iff the first row's b2 < the last column's b3
                    if (rowinfo[row0[l12] + r0].y < colinfo[col0[l12] + c0 + tcn - 1].x)
                        tc_tiles.push_back(make_int4(l12, r0, c0, tr | (tcn << 16)));
                }
        }
    }
    // longest K first (the CTAs of one launch are dealt in tile order)
    std::stable_sort(tc_tiles.begin(), tc_tiles.end(), [](const int4& a, const int4& b) { return a.x > b.x; });
    row0[NL] = (int)rowinfo.size();
    col0[NL] = (int)colinfo.size();
    const int L1 = L + 1;
    std::vector<int> lamidx((size_t)L1 * L1 * NL * L1 * L1, -1);
    for (int i = 0; i < P->nlam; ++i) {
        const int* l = &P->lam[5 * i];
        lamidx[((((size_t)l[0] * L1 + l[1]) * NL + l[2]) * L1 + l[3]) * L1 + l[4]] = i;
    }
    std::vector<int> trikey((size_t)nb * nb * nb, -1);
    for (const int4& t : P->triples) trikey[((size_t)t.x * nb + t.y) * nb + t.z] = t.w;
    // the key of every entry of every tensor-core tile, column-major ([tile][column][row]), -1 where
    // b2 >= b3 or outside the tile
    std::vector<int> tc_keys(tc_tiles.size() * 64 * 128, -1);
    for (size_t t = 0; t < tc_tiles.size(); ++t) {
        const int4 T = tc_tiles[t];
        const int l12 = T.x, tr = T.w & 0xffff, tcn = T.w >> 16;
        for (int c = 0; c < tcn; ++c)
            for (int r = 0; r < tr; ++r) {
                const int4 R = rowinfo[row0[l12] + T.y + r], C = colinfo[col0[l12] + T.z + c];
                if (R.y >= C.x) continue;
                const int lam = lamidx[((((size_t)(R.w & 0xff) * L1 + (R.w >> 8)) * NL + l12) * L1 + (C.w & 0xff)) * L1 +
                                       (C.w >> 8)];
                const int tk = trikey[((size_t)R.x * nb + R.y) * nb + C.x];
                if (lam < 0 || tk < 0) return fail(NPCF_ERR_UNSUPPORTED, "5PCF key table: missing key");
                tc_keys[(t * 64 + c) * 128 + r] = tk + (C.y - C.x - 1) * P->nlam + lam;
            }
    }
    CUDA_TRY(upload(P->d5_tckeys, tc_keys));
    CUDA_TRY(upload(P->d5_p12, p12));
    CUDA_TRY(upload(P->d5_p34, p34));
    CUDA_TRY(upload(P->d5_gx, gx));
    CUDA_TRY(upload(P->d5_gz, gz));
    CUDA_TRY(upload(P->d5_terms, terms));
    if (P->fp64) CUDA_TRY(upload(P->d5_coef, coef));
    else CUDA_TRY(upload(P->d5_coef, cast_vec<float>(coef)));
    CUDA_TRY(upload(P->d5_nlx, nlx));
    CUDA_TRY(upload(P->d5_nlz, nlz));
    CUDA_TRY(upload(P->d5_row0, row0));
    CUDA_TRY(upload(P->d5_col0, col0));
    CUDA_TRY(upload(P->d5_xrow, xrow));
    CUDA_TRY(upload(P->d5_zcol, zcol));
    CUDA_TRY(upload(P->d5_rowinfo, rowinfo));
    CUDA_TRY(upload(P->d5_colinfo, colinfo));
    CUDA_TRY(upload(P->d5_xoff, xoff));
    CUDA_TRY(upload(P->d5_zoff, zoff));
    CUDA_TRY(upload(P->d5_tiles, tiles));
    CUDA_TRY(upload(P->d5_tctiles, tc_tiles));
    CUDA_TRY(upload(P->d5_lamidx, lamidx));
    CUDA_TRY(upload(P->d5_trikey, trikey));
    D3n5Params& q = P->d5;
    q = D3n5Params{};
    q.nbins = nb;
    q.lmax = L;
    q.nq = P->nq;
    q.nlam = P->nlam;
    q.ncoeff = (int)P->ncoeff;
    q.np12 = (int)p12.size();
    q.np34 = (int)p34.size();
    q.p12 = P->d5_p12.as<int2>();
    q.p34 = P->d5_p34.as<int2>();
    q.ngx = (int)gx.size();
    q.ngz = (int)gz.size();
    q.gx = P->d5_gx.as<int4>();
    q.gz = P->d5_gz.as<int4>();
    q.terms = P->d5_terms.as<int>();
    q.coef = P->d5_coef.p;
    q.nlx = P->d5_nlx.as<int>();
    q.nlz = P->d5_nlz.as<int>();
    q.row0 = P->d5_row0.as<int>();
    q.col0 = P->d5_col0.as<int>();
    q.xrow = P->d5_xrow.as<int>();
    q.zcol = P->d5_zcol.as<int>();
    q.rowinfo = P->d5_rowinfo.as<int4>();
    q.colinfo = P->d5_colinfo.as<int4>();
    q.xoff = P->d5_xoff.as<long long>();
    q.zoff = P->d5_zoff.as<long long>();
    q.ntiles = (int)tiles.size();
    q.tiles = P->d5_tiles.as<int4>();
    q.ntc = (int)tc_tiles.size();
    q.tc_tiles = P->d5_tctiles.as<int4>();
    q.tc_keys = P->d5_tckeys.as<int>();
    P->d5_tc_k1.clear();
    for (const int4& t : tc_tiles) P->d5_tc_k1.push_back(2 * t.x + 1);
    q.form_lanes = d3n5f_form_lanes(nb, L, P->fp64, P->smem_optin);
    q.nsm = P->nsm;
    q.lamidx = P->d5_lamidx.as<int>();
    q.trikey = P->d5_trikey.as<int>();
    P->d5_unit_x = ux;
    P->d5_unit_z = uz;
    if (q.form_lanes == 0)
        return fail(NPCF_ERR_UNSUPPORTED, "the 5PCF coupling needs more shared memory than available");
    if (P->mixed && d3n5_tc_smem() > P->smem_optin)
        return fail(NPCF_ERR_UNSUPPORTED, "the tensor-core 5PCF contraction needs %d bytes of shared memory",
                    d3n5_tc_smem());
    return NPCF_OK;
}

// Primaries per chunk of the factored 5PCF coupling: its X and Z scratch near 64 MB (it stays in
// L2 between the two kernels), a multiple of 64 (whole 64-element K stages of the tensor-core
// contraction) in [64, 512].
int d3n5f_chunk(const npcf_plan_s* P, size_t budget = 0)
{
    if (budget == 0 && P->d5_npc > 0) return P->d5_npc;  // the autotuner's choice
    if (budget == 0) budget = size_t(64) << 20;
    const size_t per = (size_t)(P->d5_unit_x + P->d5_unit_z) * 2 * (P->fp64 ? 8 : 4);
    const size_t c = budget / std::max<size_t>(per, 1);
    return (int)std::max<size_t>(64, std::min<size_t>(512, c / 64 * 64));
}

bool d5_tc(const npcf_plan_s* P) { return P->N == 5 && P->mixed == 1; }

// Tensor-core 5PCF contraction: K elements per CTA (a multiple of 64).  Two CTAs fit an SM, so a
// launch takes ceil(pieces / (2 SMs)) waves of at most kpiece K each; the choice minimises
// waves x (kpiece + 128), the 128 standing for a CTA's fixed cost (its epilogue and pipeline fill).
int d3n5f_kpiece(const npcf_plan_s* P, int npc)
{
    int kmax = 1;
    for (int k1 : P->d5_tc_k1) kmax = std::max(kmax, k1);
    const int64_t nsm = 2 * std::max(P->nsm, 1);  // CTA slots: two per SM
    int best = 64;
    int64_t best_cost = (int64_t)1 << 62;
    for (int kp = 64; kp <= npc * kmax; kp += 64) {
        int64_t pieces = 0;
        for (int k1 : P->d5_tc_k1) pieces += ((int64_t)npc * k1 + kp - 1) / kp;
        const int64_t cost = (pieces + nsm - 1) / nsm * (kp + 128);
        if (cost < best_cost) best_cost = cost, best = kp;
    }
    return best;
}

// The partial rows (K slices) of the factored 5PCF coupling: about two CTAs per SM over its tiles
// (CUDA cores); the most K pieces of a tile (tensor cores).
int d3n5f_ksplit(const npcf_plan_s* P, int npc)
{
    if (d5_tc(P)) {
        int kmax = 1;
        for (int k1 : P->d5_tc_k1) kmax = std::max(kmax, k1);
        const int kp = d3n5f_kpiece(P, npc);
        return (int)(((int64_t)npc * kmax + kp - 1) / kp);
    }
    return std::max(1, std::min(npc / 8, (2 * P->nsm + P->d5.ntiles - 1) / std::max(P->d5.ntiles, 1)));
}

// The factored 5PCF coupling of ncat catalogues (a-array rows cat_first[c] ..): per chunk of npc
// primaries the formation and the contraction kernels; partial rows [cat][ksplit].
npcf_status run_d3n5f(npcf_plan_s* P, const void* a, const void* wprim, const int* nprim_dev, int64_t nprim_max,
                      const int* cat_first, const int* cat_count, int ncat, void* xs, void* zs, int npc, int ksplit,
                      double* partial, int* err, cudaStream_t s)
{
    D3n5Params q = P->d5;
    q.npc = npc;
    q.err = err;
    q.kpiece = d3n5f_kpiece(P, npc);
    const int mode = d5_tc(P) ? 2 : (P->fp64 ? 1 : 0);
    q.a = a;
    q.wprim = wprim;
    q.nprim = nprim_dev;
    q.cat_first = cat_first;
    q.cat_count = cat_count;
    q.xs = xs;
    q.zs = zs;
    q.xs_cat = (size_t)P->d5_unit_x * npc;
    q.zs_cat = (size_t)P->d5_unit_z * npc;
    q.partial = partial;
    for (int64_t c0 = 0; c0 < std::max<int64_t>(nprim_max, 1); c0 += npc) {
        const int nc = (int)std::min<int64_t>(npc, std::max<int64_t>(nprim_max - c0, 0));
        cudaError_t e = launch_d3n5f(q, mode, nc, (int)c0, ksplit, ncat, s);
        if (e != cudaSuccess) return fail(NPCF_ERR_CUDA, "5PCF coupling launch: %s", cudaGetErrorString(e));
    }
    return NPCF_OK;
}

npcf_status setup_tables(npcf_plan_s* P)
{
    const int D = P->D, nb = P->nbins;
    // pair kernel
    P->Lc = P->sphere ? pair_compiled_lmax_sph(P->fp64, P->lmax) : pair_compiled_lmax(D, P->fp64, P->lmax);
    if (P->Lc < 0) return fail(NPCF_ERR_UNSUPPORTED, "lmax=%d is not compiled for D=%d (%s)", P->lmax, D,
                                P->fp64 ? "FP64" : "FP32");
    P->nq = num_q(D, P->lmax);
    P->nq_c = num_q(D, P->Lc);
    P->max_warps = pair_threads(D, P->fp64, P->Lc) / 32;
    if (!set_pair_config(P, P->max_warps, pair_batch(rec_bytes(D, P->fp64))))
        return fail(NPCF_ERR_UNSUPPORTED, "pair kernel needs more shared memory than available");
    const int warps = P->warps;

    PairParams& pp = P->pp;
    std::memset(&pp, 0, sizeof(pp));
    pp.D = D;
    pp.nbins = nb;
    pp.lmax = P->lmax;
    pp.nq = P->nq;
    pp.periodic = P->opts.periodic;
    pp.warps = warps;
    pp.batch = P->batch;
    std::vector<unsigned char> tab(kTabBytes, (unsigned char)63);  // guards and padding: no bin
    if (!P->sphere) {
        double maxL = 0.0;
        for (int d = 0; d < D; ++d) maxL = std::max(maxL, P->box[d]);
        const double rmax = P->edges[nb], rmin = P->edges[0];
        const double tol = 4.0 * (std::sqrt((double)D) * maxL * std::ldexp(1.0, -23) + rmax * std::ldexp(1.0, -21));
        pp.tol = (float)tol;
        pp.rmax2f = (float)((rmax + 2 * tol) * (rmax + 2 * tol));
        const double rl = std::max(rmin - 2 * tol, 0.0);
        pp.rmin2f = (float)(rl * rl);
        for (int b = 0; b <= nb; ++b) {
            pp.edgef[b] = (float)P->edges[b];
            pp.edge2[b] = P->edges[b] * P->edges[b];
        }
        // radial table over r^2 (so the common path needs no square root): bucket k
        // covers [lo2 + k*w, lo2 + (k+1)*w); the entry is the bin of the whole bucket
        // (63 = outside the bins) and bit 64 marks buckets that an edge, widened by
        // the FP32 error window, touches (those pairs are decided exactly in FP64)
        const double lo2 = std::max(rmin - 2 * tol, 0.0) * std::max(rmin - 2 * tol, 0.0);
        const double hi2 = (rmax + 2 * tol) * (rmax + 2 * tol);
        const double wb = (hi2 - lo2) / kTab;
        pp.tab_lo = (float)lo2;
        pp.tab_inv = (float)(1.0 / wb);
        for (int k = 0; k < kTab; ++k) {
            // widen the bucket by the FP32 error of r^2 and of the bucket index itself
            const double a2 = lo2 + (k - 1) * wb, b2 = lo2 + (k + 2) * wb;
            const double ra = std::sqrt(std::max(a2, 0.0)) - tol, rb = std::sqrt(b2) + tol;
            const double rc = std::sqrt(lo2 + (k + 0.5) * wb);
            int b = -1;
            for (int e = 0; e < nb; ++e)
                if (rc >= P->edges[e] && rc < P->edges[e + 1]) b = e;
            bool near = false;
            for (int e = 0; e <= nb; ++e)
                if (P->edges[e] >= ra && P->edges[e] <= rb) near = true;
            tab[k + 1] = (unsigned char)((b < 0 ? 63 : b) | (near ? 64 : 0));
        }
} else {
        // the 2-sphere: the table runs over the squared chord s = 2 - 2 cos(theta) (decreasing in
        // cos theta); an edge c_e sits at s_e = 2 - 2 c_e.  tol bounds the FP32 error of s from
        // normalised, shifted coordinates; flagged buckets are decided in FP64 from the input.
        const double tol = 1e-5;
        const double slo = std::max(2.0 - 2.0 * P->edges[nb] - tol, 0.0), shi = 2.0 - 2.0 * P->edges[0] + tol;
        pp.tol = (float)tol;
        pp.rmax2f = (float)shi;
        pp.rmin2f = (float)slo;
        for (int b = 0; b <= nb; ++b) {
            pp.edgef[b] = (float)P->edges[b];
            pp.edge2[b] = P->edges[b];  // cos theta edges, FP64
        }
        const double wb = (shi - slo) / kTab;
        pp.tab_lo = (float)slo;
        pp.tab_inv = (float)(1.0 / wb);
        for (int k = 0; k < kTab; ++k) {
            const double sa = slo + (k - 1) * wb - tol, sb = slo + (k + 2) * wb + tol;
            const double cc = 1.0 - 0.5 * (slo + (k + 0.5) * wb);
            int b = -1;
            for (int e = 0; e < nb; ++e)
                if (cc >= P->edges[e] && cc < P->edges[e + 1]) b = e;
            bool near = false;
            for (int e = 0; e <= nb; ++e) {
                const double se = 2.0 - 2.0 * P->edges[e];
                if (se >= sa && se <= sb) near = true;
            }
            tab[k + 1] = (unsigned char)((b < 0 ? 63 : b) | (near ? 64 : 0));
        }
    }
    CUDA_TRY(upload(P->d_tab, tab));
    std::vector<double> qn = component_norms(D, P->lmax);
    std::vector<double> ivb(nb);
    for (int b = 0; b < nb; ++b)
        ivb[b] = P->sphere ? 1.0 / (2.0 * M_PI * (P->edges[b + 1] - P->edges[b]))  // annulus area on S^2
                           : 1.0 / (sphere_area(D) / D * (std::pow(P->edges[b + 1], D) - std::pow(P->edges[b], D)));
    if (P->fp64) {
        CUDA_TRY(upload(P->d_qnorm, qn));
        CUDA_TRY(upload(P->d_invvb, ivb));
    } else {
        CUDA_TRY(upload(P->d_qnorm, cast_vec<float>(qn)));
        CUDA_TRY(upload(P->d_invvb, cast_vec<float>(ivb)));
    }
    pp.tab = P->d_tab.as<unsigned char>();
    pp.qnorm = P->d_qnorm.p;
    pp.inv_vb = P->d_invvb.p;

    // the visible outputs' columns, when a parity selection drops keys
    if (P->nvis != P->ncoeff) {
        std::vector<int> cm(2 * P->nvis);
        for (int64_t i = 0; i < P->nvis; ++i) {
            cm[2 * i] = (int)(2 * P->vis[i]);
            cm[2 * i + 1] = (int)(2 * P->vis[i] + 1);
        }
        CUDA_TRY(upload(P->d_colmap, cm));
    }
    // remove_self: the basis at coinciding directions, summed over the coupled states of label l
    // (addition theorem): (-1)^l sqrt(dim_l) / |S^{D-1}| for D >= 3, 1 / (2 pi) for D = 2; over v_b^2
    if (P->opts.remove_self && P->N == 3) {
        std::vector<double> sc((size_t)nb * (P->lmax + 1));
        for (int b = 0; b < nb; ++b)
            for (int l = 0; l <= P->lmax; ++l) {
                double c = 1.0 / (2.0 * M_PI);
                if (D == 3) c = cx::neg1_pow(l) * std::sqrt(2.0 * l + 1.0) / sphere_area(3);
                if (D == 4) c = cx::neg1_pow(l) * (l + 1.0) / sphere_area(4);
                sc[(size_t)b * (P->lmax + 1) + l] = c * ivb[b] * ivb[b];
            }
        if (P->fp64) CUDA_TRY(upload(P->d_selfc, sc));
        else CUDA_TRY(upload(P->d_selfc, cast_vec<float>(sc)));
    }

    // coupling tables
    std::vector<double> pref(P->lmax + 1, 1.0);
    for (int l = 0; l <= P->lmax; ++l) {
        if (D == 3) pref[l] = cx::neg1_pow(l) / std::sqrt(2.0 * l + 1.0);
        if (D == 4) pref[l] = cx::neg1_pow(l) / (double)(l + 1);
    }
    if (P->fp64) CUDA_TRY(upload(P->d_pref, pref));
    else CUDA_TRY(upload(P->d_pref, cast_vec<float>(pref)));
    std::vector<int2> lam2;
    std::vector<signed char> lamodd;
    for (int i = 0; i < P->nlam; ++i) {
        lam2.push_back(make_int2(P->lam[5 * i], P->lam[5 * i + 1]));
        lamodd.push_back((signed char)((P->lam[5 * i] + P->lam[5 * i + 1] + P->lam[5 * i + 2]) & 1));
    }
    CUDA_TRY(upload(P->d_lam2, lam2));
    CUDA_TRY(upload(P->d_lamodd, lamodd));
    if (P->N == 5) return build_d3n5f_tables(P);
    if (P->opts.basis == NPCF_BASIS_LOS) {
        // the terms of every label set: the CG chain ending in the state (L, 0)
        auto cg = [](int j1, int m1, int j2, int m2, int J, int M) {
            return cx::neg1_pow(j1 - j2 + M) * std::sqrt(2.0 * J + 1.0) * cx::wigner3j(j1, j2, J, m1, m2, -M);
        };
        auto st = [](int l, int m) { return l * l + l + m; };
        std::vector<int2> ll;
        std::vector<int> terms;
        std::vector<double> coef;
        for (int i = 0; i < P->nlam; ++i) {
            const int* l = &P->lam[5 * i];
            const int t0 = (int)terms.size();
            if (P->N == 3) {
                const int l1 = l[0], l2 = l[1], LL = l[2];
                for (int m = -l1; m <= l1; ++m) {
                    if (std::abs(m) > l2) continue;
                    const double c = cg(l1, m, l2, -m, LL, 0);
                    if (c == 0.0) continue;
                    terms.push_back(st(l1, m) | (st(l2, -m) << 8));
                    coef.push_back(c);
                }
            } else {
                const int l1 = l[0], l2 = l[1], l12 = l[2], l3 = l[3], LL = l[4];
                for (int m1 = -l1; m1 <= l1; ++m1)
                    for (int m2 = -l2; m2 <= l2; ++m2) {
                        const int m12 = m1 + m2;
                        if (std::abs(m12) > l12 || std::abs(m12) > l3) continue;
                        const double c = cg(l1, m1, l2, m2, l12, m12) * cg(l12, m12, l3, -m12, LL, 0);
                        if (c == 0.0) continue;
                        terms.push_back(st(l1, m1) | (st(l2, m2) << 8) | (st(l3, -m12) << 16));
                        coef.push_back(c);
                    }
            }
            ll.push_back(make_int2(t0, (int)terms.size()));
        }
        CUDA_TRY(upload(P->d_los_lam, ll));
        CUDA_TRY(upload(P->d_los_terms, terms));
        if (P->fp64) CUDA_TRY(upload(P->d_los_coef, coef));
        else CUDA_TRY(upload(P->d_los_coef, cast_vec<float>(coef)));
        build_key_blocks(P, (int)P->ncoeff);
        CUDA_TRY(upload(P->d_pairs, P->pairs));
        CUDA_TRY(upload(P->d_pair_key, P->pair_key));
        CUDA_TRY(upload(P->d_kblocks, P->kblocks));
        CUDA_TRY(upload(P->d_task, P->task_pairs));
        CoupleParams cp{};
        cp.nbins = nb;
        cp.lmax = P->lmax;
        cp.group = los_group(nb, P->lmax, P->fp64);
        if (couple_los_smem(cp, P->fp64) > P->smem_optin)
            return fail(NPCF_ERR_UNSUPPORTED, "the line-of-sight coupling needs more shared memory than available");
        return NPCF_OK;
    }
    // key blocks: accumulators get what shared memory the per-primary copy leaves
    CoupleParams cp{};
    cp.D = D;
    cp.N = P->N;
    cp.nbins = nb;
    cp.lmax = P->lmax;
    cp.nq = P->nq;
    cp.max_block_keys = 0;
    const int base = couple_smem(cp, P->fp64);
    const int comps = (P->N == 3 && D != 2) || (P->N == 4 && D == 3) ? 1 : 2;
    const int budget = std::min(P->smem_optin, 160 * 1024) - base;
    if (tc_coupling(P) && couple_tc_smem(nb, P->nq, P->mixed == 2) > P->smem_optin)
        return fail(NPCF_ERR_UNSUPPORTED, "the tensor-core coupling needs %d bytes of shared memory",
                    couple_tc_smem(nb, P->nq, P->mixed == 2));
    if (d2n4_registers(P)) {
        // the register kernel walks every (bin pair, label) item itself: one block of all keys
        if (base > P->smem_optin) return fail(NPCF_ERR_UNSUPPORTED, "D=2 4PCF coupling needs %d bytes of shared memory", base);
        build_key_blocks(P, (int)P->ncoeff);
    } else {
        build_key_blocks(P, std::max(1, budget / (comps * (P->fp64 ? 8 : 4))));
    }
    CUDA_TRY(upload(P->d_pairs, P->pairs));
    CUDA_TRY(upload(P->d_pair_key, P->pair_key));
    CUDA_TRY(upload(P->d_kblocks, P->kblocks));
    CUDA_TRY(upload(P->d_task, P->task_pairs));
    return NPCF_OK;
}

npcf_status prepare_grid(npcf_plan_s* P, int64_t n, bool adjoint = false)
{
    if (P->grid_n == n && P->grid_c > 0 && P->grid_adj == (int)adjoint) return NPCF_OK;
    GridChoice g = choose_grid(P, n, adjoint);
    if (g.c == 0)
        return fail(NPCF_ERR_UNSUPPORTED, "no cell grid fits r_max=%g in the box (need r_max < box/2.25)",
                    P->edges[P->nbins]);
    P->grid_c = g.c;
    for (int d = 0; d < 4; ++d) P->nc[d] = g.nc[d];
    P->ncells = g.ncells;
    P->nstencil = (int)g.stencil.size();
    CUDA_TRY(upload(P->d_stencil, stencil_with_rows(g.stencil, &P->nrows)));
    CUDA_TRY(upload(P->d_geo, std::vector<CatGeom>{make_geom(P->Dp, g.nc, P->box, 0, 0)}));
    P->grid_n = n;
    P->grid_adj = (int)adjoint;
    return NPCF_OK;
}

npcf_status reserve_workspace(npcf_plan_s* P, int64_t n, int64_t nprim_max, int rows, int ncells)
{
    const int rb = rec_bytes(P->Dp, P->fp64), tb = P->fp64 ? 8 : 4;
    const size_t nc = (size_t)ncells;
    auto R = [&](DevBuf& b, size_t bytes) -> npcf_status {
        if (b.reserve(bytes) != cudaSuccess)
            return fail(NPCF_ERR_WORKSPACE, "device allocation of %zu bytes failed", bytes);
        return NPCF_OK;
    };
    npcf_status st;
    if ((st = R(P->w_cid, sizeof(int) * (n + 1))) != NPCF_OK) return st;
    if ((st = R(P->w_perm, sizeof(int) * (n + 1))) != NPCF_OK) return st;
    if ((st = R(P->w_rec, (size_t)rb * (n + 1 + kRecPad))) != NPCF_OK) return st;
    // cells: count(nc+1) start(nc+1) fill(nc) lo prims pstart items istart (nc each) scan(8192)
    if ((st = R(P->w_cells, sizeof(int) * (8 * nc + 16 + 8192))) != NPCF_OK) return st;
    if ((st = R(P->w_items, sizeof(int4) * (n + nc + 1))) != NPCF_OK) return st;
    if ((st = R(P->w_a, (size_t)tb * std::max<int64_t>(nprim_max, 1) * P->nbins * P->nq)) != NPCF_OK) return st;
    if ((st = R(P->w_wprim, (size_t)tb * std::max<int64_t>(nprim_max, 1))) != NPCF_OK) return st;
    if (P->opts.remove_self && P->N == 3 &&
        (st = R(P->w_self, (size_t)tb * std::max<int64_t>(nprim_max, 1) * P->nbins)) != NPCF_OK)
        return st;
    if ((st = R(P->w_partial, sizeof(double) * rows * 2 * P->ncoeff)) != NPCF_OK) return st;
    if ((st = R(P->w_small, 128)) != NPCF_OK) return st;
    if (P->sphere && (st = R(P->w_upos, (size_t)tb * 3 * (n + 1))) != NPCF_OK) return st;
    return NPCF_OK;
}

// The cell grid a call runs on: one catalogue (the plan's box) or a batch.
struct GridView {
    int ncells = 0;
    int ncat = 1;
    const CatGeom* geo = nullptr;      // device, ncat
    const int64_t* offsets = nullptr;  // device, ncat + 1 (ncat > 1)
    const int* cat_cells = nullptr;    // device, ncat + 1 (ncat > 1)
    const int* stencil = nullptr;      // device (cells, then rows)
    int nstencil = 0;
    int nrows = 0;
};

GridView single_view(const npcf_plan_s* P)
{
    GridView v;
    v.ncells = P->ncells;
    v.geo = P->d_geo.as<CatGeom>();
    v.stencil = P->d_stencil.as<int>();
    v.nstencil = P->nstencil;
    v.nrows = P->nrows;
    return v;
}

// Coupling-kernel parameters for the plan's tables (one catalogue).
CoupleParams couple_params(const npcf_plan_s* P, const void* a, const void* wprim, const int* nprim, int chunk,
                           double* partial)
{
    CoupleParams kp{};
    kp.D = P->D;
    kp.N = P->N;
    kp.nbins = P->nbins;
    kp.lmax = P->lmax;
    kp.nq = P->nq;
    kp.nlam = P->nlam;
    kp.a = a;
    kp.wprim = wprim;
    kp.nprim = nprim;
    kp.chunk = chunk;
    kp.ncoeff = (int)P->ncoeff;
    kp.partial = partial;
    kp.pairs = P->d_pairs.as<int2>();
    kp.pair_key = P->d_pair_key.as<int>();
    kp.kblocks = P->d_kblocks.as<int4>();
    kp.nkb = (int)P->kblocks.size();
    kp.max_block_keys = P->max_block_keys;
    kp.max_block_pairs = P->max_block_pairs;
    kp.task_pairs = P->d_task.as<int>();
    kp.lam2 = P->d_lam2.as<int2>();
    kp.lam_odd = P->d_lamodd.as<signed char>();
    kp.pref = P->d_pref.p;
    kp.group = P->opts.basis == NPCF_BASIS_LOS ? los_group(P->nbins, P->lmax, P->fp64) : d2n4_group(P->nbins, P->lmax);
    kp.los_lam = P->d_los_lam.as<int2>();
    kp.los_terms = P->d_los_terms.as<int>();
    kp.los_coef = P->d_los_coef.p;
    kp.ncat = 1;
    kp.tc_npairs = (int)P->pairs.size();
    kp.tc_glam = tc_glam(P);
    int cols = 32;
    while (cols < kp.tc_glam * couple_tc_n(P->nbins)) cols *= 2;
    kp.tc_tmem_cols = cols;
    kp.tc_span = P->tc_span_t > 0 ? P->tc_span_t : tc_span();
    kp.self = (P->opts.remove_self && P->N == 3) ? P->w_self.p : nullptr;
    kp.selfc = P->d_selfc.p;
    return kp;
}

const int* plan_colmap(const npcf_plan_s* P) { return P->nvis != P->ncoeff ? P->d_colmap.as<int>() : nullptr; }

// The coupling stage of a plan: the tensor-core kernel for split-precision plans, the factored
// 5PCF kernels (per chunk of primaries, xs/zs their scratch), the CUDA-core kernels otherwise.
// rows: the partial rows per catalogue (the 5PCF's K slices).
npcf_status plan_coupling(npcf_plan_s* P, CoupleParams kp, int* err, int rows, int64_t nprim_max, void* xs, void* zs,
                          int npc, cudaStream_t s)
{
    kp.err = err;
    cudaError_t e;
    if (P->N == 5)
        return run_d3n5f(P, kp.a, kp.wprim, kp.nprim, nprim_max, kp.cat_first, kp.cat_count, kp.ncat, xs, zs, npc,
                         rows, kp.partial, err, s);
    if (tc_coupling(P))
        e = launch_couple_d2n4_tc(kp, P->mixed == 2, rows, tc_groups(P),
                                  couple_tc_smem(P->nbins, P->nq, P->mixed == 2), s);
    else if (P->opts.basis == NPCF_BASIS_LOS)
        e = launch_couple_los(kp, P->fp64, rows, couple_los_smem(kp, P->fp64), s);
    else
        e = launch_couple(kp, P->fp64, rows, couple_smem(kp, P->fp64), s);
    if (e != cudaSuccess) return fail(NPCF_ERR_CUDA, "coupling kernel launch: %s", cudaGetErrorString(e));
    return NPCF_OK;
}

// bytes of the factored 5PCF scratch (X and Z) for npc primaries per chunk and ncat catalogues
size_t d3n5f_scratch_bytes(const npcf_plan_s* P, int npc, int ncat)
{
    return (size_t)(P->d5_unit_x + P->d5_unit_z) * npc * ncat * 2 * (P->fp64 ? 8 : 4);
}

// What the cell-list and pair stages leave for the stages after them.
struct PairStage {
    ItemBuffers ib;
    PairParams pp;
    int* small = nullptr;
    unsigned long long* stats = nullptr;
};

// Cell list, work items and the pair kernel (the a-array of every primary in
// [pb, pe)), on workspace already reserved for n particles.
npcf_status run_pairs(npcf_plan_s* P, const GridView& gv, const void* pos, const void* w, int64_t n, int64_t pb,
                      int64_t pe, cudaStream_t s, PairStage* out)
{
    const int nc = gv.ncells;
    int* cells = P->w_cells.as<int>();
    int* cell_count = cells;                // nc + 1
    int* cell_start = cells + (nc + 1);     // nc + 1
    int* cell_fill = cells + 2 * (nc + 1);  // nc
    ItemBuffers ib;
    ib.cell_lo = cell_fill + nc;
    ib.cell_prims = ib.cell_lo + nc;
    ib.prim_start = ib.cell_prims + nc;
    ib.cell_items = ib.prim_start + nc;
    ib.item_start = ib.cell_items + nc;
    ib.scan_scratch = ib.item_start + nc;
    int* small = P->w_small.as<int>();
    ib.items = P->w_items.as<int4>();
    ib.nitems = small + S_NITEMS;
    ib.nprim = small + S_NPRIM;
    ib.ticket = small + S_TICKET;
    ib.ncat = gv.ncat;
    ib.cat_cells = gv.cat_cells;
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(small + 4);

    launch_counter() = 0;
    P->timed = 0;
    if (P->opts.timing) {
        for (auto& e : P->ev)
            if (!e) CUDA_TRY(cudaEventCreate(&e));
        CUDA_TRY(cudaEventRecord(P->ev[0], s));
    }
    CUDA_TRY(cudaMemsetAsync(cells, 0, sizeof(int) * (3 * (size_t)nc + 2), s));
    CUDA_TRY(cudaMemsetAsync(small, 0, 128, s));

    const void* orig = pos;
    if (P->sphere) {  // the cell search runs on the normalised directions, shifted into [0, 2]^3
        CUDA_TRY(launch_sphere_prep(pos, n, P->fp64, P->w_upos.p, s));
        pos = P->w_upos.p;
    }
    CellParams cp{};
    cp.D = P->Dp;
    cp.n = n;
    cp.ncells = nc;
    cp.ncat = gv.ncat;
    cp.geo = gv.geo;
    cp.offsets = gv.offsets;
    cp.periodic = P->opts.periodic;
    cp.pos = pos;
    cp.w = w;
    cp.cid = P->w_cid.as<int>();
    cp.cell_count = cell_count;
    cp.cell_start = cell_start;
    cp.cell_fill = cell_fill;
    cp.perm = P->w_perm.as<int>();
    cp.rec = P->w_rec.p;
    cp.err = small + S_ERR;
    CUDA_TRY(launch_cell_ids(cp, P->fp64, s));
    CUDA_TRY(launch_exclusive_scan(cell_count, cell_start, nc + 1, ib.scan_scratch, s));
    CUDA_TRY(launch_cell_scatter(cp, P->fp64, s));
    CUDA_TRY(launch_make_items(ib, cell_start, cp.perm, nc, pb, pe, P->warps, s));

    if (P->opts.timing) CUDA_TRY(cudaEventRecord(P->ev[1], s));
    PairParams pp = P->pp;
    pp.geo = gv.geo;
    pp.nstencil = gv.nstencil;
    pp.stencil = gv.stencil;
    pp.nrows = gv.nrows;
    pp.rows = reinterpret_cast<const int2*>(gv.stencil + ((gv.nstencil + 1) & ~1));
    pp.rec = P->w_rec.p;
    pp.cell_start = cell_start;
    pp.items = ib.items;
    pp.nitems = ib.nitems;
    pp.ticket = ib.ticket;
    pp.a_out = P->w_a.p;
    pp.w_out = P->w_wprim.p;
    pp.self_out = (P->opts.remove_self && P->N == 3) ? P->w_self.p : nullptr;
    pp.stats = stats;
    pp.perm = P->w_perm.as<int>();
    pp.orig = orig;
    const int grid = P->nsm;
    cudaError_t e;
    if (P->sphere) e = launch_pairs_sph(pp, P->fp64, P->Lc, grid, P->pair_smem, s);
    else if (P->D == 2) e = launch_pairs_d2(pp, P->fp64, P->Lc, grid, P->pair_smem, s);
    else if (P->D == 3) e = launch_pairs_d3(pp, P->fp64, P->Lc, grid, P->pair_smem, s);
    else e = launch_pairs_d4(pp, P->fp64, P->Lc, grid, P->pair_smem, s);
    if (e != cudaSuccess) return fail(NPCF_ERR_CUDA, "pair kernel launch: %s", cudaGetErrorString(e));
    if (P->opts.timing) CUDA_TRY(cudaEventRecord(P->ev[2], s));
    out->ib = ib;
    out->pp = pp;
    out->small = small;
    out->stats = stats;
    return NPCF_OK;
}

// Persistent rows (CTAs along x) of the coupling launch for nprim primaries: about two CTAs per
// SM over the key blocks; one per SM for the FP32 D=2 4PCF register kernel; for N=5 the K
// slices of the factored coupling.  Never more rows than there is work.
int couple_rows(const npcf_plan_s* P, int64_t nprim, int chunk)
{
    if (tc_coupling(P)) {  // one CTA per SM over (rows x label-set groups)
        const int64_t KP = couple_tc_chunk(P->mixed == 2);
        const int r = std::max(1, P->nsm / tc_groups(P));
        return (int)std::min<int64_t>(r, std::max<int64_t>(1, (nprim + KP - 1) / KP));
    }
    if (P->N == 5) return d3n5f_ksplit(P, d3n5f_chunk(P));
    if (P->opts.basis == NPCF_BASIS_LOS) {  // groups of los_group primaries
        const int G = los_group(P->nbins, P->lmax, P->fp64);
        const int mult = P->rows_mult > 0 ? P->rows_mult : 2;
        return (int)std::min<int64_t>(mult * P->nsm, std::max<int64_t>(1, (nprim + G - 1) / G));
    }
    const int nkb = (int)P->kblocks.size();
    const int mult = P->rows_mult > 0 ? P->rows_mult : 2;
    int rows = std::max(1, (mult * P->nsm) / std::max(nkb, 1));
    if (d2n4_registers(P)) rows = std::max(1, P->nsm * mult / 2);
    return (int)std::min<int64_t>(rows, std::max<int64_t>(1, (nprim + chunk - 1) / chunk));
}

npcf_status run(npcf_plan_s* P, const void* pos, const void* w, int64_t n, double* coeffs, int64_t pb, int64_t pe,
                cudaStream_t s)
{
    npcf_status st;
    if ((st = ensure_device(P)) != NPCF_OK) return st;
    if ((st = prepare_grid(P, n)) != NPCF_OK) return st;
    const int64_t nprim_max = pe - pb;
    const int chunk = 128;
    const int rows = couple_rows(P, nprim_max, chunk);
    if ((st = reserve_workspace(P, n, nprim_max, rows, P->ncells)) != NPCF_OK) return st;
    const int npc = P->N == 5 ? d3n5f_chunk(P) : 0;
    if (P->N == 5 && (P->w_x5.reserve(d3n5f_scratch_bytes(P, npc, 1)) != cudaSuccess))
        return fail(NPCF_ERR_WORKSPACE, "device allocation of the 5PCF scratch failed");
    PairStage ps;
    if ((st = run_pairs(P, single_view(P), pos, w, n, pb, pe, s, &ps)) != NPCF_OK) return st;
    const ItemBuffers& ib = ps.ib;
    int* small = ps.small;
    unsigned long long* stats = ps.stats;
    cudaError_t e;

    CoupleParams kp = couple_params(P, P->w_a.p, P->w_wprim.p, ib.nprim, chunk, P->w_partial.as<double>());
    CUDA_TRY(cudaMemsetAsync(kp.partial, 0, sizeof(double) * rows * 2 * P->ncoeff, s));
    if ((st = plan_coupling(P, kp, small + S_ERR, rows, nprim_max, P->w_x5.p,
                            P->w_x5.as<unsigned char>() + (size_t)P->d5_unit_x * npc * 2 * (P->fp64 ? 8 : 4), npc, s)) !=
        NPCF_OK)
        return st;
    if (P->opts.timing) CUDA_TRY(cudaEventRecord(P->ev[3], s));
    CUDA_TRY(launch_reduce(kp.partial, rows, (int)(2 * P->ncoeff), plan_colmap(P), (int)(2 * P->nvis), 1.0 / P->V,
                           coeffs, s));
    if (P->opts.timing) {
        CUDA_TRY(cudaEventRecord(P->ev[4], s));
        P->timed = 1;
    }
    P->last_launches = launch_counter();
    CUDA_TRY(cudaMemcpyAsync(P->h_small, small, 16, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(P->h_stats, stats, 64, cudaMemcpyDeviceToHost, s));
    P->last_stream = s;
    P->last_nprim = nprim_max;
    return NPCF_OK;
}

// The adjoint of the N=3 estimator: recompute the a-array with the forward
// cell-list and pair stages, then the coupling adjoint (per-primary
// c-coefficients and the primary-weight terms), then the pair adjoint (every
// pair's contribution to the positions and weights), then the conversion.
npcf_status run_backward(npcf_plan_s* P, const void* pos, const void* w, int64_t n, const double* g, int64_t pb,
                         int64_t pe, void* grad_pos, void* grad_w, cudaStream_t s)
{
    npcf_status st;
    if ((st = ensure_device(P)) != NPCF_OK) return st;
    if ((st = prepare_grid(P, n, true)) != NPCF_OK) return st;
    const int La = adjoint_compiled_lmax(P->D, P->lmax);
    if (La < 0) return fail(NPCF_ERR_UNSUPPORTED, "the adjoint is not compiled for D=%d lmax=%d", P->D, P->lmax);
    const int asmem = adjoint_pair_smem(P->D, La, P->fp64, P->nbins);
    if (asmem > P->smem_optin)
        return fail(NPCF_ERR_UNSUPPORTED, "the adjoint pair kernel needs %d bytes of shared memory", asmem);
    const int64_t nprim = pe - pb;
    if ((st = reserve_workspace(P, n, nprim, 1, P->ncells)) != NPCF_OK) return st;
    const size_t tb = P->fp64 ? 8 : 4;
    const size_t n1 = (size_t)std::max<int64_t>(n, 1), p1 = (size_t)std::max<int64_t>(nprim, 1);
    if (P->w_cbuf.reserve(tb * p1 * P->nbins * P->nq) != cudaSuccess ||
        P->w_gpos.reserve(sizeof(double) * P->D * n1) != cudaSuccess ||
        P->w_gw.reserve(sizeof(double) * n1) != cudaSuccess || P->w_gwp.reserve(sizeof(double) * p1) != cudaSuccess)
        return fail(NPCF_ERR_WORKSPACE, "device allocation of the adjoint workspace failed");
    if (P->d_keybase.bytes == 0) {
        std::vector<int> kb((size_t)P->nbins * P->nbins, -1);
        for (size_t pr = 0; pr < P->pairs.size(); ++pr)
            kb[(size_t)P->pairs[pr].x * P->nbins + P->pairs[pr].y] = P->pair_key[pr];
        CUDA_TRY(upload(P->d_keybase, kb));
    }
    PairStage ps;
    if ((st = run_pairs(P, single_view(P), pos, w, n, pb, pe, s, &ps)) != NPCF_OK) return st;
    // stage times: cell list, forward pair recompute (both from run_pairs), coupling adjoint, pair adjoint
    double* gpos = P->w_gpos.as<double>();
    double* gw = P->w_gw.as<double>();
    CUDA_TRY(cudaMemsetAsync(gpos, 0, sizeof(double) * P->D * n1, s));
    CUDA_TRY(cudaMemsetAsync(gw, 0, sizeof(double) * n1, s));
    cudaError_t e = launch_couple_adjoint(P->D, P->fp64, P->nbins, P->nq, P->lmax, nprim, P->w_a.p, P->w_wprim.p, g,
                                          (int)P->ncoeff,
                                          P->d_keybase.as<int>(), P->d_pref.p, P->d_qnorm.p, P->d_invvb.p,
                                          1.0 / P->V, P->w_cbuf.p, P->w_gwp.as<double>(), P->nsm, s);
    if (e != cudaSuccess) return fail(NPCF_ERR_CUDA, "coupling adjoint launch: %s", cudaGetErrorString(e));
    if (P->opts.timing) CUDA_TRY(cudaEventRecord(P->ev[3], s));
    // work items of adjoint_pair_warps() primaries (the a-array index of a primary does not depend on it)
    CUDA_TRY(launch_make_items(ps.ib, ps.pp.cell_start, P->w_perm.as<int>(), P->ncells, pb, pe,
                               adjoint_pair_warps(), s));
    e = launch_pairs_adjoint(ps.pp, P->fp64, La, P->w_cbuf.p, P->w_gwp.as<double>(), P->w_perm.as<int>(), gpos, gw,
                             P->nsm, s);
    if (e != cudaSuccess) return fail(NPCF_ERR_CUDA, "pair adjoint launch: %s", cudaGetErrorString(e));
    CUDA_TRY(launch_finalize_grads(n, P->D, P->fp64, gpos, gw, grad_pos, grad_w, s));
    if (P->opts.timing) {
        CUDA_TRY(cudaEventRecord(P->ev[4], s));
        P->timed = 1;
    }
    P->last_launches = launch_counter();
    CUDA_TRY(cudaMemcpyAsync(P->h_small, ps.small, 16, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(P->h_stats, ps.stats, 64, cudaMemcpyDeviceToHost, s));
    P->last_stream = s;
    P->last_nprim = nprim;
    return NPCF_OK;
}

// The cell grids of a batch.  Every catalogue is cut with the same
// subdivision c (cells of side >= r_max/c), so one stencil -- built for side
// exactly r_max/c, a superset of each catalogue's own -- serves them all;
// catalogue i's cells follow catalogue i-1's.  c minimises the same
// candidates-plus-overhead cost as the single-catalogue grid, summed over the
// catalogues.  Cached: an unchanged layout uploads nothing.
npcf_status prepare_batch(npcf_plan_s* P, const int64_t* offsets, const double* boxes, int ncat)
{
    std::vector<int64_t> off(offsets, offsets + ncat + 1);
    std::vector<double> bx(boxes, boxes + (size_t)ncat * P->D);
    if (P->b_ncat == ncat && P->b_key_off == off && P->b_key_box == bx) return NPCF_OK;
    const int D = P->D;
    const double rmax = P->edges[P->nbins];
    const double reach = rmax * (1.0 + 1e-6) + 1e-12;
    int best_c = 0;
    double best_cost = 1e300;
    std::vector<int> best_stencil;
    for (int c = 1; c <= 4; ++c) {
        double side[4] = {rmax / c, rmax / c, rmax / c, rmax / c};
        std::vector<int> st = make_stencil(D, c, side, reach);
        int nrows = 0;
        stencil_with_rows(st, &nrows);
        if (nrows > kMaxJobs) continue;
        bool ok = true;
        double cost = 0.0;
        int64_t total = 0;
        for (int i = 0; i < ncat && ok; ++i) {
            int64_t cells = 1;
            for (int d = 0; d < D; ++d) {
                int k = (int)std::floor(bx[(size_t)i * D + d] * c / rmax);
                if (k < 1) k = 1;
                if (P->opts.periodic && k < 2 * c + 1) ok = false;
                if (k > 4096) k = 4096;
                cells *= k;
            }
            total += cells;
            const double ni = (double)(off[i + 1] - off[i]);
            cost += ni * (st.size() * ni / cells + 40.0 * nrows);
        }
        if (!ok || total >= (int64_t(1) << 26)) continue;
        if (cost < best_cost) {
            best_cost = cost;
            best_c = c;
            best_stencil = st;
        }
    }
    if (best_c == 0)
        return fail(NPCF_ERR_UNSUPPORTED, "no common cell grid fits r_max=%g in every box (need r_max < box/2.25)",
                    rmax);
    std::vector<CatGeom> geo(ncat);
    std::vector<int> cells(ncat + 1), first(ncat), count(ncat);
    std::vector<double> scales(ncat);
    int base = 0;
    for (int i = 0; i < ncat; ++i) {
        int nc[4] = {1, 1, 1, 1};
        double V = 1.0;
        for (int d = 0; d < D; ++d) {
            const double b = bx[(size_t)i * D + d];
            nc[d] = std::min(4096, std::max(1, (int)std::floor(b * best_c / rmax)));
            V *= b;
        }
        geo[i] = make_geom(D, nc, &bx[(size_t)i * D], base, off[i]);
        cells[i] = base;
        first[i] = (int)off[i];
        count[i] = (int)(off[i + 1] - off[i]);
        scales[i] = 1.0 / V;
        base += geo[i].ncells;
    }
    cells[ncat] = base;
    P->b_ncat = 0;  // invalid until every upload succeeded
    CUDA_TRY(upload(P->b_geo, geo));
    CUDA_TRY(upload(P->b_cells, cells));
    CUDA_TRY(upload(P->b_offsets, off));
    CUDA_TRY(upload(P->b_first, first));
    CUDA_TRY(upload(P->b_count, count));
    CUDA_TRY(upload(P->b_scales, scales));
    CUDA_TRY(upload(P->b_stencil, stencil_with_rows(best_stencil, &P->b_nrows)));
    P->b_ncells = base;
    P->b_nstencil = (int)best_stencil.size();
    P->b_key_off = off;
    P->b_key_box = bx;
    P->b_ncat = ncat;
    return NPCF_OK;
}

// ncat catalogues in one pass: one cell list over all of them, one pair-kernel
// launch over every catalogue's work items (the persistent CTAs take items
// from one queue, so small and large catalogues share the GPU), one coupling
// launch with a grid layer per catalogue and one reduction that applies each
// catalogue's 1/V.
npcf_status run_batched(npcf_plan_s* P, const void* pos, const void* w, const int64_t* offsets, const double* boxes,
                        int ncat, double* coeffs, cudaStream_t s)
{
    npcf_status st;
    if ((st = ensure_device(P)) != NPCF_OK) return st;
    if ((st = prepare_batch(P, offsets, boxes, ncat)) != NPCF_OK) return st;
    const int64_t n = offsets[ncat];
    int64_t nmax = 0;
    for (int i = 0; i < ncat; ++i) nmax = std::max<int64_t>(nmax, offsets[i + 1] - offsets[i]);
    const int chunk = 128;
    const int nkb = (int)P->kblocks.size();
    // rows per catalogue: enough that the largest catalogue's row carries about the average CTA
    // load of 2 CTAs per SM (catalogues with fewer chunks than rows leave CTAs that exit at
    // once, and the hardware scheduler balances the rest), bounded by the partial-row memory
    const int64_t max_chunks = (nmax + chunk - 1) / chunk;
    const int64_t tot_chunks = std::max<int64_t>(1, (n + chunk - 1) / chunk);
    int64_t r64 = std::max<int64_t>((2 * P->nsm + nkb * ncat - 1) / (nkb * ncat),
                                    (max_chunks * 2 * P->nsm + tot_chunks - 1) / tot_chunks);
    const int64_t row_bytes = (int64_t)sizeof(double) * 2 * P->ncoeff * ncat;
    r64 = std::min<int64_t>(r64, std::max<int64_t>(1, (int64_t(512) << 20) / std::max<int64_t>(row_bytes, 1)));
    int rows = (int)std::min<int64_t>(r64, std::max<int64_t>(1, max_chunks));
    if (tc_coupling(P)) {  // one CTA per SM over (rows x label-set groups x catalogues)
        const int64_t KP = couple_tc_chunk(P->mixed == 2);
        rows = (int)std::min<int64_t>(std::max(1, P->nsm / (tc_groups(P) * ncat)),
                                      std::max<int64_t>(1, (nmax + KP - 1) / KP));
    }
    const int npc = P->N == 5 ? d3n5f_chunk(P) : 0;
    if (P->N == 5) rows = couple_rows(P, nmax, chunk);
    if ((st = reserve_workspace(P, n, n, rows * ncat, P->b_ncells)) != NPCF_OK) return st;
    if (P->N == 5 && (P->w_x5.reserve(d3n5f_scratch_bytes(P, npc, ncat)) != cudaSuccess))
        return fail(NPCF_ERR_WORKSPACE, "device allocation of the 5PCF scratch failed");
    GridView gv;
    gv.ncells = P->b_ncells;
    gv.ncat = ncat;
    gv.geo = P->b_geo.as<CatGeom>();
    gv.offsets = P->b_offsets.as<int64_t>();
    gv.cat_cells = P->b_cells.as<int>();
    gv.stencil = P->b_stencil.as<int>();
    gv.nstencil = P->b_nstencil;
    gv.nrows = P->b_nrows;
    PairStage ps;
    if ((st = run_pairs(P, gv, pos, w, n, 0, n, s, &ps)) != NPCF_OK) return st;
    CoupleParams kp = couple_params(P, P->w_a.p, P->w_wprim.p, ps.ib.nprim, chunk, P->w_partial.as<double>());
    kp.ncat = ncat;
    kp.cat_first = P->b_first.as<int>();
    kp.cat_count = P->b_count.as<int>();
    CUDA_TRY(cudaMemsetAsync(kp.partial, 0, sizeof(double) * rows * ncat * 2 * P->ncoeff, s));
    if ((st = plan_coupling(P, kp, ps.small + S_ERR, rows, nmax, P->w_x5.p,
                            P->w_x5.as<unsigned char>() +
                                (size_t)P->d5_unit_x * npc * ncat * 2 * (P->fp64 ? 8 : 4),
                            npc, s)) != NPCF_OK)
        return st;
    if (P->opts.timing) CUDA_TRY(cudaEventRecord(P->ev[3], s));
    CUDA_TRY(launch_reduce_cats(kp.partial, rows, (int)(2 * P->ncoeff), plan_colmap(P), (int)(2 * P->nvis), ncat,
                                P->b_scales.as<double>(), coeffs, s));
    if (P->opts.timing) {
        CUDA_TRY(cudaEventRecord(P->ev[4], s));
        P->timed = 1;
    }
    P->last_launches = launch_counter();
    CUDA_TRY(cudaMemcpyAsync(P->h_small, ps.small, 16, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(P->h_stats, ps.stats, 64, cudaMemcpyDeviceToHost, s));
    P->last_stream = s;
    P->last_nprim = n;
    return NPCF_OK;
}

npcf_status check_flags(npcf_plan_s* P)
{
    if (P->h_small[S_ERR] & 1) return fail(NPCF_ERR_NONFINITE, "a position or weight is NaN or infinite");
    if (P->h_small[S_ERR] & 2) return fail(NPCF_ERR_NONFINITE, "a position lies outside [0, box)");
    if (P->h_small[S_ERR] & 4)
        return fail(NPCF_ERR_DEVICE_TIMEOUT, "a bounded wait of the tensor-core coupling ran out; the call stopped");
    return NPCF_OK;
}

// ------------------------------------------------------------ gridded field
// The complex harmonic states kept in the a-array (m >= 0): their real and imaginary components.
std::vector<int2> complex_states(int D, int lmax)
{
    std::vector<int2> cs;
    if (D == 2)
        for (int l = 0; l <= lmax; ++l) cs.push_back(make_int2(q_index_d2(l), l > 0 ? q_index_d2(l) + 1 : -1));
    else if (D == 3)
        for (int l = 0; l <= lmax; ++l)
            for (int m = 0; m <= l; ++m) cs.push_back(make_int2(q_index_d3(l, m), m > 0 ? q_index_d3(l, m) + 1 : -1));
    else
        for (int l3 = 0; l3 <= lmax; ++l3)
            for (int l2 = 0; l2 <= l3; ++l2)
                for (int l1 = 0; l1 <= l2; ++l1)
                    cs.push_back(make_int2(q_index_d4(l3, l2, l1), l1 > 0 ? q_index_d4(l3, l2, l1) + 1 : -1));
    return cs;
}

npcf_status cufft_try(cufftResult r, const char* what)
{
    if (r != CUFFT_SUCCESS) return fail(NPCF_ERR_CUDA, "%s: cuFFT error %d", what, (int)r);
    return NPCF_OK;
}

// The FFT form of the gridded estimator: the kernels' transforms (cached per grid shape), the
// field's transform, per batch of (bin, state) pairs the spectral products, inverse transforms and
// the scatter into the a-array, then the plan's coupling over the nodes (weights dV X) and the
// reduction with 1/V.
npcf_status run_grid(npcf_plan_s* P, const void* X, const int* dims, double* coeffs, cudaStream_t s)
{
    npcf_status st;
    if ((st = ensure_device(P)) != NPCF_OK) return st;
    const int D = P->D;
    const size_t csz = P->fp64 ? 16 : 8;  // complex element
    GridParams g{};
    g.ncell = 1;
    g.dV = 1.0;
    for (int a = 0; a < D; ++a) {
        g.dims[a] = dims[a];
        g.spacing[a] = P->box[a] / dims[a];
        g.ncell *= dims[a];
        g.dV *= g.spacing[a];
    }
    for (int a = D; a < 4; ++a) g.dims[a] = 1;
    g.nbins = P->nbins;
    g.nq = P->nq;
    const double sa = sphere_area(D);
    for (int b = 0; b <= P->nbins; ++b) g.edge2[b] = P->edges[b] * P->edges[b];
    for (int b = 0; b < P->nbins; ++b)
        g.inv_vb[b] = 1.0 / (sa / D * (std::pow(P->edges[b + 1], D) - std::pow(P->edges[b], D)));
    const std::vector<int2> cs = complex_states(D, P->lmax);
    g.ncs = (int)cs.size();
    g.qnorm = P->d_qnorm.p;
    const int nbs_all = P->nbins * g.ncs;
    const bool same = P->g_ready && std::equal(dims, dims + D, P->g_dims);
    if (!same) {
        P->g_ready = false;
        P->g_nbs = (int)std::max<int64_t>(1, std::min<int64_t>(nbs_all, (int64_t(1) << 30) / (g.ncell * csz)));
        if (P->g_khat.reserve(csz * g.ncell * nbs_all) != cudaSuccess ||
            P->g_xhat.reserve(csz * g.ncell) != cudaSuccess ||
            P->g_work.reserve(csz * g.ncell * P->g_nbs) != cudaSuccess || P->g_small.reserve(16) != cudaSuccess)
            return fail(NPCF_ERR_WORKSPACE, "device allocation of the grid transforms failed");
        CUDA_TRY(upload(P->g_cstate, cs));
        if ((st = cufft_try(P->g_fft_k.make(D, dims, nbs_all, P->fp64), "kernel transform plan")) != NPCF_OK ||
            (st = cufft_try(P->g_fft_x.make(D, dims, 1, P->fp64), "field transform plan")) != NPCF_OK ||
            (st = cufft_try(P->g_fft_w.make(D, dims, P->g_nbs, P->fp64), "inverse transform plan")) != NPCF_OK)
            return st;
    }
    g.cstate = P->g_cstate.as<int2>();
    g.khat = P->g_khat.p;
    g.xhat = P->g_xhat.p;
    g.work = P->g_work.p;
    for (GridFFT* h : {&P->g_fft_k, &P->g_fft_x, &P->g_fft_w})
        if ((st = cufft_try(h->stream(s), "cufftSetStream")) != NPCF_OK) return st;
    auto fwd = [&](const GridFFT& h, void* data) { return h.exec(data, P->fp64, CUFFT_FORWARD); };
    auto inv = [&](const GridFFT& h, void* data) { return h.exec(data, P->fp64, CUFFT_INVERSE); };
    launch_counter() = 0;
    P->timed = 0;
    if (!same) {
        CUDA_TRY(cudaMemsetAsync(P->g_khat.p, 0, csz * g.ncell * nbs_all, s));
        CUDA_TRY(launch_grid_kernels(g, D, P->fp64, P->lmax, s));
        if ((st = cufft_try(fwd(P->g_fft_k, P->g_khat.p), "kernel transforms")) != NPCF_OK) return st;
        std::copy(dims, dims + D, P->g_dims);
        P->g_ready = true;
    }
    // the a-array and weights of the nodes (the nodes are the primaries)
    const int chunk = 128;
    const int rows = couple_rows(P, g.ncell, chunk);
    if ((st = reserve_workspace(P, 0, g.ncell, rows, 1)) != NPCF_OK) return st;
    g.a = P->w_a.p;
    g.wprim = P->w_wprim.p;
    CUDA_TRY(launch_grid_field(g, P->fp64, X, s));
    if ((st = cufft_try(fwd(P->g_fft_x, P->g_xhat.p), "field transform")) != NPCF_OK) return st;
    for (int bs0 = 0; bs0 < nbs_all; bs0 += P->g_nbs) {
        const int nbs = std::min(P->g_nbs, nbs_all - bs0);
        CUDA_TRY(launch_grid_product(g, P->fp64, bs0, nbs, s));
        if (nbs == P->g_nbs) {
            if ((st = cufft_try(inv(P->g_fft_w, P->g_work.p), "inverse transforms")) != NPCF_OK) return st;
        } else {
            for (int i = 0; i < nbs; ++i)  // a last, partial batch: one transform at a time
                if ((st = cufft_try(inv(P->g_fft_x, P->g_work.as<unsigned char>() + csz * g.ncell * i),
                                    "inverse transform")) != NPCF_OK)
                    return st;
        }
        CUDA_TRY(launch_grid_scatter(g, P->fp64, bs0, nbs, s));
    }
    // the coupling over the nodes, as for particles
    int* nprim_dev = P->g_small.as<int>();
    const int nc32 = (int)g.ncell;
    CUDA_TRY(cudaMemcpyAsync(nprim_dev, &nc32, sizeof(int), cudaMemcpyHostToDevice, s));
    const int npc = P->N == 5 ? d3n5f_chunk(P) : 0;
    if (P->N == 5 && (P->w_x5.reserve(d3n5f_scratch_bytes(P, npc, 1)) != cudaSuccess))
        return fail(NPCF_ERR_WORKSPACE, "device allocation of the 5PCF scratch failed");
    CoupleParams kp = couple_params(P, P->w_a.p, P->w_wprim.p, nprim_dev, chunk, P->w_partial.as<double>());
    CUDA_TRY(cudaMemsetAsync(kp.partial, 0, sizeof(double) * rows * 2 * P->ncoeff, s));
    CUDA_TRY(cudaMemsetAsync(P->w_small.p, 0, 128, s));  // flags, and zero pair statistics
    if ((st = plan_coupling(P, kp, P->w_small.as<int>() + S_ERR, rows, g.ncell, P->w_x5.p,
                            P->w_x5.as<unsigned char>() + (size_t)P->d5_unit_x * npc * 2 * (P->fp64 ? 8 : 4), npc,
                            s)) != NPCF_OK)
        return st;
    CUDA_TRY(launch_reduce(kp.partial, rows, (int)(2 * P->ncoeff), plan_colmap(P), (int)(2 * P->nvis), 1.0 / P->V,
                           coeffs, s));
    P->last_launches = launch_counter();
    CUDA_TRY(cudaMemcpyAsync(P->h_small, P->w_small.p, 16, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(P->h_stats, P->w_small.as<unsigned char>() + 64, 64, cudaMemcpyDeviceToHost, s));
    P->last_stream = s;
    P->last_nprim = g.ncell;
    return NPCF_OK;
}

// ------------------------------------------------------------ autotuning
// The launch shapes a plan may run with, searched on a bounded sample of the caller's input:
// the pair kernel's warps per CTA and batch size, then the coupling's CTAs per SM (CUDA-core
// kernels), FP32 span (tensor-core kernel) or primaries per chunk (factored 5PCF).  Each
// candidate runs the plan on the sample's primaries with CUDA events around its stages; the
// fastest stage time wins.  Choices are cached per (device, D, N, lmax, bins, precision, size
// class) in the file named by NPCF_TUNE_CACHE, if set.
struct TuneShape {
    int pair_warps = 0, pair_batch = 0, rows_mult = 0, tc_span = 0, d5_npc = 0;
    // the coupling's tunable: 0 rows_mult, 1 tc_span, 2 d5_npc
    int& coupling(int which) { return which == 0 ? rows_mult : (which == 1 ? tc_span : d5_npc); }
};

std::string tune_key(const npcf_plan_s* P, int64_t n)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, P->device);
    int nlog = 0;
    while ((int64_t(1) << (nlog + 1)) <= std::max<int64_t>(n, 1)) ++nlog;
    char buf[320];
    std::snprintf(buf, sizeof(buf), "%s|D=%d|N=%d|L=%d|nb=%d|prec=%d|self=%d|n=2^%d", prop.name, P->D, P->N, P->lmax,
                  P->nbins, P->opts.precision, P->opts.remove_self, nlog);
    for (char* c = buf; *c; ++c)
        if (*c == ' ' || *c == '\t' || *c == '\n') *c = '_';
    return buf;
}

bool tune_cache_load(const std::string& key, TuneShape* t)
{
    const char* path = std::getenv("NPCF_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[512], k[340];
    bool found = false;
    while (std::fgets(line, sizeof(line), f)) {
        TuneShape v;
        if (std::sscanf(line, "%339s %d %d %d %d %d", k, &v.pair_warps, &v.pair_batch, &v.rows_mult, &v.tc_span,
                        &v.d5_npc) == 6 &&
            key == k) {
            *t = v;  // the last entry of a key wins
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void tune_cache_store(const std::string& key, const TuneShape& t)
{
    const char* path = std::getenv("NPCF_TUNE_CACHE");
    if (!path || !*path) return;
    if (FILE* f = std::fopen(path, "a")) {
        std::fprintf(f, "%s %d %d %d %d %d\n", key.c_str(), t.pair_warps, t.pair_batch, t.rows_mult, t.tc_span,
                     t.d5_npc);
        std::fclose(f);
    }
}

void apply_shape(npcf_plan_s* P, const TuneShape& t)
{
    if (t.pair_warps > 0 && t.pair_batch > 0 && !set_pair_config(P, t.pair_warps, t.pair_batch))
        set_pair_config(P, P->max_warps, pair_batch(rec_bytes(P->D, P->fp64)));
    P->rows_mult = t.rows_mult;
    P->tc_span_t = t.tc_span;
    P->d5_npc = t.d5_npc;
}

// stage times (ms) of one run of the plan on primaries [0, pe): pair kernel, coupling
// Stage times of one pass over m primaries, taken as four ranges of m/4 spread over the input
// (inputs are often ordered -- e.g. data before randoms, or clustered points last -- so a single
// leading range would tune for one part of the catalogue only).
npcf_status time_stages(npcf_plan_s* P, const void* pos, const void* w, int64_t n, int64_t m, double* coeffs,
                        cudaStream_t s, float* pair_ms, float* couple_ms)
{
    *pair_ms = *couple_ms = 0.f;
    const int parts = (m < n && m >= 4 * 32) ? 4 : 1;  // the whole input: one pass, as the real call
    for (int k = 0; k < parts; ++k) {
        const int64_t pb = parts == 1 ? 0 : k * (n / parts), pe = pb + m / parts;
        npcf_status st = run(P, pos, w, n, coeffs, pb, std::min(pe, n), s);
        if (st != NPCF_OK) return st;
        float a = 0.f, b = 0.f;
        CUDA_TRY(cudaEventSynchronize(P->ev[4]));
        CUDA_TRY(cudaEventElapsedTime(&a, P->ev[1], P->ev[2]));
        CUDA_TRY(cudaEventElapsedTime(&b, P->ev[2], P->ev[3]));
        *pair_ms += a;
        *couple_ms += b;
    }
    return NPCF_OK;
}

// The coupling stage alone, again, on the a-array the last call left (nprim_max primaries, their
// count on the device where the pair stage put it); its time in *ms.
npcf_status time_coupling_only(npcf_plan_s* P, int64_t nprim_max, double* coeffs, cudaStream_t s, float* ms)
{
    const int chunk = 128;
    const int rows = couple_rows(P, nprim_max, chunk);
    if (P->w_partial.reserve(sizeof(double) * rows * 2 * P->ncoeff) != cudaSuccess)
        return fail(NPCF_ERR_WORKSPACE, "device allocation of the partial rows failed");
    const int npc = P->N == 5 ? d3n5f_chunk(P) : 0;
    if (P->N == 5 && (P->w_x5.reserve(d3n5f_scratch_bytes(P, npc, 1)) != cudaSuccess))
        return fail(NPCF_ERR_WORKSPACE, "device allocation of the 5PCF scratch failed");
    int* small = P->w_small.as<int>();
    CoupleParams kp = couple_params(P, P->w_a.p, P->w_wprim.p, small + S_NPRIM, chunk, P->w_partial.as<double>());
    CUDA_TRY(cudaEventRecord(P->ev[2], s));
    CUDA_TRY(cudaMemsetAsync(kp.partial, 0, sizeof(double) * rows * 2 * P->ncoeff, s));
    npcf_status st = plan_coupling(P, kp, small + S_ERR, rows, nprim_max, P->w_x5.p,
                                   P->w_x5.as<unsigned char>() + (size_t)P->d5_unit_x * npc * 2 * (P->fp64 ? 8 : 4),
                                   npc, s);
    if (st != NPCF_OK) return st;
    CUDA_TRY(cudaEventRecord(P->ev[3], s));
    CUDA_TRY(launch_reduce(kp.partial, rows, (int)(2 * P->ncoeff), plan_colmap(P), (int)(2 * P->nvis), 1.0 / P->V,
                           coeffs, s));
    CUDA_TRY(cudaEventSynchronize(P->ev[3]));
    CUDA_TRY(cudaEventElapsedTime(ms, P->ev[2], P->ev[3]));
    return NPCF_OK;
}

npcf_status autotune(npcf_plan_s* P, const void* pos, const void* w, int64_t n, cudaStream_t s)
{
    npcf_status st;
    if ((st = ensure_device(P)) != NPCF_OK) return st;
    const std::string key = tune_key(P, n);
    TuneShape best;
    const bool force = std::getenv("NPCF_TUNE_FORCE") != nullptr;
    if (!force && tune_cache_load(key, &best)) {
        apply_shape(P, best);
        P->tuned = 1;
        return NPCF_OK;
    }
    if (P->w_hout.reserve(sizeof(double) * 2 * P->nvis + 16) != cudaSuccess)
        return fail(NPCF_ERR_WORKSPACE, "device allocation of the tuning output failed");
    double* out = P->w_hout.as<double>();
    // the sample: enough primaries for several waves of pair-kernel items, at most all of them
    // (inputs up to 500k particles whole; larger ones a tenth: with smaller samples the short
    // runs' tail and cache behaviour favoured shapes that were slower over the whole input)
    const int64_t pe = n <= 500000 ? n : std::max<int64_t>(500000, n / 10);
    const npcf_opts saved = P->opts;
    P->opts.timing = 1;
    auto restore = [&]() { P->opts = saved; };
    // 1. the pair kernel: warps per CTA x batch size
    const int b0 = pair_batch(rec_bytes(P->D, P->fp64));
    const int batches[4] = {b0, b0 / 2, b0 * 3 / 4, b0 * 3 / 2};  // the built-in one first
    const int mw = P->max_warps;
    const int warps[3] = {mw, std::max(1, mw * 3 / 4), std::max(1, mw / 2)};
    float bestp = 1e30f;
    for (int wi = 0; wi < 3; ++wi)
        for (int bi = 0; bi < 4; ++bi) {
            if (wi > 0 && warps[wi] == warps[wi - 1]) continue;
            if (!set_pair_config(P, warps[wi], batches[bi]) || P->warps != warps[wi]) continue;
            float pm = 0.f, cm = 0.f;
            for (int rep = 0; rep < 2; ++rep)  // the first run warms caches and the cell grid
                if ((st = time_stages(P, pos, w, n, pe, out, s, &pm, &cm)) != NPCF_OK) {
                    restore();
                    return st;
                }
            // the built-in shape (all warps, the default batch) is timed first and kept unless
            // another is faster by more than 3% (timing noise)
            if (best.pair_warps == 0 || pm < 0.97f * bestp) {
                bestp = pm;
                best.pair_warps = P->warps;
                best.pair_batch = P->batch;
            }
        }
    if (best.pair_warps == 0) {
        best.pair_warps = mw;
        best.pair_batch = b0;
    }
    set_pair_config(P, best.pair_warps, best.pair_batch);
    // 2. the coupling's launch shape, timed alone on the a-array of a larger sample (a quarter of the
    // primaries): its grid is sized by the primary count, so a small sample misjudges it
    const int64_t pe2 = std::min<int64_t>(n, std::max<int64_t>(pe, n / 4));
    if ((st = run(P, pos, w, n, out, 0, pe2, s)) != NPCF_OK) {  // the a-array of primaries [0, pe2)
        restore();
        return st;
    }
    float bestc = 1e30f;
    int cand[4];
    int which;
    if (P->N == 5) {
        const int c0 = d3n5f_chunk(P, size_t(64) << 20);
        cand[0] = std::max(64, c0 / 4 / 64 * 64);
        cand[1] = std::max(64, c0 / 2 / 64 * 64);
        cand[2] = c0;
        cand[3] = std::min(1024, c0 * 2);
        which = 2;
    } else if (tc_coupling(P)) {
        cand[0] = 4, cand[1] = 8, cand[2] = 16, cand[3] = 32;
        which = 1;
    } else {
        cand[0] = 1, cand[1] = 2, cand[2] = 3, cand[3] = 4;
        which = 0;
    }
    for (int ci = 0; ci < 4; ++ci) {
        TuneShape t = best;
        t.coupling(which) = cand[ci];
        apply_shape(P, t);
        float cm = 0.f;
        for (int rep = 0; rep < 2; ++rep)
            if ((st = time_coupling_only(P, pe2, out, s, &cm)) != NPCF_OK) {
                restore();
                return st;
            }
        if (cm < bestc) {
            bestc = cm;
            best.coupling(which) = cand[ci];
        }
    }
    apply_shape(P, best);
    restore();
    P->tuned = 1;
    tune_cache_store(key, best);
    return NPCF_OK;
}

}  // namespace

// =================================================================== C ABI
extern "C" {

void npcf_default_opts(npcf_opts* o)
{
    if (!o) return;
    o->precision = NPCF_FP32;
    o->periodic = 1;
    o->bin_order = NPCF_BINS_LE;
    o->sync_check = 1;
    o->timing = 0;
    o->remove_self = 0;
    o->parity = NPCF_PARITY_ALL;
    o->basis = NPCF_BASIS_ISOTROPIC;
    o->geometry = NPCF_GEOMETRY_BOX;
}

npcf_status npcf_plan_create(npcf_plan_t* out, int D, int N, int lmax, const double* edges, int nbins,
                             const double* box, const npcf_opts* opts)
{
    if (!out) return fail(NPCF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (D < 2 || D > 4) return fail(NPCF_ERR_UNSUPPORTED, "D=%d not supported (2..4)", D);
    if (N < 3 || N > 5) return fail(NPCF_ERR_UNSUPPORTED, "N=%d not supported (3, 4 or 5)", N);
    if (N == 5 && D != 3) return fail(NPCF_ERR_UNSUPPORTED, "N=5 is provided for D=3 only");
    if (N == 5 && lmax > 6) return fail(NPCF_ERR_UNSUPPORTED, "N=5 supports lmax <= 6");
    if (N == 5 && nbins < 4) return fail(NPCF_ERR_ARG, "N=5 needs at least 4 bins");
    if (N == 4 && D == 4) return fail(NPCF_ERR_UNSUPPORTED, "N=4 needs the SO(4) coupling, not provided");
    if (lmax < 0) return fail(NPCF_ERR_ARG, "lmax must be >= 0");
    if (N == 4 && D == 3 && lmax > couple_max_lmax_d3n4())
        return fail(NPCF_ERR_UNSUPPORTED, "N=4, D=3 supports lmax <= %d", couple_max_lmax_d3n4());
    if (nbins < 1 || nbins > kMaxBins) return fail(NPCF_ERR_UNSUPPORTED, "nbins must be in [1, %d]", kMaxBins);
    if (N == 4 && nbins < 3) return fail(NPCF_ERR_ARG, "N=4 needs at least 3 bins");
    npcf_opts o;
    npcf_default_opts(&o);
    if (opts) o = *opts;
    if (o.geometry != NPCF_GEOMETRY_BOX && o.geometry != NPCF_GEOMETRY_SPHERE) return fail(NPCF_ERR_ARG, "bad geometry");
    const bool sph = o.geometry == NPCF_GEOMETRY_SPHERE;
    if (!edges || (!box && !sph)) return fail(NPCF_ERR_ARG, "bin_edges and box are required");
    if (sph) {
        if (D != 2 || N > 4)
            return fail(NPCF_ERR_UNSUPPORTED, "the 2-sphere takes D=2 (its basis) and N=3 or 4");
        if (!(edges[0] > -1.0) || !(edges[nbins] <= 1.0))
            return fail(NPCF_ERR_ARG, "cos(theta) edges must lie in (-1, 1]");
        if (o.remove_self || o.basis != NPCF_BASIS_ISOTROPIC)
            return fail(NPCF_ERR_UNSUPPORTED, "the 2-sphere is provided without remove_self and with the isotropic basis");
        if (pair_compiled_lmax_sph(o.precision == NPCF_FP64, lmax) < 0)
            return fail(NPCF_ERR_UNSUPPORTED, "lmax=%d is not compiled for the 2-sphere", lmax);
        o.periodic = 0;
    } else if (!(edges[0] >= 0.0) || !std::isfinite(edges[0])) {
        return fail(NPCF_ERR_ARG, "bin_edges[0] must be >= 0");
    }
    for (int b = 0; b < nbins; ++b)
        if (!(edges[b + 1] > edges[b]) || !std::isfinite(edges[b + 1]))
            return fail(NPCF_ERR_ARG, "bin_edges must be finite and strictly increasing");
    if (o.precision != NPCF_FP32 && o.precision != NPCF_FP64 && o.precision != NPCF_MIXED_BF16X3 &&
        o.precision != NPCF_MIXED_TF32X3)
        return fail(NPCF_ERR_ARG, "bad precision");
    const bool mixed = o.precision == NPCF_MIXED_BF16X3 || o.precision == NPCF_MIXED_TF32X3;
    if (mixed && !(D == 2 && N == 4) && !(D == 3 && N == 5 && o.precision == NPCF_MIXED_BF16X3))
        return fail(NPCF_ERR_UNSUPPORTED,
                    "the split-precision tensor-core coupling is provided for the D=2 4PCF (BF16x3, TF32x3) and the "
                    "D=3 5PCF (BF16x3)");
    if (mixed && N == 4 && (nbins - 1) * (nbins - 2) / 2 > 128)
        return fail(NPCF_ERR_UNSUPPORTED, "the tensor-core D=2 4PCF coupling takes at most 17 bins");
    if (o.bin_order != NPCF_BINS_LE && o.bin_order != NPCF_BINS_LT) return fail(NPCF_ERR_ARG, "bad bin_order");
    if (o.remove_self != 0 && o.remove_self != 1) return fail(NPCF_ERR_ARG, "remove_self must be 0 or 1");
    if (o.parity != NPCF_PARITY_ALL && o.parity != NPCF_PARITY_EVEN && o.parity != NPCF_PARITY_ODD)
        return fail(NPCF_ERR_ARG, "bad parity");
    if (o.basis != NPCF_BASIS_ISOTROPIC && o.basis != NPCF_BASIS_LOS) return fail(NPCF_ERR_ARG, "bad basis");
    if (o.basis == NPCF_BASIS_LOS &&
        (D != 3 || N > 4 || o.remove_self || o.parity != NPCF_PARITY_ALL || o.precision >= NPCF_MIXED_BF16X3))
        return fail(NPCF_ERR_UNSUPPORTED,
                    "the line-of-sight basis is provided for D=3, N=3 or 4, without remove_self, parity or mixed precision");
    if (o.parity == NPCF_PARITY_ODD && !(N == 4 && D == 3))
        return fail(NPCF_ERR_UNSUPPORTED, "this plan has no odd-parity components (only the D=3 4PCF has them)");
    for (int d = 0; d < D && !sph; ++d) {
        if (!(box[d] > 0.0) || !std::isfinite(box[d])) return fail(NPCF_ERR_ARG, "box sides must be > 0");
        if (o.periodic && !(edges[nbins] < 0.5 * box[d]))
            return fail(NPCF_ERR_ARG, "periodic boxes need r_max < box/2 (axis %d)", d);
    }
    npcf_plan_s* P = new (std::nothrow) npcf_plan_s;
    if (!P) return fail(NPCF_ERR_WORKSPACE, "out of host memory");
    P->D = D;
    P->N = N;
    P->lmax = lmax;
    P->nbins = nbins;
    P->opts = o;
    P->fp64 = o.precision == NPCF_FP64;
    P->mixed = o.precision == NPCF_MIXED_BF16X3 ? 1 : (o.precision == NPCF_MIXED_TF32X3 ? 2 : 0);
    P->edges.assign(edges, edges + nbins + 1);
    P->V = 1.0;
    if (sph) {
        // directions n + 1 fill the cube [0, 2]^3; the cell search reaches the largest chord
        P->sphere = 1;
        P->Dp = 3;
        for (int d = 0; d < 3; ++d) P->box[d] = 2.0 + std::ldexp(1.0, -20);
        P->V = 4.0 * M_PI;
        P->rcut = std::sqrt(2.0 - 2.0 * edges[0] + 2e-5);  // covers the table's widened range
    } else {
        P->Dp = D;
        P->rcut = edges[nbins];
        for (int d = 0; d < D; ++d) {
            P->box[d] = box[d];
            P->V *= box[d];
        }
    }
    build_keys(P);
    npcf_status st = ensure_device(P);
    if (st == NPCF_OK) st = setup_tables(P);
    if (st != NPCF_OK) {
        npcf_plan_destroy(P);
        return st;
    }
    *out = P;
    return NPCF_OK;
}

npcf_status npcf_num_coeffs(npcf_plan_t P, int64_t* n)
{
    if (!P || !n) return fail(NPCF_ERR_ARG, "NULL argument");
    *n = P->nvis;
    return NPCF_OK;
}

npcf_status npcf_coeff_index(npcf_plan_t P, int64_t i, int* bins, int* ells)
{
    if (!P || !bins || !ells) return fail(NPCF_ERR_ARG, "NULL argument");
    if (i < 0 || i >= P->nvis) return fail(NPCF_ERR_ARG, "index %lld out of range", (long long)i);
    const int64_t ki = P->vis[i];
    for (int k = 0; k < P->N - 1; ++k) bins[k] = P->key_bins[4 * ki + k];
    const int il = P->key_lam[ki];
    const int ne = P->opts.basis == NPCF_BASIS_LOS ? (P->N == 3 ? 3 : 5) : (P->N == 3 ? 1 : (P->N == 4 ? 3 : 5));
    for (int k = 0; k < ne; ++k) ells[k] = P->lam[5 * il + k];
    return NPCF_OK;
}

npcf_status npcf_compute(npcf_plan_t P, const void* pos, const void* w, int64_t n, double* coeffs, int64_t pb,
                         int64_t pe, npcf_stream_t stream)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    if (n < 0 || n > (int64_t)0x7fffff00) return fail(NPCF_ERR_ARG, "n=%lld out of range", (long long)n);
    if (!coeffs) return fail(NPCF_ERR_ARG, "coeffs is NULL");
    if (n > 0 && (!pos || !w)) return fail(NPCF_ERR_ARG, "positions/weights are NULL");
    if (pb == 0 && pe == 0) pe = n;
    if (pb < 0 || pe > n || pb > pe) return fail(NPCF_ERR_ARG, "primary range [%lld, %lld) outside [0, %lld)",
                                                 (long long)pb, (long long)pe, (long long)n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    npcf_status st = run(P, pos, w, n, coeffs, pb, pe, s);
    if (st != NPCF_OK) return st;
    if (P->opts.sync_check) {
        CUDA_TRY(cudaStreamSynchronize(s));
        return check_flags(P);
    }
    return NPCF_OK;
}

npcf_status npcf_compute_host(npcf_plan_t P, const void* pos, const void* w, int64_t n, double* coeffs,
                              int64_t pb, int64_t pe, npcf_stream_t stream)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    if (n < 0 || n > (int64_t)0x7fffff00) return fail(NPCF_ERR_ARG, "n=%lld out of range", (long long)n);
    if (!coeffs || (n > 0 && (!pos || !w))) return fail(NPCF_ERR_ARG, "bad arguments");
    if (pb == 0 && pe == 0) pe = n;
    if (pb < 0 || pe > n || pb > pe) return fail(NPCF_ERR_ARG, "primary range [%lld, %lld) outside [0, %lld)",
                                                 (long long)pb, (long long)pe, (long long)n);
    npcf_status st = ensure_device(P);
    if (st != NPCF_OK) return st;
    const size_t tb = P->fp64 ? 8 : 4;
    if (P->w_hpos.reserve(tb * P->Dp * std::max<int64_t>(n, 1)) != cudaSuccess ||
        P->w_hw.reserve(tb * std::max<int64_t>(n, 1)) != cudaSuccess ||
        P->w_hout.reserve(sizeof(double) * 2 * P->nvis + 16) != cudaSuccess)
        return fail(NPCF_ERR_WORKSPACE, "device staging allocation failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n > 0) {
        CUDA_TRY(cudaMemcpyAsync(P->w_hpos.p, pos, tb * P->Dp * n, cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(P->w_hw.p, w, tb * n, cudaMemcpyHostToDevice, s));
    }
    st = run(P, P->w_hpos.p, P->w_hw.p, n, P->w_hout.as<double>(), pb, pe, s);
    if (st != NPCF_OK) return st;
    CUDA_TRY(cudaMemcpyAsync(coeffs, P->w_hout.p, sizeof(double) * 2 * P->nvis, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return check_flags(P);
}

npcf_status npcf_device_status(npcf_plan_t P)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    CUDA_TRY(cudaStreamSynchronize(P->last_stream));
    return check_flags(P);
}

npcf_status npcf_last_stats(npcf_plan_t P, int64_t* pairs, int64_t* primaries, int64_t* candidates)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    CUDA_TRY(cudaStreamSynchronize(P->last_stream));
    if (pairs) *pairs = (int64_t)P->h_stats[0];
    if (candidates) *candidates = (int64_t)P->h_stats[1];
    if (primaries) *primaries = (int64_t)P->h_small[S_NPRIM];
    return NPCF_OK;
}

npcf_status npcf_last_profile(npcf_plan_t P, double* stage_ms, int* launches)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    CUDA_TRY(cudaStreamSynchronize(P->last_stream));
    if (launches) *launches = P->last_launches;
    if (stage_ms) {
        for (int i = 0; i < 4; ++i) {
            float ms = -1.0f;
            if (P->timed) CUDA_TRY(cudaEventElapsedTime(&ms, P->ev[i], P->ev[i + 1]));
            stage_ms[i] = ms;
        }
    }
    return NPCF_OK;
}

npcf_status npcf_last_counters(npcf_plan_t P, int64_t* counters, int n)
{
    if (!P || (!counters && n > 0)) return fail(NPCF_ERR_ARG, "NULL argument");
    CUDA_TRY(cudaStreamSynchronize(P->last_stream));
    for (int i = 0; i < n; ++i) counters[i] = i < 8 ? (int64_t)P->h_stats[i] : 0;
    return NPCF_OK;
}

npcf_status npcf_compute_batched(npcf_plan_t P, const void* pos, const void* w, const int64_t* offsets,
                                 const double* boxes, int ncat, double* coeffs, npcf_stream_t stream)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    if (P->sphere) return fail(NPCF_ERR_UNSUPPORTED, "%s is not provided for the 2-sphere", "npcf_compute_batched");
    if (ncat < 1 || ncat > (1 << 20)) return fail(NPCF_ERR_ARG, "ncat=%d out of range", ncat);
    if (!offsets || !boxes || !coeffs) return fail(NPCF_ERR_ARG, "offsets/boxes/coeffs is NULL");
    if (offsets[0] != 0) return fail(NPCF_ERR_ARG, "offsets[0] must be 0");
    for (int i = 0; i < ncat; ++i)
        if (offsets[i + 1] < offsets[i]) return fail(NPCF_ERR_ARG, "offsets decrease at catalogue %d", i);
    if (offsets[ncat] > (int64_t)0x7fffff00) return fail(NPCF_ERR_ARG, "n=%lld out of range", (long long)offsets[ncat]);
    for (int i = 0; i < ncat * P->D; ++i)
        if (!(boxes[i] > 0.0) || !std::isfinite(boxes[i]))
            return fail(NPCF_ERR_ARG, "box side %d of catalogue %d is not positive", i % P->D, i / P->D);
    if (offsets[ncat] > 0 && (!pos || !w)) return fail(NPCF_ERR_ARG, "positions/weights are NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    npcf_status st = run_batched(P, pos, w, offsets, boxes, ncat, coeffs, s);
    if (st != NPCF_OK) return st;
    if (P->opts.sync_check) {
        CUDA_TRY(cudaStreamSynchronize(s));
        return check_flags(P);
    }
    return NPCF_OK;
}

npcf_status npcf_backward(npcf_plan_t P, const void* pos, const void* w, int64_t n, const double* grad_coeffs,
                          int64_t pb, int64_t pe, void* grad_pos, void* grad_w, npcf_stream_t stream)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    if (P->sphere) return fail(NPCF_ERR_UNSUPPORTED, "%s is not provided for the 2-sphere", "npcf_backward");
    if (P->N != 3) return fail(NPCF_ERR_UNSUPPORTED, "the adjoint is implemented for N=3 plans");
    if (P->opts.remove_self)
        return fail(NPCF_ERR_UNSUPPORTED, "the adjoint of the remove_self subtraction is not provided");
    if (P->opts.basis != NPCF_BASIS_ISOTROPIC)
        return fail(NPCF_ERR_UNSUPPORTED, "the adjoint is implemented for the isotropic basis");
    if (n < 0 || n > (int64_t)0x7fffff00) return fail(NPCF_ERR_ARG, "n=%lld out of range", (long long)n);
    if (!grad_coeffs) return fail(NPCF_ERR_ARG, "grad_coeffs is NULL");
    if (n > 0 && !grad_pos && !grad_w) return fail(NPCF_ERR_ARG, "grad_positions and grad_weights are both NULL");
    if (n > 0 && (!pos || !w)) return fail(NPCF_ERR_ARG, "positions/weights are NULL");
    if (pb == 0 && pe == 0) pe = n;
    if (pb < 0 || pe > n || pb > pe) return fail(NPCF_ERR_ARG, "primary range [%lld, %lld) outside [0, %lld)",
                                                 (long long)pb, (long long)pe, (long long)n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    npcf_status st = run_backward(P, pos, w, n, grad_coeffs, pb, pe, grad_pos, grad_w, s);
    if (st != NPCF_OK) return st;
    if (P->opts.sync_check) {
        CUDA_TRY(cudaStreamSynchronize(s));
        return check_flags(P);
    }
    return NPCF_OK;
}

npcf_status npcf_selftest_tc(int tf32, int n, int k, const float* a, const float* b, float* d, npcf_stream_t stream)
{
    if (tf32 != 0 && tf32 != 1) return fail(NPCF_ERR_ARG, "tf32 must be 0 or 1");
    if (n < 16 || n > 256 || n % 16) return fail(NPCF_ERR_ARG, "n must be a multiple of 16 in [16, 256]");
    const int kq = tf32 ? 32 : 64;
    if (k < kq || k > 4096 || k % kq) return fail(NPCF_ERR_ARG, "k must be a positive multiple of %d, at most 4096", kq);
    if (!a || !b || !d) return fail(NPCF_ERR_ARG, "NULL argument");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int* err = nullptr;
    CUDA_TRY(cudaMalloc(&err, sizeof(int)));
    int herr = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = launch_tc_selftest(tf32, a, b, d, n, k, err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(err);
    if (e != cudaSuccess) return fail(NPCF_ERR_CUDA, "tensor-core self-test: %s", cudaGetErrorString(e));
    if (herr & 4) return fail(NPCF_ERR_DEVICE_TIMEOUT, "a bounded wait on the MMA completion ran out");
    return NPCF_OK;
}

npcf_status npcf_compute_grid(npcf_plan_t P, const void* field, const int* dims, double* coeffs, npcf_stream_t stream)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    if (P->sphere) return fail(NPCF_ERR_UNSUPPORTED, "%s is not provided for the 2-sphere", "npcf_compute_grid");
    if (!field || !dims || !coeffs) return fail(NPCF_ERR_ARG, "field/dims/coeffs is NULL");
    if (!P->opts.periodic) return fail(NPCF_ERR_UNSUPPORTED, "the gridded estimator needs a periodic plan");
    if (P->opts.basis != NPCF_BASIS_ISOTROPIC || P->mixed || P->opts.remove_self)
        return fail(NPCF_ERR_UNSUPPORTED, "the gridded estimator takes isotropic FP32/FP64 plans");
    if (P->lmax > grid_max_lmax()) return fail(NPCF_ERR_UNSUPPORTED, "the gridded estimator supports lmax <= %d", grid_max_lmax());
    int64_t ncell = 1;
    for (int a = 0; a < P->D; ++a) {
        if (dims[a] < 1) return fail(NPCF_ERR_ARG, "dims[%d] = %d", a, dims[a]);
        const double h = P->box[a] / dims[a];
        if (2 * (int64_t)std::floor(P->edges[P->nbins] / h) >= dims[a])
            return fail(NPCF_ERR_ARG, "r_max reaches half the grid on axis %d (need 2 floor(r_max / h) < dims)", a);
        ncell *= dims[a];
    }
    if (ncell > (int64_t(1) << 30)) return fail(NPCF_ERR_ARG, "grid of %lld nodes is too large", (long long)ncell);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    npcf_status st = run_grid(P, field, dims, coeffs, s);
    if (st != NPCF_OK) return st;
    if (P->opts.sync_check) {
        CUDA_TRY(cudaStreamSynchronize(s));
        return check_flags(P);
    }
    return NPCF_OK;
}

npcf_status npcf_autotune(npcf_plan_t P, const void* pos, const void* w, int64_t n, npcf_stream_t stream)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    if (n < 1 || n > (int64_t)0x7fffff00) return fail(NPCF_ERR_ARG, "n=%lld out of range", (long long)n);
    if (!pos || !w) return fail(NPCF_ERR_ARG, "positions/weights are NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    npcf_status st = autotune(P, pos, w, n, s);
    if (st != NPCF_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(s));
    return check_flags(P);
}

npcf_status npcf_tuned_config(npcf_plan_t P, int* values, int n)
{
    if (!P || (!values && n > 0)) return fail(NPCF_ERR_ARG, "NULL argument");
    const int v[6] = {P->warps, P->batch, P->rows_mult, P->tc_span_t, P->d5_npc, P->tuned};
    for (int i = 0; i < n; ++i) values[i] = i < 6 ? v[i] : 0;
    return NPCF_OK;
}

const char* npcf_last_error(void) { return g_err.c_str(); }

void npcf_plan_destroy(npcf_plan_t P)
{
    if (!P) return;
    DevBuf* bufs[] = {&P->d_task,  &P->d_tab,   &P->d_qnorm, &P->d_invvb, &P->d_pairs, &P->d_pair_key, &P->d_kblocks,
                      &P->d_lam2,  &P->d_lamodd, &P->d_pref, &P->d_stencil, &P->w_cid,    &P->w_perm,
                      &P->w_rec,   &P->w_cells, &P->w_items, &P->w_a,     &P->w_wprim,   &P->w_partial,
                      &P->w_small, &P->w_hpos,  &P->w_hw,    &P->w_hout,  &P->d_keybase, &P->w_cbuf, &P->w_upos,
                      &P->w_gpos,  &P->w_gw,    &P->w_gwp,   &P->d_geo,   &P->b_geo,     &P->b_cells,
                      &P->b_offsets, &P->b_first, &P->b_count, &P->b_scales, &P->b_stencil,
                      &P->d5_p12,  &P->d5_p34, &P->d5_gx,  &P->d5_gz, &P->d5_terms, &P->d5_coef, &P->d5_nlx,
                      &P->d5_nlz,  &P->d5_row0, &P->d5_col0, &P->d5_xrow, &P->d5_zcol, &P->d5_rowinfo,
                      &P->d5_colinfo, &P->d5_xoff, &P->d5_zoff, &P->d5_tiles, &P->d5_tctiles, &P->d5_tckeys, &P->d5_lamidx, &P->d5_trikey,
                      &P->w_x5,    &P->w_z5,
                      &P->d_colmap,  &P->d_selfc, &P->w_self, &P->d_los_lam, &P->d_los_terms, &P->d_los_coef,
                      &P->g_khat,  &P->g_xhat, &P->g_work, &P->g_cstate, &P->g_small};
    P->g_fft_k.destroy();
    P->g_fft_x.destroy();
    P->g_fft_w.destroy();
    for (DevBuf* b : bufs) b->release();
    if (P->h_small) cudaFreeHost(P->h_small);
    for (auto& e : P->ev)
        if (e) cudaEventDestroy(e);
    delete P;
}

}  // extern "C"

// ======================================================= allocation-free entry
// npcf_compute_noalloc: the npcf_compute pipeline with every device buffer it
// needs at compute time carved out of one file-scope __device__ array instead
// of plan workspace.  It exists for callers that must not allocate device
// memory once they are running: cudaMalloc synchronises the whole device and
// may fail under memory pressure, which real-time loops and code that shares
// the GPU with a caching allocator that owns all free memory cannot accept.
// Such callers create the plan (which allocates its small tables once) during
// set-up and then call this.  Each call copies the cell grid's stencil and
// geometry (a few KB) from host memory into the array before its kernels, and
// records no stage timings.
//
// The array below is part of the module: every GPU that loads libnpcf holds
// its kNoallocBytes until the process exits.  Host code must not use the
// symbol name as an address; the device address is obtained once per device
// with cudaGetSymbolAddress on the first call made on that device (so that
// first call should happen before any stream capture begins).
namespace {

constexpr size_t kNoallocBytes = size_t(16) << 20;  // 16 MiB of static scratch
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};
std::mutex g_noalloc_mu;

npcf_status noalloc_scratch(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) return fail(NPCF_ERR_UNSUPPORTED, "device index %d too large", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return fail(NPCF_ERR_CUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
    return NPCF_OK;
}

// bump allocator over the static scratch (256-byte aligned pieces)
struct Carve {
    unsigned char* base;
    size_t used = 0;
    size_t need = 0;
    void* take(size_t bytes)
    {
        size_t off = (used + 255) & ~size_t(255);
        used = off + bytes;
        need = used;
        return used <= kNoallocBytes ? base + off : nullptr;
    }
};

npcf_status run_noalloc(npcf_plan_s* P, const void* pos, const void* w, int64_t n, double* coeffs, int64_t pb,
                        int64_t pe, cudaStream_t s)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev != P->device) return fail(NPCF_ERR_ARG, "plan was created on device %d, current device is %d", P->device, dev);
    unsigned char* base = nullptr;
    npcf_status st = noalloc_scratch(dev, &base);
    if (st != NPCF_OK) return st;

    GridChoice g = choose_grid(P, n, false);
    if (g.c == 0) return fail(NPCF_ERR_UNSUPPORTED, "no cell grid fits r_max in the box");
    const int nc = g.ncells;
    const int64_t nprim_max = pe - pb;
    const int chunk = 128;
    const int rb = rec_bytes(P->D, P->fp64), tb = P->fp64 ? 8 : 4;

    Carve cv{base};
    CatGeom* geo = static_cast<CatGeom*>(cv.take(sizeof(CatGeom)));
    int nrows = 0;
    const std::vector<int> stencil_rows = stencil_with_rows(g.stencil, &nrows);
    int* stencil = static_cast<int*>(cv.take(sizeof(int) * stencil_rows.size()));
    int* cid = static_cast<int*>(cv.take(sizeof(int) * (n + 1)));
    int* perm = static_cast<int*>(cv.take(sizeof(int) * (n + 1)));
    void* rec = cv.take((size_t)rb * (n + 1 + kRecPad));
    int* cells = static_cast<int*>(cv.take(sizeof(int) * (8 * (size_t)nc + 16 + 8192)));
    int4* items = static_cast<int4*>(cv.take(sizeof(int4) * (n + nc + 1)));
    void* a = cv.take((size_t)tb * std::max<int64_t>(nprim_max, 1) * P->nbins * P->nq);
    void* wprim = cv.take((size_t)tb * std::max<int64_t>(nprim_max, 1));
    const bool self_on = P->opts.remove_self && P->N == 3;
    void* self = self_on ? cv.take((size_t)tb * std::max<int64_t>(nprim_max, 1) * P->nbins) : nullptr;
    int* small = static_cast<int*>(cv.take(128));
    const size_t row_bytes = sizeof(double) * 2 * P->ncoeff;
    size_t left = cv.used <= kNoallocBytes ? kNoallocBytes - ((cv.used + 255) & ~size_t(255)) : 0;
    int rows = couple_rows(P, nprim_max, chunk);  // as npcf_compute, bounded by the scratch left
    rows = (int)std::min<size_t>((size_t)rows, left / row_bytes);
    if (cv.used > kNoallocBytes || rows < 1) {
        size_t need = ((cv.need + 255) & ~size_t(255)) + row_bytes;
        return fail(NPCF_ERR_WORKSPACE,
                    "npcf_compute_noalloc needs %zu bytes of scratch for n=%lld; its static scratch holds %zu",
                    need, (long long)n, kNoallocBytes);
    }
    double* partial = static_cast<double*>(cv.take(row_bytes * rows));
    // the factored 5PCF's X and Z scratch: as many primaries per chunk as the array still holds
    int npc = 0;
    void *xs = nullptr, *zs = nullptr;
    if (P->N == 5) {
        const size_t left5 = cv.used <= kNoallocBytes ? kNoallocBytes - ((cv.used + 255) & ~size_t(255)) : 0;
        npc = d3n5f_chunk(P, left5 > 4096 ? left5 - 4096 : 1);
        const size_t xb = d3n5f_scratch_bytes(P, npc, 1), ub = (size_t)P->d5_unit_x * npc * 2 * tb;
        xs = cv.take(xb);
        zs = static_cast<unsigned char*>(xs) + ub;
        if (cv.used > kNoallocBytes)
            return fail(NPCF_ERR_WORKSPACE,
                        "npcf_compute_noalloc needs %zu bytes of scratch for n=%lld; its static scratch holds %zu",
                        (cv.need + 255) & ~size_t(255), (long long)n, kNoallocBytes);
    }

    CUDA_TRY(cudaMemcpyAsync(stencil, stencil_rows.data(), sizeof(int) * stencil_rows.size(), cudaMemcpyHostToDevice, s));
    const CatGeom hgeo = make_geom(P->D, g.nc, P->box, 0, 0);
    CUDA_TRY(cudaMemcpyAsync(geo, &hgeo, sizeof(CatGeom), cudaMemcpyHostToDevice, s));
    int* cell_count = cells;
    int* cell_start = cells + (nc + 1);
    int* cell_fill = cells + 2 * (nc + 1);
    ItemBuffers ib;
    ib.cell_lo = cell_fill + nc;
    ib.cell_prims = ib.cell_lo + nc;
    ib.prim_start = ib.cell_prims + nc;
    ib.cell_items = ib.prim_start + nc;
    ib.item_start = ib.cell_items + nc;
    ib.scan_scratch = ib.item_start + nc;
    ib.items = items;
    ib.nitems = small + S_NITEMS;
    ib.nprim = small + S_NPRIM;
    ib.ticket = small + S_TICKET;
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(small + 4);
    launch_counter() = 0;
    P->timed = 0;
    CUDA_TRY(cudaMemsetAsync(cells, 0, sizeof(int) * (3 * (size_t)nc + 2), s));
    CUDA_TRY(cudaMemsetAsync(small, 0, 128, s));

    CellParams cp{};
    cp.D = P->D;
    cp.n = n;
    cp.ncells = nc;
    cp.ncat = 1;
    cp.geo = geo;
    cp.periodic = P->opts.periodic;
    cp.pos = pos;
    cp.w = w;
    cp.cid = cid;
    cp.cell_count = cell_count;
    cp.cell_start = cell_start;
    cp.cell_fill = cell_fill;
    cp.perm = perm;
    cp.rec = rec;
    cp.err = small + S_ERR;
    CUDA_TRY(launch_cell_ids(cp, P->fp64, s));
    CUDA_TRY(launch_exclusive_scan(cell_count, cell_start, nc + 1, ib.scan_scratch, s));
    CUDA_TRY(launch_cell_scatter(cp, P->fp64, s));
    CUDA_TRY(launch_make_items(ib, cell_start, perm, nc, pb, pe, P->warps, s));

    PairParams pp = P->pp;
    pp.geo = geo;
    pp.nstencil = (int)g.stencil.size();
    pp.stencil = stencil;
    pp.nrows = nrows;
    pp.rows = reinterpret_cast<const int2*>(stencil + ((pp.nstencil + 1) & ~1));
    pp.rec = rec;
    pp.cell_start = cell_start;
    pp.items = ib.items;
    pp.nitems = ib.nitems;
    pp.ticket = ib.ticket;
    pp.a_out = a;
    pp.w_out = wprim;
    pp.self_out = self;
    pp.stats = stats;
    cudaError_t e;
    if (P->D == 2) e = launch_pairs_d2(pp, P->fp64, P->Lc, P->nsm, P->pair_smem, s);
    else if (P->D == 3) e = launch_pairs_d3(pp, P->fp64, P->Lc, P->nsm, P->pair_smem, s);
    else e = launch_pairs_d4(pp, P->fp64, P->Lc, P->nsm, P->pair_smem, s);
    if (e != cudaSuccess) return fail(NPCF_ERR_CUDA, "pair kernel launch: %s", cudaGetErrorString(e));

    CoupleParams kp = couple_params(P, a, wprim, ib.nprim, chunk, partial);
    kp.self = self;
    CUDA_TRY(cudaMemsetAsync(partial, 0, row_bytes * rows, s));
    if ((st = plan_coupling(P, kp, small + S_ERR, rows, nprim_max, xs, zs, npc, s)) != NPCF_OK) return st;
    CUDA_TRY(launch_reduce(partial, rows, (int)(2 * P->ncoeff), plan_colmap(P), (int)(2 * P->nvis), 1.0 / P->V,
                           coeffs, s));
    P->last_launches = launch_counter();
    CUDA_TRY(cudaMemcpyAsync(P->h_small, small, 16, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(P->h_stats, stats, 64, cudaMemcpyDeviceToHost, s));
    P->last_stream = s;
    P->last_nprim = nprim_max;
    return NPCF_OK;
}

}  // namespace

extern "C" npcf_status npcf_compute_noalloc(npcf_plan_t P, const void* pos, const void* w, int64_t n,
                                            double* coeffs, int64_t pb, int64_t pe, npcf_stream_t stream)
{
    if (!P) return fail(NPCF_ERR_ARG, "plan is NULL");
    if (P->sphere) return fail(NPCF_ERR_UNSUPPORTED, "%s is not provided for the 2-sphere", "npcf_compute_noalloc");
    if (n < 0 || n > (int64_t)0x7fffff00) return fail(NPCF_ERR_ARG, "n=%lld out of range", (long long)n);
    if (!coeffs) return fail(NPCF_ERR_ARG, "coeffs is NULL");
    if (n > 0 && (!pos || !w)) return fail(NPCF_ERR_ARG, "positions/weights are NULL");
    if (pb == 0 && pe == 0) pe = n;
    if (pb < 0 || pe > n || pb > pe) return fail(NPCF_ERR_ARG, "primary range [%lld, %lld) outside [0, %lld)",
                                                 (long long)pb, (long long)pe, (long long)n);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    npcf_status st = run_noalloc(P, pos, w, n, coeffs, pb, pe, s);
    if (st != NPCF_OK) return st;
    if (P->opts.sync_check) {
        CUDA_TRY(cudaStreamSynchronize(s));
        return check_flags(P);
    }
    return NPCF_OK;
}
