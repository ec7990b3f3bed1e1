/*
 * npcf.h -- C ABI of libnpcf, a GB300 (sm_103a) implementation of the
 * separable isotropic N-point correlation function estimator of
 * Philcox & Slepian, arXiv:2106.10278.
 *
 * What one call computes (eq. NPCF-estimator-discrete, Sec. "Application to
 * Discrete Data"): for every primary particle j, for every secondary k with
 * |y_k - y_j| in radial bin b,
 *     a^b_l(y_j) = (1/v_b) sum_k w_k Y*_l(unit(y_k - y_j)),
 * with Y_l the D-dimensional hyperspherical harmonics (eq. hypersph-def), and
 *     zeta^{0,b}_Lambda = (1/V_D) sum_j w_j sum_[l] C^{Lambda;0} prod_i a^{b_i}_{l^i}(y_j),
 * with C the zero-total-angular-momentum coupling (eq. Coupling-C,
 * eq. zero-ang-mom-states).  Supported: N=3 for D in {2,3,4}; N=4 for
 * D in {2,3}; N=5 for D=3 (eq. D=3-NPCF, intermediate label l12, lmax <= 6).
 * Euclidean space (k = 0 in eq. metric).
 *
 * Conventions (the readings of the paper this library takes):
 *   - bins are half-open [e_b, e_{b+1}); pairs with r = 0 are skipped;
 *   - v_b = |S^{D-1}|/D (e_{b+1}^D - e_b^D); V_D = product of the box sides;
 *   - periodic boxes use the minimum image (requires r_max < min(box)/2);
 *     non-periodic runs require every position inside [0, box) and use the
 *     box volume for V_D;
 *   - tuples with two equal secondaries are kept (as in the naive N-tuplet
 *     sum of eq. NPCF-estimator-intro-discrete);
 *   - N=3 keys: b1 <= b2 (NPCF_BINS_LE) or b1 < b2 (NPCF_BINS_LT), l = 0..lmax;
 *     N=4 keys: b1 < b2 < b3 and, for D=3, (l1, l2, l3) <= lmax obeying the
 *     triangle rule (both parities); for D=2, signed (l1, l2, l3) with
 *     l1 + l2 + l3 = 0, 0 <= l1 <= lmax, |l2|, |l3| <= lmax;
 *     N=5 keys (D=3): b1 < b2 < b3 < b4 and labels (l1, l2, l12, l3, l4) <= lmax
 *     with (l1, l2, l12), (l12, l3, l4) obeying the triangle rule and
 *     l1 + l2 + l3 + l4 even.
 *
 * Ownership: the caller owns every data buffer; the plan owns its tables and
 * device workspace.  All pointers named "device" must be device memory of the
 * current CUDA device; "host" pointers are ordinary host memory.
 * Errors: every entry point returns an npcf_status; npcf_last_error() gives a
 * thread-local message for the last failure.  No C++ exception crosses the ABI.
 */
#ifndef NPCF_H
#define NPCF_H

#include <stdint.h>

#if defined(__GNUC__)
#define NPCF_API __attribute__((visibility("default")))
#else
#define NPCF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct npcf_plan_s* npcf_plan_t; /* opaque; owned by the library */
typedef void* npcf_stream_t;             /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
    NPCF_OK = 0,
    NPCF_ERR_ARG = -1,            /* invalid argument or size (detected on the host) */
    NPCF_ERR_UNSUPPORTED = -2,    /* (D, N, lmax, nbins) or an option this build does not provide */
    NPCF_ERR_CUDA = -3,           /* a CUDA runtime call failed */
    NPCF_ERR_WORKSPACE = -4,      /* device allocation failed */
    NPCF_ERR_DEVICE_TIMEOUT = -5, /* a bounded device wait ran out (the tensor-core coupling's
                                     waits on its MMA completion barriers; the kernel
                                     then stops and the context stays usable) */
    NPCF_ERR_NONFINITE = -6,      /* a position or weight was NaN/Inf, or a position left the box */
} npcf_status;

/* npcf_opts.precision.  The two split-precision modes run the pair stage as NPCF_FP32 and
 * the coupling (the contraction over primaries of eq. NPCF-estimator-discrete) on the
 * tensor cores: every FP32 operand x is split into hi + lo of BF16 (MIXED_BF16X3) or TF32
 * (MIXED_TF32X3) and a product is kept as hi*hi + hi*lo + lo*hi with FP32 accumulation over
 * spans of primaries and FP64 sums across spans.  Provided for the D=2 4PCF (both splits, at
 * most 17 bins) and for the D=3 5PCF (MIXED_BF16X3: the contraction over (primary, m12) of
 * the coupling factored through l12, FP32 accumulation over a piece of K of one chunk of
 * primaries, FP64 across pieces and chunks); other plans return NPCF_ERR_UNSUPPORTED. */
enum { NPCF_FP64 = 0, NPCF_FP32 = 1, NPCF_MIXED_BF16X3 = 2, NPCF_MIXED_TF32X3 = 3 };
enum { NPCF_BINS_LE = 0, NPCF_BINS_LT = 1 };    /* npcf_opts.bin_order (N=3 only) */
/* npcf_opts.parity: which components a plan returns, by their behaviour under r -> -r (the
 * basis parity (-1)^(l1+l2+l3) of eq. B-hypersph; the odd ones are imaginary).  Only the D=3
 * 4PCF has odd components: N=3 and the D=2 4PCF are even (in D=2, r -> -r is a rotation) and the
 * 5PCF keys are the even label sets, so NPCF_PARITY_ODD is refused for them. */
enum { NPCF_PARITY_ALL = 0, NPCF_PARITY_EVEN = 1, NPCF_PARITY_ODD = 2 };
/* npcf_opts.basis.  NPCF_BASIS_ISOTROPIC: the zero-total-angular-momentum basis of
 * eq. Coupling-C (every key above).  NPCF_BASIS_LOS (D = 3, N = 3 or 4): the basis about the
 * fixed x_3 line of sight of Sec. "Large-Scale Structure" -- the coupling's final state is (L, 0)
 * for every L the labels allow, N=3 keys (b1, b2; l1, l2, L) with l1, l2 <= lmax and
 * |l1 - l2| <= L <= l1 + l2, coupling <l1 m l2 -m|L 0>; N=4 keys (b1 < b2 < b3; l1, l2, l12, l3, L)
 * through <l1 m1 l2 m2|l12 m12><l12 m12 l3 m3|L 0>.  L = 0 gives the isotropic coefficients.
 * Coefficients are complex; npcf_coeff_index returns 3 (N=3) or 5 (N=4) labels.  Not with
 * remove_self, a parity selection, the mixed precisions or npcf_backward. */
enum { NPCF_BASIS_ISOTROPIC = 0, NPCF_BASIS_LOS = 1 };
/* npcf_opts.geometry.  NPCF_GEOMETRY_BOX: Euclidean positions in a box (everything above).
 * NPCF_GEOMETRY_SPHERE: points on the unit 2-sphere (Sec. "Cosmic Microwave Background"), with
 * the D = 2 basis about every primary: the plan has D = 2 and N = 3 or 4; a position is a
 * 3-vector (any nonzero length; the library normalises it); the radial coordinate is the
 * great-circle angle theta between two points, binned on cos theta in half-open intervals
 * [c_b, c_{b+1}) of bin_edges (-1 < c_0 < ... < c_nbins <= 1); the azimuth is that of the
 * tangent vector n_k - (n_j . n_k) n_j in a right-handed frame (e1, e2, n_j); v_b = 2 pi
 * (c_{b+1} - c_b) and 1/(4 pi) replaces 1/V_D.  box is ignored (may be NULL), periodic is
 * ignored.  Not with remove_self, the line-of-sight basis, npcf_backward,
 * npcf_compute_batched, npcf_compute_noalloc or npcf_compute_grid. */
enum { NPCF_GEOMETRY_BOX = 0, NPCF_GEOMETRY_SPHERE = 1 };

typedef struct {
    int precision;  /* NPCF_FP32 (positions/weights float, pair and coupling arithmetic FP32,
                       cross-primary sums FP64), NPCF_FP64 (double throughout), or
                       NPCF_MIXED_BF16X3 / NPCF_MIXED_TF32X3 (float inputs, FP32 pairs,
                       split-precision tensor-core coupling; see above) */
    int periodic;   /* 1: minimum image in the box; 0: open boundaries */
    int bin_order;  /* NPCF_BINS_LE (default) or NPCF_BINS_LT, N=3 only */
    int sync_check; /* 1 (default): npcf_compute waits for the stream and reports
                       device-detected input errors; 0: fully asynchronous, query
                       them later with npcf_device_status */
    int timing;     /* 1: record CUDA events between the stages of every compute
                       (read with npcf_last_profile); 0 (default): none */
    int remove_self; /* 0 (default): keep the tuples whose secondaries coincide, as the
                       naive N-tuplet sum of eq. NPCF-estimator-intro-discrete does; 1:
                       subtract them exactly.  Only N=3 keys with b1 = b2 have such tuples:
                       per primary j, sum_{k in b} w_k^2 c_l / v_b^2 is removed, c_l the
                       basis at coinciding directions ((-1)^l sqrt(dim_l)/|S^{D-1}| for
                       D >= 3, 1/(2 pi) for D = 2).  npcf_backward refuses such plans. */
    int parity;     /* NPCF_PARITY_ALL (default), NPCF_PARITY_EVEN or NPCF_PARITY_ODD: the
                       keys the plan returns (npcf_num_coeffs / npcf_coeff_index count and
                       label only those) */
    int basis;      /* NPCF_BASIS_ISOTROPIC (default) or NPCF_BASIS_LOS (see above) */
    int geometry;   /* NPCF_GEOMETRY_BOX (default) or NPCF_GEOMETRY_SPHERE (see above) */
} npcf_opts;

/* Default options: FP32, periodic, b1 <= b2, sync_check = 1, timing = 0, remove_self = 0,
 * parity = NPCF_PARITY_ALL, basis = NPCF_BASIS_ISOTROPIC, geometry = NPCF_GEOMETRY_BOX. */
NPCF_API void npcf_default_opts(npcf_opts* opts);

/*
 * Build a plan (host call; allocates the coupling tables on the current device).
 *   D, N, lmax : dimension (2..4), order (3, 4 or 5), maximum total angular momentum.
 *   bin_edges  : host, nbins+1 ascending edges, bin_edges[0] >= 0; r_max = bin_edges[nbins]
 *                (NPCF_GEOMETRY_SPHERE: cos theta edges, -1 < bin_edges[0], bin_edges[nbins] <= 1).
 *   box        : host, D side lengths (> 0).  Required in both periodic modes (gives V_D);
 *                ignored (may be NULL) for NPCF_GEOMETRY_SPHERE.
 *   opts       : host, may be NULL for the defaults.
 * Errors: NPCF_ERR_ARG for bad sizes/edges/box, NPCF_ERR_UNSUPPORTED for
 * combinations outside the list above (or nbins > 32), NPCF_ERR_CUDA.
 */
NPCF_API npcf_status npcf_plan_create(npcf_plan_t* out, int D, int N, int lmax, const double* bin_edges, int nbins,
                             const double* box, const npcf_opts* opts);

/* Number of output coefficients (each one complex: 2 doubles). */
NPCF_API npcf_status npcf_num_coeffs(npcf_plan_t plan, int64_t* ncoeff);

/* Labels of coefficient i: bins (N-1 entries, host) and ells (host; 1 for N=3: l; 3 for N=4:
 * l1, l2, l3; 5 for N=5: l1, l2, l12, l3, l4; with NPCF_BASIS_LOS 3 for N=3: l1, l2, L and 5 for
 * N=4: l1, l2, l12, l3, L).  N=5 keys have b1 < b2 < b3 < b4 and the even-parity label sets
 * (l1 + l2 + l3 + l4 even), 585 of them at lmax = 4. */
NPCF_API npcf_status npcf_coeff_index(npcf_plan_t plan, int64_t i, int* bins, int* ells);

/*
 * Compute the coefficients.
 *   positions : device, n x D row-major (n x 3 for NPCF_GEOMETRY_SPHERE), float (NPCF_FP32) or
 *               double (NPCF_FP64).
 *   weights   : device, n, same type.
 *   coeffs    : device, 2*ncoeff doubles (re, im), overwritten.
 *   [primary_begin, primary_end): the primaries summed over (indices into the
 *               input arrays); every particle is a secondary.  0, n = all.
 *   stream    : the CUDA stream every kernel is launched on.
 * Asynchronous on `stream` when opts.sync_check == 0.  Errors: NPCF_ERR_ARG
 * (bad n or range), NPCF_ERR_NONFINITE (sync_check only), NPCF_ERR_WORKSPACE,
 * NPCF_ERR_CUDA.  A plan must not be used by two calls at the same time.
 */
NPCF_API npcf_status npcf_compute(npcf_plan_t plan, const void* positions, const void* weights, int64_t n, double* coeffs,
                         int64_t primary_begin, int64_t primary_end, npcf_stream_t stream);

/*
 * Same as npcf_compute with host buffers: positions/weights are host arrays,
 * coeffs a host array of 2*ncoeff doubles.  Copies in, computes and copies out
 * on `stream`, then waits for it.
 */
NPCF_API npcf_status npcf_compute_host(npcf_plan_t plan, const void* positions, const void* weights, int64_t n,
                              double* coeffs, int64_t primary_begin, int64_t primary_end, npcf_stream_t stream);

/*
 * The coefficients of ncat independent catalogues in one pass: one cell list
 * over all of them, one persistent pair-kernel launch whose CTAs take work
 * items of every catalogue from one queue, one coupling launch and one
 * reduction (eq. NPCF-estimator-discrete applied to each catalogue on its own;
 * the paper has no batched form, this exists to keep many small catalogues
 * from leaving the GPU idle between calls).
 *   positions, weights : device, the catalogues concatenated (n = offsets[ncat]
 *               rows), plan precision; catalogue i is rows [offsets[i], offsets[i+1]).
 *   offsets    : host, ncat + 1 nondecreasing values, offsets[0] = 0.
 *   boxes      : host, ncat x D side lengths; catalogue i lies in [0, box_i) with
 *               V_i = prod box_i; the plan's own box is not used.  Periodic plans
 *               need r_max < box/2.25 on every side of every box.
 *   coeffs     : device, ncat x 2*ncoeff doubles (catalogue-major), overwritten.
 * Every particle of a catalogue is a primary of that catalogue.  The layout is
 * cached: a repeated call with the same offsets and boxes copies no tables.
 * Errors: NPCF_ERR_ARG, NPCF_ERR_UNSUPPORTED (no common grid), NPCF_ERR_NONFINITE
 * (sync_check only), NPCF_ERR_WORKSPACE, NPCF_ERR_CUDA.
 */
NPCF_API npcf_status npcf_compute_batched(npcf_plan_t plan, const void* positions, const void* weights,
                                          const int64_t* offsets, const double* boxes, int ncat, double* coeffs,
                                          npcf_stream_t stream);

/*
 * Coefficients of a field sampled on a periodic grid (Sec. "Application to
 * Gridded Data"): the integrals of eq. alm-bin-def and eq. NPCF-mult-estimator
 * become sums over nodes times the node volume dV = prod_a box[a]/dims[a], the
 * offset 0 is skipped and a^b_l keeps the 1/v_b of the particle estimator:
 *   a^b_l(c) = (1/v_b) sum_{u != 0} dV X(c + u) Y*_l(unit(u)) Theta^b(|u|),
 *   zeta     = (1/V) sum_c dV X(c) sum_[l] C prod_i a^{b_i}_{l^i}(c).
 * The sum over offsets is evaluated as a circular convolution through FFTs
 * (cuFFT, one forward transform of the field, one inverse per (bin, harmonic
 * state)); the kernels' transforms are cached in the plan for the last grid
 * shape.  The coupling is the plan's, with the nodes as primaries.
 *   field   : device, prod(dims) values of the plan's precision, row-major (the
 *             last axis fastest); node c sits at c_a box[a]/dims[a].
 *   dims    : host, D node counts; 2 floor(r_max / h_a) < dims[a] on every axis
 *             (every offset within r_max reaches a distinct node).
 *   coeffs  : device, 2*ncoeff doubles, overwritten.
 * Plans: periodic, isotropic basis, FP32 or FP64, lmax <= 6, no remove_self.
 * Device memory: 8 (FP32) or 16 (FP64) bytes x nodes x nbins x (complex
 * harmonic states) for the cached kernel transforms, plus the particle path's
 * workspace for prod(dims) primaries.
 * Errors: NPCF_ERR_ARG, NPCF_ERR_UNSUPPORTED, NPCF_ERR_WORKSPACE, NPCF_ERR_CUDA
 * (cuFFT failures included).
 */
NPCF_API npcf_status npcf_compute_grid(npcf_plan_t plan, const void* field, const int* dims, double* coeffs,
                                       npcf_stream_t stream);

/*
 * Gradient of a scalar loss through the N=3 estimator (the adjoint of
 * eq. NPCF-estimator-discrete for N=3; the inner sums of eq. alm-bin-def are
 * differentiated with the radial bin of every pair held fixed, the bin
 * indicators being piecewise constant in the separation).
 *   positions, weights, n, [primary_begin, primary_end), stream : as for
 *               npcf_compute (the same call computes the same coefficients).
 *   grad_coeffs : device, 2*ncoeff doubles: dL/dRe and dL/dIm of each coefficient.
 *   grad_positions : device, n x D row-major in the plan's precision, or NULL;
 *               overwritten with dL/dy_i (minimum-image separations when periodic).
 *   grad_weights   : device, n in the plan's precision, or NULL; overwritten with dL/dw_i.
 *               At least one of the two must be given when n > 0.
 * Per-particle sums are accumulated in FP64 with atomics (not bit-reproducible
 * from call to call).  Asynchronous on `stream` when opts.sync_check == 0.
 * Errors: NPCF_ERR_UNSUPPORTED for N=4 plans or lmax without a compiled
 * adjoint, NPCF_ERR_ARG, NPCF_ERR_NONFINITE (sync_check only),
 * NPCF_ERR_WORKSPACE, NPCF_ERR_CUDA.
 */
NPCF_API npcf_status npcf_backward(npcf_plan_t plan, const void* positions, const void* weights, int64_t n,
                                   const double* grad_coeffs, int64_t primary_begin, int64_t primary_end,
                                   void* grad_positions, void* grad_weights, npcf_stream_t stream);

/* Device-side input errors flagged by the last asynchronous npcf_compute (waits for its stream). */
NPCF_API npcf_status npcf_device_status(npcf_plan_t plan);

/*
 * Per-launch statistics of the last npcf_compute (host, after the stream has
 * finished): ordered pairs accumulated, primaries processed, candidate
 * secondaries examined.  Any pointer may be NULL.
 */
NPCF_API npcf_status npcf_last_stats(npcf_plan_t plan, int64_t* pairs, int64_t* primaries, int64_t* candidates);

/*
 * Stage timings and kernel count of the last npcf_compute or npcf_backward (host, waits for its
 * stream).  stage_ms (may be NULL) receives 4 values measured with CUDA events
 * on the compute stream when opts.timing = 1 (else -1): cell list + work items,
 * pair kernel, coupling kernel, final reduction; after npcf_backward: cell list +
 * work items, the forward pair kernel (recomputing the a-array), the coupling
 * adjoint, the pair adjoint + conversion.  launches (may be NULL) receives the
 * number of kernels the call launched.
 */
NPCF_API npcf_status npcf_last_profile(npcf_plan_t plan, double* stage_ms, int* launches);

/*
 * Allocation-free variant of npcf_compute (no counterpart in the paper; it is
 * an operational entry point).  Same arguments, same results.  For callers
 * that must not allocate device memory while running -- cudaMalloc
 * synchronises the device and can fail under memory pressure, which real-time
 * loops and processes whose caching allocator already holds the free memory
 * cannot accept.  Create the plan during set-up (that allocates its tables
 * once); this call then uses no cudaMalloc, cudaFree or allocating library
 * routine: all of its device workspace comes from one static array of 16 MiB
 * inside libnpcf (held by every GPU that loads the library until the process
 * exits).
 *   - Sizes whose workspace exceeds the array return NPCF_ERR_WORKSPACE with
 *     the bytes needed (about n*(44 + nbins*nq*4) bytes for FP32, nq = 36 at
 *     D=3, lmax=5, plus one row of partial sums; e.g. the D=3 4PCF with
 *     lmax=5 and 10 bins fits n up to about 10,000).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Each call copies the cell grid's stencil and geometry (a few KB) from
 *     host memory into the array before its kernels.
 *   - Every call shares the one array and clears what must start at zero;
 *     calls whose GPU work overlaps (two streams, two threads) race on it.
 *   - Stage timings are not recorded (npcf_last_profile reports -1 after it);
 *     the pair statistics and counters are.
 */
NPCF_API npcf_status npcf_compute_noalloc(npcf_plan_t plan, const void* positions, const void* weights, int64_t n,
                                          double* coeffs, int64_t primary_begin, int64_t primary_end,
                                          npcf_stream_t stream);

/*
 * Work counters of the pair kernel in the last call (host, waits for its
 * stream), for profiling: [0] pairs, [1] candidate secondaries examined,
 * [2] accumulation rounds of the warps' pair batches (each lane adds one pair
 * per round), [3] lane-rounds that added a pair (= pairs; [3] / (32 [2]) is the
 * lane fill), [4] candidate iterations of a warp (32 candidates each),
 * [5] pair batches, [6] candidates in an edge-flagged table bucket, [7]
 * candidates whose bin was decided in FP64.  Writes min(n, 8) entries (the
 * rest zero).
 */
NPCF_API npcf_status npcf_last_counters(npcf_plan_t plan, int64_t* counters, int n);

/*
 * Autotuning of the launch shapes (no counterpart in the paper): times candidate shapes on a
 * bounded sample of this input's primaries (all of them up to n = 500,000, else max(500,000,
 * n/10) in four ranges spread over the input; a shape replaces the built-in one only when it is
 * faster by more than 3%) and keeps the fastest in the plan for every later call (npcf_compute,
 * npcf_compute_batched, npcf_backward, npcf_compute_noalloc).  Searched: the pair kernel's warps
 * per CTA and pairs per warp batch; then, timed alone on the a-array of a quarter of the
 * primaries, the coupling's CTAs per SM (CUDA-core kernels), its FP32 span in chunks (tensor-core
 * kernel) or its primaries per chunk (factored 5PCF).  With the
 * environment variable NPCF_TUNE_CACHE naming a file, a choice is appended to it keyed by (device,
 * D, N, lmax, bins, precision, remove_self, size class 2^floor(log2 n)) and later plans load it
 * without timing (NPCF_TUNE_FORCE set: time again).  Inputs as for npcf_compute; waits for the
 * stream.  The results of later calls do not depend on the shapes beyond FP32 rounding of the
 * per-span sums.  Errors: as npcf_compute.
 */
NPCF_API npcf_status npcf_autotune(npcf_plan_t plan, const void* positions, const void* weights, int64_t n,
                                   npcf_stream_t stream);

/* The launch shapes in use (host): [0] pair-kernel warps per CTA, [1] pairs per warp batch,
 * [2] coupling CTAs per SM (0: built-in), [3] tensor-core FP32 span in chunks (0: built-in),
 * [4] 5PCF primaries per chunk (0: built-in), [5] 1 if npcf_autotune set them.  Writes
 * min(n, 6) entries (the rest zero). */
NPCF_API npcf_status npcf_tuned_config(npcf_plan_t plan, int* values, int n);

/*
 * Diagnostic (no counterpart in the paper): the split-precision tensor-core contraction
 * that the mixed couplings use, on caller data: d = a b^T with a 128 x k and b n x k
 * (row-major FP32, device), d 128 x n (FP32, device, overwritten).  tf32 = 0 splits into
 * BF16 pairs, 1 into TF32 pairs.  n a multiple of 16 in [16, 256]; k a positive multiple of
 * 64 (BF16) or 32 (TF32), at most 4096.  One CTA; waits for the stream.  Errors:
 * NPCF_ERR_ARG, NPCF_ERR_DEVICE_TIMEOUT (a bounded wait on the MMA ran out), NPCF_ERR_CUDA.
 */
NPCF_API npcf_status npcf_selftest_tc(int tf32, int n, int k, const float* a, const float* b, float* d,
                                      npcf_stream_t stream);

/* Thread-local description of the most recent error on this thread. */
NPCF_API const char* npcf_last_error(void);

/* Release the plan and its device memory (waits for nothing; the caller must
 * make sure no launch that uses the plan is still running). */
NPCF_API void npcf_plan_destroy(npcf_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* NPCF_H */
