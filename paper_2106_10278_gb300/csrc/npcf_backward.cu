// npcf_backward.cu -- the adjoint of the N=3 estimator: gradients of
//     L = sum_c g_c . zeta_c     (g = upstream gradient, re/im parts)
// with respect to every position and weight, bins held fixed (the radial
// indicators of eq. alm-bin-def are piecewise constant).
//
// With zeta = (1/V) sum_j w_j F(a_j), a_j[b][q] = (N_q/v_b) sum_k w_k Yq(u_jk):
//   dL/dw_j (primary)   = (1/V) g . F(a_j)
//   c_j[b][q]           = (w_j/V) (g . dF/da_j[b][q]) N_q / v_b
//   dL/dw_k (secondary) = sum_j h_j(u_jk),        h_j(u) = sum_q c_j[b_jk][q] Yq(u)
//   dL/dd_jk            = w_k (grad_u h - (u . grad_u h) u) / r_jk,  d_jk = y_k - y_j
// so one recomputation of the a-array (the forward pair kernel), one adjoint
// coupling kernel (c_j, dL/dw_j) and one adjoint pair kernel (h and its
// gradient by dual numbers through the same harmonic recurrences) suffice.
// Per-particle gradients accumulate in FP64 (atomics) and are converted once.
// The adjoint pair kernel compacts each warp's accepted pairs into a small ring
// so that the (expensive) dual-number evaluation always runs on full warps.
#include <cuda_runtime.h>

#include <algorithm>

#include "npcf_device.cuh"
#include "npcf_internal.h"
#include "npcf_pairs.cuh"

namespace npcf {

namespace {

// value and K partial derivatives
template <typename T, int K>
struct Dual {
    T v;
    T d[K];
};

template <typename T, int K>
__device__ __forceinline__ Dual<T, K> dconst(T c)
{
    Dual<T, K> r;
    r.v = c;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = T(0);
    return r;
}
template <typename T, int K>
__device__ __forceinline__ Dual<T, K> dvar(T x, int i)
{
    Dual<T, K> r = dconst<T, K>(x);
    r.d[i] = T(1);
    return r;
}
template <typename T, int K>
__device__ __forceinline__ Dual<T, K> operator+(const Dual<T, K>& a, const Dual<T, K>& b)
{
    Dual<T, K> r;
    r.v = a.v + b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i];
    return r;
}
template <typename T, int K>
__device__ __forceinline__ Dual<T, K> operator-(const Dual<T, K>& a, const Dual<T, K>& b)
{
    Dual<T, K> r;
    r.v = a.v - b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i];
    return r;
}
template <typename T, int K>
__device__ __forceinline__ Dual<T, K> operator*(const Dual<T, K>& a, const Dual<T, K>& b)
{
    Dual<T, K> r;
    r.v = a.v * b.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = fma(a.d[i], b.v, a.v * b.d[i]);
    return r;
}
template <typename T, int K>
__device__ __forceinline__ Dual<T, K> operator*(T s, const Dual<T, K>& a)
{
    Dual<T, K> r;
    r.v = s * a.v;
#pragma unroll
    for (int i = 0; i < K; ++i) r.d[i] = s * a.d[i];
    return r;
}

// Dual-number versions of the pair kernel's harmonic recurrences (npcf_device.cuh):
// sink(q, value) receives, for every real component q, the scaled harmonic
// (x - iy)^m Qs(z)... of a unit vector; constants are applied by the caller.
template <int LMAX, typename V, typename Sink>
__device__ __forceinline__ void harm_d2(Sink& sink, V x, V y, V one)
{
    V pr = one, pi = one - one;
    sink(0, pr);
    static_for<1, LMAX + 1>([&](auto L) {
        constexpr int l = decltype(L)::value;
        V nr = pr * x + pi * y;
        V ni = pi * x - pr * y;
        pr = nr;
        pi = ni;
        sink(q_index_d2(l), pr);
        sink(q_index_d2(l) + 1, pi);
    });
}

template <int LMAX, typename V, typename Sink, typename T>
__device__ __forceinline__ void harm_d3(Sink& sink, V x, V y, V z, V one, V rho2)
{
    V pr = one, pi = one - one;
    static_for<0, LMAX + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        if constexpr (m > 0) {
            V nr = pr * x + pi * y;
            V ni = pi * x - pr * y;
            pr = nr;
            pi = ni;
        }
        sink(q_index_d3(m, m), pr);
        if constexpr (m > 0) sink(q_index_d3(m, m) + 1, pi);
        if constexpr (m + 1 <= LMAX) {
            V t2r = pr, t2i = pi;
            V t1r = z * pr, t1i = z * pi;
            sink(q_index_d3(m + 1, m), t1r);
            if constexpr (m > 0) sink(q_index_d3(m + 1, m) + 1, t1i);
            static_for<m + 2, LMAX + 1>([&](auto L) {
                constexpr int l = decltype(L)::value;
                const V az = T(cx::leg_A(l, m)) * z;
                V nr = az * t1r - rho2 * t2r;
                V ni = az * t1i - rho2 * t2i;
                sink(q_index_d3(l, m), nr);
                if constexpr (m > 0) sink(q_index_d3(l, m) + 1, ni);
                t2r = t1r;
                t1r = nr;
                t2i = t1i;
                t1i = ni;
            });
        }
    });
}

template <int LMAX, typename V, typename Sink, typename T>
__device__ __forceinline__ void harm_d4(Sink& sink, V u1, V u2, V u3, V u4, V one)
{
    const V rho2 = u1 * u1 + u2 * u2 + u3 * u3;
    V G[LMAX + 1][LMAX + 1];
    static_for<0, LMAX + 1>([&](auto L2) {
        constexpr int l2 = decltype(L2)::value;
        constexpr int lam = l2 + 1;
        G[l2][0] = one;
        if constexpr (LMAX - l2 >= 1) G[l2][1] = u4;
        static_for<2, LMAX - l2 + 1>([&](auto Nn) {
            constexpr int n = decltype(Nn)::value;
            G[l2][n] = (T(cx::geg_B(n, lam)) * u4) * G[l2][n - 1] - G[l2][n - 2];
        });
    });
    V pr = one, pi = one - one;
    static_for<0, LMAX + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        if constexpr (m > 0) {
            V nr = pr * u1 + pi * u2;
            V ni = pi * u1 - pr * u2;
            pr = nr;
            pi = ni;
        }
        V t2r = pr - pr, t2i = pr - pr, t1r = pr, t1i = pi;
        static_for<m, LMAX + 1>([&](auto L2) {
            constexpr int l2 = decltype(L2)::value;
            V rr = pr, ri = pi;
            if constexpr (l2 == m + 1) {
                rr = u3 * pr;
                ri = u3 * pi;
                t2r = t1r;
                t2i = t1i;
                t1r = rr;
                t1i = ri;
            } else if constexpr (l2 > m + 1) {
                const V az = T(cx::leg_A(l2, m)) * u3;
                rr = az * t1r - rho2 * t2r;
                ri = az * t1i - rho2 * t2i;
                t2r = t1r;
                t2i = t1i;
                t1r = rr;
                t1i = ri;
            }
            static_for<l2, LMAX + 1>([&](auto L3) {
                constexpr int l3 = decltype(L3)::value;
                const V g = G[l2][l3 - l2];
                sink(q_index_d4(l3, l2, m), rr * g);
                if constexpr (m > 0) sink(q_index_d4(l3, l2, m) + 1, ri * g);
            });
        });
    });
}

// h(u) = sum_q c[q] Yq(u) and its gradient in u (the unit vector), for one pair
template <int D, int LMAX, typename T>
__device__ __forceinline__ Dual<T, D> adjoint_harmonics(const T* c, const T* u)
{
    using V = Dual<T, D>;
    V h = dconst<T, D>(T(0));
    auto sink = [&](int q, const V& v) {
        const T cq = c[q];
        h.v = fma(cq, v.v, h.v);
#pragma unroll
        for (int i = 0; i < D; ++i) h.d[i] = fma(cq, v.d[i], h.d[i]);
    };
    const V one = dconst<T, D>(T(1));
    if constexpr (D == 2) {
        harm_d2<LMAX, V>(sink, dvar<T, D>(u[0], 0), dvar<T, D>(u[1], 1), one);
    } else if constexpr (D == 3) {
        // on the unit sphere Qs has the plain recurrence (rho^2 = 1); the
        // extension off the sphere is immaterial after the tangential projection
        harm_d3<LMAX, V, decltype(sink), T>(sink, dvar<T, D>(u[0], 0), dvar<T, D>(u[1], 1), dvar<T, D>(u[2], 2), one,
                                            one);
    } else {
        harm_d4<LMAX, V, decltype(sink), T>(sink, dvar<T, D>(u[0], 0), dvar<T, D>(u[1], 1), dvar<T, D>(u[2], 2),
                                            dvar<T, D>(u[3], 3), one);
    }
    return h;
}

// ------------------------------------------------------------ coupling adjoint
// Per primary (compact index j): c_j[b][q] = (w_j/V) dL/da_j[b][q] * N_q / v_b
// (stride nq per bin) and gwp[j] = (1/V) g . F(a_j).
struct AdjCoupleParams {
    int nbins, nq, lmax;
    int64_t nprim;
    const void* a;         // nprim x nbins x nq (T)
    const void* wprim;     // nprim (T)
    const double* g;       // 2 * ncoeff
    const int* key_base;   // nbins x nbins: first key of the bin pair (min, max), -1 if none
    const void* pref;      // lmax + 1 (T), D >= 3
    const void* qnorm;     // nq (T)
    const void* inv_vb;    // nbins (T)
    double inv_V;
    void* cbuf;            // nprim x nbins x nq (T)
    double* gwp;           // nprim
    int ncoeff;
    int g_in_smem;         // the upstream gradient is copied to shared memory (as T)
    int tables_off;        // byte offset of that copy
};

// the l of a real component and its multiplicity in sum_[l] a(b1) conj(a(b2))
// over all signed inner labels (1 for a zero inner label, 2 otherwise)
template <int D>
__device__ __forceinline__ void q_label(int q, int* l, int* mult)
{
    if constexpr (D == 2) {
        *l = (q + 1) / 2;
        *mult = 1;
    } else if constexpr (D == 3) {
        int L = 0;
        while ((L + 1) * (L + 1) <= q) ++L;
        *l = L;
        *mult = q == L * L ? 1 : 2;
    } else {
        int L = 0;
        while (q_base_d4(L + 1) <= q) ++L;
        const int r = q - q_base_d4(L);
        int l2 = 0;
        while ((l2 + 1) * (l2 + 1) <= r) ++l2;
        *l = L;
        *mult = r == l2 * l2 ? 1 : 2;
    }
}

template <int D, typename T>
__global__ void __launch_bounds__(256) k_couple_adjoint_n3(const AdjCoupleParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nb = p.nbins, nq = p.nq, L1 = p.lmax + 1;
    T* aw = reinterpret_cast<T*>(smem) + warp * nb * nq;
    // per component: its l and multiplicity; per l: its contiguous component range [qs[l], qs[l+1])
    int* s_lq = reinterpret_cast<int*>(smem + (size_t)nw * nb * nq * sizeof(T));
    int* s_mult = s_lq + nq;
    int* s_qs = s_mult + nq;
    // loop-invariant tables: the first key of every ordered bin pair, and (when it fits) the
    // upstream gradient in T
    int* s_kb = s_qs + (L1 + 1);
    T* s_g = reinterpret_cast<T*>(smem + p.tables_off);
    for (int i = threadIdx.x; i < nb * nb; i += blockDim.x) {
        const int b = i / nb, b2 = i - (i / nb) * nb;
        s_kb[i] = p.key_base[(b < b2 ? b : b2) * nb + (b < b2 ? b2 : b)];
    }
    if (p.g_in_smem)
        for (int i = threadIdx.x; i < 2 * p.ncoeff; i += blockDim.x) s_g[i] = (T)p.g[i];
    auto gat = [&](int i) -> T { return p.g_in_smem ? s_g[i] : (T)p.g[i]; };
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        int l, mult;
        q_label<D>(q, &l, &mult);
        s_lq[q] = l;
        s_mult[q] = mult;
    }
    if (threadIdx.x <= L1) {
        const int l = threadIdx.x;
        s_qs[l] = D == 2 ? (l == 0 ? 0 : 2 * l - 1) : (D == 3 ? l * l : q_base_d4(l));
    }
    __syncthreads();
    const T* A = static_cast<const T*>(p.a);
    const T* pref = static_cast<const T*>(p.pref);
    const T* qnorm = static_cast<const T*>(p.qnorm);
    const T* ivb = static_cast<const T*>(p.inv_vb);
    T* cb = static_cast<T*>(p.cbuf);
    for (int64_t j = (int64_t)blockIdx.x * nw + warp; j < p.nprim; j += (int64_t)gridDim.x * nw) {
        for (int i = lane; i < nb * nq; i += 32) aw[i] = A[j * nb * nq + i];
        __syncwarp();
        const T wj = static_cast<const T*>(p.wprim)[j];
        for (int i = lane; i < nb * nq; i += 32) {
            const int b = i / nq, q = i - (i / nq) * nq;
            const int l = s_lq[q];
            T G = T(0);
            for (int b2 = 0; b2 < nb; ++b2) {
                const int kb = s_kb[b * nb + b2];
                if (kb < 0) continue;
                const T gre = gat(2 * (kb + l));
                if constexpr (D == 2) {
                    // zeta_l = a_l(b1) conj(a_l(b2)); this component is Re (q = 0 or odd) or Im (q even > 0)
                    const T gim = gat(2 * (kb + l) + 1);
                    const bool is_im = q > 0 && (q & 1) == 0;
                    const int qr = is_im ? q - 1 : q;
                    const T xr = aw[b2 * nq + qr];
                    const T xi = l > 0 ? aw[b2 * nq + qr + 1] : T(0);
                    if (b <= b2) G += is_im ? (gre * xi + gim * xr) : (gre * xr - gim * xi);  // b is b1
                    if (b >= b2) G += is_im ? (gre * xi - gim * xr) : (gre * xr + gim * xi);  // b is b2
                } else {
                    G = fma(gre, aw[b2 * nq + q] * (b2 == b ? T(2) : T(1)), G);
                }
            }
            if constexpr (D != 2) G *= pref[l] * T(s_mult[q]);
            cb[j * nb * nq + i] = G * wj * T(p.inv_V) * qnorm[q] * ivb[b];
        }
        double s = 0.0;
        for (int i = lane; i < nb * nb * L1; i += 32) {
            const int l = i % L1, bb = i / L1, b1 = bb / nb, b2 = bb % nb;
            if (b1 > b2) continue;
            const int kb = s_kb[b1 * nb + b2];
            if (kb < 0) continue;
            const int key = kb + l;
            if constexpr (D == 2) {
                double re, im;
                if (l == 0) {
                    re = (double)aw[b1 * nq] * aw[b2 * nq];
                    im = 0.0;
                } else {
                    const int q = 2 * l - 1;
                    const double ar = aw[b1 * nq + q], ai = aw[b1 * nq + q + 1];
                    const double br = aw[b2 * nq + q], bi = aw[b2 * nq + q + 1];
                    re = ar * br + ai * bi;
                    im = ai * br - ar * bi;
                }
                s += p.g[2 * key] * re + p.g[2 * key + 1] * im;
            } else {
                T f = T(0);
                for (int q = s_qs[l]; q < s_qs[l + 1]; ++q) f = fma(T(s_mult[q]) * aw[b1 * nq + q], aw[b2 * nq + q], f);
                s += p.g[2 * key] * (double)(pref[l] * f);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) p.gwp[j] = s * p.inv_V;
        __syncwarp();
    }
}

// --------------------------------------------------------------- pair adjoint
struct AdjPairExtra {
    const void* cbuf;   // nprim x nbins x nq (T)
    const double* gwp;  // nprim: dL/dw of each primary through its own weight
    const int* perm;    // slot -> input index
    double* gpos;       // n x D, input order
    double* gw;         // n, input order
};

constexpr int kAdjThreads = 256;
constexpr int kRing = 64;  // accepted pairs queued per warp (a power of two >= 64)

__host__ __device__ inline int adjoint_ring_bytes(int D, int tbytes) { return kRing * ((D + 1) * tbytes + 8); }

// same item, neighbour-cell and bin logic as the forward pair kernel; each
// lane takes one candidate of the current cell at a time
template <int D, int LMAX, typename T>
__global__ void __launch_bounds__(kAdjThreads) k_pairs_adjoint(const PairParams p, const AdjPairExtra x)
{
    using R = Rec<D, T>;
    constexpr int NQ = num_q(D, LMAX);
    constexpr bool kFP32 = sizeof(T) == 4;
    const unsigned full = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem[];
    const int nthreads = blockDim.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nbins = p.nbins, nq = p.nq;
    unsigned char* tab = smem;
    float* s_edge = reinterpret_cast<float*>(tab + kTabBytes);
    double* s_edge2 = reinterpret_cast<double*>(tab + kTabBytes + 192);
    int* job_a = reinterpret_cast<int*>(tab + kTabBytes + 576);
    int* job_pk = job_a + kMaxJobs;
    int* job_pre = job_pk + kMaxJobs;
    int* ws = job_pre + kMaxJobs + 4;
    CatGeom* s_geo = reinterpret_cast<CatGeom*>(smem + kGeomOffset);
    T* crow = reinterpret_cast<T*>(smem + pair_fixed_bytes(sizeof(R), nthreads)) + warp * nbins * NQ;
    // this warp's ring of accepted pairs: unit vectors, w/r, input index, c-row offset
    unsigned char* rbase = smem + pair_fixed_bytes(sizeof(R), nthreads) +
                           (nthreads / 32) * nbins * NQ * (int)sizeof(T) + warp * adjoint_ring_bytes(D, sizeof(T));
    T* ring_u = reinterpret_cast<T*>(rbase);
    T* ring_s = ring_u + D * kRing;
    int* ring_k = reinterpret_cast<int*>(ring_s + kRing);
    int* ring_b = ring_k + kRing;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (int i = threadIdx.x; i < kTabBytes / 4; i += nthreads)
        reinterpret_cast<int*>(tab)[i] = reinterpret_cast<const int*>(p.tab)[i];
    if (threadIdx.x <= nbins) {
        s_edge[threadIdx.x] = p.edgef[threadIdx.x];
        s_edge2[threadIdx.x] = p.edge2[threadIdx.x];
    }
    const R* rec = static_cast<const R*>(p.rec);
    const T* cb = static_cast<const T*>(x.cbuf);

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
        const bool active = warp < (it.z & 0xff);
        const int jslot = it.y + (active ? warp : 0);
        const int pidx = it.w + warp;
        int cc[D];
#pragma unroll
        for (int d = 0; d < D; ++d) cc[d] = ((it.x - g.base) / g.stride[d]) % g.nc[d];
        int njobs = 0, V = 0;
        for (int base = 0; base < p.nstencil; base += nthreads) {
            const int sidx = base + threadIdx.x;
            int keep = 0, len = 0, a = 0, pk = 0;
            if (sidx < p.nstencil) {
                pk = p.stencil[sidx];
                int cell = g.base;
                bool ok = true;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    int c = cc[d] + (int)(signed char)((pk >> (8 * d)) & 0xff);
                    if (c < 0) {
                        ok = ok && p.periodic;
                        c += g.nc[d];
                    } else if (c >= g.nc[d]) {
                        ok = ok && p.periodic;
                        c -= g.nc[d];
                    }
                    cell += c * g.stride[d];
                }
                if (ok) {
                    a = p.cell_start[cell];
                    len = p.cell_start[cell + 1] - a;
                    keep = len > 0;
                }
            }
            int pos, off, tcount, tlen;
            block_scan2(keep, keep ? len : 0, &pos, &off, &tcount, &tlen, ws);
            if (keep) {
                job_a[njobs + pos] = a;
                job_pk[njobs + pos] = pk;
                job_pre[njobs + pos] = V + off;
            }
            njobs += tcount;
            V += tlen;
        }
        if (threadIdx.x == 0) job_pre[njobs] = V;
        __syncthreads();
        if (!active) continue;
        // this primary's c-row, zero beyond the plan's components
        for (int i = lane; i < nbins * NQ; i += 32) {
            const int b = i / NQ, q = i - (i / NQ) * NQ;
            crow[i] = q < nq ? cb[(size_t)pidx * nbins * nq + b * nq + q] : T(0);
        }
        __syncwarp();
        const R pj = rec[jslot];
        T xj[D];
#pragma unroll
        for (int d = 0; d < D; ++d) xj[d] = pj.x(d);
        double gj[D];
#pragma unroll
        for (int d = 0; d < D; ++d) gj[d] = 0.0;
        // accepted pairs go into a per-warp ring of kRing entries; every time 32 are queued
        // all lanes evaluate one each, so the dual-number harmonics run on full warps
        int head = 0, cnt = 0;  // warp-uniform
        auto process = [&](int e) {
            T u[D];
#pragma unroll
            for (int d = 0; d < D; ++d) u[d] = ring_u[d * kRing + e];
            const T sc = ring_s[e];
            const int korig = ring_k[e];
            const Dual<T, D> h = adjoint_harmonics<D, LMAX, T>(crow + ring_b[e], u);
            atomicAdd(&x.gw[korig], (double)h.v);
            T ug = T(0);
#pragma unroll
            for (int d = 0; d < D; ++d) ug = fma(u[d], h.d[d], ug);
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const double gd = (double)(sc * (h.d[d] - ug * u[d]));
                atomicAdd(&x.gpos[(size_t)korig * D + d], gd);
                gj[d] -= gd;
            }
        };
        for (int j = 0; j < njobs; ++j) {
            const int seg_a = job_a[j];
            const int seg_n = job_pre[j + 1] - job_pre[j];
            const int packed = job_pk[j];
            T xjs[D];
            if (!cell_geometry<D, T>(p, g, cc, packed, xj, xjs)) continue;
            for (int c0 = 0; c0 < seg_n; c0 += 32) {  // warp-uniform trip count
                const int k = c0 + lane;
                const bool valid = k < seg_n;
                const R pk = ldg_rec(rec + seg_a, valid ? k : 0);
                T dx[D];
                T r2 = T(0);
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    if constexpr (kFP32) dx[d] = pk.x(d) - xjs[d];
                    else dx[d] = (pk.x(d) - xj[d]) + (xj[d] - xjs[d]);
                    r2 = fma(dx[d], dx[d], r2);
                }
                bool fl = false, ex = false;
                const int b = valid ? decide_bin<D, T>(p, g, tab, s_edge, s_edge2, cc, packed, xj, pk, r2, &fl, &ex) : -1;
                const unsigned m = __ballot_sync(full, b >= 0);
                if (b >= 0) {
                    const int e = (head + cnt + __popc(m & lt_mask)) & (kRing - 1);
                    const T rinv = rsqrt_t(r2);
#pragma unroll
                    for (int d = 0; d < D; ++d) ring_u[d * kRing + e] = dx[d] * rinv;
                    ring_s[e] = pk.w() * rinv;
                    ring_k[e] = x.perm[seg_a + k];
                    ring_b[e] = b * NQ;
                }
                cnt += __popc(m);
                __syncwarp();
                if (cnt >= 32) {
                    process((head + lane) & (kRing - 1));
                    head = (head + 32) & (kRing - 1);
                    cnt -= 32;
                    __syncwarp();
                }
            }
        }
        if (lane < cnt) process((head + lane) & (kRing - 1));
        __syncwarp();
        const int jorig = x.perm[jslot];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            double v = gj[d];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(full, v, o);
            if (lane == 0) atomicAdd(&x.gpos[(size_t)jorig * D + d], v);
        }
        if (lane == 0) atomicAdd(&x.gw[jorig], x.gwp[pidx]);
    }
}

template <typename T>
__global__ void k_finalize_grads(int64_t n, int D, const double* gpos, const double* gw, T* grad_pos, T* grad_w)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (grad_w) grad_w[i] = (T)gw[i];
    if (grad_pos)
        for (int d = 0; d < D; ++d) grad_pos[i * D + d] = (T)gpos[i * D + d];
}

}  // namespace
int adjoint_pair_smem(int D, int Lc, int fp64, int nbins);
namespace {

template <int D, int LMAX, typename T>
cudaError_t launch_adj_pairs(const PairParams& p, const AdjPairExtra& x, int nsm, cudaStream_t s)
{
    const int smem = adjoint_pair_smem(D, LMAX, sizeof(T) == 8, p.nbins);
    auto kern = k_pairs_adjoint<D, LMAX, T>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kAdjThreads, smem);
    if (e != cudaSuccess) return e;
    kern<<<nsm * (occ > 0 ? occ : 1), kAdjThreads, smem, s>>>(p, x);
    ++launch_counter();
    return cudaGetLastError();
}

}  // namespace

int adjoint_pair_warps() { return kAdjThreads / 32; }

int adjoint_pair_smem(int D, int Lc, int fp64, int nbins)
{
    const int tb = fp64 ? 8 : 4;
    const int rb = tb * 4 * (D <= 3 ? 1 : 2);
    return pair_fixed_bytes(rb, kAdjThreads) + (kAdjThreads / 32) * (nbins * num_q(D, Lc) * tb + adjoint_ring_bytes(D, tb));
}

cudaError_t launch_couple_adjoint(int D, int fp64, int nbins, int nq, int lmax, int64_t nprim, const void* a,
                                  const void* wprim, const double* g, int ncoeff, const int* key_base, const void* pref,
                                  const void* qnorm, const void* inv_vb, double inv_V, void* cbuf, double* gwp,
                                  int nsm, cudaStream_t s)
{
    if (nprim <= 0) return cudaSuccess;
    AdjCoupleParams cp{nbins, nq, lmax, nprim, a, wprim, g, key_base, pref, qnorm, inv_vb, inv_V, cbuf, gwp};
    const int tb = fp64 ? 8 : 4;
    int warps = 8;  // one primary per warp; its a-row is staged in shared memory
    while (warps > 1 && warps * nbins * nq * tb > 120 * 1024) --warps;
    const int ints = 2 * nq + lmax + 2 + nbins * nbins;
    cp.ncoeff = ncoeff;
    cp.tables_off = ((warps * nbins * nq * tb + ints * (int)sizeof(int)) + 15) / 16 * 16;
    cp.g_in_smem = 2 * ncoeff * tb <= 48 * 1024;
    const int smem = cp.tables_off + (cp.g_in_smem ? 2 * ncoeff * tb : 0);
    const int grid = (int)std::min<int64_t>((nprim + warps - 1) / warps, 8 * (int64_t)nsm);
    cudaError_t e = cudaSuccess;
    auto go = [&](auto kern) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return;
        kern<<<grid, 32 * warps, smem, s>>>(cp);
        ++launch_counter();
        e = cudaGetLastError();
    };
    switch (D * 2 + fp64) {
        case 4: go(k_couple_adjoint_n3<2, float>); break;
        case 5: go(k_couple_adjoint_n3<2, double>); break;
        case 6: go(k_couple_adjoint_n3<3, float>); break;
        case 7: go(k_couple_adjoint_n3<3, double>); break;
        case 8: go(k_couple_adjoint_n3<4, float>); break;
        case 9: go(k_couple_adjoint_n3<4, double>); break;
        default: return cudaErrorInvalidValue;
    }
    return e;
}

// lmax values the adjoint pair kernel is compiled for; a plan uses the
// smallest one not below its lmax (its c-rows are zero beyond the plan's)
#define NPCF_ADJOINT_LMAX_LIST(X) \
    X(2, 2) X(2, 4) X(2, 6) X(2, 8) X(2, 10) X(2, 12) \
    X(3, 1) X(3, 2) X(3, 3) X(3, 4) X(3, 5) X(3, 6) X(3, 8) X(3, 10) \
    X(4, 1) X(4, 2) X(4, 3) X(4, 4) X(4, 6)

int adjoint_compiled_lmax(int D, int lmax)
{
    int best = -1;
#define NPCF_AL(DD, LL) \
    if (D == DD && LL >= lmax && (best < 0 || LL < best)) best = LL;
    NPCF_ADJOINT_LMAX_LIST(NPCF_AL)
#undef NPCF_AL
    return best;
}

cudaError_t launch_pairs_adjoint(const PairParams& p, int fp64, int Lc, const void* cbuf, const double* gwp,
                                 const int* perm, double* gpos, double* gw, int nsm, cudaStream_t s)
{
    const AdjPairExtra x{cbuf, gwp, perm, gpos, gw};
    switch (p.D * 1000 + Lc * 10 + fp64) {
#define NPCF_AP(DD, LL)                                                                   \
    case DD * 1000 + LL * 10: return launch_adj_pairs<DD, LL, float>(p, x, nsm, s); \
    case DD * 1000 + LL * 10 + 1: return launch_adj_pairs<DD, LL, double>(p, x, nsm, s);
        NPCF_ADJOINT_LMAX_LIST(NPCF_AP)
#undef NPCF_AP
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_finalize_grads(int64_t n, int D, int fp64, const double* gpos, const double* gw, void* grad_pos,
                                  void* grad_w, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int t = 256;
    const int g = (int)((n + t - 1) / t);
    if (fp64) k_finalize_grads<double><<<g, t, 0, s>>>(n, D, gpos, gw, (double*)grad_pos, (double*)grad_w);
    else k_finalize_grads<float><<<g, t, 0, s>>>(n, D, gpos, gw, (float*)grad_pos, (float*)grad_w);
    ++launch_counter();
    return cudaGetLastError();
}

}  // namespace npcf
