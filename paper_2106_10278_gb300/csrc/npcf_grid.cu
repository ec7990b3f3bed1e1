// npcf_grid.cu -- the estimator of a field sampled on a periodic grid, in the FFT form of
// Sec. "Application to Gridded Data": the binned harmonic coefficients at every node are a
// convolution of the field with one kernel per (radial bin, harmonic state),
//     a^b_l(c) = sum_{u != 0} dV X(c + u) Y*_l(unit(u)) Theta^b(|u|) / v_b
//              = IFFT[ FFT(X) FFT(K^b_l) ](c),   K^b_l(u) = dV Y*_l(unit(-u)) Theta^b(|u|) / v_b,
// (the relabelling u -> -u moves the parity of Y into the kernel, reading R16), after which the
// coupling of eq. NPCF-estimator-discrete runs over the nodes with weights dV X(c).
//
// Kernels: the kernel fields K^b_l on the grid (harmonics by the pair kernel's recurrences, bins
// decided on the FP64 squared offset), the field's complex copy and node weights, the spectral
// products, and the scatter of the inverse transforms into the a-array layout of the pair kernel.
// The transforms themselves are cuFFT (single or double precision complex, batched).
#include <cuda_runtime.h>

#include "npcf_device.cuh"
#include "npcf_internal.h"

namespace npcf {

namespace {

template <typename T>
struct CxG {
    T r, i;
};

// One thread per grid offset (node index = offset, wrapped to [-n/2, n/2) per axis).
template <int D, int LMAX, typename T>
__global__ void k_grid_kernels(const GridParams g)
{
    constexpr int NQ = num_q(D, LMAX);
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= g.ncell) return;
    int64_t rem = idx;
    double u[4] = {0.0, 0.0, 0.0, 0.0};
    for (int a = D - 1; a >= 0; --a) {
        int c = (int)(rem % g.dims[a]);
        rem /= g.dims[a];
        if (c >= (g.dims[a] + 1) / 2) c -= g.dims[a];  // signed offset
        u[a] = __dmul_rn((double)c, g.spacing[a]);
    }
    // the squared offset summed in axis order without contraction, as the definition's bin rule reads it
    double r2 = __dmul_rn(u[0], u[0]);
    for (int a = 1; a < D; ++a) r2 = __dadd_rn(r2, __dmul_rn(u[a], u[a]));
    if (!(r2 > 0.0) || r2 < g.edge2[0] || !(r2 < g.edge2[g.nbins])) return;
    int b = 0;
    while (b + 1 < g.nbins && !(r2 < g.edge2[b + 1])) ++b;  // [e_b, e_{b+1})
    // harmonics of unit(-u), with the pair kernel's recurrences (w = 1)
    const double rinv = 1.0 / sqrt(r2);
    T acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = T(0);
    if constexpr (D == 2) accum_d2<LMAX, T>(acc, T(-u[0] * rinv), T(-u[1] * rinv), T(1));
    else if constexpr (D == 3) accum_d3<LMAX, T>(acc, T(-u[0] * rinv), T(-u[1] * rinv), T(-u[2] * rinv), T(1));
    else accum_d4<LMAX, T>(acc, T(-u[0] * rinv), T(-u[1] * rinv), T(-u[2] * rinv), T(-u[3] * rinv), T(1));
    const T* qnorm = static_cast<const T*>(g.qnorm);
    const T scale = T(g.dV * g.inv_vb[b]);
    CxG<T>* K = static_cast<CxG<T>*>(g.khat);
    for (int s = 0; s < g.ncs; ++s) {
        const int2 q = g.cstate[s];  // real and imaginary component (-1: real state)
        CxG<T> v;
        v.r = scale * acc[q.x] * qnorm[q.x];
        v.i = q.y >= 0 ? scale * acc[q.y] * qnorm[q.y] : T(0);
        K[((size_t)b * g.ncs + s) * g.ncell + idx] = v;
    }
}

// the field as complex values and the nodes' weights dV X
template <typename T>
__global__ void k_grid_field(const GridParams g, const T* X)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= g.ncell) return;
    static_cast<CxG<T>*>(g.xhat)[i] = CxG<T>{X[i], T(0)};
    static_cast<T*>(g.wprim)[i] = T(g.dV) * X[i];
}

// P[bs][k] = FFT(X)[k] * FFT(K^b_s)[k] for the batch of (bin, state) transforms [bs0, bs0 + nbs)
template <typename T>
__global__ void k_grid_product(const GridParams g, int bs0, int nbs)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)nbs * g.ncell) return;
    const int64_t k = i % g.ncell;
    const CxG<T> x = static_cast<const CxG<T>*>(g.xhat)[k];
    const CxG<T> c = static_cast<const CxG<T>*>(g.khat)[(size_t)bs0 * g.ncell + i];
    static_cast<CxG<T>*>(g.work)[i] = CxG<T>{x.r * c.r - x.i * c.i, x.r * c.i + x.i * c.r};
}

// a-array entries (node, bin, component) from the inverse transforms, scaled by 1/ncell
template <typename T>
__global__ void k_grid_scatter(const GridParams g, int bs0, int nbs)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)nbs * g.ncell) return;
    const int bs = bs0 + (int)(i / g.ncell);
    const int64_t node = i % g.ncell;
    const int b = bs / g.ncs, s = bs - b * g.ncs;
    const CxG<T> v = static_cast<const CxG<T>*>(g.work)[i];
    const T f = T(1.0 / (double)g.ncell);
    T* a = static_cast<T*>(g.a) + ((size_t)node * g.nbins + b) * g.nq;
    const int2 q = g.cstate[s];
    a[q.x] = v.r * f;
    if (q.y >= 0) a[q.y] = v.i * f;
}

inline int blocks(int64_t n, int t) { return (int)((n + t - 1) / t); }

template <int D, typename T>
cudaError_t launch_kernels_d(const GridParams& g, int L, cudaStream_t s)
{
    const int t = 128, nb = blocks(g.ncell, t);
    switch (L) {
        case 1: k_grid_kernels<D, 1, T><<<nb, t, 0, s>>>(g); break;
        case 2: k_grid_kernels<D, 2, T><<<nb, t, 0, s>>>(g); break;
        case 3: k_grid_kernels<D, 3, T><<<nb, t, 0, s>>>(g); break;
        case 4: k_grid_kernels<D, 4, T><<<nb, t, 0, s>>>(g); break;
        case 5: k_grid_kernels<D, 5, T><<<nb, t, 0, s>>>(g); break;
        case 6: k_grid_kernels<D, 6, T><<<nb, t, 0, s>>>(g); break;
        default: return cudaErrorInvalidValue;
    }
    ++launch_counter();
    return cudaGetLastError();
}

}  // namespace

int grid_max_lmax() { return 6; }

cudaError_t launch_grid_kernels(const GridParams& g, int D, int fp64, int L, cudaStream_t s)
{
    if (D == 2) return fp64 ? launch_kernels_d<2, double>(g, L, s) : launch_kernels_d<2, float>(g, L, s);
    if (D == 3) return fp64 ? launch_kernels_d<3, double>(g, L, s) : launch_kernels_d<3, float>(g, L, s);
    return fp64 ? launch_kernels_d<4, double>(g, L, s) : launch_kernels_d<4, float>(g, L, s);
}

cudaError_t launch_grid_field(const GridParams& g, int fp64, const void* X, cudaStream_t s)
{
    const int t = 256;
    if (fp64) k_grid_field<double><<<blocks(g.ncell, t), t, 0, s>>>(g, static_cast<const double*>(X));
    else k_grid_field<float><<<blocks(g.ncell, t), t, 0, s>>>(g, static_cast<const float*>(X));
    ++launch_counter();
    return cudaGetLastError();
}

cudaError_t launch_grid_product(const GridParams& g, int fp64, int bs0, int nbs, cudaStream_t s)
{
    const int t = 256;
    const int nb = blocks((int64_t)nbs * g.ncell, t);
    if (fp64) k_grid_product<double><<<nb, t, 0, s>>>(g, bs0, nbs);
    else k_grid_product<float><<<nb, t, 0, s>>>(g, bs0, nbs);
    ++launch_counter();
    return cudaGetLastError();
}

cudaError_t launch_grid_scatter(const GridParams& g, int fp64, int bs0, int nbs, cudaStream_t s)
{
    const int t = 256;
    const int nb = blocks((int64_t)nbs * g.ncell, t);
    if (fp64) k_grid_scatter<double><<<nb, t, 0, s>>>(g, bs0, nbs);
    else k_grid_scatter<float><<<nb, t, 0, s>>>(g, bs0, nbs);
    ++launch_counter();
    return cudaGetLastError();
}

}  // namespace npcf
