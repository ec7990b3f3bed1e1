// npcf_device.cuh -- device-side helpers of libnpcf: particle records,
// compile-time loops and the harmonic recurrences of the pair kernel.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "npcf_internal.h"
#include "npcf_math.h"

namespace npcf {

template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(static_cast<F&&>(f));
    }
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_16a; };

// A particle record: D position components followed by the weight.  One
// 4-vector for D <= 3 (D=2: x, y, w, 0; D=3: x, y, z, w), two for D = 4
// (x1..x4 | w, 0, 0, 0).  The staged pairs of the pair kernel reuse the same
// shape with the unit separation vector in place of the position.
template <int D, typename T>
struct Rec {
    using V = typename Vec4<T>::type;
    static constexpr int NV = (D <= 3) ? 1 : 2;
    V v[NV];
    __device__ __forceinline__ T x(int a) const
    {
        const T* p = reinterpret_cast<const T*>(v);
        return p[a];
    }
    __device__ __forceinline__ T w() const
    {
        const T* p = reinterpret_cast<const T*>(v);
        return p[D];
    }
    __device__ __forceinline__ void set(int a, T val)
    {
        T* p = reinterpret_cast<T*>(v);
        p[a] = val;
    }
};

// ------------------------------------------------------------ layouts
// Real components of a^b per bin (the a-array the pair kernel writes):
//   D=2: l = 0: Re; l >= 1: Re, Im                          -> 2 lmax + 1
//   D=3: (l, m >= 0) in l-major order: Re, and Im when m > 0 -> (lmax+1)^2
//   D=4: (l3, l2 <= l3, l1 in 0..l2): Re, and Im when l1 > 0 -> sum (l3+1)^2
__host__ __device__ constexpr int q_index_d2(int l) { return l == 0 ? 0 : 2 * l - 1; }
__host__ __device__ constexpr int q_index_d3(int l, int m) { return l * l + (m == 0 ? 0 : 2 * m - 1); }
__host__ __device__ constexpr int q_base_d4(int l3)
{
    int s = 0;
    for (int l = 0; l < l3; ++l) s += (l + 1) * (l + 1);
    return s;
}
__host__ __device__ constexpr int q_index_d4(int l3, int l2, int l1)
{
    return q_base_d4(l3) + l2 * l2 + (l1 == 0 ? 0 : 2 * l1 - 1);
}
__host__ __device__ constexpr int num_q(int D, int lmax)
{
    return D == 2 ? 2 * lmax + 1 : (D == 3 ? (lmax + 1) * (lmax + 1) : q_base_d4(lmax + 1));
}

// ------------------------------------------------------ harmonic kernels
// Each adds w * Y*(u) (up to the per-component constants applied at the
// end) for every component to acc[].  u is the unit separation vector.

// D=2: Y*_l = e^{-i l theta}/sqrt(2 pi) = (x - i y)^l / sqrt(2 pi)
template <int LMAX, typename T>
__device__ __forceinline__ void accum_d2(T* acc, T x, T y, T w)
{
    T pr = w, pi = T(0);
    acc[0] += w;
    static_for<1, LMAX + 1>([&](auto L) {
        constexpr int l = decltype(L)::value;
        T nr = fma(pr, x, pi * y);
        T ni = fma(pi, x, -(pr * y));
        pr = nr;
        pi = ni;
        acc[q_index_d2(l)] += pr;
        acc[q_index_d2(l) + 1] += pi;
    });
}

// D=2 in FP32 with packed pairs: acc0 the l = 0 term, accC[l - 1] = (Re, Im) of w (x - i y)^l.
template <int LMAX>
__device__ __forceinline__ void accum_d2_x2(float& acc0, float2* accC, float x, float y, float w)
{
    acc0 += w;
    float2 P = make_float2(w, 0.f);
    const float2 xx = make_float2(x, x), yy = make_float2(y, -y);
    static_for<1, LMAX + 1>([&](auto L) {
        constexpr int l = decltype(L)::value;
        // (pr, pi) (x - i y) = (pr x + pi y, pi x - pr y)
        P = __ffma2_rn(make_float2(P.y, P.x), yy, __fmul2_rn(P, xx));
        accC[l - 1] = __fadd2_rn(accC[l - 1], P);
    });
}

// D=3: w Qs_l^m(z) (x - i y)^m for l <= LMAX, 0 <= m <= l
template <int LMAX, typename T>
__device__ __forceinline__ void accum_d3(T* acc, T x, T y, T z, T w)
{
    T pr = w, pi = T(0);  // P_m = w (x - i y)^m
    static_for<0, LMAX + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        if constexpr (m > 0) {
            T nr = fma(pr, x, pi * y);
            T ni = fma(pi, x, -(pr * y));
            pr = nr;
            pi = ni;
        }
        acc[q_index_d3(m, m)] += pr;
        if constexpr (m > 0) acc[q_index_d3(m, m) + 1] += pi;
        if constexpr (m + 1 <= LMAX) {
            T t2r = pr, t2i = pi;
            T t1r = z * pr, t1i = z * pi;
            acc[q_index_d3(m + 1, m)] += t1r;
            if constexpr (m > 0) acc[q_index_d3(m + 1, m) + 1] += t1i;
            static_for<m + 2, LMAX + 1>([&](auto L) {
                constexpr int l = decltype(L)::value;
                constexpr T A = T(cx::leg_A(l, m));
                T az = A * z;
                T nr = fma(az, t1r, -t2r);
                acc[q_index_d3(l, m)] += nr;
                t2r = t1r;
                t1r = nr;
                if constexpr (m > 0) {
                    T ni = fma(az, t1i, -t2i);
                    acc[q_index_d3(l, m) + 1] += ni;
                    t2i = t1i;
                    t1i = ni;
                }
            });
        }
    });
}

// D=3 in FP32 with the complex columns as packed pairs (sm_100 FP32x2 arithmetic: one
// instruction for the real and imaginary part): the same terms as accum_d3, the m = 0 column in
// accR[l] and the (l, m >= 1) components in accC[l (l - 1) / 2 + m - 1] as (Re, Im).
__host__ __device__ constexpr int d3_cidx(int l, int m) { return l * (l - 1) / 2 + m - 1; }

template <int LMAX>
__device__ __forceinline__ void accum_d3_x2(float* accR, float2* accC, float x, float y, float z, float w)
{
    // m = 0: w Qs_l^0(z)
    accR[0] += w;
    if constexpr (LMAX >= 1) {
        float t2 = w, t1 = z * w;
        accR[1] += t1;
        static_for<2, LMAX + 1>([&](auto L) {
            constexpr int l = decltype(L)::value;
            const float nr = fmaf(float(cx::leg_A(l, 0)) * z, t1, -t2);
            accR[l] += nr;
            t2 = t1;
            t1 = nr;
        });
    }
    // m >= 1: P_m = w (x - i y)^m, then the column Qs_l^m(z) P_m
    float2 P = make_float2(w, 0.f);
    const float2 xx = make_float2(x, x), yy = make_float2(y, -y), zz = make_float2(z, z);
    static_for<1, LMAX + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;
        // (pr, pi) (x - i y) = (pr x + pi y, pi x - pr y)
        P = __ffma2_rn(make_float2(P.y, P.x), yy, __fmul2_rn(P, xx));
        accC[d3_cidx(m, m)] = __fadd2_rn(accC[d3_cidx(m, m)], P);
        if constexpr (m + 1 <= LMAX) {
            float2 t2 = P, t1 = __fmul2_rn(zz, P);
            accC[d3_cidx(m + 1, m)] = __fadd2_rn(accC[d3_cidx(m + 1, m)], t1);
            static_for<m + 2, LMAX + 1>([&](auto L) {
                constexpr int l = decltype(L)::value;
                const float az = float(cx::leg_A(l, m)) * z;
                const float2 n = __ffma2_rn(make_float2(az, az), t1, make_float2(-t2.x, -t2.y));
                accC[d3_cidx(l, m)] = __fadd2_rn(accC[d3_cidx(l, m)], n);
                t2 = t1;
                t1 = n;
            });
        }
    });
}

// D=4: w Rs_{l2}^{l1}(u1, u2, u3) Cs^{(l2+1)}_{l3-l2}(u4), l1 <= l2 <= l3 <= LMAX
template <int LMAX, typename T>
__device__ __forceinline__ void accum_d4(T* acc, T u1, T u2, T u3, T u4, T w)
{
    const T rho2 = fma(u1, u1, fma(u2, u2, u3 * u3));
    // Gegenbauer Cs^{(lam)}_n(u4) for lam = l2 + 1, n = 0..LMAX - l2
    T G[LMAX + 1][LMAX + 1];
    static_for<0, LMAX + 1>([&](auto L2) {
        constexpr int l2 = decltype(L2)::value;
        constexpr int lam = l2 + 1;
        G[l2][0] = T(1);
        if constexpr (LMAX - l2 >= 1) G[l2][1] = u4;
        static_for<2, LMAX - l2 + 1>([&](auto Nn) {
            constexpr int n = decltype(Nn)::value;
            constexpr T B = T(cx::geg_B(n, lam));
            G[l2][n] = fma(B * u4, G[l2][n - 1], -G[l2][n - 2]);
        });
    });
    T pr = w, pi = T(0);  // w (u1 - i u2)^{l1}
    static_for<0, LMAX + 1>([&](auto M) {
        constexpr int m = decltype(M)::value;  // l1
        if constexpr (m > 0) {
            T nr = fma(pr, u1, pi * u2);
            T ni = fma(pi, u1, -(pr * u2));
            pr = nr;
            pi = ni;
        }
        T t2r = T(0), t2i = T(0), t1r = pr, t1i = pi;  // Rs_{l2 = m}
        static_for<m, LMAX + 1>([&](auto L2) {
            constexpr int l2 = decltype(L2)::value;
            T rr, ri;
            if constexpr (l2 == m) {
                rr = pr;
                ri = pi;
            } else if constexpr (l2 == m + 1) {
                rr = u3 * pr;
                ri = u3 * pi;
                t2r = t1r;
                t2i = t1i;
                t1r = rr;
                t1i = ri;
            } else {
                constexpr T A = T(cx::leg_A(l2, m));
                T az = A * u3;
                rr = fma(az, t1r, -(rho2 * t2r));
                ri = fma(az, t1i, -(rho2 * t2i));
                t2r = t1r;
                t2i = t1i;
                t1r = rr;
                t1i = ri;
            }
            static_for<l2, LMAX + 1>([&](auto L3) {
                constexpr int l3 = decltype(L3)::value;
                const T g = G[l2][l3 - l2];
                acc[q_index_d4(l3, l2, m)] = fma(rr, g, acc[q_index_d4(l3, l2, m)]);
                if constexpr (m > 0) acc[q_index_d4(l3, l2, m) + 1] = fma(ri, g, acc[q_index_d4(l3, l2, m) + 1]);
            });
        });
    });
}

}  // namespace npcf
