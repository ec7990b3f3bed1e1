// npcf_math.h -- compile-time constants of libnpcf's harmonic recurrences and
// coupling coefficients.  Usable from host and device code (constexpr only).
//
// D=3 harmonics (eq. hypersph-def with K=2, the paper's two/three-dimensional
// forms): with z = cos(theta), the Ferrers function of DLMF 14.6.1 gives
//     Y_{l m}(r^) = N_lm Q_l^m(z) (x + i y)^m,  m >= 0,  r^ = (x, y, z),
//     N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),  Q_l^m = d^m P_l / dz^m,
// and Y_{l,-m} = (-1)^m Y*_{l m} (eq. complex-conj-hypersph).  Q obeys the
// derivative of Bonnet's recurrence
//     (l-m) Q_l = (2l-1) z Q_{l-1} - (l+m-1) Q_{l-2},  Q_m = (2m-1)!!,
// which the kernels run in a scaled form Qs_l = Q_l / s_lm chosen so that the
// second coefficient is -1:  Qs_l = A_lm z Qs_{l-1} - Qs_{l-2},  Qs_m = 1,
// Qs_{m+1} = z.  The constant N_lm s_lm is applied once per primary.
//
// D=4 harmonics (eq. hypersph-def with K=3): the half-odd Ferrers function of
// Theta_3 reduces to a Gegenbauer polynomial,
//     Theta_3 = c_{l2 l3} sin^{l2}(theta_3) C^{(l2+1)}_{l3-l2}(cos theta_3),
// with c > 0 fixed by the norm of Theta_3 on (0, pi) with weight sin^2.  The
// product Theta_1 Theta_2 sin^{l2}(theta_3) is the solid harmonic of
// (u1, u2, u3) = the first three components of the unit 4-vector, whose
// recurrence is the one above with z -> u3 and Qs_{l-2} -> rho^2 Qs_{l-2},
// rho^2 = u1^2 + u2^2 + u3^2.  C^{(lam)}_n runs scaled as
//     Cs_n = B_n t Cs_{n-1} - Cs_{n-2},  Cs_0 = 1, Cs_1 = t,  C_n = g_n Cs_n.
#pragma once

namespace npcf {
namespace cx {

constexpr double kPi = 3.14159265358979323846;

constexpr double fact(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return f;
}

constexpr double sqrt_newton(double x)
{
    if (x <= 0.0) return 0.0;
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 200; ++i) {
        double nr = 0.5 * (r + x / r);
        if (nr == r) break;
        r = nr;
    }
    return r;
}

constexpr double neg1_pow(int e) { return (e % 2 == 0) ? 1.0 : -1.0; }

// s_lm of the scaled Legendre-derivative recurrence (l >= m >= 0)
constexpr double leg_scale(int l, int m)
{
    double sm = 1.0;
    for (int k = 1; k <= m; ++k) sm *= (double)(2 * k - 1);  // (2m-1)!!
    if (l == m) return sm;
    double s_prev2 = sm;                      // s_{l-2} candidate chain
    double s_prev1 = (double)(2 * m + 1) * sm; // s_{m+1}
    if (l == m + 1) return s_prev1;
    double s = 0.0;
    for (int L = m + 2; L <= l; ++L) {
        s = (double)(L + m - 1) / (double)(L - m) * s_prev2;
        s_prev2 = s_prev1;
        s_prev1 = s;
    }
    return s;
}

// A_lm = ((2l-1)/(l-m)) s_{l-1,m} / s_{l,m}, for l >= m + 2
constexpr double leg_A(int l, int m)
{
    return (double)(2 * l - 1) / (double)(l - m) * leg_scale(l - 1, m) / leg_scale(l, m);
}

// g_n of the scaled Gegenbauer recurrence for C^{(lam)}_n, integer lam >= 1
constexpr double geg_scale(int n, int lam)
{
    if (n == 0) return 1.0;
    if (n == 1) return 2.0 * lam;
    double g2 = 1.0, g1 = 2.0 * lam, g = 0.0;
    for (int k = 2; k <= n; ++k) {
        g = (double)(k + 2 * lam - 2) / (double)k * g2;
        g2 = g1;
        g1 = g;
    }
    return g;
}

constexpr double geg_B(int n, int lam)
{
    return 2.0 * (double)(n + lam - 1) / (double)n * geg_scale(n - 1, lam) / geg_scale(n, lam);
}

// Wigner 3j symbol (j1 j2 j3; m1 m2 m3) by Racah's single-sum formula.
constexpr double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3)
{
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j3 < (j1 > j2 ? j1 - j2 : j2 - j1) || j3 > j1 + j2) return 0.0;
    if (m1 > j1 || -m1 > j1 || m2 > j2 || -m2 > j2 || m3 > j3 || -m3 > j3) return 0.0;
    double delta = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
    double pre = sqrt_newton(delta * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                             fact(j3 + m3) * fact(j3 - m3));
    int kmin = 0;
    if (j2 - j3 - m1 > kmin) kmin = j2 - j3 - m1;
    if (j1 - j3 + m2 > kmin) kmin = j1 - j3 + m2;
    int kmax = j1 + j2 - j3;
    if (j1 - m1 < kmax) kmax = j1 - m1;
    if (j2 + m2 < kmax) kmax = j2 + m2;
    double s = 0.0;
    for (int k = kmin; k <= kmax; ++k)
        s += neg1_pow(k) / (fact(k) * fact(j1 + j2 - j3 - k) * fact(j1 - m1 - k) * fact(j2 + m2 - k) *
                            fact(j3 - j2 + m1 + k) * fact(j3 - j1 - m2 + k));
    int ph = j1 - j2 - m3;
    return neg1_pow(ph < 0 ? -ph : ph) * pre * s;
}

// D=3, N=4 coupling: the product of the two CGs of eq. Coupling-C with the
// final one coupling to zero collapses to (-1)^{l1+l2+l3} (l1 l2 l3; m1 m2 m3).
constexpr double coupling_d3n4(int l1, int l2, int l3, int m1, int m2, int m3)
{
    return neg1_pow(l1 + l2 + l3) * wigner3j(l1, l2, l3, m1, m2, m3);
}

// number of (l1, l2, l3) <= lmax obeying the triangle rule, and the index of
// one such triple in lexicographic order
constexpr int num_lambda_d3n4(int lmax)
{
    int c = 0;
    for (int a = 0; a <= lmax; ++a)
        for (int b = 0; b <= lmax; ++b)
            for (int d = 0; d <= lmax; ++d)
                if (d >= (a > b ? a - b : b - a) && d <= a + b) ++c;
    return c;
}

constexpr int lambda_index_d3n4(int lmax, int l1, int l2, int l3)
{
    int c = 0;
    for (int a = 0; a <= lmax; ++a)
        for (int b = 0; b <= lmax; ++b)
            for (int d = 0; d <= lmax; ++d) {
                if (!(d >= (a > b ? a - b : b - a) && d <= a + b)) continue;
                if (a == l1 && b == l2 && d == l3) return c;
                ++c;
            }
    return -1;
}

}  // namespace cx
}  // namespace npcf
