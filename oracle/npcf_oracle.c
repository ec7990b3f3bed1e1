/*
 * npcf_oracle.c -- plain, slow, FP64 CPU evaluation of the isotropic NPCF
 * estimator of Philcox & Slepian, "Efficient Computation of N-Point
 * Correlation Functions in D Dimensions" (arXiv:2106.10278).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this file; only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA library.
 *
 * What it computes (each function cites the passage it follows):
 *   - hyperspherical harmonics Y_l(r^) for D = 2, 3, 4         (eq. hypersph-def)
 *   - Ferrers functions P^mu_nu for integer and half-odd nu,mu (DLMF 14.6.1,
 *     14.9.3, 18.5.8, 14.5.11-12, 14.10.1)
 *   - Wigner 3j symbols (Racah formula, DLMF 34.2.4), D=3 Clebsch-Gordan
 *     coefficients                                             (eq. CG-examples)
 *   - the zero-total-angular-momentum coupling coefficients    (eq. Coupling-C,
 *                                                               eq. zero-ang-mom-states)
 *   - the separable discrete estimator                         (eq. NPCF-estimator-discrete)
 *   - the naive O(n^N) estimator projected on the same basis   (eq. NPCF-estimator-intro-discrete
 *                                                               with eq. B-hypersph)
 *   - the N=3 estimator through the addition theorem, with its analytic
 *     gradient in positions and weights                        (Sec. "Derivation", eq. zeta-basis-decomp)
 *   - the estimator of a field on a periodic grid, by direct sums over node
 *     offsets                                                  (Sec. "Application to Gridded Data",
 *                                                               eq. alm-bin-def, eq. NPCF-mult-estimator)
 *   - the estimator of points on the 2-sphere with the D = 2 basis about each
 *     point                                                    (Sec. "Cosmic Microwave Background")
 *   - the D = 3 anisotropic basis about a fixed line of sight, N = 3, 4
 *                                                              (Sec. "Large-Scale Structure")
 *
 * Readings of the paper that this file takes where the text is silent or
 * garbled (the CUDA library takes the same ones, under the same numbers):
 *   R1 the self pair k=j and any pair with r=0 exactly are skipped (Y(0) is
 *      undefined);
 *   R2 degenerate tuples (two secondaries equal) are kept, as in the naive
 *      sum over all N-tuplets; on request (remove_self) they are excluded
 *      exactly, which concerns only N=3 keys with b1 = b2;
 *   R3 bins are half-open [e_b, e_{b+1}), decided by comparing the FP64 r^2
 *      with the FP64 square of the edge;
 *   R4 v_b is the volume of the shell, |S^{D-1}|/D (e_{b+1}^D - e_b^D);
 *   R5 theta_1 = atan2(x_2, x_1) and cos(theta_K) = x_{K+1}/|x_{1..K+1}|;
 *   R6 for D=4, N=3 the zero coupling is (-1)^(l-l_1)/sqrt(dim_l) on states
 *      with l_1' = -l_1 and equal higher indices (the D=3 value, extended);
 *   R7 periodic boxes use the minimum image; V_D is the box volume;
 *   R8 N=3 keys have b1 <= b2 (or b1 < b2 on request), N=4 keys b1<b2<b3,
 *      N=5 keys b1<b2<b3<b4;
 *   R15 the D=3 5PCF (eq. D=3-NPCF, intermediate label l12) keeps the even-parity labels
 *      (l1+l2+l3+l4 even), which give the 585 angular components the paper counts for
 *      lmax=4; its printed coefficient sqrt(2 l12 - 1) is read as sqrt(2 l12 + 1), the
 *      value the CG chain of eq. Coupling-C gives;
 *   R16 gridded data: the integrals over space and over the separation become
 *      sums over grid nodes times the node volume; a^b_l keeps the 1/v_b of
 *      eq. alm-bin-def (the FFT form printed for grids drops it) with v_b the
 *      shell volume of R4; the separation o = 0 is skipped as in R1.  The FFT
 *      form's kernel is read as Y*_l Theta^b: relabelling r -> -r in
 *      eq. alm-bin-def moves the parity sign (-1)^{l_{D-1}} out but leaves the
 *      conjugate on Y (the kernel printed as Y_l Theta^b gives other values).
 *   R17 the 2-sphere: the radial coordinate is the great-circle angle theta,
 *      binned in half-open intervals of cos theta (the paper states its bins as
 *      a range of cos theta); v_b is the area 2 pi (c_{b+1} - c_b) of the
 *      annulus and 1/(4 pi) replaces 1/V; the azimuth is counter-clockwise
 *      seen from outside the sphere (the flat D = 2 orientation at the north
 *      pole); a^b_l uses Y*_l as in eq. NPCF-estimator-discrete (the section
 *      prints e^{+il phi}, which would conjugate every coefficient).  Two
 *      points whose unit vectors coincide have no azimuth and are no pair, as
 *      r = 0 is skipped in a box (R1).
 *   R18 the anisotropic basis: the line of sight is the fixed x_3 axis (as
 *      the paper sets it); N=3 labels (l1, l2, L) with every l1, l2 <= lmax
 *      and every L of the triangle rule, coupled as printed for the
 *      redshift-space 3PCF; N=4 labels (l1, l2, l12, l3, L) through
 *      eq. Coupling-C with the final state (L, 0), l12 and L unbounded but for
 *      the triangle rules; a uses Y* and 1/v_b as in the isotropic estimator.
 *
 * Floating point: compile with -ffp-contract=off so that no multiply-add is
 * fused; r^2 is formed as ((dx*dx + dy*dy) + dz*dz) + ... left to right.
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define OR_MAXD 4
#define OR_MAXL 16
#define OR_MAXB 64

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* factorials and binomials (exact in double up to 170!, used far below) */
static double fact(int k)
{
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    return fact(n) / (fact(k) * fact(n - k));
}

static double sgn_pow(int e) { return (e % 2 == 0) ? 1.0 : -1.0; } /* (-1)^e */

/* ------------------------------------------------------------------ */
/* Ferrers (on-the-cut associated Legendre) functions.                 */

/* Legendre polynomial P_n(x) by its explicit sum (DLMF 18.5.8),
 * differentiated mu times term by term. */
static double legendre_deriv(int n, int mu, double x)
{
    double s = 0.0;
    for (int k = 0; 2 * k <= n; ++k) {
        int p = n - 2 * k;
        if (p < mu) continue;
        double c = sgn_pow(k) * binom(n, k) * binom(2 * n - 2 * k, n);
        s += c * (fact(p) / fact(p - mu)) * pow(x, (double)(p - mu));
    }
    return s / pow(2.0, (double)n);
}

/* P^mu_n(x) for integers n >= 0, |mu| <= n (DLMF 14.6.1 for mu >= 0, with
 * the (-1)^mu phase; DLMF 14.9.3 for mu < 0). */
static double ferrers_int(int n, int mu, double x)
{
    if (mu >= 0) {
        return sgn_pow(mu) * pow(1.0 - x * x, 0.5 * mu) * legendre_deriv(n, mu, x);
    }
    int m = -mu;
    return sgn_pow(m) * fact(n - m) / fact(n + m) * ferrers_int(n, m, x);
}

/* sin^{-1/2}(th) P^{-(k+1/2)}_{L+1/2}(cos th) for integers 0 <= k <= L.
 * With mu = k + 1/2, the hypergeometric factor of DLMF 14.3.1 is (1-z)^mu when
 * the degree equals minus the order, so P^{-mu}_{mu}(x) = (1-x^2)^{mu/2} /
 * (2^mu Gamma(1+mu)), i.e. sin^{-1/2} P^{-mu}_{mu} = sin^k / (2^mu Gamma(1+mu));
 * the degree recurrence DLMF 14.10.3, run upwards,
 *   (nu - m + 1) P^m_{nu+1} = (2 nu + 1) x P^m_nu - (nu + m) P^m_{nu-1}   (m = -mu),
 * whose last term vanishes at the first step, carries it to nu = L + 1/2.
 * The factor sin^{-1/2} is linear in the recurrence, so nothing is singular at
 * the poles (th = 0, pi), and the upward degree recurrence is stable there. */
static double ferrers_half_reg(int L, int k, double th)
{
    double mu = k + 0.5, m = -mu, x = cos(th);
    double prev = 0.0;
    double cur = pow(sin(th), (double)k) / (pow(2.0, mu) * tgamma(1.0 + mu));
    for (int step = k; step < L; ++step) { /* cur holds degree nu = step + 1/2 */
        double nu = step + 0.5;
        double next = ((2.0 * nu + 1.0) * x * cur - (nu + m) * prev) / (nu - m + 1.0);
        prev = cur;
        cur = next;
    }
    return cur;
}

/* P^{-(k+1/2)}_{L+1/2}(cos th) for 0 < th < pi (the D=4 factor of eq. hypersph-def) */
static double ferrers_half(int L, int k, double th)
{
    return sqrt(sin(th)) * ferrers_half_reg(L, k, th);
}

/* ------------------------------------------------------------------ */
/* Hyperspherical harmonic states and values.                          */

typedef struct { int l[OR_MAXD - 1]; } state_t; /* l[0] = l_1 (signed) ... l[D-2] = total */

/* Enumerate states obeying the selection rules (eq. selection-rules):
 * -l_2 <= l_1 <= l_2 <= ... <= l_{D-1} <= lmax; D=2 has l_1 in [-lmax, lmax]. */
static int enum_states(int D, int lmax, state_t *out)
{
    int ns = 0;
    if (D == 2) {
        for (int l1 = -lmax; l1 <= lmax; ++l1) {
            if (out) { memset(&out[ns], 0, sizeof(state_t)); out[ns].l[0] = l1; }
            ++ns;
        }
    } else if (D == 3) {
        for (int l2 = 0; l2 <= lmax; ++l2)
            for (int l1 = -l2; l1 <= l2; ++l1) {
                if (out) { memset(&out[ns], 0, sizeof(state_t)); out[ns].l[0] = l1; out[ns].l[1] = l2; }
                ++ns;
            }
    } else if (D == 4) {
        for (int l3 = 0; l3 <= lmax; ++l3)
            for (int l2 = 0; l2 <= l3; ++l2)
                for (int l1 = -l2; l1 <= l2; ++l1) {
                    if (out) {
                        memset(&out[ns], 0, sizeof(state_t));
                        out[ns].l[0] = l1; out[ns].l[1] = l2; out[ns].l[2] = l3;
                    }
                    ++ns;
                }
    }
    return ns;
}

/* Y_{l_1..l_{D-1}}(d/|d|) from eq. hypersph-def: the product of
 * Theta_1 = e^{i l_1 th_1}/sqrt(2 pi) (the D=2 form printed with the
 * paper's two- and three-dimensional harmonics) and, for 2 <= K <= D-1,
 * Theta_K = sqrt((2 l_K + K - 1)/2 (l_K + l_{K-1} + K - 2)!/(l_K - l_{K-1})!)
 *           sin^{1-K/2}(th_K) P^{-(l_{K-1}+K/2-1)}_{l_K+K/2-1}(cos th_K).
 * For odd K the factor sin^{1-K/2} P is formed as sin^{(3-K)/2} times
 * sin^{-1/2} P, which is regular at the poles.  Where x_1..x_{K+1} are all
 * zero (lattice directions such as (0, 0, 0, 1)) th_K is undefined: the first
 * factor above it with a non-zero component is proportional to
 * sin^{l_{K'-1}}(th_{K'}) = 0 unless every lower label vanishes, in which case
 * Theta_K does not depend on th_K; th_K = pi/2 is taken. */
static cplx harmonic(int D, const state_t *s, const double *d)
{
    double th1 = atan2(d[1], d[0]);
    cplx y = cexp(I * (double)s->l[0] * th1) / sqrt(2.0 * M_PI);
    double rho2 = d[0] * d[0] + d[1] * d[1];
    for (int K = 2; K <= D - 1; ++K) {
        double rhoK2 = rho2 + d[K] * d[K];          /* |x_{1..K+1}|^2 */
        double cth = rhoK2 > 0.0 ? d[K] / sqrt(rhoK2) : 0.0;
        if (cth > 1.0) cth = 1.0;
        if (cth < -1.0) cth = -1.0;
        double th = acos(cth);
        int lK = s->l[K - 1], lKm1 = s->l[K - 2];
        double norm;
        double val;
        if (K % 2 == 0) {
            /* integer degree and order: K/2 - 1 is an integer */
            int h = K / 2 - 1;
            norm = sqrt((2.0 * lK + K - 1) / 2.0 * fact(lK + lKm1 + K - 2) / fact(lK - lKm1));
            val = pow(sin(th), 1.0 - 0.5 * K) * ferrers_int(lK + h, -(lKm1 + h), cth);
        } else {
            /* half-odd degree and order: K/2 - 1 = (K-3)/2 + 1/2 */
            int h = (K - 3) / 2;
            norm = sqrt((2.0 * lK + K - 1) / 2.0 * fact(lK + lKm1 + K - 2) / fact(lK - lKm1));
            val = pow(sin(th), 1.5 - 0.5 * K) * ferrers_half_reg(lK + h, lKm1 + h, th);
        }
        y *= norm * val;
        rho2 = rhoK2;
    }
    return y;
}

/* ------------------------------------------------------------------ */
/* Wigner 3j symbol by the Racah formula (DLMF 34.2.4).               */
static double wigner3j(int j1, int j2, int j3, int m1, int m2, int m3)
{
    if (m1 + m2 + m3 != 0) return 0.0;
    if (j3 < abs(j1 - j2) || j3 > j1 + j2) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(m3) > j3) return 0.0;
    double tri = fact(j1 + j2 - j3) * fact(j1 - j2 + j3) * fact(-j1 + j2 + j3) / fact(j1 + j2 + j3 + 1);
    double pre = sqrt(tri * fact(j1 + m1) * fact(j1 - m1) * fact(j2 + m2) * fact(j2 - m2) *
                      fact(j3 + m3) * fact(j3 - m3));
    int kmin = 0;
    if (j2 - j3 - m1 > kmin) kmin = j2 - j3 - m1;
    if (j1 - j3 + m2 > kmin) kmin = j1 - j3 + m2;
    int kmax = j1 + j2 - j3;
    if (j1 - m1 < kmax) kmax = j1 - m1;
    if (j2 + m2 < kmax) kmax = j2 + m2;
    double s = 0.0;
    for (int k = kmin; k <= kmax; ++k) {
        s += sgn_pow(k) / (fact(k) * fact(j1 + j2 - j3 - k) * fact(j1 - m1 - k) * fact(j2 + m2 - k) *
                           fact(j3 - j2 + m1 + k) * fact(j3 - j1 - m2 + k));
    }
    return sgn_pow(abs(j1 - j2 - m3)) * pre * s;
}

/* D=3 Clebsch-Gordan coefficient <l1 m1, l2 m2 | L M> as printed in
 * eq. CG-examples: (-1)^(-l1+l2-M) sqrt(2L+1) (l1 l2 L; m1 m2 -M). */
static double cg_d3(int l1, int m1, int l2, int m2, int L, int M)
{
    return sgn_pow(abs(-l1 + l2 - M)) * sqrt(2.0 * L + 1.0) * wigner3j(l1, l2, L, m1, m2, -M);
}

/* ------------------------------------------------------------------ */
/* Output keys and coupling terms.                                     */

typedef struct { int b[4]; int l[5]; } okey_t;  /* unused entries are -1 (bins) / 0 (ells) */

typedef struct {
    int nl;            /* entries of Lambda used: 1 for N=3, 3 for N=4, 5 for N=5 */
    int l[5];
} lam_t;

/* Angular labels Lambda of the isotropic basis.
 * N=3: Lambda = (l), l = 0..lmax (the final CG forces l^1 = l^2 = l).
 * N=4, D=3: Lambda = (l1, l2, l3) with l^12 = l3 forced by the final CG,
 *           every l <= lmax and (l1, l2, l3) obeying the triangle rule.
 * N=4, D=2: the signed (l1, l2, l3) with l1 + l2 + l3 = 0, l1 >= 0.
 * N=5, D=3: (l1, l2, l12, l3, l4): l1..l4 <= lmax, l12 coupling l1 and l2 and then l12 and
 *           l3 coupling to l4 (triangle rules), even parity l1+l2+l3+l4 (the components the
 *           paper counts for its 5PCF, reading R15). */
static int enum_lambdas(int D, int N, int lmax, lam_t *out)
{
    int nl = 0;
    if (N == 3) {
        for (int l = 0; l <= lmax; ++l) {
            if (out) { out[nl].nl = 1; out[nl].l[0] = l; out[nl].l[1] = 0; out[nl].l[2] = 0; out[nl].l[3] = 0; out[nl].l[4] = 0; }
            ++nl;
        }
    } else if (N == 4 && D == 3) {
        for (int l1 = 0; l1 <= lmax; ++l1)
            for (int l2 = 0; l2 <= lmax; ++l2)
                for (int l3 = 0; l3 <= lmax; ++l3) {
                    if (l3 < abs(l1 - l2) || l3 > l1 + l2) continue;
                    if (out) { out[nl].nl = 3; out[nl].l[0] = l1; out[nl].l[1] = l2; out[nl].l[2] = l3; out[nl].l[3] = 0; out[nl].l[4] = 0; }
                    ++nl;
                }
    } else if (N == 4 && D == 2) {
        for (int l1 = 0; l1 <= lmax; ++l1)
            for (int l2 = -lmax; l2 <= lmax; ++l2) {
                int l3 = -l1 - l2;
                if (abs(l3) > lmax) continue;
                if (out) { out[nl].nl = 3; out[nl].l[0] = l1; out[nl].l[1] = l2; out[nl].l[2] = l3; out[nl].l[3] = 0; out[nl].l[4] = 0; }
                ++nl;
            }
    } else if (N == 5 && D == 3) {
        for (int l1 = 0; l1 <= lmax; ++l1)
            for (int l2 = 0; l2 <= lmax; ++l2)
                for (int l12 = abs(l1 - l2); l12 <= l1 + l2; ++l12)
                    for (int l3 = 0; l3 <= lmax; ++l3)
                        for (int l4 = 0; l4 <= lmax; ++l4) {
                            if (l4 < abs(l12 - l3) || l4 > l12 + l3) continue;
                            if ((l1 + l2 + l3 + l4) % 2) continue;
                            if (out) {
                                out[nl].nl = 5;
                                out[nl].l[0] = l1; out[nl].l[1] = l2; out[nl].l[2] = l12;
                                out[nl].l[3] = l3; out[nl].l[4] = l4;
                            }
                            ++nl;
                        }
    }
    return nl;
}

static int supported(int D, int N, int lmax, int nbins)
{
    if (lmax < 0 || lmax > 12 || nbins < 1 || nbins > OR_MAXB) return 0;
    if (N == 3) return D >= 2 && D <= 4;
    if (N == 4) return D == 2 || D == 3;
    if (N == 5) return D == 3 && lmax <= 6;
    return 0;
}

static int enum_keys(int D, int N, int lmax, int nbins, int bin_lt, okey_t *out)
{
    int nl = enum_lambdas(D, N, lmax, NULL);
    lam_t *lam = (lam_t *)malloc(sizeof(lam_t) * (nl > 0 ? nl : 1));
    enum_lambdas(D, N, lmax, lam);
    int nk = 0;
    if (N == 3) {
        for (int b1 = 0; b1 < nbins; ++b1)
            for (int b2 = b1 + (bin_lt ? 1 : 0); b2 < nbins; ++b2)
                for (int il = 0; il < nl; ++il) {
                    if (out) {
                        okey_t *k = &out[nk];
                        k->b[0] = b1; k->b[1] = b2; k->b[2] = -1; k->b[3] = -1;
                        k->l[0] = lam[il].l[0]; k->l[1] = 0; k->l[2] = 0; k->l[3] = 0; k->l[4] = 0;
                    }
                    ++nk;
                }
    } else if (N == 5) {
        for (int b1 = 0; b1 < nbins; ++b1)
            for (int b2 = b1 + 1; b2 < nbins; ++b2)
                for (int b3 = b2 + 1; b3 < nbins; ++b3)
                    for (int b4 = b3 + 1; b4 < nbins; ++b4)
                        for (int il = 0; il < nl; ++il) {
                            if (out) {
                                okey_t *k = &out[nk];
                                k->b[0] = b1; k->b[1] = b2; k->b[2] = b3; k->b[3] = b4;
                                for (int a = 0; a < 5; ++a) k->l[a] = lam[il].l[a];
                            }
                            ++nk;
                        }
    } else {
        for (int b1 = 0; b1 < nbins; ++b1)
            for (int b2 = b1 + 1; b2 < nbins; ++b2)
                for (int b3 = b2 + 1; b3 < nbins; ++b3)
                    for (int il = 0; il < nl; ++il) {
                        if (out) {
                            okey_t *k = &out[nk];
                            k->b[0] = b1; k->b[1] = b2; k->b[2] = b3; k->b[3] = -1;
                            k->l[0] = lam[il].l[0]; k->l[1] = lam[il].l[1]; k->l[2] = lam[il].l[2];
                            k->l[3] = 0; k->l[4] = 0;
                        }
                        ++nk;
                    }
    }
    free(lam);
    return nk;
}

/* One term of P^0_Lambda = sum_terms C prod_i Y_{s_i}(r^i) (eq. N-1-particle-basis-wavefunction). */
typedef struct { int s[4]; double c; } term_t;

static int state_index(int D, int lmax, const state_t *st)
{
    /* position of st in the enumeration order of enum_states */
    if (D == 2) return st->l[0] + lmax;
    if (D == 3) return st->l[1] * st->l[1] + (st->l[0] + st->l[1]);
    /* D == 4: states with l3' < l3 number sum_{l'<l3} (l'+1)^2 */
    int base = 0;
    for (int l = 0; l < st->l[2]; ++l) base += (l + 1) * (l + 1);
    return base + st->l[1] * st->l[1] + (st->l[0] + st->l[1]);
}

/* Terms of the coupling coefficient C^{Lambda;0} (eq. Coupling-C with
 * the CGs of eq. CG-examples), non-zero ones only. */
static int lambda_terms(int D, int N, int lmax, const lam_t *lam, term_t *out)
{
    int nt = 0;
    if (N == 3) {
        int l = lam->l[0];
        if (D == 2) {
            /* <l^1 l^2 | 0> = delta(l^1 + l^2, 0); key l means (l, -l) */
            if (out) {
                state_t a = {{l, 0, 0}}, b = {{-l, 0, 0}};
                out[nt].s[0] = state_index(D, lmax, &a);
                out[nt].s[1] = state_index(D, lmax, &b);
                out[nt].s[2] = -1;
                out[nt].s[3] = -1;
                out[nt].c = 1.0;
            }
            ++nt;
        } else if (D == 3) {
            for (int m1 = -l; m1 <= l; ++m1)
                for (int m2 = -l; m2 <= l; ++m2) {
                    double c = cg_d3(l, m1, l, m2, 0, 0);
                    if (c == 0.0) continue;
                    if (out) {
                        state_t a = {{m1, l, 0}}, b = {{m2, l, 0}};
                        out[nt].s[0] = state_index(D, lmax, &a);
                        out[nt].s[1] = state_index(D, lmax, &b);
                        out[nt].s[2] = -1;
                        out[nt].s[3] = -1;
                        out[nt].c = c;
                    }
                    ++nt;
                }
        } else if (D == 4) {
            /* reading R6 */
            double dim = (double)(l + 1) * (double)(l + 1);
            for (int l2 = 0; l2 <= l; ++l2)
                for (int l1 = -l2; l1 <= l2; ++l1) {
                    if (out) {
                        state_t a = {{l1, l2, l}}, b = {{-l1, l2, l}};
                        out[nt].s[0] = state_index(D, lmax, &a);
                        out[nt].s[1] = state_index(D, lmax, &b);
                        out[nt].s[2] = -1;
                        out[nt].s[3] = -1;
                        out[nt].c = sgn_pow(abs(l - l1)) / sqrt(dim);
                    }
                    ++nt;
                }
        }
    } else if (N == 4 && D == 2) {
        /* <l^1 l^2 | L^12> <L^12 l^3 | 0> = delta(l^1 + l^2 + l^3, 0) */
        if (out) {
            state_t a = {{lam->l[0], 0, 0}}, b = {{lam->l[1], 0, 0}}, c = {{lam->l[2], 0, 0}};
            out[nt].s[0] = state_index(D, lmax, &a);
            out[nt].s[1] = state_index(D, lmax, &b);
            out[nt].s[2] = state_index(D, lmax, &c);
            out[nt].s[3] = -1;
            out[nt].c = 1.0;
        }
        ++nt;
    } else if (N == 4 && D == 3) {
        int l1 = lam->l[0], l2 = lam->l[1], l3 = lam->l[2];
        for (int m1 = -l1; m1 <= l1; ++m1)
            for (int m2 = -l2; m2 <= l2; ++m2)
                for (int m3 = -l3; m3 <= l3; ++m3) {
                    /* sum over the intermediate [l^12] = M of the CG product */
                    double c = 0.0;
                    for (int M = -l3; M <= l3; ++M)
                        c += cg_d3(l1, m1, l2, m2, l3, M) * cg_d3(l3, M, l3, m3, 0, 0);
                    if (c == 0.0) continue;
                    if (out) {
                        state_t a = {{m1, l1, 0}}, b = {{m2, l2, 0}}, cc = {{m3, l3, 0}};
                        out[nt].s[0] = state_index(D, lmax, &a);
                        out[nt].s[1] = state_index(D, lmax, &b);
                        out[nt].s[2] = state_index(D, lmax, &cc);
                        out[nt].s[3] = -1;
                        out[nt].c = c;
                    }
                    ++nt;
                }
    } else if (N == 5 && D == 3) {
        /* <l1 m1 l2 m2 | l12 M12> <l12 M12 l3 m3 | l4 M> <l4 M l4 m4 | 0 0>, summed over the
         * intermediate projections M12 and M (eq. Coupling-C with the CGs of eq. CG-examples) */
        int l1 = lam->l[0], l2 = lam->l[1], l12 = lam->l[2], l3 = lam->l[3], l4 = lam->l[4];
        for (int m1 = -l1; m1 <= l1; ++m1)
            for (int m2 = -l2; m2 <= l2; ++m2)
                for (int m3 = -l3; m3 <= l3; ++m3)
                    for (int m4 = -l4; m4 <= l4; ++m4) {
                        double c = 0.0;
                        for (int M12 = -l12; M12 <= l12; ++M12) {
                            double c12 = cg_d3(l1, m1, l2, m2, l12, M12);
                            if (c12 == 0.0) continue;
                            for (int M = -l4; M <= l4; ++M)
                                c += c12 * cg_d3(l12, M12, l3, m3, l4, M) * cg_d3(l4, M, l4, m4, 0, 0);
                        }
                        if (c == 0.0) continue;
                        if (out) {
                            state_t a = {{m1, l1, 0}}, b = {{m2, l2, 0}}, cc = {{m3, l3, 0}}, dd = {{m4, l4, 0}};
                            out[nt].s[0] = state_index(D, lmax, &a);
                            out[nt].s[1] = state_index(D, lmax, &b);
                            out[nt].s[2] = state_index(D, lmax, &cc);
                            out[nt].s[3] = state_index(D, lmax, &dd);
                            out[nt].c = c;
                        }
                        ++nt;
                    }
    }
    return nt;
}

/* ------------------------------------------------------------------ */
/* Geometry.                                                           */

static double sphere_area(int D)
{
    /* |S^{D-1}| = 2 pi^{D/2} / Gamma(D/2) */
    return 2.0 * pow(M_PI, 0.5 * D) / tgamma(0.5 * D);
}

/* separation y_k - y_j, minimum image when periodic (reading R7) */
static void separation(int D, const double *yk, const double *yj, const double *box, int periodic, double *d)
{
    for (int a = 0; a < D; ++a) {
        double v = yk[a] - yj[a];
        if (periodic) {
            double L = box[a];
            if (v > 0.5 * L) v -= L;
            else if (v < -0.5 * L) v += L;
        }
        d[a] = v;
    }
}

static double norm2(int D, const double *d)
{
    double s = d[0] * d[0];
    for (int a = 1; a < D; ++a) s = s + d[a] * d[a];
    return s;
}

/* bin of a squared separation, -1 outside [e_0, e_nb) (reading R3) */
static int bin_of(double r2, int nbins, const double *edges)
{
    if (r2 <= 0.0) return -1; /* reading R1 */
    if (r2 < edges[0] * edges[0]) return -1;
    for (int b = 0; b < nbins; ++b)
        if (r2 < edges[b + 1] * edges[b + 1]) return b;
    return -1;
}

/*
 * The geometry of one pair (j, k): the bin of the separation (-1 outside the
 * bins, or at r = 0) and the direction handed to the harmonics.
 *   - Euclidean box (D = 2..4): the minimum-image separation y_k - y_j, binned
 *     on its squared length (readings R3, R7);
 *   - the 2-sphere (Sec. "Cosmic Microwave Background", reading R17): the
 *     radial coordinate is the great-circle angle theta between the unit
 *     vectors n_j and n_k, binned on cos theta = n_j . n_k in half-open
 *     intervals [c_b, c_{b+1}); the direction is the tangent vector
 *     n_k - (n_j . n_k) n_j in a right-handed frame (e1, e2, n_j) at the
 *     primary, so the D = 2 harmonics see the azimuth phi about n_j.  With
 *     sum l = 0 the isotropic keys do not depend on the choice of e1.
 */
typedef struct {
    int sphere;          /* 0: Euclidean box, 1: unit 2-sphere */
    int Dp;              /* components of a position: D, or 3 on the sphere */
    int Dh;              /* dimension of the harmonics: D, or 2 on the sphere */
    int nbins;
    const double *edges; /* radial edges (box) or cos(theta) edges (sphere) */
    const double *box;
    int periodic;
    double e1[3], e2[3]; /* tangent frame at the current primary (sphere) */
} geom_t;

static void geom_primary(geom_t *g, const double *yj)
{
    if (!g->sphere) return;
    /* e1: the coordinate axis least aligned with n_j, projected on the tangent plane */
    int a0 = 0;
    for (int a = 1; a < 3; ++a)
        if (fabs(yj[a]) < fabs(yj[a0])) a0 = a;
    double u[3] = {0.0, 0.0, 0.0};
    u[a0] = 1.0;
    double c = yj[a0], nu = 0.0;
    for (int a = 0; a < 3; ++a) {
        u[a] -= c * yj[a];
        nu += u[a] * u[a];
    }
    nu = sqrt(nu);
    for (int a = 0; a < 3; ++a) g->e1[a] = u[a] / nu;
    /* e2 = n_j x e1 */
    g->e2[0] = yj[1] * g->e1[2] - yj[2] * g->e1[1];
    g->e2[1] = yj[2] * g->e1[0] - yj[0] * g->e1[2];
    g->e2[2] = yj[0] * g->e1[1] - yj[1] * g->e1[0];
}

static int geom_pair(const geom_t *g, const double *yk, const double *yj, double *d)
{
    if (!g->sphere) {
        separation(g->Dp, yk, yj, g->box, g->periodic, d);
        return bin_of(norm2(g->Dp, d), g->nbins, g->edges);
    }
    /* coinciding directions have no azimuth: skipped, as r = 0 is in a box (reading R1) */
    if (yk[0] == yj[0] && yk[1] == yj[1] && yk[2] == yj[2]) return -1;
    double c = (yk[0] * yj[0] + yk[1] * yj[1]) + yk[2] * yj[2];
    if (c < g->edges[0]) return -1;
    int b = -1;
    for (int i = 0; i < g->nbins; ++i)
        if (c < g->edges[i + 1]) {
            b = i;
            break;
        }
    if (b < 0) return -1;
    double t[3];
    for (int a = 0; a < 3; ++a) t[a] = yk[a] - c * yj[a];
    d[0] = (t[0] * g->e1[0] + t[1] * g->e1[1]) + t[2] * g->e1[2];
    d[1] = (t[0] * g->e2[0] + t[1] * g->e2[1]) + t[2] * g->e2[2];
    return b;
}

/* ------------------------------------------------------------------ */
/* Public entry points (C ABI, called from Python through ctypes).     */

int npcf_oracle_nstates(int D, int lmax) { return enum_states(D, lmax, NULL); }

int npcf_oracle_states(int D, int lmax, int *l_out /* nstates x 3 */)
{
    int ns = enum_states(D, lmax, NULL);
    state_t *st = (state_t *)malloc(sizeof(state_t) * ns);
    enum_states(D, lmax, st);
    for (int i = 0; i < ns; ++i)
        for (int a = 0; a < 3; ++a) l_out[3 * i + a] = (a < D - 1) ? st[i].l[a] : 0;
    free(st);
    return ns;
}

/* Y for every state at every direction: out[(i*ns + s)*2 + {0,1}] */
int npcf_oracle_harmonics(int D, int lmax, const double *dirs, int64_t nd, double *out)
{
    if (D < 2 || D > 4) return -1;
    int ns = enum_states(D, lmax, NULL);
    state_t *st = (state_t *)malloc(sizeof(state_t) * ns);
    enum_states(D, lmax, st);
    for (int64_t i = 0; i < nd; ++i)
        for (int s = 0; s < ns; ++s) {
            cplx y = harmonic(D, &st[s], dirs + i * D);
            out[2 * (i * ns + s)] = creal(y);
            out[2 * (i * ns + s) + 1] = cimag(y);
        }
    free(st);
    return ns;
}

double npcf_oracle_wigner3j(int j1, int j2, int j3, int m1, int m2, int m3)
{
    return wigner3j(j1, j2, j3, m1, m2, m3);
}

double npcf_oracle_cg_d3(int l1, int m1, int l2, int m2, int L, int M) { return cg_d3(l1, m1, l2, m2, L, M); }

double npcf_oracle_ferrers_int(int n, int mu, double x) { return ferrers_int(n, mu, x); }

double npcf_oracle_ferrers_half(int L, int k, double th) { return ferrers_half(L, k, th); }

int npcf_oracle_nkeys(int D, int N, int lmax, int nbins, int bin_lt)
{
    if (!supported(D, N, lmax, nbins)) return -1;
    return enum_keys(D, N, lmax, nbins, bin_lt, NULL);
}

int npcf_oracle_keys(int D, int N, int lmax, int nbins, int bin_lt, int *keys /* nkeys x 9 */)
{
    if (!supported(D, N, lmax, nbins)) return -1;
    int nk = enum_keys(D, N, lmax, nbins, bin_lt, NULL);
    okey_t *k = (okey_t *)malloc(sizeof(okey_t) * (nk > 0 ? nk : 1));
    enum_keys(D, N, lmax, nbins, bin_lt, k);
    for (int i = 0; i < nk; ++i) {  /* b1..b4, l1..l5 */
        for (int a = 0; a < 4; ++a) keys[9 * i + a] = k[i].b[a];
        for (int a = 0; a < 5; ++a) keys[9 * i + 4 + a] = k[i].l[a];
    }
    free(k);
    return nk;
}

/* Coupling terms of every Lambda, flattened: for lambda index il the terms
 * are returned as (s1, s2, s3, s4, c) rows (unused states -1).  Used by the tests to pin
 * the coupling against independent formulas. */
int npcf_oracle_coupling(int D, int N, int lmax, int il, int *s_out /* nt x 4 */, double *c_out)
{
    if (!supported(D, N, lmax, 1)) return -1;
    int nl = enum_lambdas(D, N, lmax, NULL);
    if (il < 0 || il >= nl) return -1;
    lam_t *lam = (lam_t *)malloc(sizeof(lam_t) * nl);
    enum_lambdas(D, N, lmax, lam);
    int nt = lambda_terms(D, N, lmax, &lam[il], NULL);
    if (s_out && c_out) {
        term_t *t = (term_t *)malloc(sizeof(term_t) * (nt > 0 ? nt : 1));
        lambda_terms(D, N, lmax, &lam[il], t);
        for (int i = 0; i < nt; ++i) {
            for (int a = 0; a < 4; ++a) s_out[4 * i + a] = t[i].s[a];
            c_out[i] = t[i].c;
        }
        free(t);
    }
    free(lam);
    return nt;
}

/* lambda index of a key's angular labels (keys are ordered bins-major) */
static int key_lambda(const okey_t *k, const lam_t *lam, int nl)
{
    for (int i = 0; i < nl; ++i) {
        int same = 1;
        for (int a = 0; a < 5; ++a) same = same && lam[i].l[a] == k->l[a];
        if (same) return i;
    }
    return -1;
}

/*
 * The estimator.  brute = 0: separable form, eq. NPCF-estimator-discrete:
 *   zeta = (1/V) sum_j w_j sum_terms C prod_i a^{b_i}_{s_i}(y_j),
 *   a^b_s(y_j) = (1/v_b) sum_k w_k Y*_s(y_k - y_j) Theta^b(|y_k - y_j|).
 * brute = 1: the naive sum over all N-tuplets, eq. NPCF-estimator-intro-discrete,
 *   with B = P^{0*}_Lambda prod Theta^{b_i}/v_{b_i} (eq. B-hypersph; the
 *   coefficient is the projection on the conjugate basis, eq. zeta-basis-coeff).
 * Primaries are j in [pb, pe); secondaries are all particles.
 * out: 2*nkeys doubles (re, im), overwritten.
 */
int npcf_oracle_estimate_ex(int D, int N, int lmax, int nbins, int bin_lt, const double *edges,
                            const double *box, int periodic, const double *pos, const double *w, int64_t n,
                            int64_t pb, int64_t pe, int brute, int remove_self, double *out);

int npcf_oracle_estimate(int D, int N, int lmax, int nbins, int bin_lt, const double *edges,
                         const double *box, int periodic, const double *pos, const double *w, int64_t n,
                         int64_t pb, int64_t pe, int brute, double *out)
{
    return npcf_oracle_estimate_ex(D, N, lmax, nbins, bin_lt, edges, box, periodic, pos, w, n, pb, pe, brute, 0, out);
}

/*
 * remove_self = 1 excludes the tuples whose secondaries coincide (reading R2 keeps them by
 * default, as the naive sum of eq. NPCF-estimator-intro-discrete does).  Only N=3 keys with
 * b1 = b2 have such tuples (N=4, 5 keys have strictly ordered bins):
 * the separable form subtracts, per primary, sum_{k in b} w_k^2 sum_terms C Y*_s1 Y*_s2 / v_b^2;
 * the naive form skips k = k'.
 */
static int estimate_core(const geom_t *g, int N, int lmax, int bin_lt, const double *pos, const double *w,
                         int64_t n, int64_t pb, int64_t pe, int brute, int remove_self, const double *vb, double V,
                         double *out);

int npcf_oracle_estimate_ex(int D, int N, int lmax, int nbins, int bin_lt, const double *edges,
                            const double *box, int periodic, const double *pos, const double *w, int64_t n,
                            int64_t pb, int64_t pe, int brute, int remove_self, double *out)
{
    if (!supported(D, N, lmax, nbins)) return -1;
    if (pb < 0 || pe > n || pb > pe) return -2;
    for (int b = 0; b < nbins; ++b)
        if (!(edges[b + 1] > edges[b]) || edges[b] < 0.0) return -3;
    double vb[OR_MAXB];
    for (int b = 0; b < nbins; ++b)
        vb[b] = sphere_area(D) / D * (pow(edges[b + 1], (double)D) - pow(edges[b], (double)D));
    double V = 1.0;
    for (int a = 0; a < D; ++a) V *= box[a];
    geom_t g = {0, D, D, nbins, edges, box, periodic, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    return estimate_core(&g, N, lmax, bin_lt, pos, w, n, pb, pe, brute, remove_self, vb, V, out);
}

/*
 * The isotropic NPCF of points on the unit 2-sphere (Sec. "Cosmic Microwave
 * Background"): the D = 2 basis about every primary, radial bins in cos theta
 * (reading R17),
 *   zeta = (1/4pi) sum_j w_j sum_[l] C prod_i a^{b_i}_{l^i}(n_j),
 *   a^b_l(n_j) = (1/v_b) sum_k w_k Y*_l(phi_jk) Theta^b(cos theta_jk),
 * v_b = 2 pi (c_{b+1} - c_b) the area of the annulus, C the D = 2 coupling.
 * pos: n x 3 directions (normalised here); cos_edges: nbins+1 ascending values
 * with -1 < c_0 (the azimuth of an antipodal point is undefined) and c_nb <= 1.
 */
int npcf_oracle_sphere_estimate(int N, int lmax, int nbins, int bin_lt, const double *cos_edges,
                                const double *pos, const double *w, int64_t n, int64_t pb, int64_t pe,
                                int brute, double *out)
{
    if (N > 4 || !supported(2, N, lmax, nbins)) return -1;
    if (pb < 0 || pe > n || pb > pe) return -2;
    if (!(cos_edges[0] > -1.0) || cos_edges[nbins] > 1.0) return -3;
    for (int b = 0; b < nbins; ++b)
        if (!(cos_edges[b + 1] > cos_edges[b])) return -3;
    double *u = (double *)malloc(sizeof(double) * 3 * (n > 0 ? n : 1));
    for (int64_t k = 0; k < n; ++k) {
        double r = sqrt((pos[3 * k] * pos[3 * k] + pos[3 * k + 1] * pos[3 * k + 1]) + pos[3 * k + 2] * pos[3 * k + 2]);
        if (!(r > 0.0)) {
            free(u);
            return -4;
        }
        for (int a = 0; a < 3; ++a) u[3 * k + a] = pos[3 * k + a] / r;
    }
    double vb[OR_MAXB];
    for (int b = 0; b < nbins; ++b) vb[b] = 2.0 * M_PI * (cos_edges[b + 1] - cos_edges[b]);
    geom_t g = {1, 3, 2, nbins, cos_edges, NULL, 0, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}};
    int rc = estimate_core(&g, N, lmax, bin_lt, u, w, n, pb, pe, brute, 0, vb, 4.0 * M_PI, out);
    free(u);
    return rc;
}

static int estimate_core(const geom_t *g, int N, int lmax, int bin_lt, const double *pos, const double *w,
                         int64_t n, int64_t pb, int64_t pe, int brute, int remove_self, const double *vb, double V,
                         double *out)
{
    const int D = g->Dh, Dp = g->Dp, nbins = g->nbins;
    geom_t gg = *g;
    int ns = enum_states(D, lmax, NULL);
    state_t *st = (state_t *)malloc(sizeof(state_t) * ns);
    enum_states(D, lmax, st);

    int nl = enum_lambdas(D, N, lmax, NULL);
    lam_t *lam = (lam_t *)malloc(sizeof(lam_t) * nl);
    enum_lambdas(D, N, lmax, lam);
    int *tstart = (int *)malloc(sizeof(int) * (nl + 1));
    tstart[0] = 0;
    for (int i = 0; i < nl; ++i) tstart[i + 1] = tstart[i] + lambda_terms(D, N, lmax, &lam[i], NULL);
    term_t *terms = (term_t *)malloc(sizeof(term_t) * (tstart[nl] > 0 ? tstart[nl] : 1));
    for (int i = 0; i < nl; ++i) lambda_terms(D, N, lmax, &lam[i], terms + tstart[i]);

    int nk = enum_keys(D, N, lmax, nbins, bin_lt, NULL);
    okey_t *keys = (okey_t *)malloc(sizeof(okey_t) * nk);
    enum_keys(D, N, lmax, nbins, bin_lt, keys);
    int *klam = (int *)malloc(sizeof(int) * nk);
    for (int i = 0; i < nk; ++i) klam[i] = key_lambda(&keys[i], lam, nl);

    cplx *zeta = (cplx *)calloc(nk, sizeof(cplx));
    cplx *a = (cplx *)malloc(sizeof(cplx) * nbins * ns);
    cplx *self = (cplx *)malloc(sizeof(cplx) * nbins * (nl > 0 ? nl : 1)); /* N=3 coincident terms */
    /* neighbour lists for the naive sum */
    int64_t *nb_idx = NULL;
    int *nb_bin = NULL;
    cplx *nb_y = NULL;
    if (brute) {
        nb_idx = (int64_t *)malloc(sizeof(int64_t) * n);
        nb_bin = (int *)malloc(sizeof(int) * n);
        nb_y = (cplx *)malloc(sizeof(cplx) * n * ns);
    }

    double d[OR_MAXD];
    for (int64_t j = pb; j < pe; ++j) {
        const double *yj = pos + j * Dp;
        geom_primary(&gg, yj);
        if (!brute) {
            for (int i = 0; i < nbins * ns; ++i) a[i] = 0.0;
            for (int i = 0; i < nbins * nl; ++i) self[i] = 0.0;
            for (int64_t k = 0; k < n; ++k) {
                if (k == j) continue;
                int b = geom_pair(&gg, pos + k * Dp, yj, d);
                if (b < 0) continue;
                for (int s = 0; s < ns; ++s) a[b * ns + s] += w[k] * conj(harmonic(D, &st[s], d));
                if (remove_self && N == 3)
                    for (int il = 0; il < nl; ++il) {
                        cplx t = 0.0;
                        for (int q = tstart[il]; q < tstart[il + 1]; ++q)
                            t += terms[q].c * conj(harmonic(D, &st[terms[q].s[0]], d)) *
                                 conj(harmonic(D, &st[terms[q].s[1]], d));
                        self[b * nl + il] += w[k] * w[k] * t;
                    }
            }
            for (int b = 0; b < nbins; ++b)
                for (int s = 0; s < ns; ++s) a[b * ns + s] /= vb[b];
            for (int i = 0; i < nk; ++i) {
                const okey_t *kk = &keys[i];
                cplx acc = 0.0;
                for (int t = tstart[klam[i]]; t < tstart[klam[i] + 1]; ++t) {
                    cplx p = terms[t].c * a[kk->b[0] * ns + terms[t].s[0]] * a[kk->b[1] * ns + terms[t].s[1]];
                    if (N >= 4) p *= a[kk->b[2] * ns + terms[t].s[2]];
                    if (N == 5) p *= a[kk->b[3] * ns + terms[t].s[3]];
                    acc += p;
                }
                if (remove_self && N == 3 && kk->b[0] == kk->b[1])
                    acc -= self[kk->b[0] * nl + klam[i]] / (vb[kk->b[0]] * vb[kk->b[0]]);
                zeta[i] += w[j] * acc;
            }
        } else {
            int64_t nn = 0;
            for (int64_t k = 0; k < n; ++k) {
                if (k == j) continue;
                int b = geom_pair(&gg, pos + k * Dp, yj, d);
                if (b < 0) continue;
                nb_idx[nn] = k;
                nb_bin[nn] = b;
                for (int s = 0; s < ns; ++s) nb_y[nn * ns + s] = harmonic(D, &st[s], d);
                ++nn;
            }
            for (int i = 0; i < nk; ++i) {
                const okey_t *kk = &keys[i];
                cplx acc = 0.0;
                for (int64_t p1 = 0; p1 < nn; ++p1) {
                    if (nb_bin[p1] != kk->b[0]) continue;
                    for (int64_t p2 = 0; p2 < nn; ++p2) {
                        if (nb_bin[p2] != kk->b[1]) continue;
                        if (remove_self && p2 == p1) continue;
                        if (N == 3) {
                            cplx P = 0.0;
                            for (int t = tstart[klam[i]]; t < tstart[klam[i] + 1]; ++t)
                                P += terms[t].c * nb_y[p1 * ns + terms[t].s[0]] * nb_y[p2 * ns + terms[t].s[1]];
                            double wt = w[nb_idx[p1]] * w[nb_idx[p2]] / (vb[kk->b[0]] * vb[kk->b[1]]);
                            acc += wt * conj(P);
                        } else if (N == 4) {
                            for (int64_t p3 = 0; p3 < nn; ++p3) {
                                if (nb_bin[p3] != kk->b[2]) continue;
                                cplx P = 0.0;
                                for (int t = tstart[klam[i]]; t < tstart[klam[i] + 1]; ++t)
                                    P += terms[t].c * nb_y[p1 * ns + terms[t].s[0]] * nb_y[p2 * ns + terms[t].s[1]] *
                                         nb_y[p3 * ns + terms[t].s[2]];
                                double wt = w[nb_idx[p1]] * w[nb_idx[p2]] * w[nb_idx[p3]] /
                                            (vb[kk->b[0]] * vb[kk->b[1]] * vb[kk->b[2]]);
                                acc += wt * conj(P);
                            }
                        } else {
                            for (int64_t p3 = 0; p3 < nn; ++p3) {
                                if (nb_bin[p3] != kk->b[2]) continue;
                                for (int64_t p4 = 0; p4 < nn; ++p4) {
                                    if (nb_bin[p4] != kk->b[3]) continue;
                                    cplx P = 0.0;
                                    for (int t = tstart[klam[i]]; t < tstart[klam[i] + 1]; ++t)
                                        P += terms[t].c * nb_y[p1 * ns + terms[t].s[0]] * nb_y[p2 * ns + terms[t].s[1]] *
                                             nb_y[p3 * ns + terms[t].s[2]] * nb_y[p4 * ns + terms[t].s[3]];
                                    double wt = w[nb_idx[p1]] * w[nb_idx[p2]] * w[nb_idx[p3]] * w[nb_idx[p4]] /
                                                (vb[kk->b[0]] * vb[kk->b[1]] * vb[kk->b[2]] * vb[kk->b[3]]);
                                    acc += wt * conj(P);
                                }
                            }
                        }
                    }
                }
                zeta[i] += w[j] * acc;
            }
        }
    }
    for (int i = 0; i < nk; ++i) {
        out[2 * i] = creal(zeta[i]) / V;
        out[2 * i + 1] = cimag(zeta[i]) / V;
    }
    free(zeta); free(a); free(self); free(keys); free(klam); free(terms); free(tstart); free(lam); free(st);
    free(nb_idx); free(nb_bin); free(nb_y);
    return nk;
}

/* ------------------------------------------------------------------ */
/* N = 3 through the addition theorem.                                 */
/*
 * For N=3 the isotropic basis function is, by eq. zero-ang-mom-states with
 * the zero coupling of reading R6 (which for D=3 is the CG of eq. CG-examples,
 * (-1)^(l-m)/sqrt(2l+1)), proportional to the sum over the intermediate
 * labels of Y_l(r1) Y*_l(r2).  The addition theorem for hyperspherical
 * harmonics turns that sum into a Gegenbauer polynomial of r1.r2:
 *     sum_[l] Y_l(r1) Y*_l(r2) = dim_l/|S^{D-1}| C^{(lam)}_l(t)/C^{(lam)}_l(1),
 * lam = D/2 - 1, t = r1.r2, dim_l from the state count quoted after
 * eq. single-particle-eigenfun.  Hence (D >= 3)
 *   zeta_l(b1,b2) = (1/V) sum_j w_j sum_{k in b1, k' in b2} w_k w_k'
 *                   (-1)^l sqrt(dim_l)/|S^{D-1}| G_l(t_jkk') / (v_b1 v_b2),
 * with G_l = C_l/C_l(1).  This route uses no harmonic and no coupling table,
 * so it pins the separable estimator of N=3; its derivative in positions and
 * weights (bins held fixed) is the gradient oracle for the adjoint.
 * For D=2 the basis is e^{il theta}/sqrt(2 pi) and the product of one
 * secondary's conjugate with the other's is a plain exponential of the angle
 * between them: a_l(b1) conj a_l(b2) sums w_k w_k' e^{-il phi}/(2 pi v_b1 v_b2),
 * phi = theta_k - theta_k' = atan2(u_k x u_k', u_k . u_k') up to sign, so
 *   zeta_l(b1,b2) = (1/V) sum_j w_j sum w_k w_k' (cos l phi - i sin l phi)/(2 pi v_b1 v_b2).
 */

/* C^{(lam)}_n(x) by its explicit sum (DLMF 18.5.10) and its derivative */
static double gegenbauer(int n, double lam, double x, double *deriv)
{
    double s = 0.0, ds = 0.0;
    for (int k = 0; 2 * k <= n; ++k) {
        int p = n - 2 * k;
        /* (lam)_{n-k} / (k! (n-2k)!) * 2^p */
        double poch = 1.0;
        for (int i = 0; i < n - k; ++i) poch *= (lam + i);
        double c = sgn_pow(k) * poch / (fact(k) * fact(p)) * pow(2.0, (double)p);
        s += c * pow(x, (double)p);
        if (p > 0) ds += c * p * pow(x, (double)(p - 1));
    }
    if (deriv) *deriv = ds;
    return s;
}

static double gegenbauer_at_one(int n, double lam)
{
    /* C^{(lam)}_n(1) = (2 lam)_n / n! */
    double poch = 1.0;
    for (int i = 0; i < n; ++i) poch *= (2.0 * lam + i);
    return poch / fact(n);
}

static double dim_l(int D, int l)
{
    if (D == 2) return 1.0;
    return binom(l + D - 3, D - 3) * (2.0 * l + D - 2) / (double)(D - 2);
}

/*
 * zeta (2*nkeys) for N=3, D in {2,3,4} (imaginary parts zero for D >= 3); if
 * grad_coeffs is non-NULL also the gradient of
 *     L = sum_c grad_coeffs[2c] Re zeta_c + grad_coeffs[2c+1] Im zeta_c
 * with respect to every position (grad_pos, n x D) and weight (grad_w, n).
 */
int npcf_oracle_n3_closed(int D, int lmax, int nbins, int bin_lt, const double *edges, const double *box,
                          int periodic, const double *pos, const double *w, int64_t n, int64_t pb, int64_t pe,
                          const double *grad_coeffs, double *out, double *grad_pos, double *grad_w)
{
    if (D < 2 || D > 4 || !supported(D, 3, lmax, nbins)) return -1;
    if (pb < 0 || pe > n || pb > pe) return -2;
    int nk = enum_keys(D, 3, lmax, nbins, bin_lt, NULL);
    /* key index of (b1, b2, l) in enum_keys order */
    int *kidx = (int *)malloc(sizeof(int) * nbins * nbins);
    {
        int c = 0;
        for (int b1 = 0; b1 < nbins; ++b1)
            for (int b2 = 0; b2 < nbins; ++b2) kidx[b1 * nbins + b2] = -1;
        for (int b1 = 0; b1 < nbins; ++b1)
            for (int b2 = b1 + (bin_lt ? 1 : 0); b2 < nbins; ++b2) {
                kidx[b1 * nbins + b2] = c;
                c += lmax + 1;
            }
    }
    double vb[OR_MAXB];
    for (int b = 0; b < nbins; ++b)
        vb[b] = sphere_area(D) / D * (pow(edges[b + 1], (double)D) - pow(edges[b], (double)D));
    double V = 1.0;
    for (int a = 0; a < D; ++a) V *= box[a];
    double lam = 0.5 * D - 1.0;
    double S = sphere_area(D);
    double pref[OR_MAXL + 1];
    for (int l = 0; l <= lmax; ++l) pref[l] = sgn_pow(l) * sqrt(dim_l(D, l)) / S / gegenbauer_at_one(l, lam);

    double *zeta = (double *)calloc(2 * (size_t)nk, sizeof(double));
    int64_t *nb_idx = (int64_t *)malloc(sizeof(int64_t) * n);
    int *nb_bin = (int *)malloc(sizeof(int) * n);
    double *nb_u = (double *)malloc(sizeof(double) * n * D);  /* unit vectors */
    double *nb_r = (double *)malloc(sizeof(double) * n);
    if (grad_pos) memset(grad_pos, 0, sizeof(double) * n * D);
    if (grad_w) memset(grad_w, 0, sizeof(double) * n);

    double d[OR_MAXD];
    for (int64_t j = pb; j < pe; ++j) {
        int64_t nn = 0;
        for (int64_t k = 0; k < n; ++k) {
            if (k == j) continue;
            separation(D, pos + k * D, pos + j * D, box, periodic, d);
            double r2 = norm2(D, d);
            int b = bin_of(r2, nbins, edges);
            if (b < 0) continue;
            double r = sqrt(r2);
            nb_idx[nn] = k;
            nb_bin[nn] = b;
            nb_r[nn] = r;
            for (int a = 0; a < D; ++a) nb_u[nn * D + a] = d[a] / r;
            ++nn;
        }
        for (int64_t p = 0; p < nn; ++p)
            for (int64_t q = 0; q < nn; ++q) {
                int b1 = nb_bin[p], b2 = nb_bin[q];
                int kb = kidx[b1 * nbins + b2];
                if (kb < 0) continue; /* the key stores (b1 <= b2) ordered pairs only */
                double t = 0.0;
                for (int a = 0; a < D; ++a) t += nb_u[p * D + a] * nb_u[q * D + a];
                double wp = w[nb_idx[p]], wq = w[nb_idx[q]];
                double scale = 1.0 / (vb[b1] * vb[b2] * V);
                double dLdt = 0.0, L_no_w = 0.0;
                double phi = 0.0, dLdphi = 0.0;
                if (D == 2)
                    phi = atan2(nb_u[p * 2 + 1] * nb_u[q * 2] - nb_u[p * 2] * nb_u[q * 2 + 1], t); /* theta_p - theta_q */
                for (int l = 0; l <= lmax; ++l) {
                    if (D == 2) {
                        double re = cos(l * phi) / (2.0 * M_PI), im = -sin(l * phi) / (2.0 * M_PI);
                        zeta[2 * (kb + l)] += w[j] * wp * wq * re * scale;
                        zeta[2 * (kb + l) + 1] += w[j] * wp * wq * im * scale;
                        if (grad_coeffs) {
                            double Gr = grad_coeffs[2 * (kb + l)], Gi = grad_coeffs[2 * (kb + l) + 1];
                            L_no_w += Gr * re + Gi * im;
                            /* d re/d phi = l im, d im/d phi = -l re */
                            dLdphi += Gr * l * im - Gi * l * re;
                        }
                        continue;
                    }
                    double dg;
                    double g = pref[l] * gegenbauer(l, lam, t, &dg);
                    dg *= pref[l];
                    zeta[2 * (kb + l)] += w[j] * wp * wq * g * scale;
                    if (grad_coeffs) {
                        double G = grad_coeffs[2 * (kb + l)];
                        dLdt += G * dg;
                        L_no_w += G * g;
                    }
                }
                if (!grad_coeffs) continue;
                if (grad_w) {
                    grad_w[j] += wp * wq * L_no_w * scale;
                    grad_w[nb_idx[p]] += w[j] * wq * L_no_w * scale;
                    grad_w[nb_idx[q]] += w[j] * wp * L_no_w * scale;
                }
                if (grad_pos && D == 2) {
                    /* d theta/d d = (-u_y, u_x)/r for d = r (u_x, u_y) */
                    double f = w[j] * wp * wq * scale * dLdphi;
                    double gp[2], gq[2];
                    gp[0] = -f * nb_u[p * 2 + 1] / nb_r[p];
                    gp[1] = f * nb_u[p * 2] / nb_r[p];
                    gq[0] = f * nb_u[q * 2 + 1] / nb_r[q];
                    gq[1] = -f * nb_u[q * 2] / nb_r[q];
                    for (int a = 0; a < 2; ++a) {
                        grad_pos[nb_idx[p] * 2 + a] += gp[a];
                        grad_pos[nb_idx[q] * 2 + a] += gq[a];
                        grad_pos[j * 2 + a] -= gp[a] + gq[a];
                    }
                } else if (grad_pos) {
                    double f = w[j] * wp * wq * scale * dLdt;
                    for (int a = 0; a < D; ++a) {
                        /* dt/dd_p = (u_q - t u_p)/|d_p|, d_p = y_p - y_j */
                        double gp = f * (nb_u[q * D + a] - t * nb_u[p * D + a]) / nb_r[p];
                        double gq = f * (nb_u[p * D + a] - t * nb_u[q * D + a]) / nb_r[q];
                        grad_pos[nb_idx[p] * D + a] += gp;
                        grad_pos[nb_idx[q] * D + a] += gq;
                        grad_pos[j * D + a] -= gp + gq;
                    }
                }
            }
    }
    for (int i = 0; i < 2 * nk; ++i) out[i] = zeta[i];
    free(zeta); free(kidx); free(nb_idx); free(nb_bin); free(nb_u); free(nb_r);
    return nk;
}

/* ------------------------------------------------------------------ */
/* Gridded data (Sec. "Application to Gridded Data").                   */
/*
 * The field X is given at the nodes of a periodic grid with dims[a] nodes
 * along axis a of a box of sides box[a] (spacing h_a = box[a]/dims[a], node
 * volume dV = prod_a h_a; row-major storage, last axis fastest).  The
 * integrals of eq. alm-bin-def and eq. NPCF-mult-estimator become sums over
 * nodes times dV (reading R16):
 *   a^b_l(s) = (1/v_b) sum_{o != 0} dV X(s + o h) Y*_l(unit(o h)) Theta^b(|o h|),
 *   zeta     = (1/V_D) sum_s dV X(s) sum_[l] C prod_i a^{b_i}_{l^i}(s),
 * o running over integer offset vectors, node indices taken modulo dims, v_b
 * the shell volume of R4, the offset o = 0 skipped as R1 skips r = 0.  This
 * direct sum over offsets is the plain definition; the FFT form of the paper
 * evaluates the same circular convolution.  Every offset within r_max must
 * reach a distinct node: 2 floor(r_max/h_a) < dims[a].
 */
typedef struct {
    int64_t o[OR_MAXD];
    int b;
} goff_t;

/* offsets within the bins and the conjugate harmonics there; returns the count or < 0 */
static int64_t grid_offsets(int D, int lmax, int nbins, const double *edges, const double *box,
                            const int *dims, goff_t **offs_out, cplx **yc_out)
{
    double h[OR_MAXD];
    int64_t K[OR_MAXD], span = 1;
    double rmax = edges[nbins];
    for (int a = 0; a < D; ++a) {
        if (dims[a] < 1 || !(box[a] > 0.0)) return -1;
        h[a] = box[a] / dims[a];
        K[a] = (int64_t)floor(rmax / h[a]);
        if (2 * K[a] >= dims[a]) return -2;
        span *= 2 * K[a] + 1;
    }
    int ns = enum_states(D, lmax, NULL);
    state_t *st = (state_t *)malloc(sizeof(state_t) * ns);
    enum_states(D, lmax, st);
    goff_t *offs = (goff_t *)malloc(sizeof(goff_t) * span);
    cplx *yc = (cplx *)malloc(sizeof(cplx) * span * ns);
    int64_t nof = 0;
    double d[OR_MAXD];
    for (int64_t t = 0; t < span; ++t) {
        int64_t rem = t;
        goff_t g;
        for (int a = D - 1; a >= 0; --a) {
            g.o[a] = rem % (2 * K[a] + 1) - K[a];
            rem /= 2 * K[a] + 1;
            d[a] = (double)g.o[a] * h[a];
        }
        double r2 = norm2(D, d);
        if (r2 == 0.0) continue;
        g.b = bin_of(r2, nbins, edges);
        if (g.b < 0) continue;
        offs[nof] = g;
        for (int s = 0; s < ns; ++s) yc[nof * ns + s] = conj(harmonic(D, &st[s], d));
        ++nof;
    }
    free(st);
    *offs_out = offs;
    *yc_out = yc;
    return nof;
}

/* a^b_l at every node: out is ncell x nbins x nstates complex (re, im interleaved) */
static int grid_alm(int D, int lmax, int nbins, const double *edges, const double *box, const int *dims,
                    const double *X, cplx *a)
{
    goff_t *offs;
    cplx *yc;
    int64_t nof = grid_offsets(D, lmax, nbins, edges, box, dims, &offs, &yc);
    if (nof < 0) return (int)nof;
    int ns = enum_states(D, lmax, NULL);
    int64_t ncell = 1;
    double dV = 1.0;
    for (int a = 0; a < D; ++a) {
        ncell *= dims[a];
        dV *= box[a] / dims[a];
    }
    double vb[OR_MAXB];
    for (int b = 0; b < nbins; ++b)
        vb[b] = sphere_area(D) / D * (pow(edges[b + 1], (double)D) - pow(edges[b], (double)D));
    int64_t c[OR_MAXD];
    for (int64_t cell = 0; cell < ncell; ++cell) {
        int64_t rem = cell;
        for (int a = D - 1; a >= 0; --a) {
            c[a] = rem % dims[a];
            rem /= dims[a];
        }
        cplx *ac = a + cell * nbins * ns;
        for (int i = 0; i < nbins * ns; ++i) ac[i] = 0.0;
        for (int64_t q = 0; q < nof; ++q) {
            int64_t idx = 0;
            for (int a = 0; a < D; ++a) {
                int64_t x = (c[a] + offs[q].o[a]) % dims[a];
                if (x < 0) x += dims[a];
                idx = idx * dims[a] + x;
            }
            double f = dV * X[idx];
            for (int s = 0; s < ns; ++s) ac[offs[q].b * ns + s] += f * yc[q * ns + s];
        }
        for (int b = 0; b < nbins; ++b)
            for (int s = 0; s < ns; ++s) ac[b * ns + s] /= vb[b];
    }
    free(offs);
    free(yc);
    return 0;
}

int npcf_oracle_grid_alm(int D, int lmax, int nbins, const double *edges, const double *box, const int *dims,
                         const double *X, double *out)
{
    if (D < 2 || D > 4 || !supported(D, 3, lmax, nbins)) return -1;
    for (int b = 0; b < nbins; ++b)
        if (!(edges[b + 1] > edges[b]) || edges[b] < 0.0) return -3;
    return grid_alm(D, lmax, nbins, edges, box, dims, X, (cplx *)out);
}

int npcf_oracle_grid_estimate(int D, int N, int lmax, int nbins, int bin_lt, const double *edges,
                              const double *box, const int *dims, const double *X, double *out)
{
    if (!supported(D, N, lmax, nbins)) return -1;
    for (int b = 0; b < nbins; ++b)
        if (!(edges[b + 1] > edges[b]) || edges[b] < 0.0) return -3;
    int ns = enum_states(D, lmax, NULL);
    int64_t ncell = 1;
    double dV = 1.0, V = 1.0;
    for (int a = 0; a < D; ++a) {
        if (dims[a] < 1) return -2;
        ncell *= dims[a];
        dV *= box[a] / dims[a];
        V *= box[a];
    }
    cplx *a = (cplx *)malloc(sizeof(cplx) * ncell * nbins * ns);
    int rc = grid_alm(D, lmax, nbins, edges, box, dims, X, a);
    if (rc < 0) {
        free(a);
        return rc - 10;
    }
    int nl = enum_lambdas(D, N, lmax, NULL);
    lam_t *lam = (lam_t *)malloc(sizeof(lam_t) * nl);
    enum_lambdas(D, N, lmax, lam);
    int *tstart = (int *)malloc(sizeof(int) * (nl + 1));
    tstart[0] = 0;
    for (int i = 0; i < nl; ++i) tstart[i + 1] = tstart[i] + lambda_terms(D, N, lmax, &lam[i], NULL);
    term_t *terms = (term_t *)malloc(sizeof(term_t) * (tstart[nl] > 0 ? tstart[nl] : 1));
    for (int i = 0; i < nl; ++i) lambda_terms(D, N, lmax, &lam[i], terms + tstart[i]);
    int nk = enum_keys(D, N, lmax, nbins, bin_lt, NULL);
    okey_t *keys = (okey_t *)malloc(sizeof(okey_t) * nk);
    enum_keys(D, N, lmax, nbins, bin_lt, keys);
    int *klam = (int *)malloc(sizeof(int) * nk);
    for (int i = 0; i < nk; ++i) klam[i] = key_lambda(&keys[i], lam, nl);

    cplx *zeta = (cplx *)calloc(nk, sizeof(cplx));
    for (int64_t cell = 0; cell < ncell; ++cell) {
        const cplx *ac = a + cell * nbins * ns;
        for (int i = 0; i < nk; ++i) {
            const okey_t *kk = &keys[i];
            cplx acc = 0.0;
            for (int t = tstart[klam[i]]; t < tstart[klam[i] + 1]; ++t) {
                cplx p = terms[t].c * ac[kk->b[0] * ns + terms[t].s[0]] * ac[kk->b[1] * ns + terms[t].s[1]];
                if (N >= 4) p *= ac[kk->b[2] * ns + terms[t].s[2]];
                if (N == 5) p *= ac[kk->b[3] * ns + terms[t].s[3]];
                acc += p;
            }
            zeta[i] += dV * X[cell] * acc;
        }
    }
    for (int i = 0; i < nk; ++i) {
        out[2 * i] = creal(zeta[i]) / V;
        out[2 * i + 1] = cimag(zeta[i]) / V;
    }
    free(a); free(zeta); free(keys); free(klam); free(terms); free(tstart); free(lam);
    return nk;
}

/* ------------------------------------------------------------------ */
/* Anisotropic basis about a fixed line of sight (Sec. "Large-Scale     */
/* Structure"): D = 3, invariance under rotations about x_3 keeps the   */
/* states of combined angular momentum (L_1, L_2) = (0, L) (reading R18) */
/*
 * Labels:  N=3: (l1, l2, L), l1, l2 <= lmax, |l1 - l2| <= L <= l1 + l2;
 *          N=4: (l1, l2, l12, l3, L), l1, l2, l3 <= lmax, l12 and L by the
 *               triangle rules of eq. addition-triangle-conditions.
 * Coupling: N=3 as printed for the redshift-space 3PCF,
 *               C = (-1)^{l2-l1} sqrt(2L+1) (l1 l2 L; m -m 0),
 *           which is the CG <l1 m l2 -m|L 0>; N=4 by eq. Coupling-C with the
 *           final state (L, 0): <l1 m1 l2 m2|l12 m12><l12 m12 l3 m3|L 0>.
 * Bins as the isotropic keys: b1 <= b2 (or <) for N=3, b1 < b2 < b3 for N=4.
 */
typedef struct { int b[3]; int l[5]; } akey_t;

static int enum_aniso_keys(int N, int lmax, int nbins, int bin_lt, akey_t *out)
{
    int c = 0;
    if (N == 3) {
        for (int b1 = 0; b1 < nbins; ++b1)
            for (int b2 = b1 + (bin_lt ? 1 : 0); b2 < nbins; ++b2)
                for (int l1 = 0; l1 <= lmax; ++l1)
                    for (int l2 = 0; l2 <= lmax; ++l2)
                        for (int L = abs(l1 - l2); L <= l1 + l2; ++L) {
                            if (out) {
                                akey_t k = {{b1, b2, -1}, {l1, l2, L, 0, 0}};
                                out[c] = k;
                            }
                            ++c;
                        }
    } else {
        for (int b1 = 0; b1 < nbins; ++b1)
            for (int b2 = b1 + 1; b2 < nbins; ++b2)
                for (int b3 = b2 + 1; b3 < nbins; ++b3)
                    for (int l1 = 0; l1 <= lmax; ++l1)
                        for (int l2 = 0; l2 <= lmax; ++l2)
                            for (int l12 = abs(l1 - l2); l12 <= l1 + l2; ++l12)
                                for (int l3 = 0; l3 <= lmax; ++l3)
                                    for (int L = abs(l12 - l3); L <= l12 + l3; ++L) {
                                        if (out) {
                                            akey_t k = {{b1, b2, b3}, {l1, l2, l12, l3, L}};
                                            out[c] = k;
                                        }
                                        ++c;
                                    }
    }
    return c;
}

static int d3_state(int l, int m) { return l * l + l + m; }

/* the non-zero terms (state indices s[0..N-2], C) of one anisotropic label set */
static int aniso_terms(int N, const akey_t *k, term_t *out)
{
    int c = 0;
    if (N == 3) {
        int l1 = k->l[0], l2 = k->l[1], L = k->l[2];
        for (int m = -l1; m <= l1; ++m) {
            if (abs(m) > l2) continue;
            double v = sgn_pow(abs(l2 - l1)) * sqrt(2.0 * L + 1.0) * wigner3j(l1, l2, L, m, -m, 0);
            if (v == 0.0) continue;
            if (out) {
                term_t t = {{d3_state(l1, m), d3_state(l2, -m), 0, 0}, v};
                out[c] = t;
            }
            ++c;
        }
    } else {
        int l1 = k->l[0], l2 = k->l[1], l12 = k->l[2], l3 = k->l[3], L = k->l[4];
        for (int m1 = -l1; m1 <= l1; ++m1)
            for (int m2 = -l2; m2 <= l2; ++m2) {
                int m12 = m1 + m2, m3 = -m12;
                if (abs(m12) > l12 || abs(m3) > l3) continue;
                double v = cg_d3(l1, m1, l2, m2, l12, m12) * cg_d3(l12, m12, l3, m3, L, 0);
                if (v == 0.0) continue;
                if (out) {
                    term_t t = {{d3_state(l1, m1), d3_state(l2, m2), d3_state(l3, m3), 0}, v};
                    out[c] = t;
                }
                ++c;
            }
    }
    return c;
}

int npcf_oracle_aniso_nkeys(int N, int lmax, int nbins, int bin_lt)
{
    if ((N != 3 && N != 4) || lmax < 0 || lmax > OR_MAXL || nbins < 1 || nbins > OR_MAXB) return -1;
    return enum_aniso_keys(N, lmax, nbins, bin_lt, NULL);
}

/* keys: nkeys x 8 ints (b1, b2, b3, l1, l2, l3, l4, l5) with the labels of the akey_t layout */
int npcf_oracle_aniso_keys(int N, int lmax, int nbins, int bin_lt, int *keys)
{
    int nk = npcf_oracle_aniso_nkeys(N, lmax, nbins, bin_lt);
    if (nk < 0) return nk;
    akey_t *k = (akey_t *)malloc(sizeof(akey_t) * (nk > 0 ? nk : 1));
    enum_aniso_keys(N, lmax, nbins, bin_lt, k);
    for (int i = 0; i < nk; ++i) {
        for (int a = 0; a < 3; ++a) keys[8 * i + a] = k[i].b[a];
        for (int a = 0; a < 5; ++a) keys[8 * i + 3 + a] = k[i].l[a];
    }
    free(k);
    return nk;
}

/*
 * zeta^{0L}_Lambda(b) = (1/V) sum_j w_j sum_terms C prod_i a^{b_i}_{l^i m^i}(y_j),
 * a from eq. NPCF-estimator-discrete (Y*, 1/v_b); brute = 1 sums the basis over
 * every tuple of secondaries instead (eq. NPCF-intro-discrete with eq. B-hypersph).
 */
int npcf_oracle_aniso_estimate(int N, int lmax, int nbins, int bin_lt, const double *edges, const double *box,
                               int periodic, const double *pos, const double *w, int64_t n, int64_t pb, int64_t pe,
                               int brute, double *out)
{
    const int D = 3;
    int nk = npcf_oracle_aniso_nkeys(N, lmax, nbins, bin_lt);
    if (nk < 0) return -1;
    if (pb < 0 || pe > n || pb > pe) return -2;
    for (int b = 0; b < nbins; ++b)
        if (!(edges[b + 1] > edges[b]) || edges[b] < 0.0) return -3;
    int ns = enum_states(D, lmax, NULL);
    state_t *st = (state_t *)malloc(sizeof(state_t) * ns);
    enum_states(D, lmax, st);
    akey_t *keys = (akey_t *)malloc(sizeof(akey_t) * (nk > 0 ? nk : 1));
    enum_aniso_keys(N, lmax, nbins, bin_lt, keys);
    int *tstart = (int *)malloc(sizeof(int) * (nk + 1));
    tstart[0] = 0;
    for (int i = 0; i < nk; ++i) tstart[i + 1] = tstart[i] + aniso_terms(N, &keys[i], NULL);
    term_t *terms = (term_t *)malloc(sizeof(term_t) * (tstart[nk] > 0 ? tstart[nk] : 1));
    for (int i = 0; i < nk; ++i) aniso_terms(N, &keys[i], terms + tstart[i]);
    double vb[OR_MAXB];
    for (int b = 0; b < nbins; ++b)
        vb[b] = sphere_area(D) / D * (pow(edges[b + 1], (double)D) - pow(edges[b], (double)D));
    double V = box[0] * box[1] * box[2];

    cplx *zeta = (cplx *)calloc(nk > 0 ? nk : 1, sizeof(cplx));
    cplx *a = (cplx *)malloc(sizeof(cplx) * nbins * ns);
    int64_t *nb_idx = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    int *nb_bin = (int *)malloc(sizeof(int) * (n > 0 ? n : 1));
    cplx *nb_y = (cplx *)malloc(sizeof(cplx) * (n > 0 ? n : 1) * ns);
    double d[OR_MAXD];
    for (int64_t j = pb; j < pe; ++j) {
        const double *yj = pos + j * D;
        int64_t nn = 0;
        for (int i = 0; i < nbins * ns; ++i) a[i] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            if (k == j) continue;
            separation(D, pos + k * D, yj, box, periodic, d);
            int b = bin_of(norm2(D, d), nbins, edges);
            if (b < 0) continue;
            nb_idx[nn] = k;
            nb_bin[nn] = b;
            for (int s = 0; s < ns; ++s) {
                nb_y[nn * ns + s] = harmonic(D, &st[s], d);
                a[b * ns + s] += w[k] * conj(nb_y[nn * ns + s]);
            }
            ++nn;
        }
        for (int b = 0; b < nbins; ++b)
            for (int s = 0; s < ns; ++s) a[b * ns + s] /= vb[b];
        for (int i = 0; i < nk; ++i) {
            const akey_t *kk = &keys[i];
            cplx acc = 0.0;
            if (!brute) {
                for (int t = tstart[i]; t < tstart[i + 1]; ++t) {
                    cplx p = terms[t].c * a[kk->b[0] * ns + terms[t].s[0]] * a[kk->b[1] * ns + terms[t].s[1]];
                    if (N == 4) p *= a[kk->b[2] * ns + terms[t].s[2]];
                    acc += p;
                }
            } else {
                for (int64_t p1 = 0; p1 < nn; ++p1) {
                    if (nb_bin[p1] != kk->b[0]) continue;
                    for (int64_t p2 = 0; p2 < nn; ++p2) {
                        if (nb_bin[p2] != kk->b[1]) continue;
                        if (N == 3) {
                            cplx P = 0.0;
                            for (int t = tstart[i]; t < tstart[i + 1]; ++t)
                                P += terms[t].c * nb_y[p1 * ns + terms[t].s[0]] * nb_y[p2 * ns + terms[t].s[1]];
                            acc += w[nb_idx[p1]] * w[nb_idx[p2]] * conj(P) / (vb[kk->b[0]] * vb[kk->b[1]]);
                            continue;
                        }
                        for (int64_t p3 = 0; p3 < nn; ++p3) {
                            if (nb_bin[p3] != kk->b[2]) continue;
                            cplx P = 0.0;
                            for (int t = tstart[i]; t < tstart[i + 1]; ++t)
                                P += terms[t].c * nb_y[p1 * ns + terms[t].s[0]] * nb_y[p2 * ns + terms[t].s[1]] *
                                     nb_y[p3 * ns + terms[t].s[2]];
                            acc += w[nb_idx[p1]] * w[nb_idx[p2]] * w[nb_idx[p3]] * conj(P) /
                                   (vb[kk->b[0]] * vb[kk->b[1]] * vb[kk->b[2]]);
                        }
                    }
                }
            }
            zeta[i] += w[j] * acc;
        }
    }
    for (int i = 0; i < nk; ++i) {
        out[2 * i] = creal(zeta[i]) / V;
        out[2 * i + 1] = cimag(zeta[i]) / V;
    }
    free(zeta); free(a); free(nb_idx); free(nb_bin); free(nb_y); free(keys); free(tstart); free(terms); free(st);
    return nk;
}
