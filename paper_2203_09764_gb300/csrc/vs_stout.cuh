// vs_stout.cuh -- staple sums (plain loads, the one-pass link stream, the plaquette-staple
// stream), the stout candidate, and the colour-class update and AUS kernels.
//
// Stout step, Sec. II.A Eqs. (stout)/(generator):
//   Omega = Sigma U^dag,  Q = (Omega - Omega^dag)/2 - Tr(Omega - Omega^dag)/6,
//   U' = exp(rho Q) U.
// Staples, Eq. (plaq_staples) and the over-improved form Eq. (over-improvement):
//   Sigma = c0 sum_{nu != mu, +-} (3-link staple) + c1 sum_{nu != mu, +-} (R1 + R2 + R3)
// with the paths (steps from x, ending at x + mu; -nu versions by nu -> -nu):
//   staple  +nu +mu -nu
//   R1      +nu +nu +mu -nu -nu          (tall)
//   R2      +nu +mu +mu -nu -mu          (wide, forward)
//   R3      -mu +nu +mu +mu -nu          (wide, backward)
// Writing A = first step, B = U_mu(x + s nu), C = last step of the staple:
//   staple + R1 = (c0 A B + c1 A T) C,   T = (step +s nu)(U_mu)(step -s nu) one site up
//   R2 terms share the left factor A B and all end in U_mu^dag(x+mu)
//   R3 terms share the right factor B C and all start with U_mu^dag(x-mu)
// so the common end factors are applied once after the loop over (nu, s):
// 10 SU(3) products per (nu, s) plus 2, instead of 14 per (nu, s).
//
// Exponential: exp(rho Q) = exp(i H) with H = -i rho Q Hermitian traceless.
// Cayley-Hamilton, H^3 = tau H + delta I with tau = Tr(H^2)/2, delta = det H,
// so H^n = a_n I + b_n H + c_n H^2 with a_{n+1} = delta c_n,
// b_{n+1} = a_n + tau c_n, c_{n+1} = b_n, and
//   exp(iH) = f0 I + f1 H + f2 H^2,  f_j = sum_n i^n (a_n, b_n, c_n)_j / n!.
// The scalar series converges like |H|^n / n! with no cancellation for
// |H| <= 1 and needs no eigenvalues, so it has no degeneracy problem.
#pragma once

#include <atomic>
#include <mutex>

#include "vs_internal.h"

namespace vs {

template <class T> struct Tol;
template <> struct Tol<float> { static __device__ __forceinline__ float eps() { return 1.5e-8f; } };
template <> struct Tol<double> { static __device__ __forceinline__ double eps() { return 1e-17; } };

// The plane position is a sum of one term per coordinate,
//   i(x) = Xpos(x0) + Lxp x1 + Lxp Ly x2 + Lxp Ly Lz x3,  Xpos(x0) = (x0 & 3) Qp + x0/4,
// so the position of x + a e_nu + b e_mu is i(x) + D_nu(a) + D_mu(b) with
// D_d(a) = i(x + a e_d) - i(x) for the periodic shift along d alone.
__device__ __forceinline__ int shift_delta(const Geo &g, const Pt &x, int d, int a) {
    if (d == 0) {
        const int xn = wrapc(x.x0 + a, g.L[0]);
        return ((xn & 3) - (x.x0 & 3)) * g.Qp + ((xn >> 2) - (x.x0 >> 2));
    }
    // explicit selects: indexing the kernel-parameter array with a runtime d
    // would force a copy of the parameters to local memory
    const int xd = d == 1 ? x.x1 : (d == 2 ? x.x2 : x.x3);
    const int Ld = d == 1 ? g.L[1] : (d == 2 ? g.L[2] : g.L[3]);
    const int st = d == 1 ? g.Lxp : (d == 2 ? g.Lxp * g.L[1] : g.Lxp * g.L[1] * g.L[2]);
    return (wrapc(xd + a, Ld) - xd) * st;
}

// Link of direction d at plane position i, daggered when dag is true.
// St: the storage precision (FP32 links read in FP64 by the re-decision kernel).
template <class T, int NC, class St = T>
__device__ __forceinline__ M3<T> link_at(const Geo &g, const St *__restrict__ U, int d, int i, bool dag) {
    M3<T> m = load_link_as<T, NC>(U, g.P, d, i);
    return dag ? m3_dag(m) : m;
}

// Sigma_mu(x) for link (x, MU) read from field U, in three passes over the six
// directions (nu, s) so that only one accumulator is live at a time:
//   1. wide forward  F  = sum A B U_mu(x+s nu+mu) (step -s nu from x+s nu+2mu),
//                    Sigma  = c1 F U_mu^dag(x+mu)
//   2. wide backward Bk = sum (step s nu from x-mu) U_mu(x-mu+s nu) B C,
//                    Sigma += c1 U_mu^dag(x-mu) Bk
//   3. staples + tall rectangles: Sigma += A (c0 B + c1 T) C
// with A = step s nu from x, B = U_mu(x+s nu), C = step -s nu from x+s nu+mu
// and T = (step s nu from x+s nu) U_mu(x+2s nu) (step -s nu from x+2s nu+mu).
// 10 products per direction plus 2.  Without rectangles: Sigma = c0 sum A B C.
// A path step from site p along +nu is U_nu(p); along -nu it is U_nu(p - nu)^dag.
// Sites are written x + a nu + b mu and addressed as i0 + Dn(a) + Dm(b).
// Plane positions around one link: i0 and the shifts along mu (b = -1, 1, 2)
// and along the current nu (a = -2, -1, 1, 2).
struct Around {
    int i0, dmm1, dmp1, dmp2, dnm2, dnm1, dnp1, dnp2;
};

__device__ __forceinline__ int around_pos(const Around &S, int a, int b) {
    const int da = a == 0 ? 0 : (a == -1 ? S.dnm1 : (a == 1 ? S.dnp1 : (a == -2 ? S.dnm2 : S.dnp2)));
    const int db = b == 0 ? 0 : (b == -1 ? S.dmm1 : (b == 1 ? S.dmp1 : S.dmp2));
    return S.i0 + da + db;
}

__device__ __forceinline__ void around_nu(const Geo &g, const Pt &x, int nu, bool rect, Around &S) {
    S.dnm1 = shift_delta(g, x, nu, -1);
    S.dnp1 = shift_delta(g, x, nu, 1);
    S.dnm2 = rect ? shift_delta(g, x, nu, -2) : 0;
    S.dnp2 = rect ? shift_delta(g, x, nu, 2) : 0;
}

// Path step along s*nu from site x + a nu + b mu.
template <class T, int NC, class St = T>
__device__ __forceinline__ M3<T> step_fwd(const Geo &g, const St *__restrict__ U, const Around &S, int nu,
                                          int s, int a, int b) {
    return s > 0 ? link_at<T, NC>(g, U, nu, around_pos(S, a, b), false)
                 : link_at<T, NC>(g, U, nu, around_pos(S, a - 1, b), true);
}

// Path step along -s*nu from site x + a nu + b mu.
template <class T, int NC, class St = T>
__device__ __forceinline__ M3<T> step_back(const Geo &g, const St *__restrict__ U, const Around &S, int nu,
                                           int s, int a, int b) {
    return s > 0 ? link_at<T, NC>(g, U, nu, around_pos(S, a - 1, b), true)
                 : link_at<T, NC>(g, U, nu, around_pos(S, a, b), false);
}

template <class T, int NC, int MU, class St = T>
__device__ __forceinline__ M3<T> link_mu(const Geo &g, const St *__restrict__ U, const Around &S, int a, int b) {
    return link_at<T, NC>(g, U, MU, around_pos(S, a, b), false);
}

template <class T, int NC, bool RECT, int MU, class St = T>
__device__ __forceinline__ M3<T> staple_sum(const Geo &g, const St *__restrict__ U, Pt x, T c0, T c1) {
    Around S;
    S.i0 = sidx(g, x);
    S.dmm1 = shift_delta(g, x, MU, -1);
    S.dmp1 = shift_delta(g, x, MU, 1);
    S.dmp2 = RECT ? shift_delta(g, x, MU, 2) : 0;
    M3<T> sig;
    m3_zero(sig);
    if (RECT) {
        {   // 1. wide forward: F = sum A B U_mu(s,1) back(s,2); Sigma = c1 F U_mu^dag(x+mu)
            M3<T> F;
            m3_zero(F);
#pragma unroll 1
            for (int j = 1; j < 4; ++j) {
                const int nu = (MU + j) & 3;
                around_nu(g, x, nu, true, S);
#pragma unroll
                for (int s = 1; s >= -1; s -= 2) {
                    M3<T> W = m3_mul(step_fwd<T, NC>(g, U, S, nu, s, 0, 0), link_mu<T, NC, MU>(g, U, S, s, 0));
                    W = m3_mul(W, link_mu<T, NC, MU>(g, U, S, s, 1));
                    m3_madd(F, W, step_back<T, NC>(g, U, S, nu, s, s, 2));
                }
            }
            M3<T> t = m3_mul_nd(F, link_at<T, NC>(g, U, MU, S.i0 + S.dmp1, false));
            m3_axpy(sig, c1, t);
        }
        {   // 2. wide backward: Bk = sum fwd(0,-1) U_mu(s,-1) B C; Sigma += c1 U_mu^dag(x-mu) Bk
            M3<T> Bk;
            m3_zero(Bk);
#pragma unroll 1
            for (int j = 1; j < 4; ++j) {
                const int nu = (MU + j) & 3;
                around_nu(g, x, nu, true, S);
#pragma unroll
                for (int s = 1; s >= -1; s -= 2) {
                    M3<T> BC = m3_mul(link_mu<T, NC, MU>(g, U, S, s, 0), step_back<T, NC>(g, U, S, nu, s, s, 1));
                    M3<T> Y = m3_mul(step_fwd<T, NC>(g, U, S, nu, s, 0, -1), link_mu<T, NC, MU>(g, U, S, s, -1));
                    m3_madd(Bk, Y, BC);
                }
            }
            M3<T> t = m3_mul_dn(link_at<T, NC>(g, U, MU, S.i0 + S.dmm1, false), Bk);
            m3_axpy(sig, c1, t);
        }
        // 3. staples and tall rectangles: Sigma += A (c0 B + c1 fwd(s,0) U_mu(2s,0) back(2s,1)) C
#pragma unroll 1
        for (int j = 1; j < 4; ++j) {
            const int nu = (MU + j) & 3;
            around_nu(g, x, nu, true, S);
#pragma unroll
            for (int s = 1; s >= -1; s -= 2) {
                M3<T> Tt = m3_mul(step_fwd<T, NC>(g, U, S, nu, s, s, 0), link_mu<T, NC, MU>(g, U, S, 2 * s, 0));
                Tt = m3_mul(Tt, step_back<T, NC>(g, U, S, nu, s, 2 * s, 1));
                M3<T> N = link_mu<T, NC, MU>(g, U, S, s, 0);
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    N.re[k] = fma(c1, Tt.re[k], c0 * N.re[k]);
                    N.im[k] = fma(c1, Tt.im[k], c0 * N.im[k]);
                }
                M3<T> AN = m3_mul(step_fwd<T, NC>(g, U, S, nu, s, 0, 0), N);
                m3_madd(sig, AN, step_back<T, NC>(g, U, S, nu, s, s, 1));
            }
        }
    } else {
#pragma unroll 1
        for (int j = 1; j < 4; ++j) {
            const int nu = (MU + j) & 3;
            around_nu(g, x, nu, false, S);
#pragma unroll
            for (int s = 1; s >= -1; s -= 2) {
                M3<T> AB = m3_mul(step_fwd<T, NC>(g, U, S, nu, s, 0, 0), link_mu<T, NC, MU>(g, U, S, s, 0));
                m3_madd(sig, AB, step_back<T, NC>(g, U, S, nu, s, s, 1));
            }
        }
        if (c0 != T(1)) m3_scale(sig, c0);
    }
    return sig;
}

// exp(i H) coefficients by the Cayley-Hamilton series.  H given by its
// diagonal (h00, h11, h22) and upper entries h01, h02, h12 (re, im).
// Terms are summed in groups of four (i^n cycles 1, i, -1, -i) until the
// bound r^n / n! on the next term, r = |H|_F >= |H|_2, drops below the
// precision's epsilon; GROUPS caps the number of groups (4*GROUPS terms).
// Returns false if r exceeds rmax (the caller then redoes it in FP64).
template <class R, int GROUPS>
__device__ __forceinline__ bool ch_exp_coeffs(R h00, R h11, R h22, R h01r, R h01i, R h02r, R h02i,
                                              R h12r, R h12i, R rmax, R f[6]) {
    const R a01 = h01r * h01r + h01i * h01i;
    const R a02 = h02r * h02r + h02i * h02i;
    const R a12 = h12r * h12r + h12i * h12i;
    const R tau = R(0.5) * (h00 * h00 + h11 * h11 + h22 * h22) + a01 + a02 + a12;
    // det H = h00 h11 h22 + 2 Re(h01 h12 conj(h02)) - h00|h12|^2 - h11|h02|^2 - h22|h01|^2
    const R pr = h01r * h12r - h01i * h12i, pi = h01r * h12i + h01i * h12r;
    const R delta = h00 * h11 * h22 + R(2) * (pr * h02r + pi * h02i) - h00 * a12 - h11 * a02 - h22 * a01;
    const R r2 = R(2) * tau;
    R f0r = 1, f0i = 0, f1r = 0, f1i = 0, f2r = 0, f2i = 0;
    R a = 1, b = 0, c = 0, bound = 1;
    const R eps = Tol<R>::eps();
#pragma unroll
    for (int g4 = 0; g4 < GROUPS; ++g4) {
        const int n = 4 * g4 + 1;
        R na, nb, nc, inv;
        inv = R(1) / R(n);                        // i^n = i
        na = delta * c * inv; nb = (a + tau * c) * inv; nc = b * inv;
        a = na; b = nb; c = nc;
        f0i += a; f1i += b; f2i += c;
        inv = R(1) / R(n + 1);                    // i^n = -1
        na = delta * c * inv; nb = (a + tau * c) * inv; nc = b * inv;
        a = na; b = nb; c = nc;
        f0r -= a; f1r -= b; f2r -= c;
        inv = R(1) / R(n + 2);                    // i^n = -i
        na = delta * c * inv; nb = (a + tau * c) * inv; nc = b * inv;
        a = na; b = nb; c = nc;
        f0i -= a; f1i -= b; f2i -= c;
        inv = R(1) / R(n + 3);                    // i^n = 1
        na = delta * c * inv; nb = (a + tau * c) * inv; nc = b * inv;
        a = na; b = nb; c = nc;
        f0r += a; f1r += b; f2r += c;
        bound *= r2 * r2 * (R(1) / (R(n) * R(n + 1) * R(n + 2) * R(n + 3)));
        if (bound < eps) break;
    }
    f[0] = f0r; f[1] = f0i; f[2] = f1r; f[3] = f1i; f[4] = f2r; f[5] = f2i;
    return r2 <= rmax * rmax;
}

// FP64 redo of the coefficients for FP32 kernels (|H|_F > 1), out of line:
// the workloads never take it, and inlined it would put ~37 KB of cold code
// between the hot parts of the class-update kernel.
static __device__ __noinline__ void ch_exp_coeffs_fp64(double h00, double h11, double h22, double h01r, double h01i,
                                                double h02r, double h02i, double h12r, double h12i, double fd[6]) {
    ch_exp_coeffs<double, 12>(h00, h11, h22, h01r, h01i, h02r, h02i, h12r, h12i, 1e300, fd);
}

// M = exp(i H) for Hermitian traceless H given by its diagonal and upper
// entries.  fp64_used reports an FP64 redo of the coefficients.
template <class T>
__device__ __forceinline__ M3<T> exp_iH(T h00, T h11, T h22, T h01r, T h01i, T h02r, T h02i,
                                        T h12r, T h12i, bool &fp64_used) {
    T f[6];
    fp64_used = false;
    if (sizeof(T) == 4) {
        // FP32 series: 12 terms reach 1.5e-8 for |H|_F <= 1; beyond that the
        // coefficients are redone in FP64 (48 terms, accurate to |H|_F <= 8).
        if (!ch_exp_coeffs<T, 3>(h00, h11, h22, h01r, h01i, h02r, h02i, h12r, h12i, T(1.0), f)) {
            double fd[6];
            ch_exp_coeffs_fp64(h00, h11, h22, h01r, h01i, h02r, h02i, h12r, h12i, fd);
#pragma unroll
            for (int k = 0; k < 6; ++k) f[k] = T(fd[k]);
            fp64_used = true;
        }
    } else {
        ch_exp_coeffs<T, 12>(h00, h11, h22, h01r, h01i, h02r, h02i, h12r, h12i, T(1e300), f);
    }
    // M = f0 I + f1 H + f2 H^2
    M3<T> H;
    H.re[0] = h00; H.im[0] = 0; H.re[4] = h11; H.im[4] = 0; H.re[8] = h22; H.im[8] = 0;
    H.re[1] = h01r; H.im[1] = h01i; H.re[3] = h01r; H.im[3] = -h01i;
    H.re[2] = h02r; H.im[2] = h02i; H.re[6] = h02r; H.im[6] = -h02i;
    H.re[5] = h12r; H.im[5] = h12i; H.re[7] = h12r; H.im[7] = -h12i;
    // H^2 is Hermitian: its diagonal (real) and upper entries, the lower ones
    // by conjugation (a third of the operations of a general product)
    M3<T> H2;
    {
        const T a01 = h01r * h01r + h01i * h01i, a02 = h02r * h02r + h02i * h02i, a12 = h12r * h12r + h12i * h12i;
        H2.re[0] = fma(h00, h00, a01 + a02); H2.im[0] = 0;
        H2.re[4] = fma(h11, h11, a01 + a12); H2.im[4] = 0;
        H2.re[8] = fma(h22, h22, a02 + a12); H2.im[8] = 0;
        const T s01 = h00 + h11, s02 = h00 + h22, s12 = h11 + h22;
        // (0,1): h01 (h00 + h11) + h02 conj(h12)
        H2.re[1] = fma(h01r, s01, fma(h02r, h12r, h02i * h12i));
        H2.im[1] = fma(h01i, s01, fma(h02i, h12r, -(h02r * h12i)));
        // (0,2): h02 (h00 + h22) + h01 h12
        H2.re[2] = fma(h02r, s02, fma(h01r, h12r, -(h01i * h12i)));
        H2.im[2] = fma(h02i, s02, fma(h01r, h12i, h01i * h12r));
        // (1,2): h12 (h11 + h22) + conj(h01) h02
        H2.re[5] = fma(h12r, s12, fma(h01r, h02r, h01i * h02i));
        H2.im[5] = fma(h12i, s12, fma(h01r, h02i, -(h01i * h02r)));
        H2.re[3] = H2.re[1]; H2.im[3] = -H2.im[1];
        H2.re[6] = H2.re[2]; H2.im[6] = -H2.im[2];
        H2.re[7] = H2.re[5]; H2.im[7] = -H2.im[5];
    }
    M3<T> Mx;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        T re = f[2] * H.re[k] - f[3] * H.im[k] + f[4] * H2.re[k] - f[5] * H2.im[k];
        T im = f[2] * H.im[k] + f[3] * H.re[k] + f[4] * H2.im[k] + f[5] * H2.re[k];
        if (k == 0 || k == 4 || k == 8) { re += f[0]; im += f[1]; }
        Mx.re[k] = re;
        Mx.im[k] = im;
    }
    return Mx;
}

// H = -i rho Q for staple sum sig and link Ux (Eq. generator: Omega = sig
// Ux^dag, Q its traceless anti-Hermitian part), as its diagonal and upper
// entries h[0..8] = (h00, h11, h22, h01r, h01i, h02r, h02i, h12r, h12i).
// Diagonal rho (Im Om_jj - (1/3) sum_l Im Om_ll), written so that equal
// diagonal entries give exactly zero; off-diagonal
// H_jk = (rho/2) [(Im Om_jk + Im Om_kj) - i (Re Om_jk - Re Om_kj)].
template <class T>
__device__ __forceinline__ void stout_H(const M3<T> &sig, const M3<T> &Ux, T rho, T h[9]) {
    M3<T> Om = m3_mul_nd(sig, Ux);
    const T third = T(1) / T(3);
    h[0] = rho * ((T(2) * Om.im[0] - Om.im[4] - Om.im[8]) * third);
    h[1] = rho * ((T(2) * Om.im[4] - Om.im[0] - Om.im[8]) * third);
    h[2] = rho * ((T(2) * Om.im[8] - Om.im[0] - Om.im[4]) * third);
    const T hr = T(0.5) * rho;
    h[3] = hr * (Om.im[1] + Om.im[3]); h[4] = -hr * (Om.re[1] - Om.re[3]);
    h[5] = hr * (Om.im[2] + Om.im[6]); h[6] = -hr * (Om.re[2] - Om.re[6]);
    h[7] = hr * (Om.im[5] + Om.im[7]); h[8] = -hr * (Om.re[5] - Om.re[7]);
}

// Candidate U' = exp(rho Q) U for staple sum sig.
template <class T>
__device__ __forceinline__ M3<T> stout_candidate(const M3<T> &sig, const M3<T> &Ux, T rho, bool &fp64_used) {
    T h[9];
    stout_H<T>(sig, Ux, rho, h);
    M3<T> Mx = exp_iH<T>(h[0], h[1], h[2], h[3], h[4], h[5], h[6], h[7], h[8], fp64_used);
    return m3_mul(Mx, Ux);
}

#ifndef VS_SUBSWEEP_THREADS
#define VS_SUBSWEEP_THREADS 256
#endif
#ifndef VS_SUBSWEEP_MINB
#define VS_SUBSWEEP_MINB (512 / VS_SUBSWEEP_THREADS)
#endif

// Outcome of one link update, for the per-sweep counters.
template <class T>
struct Update {
    bool reject = false;   // the vortex-preservation test refused the candidate
    bool second = false;   // FP64 exponential coefficients (APE: a singular blocked matrix)
    bool labdiff = false;  // the candidate's label differs from the reference label
    bool undec = false;    // the candidate's trace lies within the precision's error band of a sector edge
    T sine = T(2);         // sine of the candidate's angular margin from a sector edge (2: no candidate)
};

// Error band of a candidate's trace, in trace units (the entries have unit
// modulus, so trace errors are absolute).  FP32: one sweep from a common FP64
// state puts an FP32 candidate within 1.7e-7 per entry of the FP64 one
// (measured along a 200-sweep trajectory), its trace within ~5e-7; within
// 2e-6 of an edge the rounding of the FP32 links and arithmetic can decide the
// vortex-preservation test, so such a candidate is counted as undecidable.
// FP64: two FP64 implementations differ by ~1e-15 per sweep.
template <class T> struct EdgeBand;
template <> struct EdgeBand<float> { static __device__ __forceinline__ float v() { return 2e-6f; } };
template <> struct EdgeBand<double> { static __device__ __forceinline__ double v() { return 1e-12; } };

// The candidate's label against the reference (Sec. VI), its distance from
// the nearest sector edge (Sec. I Eq. centre_element) and the margin sine.
template <class T>
__device__ __forceinline__ void vp_decide(bool vp, bool want_sine, int ref, T tr_re, T tr_im, Update<T> &u,
                                          T band = EdgeBand<T>::v()) {
    const int lab = z3_label<T>(tr_re, tr_im);
    const T dist = edge_distance<T>(tr_re, tr_im, lab);
    u.reject = vp && lab != ref;
    u.labdiff = lab != ref;
    u.undec = dist < band;
    if (want_sine) u.sine = edge_sine<T>(tr_re, tr_im, dist);
}

// Stout candidate for link (x, MU) at plane position i from its staple sum,
// vortex-preservation test against the reference label, store if accepted.
template <class T, int NC, int MU>
__device__ __forceinline__ void stout_store(const SubsweepParams &a, const Pt &x, int i, const M3<T> &sig,
                                            const M3<T> &Ux, Update<T> &u) {
    const Geo &g = a.g;
    const T rho = sizeof(T) == 4 ? T(a.rho_f) : T(a.rho);
    M3<T> Un = stout_candidate<T>(sig, Ux, rho, u.second);
    // 12-real storage keeps rows 0-1 and rebuilds row 2 on every load: the
    // test must see that matrix, not the one computed here
    if (NC == 12) rebuild_row2(Un);
    T tr_re, tr_im;
    vp_trace<T>(static_cast<const T *>(a.G), g.P, i, a.G ? sidx(g, mv(g, x, MU, 1)) : i, Un, tr_re, tr_im);
    vp_decide<T>(a.vp, a.counters != nullptr, (int)a.ref[(long long)MU * g.P + i], tr_re, tr_im, u);
    if constexpr (sizeof(T) == 4) {
        // within the FP32 band of an edge: leave the link to k_redecide
        if (a.defer_idx && a.vp && u.undec) {
            const unsigned slot = atomicAdd(a.defer_n, 1u);
            if (slot < (unsigned)a.defer_cap) {
                a.defer_idx[slot] = i;
                u.reject = u.labdiff = u.undec = false;
                u.sine = T(2);
                return;
            }
        }
    }
    // a rejected link keeps its value: nothing to write in place (annealed),
    // the old link into the destination when that is another buffer
    if (!u.reject) store_link<T, NC>(static_cast<T *>(a.U), g.P, MU, i, Un);
    else if (a.U != a.Usrc) store_link<T, NC>(static_cast<T *>(a.U), g.P, MU, i, Ux);
}

// Per-warp counts into a sweep's counter slots (kCnt* in vs_internal.h):
// rejects, the second count (FP64 exponentials; singular blocked matrices in
// APE), label differences, undecidable candidates, and the smallest margin
// sine (as the bits of a non-negative double, whose order is that of
// unsigned integers).
template <class T>
__device__ __forceinline__ void count_update(unsigned long long *c, const Update<T> &u) {
    if (!c) return;
    const unsigned rb = __ballot_sync(0xffffffffu, u.reject);
    const unsigned fb = __ballot_sync(0xffffffffu, u.second);
    const unsigned lb = __ballot_sync(0xffffffffu, u.labdiff);
    const unsigned ub = __ballot_sync(0xffffffffu, u.undec);
    T m = u.sine;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T v = __shfl_xor_sync(0xffffffffu, m, o);
        m = v < m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) {
        if (rb) atomicAdd(&c[kCntReject], (unsigned long long)__popc(rb));
        if (fb) atomicAdd(&c[kCntSecond], (unsigned long long)__popc(fb));
        if (lb) atomicAdd(&c[kCntLabelDiff], (unsigned long long)__popc(lb));
        if (ub) atomicAdd(&c[kCntUndecidable], (unsigned long long)__popc(ub));
        if (m < T(2)) atomicMin(&c[kCntMarginSine], (unsigned long long)__double_as_longlong((double)m));
    }
}

// Band of a candidate computed in FP64 from FP32-stored links: rounding the
// links to FP32 moves each entry by up to 6e-8 relative, the candidate's
// trace by a few 1e-7 (the staple sum adds 24 paths); within this band of an
// edge the FP32 field itself, not the arithmetic, can decide the test.
constexpr double kRedecideBand = 1e-6;

// FP64 re-decision of the FP32 candidates a class launch left to it (its
// FP32 trace within EdgeBand<float> of a sector edge, Sec. VI): the same
// candidate from the same stored links in FP64 arithmetic, decided, stored
// (rounded to FP32) if accepted.  No link of a colour class enters the staples
// of another of the class, so the field the class launch left is this
// candidate's input.  One lane per listed link; the last block to finish
// resets the list for the next class launch.
template <int NC, bool RECT, int MU>
__global__ void __launch_bounds__(32) k_redecide(SubsweepParams a) {
    const Geo &g = a.g;
    const unsigned n = min(*a.defer_n, (unsigned)a.defer_cap);
    const float *Us = static_cast<const float *>(a.Usrc);
    for (unsigned k0 = blockIdx.x * 32u; k0 < n; k0 += gridDim.x * 32u) {
        const unsigned k = k0 + (threadIdx.x & 31u);
        Update<double> up;
        if (k < n) {
            const int i = a.defer_idx[k];
            const Pt x = site_of_pos(g, i);
            const M3<double> sig = staple_sum<double, NC, RECT, MU>(g, Us, x, a.c0, a.c1);
            const M3<double> Ux = load_link_as<double, NC>(Us, g.P, MU, i);
            M3<double> Un = stout_candidate<double>(sig, Ux, a.rho, up.second);
            if (NC == 12) rebuild_row2(Un);
            double tr_re, tr_im;
            vp_trace<double>(static_cast<const float *>(a.G), g.P, i, a.G ? sidx(g, mv(g, x, MU, 1)) : i, Un, tr_re,
                             tr_im);
            const int ref = (int)a.ref[(long long)MU * g.P + i];
            vp_decide<double>(a.vp, a.counters != nullptr, ref, tr_re, tr_im, up, kRedecideBand);
            const M3<float> Uf = m3_cast<float>(Un);   // the candidate as stored
            if (!up.reject) {
                // vortex preservation holds for the stored FP32 link as every FP32
                // kernel reads it (12-real: row 2 rebuilt in FP32): a candidate whose
                // rounding crosses the edge keeps the old link (it lies within the band)
                M3<float> Uv = Uf;
                if (NC == 12) rebuild_row2(Uv);
                float fa, fb;
                vp_trace<float>(static_cast<const float *>(a.G), g.P, i, a.G ? sidx(g, mv(g, x, MU, 1)) : i, Uv, fa,
                                fb);
                if (z3_label<float>(fa, fb) != ref) up.reject = up.labdiff = up.undec = true;
            }
            if (!up.reject) store_link<float, NC>(static_cast<float *>(a.U), g.P, MU, i, Uf);
            else if (a.U != a.Usrc) store_link<float, NC>(static_cast<float *>(a.U), g.P, MU, i, m3_cast<float>(Ux));
        }
        count_update<double>(a.counters, up);
        const unsigned rb = __ballot_sync(0xffffffffu, k < n);
        if (a.counters && (threadIdx.x & 31u) == 0 && rb)
            atomicAdd(&a.counters[kCntRedecided], (unsigned long long)__popc(rb));
    }
    if ((threadIdx.x & 31u) == 0) {
        __threadfence();
        if (atomicAdd(a.defer_done, 1u) == gridDim.x - 1) {
            *a.defer_n = 0;
            *a.defer_done = 0;
        }
    }
}

// One thread per link of the colour class (or of direction MU when colour < 0).
// FP32: at most 65536 / (VS_SUBSWEEP_THREADS * VS_SUBSWEEP_MINB) registers per
// thread (128 by default), so VS_SUBSWEEP_MINB blocks fit on an SM (16 warps).
template <class T, int NC, bool RECT, int MU>
__global__ void __launch_bounds__(VS_SUBSWEEP_THREADS, sizeof(T) == 4 ? VS_SUBSWEEP_MINB : 1)
    k_subsweep(SubsweepParams a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < a.n_threads;
    Update<T> u;
    if (active) {
        const Geo &g = a.g;
        Pt x = a.colour >= 0 ? class_site<MU>(g, a.colour, t) : dir_site<MU>(g, t);
        const int i = sidx(g, x);
        const T *Us = static_cast<const T *>(a.Usrc);
        const T c0 = sizeof(T) == 4 ? T(a.c0_f) : T(a.c0), c1 = sizeof(T) == 4 ? T(a.c1_f) : T(a.c1);
        M3<T> sig = staple_sum<T, NC, RECT, MU>(g, Us, x, c0, c1);
        M3<T> Ux = load_link<T, NC>(Us, g.P, MU, i);
        stout_store<T, NC, MU>(a, x, i, sig, Ux, u);
    }
    count_update<T>(a.counters, u);
}

// ---------------------------------------------------------------------------
// FP32 link streams.  Each thread keeps the next links it will read in flight
// as asynchronous global -> shared copies (cp.async) into its own ring of
// slots in shared memory, so no register holds a pending load and the latency
// of one link is covered by the products of the links before it.  A slot is
// refilled, right after it is read, with the link that many places ahead in
// the thread's stream; every slot index is known at compile time.
// ---------------------------------------------------------------------------

#ifndef VS_RING
#define VS_RING 1
#endif
#ifndef VS_RING_THREADS
#define VS_RING_THREADS 128
#endif
#ifndef VS_RING_MINB
#define VS_RING_MINB (384 / VS_RING_THREADS)
#endif

template <int NC>
struct LinkRing {
    const float4 *v4;   // this thread's column of the float4 slots [depth][NC/4][BT]
    const float2 *v2;   // and of the float2 slots [depth][BT] (NC == 18)
    uint32_t a4, a2;    // the same as shared-window addresses
};

// Start the copy of the link at site position i of the direction whose
// links begin at base into slot SLOT, as one commit group.
template <int NC, int SLOT>
__device__ __forceinline__ void ring_fetch(const LinkRing<NC> &R, const float *base, long long P, int i) {
    constexpr int NQ = NC / 4;
    const float *b0 = base + blk_off4<NC>(i);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float4 *src = reinterpret_cast<const float4 *>(b0 + 64 * q);
        const uint32_t dst = R.a4 + (uint32_t)((SLOT * NQ + q) * VS_RING_THREADS * 16);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
    if (NC == 18) {
        const float2 *src = reinterpret_cast<const float2 *>(base + blk_off2(i));
        const uint32_t dst = R.a2 + (uint32_t)(SLOT * VS_RING_THREADS * 8);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// ring_fetch with a predicate: on == false commits an empty group.
template <int NC, int SLOT>
__device__ __forceinline__ void ring_fetch_if(const LinkRing<NC> &R, const float *base, long long P, int i,
                                              bool on) {
    constexpr int NQ = NC / 4;
    const int pr = on ? 1 : 0;
    const float *b0 = base + blk_off4<NC>(i);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float4 *src = reinterpret_cast<const float4 *>(b0 + 64 * q);
        const uint32_t dst = R.a4 + (uint32_t)((SLOT * NQ + q) * VS_RING_THREADS * 16);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n"
            " @p cp.async.cg.shared.global [%0], [%1], 16;\n}\n" ::"r"(dst), "l"(src), "r"(pr)
            : "memory");
    }
    if (NC == 18) {
        const float2 *src = reinterpret_cast<const float2 *>(base + blk_off2(i));
        const uint32_t dst = R.a2 + (uint32_t)(SLOT * VS_RING_THREADS * 8);
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n"
            " @p cp.async.ca.shared.global [%0], [%1], 8;\n}\n" ::"r"(dst), "l"(src), "r"(pr)
            : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// Past the end of the stream: an empty group keeps one group per link.
__device__ __forceinline__ void ring_skip() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// Read the link in slot SLOT, daggered if DAG; the caller has waited
// (cp.async.wait_group) until the copy into that slot is complete.
// FULL = false: only rows 0-1 are needed (a left factor of a two-row
// product), so 12-real storage skips rebuilding row 2.
template <int NC, bool DAG, int SLOT, bool FULL = true>
__device__ __forceinline__ M3<float> ring_read(const LinkRing<NC> &R) {
    constexpr int NQ = NC / 4;
    M3<float> m;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const float4 v = R.v4[(SLOT * NQ + q) * VS_RING_THREADS];
        m.re[2 * q] = v.x; m.im[2 * q] = v.y; m.re[2 * q + 1] = v.z; m.im[2 * q + 1] = v.w;
    }
    if (NC == 18) {
        const float2 v = R.v2[SLOT * VS_RING_THREADS];
        m.re[8] = v.x; m.im[8] = v.y;
    }
    if (NC == 12 && (FULL || DAG)) rebuild_row2(m);
    return DAG ? m3_dag(m) : m;
}

// ---------------------------------------------------------------------------
// One pass per (nu, s), every link read once.  With A = step(x, s nu),
// B = U_mu(x+s nu), C = step(x+s nu+mu, -s nu), the wide backward rectangle,
// the plaquette staple and the tall rectangle of (nu, s) all end in C:
//   Sigma = c1 F(x) U_mu^dag(x+mu)
//         + sum_{nu,s} [c1 U_mu^dag(x-mu) G H B + c0 A B + c1 A T] C,
// G = step(x-mu, s nu), H = U_mu(x-mu+s nu), T the upper half of the tall
// rectangle, and F(x) = sum A B D E (D = U_mu(x+s nu+mu), E = step(x+s nu+2mu,
// -s nu)) shares A B.  A unit reads its 10 distinct links once (63 per update
// with U_mu(x +- mu) and U_mu(x), against 85 + 2 in three passes), in a
// 12-entry stream slot pattern: A B G H D E T0 T1 T2 C, then two spare
// entries that carry U_mu^dag(x+mu) and U_mu(x) in the last unit.  Ring depth 6
// (slot = entry mod 6, compile-time).
// ---------------------------------------------------------------------------

template <int NC, bool DAG, int SLOT, bool FULL = true>
__device__ __forceinline__ M3<float> ring_take6(const LinkRing<NC> &R) {
    asm volatile("cp.async.wait_group 5;\n" ::: "memory");
    return ring_read<NC, DAG, SLOT, FULL>(R);
}

// Link K of the unit (nu, s): direction and site x + a nu + b mu.
template <int S, int K>
__device__ __forceinline__ void u_link(const Around &A, const float *Umu, const float *Unu, const float *&base,
                                       int &pos) {
    constexpr int f0 = S > 0 ? 0 : -1, f1 = S > 0 ? 1 : -2;
    constexpr bool mu = K == 1 || K == 3 || K == 4 || K == 7;
    constexpr int a = K == 0 ? f0 : K == 1 ? S : K == 2 ? f0 : K == 3 ? S : K == 4 ? S : K == 5 ? f0
                    : K == 6 ? f1 : K == 7 ? 2 * S : K == 8 ? f1 : f0;
    constexpr int b = K == 0 ? 0 : K == 1 ? 0 : K == 2 ? -1 : K == 3 ? -1 : K == 4 ? 1 : K == 5 ? 2
                    : K == 6 ? 0 : K == 7 ? 0 : K == 8 ? 1 : 1;
    base = mu ? Umu : Unu;
    pos = around_pos(A, a, b);
}

// Refill after entry K of unit (nu, s), into slot K mod 6: entry K + 6 of the
// same unit (the spare entries 10, 11 carry U_mu(x+mu), U_mu(x) in the last
// unit, nothing otherwise), or entry K - 6 of the next unit: (nu, -1) for
// s = +1, (next nu, +1) on An for s = -1, nothing after the last.
template <int NC, int S, int K>
__device__ __forceinline__ void u_refill(const LinkRing<NC> &R, const float *Umu, const float *Unu,
                                         const float *Un, long long P, const Around &A, const Around &An,
                                         bool last) {
    constexpr int SL = K % 6;
    const float *base;
    int pos;
    if constexpr (K + 6 <= 9) {
        u_link<S, (K + 6 <= 9 ? K + 6 : 0)>(A, Umu, Unu, base, pos);
        ring_fetch<NC, SL>(R, base, P, pos);
    } else if constexpr (K + 6 <= 11) {
        // spare entries: U_mu(x+mu) (K + 6 = 10) and U_mu(x) (11) in the last unit
        const int p = K + 6 == 10 ? A.i0 + A.dmp1 : A.i0;
        if constexpr (S > 0) ring_skip();
        else ring_fetch_if<NC, SL>(R, Umu, P, p, last);
    } else if constexpr (S > 0) {
        u_link<-1, (K >= 6 ? K - 6 : 0)>(A, Umu, Unu, base, pos);
        ring_fetch<NC, SL>(R, base, P, pos);
    } else {
        u_link<1, (K >= 6 ? K - 6 : 0)>(An, Umu, Un, base, pos);
        ring_fetch_if<NC, SL>(R, base, P, pos, !last);
    }
}

template <int NC, int S>
__device__ __forceinline__ void fused_unit(const LinkRing<NC> &R, M3<float> &Facc, M3<float> &sig, float c0,
                                           float c1, const M3<float> &Lm, const float *Umu, const float *Unu,
                                           const float *Un, long long P, const Around &A, const Around &An,
                                           bool last) {
    const M3<float> Af = ring_take6<NC, (S < 0), 0, false>(R);
    u_refill<NC, S, 0>(R, Umu, Unu, Un, P, A, An, last);
    const M3<float> B = ring_take6<NC, false, 1>(R);
    u_refill<NC, S, 1>(R, Umu, Unu, Un, P, A, An, last);
    M3<float> AB;
    m3_mul_2r(AB, Af, B);
    M3<float> X, Y;
    {   // c1 U_mu^dag(x-mu) G H B
        const M3<float> G = ring_take6<NC, (S < 0), 2>(R);
        u_refill<NC, S, 2>(R, Umu, Unu, Un, P, A, An, last);
        m3_mul_2r(X, Lm, G);
        const M3<float> H = ring_take6<NC, false, 3>(R);
        u_refill<NC, S, 3>(R, Umu, Unu, Un, P, A, An, last);
        m3_mul_2r(Y, X, H);
        m3_mul_2r(X, Y, B);
    }
    M3<float> W1 = X;
    rebuild_row2(W1);
    {   // F(x) += A B D E
        const M3<float> D = ring_take6<NC, false, 4>(R);
        u_refill<NC, S, 4>(R, Umu, Unu, Un, P, A, An, last);
        m3_mul_2r(X, AB, D);
        const M3<float> E = ring_take6<NC, (S > 0), 5>(R);
        u_refill<NC, S, 5>(R, Umu, Unu, Un, P, A, An, last);
        m3_mul_2r(Y, X, E);
        rebuild_row2(Y);
        m3_acc_f32(Facc, Y);
    }
    {   // A T, T = T0 T1 T2
        const M3<float> T0 = ring_take6<NC, (S < 0), 0, false>(R);
        u_refill<NC, S, 6>(R, Umu, Unu, Un, P, A, An, last);
        const M3<float> T1 = ring_take6<NC, false, 1>(R);
        u_refill<NC, S, 7>(R, Umu, Unu, Un, P, A, An, last);
        m3_mul_2r(X, T0, T1);
        const M3<float> T2 = ring_take6<NC, (S > 0), 2>(R);
        u_refill<NC, S, 8>(R, Umu, Unu, Un, P, A, An, last);
        m3_mul_2r(Y, X, T2);
        rebuild_row2(Y);
        m3_mul_2r(X, Af, Y);
        rebuild_row2(X);
    }
    rebuild_row2(AB);
    m3_lin3_f32(Y, c0, AB, c1, W1, X);   // Yc = c1 (W1 + A T) + c0 A B
    const M3<float> C = ring_take6<NC, (S > 0), 3>(R);
    u_refill<NC, S, 9>(R, Umu, Unu, Un, P, A, An, last);
    m3_madd(sig, Y, C);
    u_refill<NC, S, 10>(R, Umu, Unu, Un, P, A, An, last);   // spare entries: refills only
    u_refill<NC, S, 11>(R, Umu, Unu, Un, P, A, An, last);
}

template <int NC, int MU>
__device__ __forceinline__ M3<float> staple_sum_fused(const Geo &g, const float *__restrict__ U, Pt x, float c0,
                                                      float c1, const LinkRing<NC> &R, M3<float> &Ux) {
    const long long P = g.P;
    Around A, An;
    A.i0 = sidx(g, x);
    A.dmm1 = shift_delta(g, x, MU, -1);
    A.dmp1 = shift_delta(g, x, MU, 1);
    A.dmp2 = shift_delta(g, x, MU, 2);
    An = A;
    const float *Umu = U + (long long)MU * NC * P;
    const int nu1 = (MU + 1) & 3;
    around_nu(g, x, nu1, true, A);
    const float *Unu = U + (long long)nu1 * NC * P;
    {   // prologue: entries 0-5 of the first unit
        const float *b;
        int q;
        u_link<1, 0>(A, Umu, Unu, b, q); ring_fetch<NC, 0>(R, b, P, q);
        u_link<1, 1>(A, Umu, Unu, b, q); ring_fetch<NC, 1>(R, b, P, q);
        u_link<1, 2>(A, Umu, Unu, b, q); ring_fetch<NC, 2>(R, b, P, q);
        u_link<1, 3>(A, Umu, Unu, b, q); ring_fetch<NC, 3>(R, b, P, q);
        u_link<1, 4>(A, Umu, Unu, b, q); ring_fetch<NC, 4>(R, b, P, q);
        u_link<1, 5>(A, Umu, Unu, b, q); ring_fetch<NC, 5>(R, b, P, q);
    }
    // U_mu^dag(x - mu): rows 0-1 only are used (left factor of two-row products)
    const M3<float> Lm = m3_dag(load_link<float, NC>(U, P, MU, A.i0 + A.dmm1));
    M3<float> Facc, sig;
    m3_zero(Facc);
    m3_zero(sig);
#pragma unroll 1
    for (int j = 1; j < 4; ++j) {
        const bool last = j == 3;
        const int nun = (MU + (j < 3 ? j + 1 : 1)) & 3;
        around_nu(g, x, nun, true, An);
        const float *Un = U + (long long)nun * NC * P;
        fused_unit<NC, 1>(R, Facc, sig, c0, c1, Lm, Umu, Unu, Un, P, A, An, last);
        fused_unit<NC, -1>(R, Facc, sig, c0, c1, Lm, Umu, Unu, Un, P, A, An, last);
        A = An;
        Unu = Un;
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    const M3<float> Lp = ring_read<NC, false, 4>(R);     // U_mu(x + mu), entry 10 of the last unit
    Ux = ring_read<NC, false, 5>(R);                     // U_mu(x), entry 11
    M3<float> t = m3_mul_nd(Facc, Lp);
    m3_axpy(sig, c1, t);
    return sig;
}

// ---------------------------------------------------------------------------
// Plaquette staples alone (eps = 1) through the link ring.  A unit (nu, s) is
// the staple A B C with A = step(x, s nu), B = U_mu(x + s nu), C = step(x +
// s nu + mu, -s nu) (entries 0, 1 and 9 of a unit of the one-pass stream);
// units run (nu1, +), (nu1, -), (nu2, +), ...  Six slots hold two units, unit
// (nu, s) in slots 3 [s = -1] + 0..2, and each slot is refilled with the same
// entry of (next nu, s).  Every staple is SU(3), so it is formed in rows 0-1
// and its row 2 rebuilt.
// ---------------------------------------------------------------------------
template <int J>
__host__ __device__ constexpr int p_entry() { return J == 0 ? 0 : (J == 1 ? 1 : 9); }

template <int NC, int S, int J>
__device__ __forceinline__ void p_refill(const LinkRing<NC> &R, const float *Umu, const float *Un, long long P,
                                         const Around &An, bool last) {
    const float *base;
    int pos;
    u_link<S, p_entry<J>()>(An, Umu, Un, base, pos);
    ring_fetch_if<NC, (S < 0 ? 3 : 0) + J>(R, base, P, pos, !last);
}

template <int NC, int S>
__device__ __forceinline__ void plain_unit(const LinkRing<NC> &R, M3<float> &sig, const float *Umu,
                                           const float *Un, long long P, const Around &An, bool last) {
    constexpr int S0 = S < 0 ? 3 : 0;
    const M3<float> Af = ring_take6<NC, (S < 0), S0, false>(R);
    p_refill<NC, S, 0>(R, Umu, Un, P, An, last);
    const M3<float> B = ring_take6<NC, false, S0 + 1>(R);
    p_refill<NC, S, 1>(R, Umu, Un, P, An, last);
    M3<float> X, Y;
    m3_mul_2r(X, Af, B);
    const M3<float> C = ring_take6<NC, (S > 0), S0 + 2>(R);
    p_refill<NC, S, 2>(R, Umu, Un, P, An, last);
    m3_mul_2r(Y, X, C);
    rebuild_row2(Y);
#pragma unroll
    for (int k = 0; k < 9; ++k) { sig.re[k] += Y.re[k]; sig.im[k] += Y.im[k]; }
}

template <int NC, int MU>
__device__ __forceinline__ M3<float> staple_sum_plain_ring(const Geo &g, const float *__restrict__ U, Pt x,
                                                           float c0, const LinkRing<NC> &R) {
    const long long P = g.P;
    Around A, An;
    A.i0 = sidx(g, x);
    A.dmm1 = 0;
    A.dmp1 = shift_delta(g, x, MU, 1);
    A.dmp2 = 0;
    around_nu(g, x, (MU + 1) & 3, false, A);
    An = A;
    const float *Umu = U + (long long)MU * NC * P;
    const float *Unu = U + (long long)((MU + 1) & 3) * NC * P;
    {   // prologue: the two units of the first nu
        const float *b;
        int q;
        u_link<1, 0>(A, Umu, Unu, b, q); ring_fetch<NC, 0>(R, b, P, q);
        u_link<1, 1>(A, Umu, Unu, b, q); ring_fetch<NC, 1>(R, b, P, q);
        u_link<1, 9>(A, Umu, Unu, b, q); ring_fetch<NC, 2>(R, b, P, q);
        u_link<-1, 0>(A, Umu, Unu, b, q); ring_fetch<NC, 3>(R, b, P, q);
        u_link<-1, 1>(A, Umu, Unu, b, q); ring_fetch<NC, 4>(R, b, P, q);
        u_link<-1, 9>(A, Umu, Unu, b, q); ring_fetch<NC, 5>(R, b, P, q);
    }
    M3<float> sig;
    m3_zero(sig);
#pragma unroll 1
    for (int j = 1; j < 4; ++j) {
        const bool last = j == 3;
        const int nun = (MU + (j < 3 ? j + 1 : 1)) & 3;
        around_nu(g, x, nun, false, An);
        const float *Un = U + (long long)nun * NC * P;
        plain_unit<NC, 1>(R, sig, Umu, Un, P, An, last);
        plain_unit<NC, -1>(R, sig, Umu, Un, P, An, last);
    }
    if (c0 != 1.0f) m3_scale(sig, c0);
    return sig;
}

// Kernel attributes (here: the dynamic shared memory limit) are set per
// device.  Runs set() once for each device a launcher is used on; done holds
// one bit per device ordinal, published after set() has run, so a thread that
// sees the bit can launch.
template <class F>
inline void once_per_device(std::atomic<unsigned long long> &done, F &&set) {
    int d = 0;
    cudaGetDevice(&d);
    const unsigned long long bit = 1ull << (d & 63);
    if (done.load(std::memory_order_acquire) & bit) return;
    static std::mutex m;
    std::lock_guard<std::mutex> lock(m);
    if (done.load(std::memory_order_relaxed) & bit) return;
    set();
    done.fetch_or(bit, std::memory_order_release);
}

template <int NC>
constexpr int ring6_smem_bytes() {
    return 6 * VS_RING_THREADS * ((NC / 4) * 16 + (NC == 18 ? 8 : 0));
}

// This thread's column of the ring arrays of a kernel.
template <int NC>
__device__ __forceinline__ LinkRing<NC> ring_of(float4 *ring4, float2 *ring2) {
    LinkRing<NC> R;
    R.v4 = ring4 + threadIdx.x;
    R.v2 = ring2 + (NC == 18 ? threadIdx.x : 0);
    R.a4 = (uint32_t)__cvta_generic_to_shared(ring4 + threadIdx.x);
    R.a2 = (uint32_t)__cvta_generic_to_shared(ring2 + (NC == 18 ? threadIdx.x : 0));
    return R;
}

// FP32 standard-staple class update through the plain link ring.
template <int NC, int MU>
__global__ void __launch_bounds__(VS_RING_THREADS, 4) k_subsweep_pring(SubsweepParams a) {
    extern __shared__ float4 pring_dyn[];
    float4 *ring4 = pring_dyn;
    float2 *ring2 = reinterpret_cast<float2 *>(pring_dyn + 6 * (NC / 4) * VS_RING_THREADS);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < a.n_threads;
    Update<float> u;
    if (active) {
        const Geo &g = a.g;
        Pt x = a.colour >= 0 ? class_site<MU>(g, a.colour, t) : dir_site<MU>(g, t);
        const int i = sidx(g, x);
        const float *Us = static_cast<const float *>(a.Usrc);
        LinkRing<NC> R = ring_of<NC>(ring4, ring2);
        const M3<float> sig = staple_sum_plain_ring<NC, MU>(g, Us, x, a.c0_f, R);
        const M3<float> Ux = load_link<float, NC>(Us, g.P, MU, i);
        stout_store<float, NC, MU>(a, x, i, sig, Ux, u);
    }
    count_update<float>(a.counters, u);
}

template <int NC, int MU>
__global__ void __launch_bounds__(VS_RING_THREADS, VS_RING_MINB) k_subsweep_fused(SubsweepParams a) {
    extern __shared__ float4 ring6_dyn[];
    float4 *ring4 = ring6_dyn;
    float2 *ring2 = reinterpret_cast<float2 *>(ring6_dyn + 6 * (NC / 4) * VS_RING_THREADS);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < a.n_threads;
    Update<float> u;
    if (active) {
        const Geo &g = a.g;
        Pt x = a.colour >= 0 ? class_site<MU>(g, a.colour, t) : dir_site<MU>(g, t);
        const int i = sidx(g, x);
        LinkRing<NC> R = ring_of<NC>(ring4, ring2);
        M3<float> Ux;
        M3<float> sig = staple_sum_fused<NC, MU>(g, static_cast<const float *>(a.Usrc), x, a.c0_f, a.c1_f, R, Ux);
        stout_store<float, NC, MU>(a, x, i, sig, Ux, u);
    }
    count_update<float>(a.counters, u);
}

}  // namespace vs

namespace vs {

// MaxReTr towards the blocked matrix Vb (Eqs. maxReTr, def_L1, def_T1): for
// each SU(2) subgroup (p,q) in the order (0,1), (1,2), (0,2), n_hits times,
// only the 2x2 block of L = U Vb^dag is formed; a = (L_pp + conj L_qq)/2,
// b = (L_pq - conj L_qp)/2, k = sqrt(|a|^2 + |b|^2), and rows p, q of U are
// replaced by T^c U with T^c = [[conj a, -b], [conj b, a]] / k.  A singular
// subgroup, k <= 1e-6 of the block's scale (Sec. III.A: exact on vortex
// fields, where rounding would otherwise pick the link), leaves it unchanged.
template <class T>
__device__ __forceinline__ void maxretr(M3<T> &u, const M3<T> &Vb, int n_hits) {
    for (int hit = 0; hit < n_hits; ++hit) {
#pragma unroll
        for (int sgi = 0; sgi < 3; ++sgi) {
            const int p = sgi == 1 ? 1 : 0, q = sgi == 0 ? 1 : 2;
            // L_rc = sum_k u_rk conj(Vb_ck)
            T lr[2][2], li[2][2];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int rr = r ? q : p, cc = c ? q : p;
                    T sr = T(0), si = T(0);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        sr = fma(u.re[3 * rr + k], Vb.re[3 * cc + k], sr);
                        sr = fma(u.im[3 * rr + k], Vb.im[3 * cc + k], sr);
                        si = fma(u.im[3 * rr + k], Vb.re[3 * cc + k], si);
                        si = fma(-u.re[3 * rr + k], Vb.im[3 * cc + k], si);
                    }
                    lr[r][c] = sr;
                    li[r][c] = si;
                }
            const T ar = T(0.5) * (lr[0][0] + lr[1][1]), ai = T(0.5) * (li[0][0] - li[1][1]);
            const T br = T(0.5) * (lr[0][1] - lr[1][0]), bi = T(0.5) * (li[0][1] + li[1][0]);
            const T k2 = ar * ar + ai * ai + br * br + bi * bi;
            // singular subgroup (Sec. III.A): k <= 1e-6 of the block's scale
            const T sc2 = lr[0][0] * lr[0][0] + li[0][0] * li[0][0] + lr[1][1] * lr[1][1] + li[1][1] * li[1][1] +
                          lr[0][1] * lr[0][1] + li[0][1] * li[0][1] + lr[1][0] * lr[1][0] + li[1][0] * li[1][0];
            if (!(k2 > T(1e-12) * sc2)) continue;
            const T ik = T(1) / sqrt(k2);
            const T c00r = ar * ik, c00i = -ai * ik, c01r = -br * ik, c01i = -bi * ik;
            const T c10r = br * ik, c10i = -bi * ik, c11r = ar * ik, c11i = ai * ik;
#pragma unroll
            for (int col = 0; col < 3; ++col) {
                const T upr = u.re[3 * p + col], upi = u.im[3 * p + col];
                const T uqr = u.re[3 * q + col], uqi = u.im[3 * q + col];
                u.re[3 * p + col] = c00r * upr - c00i * upi + c01r * uqr - c01i * uqi;
                u.im[3 * p + col] = c00r * upi + c00i * upr + c01r * uqi + c01i * uqr;
                u.re[3 * q + col] = c10r * upr - c10i * upi + c11r * uqr - c11i * uqi;
                u.im[3 * q + col] = c10r * upi + c10i * upr + c11r * uqi + c11i * uqr;
            }
        }
    }
}

// AUS update of link (x, MU) at plane position i from its staple sum Vb and
// current value u: blocking V = (1 - alpha) u + (alpha / 6) Vb, MaxReTr,
// vortex-preservation test, store if accepted.
template <class T, int NC, int MU>
__device__ __forceinline__ void aus_finish(const AusParams &a, const Pt &x, int i, M3<T> Vb, M3<T> u,
                                           Update<T> &up) {
    const Geo &g = a.g;
    const T al = sizeof(T) == 4 ? T(a.alpha_f) : T(a.alpha);
    const T w6 = al / T(6), w1 = T(1) - al;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Vb.re[k] = fma(w1, u.re[k], w6 * Vb.re[k]);
        Vb.im[k] = fma(w1, u.im[k], w6 * Vb.im[k]);
    }
    maxretr<T>(u, Vb, a.n_hits);
    if (NC == 12) rebuild_row2(u);
    T tr_re, tr_im;
    vp_trace<T>(static_cast<const T *>(a.G), g.P, i, a.G ? sidx(g, mv(g, x, MU, 1)) : i, u, tr_re, tr_im);
    vp_decide<T>(a.vp, a.counters != nullptr, (int)a.ref[(long long)MU * g.P + i], tr_re, tr_im, up);
    if (!up.reject) store_link<T, NC>(static_cast<T *>(a.U), g.P, MU, i, u);
}

template <class T, int NC, bool RECT, int MU>
__global__ void __launch_bounds__(VS_SUBSWEEP_THREADS, sizeof(T) == 4 ? VS_SUBSWEEP_MINB : 1)
    k_aus(AusParams a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < a.n_threads;
    Update<T> up;
    if (active) {
        const Geo &g = a.g;
        const Pt x = class_site<MU>(g, a.colour, t);
        const int i = sidx(g, x);
        const T *U = static_cast<const T *>(a.U);
        const T c0 = sizeof(T) == 4 ? T(a.c0_f) : T(a.c0), c1 = sizeof(T) == 4 ? T(a.c1_f) : T(a.c1);
        const M3<T> Vb = staple_sum<T, NC, RECT, MU>(g, U, x, c0, c1);
        const M3<T> u = load_link<T, NC>(U, g.P, MU, i);
        aus_finish<T, NC, MU>(a, x, i, Vb, u, up);
    }
    count_update<T>(a.counters, up);
}

// FP32 over-improved AUS with the one-pass link stream of k_subsweep_fused.
template <int NC, int MU>
__global__ void __launch_bounds__(VS_RING_THREADS, VS_RING_MINB) k_aus_ring(AusParams a) {
    extern __shared__ float4 aus_dyn[];
    float4 *ring4 = aus_dyn;
    float2 *ring2 = reinterpret_cast<float2 *>(aus_dyn + 6 * (NC / 4) * VS_RING_THREADS);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < a.n_threads;
    Update<float> up;
    if (active) {
        const Geo &g = a.g;
        const Pt x = class_site<MU>(g, a.colour, t);
        const int i = sidx(g, x);
        LinkRing<NC> R = ring_of<NC>(ring4, ring2);
        M3<float> Ux;
        const M3<float> Vb = staple_sum_fused<NC, MU>(g, static_cast<const float *>(a.U), x, a.c0_f, a.c1_f, R, Ux);
        aus_finish<float, NC, MU>(a, x, i, Vb, Ux, up);
    }
    count_update<float>(a.counters, up);
}

// FP32 AUS + MaxReTr with plaquette staples (eps = 1; alpha = 1 is cooling)
// through the plaquette-staple ring.
template <int NC, int MU>
__global__ void __launch_bounds__(VS_RING_THREADS, 4) k_aus_pring(AusParams a) {
    extern __shared__ float4 ausp_dyn[];
    float4 *ring4 = ausp_dyn;
    float2 *ring2 = reinterpret_cast<float2 *>(ausp_dyn + 6 * (NC / 4) * VS_RING_THREADS);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < a.n_threads;
    Update<float> up;
    if (active) {
        const Geo &g = a.g;
        const Pt x = class_site<MU>(g, a.colour, t);
        const int i = sidx(g, x);
        const float *Us = static_cast<const float *>(a.U);
        LinkRing<NC> R = ring_of<NC>(ring4, ring2);
        const M3<float> Vb = staple_sum_plain_ring<NC, MU>(g, Us, x, a.c0_f, R);
        const M3<float> Ux = load_link<float, NC>(Us, g.P, MU, i);
        aus_finish<float, NC, MU>(a, x, i, Vb, Ux, up);
    }
    count_update<float>(a.counters, up);
}

}  // namespace vs
