// vs_stout.cuh -- staple sums, stout candidate and the colour-class update kernel.
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

#include "vs_internal.h"

namespace vs {

template <class T> struct Tol;
template <> struct Tol<float> { static __device__ __forceinline__ float eps() { return 1.5e-8f; } };
template <> struct Tol<double> { static __device__ __forceinline__ double eps() { return 1e-17; } };

// Step of a lattice path from site p: s > 0 -> U_d(p); s < 0 -> U_d(p - d)^dag.
template <class T, int NC>
__device__ __forceinline__ M3<T> path_step(const Geo &g, const T *__restrict__ U, Pt p, int d, int s) {
    if (s > 0) return load_link<T, NC>(U, g.P, d, sidx(g, p));
    return m3_dag(load_link<T, NC>(U, g.P, d, sidx(g, mv(g, p, d, -1))));
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
template <class T, int NC, bool RECT, int MU>
__device__ __forceinline__ M3<T> staple_sum(const Geo &g, const T *__restrict__ U, Pt x, T c0, T c1) {
    M3<T> sig;
    if (RECT) {
        {
            M3<T> F;
            m3_zero(F);
#pragma unroll 1
            for (int j = 1; j < 4; ++j) {
                const int nu = (MU + j) & 3;
#pragma unroll
                for (int s = 1; s >= -1; s -= 2) {
                    Pt xs = mv(g, x, nu, s), xsm = mv(g, xs, MU, 1);
                    M3<T> W = m3_mul(path_step<T, NC>(g, U, x, nu, s),
                                     load_link<T, NC>(U, g.P, MU, sidx(g, xs)));
                    W = m3_mul(W, load_link<T, NC>(U, g.P, MU, sidx(g, xsm)));
                    m3_madd(F, W, path_step<T, NC>(g, U, mv(g, xsm, MU, 1), nu, -s));
                }
            }
            sig = m3_mul_nd(F, load_link<T, NC>(U, g.P, MU, sidx(g, mv(g, x, MU, 1))));
            m3_scale(sig, c1);
        }
        {
            M3<T> Bk;
            m3_zero(Bk);
            const Pt xm = mv(g, x, MU, -1);
#pragma unroll 1
            for (int j = 1; j < 4; ++j) {
                const int nu = (MU + j) & 3;
#pragma unroll
                for (int s = 1; s >= -1; s -= 2) {
                    Pt xs = mv(g, x, nu, s), xsm = mv(g, xs, MU, 1);
                    M3<T> BC = m3_mul(load_link<T, NC>(U, g.P, MU, sidx(g, xs)),
                                      path_step<T, NC>(g, U, xsm, nu, -s));
                    M3<T> Y = m3_mul(path_step<T, NC>(g, U, xm, nu, s),
                                     load_link<T, NC>(U, g.P, MU, sidx(g, mv(g, xm, nu, s))));
                    m3_madd(Bk, Y, BC);
                }
            }
            M3<T> t = m3_mul_dn(load_link<T, NC>(U, g.P, MU, sidx(g, xm)), Bk);
            m3_axpy(sig, c1, t);
        }
#pragma unroll 1
        for (int j = 1; j < 4; ++j) {
            const int nu = (MU + j) & 3;
#pragma unroll
            for (int s = 1; s >= -1; s -= 2) {
                Pt xs = mv(g, x, nu, s), xsm = mv(g, xs, MU, 1), x2s = mv(g, xs, nu, s);
                M3<T> Tt = m3_mul(path_step<T, NC>(g, U, xs, nu, s),
                                  load_link<T, NC>(U, g.P, MU, sidx(g, x2s)));
                Tt = m3_mul(Tt, path_step<T, NC>(g, U, mv(g, x2s, MU, 1), nu, -s));
                M3<T> N = load_link<T, NC>(U, g.P, MU, sidx(g, xs));
#pragma unroll
                for (int k = 0; k < 9; ++k) {
                    N.re[k] = fma(c1, Tt.re[k], c0 * N.re[k]);
                    N.im[k] = fma(c1, Tt.im[k], c0 * N.im[k]);
                }
                M3<T> AN = m3_mul(path_step<T, NC>(g, U, x, nu, s), N);
                m3_madd(sig, AN, path_step<T, NC>(g, U, xsm, nu, -s));
            }
        }
    } else {
        m3_zero(sig);
#pragma unroll
        for (int j = 1; j < 4; ++j) {
            const int nu = (MU + j) & 3;
#pragma unroll
            for (int s = 1; s >= -1; s -= 2) {
                Pt xs = mv(g, x, nu, s), xsm = mv(g, xs, MU, 1);
                M3<T> AB = m3_mul(path_step<T, NC>(g, U, x, nu, s),
                                  load_link<T, NC>(U, g.P, MU, sidx(g, xs)));
                m3_madd(sig, AB, path_step<T, NC>(g, U, xsm, nu, -s));
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
            ch_exp_coeffs<double, 12>(h00, h11, h22, h01r, h01i, h02r, h02i, h12r, h12i, 1e300, fd);
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
    M3<T> H2 = m3_mul(H, H);
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

// Candidate U' = exp(rho Q) U for staple sum sig.
template <class T>
__device__ __forceinline__ M3<T> stout_candidate(const M3<T> &sig, const M3<T> &Ux, T rho, bool &fp64_used) {
    M3<T> Om = m3_mul_nd(sig, Ux);
    // H = -i rho Q: diagonal rho (Im Om_jj - (1/3) sum_l Im Om_ll), written so
    // that equal diagonal entries give exactly zero; off-diagonal
    // H_jk = (rho/2) [(Im Om_jk + Im Om_kj) - i (Re Om_jk - Re Om_kj)].
    const T third = T(1) / T(3);
    const T h00 = rho * ((T(2) * Om.im[0] - Om.im[4] - Om.im[8]) * third);
    const T h11 = rho * ((T(2) * Om.im[4] - Om.im[0] - Om.im[8]) * third);
    const T h22 = rho * ((T(2) * Om.im[8] - Om.im[0] - Om.im[4]) * third);
    const T hr = T(0.5) * rho;
    const T h01r = hr * (Om.im[1] + Om.im[3]), h01i = -hr * (Om.re[1] - Om.re[3]);
    const T h02r = hr * (Om.im[2] + Om.im[6]), h02i = -hr * (Om.re[2] - Om.re[6]);
    const T h12r = hr * (Om.im[5] + Om.im[7]), h12i = -hr * (Om.re[5] - Om.re[7]);
    M3<T> Mx = exp_iH<T>(h00, h11, h22, h01r, h01i, h02r, h02i, h12r, h12i, fp64_used);
    return m3_mul(Mx, Ux);
}

#ifndef VS_SUBSWEEP_MINB
#define VS_SUBSWEEP_MINB 4
#endif

// One thread per link of the colour class (or of direction MU when colour < 0).
// FP32: at most 65536 / (128 * VS_SUBSWEEP_MINB) registers per thread, so
// VS_SUBSWEEP_MINB blocks of 128 threads fit on an SM.
template <class T, int NC, bool RECT, int MU>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? VS_SUBSWEEP_MINB : 1) k_subsweep(SubsweepParams a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < a.n_threads;
    bool reject = false, used64 = false;
    if (active) {
        const Geo &g = a.g;
        Pt x = a.colour >= 0 ? class_site<MU>(g, a.colour, t) : site_of_index(g, t);
        const int i = sidx(g, x);
        const T *Us = static_cast<const T *>(a.Usrc);
        M3<T> sig = staple_sum<T, NC, RECT, MU>(g, Us, x, T(a.c0), T(a.c1));
        M3<T> Ux = load_link<T, NC>(Us, g.P, MU, i);
        M3<T> Un = stout_candidate<T>(sig, Ux, T(a.rho), used64);
        if (a.vp) {
            T tr_re = Un.re[0] + Un.re[4] + Un.re[8];
            T tr_im = Un.im[0] + Un.im[4] + Un.im[8];
            reject = z3_label<T>(tr_re, tr_im) != (int)a.ref[(long long)MU * g.P + i];
        }
        if (!reject) store_link<T, NC>(static_cast<T *>(a.U), g.P, MU, i, Un);
    }
    if (a.counters) {
        unsigned rb = __ballot_sync(0xffffffffu, reject);
        unsigned fb = __ballot_sync(0xffffffffu, used64);
        if ((threadIdx.x & 31) == 0) {
            if (rb) atomicAdd(&a.counters[0], (unsigned long long)__popc(rb));
            if (fb) atomicAdd(&a.counters[1], (unsigned long long)__popc(fb));
        }
    }
}

}  // namespace vs
