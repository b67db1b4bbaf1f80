// vs_kernels.cu -- load/read conversions, centrifuge, action, vortex check,
// re-unitarisation, hot-start generation and the exponential diagnostic.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "vs_internal.h"
#include "vs_stout.cuh"

namespace vs {

namespace {

constexpr int kThreads = 256;

inline int nblocks(long long n, int threads = kThreads) { return (int)((n + threads - 1) / threads); }
// grid of the grid-stride kernels that first build a per-block table
constexpr int kTableGrid = 2048;

// ---------------------------------------------------------------------------
// Load / read
// ---------------------------------------------------------------------------

// Z_mu(x) = exp(2 pi i n / 3) I, Sec. I Eq. (centre_project).  One thread per link.
template <class T, int NC>
__global__ void __launch_bounds__(kThreads) k_load_labels(Geo g, const int8_t *__restrict__ lab, T *U, int8_t *ref) {
    // e^{2 pi i n / 3} for n = -1, 0, 1, three sincospi per block instead of one
    // per link (the FP64 sincospi made this kernel FP64-bound); labels outside
    // {-1, 0, 1} (possible only from device input) take the direct evaluation.
    __shared__ double zc[3], zs[3];
    if (threadIdx.x < 3) sincospi(2.0 * ((int)threadIdx.x - 1) / 3.0, &zs[threadIdx.x], &zc[threadIdx.x]);
    __syncthreads();
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < 4ll * g.V;
         l += (long long)gridDim.x * blockDim.x) {
        int mu = (int)(l / g.V), s = (int)(l % g.V);
        int n = lab[l];
        Pt p = site_of_lex(g, s);
        int i = sidx(g, p);
        double sn, cs;
        if (n >= -1 && n <= 1) {
            sn = zs[n + 1];
            cs = zc[n + 1];
        } else {
            sincospi(2.0 * n / 3.0, &sn, &cs);
        }
        M3<T> z;
        m3_zero(z);
        z.re[0] = z.re[4] = z.re[8] = T(cs);
        z.im[0] = z.im[4] = z.im[8] = T(sn);
        store_link<T, NC>(U, g.P, mu, i, z);
        ref[(long long)mu * g.P + i] = (int8_t)n;
    }
}

// Links from FP64 host layout; the reference label is the sector of arg Tr U of the FP64 input.
template <class T, int NC>
__global__ void k_load_links(Geo g, const double *__restrict__ in, T *U, int8_t *ref) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4ll * g.V) return;
    int mu = (int)(l / g.V), s = (int)(l % g.V);
    Pt p = site_of_lex(g, s);
    int i = sidx(g, p);
    const double *q = in + l * 18;
    M3<T> m;
    double tr = 0, ti = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        m.re[k] = T(q[2 * k]);
        m.im[k] = T(q[2 * k + 1]);
    }
    tr = q[0] + q[8] + q[16];
    ti = q[1] + q[9] + q[17];
    store_link<T, NC>(U, g.P, mu, i, m);
    ref[(long long)mu * g.P + i] = (int8_t)z3_label<double>(tr, ti);
}

template <class T, int NC>
__global__ void k_read_links(Geo g, const T *__restrict__ U, double *out) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4ll * g.V) return;
    int mu = (int)(l / g.V), s = (int)(l % g.V);
    Pt p = site_of_lex(g, s);
    M3<T> m = load_link<T, NC>(U, g.P, mu, sidx(g, p));
    double *q = out + l * 18;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        q[2 * k] = double(m.re[k]);
        q[2 * k + 1] = double(m.im[k]);
    }
}

__global__ void k_read_labels(Geo g, const int8_t *__restrict__ ref, int8_t *out) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4ll * g.V) return;
    int mu = (int)(l / g.V), s = (int)(l % g.V);
    out[l] = ref[(long long)mu * g.P + sidx(g, site_of_lex(g, s))];
}

// Links with a non-finite entry (NaN or Inf), one thread per link.
template <class T, int NC>
__global__ void k_count_nonfinite(Geo g, const T *__restrict__ U, unsigned long long *count) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (l < 4ll * g.V) {
        const M3<T> m = load_link<T, NC>(U, g.P, (int)(l / g.V), sidx(g, site_of_index(g, (int)(l % g.V))));
#pragma unroll
        for (int k = 0; k < 9; ++k) bad |= !isfinite(m.re[k]) || !isfinite(m.im[k]);
    }
    const unsigned b = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, (unsigned long long)__popc(b));
}

// reference labels from lexicographic order into plane order (restore)
__global__ void k_store_ref(Geo g, const int8_t *__restrict__ lab, int8_t *ref) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4ll * g.V) return;
    int mu = (int)(l / g.V), s = (int)(l % g.V);
    ref[(long long)mu * g.P + sidx(g, site_of_lex(g, s))] = lab[l];
}

template <class T, int NC>
__global__ void k_current_labels(Geo g, const T *__restrict__ U, int8_t *out) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4ll * g.V) return;
    int mu = (int)(l / g.V), s = (int)(l % g.V);
    M3<T> m = load_link<T, NC>(U, g.P, mu, sidx(g, site_of_lex(g, s)));
    out[l] = (int8_t)z3_label<T>(m.re[0] + m.re[4] + m.re[8], m.im[0] + m.im[4] + m.im[8]);
}

// ---------------------------------------------------------------------------
// Centrifuge preconditioning, Sec. IV
// ---------------------------------------------------------------------------

// m = sum_{nu != mu} [n_nu(x) + n_mu(x+nu) - n_nu(x+mu) - n_nu(x-nu) + n_mu(x-nu)
// + n_nu(x-nu+mu)] so that sigma = m 2 pi / 18; delta = omega (sigma - lambda)
// = omega pi (m - 6n) / 9.  Pair p = SplitMix64(seed, mu V + s) mod 3 picks
// (j,k) = (0,1), (1,2), (2,0): phase j gets lambda + delta, phase k lambda - delta.
// The phases take few values: pi (2n/3 + s omega k/9) with n in {-1, 0, 1},
// k = m - 6n in [-24, 24], s = +-1 (k = 0 is the untouched phase 2n/3).  Each
// block evaluates them once into shared memory with the same FP64 expressions
// as the per-link form, so the links are bit-identical to it; values outside
// the table (labels outside {-1, 0, 1}, only from device input) are evaluated
// directly.
constexpr int kCtabK = 24, kCtabN = 3 * (2 * kCtabK + 1) * 2;

__device__ __forceinline__ double centrifuge_phase(double omega, int n, int k, bool neg) {
    const double delta = omega * (double)k / 9.0;   // in units of pi
    const double ph = 2.0 * n / 3.0;
    return neg ? ph - delta : ph + delta;
}

template <class T, int NC>
__global__ void __launch_bounds__(kThreads) k_centrifuge(Geo g, const int8_t *__restrict__ ref, double omega,
                                                          uint64_t seed, T *U) {
    __shared__ double2 tab[kCtabN];   // (cos, sin) at ((n + 1)(2K + 1) + k + K) * 2 + neg
    for (int e = threadIdx.x; e < kCtabN; e += blockDim.x) {
        const int q = e >> 1;
        double sn, cs;
        sincospi(centrifuge_phase(omega, q / (2 * kCtabK + 1) - 1, q % (2 * kCtabK + 1) - kCtabK, e & 1), &sn, &cs);
        tab[e] = make_double2(cs, sn);
    }
    __syncthreads();
    for (long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x; l < 4ll * g.V;
         l += (long long)gridDim.x * blockDim.x) {
        int mu = (int)(l / g.V), s = (int)(l % g.V);
        Pt x = site_of_lex(g, s);
        auto lab = [&](int d, const Pt &p) { return (int)ref[(long long)d * g.P + sidx(g, p)]; };
        int m = 0;
#pragma unroll
        for (int j = 1; j < 4; ++j) {
            int nu = (mu + j) & 3;
            Pt xpn = mv(g, x, nu, 1), xpm = mv(g, x, mu, 1), xmn = mv(g, x, nu, -1);
            Pt xmnpm = mv(g, xmn, mu, 1);
            m += lab(nu, x) + lab(mu, xpn) - lab(nu, xpm) - lab(nu, xmn) + lab(mu, xmn) + lab(nu, xmnpm);
        }
        const int n = lab(mu, x), k = m - 6 * n;
        int pair = (int)(splitmix64(seed, (uint64_t)mu * (uint64_t)g.V + (uint64_t)s) % 3ull);
        int jj = pair, kk = (pair + 1) % 3;
        M3<T> z;
        m3_zero(z);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int kc = c == jj ? k : c == kk ? k : 0;
            const bool neg = c == kk;
            double2 v;
            if (n >= -1 && n <= 1 && kc >= -kCtabK && kc <= kCtabK) {
                v = tab[((n + 1) * (2 * kCtabK + 1) + kc + kCtabK) * 2 + neg];
            } else {
                sincospi(centrifuge_phase(omega, n, kc, neg), &v.y, &v.x);
            }
            z.re[4 * c] = T(v.x);
            z.im[4 * c] = T(v.y);
        }
        store_link<T, NC>(U, g.P, mu, sidx(g, x), z);
    }
}

// ---------------------------------------------------------------------------
// Wilson action, Sec. V: sum_x sum_{mu<nu} (3 - Re Tr P_munu(x)); each
// plaquette in the storage precision, the sums in FP64 in a fixed order
// (block tree, then one block over the partials).
// ---------------------------------------------------------------------------

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (ln == 0) sh[w] = v;
    __syncthreads();
    v = 0;
    if (w == 0) {
        int nw = blockDim.x >> 5;
        v = ln < nw ? sh[ln] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}

template <class T, int NC>
__global__ void __launch_bounds__(kThreads) k_action(Geo g, const T *__restrict__ U, double *partials) {
    double acc = 0;
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < g.V; d += gridDim.x * blockDim.x) {
        const Pt x = site_of_index(g, d);
        const int i = sidx(g, x);
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            M3<T> Umu = load_link<T, NC>(U, g.P, mu, i);
            Pt xm = mv(g, x, mu, 1);
#pragma unroll
            for (int nu = mu + 1; nu < 4; ++nu) {
                Pt xn = mv(g, x, nu, 1);
                // P = (U_mu(x) U_nu(x+mu)) (U_nu(x) U_mu(x+nu))^dag
                M3<T> X = m3_mul(Umu, load_link<T, NC>(U, g.P, nu, sidx(g, xm)));
                M3<T> Y = m3_mul(load_link<T, NC>(U, g.P, nu, i), load_link<T, NC>(U, g.P, mu, sidx(g, xn)));
                // Re Tr(X Y^dag) in the storage precision: the FP32 products
                // already carry FP32 rounding, and an FP64 dot (18 conversions
                // and FMAs on the slow FP64 pipe) made this kernel FP64-bound
                T re = T(0);
#pragma unroll
                for (int k = 0; k < 9; ++k) re = fma(X.re[k], Y.re[k], fma(X.im[k], Y.im[k], re));
                acc += 3.0 - (double)re;
            }
        }
    }
    double b = block_sum(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = b;
}

// ---------------------------------------------------------------------------
// Smoothness observables, Sec. V: clover F_munu (the mean of the four leaves of
// the plane at x, F = (C - C^dag)/(2i), traceless), per site
//   S(x)/beta   = 1/72 sum_{mu != nu} Re Tr(1 - P_munu)
//   S_R(x)/beta = 1/72 sum_{mu != nu} Tr(F_munu^2) / 2
//   q(x)        = [Tr(F01 F23) - Tr(F02 F13) + Tr(F03 F12)] / (4 pi^2)
// (the eps-sum of Eq. 1LTopQ collapsed to its three pairings x 8 / (32 pi^2)).
// ---------------------------------------------------------------------------

template <class T, int NC>
__device__ __forceinline__ M3<T> clover_F(const Geo &g, const T *__restrict__ U, const Pt &x, int i, int mu,
                                          int nu, T &plaq_retr) {
    const Pt xpm = mv(g, x, mu, 1), xpn = mv(g, x, nu, 1), xmm = mv(g, x, mu, -1), xmn = mv(g, x, nu, -1);
    const int ipm = sidx(g, xpm), ipn = sidx(g, xpn), imm = sidx(g, xmm), imn = sidx(g, xmn);
    const int ipnmm = sidx(g, mv(g, xpn, mu, -1)), immmn = sidx(g, mv(g, xmm, nu, -1));
    const int imnpm = sidx(g, mv(g, xmn, mu, 1));
    M3<T> C, L;
    // leaf 1: +mu +nu -mu -nu
    L = m3_mul(load_link<T, NC>(U, g.P, mu, i), load_link<T, NC>(U, g.P, nu, ipm));
    L = m3_mul_nd(L, load_link<T, NC>(U, g.P, mu, ipn));
    L = m3_mul_nd(L, load_link<T, NC>(U, g.P, nu, i));
    plaq_retr = L.re[0] + L.re[4] + L.re[8];
    C = L;
    // leaf 2: +nu -mu -nu +mu
    L = m3_mul_nd(load_link<T, NC>(U, g.P, nu, i), load_link<T, NC>(U, g.P, mu, ipnmm));
    L = m3_mul_nd(L, load_link<T, NC>(U, g.P, nu, imm));
    m3_madd(C, L, load_link<T, NC>(U, g.P, mu, imm));
    // leaf 3: -mu -nu +mu +nu
    L = m3_mul_dn(load_link<T, NC>(U, g.P, mu, imm), m3_dag(load_link<T, NC>(U, g.P, nu, immmn)));
    L = m3_mul(L, load_link<T, NC>(U, g.P, mu, immmn));
    m3_madd(C, L, load_link<T, NC>(U, g.P, nu, imn));
    // leaf 4: -nu +mu +nu -mu
    L = m3_mul_dn(load_link<T, NC>(U, g.P, nu, imn), load_link<T, NC>(U, g.P, mu, imn));
    L = m3_mul(L, load_link<T, NC>(U, g.P, nu, imnpm));
    L = m3_mul_nd(L, load_link<T, NC>(U, g.P, mu, i));
    for (int k = 0; k < 9; ++k) { C.re[k] += L.re[k]; C.im[k] += L.im[k]; }
    // F = (C - C^dag) / (2i) / 4, traceless
    M3<T> F;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const T dr = C.re[3 * j + k] - C.re[3 * k + j], di = C.im[3 * j + k] + C.im[3 * k + j];
            F.re[3 * j + k] = T(0.125) * di;
            F.im[3 * j + k] = -T(0.125) * dr;
        }
    const T tr = (F.re[0] + F.re[4] + F.re[8]) / T(3);
    F.re[0] -= tr;
    F.re[4] -= tr;
    F.re[8] -= tr;
    return F;
}

// Tr(A B) for Hermitian A, B: sum_jk A_jk conj(B_jk), real, in the storage
// precision (its FP32 inputs already carry FP32 rounding; an FP64 dot made the
// kernel FP64-bound); the sums over sites run in FP64.
template <class T>
__device__ __forceinline__ T tr_herm(const M3<T> &A, const M3<T> &B) {
    T s = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) s += A.re[k] * B.re[k] + A.im[k] * B.im[k];
    return s;
}

template <class T, int NC>
__global__ void __launch_bounds__(kThreads) k_observables(Geo g, const T *__restrict__ U, double *partials,
                                                           double *S_site, double *SR_site, double *q_site) {
    double aS = 0, aSR = 0, aQ = 0;
    const int pairs[3][4] = {{0, 1, 2, 3}, {0, 2, 1, 3}, {0, 3, 1, 2}};
    const double sgn[3] = {1.0, -1.0, 1.0};
    for (int d = blockIdx.x * blockDim.x + threadIdx.x; d < g.V; d += gridDim.x * blockDim.x) {
        const Pt x = site_of_index(g, d);
        const int i = sidx(g, x);
        double s = 0, sr = 0, q = 0;
        for (int pp = 0; pp < 3; ++pp) {
            T r1, r2;
            const M3<T> Fa = clover_F<T, NC>(g, U, x, i, pairs[pp][0], pairs[pp][1], r1);
            const M3<T> Fb = clover_F<T, NC>(g, U, x, i, pairs[pp][2], pairs[pp][3], r2);
            s += (3.0 - (double)r1) + (3.0 - (double)r2);
            sr += (double)tr_herm(Fa, Fa) + (double)tr_herm(Fb, Fb);
            q += sgn[pp] * (double)tr_herm(Fa, Fb);
        }
        s *= 2.0 / 72.0;
        sr /= 72.0;
        q /= 4.0 * 9.869604401089358;
        const int lx = lexidx(g, x);
        if (S_site) S_site[lx] = s;
        if (SR_site) SR_site[lx] = sr;
        if (q_site) q_site[lx] = q;
        aS += s;
        aSR += sr;
        aQ += q;
    }
    const double b0 = block_sum(aS), b1 = block_sum(aSR), b2 = block_sum(aQ);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = b0;
        partials[3 * blockIdx.x + 1] = b1;
        partials[3 * blockIdx.x + 2] = b2;
    }
}

__global__ void k_sum_partials3(const double *__restrict__ partials, int n, double invV, double *out) {
    for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[3 * i + c];
        const double b = block_sum(acc);
        if (threadIdx.x == 0) out[c] = c < 2 ? b * invV : b;
    }
}

__global__ void k_sum_partials(const double *__restrict__ partials, int n, double scale, double *out) {
    double acc = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
    double b = block_sum(acc);
    if (threadIdx.x == 0) *out = b * scale;
}

// ---------------------------------------------------------------------------
// Correlation of two densities, Sec. VII Eq. (correlation_s):
//   C = <a b> / (sqrt<a^2> sqrt<b^2>)
// three FP64 sums in a fixed order (grid-stride loop over a fixed grid, block
// tree, then one block over the partials), so the result is bit-reproducible.
// ---------------------------------------------------------------------------

constexpr int kCorrGrid = 400;

__global__ void __launch_bounds__(kThreads) k_correlation(const double *__restrict__ a, const double *__restrict__ b,
                                                          long long n, double *partials) {
    double sab = 0, saa = 0, sbb = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = a[i], y = b[i];
        sab = fma(x, y, sab);
        saa = fma(x, x, saa);
        sbb = fma(y, y, sbb);
    }
    sab = block_sum(sab);
    saa = block_sum(saa);
    sbb = block_sum(sbb);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x] = sab;
        partials[3 * blockIdx.x + 1] = saa;
        partials[3 * blockIdx.x + 2] = sbb;
    }
}

// out[0] = C, out[1..3] = the three sums (a zero norm leaves C = NaN)
__global__ void k_correlation_finish(const double *__restrict__ partials, int nb, double *out) {
    double s[3];
    for (int c = 0; c < 3; ++c) {
        double acc = 0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partials[3 * i + c];
        s[c] = block_sum(acc);
    }
    if (threadIdx.x == 0) {
        out[1] = s[0];
        out[2] = s[1];
        out[3] = s[2];
        // the means' 1/n cancels between numerator and denominator
        out[0] = (s[1] > 0 && s[2] > 0) ? s[0] / (sqrt(s[1]) * sqrt(s[2])) : __longlong_as_double(0x7ff8000000000000ll);
    }
}

// ---------------------------------------------------------------------------
// Vortex check
// ---------------------------------------------------------------------------

__device__ __forceinline__ void count_warp(unsigned long long *ctr, bool pred) {
    unsigned b = __ballot_sync(0xffffffffu, pred);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(ctr, (unsigned long long)__popc(b));
}

template <class T, int NC>
__global__ void k_vortex_links(Geo g, const T *__restrict__ U, const int8_t *__restrict__ ref,
                               int8_t *cur, unsigned long long *counts, unsigned long long *mbits,
                               const T *__restrict__ G) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    bool diff = false, near = false;
    double margin = 1e300;
    if (l < 4ll * g.V) {
        const int mu = (int)(l / g.V);
        const Pt x = site_of_index(g, (int)(l % g.V));
        const int i = sidx(g, x);
        M3<T> m = load_link<T, NC>(U, g.P, mu, i);
        T a, b;
        vp_trace<T>(G, g.P, i, G ? sidx(g, mv(g, x, mu, 1)) : i, m, a, b);
        int lab = z3_label<T>(a, b);
        cur[(long long)mu * g.P + i] = (int8_t)lab;
        diff = lab != ref[(long long)mu * g.P + i];
        // angular distance of arg Tr U from the nearest sector edge (+-pi/3,
        // pi), in the field's precision: an FP32 trace is itself rounded to
        // ~1e-7, and an FP64 atan2 per link made this kernel FP64-bound
        if constexpr (sizeof(T) == 4) {
            const float argf = atan2f(b + 0.0f, a);
            const float pi3f = 1.04719755f;
            margin = (double)fminf(fminf(fabsf(argf - pi3f), fabsf(argf + pi3f)), 3.14159265f - fabsf(argf));
        } else {
            double arg = atan2((double)b + 0.0, (double)a);
            const double pi3 = 1.0471975511965976;
            margin = fmin(fmin(fabs(arg - pi3), fabs(arg + pi3)), 3.141592653589793 - fabs(arg));
        }
        near = margin < 1e-5;
    }
    count_warp(&counts[0], diff);
    count_warp(&counts[2], near);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) margin = fmin(margin, __shfl_xor_sync(0xffffffffu, margin, o));
    if ((threadIdx.x & 31) == 0 && margin < 1e300)
        atomicMin(mbits, (unsigned long long)__double_as_longlong(margin));
}

// centre charge p = n_mu(x) + n_nu(x+mu) - n_mu(x+nu) - n_nu(x) mod 3 in {-1,0,1}
__device__ __forceinline__ int charge(const Geo &g, const int8_t *lab, const Pt &x, int i, int mu, int nu) {
    int p = lab[(long long)mu * g.P + i] + lab[(long long)nu * g.P + sidx(g, mv(g, x, mu, 1))]
          - lab[(long long)mu * g.P + sidx(g, mv(g, x, nu, 1))] - lab[(long long)nu * g.P + i];
    p = ((p % 3) + 3) % 3;
    return p == 2 ? -1 : p;
}

__global__ void k_vortex_charges(Geo g, const int8_t *__restrict__ ref, const int8_t *__restrict__ cur,
                                 unsigned long long *counts) {
    const int dn = blockIdx.x * blockDim.x + threadIdx.x;
    int nd = 0;
    if (dn < g.V) {
        const Pt x = site_of_index(g, dn);
        const int i = sidx(g, x);
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu)
                nd += charge(g, cur, x, i, mu, nu) != charge(g, ref, x, i, mu, nu);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nd += __shfl_xor_sync(0xffffffffu, nd, o);
    if ((threadIdx.x & 31) == 0 && nd) atomicAdd(&counts[1], (unsigned long long)nd);
}

// ---------------------------------------------------------------------------
// Re-unitarisation: r0 /= |r0|; r1 -= (r0^dag r1) r0; r1 /= |r1|;
// r2 = conj(r0 x r1), all in the storage precision.  For FP32 links the
// result is unitary to the rounding of the stored rows (a few 1e-7), the
// level the FP32 sweeps themselves leave; FP64 norms would buy nothing
// measurable and make the kernel FP64-bound (GB300's FP64 pipe runs at
// 1/64 of FP32) instead of HBM-bound.
// With ref != nullptr (vortex preservation on) a re-unitarised link whose
// Z(3) label would differ from the reference is left as it was, so every
// stored link keeps its original label.
// ---------------------------------------------------------------------------

template <class T, int NC>
__global__ void k_reunit(Geo g, T *U, const int8_t *__restrict__ ref, const T *__restrict__ G) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4ll * g.V) return;
    const int mu = (int)(l / g.V);
    const Pt x = site_of_index(g, (int)(l % g.V));
    const int i = sidx(g, x);
    M3<T> m = load_link<T, NC>(U, g.P, mu, i);
    T n0 = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) n0 = fma(m.re[b], m.re[b], fma(m.im[b], m.im[b], n0));
    const T s0 = T(1) / sqrt(n0);
#pragma unroll
    for (int b = 0; b < 3; ++b) { m.re[b] *= s0; m.im[b] *= s0; }
    T pr = T(0), pi = T(0);  // r0^dag r1
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        pr = fma(m.re[b], m.re[3 + b], fma(m.im[b], m.im[3 + b], pr));
        pi = fma(m.re[b], m.im[3 + b], fma(-m.im[b], m.re[3 + b], pi));
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        m.re[3 + b] -= pr * m.re[b] - pi * m.im[b];
        m.im[3 + b] -= pr * m.im[b] + pi * m.re[b];
    }
    T n1 = T(0);
#pragma unroll
    for (int b = 0; b < 3; ++b) n1 = fma(m.re[3 + b], m.re[3 + b], fma(m.im[3 + b], m.im[3 + b], n1));
    const T s1 = T(1) / sqrt(n1);
#pragma unroll
    for (int b = 0; b < 3; ++b) { m.re[3 + b] *= s1; m.im[3 + b] *= s1; }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        T cr = m.re[j1] * m.re[3 + j2] - m.im[j1] * m.im[3 + j2] - (m.re[j2] * m.re[3 + j1] - m.im[j2] * m.im[3 + j1]);
        T ci = m.re[j1] * m.im[3 + j2] + m.im[j1] * m.re[3 + j2] - (m.re[j2] * m.im[3 + j1] + m.im[j2] * m.re[3 + j1]);
        m.re[6 + j] = cr;
        m.im[6 + j] = -ci;
    }
    if (ref) {
        T a, b;
        vp_trace<T>(G, g.P, i, G ? sidx(g, mv(g, x, mu, 1)) : i, m, a, b);
        if (z3_label<T>(a, b) != (int)ref[(long long)mu * g.P + i]) return;
    }
    store_link<T, NC>(U, g.P, mu, i, m);
}

// ---------------------------------------------------------------------------
// Exponential diagnostic: E = exp(X), X traceless anti-Hermitian, via H = -iX
// ---------------------------------------------------------------------------

template <class T>
__global__ void k_debug_expm(const double *__restrict__ X, int n, double *E) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const double *x = X + 18ll * t;
    // H_jk = -i X_jk -> re = Im X_jk, im = -Re X_jk
    auto hre = [&](int j, int k) { return T(x[2 * (3 * j + k) + 1]); };
    auto him = [&](int j, int k) { return T(-x[2 * (3 * j + k)]); };
    bool f64;
    M3<T> M = exp_iH<T>(hre(0, 0), hre(1, 1), hre(2, 2), hre(0, 1), him(0, 1), hre(0, 2), him(0, 2),
                        hre(1, 2), him(1, 2), f64);
    double *e = E + 18ll * t;
    for (int k = 0; k < 9; ++k) { e[2 * k] = double(M.re[k]); e[2 * k + 1] = double(M.im[k]); }
}

// ---------------------------------------------------------------------------
// Hot start and MaxReTr cooling (input generation)
// ---------------------------------------------------------------------------

// Haar SU(3) per link: 18 Gaussians by Box-Muller from SplitMix64 values
// 18 l .. 18 l + 17 of `seed` (pair k: radius from value 2k, angle from 2k+1),
// Z_jk = (g_{2(3j+k)} + i g_{2(3j+k)+1}) / sqrt 2, Gram-Schmidt on the columns
// (QR with positive diag R: Haar U(3), Mezzadri 2007), then divide by the
// principal cube root of det.
template <class T, int NC>
__global__ void k_haar(Geo g, uint64_t seed, T *U) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4ll * g.V) return;
    int mu = (int)(l / g.V), s = (int)(l % g.V);
    double zr[9], zi[9];
    const double inv53 = 1.0 / 9007199254740992.0;
    for (int k = 0; k < 9; ++k) {
        uint64_t c = (uint64_t)l * 18ull + 2ull * k;
        double u1 = 1.0 - (double)(splitmix64(seed, c) >> 11) * inv53;
        double u2 = (double)(splitmix64(seed, c + 1) >> 11) * inv53;
        double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        zr[k] = rad * cs * 0.7071067811865476;
        zi[k] = rad * sn * 0.7071067811865476;
    }
    // Gram-Schmidt on columns c = 0, 1, 2 (entries (j, c) at index 3j + c)
    for (int c = 0; c < 3; ++c) {
        for (int p = 0; p < c; ++p) {
            double pr = 0, pi = 0;  // <q_p, z_c> = sum conj(q_jp) z_jc
            for (int j = 0; j < 3; ++j) {
                pr += zr[3 * j + p] * zr[3 * j + c] + zi[3 * j + p] * zi[3 * j + c];
                pi += zr[3 * j + p] * zi[3 * j + c] - zi[3 * j + p] * zr[3 * j + c];
            }
            for (int j = 0; j < 3; ++j) {
                zr[3 * j + c] -= pr * zr[3 * j + p] - pi * zi[3 * j + p];
                zi[3 * j + c] -= pr * zi[3 * j + p] + pi * zr[3 * j + p];
            }
        }
        double nn = 0;
        for (int j = 0; j < 3; ++j) nn += zr[3 * j + c] * zr[3 * j + c] + zi[3 * j + c] * zi[3 * j + c];
        nn = 1.0 / sqrt(nn);
        for (int j = 0; j < 3; ++j) { zr[3 * j + c] *= nn; zi[3 * j + c] *= nn; }
    }
    // det by expansion along row 0
    auto cm = [](double ar, double ai, double br, double bi, double &rr, double &ri) {
        rr = ar * br - ai * bi; ri = ar * bi + ai * br;
    };
    double dr = 0, di = 0;
    for (int k = 0; k < 3; ++k) {
        int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        double pr, pi, qr, qi, mr, mi;
        cm(zr[3 + k1], zi[3 + k1], zr[6 + k2], zi[6 + k2], pr, pi);
        cm(zr[3 + k2], zi[3 + k2], zr[6 + k1], zi[6 + k1], qr, qi);
        cm(zr[k], zi[k], pr - qr, pi - qi, mr, mi);
        dr += mr; di += mi;
    }
    double ph = atan2(di, dr) / 3.0;
    double sn, cs;
    sincos(-ph, &sn, &cs);
    M3<T> m;
    for (int k = 0; k < 9; ++k) {
        m.re[k] = T(zr[k] * cs - zi[k] * sn);
        m.im[k] = T(zr[k] * sn + zi[k] * cs);
    }
    store_link<T, NC>(U, g.P, mu, sidx(g, site_of_lex(g, s)), m);
}

// Random gauge transformation (Sec. V.D): store G(x) (FP64 [V][3][3][2] in
// lexicographic site order) as 18 reals per site in the link layout, then
// U_mu(x) -> G(x) U_mu(x) G^dag(x + mu) for every link.
template <class T>
__global__ void k_store_gauge(Geo g, const double *__restrict__ Glex, T *Gs) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const double *q = Glex + 18ll * s;
    M3<T> m;
#pragma unroll
    for (int k = 0; k < 9; ++k) { m.re[k] = T(q[2 * k]); m.im[k] = T(q[2 * k + 1]); }
    store_link<T, 18>(Gs, g.P, 0, sidx(g, site_of_lex(g, s)), m);
}

template <class T, int NC>
__global__ void k_gauge_links(Geo g, const T *__restrict__ Gs, T *U) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4ll * g.V) return;
    const int mu = (int)(l / g.V);
    const Pt x = site_of_index(g, (int)(l % g.V));
    const int i = sidx(g, x);
    const int iy = sidx(g, mv(g, x, mu, 1));
    M3<T> u = load_link<T, NC>(U, g.P, mu, i);
    u = m3_mul(load_link<T, 18>(Gs, g.P, 0, i), u);
    u = m3_mul_nd(u, load_link<T, 18>(Gs, g.P, 0, iy));
    store_link<T, NC>(U, g.P, mu, i, u);
}

// Z(3) projection of every link: reference label from arg Tr U, link -> exp(2 pi i n/3) I.
template <class T, int NC>
__global__ void k_project(Geo g, T *U, int8_t *ref) {
    long long l = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= 4ll * g.V) return;
    const int mu = (int)(l / g.V);
    const int i = sidx(g, site_of_index(g, (int)(l % g.V)));
    M3<T> m = load_link<T, NC>(U, g.P, mu, i);
    int n = z3_label<T>(m.re[0] + m.re[4] + m.re[8], m.im[0] + m.im[4] + m.im[8]);
    double sn, cs;
    sincospi(2.0 * n / 3.0, &sn, &cs);
    M3<T> z;
    m3_zero(z);
    z.re[0] = z.re[4] = z.re[8] = T(cs);
    z.im[0] = z.im[4] = z.im[8] = T(sn);
    store_link<T, NC>(U, g.P, mu, i, z);
    ref[(long long)mu * g.P + i] = (int8_t)n;
}

}  // namespace

// ---------------------------------------------------------------------------
// Dispatch
// ---------------------------------------------------------------------------

static std::atomic<long long> g_launches{0};
void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }

#define VS_DISPATCH(prec, nc, KERNEL, ...)                                          \
    do {                                                                            \
        if ((prec) == 0 && (nc) == 18) { KERNEL<double, 18>__VA_ARGS__; }           \
        else if ((prec) == 1 && (nc) == 18) { KERNEL<float, 18>__VA_ARGS__; }       \
        else if ((prec) == 1 && (nc) == 12) { KERNEL<float, 12>__VA_ARGS__; }       \
        else return cudaErrorInvalidValue;                                          \
    } while (0)

cudaError_t launch_load_labels(int prec, int nc, const Geo &g, const int8_t *lab, void *U, int8_t *ref,
                               cudaStream_t st) {
    int b = std::min(nblocks(4ll * g.V), kTableGrid);
    if (prec == 0) k_load_labels<double, 18><<<b, kThreads, 0, st>>>(g, lab, (double *)U, ref);
    else if (nc == 18) k_load_labels<float, 18><<<b, kThreads, 0, st>>>(g, lab, (float *)U, ref);
    else k_load_labels<float, 12><<<b, kThreads, 0, st>>>(g, lab, (float *)U, ref);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_load_links(int prec, int nc, const Geo &g, const double *in, void *U, int8_t *ref,
                              cudaStream_t st) {
    int b = nblocks(4ll * g.V);
    if (prec == 0) k_load_links<double, 18><<<b, kThreads, 0, st>>>(g, in, (double *)U, ref);
    else if (nc == 18) k_load_links<float, 18><<<b, kThreads, 0, st>>>(g, in, (float *)U, ref);
    else k_load_links<float, 12><<<b, kThreads, 0, st>>>(g, in, (float *)U, ref);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_read_links(int prec, int nc, const Geo &g, const void *U, double *out, cudaStream_t st) {
    int b = nblocks(4ll * g.V);
    if (prec == 0) k_read_links<double, 18><<<b, kThreads, 0, st>>>(g, (const double *)U, out);
    else if (nc == 18) k_read_links<float, 18><<<b, kThreads, 0, st>>>(g, (const float *)U, out);
    else k_read_links<float, 12><<<b, kThreads, 0, st>>>(g, (const float *)U, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(int prec, int nc, const Geo &g, const void *U, unsigned long long *count,
                                   cudaStream_t st) {
    const int b = nblocks(4ll * g.V);
    if (prec == 0) k_count_nonfinite<double, 18><<<b, kThreads, 0, st>>>(g, (const double *)U, count);
    else if (nc == 18) k_count_nonfinite<float, 18><<<b, kThreads, 0, st>>>(g, (const float *)U, count);
    else k_count_nonfinite<float, 12><<<b, kThreads, 0, st>>>(g, (const float *)U, count);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_store_ref(const Geo &g, const int8_t *lab_lex, int8_t *ref, cudaStream_t st) {
    k_store_ref<<<nblocks(4ll * g.V), kThreads, 0, st>>>(g, lab_lex, ref);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_read_labels(const Geo &g, const int8_t *ref, int8_t *out, cudaStream_t st) {
    k_read_labels<<<nblocks(4ll * g.V), kThreads, 0, st>>>(g, ref, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_current_labels(int prec, int nc, const Geo &g, const void *U, int8_t *out, cudaStream_t st) {
    int b = nblocks(4ll * g.V);
    if (prec == 0) k_current_labels<double, 18><<<b, kThreads, 0, st>>>(g, (const double *)U, out);
    else if (nc == 18) k_current_labels<float, 18><<<b, kThreads, 0, st>>>(g, (const float *)U, out);
    else k_current_labels<float, 12><<<b, kThreads, 0, st>>>(g, (const float *)U, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_centrifuge(int prec, int nc, const Geo &g, const int8_t *ref, double omega, uint64_t seed,
                              void *U, cudaStream_t st) {
    int b = std::min(nblocks(4ll * g.V), kTableGrid);
    if (prec == 0) k_centrifuge<double, 18><<<b, kThreads, 0, st>>>(g, ref, omega, seed, (double *)U);
    else if (nc == 18) k_centrifuge<float, 18><<<b, kThreads, 0, st>>>(g, ref, omega, seed, (float *)U);
    else k_centrifuge<float, 12><<<b, kThreads, 0, st>>>(g, ref, omega, seed, (float *)U);
    count_launches(1);
    return cudaGetLastError();
}

int action_partials(const Geo &g) {
    int b = nblocks(g.V);
    return b < 1216 ? b : 1216;
}

cudaError_t launch_action(int prec, int nc, const Geo &g, const void *U, double *partials, double *out,
                          cudaStream_t st) {
    int b = action_partials(g);
    if (prec == 0) k_action<double, 18><<<b, kThreads, 0, st>>>(g, (const double *)U, partials);
    else if (nc == 18) k_action<float, 18><<<b, kThreads, 0, st>>>(g, (const float *)U, partials);
    else k_action<float, 12><<<b, kThreads, 0, st>>>(g, (const float *)U, partials);
    // <S>/beta = (1/V) sum_x (2/72) sum_{mu<nu} (3 - Re Tr P)
    k_sum_partials<<<1, 1024, 0, st>>>(partials, b, 2.0 / 72.0 / (double)g.V, out);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_observables(int prec, int nc, const Geo &g, const void *U, double *partials, double *out,
                               double *S_site, double *SR_site, double *q_site, cudaStream_t st) {
    // one balanced wave: as many blocks as are resident at once (the kernel's
    // registers allow one or two per SM), at most 400 (the partials buffer)
    int b = nblocks(g.V), dev = 0, n_sm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (prec == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_observables<double, 18>, kThreads, 0);
    else if (nc == 18)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_observables<float, 18>, kThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_observables<float, 12>, kThreads, 0);
    const int wave = std::max(1, n_sm * std::max(per_sm, 1));
    b = std::min(b, std::min(wave, 400));
    if (prec == 0)
        k_observables<double, 18><<<b, kThreads, 0, st>>>(g, (const double *)U, partials, S_site, SR_site, q_site);
    else if (nc == 18)
        k_observables<float, 18><<<b, kThreads, 0, st>>>(g, (const float *)U, partials, S_site, SR_site, q_site);
    else
        k_observables<float, 12><<<b, kThreads, 0, st>>>(g, (const float *)U, partials, S_site, SR_site, q_site);
    k_sum_partials3<<<1, 1024, 0, st>>>(partials, b, 1.0 / (double)g.V, out);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_correlation(const double *a, const double *b, long long n, double *partials, double *out,
                               cudaStream_t st) {
    const int nb = (int)std::min<long long>(nblocks(n), kCorrGrid);
    k_correlation<<<nb, kThreads, 0, st>>>(a, b, n, partials);
    k_correlation_finish<<<1, 1024, 0, st>>>(partials, nb, out);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t preload_vortex_kernels() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k_vortex_links<double, 18>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_vortex_links<float, 18>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_vortex_links<float, 12>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, k_vortex_charges);
    return e;
}

cudaError_t launch_vortex(int prec, int nc, const Geo &g, const void *U, const int8_t *ref, int8_t *cur,
                          unsigned long long *counts, unsigned long long *mbits, cudaStream_t st,
                          const void *G) {
    int b = nblocks(4ll * g.V);
    if (prec == 0)
        k_vortex_links<double, 18><<<b, kThreads, 0, st>>>(g, (const double *)U, ref, cur, counts, mbits,
                                                           (const double *)G);
    else if (nc == 18)
        k_vortex_links<float, 18><<<b, kThreads, 0, st>>>(g, (const float *)U, ref, cur, counts, mbits,
                                                          (const float *)G);
    else
        k_vortex_links<float, 12><<<b, kThreads, 0, st>>>(g, (const float *)U, ref, cur, counts, mbits,
                                                          (const float *)G);
    k_vortex_charges<<<nblocks(g.V), kThreads, 0, st>>>(g, ref, cur, counts);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_reunit(int prec, int nc, const Geo &g, void *U, const int8_t *ref, cudaStream_t st,
                          const void *G) {
    int b = nblocks(4ll * g.V);
    if (prec == 0) k_reunit<double, 18><<<b, kThreads, 0, st>>>(g, (double *)U, ref, (const double *)G);
    else if (nc == 18) k_reunit<float, 18><<<b, kThreads, 0, st>>>(g, (float *)U, ref, (const float *)G);
    else k_reunit<float, 12><<<b, kThreads, 0, st>>>(g, (float *)U, ref, (const float *)G);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_debug_expm(int prec, const double *X, int n, double *E, cudaStream_t st) {
    if (prec == 0) k_debug_expm<double><<<nblocks(n), kThreads, 0, st>>>(X, n, E);
    else k_debug_expm<float><<<nblocks(n), kThreads, 0, st>>>(X, n, E);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_haar(int prec, int nc, const Geo &g, uint64_t seed, void *U, cudaStream_t st) {
    int b = nblocks(4ll * g.V);
    if (prec == 0) k_haar<double, 18><<<b, kThreads, 0, st>>>(g, seed, (double *)U);
    else if (nc == 18) k_haar<float, 18><<<b, kThreads, 0, st>>>(g, seed, (float *)U);
    else k_haar<float, 12><<<b, kThreads, 0, st>>>(g, seed, (float *)U);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_aus_class(int prec, int nc, bool rect, int mu, const AusParams &p, cudaStream_t st) {
    if (prec == 0) return launch_aus_d18(rect, mu, p, st);
    if (nc == 18) return launch_aus_f18(rect, mu, p, st);
    return launch_aus_f12(rect, mu, p, st);
}

cudaError_t launch_gauge(int prec, int nc, const Geo &g, const double *G_lex, void *Gs, void *U,
                         cudaStream_t st) {
    if (prec == 0) {
        k_store_gauge<double><<<nblocks(g.V), kThreads, 0, st>>>(g, G_lex, (double *)Gs);
        k_gauge_links<double, 18><<<nblocks(4ll * g.V), kThreads, 0, st>>>(g, (const double *)Gs, (double *)U);
    } else {
        k_store_gauge<float><<<nblocks(g.V), kThreads, 0, st>>>(g, G_lex, (float *)Gs);
        if (nc == 18)
            k_gauge_links<float, 18><<<nblocks(4ll * g.V), kThreads, 0, st>>>(g, (const float *)Gs, (float *)U);
        else
            k_gauge_links<float, 12><<<nblocks(4ll * g.V), kThreads, 0, st>>>(g, (const float *)Gs, (float *)U);
    }
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_project(int prec, int nc, const Geo &g, void *U, int8_t *ref, cudaStream_t st) {
    int b = nblocks(4ll * g.V);
    if (prec == 0) k_project<double, 18><<<b, kThreads, 0, st>>>(g, (double *)U, ref);
    else if (nc == 18) k_project<float, 18><<<b, kThreads, 0, st>>>(g, (float *)U, ref);
    else k_project<float, 12><<<b, kThreads, 0, st>>>(g, (float *)U, ref);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vs
