// vs_device.cuh -- device-side SU(3) algebra, lattice geometry and field layout.
//
// Field layout in HBM:
//   links of direction mu: NC reals per site (NC = 18: row-major 3x3 as
//   re,im pairs; NC = 12: rows 0 and 1 only, row 2 rebuilt as
//   conj(row0 x row1) on load) at element mu NC P, in blocks of 16 site
//   positions holding each float4 / float2 / double2 vector chunk of their
//   16 links contiguously (see load_link); i = site position.
//   Site position: rows (y, z, t) in lexicographic order, and inside each
//   x-row the sites grouped by x mod 4: i = row*4Qp + (x & 3)*Qp + (x >> 2),
//   Qp = Lx/4, or 8 when Lx/4 is 5, 6 or 7 (the group then ends in unused
//   positions).  For a colour class of the annealed schedule the updated
//   sites of one row form contiguous runs of Lx/4, so a warp's loads of any
//   chunk are whole 32-byte sectors; with the padding a run of 5-7 sites
//   (80-112 bytes of a float4 chunk) never straddles a 128-byte line.
//   labels[mu][i]    int8 reference Z(3) label of link (mu, i).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace vs {

struct Geo {
    int L[4];       // Lx, Ly, Lz, Lt
    int Q;          // Lx / 4: sites of one x mod 4 group of an x-row
    int Qp;         // positions of that group in the layout (Q, or 8 for Q = 5, 6, 7)
    int Lxp;        // positions of an x-row: 4 Qp
    int V;          // sites
    long long P;    // site positions per direction (plane stride): Lxp Ly Lz Lt >= V
};

// The geometry of extents dims (each a positive multiple of 4).
__host__ __device__ inline Geo make_geo(const int dims[4]) {
    Geo g;
    for (int k = 0; k < 4; ++k) g.L[k] = dims[k];
    g.Q = dims[0] / 4;
    g.Qp = (g.Q == 5 || g.Q == 6 || g.Q == 7) ? 8 : g.Q;
    g.Lxp = 4 * g.Qp;
    g.V = (int)((long long)dims[0] * dims[1] * dims[2] * dims[3]);
    g.P = (long long)g.Lxp * dims[1] * dims[2] * dims[3];
    return g;
}

__host__ __device__ __forceinline__ int wrapc(int v, int L) {
    v = v < 0 ? v + L : v;
    return v >= L ? v - L : v;
}

struct Pt { int x0, x1, x2, x3; };

// x + k * e_d with periodic wrap (|k| <= L)
__device__ __forceinline__ Pt mv(const Geo &g, Pt p, int d, int k) {
    if (d == 0) p.x0 = wrapc(p.x0 + k, g.L[0]);
    else if (d == 1) p.x1 = wrapc(p.x1 + k, g.L[1]);
    else if (d == 2) p.x2 = wrapc(p.x2 + k, g.L[2]);
    else p.x3 = wrapc(p.x3 + k, g.L[3]);
    return p;
}

__host__ __device__ __forceinline__ int sidx(const Geo &g, int x0, int x1, int x2, int x3) {
    return ((x3 * g.L[2] + x2) * g.L[1] + x1) * g.Lxp + (x0 & 3) * g.Qp + (x0 >> 2);
}
__device__ __forceinline__ int sidx(const Geo &g, const Pt &p) { return sidx(g, p.x0, p.x1, p.x2, p.x3); }

__device__ __forceinline__ int lexidx(const Geo &g, const Pt &p) {
    return p.x0 + g.L[0] * (p.x1 + g.L[1] * (p.x2 + g.L[2] * p.x3));
}

// Site number i (0 <= i < V) in plane order, i.e. the i-th site of the
// layout skipping unused positions (its position is sidx of the result).
__device__ __forceinline__ Pt site_of_index(const Geo &g, int i) {
    Pt p;
    int w = i % g.L[0];
    int row = i / g.L[0];
    p.x0 = 4 * (w % g.Q) + w / g.Q;
    p.x1 = row % g.L[1];
    row /= g.L[1];
    p.x2 = row % g.L[2];
    p.x3 = row / g.L[2];
    return p;
}

// Thread t of a launch over every site of direction MU (the simultaneous
// schedules and the Runge-Kutta stages): odd directions take the sites in
// reverse order, so each launch starts where the previous one ended.
template <int MU>
__device__ __forceinline__ Pt dir_site(const Geo &g, int t) {
    return site_of_index(g, (MU & 1) ? g.V - 1 - t : t);
}

// The site at layout position i (the inverse of sidx on used positions).
__device__ __forceinline__ Pt site_of_pos(const Geo &g, int i) {
    Pt p;
    const int r = i % g.Lxp;
    int row = i / g.Lxp;
    p.x0 = 4 * (r % g.Qp) + r / g.Qp;
    p.x1 = row % g.L[1];
    row /= g.L[1];
    p.x2 = row % g.L[2];
    p.x3 = row / g.L[2];
    return p;
}

__device__ __forceinline__ Pt site_of_lex(const Geo &g, int s) {
    Pt p;
    p.x0 = s % g.L[0]; s /= g.L[0];
    p.x1 = s % g.L[1]; s /= g.L[1];
    p.x2 = s % g.L[2];
    p.x3 = s / g.L[2];
    return p;
}

// Thread t (0 <= t < V/4) of colour class (mu, c): the class is the set of
// sites with (2 x_mu + sum_{nu != mu} x_nu) mod 4 == c.
//  mu != 0: every x-row holds Lx/4 class sites, x = 4a + b with
//           b = (c - (x_mu + y + z + t)) mod 4 over the row's (y,z,t) coordinates.
//  mu == 0: 2x = c - (y+z+t) mod 4 needs c - (y+z+t) even: half the rows hold
//           Lx/2 class sites, x mod 4 in {b0, b0 + 2}.
// Odd colours take the sites in reverse order, so that each class launch of a
// sweep starts where the previous one ended and finds those links still in L2.
template <int MU>
__device__ __forceinline__ Pt class_site(const Geo &g, int c, int t) {
    Pt p;
    const int Q = g.Q;
    if (c & 1) t = g.V / 4 - 1 - t;
    if (MU != 0) {
        int a = t % Q;
        int row = t / Q;
        p.x1 = row % g.L[1];
        row /= g.L[1];
        p.x2 = row % g.L[2];
        p.x3 = row / g.L[2];
        int xm = MU == 1 ? p.x1 : (MU == 2 ? p.x2 : p.x3);
        int b = (c - (p.x1 + p.x2 + p.x3 + xm)) & 3;
        p.x0 = 4 * a + b;
    } else {
        int w = t % (2 * Q);
        int row = t / (2 * Q);
        int h = g.L[1] >> 1;
        int j = row % h;
        row /= h;
        p.x2 = row % g.L[2];
        p.x3 = row / g.L[2];
        p.x1 = 2 * j + ((c - p.x2 - p.x3) & 1);
        int b0 = ((c - (p.x1 + p.x2 + p.x3)) >> 1) & 1;
        p.x0 = 4 * (w % Q) + b0 + 2 * (w / Q);
    }
    return p;
}

// --------------------------------------------------------------------------
// 3x3 complex matrices in registers
// --------------------------------------------------------------------------

template <class T>
struct M3 {
    T re[9];
    T im[9];
};

template <class T>
__device__ __forceinline__ M3<T> m3_dag(const M3<T> &a) {
    M3<T> r;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            r.re[i * 3 + j] = a.re[j * 3 + i];
            r.im[i * 3 + j] = -a.im[j * 3 + i];
        }
    return r;
}

// FP32 complex entries as packed pairs (re, im) for the paired FP32 FMA of
// sm_100 and later (fma.rn.f32x2: two independent FMAs in one instruction).
// VS_FFMA2=0 selects the scalar FMA chains for FP32 as well.
#ifndef VS_FFMA2
#define VS_FFMA2 1
#endif
typedef unsigned long long f2pk;
__device__ __forceinline__ f2pk pk2(float lo, float hi) {
    f2pk r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f2pk v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2pk add2(f2pk a, f2pk b) {
    f2pk d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2pk mul2(f2pk a, f2pk b) {
    f2pk d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2pk fma2(f2pk a, f2pk b, f2pk c) {
    f2pk d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// r = c + a * b in FP32: per entry one chain of paired FMAs in k order,
//   (Re r_ij, Im r_ij) = (Re c, Im c) + sum_k [Re a_ik (Re b_kj, Im b_kj) + Im a_ik (-Im b_kj, Re b_kj)],
// with the right factor's entries also kept as swapped, negated pairs, so no
// separate additions combine real and imaginary parts (18 fewer FP32
// operations per product than two chains and a combine step).  Every entry
// goes through the same operations, so entries built from equal inputs come
// out bit-identical (a product of matrices proportional to the identity stays
// exactly so).
template <bool ACC>
__device__ __forceinline__ void m3_mul_f32(M3<float> &r, const M3<float> &a, const M3<float> &b) {
    f2pk bb[9], bs[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) { bb[e] = pk2(b.re[e], b.im[e]); bs[e] = pk2(-b.im[e], b.re[e]); }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        f2pk P[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) P[j] = ACC ? pk2(r.re[i * 3 + j], r.im[i * 3 + j]) : pk2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const f2pk ar = pk2(a.re[i * 3 + k], a.re[i * 3 + k]);
            const f2pk ai = pk2(a.im[i * 3 + k], a.im[i * 3 + k]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                P[j] = fma2(ar, bb[k * 3 + j], P[j]);
                P[j] = fma2(ai, bs[k * 3 + j], P[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) upk2(P[j], r.re[i * 3 + j], r.im[i * 3 + j]);
    }
}

// rows 0-1 of r = a * b (rows 0-1 of a, all of b); row 2 of r is not written.
__device__ __forceinline__ void m3_mul_2r(M3<float> &r, const M3<float> &a, const M3<float> &b) {
#if VS_FFMA2
    f2pk bb[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) bb[e] = pk2(b.re[e], b.im[e]);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        f2pk P[3], Q[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) { P[j] = pk2(0.f, 0.f); Q[j] = pk2(0.f, 0.f); }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const f2pk ar = pk2(a.re[i * 3 + k], a.re[i * 3 + k]);
            const f2pk ai = pk2(a.im[i * 3 + k], a.im[i * 3 + k]);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                P[j] = fma2(ar, bb[k * 3 + j], P[j]);
                Q[j] = fma2(ai, bb[k * 3 + j], Q[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float px, py, qx, qy;
            upk2(P[j], px, py);
            upk2(Q[j], qx, qy);
            r.re[i * 3 + j] = px - qy;
            r.im[i * 3 + j] = py + qx;
        }
    }
#else
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                sr = fmaf(a.re[i * 3 + k], b.re[k * 3 + j], sr);
                sr = fmaf(-a.im[i * 3 + k], b.im[k * 3 + j], sr);
                si = fmaf(a.re[i * 3 + k], b.im[k * 3 + j], si);
                si = fmaf(a.im[i * 3 + k], b.re[k * 3 + j], si);
            }
            r.re[i * 3 + j] = sr;
            r.im[i * 3 + j] = si;
        }
#endif
}

// r = a * b.  FP64: every entry is the same chain of fused multiply-adds
// started from zero; FP32: m3_mul_f32.  Either way entries built from equal
// inputs come out bit-identical.
template <class T>
__device__ __forceinline__ M3<T> m3_mul(const M3<T> &a, const M3<T> &b) {
    M3<T> r;
    if constexpr (sizeof(T) == 4 && VS_FFMA2) {
        m3_mul_f32<false>(r, a, b);
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T sr = T(0), si = T(0);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    sr = fma(a.re[i * 3 + k], b.re[k * 3 + j], sr);
                    sr = fma(-a.im[i * 3 + k], b.im[k * 3 + j], sr);
                    si = fma(a.re[i * 3 + k], b.im[k * 3 + j], si);
                    si = fma(a.im[i * 3 + k], b.re[k * 3 + j], si);
                }
                r.re[i * 3 + j] = sr;
                r.im[i * 3 + j] = si;
            }
    }
    return r;
}

// r += a * b
template <class T>
__device__ __forceinline__ void m3_madd(M3<T> &r, const M3<T> &a, const M3<T> &b) {
    if constexpr (sizeof(T) == 4 && VS_FFMA2) {
        m3_mul_f32<true>(r, a, b);
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                T sr = r.re[i * 3 + j], si = r.im[i * 3 + j];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    sr = fma(a.re[i * 3 + k], b.re[k * 3 + j], sr);
                    sr = fma(-a.im[i * 3 + k], b.im[k * 3 + j], sr);
                    si = fma(a.re[i * 3 + k], b.im[k * 3 + j], si);
                    si = fma(a.im[i * 3 + k], b.re[k * 3 + j], si);
                }
                r.re[i * 3 + j] = sr;
                r.im[i * 3 + j] = si;
            }
    }
}

// r = a * b^dagger
template <class T>
__device__ __forceinline__ M3<T> m3_mul_nd(const M3<T> &a, const M3<T> &b) {
    return m3_mul(a, m3_dag(b));
}

// r = a^dagger * b
template <class T>
__device__ __forceinline__ M3<T> m3_mul_dn(const M3<T> &a, const M3<T> &b) {
    return m3_mul(m3_dag(a), b);
}

template <class T>
__device__ __forceinline__ void m3_zero(M3<T> &r) {
#pragma unroll
    for (int k = 0; k < 9; ++k) { r.re[k] = T(0); r.im[k] = T(0); }
}

// r += s * a
template <class T>
__device__ __forceinline__ void m3_axpy(M3<T> &r, T s, const M3<T> &a) {
#pragma unroll
    for (int k = 0; k < 9; ++k) { r.re[k] = fma(s, a.re[k], r.re[k]); r.im[k] = fma(s, a.im[k], r.im[k]); }
}

// FP32 entrywise sums of matrices.  An entry's (re, im) pair is one operand
// of a paired instruction; each half rounds like the scalar operation, so
// the results equal the scalar ones while the issued instructions halve
// (the class-update kernel is bound by instruction issue).
#if VS_FFMA2
template <>
__device__ __forceinline__ void m3_axpy<float>(M3<float> &r, float s, const M3<float> &a) {
    const f2pk sp = pk2(s, s);
#pragma unroll
    for (int k = 0; k < 9; ++k) upk2(fma2(sp, pk2(a.re[k], a.im[k]), pk2(r.re[k], r.im[k])), r.re[k], r.im[k]);
}
#endif

// r += a
__device__ __forceinline__ void m3_acc_f32(M3<float> &r, const M3<float> &a) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
#if VS_FFMA2
        upk2(add2(pk2(r.re[k], r.im[k]), pk2(a.re[k], a.im[k])), r.re[k], r.im[k]);
#else
        r.re[k] += a.re[k];
        r.im[k] += a.im[k];
#endif
    }
}

// r = c0 a + c1 (b + d), rounded as fmaf(c0, a, c1 * (b + d))
__device__ __forceinline__ void m3_lin3_f32(M3<float> &r, float c0, const M3<float> &a, float c1, const M3<float> &b,
                                            const M3<float> &d) {
#if VS_FFMA2
    const f2pk c0p = pk2(c0, c0), c1p = pk2(c1, c1);
#endif
#pragma unroll
    for (int k = 0; k < 9; ++k) {
#if VS_FFMA2
        upk2(fma2(c0p, pk2(a.re[k], a.im[k]), mul2(c1p, add2(pk2(b.re[k], b.im[k]), pk2(d.re[k], d.im[k])))),
             r.re[k], r.im[k]);
#else
        r.re[k] = fmaf(c0, a.re[k], c1 * (b.re[k] + d.re[k]));
        r.im[k] = fmaf(c0, a.im[k], c1 * (b.im[k] + d.im[k]));
#endif
    }
}

template <class T>
__device__ __forceinline__ void m3_scale(M3<T> &r, T s) {
#pragma unroll
    for (int k = 0; k < 9; ++k) { r.re[k] *= s; r.im[k] *= s; }
}

// --------------------------------------------------------------------------
// Link load / store
// --------------------------------------------------------------------------

// Links of one direction mu start at element mu * NC * P and come in blocks
// of 16 consecutive plane positions (P is a multiple of 256).  Inside block
// b = i / 16 each vector chunk of the 16 links is contiguous:
//   float, 18 reals : 4 float4 chunks (complex entries 0-1, 2-3, 4-5, 6-7),
//                     then 1 float2 chunk (entry 8): 1152-byte blocks
//   float, 12 reals : 3 float4 chunks (entries 0-1, 2-3, 4-5): 768 bytes; row 2 rebuilt
//   double, 18 reals: 9 double2 chunks (one complex entry each): 2304 bytes
// so chunk c of the link at position i is one aligned vector at block offset
// (chunk bytes x 16 before c) + (i mod 16) x (chunk bytes): the chunks of a link
// sit at compile-time offsets from its first one (a single address per link),
// and every float4 chunk run of a block starts on a 128-byte line.
template <int NC>
__device__ __forceinline__ int blk_off4(int i) { return 4 * i + (i >> 4) * (16 * NC - 64); }  // float4 chunk 0
__device__ __forceinline__ int blk_off2(int i) { return 2 * i + (i >> 4) * (16 * 18 - 32) + 256; }  // float2 chunk
__device__ __forceinline__ int blk_offd(int i) { return 2 * i + (i >> 4) * (16 * 18 - 32); }  // double2 chunk 0
// row 2 = conj(row 0 x row 1): the third row of an SU(3) matrix from the first two,
// each component one chain of fused multiply-adds (four operations)
template <class T>
__device__ __forceinline__ void rebuild_row2(M3<T> &m) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        int j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        T cr = fma(m.re[j1], m.re[3 + j2], fma(-m.im[j1], m.im[3 + j2],
                   fma(-m.re[j2], m.re[3 + j1], m.im[j2] * m.im[3 + j1])));
        T ci = fma(m.re[j1], m.im[3 + j2], fma(m.im[j1], m.re[3 + j2],
                   fma(-m.re[j2], m.im[3 + j1], -(m.im[j2] * m.re[3 + j1]))));
        m.re[6 + j] = cr;
        m.im[6 + j] = -ci;
    }
}

// The stored reals of a link (row 2 of 12-real links not yet rebuilt).
template <class T, int NC>
__device__ __forceinline__ M3<T> load_link_raw(const T *__restrict__ U, long long P, int mu, int i) {
    const T *base = U + (long long)mu * NC * P;
    M3<T> m;
    if constexpr (sizeof(T) == 4) {
        const float *b0 = base + blk_off4<NC>(i);
#pragma unroll
        for (int q = 0; q < NC / 4; ++q) {
            float4 v = __ldg(reinterpret_cast<const float4 *>(b0 + 64 * q));
            m.re[2 * q] = v.x; m.im[2 * q] = v.y; m.re[2 * q + 1] = v.z; m.im[2 * q + 1] = v.w;
        }
        if (NC == 18) {
            float2 v = __ldg(reinterpret_cast<const float2 *>(base + blk_off2(i)));
            m.re[8] = v.x; m.im[8] = v.y;
        }
    } else {
        const T *b0 = base + blk_offd(i);
#pragma unroll
        for (int e = 0; e < NC / 2; ++e) {
            double2 v = __ldg(reinterpret_cast<const double2 *>(b0 + 32 * e));
            m.re[e] = v.x; m.im[e] = v.y;
        }
    }
    return m;
}

template <class T, int NC>
__device__ __forceinline__ M3<T> load_link(const T *__restrict__ U, long long P, int mu, int i) {
    M3<T> m = load_link_raw<T, NC>(U, P, mu, i);
    if (NC == 12) rebuild_row2(m);
    return m;
}

template <class T, class S>
__device__ __forceinline__ M3<T> m3_cast(const M3<S> &a) {
    M3<T> r;
#pragma unroll
    for (int k = 0; k < 9; ++k) { r.re[k] = T(a.re[k]); r.im[k] = T(a.im[k]); }
    return r;
}

// A link stored in precision S as an M3<T>: for FP32 storage read in FP64,
// the stored reals exactly, and row 2 of 12-real links rebuilt in FP64.
template <class T, int NC, class S>
__device__ __forceinline__ M3<T> load_link_as(const S *__restrict__ U, long long P, int mu, int i) {
    if constexpr (sizeof(T) == sizeof(S)) {
        return load_link<T, NC>(U, P, mu, i);
    } else {
        M3<T> m = m3_cast<T>(load_link_raw<S, NC>(U, P, mu, i));
        if (NC == 12) rebuild_row2(m);
        return m;
    }
}

template <class T, int NC>
__device__ __forceinline__ void store_link(T *__restrict__ U, long long P, int mu, int i, const M3<T> &m) {
    T *base = U + (long long)mu * NC * P;
    if constexpr (sizeof(T) == 4) {
        float *b0 = base + blk_off4<NC>(i);
#pragma unroll
        for (int q = 0; q < NC / 4; ++q)
            *reinterpret_cast<float4 *>(b0 + 64 * q) =
                make_float4(m.re[2 * q], m.im[2 * q], m.re[2 * q + 1], m.im[2 * q + 1]);
        if (NC == 18) *reinterpret_cast<float2 *>(base + blk_off2(i)) = make_float2(m.re[8], m.im[8]);
    } else {
        T *b0 = base + blk_offd(i);
#pragma unroll
        for (int e = 0; e < NC / 2; ++e)
            *reinterpret_cast<double2 *>(b0 + 32 * e) = make_double2(m.re[e], m.im[e]);
    }
}

// --------------------------------------------------------------------------
// Z(3) label of a trace t = a + ib (sector of arg t, Sec. I Eq. centre_element)
//   0  : a > 0 and b^2 < 3 a^2          (|arg| < pi/3)
//  +1  : b > 0, or b == 0 and a < 0      (arg in [pi/3, pi])
//  -1  : b < 0                           (arg in (-pi, -pi/3])
//   0  : t == 0
// --------------------------------------------------------------------------

template <class T>
__device__ __forceinline__ int z3_label(T a, T b) {
    if (a > T(0) && b * b < T(3) * a * a) return 0;
    if (b > T(0)) return 1;
    if (b < T(0)) return -1;
    return a < T(0) ? 1 : 0;
}

// Distance of the trace t = a + ib from the nearest edge of the sector of its
// label lab, in trace units (|t| times the sine of the angle to that edge).
// Sector 0 is bounded by the rays at arg = +-pi/3, at distance
// (sqrt3 a - |b|)/2; the sectors +-1 by the ray at +-pi/3, at distance
// (|b| - sqrt3 a)/2, and the ray at pi, at distance |b|.  The nearest edge is
// never more than pi/3 away, so the smaller sine belongs to it.  Errors of
// the trace are absolute (entries of unit modulus), so this is the quantity
// a rounding error is measured against.
template <class T>
__device__ __forceinline__ T edge_distance(T a, T b, int lab) {
    const T s = b < T(0) ? -b : b;
    const T r3a = T(1.7320508075688772) * a;
    const T d = lab == 0 ? T(0.5) * (r3a - s) : fmin(T(0.5) * (s - r3a), s);
    return d > T(0) ? d : T(0);
}

// sin of the angular margin of t from the nearest sector edge (0 for t = 0):
// monotone in the margin, which is asin of it
template <class T>
__device__ __forceinline__ T edge_sine(T a, T b, T d) {
    const T n2 = a * a + b * b;
    return n2 > T(0) ? d * rsqrt(n2) : T(0);
}

// Trace seen by the vortex-preservation test (Sec. VI): Tr U for the original
// gauge (G == nullptr); after a random gauge transformation G,
// Tr[G^dag(x) U G(x+mu)] = sum_jk U_jk (G(x+mu) G^dag(x))_kj.  G is stored as
// 18 reals per site in the link layout, plane position i.
template <class T, class S = T>
__device__ __forceinline__ void vp_trace(const S *__restrict__ G, long long P, int i_x, int i_xmu,
                                         const M3<T> &u, T &a, T &b) {
    if (!G) {
        a = u.re[0] + u.re[4] + u.re[8];
        b = u.im[0] + u.im[4] + u.im[8];
        return;
    }
    const M3<T> gx = load_link_as<T, 18>(G, P, 0, i_x), gy = load_link_as<T, 18>(G, P, 0, i_xmu);
    T sr = T(0), si = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            // M_kj = sum_l gy_kl conj(gx_jl)
            T mr = T(0), mi = T(0);
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                mr = fma(gy.re[3 * k + l], gx.re[3 * j + l], fma(gy.im[3 * k + l], gx.im[3 * j + l], mr));
                mi = fma(gy.im[3 * k + l], gx.re[3 * j + l], fma(-gy.re[3 * k + l], gx.im[3 * j + l], mi));
            }
            sr = fma(u.re[3 * j + k], mr, fma(-u.im[3 * j + k], mi, sr));
            si = fma(u.re[3 * j + k], mi, fma(u.im[3 * j + k], mr, si));
        }
    a = sr;
    b = si;
}

// --------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood 2014), counter mode: value i of stream seed
// --------------------------------------------------------------------------

__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace vs
