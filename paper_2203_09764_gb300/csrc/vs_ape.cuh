// vs_ape.cuh -- APE / annealed U-link smearing with unit circle projection and
// one stage of the third-order Runge-Kutta Wilson flow.  Included by
// vs_ape_f18.cu, vs_ape_f12.cu and vs_ape_d18.cu.
//
// Unit circle projection (Sec. II.C, Eqs. W and P_ucp):
//   W = V (V^dag V)^{-1/2},  P_ucp{V} = W / cbrt(det W)  (principal root).
// W is the unitary factor of the polar decomposition of V.  Here it comes
// from the scaled Newton iteration for the polar factor (Higham, "Computing
// the polar decomposition -- with applications", SIAM J. Sci. Stat. Comput.
// 7 (1986)): X_0 = V, X_{k+1} = (zeta_k X_k + X_k^{-dag} / zeta_k) / 2 with
// zeta_k = |det X_k|^{-1/3}, which converges quadratically for any
// nonsingular V and needs no eigenvalues.  The principal cube root takes
// arg det W in (-pi, pi], so the phase divided out lies in (-pi/3, pi/3].
// A blocked matrix with det(V^dag V) <= 1e-24 (Tr(V^dag V) / 3)^3 has no
// projection; the link is left unchanged and counted.
#pragma once

#include "vs_stout.cuh"

namespace vs {

// cofactor matrix transposed (adjugate) and determinant of m:
// C_ij = m[i1][j1] m[i2][j2] - m[i1][j2] m[i2][j1] with i1 = i+1, i2 = i+2,
// j1 = j+1, j2 = j+2 (mod 3); adj_ji = C_ij; det = sum_j m_0j C_0j.
template <class T>
__device__ __forceinline__ void m3_adj_det(const M3<T> &m, M3<T> &adj, T &dr, T &di) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            const int a = 3 * i1 + j1, b = 3 * i2 + j2, c = 3 * i1 + j2, d = 3 * i2 + j1;
            const T cr = (m.re[a] * m.re[b] - m.im[a] * m.im[b]) - (m.re[c] * m.re[d] - m.im[c] * m.im[d]);
            const T ci = (m.re[a] * m.im[b] + m.im[a] * m.re[b]) - (m.re[c] * m.im[d] + m.im[c] * m.re[d]);
            adj.re[3 * j + i] = cr;
            adj.im[3 * j + i] = ci;
        }
    dr = T(0);
    di = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // m_0j * C_0j, C_0j = adj_j0
        dr += m.re[j] * adj.re[3 * j] - m.im[j] * adj.im[3 * j];
        di += m.re[j] * adj.im[3 * j] + m.im[j] * adj.re[3 * j];
    }
}

template <class T> struct UcpTol;
template <> struct UcpTol<float> { static __device__ __forceinline__ float d2() { return 1e-13f; } };
template <> struct UcpTol<double> { static __device__ __forceinline__ double d2() { return 1e-28; } };

// P_ucp{V} into out; false (out untouched) if V is singular.
template <class T>
__device__ __forceinline__ bool ucp_project(const M3<T> &V, M3<T> &out) {
    M3<T> adj;
    T dr, di;
    m3_adj_det(V, adj, dr, di);
    T fro = T(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) fro += V.re[k] * V.re[k] + V.im[k] * V.im[k];
    const T t3 = fro / T(3);
    if (!(dr * dr + di * di > T(1e-24) * t3 * t3 * t3)) return false;
    M3<T> X = V;
#pragma unroll 1
    for (int it = 0; it < 40; ++it) {
        if (it > 0) m3_adj_det(X, adj, dr, di);
        const T d2 = dr * dr + di * di;
        // zeta = |det X|^{-1/3}; X^{-dag}_ij = conj(adj_ji) / conj(det) = conj(adj_ji) det / |det|^2
        const T zeta = pow(d2, T(-1) / T(6));
        const T iz = T(1) / zeta;
        const T er = dr / d2, ei = di / d2;
        T delta = T(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const T ar = adj.re[3 * j + i], ai = -adj.im[3 * j + i];
                const T yr = ar * er - ai * ei, yi = ar * ei + ai * er;
                const T nr = T(0.5) * (zeta * X.re[3 * i + j] + iz * yr);
                const T ni = T(0.5) * (zeta * X.im[3 * i + j] + iz * yi);
                const T dre = nr - X.re[3 * i + j], dim = ni - X.im[3 * i + j];
                delta += dre * dre + dim * dim;
                X.re[3 * i + j] = nr;
                X.im[3 * i + j] = ni;
            }
        if (delta <= UcpTol<T>::d2()) break;
    }
    m3_adj_det(X, adj, dr, di);
    T phi = atan2(di, dr);
    if (phi <= -T(3.14159265358979323846)) phi = T(3.14159265358979323846);
    T sn, cs;
    sincos(-phi / T(3), &sn, &cs);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        out.re[k] = X.re[k] * cs - X.im[k] * sn;
        out.im[k] = X.re[k] * sn + X.im[k] * cs;
    }
    return true;
}

// APE / AUS+UCP update of link (x, MU) at plane position i from its staple
// sum Vb and current value u: blocking, projection (a singular V keeps u),
// vortex-preservation test, store if accepted.
template <class T, int NC, int MU>
__device__ __forceinline__ void ape_finish(const ApeParams &a, const Pt &x, int i, M3<T> Vb, const M3<T> &u,
                                           Update<T> &up) {
    const Geo &g = a.g;
    const T al = sizeof(T) == 4 ? T(a.alpha_f) : T(a.alpha);
    const T w6 = al / T(6), w1 = T(1) - al;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        Vb.re[k] = fma(w1, u.re[k], w6 * Vb.re[k]);
        Vb.im[k] = fma(w1, u.im[k], w6 * Vb.im[k]);
    }
    M3<T> un;
    if (!ucp_project<T>(Vb, un)) {
        un = u;
        up.second = true;      // singular: counted in the second slot
    }
    if (NC == 12) rebuild_row2(un);
    T tr_re, tr_im;
    vp_trace<T>(static_cast<const T *>(a.G), g.P, i, a.G ? sidx(g, mv(g, x, MU, 1)) : i, un, tr_re, tr_im);
    vp_decide<T>(a.vp, a.counters != nullptr, (int)a.ref[(long long)MU * g.P + i], tr_re, tr_im, up);
    if (!up.reject) store_link<T, NC>(static_cast<T *>(a.U), g.P, MU, i, un);
    else if (a.U != a.Usrc) store_link<T, NC>(static_cast<T *>(a.U), g.P, MU, i, u);
}

// APE / AUS with unit circle projection: one thread per link of the colour
// class (annealed, in place) or of direction MU (colour < 0, from Usrc).
template <class T, int NC, bool RECT, int MU>
__global__ void __launch_bounds__(VS_SUBSWEEP_THREADS, sizeof(T) == 4 ? VS_SUBSWEEP_MINB : 1)
    k_ape(ApeParams a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < a.n_threads;
    Update<T> up;
    if (active) {
        const Geo &g = a.g;
        const Pt x = a.colour >= 0 ? class_site<MU>(g, a.colour, t) : dir_site<MU>(g, t);
        const int i = sidx(g, x);
        const T *Us = static_cast<const T *>(a.Usrc);
        const T c0 = sizeof(T) == 4 ? T(a.c0_f) : T(a.c0), c1 = sizeof(T) == 4 ? T(a.c1_f) : T(a.c1);
        const M3<T> Vb = staple_sum<T, NC, RECT, MU>(g, Us, x, c0, c1);
        const M3<T> u = load_link<T, NC>(Us, g.P, MU, i);
        ape_finish<T, NC, MU>(a, x, i, Vb, u, up);
    }
    count_update<T>(a.counters, up);
}

// FP32 over-improved AUS+UCP with the one-pass link stream of k_subsweep_fused.
template <int NC, int MU>
__global__ void __launch_bounds__(VS_RING_THREADS, VS_RING_MINB) k_ape_ring(ApeParams a) {
    extern __shared__ float4 ape_dyn[];
    float4 *ring4 = ape_dyn;
    float2 *ring2 = reinterpret_cast<float2 *>(ape_dyn + 6 * (NC / 4) * VS_RING_THREADS);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = t < a.n_threads;
    Update<float> up;
    if (active) {
        const Geo &g = a.g;
        const Pt x = a.colour >= 0 ? class_site<MU>(g, a.colour, t) : dir_site<MU>(g, t);
        const int i = sidx(g, x);
        LinkRing<NC> R = ring_of<NC>(ring4, ring2);
        M3<float> Ux;
        const M3<float> Vb =
            staple_sum_fused<NC, MU>(g, static_cast<const float *>(a.Usrc), x, a.c0_f, a.c1_f, R, Ux);
        ape_finish<float, NC, MU>(a, x, i, Vb, Ux, up);
    }
    count_update<float>(a.counters, up);
}

// End of one Runge-Kutta stage for link (MU, i) from its staple sum sig and
// link u: H_Z = -i h Q[W_i], H_S <- a H_Z + b H_S, W_{i+1} = exp(i c H_S) W_i.
template <class T, int NC, int MU>
__device__ __forceinline__ void flow_finish(const FlowParams &a, int i, const M3<T> &sig, const M3<T> &u,
                                            bool &used64, const T *s_old = nullptr) {
    const Geo &g = a.g;
    const bool f32 = sizeof(T) == 4;
    const T h = f32 ? T(a.h_f) : T(a.h), ca = f32 ? T(a.a_f) : T(a.a);
    const T cb = f32 ? T(a.b_f) : T(a.b), cc = f32 ? T(a.c_f) : T(a.c);
    T hz[9];
    stout_H<T>(sig, u, h, hz);
    T *S = static_cast<T *>(a.S) + (long long)MU * 9 * g.P;
    T hs[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        hs[k] = ca * hz[k];
        if (cb != T(0)) hs[k] = fma(cb, s_old ? s_old[k] : S[(long long)k * g.P + i], hs[k]);
        S[(long long)k * g.P + i] = hs[k];
    }
    const M3<T> E = exp_iH<T>(cc * hs[0], cc * hs[1], cc * hs[2], cc * hs[3], cc * hs[4], cc * hs[5],
                              cc * hs[6], cc * hs[7], cc * hs[8], used64);
    M3<T> un = m3_mul(E, u);
    if (NC == 12) rebuild_row2(un);
    store_link<T, NC>(static_cast<T *>(a.U), g.P, MU, i, un);
}

__device__ __forceinline__ void flow_count(const FlowParams &a, bool used64) {
    if (a.counters) {
        const unsigned fb = __ballot_sync(0xffffffffu, used64);
        if ((threadIdx.x & 31) == 0 && fb) atomicAdd(&a.counters[kCntSecond], (unsigned long long)__popc(fb));
    }
}

// One Runge-Kutta stage for every link of direction MU (thread t = site t in
// plane order), staples from plain loads (FP64, and FP32 without the ring).
template <class T, int NC, bool RECT, int MU>
__global__ void __launch_bounds__(VS_SUBSWEEP_THREADS, sizeof(T) == 4 ? VS_SUBSWEEP_MINB : 1)
    k_flow_stage(FlowParams a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool used64 = false;
    if (t < a.n_threads) {
        const Geo &g = a.g;
        const Pt x = dir_site<MU>(g, t);
        const int i = sidx(g, x);
        const T *Us = static_cast<const T *>(a.Usrc);
        const bool f32 = sizeof(T) == 4;
        const T c0 = f32 ? T(a.c0_f) : T(a.c0), c1 = f32 ? T(a.c1_f) : T(a.c1);
        const M3<T> sig = staple_sum<T, NC, RECT, MU>(g, Us, x, c0, c1);
        const M3<T> u = load_link<T, NC>(Us, g.P, MU, i);
        flow_finish<T, NC, MU>(a, i, sig, u, used64);
    }
    flow_count(a, used64);
}

// The same stage in FP32 with the staple links streamed through the per-thread
// cp.async ring: the one-pass stream of the class kernel for over-improved
// staples, the plaquette-staple ring for eps = 1.
template <int NC, bool RECT, int MU>
__global__ void __launch_bounds__(VS_RING_THREADS, RECT ? VS_RING_MINB : 4) k_flow_stage_ring(FlowParams a) {
    extern __shared__ float4 flow_dyn[];
    float4 *ring4 = flow_dyn;
    float2 *ring2 = reinterpret_cast<float2 *>(flow_dyn + 6 * (NC / 4) * VS_RING_THREADS);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool used64 = false;
    if (t < a.n_threads) {
        const Geo &g = a.g;
        const Pt x = dir_site<MU>(g, t);
        const int i = sidx(g, x);
        const float *Us = static_cast<const float *>(a.Usrc);
        LinkRing<NC> R = ring_of<NC>(ring4, ring2);
        M3<float> sig, u;
        // the exponent H_S of this link, read before the staple stream so that
        // its latency hides behind it (stage 1 of a step does not read it)
        float s_old[9];
        const float *Sp = static_cast<const float *>(a.S) + (long long)MU * 9 * g.P + i;
#pragma unroll
        for (int k = 0; k < 9; ++k) s_old[k] = a.b_f != 0.0f ? __ldg(Sp + (long long)k * g.P) : 0.0f;
        if constexpr (RECT) {
            sig = staple_sum_fused<NC, MU>(g, Us, x, a.c0_f, a.c1_f, R, u);
        } else {
            sig = staple_sum_plain_ring<NC, MU>(g, Us, x, a.c0_f, R);
            u = load_link<float, NC>(Us, g.P, MU, i);
        }
        flow_finish<float, NC, MU>(a, i, sig, u, used64, s_old);
    }
    flow_count(a, used64);
}

template <class T, int NC>
cudaError_t launch_ape_tpl(bool rect, int mu, const ApeParams &p, cudaStream_t st) {
    if (p.n_threads <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4 && VS_RING) {
        if (rect) {   // annealed classes and simultaneous sweeps alike
            const int rb = (p.n_threads + VS_RING_THREADS - 1) / VS_RING_THREADS;
            constexpr int sm = ring6_smem_bytes<NC>();
            static std::atomic<unsigned long long> attr_set{0};
            once_per_device(attr_set, [&] {
                cudaFuncSetAttribute(k_ape_ring<NC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_ape_ring<NC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_ape_ring<NC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_ape_ring<NC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            });
            switch (mu) {
                case 0: k_ape_ring<NC, 0><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 1: k_ape_ring<NC, 1><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 2: k_ape_ring<NC, 2><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                default: k_ape_ring<NC, 3><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
            }
            count_launches(1);
            return cudaGetLastError();
        }
    }
    const int threads = VS_SUBSWEEP_THREADS;
    const int blocks = (p.n_threads + threads - 1) / threads;
#define VS_LAUNCH(R, M) k_ape<T, NC, R, M><<<blocks, threads, 0, st>>>(p)
    if (rect) {
        switch (mu) {
            case 0: VS_LAUNCH(true, 0); break;
            case 1: VS_LAUNCH(true, 1); break;
            case 2: VS_LAUNCH(true, 2); break;
            default: VS_LAUNCH(true, 3); break;
        }
    } else {
        switch (mu) {
            case 0: VS_LAUNCH(false, 0); break;
            case 1: VS_LAUNCH(false, 1); break;
            case 2: VS_LAUNCH(false, 2); break;
            default: VS_LAUNCH(false, 3); break;
        }
    }
#undef VS_LAUNCH
    count_launches(1);
    return cudaGetLastError();
}

template <class T, int NC>
cudaError_t launch_flow_tpl(bool rect, int mu, const FlowParams &p, cudaStream_t st) {
    if (p.n_threads <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4 && VS_RING) {
        const int rb = (p.n_threads + VS_RING_THREADS - 1) / VS_RING_THREADS;
        constexpr int sm = ring6_smem_bytes<NC>();
        static std::atomic<unsigned long long> attr_set{0};
        once_per_device(attr_set, [&] {
            cudaFuncSetAttribute(k_flow_stage_ring<NC, true, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_flow_stage_ring<NC, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_flow_stage_ring<NC, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_flow_stage_ring<NC, true, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_flow_stage_ring<NC, false, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_flow_stage_ring<NC, false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_flow_stage_ring<NC, false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            cudaFuncSetAttribute(k_flow_stage_ring<NC, false, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
        });
#define VS_LAUNCH(R, M) k_flow_stage_ring<NC, R, M><<<rb, VS_RING_THREADS, sm, st>>>(p)
        if (rect) {
            switch (mu) {
                case 0: VS_LAUNCH(true, 0); break;
                case 1: VS_LAUNCH(true, 1); break;
                case 2: VS_LAUNCH(true, 2); break;
                default: VS_LAUNCH(true, 3); break;
            }
        } else {
            switch (mu) {
                case 0: VS_LAUNCH(false, 0); break;
                case 1: VS_LAUNCH(false, 1); break;
                case 2: VS_LAUNCH(false, 2); break;
                default: VS_LAUNCH(false, 3); break;
            }
        }
#undef VS_LAUNCH
        count_launches(1);
        return cudaGetLastError();
    }
    const int threads = VS_SUBSWEEP_THREADS;
    const int blocks = (p.n_threads + threads - 1) / threads;
#define VS_LAUNCH(R, M) k_flow_stage<T, NC, R, M><<<blocks, threads, 0, st>>>(p)
    if (rect) {
        switch (mu) {
            case 0: VS_LAUNCH(true, 0); break;
            case 1: VS_LAUNCH(true, 1); break;
            case 2: VS_LAUNCH(true, 2); break;
            default: VS_LAUNCH(true, 3); break;
        }
    } else {
        switch (mu) {
            case 0: VS_LAUNCH(false, 0); break;
            case 1: VS_LAUNCH(false, 1); break;
            case 2: VS_LAUNCH(false, 2); break;
            default: VS_LAUNCH(false, 3); break;
        }
    }
#undef VS_LAUNCH
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace vs
