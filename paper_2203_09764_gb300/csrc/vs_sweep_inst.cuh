// vs_sweep_inst.cuh -- instantiates the colour-class update kernel for one
// (precision, storage) pair.  Included by vs_sweep_f18.cu, vs_sweep_f12.cu and
// vs_sweep_d18.cu so the heavy instantiations compile in parallel.
#pragma once

#include "vs_internal.h"
#include "vs_stout.cuh"

namespace vs {

// FP64 re-decision of the candidates the FP32 class launch just made left to it.
template <int NC, bool RECT>
void launch_redecide(int mu, const SubsweepParams &p, cudaStream_t st) {
    switch (mu) {
        case 0: k_redecide<NC, RECT, 0><<<16, 32, 0, st>>>(p); break;
        case 1: k_redecide<NC, RECT, 1><<<16, 32, 0, st>>>(p); break;
        case 2: k_redecide<NC, RECT, 2><<<16, 32, 0, st>>>(p); break;
        default: k_redecide<NC, RECT, 3><<<16, 32, 0, st>>>(p); break;
    }
    count_launches(1);
}

template <class T, int NC>
cudaError_t launch_subsweep_tpl(bool rect, int mu, const SubsweepParams &p, cudaStream_t st) {
    if (p.n_threads <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4 && VS_RING) {
        // FP32: the cp.async link-ring kernels
        if (rect) {
            const int rb = (p.n_threads + VS_RING_THREADS - 1) / VS_RING_THREADS;
            constexpr int sm = ring6_smem_bytes<NC>();
            static std::atomic<unsigned long long> attr_set{0};
            once_per_device(attr_set, [&] {
                cudaFuncSetAttribute(k_subsweep_fused<NC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_subsweep_fused<NC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_subsweep_fused<NC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_subsweep_fused<NC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            });
            switch (mu) {
                case 0: k_subsweep_fused<NC, 0><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 1: k_subsweep_fused<NC, 1><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 2: k_subsweep_fused<NC, 2><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                default: k_subsweep_fused<NC, 3><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
            }
            count_launches(1);
            if (p.defer_idx) launch_redecide<NC, true>(mu, p, st);
            return cudaGetLastError();
        }
        {   // FP32 plaquette staples (eps = 1): the plaquette-staple link ring
            const int rb = (p.n_threads + VS_RING_THREADS - 1) / VS_RING_THREADS;
            constexpr int sm = ring6_smem_bytes<NC>();
            static std::atomic<unsigned long long> attr_set_p{0};
            once_per_device(attr_set_p, [&] {
                cudaFuncSetAttribute(k_subsweep_pring<NC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_subsweep_pring<NC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_subsweep_pring<NC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_subsweep_pring<NC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            });
            switch (mu) {
                case 0: k_subsweep_pring<NC, 0><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 1: k_subsweep_pring<NC, 1><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 2: k_subsweep_pring<NC, 2><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                default: k_subsweep_pring<NC, 3><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
            }
            count_launches(1);
            if (p.defer_idx) launch_redecide<NC, false>(mu, p, st);
            return cudaGetLastError();
        }
    }
    const int threads = VS_SUBSWEEP_THREADS;
    const int blocks = (p.n_threads + threads - 1) / threads;
#define VS_LAUNCH(R, M) k_subsweep<T, NC, R, M><<<blocks, threads, 0, st>>>(p)
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
    if constexpr (sizeof(T) == 4) {
        if (p.defer_idx) {
            if (rect) launch_redecide<NC, true>(mu, p, st);
            else launch_redecide<NC, false>(mu, p, st);
        }
    }
    return cudaGetLastError();
}

template <class T, int NC>
cudaError_t launch_aus_tpl(bool rect, int mu, const AusParams &p, cudaStream_t st) {
    if (p.n_threads <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4 && VS_RING) {
        // FP32: the link-ring kernels
        if (rect) {
            const int rb = (p.n_threads + VS_RING_THREADS - 1) / VS_RING_THREADS;
            constexpr int sm = ring6_smem_bytes<NC>();
            static std::atomic<unsigned long long> attr_set{0};
            once_per_device(attr_set, [&] {
                cudaFuncSetAttribute(k_aus_ring<NC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_aus_ring<NC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_aus_ring<NC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_aus_ring<NC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            });
            switch (mu) {
                case 0: k_aus_ring<NC, 0><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 1: k_aus_ring<NC, 1><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 2: k_aus_ring<NC, 2><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                default: k_aus_ring<NC, 3><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
            }
            count_launches(1);
            return cudaGetLastError();
        }
        {   // FP32 plaquette staples (cooling and eps = 1 AUS): the plaquette-staple ring
            const int rb = (p.n_threads + VS_RING_THREADS - 1) / VS_RING_THREADS;
            constexpr int sm = ring6_smem_bytes<NC>();
            static std::atomic<unsigned long long> attr_set_p{0};
            once_per_device(attr_set_p, [&] {
                cudaFuncSetAttribute(k_aus_pring<NC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_aus_pring<NC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_aus_pring<NC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
                cudaFuncSetAttribute(k_aus_pring<NC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
            });
            switch (mu) {
                case 0: k_aus_pring<NC, 0><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 1: k_aus_pring<NC, 1><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                case 2: k_aus_pring<NC, 2><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
                default: k_aus_pring<NC, 3><<<rb, VS_RING_THREADS, sm, st>>>(p); break;
            }
            count_launches(1);
            return cudaGetLastError();
        }
    }
    const int threads = VS_SUBSWEEP_THREADS;
    const int blocks = (p.n_threads + threads - 1) / threads;
#define VS_LAUNCH(R, M) k_aus<T, NC, R, M><<<blocks, threads, 0, st>>>(p)
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
