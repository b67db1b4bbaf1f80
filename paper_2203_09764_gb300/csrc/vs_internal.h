// vs_internal.h -- declarations shared between the kernel and ABI translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "vs_device.cuh"

namespace vs {

struct SubsweepParams {
    Geo g;
    void *U;             // field being updated (in place for the annealed schedule)
    const void *Usrc;    // staple source: == U (annealed) or the previous field (simultaneous)
    const int8_t *ref;   // reference labels [4][P]
    int colour;          // 0..3, or -1: every site of direction mu
    int n_threads;
    double rho, c0, c1;
    int vp;
    unsigned long long *counters;  // [0] rejects, [1] FP64 exponentials (may be null)
};

// process-wide count of direct kernel launches
void count_launches(int n);
long long launches();

cudaError_t launch_subsweep_f18(bool rect, int mu, const SubsweepParams &p, cudaStream_t st);
cudaError_t launch_subsweep_f12(bool rect, int mu, const SubsweepParams &p, cudaStream_t st);
cudaError_t launch_subsweep_d18(bool rect, int mu, const SubsweepParams &p, cudaStream_t st);

// prec: 0 = double, 1 = float; nc: 18 or 12
cudaError_t launch_load_labels(int prec, int nc, const Geo &g, const int8_t *lab_lex, void *U,
                               int8_t *ref, cudaStream_t st);
cudaError_t launch_load_links(int prec, int nc, const Geo &g, const double *links_lex, void *U,
                              int8_t *ref, cudaStream_t st);
cudaError_t launch_read_links(int prec, int nc, const Geo &g, const void *U, double *out_lex,
                              cudaStream_t st);
cudaError_t launch_read_labels(const Geo &g, const int8_t *ref, int8_t *out_lex, cudaStream_t st);
cudaError_t launch_current_labels(int prec, int nc, const Geo &g, const void *U, int8_t *out_lex,
                                  cudaStream_t st);
cudaError_t launch_centrifuge(int prec, int nc, const Geo &g, const int8_t *ref, double omega,
                              uint64_t seed, void *U, cudaStream_t st);
// mean over sites of S(x)/beta into *out (device double); partials: n_part doubles
int action_partials(const Geo &g);
cudaError_t launch_action(int prec, int nc, const Geo &g, const void *U, double *partials,
                          double *out, cudaStream_t st);
// counts[0] label diffs, counts[1] charge diffs, counts[2] near-boundary links;
// margin_bits: min angular margin as the bit pattern of a non-negative double
cudaError_t launch_vortex(int prec, int nc, const Geo &g, const void *U, const int8_t *ref,
                          int8_t *cur, unsigned long long *counts,
                          unsigned long long *margin_bits, cudaStream_t st);
cudaError_t launch_reunit(int prec, int nc, const Geo &g, void *U, const int8_t *ref, cudaStream_t st);
cudaError_t launch_debug_expm(int prec, const double *X, int n, double *E, cudaStream_t st);
cudaError_t launch_haar(int prec, int nc, const Geo &g, uint64_t seed, void *U, cudaStream_t st);
cudaError_t launch_cool_class(int prec, int nc, const Geo &g, int mu, int colour, void *U,
                              cudaStream_t st);
cudaError_t launch_project(int prec, int nc, const Geo &g, void *U, int8_t *ref, cudaStream_t st);

}  // namespace vs
