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
    const void *G;       // random gauge transformation (18 reals per site) or null
    int colour;          // 0..3, or -1: every site of direction mu
    int n_threads;
    double rho, c0, c1;
    float rho_f, c0_f, c1_f;   // the same, rounded once on the host for the FP32 kernels
    int vp;
    unsigned long long *counters;  // kSweepSlots counters of the sweep (kCnt*), or null
    // FP32 with vortex preservation and vs_anneal.fp64_redecide: candidates
    // within the FP32 band of a sector edge are left unwritten and listed here
    // for k_redecide (FP64); null: decided in FP32 and counted as undecidable
    int *defer_idx;       // [defer_cap] layout positions
    unsigned *defer_n;    // entries appended by the class launch (may exceed defer_cap)
    unsigned *defer_done; // blocks of k_redecide that have finished (reset by the last)
    int defer_cap;
};

// Counter slots of one sweep, filled by the colour-class kernels of the
// stout, AUS and APE/UCP smoothers (the Runge-Kutta flow uses the second
// only).  kCntMarginSine holds the smallest sine of a candidate's angular
// margin from a sector edge as the bits of a non-negative double; it starts
// at kMarginInit (above any sine).
enum {
    kCntReject = 0,       // vortex-preservation rejections
    kCntSecond = 1,       // FP32: FP64 exponential coefficients; APE: singular blocked matrices
    kCntLabelDiff = 2,    // candidates whose Z(3) label differs from the reference
    kCntUndecidable = 3,  // candidates whose trace lies within the precision's error band of an edge
    kCntMarginSine = 4,
    kCntRedecided = 5,    // FP32 candidates re-decided in FP64 (k_redecide)
    kSweepSlots = 8
};
constexpr unsigned long long kMarginInit = 0x7f7f7f7f7f7f7f7full;   // a double of about 1.4e306

// Capacity of a field's list of FP32 candidates left to k_redecide per class
// launch (a launch that defers more decides the rest in FP32, counted as
// undecidable).
constexpr int kDeferCap = 16384;

// process-wide count of direct kernel launches
void count_launches(int n);
long long launches();

// One colour class of annealed U-link smearing with MaxReTr (Sec. III):
// V = (1 - alpha) U + (alpha / 6) Sigma(eps); n_hits passes over the SU(2)
// subgroups; optional vortex preservation.  alpha = 1, eps = 1 is cooling.
struct AusParams {
    Geo g;
    void *U;
    const int8_t *ref;
    const void *G;       // random gauge transformation or null
    int colour;
    int n_threads;
    double alpha, c0, c1;
    float alpha_f, c0_f, c1_f;
    int n_hits;
    int vp;
    unsigned long long *counters;  // kSweepSlots counters of the sweep (kCnt*), or null
};

// One colour class (or, colour < 0, every link of direction mu) of APE
// blocking with unit circle projection (Sec. II.C): V = (1 - alpha) U +
// (alpha / 6) Sigma(eps), U <- P_ucp{V}; optional vortex preservation.
struct ApeParams {
    Geo g;
    void *U;             // destination (in place for the annealed schedule)
    const void *Usrc;    // blocking source: == U (annealed) or the previous field
    const int8_t *ref;
    const void *G;       // random gauge transformation or null
    int colour;
    int n_threads;
    double alpha, c0, c1;
    float alpha_f, c0_f, c1_f;
    int vp;
    unsigned long long *counters;  // kSweepSlots counters of the sweep (kCntSecond: singular), or null
};

// One stage of the third-order Runge-Kutta Wilson flow for every link of
// direction mu: with H_Z the Hermitian form of h Q[W_i] (Eq. generator),
// H_S <- a H_Z + b H_S (b = 0: H_S not read), W_{i+1} = exp(i c H_S) W_i.
struct FlowParams {
    Geo g;
    void *U;             // W_{i+1}
    const void *Usrc;    // W_i
    void *S;             // H_S, 9 reals per link [mu][9][P] in the field precision
    int n_threads;
    double h, a, b, c, c0, c1;
    float h_f, a_f, b_f, c_f, c0_f, c1_f;
    unsigned long long *counters;  // kCntSecond: FP64 exponentials of the step (may be null)
};

cudaError_t launch_ape_f18(bool rect, int mu, const ApeParams &p, cudaStream_t st);
cudaError_t launch_ape_f12(bool rect, int mu, const ApeParams &p, cudaStream_t st);
cudaError_t launch_ape_d18(bool rect, int mu, const ApeParams &p, cudaStream_t st);
cudaError_t launch_flow_f18(bool rect, int mu, const FlowParams &p, cudaStream_t st);
cudaError_t launch_flow_f12(bool rect, int mu, const FlowParams &p, cudaStream_t st);
cudaError_t launch_flow_d18(bool rect, int mu, const FlowParams &p, cudaStream_t st);

cudaError_t launch_aus_f18(bool rect, int mu, const AusParams &p, cudaStream_t st);
cudaError_t launch_aus_f12(bool rect, int mu, const AusParams &p, cudaStream_t st);
cudaError_t launch_aus_d18(bool rect, int mu, const AusParams &p, cudaStream_t st);

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
cudaError_t launch_store_ref(const Geo &g, const int8_t *lab_lex, int8_t *ref, cudaStream_t st);
cudaError_t launch_count_nonfinite(int prec, int nc, const Geo &g, const void *U, unsigned long long *count,
                                   cudaStream_t st);
cudaError_t launch_current_labels(int prec, int nc, const Geo &g, const void *U, int8_t *out_lex,
                                  cudaStream_t st);
cudaError_t launch_centrifuge(int prec, int nc, const Geo &g, const int8_t *ref, double omega,
                              uint64_t seed, void *U, cudaStream_t st);
// mean over sites of S(x)/beta into *out (device double); partials: n_part doubles
int action_partials(const Geo &g);
cudaError_t launch_action(int prec, int nc, const Geo &g, const void *U, double *partials,
                          double *out, cudaStream_t st);
// <S>/beta, <S_R>/beta and Q into out[0..2]; partials: 3 x 400 doubles;
// optional per-site densities in lexicographic order
cudaError_t launch_observables(int prec, int nc, const Geo &g, const void *U, double *partials, double *out,
                               double *S_site, double *SR_site, double *q_site, cudaStream_t st);
// C = <a b> / sqrt(<a^2> <b^2>) of two device densities of n values into out[0]
// (out[1..3]: the sums of a b, a^2, b^2); partials: 3 x 400 doubles
cudaError_t launch_correlation(const double *a, const double *b, long long n, double *partials, double *out,
                               cudaStream_t st);
// counts[0] label diffs, counts[1] charge diffs, counts[2] near-boundary links;
// margin_bits: min angular margin as the bit pattern of a non-negative double
cudaError_t launch_vortex(int prec, int nc, const Geo &g, const void *U, const int8_t *ref,
                          int8_t *cur, unsigned long long *counts,
                          unsigned long long *margin_bits, cudaStream_t st, const void *G = nullptr);
// load the vortex-check kernels now (a first launch would, with lazy loading)
cudaError_t preload_vortex_kernels();
cudaError_t launch_reunit(int prec, int nc, const Geo &g, void *U, const int8_t *ref, cudaStream_t st,
                          const void *G = nullptr);
// random gauge transformation: store G (FP64 host layout [V][3][3][2], on the
// device) in the field precision, and transform every link
cudaError_t launch_gauge(int prec, int nc, const Geo &g, const double *G_lex, void *Gs, void *U,
                         cudaStream_t st);
cudaError_t launch_debug_expm(int prec, const double *X, int n, double *E, cudaStream_t st);
cudaError_t launch_haar(int prec, int nc, const Geo &g, uint64_t seed, void *U, cudaStream_t st);
cudaError_t launch_aus_class(int prec, int nc, bool rect, int mu, const AusParams &p, cudaStream_t st);
cudaError_t launch_project(int prec, int nc, const Geo &g, void *U, int8_t *ref, cudaStream_t st);

}  // namespace vs
