/*
 * vs_oracle.c -- plain, slow FP64 CPU oracle for vortex-field smoothing.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: own complex arithmetic (C99 double complex), own lattice
 * geometry, own label rule, own exponential, own random-pair generator.
 *
 * Source: Virgili, Kamleh & Leinweber, "Smoothing algorithms for projected
 * center-vortex gauge fields", arXiv:2203.09764.  Each function cites the
 * section / equation it follows.  Where the paper is silent the reading used
 * is stated at the function.
 *
 * Layouts:
 *   dims[4] = {Lx, Ly, Lz, Lt}; site s = x + Lx*(y + Ly*(z + Lz*t)).
 *   links   double[4][V][3][3][2]  (== double complex [4][V][3][3], row major).
 *   labels  int8_t[4][V] in {-1, 0, +1}.
 *
 * Every entry point returns 0 on success and a negative value on bad input.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;
typedef struct { cplx m[3][3]; } mat3;

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* 3x3 complex matrix algebra                                                */
/* ------------------------------------------------------------------------ */

static mat3 m_zero(void) { mat3 r; memset(&r, 0, sizeof r); return r; }

static mat3 m_eye(void) {
    mat3 r = m_zero();
    for (int i = 0; i < 3; ++i) r.m[i][i] = 1.0;
    return r;
}

static mat3 m_mul(const mat3 *a, const mat3 *b) {
    mat3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx s = 0.0;
            for (int k = 0; k < 3; ++k) s += a->m[i][k] * b->m[k][j];
            r.m[i][j] = s;
        }
    return r;
}

static mat3 m_dag(const mat3 *a) {
    mat3 r;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.m[i][j] = conj(a->m[j][i]);
    return r;
}

static void m_axpy(mat3 *y, cplx a, const mat3 *x) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) y->m[i][j] += a * x->m[i][j];
}

static cplx m_trace(const mat3 *a) { return a->m[0][0] + a->m[1][1] + a->m[2][2]; }

/* ------------------------------------------------------------------------ */
/* Lattice geometry (periodic)                                               */
/* ------------------------------------------------------------------------ */

typedef struct { int L[4]; long V; } lattice;

static int lat_init(lattice *g, const int32_t dims[4]) {
    g->V = 1;
    for (int d = 0; d < 4; ++d) {
        if (dims[d] < 1) return -1;
        g->L[d] = dims[d];
        g->V *= dims[d];
    }
    return 0;
}

static long lat_site(const lattice *g, const int x[4]) {
    return x[0] + (long)g->L[0] * (x[1] + (long)g->L[1] * (x[2] + (long)g->L[2] * x[3]));
}

static void lat_coords(const lattice *g, long s, int x[4]) {
    for (int d = 0; d < 4; ++d) { x[d] = (int)(s % g->L[d]); s /= g->L[d]; }
}

static void lat_move(const lattice *g, int x[4], int d, int sgn) {
    x[d] = ((x[d] + sgn) % g->L[d] + g->L[d]) % g->L[d];
}

static mat3 link_get(const lattice *g, const cplx *U, int mu, long s) {
    mat3 r;
    memcpy(&r, U + ((long)mu * g->V + s) * 9, sizeof r);
    return r;
}

static void link_put(const lattice *g, cplx *U, int mu, long s, const mat3 *a) {
    memcpy(U + ((long)mu * g->V + s) * 9, a, sizeof *a);
}

/* One step of a lattice path: U_d(y) forwards, U_d^dagger(y - d) backwards. */
typedef struct { int d, sgn; } pstep;

/* Ordered product of links along a path starting at x; end receives the
 * final site.  This is the definition of a Wilson line on the lattice
 * (Sec. II, the staple and plaquette definitions). */
static mat3 path_product(const lattice *g, const cplx *U, const int x[4],
                         const pstep *p, int n, int end[4]) {
    int y[4] = {x[0], x[1], x[2], x[3]};
    mat3 acc = m_eye();
    for (int i = 0; i < n; ++i) {
        mat3 l;
        if (p[i].sgn > 0) {
            l = link_get(g, U, p[i].d, lat_site(g, y));
            lat_move(g, y, p[i].d, +1);
        } else {
            lat_move(g, y, p[i].d, -1);
            mat3 t = link_get(g, U, p[i].d, lat_site(g, y));
            l = m_dag(&t);
        }
        acc = m_mul(&acc, &l);
    }
    memcpy(end, y, sizeof y);
    return acc;
}

/* ------------------------------------------------------------------------ */
/* Z(3) projection, Eq. (centre_project) / (centre_element)                  */
/* ------------------------------------------------------------------------ */

/* Label n of a matrix from the sector of arg Tr M.  The paper's intervals are
 * open; on their common end points this oracle reads: arg in [pi/3, pi] -> +1
 * and arg in (-pi, -pi/3] -> -1 (atan2 convention, with -0 taken as +0), and
 * Tr M = 0 -> 0. */
static int label_of_trace(cplx t) {
    double a = creal(t), b = cimag(t) + 0.0;
    double arg = atan2(b, a);
    if (arg > -OR_PI / 3.0 && arg < OR_PI / 3.0) return 0;
    return arg > 0.0 ? +1 : -1;
}

/* Angular distance of arg Tr M from the nearest sector boundary: the sector
 * edges of Eq. (centre_element) lie at arg = pi/3, -pi/3 and pi (= -pi). */
static double margin_of_trace(cplx t) {
    double a = creal(t), b = cimag(t) + 0.0;
    double arg = atan2(b, a);
    double d1 = fabs(arg - OR_PI / 3.0), d2 = fabs(arg + OR_PI / 3.0), d3 = OR_PI - fabs(arg);
    double m = d1 < d2 ? d1 : d2;
    return m < d3 ? m : d3;
}

/* Trace tested by vortex preservation (Sec. VI).  In the gauge of the
 * original field (G == NULL) it is Tr U'; after the random gauge
 * transformation G it is Tr[G^dag(x) U' G(x + mu)], the candidate transformed
 * back to the original gauge. */
static cplx vp_trace(const int L[4], long V, const cplx *G, int mu, const int x[4], const mat3 *Un) {
    if (!G) return m_trace(Un);
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] = (y[mu] + 1) % L[mu];
    long sx = x[0] + (long)L[0] * (x[1] + (long)L[1] * (x[2] + (long)L[2] * x[3]));
    long sy = y[0] + (long)L[0] * (y[1] + (long)L[1] * (y[2] + (long)L[2] * y[3]));
    (void)V;
    mat3 Gx, Gy;
    memcpy(&Gx, G + sx * 9, sizeof Gx);
    memcpy(&Gy, G + sy * 9, sizeof Gy);
    mat3 Gxd = m_dag(&Gx);
    mat3 t = m_mul(&Gxd, Un);
    t = m_mul(&t, &Gy);
    return m_trace(&t);
}

int or_label_matrix(const double *M18) {
    mat3 a;
    memcpy(&a, M18, sizeof a);
    return label_of_trace(m_trace(&a));
}

int or_labels(const int32_t dims[4], const double *links, int8_t *labels, double *margin_out) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    const cplx *U = (const cplx *)links;
    for (long i = 0; i < 4 * g.V; ++i) {
        mat3 a;
        memcpy(&a, U + i * 9, sizeof a);
        labels[i] = (int8_t)label_of_trace(m_trace(&a));
        if (margin_out) margin_out[i] = margin_of_trace(m_trace(&a));
    }
    return 0;
}

/* Z_mu(x) = exp(2 pi i n / 3) * identity, Eq. (centre_project). */
int or_links_from_labels(const int32_t dims[4], const int8_t *labels, double *links) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    cplx *U = (cplx *)links;
    for (long i = 0; i < 4 * g.V; ++i) {
        if (labels[i] < -1 || labels[i] > 1) return -2;
        cplx z = cexp(I * 2.0 * OR_PI * labels[i] / 3.0);
        mat3 a = m_zero();
        for (int k = 0; k < 3; ++k) a.m[k][k] = z;
        memcpy(U + i * 9, &a, sizeof a);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Counter-mode SplitMix64 (Steele, Lea & Flood 2014)                        */
/* ------------------------------------------------------------------------ */

uint64_t or_splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Random pair choice of the centrifuge: value (mu*V + s) of stream `seed`,
 * reduced mod 3, selects (j,k) = (1,2), (2,3) or (3,1).  The paper only says
 * the pair is selected at random per link (Sec. IV). */
int or_centrifuge_pair(uint64_t seed, long V, int mu, long s) {
    return (int)(or_splitmix64(seed, (uint64_t)mu * (uint64_t)V + (uint64_t)s) % 3ULL);
}

/* ------------------------------------------------------------------------ */
/* Centrifuge preconditioning, Sec. IV, Eqs. (lambda_j), (lambda_k)         */
/* ------------------------------------------------------------------------ */

/* From the labels n (the original vortex field in non-compact form,
 * lambda = 2 pi n / 3), every link at once: staple phase sigma, random pair
 * (j,k), lambda^j = (1-w) lambda + w sigma, lambda^k = (1+w) lambda - w sigma,
 * the third phase unchanged.  All sigma use the original phases (the update
 * is applied to "each original link").  sigma_out (optional) receives sigma. */
int or_centrifuge(const int32_t dims[4], const int8_t *labels, double omega, uint64_t seed,
                  double *links, double *sigma_out) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    if (!(omega >= 0.0 && omega < 0.25)) return -2;
    cplx *U = (cplx *)links;
    static const int pj[3] = {0, 1, 2}, pk[3] = {1, 2, 0};
    for (int mu = 0; mu < 4; ++mu)
        for (long s = 0; s < g.V; ++s) {
            int x[4];
            lat_coords(&g, s, x);
#define LAM(d, y) (2.0 * OR_PI * labels[(long)(d) * g.V + lat_site(&g, (y))] / 3.0)
            double sum = 0.0;
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) continue;
                int xp_nu[4], xp_mu[4], xm_nu[4], xm_nu_p_mu[4];
                memcpy(xp_nu, x, sizeof x); lat_move(&g, xp_nu, nu, +1);
                memcpy(xp_mu, x, sizeof x); lat_move(&g, xp_mu, mu, +1);
                memcpy(xm_nu, x, sizeof x); lat_move(&g, xm_nu, nu, -1);
                memcpy(xm_nu_p_mu, xm_nu, sizeof x); lat_move(&g, xm_nu_p_mu, mu, +1);
                sum += LAM(nu, x) + LAM(mu, xp_nu) - LAM(nu, xp_mu)
                     - LAM(nu, xm_nu) + LAM(mu, xm_nu) + LAM(nu, xm_nu_p_mu);
            }
            double sigma = sum / 6.0;
            double lam = LAM(mu, x);
#undef LAM
            int p = or_centrifuge_pair(seed, g.V, mu, s);
            double ph[3] = {lam, lam, lam};
            ph[pj[p]] = (1.0 - omega) * lam + omega * sigma;
            ph[pk[p]] = (1.0 + omega) * lam - omega * sigma;
            mat3 a = m_zero();
            for (int k = 0; k < 3; ++k) a.m[k][k] = cexp(I * ph[k]);
            link_put(&g, U, mu, s, &a);
            if (sigma_out) sigma_out[(long)mu * g.V + s] = sigma;
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Staples, Eq. (plaq_staples) and Eq. (over-improvement)                    */
/* ------------------------------------------------------------------------ */

/* Over-improvement coefficients: c0 = (5 - 2 eps)/3 on the plaquette staples,
 * c1 = (eps - 1)/(12 u0^2) on the rectangles; eps = 1 gives c0 = 1, c1 = 0. */
void or_overimproved_coeffs(double eps, double u0, double *c0, double *c1) {
    *c0 = (5.0 - 2.0 * eps) / 3.0;
    *c1 = (eps - 1.0) / (12.0 * u0 * u0);
}

/* Sigma_mu(x) = c0 * sum_{nu != mu, +-} (3-link staple)
 *             + c1 * sum_{nu != mu, +-} (the three 5-link rectangle paths),
 * every path running from x to x + mu.  The paths are read off the diagrams
 * of Eq. (over-improvement) (drawn there for Sigma^dagger):
 *   staple    : +nu, +mu, -nu
 *   tall      : +nu, +nu, +mu, -nu, -nu
 *   wide fwd  : +nu, +mu, +mu, -nu, -mu
 *   wide bwd  : -mu, +nu, +mu, +mu, -nu
 * and the same with nu -> -nu.  That is 6 staples and 18 rectangles. */
static int staple_sum(const lattice *g, const cplx *U, int mu, const int x[4],
                      double c0, double c1, mat3 *S) {
    *S = m_zero();
    int target[4];
    memcpy(target, x, sizeof target);
    lat_move(g, target, mu, +1);
    for (int nu = 0; nu < 4; ++nu) {
        if (nu == mu) continue;
        for (int s = -1; s <= 1; s += 2) {
            const pstep staple[3] = {{nu, s}, {mu, +1}, {nu, -s}};
            const pstep tall[5] = {{nu, s}, {nu, s}, {mu, +1}, {nu, -s}, {nu, -s}};
            const pstep wfwd[5] = {{nu, s}, {mu, +1}, {mu, +1}, {nu, -s}, {mu, -1}};
            const pstep wbwd[5] = {{mu, -1}, {nu, s}, {mu, +1}, {mu, +1}, {nu, -s}};
            int end[4];
            mat3 p = path_product(g, U, x, staple, 3, end);
            if (memcmp(end, target, sizeof end)) return -1;
            m_axpy(S, c0, &p);
            if (c1 != 0.0) {
                const pstep *rp[3] = {tall, wfwd, wbwd};
                for (int r = 0; r < 3; ++r) {
                    p = path_product(g, U, x, rp[r], 5, end);
                    if (memcmp(end, target, sizeof end)) return -1;
                    m_axpy(S, c1, &p);
                }
            }
        }
    }
    return 0;
}

int or_staple_sum(const int32_t dims[4], const double *links, int mu, const int32_t x32[4],
                  double c0, double c1, double *S18) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    int x[4] = {x32[0], x32[1], x32[2], x32[3]};
    mat3 S;
    if (staple_sum(&g, (const cplx *)links, mu, x, c0, c1, &S)) return -2;
    memcpy(S18, &S, sizeof S);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Stout step, Eqs. (stout) and (generator)                                  */
/* ------------------------------------------------------------------------ */

/* Matrix exponential by its defining power series, 40 terms:
 * exp(X) = sum_{n=0}^{39} X^n / n!. */
static mat3 expm_series(const mat3 *X) {
    mat3 E = m_eye(), term = m_eye();
    for (int n = 1; n < 40; ++n) {
        term = m_mul(&term, X);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) term.m[i][j] /= (double)n;
        m_axpy(&E, 1.0, &term);
    }
    return E;
}

int or_expm(const double *X18, double *E18) {
    mat3 X, E;
    memcpy(&X, X18, sizeof X);
    E = expm_series(&X);
    memcpy(E18, &E, sizeof E);
    return 0;
}

/* Omega = Sigma U^dagger; Q = (Omega - Omega^dag)/2 - Tr(Omega - Omega^dag)/6;
 * candidate = exp(rho Q) U. */
static mat3 stout_candidate(const mat3 *S, const mat3 *Ux, double rho) {
    mat3 Ud = m_dag(Ux);
    mat3 Om = m_mul(S, &Ud);
    mat3 Omd = m_dag(&Om);
    mat3 A = Om;
    m_axpy(&A, -1.0, &Omd);
    cplx trA = m_trace(&A);
    mat3 X = m_zero();
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx q = 0.5 * A.m[i][j] - (i == j ? trA / 6.0 : 0.0);
            X.m[i][j] = rho * q;
        }
    mat3 E = expm_series(&X);
    return m_mul(&E, Ux);
}

int or_stout_generator(const double *Omega18, double *Q18) {
    mat3 Om, Q;
    memcpy(&Om, Omega18, sizeof Om);
    mat3 Omd = m_dag(&Om);
    mat3 A = Om;
    m_axpy(&A, -1.0, &Omd);
    cplx trA = m_trace(&A);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Q.m[i][j] = 0.5 * A.m[i][j] - (i == j ? trA / 6.0 : 0.0);
    memcpy(Q18, &Q, sizeof Q);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Annealed schedule (Sec. III.A: masked parallel updates)                   */
/* ------------------------------------------------------------------------ */

/* Reading of "appropriate masking": the links of direction mu are split into
 * four classes c_mu(x) = (2 x_mu + sum_{nu != mu} x_nu) mod 4.  A sweep visits
 * mu = 0..3, then c = 0..3, then the sites of the class in lexicographic
 * order, updating each link in place from the current field. */
int or_colour(const int32_t dims[4], int mu, const int32_t x[4]) {
    (void)dims;
    int c = 2 * x[mu];
    for (int nu = 0; nu < 4; ++nu)
        if (nu != mu) c += x[nu];
    return c % 4;
}

static long class_sites(const lattice *g, int mu, int c, long *out) {
    long n = 0;
    for (long s = 0; s < g->V; ++s) {
        int x[4];
        lat_coords(g, s, x);
        int cc = 2 * x[mu];
        for (int nu = 0; nu < 4; ++nu)
            if (nu != mu) cc += x[nu];
        if (cc % 4 == c) out[n++] = s;
    }
    return n;
}

enum { OR_ANNEALED = 0, OR_SIMULTANEOUS = 1 };

/* n_sweeps of stout smoothing in place.
 *   rho[sweep]   step size per sweep (Wilson-flow Euler step, Sec. V.B).
 *   eps, u0      over-improvement parameters (eps = 1: standard staples).
 *   schedule     OR_ANNEALED (one link at a time in the colour order above)
 *                or OR_SIMULTANEOUS (every link from the previous field).
 *   ref_labels   original vortex labels n_mu(x); with vp != 0 a candidate is
 *                accepted only if its label equals the original one (Sec. VI).
 *   n_reject     optional [n_sweeps] rejected-candidate counts.
 *   nthreads     1 = strictly sequential; >1 runs the sites of one colour
 *                class concurrently (they are independent by construction).
 *   cand_margin  optional [4][V]: angular distance of arg Tr of each link's
 *                last candidate from the nearest sector edge (last sweep).
 *   rejected     optional [4][V]: 1 where the last sweep rejected the candidate.
 *   gauge        optional [V][3][3] complex: the random gauge transformation
 *                G applied to the field (Sec. V.D); vortex preservation then
 *                tests the label of G^dag(x) U' G(x+mu) (Sec. VI). */
int or_smooth(const int32_t dims[4], double *links, const int8_t *ref_labels, int n_sweeps,
              const double *rho, double eps, double u0, int schedule, int vp,
              int64_t *n_reject, int nthreads, double *cand_margin, int8_t *rejected,
              const double *gauge) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    if (n_sweeps < 0) return -2;
    for (int d = 0; d < 4; ++d)
        if (schedule == OR_ANNEALED && g.L[d] % 4) return -3;
    if (vp && !ref_labels) return -4;
    double c0, c1;
    or_overimproved_coeffs(eps, u0, &c0, &c1);
    cplx *U = (cplx *)links;
    const cplx *G = (const cplx *)gauge;
    long *sites = (long *)malloc(sizeof(long) * g.V);
    cplx *old = NULL;
    if (schedule == OR_SIMULTANEOUS) old = (cplx *)malloc(sizeof(cplx) * 9 * 4 * g.V);
    if (!sites || (schedule == OR_SIMULTANEOUS && !old)) { free(sites); free(old); return -5; }
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#endif
    int err = 0;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        int64_t rej = 0;
        if (schedule == OR_ANNEALED) {
            for (int mu = 0; mu < 4; ++mu)
                for (int c = 0; c < 4; ++c) {
                    long n = class_sites(&g, mu, c, sites);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static) reduction(+ : rej) reduction(| : err)
#endif
                    for (long i = 0; i < n; ++i) {
                        int x[4];
                        lat_coords(&g, sites[i], x);
                        mat3 S;
                        if (staple_sum(&g, U, mu, x, c0, c1, &S)) { err |= 1; continue; }
                        mat3 Ux = link_get(&g, U, mu, sites[i]);
                        mat3 Un = stout_candidate(&S, &Ux, rho[sw]);
                        const long li = (long)mu * g.V + sites[i];
                        const cplx tr = vp_trace(g.L, g.V, G, mu, x, &Un);
                        if (cand_margin) cand_margin[li] = margin_of_trace(tr);
                        if (rejected) rejected[li] = 0;
                        if (vp && label_of_trace(tr) != ref_labels[li]) {
                            rej += 1;
                            if (rejected) rejected[li] = 1;
                            continue;
                        }
                        link_put(&g, U, mu, sites[i], &Un);
                    }
                }
        } else {
            memcpy(old, U, sizeof(cplx) * 9 * 4 * g.V);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static) reduction(+ : rej) reduction(| : err)
#endif
            for (long i = 0; i < 4 * g.V; ++i) {
                int mu = (int)(i / g.V);
                long s = i % g.V;
                int x[4];
                lat_coords(&g, s, x);
                mat3 S;
                if (staple_sum(&g, old, mu, x, c0, c1, &S)) { err |= 1; continue; }
                mat3 Ux = link_get(&g, old, mu, s);
                mat3 Un = stout_candidate(&S, &Ux, rho[sw]);
                const cplx tr = vp_trace(g.L, g.V, G, mu, x, &Un);
                if (cand_margin) cand_margin[i] = margin_of_trace(tr);
                if (rejected) rejected[i] = 0;
                if (vp && label_of_trace(tr) != ref_labels[i]) {
                    rej += 1;
                    if (rejected) rejected[i] = 1;
                    continue;
                }
                link_put(&g, U, mu, s, &Un);
            }
        }
        if (n_reject) n_reject[sw] = rej;
    }
    free(sites);
    free(old);
    return err ? -6 : 0;
}

/* ------------------------------------------------------------------------ */
/* Observables                                                               */
/* ------------------------------------------------------------------------ */

/* Wilson action density, Sec. V: S(x) = beta/(2 nc nd (nd-1)) *
 * sum_{mu != nu} Re Tr[1 - P_munu(x)], nc = 3, nd = 4, reported with
 * beta = 1.  Returns the lattice mean <S>; S_site (optional) gets S(x). */
int or_action(const int32_t dims[4], const double *links, double *mean_S, double *S_site) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    const cplx *U = (const cplx *)links;
    double total = 0.0;
    for (long s = 0; s < g.V; ++s) {
        int x[4];
        lat_coords(&g, s, x);
        double Sx = 0.0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) {
                if (mu == nu) continue;
                /* P_munu(x) = U_mu(x) U_nu(x+mu) U_mu^dag(x+nu) U_nu^dag(x) */
                const pstep plaq[4] = {{mu, +1}, {nu, +1}, {mu, -1}, {nu, -1}};
                int end[4];
                mat3 P = path_product(&g, U, x, plaq, 4, end);
                Sx += creal(3.0 - m_trace(&P));
            }
        Sx /= (2.0 * 3.0 * 4.0 * 3.0);
        if (S_site) S_site[s] = Sx;
        total += Sx;
    }
    *mean_S = total / (double)g.V;
    return 0;
}

/* Clover-leaf field strength (Sec. V, Eq. 1LFST), in lattice units (the
 * coupling of Eq. 1LFST absorbed into F): C_munu(x) is the mean of the four
 * plaquette leaves of the (mu, nu) plane that start and end at x, all with
 * the same orientation; F_munu = (C - C^dag)/(2i) with its trace removed. */
static mat3 clover_F(const lattice *g, const cplx *U, const int x[4], int mu, int nu) {
    const pstep leaves[4][4] = {{{mu, +1}, {nu, +1}, {mu, -1}, {nu, -1}},
                                {{nu, +1}, {mu, -1}, {nu, -1}, {mu, +1}},
                                {{mu, -1}, {nu, -1}, {mu, +1}, {nu, +1}},
                                {{nu, -1}, {mu, +1}, {nu, +1}, {mu, -1}}};
    mat3 C = m_zero();
    for (int l = 0; l < 4; ++l) {
        int end[4];
        mat3 P = path_product(g, U, x, leaves[l], 4, end);
        m_axpy(&C, 0.25, &P);
    }
    mat3 Cd = m_dag(&C);
    mat3 F;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F.m[i][j] = (C.m[i][j] - Cd.m[i][j]) / (2.0 * I);
    cplx tr = m_trace(&F) / 3.0;
    for (int i = 0; i < 3; ++i) F.m[i][i] -= tr;
    return F;
}

static int levi_civita(int a, int b, int c, int d) {
    int p[4] = {a, b, c, d}, sgn = 1;
    for (int i = 0; i < 4; ++i)
        for (int j = i + 1; j < 4; ++j) {
            if (p[i] == p[j]) return 0;
            if (p[i] > p[j]) sgn = -sgn;
        }
    return sgn;
}

/* Smoothness observables, Sec. V:
 *   q(x) = 1/(32 pi^2) eps_{mu nu rho sigma} Tr[F_munu(x) F_rhosigma(x)]  (Eq. 1LTopQ),
 *   S_R(x)/beta = 1/72 sum_{mu != nu} (1/2) Tr[F_munu(x) F_munu(x)],
 * the reconstructed action normalised so that S_R -> S on smooth fields
 * (P = exp(i theta) gives Re Tr(1 - P) = Tr(theta^2)/2 + O(theta^4) and
 * F = theta + O(theta^3)); the paper's print of this normalisation is garbled.
 * Outputs the means <S_R>/beta and the total charge Q = sum_x q(x), and
 * optionally the densities. */
int or_observables(const int32_t dims[4], const double *links, double *mean_SR, double *Q,
                   double *SR_site, double *q_site) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    const cplx *U = (const cplx *)links;
    double sr_tot = 0.0, q_tot = 0.0;
    for (long s = 0; s < g.V; ++s) {
        int x[4];
        lat_coords(&g, s, x);
        mat3 F[4][4];
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu)
                F[mu][nu] = mu == nu ? m_zero() : clover_F(&g, U, x, mu, nu);
        double sr = 0.0, qx = 0.0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = 0; nu < 4; ++nu) {
                if (mu == nu) continue;
                mat3 FF = m_mul(&F[mu][nu], &F[mu][nu]);
                sr += 0.5 * creal(m_trace(&FF));
                for (int rh = 0; rh < 4; ++rh)
                    for (int si = 0; si < 4; ++si) {
                        int e = levi_civita(mu, nu, rh, si);
                        if (!e) continue;
                        mat3 P = m_mul(&F[mu][nu], &F[rh][si]);
                        qx += e * creal(m_trace(&P));
                    }
            }
        sr /= 72.0;
        qx /= 32.0 * OR_PI * OR_PI;
        if (SR_site) SR_site[s] = sr;
        if (q_site) q_site[s] = qx;
        sr_tot += sr;
        q_tot += qx;
    }
    *mean_SR = sr_tot / (double)g.V;
    *Q = q_tot;
    return 0;
}

/* Vortex flux through plaquette (mu, nu) at x from labels:
 * P = Z_mu(x) Z_nu(x+mu) Z_mu^dag(x+nu) Z_nu^dag(x) = exp(2 pi i p / 3), Sec. I. */
static int centre_charge(const lattice *g, const int8_t *lab, const int x[4], int mu, int nu) {
    int xm[4], xn[4];
    memcpy(xm, x, sizeof xm); lat_move(g, xm, mu, +1);
    memcpy(xn, x, sizeof xn); lat_move(g, xn, nu, +1);
    int p = lab[(long)mu * g->V + lat_site(g, x)] + lab[(long)nu * g->V + lat_site(g, xm)]
          - lab[(long)mu * g->V + lat_site(g, xn)] - lab[(long)nu * g->V + lat_site(g, x)];
    p = ((p % 3) + 3) % 3;
    return p == 2 ? -1 : p;
}

int or_centre_charges(const int32_t dims[4], const int8_t *labels, int8_t *charges /*[6][V]*/) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    for (long s = 0; s < g.V; ++s) {
        int x[4];
        lat_coords(&g, s, x);
        int k = 0;
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu, ++k)
                charges[(long)k * g.V + s] = (int8_t)centre_charge(&g, labels, x, mu, nu);
    }
    return 0;
}

/* Counts over the field: links whose label differs from the reference, and
 * plaquettes whose centre charge differs from the reference charge; plus the
 * smallest angular distance of any arg Tr U from a sector boundary and
 * (optional) the number of links closer than near_tol to one.  With a
 * gauge transformation G the labels are those of G^dag(x) U G(x+mu). */
int or_vortex_check(const int32_t dims[4], const double *links, const int8_t *ref_labels,
                    int64_t *n_label_diff, int64_t *n_charge_diff, double *min_margin,
                    const double *gauge, double near_tol, int64_t *n_near_boundary) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    int8_t *lab = (int8_t *)malloc(4 * g.V);
    double *mar = (double *)malloc(sizeof(double) * 4 * g.V);
    if (!lab || !mar) { free(lab); free(mar); return -5; }
    const cplx *U = (const cplx *)links;
    for (int mu = 0; mu < 4; ++mu)
        for (long s = 0; s < g.V; ++s) {
            int x[4];
            lat_coords(&g, s, x);
            mat3 a = link_get(&g, U, mu, s);
            cplx tr = vp_trace(g.L, g.V, (const cplx *)gauge, mu, x, &a);
            lab[(long)mu * g.V + s] = (int8_t)label_of_trace(tr);
            mar[(long)mu * g.V + s] = margin_of_trace(tr);
        }
    int64_t nd = 0, nc = 0, nn = 0;
    double mm = 1e300;
    for (long i = 0; i < 4 * g.V; ++i) {
        nd += lab[i] != ref_labels[i];
        nn += mar[i] < near_tol;
        if (mar[i] < mm) mm = mar[i];
    }
    for (long s = 0; s < g.V; ++s) {
        int x[4];
        lat_coords(&g, s, x);
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu)
                nc += centre_charge(&g, lab, x, mu, nu) != centre_charge(&g, ref_labels, x, mu, nu);
    }
    *n_label_diff = nd;
    *n_charge_diff = nc;
    *min_margin = mm;
    if (n_near_boundary) *n_near_boundary = nn;
    free(lab);
    free(mar);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Correlation of two densities, Sec. VII Eq. (correlation_s) and the C^q   */
/* equation that follows it                                                  */
/* ------------------------------------------------------------------------ */

/* C_XY = <a(x) b(x)> / (sqrt<a(x)^2> sqrt<b(x)^2>), <.> the mean over the n
 * sites.  The paper's form is not mean-subtracted: the densities themselves
 * are correlated.  Returns -2 when either density is zero everywhere. */
int or_correlation(long n, const double *a, const double *b, double *C) {
    if (n < 1 || !a || !b || !C) return -1;
    double sab = 0.0, saa = 0.0, sbb = 0.0;
    for (long i = 0; i < n; ++i) {
        sab += a[i] * b[i];
        saa += a[i] * a[i];
        sbb += b[i] * b[i];
    }
    if (!(saa > 0.0) || !(sbb > 0.0)) return -2;
    const double mab = sab / (double)n, maa = saa / (double)n, mbb = sbb / (double)n;
    *C = mab / (sqrt(maa) * sqrt(mbb));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Gauge transformation (Sec. II.A): U_mu(x) -> G(x) U_mu(x) G^dag(x+mu)     */
/* ------------------------------------------------------------------------ */

int or_gauge_transform(const int32_t dims[4], double *links, const double *G /*[V][3][3][2]*/) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    cplx *U = (cplx *)links;
    const cplx *Gc = (const cplx *)G;
    for (int mu = 0; mu < 4; ++mu)
        for (long s = 0; s < g.V; ++s) {
            int x[4];
            lat_coords(&g, s, x);
            lat_move(&g, x, mu, +1);
            long sp = lat_site(&g, x);
            mat3 Gx, Gp;
            memcpy(&Gx, Gc + s * 9, sizeof Gx);
            memcpy(&Gp, Gc + sp * 9, sizeof Gp);
            mat3 Gpd = m_dag(&Gp);
            mat3 u = link_get(&g, U, mu, s);
            mat3 t = m_mul(&Gx, &u);
            t = m_mul(&t, &Gpd);
            link_put(&g, U, mu, s, &t);
        }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Annealed U-link smearing with MaxReTr (Sec. III, Eqs. V, maxReTr,         */
/* def_L1, def_T1); cooling is its alpha = 1 case                           */
/* ------------------------------------------------------------------------ */

/* One MaxReTr update of link U towards the blocked matrix Vb: n_hits passes
 * over the SU(2) subgroups (1,2), (2,3), (1,3).  For subgroup (p,q):
 * L = U Vb^dag, T = [[a, b], [-conj b, conj a]] with a = (L_pp + conj L_qq)/2,
 * b = (L_pq - conj L_qp)/2, k = sqrt(det T) = sqrt(|a|^2 + |b|^2),
 * T^c = T^dag / k embedded in SU(3), U <- T^c U.
 * The singular case (Sec. III.A): on vortex fields the staple sums take
 * discrete values and k can vanish exactly, where the paper notes that
 * rounding noise then picks an essentially random link.  Reading used: a
 * subgroup step with k <= 1e-6 of the block's scale
 * sqrt(|L_pp|^2 + |L_qq|^2 + |L_pq|^2 + |L_qp|^2) leaves the link unchanged,
 * which makes the result independent of rounding. */
static mat3 maxretr(const mat3 *U, const mat3 *Vb, int n_hits) {
    static const int sub[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    mat3 Vd = m_dag(Vb);
    mat3 Ux = *U;
    for (int h = 0; h < n_hits; ++h)
        for (int t = 0; t < 3; ++t) {
            int p = sub[t][0], q = sub[t][1];
            mat3 L = m_mul(&Ux, &Vd);
            cplx al = 0.5 * (L.m[p][p] + conj(L.m[q][q]));
            cplx be = 0.5 * (L.m[p][q] - conj(L.m[q][p]));
            double k = sqrt(creal(al * conj(al)) + creal(be * conj(be)));
            double scale = sqrt(creal(L.m[p][p] * conj(L.m[p][p])) + creal(L.m[q][q] * conj(L.m[q][q])) +
                                creal(L.m[p][q] * conj(L.m[p][q])) + creal(L.m[q][p] * conj(L.m[q][p])));
            if (!(k > 1e-6 * scale)) continue;
            mat3 Tc = m_eye();
            Tc.m[p][p] = conj(al) / k;
            Tc.m[p][q] = -be / k;
            Tc.m[q][p] = conj(be) / k;
            Tc.m[q][q] = al / k;
            Ux = m_mul(&Tc, &Ux);
        }
    return Ux;
}

/* n_sweeps of annealed U-link smearing in place, in the colour order of
 * or_smooth: V = (1 - alpha) U + (alpha / 6) Sigma(eps, u0) (Eq. V with the
 * staples of Eq. over-improvement), the link replaced by maxretr(U, V).
 * vp / ref_labels / n_reject / gauge as in or_smooth (Sec. VI).  alpha = 1 with
 * eps = 1 is cooling: V does not depend on U. */
int or_aus(const int32_t dims[4], double *links, const int8_t *ref_labels, int n_sweeps, double alpha,
           double eps, double u0, int n_hits, int vp, int64_t *n_reject, int nthreads,
           const double *gauge) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    for (int d = 0; d < 4; ++d)
        if (g.L[d] % 4) return -3;
    if (vp && !ref_labels) return -4;
    double c0, c1;
    or_overimproved_coeffs(eps, u0, &c0, &c1);
    cplx *U = (cplx *)links;
    const cplx *G = (const cplx *)gauge;
    long *sites = (long *)malloc(sizeof(long) * g.V);
    if (!sites) return -5;
    int err = 0;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        int64_t rej = 0;
        for (int mu = 0; mu < 4; ++mu)
            for (int c = 0; c < 4; ++c) {
                long n = class_sites(&g, mu, c, sites);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads < 1 ? 1 : nthreads) schedule(static) reduction(+ : rej) reduction(| : err)
#endif
                for (long i = 0; i < n; ++i) {
                    int x[4];
                    lat_coords(&g, sites[i], x);
                    mat3 S;
                    if (staple_sum(&g, U, mu, x, c0, c1, &S)) { err |= 1; continue; }
                    mat3 Ux = link_get(&g, U, mu, sites[i]);
                    mat3 Vb = m_zero();
                    m_axpy(&Vb, 1.0 - alpha, &Ux);
                    m_axpy(&Vb, alpha / 6.0, &S);
                    mat3 Un = maxretr(&Ux, &Vb, n_hits);
                    if (vp && label_of_trace(vp_trace(g.L, g.V, G, mu, x, &Un)) !=
                                  ref_labels[(long)mu * g.V + sites[i]]) {
                        rej += 1;
                        continue;
                    }
                    link_put(&g, U, mu, sites[i], &Un);
                }
            }
        if (n_reject) n_reject[sw] = rej;
    }
    free(sites);
    return err ? -6 : 0;
}

/* Cooling: annealed MaxReTr at alpha = 1 with the plaquette staples,
 * V = Sigma / 6 (used to generate the cooled hot-start inputs). */
int or_cool(const int32_t dims[4], double *links, int n_sweeps, int n_hits, int nthreads) {
    return or_aus(dims, links, NULL, n_sweeps, 1.0, 1.0, 1.0, n_hits, 0, NULL, nthreads, NULL);
}

/* One MaxReTr update of a single matrix (for the pins). */
int or_maxretr(const double *U18, const double *V18, int n_hits, double *out18) {
    mat3 U, Vb, R;
    memcpy(&U, U18, sizeof U);
    memcpy(&Vb, V18, sizeof Vb);
    R = maxretr(&U, &Vb, n_hits);
    memcpy(out18, &R, sizeof R);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Unit circle projection (Sec. II.C, Eqs. W and P_ucp)                       */
/* ------------------------------------------------------------------------ */

/* Eigen-decomposition A = E diag(lam) E^dag of a 3x3 Hermitian matrix by
 * cyclic Jacobi rotations.  For the pair (p,q) with A_pq = |b| e^{i phi},
 * the diagonal unitary that multiplies column q by e^{-i phi} makes the
 * (p,q) entry real; the real plane rotation by theta, tan 2 theta =
 * 2 |b| / (A_qq - A_pp), then zeroes it.  Sweeps repeat until the squared
 * off-diagonal norm is below 1e-30 of the squared diagonal norm (rounding
 * level: the off-diagonal part then changes the eigenvalues by ~1e-30). */
static void herm_eig(const mat3 *A0, double lam[3], mat3 *E) {
    mat3 A = *A0;
    *E = m_eye();
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double a2 = creal(A.m[i][j] * conj(A.m[i][j]));
                if (i == j) dia += a2; else off += a2;
            }
        if (off <= 1e-30 * dia) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double b = cabs(A.m[p][q]);
                if (b == 0.0) continue;
                cplx ph = A.m[p][q] / b;                 /* e^{i phi} */
                double th = 0.5 * atan2(2.0 * b, creal(A.m[q][q]) - creal(A.m[p][p]));
                double c = cos(th), sn = sin(th);
                /* J = D R with D = diag(1 at p, conj(ph) at q), R the rotation */
                mat3 J = m_eye();
                J.m[p][p] = c;
                J.m[p][q] = sn;
                J.m[q][p] = -sn * conj(ph);
                J.m[q][q] = c * conj(ph);
                mat3 Jd = m_dag(&J);
                mat3 T = m_mul(&A, &J);
                A = m_mul(&Jd, &T);
                *E = m_mul(E, &J);
            }
    }
    for (int i = 0; i < 3; ++i) lam[i] = creal(A.m[i][i]);
}

static cplx m_det(const mat3 *a) {
    const cplx(*m)[3] = a->m;
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
           m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

/* P_ucp{V} = W / cbrt(det W), W = V (V^dag V)^{-1/2} (Eq. W), with the
 * principal cube root: arg det W taken in (-pi, pi], so the phase divided
 * out lies in (-pi/3, pi/3] (the paper's open interval, closed at +pi/3 to
 * match the label convention at arg = pi).  Reading for a singular V (the
 * projection is undefined): det(V^dag V) <= 1e-24 (Tr(V^dag V)/3)^3 returns
 * 1 and leaves *out untouched. */
static int ucp_project(const mat3 *V, mat3 *out) {
    mat3 Vd = m_dag(V);
    mat3 A = m_mul(&Vd, V);
    double lam[3];
    mat3 E;
    herm_eig(&A, lam, &E);
    double tr = lam[0] + lam[1] + lam[2];
    if (!(lam[0] > 0.0 && lam[1] > 0.0 && lam[2] > 0.0) ||
        !(lam[0] * lam[1] * lam[2] > 1e-24 * (tr / 3.0) * (tr / 3.0) * (tr / 3.0)))
        return 1;
    mat3 R = m_zero();     /* (V^dag V)^{-1/2} = E diag(lam^{-1/2}) E^dag */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            for (int k = 0; k < 3; ++k) R.m[i][j] += E.m[i][k] * (1.0 / sqrt(lam[k])) * conj(E.m[j][k]);
    mat3 W = m_mul(V, &R);
    cplx d = m_det(&W);
    double phi = atan2(cimag(d), creal(d));
    if (phi <= -OR_PI) phi = OR_PI;
    cplx f = cexp(-I * phi / 3.0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) W.m[i][j] *= f;
    *out = W;
    return 0;
}

/* Re-unitarisation of n matrices (not a step of the paper: the FP32 storage
 * modes apply it every few sweeps to undo rounding drift).  Gram-Schmidt on the
 * rows: r0 <- r0 / |r0|; r1 <- r1 - <r0, r1> r0 with <a, b> = sum conj(a_k) b_k,
 * r1 <- r1 / |r1|; r2 <- conj(r0 x r1), the row that makes the matrix special
 * unitary. */
int or_reunit(long n, const double *in18, double *out18) {
    if (n < 0) return -1;
    for (long l = 0; l < n; ++l) {
        mat3 M;
        memcpy(&M, in18 + 18 * l, sizeof M);
        cplx *r0 = M.m[0], *r1 = M.m[1], *r2 = M.m[2];
        double n0 = 0.0;
        for (int k = 0; k < 3; ++k) n0 += creal(r0[k] * conj(r0[k]));
        for (int k = 0; k < 3; ++k) r0[k] /= sqrt(n0);
        cplx ip = 0.0;
        for (int k = 0; k < 3; ++k) ip += conj(r0[k]) * r1[k];
        for (int k = 0; k < 3; ++k) r1[k] -= ip * r0[k];
        double n1 = 0.0;
        for (int k = 0; k < 3; ++k) n1 += creal(r1[k] * conj(r1[k]));
        for (int k = 0; k < 3; ++k) r1[k] /= sqrt(n1);
        for (int k = 0; k < 3; ++k) {
            const int a = (k + 1) % 3, b = (k + 2) % 3;
            r2[k] = conj(r0[a] * r1[b] - r0[b] * r1[a]);
        }
        memcpy(out18 + 18 * l, &M, sizeof M);
    }
    return 0;
}

/* One projection of a single matrix (for the pins): 0, or 1 if singular. */
int or_ucp(const double *V18, double *out18) {
    mat3 V, P;
    memcpy(&V, V18, sizeof V);
    int r = ucp_project(&V, &P);
    if (r == 0) memcpy(out18, &P, sizeof P);
    return r;
}

/* n_sweeps of APE smearing with unit circle projection (Sec. II.C):
 * V = (1 - alpha) U + (alpha / 6) Sigma(eps, u0) (Eq. V, staples of Eq.
 * over-improvement), U <- P_ucp{V}.  schedule OR_SIMULTANEOUS is APE
 * smearing (every link from the previous field); OR_ANNEALED is annealed
 * U-link smearing with UCP (AUS+UCP, Sec. VII.A), in the colour order of
 * or_smooth.  A singular V leaves the link.  vp / ref_labels / n_reject /
 * gauge as in or_smooth (Sec. VI). */
int or_ape_ucp(const int32_t dims[4], double *links, const int8_t *ref_labels, int n_sweeps, double alpha,
               double eps, double u0, int schedule, int vp, int64_t *n_reject, int nthreads,
               const double *gauge) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    if (n_sweeps < 0) return -2;
    for (int d = 0; d < 4; ++d)
        if (schedule == OR_ANNEALED && g.L[d] % 4) return -3;
    if (vp && !ref_labels) return -4;
    double c0, c1;
    or_overimproved_coeffs(eps, u0, &c0, &c1);
    cplx *U = (cplx *)links;
    const cplx *G = (const cplx *)gauge;
    long *sites = (long *)malloc(sizeof(long) * g.V);
    cplx *old = NULL;
    if (schedule == OR_SIMULTANEOUS) old = (cplx *)malloc(sizeof(cplx) * 9 * 4 * g.V);
    if (!sites || (schedule == OR_SIMULTANEOUS && !old)) { free(sites); free(old); return -5; }
    if (nthreads < 1) nthreads = 1;
    int err = 0;
    for (int sw = 0; sw < n_sweeps; ++sw) {
        int64_t rej = 0;
        if (schedule == OR_SIMULTANEOUS) memcpy(old, U, sizeof(cplx) * 9 * 4 * g.V);
        const cplx *src = schedule == OR_SIMULTANEOUS ? old : U;
        for (int mu = 0; mu < 4; ++mu)
            for (int c = 0; c < (schedule == OR_ANNEALED ? 4 : 1); ++c) {
                long n;
                if (schedule == OR_ANNEALED) n = class_sites(&g, mu, c, sites);
                else { n = g.V; for (long s = 0; s < n; ++s) sites[s] = s; }
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static) reduction(+ : rej) reduction(| : err)
#endif
                for (long i = 0; i < n; ++i) {
                    int x[4];
                    lat_coords(&g, sites[i], x);
                    mat3 S;
                    if (staple_sum(&g, src, mu, x, c0, c1, &S)) { err |= 1; continue; }
                    mat3 Ux = link_get(&g, src, mu, sites[i]);
                    mat3 Vb = m_zero();
                    m_axpy(&Vb, 1.0 - alpha, &Ux);
                    m_axpy(&Vb, alpha / 6.0, &S);
                    mat3 Un;
                    if (ucp_project(&Vb, &Un)) Un = Ux;
                    if (vp && label_of_trace(vp_trace(g.L, g.V, G, mu, x, &Un)) !=
                                  ref_labels[(long)mu * g.V + sites[i]]) {
                        rej += 1;
                        if (schedule == OR_SIMULTANEOUS) link_put(&g, U, mu, sites[i], &Ux);
                        continue;
                    }
                    link_put(&g, U, mu, sites[i], &Un);
                }
            }
        if (n_reject) n_reject[sw] = rej;
    }
    free(sites);
    free(old);
    return err ? -6 : 0;
}

/* ------------------------------------------------------------------------ */
/* Wilson flow by a third-order Runge-Kutta scheme (Sec. V.B, Sec. VII.A)     */
/* ------------------------------------------------------------------------ */

/* The flow dU/dtau = Q[U] U of Sec. V.B, Q the generator of Eq. (generator)
 * built from the staples Sigma(eps, u0) (eps = 1: the Wilson flow), over
 * n_steps steps of size h with the third-order Runge-Kutta scheme of
 * Luscher (JHEP 08 (2010) 071, Appendix C), which the paper names as the
 * alternative to its Euler steps.  With Z_i = h Q[W_i] on every link:
 *   W_0 = U(tau),
 *   W_1 = exp(Z_0 / 4) W_0,
 *   W_2 = exp(8 Z_1 / 9 - 17 Z_0 / 36) W_1,
 *   U(tau + h) = W_3 = exp(3 Z_2 / 4 - 8 Z_1 / 9 + 17 Z_0 / 36) W_2.
 * Every Z_i is taken from the whole field W_i before any link moves. */
static int flow_generators(const lattice *g, const cplx *W, double c0, double c1, double h, mat3 *Z,
                           int nthreads) {
    int err = 0;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static) reduction(| : err)
#endif
    for (long i = 0; i < 4 * g->V; ++i) {
        int mu = (int)(i / g->V);
        long s = i % g->V;
        int x[4];
        lat_coords(g, s, x);
        mat3 S;
        if (staple_sum(g, W, mu, x, c0, c1, &S)) { err |= 1; continue; }
        mat3 Ux = link_get(g, W, mu, s);
        mat3 Ud = m_dag(&Ux);
        mat3 Om = m_mul(&S, &Ud);
        mat3 Omd = m_dag(&Om);
        mat3 A = Om;
        m_axpy(&A, -1.0, &Omd);
        cplx trA = m_trace(&A);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Z[i].m[a][b] = h * (0.5 * A.m[a][b] - (a == b ? trA / 6.0 : 0.0));
    }
    return err;
}

static void flow_apply(const lattice *g, cplx *W, const mat3 *X, int nthreads) {
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(static)
#endif
    for (long i = 0; i < 4 * g->V; ++i) {
        int mu = (int)(i / g->V);
        long s = i % g->V;
        mat3 E = expm_series(&X[i]);
        mat3 Ux = link_get(g, W, mu, s);
        mat3 Un = m_mul(&E, &Ux);
        link_put(g, W, mu, s, &Un);
    }
}

int or_flow_rk3(const int32_t dims[4], double *links, int n_steps, double h, double eps, double u0,
                int nthreads) {
    lattice g;
    if (lat_init(&g, dims)) return -1;
    if (n_steps < 0) return -2;
    double c0, c1;
    or_overimproved_coeffs(eps, u0, &c0, &c1);
    if (nthreads < 1) nthreads = 1;
    cplx *W = (cplx *)links;
    const long n = 4 * g.V;
    mat3 *Z0 = (mat3 *)malloc(sizeof(mat3) * n), *Z1 = (mat3 *)malloc(sizeof(mat3) * n);
    mat3 *Z2 = (mat3 *)malloc(sizeof(mat3) * n), *X = (mat3 *)malloc(sizeof(mat3) * n);
    if (!Z0 || !Z1 || !Z2 || !X) { free(Z0); free(Z1); free(Z2); free(X); return -5; }
    int err = 0;
    for (int st = 0; st < n_steps && !err; ++st) {
        err |= flow_generators(&g, W, c0, c1, h, Z0, nthreads);
        for (long i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) X[i].m[a][b] = 0.25 * Z0[i].m[a][b];
        flow_apply(&g, W, X, nthreads);                                 /* W_1 */
        err |= flow_generators(&g, W, c0, c1, h, Z1, nthreads);
        for (long i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    X[i].m[a][b] = (8.0 / 9.0) * Z1[i].m[a][b] - (17.0 / 36.0) * Z0[i].m[a][b];
        flow_apply(&g, W, X, nthreads);                                 /* W_2 */
        err |= flow_generators(&g, W, c0, c1, h, Z2, nthreads);
        for (long i = 0; i < n; ++i)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    X[i].m[a][b] = 0.75 * Z2[i].m[a][b] - (8.0 / 9.0) * Z1[i].m[a][b] +
                                   (17.0 / 36.0) * Z0[i].m[a][b];
        flow_apply(&g, W, X, nthreads);                                 /* W_3 */
    }
    free(Z0); free(Z1); free(Z2); free(X);
    return err ? -6 : 0;
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
