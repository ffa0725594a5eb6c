/*
 * pt_oracle.c -- plain, slow, FP64 CPU oracle for the Parallel-Tempering Metropolis
 * simulation of the smoothed-cubic 4-body random-laser model (arXiv 2511.13508).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file: only tests/, __graft_entry__.smoke() and the cpu_baseline / reference leg of
 * bench.py use it.  It shares no code, header, table or constant generator with the
 * CUDA library; the two are written independently from the paper.
 *
 * Build: gcc -std=c99 -O2 -ffp-contract=off -fno-fast-math -shared -fPIC (no FMA
 * contraction, IEEE round-to-nearest, libm sin/cos/exp/log/sqrt).
 *
 * What it computes, and where the paper defines it:
 *   - mode-locked comb graph, omega_k = k: quadruplets a<b<c<d with a+d = b+c
 *     (frequency matching condition, Eq. (1) / Sec. II.C "Graph generation");
 *   - H4 = -cc * sum_q J_q Re(conj(a_a) a_b a_c conj(a_d))  (Eq. (4), "+ c.c." gives
 *     cc = 2; the couplings are real, Sec. II);
 *   - smoothed-cubic constraint sum_k |a_k|^4 = N  (Eq. (6) after rescaling, Sec. II.B);
 *   - the constraint-preserving pair ("double") Metropolis update and the sweep of N/2
 *     pair updates (Sec. III.A.1);
 *   - exchange Monte Carlo swaps of neighbouring temperatures, proposed sequentially
 *     with p = min[1, exp((beta_i - beta_{i+1})(H_i - H_{i+1}))]  (Sec. III.A.2, Eq. (15));
 *   - observables: energy sums for the specific heat (Eq. (21)), the replica overlap
 *     q_cd = Re sum_k conj(a_k^c) a_k^d / N and its histogram (Sec. IV.C), the inverse
 *     participation ratios Y_2, Y_4 (Sec. IV.D).
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11), written
 *     from its published definition; the paper does not name its generator.
 *
 * Readings where the paper is silent or garbled (each one is also listed in the design
 * notes of the repository):
 *   R1 distinct indices only; on the integer comb the matching condition is exact equality.
 *   R2 cc = 2 ("+ c.c."), selectable.
 *   R3 the pair update draws j uniform and k uniform among the other N-1 modes; mode j
 *      receives K sqrt(cos theta), mode k receives K sqrt(sin theta).
 *   R4 all configurations of one disorder sample use the same (j,k) sequence.
 *   R5 Delta H of a pair update includes the j-k cross term (quadruplets holding both).
 *   R6 Metropolis: accept iff dH <= 0 or U < exp(-beta dH); the uniform U is always drawn.
 *   R7 swaps are proposed in ascending temperature order, index 0 = coldest.
 *   R8 the overlap histogram has 201 bins centred at -1, -0.99, ..., 1; bin = floor(100(q+1)+0.5).
 *   R9 every resync_every sweeps: a <- a (N / sum|a|^4)^(1/4), then E <- H(a).
 *   R10 random-frequency graph (Sec. II.C "Quenched random frequencies", "Graph generation",
 *      Eq. (gamma_scaling)): sorted frequencies omega_0 < ... < omega_{N-1} in [0,1]; for every
 *      4-subset a<b<c<d each of its three splittings into a conjugated pair {p,q} and a plain pair
 *      {u,v} with |omega_p + omega_q - omega_u - omega_v| < gamma is one interaction with its own
 *      coupling, stored as (p, u, v, q) so that the term is Re(conj(a_p) a_u a_v conj(a_q)); the
 *      splittings in order: {a,d}|{b,c}, {a,b}|{c,d}, {a,c}|{b,d}.  gamma = 1/(2(N-1)).
 *
 * Random-number streams (Philox4x32-10, key = (seed_lo, seed_hi), counter = 4 words):
 *   INIT     (chain, mode, 0, 1)            chain = (s*R + r)*nT + t
 *   PAIR     (sample, sweep, update, 2)     words 0,1 -> (j, k)
 *   PROPOSE  (chain, sweep, update, 3)      words: phi_j, phi_k, theta, U
 *   SWAP     (s*R + r, swap_pass, i, 4)     word 0 -> U
 *   uniform U(w) = (w + 0.5) * 2^-32.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_TAG_INIT 1u
#define OR_TAG_PAIR 2u
#define OR_TAG_PROPOSE 3u
#define OR_TAG_SWAP 4u
#define OR_NBINS 201
#define OR_TWO_PI 6.283185307179586476925286766559
#define OR_HALF_PI 1.5707963267948966192313216916398

/* ---------------------------------------------------------------- Philox4x32-10 */
/* Salmon et al., "Parallel random numbers: as easy as 1, 2, 3", SC'11: a round maps
 * (x0,x1,x2,x3) with key (k0,k1) to (hi(M1*x2)^x1^k0, lo(M1*x2), hi(M0*x0)^x3^k1, lo(M0*x0)),
 * and the key is bumped by the Weyl constants between rounds. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

double or_uniform(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* ---------------------------------------------------------------- graph */
/* Every 4-subset a<b<c<d of the comb with a+d = b+c, in lexicographic (a,b,c) order.
 * Returns the count; writes 4 indices per quadruplet if abcd != NULL. */
int64_t or_enumerate_quads(int N, int32_t *abcd) {
    int64_t n = 0;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b)
            for (int c = b + 1; c < N; ++c) {
                int d = b + c - a;
                if (d <= c || d >= N) continue;
                if (abcd) {
                    abcd[4 * n + 0] = a; abcd[4 * n + 1] = b;
                    abcd[4 * n + 2] = c; abcd[4 * n + 3] = d;
                }
                ++n;
            }
    return n;
}

/* Random-frequency mode-locked graph (reading R10), by brute force over every 4-subset and each of
 * its three splittings.  omega must be sorted ascending.  Returns the count; writes 4 indices per
 * interaction in term order if quads != NULL. */
int64_t or_fmc_graph(int N, const double *omega, double gamma, int32_t *quads) {
    int64_t n = 0;
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b)
            for (int c = b + 1; c < N; ++c)
                for (int d = c + 1; d < N; ++d) {
                    /* (conjugated p, q | plain u, v) for the three splittings */
                    const int sp[3][4] = {{a, d, b, c}, {a, b, c, d}, {a, c, b, d}};
                    for (int t = 0; t < 3; ++t) {
                        const int p = sp[t][0], q = sp[t][1], u = sp[t][2], v = sp[t][3];
                        if (fabs(omega[p] + omega[q] - omega[u] - omega[v]) < gamma) {
                            if (quads) {
                                quads[4 * n + 0] = p; quads[4 * n + 1] = u;
                                quads[4 * n + 2] = v; quads[4 * n + 3] = q;
                            }
                            ++n;
                        }
                    }
                }
    return n;
}

/* ---------------------------------------------------------------- complex helpers */
typedef struct { double re, im; } cplx;
static cplx cmul(cplx x, cplx y) { cplx r = {x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re}; return r; }
static cplx cconj(cplx x) { cplx r = {x.re, -x.im}; return r; }
static cplx cget(const double *a, int k) { cplx r = {a[2 * k], a[2 * k + 1]}; return r; }

/* Factor of mode m in the term of quadruplet q = (a,b,c,d): conj(a_m) for the outer
 * pair {a,d}, a_m for the inner pair {b,c}; the term is J * x_a x_b x_c x_d. */
static cplx xfactor(const double *a, const int32_t *q, int pos) {
    cplx v = cget(a, q[pos]);
    return (pos == 0 || pos == 3) ? cconj(v) : v;
}

/* H = -cc * sum_q J_q Re(conj(a_a) a_b a_c conj(a_d))   (Eq. (4)). */
double or_energy(int N, int64_t nq, const int32_t *abcd, const double *J, double cc, const double *a) {
    (void)N;
    double s = 0.0;
    for (int64_t q = 0; q < nq; ++q) {
        const int32_t *Q = abcd + 4 * q;
        cplx p = cmul(cmul(xfactor(a, Q, 0), xfactor(a, Q, 1)), cmul(xfactor(a, Q, 2), xfactor(a, Q, 3)));
        s += J[q] * p.re;
    }
    return -cc * s;
}

/* Local field of mode l: h_l = sum_{q containing l} J_q c_q(l) with H = -cc Re(conj(a_l) h_l) + (terms
 * without l).  c_q(l) is the product of the other three factors, conjugated when l sits in the
 * inner pair.  inc/ninc optionally restrict the scan to the quadruplets that hold l. */
static void field_core(const int32_t *abcd, const double *J, const double *a, int l,
                       const int64_t *list, int64_t nlist, int64_t nq, double h[2]) {
    double hr = 0.0, hi = 0.0;
    int64_t cnt = list ? nlist : nq;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t q = list ? list[t] : t;
        const int32_t *Q = abcd + 4 * q;
        int pos = -1;
        for (int p = 0; p < 4; ++p) if (Q[p] == l) pos = p;
        if (pos < 0) continue;
        cplx X = {J[q], 0.0};
        for (int p = 0; p < 4; ++p) if (p != pos) X = cmul(X, xfactor(a, Q, p));
        if (pos == 1 || pos == 2) X = cconj(X);
        hr += X.re; hi += X.im;
    }
    h[0] = hr; h[1] = hi;
}

void or_field(int N, int64_t nq, const int32_t *abcd, const double *J, const double *a, int l, double h[2]) {
    (void)N;
    field_core(abcd, J, a, l, NULL, 0, nq, h);
}

/* Exact change of H when (a_j, a_k) -> (aj_new, ak_new): the two local fields of the old state,
 * plus the cross term of quadruplets holding both j and k (reading R5). */
static double delta_h_core(const int32_t *abcd, const double *J, double cc, const double *a, int j, int k,
                           const double aj_new[2], const double ak_new[2],
                           const int64_t *listj, int64_t nlistj, const int64_t *listk, int64_t nlistk, int64_t nq) {
    double hj[2], hk[2];
    field_core(abcd, J, a, j, listj, nlistj, nq, hj);
    field_core(abcd, J, a, k, listk, nlistk, nq, hk);
    cplx dj = {aj_new[0] - a[2 * j], aj_new[1] - a[2 * j + 1]};
    cplx dk = {ak_new[0] - a[2 * k], ak_new[1] - a[2 * k + 1]};
    cplx Hj = {hj[0], hj[1]}, Hk = {hk[0], hk[1]};
    double lin = cmul(cconj(dj), Hj).re + cmul(cconj(dk), Hk).re;
    double cross = 0.0;
    int64_t cnt = listj ? nlistj : nq;
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t q = listj ? listj[t] : t;
        const int32_t *Q = abcd + 4 * q;
        int pj = -1, pk = -1;
        for (int p = 0; p < 4; ++p) { if (Q[p] == j) pj = p; if (Q[p] == k) pk = p; }
        if (pj < 0 || pk < 0) continue;
        cplx X = {J[q], 0.0};
        for (int p = 0; p < 4; ++p) if (p != pj && p != pk) X = cmul(X, xfactor(a, Q, p));
        cplx dxj = (pj == 0 || pj == 3) ? cconj(dj) : dj;
        cplx dxk = (pk == 0 || pk == 3) ? cconj(dk) : dk;
        cross += cmul(X, cmul(dxj, dxk)).re;
    }
    return -cc * (lin + cross);
}

double or_delta_h(int N, int64_t nq, const int32_t *abcd, const double *J, double cc, const double *a,
                  int j, int k, const double aj_new[2], const double ak_new[2]) {
    (void)N;
    return delta_h_core(abcd, J, cc, a, j, k, aj_new, ak_new, NULL, 0, NULL, 0, nq);
}

/* The bilinear (j,k) part of the pair-move energy change (reading R5), split by the conjugation of the two
 * increments: with a_j += dj, a_k += dk, the quadruplets holding both j and k change H by
 *     -cc Re[ conj(dj) dk B + conj(dj) conj(dk) A ].
 * For each such quadruplet let X = J_q times the factors of its other two positions (conjugated at
 * positions 0 and 3).  Its term X x_j x_k, with x = conj(d) at positions 0, 3 and x = d at 1, 2, adds
 * X to B (j conjugated, k plain), conj(X) to B (j plain, k conjugated), X to A (both conjugated) or
 * conj(X) to A (both plain), since Re(z) = Re(conj(z)).  On the comb, B = sum J conj(a_m) a_y over
 * quadruplets {j, m | k, y} with j+m = k+y and A = sum J a_x a_y over quadruplets {j, k | x, y}. */
void or_cross_terms(int N, int64_t nq, const int32_t *abcd, const double *J, const double *a, int j, int k,
                    double B[2], double A[2]) {
    (void)N;
    cplx Bs = {0.0, 0.0}, As = {0.0, 0.0};
    for (int64_t q = 0; q < nq; ++q) {
        const int32_t *Q = abcd + 4 * q;
        int pj = -1, pk = -1;
        for (int p = 0; p < 4; ++p) { if (Q[p] == j) pj = p; if (Q[p] == k) pk = p; }
        if (pj < 0 || pk < 0) continue;
        cplx X = {J[q], 0.0};
        for (int p = 0; p < 4; ++p) if (p != pj && p != pk) X = cmul(X, xfactor(a, Q, p));
        const int cj = (pj == 0 || pj == 3), ck = (pk == 0 || pk == 3);
        const cplx add = cj ? X : cconj(X); /* the four cases above: X when j is conjugated, else conj(X) */
        if (cj == ck) { As.re += add.re; As.im += add.im; }
        else { Bs.re += add.re; Bs.im += add.im; }
    }
    B[0] = Bs.re; B[1] = Bs.im;
    A[0] = As.re; A[1] = As.im;
}

/* ---------------------------------------------------------------- random draws */
/* Pair choice (reading R3): j = floor(w0 N / 2^32), k = (j + 1 + floor(w1 (N-1) / 2^32)) mod N. */
void or_pair(uint64_t seed, uint32_t sample, uint32_t sweep, uint32_t update, int N, int *j, int *k) {
    uint32_t w[4];
    draw(seed, sample, sweep, update, OR_TAG_PAIR, w);
    uint32_t jj = (uint32_t)(((uint64_t)w[0] * (uint64_t)N) >> 32);
    uint32_t off = (uint32_t)(((uint64_t)w[1] * (uint64_t)(N - 1)) >> 32);
    *j = (int)jj;
    *k = (int)((jj + 1u + off) % (uint32_t)N);
}

/* The pair move of Sec. III.A.1: K^4 = |a_j|^4 + |a_k|^4, theta ~ U[0, pi/2], new phases uniform,
 * |a_j'| = K sqrt(cos theta), |a_k'| = K sqrt(sin theta).  Returns the Metropolis uniform. */
double or_propose(uint64_t seed, uint32_t chain, uint32_t sweep, uint32_t update, const double *a, int j, int k,
                  double aj_new[2], double ak_new[2]) {
    uint32_t w[4];
    draw(seed, chain, sweep, update, OR_TAG_PROPOSE, w);
    double uj = a[2 * j] * a[2 * j] + a[2 * j + 1] * a[2 * j + 1];
    double uk = a[2 * k] * a[2 * k] + a[2 * k + 1] * a[2 * k + 1];
    double K4 = uj * uj + uk * uk;
    double K = sqrt(sqrt(K4));
    double phj = OR_TWO_PI * or_uniform(w[0]);
    double phk = OR_TWO_PI * or_uniform(w[1]);
    double th = OR_HALF_PI * or_uniform(w[2]);
    double Aj = K * sqrt(cos(th)), Ak = K * sqrt(sin(th));
    aj_new[0] = Aj * cos(phj); aj_new[1] = Aj * sin(phj);
    ak_new[0] = Ak * cos(phk); ak_new[1] = Ak * sin(phk);
    return or_uniform(w[3]);
}

/* Initial configuration: uniform on the constraint surface (beta = 0 law).  u = sqrt(N)|g|/||g|| with
 * g Gaussian (Box-Muller), a_k = sqrt(u_k) exp(i phi_k). */
void or_init_config(uint64_t seed, uint32_t chain, int N, double *a) {
    double *g = (double *)malloc(sizeof(double) * (size_t)N);
    double *ph = (double *)malloc(sizeof(double) * (size_t)N);
    double nrm = 0.0;
    for (int k = 0; k < N; ++k) {
        uint32_t w[4];
        draw(seed, chain, (uint32_t)k, 0u, OR_TAG_INIT, w);
        double r = sqrt(-2.0 * log(or_uniform(w[0])));
        g[k] = r * cos(OR_TWO_PI * or_uniform(w[1]));
        ph[k] = OR_TWO_PI * or_uniform(w[2]);
        nrm += g[k] * g[k];
    }
    nrm = sqrt(nrm);
    for (int k = 0; k < N; ++k) {
        double u = sqrt((double)N) * fabs(g[k]) / nrm;
        double A = sqrt(u);
        a[2 * k] = A * cos(ph[k]);
        a[2 * k + 1] = A * sin(ph[k]);
    }
    free(g); free(ph);
}

/* ---------------------------------------------------------------- observables of one state */
double or_sum_abs_pow(int N, const double *a, int p) { /* sum_k |a_k|^p for even p */
    double s = 0.0;
    for (int k = 0; k < N; ++k) {
        double u = a[2 * k] * a[2 * k] + a[2 * k + 1] * a[2 * k + 1];
        s += pow(u, 0.5 * p);
    }
    return s;
}

/* IPR Y_n = sum |a|^(2n) / (sum |a|^n)^2 (Sec. IV.D), n = 2 or 4. */
double or_ipr(int N, const double *a, int n) {
    double num = or_sum_abs_pow(N, a, 2 * n), den = or_sum_abs_pow(N, a, n);
    return num / (den * den);
}

/* Replica overlap q_cd = (1/N) Re sum_k conj(a_k^c) a_k^d (Sec. IV.C, index typo read as k). */
double or_overlap(int N, const double *ac, const double *ad) {
    double s = 0.0;
    for (int k = 0; k < N; ++k) s += ac[2 * k] * ad[2 * k] + ac[2 * k + 1] * ad[2 * k + 1];
    return s / (double)N;
}

int or_qbin(double q) {
    int b = (int)floor(100.0 * (q + 1.0) + 0.5);
    if (b < 0) b = 0;
    if (b > OR_NBINS - 1) b = OR_NBINS - 1;
    return b;
}

/* ---------------------------------------------------------------- the PT engine */
#define OR_NSTAT 7 /* n, sumE, sumE2, sumY2, sumY4, sumI, sumI2   per (sample, T) */
#define OR_NQSTAT 5 /* n, sumq, sumq2, sumq3, sumq4               per (sample, T) */

typedef struct {
    int S, R, nT;
    int *N;
    double cc;
    int swap_every, measure_every, resync_every;
    uint64_t seed;
    int64_t *nq;
    int32_t **abcd;
    double **J;
    int64_t **inc_off; /* per sample: [N+1] */
    int64_t **inc;     /* per sample: quadruplet indices holding each mode */
    double *beta;      /* [nT] */
    double **a;        /* per configuration slot (s, r, t): 2N doubles */
    double *E;         /* per configuration slot */
    int64_t sweeps_done, swap_passes;
    double *stat;      /* [S][nT][OR_NSTAT] */
    double *qstat;     /* [S][nT][OR_NQSTAT] */
    uint64_t *qhist;   /* [S][nT][OR_NBINS] */
    uint64_t *swap_acc, *swap_att; /* [S][R][nT-1] */
    uint64_t *mc_acc, *mc_att;     /* [S][nT] Metropolis acceptance by temperature */
} or_pt;

static int64_t slot(const or_pt *p, int s, int r, int t) { return ((int64_t)s * p->R + r) * p->nT + t; }

static or_pt *pt_create_impl(int S, const int32_t *N, const int32_t *graph, const double *J, const int64_t *J_off,
                             int nT, const double *temps, int R, uint64_t seed, double cc, int swap_every,
                             int measure_every, int resync_every);

/* Comb graph (Eq. (1) with omega_k = k) for every sample; J_off[s] .. J_off[s+1] are its couplings in the
 * order of or_enumerate_quads. */
or_pt *or_pt_create(int S, const int32_t *N, const double *J, const int64_t *J_off, int nT, const double *temps,
                    int R, uint64_t seed, double cc, int swap_every, int measure_every, int resync_every) {
    return pt_create_impl(S, N, NULL, J, J_off, nT, temps, R, seed, cc, swap_every, measure_every, resync_every);
}

/* Explicit interaction lists: sample s has the quadruplets graph[4 J_off[s] .. 4 J_off[s+1]) (term order,
 * Re(conj(a_q0) a_q1 a_q2 conj(a_q3))) with couplings J[J_off[s] .. J_off[s+1]). */
or_pt *or_pt_create_graph(int S, const int32_t *N, const int32_t *graph, const double *J, const int64_t *J_off,
                          int nT, const double *temps, int R, uint64_t seed, double cc, int swap_every,
                          int measure_every, int resync_every) {
    return pt_create_impl(S, N, graph, J, J_off, nT, temps, R, seed, cc, swap_every, measure_every, resync_every);
}

static or_pt *pt_create_impl(int S, const int32_t *N, const int32_t *graph, const double *J, const int64_t *J_off,
                             int nT, const double *temps, int R, uint64_t seed, double cc, int swap_every,
                             int measure_every, int resync_every) {
    or_pt *p = (or_pt *)calloc(1, sizeof(or_pt));
    p->S = S; p->R = R; p->nT = nT; p->cc = cc; p->seed = seed;
    p->swap_every = swap_every; p->measure_every = measure_every; p->resync_every = resync_every;
    p->N = (int *)malloc(sizeof(int) * (size_t)S);
    p->nq = (int64_t *)malloc(sizeof(int64_t) * (size_t)S);
    p->abcd = (int32_t **)calloc((size_t)S, sizeof(int32_t *));
    p->J = (double **)calloc((size_t)S, sizeof(double *));
    p->inc_off = (int64_t **)calloc((size_t)S, sizeof(int64_t *));
    p->inc = (int64_t **)calloc((size_t)S, sizeof(int64_t *));
    for (int s = 0; s < S; ++s) {
        int n = N[s];
        p->N[s] = n;
        int64_t nq = graph ? J_off[s + 1] - J_off[s] : or_enumerate_quads(n, NULL);
        p->nq[s] = nq;
        p->abcd[s] = (int32_t *)malloc(sizeof(int32_t) * 4 * (size_t)(nq > 0 ? nq : 1));
        if (graph) memcpy(p->abcd[s], graph + 4 * J_off[s], sizeof(int32_t) * 4 * (size_t)nq);
        else or_enumerate_quads(n, p->abcd[s]);
        p->J[s] = (double *)malloc(sizeof(double) * (size_t)(nq > 0 ? nq : 1));
        memcpy(p->J[s], J + J_off[s], sizeof(double) * (size_t)nq);
        /* incidence lists: for mode l, the quadruplets holding l, in Q order */
        int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
        for (int64_t q = 0; q < nq; ++q)
            for (int m = 0; m < 4; ++m) off[p->abcd[s][4 * q + m] + 1]++;
        for (int l = 0; l < n; ++l) off[l + 1] += off[l];
        int64_t *fill = (int64_t *)calloc((size_t)n, sizeof(int64_t));
        int64_t *inc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(4 * nq > 0 ? 4 * nq : 1));
        for (int64_t q = 0; q < nq; ++q)
            for (int m = 0; m < 4; ++m) {
                int l = p->abcd[s][4 * q + m];
                inc[off[l] + fill[l]++] = q;
            }
        free(fill);
        p->inc_off[s] = off; p->inc[s] = inc;
    }
    p->beta = (double *)malloc(sizeof(double) * (size_t)nT);
    for (int t = 0; t < nT; ++t) p->beta[t] = 1.0 / temps[t];
    int64_t nslot = (int64_t)S * R * nT;
    p->a = (double **)calloc((size_t)nslot, sizeof(double *));
    p->E = (double *)calloc((size_t)nslot, sizeof(double));
    for (int s = 0; s < S; ++s)
        for (int r = 0; r < R; ++r)
            for (int t = 0; t < nT; ++t) {
                int64_t c = slot(p, s, r, t);
                p->a[c] = (double *)malloc(sizeof(double) * 2 * (size_t)p->N[s]);
                or_init_config(seed, (uint32_t)c, p->N[s], p->a[c]);
                p->E[c] = or_energy(p->N[s], p->nq[s], p->abcd[s], p->J[s], cc, p->a[c]);
            }
    p->stat = (double *)calloc((size_t)S * nT * OR_NSTAT, sizeof(double));
    p->qstat = (double *)calloc((size_t)S * nT * OR_NQSTAT, sizeof(double));
    p->qhist = (uint64_t *)calloc((size_t)S * nT * OR_NBINS, sizeof(uint64_t));
    int npair = nT > 1 ? nT - 1 : 1;
    p->swap_acc = (uint64_t *)calloc((size_t)S * R * npair, sizeof(uint64_t));
    p->swap_att = (uint64_t *)calloc((size_t)S * R * npair, sizeof(uint64_t));
    p->mc_acc = (uint64_t *)calloc((size_t)S * nT, sizeof(uint64_t));
    p->mc_att = (uint64_t *)calloc((size_t)S * nT, sizeof(uint64_t));
    return p;
}

void or_pt_destroy(or_pt *p) {
    if (!p) return;
    for (int s = 0; s < p->S; ++s) { free(p->abcd[s]); free(p->J[s]); free(p->inc_off[s]); free(p->inc[s]); }
    int64_t nslot = (int64_t)p->S * p->R * p->nT;
    for (int64_t c = 0; c < nslot; ++c) free(p->a[c]);
    free(p->a); free(p->E); free(p->abcd); free(p->J); free(p->inc_off); free(p->inc); free(p->N); free(p->nq);
    free(p->beta); free(p->stat); free(p->qstat); free(p->qhist); free(p->swap_acc); free(p->swap_att);
    free(p->mc_acc); free(p->mc_att);
    free(p);
}

/* One pair update of configuration slot c (sample s, temperature t) at (sweep, update). */
static void pair_update(or_pt *p, int s, int r, int t, uint32_t sweep, uint32_t u, int j, int k) {
    int64_t c = slot(p, s, r, t);
    double *a = p->a[c];
    double ajn[2], akn[2];
    double U = or_propose(p->seed, (uint32_t)c, sweep, u, a, j, k, ajn, akn);
    const int64_t *off = p->inc_off[s];
    double dH = delta_h_core(p->abcd[s], p->J[s], p->cc, a, j, k, ajn, akn,
                             p->inc[s] + off[j], off[j + 1] - off[j], p->inc[s] + off[k], off[k + 1] - off[k],
                             p->nq[s]);
    p->mc_att[(int64_t)s * p->nT + t]++;
    if (dH <= 0.0 || U < exp(-p->beta[t] * dH)) {
        a[2 * j] = ajn[0]; a[2 * j + 1] = ajn[1];
        a[2 * k] = akn[0]; a[2 * k + 1] = akn[1];
        p->E[c] += dH;
        p->mc_acc[(int64_t)s * p->nT + t]++;
    }
}

/* Reading R9: rescale onto the constraint surface, then recompute H in full. */
void or_pt_resync(or_pt *p) {
    for (int s = 0; s < p->S; ++s)
        for (int r = 0; r < p->R; ++r)
            for (int t = 0; t < p->nT; ++t) {
                int64_t c = slot(p, s, r, t);
                int n = p->N[s];
                double S4 = or_sum_abs_pow(n, p->a[c], 4);
                double f = sqrt(sqrt((double)n / S4));
                for (int k = 0; k < 2 * n; ++k) p->a[c][k] *= f;
                p->E[c] = or_energy(n, p->nq[s], p->abcd[s], p->J[s], p->cc, p->a[c]);
            }
}

void or_pt_measure_now(or_pt *p) {
    for (int s = 0; s < p->S; ++s) {
        int n = p->N[s];
        for (int t = 0; t < p->nT; ++t) {
            double *st = p->stat + ((int64_t)s * p->nT + t) * OR_NSTAT;
            for (int r = 0; r < p->R; ++r) {
                int64_t c = slot(p, s, r, t);
                double E = p->E[c], I = or_sum_abs_pow(n, p->a[c], 2);
                st[0] += 1.0; st[1] += E; st[2] += E * E;
                st[3] += or_ipr(n, p->a[c], 2); st[4] += or_ipr(n, p->a[c], 4);
                st[5] += I; st[6] += I * I;
            }
            double *qs = p->qstat + ((int64_t)s * p->nT + t) * OR_NQSTAT;
            uint64_t *h = p->qhist + ((int64_t)s * p->nT + t) * OR_NBINS;
            for (int r1 = 0; r1 < p->R; ++r1)
                for (int r2 = r1 + 1; r2 < p->R; ++r2) {
                    double q = or_overlap(n, p->a[slot(p, s, r1, t)], p->a[slot(p, s, r2, t)]);
                    qs[0] += 1.0; qs[1] += q; qs[2] += q * q; qs[3] += q * q * q; qs[4] += q * q * q * q;
                    h[or_qbin(q)]++;
                }
        }
    }
}

/* One sequential swap pass on every (sample, replica) ladder (Sec. III.A.2, reading R7). */
void or_pt_swap(or_pt *p) {
    uint32_t pass = (uint32_t)p->swap_passes;
    for (int s = 0; s < p->S; ++s)
        for (int r = 0; r < p->R; ++r) {
            uint32_t ladder = (uint32_t)(s * p->R + r);
            for (int i = 0; i + 1 < p->nT; ++i) {
                uint32_t w[4];
                draw(p->seed, ladder, pass, (uint32_t)i, OR_TAG_SWAP, w);
                int64_t c0 = slot(p, s, r, i), c1 = slot(p, s, r, i + 1);
                double D = (p->beta[i] - p->beta[i + 1]) * (p->E[c0] - p->E[c1]);
                int64_t pi = ((int64_t)s * p->R + r) * (p->nT - 1) + i;
                p->swap_att[pi]++;
                if (D >= 0.0 || or_uniform(w[0]) < exp(D)) {
                    double *ta = p->a[c0]; p->a[c0] = p->a[c1]; p->a[c1] = ta;
                    double te = p->E[c0]; p->E[c0] = p->E[c1]; p->E[c1] = te;
                    p->swap_acc[pi]++;
                }
            }
        }
    p->swap_passes++;
}

/* n sweeps of every configuration; after each sweep the schedule resync -> measure -> swap. */
void or_pt_sweep(or_pt *p, int64_t nsweeps) {
    for (int64_t it = 0; it < nsweeps; ++it) {
        uint32_t sweep = (uint32_t)p->sweeps_done;
        for (int s = 0; s < p->S; ++s) {
            int n = p->N[s];
            for (int u = 0; u < n / 2; ++u) {
                int j, k;
                or_pair(p->seed, (uint32_t)s, sweep, (uint32_t)u, n, &j, &k);
                for (int r = 0; r < p->R; ++r)
                    for (int t = 0; t < p->nT; ++t) pair_update(p, s, r, t, sweep, (uint32_t)u, j, k);
            }
        }
        p->sweeps_done++;
        int64_t d = p->sweeps_done;
        if (p->resync_every > 0 && d % p->resync_every == 0) or_pt_resync(p);
        if (p->measure_every > 0 && d % p->measure_every == 0) or_pt_measure_now(p);
        if (p->swap_every > 0 && d % p->swap_every == 0 && p->nT > 1) or_pt_swap(p);
    }
}

/* State in canonical (sample, replica, temperature) order: a as interleaved (re, im). */
void or_pt_get_state(const or_pt *p, double *a_out, double *E_out) {
    int64_t pos = 0;
    for (int s = 0; s < p->S; ++s)
        for (int r = 0; r < p->R; ++r)
            for (int t = 0; t < p->nT; ++t) {
                int64_t c = slot(p, s, r, t);
                if (a_out) memcpy(a_out + pos, p->a[c], sizeof(double) * 2 * (size_t)p->N[s]);
                pos += 2 * p->N[s];
                if (E_out) E_out[c] = p->E[c];
            }
}

void or_pt_set_state(or_pt *p, const double *a_in) {
    int64_t pos = 0;
    for (int s = 0; s < p->S; ++s)
        for (int r = 0; r < p->R; ++r)
            for (int t = 0; t < p->nT; ++t) {
                int64_t c = slot(p, s, r, t);
                memcpy(p->a[c], a_in + pos, sizeof(double) * 2 * (size_t)p->N[s]);
                pos += 2 * p->N[s];
                p->E[c] = or_energy(p->N[s], p->nq[s], p->abcd[s], p->J[s], p->cc, p->a[c]);
            }
}

void or_pt_get_observables(const or_pt *p, double *stat, double *qstat, uint64_t *qhist, uint64_t *swap_acc,
                           uint64_t *swap_att, uint64_t *mc_acc, uint64_t *mc_att) {
    int64_t ST = (int64_t)p->S * p->nT;
    int64_t npair = (int64_t)p->S * p->R * (p->nT > 1 ? p->nT - 1 : 1);
    if (stat) memcpy(stat, p->stat, sizeof(double) * (size_t)(ST * OR_NSTAT));
    if (qstat) memcpy(qstat, p->qstat, sizeof(double) * (size_t)(ST * OR_NQSTAT));
    if (qhist) memcpy(qhist, p->qhist, sizeof(uint64_t) * (size_t)(ST * OR_NBINS));
    if (swap_acc) memcpy(swap_acc, p->swap_acc, sizeof(uint64_t) * (size_t)npair);
    if (swap_att) memcpy(swap_att, p->swap_att, sizeof(uint64_t) * (size_t)npair);
    if (mc_acc) memcpy(mc_acc, p->mc_acc, sizeof(uint64_t) * (size_t)ST);
    if (mc_att) memcpy(mc_att, p->mc_att, sizeof(uint64_t) * (size_t)ST);
}

void or_pt_reset_observables(or_pt *p) {
    int64_t ST = (int64_t)p->S * p->nT;
    int64_t npair = (int64_t)p->S * p->R * (p->nT > 1 ? p->nT - 1 : 1);
    memset(p->stat, 0, sizeof(double) * (size_t)(ST * OR_NSTAT));
    memset(p->qstat, 0, sizeof(double) * (size_t)(ST * OR_NQSTAT));
    memset(p->qhist, 0, sizeof(uint64_t) * (size_t)(ST * OR_NBINS));
    memset(p->swap_acc, 0, sizeof(uint64_t) * (size_t)npair);
    memset(p->swap_att, 0, sizeof(uint64_t) * (size_t)npair);
    memset(p->mc_acc, 0, sizeof(uint64_t) * (size_t)ST);
    memset(p->mc_att, 0, sizeof(uint64_t) * (size_t)ST);
}

int64_t or_pt_sweeps_done(const or_pt *p) { return p->sweeps_done; }
