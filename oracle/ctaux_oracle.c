/*
 * ctaux_oracle.c -- TEST INFRASTRUCTURE ONLY (the oracle).
 *
 * A plain, slow, FP64 CPU implementation of the CT-AUX walker that the GPU
 * library must reproduce.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this code; the product path never
 * does.  It shares no code, header, table or helper with the CUDA library.
 *
 * What it follows (DCA++ paper, Sec. 2.3 "Continuous-time auxiliary-field
 * quantum Monte Carlo"):
 *   - expansion of Z in the interaction picture with the constant K
 *     (Eq. Z_interaction_rep and the order-k expansion after it);
 *   - the auxiliary-spin decoupling  1 - beta H_int / K =
 *     (1/2N_corr) sum_s exp(gamma s (n_up - n_dn)),
 *     cosh(gamma) = 1 + U beta N_corr / (2K), with N_corr = Nc for the
 *     single-band Hubbard model (decoupling equations of Sec. 2.3);
 *   - configuration weight (K / (2 beta N_corr))^k prod_sigma det N_sigma^-1
 *     (Eq. Zk), sampled by Metropolis with single-spin insert / remove
 *     moves, each a rank-1 change of N_sigma^-1 (text after Eq. Zk);
 *   - sign tracking for the negative-sign problem (Sec. 2.3, end);
 *   - the Green's function measured from M = (e^V - 1) N (the equation for
 *     <G> in terms of M in Sec. 2.3), here on a tau grid.
 *
 * Readings taken where the paper is silent:
 *   N_sigma^-1 = e^{V_sigma} - g0_sigma (e^{V_sigma} - 1),  g0 = -G0
 *     (G0 in the paper's sign convention, negative on (0, beta)),
 *     V_p^sigma = sigma * gamma * s_p for an interacting vertex, 0 otherwise;
 *   equal-time entries use g0(0+); g0(tau - beta) = -g0(tau);
 *   insert / remove proposed with probability 1/2 each; optionally (flip_frac
 *     > 0) an auxiliary-spin flip of a uniformly chosen vertex with
 *     probability flip_frac first (R = rho_up rho_dn, order unchanged);
 *   acceptance  u < |R|,  R = K/(k+1) rho_up rho_dn (insert),
 *                         R = k/K     rho_up rho_dn (remove);
 *   a warm-up sweep is max(k, 1) proposals, k taken at the start of the
 *     sweep; at the end of warm-up the sweep length is frozen to
 *     L = max(1, round(mean of those k over the warm-up sweeps)) (or to
 *     max(k, 1) when there is no warm-up), so that the measured sweeps
 *     sample the stationary distribution (a state-dependent sweep length
 *     would bias the configurations seen at measurement time);
 *   random numbers: Philox4x32-10 (Salmon et al., SC'11) with
 *     key = (lo32(seed), hi32(seed) ^ walker_id) and
 *     counter = (lo32(j), hi32(j), tag, 0).
 *
 * The oracle does one proposal at a time with full rank-1 updates of N_sigma.
 * An insertion first extends N by the new vertex as a non-interacting one
 * (its row of N^-1 is -g0[p,:](e^V - 1), its column e_p), then changes V_p;
 * the ratio is the matrix determinant lemma det(A + c e_p^T) / det(A) =
 * 1 + e_p^T A^-1 c for A = N^-1 = I + (I - g0)(e^V - I), whose column p
 * changes by c when V_p does, and N follows by Sherman-Morrison.  A removal
 * uses Jacobi's identity (A^-1)_pp = det A_{\p\p} / det A for the ratio and
 * the Schur-complement downdate for N.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_OOM (-3)
#define ORC_ERR_NUMERIC (-5)

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from its definition in Salmon, Moraes, Dror, Shaw,  */
/* "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds  */
/* of the 4x32 S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and a   */
/* Weyl key schedule with increments 0x9E3779B9 / 0xBB67AE85.          */
/* ------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Uniform double in [0,1) with 53 random bits from two words. */
static double u53(uint32_t hi, uint32_t lo)
{
    uint64_t w = ((uint64_t)hi << 32) | (uint64_t)lo;
    return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

/* floor(w * m / 2^32): an index in [0, m) with no floating point. */
static uint32_t index_of(uint32_t w, uint32_t m)
{
    return (uint32_t)(((uint64_t)w * (uint64_t)m) >> 32);
}

enum { TAG_PROPOSAL = 0, TAG_ACCEPT = 1, TAG_INIT = 2 };

static void draw(const uint32_t key[2], uint64_t j, uint32_t tag, uint32_t out[4])
{
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)(j >> 32), tag, 0u};
    orc_philox4x32_10(ctr, key, out);
}

/* ------------------------------------------------------------------ */
/* Parameters and state                                                */
/* ------------------------------------------------------------------ */
typedef struct {
    int32_t nc;
    const int32_t* site_sub;  /* [nc*nc] index of r_i - r_j folded into the cluster */
    double U, beta, K;
    int32_t n_tau;            /* table intervals; samples at l*beta/n_tau, l=0..n_tau */
    const double* G0;         /* [2][nc][n_tau+1] paper sign convention */
    int32_t warmup_sweeps;
    int32_t n_tau_meas;       /* measurement grid: tau_a = (a + 1/2) beta / n_tau_meas */
    uint64_t seed;
    uint32_t walker_id;
    int32_t init_config_size;
    double tie_eps;           /* near-tie threshold on | |R| - u | */
    double flip_frac;         /* probability of an auxiliary-spin flip proposal (0 = none) */
    int32_t neglect_ks;       /* > 0: windows of this many proposals with the neglect rule (below) */
} orc_params;

typedef struct {
    int32_t nc, n_tau, n_meas_tau, warmup;
    double U, beta, K, gamma, tie_eps;
    int32_t* site_sub;        /* [nc*nc] */
    int32_t* site_add;        /* [nc*nc]: site_add[y*nc + d] = x with site_sub[x*nc+y] == d */
    double* g0;               /* [2][nc][n_tau+1], g0 = -G0 */
    double expV[2][2];        /* e^{sigma gamma s}: [spin 0=up,1=dn][s 0:-1, 1:+1] */
    uint32_t key[2];
    uint64_t q;               /* next proposal index */
    int32_t k, cap;
    int32_t* vsite; double* vtau; int8_t* vs;
    double* N[2];             /* k x k row-major, leading dimension cap */
    double* work;             /* scratch vectors */
    double sign;
    int64_t sweeps_done;
    int64_t warm_k_sum;       /* sum of k at the start of each warm-up sweep */
    int64_t sweep_len;        /* frozen measured-sweep length, 0 until set */
    double* Gacc;             /* [2][nc][n_tau_meas] sum of sign * G(paper convention) */
    double sign_sum;
    int64_t n_meas;
    uint8_t* log; int64_t log_n, log_cap;
    const uint8_t* hints; int64_t hints_n;
    int64_t n_prop, n_acc, n_ties, n_adopted;
    double k_sum; int64_t k_samples;   /* k_sum: sum over measurements of sign * k */
    uint32_t flip_thr;        /* a proposal is a flip when (word0 >> 2) < flip_thr */
    int32_t neglect_ks;       /* neglect rule: window length (0 = off) */
    int64_t win_id;           /* neglect rule: current window (counted over the run) */
    int64_t* changed;         /* [cap] window in which each vertex was last changed (neglect rule) */
    int64_t n_neglected;      /* proposals rejected by the neglect rule */
    double* Nsave[2];         /* copies of N while a flip is decided */
    int32_t n_omega;          /* frequency measurement: positive Matsubara frequencies, 0 = off */
    double* Macc;             /* [2][nc][n_omega][re, im]: sum of sign * M(dr, i w_n) */
    int32_t n_w4;             /* two-particle measurement: fermionic frequencies per sign, 0 = off */
    int32_t m4;               /* its bosonic transfer index, nu = 2 pi m4 / beta */
    double* kdotr;            /* [nc][nc] K_a . r_s */
    int32_t* k_dn;            /* [nc] index of Q - K for each K */
    double* G4acc;            /* [S][S][re, im]: sum of sign * M_up(s1, s2) M_dn(s1, s2) */
    double* G4d;              /* [2][S][re, im]: sum of sign * M_sigma(s, s) */
} orc_walker;

/* ------------------------------------------------------------------ */
/* g0 interpolation: linear on the uniform tau grid, antiperiodic      */
/* extension to (-beta, 0), dtau == 0 read as 0+.                      */
/* ------------------------------------------------------------------ */
static double g0_row(const double* row, int n_tau, double beta, double dtau)
{
    double sgn = 1.0;
    if (dtau < 0.0) {
        dtau += beta;
        sgn = -1.0;
    }
    double x = dtau * ((double)n_tau / beta);
    int l = (int)x;
    if (l >= n_tau) l = n_tau - 1;
    if (l < 0) l = 0;
    double f = x - (double)l;
    return sgn * (row[l] + f * (row[l + 1] - row[l]));
}

double orc_g0_interp(const double* row, int32_t n_tau, double beta, double dtau)
{
    return g0_row(row, n_tau, beta, dtau);
}

/* g0_sigma(r_a - r_b, tau_a - tau_b) */
static double g0ab(const orc_walker* w, int sp, int32_t ra, double ta, int32_t rb, double tb)
{
    int d = w->site_sub[ra * w->nc + rb];
    const double* row = w->g0 + ((size_t)sp * w->nc + d) * (size_t)(w->n_tau + 1);
    return g0_row(row, w->n_tau, w->beta, ta - tb);
}

static double ev(const orc_walker* w, int sp, int8_t s) { return w->expV[sp][s > 0 ? 1 : 0]; }

/* ------------------------------------------------------------------ */
/* Dense FP64 helpers (plain loops)                                    */
/* ------------------------------------------------------------------ */

/* Build A = e^V - g0 (e^V - 1) for the given vertices, row-major n x n. */
static void build_A(const orc_walker* w, int sp, int n, const int32_t* site, const double* tau,
                    const int8_t* s, double* A)
{
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double evj = ev(w, sp, s[j]);
            double gij = (i == j) ? g0ab(w, sp, site[i], 0.0, site[i], 0.0)
                                  : g0ab(w, sp, site[i], tau[i], site[j], tau[j]);
            A[(size_t)i * n + j] = ((i == j) ? evj : 0.0) - gij * (evj - 1.0);
        }
    }
}

/* Gauss-Jordan inverse with partial pivoting. A (n x n, row-major) is
 * destroyed; inv gets the inverse with leading dimension ldi.  Returns the
 * sign of det A (0 if singular). */
static int gj_inverse(int n, double* A, double* inv, int ldi)
{
    int sgn = 1;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[(size_t)i * ldi + j] = (i == j) ? 1.0 : 0.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = fabs(A[(size_t)c * n + c]);
        for (int r = c + 1; r < n; ++r) {
            double v = fabs(A[(size_t)r * n + c]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) return 0;
        if (piv != c) {
            sgn = -sgn;
            for (int j = 0; j < n; ++j) {
                double t = A[(size_t)c * n + j]; A[(size_t)c * n + j] = A[(size_t)piv * n + j]; A[(size_t)piv * n + j] = t;
                t = inv[(size_t)c * ldi + j]; inv[(size_t)c * ldi + j] = inv[(size_t)piv * ldi + j]; inv[(size_t)piv * ldi + j] = t;
            }
        }
        double d = A[(size_t)c * n + c];
        if (d < 0.0) sgn = -sgn;
        double rd = 1.0 / d;
        for (int j = 0; j < n; ++j) { A[(size_t)c * n + j] *= rd; inv[(size_t)c * ldi + j] *= rd; }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = A[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                A[(size_t)r * n + j] -= f * A[(size_t)c * n + j];
                inv[(size_t)r * ldi + j] -= f * inv[(size_t)c * ldi + j];
            }
        }
    }
    return sgn;
}

/* ------------------------------------------------------------------ */
/* Creation                                                            */
/* ------------------------------------------------------------------ */
static int ensure_cap(orc_walker* w, int need)
{
    if (need <= w->cap) return ORC_OK;
    int nc = w->cap ? w->cap : 16;
    while (nc < need) nc *= 2;
    int32_t* vsite = (int32_t*)realloc(w->vsite, sizeof(int32_t) * nc);
    if (!vsite) return ORC_ERR_OOM;
    w->vsite = vsite;
    double* vtau = (double*)realloc(w->vtau, sizeof(double) * nc);
    if (!vtau) return ORC_ERR_OOM;
    w->vtau = vtau;
    int8_t* vs = (int8_t*)realloc(w->vs, (size_t)nc);
    if (!vs) return ORC_ERR_OOM;
    w->vs = vs;
    for (int sp = 0; sp < 2; ++sp) {
        double* M = (double*)calloc((size_t)nc * nc, sizeof(double));
        if (!M) return ORC_ERR_OOM;
        for (int i = 0; i < w->k; ++i)
            memcpy(M + (size_t)i * nc, w->N[sp] + (size_t)i * w->cap, sizeof(double) * w->k);
        free(w->N[sp]);
        w->N[sp] = M;
    }
    double* work = (double*)realloc(w->work, sizeof(double) * 8 * (size_t)nc);
    if (!work) return ORC_ERR_OOM;
    w->work = work;
    int64_t* changed = (int64_t*)realloc(w->changed, sizeof(int64_t) * nc);
    if (!changed) return ORC_ERR_OOM;
    for (int i = w->cap; i < nc; ++i) changed[i] = -1;
    w->changed = changed;
    for (int sp = 0; sp < 2; ++sp) {
        free(w->Nsave[sp]);
        w->Nsave[sp] = (double*)malloc(sizeof(double) * (size_t)nc * nc);
        if (!w->Nsave[sp]) return ORC_ERR_OOM;
    }
    w->cap = nc;
    return ORC_OK;
}

void orc_destroy(orc_walker* w)
{
    if (!w) return;
    free(w->site_sub); free(w->site_add); free(w->g0);
    free(w->vsite); free(w->vtau); free(w->vs);
    free(w->N[0]); free(w->N[1]); free(w->work);
    free(w->Gacc); free(w->log); free(w->Macc);
    free(w->kdotr); free(w->k_dn); free(w->G4acc); free(w->G4d);
    free(w->changed); free(w->Nsave[0]); free(w->Nsave[1]);
    free(w);
}

/* Rebuild both N matrices from the vertex list; sets the sign of
 * prod_sigma det N_sigma^-1.  Returns ORC_ERR_NUMERIC if singular. */
static int rebuild_N(orc_walker* w, double* sign_out)
{
    int n = w->k;
    int total_sign = 1;
    if (n == 0) { if (sign_out) *sign_out = 1.0; return ORC_OK; }
    double* A = (double*)malloc(sizeof(double) * (size_t)n * n);
    if (!A) return ORC_ERR_OOM;
    for (int sp = 0; sp < 2; ++sp) {
        build_A(w, sp, n, w->vsite, w->vtau, w->vs, A);
        int sg = gj_inverse(n, A, w->N[sp], w->cap);
        if (sg == 0) { free(A); return ORC_ERR_NUMERIC; }
        total_sign *= sg;
    }
    free(A);
    if (sign_out) *sign_out = (double)total_sign;
    return ORC_OK;
}

orc_walker* orc_create(const orc_params* p, int* err)
{
    *err = ORC_ERR_ARG;
    if (!p || p->nc < 1 || !p->site_sub || !p->G0 || p->n_tau < 1 || !(p->beta > 0.0) ||
        !(p->K > 0.0) || p->U < 0.0 || p->n_tau_meas < 1 || p->init_config_size < 0 || p->warmup_sweeps < 0)
        return NULL;
    orc_walker* w = (orc_walker*)calloc(1, sizeof(orc_walker));
    if (!w) { *err = ORC_ERR_OOM; return NULL; }
    int nc = p->nc;
    w->nc = nc; w->n_tau = p->n_tau; w->n_meas_tau = p->n_tau_meas; w->warmup = p->warmup_sweeps;
    w->U = p->U; w->beta = p->beta; w->K = p->K;
    w->tie_eps = p->tie_eps > 0.0 ? p->tie_eps : 1e-10;
    /* cosh(gamma) = 1 + U beta N_corr / (2K), N_corr = Nc */
    w->gamma = acosh(1.0 + p->U * p->beta * (double)nc / (2.0 * p->K));
    for (int sp = 0; sp < 2; ++sp) {
        double sigma = sp == 0 ? 1.0 : -1.0;
        w->expV[sp][0] = exp(-sigma * w->gamma);
        w->expV[sp][1] = exp(sigma * w->gamma);
    }
    w->site_sub = (int32_t*)malloc(sizeof(int32_t) * nc * nc);
    w->site_add = (int32_t*)malloc(sizeof(int32_t) * nc * nc);
    size_t tsz = (size_t)2 * nc * (p->n_tau + 1);
    w->g0 = (double*)malloc(sizeof(double) * tsz);
    w->Gacc = (double*)calloc((size_t)2 * nc * p->n_tau_meas, sizeof(double));
    if (!w->site_sub || !w->site_add || !w->g0 || !w->Gacc) { orc_destroy(w); *err = ORC_ERR_OOM; return NULL; }
    memcpy(w->site_sub, p->site_sub, sizeof(int32_t) * nc * nc);
    for (int i = 0; i < nc * nc; ++i) {
        if (w->site_sub[i] < 0 || w->site_sub[i] >= nc) { orc_destroy(w); return NULL; }
        w->site_add[i] = -1;
    }
    for (int x = 0; x < nc; ++x)
        for (int y = 0; y < nc; ++y) w->site_add[y * nc + w->site_sub[x * nc + y]] = x;
    for (int i = 0; i < nc * nc; ++i)
        if (w->site_add[i] < 0) { orc_destroy(w); return NULL; }
    for (size_t i = 0; i < tsz; ++i) w->g0[i] = -p->G0[i];
    w->key[0] = (uint32_t)p->seed;
    w->key[1] = (uint32_t)(p->seed >> 32) ^ p->walker_id;
    w->sign = 1.0;
    if (!(p->flip_frac >= 0.0) || p->flip_frac > 1.0 || p->neglect_ks < 0) { orc_destroy(w); return NULL; }
    /* flip when the 30 bits of word 0 above its type and spin bits fall below
     * flip_frac of their range (the integer threshold both sides compute) */
    w->flip_thr = (uint32_t)floor(p->flip_frac * 1073741824.0);
    w->neglect_ks = p->neglect_ks;

    /* Initial configuration: init_config_size random interacting vertices
     * (App. B, "initial-configuration-size"). */
    int n0 = p->init_config_size;
    if (ensure_cap(w, n0 > 0 ? n0 : 1) != ORC_OK) { orc_destroy(w); *err = ORC_ERR_OOM; return NULL; }
    for (int i = 0; i < n0; ++i) {
        uint32_t r[4];
        draw(w->key, (uint64_t)i, TAG_INIT, r);
        w->vs[i] = (r[0] & 2u) ? 1 : -1;
        w->vsite[i] = (int32_t)index_of(r[1], (uint32_t)nc);
        w->vtau[i] = p->beta * u53(r[2], r[3]);
    }
    w->k = n0;
    int rc = rebuild_N(w, &w->sign);
    if (rc != ORC_OK) { orc_destroy(w); *err = rc; return NULL; }
    *err = ORC_OK;
    return w;
}

/* ------------------------------------------------------------------ */
/* One proposal                                                        */
/* ------------------------------------------------------------------ */
static void log_push(orc_walker* w, uint8_t v)
{
    if (!w->log) return;
    if (w->log_n < w->log_cap) w->log[w->log_n] = v;
    w->log_n++;
}

static int decide(orc_walker* w, double absR, double u, uint64_t q, int* tie)
{
    int acc = u < absR;
    *tie = fabs(absR - u) < w->tie_eps;
    if (*tie) {
        w->n_ties++;
        if (w->hints && q < (uint64_t)w->hints_n) {
            acc = w->hints[q] & 1;
            w->n_adopted++;
        }
    }
    return acc;
}

/* Ratio of inserting vertex (site, tau, s) as row/column k: fills the work
 * vectors X (new row of the extended N), col (column change of A) and
 * wv = N_ext col per spin, and rho = 1 + wv[k] (matrix determinant lemma). */
static int insert_ratio(orc_walker* w, int32_t site, double tau, int8_t s, double rho[2])
{
    int n = w->k;
    int rc = ensure_cap(w, n + 1);
    if (rc != ORC_OK) return rc;
    int ld = w->cap;
    for (int sp = 0; sp < 2; ++sp) {
        double* X = w->work + (size_t)(4 * sp + 0) * ld;
        double* col = w->work + (size_t)(4 * sp + 1) * ld;
        double* wv = w->work + (size_t)(4 * sp + 2) * ld;
        double* N = w->N[sp];
        double* urow = w->work + (size_t)(4 * sp + 3) * ld;
        /* New (non-interacting) row of the extended N: X = g0[p,:] (e^V - 1) N. */
        for (int i = 0; i < n; ++i)
            urow[i] = g0ab(w, sp, site, tau, w->vsite[i], w->vtau[i]) * (ev(w, sp, w->vs[i]) - 1.0);
        for (int j = 0; j < n; ++j) {
            double acc = 0.0;
            for (int i = 0; i < n; ++i) acc += urow[i] * N[(size_t)i * ld + j];
            X[j] = acc;
        }
        /* Column change of A when V_p goes 0 -> sigma gamma s:
         * c = (I - g0_ext)[:,p] * (e^{V'} - 1). */
        double delta = ev(w, sp, s) - 1.0;
        for (int i = 0; i < n; ++i)
            col[i] = -g0ab(w, sp, w->vsite[i], w->vtau[i], site, tau) * delta;
        col[n] = (1.0 - g0ab(w, sp, site, 0.0, site, 0.0)) * delta;
        /* wv = N_ext c ; N_ext = [[N, 0], [X, 1]]. */
        for (int i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc += N[(size_t)i * ld + j] * col[j];
            wv[i] = acc;
        }
        {
            double acc = 0.0;
            for (int j = 0; j < n; ++j) acc += X[j] * col[j];
            wv[n] = acc + col[n];
        }
        rho[sp] = 1.0 + wv[n];
    }
    return ORC_OK;
}

/* Apply the insertion whose work vectors insert_ratio left: N' = N_ext -
 * wv (e_p^T N_ext) / rho, the vertex appended as row/column k. */
static void insert_apply(orc_walker* w, int32_t site, double tau, int8_t s, const double rho[2])
{
    int n = w->k;
    int ld = w->cap;
    for (int sp = 0; sp < 2; ++sp) {
        double* N = w->N[sp];
        const double* X = w->work + (size_t)(4 * sp + 0) * ld;
        const double* wv = w->work + (size_t)(4 * sp + 2) * ld;
        for (int j = 0; j < n; ++j) { N[(size_t)n * ld + j] = X[j]; N[(size_t)j * ld + n] = 0.0; }
        N[(size_t)n * ld + n] = 1.0;
        double* rowp = w->work + (size_t)(4 * sp + 3) * ld;
        for (int j = 0; j <= n; ++j) rowp[j] = N[(size_t)n * ld + j];
        double inv = 1.0 / rho[sp];
        for (int i = 0; i <= n; ++i) {
            double f = wv[i] * inv;
            if (f == 0.0) continue;
            for (int j = 0; j <= n; ++j) N[(size_t)i * ld + j] -= f * rowp[j];
        }
    }
    w->vsite[n] = site; w->vtau[n] = tau; w->vs[n] = s;
    w->changed[n] = w->win_id;
    w->k = n + 1;
}

/* Insert vertex (site, tau, s) as row/column k. */
static int propose_insert(orc_walker* w, int32_t site, double tau, int8_t s, double u, uint64_t q)
{
    double rho[2];
    int rc = insert_ratio(w, site, tau, s, rho);
    if (rc != ORC_OK) return rc;
    double R = w->K / (double)(w->k + 1) * rho[0] * rho[1];
    if (!isfinite(R)) return ORC_ERR_NUMERIC;
    int tie;
    int acc = decide(w, fabs(R), u, q, &tie);
    w->n_prop++;
    log_push(w, (uint8_t)(acc | (tie << 1)));
    if (!acc) return ORC_OK;
    w->n_acc++;
    if (R < 0.0) w->sign = -w->sign;
    insert_apply(w, site, tau, s, rho);
    return ORC_OK;
}

/* Remove vertex p from the vertex list and N by the Schur-complement
 * downdate N'_rs = N_rs - N_rp N_ps / N_pp (r, s != p). */
static void remove_apply(orc_walker* w, int p)
{
    int n = w->k;
    int ld = w->cap;
    for (int sp = 0; sp < 2; ++sp) {
        double* N = w->N[sp];
        double* rowp = w->work + (size_t)(4 * sp + 3) * ld;
        double* colp = w->work + (size_t)(4 * sp + 2) * ld;
        for (int j = 0; j < n; ++j) { rowp[j] = N[(size_t)p * ld + j]; colp[j] = N[(size_t)j * ld + p]; }
        double inv = 1.0 / N[(size_t)p * ld + p];
        for (int i = 0, ii = 0; i < n; ++i) {
            if (i == p) continue;
            double f = colp[i] * inv;
            for (int j = 0, jj = 0; j < n; ++j) {
                if (j == p) continue;
                /* write position (ii, jj) never passes the read position (i, j) */
                N[(size_t)ii * ld + jj] = N[(size_t)i * ld + j] - f * rowp[j];
                ++jj;
            }
            ++ii;
        }
    }
    for (int i = p; i < n - 1; ++i) {
        w->vsite[i] = w->vsite[i + 1]; w->vtau[i] = w->vtau[i + 1]; w->vs[i] = w->vs[i + 1];
        w->changed[i] = w->changed[i + 1];
    }
    w->k = n - 1;
}

/* Remove vertex p.  With A = N^-1, the ratio det A_{\p\p} / det A is
 * (A^-1)_pp = N_pp (Jacobi's identity / Cramer's rule). */
static int propose_remove(orc_walker* w, int p, double u, uint64_t q)
{
    int n = w->k;
    int ld = w->cap;
    double rho[2];
    for (int sp = 0; sp < 2; ++sp) rho[sp] = w->N[sp][(size_t)p * ld + p];
    double R = (double)n / w->K * rho[0] * rho[1];
    if (!isfinite(R)) return ORC_ERR_NUMERIC;
    int tie;
    int acc = decide(w, fabs(R), u, q, &tie);
    w->n_prop++;
    log_push(w, (uint8_t)(acc | (tie << 1)));
    if (!acc) return ORC_OK;
    w->n_acc++;
    if (R < 0.0) w->sign = -w->sign;
    remove_apply(w, p);
    return ORC_OK;
}

/* Flip the auxiliary spin of vertex p (the third single-spin update of
 * Sec. 2.3): the order k is unchanged, so R = prod_sigma det A'/det A.  The
 * flip is carried out as the removal of p (Jacobi ratio N_pp, Schur
 * downdate) followed by the insertion of (r_p, tau_p, -s_p) (determinant
 * lemma, Sherman-Morrison), R = prod_sigma N_pp rho_ins, and the inserted
 * row and column are moved back to position p; a rejected flip restores the
 * saved N.  (A direct rank-1 change of column p by e^{-V_p} - e^{V_p} would
 * amplify rounding by that factor, as for removals.) */
static int propose_flip(orc_walker* w, int p, double u, uint64_t q, double* rho_out)
{
    int n = w->k;
    int ld = w->cap;
    for (int sp = 0; sp < 2; ++sp)
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) w->Nsave[sp][(size_t)i * ld + j] = w->N[sp][(size_t)i * ld + j];
    const int32_t site = w->vsite[p];
    const double tau = w->vtau[p];
    const int8_t s = w->vs[p];
    const int64_t ch = w->changed[p];
    double rho_rem[2], rho_ins[2];
    for (int sp = 0; sp < 2; ++sp) rho_rem[sp] = w->N[sp][(size_t)p * ld + p];
    remove_apply(w, p);
    int rc = insert_ratio(w, site, tau, (int8_t)-s, rho_ins);
    if (rc != ORC_OK) return rc;
    double R = rho_rem[0] * rho_ins[0] * rho_rem[1] * rho_ins[1];
    if (rho_out)
        for (int sp = 0; sp < 2; ++sp) rho_out[sp] = rho_rem[sp] * rho_ins[sp];
    if (!isfinite(R)) return ORC_ERR_NUMERIC;
    int tie;
    int acc = decide(w, fabs(R), u, q, &tie);
    w->n_prop++;
    log_push(w, (uint8_t)(acc | (tie << 1)));
    if (!acc) {
        /* restore: vertex p and the saved N */
        for (int i = n - 1; i > p; --i) {
            w->vsite[i] = w->vsite[i - 1]; w->vtau[i] = w->vtau[i - 1]; w->vs[i] = w->vs[i - 1];
            w->changed[i] = w->changed[i - 1];
        }
        w->vsite[p] = site; w->vtau[p] = tau; w->vs[p] = s; w->changed[p] = ch;
        w->k = n;
        for (int sp = 0; sp < 2; ++sp)
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) w->N[sp][(size_t)i * ld + j] = w->Nsave[sp][(size_t)i * ld + j];
        return ORC_OK;
    }
    w->n_acc++;
    if (R < 0.0) w->sign = -w->sign;
    insert_apply(w, site, tau, (int8_t)-s, rho_ins);
    /* move row and column n - 1 back to position p */
    for (int sp = 0; sp < 2; ++sp) {
        double* N = w->N[sp];
        double* tmp = w->work + (size_t)(4 * sp + 3) * ld;
        for (int j = 0; j < n; ++j) tmp[j] = N[(size_t)(n - 1) * ld + j];
        for (int i = n - 1; i > p; --i)
            for (int j = 0; j < n; ++j) N[(size_t)i * ld + j] = N[(size_t)(i - 1) * ld + j];
        for (int j = 0; j < n; ++j) N[(size_t)p * ld + j] = tmp[j];
        for (int i = 0; i < n; ++i) {
            double* row = N + (size_t)i * ld;
            double v = row[n - 1];
            for (int j = n - 1; j > p; --j) row[j] = row[j - 1];
            row[p] = v;
        }
    }
    for (int i = n - 1; i > p; --i) {
        w->vsite[i] = w->vsite[i - 1]; w->vtau[i] = w->vtau[i - 1]; w->vs[i] = w->vs[i - 1];
        w->changed[i] = w->changed[i - 1];
    }
    w->vsite[p] = site; w->vtau[p] = tau; w->vs[p] = (int8_t)-s; w->changed[p] = w->win_id;
    return ORC_OK;
}

/* Proposal number q: type (flip with probability flip_frac, else insert /
 * remove with probability 1/2 each), the new vertex or the index of the
 * vertex to remove or flip, and u for the Metropolis test.  With the
 * neglect rule on, a removal or flip of a vertex already changed in the
 * current window of neglect_ks proposals is rejected (Sec. 2.3, "Submatrix
 * updates": ignoring proposals of already chosen spins; it breaks detailed
 * balance).  Without it the chain is that of single-spin updates (the
 * abort variant of the submatrix method reaches the same chain). */
static int propose(orc_walker* w, uint64_t q)
{
    uint32_t r[4], a[4];
    draw(w->key, q, TAG_PROPOSAL, r);
    draw(w->key, q, TAG_ACCEPT, a);
    double u = u53(a[0], a[1]);
    const int flip = w->flip_thr > 0u && (r[0] >> 2) < w->flip_thr;
    if (!flip && (r[0] & 1u) == 0u) {
        int8_t s = (r[0] & 2u) ? 1 : -1;
        int32_t site = (int32_t)index_of(r[1], (uint32_t)w->nc);
        double tau = w->beta * u53(r[2], r[3]);
        return propose_insert(w, site, tau, s, u, q);
    }
    if (w->k == 0) { /* nothing to remove or flip: rejected */
        w->n_prop++;
        log_push(w, 0);
        return ORC_OK;
    }
    int p = (int)index_of(r[1], (uint32_t)w->k);
    if (w->neglect_ks > 0 && w->changed[p] == w->win_id) {
        w->n_prop++;
        w->n_neglected++;
        log_push(w, 0);
        return ORC_OK;
    }
    return flip ? propose_flip(w, p, u, q, NULL) : propose_remove(w, p, u, q);
}

/* ------------------------------------------------------------------ */
/* Measurement on the tau grid                                         */
/* G(dr, tau_a) = g0(dr, tau_a) + (1/Nc) sum_{r'} sum_{ij}             */
/*   g0(r'+dr - r_i, tau_a - tau_i) M_ij g0(r_j - r', tau_j),          */
/* M = (e^V - 1) N; accumulated as sign * (-G) (paper convention).     */
/* ------------------------------------------------------------------ */
static void measure_freq(orc_walker* w);
static void measure_g4(orc_walker* w);

static void measure(orc_walker* w)
{
    int n = w->k, nc = w->nc, nt = w->n_meas_tau, ld = w->cap;
    double* b = (double*)malloc(sizeof(double) * ((size_t)n * nc + 1));
    for (int sp = 0; sp < 2; ++sp) {
        double* N = w->N[sp];
        /* b[r'][i] = sum_j M_ij g0(r_j - r', tau_j - 0+) */
        for (int rp = 0; rp < nc; ++rp) {
            for (int i = 0; i < n; ++i) {
                double acc = 0.0;
                for (int j = 0; j < n; ++j)
                    acc += N[(size_t)i * ld + j] * g0ab(w, sp, w->vsite[j], w->vtau[j], rp, 0.0);
                b[(size_t)rp * n + i] = (ev(w, sp, w->vs[i]) - 1.0) * acc;
            }
        }
        for (int d = 0; d < nc; ++d) {
            const double* row = w->g0 + ((size_t)sp * nc + d) * (size_t)(w->n_tau + 1);
            for (int a = 0; a < nt; ++a) {
                double ta = ((double)a + 0.5) * w->beta / (double)nt;
                double G = g0_row(row, w->n_tau, w->beta, ta);
                double corr = 0.0;
                for (int rp = 0; rp < nc; ++rp) {
                    int x = w->site_add[rp * nc + d];
                    for (int i = 0; i < n; ++i)
                        corr += g0ab(w, sp, x, ta, w->vsite[i], w->vtau[i]) * b[(size_t)rp * n + i];
                }
                G += corr / (double)nc;
                w->Gacc[((size_t)sp * nc + d) * nt + a] += w->sign * (-G);
            }
        }
    }
    free(b);
    if (w->n_omega > 0) measure_freq(w);
    if (w->n_w4 > 0) measure_g4(w);
    w->sign_sum += w->sign;
    w->n_meas++;
}

/* Frequency-domain measurement of M (Sec. 2.3: the Green's function is
 * linearly related to M, whose Fourier coefficients are accumulated; the
 * delayed-NFFT paragraph evaluates exactly these sums).  With M = (e^V - 1) N
 * and fermionic w_n = (2n + 1) pi / beta,
 *   M(dr, i w_n) = 1/(beta Nc) sum_{i,j : r_i - r_j = dr} M_ij e^{i w_n (tau_i - tau_j)},
 * so that, averaged over the cluster and over time translations,
 *   G(K, i w_n) = g0(K, i w_n) + g0(K, i w_n)^2 M(K, i w_n),
 *   M(K, i w_n) = sum_dr e^{-i K.dr} M(dr, i w_n)
 * (g0 = -G0; in the paper's sign, G = G0 - G0^2 M).  Evaluated here as the
 * plain non-uniform discrete Fourier sum, one cosine and sine per pair and
 * frequency. */
static void measure_freq(orc_walker* w)
{
    const int n = w->k, nc = w->nc, nw = w->n_omega, ld = w->cap;
    const double norm = 1.0 / (w->beta * (double)nc);
    for (int sp = 0; sp < 2; ++sp) {
        const double* N = w->N[sp];
        for (int i = 0; i < n; ++i) {
            const double fi = ev(w, sp, w->vs[i]) - 1.0;
            for (int j = 0; j < n; ++j) {
                const double m = w->sign * fi * N[(size_t)i * ld + j] * norm;
                const int d = w->site_sub[w->vsite[i] * nc + w->vsite[j]];
                const double t = w->vtau[i] - w->vtau[j];
                double* acc = w->Macc + ((size_t)sp * nc + d) * (size_t)nw * 2;
                for (int k = 0; k < nw; ++k) {
                    const double ang = (double)(2 * k + 1) * 3.14159265358979323846 * t / w->beta;
                    acc[2 * k] += m * cos(ang);
                    acc[2 * k + 1] += m * sin(ang);
                }
            }
        }
    }
}

/* Switch the frequency measurement on (n_omega > 0) or off (0); clears it. */
int orc_enable_freq(orc_walker* w, int32_t n_omega)
{
    if (!w || n_omega < 0) return ORC_ERR_ARG;
    free(w->Macc);
    w->Macc = NULL;
    w->n_omega = 0;
    if (n_omega == 0) return ORC_OK;
    w->Macc = (double*)calloc((size_t)2 * w->nc * n_omega * 2, sizeof(double));
    if (!w->Macc) return ORC_ERR_OOM;
    w->n_omega = n_omega;
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Two-particle measurement, particle-particle up-down channel         */
/* ------------------------------------------------------------------ */
/* Within one configuration the problem is quadratic in each spin, so the
 * two-particle Green's function of the particle-particle up-down channel
 * (Sec. 2.5, Eq. bse_cluster; App. B four-point type
 * PARTICLE_PARTICLE_UP_DOWN) factorises into two-point functions of the two
 * spins, which carry no exchange term:
 *   G2(K, K', q) = < G_up(K, K') G_dn(q - K, q - K') >,
 * with the combined index K = (K, i w_n), q = (Q, i nu_m), nu_m = 2 pi m / beta,
 * and per configuration (the two-point form of the relation G = G0 - G0 M G0
 * of Sec. 2.3, in the paper's sign)
 *   G_sigma(k1, k2) = G0_sigma(k1) delta_{k1 k2} - G0_sigma(k1) M_sigma(k1, k2) G0_sigma(k2),
 *   M_sigma(k1, k2) = 1/(beta Nc) sum_{ij} e^{i (w1 tau_i - K1.r_i)} [(e^V - 1) N]_ij e^{-i (w2 tau_j - K2.r_j)},
 * whose diagonal M_sigma(k, k) is the single-particle M(K, i w_n) of
 * measure_freq.  The measured points are s = (K, n) for K over the cluster
 * momenta and n = -n_w4 .. n_w4 - 1 (index s = K * 2 n_w4 + n + n_w4); the
 * spin-down factor is taken at q - s = (Q - K, i w_{m - n - 1}).  What is
 * accumulated is the part that depends on the configuration,
 *   G4acc(s1, s2) = sum sign M_up(s1, s2) M_dn(q - s1, q - s2),
 *   G4d(sigma, s) = sum sign M_sigma(s, s)   (sigma = dn at q - s),
 * from which G2 follows for any G0 by expanding the product (oracle/g4.py):
 *   G2 sum_sign = G0u(s1) G0d(s1) [ delta (sum_sign - G4d_up(s1) G0u(s1) - G4d_dn(s1) G0d(s1))
 *                                  + G4acc(s1, s2) G0u(s2) G0d(s2) ]. */

/* Momentum and frequency of measured point s for spin sp. */
static void g4_point(const orc_walker* w, int sp, int s, int* K, double* wn)
{
    const int nf = 2 * w->n_w4;
    const int k = s / nf, n = s % nf - w->n_w4;
    if (sp == 0) {
        *K = k;
        *wn = (double)(2 * n + 1) * 3.14159265358979323846 / w->beta;
    } else {
        *K = w->k_dn[k];
        *wn = (double)(2 * (w->m4 - n - 1) + 1) * 3.14159265358979323846 / w->beta;
    }
}

/* M_sigma(s1, s2) of the current configuration, out [S][S][re, im] (no sign):
 * T(i, s2) = sum_j c_ij e^{-i phase_j(s2)}, then M(s1, s2) = norm sum_i
 * e^{i phase_i(s1)} T(i, s2), with c = (e^V - 1) N and phase_i(s) = w_s tau_i - K_s.r_i. */
static int g4_m2(const orc_walker* w, int sp, double* out)
{
    const int n = w->k, nc = w->nc, ld = w->cap;
    const int S = nc * 2 * w->n_w4;
    const double norm = 1.0 / (w->beta * (double)nc);
    double* ph = (double*)malloc(sizeof(double) * 2 * (size_t)S * (n > 0 ? n : 1));
    double* T = (double*)malloc(sizeof(double) * 2 * (size_t)S * (n > 0 ? n : 1));
    if (!ph || !T) { free(ph); free(T); return ORC_ERR_OOM; }
    for (int s = 0; s < S; ++s) {
        int K; double wn;
        g4_point(w, sp, s, &K, &wn);
        for (int i = 0; i < n; ++i) {
            const double a = wn * w->vtau[i] - w->kdotr[(size_t)K * nc + w->vsite[i]];
            ph[((size_t)s * n + i) * 2] = cos(a);
            ph[((size_t)s * n + i) * 2 + 1] = sin(a);
        }
    }
    const double* N = w->N[sp];
    for (int i = 0; i < n; ++i) {
        const double fi = ev(w, sp, w->vs[i]) - 1.0;
        for (int s = 0; s < S; ++s) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < n; ++j) {
                const double c = fi * N[(size_t)i * ld + j];
                re += c * ph[((size_t)s * n + j) * 2];       /* c e^{-i a_j}: (cos a, -sin a) */
                im -= c * ph[((size_t)s * n + j) * 2 + 1];
            }
            T[((size_t)i * S + s) * 2] = re;
            T[((size_t)i * S + s) * 2 + 1] = im;
        }
    }
    for (int s1 = 0; s1 < S; ++s1)
        for (int s2 = 0; s2 < S; ++s2) {
            double re = 0.0, im = 0.0;
            for (int i = 0; i < n; ++i) {
                const double c = ph[((size_t)s1 * n + i) * 2], sn = ph[((size_t)s1 * n + i) * 2 + 1];
                const double tr = T[((size_t)i * S + s2) * 2], ti = T[((size_t)i * S + s2) * 2 + 1];
                re += c * tr - sn * ti;
                im += c * ti + sn * tr;
            }
            out[((size_t)s1 * S + s2) * 2] = norm * re;
            out[((size_t)s1 * S + s2) * 2 + 1] = norm * im;
        }
    free(ph);
    free(T);
    return ORC_OK;
}

static void measure_g4(orc_walker* w)
{
    const int S = w->nc * 2 * w->n_w4;
    double* Mu = (double*)malloc(sizeof(double) * 2 * (size_t)S * S);
    double* Md = (double*)malloc(sizeof(double) * 2 * (size_t)S * S);
    if (!Mu || !Md || g4_m2(w, 0, Mu) != ORC_OK || g4_m2(w, 1, Md) != ORC_OK) {
        free(Mu); free(Md);
        w->n_w4 = -w->n_w4;  /* out of memory: the measurement stops (reported by orc_get_g4) */
        return;
    }
    for (size_t e = 0; e < (size_t)S * S; ++e) {
        const double ar = Mu[2 * e], ai = Mu[2 * e + 1], br = Md[2 * e], bi = Md[2 * e + 1];
        w->G4acc[2 * e] += w->sign * (ar * br - ai * bi);
        w->G4acc[2 * e + 1] += w->sign * (ar * bi + ai * br);
    }
    for (int s = 0; s < S; ++s) {
        const size_t e = (size_t)s * S + s;
        w->G4d[2 * s] += w->sign * Mu[2 * e];
        w->G4d[2 * s + 1] += w->sign * Mu[2 * e + 1];
        w->G4d[2 * ((size_t)S + s)] += w->sign * Md[2 * e];
        w->G4d[2 * ((size_t)S + s) + 1] += w->sign * Md[2 * e + 1];
    }
    free(Mu);
    free(Md);
}

/* Switch the two-particle measurement on (n_w4 > 0) or off (0); clears it.
 * kdotr [nc][nc] = K_a . r_s, k_dn [nc] = index of Q - K_a, m4 the bosonic
 * transfer index. */
int orc_enable_g4(orc_walker* w, int32_t n_w4, int32_t m4, const double* kdotr, const int32_t* k_dn)
{
    if (!w || n_w4 < 0 || (n_w4 > 0 && (!kdotr || !k_dn))) return ORC_ERR_ARG;
    free(w->kdotr); free(w->k_dn); free(w->G4acc); free(w->G4d);
    w->kdotr = NULL; w->k_dn = NULL; w->G4acc = NULL; w->G4d = NULL;
    w->n_w4 = 0;
    if (n_w4 == 0) return ORC_OK;
    const int nc = w->nc;
    for (int k = 0; k < nc; ++k)
        if (k_dn[k] < 0 || k_dn[k] >= nc) return ORC_ERR_ARG;
    const size_t S = (size_t)nc * 2 * n_w4;
    w->kdotr = (double*)malloc(sizeof(double) * (size_t)nc * nc);
    w->k_dn = (int32_t*)malloc(sizeof(int32_t) * (size_t)nc);
    w->G4acc = (double*)calloc(S * S * 2, sizeof(double));
    w->G4d = (double*)calloc(2 * S * 2, sizeof(double));
    if (!w->kdotr || !w->k_dn || !w->G4acc || !w->G4d) return ORC_ERR_OOM;
    for (size_t e = 0; e < (size_t)nc * nc; ++e) w->kdotr[e] = kdotr[e];
    for (int k = 0; k < nc; ++k) w->k_dn[k] = k_dn[k];
    w->n_w4 = n_w4;
    w->m4 = m4;
    return ORC_OK;
}

/* Accumulators of the two-particle measurement: A [S][S][re, im], D [2][S][re, im]. */
int orc_get_g4(const orc_walker* w, double* A, double* D)
{
    if (!w || !A || !D || !w->G4acc) return ORC_ERR_ARG;
    if (w->n_w4 < 0) return ORC_ERR_OOM;
    const size_t S = (size_t)w->nc * 2 * w->n_w4;
    for (size_t e = 0; e < S * S * 2; ++e) A[e] = w->G4acc[e];
    for (size_t e = 0; e < 2 * S * 2; ++e) D[e] = w->G4d[e];
    return ORC_OK;
}

/* M_sigma(s1, s2) of the current configuration: out [S][S][re, im]. */
int orc_m2(const orc_walker* w, int32_t sp, double* out)
{
    if (!w || !out || w->n_w4 <= 0 || sp < 0 || sp > 1) return ORC_ERR_ARG;
    return g4_m2(w, sp, out);
}

/* Accumulated sum of sign * M(dr, i w_n): out [2][nc][n_omega][re, im]. */
int orc_get_M(const orc_walker* w, double* out)
{
    if (!w || !out || !w->Macc) return ORC_ERR_ARG;
    memcpy(out, w->Macc, sizeof(double) * (size_t)2 * w->nc * w->n_omega * 2);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Sweeps                                                              */
/* ------------------------------------------------------------------ */
int orc_sweep(orc_walker* w, int32_t n_sweeps)
{
    if (!w || n_sweeps < 0) return ORC_ERR_ARG;
    for (int s = 0; s < n_sweeps; ++s) {
        int64_t len;
        if (w->sweeps_done < w->warmup) {
            len = w->k > 1 ? w->k : 1;
            w->warm_k_sum += w->k;
        } else {
            if (w->sweep_len == 0) {
                int64_t L = w->warmup > 0 ? (2 * w->warm_k_sum + w->warmup) / (2 * (int64_t)w->warmup) : w->k;
                w->sweep_len = L > 1 ? L : 1;
            }
            len = w->sweep_len;
        }
        for (int64_t t = 0; t < len; ++t) {
            /* windows of neglect_ks proposals, never across a sweep boundary */
            if (w->neglect_ks > 0 && (t % w->neglect_ks) == 0) w->win_id++;
            int rc = propose(w, w->q);
            if (rc != ORC_OK) return rc;
            w->q++;
        }
        if (w->sweeps_done >= w->warmup) {
            measure(w);
            w->k_sum += w->sign * (double)w->k;
            w->k_samples++;
        }
        w->sweeps_done++;
    }
    return ORC_OK;
}

int64_t orc_sweep_length(const orc_walker* w) { return w->sweep_len; }

/* ------------------------------------------------------------------ */
/* Accessors                                                           */
/* ------------------------------------------------------------------ */
int32_t orc_order(const orc_walker* w) { return w->k; }
double orc_sign(const orc_walker* w) { return w->sign; }
double orc_gamma(const orc_walker* w) { return w->gamma; }

/* Copies the vertex list and both N matrices (k x k, row-major, ld = k). */
int orc_get_state(const orc_walker* w, int32_t* site, double* tau, int8_t* s, double* N_up, double* N_dn)
{
    int n = w->k;
    for (int i = 0; i < n; ++i) {
        if (site) site[i] = w->vsite[i];
        if (tau) tau[i] = w->vtau[i];
        if (s) s[i] = w->vs[i];
    }
    double* out[2] = {N_up, N_dn};
    for (int sp = 0; sp < 2; ++sp) {
        if (!out[sp]) continue;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) out[sp][(size_t)i * n + j] = w->N[sp][(size_t)i * w->cap + j];
    }
    return ORC_OK;
}

/* counters: [proposals, accepts, near_ties, adopted, next_q, sweeps_done, n_meas, k_samples] */
void orc_counters(const orc_walker* w, int64_t* out)
{
    out[0] = w->n_prop; out[1] = w->n_acc; out[2] = w->n_ties; out[3] = w->n_adopted;
    out[4] = (int64_t)w->q; out[5] = w->sweeps_done; out[6] = w->n_meas; out[7] = w->k_samples;
}

double orc_k_sum(const orc_walker* w) { return w->k_sum; }

int orc_get_G(const orc_walker* w, double* G_out, double* sign_sum, int64_t* n_meas)
{
    size_t m = (size_t)2 * w->nc * w->n_meas_tau;
    if (G_out) memcpy(G_out, w->Gacc, sizeof(double) * m);
    if (sign_sum) *sign_sum = w->sign_sum;
    if (n_meas) *n_meas = w->n_meas;
    return ORC_OK;
}

void orc_reset_accumulators(orc_walker* w)
{
    memset(w->Gacc, 0, sizeof(double) * (size_t)2 * w->nc * w->n_meas_tau);
    w->sign_sum = 0.0;
    w->n_meas = 0;
    w->k_sum = 0.0;
    w->k_samples = 0;
    if (w->Macc) memset(w->Macc, 0, sizeof(double) * (size_t)2 * w->nc * w->n_omega * 2);
    if (w->G4acc) {
        const size_t S = (size_t)w->nc * 2 * w->n_w4;
        memset(w->G4acc, 0, sizeof(double) * S * S * 2);
        memset(w->G4d, 0, sizeof(double) * 2 * S * 2);
    }
}

/* Decision log: one byte per proposal, bit 0 = accepted, bit 1 = near tie. */
int orc_enable_log(orc_walker* w, int64_t cap)
{
    free(w->log);
    w->log = (uint8_t*)malloc((size_t)(cap > 0 ? cap : 1));
    if (!w->log) return ORC_ERR_OOM;
    w->log_cap = cap;
    w->log_n = 0;
    return ORC_OK;
}

int64_t orc_get_log(const orc_walker* w, uint8_t* out, int64_t cap)
{
    int64_t n = w->log_n < w->log_cap ? w->log_n : w->log_cap;
    if (out) memcpy(out, w->log, (size_t)(n < cap ? n : cap));
    return w->log_n;
}

/* At a near tie, adopt hints[q] & 1 instead of the oracle's own decision.
 * The pointer is borrowed; it must outlive the sweeps that use it. */
void orc_set_hints(orc_walker* w, const uint8_t* hints, int64_t n)
{
    w->hints = hints;
    w->hints_n = n;
}

/* Fresh N_sigma = [e^V - g0 (e^V - 1)]^-1 for the walker's current vertex
 * list; out is k x k (ld = k).  Returns the sign of det N_sigma^-1. */
int orc_fresh_N(const orc_walker* w, int32_t sp, double* out)
{
    int n = w->k;
    if (n == 0) return 1;
    double* A = (double*)malloc(sizeof(double) * (size_t)n * n);
    build_A(w, sp, n, w->vsite, w->vtau, w->vs, A);
    int sg = gj_inverse(n, A, out, n);
    free(A);
    return sg;
}

/* A_sigma = e^V - g0 (e^V - 1) for an arbitrary vertex list, with this
 * walker's tables (for brute-force determinant checks). */
int orc_build_A(const orc_walker* w, int32_t sp, int32_t n, const int32_t* site, const double* tau,
                const int8_t* s, double* A)
{
    if (n < 0) return ORC_ERR_ARG;
    build_A(w, sp, n, site, tau, s, A);
    return ORC_OK;
}

/* Replace the walker's configuration (all vertices interacting) and rebuild
 * N; used by tests that start from a chosen configuration. */
int orc_set_config(orc_walker* w, int32_t n, const int32_t* site, const double* tau, const int8_t* s)
{
    if (n < 0) return ORC_ERR_ARG;
    int rc = ensure_cap(w, n > 0 ? n : 1);
    if (rc != ORC_OK) return rc;
    for (int i = 0; i < n; ++i) {
        if (site[i] < 0 || site[i] >= w->nc || (s[i] != 1 && s[i] != -1)) return ORC_ERR_ARG;
        w->vsite[i] = site[i]; w->vtau[i] = tau[i]; w->vs[i] = s[i];
        w->changed[i] = -1;
    }
    w->k = n;
    return rebuild_N(w, &w->sign);
}

/* Apply one proposal of a given kind to the current state, forcing
 * acceptance (force = 1) or rejection (force = 0).  Used by the determinant
 * pins; does not advance the proposal counter or the decision log. */
int orc_try_insert(orc_walker* w, int32_t site, double tau, int8_t s, int32_t force)
{
    /* u = -1 accepts every finite |R|; u = 1e300 rejects every one. */
    double u = force ? -1.0 : 1.0e300;
    int64_t saved[3] = {w->n_ties, w->n_prop, w->log_n};
    int rc = propose_insert(w, site, tau, s, u, UINT64_MAX);
    w->n_ties = saved[0]; w->n_prop = saved[1]; w->log_n = saved[2];
    return rc;
}

int orc_try_remove(orc_walker* w, int32_t p, int32_t force)
{
    if (p < 0 || p >= w->k) return ORC_ERR_ARG;
    double u = force ? -1.0 : 1.0e300;
    int64_t saved[3] = {w->n_ties, w->n_prop, w->log_n};
    int rc = propose_remove(w, p, u, UINT64_MAX);
    w->n_ties = saved[0]; w->n_prop = saved[1]; w->log_n = saved[2];
    return rc;
}

/* Flip the auxiliary spin of vertex p, forced accepted (force = 1) or
 * rejected (0); rho_out (may be NULL) receives the ratio per spin. */
int orc_try_flip(orc_walker* w, int32_t p, int32_t force, double* rho_out)
{
    if (p < 0 || p >= w->k) return ORC_ERR_ARG;
    double u = force ? -1.0 : 1.0e300;
    int64_t saved[3] = {w->n_ties, w->n_prop, w->log_n};
    int rc = propose_flip(w, p, u, UINT64_MAX, rho_out);
    w->n_ties = saved[0]; w->n_prop = saved[1]; w->log_n = saved[2];
    return rc;
}

int64_t orc_neglected(const orc_walker* w) { return w->n_neglected; }

/* Determinant ratio rho_sigma (both spins) of a proposed insert or remove
 * on the current state, without changing it. */
int orc_ratio(orc_walker* w, int32_t is_remove, int32_t p, int32_t site, double tau, int8_t s, double* rho_out)
{
    int n = w->k;
    int rc = ensure_cap(w, n + 1);
    if (rc != ORC_OK) return rc;
    int ld = w->cap;
    for (int sp = 0; sp < 2; ++sp) {
        double* N = w->N[sp];
        double acc = 0.0;
        if (!is_remove) {
            double* urow = w->work;
            double* X = w->work + ld;
            for (int i = 0; i < n; ++i)
                urow[i] = g0ab(w, sp, site, tau, w->vsite[i], w->vtau[i]) * (ev(w, sp, w->vs[i]) - 1.0);
            for (int j = 0; j < n; ++j) {
                double t = 0.0;
                for (int i = 0; i < n; ++i) t += urow[i] * N[(size_t)i * ld + j];
                X[j] = t;
            }
            double delta = ev(w, sp, s) - 1.0;
            for (int j = 0; j < n; ++j) acc += X[j] * (-g0ab(w, sp, w->vsite[j], w->vtau[j], site, tau) * delta);
            acc += (1.0 - g0ab(w, sp, site, 0.0, site, 0.0)) * delta;
        } else {
            if (p < 0 || p >= n) return ORC_ERR_ARG;
            acc = N[(size_t)p * ld + p] - 1.0;
        }
        rho_out[sp] = 1.0 + acc;
    }
    return ORC_OK;
}
