/*
 * qsg_oracle.c -- plain, slow CPU oracle of the Monte Carlo hot path of
 * "The Quantum Transition of the Two-Dimensional Ising Spin Glass: A Tale of
 * Two Gaps" (arXiv 2310.07486).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The CUDA product
 * path never links or calls it, and the two share no code: this file has its
 * own Philox, its own threshold tables, its own lattice indexing.
 *
 * Representation: one int8 per spin (+1 / -1), one int8 per coupling, every
 * configuration stored separately, every site visited one at a time.
 *
 * What is computed (section / equation of the paper in brackets):
 *   - couplings J = +-1 with probability 1/2, nearest neighbours on the
 *     periodic L x L lattice                       [Methods, Model and simulations]
 *   - the classical Trotter-Suzuki action
 *       E(S) = - sum_tau [ sum_<xy> J_xy S_x,tau S_y,tau + sum_x S_x,tau S_x,tau+1 ]
 *     with weight exp(-k E(S)); space coupling k J, time coupling k
 *                                                  [Eq. (Trotter-action), Eq. (P-S-tau)]
 *     Under APBC the time bond between tau = L_tau-1 and tau = 0 has sign -1.
 *   - checkerboard Metropolis and heat-bath sweeps [Methods, Simulation details]
 *   - parallel tempering over the k ladder        [Methods, Simulation details]
 *   - the imaginary-time correlators C(tau) and Q2(tau) and the equal-time
 *     replica overlap q2 (the Tr M^2 / L^2D comparator)
 *                                                  [Eq. (C_A_transfer), Eq. (def-C-Q2-tau)]
 *
 * Readings of the paper that this oracle fixes (the paper is silent or its
 * formula is garbled at these points):
 *   R1  bonds are (x, x+e1) and (x, x+e2): 2 L^2 couplings per sample; the
 *       sum over tau runs 0 .. L_tau-1 with a periodic (or antiperiodic) wrap.
 *   R2  the estimator normalisation is (1/L_tau) sum_tau1, C / L^D, Q2 / L^2D,
 *       so C(0) = Q2(0) = 1.
 *   R3  Q2(tau) uses (sum_x S_x,tau1 S_x,tau1+tau)^2 of one configuration.
 *   R5  colour (x+y+tau) mod 2; a sweep = colour 0 then colour 1.
 *   R6  Philox4x32-10 keyed (seed_lo, seed_hi); counters given below.  The
 *       sweep cuts rows into column pairs starting at x = y & 1 and time into
 *       pairs (2m, 2m+1); one call per 2 x 2 block feeds its four sites.
 *   R7  the sweep draws ONE 32-bit uniform per site and sweep, shared by the
 *       64 disorder samples that occupy one multispin word of the GPU store
 *       (samples 64w .. 64w+63).  Different replicas and ladder positions
 *       draw different uniforms.
 *   R8  Metropolis: flip iff S h <= 0 or u < floor(2^32 exp(-2 k S h)).
 *   R9  heat bath: S = +1 iff u < min(floor(2^32 / (1 + exp(-2 k h))), 2^32-1).
 *   R10 PT: pairs i = 0 .. K-2 in order; accept iff E_{i+1} >= E_i or
 *       u < (A_i[n>>6] * B_i[n&63]) >> 32 with n = E_i - E_{i+1},
 *       A_i[m] = floor(2^32 exp(-d_i 64 m)), B_i[r] = floor(2^32 exp(-d_i r)),
 *       d_i = k_{i+1} - k_i.  An accepted swap exchanges the two
 *       configurations of that sample and replica.
 *   R11 hot start from Philox stream INIT.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_STREAM_J 1u
#define ORC_STREAM_INIT 2u
#define ORC_STREAM_SWEEP 3u
#define ORC_STREAM_PT 4u
#define ORC_MAX_TRIPLE_R 8

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two      */
/* 32x32->64 multiplications, a Feistel-like permutation of the four words,  */
/* the key added through XOR and bumped by the Weyl constants between rounds. */
/* ------------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod_a = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t prod_b = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi_a = (uint32_t)(prod_a >> 32), lo_a = (uint32_t)prod_a;
        uint32_t hi_b = (uint32_t)(prod_b >> 32), lo_b = (uint32_t)prod_b;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox(ctr, key, out);
}

/* ------------------------------------------------------------------------ */
/* Group state                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int L, Ltau, n_samples, R, K, algo, boundary, group_id;
    int first;      /* global index of local sample 0 (word (first+b)/64, bit (first+b)%64) */
    int N;          /* L*L*Ltau sites */
    int n_lag;      /* Ltau/2 + 1 */
    uint64_t seed;
    double *k;      /* [n_samples][K] ladder of each sample */
    int8_t *J;      /* [n_samples][2][L*L]: [0] bond (x,y)-(x+1,y), [1] bond (x,y)-(x,y+1) */
    int8_t *S;      /* [n_samples][R][K][N]; configuration at ladder position j */
    uint32_t *Tmet; /* [n_samples][K][3]: S h = 2, 4, 6 */
    uint32_t *Thb;  /* [n_samples][K][7]: h = 6 - 2 n, n = 0..6 */
    uint64_t *ptB;  /* [n_samples][K-1][64] */
    uint64_t **ptA; /* [n_samples*(K-1)] -> A table */
    int *ptA_len;   /* [n_samples*(K-1)] */
    int64_t *E;     /* [n_samples][R][K] action of the configuration at j */
    int64_t *Cacc;  /* [R][n_samples][K][n_lag] */
    int64_t *Qacc;  /* [R][n_samples][K][n_lag] */
    int64_t *Pacc;  /* [n_samples][K] */
    unsigned __int128 *P4acc;  /* [n_samples][K] sum of Q0^4 */
    int64_t *T3acc; /* [n_samples][K] sum over replica triples of Q_ab Q_bc Q_ca */
    int64_t *Gacc;  /* [n_samples][K][L/2+1] pair products of momentum sums, by x-distance */
    int64_t *F3acc; /* [n_samples][K][L/2+1] triple products of momentum sums, by x-distance */
    int64_t *PPacc; /* [n_samples][K][R(R-1)/2] sum of Q_ab^2 of each replica pair a < b */
    int64_t *acc;   /* [n_samples][K-1] accepted swaps, summed over replicas */
    int64_t n_meas;
    uint32_t sweep;
    uint32_t n_swaps;
} orc_group;

static int site(const orc_group *g, int x, int y, int t)
{
    return (t * g->L + y) * g->L + x;
}

static int8_t *config(orc_group *g, int b, int r, int j)
{
    return g->S + ((size_t)((size_t)b * g->R + r) * g->K + j) * (size_t)g->N;
}

/* global sample index of local sample b */
static int gsample(const orc_group *g, int b) { return g->first + b; }

/* slot index of (sample b, replica r, ladder position j): the multispin word
 * w = b / 64 holds 64 samples; each (w, r, j) owns one random stream. */
static uint32_t slot_of(const orc_group *g, int b, int r, int j)
{
    return (uint32_t)((((gsample(g, b) / 64) * g->R) + r) * g->K + j);
}

/* n_samples samples with global indices first .. first+n_samples-1 */
orc_group *orc_create(int L, int Ltau, int n_samples, int R, int K, int algo, int boundary, int group_id, int first)
{
    if (L < 2 || (L & 1) || Ltau < 2 || (Ltau & 1) || n_samples < 1 || R < 1 || K < 1 || first < 0)
        return NULL;
    orc_group *g = (orc_group *)calloc(1, sizeof(orc_group));
    g->L = L; g->Ltau = Ltau; g->n_samples = n_samples; g->R = R; g->K = K;
    g->algo = algo; g->boundary = boundary; g->group_id = group_id; g->first = first;
    g->N = L * L * Ltau;
    g->n_lag = Ltau / 2 + 1;
    size_t ns = (size_t)n_samples;
    g->k = (double *)calloc(ns * K, sizeof(double));
    g->J = (int8_t *)calloc(ns * 2 * L * L, 1);
    g->S = (int8_t *)calloc(ns * R * K * (size_t)g->N, 1);
    g->Tmet = (uint32_t *)calloc(ns * K * 3, sizeof(uint32_t));
    g->Thb = (uint32_t *)calloc(ns * K * 7, sizeof(uint32_t));
    int np = K > 1 ? K - 1 : 1;
    g->ptB = (uint64_t *)calloc(ns * np * 64, sizeof(uint64_t));
    g->ptA = (uint64_t **)calloc(ns * np, sizeof(uint64_t *));
    g->ptA_len = (int *)calloc(ns * np, sizeof(int));
    g->E = (int64_t *)calloc(ns * R * K, sizeof(int64_t));
    g->Cacc = (int64_t *)calloc((size_t)R * ns * K * g->n_lag, sizeof(int64_t));
    g->Qacc = (int64_t *)calloc((size_t)R * ns * K * g->n_lag, sizeof(int64_t));
    g->Pacc = (int64_t *)calloc(ns * K, sizeof(int64_t));
    g->P4acc = (unsigned __int128 *)calloc(ns * K, sizeof(unsigned __int128));
    g->T3acc = (int64_t *)calloc(ns * K, sizeof(int64_t));
    g->Gacc = (int64_t *)calloc(ns * K * (size_t)(L / 2 + 1), sizeof(int64_t));
    g->F3acc = (int64_t *)calloc(ns * K * (size_t)(L / 2 + 1), sizeof(int64_t));
    g->PPacc = (int64_t *)calloc(ns * K * (size_t)(R * (R - 1) / 2 + 1), sizeof(int64_t));
    g->acc = (int64_t *)calloc(ns * np, sizeof(int64_t));
    if (!g->k || !g->J || !g->S || !g->Tmet || !g->Thb || !g->ptB || !g->ptA || !g->ptA_len ||
        !g->E || !g->Cacc || !g->Qacc || !g->Pacc || !g->P4acc || !g->T3acc || !g->Gacc || !g->F3acc || !g->PPacc || !g->acc)
        return NULL;
    return g;
}

void orc_destroy(orc_group *g)
{
    if (!g) return;
    int np = g->K > 1 ? g->K - 1 : 1;
    for (int i = 0; i < g->n_samples * np; ++i) free(g->ptA[i]);
    free(g->k); free(g->J); free(g->S); free(g->Tmet); free(g->Thb); free(g->ptB);
    free(g->ptA); free(g->ptA_len); free(g->E); free(g->Cacc); free(g->Qacc);
    free(g->Pacc); free(g->P4acc); free(g->T3acc); free(g->Gacc); free(g->F3acc); free(g->PPacc); free(g->acc); free(g);
}

/* ------------------------------------------------------------------------ */
/* Acceptance tables (readings R8, R9, R10)                                  */
/* ------------------------------------------------------------------------ */
static uint32_t metropolis_threshold(double k, int Sh)
{
    double p = exp(-(2.0 * k * (double)Sh));
    return (uint32_t)floor(p * 4294967296.0);
}

static uint32_t heatbath_threshold(double k, int h)
{
    double p = 1.0 / (1.0 + exp(-(2.0 * k * (double)h)));
    double t = floor(p * 4294967296.0);
    if (t > 4294967295.0) t = 4294967295.0;
    return (uint32_t)t;
}

static uint64_t pt_entry(double delta, int64_t n)
{
    return (uint64_t)floor(exp(-(delta * (double)n)) * 4294967296.0);
}

static int build_tables(orc_group *g)
{
    int np = g->K > 1 ? g->K - 1 : 1;
    int64_t n_max = 6 * (int64_t)g->N; /* largest |E_i - E_i+1| */
    for (int b = 0; b < g->n_samples; ++b) {
        for (int j = 0; j < g->K; ++j) {
            double k = g->k[(size_t)b * g->K + j];
            for (int c = 0; c < 3; ++c)
                g->Tmet[((size_t)b * g->K + j) * 3 + c] = metropolis_threshold(k, 2 * (c + 1));
            for (int n = 0; n < 7; ++n)
                g->Thb[((size_t)b * g->K + j) * 7 + n] = heatbath_threshold(k, 6 - 2 * n);
        }
        for (int i = 0; i + 1 < g->K; ++i) {
            double delta = g->k[(size_t)b * g->K + i + 1] - g->k[(size_t)b * g->K + i];
            size_t p = (size_t)b * np + i;
            for (int r = 0; r < 64; ++r) g->ptB[p * 64 + r] = pt_entry(delta, r);
            int64_t len = 0;
            while (len <= (n_max >> 6)) {
                if (pt_entry(delta, 64 * len) == 0) break;
                ++len;
            }
            free(g->ptA[p]);
            g->ptA[p] = (uint64_t *)calloc((size_t)(len > 0 ? len : 1), sizeof(uint64_t));
            if (!g->ptA[p]) return -1;
            for (int64_t m = 0; m < len; ++m) g->ptA[p][m] = pt_entry(delta, 64 * m);
            g->ptA_len[p] = (int)len;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Initialisation: couplings (stream J) and hot start (stream INIT)          */
/* ------------------------------------------------------------------------ */
/* ladders: per_sample ? [n_samples][K] : [K]; J_in (optional): [n_samples][2][L*L] of +-1 */
int orc_init(orc_group *g, uint64_t seed, const double *ladders, int per_sample, const int8_t *J_in)
{
    g->seed = seed;
    g->sweep = 0; g->n_swaps = 0; g->n_meas = 0;
    int L = g->L, K = g->K;
    for (int b = 0; b < g->n_samples; ++b)
        for (int j = 0; j < K; ++j) {
            double k = per_sample ? ladders[(size_t)b * K + j] : ladders[j];
            if (!(k > 0.0) || !(k < 3.0)) return -1;
            if (j > 0 && !(k > g->k[(size_t)b * K + j - 1])) return -1;
            g->k[(size_t)b * K + j] = k;
        }
    if (build_tables(g)) return -1;

    uint32_t tag = (uint32_t)g->group_id << 8;
    for (int b = 0; b < g->n_samples; ++b) {
        for (int d = 0; d < 2; ++d)
            for (int n = 0; n < L * L; ++n) {
                int8_t v;
                if (J_in) {
                    v = J_in[((size_t)b * 2 + d) * L * L + n];
                } else {
                    uint32_t o[4];
                    int gb = gsample(g, b);
                    draw(seed, (uint32_t)n, (uint32_t)d, (uint32_t)(gb / 64), (ORC_STREAM_J << 24) | tag, o);
                    uint64_t bits = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
                    v = ((bits >> (gb % 64)) & 1u) ? -1 : 1;
                }
                g->J[((size_t)b * 2 + d) * L * L + n] = v;
            }
    }
    for (int b = 0; b < g->n_samples; ++b)
        for (int r = 0; r < g->R; ++r)
            for (int j = 0; j < K; ++j) {
                int8_t *S = config(g, b, r, j);
                uint32_t s = slot_of(g, b, r, j);
                for (int n = 0; n < g->N; ++n) {
                    uint32_t o[4];
                    draw(seed, (uint32_t)n, 0u, s, (ORC_STREAM_INIT << 24) | tag, o);
                    uint64_t bits = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
                    S[n] = ((bits >> (gsample(g, b) % 64)) & 1u) ? -1 : 1;
                }
            }
    memset(g->Cacc, 0, sizeof(int64_t) * (size_t)g->R * g->n_samples * K * g->n_lag);
    memset(g->Qacc, 0, sizeof(int64_t) * (size_t)g->R * g->n_samples * K * g->n_lag);
    memset(g->Pacc, 0, sizeof(int64_t) * (size_t)g->n_samples * K);
    memset(g->P4acc, 0, sizeof(unsigned __int128) * (size_t)g->n_samples * K);
    memset(g->T3acc, 0, sizeof(int64_t) * (size_t)g->n_samples * K);
    memset(g->Gacc, 0, sizeof(int64_t) * (size_t)g->n_samples * K * (g->L / 2 + 1));
    memset(g->F3acc, 0, sizeof(int64_t) * (size_t)g->n_samples * K * (g->L / 2 + 1));
    memset(g->PPacc, 0, sizeof(int64_t) * (size_t)g->n_samples * K * (g->R * (g->R - 1) / 2 + 1));
    memset(g->acc, 0, sizeof(int64_t) * (size_t)g->n_samples * (K > 1 ? K - 1 : 1));
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Local field and one site update                                           */
/* ------------------------------------------------------------------------ */
/* time-bond sign between tau and tau+1 (APBC flips the wrap bond) */
static int time_sign(const orc_group *g, int t)
{
    return (g->boundary == 1 && t == g->Ltau - 1) ? -1 : 1;
}

/* h = sum_space J S_nb + sum_time (sign) S_nb : the field that multiplies
 * S_x,tau in -E, so that the weight of S is exp(k S h). */
static int local_field(const orc_group *g, const int8_t *S, const int8_t *J, int x, int y, int t)
{
    int L = g->L, Lt = g->Ltau;
    int xp = (x + 1) % L, xm = (x + L - 1) % L;
    int yp = (y + 1) % L, ym = (y + L - 1) % L;
    int tp = (t + 1) % Lt, tm = (t + Lt - 1) % Lt;
    const int8_t *Jx = J, *Jy = J + L * L;
    int h = 0;
    h += Jx[y * L + x] * S[site(g, xp, y, t)];
    h += Jx[y * L + xm] * S[site(g, xm, y, t)];
    h += Jy[y * L + x] * S[site(g, x, yp, t)];
    h += Jy[ym * L + x] * S[site(g, x, ym, t)];
    h += time_sign(g, t) * S[site(g, x, y, tp)];
    h += time_sign(g, tm) * S[site(g, x, y, tm)];
    return h;
}

/* uniform of site (x,y,t) in sweep `sw` for slot s: every row is cut into
 * pairs of neighbouring columns, (0,1),(2,3),... in even rows and
 * (1,2),(3,4),...,(L-1,0) in odd rows, and time into pairs (2m, 2m+1); each
 * resulting block of 2 x 2 sites draws one Philox call per sweep and slot, and
 * the site at column offset dx within its pair and time offset t&1 takes word
 * (t&1)*2 + dx. */
static uint32_t sweep_uniform(const orc_group *g, uint32_t s, uint32_t sw, int x, int y, int t)
{
    int shifted = (x - (y & 1) + g->L) % g->L; /* column counted from the pair start */
    uint32_t block = (uint32_t)(((t / 2) * g->L + y) * (g->L / 2) + shifted / 2);
    uint32_t o[4];
    draw(g->seed, block, sw, s, (ORC_STREAM_SWEEP << 24) | ((uint32_t)g->group_id << 8), o);
    return o[(t & 1) * 2 + (shifted & 1)];
}

static void half_sweep(orc_group *g, int b, int r, int j, int colour)
{
    int L = g->L;
    int8_t *S = config(g, b, r, j);
    const int8_t *J = g->J + (size_t)b * 2 * L * L;
    const uint32_t *Tm = g->Tmet + ((size_t)b * g->K + j) * 3;
    const uint32_t *Th = g->Thb + ((size_t)b * g->K + j) * 7;
    uint32_t s = slot_of(g, b, r, j);
    for (int t = 0; t < g->Ltau; ++t)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                if (((x + y + t) & 1) != colour) continue;
                int n = site(g, x, y, t);
                int h = local_field(g, S, J, x, y, t);
                uint32_t u = sweep_uniform(g, s, g->sweep, x, y, t);
                if (g->algo == 0) {
                    int Sh = S[n] * h;
                    if (Sh <= 0 || u < Tm[Sh / 2 - 1]) S[n] = (int8_t)(-S[n]);
                } else {
                    S[n] = (u < Th[(6 - h) / 2]) ? 1 : -1;
                }
            }
}

void orc_sweep(orc_group *g, int n_sweeps)
{
    int total = g->n_samples * g->R * g->K;
    for (int it = 0; it < n_sweeps; ++it) {
#pragma omp parallel for schedule(dynamic)
        for (int c = 0; c < total; ++c) {
            int b = c / (g->R * g->K), r = (c / g->K) % g->R, j = c % g->K;
            half_sweep(g, b, r, j, 0);
            half_sweep(g, b, r, j, 1);
        }
        g->sweep++;
    }
}

/* ------------------------------------------------------------------------ */
/* Action of a configuration, Eq. (Trotter-action)                           */
/* ------------------------------------------------------------------------ */
static int64_t action(const orc_group *g, const int8_t *S, const int8_t *J)
{
    int L = g->L;
    const int8_t *Jx = J, *Jy = J + L * L;
    int64_t e = 0;
    for (int t = 0; t < g->Ltau; ++t)
        for (int y = 0; y < L; ++y)
            for (int x = 0; x < L; ++x) {
                int s0 = S[site(g, x, y, t)];
                e -= (int64_t)Jx[y * L + x] * s0 * S[site(g, (x + 1) % L, y, t)];
                e -= (int64_t)Jy[y * L + x] * s0 * S[site(g, x, (y + 1) % L, t)];
                e -= (int64_t)time_sign(g, t) * s0 * S[site(g, x, y, (t + 1) % g->Ltau)];
            }
    return e;
}

/* E_out: [n_samples][R][K] */
void orc_energy(orc_group *g, int64_t *E_out)
{
    int total = g->n_samples * g->R * g->K;
#pragma omp parallel for schedule(dynamic)
    for (int c = 0; c < total; ++c) {
        int b = c / (g->R * g->K), r = (c / g->K) % g->R, j = c % g->K;
        g->E[c] = action(g, config(g, b, r, j), g->J + (size_t)b * 2 * g->L * g->L);
    }
    if (E_out) memcpy(E_out, g->E, sizeof(int64_t) * (size_t)total);
}

/* ------------------------------------------------------------------------ */
/* Parallel tempering over the k ladder (reading R10)                        */
/* ------------------------------------------------------------------------ */
void orc_swap(orc_group *g)
{
    orc_energy(g, NULL);
    int K = g->K, np = K > 1 ? K - 1 : 1;
    uint32_t m = g->n_swaps;
    uint32_t tag = (ORC_STREAM_PT << 24) | ((uint32_t)g->group_id << 8);
    for (int b = 0; b < g->n_samples; ++b)
        for (int r = 0; r < g->R; ++r) {
            int64_t *E = g->E + ((size_t)b * g->R + r) * K;
            for (int i = 0; i + 1 < K; ++i) {
                uint32_t o[4];
                int gb = gsample(g, b);
                draw(g->seed, (uint32_t)(i * 16 + (gb % 64) / 4), m, (uint32_t)((gb / 64) * g->R + r), tag, o);
                uint32_t u = o[(gb % 64) & 3];
                int accept;
                if (E[i + 1] >= E[i]) {
                    accept = 1;
                } else {
                    int64_t n = E[i] - E[i + 1];
                    size_t p = (size_t)b * np + i;
                    if ((n >> 6) >= g->ptA_len[p]) {
                        accept = 0;
                    } else {
                        uint64_t thr = (g->ptA[p][n >> 6] * g->ptB[p * 64 + (n & 63)]) >> 32;
                        accept = (uint64_t)u < thr;
                    }
                }
                if (accept) {
                    int8_t *A = config(g, b, r, i), *B = config(g, b, r, i + 1);
                    for (int n = 0; n < g->N; ++n) { int8_t t = A[n]; A[n] = B[n]; B[n] = t; }
                    int64_t te = E[i]; E[i] = E[i + 1]; E[i + 1] = te;
                    g->acc[(size_t)b * np + i]++;
                }
            }
        }
    g->n_swaps++;
}

/* ------------------------------------------------------------------------ */
/* Imaginary-time correlators, Eqs. (C_A_transfer), (def-C-Q2-tau)           */
/* ------------------------------------------------------------------------ */
void orc_measure(orc_group *g)
{
    int L2 = g->L * g->L, Lt = g->Ltau, K = g->K, R = g->R, nl = g->n_lag;
    int total = g->n_samples * R * K;
#pragma omp parallel for schedule(dynamic)
    for (int c = 0; c < total; ++c) {
        int b = c / (R * K), r = (c / K) % R, j = c % K;
        const int8_t *S = config(g, b, r, j);
        size_t o = (((size_t)r * g->n_samples + b) * K + j) * nl;
        for (int lag = 0; lag < nl; ++lag) {
            int64_t csum = 0, qsum = 0;
            for (int t1 = 0; t1 < Lt; ++t1) {
                int t2 = t1 + lag;
                int sgn = 1;
                if (t2 >= Lt) { t2 -= Lt; if (g->boundary == 1) sgn = -1; }
                int64_t cc = 0;
                for (int xy = 0; xy < L2; ++xy)
                    cc += S[t1 * L2 + xy] * S[t2 * L2 + xy];
                csum += sgn * cc;
                qsum += cc * cc;
            }
            g->Cacc[o + lag] += csum;
            g->Qacc[o + lag] += qsum;
        }
    }
    /* One-time observables, Methods "One-time observables", Eqs. (def-M),
     * (chi-r), (Binder).  M_xy = <S_x S_y> at equal imaginary time, estimated
     * with independent replicas a, b, c of the same sample and k, at every
     * slice tau (the slice is arbitrary, so all of them are averaged):
     *   Tr M^2          <- Q_ab^2,                  Q_ab = sum_x S^a_x S^b_x
     *   sum <SSSS>^2    <- Q_ab^4
     *   Tr M^3          <- Q_ab Q_bc Q_ca
     *   Tr Mhat M       <- sum_{x,y} S^a_x S^b_x S^a_y S^b_y cos(p (x-y))
     *   Tr Mhat M^2     <- sum_{x,y} S^s_x S^u_x S^s_y S^v_y cos(p (x-y)) * Q_uv
     * for p = (2 pi / L, 0) and (0, 2 pi / L).  Pairs (x, y) are grouped by
     * their distance d = (x1 - y1) mod L along p, so the cosine factors out:
     * the integer sums per d (folded d ~ L - d) are accumulated and the FP64
     * finish applies cos(2 pi d / L).  All three choices of the replica s
     * shared by the two momentum-carrying overlaps are summed. */
#pragma omp parallel for schedule(dynamic)
    for (int c = 0; c < g->n_samples * K; ++c) {
        int b = c / K, j = c % K, L = g->L, H = L / 2;
        int npair = R * (R - 1) / 2;
        if (npair == 0) continue;
        int64_t p2 = 0, t3 = 0;
        unsigned __int128 p4 = 0;
        int64_t *G = g->Gacc + (size_t)c * (H + 1), *F3 = g->F3acc + (size_t)c * (H + 1);
        int64_t *Q = (int64_t *)malloc(sizeof(int64_t) * npair);
        int64_t *nx = (int64_t *)malloc(sizeof(int64_t) * npair * L);  /* column sums over y */
        int64_t *ny = (int64_t *)malloc(sizeof(int64_t) * npair * L);  /* row sums over x */
        int *pid = (int *)malloc(sizeof(int) * R * R);
        for (int t = 0; t < Lt; ++t) {
            int pi = 0;
            for (int ra = 0; ra < R; ++ra)
                for (int rb = ra + 1; rb < R; ++rb, ++pi) {
                    pid[ra * R + rb] = pid[rb * R + ra] = pi;
                    const int8_t *A = config(g, b, ra, j) + (size_t)t * L2, *B = config(g, b, rb, j) + (size_t)t * L2;
                    int64_t q = 0;
                    for (int i = 0; i < L; ++i) { nx[pi * L + i] = 0; ny[pi * L + i] = 0; }
                    for (int y = 0; y < L; ++y)
                        for (int x = 0; x < L; ++x) {
                            int o = A[y * L + x] * B[y * L + x];
                            q += o;
                            nx[pi * L + x] += o;
                            ny[pi * L + y] += o;
                        }
                    Q[pi] = q;
                    p2 += q * q;
                    g->PPacc[(size_t)c * npair + pi] += q * q;
                    p4 += (unsigned __int128)(uint64_t)(q * q) * (uint64_t)(q * q);
                    for (int c1 = 0; c1 < L; ++c1)
                        for (int c2 = 0; c2 < L; ++c2) {
                            int d = ((c2 - c1) % L + L) % L;
                            if (d > H) d = L - d;
                            G[d] += nx[pi * L + c1] * nx[pi * L + c2] + ny[pi * L + c1] * ny[pi * L + c2];
                        }
                }
            /* three-replica terms for 3 <= R <= ORC_MAX_TRIPLE_R only (their
             * number grows as R^3; the paper simulates 6 replicas) */
            for (int ra = 0; ra < R && R <= ORC_MAX_TRIPLE_R; ++ra)
                for (int rb = ra + 1; rb < R; ++rb)
                    for (int rc = rb + 1; rc < R; ++rc) {
                        int ab = pid[ra * R + rb], bc = pid[rb * R + rc], ca = pid[rc * R + ra];
                        t3 += Q[ab] * Q[bc] * Q[ca];
                        int rep[3] = {ra, rb, rc};
                        for (int rot = 0; rot < 3; ++rot) {
                            int s_ = rep[rot], u = rep[(rot + 1) % 3], v = rep[(rot + 2) % 3];
                            int su = pid[s_ * R + u], sv = pid[s_ * R + v], uv = pid[u * R + v];
                            for (int c1 = 0; c1 < L; ++c1)
                                for (int c2 = 0; c2 < L; ++c2) {
                                    int d = ((c2 - c1) % L + L) % L;
                                    if (d > H) d = L - d;
                                    F3[d] += Q[uv] * (nx[su * L + c1] * nx[sv * L + c2] + ny[su * L + c1] * ny[sv * L + c2]);
                                }
                        }
                    }
        }
        g->Pacc[c] += p2;
        g->P4acc[c] += p4;
        g->T3acc[c] += t3;
        free(Q); free(nx); free(ny); free(pid);
    }
    g->n_meas++;
}

/* Correlator sums of ONE configuration (sample b, replica r, ladder j), not
 * accumulated: C_out[lag] = sum_tau1 s c, Q_out[lag] = sum_tau1 c^2. */
void orc_measure_one(orc_group *g, int b, int r, int j, int64_t *C_out, int64_t *Q_out)
{
    int L2 = g->L * g->L, Lt = g->Ltau;
    const int8_t *S = config(g, b, r, j);
    for (int lag = 0; lag < g->n_lag; ++lag) {
        int64_t csum = 0, qsum = 0;
        for (int t1 = 0; t1 < Lt; ++t1) {
            int t2 = t1 + lag, sgn = 1;
            if (t2 >= Lt) { t2 -= Lt; if (g->boundary == 1) sgn = -1; }
            int64_t cc = 0;
            for (int xy = 0; xy < L2; ++xy) cc += S[t1 * L2 + xy] * S[t2 * L2 + xy];
            csum += sgn * cc;
            qsum += cc * cc;
        }
        C_out[lag] = csum;
        Q_out[lag] = qsum;
    }
}

/* FP64 finish: C = Cacc / (n_meas L^2 L_tau); Q2 = Qacc / (n_meas L^4 L_tau);
 * q2 = Pacc / (n_meas n_pairs L^4 L_tau).  Any output may be NULL. */
void orc_read(const orc_group *g, double *C, double *Q, double *P, int64_t *Craw, int64_t *Qraw, int64_t *Praw)
{
    size_t nc = (size_t)g->R * g->n_samples * g->K * g->n_lag;
    size_t np = (size_t)g->n_samples * g->K;
    double L2 = (double)(g->L * g->L), Lt = (double)g->Ltau, nm = (double)g->n_meas;
    double pairs = (double)(g->R * (g->R - 1) / 2);
    for (size_t i = 0; i < nc; ++i) {
        if (C) C[i] = (double)g->Cacc[i] / (nm * L2 * Lt);
        if (Q) Q[i] = (double)g->Qacc[i] / (nm * L2 * L2 * Lt);
        if (Craw) Craw[i] = g->Cacc[i];
        if (Qraw) Qraw[i] = g->Qacc[i];
    }
    for (size_t i = 0; i < np; ++i) {
        if (P) P[i] = (double)g->Pacc[i] / (nm * pairs * L2 * L2 * Lt);
        if (Praw) Praw[i] = g->Pacc[i];
    }
}

/* One-time observables of every sample and k (FP64), Eqs. (chi-r), (xi-r),
 * (Binder), and the linear susceptibility of Sect. "On the magnetic
 * susceptibilities".  Per (sample b, k j), fields in this order:
 *   q2   = <Q^2> / L^2D          q4 = <Q^4> / L^4D
 *   chi2 = <Q^2> / L^D           F2 = <|Q(p)|^2> / L^D (both p averaged)
 *   chi3 = <Q_ab Q_bc Q_ca> / L^D
 *   F3   = <Re Q_su(p) Q_sv(-p) Q_uv> / L^D (3 choices of s, both p averaged)
 *          (chi3 and F3 need 3 <= R <= 8 replicas, NaN otherwise)
 *   chi_lin = C(0) + 2 sum_{tau=1}^{L_tau/2-1} C(tau) + C(L_tau/2), C averaged
 *             over replicas (the periodic sum of C over all L_tau slices)
 * with <.> the average over measurements, slices and replica pairs/triples.
 * Per k, the disorder averages (mean over the samples of the group):
 *   chi2, F2, xi2, chi3, F3, xi3, B, chi_lin
 * with xi = sqrt(chi / F - 1) / (2 sin(pi / L)) and B = mean q4 / (mean q2)^2.
 * raw (optional): [b][j] = P2, P4 low 64 bits, P4 high 64 bits, T3,
 * G[0..L/2], F3[0..L/2]. */
void orc_read_onetime(const orc_group *g, double *per_sample, double *per_k, int64_t *raw)
{
    int L = g->L, H = L / 2, K = g->K, R = g->R, ns = g->n_samples, nl = g->n_lag;
    double LD = (double)(L * L), Lt = (double)g->Ltau, nm = (double)g->n_meas;
    double npair = (double)(R * (R - 1) / 2), ntrip = (double)(R * (R - 1) * (R - 2) / 6);
    const double pi = 3.14159265358979323846;
    for (int b = 0; b < ns; ++b)
        for (int j = 0; j < K; ++j) {
            size_t c = (size_t)b * K + j;
            double G = 0.0, F3 = 0.0;
            for (int d = 0; d <= H; ++d) {
                double w = cos(2.0 * pi * d / L);
                G += w * (double)g->Gacc[c * (H + 1) + d];
                F3 += w * (double)g->F3acc[c * (H + 1) + d];
            }
            double *o = per_sample + c * 7;
            o[0] = (double)g->Pacc[c] / (nm * npair * LD * LD * Lt);
            o[1] = (double)g->P4acc[c] / (nm * npair * LD * LD * LD * LD * Lt);
            o[2] = (double)g->Pacc[c] / (nm * npair * Lt * LD);
            o[3] = G / (2.0 * nm * npair * Lt * LD);
            o[4] = (double)g->T3acc[c] / (nm * ntrip * Lt * LD);
            o[5] = F3 / (6.0 * nm * ntrip * Lt * LD);
            if (R < 3 || R > ORC_MAX_TRIPLE_R) o[4] = o[5] = NAN;
            double cl = 0.0;
            for (int r = 0; r < R; ++r) {
                const int64_t *Cr = g->Cacc + (((size_t)r * ns + b) * K + j) * nl;
                double s = 0.0;
                for (int lag = 0; lag < nl; ++lag) {
                    double v = (double)Cr[lag] / (nm * LD * Lt);
                    s += (lag == 0 || lag == nl - 1) ? v : 2.0 * v;
                }
                cl += s;
            }
            o[6] = cl / R;
            if (raw) {
                int64_t *w = raw + c * (4 + 2 * (H + 1));
                w[0] = g->Pacc[c];
                w[1] = (int64_t)(uint64_t)g->P4acc[c];
                w[2] = (int64_t)(uint64_t)(g->P4acc[c] >> 64);
                w[3] = g->T3acc[c];
                for (int d = 0; d <= H; ++d) {
                    w[4 + d] = g->Gacc[c * (H + 1) + d];
                    w[4 + H + 1 + d] = g->F3acc[c * (H + 1) + d];
                }
            }
        }
    if (!per_k) return;
    double s2 = 2.0 * sin(pi / L);
    for (int j = 0; j < K; ++j) {
        double m[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int b = 0; b < ns; ++b)
            for (int f = 0; f < 7; ++f) m[f] += per_sample[((size_t)b * K + j) * 7 + f];
        for (int f = 0; f < 7; ++f) m[f] /= ns;
        double *o = per_k + (size_t)j * 8;
        o[0] = m[2];
        o[1] = m[3];
        o[2] = sqrt(m[2] / m[3] - 1.0) / s2;
        o[3] = m[4];
        o[4] = m[5];
        o[5] = sqrt(m[4] / m[5] - 1.0) / s2;
        o[6] = m[1] / (m[0] * m[0]);
        o[7] = m[6];
    }
}

/* Sum over measurements and slices of Q_ab^2 for each replica pair a < b
 * (pairs in the order (0,1), (0,2), ..., (R-2,R-1)): out [n_samples][K][pairs]. */
void orc_read_pair_overlaps(const orc_group *g, int64_t *out)
{
    memcpy(out, g->PPacc, sizeof(int64_t) * (size_t)g->n_samples * g->K * (g->R * (g->R - 1) / 2));
}

/* ------------------------------------------------------------------------ */
/* Accessors used by the tests                                               */
/* ------------------------------------------------------------------------ */
void orc_get_spins(const orc_group *g, int8_t *out)
{
    memcpy(out, g->S, (size_t)g->n_samples * g->R * g->K * (size_t)g->N);
}

void orc_set_spins(orc_group *g, const int8_t *in)
{
    memcpy(g->S, in, (size_t)g->n_samples * g->R * g->K * (size_t)g->N);
}

void orc_get_couplings(const orc_group *g, int8_t *out)
{
    memcpy(out, g->J, (size_t)g->n_samples * 2 * g->L * g->L);
}

void orc_get_tables(const orc_group *g, uint32_t *Tmet, uint32_t *Thb)
{
    if (Tmet) memcpy(Tmet, g->Tmet, sizeof(uint32_t) * (size_t)g->n_samples * g->K * 3);
    if (Thb) memcpy(Thb, g->Thb, sizeof(uint32_t) * (size_t)g->n_samples * g->K * 7);
}

/* PT threshold for sample b, pair i and action gap n > 0 (0 = never) */
uint64_t orc_pt_threshold(const orc_group *g, int b, int i, int64_t n)
{
    int np = g->K > 1 ? g->K - 1 : 1;
    size_t p = (size_t)b * np + i;
    if ((n >> 6) >= g->ptA_len[p]) return 0;
    return (g->ptA[p][n >> 6] * g->ptB[p * 64 + (n & 63)]) >> 32;
}

void orc_get_accepts(const orc_group *g, int64_t *out)
{
    memcpy(out, g->acc, sizeof(int64_t) * (size_t)g->n_samples * (g->K > 1 ? g->K - 1 : 1));
}

uint32_t orc_get_sweep(const orc_group *g) { return g->sweep; }
uint32_t orc_get_swaps(const orc_group *g) { return g->n_swaps; }
