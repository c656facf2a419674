/*
 * rewl_oracle.c -- plain, slow, single-threaded CPU oracle for replica-exchange
 * Wang-Landau (REWL) sampling on the 2D Ising and q-state Potts models.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference semantics the CUDA
 * path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * constant table or helper with the CUDA library, and it never reads the
 * CUDA library's output.
 *
 * Paper: Li, Vogel, Wuest, Landau, "A new paradigm for petascale Monte Carlo
 * simulation: Replica exchange Wang-Landau sampling" (arXiv:1402.2328).
 *   Sec. 2 (standard WL):      accept min[1, g(E_old)/g(E_new)], g -> f g,
 *                              H(E)++, flat H -> reset H, f -> sqrt(f).
 *   Sec. 2, Fig. 1a:           h equal-size windows with overlap o.
 *   Sec. 2:                    m independent walkers per window, each with its
 *                              own g and H; window advances when all m are flat;
 *                              the walkers' g combined and handed back.
 *   Sec. 2, Eq. (1):           replica exchange acceptance
 *                              min[1, g_i(E_X) g_j(E_Y) / (g_i(E_Y) g_j(E_X))],
 *                              impossible when an energy is outside the other
 *                              window.
 *   Sec. 2 (end):              stop when every window reached f_final.
 *   Sec. 3, Eq. (2), Fig. 2:   joining via beta(E) = d ln g/dE, 5-point stencil,
 *                              argmin |beta_i - beta_j|, rescale, piecewise join.
 *
 * Readings where the paper is silent (all carried unchanged by the CUDA path):
 *   bins:   Ising k = (E+2N)/4 in [0,N]; Potts k = E+2N in [0,2N].
 *   windows: o = 0.75 uses exact integer rounding, otherwise round(k*s), W = B/(1+(h-1)(1-o)).
 *   ln f:   f -> sqrt f is ln f -> ln f / 2; a window runs while ln f >= ln f_final.
 *   RNG:    Philox4x32-10; key = seed; ctr = (step lo, step hi, slot, inst<<8 | tag),
 *           tags 0 move, 1 prep, 2 init, 3 swap.
 *   move:   site = mulhi(w0,N); Potts new state (s+1+mulhi(w1,q-1)) mod q; u from w2.
 *           Out-of-window proposals are rejected; after every attempt ln g[k] += ln f
 *           and H[k]++ at the (possibly unchanged) current bin k.
 *   ln u:   a deterministic double-precision logarithm (exponent split + atanh series).
 *   flat:   every swap interval; over the bins any walker of the window ever visited;
 *           min H * count >= flatness * sum H; latched until the window advances.
 *   advance: ln-domain mean over the m walkers in walker order, H = 0, ln f /= 2.
 *   prep:   from the seeded random lattice, single-site moves accepted iff the distance of
 *           k to the window does not grow; after prep_budget sweeps one restart from the
 *           ground state (or, for a window in the upper half of the bins, the checkerboard).
 *   finished windows freeze ln g and H but keep moving and swapping.
 *   2D DOS (Sec. 3, Eqs. 3-4; Ising, Q = magnetisation): with the (E, M) measurement on,
 *           each walker's (bin, up spins) is counted after the moves of every round;
 *           production rounds continue after every window finished (frozen ln g: a
 *           multicanonical walk with weight 1/g_w(E) per window).  Fragments
 *           S_w = mean ln g_w(k) + ln H_w(k,j) - ln sum_j H_w(k,j); adjacent fragments
 *           join where their unit normals (dS/dE, dS/dM, -1) agree best; Eq. (4) averages
 *           g where both are present.
 *   swap:   round r pairs windows (w,w+1) with w = r mod 2; Fisher-Yates permutation of the
 *           m partners; ln P = (lg_i[kX]-lg_i[kY]) + (lg_j[kY]-lg_j[kX]).
 *   prep:   from the seeded random state, accept a move iff the distance of k to the window
 *           does not grow; after prep_budget sweeps restart from the ordered state.
 *   1/t:    (optional schedule, Sec. 2 names the "1/t algorithm" as a valid alternative) after a
 *           halving, if ln f < 1/t with t = (moves per walker) / (visited bins of the window),
 *           the window switches to ln f = 1/t, recomputed at every check, where the m walkers'
 *           ln g are averaged as at an advance, with no flatness test.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fast-math; explicit fma only).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random   */
/* numbers: as easy as 1, 2, 3"): 10 rounds of a multiply-xor bijection */
/* on four 32-bit words, Weyl-sequence key schedule.                    */
/* ------------------------------------------------------------------ */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox4(uint32_t a, uint32_t b, uint32_t c, uint32_t d,
                    const uint32_t key[2], uint32_t out[4])
{
    uint32_t ctr[4] = {a, b, c, d};
    or_philox(ctr, key, out);
}

static uint32_t mulhi32(uint32_t a, uint32_t b)
{
    return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
}

/* ------------------------------------------------------------------ */
/* ln u for u = (w + 1/2) 2^-32: u = m 2^e with m in [sqrt(1/2),sqrt(2)), */
/* ln u = e ln 2 + 2 atanh((m-1)/(m+1)), atanh by its odd Taylor series */
/* to z^11 (z = s^2 <= 0.0295, truncation < 1e-18).  Every operation is  */
/* spelled out so the value is reproducible bit for bit.                */
/* ------------------------------------------------------------------ */
static const double OR_ATANH_C[12] = {
    1.0,
    0x1.5555555555555p-2, /* 1/3  */
    0x1.999999999999ap-3, /* 1/5  */
    0x1.2492492492492p-3, /* 1/7  */
    0x1.c71c71c71c71cp-4, /* 1/9  */
    0x1.745d1745d1746p-4, /* 1/11 */
    0x1.3b13b13b13b14p-4, /* 1/13 */
    0x1.1111111111111p-4, /* 1/15 */
    0x1.e1e1e1e1e1e1ep-5, /* 1/17 */
    0x1.af286bca1af28p-5, /* 1/19 */
    0x1.8618618618618p-5, /* 1/21 */
    0x1.642c8590b2164p-5, /* 1/23 */
};
#define OR_LN2   0x1.62e42fefa39efp-1
#define OR_SQRT2 0x1.6a09e667f3bcdp+0

double or_lnu(uint32_t w)
{
    double u = ((double)w + 0.5) * 0x1p-32;
    uint64_t bits;
    memcpy(&bits, &u, 8);
    int e = (int)((bits >> 52) & 0x7ff) - 1023;
    uint64_t mb = (bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
    double m;
    memcpy(&m, &mb, 8);
    if (m > OR_SQRT2) {
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double p = OR_ATANH_C[11];
    for (int i = 10; i >= 0; i--) p = fma(p, z, OR_ATANH_C[i]);
    double r = s * p;
    r = r + r;
    return fma((double)e, OR_LN2, r);
}

/* The same logarithm for any finite x > 0 in the normal range (fragments of g(E, M)). */
double or_ln(double x)
{
    uint64_t bits;
    memcpy(&bits, &x, 8);
    int e = (int)((bits >> 52) & 0x7ff) - 1023;
    uint64_t mb = (bits & 0x000fffffffffffffull) | 0x3ff0000000000000ull;
    double m;
    memcpy(&m, &mb, 8);
    if (m > OR_SQRT2) {
        m = m * 0.5;
        e = e + 1;
    }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double p = OR_ATANH_C[11];
    for (int i = 10; i >= 0; i--) p = fma(p, z, OR_ATANH_C[i]);
    double r = s * p;
    r = r + r;
    return fma((double)e, OR_LN2, r);
}

/* ------------------------------------------------------------------ */
/* Energy windows (Sec. 2, Fig. 1a).                                    */
/* ------------------------------------------------------------------ */
int or_windows(int B, int h, double o, int *lo, int *hi)
{
    if (B < 1 || h < 1 || !(o >= 0.0 && o < 1.0)) return -1;
    if (h == 1) { lo[0] = 0; hi[0] = B; return 0; }
    if (o == 0.75) {
        long long d = 2LL * (h + 3);
        for (int k = 0; k < h; k++) {
            lo[k] = (int)((2LL * k * B + (h + 3)) / d);
            long long t = (2LL * (k + 4) * B + (h + 3)) / d;
            hi[k] = (int)(t < B ? t : B);
        }
    } else {
        double W = (double)B / (1.0 + (double)(h - 1) * (1.0 - o));
        double s = (1.0 - o) * W;
        for (int k = 0; k < h; k++) {
            lo[k] = (int)floor((double)k * s + 0.5);
            double t = floor((double)k * s + W + 0.5);
            hi[k] = (int)(t < (double)B ? t : (double)B);
        }
    }
    hi[h - 1] = B;
    for (int k = 0; k + 1 < h; k++)
        if (lo[k + 1] > hi[k] || lo[k + 1] <= lo[k]) return -2; /* no overlap / degenerate */
    return 0;
}

/* ------------------------------------------------------------------ */
/* Models.  Ising: E = -sum_<ij> s_i s_j (J = 1), spins +-1, periodic.  */
/* Potts: E = -sum_<ij> delta(s_i, s_j), s in 0..q-1, periodic.         */
/* k counts unsatisfied bonds: Ising k = n_u / 2, Potts k = n_u.        */
/* ------------------------------------------------------------------ */
static int is_ising(int model) { return model == 0; }

long long or_energy(int model, int L, const int8_t *s)
{
    long long E = 0;
    for (int y = 0; y < L; y++)
        for (int x = 0; x < L; x++) {
            int a = s[y * L + x];
            int r = s[y * L + (x + 1) % L];
            int d = s[((y + 1) % L) * L + x];
            if (is_ising(model)) E -= (long long)a * r + (long long)a * d;
            else E -= (long long)(a == r) + (long long)(a == d);
        }
    return E;
}

int or_bin_of_energy(int model, int N, long long E)
{
    if (is_ising(model)) return (int)((E + 2LL * N) / 4);
    return (int)(E + 2LL * N);
}

int or_num_bins(int model, int N) { return is_ising(model) ? N : 2 * N; }

/* Proposal for one single-site move: site and new state from w0, w1;  */
/* returns the bin change dk and stores the new state in *snew.         */
static int propose(int model, int q, int L, const int8_t *s, uint32_t w0, uint32_t w1,
                   int *site_out, int *snew)
{
    int N = L * L;
    int site = (int)mulhi32(w0, (uint32_t)N);
    int x = site % L, y = site / L;
    int nb[4];
    nb[0] = y * L + (x + L - 1) % L;
    nb[1] = y * L + (x + 1) % L;
    nb[2] = ((y + L - 1) % L) * L + x;
    nb[3] = ((y + 1) % L) * L + x;
    int a = s[site];
    int dk;
    if (is_ising(model)) {
        int sum = s[nb[0]] + s[nb[1]] + s[nb[2]] + s[nb[3]];
        dk = a * sum / 2; /* dE = 2 a sum, dk = dE / 4 */
        *snew = -a;
    } else {
        int b = (a + 1 + (int)mulhi32(w1, (uint32_t)(q - 1))) % q;
        dk = 0;
        for (int j = 0; j < 4; j++) dk += (a == s[nb[j]]) - (b == s[nb[j]]);
        *snew = b;
    }
    *site_out = site;
    return dk;
}

/* One WL attempt (Sec. 2): returns 1 if accepted.  lng/H are window-local */
/* arrays indexed by k - lo.  frozen != 0: no ln g / H update.             */
int or_wl_move(int model, int q, int L, int8_t *s, int *k, int lo, int hi,
               double *lng, uint32_t *H, double lnf, int frozen,
               uint32_t w0, uint32_t w1, uint32_t w2, int *dk_out)
{
    int site, snew;
    int dk = propose(model, q, L, s, w0, w1, &site, &snew);
    int kp = *k + dk;
    int acc = 0;
    if (kp >= lo && kp <= hi) {
        double d = lng[*k - lo] - lng[kp - lo];
        if (d >= 0.0) acc = 1;
        else if (or_lnu(w2) < d) acc = 1;
    }
    if (acc) {
        s[site] = (int8_t)snew;
        *k = kp;
    }
    if (!frozen) {
        lng[*k - lo] = lng[*k - lo] + lnf;
        H[*k - lo] += 1u;
    }
    if (dk_out) *dk_out = dk;
    return acc;
}

/* Batched replay: n independent single attempts on separate states.     */
/* spins [n][N], k [n], lo/hi [n], lng/H [n][W], lnf [n], words [n][3].   */
void or_replay_batch(int model, int q, int L, int n, int W, int8_t *spins, int *k,
                     const int *lo, const int *hi, double *lng, uint32_t *H,
                     const double *lnf, const uint8_t *frozen, const uint32_t *words,
                     int *acc, int *dk)
{
    int N = L * L;
    for (int i = 0; i < n; i++)
        acc[i] = or_wl_move(model, q, L, spins + (size_t)i * N, k + i, lo[i], hi[i],
                            lng + (size_t)i * W, H + (size_t)i * W, lnf[i], frozen[i],
                            words[3 * i], words[3 * i + 1], words[3 * i + 2], dk + i);
}

/* ------------------------------------------------------------------ */
/* Full REWL state (Sec. 2).                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    int model, q, L, N, B, h, m, nw, W;
    double overlap, lnf_final, flatness;
    uint32_t key[2];
    uint32_t inst;
    long long interval, prep_budget;
    int *lo, *hi;
    int8_t *spins;      /* [nw][N], owned by the walker slot, swapped on exchange */
    int *k;             /* [nw] current bin of the slot's configuration */
    double *lng;        /* [nw][W] window-local ln g */
    uint32_t *H;        /* [nw][W] */
    uint64_t *step;     /* [nw] WL attempts of the slot since start */
    uint64_t *acc;      /* [nw] accepted WL moves */
    uint64_t *pstep;    /* [nw] prep attempts */
    int *prep_restarts; /* [nw] */
    uint8_t *flat;      /* [nw] */
    double *lnf;        /* [h] */
    int *iter;          /* [h] */
    uint8_t *finished;  /* [h] */
    uint8_t *mask;      /* [h][W] bins visited by any walker of the window */
    uint64_t *swap_att, *swap_acc; /* [h] (index w = pair (w,w+1)) */
    long long *it1_round;  /* [h] rounds done when the first iteration ended (0: not yet) */
    double *frag;          /* [nw][W] each walker's ln g just before its window's last average */
    uint8_t *mode;         /* [h] 0: halving, 1: ln f = 1/t */
    int schedule;          /* 0: f -> sqrt f only, 1: switch to 1/t */
    long long round;
    uint32_t *hem;         /* [h][W][N+1] (bin, up spins) counts, NULL: not measured */
    int production;        /* or_rewl_run keeps going after every window finished */
} or_rewl;

static void *zalloc(size_t n) { return calloc(n ? n : 1, 1); }

void or_rewl_destroy(or_rewl *r)
{
    if (!r) return;
    free(r->lo); free(r->hi); free(r->spins); free(r->k); free(r->lng); free(r->H);
    free(r->step); free(r->acc); free(r->pstep); free(r->prep_restarts); free(r->flat);
    free(r->lnf); free(r->iter); free(r->finished); free(r->mask);
    free(r->swap_att); free(r->swap_acc); free(r->it1_round); free(r->mode); free(r->frag);
    free(r->hem);
    free(r);
}

/* Windows given by the caller (lo[0] = 0, hi[h-1] = B, each next window starting inside the
 * previous one); NULL lo/hi: the equal-size layout of Fig. 1a with overlap `overlap`. */
or_rewl *or_rewl_create_windows(int model, int L, int h, const int *lo_in, const int *hi_in,
                                double overlap, int m, double lnf_final, double flatness,
                                uint64_t seed, uint32_t inst, long long interval,
                                long long prep_budget, double lnf_init)
{
    if (L < 2 || h < 1 || m < 1 || (model != 0 && model < 2) || interval < 1) return NULL;
    or_rewl *r = (or_rewl *)zalloc(sizeof(or_rewl));
    r->model = model;
    r->q = model == 0 ? 2 : model;
    r->L = L;
    r->N = L * L;
    r->B = or_num_bins(model, r->N);
    r->h = h;
    r->m = m;
    r->nw = h * m;
    r->overlap = overlap;
    r->lnf_final = lnf_final;
    r->flatness = flatness;
    r->key[0] = (uint32_t)seed;
    r->key[1] = (uint32_t)(seed >> 32);
    r->inst = inst;
    r->interval = interval;
    r->prep_budget = prep_budget;
    r->lo = (int *)zalloc(sizeof(int) * h);
    r->hi = (int *)zalloc(sizeof(int) * h);
    if (lo_in && hi_in) {
        for (int w = 0; w < h; w++) {
            r->lo[w] = lo_in[w];
            r->hi[w] = hi_in[w];
        }
        int bad = r->lo[0] != 0 || r->hi[h - 1] != r->B;
        for (int w = 0; w < h; w++) bad |= r->hi[w] <= r->lo[w];
        for (int w = 0; w + 1 < h; w++)
            bad |= r->lo[w + 1] <= r->lo[w] || r->lo[w + 1] > r->hi[w] || r->hi[w + 1] < r->hi[w];
        if (bad) { or_rewl_destroy(r); return NULL; }
    } else if (or_windows(r->B, h, overlap, r->lo, r->hi) != 0) {
        or_rewl_destroy(r);
        return NULL;
    }
    int W = 0;
    for (int w = 0; w < h; w++)
        if (r->hi[w] - r->lo[w] + 1 > W) W = r->hi[w] - r->lo[w] + 1;
    r->W = W;
    size_t nw = (size_t)r->nw;
    r->spins = (int8_t *)zalloc(nw * r->N);
    r->k = (int *)zalloc(sizeof(int) * nw);
    r->lng = (double *)zalloc(sizeof(double) * nw * W);
    r->H = (uint32_t *)zalloc(sizeof(uint32_t) * nw * W);
    r->step = (uint64_t *)zalloc(8 * nw);
    r->acc = (uint64_t *)zalloc(8 * nw);
    r->pstep = (uint64_t *)zalloc(8 * nw);
    r->prep_restarts = (int *)zalloc(sizeof(int) * nw);
    r->flat = (uint8_t *)zalloc(nw);
    r->lnf = (double *)zalloc(sizeof(double) * h);
    r->iter = (int *)zalloc(sizeof(int) * h);
    r->finished = (uint8_t *)zalloc(h);
    r->mask = (uint8_t *)zalloc((size_t)h * W);
    r->swap_att = (uint64_t *)zalloc(8 * (size_t)h);
    r->swap_acc = (uint64_t *)zalloc(8 * (size_t)h);
    r->it1_round = (long long *)zalloc(8 * (size_t)h);
    r->frag = (double *)zalloc(sizeof(double) * nw * W);
    r->mode = (uint8_t *)zalloc(h);
    for (int w = 0; w < h; w++) {
        r->lnf[w] = lnf_init;
        r->finished[w] = lnf_init < lnf_final;
    }
    return r;
}

or_rewl *or_rewl_create(int model, int L, int h, double overlap, int m, double lnf_final,
                        double flatness, uint64_t seed, uint32_t inst, long long interval,
                        long long prep_budget, double lnf_init)
{
    return or_rewl_create_windows(model, L, h, NULL, NULL, overlap, m, lnf_final, flatness, seed,
                                  inst, interval, prep_budget, lnf_init);
}

/* Optional warm start: ln g over all B+1 bins copied into every walker. */
void or_rewl_set_lng(or_rewl *r, const double *lng_bins)
{
    for (int w = 0; w < r->h; w++)
        for (int i = 0; i < r->m; i++) {
            double *g = r->lng + (size_t)(w * r->m + i) * r->W;
            for (int b = r->lo[w]; b <= r->hi[w]; b++) g[b - r->lo[w]] = lng_bins[b];
        }
}

static int dist_to(int k, int lo, int hi) { return k < lo ? lo - k : (k > hi ? k - hi : 0); }

/* Seeded start + prep into the window (silent in the paper; readings above). */
int or_rewl_init(or_rewl *r)
{
    int N = r->N;
    int fails = 0;
    for (int w = 0; w < r->h; w++)
        for (int i = 0; i < r->m; i++) {
            int g = w * r->m + i;
            int8_t *s = r->spins + (size_t)g * N;
            uint32_t out[4];
            for (int c = 0; 4 * c < N; c++) {
                philox4((uint32_t)c, 0u, (uint32_t)g, (r->inst << 8) | 2u, r->key, out);
                for (int j = 0; j < 4 && 4 * c + j < N; j++) {
                    if (is_ising(r->model)) s[4 * c + j] = (out[j] >> 31) ? -1 : 1;
                    else s[4 * c + j] = (int8_t)mulhi32(out[j], (uint32_t)r->q);
                }
            }
            int k = or_bin_of_energy(r->model, N, or_energy(r->model, r->L, s));
            int lo = r->lo[w], hi = r->hi[w];
            uint64_t ps = 0;
            uint64_t budget = (uint64_t)r->prep_budget * (uint64_t)N;
            for (int phase = 0; phase < 2 && dist_to(k, lo, hi) > 0; phase++) {
                if (phase == 1) {
                    /* restart from the ordered state nearer the window: the ground state, or
                     * for a window in the upper half of the bins the checkerboard (every bond
                     * unsatisfied for even L) */
                    int top = 2 * lo > r->B;
                    for (int j = 0; j < N; j++) {
                        int odd = top && (((j % r->L) + (j / r->L)) & 1);
                        s[j] = is_ising(r->model) ? (odd ? -1 : 1) : (odd ? 1 : 0);
                    }
                    k = top ? or_bin_of_energy(r->model, N, or_energy(r->model, r->L, s)) : 0;
                    r->prep_restarts[g]++;
                }
                uint64_t end = ps + budget;
                while (dist_to(k, lo, hi) > 0 && ps < end) {
                    philox4((uint32_t)ps, (uint32_t)(ps >> 32), (uint32_t)g, (r->inst << 8) | 1u,
                            r->key, out);
                    int site, snew;
                    int dk = propose(r->model, r->q, r->L, s, out[0], out[1], &site, &snew);
                    if (dist_to(k + dk, lo, hi) <= dist_to(k, lo, hi)) {
                        s[site] = (int8_t)snew;
                        k += dk;
                    }
                    ps++;
                }
            }
            r->pstep[g] = ps;
            r->k[g] = k;
            if (dist_to(k, lo, hi) > 0) fails++;
        }
    return fails ? -1 : 0;
}

/* Per-walker flatness and window advance (Sec. 2; readings above). */
static void check_window(or_rewl *r, int w)
{
    int W = r->W, m = r->m;
    int nb = r->hi[w] - r->lo[w] + 1;
    uint8_t *mask = r->mask + (size_t)w * W;
    for (int i = 0; i < m; i++) {
        const uint32_t *H = r->H + (size_t)(w * m + i) * W;
        for (int b = 0; b < nb; b++)
            if (H[b] > 0) mask[b] = 1;
    }
    int all = 1;
    long long nvis = 0;
    for (int b = 0; b < nb; b++) nvis += mask[b];
    for (int i = 0; i < m && !r->mode[w]; i++) {
        int g = w * m + i;
        if (!r->flat[g]) {
            const uint32_t *H = r->H + (size_t)g * W;
            uint64_t sum = 0;
            uint32_t mn = 0xffffffffu;
            long long cnt = 0;
            for (int b = 0; b < nb; b++)
                if (mask[b]) {
                    sum += H[b];
                    if (H[b] < mn) mn = H[b];
                    cnt++;
                }
            if (cnt > 0 && (double)mn * (double)cnt >= r->flatness * (double)sum) r->flat[g] = 1;
        }
        all &= r->flat[g];
    }
    if (!all) return; /* in 1/t mode no walker is ever flagged flat: all stays 1 */
    /* ln f after this advance (same arithmetic as below): a window about to finish keeps its
       walkers' last fragments for resampling error bars (Sec. 3) */
    double inv_t0 = nvis > 0 ? (double)nvis / (double)r->step[w * m] : 0.0;
    double nl0 = r->mode[w] ? inv_t0 : r->lnf[w] * 0.5;
    if (!r->mode[w] && r->schedule == 1 && nl0 < inv_t0) nl0 = inv_t0;
    if (nl0 < r->lnf_final)
        for (int i = 0; i < m; i++)
            memcpy(r->frag + (size_t)(w * m + i) * W, r->lng + (size_t)(w * m + i) * W,
                   sizeof(double) * (size_t)nb);
    for (int b = 0; b < nb; b++) {
        double acc = 0.0;
        for (int i = 0; i < m; i++) acc = acc + r->lng[(size_t)(w * m + i) * W + b];
        double avg = acc / (double)m;
        for (int i = 0; i < m; i++) {
            r->lng[(size_t)(w * m + i) * W + b] = avg;
            r->H[(size_t)(w * m + i) * W + b] = 0u;
        }
    }
    for (int i = 0; i < m; i++) r->flat[w * m + i] = 0;
    /* 1/t with t = moves per walker / visited bins, i.e. ln f = visited bins / moves */
    double inv_t = nvis > 0 ? (double)nvis / (double)r->step[w * m] : 0.0;
    if (r->mode[w]) {
        r->lnf[w] = inv_t;
    } else {
        r->lnf[w] = r->lnf[w] * 0.5;
        if (r->schedule == 1 && r->lnf[w] < inv_t) {
            r->mode[w] = 1;
            r->lnf[w] = inv_t;
        }
    }
    if (r->iter[w] == 0) r->it1_round[w] = r->round + 1;
    r->iter[w] += 1;
    if (r->lnf[w] < r->lnf_final) r->finished[w] = 1;
}

void or_rewl_set_schedule(or_rewl *r, int schedule) { r->schedule = schedule; }
void or_rewl_get_extra(const or_rewl *r, long long *it1_round, uint8_t *mode, double *frag)
{
    if (it1_round) memcpy(it1_round, r->it1_round, 8 * (size_t)r->h);
    if (mode) memcpy(mode, r->mode, (size_t)r->h);
    if (frag) memcpy(frag, r->frag, sizeof(double) * (size_t)r->nw * r->W);
}

/* Replica exchange between windows w and w+1 in round rd (Sec. 2, Eq. 1). */
static void swap_pair(or_rewl *r, int w, long long rd)
{
    int m = r->m, W = r->W, N = r->N;
    int perm[4096];
    uint32_t out[4];
    uint32_t tag = (r->inst << 8) | 3u;
    for (int i = 0; i < m; i++) perm[i] = i;
    for (int i = m - 1; i >= 1; i--) {
        philox4((uint32_t)i, (uint32_t)rd, (uint32_t)w, tag, r->key, out);
        int j = (int)mulhi32(out[0], (uint32_t)(i + 1));
        int t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    int loA = r->lo[w], hiA = r->hi[w], loB = r->lo[w + 1], hiB = r->hi[w + 1];
    for (int i = 0; i < m; i++) {
        int a = w * m + i, b = (w + 1) * m + perm[i];
        int kx = r->k[a], ky = r->k[b];
        r->swap_att[w]++;
        if (kx < loB || kx > hiB || ky < loA || ky > hiA) continue;
        const double *ga = r->lng + (size_t)a * W;
        const double *gb = r->lng + (size_t)b * W;
        double lnP = (ga[kx - loA] - ga[ky - loA]) + (gb[ky - loB] - gb[kx - loB]);
        int acc = lnP >= 0.0;
        if (!acc) {
            philox4((uint32_t)(m + i), (uint32_t)rd, (uint32_t)w, tag, r->key, out);
            acc = or_lnu(out[0]) < lnP;
        }
        if (acc) {
            int8_t *sa = r->spins + (size_t)a * N, *sb = r->spins + (size_t)b * N;
            for (int j = 0; j < N; j++) { int8_t t = sa[j]; sa[j] = sb[j]; sb[j] = t; }
            r->k[a] = ky;
            r->k[b] = kx;
            r->swap_acc[w]++;
        }
    }
}

/* The exchange of one window pair alone (round number rd), for tests of the exchange logic. */
void or_rewl_swap(or_rewl *r, int w, long long rd)
{
    if (w >= 0 && w + 1 < r->h) swap_pair(r, w, rd);
}

/* One round: interval moves for every walker, flatness/advance, swaps. */
void or_rewl_round(or_rewl *r)
{
    int W = r->W, N = r->N;
    uint32_t out[4];
    for (int w = 0; w < r->h; w++) {
        int lo = r->lo[w], hi = r->hi[w];
        for (int i = 0; i < r->m; i++) {
            int g = w * r->m + i;
            int8_t *s = r->spins + (size_t)g * N;
            double *lng = r->lng + (size_t)g * W;
            uint32_t *H = r->H + (size_t)g * W;
            int k = r->k[g];
            for (long long t = 0; t < r->interval; t++) {
                uint64_t st = r->step[g]++;
                philox4((uint32_t)st, (uint32_t)(st >> 32), (uint32_t)g, (r->inst << 8) | 0u,
                        r->key, out);
                r->acc[g] += (uint64_t)or_wl_move(r->model, r->q, r->L, s, &k, lo, hi, lng, H,
                                                  r->lnf[w], r->finished[w], out[0], out[1],
                                                  out[2], NULL);
            }
            r->k[g] = k;
        }
    }
    if (r->hem) {
        for (int g = 0; g < r->nw; g++) {
            int w = g / r->m, up = 0;
            const int8_t *sp = r->spins + (size_t)g * N;
            for (int i = 0; i < N; i++) up += sp[i] > 0;
            r->hem[((size_t)w * W + (size_t)(r->k[g] - r->lo[w])) * (size_t)(N + 1) + up] += 1u;
        }
    }
    for (int w = 0; w < r->h; w++)
        if (!r->finished[w]) check_window(r, w);
    for (int w = (int)(r->round & 1); w + 1 < r->h; w += 2) swap_pair(r, w, r->round);
    r->round++;
}

/* Runs rounds until every window finished or max_rounds; returns rounds done. */
long long or_rewl_run(or_rewl *r, long long max_rounds)
{
    long long n = 0;
    while (n < max_rounds) {
        int done = !r->production;
        for (int w = 0; w < r->h; w++) done &= r->finished[w];
        if (done) break;
        or_rewl_round(r);
        n++;
    }
    return n;
}

/* Accessors for the tests. */
int or_rewl_dims(const or_rewl *r, int *out /* N,B,h,m,W */)
{
    out[0] = r->N; out[1] = r->B; out[2] = r->h; out[3] = r->m; out[4] = r->W;
    return 0;
}
void or_rewl_windows_get(const or_rewl *r, int *lo, int *hi)
{
    memcpy(lo, r->lo, sizeof(int) * r->h);
    memcpy(hi, r->hi, sizeof(int) * r->h);
}
void or_rewl_get(const or_rewl *r, int8_t *spins, int *k, double *lng, uint32_t *H,
                 uint64_t *step, uint64_t *acc, uint8_t *flat, double *lnf, int *iter,
                 uint8_t *finished, uint8_t *mask, uint64_t *swap_att, uint64_t *swap_acc,
                 uint64_t *pstep, int *prep_restarts, long long *round)
{
    size_t nw = (size_t)r->nw;
    if (spins) memcpy(spins, r->spins, nw * r->N);
    if (k) memcpy(k, r->k, sizeof(int) * nw);
    if (lng) memcpy(lng, r->lng, sizeof(double) * nw * r->W);
    if (H) memcpy(H, r->H, sizeof(uint32_t) * nw * r->W);
    if (step) memcpy(step, r->step, 8 * nw);
    if (acc) memcpy(acc, r->acc, 8 * nw);
    if (flat) memcpy(flat, r->flat, nw);
    if (lnf) memcpy(lnf, r->lnf, sizeof(double) * r->h);
    if (iter) memcpy(iter, r->iter, sizeof(int) * r->h);
    if (finished) memcpy(finished, r->finished, r->h);
    if (mask) memcpy(mask, r->mask, (size_t)r->h * r->W);
    if (swap_att) memcpy(swap_att, r->swap_att, 8 * (size_t)r->h);
    if (swap_acc) memcpy(swap_acc, r->swap_acc, 8 * (size_t)r->h);
    if (pstep) memcpy(pstep, r->pstep, 8 * nw);
    if (prep_restarts) memcpy(prep_restarts, r->prep_restarts, sizeof(int) * nw);
    if (round) *round = r->round;
}
/* Test hook: overwrite the dynamic state (used to plant states in tests). */
void or_rewl_put(or_rewl *r, const int8_t *spins, const int *k, const double *lng,
                 const uint32_t *H, const uint64_t *step)
{
    size_t nw = (size_t)r->nw;
    if (spins) memcpy(r->spins, spins, nw * r->N);
    if (k) memcpy(r->k, k, sizeof(int) * nw);
    if (lng) memcpy(r->lng, lng, sizeof(double) * nw * r->W);
    if (H) memcpy(r->H, H, sizeof(uint32_t) * nw * r->W);
    if (step) memcpy(r->step, step, 8 * nw);
}

/* Test hook: overwrite the window-level state and the round counter (NULL: keep). */
void or_rewl_put_window(or_rewl *r, const double *lnf, const int *iter, const uint8_t *flat,
                        const uint8_t *finished, const uint8_t *mask, const uint8_t *mode,
                        const long long *round)
{
    size_t h = (size_t)r->h;
    if (lnf) memcpy(r->lnf, lnf, sizeof(double) * h);
    if (iter) memcpy(r->iter, iter, sizeof(int) * h);
    if (flat) memcpy(r->flat, flat, (size_t)r->nw);
    if (finished) memcpy(r->finished, finished, h);
    if (mask) memcpy(r->mask, mask, h * (size_t)r->W);
    if (mode) memcpy(r->mode, mode, h);
    if (round) r->round = *round;
}

/* Test hook: the flatness test and window advance of window w alone, as a round runs it
 * (skipped for a finished window). */
void or_rewl_check(or_rewl *r, int w)
{
    if (w >= 0 && w < r->h && !r->finished[w]) check_window(r, w);
}

/* Window average of ln g (O-8 formula, walker order) for window w. */
void or_rewl_window_mean(const or_rewl *r, int w, double *out)
{
    int nb = r->hi[w] - r->lo[w] + 1;
    for (int b = 0; b < nb; b++) {
        double acc = 0.0;
        for (int i = 0; i < r->m; i++) acc = acc + r->lng[(size_t)(w * r->m + i) * r->W + b];
        out[b] = acc / (double)r->m;
    }
}

/* ------------------------------------------------------------------ */
/* Joining (Sec. 3, Eq. 2, Fig. 2).  lngw: [h][W] window-local ln g,    */
/* valid: [h][W].  out: B+1 values, -INFINITY where no window is valid. */
/* de: energy per bin (4 Ising, 1 Potts); step: stencil spacing in bins.*/
/* norm_target: if norm == 0, logsumexp(out) == norm_target;            */
/* if norm == 1, out[lowest valid bin] == norm_target.                  */
/* joins[h-1] receives the join bins.  Returns 0 or -1 (cannot join).   */
/* ------------------------------------------------------------------ */
static int stencil_beta(const double *l, const uint8_t *v, int nb, int b, int step, int npts,
                        double de, double *beta)
{
    if (npts == 5) {
        if (b - 2 * step < 0 || b + 2 * step >= nb) return 0;
        if (!(v[b - 2 * step] && v[b - step] && v[b + step] && v[b + 2 * step])) return 0;
        double num = ((-l[b + 2 * step] + 8.0 * l[b + step]) - 8.0 * l[b - step]) + l[b - 2 * step];
        *beta = num / (12.0 * de * (double)step);
        return 1;
    }
    if (b - step < 0 || b + step >= nb) return 0;
    if (!(v[b - step] && v[b + step])) return 0;
    *beta = (l[b + step] - l[b - step]) / (2.0 * de * (double)step);
    return 1;
}

int or_stitch(int h, int W, int B, const int *lo, const int *hi, const double *lngw,
              const uint8_t *valid, double de, int step, int norm, double norm_target,
              double *out, int *joins)
{
    for (int b = 0; b <= B; b++) out[b] = -INFINITY;
    double shift = 0.0;
    int prev = -1;
    for (int b = lo[0]; b <= hi[0]; b++)
        if (valid[b - lo[0]]) out[b] = lngw[b - lo[0]];
    for (int w = 0; w + 1 < h; w++) {
        const double *la = lngw + (size_t)w * W, *lb = lngw + (size_t)(w + 1) * W;
        const uint8_t *va = valid + (size_t)w * W, *vb = valid + (size_t)(w + 1) * W;
        int nba = hi[w] - lo[w] + 1, nbb = hi[w + 1] - lo[w + 1] + 1;
        int kj = -1;
        for (int npts = 5; npts >= 3 && kj < 0; npts -= 2) {
            double best = INFINITY;
            for (int k = lo[w + 1]; k <= hi[w]; k++) {
                if (k <= prev) continue;
                double ba, bb;
                if (!va[k - lo[w]] || !vb[k - lo[w + 1]]) continue;
                if (!stencil_beta(la, va, nba, k - lo[w], step, npts, de, &ba)) continue;
                if (!stencil_beta(lb, vb, nbb, k - lo[w + 1], step, npts, de, &bb)) continue;
                double dbeta = fabs(ba - bb);
                if (dbeta < best) { best = dbeta; kj = k; }
            }
        }
        if (kj < 0) { /* valid-in-both bin nearest the overlap midpoint, ties -> smaller */
            int mid2 = lo[w + 1] + hi[w]; /* twice the midpoint */
            int bestd = 1 << 30;
            for (int k = lo[w + 1]; k <= hi[w]; k++) {
                if (k <= prev || !va[k - lo[w]] || !vb[k - lo[w + 1]]) continue;
                int d = 2 * k - mid2; if (d < 0) d = -d;
                if (d < bestd) { bestd = d; kj = k; }
            }
        }
        if (kj < 0) return -1;
        /* left value at the join point is the already-shifted window w */
        shift = (la[kj - lo[w]] + shift) - lb[kj - lo[w + 1]];
        for (int b = lo[w + 1]; b <= hi[w + 1]; b++)
            if (b >= kj) out[b] = vb[b - lo[w + 1]] ? lb[b - lo[w + 1]] + shift : -INFINITY;
        joins[w] = kj;
        prev = kj;
    }
    if (norm == 0) {
        double mx = -INFINITY;
        for (int b = 0; b <= B; b++) if (out[b] > mx) mx = out[b];
        double s = 0.0;
        for (int b = 0; b <= B; b++) if (out[b] > -INFINITY) s += exp(out[b] - mx);
        double c = (mx + log(s)) - norm_target;
        for (int b = 0; b <= B; b++) if (out[b] > -INFINITY) out[b] -= c;
    } else {
        int b0 = 0;
        while (b0 <= B && out[b0] == -INFINITY) b0++;
        if (b0 > B) return -1;
        double c = out[b0] - norm_target;
        for (int b = 0; b <= B; b++) if (out[b] > -INFINITY) out[b] -= c;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Joint density of states g(E, M) (Sec. 3, Eqs. 3-4), Ising only.      */
/* ------------------------------------------------------------------ */
int or_rewl_measure_em(or_rewl *r, int on)
{
    free(r->hem);
    r->hem = NULL;
    if (!on) return 0;
    if (r->model != 0) return -1;
    r->hem = (uint32_t *)zalloc(sizeof(uint32_t) * (size_t)r->h * r->W * (size_t)(r->N + 1));
    return 0;
}

void or_rewl_set_production(or_rewl *r, int on) { r->production = on; }

int or_rewl_get_hem(const or_rewl *r, uint32_t *out)
{
    if (!r->hem) return -1;
    memcpy(out, r->hem, sizeof(uint32_t) * (size_t)r->h * r->W * (size_t)(r->N + 1));
    return 0;
}

/* Fragments: S[w][b][j] = mean[w][b] + ln H[w][b][j] - ln sum_j H[w][b][j] where bin b of
 * window w is valid and H > 0, else -INFINITY.  Rows b >= hi-lo+1 are -INFINITY. */
void or_frag_em(int h, int W, int N1, const int *lo, const int *hi, const double *mean,
                const uint8_t *valid, const uint32_t *hem, double *S)
{
    for (int w = 0; w < h; w++)
        for (int b = 0; b < W; b++) {
            const uint32_t *row = hem + ((size_t)w * W + b) * N1;
            double *out = S + ((size_t)w * W + b) * N1;
            uint64_t tot = 0;
            for (int j = 0; j < N1; j++) tot += row[j];
            int ok = b <= hi[w] - lo[w] && valid[(size_t)w * W + b] && tot > 0;
            double lt = ok ? or_ln((double)tot) : 0.0;
            for (int j = 0; j < N1; j++)
                out[j] = (ok && row[j] > 0) ? (mean[(size_t)w * W + b] + or_ln((double)row[j])) - lt
                                           : -INFINITY;
        }
}

/* Derivative of one fragment along an axis at index i (n points, stride st): 5-point stencil
 * where the four neighbours are present, else 3-point, else none. */
static int em_deriv(const double *S, int i, int n, int st, double d, double *out)
{
    if (i - 2 >= 0 && i + 2 < n && S[(i - 2) * st] > -INFINITY && S[(i - 1) * st] > -INFINITY &&
        S[(i + 1) * st] > -INFINITY && S[(i + 2) * st] > -INFINITY) {
        double num = ((-S[(i + 2) * st] + 8.0 * S[(i + 1) * st]) - 8.0 * S[(i - 1) * st]) + S[(i - 2) * st];
        *out = num / (12.0 * d);
        return 1;
    }
    if (i - 1 >= 0 && i + 1 < n && S[(i - 1) * st] > -INFINITY && S[(i + 1) * st] > -INFINITY) {
        *out = (S[(i + 1) * st] - S[(i - 1) * st]) / (2.0 * d);
        return 1;
    }
    return 0;
}

/* Unit-normal gradient of fragment Sw (nb rows x N1 columns) at (b, j): Eq. (3). */
static int em_grad(const double *Sw, int nb, int N1, int b, int j, double de, double dq,
                   double *gE, double *gQ)
{
    const double *col = Sw + j;            /* column j, stride N1 */
    const double *row = Sw + (size_t)b * N1;
    return em_deriv(col, b, nb, N1, de, gE) && em_deriv(row, j, N1, 1, dq, gQ);
}

/* Joins adjacent fragments (w, w+1) at the point where n_w . n_(w+1) is largest (ties: the
 * smallest bin, then the smallest j; with no normals in both: the point present in both
 * nearest to the middle of the overlap rows), shifts window w+1 to agree there with the
 * already shifted window w, then merges the windows in order with Eq. (4).  out: (B+1) x N1,
 * -INFINITY where absent; logsumexp(out) == norm_target.  joins: [h-1][2] (bin, j).
 * Returns 0 or -1 (two adjacent fragments share no point). */
int or_join_em(int h, int W, int B, int N1, const int *lo, const int *hi, const double *S,
               double de, double dq, double norm_target, double *out, int *joins)
{
    double *shift = (double *)zalloc(sizeof(double) * (size_t)h);
    for (int w = 0; w + 1 < h; w++) {
        const double *Sa = S + (size_t)w * W * N1, *Sb = S + (size_t)(w + 1) * W * N1;
        int nba = hi[w] - lo[w] + 1, nbb = hi[w + 1] - lo[w + 1] + 1;
        int bk = -1, bj = -1;
        double best = -INFINITY;
        for (int k = lo[w + 1]; k <= hi[w]; k++)
            for (int j = 0; j < N1; j++) {
                int a = k - lo[w], b = k - lo[w + 1];
                if (!(Sa[(size_t)a * N1 + j] > -INFINITY && Sb[(size_t)b * N1 + j] > -INFINITY)) continue;
                double aE, aQ, bE, bQ;
                if (!em_grad(Sa, nba, N1, a, j, de, dq, &aE, &aQ)) continue;
                if (!em_grad(Sb, nbb, N1, b, j, de, dq, &bE, &bQ)) continue;
                double num = (aE * bE + aQ * bQ) + 1.0;
                double den = sqrt((aE * aE + aQ * aQ) + 1.0) * sqrt((bE * bE + bQ * bQ) + 1.0);
                double dot = num / den;
                if (dot > best) { best = dot; bk = k; bj = j; }
            }
        if (bk < 0) {
            int mid2 = lo[w + 1] + hi[w], bestd = 1 << 30;
            for (int k = lo[w + 1]; k <= hi[w]; k++) {
                int d = 2 * k - mid2;
                if (d < 0) d = -d;
                if (d >= bestd) continue;
                for (int j = 0; j < N1; j++)
                    if (Sa[(size_t)(k - lo[w]) * N1 + j] > -INFINITY &&
                        Sb[(size_t)(k - lo[w + 1]) * N1 + j] > -INFINITY) {
                        bestd = d; bk = k; bj = j;
                        break;
                    }
            }
        }
        if (bk < 0) { free(shift); return -1; }
        shift[w + 1] = (Sa[(size_t)(bk - lo[w]) * N1 + bj] + shift[w]) - Sb[(size_t)(bk - lo[w + 1]) * N1 + bj];
        joins[2 * w] = bk;
        joins[2 * w + 1] = bj;
    }
    for (size_t i = 0; i < (size_t)(B + 1) * N1; i++) out[i] = -INFINITY;
    for (int w = 0; w < h; w++)
        for (int k = lo[w]; k <= hi[w]; k++)
            for (int j = 0; j < N1; j++) {
                double v = S[((size_t)w * W + (k - lo[w])) * N1 + j];
                if (!(v > -INFINITY)) continue;
                v = v + shift[w];
                double *o = out + (size_t)k * N1 + j;
                if (*o > -INFINITY) {            /* Eq. (4): (g_i + g_j) / 2 */
                    double mx = *o > v ? *o : v, mn = *o > v ? v : *o;
                    *o = (mx + log1p(exp(mn - mx))) - OR_LN2;
                } else {
                    *o = v;
                }
            }
    free(shift);
    double mx = -INFINITY;
    for (size_t i = 0; i < (size_t)(B + 1) * N1; i++) if (out[i] > mx) mx = out[i];
    double sum = 0.0;
    for (size_t i = 0; i < (size_t)(B + 1) * N1; i++) if (out[i] > -INFINITY) sum += exp(out[i] - mx);
    double c = (mx + log(sum)) - norm_target;
    for (size_t i = 0; i < (size_t)(B + 1) * N1; i++) if (out[i] > -INFINITY) out[i] -= c;
    return 0;
}
