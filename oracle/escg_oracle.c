/*
 * escg_oracle.c -- plain, slow, single-threaded CPU oracle for the ESCG
 * Monte Carlo step.  TEST INFRASTRUCTURE ONLY (see escg_oracle.h): the
 * product path never includes, links or calls this file.
 *
 * Everything here is written straight from the paper's definitions
 * (Section 3.1 "Implementation": lattice indexing and periodic neighbours,
 * Alg. 2 "Dominance Check", the circulant dominance definition, the three
 * actions and their rates with epsilon = 2MN, Alg. 3 "Elementary Step",
 * Alg. 4 "Overall ESCG Loop") and from the schedule-version-1 definition of
 * the coloured sublattice decomposition, with no blocking, fusion or
 * reordering beyond what those definitions state.
 */
#include "escg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, Salmon et al. SC'11, Section 3: each round multiplies the
 * counter words 0 and 2 by two fixed odd constants, takes the 64-bit
 * products apart into high and low halves, XORs the high halves with the
 * other two counter words and the round key, and permutes; the key is
 * bumped by two Weyl constants between rounds.  Ten rounds. */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_many(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i)
        orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}

static void philox_at(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                      uint32_t out[4])
{
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* Counter tags (word 3 of the Philox counter) of schedule v1. */
enum { TAG_INIT = 1, TAG_ORDER = 2, TAG_FORDER = 3, TAG_STEP = 4, TAG_RS = 5 };

/* floor(x * n / 2^32) */
static uint32_t umulhi32(uint32_t x, uint32_t n) { return (uint32_t)(((uint64_t)x * n) >> 32); }

/* ------------------------------------------------------------------------ */
/* Dominance: circulant C(S, K) and Alg. 2. */
int orc_circulant(int32_t S, const int32_t* K, int32_t nK, uint8_t* D)
{
    if (S < 1 || nK < 0 || (nK > 0 && !K) || !D) return -1;
    for (int32_t i = 0; i < S; ++i)
        for (int32_t j = 0; j < S; ++j) {
            int32_t off = (j - i + S) % S;
            uint8_t v = 0;
            for (int32_t k = 0; k < nK; ++k)
                if (off == K[k]) v = 1;
            D[i * S + j] = v;
        }
    return 0;
}

int orc_dominates(int32_t a, int32_t b, int32_t S, const uint8_t* D)
{
    if (a == 0 || b == 0) return 0;               /* empty sites cannot dominate */
    return D[(a - 1) * S + (b - 1)] == 1;
}

/* Alg. 3 from the point where the action is known: same species -> no
 * change; exchange swaps; interaction empties the dominated one (the
 * selected site's dominance is tested first); reproduction fills an empty
 * neighbour with the selected species, else an empty selected site with the
 * neighbour's species. */
void orc_rule(int32_t action, int32_t S, const uint8_t* D, uint8_t* a, uint8_t* b)
{
    uint8_t species = *a, neighbour = *b;
    if (species == neighbour || action == ORC_INTERACT_FAIL) return;
    if (action == ORC_EXCHANGE) {
        *a = neighbour;
        *b = species;
    } else if (action == ORC_INTERACT) {
        if (neighbour != 0) {
            if (orc_dominates(species, neighbour, S, D))
                *b = 0;
            else if (orc_dominates(neighbour, species, S, D))
                *a = 0;
        }
    } else {
        if (neighbour == 0)
            *b = species;
        else if (species == 0)
            *a = neighbour;
    }
}

double orc_exchange_from_mobility(double M, int64_t N) { return 2.0 * M * (double)N; }

int orc_thresholds(double I, double P, double X, uint64_t* TX, uint64_t* TXI)
{
    if (!(I >= 0.0) || !(P >= 0.0) || !(X >= 0.0)) return -1;
    double R = (X + I) + P;
    if (!(R > 0.0) || isinf(R)) return -1;
    *TX = (uint64_t)floor(ldexp(X / R, 32) + 0.5);
    *TXI = (uint64_t)floor(ldexp((X + I) / R, 32) + 0.5);
    return 0;
}

/* Park, Chen and Szolnoki's probabilistic dominance (Section "Park, Chen,
 * Szolnoki"): the edge between the two species of a pair carries the
 * probability that an interaction across it takes place.  Pairs without an
 * edge, with an empty site, or of equal species: 1 (Alg. 2 already makes
 * their interaction a no-op). */
double orc_pair_prob(int32_t a, int32_t b, int32_t S, const uint8_t* D, const double* Pd)
{
    if (!Pd || a == 0 || b == 0 || a == b) return 1.0;
    if (orc_dominates(a, b, S, D)) return Pd[(a - 1) * S + (b - 1)];
    if (orc_dominates(b, a, S, D)) return Pd[(b - 1) * S + (a - 1)];
    return 1.0;
}

uint64_t orc_interaction_threshold(uint64_t TX, uint64_t TXI, double p)
{
    if (!(p > 0.0)) return TX;
    if (p >= 1.0) return TXI;
    /* q = p in 0.32 fixed point, rounded; the product is exact in 128 bits */
    uint64_t q = (uint64_t)floor(ldexp(p, 32) + 0.5);
    unsigned __int128 w = (unsigned __int128)(TXI - TX) * q + ((unsigned __int128)1 << 31);
    return TX + (uint64_t)(w >> 32);
}

int orc_counts(int64_t n, const uint8_t* lattice, int32_t S, uint64_t* counts)
{
    if (n < 0 || S < 1 || !counts || (n > 0 && !lattice)) return -1;
    for (int32_t s = 0; s <= S; ++s) counts[s] = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (lattice[i] > S) return -2;
        counts[lattice[i]]++;
    }
    return 0;
}

/* Neighbour in one of the paper's neighbourhoods (Alg. 3: a direction from
 * [0, neighbourhood), "von-Neumann or Moore"): 0 up, 1 down, 2 left, 3 right,
 * then the diagonals 4 up-left, 5 up-right, 6 down-left, 7 down-right.  At
 * the lattice edge the step wraps ("flux") or, with reflect, is mirrored:
 * a coordinate that would leave the lattice moves the other way instead. */
static const int8_t kDirRow[8] = {-1, 1, 0, 0, -1, -1, 1, 1};
static const int8_t kDirCol[8] = {0, 0, -1, 1, -1, 1, -1, 1};
static int64_t neighbour_v(int32_t L, int32_t H, int32_t row, int32_t col, int32_t dir, int32_t reflect)
{
    int32_t nr = row + kDirRow[dir], nc = col + kDirCol[dir];
    if (reflect) {
        if (nr < 0 || nr >= H) nr = row - kDirRow[dir];
        if (nc < 0 || nc >= L) nc = col - kDirCol[dir];
    } else {
        nr = (nr + H) % H;
        nc = (nc + L) % L;
    }
    return (int64_t)nr * L + nc;
}

static int check_variant(const orc_variant* v)
{
    if (!v) return 0;
    if (v->neighbourhood != 4 && v->neighbourhood != 8) return -1;
    if (v->reflect != 0 && v->reflect != 1) return -1;
    if (v->height < 0) return -1;
    return 0;
}

static int check_common(int32_t S, const uint8_t* D)
{
    if (S < 1 || S > 255 || !D) return -1;
    for (int32_t i = 0; i < S; ++i)
        for (int32_t j = 0; j < S; ++j)
            if (D[i * S + j] > 1) return -1;
    return 0;
}

static int check_prob(int32_t S, const double* Pd)
{
    if (!Pd) return 0;
    for (int32_t i = 0; i < S * S; ++i)
        if (!(Pd[i] >= 0.0 && Pd[i] <= 1.0)) return -1;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Random-sequential oracle (Alg. 3 + Alg. 4).  Its random stream: Philox
 * keyed by the seed, counters (j, stream, mcs, TAG_RS), consumed one 32-bit
 * word at a time. */
typedef struct {
    uint64_t seed;
    uint32_t stream, mcs, j;
    uint32_t buf[4];
    int pos;
} rs_stream;

static uint32_t rs_next(rs_stream* s)
{
    if (s->pos == 4) {
        philox_at(s->seed, s->j++, s->stream, s->mcs, TAG_RS, s->buf);
        s->pos = 0;
    }
    return s->buf[s->pos++];
}

/* Uniform integer in [0, n), Lemire's multiply-and-reject method (ACM TOMACS
 * 2019): unbiased. */
static uint32_t rs_bounded(rs_stream* s, uint32_t n)
{
    uint64_t m = (uint64_t)rs_next(s) * n;
    uint32_t l = (uint32_t)m;
    if (l < n) {
        uint32_t t = (0u - n) % n;
        while (l < t) {
            m = (uint64_t)rs_next(s) * n;
            l = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

/* Uniform double in [0, 1) with 53 random bits. */
static double rs_unit(rs_stream* s)
{
    uint64_t a = rs_next(s) >> 5, b = rs_next(s) >> 6;
    return (double)(a * 67108864u + b) * (1.0 / 9007199254740992.0);
}

int orc_rs_attempts(int32_t L, int32_t H, int32_t S, const uint8_t* D,
                    double I, double P, double X, uint64_t seed, uint32_t stream,
                    uint32_t mcs, int64_t n_attempts, uint8_t* lattice)
{
    return orc_rs_attempts_p(L, H, S, D, NULL, I, P, X, seed, stream, mcs, n_attempts, lattice);
}

int orc_rs_attempts_p(int32_t L, int32_t H, int32_t S, const uint8_t* D, const double* Pd,
                      double I, double P, double X, uint64_t seed, uint32_t stream,
                      uint32_t mcs, int64_t n_attempts, uint8_t* lattice)
{
    orc_variant v = {4, 0, Pd, 0};
    return orc_rs_attempts_v(L, H, S, D, &v, I, P, X, seed, stream, mcs, n_attempts, lattice);
}

int orc_rs_attempts_v(int32_t L, int32_t H, int32_t S, const uint8_t* D, const orc_variant* var,
                      double I, double P, double X, uint64_t seed, uint32_t stream,
                      uint32_t mcs, int64_t n_attempts, uint8_t* lattice)
{
    const double* Pd = var ? var->prob : NULL;
    const int32_t nb = var ? var->neighbourhood : 4, reflect = var ? var->reflect : 0;
    if (L < 3 || H < 3 || check_common(S, D) || check_prob(S, Pd) || check_variant(var) || !lattice ||
        n_attempts < 0)
        return -1;
    if (!(I >= 0.0) || !(P >= 0.0) || !(X >= 0.0)) return -1;
    double R = X + I + P;          /* mu + sigma + epsilon, normalised below */
    if (!(R > 0.0)) return -1;
    int64_t N = (int64_t)L * H;
    if (N > 0xFFFFFFFFll) return -1;
    rs_stream s = {seed, stream, mcs, 0, {0, 0, 0, 0}, 4};
    for (int64_t n = 0; n < n_attempts; ++n) {
        uint32_t i = rs_bounded(&s, (uint32_t)N);          /* random cell */
        uint32_t dir = rs_bounded(&s, (uint32_t)nb);        /* von Neumann or Moore direction */
        double r = rs_unit(&s) * R;                         /* action draw in [0, R) */
        int32_t row = (int32_t)(i / (uint32_t)L), col = (int32_t)(i % (uint32_t)L);
        int64_t ni = neighbour_v(L, H, row, col, (int32_t)dir, reflect);
        int32_t action;
        if (r < X)
            action = ORC_EXCHANGE;
        else if (r < X + I)
            /* the draw's position inside the interaction band is a fresh
               uniform: the interaction happens with the edge's probability */
            action = (r < X + orc_pair_prob(lattice[i], lattice[ni], S, D, Pd) * I) ? ORC_INTERACT
                                                                                  : ORC_INTERACT_FAIL;
        else
            action = ORC_REPRODUCE;
        orc_rule(action, S, D, &lattice[i], &lattice[ni]);
    }
    return 0;
}

int orc_rs_run(int32_t L, int32_t H, int32_t S, const uint8_t* D,
               double I, double P, double X, uint64_t seed, uint32_t stream,
               uint32_t mcs_begin, uint32_t n_mcs, uint8_t* lattice)
{
    return orc_rs_run_p(L, H, S, D, NULL, I, P, X, seed, stream, mcs_begin, n_mcs, lattice);
}

int orc_rs_run_p(int32_t L, int32_t H, int32_t S, const uint8_t* D, const double* Pd,
                 double I, double P, double X, uint64_t seed, uint32_t stream,
                 uint32_t mcs_begin, uint32_t n_mcs, uint8_t* lattice)
{
    orc_variant v = {4, 0, Pd, 0};
    return orc_rs_run_v(L, H, S, D, &v, I, P, X, seed, stream, mcs_begin, n_mcs, lattice);
}

int orc_rs_run_v(int32_t L, int32_t H, int32_t S, const uint8_t* D, const orc_variant* var,
                 double I, double P, double X, uint64_t seed, uint32_t stream,
                 uint32_t mcs_begin, uint32_t n_mcs, uint8_t* lattice)
{
    int64_t N = (int64_t)L * H;
    for (uint32_t k = 0; k < n_mcs; ++k) {
        int rc = orc_rs_attempts_v(L, H, S, D, var, I, P, X, seed, stream, mcs_begin + k, N, lattice);
        if (rc) return rc;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Schedule v1: partition. */
static void split_even(int32_t n, int32_t parts, int32_t* start)
{
    int32_t q = n / parts, r = n % parts;
    start[0] = 0;
    for (int32_t k = 0; k < parts; ++k) start[k + 1] = start[k] + q + (k < r ? 1 : 0);
}

static int32_t v1_coarse_segments(int32_t L)
{
    int32_t h = (L + 64) / 128;
    return 2 * (h < 1 ? 1 : h);
}

static int32_t v1_fine_segments(int32_t w) { return 2 * (w / 4); }

int orc_v1_partition(int32_t L, int32_t* P_out, int32_t* GQ_out,
                     int32_t* coarse_start, int32_t* fine_start, int32_t* fine_of_coarse)
{
    if (L < 8 || L > 65535) return -1;
    int32_t P = v1_coarse_segments(L);
    int32_t* cs = (int32_t*)malloc(sizeof(int32_t) * (P + 1));
    split_even(L, P, cs);
    int32_t GQ = 0;
    for (int32_t k = 0; k < P; ++k) GQ += v1_fine_segments(cs[k + 1] - cs[k]);
    if (P_out) *P_out = P;
    if (GQ_out) *GQ_out = GQ;
    if (coarse_start) memcpy(coarse_start, cs, sizeof(int32_t) * (P + 1));
    if (fine_start || fine_of_coarse) {
        int32_t g = 0;
        for (int32_t k = 0; k < P; ++k) {
            int32_t w = cs[k + 1] - cs[k], Q = v1_fine_segments(w);
            int32_t* fs = (int32_t*)malloc(sizeof(int32_t) * (Q + 1));
            split_even(w, Q, fs);
            if (fine_of_coarse) fine_of_coarse[k] = g;
            for (int32_t q = 0; q < Q; ++q)
                if (fine_start) fine_start[g + q] = cs[k] + fs[q];
            g += Q;
            free(fs);
        }
        if (fine_start) fine_start[GQ] = L;
        if (fine_of_coarse) fine_of_coarse[P] = GQ;
    }
    free(cs);
    return 0;
}

int orc_v1_cycles(int32_t L, int32_t* G_out, int32_t* F_out)
{
    if (L < 8) return -1;
    /* One coarse cycle and one fine cycle per MCS for every L: each fine
     * sub-block performs all of its n_k attempts of the MCS in one visit. */
    *G_out = 1;
    *F_out = 1;
    return 0;
}

/* The 24 orderings of the four colours, in lexicographic order. */
static void colour_orders(uint8_t perms[24][4])
{
    int n = 0;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            for (int c = 0; c < 4; ++c)
                for (int d = 0; d < 4; ++d)
                    if (a != b && a != c && a != d && b != c && b != d && c != d) {
                        perms[n][0] = (uint8_t)a; perms[n][1] = (uint8_t)b;
                        perms[n][2] = (uint8_t)c; perms[n][3] = (uint8_t)d;
                        ++n;
                    }
}

int orc_init(int32_t L, int32_t S, double p_empty, uint64_t seed, uint8_t* lattice)
{
    return orc_init_rect(L, L, S, p_empty, seed, lattice);
}

int orc_init_rect(int32_t L, int32_t H, int32_t S, double p_empty, uint64_t seed, uint8_t* lattice)
{
    if (L < 1 || H < 1 || S < 1 || S > 255 || !lattice || !(p_empty >= 0.0) || p_empty > 1.0) return -1;
    uint64_t TE = (uint64_t)floor(ldexp(p_empty, 32) + 0.5);
    int64_t N = (int64_t)L * H;
    if (N > 0xFFFFFFFFll) return -1;
    for (int64_t i = 0; i < N; ++i) {
        uint32_t x[4];
        philox_at(seed, (uint32_t)i, 0, 0, TAG_INIT, x);
        lattice[i] = ((uint64_t)x[0] < TE) ? 0 : (uint8_t)(1 + umulhi32(x[1], (uint32_t)S));
    }
    return 0;
}

/* splitmix-style index shuffle used only to permute independent work. */
static uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void shuffle_ints(int32_t* v, int32_t n, uint64_t* state)
{
    for (int32_t k = n - 1; k > 0; --k) {
        *state = mix64(*state);
        int32_t j = (int32_t)(*state % (uint64_t)(k + 1));
        int32_t t = v[k]; v[k] = v[j]; v[j] = t;
    }
}

int orc_replay_run(int32_t L, int32_t S, const uint8_t* D,
                   double I, double P, double X, uint64_t seed,
                   int32_t G, int32_t F, uint32_t mcs_begin, uint32_t n_mcs,
                   uint8_t* lattice, uint32_t flags, uint64_t shuffle_seed,
                   orc_trace_rec* trace, int64_t trace_cap, int64_t* attempts_out)
{
    return orc_replay_run_p(L, S, D, NULL, I, P, X, seed, G, F, mcs_begin, n_mcs, lattice, flags,
                            shuffle_seed, trace, trace_cap, attempts_out);
}

int orc_replay_run_p(int32_t L, int32_t S, const uint8_t* D, const double* Pd,
                     double I, double P, double X, uint64_t seed,
                     int32_t G, int32_t F, uint32_t mcs_begin, uint32_t n_mcs,
                     uint8_t* lattice, uint32_t flags, uint64_t shuffle_seed,
                     orc_trace_rec* trace, int64_t trace_cap, int64_t* attempts_out)
{
    orc_variant v = {4, 0, Pd, 0};
    return orc_replay_run_v(L, S, D, &v, I, P, X, seed, G, F, mcs_begin, n_mcs, lattice, flags,
                            shuffle_seed, trace, trace_cap, attempts_out);
}

int orc_replay_run_v(int32_t L, int32_t S, const uint8_t* D, const orc_variant* var,
                     double I, double P, double X, uint64_t seed,
                     int32_t G, int32_t F, uint32_t mcs_begin, uint32_t n_mcs,
                     uint8_t* lattice, uint32_t flags, uint64_t shuffle_seed,
                     orc_trace_rec* trace, int64_t trace_cap, int64_t* attempts_out)
{
    const double* Pd = var ? var->prob : NULL;
    const uint32_t nbh = var ? (uint32_t)var->neighbourhood : 4u;   /* directions */
    const int32_t reflect = var ? var->reflect : 0;
    const int32_t H = (var && var->height) ? var->height : L;         /* rows */
    if (L < 8 || L > 65535 || H < 8 || H > 65535 || check_common(S, D) || check_prob(S, Pd) ||
        check_variant(var) || !lattice || G < 1 || F < 1)
        return -1;
    if ((uint64_t)mcs_begin + n_mcs > 0xFFFFFFFFull) return -1;
    uint64_t TX, TXI;
    if (orc_thresholds(I, P, X, &TX, &TXI)) return -1;
    /* interaction happens iff u < TP[a][b] (TX <= TP <= TXI) */
    const int32_t s1 = S + 1;
    uint64_t* TP = (uint64_t*)malloc(sizeof(uint64_t) * s1 * s1);
    for (int32_t a = 0; a < s1; ++a)
        for (int32_t b = 0; b < s1; ++b)
            TP[a * s1 + b] = orc_interaction_threshold(TX, TXI, orc_pair_prob(a, b, S, D, Pd));

    /* each axis partitioned on its own: columns (L) and rows (H) */
    int32_t Pc, GQ, Pr, GQr;
    orc_v1_partition(L, &Pc, &GQ, NULL, NULL, NULL);
    orc_v1_partition(H, &Pr, &GQr, NULL, NULL, NULL);
    int32_t* cs = (int32_t*)malloc(sizeof(int32_t) * (Pc + 1));
    int32_t* fs = (int32_t*)malloc(sizeof(int32_t) * (GQ + 1));
    int32_t* fc = (int32_t*)malloc(sizeof(int32_t) * (Pc + 1));
    orc_v1_partition(L, NULL, NULL, cs, fs, fc);
    int32_t* rcs = (int32_t*)malloc(sizeof(int32_t) * (Pr + 1));
    int32_t* rfs = (int32_t*)malloc(sizeof(int32_t) * (GQr + 1));
    int32_t* rfc = (int32_t*)malloc(sizeof(int32_t) * (Pr + 1));
    orc_v1_partition(H, NULL, NULL, rcs, rfs, rfc);

    uint8_t perms[24][4];
    colour_orders(perms);
    const int32_t V = G * F;
    int32_t* blocks = (int32_t*)malloc(sizeof(int32_t) * Pc * Pr);
    int32_t* subs = (int32_t*)malloc(sizeof(int32_t) * GQ * GQr);
    uint64_t shuf = shuffle_seed;
    int64_t attempts = 0, nrec = 0;
    uint32_t coarse_phase = 0, fine_phase = 0;

    for (uint32_t mi = 0; mi < n_mcs; ++mi) {
        uint32_t m = mcs_begin + mi;
        for (int32_t gc = 0; gc < G; ++gc) {
            uint32_t x[4];
            philox_at(seed, (uint32_t)gc, 0, m, TAG_ORDER, x);
            const uint8_t* order = perms[umulhi32(x[0], 24)];
            for (int ci = 0; ci < 4; ++ci, ++coarse_phase) {
                int32_t colour = order[ci], nb = 0;
                for (int32_t by = 0; by < Pr; ++by)
                    for (int32_t bx = 0; bx < Pc; ++bx)
                        if (2 * (by & 1) + (bx & 1) == colour) blocks[nb++] = by * Pc + bx;
                if (flags & ORC_SHUFFLE_BLOCKS) shuffle_ints(blocks, nb, &shuf);
                for (int32_t bi = 0; bi < nb; ++bi) {
                    int32_t b = blocks[bi], by = b / Pc, bx = b % Pc;
                    for (int32_t f = 0; f < F; ++f) {
                        int32_t v = gc * F + f;
                        philox_at(seed, (uint32_t)v, (uint32_t)b, m, TAG_FORDER, x);
                        const uint8_t* forder = perms[umulhi32(x[0], 24)];
                        for (int fi = 0; fi < 4; ++fi, ++fine_phase) {
                            int32_t fcol = forder[fi], ns = 0;
                            for (int32_t gy = rfc[by]; gy < rfc[by + 1]; ++gy)
                                for (int32_t gx = fc[bx]; gx < fc[bx + 1]; ++gx)
                                    if (2 * (gy & 1) + (gx & 1) == fcol) subs[ns++] = gy * GQ + gx;
                            if (flags & ORC_SHUFFLE_SUBS) shuffle_ints(subs, ns, &shuf);
                            for (int32_t si = 0; si < ns; ++si) {
                                int32_t g = subs[si], gy = g / GQ, gx = g % GQ;
                                int32_t x0 = fs[gx], wx = fs[gx + 1] - fs[gx];
                                int32_t y0 = rfs[gy], wy = rfs[gy + 1] - rfs[gy];
                                uint32_t nk = (uint32_t)(wx * wy);
                                uint32_t t0 = (uint32_t)(((uint64_t)v * nk) / V);
                                uint32_t t1 = (uint32_t)(((uint64_t)(v + 1) * nk) / V);
                                for (uint32_t t = t0; t < t1; ++t) {
                                    uint32_t w4[4];
                                    philox_at(seed, t >> 2, (uint32_t)g, m, TAG_STEP, w4);
                                    uint32_t w = w4[t & 3];
                                    /* p = w * (nb * n_g): the high word picks the cell and
                                       the direction, the low word is the action draw */
                                    uint64_t prod = (uint64_t)w * (nbh * nk);
                                    uint32_t hi = (uint32_t)(prod >> 32), u = (uint32_t)prod;
                                    uint32_t site = hi / nbh, dir = hi % nbh;
                                    int32_t row = y0 + (int32_t)(site / (uint32_t)wx);
                                    int32_t col = x0 + (int32_t)(site % (uint32_t)wx);
                                    int64_t i = (int64_t)row * L + col;
                                    int64_t j = neighbour_v(L, H, row, col, (int32_t)dir, reflect);
                                    int32_t action = ((uint64_t)u < TX)    ? ORC_EXCHANGE
                                                     : ((uint64_t)u < TXI) ? ORC_INTERACT
                                                                           : ORC_REPRODUCE;
                                    if (action == ORC_INTERACT && (uint64_t)u >= TP[lattice[i] * s1 + lattice[j]])
                                        action = ORC_INTERACT_FAIL;
                                    orc_rule(action, S, D, &lattice[i], &lattice[j]);
                                    if (trace && nrec < trace_cap) {
                                        orc_trace_rec* r = &trace[nrec++];
                                        r->mcs = m; r->coarse_phase = coarse_phase;
                                        r->fine_phase = fine_phase; r->block = (uint32_t)b;
                                        r->sub = (uint32_t)g; r->t = t;
                                        r->site = (uint32_t)i; r->nbr = (uint32_t)j;
                                        r->dir = (uint8_t)dir; r->action = (uint8_t)action;
                                        r->pad[0] = r->pad[1] = 0;
                                    }
                                    ++attempts;
                                }
                            }
                        }
                    }
                }
            }
        }
    }
    free(cs); free(fs); free(fc); free(rcs); free(rfs); free(rfc); free(blocks); free(subs); free(TP);
    if (attempts_out) *attempts_out = attempts;
    return 0;
}

/* ------------------------------------------------------------------------ */
static int alive_species(const uint64_t* counts, int32_t S)
{
    int alive = 0;
    for (int32_t s = 1; s <= S; ++s) alive += counts[s] > 0;
    return alive;
}

int orc_run_observed(int32_t use_rs, int32_t L, int32_t S, const uint8_t* D,
                     double I, double P, double X, uint64_t seed,
                     uint32_t mcs_begin, uint32_t n_mcs, uint32_t log_every,
                     int32_t stop_at_extinction, uint8_t* lattice,
                     uint64_t* counts_log, int64_t log_cap, int64_t* n_logged,
                     uint32_t* mcs_end)
{
    return orc_run_observed_p(use_rs, L, S, D, NULL, I, P, X, seed, mcs_begin, n_mcs, log_every,
                              stop_at_extinction, lattice, counts_log, log_cap, n_logged, mcs_end);
}

int orc_run_observed_p(int32_t use_rs, int32_t L, int32_t S, const uint8_t* D, const double* Pd,
                       double I, double P, double X, uint64_t seed,
                       uint32_t mcs_begin, uint32_t n_mcs, uint32_t log_every,
                       int32_t stop_at_extinction, uint8_t* lattice,
                       uint64_t* counts_log, int64_t log_cap, int64_t* n_logged,
                       uint32_t* mcs_end)
{
    orc_variant v = {4, 0, Pd, 0};
    return orc_run_observed_v(use_rs, L, S, D, &v, I, P, X, seed, mcs_begin, n_mcs, log_every,
                              stop_at_extinction, lattice, counts_log, log_cap, n_logged, mcs_end);
}

int orc_run_observed_v(int32_t use_rs, int32_t L, int32_t S, const uint8_t* D, const orc_variant* var,
                       double I, double P, double X, uint64_t seed,
                       uint32_t mcs_begin, uint32_t n_mcs, uint32_t log_every,
                       int32_t stop_at_extinction, uint8_t* lattice,
                       uint64_t* counts_log, int64_t log_cap, int64_t* n_logged,
                       uint32_t* mcs_end)
{
    if (log_every == 0 || !lattice) return -1;
    int32_t G, F;
    if (orc_v1_cycles(L, &G, &F)) return -1;
    const int32_t H = (var && var->height) ? var->height : L;
    int64_t N = (int64_t)L * H, nl = 0;
    uint64_t* c = (uint64_t*)malloc(sizeof(uint64_t) * (S + 1));
    uint32_t m = mcs_begin;
    int rc = 0;
    for (;;) {
        if (m % log_every == 0) {
            orc_counts(N, lattice, S, c);
            if (counts_log && nl < log_cap) memcpy(counts_log + nl * (S + 1), c, sizeof(uint64_t) * (S + 1));
            ++nl;
            if (stop_at_extinction && alive_species(c, S) <= 1) break;
        }
        if (m == mcs_begin + n_mcs) break;
        rc = use_rs ? orc_rs_run_v(L, H, S, D, var, I, P, X, seed, 0, m, 1, lattice)
                    : orc_replay_run_v(L, S, D, var, I, P, X, seed, G, F, m, 1, lattice, 0, 0, NULL, 0, NULL);
        if (rc) break;
        ++m;
    }
    free(c);
    if (n_logged) *n_logged = nl;
    if (mcs_end) *mcs_end = m;
    return rc;
}
