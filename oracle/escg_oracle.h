/*
 * escg_oracle.h -- plain, single-threaded CPU oracle for the Evolutionary
 * Spatial Cyclic Game (ESCG) Monte Carlo step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library
 * and its Python binding) includes, links or calls this code.  It is used by
 * tests/, by __graft_entry__.smoke() and by the cpu_baseline leg of bench.py.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Two oracles live here:
 *   - the random-sequential (RS) oracle: Alg. 3 ("Elementary Step") and
 *     Alg. 4 ("Overall ESCG Loop") of the paper, literally: N = L*H elementary
 *     steps per MCS, each at a uniformly drawn site, direction and action;
 *   - the replay oracle: the coloured two-level sublattice schedule (version 1)
 *     executed serially, one attempt after another, in the schedule's order.
 *     The GPU path must reproduce its lattice bit for bit.
 *
 * Conventions (paper, Section 3.1 "Implementation"): lattice values are
 * 0 = empty, 1..S = species; index = row*L + col; the dominance matrix is
 * S*S row-major with D[(a-1)*S + (b-1)] = 1 iff species a dominates b.
 * Directions: 0 up (row-1), 1 down (row+1), 2 left (col-1), 3 right (col+1),
 * in the order the paper lists the periodic neighbours.
 *
 * All functions return 0 on success and a negative value on bad arguments.
 */
#ifndef ESCG_ORACLE_H
#define ESCG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
 *      as easy as 1, 2, 3", SC'11): counter-based generator. ---- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* n independent evaluations: ctr is n x 4, key is n x 2, out is n x 4. */
void orc_philox_many(int64_t n, const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* ---- Dominance (Section 3.1, circulant definition and Alg. 2) ---- */
/* D[i*S + j] = 1 iff (j - i + S) mod S is in K (species indices 0-based). */
int orc_circulant(int32_t S, const int32_t* K, int32_t nK, uint8_t* D);
/* Alg. 2: false if either site is empty, else D[(a-1)*S + (b-1)] == 1. */
int orc_dominates(int32_t a, int32_t b, int32_t S, const uint8_t* D);

/* Action codes, in the order Alg. 3 tests them; ORC_INTERACT_FAIL is an
 * interaction across a probabilistic edge that did not take place. */
enum { ORC_EXCHANGE = 0, ORC_INTERACT = 1, ORC_REPRODUCE = 2, ORC_INTERACT_FAIL = 3 };
/* Alg. 3 applied to the pair (selected site a, neighbour b) for a given
 * action; a and b are updated in place. */
void orc_rule(int32_t action, int32_t S, const uint8_t* D, uint8_t* a, uint8_t* b);

/* epsilon = 2 M N (Section 3.1, rate initialisation). */
double orc_exchange_from_mobility(double M, int64_t N);

/* Integer thresholds on a 32-bit draw u (schedule v1): exchange iff
 * u < TX, interaction iff TX <= u < TXI, reproduction otherwise, with
 * R = (X + I) + P, TX = floor(2^32 X/R + 1/2), TXI = floor(2^32 (X+I)/R + 1/2). */
int orc_thresholds(double I, double P, double X, uint64_t* TX, uint64_t* TXI);

/* Probabilistic dominance (Park, Chen and Szolnoki's model, Section "Park,
 * Chen, Szolnoki"): Pd is S*S row-major, Pd[(a-1)*S + (b-1)] = probability
 * that an interaction across the edge a -> b (D[(a-1)*S + (b-1)] = 1) takes
 * place; NULL means every edge is certain.  orc_pair_prob returns the
 * probability that applies to the pair (selected a, neighbour b): that of
 * the edge between them, whichever its direction, else 1.
 * Random-sequential oracle: an interaction draw r in [X, X+I) takes place iff
 * r < X + p*I.  Schedule v1: iff u < orc_interaction_threshold(TX, TXI, p)
 * = TX + floor((TXI - TX) * q / 2^32 + 1/2), q = floor(p * 2^32 + 1/2), in
 * exact integer arithmetic (p = 0 gives TX, p = 1 gives TXI). */
double orc_pair_prob(int32_t a, int32_t b, int32_t S, const uint8_t* D, const double* Pd);
uint64_t orc_interaction_threshold(uint64_t TX, uint64_t TXI, double p);

/* Rule variant (the paper's --neighbourhood and --flux options): a
 * neighbourhood of 4 (von Neumann) or 8 (Moore) directions -- 0 up, 1 down,
 * 2 left, 3 right, 4 up-left, 5 up-right, 6 down-left, 7 down-right -- and
 * a periodic ("flux") or reflecting boundary (a step that would leave the
 * lattice is mirrored back), with optional edge probabilities.  In the
 * schedule an attempt's word w gives p = w * (neighbourhood * n_g): cell =
 * floor(hi / neighbourhood), direction = hi mod neighbourhood. */
typedef struct {
    int32_t neighbourhood;   /* 4 or 8 */
    int32_t reflect;         /* 0 periodic, 1 reflecting */
    const double* prob;      /* S*S edge probabilities or NULL */
    int32_t height;          /* rows H of an L x H lattice (the paper's --length
                                and --height); 0: H = L.  The schedule
                                partitions columns and rows independently
                                (Pc x Pr blocks, block id by*Pc + bx, sub-block
                                id gy*GQ + gx with GQ the column count). */
} orc_variant;

/* Histogram of lattice values 0..S (Alg. 4 densities(), as counts). */
int orc_counts(int64_t n, const uint8_t* lattice, int32_t S, uint64_t* counts);

/* ---- Random-sequential oracle (Alg. 3 + Alg. 4) ---- */
/* Performs n_attempts elementary steps of MCS number `mcs` on an L x H
 * periodic lattice (L columns, H rows).  The random stream of MCS `mcs` is
 * Philox keyed by seed with counters (j, stream, mcs, 5), j = 0, 1, ...,
 * consumed word by word; each attempt draws a site by Lemire's unbiased
 * bounded-integer method, a direction from 2 bits and r = U*(X+I+P) with a
 * 53-bit U in [0,1), in fp64.  Per-attempt action: r < X exchange,
 * r < X+I interaction, else reproduction (Alg. 3). */
int orc_rs_attempts(int32_t L, int32_t H, int32_t S, const uint8_t* D,
                    double I, double P, double X, uint64_t seed, uint32_t stream,
                    uint32_t mcs, int64_t n_attempts, uint8_t* lattice);
/* n_mcs full MCS (N attempts each) starting at MCS number mcs_begin. */
int orc_rs_run(int32_t L, int32_t H, int32_t S, const uint8_t* D,
               double I, double P, double X, uint64_t seed, uint32_t stream,
               uint32_t mcs_begin, uint32_t n_mcs, uint8_t* lattice);
/* The same with edge probabilities Pd (may be NULL). */
int orc_rs_attempts_p(int32_t L, int32_t H, int32_t S, const uint8_t* D, const double* Pd,
                      double I, double P, double X, uint64_t seed, uint32_t stream,
                      uint32_t mcs, int64_t n_attempts, uint8_t* lattice);
int orc_rs_run_p(int32_t L, int32_t H, int32_t S, const uint8_t* D, const double* Pd,
                 double I, double P, double X, uint64_t seed, uint32_t stream,
                 uint32_t mcs_begin, uint32_t n_mcs, uint8_t* lattice);
/* The same for a rule variant (NULL: von Neumann, periodic, certain edges). */
int orc_rs_attempts_v(int32_t L, int32_t H, int32_t S, const uint8_t* D, const orc_variant* var,
                      double I, double P, double X, uint64_t seed, uint32_t stream,
                      uint32_t mcs, int64_t n_attempts, uint8_t* lattice);
int orc_rs_run_v(int32_t L, int32_t H, int32_t S, const uint8_t* D, const orc_variant* var,
                 double I, double P, double X, uint64_t seed, uint32_t stream,
                 uint32_t mcs_begin, uint32_t n_mcs, uint8_t* lattice);

/* ---- Schedule v1 (coloured two-level sublattice), replay oracle ---- */
/* Coarse partition of one axis: P segments (P even); fine partition: GQ
 * segments in total.  coarse_start has P+1 entries, fine_start GQ+1,
 * fine_of_coarse P+1 (first global fine index of each coarse segment). */
int orc_v1_partition(int32_t L, int32_t* P_out, int32_t* GQ_out,
                     int32_t* coarse_start, int32_t* fine_start, int32_t* fine_of_coarse);
/* Coarse cycles G and fine cycles F per MCS that version 1 fixes for L. */
int orc_v1_cycles(int32_t L, int32_t* G_out, int32_t* F_out);

/* Initialisation (schedule v1): site i gets x = Philox(seed, (i, 0, 0, 1));
 * empty iff x0 < floor(2^32 p_empty + 1/2), else 1 + floor(x1 * S / 2^32). */
int orc_init(int32_t L, int32_t S, double p_empty, uint64_t seed, uint8_t* lattice);
/* The same for L columns and H rows (site i = row*L + col). */
int orc_init_rect(int32_t L, int32_t H, int32_t S, double p_empty, uint64_t seed, uint8_t* lattice);

/* Trace record of one attempt (for structural tests on small lattices). */
typedef struct {
    uint32_t mcs, coarse_phase, fine_phase, block;
    uint32_t sub, t, site, nbr;
    uint8_t dir, action, pad[2];
} orc_trace_rec;

enum {
    ORC_SHUFFLE_BLOCKS = 1,   /* visit the blocks of a coarse phase in a random order */
    ORC_SHUFFLE_SUBS = 2      /* visit the sub-blocks of a fine phase in a random order */
};

/* Runs n_mcs MCS of schedule v1 with G coarse and F fine cycles starting at
 * MCS number mcs_begin.  flags/shuffle_seed only permute the order of
 * independent work inside a phase (which must not change the result).
 * If trace != NULL, up to trace_cap attempts are recorded.  attempts_out
 * (may be NULL) receives the number of elementary steps performed. */
int orc_replay_run(int32_t L, int32_t S, const uint8_t* D,
                   double I, double P, double X, uint64_t seed,
                   int32_t G, int32_t F, uint32_t mcs_begin, uint32_t n_mcs,
                   uint8_t* lattice, uint32_t flags, uint64_t shuffle_seed,
                   orc_trace_rec* trace, int64_t trace_cap, int64_t* attempts_out);
/* The same with edge probabilities Pd (may be NULL), or a rule variant. */
int orc_replay_run_v(int32_t L, int32_t S, const uint8_t* D, const orc_variant* var,
                     double I, double P, double X, uint64_t seed,
                     int32_t G, int32_t F, uint32_t mcs_begin, uint32_t n_mcs,
                     uint8_t* lattice, uint32_t flags, uint64_t shuffle_seed,
                     orc_trace_rec* trace, int64_t trace_cap, int64_t* attempts_out);
int orc_replay_run_p(int32_t L, int32_t S, const uint8_t* D, const double* Pd,
                     double I, double P, double X, uint64_t seed,
                     int32_t G, int32_t F, uint32_t mcs_begin, uint32_t n_mcs,
                     uint8_t* lattice, uint32_t flags, uint64_t shuffle_seed,
                     orc_trace_rec* trace, int64_t trace_cap, int64_t* attempts_out);

/* Run with observation: counts after every log_every-th MCS (absolute MCS
 * number a multiple of log_every) are appended to counts_log
 * ((S+1) per entry, up to log_cap entries), and, if stop_at_extinction,
 * the run ends after the first such MCS at which at most one non-empty
 * species has a nonzero count.  *mcs_end receives the final MCS number.
 * use_rs selects the random-sequential oracle instead of the replay. */
int orc_run_observed(int32_t use_rs, int32_t L, int32_t S, const uint8_t* D,
                     double I, double P, double X, uint64_t seed,
                     uint32_t mcs_begin, uint32_t n_mcs, uint32_t log_every,
                     int32_t stop_at_extinction, uint8_t* lattice,
                     uint64_t* counts_log, int64_t log_cap, int64_t* n_logged,
                     uint32_t* mcs_end);
int orc_run_observed_v(int32_t use_rs, int32_t L, int32_t S, const uint8_t* D, const orc_variant* var,
                       double I, double P, double X, uint64_t seed,
                       uint32_t mcs_begin, uint32_t n_mcs, uint32_t log_every,
                       int32_t stop_at_extinction, uint8_t* lattice,
                       uint64_t* counts_log, int64_t log_cap, int64_t* n_logged,
                       uint32_t* mcs_end);
int orc_run_observed_p(int32_t use_rs, int32_t L, int32_t S, const uint8_t* D, const double* Pd,
                       double I, double P, double X, uint64_t seed,
                       uint32_t mcs_begin, uint32_t n_mcs, uint32_t log_every,
                       int32_t stop_at_extinction, uint8_t* lattice,
                       uint64_t* counts_log, int64_t log_cap, int64_t* n_logged,
                       uint32_t* mcs_end);

#ifdef __cplusplus
}
#endif
#endif
