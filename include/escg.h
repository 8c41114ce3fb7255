/*
 * escg.h -- C ABI of libescg, a GB300 (sm_103a) implementation of the Monte
 * Carlo step (MCS) of an Evolutionary Spatial Cyclic Game (ESCG) on an L x L
 * periodic von Neumann lattice (arXiv 2508.16639); options add L x H
 * rectangles, the Moore neighbourhood, a reflecting boundary, probabilistic
 * dominance edges and bit-packed device storage (escg_options).
 *
 * The model (Section 3.1 "Implementation" of the paper): lattice value 0 is
 * an empty site, 1..S a species; species a dominates species b iff
 * digraph[(a-1)*S + (b-1)] == 1 (Alg. 2, "Dominance Check"; the circulant
 * C(S,K) definition gives RPS = C(3,{1}) and RPSLS = C(5,{1,2})).  One MCS is
 * N = L*L elementary steps (Alg. 4, "Overall ESCG Loop"); an elementary step
 * (Alg. 3, "Elementary Step") picks a site and one of its four neighbours
 * and applies, with probabilities proportional to the rates, exchange
 * (migration, epsilon), interaction (mu: the dominated one of the pair
 * becomes empty) or reproduction (sigma: an occupied site fills an empty
 * neighbour).  epsilon = 2 M N for mobility M (Section 3.1, rate set-up).
 *
 * Parallel order.  The N elementary steps of an MCS run in the race-free
 * order of schedule version 1: the lattice is cut into an even number P of
 * coarse blocks per axis (about 64 sites wide) coloured 2x2, each block into
 * fine sub-blocks of 2..4 sites per axis coloured 2x2; the four coarse
 * colours run one after another in a per-MCS random order, and inside a
 * block the four fine colours likewise, every sub-block performing all of
 * its attempts of the MCS in one visit.  Every random choice (colour orders,
 * cell, direction, action) is a Philox4x32-10 draw keyed by the seed and
 * counted by (attempt, sub-block, MCS), compared against integer
 * thresholds.  Results are deterministic: the lattice after m MCS depends
 * only on (L, S, digraph, rates, seed, initial lattice, m), never on the
 * device, stream, launch shape or on other lattices in a batch.
 *
 * Conventions.
 *   - All functions except escg_create*, escg_batch_create and the
 *     escg_server constructors return an escg_status; 0 is success.
 *   - Host pointers passed in are read during the call only (copied, never
 *     retained).  Output buffers are caller-owned.
 *   - Handles are not thread-safe: one thread at a time per handle.
 *   - escg_last_error() returns a thread-local message for the last failure.
 *   - Work is enqueued on the handle's CUDA stream; calls that return data
 *     to the host synchronise that stream first.
 */
#ifndef ESCG_H
#define ESCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ESCG_OK = 0,
    ESCG_EINVAL = -1,   /* bad argument (message in escg_last_error)      */
    ESCG_ENOMEM = -2,   /* device or host allocation failed               */
    ESCG_ECUDA = -3,    /* a CUDA runtime call failed                     */
    ESCG_ESTATE = -4,   /* call not valid in the handle's current state   */
    ESCG_ETIMEOUT = -5  /* a bounded device-side wait gave up             */
} escg_status;

/* Rates by role: interaction (the paper's mu), reproduction (sigma),
 * exchange (epsilon).  Each >= 0, sum > 0.  Only their ratios matter. */
typedef struct {
    double interact;
    double reproduce;
    double exchange;
} escg_rates;

typedef struct {
    double p_empty;              /* initial empty-site probability, [0,1]      */
    uint32_t log_every;          /* counts kept every k MCS (0: default 10)    */
    int32_t stop_at_extinction;  /* stop at the first logged MCS with <= 1
                                    non-empty species alive (stasis())        */
    uint32_t schedule_version;   /* 0 or 1 (only version 1 exists)            */
    int32_t persistent;          /* 1: persistent dataflow launches (default;
                                    uniform partitions use the block owners
                                    of 5 from 3 x 3
                                    groups of blocks while they need at most
                                    3 CTAs per SM, generic
                                    partitions of 2 x 2 coarse blocks the
                                    whole-lattice residency of 4);
                                    2: same, uniform partitions staged by a
                                    TMA producer warp (warp-specialised);
                                    3: persistent, epoch flags only (no
                                    mailbox kernel);
                                    4: whole-lattice residency: one CTA keeps
                                    the lattice in shared memory for the
                                    whole launch (lattices with at most 8
                                    coarse blocks per axis whose image fits
                                    one CTA's shared memory, about 470 x 470;
                                    larger ones run as 3);
                                    5: block owners: one CTA per 2 x 2 group
                                    of 64 x 64 blocks keeps their tiles in
                                    shared memory for the whole launch and
                                    exchanges only boundary records (L and H
                                    multiples of 128, any bits_per_site,
                                    (L/128)(H/128) CTAs resident at once, so
                                    the launches of several handles take
                                    turns; other lattices run as 3);
                                    6: boundary mailbox: the work items of 3
                                    taken from a ticket counter, neighbours'
                                    edge and rim lines read from epoch-tagged
                                    records (same lattices as 5, no residency
                                    requirement; others run as 3);
                                    0: one launch per coarse phase            */
    void* cuda_stream;           /* cudaStream_t to enqueue on, or NULL for a
                                    stream owned by the handle                */
    void* device_lattice;        /* optional caller-owned device buffer of
                                    escg_lattice_bytes_rect(L, H) bytes (e.g. a torch
                                    tensor), 16-byte aligned (ESCG_EINVAL
                                    otherwise); NULL: the library allocates   */
    int32_t time_kernels;        /* 1: bracket every lattice-update launch with
                                    CUDA events on the handle's stream (read
                                    back with escg_kernel_time)               */
    int32_t ctas_per_sm;         /* persistent CTAs per SM (0: as many as fit);
                                    for the block owners (one CTA per group of
                                    2x2 blocks) the least packing: at least
                                    this many per SM, leaving the other SMs to
                                    other streams; physical mapping only,
                                    results unchanged                         */
    const double* dominance_prob;/* optional S*S row-major edge probabilities
                                    (Park, Chen and Szolnoki's probabilistic
                                    dominance, the paper's section "Park,
                                    Chen, Szolnoki"): entry (a-1)*S+(b-1) in
                                    [0,1] is the probability that an
                                    interaction across the edge a -> b takes
                                    place; read during creation; NULL: every
                                    edge certain.  An interaction draw u in
                                    [T_X, T_XI) takes place iff u < T_X +
                                    round((T_XI - T_X) round(p 2^32) / 2^32)  */
    int32_t neighbourhood;       /* 4 (von Neumann, default; 0 means 4) or 8
                                    (Moore): Alg. 3 draws the direction from
                                    [0, neighbourhood); the attempt's word w
                                    gives p = w * (neighbourhood * n_g), cell
                                    floor(hi / neighbourhood), direction hi mod
                                    neighbourhood (0 up, 1 down, 2 left,
                                    3 right, 4 up-left, 5 up-right, 6 down-
                                    left, 7 down-right)                       */
    int32_t reflecting_boundary; /* 1: a step that would leave the lattice is
                                    mirrored back (the paper's "reflect");
                                    0: periodic ("flux", default)             */
    int32_t height;              /* rows H of an L x H lattice (the paper's
                                    --length and --height; 8 <= H <= 16384;
                                    0: H = L).  N = L*H; each axis is
                                    partitioned on its own (P x Py coarse
                                    blocks, block id by*P + bx; sub-block id
                                    gy*GQ + gx, GQ fine segments along the
                                    columns); site i = row*L + col.  The
                                    lattice buffers of the calls below hold H
                                    rows of L (host) or pitch (device) bytes. */
    int32_t bits_per_site;       /* device storage of a site: 8 (one byte,
                                    default; 0 means 8), 4 or 2 (bit-packed
                                    rows: site c at bits [c*b, (c+1)*b) of the
                                    row, little endian; 2 needs S <= 3; packed
                                    needs L, H >= 64).  Kernels stage packed
                                    groups of 4 sites and work on one byte per
                                    site in shared memory; host buffers stay
                                    one byte per site (converted on the device
                                    through a byte image allocated on first
                                    use).  Results are identical for all three;
                                    the device buffer is H rows of
                                    escg_lattice_pitch_ex(L, b) bytes.        */
    int32_t autotune;            /* 1 (with persistent = 1): on the first
                                    handle of its (device, L, H, S,
                                    bits_per_site, neighbourhood, boundary),
                                    time every distinct launch mode and CTA
                                    count on a copy of the initial lattice
                                    (10 MCS of warm-up, 20 timed) and keep the
                                    fastest, cached for the process; later
                                    handles of that key take the cached
                                    choice.  Physical mapping only: results
                                    are those of every mode.  0: the size rule
                                    of persistent = 1 (default).             */
} escg_options;

typedef struct escg escg_t;

/* Fills *opt with defaults: p_empty 0, log_every 10, no stop, version 1,
 * persistent, library-owned stream and memory. */
void escg_default_options(escg_options* opt);

/* Bytes of device memory a lattice of side L occupies: L rows of pitch
 * escg_lattice_pitch(L) (L rounded up to 16) bytes; an L x H lattice: H
 * rows of that pitch. */
size_t escg_lattice_bytes(int32_t L);
size_t escg_lattice_bytes_rect(int32_t L, int32_t H);
/* Row pitch and bytes of an L x H lattice stored with bits_per_site bits per
 * site (8, 4 or 2; 0 means 8): ceil(L*b/8) rounded up to 16 bytes per row;
 * 0 for an invalid argument. */
int32_t escg_lattice_pitch_ex(int32_t L, int32_t bits_per_site);
size_t escg_lattice_bytes_ex(int32_t L, int32_t H, int32_t bits_per_site);
int32_t escg_lattice_pitch(int32_t L);

/* Creates a lattice of side L (8 <= L <= 16384) with S species
 * (2 <= S <= 15), dominance digraph (S*S row-major bytes in {0,1}, zero
 * diagonal), rates, and seed, and initialises it on the device: site i is
 * empty with probability p_empty, else a uniform species (schedule v1
 * initialisation).  Returns NULL on error (see escg_last_error). */
escg_t* escg_create(int32_t L, int32_t S, const uint8_t* digraph, const escg_rates* rates,
                    uint64_t seed);
escg_t* escg_create_ex(int32_t L, int32_t S, const uint8_t* digraph, const escg_rates* rates,
                       uint64_t seed, const escg_options* opt);

/* Enqueues n_mcs Monte Carlo steps (N elementary steps each).  Counts are
 * recorded after every MCS whose absolute number is a multiple of
 * log_every.  With stop_at_extinction the run ends at the first such MCS at
 * which at most one non-empty species is alive.  Asynchronous. */
int escg_run(escg_t* h, uint64_t n_mcs);

/* Waits for all enqueued work; surfaces device-side errors. */
int escg_sync(escg_t* h);

/* Current species counts out[0..S] (out[0] = empty sites) and the absolute
 * MCS number of the lattice.  Synchronises. */
int escg_counts(escg_t* h, uint64_t* out, uint64_t* mcs_out);

/* Logged counts: copies up to cap entries of (S+1) uint64 each, oldest
 * first, for the MCS numbers written to mcs_out (may be NULL); *n_out gets
 * the number of entries copied.  Synchronises. */
int escg_counts_log(escg_t* h, uint64_t* out, uint64_t* mcs_out, int64_t cap, int64_t* n_out);

/* Copies the lattice (L*H bytes, row-major, no padding) to host memory.
 * Synchronises. */
int escg_snapshot(escg_t* h, uint8_t* host_out);

/* Replaces the lattice with host_lattice (L*H bytes, values 0..S) at
 * absolute MCS number mcs; running on from there is bit-exact with a run
 * that reached this state itself.  Clears the counts log. */
int escg_restore(escg_t* h, const uint8_t* host_lattice, uint64_t mcs);

/* End-to-end host call: restore(host_in, mcs), run n_mcs, snapshot into
 * host_out and counts into counts_out (S+1, may be NULL).  host_in and
 * host_out may alias.  Synchronises. */
int escg_step_host(escg_t* h, const uint8_t* host_in, uint64_t mcs, uint64_t n_mcs,
                   uint8_t* host_out, uint64_t* counts_out);

/* The same step, enqueued without waiting: returns once the copies and
 * kernels are on the handle's stream.  host_in, host_out and counts_out must
 * stay valid (and host_out / counts_out unread) until escg_step_host_wait,
 * which synchronises and reports the step's errors as escg_step_host does.
 * One step at a time per handle (ESCG_ESTATE otherwise); steps on different
 * handles (each with its own stream) overlap their copies with each other's
 * kernels -- e.g. two handles used alternately for a stream of lattices.
 * With pageable host buffers the copies are synchronous (CUDA semantics), so
 * overlap needs pinned buffers. */
int escg_step_host_async(escg_t* h, const uint8_t* host_in, uint64_t mcs, uint64_t n_mcs,
                         uint8_t* host_out, uint64_t* counts_out);
int escg_step_host_wait(escg_t* h);

/* Device address of the lattice (row pitch escg_lattice_pitch(L)) and the
 * handle's stream, for zero-copy interop (e.g. a torch tensor view). */
void* escg_device_lattice(escg_t* h);
void* escg_stream(escg_t* h);
uint64_t escg_current_mcs(escg_t* h);

/* Number of kernel launches this handle has enqueued so far. */
uint64_t escg_launch_count(escg_t* h);

/* With time_kernels set: total device time (ms, CUDA events on the
 * handle's stream) and number of lattice-update launches (persistent or
 * phase kernels) since the last reset.  Synchronises. */
int escg_kernel_time(escg_t* h, double* ms_total, uint64_t* n_launches, int reset);

void escg_destroy(escg_t* h);

/* Thread-local message of the last failure on this thread ("" if none). */
const char* escg_last_error(void);

/* ---- Batched ensembles ------------------------------------------------
 * Many independent replicas (the paper runs its trials one after another;
 * here they share one GPU): each replica is a lattice with its own L, S,
 * digraph, rates, seed, initial empty fraction and MCS budget, and runs until
 * its budget is spent or -- with stop_at_extinction -- until the first log
 * point at which at most one non-empty species is alive.  The replicas' work
 * items share persistent launches of log_every MCS each; a device-side
 * compaction step between launches retires finished replicas, so the whole
 * run is enqueued (and captured in a CUDA graph) without host round trips.
 * A replica's lattice and counts are bit-identical to running it alone with
 * escg_create_ex/escg_run with the same parameters. */
typedef struct {
    int32_t L, S;                 /* as escg_create                              */
    const uint8_t* digraph;       /* S*S bytes, read during escg_batch_create    */
    escg_rates rates;
    uint64_t seed;
    double p_empty;
    uint64_t max_mcs;             /* budget (absolute MCS number to stop at)     */
    int32_t stop_at_extinction;
    const double* dominance_prob; /* optional S*S edge probabilities, as in
                                     escg_options (copied on submission)       */
} escg_replica_spec;

typedef struct {
    uint32_t log_every;           /* stasis checks / counts every k MCS (0: 10)  */
    int32_t threads;              /* CTA size 64, 128 or 256; 0: autotune        */
    int32_t use_graph;            /* capture chunk sequences in a CUDA graph     */
    void* cuda_stream;            /* cudaStream_t or NULL (library-owned)        */
    int32_t resident;             /* 1: replicas whose lattice fits one CTA's
                                     shared memory (L up to about 470) run with
                                     the whole lattice resident there for each
                                     chunk; 0 (default, faster on GB300 for
                                     every size measured): every replica in the
                                     block-by-block chunk kernel.  Results are
                                     identical.                                   */
} escg_batch_options;

typedef struct escg_batch escg_batch_t;

void escg_batch_default_options(escg_batch_options* opt);

/* Creates n replicas (n >= 1), allocates one device arena for all of them
 * and initialises every lattice.  Returns NULL on error. */
escg_batch_t* escg_batch_create(int32_t n, const escg_replica_spec* specs,
                                const escg_batch_options* opt);

/* Enqueues work until every replica is finished or has advanced max_mcs
 * more MCS (0: until every replica is finished).  Asynchronous. */
int escg_batch_run(escg_batch_t* b, uint64_t max_mcs);
int escg_batch_sync(escg_batch_t* b);

/* Per replica: MCS reached, 1 if stopped by extinction, and the counts
 * (S+1 values, padded to 16 per replica) at its last log point.  Any output
 * pointer may be NULL.  Synchronises. */
int escg_batch_status(escg_batch_t* b, uint64_t* mcs_out, int32_t* extinct_out,
                      uint64_t* counts16_out);

/* Number of replicas still running (synchronises). */
int32_t escg_batch_active(escg_batch_t* b);

/* Copies replica i's lattice (L*L bytes) to host memory.  Synchronises. */
int escg_batch_snapshot(escg_batch_t* b, int32_t i, uint8_t* host_out);

/* CTA size in use (after autotuning: the first chunks time the chunk kernel
 * at 64, 128 and 256 threads, TMA-staged and plain, and keep the fastest),
 * whether the TMA-staged chunk kernel is in use, and kernel launches so far. */
int32_t escg_batch_threads(escg_batch_t* b);
int32_t escg_batch_uses_tma(escg_batch_t* b);
uint64_t escg_batch_launch_count(escg_batch_t* b);

void escg_batch_destroy(escg_batch_t* b);

/* ---- Serving ------------------------------------------------------------
 * A request loop with continuous batching: runs (replica specs) are
 * submitted as they arrive and queue in FIFO order; escg_server_step admits
 * queued runs into free slots while the device arena has room for them,
 * advances every resident run by chunks_per_step * log_every MCS in shared
 * persistent launches, and retires the runs that went extinct or spent their
 * budget (their memory is freed for the next admissions).  A run's result is
 * bit-identical to running it alone, whatever else shares the GPU. */
typedef struct {
    uint64_t arena_bytes;         /* device memory for resident runs             */
    int32_t max_slots;            /* runs resident at once                       */
    uint32_t log_every;           /* 0: 10                                       */
    int32_t threads;              /* CTA size 64/128/256, 0: autotune            */
    uint32_t chunks_per_step;     /* chunks of log_every MCS per step (0: 4)     */
    int32_t keep_lattice;         /* 1: copy each finished lattice to the host   */
    void* cuda_stream;
} escg_server_options;

typedef struct escg_server escg_server_t;

void escg_server_default_options(escg_server_options* opt);
escg_server_t* escg_server_create(const escg_server_options* opt);

/* Queues a run; returns its id (>= 0) or a negative escg_status.  The spec's
 * digraph is copied.  Runs larger than the whole arena are rejected. */
int64_t escg_server_submit(escg_server_t* s, const escg_replica_spec* spec);

/* Admits, advances and retires (see above); synchronises at its end.
 * *finished_out (may be NULL) receives the number of runs retired. */
int escg_server_step(escg_server_t* s, int32_t* finished_out);

/* Cancels run id between steps.  A queued run is dropped (its result: MCS
 * 0, no counts); a running one stops at the MCS it has reached (its result:
 * that MCS, the counts of its last log point, its lattice with
 * keep_lattice) and frees its slot and arena memory.  Either way the id is
 * reported by the next poll.  ESCG_ESTATE if the run already finished or
 * is unknown. */
int escg_server_cancel(escg_server_t* s, int64_t id);

/* Ids of runs finished since the previous poll (up to cap). */
int escg_server_poll(escg_server_t* s, int64_t* ids_out, int32_t cap, int32_t* n_out);

/* Result of a finished run: MCS reached, extinct flag, counts at its last
 * log point (16 values), and -- with keep_lattice -- its lattice (L*L bytes;
 * lattice_out may be NULL).  ESCG_ESTATE if the run has not finished. */
int escg_server_result(escg_server_t* s, int64_t id, uint64_t* mcs_out, int32_t* extinct_out,
                       uint64_t* counts16_out, uint8_t* lattice_out);

/* Host-clock times of a finished run, in seconds since the server was
 * created: when it was submitted, when a step admitted it to a slot, and when
 * the step that retired it had synchronised (queue wait = admitted -
 * submitted; in service = finished - admitted, whole steps of
 * chunks_per_step * log_every MCS).  A run cancelled while queued has
 * admitted = finished.  ESCG_ESTATE if the run has not finished. */
int escg_server_timing(escg_server_t* s, int64_t id, double* submitted_s, double* admitted_s, double* finished_s);

/* Runs resident, runs queued, arena bytes in use. */
int escg_server_stats(escg_server_t* s, int32_t* resident, int32_t* queued, uint64_t* bytes_in_use);
int32_t escg_server_threads(escg_server_t* s);
int32_t escg_server_uses_tma(escg_server_t* s);
uint64_t escg_server_launch_count(escg_server_t* s);
void escg_server_destroy(escg_server_t* s);

/* ---- Allocation-free entry point ------------------------------------------
 * The paper has no counterpart of this call.  It exists for callers that
 * cannot let a library allocate device memory: applications that own a fixed
 * GPU memory budget (their own pool, a service that reserves all device
 * memory at start-up) and loops in which a cudaMalloc or cudaFree would
 * synchronise the device or is not permitted.
 *
 * Runs n_mcs Monte Carlo steps (schedule version 1, exactly as escg_run)
 * from absolute MCS number mcs_begin on the caller's device lattice
 * d_lattice (L rows of escg_lattice_pitch(L) bytes, 16-byte aligned, values
 * 0..S, updated in place), then, if d_counts_out is not NULL, writes the
 * species counts (S+1 uint64 values, device memory, 8-byte aligned) of the
 * final lattice there.  Inputs and outputs are the caller's; the library
 * allocates nothing, neither device nor pinned memory.  Its scratch state
 * (run state, block epochs, transition table) lives in one fixed 64 KiB
 * device array that every GPU loading the library keeps until the process
 * exits; L is therefore limited to 8..4096 (larger lattices are rejected
 * with ESCG_EINVAL and a message).  Every call clears and rewrites that
 * array, so calls whose work overlaps on the GPU (from several host threads
 * or streams) race and must be serialised by the caller.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  digraph and rates are host
 * memory read during the call; cuda_stream may be NULL (the legacy default
 * stream).  Arguments are checked on the host before any device work
 * (ESCG_EINVAL: NULL or misaligned buffers, L or S out of range, a bad
 * digraph or rates, mcs_begin + n_mcs >= 2^31); the lattice's values are
 * checked on the device before the first step, and a value outside 0..S
 * fails the call with ESCG_EINVAL, the lattice unchanged.  Returns when the
 * work has finished; ESCG_ETIMEOUT if a bounded device-side wait gave up.
 * No counts log, no stop at extinction. */
int escg_run_noalloc(uint8_t* d_lattice, int32_t L, int32_t S, const uint8_t* digraph,
                     const escg_rates* rates, uint64_t seed, uint64_t mcs_begin, uint64_t n_mcs,
                     uint64_t* d_counts_out, void* cuda_stream);

/* epsilon = 2 M N (Section 3.1, rate initialisation). */
double escg_exchange_from_mobility(double M, int64_t N);

/* Fills D (S*S) with the circulant dominance digraph C(S,K):
 * D[i*S+j] = 1 iff (j - i + S) mod S is one of K[0..nK-1]. */
int escg_circulant(int32_t S, const int32_t* K, int32_t nK, uint8_t* D);

#ifdef __cplusplus
}
#endif
#endif /* ESCG_H */
