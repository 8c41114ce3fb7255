/*
 * escg_diag.h -- diagnostics of libescg that are not part of the model: a
 * measurement of the GPU's integer-issue rate (the denominator of the
 * Monte Carlo kernels' roofline; the paper has no counterpart) and a
 * host-controlled stall used to test the bounded device-side waits of the
 * persistent kernel without hanging or faulting the GPU.
 */
#ifndef ESCG_DIAG_H
#define ESCG_DIAG_H

#include <stdint.h>

#include "escg.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Runs a kernel of independent integer chains on every SM of the current
 * device -- each step one 32x32+32->64-bit multiply-add and one
 * three-input XOR, the two instruction kinds of a Philox round -- and
 * reports the achieved rate in thread-level integer instructions per second
 * (*ops_per_s) and per SM per SM clock cycle (*ops_per_sm_clk, may be NULL).
 * Allocates and frees a small device buffer; synchronises. */
int escg_diag_int_throughput(double* ops_per_s, double* ops_per_sm_clk);

/* The same kind of probe for the instruction mix of one elementary step:
 * 24 integer instructions per step (a quarter of a Philox4x32-10 call --
 * 5 wide multiplies and 5 three-input XORs -- and the cell and neighbour
 * offsets, action select, table index and unpacking: 2 byte permutes,
 * 4 shifts, 3 adds, 2 compares, 1 select, 1 multiply-add, 1 and).
 * *alg_per_s: instructions of that mix per second (the denominator of the
 * Monte Carlo kernels' integer roofline, which counts the same 24 per
 * attempt); *alg_per_sm_clk (may be NULL) per SM per SM clock.  Allocates
 * and frees a small device buffer; synchronises. */
int escg_diag_alg_throughput(double* alg_per_s, double* alg_per_sm_clk);

/* Device-to-device copy bandwidth between two buffers of `bytes` each that
 * stay in L2 (16-byte vectors, loads through L2 as the Monte Carlo kernels'
 * tile loads): one launch copying the buffer reps times, after a warm-up
 * launch of three copies; *gbs = bytes read + bytes written per second /
 * 1e9.  Allocates and frees the two buffers; synchronises. */
int escg_diag_l2_copy(size_t bytes, int reps, double* gbs);

/* Test hook: the next persistent launches of h never publish the epoch of
 * coarse block `block` (0 <= block < P*P), so its neighbours' waits run out
 * after `spin_limit` polls; escg_sync then returns ESCG_ETIMEOUT and the
 * handle refuses to run until escg_restore.  block < 0 clears the hook;
 * spin_limit 0 restores the default limit. */
int escg_debug_stall_block(escg_t* h, int32_t block, uint32_t spin_limit);

/* The autotuner's choice for a handle created with escg_options.autotune:
 * the launch mode (escg_options.persistent) and CTAs per SM it runs with,
 * the winner's device time per MCS, and how many distinct configurations
 * were timed (0: the choice came from the process's cache).  ESCG_ESTATE for
 * a handle created without autotune. */
int escg_autotune_result(escg_t* h, int32_t* persistent, int32_t* ctas_per_sm, double* ms_per_mcs,
                         int32_t* candidates);

/* Coarse blocks per axis (P) of the handle's schedule-v1 partition. */
int32_t escg_coarse_blocks(escg_t* h);

/* Name of the kernel that advances the handle's lattice ("persistent_own_
 * kernel", "persistent_ll_kernel", "persistent_kernel", "persistent_tma_
 * kernel", "resident_kernel" or "phase_kernel"), fixed at creation by the
 * options, the partition and the device's occupancy; a static string, or ""
 * for a NULL handle.  The choice never changes results. */
const char* escg_update_kernel(escg_t* h);

#ifdef __cplusplus
}
#endif
#endif /* ESCG_DIAG_H */
