/*
 * phmm.h -- C ABI of the GB300 (sm_103a) batched Pair-HMM library (libphmm.so).
 *
 * The library scores read/haplotype pairs with the Pair-HMM forward algorithm of
 * gpuPairHMM (Schmidt et al., arXiv 2411.11547), Sec. II-A:
 *   Eq. 1  M(i,j) = lambda(i,j) (alpha_i M(i-1,j-1) + beta (I(i-1,j-1) + D(i-1,j-1)))
 *   Eq. 2  I(i,j) = delta_i M(i-1,j) + eps I(i-1,j)
 *   Eq. 3  D(i,j) = zeta_i M(i,j-1) + eps D(i,j-1)
 *   init   M(i,0)=I(i,0)=D(i,0)=0, M(0,j)=I(0,j)=0, D(0,j)=1/n
 *   Eq. 4  lambda(i,j) = 1-Q_i if r_i == h_j else Q_i/3
 *   result L = sum_j M(m,j) + I(m,j), returned as log10 L,
 * and gives the adjoint of log10 L with respect to the per-base Phred qualities and the
 * gap-continuation penalty.  Transition probabilities come from Phred values (Sec. III-A
 * names the inputs; the conversion is this library's reading):
 *   Q_i = 10^(-bq_i/10), delta_i = 10^(-iq_i/10), zeta_i = 10^(-dq_i/10),
 *   eps = 10^(-gcp/10), beta = 1 - eps, alpha_i = 1 - (delta_i + zeta_i)
 *   (alpha_mode 1: alpha_i = 1 - 10^(-(iq_i+dq_i)/10)).
 * With a per-base gap-continuation track gcp_i, eps_i = 10^(-gcp_i/10) and beta_i = 1 - eps_i
 * replace eps and beta in the rows they enter (Eq. 1-3 index every transition of row i by
 * read position i: eps_i in I(i,j) and D(i,j), beta_i in M(i,j)).
 * 'N' on either side matches every base; bases are ASCII A C G T N, either case.
 *
 * Conventions shared by every call:
 *   - Every data pointer in phmm_batch and every output pointer is DEVICE memory owned by
 *     the caller.  The library never frees or retains caller memory beyond the plan.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default stream.
 *   - Return value: PHMM_OK (0) or a negative PHMM_E* code.  No exception crosses the ABI,
 *     no kernel traps, and no call spins without a bound.
 *   - Calls are thread-compatible: one plan must not be used from two host threads at once.
 */
#ifndef PHMM_H
#define PHMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define PHMM_OK 0
#define PHMM_EINVAL -1   /* bad argument: offsets, lengths, bases, quals, gcp, pair ids */
#define PHMM_ETOOLONG -2 /* a read longer than the call supports */
#define PHMM_ENOMEM -3   /* workspace smaller than phmm_workspace_bytes() */
#define PHMM_ECUDA -4    /* a CUDA runtime call failed; see phmm_last_cuda_error() */
#define PHMM_ESTATE -5   /* call out of order (e.g. backward on a plan never run forward) */
#define PHMM_EGUARD -6   /* debug builds only: a workspace guard region was overwritten, or a
                            kernel's index check failed (the pair was flagged invalid) */

#define PHMM_MAX_READ_LEN 512 /* longest read (rows) one wavefront group holds */
/* Longest read a plan takes: reads beyond PHMM_MAX_READ_LEN are swept in row tiles of
 * PHMM_MAX_READ_LEN rows, forward and adjoint (Sec. III-C supports reads up to 1,024).
 * phmm_forward_noalloc takes reads up to PHMM_MAX_READ_LEN only. */
#define PHMM_MAX_READ_LEN_FWD 2048

/* ---- per-pair flags written by phmm_forward ---------------------------------------- */
#define PHMM_FLAG_FP32 1       /* result from the FP32 wavefront (|err| <= 1e-3 log10) */
#define PHMM_FLAG_RESCUED64 2  /* FP32 result underflowed: recomputed in FP64          */
#define PHMM_FLAG_EXTENDED 4   /* recomputed with per-lane power-of-two exponents       */
#define PHMM_FLAG_INVALID 8    /* invalid pair (bad ids or data): output is NaN         */

/* ---- quality dtypes ------------------------------------------------------------------ */
#define PHMM_QUAL_U8 0  /* uint8 Phred values (forward only)                  */
#define PHMM_QUAL_F32 1 /* float Phred values, continuous (differentiable)    */

/*
 * A batch of reads, haplotypes and the pairs to score (Sec. II-A: batches B_q = (R_q, H_q);
 * Sec. III-A: reads carry per-base quality scores plus insertion and deletion gap
 * qualities).  All arrays are device memory; the plan keeps the pointers (not copies), so
 * the caller keeps them alive and unchanged while the plan is used.
 */
typedef struct phmm_batch {
  int64_t n_reads;            /* R >= 1 */
  int64_t n_haps;             /* H >= 1 */
  int64_t n_pairs;            /* P >= 0 */
  const uint8_t *read_bases;  /* [sum m] ASCII bases, reads concatenated */
  const void *base_q;         /* [sum m] Phred base qualities, dtype qual_dtype */
  const void *ins_q;          /* [sum m] Phred insertion gap-open qualities */
  const void *del_q;          /* [sum m] Phred deletion gap-open qualities */
  int32_t qual_dtype;         /* PHMM_QUAL_U8 or PHMM_QUAL_F32 */
  int32_t alpha_mode;         /* 0: alpha = 1-(delta+zeta)  1: alpha = 1-10^(-(iq+dq)/10) */
  const int64_t *read_off;    /* [R+1] read r = read_bases[read_off[r] .. read_off[r+1]) */
  const uint8_t *hap_bases;   /* [sum n] ASCII bases, haplotypes concatenated */
  const int64_t *hap_off;     /* [H+1] */
  const int32_t *pair_read;   /* [P] read index of each pair */
  const int32_t *pair_hap;    /* [P] haplotype index of each pair */
  double gcp;                 /* Phred gap-continuation penalty, > 0 */
  const void *gcp_q;          /* [sum m] per-base gap-continuation Phred values (qual_dtype,
                                 each > 0), or NULL: gcp at every read position.  A plan with
                                 a track uses the extended-range FP32 first line and a fixed
                                 read-length -> group table (the options' tables are ignored;
                                 first_line = PHMM_FIRST_PLAIN32 is rejected with EINVAL) */
} phmm_batch;

/* First-line (bulk) arithmetic of the forward pass. */
#define PHMM_FIRST_PLAIN32 0 /* FP32, initial constant 2^120 (rescue below 1e-28 scaled) */
#define PHMM_FIRST_EXT32 1   /* FP32 with per-lane power-of-two exponents: never underflows */

/*
 * Launch options.  phmm_options_default() fills the recommended values; fields may then be
 * changed.  A NULL options pointer means the defaults.
 */
typedef struct phmm_options {
  int32_t first_line;  /* PHMM_FIRST_PLAIN32 or PHMM_FIRST_EXT32 */
  int32_t rescue;      /* 1: FP64 rescue of pairs below the FP32 threshold; 0: none */
  int32_t binning;     /* 1: length binning + packing; 0: one fixed (lanes, rows) group */
  int32_t lanes;       /* fixed group when binning == 0: lanes per pair, 4/8/16/32 */
  int32_t rows;        /* fixed group when binning == 0: rows per lane, 4/8/12/16/20 */
  int32_t persistent;  /* 1: persistent work-queue kernels; 0: one warp group per item */
  int32_t use_graph;   /* 1: replay the launch sequence from a captured CUDA graph:
                          phmm_forward always (one capture per workspace/output pointer
                          set); phmm_forward_partials / phmm_backward_partials on batches of
                          at most 2^30 cells, captured when a call repeats the previous
                          call's pointers (their kernel-time events are then not recorded) */
  int32_t warps_per_block; /* 1..4 warps per block (0 = 4) */
  int32_t bin_rows[PHMM_MAX_READ_LEN / 4 + 1]; /* optional read-length -> group table: entry
                          (m + 3) / 4 is the group of reads of length m, as an index
                          li * 17 + (rows - 4) with lanes 4 << li (li = 0..3) and rows per lane
                          4..20 (the forward is built for even rows, the adjoint for 4-12 and
                          some others: see bwd_rows); -1 or an unbuilt group: the default */
  int32_t bin_table_valid; /* 1 if bin_rows holds a table */
  int32_t adjoint_rescue;  /* 1: adjoints out of the FP32 range are redone in FP64; 0: NaN;
                              2: every pair's adjoint in FP64 (reference gradients, slower) */
  int32_t bwd_rows[PHMM_MAX_READ_LEN / 4 + 1]; /* optional read-length -> adjoint group table
                          (indices as bin_rows; adjoint groups: rows 4, 6, 8, 10, 12 with any
                          lanes, 16 x 14, 32 x 16, and 4 x 9/11, 8 x 7/9/11, 16 x 7/9/11/13,
                          32 x 7/9) */
  int32_t bwd_table_valid; /* 1 if bwd_rows holds a table */
  int32_t bwd_warps_per_block; /* adjoint launches: 1..4 (0 = warps_per_block) */
} phmm_options;

void phmm_options_default(phmm_options *opt);

typedef struct phmm_plan phmm_plan;

/*
 * Validate a batch and build a plan.  Runs one validation kernel on `stream` and waits for
 * it (the only host synchronisation of the library): read and haplotype offsets must be
 * non-decreasing from 0, every read and haplotype non-empty, bases in {A,C,G,T,N} (either
 * case), Phred values finite-or-+inf and >= 0 with delta+zeta <= 1 (alpha_mode 0), pair ids
 * in range, gcp > 0, reads at most PHMM_MAX_READ_LEN_FWD long.  Returns PHMM_EINVAL /
 * PHMM_ETOOLONG on bad input (no plan is created), PHMM_OK otherwise with *plan set.  The
 * plan keeps the batch pointers.
 */
int phmm_plan_create(const phmm_batch *batch, const phmm_options *opt, void *stream,
                     phmm_plan **plan);

/* Bytes of device workspace phmm_forward / phmm_backward need (256-byte aligned start). */
size_t phmm_workspace_bytes(const phmm_plan *plan);

/* Plan facts: total read bases, total haplotype bases, sum over pairs of m*n (Eq. 5). */
int phmm_plan_info(const phmm_plan *plan, int64_t *sum_m, int64_t *sum_n, int64_t *cells);

/*
 * Forward pass: out_log10[p] = log10 P(read | haplotype) for every pair p (device double
 * [P]) and out_flags[p] (device uint8 [P], PHMM_FLAG_*).  Asynchronous on `stream`; no host
 * synchronisation.  ws: device workspace of at least phmm_workspace_bytes(plan) bytes,
 * 256-byte aligned, used as scratch (contents need not be preserved between calls except
 * that phmm_backward reads what the latest phmm_forward on the same ws left there).
 * Returns PHMM_ENOMEM if ws_bytes is too small, PHMM_EINVAL for NULL/misaligned pointers.
 */
int phmm_forward(phmm_plan *plan, void *ws, size_t ws_bytes, double *out_log10,
                 uint8_t *out_flags, void *stream);

/*
 * Adjoint: given dL[p] = d(loss)/d(log10 L_p) (device double [P]), writes
 *   d_base_q, d_ins_q, d_del_q : device float [sum m], d(loss)/d(Phred) summed over the
 *                                pairs that share each read (overwritten, FP64-accumulated);
 *   d_gcp_q                    : device float [sum m], the same for the per-base
 *                                gap-continuation track (required when the batch has one,
 *                                else ignored and may be NULL);
 *   d_gcp                      : device double [1], d(loss)/d(gcp) summed over all pairs (with
 *                                a track: the sum of d_gcp_q, the derivative for one shift
 *                                of every gap-continuation value).
 * Invalid pairs contribute nothing.  Requires a preceding phmm_forward with the same plan and
 * ws (PHMM_ESTATE otherwise).  Reads longer than PHMM_MAX_READ_LEN are swept in the same row
 * tiles as the forward.  Asynchronous on `stream`.
 */
int phmm_backward(phmm_plan *plan, void *ws, size_t ws_bytes, const double *dL,
                  float *d_base_q, float *d_ins_q, float *d_del_q, float *d_gcp_q,
                  double *d_gcp, void *stream);

/*
 * Fused training step, part 1: the adjoint sweep with dL = 1 for every pair.  Its own forward
 * pass (the per-lane-exponent FP32 recurrence of Eq. 1-3; pairs it cannot represent finished
 * in FP64) writes out_log10 / out_flags exactly as phmm_forward documents them (flags
 * PHMM_FLAG_FP32 or PHMM_FLAG_RESCUED64, with PHMM_FLAG_EXTENDED), and every pair's
 * d log10 L_p / d(Phred inputs) stays in ws.  A pair's gradient is linear in dL[p], so
 * phmm_backward_partials then only weights and reduces them: one forward sweep per step
 * instead of phmm_forward's plus the adjoint's.  Same arguments, ownership and errors as
 * phmm_forward.  Asynchronous on `stream`.
 */
int phmm_forward_partials(phmm_plan *plan, void *ws, size_t ws_bytes, double *out_log10,
                          uint8_t *out_flags, void *stream);

/*
 * Fused training step, part 2: writes d_base_q, d_ins_q, d_del_q, d_gcp_q and d_gcp as
 * phmm_backward does, from the partials the latest phmm_forward_partials on this plan and ws left there,
 * each pair's weighted by dL[p] (device double [P]) in the FP64 per-read reduction.  May be
 * called again with another dL.  PHMM_ESTATE without a preceding phmm_forward_partials, or
 * after a phmm_backward (which overwrites the partials).  Asynchronous on `stream`.
 */
int phmm_backward_partials(phmm_plan *plan, void *ws, size_t ws_bytes, const double *dL,
                           float *d_base_q, float *d_ins_q, float *d_del_q, float *d_gcp_q,
                           double *d_gcp, void *stream);

void phmm_plan_destroy(phmm_plan *plan);

const char *phmm_status_str(int status);

/* The cudaError_t of the most recent PHMM_ECUDA return on this host thread. */
int phmm_last_cuda_error(void);

/*
 * Kernel-time instrumentation: number of kernel launches the latest phmm_forward /
 * phmm_backward on this plan issued (graph nodes count as launches), and the elapsed time of
 * the FP32 wavefront kernels and of the FP64 rescue kernels of the latest forward, from CUDA
 * events recorded on the launching stream.  Only a forward run without a CUDA graph
 * (use_graph = 0) records those events; otherwise, or before the work has finished, both
 * times are -1.  For throughput reporting only.
 */
int phmm_plan_launch_count(const phmm_plan *plan, int which /* 0 fwd, 1 bwd */);
int phmm_plan_wavefront_ms(phmm_plan *plan, float *ms_fp32, float *ms_rescue);

/*
 * Elapsed time of the latest phmm_backward's adjoint wavefront kernels (FP32 pass and its
 * FP64 hand-off pass) and of its FP64 gradient reduction, from CUDA events on the launching
 * stream; -1 before the work has finished.
 */
int phmm_plan_backward_ms(phmm_plan *plan, float *ms_adjoint, float *ms_reduce);

/*
 * Rescue statistics of the latest calls on this plan and workspace, copied to the host
 * (waits for `stream`): counts[0] pairs the forward recomputed in FP64, counts[1] of those
 * that went on to the per-lane-exponent FP64 kernel, counts[2] pairs whose adjoint was
 * finished in FP64, counts[3] / counts[4] of those handed off because forward and adjoint
 * mass lay beyond one FP32 exponent range / because a partial sum was not finite, and
 * counts[5] reserved (0).  counts holds 6 values.
 */
int phmm_plan_rescue_counts(phmm_plan *plan, const void *ws, void *stream, int64_t *counts);

/*
 * Autotune the read-length -> group tables for this batch's length mix (Sec. III-C picks
 * rows per thread by read length; here the choice is measured).  For every 16-row
 * read-length range that holds pairs, a strided sample of at most `sample_pairs` of its
 * pairs is gathered into a compact device batch and each built group (lanes x rows) whose
 * capacity covers the range, up to twice the range's longest read, is timed with CUDA
 * events around phmm_forward (which & 1, on samples 8x larger) and phmm_backward (which & 2).
 * The fastest group of each range is written into opt->bin_rows / opt->bwd_rows if it beats
 * the built-in group by at least 2% (other entries: -1, meaning the built-in default, or the
 * caller's previous entries) and bin_table_valid / bwd_table_valid are set.  Then warps_per_block (forward) and bwd_warps_per_block (adjoint),
 * each 1, 2 or 4 (pairs per block = warps x the group's pairs per warp), are timed with the
 * tuned tables on a strided sample of the whole batch and the fastest are written.  The other
 * fields of *opt are used as given.
 *
 * The batch is validated as by phmm_plan_create (same errors).  A batch with a per-base
 * gap-continuation track runs a fixed group table: nothing is tuned and *opt is unchanged.  Allocates temporary device
 * memory with cudaMallocAsync on `stream`, copies the offsets and pair lists to the host
 * and synchronises `stream` repeatedly: run it once per workload shape, before timing.
 */
int phmm_autotune(const phmm_batch *batch, phmm_options *opt, int which, int64_t sample_pairs,
                  void *stream);

/*
 * End-to-end scoring of a batch held in HOST memory (the host workflow of Sec. III-A:
 * partition, transfer, score, transfer back).  Every pointer of *host_batch is host memory
 * (pageable or pinned); out_log10 / out_flags are host arrays of n_pairs.  Pairs are grouped by
 * read and cut into subsets of about `subset_cells` cells (Eq. 5; at least one read each).
 * Each subset is packed into pinned staging memory, copied to the device in one transfer
 * (on a device that reads pageable host memory coherently, e.g. over NVLink-C2C, only its
 * offsets and pair ids are: the kernels read bases, qualities and haplotypes in place),
 * validated and scored with phmm_plan_create / phmm_forward (options `opt`, NULL = defaults;
 * CUDA graphs are not used), and its results copied back, on one of two streams, so the host
 * packing and copies of one subset overlap the scoring of the previous one.  Returns when
 * every result is in host memory.  Its pinned staging and device buffers grow to the largest
 * subset seen and are kept for later calls on the same device (pinned allocation is slow);
 * phmm_score_host_release() frees them.  Calls are serialised by a lock.  Errors: those of
 * phmm_plan_create for a subset's inputs, PHMM_ENOMEM if a buffer cannot be allocated,
 * PHMM_ECUDA (buffers are then freed).
 */
int phmm_score_host(const phmm_batch *host_batch, const phmm_options *opt,
                    int64_t subset_cells, double *out_log10, uint8_t *out_flags);
void phmm_score_host_release(void);

/*
 * The same pipeline for the gradient: given dL[p] = d(loss)/d(log10 L_p) in host memory
 * (double [P]; known before the call, e.g. a fixed weighting of the log-likelihoods), every
 * subset runs the fused step (phmm_forward_partials, then phmm_backward_partials with the
 * subset's dL) and returns out_log10 / out_flags as phmm_score_host does, and
 *   d_base_q, d_ins_q, d_del_q : host float [sum m], as phmm_backward (reads without pairs: 0);
 *   d_gcp_q                    : host float [sum m] for a batch with a per-base track (else
 *                                ignored, may be NULL);
 *   d_gcp                      : host double [1], summed over the subsets in order.
 * A subset holds every pair of its reads, so each read's gradient comes from one subset's
 * FP64 reduction.  The first three subsets take 1/8, 1/4 and 1/2 of subset_cells and the last
 * ones halve what is left (down to 1/8), so the transfers that cannot overlap any computation
 * stay small.  The copies of one subset overlap the computation of the previous one.
 * Errors: those of phmm_score_host, PHMM_EINVAL for a NULL dL or gradient array.  Shares
 * phmm_score_host's buffers and lock.
 */
int phmm_grad_host(const phmm_batch *host_batch, const phmm_options *opt,
                   int64_t subset_cells, const double *dL, double *out_log10,
                   uint8_t *out_flags, float *d_base_q, float *d_ins_q, float *d_del_q,
                   float *d_gcp_q, double *d_gcp);

/*
 * Forward scoring for callers that cannot allocate device memory.
 *
 * Some callers may not call cudaMalloc at all: code running inside a framework that owns
 * every device allocation through its own pool, request paths of a server where an
 * allocation (and the device-wide synchronisation cudaMalloc/cudaFree can imply) is not
 * allowed, or a plug-in that is only handed its input and output buffers.  This entry
 * point needs no plan and no workspace: its scratch (per-position parameters, base codes,
 * padded haplotype codes) lives in one static device array of PHMM_NOALLOC_SCRATCH_BYTES
 * that every GPU loading the library holds until the process exits.  It allocates nothing
 * (no cudaMalloc, cudaFree or allocating library call).
 *
 * Arguments are those of phmm_batch (device memory, caller-owned) plus out_log10[P] and
 * out_flags[P] (device).  It scores every pair with the extended-range FP32 wavefront in one
 * lanes x rows group sized by the longest read (no length binning, no FP64 rescue: flags
 * are PHMM_FLAG_FP32 | PHMM_FLAG_EXTENDED, or PHMM_FLAG_INVALID with a NaN result for
 * out-of-range pair ids).  The offsets are checked on the device (read_off[0] == hap_off[0]
 * == 0, every read and haplotype non-empty); bases and qualities are not validated (use
 * phmm_plan_create for that where allocation is allowed).  It waits once on `stream` to
 * read the batch sizes and the offset check.
 *
 * Returns PHMM_ENOMEM if the batch's scratch (16 B per read base + 1 B per read base + the
 * padded haplotype codes, about 1 B per haplotype base + 112 B per haplotype) exceeds
 * PHMM_NOALLOC_SCRATCH_BYTES, PHMM_ETOOLONG for a read longer than PHMM_MAX_READ_LEN,
 * PHMM_EINVAL for bad arguments or offsets or a batch with a per-base gap-continuation
 * track (this entry point takes the scalar gcp only), PHMM_ECUDA on a CUDA error.  A batch
 * without pairs returns PHMM_OK after the checks.
 *
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * with that device current; make that first call before any stream capture.  Every call
 * shares the one array, which keeps the previous call's contents: calls that overlap on
 * the GPU (other streams or threads) race and must be serialised by the caller.  The paper
 * has no counterpart to this entry point.
 */
#define PHMM_NOALLOC_SCRATCH_BYTES (64 << 20)
int phmm_forward_noalloc(const phmm_batch *batch, double *out_log10, uint8_t *out_flags,
                         void *stream);

/*
 * Debug builds (libphmm_debug.so, compiled with -DPHMM_DEBUG; no counterpart in the paper):
 * the plan's workspace holds a 256-byte guard region after every region, filled with 0xA5
 * before each call and checked after it, and the kernels check each pair's read positions,
 * haplotype codes, scratch slot and checkpoints against the plan's sizes, flagging the pair
 * invalid (NaN result) instead of touching memory outside them.  phmm_forward,
 * phmm_backward, phmm_forward_partials and phmm_backward_partials then wait for `stream`
 * and return PHMM_EGUARD if a check failed.
 *   phmm_debug_guard_offset: byte offset in the workspace of guard region k (PHMM_EINVAL
 *     past the last one);
 *   phmm_debug_check: checks the guards now (waits for `stream`).
 * In the release library both return PHMM_ESTATE.
 */
int phmm_debug_guard_offset(const phmm_plan *plan, int k, size_t *offset);
int phmm_debug_check(phmm_plan *plan, void *ws, void *stream);

/*
 * Arithmetic-pipe probe (roofline denominators): lane multiply-adds per second sustained
 * by one kernel on the current device.  kind 0 = FP32 FFMA, 1 = packed fma.rn.f32x2
 * (counted as two lane operations), 2 = FP64 DFMA.  Allocates and frees a small buffer.
 */
int phmm_probe_pipe(int kind, int iters, double *lane_ops_per_s, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* PHMM_H */
