/*
 * tcorr: closed-shell CCSD(T) triples-correction energy on GB300 (sm_103a).
 *
 * The operation (Sec. 2.2 of Eriksen, arXiv:1609.08094):
 *
 *   E(T) = E[4] + E[5],
 *   E[4] = sum_{ijk} sum_{abc} W~ W / D,   E[5] = sum_{ijk} sum_{abc} Y~ W / D,
 *   W^{abc}_{ijk} = P^{abc}_{ijk} [ sum_d t^{ad}_{ij} (ck|bd) - sum_l t^{ab}_{il} (ck|lj) ]
 *                                                  (Eqs. analytical_triples_ampl, symm_operator)
 *   Y^{abc}_{ijk} = t^a_i (jb|kc) + t^b_j (ia|kc) + t^c_k (ia|jb)   (Eq. piecuch_z_coefficients)
 *   x~^{abc}     = 4/3 x^{abc} - 2 x^{acb} + 2/3 x^{bca}             (Eq. piecuch_tilde_quantity)
 *   D^{abc}_{ijk} = e_i + e_j + e_k - e_a - e_b - e_c                (Eq. e_orb_diff, sign: occ - vir)
 *
 * evaluated as the restricted loop over occupied triples i <= j <= k of
 * Sec. 3 ("tasks", Eq. tasks_ccsdpt: C(o+2,3) of them, numbered
 * lexicographically in (i, j, k)).  Integrals are real, in Mulliken
 * notation, with 8-fold permutational symmetry; t^{ab}_{ij} = t^{ba}_{ji}.
 *
 * Conventions for every entry point:
 *  - All arrays are row-major C order, float64.
 *  - Every call returns a tcorr_status and never throws, aborts or exits.
 *    Details of the last failure: tcorr_last_error(handle) (or NULL for a
 *    failure of tcorr_create).
 *  - A handle is not thread-safe; use one handle per host thread.
 *  - Device work runs on the stream given to tcorr_create (NULL = the legacy
 *    default stream).  Calls that return host results synchronise that
 *    stream before returning.
 */
#ifndef TCORR_H
#define TCORR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tcorr_s *tcorr_t;

typedef enum {
    TCORR_OK = 0,
    TCORR_EINVAL = 1,       /* bad argument: NULL pointer, size < 1, range outside the task list */
    TCORR_ENOMEM = 2,       /* footprint larger than free device memory, or host allocation failed */
    TCORR_ECUDA = 3,        /* a CUDA runtime/driver call failed (message in tcorr_last_error) */
    TCORR_ETIMEOUT = 4,     /* a bounded device-side wait expired; the context stays usable */
    TCORR_EUNSUPPORTED = 5  /* precision or size not supported on this device */
} tcorr_status;

typedef enum {
    TCORR_FP64 = 0,    /* W contractions and energy in FP64 (FP64 pipe) */
    TCORR_TF32X3 = 1,  /* W contractions on tcgen05 tensor cores, TF32 hi+lo split, 3 products,
                          FP32 accumulation, W stored in FP32 (Sec. 3 mixed precision,
                          re-designed).  Energy epilogue: the numerators sum Z W and sum Z Y of
                          each element orbit in FP32; the denominator e_i+e_j+e_k-e_a-e_b-e_c,
                          its reciprocal and numerator x 1/D to FP64 accuracy (float-float
                          arithmetic on the FP32 pipe, relative error ~2^-44); every sum
                          (per thread, CTA, orbit, task, problem) in FP64 or float-float */
    TCORR_BF16X3 = 2,  /* as TF32X3 with BF16 hi+lo operands.  A BF16 hi+lo split keeps 16
                          significant bits, and its residual averages below the 1e-6 bound only
                          over enough work: problems below 1e11 algorithmic flops (12 v^3 (v+o)
                          per task with i, j, k not all equal) run on TF32 hi+lo operands
                          instead (same products and kernels, so their results are identical
                          to TCORR_TF32X3's) -- in single, batch and server handles alike */
    TCORR_FP64_OZ = 3  /* FP64-accurate W contractions on the BF16 tensor cores: each operand split
                          into 5 signed 7-bit slices under one power-of-two scale per operand side
                          (Ozaki scheme), slice products summed exactly in FP32 per 32-element K
                          chunk and in int64 across chunks, U rounded once to FP64 and stored as
                          a float-float (hi, lo) pair (~48 significant bits); the energy epilogue
                          in float-float arithmetic on the FP32 pipe (relative error ~2^-44 per
                          operation) with FP64 sums from the orbit on.  sm_103 only; device or
                          host inputs; batch and server too */
} tcorr_precision;

/* TCORR_BF16X3 problems below this many algorithmic flops run on TF32 operands */
#define TCORR_BF16_MIN_FLOPS 1e11
/* TCORR_BF16X3 RI-MP2 problems below this many (pair, a, b, gamma) terms run on TF32 operands */
#define TCORR_MP2_BF16_MIN_TERMS 16777216.0

typedef struct {
    int prec;           /* tcorr_precision; 0 = TCORR_FP64 */
    int host_inputs;    /* 0: the array arguments of tcorr_create are device pointers;
                           1: they are host pointers (pageable or pinned), copied in */
    int batch_tasks;    /* tasks per internal batch (batch handle: at most this many tasks per
                           wave), 0 = chosen from the scratch budget (single handle: U scratch
                           of min(16 GiB, free device memory / 8)) */
    int profile;        /* 1: time every kernel class with CUDA events (tcorr_kernel_times) */
    int test_stall;     /* testing only, 0 in normal use: 1 makes the tensor-core kernel withhold
                           one chunk's loads so that a bounded device-side wait expires; the
                           energy call then returns TCORR_ETIMEOUT and the context stays usable */
    int tune;           /* tensor-core tile shape per problem shape: 0 = cost model (fewest padded
                           tiles), 1 = measured at create time (each candidate timed on the
                           problem's own operands; cached per (precision, o, v) in the process) */
    int eager;          /* batch handle: 1 = launch the waves directly on every call instead of
                           replaying the CUDA graph captured on the first call */
    int wave_mb;        /* batch handle: U scratch per wave in MiB (0 = 2048); raised to one
                           task of the largest problem when smaller.  Server: its wave scratch
                           (0 = 2048) */
    int single_sm;      /* split precisions: 0 = W contractions on SM pairs (2-CTA clusters,
                           tcgen05 cta_group::2, M = 256 tiles: each SM loads its own A tile and
                           half of B); 1 = one SM per tile (M = 128) */
} tcorr_opts;           /* zero-initialised = defaults */

/*
 * Create a handle for one (T) problem with o occupied and v virtual orbitals:
 * the inputs of the operation above (Sec. 2.2), which the handle re-lays out
 * for the W contractions of Eq. analytical_triples_ampl and the energy terms
 * of Eqs. piecuch_4th_order, piecuch_5th_order.
 *
 *   eps_occ [o]           orbital energies e_i
 *   eps_vir [v]           orbital energies e_a
 *   t1      [o][v]        t^a_i
 *   t2      [o][o][v][v]  t^{ab}_{ij}
 *   vvvo    [v][v][v][o]  (ab|ci)
 *   ooov    [o][o][o][v]  (ij|ka)
 *   ovov    [o][v][o][v]  (ia|jb)
 *
 * The arrays are owned by the caller and are only read during this call:
 * the handle keeps its own re-laid-out copies (kernel layouts, and for the
 * mixed precisions the hi/lo split operands), so the caller may free them
 * once tcorr_create returns.  opts may be NULL (defaults).  stream is a
 * cudaStream_t or NULL.  On success *out receives the handle; on failure
 * *out is set to NULL and nothing is leaked.
 * Errors: EINVAL (NULL pointer, o < 1, v < 1, an option outside its range,
 * unknown precision), ENOMEM (footprint above free device memory),
 * EUNSUPPORTED (mixed precision on a device other than sm_103),
 * ECUDA.
 */
tcorr_status tcorr_create(tcorr_t *out, int o, int v,
                          const double *eps_occ, const double *eps_vir,
                          const double *t1, const double *t2,
                          const double *vvvo, const double *ooov,
                          const double *ovov, const tcorr_opts *opts,
                          void *stream);

/* Number of tasks (sorted occupied triples i <= j <= k), C(o+2, 3). */
int64_t tcorr_num_tasks(tcorr_t h);

/* Occupied indices of task idx: ijk[0] <= ijk[1] <= ijk[2].  EINVAL if idx
 * is outside [0, tcorr_num_tasks). */
tcorr_status tcorr_task(tcorr_t h, int64_t idx, int *ijk);

/*
 * Full energy: E[4], E[5] (Eqs. piecuch_4th_order, piecuch_5th_order) and
 * E(T) summed over every task of the restricted loop (Sec. 3).  e_out (host,
 * 3 doubles) receives E[4], E[5], E(T).  Synchronous on the handle's stream.
 * Deterministic: the same handle returns bit-identical results.
 */
tcorr_status tcorr_energy(tcorr_t h, double *e_out);

/*
 * Energy of the tasks first .. first+count-1 (the collapsed loop of Sec. 3
 * cut into a contiguous range; tasks have equal weight, Sec. 5).
 * e_out (host, 3 doubles): the range's E[4], E[5], E(T).
 * e_task (host, [count][2] doubles, or NULL): E[4] and E[5] share of each
 * task.  EINVAL if the range leaves [0, tcorr_num_tasks).
 */
tcorr_status tcorr_energy_range(tcorr_t h, int64_t first, int64_t count,
                                double *e_out, double *e_task);

/*
 * Per-kernel-class device time accumulated since create (or the last reset)
 * when opts.profile = 1, measured with CUDA events on the handle's stream.
 * Classes: 0 = layout prep, 1 = W contraction (U) GEMM, 2 = fused energy
 * epilogue, 3 = reductions.  ms[4] and launches[4] are host arrays; either
 * may be NULL.  reset != 0 zeroes the counters after reading.
 */
tcorr_status tcorr_kernel_times(tcorr_t h, double *ms, int64_t *launches, int reset);

/* Device bytes held by the handle. */
int64_t tcorr_device_bytes(tcorr_t h);

/* Release every resource of the handle.  NULL is accepted (no-op). */
tcorr_status tcorr_destroy(tcorr_t h);

/* Text of the last failure on h (h = NULL: last failure of tcorr_create on
 * this thread).  Never NULL; owned by the library. */
const char *tcorr_last_error(tcorr_t h);

/* Static name of a status code. */
const char *tcorr_status_string(tcorr_status s);

/* ABI version (incremented on incompatible change). */
int tcorr_version(void);

/*
 * Batch of independent problems ("molecules" of uneven o, v) evaluated
 * together: the flattening of the per-problem task loops of Sec. 3 one level
 * further, across problems.  All problems share one precision, one stream and
 * one scratch; their tasks are cut into waves that fill the scratch, and each
 * wave runs the same three launches as a single handle (persistent W
 * contraction over the wave's (problem, task, group, tile) units, fused
 * epilogue, per-task reduction), followed by one per-problem Kahan sum.  The
 * launch sequence of a whole energy call is captured once into a CUDA graph
 * (on the first call) and every call replays it (opts.eager = 1: launch the
 * kernels directly instead; opts.profile and opts.test_stall imply it).  Tile
 * shapes of the tensor-core contraction are chosen per problem shape
 * (opts.tune).  Results do not depend on the other problems of the batch, on
 * the wave cut or on graph replay: each problem's energies are bit-identical
 * to those of a single handle with the same precision and tile shape.
 */
typedef struct tcorr_batch_s *tcorr_batch_t;

typedef struct {
    int o, v;           /* orbitals of this problem */
    const double *eps_occ, *eps_vir, *t1, *t2, *vvvo, *ooov, *ovov;  /* as for tcorr_create */
} tcorr_problem;

/*
 * Create a batch of n >= 1 problems.  problems[n] describes each as the
 * arguments of tcorr_create do (device or host pointers per opts.host_inputs,
 * read only during the call).  opts as for tcorr_create plus eager, wave_mb;
 * opts.batch_tasks caps the tasks per wave.  Errors as for tcorr_create; the
 * message of a failure is in tcorr_last_error(NULL).
 */
tcorr_status tcorr_batch_create(tcorr_batch_t *out, int n, const tcorr_problem *problems,
                                const tcorr_opts *opts, void *stream);

/* Number of problems in the batch (-1 for NULL). */
int tcorr_batch_size(tcorr_batch_t b);

/* Energies of every problem: e_out (host, [n][3] doubles) receives E[4], E[5],
 * E(T) of each.  Synchronous on the batch's stream. */
tcorr_status tcorr_batch_energy(tcorr_batch_t b, double *e_out);

/* Tensor-core tile of problem idx: tile[0] = b values per pair tile (pb, with
 * 128/pb values of c), tile[1] = K chunks per accumulator block.  {0, 0} for
 * FP64 batches.  EINVAL if idx is out of range. */
tcorr_status tcorr_batch_tile(tcorr_batch_t b, int idx, int *tile);

/* Waves per energy call and the number of kernel launches they make. */
tcorr_status tcorr_batch_plan(tcorr_batch_t b, int64_t *waves, int64_t *launches);

/* As tcorr_kernel_times / tcorr_device_bytes / tcorr_last_error / tcorr_destroy. */
tcorr_status tcorr_batch_kernel_times(tcorr_batch_t b, double *ms, int64_t *launches, int reset);
int64_t tcorr_batch_device_bytes(tcorr_batch_t b);
const char *tcorr_batch_last_error(tcorr_batch_t b);
tcorr_status tcorr_batch_destroy(tcorr_batch_t b);

/*
 * Server: continuous batching of (T) jobs that arrive over time (each job
 * the operation above; its tasks are the restricted loop of Sec. 3, of equal
 * weight, Sec. 5, so tasks of different jobs can share a wave).
 *
 * Jobs are submitted at any time and queue in arrival order.  Each
 * tcorr_server_step admits queued jobs, in order, while their device
 * footprint fits the memory budget (layout preparation runs on the device,
 * allocations are stream-ordered from the server's own pool), then enqueues
 * one wave: tasks of every running job, each job first taking an equal share
 * of the wave scratch and the remainder going to the oldest jobs, cut into
 * segments of the same kernels the other handles use.  A job that arrives while
 * others run joins the next wave; a job whose last tasks are in a wave gets
 * its Kahan sum at the end of that wave and frees its memory when the wave
 * completes.  Up to three waves are in flight; a step blocks only when all
 * three are.  The per-task work does not depend on which other jobs share a
 * wave, so a job's energies are bit-identical alone and in any mix.
 * Device waits are bounded: a wave whose wait expires fails the jobs that were
 * running (TCORR_ETIMEOUT) and the server continues with the next jobs.
 */
typedef struct tcorr_server_s *tcorr_server_t;

typedef enum {
    TCORR_JOB_QUEUED = 0,   /* submitted, not yet admitted */
    TCORR_JOB_RUNNING = 1,  /* admitted: state resident on the device, tasks in waves */
    TCORR_JOB_DONE = 2,     /* energies available from tcorr_server_poll */
    TCORR_JOB_FAILED = 3    /* see the status of tcorr_server_poll */
} tcorr_job_state;

/*
 * Create a server.  opts: prec, profile, test_stall as for tcorr_create;
 * batch_tasks caps the tasks per wave (0 = 4096); wave_mb sizes the wave
 * scratch (0 = 2048 MiB): a job whose single task needs more is rejected at
 * submit.  hbm_bytes: device memory for admitted jobs' resident state
 * (0 = 80% of the free memory after the server's own scratch).  host_inputs
 * must be 0 (jobs pass device arrays).  Errors as for tcorr_create; the
 * message of a failure is in tcorr_last_error(NULL).
 */
tcorr_status tcorr_server_create(tcorr_server_t *out, const tcorr_opts *opts, int64_t hbm_bytes,
                                 void *stream);

/*
 * Queue a job; *id receives its identifier (0, 1, 2, ... in submit order).
 * The problem's arrays are device pointers in the layouts of tcorr_create and
 * must stay valid and unchanged until the job is DONE or FAILED.  Errors:
 * EINVAL (bad problem), ENOMEM (footprint above the whole budget, or a
 * single task above the wave scratch).  Does not touch the device.
 */
tcorr_status tcorr_server_submit(tcorr_server_t s, const tcorr_problem *p, int64_t *id);

/*
 * One scheduling step (see above).  *pending (may be NULL) receives the
 * number of jobs not yet DONE or FAILED.  Returns an error only for a
 * failure of the server itself; failed jobs are reported by poll.
 */
tcorr_status tcorr_server_step(tcorr_server_t s, int *pending);

/*
 * State of job id (non-blocking): *state a tcorr_job_state; when DONE,
 * e_out (host, 3 doubles, may be NULL) receives E[4], E[5], E(T); when FAILED,
 * *job_status (may be NULL) receives the job's tcorr_status.  EINVAL for an
 * unknown id.
 */
tcorr_status tcorr_server_poll(tcorr_server_t s, int64_t id, int *state, double *e_out,
                               int *job_status);

/* Step until every submitted job is DONE or FAILED. */
tcorr_status tcorr_server_drain(tcorr_server_t s);

/* Counters (host, 8 int64): submitted, done, failed, running, queued,
 * device bytes admitted now, peak bytes admitted, waves launched. */
tcorr_status tcorr_server_stats(tcorr_server_t s, int64_t *stats);

const char *tcorr_server_last_error(tcorr_server_t s);
/* Waits for the waves in flight, then releases everything (NULL: no-op). */
tcorr_status tcorr_server_destroy(tcorr_server_t s);

/*
 * RI-MP2 correlation energy (the paper's second workload, Sec. 2.1):
 *
 *   E_MP2 = - sum_{ij} sum_{ab} g_aibj (2 g_aibj - g_ajbi) / eps^{ab}_{ij},
 *   g_aibj = sum_gamma C^gamma_ai C^gamma_bj           (Eqs. mp2_energy, eri_sym_decomp)
 *   eps^{ab}_{ij} = e_a + e_b - e_i - e_j                (Eq. e_orb_diff)
 *
 * evaluated over the occupied pairs i <= j (Eq. tasks_rimp2) with the ERI
 * assembly and the energy fused in one kernel (g is never stored): in FP64
 * on the FP64 pipe, or -- the paper's mixed-precision variant, re-designed --
 * with the assembly on the sm_103 tensor cores in TF32 or BF16 hi + lo split
 * precision (all four products: the lo*lo term is kept, as the same-index
 * elements of i = j pairs are sums of squares; FP32 accumulation, FP32 energy
 * terms, FP64 sums).  TCORR_BF16X3 problems with fewer than 2^24
 * (pair i <= j, a, b, gamma) terms run on TF32 hi + lo operands instead (the
 * BF16 split's residual averages below 1e-6 only over more terms); their
 * results are identical to TCORR_TF32X3's.
 *
 *   eps_occ [o], eps_vir [v], C [naux][v][o] = C^gamma_ai (row-major float64;
 *   device pointers, or host pointers with opts.host_inputs = 1; read only
 *   during tcorr_mp2_create).
 *
 * opts.prec: TCORR_FP64, TCORR_TF32X3 or TCORR_BF16X3 (EUNSUPPORTED for
 * TCORR_FP64_OZ, and for the split precisions on a device other than sm_103);
 * opts.profile times the kernels (tcorr_mp2_kernel_times: class 0 = layout
 * prep, 1 = the fused pair kernel, 3 = the final sum).  The split-precision
 * kernel's device waits are bounded: ETIMEOUT if one expires.  tcorr_mp2_energy writes e_out[3] = (E_J, E_K, E_MP2) with
 * E_J = -2 sum g^2/eps (Coulomb) and E_K = +sum g_aibj g_ajbi/eps (exchange).
 * Errors as for tcorr_create; create failures in tcorr_mp2_last_error(NULL).
 */
typedef struct tcorr_mp2_s *tcorr_mp2_t;
tcorr_status tcorr_mp2_create(tcorr_mp2_t *out, int o, int v, int naux, const double *eps_occ,
                              const double *eps_vir, const double *C, const tcorr_opts *opts,
                              void *stream);
tcorr_status tcorr_mp2_energy(tcorr_mp2_t h, double *e_out);
tcorr_status tcorr_mp2_kernel_times(tcorr_mp2_t h, double *ms, int64_t *launches, int reset);
int64_t tcorr_mp2_device_bytes(tcorr_mp2_t h);
const char *tcorr_mp2_last_error(tcorr_mp2_t h);
tcorr_status tcorr_mp2_destroy(tcorr_mp2_t h);

/*
 * Allocation-free variant (the paper has no counterpart; it exists for
 * callers that must not allocate device memory: applications whose device
 * memory is owned entirely by their own pool or budget, and latency-sensitive
 * loops that cannot afford cudaMalloc/cudaFree, which synchronise the device).
 *
 * E[4] and E[5] share of one task (i <= j <= k) in FP64, computed from the
 * caller's canonical device arrays (same layouts as tcorr_create, device
 * pointers only), written to e_out (device pointer, 2 doubles).  Every
 * intermediate lives in one fixed file-scope device array of
 * TCORR_NOALLOC_SCRATCH_BYTES that each GPU loading the library holds until
 * the process exits; no call allocates or frees memory.
 *  - Sizes: 1 <= v <= TCORR_NOALLOC_MAX_V, 1 <= o <= 4096; anything else,
 *    a NULL pointer or an unsorted/out-of-range task returns EINVAL before
 *    any device work.
 *  - The first call on a device resolves the scratch address for that device
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.
 *  - Asynchronous on stream (NULL = legacy default stream): e_out is valid
 *    once the stream has been synchronised.
 *  - The scratch is shared by every call on a device and keeps the last
 *    call's contents (nothing in it needs to start at zero).  Calls that
 *    overlap on the GPU (other streams, other host threads) race on it:
 *    serialise them.
 */
#define TCORR_NOALLOC_MAX_V 64
#define TCORR_NOALLOC_SCRATCH_BYTES 6299648
tcorr_status tcorr_task_energy_noalloc(int o, int v, const double *eps_occ,
                                       const double *eps_vir, const double *t1,
                                       const double *t2, const double *vvvo,
                                       const double *ooov, const double *ovov,
                                       int i, int j, int k, double *e_out,
                                       void *stream);

#ifdef __cplusplus
}
#endif

#endif /* TCORR_H */
