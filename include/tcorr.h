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
                          FP32 accumulation; denominators and energy sum in FP64 (Sec. 3 mixed
                          precision, re-designed) */
    TCORR_BF16X3 = 2   /* as TF32X3 with BF16 hi+lo operands */
} tcorr_precision;

typedef struct {
    int prec;           /* tcorr_precision; 0 = TCORR_FP64 */
    int host_inputs;    /* 0: the array arguments of tcorr_create are device pointers;
                           1: they are host pointers (pageable or pinned), copied in */
    int batch_tasks;    /* tasks per internal batch, 0 = chosen from the scratch budget */
    int profile;        /* 1: time every kernel class with CUDA events (tcorr_kernel_times) */
    int test_stall;     /* testing only, 0 in normal use: 1 makes the tensor-core kernel withhold
                           one chunk's loads so that a bounded device-side wait expires; the
                           energy call then returns TCORR_ETIMEOUT and the context stays usable */
    int reserved[3];    /* must be zero */
} tcorr_opts;           /* zero-initialised = defaults */

/*
 * Create a handle for one (T) problem with o occupied and v virtual orbitals.
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
 * Errors: EINVAL (NULL pointer, o < 1, v < 1, nonzero reserved field,
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
 * Full energy.  e_out (host, 3 doubles) receives E[4], E[5], E(T).
 * Synchronous on the handle's stream.  Deterministic: the same handle
 * returns bit-identical results.
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
#define TCORR_NOALLOC_SCRATCH_BYTES 6295552
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
