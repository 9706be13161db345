// Host runtime shared by the C ABI front ends (single problem, batch,
// server): problem preparation (S0/S1), wave planning and the launch
// sequence of S2-S5, allocation and error plumbing.
#pragma once

#include <string>
#include <vector>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace rt {

constexpr int EPI_TE = 8;  // epilogue cube edge
// padded virtual extent of the FP32 epilogue inputs (t1 rows, ovov slabs)
inline int epi_vp(int v) { return (v + EPI_TE - 1) / EPI_TE * EPI_TE; }
constexpr int TC_KB = 2;   // K chunks per tensor-core accumulator block (accuracy: see gemm_tc.cu)

extern thread_local std::string g_create_error;

struct Fail {
    tcorr_status st;
    std::string msg;
};

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            throw Fail{TCORR_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)

// One (T) problem resident on the device: re-laid-out operands, epilogue
// inputs, its task list and per-task energies, and its kernel descriptor.
struct Problem {
    Dims dm{};
    Operands op;
    double *eps_o = nullptr, *eps_v = nullptr;  // FP64
    void *t1 = nullptr;      // FP64 or FP32 copy
    void *ovov = nullptr;    // FP64 copy [o][v][o][v] or FP32 blocks (see launch_epilogue_f32_inputs)
    float2 *evf = nullptr;   // mixed paths and FP64 emulation: eps_v as float-float pairs
    int64_t ntask = 0;
    int *tasks = nullptr;      // device [ntask][3]
    double *task_e = nullptr;  // device [ntask][2] (E4, E5 share)
    int norb = 0;              // epilogue block orbits per task
    int *orbits = nullptr;     // device [norb][3]
    int64_t u_task = 0;        // U elements per task: 3 ug
    unsigned long long *oz_max = nullptr;  // FP64 emulation: device [3] max |vvvo|, |t2|, |ooov| (bit patterns)
    int *oz_e = nullptr;                   // FP64 emulation: device [2] scale exponents
    int64_t gemm_units = 0;    // W-contraction work units per task
    InstDesc desc{};           // host copy
};

// Execution state: stream, scratch, device descriptors, error flag, timers.
struct Exec {
    int prec = TCORR_FP64;
    int profile = 0;
    int inject_stall = 0;
    bool pair = true;              // split precisions: tensor-core tiles on SM pairs
    int sm_count = 0, cc_major = 0, cc_minor = 0;
    cudaStream_t stream = nullptr;
    size_t bytes = 0;              // device bytes held
    std::vector<void *> dev;       // every device allocation
    std::vector<void *> host;      // every pinned host allocation
    cudaMemPool_t pool = nullptr;  // set: stream-ordered allocations from this pool (freed in stream order)

    void *U = nullptr;             // wave scratch
    int64_t u_cap = 0;             // elements
    double *partials = nullptr;    // orbit partials of a wave
    int64_t part_cap = 0;          // doubles
    int64_t wave_tasks = 0;        // tasks per wave (cap)
    InstDesc *d_descs = nullptr;   // device [ninst]
    int *err = nullptr, *h_err = nullptr;

    // per-call tables: segments of every wave and the spans to sum
    unsigned char *d_stage = nullptr, *h_stage = nullptr;
    size_t stage_cap = 0;
    double *d_sums = nullptr, *h_sums = nullptr;
    int sums_cap = 0;

    struct Pending { int cls; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    double k_ms[KC_COUNT] = {0, 0, 0, 0};
    int64_t k_launch[KC_COUNT] = {0, 0, 0, 0};
    std::string last_error;
};

template <typename T>
void dalloc(Exec &ex, T *&ptr, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = ex.pool ? cudaMallocFromPoolAsync(&p, bytes, ex.pool, ex.stream) : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Fail{TCORR_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                     cudaGetErrorString(e)};
    }
    ex.dev.push_back(p);
    ex.bytes += bytes;
    ptr = static_cast<T *>(p);
}

template <typename T>
void halloc(Exec &ex, T *&ptr, size_t bytes) {
    void *p = nullptr;
    CK(cudaMallocHost(&p, bytes ? bytes : 16));
    ex.host.push_back(p);
    ptr = static_cast<T *>(p);
}

struct Timer {
    Exec &ex;
    int cls;
    cudaEvent_t a = nullptr;
    Timer(Exec &e, int c) : ex(e), cls(c) {
        if (!ex.profile) return;
        CK(cudaEventCreate(&a));
        CK(cudaEventRecord(a, ex.stream));
    }
    void stop() {
        if (!ex.profile || !a) return;
        cudaEvent_t b = nullptr;
        CK(cudaEventCreate(&b));
        CK(cudaEventRecord(b, ex.stream));
        ex.pending.push_back({cls, a, b});
        a = nullptr;
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
    }
};

// ---- waves ------------------------------------------------------------------
// A span is a contiguous task range of one problem; a plan cuts the spans of
// a call into waves that fit the scratch (U elements, orbit partials, task cap).
struct Span {
    int inst;
    int64_t first, count;
};
struct WaveRec {
    int seg0, nseg;
    int64_t n_gemm, n_epi, n_red;
    int tc_brows;  // largest tensor-core B tile of the wave's problems
};
struct Plan {
    std::vector<Seg> segs;
    std::vector<WaveRec> waves;
    std::vector<SumSpan> sums;  // span n sums into d_sums[3n .. 3n+2] (out set at upload)
};

void dfree(Exec &ex, void *p, size_t bytes);
void hfree(Exec &ex, void *p);
void release(Exec &ex);
const double *device_view(Exec &ex, const double *src, size_t n, bool host, double *&tmp);
void free_tmp(Exec &ex, double *&tmp, size_t n);
void resolve_timers(Exec &ex);
// Algorithmic flops of a problem: 12 v^3 (v + o) per task, i = j = k excluded.
double problem_flops(int o, int v);
// Operand precision of a problem run at precision prec.  A BF16 hi + lo split
// leaves up to 2^-17 of each operand unrepresented (16 significant bits); on
// E(T) that residual averages below the 1e-6 bound only over enough work:
// over seeded problems across o = 4..40, v = 20..300 the BF16X3 error reached
// 1.5e-6 on problems below 1e10 flops and at most 2.8e-7 above 1e11, while
// TF32X3 stayed within 1.4e-7 .. 2.1e-7 throughout.  So BF16X3 problems below
// BF16_MIN_FLOPS run on TF32 hi + lo operands (same three products, same
// kernels); every other precision is unchanged.
constexpr double BF16_MIN_FLOPS = TCORR_BF16_MIN_FLOPS;
int operand_prec(int prec, int o, int v);
int elem_kind(int prec);
bool is_split(int prec);     // TF32x3 / BF16x3 (hi + lo operands, FP32 U and epilogue)
bool fp64_epilogue(int prec);  // FP64 and FP64 emulation: FP64 U, epilogue inputs and epilogue
size_t elem_bytes(int prec);
size_t u_elem_bytes(int prec);
void build_operands(Exec &ex, Problem &pb, const double *t2, const double *vvvo, const double *ooov,
                    bool host);
void build_epilogue_inputs(Exec &ex, Problem &pb, const double *eps_occ, const double *eps_vir,
                           const double *t1, const double *ovov, bool host);
void build_schedule(Exec &ex, Problem &pb);
void build_problem(Exec &ex, Problem &pb, int o, int v, const double *eps_occ, const double *eps_vir,
                   const double *t1, const double *t2, const double *vvvo, const double *ooov,
                   const double *ovov, bool host);
size_t problem_bytes(const Dims &d, int prec);
size_t host_staging_bytes(const Dims &d);
int model_pb(int v);
void fill_desc(Exec &ex, Problem &pb, int pbt);
Plan make_plan(const Exec &ex, const std::vector<Problem *> &pbs, const std::vector<Span> &spans);
void upload_plan(Exec &ex, Plan &pl, Seg *&d_segs, SumSpan *&d_spans);
void launch_plan(Exec &ex, const Plan &pl, const Seg *d_segs, const SumSpan *d_spans, cudaStream_t st);
void check_err_flag(Exec &ex);
void finish_call(Exec &ex, int nspans);
tcorr_status check_opts(const tcorr_opts &op, std::string &msg);
bool sizes_supported(int o, int v);
void init_exec(Exec &ex, const tcorr_opts &op, void *stream);
void alloc_common(Exec &ex);
void upload_descs(Exec &ex, const std::vector<Problem *> &pbs);
int tuned_pb(Exec &ex, Problem &pb);

}  // namespace rt
}  // namespace tcorr
