// C ABI of libtcorr (declared in include/tcorr.h): handle life cycle, input
// validation, footprint check, layout preparation (S0), the task schedule
// (S1: the collapsed i <= j <= k loop of Sec. 3, cut into waves), and the
// launch sequence W contractions (S2/S3) -> fused epilogue (S4) -> Kahan
// reductions (S5) for every wave.  A single handle holds one problem; a
// batch handle holds many problems of uneven (o, v) that share the waves.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "tcorr_internal.cuh"

using namespace tcorr;

namespace {

thread_local std::string g_create_error;

const char *kStatusNames[] = {"TCORR_OK", "TCORR_EINVAL", "TCORR_ENOMEM",
                              "TCORR_ECUDA", "TCORR_ETIMEOUT", "TCORR_EUNSUPPORTED"};

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
    void *ovov = nullptr;    // FP64 or FP32 copy [o][v][o][v]
    float *dev_f = nullptr;  // FP32 block-relative virtual energies (mixed epilogue)
    int64_t ntask = 0;
    int *tasks = nullptr;      // device [ntask][3]
    double *task_e = nullptr;  // device [ntask][2] (E4, E5 share)
    int norb = 0;              // epilogue block orbits per task
    int *orbits = nullptr;     // device [norb][3]
    int64_t u_task = 0;        // U elements per task: 3 v v vc
    int64_t gemm_units = 0;    // W-contraction work units per task
    InstDesc desc{};           // host copy
};

// Execution state: stream, scratch, device descriptors, error flag, timers.
struct Exec {
    int prec = TCORR_FP64;
    int profile = 0;
    int inject_stall = 0;
    int sm_count = 0, cc_major = 0, cc_minor = 0;
    cudaStream_t stream = nullptr;
    size_t bytes = 0;              // device bytes held
    std::vector<void *> dev;       // every device allocation
    std::vector<void *> host;      // every pinned host allocation

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
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Fail{TCORR_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                     cudaGetErrorString(e)};
    }
    ex.dev.push_back(p);
    ex.bytes += bytes;
    ptr = static_cast<T *>(p);
}

void dfree(Exec &ex, void *p, size_t bytes) {
    if (!p) return;
    auto it = std::find(ex.dev.begin(), ex.dev.end(), p);
    if (it != ex.dev.end()) ex.dev.erase(it);
    cudaFree(p);
    ex.bytes -= (bytes ? bytes : 16);
}

template <typename T>
void halloc(Exec &ex, T *&ptr, size_t bytes) {
    void *p = nullptr;
    CK(cudaMallocHost(&p, bytes ? bytes : 16));
    ex.host.push_back(p);
    ptr = static_cast<T *>(p);
}

void hfree(Exec &ex, void *p) {
    if (!p) return;
    auto it = std::find(ex.host.begin(), ex.host.end(), p);
    if (it != ex.host.end()) ex.host.erase(it);
    cudaFreeHost(p);
}

void release(Exec &ex) {
    for (void *p : ex.dev) cudaFree(p);
    for (void *p : ex.host) cudaFreeHost(p);
    for (auto &pe : ex.pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    ex.dev.clear();
    ex.host.clear();
    ex.pending.clear();
}

// Copy (or reference) one caller array on the device.  For host inputs the
// data is staged into a temporary device buffer that free_tmp releases.
const double *device_view(Exec &ex, const double *src, size_t n, bool host, double *&tmp) {
    tmp = nullptr;
    if (!host) return src;
    dalloc(ex, tmp, n * sizeof(double));
    CK(cudaMemcpyAsync(tmp, src, n * sizeof(double), cudaMemcpyHostToDevice, ex.stream));
    return tmp;
}

void free_tmp(Exec &ex, double *&tmp, size_t n) {
    if (!tmp) return;
    CK(cudaStreamSynchronize(ex.stream));
    dfree(ex, tmp, n * sizeof(double));
    tmp = nullptr;
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

// Accumulate the recorded event pairs; call after a stream synchronisation.
void resolve_timers(Exec &ex) {
    for (auto &pe : ex.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
            ex.k_ms[pe.cls] += ms;
            ex.k_launch[pe.cls] += 1;
        }
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    ex.pending.clear();
}

int elem_kind(int prec) { return prec == TCORR_FP64 ? 0 : (prec == TCORR_TF32X3 ? 1 : 2); }
size_t elem_bytes(int prec) { return prec == TCORR_FP64 ? 8 : (prec == TCORR_TF32X3 ? 4 : 2); }
size_t u_elem_bytes(int prec) { return prec == TCORR_FP64 ? 8 : 4; }
constexpr int EPI_TE = 8;  // epilogue cube edge

Dims make_dims(int o, int v) { return Dims{o, v, round_up(v, KPAD), round_up(o, KPAD), round_up(v, UPAD)}; }

void build_operands(Exec &ex, Problem &pb, const double *t2, const double *vvvo, const double *ooov,
                    bool host) {
    const int o = pb.dm.o, v = pb.dm.v, dp = pb.dm.dp, lp = pb.dm.lp;
    const int64_t v2 = (int64_t)v * v;
    const int kind = elem_kind(ex.prec);
    const size_t eb = elem_bytes(ex.prec);
    const bool split = ex.prec != TCORR_FP64;
    const size_t nG = (size_t)o * v2 * dp, nT2K = (size_t)o * v2 * lp;
    const size_t nT2R = (size_t)o * o * v * dp, nAoN = (size_t)o * o * v * lp;
    Operands &op = pb.op;
    dalloc(ex, op.G, nG * eb);
    dalloc(ex, op.T2K, nT2K * eb);
    dalloc(ex, op.T2R, nT2R * eb);
    dalloc(ex, op.AoN, nAoN * eb);
    if (split) {
        dalloc(ex, op.Glo, nG * eb);
        dalloc(ex, op.T2Klo, nT2K * eb);
        dalloc(ex, op.T2Rlo, nT2R * eb);
        dalloc(ex, op.AoNlo, nAoN * eb);
    }
    Timer tm(ex, KC_PREP);
    // G[q][xy][d] = vvvo[d][xy][q]; staged in chunks of d rows for host inputs
    CK(cudaMemsetAsync(op.G, 0, nG * eb, ex.stream));
    if (split) CK(cudaMemsetAsync(op.Glo, 0, nG * eb, ex.stream));
    const size_t row = (size_t)v2 * o;  // doubles per d row of vvvo
    if (!host) {
        CK(launch_transpose_pad(kind, vvvo, op.G, op.Glo, v2, v, v, o, o, (int64_t)row, 1, dp,
                                (int64_t)v2 * dp, 1.0, ex.stream));
    } else {
        size_t rows_per = (size_t)((512ull << 20) / (row * sizeof(double)));
        if (rows_per < 1) rows_per = 1;
        if (rows_per > (size_t)v) rows_per = v;
        double *stage = nullptr;
        dalloc(ex, stage, rows_per * row * sizeof(double));
        for (int d0 = 0; d0 < v; d0 += (int)rows_per) {
            const int nr = (int)((size_t)(v - d0) < rows_per ? (size_t)(v - d0) : rows_per);
            CK(cudaMemcpyAsync(stage, vvvo + (size_t)d0 * row, nr * row * sizeof(double),
                               cudaMemcpyHostToDevice, ex.stream));
            char *ghi = static_cast<char *>(op.G) + (size_t)d0 * eb;
            char *glo = split ? static_cast<char *>(op.Glo) + (size_t)d0 * eb : nullptr;
            CK(launch_transpose_pad(kind, stage, ghi, glo, v2, nr, nr, o, o, (int64_t)row, 1, dp,
                                    (int64_t)v2 * dp, 1.0, ex.stream));
        }
        free_tmp(ex, stage, rows_per * row);
    }
    double *tmp_t2 = nullptr, *tmp_oo = nullptr;
    const double *dt2 = device_view(ex, t2, (size_t)o * o * v2, host, tmp_t2);
    // T2K[q][xy][l] = t2[q][l][xy]
    CK(launch_transpose_pad(kind, dt2, op.T2K, op.T2Klo, o, o, lp, v2, (int64_t)o * v2, v2, 1,
                            (int64_t)v2 * lp, lp, 1.0, ex.stream));
    // T2R[spa][d] = t2[spa][d]  (row copy with padding: C = 1)
    CK(launch_transpose_pad(kind, dt2, op.T2R, op.T2Rlo, (int64_t)o * o * v, v, dp, 1, v, 1, 0,
                            dp, 0, 1.0, ex.stream));
    const double *doo = device_view(ex, ooov, (size_t)o * o * o * v, host, tmp_oo);
    // AoN[qsa][l] = -ooov[l][qsa]
    CK(launch_transpose_pad(kind, doo, op.AoN, op.AoNlo, 1, o, lp, (int64_t)o * o * v, 0,
                            (int64_t)o * o * v, 1, 0, lp, -1.0, ex.stream));
    tm.stop();
    free_tmp(ex, tmp_t2, (size_t)o * o * v2);
    free_tmp(ex, tmp_oo, (size_t)o * o * o * v);
}

void build_epilogue_inputs(Exec &ex, Problem &pb, const double *eps_occ, const double *eps_vir,
                           const double *t1, const double *ovov, bool host) {
    const int o = pb.dm.o, v = pb.dm.v;
    const size_t nov2 = (size_t)o * v * o * v;
    dalloc(ex, pb.eps_o, o * sizeof(double));
    dalloc(ex, pb.eps_v, v * sizeof(double));
    const cudaMemcpyKind kd = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(pb.eps_o, eps_occ, o * sizeof(double), kd, ex.stream));
    CK(cudaMemcpyAsync(pb.eps_v, eps_vir, v * sizeof(double), kd, ex.stream));
    if (ex.prec == TCORR_FP64) {
        dalloc(ex, pb.t1, (size_t)o * v * sizeof(double));
        dalloc(ex, pb.ovov, nov2 * sizeof(double));
        CK(cudaMemcpyAsync(pb.t1, t1, (size_t)o * v * sizeof(double), kd, ex.stream));
        CK(cudaMemcpyAsync(pb.ovov, ovov, nov2 * sizeof(double), kd, ex.stream));
    } else {
        dalloc(ex, pb.t1, (size_t)o * v * sizeof(float));
        dalloc(ex, pb.ovov, nov2 * sizeof(float));
        double *tmp1 = nullptr, *tmp2 = nullptr;
        const double *d1 = device_view(ex, t1, (size_t)o * v, host, tmp1);
        CK(launch_to_float(d1, static_cast<float *>(pb.t1), (int64_t)o * v, ex.stream));
        const double *d2 = device_view(ex, ovov, nov2, host, tmp2);
        CK(launch_to_float(d2, static_cast<float *>(pb.ovov), (int64_t)nov2, ex.stream));
        free_tmp(ex, tmp1, (size_t)o * v);
        free_tmp(ex, tmp2, nov2);
        dalloc(ex, pb.dev_f, v * sizeof(float));
        CK(launch_block_deltas(pb.eps_v, pb.dev_f, v, EPI_TE, ex.stream));
    }
}

void build_schedule(Exec &ex, Problem &pb) {
    const int o = pb.dm.o;
    std::vector<int> tl;
    for (int i = 0; i < o; i++)
        for (int j = i; j < o; j++)
            for (int k = j; k < o; k++) {
                tl.push_back(i);
                tl.push_back(j);
                tl.push_back(k);
            }
    pb.ntask = (int64_t)tl.size() / 3;
    dalloc(ex, pb.tasks, tl.size() * sizeof(int));
    CK(cudaMemcpy(pb.tasks, tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice));
    dalloc(ex, pb.task_e, (size_t)pb.ntask * 2 * sizeof(double));
    CK(cudaMemsetAsync(pb.task_e, 0, (size_t)pb.ntask * 2 * sizeof(double), ex.stream));
    const int nb = (pb.dm.v + EPI_TE - 1) / EPI_TE;
    std::vector<int> ob;
    for (int a = 0; a < nb; a++)
        for (int b = a; b < nb; b++)
            for (int c = b; c < nb; c++) {
                ob.push_back(a);
                ob.push_back(b);
                ob.push_back(c);
            }
    pb.norb = (int)(ob.size() / 3);
    dalloc(ex, pb.orbits, ob.size() * sizeof(int));
    CK(cudaMemcpy(pb.orbits, ob.data(), ob.size() * sizeof(int), cudaMemcpyHostToDevice));
}

// Device bytes of one problem's resident data (operands, epilogue inputs, tables).
size_t problem_bytes(const Dims &d, int prec) {
    const size_t o = d.o, v = d.v, v2 = v * v;
    const size_t eb = elem_bytes(prec), parts = prec == TCORR_FP64 ? 1 : 2;
    size_t b = parts * eb * (o * v2 * d.dp + o * v2 * d.lp + o * o * v * d.dp + o * o * v * d.lp);
    b += (o * o * v2 + o * v) * u_elem_bytes(prec) + (o + v) * 8 + v * 4;
    const size_t nb = (v + EPI_TE - 1) / EPI_TE;
    b += nb * (nb + 1) * (nb + 2) / 6 * 12;
    b += o * (o + 1) * (o + 2) / 6 * 28;
    return b;
}
size_t host_staging_bytes(const Dims &d) {
    const size_t o = d.o, v = d.v;
    return std::max<size_t>(o * o * v * v * 8, (size_t)512 << 20);
}

// Tensor-core tile of a problem shape.  Cost model: every (pair tile, N
// pass) unit costs the same, so take the pb with the fewest tiles; ties go to
// pb = 8 (16-wide c rows), then pb = 4.
int model_pb(int v) {
    int best = 8;
    int64_t best_tiles = -1;
    for (int pb : {8, 4, 16}) {
        const int pc = 128 / pb;
        const int64_t t = (int64_t)((v + pb - 1) / pb) * ((v + pc - 1) / pc);
        if (best_tiles < 0 || t < best_tiles) { best = pb; best_tiles = t; }
    }
    return best;
}
constexpr int TC_KB = 2;  // K chunks per accumulator block (accuracy: see gemm_tc.cu)

void fill_desc(Exec &ex, Problem &pb, int pbt) {
    InstDesc &d = pb.desc;
    d.dm = pb.dm;
    d.norb = pb.norb;
    d.G = pb.op.G;
    d.T2K = pb.op.T2K;
    d.T2R = pb.op.T2R;
    d.AoN = pb.op.AoN;
    d.eps_o = pb.eps_o;
    d.eps_v = pb.eps_v;
    d.t1 = pb.t1;
    d.ovov = pb.ovov;
    d.dev_f = pb.dev_f;
    d.tasks = pb.tasks;
    d.orbits = pb.orbits;
    d.task_e = pb.task_e;
    pb.u_task = (int64_t)3 * pb.dm.v * pb.dm.v * pb.dm.vc;
    if (ex.prec == TCORR_FP64) {
        pb.gemm_units = f64_units_per_task(pb.dm);
    } else {
        std::string msg;
        if (tc_fill_desc(d, ex.prec, pb.op, pbt, TC_KB, msg) != cudaSuccess) throw Fail{TCORR_EUNSUPPORTED, msg};
        pb.gemm_units = tc_units_per_task(d);
    }
}

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

Plan make_plan(const Exec &ex, const std::vector<Problem *> &pbs, const std::vector<Span> &spans) {
    Plan pl;
    WaveRec cur{0, 0, 0, 0, 0, 0};
    int64_t u_used = 0, p_used = 0, t_used = 0;
    auto close = [&]() {
        if (cur.nseg > 0) pl.waves.push_back(cur);
        cur = WaveRec{(int)pl.segs.size(), 0, 0, 0, 0, 0};
        u_used = p_used = t_used = 0;
    };
    for (const Span &sp : spans) {
        const Problem &pb = *pbs[sp.inst];
        int64_t t = sp.first, left = sp.count;
        while (left > 0) {
            const int64_t fit_u = (ex.u_cap - u_used) / pb.u_task;
            const int64_t fit_p = (ex.part_cap - p_used) / ((int64_t)pb.norb * 2);
            const int64_t fit_t = ex.wave_tasks - t_used;
            const int64_t fit_e = ((int64_t)0x7fffffff - cur.n_epi) / pb.norb;
            const int64_t n = std::min({left, fit_u, fit_p, fit_t, fit_e});
            if (n <= 0) {
                if (cur.nseg == 0) throw Fail{TCORR_ENOMEM, "wave scratch smaller than one task"};
                close();
                continue;
            }
            Seg s{};
            s.inst = sp.inst;
            s.ntb = (int)n;
            s.task0 = t;
            s.u_off = u_used;
            s.gemm0 = cur.n_gemm;
            s.epi0 = cur.n_epi;
            s.red0 = cur.n_red;
            s.part_off = p_used;
            pl.segs.push_back(s);
            cur.nseg++;
            cur.tc_brows = std::max(cur.tc_brows, pb.desc.brows);
            cur.n_gemm += n * pb.gemm_units;
            cur.n_epi += n * pb.norb;
            cur.n_red += n;
            u_used += n * pb.u_task;
            p_used += n * (int64_t)pb.norb * 2;
            t_used += n;
            t += n;
            left -= n;
        }
        pl.sums.push_back(SumSpan{pb.task_e, sp.first, sp.count, nullptr});
    }
    close();
    return pl;
}

// Uploads the plan's tables (one copy from pinned staging); returns the
// device segment and span arrays.
void upload_plan(Exec &ex, Plan &pl, Seg *&d_segs, SumSpan *&d_spans) {
    const size_t seg_b = pl.segs.size() * sizeof(Seg);
    const size_t span_off = (seg_b + 255) / 256 * 256;
    const size_t total = span_off + pl.sums.size() * sizeof(SumSpan);
    if ((int)pl.sums.size() > ex.sums_cap || total > ex.stage_cap) {
        CK(cudaStreamSynchronize(ex.stream));  // the old tables may still be in use
        if ((int)pl.sums.size() > ex.sums_cap) {
            dfree(ex, ex.d_sums, (size_t)ex.sums_cap * 3 * sizeof(double));
            dalloc(ex, ex.d_sums, pl.sums.size() * 3 * sizeof(double));
            hfree(ex, ex.h_sums);
            halloc(ex, ex.h_sums, pl.sums.size() * 3 * sizeof(double));
            ex.sums_cap = (int)pl.sums.size();
        }
        if (total > ex.stage_cap) {
            dfree(ex, ex.d_stage, ex.stage_cap);
            dalloc(ex, ex.d_stage, total);
            hfree(ex, ex.h_stage);
            halloc(ex, ex.h_stage, total);
            ex.stage_cap = total;
        }
    }
    for (size_t n = 0; n < pl.sums.size(); n++) pl.sums[n].out = ex.d_sums + 3 * n;
    memcpy(ex.h_stage, pl.segs.data(), seg_b);
    memcpy(ex.h_stage + span_off, pl.sums.data(), pl.sums.size() * sizeof(SumSpan));
    CK(cudaMemcpyAsync(ex.d_stage, ex.h_stage, total, cudaMemcpyHostToDevice, ex.stream));
    d_segs = reinterpret_cast<Seg *>(ex.d_stage);
    d_spans = reinterpret_cast<SumSpan *>(ex.d_stage + span_off);
}

// The launch sequence of a plan on stream st (no host synchronisation).
void launch_plan(Exec &ex, const Plan &pl, const Seg *d_segs, const SumSpan *d_spans, cudaStream_t st) {
    for (const WaveRec &wr : pl.waves) {
        Wave w{};
        w.descs = ex.d_descs;
        w.segs = d_segs + wr.seg0;
        w.nseg = wr.nseg;
        w.n_gemm = wr.n_gemm;
        w.n_epi = wr.n_epi;
        w.n_red = wr.n_red;
        w.U = ex.U;
        w.partials = ex.partials;
        w.err = ex.err;
        w.inject_stall = ex.inject_stall;
        w.tc_brows = wr.tc_brows;
        {
            Timer tm(ex, KC_GEMM);
            if (ex.prec == TCORR_FP64) CK(launch_ugemm_f64(w, st));
            else CK(launch_ugemm_tc(ex.prec, ex.sm_count, w, st));
            tm.stop();
        }
        {
            Timer tm(ex, KC_EPI);
            CK(launch_epilogue(ex.prec, w, st));
            tm.stop();
        }
        {
            Timer tm(ex, KC_RED);
            CK(launch_task_reduce(w, st));
            tm.stop();
        }
    }
    Timer tm(ex, KC_RED);
    CK(launch_span_sums(d_spans, (int)pl.sums.size(), st));
    tm.stop();
}

void check_err_flag(Exec &ex) {
    CK(cudaMemcpyAsync(ex.h_err, ex.err, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
    CK(cudaStreamSynchronize(ex.stream));
    if (*ex.h_err) {
        const int e = *ex.h_err;
        *ex.h_err = 0;
        CK(cudaMemsetAsync(ex.err, 0, sizeof(int), ex.stream));
        if (e & (DERR_TIMEOUT_FULL | DERR_TIMEOUT_EMPTY | DERR_TIMEOUT_TMEM))
            throw Fail{TCORR_ETIMEOUT, "device pipeline wait expired (flags " + std::to_string(e) + ")"};
        throw Fail{TCORR_ECUDA, "device reported bad configuration (flags " + std::to_string(e) + ")"};
    }
}

// Copies the span sums back, waits, resolves timers, checks the error flag.
void finish_call(Exec &ex, int nspans) {
    CK(cudaMemcpyAsync(ex.h_sums, ex.d_sums, (size_t)nspans * 3 * sizeof(double), cudaMemcpyDeviceToHost,
                       ex.stream));
    CK(cudaStreamSynchronize(ex.stream));
    resolve_timers(ex);
    check_err_flag(ex);
}

// ---- create-time helpers ------------------------------------------------------
tcorr_status check_opts(const tcorr_opts &op, std::string &msg) {
    if (op.test_stall != 0 && op.test_stall != 1) {
        msg = "test_stall must be 0 or 1";
        return TCORR_EINVAL;
    }
    if (op.prec < TCORR_FP64 || op.prec > TCORR_BF16X3 || op.batch_tasks < 0 ||
        (op.host_inputs != 0 && op.host_inputs != 1) || (op.tune != 0 && op.tune != 1) ||
        (op.eager != 0 && op.eager != 1) || op.wave_mb < 0) {
        msg = "invalid option (precision, batch_tasks, host_inputs, tune, eager or wave_mb)";
        return TCORR_EINVAL;
    }
    return TCORR_OK;
}

bool sizes_supported(int o, int v) {
    const int64_t v64 = v, o64 = o;
    return !(v64 * v64 * v64 * o64 > ((int64_t)1 << 40) || o > 4096 || v > 8192);
}

void init_exec(Exec &ex, const tcorr_opts &op, void *stream) {
    ex.stream = static_cast<cudaStream_t>(stream);
    ex.prec = op.prec;
    ex.profile = op.profile;
    ex.inject_stall = op.test_stall;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&ex.sm_count, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&ex.cc_major, cudaDevAttrComputeCapabilityMajor, dev));
    CK(cudaDeviceGetAttribute(&ex.cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
    if (ex.prec != TCORR_FP64 && !tc_supported(ex.cc_major, ex.cc_minor))
        throw Fail{TCORR_EUNSUPPORTED, "mixed precision needs the sm_103 tensor-core path (device is sm_" +
                                           std::to_string(ex.cc_major * 10 + ex.cc_minor) + ")"};
    if (ex.prec != TCORR_FP64) CK(tc_prepare(ex.prec));  // kernel attributes, before any capture
}

void build_problem(Exec &ex, Problem &pb, int o, int v, const double *eps_occ, const double *eps_vir,
                   const double *t1, const double *t2, const double *vvvo, const double *ooov,
                   const double *ovov, bool host) {
    pb.dm = make_dims(o, v);
    build_operands(ex, pb, t2, vvvo, ooov, host);
    build_epilogue_inputs(ex, pb, eps_occ, eps_vir, t1, ovov, host);
    build_schedule(ex, pb);
}

void alloc_common(Exec &ex) {
    dalloc(ex, ex.err, sizeof(int));
    CK(cudaMemsetAsync(ex.err, 0, sizeof(int), ex.stream));
    halloc(ex, ex.h_err, sizeof(int));
    *ex.h_err = 0;
}

void upload_descs(Exec &ex, const std::vector<Problem *> &pbs) {
    std::vector<InstDesc> hd(pbs.size());
    for (size_t n = 0; n < pbs.size(); n++) hd[n] = pbs[n]->desc;
    dalloc(ex, ex.d_descs, hd.size() * sizeof(InstDesc));
    CK(cudaMemcpy(ex.d_descs, hd.data(), hd.size() * sizeof(InstDesc), cudaMemcpyHostToDevice));
}

// Measured tile choice: times the W contraction of a few tasks of the problem
// for each candidate pb and keeps the fastest.  Results are cached per
// (precision, o, v) for the life of the process.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune_cache;

int tuned_pb(Exec &ex, Problem &pb) {
    const auto key = std::make_tuple(ex.prec, pb.dm.o, pb.dm.v);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) return it->second;
    }
    // tasks to time: the scratch's worth, at most 16 (skip i = j = k: the first task)
    const int64_t first = pb.ntask > 1 ? 1 : 0;
    const int64_t n = std::max<int64_t>(1, std::min<int64_t>({pb.ntask - first, 16, ex.u_cap / pb.u_task}));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = model_pb(pb.dm.v);
    float best_ms = -1.f;
    InstDesc *d_one = nullptr;
    Seg *d_seg = nullptr;
    dalloc(ex, d_one, sizeof(InstDesc));
    dalloc(ex, d_seg, sizeof(Seg));
    for (int cand : {8, 4, 16}) {
        InstDesc d = pb.desc;
        std::string msg;
        if (tc_fill_desc(d, ex.prec, pb.op, cand, TC_KB, msg) != cudaSuccess) continue;
        Seg s{};
        s.ntb = (int)n;
        s.task0 = first;
        CK(cudaMemcpy(d_one, &d, sizeof(InstDesc), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(d_seg, &s, sizeof(Seg), cudaMemcpyHostToDevice));
        Wave w{};
        w.descs = d_one;
        w.segs = d_seg;
        w.nseg = 1;
        w.n_gemm = n * tc_units_per_task(d);
        w.U = ex.U;
        w.err = ex.err;
        w.tc_brows = d.brows;
        float ms_min = -1.f;
        for (int rep = 0; rep < 3; rep++) {
            CK(cudaEventRecord(e0, ex.stream));
            CK(launch_ugemm_tc(ex.prec, ex.sm_count, w, ex.stream));
            CK(cudaEventRecord(e1, ex.stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (rep > 0 && (ms_min < 0 || ms < ms_min)) ms_min = ms;
        }
        if (best_ms < 0 || ms_min < best_ms * 0.97f) { best = cand; best_ms = ms_min; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(ex, d_one, sizeof(InstDesc));
    dfree(ex, d_seg, sizeof(Seg));
    check_err_flag(ex);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
    return best;
}

}  // namespace

// ---- handles -------------------------------------------------------------------
struct tcorr_s {
    Exec ex;
    Problem pb;
    int batch = 1;  // tasks per wave
};

struct tcorr_batch_s {
    Exec ex;
    std::vector<Problem> pbs;
    std::vector<int> pbt;  // tile pb per problem (0 for FP64)
    Plan plan;
    Seg *d_segs = nullptr;
    SumSpan *d_spans = nullptr;
    bool eager = false;
    cudaGraphExec_t graph = nullptr;
    cudaStream_t cap_stream = nullptr;
};

namespace {

void run_range(tcorr_s &hs, int64_t first, int64_t count, double *e_out, double *e_task) {
    Exec &ex = hs.ex;
    std::vector<Problem *> pbs{&hs.pb};
    Plan pl = make_plan(ex, pbs, {Span{0, first, count}});
    Seg *d_segs = nullptr;
    SumSpan *d_spans = nullptr;
    upload_plan(ex, pl, d_segs, d_spans);
    launch_plan(ex, pl, d_segs, d_spans, ex.stream);
    if (e_task)
        CK(cudaMemcpyAsync(e_task, hs.pb.task_e + 2 * first, (size_t)count * 2 * sizeof(double),
                           cudaMemcpyDeviceToHost, ex.stream));
    finish_call(ex, 1);
    e_out[0] = ex.h_sums[0];
    e_out[1] = ex.h_sums[1];
    e_out[2] = ex.h_sums[2];
}

void destroy_batch(tcorr_batch_s *b) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    release(b->ex);
    delete b;
}

}  // namespace

extern "C" {

int tcorr_version(void) { return 2; }

const char *tcorr_status_string(tcorr_status s) {
    if ((int)s < 0 || (int)s > 5) return "TCORR_UNKNOWN";
    return kStatusNames[(int)s];
}

const char *tcorr_last_error(tcorr_t h) {
    if (!h) return g_create_error.c_str();
    return h->ex.last_error.c_str();
}

tcorr_status tcorr_create(tcorr_t *out, int o, int v, const double *eps_occ,
                          const double *eps_vir, const double *t1, const double *t2,
                          const double *vvvo, const double *ooov, const double *ovov,
                          const tcorr_opts *opts, void *stream) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return TCORR_EINVAL;
    }
    *out = nullptr;
    if (o < 1 || v < 1 || !eps_occ || !eps_vir || !t1 || !t2 || !vvvo || !ooov || !ovov) {
        g_create_error = "o, v must be >= 1 and every array pointer non-NULL";
        return TCORR_EINVAL;
    }
    tcorr_opts op{};
    if (opts) op = *opts;
    {
        const tcorr_status st = check_opts(op, g_create_error);
        if (st != TCORR_OK) return st;
    }
    if (!sizes_supported(o, v)) {
        g_create_error = "sizes beyond the supported range";
        return TCORR_EUNSUPPORTED;
    }
    tcorr_s *hs = new (std::nothrow) tcorr_s();
    if (!hs) {
        g_create_error = "host allocation failed";
        return TCORR_ENOMEM;
    }
    Exec &ex = hs->ex;
    Problem &pb = hs->pb;
    try {
        init_exec(ex, op, stream);
        const Dims dm = make_dims(o, v);
        const int64_t ntask = (int64_t)o * (o + 1) * (o + 2) / 6;
        const int64_t u_task = (int64_t)3 * v * v * dm.vc;
        const size_t u_task_bytes = (size_t)u_task * u_elem_bytes(ex.prec);
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        if (op.batch_tasks > 0) {
            hs->batch = op.batch_tasks;
        } else {
            size_t budget = std::min<size_t>((size_t)4 << 30, free_b / 8);
            int64_t b = (int64_t)(budget / u_task_bytes);
            hs->batch = (int)std::max<int64_t>(1, std::min<int64_t>(b, std::min<int64_t>(ntask, 4096)));
        }
        if (hs->batch > ntask) hs->batch = (int)ntask;
        const int norb = epilogue_orbits(v);
        const size_t need = problem_bytes(dm, ex.prec) + (size_t)hs->batch * u_task_bytes +
                            (size_t)hs->batch * norb * 16 + (op.host_inputs ? host_staging_bytes(dm) : 0) +
                            (64u << 20);
        if (need > free_b)
            throw Fail{TCORR_ENOMEM, "footprint " + std::to_string(need) + " bytes exceeds free device memory " +
                                         std::to_string(free_b)};
        build_problem(ex, pb, o, v, eps_occ, eps_vir, t1, t2, vvvo, ooov, ovov, op.host_inputs == 1);
        ex.wave_tasks = hs->batch;
        ex.u_cap = (int64_t)hs->batch * u_task;
        ex.part_cap = (int64_t)hs->batch * pb.norb * 2;
        dalloc(ex, ex.U, (size_t)ex.u_cap * u_elem_bytes(ex.prec));
        dalloc(ex, ex.partials, (size_t)ex.part_cap * sizeof(double));
        alloc_common(ex);
        fill_desc(ex, pb, model_pb(v));
        if (ex.prec != TCORR_FP64 && op.tune == 1) fill_desc(ex, pb, tuned_pb(ex, pb));
        upload_descs(ex, {&pb});
        {   // staging for the largest plan (the whole task list), so that calls do not allocate
            Plan pl = make_plan(ex, {&pb}, {Span{0, 0, pb.ntask}});
            Seg *ds = nullptr;
            SumSpan *dsp = nullptr;
            upload_plan(ex, pl, ds, dsp);
        }
        CK(cudaStreamSynchronize(ex.stream));
        CK(cudaGetLastError());
        resolve_timers(ex);
    } catch (const Fail &f) {
        g_create_error = f.msg;
        cudaStreamSynchronize(ex.stream);
        cudaGetLastError();
        release(ex);
        delete hs;
        return f.st;
    } catch (const std::bad_alloc &) {
        g_create_error = "host allocation failed";
        release(ex);
        delete hs;
        return TCORR_ENOMEM;
    }
    *out = hs;
    return TCORR_OK;
}

int64_t tcorr_num_tasks(tcorr_t h) { return h ? h->pb.ntask : -1; }

tcorr_status tcorr_task(tcorr_t h, int64_t idx, int *ijk) {
    if (!h || !ijk) return TCORR_EINVAL;
    if (idx < 0 || idx >= h->pb.ntask) {
        h->ex.last_error = "task index out of range";
        return TCORR_EINVAL;
    }
    // inverse of the lexicographic enumeration of i <= j <= k
    const int o = h->pb.dm.o;
    int64_t n = idx;
    for (int i = 0; i < o; i++) {
        const int64_t m = (int64_t)(o - i) * (o - i + 1) / 2;  // tasks with this i
        if (n >= m) { n -= m; continue; }
        for (int j = i; j < o; j++) {
            const int64_t mj = o - j;
            if (n >= mj) { n -= mj; continue; }
            ijk[0] = i;
            ijk[1] = j;
            ijk[2] = j + (int)n;
            return TCORR_OK;
        }
    }
    return TCORR_EINVAL;
}

tcorr_status tcorr_energy_range(tcorr_t hh, int64_t first, int64_t count, double *e_out,
                                double *e_task) {
    if (!hh) return TCORR_EINVAL;
    Exec &ex = hh->ex;
    ex.last_error.clear();
    if (!e_out || first < 0 || count < 0 || first + count > hh->pb.ntask) {
        ex.last_error = "e_out is NULL or the range leaves the task list";
        return TCORR_EINVAL;
    }
    try {
        if (count == 0) {
            e_out[0] = e_out[1] = e_out[2] = 0.0;
            return TCORR_OK;
        }
        run_range(*hh, first, count, e_out, e_task);
    } catch (const Fail &f) {
        ex.last_error = f.msg;
        cudaStreamSynchronize(ex.stream);
        cudaGetLastError();
        return f.st;
    }
    return TCORR_OK;
}

tcorr_status tcorr_energy(tcorr_t h, double *e_out) {
    if (!h) return TCORR_EINVAL;
    return tcorr_energy_range(h, 0, h->pb.ntask, e_out, nullptr);
}

static tcorr_status kernel_times(Exec &ex, double *ms, int64_t *launches, int reset) {
    for (int c = 0; c < KC_COUNT; c++) {
        if (ms) ms[c] = ex.k_ms[c];
        if (launches) launches[c] = ex.k_launch[c];
        if (reset) { ex.k_ms[c] = 0; ex.k_launch[c] = 0; }
    }
    return TCORR_OK;
}

tcorr_status tcorr_kernel_times(tcorr_t hh, double *ms, int64_t *launches, int reset) {
    if (!hh) return TCORR_EINVAL;
    return kernel_times(hh->ex, ms, launches, reset);
}

int64_t tcorr_device_bytes(tcorr_t h) { return h ? (int64_t)h->ex.bytes : -1; }

tcorr_status tcorr_destroy(tcorr_t h) {
    if (!h) return TCORR_OK;
    cudaStreamSynchronize(h->ex.stream);
    release(h->ex);
    delete h;
    return TCORR_OK;
}

// ---- batch -------------------------------------------------------------------------

tcorr_status tcorr_batch_create(tcorr_batch_t *out, int n, const tcorr_problem *problems,
                                const tcorr_opts *opts, void *stream) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return TCORR_EINVAL;
    }
    *out = nullptr;
    if (n < 1 || !problems) {
        g_create_error = "n must be >= 1 and problems non-NULL";
        return TCORR_EINVAL;
    }
    tcorr_opts op{};
    if (opts) op = *opts;
    {
        const tcorr_status st = check_opts(op, g_create_error);
        if (st != TCORR_OK) return st;
    }
    for (int m = 0; m < n; m++) {
        const tcorr_problem &p = problems[m];
        if (p.o < 1 || p.v < 1 || !p.eps_occ || !p.eps_vir || !p.t1 || !p.t2 || !p.vvvo || !p.ooov ||
            !p.ovov) {
            g_create_error = "problem " + std::to_string(m) + ": o, v must be >= 1 and every array non-NULL";
            return TCORR_EINVAL;
        }
        if (!sizes_supported(p.o, p.v)) {
            g_create_error = "problem " + std::to_string(m) + ": sizes beyond the supported range";
            return TCORR_EUNSUPPORTED;
        }
    }
    tcorr_batch_s *b = new (std::nothrow) tcorr_batch_s();
    if (!b) {
        g_create_error = "host allocation failed";
        return TCORR_ENOMEM;
    }
    Exec &ex = b->ex;
    try {
        init_exec(ex, op, stream);
        b->eager = op.eager == 1 || op.profile != 0 || op.test_stall != 0;
        const size_t ueb = u_elem_bytes(ex.prec);
        size_t need = 64u << 20, stage = 0;
        int64_t u_task_max = 0, norb_max = 0;
        for (int m = 0; m < n; m++) {
            const Dims dm = make_dims(problems[m].o, problems[m].v);
            need += problem_bytes(dm, ex.prec);
            if (op.host_inputs) stage = std::max(stage, host_staging_bytes(dm));
            u_task_max = std::max<int64_t>(u_task_max, (int64_t)3 * dm.v * dm.v * dm.vc);
            norb_max = std::max<int64_t>(norb_max, epilogue_orbits(dm.v));
        }
        const size_t wave_bytes = (size_t)(op.wave_mb > 0 ? op.wave_mb : 96) << 20;
        ex.u_cap = std::max<int64_t>(u_task_max, (int64_t)(wave_bytes / ueb));
        ex.wave_tasks = op.batch_tasks > 0 ? op.batch_tasks : ((int64_t)1 << 40);
        // partials: room for as many tasks as the U scratch can hold of the smallest problem
        int64_t u_task_min = u_task_max;
        for (int m = 0; m < n; m++) {
            const Dims dm = make_dims(problems[m].o, problems[m].v);
            u_task_min = std::min<int64_t>(u_task_min, (int64_t)3 * dm.v * dm.v * dm.vc);
        }
        const int64_t max_wave_tasks = std::min<int64_t>(ex.wave_tasks, ex.u_cap / u_task_min + 1);
        ex.part_cap = std::max<int64_t>(norb_max * 2, max_wave_tasks * norb_max * 2);
        need += (size_t)ex.u_cap * ueb + (size_t)ex.part_cap * 8 + stage;
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        if (need > free_b)
            throw Fail{TCORR_ENOMEM, "footprint " + std::to_string(need) + " bytes exceeds free device memory " +
                                         std::to_string(free_b)};
        dalloc(ex, ex.U, (size_t)ex.u_cap * ueb);
        dalloc(ex, ex.partials, (size_t)ex.part_cap * sizeof(double));
        alloc_common(ex);
        b->pbs.resize(n);
        b->pbt.assign(n, 0);
        for (int m = 0; m < n; m++) {
            const tcorr_problem &p = problems[m];
            Problem &pb = b->pbs[m];
            build_problem(ex, pb, p.o, p.v, p.eps_occ, p.eps_vir, p.t1, p.t2, p.vvvo, p.ooov, p.ovov,
                          op.host_inputs == 1);
            const int t = ex.prec == TCORR_FP64 ? 0 : model_pb(p.v);
            fill_desc(ex, pb, t ? t : 8);
            if (ex.prec != TCORR_FP64 && op.tune == 1) {
                const int tt = tuned_pb(ex, pb);
                fill_desc(ex, pb, tt);
                b->pbt[m] = tt;
            } else {
                b->pbt[m] = t;
            }
        }
        std::vector<Problem *> pp(n);
        std::vector<Span> spans(n);
        for (int m = 0; m < n; m++) {
            pp[m] = &b->pbs[m];
            spans[m] = Span{m, 0, b->pbs[m].ntask};
        }
        upload_descs(ex, pp);
        b->plan = make_plan(ex, pp, spans);
        upload_plan(ex, b->plan, b->d_segs, b->d_spans);
        CK(cudaStreamSynchronize(ex.stream));
        CK(cudaGetLastError());
        resolve_timers(ex);
    } catch (const Fail &f) {
        g_create_error = f.msg;
        cudaStreamSynchronize(ex.stream);
        cudaGetLastError();
        destroy_batch(b);
        return f.st;
    } catch (const std::bad_alloc &) {
        g_create_error = "host allocation failed";
        destroy_batch(b);
        return TCORR_ENOMEM;
    }
    *out = b;
    return TCORR_OK;
}

int tcorr_batch_size(tcorr_batch_t b) { return b ? (int)b->pbs.size() : -1; }

tcorr_status tcorr_batch_energy(tcorr_batch_t b, double *e_out) {
    if (!b) return TCORR_EINVAL;
    Exec &ex = b->ex;
    ex.last_error.clear();
    if (!e_out) {
        ex.last_error = "e_out is NULL";
        return TCORR_EINVAL;
    }
    try {
        if (b->eager) {
            launch_plan(ex, b->plan, b->d_segs, b->d_spans, ex.stream);
        } else {
            if (!b->graph) {
                // capture on a private stream (the caller's may be the legacy default stream)
                CK(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
                cudaGraph_t g = nullptr;
                CK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
                try {
                    launch_plan(ex, b->plan, b->d_segs, b->d_spans, b->cap_stream);
                } catch (...) {
                    cudaStreamEndCapture(b->cap_stream, &g);
                    if (g) cudaGraphDestroy(g);
                    throw;
                }
                CK(cudaStreamEndCapture(b->cap_stream, &g));
                const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
                cudaGraphDestroy(g);
                CK(e);
            }
            CK(cudaGraphLaunch(b->graph, ex.stream));
        }
        finish_call(ex, (int)b->pbs.size());
        for (size_t m = 0; m < b->pbs.size(); m++)
            for (int c = 0; c < 3; c++) e_out[3 * m + c] = ex.h_sums[3 * m + c];
    } catch (const Fail &f) {
        ex.last_error = f.msg;
        cudaStreamSynchronize(ex.stream);
        cudaGetLastError();
        return f.st;
    }
    return TCORR_OK;
}

tcorr_status tcorr_batch_tile(tcorr_batch_t b, int idx, int *tile) {
    if (!b || !tile || idx < 0 || idx >= (int)b->pbs.size()) return TCORR_EINVAL;
    tile[0] = b->pbt[idx];
    tile[1] = b->ex.prec == TCORR_FP64 ? 0 : TC_KB;
    return TCORR_OK;
}

tcorr_status tcorr_batch_plan(tcorr_batch_t b, int64_t *waves, int64_t *launches) {
    if (!b) return TCORR_EINVAL;
    if (waves) *waves = (int64_t)b->plan.waves.size();
    if (launches) *launches = 3 * (int64_t)b->plan.waves.size() + 1;
    return TCORR_OK;
}

tcorr_status tcorr_batch_kernel_times(tcorr_batch_t b, double *ms, int64_t *launches, int reset) {
    if (!b) return TCORR_EINVAL;
    return kernel_times(b->ex, ms, launches, reset);
}

int64_t tcorr_batch_device_bytes(tcorr_batch_t b) { return b ? (int64_t)b->ex.bytes : -1; }

const char *tcorr_batch_last_error(tcorr_batch_t b) {
    if (!b) return g_create_error.c_str();
    return b->ex.last_error.c_str();
}

tcorr_status tcorr_batch_destroy(tcorr_batch_t b) {
    if (!b) return TCORR_OK;
    cudaStreamSynchronize(b->ex.stream);
    destroy_batch(b);
    return TCORR_OK;
}

}  // extern "C"
