// Host runtime shared by the C ABI front ends: see runtime.cuh.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "runtime.cuh"

namespace tcorr {
namespace rt {

thread_local std::string g_create_error;

void dfree(Exec &ex, void *p, size_t bytes) {
    if (!p) return;
    auto it = std::find(ex.dev.begin(), ex.dev.end(), p);
    if (it != ex.dev.end()) ex.dev.erase(it);
    if (ex.pool) cudaFreeAsync(p, ex.stream);
    else cudaFree(p);
    ex.bytes -= (bytes ? bytes : 16);
}

void hfree(Exec &ex, void *p) {
    if (!p) return;
    auto it = std::find(ex.host.begin(), ex.host.end(), p);
    if (it != ex.host.end()) ex.host.erase(it);
    cudaFreeHost(p);
}

void release(Exec &ex) {
    for (void *p : ex.dev) {
        if (ex.pool) cudaFreeAsync(p, ex.stream);
        else cudaFree(p);
    }
    ex.bytes = 0;
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

// Accumulate the recorded event pairs; call after a stream synchronisation.
void resolve_timers(Exec &ex) {
    std::vector<Exec::Pending> keep;
    for (auto &pe : ex.pending) {
        if (cudaEventQuery(pe.b) == cudaErrorNotReady) {  // still in flight: keep for later
            keep.push_back(pe);
            continue;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
            ex.k_ms[pe.cls] += ms;
            ex.k_launch[pe.cls] += 1;
        }
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    cudaGetLastError();
    ex.pending.swap(keep);
}

double problem_flops(int o, int v) {
    const double tasks = (double)o * (o + 1) * (o + 2) / 6.0 - o;  // i = j = k tasks carry no work
    return tasks * 12.0 * (double)v * v * v * (double)(v + o);
}

int operand_prec(int prec, int o, int v) {
    if (prec == TCORR_BF16X3 && problem_flops(o, v) < BF16_MIN_FLOPS) return TCORR_TF32X3;
    return prec;
}

int elem_kind(int prec) { return prec == TCORR_FP64 ? 0 : (prec == TCORR_TF32X3 ? 1 : (prec == TCORR_BF16X3 ? 2 : 3)); }
bool is_split(int prec) { return prec == TCORR_TF32X3 || prec == TCORR_BF16X3; }
bool fp64_epilogue(int prec) { return prec == TCORR_FP64 || prec == TCORR_FP64_OZ; }
size_t elem_bytes(int prec) { return prec == TCORR_FP64 ? 8 : (prec == TCORR_TF32X3 ? 4 : 2); }
size_t u_elem_bytes(int prec) { return fp64_epilogue(prec) ? 8 : 4; }
// operand planes per element: 1 (FP64), 2 (hi + lo), or the FP64-emulation slices
static size_t operand_planes(int prec) { return prec == TCORR_FP64 ? 1 : (is_split(prec) ? 2 : (size_t)oz_slices()); }

// Streams a host array of v rows of `row` doubles to the device in chunks of
// up to 512 MB and calls consume(stage, d0, nr) for each, which enqueues the
// chunk's kernels on ex.stream.  Two staging buffers and a copy stream of
// its own: the copy of chunk n+1 overlaps the kernels of chunk n (the host
// array should be pinned for the copies to run asynchronously).
struct CopyPipe {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[5] = {};  // start, copied[2], used[2]
    ~CopyPipe() {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
    }
};
template <typename F>
static void stream_rows(Exec &ex, const double *host, size_t row, int v, F consume) {
    size_t rows_per = (size_t)((512ull << 20) / (row * sizeof(double)));
    if (rows_per < 1) rows_per = 1;
    if (rows_per > (size_t)v) rows_per = v;
    const int nbuf = rows_per < (size_t)v ? 2 : 1;
    double *stage[2] = {nullptr, nullptr};
    for (int b = 0; b < nbuf; b++) dalloc(ex, stage[b], rows_per * row * sizeof(double));
    CopyPipe cp;
    CK(cudaStreamCreateWithFlags(&cp.cs, cudaStreamNonBlocking));
    for (cudaEvent_t &e : cp.ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventRecord(cp.ev[0], ex.stream));  // the buffers exist in ex.stream's order
    CK(cudaStreamWaitEvent(cp.cs, cp.ev[0], 0));
    int k = 0;
    for (int d0 = 0; d0 < v; d0 += (int)rows_per, k++) {
        const int nr = (int)((size_t)(v - d0) < rows_per ? (size_t)(v - d0) : rows_per);
        const int b = k % nbuf;
        if (k >= nbuf) CK(cudaStreamWaitEvent(cp.cs, cp.ev[3 + b], 0));  // chunk k - nbuf consumed
        CK(cudaMemcpyAsync(stage[b], host + (size_t)d0 * row, nr * row * sizeof(double), cudaMemcpyHostToDevice,
                           cp.cs));
        CK(cudaEventRecord(cp.ev[1 + b], cp.cs));
        CK(cudaStreamWaitEvent(ex.stream, cp.ev[1 + b], 0));
        consume(stage[b], d0, nr);
        CK(cudaEventRecord(cp.ev[3 + b], ex.stream));
    }
    for (int b = 0; b < nbuf; b++) free_tmp(ex, stage[b], rows_per * row);  // synchronises ex.stream
    CK(cudaStreamSynchronize(cp.cs));
}

// FP64 emulation: the operands as oz_slices() BF16 slice planes under one
// power-of-two scale per operand side (exponents computed on the device from
// max |vvvo|, |t2|, |ooov|, so nothing here waits for the device).
static void build_operands_oz(Exec &ex, Problem &pb, const double *t2, const double *vvvo, const double *ooov,
                              bool host) {
    const int o = pb.dm.o, v = pb.dm.v, dp = pb.dm.dp, lp = pb.dm.lp;
    const int64_t v2 = (int64_t)v * v;
    const size_t S = (size_t)oz_slices();
    const size_t nG = (size_t)o * v2 * dp, nT2K = (size_t)o * v2 * lp;
    const size_t nT2R = (size_t)o * o * v * dp, nAoN = (size_t)o * o * v * lp;
    Operands &op = pb.op;
    dalloc(ex, op.G, nG * 2 * S);
    dalloc(ex, op.T2K, nT2K * 2 * S);
    dalloc(ex, op.T2R, nT2R * 2 * S);
    dalloc(ex, op.AoN, nAoN * 2 * S);
    dalloc(ex, pb.oz_max, 3 * sizeof(unsigned long long));
    dalloc(ex, pb.oz_e, 2 * sizeof(int));
    Timer tm(ex, KC_PREP);
    CK(cudaMemsetAsync(pb.oz_max, 0, 3 * sizeof(unsigned long long), ex.stream));
    CK(cudaMemsetAsync(op.G, 0, nG * 2 * S, ex.stream));
    double *tmp_t2 = nullptr, *tmp_oo = nullptr;
    const double *dt2 = device_view(ex, t2, (size_t)o * o * v2, host, tmp_t2);
    const double *doo = device_view(ex, ooov, (size_t)o * o * o * v, host, tmp_oo);
    const size_t row = (size_t)v2 * o;  // doubles per d row of vvvo
    if (!host) {
        CK(launch_maxabs(vvvo, (int64_t)(row * v), pb.oz_max, ex.stream));
    } else {
        double m = 0.0;
        for (size_t k = 0; k < row * v; k++) m = std::max(m, std::fabs(vvvo[k]));
        CK(launch_seed_max(pb.oz_max, m, ex.stream));
    }
    CK(launch_maxabs(dt2, (int64_t)o * o * v2, pb.oz_max + 1, ex.stream));
    CK(launch_maxabs(doo, (int64_t)o * o * o * v, pb.oz_max + 2, ex.stream));
    CK(launch_oz_exponents(pb.oz_max, pb.oz_e, ex.stream));
    const int *eA = pb.oz_e, *eB = pb.oz_e + 1;
    // G[p][q][xy][d] = slices of vvvo[d][xy][q]
    if (!host) {
        CK(launch_slice_pad(vvvo, op.G, v2, v, v, o, o, (int64_t)row, 1, dp, (int64_t)v2 * dp, (int64_t)nG, eA, 1.0,
                            ex.stream));
    } else {
        stream_rows(ex, vvvo, row, v, [&](const double *stage, int d0, int nr) {
            char *g = static_cast<char *>(op.G) + (size_t)d0 * 2;
            CK(launch_slice_pad(stage, g, v2, nr, nr, o, o, (int64_t)row, 1, dp, (int64_t)v2 * dp, (int64_t)nG, eA,
                                1.0, ex.stream));
        });
    }
    // T2K[p][q][xy][l] = slices of t2[q][l][xy]; T2R[p][spa][d] = slices of t2[spa][d]
    CK(launch_slice_pad(dt2, op.T2K, o, o, lp, v2, (int64_t)o * v2, v2, 1, (int64_t)v2 * lp, lp, (int64_t)nT2K, eA,
                        1.0, ex.stream));
    CK(launch_slice_pad(dt2, op.T2R, (int64_t)o * o * v, v, dp, 1, v, 1, 0, dp, 0, (int64_t)nT2R, eB, 1.0,
                        ex.stream));
    // AoN[p][qsa][l] = slices of -ooov[l][qsa]
    CK(launch_slice_pad(doo, op.AoN, 1, o, lp, (int64_t)o * o * v, 0, (int64_t)o * o * v, 1, 0, lp, (int64_t)nAoN,
                        eB, -1.0, ex.stream));
    tm.stop();
    free_tmp(ex, tmp_t2, (size_t)o * o * v2);
    free_tmp(ex, tmp_oo, (size_t)o * o * o * v);
}

void build_operands(Exec &ex, Problem &pb, const double *t2, const double *vvvo, const double *ooov,
                    bool host) {
    if (ex.prec == TCORR_FP64_OZ) {
        build_operands_oz(ex, pb, t2, vvvo, ooov, host);
        return;
    }
    const int o = pb.dm.o, v = pb.dm.v, dp = pb.dm.dp, lp = pb.dm.lp;
    const int64_t v2 = (int64_t)v * v;
    const int pprec = operand_prec(ex.prec, o, v);
    const int kind = elem_kind(pprec);
    const size_t eb = elem_bytes(pprec);
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
        stream_rows(ex, vvvo, row, v, [&](const double *stage, int d0, int nr) {
            char *ghi = static_cast<char *>(op.G) + (size_t)d0 * eb;
            char *glo = split ? static_cast<char *>(op.Glo) + (size_t)d0 * eb : nullptr;
            CK(launch_transpose_pad(kind, stage, ghi, glo, v2, nr, nr, o, o, (int64_t)row, 1, dp,
                                    (int64_t)v2 * dp, 1.0, ex.stream));
        });
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
    if (fp64_epilogue(ex.prec)) {
        dalloc(ex, pb.t1, (size_t)o * v * sizeof(double));
        dalloc(ex, pb.ovov, nov2 * sizeof(double));
        CK(cudaMemcpyAsync(pb.t1, t1, (size_t)o * v * sizeof(double), kd, ex.stream));
        CK(cudaMemcpyAsync(pb.ovov, ovov, nov2 * sizeof(double), kd, ex.stream));
        if (ex.prec == TCORR_FP64_OZ) {  // the emulation's epilogue works in float-float
            dalloc(ex, pb.evf, (size_t)v * sizeof(float2));
            CK(launch_epilogue_ff_inputs(static_cast<double *>(pb.t1), static_cast<double *>(pb.ovov), pb.eps_v,
                                         pb.evf, o, v, ex.stream));
        }
    } else {
        const size_t vp = epi_vp(v);
        dalloc(ex, pb.t1, (size_t)o * vp * sizeof(float));
        dalloc(ex, pb.ovov, (size_t)o * o * vp * vp * sizeof(float));
        dalloc(ex, pb.evf, vp * sizeof(float2));
        double *tmp1 = nullptr, *tmp2 = nullptr;
        const double *d1 = device_view(ex, t1, (size_t)o * v, host, tmp1);
        const double *d2 = device_view(ex, ovov, nov2, host, tmp2);
        CK(launch_epilogue_f32_inputs(d1, d2, pb.eps_v, static_cast<float *>(pb.t1), static_cast<float *>(pb.ovov),
                                      pb.evf, o, v, (int)vp, ex.stream));
        free_tmp(ex, tmp1, (size_t)o * v);
        free_tmp(ex, tmp2, nov2);
    }
}

void build_schedule(Exec &ex, Problem &pb) {
    const int64_t o = pb.dm.o;
    pb.ntask = o * (o + 1) * (o + 2) / 6;
    const int nb = (pb.dm.v + EPI_TE - 1) / EPI_TE;
    pb.norb = nb * (nb + 1) * (nb + 2) / 6;
    dalloc(ex, pb.tasks, (size_t)pb.ntask * 3 * sizeof(int));
    dalloc(ex, pb.task_e, (size_t)pb.ntask * 2 * sizeof(double));
    dalloc(ex, pb.orbits, (size_t)pb.norb * 3 * sizeof(int));
    CK(cudaMemsetAsync(pb.task_e, 0, (size_t)pb.ntask * 2 * sizeof(double), ex.stream));
    CK(launch_build_tables(pb.dm.o, nb, pb.tasks, pb.orbits, ex.stream));
}

// Device bytes of one problem's resident data (operands, epilogue inputs, tables).
size_t problem_bytes(const Dims &d, int prec) {
    prec = operand_prec(prec, d.o, d.v);
    const size_t o = d.o, v = d.v, v2 = v * v;
    const size_t eb = elem_bytes(prec), parts = operand_planes(prec);
    size_t b = parts * eb * (o * v2 * d.dp + o * v2 * d.lp + o * o * v * d.dp + o * o * v * d.lp);
    const size_t ve = fp64_epilogue(prec) ? v : (size_t)epi_vp((int)v);  // FP32 inputs are padded
    b += (o * o * ve * ve + o * ve) * u_elem_bytes(prec) + (o + v) * 8 + ve * 8;
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
    d.evf = pb.evf;
    d.tasks = pb.tasks;
    d.orbits = pb.orbits;
    d.task_e = pb.task_e;
    pb.u_task = 3 * pb.dm.ug;
    if (ex.prec == TCORR_FP64) {
        pb.gemm_units = f64_units_per_task(pb.dm);
    } else if (ex.prec == TCORR_FP64_OZ) {
        std::string msg;
        if (oz_fill_desc(d, pb.op, pb.oz_e, msg) != cudaSuccess) throw Fail{TCORR_EUNSUPPORTED, msg};
        pb.gemm_units = oz_units_per_task(d);
    } else {
        std::string msg;
        if (tc_fill_desc(d, operand_prec(ex.prec, pb.dm.o, pb.dm.v), pb.op, pbt, TC_KB, ex.pair, msg) != cudaSuccess)
            throw Fail{TCORR_EUNSUPPORTED, msg};
        if (epi_fill_desc(d, msg) != cudaSuccess) throw Fail{TCORR_EUNSUPPORTED, msg};
        pb.gemm_units = tc_units_per_task(d);
    }
}

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
            else if (ex.prec == TCORR_FP64_OZ) CK(launch_ugemm_oz(ex.sm_count, w, st));
            else CK(launch_ugemm_tc(ex.prec, ex.sm_count, w, st, ex.pair));
            tm.stop();
        }
        {
            Timer tm(ex, KC_EPI);
            CK(launch_epilogue(ex.prec, ex.sm_count, w, st));
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
    if (op.prec < TCORR_FP64 || op.prec > TCORR_FP64_OZ || op.batch_tasks < 0 ||
        (op.host_inputs != 0 && op.host_inputs != 1) || (op.tune != 0 && op.tune != 1) ||
        (op.eager != 0 && op.eager != 1) || op.wave_mb < 0 || (op.single_sm != 0 && op.single_sm != 1)) {
        msg = "invalid option (precision, batch_tasks, host_inputs, tune, eager, wave_mb or single_sm)";
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
    ex.pair = op.single_sm == 0;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&ex.sm_count, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&ex.cc_major, cudaDevAttrComputeCapabilityMajor, dev));
    CK(cudaDeviceGetAttribute(&ex.cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
    if (ex.prec != TCORR_FP64 && !tc_supported(ex.cc_major, ex.cc_minor))
        throw Fail{TCORR_EUNSUPPORTED, "mixed precision needs the sm_103 tensor-core path (device is sm_" +
                                           std::to_string(ex.cc_major * 10 + ex.cc_minor) + ")"};
    if (is_split(ex.prec)) {  // kernel attributes, before any capture
        CK(tc_prepare(ex.prec));
        CK(epi_prepare());
    }
    if (ex.prec == TCORR_FP64_OZ) CK(oz_prepare());
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
    const int pprec = operand_prec(ex.prec, pb.dm.o, pb.dm.v);
    const auto key = std::make_tuple(pprec * 2 + (ex.pair ? 1 : 0), pb.dm.o, pb.dm.v);
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
        if (tc_fill_desc(d, pprec, pb.op, cand, TC_KB, ex.pair, msg) != cudaSuccess) continue;
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
            CK(launch_ugemm_tc(ex.prec, ex.sm_count, w, ex.stream, ex.pair));
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


}  // namespace rt
}  // namespace tcorr
