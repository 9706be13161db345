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

#include "runtime.cuh"

using namespace tcorr;
using namespace tcorr::rt;

namespace {

const char *kStatusNames[] = {"TCORR_OK", "TCORR_EINVAL", "TCORR_ENOMEM",
                              "TCORR_ECUDA", "TCORR_ETIMEOUT", "TCORR_EUNSUPPORTED"};

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

int tcorr_version(void) { return 3; }

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
        const int64_t u_task = 3 * dm.ug;
        const size_t u_task_bytes = (size_t)u_task * u_elem_bytes(ex.prec);
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        if (op.batch_tasks > 0) {
            hs->batch = op.batch_tasks;
        } else {
            // U scratch of up to 16 GiB (an eighth of the free memory at most):
            // fewer waves per call, each of which drains the kernels and ends
            // with a task reduction on as many SMs as it has tasks
            size_t budget = std::min<size_t>((size_t)16 << 30, free_b / 8);
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
        if (is_split(ex.prec) && op.tune == 1) fill_desc(ex, pb, tuned_pb(ex, pb));
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
            u_task_max = std::max<int64_t>(u_task_max, 3 * dm.ug);
            norb_max = std::max<int64_t>(norb_max, epilogue_orbits(dm.v));
        }
        // 2 GiB of U per wave: fewer wave boundaries (each drains the GEMM and the
        // epilogue) measured faster than waves sized for L2 (96 MiB: 0.83x of one
        // handle per molecule in BF16x3; 512 MiB: 0.99x; 2 GiB: 1.02x)
        const size_t wave_bytes = (size_t)(op.wave_mb > 0 ? op.wave_mb : 2048) << 20;
        ex.u_cap = std::max<int64_t>(u_task_max, (int64_t)(wave_bytes / ueb));
        ex.wave_tasks = op.batch_tasks > 0 ? op.batch_tasks : ((int64_t)1 << 40);
        // partials: room for as many tasks as the U scratch can hold of the smallest problem
        int64_t u_task_min = u_task_max;
        for (int m = 0; m < n; m++) {
            const Dims dm = make_dims(problems[m].o, problems[m].v);
            u_task_min = std::min<int64_t>(u_task_min, 3 * dm.ug);
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
            const int t = ex.prec == TCORR_FP64 ? 0 : (is_split(ex.prec) ? model_pb(p.v) : 8);
            fill_desc(ex, pb, t ? t : 8);
            if (is_split(ex.prec) && op.tune == 1) {
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
    tile[1] = b->ex.prec == TCORR_FP64 ? 0 : (is_split(b->ex.prec) ? TC_KB : 1);
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
