// Server: continuous batching of (T) jobs (declared in include/tcorr.h).
//
// Host side of the scheduler.  Queued jobs are admitted in arrival order
// while their footprint fits the budget; admission builds the job's operand
// layouts and tables on the server stream with stream-ordered allocations
// from a private memory pool, and writes its kernel descriptor into a device
// slot.  Each step cuts one wave from the remaining tasks of the running jobs
// (equal scratch shares first, then the oldest jobs), uploads its segment
// table from a pinned ring, and enqueues the wave's kernels, the Kahan sums of
// the jobs that finish in it (written straight to mapped host memory) and a
// copy of the device error flag, then records the wave's event.  Completed
// waves retire jobs: results are read, memory is freed in stream order and
// the descriptor slot is reused.  Nothing here waits on the device except
// when the ring of in-flight waves is full.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "runtime.cuh"

using namespace tcorr;
using namespace tcorr::rt;

namespace {

constexpr int DEPTH = 3;        // waves in flight
constexpr int MAX_SLOTS = 512;  // running jobs (device descriptor slots)

__global__ void store_desc_kernel(const InstDesc d, InstDesc *dst) {
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&d);
    uint32_t *out = reinterpret_cast<uint32_t *>(dst);
    for (int w = threadIdx.x; w < (int)(sizeof(InstDesc) / 4); w += blockDim.x) out[w] = src[w];
}

struct Job {
    int64_t id = 0;
    int state = TCORR_JOB_QUEUED;
    int status = TCORR_OK;
    tcorr_problem in{};
    size_t bytes = 0;          // footprint charged against the budget
    Exec ex;                   // the job's allocations (pool, server stream)
    Problem pb;
    int slot = -1;
    int64_t next = 0;          // next task to schedule
    double e[3] = {0, 0, 0};
};

struct RingSlot {
    unsigned char *d_tab = nullptr, *h_tab = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    int *h_err = nullptr;      // pinned copy of the device error flag after the wave
    int64_t wave = -1;         // wave using this slot (-1: free)
    std::vector<Job *> finishing;
    std::vector<Job *> members;
};

size_t job_footprint(const Dims &dm, int prec) {
    // resident state plus the pool's allocation granularity for its ~14 buffers
    return problem_bytes(dm, prec) + ((size_t)32 << 20);
}

}  // namespace

struct tcorr_server_s {
    Exec ex;                       // scratch, descriptor slots, error flag
    cudaMemPool_t pool = nullptr;
    size_t budget = 0, used = 0, peak = 0;
    int64_t wave_tasks = 0;
    std::vector<int> free_slots;
    double *h_res = nullptr, *d_res = nullptr;  // mapped pinned [MAX_SLOTS][3]
    std::deque<Job *> queue;
    std::vector<Job *> running;    // admission order
    std::map<int64_t, std::unique_ptr<Job>> jobs;
    RingSlot ring[DEPTH];
    int64_t waves_issued = 0, waves_done = 0, ignore_err_before = 0;
    int64_t next_id = 0, n_done = 0, n_failed = 0;
};

namespace {

void fail_running(tcorr_server_s &s, tcorr_status st) {
    for (Job *j : s.running) {
        j->state = TCORR_JOB_FAILED;
        j->status = st;
        release(j->ex);
        s.used -= j->bytes;
        s.free_slots.push_back(j->slot);
        s.n_failed++;
    }
    s.running.clear();
    for (RingSlot &r : s.ring) {
        r.finishing.clear();
        r.members.clear();
    }
}

// Retires the oldest in-flight wave if it has completed (blocking: wait for it).
bool retire_one(tcorr_server_s &s, bool blocking) {
    if (s.waves_done == s.waves_issued) return false;
    RingSlot &r = s.ring[s.waves_done % DEPTH];
    if (blocking) {
        CK(cudaEventSynchronize(r.ev));
    } else {
        const cudaError_t q = cudaEventQuery(r.ev);
        if (q == cudaErrorNotReady) return false;
        CK(q);
    }
    const int64_t w = r.wave;
    r.wave = -1;
    s.waves_done++;
    if (*r.h_err && w >= s.ignore_err_before) {
        const int e = *r.h_err;
        CK(cudaMemsetAsync(s.ex.err, 0, sizeof(int), s.ex.stream));
        s.ignore_err_before = s.waves_issued;  // later waves already copied the stale flag
        fail_running(s, (e & (DERR_TIMEOUT_FULL | DERR_TIMEOUT_EMPTY | DERR_TIMEOUT_TMEM)) ? TCORR_ETIMEOUT
                                                                                              : TCORR_ECUDA);
        r.finishing.clear();
        r.members.clear();
        return true;
    }
    for (Job *j : r.finishing) {
        if (j->state != TCORR_JOB_RUNNING) continue;
        for (int c = 0; c < 3; c++) j->e[c] = s.h_res[3 * j->slot + c];
        j->state = TCORR_JOB_DONE;
        release(j->ex);  // stream-ordered frees: after every wave that read the job
        s.used -= j->bytes;
        s.free_slots.push_back(j->slot);
        s.running.erase(std::find(s.running.begin(), s.running.end(), j));
        s.n_done++;
    }
    r.finishing.clear();
    r.members.clear();
    return true;
}

void admit(tcorr_server_s &s) {
    while (!s.queue.empty() && !s.free_slots.empty()) {
        Job *j = s.queue.front();
        if (s.used + j->bytes > s.budget) break;  // strict arrival order
        s.queue.pop_front();
        j->slot = s.free_slots.back();
        s.free_slots.pop_back();
        s.used += j->bytes;
        s.peak = std::max(s.peak, s.used);
        j->ex.prec = s.ex.prec;
        j->ex.pair = s.ex.pair;
        j->ex.stream = s.ex.stream;
        j->ex.pool = s.pool;
        j->ex.sm_count = s.ex.sm_count;
        const tcorr_problem &p = j->in;
        try {
            build_problem(j->ex, j->pb, p.o, p.v, p.eps_occ, p.eps_vir, p.t1, p.t2, p.vvvo, p.ooov, p.ovov,
                          false);
            fill_desc(j->ex, j->pb, model_pb(p.v));
            store_desc_kernel<<<1, 128, 0, s.ex.stream>>>(j->pb.desc, s.ex.d_descs + j->slot);
            CK(cudaGetLastError());
        } catch (const Fail &f) {
            release(j->ex);
            s.used -= j->bytes;
            s.free_slots.push_back(j->slot);
            j->state = TCORR_JOB_FAILED;
            j->status = f.st;
            s.n_failed++;
            if (f.st == TCORR_ECUDA) throw;
            continue;
        }
        j->state = TCORR_JOB_RUNNING;
        j->next = 0;
        s.running.push_back(j);
    }
}

// Cuts one wave from the running jobs' remaining tasks and enqueues it.
void launch_wave(tcorr_server_s &s) {
    auto has_work = [&]() {
        for (Job *j : s.running)
            if (j->next < j->pb.ntask) return true;
        return false;
    };
    if (!has_work()) return;
    // ring full: wait for the oldest wave first (it may retire or fail jobs)
    if (s.waves_issued - s.waves_done == DEPTH) retire_one(s, true);
    std::vector<Job *> act;
    for (Job *j : s.running)
        if (j->next < j->pb.ntask) act.push_back(j);
    if (act.empty()) return;
    Exec &ex = s.ex;
    // task counts: equal shares of the U scratch, then the rest to the oldest jobs
    std::vector<int64_t> take(act.size(), 0);
    int64_t u_left = ex.u_cap, p_left = ex.part_cap, t_left = s.wave_tasks;
    int64_t e_left = 0x7fffffff;
    auto grant = [&](size_t n, int64_t want) {
        const Problem &pb = act[n]->pb;
        int64_t g = std::min({want, act[n]->pb.ntask - act[n]->next - take[n], u_left / pb.u_task,
                              p_left / ((int64_t)pb.norb * 2), t_left, e_left / pb.norb});
        if (g <= 0) return;
        take[n] += g;
        u_left -= g * pb.u_task;
        p_left -= g * (int64_t)pb.norb * 2;
        t_left -= g;
        e_left -= g * pb.norb;
    };
    for (size_t n = 0; n < act.size(); n++)
        grant(n, std::max<int64_t>(1, ex.u_cap / ((int64_t)act.size() * act[n]->pb.u_task)));
    for (size_t n = 0; n < act.size(); n++) grant(n, INT64_MAX);
    // segments (one per job) and the sums of the jobs that finish
    std::vector<Seg> segs;
    std::vector<SumSpan> sums;
    std::vector<Job *> finishing, members;
    WaveRec wr{0, 0, 0, 0, 0, 0};
    int64_t u_off = 0, p_off = 0;
    for (size_t n = 0; n < act.size(); n++) {
        if (take[n] == 0) continue;
        Job *j = act[n];
        Seg sg{};
        sg.inst = j->slot;
        sg.ntb = (int)take[n];
        sg.task0 = j->next;
        sg.u_off = u_off;
        sg.gemm0 = wr.n_gemm;
        sg.epi0 = wr.n_epi;
        sg.red0 = wr.n_red;
        sg.part_off = p_off;
        segs.push_back(sg);
        wr.nseg++;
        wr.tc_brows = std::max(wr.tc_brows, j->pb.desc.brows);
        wr.n_gemm += take[n] * j->pb.gemm_units;
        wr.n_epi += take[n] * j->pb.norb;
        wr.n_red += take[n];
        u_off += take[n] * j->pb.u_task;
        p_off += take[n] * (int64_t)j->pb.norb * 2;
        j->next += take[n];
        members.push_back(j);
        if (j->next == j->pb.ntask) {
            sums.push_back(SumSpan{j->pb.task_e, 0, j->pb.ntask, s.d_res + 3 * j->slot});
            finishing.push_back(j);
        }
    }
    if (segs.empty()) throw Fail{TCORR_ECUDA, "wave scheduler made no progress"};
    RingSlot &r = s.ring[s.waves_issued % DEPTH];
    const size_t seg_b = segs.size() * sizeof(Seg);
    const size_t span_off = (seg_b + 255) / 256 * 256;
    const size_t total = span_off + std::max<size_t>(1, sums.size()) * sizeof(SumSpan);
    if (total > r.cap) {  // the slot's previous wave has retired (ring discipline)
        dfree(ex, r.d_tab, r.cap);
        hfree(ex, r.h_tab);
        dalloc(ex, r.d_tab, total);
        halloc(ex, r.h_tab, total);
        r.cap = total;
    }
    memcpy(r.h_tab, segs.data(), seg_b);
    if (!sums.empty()) memcpy(r.h_tab + span_off, sums.data(), sums.size() * sizeof(SumSpan));
    CK(cudaMemcpyAsync(r.d_tab, r.h_tab, total, cudaMemcpyHostToDevice, ex.stream));
    Plan pl;
    wr.seg0 = 0;
    pl.waves.push_back(wr);
    pl.sums = sums;
    launch_plan(ex, pl, reinterpret_cast<Seg *>(r.d_tab), reinterpret_cast<SumSpan *>(r.d_tab + span_off),
                ex.stream);
    CK(cudaMemcpyAsync(r.h_err, ex.err, sizeof(int), cudaMemcpyDeviceToHost, ex.stream));
    CK(cudaEventRecord(r.ev, ex.stream));
    r.wave = s.waves_issued++;
    r.finishing = finishing;
    r.members = members;
}

void server_step(tcorr_server_s &s) {
    while (retire_one(s, false)) {
    }
    admit(s);
    launch_wave(s);
    resolve_timers(s.ex);
}

int pending_jobs(const tcorr_server_s &s) {
    return (int)(s.queue.size() + s.running.size());
}

void destroy_server(tcorr_server_s *s) {
    cudaStreamSynchronize(s->ex.stream);
    for (auto &kv : s->jobs) release(kv.second->ex);
    for (RingSlot &r : s->ring)
        if (r.ev) cudaEventDestroy(r.ev);
    cudaStreamSynchronize(s->ex.stream);
    release(s->ex);
    if (s->h_res) cudaFreeHost(s->h_res);
    if (s->pool) cudaMemPoolDestroy(s->pool);
    delete s;
}

}  // namespace

extern "C" {

tcorr_status tcorr_server_create(tcorr_server_t *out, const tcorr_opts *opts, int64_t hbm_bytes,
                                 void *stream) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return TCORR_EINVAL;
    }
    *out = nullptr;
    tcorr_opts op{};
    if (opts) op = *opts;
    {
        const tcorr_status st = check_opts(op, g_create_error);
        if (st != TCORR_OK) return st;
    }
    if (op.host_inputs != 0 || hbm_bytes < 0) {
        g_create_error = "the server takes device inputs (host_inputs = 0) and hbm_bytes >= 0";
        return TCORR_EINVAL;
    }
    tcorr_server_s *s = new (std::nothrow) tcorr_server_s();
    if (!s) {
        g_create_error = "host allocation failed";
        return TCORR_ENOMEM;
    }
    Exec &ex = s->ex;
    try {
        init_exec(ex, op, stream);
        int dev = 0;
        CK(cudaGetDevice(&dev));
        cudaMemPoolProps pp{};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = dev;
        CK(cudaMemPoolCreate(&s->pool, &pp));
        uint64_t keep = UINT64_MAX;  // keep freed blocks in the pool for the next jobs
        CK(cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep));
        const size_t ueb = u_elem_bytes(ex.prec);
        const size_t wave_bytes = (size_t)(op.wave_mb > 0 ? op.wave_mb : 2048) << 20;
        ex.u_cap = (int64_t)(wave_bytes / ueb);
        s->wave_tasks = op.batch_tasks > 0 ? op.batch_tasks : 4096;
        ex.wave_tasks = s->wave_tasks;
        ex.part_cap = (int64_t)8 << 20;  // 64 MiB of orbit partials per wave
        dalloc(ex, ex.U, (size_t)ex.u_cap * ueb);
        dalloc(ex, ex.partials, (size_t)ex.part_cap * sizeof(double));
        dalloc(ex, ex.d_descs, (size_t)MAX_SLOTS * sizeof(InstDesc));
        alloc_common(ex);
        CK(cudaHostAlloc(&s->h_res, (size_t)MAX_SLOTS * 3 * sizeof(double), cudaHostAllocMapped));
        CK(cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->d_res), s->h_res, 0));
        for (RingSlot &r : s->ring) {
            CK(cudaEventCreateWithFlags(&r.ev, cudaEventDisableTiming));
            halloc(ex, r.h_err, sizeof(int));
            *r.h_err = 0;
        }
        for (int k = MAX_SLOTS - 1; k >= 0; k--) s->free_slots.push_back(k);
        CK(cudaStreamSynchronize(ex.stream));
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        s->budget = hbm_bytes > 0 ? (size_t)hbm_bytes : free_b / 10 * 8;
        if (s->budget > free_b)
            throw Fail{TCORR_ENOMEM, "budget " + std::to_string(s->budget) + " bytes exceeds free device memory " +
                                         std::to_string(free_b)};
    } catch (const Fail &f) {
        g_create_error = f.msg;
        cudaGetLastError();
        destroy_server(s);
        return f.st;
    } catch (const std::bad_alloc &) {
        g_create_error = "host allocation failed";
        destroy_server(s);
        return TCORR_ENOMEM;
    }
    *out = s;
    return TCORR_OK;
}

tcorr_status tcorr_server_submit(tcorr_server_t s, const tcorr_problem *p, int64_t *id) {
    if (!s) return TCORR_EINVAL;
    s->ex.last_error.clear();
    if (!p || !id || p->o < 1 || p->v < 1 || !p->eps_occ || !p->eps_vir || !p->t1 || !p->t2 || !p->vvvo ||
        !p->ooov || !p->ovov) {
        s->ex.last_error = "problem: o, v must be >= 1 and every array non-NULL; id non-NULL";
        return TCORR_EINVAL;
    }
    if (!sizes_supported(p->o, p->v)) {
        s->ex.last_error = "sizes beyond the supported range";
        return TCORR_EUNSUPPORTED;
    }
    const Dims dm = make_dims(p->o, p->v);
    const size_t fp = job_footprint(dm, s->ex.prec);
    const int64_t u_task = 3 * dm.ug;
    const int64_t norb = epilogue_orbits(dm.v);
    if (fp > s->budget || u_task > s->ex.u_cap || norb * 2 > s->ex.part_cap) {
        s->ex.last_error = "job footprint " + std::to_string(fp) + " bytes or one task's scratch exceeds the server's";
        return TCORR_ENOMEM;
    }
    try {
        auto j = std::make_unique<Job>();
        j->id = s->next_id++;
        j->in = *p;
        j->bytes = fp;
        *id = j->id;
        s->queue.push_back(j.get());
        s->jobs[j->id] = std::move(j);
    } catch (const std::bad_alloc &) {
        s->ex.last_error = "host allocation failed";
        return TCORR_ENOMEM;
    }
    return TCORR_OK;
}

tcorr_status tcorr_server_step(tcorr_server_t s, int *pending) {
    if (!s) return TCORR_EINVAL;
    try {
        server_step(*s);
    } catch (const Fail &f) {
        s->ex.last_error = f.msg;
        cudaGetLastError();
        return f.st;
    } catch (const std::bad_alloc &) {
        s->ex.last_error = "host allocation failed";
        return TCORR_ENOMEM;
    }
    if (pending) *pending = pending_jobs(*s);
    return TCORR_OK;
}

tcorr_status tcorr_server_poll(tcorr_server_t s, int64_t id, int *state, double *e_out, int *job_status) {
    if (!s || !state) return TCORR_EINVAL;
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) {
        s->ex.last_error = "unknown job id";
        return TCORR_EINVAL;
    }
    try {
        while (retire_one(*s, false)) {
        }
    } catch (const Fail &f) {
        s->ex.last_error = f.msg;
        return f.st;
    }
    const Job &j = *it->second;
    *state = j.state;
    if (j.state == TCORR_JOB_DONE && e_out)
        for (int c = 0; c < 3; c++) e_out[c] = j.e[c];
    if (job_status) *job_status = j.status;
    return TCORR_OK;
}

tcorr_status tcorr_server_drain(tcorr_server_t s) {
    if (!s) return TCORR_EINVAL;
    try {
        while (pending_jobs(*s) > 0) {
            const int64_t before = s->waves_issued;
            server_step(*s);
            if (s->waves_issued == before && !retire_one(*s, true) && pending_jobs(*s) > 0)
                throw Fail{TCORR_ECUDA, "no progress possible: queued jobs cannot be admitted"};
        }
        while (retire_one(*s, true)) {
        }
        resolve_timers(s->ex);
    } catch (const Fail &f) {
        s->ex.last_error = f.msg;
        cudaGetLastError();
        return f.st;
    }
    return TCORR_OK;
}

tcorr_status tcorr_server_stats(tcorr_server_t s, int64_t *st) {
    if (!s || !st) return TCORR_EINVAL;
    st[0] = s->next_id;
    st[1] = s->n_done;
    st[2] = s->n_failed;
    st[3] = (int64_t)s->running.size();
    st[4] = (int64_t)s->queue.size();
    st[5] = (int64_t)s->used;
    st[6] = (int64_t)s->peak;
    st[7] = s->waves_issued;
    return TCORR_OK;
}

const char *tcorr_server_last_error(tcorr_server_t s) {
    if (!s) return g_create_error.c_str();
    return s->ex.last_error.c_str();
}

tcorr_status tcorr_server_destroy(tcorr_server_t s) {
    if (!s) return TCORR_OK;
    destroy_server(s);
    return TCORR_OK;
}

}  // extern "C"
