// C ABI of libtcorr (declared in include/tcorr.h): handle life cycle, input
// validation, footprint check, layout preparation (S0), the task schedule
// (S1: the collapsed i <= j <= k loop of Sec. 3, cut into batches), and the
// launch sequence W contractions (S2/S3) -> fused epilogue (S4) -> Kahan
// reductions (S5) for every batch.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "tcorr_internal.cuh"

using namespace tcorr;

struct tcorr_s {
    Handle h;
};

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

template <typename T>
void dalloc(Handle &h, T *&ptr, size_t bytes) {
    void *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw Fail{TCORR_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                     cudaGetErrorString(e)};
    }
    h.bytes += bytes;
    ptr = static_cast<T *>(p);
}

void release(Handle &h) {
    void *ptrs[] = {h.op.G, h.op.T2K, h.op.T2R, h.op.AoN, h.op.Glo, h.op.T2Klo, h.op.T2Rlo,
                    h.op.AoNlo, h.eps_o, h.eps_v, h.t1, h.ovov, h.dev_f, h.tasks, h.task_e,
                    h.U, h.orbits, h.partials, h.sums, h.err};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h.h_sums) cudaFreeHost(h.h_sums);
    if (h.h_err) cudaFreeHost(h.h_err);
    for (auto &pe : h.pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    free(h.tmaps);
    h = Handle();
}

// Copy (or reference) one caller array on the device.  For host inputs the
// data is staged into a temporary device buffer that the caller frees.
const double *device_view(Handle &h, const double *src, size_t n, bool host, double *&tmp) {
    tmp = nullptr;
    if (!host) return src;
    dalloc(h, tmp, n * sizeof(double));
    CK(cudaMemcpyAsync(tmp, src, n * sizeof(double), cudaMemcpyHostToDevice, h.stream));
    return tmp;
}

void free_tmp(Handle &h, double *&tmp, size_t n) {
    if (!tmp) return;
    CK(cudaStreamSynchronize(h.stream));
    cudaFree(tmp);
    h.bytes -= (n ? n * sizeof(double) : 16);
    tmp = nullptr;
}

struct Timer {
    Handle &h;
    int cls;
    cudaEvent_t a = nullptr;
    Timer(Handle &hh, int c) : h(hh), cls(c) {
        if (!h.profile) return;
        CK(cudaEventCreate(&a));
        CK(cudaEventRecord(a, h.stream));
    }
    void stop() {
        if (!h.profile || !a) return;
        cudaEvent_t b = nullptr;
        CK(cudaEventCreate(&b));
        CK(cudaEventRecord(b, h.stream));
        h.pending.push_back({cls, a, b});
        a = nullptr;
    }
    ~Timer() {
        if (a) cudaEventDestroy(a);
    }
};

// Accumulate the recorded event pairs; call after a stream synchronisation.
void resolve_timers(Handle &h) {
    for (auto &pe : h.pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pe.a, pe.b) == cudaSuccess) {
            h.k_ms[pe.cls] += ms;
            h.k_launch[pe.cls] += 1;
        }
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    h.pending.clear();
}

int elem_kind(int prec) { return prec == TCORR_FP64 ? 0 : (prec == TCORR_TF32X3 ? 1 : 2); }
size_t elem_bytes(int prec) { return prec == TCORR_FP64 ? 8 : (prec == TCORR_TF32X3 ? 4 : 2); }

void build_operands(Handle &h, const double *t2, const double *vvvo, const double *ooov,
                    bool host) {
    const int o = h.dm.o, v = h.dm.v, dp = h.dm.dp, lp = h.dm.lp;
    const int64_t v2 = (int64_t)v * v;
    const int kind = elem_kind(h.prec);
    const size_t eb = elem_bytes(h.prec);
    const bool split = h.prec != TCORR_FP64;
    const size_t nG = (size_t)o * v2 * dp, nT2K = (size_t)o * v2 * lp;
    const size_t nT2R = (size_t)o * o * v * dp, nAoN = (size_t)o * o * v * lp;
    dalloc(h, h.op.G, nG * eb);
    dalloc(h, h.op.T2K, nT2K * eb);
    dalloc(h, h.op.T2R, nT2R * eb);
    dalloc(h, h.op.AoN, nAoN * eb);
    if (split) {
        dalloc(h, h.op.Glo, nG * eb);
        dalloc(h, h.op.T2Klo, nT2K * eb);
        dalloc(h, h.op.T2Rlo, nT2R * eb);
        dalloc(h, h.op.AoNlo, nAoN * eb);
    }
    Timer tm(h, KC_PREP);
    // G[q][xy][d] = vvvo[d][xy][q]; staged in chunks of d rows for host inputs
    CK(cudaMemsetAsync(h.op.G, 0, nG * eb, h.stream));
    if (split) CK(cudaMemsetAsync(h.op.Glo, 0, nG * eb, h.stream));
    const size_t row = (size_t)v2 * o;  // doubles per d row of vvvo
    if (!host) {
        CK(launch_transpose_pad(kind, vvvo, h.op.G, h.op.Glo, v2, v, v, o, o, (int64_t)row, 1, dp,
                                (int64_t)v2 * dp, 1.0, h.stream));
    } else {
        size_t rows_per = (size_t)((512ull << 20) / (row * sizeof(double)));
        if (rows_per < 1) rows_per = 1;
        if (rows_per > (size_t)v) rows_per = v;
        double *stage = nullptr;
        dalloc(h, stage, rows_per * row * sizeof(double));
        for (int d0 = 0; d0 < v; d0 += (int)rows_per) {
            const int nr = (int)((size_t)(v - d0) < rows_per ? (size_t)(v - d0) : rows_per);
            CK(cudaMemcpyAsync(stage, vvvo + (size_t)d0 * row, nr * row * sizeof(double),
                               cudaMemcpyHostToDevice, h.stream));
            char *ghi = static_cast<char *>(h.op.G) + (size_t)d0 * eb;
            char *glo = split ? static_cast<char *>(h.op.Glo) + (size_t)d0 * eb : nullptr;
            CK(launch_transpose_pad(kind, stage, ghi, glo, v2, nr, nr, o, o, (int64_t)row, 1, dp,
                                    (int64_t)v2 * dp, 1.0, h.stream));
        }
        free_tmp(h, stage, rows_per * row);
    }
    double *tmp_t2 = nullptr, *tmp_oo = nullptr;
    const double *dt2 = device_view(h, t2, (size_t)o * o * v2, host, tmp_t2);
    // T2K[q][xy][l] = t2[q][l][xy]
    CK(launch_transpose_pad(kind, dt2, h.op.T2K, h.op.T2Klo, o, o, lp, v2, (int64_t)o * v2, v2, 1,
                            (int64_t)v2 * lp, lp, 1.0, h.stream));
    // T2R[spa][d] = t2[spa][d]  (row copy with padding: C = 1)
    CK(launch_transpose_pad(kind, dt2, h.op.T2R, h.op.T2Rlo, (int64_t)o * o * v, v, dp, 1, v, 1, 0,
                            dp, 0, 1.0, h.stream));
    const double *doo = device_view(h, ooov, (size_t)o * o * o * v, host, tmp_oo);
    // AoN[qsa][l] = -ooov[l][qsa]
    CK(launch_transpose_pad(kind, doo, h.op.AoN, h.op.AoNlo, 1, o, lp, (int64_t)o * o * v, 0,
                            (int64_t)o * o * v, 1, 0, lp, -1.0, h.stream));
    tm.stop();
    free_tmp(h, tmp_t2, (size_t)o * o * v2);
    free_tmp(h, tmp_oo, (size_t)o * o * o * v);
}

void build_epilogue_inputs(Handle &h, const double *eps_occ, const double *eps_vir,
                           const double *t1, const double *ovov, bool host) {
    const int o = h.dm.o, v = h.dm.v;
    const size_t nov2 = (size_t)o * v * o * v;
    dalloc(h, h.eps_o, o * sizeof(double));
    dalloc(h, h.eps_v, v * sizeof(double));
    const cudaMemcpyKind kd = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    CK(cudaMemcpyAsync(h.eps_o, eps_occ, o * sizeof(double), kd, h.stream));
    CK(cudaMemcpyAsync(h.eps_v, eps_vir, v * sizeof(double), kd, h.stream));
    if (h.prec == TCORR_FP64) {
        dalloc(h, h.t1, (size_t)o * v * sizeof(double));
        dalloc(h, h.ovov, nov2 * sizeof(double));
        CK(cudaMemcpyAsync(h.t1, t1, (size_t)o * v * sizeof(double), kd, h.stream));
        CK(cudaMemcpyAsync(h.ovov, ovov, nov2 * sizeof(double), kd, h.stream));
    } else {
        dalloc(h, h.t1, (size_t)o * v * sizeof(float));
        dalloc(h, h.ovov, nov2 * sizeof(float));
        double *tmp1 = nullptr, *tmp2 = nullptr;
        const double *d1 = device_view(h, t1, (size_t)o * v, host, tmp1);
        CK(launch_to_float(d1, static_cast<float *>(h.t1), (int64_t)o * v, h.stream));
        const double *d2 = device_view(h, ovov, nov2, host, tmp2);
        CK(launch_to_float(d2, static_cast<float *>(h.ovov), (int64_t)nov2, h.stream));
        free_tmp(h, tmp1, (size_t)o * v);
        free_tmp(h, tmp2, nov2);
        dalloc(h, h.dev_f, v * sizeof(float));
        CK(launch_block_deltas(h.eps_v, h.dev_f, v, h.epi_te, h.stream));
    }
}

void build_schedule(Handle &h) {
    const int o = h.dm.o;
    std::vector<int> tl;
    for (int i = 0; i < o; i++)
        for (int j = i; j < o; j++)
            for (int k = j; k < o; k++) {
                tl.push_back(i);
                tl.push_back(j);
                tl.push_back(k);
            }
    h.ntask = (int64_t)tl.size() / 3;
    dalloc(h, h.tasks, tl.size() * sizeof(int));
    CK(cudaMemcpy(h.tasks, tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice));
    dalloc(h, h.task_e, (size_t)h.ntask * 2 * sizeof(double));
    CK(cudaMemsetAsync(h.task_e, 0, (size_t)h.ntask * 2 * sizeof(double), h.stream));
    const int nb = (h.dm.v + h.epi_te - 1) / h.epi_te;
    std::vector<int> ob;
    for (int a = 0; a < nb; a++)
        for (int b = a; b < nb; b++)
            for (int c = b; c < nb; c++) {
                ob.push_back(a);
                ob.push_back(b);
                ob.push_back(c);
            }
    h.norb = (int)(ob.size() / 3);
    dalloc(h, h.orbits, ob.size() * sizeof(int));
    CK(cudaMemcpy(h.orbits, ob.data(), ob.size() * sizeof(int), cudaMemcpyHostToDevice));
}

size_t footprint(const Dims &d, int prec, int batch, int te, bool host) {
    const size_t o = d.o, v = d.v, v2 = v * v;
    const size_t eb = elem_bytes(prec), parts = prec == TCORR_FP64 ? 1 : 2;
    size_t b = parts * eb * (o * v2 * d.dp + o * v2 * d.lp + o * o * v * d.dp + o * o * v * d.lp);
    const size_t ub = prec == TCORR_FP64 ? 8 : 4;
    b += (o * o * v2 + o * v) * ub + (o + v) * 8 + v * 4;
    b += (size_t)batch * 3 * v2 * d.vc * ub;
    const size_t nb = (v + te - 1) / te;
    const size_t norb = nb * (nb + 1) * (nb + 2) / 6;
    b += (size_t)batch * norb * 16 + norb * 12;
    const size_t nt = o * (o + 1) * (o + 2) / 6;
    b += nt * 28;
    if (host) b += std::max<size_t>(o * o * v2 * 8, (size_t)512 << 20);
    return b + (64u << 20);
}

void check_err_flag(Handle &h) {
    CK(cudaMemcpyAsync(h.h_err, h.err, sizeof(int), cudaMemcpyDeviceToHost, h.stream));
    CK(cudaStreamSynchronize(h.stream));
    if (*h.h_err) {
        const int e = *h.h_err;
        *h.h_err = 0;
        CK(cudaMemsetAsync(h.err, 0, sizeof(int), h.stream));
        if (e & (DERR_TIMEOUT_FULL | DERR_TIMEOUT_EMPTY | DERR_TIMEOUT_TMEM))
            throw Fail{TCORR_ETIMEOUT, "device pipeline wait expired (flags " + std::to_string(e) + ")"};
        throw Fail{TCORR_ECUDA, "device reported bad configuration (flags " + std::to_string(e) + ")"};
    }
}

void run_range(Handle &h, int64_t first, int64_t count, double *e_out, double *e_task) {
    for (int64_t b0 = first; b0 < first + count; b0 += h.batch) {
        const int ntb = (int)std::min<int64_t>(h.batch, first + count - b0);
        GemmArgs ga{h.dm, h.tasks, b0, ntb, h.U};
        {
            Timer tm(h, KC_GEMM);
            if (h.prec == TCORR_FP64) CK(launch_ugemm_f64(h.op, ga, h.stream));
            else CK(launch_ugemm_tc(&h, ga, h.stream));
            tm.stop();
        }
        EpiArgs ea{h.dm, h.tasks, b0, ntb, h.U, h.eps_o, h.eps_v, h.t1, h.ovov, h.dev_f,
                   h.orbits, h.norb, h.epi_te, h.partials, h.task_e};
        {
            Timer tm(h, KC_EPI);
            CK(launch_epilogue(h.prec, ea, h.stream));
            tm.stop();
        }
        {
            Timer tm(h, KC_RED);
            CK(launch_task_reduce(ea, h.stream));
            tm.stop();
        }
    }
    {
        Timer tm(h, KC_RED);
        CK(launch_range_sum(h.task_e, first, count, h.sums, h.stream));
        tm.stop();
    }
    CK(cudaMemcpyAsync(h.h_sums, h.sums, 3 * sizeof(double), cudaMemcpyDeviceToHost, h.stream));
    if (e_task)
        CK(cudaMemcpyAsync(e_task, h.task_e + 2 * first, (size_t)count * 2 * sizeof(double),
                           cudaMemcpyDeviceToHost, h.stream));
    CK(cudaStreamSynchronize(h.stream));
    resolve_timers(h);
    check_err_flag(h);
    e_out[0] = h.h_sums[0];
    e_out[1] = h.h_sums[1];
    e_out[2] = h.h_sums[2];
}

}  // namespace

extern "C" {

int tcorr_version(void) { return 1; }

const char *tcorr_status_string(tcorr_status s) {
    if ((int)s < 0 || (int)s > 5) return "TCORR_UNKNOWN";
    return kStatusNames[(int)s];
}

const char *tcorr_last_error(tcorr_t h) {
    if (!h) return g_create_error.c_str();
    return h->h.last_error.c_str();
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
    if (op.test_stall != 0 && op.test_stall != 1) {
        g_create_error = "test_stall must be 0 or 1";
        return TCORR_EINVAL;
    }
    for (int r : op.reserved)
        if (r != 0) {
            g_create_error = "reserved option fields must be zero";
            return TCORR_EINVAL;
        }
    if (op.prec < TCORR_FP64 || op.prec > TCORR_BF16X3 || op.batch_tasks < 0 ||
        (op.host_inputs != 0 && op.host_inputs != 1)) {
        g_create_error = "invalid option (precision, batch_tasks or host_inputs)";
        return TCORR_EINVAL;
    }
    const int64_t v64 = v, o64 = o;
    if (v64 * v64 * v64 * o64 > ((int64_t)1 << 40) || o > 4096 || v > 8192) {
        g_create_error = "sizes beyond the supported range";
        return TCORR_EUNSUPPORTED;
    }
    tcorr_s *hs = new (std::nothrow) tcorr_s();
    if (!hs) {
        g_create_error = "host allocation failed";
        return TCORR_ENOMEM;
    }
    Handle &h = hs->h;
    try {
        h.stream = static_cast<cudaStream_t>(stream);
        h.prec = op.prec;
        h.profile = op.profile;
        h.inject_stall = op.test_stall;
        int dev = 0;
        CK(cudaGetDevice(&dev));
        CK(cudaDeviceGetAttribute(&h.sm_count, cudaDevAttrMultiProcessorCount, dev));
        CK(cudaDeviceGetAttribute(&h.cc_major, cudaDevAttrComputeCapabilityMajor, dev));
        CK(cudaDeviceGetAttribute(&h.cc_minor, cudaDevAttrComputeCapabilityMinor, dev));
        if (h.prec != TCORR_FP64 && !tc_supported(h.cc_major, h.cc_minor))
            throw Fail{TCORR_EUNSUPPORTED, "mixed precision needs the sm_103 tensor-core path (device is sm_" +
                                               std::to_string(h.cc_major * 10 + h.cc_minor) + ")"};
        h.dm.o = o;
        h.dm.v = v;
        h.dm.dp = round_up(v, KPAD);
        h.dm.lp = round_up(o, KPAD);
        h.dm.vc = round_up(v, UPAD);
        h.epi_te = 8;
        const int64_t ntask = o64 * (o64 + 1) * (o64 + 2) / 6;
        h.u_task_bytes = (size_t)3 * v * v * h.dm.vc * (h.prec == TCORR_FP64 ? 8 : 4);
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        if (op.batch_tasks > 0) {
            h.batch = op.batch_tasks;
        } else {
            size_t budget = std::min<size_t>((size_t)4 << 30, free_b / 8);
            int64_t b = (int64_t)(budget / h.u_task_bytes);
            h.batch = (int)std::max<int64_t>(1, std::min<int64_t>(b, std::min<int64_t>(ntask, 4096)));
        }
        if (h.batch > ntask) h.batch = (int)ntask;
        const size_t need = footprint(h.dm, h.prec, h.batch, h.epi_te, op.host_inputs);
        if (need > free_b)
            throw Fail{TCORR_ENOMEM, "footprint " + std::to_string(need) + " bytes exceeds free device memory " +
                                         std::to_string(free_b)};
        const bool host = op.host_inputs == 1;
        build_operands(h, t2, vvvo, ooov, host);
        build_epilogue_inputs(h, eps_occ, eps_vir, t1, ovov, host);
        build_schedule(h);
        dalloc(h, h.U, h.u_task_bytes * h.batch);
        dalloc(h, h.partials, (size_t)h.batch * h.norb * 2 * sizeof(double));
        dalloc(h, h.sums, 3 * sizeof(double));
        dalloc(h, h.err, sizeof(int));
        CK(cudaMemsetAsync(h.err, 0, sizeof(int), h.stream));
        CK(cudaMallocHost(&h.h_sums, 3 * sizeof(double)));
        CK(cudaMallocHost(&h.h_err, sizeof(int)));
        *h.h_err = 0;
        if (h.prec != TCORR_FP64) {
            std::string msg;
            if (tc_build_tensor_maps(&h, msg) != cudaSuccess) throw Fail{TCORR_EUNSUPPORTED, msg};
        }
        CK(cudaStreamSynchronize(h.stream));
        CK(cudaGetLastError());
        resolve_timers(h);
    } catch (const Fail &f) {
        g_create_error = f.msg;
        cudaStreamSynchronize(h.stream);
        cudaGetLastError();
        release(h);
        delete hs;
        return f.st;
    } catch (const std::bad_alloc &) {
        g_create_error = "host allocation failed";
        release(h);
        delete hs;
        return TCORR_ENOMEM;
    }
    *out = hs;
    return TCORR_OK;
}

int64_t tcorr_num_tasks(tcorr_t h) { return h ? h->h.ntask : -1; }

tcorr_status tcorr_task(tcorr_t h, int64_t idx, int *ijk) {
    if (!h || !ijk) return TCORR_EINVAL;
    if (idx < 0 || idx >= h->h.ntask) {
        h->h.last_error = "task index out of range";
        return TCORR_EINVAL;
    }
    // inverse of the lexicographic enumeration of i <= j <= k
    const int o = h->h.dm.o;
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
    Handle &h = hh->h;
    h.last_error.clear();
    if (!e_out || first < 0 || count < 0 || first + count > h.ntask) {
        h.last_error = "e_out is NULL or the range leaves the task list";
        return TCORR_EINVAL;
    }
    try {
        if (count == 0) {
            e_out[0] = e_out[1] = e_out[2] = 0.0;
            return TCORR_OK;
        }
        run_range(h, first, count, e_out, e_task);
    } catch (const Fail &f) {
        h.last_error = f.msg;
        cudaStreamSynchronize(h.stream);
        cudaGetLastError();
        return f.st;
    }
    return TCORR_OK;
}

tcorr_status tcorr_energy(tcorr_t h, double *e_out) {
    if (!h) return TCORR_EINVAL;
    return tcorr_energy_range(h, 0, h->h.ntask, e_out, nullptr);
}

tcorr_status tcorr_kernel_times(tcorr_t hh, double *ms, int64_t *launches, int reset) {
    if (!hh) return TCORR_EINVAL;
    Handle &h = hh->h;
    for (int c = 0; c < KC_COUNT; c++) {
        if (ms) ms[c] = h.k_ms[c];
        if (launches) launches[c] = h.k_launch[c];
        if (reset) { h.k_ms[c] = 0; h.k_launch[c] = 0; }
    }
    return TCORR_OK;
}

int64_t tcorr_device_bytes(tcorr_t h) { return h ? (int64_t)h->h.bytes : -1; }

tcorr_status tcorr_destroy(tcorr_t h) {
    if (!h) return TCORR_OK;
    cudaStreamSynchronize(h->h.stream);
    release(h->h);
    delete h;
    return TCORR_OK;
}

}  // extern "C"
