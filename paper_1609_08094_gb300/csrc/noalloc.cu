// Allocation-free entry point: one task's FP64 energy share from the
// caller's canonical device arrays, with every intermediate in a fixed
// file-scope device array instead of memory obtained from cudaMalloc.
//
// Who needs it: callers that must not allocate device memory themselves or
// through a library -- applications whose device memory is owned entirely by
// their own pool or budget, and latency-sensitive loops that cannot afford
// cudaMalloc/cudaFree, which synchronise the device.  The price is a fixed
// TCORR_NOALLOC_SCRATCH_BYTES array that every GPU loading libtcorr holds
// until the process exits, and a size limit (v <= TCORR_NOALLOC_MAX_V).
//
// Work: a variant of the FP64 W-contraction kernel that reads t2, vvvo and
// ooov in their canonical layouts (no re-laid-out copies, so nothing to
// allocate) and writes the three group tensors U of the task into the
// scratch array; the existing fused epilogue and task reduction then run on
// pointers into the same array and write E[4], E[5] to the caller's output.
#include <mutex>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int NA_VMAX = TCORR_NOALLOC_MAX_V;
constexpr int NA_TE = 8;                                   // FP64 epilogue cube edge
constexpr int NA_NB = (NA_VMAX + NA_TE - 1) / NA_TE;
constexpr int NA_NORB = NA_NB * (NA_NB + 1) * (NA_NB + 2) / 6;
constexpr size_t NA_U_BYTES = (size_t)3 * NA_VMAX * NA_VMAX * NA_VMAX * sizeof(double);  // 3 ug <= 3 NA_VMAX^3
constexpr size_t NA_PART_OFF = NA_U_BYTES;
constexpr size_t NA_TASK_OFF = NA_PART_OFF + (size_t)NA_NORB * 2 * sizeof(double);
constexpr size_t NA_ORB_OFF = NA_TASK_OFF + 16;
constexpr size_t NA_SEG_OFF = (NA_ORB_OFF + (size_t)NA_NORB * 3 * sizeof(int) + 63) / 64 * 64;
constexpr size_t NA_DESC_OFF = (NA_SEG_OFF + sizeof(Seg) + alignof(InstDesc) - 1) / alignof(InstDesc) * alignof(InstDesc);
constexpr size_t NA_END = NA_DESC_OFF + sizeof(InstDesc);
static_assert(NA_END <= TCORR_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the declared size");
static_assert(NA_VMAX % UPAD == 0, "maximum v must be a multiple of the U row padding");

// The scratch: U [3][ug] doubles (each group [v][v][vc]), orbit partials [norb][2] doubles,
// the task (3 ints), the block-orbit table [norb][3] ints, and the work
// description the shared epilogue kernels read (one segment, one instance).
static __device__ __align__(256) unsigned char g_noalloc_scratch[TCORR_NOALLOC_SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void *g_ptr[MAX_DEVICES] = {};

// Writes the work description, the task and the block orbits A <= B <= C
// (blocks of NA_TE) into the scratch.
__global__ void noalloc_tables_kernel(const InstDesc d, const Seg sg, InstDesc *d_out, Seg *sg_out, int *task,
                                      int *orb, int nb, int i, int j, int k) {
    static_assert(sizeof(InstDesc) % 4 == 0 && sizeof(Seg) % 4 == 0, "word copy");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&d);
    uint32_t *dst = reinterpret_cast<uint32_t *>(d_out);
    for (int w = threadIdx.x; w < (int)(sizeof(InstDesc) / 4); w += blockDim.x) dst[w] = src[w];
    if (threadIdx.x == 0) *sg_out = sg;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    task[0] = i;
    task[1] = j;
    task[2] = k;
    int n = 0;
    for (int a = 0; a < nb; a++)
        for (int b = a; b < nb; b++)
            for (int c = b; c < nb; c++) {
                orb[3 * n] = a;
                orb[3 * n + 1] = b;
                orb[3 * n + 2] = c;
                n++;
            }
}

// U^{s;p,q}[a][b][c] for the three groups of task (i,j,k), FP64, from the
// canonical arrays (same sums as the layout-based FP64 kernel):
//   sum_d t2[s][p][a][d] (db|cq) + sum_d t2[s][q][a][d] (dc|bp)
//   - sum_l (as|lq) t2[p][l][b][c] - sum_l (as|lp) t2[q][l][c][b],
// with (db|cq) = vvvo[d][b][c][q] and (as|lq) = ooov[l][q][s][a].
constexpr int CT_P = 128, CT_A = 32, CT_K = 8;
__global__ void __launch_bounds__(256) ugemm_f64_canon_kernel(int o, int v, int vc, int64_t ug,
                                                              const double *__restrict__ t2,
                                                              const double *__restrict__ vvvo,
                                                              const double *__restrict__ ooov, int ti, int tj,
                                                              int tk, double *__restrict__ U) {
    __shared__ double As[CT_K][CT_P + 1];
    __shared__ double Bs[CT_K][CT_A + 1];
    if (ti == tj && tj == tk) return;
    const int tid = threadIdx.x;
    const int64_t v2 = (int64_t)v * v;
    const int64_t p0 = (int64_t)blockIdx.x * CT_P;
    const int a0 = blockIdx.y * CT_A;
    const int g = blockIdx.z;
    int s, pp, q;
    if (g == 0) { s = ti; pp = tj; q = tk; }
    else if (g == 1) { s = tj; pp = ti; q = tk; }
    else { s = tk; pp = ti; q = tj; }
    const int tp = tid & 31, ta = tid >> 5;
    double acc[4][4] = {};
    for (int seg = 0; seg < 4; seg++) {
        const int klen = seg < 2 ? v : o;
        for (int k0 = 0; k0 < klen; k0 += CT_K) {
            for (int e = tid; e < CT_P * CT_K; e += 256) {
                const int r = e / CT_K, kk = e % CT_K, kx = k0 + kk;
                const int64_t pidx = p0 + r;
                double x = 0.0;
                if (pidx < v2 && kx < klen) {
                    const int64_t b = pidx / v, c = pidx % v;
                    if (seg == 0) x = vvvo[((kx * (int64_t)v + b) * v + c) * o + q];
                    else if (seg == 1) x = vvvo[((kx * (int64_t)v + c) * v + b) * o + pp];
                    else if (seg == 2) x = t2[(((int64_t)pp * o + kx) * v + b) * v + c];
                    else x = t2[(((int64_t)q * o + kx) * v + c) * v + b];
                }
                As[kk][r] = x;
            }
            {
                const int r = tid / CT_K, kk = tid % CT_K, kx = k0 + kk, a = a0 + r;
                double x = 0.0;
                if (a < v && kx < klen) {
                    if (seg == 0) x = t2[(((int64_t)s * o + pp) * v + a) * v + kx];
                    else if (seg == 1) x = t2[(((int64_t)s * o + q) * v + a) * v + kx];
                    else if (seg == 2) x = -ooov[(((int64_t)kx * o + q) * o + s) * v + a];
                    else x = -ooov[(((int64_t)kx * o + pp) * o + s) * v + a];
                }
                Bs[kk][r] = x;
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < CT_K; kk++) {
                double av[4], bv[4];
#pragma unroll
                for (int r = 0; r < 4; r++) av[r] = As[kk][tp + 32 * r];
#pragma unroll
                for (int c = 0; c < 4; c++) bv[c] = Bs[kk][ta * 4 + c];
#pragma unroll
                for (int r = 0; r < 4; r++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
            }
            __syncthreads();
        }
    }
    double *Ug = U + (int64_t)g * ug;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int a = a0 + ta * 4 + c;
        if (a >= v) continue;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int64_t pidx = p0 + tp + 32 * r;
            if (pidx >= v2) continue;
            Ug[((int64_t)a * v + pidx / v) * vc + pidx % v] = acc[r][c];
        }
    }
}

}  // namespace
}  // namespace tcorr

using namespace tcorr;

extern "C" tcorr_status tcorr_task_energy_noalloc(int o, int v, const double *eps_occ, const double *eps_vir,
                                                  const double *t1, const double *t2, const double *vvvo,
                                                  const double *ooov, const double *ovov, int i, int j, int k,
                                                  double *e_out, void *stream) {
    if (o < 1 || v < 1 || !eps_occ || !eps_vir || !t1 || !t2 || !vvvo || !ooov || !ovov || !e_out)
        return TCORR_EINVAL;
    if (v > TCORR_NOALLOC_MAX_V || o > 4096) return TCORR_EINVAL;  // beyond the fixed scratch
    if (i < 0 || i > j || j > k || k >= o) return TCORR_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return TCORR_ECUDA;
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_ptr[dev]) {  // once per device, with that device current
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return TCORR_ECUDA;
            }
            g_ptr[dev] = ptr;
        }
        base = g_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char *sc = static_cast<unsigned char *>(base);
    double *U = reinterpret_cast<double *>(sc);
    double *partials = reinterpret_cast<double *>(sc + NA_PART_OFF);
    int *task = reinterpret_cast<int *>(sc + NA_TASK_OFF);
    int *orbits = reinterpret_cast<int *>(sc + NA_ORB_OFF);
    Seg *seg = reinterpret_cast<Seg *>(sc + NA_SEG_OFF);
    InstDesc *desc = reinterpret_cast<InstDesc *>(sc + NA_DESC_OFF);
    const int nb = (v + NA_TE - 1) / NA_TE;
    InstDesc d{};
    d.dm = make_dims(o, v);
    d.norb = nb * (nb + 1) * (nb + 2) / 6;
    d.eps_o = eps_occ;
    d.eps_v = eps_vir;
    d.t1 = t1;
    d.ovov = ovov;
    d.tasks = task;
    d.orbits = orbits;
    d.task_e = e_out;
    Seg sg{};
    sg.inst = 0;
    sg.ntb = 1;
    noalloc_tables_kernel<<<1, 128, 0, st>>>(d, sg, desc, seg, task, orbits, nb, i, j, k);
    const int64_t v2 = (int64_t)v * v;
    dim3 grid((unsigned)((v2 + CT_P - 1) / CT_P), (unsigned)((v + CT_A - 1) / CT_A), 3);
    ugemm_f64_canon_kernel<<<grid, 256, 0, st>>>(o, v, d.dm.vc, d.dm.ug, t2, vvvo, ooov, i, j, k, U);
    Wave w{};
    w.descs = desc;
    w.segs = seg;
    w.nseg = 1;
    w.n_gemm = 0;
    w.n_epi = d.norb;
    w.n_red = 1;
    w.U = U;
    w.partials = partials;
    if (launch_epilogue(TCORR_FP64, 0, w, st) != cudaSuccess) return TCORR_ECUDA;
    if (launch_task_reduce(w, st) != cudaSuccess) return TCORR_ECUDA;
    return cudaGetLastError() == cudaSuccess ? TCORR_OK : TCORR_ECUDA;
}
