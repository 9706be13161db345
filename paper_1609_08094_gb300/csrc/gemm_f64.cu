// FP64 W contractions (S2, FP64 precision): for every task (i,j,k) of a batch
// and each of its three groups (s;p,q), the GEMM
//   U^{s;p,q}[a][(b,c)] = sum over K = [d | d | l | l] of A[(b,c)][K] * B[a][K]
// with the four K segments of Eq. (analytical_triples_ampl) after grouping the
// six permutations of Eq. (symm_operator) by their "single" virtual index
// (layouts and the identity are documented in tcorr_internal.cuh).
//
// GB300's FP64 rate is far below its tensor rates, so this kernel is bound by
// the FP64 pipe: a register-tiled DFMA GEMM (CTA tile 128 pairs x 32 a, 16
// outputs per thread, K staged through shared memory in chunks of 8 with a
// register prefetch of the next chunk).  One flattened grid covers the work
// units of every segment of a wave (one or many problems).  Operand rows are K-contiguous, so
// the swapped pair order (c,b) of two segments only changes which rows are
// read, never the coalescing.
#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int TP = 128;  // pairs per CTA tile
constexpr int TA = 32;   // a values per CTA tile
constexpr int KC = 8;    // K chunk
constexpr int NT = 256;  // threads

__global__ void __launch_bounds__(NT) ugemm_f64_kernel(const Wave w) {
    __shared__ __align__(16) double As[KC][TP + 4];
    __shared__ __align__(16) double Bs[KC][TA + 4];

    // work unit -> segment -> (task, group, pair tile, a tile); a tiles fastest,
    // so the CTAs sharing one pair tile (the large A operand) run back to back
    // and it is read from HBM once, then from L2
    const int64_t unit = blockIdx.x;
    const Seg sg = w.segs[seg_find(w.segs, w.nseg, unit, [](const Seg &x) { return x.gemm0; })];
    const InstDesc &d = w.descs[sg.inst];
    const int o = d.dm.o, v = d.dm.v, dp = d.dm.dp, lp = d.dm.lp, vc = d.dm.vc;
    const int64_t v2 = (int64_t)v * v;
    const int nat = (v + TA - 1) / TA;
    const int64_t per_g = ((v2 + TP - 1) / TP) * nat;
    int64_t local = unit - sg.gemm0;
    const int tb = (int)(local / (3 * per_g));
    local -= (int64_t)tb * 3 * per_g;
    const int g = (int)(local / per_g);
    const int64_t tile = local % per_g;
    const int64_t p0 = (tile / nat) * TP;
    const int a0 = (int)(tile % nat) * TA;
    const int tid = threadIdx.x;
    const int *tk = d.tasks + 3 * (sg.task0 + tb);
    const int ti = tk[0], tj = tk[1], tkk = tk[2];
    if (ti == tj && tj == tkk) return;  // i = j = k: zero energy, U never read
    int s, pp, q;
    if (g == 0) { s = ti; pp = tj; q = tkk; }
    else if (g == 1) { s = tj; pp = ti; q = tkk; }
    else { s = tkk; pp = ti; q = tj; }
    const double *Gm = static_cast<const double *>(d.G);
    const double *T2K = static_cast<const double *>(d.T2K);
    const double *T2R = static_cast<const double *>(d.T2R);
    const double *AoN = static_cast<const double *>(d.AoN);

    // A-row loader: row = tid>>1, half = tid&1 (4 doubles each)
    const int arow = tid >> 1, ahalf = tid & 1;
    const int64_t apair = p0 + arow;
    const bool a_ok = apair < v2;
    const int64_t ab = a_ok ? apair / v : 0, ac = a_ok ? apair % v : 0;
    const int64_t row_nat = ab * v + ac, row_swp = ac * v + ab;
    // B-row loader: tid < 128: row = tid>>2, quarter = tid&3 (2 doubles each)
    const int brow = (tid & 127) >> 2, bq = tid & 3;
    const int ba = a0 + brow;
    const bool b_ok = (tid < 128) && (ba < v);

    const int KV = round_up(v, KC), KO = round_up(o, KC);
    const int nchunk_v = KV / KC, nchunk_o = KO / KC;
    const int nchunk = 2 * nchunk_v + 2 * nchunk_o;

    auto src_ptrs = [&](int chunk, const double *&aptr, const double *&bptr) {
        int seg, kk;
        if (chunk < nchunk_v) { seg = 0; kk = chunk * KC; }
        else if (chunk < 2 * nchunk_v) { seg = 1; kk = (chunk - nchunk_v) * KC; }
        else if (chunk < 2 * nchunk_v + nchunk_o) { seg = 2; kk = (chunk - 2 * nchunk_v) * KC; }
        else { seg = 3; kk = (chunk - 2 * nchunk_v - nchunk_o) * KC; }
        switch (seg) {
            case 0:
                aptr = Gm + ((int64_t)q * v2 + row_nat) * dp + kk;
                bptr = T2R + (((int64_t)s * o + pp) * v + ba) * dp + kk;
                break;
            case 1:
                aptr = Gm + ((int64_t)pp * v2 + row_swp) * dp + kk;
                bptr = T2R + (((int64_t)s * o + q) * v + ba) * dp + kk;
                break;
            case 2:
                aptr = T2K + ((int64_t)pp * v2 + row_nat) * lp + kk;
                bptr = AoN + (((int64_t)q * o + s) * v + ba) * lp + kk;
                break;
            default:
                aptr = T2K + ((int64_t)q * v2 + row_swp) * lp + kk;
                bptr = AoN + (((int64_t)pp * o + s) * v + ba) * lp + kk;
                break;
        }
    };

    double2 ra0 = make_double2(0, 0), ra1 = make_double2(0, 0), rb = make_double2(0, 0);
    auto load_chunk = [&](int chunk) {
        const double *aptr, *bptr;
        src_ptrs(chunk, aptr, bptr);
        if (a_ok) {
            const double2 *pa = reinterpret_cast<const double2 *>(aptr + ahalf * 4);
            ra0 = __ldg(pa);
            ra1 = __ldg(pa + 1);
        } else {
            ra0 = make_double2(0, 0);
            ra1 = make_double2(0, 0);
        }
        if (b_ok) rb = __ldg(reinterpret_cast<const double2 *>(bptr + bq * 2));
        else rb = make_double2(0, 0);
    };
    auto store_chunk = [&]() {
        const int k = ahalf * 4;
        As[k + 0][arow] = ra0.x;
        As[k + 1][arow] = ra0.y;
        As[k + 2][arow] = ra1.x;
        As[k + 3][arow] = ra1.y;
        if (tid < 128) {
            Bs[bq * 2 + 0][brow] = rb.x;
            Bs[bq * 2 + 1][brow] = rb.y;
        }
    };

    const int tp = tid & 31, ta = tid >> 5;
    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int c = 0; c < 4; c++) acc[r][c] = 0.0;

    // Padding costs FP64-pipe time only where a warp issues it: a warp whose
    // four a values all lie at or past v (the ragged last a tile) issues no
    // FMA, and the last chunk of each K segment stops at the segment's end
    // (the zero padding of d to a multiple of KC and of l is never multiplied).
    const bool active = a0 + ta * 4 < v;
    auto mma_step = [&](int k) {
        double av[4], bv[4];
#pragma unroll
        for (int r = 0; r < 4; r++) av[r] = As[k][tp + 32 * r];
        const double2 b01 = *reinterpret_cast<const double2 *>(&Bs[k][ta * 4]);
        const double2 b23 = *reinterpret_cast<const double2 *>(&Bs[k][ta * 4 + 2]);
        bv[0] = b01.x; bv[1] = b01.y; bv[2] = b23.x; bv[3] = b23.y;
#pragma unroll
        for (int r = 0; r < 4; r++)
#pragma unroll
            for (int c = 0; c < 4; c++) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    };
    const int tail_v = v - (nchunk_v - 1) * KC, tail_o = o - (nchunk_o - 1) * KC;

    load_chunk(0);
    for (int chunk = 0; chunk < nchunk; chunk++) {
        store_chunk();
        __syncthreads();
        if (chunk + 1 < nchunk) load_chunk(chunk + 1);
        // valid k of this chunk: KC except at the end of a segment
        int kn = KC;
        if (chunk == nchunk_v - 1 || chunk == 2 * nchunk_v - 1) kn = tail_v;
        else if (chunk == 2 * nchunk_v + nchunk_o - 1 || chunk == nchunk - 1) kn = tail_o;
        if (active) {
            if (kn == KC) {
#pragma unroll
                for (int k = 0; k < KC; k++) mma_step(k);
            } else {
#pragma unroll
                for (int k = 0; k < KC; k++)
                    if (k < kn) mma_step(k);
            }
        }
        __syncthreads();
    }

    double *Ug = static_cast<double *>(w.U) + sg.u_off + (int64_t)(tb * 3 + g) * d.dm.ug;
#pragma unroll
    for (int c = 0; c < 4; c++) {
        const int a = a0 + ta * 4 + c;
        if (a >= v) continue;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int64_t pidx = p0 + tp + 32 * r;
            if (pidx >= v2) continue;
            const int64_t b = pidx / v, cc = pidx % v;
            Ug[((int64_t)a * v + b) * vc + cc] = acc[r][c];
        }
    }
}

}  // namespace

int64_t f64_units_per_task(const Dims &dm) {
    const int64_t v2 = (int64_t)dm.v * dm.v;
    return 3 * ((v2 + TP - 1) / TP) * ((dm.v + TA - 1) / TA);
}

cudaError_t launch_ugemm_f64(const Wave &w, cudaStream_t st) {
    if (w.n_gemm <= 0) return cudaSuccess;
    if (w.n_gemm > 0x7fffffff) return cudaErrorInvalidConfiguration;
    ugemm_f64_kernel<<<(unsigned)w.n_gemm, NT, 0, st>>>(w);
    return cudaGetLastError();
}

}  // namespace tcorr
