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
// register prefetch of the next chunk).  CTAs are ordered a-tile fastest so
// that each pair tile of the large operand comes from HBM once.  Operand rows are K-contiguous, so
// the swapped pair order (c,b) of two segments only changes which rows are
// read, never the coalescing.
#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int TP = 128;  // pairs per CTA tile
constexpr int TA = 32;   // a values per CTA tile
constexpr int KC = 8;    // K chunk
constexpr int NT = 256;  // threads

struct F64Params {
    Dims dm;
    const double *G, *T2K, *T2R, *AoN;
    const int *tasks;
    int64_t task0;
    double *U;
};

__global__ void __launch_bounds__(NT) ugemm_f64_kernel(const F64Params p) {
    __shared__ __align__(16) double As[KC][TP + 4];
    __shared__ __align__(16) double Bs[KC][TA + 4];

    const int o = p.dm.o, v = p.dm.v, dp = p.dm.dp, lp = p.dm.lp, vc = p.dm.vc;
    const int64_t v2 = (int64_t)v * v;
    const int tid = threadIdx.x;
    // a tiles fastest: the CTAs sharing one pair tile (the large A operand)
    // run back to back, so it is read from HBM once and then hits L2
    const int nat = (v + TA - 1) / TA;
    const int64_t p0 = (int64_t)(blockIdx.x / nat) * TP;
    const int a0 = (blockIdx.x % nat) * TA;
    const int tb = blockIdx.z / 3, g = blockIdx.z % 3;
    const int *tk = p.tasks + 3 * (p.task0 + tb);
    const int ti = tk[0], tj = tk[1], tkk = tk[2];
    if (ti == tj && tj == tkk) return;  // i = j = k: zero energy, U never read
    int s, pp, q;
    if (g == 0) { s = ti; pp = tj; q = tkk; }
    else if (g == 1) { s = tj; pp = ti; q = tkk; }
    else { s = tkk; pp = ti; q = tj; }

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
                aptr = p.G + ((int64_t)q * v2 + row_nat) * dp + kk;
                bptr = p.T2R + (((int64_t)s * o + pp) * v + ba) * dp + kk;
                break;
            case 1:
                aptr = p.G + ((int64_t)pp * v2 + row_swp) * dp + kk;
                bptr = p.T2R + (((int64_t)s * o + q) * v + ba) * dp + kk;
                break;
            case 2:
                aptr = p.T2K + ((int64_t)pp * v2 + row_nat) * lp + kk;
                bptr = p.AoN + (((int64_t)q * o + s) * v + ba) * lp + kk;
                break;
            default:
                aptr = p.T2K + ((int64_t)q * v2 + row_swp) * lp + kk;
                bptr = p.AoN + (((int64_t)pp * o + s) * v + ba) * lp + kk;
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

    load_chunk(0);
    for (int chunk = 0; chunk < nchunk; chunk++) {
        store_chunk();
        __syncthreads();
        if (chunk + 1 < nchunk) load_chunk(chunk + 1);
#pragma unroll
        for (int k = 0; k < KC; k++) {
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
        }
        __syncthreads();
    }

    double *Ug = p.U + (int64_t)(tb * 3 + g) * v2 * vc;
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

cudaError_t launch_ugemm_f64(const Operands &op, const GemmArgs &ga, cudaStream_t st) {
    F64Params p;
    p.dm = ga.dm;
    p.G = static_cast<const double *>(op.G);
    p.T2K = static_cast<const double *>(op.T2K);
    p.T2R = static_cast<const double *>(op.T2R);
    p.AoN = static_cast<const double *>(op.AoN);
    p.tasks = ga.tasks;
    p.task0 = ga.task0;
    p.U = static_cast<double *>(ga.U);
    const int64_t v2 = (int64_t)ga.dm.v * ga.dm.v;
    const int64_t tiles = ((v2 + TP - 1) / TP) * ((ga.dm.v + TA - 1) / TA);
    dim3 grid((unsigned)tiles, 1, (unsigned)(3 * ga.ntb));
    if (tiles > 0x7fffffff || grid.z > 65535) return cudaErrorInvalidConfiguration;
    ugemm_f64_kernel<<<grid, NT, 0, st>>>(p);
    return cudaGetLastError();
}

}  // namespace tcorr
