// FP64-accurate W contractions on the BF16 tensor cores (Ozaki scheme,
// Ozaki et al. 2012; Mukunoki et al. 2020 on tensor cores): the same grouped
// GEMMs as the FP64 path (see tcorr_internal.cuh), with every operand split
// into OZ_S signed integer slices of OZ_BETA bits.
//
//   x = 2^E x',  |x'| <= 1,  x' = sum_{i=1..S} a_i 2^{-beta i} + r,  |r| <= 2^{-beta S - 1}
//
// with one power-of-two scale per operand side (E_A for G and T2K, E_B for
// T2R and AoN), so the four K segments of a group share one accumulator.  A
// slice value is an integer with |a_1| <= 2^beta and |a_i| <= 2^(beta-1)
// after that, exact in BF16.  The product of two scaled operands keeps the
// slice pairs with i + j <= S + 1:
//
//   x'y' ~ sum_{t=2..S+1} 2^{-beta t} P_t,   P_t = sum_{i+j=t} a_i b_j.
//
// Over a block of OZ_KB K chunks of 32 elements |P_t| < 2^24 (bounds below),
// so the FP32 tensor-core accumulation of P_t (a fresh TMEM accumulator per
// weight t and block) is exact: no rounding happens anywhere in the products.
// The epilogue warps convert each block's P_t to int32 (exact) and add it,
// shifted by beta (S + 1 - t) bits, into int64 running totals, exact too;
// the U element is total * 2^{E_A + E_B - beta (S + 1)} rounded once to FP64.
// The error is that of representing each operand with beta S bits below its
// side's largest magnitude.  U is stored in the FP64 path's layout and the
// FP64 epilogue does the rest.
//
// Kernel structure (one persistent CTA per SM, 10 warps; the same roles as the
// split-precision kernel): warp 0 loads per chunk the S A planes (128 pair
// rows, 64-byte K rows) and S B planes (OZ_N rows of a) with 5-D / 4-D tensor
// maps whose outermost coordinate is the slice; warp 1 issues the S(S+1)/2
// slice-pair MMAs (M = 128, N = OZ_N) into the S weight accumulators of a
// TMEM block of OZ_KB chunks; warps 2-9 drain and accumulate.  Every wait is
// bounded as in the split-precision kernel.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "tc_common.cuh"

namespace tcorr {
namespace {

// t * 2^k as a float-float pair (hi, lo), hi + lo = t 2^k to about 2^-48
// relative, with integer and FP32 operations only: t = t2 2^48 + t1 2^24 + t0
// with |t2| < 2^15 and 0 <= t1, t0 < 2^24, each part exact in FP32; Knuth's
// TwoSum of the two largest, then the smallest added (one rounding, of the
// small parts only); the power-of-two scale is exact in the normal range.
__device__ __forceinline__ float2 int64_to_ff(long long t, int k) {
    const long long t2 = t >> 48;
    const long long rem = t - (t2 << 48);
    const float f2 = (float)(int)t2 * 0x1p48f, f1 = (float)(int)(rem >> 24) * 0x1p24f;
    const float f0 = (float)(int)(rem & 0xffffff);
    float s = f2 + f1, bb = s - f2;
    float e = (f2 - (s - bb)) + (f1 - bb);  // s + e == f2 + f1
    const float s2 = s + f0, b2 = s2 - s;
    e += (s - (s2 - b2)) + (f0 - b2);       // s2 + e == t up to the rounding of e
    const float hi = s2 + e, lo = e - (hi - s2);
    return make_float2(ldexpf(hi, k), ldexpf(lo, k));
}


using namespace tcx;

constexpr int OZ_S = 5;          // slices per operand
constexpr int OZ_BETA = 7;       // bits per slice
constexpr int OZ_N = 96;         // a columns per item
constexpr int OZ_THREADS = 320;
constexpr int OZ_EPI = 256;      // warps 2-9
constexpr int OZ_BM = 128;       // pair rows per tile
constexpr int OZ_ROW = 64;       // K bytes per shared-memory row (32 BF16)
constexpr int OZ_A = OZ_BM * OZ_ROW;        // 8 KB per A plane
constexpr int OZ_B = OZ_N * OZ_ROW;         // 3 KB per B plane
constexpr int OZ_STAGE = OZ_S * (OZ_A + OZ_B);
constexpr int OZ_STAGES = 3;
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE + 1024;
constexpr int OZ_HALF = OZ_N / 2;  // columns per epilogue warp
// One TMEM accumulator block of OZ_S weights x OZ_N columns (single-buffered:
// a block spans OZ_KB chunks, so its drain is short against its MMAs)
static_assert(OZ_S * OZ_N <= 512, "weight accumulators exceed the 512 TMEM columns");
static_assert(OZ_A % 1024 == 0 && OZ_B % 1024 == 0, "planes keep the 64-byte swizzle pattern aligned");
constexpr int OZ_KB = 8;         // K chunks accumulated in TMEM per block (exact, see below)
// Exactness of a block's weight sums in FP32: |a_1| <= 2^beta, |a_i| <= 2^(beta-1)
// for i >= 2; weight t = 0 holds the single pair (1, 1), every other weight
// at most S pairs each with one factor <= 2^(beta-1).
static_assert(32 * OZ_KB * (1 << (2 * OZ_BETA)) < (1 << 24), "weight (1,1) must stay exact in FP32");
static_assert(OZ_S * 32 * OZ_KB * (1 << (2 * OZ_BETA - 1)) < (1 << 24), "weight sums must stay exact in FP32");
static_assert(OZ_HALF % 16 == 0, "the drain loads 16 columns at a time");


// The 15 slice products (i + j <= S + 1) of one K chunk into the five weight
// accumulators (columns t * OZ_N of tmem, t = i + j - 2); a0, b0: descriptor
// low words of the stage's A and B slice planes.  FIRST: the chunk opens the
// accumulator block, so each weight's first product zeroes its accumulator.
template <bool FIRST>
__device__ __forceinline__ void oz_chunk(uint32_t tmem, uint32_t a0, uint32_t b0, uint32_t idesc, int nks) {
#pragma unroll
    for (int t = 0; t < OZ_S; t++) {
#pragma unroll
        for (int ia = 0; ia <= t; ia++) {
            const uint32_t d = tmem + (uint32_t)(t * OZ_N);
            const uint32_t a = a0 + (uint32_t)((ia * OZ_A) >> 4), b = b0 + (uint32_t)(((t - ia) * OZ_B) >> 4);
            if (FIRST && ia == 0) mma_lo<2, 1, false>(d, a, b, idesc);
            else mma_lo<2, 1, true>(d, a, b, idesc);
        }
    }
    if (nks > 1) {
#pragma unroll
        for (int t = 0; t < OZ_S; t++) {
#pragma unroll
            for (int ia = 0; ia <= t; ia++)
                mma_lo<2, 1, true>(tmem + (uint32_t)(t * OZ_N), a0 + (uint32_t)((ia * OZ_A) >> 4) + 2,
                                   b0 + (uint32_t)(((t - ia) * OZ_B) >> 4) + 2, idesc);
        }
    }
}

__global__ void __launch_bounds__(OZ_THREADS, 1) ugemm_oz_kernel(const __grid_constant__ Wave wv) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t bar_full[OZ_STAGES], bar_empty[OZ_STAGES];
    __shared__ __align__(8) uint64_t bar_hfull[2], bar_hempty[2];
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_sh;
    __shared__ SegCache ecache[OZ_EPI / 32];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_dyn) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < OZ_STAGES; s++) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(smem_u32(&bar_hfull[b]), 1);
            mbar_init(smem_u32(&bar_hempty[b]), OZ_EPI);
        }
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    // D = F32, A = B = BF16, K-major, M = 128, N = OZ_N
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_N >> 3) << 17) |
                               ((uint32_t)(OZ_BM >> 4) << 24);

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[OZ_STAGES];
            for (int s = 0; s < OZ_STAGES; s++) last_phase[s] = -1;
            bool ok = true;
            bool inject = wv.inject_stall != 0 && blockIdx.x == 0;
            SegCache sc;
            seg_reset(sc);
            for (int64_t it = blockIdx.x; it < wv.n_gemm && ok; it += gridDim.x) {
                const Item w = decode(wv, it, sc);
                if (w.diag) continue;
                const InstDesc &d = *sc.d;
                const int o = d.dm.o, kv = d.kv, ko = d.ko, nch = 2 * kv + 2 * ko;
                const int s = w.s, pp = w.p, q = w.q;
                const int cb = w.bt * d.pb, cc = w.ct * d.pc, ca = w.n * OZ_N;
                const uint32_t stage_tx = d.stage_tx;
                for (int ch = 0; ch < nch; ch++) {
                    if (!mbar_wait(smem_u32(&bar_empty[stage]), phase ^ 1u, &abort_sh)) {
                        fail(&abort_sh, wv.err, DERR_TIMEOUT_EMPTY);
                        ok = false;
                        break;
                    }
                    const uint32_t full = smem_u32(&bar_full[stage]);
                    mbar_expect_tx(full, stage_tx);
                    last_phase[stage] = (int)phase;
                    const uint32_t sA = sbase + stage * OZ_STAGE, sB = sA + OZ_S * OZ_A;
                    int seg, kk;
                    if (ch < kv) { seg = 0; kk = ch; }
                    else if (ch < 2 * kv) { seg = 1; kk = ch - kv; }
                    else if (ch < 2 * kv + ko) { seg = 2; kk = ch - 2 * kv; }
                    else { seg = 3; kk = ch - 2 * kv - ko; }
                    const int k0 = kk * 32;
                    int amap, aslice, bmap, brow;
                    switch (seg) {
                        case 0: amap = MAP_G_NAT; aslice = q; bmap = MAP_T2R; brow = s * o + pp; break;
                        case 1: amap = MAP_G_SWP; aslice = pp; bmap = MAP_T2R; brow = s * o + q; break;
                        case 2: amap = MAP_T2K_NAT; aslice = pp; bmap = MAP_AON; brow = q * o + s; break;
                        default: amap = MAP_T2K_SWP; aslice = q; bmap = MAP_AON; brow = pp * o + s; break;
                    }
                    if (inject) {
                        inject = false;
                        last_phase[stage] = -1;  // nothing in flight: the consumer's wait must expire
                    } else {
                        for (int pl = 0; pl < OZ_S; pl++) {
                            tma_load_5d(sA + pl * OZ_A, &d.maps[amap][0], full, k0, cc, cb, aslice, pl);
                            tma_load_4d(sB + pl * OZ_B, &d.maps[bmap][0], full, k0, ca, brow, pl);
                        }
                    }
                    if (++stage == OZ_STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {  // let this CTA's copies in flight land before exiting
                for (int s = 0; s < OZ_STAGES; s++) {
                    if (last_phase[s] < 0) continue;
                    const uint64_t t0 = gtimer();
                    while (!mbar_test(smem_u32(&bar_full[s]), (uint32_t)last_phase[s]) &&
                           gtimer() - t0 < WAIT_LIMIT_NS) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t hblk = 0;  // blocks of OZ_KB chunks issued: accumulator phase hblk & 1
            bool ok = true;
            SegCache sc;
            seg_reset(sc);
            for (int64_t it = blockIdx.x; it < wv.n_gemm && ok; it += gridDim.x) {
                const Item w = decode(wv, it, sc);
                if (w.diag) continue;
                const InstDesc &d = *sc.d;
                const int kv = d.kv, ko = d.ko, dp = d.dm.dp, lp = d.dm.lp;
                const int nch = 2 * kv + 2 * ko;
                for (int c0 = 0; c0 < nch && ok; c0 += OZ_KB) {
                    const int nb = min(OZ_KB, nch - c0);
                    for (int cb = 0; cb < nb; cb++) {
                        const int ch = c0 + cb;
                        if (!mbar_wait(smem_u32(&bar_full[stage]), phase, &abort_sh)) {
                            fail(&abort_sh, wv.err, DERR_TIMEOUT_FULL);
                            ok = false;
                            break;
                        }
                        if (cb == 0 && !mbar_wait(smem_u32(&bar_hempty[0]), (hblk & 1u) ^ 1u, &abort_sh)) {
                            fail(&abort_sh, wv.err, DERR_TIMEOUT_TMEM);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t sA = sbase + stage * OZ_STAGE, sB = sA + OZ_S * OZ_A;
                        const int nks = chunk_ksteps(2, kv, ko, dp, lp, ch);
                        // descriptor low words (see mma_lo): plane and K-step offsets are
                        // constants added to the stage's base words.  Every slice product
                        // is exact in FP32, so their order within a block is free: the
                        // first K step of every weight first (the block's opening MMA of
                        // each weight zeroes it), then the second
                        const uint32_t a0 = desc_lo(sA), b0 = desc_lo(sB);
                        if (cb == 0) oz_chunk<true>(tmem, a0, b0, idesc, nks);
                        else oz_chunk<false>(tmem, a0, b0, idesc, nks);
                        tc_commit(smem_u32(&bar_empty[stage]));  // the stage is free once these MMAs are done
                        if (++stage == OZ_STAGES) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    tc_commit(smem_u32(&bar_hfull[0]));
                    hblk++;
                }
            }
        }
    } else {
        const int wq = warp & 3;              // TMEM lane quarter of this warp
        const int half = (warp - 2) >> 2;     // column half of each weight block
        const int row = wq * 32 + lane;       // accumulator row = pair in tile
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        uint32_t hblk = 0;
        bool ok = true;
        SegCache &cs = ecache[warp - 2];
        if (lane == 0) seg_reset(cs);
        __syncwarp();
        for (int64_t it = blockIdx.x; it < wv.n_gemm && ok; it += gridDim.x) {
            SegCache sc = cs;
            const Item w = decode(wv, it, sc);
            __syncwarp();
            if (lane == 0) cs = sc;
            __syncwarp();
            if (w.diag) continue;
            const InstDesc &d = *sc.d;
            const int64_t u_seg = sc.u_off;
            const int v = d.dm.v, vc = d.dm.vc;
            const int nhb = (num_chunks(d) + OZ_KB - 1) / OZ_KB;
            const int lb = row / d.pc, lc = row % d.pc;
            long long tot[OZ_HALF];
#pragma unroll
            for (int j = 0; j < OZ_HALF; j++) tot[j] = 0;
            for (int hb = 0; hb < nhb; hb++) {
                int good = 1;
                if (lane == 0) good = mbar_wait(smem_u32(&bar_hfull[0]), hblk & 1u, &abort_sh) ? 1 : 0;
                good = __shfl_sync(0xffffffffu, good, 0);
                __syncwarp();
                if (!good) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int t = 0; t < OZ_S; t++) {
                    const long long wgt = 1LL << (OZ_BETA * (OZ_S - 1 - t));
#pragma unroll
                    for (int c16 = 0; c16 < OZ_HALF / 16; c16++) {
                        uint32_t r[16];
                        tc_ld16(tmem + lane_off + (uint32_t)(t * OZ_N + half * OZ_HALF + c16 * 16), r);
                        tc_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; j++)
                            tot[c16 * 16 + j] += (long long)__float2int_rn(__uint_as_float(r[j])) * wgt;
                    }
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&bar_hempty[0]));
                hblk++;
            }
            if (!ok) {
                if (lane == 0) fail(&abort_sh, wv.err, DERR_TIMEOUT_TMEM);
                break;
            }
            // U^g[a][b][c] in the FP64 path's layout, each value as a float-float
            // (hi, lo) pair in its 8 bytes (about 48 significant bits), so that the
            // epilogue works on the FP32 pipe; formed from the exact int64 total
            // without the FP64 pipe (int64_to_ff)
            const int b = w.bt * d.pb + lb, c = w.ct * d.pc + lc;
            if (b < v && c < v) {
                const int scale_exp = d.oz_e[0] + d.oz_e[1] - OZ_BETA * (OZ_S + 1);
                const int a0 = w.n * OZ_N + half * OZ_HALF;
                const int64_t stride = (int64_t)v * vc;
                float2 *Ug = static_cast<float2 *>(wv.U) + u_seg + (int64_t)(w.tb * 3 + w.g) * d.dm.ug +
                             (int64_t)b * vc + c + (int64_t)a0 * stride;
#pragma unroll
                for (int j = 0; j < OZ_HALF; j++) {
                    if (a0 + j < v) *Ug = int64_to_ff(tot[j], scale_exp);
                    Ug += stride;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                     : "memory");
    }
}

// ---- slicing ------------------------------------------------------------------------
// Max |x| over n doubles: non-negative doubles order like their bit patterns.
__global__ void maxabs_kernel(const double *__restrict__ x, int64_t n, unsigned long long *out) {
    unsigned long long m = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        m = max(m, (unsigned long long)__double_as_longlong(fabs(x[k])));
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Scale exponents: e[0] for the A side (max of vvvo and t2), e[1] for the B
// side (max of t2 and ooov): the smallest E with max |x| <= 2^E.
__global__ void oz_exponents_kernel(const unsigned long long *m, int *e) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double a = fmax(__longlong_as_double((long long)m[0]), __longlong_as_double((long long)m[1]));
    const double b = fmax(__longlong_as_double((long long)m[1]), __longlong_as_double((long long)m[2]));
    int ea = 0, eb = 0;
    if (a > 0.0) frexp(a, &ea);  // a = f 2^ea, f in [0.5, 1): a < 2^ea
    if (b > 0.0) frexp(b, &eb);
    e[0] = ea;
    e[1] = eb;
}
__global__ void seed_max_kernel(unsigned long long *m, double x) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicMax(m, (unsigned long long)__double_as_longlong(fabs(x)));
}

// out[p][b][c][r] = slice p of scale * in[b*sb + r*sr + c*sc] (r < R), zero for R <= r < Rp,
// with scale = sign * 2^-e[0] read on the device.
// Slices: y = scale * x (|y| <= 1 by choice of scale); for p = 0..S-1:
// y *= 2^beta, a = rint(y), y -= a; all steps exact in FP64.
constexpr int ST = 32;
__global__ void __launch_bounds__(256) slice_pad_kernel(const double *__restrict__ in, __nv_bfloat16 *__restrict__ out,
                                                        int64_t B, int R, int Rp, int64_t C, int64_t sb, int64_t sr,
                                                        int64_t sc, int64_t ob, int64_t oc, int64_t plane,
                                                        const int *e, double sign) {
    __shared__ double tile[ST][ST + 1];
    const double scale = sign * ldexp(1.0, -e[0]);
    const int64_t ntc = (C + ST - 1) / ST, ntr = (Rp + ST - 1) / ST;
    const int64_t ntiles = B * ntc * ntr;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t b = tl / (ntc * ntr);
        const int64_t rem = tl % (ntc * ntr);
        const int64_t c0 = (rem / ntr) * ST;
        const int r0 = (int)(rem % ntr) * ST;
        // load: threads along c when sc == 1, else along r (coalesced either way for the layouts used)
        for (int e = threadIdx.y; e < ST; e += blockDim.y) {
            const int64_t cidx = sc == 1 ? c0 + threadIdx.x : c0 + e;
            const int ridx = sc == 1 ? r0 + e : r0 + threadIdx.x;
            double x = 0.0;
            if (cidx < C && ridx < R) x = in[b * sb + (int64_t)ridx * sr + cidx * sc];
            if (sc == 1) tile[e][threadIdx.x] = x; else tile[threadIdx.x][e] = x;
        }
        __syncthreads();
        for (int e = threadIdx.y; e < ST; e += blockDim.y) {
            const int64_t cidx = c0 + e;
            const int ridx = r0 + threadIdx.x;
            if (cidx < C && ridx < Rp) {
                double y = tile[threadIdx.x][e] * scale;
                const int64_t o = b * ob + cidx * oc + ridx;
#pragma unroll
                for (int p = 0; p < OZ_S; p++) {
                    y *= (double)(1 << OZ_BETA);
                    const double a = rint(y);
                    y -= a;
                    out[p * plane + o] = __double2bfloat16(a);
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

int oz_slices() { return OZ_S; }

cudaError_t launch_maxabs(const double *x, int64_t n, unsigned long long *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 2048);
    maxabs_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, n, out);
    return cudaGetLastError();
}

cudaError_t launch_oz_exponents(const unsigned long long *m, int *e, cudaStream_t st) {
    oz_exponents_kernel<<<1, 32, 0, st>>>(m, e);
    return cudaGetLastError();
}

cudaError_t launch_seed_max(unsigned long long *m, double x, cudaStream_t st) {
    seed_max_kernel<<<1, 32, 0, st>>>(m, x);
    return cudaGetLastError();
}

cudaError_t launch_slice_pad(const double *in, void *out, int64_t B, int R, int Rp, int64_t C, int64_t sb,
                             int64_t sr, int64_t sc, int64_t ob, int64_t oc, int64_t plane, const int *e,
                             double sign, cudaStream_t st) {
    const int64_t ntiles = B * ((C + ST - 1) / ST) * ((Rp + ST - 1) / ST);
    if (ntiles == 0) return cudaSuccess;
    const unsigned grid = (unsigned)(ntiles < ((int64_t)1 << 22) ? ntiles : ((int64_t)1 << 22));
    slice_pad_kernel<<<grid, dim3(ST, 8), 0, st>>>(in, static_cast<__nv_bfloat16 *>(out), B, R, Rp, C, sb, sr, sc,
                                                   ob, oc, plane, e, sign);
    return cudaGetLastError();
}

cudaError_t oz_fill_desc(InstDesc &d, const Operands &op, const int *exps, std::string &err) {
    const int o = d.dm.o, v = d.dm.v, dp = d.dm.dp, lp = d.dm.lp;
    const uint64_t eb = 2;
    const CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const int pb = 8, pc = 16;  // 128 pair rows
    d.pb = pb;
    d.pc = pc;
    d.kb = 1;
    d.nbt = (v + pb - 1) / pb;
    d.nct = (v + pc - 1) / pc;
    d.npass = (v + OZ_N - 1) / OZ_N;
    d.kv = (v + 31) / 32;
    d.ko = (o + 31) / 32;
    d.brows = OZ_N;
    d.stage_tx = (uint32_t)(OZ_S * (OZ_A + OZ_N * OZ_ROW));
    d.oz_e = exps;
    const uint64_t V = v, O = o, S = OZ_S;
    // plane strides (bytes): one slice plane of each operand layout
    const uint64_t pG = (uint64_t)O * V * V * dp * eb, pT2K = (uint64_t)O * V * V * lp * eb;
    const uint64_t pT2R = (uint64_t)O * O * V * dp * eb, pAoN = (uint64_t)O * O * V * lp * eb;
    const uint32_t bk = 32, bpc = (uint32_t)pc, bpb = (uint32_t)pb, bn = (uint32_t)OZ_N;
    {
        uint64_t dims[5] = {V, V, V, O, S};
        uint64_t st[4] = {dp * eb, V * dp * eb, V * V * dp * eb, pG};
        uint32_t box[5] = {bk, bpc, bpb, 1, 1};
        if (!encode(&d.maps[MAP_G_NAT][0], dt, 5, op.G, dims, st, box, err, "G slices")) return cudaErrorInvalidValue;
        uint64_t st2[4] = {V * dp * eb, dp * eb, V * V * dp * eb, pG};
        if (!encode(&d.maps[MAP_G_SWP][0], dt, 5, op.G, dims, st2, box, err, "G slices swapped"))
            return cudaErrorInvalidValue;
    }
    {
        uint64_t dims[5] = {O, V, V, O, S};
        uint64_t st[4] = {lp * eb, V * lp * eb, V * V * lp * eb, pT2K};
        uint32_t box[5] = {bk, bpc, bpb, 1, 1};
        if (!encode(&d.maps[MAP_T2K_NAT][0], dt, 5, op.T2K, dims, st, box, err, "T2K slices"))
            return cudaErrorInvalidValue;
        uint64_t st2[4] = {V * lp * eb, lp * eb, V * V * lp * eb, pT2K};
        if (!encode(&d.maps[MAP_T2K_SWP][0], dt, 5, op.T2K, dims, st2, box, err, "T2K slices swapped"))
            return cudaErrorInvalidValue;
    }
    {
        uint64_t dims[4] = {V, V, O * O, S};
        uint64_t st[3] = {dp * eb, V * dp * eb, pT2R};
        uint32_t box[4] = {bk, bn, 1, 1};
        if (!encode(&d.maps[MAP_T2R][0], dt, 4, op.T2R, dims, st, box, err, "T2R slices")) return cudaErrorInvalidValue;
    }
    {
        uint64_t dims[4] = {O, V, O * O, S};
        uint64_t st[3] = {lp * eb, V * lp * eb, pAoN};
        uint32_t box[4] = {bk, bn, 1, 1};
        if (!encode(&d.maps[MAP_AON][0], dt, 4, op.AoN, dims, st, box, err, "AoN slices")) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

int64_t oz_units_per_task(const InstDesc &d) { return (int64_t)3 * d.nbt * d.nct * d.npass; }

cudaError_t oz_prepare() {
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lk(mu);
    if (done) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(ugemm_oz_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_ugemm_oz(int sm_count, const Wave &w, cudaStream_t st) {
    const int grid = (int)std::min<int64_t>(sm_count, w.n_gemm);
    if (grid <= 0) return cudaSuccess;
    const cudaError_t e = oz_prepare();
    if (e != cudaSuccess) return e;
    ugemm_oz_kernel<<<grid, OZ_THREADS, OZ_SMEM, st>>>(w);
    return cudaGetLastError();
}

}  // namespace tcorr
