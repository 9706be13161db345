// Tensor-core W contractions (S2 + S3, mixed precision) on sm_103a.
//
// Same GEMMs as the FP64 path (see tcorr_internal.cuh): per task and group
// (s;p,q), U^{s;p,q}[a][(b,c)] = sum over K = [d | d | l | l] of
// A[(b,c)][K] * B[a][K].  Each operand x is held as x_hi + x_lo (TF32 or
// BF16, split once in the layout prep); the product uses the three terms
// hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory -- the
// split-precision scheme that replaces the paper's dgemm -> sgemm swap
// (Sec. 3) and keeps the error near FP32 rounding.
//
// Accumulation.  The tensor core adds each instruction's products into the
// FP32 accumulator with truncation, so a long chain of MMAs into one
// accumulator shrinks |U| systematically (relative bias ~ number of chained
// instructions x 2^-24; Ootomo & Yokota 2022 recover FP32 accuracy by
// accumulating outside the tensor core).  Here the three products of each
// K block of KB chunks go into a fresh TMEM accumulator, and the epilogue
// warps fold every block into a register-resident total with
// round-to-nearest FP32 adds.  The block accumulator is double-buffered
// (H0 = TMEM columns [0,256), H1 = [256,512)), so the MMAs of block n+1 run
// while block n is drained.
//
// Kernel structure (one persistent CTA per SM, 10 warps):
//   warp 0  : TMA producer.  Per K chunk it loads A_hi, A_lo (128 pair rows
//             = 8 b x 16 c, one 4-D box of the K-major layout; the swapped
//             pair order (c,b) of two segments is a tensor map with permuted
//             strides, so the tile rows always come out in (b,c) order) and
//             B_hi, B_lo (up to 256 rows of a) into a 4-stage ring, 64-byte
//             swizzled rows.
//   warp 1  : allocates 512 TMEM columns; one thread issues tcgen05.mma
//             (M = 128, N <= 256, 2 K-steps x 3 products per chunk) into the
//             accumulator of the current K block of KB = 2 chunks.
//   warps 2-9: two warps per TMEM lane quarter, 128 columns each: drain each
//             block into the register total, then store the U rows (rows of
//             16 consecutive c, coalesced) at the end of the tile.
// A work item is (task, group, pair tile, N pass of 256 a values).  Every
// mbarrier wait is bounded (wall clock): on expiry the kernel sets an error
// flag, stops all roles, waits (bounded) for its own copies in flight, frees
// TMEM and returns; the host reports TCORR_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int TC_THREADS = 320;
constexpr int EPI_THREADS = 256;  // warps 2-9
constexpr int STAGES = 4;
constexpr int BM = 128;                 // pair rows per tile
constexpr int PB = 8, PC = 16;          // pair tile = PB values of b x PC values of c
constexpr int BN = 256;                 // a columns per accumulator
constexpr int ROW_BYTES = 64;           // K bytes per smem row (SWIZZLE_64B span)
constexpr int A_BYTES = BM * ROW_BYTES; // 8 KB
constexpr int B_BYTES = BN * ROW_BYTES; // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s of wall time per wait ...
constexpr uint32_t WAIT_MIN_POLLS = 1u << 18;      // ... and at least this many polls, so that time
                                                   // spent off the GPU (pre-emption) never counts

enum { MAP_G_NAT = 0, MAP_G_SWP, MAP_T2K_NAT, MAP_T2K_SWP, MAP_T2R, MAP_AON, NMAP };

struct TcParams {
    CUtensorMap map[NMAP][2];  // [operand map][hi, lo]
    Dims dm;
    const int *tasks;
    int64_t task0;
    float *U;
    int *err;
    int nbt, nct, npass, kv, ko, brows;
    int64_t nitems;
    uint32_t idesc_base;
    uint32_t stage_tx;
    int kb;            // K chunks per accumulator block
    int inject_stall;  // testing only: CTA 0 withholds the loads of its first chunk
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on one mbarrier phase; false on expiry (both the wall-time
// and the poll limit passed) or when another role has already aborted.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    if (mbar_test(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_test(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (*abort_flag) return false;
            if (it >= WAIT_MIN_POLLS && gtimer() - t0 > WAIT_LIMIT_NS) return false;
        }
    }
}
__device__ __forceinline__ void fail(volatile int *abort_flag, int *err, int code) {
    *abort_flag = 1;
    atomicOr(err, code);
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
// K-major operand tile with 64-byte rows and 64-byte swizzle: 8-row groups
// are 512 bytes apart (SBO); LBO is unused for swizzled K-major layouts.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
template <int KIND>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
    if constexpr (KIND == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct Item {
    int tb, g, bt, ct, n;
};
__device__ __forceinline__ Item decode(const TcParams &p, int64_t it) {
    Item r;
    r.n = (int)(it % p.npass);
    it /= p.npass;
    r.ct = (int)(it % p.nct);
    it /= p.nct;
    r.bt = (int)(it % p.nbt);
    it /= p.nbt;
    r.g = (int)(it % 3);
    r.tb = (int)(it / 3);
    return r;
}
// (s; p, q) of group g of the task
__device__ __forceinline__ void group_indices(const TcParams &p, const Item &w, int &s, int &pp, int &q,
                                              bool &diag) {
    const int *tk = p.tasks + 3 * (p.task0 + w.tb);
    const int i = tk[0], j = tk[1], k = tk[2];
    diag = (i == j && j == k);
    if (w.g == 0) { s = i; pp = j; q = k; }
    else if (w.g == 1) { s = j; pp = i; q = k; }
    else { s = k; pp = i; q = j; }
}

template <int KIND>
__global__ void __launch_bounds__(TC_THREADS, 1) ugemm_tc_kernel(const __grid_constant__ TcParams p) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t bar_full[STAGES], bar_empty[STAGES];
    __shared__ __align__(8) uint64_t bar_hfull[2], bar_hempty[2];
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_dyn) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(smem_u32(&bar_hfull[b]), 1);
            mbar_init(smem_u32(&bar_hempty[b]), EPI_THREADS);
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

    const int v = p.dm.v, o = p.dm.o;
    const int nch = 2 * p.kv + 2 * p.ko;
    const int kch = ROW_BYTES / (KIND == 1 ? 4 : 2);

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[STAGES];
            for (int s = 0; s < STAGES; s++) last_phase[s] = -1;
            bool ok = true;
            bool inject = p.inject_stall != 0 && blockIdx.x == 0;
            for (int64_t it = blockIdx.x; it < p.nitems && ok; it += gridDim.x) {
                const Item w = decode(p, it);
                int s, pp, q;
                bool diag;
                group_indices(p, w, s, pp, q, diag);
                if (diag) continue;
                const int cb = w.bt * PB, cc = w.ct * PC, ca = w.n * BN;
                for (int ch = 0; ch < nch; ch++) {
                    if (!mbar_wait(smem_u32(&bar_empty[stage]), phase ^ 1u, &abort_sh)) {
                        fail(&abort_sh, p.err, DERR_TIMEOUT_EMPTY);
                        ok = false;
                        break;
                    }
                    const uint32_t full = smem_u32(&bar_full[stage]);
                    mbar_expect_tx(full, p.stage_tx);
                    last_phase[stage] = (int)phase;
                    const uint32_t sA = sbase + stage * STAGE_BYTES, sAl = sA + A_BYTES;
                    const uint32_t sB = sAl + A_BYTES, sBl = sB + B_BYTES;
                    int seg, kk;
                    if (ch < p.kv) { seg = 0; kk = ch; }
                    else if (ch < 2 * p.kv) { seg = 1; kk = ch - p.kv; }
                    else if (ch < 2 * p.kv + p.ko) { seg = 2; kk = ch - 2 * p.kv; }
                    else { seg = 3; kk = ch - 2 * p.kv - p.ko; }
                    const int k0 = kk * kch;
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
                        tma_load_4d(sA, &p.map[amap][0], full, k0, cc, cb, aslice);
                        tma_load_4d(sAl, &p.map[amap][1], full, k0, cc, cb, aslice);
                        tma_load_3d(sB, &p.map[bmap][0], full, k0, ca, brow);
                        tma_load_3d(sBl, &p.map[bmap][1], full, k0, ca, brow);
                    }
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {  // let this CTA's copies in flight land before exiting
                for (int s = 0; s < STAGES; s++) {
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
            uint32_t hblk = 0;  // K blocks issued so far: buffer hblk & 1, phase (hblk >> 1) & 1
            bool ok = true;
            for (int64_t it = blockIdx.x; it < p.nitems && ok; it += gridDim.x) {
                const Item w = decode(p, it);
                int s, pp, q;
                bool diag;
                group_indices(p, w, s, pp, q, diag);
                if (diag) continue;
                const int nvalid = min(BN, v - w.n * BN);
                const int N = (nvalid + 15) / 16 * 16;
                const uint32_t idesc = p.idesc_base | ((uint32_t)(N >> 3) << 17);
                // K blocks of kb chunks: the small hi*lo and lo*hi products of each
                // chunk are issued as its data lands, the dominant hi*hi products of
                // the whole block last, so that the truncation of every instruction
                // acts on the smallest possible accumulator; the block's stages are
                // released together once its last MMA is issued.
                for (int c0 = 0; c0 < nch && ok; c0 += p.kb) {
                    const int nb = min(p.kb, nch - c0);
                    const uint32_t buf = hblk & 1u;
                    int st0 = stage;
                    for (int cb = 0; cb < nb; cb++) {
                        if (!mbar_wait(smem_u32(&bar_full[stage]), phase, &abort_sh)) {
                            fail(&abort_sh, p.err, DERR_TIMEOUT_FULL);
                            ok = false;
                            break;
                        }
                        if (cb == 0 &&
                            !mbar_wait(smem_u32(&bar_hempty[buf]), ((hblk >> 1) & 1u) ^ 1u, &abort_sh)) {
                            fail(&abort_sh, p.err, DERR_TIMEOUT_TMEM);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t d = tmem + buf * (uint32_t)BN;
                        const uint32_t sA = sbase + stage * STAGE_BYTES, sAl = sA + A_BYTES;
                        const uint32_t sB = sAl + A_BYTES, sBl = sB + B_BYTES;
#pragma unroll
                        for (int kk = 0; kk < 2; kk++) {
                            const uint32_t off = kk * 32;
                            tc_mma<KIND>(d, sdesc(sA + off), sdesc(sBl + off), idesc,
                                         (cb > 0 || kk > 0) ? 1u : 0u);
                            tc_mma<KIND>(d, sdesc(sAl + off), sdesc(sB + off), idesc, 1u);
                        }
                        if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    const uint32_t d = tmem + buf * (uint32_t)BN;
                    int sj = st0;
                    for (int cb = 0; cb < nb; cb++) {
                        const uint32_t sA = sbase + sj * STAGE_BYTES, sB = sA + 2 * A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < 2; kk++) {
                            const uint32_t off = kk * 32;
                            tc_mma<KIND>(d, sdesc(sA + off), sdesc(sB + off), idesc, 1u);
                        }
                        if (++sj == STAGES) sj = 0;
                    }
                    sj = st0;
                    for (int cb = 0; cb < nb; cb++) {
                        tc_commit(smem_u32(&bar_empty[sj]));
                        if (++sj == STAGES) sj = 0;
                    }
                    tc_commit(smem_u32(&bar_hfull[buf]));
                    hblk++;
                }
            }
        }
    } else {
        const int wq = warp & 3;              // TMEM lane quarter of this warp
        const int half = (warp - 2) >> 2;     // column half [half*128, half*128 + 128)
        const int row = wq * 32 + lane;       // accumulator row = pair in tile
        const int lb = row / PC, lc = row % PC;
        const int64_t v2 = (int64_t)v * v;
        const int vc = p.dm.vc;
        const int nhb = (nch + p.kb - 1) / p.kb;
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        uint32_t hblk = 0;
        bool ok = true;
        for (int64_t it = blockIdx.x; it < p.nitems && ok; it += gridDim.x) {
            const Item w = decode(p, it);
            int s, pp, q;
            bool diag;
            group_indices(p, w, s, pp, q, diag);
            if (diag) continue;
            float total[128];
#pragma unroll
            for (int j = 0; j < 128; j++) total[j] = 0.f;
            for (int hb = 0; hb < nhb; hb++) {
                const uint32_t buf = hblk & 1u;
                int good = 1;
                if (lane == 0) good = mbar_wait(smem_u32(&bar_hfull[buf]), (hblk >> 1) & 1u, &abort_sh) ? 1 : 0;
                good = __shfl_sync(0xffffffffu, good, 0);
                __syncwarp();
                if (!good) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int c4 = 0; c4 < 4; c4++) {
                    uint32_t r[32];
                    tc_ld32(tmem + lane_off + buf * (uint32_t)BN + (uint32_t)(half * 128 + c4 * 32), r);
#pragma unroll
                    for (int j = 0; j < 32; j++) total[c4 * 32 + j] += __uint_as_float(r[j]);
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&bar_hempty[buf]));
                hblk++;
            }
            if (!ok) {
                if (lane == 0) fail(&abort_sh, p.err, DERR_TIMEOUT_TMEM);
                break;
            }
            // rows of 16 consecutive c per half warp: group 0 and 2 in their own
            // [a][b][c] order, group 1 at [b][a][c] (aligned with W, see tcorr_internal.cuh)
            const int b = w.bt * PB + lb, c = w.ct * PC + lc;
            if (b < v && c < v) {
                const int a0 = w.n * BN + half * 128;
                const int64_t stride = w.g == 1 ? (int64_t)vc : (int64_t)v * vc;
                const int64_t base = w.g == 1 ? (int64_t)b * v * vc + c : (int64_t)b * vc + c;
                float *Ug = p.U + (int64_t)(w.tb * 3 + w.g) * v2 * vc + base + (int64_t)a0 * stride;
                const int na = min(128, v - a0);
                if (na == 128) {
#pragma unroll
                    for (int j = 0; j < 128; j++) {
                        *Ug = total[j];
                        Ug += stride;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 128; j++) {
                        if (j < na) *Ug = total[j];
                        Ug += stride;
                    }
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

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    return fn;
}

bool encode(CUtensorMap *m, CUtensorMapDataType dt, int rank, void *base, const uint64_t *dims,
            const uint64_t *strides_bytes, const uint32_t *box, std::string &err, const char *what) {
    auto fn = get_encode();
    if (!fn) {
        err = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    uint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(m, dt, (cuuint32_t)rank, base, (const cuuint64_t *)dims, (const cuuint64_t *)strides_bytes,
                    (const cuuint32_t *)box, (const cuuint32_t *)es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = std::string("cuTensorMapEncodeTiled failed for ") + what + " (CUresult " + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}

}  // namespace

bool tc_supported(int cc_major, int cc_minor) { return cc_major == 10 && cc_minor == 3; }

cudaError_t tc_build_tensor_maps(Handle *h, std::string &err) {
    const int o = h->dm.o, v = h->dm.v, dp = h->dm.dp, lp = h->dm.lp;
    const bool tf = h->prec == TCORR_TF32X3;
    const uint64_t eb = tf ? 4 : 2;
    const CUtensorMapDataType dt = tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const uint32_t kch = ROW_BYTES / (uint32_t)eb;
    const uint32_t brows = (uint32_t)std::min(BN, round_up(v, 16));
    auto *maps = static_cast<CUtensorMap *>(aligned_alloc(64, sizeof(CUtensorMap) * NMAP * 2));
    if (!maps) {
        err = "host allocation failed";
        return cudaErrorMemoryAllocation;
    }
    free(h->tmaps);
    h->tmaps = maps;
    const uint64_t V = v, O = o;
    void *hi[4] = {h->op.G, h->op.T2K, h->op.T2R, h->op.AoN};
    void *lo[4] = {h->op.Glo, h->op.T2Klo, h->op.T2Rlo, h->op.AoNlo};
    for (int part = 0; part < 2; part++) {
        void *const *src = part == 0 ? hi : lo;
        {   // G natural: (d, c, b, q) with c = y index, b = x index
            uint64_t dims[4] = {V, V, V, O};
            uint64_t st[3] = {dp * eb, V * dp * eb, V * V * dp * eb};
            uint32_t box[4] = {kch, PC, PB, 1};
            if (!encode(&maps[MAP_G_NAT * 2 + part], dt, 4, src[0], dims, st, box, err, "G")) return cudaErrorInvalidValue;
        }
        {   // G swapped: (d, c, b, q) with c = x index, b = y index
            uint64_t dims[4] = {V, V, V, O};
            uint64_t st[3] = {V * dp * eb, dp * eb, V * V * dp * eb};
            uint32_t box[4] = {kch, PC, PB, 1};
            if (!encode(&maps[MAP_G_SWP * 2 + part], dt, 4, src[0], dims, st, box, err, "G swapped"))
                return cudaErrorInvalidValue;
        }
        {   // T2K natural
            uint64_t dims[4] = {O, V, V, O};
            uint64_t st[3] = {lp * eb, V * lp * eb, V * V * lp * eb};
            uint32_t box[4] = {kch, PC, PB, 1};
            if (!encode(&maps[MAP_T2K_NAT * 2 + part], dt, 4, src[1], dims, st, box, err, "T2K")) return cudaErrorInvalidValue;
        }
        {   // T2K swapped
            uint64_t dims[4] = {O, V, V, O};
            uint64_t st[3] = {V * lp * eb, lp * eb, V * V * lp * eb};
            uint32_t box[4] = {kch, PC, PB, 1};
            if (!encode(&maps[MAP_T2K_SWP * 2 + part], dt, 4, src[1], dims, st, box, err, "T2K swapped"))
                return cudaErrorInvalidValue;
        }
        {   // T2R: (d, a, s*o+p)
            uint64_t dims[3] = {V, V, O * O};
            uint64_t st[2] = {dp * eb, V * dp * eb};
            uint32_t box[3] = {kch, brows, 1};
            if (!encode(&maps[MAP_T2R * 2 + part], dt, 3, src[2], dims, st, box, err, "T2R")) return cudaErrorInvalidValue;
        }
        {   // AoN: (l, a, q*o+s)
            uint64_t dims[3] = {O, V, O * O};
            uint64_t st[2] = {lp * eb, V * lp * eb};
            uint32_t box[3] = {kch, brows, 1};
            if (!encode(&maps[MAP_AON * 2 + part], dt, 3, src[3], dims, st, box, err, "AoN")) return cudaErrorInvalidValue;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_ugemm_tc(Handle *h, const GemmArgs &ga, cudaStream_t st) {
    static_assert(sizeof(TcParams) < 4000, "kernel parameter block too large");
    const bool tf = h->prec == TCORR_TF32X3;
    const int v = ga.dm.v, o = ga.dm.o;
    const int kch = ROW_BYTES / (tf ? 4 : 2);
    TcParams p;
    memcpy(p.map, h->tmaps, sizeof(p.map));
    p.dm = ga.dm;
    p.tasks = ga.tasks;
    p.task0 = ga.task0;
    p.U = static_cast<float *>(ga.U);
    p.err = h->err;
    p.nbt = (v + PB - 1) / PB;
    p.nct = (v + PC - 1) / PC;
    p.npass = (v + BN - 1) / BN;
    p.kv = (v + kch - 1) / kch;
    p.ko = (o + kch - 1) / kch;
    p.brows = std::min(BN, round_up(v, 16));
    p.nitems = (int64_t)ga.ntb * 3 * p.nbt * p.nct * p.npass;
    // instruction descriptor: D = F32, A/B = TF32 (2) or BF16 (1), K-major, M = 128
    const uint32_t fmt = tf ? 2u : 1u;
    p.idesc_base = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BM >> 4) << 24);
    p.stage_tx = (uint32_t)(2 * A_BYTES + 2 * p.brows * ROW_BYTES);
    p.kb = 2;  // chunks per accumulator block (at most STAGES - 1: a block holds its stages)
    p.inject_stall = h->inject_stall;
    const int grid = (int)std::min<int64_t>(h->sm_count, p.nitems);
    if (grid <= 0) return cudaSuccess;
    cudaError_t e;
    if (tf) {
        static bool attr = false;
        if (!attr) {
            e = cudaFuncSetAttribute(ugemm_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        ugemm_tc_kernel<1><<<grid, TC_THREADS, SMEM_BYTES, st>>>(p);
    } else {
        static bool attr = false;
        if (!attr) {
            e = cudaFuncSetAttribute(ugemm_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        ugemm_tc_kernel<2><<<grid, TC_THREADS, SMEM_BYTES, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace tcorr
