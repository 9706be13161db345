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
//             block into the register total, then store the tile into the
//             8^3-cube layout of U (whole 32-byte sectors per 8 values of a).
// A work item is (task, group, pair tile, N pass).  The v values of a are cut
// into ceil(v / 256) passes of equal width (a multiple of 16, at most 256), so
// the B tiles carry no more padding rows than the rounding needs.  Every
// mbarrier wait is bounded (wall clock): on expiry the kernel sets an error
// flag, stops all roles, waits (bounded) for its own copies in flight, frees
// TMEM and returns; the host reports TCORR_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "tc_common.cuh"

namespace tcorr {
namespace {

using namespace tcx;

constexpr int TC_THREADS = 320;
constexpr int EPI_THREADS = 256;  // warps 2-9
constexpr int MAX_STAGES = 8;
constexpr int BM = 128;                 // pair rows per tile (pb values of b x pc values of c)
constexpr int BN = 256;                 // a columns per accumulator
constexpr int ROW_BYTES = 64;           // K bytes per smem row (SWIZZLE_64B span)
constexpr int A_BYTES = BM * ROW_BYTES; // 8 KB
constexpr int B_BYTES = BN * ROW_BYTES; // 16 KB
// The ring: 192 KB cut into stages of 2 A planes + 2 B planes of the wave's
// largest B tile (brows rows): 4 stages for 256-row B tiles, up to 8 for small v
constexpr int RING_BYTES = 4 * (2 * A_BYTES + 2 * B_BYTES);
constexpr int SMEM_BYTES = RING_BYTES + 1024;
// The operand type (TF32 or BF16) is a property of each problem (InstDesc::kind),
// so problems of both types can share a wave.
__global__ void __launch_bounds__(TC_THREADS, 1) ugemm_tc_kernel(const __grid_constant__ Wave wv) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t bar_full[MAX_STAGES], bar_empty[MAX_STAGES];
    __shared__ __align__(8) uint64_t bar_hfull[2], bar_hempty[2];
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_sh;
    __shared__ SegCache ecache[EPI_THREADS / 32];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_dyn) + 1023u) & ~1023u;
    const uint32_t b_plane = (uint32_t)wv.tc_brows * ROW_BYTES;     // multiple of 1024
    const uint32_t stage_bytes = 2u * A_BYTES + 2u * b_plane;
    const int nst = min(MAX_STAGES, (int)(RING_BYTES / stage_bytes));

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; s++) {
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

    // instruction descriptor: D = F32, A/B = TF32 (2) or BF16 (1), K-major, M = 128
    constexpr uint32_t idesc_m = (1u << 4) | ((uint32_t)(BM >> 4) << 24);

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[MAX_STAGES];
            for (int s = 0; s < MAX_STAGES; s++) last_phase[s] = -1;
            bool ok = true;
            bool inject = wv.inject_stall != 0 && blockIdx.x == 0;
            SegCache sc;
            seg_reset(sc);
            for (int64_t it = blockIdx.x; it < wv.n_gemm && ok; it += gridDim.x) {
                const Item w = decode(wv, it, sc);
                if (w.diag) continue;
                const InstDesc &d = *sc.d;
                const int o = d.dm.o, kv = d.kv, ko = d.ko, nch = num_chunks(d);
                const int kch = ROW_BYTES / (d.kind == 1 ? 4 : 2);
                const int s = w.s, pp = w.p, q = w.q;
                const int cb = w.bt * d.pb, cc = w.ct * d.pc, ca = w.n * d.brows;
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
                    const uint32_t sA = sbase + stage * stage_bytes, sAl = sA + A_BYTES;
                    const uint32_t sB = sAl + A_BYTES, sBl = sB + b_plane;
                    int seg, kk;
                    if (ch < kv) { seg = 0; kk = ch; }
                    else if (ch < 2 * kv) { seg = 1; kk = ch - kv; }
                    else if (ch < 2 * kv + ko) { seg = 2; kk = ch - 2 * kv; }
                    else { seg = 3; kk = ch - 2 * kv - ko; }
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
                        tma_load_4d(sA, &d.maps[amap][0], full, k0, cc, cb, aslice);
                        tma_load_4d(sAl, &d.maps[amap][1], full, k0, cc, cb, aslice);
                        tma_load_3d(sB, &d.maps[bmap][0], full, k0, ca, brow);
                        tma_load_3d(sBl, &d.maps[bmap][1], full, k0, ca, brow);
                    }
                    if (++stage == nst) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {  // let this CTA's copies in flight land before exiting
                for (int s = 0; s < nst; s++) {
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
            MmaRing rg;
            rg.full0 = smem_u32(&bar_full[0]);
            rg.empty0 = smem_u32(&bar_empty[0]);
            rg.hfull0 = smem_u32(&bar_hfull[0]);
            rg.hempty0 = smem_u32(&bar_hempty[0]);
            rg.lo0 = desc_lo(sbase);
            rg.step = stage_bytes >> 4;
            rg.a16 = A_BYTES >> 4;
            rg.b16 = b_plane >> 4;
            rg.nst = nst;
            rg.stage = 0;
            rg.phase = 0;
            rg.hblk = 0;
            SegCache sc;
            seg_reset(sc);
            for (int64_t it = blockIdx.x; it < wv.n_gemm; it += gridDim.x) {
                const Item w = decode(wv, it, sc);
                if (w.diag) continue;
                const InstDesc &d = *sc.d;
                const int kv = d.kv, ko = d.ko, nch = 2 * kv + 2 * ko, kind = d.kind;
                const bool dh = kind == 2 && (d.dm.dp & 31) != 0, lh = kind == 2 && (d.dm.lp & 31) != 0;
                const int nvalid = min(d.brows, d.dm.v - w.n * d.brows);
                const int N = (nvalid + 15) / 16 * 16;
                const uint32_t fmt = kind == 1 ? 2u : 1u;
                const uint32_t idesc = idesc_m | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17);
                // the small hi*lo and lo*hi products of each chunk are issued as it
                // lands, the dominant hi*hi products of the K block last, so that the
                // truncation of every instruction acts on the smallest possible
                // accumulator; each stage is released right after its last product
                int code = 0;
                const bool good = kind == 1
                    ? mma_item<1, 1>(rg, tmem, idesc, nch, -1, -1, -1, -1, &abort_sh, &code)
                    : mma_item<2, 1>(rg, tmem, idesc, nch, dh ? kv - 1 : -1, dh ? 2 * kv - 1 : -1,
                                     lh ? 2 * kv + ko - 1 : -1, lh ? nch - 1 : -1, &abort_sh, &code);
                if (!good) {
                    fail(&abort_sh, wv.err, code);
                    break;
                }
            }
        }
    } else {
        const int wq = warp & 3;              // TMEM lane quarter of this warp
        const int half = (warp - 2) >> 2;     // column half of the accumulator
        const int row = wq * 32 + lane;       // accumulator row = pair in tile
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        uint32_t hblk = 0;
        bool ok = true;
        // the decode cache of an epilogue warp lives in shared memory: in
        // registers it would compete with the 128-column running total
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
            const int v = d.dm.v;
            const int nhb = (num_chunks(d) + d.kb - 1) / d.kb;
            const int lb = row / d.pc, lc = row % d.pc;
            // the two warps of a lane quarter split the accumulator's N columns:
            // 128 each for N > 128, else 32 or 64 each (only columns < N are read)
            const int pass0 = w.n * d.brows, pass_end = min(v, pass0 + d.brows);
            const int N = (pass_end - pass0 + 15) / 16 * 16;
            const int wh = N > 128 ? 128 : (N > 64 ? 64 : 32);
            const int nld = wh / 32;
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
                // 32 columns per wait, loaded as two 16-column halves (register budget)
#pragma unroll
                for (int c4 = 0; c4 < 4; c4++) {
                    if (c4 < nld) {  // warp-uniform
                        uint32_t r[16], r2[16];
                        const uint32_t ta = tmem + lane_off + buf * (uint32_t)BN + (uint32_t)(half * wh + c4 * 32);
                        tc_ld16(ta, r);
                        tc_ld16(ta + 16, r2);
                        tc_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; j++) total[c4 * 32 + j] += __uint_as_float(r[j]);
#pragma unroll
                        for (int j = 0; j < 16; j++) total[c4 * 32 + 16 + j] += __uint_as_float(r2[j]);
                    }
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&bar_hempty[buf]));
                hblk++;
            }
            if (!ok) {
                if (lane == 0) fail(&abort_sh, wv.err, DERR_TIMEOUT_TMEM);
                break;
            }
            // each group as its term of W, in 8^3 cubes (tcorr_internal.cuh)
            const int b = w.bt * d.pb + lb, c = w.ct * d.pc + lc;
            if (b < v && c < v) {
                const int a0 = pass0 + half * wh;  // a multiple of 8
                float *Ut = static_cast<float *>(wv.U) + u_seg + (int64_t)w.tb * 3 * d.dm.ug;
                store_u_cubes(Ut, (v + 7) >> 3, w.g, a0, b, c, min(wh, pass_end - a0), total);
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

// ---- SM-pair variant (tcgen05 cta_group::2) ---------------------------------
//
// Two CTAs of a thread-block cluster (one per SM of an SM pair) compute one
// M = 256 tile: each loads its own 128-pair A tile and half of the B tile
// (N/2 rows of a), and one thread of the even CTA ("leader") issues
// tcgen05.mma.cta_group::2, which reads A and B from both CTAs' shared memory
// and accumulates each CTA's 128 rows in that CTA's tensor memory.  Per K
// chunk an SM then ingests 16 KB of A and N/2 x 128 bytes of B (32 KB at
// N = 256) instead of 48 KB, for the same tensor work per SM: the per-SM
// operand-ingest rate, not the tensor pipe, bounds the single-SM kernel.
//
// The pair's two 128-pair tiles are consecutive tiles of the flattened
// (b tile, c tile) list of a group: work item = (task, tile pair, group,
// N pass); a tile index past the list is TMA zero fill and is not stored.
//
// Hand-offs (all bounded waits, as in the single-SM kernel):
//  - each CTA's producer waits on its own "empty" barrier of a stage (the
//    leader's MMA commits arrive on both CTAs' barriers), and signals its
//    loads on the LEADER's "full" barrier, for which the leader's producer
//    expects the bytes of both CTAs;
//  - the leader's MMA commits each accumulator block to both CTAs' "hfull"
//    barriers; each drain warp of either CTA arrives once on the leader's
//    "hempty" barrier (16 arrivals) when it has read the block;
//  - an expired wait sets the abort flag of both CTAs and the device error
//    flag; before the pair tears down, the leader waits (bounded) for its
//    issued MMAs, and a producer that aborted lets its copies in flight land.
// Teardown: a cluster barrier (every role of both CTAs ends after bounded
// waits), then both CTAs free the pair's tensor memory.
constexpr int PAIR_HEMPTY_ARRIVALS = 2 * (EPI_THREADS / 32);

struct PairItem {
    Item it;
    bool empty;  // this CTA's tile index lies past the group's tile list
};
__device__ __forceinline__ PairItem decode_pair(const Wave &w, int64_t it, SegCache &c, uint32_t rank) {
    seg_update(w, it, c);
    PairItem r;
    const int npt = c.nbt * c.nct;
    const int npair = (npt + 1) / 2;
    int64_t x = it - c.begin;
    r.it.n = (int)(x % c.npass);  // N pass fastest, then group, then tile pair (as decode)
    x /= c.npass;
    r.it.g = (int)(x % 3);
    x /= 3;
    const int t = (int)(x % npair) * 2 + (int)rank;
    r.it.tb = (int)(x / npair);
    r.empty = t >= npt;
    r.it.bt = r.empty ? c.nbt : t / c.nct;  // past the list: b >= v, all TMA fill
    r.it.ct = r.empty ? 0 : t % c.nct;
    if (r.it.tb != c.tcached) {
        const int *tk = c.d->tasks + 3 * (c.task0 + r.it.tb);
        c.ti = tk[0];
        c.tj = tk[1];
        c.tk = tk[2];
        c.tcached = r.it.tb;
    }
    const int i = c.ti, j = c.tj, k = c.tk;
    r.it.diag = (i == j && j == k);
    if (r.it.g == 0) { r.it.s = i; r.it.p = j; r.it.q = k; }
    else if (r.it.g == 1) { r.it.s = j; r.it.p = i; r.it.q = k; }
    else { r.it.s = k; r.it.p = i; r.it.q = j; }
    return r;
}
// abort both CTAs of the pair and raise the device error flag
__device__ __forceinline__ void fail_pair(volatile int *abort_flag, uint32_t peer_abort_cl, int *err, int code) {
    *abort_flag = 1;
    st_cluster_u32(peer_abort_cl, 1u);
    atomicOr(err, code);
}
__device__ __forceinline__ void spin_ns(uint64_t ns) {
    const uint64_t t0 = gtimer();
    while (gtimer() - t0 < ns) {
    }
}

__global__ void __launch_bounds__(TC_THREADS, 1) ugemm_tc_pair_kernel(const __grid_constant__ Wave wv) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t bar_full[MAX_STAGES], bar_empty[MAX_STAGES];
    __shared__ __align__(8) uint64_t bar_hfull[2], bar_hempty[2];
    __shared__ __align__(8) uint64_t bar_fin;
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_sh;
    __shared__ SegCache ecache[EPI_THREADS / 32];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_rank(), cid = cluster_id(), ncl = cluster_count();
    const bool leader = rank == 0;
    const uint32_t sbase = (smem_u32(smem_dyn) + 1023u) & ~1023u;
    const uint32_t b_half = (uint32_t)wv.tc_brows / 2;                       // B rows per CTA
    const uint32_t b_plane = (b_half * ROW_BYTES + 1023u) & ~1023u;
    const uint32_t stage_bytes = 2u * A_BYTES + 2u * b_plane;
    const int nst = min(MAX_STAGES, (int)(RING_BYTES / stage_bytes));
    const uint32_t peer_abort = peer_addr(smem_u32((const void *)&abort_sh), rank ^ 1u);

    if (threadIdx.x == 0) {
        for (int s = 0; s < nst; s++) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(smem_u32(&bar_hfull[b]), 1);
            mbar_init(smem_u32(&bar_hempty[b]), PAIR_HEMPTY_ARRIVALS);
        }
        mbar_init(smem_u32(&bar_fin), 1);
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // both CTAs' barriers exist before any remote signal
    tc_fence_after();
    const uint32_t tmem = tmem_holder;
    // instruction descriptor: D = F32, K-major A and B, M = 256 over the pair
    constexpr uint32_t idesc_m = (1u << 4) | ((uint32_t)(2 * BM >> 4) << 24);

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[MAX_STAGES];
            for (int s = 0; s < MAX_STAGES; s++) last_phase[s] = -1;
            bool ok = true;
            bool inject = wv.inject_stall != 0 && cid == 0 && leader;
            SegCache sc;
            seg_reset(sc);
            for (int64_t it = cid; it < wv.n_gemm && ok; it += ncl) {
                const PairItem pw = decode_pair(wv, it, sc, rank);
                const Item &w = pw.it;
                if (w.diag) continue;
                const InstDesc &d = *sc.d;
                const int o = d.dm.o, kv = d.kv, ko = d.ko, nch = num_chunks(d);
                const int kch = ROW_BYTES / (d.kind == 1 ? 4 : 2);
                const int s = w.s, pp = w.p, q = w.q;
                const int nvalid = min(d.brows, d.dm.v - w.n * d.brows);
                const int N = (nvalid + 15) / 16 * 16;
                const int cb = w.bt * d.pb, cc = w.ct * d.pc, ca = w.n * d.brows + (int)rank * (N / 2);
                const uint32_t stage_tx = d.stage_tx;  // both CTAs' bytes
                for (int ch = 0; ch < nch; ch++) {
                    if (!mbar_wait(smem_u32(&bar_empty[stage]), phase ^ 1u, &abort_sh)) {
                        fail_pair(&abort_sh, peer_abort, wv.err, DERR_TIMEOUT_EMPTY);
                        ok = false;
                        break;
                    }
                    const uint32_t full = smem_u32(&bar_full[stage]);
                    if (leader) mbar_expect_tx(full, stage_tx);
                    const uint32_t full_l = peer_addr(full, 0);
                    last_phase[stage] = (int)phase;
                    const uint32_t sA = sbase + stage * stage_bytes, sAl = sA + A_BYTES;
                    const uint32_t sB = sAl + A_BYTES, sBl = sB + b_plane;
                    int seg, kk;
                    if (ch < kv) { seg = 0; kk = ch; }
                    else if (ch < 2 * kv) { seg = 1; kk = ch - kv; }
                    else if (ch < 2 * kv + ko) { seg = 2; kk = ch - 2 * kv; }
                    else { seg = 3; kk = ch - 2 * kv - ko; }
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
                        last_phase[stage] = -1;  // the leader's bytes never come: the MMA's wait must expire
                    } else {
                        tma_load_4d_pair(sA, &d.maps[amap][0], full_l, k0, cc, cb, aslice);
                        tma_load_4d_pair(sAl, &d.maps[amap][1], full_l, k0, cc, cb, aslice);
                        tma_load_3d_pair(sB, &d.maps[bmap][0], full_l, k0, ca, brow);
                        tma_load_3d_pair(sBl, &d.maps[bmap][1], full_l, k0, ca, brow);
                    }
                    if (++stage == nst) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {
                // let the copies in flight land: the leader sees both CTAs' bytes on
                // its own full barriers; the peer gives its own copies a fixed time
                if (leader) {
                    for (int s = 0; s < nst; s++) {
                        if (last_phase[s] < 0) continue;
                        const uint64_t t0 = gtimer();
                        while (!mbar_test(smem_u32(&bar_full[s]), (uint32_t)last_phase[s]) &&
                               gtimer() - t0 < WAIT_LIMIT_NS) {
                        }
                    }
                }
                spin_ns(1000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && leader) {
            MmaRing rg;
            rg.full0 = smem_u32(&bar_full[0]);
            rg.empty0 = smem_u32(&bar_empty[0]);
            rg.hfull0 = smem_u32(&bar_hfull[0]);
            rg.hempty0 = smem_u32(&bar_hempty[0]);
            rg.lo0 = desc_lo(sbase);
            rg.step = stage_bytes >> 4;
            rg.a16 = A_BYTES >> 4;
            rg.b16 = b_plane >> 4;
            rg.nst = nst;
            rg.stage = 0;
            rg.phase = 0;
            rg.hblk = 0;
            SegCache sc;
            seg_reset(sc);
            for (int64_t it = cid; it < wv.n_gemm; it += ncl) {
                const PairItem pw = decode_pair(wv, it, sc, rank);
                const Item &w = pw.it;
                if (w.diag) continue;
                const InstDesc &d = *sc.d;
                const int kv = d.kv, ko = d.ko, nch = 2 * kv + 2 * ko, kind = d.kind;
                const bool dh = kind == 2 && (d.dm.dp & 31) != 0, lh = kind == 2 && (d.dm.lp & 31) != 0;
                const int nvalid = min(d.brows, d.dm.v - w.n * d.brows);
                const int N = (nvalid + 15) / 16 * 16;
                const uint32_t fmt = kind == 1 ? 2u : 1u;
                const uint32_t idesc = idesc_m | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17);
                int code = 0;
                const bool good = kind == 1
                    ? mma_item<1, 2>(rg, tmem, idesc, nch, -1, -1, -1, -1, &abort_sh, &code)
                    : mma_item<2, 2>(rg, tmem, idesc, nch, dh ? kv - 1 : -1, dh ? 2 * kv - 1 : -1,
                                     lh ? 2 * kv + ko - 1 : -1, lh ? nch - 1 : -1, &abort_sh, &code);
                if (!good) {
                    fail_pair(&abort_sh, peer_abort, wv.err, code);
                    break;
                }
            }
            // every MMA issued by this thread has completed before the pair tears down
            tc_commit_pair(smem_u32(&bar_fin), (uint16_t)1);
            const uint64_t t0 = gtimer();
            while (!mbar_test(smem_u32(&bar_fin), 0u) && gtimer() - t0 < WAIT_LIMIT_NS) {
            }
        }
    } else {
        const int wq = warp & 3;
        const int half = (warp - 2) >> 2;
        const int row = wq * 32 + lane;
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        uint32_t hblk = 0;
        bool ok = true;
        SegCache &cs = ecache[warp - 2];
        if (lane == 0) seg_reset(cs);
        __syncwarp();
        for (int64_t it = cid; it < wv.n_gemm && ok; it += ncl) {
            SegCache sc = cs;
            const PairItem pw = decode_pair(wv, it, sc, rank);
            const Item &w = pw.it;
            __syncwarp();
            if (lane == 0) cs = sc;
            __syncwarp();
            if (w.diag) continue;
            const InstDesc &d = *sc.d;
            const int64_t u_seg = sc.u_off;
            const int v = d.dm.v;
            const int nhb = (num_chunks(d) + d.kb - 1) / d.kb;
            const int lb = row / d.pc, lc = row % d.pc;
            const int pass0 = w.n * d.brows, pass_end = min(v, pass0 + d.brows);
            const int N = (pass_end - pass0 + 15) / 16 * 16;
            const int wh = N > 128 ? 128 : (N > 64 ? 64 : 32);
            const int nld = wh / 32;
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
                    if (c4 < nld) {
                        uint32_t r[16], r2[16];
                        const uint32_t ta = tmem + lane_off + buf * (uint32_t)BN + (uint32_t)(half * wh + c4 * 32);
                        tc_ld16(ta, r);
                        tc_ld16(ta + 16, r2);
                        tc_wait_ld();
#pragma unroll
                        for (int j = 0; j < 16; j++) total[c4 * 32 + j] += __uint_as_float(r[j]);
#pragma unroll
                        for (int j = 0; j < 16; j++) total[c4 * 32 + 16 + j] += __uint_as_float(r2[j]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive_cluster(peer_addr(smem_u32(&bar_hempty[buf]), 0));
                hblk++;
            }
            if (!ok) {
                if (lane == 0) fail_pair(&abort_sh, peer_abort, wv.err, DERR_TIMEOUT_TMEM);
                break;
            }
            if (pw.empty) continue;
            const int b = w.bt * d.pb + lb, c = w.ct * d.pc + lc;
            if (b < v && c < v) {
                const int a0 = pass0 + half * wh;  // a multiple of 8
                float *Ut = static_cast<float *>(wv.U) + u_seg + (int64_t)w.tb * 3 * d.dm.ug;
                store_u_cubes(Ut, (v + 7) >> 3, w.g, a0, b, c, min(wh, pass_end - a0), total);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    cluster_sync_all();  // the peer no longer signals this CTA's barriers or reads its operands
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                     : "memory");
    }
}

}  // namespace

using tcx::encode;

bool tc_supported(int cc_major, int cc_minor) { return cc_major == 10 && cc_minor == 3; }

cudaError_t tc_fill_desc(InstDesc &d, int prec, const Operands &op, int pb, int kb, bool pair, std::string &err) {
    if (pb != 4 && pb != 8 && pb != 16) {
        err = "tensor-core pair tile: pb must be 4, 8 or 16";
        return cudaErrorInvalidValue;
    }
    if (kb != 2) {  // the MMA issuer works in K blocks of two chunks (mma_item)
        err = "tensor-core accumulator block: kb must be 2";
        return cudaErrorInvalidValue;
    }
    const int o = d.dm.o, v = d.dm.v, dp = d.dm.dp, lp = d.dm.lp;
    const bool tf = prec == TCORR_TF32X3;
    const uint64_t eb = tf ? 4 : 2;
    const CUtensorMapDataType dt = tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const int kch = ROW_BYTES / (int)eb;
    const int pc = BM / pb;
    d.pb = pb;
    d.pc = pc;
    d.kb = kb;
    d.kind = tf ? 1 : 2;
    d.pair = pair ? 1 : 0;
    d.nbt = (v + pb - 1) / pb;
    d.nct = (v + pc - 1) / pc;
    d.npass = (v + BN - 1) / BN;
    // pass width: <= BN, a multiple of 16 (single SM) or of 32 (SM pair: each SM
    // holds brows / 2 rows of B, a multiple of 16; the MMA's N is the pass's valid
    // width rounded to 16, the peer's half starting at N / 2, a multiple of 8)
    const int wq = pair ? 32 : 16;
    d.brows = round_up((v + d.npass - 1) / d.npass, wq);
    d.kv = (v + kch - 1) / kch;
    d.ko = (o + kch - 1) / kch;
    // bytes per stage: one CTA's (single SM), or both CTAs' (the pair's leader expects them all)
    d.stage_tx = pair ? (uint32_t)(2 * (2 * A_BYTES + 2 * (d.brows / 2) * ROW_BYTES))
                      : (uint32_t)(2 * A_BYTES + 2 * d.brows * ROW_BYTES);
    const uint64_t V = v, O = o;
    const uint32_t bk = (uint32_t)kch, bpc = (uint32_t)pc, bpb = (uint32_t)pb;
    const uint32_t brows = (uint32_t)(pair ? d.brows / 2 : d.brows);  // B box rows per CTA
    void *hi[4] = {op.G, op.T2K, op.T2R, op.AoN};
    void *lo[4] = {op.Glo, op.T2Klo, op.T2Rlo, op.AoNlo};
    for (int part = 0; part < 2; part++) {
        void *const *src = part == 0 ? hi : lo;
        {   // G natural: (d, c, b, q) with c = y index, b = x index
            uint64_t dims[4] = {V, V, V, O};
            uint64_t st[3] = {dp * eb, V * dp * eb, V * V * dp * eb};
            uint32_t box[4] = {bk, bpc, bpb, 1};
            if (!encode(&d.maps[MAP_G_NAT][part], dt, 4, src[0], dims, st, box, err, "G")) return cudaErrorInvalidValue;
        }
        {   // G swapped: (d, c, b, q) with c = x index, b = y index
            uint64_t dims[4] = {V, V, V, O};
            uint64_t st[3] = {V * dp * eb, dp * eb, V * V * dp * eb};
            uint32_t box[4] = {bk, bpc, bpb, 1};
            if (!encode(&d.maps[MAP_G_SWP][part], dt, 4, src[0], dims, st, box, err, "G swapped"))
                return cudaErrorInvalidValue;
        }
        {   // T2K natural
            uint64_t dims[4] = {O, V, V, O};
            uint64_t st[3] = {lp * eb, V * lp * eb, V * V * lp * eb};
            uint32_t box[4] = {bk, bpc, bpb, 1};
            if (!encode(&d.maps[MAP_T2K_NAT][part], dt, 4, src[1], dims, st, box, err, "T2K")) return cudaErrorInvalidValue;
        }
        {   // T2K swapped
            uint64_t dims[4] = {O, V, V, O};
            uint64_t st[3] = {V * lp * eb, lp * eb, V * V * lp * eb};
            uint32_t box[4] = {bk, bpc, bpb, 1};
            if (!encode(&d.maps[MAP_T2K_SWP][part], dt, 4, src[1], dims, st, box, err, "T2K swapped"))
                return cudaErrorInvalidValue;
        }
        {   // T2R: (d, a, s*o+p)
            uint64_t dims[3] = {V, V, O * O};
            uint64_t st[2] = {dp * eb, V * dp * eb};
            uint32_t box[3] = {bk, brows, 1};
            if (!encode(&d.maps[MAP_T2R][part], dt, 3, src[2], dims, st, box, err, "T2R")) return cudaErrorInvalidValue;
        }
        {   // AoN: (l, a, q*o+s)
            uint64_t dims[3] = {O, V, O * O};
            uint64_t st[2] = {lp * eb, V * lp * eb};
            uint32_t box[3] = {bk, brows, 1};
            if (!encode(&d.maps[MAP_AON][part], dt, 3, src[3], dims, st, box, err, "AoN")) return cudaErrorInvalidValue;
        }
    }
    return cudaSuccess;
}

int64_t tc_units_per_task(const InstDesc &d) {
    const int64_t tiles = (int64_t)d.nbt * d.nct;
    return (int64_t)3 * (d.pair ? (tiles + 1) / 2 : tiles) * d.npass;
}

cudaError_t tc_prepare(int) {
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lk(mu);
    if (done) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(ugemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ugemm_tc_pair_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
    if (e == cudaSuccess) done = true;
    return e;
}

// Co-resident 2-CTA clusters of the pair kernel on the current device (one
// per SM pair that the cluster scheduler can place), queried once per device.
static int pair_clusters(int sm_count) {
    static std::mutex mu;
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return sm_count / 2;
    std::lock_guard<std::mutex> lk(mu);
    if (cache[dev] > 0) return cache[dev];
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(sm_count / 2 * 2), 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, ugemm_tc_pair_kernel, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = sm_count / 2;
    }
    cache[dev] = std::min(n, sm_count / 2);
    return cache[dev];
}

cudaError_t launch_ugemm_tc(int prec, int sm_count, const Wave &w, cudaStream_t st, bool pair) {
    if (w.n_gemm <= 0) return cudaSuccess;
    if (w.tc_brows < 16 || w.tc_brows > BN || w.tc_brows % (pair ? 32 : 16) != 0) return cudaErrorInvalidValue;
    cudaError_t e = tc_prepare(prec);
    if (e != cudaSuccess) return e;
    if (!pair) {
        const int grid = (int)std::min<int64_t>(sm_count, w.n_gemm);
        ugemm_tc_kernel<<<grid, TC_THREADS, SMEM_BYTES, st>>>(w);
        return cudaGetLastError();
    }
    const int ncl = (int)std::min<int64_t>(pair_clusters(sm_count), w.n_gemm);
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * ncl), 1, 1);
    cfg.blockDim = dim3(TC_THREADS, 1, 1);
    cfg.dynamicSmemBytes = SMEM_BYTES;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, ugemm_tc_pair_kernel, w);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace tcorr
