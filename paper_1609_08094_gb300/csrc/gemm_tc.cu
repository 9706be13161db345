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
template <int KIND>
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

    const int kch = ROW_BYTES / (KIND == 1 ? 4 : 2);
    // instruction descriptor: D = F32, A/B = TF32 (2) or BF16 (1), K-major, M = 128
    constexpr uint32_t fmt = KIND == 1 ? 2u : 1u;
    constexpr uint32_t idesc_base = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(BM >> 4) << 24);

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
            int stage = 0;
            uint32_t phase = 0;
            uint32_t hblk = 0;  // K blocks issued so far: buffer hblk & 1, phase (hblk >> 1) & 1
            bool ok = true;
            SegCache sc;
            seg_reset(sc);
            for (int64_t it = blockIdx.x; it < wv.n_gemm && ok; it += gridDim.x) {
                const Item w = decode(wv, it, sc);
                if (w.diag) continue;
                const InstDesc &d = *sc.d;
                // per-item constants in registers: the issue loop reads no memory
                const int kv = d.kv, ko = d.ko, dp = d.dm.dp, lp = d.dm.lp;
                const int nch = 2 * kv + 2 * ko, kb = d.kb;
                const int nvalid = min(d.brows, d.dm.v - w.n * d.brows);
                const int N = (nvalid + 15) / 16 * 16;
                const uint32_t idesc = idesc_base | ((uint32_t)(N >> 3) << 17);
                // K blocks of kb chunks: the small hi*lo and lo*hi products of each
                // chunk are issued as its data lands, the dominant hi*hi products of
                // the whole block last, so that the truncation of every instruction
                // acts on the smallest possible accumulator; the block's stages are
                // released together once its last MMA is issued.
                for (int c0 = 0; c0 < nch && ok; c0 += kb) {
                    const int nb = min(kb, nch - c0);
                    const uint32_t buf = hblk & 1u;
                    int st0 = stage;
                    for (int cb = 0; cb < nb; cb++) {
                        if (!mbar_wait(smem_u32(&bar_full[stage]), phase, &abort_sh)) {
                            fail(&abort_sh, wv.err, DERR_TIMEOUT_FULL);
                            ok = false;
                            break;
                        }
                        if (cb == 0 &&
                            !mbar_wait(smem_u32(&bar_hempty[buf]), ((hblk >> 1) & 1u) ^ 1u, &abort_sh)) {
                            fail(&abort_sh, wv.err, DERR_TIMEOUT_TMEM);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t dt = tmem + buf * (uint32_t)BN;
                        const uint32_t sA = sbase + stage * stage_bytes, sAl = sA + A_BYTES;
                        const uint32_t sB = sAl + A_BYTES, sBl = sB + b_plane;
                        const int nks = chunk_ksteps<KIND>(kv, ko, dp, lp, c0 + cb);
                        for (int kk = 0; kk < nks; kk++) {
                            const uint32_t off = kk * 32;
                            tc_mma<KIND>(dt, sdesc(sA + off), sdesc(sBl + off), idesc,
                                         (cb > 0 || kk > 0) ? 1u : 0u);
                            tc_mma<KIND>(dt, sdesc(sAl + off), sdesc(sB + off), idesc, 1u);
                        }
                        if (++stage == nst) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    const uint32_t dt = tmem + buf * (uint32_t)BN;
                    // each stage is released (commit: arrives once every MMA issued
                    // so far has completed) right after its last product is issued
                    int sj = st0;
                    for (int cb = 0; cb < nb; cb++) {
                        const uint32_t sA = sbase + sj * stage_bytes, sB = sA + 2 * A_BYTES;
                        const int nks = chunk_ksteps<KIND>(kv, ko, dp, lp, c0 + cb);
                        for (int kk = 0; kk < nks; kk++) {
                            const uint32_t off = kk * 32;
                            tc_mma<KIND>(dt, sdesc(sA + off), sdesc(sB + off), idesc, 1u);
                        }
                        tc_commit(smem_u32(&bar_empty[sj]));
                        if (++sj == nst) sj = 0;
                    }
                    tc_commit(smem_u32(&bar_hfull[buf]));
                    hblk++;
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
            const int v = d.dm.v, vc = d.dm.vc;
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
            // rows of 16 consecutive c per half warp: group 0 and 2 in their own
            // [a][b][c] order, group 1 at [b][a][c] (aligned with W, see tcorr_internal.cuh)
            const int b = w.bt * d.pb + lb, c = w.ct * d.pc + lc;
            if (b < v && c < v) {
                const int a0 = pass0 + half * wh;
                const int64_t stride = w.g == 1 ? (int64_t)vc : (int64_t)v * vc;
                const int64_t base = w.g == 1 ? (int64_t)b * v * vc + c : (int64_t)b * vc + c;
                const int64_t u_off = u_seg + (int64_t)(w.tb * 3 + w.g) * v * v * vc;
                float *Ug = static_cast<float *>(wv.U) + u_off + base + (int64_t)a0 * stride;
                const int na = min(wh, pass_end - a0);
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

}  // namespace

using tcx::encode;

bool tc_supported(int cc_major, int cc_minor) { return cc_major == 10 && cc_minor == 3; }

cudaError_t tc_fill_desc(InstDesc &d, int prec, const Operands &op, int pb, int kb, std::string &err) {
    if (pb != 4 && pb != 8 && pb != 16) {
        err = "tensor-core pair tile: pb must be 4, 8 or 16";
        return cudaErrorInvalidValue;
    }
    if (kb < 1 || kb > 3) {  // a K block holds its stages until its last MMA (>= 4 stages)
        err = "tensor-core accumulator block: kb must be 1 .. 3";
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
    d.nbt = (v + pb - 1) / pb;
    d.nct = (v + pc - 1) / pc;
    d.npass = (v + BN - 1) / BN;
    d.brows = round_up((v + d.npass - 1) / d.npass, 16);  // pass width: <= BN
    d.kv = (v + kch - 1) / kch;
    d.ko = (o + kch - 1) / kch;
    d.stage_tx = (uint32_t)(2 * A_BYTES + 2 * d.brows * ROW_BYTES);
    const uint64_t V = v, O = o;
    const uint32_t bk = (uint32_t)kch, bpc = (uint32_t)pc, bpb = (uint32_t)pb, brows = (uint32_t)d.brows;
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

int64_t tc_units_per_task(const InstDesc &d) { return (int64_t)3 * d.nbt * d.nct * d.npass; }

cudaError_t tc_prepare(int prec) {
    static std::mutex mu;
    static bool done[2] = {false, false};
    std::lock_guard<std::mutex> lk(mu);
    const int t = prec == TCORR_TF32X3 ? 0 : 1;
    if (done[t]) return cudaSuccess;
    const cudaError_t e = t == 0 ? cudaFuncSetAttribute(ugemm_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        SMEM_BYTES)
                                 : cudaFuncSetAttribute(ugemm_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        SMEM_BYTES);
    if (e == cudaSuccess) done[t] = true;
    return e;
}

cudaError_t launch_ugemm_tc(int prec, int sm_count, const Wave &w, cudaStream_t st) {
    const int grid = (int)std::min<int64_t>(sm_count, w.n_gemm);
    if (grid <= 0) return cudaSuccess;
    if (w.tc_brows < 16 || w.tc_brows > BN || w.tc_brows % 16 != 0) return cudaErrorInvalidValue;
    const cudaError_t e = tc_prepare(prec);
    if (e != cudaSuccess) return e;
    if (prec == TCORR_TF32X3) ugemm_tc_kernel<1><<<grid, TC_THREADS, SMEM_BYTES, st>>>(w);
    else ugemm_tc_kernel<2><<<grid, TC_THREADS, SMEM_BYTES, st>>>(w);
    return cudaGetLastError();
}

}  // namespace tcorr
