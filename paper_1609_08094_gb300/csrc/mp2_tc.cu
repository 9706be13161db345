// RI-MP2 correlation energy in mixed precision on the tcgen05 tensor cores:
// the paper's mixed-precision variant of the RI-MP2 kernel (Sec. 2.1, with
// the dgemm of the integral assembly done in reduced precision, Sec. 3),
// re-designed with the split-precision scheme of the (T) contractions.
//
//   E_MP2 = - sum_{ij} sum_{ab} g_aibj (2 g_aibj - g_ajbi) / (e_a + e_b - e_i - e_j),
//   g_aibj = sum_gamma C^gamma_ai C^gamma_bj          (Eqs. mp2_energy, eri_sym_decomp)
//
// over the occupied pairs i <= j (Eq. tasks_rimp2; i < j counts twice).  A
// work item is (pair, tile pair A <= B of 128 virtual indices).  Per 64-byte K
// chunk the producer loads C_i[A], C_j[B], C_j[A], C_i[B] (hi and lo planes
// of the K-major C^T, rows past v are TMA zero fill); the MMA thread forms
// G = C_i[A] C_j[B]^T (= g on A x B) and H = C_j[A] C_i[B]^T (= g on B x A,
// transposed) in two M = N = 128 TMEM accumulators with all four products
// lo*lo + hi*lo + lo*hi + hi*hi of each operand pair, each K block of MP_KB
// chunks in a fresh, double-buffered accumulator (smallest products first,
// hi*hi last, as in the (T) kernel: the tensor core's truncating accumulation
// then acts on the smallest partial sums).  Unlike the (T) contractions the
// lo*lo product is kept: for i = j the same-index elements g_aa are sums of
// squares, where the dropped lo^2 would bias g one-signedly by the mean
// square of the split's relative residual (~3e-6 with BF16; those elements
// carry most of E for small o); the kernel is bound by operand ingest, so
// the fourth product costs no time.  The epilogue warps fold every block into register totals
// with round-to-nearest FP32 adds, and at the end of the item form the energy
// terms of their (a, b): over A x B and B x A together -2 (g^2 + h^2) / eps and
// 2 g h / eps; a diagonal tile pair covers its block once, -2 g^2 / eps and
// g h / eps.  g never reaches memory.  Denominators and the item's terms are
// FP32, the running sums FP64; one FP64 partial pair per CTA, summed by the
// FP64 path's deterministic Kahan kernel.
//
// Kernel structure: one persistent CTA per SM, 10 warps.  Warp 0: TMA
// producer, a ring of 3 stages of 8 planes of 128 rows x 64 bytes (64 KB).
// Warp 1: TMEM allocation (512 columns: G and H of two K blocks) and the MMA
// issue.  Warps 2-9: two per TMEM lane quarter, 64 columns of G and of H
// each.  Every mbarrier wait is bounded (wall clock): on expiry the kernel
// sets an error flag, stops all roles, waits (bounded) for its own copies in
// flight, frees TMEM and returns; the host reports TCORR_ETIMEOUT.
#include <mutex>

#include "tc_common.cuh"

namespace tcorr {
namespace {

using namespace tcx;

constexpr int MP_BM = MP2_TC_TILE;          // virtual indices per tile: M = N = 128
constexpr int MP_ROW = 64;                  // K bytes per shared-memory row (SWIZZLE_64B span)
constexpr int MP_TILE = MP_BM * MP_ROW;     // 8 KB: one plane of one operand tile
constexpr int MP_STAGE = 8 * MP_TILE;       // C_i[A], C_j[B], C_j[A], C_i[B] x (hi, lo)
constexpr int MP_STAGES = 3;
constexpr int MP_SMEM = MP_STAGES * MP_STAGE + 1024;
constexpr int MP_THREADS = 320;
constexpr int MP_EPI = 256;                 // warps 2-9
constexpr int MP_KB = 2;                    // K chunks per TMEM accumulator block
constexpr int MP_HALF = MP_BM / 2;          // columns of G (and of H) per epilogue warp
static_assert(MP_KB < MP_STAGES, "a K block holds its stages until its last MMA is issued");
static_assert(4 * MP_BM <= 512, "G and H of two K blocks fill the 512 TMEM columns");
static_assert(MP_TILE % 1024 == 0, "planes keep the 64-byte swizzle pattern aligned");
// stage plane order
enum { P_AI_HI = 0, P_AI_LO, P_BJ_HI, P_BJ_LO, P_AJ_HI, P_AJ_LO, P_BI_HI, P_BI_LO };

template <int KIND>
__global__ void __launch_bounds__(MP_THREADS, 1) mp2_tc_kernel(const __grid_constant__ Mp2TcArgs a) {
    extern __shared__ __align__(1024) uint8_t smem_dyn[];
    __shared__ __align__(8) uint64_t bar_full[MP_STAGES], bar_empty[MP_STAGES];
    __shared__ __align__(8) uint64_t bar_hfull[2], bar_hempty[2];
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_sh;
    __shared__ double red[MP_EPI / 32][2];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_dyn) + 1023u) & ~1023u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < MP_STAGES; s++) {
            mbar_init(smem_u32(&bar_full[s]), 1);
            mbar_init(smem_u32(&bar_empty[s]), 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(smem_u32(&bar_hfull[b]), 1);
            mbar_init(smem_u32(&bar_hempty[b]), MP_EPI);
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

    const int kch = MP_ROW / (KIND == 1 ? 4 : 2);  // K elements per chunk
    const int nch = a.nch;
    // D = F32, A/B = TF32 (2) or BF16 (1), K-major, M = N = 128
    constexpr uint32_t fmt = KIND == 1 ? 2u : 1u;
    constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(MP_BM >> 3) << 17) |
                               ((uint32_t)(MP_BM >> 4) << 24);
    double ej = 0.0, ek = 0.0;  // epilogue threads: weighted Coulomb and exchange sums

    if (warp == 0) {
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[MP_STAGES];
            for (int s = 0; s < MP_STAGES; s++) last_phase[s] = -1;
            bool ok = true;
            for (int64_t it = blockIdx.x; it < a.items && ok; it += gridDim.x) {
                const int pr = (int)(it / a.ntp), tp = (int)(it % a.ntp);
                const int i = a.pairs[2 * pr], j = a.pairs[2 * pr + 1];
                const int A0 = a.tiles[2 * tp] * MP_BM, B0 = a.tiles[2 * tp + 1] * MP_BM;
                for (int ch = 0; ch < nch; ch++) {
                    if (!mbar_wait(smem_u32(&bar_empty[stage]), phase ^ 1u, &abort_sh)) {
                        fail(&abort_sh, a.err, DERR_TIMEOUT_EMPTY);
                        ok = false;
                        break;
                    }
                    const uint32_t full = smem_u32(&bar_full[stage]);
                    mbar_expect_tx(full, (uint32_t)MP_STAGE);
                    last_phase[stage] = (int)phase;
                    const uint32_t s = sbase + stage * MP_STAGE;
                    const int k0 = ch * kch;
                    tma_load_3d(s + P_AI_HI * MP_TILE, &a.map[0], full, k0, A0, i);
                    tma_load_3d(s + P_AI_LO * MP_TILE, &a.map[1], full, k0, A0, i);
                    tma_load_3d(s + P_BJ_HI * MP_TILE, &a.map[0], full, k0, B0, j);
                    tma_load_3d(s + P_BJ_LO * MP_TILE, &a.map[1], full, k0, B0, j);
                    tma_load_3d(s + P_AJ_HI * MP_TILE, &a.map[0], full, k0, A0, j);
                    tma_load_3d(s + P_AJ_LO * MP_TILE, &a.map[1], full, k0, A0, j);
                    tma_load_3d(s + P_BI_HI * MP_TILE, &a.map[0], full, k0, B0, i);
                    tma_load_3d(s + P_BI_LO * MP_TILE, &a.map[1], full, k0, B0, i);
                    if (++stage == MP_STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            if (!ok) {  // let this CTA's copies in flight land before exiting
                for (int s = 0; s < MP_STAGES; s++) {
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
            for (int64_t it = blockIdx.x; it < a.items && ok; it += gridDim.x) {
                for (int c0 = 0; c0 < nch && ok; c0 += MP_KB) {
                    const int nb = min(MP_KB, nch - c0);
                    const uint32_t buf = hblk & 1u;
                    const uint32_t dG = tmem + buf * (uint32_t)(2 * MP_BM), dH = dG + (uint32_t)MP_BM;
                    const int st0 = stage;
                    for (int cb = 0; cb < nb; cb++) {
                        if (!mbar_wait(smem_u32(&bar_full[stage]), phase, &abort_sh)) {
                            fail(&abort_sh, a.err, DERR_TIMEOUT_FULL);
                            ok = false;
                            break;
                        }
                        if (cb == 0 &&
                            !mbar_wait(smem_u32(&bar_hempty[buf]), ((hblk >> 1) & 1u) ^ 1u, &abort_sh)) {
                            fail(&abort_sh, a.err, DERR_TIMEOUT_TMEM);
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        // descriptor low words of the stage's planes (see mma_lo): one K
                        // step of 32 bytes is +2; the block's first products zero D
                        const uint32_t s = desc_lo(sbase + stage * MP_STAGE);
                        const uint32_t ai = s + P_AI_HI * (MP_TILE >> 4), bj = s + P_BJ_HI * (MP_TILE >> 4);
                        const uint32_t aj = s + P_AJ_HI * (MP_TILE >> 4), bi = s + P_BI_HI * (MP_TILE >> 4);
                        constexpr uint32_t LO = MP_TILE >> 4;  // hi plane -> lo plane
                        if (cb == 0) mma_lo<KIND, 1, false>(dG, ai + LO, bj + LO, idesc);
                        else mma_lo<KIND, 1, true>(dG, ai + LO, bj + LO, idesc);
                        mma_lo<KIND, 1, true>(dG, ai, bj + LO, idesc);
                        mma_lo<KIND, 1, true>(dG, ai + LO, bj, idesc);
                        if (cb == 0) mma_lo<KIND, 1, false>(dH, aj + LO, bi + LO, idesc);
                        else mma_lo<KIND, 1, true>(dH, aj + LO, bi + LO, idesc);
                        mma_lo<KIND, 1, true>(dH, aj, bi + LO, idesc);
                        mma_lo<KIND, 1, true>(dH, aj + LO, bi, idesc);
                        mma_lo<KIND, 1, true>(dG, ai + LO + 2, bj + LO + 2, idesc);
                        mma_lo<KIND, 1, true>(dG, ai + 2, bj + LO + 2, idesc);
                        mma_lo<KIND, 1, true>(dG, ai + LO + 2, bj + 2, idesc);
                        mma_lo<KIND, 1, true>(dH, aj + LO + 2, bi + LO + 2, idesc);
                        mma_lo<KIND, 1, true>(dH, aj + 2, bi + LO + 2, idesc);
                        mma_lo<KIND, 1, true>(dH, aj + LO + 2, bi + 2, idesc);
                        if (++stage == MP_STAGES) { stage = 0; phase ^= 1u; }
                    }
                    if (!ok) break;
                    // the dominant hi*hi products of the block last; each stage is
                    // released (commit: arrives once every MMA issued so far has
                    // completed) right after its last product is issued
                    int sj = st0;
                    for (int cb = 0; cb < nb; cb++) {
                        const uint32_t s = desc_lo(sbase + sj * MP_STAGE);
                        const uint32_t ai = s + P_AI_HI * (MP_TILE >> 4), bj = s + P_BJ_HI * (MP_TILE >> 4);
                        const uint32_t aj = s + P_AJ_HI * (MP_TILE >> 4), bi = s + P_BI_HI * (MP_TILE >> 4);
                        mma_lo<KIND, 1, true>(dG, ai, bj, idesc);
                        mma_lo<KIND, 1, true>(dH, aj, bi, idesc);
                        mma_lo<KIND, 1, true>(dG, ai + 2, bj + 2, idesc);
                        mma_lo<KIND, 1, true>(dH, aj + 2, bi + 2, idesc);
                        tc_commit(smem_u32(&bar_empty[sj]));
                        if (++sj == MP_STAGES) sj = 0;
                    }
                    tc_commit(smem_u32(&bar_hfull[buf]));
                    hblk++;
                }
            }
        }
    } else {
        const int wq = warp & 3;              // TMEM lane quarter of this warp
        const int half = (warp - 2) >> 2;     // column half of G and of H
        const int row = wq * 32 + lane;       // accumulator row = a in tile A
        const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
        const int nhb = (nch + MP_KB - 1) / MP_KB;
        const int v = a.v;
        uint32_t hblk = 0;
        bool ok = true;
        for (int64_t it = blockIdx.x; it < a.items && ok; it += gridDim.x) {
            const int pr = (int)(it / a.ntp), tp = (int)(it % a.ntp);
            const int i = a.pairs[2 * pr], j = a.pairs[2 * pr + 1];
            const int A0 = a.tiles[2 * tp] * MP_BM, B0 = a.tiles[2 * tp + 1] * MP_BM;
            float tg[MP_HALF], th[MP_HALF];
#pragma unroll
            for (int c = 0; c < MP_HALF; c++) tg[c] = th[c] = 0.f;
            for (int hb = 0; hb < nhb; hb++) {
                const uint32_t buf = hblk & 1u;
                int good = 1;
                if (lane == 0) good = mbar_wait(smem_u32(&bar_hfull[buf]), (hblk >> 1) & 1u, &abort_sh) ? 1 : 0;
                good = __shfl_sync(0xffffffffu, good, 0);
                __syncwarp();
                if (!good) { ok = false; break; }
                tc_fence_after();
                const uint32_t tg0 = tmem + lane_off + buf * (uint32_t)(2 * MP_BM) + (uint32_t)(half * MP_HALF);
#pragma unroll
                for (int c16 = 0; c16 < MP_HALF / 16; c16++) {
                    uint32_t r[16], r2[16];
                    tc_ld16(tg0 + (uint32_t)(c16 * 16), r);
                    tc_ld16(tg0 + (uint32_t)(MP_BM + c16 * 16), r2);
                    tc_wait_ld();
#pragma unroll
                    for (int x = 0; x < 16; x++) tg[c16 * 16 + x] += __uint_as_float(r[x]);
#pragma unroll
                    for (int x = 0; x < 16; x++) th[c16 * 16 + x] += __uint_as_float(r2[x]);
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&bar_hempty[buf]));
                hblk++;
            }
            if (!ok) {
                if (lane == 0) fail(&abort_sh, a.err, DERR_TIMEOUT_TMEM);
                break;
            }
            // energy terms of this thread's row a and 64 columns b
            const int ar = A0 + row;
            if (ar < v) {
                const float ea = (float)(a.eps_v[ar] - (a.eps_o[i] + a.eps_o[j]));
                const bool dg = (A0 == B0);
                const int b0 = B0 + half * MP_HALF;
                float sj = 0.f, sk = 0.f;
#pragma unroll
                for (int x = 0; x < MP_HALF; x++) {
                    if (b0 + x < v) {  // b grows with x
                        const float rd = 1.0f / (ea + a.eps_vf[b0 + x]);
                        const float g = tg[x], h = th[x];
                        if (!dg) {
                            sj = fmaf(-2.f * (g * g + h * h), rd, sj);
                            sk = fmaf(2.f * g * h, rd, sk);
                        } else {
                            sj = fmaf(-2.f * g * g, rd, sj);
                            sk = fmaf(g * h, rd, sk);
                        }
                    }
                }
                const double w = (i == j) ? 1.0 : 2.0;  // the pair (j, i) has the same energy
                ej += w * (double)sj;
                ek += w * (double)sk;
            }
        }
        for (int off = 16; off > 0; off >>= 1) {
            ej += __shfl_xor_sync(0xffffffffu, ej, off);
            ek += __shfl_xor_sync(0xffffffffu, ek, off);
        }
        if (lane == 0) { red[warp - 2][0] = ej; red[warp - 2][1] = ek; }
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {  // fixed order: the CTA's partial is deterministic
        double sj = 0.0, sk = 0.0;
        for (int w = 0; w < MP_EPI / 32; w++) { sj += red[w][0]; sk += red[w][1]; }
        a.partials[2 * blockIdx.x] = sj;
        a.partials[2 * blockIdx.x + 1] = sk;
    }
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                     : "memory");
    }
}

}  // namespace

using tcx::encode;

cudaError_t mp2_tc_fill(Mp2TcArgs &a, int prec, void *hi, void *lo, int o, int v, int kp, std::string &err) {
    const bool tf = prec == TCORR_TF32X3;
    const uint64_t eb = tf ? 4 : 2;
    const int kch = MP_ROW / (int)eb;
    if (kp % kch != 0) {
        err = "RI-MP2 tensor-core path: K extent not a multiple of the chunk";
        return cudaErrorInvalidValue;
    }
    const CUtensorMapDataType dt = tf ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    // Ct[i][a][gamma]: (gamma, a, i), rows past v read as zeros
    uint64_t dims[3] = {(uint64_t)kp, (uint64_t)v, (uint64_t)o};
    uint64_t st[2] = {(uint64_t)kp * eb, (uint64_t)v * kp * eb};
    uint32_t box[3] = {(uint32_t)kch, (uint32_t)MP_BM, 1};
    if (!encode(&a.map[0], dt, 3, hi, dims, st, box, err, "C hi")) return cudaErrorInvalidValue;
    if (!encode(&a.map[1], dt, 3, lo, dims, st, box, err, "C lo")) return cudaErrorInvalidValue;
    a.nch = kp / kch;
    return cudaSuccess;
}

cudaError_t launch_mp2_tc(int prec, int sm_count, const Mp2TcArgs &a, cudaStream_t st) {
    static std::mutex mu;
    static bool done[2] = {false, false};
    const int t = prec == TCORR_TF32X3 ? 0 : 1;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!done[t]) {
            const cudaError_t e =
                t == 0 ? cudaFuncSetAttribute(mp2_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, MP_SMEM)
                       : cudaFuncSetAttribute(mp2_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, MP_SMEM);
            if (e != cudaSuccess) return e;
            done[t] = true;
        }
    }
    const int grid = (int)std::min<int64_t>(sm_count, a.items);
    if (grid <= 0) return cudaSuccess;
    if (t == 0) mp2_tc_kernel<1><<<grid, MP_THREADS, MP_SMEM, st>>>(a);
    else mp2_tc_kernel<2><<<grid, MP_THREADS, MP_SMEM, st>>>(a);
    return cudaGetLastError();
}

}  // namespace tcorr
