// Device helpers shared by the tcgen05 kernels (W contractions in split
// precision and in FP64 emulation): bounded mbarrier waits, TMA loads, tcgen05
// MMA / commit / TMEM loads, shared-memory matrix descriptors, the work-item
// decode of a wave, and host-side tensor-map encoding.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <string>

#include "tcorr_internal.cuh"

namespace tcorr {
namespace tcx {

constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s of wall time per wait ...
constexpr uint32_t WAIT_MIN_POLLS = 1u << 18;      // ... and at least this many polls, so that time
                                                   // spent off the GPU (pre-emption) never counts

enum { MAP_G_NAT = 0, MAP_G_SWP, MAP_T2K_NAT, MAP_T2K_SWP, MAP_T2R, MAP_AON, NMAP };
static_assert(NMAP == 6, "InstDesc::maps holds six operand maps");

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
static __device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
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
// 16 consecutive accumulator columns of this warp's 32 TMEM lanes (the
// caller waits with tc_wait_ld before reading r)
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

struct SegCache {
    int si;                    // cached segment (-1: none)
    int64_t begin, end;        // its item range
    const InstDesc *d;
    int64_t task0, u_off;
    int npass, nct, nbt;
    int tcached;               // task (index in the segment) whose indices are cached
    int ti, tj, tk;
};
__device__ __forceinline__ void seg_reset(SegCache &c) {
    c.si = -1;
    c.tcached = -1;
}
__device__ __forceinline__ void seg_update(const Wave &w, int64_t it, SegCache &c) {
    if (c.si >= 0 && it < c.end) return;
    int lo = c.si < 0 ? 0 : c.si, hi = w.nseg - 1;  // items only grow: search forward
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (w.segs[mid].gemm0 <= it) lo = mid; else hi = mid - 1;
    }
    const Seg &sg = w.segs[lo];
    c.si = lo;
    c.begin = sg.gemm0;
    c.end = lo + 1 < w.nseg ? w.segs[lo + 1].gemm0 : w.n_gemm;
    c.d = w.descs + sg.inst;
    c.task0 = sg.task0;
    c.u_off = sg.u_off;
    c.npass = c.d->npass;
    c.nct = c.d->nct;
    c.nbt = c.d->nbt;
    c.tcached = -1;
}
struct Item {
    int tb, g, bt, ct, n;
    int s, p, q;     // (s; p, q) of the group
    bool diag;       // i = j = k: no work
};
__device__ __forceinline__ Item decode(const Wave &w, int64_t it, SegCache &c) {
    seg_update(w, it, c);
    Item r;
    int64_t x = it - c.begin;
    // order within a task: N pass fastest, then group, then pair tile, so the
    // items running at the same time read each operand tile of a slice from
    // L2 for both groups that use it (each slice of a task is read by two of
    // its three groups) and for both N passes
    r.n = (int)(x % c.npass);
    x /= c.npass;
    r.g = (int)(x % 3);
    x /= 3;
    r.ct = (int)(x % c.nct);
    x /= c.nct;
    r.bt = (int)(x % c.nbt);
    r.tb = (int)(x / c.nbt);
    if (r.tb != c.tcached) {
        const int *tk = c.d->tasks + 3 * (c.task0 + r.tb);
        c.ti = tk[0];
        c.tj = tk[1];
        c.tk = tk[2];
        c.tcached = r.tb;
    }
    const int i = c.ti, j = c.tj, k = c.tk;
    r.diag = (i == j && j == k);
    if (r.g == 0) { r.s = i; r.p = j; r.q = k; }
    else if (r.g == 1) { r.s = j; r.p = i; r.q = k; }
    else { r.s = k; r.p = i; r.q = j; }
    return r;
}
__device__ __forceinline__ int num_chunks(const InstDesc &d) { return 2 * d.kv + 2 * d.ko; }
// K steps of chunk ch that carry data: the K extent of each segment is padded
// only to 16, so the last BF16 chunk of a segment may hold a single K step
// (the rest of its 64-byte rows is TMA zero fill); a TF32 chunk (16 elements)
// is always all data.  kind: 1 = TF32, 2 = BF16; kv, ko: chunks of the d and l
// segments; dp, lp: their padded extents.
__device__ __forceinline__ int chunk_ksteps(int kind, int kv, int ko, int dp, int lp, int ch) {
    if (kind == 1) return 2;
    int kk, kext;
    if (ch < 2 * kv) { kk = ch < kv ? ch : ch - kv; kext = dp; }
    else { kk = ch - 2 * kv; kk = kk < ko ? kk : kk - ko; kext = lp; }
    return kext - kk * 32 >= 32 ? 2 : 1;
}

// ---- SM pairs (thread-block clusters of 2 CTAs, tcgen05 cta_group::2) -----
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// shared::cluster address of the variable at shared::cta address a in CTA rank
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// arrive on an mbarrier of either CTA of the cluster (shared::cluster
// address).  Default (CTA-scope release) semantics: the hand-offs it signals
// are tensor-memory reads, ordered by tcgen05 fences around the barrier; a
// cluster-scope release would also wait for this thread's earlier global
// stores (the U rows), which the other CTA never reads.
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cl) {
    asm volatile("mbarrier.arrive.shared::cluster.b64 _, [%0];" ::"r"(bar_cl) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t addr_cl, uint32_t v) {
    asm volatile("st.relaxed.cluster.shared::cluster.u32 [%0], %1;" ::"r"(addr_cl), "r"(v) : "memory");
}
// TMA loads into this CTA's shared memory whose completion is signalled on an
// mbarrier of either CTA of the pair (bar_cl: shared::cluster address)
__device__ __forceinline__ void tma_load_4d_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar_cl,
                                                 int c0, int c1, int c2, int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%3, %4, %5, %6}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar_cl), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}
__device__ __forceinline__ void tma_load_3d_pair(uint32_t dst, const CUtensorMap *map, uint32_t bar_cl,
                                                 int c0, int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cta.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar_cl), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
// tcgen05.mma over the SM pair (M = 256: A rows 0-127 from this CTA's shared
// memory, 128-255 from the peer's at the same offsets; B's N columns split in
// halves the same way; each CTA's tensor memory receives its own 128 rows)
template <int KIND>
__device__ __forceinline__ void tc_mma_pair(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (KIND == 1) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
}
// arrives once on the mbarrier at shared::cta offset bar in every CTA of
// cta_mask when every pair MMA issued so far by this thread has completed
__device__ __forceinline__ void tc_commit_pair(uint32_t bar, uint16_t cta_mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            bar),
        "h"(cta_mask)
        : "memory");
}

// ---- lean MMA issue ---------------------------------------------------------
// One thread issues every MMA of a CTA (or of an SM pair), and between two
// MMAs it runs a few dependent instructions of its own, each several clocks
// long: at M = 128, N = 256, K = 16 an MMA is ~128 tensor clocks, so the
// issue path has to stay near ten instructions per MMA.  Descriptors are
// therefore kept as their low 32-bit word (start address >> 4 and the LBO
// field; one K step of 32 bytes is +2), paired with a constant high word in
// the asm, and the accumulate flag is a compile-time constant.
constexpr uint32_t DESC_LO_FLAGS = 1u << 16;                 // LBO = 1 (unused for swizzled K-major tiles)
constexpr uint32_t DESC_HI = 32u | (1u << 14) | (4u << 29);  // SBO = 512 bytes, bit 46, 64-byte swizzle
static_assert(((uint64_t)DESC_HI << 32 | DESC_LO_FLAGS) == (((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
                                                             ((uint64_t)1 << 46) | ((uint64_t)4 << 61)),
              "same descriptor fields as sdesc");
__device__ __forceinline__ uint32_t desc_lo(uint32_t addr) { return ((addr & 0x3FFFFu) >> 4) | DESC_LO_FLAGS; }

#define TCX_MMA_ASM(CGS, KINDS, PRED)                                                             \
    asm volatile("{\n\t.reg .b64 da, db;\n\t.reg .pred p;\n\t"                                  \
                 "mov.b64 da, {%1, %4};\n\tmov.b64 db, {%2, %4};\n\t" PRED                      \
                 "tcgen05.mma.cta_group::" CGS ".kind::" KINDS " [%0], da, db, %3, p;\n\t}\n" ::"r"(d), \
                 "r"(a_lo), "r"(b_lo), "r"(idesc), "r"(DESC_HI))
template <int KIND, int CG, bool ACC>
__device__ __forceinline__ void mma_lo(uint32_t d, uint32_t a_lo, uint32_t b_lo, uint32_t idesc) {
    if constexpr (CG == 1 && KIND == 1 && ACC) TCX_MMA_ASM("1", "tf32", "setp.eq.u32 p, 0, 0;\n\t");
    else if constexpr (CG == 1 && KIND == 1) TCX_MMA_ASM("1", "tf32", "setp.ne.u32 p, 0, 0;\n\t");
    else if constexpr (CG == 1 && ACC) TCX_MMA_ASM("1", "f16", "setp.eq.u32 p, 0, 0;\n\t");
    else if constexpr (CG == 1) TCX_MMA_ASM("1", "f16", "setp.ne.u32 p, 0, 0;\n\t");
    else if constexpr (KIND == 1 && ACC) TCX_MMA_ASM("2", "tf32", "setp.eq.u32 p, 0, 0;\n\t");
    else if constexpr (KIND == 1) TCX_MMA_ASM("2", "tf32", "setp.ne.u32 p, 0, 0;\n\t");
    else if constexpr (ACC) TCX_MMA_ASM("2", "f16", "setp.eq.u32 p, 0, 0;\n\t");
    else TCX_MMA_ASM("2", "f16", "setp.ne.u32 p, 0, 0;\n\t");
}
#undef TCX_MMA_ASM

// Barriers and ring state of the MMA issuer (shared::cta addresses).
struct MmaRing {
    uint32_t full0, empty0, hfull0, hempty0;  // first barrier of each array (8 bytes apart)
    uint32_t lo0, step;                       // desc_lo of stage 0's A_hi plane; stage stride >> 4
    uint32_t a16, b16;                        // plane sizes >> 4: A (A_hi -> A_lo), B (B_hi -> B_lo)
    int nst;
    int stage;
    uint32_t phase, hblk;
};
// Inline fast path of a bounded wait.
__device__ __forceinline__ bool wait_fast(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    return mbar_test(bar, parity) || mbar_wait(bar, parity, abort_flag);
}
template <int CG>
__device__ __forceinline__ void commit_to(uint32_t bar) {
    if constexpr (CG == 1) tc_commit(bar);
    else tc_commit_pair(bar, (uint16_t)3);
}
// The split products of one K chunk in stage st: lo = hi*lo + lo*hi, hi = hi*hi.
// nks = 1: only the first K step holds data (BF16 segment tail).
template <int KIND, int CG, bool FIRST>
__device__ __forceinline__ void chunk_lo(const MmaRing &r, int st, uint32_t dt, uint32_t idesc, int nks) {
    const uint32_t a = r.lo0 + (uint32_t)st * r.step, b = a + 2 * r.a16;
    mma_lo<KIND, CG, !FIRST>(dt, a, b + r.b16, idesc);
    mma_lo<KIND, CG, true>(dt, a + r.a16, b, idesc);
    if (KIND == 1 || nks > 1) {
        mma_lo<KIND, CG, true>(dt, a + 2, b + r.b16 + 2, idesc);
        mma_lo<KIND, CG, true>(dt, a + r.a16 + 2, b + 2, idesc);
    }
}
template <int KIND, int CG>
__device__ __forceinline__ void chunk_hi(const MmaRing &r, int st, uint32_t dt, uint32_t idesc, int nks) {
    const uint32_t a = r.lo0 + (uint32_t)st * r.step, b = a + 2 * r.a16;
    mma_lo<KIND, CG, true>(dt, a, b, idesc);
    if (KIND == 1 || nks > 1) mma_lo<KIND, CG, true>(dt, a + 2, b + 2, idesc);
}
// Every MMA of one work item: K blocks of two chunks, each into a fresh TMEM
// accumulator buffer (tmem + 256 * (block & 1)); within a block the small
// products of each chunk are issued as the chunk lands and the block's hi*hi
// products last, then each stage is released and the block handed to the
// drain (see the kernels).  nch: chunks of the item; dtail, ltail: chunk
// indices of the last chunk of the d and l segments (two each) that hold a
// single K step (BF16 with the segment's extent 16 mod 32), -1 if none.
// Returns false (after flagging) when a bounded wait expired.
template <int KIND, int CG>
__device__ __forceinline__ bool mma_item(MmaRing &r, uint32_t tmem, uint32_t idesc, int nch, int dt0, int dt1,
                                         int lt0, int lt1, volatile int *abort_flag, int *fail_code) {
    for (int c0 = 0; c0 < nch; c0 += 2) {
        const bool two = c0 + 1 < nch;
        const uint32_t buf = r.hblk & 1u;
        const uint32_t dt = tmem + buf * 256u;
        const int s0 = r.stage;
        if (!wait_fast(r.full0 + 8u * (uint32_t)s0, r.phase, abort_flag)) { *fail_code = DERR_TIMEOUT_FULL; return false; }
        if (!wait_fast(r.hempty0 + 8u * buf, ((r.hblk >> 1) & 1u) ^ 1u, abort_flag)) {
            *fail_code = DERR_TIMEOUT_TMEM;
            return false;
        }
        tc_fence_after();
        const int n0 = (c0 == dt0 || c0 == dt1 || c0 == lt0 || c0 == lt1) ? 1 : 2;
        chunk_lo<KIND, CG, true>(r, s0, dt, idesc, n0);
        if (++r.stage == r.nst) { r.stage = 0; r.phase ^= 1u; }
        int s1 = -1, n1 = 2;
        if (two) {
            s1 = r.stage;
            if (!wait_fast(r.full0 + 8u * (uint32_t)s1, r.phase, abort_flag)) { *fail_code = DERR_TIMEOUT_FULL; return false; }
            tc_fence_after();
            n1 = (c0 + 1 == dt0 || c0 + 1 == dt1 || c0 + 1 == lt0 || c0 + 1 == lt1) ? 1 : 2;
            chunk_lo<KIND, CG, false>(r, s1, dt, idesc, n1);
            if (++r.stage == r.nst) { r.stage = 0; r.phase ^= 1u; }
        }
        chunk_hi<KIND, CG>(r, s0, dt, idesc, n0);
        commit_to<CG>(r.empty0 + 8u * (uint32_t)s0);
        if (two) {
            chunk_hi<KIND, CG>(r, s1, dt, idesc, n1);
            commit_to<CG>(r.empty0 + 8u * (uint32_t)s1);
        }
        commit_to<CG>(r.hfull0 + 8u * buf);
        r.hblk++;
    }
    return true;
}

__device__ __forceinline__ void tma_load_5d(uint32_t dst, const CUtensorMap *map, uint32_t bar,
                                            int c0, int c1, int c2, int c3, int c4) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4)
        : "memory");
}
// 8 consecutive accumulator columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tc_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr));
}

inline PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
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

inline bool encode(CUtensorMap *m, CUtensorMapDataType dt, int rank, void *base, const uint64_t *dims,
            const uint64_t *strides_bytes, const uint32_t *box, std::string &err, const char *what,
            CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_64B) {
    auto fn = get_encode();
    if (!fn) {
        err = "cuTensorMapEncodeTiled unavailable";
        return false;
    }
    uint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(m, dt, (cuuint32_t)rank, base, (const cuuint64_t *)dims, (const cuuint64_t *)strides_bytes,
                    (const cuuint32_t *)box, (const cuuint32_t *)es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        err = std::string("cuTensorMapEncodeTiled failed for ") + what + " (CUresult " + std::to_string((int)r) + ")";
        return false;
    }
    return true;
}


// Stores one thread's U row (fixed b < v, c < v of group g; a = a0 + j for
// j < na, a0 a multiple of 8) into the mixed paths' cube layout
// (tcorr_internal.cuh): group 0 at C0[a][b][c], 1 at C1[b][a][c], 2 at
// C2[b][c][a].  Ut: the task's U block; nb: cubes per edge.  Every 8 values of
// a lie in one cube; the swizzle is linear, so an element's offset in its
// cube is the thread's part XOR the part of a & 7.  In every group the 8
// values of c & 7 at fixed (a, b) fill one aligned 32-byte row, so a warp's
// store (2 values of b x 16 of c) writes 4 whole sectors.
__device__ __forceinline__ void store_u_cubes(float *Ut, int nb, int g, int a0, int b, int c, int na,
                                              const float (&total)[128]) {
    const int A0 = a0 >> 3, B = b >> 3, C = c >> 3, lb = b & 7, lc = c & 7;
    int64_t base, step;
    int offs[8];
    if (g == 0) {
        base = (((int64_t)A0 * nb + B) * nb + C) * 3 * 512;
        step = (int64_t)nb * nb * 3 * 512;
#pragma unroll
        for (int q = 0; q < 8; q++) offs[q] = ucube_off(0, lb, lc) ^ ucube_off(q, 0, 0);
    } else if (g == 1) {
        base = ((((int64_t)B * nb + A0) * nb + C) * 3 + 1) * 512;
        step = (int64_t)nb * 3 * 512;
#pragma unroll
        for (int q = 0; q < 8; q++) offs[q] = ucube_off(lb, 0, lc) ^ ucube_off(0, q, 0);
    } else {  // element (x, y, z) = (b, c, a) of C2 at ucube_off(x, z, y)
        base = ((((int64_t)B * nb + C) * nb + A0) * 3 + 2) * 512;
        step = 3 * 512;
#pragma unroll
        for (int q = 0; q < 8; q++) offs[q] = ucube_off(lb, 0, lc) ^ ucube_off(0, q, 0);
    }
    float *p = Ut + base;
    if (na >= 128) {
#pragma unroll
        for (int j = 0; j < 128; j++) {
            p[offs[j & 7]] = total[j];
            if ((j & 7) == 7) p += step;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 128; j++) {
            if (j < na) p[offs[j & 7]] = total[j];
            if ((j & 7) == 7) p += step;
        }
    }
}

}  // namespace tcx
}  // namespace tcorr
