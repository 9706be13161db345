// Fused energy epilogue (S4) and deterministic reductions (S5).
//
// For a task (i,j,k) with i <= j <= k the energy share is
//   e_ijk = (m/6) sum_{abc} Z^{abc} (W^{abc} + Y^{abc}) / D^{abc},
//   Z = 8 W^{abc} - 4 (W^{acb} + W^{bac} + W^{cba}) + 2 (W^{bca} + W^{cab}),
// m the number of distinct orderings of (i,j,k).  This is the sum over those
// orderings of sum_abc W~ V / D (Eqs. piecuch_4th_order/5th_order with the
// tilde of Eq. piecuch_tilde_quantity): W, Y and D are invariant under the
// simultaneous permutations of Eq. (symm_operator), so the orderings of ijk
// become permutations of abc, and the tilde coefficients (4/3, -2, 2/3)
// summed over the six orderings give (8, -4 per transposition, 2 per
// 3-cycle).  E[4] uses W in place of V.
//
// One CTA takes one block orbit {A <= B <= C} (blocks of TE virtual indices)
// of one task: it assembles the W cubes of all six block permutations in
// shared memory from the three group tensors,
//   W[x][y][z] = U0[x][y][z] + U1[y][x][z] + U2[z][x][y],
// reading each U row contiguously, then evaluates Z, Y, D and the two energy
// sums for every element of the distinct cubes, and reduces them with warp
// shuffles to one FP64 pair.  Every element (a,b,c) of the task lies in
// exactly one distinct cube of exactly one orbit.
#include "tcorr_internal.cuh"

namespace tcorr {
namespace {

constexpr int NT = 256;

__device__ __forceinline__ void kahan_add(double &s, double &c, double x) {
    const double y = x - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
}

// Position (0, 1, 2) of dimension d of the cube at slot s, for the slots in
// the order abc, acb, bac, bca, cab, cba, computed in registers.
__device__ __forceinline__ int perm_pos(int s, int d) {
    const int p0 = s >> 1;
    const int lo = p0 == 0 ? 1 : 0, hi = p0 == 2 ? 1 : 2;
    return d == 0 ? p0 : ((d == 1) == ((s & 1) == 0) ? lo : hi);
}
__device__ __forceinline__ int pick3(int a, int b, int c, int k) { return k == 0 ? a : (k == 1 ? b : c); }

// ---- float-float (double-FP32) arithmetic ------------------------------------
// A value hi + lo with |lo| <= ulp(hi) / 2 carries ~48 significant bits.  The
// split-precision epilogue forms its denominators, their reciprocals and the
// products with them this way, on the FP32 pipe: GB300's FP64 pipe runs at
// 1/64 of the FP32 rate, and with one FP64 Newton step per element orbit it
// bounded that kernel.  TwoSum (Knuth) and Fast2Sum (Dekker) are error-free
// transformations of a sum; fmaf gives the exact error of a product.
struct ff {
    float hi, lo;
};
__device__ __forceinline__ ff ff_two_sum(float a, float b) {  // s + e == a + b exactly
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff ff_fast(float a, float b) {  // |a| >= |b|: s + e == a + b exactly
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ff ff_sub(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, -b.hi);
    return ff_fast(s.hi, s.lo + (a.lo - b.lo));
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = ff_two_sum(a.hi, b.hi);
    return ff_fast(s.hi, s.lo + (a.lo + b.lo));
}
// 1/d: an FP32 reciprocal r of d.hi (relative error e ~ 2^-22) and its first
// Newton correction r (1 - d r) from the exact residual (two FMAs): error ~e^2
__device__ __forceinline__ ff ff_recip(ff d) {
    const float r = __fdividef(1.f, d.hi);
    const float e = fmaf(-d.lo, r, fmaf(-d.hi, r, 1.f));
    return {r, r * e};
}
// x * r for an FP32 x: the exact product error of x * r.hi plus x * r.lo
__device__ __forceinline__ ff ff_mul(float x, ff r) {
    const float p = x * r.hi;
    return ff_fast(p, fmaf(x, r.lo, fmaf(x, r.hi, -p)));
}
__device__ __forceinline__ ff ff_of(double x) {  // x rounded to ~48 bits
    const float hi = (float)x;
    return {hi, (float)(x - (double)hi)};
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// As cta_sum2 for float-float pairs: summed in float-float (FP32 pipe) and
// converted to FP64 once, by thread 0.
__device__ __forceinline__ void cta_sum2_ff(ff a4, ff a5, ff (*red)[2], double *out, int tid) {
    red[tid][0] = a4;
    red[tid][1] = a5;
    __syncthreads();
    if (tid < 32) {
        ff b4 = red[tid][0], b5 = red[tid][1];
#pragma unroll
        for (int k = 1; k < NT / 32; k++) {
            b4 = ff_add(b4, red[tid + 32 * k][0]);
            b5 = ff_add(b5, red[tid + 32 * k][1]);
        }
        for (int off = 16; off > 0; off >>= 1) {
            const ff c4 = {__shfl_xor_sync(0xffffffffu, b4.hi, off), __shfl_xor_sync(0xffffffffu, b4.lo, off)};
            const ff c5 = {__shfl_xor_sync(0xffffffffu, b5.hi, off), __shfl_xor_sync(0xffffffffu, b5.lo, off)};
            b4 = ff_add(b4, c4);
            b5 = ff_add(b5, c5);
        }
        if (tid == 0) {
            out[0] = ff_to_double(b4);
            out[1] = ff_to_double(b5);
        }
    }
}

// Sum over the CTA of one (E4, E5) pair per thread, in a fixed order, into
// out[0..1]: the NT pairs through shared memory, NT / 32 per lane of warp 0,
// then a shuffle tree.  (A shuffle tree over all NT threads would put ten
// FP64 adds per thread on the FP64 pipe, which bounds these kernels.)
__device__ __forceinline__ void cta_sum2(double a4, double a5, double (*red)[2], double *out, int tid) {
    red[tid][0] = a4;
    red[tid][1] = a5;
    __syncthreads();
    if (tid < 32) {
        double b4 = red[tid][0], b5 = red[tid][1];
#pragma unroll
        for (int k = 1; k < NT / 32; k++) {
            b4 += red[tid + 32 * k][0];
            b5 += red[tid + 32 * k][1];
        }
        for (int off = 16; off > 0; off >>= 1) {
            b4 += __shfl_xor_sync(0xffffffffu, b4, off);
            b5 += __shfl_xor_sync(0xffffffffu, b5, off);
        }
        if (tid == 0) {
            out[0] = b4;
            out[1] = b5;
        }
    }
}

// FP64 epilogue; TE: cube edge.  Orbits of three distinct blocks take the
// element-orbit form (the six orderings of one (a,b,c) share one denominator
// and the E/O expansion of Z, as in the mixed epilogue), orbits with repeated
// blocks the generic per-element form.
template <typename UT, typename CT, int TE>
__global__ void __launch_bounds__(NT, 3) epilogue_kernel(const Wave wv) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT *Ws = reinterpret_cast<CT *>(smem_raw);
    constexpr int TP = TE + 1;               // padded innermost extent
    constexpr int CUBE = TE * TE * TP;       // smem elements per cube
    constexpr int NE = TE * TE * TE;         // elements per cube
    __shared__ int comp[6][6];
    __shared__ int distinct[6];
    __shared__ double red[NT][2];

    const int64_t item = blockIdx.x;
    const Seg sg = wv.segs[seg_find(wv.segs, wv.nseg, item, [](const Seg &x) { return x.epi0; })];
    const InstDesc &p = wv.descs[sg.inst];
    const int o = p.dm.o, v = p.dm.v, vc = p.dm.vc;
    const int64_t v2 = (int64_t)v * v;
    const int tb = (int)((item - sg.epi0) / p.norb), orb = (int)((item - sg.epi0) % p.norb);
    const int *tk = p.tasks + 3 * (sg.task0 + tb);
    const int ti = tk[0], tj = tk[1], tkk = tk[2];
    double *out = wv.partials + sg.part_off + ((int64_t)tb * p.norb + orb) * 2;
    if (ti == tj && tj == tkk) {  // Z = 0 identically
        if (threadIdx.x == 0) { out[0] = 0.0; out[1] = 0.0; }
        return;
    }
    const int tid = threadIdx.x;
    // the orbit's blocks in registers (every thread reads them), so the U loads
    // below are issued before any barrier
    const int ob0 = p.orbits[3 * orb], ob1 = p.orbits[3 * orb + 1], ob2 = p.orbits[3 * orb + 2];
#define OBP(s, d) pick3(ob0, ob1, ob2, perm_pos((s), (d)))
    const UT *U0 = static_cast<const UT *>(wv.U) + sg.u_off + (int64_t)(tb * 3 + 0) * v2 * vc;
    const UT *U1 = U0 + v2 * vc;
    const UT *U2 = U1 + v2 * vc;
    static_assert(sizeof(UT) == 8 && TE == 8, "16-byte loads of 8-element FP64 rows");
    // pass A loads: W = U0[x][y][z] + U1[y][x][z] (z fastest, pairs of z); pass B
    // loads: U2[z][x][y] (y fastest, pairs of y).  A row never ends within a
    // pair (rows are padded to 16), so a pair that starts inside [0, v) is in bounds.
    double2 ra[6], rb[6], rc[6];
#pragma unroll
    for (int it = 0; it < 6; it++) {
        const int e2 = tid + it * NT;             // 6 slots x 256 pairs
        const int s = e2 >> 8, l = (e2 & 255) * 2;
        const int l0 = l / (TE * TE), l1 = (l / TE) % TE, l2 = l % TE;
        const int x = OBP(s, 0) * TE + l0, y = OBP(s, 1) * TE + l1, z = OBP(s, 2) * TE + l2;
        ra[it] = rb[it] = rc[it] = make_double2(0.0, 0.0);
        if (x < v && y < v && z < v) {
            ra[it] = __ldg(reinterpret_cast<const double2 *>(U0 + ((int64_t)x * v + y) * vc + z));
            rb[it] = __ldg(reinterpret_cast<const double2 *>(U1 + ((int64_t)y * v + x) * vc + z));
        }
        // pass B element pair: (l2', l0', l1') with y fastest
        const int m2 = l / (TE * TE), m0 = (l / TE) % TE, m1 = l % TE;
        const int xb = OBP(s, 0) * TE + m0, yb = OBP(s, 1) * TE + m1, zb = OBP(s, 2) * TE + m2;
        if (xb < v && yb < v && zb < v)
            rc[it] = __ldg(reinterpret_cast<const double2 *>(U2 + ((int64_t)zb * v + xb) * vc + yb));
    }
    if (tid < 36) {  // comp[pi][q]: the slot of permutation pi composed with q
        const int pi = tid / 6, q = tid % 6;
        const int t0 = perm_pos(pi, perm_pos(q, 0)), t1v = perm_pos(pi, perm_pos(q, 1));
        int sig = 0;
        for (int s2 = 0; s2 < 6; s2++)
            if (perm_pos(s2, 0) == t0 && perm_pos(s2, 1) == t1v) sig = s2;
        comp[pi][q] = sig;
    }
    if (tid >= 64 && tid < 70) {
        const int t = tid - 64;
        int d = 1;
        for (int s2 = 0; s2 < t; s2++)
            if (OBP(s2, 0) == OBP(t, 0) && OBP(s2, 1) == OBP(t, 1) && OBP(s2, 2) == OBP(t, 2)) d = 0;
        distinct[t] = d;
    }
#pragma unroll
    for (int it = 0; it < 6; it++) {
        const int e2 = tid + it * NT;
        const int s = e2 >> 8, l = (e2 & 255) * 2;
        const int l0 = l / (TE * TE), l1 = (l / TE) % TE, l2 = l % TE;
        const int z = OBP(s, 2) * TE + l2;
        CT *wp = Ws + s * CUBE + (l0 * TE + l1) * TP + l2;
        wp[0] = (z < v) ? CT(ra[it].x) + CT(rb[it].x) : CT(0);     // row padding is not data
        wp[1] = (z + 1 < v) ? CT(ra[it].y) + CT(rb[it].y) : CT(0);
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < 6; it++) {
        const int e2 = tid + it * NT;
        const int s = e2 >> 8, l = (e2 & 255) * 2;
        const int m2 = l / (TE * TE), m0 = (l / TE) % TE, m1 = l % TE;
        const int yb = OBP(s, 1) * TE + m1;
        CT *wp = Ws + s * CUBE + (m0 * TE + m1) * TP + m2;
        if (yb < v) wp[0] += CT(rc[it].x);
        if (yb + 1 < v) wp[TP] += CT(rc[it].y);
    }
    __syncthreads();

    const CT *t1 = static_cast<const CT *>(p.t1);
    const CT *ov = static_cast<const CT *>(p.ovov);
    const double eijk = p.eps_o[ti] + p.eps_o[tj] + p.eps_o[tkk];
    const CT coef[6] = {CT(8), CT(-4), CT(-4), CT(2), CT(2), CT(-4)};
    // ovov rows used by Y: (j y | k z), (i x | k z), (i x | j y)
    const CT *ov_jk = ov + ((int64_t)tj * v * o + tkk) * v;   // [y][z] stride o*v in y
    const CT *ov_ik = ov + ((int64_t)ti * v * o + tkk) * v;   // [x][z]
    const CT *ov_ij = ov + ((int64_t)ti * v * o + tj) * v;    // [x][y]
    const int64_t ovs = (int64_t)o * v;

    double s4 = 0.0, c4 = 0.0, s5 = 0.0, c5 = 0.0;
    if (ob0 < ob1 && ob1 < ob2) {
        // distinct blocks A < B < C: element orbits; slot q holds the element
        // with indices ordered as q (abc, acb, bac, bca, cab, cba); even slots
        // 0, 3, 4, odd 1, 2, 5; Z_q = 6 w_q + 2E - 4O (even) or 6 w_q + 2O - 4E (odd)
        // thread: fixed (b, c), a = la0 and la0 + TE/2 (the TE^3 element orbits
        // over NT = TE^3 / 2 threads); what depends only on b and c is read once
        static_assert(NE == 2 * NT, "two element orbits per thread");
        const int A0 = ob0 * TE, B0 = ob1 * TE, C0 = ob2 * TE;
        const int lb = (tid / TE) % TE, lc = tid % TE, la0 = tid / (TE * TE);
        const int b = B0 + lb, c = C0 + lc;
        CT a4 = CT(0), a5 = CT(0);
        if (b < v && c < v) {
        const CT tib = t1[ti * v + b], tic = t1[ti * v + c];
        const CT tjb = t1[tj * v + b], tjc = t1[tj * v + c];
        const CT tkb = t1[tkk * v + b], tkc = t1[tkk * v + c];
        const CT jk_bc = ov_jk[b * ovs + c], jk_cb = ov_jk[c * ovs + b];
        const CT ik_bc = ov_ik[b * ovs + c], ik_cb = ov_ik[c * ovs + b];
        const CT ij_bc = ov_ij[b * ovs + c], ij_cb = ov_ij[c * ovs + b];
        const CT ebc = eijk - p.eps_v[b] - p.eps_v[c];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int la = la0 + h * (TE / 2), a = A0 + la;
            if (a >= v) break;  // a grows with h
            const CT w0 = Ws[0 * CUBE + (la * TE + lb) * TP + lc];
            const CT w1 = Ws[1 * CUBE + (la * TE + lc) * TP + lb];
            const CT w2 = Ws[2 * CUBE + (lb * TE + la) * TP + lc];
            const CT w3 = Ws[3 * CUBE + (lb * TE + lc) * TP + la];
            const CT w4 = Ws[4 * CUBE + (lc * TE + la) * TP + lb];
            const CT w5 = Ws[5 * CUBE + (lc * TE + lb) * TP + la];
            const CT tia = t1[ti * v + a], tja = t1[tj * v + a], tka = t1[tkk * v + a];
            // (j u | k w), (i u | k w), (i u | j w) over the ordered pairs of {a, b, c} that hold a
            const CT jk_ac = ov_jk[a * ovs + c], jk_ca = ov_jk[c * ovs + a];
            const CT jk_ab = ov_jk[a * ovs + b], jk_ba = ov_jk[b * ovs + a];
            const CT ik_ac = ov_ik[a * ovs + c], ik_ca = ov_ik[c * ovs + a];
            const CT ik_ab = ov_ik[a * ovs + b], ik_ba = ov_ik[b * ovs + a];
            const CT ij_ac = ov_ij[a * ovs + c], ij_ca = ov_ij[c * ovs + a];
            const CT ij_ab = ov_ij[a * ovs + b], ij_ba = ov_ij[b * ovs + a];
            // Y at each ordering q of (a,b,c): t^{q0}_i (j q1|k q2) + t^{q1}_j (i q0|k q2) + t^{q2}_k (i q0|j q1)
            const CT y0 = tia * jk_bc + tjb * ik_ac + tkc * ij_ab;
            const CT y1 = tia * jk_cb + tjc * ik_ab + tkb * ij_ac;
            const CT y2 = tib * jk_ac + tja * ik_bc + tkc * ij_ba;
            const CT y3 = tib * jk_ca + tjc * ik_ba + tka * ij_bc;
            const CT y4 = tic * jk_ab + tja * ik_cb + tkb * ij_ca;
            const CT y5 = tic * jk_ba + tjb * ik_ca + tka * ij_cb;
            const CT E = w0 + w3 + w4, O = w1 + w2 + w5;
            const CT ww = w0 * w0 + w1 * w1 + w2 * w2 + w3 * w3 + w4 * w4 + w5 * w5;
            const CT wy = w0 * y0 + w1 * y1 + w2 * y2 + w3 * y3 + w4 * y4 + w5 * y5;
            const CT q4 = CT(6) * ww + CT(2) * (E * E + O * O) - CT(8) * E * O;
            const CT q5 = CT(6) * wy + (CT(2) * E - CT(4) * O) * (y0 + y3 + y4) + (CT(2) * O - CT(4) * E) * (y1 + y2 + y5);
            const CT r = CT(1) / (ebc - p.eps_v[a]);
            a4 += q4 * r;
            a5 += q5 * r;
        }
        }
        kahan_add(s4, c4, double(a4));
        kahan_add(s5, c5, double(a5));
    } else
    for (int s = 0; s < 6; s++) {
        if (!distinct[s]) continue;
        CT a4 = CT(0), a5 = CT(0);
        const int X0 = OBP(s, 0) * TE, Y0 = OBP(s, 1) * TE, Z0 = OBP(s, 2) * TE;
        for (int l = tid; l < NE; l += NT) {
            const int lv0 = l / (TE * TE), lv1 = (l / TE) % TE, lv2 = l % TE;
            const int x = X0 + lv0, y = Y0 + lv1, z = Z0 + lv2;
            if (x >= v || y >= v || z >= v) continue;
            CT zv = CT(0);
#pragma unroll
            for (int q = 0; q < 6; q++) {
                const int sg = comp[s][q];
                const int m0 = pick3(lv0, lv1, lv2, perm_pos(q, 0)), m1 = pick3(lv0, lv1, lv2, perm_pos(q, 1)),
                          m2 = pick3(lv0, lv1, lv2, perm_pos(q, 2));
                zv += coef[q] * Ws[sg * CUBE + (m0 * TE + m1) * TP + m2];
            }
            const CT w0 = Ws[s * CUBE + (lv0 * TE + lv1) * TP + lv2];
            const CT yv = t1[ti * v + x] * ov_jk[y * ovs + z] + t1[tj * v + y] * ov_ik[x * ovs + z] +
                          t1[tkk * v + z] * ov_ij[x * ovs + y];
            const CT dn = eijk - p.eps_v[x] - p.eps_v[y] - p.eps_v[z];
            const CT r = CT(1) / dn;
            a4 += zv * w0 * r;
            a5 += zv * yv * r;
        }
        kahan_add(s4, c4, double(a4));
        kahan_add(s5, c5, double(a5));
    }
    cta_sum2(s4 - c4, s5 - c5, red, out, tid);  // the compensation folded
}


#undef OBP

// Mixed-precision epilogue: the same block-orbit algorithm with 8^3 cubes of
// FP32 W (the tensor-core contractions' output), sized for occupancy (about
// 20 KB of shared memory, 5 CTAs per SM).  The U loads of a thread are issued
// first, right after the orbit's block indices are read, and consumed after
// the Y operands have been staged, so their latency overlaps the staging.
// The Y operands of the orbit (t1 rows and the three ovov sub-blocks) are
// staged in shared memory, with the orbit's virtual energies in FP64 and as
// FP32 offsets from their block origins.
//
// Precision of the energy terms (the numerators are FP32; denominators, their
// reciprocals, the products with them and all sums to FP64 accuracy):
//  - the element-orbit numerators sum_q Z_q W_q and sum_q Z_q Y_q (six
//    orderings of one (a,b,c), or one element of an orbit with repeated
//    blocks) are formed in FP32 from the FP32 W, Y;
//  - the denominator D = e_i+e_j+e_k - e_a - e_b - e_c, its reciprocal and
//    numerator x 1/D are formed in float-float (double-FP32) arithmetic from
//    the orbital energies rounded to ~48 bits: relative error ~2^-44, on the
//    FP32 pipe (see ff above);
//  - the terms are summed in float-float per thread and over the CTA (a
//    fixed order), converted to FP64 once per orbit; the orbit partials of a
//    task are summed in FP64 (Kahan) by the task reduction.
constexpr int F8 = 8;
constexpr int FP0 = 69, FP1 = 8;    // plane / row pitch of a cube: at most 2-way bank conflicts
constexpr int FSLOT = F8 * FP0;     // floats per cube slot
#ifndef EPI_F32_CTAS
#define EPI_F32_CTAS 5
#endif

__global__ void __launch_bounds__(NT, EPI_F32_CTAS) epilogue_f32_kernel(const Wave wv) {
    __shared__ float Ws[6 * FSLOT];
    __shared__ float T1s[3][3][F8];          // [occupied i,j,k][orbit block][local]
    __shared__ __align__(16) float OVs[3][3][3][F8 * F8];  // [(jk),(ik),(ij)][block][block][8x8]
    __shared__ ff Evs[3][F8];                // [orbit block][local] virtual energies (float-float)
    __shared__ ff eijk_s;                    // e_i + e_j + e_k (float-float)
    __shared__ int comp[6][6];
    __shared__ int distinct[6];
    __shared__ ff red[NT][2];

    const int64_t item = blockIdx.x;
    const Seg sg = wv.segs[seg_find(wv.segs, wv.nseg, item, [](const Seg &x) { return x.epi0; })];
    const InstDesc &p = wv.descs[sg.inst];
    const int o = p.dm.o, v = p.dm.v, vc = p.dm.vc;
    const int64_t v2 = (int64_t)v * v;
    const int tb = (int)((item - sg.epi0) / p.norb), orb = (int)((item - sg.epi0) % p.norb);
    const int tid = threadIdx.x;
    const int *tk = p.tasks + 3 * (sg.task0 + tb);
    const int ti = tk[0], tj = tk[1], tkk = tk[2];
    double *out = wv.partials + sg.part_off + ((int64_t)tb * p.norb + orb) * 2;
    if (ti == tj && tj == tkk) {
        if (tid == 0) { out[0] = 0.0; out[1] = 0.0; }
        return;
    }
    // every thread reads the orbit's blocks itself (no shared-memory round trip),
    // so the U loads below can be issued before any barrier
    const int ob0 = p.orbits[3 * orb], ob1 = p.orbits[3 * orb + 1], ob2 = p.orbits[3 * orb + 2];
#define OBP(s, d) pick3(ob0, ob1, ob2, perm_pos((s), (d)))

    // W[x][y][z] = S0[x][y][z] + S1[x][y][z] + S2[z][x][y]: slots 0 and 1 read
    // along z, slot 2 along y (all rows contiguous); the loads are issued first
    // and consumed after the Y operands have been staged.
    const float *S0 = static_cast<const float *>(wv.U) + sg.u_off + (int64_t)(tb * 3 + 0) * v2 * vc;
    const int64_t gs = v2 * vc;
    float4 ra[3], rb[3], rc[3];
#pragma unroll
    for (int it = 0; it < 3; it++) {
        const int idx = tid + it * NT;            // 6 slots x 64 rows x 2 halves = 768
        const int s = idx >> 7, row = (idx >> 1) & 63, hf = idx & 1;
        const int x = OBP(s, 0) * F8 + (row >> 3), y = OBP(s, 1) * F8 + (row & 7);
        const int z0 = OBP(s, 2) * F8 + hf * 4;
        ra[it] = rb[it] = rc[it] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x < v && y < v && z0 < v) {
            const float4 *q = reinterpret_cast<const float4 *>(S0 + ((int64_t)x * v + y) * vc + z0);
            ra[it] = __ldg(q);
            rb[it] = __ldg(q + gs / 4);
        }
        const int z = OBP(s, 2) * F8 + (row >> 3), x2 = OBP(s, 0) * F8 + (row & 7);
        const int y0 = OBP(s, 1) * F8 + hf * 4;
        if (z < v && x2 < v && y0 < v)
            rc[it] = __ldg(reinterpret_cast<const float4 *>(S0 + 2 * gs + ((int64_t)z * v + x2) * vc + y0));
    }

    if (tid < 36) {  // comp[pi][q]: the slot of permutation pi composed with q
        const int pi = tid / 6, q = tid % 6;
        const int t0 = perm_pos(pi, perm_pos(q, 0)), t1v = perm_pos(pi, perm_pos(q, 1));
        int sig = 0;
        for (int s = 0; s < 6; s++)
            if (perm_pos(s, 0) == t0 && perm_pos(s, 1) == t1v) sig = s;
        comp[pi][q] = sig;
    }
    if (tid >= 64 && tid < 70) {
        const int t = tid - 64;
        int d = 1;
        for (int s = 0; s < t; s++)
            if (OBP(s, 0) == OBP(t, 0) && OBP(s, 1) == OBP(t, 1) && OBP(s, 2) == OBP(t, 2)) d = 0;
        distinct[t] = d;
    }
    if (tid == 96) eijk_s = ff_of(p.eps_o[ti] + p.eps_o[tj] + p.eps_o[tkk]);
    // stage t1, ovov sub-blocks and block-relative energies.  The FP32 inputs
    // are zero padded to vp (t1 rows [p][x], ovov slabs [p][q][x][z]): every
    // orbit block lies inside, and a sub-block row is two aligned float4 loads.
    const int vp = (v + F8 - 1) / F8 * F8;
    const float *t1 = static_cast<const float *>(p.t1);
    const float *ov = static_cast<const float *>(p.ovov);
    if (tid < 3 * 3 * F8) {
        const int oc = tid / (3 * F8), b = (tid / F8) % 3, m = tid % F8;
        const int occ = oc == 0 ? ti : (oc == 1 ? tj : tkk);
        T1s[oc][b][m] = t1[occ * vp + pick3(ob0, ob1, ob2, b) * F8 + m];
    } else if (tid >= 96 + 32 && tid < 96 + 32 + 3 * F8) {
        const int e = tid - 128, b = e / F8, m = e % F8, x = pick3(ob0, ob1, ob2, b) * F8 + m;
        Evs[b][m] = ff_of(x < v ? p.eps_v[x] : 0.0);
    }
    // slices: 0 = (j y | k z), 1 = (i x | k z), 2 = (i x | j y); 3 x 9 sub-blocks
    // x 8 rows x 2 halves = 432 float4
    for (int e = tid; e < 3 * 9 * F8 * 2; e += NT) {
        const int sl = e / 144, rem = e - sl * 144, bb = rem >> 4, m = (rem >> 1) & 7, h = rem & 1;
        const int ba = bb / 3, bc = bb - 3 * ba;
        const int r = pick3(ob0, ob1, ob2, ba) * F8 + m, c = pick3(ob0, ob1, ob2, bc) * F8 + 4 * h;
        const int first = sl == 0 ? tj : ti, second = sl == 2 ? tj : tkk;
        const float4 val = __ldg(reinterpret_cast<const float4 *>(ov + ((int64_t)(first * o + second) * vp + r) * vp + c));
        *reinterpret_cast<float4 *>(&OVs[sl][ba][bc][m * F8 + 4 * h]) = val;
    }

#pragma unroll
    for (int it = 0; it < 3; it++) {
        const int idx = tid + it * NT;
        const int s = idx >> 7, row = (idx >> 1) & 63, hf = idx & 1;
        const int z0 = OBP(s, 2) * F8 + hf * 4;
        float *wrow = Ws + s * FSLOT + (row >> 3) * FP0 + (row & 7) * FP1 + hf * 4;
        const float w[4] = {ra[it].x + rb[it].x, ra[it].y + rb[it].y, ra[it].z + rb[it].z, ra[it].w + rb[it].w};
#pragma unroll
        for (int m = 0; m < 4; m++) wrow[m] = (z0 + m < v) ? w[m] : 0.f;  // U row padding is not data
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < 3; it++) {
        const int idx = tid + it * NT;
        const int s = idx >> 7, row = (idx >> 1) & 63, hf = idx & 1;
        const int lz = row >> 3, lx = row & 7;
        const int y0 = OBP(s, 1) * F8 + hf * 4;
        const float w[4] = {rc[it].x, rc[it].y, rc[it].z, rc[it].w};
#pragma unroll
        for (int m = 0; m < 4; m++)
            if (y0 + m < v) Ws[s * FSLOT + lx * FP0 + (hf * 4 + m) * FP1 + lz] += w[m];
    }
    __syncthreads();

    const ff eijk = eijk_s;
    ff A4 = {0.f, 0.f}, A5 = {0.f, 0.f};
    if (ob0 < ob1 && ob1 < ob2) {
        // Distinct blocks: each thread takes element orbits, the six orderings
        // of one (a,b,c) with a in A, b in B, c in C.  Slot q holds the element
        // with indices ordered as q (slots 0..5 = abc, acb, bac, bca, cab, cba);
        // even slots 0,3,4, odd slots 1,2,5.  With E and O the sums of W over
        // the even and odd slots, Z at slot q is 6 w_q + 2E - 4O (q even) or
        // 6 w_q + 2O - 4E (q odd), and all six share one denominator.
        // thread: fixed (b, c) = (lb, lc), a = la0 and la0 + 4 (the 512 element
        // orbits of the cube over 256 threads); what depends only on b and c is
        // read once
        const int A0 = ob0 * F8, B0 = ob1 * F8, C0 = ob2 * F8;
        const int lb = (tid >> 3) & 7, lc = tid & 7, la0 = tid >> 6;
#define OVV(sl, pu, pw, lu, lw) OVs[sl][pu][pw][(lu) * F8 + (lw)]
        const float tib = T1s[0][1][lb], tic = T1s[0][2][lc];
        const float tjb = T1s[1][1][lb], tjc = T1s[1][2][lc];
        const float tkb = T1s[2][1][lb], tkc = T1s[2][2][lc];
        const float jk_bc = OVV(0, 1, 2, lb, lc), jk_cb = OVV(0, 2, 1, lc, lb);
        const float ik_bc = OVV(1, 1, 2, lb, lc), ik_cb = OVV(1, 2, 1, lc, lb);
        const float ij_bc = OVV(2, 1, 2, lb, lc), ij_cb = OVV(2, 2, 1, lc, lb);
        const ff dbc = ff_sub(ff_sub(eijk, Evs[1][lb]), Evs[2][lc]);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int la = la0 + 4 * h;
            if (A0 + la >= v || B0 + lb >= v || C0 + lc >= v) break;  // a grows with h
            const float w0 = Ws[0 * FSLOT + la * FP0 + lb * FP1 + lc];
            const float w1 = Ws[1 * FSLOT + la * FP0 + lc * FP1 + lb];
            const float w2 = Ws[2 * FSLOT + lb * FP0 + la * FP1 + lc];
            const float w3 = Ws[3 * FSLOT + lb * FP0 + lc * FP1 + la];
            const float w4 = Ws[4 * FSLOT + lc * FP0 + la * FP1 + lb];
            const float w5 = Ws[5 * FSLOT + lc * FP0 + lb * FP1 + la];
            // t1 of occupied i, j, k at a (at b and c above)
            const float tia = T1s[0][0][la], tja = T1s[1][0][la], tka = T1s[2][0][la];
            // (j u | k w), (i u | k w), (i u | j w) for the ordered pairs of {a, b, c} that hold a
            const float jk_ac = OVV(0, 0, 2, la, lc), jk_ca = OVV(0, 2, 0, lc, la);
            const float jk_ab = OVV(0, 0, 1, la, lb), jk_ba = OVV(0, 1, 0, lb, la);
            const float ik_ac = OVV(1, 0, 2, la, lc), ik_ca = OVV(1, 2, 0, lc, la);
            const float ik_ab = OVV(1, 0, 1, la, lb), ik_ba = OVV(1, 1, 0, lb, la);
            const float ij_ac = OVV(2, 0, 2, la, lc), ij_ca = OVV(2, 2, 0, lc, la);
            const float ij_ab = OVV(2, 0, 1, la, lb), ij_ba = OVV(2, 1, 0, lb, la);
            // Y at each ordering q of (a,b,c): t^{q0}_i (j q1|k q2) + t^{q1}_j (i q0|k q2) + t^{q2}_k (i q0|j q1)
            const float y0 = tia * jk_bc + tjb * ik_ac + tkc * ij_ab;
            const float y1 = tia * jk_cb + tjc * ik_ab + tkb * ij_ac;
            const float y2 = tib * jk_ac + tja * ik_bc + tkc * ij_ba;
            const float y3 = tib * jk_ca + tjc * ik_ba + tka * ij_bc;
            const float y4 = tic * jk_ab + tja * ik_cb + tkb * ij_ca;
            const float y5 = tic * jk_ba + tjb * ik_ca + tka * ij_cb;
            const float E = w0 + w3 + w4, O = w1 + w2 + w5;
            const float ww = w0 * w0 + w1 * w1 + w2 * w2 + w3 * w3 + w4 * w4 + w5 * w5;
            const float wy = w0 * y0 + w1 * y1 + w2 * y2 + w3 * y3 + w4 * y4 + w5 * y5;
            const float s4 = 6.f * ww + 2.f * (E * E + O * O) - 8.f * E * O;
            const float s5 = 6.f * wy + (2.f * E - 4.f * O) * (y0 + y3 + y4) + (2.f * O - 4.f * E) * (y1 + y2 + y5);
            const ff r = ff_recip(ff_sub(dbc, Evs[0][la]));
            A4 = ff_add(A4, ff_mul(s4, r));
            A5 = ff_add(A5, ff_mul(s5, r));
        }
#undef OVV
    } else {
        // blocks repeat: element by element over the distinct cube slots
        for (int s = 0; s < 6; s++) {
            if (!distinct[s]) continue;
            const int p0 = perm_pos(s, 0), p1 = perm_pos(s, 1), p2 = perm_pos(s, 2);
            const float *W0 = Ws + comp[s][0] * FSLOT, *W1 = Ws + comp[s][1] * FSLOT;
            const float *W2 = Ws + comp[s][2] * FSLOT, *W3 = Ws + comp[s][3] * FSLOT;
            const float *W4 = Ws + comp[s][4] * FSLOT, *W5 = Ws + comp[s][5] * FSLOT;
            for (int l = tid; l < 512; l += NT) {
                const int l0 = l >> 6, l1 = (l >> 3) & 7, l2 = l & 7;
                const int x = pick3(ob0, ob1, ob2, p0) * F8 + l0, y = pick3(ob0, ob1, ob2, p1) * F8 + l1,
                          z = pick3(ob0, ob1, ob2, p2) * F8 + l2;
                if (x >= v || y >= v || z >= v) continue;
                const float w0 = W0[l0 * FP0 + l1 * FP1 + l2];
                // Z = 8 W(abc) - 4 (W(acb) + W(bac) + W(cba)) + 2 (W(bca) + W(cab))
                const float zv = 8.f * w0 -
                                 4.f * (W1[l0 * FP0 + l2 * FP1 + l1] + W2[l1 * FP0 + l0 * FP1 + l2] +
                                        W5[l2 * FP0 + l1 * FP1 + l0]) +
                                 2.f * (W3[l1 * FP0 + l2 * FP1 + l0] + W4[l2 * FP0 + l0 * FP1 + l1]);
                const float yv = T1s[0][p0][l0] * OVs[0][p1][p2][l1 * F8 + l2] +
                                 T1s[1][p1][l1] * OVs[1][p0][p2][l0 * F8 + l2] +
                                 T1s[2][p2][l2] * OVs[2][p0][p1][l0 * F8 + l1];
                const ff r = ff_recip(ff_sub(ff_sub(ff_sub(eijk, Evs[p0][l0]), Evs[p1][l1]), Evs[p2][l2]));
                A4 = ff_add(A4, ff_mul(zv * w0, r));
                A5 = ff_add(A5, ff_mul(zv * yv, r));
            }
        }
    }
    // the orbit partials of a task are summed in FP64 (Kahan) by the task reduction
    cta_sum2_ff(A4, A5, red, out, tid);
}
#undef OBP

// One CTA per task of the wave: Kahan sum of its orbit partials, times m/6.
__global__ void __launch_bounds__(NT) task_reduce_kernel(const Wave wv) {
    __shared__ double red[NT][2];
    const int64_t t = blockIdx.x;
    const int tid = threadIdx.x;
    const Seg sg = wv.segs[seg_find(wv.segs, wv.nseg, t, [](const Seg &x) { return x.red0; })];
    const InstDesc &d = wv.descs[sg.inst];
    const int tb = (int)(t - sg.red0);
    const int norb = d.norb;
    const double *pp = wv.partials + sg.part_off + (int64_t)tb * norb * 2;
    double s4 = 0.0, c4 = 0.0, s5 = 0.0, c5 = 0.0;
    for (int n = tid; n < norb; n += NT) { kahan_add(s4, c4, pp[2 * n]); kahan_add(s5, c5, pp[2 * n + 1]); }
    red[tid][0] = s4 - c4;
    red[tid][1] = s5 - c5;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (tid < w) { red[tid][0] += red[tid + w][0]; red[tid][1] += red[tid + w][1]; }
        __syncthreads();
    }
    if (tid == 0) {
        const int *tk = d.tasks + 3 * (sg.task0 + tb);
        const int i = tk[0], j = tk[1], k = tk[2];
        const double m = (i == j && j == k) ? 0.0 : ((i == j || j == k) ? 3.0 : 6.0);
        d.task_e[2 * (sg.task0 + tb)] = red[0][0] * (m / 6.0);
        d.task_e[2 * (sg.task0 + tb) + 1] = red[0][1] * (m / 6.0);
    }
}

// One CTA per span: Kahan sum of task energies first..first+count-1 of the
// span's problem -> (E4, E5, E).
__global__ void __launch_bounds__(NT) span_sum_kernel(const SumSpan *spans) {
    __shared__ double red[NT][2];
    const SumSpan sp = spans[blockIdx.x];
    const int tid = threadIdx.x;
    double s4 = 0.0, c4 = 0.0, s5 = 0.0, c5 = 0.0;
    for (int64_t n = tid; n < sp.count; n += NT) {
        kahan_add(s4, c4, sp.task_e[2 * (sp.first + n)]);
        kahan_add(s5, c5, sp.task_e[2 * (sp.first + n) + 1]);
    }
    red[tid][0] = s4 - c4;
    red[tid][1] = s5 - c5;
    __syncthreads();
    for (int w = NT / 2; w > 0; w >>= 1) {
        if (tid < w) { red[tid][0] += red[tid + w][0]; red[tid][1] += red[tid + w][1]; }
        __syncthreads();
    }
    if (tid == 0) {
        sp.out[0] = red[0][0];
        sp.out[1] = red[0][1];
        sp.out[2] = red[0][0] + red[0][1];
    }
}

}  // namespace

int epilogue_orbits(int v) {
    const int nb = (v + 7) / 8;
    return nb * (nb + 1) * (nb + 2) / 6;
}

cudaError_t launch_epilogue(int prec, const Wave &w, cudaStream_t st) {
    if (w.n_epi <= 0) return cudaSuccess;
    if (w.n_epi > 0x7fffffff) return cudaErrorInvalidConfiguration;
    if (prec == TCORR_FP64) {
        const size_t smem = sizeof(double) * 6 * 8 * 8 * 9;
        epilogue_kernel<double, double, 8><<<(unsigned)w.n_epi, NT, smem, st>>>(w);
    } else {
        epilogue_f32_kernel<<<(unsigned)w.n_epi, NT, 0, st>>>(w);
    }
    return cudaGetLastError();
}

cudaError_t launch_task_reduce(const Wave &w, cudaStream_t st) {
    if (w.n_red <= 0) return cudaSuccess;
    task_reduce_kernel<<<(unsigned)w.n_red, NT, 0, st>>>(w);
    return cudaGetLastError();
}

cudaError_t launch_span_sums(const SumSpan *spans, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    span_sum_kernel<<<n, NT, 0, st>>>(spans);
    return cudaGetLastError();
}

}  // namespace tcorr
