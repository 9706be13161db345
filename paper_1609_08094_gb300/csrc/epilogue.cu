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
// exactly one distinct cube of exactly one orbit.  (The mixed-precision
// kernel further down takes the same orbits in a persistent, pipelined form.)
#include <algorithm>
#include <cstddef>
#include <mutex>

#include "tc_common.cuh"

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

// A float-float number with arithmetic operators, the compute type of the
// FP64-emulation epilogue: W, t1, ovov and the orbital energies arrive as
// (hi, lo) pairs, so the epilogue runs on the FP32 pipe (64x GB300's FP64
// rate).  Sums as ff_add; products a.hi b.hi exactly (FMA residual) plus the
// cross terms a.hi b.lo + a.lo b.hi; quotients as a product with ff_recip.
// Relative error per operation about 2^-44 of the operands' magnitudes.
struct dd {
    float hi, lo;
    dd() = default;
    __device__ __forceinline__ explicit dd(int c) : hi((float)c), lo(0.f) {}  // small integers: exact
    __device__ __forceinline__ explicit dd(double x) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
    __device__ __forceinline__ dd(ff a) : hi(a.hi), lo(a.lo) {}
    __device__ __forceinline__ operator ff() const { return ff{hi, lo}; }
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ dd &operator+=(dd b) { return *this = dd(ff_add(*this, b)); }
};
__device__ __forceinline__ dd operator+(dd a, dd b) { return dd(ff_add(a, b)); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return dd(ff_sub(a, b)); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    return dd(ff_fast(p, e));
}
__device__ __forceinline__ dd operator/(dd a, dd b) { return a * dd(ff_recip(b)); }
// a U value of the FP64-emulation path: (hi, lo) floats in the 8 bytes of a double
__device__ __forceinline__ dd dd_bits(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return dd(ff{__int_as_float((int)(unsigned)u), __int_as_float((int)(unsigned)(u >> 32))});
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

// A U value as the compute type: FP64 as is, or the (hi, lo) pair of the
// FP64-emulation path; and the virtual orbital energy x in the compute type
template <typename CT> __device__ __forceinline__ CT u_val(double bits);
template <> __device__ __forceinline__ double u_val<double>(double bits) { return bits; }
template <> __device__ __forceinline__ dd u_val<dd>(double bits) { return dd_bits(bits); }
template <typename CT> __device__ __forceinline__ CT eps_vir(const InstDesc &p, int x);
template <> __device__ __forceinline__ double eps_vir<double>(const InstDesc &p, int x) { return p.eps_v[x]; }
template <> __device__ __forceinline__ dd eps_vir<dd>(const InstDesc &p, int x) {
    const float2 e = p.evf[x];
    return dd(ff{e.x, e.y});
}

// FP64 epilogue; TE: cube edge.  Orbits of three distinct blocks take the
// element-orbit form (the six orderings of one (a,b,c) share one denominator
// and the E/O expansion of Z, as in the mixed epilogue), orbits with repeated
// blocks the generic per-element form.  CT = double (FP64 path: U, t1, ovov
// in FP64) or dd (FP64 emulation: all of them float-float pairs, so that no
// operation per element runs on the FP64 pipe).
template <typename CT, int TE>
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
    const double *U0 = static_cast<const double *>(wv.U) + sg.u_off + (int64_t)(tb * 3 + 0) * p.dm.ug;
    const double *U1 = U0 + p.dm.ug;
    const double *U2 = U1 + p.dm.ug;
    static_assert(sizeof(CT) == 8 && TE == 8, "16-byte loads of 8-element rows of 8-byte values");
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
        wp[0] = (z < v) ? u_val<CT>(ra[it].x) + u_val<CT>(rb[it].x) : CT(0);  // row padding is not data
        wp[1] = (z + 1 < v) ? u_val<CT>(ra[it].y) + u_val<CT>(rb[it].y) : CT(0);
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < 6; it++) {
        const int e2 = tid + it * NT;
        const int s = e2 >> 8, l = (e2 & 255) * 2;
        const int m2 = l / (TE * TE), m0 = (l / TE) % TE, m1 = l % TE;
        const int yb = OBP(s, 1) * TE + m1;
        CT *wp = Ws + s * CUBE + (m0 * TE + m1) * TP + m2;
        if (yb < v) wp[0] += u_val<CT>(rc[it].x);
        if (yb + 1 < v) wp[TP] += u_val<CT>(rc[it].y);
    }
    __syncthreads();

    const CT *t1 = static_cast<const CT *>(p.t1);
    const CT *ov = static_cast<const CT *>(p.ovov);
    const CT eijk = CT(p.eps_o[ti] + p.eps_o[tj] + p.eps_o[tkk]);
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
        const CT ebc = eijk - eps_vir<CT>(p, b) - eps_vir<CT>(p, c);
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
            const CT r = CT(1) / (ebc - eps_vir<CT>(p, a));
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
            const CT dn = eijk - eps_vir<CT>(p, x) - eps_vir<CT>(p, y) - eps_vir<CT>(p, z);
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

// Mixed-precision epilogue: the same block-orbit algorithm on 8^3 cubes of
// FP32 W, as a persistent kernel (2 CTAs per SM) with two producer warps and a
// ring of two orbit stages in shared memory.
//
// The tensor-core contractions store each group tensor as its term of W in
// W's own index order, in swizzled 8^3 cubes (tcorr_internal.cuh), so the
// three cubes that make up one W cube sit at the same cube coordinates and
// W = C0 + C1 + C2 element by element, and the three terms of a cube are
// stored side by side.  Per orbit two producer warps fill a free stage, every
// copy completing on the stage's mbarrier: one 6 KB bulk copy (cp.async.bulk)
// per distinct slot (6 for three distinct blocks), and 4-row TMA gathers
// (tile::gather4) from row maps of the blocked FP32 ovov copy (27 8x8
// sub-blocks: 7 gathers), of t1 (9 rows: 3) and of the float-float virtual
// energies (3 blocks: 1) -- 17 copies per orbit, issued by the lanes side by
// side.  The copy issue rate per warp bounded the first versions of this
// kernel: one warp issuing 57 copies per orbit took 0.38 ms per task at
// o=50, v=450 (0.27 ms now; 16-byte cp.async for the small operands was
// slower still).  Eight compute warps evaluate the orbit held in the other
// stage meanwhile.  The cube swizzle makes every W read conflict-free, and
// the index arithmetic per element orbit is a handful of precomputed offsets.
//
// The per-orbit sum over the CTA goes through shared memory in a fixed
// order, summed by one compute warp per orbit in rotation, with
// mbarriers instead of CTA barriers: every wait here is bounded (a wait
// that expires sets the error flag, the other roles see the abort flag,
// and the producer lets its copies in flight land before it returns).
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
constexpr int EPI_CW = NT / 32;                 // compute warps
#ifndef EPI_F32_PRODUCERS
#define EPI_F32_PRODUCERS 2
#endif
constexpr int EPI_PRODUCERS = EPI_F32_PRODUCERS;  // producer warps (one warp issues all copies if 1)
static_assert(EPI_PRODUCERS == 1 || EPI_PRODUCERS == 2, "one or two producer warps");
constexpr int EPI_THREADS = NT + 32 * EPI_PRODUCERS;
#ifndef EPI_F32_STAGES
#define EPI_F32_STAGES 2
#endif
#ifndef EPI_F32_CTAS
#define EPI_F32_CTAS 2
#endif
constexpr int EPI_STAGES = EPI_F32_STAGES;      // orbit stages in shared memory (44 KB each)
constexpr int EPI_CTAS = EPI_F32_CTAS;          // CTAs per SM

struct EpiStage {
    float cube[6][3][512];       // [slot][group]: the three terms of the slot's W cube (as stored in U)
    float ov[3][3][3][F8 * F8];  // [(j y|k z), (i x|k z), (i x|j y)][block][block][8x8]
    float ov_pad[F8 * F8];       // the fourth row of the last 4-row gather
    float t1[3][3][F8];          // [occupied i, j, k][orbit block][local]
    float t1_pad[3][F8];
    float2 ev[3][F8];            // [orbit block][local] eps_v as float-float (hi, lo)
    float2 ev_pad[F8];
};
// each 4-row gather lands 128-byte aligned, rows back to back
static_assert(offsetof(EpiStage, ov) % 128 == 0 && offsetof(EpiStage, t1) % 128 == 0 &&
                  offsetof(EpiStage, ev) % 128 == 0 && sizeof(EpiStage) % 128 == 0,
              "gather destinations are 128-byte aligned");
static_assert(offsetof(EpiStage, ov_pad) == offsetof(EpiStage, ov) + 27 * 256 &&
                  offsetof(EpiStage, t1_pad) == offsetof(EpiStage, t1) + 9 * 32 &&
                  offsetof(EpiStage, ev_pad) == offsetof(EpiStage, ev) + 3 * 64,
              "gather rows are contiguous");
constexpr size_t EPI_SMEM = EPI_STAGES * sizeof(EpiStage) + 128;  // + alignment slack

struct EpiMeta {
    double *out;                 // the orbit's (E4, E5) partial
    ff eijk;                     // e_i + e_j + e_k
    int ob[3];                   // blocks A <= B <= C
    int smap[6];                 // slot whose cubes hold slot s's data (the first with its block triple)
    int kind;                    // 0: no more orbits, 1: three distinct blocks, 2: repeated blocks
    int v;                       // virtual orbitals of the problem
};

// Four rows r0..r3 of a 2-D tensor map (box: one row) to dst, back to back.
__device__ __forceinline__ void gather4_load(uint32_t dst, const CUtensorMap *map, uint32_t bar, int r0, int r1,
                                             int r2, int r3) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5, %6, %7}], [%2];" ::"r"(dst),
        "l"(map), "r"(bar), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3)
        : "memory");
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__global__ void __launch_bounds__(EPI_THREADS, EPI_CTAS) epilogue_f32_kernel(const __grid_constant__ Wave wv) {
    using namespace tcx;
    extern __shared__ __align__(128) unsigned char epi_smem[];
    EpiStage *stg = reinterpret_cast<EpiStage *>(epi_smem + (((smem_u32(epi_smem) + 127u) & ~127u) - smem_u32(epi_smem)));
    __shared__ EpiMeta meta[EPI_STAGES];
    __shared__ __align__(8) uint64_t bar_full[EPI_STAGES], bar_empty[EPI_STAGES];
    __shared__ __align__(8) uint64_t bar_rfull[2], bar_rempty[2];
    __shared__ __align__(16) float4 red[2][NT];
    __shared__ int comp[6][6];
    __shared__ volatile int abort_sh;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        for (int s = 0; s < EPI_STAGES; s++) {
            mbar_init(smem_u32(&bar_full[s]), EPI_PRODUCERS);  // one expect_tx arrival per producer warp
            mbar_init(smem_u32(&bar_empty[s]), EPI_CW);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(smem_u32(&bar_rfull[b]), EPI_CW);
            mbar_init(smem_u32(&bar_rempty[b]), 1);
        }
        abort_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (tid < 36) {  // comp[pi][q]: the slot of permutation pi composed with q
        const int pi = tid / 6, q = tid % 6;
        const int t0 = perm_pos(pi, perm_pos(q, 0)), t1v = perm_pos(pi, perm_pos(q, 1));
        int sig = 0;
        for (int s = 0; s < 6; s++)
            if (perm_pos(s, 0) == t0 && perm_pos(s, 1) == t1v) sig = s;
        comp[pi][q] = sig;
    }
    __syncthreads();  // the last CTA-wide barrier: from here on the roles meet only at mbarriers

    if (warp >= EPI_CW) {
        const int pw = warp - EPI_CW;  // 0: meta, U cubes, energies; 1: ovov and t1 gathers
        // ---------------- producer warp ----------------
        // Every lane runs the same decode (uniform loads).  The segment's and
        // the task's fields live in registers and are reloaded only when they
        // change; the next item's orbit triple is loaded one item ahead, so no
        // dependent global load sits on the path of an orbit's copies.
        int si = -1, tb_c = -1, n = 0;
        int tb_at = 0, orb_at = 0;  // (task, orbit) of the item at hand, advanced by gridDim.x per item
        int64_t sbeg = 0, send = 0, task0 = 0, part_off = 0;
        int o = 0, v = 0, nb = 0, norb = 1;
        int64_t ug = 0;
        const int *tasks = nullptr, *orbits = nullptr;
        const double *eps_o = nullptr;
        const float *Useg = nullptr;
        const CUtensorMap *emaps = nullptr;
        int ti = 0, tj = 0, tkk = 0;
        ff eijk = {0.f, 0.f};
        int pf_orb = -1, pf0 = 0, pf1 = 0, pf2 = 0;  // prefetched orbit triple (current segment)
        bool ok = true;
        for (int64_t it = blockIdx.x; it < wv.n_epi && ok; it += gridDim.x) {
            if (si < 0 || it >= send) {
                si = seg_find(wv.segs, wv.nseg, it, [](const Seg &x) { return x.epi0; });
                const Seg sg = wv.segs[si];
                const InstDesc &p = wv.descs[sg.inst];
                sbeg = sg.epi0;
                send = si + 1 < wv.nseg ? wv.segs[si + 1].epi0 : wv.n_epi;
                task0 = sg.task0;
                part_off = sg.part_off;
                o = p.dm.o;
                v = p.dm.v;
                nb = (v + F8 - 1) / F8;
                norb = p.norb;
                ug = p.dm.ug;
                tasks = p.tasks;
                orbits = p.orbits;
                Useg = static_cast<const float *>(wv.U) + sg.u_off;
                emaps = p.emaps;
                eps_o = p.eps_o;
                tb_c = -1;
                pf_orb = -1;
                tb_at = (int)((it - sbeg) / norb);
                orb_at = (int)((it - sbeg) % norb);
            }
            const int tb = tb_at, orb = orb_at;
            int ob0, ob1, ob2;
            if (pf_orb == orb) {
                ob0 = pf0; ob1 = pf1; ob2 = pf2;
            } else {
                ob0 = orbits[3 * orb]; ob1 = orbits[3 * orb + 1]; ob2 = orbits[3 * orb + 2];
            }
            // the next item's (task, orbit), and its triple when it lies in this segment
            orb_at += gridDim.x;
            if (orb_at >= norb) {
                const int q = orb_at / norb;
                tb_at += q;
                orb_at -= q * norb;
            }
            pf_orb = -1;
            if (it + gridDim.x < send) {
                pf_orb = orb_at;
                pf0 = orbits[3 * pf_orb]; pf1 = orbits[3 * pf_orb + 1]; pf2 = orbits[3 * pf_orb + 2];
            }
            if (tb != tb_c) {
                const int *tk = tasks + 3 * (task0 + tb);
                ti = tk[0]; tj = tk[1]; tkk = tk[2];
                if (!(ti == tj && tj == tkk)) eijk = ff_of(eps_o[ti] + eps_o[tj] + eps_o[tkk]);
                tb_c = tb;
            }
            double *out = wv.partials + part_off + ((int64_t)tb * norb + orb) * 2;
            if (ti == tj && tj == tkk) {  // no energy: nothing to load
                if (lane == 0) { out[0] = 0.0; out[1] = 0.0; }
                continue;
            }
            const int stage = n % EPI_STAGES;
            if (n >= EPI_STAGES &&
                !mbar_wait(smem_u32(&bar_empty[stage]), (uint32_t)((n / EPI_STAGES - 1) & 1), &abort_sh)) {
                if (lane == 0) fail(&abort_sh, wv.err, DERR_TIMEOUT_EMPTY);
                ok = false;
                break;
            }
            // slot s holds the cube with block pick3(ob, perm_pos(s, d)) along axis d;
            // a slot whose triple repeats an earlier one's is not loaded
            int smap[6], loaded = 0, nload = 0;
#pragma unroll
            for (int s = 0; s < 6; s++) {
                smap[s] = s;
#pragma unroll
                for (int t = s - 1; t >= 0; t--)
                    if (pick3(ob0, ob1, ob2, perm_pos(t, 0)) == pick3(ob0, ob1, ob2, perm_pos(s, 0)) &&
                        pick3(ob0, ob1, ob2, perm_pos(t, 1)) == pick3(ob0, ob1, ob2, perm_pos(s, 1)) &&
                        pick3(ob0, ob1, ob2, perm_pos(t, 2)) == pick3(ob0, ob1, ob2, perm_pos(s, 2)))
                        smap[s] = t;
                if (smap[s] == s) { loaded |= 1 << s; nload++; }
            }
            const uint32_t full = smem_u32(&bar_full[stage]);
            // the copies of an orbit: the U cubes of each distinct slot (the three
            // group terms side by side, one 6 KB bulk copy each); the 27 ovov
            // sub-blocks, the 9 t1 rows and the 3 energy blocks as 4-row gathers
            // of their row maps (7, 3 and 1 gathers; a gather's spare rows repeat
            // a valid one and land in the pad rows).  Warp 0 takes the cubes and
            // the energies (and writes the stage's meta), warp 1 ovov and t1.
            constexpr uint32_t ovt1_bytes = 7 * 4 * 256 + 3 * 4 * 32, ev_bytes = 4 * 64;  // gathers write whole 4-row groups
            const uint32_t u_bytes = (uint32_t)nload * 3 * 2048;
            if (lane == 0 && pw != 0) mbar_expect_tx(full, ovt1_bytes);
            if (lane == 0 && pw == 0) {
                EpiMeta &m = meta[stage];
                m.out = out;
                m.eijk = eijk;
                m.ob[0] = ob0; m.ob[1] = ob1; m.ob[2] = ob2;
#pragma unroll
                for (int s = 0; s < 6; s++) m.smap[s] = smap[s];
                m.kind = (ob0 < ob1 && ob1 < ob2) ? 1 : 2;
                m.v = v;
                mbar_expect_tx(full, u_bytes + ev_bytes + (EPI_PRODUCERS == 1 ? ovt1_bytes : 0u));
            }
            __syncwarp();
            const float *Ut = Useg + (int64_t)tb * 3 * ug;
            const uint32_t sb = smem_u32(&stg[stage]);
            // e in [0, 6): cube of slot e; 6: energies; [7, 14): ovov gathers; [14, 17): t1 gathers
            const int e = EPI_PRODUCERS == 1 ? lane : (pw == 0 ? lane : lane + 7);
            if (lane < (EPI_PRODUCERS == 1 ? 17 : (pw == 0 ? 7 : 10))) {
                if (e < 6) {
                    if ((loaded >> e) & 1) {
                        const int X = pick3(ob0, ob1, ob2, perm_pos(e, 0)), Y = pick3(ob0, ob1, ob2, perm_pos(e, 1)),
                                  Z = pick3(ob0, ob1, ob2, perm_pos(e, 2));
                        bulk_load(sb + (uint32_t)offsetof(EpiStage, cube) + (uint32_t)e * 6144u,
                                  Ut + (((int64_t)X * nb + Y) * nb + Z) * 3 * 512, 6144u, full);
                    }
                } else if (e == 6) {
                    gather4_load(sb + (uint32_t)offsetof(EpiStage, ev), emaps + 2, full, ob0, ob1, ob2, ob0);
                } else if (e < 14) {
                    // rows ((p o + q) nb + X) nb + Z of the sub-blocks q = 4 k .. 4 k + 3
                    int r[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int q = min(4 * (e - 7) + u, 26), sl = q / 9, ba = (q / 3) % 3, bc = q % 3;
                        const int first = sl == 0 ? tj : ti, second = sl == 2 ? tj : tkk;
                        r[u] = ((first * o + second) * nb + pick3(ob0, ob1, ob2, ba)) * nb + pick3(ob0, ob1, ob2, bc);
                    }
                    gather4_load(sb + (uint32_t)offsetof(EpiStage, ov) + (uint32_t)(e - 7) * 1024u, emaps + 0, full,
                                 r[0], r[1], r[2], r[3]);
                } else {
                    int r[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        const int q = min(4 * (e - 14) + u, 8), oc = q / 3, b = q - 3 * oc;
                        r[u] = (oc == 0 ? ti : (oc == 1 ? tj : tkk)) * nb + pick3(ob0, ob1, ob2, b);
                    }
                    gather4_load(sb + (uint32_t)offsetof(EpiStage, t1) + (uint32_t)(e - 14) * 128u, emaps + 1, full,
                                 r[0], r[1], r[2], r[3]);
                }
            }
            n++;
        }
        if (ok) {  // end marker
            const int stage = n % EPI_STAGES;
            if (n >= EPI_STAGES &&
                !mbar_wait(smem_u32(&bar_empty[stage]), (uint32_t)((n / EPI_STAGES - 1) & 1), &abort_sh)) {
                if (lane == 0) fail(&abort_sh, wv.err, DERR_TIMEOUT_EMPTY);
                ok = false;
            } else if (lane == 0) {
                if (pw == 0) meta[stage].kind = 0;
                mbar_arrive(smem_u32(&bar_full[stage]));
            }
        }
        if (!ok) {  // let the copies of the stages still in flight land (bounded)
            volatile int no_abort = 0;
            for (int m = n - EPI_STAGES < 0 ? 0 : n - EPI_STAGES; m < n; m++)
                mbar_wait(smem_u32(&bar_full[m % EPI_STAGES]), (uint32_t)((m / EPI_STAGES) & 1), &no_abort);
        }
        return;
    }

    // ---------------- compute warps ----------------
    // thread: fixed (b, c) = (lb, lc), a = la0 and la0 + 4 (the 512 element
    // orbits of a cube with three distinct blocks over 256 threads)
    const int lb = (tid >> 3) & 7, lc = tid & 7, la0 = tid >> 6;
    // cube offsets of the six orderings (abc, acb, bac, bca, cab, cba) in C0
    // and C1 (offd) and in C2 (offd2: its y index innermost)
    int offd[2][6], offd2[2][6];
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const int la = la0 + 4 * h;
        offd[h][0] = ucube_off(la, lb, lc);
        offd[h][1] = ucube_off(la, lc, lb);
        offd[h][2] = ucube_off(lb, la, lc);
        offd[h][3] = ucube_off(lb, lc, la);
        offd[h][4] = ucube_off(lc, la, lb);
        offd[h][5] = ucube_off(lc, lb, la);
        offd2[h][0] = ucube_off(la, lc, lb);
        offd2[h][1] = ucube_off(la, lb, lc);
        offd2[h][2] = ucube_off(lb, lc, la);
        offd2[h][3] = ucube_off(lb, la, lc);
        offd2[h][4] = ucube_off(lc, lb, la);
        offd2[h][5] = ucube_off(lc, la, lb);
    }
    for (int n = 0;; n++) {
        const int stage = n % EPI_STAGES;
        if (!mbar_wait(smem_u32(&bar_full[stage]), (uint32_t)((n / EPI_STAGES) & 1), &abort_sh)) {
            if (lane == 0) fail(&abort_sh, wv.err, DERR_TIMEOUT_FULL);
            return;
        }
        const int kind = meta[stage].kind;
        if (kind == 0) return;
        double *const out = meta[stage].out;
        const ff eijk = meta[stage].eijk;
        const int ob0 = meta[stage].ob[0], ob1 = meta[stage].ob[1], ob2 = meta[stage].ob[2];
        const int v = meta[stage].v;
        const EpiStage &S = stg[stage];
        ff A4 = {0.f, 0.f}, A5 = {0.f, 0.f};
        if (kind == 1) {
            // Distinct blocks: each thread takes element orbits, the six orderings
            // of one (a,b,c) with a in A, b in B, c in C.  Slot q holds the element
            // with indices ordered as q (slots 0..5 = abc, acb, bac, bca, cab, cba);
            // even slots 0,3,4, odd slots 1,2,5.  With E and O the sums of W over
            // the even and odd slots, Z at slot q is 6 w_q + 2E - 4O (q even) or
            // 6 w_q + 2O - 4E (q odd), and all six share one denominator.  What
            // depends only on b and c is read once for the thread's two orbits.
            const int A0 = ob0 * F8, B0 = ob1 * F8, C0 = ob2 * F8;
#define OVV(sl, pu, pw, lu, lw) S.ov[sl][pu][pw][(lu) * F8 + (lw)]
#define WQ(q, h) (S.cube[q][0][offd[h][q]] + S.cube[q][1][offd[h][q]] + S.cube[q][2][offd2[h][q]])
            const float tib = S.t1[0][1][lb], tic = S.t1[0][2][lc];
            const float tjb = S.t1[1][1][lb], tjc = S.t1[1][2][lc];
            const float tkb = S.t1[2][1][lb], tkc = S.t1[2][2][lc];
            const float jk_bc = OVV(0, 1, 2, lb, lc), jk_cb = OVV(0, 2, 1, lc, lb);
            const float ik_bc = OVV(1, 1, 2, lb, lc), ik_cb = OVV(1, 2, 1, lc, lb);
            const float ij_bc = OVV(2, 1, 2, lb, lc), ij_cb = OVV(2, 2, 1, lc, lb);
            const ff evb = {S.ev[1][lb].x, S.ev[1][lb].y}, evc = {S.ev[2][lc].x, S.ev[2][lc].y};
            const ff dbc = ff_sub(ff_sub(eijk, evb), evc);
            const bool bc_in = B0 + lb < v && C0 + lc < v;
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int la = la0 + 4 * h;
                if (!bc_in || A0 + la >= v) break;  // a grows with h
                const float w0 = WQ(0, h), w1 = WQ(1, h), w2 = WQ(2, h);
                const float w3 = WQ(3, h), w4 = WQ(4, h), w5 = WQ(5, h);
                // t1 of occupied i, j, k at a (at b and c above)
                const float tia = S.t1[0][0][la], tja = S.t1[1][0][la], tka = S.t1[2][0][la];
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
                const ff eva = {S.ev[0][la].x, S.ev[0][la].y};
                const ff r = ff_recip(ff_sub(dbc, eva));
                A4 = ff_add(A4, ff_mul(s4, r));
                A5 = ff_add(A5, ff_mul(s5, r));
            }
#undef WQ
#undef OVV
        } else {
            // blocks repeat: element by element over the distinct slots
            for (int s = 0; s < 6; s++) {
                if (meta[stage].smap[s] != s) continue;
                const int p0 = perm_pos(s, 0), p1 = perm_pos(s, 1), p2 = perm_pos(s, 2);
                const float *W[6];
#pragma unroll
                for (int q = 0; q < 6; q++) W[q] = S.cube[meta[stage].smap[comp[s][q]]][0];
#define WAT(q, x, y, z) (W[q][ucube_off(x, y, z)] + W[q][512 + ucube_off(x, y, z)] + W[q][1024 + ucube_off(x, z, y)])
                for (int l = tid; l < 512; l += NT) {
                    const int l0 = l >> 6, l1 = (l >> 3) & 7, l2 = l & 7;
                    const int x = pick3(ob0, ob1, ob2, p0) * F8 + l0, y = pick3(ob0, ob1, ob2, p1) * F8 + l1,
                              z = pick3(ob0, ob1, ob2, p2) * F8 + l2;
                    if (x >= v || y >= v || z >= v) continue;
                    const float w0 = WAT(0, l0, l1, l2);
                    // Z = 8 W(abc) - 4 (W(acb) + W(bac) + W(cba)) + 2 (W(bca) + W(cab))
                    const float zv = 8.f * w0 - 4.f * (WAT(1, l0, l2, l1) + WAT(2, l1, l0, l2) + WAT(5, l2, l1, l0)) +
                                     2.f * (WAT(3, l1, l2, l0) + WAT(4, l2, l0, l1));
                    const float yv = S.t1[0][p0][l0] * S.ov[0][p1][p2][l1 * F8 + l2] +
                                     S.t1[1][p1][l1] * S.ov[1][p0][p2][l0 * F8 + l2] +
                                     S.t1[2][p2][l2] * S.ov[2][p0][p1][l0 * F8 + l1];
                    const ff e0 = {S.ev[p0][l0].x, S.ev[p0][l0].y}, e1 = {S.ev[p1][l1].x, S.ev[p1][l1].y},
                             e2 = {S.ev[p2][l2].x, S.ev[p2][l2].y};
                    const ff r = ff_recip(ff_sub(ff_sub(ff_sub(eijk, e0), e1), e2));
                    A4 = ff_add(A4, ff_mul(zv * w0, r));
                    A5 = ff_add(A5, ff_mul(zv * yv, r));
                }
#undef WAT
            }
        }
        // the stage is free once every warp has read it
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_empty[stage]));

        // sum over the CTA: every thread's pair into red[n & 1], then warp
        // n % 8 sums the 256 pairs in a fixed order (32 per lane, then a
        // shuffle tree) and writes the orbit's FP64 partial
        const int rb = n & 1;
        if (n >= 2 && !mbar_wait(smem_u32(&bar_rempty[rb]), (uint32_t)(((n >> 1) - 1) & 1), &abort_sh)) {
            if (lane == 0) fail(&abort_sh, wv.err, DERR_TIMEOUT_EMPTY);
            return;
        }
        red[rb][tid] = make_float4(A4.hi, A4.lo, A5.hi, A5.lo);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&bar_rfull[rb]));
        if (warp == (n % EPI_CW)) {
            if (!mbar_wait(smem_u32(&bar_rfull[rb]), (uint32_t)((n >> 1) & 1), &abort_sh)) {
                if (lane == 0) fail(&abort_sh, wv.err, DERR_TIMEOUT_FULL);
                return;
            }
            float4 t = red[rb][lane];
            ff b4 = {t.x, t.y}, b5 = {t.z, t.w};
#pragma unroll
            for (int k = 1; k < NT / 32; k++) {
                t = red[rb][lane + 32 * k];
                b4 = ff_add(b4, ff{t.x, t.y});
                b5 = ff_add(b5, ff{t.z, t.w});
            }
            for (int off = 16; off > 0; off >>= 1) {
                const ff c4 = {__shfl_xor_sync(0xffffffffu, b4.hi, off), __shfl_xor_sync(0xffffffffu, b4.lo, off)};
                const ff c5 = {__shfl_xor_sync(0xffffffffu, b5.hi, off), __shfl_xor_sync(0xffffffffu, b5.lo, off)};
                b4 = ff_add(b4, c4);
                b5 = ff_add(b5, c5);
            }
            __syncwarp();
            if (lane == 0) {
                out[0] = ff_to_double(b4);
                out[1] = ff_to_double(b5);
                mbar_arrive(smem_u32(&bar_rempty[rb]));
            }
        }
    }
}

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

cudaError_t epi_fill_desc(InstDesc &d, std::string &err) {
    const uint64_t o = (uint64_t)d.dm.o, nb = (uint64_t)(d.dm.v + F8 - 1) / F8;
    if (!d.ovov || !d.t1 || !d.evf) {
        err = "mixed epilogue inputs missing";
        return cudaErrorInvalidValue;
    }
    if (o * o * nb * nb >= ((uint64_t)1 << 31)) {  // gather rows are 32-bit coordinates
        err = "o, v beyond the mixed epilogue's row range";
        return cudaErrorInvalidValue;
    }
    // row maps for 4-row gathers (box: one row, no swizzle): ovov 8x8 blocks
    // [p][q][X][Z] as rows of 64 floats, t1 as rows [p][X] of 8, eps_v (hi, lo)
    // as rows [X] of 16 floats
    struct M {
        void *base;
        uint64_t cols, rows;
        const char *what;
    } ms[3] = {{const_cast<void *>(d.ovov), 64, o * o * nb * nb, "ovov blocks"},
               {const_cast<void *>(d.t1), 8, o * nb, "t1 rows"},
               {const_cast<float2 *>(d.evf), 16, nb, "eps_v blocks"}};
    for (int k = 0; k < 3; k++) {
        const uint64_t dims[2] = {ms[k].cols, ms[k].rows}, strides[1] = {ms[k].cols * 4};
        const uint32_t box[2] = {(uint32_t)ms[k].cols, 1};
        if (!tcx::encode(&d.emaps[k], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, ms[k].base, dims, strides, box, err,
                         ms[k].what, CU_TENSOR_MAP_SWIZZLE_NONE))
            return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

cudaError_t epi_prepare() {
    static std::mutex mu;
    static bool done = false;
    std::lock_guard<std::mutex> lk(mu);
    if (done) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(epilogue_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EPI_SMEM);
    if (e == cudaSuccess) done = true;
    return e;
}

cudaError_t launch_epilogue(int prec, int sm_count, const Wave &w, cudaStream_t st) {
    if (w.n_epi <= 0) return cudaSuccess;
    if (w.n_epi > 0x7fffffff) return cudaErrorInvalidConfiguration;
    if (prec == TCORR_FP64) {
        const size_t smem = sizeof(double) * 6 * 8 * 8 * 9;
        epilogue_kernel<double, 8><<<(unsigned)w.n_epi, NT, smem, st>>>(w);
        return cudaGetLastError();
    }
    if (prec == TCORR_FP64_OZ) {
        const size_t smem = sizeof(dd) * 6 * 8 * 8 * 9;
        epilogue_kernel<dd, 8><<<(unsigned)w.n_epi, NT, smem, st>>>(w);
        return cudaGetLastError();
    }
    cudaError_t e = epi_prepare();
    if (e != cudaSuccess) return e;
    if (sm_count <= 0) {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    }
    const int64_t grid = std::min<int64_t>(w.n_epi, (int64_t)sm_count * EPI_CTAS);
    epilogue_f32_kernel<<<(unsigned)grid, EPI_THREADS, EPI_SMEM, st>>>(w);
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
