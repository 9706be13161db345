// Internal declarations shared by the CUDA translation units of libtcorr.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "../../include/tcorr.h"

namespace tcorr {

// Padded extents.  K-major operand rows are padded with zeros to a multiple
// of KPAD elements so that every row starts on a 64-byte boundary (TMA
// strides must be multiples of 16 bytes).  U rows (the innermost virtual
// index c) are padded to a multiple of UPAD.
constexpr int KPAD = 16;
constexpr int UPAD = 16;
__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Kernel classes timed when profiling is on.
enum { KC_PREP = 0, KC_GEMM = 1, KC_EPI = 2, KC_RED = 3, KC_COUNT = 4 };

// Device error flags (bit set by a kernel whose bounded wait expired).
enum { DERR_TIMEOUT_FULL = 1, DERR_TIMEOUT_EMPTY = 2, DERR_TIMEOUT_TMEM = 4, DERR_BAD_CONFIG = 8 };

struct Dims {
    int o, v;
    int dp;      // padded d extent (K of the vvvo segments)
    int lp;      // padded l extent (K of the ooov segments)
    int vc;      // padded c extent of U (FP64 layouts)
    int64_t ug;  // U elements per group tensor: room for either layout below
};
constexpr int UCUBE = 8;  // edge of the U cubes of the mixed paths (and of the epilogue's block orbits)
__host__ __device__ inline Dims make_dims(int o, int v) {
    const int vc = round_up(v, UPAD);
    const int64_t vp = round_up(v, UCUBE);
    const int64_t flat = (int64_t)v * v * vc, cubes = vp * vp * vp;
    return Dims{o, v, round_up(v, KPAD), round_up(o, KPAD), vc, flat > cubes ? flat : cubes};
}
// Offset of element (x, y, z) (each < 8) inside a U cube of the mixed paths.
// An XOR swizzle, linear over GF(2) in the bits of x, y, z, so that the six
// ways the epilogue walks a cube (a warp holds 4 consecutive values of one
// index and all 8 of another, the third fixed, in any assignment to x, y, z)
// each touch 32 distinct shared-memory banks.
__host__ __device__ inline int ucube_off(int x, int y, int z) {
    return (x << 6) | ((y ^ (x & 3)) << 3) | (z ^ y ^ (x & 4));
}

// Operand layouts built by the prep kernels (element type T = double, float
// (TF32 container) or __nv_bfloat16):
//   G  [q][x][y][d]  = (dx|yq)        = vvvo[d][x][y][q],  d < dp (zero pad)
//   T2K[q][x][y][l]  = t^{xy}_{ql}    = t2[q][l][x][y],    l < lp
//   T2R[s][p][a][d]  = t^{ad}_{sp}    = t2[s][p][a][d],    d < dp
//   AoN[q][s][a][l]  = -(as|lq)       = -ooov[l][q][s][a], l < lp
// With these, for the task (i,j,k) and its three groups
// (s;p,q) in {(i;j,k), (j;i,k), (k;i,j)}:
//   U^{s;p,q}[a][b][c] = sum_d T2R[s][p][a][d] G[q][b][c][d]
//                      + sum_d T2R[s][q][a][d] G[p][c][b][d]
//                      + sum_l AoN[q][s][a][l] T2K[p][b][c][l]
//                      + sum_l AoN[p][s][a][l] T2K[q][c][b][l]
// and W^{abc}_{ijk} = U^{i;j,k}[a][b][c] + U^{j;i,k}[b][a][c] + U^{k;i,j}[c][a][b].
// Storage of the three group tensors in the U scratch (3 ug elements per task):
//   FP64 paths: each U^g as [a][b][c] with rows of vc (read transposed by the
//   FP64 epilogue);
//   mixed paths: each group as its term of W in W's own index order,
//   C0[a][b][c] = U^0[a][b][c], C1[b][a][c] = U^1[a][b][c], C2[b][c][a] =
//   U^2[a][b][c], so that W[x][y][z] = C0[x][y][z] + C1[x][y][z] +
//   C2[x][y][z]; as cubes of 8^3 (nb = ceil(v / 8) per edge) with the three
//   groups interleaved: cube (X, Y, Z) of group g at (((X nb + Y) nb + Z) 3
//   + g) * 512 in the task's block, element (x, y, z) of it at
//   ucube_off(x, y, z) in C0 and C1 and at ucube_off(x, z, y) in C2 (so that
//   the contraction's stores, 8 consecutive c at fixed a and b, fill one
//   32-byte sector in every group).  An epilogue block orbit reads the three
//   terms of one W cube as one contiguous 6 KB copy.
struct Operands {
    void *G = nullptr, *T2K = nullptr, *T2R = nullptr, *AoN = nullptr;       // FP64 or hi part
    void *Glo = nullptr, *T2Klo = nullptr, *T2Rlo = nullptr, *AoNlo = nullptr;  // lo part (mixed)
};

// ---- work description shared by all kernels ------------------------------
// One problem ("instance") as the kernels see it.  Lives in device memory;
// a single handle has one, a batch one per problem.  Aligned like its tensor
// maps (alignof(CUtensorMap)), so an array of them keeps every map aligned.
struct InstDesc {
    CUtensorMap maps[6][2];   // tensor-core operand maps [G, G swapped, T2K, T2K swapped, T2R, AoN][hi, lo]
    CUtensorMap emaps[3];     // mixed epilogue row maps for 4-row gathers: ovov 8x8 blocks, t1 rows, eps_v blocks
    Dims dm;
    int pb, pc;               // tensor-core pair tile: pb values of b x pc values of c (pb * pc = 128)
    int kb;                   // K chunks per tensor-core accumulator block
    int kind;                 // split-precision operand type: 1 = TF32, 2 = BF16 hi + lo
    int pair;                 // tensor-core tiles on SM pairs (cta_group::2, M = 256)
    int nbt, nct, npass, kv, ko, brows;
    uint32_t stage_tx;        // TMA bytes per pipeline stage
    int norb;                 // epilogue block orbits per task (cube edge 8)
    const int *oz_e;          // FP64 emulation: device [2] scale exponents of the A and B operand sides
    const void *G, *T2K, *T2R, *AoN;  // FP64 operand layouts (FP64 W contractions)
    const double *eps_o, *eps_v;
    const void *t1, *ovov;    // epilogue copies: FP64, float-float pairs (FP64 emulation) or FP32
    const float2 *evf;        // eps_v as float-float (hi, lo): mixed (zero padded to 8 nb) and FP64 emulation
    const int *tasks;         // [ntask][3]
    const int *orbits;        // [norb][3]
    double *task_e;           // [ntask][2]
};
static_assert(alignof(InstDesc) % 64 == 0 && sizeof(InstDesc) % alignof(InstDesc) == 0,
              "tensor maps need (at least) 64-byte alignment in every array element");

// A contiguous run of one instance's tasks inside one launch ("wave").
// The prefix counts let every kernel find its segment by binary search.
struct Seg {
    int inst;                 // index into the InstDesc array
    int ntb;                  // tasks in the segment
    int64_t task0;            // first task of the segment in the instance's list
    int64_t u_off;            // element offset of the segment's U block: [ntb][3 ug]
    int64_t gemm0;            // prefix of W-contraction work units
    int64_t epi0;             // prefix of epilogue items (task, block orbit)
    int64_t red0;             // prefix of tasks
    int64_t part_off;         // double offset of the segment's orbit partials [ntb][norb][2]
};

// last segment s with key(s) <= x (segments sorted by key, key(0) = 0)
template <typename F>
__device__ __forceinline__ int seg_find(const Seg *segs, int nseg, int64_t x, F key) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (key(segs[mid]) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct Wave {
    const InstDesc *descs;    // device
    const Seg *segs;          // device, nseg entries
    int nseg;
    int64_t n_gemm, n_epi, n_red;  // totals of the three work kinds
    void *U;                  // device scratch
    double *partials;         // device scratch
    int *err;                 // device error flags
    int inject_stall;
    int tc_brows;             // tensor-core path: largest B tile (rows) of the wave's problems
};

// ---- prep.cu -------------------------------------------------------------
// out[b][c][r] = conv(scale * in[b*sb + r*sr + c*sc]) for r < R; zero for
// R <= r < Rp; out index b*ob + c*oc + r.  Writes hi (and lo when non-null).
// kind: 0 = FP64, 1 = TF32 hi+lo (float containers), 2 = BF16 hi+lo.
cudaError_t launch_transpose_pad(int kind, const double *in, void *out_hi, void *out_lo,
                                 int64_t B, int R, int Rp, int64_t C,
                                 int64_t sb, int64_t sr, int64_t sc,
                                 int64_t ob, int64_t oc, double scale, cudaStream_t st);
// FP32 epilogue inputs, zero padded to vp = 8 nb: t1 as rows [o][vp]; (p x | q z)
// as [p][q][X][Z][8][8] (8x8 blocks of x, z, each 256 contiguous bytes); eps_v
// as float-float pairs [vp]
cudaError_t launch_epilogue_f32_inputs(const double *t1, const double *ovov, const double *eps_v, float *t1f,
                                       float *ovf, float2 *evf, int o, int v, int vp, cudaStream_t st);
// FP64-emulation epilogue inputs: t1 [o][v] and ovov [o][v][o][v] converted in
// place to float-float (hi, lo) pairs; evf[x] = eps_v[x] as a pair, x < v
cudaError_t launch_epilogue_ff_inputs(double *t1, double *ovov, const double *eps_v, float2 *evf, int o, int v,
                                      cudaStream_t st);
// tasks[n] = (i, j, k): the sorted occupied triples i <= j <= k of o orbitals
// in lexicographic order; orbits[n] = (A, B, C): the sorted block triples
// A <= B <= C of nb virtual blocks, lexicographic
cudaError_t launch_build_tables(int o, int nb, int *tasks, int *orbits, cudaStream_t st);

// ---- gemm_f64.cu ---------------------------------------------------------
// FP64 work units of a segment: ntb * 3 * pair tiles * a tiles
int64_t f64_units_per_task(const Dims &dm);
cudaError_t launch_ugemm_f64(const Wave &w, cudaStream_t st);

// ---- epilogue.cu ---------------------------------------------------------
// sm_count: persistent CTAs of the mixed epilogue (2 per SM); unused by FP64
cudaError_t launch_epilogue(int prec, int sm_count, const Wave &w, cudaStream_t st);
// sets the mixed epilogue's shared-memory attribute once per process (before any capture)
cudaError_t epi_prepare();
// encodes d.emaps from d.ovov, d.t1, d.evf (the FP32 epilogue inputs) and d.dm
cudaError_t epi_fill_desc(InstDesc &d, std::string &err);
cudaError_t launch_task_reduce(const Wave &w, cudaStream_t st);
// One range of one problem's task energies, summed (Kahan) into out[0..2] =
// (E4, E5, E4 + E5) by launch_span_sums (one CTA per span).
struct SumSpan {
    const double *task_e;
    int64_t first, count;
    double *out;
};
cudaError_t launch_span_sums(const SumSpan *spans, int n, cudaStream_t st);
int epilogue_orbits(int v);   // block orbits per task (cube edge 8)

// ---- gemm_tc.cu ----------------------------------------------------------
bool tc_supported(int cc_major, int cc_minor);
// fills the tensor-core fields of d (maps, tile shape, derived counts) for
// the operand layouts in op; pb in {4, 8, 16}, kb in {1, 2}
// pair: tiles on SM pairs (2-CTA clusters, M = 256; B boxes of brows / 2 rows)
cudaError_t tc_fill_desc(InstDesc &d, int prec, const Operands &op, int pb, int kb, bool pair, std::string &err);
int64_t tc_units_per_task(const InstDesc &d);
// sets the kernel attributes once per process (call before any stream capture)
cudaError_t tc_prepare(int prec);

// ---- gemm_oz.cu (FP64 emulation on the BF16 tensor cores) -----------------------
int oz_slices();  // slice planes per operand
// *out = max over k of the bit pattern of |x[k]| (out zeroed by the caller)
cudaError_t launch_maxabs(const double *x, int64_t n, unsigned long long *out, cudaStream_t st);
// *m = max(*m, bit pattern of |x|) for a value known on the host
cudaError_t launch_seed_max(unsigned long long *m, double x, cudaStream_t st);
// e[0], e[1]: scale exponents of the A side (m[0] vvvo, m[1] t2) and B side (m[1] t2, m[2] ooov)
cudaError_t launch_oz_exponents(const unsigned long long *m, int *e, cudaStream_t st);
// out[p*plane + b*ob + c*oc + r] = slice p of sign * 2^-e[0] * in[b*sb + r*sr + c*sc], r < Rp (zero for r >= R)
cudaError_t launch_slice_pad(const double *in, void *out, int64_t B, int R, int Rp, int64_t C, int64_t sb,
                             int64_t sr, int64_t sc, int64_t ob, int64_t oc, int64_t plane, const int *e,
                             double sign, cudaStream_t st);
cudaError_t oz_fill_desc(InstDesc &d, const Operands &op, const int *exps, std::string &err);
int64_t oz_units_per_task(const InstDesc &d);
cudaError_t oz_prepare();
cudaError_t launch_ugemm_oz(int sm_count, const Wave &w, cudaStream_t st);
// pair: the SM-pair kernel (the wave's problems were described with pair = true)
cudaError_t launch_ugemm_tc(int prec, int sm_count, const Wave &w, cudaStream_t st, bool pair);

// ---- RI-MP2 in split precision on the tensor cores (mp2_tc.cu) ------------------
constexpr int MP2_TC_TILE = 128;  // virtual indices per tile (M = N of the MMAs)
struct Mp2TcArgs {
    CUtensorMap map[2];       // hi, lo planes of C^T as [o][v][kp] (K-major), box {chunk, 128, 1}
    const int *pairs;         // [npair][2], i <= j
    const int *tiles;         // [ntp][2], A <= B (tiles of MP2_TC_TILE)
    const double *eps_o, *eps_v;
    const float *eps_vf;      // eps_v rounded to FP32
    double *partials;         // [grid][2]: (E_J, E_K) of each CTA, pair weights applied
    int *err;                 // DERR_* flags of bounded waits that expired
    int v, nch, ntp;          // nch: K chunks of 64 bytes (set by mp2_tc_fill)
    int64_t items;            // npair * ntp
};
// Encodes the two operand maps of the planes hi / lo ([o][v][kp], TF32 or BF16)
// and sets a.nch; kp must be a multiple of the chunk (16 TF32, 32 BF16 values).
cudaError_t mp2_tc_fill(Mp2TcArgs &a, int prec, void *hi, void *lo, int o, int v, int kp, std::string &err);
// One persistent CTA per SM (at most items); writes min(sm_count, items) partial pairs.
cudaError_t launch_mp2_tc(int prec, int sm_count, const Mp2TcArgs &a, cudaStream_t st);

}  // namespace tcorr
