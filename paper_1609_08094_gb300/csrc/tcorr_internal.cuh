// Internal declarations shared by the CUDA translation units of libtcorr.
#pragma once

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
    int dp;   // padded d extent (K of the vvvo segments)
    int lp;   // padded l extent (K of the ooov segments)
    int vc;   // padded c extent of U
};

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
// Storage of the three group tensors in the U scratch ([ntb][3][v][v][vc]):
//   FP64 path: each U^g in its own [a][b][c] order (read transposed by the
//   FP64 epilogue);  mixed paths: slots 0 and 2 in their own [a][b][c] order,
//   slot 1 transposed to [b][a][c], so that W[x][y][z] = S0[x][y][z] +
//   S1[x][y][z] + S2[z][x][y] (S = stored slot).
struct Operands {
    void *G = nullptr, *T2K = nullptr, *T2R = nullptr, *AoN = nullptr;       // FP64 or hi part
    void *Glo = nullptr, *T2Klo = nullptr, *T2Rlo = nullptr, *AoNlo = nullptr;  // lo part (mixed)
};

struct Handle {
    Dims dm{};
    int prec = TCORR_FP64;
    int profile = 0;
    int inject_stall = 0;   // testing: make a tensor-core pipeline wait expire
    int batch = 1;          // tasks per batch
    int sm_count = 0, cc_major = 0, cc_minor = 0;
    cudaStream_t stream = nullptr;
    size_t bytes = 0;       // device bytes held

    Operands op;
    double *eps_o = nullptr, *eps_v = nullptr;  // FP64
    void *t1 = nullptr;      // FP64 or FP32 copy
    void *ovov = nullptr;    // FP64 or FP32 copy [o][v][o][v]
    float *dev_f = nullptr;  // FP32 block-relative virtual energies (mixed epilogue)

    int64_t ntask = 0;
    int *tasks = nullptr;          // device [ntask][3]
    double *task_e = nullptr;      // device [ntask][2] (E4, E5 share)
    void *U = nullptr;             // device scratch [batch][3][v][v][vc]
    size_t u_task_bytes = 0;
    int epi_te = 8;                // epilogue cube edge
    int norb = 0;                  // block orbits per task
    int *orbits = nullptr;         // device [norb][3]
    double *partials = nullptr;    // device [batch][norb][2]
    double *sums = nullptr;        // device [3]
    double *h_sums = nullptr;      // pinned host [3]
    int *err = nullptr;            // device error flags
    int *h_err = nullptr;          // pinned host copy

    // tcgen05 path
    void *tmaps = nullptr;   // host-side tensor maps (CUtensorMap array), built at create

    // profiling: event pairs recorded around launches, resolved after the
    // call's final stream synchronisation (no sync inside the launch sequence)
    struct Pending { int cls; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    double k_ms[KC_COUNT] = {0, 0, 0, 0};
    int64_t k_launch[KC_COUNT] = {0, 0, 0, 0};

    std::string last_error;
};

// ---- prep.cu -------------------------------------------------------------
// out[b][c][r] = conv(scale * in[b*sb + r*sr + c*sc]) for r < R; zero for
// R <= r < Rp; out index b*ob + c*oc + r.  Writes hi (and lo when non-null).
// kind: 0 = FP64, 1 = TF32 hi+lo (float containers), 2 = BF16 hi+lo.
cudaError_t launch_transpose_pad(int kind, const double *in, void *out_hi, void *out_lo,
                                 int64_t B, int R, int Rp, int64_t C,
                                 int64_t sb, int64_t sr, int64_t sc,
                                 int64_t ob, int64_t oc, double scale, cudaStream_t st);
// out[n] = (float) in[n]
cudaError_t launch_to_float(const double *in, float *out, int64_t n, cudaStream_t st);
// dev_f[x] = (float)(eps_v[block_start(x)] - eps_v[x]), block edge te
cudaError_t launch_block_deltas(const double *eps_v, float *dev_f, int v, int te, cudaStream_t st);

// ---- gemm_f64.cu ---------------------------------------------------------
struct GemmArgs {
    Dims dm;
    const int *tasks;     // device task list
    int64_t task0;        // first task index of the batch
    int ntb;              // tasks in the batch
    void *U;              // [ntb][3][v][v][vc]
};
cudaError_t launch_ugemm_f64(const Operands &op, const GemmArgs &ga, cudaStream_t st);

// ---- epilogue.cu ---------------------------------------------------------
struct EpiArgs {
    Dims dm;
    const int *tasks;
    int64_t task0;
    int ntb;
    const void *U;
    const double *eps_o, *eps_v;
    const void *t1, *ovov;
    const float *dev_f;
    const int *orbits;
    int norb;
    int te;
    double *partials;     // [ntb][norb][2]
    double *task_e;       // [ntask][2]
};
cudaError_t launch_epilogue(int prec, const EpiArgs &ea, cudaStream_t st);
cudaError_t launch_task_reduce(const EpiArgs &ea, cudaStream_t st);
cudaError_t launch_range_sum(const double *task_e, int64_t first, int64_t count,
                             double *sums, cudaStream_t st);

// ---- gemm_tc.cu ----------------------------------------------------------
bool tc_supported(int cc_major, int cc_minor);
cudaError_t tc_build_tensor_maps(Handle *h, std::string &err);
cudaError_t launch_ugemm_tc(Handle *h, const GemmArgs &ga, cudaStream_t st);

}  // namespace tcorr
