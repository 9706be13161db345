// RI-MP2 correlation energy (Sec. 2.1, Eqs. mp2_energy, eri_sym_decomp,
// e_orb_diff) on the FP64 pipe, declared in include/tcorr.h.
//
//   E_MP2 = - sum_{ij} sum_{ab} g_aibj (2 g_aibj - g_ajbi) / (e_a + e_b - e_i - e_j),
//   g_aibj = sum_gamma C^gamma_ai C^gamma_bj.
//
// Tasks are the occupied pairs i <= j (Eq. tasks_rimp2: o(o+1)/2 of them;
// the pair (j,i) has the same energy, so i < j counts twice).  For a pair,
// g[a][b] = (C_i^T C_j)[a][b] and the exchange integral g_ajbi = g[b][a].
// One CTA takes a pair and a tile pair A <= B of 48 virtual indices each and
// computes both G = C_i[A] C_j[B]^T (= g on A x B) and H = C_j[A] C_i[B]^T
// (= g on B x A, transposed), so every thread holds g_ab and g_ba for the same
// (a, b) and the energy terms are formed in registers: g never reaches
// memory.  On a diagonal tile pair H = G^T is taken from G through shared
// memory instead of being computed.  Over A x B and B x A together the Coulomb part is 2 (G^2 + H^2)/eps
// and the exchange part 2 G H / eps; a diagonal tile pair (A = B) covers its
// block once, G^2 and G H.  The GEMM is a register-tiled DFMA loop (3 x 3
// outputs of each of G and H per thread: rows a = ta + 16 r, three
// consecutive columns b = 3 tb + c; K = naux in chunks of 8 staged through
// double-buffered shared memory).  A warp's six b columns are consecutive, so
// on the ragged last tile the warps whose columns all lie past v issue no
// FMA: the tile padding costs no FP64-pipe time.  Per-CTA sums are reduced
// with a deterministic Kahan pass.
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "runtime.cuh"

using namespace tcorr;
using namespace tcorr::rt;

namespace {

constexpr int MT = 48;    // virtual tile edge
constexpr int MK = 8;     // K chunk
constexpr int MNT = 256;  // threads (16 x 16, 3 x 3 outputs of G and of H each)

__device__ __forceinline__ void kahan(double &s, double &c, double x) {
    const double y = x - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
}

struct Mp2Args {
    const double *Ct;        // [o][v][kp]: Ct[i][a][gamma] = C^gamma_ai, zero for gamma >= naux
    const double *eps_o, *eps_v;
    const int *pairs;        // [npair][2] (i <= j)
    const int *tiles;        // [ntp][2] (A <= B)
    int v, kp, ntp;
    double *partials;        // [items][2]: (E_J, E_K) of the item, pair weight applied
};

__global__ void __launch_bounds__(MNT, 2) mp2_pair_kernel(const Mp2Args p) {
    __shared__ __align__(16) double sm[2][4][MK][MT];  // [buffer][Ai, Bj, Aj, Bi][k][row]
    __shared__ double red[MNT / 32][2];
    const int item = blockIdx.x;
    const int pr = item / p.ntp, tp = item % p.ntp;
    const int i = p.pairs[2 * pr], j = p.pairs[2 * pr + 1];
    const int A = p.tiles[2 * tp], B = p.tiles[2 * tp + 1];
    const int tid = threadIdx.x, ta = tid & 15, tb = tid >> 4;
    const int v = p.v, kp = p.kp;
    const int64_t vk = (int64_t)v * kp;

    // loader: 4 blocks x 48 rows x 4 double2 = 768 double2, 3 per thread
    const double2 *src[3];
    bool ok[3];
    int dblk[3], drow[3], dpart[3];
#pragma unroll
    for (int it = 0; it < 3; it++) {
        const int idx = tid + it * MNT;
        const int blk = idx / (MT * 4), rem = idx % (MT * 4);
        const int row = rem >> 2, part = rem & 3;
        const int occ = (blk == 0 || blk == 3) ? i : j;
        const int tile = (blk == 0 || blk == 2) ? A : B;
        const int a = tile * MT + row;
        ok[it] = a < v;
        src[it] = reinterpret_cast<const double2 *>(p.Ct + occ * vk + (int64_t)(ok[it] ? a : 0) * kp) + part;
        dblk[it] = blk;
        drow[it] = row;
        dpart[it] = part;
    }
    double2 pre[3];
    auto fetch = [&](int k0) {
#pragma unroll
        for (int it = 0; it < 3; it++) pre[it] = ok[it] ? __ldg(src[it] + k0 / 2) : make_double2(0.0, 0.0);
    };
    auto stash = [&](int buf) {
#pragma unroll
        for (int it = 0; it < 3; it++) {
            sm[buf][dblk[it]][2 * dpart[it]][drow[it]] = pre[it].x;
            sm[buf][dblk[it]][2 * dpart[it] + 1][drow[it]] = pre[it].y;
        }
    };

    double G[3][3], H[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int c = 0; c < 3; c++) G[r][c] = H[r][c] = 0.0;

    const int nch = kp / MK;
    const bool diag = (A == B);  // H = G^T on a diagonal tile pair: computed from G below
    // warp w holds the columns b = 6 w .. 6 w + 5 of tile B
    const bool active = B * MT + 6 * (tid >> 5) < v;
    fetch(0);
    stash(0);
    __syncthreads();
    for (int ch = 0; ch < nch; ch++) {
        const int buf = ch & 1;
        if (ch + 1 < nch) fetch((ch + 1) * MK);
        if (!active) {
        } else if (!diag) {
#pragma unroll
            for (int k = 0; k < MK; k++) {
                double ai[3], bj[3], aj[3], bi[3];
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    ai[r] = sm[buf][0][k][ta + 16 * r];
                    aj[r] = sm[buf][2][k][ta + 16 * r];
                    bj[r] = sm[buf][1][k][3 * tb + r];
                    bi[r] = sm[buf][3][k][3 * tb + r];
                }
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        G[r][c] = fma(ai[r], bj[c], G[r][c]);
                        H[r][c] = fma(aj[r], bi[c], H[r][c]);
                    }
            }
        } else {
#pragma unroll
            for (int k = 0; k < MK; k++) {
                double ai[3], bj[3];
#pragma unroll
                for (int r = 0; r < 3; r++) {
                    ai[r] = sm[buf][0][k][ta + 16 * r];
                    bj[r] = sm[buf][1][k][3 * tb + r];
                }
#pragma unroll
                for (int r = 0; r < 3; r++)
#pragma unroll
                    for (int c = 0; c < 3; c++) G[r][c] = fma(ai[r], bj[c], G[r][c]);
            }
        }
        if (ch + 1 < nch) stash(buf ^ 1);
        __syncthreads();
    }
    if (diag) {  // H[a][b] = g[b][a] = G at (b, a), through shared memory (the K loop is done with it)
        double *Gs = &sm[0][0][0][0];  // 48 x 48 doubles (2 x 4 x 8 x 48 available)
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) Gs[(ta + 16 * r) * MT + 3 * tb + c] = G[r][c];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 3; r++)
#pragma unroll
            for (int c = 0; c < 3; c++) H[r][c] = Gs[(3 * tb + c) * MT + ta + 16 * r];
    }

    // energy terms of this thread's (a, b)
    const double eij = p.eps_o[i] + p.eps_o[j];
    double sj = 0.0, sk = 0.0;
#pragma unroll
    for (int r = 0; r < 3; r++) {
        const int a = A * MT + ta + 16 * r;
        if (a >= v) continue;
        const double ea = p.eps_v[a] - eij;
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int b = B * MT + 3 * tb + c;
            if (b >= v) continue;
            const double rd = 1.0 / (ea + p.eps_v[b]);
            const double g = G[r][c], h = H[r][c];
            if (A != B) {  // (a, b) in A x B and (b, a) in B x A
                sj -= 2.0 * (g * g + h * h) * rd;
                sk += 2.0 * g * h * rd;
            } else {       // the diagonal block is covered once
                sj -= 2.0 * g * g * rd;
                sk += g * h * rd;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        sj += __shfl_xor_sync(0xffffffffu, sj, off);
        sk += __shfl_xor_sync(0xffffffffu, sk, off);
    }
    if ((tid & 31) == 0) { red[tid >> 5][0] = sj; red[tid >> 5][1] = sk; }
    __syncthreads();
    if (tid == 0) {
        double tj = 0.0, cj = 0.0, tk = 0.0, ck = 0.0;
        for (int w = 0; w < MNT / 32; w++) { kahan(tj, cj, red[w][0]); kahan(tk, ck, red[w][1]); }
        const double w = (i == j) ? 1.0 : 2.0;  // the pair (j, i) has the same energy
        p.partials[2 * item] = w * (tj - cj);
        p.partials[2 * item + 1] = w * (tk - ck);
    }
}

// Single CTA: Kahan sums of the partials -> (E_J, E_K, E_J + E_K).
__global__ void __launch_bounds__(MNT) mp2_sum_kernel(const double *partials, int64_t n, double *out) {
    __shared__ double red[MNT][2];
    const int tid = threadIdx.x;
    double sj = 0.0, cj = 0.0, sk = 0.0, ck = 0.0;
    for (int64_t m = tid; m < n; m += MNT) {
        kahan(sj, cj, partials[2 * m]);
        kahan(sk, ck, partials[2 * m + 1]);
    }
    red[tid][0] = sj - cj;
    red[tid][1] = sk - ck;
    __syncthreads();
    for (int w = MNT / 2; w > 0; w >>= 1) {
        if (tid < w) { red[tid][0] += red[tid + w][0]; red[tid][1] += red[tid + w][1]; }
        __syncthreads();
    }
    if (tid == 0) {
        out[0] = red[0][0];
        out[1] = red[0][1];
        out[2] = red[0][0] + red[0][1];
    }
}

}  // namespace

struct tcorr_mp2_s {
    Exec ex;
    int o = 0, v = 0, naux = 0, kp = 0, nt = 0, ntp = 0;
    int64_t npair = 0, items = 0, nparts = 0;
    double *Ct = nullptr, *eps_o = nullptr, *eps_v = nullptr, *partials = nullptr, *d_out = nullptr;
    double *h_out = nullptr;
    int *pairs = nullptr, *tiles = nullptr;
    // split precision (TF32X3 / BF16X3): hi and lo planes of C^T, FP32 eps_v, tensor maps
    void *ct_hi = nullptr, *ct_lo = nullptr;
    float *eps_vf = nullptr;
    Mp2TcArgs tc{};
};

extern "C" {

tcorr_status tcorr_mp2_create(tcorr_mp2_t *out, int o, int v, int naux, const double *eps_occ,
                              const double *eps_vir, const double *C, const tcorr_opts *opts, void *stream) {
    g_create_error.clear();
    if (!out) {
        g_create_error = "out is NULL";
        return TCORR_EINVAL;
    }
    *out = nullptr;
    if (o < 1 || v < 1 || naux < 1 || !eps_occ || !eps_vir || !C) {
        g_create_error = "o, v, naux must be >= 1 and every array pointer non-NULL";
        return TCORR_EINVAL;
    }
    tcorr_opts op{};
    if (opts) op = *opts;
    {
        const tcorr_status st = check_opts(op, g_create_error);
        if (st != TCORR_OK) return st;
    }
    if (op.prec != TCORR_FP64 && op.prec != TCORR_TF32X3 && op.prec != TCORR_BF16X3) {
        g_create_error = "RI-MP2 is implemented in FP64, TF32X3 and BF16X3";
        return TCORR_EUNSUPPORTED;
    }
    if (o > 4096 || v > 65536 || naux > (1 << 20) || (int64_t)o * v * naux > ((int64_t)1 << 36)) {
        g_create_error = "sizes beyond the supported range";
        return TCORR_EUNSUPPORTED;
    }
    tcorr_mp2_s *h = new (std::nothrow) tcorr_mp2_s();
    if (!h) {
        g_create_error = "host allocation failed";
        return TCORR_ENOMEM;
    }
    Exec &ex = h->ex;
    // BF16 hi + lo operands on small problems: the split's residual (up to 2^-17
    // of each operand) averages below the 1e-6 bound only over enough terms.  Over
    // seeded shapes the BF16X3 error reached 1.3e-6 at 1.2e3 (pair, a, b, gamma)
    // terms and 3.5e-7 at 4e6, and stayed below 3.1e-7 above 1e7, while TF32X3
    // stayed within 2.9e-7 throughout: problems below 2^24 terms run on TF32
    // hi + lo operands (same four products, same kernel).
    if (op.prec == TCORR_BF16X3 && (double)o * (o + 1) / 2 * v * v * naux < TCORR_MP2_BF16_MIN_TERMS) op.prec = TCORR_TF32X3;
    try {
        init_exec(ex, op, stream);  // SM count; split precision only on the sm_103 tensor cores
        const bool split = op.prec != TCORR_FP64;
        const int tile = split ? MP2_TC_TILE : MT;
        h->o = o;
        h->v = v;
        h->naux = naux;
        // K padded to whole 64-byte chunks of the tensor-core path (16 TF32 / 32 BF16
        // values), or to the FP64 kernel's chunk
        h->kp = round_up(naux, split ? 32 : MK);
        h->nt = (v + tile - 1) / tile;
        h->ntp = h->nt * (h->nt + 1) / 2;
        h->npair = (int64_t)o * (o + 1) / 2;
        h->items = h->npair * h->ntp;
        if (h->items > 0x7fffffff) throw Fail{TCORR_EUNSUPPORTED, "too many work items"};
        // partials: one per item (FP64 kernel) or one per persistent CTA (tensor-core kernel)
        h->nparts = split ? std::min<int64_t>(ex.sm_count, h->items) : h->items;
        const size_t ct_bytes = (size_t)o * v * h->kp * elem_bytes(op.prec) * (split ? 2 : 1);  // hi + lo
        size_t free_b = 0, total_b = 0;
        CK(cudaMemGetInfo(&free_b, &total_b));
        const size_t need = ct_bytes + (size_t)h->nparts * 16 + (op.host_inputs ? (size_t)o * v * naux * 8 : 0) +
                            ((size_t)64 << 20);
        if (need > free_b)
            throw Fail{TCORR_ENOMEM, "footprint " + std::to_string(need) + " bytes exceeds free device memory"};
        if (split) {
            const size_t plane = ct_bytes / 2;
            dalloc(ex, h->ct_hi, plane);
            dalloc(ex, h->ct_lo, plane);
            dalloc(ex, h->eps_vf, (size_t)v * sizeof(float));
            alloc_common(ex);  // device error flag of the bounded waits
        } else {
            dalloc(ex, h->Ct, ct_bytes);
        }
        dalloc(ex, h->eps_o, (size_t)o * sizeof(double));
        dalloc(ex, h->eps_v, (size_t)v * sizeof(double));
        dalloc(ex, h->partials, (size_t)h->nparts * 2 * sizeof(double));
        dalloc(ex, h->d_out, 3 * sizeof(double));
        halloc(ex, h->h_out, 3 * sizeof(double));
        const bool host = op.host_inputs == 1;
        const cudaMemcpyKind kd = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        CK(cudaMemcpyAsync(h->eps_o, eps_occ, (size_t)o * sizeof(double), kd, ex.stream));
        CK(cudaMemcpyAsync(h->eps_v, eps_vir, (size_t)v * sizeof(double), kd, ex.stream));
        double *tmp = nullptr;
        const double *dC = device_view(ex, C, (size_t)o * v * naux, host, tmp);
        {   // Ct[i][a][gamma] = C[gamma][a][i], gamma padded to kp with zeros (split:
            // hi and lo planes in TF32 or BF16)
            Timer tm(ex, KC_PREP);
            const int kind = op.prec == TCORR_TF32X3 ? 1 : (op.prec == TCORR_BF16X3 ? 2 : 0);
            CK(launch_transpose_pad(kind, dC, split ? h->ct_hi : h->Ct, split ? h->ct_lo : nullptr, o, naux, h->kp,
                                    v, 1, (int64_t)v * o, o, (int64_t)v * h->kp, h->kp, 1.0, ex.stream));
            tm.stop();
        }
        free_tmp(ex, tmp, (size_t)o * v * naux);
        if (split) {  // FP32 copy of the virtual energies for the FP32 denominators
            std::vector<double> ev(v);
            CK(cudaMemcpyAsync(ev.data(), h->eps_v, (size_t)v * sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
            CK(cudaStreamSynchronize(ex.stream));
            std::vector<float> evf(ev.begin(), ev.end());
            CK(cudaMemcpy(h->eps_vf, evf.data(), (size_t)v * sizeof(float), cudaMemcpyHostToDevice));
        }
        std::vector<int> pr, tl;
        for (int i = 0; i < o; i++)
            for (int j = i; j < o; j++) { pr.push_back(i); pr.push_back(j); }
        for (int a = 0; a < h->nt; a++)
            for (int b = a; b < h->nt; b++) { tl.push_back(a); tl.push_back(b); }
        dalloc(ex, h->pairs, pr.size() * sizeof(int));
        dalloc(ex, h->tiles, tl.size() * sizeof(int));
        CK(cudaMemcpy(h->pairs, pr.data(), pr.size() * sizeof(int), cudaMemcpyHostToDevice));
        CK(cudaMemcpy(h->tiles, tl.data(), tl.size() * sizeof(int), cudaMemcpyHostToDevice));
        if (split) {
            Mp2TcArgs &a = h->tc;
            a.pairs = h->pairs;
            a.tiles = h->tiles;
            a.eps_o = h->eps_o;
            a.eps_v = h->eps_v;
            a.eps_vf = h->eps_vf;
            a.partials = h->partials;
            a.err = ex.err;
            a.v = v;
            a.ntp = h->ntp;
            a.items = h->items;
            std::string err;
            if (mp2_tc_fill(a, op.prec, h->ct_hi, h->ct_lo, o, v, h->kp, err) != cudaSuccess)
                throw Fail{TCORR_ECUDA, err};
        }
        CK(cudaStreamSynchronize(ex.stream));
        resolve_timers(ex);
    } catch (const Fail &f) {
        g_create_error = f.msg;
        cudaStreamSynchronize(ex.stream);
        cudaGetLastError();
        release(ex);
        delete h;
        return f.st;
    } catch (const std::bad_alloc &) {
        g_create_error = "host allocation failed";
        release(ex);
        delete h;
        return TCORR_ENOMEM;
    }
    *out = h;
    return TCORR_OK;
}

tcorr_status tcorr_mp2_energy(tcorr_mp2_t h, double *e_out) {
    if (!h) return TCORR_EINVAL;
    Exec &ex = h->ex;
    ex.last_error.clear();
    if (!e_out) {
        ex.last_error = "e_out is NULL";
        return TCORR_EINVAL;
    }
    try {
        {
            Timer tm(ex, KC_GEMM);
            if (ex.prec == TCORR_FP64) {
                Mp2Args a{h->Ct, h->eps_o, h->eps_v, h->pairs, h->tiles, h->v, h->kp, h->ntp, h->partials};
                mp2_pair_kernel<<<(unsigned)h->items, MNT, 0, ex.stream>>>(a);
                CK(cudaGetLastError());
            } else {
                CK(launch_mp2_tc(ex.prec, ex.sm_count, h->tc, ex.stream));
            }
            tm.stop();
        }
        {
            Timer tm(ex, KC_RED);
            mp2_sum_kernel<<<1, MNT, 0, ex.stream>>>(h->partials, h->nparts, h->d_out);
            CK(cudaGetLastError());
            tm.stop();
        }
        CK(cudaMemcpyAsync(h->h_out, h->d_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, ex.stream));
        CK(cudaStreamSynchronize(ex.stream));
        resolve_timers(ex);
        if (ex.prec != TCORR_FP64) check_err_flag(ex);
        for (int c = 0; c < 3; c++) e_out[c] = h->h_out[c];
    } catch (const Fail &f) {
        ex.last_error = f.msg;
        cudaStreamSynchronize(ex.stream);
        cudaGetLastError();
        return f.st;
    }
    return TCORR_OK;
}

tcorr_status tcorr_mp2_kernel_times(tcorr_mp2_t h, double *ms, int64_t *launches, int reset) {
    if (!h) return TCORR_EINVAL;
    for (int c = 0; c < KC_COUNT; c++) {
        if (ms) ms[c] = h->ex.k_ms[c];
        if (launches) launches[c] = h->ex.k_launch[c];
        if (reset) { h->ex.k_ms[c] = 0; h->ex.k_launch[c] = 0; }
    }
    return TCORR_OK;
}

int64_t tcorr_mp2_device_bytes(tcorr_mp2_t h) { return h ? (int64_t)h->ex.bytes : -1; }

const char *tcorr_mp2_last_error(tcorr_mp2_t h) {
    if (!h) return g_create_error.c_str();
    return h->ex.last_error.c_str();
}

tcorr_status tcorr_mp2_destroy(tcorr_mp2_t h) {
    if (!h) return TCORR_OK;
    cudaStreamSynchronize(h->ex.stream);
    release(h->ex);
    delete h;
    return TCORR_OK;
}

}  // extern "C"
