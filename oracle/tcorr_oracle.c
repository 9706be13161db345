/*
 * Plain FP64 CPU oracle for the closed-shell CCSD(T) triples correction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * What it computes (Sec. 2.2 of the paper, with the sign reading below):
 *
 *   X^{abc}_{ijk} = sum_d t^{ad}_{ij} (ck|bd) - sum_l t^{ab}_{il} (ck|lj)
 *       -- the bracket of Eq. (analytical_triples_ampl), Mulliken integrals;
 *   W^{abc}_{ijk} = X^{abc}_{ijk} + X^{acb}_{ikj} + X^{bac}_{jik}
 *                 + X^{bca}_{jki} + X^{cab}_{kij} + X^{cba}_{kji}
 *       -- the symmetriser P of Eq. (symm_operator);
 *   Y^{abc}_{ijk} = t^a_i (jb|kc) + t^b_j (ia|kc) + t^c_k (ia|jb)
 *       -- the bracket of Eq. (piecuch_z_coefficients);
 *   x~^{abc}_{ijk} = 4/3 x^{abc} - 2 x^{acb} + 2/3 x^{bca}
 *       -- Eq. (piecuch_tilde_quantity), ijk fixed;
 *   D^{abc}_{ijk} = e_i + e_j + e_k - e_a - e_b - e_c   (< 0)
 *   E[4] = sum_{ijk} sum_{abc} W~ W / D,   E[5] = sum_{ijk} sum_{abc} Y~ W / D
 *       -- Eqs. (piecuch_4th_order), (piecuch_5th_order) with t = W/D and
 *          z = Y/D.  Read literally, with epsilon = e_a+e_b+e_c-e_i-e_j-e_k
 *          as in Eq. (e_orb_diff), the two equations give -E(T); the
 *          denominator D above (occupied minus virtual) is the reading taken.
 *
 * Loop structure: the sum over all ordered (i,j,k) is organised as the
 * restricted loop over i <= j <= k of Sec. 3 (one task per sorted triple),
 * each task summing over the distinct orderings (p,q,r) of its three indices.
 * W is built once per task for (i,j,k) by the definition above; W for another
 * ordering is the same tensor with its virtual indices permuted, because P
 * sums over all simultaneous permutations of the pairs (a,i), (b,j), (c,k):
 *   W^{a_0 a_1 a_2}_{pqr} = W^{b_0 b_1 b_2}_{ijk},  b_{pos[n]} = a_n,
 * where (p,q,r) = (ijk[pos[0]], ijk[pos[1]], ijk[pos[2]]).  Y and D are
 * evaluated directly for each ordering.
 *
 * Inputs are row-major float64:
 *   eps_occ[o], eps_vir[v], t1[o][v] = t^a_i, t2[o][o][v][v] = t^{ab}_{ij},
 *   vvvo_slice[q] -> [v][v][v] with element [x][y][z] = (xy|zq)
 *                    (NULL allowed for occupied indices no task touches),
 *   ooov[o][o][o][v] = (ij|ka), ovov[o][v][o][v] = (ia|jb).
 * Outputs: e_out[t][0] = E[4] share, e_out[t][1] = E[5] share of task t.
 * Parallel over the virtual index a with OpenMP (Sec. 3 parallelises the
 * triple loop; here the tasks are evaluated one at a time so that the
 * v^3-sized intermediates exist once).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX2(a, b, n1) ((size_t)(a) * (size_t)(n1) + (size_t)(b))
#define IDX3(a, b, c, n1, n2) (((size_t)(a) * (size_t)(n1) + (size_t)(b)) * (size_t)(n2) + (size_t)(c))
#define IDX4(a, b, c, d, n1, n2, n3) \
    ((((size_t)(a) * (size_t)(n1) + (size_t)(b)) * (size_t)(n2) + (size_t)(c)) * (size_t)(n3) + (size_t)(d))

int oracle_version(void) { return 1; }

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* X(p,q,r)[x][y][z] = sum_d t2[p][q][x][d] (yd|zr) - sum_l t2[p][l][x][y] (lq|rz)
 * i.e. X^{xyz}_{pqr} with (zr|yd) = (yd|zr) and (zr|lq) = (lq|rz). */
static void build_x(int o, int v, int p, int q, int r, const double *t2,
                    const double *slice_r, const double *ooov, double *X) {
    const size_t vv = (size_t)v * v;
#pragma omp parallel for schedule(static)
    for (int x = 0; x < v; x++) {
        double *Xx = X + (size_t)x * vv;
        memset(Xx, 0, vv * sizeof(double));
        for (int y = 0; y < v; y++) {
            double *row = Xx + (size_t)y * v;
            for (int d = 0; d < v; d++) {
                const double t = t2[IDX4(p, q, x, d, o, v, v)];
                const double *s = slice_r + IDX3(y, d, 0, v, v);
                for (int z = 0; z < v; z++) row[z] += t * s[z];
            }
            for (int l = 0; l < o; l++) {
                const double t = t2[IDX4(p, l, x, y, o, v, v)];
                const double *g = ooov + IDX4(l, q, r, 0, o, o, v);
                for (int z = 0; z < v; z++) row[z] -= t * g[z];
            }
        }
    }
}

/* W[a][b][c] += X[...] read at the permutation of term n of P. */
static void add_term(int v, int n, const double *X, double *W) {
#pragma omp parallel for schedule(static)
    for (int a = 0; a < v; a++)
        for (int b = 0; b < v; b++)
            for (int c = 0; c < v; c++) {
                size_t src;
                switch (n) {
                case 0: src = IDX3(a, b, c, v, v); break; /* X^{abc}_{ijk} */
                case 1: src = IDX3(a, c, b, v, v); break; /* X^{acb}_{ikj} */
                case 2: src = IDX3(b, a, c, v, v); break; /* X^{bac}_{jik} */
                case 3: src = IDX3(b, c, a, v, v); break; /* X^{bca}_{jki} */
                case 4: src = IDX3(c, a, b, v, v); break; /* X^{cab}_{kij} */
                default: src = IDX3(c, b, a, v, v); break; /* X^{cba}_{kji} */
                }
                W[IDX3(a, b, c, v, v)] += X[src];
            }
}

/* W_{ijk} for all (a,b,c); X is scratch of v^3. */
static void build_w(int o, int v, int i, int j, int k, const double *t2,
                    const double *const *vvvo_slice, const double *ooov,
                    double *X, double *W) {
    const int occ[6][3] = {{i, j, k}, {i, k, j}, {j, i, k},
                           {j, k, i}, {k, i, j}, {k, j, i}};
    memset(W, 0, (size_t)v * v * v * sizeof(double));
    for (int n = 0; n < 6; n++) {
        build_x(o, v, occ[n][0], occ[n][1], occ[n][2], t2,
                vvvo_slice[occ[n][2]], ooov, X);
        add_term(v, n, X, W);
    }
}

int oracle_triple_energies(int o, int v, const double *eps_occ,
                           const double *eps_vir, const double *t1,
                           const double *t2, const double *const *vvvo_slice,
                           const double *ooov, const double *ovov,
                           long long ntask, const int *task, double *e_out,
                           int nthreads) {
    if (o < 1 || v < 1 || !eps_occ || !eps_vir || !t1 || !t2 || !vvvo_slice ||
        !ooov || !ovov || ntask < 0 || (ntask > 0 && (!task || !e_out)))
        return 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (long long t = 0; t < ntask; t++) {
        const int i = task[3 * t], j = task[3 * t + 1], k = task[3 * t + 2];
        if (i < 0 || k >= o || i > j || j > k) return 2;
        if (!vvvo_slice[i] || !vvvo_slice[j] || !vvvo_slice[k]) return 3;
    }
    const size_t v3 = (size_t)v * v * v;
    double *X = (double *)malloc(v3 * sizeof(double));
    double *W = (double *)malloc(v3 * sizeof(double));
    if (!X || !W) {
        free(X);
        free(W);
        return 4;
    }
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2},
                                    {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (long long t = 0; t < ntask; t++) {
        const int ijk[3] = {task[3 * t], task[3 * t + 1], task[3 * t + 2]};
        build_w(o, v, ijk[0], ijk[1], ijk[2], t2, vvvo_slice, ooov, X, W);
        double e4 = 0.0, e5 = 0.0;
        /* distinct orderings (p,q,r) of (i,j,k) */
        int seen[6][3];
        int nseen = 0;
        for (int s = 0; s < 6; s++) {
            const int *pos = perms[s];
            const int p = ijk[pos[0]], q = ijk[pos[1]], r = ijk[pos[2]];
            int dup = 0;
            for (int u = 0; u < nseen; u++)
                if (seen[u][0] == p && seen[u][1] == q && seen[u][2] == r) dup = 1;
            if (dup) continue;
            seen[nseen][0] = p;
            seen[nseen][1] = q;
            seen[nseen][2] = r;
            nseen++;
            /* inverse placement: W_{pqr}[a0][a1][a2] = W_{ijk}[b0][b1][b2],
               b[pos[n]] = a[n] */
            const double eocc = eps_occ[p] + eps_occ[q] + eps_occ[r];
            double s4 = 0.0, s5 = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s4, s5)
            for (int a = 0; a < v; a++) {
                for (int b = 0; b < v; b++) {
                    for (int c = 0; c < v; c++) {
                        int xa[3], bb[3];
                        double w[3], y[3];
                        /* the three index tuples (abc), (acb), (bca) */
                        const int tup[3][3] = {{a, b, c}, {a, c, b}, {b, c, a}};
                        for (int m = 0; m < 3; m++) {
                            xa[0] = tup[m][0];
                            xa[1] = tup[m][1];
                            xa[2] = tup[m][2];
                            bb[pos[0]] = xa[0];
                            bb[pos[1]] = xa[1];
                            bb[pos[2]] = xa[2];
                            w[m] = W[IDX3(bb[0], bb[1], bb[2], v, v)];
                            /* Y^{x0 x1 x2}_{pqr} */
                            y[m] = t1[IDX2(p, xa[0], v)] * ovov[IDX4(q, xa[1], r, xa[2], v, o, v)] +
                                   t1[IDX2(q, xa[1], v)] * ovov[IDX4(p, xa[0], r, xa[2], v, o, v)] +
                                   t1[IDX2(r, xa[2], v)] * ovov[IDX4(p, xa[0], q, xa[1], v, o, v)];
                        }
                        const double D = eocc - eps_vir[a] - eps_vir[b] - eps_vir[c];
                        const double wt = 4.0 / 3.0 * w[0] - 2.0 * w[1] + 2.0 / 3.0 * w[2];
                        const double yt = 4.0 / 3.0 * y[0] - 2.0 * y[1] + 2.0 / 3.0 * y[2];
                        s4 += wt * w[0] / D;
                        s5 += yt * w[0] / D;
                    }
                }
            }
            e4 += s4;
            e5 += s5;
        }
        e_out[2 * t] = e4;
        e_out[2 * t + 1] = e5;
    }
    free(X);
    free(W);
    return 0;
}
