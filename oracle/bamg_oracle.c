/*
 * FP64 CPU oracle of the monolithic block AMG V-cycle and its FGMRES wrapper.
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).
 * Sequential, unblocked, unfused: every loop follows the definition it cites,
 * so that a reader can check it against the paper by eye.  See
 * bamg_oracle.h for the interface and the list of paper passages.
 *
 * Compiled with -ffp-contract=off so that no multiply-add is fused and the
 * result is the same on every host.
 */
#include "bamg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* sparse block helpers                                                     */
/* ------------------------------------------------------------------------ */

/* y = A x with block CSR A (b x b blocks, row-major). */
int oracle_spmv(int n, int b, const int* row_ptr, const int* col_idx, const double* vals,
                const double* x, double* y) {
    for (int i = 0; i < n; ++i) {
        for (int r = 0; r < b; ++r) {
            double acc = 0.0;
            for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                const double* blk = vals + (size_t)k * b * b;
                int j = col_idx[k];
                for (int c = 0; c < b; ++c) acc += blk[r * b + c] * x[(size_t)j * b + c];
            }
            y[(size_t)i * b + r] = acc;
        }
    }
    return ORACLE_OK;
}

static double dot(size_t m, const double* a, const double* b) {
    double s = 0.0;
    for (size_t i = 0; i < m; ++i) s += a[i] * b[i];
    return s;
}

static double nrm2(size_t m, const double* a) { return sqrt(dot(m, a, a)); }

/* ------------------------------------------------------------------------ */
/* Aggregation (Sec. 4.3.1): the aggregates are a disjoint cover of the     */
/* nodes, each gives one coarse node, and they are formed greedily on the   */
/* node graph of the matrix.  The greedy rule (the paper names none):       */
/*  1. visit nodes in ascending index; a node whose neighbours and itself   */
/*     are all still free becomes a root, and it and its neighbours form    */
/*     one aggregate;                                                       */
/*  2. every node still free joins the aggregate of step 1 that holds most  */
/*     of its neighbours (ties: the smallest aggregate id), judged on the   */
/*     membership of step 1 only;                                           */
/*  3. aggregate ids are the ranks of the roots in ascending index.         */
/* After step 1 every free node has a neighbour in some aggregate (a node   */
/* with all neighbours free would have become a root), so step 2 places     */
/* every node.                                                              */
/* ------------------------------------------------------------------------ */
int oracle_aggregate(int n, const int* row_ptr, const int* col_idx, int* agg, int* is_root) {
    if (n < 0) return ORACLE_EINVAL;
    for (int i = 0; i < n; ++i) {
        agg[i] = -1;
        is_root[i] = 0;
    }
    int n_agg = 0;
    /* step 1: roots in ascending index; ids are assigned in the same order */
    for (int i = 0; i < n; ++i) {
        if (agg[i] != -1) continue;
        int all_free = 1;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int j = col_idx[k];
            if (j != i && agg[j] != -1) all_free = 0;
        }
        if (!all_free) continue;
        is_root[i] = 1;
        agg[i] = n_agg;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) agg[col_idx[k]] = n_agg;
        n_agg++;
    }
    /* step 2: attach the remaining nodes by step-1 membership */
    int* phase1 = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!phase1) return ORACLE_ENOMEM;
    memcpy(phase1, agg, sizeof(int) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        if (phase1[i] != -1) continue;
        int best = -1, best_count = 0;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int j = col_idx[k];
            if (j == i || phase1[j] == -1) continue;
            int a = phase1[j];
            int count = 0;
            for (int k2 = row_ptr[i]; k2 < row_ptr[i + 1]; ++k2) {
                int j2 = col_idx[k2];
                if (j2 != i && phase1[j2] == a) count++;
            }
            if (count > best_count || (count == best_count && a < best)) {
                best = a;
                best_count = count;
            }
        }
        agg[i] = best;
    }
    free(phase1);
    for (int i = 0; i < n; ++i)
        if (agg[i] < 0) return ORACLE_EINVAL; /* unreachable for a structurally symmetric graph */
    return n_agg;
}

/* ------------------------------------------------------------------------ */
/* Colouring for the multicolour node-block Gauss-Seidel sub-solve:         */
/* first fit in ascending index, colour(i) = smallest colour not used by a  */
/* neighbour j < i.                                                         */
/* ------------------------------------------------------------------------ */
int oracle_colour(int n, const int* row_ptr, const int* col_idx, int* colour) {
    int max_deg = 0;
    for (int i = 0; i < n; ++i)
        if (row_ptr[i + 1] - row_ptr[i] > max_deg) max_deg = row_ptr[i + 1] - row_ptr[i];
    int* used = (int*)calloc((size_t)max_deg + 2, sizeof(int));
    if (!used) return ORACLE_ENOMEM;
    int n_colours = 0;
    for (int i = 0; i < n; ++i) {
        for (int c = 0; c < max_deg + 2; ++c) used[c] = 0;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int j = col_idx[k];
            if (j < i && colour[j] <= max_deg) used[colour[j]] = 1;
        }
        int c = 0;
        while (used[c]) c++;
        colour[i] = c;
        if (c + 1 > n_colours) n_colours = c + 1;
    }
    free(used);
    return n_colours;
}

/* ------------------------------------------------------------------------ */
/* Galerkin coarse operator A_c = R A P (Sec. 3) with R = P^T and the       */
/* piecewise-constant P of Sec. 4.3.1: P[(i,d),(agg(i),d)] = 1 for every    */
/* dof d, the same aggregates for every field (cloned), so P is block       */
/* diagonal across fields (eq. blocktransfers).  Then                       */
/*   A_c[I,J] = sum_{i in I} sum_{j in J} A[i,j]      (b x b block sums),   */
/* pattern = every (agg(i), agg(j)) with (i,j) stored, columns ascending,   */
/* values accumulated with i ascending, then j in stored order.             */
/* ------------------------------------------------------------------------ */
static int cmp_int(const void* a, const void* b) {
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

/* members of every aggregate in ascending node order (counting sort) */
static int aggregate_members(int n, const int* agg, int nc, int** mptr_out, int** mem_out) {
    int* mptr = (int*)calloc((size_t)nc + 1, sizeof(int));
    int* mem = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int* fill = (int*)malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    if (!mptr || !mem || !fill) return ORACLE_ENOMEM;
    for (int i = 0; i < n; ++i) {
        if (agg[i] < 0 || agg[i] >= nc) return ORACLE_EINVAL;
        mptr[agg[i] + 1]++;
    }
    for (int I = 0; I < nc; ++I) mptr[I + 1] += mptr[I];
    for (int I = 0; I < nc; ++I) fill[I] = mptr[I];
    for (int i = 0; i < n; ++i) mem[fill[agg[i]]++] = i;
    free(fill);
    *mptr_out = mptr;
    *mem_out = mem;
    return ORACLE_OK;
}

int oracle_rap_tentative(int n, int b, const int* row_ptr, const int* col_idx, const double* vals,
                         const int* agg, int nc, int* rp_c, int* ci_c, double* vals_c) {
    if (!rp_c) return ORACLE_EINVAL;
    int *mptr, *mem;
    int st = aggregate_members(n, agg, nc, &mptr, &mem);
    if (st) return st;
    int* mark = (int*)malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    if (!mark) return ORACLE_ENOMEM;
    for (int J = 0; J < nc; ++J) mark[J] = -1;
    if (!ci_c) {
        /* pattern sizes: for every coarse row I the number of distinct agg(j) */
        rp_c[0] = 0;
        for (int I = 0; I < nc; ++I) {
            int count = 0;
            for (int q = mptr[I]; q < mptr[I + 1]; ++q) {
                int i = mem[q];
                for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                    int J = agg[col_idx[k]];
                    if (mark[J] != I) {
                        mark[J] = I;
                        count++;
                    }
                }
            }
            rp_c[I + 1] = rp_c[I] + count;
        }
        free(mark);
        free(mptr);
        free(mem);
        return rp_c[nc];
    }
    /* column indices: the distinct agg(j) of each coarse row, sorted */
    for (int I = 0; I < nc; ++I) {
        int fill = rp_c[I];
        for (int q = mptr[I]; q < mptr[I + 1]; ++q) {
            int i = mem[q];
            for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int J = agg[col_idx[k]];
                if (mark[J] != I) {
                    mark[J] = I;
                    ci_c[fill++] = J;
                }
            }
        }
        if (fill != rp_c[I + 1]) return ORACLE_EINVAL;
        qsort(ci_c + rp_c[I], (size_t)(rp_c[I + 1] - rp_c[I]), sizeof(int), cmp_int);
    }
    free(mark);
    free(mptr);
    free(mem);
    /* values: i ascending, then stored order of row i */
    const size_t bb = (size_t)b * b;
    memset(vals_c, 0, sizeof(double) * bb * (size_t)rp_c[nc]);
    for (int i = 0; i < n; ++i) {
        int I = agg[i];
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int J = agg[col_idx[k]];
            int p = -1;
            for (int q = rp_c[I]; q < rp_c[I + 1]; ++q)
                if (ci_c[q] == J) p = q;
            if (p < 0) return ORACLE_EINVAL;
            for (size_t e = 0; e < bb; ++e) vals_c[(size_t)p * bb + e] += vals[(size_t)k * bb + e];
        }
    }
    return rp_c[nc];
}

/* ------------------------------------------------------------------------ */
/* Smoothed transfers (beyond the paper, whose P is the tentative one).     */
/* Per field f the prolongator is P_f = (I - W_f D_ff^{-1} A_ff) P^_f:      */
/* the tentative P^_f of the cloned aggregates, smoothed by one damped      */
/* block-Jacobi step on the field-f block A_ff only, so P keeps the         */
/* field-block-diagonal form of eq. (blocktransfers).  Entry (i, J):        */
/*   P_f[i,J] = [J = agg(i)] I - w_{agg(i),f} D_ff,i^{-1} S_f[i,J],         */
/*   S_f[i,J] = sum over stored j of row i with agg(j) = J of A_ff[i,j]     */
/* (stored order), D^{-1} S summed over the inner index ascending.          */
/* ------------------------------------------------------------------------ */
static int field_layout(int b, const int* fmap, int* F, int* fb, int* fstart) {
    int nf = 0;
    if (b < 1 || b > ORACLE_MAX_B || fmap[0] != 0) return ORACLE_EINVAL;
    for (int d = 0; d < b; ++d) {
        if (d > 0 && fmap[d] != fmap[d - 1] && fmap[d] != fmap[d - 1] + 1) return ORACLE_EINVAL;
        if (fmap[d] + 1 > nf) nf = fmap[d] + 1;
    }
    if (b % nf) return ORACLE_EINVAL;
    *F = nf;
    *fb = b / nf;
    for (int f = 0; f < nf; ++f) {
        fstart[f] = -1;
        int cnt = 0;
        for (int d = 0; d < b; ++d)
            if (fmap[d] == f) {
                if (fstart[f] < 0) fstart[f] = d;
                cnt++;
            }
        if (cnt != *fb) return ORACLE_EINVAL;
    }
    return ORACLE_OK;
}

/* distinct values of list[0..m) ascending, in place; returns the count */
static int sort_unique(int* list, int m) {
    if (m == 0) return 0;
    qsort(list, (size_t)m, sizeof(int), cmp_int);
    int u = 1;
    for (int q = 1; q < m; ++q)
        if (list[q] != list[u - 1]) list[u++] = list[q];
    return u;
}

/* position of col in the ascending ci[k0..k1), or -1 */
static int find_pos(const int* ci, int k0, int k1, int col) {
    for (int k = k0; k < k1; ++k)
        if (ci[k] == col) return k;
    return -1;
}

/* ------------------------------------------------------------------------ */
/* ILU(0) of A_ff, the field-f part of the block matrix (Algorithm 1's       */
/* sub-solve in the paper's runs, Sec. 4.3.2 and Sec. 5.1).                   */
/* ------------------------------------------------------------------------ */
/* elimination position of node i: pos[i] (NULL: i) */
static inline int epos(const int* pos, int i) { return pos ? pos[i] : i; }

int oracle_ilu0_field_ordered(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                              const double* vals, int f, const int* pos, double* lu) {
    int F, fb, fstart[ORACLE_MAX_B];
    int st = field_layout(b, field_of_dof, &F, &fb, fstart);
    if (st) return st;
    if (f < 0 || f >= F || n < 0) return ORACLE_EINVAL;
    const int f0 = fstart[f];
    const size_t bb = (size_t)b * b, ff = (size_t)fb * fb;
    const int nnzb = row_ptr[n];
    int* node_at = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));  /* inverse of pos */
    if (!node_at) return ORACLE_ENOMEM;
    for (int i = 0; i < n; ++i) node_at[epos(pos, i)] = i;
    for (int k = 0; k < nnzb; ++k)
        for (int r = 0; r < fb; ++r)
            for (int c = 0; c < fb; ++c) lu[k * ff + r * fb + c] = vals[k * bb + (size_t)(f0 + r) * b + f0 + c];
    int order[64];  /* the blocks of a row by elimination position of their column */
    for (int e = 0; e < n; ++e) {
        const int i = node_at[e];
        const int k0 = row_ptr[i], len = row_ptr[i + 1] - k0;
        if (len > 64) {
            free(node_at);
            return ORACLE_EINVAL;
        }
        for (int t = 0; t < len; ++t) order[t] = k0 + t;
        for (int t = 1; t < len; ++t)  /* insertion sort by epos(col) */
            for (int u = t; u > 0 && epos(pos, col_idx[order[u]]) < epos(pos, col_idx[order[u - 1]]); --u) {
                const int tmp = order[u];
                order[u] = order[u - 1];
                order[u - 1] = tmp;
            }
        for (int r = 0; r < fb; ++r) {  /* scalar row p = pos(i)*fb + r in elimination order */
            const int p = e * fb + r;
            /* the entries q < p of row p in ascending elimination order */
            for (int t = 0; t < len; ++t) {
                const int k = order[t];
                const int j = col_idx[k];
                const int e2 = epos(pos, j);
                if (e2 > e) break;
                for (int c = 0; c < fb; ++c) {
                    const int q = e2 * fb + c;
                    if (q >= p) continue;
                    const int kd = find_pos(col_idx, row_ptr[j], row_ptr[j + 1], j);
                    if (kd < 0) {
                        free(node_at);
                        return ORACLE_EINVAL;
                    }
                    const double uqq = lu[kd * ff + c * fb + c];
                    if (uqq == 0.0) {
                        free(node_at);
                        return ORACLE_ESINGULAR_BLOCK;
                    }
                    const double l = lu[k * ff + r * fb + c] / uqq;
                    lu[k * ff + r * fb + c] = l;
                    /* a_pt -= l u_qt for t > q held by both rows p and q */
                    for (int k2 = row_ptr[i]; k2 < row_ptr[i + 1]; ++k2) {
                        const int j2 = col_idx[k2];
                        const int kq = find_pos(col_idx, row_ptr[j], row_ptr[j + 1], j2);
                        if (kq < 0) continue;
                        for (int c2 = 0; c2 < fb; ++c2) {
                            if (epos(pos, j2) * fb + c2 <= q) continue;
                            lu[k2 * ff + r * fb + c2] -= l * lu[kq * ff + c * fb + c2];
                        }
                    }
                }
            }
        }
    }
    free(node_at);
    return ORACLE_OK;
}

int oracle_ilu0_field(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                      const double* vals, int f, double* lu) {
    return oracle_ilu0_field_ordered(n, b, field_of_dof, row_ptr, col_idx, vals, f, NULL, lu);
}

int oracle_ilu0_solve_ordered(int n, int fb, const int* row_ptr, const int* col_idx, const int* pos,
                              const double* lu, const double* r, double* x) {
    const size_t ff = (size_t)fb * fb;
    int* node_at = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    if (!node_at) return ORACLE_ENOMEM;
    for (int i = 0; i < n; ++i) node_at[epos(pos, i)] = i;
    /* L y = r (unit lower), elimination order ascending; y in x */
    for (int e = 0; e < n; ++e) {
        const int i = node_at[e];
        for (int rr = 0; rr < fb; ++rr) {
            const int p = e * fb + rr;
            double s = r[(size_t)i * fb + rr];
            for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                const int j = col_idx[k];
                for (int c = 0; c < fb; ++c)
                    if (epos(pos, j) * fb + c < p) s -= lu[k * ff + rr * fb + c] * x[(size_t)j * fb + c];
            }
            x[(size_t)i * fb + rr] = s;
        }
    }
    /* U x = y, elimination order descending */
    for (int e = n - 1; e >= 0; --e) {
        const int i = node_at[e];
        for (int rr = fb - 1; rr >= 0; --rr) {
            const int p = e * fb + rr;
            double s = x[(size_t)i * fb + rr], d = 0.0;
            for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                const int j = col_idx[k];
                for (int c = 0; c < fb; ++c) {
                    const int t = epos(pos, j) * fb + c;
                    if (t > p) s -= lu[k * ff + rr * fb + c] * x[(size_t)j * fb + c];
                    else if (t == p) d = lu[k * ff + rr * fb + c];
                }
            }
            if (d == 0.0) {
                free(node_at);
                return ORACLE_ESINGULAR_BLOCK;
            }
            x[(size_t)i * fb + rr] = s / d;
        }
    }
    free(node_at);
    return ORACLE_OK;
}

int oracle_ilu0_solve(int n, int fb, const int* row_ptr, const int* col_idx, const double* lu,
                      const double* r, double* x) {
    return oracle_ilu0_solve_ordered(n, fb, row_ptr, col_idx, NULL, lu, r, x);
}

int oracle_prolongator(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                       const double* vals, const int* agg, int nc, const double* omega_p, int* p_rp,
                       int* p_ci, double* p_v) {
    int F, fb, fstart[ORACLE_MAX_B];
    if (!p_rp || field_layout(b, field_of_dof, &F, &fb, fstart)) return ORACLE_EINVAL;
    const size_t bb = (size_t)b * b, pbs = (size_t)F * fb * fb;
    int maxrow = 1;
    for (int i = 0; i < n; ++i)
        if (row_ptr[i + 1] - row_ptr[i] > maxrow) maxrow = row_ptr[i + 1] - row_ptr[i];
    int* cols = (int*)malloc(sizeof(int) * (size_t)maxrow);
    if (!cols) return ORACLE_ENOMEM;
    if (!p_ci) {
        p_rp[0] = 0;
        for (int i = 0; i < n; ++i) {
            int m = 0;
            for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                int J = agg[col_idx[k]];
                if (J < 0 || J >= nc) {
                    free(cols);
                    return ORACLE_EINVAL;
                }
                cols[m++] = J;
            }
            p_rp[i + 1] = p_rp[i] + sort_unique(cols, m);
        }
        free(cols);
        return p_rp[n];
    }
    for (int i = 0; i < n; ++i) {
        int m = 0;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) cols[m++] = agg[col_idx[k]];
        m = sort_unique(cols, m);
        if (m != p_rp[i + 1] - p_rp[i]) {
            free(cols);
            return ORACLE_EINVAL;
        }
        int kd = find_pos(col_idx, row_ptr[i], row_ptr[i + 1], i);
        if (kd < 0) {
            free(cols);
            return ORACLE_EINVAL;
        }
        for (int f = 0; f < F; ++f) {
            const int f0 = fstart[f];
            double dblk[ORACLE_MAX_B * ORACLE_MAX_B], dinv[ORACLE_MAX_B * ORACLE_MAX_B];
            for (int r = 0; r < fb; ++r)
                for (int c = 0; c < fb; ++c) dblk[r * fb + c] = vals[(size_t)kd * bb + (f0 + r) * b + (f0 + c)];
            int st = oracle_block_inverse(fb, dblk, dinv);
            if (st) {
                free(cols);
                return st;
            }
            const double w = omega_p[(size_t)agg[i] * F + f];
            for (int q = 0; q < m; ++q) {
                const int J = cols[q];
                const size_t K = (size_t)p_rp[i] + q;
                p_ci[K] = J;
                double S[ORACLE_MAX_B * ORACLE_MAX_B];
                for (int e = 0; e < fb * fb; ++e) S[e] = 0.0;
                for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
                    if (agg[col_idx[k]] != J) continue;
                    for (int r = 0; r < fb; ++r)
                        for (int c = 0; c < fb; ++c) S[r * fb + c] += vals[(size_t)k * bb + (f0 + r) * b + (f0 + c)];
                }
                double* P = p_v + K * pbs + (size_t)f * fb * fb;
                for (int r = 0; r < fb; ++r)
                    for (int c = 0; c < fb; ++c) {
                        double t = 0.0;
                        for (int s = 0; s < fb; ++s) t += dinv[r * fb + s] * S[s * fb + c];
                        const double delta = (J == agg[i] && r == c) ? 1.0 : 0.0;
                        P[r * fb + c] = delta - w * t;
                    }
            }
        }
    }
    free(cols);
    return p_rp[n];
}

/* ------------------------------------------------------------------------ */
/* Galerkin product A_c = P^T (A P) with a field-block-diagonal P (Sec. 3). */
/*   (A P)[i,J] = sum over stored j of row i (stored order), then over the  */
/*                stored J of P's row j, of A[i,j] P[j,J];                  */
/*   A_c[I,J]   = sum over fine i ascending with P[i,I] stored, then over   */
/*                the stored J of (AP)'s row i, of P[i,I]^T (A P)[i,J];     */
/* each block product sums over the inner field index ascending.  Patterns: */
/* the structural unions, ascending.                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
    int *rp, *ci;
    double* v;
} obsr;

/* A P: pattern and values (b x b blocks) */
static int product_ap(int n, int b, int F, int fb, const int* fstart, const int* fmap, const int* rp,
                      const int* ci, const double* vals, int nc, const int* p_rp, const int* p_ci,
                      const double* p_v, obsr* ap) {
    const size_t bb = (size_t)b * b, pbs = (size_t)F * fb * fb;
    (void)nc;
    int maxc = 1;
    for (int i = 0; i < n; ++i) {
        int c = 0;
        for (int k = rp[i]; k < rp[i + 1]; ++k) c += p_rp[ci[k] + 1] - p_rp[ci[k]];
        if (c > maxc) maxc = c;
    }
    int* cols = (int*)malloc(sizeof(int) * (size_t)maxc);
    ap->rp = (int*)malloc(sizeof(int) * (size_t)(n + 1));
    if (!cols || !ap->rp) return ORACLE_ENOMEM;
    ap->rp[0] = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            ap->ci = (int*)malloc(sizeof(int) * (size_t)(ap->rp[n] > 0 ? ap->rp[n] : 1));
            ap->v = (double*)calloc((size_t)(ap->rp[n] > 0 ? ap->rp[n] : 1) * bb, sizeof(double));
            if (!ap->ci || !ap->v) return ORACLE_ENOMEM;
        }
        for (int i = 0; i < n; ++i) {
            int m = 0;
            for (int k = rp[i]; k < rp[i + 1]; ++k)
                for (int q = p_rp[ci[k]]; q < p_rp[ci[k] + 1]; ++q) cols[m++] = p_ci[q];
            m = sort_unique(cols, m);
            if (pass == 0) {
                ap->rp[i + 1] = ap->rp[i] + m;
                continue;
            }
            memcpy(ap->ci + ap->rp[i], cols, sizeof(int) * (size_t)m);
            for (int k = rp[i]; k < rp[i + 1]; ++k) {
                const int j = ci[k];
                const double* A = vals + (size_t)k * bb;
                for (int q = p_rp[j]; q < p_rp[j + 1]; ++q) {
                    const int pos = find_pos(ap->ci, ap->rp[i], ap->rp[i + 1], p_ci[q]);
                    double* out = ap->v + (size_t)pos * bb;
                    const double* P = p_v + (size_t)q * pbs;
                    for (int r = 0; r < b; ++r)
                        for (int c = 0; c < b; ++c) {
                            const int g = fmap[c], g0 = fstart[g], cl = c - g0;
                            double t = 0.0;
                            for (int s = 0; s < fb; ++s) t += A[r * b + g0 + s] * P[(size_t)g * fb * fb + s * fb + cl];
                            out[r * b + c] += t;
                        }
                }
            }
        }
    }
    free(cols);
    return ORACLE_OK;
}

/* transpose pattern of P: for every coarse I the positions q of P's stored
 * (i, I), i ascending */
static int transpose_p(int n, int nc, const int* p_rp, const int* p_ci, int** r_rp, int** r_q, int** r_i) {
    int* rr = (int*)calloc((size_t)nc + 1, sizeof(int));
    const int nnz = p_rp[n];
    int* rq = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    int* ri = (int*)malloc(sizeof(int) * (size_t)(nnz > 0 ? nnz : 1));
    int* fill = (int*)malloc(sizeof(int) * (size_t)(nc > 0 ? nc : 1));
    if (!rr || !rq || !ri || !fill) return ORACLE_ENOMEM;
    for (int q = 0; q < nnz; ++q) rr[p_ci[q] + 1]++;
    for (int I = 0; I < nc; ++I) rr[I + 1] += rr[I];
    for (int I = 0; I < nc; ++I) fill[I] = rr[I];
    for (int i = 0; i < n; ++i)
        for (int q = p_rp[i]; q < p_rp[i + 1]; ++q) {
            const int p = fill[p_ci[q]]++;
            rq[p] = q;
            ri[p] = i;
        }
    free(fill);
    *r_rp = rr;
    *r_q = rq;
    *r_i = ri;
    return ORACLE_OK;
}

int oracle_rap_general(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                       const double* vals, int nc, const int* p_rp, const int* p_ci, const double* p_v,
                       int* rp_c, int* ci_c, double* vals_c) {
    int F, fb, fstart[ORACLE_MAX_B];
    if (!rp_c || field_layout(b, field_of_dof, &F, &fb, fstart)) return ORACLE_EINVAL;
    const size_t bb = (size_t)b * b, pbs = (size_t)F * fb * fb;
    obsr ap = {0, 0, 0};
    int st = product_ap(n, b, F, fb, fstart, field_of_dof, row_ptr, col_idx, vals, nc, p_rp, p_ci, p_v, &ap);
    if (st) return st;
    int *r_rp, *r_q, *r_i;
    st = transpose_p(n, nc, p_rp, p_ci, &r_rp, &r_q, &r_i);
    if (st) return st;
    int maxc = 1;
    for (int I = 0; I < nc; ++I) {
        int c = 0;
        for (int t = r_rp[I]; t < r_rp[I + 1]; ++t) c += ap.rp[r_i[t] + 1] - ap.rp[r_i[t]];
        if (c > maxc) maxc = c;
    }
    int* cols = (int*)malloc(sizeof(int) * (size_t)maxc);
    if (!cols) return ORACLE_ENOMEM;
    if (!ci_c) rp_c[0] = 0;
    else memset(vals_c, 0, sizeof(double) * bb * (size_t)rp_c[nc]);
    for (int I = 0; I < nc && st == ORACLE_OK; ++I) {
        int m = 0;
        for (int t = r_rp[I]; t < r_rp[I + 1]; ++t)
            for (int a = ap.rp[r_i[t]]; a < ap.rp[r_i[t] + 1]; ++a) cols[m++] = ap.ci[a];
        m = sort_unique(cols, m);
        if (!ci_c) {
            rp_c[I + 1] = rp_c[I] + m;
            continue;
        }
        if (m != rp_c[I + 1] - rp_c[I]) {
            st = ORACLE_EINVAL;
            break;
        }
        memcpy(ci_c + rp_c[I], cols, sizeof(int) * (size_t)m);
        for (int t = r_rp[I]; t < r_rp[I + 1]; ++t) {
            const int i = r_i[t];
            const double* P = p_v + (size_t)r_q[t] * pbs;
            for (int a = ap.rp[i]; a < ap.rp[i + 1]; ++a) {
                const int pos = find_pos(ci_c, rp_c[I], rp_c[I + 1], ap.ci[a]);
                double* out = vals_c + (size_t)pos * bb;
                const double* X = ap.v + (size_t)a * bb;
                for (int r = 0; r < b; ++r) {
                    const int f = field_of_dof[r], f0 = fstart[f], rl = r - f0;
                    for (int c = 0; c < b; ++c) {
                        double s = 0.0;
                        for (int u = 0; u < fb; ++u) s += P[(size_t)f * fb * fb + u * fb + rl] * X[(f0 + u) * b + c];
                        out[r * b + c] += s;
                    }
                }
            }
        }
    }
    free(cols);
    free(ap.rp);
    free(ap.ci);
    free(ap.v);
    free(r_rp);
    free(r_q);
    free(r_i);
    if (st) return st;
    return rp_c[nc];
}

/* ------------------------------------------------------------------------ */
/* Small dense inverses (node-block diagonal of one field): Gauss-Jordan    */
/* elimination with partial pivoting on [a | I].                            */
/* ------------------------------------------------------------------------ */
int oracle_block_inverse(int m, const double* a, double* ainv) {
    double w[ORACLE_MAX_B * ORACLE_MAX_B], v[ORACLE_MAX_B * ORACLE_MAX_B];
    if (m < 1 || m > ORACLE_MAX_B) return ORACLE_EINVAL;
    double norm = 0.0;
    for (int r = 0; r < m; ++r) {
        double s = 0.0;
        for (int c = 0; c < m; ++c) s += fabs(a[r * m + c]);
        if (s > norm) norm = s;
    }
    for (int e = 0; e < m * m; ++e) w[e] = a[e];
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) v[r * m + c] = (r == c) ? 1.0 : 0.0;
    for (int k = 0; k < m; ++k) {
        int p = k;
        for (int r = k + 1; r < m; ++r)
            if (fabs(w[r * m + k]) > fabs(w[p * m + k])) p = r;
        if (!(fabs(w[p * m + k]) >= 1e-14 * norm) || norm == 0.0) return ORACLE_ESINGULAR_BLOCK;
        if (p != k) {
            for (int c = 0; c < m; ++c) {
                double t = w[k * m + c];
                w[k * m + c] = w[p * m + c];
                w[p * m + c] = t;
                t = v[k * m + c];
                v[k * m + c] = v[p * m + c];
                v[p * m + c] = t;
            }
        }
        double piv = w[k * m + k];
        for (int c = 0; c < m; ++c) {
            w[k * m + c] /= piv;
            v[k * m + c] /= piv;
        }
        for (int r = 0; r < m; ++r) {
            if (r == k) continue;
            double f = w[r * m + k];
            for (int c = 0; c < m; ++c) {
                w[r * m + c] -= f * w[k * m + c];
                v[r * m + c] -= f * v[k * m + c];
            }
        }
    }
    for (int e = 0; e < m * m; ++e) ainv[e] = v[e];
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense LU with partial pivoting for the direct solve on the coarsest      */
/* level (Fig. 1, "u <- A^{-1} b" at l_max).                                */
/* ------------------------------------------------------------------------ */
int oracle_lu_factor(int n, double* a, int* piv) {
    double norm = 0.0;
    for (int r = 0; r < n; ++r) {
        double s = 0.0;
        for (int c = 0; c < n; ++c) s += fabs(a[(size_t)r * n + c]);
        if (s > norm) norm = s;
    }
    for (int k = 0; k < n; ++k) {
        int p = k;
        for (int r = k + 1; r < n; ++r)
            if (fabs(a[(size_t)r * n + k]) > fabs(a[(size_t)p * n + k])) p = r;
        if (!(fabs(a[(size_t)p * n + k]) >= 1e-14 * norm) || norm == 0.0)
            return ORACLE_ESINGULAR_COARSE;
        piv[k] = p;
        if (p != k)
            for (int c = 0; c < n; ++c) {
                double t = a[(size_t)k * n + c];
                a[(size_t)k * n + c] = a[(size_t)p * n + c];
                a[(size_t)p * n + c] = t;
            }
        for (int r = k + 1; r < n; ++r) {
            double l = a[(size_t)r * n + k] / a[(size_t)k * n + k];
            a[(size_t)r * n + k] = l;
            for (int c = k + 1; c < n; ++c) a[(size_t)r * n + c] -= l * a[(size_t)k * n + c];
        }
    }
    return ORACLE_OK;
}

int oracle_lu_solve(int n, const double* lu, const int* piv, const double* rhs, double* x) {
    for (int i = 0; i < n; ++i) x[i] = rhs[i];
    for (int k = 0; k < n; ++k) {
        double t = x[k];
        x[k] = x[piv[k]];
        x[piv[k]] = t;
    }
    for (int i = 0; i < n; ++i) { /* L y = P rhs, unit lower */
        double s = x[i];
        for (int c = 0; c < i; ++c) s -= lu[(size_t)i * n + c] * x[c];
        x[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) { /* U x = y */
        double s = x[i];
        for (int c = i + 1; c < n; ++c) s -= lu[(size_t)i * n + c] * x[c];
        x[i] = s / lu[(size_t)i * n + i];
    }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Hierarchy                                                                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n, nnzb, n_colours, n_agg;
    int *row_ptr, *col_idx;
    double* vals;
    int* agg;       /* [n] aggregate of each node (levels above the coarsest) */
    int* colour;    /* [n] */
    double* dinv;   /* [n][F][fb*fb] */
    double* ilu[ORACLE_MAX_B]; /* sub_ilu: ILU(0) factors of A_ff per field, [nnzb][fb][fb] */
    int* ilu_pos;   /* sub_ilu = 2: elimination position of every node (colour, then index) */
    double *u, *rhs, *res; /* work vectors of n*b */
    double* omega_s; /* [n][F] smoother damping of every node and field */
    double* omega_p; /* [n_agg][F] prolongator smoothing weights (smooth_p) */
    /* smoothed prolongator (smooth_p): field-block-diagonal blocks, and the
     * positions of its entries by coarse column (i ascending) for R = P^T */
    int smoothed; /* this level's P is the smoothed one */
    int p_nnz;
    int *p_rp, *p_ci;
    double* p_v;
    int *r_rp, *r_q, *r_i;
    /* fields on disjoint node sets (n_node_fields > 1) */
    int* foff; /* [NF+1] nodes of field g: foff[g] <= i < foff[g+1] */
    int* coff; /* [NF+1] colours of field g: coff[g] <= c < coff[g+1] */
    /* sub_schwarz: subdomains, one per aggregate and field */
    int n_sd, sd_max_m;
    int* sd_field;         /* [n_sd] field of the subdomain */
    int* sd_ptr;           /* [n_sd+1] into sd_nodes, sd_own */
    int* sd_nodes;         /* nodes of each subdomain, ascending */
    unsigned char* sd_own; /* 1: the node belongs to the subdomain's aggregate */
    size_t* sd_lu_off;     /* [n_sd+1] dense LU factors of A_I in sd_lu */
    double* sd_lu;
    int* sd_piv;           /* pivots of subdomain I at sd_ptr[I] * (dofs per node) */
    /* sub_ilu with node fields: A_gg of every field as its own block matrix
     * (nodes renumbered from 0), its elimination positions, factors in ilu[g] */
    int* nf_rp[ORACLE_MAX_NODE_FIELDS];
    int* nf_ci[ORACLE_MAX_NODE_FIELDS];
    int* nf_pos[ORACLE_MAX_NODE_FIELDS];
} olevel;

struct oracle_hier {
    int nlev, b, F, fb;
    int NF; /* fields on disjoint node sets (1: co-located fields only) */
    int field_of_dof[ORACLE_MAX_B];
    int fstart[ORACLE_MAX_B]; /* first dof of each field inside a node */
    int fsize[ORACLE_MAX_B];  /* dofs of each field (fb = the largest) */
    int doff[ORACLE_MAX_B];   /* offset of field f's inverse block in a node's dinv entries */
    int dstride;              /* dinv entries per node: sum over the fields of fsize^2 */
    oracle_params p;
    olevel lev[ORACLE_MAX_LEVELS];
    double* lu; /* coarsest level, dense LU */
    int* piv;
    int nc_dense;
    double* xt; /* smoother scratch: x~ and r_f of one field, n*fb each */
    double* rf;
};

static void level_free(olevel* L) {
    free(L->row_ptr);
    free(L->col_idx);
    free(L->vals);
    free(L->agg);
    free(L->colour);
    free(L->dinv);
    free(L->u);
    free(L->rhs);
    free(L->res);
    free(L->omega_s);
    free(L->omega_p);
    free(L->p_rp);
    free(L->p_ci);
    free(L->p_v);
    free(L->r_rp);
    free(L->r_q);
    free(L->r_i);
    for (int f = 0; f < ORACLE_MAX_B; ++f) free(L->ilu[f]);
    free(L->ilu_pos);
    free(L->foff);
    free(L->coff);
    free(L->sd_field);
    free(L->sd_ptr);
    free(L->sd_nodes);
    free(L->sd_own);
    free(L->sd_lu_off);
    free(L->sd_lu);
    free(L->sd_piv);
    for (int g = 0; g < ORACLE_MAX_NODE_FIELDS; ++g) {
        free(L->nf_rp[g]);
        free(L->nf_ci[g]);
        free(L->nf_pos[g]);
    }
}

/* ------------------------------------------------------------------------ */
/* Fields on disjoint node sets (Sec. 4.3.1; Sec. 5, mixed elements).       */
/* The graph of A_gg: the nodes of field g renumbered from 0 and the stored */
/* blocks between two of them (columns keep their ascending order).         */
/* ------------------------------------------------------------------------ */
static int field_subgraph(const olevel* L, int g, int** rp_out, int** ci_out) {
    const int o0 = L->foff[g], o1 = L->foff[g + 1], m = o1 - o0;
    int* rp = (int*)malloc(sizeof(int) * (size_t)(m + 1));
    int* ci = (int*)malloc(sizeof(int) * (size_t)(L->row_ptr[o1] - L->row_ptr[o0] + 1));
    if (!rp || !ci) {
        free(rp);
        free(ci);
        return ORACLE_ENOMEM;
    }
    int e = 0;
    rp[0] = 0;
    for (int i = o0; i < o1; ++i) {
        for (int k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) {
            const int j = L->col_idx[k];
            if (j >= o0 && j < o1) ci[e++] = j - o0;
        }
        rp[i - o0 + 1] = e;
    }
    *rp_out = rp;
    *ci_out = ci;
    return ORACLE_OK;
}

/* separate aggregation of every field on the graph of its own diagonal
 * block; field g's aggregate ids follow those of fields 0..g-1, so the
 * piecewise-constant P = diag(P_0, P_1, ...) (eq. blocktransfers) and the
 * coarse field ranges are foff_c[g] = the aggregates of fields before g.
 * Returns the total number of aggregates. */
static int aggregate_node_fields(const oracle_hier* h, const olevel* L, int* agg, int* foff_c) {
    int base = 0;
    foff_c[0] = 0;
    for (int g = 0; g < h->NF; ++g) {
        const int o0 = L->foff[g], m = L->foff[g + 1] - o0;
        int *rp = NULL, *ci = NULL;
        int st = field_subgraph(L, g, &rp, &ci);
        if (st) return st;
        int* is_root = (int*)malloc(sizeof(int) * (size_t)m);
        int nc = is_root ? oracle_aggregate(m, rp, ci, agg + o0, is_root) : ORACLE_ENOMEM;
        free(is_root);
        free(rp);
        free(ci);
        if (nc < 0) return nc;
        for (int i = 0; i < m; ++i) agg[o0 + i] += base;
        base += nc;
        foff_c[g + 1] = base;
    }
    return base;
}

/* ILU(0) of every node field's diagonal block A_gg (Algorithm 1's sub-solve,
 * Sec. 4.3.2), as a block matrix of its own: the field's nodes renumbered from
 * 0, the stored blocks between them; sub_ilu = 2 eliminates the field's nodes
 * in (colour, index) order */
static int ilu_node_fields(oracle_hier* h, olevel* L) {
    const int b = h->b;
    const size_t bb = (size_t)b * b;
    int zeros[ORACLE_MAX_B] = {0};
    for (int g = 0; g < h->NF; ++g) {
        const int o0 = L->foff[g], o1 = L->foff[g + 1], m = o1 - o0;
        int st = field_subgraph(L, g, &L->nf_rp[g], &L->nf_ci[g]);
        if (st) return st;
        const int nnz = L->nf_rp[g][m];
        double* v = (double*)malloc(sizeof(double) * bb * (size_t)(nnz > 0 ? nnz : 1));
        L->ilu[g] = (double*)malloc(sizeof(double) * bb * (size_t)(nnz > 0 ? nnz : 1));
        if (!v || !L->ilu[g]) {
            free(v);
            return ORACLE_ENOMEM;
        }
        int e = 0;
        for (int i = o0; i < o1; ++i)
            for (int k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k)
                if (L->col_idx[k] >= o0 && L->col_idx[k] < o1) memcpy(v + (size_t)(e++) * bb, L->vals + (size_t)k * bb,
                                                                      sizeof(double) * bb);
        if (h->p.sub_ilu == 2) {
            L->nf_pos[g] = (int*)malloc(sizeof(int) * (size_t)m);
            if (!L->nf_pos[g]) {
                free(v);
                return ORACLE_ENOMEM;
            }
            int q = 0;
            for (int c = L->coff[g]; c < L->coff[g + 1]; ++c)
                for (int i = o0; i < o1; ++i)
                    if (L->colour[i] == c) L->nf_pos[g][i - o0] = q++;
        }
        st = oracle_ilu0_field_ordered(m, b, zeros, L->nf_rp[g], L->nf_ci[g], v, 0, L->nf_pos[g], L->ilu[g]);
        free(v);
        if (st) return st;
    }
    return ORACLE_OK;
}

/* first-fit colours of every field on the graph of its diagonal block,
 * numbered after the colours of the earlier fields (coff) */
static int colour_node_fields(const oracle_hier* h, olevel* L) {
    int base = 0;
    L->coff[0] = 0;
    for (int g = 0; g < h->NF; ++g) {
        const int o0 = L->foff[g], m = L->foff[g + 1] - o0;
        int *rp = NULL, *ci = NULL;
        int st = field_subgraph(L, g, &rp, &ci);
        if (st) return st;
        int nc = oracle_colour(m, rp, ci, L->colour + o0);
        free(rp);
        free(ci);
        if (nc < 0) return nc;
        for (int i = 0; i < m; ++i) L->colour[o0 + i] += base;
        base += nc;
        L->coff[g + 1] = base;
    }
    return base;
}

static int level_schwarz(oracle_hier* h, olevel* L);

/* per-field inverses of the node diagonal blocks of level L: node i, field f
 * at dinv + i*dstride + doff[f] (fsize[f]^2 entries, row-major; with equal
 * fields this is [n][F][fb*fb]) */
static int level_dinv(oracle_hier* h, olevel* L) {
    const int b = h->b, F = h->F;
    const size_t bb = (size_t)b * b;
    L->dinv = (double*)malloc(sizeof(double) * (size_t)L->n * h->dstride);
    if (!L->dinv) return ORACLE_ENOMEM;
    for (int i = 0; i < L->n; ++i) {
        int kd = find_pos(L->col_idx, L->row_ptr[i], L->row_ptr[i + 1], i);
        if (kd < 0) return ORACLE_EINVAL;
        for (int f = 0; f < F; ++f) {
            double blk[ORACLE_MAX_B * ORACLE_MAX_B];
            const int s = h->fstart[f], fb = h->fsize[f];
            for (int r = 0; r < fb; ++r)
                for (int c = 0; c < fb; ++c) blk[r * fb + c] = L->vals[(size_t)kd * bb + (s + r) * b + (s + c)];
            int st = oracle_block_inverse(fb, blk, L->dinv + (size_t)i * h->dstride + h->doff[f]);
            if (st != ORACLE_OK) return st;
        }
    }
    return ORACLE_OK;
}

/* the damping weights of a level that is being coarsened: from the MLP on
 * the level's features, from the caller's arrays, or the constants */
static int level_weights(oracle_hier* h, int l, olevel* L, long long* used_s, long long* used_p) {
    const int F = h->F;
    const oracle_params* p = &h->p;
    const size_t ns = (size_t)L->n * F, np = (size_t)L->n_agg * F;
    L->omega_s = (double*)malloc(sizeof(double) * ns);
    L->omega_p = (double*)calloc(np > 0 ? np : 1, sizeof(double));
    if (!L->omega_s || !L->omega_p) return ORACLE_ENOMEM;
    if (p->mlp && p->mlp_levels > 0 && l >= p->mlp_levels) { /* beyond the network's depths */
        for (size_t e = 0; e < ns; ++e) L->omega_s[e] = p->omega;
        L->smoothed = 0;
        return ORACLE_OK;
    }
    if (p->mlp) {
        double* nf = (double*)malloc(sizeof(double) * ns * ORACLE_NFEAT);
        double* af = (double*)malloc(sizeof(double) * (np > 0 ? np : 1) * ORACLE_NFEAT);
        double* yn = (double*)malloc(sizeof(double) * ns * ORACLE_MLP_OUT);
        double* ya = (double*)malloc(sizeof(double) * (np > 0 ? np : 1) * ORACLE_MLP_OUT);
        if (!nf || !af || !yn || !ya) return ORACLE_ENOMEM;
        int fmap[ORACLE_MAX_B];
        for (int d = 0; d < h->b; ++d) fmap[d] = h->field_of_dof[d];
        int st = oracle_features(L->n, h->b, fmap, L->row_ptr, L->col_idx, L->vals, L->agg, L->n_agg, l, nf, af);
        if (st == ORACLE_OK) st = oracle_mlp_forward(p->mlp, nf, (int)ns, yn);
        if (st == ORACLE_OK) st = oracle_mlp_forward(p->mlp, af, (int)np, ya);
        for (size_t e = 0; e < ns && st == ORACLE_OK; ++e) L->omega_s[e] = oracle_mlp_clip(0, yn[e * ORACLE_MLP_OUT]);
        /* P is smoothed on this level only where a weight survives the clip */
        L->smoothed = 0;
        for (size_t e = 0; e < np && st == ORACLE_OK; ++e) {
            L->omega_p[e] = oracle_mlp_clip(1, ya[e * ORACLE_MLP_OUT + 1]);
            if (L->omega_p[e] > 0.0) L->smoothed = 1;
        }
        free(nf);
        free(af);
        free(yn);
        free(ya);
        return st;
    }
    L->smoothed = p->smooth_p != 0;
    if (p->omega_s_arr) {
        if (*used_s + (long long)ns > p->omega_s_len) return ORACLE_EINVAL;
        memcpy(L->omega_s, p->omega_s_arr + *used_s, sizeof(double) * ns);
        *used_s += (long long)ns;
    } else {
        for (size_t e = 0; e < ns; ++e) L->omega_s[e] = p->omega;
    }
    if (p->smooth_p && p->omega_p_arr) {
        if (*used_p + (long long)np > p->omega_p_len) return ORACLE_EINVAL;
        memcpy(L->omega_p, p->omega_p_arr + *used_p, sizeof(double) * np);
        *used_p += (long long)np;
    } else if (p->smooth_p) {
        for (size_t e = 0; e < np; ++e) L->omega_p[e] = p->omega_p;
    }
    return ORACLE_OK;
}

void oracle_free(oracle_hier* h) {
    if (!h) return;
    for (int l = 0; l < h->nlev; ++l) level_free(&h->lev[l]);
    free(h->lu);
    free(h->piv);
    free(h->xt);
    free(h->rf);
    free(h);
}

int oracle_setup(int n, int nnzb, int b, const int* row_ptr, const int* col_idx,
                 const double* vals, const int* field_of_dof, const oracle_params* p,
                 oracle_hier** out) {
    *out = NULL;
    if (n <= 0 || b < 1 || b > ORACLE_MAX_B || p->max_levels < 1 || p->max_levels > ORACLE_MAX_LEVELS)
        return ORACLE_EINVAL;
    oracle_hier* h = (oracle_hier*)calloc(1, sizeof(oracle_hier));
    if (!h) return ORACLE_ENOMEM;
    h->b = b;
    h->p = *p;
    /* fields: contiguous, non-decreasing 0..F-1, equal sizes */
    int F = 0;
    for (int d = 0; d < b; ++d) {
        h->field_of_dof[d] = field_of_dof[d];
        if (d > 0 && field_of_dof[d] != field_of_dof[d - 1] && field_of_dof[d] != field_of_dof[d - 1] + 1) {
            free(h);
            return ORACLE_EINVAL;
        }
        if (field_of_dof[d] + 1 > F) F = field_of_dof[d] + 1;
    }
    if (field_of_dof[0] != 0) {
        free(h);
        return ORACLE_EINVAL;
    }
    /* field blocks of unequal size (Algorithm 1 needs none equal): each field
     * its own fsize x fsize diagonal blocks and sub-solve; the options built
     * on one common field size (smoothed P, learned weights, ILU(0), Schwarz,
     * fields on node sets) need equal sizes */
    h->F = F;
    h->fb = 0;
    h->dstride = 0;
    int unequal = 0;
    for (int f = 0; f < F; ++f) {
        int cnt = 0, first = -1;
        for (int d = 0; d < b; ++d)
            if (field_of_dof[d] == f) {
                if (first < 0) first = d;
                cnt++;
            }
        h->fstart[f] = first;
        h->fsize[f] = cnt;
        h->doff[f] = h->dstride;
        h->dstride += cnt * cnt;
        if (cnt > h->fb) h->fb = cnt;
        if (cnt != h->fsize[0]) unequal = 1;
    }
    if (unequal && (p->smooth_p || p->omega_p_arr || p->mlp || p->sub_ilu || p->sub_schwarz ||
                    p->n_node_fields > 1)) {
        free(h);
        return ORACLE_EINVAL;
    }
    /* fields on disjoint node sets: contiguous non-empty node ranges, one
     * field per node, and only the plain method (tentative P, constant
     * damping, the multicolour sub-solve) */
    h->NF = p->n_node_fields > 1 ? p->n_node_fields : 1;
    if (h->NF > 1) {
        const int* off = p->node_field_off;
        int bad = h->NF > ORACLE_MAX_NODE_FIELDS || !off || F != 1 || p->smooth_p ||
                  p->omega_s_arr || p->omega_p_arr || p->mlp;
        if (!bad) {
            bad = off[0] != 0 || off[h->NF] != n;
            for (int g = 0; g < h->NF && !bad; ++g) bad = off[g + 1] <= off[g];
        }
        if (bad) {
            free(h);
            return ORACLE_EINVAL;
        }
    }
    const size_t bb = (size_t)b * b;
    /* level 0 = a copy of A */
    olevel* L0 = &h->lev[0];
    if (h->NF > 1) {
        L0->foff = (int*)malloc(sizeof(int) * (size_t)(h->NF + 1));
        memcpy(L0->foff, p->node_field_off, sizeof(int) * (size_t)(h->NF + 1));
    }
    L0->n = n;
    L0->nnzb = nnzb;
    L0->row_ptr = (int*)malloc(sizeof(int) * (size_t)(n + 1));
    L0->col_idx = (int*)malloc(sizeof(int) * (size_t)nnzb);
    L0->vals = (double*)malloc(sizeof(double) * bb * (size_t)nnzb);
    memcpy(L0->row_ptr, row_ptr, sizeof(int) * (size_t)(n + 1));
    memcpy(L0->col_idx, col_idx, sizeof(int) * (size_t)nnzb);
    memcpy(L0->vals, vals, sizeof(double) * bb * (size_t)nnzb);
    h->nlev = 1;
    int st = ORACLE_OK;
    long long used_s = 0, used_p = 0;
    if ((p->omega_s_arr && p->omega_s_len < 0) || (p->omega_p_arr && p->omega_p_len < 0) || p->mlp_levels < 0 ||
        p->sub_schwarz < 0 || p->sub_schwarz > 2 || p->schwarz_overlap < 0 || p->schwarz_overlap > 1 ||
        (p->sub_schwarz && p->sub_ilu) || p->inner_sweeps < 0 || p->inner_sweeps > 64 ||
        (p->inner_sweeps > 1 && (p->sub_ilu || p->sub_schwarz || p->n_node_fields > 1)))
        st = ORACLE_EINVAL;
    if (st != ORACLE_OK) {
        oracle_free(h);
        return st;
    }
    /* coarsen while n*b > max_coarse and fewer than max_levels levels */
    while (h->nlev < p->max_levels && (long)h->lev[h->nlev - 1].n * b > p->max_coarse) {
        olevel* F_ = &h->lev[h->nlev - 1];
        F_->agg = (int*)malloc(sizeof(int) * (size_t)F_->n);
        int nc;
        if (h->NF > 1) {
            /* separate aggregates per field block (Sec. 4.3.1) */
            olevel* Cf = &h->lev[h->nlev];
            Cf->foff = (int*)malloc(sizeof(int) * (size_t)(h->NF + 1));
            nc = Cf->foff ? aggregate_node_fields(h, F_, F_->agg, Cf->foff) : ORACLE_ENOMEM;
        } else {
            int* is_root = (int*)malloc(sizeof(int) * (size_t)F_->n);
            nc = oracle_aggregate(F_->n, F_->row_ptr, F_->col_idx, F_->agg, is_root);
            free(is_root);
        }
        if (nc < 0) {
            free(h->lev[h->nlev].foff);
            h->lev[h->nlev].foff = NULL;
            st = nc;
            break;
        }
        if (nc == 0 || nc == F_->n) { /* no coarsening possible */
            free(F_->agg);
            F_->agg = NULL;
            free(h->lev[h->nlev].foff);
            h->lev[h->nlev].foff = NULL;
            break;
        }
        F_->n_agg = nc;
        st = level_dinv(h, F_);
        if (st == ORACLE_OK) st = level_weights(h, h->nlev - 1, F_, &used_s, &used_p);
        if (st != ORACLE_OK) break;
        olevel* C = &h->lev[h->nlev];
        C->n = nc;
        C->row_ptr = (int*)malloc(sizeof(int) * (size_t)(nc + 1));
        if (F_->smoothed) {
            /* A_c = P^T A P with the smoothed prolongator */
            F_->p_rp = (int*)malloc(sizeof(int) * (size_t)(F_->n + 1));
            int nnzp = oracle_prolongator(F_->n, b, h->field_of_dof, F_->row_ptr, F_->col_idx, F_->vals, F_->agg,
                                          nc, F_->omega_p, F_->p_rp, NULL, NULL);
            if (nnzp < 0) {
                st = nnzp;
                break;
            }
            F_->p_nnz = nnzp;
            F_->p_ci = (int*)malloc(sizeof(int) * (size_t)(nnzp > 0 ? nnzp : 1));
            F_->p_v = (double*)malloc(sizeof(double) * (size_t)(nnzp > 0 ? nnzp : 1) * F * h->fb * h->fb);
            nnzp = oracle_prolongator(F_->n, b, h->field_of_dof, F_->row_ptr, F_->col_idx, F_->vals, F_->agg, nc,
                                      F_->omega_p, F_->p_rp, F_->p_ci, F_->p_v);
            if (nnzp < 0) {
                st = nnzp;
                break;
            }
            st = transpose_p(F_->n, nc, F_->p_rp, F_->p_ci, &F_->r_rp, &F_->r_q, &F_->r_i);
            if (st) break;
            int nnzc = oracle_rap_general(F_->n, b, h->field_of_dof, F_->row_ptr, F_->col_idx, F_->vals, nc,
                                          F_->p_rp, F_->p_ci, F_->p_v, C->row_ptr, NULL, NULL);
            if (nnzc < 0) {
                st = nnzc;
                break;
            }
            C->nnzb = nnzc;
            C->col_idx = (int*)malloc(sizeof(int) * (size_t)(nnzc > 0 ? nnzc : 1));
            C->vals = (double*)malloc(sizeof(double) * bb * (size_t)(nnzc > 0 ? nnzc : 1));
            nnzc = oracle_rap_general(F_->n, b, h->field_of_dof, F_->row_ptr, F_->col_idx, F_->vals, nc, F_->p_rp,
                                      F_->p_ci, F_->p_v, C->row_ptr, C->col_idx, C->vals);
            if (nnzc < 0) {
                st = nnzc;
                break;
            }
        } else {
            int nnzc = oracle_rap_tentative(F_->n, b, F_->row_ptr, F_->col_idx, F_->vals, F_->agg, nc,
                                            C->row_ptr, NULL, NULL);
            C->nnzb = nnzc;
            C->col_idx = (int*)malloc(sizeof(int) * (size_t)nnzc);
            C->vals = (double*)malloc(sizeof(double) * bb * (size_t)nnzc);
            oracle_rap_tentative(F_->n, b, F_->row_ptr, F_->col_idx, F_->vals, F_->agg, nc, C->row_ptr,
                                 C->col_idx, C->vals);
        }
        h->nlev++;
    }
    if (st == ORACLE_OK && p->mlp == NULL &&
        ((p->omega_s_arr && used_s != p->omega_s_len) || (p->smooth_p && p->omega_p_arr && used_p != p->omega_p_len)))
        st = ORACLE_EINVAL;
    if (st != ORACLE_OK) {
        oracle_free(h);
        return st;
    }
    /* smoother data on every level except the coarsest */
    size_t max_n = 0;
    for (int l = 0; l < h->nlev; ++l) {
        olevel* L = &h->lev[l];
        if ((size_t)L->n > max_n) max_n = (size_t)L->n;
        L->u = (double*)calloc((size_t)L->n * b, sizeof(double));
        L->rhs = (double*)calloc((size_t)L->n * b, sizeof(double));
        L->res = (double*)calloc((size_t)L->n * b, sizeof(double));
        if (l == h->nlev - 1) break;
        L->colour = (int*)malloc(sizeof(int) * (size_t)L->n);
        if (h->NF > 1) {
            L->coff = (int*)malloc(sizeof(int) * (size_t)(h->NF + 1));
            L->n_colours = L->coff ? colour_node_fields(h, L) : ORACLE_ENOMEM;
            if (L->n_colours < 0) {
                st = L->n_colours;
                break;
            }
        } else {
            L->n_colours = oracle_colour(L->n, L->row_ptr, L->col_idx, L->colour);
        }
        if (!L->dinv) st = level_dinv(h, L); /* computed while coarsening */
        if (st != ORACLE_OK) break;
        if (p->sub_ilu == 2 && h->NF == 1) {  /* colour order: colour ascending, then node index */
            L->ilu_pos = (int*)malloc(sizeof(int) * (size_t)L->n);
            if (!L->ilu_pos) st = ORACLE_ENOMEM;
            int e = 0;
            for (int c = 0; c < L->n_colours && st == ORACLE_OK; ++c)
                for (int i = 0; i < L->n; ++i)
                    if (L->colour[i] == c) L->ilu_pos[i] = e++;
        }
        if (p->sub_schwarz && st == ORACLE_OK) st = level_schwarz(h, L);
        if (p->sub_ilu && h->NF > 1) {
            if (st == ORACLE_OK) st = ilu_node_fields(h, L);
        } else if (p->sub_ilu)
            for (int f = 0; f < h->F && st == ORACLE_OK; ++f) {
                L->ilu[f] = (double*)malloc(sizeof(double) * (size_t)L->nnzb * h->fb * h->fb);
                st = L->ilu[f] ? oracle_ilu0_field_ordered(L->n, b, h->field_of_dof, L->row_ptr, L->col_idx,
                                                           L->vals, f, L->ilu_pos, L->ilu[f])
                               : ORACLE_ENOMEM;
            }
        if (st != ORACLE_OK) break;
    }
    if (st == ORACLE_OK) {
        h->xt = (double*)calloc(max_n * h->fb, sizeof(double));
        h->rf = (double*)calloc(max_n * h->fb, sizeof(double));
        /* coarsest level: dense copy and LU */
        olevel* L = &h->lev[h->nlev - 1];
        int nd = L->n * b;
        h->nc_dense = nd;
        h->lu = (double*)calloc((size_t)nd * nd, sizeof(double));
        h->piv = (int*)malloc(sizeof(int) * (size_t)nd);
        if (!h->lu || !h->piv) st = ORACLE_ENOMEM;
        for (int i = 0; i < L->n && st == ORACLE_OK; ++i)
            for (int k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) {
                int j = L->col_idx[k];
                for (int r = 0; r < b; ++r)
                    for (int c = 0; c < b; ++c)
                        h->lu[(size_t)(i * b + r) * nd + (j * b + c)] = L->vals[(size_t)k * bb + r * b + c];
            }
        if (st == ORACLE_OK) st = oracle_lu_factor(nd, h->lu, h->piv);
    }
    if (st != ORACLE_OK) {
        oracle_free(h);
        return st;
    }
    *out = h;
    return ORACLE_OK;
}

int oracle_num_levels(const oracle_hier* h) { return h->nlev; }

int oracle_level_sizes(const oracle_hier* h, int l, int* n, int* nnzb, int* n_colours, int* n_agg) {
    if (l < 0 || l >= h->nlev) return ORACLE_EINVAL;
    const olevel* L = &h->lev[l];
    if (n) *n = L->n;
    if (nnzb) *nnzb = L->nnzb;
    if (n_colours) *n_colours = L->n_colours;
    if (n_agg) *n_agg = (l < h->nlev - 1) ? L->n_agg : 0;
    return ORACLE_OK;
}

int oracle_level_get(const oracle_hier* h, int l, int* row_ptr, int* col_idx, double* vals, int* agg,
                     int* colour, double* dinv) {
    if (l < 0 || l >= h->nlev) return ORACLE_EINVAL;
    const olevel* L = &h->lev[l];
    size_t bb = (size_t)h->b * h->b;
    if (row_ptr) memcpy(row_ptr, L->row_ptr, sizeof(int) * (size_t)(L->n + 1));
    if (col_idx) memcpy(col_idx, L->col_idx, sizeof(int) * (size_t)L->nnzb);
    if (vals) memcpy(vals, L->vals, sizeof(double) * bb * (size_t)L->nnzb);
    int has_smoother = l < h->nlev - 1;
    if (agg && has_smoother) memcpy(agg, L->agg, sizeof(int) * (size_t)L->n);
    if (colour && has_smoother) memcpy(colour, L->colour, sizeof(int) * (size_t)L->n);
    if (dinv && has_smoother) memcpy(dinv, L->dinv, sizeof(double) * (size_t)L->n * h->dstride);
    return ORACLE_OK;
}

int oracle_level_fields(const oracle_hier* h, int l, int* node_off, int* colour_off) {
    if (l < 0 || l >= h->nlev) return ORACLE_EINVAL;
    const olevel* L = &h->lev[l];
    if (h->NF > 1) {
        if (node_off) memcpy(node_off, L->foff, sizeof(int) * (size_t)(h->NF + 1));
        if (colour_off && L->coff) memcpy(colour_off, L->coff, sizeof(int) * (size_t)(h->NF + 1));
    } else {
        if (node_off) {
            node_off[0] = 0;
            node_off[1] = L->n;
        }
        if (colour_off) {
            colour_off[0] = 0;
            colour_off[1] = l < h->nlev - 1 ? L->n_colours : 0;
        }
    }
    return h->NF;
}

int oracle_level_p_nnz(const oracle_hier* h, int l) {
    if (l < 0 || l >= h->nlev) return ORACLE_EINVAL;
    return h->lev[l].p_v ? h->lev[l].p_nnz : 0;
}

int oracle_level_get_p(const oracle_hier* h, int l, int* p_rp, int* p_ci, double* p_v) {
    if (l < 0 || l >= h->nlev || !h->lev[l].p_v) return ORACLE_EINVAL;
    const olevel* L = &h->lev[l];
    if (p_rp) memcpy(p_rp, L->p_rp, sizeof(int) * (size_t)(L->n + 1));
    if (p_ci) memcpy(p_ci, L->p_ci, sizeof(int) * (size_t)L->p_nnz);
    if (p_v) memcpy(p_v, L->p_v, sizeof(double) * (size_t)L->p_nnz * h->F * h->fb * h->fb);
    return ORACLE_OK;
}

int oracle_level_omega(const oracle_hier* h, int l, double* omega_s, double* omega_p) {
    if (l < 0 || l >= h->nlev - 1) return ORACLE_EINVAL;
    const olevel* L = &h->lev[l];
    if (omega_s) memcpy(omega_s, L->omega_s, sizeof(double) * (size_t)L->n * h->F);
    if (omega_p) memcpy(omega_p, L->omega_p, sizeof(double) * (size_t)L->n_agg * h->F);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------------ */
/* Damped block Gauss-Seidel smoother, Algorithm 1 (Sec. 4.3.2), for F      */
/* field blocks.  One sweep visits the fields in order; for field f:        */
/*   r_f := b_f - sum_g A_fg x_g        with the current x (which includes  */
/*                                       the update of field f-1);          */
/*   solve A_ff x~_f = r_f approximately: one multicolour node-block        */
/*     Gauss-Seidel sweep from x~ = 0 (colours ascending; node i of colour  */
/*     c: x~_i = D_ff,i^{-1} (r_f,i - sum_{j != i} A_ff[i,j] x~_j));        */
/*   x_f := x_f + omega x~_f.                                               */
/* ------------------------------------------------------------------------ */
/* ------------------------------------------------------------------------ */
/* Additive Schwarz with overlap as Algorithm 1's sub-solve (Sec. 5: one    */
/* additive Schwarz iteration with overlap one approximates A_ff^{-1}).     */
/* Subdomains are the level's aggregates, one per aggregate and field (the  */
/* aggregates of a field on disjoint node sets carry that field only),      */
/* extended by `overlap` layers of neighbours in the graph of A_ff.  With   */
/* R_I the restriction to the subdomain's dofs of field f and               */
/* A_I = R_I A_ff R_I^T:                                                    */
/*   additive:   x~_f = sum_I R_I^T A_I^{-1} R_I r_f;                       */
/*   restricted: every node takes its value from its own aggregate's solve. */
/* ------------------------------------------------------------------------ */
static int level_schwarz(oracle_hier* h, olevel* L) {
    const int b = h->b, n = L->n;
    const int fb = h->NF > 1 ? b : h->fb;  /* dofs of one field per node */
    const int nfs = h->NF > 1 ? 1 : h->F;  /* subdomains per aggregate */
    const size_t bb = (size_t)b * b;
    int *mptr = NULL, *mem = NULL;
    int st = aggregate_members(n, L->agg, L->n_agg, &mptr, &mem);
    if (st) return st;
    int* nfield = (int*)calloc((size_t)n, sizeof(int));
    int* mark = (int*)malloc(sizeof(int) * (size_t)n);
    int* list = (int*)malloc(sizeof(int) * (size_t)(n + L->nnzb));
    const size_t cap = (size_t)nfs * (size_t)(n + L->nnzb);
    L->n_sd = L->n_agg * nfs;
    L->sd_field = (int*)malloc(sizeof(int) * (size_t)L->n_sd);
    L->sd_ptr = (int*)malloc(sizeof(int) * (size_t)(L->n_sd + 1));
    L->sd_nodes = (int*)malloc(sizeof(int) * cap);
    L->sd_own = (unsigned char*)malloc(cap);
    L->sd_lu_off = (size_t*)malloc(sizeof(size_t) * (size_t)(L->n_sd + 1));
    if (!nfield || !mark || !list || !L->sd_field || !L->sd_ptr || !L->sd_nodes || !L->sd_own || !L->sd_lu_off) {
        st = ORACLE_ENOMEM;
        goto done;
    }
    if (h->NF > 1)
        for (int g = 0; g < h->NF; ++g)
            for (int i = L->foff[g]; i < L->foff[g + 1]; ++i) nfield[i] = g;
    for (int i = 0; i < n; ++i) mark[i] = -1;
    /* node lists */
    int e = 0;
    size_t lu_total = 0;
    L->sd_max_m = 0;
    L->sd_ptr[0] = 0;
    L->sd_lu_off[0] = 0;
    for (int I = 0; I < L->n_agg; ++I) {
        int cnt = 0;
        for (int t = mptr[I]; t < mptr[I + 1]; ++t) {
            list[cnt++] = mem[t];
            mark[mem[t]] = I;
        }
        for (int layer = 0; layer < h->p.schwarz_overlap; ++layer) {
            const int c0 = cnt;
            for (int t = 0; t < c0; ++t) {
                const int i = list[t];
                for (int k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) {
                    const int j = L->col_idx[k];
                    if (mark[j] == I || nfield[j] != nfield[i]) continue;
                    mark[j] = I;
                    list[cnt++] = j;
                }
            }
        }
        qsort(list, (size_t)cnt, sizeof(int), cmp_int);
        for (int fs = 0; fs < nfs; ++fs) {
            const int q = I * nfs + fs;
            L->sd_field[q] = h->NF > 1 ? nfield[mem[mptr[I]]] : fs;
            for (int t = 0; t < cnt; ++t) {
                L->sd_nodes[e + t] = list[t];
                L->sd_own[e + t] = L->agg[list[t]] == I;
            }
            e += cnt;
            L->sd_ptr[q + 1] = e;
            const size_t m = (size_t)cnt * fb;
            lu_total += m * m;
            L->sd_lu_off[q + 1] = lu_total;
            if ((int)m > L->sd_max_m) L->sd_max_m = (int)m;
        }
    }
    /* dense A_I and its LU */
    L->sd_lu = (double*)calloc(lu_total > 0 ? lu_total : 1, sizeof(double));
    L->sd_piv = (int*)malloc(sizeof(int) * (size_t)(e > 0 ? e : 1) * fb);
    if (!L->sd_lu || !L->sd_piv) {
        st = ORACLE_ENOMEM;
        goto done;
    }
    for (int q = 0; q < L->n_sd && st == ORACLE_OK; ++q) {
        const int s0 = L->sd_ptr[q], cnt = L->sd_ptr[q + 1] - s0, m = cnt * fb;
        const int f0 = h->NF > 1 ? 0 : h->fstart[L->sd_field[q]];
        double* A = L->sd_lu + L->sd_lu_off[q];
        for (int p = 0; p < cnt; ++p) {
            const int i = L->sd_nodes[s0 + p];
            for (int k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) {
                /* position of column j in the subdomain's ascending node list */
                const int j = L->col_idx[k];
                int lo = 0, hi = cnt;
                while (lo < hi) {
                    const int mid = (lo + hi) / 2;
                    if (L->sd_nodes[s0 + mid] < j) lo = mid + 1;
                    else hi = mid;
                }
                if (lo == cnt || L->sd_nodes[s0 + lo] != j) continue;
                const double* blk = L->vals + (size_t)k * bb;
                for (int r = 0; r < fb; ++r)
                    for (int c = 0; c < fb; ++c)
                        A[(size_t)(p * fb + r) * m + (lo * fb + c)] = blk[(f0 + r) * b + (f0 + c)];
            }
        }
        if (oracle_lu_factor(m, A, L->sd_piv + (size_t)s0 * fb) != ORACLE_OK) st = ORACLE_ESINGULAR_BLOCK;
    }
done:
    free(mptr);
    free(mem);
    free(nfield);
    free(mark);
    free(list);
    return st;
}

/* x~ += the Schwarz sub-solve of r for field f; r and x~ hold the field's dofs
 * of nodes base.. with stride fb */
static int schwarz_apply(const oracle_hier* h, const olevel* L, int f, int base, int fb, const double* r,
                         double* xt) {
    const int m_max = L->sd_max_m > 0 ? L->sd_max_m : 1;
    double* rl = (double*)malloc(sizeof(double) * (size_t)m_max);
    double* y = (double*)malloc(sizeof(double) * (size_t)m_max);
    if (!rl || !y) {
        free(rl);
        free(y);
        return ORACLE_ENOMEM;
    }
    for (int q = 0; q < L->n_sd; ++q) {
        if (L->sd_field[q] != f) continue;
        const int s0 = L->sd_ptr[q], cnt = L->sd_ptr[q + 1] - s0, m = cnt * fb;
        for (int p = 0; p < cnt; ++p)
            for (int c = 0; c < fb; ++c) rl[p * fb + c] = r[(size_t)(L->sd_nodes[s0 + p] - base) * fb + c];
        oracle_lu_solve(m, L->sd_lu + L->sd_lu_off[q], L->sd_piv + (size_t)s0 * fb, rl, y);
        for (int p = 0; p < cnt; ++p) {
            if (h->p.sub_schwarz == 2 && !L->sd_own[s0 + p]) continue;
            for (int c = 0; c < fb; ++c) xt[(size_t)(L->sd_nodes[s0 + p] - base) * fb + c] += y[p * fb + c];
        }
    }
    free(rl);
    free(y);
    return ORACLE_OK;
}

/* Algorithm 1 with the field blocks on disjoint node sets: field g owns the */
/* nodes o_g <= i < o_{g+1} with all their dofs, A_gg is the block matrix    */
/* between those nodes.  One sweep visits the fields in order; for field g: */
/*   r_g := b_g - sum_h A_gh x_h        (rows of field g, all columns);     */
/*   x~_g := one multicolour node-block Gauss-Seidel sweep on A_gg from 0   */
/*     (field g's colours ascending; only columns of field g take part);    */
/*   x_g := x_g + omega x~_g.                                               */
static int bgs_node_fields(oracle_hier* h, int l, double* x, const double* rhs, int sweeps, int unit_damping) {
    olevel* L = &h->lev[l];
    const int b = h->b;
    const size_t bb = (size_t)b * b;
    double* rf = h->rf;
    double* xt = h->xt;
    for (int s = 0; s < sweeps; ++s) {
        for (int g = 0; g < h->NF; ++g) {
            const int o0 = L->foff[g], o1 = L->foff[g + 1];
            for (int i = o0; i < o1; ++i)
                for (int r = 0; r < b; ++r) {
                    double acc = rhs[(size_t)i * b + r];
                    for (int k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) {
                        const double* blk = L->vals + (size_t)k * bb;
                        int j = L->col_idx[k];
                        for (int c = 0; c < b; ++c) acc -= blk[r * b + c] * x[(size_t)j * b + c];
                    }
                    rf[(size_t)(i - o0) * b + r] = acc;
                }
            for (size_t e = 0; e < (size_t)(o1 - o0) * b; ++e) xt[e] = 0.0;
            if (h->p.sub_schwarz) {
                int st = schwarz_apply(h, L, g, o0, b, rf, xt);
                if (st) return st;
            } else if (h->p.sub_ilu) {
                int st = oracle_ilu0_solve_ordered(o1 - o0, b, L->nf_rp[g], L->nf_ci[g], L->nf_pos[g], L->ilu[g], rf, xt);
                if (st) return st;
            }
            const int sweep = !h->p.sub_schwarz && !h->p.sub_ilu;
            for (int col = L->coff[g]; col < (sweep ? L->coff[g + 1] : L->coff[g]); ++col) {
                for (int i = o0; i < o1; ++i) {
                    if (L->colour[i] != col) continue;
                    double t[ORACLE_MAX_B];
                    for (int r = 0; r < b; ++r) {
                        double acc = rf[(size_t)(i - o0) * b + r];
                        for (int k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) {
                            int j = L->col_idx[k];
                            if (j == i || j < o0 || j >= o1) continue;
                            const double* blk = L->vals + (size_t)k * bb;
                            for (int c = 0; c < b; ++c) acc -= blk[r * b + c] * xt[(size_t)(j - o0) * b + c];
                        }
                        t[r] = acc;
                    }
                    const double* Di = L->dinv + (size_t)i * bb;
                    for (int r = 0; r < b; ++r) {
                        double acc = 0.0;
                        for (int c = 0; c < b; ++c) acc += Di[r * b + c] * t[c];
                        xt[(size_t)(i - o0) * b + r] = acc;
                    }
                }
            }
            for (int i = o0; i < o1; ++i) {
                const double om = unit_damping ? 1.0 : L->omega_s[i];
                for (int r = 0; r < b; ++r) x[(size_t)i * b + r] += om * xt[(size_t)(i - o0) * b + r];
            }
        }
    }
    return ORACLE_OK;
}

/* unit_damping: omega = 1 everywhere (used by the training targets) */
static int bgs_impl(oracle_hier* h, int l, double* x, const double* rhs, int sweeps, int unit_damping) {
    if (l < 0 || l >= h->nlev - 1) return ORACLE_EINVAL;
    if (h->NF > 1) return bgs_node_fields(h, l, x, rhs, sweeps, unit_damping);
    olevel* L = &h->lev[l];
    const int b = h->b, F = h->F;
    const size_t bb = (size_t)b * b;
    double* rf = h->rf;
    double* xt = h->xt;
    for (int s = 0; s < sweeps; ++s) {
        for (int f = 0; f < F; ++f) {
            const int f0 = h->fstart[f], fb = h->fsize[f]; /* field f: dofs f0 .. f0 + fb - 1 */
            /* residual of the rows of field f, all columns */
            for (int i = 0; i < L->n; ++i)
                for (int r = 0; r < fb; ++r) {
                    double acc = rhs[(size_t)i * b + f0 + r];
                    for (int k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) {
                        const double* blk = L->vals + (size_t)k * bb;
                        int j = L->col_idx[k];
                        for (int c = 0; c < b; ++c) acc -= blk[(f0 + r) * b + c] * x[(size_t)j * b + c];
                    }
                    rf[(size_t)i * fb + r] = acc;
                }
            /* approximate A_ff^{-1} r_f: ILU(0) of A_ff, or one multicolour
             * node-block GS sweep from zero */
            for (size_t e = 0; e < (size_t)L->n * fb; ++e) xt[e] = 0.0;
            if (h->p.sub_ilu) {
                int st = oracle_ilu0_solve_ordered(L->n, fb, L->row_ptr, L->col_idx, L->ilu_pos, L->ilu[f], rf, xt);
                if (st) return st;
            } else if (h->p.sub_schwarz) {
                int st = schwarz_apply(h, L, f, 0, fb, rf, xt);
                if (st) return st;
            }
            /* inner sweeps of the multicolour Gauss-Seidel sub-solve: the formula
             * below takes every j != i with its current x~, which is zero for the
             * later colours in the first sweep and the previous sweep's value after */
            const int inner = h->p.inner_sweeps > 1 ? h->p.inner_sweeps : 1;
            for (int q = 0; q < ((h->p.sub_ilu || h->p.sub_schwarz) ? 0 : inner); ++q)
            for (int col = 0; col < L->n_colours; ++col) {
                for (int i = 0; i < L->n; ++i) {
                    if (L->colour[i] != col) continue;
                    double t[ORACLE_MAX_B];
                    for (int r = 0; r < fb; ++r) {
                        double acc = rf[(size_t)i * fb + r];
                        for (int k = L->row_ptr[i]; k < L->row_ptr[i + 1]; ++k) {
                            int j = L->col_idx[k];
                            if (j == i) continue;
                            const double* blk = L->vals + (size_t)k * bb;
                            for (int c = 0; c < fb; ++c) acc -= blk[(f0 + r) * b + (f0 + c)] * xt[(size_t)j * fb + c];
                        }
                        t[r] = acc;
                    }
                    const double* Di = L->dinv + (size_t)i * h->dstride + h->doff[f];
                    for (int r = 0; r < fb; ++r) {
                        double acc = 0.0;
                        for (int c = 0; c < fb; ++c) acc += Di[r * fb + c] * t[c];
                        xt[(size_t)i * fb + r] = acc;
                    }
                }
            }
            /* damped update of field f, damping omega_{i,f} of node i */
            for (int i = 0; i < L->n; ++i) {
                const double om = unit_damping ? 1.0 : L->omega_s[(size_t)i * F + f];
                for (int r = 0; r < fb; ++r) x[(size_t)i * b + f0 + r] += om * xt[(size_t)i * fb + r];
            }
        }
    }
    return ORACLE_OK;
}

int oracle_bgs(oracle_hier* h, int l, double* x, const double* rhs, int sweeps) {
    return bgs_impl(h, l, x, rhs, sweeps, 0);
}

/* ------------------------------------------------------------------------ */
/* V-cycle MGV(u, b, l) of Fig. 1, u = 0 on entry:                          */
/*   l < l_max: u <- S_pre(A, u, b); r <- b - A u; u_c <- 0;                */
/*              u_c <- MGV(u_c, R r, l+1); u <- u + P u_c; u <- S_post(...) */
/*   l = l_max: u <- A^{-1} b                                               */
/* R r sums r over the members of each aggregate (ascending node order),    */
/* P u_c copies u_c[agg(i)] to node i, dof by dof.                          */
/* ------------------------------------------------------------------------ */
static int mgv(oracle_hier* h, int l, double* u, const double* rhs) {
    olevel* L = &h->lev[l];
    const int b = h->b;
    const size_t nb = (size_t)L->n * b;
    if (l == h->nlev - 1) return oracle_lu_solve((int)nb, h->lu, h->piv, rhs, u);
    int st = oracle_bgs(h, l, u, rhs, h->p.n_pre);
    if (st) return st;
    oracle_spmv(L->n, b, L->row_ptr, L->col_idx, L->vals, u, L->res);
    for (size_t e = 0; e < nb; ++e) L->res[e] = rhs[e] - L->res[e];
    olevel* C = &h->lev[l + 1];
    const size_t ncb = (size_t)C->n * b;
    for (size_t e = 0; e < ncb; ++e) {
        C->rhs[e] = 0.0;
        C->u[e] = 0.0;
    }
    if (L->p_v) {
        /* R r = P^T r: coarse row I sums P_f[i,I]^T r_f,i over i ascending */
        const int F = h->F, fb = h->fb;
        const size_t pbs = (size_t)F * fb * fb;
        for (int I = 0; I < C->n; ++I)
            for (int t = L->r_rp[I]; t < L->r_rp[I + 1]; ++t) {
                const int i = L->r_i[t];
                const double* P = L->p_v + (size_t)L->r_q[t] * pbs;
                for (int r = 0; r < b; ++r) {
                    const int f = h->field_of_dof[r], f0 = h->fstart[f], rl = r - f0;
                    double s = 0.0;
                    for (int m = 0; m < fb; ++m) s += P[(size_t)f * fb * fb + m * fb + rl] * L->res[(size_t)i * b + f0 + m];
                    C->rhs[(size_t)I * b + r] += s;
                }
            }
    } else {
        for (int i = 0; i < L->n; ++i)
            for (int d = 0; d < b; ++d) C->rhs[(size_t)L->agg[i] * b + d] += L->res[(size_t)i * b + d];
    }
    st = mgv(h, l + 1, C->u, C->rhs);
    if (st) return st;
    if (L->p_v) {
        /* u += P u_c: row i sums P_f[i,J] u_c,J over its stored J ascending */
        const int F = h->F, fb = h->fb;
        const size_t pbs = (size_t)F * fb * fb;
        for (int i = 0; i < L->n; ++i)
            for (int r = 0; r < b; ++r) {
                const int f = h->field_of_dof[r], f0 = h->fstart[f], rl = r - f0;
                double y = 0.0;
                for (int q = L->p_rp[i]; q < L->p_rp[i + 1]; ++q) {
                    const double* P = L->p_v + (size_t)q * pbs + (size_t)f * fb * fb;
                    double s = 0.0;
                    for (int m = 0; m < fb; ++m) s += P[rl * fb + m] * C->u[(size_t)L->p_ci[q] * b + f0 + m];
                    y += s;
                }
                u[(size_t)i * b + r] += y;
            }
    } else {
        for (int i = 0; i < L->n; ++i)
            for (int d = 0; d < b; ++d) u[(size_t)i * b + d] += C->u[(size_t)L->agg[i] * b + d];
    }
    return oracle_bgs(h, l, u, rhs, h->p.n_post);
}

int oracle_vcycle(oracle_hier* h, const double* r, double* z) {
    size_t nb = (size_t)h->lev[0].n * h->b;
    for (size_t e = 0; e < nb; ++e) z[e] = 0.0;
    return mgv(h, 0, z, r);
}


/* ------------------------------------------------------------------------ */
/* Restarted flexible GMRES (Saad 1993) with right preconditioning:         */
/*   r0 = b - A x0, beta = ||r0||, v1 = r0 / beta; for j = 1..m:            */
/*   z_j = M v_j; w = A z_j; modified Gram-Schmidt against v_1..v_j;        */
/*   h_{j+1,j} = ||w||; Givens rotations on the Hessenberg column; stop     */
/*   when |g_{j+1}| / ||b|| <= tol; x = x0 + Z y at the end of the cycle.   */
/* Happy breakdown when h_{j+1,j} <= 1e-14 ||w|| (w before orthogonalising).*/
/* ------------------------------------------------------------------------ */
int oracle_fgmres(oracle_hier* h, const double* b, double* x, double tol, int m, int max_iter,
                  int prec, int* iters, double* relres) {
    olevel* L = &h->lev[0];
    const size_t N = (size_t)L->n * h->b;
    if (m < 1) return ORACLE_EINVAL;
    double* V = (double*)malloc(sizeof(double) * N * (size_t)(m + 1));
    double* Z = (double*)malloc(sizeof(double) * N * (size_t)m);
    double* w = (double*)malloc(sizeof(double) * N);
    double* H = (double*)calloc((size_t)(m + 1) * m, sizeof(double));
    double* cs = (double*)calloc((size_t)m, sizeof(double));
    double* sn = (double*)calloc((size_t)m, sizeof(double));
    double* g = (double*)calloc((size_t)m + 1, sizeof(double));
    double* y = (double*)calloc((size_t)m, sizeof(double));
    if (!V || !Z || !w || !H || !cs || !sn || !g || !y) return ORACLE_ENOMEM;
#define HH(i, j) H[(size_t)(i) * m + (j)]
    int total = 0, converged = 0, st = ORACLE_OK;
    double bnorm = nrm2(N, b), rel = 0.0;
    if (bnorm == 0.0) {
        for (size_t e = 0; e < N; ++e) x[e] = 0.0;
        converged = 1;
    }
    while (!converged) {
        oracle_spmv(L->n, h->b, L->row_ptr, L->col_idx, L->vals, x, w);
        for (size_t e = 0; e < N; ++e) w[e] = b[e] - w[e];
        double beta = nrm2(N, w);
        rel = beta / bnorm;
        if (rel <= tol) {
            converged = 1;
            break;
        }
        if (total >= max_iter) break;
        for (size_t e = 0; e < N; ++e) V[e] = w[e] / beta;
        for (int i = 0; i <= m; ++i) g[i] = 0.0;
        g[0] = beta;
        int k = 0;
        for (int j = 0; j < m; ++j) {
            double* vj = V + (size_t)j * N;
            double* zj = Z + (size_t)j * N;
            if (prec == 0) {
                st = oracle_vcycle(h, vj, zj);
                if (st) break;
            } else {
                for (size_t e = 0; e < N; ++e) zj[e] = vj[e];
            }
            oracle_spmv(L->n, h->b, L->row_ptr, L->col_idx, L->vals, zj, w);
            double wnorm0 = nrm2(N, w);
            for (int i = 0; i <= j; ++i) {
                const double* vi = V + (size_t)i * N;
                HH(i, j) = dot(N, w, vi);
                for (size_t e = 0; e < N; ++e) w[e] -= HH(i, j) * vi[e];
            }
            double hn = nrm2(N, w);
            HH(j + 1, j) = hn;
            total++;
            k = j + 1;
            int breakdown = !(hn > 1e-14 * wnorm0);
            if (!breakdown) {
                double* vn = V + (size_t)(j + 1) * N;
                for (size_t e = 0; e < N; ++e) vn[e] = w[e] / hn;
            }
            for (int i = 0; i < j; ++i) {
                double t = cs[i] * HH(i, j) + sn[i] * HH(i + 1, j);
                HH(i + 1, j) = -sn[i] * HH(i, j) + cs[i] * HH(i + 1, j);
                HH(i, j) = t;
            }
            double d = sqrt(HH(j, j) * HH(j, j) + HH(j + 1, j) * HH(j + 1, j));
            if (d == 0.0) {
                cs[j] = 1.0;
                sn[j] = 0.0;
            } else {
                cs[j] = HH(j, j) / d;
                sn[j] = HH(j + 1, j) / d;
            }
            HH(j, j) = d;
            HH(j + 1, j) = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            if (fabs(g[j + 1]) / bnorm <= tol || breakdown || total >= max_iter) break;
        }
        if (st) break;
        /* y = H(0:k,0:k)^{-1} g(0:k), upper triangular */
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int c = i + 1; c < k; ++c) s -= HH(i, c) * y[c];
            y[i] = s / HH(i, i);
        }
        for (int i = 0; i < k; ++i) {
            const double* zi = Z + (size_t)i * N;
            for (size_t e = 0; e < N; ++e) x[e] += y[i] * zi[e];
        }
    }
#undef HH
    free(V);
    free(Z);
    free(w);
    free(H);
    free(cs);
    free(sn);
    free(g);
    free(y);
    *iters = total;
    *relres = rel;
    if (st) return st;
    return converged ? ORACLE_OK : ORACLE_NOT_CONVERGED;
}
