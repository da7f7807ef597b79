/*
 * FP64 CPU oracle of the learned damping weights (beyond the paper).
 * TEST INFRASTRUCTURE ONLY, like bamg_oracle.c: the tests, the smoke check
 * and the benchmark's CPU-baseline leg call it, the CUDA library never does.
 *
 * The paper shows that the damping of its block Gauss-Seidel smoother
 * decides convergence for small viscosities (Sec. 5, generator example, the
 * figure of iterations against the BGS damping) and fixes one value near
 * 0.5.  Here a small network predicts the damping per node and field, and
 * the weight of a smoothed prolongator per aggregate and field, from
 * features of the level's matrix:
 *   features   oracle_features
 *   network    oracle_mlp_forward: 8 -> 64 (tanh) -> 64 (tanh) -> 2
 *   training   oracle_mlp_grad (mean squared error), oracle_adam
 * Sequential, unblocked; compiled with -ffp-contract=off like the rest.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "bamg_oracle.h"

#define NF ORACLE_NFEAT
#define NH ORACLE_MLP_H
#define NO ORACLE_MLP_OUT

/* parameter offsets */
#define O_W1 0
#define O_B1 (O_W1 + NH * NF)
#define O_W2 (O_B1 + NH)
#define O_B2 (O_W2 + NH * NH)
#define O_W3 (O_B2 + NH)
#define O_B3 (O_W3 + NO * NH)
#define O_XM (O_B3 + NO)
#define O_XS (O_XM + NF)

double oracle_mlp_clip(int head, double w) {
    if (head == 0) {
        if (!(w >= 0.05)) return 0.05; /* NaN maps to the lower end */
        return w > 1.5 ? 1.5 : w;
    }
    if (!(w >= 0.05)) return 0.0;
    return w > 1.5 ? 1.5 : w;
}

static double frob(const double* blk, int b, int r0, int c0, int m) {
    double s = 0.0;
    for (int r = 0; r < m; ++r)
        for (int c = 0; c < m; ++c) s += blk[(r0 + r) * b + c0 + c] * blk[(r0 + r) * b + c0 + c];
    return sqrt(s);
}

/*
 * Features of node i, field f on level `level` (Frobenius norms of the fb x
 * fb sub-blocks of the stored blocks of row i):
 *   d = ||A_ff[i,i]||, o = sum_{j != i} ||A_ff[i,j]||,
 *   c = sum_j sum_{g != f} ||A_fg[i,j]||
 *   0  log d                     scale of the field at the node
 *   1  o / d                     off-diagonal weight of the field block
 *   2  c / (d + o)               coupling to the other fields
 *   3  log d - mean_g log d_g    scale relative to the node's other fields
 *   4  tr A_ff[i,i] / (sqrt(fb) d)  sign / definiteness of the diagonal block
 *   5  log |agg(i)|              size of the node's aggregate
 *   6  level
 *   7  f
 * Aggregate I, field f: the mean of its members' rows (ascending members).
 */
int oracle_features(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                    const double* vals, const int* agg, int nc, int level, double* node_feat,
                    double* agg_feat) {
    int F = 0;
    for (int d = 0; d < b; ++d)
        if (field_of_dof[d] + 1 > F) F = field_of_dof[d] + 1;
    if (b < 1 || b > ORACLE_MAX_B || F < 1 || b % F) return ORACLE_EINVAL;
    const int fb = b / F;
    const size_t bb = (size_t)b * b;
    int fstart[ORACLE_MAX_B];
    for (int f = 0; f < F; ++f) {
        fstart[f] = -1;
        for (int d = b - 1; d >= 0; --d)
            if (field_of_dof[d] == f) fstart[f] = d;
        if (fstart[f] < 0) return ORACLE_EINVAL;
    }
    int* cnt = (int*)calloc(nc > 0 ? (size_t)nc : 1, sizeof(int));
    if (!cnt) return ORACLE_ENOMEM;
    for (int i = 0; i < n; ++i) {
        if (agg[i] < 0 || agg[i] >= nc) {
            free(cnt);
            return ORACLE_EINVAL;
        }
        cnt[agg[i]]++;
    }
    for (int i = 0; i < n; ++i) {
        double d[ORACLE_MAX_B], o[ORACLE_MAX_B], c[ORACLE_MAX_B], tr[ORACLE_MAX_B];
        for (int f = 0; f < F; ++f) d[f] = o[f] = c[f] = tr[f] = 0.0;
        for (int k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            const double* blk = vals + (size_t)k * bb;
            const int j = col_idx[k];
            for (int f = 0; f < F; ++f) {
                for (int g = 0; g < F; ++g) {
                    const double nrm = frob(blk, b, fstart[f], fstart[g], fb);
                    if (g != f) c[f] += nrm;
                    else if (j == i) d[f] = nrm;
                    else o[f] += nrm;
                }
                if (j == i)
                    for (int r = 0; r < fb; ++r) tr[f] += blk[(fstart[f] + r) * b + fstart[f] + r];
            }
        }
        double mean_log = 0.0;
        for (int f = 0; f < F; ++f) {
            if (!(d[f] > 0.0)) {
                free(cnt);
                return ORACLE_ESINGULAR_BLOCK;
            }
            mean_log += log(d[f]);
        }
        mean_log /= F;
        for (int f = 0; f < F; ++f) {
            double* x = node_feat + ((size_t)i * F + f) * NF;
            x[0] = log(d[f]);
            x[1] = o[f] / d[f];
            x[2] = c[f] / (d[f] + o[f]);
            x[3] = log(d[f]) - mean_log;
            x[4] = tr[f] / (sqrt((double)fb) * d[f]);
            x[5] = log((double)cnt[agg[i]]);
            x[6] = (double)level;
            x[7] = (double)f;
        }
    }
    if (agg_feat) {
        memset(agg_feat, 0, sizeof(double) * (size_t)nc * F * NF);
        for (int i = 0; i < n; ++i)
            for (int f = 0; f < F; ++f)
                for (int m = 0; m < NF; ++m)
                    agg_feat[((size_t)agg[i] * F + f) * NF + m] += node_feat[((size_t)i * F + f) * NF + m];
        for (int I = 0; I < nc; ++I)
            for (int f = 0; f < F; ++f)
                for (int m = 0; m < NF; ++m) agg_feat[((size_t)I * F + f) * NF + m] /= (double)cnt[I];
    }
    free(cnt);
    return ORACLE_OK;
}

/* forward pass of one row; keeps the activations for the backward pass */
static void forward_row(const double* p, const double* x, double* xh, double* h1, double* h2, double* y) {
    for (int m = 0; m < NF; ++m) xh[m] = (x[m] - p[O_XM + m]) * p[O_XS + m];
    for (int k = 0; k < NH; ++k) {
        double a = 0.0;
        for (int m = 0; m < NF; ++m) a += p[O_W1 + k * NF + m] * xh[m];
        h1[k] = tanh(a + p[O_B1 + k]);
    }
    for (int j = 0; j < NH; ++j) {
        double a = 0.0;
        for (int k = 0; k < NH; ++k) a += p[O_W2 + j * NH + k] * h1[k];
        h2[j] = tanh(a + p[O_B2 + j]);
    }
    for (int o = 0; o < NO; ++o) {
        double a = 0.0;
        for (int j = 0; j < NH; ++j) a += p[O_W3 + o * NH + j] * h2[j];
        y[o] = a + p[O_B3 + o];
    }
}

int oracle_mlp_forward(const double* params, const double* x, int n, double* y) {
    double xh[NF], h1[NH], h2[NH];
    if (n < 0) return ORACLE_EINVAL;
    for (int r = 0; r < n; ++r) forward_row(params, x + (size_t)r * NF, xh, h1, h2, y + (size_t)r * NO);
    return ORACLE_OK;
}

/* reverse-mode differentiation of the mean squared error, row by row */
int oracle_mlp_grad(const double* params, const double* x, const double* t, const int* head, int n,
                    double* grad, double* loss) {
    double xh[NF], h1[NH], h2[NH], y[NO], dy[NO], da2[NH], da1[NH];
    if (n < 1) return ORACLE_EINVAL;
    memset(grad, 0, sizeof(double) * ORACLE_MLP_NTRAIN);
    double l = 0.0;
    for (int r = 0; r < n; ++r) {
        if (head[r] < 0 || head[r] >= NO) return ORACLE_EINVAL;
        forward_row(params, x + (size_t)r * NF, xh, h1, h2, y);
        const double err = y[head[r]] - t[r];
        l += err * err;
        for (int o = 0; o < NO; ++o) dy[o] = o == head[r] ? 2.0 * err / n : 0.0;
        for (int o = 0; o < NO; ++o) {
            grad[O_B3 + o] += dy[o];
            for (int j = 0; j < NH; ++j) grad[O_W3 + o * NH + j] += dy[o] * h2[j];
        }
        for (int j = 0; j < NH; ++j) {
            double g = 0.0;
            for (int o = 0; o < NO; ++o) g += dy[o] * params[O_W3 + o * NH + j];
            da2[j] = g * (1.0 - h2[j] * h2[j]);
            grad[O_B2 + j] += da2[j];
            for (int k = 0; k < NH; ++k) grad[O_W2 + j * NH + k] += da2[j] * h1[k];
        }
        for (int k = 0; k < NH; ++k) {
            double g = 0.0;
            for (int j = 0; j < NH; ++j) g += params[O_W2 + j * NH + k] * da2[j];
            da1[k] = g * (1.0 - h1[k] * h1[k]);
            grad[O_B1 + k] += da1[k];
            for (int m = 0; m < NF; ++m) grad[O_W1 + k * NF + m] += da1[k] * xh[m];
        }
    }
    *loss = l / n;
    return ORACLE_OK;
}

/* Adam (Kingma and Ba 2015) with bias-corrected moments */
int oracle_adam(double* params, const double* grad, double* m, double* v, int t, double lr, double beta1,
                double beta2, double eps) {
    if (t < 1) return ORACLE_EINVAL;
    const double c1 = 1.0 - pow(beta1, t), c2 = 1.0 - pow(beta2, t);
    for (int q = 0; q < ORACLE_MLP_NTRAIN; ++q) {
        m[q] = beta1 * m[q] + (1.0 - beta1) * grad[q];
        v[q] = beta2 * v[q] + (1.0 - beta2) * grad[q] * grad[q];
        params[q] -= lr * (m[q] / c1) / (sqrt(v[q] / c2) + eps);
    }
    return ORACLE_OK;
}
