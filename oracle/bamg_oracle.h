/*
 * FP64 CPU oracle of the monolithic block AMG (arXiv 2103.07537) used as an
 * FGMRES preconditioner.  TEST INFRASTRUCTURE ONLY: it is called by the test
 * suite, by the smoke check and by the benchmark's CPU-baseline leg, never by
 * the CUDA library.  It shares no code with the CUDA path.
 *
 * Plain, slow, sequential and written to be read against the paper:
 *   - V-cycle MGV(u, b, l)                        Sec. 3, Fig. 1
 *   - Galerkin coarse operator A_{l+1} = R A P    Sec. 3 (display after Fig. 1)
 *   - block-diagonal transfers R = diag(R00, R11), P = diag(P00, P11)
 *                                                  Sec. 4.3.1, eq. (blocktransfers)
 *   - aggregates: a disjoint cover of the nodes, one coarse node each, built
 *     greedily on the graph of A00 and cloned to the Maxwell block
 *                                                  Sec. 4.3.1, cloned-aggregation figure
 *     or, for fields on different node sets, built separately on the graph
 *     of each diagonal block                       Sec. 4.3.1; Sec. 5, mixed elements
 *   - piecewise-constant interpolation per solution component  Sec. 4.3.1
 *   - damped block Gauss-Seidel smoother           Sec. 4.3.2, Algorithm 1
 *   - direct solve on the coarsest level           Fig. 1; Sec. 5.1
 * and, beyond the paper, restarted flexible GMRES with the V-cycle as right
 * preconditioner (the paper applies the V-cycle inside GMRES: Sec. 3, Sec. 5.1).
 *
 * Every function here is pinned by tests/test_oracle_pins.py against facts
 * that do not come from this file (dense linear algebra, brute force on tiny
 * graphs, closed forms, invariants).
 *
 * Layout: block CSR over nodes, int32 indices, columns ascending, b x b
 * blocks row-major, dofs of a node interleaved in field order.  Vectors have
 * n*b entries, node-major.  Every function returns 0 on success or a
 * negative status (see ORACLE_E*).
 */
#ifndef BAMG_ORACLE_H
#define BAMG_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ENOMEM (-2)
#define ORACLE_ESINGULAR_BLOCK (-3)
#define ORACLE_ESINGULAR_COARSE (-4)
#define ORACLE_NOT_CONVERGED 1

#define ORACLE_MAX_LEVELS 16
#define ORACLE_MAX_B 8
#define ORACLE_MAX_NODE_FIELDS 8

typedef struct oracle_hier oracle_hier;

/* ---- standalone steps (each one is also used inside the hierarchy) ---- */

/* y = A x */
int oracle_spmv(int n, int b, const int* row_ptr, const int* col_idx, const double* vals,
                const double* x, double* y);

/* Aggregation of the node graph (structural, diagonal excluded).
 * agg[n] receives the aggregate id of every node, is_root[n] 1 for roots.
 * Returns the number of aggregates (>= 0) or a negative status. */
int oracle_aggregate(int n, const int* row_ptr, const int* col_idx, int* agg, int* is_root);

/* First-fit colouring in ascending node order.  Returns the colour count. */
int oracle_colour(int n, const int* row_ptr, const int* col_idx, int* colour);

/* Galerkin product with the tentative prolongator of agg[]: A_c = P^T A P.
 * Two calls: with rp_c != NULL and ci_c == NULL it fills rp_c[nc+1] and
 * returns nnzb_c; with ci_c and vals_c it fills them (rp_c as filled). */
int oracle_rap_tentative(int n, int b, const int* row_ptr, const int* col_idx, const double* vals,
                         const int* agg, int nc, int* rp_c, int* ci_c, double* vals_c);

/* Inverse of a dense m x m matrix (row-major) by Gauss-Jordan elimination
 * with partial pivoting.  ORACLE_ESINGULAR_BLOCK if a pivot magnitude is
 * below 1e-14 * (infinity norm of the matrix). */
int oracle_block_inverse(int m, const double* a, double* ainv);

/* Dense LU with partial pivoting (first row of maximal magnitude wins),
 * in place on a[n*n] row-major; piv[k] = row swapped with row k. */
int oracle_lu_factor(int n, double* a, int* piv);
int oracle_lu_solve(int n, const double* lu, const int* piv, const double* rhs, double* x);

/* Smoothed prolongator of one level (beyond the paper; the paper's P is
 * the tentative one).  Per field f, P_f = (I - W_f D_ff^{-1} A_ff) P^_f with
 * P^ the piecewise-constant prolongator of agg[], D_ff,i the field-f
 * diagonal sub-block of A[i,i] and W_f = diag over fine nodes i of
 * omega_p[agg(i)*F + f].  P keeps the field-block-diagonal form of the
 * transfers (Sec. 4.3.1), so a stored block (i, J) holds F sub-blocks of
 * fb x fb, field-major, row-major: p_v[(k*F + f)*fb*fb + r*fb + c].
 * Pattern of row i: the distinct agg(j) over the stored j of row i,
 * ascending.  Two calls like oracle_rap_tentative (p_ci == NULL: fills
 * p_rp[n+1], returns nnz). */
int oracle_prolongator(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                       const double* vals, const int* agg, int nc, const double* omega_p, int* p_rp,
                       int* p_ci, double* p_v);

/* Galerkin product A_c = P^T A P (Sec. 3) with a field-block-diagonal P in
 * the layout of oracle_prolongator.  Pattern: the structural union,
 * ascending.  Two calls (ci_c == NULL: fills rp_c[nc+1], returns nnz). */
int oracle_rap_general(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                       const double* vals, int nc, const int* p_rp, const int* p_ci, const double* p_v,
                       int* rp_c, int* ci_c, double* vals_c);

/* ---- ILU(0) of a field's diagonal part (Algorithm 1's sub-solve, Sec. 4.3.2) ----
 * A_ff is the scalar matrix of the fb x fb field-f sub-blocks of every stored
 * block, rows and columns in node-then-dof order (scalar row i*fb + r).  Its
 * incomplete LU with zero fill keeps that pattern: for the scalar rows in
 * order, and for each entry q < p of row p in ascending column order,
 * l_pq = a_pq / u_qq, then a_pt -= l_pq u_qt for every t > q of row p that
 * row q also holds.  lu[nnzb][fb][fb] (sub-block layout): entry (k, r, c) of
 * block k = (i, j) holds L (unit lower, strictly below the scalar diagonal)
 * or U (on and above it) at scalar row i*fb + r, column j*fb + c.
 * ORACLE_ESINGULAR_BLOCK if a pivot u_qq is zero. */
int oracle_ilu0_field(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                      const double* vals, int f, double* lu);
/* x = (L U)^{-1} r with the factors of oracle_ilu0_field (r, x: n*fb) */
int oracle_ilu0_solve(int n, int fb, const int* row_ptr, const int* col_idx, const double* lu,
                      const double* r, double* x);
/* The same in the elimination order given by pos[i] (the position of node i;
 * scalar row i*fb + r is eliminated as pos[i]*fb + r).  With nodes ordered by
 * colour (sub_ilu = 2) the nodes of one colour do not couple, so each colour's
 * rows of the triangular solves depend on earlier colours only. */
int oracle_ilu0_field_ordered(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                              const double* vals, int f, const int* pos, double* lu);
int oracle_ilu0_solve_ordered(int n, int fb, const int* row_ptr, const int* col_idx, const int* pos,
                              const double* lu, const double* r, double* x);

/* ---- hierarchy ---- */

typedef struct {
    int max_levels;   /* >= 1 */
    int max_coarse;   /* coarsen while n*b > max_coarse */
    int n_pre;        /* BGS sweeps before the coarse correction */
    int n_post;       /* BGS sweeps after it */
    double omega;     /* BGS damping */
    /* ---- beyond the paper: smoothed transfers and per-node damping ---- */
    int smooth_p;     /* 0: tentative P; 1: P_f = (I - W_f D_ff^{-1} A_ff) P^_f per field */
    double omega_p;   /* W_f weight of every aggregate when omega_p_arr is NULL */
    /* per-level weights, consumed level by level from the finest: omega_s_arr
     * holds n_l*F values (node-major, then field) for every level that gets a
     * smoother, omega_p_arr n_agg_l*F values for every level that is coarsened.
     * NULL: omega / omega_p everywhere.  A length that does not match the
     * hierarchy exactly is ORACLE_EINVAL. */
    const double* omega_s_arr;
    long long omega_s_len;
    const double* omega_p_arr;
    long long omega_p_len;
    /* learned weights: MLP parameters (ORACLE_MLP_NPARAMS values) or NULL.
     * When set, every coarsened level takes omega_s and omega_p from the MLP
     * applied to its features, clipped by oracle_mlp_clip (overriding the
     * arrays above and smooth_p); a level smooths P only when some weight
     * of its aggregates is nonzero after the clip. */
    const double* mlp;
    int mlp_levels;   /* with mlp: levels 0..mlp_levels-1 take the network's weights, deeper
                         levels omega and the tentative P; 0 = every level */
    int sub_ilu;      /* Algorithm 1's approximate sub-solve of A_ff: 0 = one multicolour
                         node-block Gauss-Seidel sweep from zero; 1 = ILU(0) of A_ff (the
                         paper's sub-solver, Sec. 4.3.2 and Sec. 5.1), natural order; 2 = ILU(0)
                         with the nodes eliminated in colour order (colour, then index) */
    /* ---- fields on disjoint node sets (fields that are not co-located: the
     * mixed-element case of Sec. 4.3.1 and Sec. 5) ----
     * n_node_fields > 1: the nodes form n_node_fields contiguous ranges
     * [node_field_off[g], node_field_off[g+1]), and every dof of a node belongs
     * to the node's field (field_of_dof all 0).  On every level the aggregates
     * of field g are built separately on the graph of A_gg (the blocks between
     * nodes of field g), numbered after those of the earlier fields, so that
     * P = diag(P_0, P_1, ...) and the coarse nodes keep contiguous field ranges.
     * Colours are per field too (first fit on the graph of A_gg), numbered after
     * those of the earlier fields, and Algorithm 1 takes the node fields as its
     * field blocks (with sub_ilu, the ILU(0) of each A_gg as a block matrix of its own).
     * Requires smooth_p = 0, no weight arrays and no mlp.  n_node_fields <= 1: the
     * co-located case above. */
    int n_node_fields;
    const int* node_field_off;
    /* ---- additive Schwarz as Algorithm 1's sub-solve (the paper's choice in Sec. 5:
     * one additive Schwarz iteration with overlap one) ----
     * sub_schwarz: 0 = off; 1 = additive, x~_f = sum_I R_I^T A_I^{-1} R_I r_f; 2 = restricted
     * additive (every node takes the value of its own subdomain's solve only).
     * Subdomains: the level's aggregates (one per aggregate and field), extended by
     * schwarz_overlap (0 or 1) layers of neighbours in the graph of A_ff; A_I = the field-f
     * sub-blocks between the subdomain's nodes (nodes ascending, dofs in field order),
     * solved exactly by dense LU with partial pivoting.  Not with sub_ilu. */
    int sub_schwarz;
    int schwarz_overlap;
    /* inner_sweeps > 1: the multicolour Gauss-Seidel sub-solve of A_ff runs that many
     * forward sweeps (the first from x~ = 0, each later one from the previous x~, the
     * higher colours' values taken from the previous sweep); 0 and 1 = one sweep.
     * Only with the multicolour sub-solve of co-located fields (not with sub_ilu,
     * sub_schwarz or n_node_fields > 1); at most 64. */
    int inner_sweeps;
} oracle_params;

int oracle_setup(int n, int nnzb, int b, const int* row_ptr, const int* col_idx,
                 const double* vals, const int* field_of_dof, const oracle_params* p,
                 oracle_hier** out);
void oracle_free(oracle_hier* h);

int oracle_num_levels(const oracle_hier* h);
/* sizes of level l: nodes, stored blocks, colours, aggregates below (0 on the coarsest) */
int oracle_level_sizes(const oracle_hier* h, int l, int* n, int* nnzb, int* n_colours, int* n_agg);
/* copies of level l's data; any pointer may be NULL.  dinv has n*F*fb*fb entries:
 * node-major, then field, then the fb x fb inverse row-major. */
int oracle_level_get(const oracle_hier* h, int l, int* row_ptr, int* col_idx, double* vals,
                     int* agg, int* colour, double* dinv);

/* Field ranges of level l with n_node_fields > 1: node_off[NF+1] (nodes of
 * field g), colour_off[NF+1] (colours of field g; levels with a smoother).
 * Either pointer may be NULL.  Returns NF (1 in the co-located case). */
int oracle_level_fields(const oracle_hier* h, int l, int* node_off, int* colour_off);
/* Smoothed prolongator of level l (levels that were coarsened with
 * smooth_p = 1): stored blocks, then the copies (any pointer may be NULL). */
int oracle_level_p_nnz(const oracle_hier* h, int l);
int oracle_level_get_p(const oracle_hier* h, int l, int* p_rp, int* p_ci, double* p_v);
/* damping weights of level l: omega_s[n*F] (smoother), omega_p[n_agg*F]
 * (prolongator smoothing; zeros with smooth_p = 0) */
int oracle_level_omega(const oracle_hier* h, int l, double* omega_s, double* omega_p);

/* The smoother S on level l applied in place to x for `sweeps` sweeps. */
int oracle_bgs(oracle_hier* h, int l, double* x, const double* rhs, int sweeps);
/* z = MGV(0, r, 0): one V-cycle from a zero initial guess. */
int oracle_vcycle(oracle_hier* h, const double* r, double* z);

/* Right-preconditioned restarted FGMRES(restart) on the finest operator.
 * prec = 0: V-cycle, 1: identity.  x holds x0 on entry.  *iters = total
 * inner steps, *relres = ||b - A x|| / ||b|| recomputed at exit.
 * Returns 0 when converged, ORACLE_NOT_CONVERGED otherwise. */
int oracle_fgmres(oracle_hier* h, const double* b, double* x, double tol, int restart,
                  int max_iter, int prec, int* iters, double* relres);

/* ---- learned damping (beyond the paper) ---- */


#define ORACLE_NFEAT 8
#define ORACLE_MLP_H 64
#define ORACLE_MLP_OUT 2
/* parameters: W1[H][NFEAT], b1[H], W2[H][H], b2[H], W3[OUT][H], b3[OUT]
 * (trained), then the fixed input normalisation xm[NFEAT], xs[NFEAT] */
#define ORACLE_MLP_NTRAIN (ORACLE_MLP_H * ORACLE_NFEAT + ORACLE_MLP_H + ORACLE_MLP_H * ORACLE_MLP_H + \
                           ORACLE_MLP_H + ORACLE_MLP_OUT * ORACLE_MLP_H + ORACLE_MLP_OUT)
#define ORACLE_MLP_NPARAMS (ORACLE_MLP_NTRAIN + 2 * ORACLE_NFEAT)

/* Features of every node and field of one level (NFEAT per row, rows
 * node-major then field) and of every aggregate and field (the mean over its
 * members, ascending).  See the definition in bamg_oracle.c. */
int oracle_features(int n, int b, const int* field_of_dof, const int* row_ptr, const int* col_idx,
                    const double* vals, const int* agg, int nc, int level, double* node_feat,
                    double* agg_feat);

/* y[n][OUT] = MLP(x[n][NFEAT]): h1 = tanh(W1 xh + b1), h2 = tanh(W2 h1 + b2),
 * y = W3 h2 + b3, with xh = (x - xm) * xs. */
int oracle_mlp_forward(const double* params, const double* x, int n, double* y);
/* loss = (1/n) sum_r (y[r][head[r]] - t[r])^2 and its gradient with respect
 * to the trained parameters (grad[NTRAIN]). */
int oracle_mlp_grad(const double* params, const double* x, const double* t, const int* head, int n,
                    double* grad, double* loss);
/* one Adam step (step count t >= 1) on the trained parameters */
int oracle_adam(double* params, const double* grad, double* m, double* v, int t, double lr, double beta1,
                double beta2, double eps);
/* the weight ranges: head 0 (smoother damping) [0.05, 1.5]; head 1 (P
 * smoothing) [0, 1.5], values below 0.05 set to 0 (no smoothing) */
double oracle_mlp_clip(int head, double w);

#ifdef __cplusplus
}
#endif
#endif
