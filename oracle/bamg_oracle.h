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

/* ---- hierarchy ---- */

typedef struct {
    int max_levels;   /* >= 1 */
    int max_coarse;   /* coarsen while n*b > max_coarse */
    int n_pre;        /* BGS sweeps before the coarse correction */
    int n_post;       /* BGS sweeps after it */
    double omega;     /* BGS damping */
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

#ifdef __cplusplus
}
#endif
#endif
