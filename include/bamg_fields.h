/*
 * bamg_fields: fields on disjoint node sets (fields that are not co-located,
 * for example a mixed finite-element discretisation with the hydrodynamic
 * unknowns on Q2 nodes and the magnetic unknowns on Q1 vertices).
 * Method: Sec. 4.3.1 of arXiv 2103.07537 (separate aggregates built on the
 * graph of each diagonal block, combined into block-diagonal transfers) and
 * the mixed-element example of Sec. 5.
 *
 * The conventions of bamg.h hold (block CSR, device pointers, statuses, the
 * stream); a handle made here is used with amg_apply, fgmres_solve,
 * amg_level_info, amg_level_get, amg_stats_json and amg_destroy of bamg.h.
 */
#ifndef BAMG_FIELDS_H
#define BAMG_FIELDS_H

#include "bamg.h"

#ifdef __cplusplus
extern "C" {
#endif

#define BAMG_MAX_NODE_FIELDS 8

/*
 * amg_setup_fields - build the hierarchy of a system whose fields live on
 * disjoint node sets.
 *   Layout: field g owns the nodes field_node_off[g] .. field_node_off[g+1]-1
 *   (HOST array of n_fields+1 ints: 0 = field_node_off[0] < ... <
 *   field_node_off[n_fields] = n_nodes); every node carries b dofs of its
 *   own field (b in {1, 2, 3, 4, 6}, the same for every field).  row_ptr,
 *   col_idx, vals: device block CSR as in amg_setup (blocks between nodes of
 *   different fields are the coupling blocks A_gh).
 *   Per level: the aggregates of field g are built separately on the graph of
 *   A_gg (the stored blocks between two nodes of field g) and numbered after
 *   those of fields 0..g-1, so that P = diag(P_0, P_1, ...) and the coarse
 *   nodes of every field again form one contiguous range; the Galerkin
 *   product keeps the coupling blocks; colours are first fit on the graph of
 *   A_gg, field g's after those of fields 0..g-1.  Algorithm 1 (Sec. 4.3.2)
 *   takes the node fields as its field blocks: one field step updates the
 *   nodes of one field from the residual of its rows, with one multicolour
 *   node-block Gauss-Seidel sweep on A_gg (or sub_solver's ILU(0) or
 *   restricted Schwarz) as the approximate sub-solve; the other fields'
 *   nodes are copied by a kernel of the cycle.
 *   p: as in amg_setup, with smooth_p = 0, no weight arrays and no mlp
 *   (BAMG_EINVAL otherwise); tail_dofs and tail_grid are ignored (the
 *   single-launch tail records no copies of the other fields' nodes).
 *   n_fields = 1 builds the same hierarchy as amg_setup with one field.
 *   Errors: BAMG_EINVAL for bad ranges or parameters, the other statuses as
 *   for amg_setup; *out is NULL after an error.
 */
int amg_setup_fields(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int nnzb, int b,
                     int n_fields, const int* field_node_off, const amg_params* p, void* stream, bamg_t* out);

/*
 * amg_solve_fields_host - end-to-end solve of a system with fields on node
 *   sets, with HOST buffers: copies A and the right-hand side to the device,
 *   runs amg_setup_fields and fgmres_solve on `stream`, copies the solution
 *   back to x_host (initial guess on entry) and frees everything it
 *   allocated.  Arguments and statuses as those two calls, all arrays on the
 *   host.
 */
int amg_solve_fields_host(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int nnzb, int b,
                          int n_fields, const int* field_node_off, const amg_params* p, const double* rhs_host,
                          double* x_host, double tol, int restart, int max_iter, int* iters, double* relres,
                          void* stream);

/*
 * amg_level_fields - field ranges of level `level` of a hierarchy:
 *   node_off[n_fields+1] (nodes of field g) and colour_off[n_fields+1]
 *   (colours of field g; zeros on the coarsest level), host arrays, either
 *   may be NULL.  Returns n_fields (1 for a hierarchy of amg_setup, with the
 *   whole level as field 0), or BAMG_EINVAL for a bad handle or level.
 */
int amg_level_fields(bamg_t h, int level, int* node_off, int* colour_off);

#ifdef __cplusplus
}
#endif

#endif
