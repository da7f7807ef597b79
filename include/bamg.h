/*
 * bamg: monolithic block algebraic multigrid for coupled multi-field block
 * systems on one GB300 GPU (sm_103a), used as a preconditioner for FP64
 * flexible GMRES.  Method: Ohm, Wiesner, Cyr, Hu, Shadid, Tuminaro,
 * "A monolithic algebraic multigrid framework for multiphysics applications
 * with examples from resistive MHD" (arXiv 2103.07537).
 *
 * ---------------------------------------------------------------------------
 * Conventions shared by every entry point
 * ---------------------------------------------------------------------------
 * Matrix layout (block CSR, "BSR"): n_nodes block rows; row_ptr[n_nodes+1]
 * and col_idx[nnzb] are int32; column indices strictly ascending within a row;
 * the diagonal block present in every row; the pattern structurally
 * symmetric; vals[nnzb*b*b] FP64, each b x b block row-major.  The b dofs of a
 * node are interleaved in field order: field_of_dof[b] (HOST array) maps each
 * dof to its field block 0..F-1; it must be non-decreasing with all fields of
 * equal size (F = 1 or 2 with b in {3, 4, 6}, or F = 1 with b in {1, 2}).
 * Stored zeros count: the node graph is the stored pattern.
 *
 * Vectors are FP64, n_nodes*b entries, node-major (dof d of node i at
 * i*b + d).
 *
 * Pointers named "device" are CUDA device pointers (for example the storage
 * of torch CUDA tensors) on the current device; the caller owns them.  All
 * work is ordered on the CUDA stream `stream` (a cudaStream_t passed as
 * void*; NULL = the legacy default stream).  Entry points that return a
 * result to the host (status, iteration counts) synchronise that stream.
 *
 * Return values: BAMG_OK (0) on success, BAMG_NOT_CONVERGED (1) when FGMRES
 * stopped at max_iter (x then holds the last iterate and iters / relres are
 * set), or a negative BAMG_E* status.  amg_strerror() names a status.  On an
 * error no output other than the status is meaningful; a handle stays valid
 * (or stays NULL after a failed amg_setup).  No entry point traps the GPU:
 * device-side failures (a singular block, a non-finite value, a wait that
 * ran out) are reported through these statuses.
 * ---------------------------------------------------------------------------
 */
#ifndef BAMG_H
#define BAMG_H

#ifdef __cplusplus
extern "C" {
#endif

#define BAMG_OK 0
#define BAMG_NOT_CONVERGED 1
#define BAMG_EINVAL (-1)           /* bad argument, unsorted columns, missing diagonal block ... */
#define BAMG_ECUDA (-2)            /* a CUDA runtime call failed (includes out of memory)       */
#define BAMG_ESINGULAR_BLOCK (-3)  /* a node-block diagonal of one field is singular            */
#define BAMG_ESINGULAR_COARSE (-4) /* the coarsest operator is singular                          */
#define BAMG_ENAN (-5)             /* a non-finite value appeared in the solve                   */
#define BAMG_ETIMEOUT (-6)         /* an iterative setup phase did not finish in its bound       */
#define BAMG_EUNSUPPORTED (-7)     /* a size outside what this build handles                     */

typedef struct bamg_ctx* bamg_t; /* opaque; owns every device buffer of one hierarchy */

typedef struct {
    int max_levels;   /* at most this many levels (>= 1); default 10                          */
    int max_coarse;   /* coarsen while n_nodes*b > max_coarse; default 2500                    */
    int n_pre;        /* block Gauss-Seidel sweeps before the coarse correction; default 1     */
    int n_post;       /* sweeps after it; default 1                                            */
    double omega;     /* damping of Algorithm 1 (same for every field); default 0.5            */
    int cycle_prec;   /* 64: the V-cycle in FP64; 32: FP32 storage and arithmetic inside the
                         cycle (the outer FGMRES, its SpMV and the coarsest solve stay FP64)   */
    int use_graph;    /* 1: replay the V-cycle from a captured CUDA graph; default 1           */
    int tail_dofs;    /* levels whose n_nodes*b is at most this (and every level below them) run
                         as one thread-block-cluster launch per V-cycle; 0 = one launch per
                         step on every level; default 0                                        */
    int autotune;     /* row mapping of the smoother and SpMV kernels: 1 = time warp-per-row and
                         thread-per-row on every level at setup and keep the faster (default);
                         0 = warp-per-row everywhere; 2 = thread-per-row everywhere             */
} amg_params;

/* Fills *p with the defaults above (cycle_prec 64). */
void amg_default_params(amg_params* p);

/*
 * amg_setup - build the multigrid hierarchy of A (setup phase of the paper's
 * monolithic AMG: Sec. 4.4, standard and 2x2-block setup layouts).
 *   Per level: node graph of the stored pattern; aggregation (a disjoint
 *   cover of the nodes, greedy, Sec. 4.3.1) shared by all fields (cloned
 *   aggregates); piecewise-constant prolongator P (unit entries, every dof)
 *   and R = P^T, block diagonal across fields (eq. blocktransfers); Galerkin
 *   coarse operator A_{l+1} = R A_l P (Sec. 3); per-node, per-field inverses
 *   of the diagonal blocks and a colouring of the node graph for the
 *   smoother.  The coarsest operator is factorised (LU with partial pivoting)
 *   and inverted in FP64.
 * row_ptr, col_idx, vals: device, the BSR matrix (read only; may be freed
 *   after the call returns - the hierarchy holds its own copy).
 * n_nodes >= 1, nnzb >= n_nodes, b: see the conventions above.
 * field_of_dof: host, b entries.  p: host; NULL = defaults.
 * out: host; receives the handle (NULL on failure).
 * Errors: BAMG_EINVAL, BAMG_EUNSUPPORTED, BAMG_ECUDA, BAMG_ESINGULAR_BLOCK,
 *   BAMG_ESINGULAR_COARSE, BAMG_ETIMEOUT.
 */
int amg_setup(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int nnzb,
              int b, const int* field_of_dof, const amg_params* p, void* stream, bamg_t* out);

/*
 * amg_apply - z = MGV(0, r, 0): one V-cycle (Fig. 1 of the paper) from a zero
 *   initial guess: pre-smoothing with the damped block Gauss-Seidel smoother
 *   (Algorithm 1; the approximate solve of each field block is one
 *   multicolour node-block Gauss-Seidel sweep), residual, restriction,
 *   recursion, prolongation and correction, post-smoothing; the coarsest
 *   level is solved directly.
 * r, z: device, n_nodes*b FP64, must not overlap.  Asynchronous on `stream`.
 */
int amg_apply(bamg_t h, const double* r, double* z, void* stream);

/*
 * fgmres_solve - restarted flexible GMRES(restart) on the finest operator
 *   with the V-cycle as right preconditioner (the paper applies the V-cycle
 *   inside an outer GMRES: Sec. 3 and Sec. 5.1).  FP64 throughout the outer
 *   iteration.  Stops when the residual estimate |g_{j+1}| / ||b|| <= tol,
 *   then recomputes the true residual (and restarts if it is above tol).
 * b: device, right-hand side.  x: device, initial guess on entry, solution on
 *   exit.  restart in 1..64; max_iter >= 0 bounds the total inner steps.
 * iters, relres: host, may be NULL: total inner steps and the true relative
 *   residual ||b - A x|| / ||b|| at exit.  Synchronises `stream`.
 * Returns BAMG_OK, BAMG_NOT_CONVERGED, or an error (BAMG_ENAN, BAMG_ECUDA ...).
 */
int fgmres_solve(bamg_t h, const double* b, double* x, double tol, int restart, int max_iter,
                 int* iters, double* relres, void* stream);

/*
 * amg_solve_host - end-to-end solve with HOST buffers: copies A and the
 *   right-hand side to the device, runs amg_setup and fgmres_solve on
 *   `stream`, copies the solution back to x_host and frees everything it
 *   allocated.  Arguments as amg_setup / fgmres_solve, all arrays on the host
 *   (pinned memory gives the fastest copies).  x_host holds the initial guess
 *   on entry.
 */
int amg_solve_host(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int nnzb,
                   int b, const int* field_of_dof, const amg_params* p, const double* rhs_host,
                   double* x_host, double tol, int restart, int max_iter, int* iters, double* relres,
                   void* stream);

/*
 * amg_setup_batched - one hierarchy for nsys independent systems given as a
 *   single block-diagonal BSR matrix: system q owns the block rows
 *   sys_node_off[q] .. sys_node_off[q+1]-1 and couples only within them
 *   (column indices are global).  Every V-cycle step is one launch over all
 *   systems' rows; the aggregation, colouring and Galerkin products of the
 *   block-diagonal matrix are those of the systems separately (the greedy rules
 *   run in ascending node order and never cross a system); the coarsest level
 *   keeps one dense FP64 inverse per system.  All systems get the same number
 *   of levels (coarsening stops for the batch as a whole).
 * nsys >= 1; sys_node_off: HOST, nsys+1 strictly increasing ints, 0 and n_nodes
 *   at the ends.  Other arguments and errors as amg_setup; BAMG_EINVAL when a
 *   block couples two systems.
 */
int amg_setup_batched(int nsys, const int* sys_node_off, const int* row_ptr, const int* col_idx,
                      const double* vals, int n_nodes, int nnzb, int b, const int* field_of_dof,
                      const amg_params* p, void* stream, bamg_t* out);

/*
 * fgmres_solve_batched - FGMRES(restart) for every system of a batch, each
 *   with its own Krylov basis, Hessenberg matrix, rotations, stopping test and
 *   count (restarts happen for all systems together, after `restart` steps or
 *   when every system in the cycle has stopped); reductions are per system.
 * b, x: device, concatenated vectors (x: initial guess in, solution out).
 * iters, relres: host, nsys entries each (may be NULL): inner steps and the
 *   true relative residual of every system at exit.
 * Returns BAMG_OK when every system converged, BAMG_NOT_CONVERGED otherwise.
 */
int fgmres_solve_batched(bamg_t h, const double* b, double* x, double tol, int restart, int max_iter,
                         int* iters, double* relres, void* stream);

/* number of systems of the handle (1 for amg_setup) */
int amg_num_systems(bamg_t h);
/* node range of every system on level l: sys_node_off[nsys+1] (host) */
int amg_level_systems(bamg_t h, int level, int* sys_node_off);

/*
 * bsr_spmv - y = A x for a BSR matrix (the SpMV of the outer Krylov method and
 *   of every residual).  All pointers device; b in 1..8.  Asynchronous.
 */
int bsr_spmv(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int b,
             const double* x, double* y, void* stream);

/*
 * amg_colour_noalloc - the node colouring that amg_setup computes for the
 *   finest level (first fit in ascending node order over the stored pattern),
 *   computed without allocating any memory.  The paper has no counterpart:
 *   this entry point exists for callers that must not allocate at the time of
 *   the call - code running while a stream is captured into a CUDA graph
 *   (cudaMalloc is not allowed during capture), allocation-free real-time or
 *   callback paths, and applications whose device memory is reserved in
 *   advance by their own allocator.  It calls no cudaMalloc, cudaFree or
 *   allocating library routine; its work queues live in a fixed device array
 *   inside the library (320,016 bytes, held on every GPU that loads the
 *   library until the process exits).
 * row_ptr, col_idx: device, the BSR pattern (conventions above); n_nodes in
 *   1..40000 (BAMG_EUNSUPPORTED above 40000).
 * colour: device, n_nodes ints, receives the colour of every node.
 * n_colours: device, one int, receives the number of colours, or -1 if the
 *   pattern needs more than 255 colours or is not structurally symmetric.
 * The first call on a device looks up the device address of the scratch array
 *   (a host-side call, done once per device with that device current); make
 *   that first call before capturing a stream.  Asynchronous on `stream`.
 *   Every call on a device shares the one scratch array, which keeps the last
 *   call's contents (nothing in it needs to start at zero): calls that overlap
 *   on the GPU (different streams, no ordering between them) race and must
 *   not be issued.
 */
int amg_colour_noalloc(const int* row_ptr, const int* col_idx, int n_nodes, int* colour, int* n_colours,
                       void* stream);

/* ---- introspection (host outputs; synchronise the handle's setup stream) ---- */

/* number of levels (>= 1), or a negative status */
int amg_num_levels(bamg_t h);

/* sizes of level l: nodes, stored blocks, colours (0 on the coarsest) and the
 * number of aggregates it is coarsened into (0 on the coarsest). */
int amg_level_info(bamg_t h, int level, int* n_nodes, int* nnzb, int* n_colours, int* n_agg);

/* host copies of level l (any pointer may be NULL): row_ptr[n+1], col_idx[nnzb],
 * vals[nnzb*b*b] (FP64), agg[n] and colour[n] (not on the coarsest level),
 * dinv[n*F*fb*fb] (FP64 node-major, then field, then the fb x fb inverse
 * row-major; not on the coarsest level). */
int amg_level_copy(bamg_t h, int level, int* row_ptr, int* col_idx, double* vals, int* agg,
                   int* colour, double* dinv);

/* JSON summary of the hierarchy (levels, sizes, colours, bytes) into json[cap];
 * returns the length written (without the terminating zero) or a negative status. */
int amg_stats(bamg_t h, char* json, int cap);

/* ---- measurement ----
 * amg_profile(h, 1) makes the handle record a CUDA event pair around every
 * kernel it launches from then on (V-cycles run as direct launches, not from
 * the captured graph, while profiling is on) and prepares the per-launch
 * algorithmic byte and flop counts; amg_profile(h, 0) stops it.
 * amg_profile_read synchronises, returns for one kernel kind the summed
 * device time (ms), the number of launches and the summed algorithmic bytes
 * and flops since the last read of that kind, and clears them. */
#define BAMG_K_SMOOTH 0   /* one colour of one field step of block Gauss-Seidel */
#define BAMG_K_RESIDUAL 1 /* r = b - A u inside the cycle                     */
#define BAMG_K_RESTRICT 2
#define BAMG_K_PROLONG 3
#define BAMG_K_COARSE 4   /* dense coarsest solve                             */
#define BAMG_K_SPMV 5     /* FP64 SpMV / residual of the outer Krylov method  */
#define BAMG_K_KRYLOV 6   /* Gram-Schmidt, norms, rotations, updates          */
#define BAMG_K_CAST 7
#define BAMG_K_TAIL 8     /* the cluster launch that runs the coarse levels of one V-cycle */
#define BAMG_K_COUNT 9
int amg_profile(bamg_t h, int enable);
int amg_profile_read(bamg_t h, int kind, double* ms, long long* launches, double* bytes, double* flops);

/* number of kernels this library has launched in the process so far (kernels
 * replayed from a captured graph count once per replay) */
long long amg_launch_count(void);

/* frees every device buffer of the handle; NULL is accepted */
int amg_destroy(bamg_t h);

/* static description of a status code */
const char* amg_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* BAMG_H */
