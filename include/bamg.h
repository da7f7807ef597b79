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
 * dof to its field block 0..F-1; it must start at 0 and be non-decreasing in
 * steps of 0 or 1 (BAMG_EINVAL otherwise).  With fields of equal size fb = b / F,
 * (b, fb) must be one of: fb = b for b = 1..8 (one field), fb = 2 for
 * b = 4, 6, 8, fb = 3 for b = 6, fb = 4 for b = 8 (BAMG_EUNSUPPORTED otherwise).
 * Fields of unequal size (Algorithm 1 takes field blocks of any width, e.g.
 * velocity | pressure = {2, 1}) run padded: every field is filled up to the
 * widest field's size fmax with dummy dofs that have one nonzero, on their own
 * diagonal (the largest magnitude of the node's diagonal block), no coupling,
 * a zero right-hand side and a zero iterate.  They stay zero in every step, so
 * the results at the given dofs are the method's on the unpadded system (up to
 * the order of rounding); the cost is that of the padded block size
 * b' = F * fmax, which with fb = fmax must be a supported pair above
 * (BAMG_EUNSUPPORTED otherwise, e.g. {3, 3, 1}).  Vectors passed to the calls
 * keep the given size n_nodes*b; the introspection calls describe the padded
 * levels (amg_block_size gives b').  Unequal fields take the tentative P, no
 * learned weights and sub_solver 0 (BAMG_EUNSUPPORTED otherwise).
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

#include <stdint.h>

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
                         thread-per-row on every level at setup (smoother: also in half-size
                         CTAs) and keep the fastest (default); 0 = warp-per-row everywhere;
                         2 = thread-per-row everywhere; 3 = as 2 with half-size smoother CTAs;
                         4 = as 2 with four lanes per smoother row (each a quarter of the
                         row's blocks) and per row of the FP64 outer SpMV; 5 = as 4 with every node's row staged in shared memory
                         by asynchronous copies ahead of use (levels whose steps read whole blocks:
                         one field, or the field-major layout; elsewhere 4; the same values
                         as 4 bit for bit); 6 = four warps per smoother node, one node per
                         CTA, thread-per-row SpMV (long rows on small levels); 7 / 8 = sixteen /
                         eight lanes per smoother node, each lane taking whole blocks of the
                         row (several loads in flight per lane; blocks of at most 16 values of
                         the field rows, fb * b <= 16, elsewhere 4); 1 also times the
                         variants of 3 to 8, and the persistent sweep (see sweep). With 1 the choices are kept for the
                         life of the process per level shape (device, sizes of the level and
                         of its colours, block and field shape, precision, layout, launch mode,
                         sub-solver): a later setup of a level of the same shape reuses them
                         without timing (amg_stats: tune_cached)                               */
    /* ---- beyond the paper: smoothed transfers, per-node damping, learned weights ---- */
    int smooth_p;     /* 0: tentative P (default); 1: on every coarsened level the smoothed
                         P_f = (I - W_f D_ff^{-1} A_ff) P^_f per field (see amg_setup)        */
    double omega_p;   /* W_f of every aggregate when omega_p_arr is NULL; default 0           */
    /* host arrays read during amg_setup only, consumed level by level from the finest:
     * omega_s_arr holds n_l*F smoother dampings (node-major, then field) for every level
     * that gets a smoother, omega_p_arr n_agg_l*F smoothing weights for every coarsened
     * level (with smooth_p = 1).  NULL: omega / omega_p everywhere.  Lengths that do not
     * match the hierarchy exactly are BAMG_EINVAL. */
    const double* omega_s_arr;
    long long omega_s_len;
    const double* omega_p_arr;
    long long omega_p_len;
    /* learned weights: host, BAMG_MLP_NPARAMS floats (layout at mlp_forward) or NULL.
     * When set, every coarsened level takes its smoother damping (head 0) and its P
     * smoothing weights (head 1) from the network applied to the level's features
     * (amg_features) with FP16 weights, clipped as in mlp_clip; a level smooths P only
     * when a weight of its aggregates is nonzero after the clip.  Overrides the arrays
     * above and smooth_p. */
    const float* mlp;
    int pr_storage;   /* values of explicit (smoothed) P and R inside an FP32 cycle: 32 (default)
                         or 16 = BF16 storage, FP32 arithmetic                                 */
    int mlp_levels;   /* with mlp: the network gives the weights of levels 0..mlp_levels-1 (the
                         depths it was trained on); deeper levels keep omega and the tentative P.
                         0 (default) = every level                                             */
    int use_pdl;      /* 1 (default): the V-cycle's kernels are launched as programmatic
                         dependent launches (each is scheduled while its predecessor drains,
                         loads the matrix entries of its first block, then waits for its
                         inputs in hardware); 0: ordinary launches. Same results (bitwise).   */
    int coarse_prec;  /* precision of the coarsest direct solve (LU with partial pivoting, its
                         inverse, and the per-cycle product with it) of a single system:
                         64 (default) or 32 (FP32, only with cycle_prec 32: GB300 runs FP32 at
                         64 times its FP64 rate). The LU is of the coarsest Galerkin matrix
                         rounded to FP32; a pivot below 1e-9 times its infinity norm reports
                         BAMG_ESINGULAR_COARSE (pivots near FP32 rounding make the coarse solve
                         inexact along near-null directions; FGMRES absorbs that, at the cost
                         of iterations if any). Batches keep FP64 per-system inverses.        */
    int tail_grid;    /* with tail_dofs: 1 = the levels of the tail run as one cooperative
                         launch over every SM with a grid barrier between the recorded phases
                         (instead of one thread-block cluster); the V-cycle is then launched
                         directly, not from a CUDA graph. A barrier wait that runs out (it
                         cannot while all CTAs are resident, which the cooperative launch
                         guarantees) is reported as BAMG_ETIMEOUT by fgmres_solve. Default 0. */
    int value_layout; /* FP32 copy of a level's values in a cycle with F > 1 fields: 0 (default) =
                         field-major rows (each block row holds field 0's rows of all its blocks,
                         then field 1's, ...) on levels whose FP32 values exceed the L2 cache,
                         block-major elsewhere; 1 = block-major everywhere; 2 = field-major
                         everywhere. Same results either way (bitwise).                       */
    int sweep;        /* smoother launches per field step of Algorithm 1: 0 (default) = with
                         autotune 1, one persistent launch for all colours of the step (tiles
                         taken in colour order, each waiting in bounded spins for the tiles of
                         its lower-colour neighbours) where it times faster than one launch per
                         colour, else one launch per colour; 1 = one launch per colour always;
                         2 = the persistent launch on every level (one thread per scalar row);
                         3 = as 2 with four lanes per row. The persistent launch computes the
                         values of the thread-per-row (2) or four-lanes (3) kernels bit for bit.
                         A wait that runs out is reported as BAMG_ETIMEOUT by fgmres_solve.    */
    int sub_solver;   /* the approximate solve of A_ff inside each field step of Algorithm 1:
                         0 (default) = one multicolour node-block Gauss-Seidel sweep from zero;
                         1 = ILU(0) of A_ff (Sec. 4.3.2, the paper's sub-solver; Sec. 5.1) with
                         the nodes eliminated in colour order (colour, then index), its forward
                         and backward solves one launch per colour each (the nodes of a colour
                         do not couple). With 1 or 2 the cycle runs without the tail and the
                         persistent sweep (tail_dofs, tail_grid, sweep are ignored); a zero
                         pivot is BAMG_ESINGULAR_BLOCK, a row of more than 64 blocks of its
                         field BAMG_EUNSUPPORTED; 2 = restricted additive Schwarz (Sec. 5: one
                         Schwarz iteration per field block): one subdomain per aggregate and
                         field block, the aggregate extended by schwarz_overlap layers of
                         neighbours in the graph of A_ff, solved exactly (LU with partial
                         pivoting in FP64 at setup; the rows of the local inverse that belong
                         to the aggregate are kept), every node taking its own aggregate's
                         local solution; at most 160 unknowns per subdomain (else
                         BAMG_EUNSUPPORTED), a singular local matrix BAMG_ESINGULAR_BLOCK.     */
    int schwarz_overlap; /* layers of neighbours added to each Schwarz subdomain: 1 (default,
                         the paper's overlap one) or 0 (block Jacobi over the aggregates)     */
    int ortho;        /* Arnoldi orthogonalisation of fgmres_solve: 0 (default) = classical
                         Gram-Schmidt with a second projection only where the norm of w left
                         after the first is below 0.01 of the norm before it (the selective
                         test of Daniel, Gragg, Kaufman and Stewart with eta = 0.01); 1 =
                         classical Gram-Schmidt applied twice at every step. Batches use 1.   */
    int coarse_tc;    /* FP32 coarsest solve (coarse_prec 32) of 224 to 2048 unknowns: 1 (default)
                         = blocked LU with partial pivoting (panels of 16 columns) and the
                         inverse by blocked triangular solves on the identity, every matrix
                         product of both on the tensor cores (tcgen05 kind::tf32, each FP32
                         operand split into two TF32 parts, three products per pair: FP32
                         accuracy); 0 = the CUDA-core cooperative LU and column-by-column
                         inverse. Pivots may differ between the two (ties, rounding); both
                         are backward stable.                                                 */
    int inner_sweeps; /* multicolour Gauss-Seidel sweeps of the sub-solve A_ff x~ = r_f in each
                         field step of Algorithm 1 (sub_solver 0): 1 (default) = one sweep from
                         zero; k in 2..64 = k sweeps, the first from zero, each later one taking
                         the previous sweep's x~ for the neighbours of higher colour (x~ tends to
                         A_ff^{-1} r_f as k grows). k > 1 forms r_f = b_f - A_f* x for all nodes
                         first, then one launch per colour and sweep; it runs without the tail,
                         the persistent sweep and the upper-part residual, and needs sub_solver 0
                         and dof fields (amg_setup, amg_setup_batched; else BAMG_EINVAL).  0 is
                         taken as 1.                                                          */
} amg_params;

/* Fills *p with the defaults above (cycle_prec 64, tentative P, no learned weights). */
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
 *   With smooth_p = 1 (or learned weights) the prolongator of a coarsened
 *   level is P_f = (I - W_f D_ff^{-1} A_ff) P^_f for every field f: the
 *   tentative P^ smoothed by one damped block-Jacobi step on the field block
 *   A_ff only, so P stays block diagonal across fields; W_f = diag over fine
 *   nodes i of the weight of agg(i).  Stored block (i, J) has F sub-blocks of
 *   fb x fb; pattern of row i = the distinct agg(j) over the stored j of row
 *   i.  R = P^T is stored explicitly, and A_{l+1} = R (A_l P) is a general
 *   sparse triple product whose patterns are structural unions (no dropping).
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
 *   on entry.  The matrix values are copied on a second stream straight into
 *   the hierarchy's level-0 array while the setup's pattern phases (pattern
 *   check, aggregation of level 0, the Galerkin pattern) run on `stream`; the
 *   first use of the values waits for that copy.  With pageable memory the
 *   copy is staged by the driver and does not overlap.
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

/*
 * amg_solve_batched_host - end-to-end solve of a batch with HOST buffers:
 *   copies the block-diagonal A and the right-hand sides to the device, runs
 *   amg_setup_batched and fgmres_solve_batched on `stream`, copies the
 *   solutions back to x_host (initial guesses on entry) and frees everything
 *   it allocated.  Arguments and statuses as those two calls, all arrays on
 *   the host (pinned memory gives the fastest copies).
 */
int amg_solve_batched_host(int nsys, const int* sys_node_off, const int* row_ptr, const int* col_idx,
                           const double* vals, int n_nodes, int nnzb, int b, const int* field_of_dof,
                           const amg_params* p, const double* rhs_host, double* x_host, double tol, int restart,
                           int max_iter, int* iters, double* relres, void* stream);

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
 *   pattern needs more than 255 colours or breaks the conventions above (a
 *   row bound or column out of range, columns not strictly ascending, a
 *   missing diagonal block, or a block (i, j) stored without (j, i)); the
 *   colours are then -1 where not computed.
 * The first call on a device looks up the device address of the scratch array
 *   (a host-side call, done once per device with that device current); make
 *   that first call before capturing a stream.  Asynchronous on `stream`.
 *   Every call on a device shares the one scratch array, which keeps the last
 *   call's contents (nothing in it needs to start at zero): calls that overlap
 *   on the GPU (different streams, no ordering between them) race and must
 *   not be issued.  The device address found by the first call is kept for
 *   the life of the process: do not call this entry point after a
 *   cudaDeviceReset.
 */
int amg_colour_noalloc(const int* row_ptr, const int* col_idx, int n_nodes, int* colour, int* n_colours,
                       void* stream);

/* ---- learned damping (beyond the paper: the paper fixes one damping near 0.5,
 *      Sec. 5, and shows that its value decides convergence for small viscosity) ---- */

#define BAMG_NFEAT 8
#define BAMG_MLP_H 64
#define BAMG_MLP_OUT 2
/* trained parameters: W1[H][NFEAT], b1[H], W2[H][H], b2[H], W3[OUT][H], b3[OUT] */
#define BAMG_MLP_NTRAIN (BAMG_MLP_H * BAMG_NFEAT + BAMG_MLP_H + BAMG_MLP_H * BAMG_MLP_H + BAMG_MLP_H + \
                         BAMG_MLP_OUT * BAMG_MLP_H + BAMG_MLP_OUT)
/* followed by the fixed input normalisation xm[NFEAT], xs[NFEAT] */
#define BAMG_MLP_NPARAMS (BAMG_MLP_NTRAIN + 2 * BAMG_NFEAT)

/*
 * amg_features - the network inputs of one level (computed in FP64, stored
 * FP32).  Node i, field f (Frobenius norms of fb x fb sub-blocks of row i):
 * d = ||A_ff[i,i]||, o = sum_{j!=i} ||A_ff[i,j]||, c = sum_j sum_{g!=f}
 * ||A_fg[i,j]||; features: log d, o/d, c/(d+o), log d - mean_g log d_g,
 * tr(A_ff[i,i])/(sqrt(fb) d), log |agg(i)|, level, f.  Aggregate I, field f:
 * the mean of its members' rows.
 * row_ptr, col_idx, vals, agg (n_nodes), node_feat ([n_nodes][F][NFEAT]),
 * agg_feat ([n_agg][F][NFEAT], may be NULL): device.  field_of_dof: host.
 * Errors: BAMG_EINVAL (sizes, aggregate ids out of range), BAMG_EUNSUPPORTED
 * (block layout), BAMG_ESINGULAR_BLOCK (a zero diagonal sub-block), BAMG_ECUDA.
 */
int amg_features(const int* row_ptr, const int* col_idx, const double* vals, int n_nodes, int b,
                 const int* field_of_dof, const int* agg, int n_agg, int level, float* node_feat,
                 float* agg_feat, void* stream);

/* params (device, BAMG_MLP_NPARAMS floats) -> params16 (device, FP16 bit patterns, same
 * count, round to nearest even).  Errors: BAMG_EINVAL (NULL), BAMG_ECUDA. */
int mlp_pack(const float* params, uint16_t* params16, void* stream);

/*
 * mlp_forward - y[n][OUT] = MLP(x[n][NFEAT]) with FP16 parameters and FP32
 * arithmetic: xh = (x - xm) * xs, h1 = tanh(W1 xh + b1), h2 = tanh(W2 h1 + b2),
 * y = W3 h2 + b3.  All pointers device.  n = 0 is a no-op.
 * Errors: BAMG_EINVAL (n < 0, NULL), BAMG_ECUDA.
 */
int mlp_forward(const uint16_t* params16, const float* x, int n, float* y, void* stream);

/*
 * mlp_grad - loss = (1/n) sum_r (y[r][head[r]] - t[r])^2 over the rows of x
 * and its gradient grad[BAMG_MLP_NTRAIN] with respect to the trained
 * parameters, evaluated at the FP16 parameters (FP32 arithmetic; the sum
 * over rows is deterministic).  All pointers device; loss: 1 float.
 * Errors: BAMG_EINVAL (n < 1, head outside 0..OUT-1 is not checked), BAMG_ECUDA.
 */
int mlp_grad(const uint16_t* params16, const float* x, const float* t, const int* head, int n, float* grad,
             float* loss, void* stream);

/*
 * mlp_adam - one Adam step (bias-corrected moments, step count t >= 1) on
 * the trained parameters of params (FP32 master copy), then params16 =
 * FP16(params).  params, params16, grad, m, v: device.
 * Errors: BAMG_EINVAL (t < 1, NULL), BAMG_ECUDA.
 */
int mlp_adam(float* params, uint16_t* params16, const float* grad, float* m, float* v, int t, float lr,
             float beta1, float beta2, float eps, void* stream);

/* the weight ranges applied to the network outputs: head 0 (smoother damping)
 * [0.05, 1.5]; head 1 (P smoothing) [0, 1.5] with values below 0.05 set to 0 */
double mlp_clip(int head, double w);

/*
 * amg_set_omega - replace the smoother damping of level `level` (< levels-1)
 * by omega_s (device, n_nodes*F doubles, node-major then field); the
 * hierarchy is otherwise unchanged (used to search dampings without a new
 * setup).  Errors: BAMG_EINVAL, BAMG_ECUDA.
 */
int amg_set_omega(bamg_t h, int level, const double* omega_s, void* stream);

/*
 * amg_select - the fallback rule of the learned hierarchy: solve A x = b
 * (device, x0 = 0) with FGMRES preconditioned by each hierarchy (same matrix)
 * and keep the plain one unless the learned one converges in no more
 * iterations.  *choice = 0 (learned) or 1 (plain); iters_learned /
 * iters_plain (host, may be NULL) receive the counts.
 * Errors: those of fgmres_solve other than BAMG_NOT_CONVERGED; BAMG_EINVAL on
 * hierarchies of different sizes.
 */
int amg_select(bamg_t learned, bamg_t plain, const double* b, double tol, int restart, int max_iter,
               int* choice, int* iters_learned, int* iters_plain, void* stream);

/* damping weights of level l < levels-1 (host copies): omega_s[n*F],
 * omega_p[n_agg*F] (zeros on a level with the tentative P); either may be NULL */
int amg_level_omega(bamg_t h, int level, double* omega_s, double* omega_p);
/* explicit prolongator of level l (host): *nnz = stored blocks (0: tentative P);
 * then copies into p_rp[n+1], p_ci[nnz], p_v[nnz][F][fb][fb] where not NULL */
int amg_level_p(bamg_t h, int level, int* nnz, int* p_rp, int* p_ci, double* p_v);

/* ---- introspection (host outputs; synchronise the handle's setup stream) ---- */

/* number of levels (>= 1), or a negative status */
int amg_num_levels(bamg_t h);

/* dofs per node of the hierarchy's levels: b, or the padded b' of fields of
 * unequal size (see the conventions above); a negative status for a null handle */
int amg_block_size(bamg_t h);

/* sizes of level l: nodes, stored blocks, colours (0 on the coarsest) and the
 * number of aggregates it is coarsened into (0 on the coarsest). */
int amg_level_info(bamg_t h, int level, int* n_nodes, int* nnzb, int* n_colours, int* n_agg);

/* copies of level l into host or device memory (any pointer the CUDA runtime
 * addresses; any may be NULL): row_ptr[n+1], col_idx[nnzb],
 * vals[nnzb*b*b] (FP64), agg[n] and colour[n] (not on the coarsest level),
 * dinv[n*F*fb*fb] (FP64 node-major, then field, then the fb x fb inverse
 * row-major; not on the coarsest level). */
int amg_level_copy(bamg_t h, int level, int* row_ptr, int* col_idx, double* vals, int* agg,
                   int* colour, double* dinv);

/* amg_level_ilu - the FP64 ILU(0) factors of level l (sub_solver 1: the
 * incomplete factorisation of every field's A_ff in colour order, Sec. 4.3.2)
 * into lu[F*nnzb*fb*fb] (host or device): field-major planes, then block k,
 * then the fb x fb sub-block row-major; entry (k, r, c) of block (i, j)
 * holds L (unit lower, strictly before the scalar diagonal in elimination
 * order, whose diagonal 1 is not stored) or U.  BAMG_EINVAL on the coarsest
 * level or without ILU. */
int amg_level_ilu(bamg_t h, int level, double* lu);

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
/* The same for the launches of one hierarchy level (level -1: the outer
 * FGMRES kernels, which belong to no level); clears only those. */
int amg_profile_read_level(bamg_t h, int kind, int level, double* ms, long long* launches, double* bytes,
                           double* flops);

/* Dense kernels of the coarsest direct solve (Sec. 4.1), callable on their own;
 * both synchronise the stream and allocate (and free) their scratch.
 *
 * amg_dense_inverse_f32: inv = a^-1 for a row-major nd x nd FP32 matrix a on
 * the device (a is not modified: a copy is factored), by LU with partial
 * pivoting.  method 1: the tensor-core path of coarse_tc (0 < nd <= 2048, else
 * BAMG_EUNSUPPORTED); 0: the CUDA-core LU and column-by-column inverse.
 * BAMG_ESINGULAR_COARSE: a pivot below 1e-9 ||a||_inf; BAMG_ETIMEOUT: a
 * bounded wait of a tensor-core kernel ran out.
 *
 * amg_gemm_tc_f32: C += A B, row-major FP32 on the device (A m x k, B k x n,
 * C m x n; leading dimensions lda >= k, ldb >= n, ldc >= n; C may not overlap
 * A or B), on the tensor cores: tcgen05 kind::tf32 with each operand split
 * into two TF32 parts and three products per pair (FP32 accuracy). */
int amg_dense_inverse_f32(int nd, const float* a, float* inv, int method, void* stream);
int amg_gemm_tc_f32(int m, int n, int k, const float* A, int lda, const float* B, int ldb, float* C, int ldc,
                    void* stream);

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
