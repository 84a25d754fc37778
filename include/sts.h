/*
 * sts.h -- C ABI of the GB300 block r1-sparse Jacobian library (libsts.so).
 *
 * The library stores a first-order finite-volume Jacobian the way the paper
 * does (Gouasmi & Murman, "Sparse Data Structures for Efficient State-to-State
 * Kinetic Simulations", Sections 4-6): every nonzero block is a sparse matrix
 * plus a few rank-one pairs,
 *
 *     J_ij = S_ij + sum_k u_ijk v_ijk^T                  (Section 4.3, Eq. r1_flux_left/right, r1_chem)
 *
 * and offers the Jacobian-vector product (Section 5.2), a block-Jacobi
 * preconditioner applied through the Sherman-Morrison-Woodbury formula
 * (Section 6, steps SMW-1..3), restarted right- or left-preconditioned (F)GMRES
 * (Section 6, Eqs. right_precond_system / left_precond_system), the transposed
 * operators and the adjoint outer products used to differentiate x = J^-1 b.
 * Pair counts may differ from block to block (BR1-BSR pair_indptr, Section 5.1).
 * A second handle type, sts_flow_t, generates the residual and the Jacobian of a
 * toy HLL-flux flow model directly in this form (two rank-one pairs per face,
 * Section 4.1) and runs an implicit Newton pseudo-time step around the solver
 * (Section 3.3).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every function returns an sts_status; STS_OK (0) on success.  On failure
 *   sts_last_error() returns a message for the calling thread.  No C++
 *   exception crosses this boundary.
 * - Cells are numbered 0..n_cells-1.  The block size b is the number of
 *   unknowns per cell (b = N + 3 for N quantum levels, two momenta and one
 *   energy, Section 2.1; any b >= 1 is accepted).
 * - Vectors have n_cells * b entries.  Their layout is fixed per handle by
 *   sts_jac_desc.vec_layout: STS_LAYOUT_CELL_MAJOR stores cell c's b values
 *   contiguously (x[c*b + p]); STS_LAYOUT_COMPONENT_MAJOR stores component p of
 *   all cells contiguously (x[p*n_cells + c]), the layout the kernels use
 *   internally, so it avoids two transposes per call.
 * - "device" pointers are CUDA device (or managed) memory on the current
 *   device; "host" pointers are ordinary host memory.  The library never takes
 *   ownership of caller memory; arguments need to stay valid only for the
 *   duration of the call (asynchronous calls: until the work on the handle's
 *   stream has finished).
 * - All GPU work is issued on the stream given at creation.  Calls marked
 *   "asynchronous" return before the work finishes; the others synchronise
 *   that stream before returning.
 * - A handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef STS_H
#define STS_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int sts_status;

enum {
    STS_OK = 0,
    STS_ERR_INVALID_ARG = 1,   /* a size, pointer, index array or option is invalid   */
    STS_ERR_ALLOC = 2,         /* device or host allocation failed                      */
    STS_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed          */
    STS_ERR_SINGULAR = 4,      /* zero pivot in S_ii or singular capacitance C_k        */
    STS_ERR_NOT_CONVERGED = 5, /* GMRES hit max_iters; the returned x is still valid    */
    STS_ERR_NUMERIC = 6,       /* NaN or Inf met in a residual or Krylov quantity       */
    STS_ERR_TIMEOUT = 7,       /* a bounded device-side wait gave up (see bjacobi_apply) */
    STS_ERR_NOT_SETUP = 8,     /* block-Jacobi used before sts_jac_bjacobi_setup        */
    STS_ERR_COMM = 9           /* a communication or operation callback reported failure */
};

enum { STS_F64 = 0, STS_MIXED = 2 };                       /* sts_jac_desc.dtype        */
enum { STS_LAYOUT_CELL_MAJOR = 0, STS_LAYOUT_COMPONENT_MAJOR = 1 };
enum { STS_REP_FACTORED = 0, STS_REP_DENSE_BSR = 1 };      /* sts_jac_desc.representation */
enum { STS_PRECOND_BJ = 0, STS_PRECOND_NONE = 1 };         /* sts_gmres_opts.precond     */
enum { STS_ARNOLDI_GRAPH = 0, STS_ARNOLDI_HOST = 1 };      /* sts_gmres_opts.arnoldi     */

typedef struct sts_jac_s *sts_jac_t;

/*
 * Problem statement of one Jacobian (Section 3.4: one block per cell and per
 * interior face; Section 5.1: BSR index arrays fixed by the mesh adjacency;
 * Section 6, Eq. R1_Block_Jacobian: A_k = A_k^0 + U_k V_k^T).
 *
 *   n_cells, block_size    number of cells and unknowns per cell (b)
 *   n_levels               quantum levels N (informational; b = N + 3 in the paper's model)
 *   dtype                  STS_F64: FP64 operators only.
 *                          STS_MIXED: also keep FP32 copies of the operators for the
 *                          mixed-precision solver and the *_f32 calls (+50% memory).
 *   vec_layout             layout of every vector argument (see above)
 *   representation         STS_REP_FACTORED: the paper's S + rank-one storage.
 *                          STS_REP_DENSE_BSR: the standard dense-block BSR storage of
 *                          Section 3.4 (blocks assembled once, b*b values each), kept
 *                          as the baseline the factored storage is measured against.
 *   block_indptr[n_cells+1], block_indices[nnzb]   HOST int32.  Block CSR of the mesh
 *                          adjacency including the diagonal; each row sorted
 *                          ascending, no duplicates, every row holds its diagonal.
 *   d_indptr[b+1], d_indices[nnz_d]   HOST int32.  CSR pattern of S_ii, shared by all
 *                          diagonal blocks; rows sorted, every diagonal entry present.
 *   o_indptr[b+1], o_indices[nnz_o]   HOST int32.  CSR pattern of S_ij (i != j), shared
 *                          by all off-diagonal blocks (may be empty).
 *   r_diag, r_off          rank-one pairs per diagonal / off-diagonal block (>= 0),
 *                          used when pair_indptr is NULL.  The BR1-BSR pair_indptr of
 *                          Section 5.1 then follows from them: pairs are numbered in
 *                          block order.
 *   pair_indptr[nnzb+1]    HOST int32 or NULL.  The BR1-BSR pair_indptr of Section 5.1
 *                          for pair counts that differ from block to block (Section 4.3:
 *                          a diagonal block gathers one pair per source term and two per
 *                          face, so boundary cells hold fewer): the pairs of block k are
 *                          [pair_indptr[k], pair_indptr[k+1]).  pair_indptr[0] = 0 and it
 *                          never decreases, else STS_ERR_INVALID_ARG.  When given,
 *                          r_diag and r_off are ignored.  The handle stores every block
 *                          with the largest count of its kind (diagonal / off-diagonal),
 *                          the missing pairs as exact zeros, so memory and time follow
 *                          those maxima.
 *   S, U, V                FP64 values.  S: block order, nnz_d values per diagonal
 *                          block and nnz_o per off-diagonal block, each in pattern
 *                          order.  U (column_data) and V (row_data): [n_pairs][b].
 *                          Device pointers, or host pointers if values_on_host = 1.
 *   values_on_host         0: S/U/V are device pointers; 1: host pointers
 *   enable_transpose       1: also build the transposed operators (needed by
 *                          trans = 1 calls, the adjoint solve and sts_jac_grad)
 *   stream                 cudaStream_t to issue all work on (NULL = legacy default)
 */
typedef struct {
    int n_cells;
    int block_size;
    int n_levels;
    int dtype;
    int vec_layout;
    int representation;
    const int *block_indptr;
    const int *block_indices;
    const int *d_indptr;
    const int *d_indices;
    const int *o_indptr;
    const int *o_indices;
    int r_diag;
    int r_off;
    const int *pair_indptr;
    const double *S;
    const double *U;
    const double *V;
    int values_on_host;
    int enable_transpose;
    void *stream;
} sts_jac_desc;

/* Options of sts_gmres_solve.  Zero-initialised fields take the defaults shown. */
typedef struct {
    int restart;          /* Krylov dimension m per cycle (default 30)                        */
    int max_iters;        /* total Arnoldi steps over all cycles (default 1000)               */
    double rtol;          /* stop when ||b - J x|| / ||b|| <= rtol, true FP64 residual (1e-10) */
    int precond;          /* STS_PRECOND_BJ (default, 0) or STS_PRECOND_NONE                  */
    int flexible;         /* 1: FGMRES (stores the preconditioned vectors Z)                  */
    int trans;            /* 1: solve J^T x = b with the transposed operators                 */
    int mixed;            /* 1: FP32 matvec + FP32 block-Jacobi inside FP64 FGMRES            */
    double inner_rtol;    /* mixed mode: relative reduction per cycle (default 1e-6)          */
    int vectors_on_host;  /* 1: b and x are host pointers (copied in and out inside the call) */
    double *history;      /* optional host array [max_iters]: rotated residual / ||b|| per step */
    int left;             /* 1: left preconditioning, (M A) x = M b (Section 6, Eq.
                             left_precond_system); needs STS_PRECOND_BJ, not mixed       */
    int arnoldi;          /* STS_ARNOLDI_GRAPH (default, 0): for right preconditioning in
                             FP64 with restart <= 64, each cycle's Arnoldi steps run as
                             one CUDA graph, every step under a conditional node nested
                             in the previous step's body, which a device-side Givens
                             kernel switches off once the cycle is done: the host
                             synchronises once per cycle.  The graph of a (direction,
                             preconditioning) is built on first use and kept.
                             STS_ARNOLDI_HOST (1): the host rotates after every step (a
                             synchronisation per step); left and mixed solves always do */
} sts_gmres_opts;

/* Result of sts_gmres_solve. */
typedef struct {
    int iterations;       /* Arnoldi steps taken                                   */
    int restarts;         /* cycles completed                                      */
    int converged;        /* 1 if the true relative residual reached rtol          */
    double true_rel_residual;  /* ||b - J x|| / ||b||, recomputed in FP64 at the end */
    int matvecs;          /* FP64 products J x (or J^T x) the solve made: one per
                             Arnoldi step except in mixed mode, one per
                             true-residual check except the first when x0 = 0 */
    int applies;          /* FP64 block-Jacobi applies: one per Arnoldi step
                             when preconditioned (not in mixed mode), plus one
                             per cycle with left preconditioning              */
} sts_gmres_info;

/* Message of the last failed call on this thread ("" if none).  Never NULL. */
const char *sts_last_error(void);

/* Library version string. */
const char *sts_version(void);

/*
 * Create a Jacobian handle from a problem statement (see sts_jac_desc).
 * Validates every index array (sorted, in range, diagonal present, sizes),
 * builds the kernels' internal layouts on the host and copies and repacks the
 * values on the device.  Synchronous.  *out receives the handle (NULL on error).
 * Errors: STS_ERR_INVALID_ARG, STS_ERR_ALLOC, STS_ERR_CUDA.
 */
sts_status sts_jac_create(const sts_jac_desc *desc, sts_jac_t *out);

/*
 * Replace the values S, U, V (same layouts and residency flag as at creation),
 * e.g. after a Newton update.  Invalidates the block-Jacobi setup.  Asynchronous.
 * With values_on_host = 1 the host arrays are copied through a device staging
 * buffer that the handle allocates on the first update (or creation) from host
 * memory and keeps until destroy (it counts in sts_jac_memory); the host arrays
 * must stay valid until the handle's stream has finished the copies.
 */
sts_status sts_jac_update_values(sts_jac_t h, const double *S, const double *U,
                                 const double *V, int values_on_host);

/*
 * y = J x (trans = 0) or y = J^T x (trans = 1), FP64, device vectors in the
 * handle's layout (Section 5.2: c_p = v_p . x_col(p) for every pair, then
 * y_i = sum_j S_ij x_j + sum_{p in row i} c_p u_p).  x and y must not overlap.
 * trans = 1 needs enable_transpose.  Asynchronous.
 */
sts_status sts_jac_matvec(sts_jac_t h, const double *x, double *y, int trans);

/*
 * The same product as sts_jac_matvec (same arguments, same result), for
 * callers that must not allocate device memory while they run: code that has
 * reserved all device memory up front under a fixed budget, or that cannot
 * afford cudaMalloc / cudaFree, which may synchronise the whole device, in the
 * middle of its stream work.  This call allocates nothing: the per-block dot
 * products of the first pass go to a library-owned static device buffer of
 * 4 MiB (2^19 doubles) instead of handle memory.  That buffer exists on every
 * GPU that loads the library until the process exits.
 *
 * Limit: the handle needs ceil(n_cells / 32) x (dot tasks per cell) x 32
 * doubles of scratch, at most 2^19 (for example 16384 cells with 21 dot tasks,
 * the 128x128, N = 60 workload, use 344064); larger handles get
 * STS_ERR_INVALID_ARG and should use sts_jac_matvec.
 * The handle's device (the one current at sts_jac_create) must be the current
 * device during the call, else STS_ERR_INVALID_ARG.  The first call for a
 * handle of a given device looks up that device's buffer address with
 * cudaGetSymbolAddress; make that first call before any stream capture.  All calls share the one buffer: calls that overlap on
 * the GPU (different streams or threads) race on it and must be serialised by
 * the caller.  Factored representation only; trans = 1 needs enable_transpose.
 * The paper has no counterpart to this entry point.  Asynchronous.
 */
sts_status sts_jac_matvec_noalloc(sts_jac_t h, const double *x, double *y, int trans);

/* FP32 operator, FP32 device vectors (needs dtype STS_MIXED).  Asynchronous. */
sts_status sts_jac_matvec_f32(sts_jac_t h, const float *x, float *y, int trans);

/*
 * Block-Jacobi setup (Section 6).  Factored representation: per cell a static-
 * pivot sparse LU of S_ii on the symbolic schedule of the shared pattern,
 * W_k = S_ii^-1 U_k, C_k = I + V_k^T W_k (FP64) and C_k^-1.  Dense-BSR
 * representation: per-cell dense LU with partial pivoting.  Synchronous.
 * Errors: STS_ERR_SINGULAR when a pivot fails |p| > 1e-14 * max|row of S_ii|, or
 * C_k is singular; the message names the first failing cell.  STS_ERR_TIMEOUT
 * when an apply since the last check reported a timed-out wait (see below).
 */
sts_status sts_jac_bjacobi_setup(sts_jac_t h);

/*
 * z = M x with M = blockdiag(J)^-1 (trans = 0) or M^T x (trans = 1):
 * x0 = S_ii^-1 x_i, t = V^T x0, z_i = x0 - W C^-1 t (Section 6 SMW-1..3, with the
 * minus sign the Woodbury identity requires).  FP64 device vectors; x and z
 * must not overlap.  Errors: STS_ERR_NOT_SETUP.  Asynchronous.
 * The structured-pattern kernel streams its coefficients through shared memory
 * with bulk copies and waits for each at most about one second; a wait that
 * gives up leaves z invalid and sets a flag on the handle that the next
 * sts_gmres_solve or sts_jac_bjacobi_setup reports as STS_ERR_TIMEOUT.
 */
sts_status sts_jac_bjacobi_apply(sts_jac_t h, const double *x, double *z, int trans);

/* FP32 apply (LU values, W and V rounded to FP32; the r x r solve stays FP64). */
sts_status sts_jac_bjacobi_apply_f32(sts_jac_t h, const float *x, float *z, int trans);

/*
 * Solve J x = b (or J^T x = b) by restarted right-preconditioned GMRES(m)
 * (Section 6, Eq. right_precond_system; Saad & Schultz), classical Gram-Schmidt
 * with a second pass, Givens rotations on the host in FP64.  x holds the
 * initial guess on entry and the solution on exit (pass zeros for x0 = 0).  A
 * zero guess (||x0|| = 0, found in the same pass as ||b||) starts from r = b
 * without the product J x0.
 * Left preconditioning (opts.left, Eq. left_precond_system): each cycle starts
 * from z = M (b - J x), the Arnoldi operator is M J, x += V y, and a cycle stops
 * once |g| has fallen below ||z|| times the factor rtol ||b|| / ||b - J x|| that
 * the true residual still needs; history then holds |g| / ||z|| times the
 * cycle's starting true relative residual.
 * Mixed mode: FP32 matvec and block-Jacobi, FP64 Krylov basis, Arnoldi,
 * residual refresh and capacitance solves, flexible GMRES.  Convergence is
 * declared on the FP64 true residual only.  Synchronous; info may be NULL.
 * Errors: STS_ERR_NOT_CONVERGED (x valid), STS_ERR_NUMERIC, STS_ERR_NOT_SETUP,
 * STS_ERR_TIMEOUT (see sts_jac_bjacobi_apply).
 */
sts_status sts_gmres_solve(sts_jac_t h, const double *b, double *x, const sts_gmres_opts *opts,
                           sts_gmres_info *info);

/*
 * Adjoint outer products of x = J^-1 b for the adjoint lambda = J^-T g
 * (derivative of the implicit solve): gS = -lambda_i x_j^T restricted to the
 * stored pattern of every block, gU[p] = -(v_p . x_j) lambda_i,
 * gV[p] = -(u_p . lambda_i) x_j.  lambda, x: device vectors in the handle's
 * layout; gS, gU, gV: device arrays in the public S / U / V layouts.
 * Needs the factored representation with enable_transpose.  Asynchronous.
 */
sts_status sts_jac_grad(sts_jac_t h, const double *lambda, const double *x, double *gS,
                        double *gU, double *gV);

/*
 * Device bytes held by the handle (values, internal layouts, setup data,
 * workspaces).  Synchronous; never fails for a valid handle.
 */
sts_status sts_jac_memory(sts_jac_t h, size_t *bytes);

/*
 * Number of CUDA kernels this library has launched since it was loaded, over
 * all handles and threads (instrumentation for benchmarks).  Never fails for a
 * non-NULL count.
 */
sts_status sts_launch_count(unsigned long long *count);

/*
 * Self-test of the bounded device wait used by the bulk-copy rings (no paper
 * counterpart): one warp waits on an mbarrier phase that nothing completes,
 * gives up after about one second and reports it, as a real timed-out wait
 * would.  Returns STS_ERR_TIMEOUT when the wait gave up and the device is
 * still usable afterwards, STS_ERR_CUDA otherwise.  Synchronous on the given
 * stream (NULL: the legacy default stream).
 */
sts_status sts_selftest_bounded_wait(void *stream);

/* Destroy a handle and free its device memory.  NULL is accepted. */
sts_status sts_jac_destroy(sts_jac_t h);

/* ---------------------------------------------------------------------------
 * Domain decomposition (spatial partition of the cells over several parts,
 * one sub-domain handle per part).
 *
 * The block adjacency of Section 5.1 couples a cell only with its face
 * neighbours, and the block-Jacobi preconditioner of Section 6 is one block per
 * cell, so the hot path shards by cells: a part owns the block rows of its
 * cells, the matvec needs the vector at a halo of neighbouring cells ("ghost"
 * cells, owned by other parts) and the preconditioner needs nothing from other
 * parts.  GMRES then needs sums over all parts for its dot products.
 *
 * Part p's sub-domain is an ordinary square sts_jac_t over its local cells:
 * the owned cells (ascending global id) followed by the ghost cells (ascending
 * global id), ghosts being the cells of other parts that share a block with an
 * owned cell in either direction.  An owned row keeps all its blocks; a ghost
 * row keeps its diagonal block and its blocks into owned columns.  Once the
 * ghost entries of x hold the neighbours' values, the local product gives the
 * exact rows of J x at owned cells, and the local transposed product the exact
 * rows of J^T x at owned cells; the values at ghost rows are not used.
 */
typedef struct sts_dd_plan_s *sts_dd_plan_t;

/*
 * Build part `part`'s sub-domain plan from the global block CSR (HOST int32,
 * the sts_jac_desc arrays) and a partition part_of_cell[n_cells] with values
 * in [0, n_parts).  Every part computes its own plan; the plans of two
 * neighbouring parts agree on the order of the cells they exchange (ascending
 * global id).  Errors: STS_ERR_INVALID_ARG (bad CSR or partition, a part with
 * no cell).  Host only; no GPU is used.
 */
sts_status sts_dd_plan_create(int n_cells, const int *block_indptr, const int *block_indices, int n_parts,
                              const int *part_of_cell, int part, sts_dd_plan_t *out);

typedef struct {
    int n_owned, n_ghost, n_local;   /* n_local = n_owned + n_ghost                          */
    int nnzb;                        /* blocks of the local block CSR                        */
    int n_neighbors;                 /* parts this part exchanges with                       */
    int n_send, n_recv;              /* cells sent / received over all neighbours            */
} sts_dd_sizes;

sts_status sts_dd_plan_sizes(sts_dd_plan_t plan, sts_dd_sizes *sizes);

/*
 * Copy the plan into HOST int32 arrays sized by sts_dd_plan_sizes:
 *   local_to_global[n_local]       global cell of every local cell
 *   block_indptr[n_local+1], block_indices[nnzb]   local block CSR (local cell ids,
 *                                  rows ascending), ready for sts_jac_desc
 *   block_map[nnzb]                global block id (position in the global
 *                                  block_indices) of every local block
 *   neighbors[n_neighbors]         neighbour part ids, ascending
 *   send_ptr[n_neighbors+1], send_cells[n_send]   owned local cells sent to neighbour k:
 *                                  send_cells[send_ptr[k] .. send_ptr[k+1])
 *   recv_ptr[n_neighbors+1], recv_cells[n_recv]   ghost local cells received from
 *                                  neighbour k, in the order neighbour k sends them
 * Any pointer may be NULL to skip that array.
 */
sts_status sts_dd_plan_get(sts_dd_plan_t plan, int *local_to_global, int *block_indptr, int *block_indices,
                           int *block_map, int *neighbors, int *send_ptr, int *send_cells, int *recv_ptr,
                           int *recv_cells);

/*
 * Sizes of the local value arrays for the global layout given (pair_indptr,
 * the global BR1-BSR pair_indptr[nnzb+1] HOST, or NULL with uniform r_diag /
 * r_off): *nnz_S values of S and *n_pairs pairs, and the local pair_indptr
 * (HOST [nnzb_local+1]; may be NULL).
 */
sts_status sts_dd_plan_value_sizes(sts_dd_plan_t plan, int nnz_d, int nnz_o, const int *pair_indptr, int r_diag,
                                   int r_off, long long *nnz_S, int *n_pairs, int *local_pair_indptr);

/*
 * Gather the local values (the blocks listed in block_map, in local order, and
 * their pairs) from the global S, U, V of the public layout.  on_host = 0:
 * device pointers, one gather kernel on `stream` (asynchronous); on_host = 1:
 * host pointers, copied on the host (synchronous).  The local arrays are sized
 * by sts_dd_plan_value_sizes (U, V: [n_pairs][block_size]).
 */
sts_status sts_dd_plan_gather(sts_dd_plan_t plan, int block_size, int nnz_d, int nnz_o, const int *pair_indptr,
                              int r_diag, int r_off, const double *S, const double *U, const double *V,
                              double *S_local, double *U_local, double *V_local, int on_host, void *stream);

sts_status sts_dd_plan_destroy(sts_dd_plan_t plan);

/*
 * Communication with the parts held by other processes, supplied by the
 * caller (for instance torch.distributed over NCCL).  Both callbacks return 0
 * on success; any other value makes the calling library function return
 * STS_ERR_COMM.
 *   exchange: send n_send messages and receive n_recv messages at once;
 *             send message k goes from part send_from[k] (held here) to part
 *             send_to[k], receive message k from part recv_from[k] to part
 *             recv_to[k] (held here); a (from, to) pair names one message.  A
 *             message holds send_len[k] (recv_len[k]) doubles: the b values of
 *             each listed cell, cell after cell, in the plans' order.  Buffers are
 *             device memory written (read) by work on `stream`: the callback
 *             must order its transfers after the work already queued on
 *             `stream`, and the work queued afterwards after its receives.
 *   allreduce: replace vals[0 .. count) (HOST memory) by their sums over all
 *             processes; every process calls it with the same count.
 */
typedef struct {
    void *ctx;
    int (*exchange)(void *ctx, int n_send, const int *send_from, const int *send_to, const double *const *send_buf,
                    const int *send_len, int n_recv, const int *recv_from, const int *recv_to,
                    double *const *recv_buf, const int *recv_len, void *stream);
    int (*allreduce)(void *ctx, double *vals, int count);
} sts_dd_comm;

typedef struct sts_dd_s *sts_dd_t;

/*
 *   n_parts              parts held by this process (>= 1)
 *   part_ids[n_parts]    their ids in the partition
 *   jac[n_parts]         sub-domain handles created from the plans' local layouts
 *                        (sts_dd_plan_get, sts_dd_plan_gather), factored
 *                        representation, one stream shared by all of them
 *   plans[n_parts]       the plans of those parts (kept by the caller until destroy)
 *   comm                 NULL when every part of the partition is in this process;
 *                        otherwise the callbacks above
 */
typedef struct {
    int n_parts;
    const int *part_ids;
    sts_jac_t *jac;
    sts_dd_plan_t *plans;
    const sts_dd_comm *comm;
} sts_dd_desc;

/* Check the parts and upload the exchange lists.  Synchronous. */
sts_status sts_dd_create(const sts_dd_desc *desc, sts_dd_t *out);

/*
 * y = J x (trans = 0) or J^T x (trans = 1) over the whole partition.  x[k],
 * y[k]: device vectors of local part k (n_local * b entries, the handle's
 * layout).  The ghost entries of x are ignored (their values come from the
 * neighbours, by one halo exchange); the ghost entries of y are set to zero.
 * Asynchronous on the parts' stream.
 */
sts_status sts_dd_matvec(sts_dd_t dd, const double *const *x, double *const *y, int trans);

/* z = M x per part (Section 6, block-Jacobi through SMW; no communication);
 * needs sts_jac_bjacobi_setup on every part.  Ghost entries of z are set to zero. */
sts_status sts_dd_bjacobi_apply(sts_dd_t dd, const double *const *x, double *const *z, int trans);

/*
 * Solve J x = b (or J^T x = b) over the partition by right-preconditioned
 * restarted GMRES (Section 6, Eq. right_precond_system), the same algorithm as
 * sts_gmres_solve (classical Gram-Schmidt with a second pass, Givens rotations
 * on the host in FP64), with one halo exchange per matvec and three sums over
 * the processes per Arnoldi step (the first and second Gram-Schmidt dot
 * products, the norm).  b[k], x[k] as in sts_dd_matvec (x: initial guess on
 * entry, solution on exit; ghost entries ignored on entry, zero on exit).
 * opts: restart, max_iters, rtol, precond, trans, history; left and mixed are
 * not supported here (STS_ERR_INVALID_ARG).  Every process must call it with
 * the same options.  Synchronous.  Errors as sts_gmres_solve, plus STS_ERR_COMM.
 */
sts_status sts_dd_gmres_solve(sts_dd_t dd, const double *const *b, double *const *x, const sts_gmres_opts *opts,
                              sts_gmres_info *info);

sts_status sts_dd_destroy(sts_dd_t dd);

/*
 * The same GMRES driver over operations supplied by the caller, for a local
 * operator or a communication layer that this library does not provide (it is
 * how the driver is tested on CPU ranks).  Vectors are named by index:
 *   0 .. m          the Krylov basis v_0 .. v_m        (m = opts->restart)
 *   m+1 .. 2m       the preconditioned vectors z_0 .. z_{m-1}
 *   2m+1 w, 2m+2 r, 2m+3 x (initial guess on entry, solution on exit), 2m+4 b.
 * The callbacks act on this process's share of each vector and return 0 on
 * success (else the driver returns STS_ERR_COMM):
 *   matvec(in, out)      out = A in, including any halo exchange it needs
 *   apply(in, out)       out = M in
 *   copy(out, in), sub(out, a, b): out = a - b, scale(out, in, s): out = s in (s = 0 writes zeros)
 *   dots(v0, k, w, self, out)    out[i] = v_{v0+i} . w over this process's share,
 *                        i < k, and out[k] = w . w when self is 1
 *   update(w, v0, k, h, norm, out)   w -= sum_{i<k} h[i] v_{v0+i}; out[0] = w . w
 *                        (this process's share) when norm is 1
 *   norm2(v, out)        out[0] = v . v over this process's share
 *   axpy(x, v0, k, y)    x += sum_{i<k} y[i] v_{v0+i}
 *   allreduce(vals, n)   sum over all processes, in place (HOST memory)
 */
typedef struct {
    void *ctx;
    int (*matvec)(void *ctx, int in, int out);
    int (*apply)(void *ctx, int in, int out);
    int (*copy)(void *ctx, int out, int in);
    int (*sub)(void *ctx, int out, int a, int b);
    int (*scale)(void *ctx, int out, int in, double s);
    int (*dots)(void *ctx, int v0, int k, int w, int self, double *out);
    int (*update)(void *ctx, int w, int v0, int k, const double *h, int norm, double *out);
    int (*norm2)(void *ctx, int v, double *out);
    int (*axpy)(void *ctx, int x, int v0, int k, const double *y);
    int (*allreduce)(void *ctx, double *vals, int count);
} sts_dd_ops;

sts_status sts_dd_gmres_ops(const sts_dd_ops *ops, const sts_gmres_opts *opts, sts_gmres_info *info);

/* ---------------------------------------------------------------------------
 * Jacobian generator of a toy flow model: the first-order finite-volume
 * residual with an HLL flux (Section 3.2, Eq. HLL_flux; Section 3.3, Eq.
 * system_residual) and its Jacobian dR/dQ written directly in the BR1-BSR form
 * above, the flux Jacobians split as in Section 4.1 (Eqs. r1_flux_left /
 * r1_flux_right) into a sparse part plus two rank-one pairs per face.
 *
 * Model, per cell q = (rho_0 .. rho_{N-1}, u, v, T), block size b = N + 3
 * (Section 2.1 with synthetic constants):
 *   e_k(T) = e0_k + cv_k T,  p = sum rho_k r_k T,  rho e_tot = sum rho_k e_k + rho (u^2+v^2)/2,
 *   gamma = (c_v + r) / c_v with c_v, r the mass-fraction averages of cv_k, r_k,
 *   a = sqrt(gamma r T);  conserved u(q) = (rho_k, rho u, rho v, rho e_tot);
 *   f_n(q) = (rho_k u_n, rho u u_n + p n_x, rho v u_n + p n_y, (rho e_tot + p) u_n).
 *   HLL wave-speed bounds: s_L = min(0, u_nL - a_L, u_nR - a_R),
 *   s_R = max(0, u_nL + a_L, u_nR + a_R), ties to the first candidate.
 *   Source (level rows only): Omega_k = -sum_{|l-k|<=w} K[k][l-k+w] rho_l
 *                                       + ws_k A exp(-theta/T) sum_l beta_l rho_l.
 * Grid: Lx x Ly unit cells, id iy*Lx + ix, faces to i-Lx, i-1, i+1, i+Lx with
 * outward unit normals; no flux through the outer boundary.
 *   R_i = u(q_i) - u(q_i^n) + dt (sum over faces f(q_i, q_j, n_ij) - Omega(q_i)).
 * Jacobian layout (sts_flow_get_layout):
 *   block CSR: the mesh adjacency including the diagonal, rows ascending;
 *   diagonal pattern: level row p holds columns max(0,p-w)..min(N-1,p+w) then
 *     N, N+1, N+2; the three flow rows are dense;
 *   neighbour pattern: level row p holds p, N, N+1, N+2; flow rows dense;
 *   pairs of the diagonal block of cell i (1 + 2 per face): (-dt ws, d omega/dq),
 *     then per face in block order (-dt (f_R - f_L), d a_f / d q_i) and
 *     (dt (u_R - u_L), d c_f / d q_i), with a_f = (s_L + s_R) / (2 (s_R - s_L)),
 *     c_f = s_L s_R / (s_R - s_L), L = i and R = the neighbour;
 *   pairs of the neighbour block (i, j): the same two face vectors with
 *     d a_f / d q_j and d c_f / d q_j;
 *   S values: diagonal block H(q_i) + dt (sum over faces A0_L + K band), with
 *     H = du/dq and A0_L = (1/2 + a_f) A_n(q_i) - c_f H(q_i); neighbour block
 *     dt A0_R = dt ((1/2 - a_f) A_n(q_j) + c_f H(q_j)).
 * States must have sum rho_k > 0, sum rho_k cv_k > 0, sum rho_k r_k > 0 and
 * T > 0; others give NaN or infinite values (not checked on the device).
 */
typedef struct {
    int Lx, Ly;                 /* grid size (>= 1 each)                                  */
    int n_species;              /* N >= 1                                                  */
    int band;                   /* w >= 0: level band of K and of the diagonal pattern     */
    const double *r;            /* HOST [N] species gas constants (> 0)                    */
    const double *cv;           /* HOST [N] specific heats (> 0)                           */
    const double *e0;           /* HOST [N] energies at T = 0                              */
    const double *beta;         /* HOST [N] source weights                                 */
    const double *ws;           /* HOST [N] source stoichiometry                           */
    const double *K;            /* HOST [N][2w+1] band, K[k][l - k + w]                    */
    double A, theta;            /* source rate A exp(-theta / T)                           */
    double dt;                  /* pseudo time step                                        */
    void *stream;               /* cudaStream_t for all work (NULL = legacy default)       */
} sts_flow_desc;

typedef struct {
    int n_cells, block_size, nnzb, nnz_d, nnz_o, n_pairs;
    long long nnz_S;            /* length of S                                             */
} sts_flow_sizes;

typedef struct sts_flow_s *sts_flow_t;

/* Copy the constants and build the layout tables.  STS_ERR_INVALID_ARG on a bad size, a
 * NULL array, r_k <= 0 or cv_k <= 0, or a non-finite constant. */
sts_status sts_flow_create(const sts_flow_desc *d, sts_flow_t *out);   /* b = N + 3 <= 256 */
/* Sizes of the layout and of the S, U, V arrays (U, V: [n_pairs][block_size]). */
sts_status sts_flow_get_sizes(sts_flow_t f, sts_flow_sizes *s);
/* Copy the layout into HOST int32 arrays sized by sts_flow_get_sizes (block_indptr
 * n_cells+1, block_indices nnzb, d_indptr / o_indptr b+1, d_indices nnz_d, o_indices
 * nnz_o, pair_indptr nnzb+1); they can be handed to sts_jac_create as they are. */
sts_status sts_flow_get_layout(sts_flow_t f, int *block_indptr, int *block_indices, int *d_indptr,
                               int *d_indices, int *o_indptr, int *o_indices, int *pair_indptr);
/* R = residual of the states Q given Qn; DEVICE pointers, [n_cells][b] cell-major; async. */
sts_status sts_flow_residual(sts_flow_t f, const double *Q, const double *Qn, double *R);
/* S, U, V of dR/dQ at Q in the layout above; DEVICE pointers; async. */
sts_status sts_flow_jacobian(sts_flow_t f, const double *Q, double *S, double *U, double *V);
/* Free the generator.  NULL is accepted. */
sts_status sts_flow_destroy(sts_flow_t f);

/*
 * One implicit pseudo-time step by Newton's method (Section 3.3): starting from
 * the Q given, iterate Q <- Q + alpha dQ with (dR/dQ) dQ = -R(Q) (Eq.
 * LinearSystem), the Jacobian written by sts_flow_jacobian into jac
 * (sts_jac_update_values), block-Jacobi set up and the system solved by
 * sts_gmres_solve with opts->gmres.  alpha (the line-search coefficient) starts
 * at 1 and is halved while ||R|| does not decrease, at most max_halvings times.
 * A linear solve that stops at max_iters without converging still gives a step
 * (inexact Newton).  Stops when ||R(Q)||_2 <= max(rtol ||R(Q^0)||, atol).
 *   jac: a handle created from this generator's layout (sts_flow_get_layout),
 *        vec_layout STS_LAYOUT_CELL_MAJOR, factored or dense-BSR; its values are
 *        overwritten.
 *   Q: DEVICE [n_cells][b], the initial iterate on entry, the result on exit;
 *   Qn: DEVICE, the previous time level.
 * Synchronous.  STS_ERR_NOT_CONVERGED (Q holds the last accepted iterate) when
 * max_newton iterations end above the tolerance or the line search finds no
 * decrease; the errors of the calls it makes pass through.
 */
typedef struct {
    int max_newton;           /* Newton iterations (default 20)                          */
    double rtol;              /* relative tolerance on ||R|| (default 1e-10)             */
    double atol;              /* absolute tolerance on ||R|| (default 0)                 */
    int max_halvings;         /* line-search halvings of alpha (default 8)               */
    sts_gmres_opts gmres;     /* linear solves; vectors_on_host must be 0                */
    double *history;          /* optional HOST [max_newton + 1]: ||R|| before iteration 1,
                                 then after every iteration                              */
    int forcing;              /* 0: every linear solve to gmres.rtol.  1: inexact Newton,
                                 solve k to eta_k ||R_k|| (Eisenstat & Walker's choice 2,
                                 gamma = 0.9, with the safeguards of Kelley 2003):
                                 eta_0 = 0.9, eta_k = min(0.9, max(0.9 (r_k / r_{k-1})^2,
                                 0.9 eta_{k-1}^2 if that exceeds 0.1,
                                 0.5 tol / r_k)); gmres.rtol is then ignored             */
} sts_newton_opts;

typedef struct {
    int iterations;           /* Newton iterations taken                                 */
    int linear_iterations;    /* GMRES iterations over all solves                        */
    int halvings;             /* line-search halvings over all iterations                */
    int converged;
    double res0, res;         /* ||R(Q^0)||_2 and ||R(Q)||_2 at exit                     */
} sts_newton_info;

sts_status sts_flow_newton(sts_flow_t f, sts_jac_t jac, double *Q, const double *Qn,
                           const sts_newton_opts *opts, sts_newton_info *info);

#ifdef __cplusplus
}
#endif

#endif /* STS_H */
