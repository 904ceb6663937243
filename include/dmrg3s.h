/*
 * dmrg3s.h -- C ABI of the GB300 (sm_103a) DMRG3S hot path.
 *
 * DMRG3S is the strictly single-site DMRG with subspace expansion of
 * C. Hubig, I. P. McCulloch, U. Schollwoeck, F. A. Wolf, "A Strictly
 * Single-Site DMRG Algorithm with Subspace Expansion", arXiv:1501.05504.
 * Citations below name the paper's sections and equations.
 *
 * Conventions shared by every entry point
 * --------------------------------------
 * Tensors are block sparse under up to two abelian U(1) charges.  A bond is a
 * list of charge sectors (strictly increasing charge vectors, lexicographic)
 * with one dimension each.  All floating-point data is IEEE double, stored on
 * the device, owned by the caller unless stated otherwise.
 *
 *  - MPS site tensor M[s](al, ar), shape (d, m_{i-1}, m_i) (Sec. II).  Block
 *    (s, i, j) exists iff q_left[i] + qp[s] == q_right[j].  Canonical block
 *    order: s ascending, then left sector i ascending; each block is a
 *    row-major D_left[i] x D_right[j] matrix; blocks are packed back to back.
 *  - Environment E[b](a_bra, a_ket) (L_i or R_i of Sec. II), shape (w, m, m);
 *    bra and ket share one bond.  Block (b, ib, ik) exists iff
 *    q[ik] + t[b] == q[ib].  Canonical order: b ascending, then ket sector ik
 *    ascending; each block is row-major D[ib] x D[ik].
 *  - MPO site tensor W[s_out][s_in][bl][br] (Sec. II, rank 4, (d, d, w_{i-1},
 *    w_i)), dense, row-major, on the HOST; s_out is the bra index.  A channel
 *    charge t[b] is the charge the operators left of the MPO bond have added;
 *    W may be non-zero only where qp[s_out] - qp[s_in] + tl[bl] == tr[br].
 *
 * Errors: argument, shape and charge errors are detected on the host before
 * any launch and return a status without touching device memory.  Device
 * results are stream ordered: a call returns once its work is enqueued on the
 * given stream (NULL = the legacy default stream), except where stated.
 * No entry point aborts, traps or prints.
 *
 * Thread safety: a context may be used by one host thread at a time.
 */
#ifndef DMRG3S_H
#define DMRG3S_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* dmrg3s_stream;   /* same type as cudaStream_t */
typedef struct dmrg3s_ctx_s* dmrg3s_ctx;

typedef enum dmrg3s_status {
  DMRG3S_OK = 0,
  DMRG3S_ERR_ARG = 1,           /* null pointer, bad enum, negative size       */
  DMRG3S_ERR_SHAPE = 2,         /* bonds/dimensions inconsistent between args   */
  DMRG3S_ERR_QN = 3,            /* charge tables malformed or W breaks charges */
  DMRG3S_ERR_OOM = 4,           /* context workspace too small                  */
  DMRG3S_ERR_CUDA = 5,          /* a CUDA runtime or library call failed        */
  DMRG3S_ERR_NOT_CONVERGED = 6, /* iteration limit reached                      */
  DMRG3S_ERR_BREAKDOWN = 7,     /* Lanczos start vector is zero                 */
  DMRG3S_ERR_TIMEOUT = 8,       /* a bounded device wait gave up                */
  DMRG3S_ERR_NUMERIC = 9,       /* NaN or Inf detected                          */
  DMRG3S_ERR_UNSUPPORTED = 10,  /* valid request this build does not implement  */
  DMRG3S_ERR_LIMIT = 11         /* request exceeds a fixed static capacity      */
} dmrg3s_status;

/* Arithmetic of the block products (stages 1 and 3 of the order of Sec. V).
 * The eigensolver's vector algebra, the SVD and all data the caller sees stay
 * FP64 in every mode.  In the tensor-core modes each FP64 operand is split
 * once into two FP32 arrays, x = hi + lo with hi = tf32(x), lo = tf32(x - hi);
 * 3xTF32 sums hi*hi + hi*lo + lo*hi (relative error of a block product
 * ~1e-6), TF32 only hi*hi (~1e-3); the block products leave double-float
 * (FP32 pair) results, which the MPO combination (stage 2) and the split-K
 * sum combine in double-float arithmetic (~48 bits). */
typedef enum dmrg3s_precision {
  DMRG3S_FP64 = 0,    /* double precision on the CUDA cores                          */
  DMRG3S_TF32X3 = 1,  /* 3xTF32 split products on tcgen05 tensor cores, FP32 accum.  */
  DMRG3S_TF32 = 2     /* single-pass TF32 on tcgen05 tensor cores, FP32 accumulate   */
} dmrg3s_precision;

#define DMRG3S_MAX_NSYM 2

typedef struct dmrg3s_bond {
  int32_t nsec;          /* number of sectors, >= 1 (exactly 1 when nsym == 0)  */
  const int32_t* q;      /* host [nsec][nsym]; may be NULL when nsym == 0       */
  const int64_t* dim;    /* host [nsec], every entry >= 1                       */
} dmrg3s_bond;

typedef struct dmrg3s_site {   /* MPS site tensor M[s](al, ar) */
  int32_t nsym;          /* 0, 1 or 2 charges                                   */
  int32_t d;             /* physical dimension                                  */
  const int32_t* qp;     /* host [d][nsym] charge of each physical state        */
  dmrg3s_bond left, right;
  double* data;          /* device, blocks in canonical order                   */
} dmrg3s_site;

typedef struct dmrg3s_env {    /* environment E[b](a_bra, a_ket) */
  int32_t nsym;
  int32_t w;             /* MPO bond dimension                                   */
  const int32_t* t;      /* host [w][nsym] channel charges                       */
  dmrg3s_bond bond;      /* shared by bra and ket                                */
  double* data;          /* device, blocks in canonical order                    */
} dmrg3s_env;

typedef struct dmrg3s_mpo_site {
  int32_t nsym, d, wl, wr;
  const int32_t* qp;     /* host [d][nsym]  */
  const int32_t* tl;     /* host [wl][nsym] */
  const int32_t* tr;     /* host [wr][nsym] */
  const double* W;       /* host [d][d][wl][wr] */
} dmrg3s_mpo_site;

/* ---- context -------------------------------------------------------------- */

/* Creates a context on CUDA device `device` with a device workspace arena of
 * `workspace_bytes` (0 = 256 MiB) from which all intermediates (T1/T2 of the
 * contraction order of Sec. V, task tables) are carved.  Errors: ARG, CUDA. */
dmrg3s_status dmrg3s_create(dmrg3s_ctx* ctx, int device, size_t workspace_bytes);

/* Releases the context and its workspace.  Synchronises the device first. */
dmrg3s_status dmrg3s_destroy(dmrg3s_ctx ctx);

/* Static, human-readable name of a status code. */
const char* dmrg3s_status_string(dmrg3s_status status);

/* Message of the last error a call on `ctx` returned (valid until the next
 * call on ctx; "" when none). */
const char* dmrg3s_last_error(dmrg3s_ctx ctx);

/* Synchronises `stream` and returns the device-side error latched by the
 * context's kernels since the last call: DMRG3S_ERR_TIMEOUT when a
 * tensor-core kernel gave up a bounded wait (its output is then invalid).
 * The latch is cleared.  Errors: ARG, CUDA, TIMEOUT. */
dmrg3s_status dmrg3s_sync(dmrg3s_ctx ctx, dmrg3s_stream stream);

/* Limit of every bounded wait inside this library's kernels (the tensor-core
 * kernel's waits for bulk copies, products and drains), in seconds of
 * elapsed device time (%globaltimer); default 1.0.  A wait that runs out makes
 * its CTA stop (after the copies and products already in flight have
 * finished), latches DMRG3S_ERR_TIMEOUT for dmrg3s_sync and the eigensolver,
 * and leaves the context usable; the results of that launch are invalid.
 * seconds = 0 makes every wait that does not succeed at once run out (for
 * testing the error path).  Errors: ARG (negative or not finite). */
dmrg3s_status dmrg3s_set_wait_limit(dmrg3s_ctx ctx, double seconds);

/* Kernel timing.  While enabled, the context records CUDA events on the
 * launching stream around every grouped-GEMM launch of the contractions
 * (kernel 0: the block products of stages 1 and 3 of the contraction order
 * of Sec. V) and every MPO combination launch (kernel 1: stage 2), around
 * the phases of every local update (2: eigensolver, 3: expansion term,
 * 4: gather + SVD + new tensors, 5: S V^dagger into the neighbour,
 * 6: environment update, 7: energy after truncation; flops and bytes are 0
 * for phases), around the other FP64 grouped GEMMs (kernel 8: the
 * truncation's S V^dagger products and the MPO-entry gradient), and around
 * each sweep of the truncation's Jacobi SVD (kernel 9: one record per sweep,
 * counting its launches: the sweep-counter kernel and one launch per round;
 * flops: 6n per column-pair test plus, per rotation, 6n (12n when the left
 * vectors' rotations are accumulated too); bytes: 16n per pair test plus,
 * per rotation, 16n (48n with the left vectors)).
 * dmrg3s_profile(ctx, 1) resets and enables, 0 disables;
 * dmrg3s_profile_read synchronises on the recorded events and
 * returns, for one kernel, the number of launches, their summed device time
 * (for kernel 9 the time of whole sweeps, gaps between launches included)
 * and their summed algorithmic flops and bytes (each distinct operand block
 * read once, each output written once). */
typedef struct dmrg3s_kernel_stats {
  int64_t launches;
  double ms, flops, bytes;
} dmrg3s_kernel_stats;
dmrg3s_status dmrg3s_profile(dmrg3s_ctx ctx, int32_t enable);
dmrg3s_status dmrg3s_profile_read(dmrg3s_ctx ctx, int32_t kernel, dmrg3s_kernel_stats* out);

/* Process-wide number of kernels this library has launched (its own kernels
 * only; cuSOLVER's are not counted). */
dmrg3s_status dmrg3s_launch_count(int64_t* n);

/* Number of doubles a site tensor / environment occupies in canonical layout.
 * Pure host functions (no CUDA call); they also validate the charge tables. */
dmrg3s_status dmrg3s_site_size(const dmrg3s_site* M, int64_t* nelem);
dmrg3s_status dmrg3s_env_size(const dmrg3s_env* E, int64_t* nelem);

/* Block tables of the canonical layout.  `table` receives nblocks rows of
 * 6 int64: (s, i, j, offset, rows, cols) for a site tensor and
 * (b, ib, ik, offset, rows, cols) for an environment, in canonical order.
 * With table == NULL only *nblocks is written.  Host functions. */
dmrg3s_status dmrg3s_site_blocks(const dmrg3s_site* M, int64_t* nblocks, int64_t* table);
dmrg3s_status dmrg3s_env_blocks(const dmrg3s_env* E, int64_t* nblocks, int64_t* table);

/* Bond of the expanded basis of Sec. IV A.  For a bond with sectors (q_j, D_j)
 * and MPO channels with charges t[b], the expansion term adds, for every
 * channel b and sector j, D_j states of charge q_j + t[b] (the right bond of
 * P for a left-to-right sweep with t = W->tr, or its left bond for a
 * right-to-left sweep with t = W->tl).  The fused bond has one sector per
 * distinct charge, ascending; inside a sector the states are ordered: first
 * the original states of that charge when include_base != 0 (the M part of
 * [M P] or [M; P]), then channel b ascending, each followed by the states of
 * its source sector.  When `q`/`dim` are NULL only `*nsec` is written;
 * otherwise they must hold *nsec (q: *nsec * nsym) entries.
 * Host function.  Errors: ARG, QN. */
dmrg3s_status dmrg3s_expanded_bond(int32_t nsym, const dmrg3s_bond* bond, int32_t w,
                                   const int32_t* t, int32_t include_base, int32_t* nsec,
                                   int32_t* q, int64_t* dim);

/* ---- the hot path -------------------------------------------------------------- */

/* FP64 singular value decomposition of a batch of matrices: the factorisation
 * of the truncation step (Sec. IV A, Sec. V step 4; DMRG3S_SVD_JACOBI).
 * Matrix k is A_k (m[k] x n[k], 1 <= n[k] <= m[k], n[k] <= 32768),
 * column-major with leading dimension m[k], stored back to back in `A`
 * (device; not modified).  With its columns in descending norm order (A P),
 * each is factorised A P = Q R (cuSOLVER Householder QR, on a copy) and R^T
 * is orthogonalised by one-sided Jacobi rotations (the parallel
 * round-robin order over column pairs, one warp per pair, every matrix in each
 * launch) until no pair has |<y_a, y_b>| > max(sqrt(n), 32) 2^-52 |y_a| |y_b|.
 * Outputs, back to back per matrix (device): S (n[k] singular values,
 * descending), VT (n[k] x n[k], ld n[k]; row c = right singular vector c,
 * zero for a zero singular value) and, when U is not NULL, U (m[k] x n[k],
 * ld m[k]; column c = left singular vector c).  Runs on `stream` and on a
 * cuSOLVER handle and stream created for the call (the local update reuses
 * its state's); synchronous (one host read per sweep).
 * Errors: ARG (shapes), CUDA, NOT_CONVERGED (a matrix still rotating after
 * 40 sweeps, or after the number 1..40 in the environment variable
 * DMRG3S_JACOBI_SWEEPS; outputs then invalid). */
dmrg3s_status dmrg3s_svd(dmrg3s_ctx ctx, int32_t nmat, const int64_t* m, const int64_t* n,
                         double* A, double* S, double* VT, double* U, dmrg3s_stream stream);

/* Algorithmic cost of one dmrg3s_apply_heff with these structures, without
 * touching the device (the data pointers are not read and may be NULL):
 * *flops = the sum of 2 M N K over the block products of stages 1 and 3
 * plus 2 rows cols per MPO term of stage 2 (the order of Sec. V); *bytes
 * (may be NULL) = each distinct operand block read once and each output
 * block written once, 8 bytes per element, summed over the three stages.
 * Host function.  Errors: ARG, SHAPE, QN. */
dmrg3s_status dmrg3s_heff_cost(const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                               const dmrg3s_env* R, const dmrg3s_site* A, double* flops,
                               double* bytes);

/* HA = L W A R: the left-hand side of the local eigenproblem
 *   L_{i-1} R_{i+1} W_i M_i = lambda M_i           (Eq. es-iter, Sec. V)
 * i.e. HA[s'](al', ar') = sum L[bl](al', al) W[s', s, bl, br] A[s](al, ar) R[br](ar', ar),
 * contracted in the order (((L A) W) R) of Sec. V.
 * L: left environment on A's left bond, L->w == W->wl, L->t == W->tl.
 * R: right environment on A's right bond, R->w == W->wr, R->t == W->tr.
 * HA: same structure as A (same bonds and charges); overwritten.
 * `prec` selects the arithmetic; A, L, R, HA stay double in memory.
 * Errors: ARG, SHAPE, QN, OOM, CUDA, UNSUPPORTED. */
dmrg3s_status dmrg3s_apply_heff(dmrg3s_ctx ctx, const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                                const dmrg3s_env* R, const dmrg3s_site* A, dmrg3s_site* HA,
                                dmrg3s_precision prec, dmrg3s_stream stream);

/* Prepared H_eff operator for repeated application with fixed environments,
 * as in the Lanczos iteration of Sec. V step 1 (H_eff = L_{i-1} W_i . R_{i+1}
 * of Eq. es-iter, contracted as dmrg3s_apply_heff does).  dmrg3s_heff_create
 * plans the contraction for the structures of L, W, R and A (A->data is not
 * read) and, in the tensor-core modes, packs L and R once into device memory
 * owned by the handle (on `stream`); dmrg3s_heff_apply then computes
 * HA = H_eff A for a vector A (device, canonical layout of A's structure, and
 * HA likewise; both caller-owned) on `stream`, using the context's workspace.
 * In DMRG3S_FP64 the handle reads L->data and R->data at every application:
 * they must stay allocated and unchanged while the handle is used.  The
 * handle must not outlive its context; one host thread at a time.
 * Errors: as dmrg3s_apply_heff. */
typedef struct dmrg3s_heff_s* dmrg3s_heff;
dmrg3s_status dmrg3s_heff_create(dmrg3s_ctx ctx, const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                                 const dmrg3s_env* R, const dmrg3s_site* A,
                                 dmrg3s_precision prec, dmrg3s_heff* out, dmrg3s_stream stream);
dmrg3s_status dmrg3s_heff_apply(dmrg3s_heff op, const double* A, double* HA,
                                dmrg3s_stream stream);
/* Synchronises the device, then frees the handle. */
dmrg3s_status dmrg3s_heff_destroy(dmrg3s_heff op);

/* H_eff application for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is a deployment variant of
 * dmrg3s_apply_heff.  Some callers cannot call cudaMalloc: a host process
 * whose device memory is reserved up front by another allocator (a
 * framework's caching pool or a fixed arena) gets nothing more from the
 * driver, and a real-time loop may not risk the latency or the failure of an
 * allocation in the middle of its work.  Such callers cannot create a context
 * (whose workspace is allocated).  This entry point needs no context and
 * allocates nothing on the device: it computes exactly what
 * dmrg3s_apply_heff computes in DMRG3S_FP64, keeping its intermediates
 * (T1 = L A, T2 = W T1) and task tables in fixed-size static device arrays of
 * this library (DMRG3S_NOALLOC_SCRATCH_DOUBLES doubles of scratch plus about
 * 16 MiB of tables), which every GPU that loads the library holds until the
 * process exits.  The caller passes inputs and output as for
 * dmrg3s_apply_heff, on the current CUDA device.
 *  - The first call on a device looks up the arrays' device addresses (a
 *    one-time set-up with that device current); make that first call before
 *    any stream capture.
 *  - Each call uploads its task tables into the static arrays with ordinary
 *    host-to-device copies from pageable host memory on `stream`.
 *  - All calls share the arrays, which keep the last call's contents: calls
 *    that overlap on the GPU (different streams, or threads) race and give
 *    wrong results; calls on one stream are ordered and correct.  Every
 *    intermediate element is written before it is read, so nothing has to be
 *    cleared between calls.
 *  - A CUDA error already pending on the calling thread (from earlier,
 *    unrelated work) makes the call return DMRG3S_ERR_CUDA before it does
 *    anything; the pending error is left for its owner.
 *  - Returns DMRG3S_ERR_LIMIT, before touching the device, when the
 *    intermediates need more than DMRG3S_NOALLOC_SCRATCH_DOUBLES doubles or
 *    the block structure needs more tasks than the static tables hold.
 * Errors: ARG, SHAPE, QN, LIMIT, CUDA. */
#define DMRG3S_NOALLOC_SCRATCH_DOUBLES 2097152
dmrg3s_status dmrg3s_apply_heff_noalloc(const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                                        const dmrg3s_env* R, const dmrg3s_site* A,
                                        dmrg3s_site* HA, dmrg3s_stream stream);

/* Expansion term of Sec. IV B (Eq. subexp-ourt):
 *   dir = +1 (left-to-right sweep): P = alpha L_{i-1} M_i W_i, in (d, m_{i-1}, w_i m_i),
 *      P[s'](al', (br, ar)) = alpha sum L[bl](al', al) W[s', s, bl, br] M[s](al, ar);
 *      `env` is L_{i-1}; P->left == M->left; P->right is
 *      dmrg3s_expanded_bond(M->right, W->wr, W->tr, include_base = 0).
 *   dir = -1 (right-to-left): P = alpha R_{i+1} M_i W_i, in (d, w_{i-1} m_{i-1}, m_i),
 *      P[s']((bl, al), ar') = alpha sum W[s', s, bl, br] M[s](al, ar) R[br](ar', ar);
 *      `env` is R_{i+1}; P->right == M->right; P->left is
 *      dmrg3s_expanded_bond(M->left, W->wl, W->tl, include_base = 0).
 * P is overwritten.  Errors as dmrg3s_apply_heff. */
dmrg3s_status dmrg3s_expand(dmrg3s_ctx ctx, int32_t dir, const dmrg3s_env* env,
                            const dmrg3s_mpo_site* W, const dmrg3s_site* M, double alpha,
                            dmrg3s_site* P, dmrg3s_precision prec, dmrg3s_stream stream);

/* Environment recursion of Sec. II:
 *   dir = +1: L_i = L_{i-1} A_i^dagger W_i A_i   (env = L_{i-1}, out on A's right bond, t = W->tr)
 *   dir = -1: R_i = R_{i+1} B_i^dagger W_i B_i   (env = R_{i+1}, out on B's left bond,  t = W->tl)
 * `out` is overwritten.  Errors as dmrg3s_apply_heff. */
dmrg3s_status dmrg3s_update_env(dmrg3s_ctx ctx, int32_t dir, const dmrg3s_env* env,
                                const dmrg3s_mpo_site* W, const dmrg3s_site* A,
                                dmrg3s_env* out, dmrg3s_precision prec, dmrg3s_stream stream);

/* MPO-entry gradient of <M|H_eff|M> (the network of Sec. II with W_i taken
 * out; <Psi|H|Psi> is linear in each W_i):
 *   G[s', s, bl, br] = sum L[bl](al', al) M[s'](al', ar') M[s](al, ar) R[br](ar', ar)
 * L, W, R, M as for dmrg3s_apply_heff (only W's structure is used, not its
 * values).  G: device, d*d*wl*wr doubles in the layout of W (row-major
 * [s'][s][bl][br]); overwritten, zero where the charge rule forbids an entry.
 * With L, R the environments of the current MPS and M its orthogonality
 * centre, sum_{entries} G * dW/dtheta / <M|M> is the Hellmann-Feynman
 * derivative of the energy.  FP64 on the CUDA cores; intermediates in the
 * context workspace.  Errors as dmrg3s_apply_heff. */
dmrg3s_status dmrg3s_mpo_grad_site(dmrg3s_ctx ctx, const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                                   const dmrg3s_env* R, const dmrg3s_site* M, double* G,
                                   dmrg3s_stream stream);

/* Local eigensolver, step 1 of Sec. V: the smallest eigenpair (lambda*, M*)
 * of L_{i-1} R_{i+1} W_i M_i = lambda M_i (Eq. es-iter) by Lanczos with full
 * reorthogonalisation (classical Gram-Schmidt applied twice), all in FP64 on
 * the device; the tridiagonal eigenproblem is solved in a device kernel by
 * Sturm multisection (double-float counts), inverse iteration and the
 * Rayleigh quotient of the resulting vector.  M: start vector on input, the
 * normalised Ritz vector on output.  Stops when the Ritz residual
 * |beta_k y_k| <= tol * max(1, |lambda|), when beta_k < 1e-14 or after kmax
 * (<= 128) products.  The tridiagonal solve of iteration k runs on a side
 * stream of the context while `stream` already computes the product of the
 * next basis vector; the host waits once per iteration for the solve's
 * result.  When iteration k is the last, that product is discarded (the
 * profiler does not count its flops), so a run issues one product more
 * than it reports.  Errors: as dmrg3s_apply_heff, plus BREAKDOWN (zero
 * start vector) and NUMERIC (NaN). */
dmrg3s_status dmrg3s_eigensolve(dmrg3s_ctx ctx, const dmrg3s_env* L, const dmrg3s_mpo_site* W,
                                const dmrg3s_env* R, dmrg3s_site* M, int32_t kmax, double tol,
                                dmrg3s_precision prec, double* lambda, int32_t* iters,
                                dmrg3s_stream stream);

/* ---- model MPOs ----------------------------------------------------------------- */

/* Built-in Hamiltonians as MPOs (Sec. II: H = W_1 ... W_l), lower-triangular
 * finite-state form: channel 0 = all terms finished, last channel = nothing
 * placed yet; the first site keeps only the last row, the last site only
 * column 0; a channel's charge is what the operators already placed add.
 *  XXZ      params {J, Delta}: J sum_i [(S+_i S-_{i+1} + h.c.)/2 + Delta Sz_i Sz_{i+1}],
 *           w = 5, d = 2 (up, down), one charge 2 S^z.
 *  HUBBARD  params {t, U}: -t sum_{i,s} (c+_{i,s} c_{i+1,s} + h.c.) + U sum_i n_up n_dn,
 *           Jordan-Wigner string, w = 6, d = 4 (index 2 n_up + n_dn), charges (N, 2 S^z).
 *  SPIN_BONDS: sum over `nbonds` pairs bonds[2k] < bonds[2k+1] of
 *           couplings[2k]/2 (S+ S- + S- S+) + couplings[2k+1] Sz Sz, e.g. the
 *           snake-ordered cylinder or a ring (the S = 1 chain of Sec. VII B 1
 *           with its periodic link (0, l-1)); channels (S+, S-, Sz) per open
 *           site.  params NULL: spin 1/2; else params[0] = 2S (1..8): d = 2S+1,
 *           basis m = S, S-1, ..., -S, charge 2m.
 * XXZ and HUBBARD have open boundary conditions.  Host-only. */
typedef enum dmrg3s_model {
  DMRG3S_MODEL_XXZ = 0,
  DMRG3S_MODEL_HUBBARD = 1,
  DMRG3S_MODEL_SPIN_BONDS = 2
} dmrg3s_model;

typedef struct dmrg3s_mpo_s* dmrg3s_mpo;

dmrg3s_status dmrg3s_mpo_create(int32_t model, int32_t nsites, const double* params,
                                int32_t nbonds, const int32_t* bonds, const double* couplings,
                                dmrg3s_mpo* out);
dmrg3s_status dmrg3s_mpo_destroy(dmrg3s_mpo mpo);
/* View of site i (pointers into the handle, valid until dmrg3s_mpo_destroy). */
dmrg3s_status dmrg3s_mpo_get_site(dmrg3s_mpo mpo, int32_t i, dmrg3s_mpo_site* site);

/* ---- library-owned DMRG3S state: the local update and the sweep ------------- */

typedef struct dmrg3s_state_s* dmrg3s_state;

/* Factorisation of the truncation's per-sector SVD (Sec. V step 4); all FP64.
 * DMRG3S_SVD_GESVD is the value of a zero-initialised struct;
 * DMRG3S_SVD_AUTO is the Python binding's default. */
typedef enum dmrg3s_svd_method {
  DMRG3S_SVD_GESVD = 0,   /* cuSOLVER gesvd per sector on concurrent streams      */
  DMRG3S_SVD_JACOBI = 1,  /* cuSOLVER QR, then one-sided Jacobi on R^T in this
                             library's kernels, every sector in each launch
                             (dmrg3s_svd); an update whose Jacobi sweeps do not
                             converge redoes its SVD with gesvd
                             (dmrg3s_update_info.svd_fallback)                    */
  DMRG3S_SVD_AUTO = 2     /* per update (per batched step): JACOBI when the
                             update is FP64 and its largest sector's smaller
                             side is >= 192, else GESVD (measured on GB300:
                             the Jacobi rounds win on the large sectors of
                             FP64 updates; gesvd on mid-size sectors, and
                             after 3xTF32 / TF32 eigensolvers, whose ~1e-7
                             noise slows the Jacobi sweeps)                   */
} dmrg3s_svd_method;

typedef struct dmrg3s_update_opts {
  int32_t m_max;            /* bond dimension kept after truncation (Sec. V step 4) */
  int32_t lanczos_kmax;     /* <= 0: 40                                            */
  double lanczos_tol;       /* <= 0: 1e-10; with 3xTF32 products at least 3e-7 and
                               with TF32 at least 3e-4 (the products' accuracy)      */
  double trunc_eps;         /* singular values <= eps * s_max are dropped; <= 0: 1e-12 */
  dmrg3s_precision precision;
  int32_t skip_eigensolver; /* != 0: keep M as is (a pure gauge/expansion move)    */
  dmrg3s_svd_method svd;    /* factorisation of the truncation                     */
} dmrg3s_update_opts;

typedef struct dmrg3s_update_info {
  double lambda;            /* eigensolver value lambda* (step 1)                 */
  double energy_before;     /* E_i: energy of the state entering the update        */
  double energy_after;      /* E_f: Rayleigh quotient after truncation (step 7)    */
  double discarded_weight;  /* sum of the squared discarded singular values        */
  int32_t lanczos_iters;
  int32_t new_bond_dim;
  int32_t svd_fallback;     /* 1: the Jacobi SVD did not converge and gesvd was used */
  int32_t svd_sweeps;       /* Jacobi sweeps of the truncation's SVD (0 with gesvd)  */
} dmrg3s_update_info;

/* Creates a state for a chain of `nsites` sites: MPO tensors W[0..n-1] (host,
 * copied) and site tensors M[0..n-1] (device data, copied).  The MPS must be
 * in mixed-canonical form with orthogonality centre `centre` (sites left of
 * it left-normalised, right of it right-normalised, Sec. II).  left_env /
 * right_env are the boundary environments L_0 / R_{l+1} (device data, copied);
 * NULL means the trivial 1x1x1 environment equal to 1, which requires bond
 * and MPO bond dimension 1 there.  All environments up to the centre are
 * built on the device.  The truncation's per-sector SVDs run on several
 * streams at once, each with its own cuSOLVER handle and host thread: about
 * one per four charge sectors, at least four, at most 8 (or the value 1..16
 * of the environment variable DMRG3S_SVD_STREAMS read here).  The copies
 * and environment builds run on `stream` (the inputs must be ready there);
 * synchronous.  Errors: ARG, SHAPE, QN, CUDA, OOM. */
dmrg3s_status dmrg3s_state_create(dmrg3s_ctx ctx, int32_t nsites, const dmrg3s_mpo_site* W,
                                  const dmrg3s_site* M, const dmrg3s_env* left_env,
                                  const dmrg3s_env* right_env, int32_t centre,
                                  dmrg3s_state* out, dmrg3s_stream stream);
dmrg3s_status dmrg3s_state_destroy(dmrg3s_state state);

/* One DMRG3S local update at the current centre i (Sec. V, steps 1-7), moving
 * the centre to i + dir:
 *   dir = +1: Lanczos for M_i; P_i = alpha L_{i-1} M_i W_i (Eq. subexp-ourt);
 *     M~ = [M_i P_i], B~_{i+1} = [B_{i+1}; 0] (Sec. IV A); FP64 SVD per charge
 *     sector, truncation to m_max states; A~_i = U; B~_{i+1} = S V^dagger B~;
 *     L_i from A~_i; E_f = <B~|H_eff(i+1)|B~> / <B~|B~>.
 *   dir = -1: the mirror image with P_i = alpha R_{i+1} M_i W_i, M~ = [M_i; P_i].
 * alpha = 0 skips the expansion (plain single-site update).  Synchronous
 * (the SVD's singular values are read back to choose the kept states).  An
 * error in the middle of an update leaves the state in an unspecified (but
 * freeable) condition. */
dmrg3s_status dmrg3s_local_update(dmrg3s_state state, int32_t dir, double alpha,
                                  const dmrg3s_update_opts* opts, dmrg3s_update_info* info,
                                  dmrg3s_stream stream);

/* Adaptive mixing factor (Sec. VI).  With dE_O = lambda* - E_i and
 * dE_T = E_f - lambda*, r = dE_T / |dE_O|, after every local update:
 *   |dE_O| < 1e-13 |lambda*|       -> alpha *= down
 *   dE_T < 0 or r < target          -> alpha *= up
 *   r > 1                           -> alpha *= down^2
 *   otherwise                       -> alpha *= down
 * clamped to [alpha_min, alpha_max]; fixed != 0 keeps alpha constant. */
typedef struct dmrg3s_alpha_rule {
  double alpha0, target, up, down, alpha_min, alpha_max;
  int32_t fixed;
} dmrg3s_alpha_rule;

typedef struct dmrg3s_sweep_opts {
  int32_t max_sweeps;
  double conv_tol;          /* stop when |E_k - E_{k-1}| / |E_k| < conv_tol        */
  dmrg3s_update_opts update;
  /* Precision ladder.  With switch_tol > 0 the sweeps run with
   * update.precision (the bulk precision, e.g. DMRG3S_TF32X3) until the
   * relative energy change between two sweeps drops below switch_tol, and
   * with final_precision (normally DMRG3S_FP64) from the next sweep on;
   * conv_tol is then tested only between two sweeps that both ran with
   * final_precision.  switch_tol <= 0: update.precision throughout. */
  dmrg3s_precision final_precision;
  double switch_tol;
  /* Optional traces (host arrays, may be NULL), max_sweeps * 2 * (l - 1)
   * entries for alphas and max_sweeps entries for seconds:
   *  alphas[k]  = the mixing factor after local update k (the value the
   *               alpha rule returns, i.e. the one update k + 1 uses);
   *  seconds[s] = host wall time from the call's start to the end of sweep s. */
  double* alphas;
  double* seconds;
} dmrg3s_sweep_opts;

typedef struct dmrg3s_sweep_report {
  int32_t sweeps, converged, lanczos_iters;
  int32_t svd_fallbacks;   /* updates whose Jacobi SVD fell back to gesvd */
  double energy, alpha;
  int32_t bulk_sweeps;     /* sweeps run with the bulk precision (all without a ladder) */
  int32_t pad;
} dmrg3s_sweep_report;

/* Sweeps (Sec. V): each sweep is a right-to-left pass over sites l..2 followed
 * by a left-to-right pass over sites 1..l-1, one local update per site with
 * the adaptive alpha; the state's centre must be on the last site.  energies
 * (may be NULL) receives E_f after every sweep (max_sweeps entries); E_f is
 * an FP64 Rayleigh quotient in every precision.  Errors: those of
 * dmrg3s_local_update, ARG (opts). */
dmrg3s_status dmrg3s_sweep(dmrg3s_state state, const dmrg3s_alpha_rule* rule,
                           const dmrg3s_sweep_opts* opts, double* energies,
                           dmrg3s_sweep_report* report, dmrg3s_stream stream);

/* Batches of independent states (chains), one context.  The local updates
 * of all states of a batch run together: every contraction stage (the H_eff
 * products of the Lanczos recursion, the expansion terms, the environment
 * updates, the energy after truncation) is one grouped launch over the
 * blocks of every state (the plans of the states merged, their operands
 * copied into shared arrays), the Lanczos dot products and updates are one
 * launch each over all states' vectors, and the truncation SVD is one call
 * over every charge sector of every state.  Each state keeps its own
 * options, direction, alpha and stopping rules, so that every state gets
 * the result of its own dmrg3s_local_update / dmrg3s_sweep (up to the
 * summation order of the merged reductions).  The states must be distinct
 * and share one context and one SVD method (update.svd).  Synchronous.
 * Errors: those of dmrg3s_local_update; ARG (mixed contexts or SVD methods,
 * a state twice).  As with dmrg3s_local_update, an error in the middle of a
 * step leaves the states of the batch in an unspecified (but freeable)
 * condition: destroy them and start again. */
/* One local update on each of nstates states: dirs[k], alphas[k], opts[k]
 * for state k, infos[k] its result (as dmrg3s_local_update). */
dmrg3s_status dmrg3s_local_update_batch(const dmrg3s_state* states, int32_t nstates,
                                        const int32_t* dirs, const double* alphas,
                                        const dmrg3s_update_opts* opts, dmrg3s_update_info* infos,
                                        dmrg3s_stream stream);
/* dmrg3s_sweep on each of nstates states with rules[k], opts[k] (its own
 * max_sweeps, conv_tol, ladder and traces), energies[k] (may be NULL, or the
 * array itself may be NULL) and reports[k].  The states advance one local
 * update per step, all states that are still sweeping together; a state
 * that has converged or run its max_sweeps leaves the batch.  The states may
 * differ in length, bond dimensions, MPO and precision (states in different
 * precisions share the launches of their precision). */
dmrg3s_status dmrg3s_sweep_batch(const dmrg3s_state* states, int32_t nstates,
                                 const dmrg3s_alpha_rule* rules, const dmrg3s_sweep_opts* opts,
                                 double* const* energies, dmrg3s_sweep_report* reports,
                                 dmrg3s_stream stream);

/* Current centre and energy (E_f of the last update, or the Rayleigh quotient
 * at creation). */
dmrg3s_status dmrg3s_state_centre(dmrg3s_state state, int32_t* centre, double* energy);

/* Bonds of site i (nsec, charges [nsec][nsym], dims) and its element count;
 * any output may be NULL.  Arrays must hold the current nsec entries (query
 * with NULL first). */
dmrg3s_status dmrg3s_state_site_info(dmrg3s_state state, int32_t i, int32_t* nsec_left,
                                     int32_t* q_left, int64_t* dim_left, int32_t* nsec_right,
                                     int32_t* q_right, int64_t* dim_right, int64_t* nelem);

/* MPO-entry gradients of <Psi|H|Psi> for every site of the state's current
 * MPS (mixed canonical around its centre): G_i as dmrg3s_mpo_grad_site, with
 * the stored environments on the near side of the centre and environments
 * of the current tensors rebuilt on the far side.  G (HOST, may be NULL)
 * receives the G_i concatenated in site order, each d*d*wl_i*wr_i doubles;
 * dW (HOST, may be NULL) holds dW_i/dtheta in the same layout, and
 *   *dE = sum_i <G_i, dW_i/dtheta> / <Psi|Psi>
 * (0 when dW is NULL).  len is the summed size (checked when G or dW is
 * given).  *norm2 = <Psi|Psi> = <M_c|M_c>.  Runs on `stream`; synchronous.
 * Errors: ARG, SHAPE, OOM, CUDA, NUMERIC (zero norm). */
dmrg3s_status dmrg3s_mpo_grad(dmrg3s_state state, double* G, const double* dW, int64_t len,
                              double* dE, double* norm2, dmrg3s_stream stream);

/* Ground-state energy and its derivatives with respect to the couplings of
 * a built-in model, for a state whose MPO is that model at `params`
 * (DMRG3S_MODEL_XXZ: {J, Delta}; DMRG3S_MODEL_HUBBARD: {t, U}; nparams = 2):
 *   *energy   = <Psi|H|Psi> / <Psi|Psi> = <G_c, W_c> / <Psi|Psi> at the centre c,
 *   dE[k]     = sum_i <G_i, dW_i/dtheta_k> / <Psi|Psi>  (Hellmann-Feynman),
 * with G_i the MPO-entry gradients of dmrg3s_mpo_grad.  Every MPO tensor of
 * these models is affine in each coupling, so the library builds
 * dW_i/dtheta_k = W_i(theta + e_k) - W_i(theta) exactly.  The derivative is
 * that of the energy of the given state; it equals the derivative of the
 * ground-state energy to first order in the state's error.  Runs on
 * `stream`; synchronous.  Errors: ARG, SHAPE (the state's MPO is not the
 * model at params), UNSUPPORTED (other models), OOM, CUDA, NUMERIC. */
dmrg3s_status dmrg3s_energy_grad(dmrg3s_state state, int32_t model, int32_t nparams,
                                 const double* params, double* energy, double* dE,
                                 dmrg3s_stream stream);

/* Copies site i (canonical layout, nelem doubles) to dst (device or host). */
dmrg3s_status dmrg3s_state_site_copy(dmrg3s_state state, int32_t i, double* dst,
                                     dmrg3s_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* DMRG3S_H */
