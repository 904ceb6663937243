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
  DMRG3S_ERR_UNSUPPORTED = 10   /* valid request this build does not implement  */
} dmrg3s_status;

typedef enum dmrg3s_precision {
  DMRG3S_FP64 = 0,    /* all contractions in double precision (CUDA cores)          */
  DMRG3S_TF32X3 = 1,  /* 3xTF32 split products on tcgen05 tensor cores, FP32 accum. */
  DMRG3S_TF32 = 2     /* single-pass TF32 on tcgen05 tensor cores, FP32 accumulate  */
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

#ifdef __cplusplus
}
#endif
#endif /* DMRG3S_H */
