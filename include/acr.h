/*
 * acr.h -- C ABI of the GB300 block cyclic reduction solver (Accelerated
 * Cyclic Reduction, Chavez, Turkiyyah & Keyes, "A Direct Elliptic Solver Based
 * on Hierarchically Low-rank Schur Complements").
 *
 * The solver handles a block tridiagonal system  M u = f,
 *
 *     M = tridiag(A_i, D_i, C_i),   i = 0 .. nblk-1,  blocks blksz x blksz,
 *
 * (Section 3, the block tridiagonal form of the 2D operator; the paper names
 * the off-diagonal blocks E_i and F_i, here A_i = E_i is the sub-diagonal
 * block of row i and C_i = F_i the super-diagonal one).  acr_factor runs the
 * reduction phase of block cyclic reduction (Section 3: even/odd permutation,
 * block-wise inversion of the eliminated diagonal blocks, Schur complement of
 * Eq. "fund", recursion down to one block) and keeps every level's factors
 * resident on the GPU; acr_solve runs the forward right-hand-side reduction
 * (f^(1) = f_odd - H21 H11^-1 f_even, Eq. "fund") and the back-substitution.
 *
 * Conventions common to every call
 *  - Blocks are column-major (element (r, c) of a block at r + c*blksz) and
 *    the nblk blocks of each of A, D, C are contiguous (block stride
 *    blksz*blksz).  A[0] and C[nblk-1] are never read.
 *  - Right-hand sides B are N x nrhs column-major with leading dimension
 *    N = nblk*blksz, in natural block order.
 *  - Every pointer may be host or device memory; the library detects which
 *    (cudaPointerGetAttributes).  Device memory must belong to the handle's
 *    device (the current device at acr_factor time); memory of another GPU is
 *    rejected with ACR_ERR_INVALID_ARG.  The caller keeps ownership of its buffers
 *    and may free them as soon as the call returns; the library copies what
 *    it keeps.
 *  - Every call is synchronous with respect to the host: when it returns, the
 *    work it queued on its stream has finished (results are in B).
 *  - Every call returns an acr_status.  On failure nothing is leaked, *out is
 *    set to NULL, and acr_last_error() describes the failure (for a singular
 *    block: the reduction level and the block index at that level).
 *  - One GPU: the current CUDA device at acr_factor time is used for the
 *    lifetime of the handle.
 */
#ifndef ACR_H
#define ACR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct acr_ctx *acr_handle; /* opaque; owned by the library */

enum acr_status {
    ACR_OK = 0,
    ACR_ERR_INVALID_ARG = -1,   /* bad size, NULL pointer, NaN/Inf in input */
    ACR_ERR_OOM = -2,           /* device allocation failed / over budget */
    ACR_ERR_SINGULAR = -3,      /* an eliminated block has a zero pivot */
    ACR_ERR_NOT_CONVERGED = -4, /* refinement missed ir_tol in ir_max_iter */
    ACR_ERR_CUDA = -5,          /* a CUDA call failed */
    ACR_ERR_TIMEOUT = -6        /* a bounded device-side wait gave up */
};

enum acr_precision {
    /* every step in FP64 (the plain GPU FP64 path) */
    ACR_FP64 = 0,
    /* factor and sweeps in FP32 with the block products on TF32 tensor cores
     * (three-term split, FP32-accurate), wrapped in iterative refinement whose
     * residual r = f - M x (original operator) and correction x += d are FP64 */
    ACR_FP32TC_IR = 1,
    /* as ACR_FP32TC_IR but the block products on FP32 CUDA cores */
    ACR_FP32_IR = 2
};

enum acr_input_kind {
    /* A, D, C: nblk dense blksz x blksz blocks each (layout above) */
    ACR_DENSE = 0,
    /* compact form of a 5-point stencil: D holds 3*blksz values per block,
     * [sub-diagonal, diagonal, super-diagonal] of the tridiagonal D_i
     * (sub[0] and super[blksz-1] ignored); A and C hold blksz values per block,
     * the diagonals of the diagonal blocks A_i and C_i (Section 3: D_i is
     * tridiagonal, E_i and F_i are diagonal) */
    ACR_BANDED = 1
};

typedef struct {
    int precision;      /* enum acr_precision, default ACR_FP64 */
    int input_kind;     /* enum acr_input_kind, default ACR_DENSE */
    int leaf;           /* HODLR leaf size for tol > 0 (0: library choice) */
    int max_rank;       /* cap on HODLR off-diagonal ranks (0: none) */
    int m_stop;         /* stop the reduction at this many blocks; 1 only */
    double ir_tol;      /* refinement target ||f - M x||_2 / ||f||_2 per column
                           (default 1e-8) */
    int ir_max_iter;    /* cap on preconditioner solves per acr_solve (default 20) */
    void *stream;       /* cudaStream_t to run on (it must outlive the handle:
                           the factorization's memory is allocated and freed
                           in stream order on it); NULL: a library stream */
    int refine;         /* enum acr_refine, default ACR_REFINE_FGMRES */
    int h_levels;       /* tol > 0 with ACR_BANDED input: reduction levels carried
                           out in HODLR arithmetic (Section 3: H-inverse of the
                           eliminated blocks, H-products and H-sums truncated to
                           tol / 10), the remaining levels with dense blocks
                           compressed afterwards.  0 (default): from level 0 on, as long as
                           the ranks stay small (at most ACR_HRANK_SWITCH);
                           k > 0: at most k levels; -1: none (every level dense,
                           compressed after the reduction) */
    int h_sketch;       /* 1 (default): in HODLR arithmetic, a node whose summed
                           factors are much wider than the operands' ranks is
                           first truncated through a randomized range sketch
                           (Rademacher test matrix, oversampling >= 6), with the
                           exact truncation only where the sketch's rank comes
                           within 6 of its width; 0: exact truncation only */
} acr_opts;

/* Largest off-diagonal rank of a level's blocks for which the automatic
 * choice (h_levels = 0) continues in HODLR arithmetic.  A level also goes
 * dense when its HODLR inverses miss the identity on random vectors by more
 * than 1e4 times the truncation tolerance (see h_check in acr_stats_t), and
 * for the FP32 factor the automatic choice tries no further level once the
 * misses' growth, extrapolated geometrically from the last two levels,
 * passes that limit (there the miss grows by orders of magnitude per level
 * once the reduced blocks turn ill-conditioned).  The
 * HODLR arithmetic truncates at max(tol / 10, a few units of the factor's
 * rounding), so that the truncations accumulated over the levels keep the
 * solve near tol. */
#define ACR_HRANK_SWITCH 32

#define ACR_FGMRES_RESTART 50

enum acr_refine {
    /* restarted FGMRES(ACR_FGMRES_RESTART) in FP64, right-preconditioned by the factor's
     * sweeps (converges where plain refinement diverges, e.g. indefinite
     * Helmholtz, whose reduced blocks amplify rounding errors) */
    ACR_REFINE_FGMRES = 0,
    /* classic iterative refinement x += M^-1 (f - A x) */
    ACR_REFINE_IR = 1,
    /* no refinement: one sweep (ACR_ERR_NOT_CONVERGED if the residual misses
     * ir_tol) */
    ACR_REFINE_NONE = 2
};

/* Fill *o with the defaults listed above. */
void acr_default_opts(acr_opts *o);

/* Factor (reduction phase of Section 3) with default options.
 *  nblk, blksz >= 1.  tol <= 0: uncompressed blocks (dense block cyclic
 *  reduction, FP64).  tol > 0: blocks stored in HODLR form with off-diagonal
 *  ranks truncated at sigma_k > max(tol, c eps) * sigma_1 of each node (eps
 *  of the factor's precision; c = 8 for FP32 factors, 32 for FP64).
 *  On success *out receives a handle that keeps the factorization on the GPU
 *  until acr_free. */
int acr_factor(int nblk, int blksz, const double *A, const double *D, const double *C,
               double tol, acr_handle *out);

/* As acr_factor with explicit options (o may be NULL for the defaults). */
int acr_factor_ex(int nblk, int blksz, const double *A, const double *D, const double *C,
                  double tol, const acr_opts *o, acr_handle *out);

/* Solve M X = B in place (forward reduction + back-substitution of Section 3,
 * refinement in the mixed-precision modes).  B: N x nrhs, overwritten with X.
 * nrhs >= 0.  Solves on one handle may run concurrently from several host
 * threads: each call uses its own workspace.  From its second preconditioner
 * application on, a solve replays its sweeps as a CUDA graph captured on the
 * handle's stream (not on the legacy NULL stream, nor on a stream that is
 * already being captured, where the same launches are issued directly). */
int acr_solve(acr_handle h, double *B, int nrhs);

/* As acr_solve, also returning per column the final relative residual
 * ||b - M x||_2 / ||b||_2 (resid_out, nrhs doubles, may be NULL; computed in
 * FP64 with the original operator) and the refinement iterations taken
 * (iters_out, may be NULL; 0 when no refinement ran). */
int acr_solve_ex(acr_handle h, double *B, int nrhs, double *resid_out, int *iters_out);

/* Release everything the handle holds.  NULL is a no-op.  Device memory goes
 * back, in stream order, to the device's default stream-ordered pool; the
 * library raises that pool's release threshold to 64 GiB (once per device,
 * never lowering it), so freed memory stays mapped in this process for the
 * next factorization instead of being returned to the driver. */
void acr_free(acr_handle h);

typedef struct {
    int nblk, blksz, levels, precision, compressed;
    size_t factor_bytes;     /* device bytes held by the factorization */
    size_t operator_bytes;   /* device bytes of the FP64 operator copy */
    double factor_flops;     /* algorithmic flops of the last factor */
    double factor_ms;        /* device time of the last factor */
    double solve_ms;         /* device time of the last solve (all iterations) */
    int ir_iters;            /* refinement iterations of the last solve */
    double ir_resid_max;     /* max relative residual over columns, last solve */
    int rank_max[32];        /* HODLR: max off-diagonal rank per level */
    double rank_mean[32];    /* HODLR: mean off-diagonal rank per level */
    /* per kernel class, last factor / last solve: device time (CUDA events
     * on the library stream), algorithmic work, launches */
    double gemm_ms, gemm_flops;          /* block products (factor) */
    double inv_ms, inv_flops;            /* block inversions (factor) */
    double sweep_ms, sweep_bytes;        /* solve sweeps, all passes */
    long long gemm_launches, inv_launches, sweep_launches;
    long long launches_factor;           /* all kernel launches, last factor */
    long long launches_solve;            /* all kernel launches, last solve */
    double compress_ms;                  /* HODLR compression of the last factor
                                            (sketches, node SVDs, packing; 0 when
                                            tol <= 0); included in factor_ms */
    int h_levels;                        /* levels reduced in HODLR arithmetic */
    double h_ms;                         /* their device time (included in factor_ms) */
    double h_flops;                      /* algorithmic flops of their products */
    double h_host_ms;                    /* host time spent building their launches */
    double h_check[32];                  /* per level reduced in HODLR arithmetic (and the
                                            first level that failed it): the inverse check
                                            max_j ||D_j (D_j^-1 x) - x|| / ||x|| on random x */
    long long h_nodes;                   /* node truncations in HODLR arithmetic */
    long long h_sketch_redo;             /* of which the sketch left to the exact pass */
    long long sweep_passes;              /* preconditioner applications (forward +
                                            back-substitution sweeps) in sweep_ms */
} acr_stats_t;

/* Copy the handle's statistics into *s. */
int acr_stats(acr_handle h, acr_stats_t *s);

/* Device bytes that acr_factor_ex would keep for these sizes and options
 * (uncompressed storage; an upper bound when tol > 0).  Used for admission
 * under a memory budget. */
int acr_factor_bytes(int nblk, int blksz, double tol, const acr_opts *o, size_t *bytes);

/* Upper bound of the device bytes one acr_solve_ex call allocates for its
 * workspace (FGMRES bases, sweep vectors, partial sums) for nrhs right-hand
 * sides with these options; the factorization's own bytes are not included.
 * Used, with acr_factor_bytes, for admission under a memory budget. */
int acr_solve_bytes(int nblk, int blksz, int nrhs, const acr_opts *o, size_t *bytes);

/* Message of the last failed call on this host thread ("" if none). */
const char *acr_last_error(void);

/* ---- batched block inversion without device allocation -------------------
 * The paper has no counterpart to this call: it is a service for callers that
 * cannot allocate device memory when they need it -- code running inside
 * another framework's memory pool that has reserved nearly all of the GPU,
 * latency-critical paths that cannot absorb an allocation, its failure or the
 * device synchronisation that freeing can cause.
 *
 * Inverts, in place, `count` blocks of blksz x blksz (column-major, block
 * stride blksz*blksz) with the same partial-pivoting Gauss-Jordan kernels as
 * the factorization, in FP64.  mats and info are device memory of the
 * current device, owned by the caller (host memory or memory of another GPU
 * returns ACR_ERR_INVALID_ARG before anything is launched); info receives per
 * block 0, or k+1 if pivot k was zero or not finite (that block's contents are
 * then meaningless).
 *
 * Every temporary lives in one fixed scratch array of
 * ACR_NOALLOC_SCRATCH_BYTES compiled into the library, which each GPU that
 * loads the library holds until the process exits; the call allocates and
 * frees nothing.  A batch whose temporaries exceed that size returns
 * ACR_ERR_INVALID_ARG (split the batch); blocks up to blksz 159 need no
 * scratch at all.
 *
 * The work is queued on `stream` (a cudaStream_t, NULL for the legacy
 * default stream) and the call returns without waiting for it.  All calls
 * share the one scratch array per device, so calls whose work can overlap on
 * the GPU (different streams, or host threads racing) corrupt each other:
 * order them on one stream.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call outside any stream capture.  The address is kept per
 * device and CUDA context: after a device reset the next call looks it up
 * again (make that call outside capture too). */
#define ACR_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
int acr_block_inverse_noalloc(int blksz, int count, double *mats, int *info, void *stream);

/* Batched low-rank truncation (Section 3: the recompression that follows
 * every H-sum and H-product of the reduction in HODLR arithmetic, here on
 * caller-supplied factors).  For each of `count` nodes, U_i and V_i (s x R,
 * column-major, FP64, node i at offset i*s*R) define M_i = U_i V_i^T.  The
 * kept rank r_i is the number of singular values of M_i above
 * tol * sigma_1(M_i) (tol in [0, 1); at most min(s, R)).  Outputs, same
 * layout: Vout_i holds r_i orthonormal columns spanning the leading right
 * singular vectors, then zero columns; Uout_i = U_i V_i^T Vout_i, so that
 * Uout_i Vout_i^T is the truncation of M_i; ranks[i] = r_i.
 *
 * Method: QR of U, Y = V R_U^T, QR of Y, one-sided Jacobi SVD of R_Y (the
 * exact pass); with sketch = k > 0 (k < min(s, R)) the randomized first pass
 * instead works on the range of U (V^T Omega) for a k-column Rademacher
 * Omega, and a node whose rank comes within 6 of k is redone by the exact
 * pass (*exact_redo, if not NULL, receives how many).  precision: ACR_FP64,
 * or ACR_FP32TC_IR / ACR_FP32_IR for FP32 arithmetic (inputs and outputs
 * stay FP64).  U, V, Uout, Vout, ranks may be host or device memory (of the
 * current device); the caller owns them.  Synchronous.  Errors:
 * ACR_ERR_INVALID_ARG (sizes, NULL, tol, memory of another GPU, panels above
 * the kernel's shared memory), ACR_ERR_OOM, ACR_ERR_CUDA. */
int acr_lowrank_truncate(int count, int s, int R, const double *U, const double *V, double tol,
                         int precision, int sketch, double *Uout, double *Vout, int *ranks,
                         int *exact_redo);

#ifdef __cplusplus
}
#endif
#endif /* ACR_H */
