/*
 * tk.h -- C ABI of the GB300 symmetric TensorMap contraction library (libtk).
 *
 * The library contracts two symmetric tensor maps whose legs are graded spaces of Z2, U(1) or
 * SU(2) sectors with multiplicities, following the statement of the problem in the TensorKit
 * paper (arXiv 2508.10076):
 *   - a graded space is a list of (sector, multiplicity) pairs plus a duality flag (Sec. 5.2);
 *   - a tensor map t : W_1 (x) ... (x) W_N2 -> V_1 (x) ... (x) V_N1 is stored as one block per
 *     coupled sector, each block holding the reduced arrays of its fusion-tree pairs
 *     (Sec. 3.2 eq. abeliangrouping, Sec. 4.1 canonical trees and block embedding);
 *   - permute(t, (p, q)) follows Algorithm 2 (non-abelian: Algorithm 10);
 *   - contract follows Algorithm 4 / Algorithm 8: permute A, permute B, one GEMM per coupled
 *     sector (zero block when the inner dimension is empty), permute the result.
 *
 * Conventions
 *   - Sector encoding: Z2 in {0,1}; U(1) integer charge; SU(2) twice the spin (2j).
 *   - Leg numbering is 0-based: codomain legs 0..N1-1, then domain legs N1..N1+N2-1 in forward
 *     order (the paper numbers them from 1, Algorithm 2).
 *   - Storage layout (fixed; the paper leaves the order "arbitrary but fixed"): blocks by coupled
 *     sector ascending, each block a column-major rows x cols matrix, blocks concatenated; inside a
 *     block the canonical trees occupy consecutive row (splitting) / column (fusion) ranges,
 *     trees ordered colexicographically (first leg fastest) by uncoupled labels, then by inner
 *     labels; a reduced array is column-major with the first leg fastest.  A leg of a dual space
 *     carries the dual sector as its tree label.
 *   - Element types: TK_F64 (double) and TK_C128 (interleaved double real/imag).
 *
 * Ownership: every object returned through an out-parameter is owned by the caller and released
 * with the matching *_destroy.  Device buffers passed to execution calls are borrowed; the
 * library never frees them.  Plans own their device-resident task tables.
 *
 * Errors: every int-returning call returns TK_OK (0) or a TK_ERR_* code; no exception crosses the
 * ABI.  tk_ctx_last_error() gives a message for the last failure on that context.  Kernel
 * launches are asynchronous: device-side failures (a bounded wait that gave up, a launch error)
 * are reported by the next tk_ctx_sync().
 */
#ifndef TK_H
#define TK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define TK_OK 0
#define TK_ERR_ARG 1            /* invalid argument (null pointer, bad size, bad enum)        */
#define TK_ERR_SPACE_MISMATCH 2 /* domain(A~) != codomain(B~) including duality (Sec. 2.3)    */
#define TK_ERR_PERM 3           /* (p, q) is not a permutation of the legs (Algorithm 2)      */
#define TK_ERR_SECTOR 4         /* sector label not valid for the symmetry                    */
#define TK_ERR_OOM 5            /* host or device allocation failed                           */
#define TK_ERR_CUDA 6           /* a CUDA runtime call failed                                 */
#define TK_ERR_UNSUPPORTED 7    /* valid request this build does not implement                */
#define TK_ERR_TIMEOUT 8        /* a bounded device-side wait gave up                         */
#define TK_ERR_WORKSPACE 9      /* workspace too small                                        */
#define TK_ERR_NO_DEVICE 10     /* execution call on a host-only context                      */
#define TK_ERR_BUDGET 11        /* the context's device-memory budget would be exceeded       */

/* ---- enums ------------------------------------------------------------------------------ */
#define TK_SYM_Z2 0
#define TK_SYM_U1 1
#define TK_SYM_SU2 2
/* Deligne products (Sec. 5.2, product sectors): a sector is a pair (a1, a2) of the factors'
 * labels, passed as the int32 a1 * 4096 + f(a2) with f(a2) = a2 + 2048 for a U(1) second factor
 * (|a2| < 2048) and f(a2) = a2 otherwise (SU(2): 2j <= 4095).  The integer order is then the
 * lexicographic order of the pairs.  Fusion, duals and dimensions act factor by factor; F and R
 * symbols are products of the factors' symbols. */
#define TK_SYM_U1_SU2 3 /* U(1) x SU(2), e.g. charge x spin */
#define TK_SYM_Z2_U1 4  /* Z2 x U(1), e.g. fermion parity x charge (bosonic braiding) */

#define TK_F64 0
#define TK_C128 1

/* GEMM arithmetic of the per-sector products (step 2 of Algorithm 8). */
#define TK_GEMM_FP64 0       /* plain FP64 on the CUDA cores                                   */
#define TK_GEMM_OZAKI_BF16 1 /* FP64 operands split into BF16 slices, tcgen05 products, FP32
                                exact accumulation of the leading levels, FP64 recombination */
#define TK_GEMM_TF32X3 2     /* 3xTF32 on tcgen05 (about FP32 accuracy; reported, not gated)   */

typedef struct tk_ctx tk_ctx;
typedef struct tk_space tk_space;
typedef struct tk_tmap tk_tmap;
typedef struct tk_plan tk_plan;

/* ---- library ---------------------------------------------------------------------------- */
int tk_version(void);                       /* major*10000 + minor*100 + patch              */
const char* tk_status_string(int status);   /* static string, never NULL                    */

/* ---- context ------------------------------------------------------------------------------
 * device >= 0: the CUDA device all plans and launches of this context use (it is made current
 * inside every call).  device < 0: host-only context -- spaces, tensor structures and plans can
 * be built and inspected, execution calls return TK_ERR_NO_DEVICE.
 *
 * stream (a cudaStream_t, may be NULL = legacy default stream): the context's stream.  Execution
 * calls given a NULL stream run on it, and plan tables are uploaded on it (each upload waits for
 * the stream).
 *
 * Allocator hooks: every device allocation the library makes itself -- plan tables, the context's
 * status word, tk_ctx_alloc / tk_tmap_alloc buffers -- goes through alloc(bytes, user), which
 * returns device memory of the context's device (at least 256-byte aligned) or NULL, and is given
 * back through release(ptr, bytes, user).  With both hooks NULL the library uses cudaMalloc /
 * cudaFree; giving only one of them is TK_ERR_ARG.  A hook is called with the context's device
 * current, from the thread that made the library call.  The hooks and `user` must stay valid
 * until every plan built by the context has been destroyed (plan tables are released when the
 * last reference to a plan goes, which may be after tk_ctx_destroy).  Scratch memory of execution
 * calls is never allocated by the library: the caller passes it (workspace arguments). */
typedef void* (*tk_alloc_fn)(size_t bytes, void* user);
typedef void (*tk_free_fn)(void* ptr, size_t bytes, void* user);

/* Concurrency: plans are built and cached under a mutex of the context, so several host threads
 * may plan at once; executions on different streams are independent (each call uses only the
 * buffers and workspace it is given), except that the short fork / join section of a
 * split-precision contraction (its second stream and two events belong to the context) is taken
 * by one call at a time.  Calls that share a workspace must not overlap: a contraction's
 * split-K partials and arrival counters live in its workspace (a plan may serve overlapping
 * calls that each have their own).  A plan must not be destroyed while launches that use it are
 * in flight (with caller hooks nothing waits for them before release is called). */
int tk_ctx_create(int device, void* stream, tk_alloc_fn alloc, tk_free_fn release, void* alloc_user,
                  tk_ctx** out);
void tk_ctx_destroy(tk_ctx* ctx);
const char* tk_ctx_last_error(const tk_ctx* ctx);
/* Waits for `stream` (a cudaStream_t, NULL = the context's stream) and reports deferred device errors
 * (TK_ERR_TIMEOUT if a bounded wait gave up, TK_ERR_CUDA for launch/runtime failures). */
int tk_ctx_sync(tk_ctx* ctx, void* stream);
/* Number of the library's own kernels launched through this context so far. */
int64_t tk_ctx_launch_count(const tk_ctx* ctx);
/* Failure-path self-test of the device-side bounded waits: launches (asynchronously, on
 * `stream`) one CTA that waits on an mbarrier nobody completes, using the same bounded wait as
 * the split-precision GEMM pipeline (limit 2 s).  When the limit runs out the kernel writes the
 * timeout into the context's status word and returns, so the next tk_ctx_sync() returns
 * TK_ERR_TIMEOUT (kernel tag 9 in tk_ctx_last_error), clears the word, and the context stays
 * usable.  Returns TK_OK once launched; TK_ERR_NO_DEVICE for a host-only context. */
int tk_ctx_selftest_timeout(tk_ctx* ctx, void* stream);
/* Device-memory budget (HBM admission).  bytes = 0 removes the budget.  Counted against it: the
 * bytes the library holds (plan tables, status word, tk_ctx_alloc buffers) plus the bytes the
 * caller has reserved.  A library allocation that would exceed it fails with TK_ERR_BUDGET (plan
 * creation returns that code), and so does a reservation: tk_ctx_reserve(bytes) admits work whose
 * memory the caller allocates itself (outputs, workspaces, resident inputs), tk_ctx_release gives
 * the bytes back (TK_ERR_ARG if more than reserved).  Setting a budget below the current use is
 * allowed; later allocations and reservations then fail until use drops.  tk_ctx_memory reports
 * the library's bytes, the reserved bytes, the budget and the number of live library allocations
 * (any out pointer may be NULL). */
int tk_ctx_set_budget(tk_ctx* ctx, size_t bytes);
int tk_ctx_reserve(tk_ctx* ctx, size_t bytes);
int tk_ctx_release(tk_ctx* ctx, size_t bytes);
int tk_ctx_memory(tk_ctx* ctx, size_t* library_bytes, size_t* reserved_bytes, size_t* budget_bytes,
                  int64_t* allocations);
/* Device buffers through the context's allocator, counted against its budget (TK_ERR_BUDGET,
 * TK_ERR_OOM).  tk_ctx_free takes only pointers returned by tk_ctx_alloc / tk_tmap_alloc
 * (TK_ERR_ARG otherwise; NULL is a no-op); the caller makes sure no launch still uses the buffer. */
int tk_ctx_alloc(tk_ctx* ctx, size_t bytes, void** out);
int tk_ctx_free(tk_ctx* ctx, void* ptr);
/* Kernel profiling.  enable != 0: every later launch through ctx is bracketed by CUDA events
 * recorded on its own stream; enable == 0 stops recording.  tk_ctx_profile_read waits for the
 * recorded events and returns, per kernel name (at most max entries, names NUL-terminated in
 * 32-byte slots of `names`), the number of launches and the summed event-measured time in
 * milliseconds; *n_out receives the number of distinct kernels.  Reading clears the record. */
int tk_ctx_profile(tk_ctx* ctx, int enable);
int tk_ctx_profile_read(tk_ctx* ctx, int max, char* names, int64_t* counts, double* total_ms,
                        int* n_out);

/* ---- graded spaces (Sec. 3.1 eq. gradedbasis, Sec. 5.2) ----------------------------------
 * sectors[i], mults[i] for i < nsec: sector labels (unique) and positive multiplicities.
 * is_dual != 0 makes the space V*.  The object is immutable. */
int tk_space_create(tk_ctx* ctx, int sym, int nsec, const int32_t* sectors, const int64_t* mults,
                    int is_dual, tk_space** out);
int tk_space_dual(tk_ctx* ctx, const tk_space* v, tk_space** out);  /* V -> V*              */
void tk_space_destroy(tk_space* v);
int64_t tk_space_dim(const tk_space* v);          /* sum_a n_a d_a  (-1 on NULL)              */
int64_t tk_space_reduced_dim(const tk_space* v);  /* sum_a n_a      (-1 on NULL)              */

/* ---- tensor map structures ----------------------------------------------------------------
 * t : dom[0] (x) ... (x) dom[n_dom-1] -> cod[0] (x) ... (x) cod[n_cod-1]; n_cod + n_dom in
 * [1, 8].  The structure owns copies of the spaces.  Data is not attached: execution calls
 * take device pointers laid out as described at the top of this file. */
int tk_tmap_create(tk_ctx* ctx, int n_cod, const tk_space* const* cod, int n_dom,
                   const tk_space* const* dom, tk_tmap** out);
void tk_tmap_destroy(tk_tmap* t);
int64_t tk_tmap_numel(const tk_tmap* t);          /* number of stored scalars                  */
int tk_tmap_nlegs(const tk_tmap* t, int* n_cod, int* n_dom);
int tk_tmap_leg(tk_ctx* ctx, const tk_tmap* t, int leg, tk_space** out);  /* copy of a leg   */
uint64_t tk_tmap_hash(const tk_tmap* t);          /* structure hash (spaces and duality)       */
int tk_tmap_nblocks(const tk_tmap* t);
/* i-th block (coupled sector ascending): sector label, rows, cols, element offset. */
int tk_tmap_block(const tk_tmap* t, int i, int32_t* sector, int64_t* rows, int64_t* cols,
                  int64_t* offset);
int64_t tk_tmap_ntreepairs(const tk_tmap* t);
/* i-th fusion-tree pair (block order, then splitting tree, then fusion tree).  labels receives
 * N1 + N2 uncoupled labels, then max(N1-2,0) splitting inner labels, the coupled sector, and
 * max(N2-2,0) fusion inner labels; dims receives the N1 + N2 extents of the reduced array.
 * offset = element offset of its first entry, ld = rows of its block.  Any out pointer may be
 * NULL. */
int tk_tmap_treepair(const tk_tmap* t, int64_t i, int32_t* labels, int64_t* offset, int64_t* ld,
                     int64_t* dims);

/* Data of a tensor map (Sec. 2: a TensorMap is its structure plus one block per coupled sector).
 * The device buffer holds the blocks in canonical order (the storage layout above), so host data
 * in that order moves as one copy.  bytes must equal tk_tmap_numel(t) * element size of dtype
 * (8 for TK_F64, 16 for TK_C128), else TK_ERR_ARG.  Asynchronous on stream (NULL: the context's);
 * pinned host memory makes the copy truly asynchronous.  tk_tmap_alloc allocates a device buffer
 * of that size through the context's allocator (release it with tk_ctx_free). */
int tk_tmap_upload(tk_ctx* ctx, const tk_tmap* t, int dtype, const void* host, size_t bytes, void* device,
                   void* stream);
int tk_tmap_download(tk_ctx* ctx, const tk_tmap* t, int dtype, const void* device, void* host, size_t bytes,
                     void* stream);
int tk_tmap_alloc(tk_ctx* ctx, const tk_tmap* t, int dtype, void** out);

/* ---- plans ------------------------------------------------------------------------------------
 * A plan holds everything that depends only on structure: output spaces (Algorithm 2),
 * recoupling coefficients of every fusion-tree transform (F-, B- and R-moves with 6j symbols
 * from the Racah formula, Sec. 4.2), sector matching and the GEMM/zero-fill lists
 * (Algorithm 8), and the device task tables.  Plans are cached per context by structure hash,
 * so creating the same plan twice is cheap. */
int tk_permute_plan(tk_ctx* ctx, const tk_tmap* a, int np, const int* p, int nq, const int* q,
                    int dtype, tk_plan** out);
/* Adjoint t^dagger : dom <- cod of t : cod <- dom (Sec. 2; conjugate for complex data).  With
 * the orthonormal canonical trees, block c of the result is the conjugate transpose of block c of
 * t.  The result is a permute-kind plan: run it with tk_permute, inspect it with tk_plan_output. */
int tk_adjoint_plan(tk_ctx* ctx, const tk_tmap* a, int dtype, tk_plan** out);
/* Algorithm 4: A~ = permute(A, (pa, qa)), B~ = permute(B, (pb, qb)), C~ = A~ o B~,
 * C = permute(C~, (pab, qab)).  (pab, qab) index the legs of C~ = codomain(A~) then domain(B~).
 * gemm_mode is TK_GEMM_*; slices is the number of BF16 slices per operand for
 * TK_GEMM_OZAKI_BF16 (0 = default), ignored otherwise.  Complex data (TK_C128) in a
 * split-precision mode runs as the four real products Re A Re B, Im A Im B, Re A Im B, Im A Re B
 * (the recoupling coefficients are real) on de-interleaved copies in the workspace, combined as
 * (RR - II) + i (RI + IR). */
int tk_contract_plan(tk_ctx* ctx, const tk_tmap* a, int npa, const int* pa, int nqa, const int* qa,
                     const tk_tmap* b, int npb, const int* pb, int nqb, const int* qb,
                     int npab, const int* pab, int nqab, const int* qab, int dtype, int gemm_mode,
                     int slices, tk_plan** out);
/* Composition A o B : cod(A) <- dom(B) of A : cod(A) <- dom(A) and B : cod(B) <- dom(B) with
 * dom(A) = cod(B) (Sec. 2.3): the contraction plan with every leg kept in place (TK_ERR_SPACE_MISMATCH
 * if the spaces or their duality differ). */
int tk_compose_plan(tk_ctx* ctx, const tk_tmap* a, const tk_tmap* b, int dtype, int gemm_mode, int slices,
                    tk_plan** out);
void tk_plan_destroy(tk_plan* plan);
int tk_plan_output(tk_ctx* ctx, const tk_plan* plan, tk_tmap** out);  /* result structure     */
size_t tk_plan_workspace_bytes(const tk_plan* plan);  /* device scratch needed by tk_contract  */
/* Block flops of the plan: sum over executed sector GEMMs of 2 M K N (8 M K N complex), using
 * reduced sizes -- each SU(2) block once (Sec. 4.4). */
double tk_plan_flops(const tk_plan* plan);
/* The part of tk_plan_flops routed to the split-precision tensor-core GEMM (0 for FP64 plans and
 * for products too thin for tensor tiles, which stay on CUDA cores). */
double tk_plan_tensor_flops(const tk_plan* plan);
/* Algorithmic bytes moved by the plan's permute launches (each source element read once per
 * use, each output element written once). */
double tk_plan_permute_bytes(const tk_plan* plan);

/* Host-side inspection of a plan's permute transforms (works on host-only contexts).
 * which: 0 = permute of A (or the permute plan), 1 = permute of B, 2 = permute of the result.
 * Entry k is one (source tree pair, destination tree pair, coefficient) term of Algorithm 10,
 * tree pairs identified by the element offsets of their first entries.  Returns the count, or -1
 * if that permute is absent (identity permutes are skipped). */
int64_t tk_plan_ntransform(const tk_plan* plan, int which);
/* How the device executes one of the plan's permutes (which as above), for tuning and tests:
 * stats[0..2] = contiguous-run tasks, their elements, runs; stats[3..4] = transpose-tile tasks
 * (scalar tiles, or tiles of short vectors contiguous on both sides), their elements; stats[5..6] = element-wise tasks, their elements; stats[7] = tiles. */
int tk_plan_permute_stats(const tk_plan* plan, int which, int64_t* stats);
int tk_plan_transform(const tk_plan* plan, int which, int64_t k, int64_t* src_offset,
                      int64_t* dst_offset, double* coef);

/* ---- execution (asynchronous on `stream`, a cudaStream_t; NULL = the context's stream) --------
 * All pointers are device pointers to buffers laid out as the plan's input/output structures; a
 * pointer may be NULL only when its structure has no elements (no admissible coupled sector), and
 * a call whose output has no elements launches nothing.
 * C is fully overwritten.  A and B are never modified.  In the split-precision modes the products
 * left to the CUDA cores run on a second stream owned by the context, forked from `stream` after
 * the input permutes and joined back before the output permute (a fork and a join in a captured
 * CUDA graph); all work is still ordered after earlier and before later work on `stream`. */
int tk_permute(tk_ctx* ctx, const tk_plan* plan, const void* a, void* c, void* stream);
int tk_contract(tk_ctx* ctx, const tk_plan* plan, const void* a, const void* b, void* c,
                void* workspace, size_t workspace_bytes, void* stream);

/* n planned contractions executed together (batching of concurrent requests; not in the paper,
 * whose contractions run one by one).  Request i reads a[i], b[i], writes c[i] and uses
 * workspace[i] of workspace_bytes[i] >= tk_plan_workspace_bytes(plans[i]); requests may share a
 * plan but not a workspace or an output.  The blocks of all requests share one launch per stage:
 * every input permute in one launch, the zero fill in one, every sector GEMM tile in one grouped
 * GEMM, every output permute in one (a stage with more than 160 segments is split into several
 * launches).  In the split-precision modes the double-float row blocks of all requests share one
 * launch, and up to 32 requests with the same tile width and slice count share one scaling, one
 * slicing and one tensor-core launch.
 * Each c[i] equals what tk_contract would write for that request alone.  All plans must share
 * the dtype and the gemm mode, and complex split-precision plans are not batched (else
 * TK_ERR_UNSUPPORTED); pointer arrays are host arrays of device pointers; n = 0 is a no-op. */
int tk_contract_batch(tk_ctx* ctx, int n, const tk_plan* const* plans, const void* const* a,
                      const void* const* b, void* const* c, void* const* workspace,
                      const size_t* workspace_bytes, void* stream);

/* ---- block SVD and truncation (Algorithm 9, the decomposition after the two-site step of
 * Algorithm 12).  For t : cod <- dom the SVD is block-wise: t = U S V^dagger with the bond space
 * W = sum_c (c, r_c), r_c = min(rows_c, cols_c) over the coupled sectors c of t, U : cod <- W,
 * V^dagger : W <- dom, and the singular values concatenated by sector (descending within a
 * sector; SU(2) values stand for d_c states each).  All blocks are factorised in one launch of a
 * grouped one-sided (Hestenes) Jacobi kernel, one CTA per block, on copies in the workspace; a map
 * without blocks is a no-op (its buffers may then be NULL).
 *   tk_svd_plan     plan for t's structure (dtype TK_F64 or TK_C128);
 *   tk_svd_outputs  structures of U and V^dagger (caller frees with tk_tmap_destroy) and the number
 *                   of singular values;
 *   tk_svd_block    block i: coupled sector, rows, columns and the offset of its singular values;
 *   tk_svd          t -> U, S, V^dagger (device buffers; workspace of tk_plan_workspace_bytes);
 *   tk_svd_truncate keep[i] (0..min(rows, cols)) leading triplets of block i into the truncated
 *                   U : cod <- W', S, V^dagger : W' <- dom with W' = sum_c (c, keep_c) (sectors with
 *                   keep 0 dropped), all concatenated in sector order; with nothing kept it
 *                   copies nothing and the buffers may be NULL. */
int tk_svd_plan(tk_ctx* ctx, const tk_tmap* a, int dtype, tk_plan** out);
int tk_svd_outputs(tk_ctx* ctx, const tk_plan* plan, tk_tmap** u, tk_tmap** vh, int64_t* nvalues);
int64_t tk_svd_nblocks(const tk_plan* plan);
int tk_svd_block(const tk_plan* plan, int64_t i, int32_t* sector, int64_t* rows, int64_t* cols,
                 int64_t* values_offset);
int tk_svd(tk_ctx* ctx, const tk_plan* plan, const void* a, void* u, double* s, void* vh, void* workspace,
           size_t workspace_bytes, void* stream);
int tk_svd_truncate(tk_ctx* ctx, const tk_plan* plan, const int64_t* keep, const void* u, const double* s,
                    const void* vh, void* ut, double* st, void* vht, void* stream);

/* Autotuner (not in the paper): times the candidate work lists of a contraction plan on the given
 * buffers (median of three runs each, CUDA events on `stream`, which is synchronised) and keeps the
 * fastest: FP64 tiles 32 or 64 wide with split-K off or at its maximum, or the built-in heuristic;
 * for split-precision plans then also the tensor-core tile width (64 / 128 columns) and its
 * split-K, and the operand preparation without its k-chunks in shared memory.  Candidates whose workspace would exceed workspace_bytes are skipped, so the plan's
 * tk_plan_workspace_bytes() stays <= workspace_bytes.  The plan's device tables are rebuilt: call
 * it before capturing the plan in a CUDA graph and while no launch of the plan is in flight.
 * c and the workspace are overwritten.  *choice (if not NULL) receives 64 * preparation candidate
 * + 8 * fp64 candidate + split-precision candidate (candidate 0 = heuristic; preparation 1 = no
 * chunks in shared memory, 2 = chunks in shared memory). */
int tk_plan_autotune(tk_ctx* ctx, tk_plan* plan, const void* a, const void* b, void* c, void* workspace,
                     size_t workspace_bytes, void* stream, int* choice);
/* Apply a choice in tk_plan_autotune's encoding without timing anything (to reuse a choice found
 * earlier, or to pin one): the plan's device tables are rebuilt, so call it while no launch of the
 * plan is in flight, and size the workspace from tk_plan_workspace_bytes() afterwards.  Returns
 * TK_ERR_ARG for a value the autotuner cannot produce. */
int tk_plan_set_choice(tk_ctx* ctx, tk_plan* plan, int choice);

/* Contraction without any device allocation -- no counterpart in the paper.  Same result and
 * launch sequence as tk_contract, but the scratch memory (permuted operands and the intermediate
 * C~) comes from a fixed array compiled into libtk instead of a caller-allocated workspace.  It
 * is for callers that cannot allocate device memory: programs whose device memory is owned by
 * another framework's allocator, serving loops that must not take the synchronisation a
 * cudaMalloc can cause, plug-ins handed only their input and output buffers.  The call itself
 * calls no cudaMalloc/cudaFree and no allocating library routine (the plan, built earlier,
 * already holds its device tables).
 *   - Limit: plans whose tk_plan_workspace_bytes() exceeds TK_NOALLOC_SCRATCH_BYTES are rejected
 *     with TK_ERR_WORKSPACE.  Every GPU that loads libtk holds the array until the process exits.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 *     that device current and keeps it for the life of the process; make that first call before
 *     any stream capture, and do not call cudaDeviceReset on that device afterwards (the kept
 *     address would then be stale).
 *   - All calls share the one array, which keeps the previous call's contents; a call writes every
 *     scratch byte it reads, so nothing has to start at zero.  Calls whose kernels overlap on the
 *     GPU (other streams, other host threads) race on the array: serialise them. */
#define TK_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)
size_t tk_noalloc_scratch_bytes(void);  /* TK_NOALLOC_SCRATCH_BYTES as built into the library */
int tk_contract_noalloc(tk_ctx* ctx, const tk_plan* plan, const void* a, const void* b, void* c,
                        void* stream);  /* stream NULL: the context's stream */

/* Host <-> device copies on the context's device (cudaMemcpyAsync; pinned host memory makes
 * them asynchronous). */
int tk_copy_h2d(tk_ctx* ctx, void* dst_device, const void* src_host, size_t bytes, void* stream);
int tk_copy_d2h(tk_ctx* ctx, void* dst_host, const void* src_device, size_t bytes, void* stream);

/* ---- measurement --------------------------------------------------------------------------
 * Peak probe of the FP64 pipe (not in the paper; the denominator of the FP64 sector GEMMs'
 * roofline): a register-only kernel of independent FMA chains on every SM, sized to run about
 * `seconds` (0 < seconds <= 30) on `stream` (NULL: the context's), timed with CUDA events.
 * *tflops = 2 x FMAs / elapsed time; *ms (may be NULL) = the timed launch's duration. */
int tk_probe_fp64_peak(tk_ctx* ctx, double seconds, double* tflops, double* ms, void* stream);

/* ---- topological data (host, exact) ----------------------------------------------------------
 * F^{abc}_d[e; f] (e couples (a b), f couples (b c)): for SU(2) eq. SU2FSymbol with the 6j symbol
 * from Racah's formula evaluated in exact integer arithmetic and rounded once to the nearest
 * double; 1 or 0 for abelian symmetries.  R^{ab}_c (eq. braiding): SU(2) (-1)^(a+b-c).
 * Inadmissible labels give 0. */
double tk_fsymbol(int sym, int32_t a, int32_t b, int32_t c, int32_t d, int32_t e, int32_t f);
double tk_rsymbol(int sym, int32_t a, int32_t b, int32_t c);

#ifdef __cplusplus
}
#endif
#endif /* TK_H */
