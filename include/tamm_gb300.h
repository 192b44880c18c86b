/*
 * tamm_gb300.h -- C ABI of a single-GPU (GB300, sm_103a) library for
 * contractions of tiled, spin/irrep block-sparse tensors, following TAMM
 * (Tensor Algebra for Many-body Methods, arXiv:2201.01257).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Plain C types only.  "device" pointers are CUDA device addresses of the
 *    context's device; "host" pointers are ordinary host memory.
 *  - Every call returns a tamm_status.  No C++ exception crosses this ABI.  On
 *    failure the context keeps a message for tamm_last_error().
 *  - Asynchrony: every operation is enqueued on the context's CUDA stream and
 *    returns at once, except the calls that hand a host result back
 *    (tamm_energy, tamm_norm, tamm_sync), which synchronise the stream first.
 *  - Device-side failures (a bounded wait that ran out) are recorded in a
 *    device status word and reported by the next synchronising call as
 *    TAMM_ETIMEOUT.  Kernels never trap: a kernel whose wait ran out stops its
 *    own work, lets its copies in flight land, frees its tensor memory and
 *    returns, so the context stays usable.
 *  - Tensors store only their nonzero blocks (sparsity-aware allocation,
 *    Sec. III.B): blocks in lexicographic tile order (mode 0 slowest), each
 *    block row-major over the modes in declared order, packed one after
 *    another in a single FP64 buffer.
 *  - Labels are single characters, one per mode.  A label found in A and B but
 *    not in C is summed (Einstein convention, Sec. IV.A); every label of C
 *    must occur in exactly one of A, B; a label must name the same tamm_space
 *    object everywhere it occurs.
 *  - There is no CPU execution path.  A precision the device cannot run returns
 *    TAMM_EUNSUPPORTED; nothing is silently downgraded.
 */
#ifndef TAMM_GB300_H
#define TAMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TAMM_API __attribute__((visibility("default")))
#else
#define TAMM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef int tamm_status;
#define TAMM_OK 0
#define TAMM_EINVAL 1       /* bad argument: labels, spaces, sizes, null pointers */
#define TAMM_ENOMEM 2       /* the allocator returned NULL */
#define TAMM_ECUDA 3        /* a CUDA runtime/driver call failed */
#define TAMM_EUNSUPPORTED 4 /* valid request this build/device cannot run */
#define TAMM_ETIMEOUT 5     /* a bounded device-side wait ran out */
#define TAMM_ECHECK 6       /* reserved: no call of this build returns it */
#define TAMM_ELIMIT 7       /* a size exceeds a fixed limit of the call */

/* Block-sparsity rule of a tensor (Sec. III.A: spin attributes on tiles and a
 * user-definable non-zero check). */
#define TAMM_SYM_DENSE 0      /* every block stored */
#define TAMM_SYM_SPIN 1       /* sum of spins of the upper modes == that of the lower modes */
#define TAMM_SYM_SPIN_IRREP 2 /* spin rule and XOR of tile irreps == 0 (D2h, totally symmetric) */

/* Arithmetic of a contraction's block products. */
#define TAMM_PREC_F64 0        /* FP64 throughout */
#define TAMM_PREC_OZAKI_BF16 1 /* FP64 operands split into BF16 integer slices, tensor-core products with
                                  exact FP32 accumulation per chunk, FP64 reconstruction */
#define TAMM_PREC_OZAKI_I8 2   /* INT8 slices: sm_103a has no tcgen05 kind::i8, always TAMM_EUNSUPPORTED */
#define TAMM_PREC_BF16X3 3     /* each FP64 element rounded to FP32 and split into three BF16 pieces
                                  (floating, ~24 bits of the element); the six products k+l <= 4 with
                                  FP32 tensor-core accumulation (error ~1e-7) */

typedef struct tamm_ctx tamm_ctx;
typedef struct tamm_space tamm_space;
typedef struct tamm_tensor tamm_tensor;
typedef struct tamm_graph tamm_graph;

/* Stream-ordered device allocator: return `bytes` of device memory usable by
 * work enqueued on `stream` after this call, or NULL.  `release` may be
 * called with memory still in use by work already enqueued on `stream`; the
 * allocator must not hand it out to other streams before that work ends
 * (cudaFreeAsync and PyTorch's caching allocator both behave this way). */
typedef void* (*tamm_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*tamm_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* ---------------------------------------------------------------- context */

/* Execution context (Sec. III.A/III.B "execution context": where and how
 * operations run).  `device` is a CUDA ordinal; `stream` a cudaStream_t (NULL
 * = the legacy default stream).  `alloc`/`release` may both be NULL, in which
 * case cudaMallocAsync/cudaFreeAsync on the stream are used for scratch.  The
 * context owns its scratch and plan caches; the caller owns the stream.
 * `device` = -1 makes a host-only context: spaces, tensors' block tables and
 * tamm_contract_flops work, every call that needs the device returns
 * TAMM_ECUDA.  Errors: TAMM_EINVAL (null out), TAMM_ECUDA (bad device). */
TAMM_API tamm_status tamm_ctx_create(int device, void* stream, tamm_alloc_fn alloc, tamm_free_fn release, void* user,
                            tamm_ctx** out);
/* Change the stream later calls enqueue on (scratch stays stream-ordered by
 * synchronising the old stream first). */
TAMM_API tamm_status tamm_ctx_set_stream(tamm_ctx* ctx, void* stream);
/* Waits for the stream, frees scratch and plans.  NULL is ignored. */
TAMM_API void tamm_ctx_destroy(tamm_ctx* ctx);
/* Message of the last failed call on this context ("" if none); owned by ctx. */
TAMM_API const char* tamm_last_error(const tamm_ctx* ctx);
/* Tuning options of a context. */
#define TAMM_OPT_OZAKI_CHUNK_K 0 /* split precision: summed indices per exact FP32 accumulation chunk,
                                    a multiple of 16 in 16..1280 (default 640); shorter chunks read the
                                    accumulators more often and shrink the rounding of the tail group */
#define TAMM_OPT_OZAKI_PERSISTENT 1 /* split precision: 1 = one CTA per SM walks the work items, 0 = one CTA
                                       per work item (default) */
#define TAMM_OPT_OZAKI_TILE_POLICY 2 /* split precision: output columns per work item (= rows per sliced B
                                        tile) for an output block of N columns.  0 = 128; 1 (default) = 128,
                                        or N rounded up to 16 when N < 128; 2 = the fewest tiles of at most
                                        128 columns, of equal width rounded up to 16 (N = 400 -> 4 x 112);
                                        3 = as 2 with at most 64 columns (N = 400 -> 7 x 64).  Tiles of at
                                        most 64 (32) columns keep two (four) accumulators in flight */
#define TAMM_OPT_OZAKI_PANELS 3 /* split precision: 1 (default) = output blocks that have the same rows and
                                   the same A block in every summed-tile pair run as one column panel
                                   (their B blocks stacked into one image: wider N, A tiles read once);
                                   0 = every output block alone */
#define TAMM_OPT_OZAKI_SPLIT_K 4 /* split precision: 1 (default) = when a contraction has fewer than two
                                    128 x 128 output tiles per SM, cut every output block's summed tile
                                    pairs into up to 8 consecutive ranges, computed in parallel into a
                                    workspace and added in range order (deterministic; a different
                                    rounding from the unsplit sum); 0 = never split */
#define TAMM_OPT_OZAKI_SHARED_SCALE 7 /* split precision: 0 (default) = each block's rows and columns are
                                         scaled by their own maxima; 1 = every output row (column) takes one
                                         exponent, the maximum over all operand blocks that feed it, so that
                                         all block pairs of an output tile share their scaling and the exact
                                         accumulation chunks run across block pairs (fewer accumulator
                                         drains when each pair's summed range is short; a pre-pass of row
                                         maxima and some precision for blocks far below their row's maximum) */
#define TAMM_OPT_OZAKI_FUSED_A 8 /* split precision: 1 = a contraction whose block pairs each sum at most
                                    48 indices and whose output blocks have at most 64 columns (a singles
                                    amplitude against a 4-index block) runs through the GEMM that slices
                                    its A operand from FP64 in its own pipeline and writes C through C's
                                    strides (A read once, no A image, no output permutation); its rows and
                                    columns keep their per-block scaling; 0 (default) = the pre-sliced path.
                                    The autotuner times both where the first applies */
#define TAMM_OPT_WAIT_CYCLES 5 /* split precision: SM clock cycles a kernel waits for one dependency (an
                                  operand copy, an MMA batch, a drained accumulator) before it records
                                  TAMM_ETIMEOUT and stops; >= 1000, default 4,000,000,000 (about 2 s).
                                  The wait for copies already in flight to land before a kernel exits
                                  keeps the default */
#define TAMM_OPT_TEST_WITHHOLD_COPY 6 /* failure-path test hook: 1 = in the next split-precision GEMM
                                         launch, CTA 0 does not issue its first operand copy (nor arrive
                                         on that stage), so the MMA issuer's wait for it runs out and the
                                         launch records TAMM_ETIMEOUT; reset to 0 by that launch */
/* Set option `option` to `value`.  Errors: TAMM_EINVAL (unknown option or value out of range). */
TAMM_API tamm_status tamm_ctx_set_option(tamm_ctx* ctx, int option, int64_t value);

/* Kernel classes for launch counting and timing. */
#define TAMM_KERNEL_ADD 0       /* permuted add / operand and output permutation */
#define TAMM_KERNEL_REDUCE 1    /* energy and norm partial sums and final reduction */
#define TAMM_KERNEL_GEMM_F64 2  /* FP64 block GEMM */
#define TAMM_KERNEL_SLICE 3     /* split-precision operand slicing */
#define TAMM_KERNEL_GEMM_OZ 4   /* split-precision tcgen05 block GEMM */
#define TAMM_KERNEL_SPLIT_REDUCE 5 /* split precision: sum of split summed ranges into C */
#define TAMM_KERNEL_TRIPLES 6   /* (T) correction: fused W, Y, denominators and reduction to a scalar */
#define TAMM_KERNEL_CLASSES 7
/* Number of kernels this context has launched since creation. */
TAMM_API tamm_status tamm_ctx_launch_count(const tamm_ctx* ctx, int64_t* launches);
/* enable != 0: bracket every later kernel launch with CUDA events on the
 * context's stream.  enable == 0 stops recording.  Recorded times are kept until
 * read. */
TAMM_API tamm_status tamm_ctx_profile(tamm_ctx* ctx, int enable);
/* Synchronise, then return and clear, per kernel class (TAMM_KERNEL_*), the
 * summed device time in milliseconds and the number of timed launches.
 * `ms` and `launches` hold TAMM_KERNEL_CLASSES entries (either may be NULL). */
TAMM_API tamm_status tamm_ctx_profile_read(tamm_ctx* ctx, double* ms, int64_t* launches);
/* Synchronise the stream and report any device-side status (TAMM_ETIMEOUT)
 * recorded since the last synchronising call, then clear it. */
TAMM_API tamm_status tamm_sync(tamm_ctx* ctx);

/* ----------------------------------------------------------- index spaces */

/* Tiled index space (Sec. III.A, Fig. "tensor_const": IndexSpace with named
 * sub-ranges, TiledIndexSpace with fixed or explicit tile sizes; spin sub-spaces
 * as in Sec. IV.A eq. "tamm_cc-Spin").  The space is `n_groups` contiguous
 * groups of orbitals; group g has `group_size[g]` orbitals, spin
 * `group_spin[g]` (+1 alpha, -1 beta, 0 spinless: an auxiliary index such as
 * the Cholesky vectors' of Eq. cc12) and irrep `group_irrep[g]` in 0..7 (NULL
 * = all 0).  Tiling: if `fixed_tile` > 0 each group is cut into tiles of that
 * size, the last tile of a group taking the remainder; otherwise the
 * `n_tiles` sizes in `tile_sizes` are laid over the groups in order and must
 * cover each group exactly (a tile never straddles a group).
 * Errors: TAMM_EINVAL on any inconsistency. */
TAMM_API tamm_status tamm_space_create(tamm_ctx* ctx, int n_groups, const int64_t* group_size, const int* group_spin,
                              const int* group_irrep, int n_tiles, const int64_t* tile_sizes, int64_t fixed_tile,
                              tamm_space** out);
/* Number of tiles and of orbitals. */
TAMM_API tamm_status tamm_space_info(const tamm_space* s, int* n_tiles, int64_t* n);
/* Copy per-tile offset, size, spin and irrep into host arrays of n_tiles entries (any may be NULL). */
TAMM_API tamm_status tamm_space_tiles(const tamm_space* s, int64_t* offset, int64_t* size, int* spin, int* irrep);
/* Spaces must outlive every tensor built on them.  NULL is ignored. */
TAMM_API void tamm_space_destroy(tamm_space* s);

/* ---------------------------------------------------------------- tensors */

/* Block-sparse FP64 tensor (Sec. III.A "Tensor<T>{tIS...}"; Sec. III.B
 * sparsity-aware allocation).  `n_modes` (1..8) spaces; the first `n_upper`
 * modes are "upper" for the spin rule; `symmetry` is a TAMM_SYM_* rule.  Only
 * metadata is built here; device storage is attached by tamm_tensor_bind or
 * tamm_tensor_allocate.  Errors: TAMM_EINVAL. */
TAMM_API tamm_status tamm_tensor_create(tamm_ctx* ctx, int n_modes, tamm_space* const* modes, int n_upper, int symmetry,
                               tamm_tensor** out);
/* Tensor over the same spaces as `like` with its modes reordered: mode m of the
 * new tensor is mode perm[m] of `like` (perm a permutation of 0..n_modes-1),
 * and it stores exactly the images of like's stored blocks.  This is the layout
 * of a transposed copy (Sec. III.A tensor transpose), e.g. a product kept in
 * GEMM order.  Errors: TAMM_EINVAL. */
TAMM_API tamm_status tamm_tensor_create_permuted(tamm_ctx* ctx, const tamm_tensor* like, const int* perm,
                                                 tamm_tensor** out);
/* Number of stored blocks and of stored FP64 elements. */
TAMM_API tamm_status tamm_tensor_info(const tamm_tensor* t, int64_t* n_blocks, int64_t* n_elems);
/* Host copies of the block table: `block_tiles` (n_blocks * n_modes tile
 * indices) and `block_offsets` (n_blocks element offsets); either may be NULL. */
TAMM_API tamm_status tamm_tensor_blocks(const tamm_tensor* t, int64_t* block_tiles, int64_t* block_offsets);
/* Attach caller-owned device memory of n_elems doubles (8-byte aligned; 256-byte
 * alignment recommended).  The caller keeps ownership and must keep it alive
 * while work using the tensor is in flight. */
TAMM_API tamm_status tamm_tensor_bind(tamm_tensor* t, double* device_data);
/* Allocate n_elems doubles through the context allocator (freed by destroy). */
TAMM_API tamm_status tamm_tensor_allocate(tamm_tensor* t);
/* Copy the tensor's n_elems doubles from / to host memory, enqueued on the
 * context's stream (asynchronous when the host buffer is page-locked, e.g.
 * cudaMallocHost; pageable buffers make the copy synchronous).  The host buffer
 * uses the same packed block layout as the device data.  Errors: TAMM_EINVAL,
 * TAMM_ECUDA. */
TAMM_API tamm_status tamm_tensor_copy_from_host(tamm_ctx* ctx, tamm_tensor* t, const double* host);
TAMM_API tamm_status tamm_tensor_copy_to_host(tamm_ctx* ctx, const tamm_tensor* t, double* host);
/* Device pointer of the tensor's packed data (NULL if unbound). */
TAMM_API double* tamm_tensor_data(const tamm_tensor* t);
/* NULL is ignored.  Storage obtained by tamm_tensor_allocate is released
 * stream-ordered on the context's stream. */
TAMM_API void tamm_tensor_destroy(tamm_tensor* t);

/* Cholesky lambda tensor (Sec. III.A "lambda tensor": blocks computed on
 * demand, never stored; Sec. IV.A Eq. cc12 Cholesky decomposition of the
 * two-electron tensor):
 *     V[p,q,r,s] = sum_L X[p,r,L] X[q,s,L] - X[p,s,L] X[q,r,L]
 * `X` is a stored 3-mode tensor of Cholesky vectors with modes (P, R, aux);
 * V has modes (P, P, R, R) with two upper modes and X's symmetry kind, and
 * stores a block exactly when some aux tile links the X blocks of one of the
 * two products.  V is read-only and only feeds tamm_contract (as A or B):
 * the contraction forms V in slabs of consecutive first-mode tiles (one
 * X-by-X product into an internal buffer in the contraction's precision, then
 * the FP64 difference of its two permuted images into a slab buffer) and runs
 * the contraction on each slab, the first with the caller's beta and the rest
 * with beta = 1.
 * `slab_bytes` bounds the two slab buffers together (0 = 8 GiB; a tile that
 * alone needs more gets a slab of its own); they are allocated here through
 * the context allocator and freed by tamm_tensor_destroy.  X must stay alive
 * and bound while V is used.  tamm_tensor_info/blocks describe V's block
 * table as if it were stored; bind, allocate, copies, tamm_add, tamm_energy,
 * tamm_norm, tamm_autotune and contraction groups refuse V
 * (TAMM_EUNSUPPORTED), and V can never be an output.
 * Errors: TAMM_EINVAL (X not a stored 3-mode tensor), TAMM_ENOMEM. */
TAMM_API tamm_status tamm_tensor_create_cholesky(tamm_ctx* ctx, const tamm_tensor* X, int64_t slab_bytes,
                                                 tamm_tensor** out);
/* Slab count, FP64-equivalent flops that forming all of V once costs (the
 * X-by-X products; 2*M*N*K per block pair), and the bytes of the two slab
 * buffers (any pointer may be NULL).  Errors: TAMM_EINVAL (not a lambda tensor). */
TAMM_API tamm_status tamm_cholesky_info(const tamm_tensor* V, int* n_slabs, double* form_flops,
                                        int64_t* buffer_bytes);
/* Form all of V into `out`, a stored tensor with V's spaces and block table
 * (e.g. from tamm_tensor_create on V's spaces with n_upper 2 and X's
 * symmetry), slab by slab in `precision` / `slices` as tamm_contract takes them.
 * Errors: TAMM_EINVAL (block tables differ), as tamm_contract otherwise. */
TAMM_API tamm_status tamm_cholesky_form(tamm_ctx* ctx, const tamm_tensor* V, tamm_tensor* out, int precision,
                                        int slices);

/* ------------------------------------------------------------- operations */

/* MultOp (Sec. III.A, grammar figure "tensor_ops", the rule alpha * A * B):
 *     C(lc) = beta * C(lc) + alpha * sum_{summed labels} A(la) * B(lb)
 * over the stored blocks of C.  beta must be 0 ("=") or 1 ("+="); "-=" is a
 * negative alpha.  Each nonzero block pair becomes an operand index
 * permutation where the block layout needs it, a dense block GEMM and an
 * accumulation into the output block.  `precision` is a TAMM_PREC_*; for
 * TAMM_PREC_OZAKI_BF16, `slices` is the number of BF16 slices per operand
 * (3..8; 0 = the autotuned choice for these tensors and labels if
 * tamm_autotune ran on them, else 6 with the context's chunk length).  C must not alias A or B.
 * Errors: TAMM_EINVAL (labels/spaces/beta), TAMM_EUNSUPPORTED (precision),
 * TAMM_ENOMEM, TAMM_ECUDA. */
TAMM_API tamm_status tamm_contract(tamm_ctx* ctx, double alpha, tamm_tensor* C, const char* lc, double beta,
                          const tamm_tensor* A, const char* la, const tamm_tensor* B, const char* lb, int precision,
                          int slices);

/* Nonzero-block flop count 2*M*N*K summed over the block pairs of the same
 * contraction (host only, no device work). */
TAMM_API tamm_status tamm_contract_flops(tamm_ctx* ctx, const tamm_tensor* C, const char* lc, const tamm_tensor* A,
                                const char* la, const tamm_tensor* B, const char* lb, double* flops);

/* AddOp with label permutation (Sec. III.A, grammar rule alpha * A):
 *     C(lc) = beta * C(lc) + sum_t alpha[t] * A(la[t])
 * for `n_terms` (1..4) label orders of the same tensor A (each a permutation of
 * lc), in one pass over C.  With n_terms = 4, lc = "abij" and
 * la = {"abij","baij","abji","baji"}, alpha = {1,-1,-1,1} it applies the
 * antisymmetriser P(ab)P(ij).  beta must be 0 or 1.  C must not alias A.
 * Errors: TAMM_EINVAL. */
TAMM_API tamm_status tamm_add(tamm_ctx* ctx, tamm_tensor* C, const char* lc, double beta, const tamm_tensor* A,
                     int n_terms, const char* const* la, const double* alpha);

/* The same AddOp with every alpha[t] multiplied by the device scalar
 * *scale_device (one double of device memory, 8-byte aligned, read by the
 * kernel when it runs), so that a scale computed on the device, such as the
 * incoming derivative of a scalar in reverse-mode differentiation, needs no
 * host round trip.  Errors: as tamm_add; TAMM_EINVAL for a null or misaligned
 * scale pointer. */
TAMM_API tamm_status tamm_add_scaled(tamm_ctx* ctx, tamm_tensor* C, const char* lc, double beta,
                                     const tamm_tensor* A, int n_terms, const char* const* la, const double* alpha,
                                     const double* scale_device);

/* Adjoint of a MultOp (Sec. III.A, grammar figure "tensor_ops", rule
 * alpha * A * B): for the forward C(lc) = alpha * sum A(la) * B(lb) and an
 * incoming adjoint dC with C's block structure,
 *     dA(la) = beta * dA(la) + alpha * sum dC(lc) * B(lb)
 *     dB(lb) = beta * dB(lb) + alpha * sum A(la) * dC(lc)
 * (either of dA, dB may be NULL).  The adjoint of a MultOp is again a MultOp
 * whose label roles are exchanged: the labels summed in the forward become
 * free labels of the result, and the free labels of the other operand become
 * summed.  Each runs through the same block-sparse path as tamm_contract
 * (`precision`, `slices` as there; stored blocks of dA/dB only).  dA must have
 * A's spaces and block table, dB B's (e.g. tamm_tensor_create_permuted with the
 * identity permutation), so that gradients share their operands' packed layout.
 * Derivatives are taken with respect to every stored entry as an independent
 * variable.  Errors: TAMM_EINVAL (the forward's labels or spaces, a block table
 * that differs, aliasing, beta not 0 or 1), as tamm_contract otherwise. */
TAMM_API tamm_status tamm_contract_adjoint(tamm_ctx* ctx, double alpha, const tamm_tensor* dC, const char* lc,
                                           const tamm_tensor* A, const char* la, const tamm_tensor* B,
                                           const char* lb, tamm_tensor* dA, tamm_tensor* dB, double beta,
                                           int precision, int slices);

/* Full contraction to a scalar (Sec. III.A: inner products / reductions):
 *     result = alpha * sum over all entries A(la) * B(lb)
 * with lb a permutation of la.  FP64, deterministic summation order.
 * `result_host` receives the value after the stream is synchronised.
 * Errors: TAMM_EINVAL, TAMM_ECUDA, TAMM_ETIMEOUT (pending device status). */
TAMM_API tamm_status tamm_energy(tamm_ctx* ctx, double alpha, const tamm_tensor* A, const char* la, const tamm_tensor* B,
                        const char* lb, double* result_host);
/* Same, asynchronous: writes the value to `result_device` (one double of device memory). */
TAMM_API tamm_status tamm_energy_async(tamm_ctx* ctx, double alpha, const tamm_tensor* A, const char* la,
                              const tamm_tensor* B, const char* lb, double* result_device);

/* Frobenius norm over the stored entries (Sec. III.A utility routines: norm).
 * FP64, deterministic.  Synchronises. */
TAMM_API tamm_status tamm_norm(tamm_ctx* ctx, const tamm_tensor* t, double* result_host);
TAMM_API tamm_status tamm_norm_async(tamm_ctx* ctx, const tamm_tensor* t, double* result_device);

/* Allocation-free norm.  The paper has no counterpart to this call; it exists
 * for callers that must not allocate device memory while they run: programs
 * whose GPU memory is entirely owned by another allocator or pool, latency-
 * critical loops where a cudaMalloc would synchronise the device, or processes
 * that reserved all device memory up front.  It needs no context.
 *   *result_device = sqrt(sum_{e < n} x_device[e]^2)
 * for n doubles at x_device (device memory, any layout), enqueued on `stream`
 * (a cudaStream_t, NULL = legacy default stream) of the current device; the
 * result is one double of device memory written by the call.  Nothing is
 * allocated: the partial sums live in a fixed 256 KB array inside the library
 * that every device using the library holds until the process exits.  The
 * first call on a device looks that array's device address up and keeps it
 * for the life of the process, so make it before any stream capture; the kept
 * address does not survive a device reset (cudaDeviceReset) or a recreated
 * primary context, after which this call must not be used in that process.
 * All calls on a device share the array, so calls whose kernels overlap on
 * the GPU (e.g. on two streams) race and must be serialised by the caller.
 * Limit: n <= 2^29 (536,870,912 doubles).
 * Errors: TAMM_EINVAL (n < 0, a null pointer, or a pointer that is not 8-byte
 * aligned; refused before any launch), TAMM_ELIMIT (n above the limit),
 * TAMM_ECUDA (no usable current device or a failed launch). */
TAMM_API tamm_status tamm_norm_noalloc(const double* x_device, int64_t n, double* result_device, void* stream);

/* Perturbative triples correction of CCSD(T) (Sec. IV.B, Eqs. cc13-cc14,
 * tensort, tensort2), real amplitudes, fused to a scalar:
 *     E(T) = sum_{i<j<k} sum_{a<b<c} (W + Y) W / D,
 *     D    = e_i + e_j + e_k - e_a - e_b - e_c,
 * with W = <Phi_ijk^abc|V_N T2|Phi> (Eq. tensort: nine contractions over an
 * occupied index m, nine over a virtual index e; its sixth term is taken with
 * a minus sign, which the antisymmetry of W under j <-> k requires) and
 * Y = <Phi_ijk^abc|V_N T1|Phi> (Eq. tensort2).  Tensors, upper indices first:
 *     T2[a,b,i,j] = t^{ij}_{ab}   T1[a,i] = t^i_a   Vooov[i,j,m,a] = v^{ij}_{ma}
 *     Vvovv[e,i,a,b] = v^{ei}_{ab}   Voovv[i,j,a,b] = v^{ij}_{ab}
 * all on one occupied space (T2's modes 2, 3) and one virtual space (modes 0,
 * 1), any block rule, with storage.  eps_occ / eps_virt: the n_o / n_v orbital
 * energies in device memory.
 * Method: for each occupied triple i<j<k one block-sparse accumulation gives
 *     U[x,y,z] = sum over the cyclic rotations (p,q,r) of (i,j,k) of
 *                sum_m T2[x,y,m,r] Vooov[p,q,m,z] + sum_e Vvovv[e,p,y,x] T2[e,z,q,r]
 * (the signs of Eq. tensort absorbed by the antisymmetry of the inputs), so
 * that W[a,b,c] = U[a,b,c] - U[a,c,b] + U[b,c,a].  U is computed by the block
 * GEMMs (`precision` TAMM_PREC_F64 or TAMM_PREC_OZAKI_BF16, `slices` as in
 * tamm_contract; the context's chunk, tile policy and grid options apply) for
 * a batch of triples in a workspace of at most `workspace_bytes` (0 = 1 GiB),
 * and a fused kernel forms W, Y and D for every a<b<c and reduces to the
 * scalar: no six-index tensor is kept beyond one batch.  The inputs are first
 * copied into GEMM order (scratch the size of T2 twice and of Vvovv).
 * `energy_device`: one double of device memory; `triple_energies_device` (may
 * be NULL): each occupied triple's contribution, triples i<j<k in
 * lexicographic order (n_o (n_o - 1)(n_o - 2) / 6 doubles).  Deterministic;
 * asynchronous.  Errors: TAMM_EINVAL (spaces, modes, null pointers, inside a
 * group), TAMM_EUNSUPPORTED (precision, a lambda tensor), TAMM_ENOMEM, TAMM_ECUDA. */
TAMM_API tamm_status tamm_triples_energy(tamm_ctx* ctx, const tamm_tensor* T2, const tamm_tensor* T1,
                                         const tamm_tensor* Vooov, const tamm_tensor* Vvovv, const tamm_tensor* Voovv,
                                         const double* eps_occ, const double* eps_virt, int precision, int slices,
                                         int64_t workspace_bytes, double* energy_device,
                                         double* triple_energies_device);
/* Host-only counts for the same inputs: the number of occupied triples, the
 * FP64-equivalent block-GEMM flops of one evaluation (2 M N K summed over the
 * block pairs of every triple's U) and the number of workspace batches (any
 * pointer may be NULL).  Errors: TAMM_EINVAL. */
TAMM_API tamm_status tamm_triples_info(tamm_ctx* ctx, const tamm_tensor* T2, const tamm_tensor* T1,
                                       const tamm_tensor* Vooov, const tamm_tensor* Vvovv, const tamm_tensor* Voovv,
                                       int64_t workspace_bytes, int64_t* n_triples, double* gemm_flops,
                                       int* n_batches);

/* FP64 throughput of this device, measured: the denominator of the FP64
 * path's roofline (the paper has no counterpart; it gives no kernel rates).
 * kind 0: scalar fused multiply-adds (DFMA), 8 independent chains per thread;
 * kind 1: the warp-wide FP64 tensor-core MMA (mma.sync m8n8k4 f64), 8
 * independent accumulators per warp.  8 CTAs of 256 threads per SM, 4096
 * steps, one untimed launch then one timed with CUDA events on the context's
 * stream; `tflops` receives the flop rate.  Synchronises.
 * Errors: TAMM_EINVAL (kind, null pointer, inside a group or capture), TAMM_ECUDA. */
TAMM_API tamm_status tamm_fp64_peak(tamm_ctx* ctx, int kind, double* tflops);

/* Autotuner of the split-precision path (TAMM_PREC_OZAKI_BF16) for one
 * contraction, the same tensors and labels as tamm_contract.  It runs the FP64
 * contraction once as the reference, then for each exact-chunk length (1280,
 * 800, 640, 320 summed indices) and for each scaling mode (TAMM_OPT_OZAKI_SHARED_SCALE
 * 0 and 1, and, where it applies, TAMM_OPT_OZAKI_FUSED_A = 1 at one chunk length)
 * the smallest slice count (3..8) whose normwise relative error
 * against that reference is at most target_rel_err / 2 on the given operands,
 * times each such candidate under every tile policy
 * (TAMM_OPT_OZAKI_TILE_POLICY) and grid kind (TAMM_OPT_OZAKI_PERSISTENT;
 * CUDA events, mean of three runs after one untimed run) and keeps the
 * fastest.  C's data is not touched: the
 * trial outputs go to two temporary buffers of C's size from the context
 * allocator.  The choice (slices, chunk, tile policy, grid) is remembered in the
 * context and used by every later tamm_contract of the same tensors and
 * labels with precision TAMM_PREC_OZAKI_BF16 and slices = 0.  Outputs (each
 * may be NULL): the slice count, the chunk length, the tile policy, the grid
 * kind (1 = persistent; always 1 in mode 2, whose GEMM walks its items), the
 * scaling mode (0 = per block, 1 = shared, 2 = per block with A sliced inside
 * the GEMM, timed once where the contraction qualifies), the measured error and the
 * mean time in ms of the chosen configuration.  Tune
 * on representative operands: a zero product is refused (TAMM_EINVAL).  Synchronises.  Errors: TAMM_EINVAL, TAMM_ENOMEM,
 * TAMM_ECUDA, TAMM_EUNSUPPORTED (no candidate reaches the target). */
TAMM_API tamm_status tamm_autotune(tamm_ctx* ctx, const tamm_tensor* C, const char* lc, const tamm_tensor* A,
                                   const char* la, const tamm_tensor* B, const char* lb, double target_rel_err,
                                   int* slices, int* chunk_k, int* tile_policy, int* persistent, int* shared_scale,
                                   double* rel_err, double* ms);

/* ------------------------------------------------------ grouped execution */

/* Contraction groups: the independent contractions of one dependency level
 * executed together (Sec. III.A deferred execution; the scheduler runs the
 * operations of a level as one batch with no synchronisation between them).
 * Between tamm_group_begin and tamm_group_end, split-precision tamm_contract
 * calls (TAMM_PREC_OZAKI_BF16 / TAMM_PREC_BF16X3) are validated, planned and
 * recorded but not run; every other operation (FP64 contractions, adds,
 * energies, norms, stream changes) is refused with TAMM_EINVAL.  tamm_group_end
 * checks that no recorded output overlaps another contraction's input or
 * output (TAMM_EINVAL otherwise, and nothing runs), then enqueues, on the
 * context's stream: the operand slicing of every contraction, one persistent
 * grouped tcgen05 GEMM launch over all their block tasks per slice count (at
 * most 64 contractions per launch), and the output permutations.  Results are
 * bitwise those of running the contractions one by one.  The group's scratch
 * (all operand slice images at once) comes from the context's scratch buffer.
 * Errors: TAMM_EINVAL (nesting, refused call, aliasing), TAMM_ENOMEM,
 * TAMM_ECUDA. */
TAMM_API tamm_status tamm_group_begin(tamm_ctx* ctx);
TAMM_API tamm_status tamm_group_end(tamm_ctx* ctx);
/* Close the open group without running what it recorded.  Errors: TAMM_EINVAL (no open group). */
TAMM_API tamm_status tamm_group_cancel(tamm_ctx* ctx);

/* Scheduler (Sec. III.A: operations are declared and executed through a
 * scheduler; Sec. III.B: its data-flow analysis marks operations that share a
 * tensor one of them updates as conflicting, and a levelized execution runs
 * each batch of independent operations together).  tamm_sched_contract / _add / _energy
 * record an operation with the arguments of tamm_contract / tamm_add /
 * tamm_energy_async (strings are copied; tensors must stay alive until the
 * scheduler is destroyed).  Two operations conflict when one writes storage
 * the other reads or writes (device byte ranges; a tensor without storage
 * counts as itself; a contraction with beta = 1 or an add with beta = 1 reads
 * its output; a contraction reading a Cholesky lambda tensor reads the
 * Cholesky vectors; an energy writes its 8-byte result).  An operation's level
 * is one more than the highest level of an earlier operation it conflicts
 * with, else 0.  tamm_sched_execute enqueues the levels in order; inside a
 * level, first the split-precision contractions that do not read a lambda
 * tensor as one contraction group (tamm_group_begin/end), then the other
 * contractions, the adds and the energies in recorded order.  Results equal
 * running the operations in recorded order (bitwise: groups reproduce single
 * contractions).  It may run inside a graph capture and any number of times.
 * tamm_sched_levels reports the number of operations and levels and, if
 * `op_level` is not NULL, each operation's level (n_ops entries); it needs no
 * device.  Errors: TAMM_EINVAL (arguments, or a group open at execution);
 * at execution, the status of the first operation that fails (its message in
 * tamm_last_error; the operations after it do not run). */
typedef struct tamm_sched tamm_sched;
TAMM_API tamm_status tamm_sched_create(tamm_ctx* ctx, tamm_sched** out);
TAMM_API tamm_status tamm_sched_contract(tamm_sched* s, double alpha, tamm_tensor* C, const char* lc, double beta,
                                         const tamm_tensor* A, const char* la, const tamm_tensor* B, const char* lb,
                                         int precision, int slices);
TAMM_API tamm_status tamm_sched_add(tamm_sched* s, tamm_tensor* C, const char* lc, double beta,
                                    const tamm_tensor* A, int n_terms, const char* const* la, const double* alpha);
TAMM_API tamm_status tamm_sched_energy(tamm_sched* s, double alpha, const tamm_tensor* A, const char* la,
                                       const tamm_tensor* B, const char* lb, double* result_device);
TAMM_API tamm_status tamm_sched_levels(tamm_sched* s, int* n_ops, int* n_levels, int* op_level);
TAMM_API tamm_status tamm_sched_execute(tamm_sched* s);
/* NULL is ignored. */
TAMM_API void tamm_sched_destroy(tamm_sched* s);

/* CUDA-graph capture of a sequence of library calls on the context's stream,
 * replayed with one launch (Sec. III.A: the deferred operation list executed
 * as a unit).  The context must be on a created stream (not the legacy or
 * per-thread default stream) and not profiling.  Calls between begin and end
 * are captured, not run; they may not allocate device memory (plans, scratch
 * and reduction buffers must already exist: run the same calls once before
 * capturing) nor synchronise (tamm_energy, tamm_norm, tamm_sync are refused;
 * use the _async forms).  A refused call makes tamm_graph_end fail.  Groups
 * may be opened and closed inside a capture.  The graph holds the device
 * pointers it was captured with: the tensors and their data must stay alive
 * and bound to the same buffers while it is launched; their contents may
 * change between launches.  tamm_graph_launch enqueues the graph on the
 * context's stream and adds its kernel count to tamm_ctx_launch_count.
 * Errors: TAMM_EINVAL, TAMM_ECUDA. */
TAMM_API tamm_status tamm_graph_begin(tamm_ctx* ctx);
TAMM_API tamm_status tamm_graph_end(tamm_ctx* ctx, tamm_graph** graph);
TAMM_API tamm_status tamm_graph_launch(tamm_graph* graph);
/* Number of library kernels one launch of the graph runs. */
TAMM_API tamm_status tamm_graph_info(const tamm_graph* graph, int64_t* kernel_launches);
/* NULL is ignored.  The graph must not be running (synchronise first).  A
 * graph destroyed while its context has a capture open is freed when that
 * capture ends (freeing it inside the capture would invalidate the capture). */
TAMM_API void tamm_graph_destroy(tamm_graph* graph);

#ifdef __cplusplus
}
#endif

#endif /* TAMM_GB300_H */
