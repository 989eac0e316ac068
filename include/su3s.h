/*
 * su3s -- site-local evaluation of lattice expressions on one GB300 GPU.
 *
 * C ABI.  No C++ or framework types cross this boundary: only plain integers,
 * doubles, host or device pointers, sizes and opaque handles.  A stream
 * argument is a cudaStream_t passed as void* (NULL = the legacy default
 * stream).  Every call returns an int status (SU3S_OK = 0); on failure
 * su3s_last_error() returns a message for the calling thread.  No call aborts
 * the process or throws.
 *
 * The objects follow arXiv:1710.09409:
 *   - a lattice is a 4-d Cartesian grid Lx*Ly*Lz*Lt (Sec. 3, Listing 2:
 *     Lattice<T> v(&grid); Sec. 4, Listing 3);
 *   - a field is a lattice-wide array of site objects: complex 3x3 colour
 *     matrices (Su3f in Sec. 4), complex colour vectors, or reals
 *     (Lattice<double>, Listing 2), optionally with `nmu` objects per site
 *     (Lorentz-indexed link fields, nmu = 4);
 *   - an expression is a tree of products, sums, differences, real scalings
 *     and Hermitian adjoints of fields (the expression-template engine of
 *     Sec. 3, Listing 1), and evaluating it into a destination field computes
 *     _odata[ss] = eval(ss, expr) for every site ss in one pass.
 *
 * Canonical host layout ("canonical AoS"): double[V][nmu][w] with
 * w = 18 (matrix: row, column, re/im), 6 (vector) or 1 (real), site index
 * x + Lx*(y + Ly*(z + Lz*t)).  Device layouts are described at
 * su3s_field_bytes.
 */
#ifndef SU3S_H
#define SU3S_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SU3S_OK 0
#define SU3S_EINVAL 1       /* bad argument: null handle, value out of range      */
#define SU3S_ETYPE 2        /* ill-typed expression (e.g. vector * matrix)        */
#define SU3S_ESHAPE 3       /* fields disagree in lattice, links, layout or size  */
#define SU3S_ENOMEM 4       /* an allocation made by the library failed           */
#define SU3S_ECUDA 5        /* a CUDA call failed; the message names it           */
#define SU3S_EUNSUPPORTED 6 /* well-formed request this library does not handle   */

/* ---- field kinds ---- */
#define SU3S_MATRIX 0 /* complex 3x3 colour matrix */
#define SU3S_VECTOR 1 /* complex colour 3-vector   */
#define SU3S_REAL 2   /* one real per site object   */

/* ---- storage precisions ---- */
#define SU3S_F64 0     /* complex: 2 x FP64                                            */
#define SU3S_F32 1     /* complex: 2 x FP32 (round to nearest even on store)          */
#define SU3S_BF16 2    /* complex: 2 x BF16                                            */
#define SU3S_F16 3     /* complex: 2 x FP16                                            */
#define SU3S_F64_C12 4 /* SU(3) matrix as rows 0,1 only (12 FP64); row 2 rebuilt      */
#define SU3S_F32_C12 5 /* SU(3) matrix as rows 0,1 only (12 FP32); row 2 rebuilt      */

/* ---- device layouts ---- */
#define SU3S_SOA 0   /* component-major: [mu][component][Vpad]                      */
#define SU3S_AOSOA 1 /* site-blocked:    [Vpad/B][mu][component][B], B = block      */

/* ---- arithmetic used for FP64 storage ---- */
#define SU3S_MATH_DEFAULT 0 /* the library default (see su3s_set_default_math)     */
#define SU3S_MATH_F64 1     /* native IEEE FP64 with fused multiply-add              */
#define SU3S_MATH_DF32 2    /* FP64-accurate pair-of-FP32 arithmetic (see below)     */
#define SU3S_MATH_FX 3      /* FP64-accurate shared-exponent fixed point (see below) */

typedef struct su3s_lattice su3s_lattice;
typedef struct su3s_field su3s_field;
typedef struct su3s_expr su3s_expr;
typedef struct su3s_batch su3s_batch;

/* Message of the last failed call on this thread ("" if none).  The pointer
 * stays valid until the next call on the same thread. */
const char* su3s_last_error(void);

/* Library version as 10000*major + 100*minor + patch. */
int su3s_version(void);

/* ------------------------------------------------------------------------
 * Lattice (Sec. 3, Listing 2 / Sec. 4, Listing 3: the grid that fields live on)
 * ---------------------------------------------------------------------- */

/* Create a lattice of lx*ly*lz*lt sites.  Each extent must be >= 1 and the
 * volume must be < 2^31.  *out receives a handle owned by the caller.
 * EINVAL on a bad extent or null out. */
int su3s_lattice_create(int lx, int ly, int lz, int lt, su3s_lattice** out);

/* Destroy a lattice handle.  Fields keep their own copy of the geometry, so a
 * lattice may be destroyed while fields made from it live on.  NULL is a
 * no-op. */
int su3s_lattice_destroy(su3s_lattice* lat);

/* Number of sites of a lattice in *out.  EINVAL on null arguments. */
int su3s_lattice_volume(const su3s_lattice* lat, int64_t* out);

/* ------------------------------------------------------------------------
 * Fields (lattice-wide arrays of site objects)
 * ---------------------------------------------------------------------- */

/* Bytes of device memory a field needs, in *bytes.
 *   kind   SU3S_MATRIX / SU3S_VECTOR / SU3S_REAL
 *   nmu    objects per site, 1..8 (4 for Lorentz-indexed link fields)
 *   prec   SU3S_F64 ... SU3S_F32_C12 (C12 only for matrices; reals only F64)
 *   layout SU3S_SOA or SU3S_AOSOA
 *   block  B for SU3S_AOSOA: a power of two, 4..1024; ignored for SU3S_SOA
 * The volume is padded to Vpad (a multiple of 64 for SOA, of max(B,4) for
 * AOSOA).  With ncomp complex components per object (9 matrix, 6 two-row
 * matrix, 3 vector) the element at (site s, link mu, component c) is at
 *   SOA:   (mu*ncomp + c)*Vpad + s
 *   AOSOA: ((s/B)*nmu + mu)*ncomp*B + c*B + s%B
 * in units of one complex (reals: one real, ncomp = 1). */
int su3s_field_bytes(const su3s_lattice* lat, int kind, int nmu, int prec, int layout, int block,
                     size_t* bytes);

/* Wrap caller-owned device memory as a field.  dev_ptr must be 16-byte
 * aligned and hold at least su3s_field_bytes(...) bytes; the library never
 * frees it, and the memory must outlive the handle and every queued kernel
 * that uses it.  The contents are not touched.  *out receives a handle owned
 * by the caller.  EINVAL on a bad argument or alignment, ESHAPE if bytes is
 * too small, EUNSUPPORTED for a kind/precision pair that has no storage. */
int su3s_field_wrap(const su3s_lattice* lat, int kind, int nmu, int prec, int layout, int block,
                    void* dev_ptr, size_t bytes, su3s_field** out);

/* Destroy a field handle (the wrapped memory is untouched).  NULL is a no-op. */
int su3s_field_destroy(su3s_field* f);

/* Pack (Grid's vector layout, Sec. 5, done once on the device): read the
 * canonical AoS FP64 array at dev_canonical (device memory, V*nmu*w doubles)
 * and write the field in its device layout and precision, rounding to
 * nearest-even for FP32/BF16/FP16 and keeping rows 0,1 for the C12 formats.
 * Pad sites are set to zero.  Asynchronous on `stream`. */
int su3s_field_pack(su3s_field* f, const double* dev_canonical, void* stream);

/* Unpack: write the canonical AoS FP64 array (V*nmu*w doubles, device memory)
 * from the field, widening reduced precisions exactly and rebuilding row 2 of
 * C12 matrices as conj(row0 x row1).  Asynchronous on `stream`. */
int su3s_field_unpack(const su3s_field* f, double* dev_canonical, void* stream);

/* Upload from host memory: copy n_doubles (must equal V*nmu*w) canonical AoS
 * doubles from host_canonical to a device staging buffer and pack it into the
 * field.  The staging buffer is allocated and freed by the library in stream
 * order (cudaMallocAsync / cudaFreeAsync).  Pinned host memory makes the copy
 * asynchronous; the host buffer must not change until the stream reaches
 * this point.  ESHAPE if n_doubles is wrong, ENOMEM if staging fails. */
int su3s_field_upload(su3s_field* f, const double* host_canonical, size_t n_doubles, void* stream);

/* Download to host memory: unpack into a library-owned staging buffer and
 * copy n_doubles canonical AoS doubles to host_canonical.  The data is in
 * place once the stream reaches this point (synchronise before reading). */
int su3s_field_download(const su3s_field* f, double* host_canonical, size_t n_doubles,
                        void* stream);

/* Download without allocating device memory (the paper has no counterpart:
 * this is a service of the library).  Same result as su3s_field_download, but
 * the unpack kernel stages the canonical array in a fixed 16 MiB array in the
 * library's own device memory instead of a buffer allocated for the call.  It
 * is meant for callers that cannot allocate device memory at that point: a
 * framework whose caching allocator already holds the device's memory, or
 * code that must not pay the latency or implicit synchronisation of
 * allocating and freeing.  The call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).
 *   - Limit: V*nmu*w <= 2^21 doubles (16 MiB, e.g. a 16^4 matrix field, an
 *     8^4 Lorentz field); larger fields return ESHAPE with a message pointing
 *     to su3s_field_download.
 *   - The staging array is held by every GPU on which the library is used
 *     until the process exits.  It is placed in device memory when the
 *     library's module that holds it is loaded on a device, which
 *     su3s_field_wrap does for the current device (field creation is allowed
 *     to allocate), so the download finds its address ready.  Only a call on
 *     a device where no field was ever wrapped loads the module itself; make
 *     such a call before any stream capture and before the device's memory is
 *     exhausted.  A device reset while the library is loaded is not
 *     supported (the cached address would go stale).
 *   - Every call shares the array and it keeps the last call's contents; calls
 *     whose work overlaps on the GPU (other streams, other threads) race on it.
 *     Calls ordered on one stream do not.
 * The data is in host_canonical once the stream reaches this point. */
int su3s_field_download_static(const su3s_field* f, double* host_canonical, size_t n_doubles,
                               void* stream);

/* Stored-format transfer (the paper has no counterpart: a service of the
 * library for callers that hold data in a reduced storage format).  The host
 * array is site-major like the canonical one, but each (site, link) object
 * holds only its stored complex components (9 for a matrix, rows 0 and 1 =
 * 6 for a C12 matrix, 3 for a vector; 1 real for a real field), each in the
 * field's storage format: (re, im) pairs of doubles (F64, F64_C12), floats
 * (F32, F32_C12), bfloat16 or binary16 values (BF16, F16); reals are doubles.
 * Element ((s*nmu + mu)*ncomp + c) is component c of link mu at site s.  The
 * bytes are moved as they are: no rounding, no widening, no row rebuilt, so a
 * download after an upload returns the same bytes, and a C12 download gives
 * the two stored rows.  su3s_field_stored_bytes gives the array's size. */
int su3s_field_stored_bytes(const su3s_field* f, size_t* bytes);

/* Upload a stored-format host array of nbytes bytes (must equal
 * su3s_field_stored_bytes) into the field; pad sites are set to zero.  Staging
 * as in su3s_field_upload.  EINVAL on a null argument, ESHAPE on a wrong size,
 * ENOMEM if staging fails. */
int su3s_field_upload_stored(su3s_field* f, const void* host_stored, size_t nbytes, void* stream);

/* Download the field to a stored-format host array of nbytes bytes.  Errors
 * and ordering as su3s_field_upload_stored / su3s_field_download. */
int su3s_field_download_stored(const su3s_field* f, void* host_stored, size_t nbytes, void* stream);

/* ------------------------------------------------------------------------
 * Expressions (Sec. 3, Listing 1: the expression-template tree)
 * ---------------------------------------------------------------------- */

/* Nodes are immutable and reference-counted: a node holds references to its
 * children, so the caller may free children after building a parent.  The
 * caller frees every handle it receives with su3s_expr_free.  A leaf refers to
 * its field handle without owning it: the field handle (and its memory) must
 * outlive every expression and batch that uses it.  Type rules:
 * matrix*matrix -> matrix, matrix*vector -> vector, real*real -> real;
 * add/sub need equal kinds; adj only on matrices; scale keeps the kind.
 * ETYPE on a violation, EINVAL on null arguments.  Trees are evaluated as
 * written (a*b*c built as mul(mul(a,b),c) is (a*b)*c, as C++ operators
 * associate in Listing 2). */
int su3s_expr_leaf(su3s_field* f, su3s_expr** out);
int su3s_expr_mul(const su3s_expr* x, const su3s_expr* y, su3s_expr** out);
int su3s_expr_add(const su3s_expr* x, const su3s_expr* y, su3s_expr** out);
int su3s_expr_sub(const su3s_expr* x, const su3s_expr* y, su3s_expr** out);
int su3s_expr_scale(double s, const su3s_expr* x, su3s_expr** out);
int su3s_expr_adj(const su3s_expr* x, su3s_expr** out);
int su3s_expr_free(su3s_expr* e);

/* Canonical signature of a tree (leaves numbered by first appearance, e.g.
 * "add(mul(M0,M1),mul(M2,M3))") copied into buf (NUL-terminated, truncated
 * to cap bytes).  Used to see which kernel a tree maps to. */
int su3s_expr_signature(const su3s_expr* e, char* buf, size_t cap);

/* ------------------------------------------------------------------------
 * Evaluation: dest = expr at every site, in one read/write sweep
 * (Sec. 3, Listing 1: for(ss) _odata[ss] = eval(ss, expr);
 *  Sec. 4, Listing 3: z = x*y)
 * ---------------------------------------------------------------------- */

/* Evaluate `e` into `dest` on `stream` with the default arithmetic.  Every
 * leaf and dest must share lattice geometry, nmu, layout (and block) and
 * precision; dest's kind must equal the tree's kind.  dest may be one of the
 * leaves: every site object is read in full before it is written.  Trees in
 * the compiled catalogue run a specialised fused kernel; others run a
 * uniform per-site interpreter kernel (still one pass).  Reduced precisions
 * (FP32/BF16/FP16, FP32 accumulation) and the C12 formats support the
 * catalogue trees listed by su3s_catalogue; others return EUNSUPPORTED.
 * C12 destinations accept only products of special unitary matrices. */
int su3s_eval(su3s_field* dest, const su3s_expr* e, void* stream);

/* As su3s_eval with an explicit arithmetic for FP64 storage:
 *   SU3S_MATH_F64   IEEE FP64 with FMA (the GB300's FP64 pipe is narrow, so
 *                   this path is bound by FP64 throughput, not memory);
 *   SU3S_MATH_DF32  each FP64 input is split exactly-enough into a pair of
 *                   FP32 values (integer bit operations, no FP64 instruction),
 *                   products and sums use error-free transformations in FP32,
 *                   and results are re-assembled into FP64 bit patterns.
 *                   Error per output <= ~2^-46 * sum_t |x_t y_t| (+ 2^-52 |z|),
 *                   plus an absolute error below 2^-126 times the other
 *                   factors' magnitudes for inputs below 2^-126 (flushed).
 *   SU3S_MATH_FX    the reals of each site object (matrix, vector, real)
 *                   share the exponent of the object's largest element and
 *                   become 53-bit signed integers; products are exact 32-bit
 *                   integer multiply-adds into 64-bit accumulators (the
 *                   lowest partial product is dropped), sums of terms with
 *                   different scales are aligned by shifts, and each result
 *                   is converted to FP64 once.  Error per output
 *                   <= ~2^-47 * 6 * max|x| * max|y| over the two operand
 *                   objects; objects whose largest magnitude is below 2^-958
 *                   are flushed to zero; results must stay below 2^960 in
 *                   magnitude, and results below 2^-1022 are returned with an
 *                   absolute error below 2^-1022.
 * Range guard of SU3S_MATH_DF32 and SU3S_MATH_FX (every kernel that evaluates
 * in them, forward, reverse mode, batch, interpreter and neighbour terms):
 * each site's FP64 inputs (leaves, dL/dZ and the real factors of the tree)
 * are checked as they are read.  A site with an input that is NaN, +-Inf or
 * at least 2^t(d) in magnitude, t(d) = floor((120 - 3 (d - 1)) / d) for a
 * tree whose terms have at most d factors (d = 2: 2^58, d = 3: 2^38), is
 * evaluated again in native FP64 (SU3S_MATH_F64) in the same kernel before
 * anything of it is stored.  Such sites therefore get IEEE results (NaN and
 * Inf propagate, large values do not overflow early); sites in range keep
 * the arithmetic's own results.  Nothing is reported: no status, no error
 * word.  The bound keeps every intermediate of a site in range below 2^127.
 * Ignored for reduced-precision storage.  EINVAL for another value. */
int su3s_eval_math(su3s_field* dest, const su3s_expr* e, int math, void* stream);

/* Set the arithmetic SU3S_MATH_DEFAULT stands for (process-wide; initially
 * SU3S_MATH_DF32): SU3S_MATH_F64, SU3S_MATH_DF32 or SU3S_MATH_FX; EINVAL for
 * other values. */
int su3s_set_default_math(int math);

/* The compiled kernels, one per line, into buf (truncated to cap bytes,
 * NUL-terminated): "eval <signature> <storage> <arithmetic>" for the forward
 * catalogue and "adjoint <signature> f64 <arithmetic>" for the reverse mode,
 * storage one of f64 f32 bf16 f16 f64_c12 f32_c12 and arithmetic one of f64
 * df32 fx (FP64 storage) or f32 (reduced storage).  EINVAL on a null buffer. */
int su3s_catalogue(char* buf, size_t cap);

/* Fix the launch geometry used for `e` into `dest` (threads per block
 * 32..256, multiple of 32; blocks_per_sm 0..64: 0 = one thread per
 * site-vector, else a grid-stride grid of blocks_per_sm * SMs blocks) with the
 * data movement set by su3s_set_pipeline at this call.  Results do not depend
 * on the geometry.  Applies to later su3s_eval calls with the same kernel and
 * volume.  EINVAL for values out of range. */
int su3s_set_launch(const su3s_field* dest, const su3s_expr* e, int math, int threads,
                    int blocks_per_sm);

/* Choose how FP64-storage kernels move data (process-wide; results do not
 * depend on it):
 *   -1  the library's choice per kernel (default);
 *    0  plain 16-byte vector loads;
 *    1  TMA-staged tiles: each warp stages its next 32-site tile of every leaf
 *       into shared memory while it computes the current one, one 2-D tensor
 *       copy per matrix or vector object (the field's tensor map, made when
 *       the field is wrapped);
 *    2  TMA-staged per leaf: each leaf has its own buffer and barrier, is read
 *       when first needed and refilled after its last use;
 *    3  TMA-staged through a ring of three buffers per warp, for trees that
 *       read every object once per tile (others use their default): reading
 *       the object at position j of the tile's read order hands its buffer to
 *       position j + 3, of this tile or of the warp's next one;
 *    4  TMA-staged two tiles at a time, two sites per lane: each warp stages
 *       two 32-site tiles and every FP32 operation of SU3S_MATH_DF32 is one
 *       packed instruction over the same real of two sites; for products of
 *       two distinct matrix leaves (either may be an adjoint), sums and
 *       differences of two such products over four distinct leaves, and the
 *       reverse mode of such a product (others use their default).
 * All modes give bitwise identical results.  Staging needs 32 sites of a
 * component to be contiguous (SOA, or AOSOA with block >= 32); otherwise plain
 * loads are used.  EINVAL for other values. */
int su3s_set_pipeline(int mode);

/* Read and clear the library's device error word (a stream-ordered copy
 * followed by a synchronisation of `stream`): 0 if every bounded wait inside
 * the library's kernels completed since the last call, 1 if a TMA pipeline
 * wait gave up, 2 if a staged kernel found its shared memory misaligned for
 * tensor copies and staged nothing (results are incomplete in both cases). */
int su3s_device_error(int* code, void* stream);

/* Diagnostic of the bounded waits (the paper has no counterpart): one warp
 * waits, with the pipelines' bounded-wait routine cut to `polls` polls
 * (1..2^20, EINVAL otherwise), on a staging barrier that nothing completes.
 * The wait gives up, the kernel records code 1 in the device error word (read
 * it with su3s_device_error) and returns; *cycles receives the SM clock
 * cycles the wait took (-1 if it did not give up).  Nothing faults and the
 * context stays usable.  Synchronises `stream`.  The pipelines themselves give
 * up after 2^18 polls: a poll that finds the phase incomplete suspends the
 * thread for ~7,800 cycles on GB300, so about one second. */
int su3s_selftest_bounded_wait(uint32_t polls, int64_t* cycles, void* stream);

/* Autotune the launch geometry for `e` into `dest`: times each candidate
 * (data movement 0..4 as for su3s_set_pipeline, threads 64..256, full or
 * grid-stride grids) with CUDA events on `stream` (synchronising it; dest is
 * overwritten, so a dest that is one of the leaves changes that leaf), keeps
 * the fastest for later su3s_eval calls and reports it in
 * *threads, *blocks_per_sm, *variant and its time in *best_ms (any may be
 * NULL).  Not to be called while `stream` is being captured. */
int su3s_tune(su3s_field* dest, const su3s_expr* e, int math, void* stream, int* threads,
              int* blocks_per_sm, int* variant, float* best_ms);

/* ------------------------------------------------------------------------
 * Batching: many (dest, expr) pairs of uneven volumes in one persistent
 * launch, captured in a CUDA graph.  Each item is the one-pass evaluation of
 * Sec. 3, Listing 1 (_odata[ss] = eval(ss, expr)) on its own lattice; the
 * paper evaluates one lattice per launch and has no batching, which is a
 * service of this library.
 * ---------------------------------------------------------------------- */

int su3s_batch_create(su3s_batch** out);
/* Queue dest = e.  The batch keeps references to the expression; fields must
 * outlive the batch.  Items must use FP64 storage.  Items run concurrently and
 * in no defined order: an item's dest may be one of its own leaves, but must
 * not overlap another item's dest or leaves (su3s_batch_build returns EINVAL). */
int su3s_batch_add(su3s_batch* b, su3s_field* dest, const su3s_expr* e);
/* Freeze the batch: build the tile list (tile_sites sites per tile; 0 = 2 x
 * threads) and item table in library-owned device memory, choose the
 * persistent grids (threads per block, a multiple of 32 up to 256; 0 = 256)
 * and capture the launches into a CUDA graph on `stream`: one persistent
 * kernel per tree present in the batch, compiled for that tree.  Items whose
 * tree no persistent kernel covers are captured as separate launches in the
 * same graph.  math as for su3s_eval_math. */
int su3s_batch_build(su3s_batch* b, int math, int threads, int tile_sites, void* stream);
/* Autotune and build: for every candidate launch shape (threads per block 64,
 * 128, 256; persistent grids of at most 1, 2, 4 blocks per SM or as many as
 * fit; tiles of 1, 2, 4 blocks' sites for the plain-load kernels) build the
 * batch, time its graph with CUDA events on `stream` (synchronising it; the
 * destinations are overwritten, so an item whose dest is one of its leaves
 * changes that leaf), then leave the batch built with the fastest.  The
 * batch may already be built (it is rebuilt).  The choice is reported in
 * *threads, *tile_sites, *blocks_per_sm (0 = as many as fit) and its time per
 * launch in *best_ms (any may be NULL).  Results do not depend on the launch
 * shape.  EINVAL for a null batch, a bad arithmetic or items that overlap;
 * not to be called while `stream` is being captured. */
int su3s_batch_tune(su3s_batch* b, int math, void* stream, int* threads, int* tile_sites,
                    int* blocks_per_sm, float* best_ms);
/* Replay the graph on `stream`. */
int su3s_batch_launch(su3s_batch* b, void* stream);
/* Sites in the batch (sum of padded volumes times links) in *sites and the
 * number of tiles in *tiles (either may be NULL). */
int su3s_batch_info(const su3s_batch* b, int64_t* sites, int64_t* tiles);
int su3s_batch_destroy(su3s_batch* b);

/* ------------------------------------------------------------------------
 * Differentiation: the reverse mode of the evaluation of Sec. 3, Listing 1
 * (the paper has no counterpart; for z = x*y of Sec. 4, Listing 3 it gives
 * dX = dZ Y^dagger, dY = X^dagger dZ)
 * ---------------------------------------------------------------------- */

/* Reverse mode through `e` for a real loss L whose gradient with respect to
 * the tree's value is the field `grad_out` (same shape as the tree's value;
 * gradient convention dL/dRe + i dL/dIm).  Writes dL/d(leaf) for the unique
 * leaves of `e` in order of first appearance into grad_leaves[k]
 * (overwritten, not accumulated; NULL entries are skipped; a gradient field
 * that overlaps a leaf, grad_out or another gradient returns EINVAL, since
 * leaves are read while gradients are written).  nleaves must
 * equal the number of unique leaves.  For z = a*b this is dA = G B^dagger,
 * dB = A^dagger G; sums, scalings and adjoints follow the chain rule.
 * One pass: every leaf and grad_out is read once, every gradient written
 * once (a sum of two products of distinct leaves may instead run as two
 * single-product passes, see su3s_tune_adjoint).  FP64 storage only;
 * catalogue trees only (EUNSUPPORTED otherwise). */
int su3s_eval_adjoint(const su3s_expr* e, const su3s_field* grad_out, su3s_field* const* grad_leaves,
                      int nleaves, int math, void* stream);

/* Autotune the reverse-mode kernel of `e` as su3s_tune does the forward one:
 * arguments as for su3s_eval_adjoint (grad_leaves are overwritten while
 * timing), result as for su3s_tune; later su3s_eval_adjoint calls on fields
 * of this shape use the fastest geometry.  For a sum or difference of two
 * products of four distinct leaves (a*b + c*d, a*b - c*d, s0 a*b + s1 c*d) it
 * also times the reverse mode split into two single-product launches,
 * (a, b, grad_out -> dA, dB) then (c, d, grad_out -> dC, dD), which read
 * grad_out twice but hold the operands of one product at a time, and keeps
 * the faster form for later calls (a split choice is reported as
 * *variant = 10 + the halves' data-movement variant).  Untuned calls of such
 * trees run split. */
int su3s_tune_adjoint(const su3s_expr* e, const su3s_field* grad_out, su3s_field* const* grad_leaves,
                      int nleaves, int math, void* stream, int* threads, int* blocks_per_sm,
                      int* variant, float* best_ms);

/* How su3s_eval_adjoint runs the reverse mode of a sum or difference of two
 * products of distinct leaves (process-wide; results agree within the
 * arithmetic's error either way): -1 the tuned choice, split when untuned
 * (default); 0 always one fused pass; 1 always two single-product passes.
 * EINVAL for other values. */
int su3s_set_adjoint_split(int mode);

/* Number of unique leaves of `e` in *n. */
int su3s_expr_num_leaves(const su3s_expr* e, int* n);

/* ------------------------------------------------------------------------
 * Reductions and projections (no counterpart in the paper: the loss of the
 * reverse mode, and the FP64 projection to SU(3) of fields kept in reduced
 * precision)
 * ---------------------------------------------------------------------- */

/* *dev_out (device memory, one double) = sum over sites, links and
 * components of x*y over all reals = sum_x Re tr(X^dagger Y) for matrix
 * fields.  FP64 storage, same shape.  Deterministic (fixed reduction order);
 * uses library-allocated stream-ordered scratch for block partial sums. */
int su3s_field_redot(const su3s_field* x, const su3s_field* y, double* dev_out, void* stream);

/* dst = projection of src to SU(3) at every site object: Gram-Schmidt over
 * rows (two sweeps) and division by the principal cube root of the
 * determinant's phase, in native FP64 after widening the stored values; the
 * result is rounded to dst's precision on store.  Matrix fields of equal
 * shape and precision (FP64, FP32, BF16 or FP16; two-row storage is special
 * unitary by construction and returns EUNSUPPORTED).  dst may equal src.
 * Pad sites are not touched. */
int su3s_reunitarize(su3s_field* dst, const su3s_field* src, void* stream);

/* ------------------------------------------------------------------------
 * Nearest-neighbour operations (arXiv:1710.09409 Sec. 6, Summary and
 * Outlook: the Dslash operator and the Cshift operations outside the
 * expression templates are the paper's next step).  Sites are
 * s = x + Lx (y + Ly (z + Lz t)); directions 0..3 are x, y, z, t; every
 * direction is periodic.
 * ---------------------------------------------------------------------- */

/* dst(x) = src(x + shift * e_dim) at every site, link and component: a copy
 * of the stored objects in their storage format (any kind and precision,
 * bit exact).  dst and src have the same kind (ETYPE otherwise), the same
 * lattice, links, precision and layout (ESHAPE otherwise), and do not overlap
 * (EINVAL).  dim in 0..3 (EINVAL otherwise); any shift, taken modulo the
 * extent.  Pad sites are not touched. */
int su3s_cshift(su3s_field* dst, const su3s_field* src, int dim, int shift, void* stream);

/* dst(x) = sum_mu [ U_mu(x) v(x + mu) + U_mu(x - mu)^dagger v(x - mu) ]: the
 * colour part of the Wilson Dslash hopping term.  U: matrix field with 4 links
 * per site; v, dst: matrix or colour-vector fields with one object per site,
 * of the same kind (ETYPE otherwise); all FP64 storage (EUNSUPPORTED
 * otherwise) on one lattice (ESHAPE otherwise), in any layouts.  Each of the
 * 8 products is accumulated on its own and the products are added in the
 * arithmetic `math` (as for su3s_eval_math; EINVAL for another value).  dst
 * overlapping U or v: EINVAL.  Pad sites are not touched. */
int su3s_hop(su3s_field* dst, const su3s_field* U, const su3s_field* v, int math, void* stream);

/* The Wilson Dslash hopping term with its spin structure (the operator the
 * paper names for its port to GPUs, Sec. 6):
 *   dst(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
 *                   + (1 + gamma_mu) U_mu(x - mu)^dagger psi(x - mu) ]
 * with Euclidean gamma matrices in the chiral basis:
 *   gamma_mu = [[0, s_mu], [s_mu^dagger, 0]] in 2x2 spin blocks,
 *   s_x = [[0, i], [i, 0]], s_y = [[0, -1], [1, 0]], s_z = [[i, 0], [0, -i]],
 *   s_t = 1 (so gamma_5 = gamma_x gamma_y gamma_z gamma_t = diag(1, 1, -1, -1)).
 * A spinor field is a colour-vector field with nmu = 4 objects per site,
 * object s being spin component s (canonical host layout
 * double[V][4][3][2]: site, spin, colour, re/im).  psi and dst: such fields;
 * U: a matrix field with 4 links per site (ETYPE otherwise); all FP64
 * storage (EUNSUPPORTED otherwise), one lattice (ESHAPE otherwise), any
 * layouts.  Each term projects psi to a two-component half spinor, multiplies
 * it by the link and rebuilds the four spin components; the products are
 * accumulated in the arithmetic `math` (as for su3s_eval_math, with its range
 * guard; EINVAL for another value).  dst overlapping U or psi: EINVAL.  Pad
 * sites are not touched. */
int su3s_dslash(su3s_field* dst, const su3s_field* U, const su3s_field* psi, int math,
                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SU3S_H */
