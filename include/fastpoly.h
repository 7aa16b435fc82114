/*
 * fastpoly -- GB300 (sm_103a) library for fast polynomial evaluation and
 * composition through evaluation trees, after G. Moroz, "Fast polynomial
 * evaluation and composition" (arXiv:1307.5655).
 *
 * C ABI.  Plain pointers and sizes only.  Unless stated otherwise:
 *   - every function returns FP_OK (0) or a negative fp_status code and
 *     leaves its outputs untouched on error;
 *   - "host" pointers are ordinary CPU memory, "device" pointers are CUDA
 *     global memory of the current device, owned by the caller;
 *   - device work is enqueued asynchronously on `stream` (a cudaStream_t,
 *     NULL = the legacy default stream); the call returns once the work is
 *     enqueued, and inputs must stay valid until the stream reaches it;
 *   - a tree is owned by the library from fp_compile until fp_free; it is
 *     immutable, so one tree may serve concurrent calls on several streams.
 */
#ifndef FASTPOLY_H
#define FASTPOLY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
typedef enum {
  FP_OK = 0,
  FP_E_BAD_VALUE = -1,   /* null pointer, negative size or exponent, NaN coefficient, coefficient not < p */
  FP_E_DUP_TERM = -2,    /* two terms with the same exponent vector */
  FP_E_BAD_SCHEME = -3,  /* unknown scheme, or a custom f with f(n) outside (0, n] */
  FP_E_DTYPE = -4,       /* value type not available for this tree */
  FP_E_NOMEM = -5,       /* host or device allocation failed */
  FP_E_TOO_LARGE = -6,   /* a size beyond the documented limits */
  FP_E_CUDA = -7,        /* a CUDA call or kernel launch failed */
  FP_E_TIMEOUT = -8,     /* a bounded device-side wait gave up */
  FP_E_INTERNAL = -9     /* a compiled schedule failed the library's own bounds check (a library fault) */
} fp_status;

/* Function schemes f (Sec. 1.1, Def. 1.2, and the balanced scheme of Sec. 1.2).
 * With n = #terms - 1 of the (sub)polynomial, p = a(x) x^(e) + b(x) where b
 * holds the f(n) lowest terms:
 *   FP_SCHEME_D  Direct   f(n) = n
 *   FP_SCHEME_H  Horner   f(n) = 1
 *   FP_SCHEME_E  Estrin   f(n) = 2^floor(log2 n)
 *   FP_SCHEME_B  Balanced f(n) = floor((n+1)/2), i.e. floor(#terms/2) low terms
 *   FP_SCHEME_CUSTOM  f(n) = f_table[n] for 1 <= n < f_table_len (the paper's
 *                user-defined schemes, e.g. Estrin above a threshold and Horner
 *                below, Remark of Sec. 1.1). */
typedef enum {
  FP_SCHEME_D = 0,
  FP_SCHEME_H = 1,
  FP_SCHEME_E = 2,
  FP_SCHEME_B = 3,
  FP_SCHEME_CUSTOM = 4
} fp_scheme;

/* Value types (the paper evaluates over any ring-like type, Sec. 2.3):
 *   FP_F64   IEEE double, round to nearest; fused multiply-adds.
 *   FP_F32C  float with compensation (error-free transformations); the result
 *            is an unevaluated pair hi + lo.
 *   FP_IV64  closed intervals of doubles [lo, hi] with directed rounding.
 *   FP_MODP  integers modulo p = 2^64 - 2^32 + 1, canonical in [0, p). */
typedef enum { FP_F64 = 0, FP_F32C = 1, FP_IV64 = 2, FP_MODP = 3 } fp_dtype;

typedef struct fp_tree fp_tree;

/* Limits. */
#define FP_MAX_VARS 8
#define FP_MAX_TERMS (1 << 24)
#define FP_MAX_LAZY_HEIGHT 63

/*
 * fp_compile -- build the evaluation tree of a polynomial (Def. 1.1, 1.2,
 * the multivariate Remark of Sec. 1.1, lazy heights Def. 1.3, powers Sec. 2.2)
 * and upload its evaluation schedule to the current device.
 *
 *   nvars        number of variables, 1..FP_MAX_VARS.
 *   nterms       number of terms, 0..FP_MAX_TERMS (0, or all coefficients
 *                zero, gives the zero polynomial).
 *   exps         host, int32 [nterms][nvars], non-negative; any term order
 *                (terms are sorted into decreasing lex order, x1 > x2 > ...).
 *   coeffs       host; double [nterms] when coeff_type is FP_F64, uint64
 *                [nterms] (each < p) when coeff_type is FP_MODP.  Terms with a
 *                zero coefficient are dropped.
 *   coeff_type   FP_F64 (the tree then serves FP_F64, FP_F32C and FP_IV64;
 *                FP_F32C rounds the coefficients to float, FP_IV64 uses the
 *                degenerate intervals [c, c]) or FP_MODP (serves FP_MODP).
 *   scheme       see fp_scheme; f_table/f_table_len only for FP_SCHEME_CUSTOM.
 *   out          receives the new tree.
 * Errors: FP_E_BAD_VALUE, FP_E_DUP_TERM, FP_E_BAD_SCHEME, FP_E_TOO_LARGE
 * (nvars, nterms, or lazy height above the limits), FP_E_NOMEM, FP_E_CUDA,
 * FP_E_INTERNAL (every schedule is checked against the bounds of the arrays
 * and tables the kernels index before it is uploaded; a failure is a fault of
 * the library's compiler, reported instead of running the kernels on it).
 * Synchronous: returns after the schedule is resident on the device.
 */
int fp_compile(int nvars, int64_t nterms, const int32_t* exps, const void* coeffs,
               fp_dtype coeff_type, fp_scheme scheme, const int32_t* f_table,
               int64_t f_table_len, fp_tree** out);

/* fp_compile_host -- the same tree construction as fp_compile, on the host
 * only: nothing is uploaded and no CUDA call is made.  The tree can be
 * inspected with fp_tree_info / fp_tree_export; fp_eval on it returns
 * FP_E_DTYPE.  Same arguments and errors as fp_compile (no FP_E_CUDA). */
int fp_compile_host(int nvars, int64_t nterms, const int32_t* exps, const void* coeffs,
                    fp_dtype coeff_type, fp_scheme scheme, const int32_t* f_table,
                    int64_t f_table_len, fp_tree** out);

/* fp_free -- release a tree and its device memory (NULL is a no-op). The
 * caller must make sure no enqueued work still uses it. */
void fp_free(fp_tree* t);

/*
 * fp_eval -- evaluate a compiled tree at npts points (the coefficient walk of
 * Sec. 2.1 with the powers of Sec. 2.2), one point per GPU lane group.
 *
 * Layouts (all device memory, structure of arrays, v = variable index):
 *   FP_F64   points double [nvars][npts];       out double [npts]
 *   FP_F32C  points float  [nvars][npts];       out float [2][npts] (hi, then lo)
 *   FP_IV64  points double [nvars][2][npts]     (per variable: npts lower
 *            bounds, then npts upper bounds);   out double [2][npts] (lo, hi)
 *   FP_MODP  points uint64 [nvars][npts];       out uint64 [npts], in [0, p)
 *            (points >= p are taken modulo p).
 * The IV64 result is bit-identical to the walk run with directed rounding on
 * the CPU in the tree's operation order; FP_MODP is exact; FP_F64 satisfies
 * |r - p(x)| <= 4 n u sum_e |c_e x^e| (n = #terms - 1, u = 2^-53).
 * Errors: FP_E_BAD_VALUE, FP_E_DTYPE, FP_E_CUDA.  npts = 0 does nothing.
 */
int fp_eval(const fp_tree* t, fp_dtype dtype, const void* points, int64_t npts, void* out,
            void* stream);

/* Launch configuration for fp_eval_ex.
 *   kernel  0: automatic;
 *           1: grouped ops -- chains of single-child nodes run as a register
 *              loop; under schemes E and B, dense runs of <= 16 terms of the
 *              innermost variable (whole subtrees, or a node with its last
 *              children) by a compiled template of the scheme's split (MODP:
 *              Horner's rule over the run, the same residue); FP64, FP32C and
 *              MODP only, power table in shared memory (else FP_E_TOO_LARGE);
 *           2: node by node (any tree and value type).
 * MODP results are identical for every configuration; FP64 and FP32C results
 * of configuration 1 may differ in the last bits (another summation order
 * inside blocks) and satisfy the same error bounds. */
typedef struct {
  int kernel;
  int points_per_thread;  /* 0: automatic; 1, 2 or 4 (FP64 and IV64: 1 or 2) */
  int reserved[2];
} fp_launch_cfg;

/* fp_eval_ex -- fp_eval with an explicit launch configuration (cfg may be
 * NULL: automatic).  Points per thread change the launch shape only: results
 * are identical for every count. */
int fp_eval_ex(const fp_tree* t, fp_dtype dtype, const void* points, int64_t npts, void* out,
               void* stream, const fp_launch_cfg* cfg);

/* fp_tune -- the autotuner: times every launch configuration (kernel x points
 * per thread) on the caller's points (three runs each after a warm-up),
 * stores the fastest in the tree for this value type -- fp_eval then uses it
 * -- and in a process-wide cache keyed by (value type, variables, scheme,
 * log2 node count, log2 point count) that fp_eval consults for untuned trees
 * of the same shape.  Leaves the tuned result in `out`; synchronises
 * `stream`; writes the choice to *best when non-NULL. */
int fp_tune(fp_tree* t, fp_dtype dtype, const void* points, int64_t npts, void* out, void* stream,
            fp_launch_cfg* best);

/* fp_tune_scheme -- compile a polynomial under the function scheme that
 * evaluates it fastest on the given points.  Candidates: the combined scheme
 * of the Remark of Sec. 1.1 -- Estrin's split f(n) = 2^floor(log2 n) for runs
 * of more than k0 terms, Horner's f(n) = 1 below -- for k0 = 1 (Estrin
 * everywhere), 2, 4, ..., the first power of two >= nterms (Horner
 * everywhere), and the Balanced scheme; each compiled and tuned as fp_tune
 * does, the fastest kept and the others freed.
 *   nvars ... coeff_type: as fp_compile.   dtype, points, npts, out, stream:
 *   as fp_tune (`out` holds the winner's result).
 *   k0_out (may be NULL): the chosen k0, 0 for the Balanced scheme.
 *   tree_out: the chosen tree, compiled and tuned; the caller frees it.
 * Synchronous.  Errors: those of fp_compile (invalid terms) and fp_tune. */
int fp_tune_scheme(int nvars, int64_t nterms, const int32_t* exps, const void* coeffs,
                   fp_dtype coeff_type, fp_dtype dtype, const void* points, int64_t npts,
                   void* out, void* stream, int64_t* k0_out, fp_tree** tree_out);

/* fp_eval_host -- the same as fp_eval with host buffers (same layouts):
 * copies the points to the device, evaluates, copies the result back and
 * synchronises `stream`.  Above 2^22 points the work runs in up to 16 chunks
 * as a pipeline -- the copy in of one chunk and the copy out of another
 * overlap the evaluation of a third, on two copy streams of the library
 * ordered after the work already on `stream` -- with pinned host buffers the
 * copies then hide behind the evaluation.  Results are identical to fp_eval.
 * Device buffers come from the library's stream-ordered pool. */
int fp_eval_host(const fp_tree* t, fp_dtype dtype, const void* points_host, int64_t npts,
                 void* out_host, void* stream);

/* Tree introspection (host).  fp_tree_info fills, when non-NULL: node count
 * (terms plus virtual group roots), variables, maximal lazy height, number of
 * distinct powers in the power table, coefficient type. */
int fp_tree_info(const fp_tree* t, int64_t* nnodes, int* nvars, int* max_lazy_height,
                 int* npowers, int* coeff_type);

/* fp_tree_export -- copy the tree (node index order <_t of Sec. 1): per node
 * its exponent vector int32 [nnodes][nvars], the index of the input term it
 * came from (-1 for a virtual node), parent index (-1 for the root), the
 * variable and degree of its partial degree, and its lazy height.  Any
 * pointer may be NULL. */
int fp_tree_export(const fp_tree* t, int32_t* node_exps, int64_t* term_of_node, int64_t* parent,
                   int32_t* pd_var, int64_t* pd, int32_t* lazy_height);

/* fp_tree_schedule -- the grouped schedule that the FP64, FP32C and MODP
 * kernels replay: the walk of Sec. 2.1 in node index order, grouped into ops,
 * with the per-point table those kernels use (no counterpart in the paper;
 * for inspection and host-side checks).  Every op ends with the multiply-add
 * of its last node into its parent's slot.
 *   *nops, *stream_len, *nprog: sizes (always written when non-NULL; call
 *       once with the arrays NULL to size them).
 *   op_words [nops][4] uint32: word 0 = kind (bits 0..1: 0 one node, 1 chain
 *       of single-child nodes, 2 dense subtree block evaluated by the scheme's
 *       own splits, 3 partial block = a node N and its last children forming
 *       the lower part b of a split of N's run, evaluated with N's slot as
 *       N's value) | S (the slot read, bits 2..7) | D (the parent's slot,
 *       8..13) | LEAF (14) | FIRST (15: the last node is its parent's first
 *       child) | UNIFORM (16: one power along a chain) | PID (17..31: table
 *       position of the outgoing edge's power; 0x7FFF: recomputed, see word
 *       2); word 1 = length - 1 (bits 0..7), and for a floating-point
 *       Balanced block of 17 to 22 nodes f = the scheme's split of its run
 *       (bits 8..15) and the table position of x^f (16..31): the run is
 *       T(b) + T(a) x^f, its coefficients stored as the runs a and b, each
 *       from a multiple of 4 elements; word 2 = first node, or for PID 0x7FFF
 *       (a block or partial block of a large Balanced tree whose edge power
 *       few ops read) base | m << 15 | (d mod 2^m) << 19: the edge power x^d
 *       is rebuilt from the table entry at position base (0x7FFF: x) by m
 *       steps of squaring and, where the bit of d is set, multiplying by x
 *       (the power program's own steps); word 3 = stream offset (bits
 *       0..30) | ROOT_EDGE (31: an op past the split, see layout, whose edge
 *       goes into the root's slot).
 *   op_a_node, op_b_node [nops]: node whose coefficient is the op's leaf value
 *       (single-node ops) / initialises the parent's slot when FIRST; -1 = 0.
 *   stream [stream_len]: node whose coefficient sits in each slot of the
 *       coefficient stream of chains and blocks, -1 for padding.
 *   prog [nprog][2]: the power program per point, {op | A1 << 2 | A2 << 17,
 *       destination position}; op 0 loads variable A1, 1 squares position
 *       A1, 2 multiplies positions A1 and A2.
 *   chain_pid [nnodes - 1]: table position of each node's edge power (read
 *       inside chains).
 *   block_pow [17]: table position of x_b^d read by the block templates
 *       after the program (-1: absent); b = nvars - 1, the innermost
 *       variable, whose groups are univariate polynomials under the scheme.
 *   layout [8]: nlive (the walk's powers sit at positions [0, nlive)),
 *       nslot (slot s sits at position nlive + s), table entries per point,
 *       block scheme (FP_SCHEME_E / FP_SCHEME_B when blocks are used, else 0),
 *       root is a leaf, root slot, position of the root's power (-1: none),
 *       split: the first op of the root's later children (0: none) -- ops
 *       [0, split) evaluate the root's first child's subtree (nodes 0 .. its
 *       root) and its edge into the root's slot, ops [split, nops) the other
 *       children, so small grids run the two ranges in two warps with tables
 *       of their own; the second keeps the values of its ROOT_EDGE ops and,
 *       after the first is done, applies them in walk order to the first's
 *       root slot (the walk's own operations in its order: the result is
 *       bit-identical to one warp's).
 * Any array pointer may be NULL.  FP_E_BAD_VALUE for a NULL tree. */
int fp_tree_schedule(const fp_tree* t, int64_t* nops, uint32_t* op_words, int64_t* op_a_node,
                     int64_t* op_b_node, int64_t* stream_len, int64_t* stream, int32_t* nprog,
                     uint32_t* prog, uint32_t* chain_pid, int32_t* block_pow, int32_t* layout);

/*
 * Batched evaluation: many jobs (trees of uneven size, each with its own
 * points) of one value type in one launch per shared-memory class.  Each job
 * uses the layouts of fp_eval and gets the result fp_eval would give it; the
 * most expensive jobs are scheduled first.  Jobs with npts = 0 are skipped;
 * zero polynomials are refused (FP_E_BAD_VALUE: use fp_eval).
 */
typedef struct {
  const fp_tree* tree;  /* compiled tree (serves the batch's value type) */
  const void* points;   /* device, layout of fp_eval */
  int64_t npts;
  void* out;            /* device, layout of fp_eval */
} fp_job;

typedef struct fp_batch fp_batch;

/* fp_eval_batch -- one-shot: plan, upload the job table (stream-ordered
 * allocation, released after the launches) and launch. */
int fp_eval_batch(fp_dtype dtype, const fp_job* jobs, int64_t njobs, void* stream);

/* fp_batch_create -- plan a batch once and upload its job table (synchronous);
 * fp_batch_launch enqueues its kernels only (no allocation, no copy), so it can
 * be captured into a CUDA graph and replayed while the trees and buffers named
 * by the jobs stay alive; fp_batch_free releases the table. */
int fp_batch_create(fp_dtype dtype, const fp_job* jobs, int64_t njobs, fp_batch** out);
int fp_batch_launch(const fp_batch* batch, void* stream);
void fp_batch_free(fp_batch* batch);

/*
 * A resident evaluation kernel with a device work queue: persistent blocks
 * that stay on the GPU and take tiles of jobs published while they run, so
 * new work enters a running kernel without a launch (no counterpart in the
 * paper).  One value type per resident kernel.  Jobs use the layouts and give
 * the results of fp_eval.  The queue lives in pinned host memory mapped into
 * the device: fp_resident_submit writes a job's descriptor and publishes its
 * tiles with plain stores (no stream operation); blocks claim tiles one at a
 * time (dynamic balance over the SMs); the block that finishes a job's last
 * tile sets its completion flag, which fp_resident_query reads.
 * Waits are bounded: idle blocks sleep between polls and exit after
 * idle_exit_s without work; a later submission (or fp_resident_wait) launches
 * the kernel again.  The kernel occupies up to blocks_per_sm blocks on every
 * SM while it runs.  One host thread should drive a resident kernel.  The
 * kernel follows no stream: a job's points (and anything that writes its
 * output buffer) must be complete on the device when it is submitted.
 */
typedef struct fp_resident fp_resident;
typedef struct {
  fp_dtype dtype;       /* value type of every job */
  int max_jobs;         /* capacity of the job table (1 .. 2^24) */
  size_t smem_bytes;    /* shared memory per block (0: 48 KB): a job whose
                           per-point table needs more is refused (FP_E_TOO_LARGE) */
  int blocks_per_sm;    /* <= 0: as many as fit */
  double idle_exit_s;   /* blocks exit after this long without work (<= 0: 0.05 s) */
  int64_t max_items;    /* capacity of the work-item table (<= 0: the larger of
                           16 max_jobs and 65536; 16 bytes each); a
                           job takes one item per 4 tiles of 128 (FP32C, MODP:
                           256) points */
} fp_resident_cfg;

/* Allocates the queue and launches the kernel on a stream of its own.
 * Errors: FP_E_BAD_VALUE, FP_E_DTYPE, FP_E_TOO_LARGE, FP_E_NOMEM, FP_E_CUDA. */
int fp_resident_create(const fp_resident_cfg* cfg, fp_resident** out);
/* Publish a job (tree, device points and output; see fp_job) and return its
 * ticket.  The job's buffers and tree must stay valid until it completes.
 * Errors: FP_E_BAD_VALUE (zero polynomial included: use fp_eval), FP_E_DTYPE,
 * FP_E_TOO_LARGE (table too large for the blocks, or the job or item table
 * is full). */
int fp_resident_submit(fp_resident* r, const fp_job* job, int64_t* ticket);
/* FP_OK when the job has completed, 1 while it is pending. */
int fp_resident_query(const fp_resident* r, int64_t ticket);
/* Wait at most timeout_s seconds for the job: FP_OK or FP_E_TIMEOUT. */
int fp_resident_wait(fp_resident* r, int64_t ticket, double timeout_s);
/* Whether the kernel is running, whether its blocks have ever left on the
 * idle timeout (the device-side wait that ran out), jobs submitted. */
int fp_resident_state(const fp_resident* r, int* running, int* idle_exits, int64_t* jobs);
/* Ask the blocks to exit once the published tiles are taken, and wait at most
 * timeout_s (<= 0: 60) for them: FP_OK or FP_E_TIMEOUT.  Submissions after a
 * stop are refused (FP_E_BAD_VALUE). */
int fp_resident_stop(fp_resident* r, double timeout_s);
/* Stops the kernel (waiting up to 60 s) and releases everything. */
void fp_resident_free(fp_resident* r);

/*
 * Serving with continuous batching.  Requests (a resident compiled tree, a
 * value type, host points, a host result buffer) are submitted from any
 * thread and complete asynchronously.  A worker thread admits pending
 * requests oldest first while their device footprint (points + results) fits
 * in hbm_budget_bytes (a request larger than the whole budget runs alone),
 * groups requests of one value type into one batched launch in one of
 * `streams` slots (copies in, fp_eval_batch, copies out), and retires
 * batches as they finish, so requests that arrive while batches run are
 * admitted as soon as a slot and memory free up.  A batch lasts as long as
 * its largest request: small requests (estimated work below about 1.7 ms of
 * FP64 evaluation) are batched apart from large ones and launched on a
 * stream of the highest priority (each slot has one beside its
 * default-priority stream), and with two or more slots the first takes
 * small requests only.  Results equal fp_eval's.
 * Host buffers should be pinned (page-locked) for the copies to overlap; they
 * must stay valid until the request completes.  Trees must outlive the
 * requests that use them.
 */
typedef struct fp_server fp_server;
typedef struct {
  size_t hbm_budget_bytes;  /* device bytes for the points and results in flight (> 0) */
  int max_batch_jobs;       /* requests per batched launch (<= 0: 1024) */
  int streams;              /* slots: batches in flight at once (<= 0: 4) */
} fp_server_cfg;
typedef struct {
  int64_t ticket;     /* as returned by fp_server_submit */
  int status;         /* FP_OK or an error code */
  double latency_us;  /* from submission to observed completion */
} fp_completion;

int fp_server_create(const fp_server_cfg* cfg, fp_server** out);
/* npts = 0 completes at once.  Errors: FP_E_BAD_VALUE, FP_E_DTYPE. */
int fp_server_submit(fp_server* s, const fp_tree* tree, fp_dtype dtype, const void* points_host,
                     int64_t npts, void* out_host, int64_t* ticket);
/* Up to `max` completions since the last poll (any order), count in *n. */
int fp_server_poll(fp_server* s, fp_completion* done, int max, int* n);
/* Wait (at most timeout_s seconds; <= 0: 60) until every submitted request has
 * completed; FP_E_TIMEOUT otherwise. */
int fp_server_drain(fp_server* s, double timeout_s);
/* Peak device bytes admitted at once, number of batches launched. */
int fp_server_stats(const fp_server* s, size_t* peak_bytes, int64_t* batches);
/* Stops after the requests already submitted have completed. */
void fp_server_destroy(fp_server* s);

/*
 * fp_compose -- batched composition r_j(y) = p_j(q_j(y)) for j < npairs: the
 * coefficient walk (Sec. 2.1) of p's tree run over polynomial values, the
 * "composition" of the paper's title, where values grow with each product
 * (Sec. 1.2).  Every pair shares the tree of p (its terms and scheme); the
 * coefficients may differ per pair.  Univariate trees only.
 *
 *   p        tree from fp_compile (nvars = 1).  FP_MODP needs a FP_MODP tree,
 *            FP_F64 a FP_F64 tree.
 *   dtype    FP_MODP (exact; products by number-theoretic transforms) or
 *            FP_F64: products whose operands both have at least 256
 *            coefficients run on the tensor cores -- each operand cut into
 *            blocks of 64 coefficients with an exponent each, every value
 *            split into 7 signed 7-bit slices (bf16), the slice products
 *            summed exactly in FP32 and recombined in 64-bit fixed point per
 *            block of the result; shorter products by direct convolution.
 *            The tensor-core products are accurate blockwise: the error at a
 *            coefficient is about 2^-45 (8 slices: 2^-52) of the largest
 *            block products meeting there, not of the coefficient itself (a
 *            coefficient far below its 64-coefficient neighbourhood, as in
 *            the steep tails of q^e, keeps only that absolute accuracy); the
 *            direct convolution (fp_set_compose_f64 with min_len < 0) is
 *            componentwise: |error|_i <= gamma (|p| o |q|)_i.
 *   pcoeffs  device, [npairs][nterms] in the term order given to fp_compile,
 *            or NULL to use the tree's own coefficients for every pair.  Terms
 *            whose compile-time coefficient was zero are not in the tree and
 *            are ignored (compile with non-zero placeholders).
 *   q        device, [npairs][degq + 1], coefficient of y^i at index i.
 *   out      device, [npairs][deg(p) * degq + 1].
 * Work space (about (lazy height + 6) x npairs x deg(p) x degq x 8 bytes) is
 * allocated on `stream` from the library's stream-ordered pool (which keeps
 * up to 4 GiB of freed device memory mapped for reuse) and released before returning;
 * the call synchronises `stream` while it uploads its tables, and an FP64
 * composition that used the tensor cores synchronises it again at the end
 * to report FP_E_TIMEOUT (a bounded wait for tensor-core work gave up).
 * Errors: FP_E_BAD_VALUE, FP_E_DTYPE, FP_E_TOO_LARGE (output longer than
 * 2^26), FP_E_NOMEM, FP_E_CUDA, FP_E_TIMEOUT.
 */
int fp_compose(const fp_tree* p, fp_dtype dtype, const void* pcoeffs, const void* q, int32_t degq,
               int64_t npairs, void* out, void* stream);

/* fp_set_compose_f64 -- process-wide settings of FP64 composition products
 * (no counterpart in the paper): slices per operand on the tensor cores (6,
 * 7 or 8; 0 = 7) and the shortest operand length sent to them (0 = 256;
 * negative: never, every product by direct convolution).  Calls already
 * enqueued keep the settings they started with.  Errors: FP_E_BAD_VALUE. */
int fp_set_compose_f64(int slices, int min_len);

/* fp_compose_workspace -- the device work space, in bytes, that fp_compose
 * and fp_compose_noalloc use for these arguments (per_pair_coeffs: non-zero
 * when pcoeffs will be given, zero for the tree's own coefficients), counted
 * by running the composition driver without launching, copying or allocating
 * anything (each buffer rounded up to 256 bytes).  Host only; no CUDA call.
 * The paper has no counterpart: this is a property of the library.
 * Errors: those of fp_compose's argument checks (FP_E_BAD_VALUE, FP_E_DTYPE,
 * FP_E_TOO_LARGE). */
int fp_compose_workspace(const fp_tree* p, fp_dtype dtype, int per_pair_coeffs, int32_t degq, int64_t npairs,
                         size_t* bytes);

/*
 * fp_compose_noalloc -- fp_compose for callers that must not allocate device
 * memory: code running under a memory manager that owns the whole device
 * (a serving engine that reserves HBM up front and forbids libraries from
 * calling cudaMalloc / cudaMallocAsync), or code running where allocation
 * calls are not allowed.  The paper has no counterpart; this is a property of
 * the library, not of the method.
 *
 * Same arguments, layouts and results as fp_compose.  The work space comes
 * from one region of FP_NOALLOC_SCRATCH_BYTES that every GPU loading the
 * library holds until the process exits; nothing is allocated or freed.
 *   - The first call on a device looks up that region's device address
 *     (cudaGetSymbolAddress).
 *   - All calls share the region and it keeps the last call's contents, so
 *     calls that overlap on the GPU (other streams, other threads) race:
 *     serialise them.
 *   - A problem whose work space (fp_compose_workspace) exceeds the region
 *     returns FP_E_TOO_LARGE before any work is enqueued (roughly: npairs x
 *     deg(p) x degq x 8 bytes x (lazy height + 6) must fit).
 * The call synchronises `stream` while it uploads its small tables.
 */
#define FP_NOALLOC_SCRATCH_BYTES (64ull << 20)
int fp_compose_noalloc(const fp_tree* p, fp_dtype dtype, const void* pcoeffs, const void* q,
                       int32_t degq, int64_t npairs, void* out, void* stream);

/* fp_measure_rates -- sustained arithmetic rates of this GPU for the
 * operations the evaluation kernels are bound by: the roofline denominators
 * (no counterpart in the paper).  Each rate is measured with the library's
 * own arithmetic, 8 independent dependent chains per thread, 8 blocks of 256
 * threads per SM, one warm-up launch, then 3 launches timed with CUDA events
 * on `stream` (synchronous; a few tens of ms per rate).  rates[i], in G
 * operations per second, for i < nrates (at most FP_RATE_COUNT):
 *   FP_RATE_DFMA         FP64 fused multiply-add (one FP64 node of the walk)
 *   FP_RATE_DADD_RD      FP64 add rounded down
 *   FP_RATE_DMUL_RU      FP64 multiply rounded up
 *   FP_RATE_FFMA         FP32 fused multiply-add
 *   FP_RATE_F32C_MAD     compensated FP32 multiply-add, general form (one
 *                        FP32C node with no operand known exact)
 *   FP_RATE_F32C_HORNER  the same with a coefficient added and x a point
 *                        (exact zero low parts dropped: a Horner step)
 *   FP_RATE_MODP_MULADD  (a b + c) mod p (one MODP node)
 *   FP_RATE_MODP_BUTTERFLY  (a, b) -> (a + w b, a - w b) mod p (one radix-2
 *                        butterfly of the number-theoretic transforms)
 *   FP_RATE_IMAD         32-bit integer multiply-add, a b + c mod 2^32
 *   FP_RATE_IMAD_WIDE    32 x 32 -> 64-bit product plus a 64-bit addend (the
 *                        partial products of the 64-bit arithmetic mod p)
 * An interval walk costs 4 directed-rounding operations per node (a product,
 * 2, plus the coefficient's addition at a parent or the accumulation at a
 * non-first child, 2): its bound is FP_RATE_DADD_RD / 4 (products issue at
 * the additions' rate). 
 * Errors: FP_E_BAD_VALUE (NULL rates, negative nrates), FP_E_NOMEM, FP_E_CUDA. */
enum {
  FP_RATE_DFMA = 0,
  FP_RATE_DADD_RD = 1,
  FP_RATE_DMUL_RU = 2,
  FP_RATE_FFMA = 3,
  FP_RATE_F32C_MAD = 4,
  FP_RATE_F32C_HORNER = 5,
  FP_RATE_MODP_MULADD = 6,
  FP_RATE_MODP_BUTTERFLY = 7,
  FP_RATE_IMAD = 8,
  FP_RATE_IMAD_WIDE = 9,
  FP_RATE_COUNT = 10
};
int fp_measure_rates(double* rates, int nrates, void* stream);

/* fp_eval_plain_f64 -- the comparison baseline: one launch per polynomial,
 * one thread per point, Horner's rule over the dense coefficient vector
 * coeffs[0..ncoeffs-1] (index = degree), FP64, no tree.  Device pointers. */
int fp_eval_plain_f64(const double* coeffs, int64_t ncoeffs, const double* points, int64_t npts,
                      double* out, void* stream);

/*
 * Exact integer values through residues (a residue number system): the
 * paper evaluates polynomials with multi-precision integer coefficients at
 * multi-precision points (Sec. 3); here a value is represented by its
 * residues modulo k primes q_i = 2^64 - c_i (the k largest primes of that
 * form with c_i < 2^32, largest first), the walk runs once per prime, and
 * the Chinese remainder theorem gives back the integer when it lies in
 * (-Q/2, Q/2], Q = q_0 ... q_{k-1}.
 */
#define FP_RNS_MAX_PRIMES 64
#define FP_RNS_COEFFS 100  /* coeff_type reported by fp_tree_info for such trees */

/* fp_rns_primes -- the first k primes q_0 > q_1 > ... (k <= FP_RNS_MAX_PRIMES),
 * host uint64 [k].  Errors: FP_E_BAD_VALUE. */
int fp_rns_primes(int k, uint64_t* q);

/* fp_compile_rns -- fp_compile for integer coefficients given by residues:
 * residues host uint64 [k][nterms], residues[i][t] = c_t mod q_i (each < q_i,
 * else FP_E_BAD_VALUE).  A term whose residues are all zero is dropped.  The
 * tree serves fp_eval_rns only (fp_eval returns FP_E_DTYPE).  Other arguments
 * and errors as fp_compile. */
int fp_compile_rns(int nvars, int64_t nterms, const int32_t* exps, int k, const uint64_t* residues,
                   fp_scheme scheme, const int32_t* f_table, int64_t f_table_len, fp_tree** out);

/* fp_eval_rns -- the walk modulo each prime of the tree: points device uint64
 * [k][nvars][npts] (residues of the points; values >= q_i are reduced), out
 * device uint64 [k][npts], out[i][j] = p(x_j) mod q_i exactly.  One launch:
 * blocks over points by primes.  Errors as fp_eval. */
int fp_eval_rns(const fp_tree* t, const uint64_t* points, int64_t npts, uint64_t* out, void* stream);

/* fp_crt -- integers from residues (Garner's mixed-radix algorithm):
 * residues device uint64 [k][npts] (each < q_i), limbs device uint64
 * [npts][k]: the value X in (-Q/2, Q/2] with X = residues[i][j] mod q_i,
 * as k 64-bit limbs, least significant first, two's complement.  Work per
 * value O(k^2).  Errors: FP_E_BAD_VALUE, FP_E_NOMEM, FP_E_CUDA. */
int fp_crt(int k, const uint64_t* residues, int64_t npts, uint64_t* limbs, void* stream);

/* Human-readable name of a status code (static storage). */
const char* fp_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* FASTPOLY_H */
