/*
 * bmlp.h - C ABI of the GB300 (sm_103a) Boolean Matrix Logic Programming
 * library: bottom-up evaluation of linear dyadic recursive datalog
 *
 *     p(X,Y) <- r(X,Y).
 *     p(X,Y) <- r(X,Z), p(Z,Y).
 *
 * as Boolean matrix algebra (paper: "Boolean Matrix Logic Programming on the
 * GPU", Sec. 2-4). A relation over n constants is an n x n Boolean matrix R:
 * R[i][j] = 1 iff r(c_i, c_j) holds (Sec. 3.2; constants are mapped to
 * 0..n-1 by the caller). Boolean "+" is OR and the product is OR-of-ANDs
 * (Sec. 2).
 *
 * Matrix formats (argument `fmt`):
 *   BMLP_FMT_U8        n x n bytes, row-major, leading dimension n. Any
 *                      nonzero input byte means 1; outputs are 0 or 1.
 *   BMLP_FMT_PACKED64  n rows of ceil(n/64) uint64 words, row-major. Bit j of
 *                      row i is bit (j % 64), least significant first, of word
 *                      j / 64 (the bit code b_i of Sec. 3.2). Input bits at
 *                      columns >= n are ignored; output padding bits are 0.
 *   BMLP_FMT_I8        n x n int8, row-major: read and written as BMLP_FMT_U8
 *                      (nonzero means 1; outputs 0 or 1).
 *   BMLP_FMT_E4M3      n x n FP8 E4M3 bytes, row-major, the operand form of the
 *                      8-bit tensor-core path: 0x00 and 0x80 (the two zeros)
 *                      mean 0, any other byte means 1; outputs are 0x00 or
 *                      0x38 (1.0). Inputs are converted in a context buffer
 *                      and outputs written back from one (two extra passes
 *                      over n^2 bytes). Not accepted by bmlp_batch_run or
 *                      bmlp_rms_tc_noalloc (BMLP_ERR_INVALID_ARG).
 *
 * Pointers: every matrix pointer may be device memory or host memory
 * (pageable or pinned); the library detects which with
 * cudaPointerGetAttributes and stages host buffers through its own device
 * workspace. The caller owns all input and output buffers; the context owns
 * its workspace. Inputs and outputs must not overlap.
 *
 * Streams: every call is ordered on `stream` (0 = legacy default stream).
 * Calls with device outputs return once the work is enqueued and the fixpoint
 * has been decided (see bmlp_options.loop); host outputs are complete on
 * return.
 *
 * Errors: every entry point returns a bmlp_status; nothing is thrown across
 * the ABI. bmlp_last_error() gives a message for the last failure on a
 * context. A context may be used by one host thread at a time.
 */
#ifndef BMLP_H
#define BMLP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cudaStream_t; /* the CUDA runtime's stream handle */

typedef enum bmlp_status {
    BMLP_OK = 0,
    BMLP_ERR_INVALID_ARG = 1,   /* null pointer with n > 0, n < 0, bad enum  */
    BMLP_ERR_OOM = 2,           /* device workspace allocation failed        */
    BMLP_ERR_CUDA = 3,          /* a CUDA runtime/driver call failed         */
    BMLP_ERR_TIMEOUT = 4,       /* a bounded in-kernel wait ran out           */
    BMLP_ERR_NOT_CONVERGED = 5, /* fixpoint not reached within max_iters      */
    BMLP_ERR_UNSUPPORTED = 6,   /* size or variant outside what is built      */
    BMLP_ERR_BUDGET = 7         /* stopped at options.budget_ns; output undefined */
} bmlp_status;

typedef enum bmlp_format {
    BMLP_FMT_U8 = 0,
    BMLP_FMT_PACKED64 = 1,
    BMLP_FMT_I8 = 2,
    BMLP_FMT_E4M3 = 3
} bmlp_format;

/* Which kernel family evaluates the fixpoint. Every variant returns the same
 * bits; they differ only in speed. */
typedef enum bmlp_variant {
    BMLP_AUTO = 0,        /* library choice (learned dispatcher if trained)    */
    BMLP_RMS_TC = 1,      /* repeated squaring on the tcgen05 tensor cores: E4M3
                             operands while R is block-sparse (empty K blocks
                             skipped), packed E2M1 (kind::mxf4) once dense     */
    BMLP_RMS_PACKED = 2,  /* repeated squaring on uint64 row bitsets            */
    BMLP_SMP_TC = 3,      /* frontier expansion, tensor-core frontier product   */
    BMLP_SMP_PACKED = 4   /* frontier expansion on uint64 row bitsets           */
} bmlp_variant;

typedef enum bmlp_loop {
    BMLP_LOOP_HOST = 0,   /* host loop: one product launch per iteration, the
                             changed flag is read back after each             */
    BMLP_LOOP_GRAPH = 1   /* device loop: the iteration runs inside a CUDA graph
                             conditional WHILE node; no host round trip per
                             iteration                                        */
} bmlp_loop;

typedef struct bmlp_options {
    int32_t variant;     /* bmlp_variant                                       */
    int32_t reflexive;   /* 0: R1+ (paths of >= 1 edge, Eq. 1); 1: I + R1+     */
    int32_t max_iters;   /* iteration cap; 0 = the bound of Appendix C
                            (ceil(log2 n) + 2 products for squaring, n + 1
                            levels for frontier expansion)                     */
    int32_t loop;        /* bmlp_loop                                          */
    int32_t profile;     /* 1: time the product kernel with CUDA events        */
    int32_t tc_only;     /* BMLP_RMS_TC closures with n >= 4096: 0 = squarings
                            run on word-indexed bit rows for as long as one
                            costs less than a tensor-core product (R sparse),
                            then on the tensor cores from their result (same
                            fixpoint, same number of products); 1 = every
                            squaring on the tensor cores                      */
    uint64_t timeout_ns; /* bound of every in-kernel wait; 0 = 2 s             */
    uint64_t budget_ns;  /* 0 = none; else the call gives up (BMLP_ERR_BUDGET)
                            once about this much time has passed: checked
                            between launches and, in the packed kernels, by
                            every warp before each row / query (used to time
                            variants with a cap, e.g. by the dispatcher's
                            training sweep)                                    */
    int32_t e4m3_only;   /* BMLP_RMS_TC: 0 = dense squarings run on packed E2M1
                            operands (tcgen05 kind::mxf4, half the bytes per
                            Boolean operation); 1 = every tensor-core squaring
                            on E4M3 operands (kind::f8f6f4). Same bits.       */
    int32_t reserved;    /* 0                                                  */
} bmlp_options;

/* Per-call statistics of the last call on a context. */
typedef struct bmlp_stats {
    int32_t iterations;        /* products (squaring) or levels (frontier)      */
    int32_t variant;           /* variant that ran                              */
    int32_t product_launches;  /* launches of the product kernel                */
    int32_t launches;          /* all kernel launches of the call               */
    int64_t n_pad;             /* padded matrix size used by the kernels        */
    double product_ms;         /* summed device time of the product launches
                                  (only with options.profile = 1)               */
    double issued_ops;         /* Boolean multiply-adds issued x 2 (tensor core
                                  path: 2 * M * N * K per tile actually run)    */
    int32_t e2m1_products;     /* squarings run on packed E2M1 (4-bit) operands */
    int32_t frontier_squarings; /* BMLP_SMP_PACKED closures (n >= 4096): steps
                                  R <- R + R R taken before the frontier
                                  expansion (path-like relations; same closure,
                                  fewer levels)                                 */
    int32_t sparse_squarings;  /* squarings run on word-indexed bit rows:
                                  BMLP_RMS_TC before the tensor cores took over
                                  (counted in iterations, not in
                                  product_launches); BMLP_RMS_PACKED while
                                  fewer than half of R's words were nonzero
                                  (counted in both)                             */
    int32_t sliced_closures;   /* BMLP_SMP_PACKED closures, and query batches
                                  of >= 64 rows (n >= 4096), whose relation
                                  widens the rows fast (R + R R has > 2.8 x
                                  the words of R): expanded 64 rows at a time
                                  (bit-sliced frontiers, one thread-block
                                  cluster per 64 rows for n <= 65,536)          */
    double sparse_ms;          /* their summed device time (options.profile)    */
    double sparse_words;       /* the word ORs they issued                      */
    int32_t host_syncs;        /* times the host waited for the device during
                                  the call to read back a flag, a decision or
                                  the results (1 for a batch that ran as one
                                  device-driven graph: the final read)          */
    int32_t cluster_frontiers; /* of sliced_closures, those run one thread-block
                                  cluster per 64 rows with the frontier in
                                  the cluster's shared memory (query batches,
                                  and closures whose columns are skewed)        */
    int32_t thin_squarings;    /* BMLP_RMS_TC: squarings computed only on the
                                  rows and columns of R that still held zeros
                                  (few, and holding few ones: R close to its
                                  closure); counted in iterations, not in
                                  product_launches                              */
    int32_t table_squarings;   /* BMLP_RMS_PACKED: whole-row squarings run on
                                  shared-memory tables of 4-row ORs (Four
                                  Russians; once R's nonzero words hold >= 10
                                  bits on average, and the first whole-row
                                  step); the others gathered the named rows   */
} bmlp_stats;

typedef struct bmlp_ctx bmlp_ctx;

/* Create a context on CUDA device `device`. The context owns a grow-only
 * device workspace and a few CUDA events. */
bmlp_status bmlp_ctx_create(bmlp_ctx** ctx, int32_t device);

/* Free the workspace and the context (synchronises the device first). */
bmlp_status bmlp_ctx_destroy(bmlp_ctx* ctx);

/* Message of the last failure on ctx (static storage inside ctx). */
const char* bmlp_last_error(const bmlp_ctx* ctx);

/* Fill *opts with the defaults (variant AUTO, host loop, no profiling). */
void bmlp_default_options(bmlp_options* opts);

/* Statistics of the last completed call on ctx. */
bmlp_status bmlp_get_stats(const bmlp_ctx* ctx, bmlp_stats* out);

/*
 * bmlp_rms - all derivable groundings of r2 (BMLP-RMS, paper Sec. 3.3 Eq. 4,
 * Algorithm 1; Def. 1 of Sec. 3.1 for the output):
 *
 *     out = R1+ = sum_{k>=1} R1^k        (out = I + R1+ if opts->reflexive)
 *
 * computed by the fixpoint R <- R + R.R started from R1 (same result as
 * Algorithm 1's (I + R1)^(2^k) followed by one product with R1). R and out
 * are n x n in format fmt. *iters_out (if not null) receives the number of
 * products issued (ceil(log2 L) + 1, L the longest shortest path), or for
 * the frontier variants the deepest level + 1. n = 0 is a no-op that returns
 * BMLP_OK.
 * Variants: BMLP_RMS_TC (n >= 4096: bit-row squarings while R is sparse,
 * see options.tc_only; then tensor cores), BMLP_RMS_PACKED, BMLP_SMP_PACKED
 * (all n rows as frontiers: path-like R is squared first and expanded one
 * row per warp, R whose rows widen fast is expanded 64 rows per CTA), BMLP_SMP_TC,
 * BMLP_AUTO (the learned dispatcher once trained or loaded, else BMLP_RMS_TC).
 */
bmlp_status bmlp_rms(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, void* out,
                     const bmlp_options* opts, int32_t* iters_out, cudaStream_t stream);

/*
 * bmlp_rms_alg1 - R1+ in the literal form of paper Algorithm 1 (Sec. 3.3):
 *
 *     R* = (I + R1)^(2^k)   squaring until a squaring changes nothing
 *     out = R* R1           one more product
 *
 * Same result as bmlp_rms (the squaring form R <- R + R R from R1 saves the
 * last product). *iters_out receives the squarings plus 1: ceil(log2 L0) + 2,
 * with L0 the longest shortest path between two different constants (2 when
 * L0 <= 1). The squarings run as bmlp_rms with BMLP_RMS_TC (bit-row start,
 * operand forms, options.tc_only), the final product on the tensor cores
 * with E4M3 operands. Variants: BMLP_RMS_TC or BMLP_AUTO (the same). R and
 * out as in bmlp_rms; options.reflexive gives I + R1+.
 */
bmlp_status bmlp_rms_alg1(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, void* out,
                          const bmlp_options* opts, int32_t* iters_out, cudaStream_t stream);

/*
 * bmlp_smp - partially grounded queries r2(c, Y) (BMLP-SMP, paper Sec. 3.3
 * Eq. 5, Algorithm 2):
 *
 *     out_q = v_q R1+     for every query row q = 0..nq-1
 *
 * v_q is row q of src_rows (nq rows of ceil(n/64) uint64 words, packed as
 * above; several set bits = a union of constants). out_rows has the same
 * layout. A source is in its own output row only if it lies on a cycle.
 * R is n x n in format fmt. *iters_out receives the deepest frontier level.
 * Variants: BMLP_SMP_PACKED, BMLP_SMP_TC, BMLP_AUTO. BMLP_SMP_PACKED expands
 * one query row per warp, or, for batches of >= 64 rows over a relation whose
 * rows widen fast (n >= 4096), 64 rows at a time with bit-sliced frontiers.
 */
bmlp_status bmlp_smp(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt,
                     const uint64_t* src_rows, int64_t nq, uint64_t* out_rows,
                     const bmlp_options* opts, int32_t* iters_out, cudaStream_t stream);

/*
 * bmlp_insert - incremental closure for a growing database (the dynamic
 * setting of paper Sec. 7): given closure = R1+ (any transitive relation,
 * e.g. the output of bmlp_rms), add the facts r1(u_k, v_k) of `pairs` (m
 * pairs of int32 constants, device or host memory) and update closure in
 * place to (R1 + E)+. Each fact is one rank-1 update: every constant that
 * reaches u_k (and u_k) gains v_k and everything v_k reaches. closure is
 * n x n in format fmt (device or host memory). Facts already derivable cost
 * one word read. Constants outside [0, n) give BMLP_ERR_INVALID_ARG before
 * anything changes. Deleting facts is not incremental: recompute with
 * bmlp_rms.
 */
bmlp_status bmlp_insert(bmlp_ctx* ctx, void* closure, int64_t n, int32_t fmt, const int32_t* pairs, int64_t m,
                        cudaStream_t stream);

/*
 * bmlp_compose - the general binary linear recursion of paper Sec. 3.4
 * (Thm. 1):
 *
 *     p(X,Y) <- r1(X,Y).
 *     p(X,Y) <- r2(X,Z), p(Z,Y).        out = (I + R2+) R1
 *
 * R1, R2 and out are n x n in format fmt over one shared constant index.
 * *iters_out receives the products of the R2 closure. Variants: BMLP_RMS_TC
 * (closure and final product on tensor cores), BMLP_RMS_PACKED, BMLP_AUTO.
 */
bmlp_status bmlp_compose(bmlp_ctx* ctx, const void* R1, const void* R2, int64_t n, int32_t fmt,
                         void* out, const bmlp_options* opts, int32_t* iters_out, cudaStream_t stream);

/*
 * Boolean matrix operators that join BMLP algorithms into larger programs
 * (paper Sec. 3.4, Fig. 3). All take n x n matrices in format fmt (device or
 * host memory, like bmlp_rms) and run on the given stream.
 *
 * bmlp_transpose - TRANSP: out = R^T, i.e. the relation with its arguments
 *     swapped (clauses such as p(X,Y) <- q(Y,X)).
 * bmlp_union - the union of two relations (two clauses with one head):
 *     out = A OR B.
 * bmlp_negate - NEG with the type literals of a stratified negation
 *     (p(X,Y) <- t(X), t(Y), not q(X,Y)): out[i][j] = rows(i) AND cols(j)
 *     AND NOT R[i][j]. rows and cols are packed bit vectors of ceil(n/64)
 *     uint64 words (the monadic type predicates, device or host memory); a
 *     null vector admits every constant.
 * out may alias an input for bmlp_union and bmlp_negate, not for
 * bmlp_transpose.
 */
bmlp_status bmlp_transpose(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, void* out,
                           cudaStream_t stream);
bmlp_status bmlp_union(bmlp_ctx* ctx, const void* A, const void* B, int64_t n, int32_t fmt, void* out,
                       cudaStream_t stream);
bmlp_status bmlp_negate(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, const uint64_t* rows,
                        const uint64_t* cols, void* out, cudaStream_t stream);

/*
 * bmlp_is_foreign - the composed program P3 u P4 u P5 of paper Sec. 3.4
 * (Fig. 3), in one call:
 *
 *     hasPlace          = contains+                          (BMLP-RMS)
 *     indirectlyPartOf  = (I + hasPlace^T) (adjoins OR adjoins^T)
 *                         (the recursion through hasPlace(Z,X) is a
 *                          composition with the transposed closure, Thm. 1)
 *     isForeign         = location x location AND NOT indirectlyPartOf
 *
 * contains, adjoins and out are n x n in format fmt; location is a packed
 * bit vector (ceil(n/64) uint64 words) or null for "every constant is a
 * location". The closure of contains runs with opts->variant (BMLP_AUTO: the
 * learned dispatcher when trained, else tensor cores); the composition runs
 * on the tensor cores for BMLP_RMS_TC / BMLP_SMP_TC and on packed rows
 * otherwise. iters_out (2 entries, may be null) receives the products of the
 * closure of contains and of the closure inside the composition.
 */
bmlp_status bmlp_is_foreign(bmlp_ctx* ctx, const void* contains, const void* adjoins, const uint64_t* location,
                            int64_t n, int32_t fmt, void* out, const bmlp_options* opts, int32_t* iters_out,
                            cudaStream_t stream);

/*
 * bmlp_mma_issue_rate - a measurement helper, not part of the paper's method:
 * the tensor-core FLOP rate of back-to-back tcgen05.mma instructions issued
 * by one CTA per SM from fixed shared-memory tiles (no operand traffic), so
 * that the squaring kernels can be compared with what this GPU issues.
 * kind 0: kind::f8f6f4, E4M3, M128 N256 K32 (the block-sparse squarings);
 * kind 1: kind::mxf4, E2M1 with unit UE8M0 scales, M128 N256 K64;
 * kind 2: the same as one M256 N256 K64 .cta_group::2 MMA per CTA pair (the
 * form of the dense squaring kernel). iters: MMA groups of 4 per CTA or pair
 * (e.g. 20000, about 5 ms). *tflops receives 2 M N K x MMAs / time.
 * kind 3: the integer ALU instead: 64-bit word ORs from registers by 8
 * warps per SM scheduler (the operation of the bit-row kernels); iters: 128
 * ORs per thread each (e.g. 20000); *tflops receives tera word-ORs per
 * second.
 * kind 4: the dense squaring kernel's exact MMA mix: per 64-deep K step one
 * M256 N256 K64 and one M256 N224 K64 .cta_group::2 kind::mxf4 MMA per CTA
 * pair (its 256 x 480 pair tile).
 * Runs on the legacy default stream and synchronises the device.
 */
bmlp_status bmlp_mma_issue_rate(bmlp_ctx* ctx, int32_t kind, int32_t iters, double* tflops);

/* One problem of a grouped batch. */
typedef enum bmlp_problem_kind {
    BMLP_PROBLEM_CLOSURE = 0,  /* out = R1+ (or I + R1+): program P2 of Sec. 3.3   */
    BMLP_PROBLEM_COMPOSE = 1   /* out = (I + R2+) R1: p <- r1 ; p <- r2, p (Thm. 1) */
} bmlp_problem_kind;

typedef struct bmlp_problem {
    int32_t kind;       /* bmlp_problem_kind                                      */
    int32_t fmt;        /* bmlp_format of R1, R2 and out                          */
    int32_t reflexive;  /* closures only: 1 gives I + R1+                         */
    int32_t variant;    /* closures only: 0 = the batch's choice, else
                           BMLP_RMS_TC, BMLP_RMS_PACKED or BMLP_SMP_PACKED
                           (every row by frontier expansion) for this problem */
    int64_t n;          /* matrix size (0 = nothing to do)                        */
    const void* R1;     /* device memory                                          */
    const void* R2;     /* device memory, compositions only                       */
    void* out;          /* device memory                                          */
} bmlp_problem;

/*
 * bmlp_batch_run - evaluate many independent linear recursive programs of
 * uneven sizes together (the grouped form of bmlp_rms / bmlp_compose; paper
 * Sec. 3.3-3.4, composability by reuse of outputs).
 *
 * All squaring steps of all unconverged problems of one iteration run in ONE
 * persistent launch over a device work list of (problem, tile) items; a
 * planner kernel retires problems whose changed flag stayed 0 (or that hit
 * their cap of ceil(log2 n) + 2 products) and builds the next work list; the
 * iteration runs inside a CUDA graph conditional WHILE node, so the host does
 * not take part until the whole batch has converged. Each problem runs on
 * the tensor cores or on packed rows, chosen per size bucket by the autotuner
 * (bmlp_batch_autotune) or forced by opts->variant (BMLP_RMS_TC /
 * BMLP_RMS_PACKED; compositions always use the tensor cores). Closures with
 * variant BMLP_SMP_PACKED (the problem's or the batch's) take no part in the
 * squaring loop: every row of every such closure is one query of a single
 * grouped frontier launch (Algorithm 2 from each constant), after grouped
 * launches that build their transposes and word indexes; their iteration
 * count is the deepest level + 1.
 * Problems large enough to fill the GPU alone (n >= 4096 by default, the
 * environment variable BMLP_BATCH_SOLO_N changes it, 0 = never) that are not
 * forced onto packed rows run in the same graph, one after another, as
 * device-driven single-problem pipelines: squarings on word-indexed bit rows
 * while the next one is predicted cheaper than a tensor-core product (a
 * one-thread decision kernel sets the condition of a WHILE node), then
 * squarings on packed E2M1 operands on the tensor cores (a second WHILE
 * node), then the decode or, for a composition, I + R2+ and the product with
 * R1. The whole batch is one graph launch and one read of the results
 * (bmlp_stats.host_syncs = 1).
 * iters_out (count entries, may be null) receives each problem's products.
 * All matrix pointers must be device memory. The instantiated graph is cached
 * in the context and reused while the problem list is unchanged.
 * Returns BMLP_ERR_NOT_CONVERGED if any problem hit its cap.
 */
bmlp_status bmlp_batch_run(bmlp_ctx* ctx, const bmlp_problem* probs, int64_t count, const bmlp_options* opts,
                           int32_t* iters_out, cudaStream_t stream);

/*
 * bmlp_batch_autotune - time the tensor-core and the packed engine on the
 * closures of `probs`, per size bucket (n rounded up to a power of two), and
 * keep the faster one per bucket in the context for later bmlp_batch_run
 * calls with variant BMLP_AUTO. When cache_path is not null the table is
 * read from that file if it holds an entry for this GPU, else measured and
 * written there (one line per GPU name and bucket).
 */
bmlp_status bmlp_batch_autotune(bmlp_ctx* ctx, const bmlp_problem* probs, int64_t count, const char* cache_path,
                                cudaStream_t stream);

/*
 * Learned dispatcher. Every variant returns the same bits; which is fastest
 * depends on the graph (Appendix C: squaring costs O(n^3 log n) whatever the
 * density, frontier expansion O(n^3) in the worst case but far less on sparse
 * inputs). A small MLP predicts the log2 run time (ms) of the four variants
 * from 16 features computed on the GPU, and BMLP_AUTO runs the argmin once a
 * model is trained or loaded (without one, BMLP_AUTO means BMLP_RMS_TC).
 *
 * Features (index: meaning): 0 log2 n; 1 log2(1 + nnz); 2 mean out-degree;
 * 3 std out-degree; 4 max out-degree / n; 5 fraction of empty rows; 6 std
 * in-degree and 7 max in-degree / n, 8 fraction of empty columns (estimated
 * from min(n, 1024) evenly spaced rows); 9 self-loop fraction; 10 reciprocity
 * of the sampled edges; 11 nonzero 64-bit words / all words; 12 mean |i - j|
 * / n of the sampled edges; 13 mean two-step probe reach / n; 14 log2 of the
 * probe growth from step one to step two; 15 fraction of probes whose second
 * step is empty. Probes: the first 64 sampled rows, second step = OR of up to
 * 64 rows of the first-step frontier.
 *
 * Network: 16 -> 64 -> 64 -> 4, ReLU, inputs normalised by (x - mu) / sigma
 * of the training features. Parameters (BMLP_MLP_PARAMS floats, this order):
 * W1[64][16], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]. Weights are used
 * in FP16 with FP32 accumulation; training keeps FP32 master weights (Adam).
 * Outputs are ordered BMLP_RMS_TC, BMLP_RMS_PACKED, BMLP_SMP_TC,
 * BMLP_SMP_PACKED. Loss: mean squared error of the log2 times, where a
 * censored time (the run hit its budget) only penalises predictions below it.
 */
#define BMLP_NFEAT 16
#define BMLP_NVAR 4
#define BMLP_MLP_PARAMS 5508

typedef struct bmlp_train_cfg {
    int32_t epochs;      /* passes over the training set                       */
    int32_t batch;       /* mini-batch size (0 = 256)                          */
    float lr;            /* Adam step size                                      */
    float weight_decay;  /* L2 added to the gradient                            */
    uint64_t seed;       /* initialisation and shuffling                       */
} bmlp_train_cfg;

/* The 16 features of an n x n matrix R (format fmt, device or host memory);
 * feats is a host array of BMLP_NFEAT floats. */
bmlp_status bmlp_dispatch_features(bmlp_ctx* ctx, const void* R, int64_t n, int32_t fmt, float* feats,
                                   cudaStream_t stream);

/* Train the network on m samples (host arrays): feats m x 16, log2_ms m x 4,
 * censored m x 4 (1 = that run hit its budget). Re-initialises the weights
 * from cfg->seed, sets the normalisation from feats, runs on the GPU and
 * leaves the model active. final_loss (may be null) gets the last epoch's
 * mean loss. */
bmlp_status bmlp_dispatch_train(bmlp_ctx* ctx, const float* feats, const float* log2_ms, const uint8_t* censored,
                                int64_t m, const bmlp_train_cfg* cfg, float* final_loss);

/* Predicted log2 ms (m x 4, may be null) and chosen bmlp_variant (m, may be
 * null) for m host feature rows. */
bmlp_status bmlp_dispatch_predict(bmlp_ctx* ctx, const float* feats, int64_t m, float* pred, int32_t* choice);

/* The batched form of bmlp_dispatch_features + bmlp_dispatch_predict: for m
 * matrices R[i] (n[i] x n[i], all in format fmt, each in device or host
 * memory), choice (m host ints) receives the predicted fastest bmlp_variant
 * and feats (m x 16 host floats, may be null) the features. The features of
 * every matrix and one prediction over all of them run on the GPU in stream
 * order, and the host waits once (bmlp_dispatch_features waits per matrix).
 * Packed device rows with an even word count and 16-byte alignment are read
 * in place; other matrices are converted into one workspace. Needs an active
 * model (trained, loaded or set): else BMLP_ERR_UNSUPPORTED. Errors:
 * BMLP_ERR_INVALID_ARG for m < 0, a null array with m > 0, a null R[i] or
 * n[i] <= 0, or a bad format. */
bmlp_status bmlp_dispatch_choose_many(bmlp_ctx* ctx, const void* const* R, const int64_t* n, int64_t m, int32_t fmt,
                                      int32_t* choice, float* feats, cudaStream_t stream);

/* Loss and gradient (BMLP_MLP_PARAMS floats) over m samples at the current
 * weights, computed by the training kernels' forward and backward code. */
bmlp_status bmlp_dispatch_loss_grad(bmlp_ctx* ctx, const float* feats, const float* log2_ms, const uint8_t* censored,
                                    int64_t m, float* loss, float* grad);

/* Set / get the FP32 parameters and the normalisation (mu, sigma: 16 each;
 * any pointer may be null). Setting marks the model active. */
bmlp_status bmlp_dispatch_set_params(bmlp_ctx* ctx, const float* params, const float* mu, const float* sigma);
bmlp_status bmlp_dispatch_get_params(bmlp_ctx* ctx, float* params, float* mu, float* sigma);

/* Save / load the model (binary: magic, sizes, mu, sigma, parameters). */
bmlp_status bmlp_dispatch_save(bmlp_ctx* ctx, const char* path);
bmlp_status bmlp_dispatch_load(bmlp_ctx* ctx, const char* path);

/*
 * bmlp_rms_tc_noalloc - the tensor-core closure of bmlp_rms (variant
 * BMLP_RMS_TC) for callers that must not allocate device memory. The paper
 * has no counterpart: this is a deployment form of the same computation.
 *
 * Who needs it: code whose device memory is owned by someone else (a pool
 * or caching allocator that has reserved the GPU, a plugin inside a host
 * framework with a fixed memory budget) and code on latency-critical paths
 * where cudaMalloc / cudaFree, which may synchronise the device, is not
 * acceptable. Such callers cannot create a bmlp_ctx, whose workspace grows
 * with cudaMalloc.
 *
 * Scratch: the ping-pong E4M3 R / R^T matrices and two control words live in
 * one file-scope __device__ array of 4 * 2048 * 2048 + 256 bytes (16 MiB),
 * which every GPU that loads this library holds until the process exits.
 * The call allocates nothing: no cudaMalloc, cudaFree or allocating library
 * routine.
 *
 * Arguments: as bmlp_rms, on the calling thread's current CUDA device. R and
 * out must be device memory of that device, or managed memory (host
 * pointers and other devices' memory give BMLP_ERR_INVALID_ARG, since
 * staging them would need an allocation). reflexive: 0 gives R1+, 1 gives
 * I + R1+. max_iters: 0 = ceil(log2 n) + 2. Sizes n > BMLP_NOALLOC_MAX_N give
 * BMLP_ERR_UNSUPPORTED. Errors are status codes only (there is no context to
 * hold a message).
 *
 * Set-up: each call looks up the scratch's device address
 * (cudaGetSymbolAddress, with the device current), so a context that was
 * torn down and recreated is followed. The first call on a device does the
 * set-up there (it loads the library's device code, which places the
 * scratch); make that first call before any stream capture on the device.
 * After each squaring the call copies the changed flag to the host and
 * synchronises `stream`.
 *
 * Sharing: every call on a device uses the same scratch, which keeps the last
 * call's contents (each call rewrites all of it that it reads). Calls whose
 * work overlaps on the GPU (other host threads, other streams) race on it:
 * serialise them.
 */
#define BMLP_NOALLOC_MAX_N 2048
bmlp_status bmlp_rms_tc_noalloc(const void* R, int64_t n, int32_t fmt, void* out, int32_t reflexive,
                                int32_t max_iters, int32_t* iters_out, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* BMLP_H */
