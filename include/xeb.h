/*
 * xeb.h -- C ABI of the GB300 multi-amplitude contraction library.
 *
 * The library computes the amplitudes <s_i|C|0^n> of a quantum circuit C for
 * a set of k bitstrings s_1..s_k by evaluating ONE contraction tree T of the
 * circuit's tensor network on k leaf assignments (Sec. "Multi-batch
 * simulator"), where every subtree T' is contracted once per distinct value
 * of the output bits it depends on (the memoization of Sec. "Multi-tensor
 * contraction algorithm", Fig. "main idea", Alg. 1-4).  Legs may be sliced
 * (App. A, "Slicing"): the contraction runs once per value of the sliced legs
 * and the results are summed in FP64.  The squared moduli are then folded
 * into the linear XEB F = 2^n/k sum_i |<s_i|C|0^n>|^2 - 1 (Eq. 1).
 *
 * General rules
 *  - Every function returns an xeb_status; nothing throws across the ABI.
 *    On a non-OK status xeb_last_error() returns a thread-local message.
 *  - The caller owns every array it passes in; the library copies what it
 *    keeps.  Pointers documented as "device" must be CUDA device pointers
 *    of the current device; "host" pointers are ordinary host memory.
 *  - Work is enqueued on the CUDA stream the caller passes (cudaStream_t cast
 *    to uintptr_t; 0 = legacy default stream).  Functions that return host
 *    results synchronise that stream.
 *  - Bitstrings: bit q of a uint64 word is qubit q's measured value (n <= 64).
 *  - Complex numbers are interleaved (re, im) pairs.
 *
 * Tensor-network convention (interface shared by every user of the tree and
 * slice formats):
 *  - one leaf per 2-qubit gate, numbered in time order;
 *  - a 1-qubit gate on q is fused into the output side of the latest 2-qubit
 *    gate on q before it; 1-qubit gates before the first 2-qubit gate on q
 *    act on |0> and that vector is contracted into the first 2-qubit gate's
 *    input for q;  a qubit without 2-qubit gates gets a rank-1 leaf appended
 *    after the gate leaves (qubit order);
 *  - bond legs are numbered in the order they are closed: at a 2-qubit gate
 *    on (qa, qb), first qa's incoming wire (if any), then qb's;
 *  - the open (output) leg of qubit q sits on the last leaf touching q; a leaf
 *    with two open legs lists them in its gate's qubit order.
 *  - Trees are lists of (left, right) pairs in post-order; a child c >= 0 is an
 *    earlier pair, c < 0 is leaf -1-c; the last pair is the root.
 *  - Output bits are ordered by an in-order walk of the tree (pi); a node's
 *    bits form a contiguous range of pi, read as a binary number with pi's
 *    first bit most significant; key ids are ranks of the distinct values in
 *    ascending order (App. C: variables numbered by position, lexicographic
 *    order of the index tuples).
 */
#ifndef XEB_H_
#define XEB_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    XEB_OK = 0,
    XEB_EINVAL = 1,        /* invalid argument (message says which)            */
    XEB_ENOMEM = 2,        /* device or host allocation failed / too small     */
    XEB_ECUDA = 3,         /* a CUDA runtime call failed                       */
    XEB_ETIMEOUT = 4,      /* a device-side bounded wait gave up               */
    XEB_EUNSUPPORTED = 5,  /* valid request the library does not support       */
    XEB_ECANCELLED = 6,    /* reserved: no call of this version returns it     */
    XEB_EDEVICE = 7        /* a device-side consistency check failed           */
} xeb_status;

/* Arithmetic of the pairwise contractions (Eq. elem-cont). */
enum {
    XEB_PREC_FP32 = 0,     /* plain FP32 complex FMA on CUDA cores             */
    XEB_PREC_TF32X3 = 1,   /* tcgen05 kind::tf32, big/small split, 4 products
                              (opts.split_terms), FP32 accumulate        */
    XEB_PREC_FP64 = 2      /* FP64 complex FMA on CUDA cores (checks)          */
};

/* Planner strategies (App. A objective f(T) picks among candidates). */
enum {
    XEB_PLANNER_AUTO = 0,
    XEB_PLANNER_GREEDY = 1,  /* memo-aware greedy pairwise merging             */
    XEB_PLANNER_SWEEP = 2,   /* time-ordered body of gate blocks + output trie */
    XEB_PLANNER_ANNEAL = 3   /* the best of the above refined by the local
                                search of App. A (tree rewrites + slicing
                                moves); AUTO also runs it when the constructed
                                trees needed slicing                          */
};

typedef struct {
    int n_qubits;
    int n_gates;
    const int32_t* kinds;  /* host [n_gates]: 1 = one-qubit gate, 2 = two-qubit */
    const int32_t* q0;     /* host [n_gates]                                     */
    const int32_t* q1;     /* host [n_gates]; ignored for one-qubit gates        */
    const double* mats;    /* host [n_gates][4][4] complex, row-major; a 2x2 gate
                              uses the top-left block; a 4x4 gate on (qa, qb) is
                              in the basis |b_a b_b> (qa's bit high)             */
} xeb_circuit;

typedef struct {
    int n_nodes;              /* = number of leaves - 1                          */
    const int32_t* children;  /* host [2*n_nodes], see the tree convention       */
} xeb_tree;

typedef struct {
    int n;                    /* number of sliced bond legs                      */
    const int32_t* legs;      /* host [n] bond-leg ids                           */
} xeb_slices;

typedef struct {
    int precision;        /* XEB_PREC_*                                          */
    int planner;          /* XEB_PLANNER_*                                       */
    int block_qubits;     /* sweep planner: max qubits per body block (0 = try)  */
    int group_leaves;     /* sweep planner: output leaves per trie level (0=try) */
    double alpha;         /* objective: arithmetic intensity alpha of
                             log2(C + alpha RW); 0 = use log2 of a time
                             estimate from a GB300 efficiency profile instead */
    double beta;          /* objective: memory penalty factor                    */
    uint64_t mem_budget;  /* M_max in bytes for the contraction arena            */
    uint64_t seed;        /* planner randomisation                               */
    int greedy_trials;    /* randomised greedy restarts                          */
    int reserved[8];      /* [0] = 1: permute operands into [free][summed] blocks
                             before each contraction instead of gathering them in
                             place; [1]: rounding of the leaves and folded
                             constants of a complex64 plan: 0 keeps each
                             tensor's norm (xeb_round_keep_norm), 1 rounds to
                             nearest; an FP64 plan with 1 or 2 takes those
                             complex64 values (the error the rounding alone
                             causes);
                             [2] = 1: launch kernels one by one instead of
                             replaying one captured CUDA graph per step;
                             [3] = 1: tensor-core contractions gather A with
                             plain loads even where TMA boxes could load it;
                             [4] = 1: memo-trie levels with long groups run as
                             grouped tensor-core GEMMs (default: the SIMT
                             memo-level kernel, faster for K = 16 tiles);
                             [5] = local-search proposals in thousands
                             (0: 2000 per leaf);
                             [6] = 1: keyed contractions (k_v > 1, 128+
                             rows, 16 <= K, N <= 64) use the keyed tensor-core
                             form by default (TF32x3 only; otherwise it is
                             one of the forms xeb_plan_autotune times);
                             [7] = 1: no cross-slice reuse (every contraction
                             runs in every slice; see xeb_plan_step_flops);
                             others 0 */
    int split_bits;       /* XEB_PREC_TF32X3: bits of the big part of each
                             operand, 8..11 (0 = 10).  Big parts of one state
                             row of a K-chunk (32 real values) and of one row of
                             W^T lie on a common grid of 2^-split_bits of that
                             group's largest magnitude, so the big*big sums are
                             exact in the FP32 accumulator (no truncation bias)
                             while they stay below 2^24 grid units            */
    int split_terms;      /* XEB_PREC_TF32X3: products per term, 3 (big*big,
                             big*small, small*big) or 4 (+ small*small);
                             0 = 4                                           */
    uint32_t timeout_ms;  /* limit of every device-side wait of the
                             tensor-core kernels (mbarrier hand-offs, copies);
                             a wait that runs out sets the plan's error word
                             and the call returns XEB_ETIMEOUT (0 = 2000)     */
    int fold_legs;        /* constant folding: a subtree that depends on no
                             output bit, sliced leg or open leg, and whose
                             tensors have at most fold_legs legs, is contracted
                             once on the host in FP64 when the plan is created
                             and its result is uploaded at bind, rounded like
                             the leaves (xeb_round_keep_norm); its leaves and
                             contractions never run on the device.  0 = 16,
                             -1 = no folding                                  */
} xeb_plan_opts;

typedef struct {
    int n_qubits, n_leaves, n_legs, n_nodes;
    int n_sliced;
    uint64_t k;                 /* bitstrings                                    */
    uint64_t k_distinct;        /* distinct bitstrings (root evaluations)        */
    double flops_per_slice;     /* 8 * sum_v k_v 2^(q_v + r_v)                    */
    double single_amp_flops;    /* 8 * k * sum_v 2^(q_v + r_v) (no memoization)  */
    double rw_elems_per_slice;  /* sum_v k_v (m(L) + m(R) + m(v))                 */
    double permute_elems_per_slice;  /* elements moved by layout permutations     */
    double objective;           /* f(T) of App. A                                 */
    uint64_t arena_bytes;       /* exact peak of the contraction arena (emulated) */
    uint64_t device_bytes;      /* total device memory the plan needs             */
    uint64_t n_slices;          /* 2^n_sliced                                     */
    int n_gemm_ops, n_permute_ops;
    int planner_used;
    int n_tc_launches;          /* tensor-core contractions per slice (after bind) */
    int n_tc_tma;               /* ... of which load A with TMA boxes             */
    int reserved[3];            /* [0]: nodes whose result is kept across slices
                                   (cross-slice reuse, see xeb_plan_step_flops);
                                   [1]: nodes evaluated on the host (constant
                                   folding, opts.fold_legs), leaves included;
                                   [2]: folded subtrees uploaded at bind      */
} xeb_stats;

/* Single-precision rounding that keeps the sum of squares (host only; the
 * library rounds every leaf tensor of a complex64 plan with it, real and
 * imaginary parts as 2m values).  x: host [n] doubles, y: host [n] floats
 * (caller-owned).  Every y[i] is one of the two floats nearest x[i]: first the
 * nearest, then, in order of increasing extra rounding error, a value moves
 * to its other neighbour whenever that brings sum_i y_i^2 closer to sum_i
 * x_i^2.  Why: the leaves are gate tensors (App. B, "leaf value tables")
 * whose squared norm is fixed by unitarity; nearest rounding of the fused
 * gates of these circuits shrinks it systematically, and the circuit's
 * output norm with it (a shift of a few 1e-7 in F at 20-30 qubits).  NULL
 * pointers: no effect. */
void xeb_round_keep_norm(const double* x, size_t n, float* y);

/* Default options (FP32, AUTO planner, 64 GiB budget). */
void xeb_default_opts(xeb_plan_opts* opts);

/* Leaf/leg counts of the circuit's tensor network (convention above). */
xeb_status xeb_network_info(const xeb_circuit* circuit, int* n_leaves, int* n_legs);

/* Per leaf: its output qubits (out_bits[2*j..2*j+1], -1 padded) and bond legs
 * (legs[4*j..4*j+3], -1 padded).  Host arrays of 2*n_leaves and 4*n_leaves. */
xeb_status xeb_network_leaves(const xeb_circuit* circuit, int32_t* out_bits, int32_t* legs);

/* Build a plan (host only; touches no GPU).  bitstrings: host [k].  tree and
 * slices may be NULL, then the planner chooses them by the objective
 * f(T) = beta*max(log2(M/M_max), 0) + log2(C + alpha*RW) (App. A).  The plan
 * evaluates exactly these k bitstrings (exact evaluation counts k_v). */
xeb_status xeb_plan_create(const xeb_circuit* circuit, const uint64_t* bitstrings, size_t k,
                           const xeb_tree* tree, const xeb_slices* slices,
                           const xeb_plan_opts* opts, struct xeb_plan_s** out);

/* Multi-batch plan (Sec. "Multi-batch simulator"): the output legs of the
 * qubits set in open_mask (bit q = qubit q) are not contracted, so every
 * input bitstring stands for the batch of 2^w bitstrings (w = popcount of
 * open_mask, 1 <= w <= 16, w < n) that share its other bits; its open bits are
 * ignored.  xeb_amplitudes then writes k x 2^w complex128 values,
 * out[i * 2^w + x] = <s_i with the open qubits set to x | C | 0^n>, where bit j
 * of x is the j-th open qubit in ascending order; xeb_fidelity's F, mean of
 * 2^n p and mean of (2^n p)^2 run over those k 2^w values (Eq. 1 over the
 * batches' bitstrings).  The network is the one of xeb_network_leaves with
 * each open qubit's output bit turned into a leg of its own (ids n_legs ..
 * n_legs + w - 1, ascending qubit order; bond legs keep their ids), so trees
 * and slices of the plain network apply; an open leg cannot be sliced
 * (XEB_EINVAL).  Other arguments, ownership and errors as xeb_plan_create;
 * XEB_EINVAL for an open qubit >= n, XEB_EUNSUPPORTED for w > 16 or w = n. */
xeb_status xeb_plan_create_batched(const xeb_circuit* circuit, const uint64_t* bitstrings, size_t k,
                                   uint64_t open_mask, const xeb_tree* tree, const xeb_slices* slices,
                                   const xeb_plan_opts* opts, struct xeb_plan_s** out);

void xeb_plan_destroy(struct xeb_plan_s* plan);

/* Statistics of a plan (host only). */
xeb_status xeb_plan_stats(struct xeb_plan_s* plan, xeb_stats* out);

/* The chosen tree (host [2*(n_leaves-1)]) and slices (host [n_sliced]). */
xeb_status xeb_plan_tree(struct xeb_plan_s* plan, int32_t* children, int32_t* sliced_legs);

/* Exact evaluation count k_v and pi-range [a, b) of internal node `node`
 * (host only); counts come from the plan's bitstrings. */
xeb_status xeb_plan_node(struct xeb_plan_s* plan, int node, int64_t* kv, int32_t* a,
                         int32_t* b, int32_t* n_legs, int32_t* n_shared);

/* Device memory the plan needs (bytes) for xeb_plan_bind.  Tensor sizes
 * saturate at 2^48 elements, so a plan with a wider intermediate reports a
 * huge but finite size (below 2^62) and xeb_plan_bind refuses it with
 * XEB_ENOMEM before touching the device. */
size_t xeb_plan_device_bytes(struct xeb_plan_s* plan);

/* Attach device memory and upload the plan's constant tables on `stream`.
 * workspace: device pointer of >= xeb_plan_device_bytes() bytes owned by the
 * caller (kept until destroy), or NULL to let the library allocate it. */
xeb_status xeb_plan_bind(struct xeb_plan_s* plan, void* workspace, size_t bytes,
                         uintptr_t stream);

/* Copy `k` bitstrings from device memory into the plan (k must equal the
 * plan's k, and the bitstrings must give the plan's counts -- a mismatch is
 * reported as XEB_EDEVICE by xeb_fidelity).  The memo key tables (a1: the key
 * id of each bitstring per node, the children's key ids (uL, uR) of each key)
 * are rebuilt on the device by the next xeb_amplitudes / xeb_plan_keys. */
xeb_status xeb_set_bitstrings(struct xeb_plan_s* plan, const uint64_t* bitstrings_dev,
                              size_t k, uintptr_t stream);

/* One step: build the key tables of the current bitstrings (a1), contract
 * every slice (a2..a6) and write the k amplitudes, in input order, as
 * complex128 to device memory out_dev [2*k doubles; 2*k*2^w for a
 * multi-batch plan, see xeb_plan_create_batched] (NULL: the plan's own
 * buffer), plus the XEB sums (a7).  The first call per output pointer
 * captures the step as a CUDA graph on a private stream; later calls replay
 * it on `stream` (not while profiling, or with opts.reserved[2] = 1). */
xeb_status xeb_amplitudes(struct xeb_plan_s* plan, double* out_dev, uintptr_t stream);

/* Restrict the slice loop of xeb_amplitudes to a seeded subset of the
 * 2^|S| slice values (App. A, "Slicing": an amplitude is the sum over all
 * values of the sliced legs; a subset gives a partial sum -- not an
 * amplitude -- used to time and check plans whose full sum takes too long).
 * The subset holds max(1, round(frac * 2^|S|)) values: the first ones of a
 * partial Fisher-Yates shuffle of 0 .. 2^|S|-1 whose draws are successive
 * outputs of splitmix64 started at `seed` (draw j uses x mod (2^|S| - j)).
 * frac >= 1 restores the full sum.  *n_chosen (may be NULL) receives the
 * subset size; XEB_EINVAL for frac <= 0 or a subset above 2^26 values.  The
 * next xeb_amplitudes call recaptures its graph. */
xeb_status xeb_set_slice_subset(struct xeb_plan_s* plan, double frac, uint64_t seed, int64_t* n_chosen);

/* Restrict the slice loop to a contiguous block of slice values, for ranks
 * that share one sum over slices (App. A, "Slicing": the values of the sliced
 * legs are independent terms, contracted apart and added at the end).  The
 * loop runs positions lo .. hi-1 of the list xeb_set_slice_subset(frac, seed)
 * would choose (frac >= 1: all 2^|S| values in counting order), in that order;
 * xeb_amplitudes then writes the FP64 partial sums over those values (not
 * amplitudes; the ranks' partial sums add up to the amplitudes, and an empty
 * block gives zeros).  Blocks [lo_r, hi_r) that tile [0, n) give every value
 * to exactly one rank.  *n_chosen (may be NULL) receives hi - lo; XEB_EINVAL
 * for frac <= 0, lo < 0, hi < lo, hi beyond the list or a block above 2^26
 * values.  Host only; the next xeb_amplitudes call recaptures its graph. */
xeb_status xeb_set_slice_block(struct xeb_plan_s* plan, double frac, uint64_t seed, int64_t lo, int64_t hi,
                               int64_t* n_chosen);

/* The slice values the loop runs, in loop order (the block's or the
 * subset's, else all 0 .. 2^|S|-1); ids needs room for the count
 * xeb_set_slice_block / xeb_set_slice_subset returned (2^|S| without
 * either).  Bit b of a value is the value of sliced leg b in
 * the order xeb_plan_tree reports the sliced legs. */
xeb_status xeb_plan_slice_ids(const struct xeb_plan_s* plan, int64_t* ids);

/* Linear XEB of the last xeb_amplitudes call (Eq. 1): F, mean of 2^n p and
 * mean of (2^n p)^2 over the sequence; host outputs; synchronises. */
xeb_status xeb_fidelity(struct xeb_plan_s* plan, double* F, double* mean_2np,
                        double* mean_2np_sq, uintptr_t stream);

/* End to end from host memory: copy bitstrings_host [k] (pinned for async
 * speed) to the device, build key tables, contract, copy amplitudes
 * [2*k doubles; 2*k*2^w for a multi-batch plan] and F to host.
 * Synchronises. */
xeb_status xeb_run(struct xeb_plan_s* plan, const uint64_t* bitstrings_host, size_t k,
                   double* amps_host, double* F_host, uintptr_t stream);

/* Streamed evaluation for bitstring sets whose key tables and arena would
 * not fit at once, in the lexicographic order of Alg. 4.  Without a tree the
 * planner plans the first min(chunk, k) input bitstrings (a sample of the
 * set); the bitstrings are then sorted by their bits read in that tree's bit
 * order pi (first bit most significant), so neighbours share the longest key
 * prefixes, and evaluated `chunk` at a time with the same tree and slices
 * (slices NULL: the planner's, chosen on the sample).  The library allocates
 * one workspace, grown to the largest chunk's xeb_plan_device_bytes, and
 * frees it before returning; memory scales with the chunk, not with k.  A key
 * prefix shared by two chunks is contracted once in each.  Outputs (host,
 * each may be NULL): amps_host [2*k doubles] in input order, and over all k
 * bitstrings F, the mean of 2^n p and the mean of (2^n p)^2 (Eq. 1).
 * XEB_EINVAL for k = 0, chunk = 0 or a NULL bitstring pointer;
 * XEB_EUNSUPPORTED for chunk above 2^24 or k above 2^32 - 1; errors of xeb_plan_create and
 * xeb_run otherwise.  Synchronises `stream`. */
xeb_status xeb_run_chunked(const xeb_circuit* circuit, const uint64_t* bitstrings_host, size_t k,
                           const xeb_tree* tree, const xeb_slices* slices, const xeb_plan_opts* opts,
                           size_t chunk, double* amps_host, double* F_host, double* mean_2np_host,
                           double* mean_2np_sq_host, uintptr_t stream);

/* Copy node `node`'s device key tables to host (for checks): key_of_bitstring
 * [k] int32, uL [k_v], uR [k_v] int32 (any may be NULL).  Synchronises. */
xeb_status xeb_plan_keys(struct xeb_plan_s* plan, int node, int32_t* key_of_bitstring,
                         int32_t* uL, int32_t* uR, uintptr_t stream);

/* Kernel classes reported by xeb_plan_profile_read. */
enum {
    XEB_KC_TRIE = 0,          /* a1 key tables                                   */
    XEB_KC_LEAVES = 1,        /* a2 leaf projection                              */
    XEB_KC_PERMUTE = 2,       /* a3 leg permutation                              */
    XEB_KC_GEMM_TILED = 3,    /* a4 FP32/FP64 SIMT tiled complex GEMM            */
    XEB_KC_GEMM_GEMV = 4,     /* a4 grouped matrix-vector (memo trie levels)     */
    XEB_KC_GEMM_TAIL = 5,     /* a5 warp-per-key dot products                    */
    XEB_KC_GEMM_GENERIC = 6,  /* a4 small contractions                           */
    XEB_KC_ACCUM = 7,         /* a6 FP64 accumulation over slices                */
    XEB_KC_XEB = 8,           /* a7 gather + linear XEB                          */
    XEB_KC_GEMM_TC = 9,       /* a4 tcgen05 split-precision complex GEMM         */
    XEB_KC_GEMM_STREAM = 10,  /* a4 memory-bound streaming contraction (SIMT)    */
    XEB_KC_GEMM_MEMO = 11,    /* a4 memo-trie levels: keys grouped by left key   */
    XEB_KC_GEMM_KDEEP = 12,   /* a4 keyed contractions with a deep summed index  */
    XEB_KC_GEMM_TC_KDEEP = 13, /* a4 the same on tcgen05, split precision       */
    XEB_KC_GEMM_KEYED = 14,   /* a4 keyed, few summed values, narrow results   */
    XEB_N_KC = 16
};

/* Enable (1) or disable (0) per-launch CUDA-event timing of the plan's
 * kernels on the stream they are launched on (adds two event records per
 * launch; host only otherwise).  Enabling resets the accumulated totals. */
xeb_status xeb_plan_profile(struct xeb_plan_s* plan, int enable);

/* Per contraction of the plan's program (in program order): accumulated
 * device milliseconds and launches since profiling was enabled, its kernel
 * class (XEB_KC_*, -1 before xeb_plan_bind) and its shape (M, N, K, k_v as
 * doubles, [n][4]).  Writes min(cap, n) entries of each non-NULL host array;
 * *n_ops receives n.  Synchronises on the recorded events. */
xeb_status xeb_plan_profile_ops(struct xeb_plan_s* plan, int cap, double* ms, double* launches, int32_t* cls,
                                double* shape, int32_t* n_ops);

/* Kernel form of contraction step op_index of a bound plan (the fixed rule's,
 * or the autotuner's choice after xeb_plan_autotune); host only.  Writes five
 * values to form: [0] kernel class (XEB_KC_*); [1] rows per lane of the keyed
 * SIMT kernel; [2] result columns per thread and [3] rows per tile of the
 * streaming kernel; [4] 1 when the tensor-core kernel loads A with TMA boxes
 * (entries that do not apply to the kernel are 0).  XEB_EINVAL for a NULL plan
 * or form, an unbound plan, or an index that is not a contraction step. */
xeb_status xeb_plan_op_form(const struct xeb_plan_s* plan, int op_index, int32_t* form);

/* Work of one xeb_amplitudes step over the slices it runs (all, or the
 * subset of xeb_set_slice_subset), with cross-slice reuse: a node whose
 * subtree holds sliced legs S_v is contracted only in the slices where a leg
 * of S_v (or, for a node recomputed with its parent, of the parent's set)
 * changed value from the previous slice, so slice-invariant subtrees run once
 * (the sharing of common subexpressions across slices that the paper's
 * introduction cites, applied to the slice loop of App. A "Slicing").  Writes
 * the algorithmic flops (8 per complex multiply-add) and the number of
 * contractions launched per step; either pointer may be NULL.  Host only. */
xeb_status xeb_plan_step_flops(const struct xeb_plan_s* plan, double* flops, double* contractions);

/* Per tree node v (leaves 0 .. n_leaves-1, then internal nodes in post-order;
 * host only): the arena placement of its tensor from the emulation-mode
 * allocator -- element offset off[v] and size elems[v] (complex elements) --
 * and the cross-slice mask[v]: the slice bits whose change makes the node be
 * contracted again (all ones without reuse).  Arrays of *n_nodes entries, any
 * may be NULL; call with all NULL to read *n_nodes first. */
xeb_status xeb_plan_buffers(const struct xeb_plan_s* plan, int64_t* off, int64_t* elems, uint32_t* mask,
                            int32_t* n_nodes);

/* Operand and result addressing of step `op_index` of the plan's contraction
 * program (host only; the program of App. A/C's tree, one step per
 * contraction or permutation).  Writes min(cap, n) int32 values to out (may be
 * NULL) and n to *n_out: kind (1 permute, 2 contraction), node, A node, B
 * node, then the lengths of the six lists a_pos_m, a_pos_k, b_pos_k, b_pos_n,
 * c_pos_m, c_pos_n, then the lists themselves.  Entry i of a list is the
 * address bit (legs have dimension 2) of bit i of the row (m), summed (k) or
 * column (n) index in operand A, B or the result C.  XEB_EINVAL for a NULL
 * plan or n_out, or an index outside the program. */
xeb_status xeb_plan_op_layout(const struct xeb_plan_s* plan, int op_index, int32_t* out, int cap, int32_t* n_out);

/* Accumulated totals per kernel class since profiling was enabled: device
 * milliseconds, launches, algorithmic flops (8 per complex multiply-add) and
 * algorithmic bytes (each operand tensor read once, each result written
 * once).  Each output is a host array of XEB_N_KC doubles (may be NULL).
 * Synchronises on the recorded events. */
xeb_status xeb_plan_profile_read(struct xeb_plan_s* plan, double* ms, double* launches, double* flops,
                                 double* bytes);

/* ---- learned cost model ------------------------------------------------
 * Candidates of the planner for a circuit and bitstring set: every tree the
 * planner would weigh (greedy restarts, sweep family) with the slice set its
 * slicing step gives it, and XEB_N_FEATURES features per candidate (exact
 * counter totals over slices, the hand time model, per kernel class counts,
 * bytes and flops).  Writes up to max_cands candidates: trees as
 * [max_cands][n_leaves-1][2] (post-order pairs, as xeb_tree), slices as
 * [max_cands][30] (-1 padded), n_sliced, features [max_cands][XEB_N_FEATURES]
 * and the planner family (XEB_PLANNER_*); any output may be NULL.  n_out
 * receives the number written.  Host only. */
#define XEB_N_FEATURES 32
xeb_status xeb_plan_candidates(const xeb_circuit* circuit, const uint64_t* bitstrings, size_t k,
                               const xeb_plan_opts* opts, int max_cands, int32_t* trees, int32_t* slices,
                               int32_t* n_sliced, double* features, int32_t* planner, int32_t* n_out);

/* The model: n_layers hidden ReLU layers of n_hidden units and one linear
 * output, predicting log2 of the step time from the features.  Parameters,
 * gradients and Adam moments live on the device; parameters are laid out
 * layer by layer as W_l (out x in, row-major) then b_l.  Inputs are
 * normalised as (x - mean) * scale with xeb_mlp_set_norm.  Inputs and targets
 * are float32 device arrays ([n][n_in], [n]).  Forward/train run on
 * `stream`; xeb_mlp_gradients (mean squared error gradients to host, for
 * checks) synchronises it. */
struct xeb_mlp_s;
xeb_status xeb_mlp_create(int n_in, int n_hidden, int n_layers, uint64_t seed, struct xeb_mlp_s** out);
void xeb_mlp_destroy(struct xeb_mlp_s* mlp);
size_t xeb_mlp_n_params(struct xeb_mlp_s* mlp);
xeb_status xeb_mlp_weights(struct xeb_mlp_s* mlp, float* host, int set);   /* set = 1: upload, 0: download */
xeb_status xeb_mlp_set_norm(struct xeb_mlp_s* mlp, const float* mean, const float* scale);
xeb_status xeb_mlp_forward(struct xeb_mlp_s* mlp, const float* x_dev, int n, float* y_dev, uintptr_t stream);
xeb_status xeb_mlp_gradients(struct xeb_mlp_s* mlp, const float* x_dev, const float* t_dev, int n,
                             float* grad_host, float* loss_host, uintptr_t stream);
xeb_status xeb_mlp_train_step(struct xeb_mlp_s* mlp, const float* x_dev, const float* t_dev, int n, float lr,
                              float* loss_dev, uintptr_t stream);   /* one Adam step; loss_dev may be NULL */

/* The planner with the learned cost model (the paper's planner has no learned
 * part; here the model re-ranks the plain planner's candidates): builds up to
 * max_cands candidate trees and slice sets (xeb_plan_candidates, with opts),
 * predicts their step time with `model` (xeb_mlp_forward on `stream`, the
 * project's own inference kernels, on the candidates' XEB_N_FEATURES features
 * rounded to float) and creates the plan of the fastest-predicted candidate,
 * as xeb_plan_create would with that tree and slice set.  With no candidate it
 * falls back to the plain planner (xeb_plan_create with no tree).  The
 * candidates are not timed here: timing the best few against the plain plan
 * is the caller's choice (the Python `costmodel.choose_verified`).
 * *predicted_log2_ms (may be NULL) receives the model's prediction for the
 * chosen candidate (NaN for the fallback).  XEB_EINVAL for a NULL circuit,
 * bitstrings, model or out or max_cands < 1; errors of the calls it makes are
 * passed on.  Allocates two small device buffers and synchronises `stream`. */
xeb_status xeb_plan_create_learned(const xeb_circuit* circuit, const uint64_t* bitstrings, size_t k,
                                   const xeb_plan_opts* opts, struct xeb_mlp_s* model, int max_cands,
                                   uintptr_t stream, double* predicted_log2_ms, struct xeb_plan_s** out);

/* Autotuner (the plan's own form of "tile shapes picked by an autotuner"):
 * runs one step to fill the operands, then for every contraction times each
 * kernel form and tile shape that fits it -- tcgen05 with TMA loads, tcgen05
 * with gathered loads (also per key of a keyed contraction), grouped tcgen05
 * (memo levels), deep-K tcgen05, SIMT streaming with its default tile, with
 * two result columns per thread (a warp stores whole result rows) and with
 * half the rows per tile, keyed SIMT with one or two rows per lane (also for
 * single-key contractions) -- `reps` times with CUDA events on `stream`, and
 * keeps the fastest.  Later steps use (and recapture) the chosen forms.
 * Synchronises `stream`.  n_changed (may be NULL): contractions whose form
 * changed. */
xeb_status xeb_plan_autotune(struct xeb_plan_s* plan, int reps, uintptr_t stream, int32_t* n_changed);

/* Linear XEB of k complex128 amplitudes already in device memory (amps_dev,
 * 2*k doubles): writes F, the mean of 2^n p and the mean of (2^n p)^2 to
 * out_dev (3 doubles, device) on `stream`, asynchronously, and allocates
 * nothing.  The paper has no counterpart.  It exists for callers that cannot
 * allocate device memory: a process whose device memory belongs to its own
 * pool allocator (cudaMalloc there fails or competes with the pool), or a
 * latency-critical caller that cannot take the implicit device
 * synchronisation of an allocation.  Its block partial sums live in a fixed
 * array inside the library (64 KiB on every device that loads the library,
 * held until the process exits), which limits k to 16,777,216; larger k
 * returns XEB_EINVAL.  The first call on a device looks up that array's
 * device address (with the device current); make that first call before any
 * stream capture.  All calls share the array, so calls whose kernels overlap
 * on the GPU race.  amps_dev must be 16-byte aligned (each amplitude is read as
 * one 16-byte value; a torch complex128 tensor's storage is); a pointer that is
 * not is refused with XEB_EINVAL before anything is launched, and so are NULL
 * pointers and n_qubits outside [1, 64]. */
xeb_status xeb_linear_xeb_noalloc(const double* amps_dev, size_t k, int n_qubits, double* out_dev,
                                  uintptr_t stream);

/* Testing aid for the bounded waits (not part of the paper's method): with
 * enable != 0 every tensor-core contraction of the plan first waits on a
 * barrier that nothing completes, so that wait runs out after opts.timeout_ms;
 * the kernel records the timeout in the plan's error word, its threads leave
 * their loops (copies in flight drained, MMAs finished, tensor memory freed)
 * and the next xeb_fidelity / xeb_run returns XEB_ETIMEOUT.  enable = 0
 * restores normal steps (the error word is cleared once it is reported).
 * Host only; the next xeb_amplitudes call recaptures its graph.  XEB_EINVAL
 * for a NULL plan. */
xeb_status xeb_plan_test_wait(struct xeb_plan_s* plan, int enable);

/* Thread-local message of the last failure in this thread. */
const char* xeb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* XEB_H_ */
