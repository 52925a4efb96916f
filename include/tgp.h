/*
 * tgp.h -- C ABI of the GB300 (sm_103a) library for population-wide fitness
 * evaluation of tensorized tree-based genetic programming.
 *
 * Method: arXiv 2501.17168 ("EvoGP").  The population is the paper's three
 * NaN-padded tensors (Sec. III-A): node types, node values and subtree sizes,
 * each [pop, max_len] row-major.  Each tree is interpreted over every data
 * point (Sec. II-A node semantics; Sec. III-C evaluation of the prefix
 * encoding) and reduced to a mean squared error against the targets
 * (Sec. III-C, symbolic-regression fitness).  Multi-output trees use Modi
 * nodes (Sec. IV-C).  Reverse-mode gradients and the batched persistent
 * launch are additions of this library; the paper has no counterpart.
 *
 * Encoding of one node (the paper leaves the codes open; this is the
 * library's fixed reading):
 *   type  0 variable, 1 constant, 2 unary function, 3 binary function,
 *         4 ternary function; 18 / 19 / 20 are unary / binary / ternary Modi
 *         function nodes (16 + 2, 16 + 3, 16 + 4).
 *   value variable: feature index (integer in [0, n_features));
 *         constant: the constant (finite);
 *         function: func_id + 256 * out_index, an integer below 65536, where
 *         out_index (Modi nodes only, 0 on plain nodes) is in [0, n_outputs).
 *   size  the subtree size; size[0] is the tree length len (1..max_len).
 *   Entries at positions >= len are never read.
 * Functions (first prefix child = left operand):
 *   0 add, 1 sub, 2 mul, 3 pdiv(a,b) = |b| > 1e-6f ? a/b : 1,
 *   4 max (IEEE fmax), 5 sin, 6 cos, 7 plog(a) = |a| > 1e-6f ? log|a| : 0,
 *   8 cexp(a) = exp(min(a, 80)), 9 tan, 10 ite(a, b, c) = a > 0 ? b : c (a NaN
 *   condition selects c; the only ternary function).
 * Outputs: with n_outputs == 1 and no Modi node in the tree the output is the
 * root value; otherwise output k is the sum of the function values of the
 * Modi nodes tagged k (0 if none), and a Modi node hands its parent the value
 * of its rightmost child (c for ite).
 *
 * Conventions for every entry point:
 *   - Pointers marked [device] are CUDA device memory owned by the caller;
 *     [host] pointers are host memory owned by the caller.
 *   - The library never allocates, frees or synchronizes.  All work is
 *     enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and
 *     is asynchronous; the calls are legal inside CUDA stream capture.
 *   - Scratch memory is the caller's workspace `ws` of `ws_bytes` bytes
 *     ([device], 256-byte aligned), sized by tgp_workspace_size for the same
 *     arguments.  It may be reused by the next call on the same stream.
 *   - Argument errors (null pointer, bad size, short workspace, unsupported
 *     shape) are returned synchronously and nothing is launched.
 *   - Per-tree problems found on the device are reported in tree_status
 *     (bitmask below); that tree's outputs, MSE and gradients are NaN and the
 *     call still returns TGP_OK.
 *   - Computation is FP32; the per-tree MSE is accumulated in FP64.
 */
#ifndef TGP_H
#define TGP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TGP_OK = 0,
  TGP_ERR_INVALID_ARG = 1,  /* null pointer, negative or inconsistent size   */
  TGP_ERR_INVALID_TREE = 2, /* reserved: trees are reported per tree          */
  TGP_ERR_WORKSPACE = 3,    /* ws null, misaligned or smaller than required  */
  TGP_ERR_CUDA = 4,         /* a CUDA runtime call failed (launch, attribute) */
  TGP_ERR_TIMEOUT = 5,      /* reported by tgp_check_device_error            */
  TGP_ERR_UNSUPPORTED = 6   /* shape beyond the library limits               */
} tgp_status;

/* Per-tree status bits (Sec. III-A encoding rules). */
enum {
  TGP_TREE_OK = 0,
  TGP_TREE_LEN = 1,     /* size[0] not an integer in [1, max_len]                 */
  TGP_TREE_TYPE = 2,    /* a type code not in {0,1,2,3,4,18,19,20}               */
  TGP_TREE_FUNC = 4,    /* function id unknown, arity disagrees with the type,
                           or an output index on a plain function node           */
  TGP_TREE_VAR = 8,     /* variable index not an integer in [0, n_features)      */
  TGP_TREE_MODI = 16,   /* Modi output index not in [0, n_outputs)               */
  TGP_TREE_CONST = 32,  /* constant not finite                                   */
  TGP_TREE_SIZE = 64,   /* subtree sizes disagree with the prefix structure      */
  TGP_TREE_DEPTH = 128, /* nests deeper than the evaluation registers and stack
                           hold (never for trees of up to 1024 nodes without
                           ite), or more than 8 ite nodes whose branches are
                           pending at once (ite nested in ite branches)        */
  TGP_TREE_NO_ADJOINT = 256 /* tgp_eval_backward only: the tree has an ite node,
                           which the adjoint does not differentiate; its MSE
                           and gradients are NaN                               */
};

/* Library limits. */
#define TGP_MAX_LEN 1024       /* largest supported max_len                */
#define TGP_MAX_OUTPUTS 16     /* largest supported n_outputs              */
#define TGP_MAX_FEATURES 256   /* largest supported n_features             */

/* The paper's population tensors P_type, P_val, P_size (Sec. III-A). */
typedef struct tgp_population {
  const float* type;  /* [device] [pop, ld]                                  */
  const float* value; /* [device] [pop, ld]                                  */
  const float* size;  /* [device] [pop, ld]                                  */
  int64_t pop;        /* number of trees P >= 0                              */
  int32_t max_len;    /* |T|_max, 1..TGP_MAX_LEN                             */
  int64_t ld;         /* row stride in elements, ld >= max_len               */
} tgp_population;

/* Feature matrix X [n_points, n_features] row-major with row stride ldx. */
typedef struct tgp_data {
  const float* X;     /* [device]                                            */
  int64_t n_points;   /* D >= 0                                              */
  int32_t n_features; /* F, 1..TGP_MAX_FEATURES                              */
  int64_t ldx;        /* row stride in elements, ldx >= n_features           */
} tgp_data;

/* Launch shape of the evaluation kernels and call options.  Zero fields take
 * the library's heuristic and defaults; the autotuner fills the shape fields
 * from measurements. */
typedef struct tgp_config {
  int32_t trees_per_block;  /* trees staged together in shared memory (1..64) */
  int32_t points_per_tile;  /* points of X staged per tile; a multiple of
                               32 * points_per_lane (up to 4096)              */
  int32_t tiles_per_item;   /* consecutive tiles one work item sweeps         */
  int32_t points_per_lane;  /* 4 or 8 points evaluated per thread             */
  void* eval_begin_event;   /* optional cudaEvent_t recorded on the stream just
                               before the evaluation kernel(s), NULL = none  */
  void* eval_end_event;     /* optional cudaEvent_t recorded just after them  */
  int32_t flags;            /* TGP_FLAG_* bits, 0 = none                     */
  int32_t max_wait_polls;   /* limit of the bounded wait for the program
                               copies: 0 = the library default (about 4 M
                               polls, seconds); a negative value gives up at
                               once, which drives the TGP_ERR_TIMEOUT path
                               (tgp_check_device_error) without a fault      */
  int32_t cta_width;        /* 0 = the library's choice; 1 = CTAs of 8 warps,
                               several per SM; 2 = one wide CTA per SM (32
                               warps for the single-output kernel at 8 points
                               per lane, 28 for the Modi kernel, narrower
                               where shared memory does not hold it) whose
                               warps share one X tile and program area; other
                               values are TGP_ERR_INVALID_ARG                */
} tgp_config;

/* tgp_config.flags bits. */
#define TGP_FLAG_SSE 1  /* MSE calls write the FP64 sum of squared residuals
                           over this call's points instead of dividing it
                           by n_points: the partial sums of a data set
                           split by points across calls or ranks add up to
                           D_total * MSE of the whole set (Sec. III-C
                           fitness, sharded by points), and the caller
                           divides once by D_total                        */

/* Bytes of workspace the calls below need for these arguments (0 on invalid
 * arguments).  cfg may be NULL. */
size_t tgp_workspace_size(const tgp_population* pop, const tgp_data* data, int32_t n_outputs,
                          const tgp_config* cfg);

/* Validates every tree (Sec. III-A rules) and writes tree_status [device]
 * [pop] int32.  Also compiles the trees into the workspace. */
tgp_status tgp_validate(const tgp_population* pop, int32_t n_features, int32_t n_outputs,
                        int32_t* tree_status, void* ws, size_t ws_bytes, void* stream);

/* Forward outputs (Sec. II-A, Sec. IV-C): out [device] float [pop, n_outputs,
 * n_points]; tree_status [device] int32 [pop] or NULL. */
tgp_status tgp_eval_forward(const tgp_population* pop, const tgp_data* data, int32_t n_outputs,
                            float* out, int32_t* tree_status, void* ws, size_t ws_bytes,
                            void* stream);
tgp_status tgp_eval_forward_cfg(const tgp_population* pop, const tgp_data* data,
                                int32_t n_outputs, float* out, int32_t* tree_status, void* ws,
                                size_t ws_bytes, void* stream, const tgp_config* cfg);

/* SR fitness (Sec. III-C): mse [device] double [pop, n_outputs] with
 * mse[p,k] = (1/D) sum_d (o_k(x_d) - y[d,k])^2; y [device] float
 * [n_points, n_outputs] row-major (contiguous).  n_points must be >= 1. */
tgp_status tgp_fitness_mse(const tgp_population* pop, const tgp_data* data, const float* y,
                           int32_t n_outputs, double* mse, int32_t* tree_status, void* ws,
                           size_t ws_bytes, void* stream);
tgp_status tgp_fitness_mse_cfg(const tgp_population* pop, const tgp_data* data, const float* y,
                               int32_t n_outputs, double* mse, int32_t* tree_status, void* ws,
                               size_t ws_bytes, void* stream, const tgp_config* cfg);

/* One SR problem of a batch: its population, data, targets and outputs. */
typedef struct tgp_problem {
  tgp_population pop;
  tgp_data data;
  const float* y;         /* [device] [n_points, n_outputs]                  */
  int32_t n_outputs;
  double* mse;            /* [device] [pop, n_outputs] output                */
  int32_t* tree_status;   /* [device] [pop] output, or NULL                  */
  tgp_config cfg;         /* launch shape (all zero = heuristic) and flags;
                             the events and max_wait_polls are ignored       */
} tgp_problem;

#define TGP_MAX_PROBLEMS 16

/* Workspace bytes of tgp_batch_fitness_mse for these problems (0 = invalid). */
size_t tgp_batch_workspace_size(const tgp_problem* probs, int32_t n);

/* SR fitness of n independent problems of uneven sizes (populations, tree
 * lengths, point counts, feature counts) in one stage launch, one persistent
 * evaluation launch per occupancy group and one finalize launch.  Problems
 * whose shared-memory footprint allows the same number of resident CTAs per
 * SM form a group (for each of the two kernel variants when single-output
 * and Modi populations are mixed); within a group the persistent CTAs pull work items
 * of every problem from one counter, so small and large problems fill the
 * GPU together.  Same per-problem results as tgp_fitness_mse.  All problems
 * with one output must use the same points_per_lane.  Legal in
 * stream capture (the batched call of one generation is a CUDA graph). */
tgp_status tgp_batch_fitness_mse(const tgp_problem* probs, int32_t n, void* ws, size_t ws_bytes,
                                 void* stream);

/* Batch plan: the problems of tgp_batch_fitness_mse planned once on the host
 * (launch shapes, workspace layout, launch grouping), then run any number of
 * times.  tgp_batch_plan makes no CUDA call that touches the device's work
 * (no allocation, no synchronization, no launch); it reads the device's SM
 * count and shared-memory limit once per device.  The plan keeps a copy of
 * the problem descriptors (the pointers in them, not the data): the buffers
 * they name must stay valid, and their contents may change, between runs.
 *   probs, n     as for tgp_batch_fitness_mse (1..TGP_MAX_PROBLEMS problems)
 *   tune_cache   [host] path of the autotuner's cache file, or NULL.  For each
 *                problem whose cfg shape fields are all zero, an entry for
 *                this GPU and the problem's shape bucket (log2 of population,
 *                points and max_len, features, outputs) supplies the launch
 *                shape; otherwise the library's heuristic does.  A missing or
 *                unreadable file is the same as NULL.  Format, one entry per
 *                line ('#' starts a comment):
 *                  <GPU name, spaces as '_'>|P<lg P>_D<lg D>_F<F>_O<O>_L<lg L>
 *                  trees_per_block=<n> points_per_tile=<n> tiles_per_item=<n>
 *                  points_per_lane=<n> [cta_width=<0..2>]
 *                  [other name=value pairs are ignored]
 *                (all on one line; lg x = log2(x) rounded to the nearest
 *                integer).
 *   plan         [host] out: the plan (host memory the library allocates with
 *                malloc; release it with tgp_batch_free).
 * Returns the same argument errors as tgp_batch_fitness_mse. */
typedef struct tgp_batch_plan_s tgp_batch_plan_t;
tgp_status tgp_batch_plan(const tgp_problem* probs, int32_t n, const char* tune_cache,
                          tgp_batch_plan_t** plan);

/* Host-only lookup in an autotuner cache file (the format of tgp_batch_plan):
 * the launch shape stored for `key` (the whole first field of a line, e.g.
 * "NVIDIA_GB300|P13_D17_F16_O1_L8"), the last line for the key winning.
 * Makes no CUDA call.  Returns TGP_OK and fills the shape fields of *shape
 * (the rest zero), or TGP_ERR_INVALID_ARG when the file, the key or a valid
 * entry is missing. */
tgp_status tgp_tune_cache_lookup(const char* tune_cache, const char* key, tgp_config* shape);

/* Workspace bytes a run of the plan needs (0 for a NULL plan). */
size_t tgp_batch_plan_workspace_size(const tgp_batch_plan_t* plan);

/* Launch shape the plan chose for problem i (cfg events are NULL), so that a
 * caller can see whether the cache or the heuristic supplied it.  Returns
 * TGP_ERR_INVALID_ARG for a NULL plan or pointer or i out of range. */
tgp_status tgp_batch_plan_shape(const tgp_batch_plan_t* plan, int32_t i, tgp_config* shape,
                                int32_t* from_cache);

/* Runs the plan: one stage launch, one persistent evaluation launch per
 * occupancy group and one finalize launch on `stream`, exactly as
 * tgp_batch_fitness_mse.  Legal in stream capture: a captured run is a CUDA
 * graph that evaluates the batch every time it is replayed. */
tgp_status tgp_batch_run(const tgp_batch_plan_t* plan, void* ws, size_t ws_bytes, void* stream);

/* Releases a plan (NULL is ignored). */
void tgp_batch_free(tgp_batch_plan_t* plan);

/* Reverse-mode gradient of L = sum_{p,k} grad_mse[p,k] * MSE[p,k] (the
 * adjoint is not in the paper; it differentiates the Sec. III-C fitness).
 *   grad_mse   [device] double [pop, n_outputs]  upstream gradient
 *   mse_out    [device] double [pop, n_outputs]  MSE of the same pass, or NULL
 *              (then trees whose grad_mse row is zero are skipped)
 *   grad_value [device] float  [pop, ld] or NULL: dL/d(constant) at constant
 *              nodes, 0 at every other and every padding position, NaN rows
 *              for invalid trees
 *   grad_X     [device] float  [n_points, n_features] (contiguous) or NULL:
 *              dL/dX is ADDED to it (zero it first), so calls accumulate.
 * Derivative conventions: max sends the gradient to the operand fmax
 * returned (the left one on a tie); the guard branches of pdiv and plog and
 * the clamp of cexp have zero derivative.  n_features is bounded by the
 * shared memory that holds one 128-point tile of X and of its gradient
 * (about 175 features for trees of up to 127 nodes, 164 for 255, 95 for
 * 1024); beyond it the call returns TGP_ERR_UNSUPPORTED.  Intermediate values are recomputed
 * per point tile (a per-thread tape of at most one value per node), never
 * stored per population x length x points.  Sums of gradients use atomic
 * additions, so their last bits may differ between runs. */
tgp_status tgp_eval_backward(const tgp_population* pop, const tgp_data* data, const float* y,
                             int32_t n_outputs, const double* grad_mse, double* mse_out,
                             float* grad_value, float* grad_X, int32_t* tree_status, void* ws,
                             size_t ws_bytes, void* stream);

/* tgp_eval_backward with call options: cfg->points_per_tile (a multiple of
 * 128 up to 4096, 0 = the library's choice) is the point tile one CTA owns
 * for every tree, cfg->eval_begin_event / eval_end_event bracket the adjoint
 * kernel(s); the other fields are ignored.  TGP_ERR_UNSUPPORTED when the
 * given tile does not fit shared memory. */
tgp_status tgp_eval_backward_cfg(const tgp_population* pop, const tgp_data* data, const float* y,
                                 int32_t n_outputs, const double* grad_mse, double* mse_out,
                                 float* grad_value, float* grad_X, int32_t* tree_status, void* ws,
                                 size_t ws_bytes, void* stream, const tgp_config* cfg);

/* ---------------------------------------------------------------------------
 * Genetic operators on the same encoding (Sec. III-B "Tensorized Operations";
 * Algorithm 1).  Random choices are made by the caller: every random number
 * an operator uses is a 32-bit word passed in, so results are reproducible
 * and independent of the launch shape.  These calls need no workspace.
 * ------------------------------------------------------------------------- */

/* How tgp_subtree_exchange finds the replaced node k of the old tree and the
 * root j of the inserted subtree in the donor tree. */
typedef enum {
  TGP_PICK_NODES = 0,  /* node[i] = k and donor_node[i] = j are positions      */
  TGP_PICK_RANDOM = 1, /* k = node[i] mod len(old), j = donor_node[i] mod
                          len(donor): one-point crossover (donor = the second
                          parent) and subtree mutation (donor = new trees)     */
  TGP_PICK_HOIST = 2   /* hoist mutation: the donor is the old tree itself;
                          k = node[i] mod len, j = k + donor_node[i] mod
                          size[k], so a subtree of the subtree at k replaces it */
} tgp_pick_mode;

/* Per-child result of tgp_subtree_exchange. */
enum {
  TGP_XCHG_TOO_LARGE = 0,  /* the child would exceed max_size: it is the old
                              tree unchanged (the paper's size rule)          */
  TGP_XCHG_DONE = 1,       /* the child is exchange(T_old, k, T_new)          */
  TGP_XCHG_SKIPPED = 2,    /* apply_word[i] >= apply_below: a copy of T_old   */
  TGP_XCHG_BAD_INDEX = -1, /* a tree index or (TGP_PICK_NODES) a position out
                              of range; the child row is all NaN              */
  TGP_XCHG_BAD_TREE = -2   /* a length or subtree size that is not an integer
                              within its tree; the child row is all NaN       */
};

/* Subtree exchange (Sec. III-B): child i is
 *   T* = T_old[0..k) (+) T_new (+) T_old[k + size_old[k] .. len_old)
 * for all three tensors, where T_new is the subtree of the donor rooted at j
 * and every ancestor of k in the prefix has its subtree size grown by
 * dn = size_donor[j] - size_old[k].  A child longer than max_size is the old
 * tree unchanged.
 *   old          population the children start from ([device] rows)
 *   donor        population the inserted subtrees come from; ignored (may be
 *                NULL) with TGP_PICK_HOIST
 *   old_index    [device] int32 [n]: row of `old` for child i
 *   node         [device] uint32 [n]: position or random word for k
 *   donor_index  [device] int32 [n]: row of `donor` (ignored with HOIST)
 *   donor_node   [device] uint32 [n] or NULL (= 0): position or random word
 *                for j
 *   apply_word   [device] uint32 [n] or NULL: child i takes part only when
 *                apply_word[i] < apply_below (the operator's probability p as
 *                the threshold p * 2^32); the others are copies of T_old
 *   max_size     the maximum tree size, 1..TGP_MAX_LEN
 *   out_type, out_value, out_size
 *                [device] float [n, out_ld] each: the children, NaN-padded over
 *                the whole row; out_ld >= max(max_size, old->max_len).  They
 *                must not overlap the inputs (checked on the host).
 *   xchg_status  [device] int32 [n] or NULL: TGP_XCHG_* per child.
 * The exchange assumes trees that pass tgp_validate; other trees are never
 * read outside their rows, and the checks listed for TGP_XCHG_BAD_TREE are
 * the only ones made.  Bit-exact: each output element is a copy of an input
 * element, or a subtree size plus dn (exact in float). */
tgp_status tgp_subtree_exchange(const tgp_population* old, const tgp_population* donor,
                                const int32_t* old_index, const uint32_t* node,
                                const int32_t* donor_index, const uint32_t* donor_node,
                                const uint32_t* apply_word, uint32_t apply_below, int64_t n,
                                int32_t mode, int32_t max_size, float* out_type, float* out_value,
                                float* out_size, int64_t out_ld, int32_t* xchg_status,
                                void* stream);

/* Tournament selection (Algorithm 1, "Select parents"; the tournament size is
 * a parameter of the table "Configuration of Genetic Programming"):
 * contestant m of selection i is tree words[i * tournament_size + m] mod pop;
 * winners[i] is the contestant with the lowest (minimize != 0) or highest
 * fitness; ties go to the earliest contestant and NaN loses to every number.
 *   fitness  [device] double, tree p at fitness[p * stride] (stride >= 1, so a
 *            column of an MSE matrix [pop, n_outputs] can be used directly)
 *   words    [device] uint32 [n, tournament_size], tournament_size 1..4096
 *   winners  [device] int32 [n]
 * pop must be in [1, 2^31).  Bit-exact. */
tgp_status tgp_tournament_select(const double* fitness, int64_t stride, int64_t pop,
                                 const uint32_t* words, int64_t n, int32_t tournament_size,
                                 int32_t minimize, int32_t* winners, void* stream);

/* Classification fitness (Sec. V-D, measured by accuracy) from forward
 * outputs: the predicted class of point d is the first index k of the largest
 * non-NaN out[p, k, d] (no prediction when all are NaN), and correct[p] counts
 * the points whose prediction equals labels[d].
 *   out       [device] float [pop, n_classes, n_points] (tgp_eval_forward's
 *             layout), n_classes 1..TGP_MAX_OUTPUTS, n_points >= 1
 *   labels    [device] int32 [n_points]
 *   correct   [device] int64 [pop] (overwritten)
 *   accuracy  [device] double [pop] or NULL: correct / n_points
 * Bit-exact (integer counts). */
tgp_status tgp_accuracy_from_outputs(const float* out, int64_t pop, int32_t n_classes,
                                     int64_t n_points, const int32_t* labels, int64_t* correct,
                                     double* accuracy, void* stream);

/* Workspace bytes of tgp_fitness_accuracy (0 on invalid arguments). */
size_t tgp_accuracy_workspace_size(const tgp_population* pop, const tgp_data* data,
                                   int32_t n_classes);

/* Classification accuracy of every tree: the outputs of Modi nodes tagged
 * 0..n_classes-1 (Sec. IV-C) are the class scores, evaluated by the forward
 * kernels over chunks of points (a [pop, n_classes, chunk] buffer of at most
 * 256 MiB, or 256 points, inside ws) and reduced as in
 * tgp_accuracy_from_outputs.  accuracy [device] double [pop] (NaN for trees
 * that fail validation), correct [device] int64 [pop] or NULL, tree_status
 * [device] int32 [pop] or NULL. */
tgp_status tgp_fitness_accuracy(const tgp_population* pop, const tgp_data* data,
                                const int32_t* labels, int32_t n_classes, double* accuracy,
                                int64_t* correct, int32_t* tree_status, void* ws, size_t ws_bytes,
                                void* stream);

/* Largest scratch tgp_fitness_mse_noalloc can use (32 MiB). */
#define TGP_NOALLOC_WS_BYTES (32u << 20)

/* tgp_fitness_mse for callers that cannot allocate device memory.  The paper
 * has no counterpart; this is a deployment convenience of the library.
 * Some callers have no way to obtain a device buffer for the workspace: a
 * plain C host that links only this library and the CUDA runtime but owns no
 * device allocator, a plugin whose host application manages all device
 * memory itself, or a latency-bound loop that must not call cudaMalloc (which
 * can synchronize the device).  This entry point takes the same arguments as
 * tgp_fitness_mse minus ws/ws_bytes and returns the same results; its scratch
 * is a fixed array of TGP_NOALLOC_WS_BYTES in the library's own device memory
 * (one per GPU that loads the library, held until the process exits).  It
 * calls no cudaMalloc, cudaFree or allocating library routine.
 *   - TGP_ERR_WORKSPACE when the problem needs more scratch than
 *     TGP_NOALLOC_WS_BYTES (tgp_workspace_size with cfg = NULL tells);
 *     nothing is launched then.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before capturing a stream.
 *   - Every call uses the same array and leaves its contents there; the
 *     words that must start at zero are cleared by each call.  Calls whose
 *     work can overlap on the GPU (unordered streams, or several host threads)
 *     race on the array and give wrong results: order them on one stream. */
tgp_status tgp_fitness_mse_noalloc(const tgp_population* pop, const tgp_data* data,
                                   const float* y, int32_t n_outputs, double* mse,
                                   int32_t* tree_status, void* stream);

/* tgp_check_device_error for the scratch array of tgp_fitness_mse_noalloc
 * (whose callers never see a workspace pointer): reads and clears the error
 * word the last no-allocation call left there, after synchronizing `stream`.
 * Call it before the next no-allocation call, which clears the word.
 * Returns TGP_OK, TGP_ERR_TIMEOUT (that call's results are not valid) or
 * TGP_ERR_CUDA. */
tgp_status tgp_check_device_error_noalloc(void* stream);

/* Reads and clears the device error word left in ws by the last calls on
 * this workspace (a bounded wait that gave up).  Synchronizes `stream`.
 * Returns TGP_OK or TGP_ERR_TIMEOUT. */
tgp_status tgp_check_device_error(void* ws, size_t ws_bytes, void* stream);

/* Human-readable name of a status code. */
const char* tgp_status_string(tgp_status s);

/* Library version string. */
const char* tgp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TGP_H */
