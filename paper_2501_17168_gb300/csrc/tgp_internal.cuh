// tgp_internal.cuh -- shared definitions of the sm_103a kernels: the compiled
// instruction sets, workspace layout and kernel argument blocks.
//
// Evaluation model.  The paper evaluates a prefix tree with a value stack,
// walking the nodes from the end to the start (Sec. III-C).  Here each tree is
// first compiled (stage kernel) into a register-machine program for a warp:
//   * one warp evaluates one tree over 32*K data points (K points per lane);
//     every lane runs the same instruction, so dispatch never diverges;
//   * operands are evaluated in Sethi-Ullman order (the child that needs more
//     registers first), which bounds the registers by log2(leaves) + 1: nine
//     cover every binary/unary tree of up to 1023 nodes;
//   * leaves are fused into their parent's instruction (a variable operand is
//     read from the shared-memory tile of X, a constant rides in the
//     instruction word), so leaves cost no dispatch of their own;
//   * a Modi node (Sec. IV-C) is one instruction that adds its function value
//     into its output accumulator and hands its parent its rightmost child's
//     value.
// Two instruction sets share this scheme.  The forward kernels run the
// level-register set of isa_fwd.cuh (generated with its interpreter by
// gen_interp.py): the value of a subtree at nesting level d lives in register
// group G[d], so evaluation order costs no copies, and a binary node with two
// leaf children is one instruction.  The adjoint runs the accumulator-and-
// slots set below (enum Op): the top of the stack in "acc", the rest in R = 8
// slots, and every leaf operand carries its node position for the constant
// gradients.
// Reordering the operand evaluation does not change any value: every
// function is pure, only the order in which Modi contributions are summed
// into an output changes.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tgp {

// ------------------------------------------------------------- encoding
enum NodeType : int { T_VAR = 0, T_CONST = 1, T_UFUNC = 2, T_BFUNC = 3, T_TFUNC = 4, T_MODI = 16 };
enum Func : int { F_ADD = 0, F_SUB, F_MUL, F_PDIV, F_MAX, F_SIN, F_COS, F_PLOG, F_CEXP, F_TAN, F_ITE, F_COUNT };
enum TreeStatus : int {
  S_LEN = 1, S_TYPE = 2, S_FUNC = 4, S_VAR = 8, S_MODI = 16, S_CONST = 32, S_SIZE = 64, S_DEPTH = 128,
  S_NOADJ = 256   // a node the adjoint does not differentiate (ite)
};

constexpr int R = 8;            // register slots below the accumulator
constexpr int MAX_LEN = 1024;   // longest supported tree
constexpr int MAX_OUT = 16;     // outputs
constexpr int MAX_FEAT = 256;   // features

// ------------------------------------------------------------- adjoint instruction set
// One instruction is a uint2: .x = opcode | out_index << 8 | leaf_node << 16;
// .y = the leaf operand (feature index for *V forms, float bits of the
// constant for *C forms).  leaf_node is the prefix position of the leaf
// operand (used by the adjoint to route constant gradients).  f = function
// id 0..9, d = slot 0..7.
enum Op : uint32_t {
  OP_END_ROOT = 0,   // output 0 := acc (single output, no Modi node)
  OP_END_MODI = 1,   // outputs are the Modi accumulators
  OP_LDV = 2,        // acc = x[v]
  OP_LDC = 3,        // acc = c
  OP_UN = 4,         // + (f-5):   acc = f(acc)                       4..8
  OP_UNV = 9,        // + (f-5):   acc = f(x[v])                      9..13
  OP_BV = 14,        // + f:       acc = f(acc, x[v])                14..18
  OP_BC = 19,        // + f:       acc = f(acc, c)                   19..23
  OP_RV = 24,        // + f:       acc = f(x[v], acc)                24..28
  OP_RC = 29,        // + f:       acc = f(c, acc)                   29..33
  OP_UN_M = 34,      // + (f-5):   out[o] += f(acc)                  34..38
  OP_BV_M = 39,      // + f:       out[o] += f(acc, x[v]); acc = x[v]
  OP_BC_M = 44,      // + f:       out[o] += f(acc, c);    acc = c
  OP_RV_M = 49,      // + f:       out[o] += f(x[v], acc)
  OP_RC_M = 54,      // + f:       out[o] += f(c, acc)               54..58
  OP_SPV = 59,       // + d:       s[d] = acc; acc = x[v]            59..66
  OP_SPC = 67,       // + d:       s[d] = acc; acc = c               67..74
  OP_BS = 75,        // + f*R + d: acc = f(s[d], acc)                75..114
  OP_RS = 115,       // + f*R + d: acc = f(acc, s[d])               115..154
  OP_BS_M = 155,     // + f*R + d: out[o] += f(s[d], acc)           155..194
  OP_RS_M = 195,     // + f*R + d: out[o] += f(acc, s[d]); acc = s[d]  195..234
  OP_COUNT = 235
};

__host__ __device__ constexpr int arity(int f) { return f <= F_MAX ? 2 : f == F_ITE ? 3 : 1; }

// ------------------------------------------------------------- FP32 functions
// The function bodies (protected division and log with the 1e-6f guard,
// exp clamped at 80, sin/cos with a two-constant Cody-Waite reduction on the
// MUFU approximations) live in the generated interpreter, gen_interp.py.

// ------------------------------------------------------------- workspace
// All regions are 256-byte aligned offsets from the workspace base.
struct WsLayout {
  size_t prog;      // uint2 [pop, pcap]  compiled programs
  size_t plen;      // int32 [pop]        instruction count (0 = invalid tree)
  size_t status;    // int32 [pop]        per-tree status
  size_t partial;   // double [pop, n_out, n_groups]  per-item partial SSE
  size_t gval64;    // double [pop, max_len]  constant gradients (adjoint)
  size_t mse64;     // double [pop, n_out]    squared-residual sums (adjoint)
  size_t ctrl;      // uint32 [64]: [0] work counter, [1] any-Modi flag, [2] error word
  size_t total;
  int pcap;         // instructions per program slot (even)
  int n_groups;     // partial sums per tree and output
};

// Launch shape after the heuristic.
struct Shape {
  int K;         // points per lane
  int nw;        // warps per CTA
  int bt;        // trees per block
  int tp;        // points per tile
  int g;         // tiles per item
  int n_tiles;
  int n_groups;
  int n_blocks;
  long long n_items;
  bool cramped;  // shared memory forced fewer trees or points than the heuristic wanted
};

struct StageArgs {
  const float* type;
  const float* val;
  const float* size;
  long long pop, ld;
  int max_len, n_features, n_outputs;
  uint2* prog;
  int pcap;
  int* plen;
  int* status;
  int* user_status;   // may be null
  unsigned* ctrl;
  int want_nodes;      // 1: adjoint programs (enum Op, leaf node positions in bits
                       // 16-31); 0: forward programs (isa_fwd.cuh)
};

struct EvalArgs {
  const uint2* prog;
  const int* plen;
  const int* status;
  int pcap;
  long long pop;
  const float* X;
  long long D;
  int F;
  long long ldx;
  int x_vec4;         // 1: X 16-byte aligned, F and ldx multiples of 4 (float4 rows)
  const float* y;     // [D, O] (MSE mode)
  int O;
  float* out;         // [pop, O, D] (forward mode)
  double* partial;    // [pop, O, n_groups] (MSE mode)
  int bt, tp, g, n_tiles, n_groups, n_blocks;
  long long n_items;
  unsigned* ctrl;
};

struct FinalArgs {
  const double* partial;
  const int* status;
  double* mse;
  long long pop;
  int O, n_groups;
  long long D;
  int sse;            // 1: write the sum of squared residuals (no division by D)
};

struct AdjArgs {
  const uint2* prog;
  const int* plen;
  const int* status;
  int pcap;
  long long pop;
  int max_len;
  const float* X;
  long long D;
  int F;
  long long ldx;
  const float* y;      // [D, O]
  int O;
  const double* g;     // [pop, O] upstream gradient of the MSE
  bool want_mse;       // accumulate the MSE too (else trees with g == 0 are skipped)
  double* gval64;      // [pop, max_len] constant gradients (FP64)
  double* mse64;       // [pop, O] sum of squared residuals (FP64)
  float* grad_X;       // [D, F] accumulated into (may be null)
  int tp, n_tiles;
  int tree_chunks;           // the population split into this many tree ranges
  long long trees_per_chunk;
  double two_over_D;         // 2 / n_points: dL/d(output) = g (o - y) 2 / D
  unsigned* ctrl;
};

struct AdjFinalArgs {
  const double* gval64;
  const double* mse64;
  const int* status;
  float* grad_value;   // [pop, ld] or null
  double* mse;         // [pop, O] or null
  long long pop, ld;
  int max_len, O;
  long long D;
};

// Several problems in one launch: a table of per-problem arguments passed as
// a __grid_constant__ kernel parameter; global indices (work items, trees,
// outputs) are split by the cumulative counts.
constexpr int MAX_PROBLEMS = 16;

struct StageBatch {
  int n;
  int lmax;                          // node records per warp: max max_len, multiple of 16
  long long end[MAX_PROBLEMS];       // cumulative tree counts
  StageArgs p[MAX_PROBLEMS];
};

struct EvalBatch {
  int n;
  int max_polls;                     // bounded-wait limit (negative: give up at once)
  unsigned* counter;                 // work counter of this kernel variant
  unsigned* err;                     // error word of the call (control block of ws)
  long long end[MAX_PROBLEMS];       // cumulative work items
  EvalArgs p[MAX_PROBLEMS];
};

struct FinalBatch {
  int n;
  long long end[MAX_PROBLEMS];       // cumulative pop * n_outputs
  FinalArgs p[MAX_PROBLEMS];
};

__host__ __device__ inline int batch_find(const long long* end, int n, long long g) {
  int i = 0;
  while (i < n - 1 && g >= end[i]) ++i;
  return i;
}

// control word indices
// (CTRL_COUNTER_GROUP + 2*g + variant: work counters of the evaluation
// launches, one per launch group g and kernel variant)
enum { CTRL_COUNTER = 0, CTRL_ANY_MODI = 1, CTRL_ERROR = 2, CTRL_COUNTER_MODI = 3,
       CTRL_COUNTER_GROUP = 8, CTRL_WORDS = 64 };
// bits of the error word
enum { ERR_MBAR_TIMEOUT = 1 };
// polls of a bounded mbarrier wait before it gives up (each poll suspends the
// thread for a while, so this is seconds)
constexpr int kDefaultWaitPolls = 1 << 22;

}  // namespace tgp
