// isa_fwd.cuh -- GENERATED by gen_interp.py; do not edit by hand.
// Opcodes of the forward instruction set run by interp_fwd (level registers
// G[0..NREG-1], a memory stack of NSM shared-memory entries per warp and
// MAXS local-memory entries per thread).  A level form's
// opcode is base + sub * NREG + d, a memory form's base + sub; sub is the
// unary index f - F_SIN, the binary function f, or for the forms that exist
// only for non-commutative functions nc_index(f).  Word: .x = opcode |
// out_index << 16 (Modi forms), .y = operand; VC/CV/CC take a second word
// whose .x is the feature index (VC, CV) or the bits of the second constant
// (CC).
#pragma once
#include <cstdint>
namespace tgp {
namespace fx {
constexpr int NREG = 3;
constexpr int MAXS = 6;
constexpr int NSM = 1;   // stack entries in shared memory (SAVES/MSS/SMS forms; the
                           // Modi kernel keeps them in local memory)
enum : uint32_t {
  END_ROOT = 0,  // output := G[0] (one output, no Modi node)
  END_MODI = 1,  // outputs are the Modi accumulators
  LDV = 2,
  LDC = 5,
  UN = 8,
  UNV = 23,
  UNC = 38,
  BV = 53,
  BC = 68,
  RV = 83,
  RC = 89,
  VV = 95,
  VC = 110,
  CV = 125,
  CC = 131,
  BS = 146,
  RS = 161,
  UN_M = 167,
  UNV_M = 182,
  UNC_M = 197,
  BV_M = 212,
  BC_M = 227,
  RV_M = 242,
  RC_M = 257,
  BS_M = 272,
  RS_M = 287,
  SAVE = 302,
  MS = 303,
  SM = 308,
  MS_M = 310,
  SM_M = 315,
  SAVES = 320,
  MSS = 321,
  SMS = 326,
  MSS_M = 328,
  SMS_M = 333,
  COUNT = 338
};
// index of a non-commutative binary function among the two-entry forms
__host__ __device__ constexpr int nc_index(int f) { return f == 1 ? 0 : f == 3 ? 1 : -1; }
}  // namespace fx
}  // namespace tgp
