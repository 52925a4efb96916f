// stage.cu -- validation and compilation of the population tensors.
//
// One warp per tree.  The lanes read the tree's three rows (Sec. III-A
// encoding) coalesced, check every node in parallel, and check the subtree
// sizes locally: a node of arity a at position i with size s is consistent iff
// its children, found from the sizes (first child at i+1, second at
// i+1+size[i+1]), tile [i+1, i+s) exactly.  These local rules hold at every
// position of [0, len) exactly when the arrays encode one tree of len nodes.
// Lane 0 then compiles the tree into the register-machine program described
// in tgp_internal.cuh: a bottom-up pass computes how many registers each
// subtree needs when the hungrier child is evaluated first (Sethi-Ullman
// numbering), and a stack-free walk over parent links emits the post-order
// instruction stream with leaves fused into their parents.
#include "tgp_internal.cuh"
#include "isa_fwd.cuh"

namespace tgp {

// per-warp shared memory: node records of one tree, lmax entries per array
// (lmax = the longest max_len of the launch, a multiple of 16)
struct NodeSmem {
  uint32_t* info;   // bits 0-3 func, 4-6 kind (0 var, 1 const, 2 unary, 3 binary, 4 ternary),
                    // 7 modi, 8-15 out, 16 scratch of the compiler
  int16_t* sz;      // subtree size (0 = not a valid size)
  int16_t* par;     // parent index
  uint8_t* need;    // registers (levels) the subtree needs
  uint8_t* slot;    // the subtree's level (first free slot for the adjoint set)
  const float* V;   // the tree's value row in global memory (read again for
                    // leaf operands: 10 bytes per node in shared memory
                    // instead of 14 let more trees compile at once)
  // a validated leaf's operand: variable index or constant bits
  __device__ __forceinline__ uint32_t leaf(int i) const {
    const float v = __ldg(V + i);
    return (info[i] >> 4 & 7) == 0 ? (uint32_t)v : __float_as_uint(v);
  }
};

__host__ __device__ constexpr size_t node_smem_bytes(int lmax) { return (size_t)lmax * 10; }

__device__ NodeSmem node_smem(unsigned char* base, int lmax) {
  NodeSmem ns;
  ns.info = reinterpret_cast<uint32_t*>(base);
  ns.sz = reinterpret_cast<int16_t*>(ns.info + lmax);
  ns.par = ns.sz + lmax;
  ns.need = reinterpret_cast<uint8_t*>(ns.par + lmax);
  ns.slot = ns.need + lmax;
  return ns;
}

constexpr int STAGE_WARPS = 4;

__device__ __forceinline__ bool is_int(float v) { return isfinite(v) && v == floorf(v); }

__device__ __forceinline__ int kind_of(uint32_t in) { return (in >> 4) & 7; }

// Emits the forward program of a validated tree in the level-register
// instruction set (isa_fwd.cuh): the value of a subtree evaluated at level d
// goes to register group G[d]; of a binary node's two subtrees the one that
// needs more levels is evaluated first at the node's level, the other one
// level deeper (at level NREG-1 the first result is saved to the memory
// stack instead and the other subtree reuses the level; the push rides in
// the word of that subtree's first instruction).  Leaf operands ride in
// their parent's instruction.  Returns the number of words, or -1 if the
// program would exceed cap words or the memory stack (neither happens for
// trees of up to 1024 nodes: every non-leaf subtree has a leaf without a
// word of its own, and the Sethi-Ullman number stays below NREG + MAXS).
// bit of a ternary node's info word once its condition has been pushed
constexpr uint32_t COND_DONE = 1u << 16;

// The two operands of node q's binary instruction: a binary node's children,
// or the branches (second and third children) of an ite node, whose first
// child is its condition.
__device__ __forceinline__ void bin_ops(const NodeSmem& ns, int q, int* ca, int* cb) {
  int a = q + 1;
  if (kind_of(ns.info[q]) == 4) a += ns.sz[a];
  *ca = a;
  *cb = a + ns.sz[a];
}

static_assert(fx::NSM == 1, "fused pushes address shared-memory entry 0 only");

__device__ int compile_fx(NodeSmem& ns, bool single_out, uint2* prog, int cap) {
  using namespace fx;
  int pc = 0, n = 0, sdepth = 0, cdepth = 0;
  int pend = 0;  // a push of G[NREG-1] not yet emitted: 1 to shared-memory entry 0, 2 to local memory
  bool down = true;
  auto put = [&](uint32_t x, uint32_t y) {
    if (pc >= cap) return false;
    prog[pc++] = make_uint2(x, y);
    return true;
  };
  // the first word of an instruction: a pending push rides in it (the
  // instruction after a push starts the next subtree at level NREG-1, so it
  // loads a leaf and has a fused push form); else the push is a word of its own
  auto emit = [&](uint32_t x, uint32_t y) {
    if (pend) {
      uint32_t fused = PUSH_FORM_TABLE[x & 0xFFFFu];  // push_form(op, false)
      if (fused) x = (fused + (pend == 2 ? (uint32_t)NSTART : 0u)) | (x & ~0xFFFFu);
      else if (!put(pend == 1 ? (uint32_t)SAVES : (uint32_t)SAVE, 0)) return false;
      pend = 0;
    }
    return put(x, y);
  };
  ns.slot[0] = 0;
  for (;;) {
    const uint32_t in = ns.info[n];
    const int k = kind_of(in);
    if (down) {
      const int lv = ns.slot[n];
      if (k <= 1) {  // a lone leaf: the root, or the first operand of a Modi node
        if (!emit((k == 0 ? LDV : LDC) + lv, ns.leaf(n))) return -1;
        down = false;
        continue;
      }
      const bool modi = in & 128;
      const int f = in & 15;
      const uint32_t o16 = modi ? ((in >> 8) & 255) << 16 : 0;
      if (k == 2) {
        const int c = n + 1, ck = kind_of(ns.info[c]);
        if (ck <= 1) {  // unary of a leaf: one instruction
          const uint32_t base = modi ? (ck == 0 ? UNV_M : UNC_M) : (ck == 0 ? UNV : UNC);
          if (!emit((base + (f - F_SIN) * NREG + lv) | o16, ns.leaf(c))) return -1;
          down = false;
          continue;
        }
        ns.slot[c] = lv;
        n = c;
        continue;
      }
      if (k == 4 && !(in & COND_DONE)) {
        // ite: the condition first, at the node's level; its sign bits go to
        // the condition stack and the branches follow as a binary form
        const int a = n + 1, ka = kind_of(ns.info[a]);
        if (ka <= 1) {
          if (cdepth >= MAXC || !emit((ka == 0 ? CDV : CDC) + lv, ns.leaf(a))) return -1;
          ++cdepth;
          ns.info[n] = in | COND_DONE;
          continue;
        }
        ns.slot[a] = lv;
        n = a;
        continue;
      }
      const int fb = k == 4 ? (int)F_ITE : f, bfn = bin_index(fb);
      int ca, cb;
      bin_ops(ns, n, &ca, &cb);
      const int ka = kind_of(ns.info[ca]), kb = kind_of(ns.info[cb]);
      if (ka <= 1 && kb <= 1 && !modi) {  // two leaves: one instruction
        const uint32_t la = ns.leaf(ca), lb = ns.leaf(cb);
        const int nc = nc_index(fb);
        bool ok;
        if (ka == 0 && kb == 0) ok = emit(VV + bfn * NREG + lv, la | (lb << 16));
        else if (ka == 0) ok = emit(VC + bfn * NREG + lv, lb) && put(la, 0);
        else if (kb == 0 && nc < 0) ok = emit(VC + bfn * NREG + lv, la) && put(lb, 0);
        else if (kb == 0) ok = emit(CV + nc * NREG + lv, la) && put(lb, 0);
        else ok = emit(CC + bfn * NREG + lv, la) && put(lb, 0);
        if (!ok) return -1;
        if (k == 4) --cdepth;  // the selection pops the condition
        down = false;
        continue;
      }
      const int first = kb <= 1 ? ca : ka <= 1 ? cb : (ns.need[ca] >= ns.need[cb] ? ca : cb);
      ns.slot[first] = lv;
      n = first;
      continue;
    }
    // ---- n is done: continue with its parent
    if (n == 0) break;
    const int q = ns.par[n];
    const uint32_t qin = ns.info[q];
    const int qk = kind_of(qin), f = qin & 15, lv = ns.slot[q];
    const bool modi = qin & 128;
    const uint32_t o16 = modi ? ((qin >> 8) & 255) << 16 : 0;
    if (qk == 4 && n == q + 1) {  // ite's condition is done: push its sign bits
      if (cdepth >= MAXC || !emit(CD + lv, 0)) return -1;
      ++cdepth;
      ns.info[q] = qin | COND_DONE;
      n = q;
      down = true;
      continue;
    }
    uint32_t x, y = 0;
    if (qk == 2) {
      x = (modi ? UN_M : UN) + (f - F_SIN) * NREG + lv;
    } else {
      const int fb = qk == 4 ? (int)F_ITE : f, bfn = bin_index(fb);
      int ca, cb;
      bin_ops(ns, q, &ca, &cb);
      const int ka = kind_of(ns.info[ca]), kb = kind_of(ns.info[cb]);
      const int nc = nc_index(fb);
      if (kb <= 1) {  // b is a leaf, a is in G[lv]
        x = (modi ? (kb == 0 ? BV_M : BC_M) : (kb == 0 ? BV : BC)) + bfn * NREG + lv;
        y = ns.leaf(cb);
      } else if (ka <= 1) {  // a is a leaf, b is in G[lv]
        if (modi) x = (ka == 0 ? RV_M : RC_M) + bfn * NREG + lv;
        else if (nc < 0) x = (ka == 0 ? BV : BC) + bfn * NREG + lv;
        else x = (ka == 0 ? RV : RC) + nc * NREG + lv;
        y = ns.leaf(ca);
      } else {
        const bool a_first = ns.need[ca] >= ns.need[cb];
        const int first = a_first ? ca : cb, second = a_first ? cb : ca;
        const bool mem = lv + 1 >= NREG;
        if (n == first) {  // first operand done: evaluate the second one
          if (mem) {
            if (sdepth >= NSM + MAXS) return -1;
            pend = sdepth < NSM ? 1 : 2;
            ++sdepth;
            ns.slot[second] = lv;
          } else {
            ns.slot[second] = lv + 1;
          }
          n = second;
          down = true;
          continue;
        }
        if (!mem) {  // first operand in G[lv], second in G[lv+1]
          if (a_first) x = (modi ? BS_M : BS) + bfn * NREG + lv;
          else if (modi) x = RS_M + bfn * NREG + lv;
          else if (nc < 0) x = BS + bfn * NREG + lv;
          else x = RS + nc * NREG + lv;
        } else {  // first operand on the memory stack, second in G[NREG-1]
          const int sq = --sdepth;
          if (sq < NSM) {  // entry in the warp's shared-memory rows
            if (a_first) x = (modi ? MSS_M : MSS) + bfn * NSM + sq;
            else if (modi) x = SMS_M + bfn * NSM + sq;
            else if (nc < 0) x = MSS + bfn * NSM + sq;
            else x = SMS + nc * NSM + sq;
          } else if (a_first) {
            x = (modi ? MS_M : MS) + bfn;
          } else if (modi) {
            x = SM_M + bfn;
          } else if (nc < 0) {
            x = MS + bfn;
          } else {
            x = SM + nc;
          }
        }
      }
      if (qk == 4) --cdepth;  // the selection pops the condition
    }
    if (!emit(x | o16, y)) return -1;
    n = q;
  }
  if (!emit(single_out ? END_ROOT : END_MODI, 0)) return -1;
  return pc;
}

// Emits the adjoint program of a validated tree in the accumulator-and-slots
// instruction set (enum Op): a post-order walk over parent links with leaves
// fused into their parents; every leaf operand records its node position in
// bits 16-31 (the adjoint routes constant gradients with it).  Returns the
// number of words, or -1 when the tree needs more than R slots.
__device__ int compile_adj(NodeSmem& ns, bool single_out, uint2* prog) {
  int pc = 0;
  int n = 0, pend = -1, last_ldv = -1;
  bool down = true, deep = false;
  ns.slot[0] = 0;
  for (;;) {
    uint32_t in = ns.info[n];
    int k = kind_of(in);
    if (down) {
      int c = -1;
      if (k == 2) {
        c = n + 1;
      } else if (k == 3) {
        int ca = n + 1, cb = ca + ns.sz[ca];
        bool la = kind_of(ns.info[ca]) <= 1, lb = kind_of(ns.info[cb]) <= 1;
        c = lb ? ca : la ? cb : (ns.need[ca] >= ns.need[cb] ? ca : cb);
      }
      if (c < 0) {  // a leaf evaluated on its own: load it (spilling acc first if pending)
        uint2 ins;
        bool var = k == 0;
        if (pend >= 0) {
          ins.x = (var ? OP_SPV : OP_SPC) + pend;
          pend = -1;
          last_ldv = -1;
        } else {
          ins.x = var ? OP_LDV : OP_LDC;
          last_ldv = var ? pc : -1;
        }
        ins.y = ns.leaf(n);
        ins.x |= (uint32_t)n << 16;  // leaf node index (constant gradients)
        prog[pc++] = ins;
        down = false;
      } else {
        ns.slot[c] = ns.slot[n];
        n = c;
      }
      continue;
    }
    if (n == 0) break;
    int q = ns.par[n];
    uint32_t qin = ns.info[q];
    int qk = kind_of(qin);
    int ca = q + 1, cb = ca + ns.sz[ca];
    bool la = false, lb = false, a_first = true;
    if (qk == 3) {
      la = kind_of(ns.info[ca]) <= 1;
      lb = kind_of(ns.info[cb]) <= 1;
      a_first = ns.need[ca] >= ns.need[cb];
      if (!la && !lb) {
        int second = a_first ? cb : ca;
        if (n != second) {  // first child done: spill it, evaluate the other one
          pend = ns.slot[q];
          if (pend >= R) { deep = true; break; }
          ns.slot[second] = ns.slot[q] + 1;
          n = second;
          down = true;
          continue;
        }
      }
    }
    // ---- emit the instruction of node q
    int f = qin & 15;
    bool modi = qin & 128;
    uint32_t o8 = ((qin >> 8) & 255) << 8;
    uint2 ins;
    ins.y = 0;
    if (qk == 2) {
      if (modi) {
        ins.x = (OP_UN_M + (f - F_SIN)) | o8;
      } else if (last_ldv == pc - 1 && last_ldv >= 0) {
        ins.x = OP_UNV + (f - F_SIN);  // fuse with the variable load just emitted
        ins.y = prog[pc - 1].y;
        --pc;
      } else {
        ins.x = OP_UN + (f - F_SIN);
      }
    } else if (lb) {
      bool var = kind_of(ns.info[cb]) == 0;
      ins.x = (modi ? (var ? OP_BV_M : OP_BC_M) : (var ? OP_BV : OP_BC)) + f;
      ins.x |= modi ? o8 : 0;
      ins.y = ns.leaf(cb);
      ins.x |= (uint32_t)cb << 16;
    } else if (la) {
      bool var = kind_of(ns.info[ca]) == 0;
      if (modi) ins.x = ((var ? OP_RV_M : OP_RC_M) + f) | o8;
      else if (f == F_ADD || f == F_MUL) ins.x = (var ? OP_BV : OP_BC) + f;
      else ins.x = (var ? OP_RV : OP_RC) + f;
      ins.y = ns.leaf(ca);
      ins.x |= (uint32_t)ca << 16;
    } else {
      int d = ns.slot[q];
      if (d >= R) { deep = true; break; }
      uint32_t base = a_first ? (modi ? OP_BS_M : OP_BS) : (modi ? OP_RS_M : OP_RS);
      ins.x = (base + f * R + d) | (modi ? o8 : 0);
    }
    prog[pc++] = ins;
    last_ldv = -1;
    n = q;
  }
  if (deep) return -1;
  prog[pc++] = make_uint2(single_out ? OP_END_ROOT : OP_END_MODI, 0u);
  return pc;
}

__global__ void __launch_bounds__(STAGE_WARPS * 32) stage_kernel(const __grid_constant__ StageBatch b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  NodeSmem ns = node_smem(smem_raw + (size_t)warp * node_smem_bytes(b.lmax), b.lmax);
  const long long total = b.end[b.n - 1];

  for (long long gt = (long long)blockIdx.x * STAGE_WARPS + warp; gt < total;
       gt += (long long)gridDim.x * STAGE_WARPS) {
    const int pi = batch_find(b.end, b.n, gt);
    const StageArgs& a = b.p[pi];
    const long long p = gt - (pi ? b.end[pi - 1] : 0);
    const float* T = a.type + p * a.ld;
    const float* V = a.val + p * a.ld;
    const float* S = a.size + p * a.ld;
    ns.V = V;
    int len = 0;
    if (lane == 0) {
      float s0 = S[0];
      len = (is_int(s0) && s0 >= 1.0f && s0 <= (float)a.max_len) ? (int)s0 : 0;
    }
    len = __shfl_sync(0xffffffffu, len, 0);
    int st = 0;
    bool modi_here = false;
    if (len == 0) {
      st = S_LEN;
    } else {
      // ---- per-node checks (lane-parallel)
      for (int i = lane; i < len; i += 32) {
        float tv = T[i], vv = V[i], sv = S[i];
        int ty = is_int(tv) && tv >= 0.0f && tv < 64.0f ? (int)tv : -1;
        uint32_t info = 0;
        int base = ty >= 0 ? (ty & ~T_MODI) : -1;
        bool modi = ty >= 0 && (ty & T_MODI);
        if (!(ty == 0 || ty == 1 || ty == 2 || ty == 3 || ty == 4 || ty == 18 || ty == 19 ||
              ty == 20)) {
          st |= S_TYPE;
        } else if (base == T_VAR) {
          if (!is_int(vv) || vv < 0.0f || vv >= (float)a.n_features) st |= S_VAR;
          info = 0u << 4;
        } else if (base == T_CONST) {
          if (!isfinite(vv)) st |= S_CONST;
          info = 1u << 4;
        } else {
          if (!is_int(vv) || vv < 0.0f || vv >= 65536.0f) {
            st |= S_FUNC;
          } else {
            int iv = (int)vv;
            int f = iv & 255, o = iv >> 8;
            // the type names the arity: 2 unary, 3 binary, 4 ternary
            if (f >= F_COUNT || arity(f) != base - 1) st |= S_FUNC;
            if (modi) {
              if (o >= a.n_outputs) st |= S_MODI;
            } else if (o != 0) {
              st |= S_FUNC;
            }
            info = (uint32_t)(f & 15) | ((uint32_t)base << 4) | (modi ? 128u : 0u) |
                   ((uint32_t)(o & 255) << 8);
            modi_here |= modi;
          }
        }
        ns.info[i] = info;
        ns.sz[i] = (is_int(sv) && sv >= 1.0f && sv <= (float)(len - i)) ? (int16_t)sv : (int16_t)0;
      }
      st = __reduce_or_sync(0xffffffffu, st);
      modi_here = __any_sync(0xffffffffu, modi_here);
      __syncwarp();
      if (!(st & (S_TYPE | S_FUNC))) {
        // ---- local subtree-size rules (lane-parallel)
        int bad = 0;
        for (int i = lane; i < len; i += 32) {
          int s = ns.sz[i];
          int k = kind_of(ns.info[i]);
          if (s == 0) { bad = 1; continue; }
          if (k <= 1) {
            if (s != 1) bad = 1;
          } else if (k == 2) {
            if (s < 2 || ns.sz[i + 1] == 0 || s != 1 + ns.sz[i + 1]) bad = 1;
            else ns.par[i + 1] = (int16_t)i;
          } else if (k == 3) {
            if (s < 3) { bad = 1; continue; }
            int s1 = ns.sz[i + 1];
            int c2 = i + 1 + s1;
            if (s1 == 0 || c2 >= i + s) { bad = 1; continue; }
            int s2 = ns.sz[c2];
            if (s2 == 0 || s != 1 + s1 + s2) { bad = 1; continue; }
            ns.par[i + 1] = (int16_t)i;
            ns.par[c2] = (int16_t)i;
          } else {  // ternary: three children tile [i+1, i+s)
            if (s < 4) { bad = 1; continue; }
            int s1 = ns.sz[i + 1];
            int c2 = i + 1 + s1;
            if (s1 == 0 || c2 >= i + s) { bad = 1; continue; }
            int s2 = ns.sz[c2];
            int c3 = c2 + s2;
            if (s2 == 0 || c3 >= i + s) { bad = 1; continue; }
            int s3 = ns.sz[c3];
            if (s3 == 0 || s != 1 + s1 + s2 + s3) { bad = 1; continue; }
            ns.par[i + 1] = (int16_t)i;
            ns.par[c2] = (int16_t)i;
            ns.par[c3] = (int16_t)i;
          }
        }
        if (__any_sync(0xffffffffu, bad)) st |= S_SIZE;
      }
      __syncwarp();
    }

    int pc = 0;
    bool ternary = false;
    if (st == 0) {
      // ---- registers needed per subtree (bottom-up), lane-parallel over
      // blocks of 32 nodes from the end: a node is done once its children
      // (all at larger indices) are, so a block takes as many rounds as its
      // longest parent chain
      for (int i = lane; i < len; i += 32) {
        ns.need[i] = 0;  // 0 = not known yet (every subtree needs >= 1)
        ternary |= kind_of(ns.info[i]) == 4;
      }
      ternary = __any_sync(0xffffffffu, ternary);
      __syncwarp();
      for (int base = (len - 1) & ~31; base >= 0; base -= 32) {
        const int i = base + lane;
        bool todo = i < len;
        while (__any_sync(0xffffffffu, todo)) {
          if (todo) {
            const int k = kind_of(ns.info[i]);
            int nd = 0;
            if (k <= 1) {
              nd = 1;
            } else if (k == 2) {
              nd = ns.need[i + 1];
            } else {
              // a binary node's operands, or an ite node's branches (its
              // condition is evaluated first at the same level, then popped)
              int ca, cb;
              bin_ops(ns, i, &ca, &cb);
              const int na = ns.need[ca], nb = ns.need[cb], nc = k == 4 ? ns.need[i + 1] : 1;
              if (na && nb && nc) {
                const bool la = kind_of(ns.info[ca]) <= 1, lb = kind_of(ns.info[cb]) <= 1;
                if (lb) nd = na;
                else if (la) nd = nb;
                else nd = na >= nb ? max(na, nb + 1) : max(nb, na + 1);
                if (k == 4) nd = max(nd, nc);
              }
            }
            if (nd) {
              ns.need[i] = (uint8_t)min(nd, 255);
              todo = false;
            }
          }
          __syncwarp();
        }
      }
    }
    if (st == 0 && lane == 0) {
      uint2* prog = a.prog + p * a.pcap;
      if (!a.want_nodes) {
        pc = compile_fx(ns, a.n_outputs == 1 && !modi_here, prog, a.pcap);
      } else if (ternary) {
        pc = -2;  // the adjoint set has no ite
      } else {
        pc = compile_adj(ns, a.n_outputs == 1 && !modi_here, prog);
      }
      if (pc < 0) {
        st = pc == -2 ? S_NOADJ : S_DEPTH;
        pc = 0;
      }
    }
    st = __shfl_sync(0xffffffffu, st, 0);
    pc = __shfl_sync(0xffffffffu, pc, 0);
    if (lane == 0) {
      a.status[p] = st;
      if (a.user_status) a.user_status[p] = st;
      a.plen[p] = st == 0 ? pc : 0;
      if (st == 0 && modi_here) atomicOr(&a.ctrl[CTRL_ANY_MODI], 1u);
    }
    __syncwarp();
  }
}

size_t stage_smem_bytes(int lmax) { return node_smem_bytes(lmax) * STAGE_WARPS; }
int stage_threads() { return STAGE_WARPS * 32; }
const void* stage_kernel_ptr() { return (const void*)stage_kernel; }

}  // namespace tgp
