// adjoint.cu -- fused forward + reverse-mode gradient of the population MSE
// (the adjoint is not in the paper; it differentiates the Sec. III-C fitness
// of the Sec. II-A / IV-C tree semantics).
//
// Loss L = sum_{p,k} g[p,k] * MSE[p,k].  Work decomposition: a work item is a
// tile of tp data points and a range of trees (the population split into
// tree_chunks ranges), owned by one CTA, which sweeps the range over the
// tile.  The gradient of X for the tile's points is accumulated in shared
// memory (by every warp, with shared-memory reductions) and written back
// once per item: a plain read-modify-write when one item covers the whole
// population, else global float atomics (one per point and feature per
// item).  Large tiles amortise the per-(tree, tile) work (staging the
// program, clearing and flushing the constant gradients); splitting the
// population keeps enough items for the persistent grid.  Warps work
// independently: each pulls a tree of the range (starting at a
// tile-dependent offset so concurrent CTAs touch different trees), copies
// its compiled program into its own shared-memory slot, and for every
// 32*K-point chunk of the tile
//   1. runs the program forward, writing the local partials the reverse
//      needs to a per-thread tape in local memory (at most one entry per
//      node, so no population x length x points activations are stored);
//   2. forms the seeds dL/d(output) = 2 g (o - y) / D at the valid points;
//   3. runs the program backward (interp_bwd.cuh).
// Constant gradients are summed per warp and node in shared memory over the
// tile and added once per (tree, tile) into an FP64 workspace array; the MSE
// is accumulated the same way.  A final kernel converts to the outputs.
#include "tgp_internal.cuh"
#include "interp_bwd.cuh"

namespace tgp {

__device__ __forceinline__ uint32_t sm_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

struct AdjSmem {
  size_t xs, gx, ys, warp, total;
  size_t per_warp, w_prog, w_cg, w_mo, w_sd, w_g2, w_slot;
  int xs_stride;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) / 16 * 16; }

__host__ __device__ inline AdjSmem adj_smem_layout(int K, int nw, bool modi, int pcap, int max_len, int tp,
                                                   int F, int O) {
  AdjSmem L;
  L.xs_stride = tp + 4;
  size_t off = 0;
  L.xs = off; off = al16(off + (size_t)F * L.xs_stride * 4);
  L.gx = off; off = al16(off + (size_t)F * L.xs_stride * 4);
  L.ys = off; off = al16(off + (size_t)O * tp * 4);
  // per warp: 16-byte pad (the reverse prefetch reads one word below the
  // program), program, constant-gradient row, Modi outputs, seeds, 2g/D
  size_t w = 0;
  L.w_prog = 16; w = al16(16 + (size_t)pcap * 8);
  L.w_cg = w; w = al16(w + (size_t)max_len * 4);
  // the Modi outputs of the forward; each output's seed of the reverse
  // overwrites it once read
  L.w_mo = w; w = al16(w + (modi ? (size_t)O * 32 * K * 4 : 0));
  L.w_sd = L.w_mo;
  L.w_g2 = w; w = al16(w + (size_t)O * 4);
  L.w_slot = w; w = al16(w + (size_t)R * 32 * K * 4);  // register-machine slots
  L.per_warp = w;
  L.warp = off; off = al16(off + (size_t)nw * w);
  off = al16(off + 64);  // item / tree counters
  L.total = off;
  return L;
}

// The lane's K points of a chunk, 128 (j / 4) + 4 lane + j % 4 (p points at
// the lane's first one): K / 4 16-byte shared-memory accesses.
template <int K>
__device__ __forceinline__ void ld_lane_pts(float (&v)[K], const float* p) {
#pragma unroll
  for (int h = 0; h < K / 4; ++h) {
    const float4 u = *reinterpret_cast<const float4*>(p + 128 * h);
    v[4 * h] = u.x; v[4 * h + 1] = u.y; v[4 * h + 2] = u.z; v[4 * h + 3] = u.w;
  }
}
template <int K>
__device__ __forceinline__ void st_lane_pts(float* p, const float (&v)[K]) {
#pragma unroll
  for (int h = 0; h < K / 4; ++h)
    *reinterpret_cast<float4*>(p + 128 * h) = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
}

template <int K, int NW, bool MODI, int CAP>
__global__ void __launch_bounds__(NW * 32, NW > 8 ? 1 : 3) adjoint_kernel(AdjArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int CH = 32 * K;
  if (a.O == 1) {
    const bool any_modi = *((volatile unsigned*)&a.ctrl[CTRL_ANY_MODI]) != 0;
    if (any_modi != MODI) return;
  }
  const AdjSmem lay = adj_smem_layout(K, NW, MODI, a.pcap, a.max_len, a.tp, a.F, a.O);
  float* xs = reinterpret_cast<float*>(smem + lay.xs);
  float* gxs = reinterpret_cast<float*>(smem + lay.gx);
  float* ys = reinterpret_cast<float*>(smem + lay.ys);
  unsigned char* wbase = smem + lay.warp + (size_t)warp * lay.per_warp;
  uint2* prog_w = reinterpret_cast<uint2*>(wbase + lay.w_prog);
  float* cg_w = reinterpret_cast<float*>(wbase + lay.w_cg);
  float* mo_w = reinterpret_cast<float*>(wbase + lay.w_mo);
  float* sd_w = reinterpret_cast<float*>(wbase + lay.w_sd);
  float* g2_w = reinterpret_cast<float*>(wbase + lay.w_g2);
  float* slot_w = reinterpret_cast<float*>(wbase + lay.w_slot);
  int* s_item = reinterpret_cast<int*>(smem + lay.total - 64);
  int* s_tree = s_item + 1;
  const int XS = lay.xs_stride;
  const int O = a.O;
  float tape[CAP * K];
  const unsigned tape_addr = (unsigned)__cvta_generic_to_local(tape);

  for (;;) {
    if (tid == 0) {
      *s_item = (int)atomicAdd(&a.ctrl[CTRL_COUNTER], 1u);
      *s_tree = 0;
    }
    __syncthreads();
    const int item = *s_item;
    if (item >= a.n_tiles * a.tree_chunks) break;
    // tree-range-major: the items of one tile run at different times
    const int tc = item / a.n_tiles, tile = item - tc * a.n_tiles;
    const long long tr0 = (long long)tc * a.trees_per_chunk;
    const long long tr1 = min(a.pop, tr0 + a.trees_per_chunk);
    const long long ntr = tr1 - tr0;
    const long long p0 = (long long)tile * a.tp;
    const int np = (int)min((long long)a.tp, a.D - p0);
    // X tile (rows past the end repeat the last point so that padded lanes
    // compute finite values; their seeds are zero), zeroed gradient tile, y
    for (int i = tid; i < a.F * a.tp; i += NW * 32) {
      const int q = i / a.F, f = i - (i / a.F) * a.F;
      const int qq = q < np ? q : np - 1;
      xs[f * XS + q] = __ldg(a.X + (p0 + qq) * a.ldx + f);
      gxs[f * XS + q] = 0.0f;
    }
    for (int i = tid; i < O * a.tp; i += NW * 32) {
      const int o = i / a.tp, q = i - (i / a.tp) * a.tp;
      ys[o * a.tp + q] = q < np ? __ldg(a.y + (p0 + q) * O + o) : 0.0f;
    }
    __syncthreads();
    const int nch = (np + CH - 1) / CH;
    const long long stagger = (long long)tile * 7919;  // spread concurrent CTAs over trees
    for (;;) {
      int t = 0;
      if (lane == 0) t = atomicAdd(s_tree, 1);
      t = __shfl_sync(0xffffffffu, t, 0);
      if ((long long)t >= ntr) break;
      const long long p = tr0 + (t + stagger) % ntr;
      const int plen = a.plen[p];
      if (plen <= 0) continue;
      // a tree with zero upstream gradient only needs the forward (for its
      // MSE); its reverse sweep is skipped, so that 0 * inf seeds of points
      // where it overflows cannot put NaN into the shared X gradient
      bool any_g = false;
      for (int o = 0; o < O; ++o) any_g |= a.g[p * O + o] != 0.0;
      if (!any_g && !a.want_mse) continue;
      // stage the program, clear the constant-gradient row, 2g/D per output
      for (int i = lane; i < plen; i += 32) prog_w[i] = a.prog[p * a.pcap + i];
      for (int i = lane; i < a.max_len; i += 32) cg_w[i] = 0.0f;
      for (int o = lane; o < O; o += 32) g2_w[o] = (float)(a.g[p * O + o] * a.two_over_D);
      __syncwarp();
      float sse[MAX_OUT];
#pragma unroll
      for (int o = 0; o < MAX_OUT; ++o) sse[o] = 0.0f;
      for (int ch = 0; ch < nch; ++ch) {
        const int qb = ch * CH + 4 * lane;
        if constexpr (MODI) {
          float z[K];
#pragma unroll
          for (int j = 0; j < K; ++j) z[j] = 0.0f;
          for (int o = 0; o < O; ++o) st_lane_pts<K>(mo_w + o * CH + 4 * lane, z);
        }
        __syncwarp();
        float acc[K];
        unsigned tend = tape_addr;
        const unsigned flag = bwd_forward<K, MODI>(sm_addr(prog_w), sm_addr(xs + qb), (unsigned)XS * 4u,
                                                   sm_addr(mo_w + 4 * lane), tape_addr,
                                                   sm_addr(slot_w + 4 * lane), acc, tend);
        float seed[K];
#pragma unroll
        for (int j = 0; j < K; ++j) seed[j] = 0.0f;
        for (int o = 0; o < O; ++o) {
          float v[K];
          if (MODI && flag) {
            ld_lane_pts<K>(v, mo_w + o * CH + 4 * lane);
          } else {
#pragma unroll
            for (int j = 0; j < K; ++j) v[j] = o == 0 ? acc[j] : 0.0f;
          }
          float yv[K];
          ld_lane_pts<K>(yv, ys + o * a.tp + qb);
          const float g2 = g2_w[o];
          float sv[K];
#pragma unroll
          for (int j = 0; j < K; ++j) {
            // the lane's point j of the chunk: 128 (j / 4) + 4 lane + j % 4
            const bool ok = qb + 128 * (j >> 2) + (j & 3) < np;
            const float r = __fsub_rn(v[j], yv[j]);
            if (ok) sse[o] = fmaf(r, r, sse[o]);
            sv[j] = ok ? __fmul_rn(g2, r) : 0.0f;
          }
          if (MODI && flag) {
            st_lane_pts<K>(sd_w + o * CH + 4 * lane, sv);
          } else if (o == 0) {
#pragma unroll
            for (int j = 0; j < K; ++j) seed[j] = sv[j];
          }
        }
        __syncwarp();
        if (any_g)
          bwd_reverse<K, MODI>(sm_addr(prog_w + (plen - 1)), sm_addr(prog_w), sm_addr(xs + qb),
                               (unsigned)XS * 4u, sm_addr(gxs + ch * CH + lane), sm_addr(cg_w),
                               sm_addr(sd_w + 4 * lane), tend, (unsigned)lane,
                               sm_addr(slot_w + 4 * lane), seed);
        __syncwarp();
      }
      // flush the tree's constant gradients and squared residuals
      for (int i = lane; i < a.max_len; i += 32) {
        const float v = cg_w[i];
        if (v != 0.0f) atomicAdd(&a.gval64[p * a.max_len + i], (double)v);
      }
      for (int o = 0; o < O && o < MAX_OUT; ++o) {
        float s = sse[o];
#pragma unroll
        for (int m = 16; m > 0; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
        if (lane == 0 && a.want_mse) atomicAdd(&a.mse64[p * O + o], (double)s);
      }
      __syncwarp();
    }
    __syncthreads();
    // the tile's gradient of X over the item's trees: a plain update when
    // this CTA owns the points, atomics when other tree ranges add to them
    if (a.grad_X) {
      for (int i = tid; i < np * a.F; i += NW * 32) {
        const int q = i / a.F, f = i - (i / a.F) * a.F;
        // tile layout [f][chunk][j][lane]: point q = chunk*CH + 128*(j/4) +
        // 4*lane + j%4
        const int c = q / CH, r = q - c * CH, h = r >> 7, rr = r & 127;
        const float v = gxs[f * XS + c * CH + (4 * h + (rr & 3)) * 32 + (rr >> 2)];
        float* dst = a.grad_X + (p0 + q) * a.F + f;
        if (a.tree_chunks == 1) *dst += v;
        else if (v != 0.0f) atomicAdd(dst, v);
      }
    }
    __syncthreads();
  }
}

__global__ void adj_finalize_kernel(AdjFinalArgs a) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n_val = a.pop * a.ld;
  if (a.grad_value && i < n_val) {
    const long long p = i / a.ld, k = i - p * a.ld;
    float v = 0.0f;
    if (a.status[p] != 0) v = __int_as_float(0x7fc00000);
    else if (k < a.max_len) v = (float)a.gval64[p * a.max_len + k];
    a.grad_value[i] = v;
  }
  if (a.mse && i < a.pop * a.O) {
    const long long p = i / a.O;
    a.mse[i] = a.status[p] != 0 ? __longlong_as_double(0x7ff8000000000000ll) : a.mse64[i] / (double)a.D;
  }
}

// ----------------------------------------------------------- host-side table
struct AdjKernelInfo {
  const void* fn;
  int K, nw, cap;
  bool modi;
};

#define TGP_ADJ_INST(K, NW, M, C) {(const void*)adjoint_kernel<K, NW, M, C>, K, NW, C, M}
static const AdjKernelInfo kAdjKernels[] = {
    TGP_ADJ_INST(4, 32, false, 128), TGP_ADJ_INST(4, 32, false, 256), TGP_ADJ_INST(4, 32, false, 1024),
    TGP_ADJ_INST(4, 32, true, 128),  TGP_ADJ_INST(4, 32, true, 256),  TGP_ADJ_INST(4, 32, true, 1024),
    TGP_ADJ_INST(4, 16, false, 128), TGP_ADJ_INST(4, 16, false, 256), TGP_ADJ_INST(4, 16, false, 1024),
    TGP_ADJ_INST(4, 16, true, 128),  TGP_ADJ_INST(4, 16, true, 256),  TGP_ADJ_INST(4, 16, true, 1024),
    TGP_ADJ_INST(4, 8, false, 128),  TGP_ADJ_INST(4, 8, false, 256),  TGP_ADJ_INST(4, 8, false, 1024),
    TGP_ADJ_INST(4, 8, true, 128),   TGP_ADJ_INST(4, 8, true, 256),   TGP_ADJ_INST(4, 8, true, 1024),
};
#undef TGP_ADJ_INST

const void* find_adj_kernel(int K, int nw, bool modi, int max_len, int* cap_out) {
  for (const auto& k : kAdjKernels)
    if (k.K == K && k.nw == nw && k.modi == modi && k.cap >= max_len) {
      *cap_out = k.cap;
      return k.fn;
    }
  return nullptr;
}

size_t adj_smem_bytes(int K, int nw, bool modi, int pcap, int max_len, int tp, int F, int O) {
  return adj_smem_layout(K, nw, modi, pcap, max_len, tp, F, O).total;
}

const void* adj_finalize_ptr() { return (const void*)adj_finalize_kernel; }

}  // namespace tgp
