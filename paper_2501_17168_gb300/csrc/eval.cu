// eval.cu -- population forward evaluation and MSE fitness (Sec. III-C).
//
// Work decomposition.  A work item is (a block of bt trees) x (a group of g
// consecutive point tiles of tp points).  A persistent grid of CTAs pulls
// items from an atomic counter; items are ordered tile-group-major so the
// CTAs running at the same time share the same X tiles in L2.  Per item:
//   1. one thread stages the block's compiled programs into shared memory
//      with bulk asynchronous copies (cp.async.bulk, completion on an
//      mbarrier); they stay there for all g tiles;
//   2. for every tile the CTA loads X (coalesced, transposed to
//      feature-major [F][tp] so a lane reads its points with 16-byte loads)
//      and the targets;
//   3. the warps pull (tree, 32*K-point chunk) sub-items, longest program
//      first, and run the tree's program over the chunk (K points per lane;
//      the interpreter's first memory-stack entry is a per-warp row of
//      shared memory, deeper entries are in local memory);
//   4. MSE mode: each chunk's squared residuals are summed in FP32 per lane
//      and across the warp with shuffles; chunk sums are folded into FP64
//      per-tree accumulators in a fixed order, so the result does not depend
//      on which warp ran which chunk; one FP64 partial per (tree, output,
//      tile group) goes to the workspace and a finalize kernel sums the
//      groups in order and divides by D.
//   Forward mode writes every output point instead.
#include "tgp_internal.cuh"
#include "isa_fwd.cuh"
#include "interp_fwd.cuh"

namespace tgp {

// ----------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// 1-D bulk copy global -> shared (TMA engine); bytes a multiple of 16, both
// addresses 16-byte aligned.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Bounded wait on an mbarrier phase, run by ONE thread of the CTA: gives up
// after max_polls polls (each poll itself suspends for a while; a negative
// limit gives up at once), records the error and reports failure.  The
// caller publishes the verdict through shared memory and a barrier so that
// every thread of the CTA leaves (or goes on) together.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* err,
                                                  int max_polls) {
  for (int it = 0; it < max_polls; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(err, (unsigned)ERR_MBAR_TIMEOUT);
  // give the copies still in flight a second bounded window to land before
  // the CTA (and its shared memory) goes away
  for (int it = 0; it < (1 << 20); ++it)
    if (mbar_try_wait(bar, parity)) break;
  return false;
}

// ----------------------------------------------------------- lane points
// A lane owns K points of a chunk of 32*K: the points 128*h + 4*lane +
// {0..3} for h < K/4, each group of four one 16-byte shared-memory load.
template <int K>
__device__ __forceinline__ void ld_pts(float (&v)[K], const float* p) {
#pragma unroll
  for (int h = 0; h < K / 4; ++h) {
    const float4 u = *reinterpret_cast<const float4*>(p + 128 * h);
    v[4 * h] = u.x; v[4 * h + 1] = u.y; v[4 * h + 2] = u.z; v[4 * h + 3] = u.w;
  }
}
template <int K>
__device__ __forceinline__ void st_pts(float* p, const float (&v)[K]) {
#pragma unroll
  for (int h = 0; h < K / 4; ++h)
    *reinterpret_cast<float4*>(p + 128 * h) = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
}
template <int K>
__device__ __forceinline__ int pt_index(int lane, int j) {
  return 128 * (j >> 2) + 4 * lane + (j & 3);
}

// ----------------------------------------------------------- smem layout
struct EvalSmem {
  size_t prog, xs, ys, mo, stk, cpart, tacc, order, lens, poff, misc, total;
  int xs_stride;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Words of the shared-memory program area of a block of bt trees: the
// programs are packed back to back; a block whose programs do not fit is
// evaluated in rounds (compiled programs average well below their capacity
// pcap, so one round is the rule).  Two words of padding follow the area
// (the interpreter prefetches the word after a program's end).
__host__ __device__ inline int prog_area_words(int bt, int pcap) {
  const long long full = (long long)bt * pcap;
  const long long half = full / 2 + pcap;
  return (int)((full < half ? full : half) + 1) & ~1;
}

__host__ __device__ inline EvalSmem eval_smem_layout(int K, int nw, bool modi, bool mse, int bt,
                                                     int pcap, int tp, int F, int O) {
  EvalSmem L;
  size_t off = 0;
  L.prog = off; off = align_up(off + ((size_t)prog_area_words(bt, pcap) + 2) * 8, 16);
  L.xs_stride = tp + 4;
  L.xs = off; off = align_up(off + (size_t)F * L.xs_stride * 4, 16);
  L.ys = off; off = align_up(off + (mse ? (size_t)O * tp * 4 : 0), 16);
  L.mo = off; off = align_up(off + (modi ? (size_t)nw * O * 32 * K * 4 : 0), 16);
  L.stk = off; off = align_up(off + (modi ? 0 : (size_t)nw * fx::NSM * 32 * K * 4), 16);  // memory-stack rows
  int cpt = tp / (32 * K);
  L.cpart = off; off = align_up(off + (size_t)bt * cpt * O * 4, 16);
  L.tacc = off; off = align_up(off + (size_t)bt * O * 8, 16);
  L.order = off; off = align_up(off + (size_t)bt * 4, 16);
  L.lens = off; off = align_up(off + (size_t)bt * 4, 16);
  L.poff = off; off = align_up(off + (size_t)bt * 4, 16);
  L.misc = off; off = align_up(off + 64, 16);
  L.total = off;
  return L;
}

// ----------------------------------------------------------- kernel
template <int K, int NW, bool MODI, bool OUT>
__global__ void __launch_bounds__(NW * 32, NW >= 16 ? 1 : (K >= 16 ? 2 : 3))
    eval_kernel(const __grid_constant__ EvalBatch b) {
  extern __shared__ __align__(16) unsigned char smem_all[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int CH = 32 * K;
  // fixed words first, the per-problem layout after them
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_all);
  long long* s_item = reinterpret_cast<long long*>(smem_all + 8);
  int* s_sub = reinterpret_cast<int*>(smem_all + 16);
  int* s_ok = reinterpret_cast<int*>(smem_all + 20);
  unsigned char* smem = smem_all + 64;
  const long long total = b.end[b.n - 1];

  // Return at once when this variant serves no problem of the batch (a
  // single-output population without a Modi node skips the Modi kernel and
  // vice versa), so the unused variant costs one short launch.
  if (tid == 0) {
    int served = 0;
    for (int i = 0; i < b.n; ++i) {
      const EvalArgs& q = b.p[i];
      served |= q.O > 1 ? (int)MODI
                        : (int)((*((volatile unsigned*)&q.ctrl[CTRL_ANY_MODI]) != 0) == MODI);
    }
    *s_sub = served;
    mbar_init(mbar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (*s_sub == 0) return;
  uint32_t phase = 0;

  for (;;) {
    if (tid == 0) *s_item = (long long)atomicAdd(b.counter, 1u);
    __syncthreads();
    const long long gitem = *s_item;
    if (gitem >= total) break;
    const int pi = batch_find(b.end, b.n, gitem);
    const EvalArgs& a = b.p[pi];
    const long long item = gitem - (pi ? b.end[pi - 1] : 0);
    // Which kernel serves a single-output population depends on whether the
    // stage pass found a Modi node; the other variant skips its items.
    if (a.O == 1) {
      const bool any_modi = *((volatile unsigned*)&a.ctrl[CTRL_ANY_MODI]) != 0;
      if (any_modi != MODI) {
        __syncthreads();
        continue;
      }
    }
    const EvalSmem lay = eval_smem_layout(K, NW, MODI, !OUT, a.bt, a.pcap, a.tp, a.F, a.O);
    uint2* prog_s = reinterpret_cast<uint2*>(smem + lay.prog);
    float* xs = reinterpret_cast<float*>(smem + lay.xs);
    float* ys = reinterpret_cast<float*>(smem + lay.ys);
    float* mo = reinterpret_cast<float*>(smem + lay.mo) + warp * a.O * CH;
    float* stk = reinterpret_cast<float*>(smem + lay.stk) + warp * fx::NSM * CH;
    float* cpart = reinterpret_cast<float*>(smem + lay.cpart);
    double* tacc = reinterpret_cast<double*>(smem + lay.tacc);
    int* order = reinterpret_cast<int*>(smem + lay.order);
    int* lens = reinterpret_cast<int*>(smem + lay.lens);
    int* poff = reinterpret_cast<int*>(smem + lay.poff);
    int* s_r1 = reinterpret_cast<int*>(smem + lay.misc);
    const int pw = prog_area_words(a.bt, a.pcap);
    const int XS = lay.xs_stride;
    const int cpt = a.tp / CH;
    const int O = a.O;
    const int grp = (int)(item / a.n_blocks);
    const long long blk = item - (long long)grp * a.n_blocks;
    const long long t0 = blk * a.bt;
    const int nt = (int)min((long long)a.bt, a.pop - t0);

    if (!OUT)
      for (int i = tid; i < nt * O; i += NW * 32) tacc[i] = 0.0;
    // rounds over the block: trees [r0, r1) whose programs fit the area
    for (int r0 = 0; r0 < nt;) {
      // 1. stage the round's programs, packed back to back
      if (tid == 0) {
        fence_proxy_async_smem();
        int off = 0, r1 = r0;
        for (; r1 < nt; ++r1) {
          const int w = (a.plen[t0 + r1] + 1) & ~1;
          if (r1 > r0 && off + w > pw) break;
          poff[r1] = off;
          off += w;
        }
        *s_r1 = r1;
        mbar_arrive_expect_tx(mbar, (uint32_t)off * 8u);
        for (int t = r0; t < r1; ++t) {
          const int L = a.plen[t0 + t];
          if (L > 0)
            bulk_g2s(prog_s + poff[t], a.prog + (size_t)(t0 + t) * a.pcap, (uint32_t)((L + 1) & ~1) * 8u,
                     mbar);
        }
      }
      __syncthreads();
      const int r1 = *s_r1;
      const int nr = r1 - r0;
      // longest program first
      for (int t = r0 + tid; t < r1; t += NW * 32) {
        int Lt = a.plen[t0 + t];
        int rank = 0;
        for (int u = r0; u < r1; ++u) {
          int Lu = a.plen[t0 + u];
          rank += (Lu > Lt) || (Lu == Lt && u < t);
        }
        order[rank] = t;
        lens[t] = Lt;
      }
      // one thread waits for the copies; the verdict reaches every thread
      // through shared memory, so the whole CTA returns (or goes on) together
      if (tid == 0) *s_ok = mbar_wait_bounded(mbar, phase, b.err, b.max_polls) ? 1 : 0;
      __syncthreads();
      if (*s_ok == 0) return;
      // every thread observes the completed phase itself (succeeds at once),
      // which orders its reads of the staged programs after the copies
      (void)mbar_try_wait(mbar, phase);
      phase ^= 1u;

      for (int gi = 0; gi < a.g; ++gi) {
        const long long tile = (long long)grp * a.g + gi;
        if (tile >= a.n_tiles) break;
        const long long p0 = tile * a.tp;
        const int np = (int)min((long long)a.tp, a.D - p0);

        // 2. X tile -> xs[f][q] (zero beyond D), targets -> ys[o][q]; rows of
        //    X are read with 16-byte loads when their layout allows
        {
          if (a.x_vec4) {
            const int F4 = a.F >> 2;
            const int fw = min(F4, 32), rows = 32 / fw, rr = lane / fw, ff = lane - rr * fw;
            for (int f0 = 0; f0 < F4; f0 += 32) {
              const int f4 = f0 + ff;
              const bool act = rr < rows && f4 < F4;
  #pragma unroll 2
              for (int r0 = warp * rows; r0 < a.tp; r0 += NW * rows) {
                const int q = r0 + rr;
                if (act && q < a.tp) {
                  float4 v = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                  if (q < np) v = __ldg(reinterpret_cast<const float4*>(a.X + (p0 + q) * a.ldx) + f4);
                  float* d = xs + 4 * f4 * XS + q;
                  d[0] = v.x; d[XS] = v.y; d[2 * XS] = v.z; d[3 * XS] = v.w;
                }
              }
            }
          } else {
            const int fw = min(a.F, 32), rows = 32 / fw, rr = lane / fw, ff = lane - rr * fw;
            for (int f0 = 0; f0 < a.F; f0 += 32) {
              const int f = f0 + ff;
              const bool act = rr < rows && f < a.F;
  #pragma unroll 4
              for (int r0 = warp * rows; r0 < a.tp; r0 += NW * rows) {
                const int q = r0 + rr;
                if (act && q < a.tp) {
                  float v = 0.0f;
                  if (q < np) v = __ldg(a.X + (p0 + q) * a.ldx + f);
                  xs[f * XS + q] = v;
                }
              }
            }
          }
          if (!OUT) {
            const int ow = min(O, 32), orows = 32 / ow, orr = lane / ow, off = lane - orr * ow;
            const bool oact = orr < orows;
  #pragma unroll 4
            for (int r0 = warp * orows; r0 < a.tp; r0 += NW * orows) {
              const int q = r0 + orr;
              if (oact && q < a.tp) {
                float v = 0.0f;
                if (q < np) v = __ldg(a.y + (p0 + q) * O + off);
                ys[off * a.tp + q] = v;
              }
            }
          }
        }
        if (tid == 0) *s_sub = 0;
        __syncthreads();

        // 3. sub-items: (tree, chunk), longest program first
        const int nch = (np + CH - 1) / CH;
        const int nsub = nr * nch;
        for (;;) {
          int s = 0;
          if (lane == 0) s = atomicAdd(s_sub, 1);
          s = __shfl_sync(0xffffffffu, s, 0);
          if (s >= nsub) break;
          const int t = order[s / nch];
          const int ch = s - (s / nch) * nch;
          const long long p = t0 + t;
          const int qbase = ch * CH;
          float res[K];
          bool modi_out = false;
          const bool valid = lens[t] > 0;
          if (valid) {
            if constexpr (MODI) {
              float z[K];
  #pragma unroll
              for (int j = 0; j < K; ++j) z[j] = 0.0f;
              for (int oo = 0; oo < O; ++oo) st_pts<K>(mo + oo * CH + 4 * lane, z);
            }
            modi_out = interp_fwd<K, MODI>(smem_u32(prog_s + poff[t]),
                                            smem_u32(xs + qbase + 4 * lane), (unsigned)XS * 4u,
                                            smem_u32(mo + 4 * lane), smem_u32(stk + 4 * lane), res) != 0;
          }
          if constexpr (!MODI) {
            // one output: the lane's points inside the data first, then its
            // squared residuals (or outputs) and the warp sum
            bool inb[K];
  #pragma unroll
            for (int j = 0; j < K; ++j) inb[j] = qbase + pt_index<K>(lane, j) < np;
            float v[K];
  #pragma unroll
            for (int j = 0; j < K; ++j) v[j] = valid ? res[j] : __int_as_float(0x7fc00000);
            if constexpr (OUT) {
              float* dst = a.out + p * a.D + p0;
  #pragma unroll
              for (int j = 0; j < K; ++j)
                if (inb[j]) dst[qbase + pt_index<K>(lane, j)] = v[j];
            } else {
              float yv[K];
              ld_pts<K>(yv, ys + qbase + 4 * lane);
              float sse = 0.0f;
  #pragma unroll
              for (int j = 0; j < K; ++j) {
                const float r = __fsub_rn(v[j], yv[j]);
                if (inb[j]) sse = fmaf(r, r, sse);
              }
  #pragma unroll
              for (int m = 16; m > 0; m >>= 1) sse += __shfl_xor_sync(0xffffffffu, sse, m);
              if (lane == 0) cpart[(t * cpt + ch) * O] = valid ? sse : 0.0f;
            }
          } else {
            for (int oo = 0; oo < O; ++oo) {
              float v[K];
              if (!valid) {
  #pragma unroll
                for (int j = 0; j < K; ++j) v[j] = __int_as_float(0x7fc00000);
              } else if (MODI && modi_out) {
                ld_pts<K>(v, mo + oo * CH + 4 * lane);
              } else {
  #pragma unroll
                for (int j = 0; j < K; ++j) v[j] = oo == 0 ? res[j] : 0.0f;
              }
              if constexpr (OUT) {
                float* dst = a.out + (p * O + oo) * a.D + p0;
  #pragma unroll
                for (int j = 0; j < K; ++j) {
                  const int q = qbase + pt_index<K>(lane, j);
                  if (q < np) dst[q] = v[j];
                }
              } else {
                float yv[K];
                ld_pts<K>(yv, ys + oo * a.tp + qbase + 4 * lane);
                float sse = 0.0f;
  #pragma unroll
                for (int j = 0; j < K; ++j) {
                  const int q = qbase + pt_index<K>(lane, j);
                  const float r = __fsub_rn(v[j], yv[j]);
                  if (q < np) sse = fmaf(r, r, sse);
                }
  #pragma unroll
                for (int m = 16; m > 0; m >>= 1) sse += __shfl_xor_sync(0xffffffffu, sse, m);
                if (lane == 0) cpart[(t * cpt + ch) * O + oo] = valid ? sse : 0.0f;
              }
            }
          }
        }
        __syncthreads();
        // 4. fold chunk sums into the per-tree FP64 accumulators in chunk order
        if (!OUT) {
          for (int i = r0 * O + tid; i < r1 * O; i += NW * 32) {
            const int t = i / O, oo = i - (i / O) * O;
            double acc = tacc[i];
            for (int ch = 0; ch < nch; ++ch) acc += (double)cpart[(t * cpt + ch) * O + oo];
            tacc[i] = acc;
          }
          __syncthreads();
        }
      }
      r0 = r1;
    }
    if (!OUT) {
      for (int i = tid; i < nt * O; i += NW * 32) {
        const int t = i / O, oo = i - (i / O) * O;
        a.partial[((t0 + t) * O + oo) * a.n_groups + grp] = tacc[i];
      }
    }
    __syncthreads();
  }
}

// MSE[p,k] = (sum of the tile-group partials in order) / D (the sum itself in
// SSE mode); NaN for invalid trees.
__global__ void finalize_kernel(const __grid_constant__ FinalBatch b) {
  const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= b.end[b.n - 1]) return;
  const int pi = batch_find(b.end, b.n, gi);
  const FinalArgs& a = b.p[pi];
  const long long i = gi - (pi ? b.end[pi - 1] : 0);
  const long long p = i / a.O;
  double s = 0.0;
  const double* src = a.partial + i * a.n_groups;
  for (int g = 0; g < a.n_groups; ++g) s += src[g];
  a.mse[i] = a.status[p] != 0 ? __longlong_as_double(0x7ff8000000000000ll)
                               : (a.sse ? s : s / (double)a.D);
}

// ----------------------------------------------------------- host-side table
struct EvalKernelInfo {
  const void* fn;
  int K, nw;
  bool modi, out;
};

#define TGP_EVAL_INST(K, NW, M, O) {(const void*)eval_kernel<K, NW, M, O>, K, NW, M, O}
static const EvalKernelInfo kEvalKernels[] = {
    TGP_EVAL_INST(8, 32, false, false), TGP_EVAL_INST(8, 8, false, false),
    TGP_EVAL_INST(4, 8, false, false),  TGP_EVAL_INST(4, 28, true, false),
    TGP_EVAL_INST(4, 16, true, false),  TGP_EVAL_INST(4, 8, true, false),
    TGP_EVAL_INST(8, 32, false, true),  TGP_EVAL_INST(8, 8, false, true),
    TGP_EVAL_INST(4, 8, false, true),   TGP_EVAL_INST(4, 28, true, true),
    TGP_EVAL_INST(4, 16, true, true),   TGP_EVAL_INST(4, 8, true, true),
};
#undef TGP_EVAL_INST

const void* find_eval_kernel(int K, int nw, bool modi, bool out) {
  for (const auto& k : kEvalKernels)
    if (k.K == K && k.nw == nw && k.modi == modi && k.out == out) return k.fn;
  return nullptr;
}

size_t eval_smem_bytes(int K, int nw, bool modi, bool mse, int bt, int pcap, int tp, int F, int O) {
  return 64 + eval_smem_layout(K, nw, modi, mse, bt, pcap, tp, F, O).total;
}

const void* finalize_kernel_ptr() { return (const void*)finalize_kernel; }

}  // namespace tgp
