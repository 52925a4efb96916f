// genetic.cu -- population-parallel genetic operators on the three-tensor
// encoding: the subtree exchange of Sec. III-B (one-point crossover, subtree
// mutation and hoist mutation are the same primitive with different node
// choices), tournament selection (Algorithm 1, "Select parents") and the
// classification accuracy of Sec. V-D.  All three are HBM-bound gathers or
// small reductions: one warp per child (or per selection), lanes striding
// over consecutive positions so that every load and store of a row is
// coalesced, grids sized to the SM count.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/tgp.h"

namespace tgp {
namespace {

constexpr int kWarps = 8;  // warps per CTA of the exchange / tournament kernels

// ------------------------------------------------------------- exchange
struct XchgArgs {
  const float *ot, *ov, *os;  // old population
  long long o_pop, o_ld;
  int o_max_len;
  const float *dt, *dv, *ds;  // donor population (== old in hoist mode)
  long long d_pop, d_ld;
  int d_max_len;
  const int32_t* old_index;
  const uint32_t* node;
  const int32_t* donor_index;  // null in hoist mode
  const uint32_t* donor_node;  // null = 0
  const uint32_t* apply_word;  // null = every child takes part
  uint32_t apply_below;
  long long n;
  int mode;
  int max_size;
  float *xt, *xv, *xs;  // children [n, out_ld]
  long long out_ld;
  int32_t* status;  // [n] or null
};

// x as a count if it is an integer in [1, hi], else 0.  hi <= 2^24, so every
// candidate is exact in float.
__device__ __forceinline__ int as_count(float x, int hi) {
  if (!(x >= 1.0f && x <= (float)hi)) return 0;
  const int c = (int)x;
  return (float)c == x ? c : 0;
}

// Where child i's row comes from: positions [0, s) from the old row at o_off
// (subtree sizes of the ancestors of s grown by dn), [s, s+m) from the donor
// at q_off (the inserted subtree), [s+m, nl) from the old row again starting
// at e, NaN from nl on.  A node p < s is an ancestor of s exactly when its
// subtree reaches past s (p + size[p] > s).
struct Plan {
  int s, m, e, nl, dn;
  long long o_off, q_off;
};

// The checks and node choices of one child, in the order the header lists
// them (these few loads form a dependent chain per child).
__device__ __forceinline__ int plan_child(const XchgArgs& a, long long i, Plan& pl) {
  pl = Plan{0, 0, 0, 0, 0, 0, 0};
  const long long ai = __ldg(a.old_index + i);
  const unsigned r = __ldg(a.node + i);
  const unsigned r2 = a.donor_node ? __ldg(a.donor_node + i) : 0u;
  const unsigned aw = a.apply_word ? __ldg(a.apply_word + i) : 0u;
  const long long bi_in = a.mode == TGP_PICK_HOIST ? ai : (long long)__ldg(a.donor_index + i);
  if (ai < 0 || ai >= a.o_pop) return TGP_XCHG_BAD_INDEX;
  const float* rs = a.os + ai * a.o_ld;
  pl.o_off = ai * a.o_ld;
  const int n_old = as_count(__ldg(rs), a.o_max_len);
  if (!n_old) return TGP_XCHG_BAD_TREE;
  if (a.apply_word && aw >= a.apply_below) {
    pl.s = pl.e = pl.nl = n_old;
    return TGP_XCHG_SKIPPED;
  }
  // in hoist mode the donor arrays are the old ones (set on the host)
  if (bi_in < 0 || bi_in >= a.d_pop) return TGP_XCHG_BAD_INDEX;
  const int dml = a.mode == TGP_PICK_HOIST ? a.o_max_len : a.d_max_len;
  const float* qs = a.ds + bi_in * a.d_ld;
  const int n_don = as_count(__ldg(qs), dml);
  if (!n_don) return TGP_XCHG_BAD_TREE;
  const unsigned k = a.mode == TGP_PICK_NODES ? r : r % (unsigned)n_old;
  if (k >= (unsigned)n_old) return TGP_XCHG_BAD_INDEX;
  const int sub_old = as_count(__ldg(rs + k), n_old - (int)k);
  if (!sub_old) return TGP_XCHG_BAD_TREE;
  const unsigned j = a.mode == TGP_PICK_NODES    ? r2
                     : a.mode == TGP_PICK_RANDOM ? r2 % (unsigned)n_don
                                                 : k + r2 % (unsigned)sub_old;
  if (j >= (unsigned)n_don) return TGP_XCHG_BAD_INDEX;
  const int m = as_count(__ldg(qs + j), n_don - (int)j);
  if (!m) return TGP_XCHG_BAD_TREE;
  if (n_old - sub_old + m > a.max_size) {  // the paper's size rule: keep T_old
    pl.s = pl.e = pl.nl = n_old;
    return TGP_XCHG_TOO_LARGE;
  }
  pl.s = (int)k;
  pl.m = m;
  pl.e = (int)k + sub_old;
  pl.nl = n_old - sub_old + m;
  pl.dn = m - sub_old;
  pl.q_off = bi_in * a.d_ld + j;
  return TGP_XCHG_DONE;
}

// A warp takes `cpt` consecutive children.  Lane c plans child c (so the
// header loads of all of them are in flight together) and writes its status;
// then the warp writes the rows one child at a time, each lane covering
// positions lane + 32u, 8 per pass so that 24 loads are in flight per lane.
// Rows of invalid children are all NaN.
__global__ void __launch_bounds__(kWarps * 32, 4) exchange_kernel(XchgArgs a, int cpt) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * kWarps;
  const float nan = __int_as_float(0x7fc00000);
  for (long long task = (long long)blockIdx.x * kWarps + (threadIdx.x >> 5); task * cpt < a.n;
       task += nwarps) {
    const long long i0 = task * cpt;
    const int cnt = (int)(a.n - i0 < cpt ? a.n - i0 : cpt);
    Plan mine{0, 0, 0, 0, 0, 0, 0};
    if (lane < cnt) {
      const int st = plan_child(a, i0 + lane, mine);
      if (st == TGP_XCHG_BAD_INDEX || st == TGP_XCHG_BAD_TREE) mine = Plan{0, 0, 0, 0, 0, 0, 0};
      if (a.status) a.status[i0 + lane] = st;
    }
    for (int c = 0; c < cnt; ++c) {
      const int s = __shfl_sync(0xffffffffu, mine.s, c);
      const int m = __shfl_sync(0xffffffffu, mine.m, c);
      const int e = __shfl_sync(0xffffffffu, mine.e, c);
      const int nl = __shfl_sync(0xffffffffu, mine.nl, c);
      const float fdn = (float)__shfl_sync(0xffffffffu, mine.dn, c);
      const long long o_off = __shfl_sync(0xffffffffu, mine.o_off, c);
      const long long q_off = __shfl_sync(0xffffffffu, mine.q_off, c);
      const float *rt = a.ot + o_off, *rv = a.ov + o_off, *rs = a.os + o_off;
      const float *qt = a.dt + q_off, *qv = a.dv + q_off, *qs = a.ds + q_off;
      const long long row = (i0 + c) * a.out_ld;
      float* xt = a.xt + row;
      float* xv = a.xv + row;
      float* xs = a.xs + row;
      for (int base = 0; base < (int)a.out_ld; base += 256) {
        float t[8], v[8], z[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int p = base + lane + 32 * u;
          t[u] = v[u] = z[u] = nan;
          if (p < s) {
            t[u] = __ldg(rt + p);
            v[u] = __ldg(rv + p);
            z[u] = __ldg(rs + p);
            if (z[u] > (float)(s - p)) z[u] += fdn;
          } else if (p < s + m) {
            t[u] = __ldg(qt + (p - s));
            v[u] = __ldg(qv + (p - s));
            z[u] = __ldg(qs + (p - s));
          } else if (p < nl) {
            const int q = e + (p - s - m);
            t[u] = __ldg(rt + q);
            v[u] = __ldg(rv + q);
            z[u] = __ldg(rs + q);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int p = base + lane + 32 * u;
          if (p < (int)a.out_ld) {
            xt[p] = t[u];
            xv[p] = v[u];
            xs[p] = z[u];
          }
        }
      }
    }
  }
}

// ------------------------------------------------------------ tournament
struct TournArgs {
  const double* fit;
  long long stride;
  long long P;
  const uint32_t* words;  // [n, t]
  long long n;
  int t;
  int minimize;
  int32_t* winners;
};

// One thread per selection: the contestants' words and fitness values are
// independent loads, so a thread has all of them in flight before it scans
// them in draw order, keeping the first best (a number beats NaN).
__global__ void __launch_bounds__(256) tournament_kernel(TournArgs a) {
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const unsigned P = (unsigned)a.P;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += nthreads) {
    const uint32_t* w = a.words + i * a.t;
    unsigned bc = __ldg(w) % P;
    double bv = __ldg(a.fit + (long long)bc * a.stride);
    for (int m0 = 1; m0 < a.t; m0 += 8) {
      unsigned c[8];
      double f[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (m0 + u < a.t) c[u] = __ldg(w + m0 + u) % P;
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (m0 + u < a.t) f[u] = __ldg(a.fit + (long long)c[u] * a.stride);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (m0 + u >= a.t || isnan(f[u])) continue;
        if (isnan(bv) || (a.minimize ? f[u] < bv : f[u] > bv)) bv = f[u], bc = c[u];
      }
    }
    a.winners[i] = (int32_t)bc;
  }
}

// -------------------------------------------------------------- accuracy
struct AccArgs {
  const float* out;  // [P, C, ld]: output k of tree p at point d is out[(p*C + k)*ld + d]
  long long P;
  int C;
  long long D;  // points in this call
  long long ld;
  const int32_t* labels;  // [D]
  unsigned long long* cnt;  // [P], accumulated
  long long nblk;           // point blocks of 256 per tree
};

// One CTA-sized block of 256 points of one tree per item: each thread takes
// one point, reads its C outputs (coalesced along the points), predicts the
// first index of the largest non-NaN output and compares it with the label;
// the CTA adds its count to the tree's total.
__global__ void __launch_bounds__(256) accuracy_count_kernel(AccArgs a) {
  const long long items = a.P * a.nblk;
  for (long long it = blockIdx.x; it < items; it += gridDim.x) {
    const long long p = it / a.nblk;
    const long long d = (it % a.nblk) * 256 + threadIdx.x;
    int ok = 0;
    if (d < a.D) {
      int pred = -1;
      float best = 0.0f;
      const float* o = a.out + p * a.C * a.ld + d;
      for (int k = 0; k < a.C; ++k) {
        const float v = __ldg(o + (long long)k * a.ld);
        if (v == v && (pred < 0 || v > best)) pred = k, best = v;
      }
      ok = pred >= 0 && pred == __ldg(a.labels + d);
    }
    const int total = __syncthreads_count(ok);
    if (threadIdx.x == 0 && total) atomicAdd(a.cnt + p, (unsigned long long)total);
  }
}

__global__ void accuracy_final_kernel(const unsigned long long* cnt, long long P, long long D,
                                      const int32_t* status, double* acc) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  acc[p] = (status && status[p] != 0) ? __longlong_as_double(0x7ff8000000000000LL)
                                      : (double)cnt[p] / (double)D;
}

// ----------------------------------------------------------------- host
inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }
inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

int sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(mu);
  if (!cache[dev] &&
      cudaDeviceGetAttribute(&cache[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    cache[dev] = 0;
  return cache[dev];
}

bool pop_shape_ok(const tgp_population* p) {
  if (!p || p->pop < 0 || p->max_len < 1 || p->max_len > TGP_MAX_LEN || p->ld < p->max_len)
    return false;
  return p->pop == 0 || (p->type && p->value && p->size);
}

bool overlaps(const void* a, size_t an, const void* b, size_t bn) {
  const char *x = (const char*)a, *y = (const char*)b;
  return an && bn && x < y + bn && y < x + an;
}

size_t rows_bytes(const tgp_population* p) { return p->pop > 0 ? (size_t)p->pop * p->ld * 4 : 0; }

// Accuracy of forward outputs [P, C, ld] for D points into cnt (accumulated).
tgp_status launch_count(const float* out, long long P, int C, long long D, long long ld,
                        const int32_t* labels, unsigned long long* cnt, cudaStream_t st) {
  if (P == 0 || D == 0) return TGP_OK;
  const int sms = sm_count();
  if (!sms) return TGP_ERR_CUDA;
  AccArgs a{out, P, C, D, ld, labels, cnt, cdiv(D, 256)};
  long long grid = P * a.nblk;
  if (grid > (long long)sms * 8 * 4) grid = (long long)sms * 8 * 4;
  accuracy_count_kernel<<<(unsigned)grid, 256, 0, st>>>(a);
  return cudaGetLastError() == cudaSuccess ? TGP_OK : TGP_ERR_CUDA;
}

tgp_status launch_acc_final(const unsigned long long* cnt, long long P, long long D,
                            const int32_t* status, double* acc, cudaStream_t st) {
  if (P == 0 || !acc) return TGP_OK;
  accuracy_final_kernel<<<(unsigned)cdiv(P, 256), 256, 0, st>>>(cnt, P, D, status, acc);
  return cudaGetLastError() == cudaSuccess ? TGP_OK : TGP_ERR_CUDA;
}

// Points per forward chunk of the fused accuracy: the [P, C, chunk] output
// buffer stays within 256 MiB (at least 256 points, at most D).
long long acc_chunk(long long P, int C, long long D) {
  const long long per_point = (P > 0 ? P : 1) * C * 4;
  long long c = (256LL << 20) / per_point;
  if (c < 256) c = 256;
  c = c / 256 * 256;
  return c < D ? c : D;
}

struct AccWs {
  size_t fwd, out, cnt, st, total;
  long long chunk;
};

bool acc_ws(const tgp_population* pop, const tgp_data* data, int C, AccWs* w) {
  const size_t fwd = tgp_workspace_size(pop, nullptr, C, nullptr);
  if (!fwd) return false;
  w->chunk = acc_chunk(pop->pop, C, data->n_points);
  w->fwd = 0;
  w->out = al256(fwd);
  w->cnt = w->out + al256((size_t)pop->pop * C * w->chunk * 4);
  w->st = w->cnt + al256((size_t)pop->pop * 8);
  w->total = w->st + al256((size_t)pop->pop * 4);
  return true;
}

}  // namespace
}  // namespace tgp

using namespace tgp;

extern "C" {

tgp_status tgp_subtree_exchange(const tgp_population* old, const tgp_population* donor,
                                const int32_t* old_index, const uint32_t* node,
                                const int32_t* donor_index, const uint32_t* donor_node,
                                const uint32_t* apply_word, uint32_t apply_below, int64_t n,
                                int32_t mode, int32_t max_size, float* out_type, float* out_value,
                                float* out_size, int64_t out_ld, int32_t* xchg_status,
                                void* stream) {
  if (mode != TGP_PICK_NODES && mode != TGP_PICK_RANDOM && mode != TGP_PICK_HOIST)
    return TGP_ERR_INVALID_ARG;
  const bool hoist = mode == TGP_PICK_HOIST;
  if (!pop_shape_ok(old) || (!hoist && !pop_shape_ok(donor)) || n < 0) return TGP_ERR_INVALID_ARG;
  if (max_size < 1 || max_size > TGP_MAX_LEN || out_ld < max_size || out_ld < old->max_len ||
      out_ld > (1LL << 24))
    return TGP_ERR_INVALID_ARG;
  if (n == 0) return TGP_OK;
  if (!old_index || !node || (!hoist && !donor_index) || !out_type || !out_value || !out_size)
    return TGP_ERR_INVALID_ARG;
  // children are written out of place: no output row may overlap an input row
  const size_t ob = (size_t)n * out_ld * 4;
  const tgp_population* ins[2] = {old, hoist ? nullptr : donor};
  for (const tgp_population* p : ins) {
    if (!p) continue;
    const void* in[3] = {p->type, p->value, p->size};
    float* outs[3] = {out_type, out_value, out_size};
    for (const void* x : in)
      for (float* y : outs)
        if (overlaps(x, rows_bytes(p), y, ob)) return TGP_ERR_INVALID_ARG;
  }
  if (overlaps(out_type, ob, out_value, ob) || overlaps(out_type, ob, out_size, ob) ||
      overlaps(out_value, ob, out_size, ob))
    return TGP_ERR_INVALID_ARG;
  const int sms = sm_count();
  if (!sms) return TGP_ERR_CUDA;
  XchgArgs a;
  a.ot = old->type, a.ov = old->value, a.os = old->size;
  a.o_pop = old->pop, a.o_ld = old->ld, a.o_max_len = old->max_len;
  const tgp_population* d = hoist ? old : donor;
  a.dt = d->type, a.dv = d->value, a.ds = d->size;
  a.d_pop = d->pop, a.d_ld = d->ld, a.d_max_len = d->max_len;
  a.old_index = old_index;
  a.node = node;
  a.donor_index = hoist ? nullptr : donor_index;
  a.donor_node = donor_node;
  a.apply_word = apply_word;
  a.apply_below = apply_below;
  a.n = n;
  a.mode = mode;
  a.max_size = max_size;
  a.xt = out_type, a.xv = out_value, a.xs = out_size;
  a.out_ld = out_ld;
  a.status = xchg_status;
  // One wave of warps (4 resident CTAs of 8 warps per SM), each taking
  // enough consecutive children (1..32) to cover all of them.
  const long long warps = (long long)sms * 4 * kWarps;
  const int cpt = (int)(cdiv(n, warps) < 32 ? cdiv(n, warps) : 32);
  const long long grid = cdiv(cdiv(n, cpt), kWarps);
  exchange_kernel<<<(unsigned)grid, kWarps * 32, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a, cpt);
  return cudaGetLastError() == cudaSuccess ? TGP_OK : TGP_ERR_CUDA;
}

tgp_status tgp_tournament_select(const double* fitness, int64_t stride, int64_t pop,
                                 const uint32_t* words, int64_t n, int32_t tournament_size,
                                 int32_t minimize, int32_t* winners, void* stream) {
  if (n < 0 || tournament_size < 1 || tournament_size > 4096) return TGP_ERR_INVALID_ARG;
  if (n == 0) return TGP_OK;
  if (!fitness || !words || !winners || pop < 1 || pop > 0x7fffffffLL || stride < 1)
    return TGP_ERR_INVALID_ARG;
  const int sms = sm_count();
  if (!sms) return TGP_ERR_CUDA;
  TournArgs a{fitness, stride, pop, words, n, tournament_size, minimize ? 1 : 0, winners};
  long long grid = cdiv(n, 256);
  if (grid > (long long)sms * 8) grid = (long long)sms * 8;  // 8 CTAs of 256 threads fill an SM
  tournament_kernel<<<(unsigned)grid, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(a);
  return cudaGetLastError() == cudaSuccess ? TGP_OK : TGP_ERR_CUDA;
}

tgp_status tgp_accuracy_from_outputs(const float* out, int64_t pop, int32_t n_classes,
                                     int64_t n_points, const int32_t* labels, int64_t* correct,
                                     double* accuracy, void* stream) {
  if (pop < 0 || n_classes < 1 || n_classes > TGP_MAX_OUTPUTS || n_points < 1)
    return TGP_ERR_INVALID_ARG;
  if (pop == 0) return TGP_OK;
  if (!out || !labels || !correct) return TGP_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(correct);
  if (cudaMemsetAsync(cnt, 0, (size_t)pop * 8, st) != cudaSuccess) return TGP_ERR_CUDA;
  tgp_status s = launch_count(out, pop, n_classes, n_points, n_points, labels, cnt, st);
  if (s != TGP_OK) return s;
  return launch_acc_final(cnt, pop, n_points, nullptr, accuracy, st);
}

size_t tgp_accuracy_workspace_size(const tgp_population* pop, const tgp_data* data,
                                   int32_t n_classes) {
  if (!pop || !data || data->n_points < 1 || n_classes < 1 || n_classes > TGP_MAX_OUTPUTS)
    return 0;
  AccWs w;
  return acc_ws(pop, data, n_classes, &w) ? w.total : 0;
}

tgp_status tgp_fitness_accuracy(const tgp_population* pop, const tgp_data* data,
                                const int32_t* labels, int32_t n_classes, double* accuracy,
                                int64_t* correct, int32_t* tree_status, void* ws, size_t ws_bytes,
                                void* stream) {
  if (!pop || !data || data->n_points < 1 || n_classes < 1 || n_classes > TGP_MAX_OUTPUTS)
    return TGP_ERR_INVALID_ARG;
  if (pop->pop > 0 && (!labels || !accuracy)) return TGP_ERR_INVALID_ARG;
  AccWs w;
  if (!acc_ws(pop, data, n_classes, &w)) return TGP_ERR_INVALID_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < w.total)
    return TGP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wsb = reinterpret_cast<char*>(ws);
  float* out = reinterpret_cast<float*>(wsb + w.out);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(wsb + w.cnt);
  int32_t* status = tree_status ? tree_status : reinterpret_cast<int32_t*>(wsb + w.st);
  if (pop->pop > 0 && cudaMemsetAsync(cnt, 0, (size_t)pop->pop * 8, st) != cudaSuccess)
    return TGP_ERR_CUDA;
  for (long long d0 = 0; d0 < data->n_points; d0 += w.chunk) {
    const long long dc = data->n_points - d0 < w.chunk ? data->n_points - d0 : w.chunk;
    tgp_data part{data->X + d0 * data->ldx, dc, data->n_features, data->ldx};
    tgp_status s = tgp_eval_forward(pop, &part, n_classes, out, status, wsb + w.fwd, w.out,
                                    stream);
    if (s != TGP_OK) return s;
    s = launch_count(out, pop->pop, n_classes, dc, dc, labels + d0, cnt, st);
    if (s != TGP_OK) return s;
  }
  if (correct && pop->pop > 0 &&
      cudaMemcpyAsync(correct, cnt, (size_t)pop->pop * 8, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess)
    return TGP_ERR_CUDA;
  return launch_acc_final(cnt, pop->pop, data->n_points, status, accuracy, st);
}

}  // extern "C"
