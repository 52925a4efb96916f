// api.cu -- host side of the C ABI declared in include/tgp.h: argument
// checks, launch-shape heuristic, workspace layout and kernel launches.  No
// allocation, no synchronization; everything goes onto the caller's stream.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "../../include/tgp.h"
#include "tgp_internal.cuh"

namespace tgp {
size_t stage_smem_bytes(int lmax);
int stage_threads();
const void* stage_kernel_ptr();
const void* find_eval_kernel(int K, int nw, bool modi, bool out);
size_t eval_smem_bytes(int K, int nw, bool modi, bool mse, int bt, int pcap, int tp, int F, int O);
const void* finalize_kernel_ptr();
const void* find_adj_kernel(int K, int nw, bool modi, int max_len, int* cap_out);
size_t adj_smem_bytes(int K, int nw, bool modi, int pcap, int max_len, int tp, int F, int O);
const void* adj_finalize_ptr();

namespace {

constexpr int kMaxDevices = 64;
// Warps per CTA of the evaluation kernels.  A wide CTA (one per SM) shares
// its X tile and program area among all its warps, so more warps fit in
// shared memory: 32 for the plain kernel at 8 points per lane (C2 5.95 ->
// 5.65 ms against 3 CTAs of 8 warps; 62 registers), 28 for the Modi kernel
// beside the warps' output accumulators (C5 at 250k points 184 -> 130 ms;
// 72 registers allow 28).  Narrower CTAs (16, then 8 warps) take over
// where shared memory would cramp the wide one.
constexpr int kNW = 8;            // the narrow CTA (3 per SM)
constexpr int kPlainNW = 32;      // plain kernel at 8 points per lane
constexpr int kModiNW = 28;       // Modi kernel (4 points per lane)
constexpr long long kWideMinPoints = 16384;  // the plain kernel's wide CTA from this many points
constexpr int kCtasPerSm = 3;     // resident evaluation CTAs the shape heuristic aims for
constexpr int kMaxCtasPerSm = 8;  // 2048 threads per SM / 256 per CTA
constexpr int kMaxGroups = TGP_MAX_PROBLEMS;  // evaluation launches per kernel variant in a batch
static_assert(CTRL_COUNTER_GROUP + 2 * kMaxGroups <= CTRL_WORDS, "control block too small");

struct DevInfo {
  bool init = false;
  int sms = 0;
  int smem_optin = 0;
  char name[256] = {0};  // device name with spaces as '_' (autotune cache key)
};
std::mutex g_mu;
DevInfo g_dev[kMaxDevices];

struct AttrEntry {
  const void* fn;
  int dev;
  int bytes;
};
AttrEntry g_attr[256];
int g_nattr = 0;

bool dev_info(DevInfo* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  DevInfo& d = g_dev[dev];
  if (!d.init) {
    if (cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      return false;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return false;
    size_t i = 0;
    for (; i + 1 < sizeof(d.name) && prop.name[i]; ++i) d.name[i] = prop.name[i] == ' ' ? '_' : prop.name[i];
    d.name[i] = 0;
    d.init = true;
  }
  *out = d;
  return true;
}

// Raises the dynamic shared memory limit of fn on the current device once.
bool ensure_smem(const void* fn, size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lk(g_mu);
  for (int i = 0; i < g_nattr; ++i)
    if (g_attr[i].fn == fn && g_attr[i].dev == dev && g_attr[i].bytes >= (int)bytes) return true;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess)
    return false;
  for (int i = 0; i < g_nattr; ++i)
    if (g_attr[i].fn == fn && g_attr[i].dev == dev) {
      g_attr[i].bytes = (int)bytes;
      return true;
    }
  if (g_nattr < 256) g_attr[g_nattr++] = {fn, dev, (int)bytes};
  return true;
}

inline long long cdiv(long long a, long long b) { return (a + b - 1) / b; }
inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

int pcap_of(int max_len) { return (max_len + 2 + 1) & ~1; }

// Launch shape for K points per lane: the caller's config where given, else
// the heuristic.
bool shape_for_k(int K, int nw, long long P, long long D, int F, int O, int max_len,
                 const tgp_config* cfg, bool modi, bool mse, const DevInfo& dv, Shape* sh) {
  Shape s{};
  s.nw = nw;
  s.K = K;
  if (s.K != 4 && s.K != 8) return false;
  const int CH = 32 * s.K;
  const int pcap = pcap_of(max_len);
  s.bt = (cfg && cfg->trees_per_block) ? cfg->trees_per_block : (s.nw > kNW ? (modi ? 48 : 64) : 32);
  if (s.bt < 1 || s.bt > 64) return false;
  const long long Dr = D < 1 ? 1 : D;
  if (cfg && cfg->points_per_tile) {
    s.tp = cfg->points_per_tile;
    if (s.tp % CH != 0 || s.tp < CH || s.tp > 4096) return false;
  } else {
    s.tp = 4 * CH;
    while (s.tp > CH && (long long)(s.tp / 2) >= Dr) s.tp /= 2;
  }
  // enough items to balance a persistent grid (a wide CTA is one per SM)
  const long long target = (s.nw > kNW ? 2LL : 4LL) * dv.sms;
  if (!(cfg && cfg->trees_per_block)) {
    // small problems: fewer trees per block so that every SM gets work, but
    // a wide CTA keeps at least half as many (tree, chunk) sub-items per
    // tile as it has warps (one tree's chunks would leave most of it idle)
    const long long min_sub = s.nw > kNW ? s.nw / 2 : 1;
    const long long chunks = cdiv(Dr < s.tp ? Dr : s.tp, CH);
    while (s.bt > 1 && cdiv(P, s.bt) * cdiv(Dr, s.tp) < target && (s.bt / 2) * chunks >= min_sub)
      s.bt /= 2;
  }
  // fit shared memory: kCtasPerSm CTAs per SM when the heuristic picks the
  // shape, the per-CTA maximum when the caller does
  const int bt0 = s.bt, tp0 = s.tp;
  const size_t limit = (size_t)dv.smem_optin;
  auto bytes = [&]() { return eval_smem_bytes(s.K, s.nw, modi, mse, s.bt, pcap, s.tp, F, O); };
  {
    // three CTAs per SM when that keeps tiles of >= 2 chunks and blocks of
    // >= 8 trees, else two (wide X tiles, long programs); one wide CTA
    const Shape s0 = s;
    bool fit = false;
    const int c_hi = s.nw > kNW ? 1 : kCtasPerSm, c_lo = s.nw > kNW ? 1 : 2;
    for (int ctas = c_hi; ctas >= c_lo && !fit; --ctas) {
      s = s0;
      const size_t per_cta = limit / ctas - 1024;
      const int tp_min = ctas > 2 ? 2 * CH : CH, bt_min = ctas > 2 ? 8 : 4;
      if (s.nw > kNW) {
        // a wide CTA keeps its tiles and gives up trees first (Modi C5 at
        // 250k points: 48 trees x 256 points 144 ms, 40 x 512 133 ms)
        while (bytes() > per_cta && s.bt > 16 && !(cfg && cfg->trees_per_block)) --s.bt;
      }
      while (bytes() > per_cta && s.tp > tp_min && !(cfg && cfg->points_per_tile)) s.tp /= 2;
      while (bytes() > per_cta && s.bt > bt_min && !(cfg && cfg->trees_per_block)) --s.bt;
      fit = bytes() <= per_cta;
    }
  }
  while (bytes() > limit && s.tp > CH && !(cfg && cfg->points_per_tile)) s.tp /= 2;
  while (bytes() > limit && s.bt > 1 && !(cfg && cfg->trees_per_block)) s.bt /= 2;
  if (bytes() > limit) return false;
  s.n_tiles = (int)cdiv(Dr, s.tp);
  s.n_blocks = (int)cdiv(P < 1 ? 1 : P, s.bt);
  if (cfg && cfg->tiles_per_item) {
    s.g = cfg->tiles_per_item;
    if (s.g < 1) return false;
  } else {
    s.g = (int)cdiv(s.n_tiles, 64);  // at most 64 partial sums per tree and output
    while (s.g > 1 && (long long)s.n_blocks * cdiv(s.n_tiles, s.g) < target) s.g /= 2;
    if (s.g < 1) s.g = 1;
    if (cdiv(s.n_tiles, s.g) > 64) s.g = (int)cdiv(s.n_tiles, 64);
  }
  s.n_groups = (int)cdiv(s.n_tiles, s.g);
  s.n_items = (long long)s.n_blocks * s.n_groups;
  s.cramped = s.bt < (bt0 < 16 ? bt0 : 16) || s.tp < (tp0 < 2 * CH ? tp0 : 2 * CH);
  *sh = s;
  return true;
}

// Warps per CTA: the wide CTA for K (one per SM), then narrower ones down to
// kNW, for as long as shared memory cramps the wider one (many Modi outputs,
// wide feature sets).
bool shape_nw(int K, long long P, long long D, int F, int O, int max_len, const tgp_config* cfg,
              bool modi, bool mse, const DevInfo& dv, Shape* sh) {
  static const int kModiCand[] = {kModiNW, 16, kNW}, kPlainCand[] = {kPlainNW, kNW};
  const int* cand = modi ? kModiCand : kPlainCand;
  const int n = modi ? 3 : 2;
  const int width = cfg ? cfg->cta_width : 0;  // 0 choose, 1 narrow, 2 wide
  // The single-output kernel takes the wide CTA for large data sets only: on
  // a few thousand points the narrow CTAs, several per SM, overlap one
  // another's program staging and tile barriers (10,000 trees x 1,024
  // points: 0.55 vs 0.62 ms; x 4,096: 1.92 vs 2.05 ms; 100,000 x 20,640:
  // 91.0 vs 88.9 ms; C2 at 100,000 points: 5.94 vs 5.64 ms).
  const bool wide_ok = modi || width == 2 || D >= kWideMinPoints;
  if (width != 1 && wide_ok) {
    for (int i = 0; i < n; ++i) {
      const int nw = (!modi && K != 8) ? kNW : cand[i];
      if (nw == kNW) continue;
      if (!shape_for_k(K, nw, P, D, F, O, max_len, cfg, modi, mse, dv, sh)) continue;
      // a caller who asks for the wide CTA takes the widest that fits
      if (!sh->cramped || width == 2) return true;
    }
  }
  return shape_for_k(K, kNW, P, D, F, O, max_len, cfg, modi, mse, dv, sh);
}

// Launch shape: 8 points per lane for single-output populations unless the
// caller says otherwise or the X tile of a wide feature set does not fit,
// then 4; Modi populations always 4 (their accumulators live in shared
// memory, and the Modi interpreter at 8 points per lane no longer fits the
// instruction cache: 2.6x slower, measured).  A single problem of at most
// 128 points also takes 4: a warp's 256 slots at 8 per lane would leave most
// lanes idle (60 points: 14% faster with 4 per lane, measured).  Problems
// of a batch get the shapes they would get alone (a batch launches one
// kernel per points-per-lane value and CTA width).
bool choose_shape(long long P, long long D, int F, int O, int max_len, const tgp_config* cfg,
                  bool modi, bool mse, const DevInfo& dv, Shape* sh) {
  if (modi) return shape_nw(4, P, D, F, O, max_len, cfg, modi, mse, dv, sh);
  if (cfg && cfg->points_per_lane)
    return shape_nw(cfg->points_per_lane, P, D, F, O, max_len, cfg, modi, mse, dv, sh);
  if (D <= 32 * 4 && shape_nw(4, P, D, F, O, max_len, cfg, modi, mse, dv, sh))
    return true;
  return shape_nw(8, P, D, F, O, max_len, cfg, modi, mse, dv, sh) ||
         shape_nw(4, P, D, F, O, max_len, cfg, modi, mse, dv, sh);
}

WsLayout ws_layout(long long P, int max_len, int O, int n_groups) {
  WsLayout w{};
  w.pcap = pcap_of(max_len);
  w.n_groups = n_groups;
  size_t off = 0;
  w.ctrl = off; off = al256(off + CTRL_WORDS * 4);
  w.prog = off; off = al256(off + (size_t)P * w.pcap * 8);
  w.plen = off; off = al256(off + (size_t)P * 4);
  w.status = off; off = al256(off + (size_t)P * 4);
  w.partial = off; off = al256(off + (size_t)P * O * n_groups * 8);
  w.gval64 = off; off = al256(off + (size_t)P * max_len * 8);
  w.mse64 = off; off = al256(off + (size_t)P * O * 8);
  w.total = off;
  return w;
}

bool pop_ok(const tgp_population* p) {
  if (!p || p->pop < 0 || p->max_len < 1 || p->max_len > TGP_MAX_LEN || p->ld < p->max_len) return false;
  if (p->pop > 0 && (!p->type || !p->value || !p->size)) return false;
  return true;
}
bool data_ok(const tgp_data* d) {
  if (!d || d->n_points < 0 || d->n_features < 1 || d->n_features > TGP_MAX_FEATURES ||
      d->ldx < d->n_features)
    return false;
  if (d->n_points > 0 && !d->X) return false;
  return true;
}

// Shapes of both kernel variants share n_groups so one partial buffer serves.
bool shapes_for(const tgp_population* pop, const tgp_data* data, int O, const tgp_config* cfg,
                bool mse, const DevInfo& dv, Shape* plain, Shape* modi) {
  long long D = data ? data->n_points : 0;
  int F = data ? data->n_features : 1;
  if (!choose_shape(pop->pop, D, F, O, pop->max_len, cfg, true, mse, dv, modi)) return false;
  if (O == 1) {
    if (!choose_shape(pop->pop, D, F, O, pop->max_len, cfg, false, mse, dv, plain))
      return false;
  } else {
    *plain = *modi;
  }
  return true;
}

// One problem of a launch after planning.
struct Planned {
  const tgp_population* pop;
  const tgp_data* data;
  const float* y;
  int O;
  float* out;
  double* mse_out;
  int32_t* status_out;
  Shape sp, sm;     // plain / Modi kernel shapes, n_groups equalised
  WsLayout w;       // offsets relative to base
  size_t base;      // offset of this problem's workspace region
  int flags = 0;    // TGP_FLAG_* of the problem
};

tgp_status plan(Planned& q, const tgp_config* cfg, bool mse, const DevInfo& dv) {
  if (!shapes_for(q.pop, q.data, q.O, cfg, mse, dv, &q.sp, &q.sm)) return TGP_ERR_UNSUPPORTED;
  const int n_groups = q.sm.n_groups > q.sp.n_groups ? q.sm.n_groups : q.sp.n_groups;
  q.w = ws_layout(q.pop->pop, q.pop->max_len, q.O, mse ? n_groups : 0);
  for (Shape* sh : {&q.sp, &q.sm}) {
    sh->n_groups = n_groups;
    sh->g = (int)cdiv(sh->n_tiles, n_groups);
    sh->n_items = (long long)sh->n_blocks * n_groups;
  }
  return TGP_OK;
}

tgp_status launch_stage(Planned* qs, int n, char* ws, cudaStream_t st, const DevInfo& dv,
                        bool want_nodes = false) {
  StageBatch b{};
  long long total = 0;
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const Planned& q = qs[i];
    if (q.pop->pop == 0) continue;
    char* w = ws + q.base;
    StageArgs& a = b.p[m];
    a.type = q.pop->type;
    a.val = q.pop->value;
    a.size = q.pop->size;
    a.pop = q.pop->pop;
    a.ld = q.pop->ld;
    a.max_len = q.pop->max_len;
    a.n_features = q.data->n_features;
    a.n_outputs = q.O;
    a.prog = reinterpret_cast<uint2*>(w + q.w.prog);
    a.pcap = q.w.pcap;
    a.plen = reinterpret_cast<int*>(w + q.w.plen);
    a.status = reinterpret_cast<int*>(w + q.w.status);
    a.user_status = q.status_out;
    a.ctrl = reinterpret_cast<unsigned*>(w + q.w.ctrl);
    a.want_nodes = want_nodes ? 1 : 0;
    total += q.pop->pop;
    b.end[m] = total;
    ++m;
  }
  if (m == 0) return TGP_OK;
  b.n = m;
  int lmax = 16;
  for (int i = 0; i < m; ++i) lmax = b.p[i].max_len > lmax ? b.p[i].max_len : lmax;
  b.lmax = (lmax + 15) & ~15;
  const void* fn = stage_kernel_ptr();
  size_t smem = stage_smem_bytes(b.lmax);
  if (!ensure_smem(fn, smem)) return TGP_ERR_CUDA;
  const int warps_per_cta = stage_threads() / 32;
  long long grid = cdiv(total, warps_per_cta);
  if (grid > (long long)dv.sms * 16) grid = (long long)dv.sms * 16;
  void* args[] = {&b};
  if (cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(stage_threads()), args, smem, st) != cudaSuccess)
    return TGP_ERR_CUDA;
  return TGP_OK;
}

// Launches the evaluation kernels over every problem's work items (the plain
// variant only when some problem has a single output; each variant skips the
// items of problems whose Modi flag does not match it).  Problems are grouped
// by the number of CTAs of their shared-memory footprint that fit on an SM
// and by the carve-out that occupancy needs, and each group gets one
// persistent launch sized for it, so a problem with wide tiles lowers neither
// the occupancy nor the L1 share of the others.
// Index of the smallest shared-memory carve-out step (KB) of an SM that
// holds `bytes`.
int carveout_step(size_t bytes) {
  static const int kSteps[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};
  for (int i = 0; i < 10; ++i)
    if (bytes <= (size_t)kSteps[i] * 1024) return i;
  return 10;
}

tgp_status launch_eval(Planned* qs, int n, char* ws, unsigned* counters, cudaStream_t st,
                       const DevInfo& dv, bool mse, int max_polls = 0) {
  bool any_single = false;
  for (int i = 0; i < n; ++i) any_single |= qs[i].O == 1;
  const size_t limit = (size_t)dv.smem_optin;
  for (int variant = 0; variant < 2; ++variant) {
    const bool modi = variant == 1;
    if (!modi && !any_single) continue;
    int occ[TGP_MAX_PROBLEMS];
    size_t sbytes[TGP_MAX_PROBLEMS];
    const void* fns[TGP_MAX_PROBLEMS];  // each problem's kernel (points per lane, CTA width)
    int nws[TGP_MAX_PROBLEMS];
    for (int i = 0; i < n; ++i) {
      occ[i] = 0;
      fns[i] = nullptr;
      const Planned& q = qs[i];
      if (q.pop->pop == 0 || q.data->n_points == 0) continue;
      if (!modi && q.O > 1) continue;
      const Shape& sh = modi ? q.sm : q.sp;
      sbytes[i] = eval_smem_bytes(sh.K, sh.nw, modi, mse, sh.bt, q.w.pcap, sh.tp, q.data->n_features, q.O);
      if (sbytes[i] > limit) return TGP_ERR_UNSUPPORTED;
      const void* fn = find_eval_kernel(sh.K, sh.nw, modi, !mse);
      if (!fn) return TGP_ERR_UNSUPPORTED;
      if (!ensure_smem(fn, sbytes[i])) return TGP_ERR_CUDA;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[i], fn, sh.nw * 32, sbytes[i]) != cudaSuccess)
        return TGP_ERR_CUDA;
      if (occ[i] < 1) return TGP_ERR_UNSUPPORTED;
      if (occ[i] > kMaxCtasPerSm) occ[i] = kMaxCtasPerSm;
      // group key: occupancy, then the L1/shared-memory split the SM needs
      // for it (a larger shared-memory carve-out leaves less L1 for the
      // others, so problems are not mixed across carve-out steps)
      occ[i] = occ[i] * 16 + carveout_step((size_t)occ[i] * (sbytes[i] + 1024));
      fns[i] = fn;
      nws[i] = sh.nw;
    }
    // one launch per (kernel, group key): problems of different points per
    // lane or CTA width run as separate persistent launches, each problem in
    // the shape it would get alone
    int ngroup = 0;
    for (int key = kMaxCtasPerSm * 16 + 15; key >= 16; --key) {
     for (int lead = 0; lead < n; ++lead) {
      if (!fns[lead] || occ[lead] != key) continue;
      bool seen = false;  // this kernel's group of this key launched already
      for (int j = 0; j < lead; ++j) seen |= fns[j] == fns[lead] && occ[j] == key;
      if (seen) continue;
      const void* fn = fns[lead];
      const int nw = nws[lead];
      EvalBatch b{};
      const int per_sm = key / 16;
      long long total = 0;
      size_t smem = 0;
      int m = 0;
      for (int i = 0; i < n; ++i) {
        if (occ[i] != key || fns[i] != fn) continue;
        const Planned& q = qs[i];
        const Shape& sh = modi ? q.sm : q.sp;
        char* w = ws + q.base;
        EvalArgs& a = b.p[m];
        a.prog = reinterpret_cast<const uint2*>(w + q.w.prog);
        a.plen = reinterpret_cast<const int*>(w + q.w.plen);
        a.status = reinterpret_cast<const int*>(w + q.w.status);
        a.pcap = q.w.pcap;
        a.pop = q.pop->pop;
        a.X = q.data->X;
        a.D = q.data->n_points;
        a.F = q.data->n_features;
        a.ldx = q.data->ldx;
        a.x_vec4 = (reinterpret_cast<uintptr_t>(q.data->X) & 15) == 0 && q.data->n_features % 4 == 0 &&
                   q.data->ldx % 4 == 0;
        a.y = q.y;
        a.O = q.O;
        a.out = q.out;
        a.partial = reinterpret_cast<double*>(w + q.w.partial);
        a.bt = sh.bt;
        a.tp = sh.tp;
        a.g = sh.g;
        a.n_tiles = sh.n_tiles;
        a.n_groups = sh.n_groups;
        a.n_blocks = sh.n_blocks;
        a.n_items = sh.n_items;
        a.ctrl = reinterpret_cast<unsigned*>(w + q.w.ctrl);
        total += sh.n_items;
        b.end[m] = total;
        if (sbytes[i] > smem) smem = sbytes[i];
        ++m;
      }
      if (m == 0) continue;
      if (ngroup >= kMaxGroups) return TGP_ERR_UNSUPPORTED;
      b.counter = counters + CTRL_COUNTER_GROUP + 2 * ngroup++ + (modi ? 1 : 0);
      b.err = counters + CTRL_ERROR;
      b.max_polls = max_polls == 0 ? kDefaultWaitPolls : (max_polls < 0 ? 0 : max_polls);
      b.n = m;
      long long grid = (long long)dv.sms * per_sm;
      if (grid > total) grid = total;
      void* args[] = {&b};
      if (cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(nw * 32), args, smem, st) != cudaSuccess)
        return TGP_ERR_CUDA;
     }
    }
  }
  return TGP_OK;
}

tgp_status launch_final(Planned* qs, int n, char* ws, cudaStream_t st) {
  FinalBatch b{};
  long long total = 0;
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const Planned& q = qs[i];
    if (q.pop->pop == 0) continue;
    char* w = ws + q.base;
    FinalArgs& f = b.p[m];
    f.partial = reinterpret_cast<const double*>(w + q.w.partial);
    f.status = reinterpret_cast<const int*>(w + q.w.status);
    f.mse = q.mse_out;
    f.pop = q.pop->pop;
    f.O = q.O;
    f.n_groups = q.sp.n_groups;
    f.D = q.data->n_points;
    f.sse = (q.flags & TGP_FLAG_SSE) ? 1 : 0;
    total += q.pop->pop * q.O;
    b.end[m] = total;
    ++m;
  }
  if (m == 0) return TGP_OK;
  b.n = m;
  void* args[] = {&b};
  if (cudaLaunchKernel(finalize_kernel_ptr(), dim3((unsigned)cdiv(total, 256)), dim3(256), args, 0, st) !=
      cudaSuccess)
    return TGP_ERR_CUDA;
  return TGP_OK;
}

bool problem_ok(const tgp_population* pop, const tgp_data* data, int O) {
  return pop_ok(pop) && data_ok(data) && O >= 1 && O <= TGP_MAX_OUTPUTS;
}

tgp_status run(const tgp_population* pop, const tgp_data* data, const float* y, int O, float* out,
               double* mse_out, bool mse, int32_t* tree_status, void* ws, size_t ws_bytes,
               void* stream, const tgp_config* cfg) {
  if (!problem_ok(pop, data, O)) return TGP_ERR_INVALID_ARG;
  if (mse && (data->n_points < 1 || (pop->pop > 0 && (!y || !mse_out)))) return TGP_ERR_INVALID_ARG;
  if (!mse && pop->pop > 0 && data->n_points > 0 && !out) return TGP_ERR_INVALID_ARG;
  DevInfo dv;
  if (!dev_info(&dv)) return TGP_ERR_CUDA;
  if (cfg && ((cfg->flags & ~TGP_FLAG_SSE) != 0 || cfg->cta_width < 0 || cfg->cta_width > 2))
    return TGP_ERR_INVALID_ARG;
  Planned q{pop, data, y, O, out, mse_out, tree_status};
  q.base = 0;
  q.flags = cfg ? cfg->flags : 0;
  tgp_status s = plan(q, cfg, mse, dv);
  if (s != TGP_OK) return s;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < q.w.total) return TGP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wsb = reinterpret_cast<char*>(ws);
  if (cudaMemsetAsync(wsb + q.w.ctrl, 0, CTRL_WORDS * 4, st) != cudaSuccess) return TGP_ERR_CUDA;
  s = launch_stage(&q, 1, wsb, st, dv);
  if (s != TGP_OK) return s;
  if (pop->pop == 0 || data->n_points == 0) return TGP_OK;
  if (cfg && cfg->eval_begin_event &&
      cudaEventRecord(reinterpret_cast<cudaEvent_t>(cfg->eval_begin_event), st) != cudaSuccess)
    return TGP_ERR_CUDA;
  s = launch_eval(&q, 1, wsb, reinterpret_cast<unsigned*>(wsb + q.w.ctrl), st, dv, mse,
                  cfg ? cfg->max_wait_polls : 0);
  if (s != TGP_OK) return s;
  if (cfg && cfg->eval_end_event &&
      cudaEventRecord(reinterpret_cast<cudaEvent_t>(cfg->eval_end_event), st) != cudaSuccess)
    return TGP_ERR_CUDA;
  if (mse) return launch_final(&q, 1, wsb, st);
  return TGP_OK;
}

// Several independent problems in one stage, one persistent evaluation and one
// finalize launch.  Workspace: a 256-byte control block (the shared work
// counters) followed by one region per problem.
bool shape_given(const tgp_config& c) {
  return c.trees_per_block || c.points_per_tile || c.tiles_per_item || c.points_per_lane || c.cta_width;
}

// tuned: NULL, or per problem a shape to use when the problem's own cfg gives
// none (all shape fields zero = no tuned shape either).
tgp_status plan_batch(const tgp_problem* probs, int n, const DevInfo& dv, Planned* qs, size_t* total,
                      const tgp_config* tuned = nullptr) {
  if (n < 1 || n > TGP_MAX_PROBLEMS || !probs) return TGP_ERR_INVALID_ARG;
  size_t off = al256(CTRL_WORDS * 4);
  for (int i = 0; i < n; ++i) {
    const tgp_problem& p = probs[i];
    if (!problem_ok(&p.pop, &p.data, p.n_outputs)) return TGP_ERR_INVALID_ARG;
    if (p.data.n_points < 1 || (p.pop.pop > 0 && (!p.y || !p.mse))) return TGP_ERR_INVALID_ARG;
    if ((p.cfg.flags & ~TGP_FLAG_SSE) != 0 || p.cfg.cta_width < 0 || p.cfg.cta_width > 2)
      return TGP_ERR_INVALID_ARG;
    Planned& q = qs[i];
    q = Planned{&p.pop, &p.data, p.y, p.n_outputs, nullptr, p.mse, p.tree_status};
    q.flags = p.cfg.flags;
    const tgp_config* cfg = shape_given(p.cfg) ? &p.cfg
                            : (tuned && shape_given(tuned[i])) ? &tuned[i]
                                                                : nullptr;
    tgp_status s = plan(q, cfg, true, dv);
    if (s != TGP_OK) return s;
    q.base = off;
    off = al256(off + q.w.total);
  }
  *total = off;
  return TGP_OK;
}

// Launches a planned batch (qs[0..n) with their workspace regions laid out
// behind the shared control block).
tgp_status launch_batch(Planned* qs, int n, size_t need, const DevInfo& dv, void* ws, size_t ws_bytes,
                        void* stream) {
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < need) return TGP_ERR_WORKSPACE;
  tgp_status s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wsb = reinterpret_cast<char*>(ws);
  if (cudaMemsetAsync(wsb, 0, CTRL_WORDS * 4, st) != cudaSuccess) return TGP_ERR_CUDA;
  for (int i = 0; i < n; ++i)
    if (cudaMemsetAsync(wsb + qs[i].base + qs[i].w.ctrl, 0, CTRL_WORDS * 4, st) != cudaSuccess)
      return TGP_ERR_CUDA;
  s = launch_stage(qs, n, wsb, st, dv);
  if (s != TGP_OK) return s;
  s = launch_eval(qs, n, wsb, reinterpret_cast<unsigned*>(wsb), st, dv, true);
  if (s != TGP_OK) return s;
  return launch_final(qs, n, wsb, st);
}

tgp_status run_batch(const tgp_problem* probs, int n, void* ws, size_t ws_bytes, void* stream) {
  DevInfo dv;
  if (!dev_info(&dv)) return TGP_ERR_CUDA;
  Planned qs[TGP_MAX_PROBLEMS];
  size_t need = 0;
  tgp_status s = plan_batch(probs, n, dv, qs, &need);
  if (s != TGP_OK) return s;
  return launch_batch(qs, n, need, dv, ws, ws_bytes, stream);
}

// ------------------------------------------------------------- autotune cache
// Shape bucket of a problem, as the autotuner writes it:
// <GPU name>|P<lg P>_D<lg D>_F<F>_O<O>_L<lg max_len>, lg = rounded log2.
int lg_round(long long x) { return (int)std::lround(std::log2((double)(x < 1 ? 1 : x))); }

void cache_key(const DevInfo& dv, const tgp_problem& p, char* out, size_t n) {
  std::snprintf(out, n, "%s|P%d_D%d_F%d_O%d_L%d", dv.name, lg_round(p.pop.pop), lg_round(p.data.n_points),
                (int)p.data.n_features, (int)p.n_outputs, lg_round(p.pop.max_len));
}

// Reads the entries of the cache file for the given keys (the last line of a
// key wins).  Unknown names on a line are ignored; a malformed value leaves
// the entry unused.
void cache_read(const char* path, char (*keys)[320], int n, tgp_config* out, int* found) {
  for (int i = 0; i < n; ++i) found[i] = 0;
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char line[2048];
  while (std::fgets(line, sizeof line, f)) {
    char* save = nullptr;
    char* tok = strtok_r(line, " \t\r\n", &save);
    if (!tok || tok[0] == '#') continue;
    int which = -1;
    for (int i = 0; i < n; ++i)
      if (std::strcmp(tok, keys[i]) == 0) which = i;
    if (which < 0) continue;
    tgp_config c{};
    bool ok = true;
    while ((tok = strtok_r(nullptr, " \t\r\n", &save)) != nullptr) {
      char* eq = std::strchr(tok, '=');
      if (!eq) continue;
      *eq = 0;
      char* end = nullptr;
      const long v = std::strtol(eq + 1, &end, 10);
      const bool num = end != eq + 1 && (*end == 0);
      int32_t* dst = std::strcmp(tok, "trees_per_block") == 0   ? &c.trees_per_block
                     : std::strcmp(tok, "points_per_tile") == 0 ? &c.points_per_tile
                     : std::strcmp(tok, "tiles_per_item") == 0  ? &c.tiles_per_item
                     : std::strcmp(tok, "points_per_lane") == 0 ? &c.points_per_lane
                     : std::strcmp(tok, "cta_width") == 0       ? &c.cta_width
                                                                : nullptr;
      if (!dst) continue;
      if (!num || v < 0 || v > 65536 || (dst == &c.cta_width && v > 2)) ok = false;
      else *dst = (int32_t)v;
    }
    // Every line for a key replaces the earlier one; a malformed line drops it.
    found[which] = ok && shape_given(c) ? 1 : 0;
    if (found[which]) out[which] = c;
  }
  std::fclose(f);
}

// Fused forward + reverse sweep: one CTA per point tile over all trees.
tgp_status run_backward(const tgp_population* pop, const tgp_data* data, const float* y, int O,
                        const double* grad_mse, double* mse_out, float* grad_value, float* grad_X,
                        int32_t* tree_status, void* ws, size_t ws_bytes, void* stream,
                        const tgp_config* cfg) {
  if (!pop_ok(pop) || !data_ok(data) || O < 1 || O > TGP_MAX_OUTPUTS) return TGP_ERR_INVALID_ARG;
  if (cfg && (cfg->points_per_tile < 0 || cfg->points_per_tile % 128 != 0 || cfg->points_per_tile > 4096))
    return TGP_ERR_INVALID_ARG;
  if (data->n_points < 1) return TGP_ERR_INVALID_ARG;
  if (pop->pop > 0 && (!y || !grad_mse)) return TGP_ERR_INVALID_ARG;
  DevInfo dv;
  if (!dev_info(&dv)) return TGP_ERR_CUDA;
  Shape sp, sm;
  if (!shapes_for(pop, data, O, nullptr, true, dv, &sp, &sm)) return TGP_ERR_UNSUPPORTED;
  const int n_groups = sm.n_groups > sp.n_groups ? sm.n_groups : sp.n_groups;
  WsLayout w = ws_layout(pop->pop, pop->max_len, O, n_groups);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < w.total) return TGP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wsb = reinterpret_cast<char*>(ws);
  if (cudaMemsetAsync(wsb + w.ctrl, 0, CTRL_WORDS * 4, st) != cudaSuccess) return TGP_ERR_CUDA;
  if (pop->pop == 0) return TGP_OK;
  if (cudaMemsetAsync(wsb + w.gval64, 0, w.mse64 + (size_t)pop->pop * O * 8 - w.gval64, st) != cudaSuccess)
    return TGP_ERR_CUDA;
  Planned q{pop, data, y, O, nullptr, mse_out, tree_status};
  q.w = w;
  q.base = 0;
  tgp_status s = launch_stage(&q, 1, wsb, st, dv, true);
  if (s != TGP_OK) return s;
  // the events bracket every adjoint launch of the call: begin before the
  // first variant, end after the last (a single-output call runs both)
  for (int variant = 0; variant < 2; ++variant) {
    const bool modi = variant == 1;
    if (!modi && O > 1) continue;
    const bool first = variant == 0 || O > 1, last = variant == 1;
    // 4 points per lane: at 8 the per-thread tape doubles and the kernel
    // runs 1.5x slower (156 vs 103 ms on the differentiation workload)
    const int K = 4;
    const bool fixed_tp = cfg && cfg->points_per_tile;
    // One CTA of 32 warps per SM (64 registers, no spills; 3 CTAs of 8
    // warps hold 24) over tiles of up to 1024 points where its shared memory
    // fits (C4: 93.0 -> 81.9 ms; 28 warps: 85.2 ms), else one of 16 warps
    // (Modi populations: the per-warp output rows), else 3 CTAs of 8 warps
    // over tiles of up to 512 points.  Tiles of several chunks
    // amortise the per-(tree, tile) work (128 points: 127 ms, 512: 107 ms
    // with one item per tile); smaller when the data has fewer points, or
    // when wide X tiles would leave fewer than 3 CTAs per SM.  The
    // population is then split into tree ranges so that the persistent grid
    // gets about 8 items per CTA.
    int nw = 0, tp = 0, per_sm = 0;
    size_t smem = 0;
    const void* fn = nullptr;
    for (const int cand : {32, 16, 8}) {
      int cap = 0;
      fn = find_adj_kernel(K, cand, modi, pop->max_len, &cap);
      if (!fn) return TGP_ERR_UNSUPPORTED;
      const bool wide = cand > 8;
      tp = fixed_tp ? cfg->points_per_tile : (wide ? 1024 : 512);
      if (!fixed_tp)
        while (tp > 32 * K && tp / 2 >= data->n_points) tp /= 2;
      const int tp_floor = 32 * K;
      bool ok = false;
      for (;;) {
        smem = adj_smem_bytes(K, cand, modi, w.pcap, pop->max_len, tp, data->n_features, O);
        if (smem > (size_t)dv.smem_optin) {
          if (fixed_tp || tp <= tp_floor) break;
          tp /= 2;
          continue;
        }
        if (!ensure_smem(fn, smem)) return TGP_ERR_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, cand * 32, smem) != cudaSuccess)
          return TGP_ERR_CUDA;
        if (per_sm < 1) break;
        ok = true;
        if (wide || fixed_tp || tp <= 32 * K || per_sm >= 3) break;
        tp /= 2;
      }
      if (ok) {
        nw = cand;
        break;
      }
    }
    if (!nw) return TGP_ERR_UNSUPPORTED;
    const long long n_tiles = cdiv(data->n_points, tp);
    const long long slots = (long long)dv.sms * per_sm;
    long long chunks = cdiv(8 * slots, n_tiles);
    const long long max_chunks = cdiv(pop->pop, 8 * nw);  // >= 8 trees per warp per item
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    const long long per_chunk = cdiv(pop->pop, chunks);
    chunks = cdiv(pop->pop, per_chunk);
    AdjArgs a;
    a.prog = reinterpret_cast<const uint2*>(wsb + w.prog);
    a.plen = reinterpret_cast<const int*>(wsb + w.plen);
    a.status = reinterpret_cast<const int*>(wsb + w.status);
    a.pcap = w.pcap;
    a.pop = pop->pop;
    a.max_len = pop->max_len;
    a.X = data->X;
    a.D = data->n_points;
    a.F = data->n_features;
    a.ldx = data->ldx;
    a.y = y;
    a.O = O;
    a.g = grad_mse;
    a.want_mse = mse_out != nullptr;
    a.gval64 = reinterpret_cast<double*>(wsb + w.gval64);
    a.mse64 = reinterpret_cast<double*>(wsb + w.mse64);
    a.grad_X = grad_X;
    a.tp = tp;
    a.n_tiles = (int)n_tiles;
    a.tree_chunks = (int)chunks;
    a.trees_per_chunk = per_chunk;
    a.two_over_D = 2.0 / (double)data->n_points;
    a.ctrl = reinterpret_cast<unsigned*>(wsb + w.ctrl);
    long long grid = slots;
    if (grid > n_tiles * chunks) grid = n_tiles * chunks;
    void* args[] = {&a};
    if (first && cfg && cfg->eval_begin_event &&
        cudaEventRecord(reinterpret_cast<cudaEvent_t>(cfg->eval_begin_event), st) != cudaSuccess)
      return TGP_ERR_CUDA;
    if (cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(nw * 32), args, smem, st) != cudaSuccess)
      return TGP_ERR_CUDA;
    if (last && cfg && cfg->eval_end_event &&
        cudaEventRecord(reinterpret_cast<cudaEvent_t>(cfg->eval_end_event), st) != cudaSuccess)
      return TGP_ERR_CUDA;
  }
  AdjFinalArgs f;
  f.gval64 = reinterpret_cast<const double*>(wsb + w.gval64);
  f.mse64 = reinterpret_cast<const double*>(wsb + w.mse64);
  f.status = reinterpret_cast<const int*>(wsb + w.status);
  f.grad_value = grad_value;
  f.mse = mse_out;
  f.pop = pop->pop;
  f.ld = pop->ld;
  f.max_len = pop->max_len;
  f.O = O;
  f.D = data->n_points;
  long long n = pop->pop * (pop->ld > O ? pop->ld : O);
  void* args[] = {&f};
  if (cudaLaunchKernel(adj_finalize_ptr(), dim3((unsigned)cdiv(n, 256)), dim3(256), args, 0, st) !=
      cudaSuccess)
    return TGP_ERR_CUDA;
  return TGP_OK;
}

}  // namespace
}  // namespace tgp

// A planned batch: copies of the problem descriptors, their launch shapes and
// workspace layout, and the device they were planned for.
struct tgp_batch_plan_s {
  int n = 0;
  int dev = -1;
  size_t ws_bytes = 0;
  tgp::DevInfo dv;
  tgp_problem probs[TGP_MAX_PROBLEMS];
  tgp::Planned qs[TGP_MAX_PROBLEMS];
  tgp_config shape[TGP_MAX_PROBLEMS];
  int from_cache[TGP_MAX_PROBLEMS];
};

using namespace tgp;

extern "C" {

size_t tgp_workspace_size(const tgp_population* pop, const tgp_data* data, int32_t n_outputs,
                          const tgp_config* cfg) {
  if (!pop_ok(pop) || n_outputs < 1 || n_outputs > TGP_MAX_OUTPUTS) return 0;
  if (data && !data_ok(data)) return 0;
  DevInfo dv;
  if (!dev_info(&dv)) return 0;
  int n_groups = 0;
  if (data && data->n_points > 0) {
    Shape sp, sm;
    if (!shapes_for(pop, data, n_outputs, cfg, true, dv, &sp, &sm)) return 0;
    n_groups = sm.n_groups > sp.n_groups ? sm.n_groups : sp.n_groups;
  }
  return ws_layout(pop->pop, pop->max_len, n_outputs, n_groups).total;
}

tgp_status tgp_validate(const tgp_population* pop, int32_t n_features, int32_t n_outputs,
                        int32_t* tree_status, void* ws, size_t ws_bytes, void* stream) {
  if (!pop_ok(pop) || n_features < 1 || n_features > TGP_MAX_FEATURES || n_outputs < 1 ||
      n_outputs > TGP_MAX_OUTPUTS)
    return TGP_ERR_INVALID_ARG;
  if (pop->pop > 0 && !tree_status) return TGP_ERR_INVALID_ARG;
  DevInfo dv;
  if (!dev_info(&dv)) return TGP_ERR_CUDA;
  WsLayout w = ws_layout(pop->pop, pop->max_len, n_outputs, 0);
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255) != 0 || ws_bytes < w.total) return TGP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* wsb = reinterpret_cast<char*>(ws);
  if (cudaMemsetAsync(wsb + w.ctrl, 0, CTRL_WORDS * 4, st) != cudaSuccess) return TGP_ERR_CUDA;
  tgp_data dummy{nullptr, 0, n_features, n_features};
  Planned q{pop, &dummy, nullptr, n_outputs, nullptr, nullptr, tree_status};
  q.w = w;
  q.base = 0;
  return launch_stage(&q, 1, wsb, st, dv);
}

tgp_status tgp_eval_forward_cfg(const tgp_population* pop, const tgp_data* data, int32_t n_outputs,
                                float* out, int32_t* tree_status, void* ws, size_t ws_bytes,
                                void* stream, const tgp_config* cfg) {
  return run(pop, data, nullptr, n_outputs, out, nullptr, false, tree_status, ws, ws_bytes, stream,
             cfg);
}

tgp_status tgp_eval_forward(const tgp_population* pop, const tgp_data* data, int32_t n_outputs,
                            float* out, int32_t* tree_status, void* ws, size_t ws_bytes,
                            void* stream) {
  return run(pop, data, nullptr, n_outputs, out, nullptr, false, tree_status, ws, ws_bytes, stream,
             nullptr);
}

tgp_status tgp_fitness_mse_cfg(const tgp_population* pop, const tgp_data* data, const float* y,
                               int32_t n_outputs, double* mse, int32_t* tree_status, void* ws,
                               size_t ws_bytes, void* stream, const tgp_config* cfg) {
  return run(pop, data, y, n_outputs, nullptr, mse, true, tree_status, ws, ws_bytes, stream, cfg);
}

tgp_status tgp_fitness_mse(const tgp_population* pop, const tgp_data* data, const float* y,
                           int32_t n_outputs, double* mse, int32_t* tree_status, void* ws,
                           size_t ws_bytes, void* stream) {
  return tgp_fitness_mse_cfg(pop, data, y, n_outputs, mse, tree_status, ws, ws_bytes, stream, nullptr);
}

tgp_status tgp_eval_backward(const tgp_population* pop, const tgp_data* data, const float* y,
                             int32_t n_outputs, const double* grad_mse, double* mse_out,
                             float* grad_value, float* grad_X, int32_t* tree_status, void* ws,
                             size_t ws_bytes, void* stream) {
  return run_backward(pop, data, y, n_outputs, grad_mse, mse_out, grad_value, grad_X, tree_status, ws,
                      ws_bytes, stream, nullptr);
}

tgp_status tgp_eval_backward_cfg(const tgp_population* pop, const tgp_data* data, const float* y,
                                 int32_t n_outputs, const double* grad_mse, double* mse_out,
                                 float* grad_value, float* grad_X, int32_t* tree_status, void* ws,
                                 size_t ws_bytes, void* stream, const tgp_config* cfg) {
  return run_backward(pop, data, y, n_outputs, grad_mse, mse_out, grad_value, grad_X, tree_status, ws,
                      ws_bytes, stream, cfg);
}

size_t tgp_batch_workspace_size(const tgp_problem* probs, int32_t n) {
  DevInfo dv;
  if (!dev_info(&dv)) return 0;
  Planned qs[TGP_MAX_PROBLEMS];
  size_t need = 0;
  if (plan_batch(probs, n, dv, qs, &need) != TGP_OK) return 0;
  return need;
}

tgp_status tgp_batch_fitness_mse(const tgp_problem* probs, int32_t n, void* ws, size_t ws_bytes,
                                 void* stream) {
  return run_batch(probs, n, ws, ws_bytes, stream);
}

tgp_status tgp_batch_plan(const tgp_problem* probs, int32_t n, const char* tune_cache,
                          tgp_batch_plan_t** plan) {
  if (!plan) return TGP_ERR_INVALID_ARG;
  *plan = nullptr;
  if (!probs || n < 1 || n > TGP_MAX_PROBLEMS) return TGP_ERR_INVALID_ARG;
  DevInfo dv;
  if (!dev_info(&dv)) return TGP_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TGP_ERR_CUDA;
  tgp_batch_plan_s* pl = static_cast<tgp_batch_plan_s*>(std::calloc(1, sizeof(tgp_batch_plan_s)));
  if (!pl) return TGP_ERR_INVALID_ARG;
  new (pl) tgp_batch_plan_s();
  pl->n = n;
  pl->dev = dev;
  pl->dv = dv;
  for (int i = 0; i < n; ++i) pl->probs[i] = probs[i];
  char keys[TGP_MAX_PROBLEMS][320];
  tgp_config tuned[TGP_MAX_PROBLEMS] = {};
  int found[TGP_MAX_PROBLEMS] = {};
  for (int i = 0; i < n; ++i) {
    cache_key(dv, pl->probs[i], keys[i], sizeof keys[i]);
    pl->probs[i].cfg.eval_begin_event = pl->probs[i].cfg.eval_end_event = nullptr;
  }
  cache_read(tune_cache, keys, n, tuned, found);
  tgp_status s = plan_batch(pl->probs, n, dv, pl->qs, &pl->ws_bytes, tuned);
  if (s != TGP_OK) {
    std::free(pl);
    return s;
  }
  for (int i = 0; i < n; ++i) {
    const bool own = shape_given(pl->probs[i].cfg);
    pl->from_cache[i] = !own && found[i];
    // the shape of the variant that serves the problem
    const Shape& sh = pl->qs[i].O > 1 ? pl->qs[i].sm : pl->qs[i].sp;
    tgp_config c{};
    c.trees_per_block = sh.bt;
    c.points_per_tile = sh.tp;
    c.tiles_per_item = sh.g;
    c.points_per_lane = sh.K;
    c.cta_width = sh.nw > kNW ? 2 : 1;
    c.flags = pl->probs[i].cfg.flags;
    pl->shape[i] = c;
  }
  *plan = pl;
  return TGP_OK;
}

size_t tgp_batch_plan_workspace_size(const tgp_batch_plan_t* plan) { return plan ? plan->ws_bytes : 0; }

tgp_status tgp_tune_cache_lookup(const char* tune_cache, const char* key, tgp_config* shape) {
  if (!tune_cache || !key || !shape || std::strlen(key) >= 320) return TGP_ERR_INVALID_ARG;
  char keys[1][320];
  std::strcpy(keys[0], key);
  tgp_config c{};
  int found = 0;
  cache_read(tune_cache, keys, 1, &c, &found);
  if (!found) return TGP_ERR_INVALID_ARG;
  *shape = c;
  return TGP_OK;
}

tgp_status tgp_batch_plan_shape(const tgp_batch_plan_t* plan, int32_t i, tgp_config* shape,
                                int32_t* from_cache) {
  if (!plan || !shape || i < 0 || i >= plan->n) return TGP_ERR_INVALID_ARG;
  *shape = plan->shape[i];
  if (from_cache) *from_cache = plan->from_cache[i];
  return TGP_OK;
}

tgp_status tgp_batch_run(const tgp_batch_plan_t* plan, void* ws, size_t ws_bytes, void* stream) {
  if (!plan) return TGP_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TGP_ERR_CUDA;
  if (dev != plan->dev) return TGP_ERR_INVALID_ARG;
  // the launches only read the plan; a run works on its own copy of the
  // per-problem records so that concurrent runs of one plan do not interfere
  Planned qs[TGP_MAX_PROBLEMS];
  for (int i = 0; i < plan->n; ++i) qs[i] = plan->qs[i];
  return launch_batch(qs, plan->n, plan->ws_bytes, plan->dv, ws, ws_bytes, stream);
}

void tgp_batch_free(tgp_batch_plan_t* plan) {
  if (!plan) return;
  plan->~tgp_batch_plan_s();
  std::free(plan);
}

tgp_status tgp_check_device_error(void* ws, size_t ws_bytes, void* stream) {
  if (!ws || ws_bytes < CTRL_WORDS * 4) return TGP_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned word = 0;
  unsigned* ctrl = reinterpret_cast<unsigned*>(ws);
  if (cudaMemcpyAsync(&word, ctrl + CTRL_ERROR, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return TGP_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return TGP_ERR_CUDA;
  if (word != 0) {
    if (cudaMemsetAsync(ctrl + CTRL_ERROR, 0, 4, st) != cudaSuccess) return TGP_ERR_CUDA;
    return TGP_ERR_TIMEOUT;
  }
  return TGP_OK;
}

const char* tgp_status_string(tgp_status s) {
  switch (s) {
    case TGP_OK: return "TGP_OK";
    case TGP_ERR_INVALID_ARG: return "TGP_ERR_INVALID_ARG";
    case TGP_ERR_INVALID_TREE: return "TGP_ERR_INVALID_TREE";
    case TGP_ERR_WORKSPACE: return "TGP_ERR_WORKSPACE";
    case TGP_ERR_CUDA: return "TGP_ERR_CUDA";
    case TGP_ERR_TIMEOUT: return "TGP_ERR_TIMEOUT";
    case TGP_ERR_UNSUPPORTED: return "TGP_ERR_UNSUPPORTED";
  }
  return "TGP_ERR_UNKNOWN";
}

const char* tgp_version(void) { return "tgp-gb300 0.1 (sm_103a)"; }

}  // extern "C"
