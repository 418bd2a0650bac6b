// C ABI of octfuse: context management and the orchestration of the kernels
// of build.cu / solve.cu on the caller's stream.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "descent.cuh"
#include "frames.cuh"
#include "mesh.cuh"
#include "ofu_internal.cuh"
#include "quant.cuh"

namespace ofu {
namespace {
std::atomic<int64_t> g_launches{0};
}
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace ofu

using namespace ofu;

namespace {

thread_local std::string g_create_error;

// Persistent device buffers by role (content not kept across growth).
enum Buf {
  B_SCAN, B_U0, B_PYR, B_FLAGS, B_POS, B_CNT, B_OVFC, B_CLS, B_OUTC, B_JL, B_SRC, B_LIST,
  B_SMALL, B_PART, B_BIG, B_LONGQ, B_FWD, B_AUX, B_FULL, B_PENDQ, B_Q, B_QF, B_QD, B_QT, B_LFL,
  B_MG, B_MC, B_MN, B_MV, B_MT, B_FTC, B_FTT, B_FTL, B_FTH, B_RPYR, B_DRS, B_DRR, B_DRW, B_DRC,
  B_GRS, B_GRR, B_GRW, B_NUM
};

struct Bufs {
  void* p[B_NUM] = {};
  size_t bytes[B_NUM] = {};
};

Bufs& bufs(ofu_ctx* c) {
  // stored behind the scratch pointer of the context
  return *reinterpret_cast<Bufs*>(c->scratch);
}

ofu_status fail(ofu_ctx* c, ofu_status st, const std::string& msg) {
  c->err = msg;
  return st;
}

ofu_status fail_cuda(ofu_ctx* c, cudaError_t e, const char* what) {
  c->poisoned = true;
  c->err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? OFU_ENOMEM : OFU_ECUDA;
}

#define CU(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return fail_cuda(ctx, e_, #call);       \
  } while (0)

#define ST(call)                                \
  do {                                          \
    ofu_status s_ = (call);                     \
    if (s_ != OFU_OK) return s_;                \
  } while (0)

// Device memory of a context: the caller's allocator when one was given,
// else cudaMalloc / cudaFree.  Live blocks are recorded with their sizes.
template <typename T>
cudaError_t dalloc(ofu_ctx* ctx, T** p, size_t bytes) {
  void* q = nullptr;
  if (ctx->alloc_fn) {
    q = ctx->alloc_fn(bytes, ctx->alloc_user);
    if (!q) return cudaErrorMemoryAllocation;
  } else {
    const cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return e;
  }
  ctx->live[q] = bytes;
  *p = static_cast<T*>(q);
  return cudaSuccess;
}

cudaError_t dfree(ofu_ctx* ctx, void* p) {
  if (!p) return cudaSuccess;
  size_t bytes = 0;
  const auto it = ctx->live.find(p);
  if (it != ctx->live.end()) {
    bytes = it->second;
    ctx->live.erase(it);
  }
  if (ctx->free_fn) {
    ctx->free_fn(p, bytes, ctx->alloc_user);
    return cudaSuccess;
  }
  return cudaFree(p);
}

template <typename T>
ofu_status ensure(ofu_ctx* ctx, Buf b, size_t count, T** out) {
  Bufs& B = bufs(ctx);
  const size_t need = std::max<size_t>(count * sizeof(T), 256);
  if (B.bytes[b] < need) {
    if (B.p[b]) CU(dfree(ctx, B.p[b]));
    B.p[b] = nullptr;
    B.bytes[b] = 0;
    const size_t nb = need + need / 4;
    CU(dalloc(ctx, &B.p[b], nb));
    B.bytes[b] = nb;
  }
  *out = reinterpret_cast<T*>(B.p[b]);
  return OFU_OK;
}

void free_leaves(ofu_ctx* ctx, Leaves& L) {
  for (void* q : {static_cast<void*>(L.key), static_cast<void*>(L.level), static_cast<void*>(L.u),
                  static_cast<void*>(L.ubar), static_cast<void*>(L.p), static_cast<void*>(L.tau),
                  static_cast<void*>(L.sigma), static_cast<void*>(L.nbr),
                  static_cast<void*>(L.soff), static_cast<void*>(L.khint), static_cast<void*>(L.ovf)})
    dfree(ctx, q);
  L = Leaves{};
}

ofu_status ensure_leaves(ofu_ctx* ctx, int which, int64_t need) {
  Leaves& L = ctx->L[which];
  if (L.cap >= need) return OFU_OK;
  free_leaves(ctx, L);
  const int64_t cap = std::max<int64_t>(need + need / 4, 1024);
  CU(dalloc(ctx, &L.key, cap * sizeof(uint64_t)));
  CU(dalloc(ctx, &L.level, cap));
  CU(dalloc(ctx, &L.u, cap * sizeof(float)));
  CU(dalloc(ctx, &L.ubar, cap * sizeof(float)));
  CU(dalloc(ctx, &L.p, 3 * cap * sizeof(float)));
  CU(dalloc(ctx, &L.tau, cap * sizeof(float)));
  CU(dalloc(ctx, &L.sigma, cap * sizeof(float)));
  CU(dalloc(ctx, &L.nbr, 6 * cap * sizeof(int32_t)));
  CU(dalloc(ctx, &L.soff, (cap + 1) * sizeof(uint32_t)));
  CU(dalloc(ctx, &L.khint, cap * sizeof(uint16_t)));
  L.cap = cap;
  return OFU_OK;
}

size_t sample_bytes(const ofu_ctx* ctx) { return ctx->prm.sample_fp16 ? 2 : 4; }

ofu_status ensure_samples(ofu_ctx* ctx, int which, int64_t need) {
  if (ctx->samp_cap[which] >= need && ctx->samp[which]) return OFU_OK;
  if (ctx->samp[which]) CU(dfree(ctx, ctx->samp[which]));
  ctx->samp[which] = nullptr;
  const int64_t cap = std::max<int64_t>(need + need / 4, 4096);
  CU(dalloc(ctx, &ctx->samp[which], size_t(cap) * sample_bytes(ctx) + 16));
  ctx->samp_cap[which] = cap;
  return OFU_OK;
}

View view_of(const ofu_ctx* ctx) {
  const Leaves& L = ctx->L[ctx->cur];
  View v;
  v.n = ctx->n;
  v.D = ctx->prm.max_depth;
  v.key = L.key;
  v.level = L.level;
  v.nbr = L.nbr;
  v.ovf = L.ovf;
  v.stride = L.cap;
  v.map = ctx->map;
  return v;
}

Geo geo_of(const ofu_ctx* ctx) {
  Geo g;
  for (int k = 0; k < 3; ++k) g.org[k] = float(ctx->prm.origin[k]);
  g.vox = float(ctx->prm.extent) / float(1 << ctx->prm.max_depth);
  g.delta = float(ctx->prm.delta);
  g.eta = float(ctx->prm.eta);
  g.D = ctx->prm.max_depth;
  return g;
}

// Heavy and list leaves of the current structure for the dual (or primal) step.
LeafSets dual_sets(const ofu_ctx* ctx) {
  LeafSets ls;
  ls.heavy = ctx->heavy;
  ls.n_heavy = ctx->n_heavy_dual;
  ls.list = ctx->heavy + 2 * ctx->heavy_cap;
  ls.n_list = ctx->n_list_dual;
  return ls;
}
LeafSets primal_sets(const ofu_ctx* ctx) {
  LeafSets ls;
  ls.heavy = ctx->heavy + ctx->heavy_cap;
  ls.n_heavy = ctx->n_heavy_primal;
  ls.list = ctx->heavy + 3 * ctx->heavy_cap;
  ls.n_list = ctx->n_list_primal;
  return ls;
}

// Copies `bytes` from device to a pinned host staging area and waits.
ofu_status read_back(ofu_ctx* ctx, const void* dev, size_t bytes, void* host) {
  CU(cudaMemcpyAsync(ctx->pinned, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  std::memcpy(host, ctx->pinned, bytes);
  return OFU_OK;
}

// Events of the per-launch timing: 3 per iteration, at least 8192 iterations;
// at most 2^20 iterations.
constexpr size_t kProfEvents = 3 * 8192;
constexpr int32_t kProfMaxIters = 1 << 20;

int64_t max_leaves(const ofu_ctx* ctx) {
  return ctx->prm.max_leaves > 0 ? std::min<int64_t>(ctx->prm.max_leaves, kMaxLeaves) : kMaxLeaves;
}

// The per-frame trees handed to the sample kernels (empty: Eq. 1 at centres).
FrameTrees trees_of(const ofu_ctx* ctx) {
  FrameTrees t;
  if (ctx->prm.data_term == 1 && ctx->ft_start) {
    t.start = ctx->ft_start;
    t.key = ctx->ft_key;
    t.level = ctx->ft_level;
    t.cnt = ctx->ft_cnt;
    t.tot = ctx->ft_tot;
    t.pcnt = ctx->ft_pcnt;
    t.ptot = ctx->ft_ptot;
  }
  return t;
}

void free_frame_trees(ofu_ctx* ctx) {
  for (void* q : {static_cast<void*>(ctx->ft_start), static_cast<void*>(ctx->ft_key),
                  static_cast<void*>(ctx->ft_level), static_cast<void*>(ctx->ft_cnt),
                  static_cast<void*>(ctx->ft_tot), static_cast<void*>(ctx->ft_pcnt),
                  static_cast<void*>(ctx->ft_ptot)})
    dfree(ctx, q);
  ctx->ft_start = nullptr;
  ctx->ft_key = nullptr;
  ctx->ft_level = nullptr;
  ctx->ft_cnt = nullptr;
  ctx->ft_tot = nullptr;
  ctx->ft_pcnt = nullptr;
  ctx->ft_ptot = nullptr;
  ctx->ft_cap = 0;
  ctx->ft_host_start.clear();
}

// Grows the tree-leaf arrays to hold `need` leaves, keeping the first `keep`.
ofu_status grow_frame_trees(ofu_ctx* ctx, int64_t need, int64_t keep) {
  if (need <= ctx->ft_cap) return OFU_OK;
  const int64_t cap = std::max<int64_t>(need + need / 2, 1 << 16);
  uint64_t *key, *cnt;
  uint8_t* level;
  double* tot;
  CU(dalloc(ctx, &key, size_t(cap) * 8));
  CU(dalloc(ctx, &level, size_t(cap)));
  CU(dalloc(ctx, &cnt, size_t(cap) * 8));
  CU(dalloc(ctx, &tot, size_t(cap) * 8));
  if (keep > 0) {
    CU(cudaMemcpyAsync(key, ctx->ft_key, size_t(keep) * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(level, ctx->ft_level, size_t(keep), cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(cnt, ctx->ft_cnt, size_t(keep) * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    CU(cudaMemcpyAsync(tot, ctx->ft_tot, size_t(keep) * 8, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  for (void* q : {static_cast<void*>(ctx->ft_key), static_cast<void*>(ctx->ft_level),
                  static_cast<void*>(ctx->ft_cnt), static_cast<void*>(ctx->ft_tot)})
    CU(dfree(ctx, q));
  ctx->ft_key = key;
  ctx->ft_level = level;
  ctx->ft_cnt = cnt;
  ctx->ft_tot = tot;
  ctx->ft_cap = cap;
  return OFU_OK;
}

// Per-frame TSDF octrees of the current frames (data_term = 1), frame by
// frame: pyramid and leaf flags, scan, one read-back of the frame's leaf
// count, emission; then prefix sums of counts and sums over all frames.
ofu_status build_frame_trees(ofu_ctx* ctx) {
  const int D = ctx->prm.max_depth;
  const int64_t nvox = int64_t(1) << (3 * D);
  const size_t npyr = frame_pyramid_nodes(D);
  uint32_t *pc, *flags, *pos, *tmp;
  double* pt;
  float *pl, *ph;
  ST(ensure(ctx, B_FTC, std::max<size_t>(npyr, 1), &pc));
  ST(ensure(ctx, B_FTT, std::max<size_t>(npyr, 1), &pt));
  ST(ensure(ctx, B_FTL, std::max<size_t>(npyr, 1), &pl));
  ST(ensure(ctx, B_FTH, std::max<size_t>(npyr, 1), &ph));
  ST(ensure(ctx, B_FLAGS, size_t(nvox), &flags));
  ST(ensure(ctx, B_POS, size_t(nvox + 1), &pos));
  ST(ensure(ctx, B_SCAN, scan_tmp_items<uint32_t>(nvox) * 2, &tmp));
  const Geo g = geo_of(ctx);
  std::vector<int64_t> start(size_t(ctx->F) + 1, 0);
  for (int i = 0; i < ctx->F; ++i) {
    const float* range = ctx->depth + size_t(i) * ctx->H * ctx->W;
    CU(launch_frame_tree_flags(range, ctx->cams + i, ctx->H, ctx->W, g, ctx->prm.spread_tau, pc, pt,
                               pl, ph, flags, ctx->stream));
    CU(scan_exclusive<uint32_t>(flags, pos, nvox, tmp, ctx->stream));
    uint32_t ni = 0;
    ST(read_back(ctx, pos + nvox, sizeof(uint32_t), &ni));
    ST(grow_frame_trees(ctx, start[i] + int64_t(ni), start[i]));
    const int64_t o = start[i];
    CU(launch_frame_tree_emit(flags, pos, pc, pt, pl, ph, ctx->prm.spread_tau, range, ctx->cams + i,
                              ctx->H, ctx->W, g, ctx->ft_key + o, ctx->ft_level + o, ctx->ft_cnt + o,
                              ctx->ft_tot + o, ctx->stream));
    start[i + 1] = o + int64_t(ni);
  }
  const int64_t total = start[ctx->F];
  for (void* q : {static_cast<void*>(ctx->ft_start), static_cast<void*>(ctx->ft_pcnt),
                  static_cast<void*>(ctx->ft_ptot)})
    CU(dfree(ctx, q));
  ctx->ft_start = nullptr;
  ctx->ft_pcnt = nullptr;
  ctx->ft_ptot = nullptr;
  CU(dalloc(ctx, &ctx->ft_start, start.size() * 8));
  CU(dalloc(ctx, &ctx->ft_pcnt, size_t(total + 1) * 8));
  CU(dalloc(ctx, &ctx->ft_ptot, size_t(total + 1) * 8));
  CU(cudaMemcpyAsync(ctx->ft_start, start.data(), start.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
  uint64_t* t64;
  ST(ensure(ctx, B_OUTC, scan_tmp_items<uint64_t>(total) * 2 + scan_tmp_items<double>(total) * 2, &t64));
  CU(scan_exclusive<uint64_t>(ctx->ft_cnt, ctx->ft_pcnt, total, t64, ctx->stream));
  CU(scan_exclusive<double>(ctx->ft_tot, ctx->ft_ptot, total, reinterpret_cast<double*>(t64),
                            ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));   // the host copy of start is released on return
  ctx->ft_host_start = start;
  return OFU_OK;
}

// Voxel -> leaf map of the current structure.
ofu_status rebuild_map(ofu_ctx* ctx) {
  const int D = ctx->prm.max_depth;
  if (!ctx->map) CU(dalloc(ctx, &ctx->map, (size_t(1) << (3 * D)) * sizeof(uint32_t)));
  uint32_t* big;
  uint64_t* small;
  ST(ensure(ctx, B_BIG, size_t(ctx->n), &big));
  ST(ensure(ctx, B_SMALL, 8, &small));
  Leaves& L = ctx->L[ctx->cur];
  CU(launch_map(L.key, L.level, ctx->n, D, ctx->map, big,
                reinterpret_cast<unsigned long long*>(small + 5), ctx->stream));
  return OFU_OK;
}

// Voxel map, face neighbours, heavy leaves and step sizes of the current
// structure.  One host synchronisation (the size of the neighbour lists, the
// heavy-leaf counts and, when `samples_total` is given, the sample count).
// With `carry` (the structure before a split/join pass) the entries of kept
// leaves among kept neighbours are carried over instead of searched.
ofu_status rebuild_topology(ofu_ctx* ctx, const uint32_t* samples_total = nullptr,
                            Carry carry = Carry{}) {
  const int64_t n = ctx->n;
  // new leaves: no prox hint yet (0xffff is clamped to W, i.e. a full search)
  CU(cudaMemsetAsync(ctx->L[ctx->cur].khint, 0xff, size_t(std::max<int64_t>(n, 1)) * sizeof(uint16_t),
                     ctx->stream));
  ST(rebuild_map(ctx));
  uint32_t* ovfc;
  uint32_t* tmp;
  uint32_t* longq;
  uint64_t* small;
  ST(ensure(ctx, B_OVFC, size_t(6 * n + 1), &ovfc));
  ST(ensure(ctx, B_SCAN, scan_tmp_items<uint32_t>(6 * n) * 2, &tmp));
  ST(ensure(ctx, B_LONGQ, size_t(6 * n), &longq));
  uint32_t* pendq;
  ST(ensure(ctx, B_PENDQ, size_t(6 * n), &pendq));
  ST(ensure(ctx, B_SMALL, 16, &small));
  if (ctx->heavy_cap < n) {
    if (ctx->heavy) CU(dfree(ctx, ctx->heavy));
    ctx->heavy = nullptr;
    ctx->heavy_cap = 0;
    const int64_t cap = std::max<int64_t>(n + n / 4, 1024);
    CU(dalloc(ctx, &ctx->heavy, 4 * size_t(cap) * sizeof(uint32_t)));
    ctx->heavy_cap = cap;
  }
  unsigned long long* nlong = reinterpret_cast<unsigned long long*>(small + 8);
  unsigned long long* npend = reinterpret_cast<unsigned long long*>(small + 11);
  uint64_t *hflags, *lflags, *htmp;
  ST(ensure(ctx, B_CLS, size_t(n + 1), &hflags));
  ST(ensure(ctx, B_LFL, size_t(n + 1), &lflags));
  ST(ensure(ctx, B_OUTC, scan_tmp_items<uint64_t>(n) * 2, &htmp));
  if (carry.nbr) {
    ST(ensure(ctx, B_AUX, size_t(6 * n), &carry.aux));
    ST(ensure(ctx, B_FULL, size_t(6 * n), &carry.full));
  }
  Leaves& L = ctx->L[ctx->cur];
  View v = view_of(ctx);
  CU(launch_nbr_count(v, carry, L.nbr, ovfc, longq, nlong, pendq, npend, ctx->stream));
  CU(launch_leaf_sets(v, ovfc, hflags, lflags, htmp, ctx->heavy, ctx->heavy_cap, ctx->stream));
  CU(scan_exclusive<uint32_t>(ovfc, ovfc, 6 * n, tmp, ctx->stream));
  // one read-back: packed heavy counts (slot 9), [list total, samples] (slot 10),
  // packed list-leaf counts (slot 13)
  CU(cudaMemcpyAsync(small + 9, hflags + n, sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream));
  CU(cudaMemcpyAsync(small + 13, lflags + n, sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream));
  CU(cudaMemcpyAsync(reinterpret_cast<uint32_t*>(small + 10), ovfc + 6 * n, sizeof(uint32_t),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  if (samples_total)
    CU(cudaMemcpyAsync(reinterpret_cast<uint32_t*>(small + 10) + 1, samples_total, sizeof(uint32_t),
                       cudaMemcpyDeviceToDevice, ctx->stream));
  uint64_t hs[5];
  ST(read_back(ctx, small + 9, 5 * sizeof(uint64_t), hs));
  ctx->n_heavy_dual = int(hs[0] & 0xffffffffu);
  ctx->n_heavy_primal = int(hs[0] >> 32);
  ctx->n_list_dual = int(hs[4] & 0xffffffffu);
  ctx->n_list_primal = int(hs[4] >> 32);
  const uint32_t total = uint32_t(hs[1] & 0xffffffffu);
  if (samples_total) ctx->n_samples = int64_t(hs[1] >> 32);
  if (int64_t(total) + 1 > L.ovf_cap) {
    if (L.ovf) CU(dfree(ctx, L.ovf));
    L.ovf = nullptr;
    L.ovf_cap = 0;
    const int64_t cap = std::max<int64_t>(int64_t(total) + int64_t(total) / 4 + 1, 1024);
    if (cap >= 0x7fffffffLL) return fail(ctx, OFU_ECAPACITY, "neighbour lists exceed 2^31 entries");
    CU(dalloc(ctx, &L.ovf, size_t(cap) * sizeof(int32_t)));
    L.ovf_cap = cap;
  }
  v = view_of(ctx);
  CU(launch_nbr_fill(v, carry, ovfc, L.nbr, L.ovf, longq, nlong, pendq, npend, ctx->stream));
  v = view_of(ctx);
  CU(launch_precond(v, carry, L.tau, L.sigma, ctx->heavy + ctx->heavy_cap, ctx->n_heavy_primal,
                    ctx->stream));
  // neighbour records of the heavy and list leaves (the dual step's +face
  // gradient records, the primal step's -face divergence records): at most
  // every list entry plus three single neighbours per leaf, so no read-back
  for (int plus = 0; plus < 2; ++plus) {
    const LeafSets ls = plus ? dual_sets(ctx) : primal_sets(ctx);
    const int64_t ng = int64_t(ls.n_heavy) + ls.n_list;
    uint32_t *rstart, *rrec;
    float *rw, *rcp = nullptr;
    ST(ensure(ctx, plus ? B_GRS : B_DRS, size_t(ng + 1), &rstart));
    ST(ensure(ctx, plus ? B_GRR : B_DRR, size_t(total) + 3 * size_t(ng) + 1, &rrec));
    ST(ensure(ctx, plus ? B_GRW : B_DRW, size_t(total) + 3 * size_t(ng) + 1, &rw));
    if (!plus) ST(ensure(ctx, B_DRC, 3 * size_t(ng) + 1, &rcp));
    if (ng > 0) {
      CU(launch_recs_count(v, ls, plus != 0, rstart, ctx->stream));
      CU(scan_exclusive<uint32_t>(rstart, rstart, ng, tmp, ctx->stream));
      CU(launch_recs_fill(v, ls, plus != 0, rstart, rrec, rw, rcp, ctx->stream));
    }
  }
  return OFU_OK;
}

// The records built by rebuild_topology (gradient: the dual step's sets;
// divergence: the primal step's).
NbrRecs nbr_recs(ofu_ctx* ctx, bool gradient) {
  Bufs& B = bufs(ctx);
  NbrRecs d;
  d.start = static_cast<const uint32_t*>(B.p[gradient ? B_GRS : B_DRS]);
  d.rec = static_cast<const uint32_t*>(B.p[gradient ? B_GRR : B_DRR]);
  d.w = static_cast<const float*>(B.p[gradient ? B_GRW : B_DRW]);
  d.cp = gradient ? nullptr : static_cast<const float*>(B.p[B_DRC]);
  return d;
}

// Eq. 1 samples of all current leaves; with init, u = ubar = median, p = 0.
ofu_status integrate_all(ofu_ctx* ctx, bool init) {
  const int64_t n = ctx->n;
  Leaves& L = ctx->L[ctx->cur];
  const Geo g = geo_of(ctx);
  uint32_t* tmp;
  ST(ensure(ctx, B_SCAN, scan_tmp_items<uint32_t>(n) * 2, &tmp));
  CU(launch_leaf_count(L.key, L.level, nullptr, nullptr, n, ctx->depth, ctx->cams, ctx->F, ctx->H,
                       ctx->W, g, trees_of(ctx), L.soff, ctx->stream));
  CU(scan_exclusive<uint32_t>(L.soff, L.soff, n, tmp, ctx->stream));
  uint32_t total = 0;
  ST(read_back(ctx, L.soff + n, sizeof(uint32_t), &total));
  ST(ensure_samples(ctx, ctx->cur, int64_t(total)));
  ctx->n_samples = total;
  CU(launch_leaf_fill(L.key, L.level, nullptr, nullptr, n, ctx->depth, ctx->cams, ctx->F, ctx->H,
                      ctx->W, g, trees_of(ctx), L.soff, ctx->samp[ctx->cur], ctx->prm.sample_fp16 != 0,
                      init ? L.u : nullptr, init ? L.ubar : nullptr, ctx->stream));
  if (init) CU(cudaMemsetAsync(L.p, 0, 3 * L.cap * sizeof(float), ctx->stream));
  return OFU_OK;
}

// Count check on the sample total (offsets are 32-bit).
bool samples_fit(int64_t n, int F) { return n * int64_t(F) < int64_t(0xffffffffu); }

ofu_status check_ready(ofu_ctx* ctx) {
  if (!ctx) return OFU_EINVAL;
  if (ctx->poisoned) return fail(ctx, OFU_ESTATE, "context poisoned by an earlier CUDA error: " + ctx->err);
  return OFU_OK;
}

ofu_status check_built(ofu_ctx* ctx) {
  ST(check_ready(ctx));
  if (!ctx->have_frames || ctx->n == 0) return fail(ctx, OFU_ESTATE, "no octree: call ofu_integrate_frames first");
  return OFU_OK;
}

ofu_status validate(const ofu_params* p, std::string* why) {
  auto bad = [&](const char* m) { *why = m; return OFU_EINVAL; };
  if (!p) return bad("params is NULL");
  if (!(p->extent > 0) || !std::isfinite(p->extent)) return bad("extent must be finite and > 0");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(p->origin[k])) return bad("origin must be finite");
  if (p->max_depth < 1 || p->max_depth > kMaxDepth) return bad("max_depth must be in 1..15");
  if (!(p->delta > 0) || !std::isfinite(p->delta)) return bad("delta must be finite and > 0");
  if (!(p->eta >= 0) || !std::isfinite(p->eta)) return bad("eta must be finite and >= 0");
  if (!(p->lambda >= 0) || !std::isfinite(p->lambda)) return bad("lambda must be finite and >= 0");
  if (!(p->gamma > 0) || !std::isfinite(p->gamma)) return bad("gamma must be finite and > 0");
  if (std::isnan(p->tau_split) || std::isnan(p->tau_join) || std::isnan(p->spread_tau))
    return bad("thresholds must not be NaN");
  if (p->tau_join < p->tau_split) return bad("tau_join must be >= tau_split");
  if (p->sample_fp16 != 0 && p->sample_fp16 != 1) return bad("sample_fp16 must be 0 or 1");
  if (p->max_leaves < 0) return bad("max_leaves must be >= 0");
  if (p->data_term != 0 && p->data_term != 1) return bad("data_term must be 0 or 1");
  if (p->reserved != 0) return bad("reserved must be 0");
  return OFU_OK;
}

}  // namespace

extern "C" {

void ofu_default_params(ofu_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  for (int k = 0; k < 3; ++k) p->origin[k] = -0.5;
  p->extent = 1.0;
  p->max_depth = 6;
  p->sample_fp16 = 0;
  p->delta = 4.0 / 64.0;
  p->eta = 2.0 * p->delta;
  p->lambda = 0.5;
  p->gamma = 1e-3;
  p->tau_split = 0.95;
  p->tau_join = 0.99;
  p->spread_tau = 0.1;
  p->max_leaves = 0;
}

ofu_status ofu_create_octree(const ofu_params* params, void* cuda_stream, ofu_ctx** out) {
  return ofu_create_octree_ex(params, cuda_stream, nullptr, nullptr, nullptr, out);
}

ofu_status ofu_create_octree_ex(const ofu_params* params, void* cuda_stream, ofu_alloc_fn alloc,
                                ofu_free_fn free_fn, void* user, ofu_ctx** out) {
  if (!out) {
    g_create_error = "out is NULL";
    return OFU_EINVAL;
  }
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    *out = nullptr;
    g_create_error = "create_octree_ex: give both alloc and free_fn, or neither";
    return OFU_EINVAL;
  }
  *out = nullptr;
  std::string why;
  if (validate(params, &why) != OFU_OK) {
    g_create_error = why;
    return OFU_EINVAL;
  }
  ofu_ctx* ctx = new ofu_ctx();
  ctx->prm = *params;
  ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  ctx->alloc_fn = alloc;
  ctx->free_fn = free_fn;
  ctx->alloc_user = user;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->pinned, 256);
  if (e != cudaSuccess) {
    g_create_error = std::string("CUDA initialisation failed: ") + cudaGetErrorString(e);
    cudaGetLastError();
    delete ctx;
    return e == cudaErrorMemoryAllocation ? OFU_ENOMEM : OFU_ECUDA;
  }
  ctx->scratch = new Bufs();
  *out = ctx;
  return OFU_OK;
}

void ofu_destroy(ofu_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  free_leaves(ctx, ctx->L[0]);
  free_leaves(ctx, ctx->L[1]);
  dfree(ctx, ctx->samp[0]);
  dfree(ctx, ctx->samp[1]);
  dfree(ctx, ctx->depth);
  dfree(ctx, ctx->cams);
  dfree(ctx, ctx->map);
  dfree(ctx, ctx->heavy);
  free_frame_trees(ctx);
  if (ctx->scratch) {
    Bufs& B = bufs(ctx);
    for (int b = 0; b < B_NUM; ++b) dfree(ctx, B.p[b]);
    delete &B;
  }
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
  cudaGetLastError();
  delete ctx;
}

const char* ofu_last_error(const ofu_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

ofu_status ofu_integrate_frames(ofu_ctx* ctx, int32_t F, int32_t H, int32_t W, const float* depth,
                                const double* intr, const double* pose) {
  ST(check_ready(ctx));
  if (F < 1 || H < 1 || W < 1 || !depth || !intr || !pose)
    return fail(ctx, OFU_EINVAL, "integrate_frames: F, H, W must be >= 1 and pointers non-NULL");
  if (F > 512) return fail(ctx, OFU_EINVAL, "integrate_frames: at most 512 frames");
  if (int64_t(H) * W >= (int64_t(1) << 31)) return fail(ctx, OFU_EINVAL, "integrate_frames: frame too large");
  const int D = ctx->prm.max_depth;
  const int64_t nvox = int64_t(1) << (3 * D);
  if (nvox >= (int64_t(1) << 32)) return fail(ctx, OFU_ECAPACITY, "max_depth too large for the dense construction pass");

  // frames
  std::vector<double> hi(size_t(F) * 4), hp(size_t(F) * 16);
  CU(cudaMemcpy(hi.data(), intr, hi.size() * sizeof(double), cudaMemcpyDefault));
  CU(cudaMemcpy(hp.data(), pose, hp.size() * sizeof(double), cudaMemcpyDefault));
  std::vector<Cam> cams(F);
  for (int i = 0; i < F; ++i) {
    const double* P = &hp[size_t(i) * 16];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) cams[i].r[r * 3 + c] = float(P[r * 4 + c]);
    for (int r = 0; r < 3; ++r) cams[i].c[r] = float(P[r * 4 + 3]);
    cams[i].fx = float(hi[size_t(i) * 4 + 0]);
    cams[i].fy = float(hi[size_t(i) * 4 + 1]);
    cams[i].cx = float(hi[size_t(i) * 4 + 2]);
    cams[i].cy = float(hi[size_t(i) * 4 + 3]);
    if (!(cams[i].fx != 0.0f) || !(cams[i].fy != 0.0f))
      return fail(ctx, OFU_EINVAL, "integrate_frames: focal lengths must be non-zero");
  }
  const size_t dbytes = size_t(F) * H * W * sizeof(float);
  if (ctx->depth && size_t(ctx->F) * ctx->H * ctx->W * sizeof(float) < dbytes) {
    CU(dfree(ctx, ctx->depth));
    ctx->depth = nullptr;
  }
  if (!ctx->depth) CU(dalloc(ctx, &ctx->depth, dbytes));
  if (ctx->cams) CU(dfree(ctx, ctx->cams));
  ctx->cams = nullptr;
  CU(dalloc(ctx, &ctx->cams, size_t(F) * sizeof(Cam)));
  CU(cudaMemcpyAsync(ctx->depth, depth, dbytes, cudaMemcpyDefault, ctx->stream));
  CU(cudaMemcpyAsync(ctx->cams, cams.data(), size_t(F) * sizeof(Cam), cudaMemcpyHostToDevice, ctx->stream));
  CU(launch_range_map(ctx->depth, ctx->cams, F, H, W, ctx->stream));
  ctx->F = F;
  ctx->H = H;
  ctx->W = W;
  ctx->have_frames = true;
  ctx->n = 0;
  if (ctx->prm.data_term == 1) ST(build_frame_trees(ctx));

  // Eq. 2 construction on the median field
  const Geo g = geo_of(ctx);
  double *u0, *pyr;
  uint32_t *flags, *pos, *tmp;
  ST(ensure(ctx, B_U0, size_t(nvox), &u0));
  const int64_t npyr = ((int64_t(1) << (3 * D)) - 1) / 7;
  ST(ensure(ctx, B_PYR, size_t(2 * npyr), &pyr));
  ST(ensure(ctx, B_FLAGS, size_t(nvox), &flags));
  ST(ensure(ctx, B_POS, size_t(nvox + 1), &pos));
  ST(ensure(ctx, B_SCAN, scan_tmp_items<uint32_t>(nvox) * 2, &tmp));
  uint64_t* small;
  ST(ensure(ctx, B_SMALL, 16, &small));
  // min / max pyramid of the range maps for the scan's frame classification
  RangePyr rp = range_pyr_dims(H, W);
  float2* rtex = nullptr;
  ST(ensure(ctx, B_RPYR, size_t(std::max<int64_t>(int64_t(F) * rp.frame_texels, 1)), &rtex));
  rp.tex = rtex;
  CU(launch_range_pyr(ctx->depth, F, H, W, rp, rtex, ctx->stream));
  // pos is free until the leaf flags are scanned: it holds the voxels whose
  // median needs a sort
  CU(launch_dense_u0(ctx->depth, ctx->cams, F, H, W, g, rp, u0, pos,
                     reinterpret_cast<unsigned long long*>(small + 12), ctx->stream));
  CU(launch_pyramid(u0, D, pyr, pyr + npyr, ctx->stream));
  CU(launch_leaf_flags(pyr, pyr + npyr, D, ctx->prm.spread_tau, flags, ctx->stream));
  CU(scan_exclusive<uint32_t>(flags, pos, nvox, tmp, ctx->stream));
  uint32_t N = 0;
  ST(read_back(ctx, pos + nvox, sizeof(uint32_t), &N));
  if (int64_t(N) > max_leaves(ctx)) return fail(ctx, OFU_ECAPACITY, "construction exceeds max_leaves");
  if (!samples_fit(N, F)) return fail(ctx, OFU_ECAPACITY, "sample count may exceed 2^32");
  ST(ensure_leaves(ctx, ctx->cur, N));
  Leaves& L = ctx->L[ctx->cur];
  CU(launch_emit_constructed(flags, pos, pyr, pyr + npyr, D, ctx->prm.spread_tau, L.key, L.level,
                             ctx->stream));
  ctx->n = N;
  ST(integrate_all(ctx, true));
  ST(rebuild_topology(ctx));
  return OFU_OK;
}

ofu_status ofu_iterate(ofu_ctx* ctx, int32_t n) {
  ST(check_built(ctx));
  if (n < 0) return fail(ctx, OFU_EINVAL, "iterate: n must be >= 0");
  Leaves& L = ctx->L[ctx->cur];
  const View v = view_of(ctx);
  const bool h16 = ctx->prm.sample_fp16 != 0;
  for (int k = 0; k < n; ++k) {
    // events come from a pool created by ofu_profile(ctx, 1); recording stops
    // (silently) once the pool is used up
    const bool rec = ctx->prof_on && ctx->prof_used + 3 <= ctx->prof_ev.size();
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    if (rec) {
      for (int j = 0; j < 3; ++j) ev[j] = ctx->prof_ev[ctx->prof_used + j];
      ctx->prof_used += 3;
      CU(cudaEventRecord(ev[0], ctx->stream));
    }
    CU(launch_dual(v, L.ubar, L.p, L.sigma, float(ctx->prm.lambda), dual_sets(ctx),
                   nbr_recs(ctx, true), ctx->stream));
    if (rec) CU(cudaEventRecord(ev[1], ctx->stream));
    CU(launch_primal(v, L.u, L.ubar, L.p, L.tau, L.soff, ctx->samp[ctx->cur], h16,
                     float(ctx->prm.gamma), L.khint, primal_sets(ctx), nbr_recs(ctx, false), ctx->stream));
    if (rec) {
      CU(cudaEventRecord(ev[2], ctx->stream));
      ctx->prof_launches[0] += 1;
      ctx->prof_launches[1] += 1;
      ctx->prof_bytes[0] += 45.0 * double(ctx->n);
      ctx->prof_bytes[1] += 57.0 * double(ctx->n) + double(ctx->n_samples) * double(sample_bytes(ctx));
    }
  }
  return OFU_OK;
}

ofu_status ofu_restructure(ofu_ctx* ctx, int64_t* n_split, int64_t* n_join, int64_t* n_leaves) {
  ST(check_built(ctx));
  const int64_t n = ctx->n;
  const int D = ctx->prm.max_depth;
  Leaves& L = ctx->L[ctx->cur];
  uint64_t *cls, *outc, *tmp64, *small;
  int8_t* jl;
  ST(ensure(ctx, B_CLS, size_t(n + 1), &cls));
  ST(ensure(ctx, B_OUTC, size_t(n + 1), &outc));
  ST(ensure(ctx, B_JL, size_t(n), &jl));
  ST(ensure(ctx, B_SCAN, scan_tmp_items<uint64_t>(n) * 2, &tmp64));
  ST(ensure(ctx, B_SMALL, 8, &small));
  View v = view_of(ctx);
  CU(cudaMemsetAsync(small, 0, 8 * sizeof(uint64_t), ctx->stream));
  CU(launch_classify(L.u, n, ctx->prm.tau_join, cls, ctx->stream));
  CU(scan_exclusive<uint64_t>(cls, cls, n, tmp64, ctx->stream));
  CU(launch_mark(v, L.u, cls, ctx->prm.tau_split, ctx->prm.tau_join, outc, jl,
                 reinterpret_cast<unsigned long long*>(small), ctx->stream));
  CU(scan_exclusive<uint64_t>(outc, outc, n, tmp64, ctx->stream));
  CU(cudaMemcpyAsync(small + 2, outc + n, sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream));
  uint64_t hs[3];
  ST(read_back(ctx, small, 3 * sizeof(uint64_t), hs));
  const int64_t ns = int64_t(hs[0]), nj = int64_t(hs[1]), n_new = int64_t(hs[2]);
  if (ns == 0 && nj == 0) {
    CU(cudaMemcpyAsync(L.ubar, L.u, size_t(n) * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    if (n_split) *n_split = 0;
    if (n_join) *n_join = 0;
    if (n_leaves) *n_leaves = n;
    return OFU_OK;
  }
  if (n_new > max_leaves(ctx)) return fail(ctx, OFU_ECAPACITY, "restructure exceeds max_leaves");
  if (!samples_fit(n_new, ctx->F)) return fail(ctx, OFU_ECAPACITY, "sample count may exceed 2^32");
  const int nx = 1 - ctx->cur;
  ST(ensure_leaves(ctx, nx, n_new));
  Leaves& N2 = ctx->L[nx];
  int32_t* src;
  uint32_t *list, *tmp32;
  ST(ensure(ctx, B_SRC, size_t(n_new), &src));
  ST(ensure(ctx, B_LIST, size_t(n_new), &list));
  ST(ensure(ctx, B_SCAN, std::max(scan_tmp_items<uint64_t>(n) * 2, scan_tmp_items<uint32_t>(n_new) * 2 / 2 + 1), &tmp64));
  tmp32 = reinterpret_cast<uint32_t*>(tmp64);
  v = view_of(ctx);
  uint32_t* big;
  int32_t* fwd;
  ST(ensure(ctx, B_BIG, size_t(n), &big));
  ST(ensure(ctx, B_FWD, size_t(n), &fwd));
  CU(launch_emit(v, L.u, L.p, outc, jl, N2.key, N2.level, N2.u, N2.ubar, N2.p, N2.cap, src, fwd,
                 big, reinterpret_cast<unsigned long long*>(small + 4), ctx->stream));
  // new leaves (split children, joined nodes) are listed on the device and
  // integrated without a host round trip; the sample buffer is sized for the
  // worst case (every frame observes every new leaf)
  unsigned long long* nlist = reinterpret_cast<unsigned long long*>(small + 3);
  CU(cudaMemsetAsync(nlist, 0, sizeof(uint64_t), ctx->stream));
  CU(launch_new_list(src, n_new, list, nlist, ctx->stream));
  CU(launch_kept_counts(src, L.soff, n_new, N2.soff, ctx->stream));
  const Geo g = geo_of(ctx);
  CU(launch_leaf_count(N2.key, N2.level, list, nlist, n_new, ctx->depth, ctx->cams, ctx->F, ctx->H,
                       ctx->W, g, trees_of(ctx), N2.soff, ctx->stream));
  CU(scan_exclusive<uint32_t>(N2.soff, N2.soff, n_new, tmp32, ctx->stream));
  ST(ensure_samples(ctx, nx, n_new * int64_t(ctx->F)));
  const bool h16 = ctx->prm.sample_fp16 != 0;
  CU(launch_copy_kept_samples(src, n_new, L.soff, ctx->samp[ctx->cur], N2.soff, ctx->samp[nx], h16,
                              ctx->stream));
  CU(launch_leaf_fill(N2.key, N2.level, list, nlist, n_new, ctx->depth, ctx->cams, ctx->F, ctx->H,
                      ctx->W, g, trees_of(ctx), N2.soff, ctx->samp[nx], h16, nullptr, nullptr, ctx->stream));
  Carry carry;
  carry.nbr = L.nbr;
  carry.ovf = L.ovf;
  carry.stride = L.cap;
  carry.src = src;
  carry.fwd = fwd;
  carry.tau = L.tau;
  carry.sigma = L.sigma;
  ctx->cur = nx;
  ctx->n = n_new;
  (void)D;
  ST(rebuild_topology(ctx, N2.soff + n_new, carry));
  if (n_split) *n_split = ns;
  if (n_join) *n_join = nj;
  if (n_leaves) *n_leaves = n_new;
  return OFU_OK;
}

ofu_status ofu_descend(ofu_ctx* ctx, int32_t n, int32_t t0, double eps, double xi0,
                       int32_t halve_every) {
  ST(check_built(ctx));
  if (n < 0 || t0 < 0) return fail(ctx, OFU_EINVAL, "descend: n and t0 must be >= 0");
  if (!(eps > 0) || !(xi0 > 0) || !std::isfinite(eps) || !std::isfinite(xi0))
    return fail(ctx, OFU_EINVAL, "descend: eps and xi0 must be finite and > 0");
  if (halve_every < 1) return fail(ctx, OFU_EINVAL, "descend: halve_every must be >= 1");
  Leaves& L = ctx->L[ctx->cur];
  float* q;
  ST(ensure(ctx, B_Q, size_t(3 * L.cap), &q));
  const View v = view_of(ctx);
  for (int32_t i = 0; i < n; ++i) {
    const int64_t t = int64_t(t0) + i;
    const double xi = xi0 * std::ldexp(1.0, -int(std::min<int64_t>(t / halve_every, 2000)));
    CU(launch_descent_step(v, L.u, L.ubar, q, L.soff, ctx->samp[ctx->cur], ctx->prm.sample_fp16 != 0,
                           float(eps), float(xi), float(ctx->prm.lambda), float(ctx->prm.gamma),
                           dual_sets(ctx), primal_sets(ctx), ctx->stream));
  }
  return OFU_OK;
}

ofu_status ofu_quantisation_error(ofu_ctx* ctx, const float* fine, int64_t n_fine, double* err) {
  ST(check_built(ctx));
  const int64_t nf = int64_t(1) << (3 * ctx->prm.max_depth);
  if (!fine || !err) return fail(ctx, OFU_EINVAL, "quantisation_error: fine and err must be non-NULL");
  if (n_fine != nf)
    return fail(ctx, OFU_EINVAL, "quantisation_error: fine must hold 8^max_depth values");
  float* f;
  double *cfine, *terms, *tmp;
  ST(ensure(ctx, B_QF, size_t(nf), &f));
  ST(ensure(ctx, B_QD, size_t(nf + 1), &cfine));
  ST(ensure(ctx, B_QT, size_t(ctx->n + 1), &terms));
  ST(ensure(ctx, B_SCAN, scan_tmp_items<double>(std::max(nf, ctx->n)), &tmp));
  CU(cudaMemcpyAsync(f, fine, size_t(nf) * sizeof(float), cudaMemcpyDefault, ctx->stream));
  CU(launch_quant_error(view_of(ctx), ctx->L[ctx->cur].u, f, cfine, terms, tmp, ctx->stream));
  ST(read_back(ctx, terms + ctx->n, sizeof(double), err));
  return OFU_OK;
}

ofu_status ofu_export_frame_tree(ofu_ctx* ctx, int32_t frame, uint64_t* keys, uint8_t* levels,
                                 int64_t cap, int64_t* n) {
  ST(check_ready(ctx));
  if (ctx->prm.data_term != 1 || ctx->ft_host_start.empty())
    return fail(ctx, OFU_ESTATE, "export_frame_tree: no per-frame trees (data_term 1 and frames needed)");
  if (frame < 0 || frame >= ctx->F) return fail(ctx, OFU_EINVAL, "export_frame_tree: frame out of range");
  const int64_t o = ctx->ft_host_start[frame], m = ctx->ft_host_start[frame + 1] - o;
  if (n) *n = m;
  if (!keys && !levels) return OFU_OK;
  if (cap < m) return fail(ctx, OFU_ECAPACITY, "export_frame_tree: capacity smaller than the tree");
  if (keys) CU(cudaMemcpyAsync(keys, ctx->ft_key + o, size_t(m) * 8, cudaMemcpyDefault, ctx->stream));
  if (levels) CU(cudaMemcpyAsync(levels, ctx->ft_level + o, size_t(m), cudaMemcpyDefault, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return OFU_OK;
}

ofu_status ofu_data_term_memory(ofu_ctx* ctx, int64_t* nodes, int64_t* dense_bytes,
                                int64_t* octree_bytes, int64_t* device_bytes) {
  ST(check_ready(ctx));
  if (ctx->prm.data_term != 1 || ctx->ft_host_start.empty())
    return fail(ctx, OFU_ESTATE, "data_term_memory: no per-frame trees (data_term 1 and frames needed)");
  // a tree with m leaves has (m - 1) / 7 inner nodes (every split adds 8 children)
  int64_t all = 0;
  for (int i = 0; i < ctx->F; ++i) {
    const int64_t m = ctx->ft_host_start[i + 1] - ctx->ft_host_start[i];
    const int64_t k = m + (m - 1) / 7;
    if (nodes) nodes[i] = k;
    all += k;
  }
  const int64_t total = ctx->ft_host_start[ctx->F];
  if (dense_bytes) *dense_bytes = int64_t(ctx->F) * (int64_t(1) << (3 * ctx->prm.max_depth)) * 8;
  if (octree_bytes) *octree_bytes = all * (9 * 8 + 3 * 4);
  if (device_bytes) *device_bytes = total * (8 + 1 + 8 + 8) + (total + 1) * 16 + (int64_t(ctx->F) + 1) * 8;
  return OFU_OK;
}

ofu_status ofu_extract_mesh(ofu_ctx* ctx, float* verts, int64_t vcap, int32_t* tris, int64_t tcap,
                            int64_t* n_verts, int64_t* n_tris) {
  ST(check_built(ctx));
  const int D = ctx->prm.max_depth;
  const int64_t nvox = int64_t(1) << (3 * D);
  float* grid;
  uint8_t* cm;
  uint64_t *cnt, *tmp;
  ST(ensure(ctx, B_MG, size_t(nvox), &grid));
  ST(ensure(ctx, B_MC, size_t(nvox), &cm));
  ST(ensure(ctx, B_MN, size_t(nvox + 1), &cnt));
  ST(ensure(ctx, B_SCAN, scan_tmp_items<uint64_t>(nvox) * 2, &tmp));
  Leaves& L = ctx->L[ctx->cur];
  CU(launch_mesh_count(view_of(ctx), L.u, grid, cm, cnt, ctx->stream));
  CU(scan_exclusive<uint64_t>(cnt, cnt, nvox, tmp, ctx->stream));
  uint64_t tot = 0;
  ST(read_back(ctx, cnt + nvox, sizeof(uint64_t), &tot));
  const int64_t V = int64_t(tot & 0xffffffffu), T = int64_t(tot >> 32);
  if (n_verts) *n_verts = V;
  if (n_tris) *n_tris = T;
  if (!verts && !tris) return OFU_OK;
  if ((verts && vcap < V) || (tris && tcap < T))
    return fail(ctx, OFU_ECAPACITY, "extract_mesh: capacity smaller than the mesh (" + std::to_string(V) +
                                        " vertices, " + std::to_string(T) + " triangles)");
  if (V >= (int64_t(1) << 31)) return fail(ctx, OFU_ECAPACITY, "extract_mesh: more than 2^31 vertices");
  float* dv;
  int32_t* dt;
  ST(ensure(ctx, B_MV, size_t(3 * V + 3), &dv));
  ST(ensure(ctx, B_MT, size_t(3 * T + 3), &dt));
  const double spacing = ctx->prm.extent / double(int64_t(1) << D);
  CU(launch_mesh_emit(D, grid, cm, cnt, ctx->prm.origin, spacing, dv, dt, ctx->stream));
  if (verts && V) CU(cudaMemcpyAsync(verts, dv, size_t(3 * V) * sizeof(float), cudaMemcpyDefault, ctx->stream));
  if (tris && T) CU(cudaMemcpyAsync(tris, dt, size_t(3 * T) * sizeof(int32_t), cudaMemcpyDefault, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return OFU_OK;
}

ofu_status ofu_energy(ofu_ctx* ctx, double* primal, double* dual, double* gap) {
  ST(check_built(ctx));
  Leaves& L = ctx->L[ctx->cur];
  double *part, *small;
  ST(ensure(ctx, B_PART, energy_tmp_bytes(ctx->n) / sizeof(double) + 4, &part));
  small = part + energy_tmp_bytes(ctx->n) / sizeof(double);
  CU(launch_energy(view_of(ctx), L.u, L.p, L.soff, ctx->samp[ctx->cur], ctx->prm.sample_fp16 != 0,
                   ctx->prm.lambda, ctx->prm.gamma, primal_sets(ctx), part, small, ctx->stream));
  double h[3];
  ST(read_back(ctx, small, 3 * sizeof(double), h));
  if (primal) *primal = h[0];
  if (dual) *dual = h[1];
  if (gap) *gap = h[2];
  return OFU_OK;
}

ofu_status ofu_num_leaves(ofu_ctx* ctx, int64_t* n) {
  ST(check_ready(ctx));
  if (!n) return fail(ctx, OFU_EINVAL, "num_leaves: n is NULL");
  *n = ctx->n;
  return OFU_OK;
}

ofu_status ofu_export_leaves(ofu_ctx* ctx, uint64_t* keys, uint8_t* levels, float* u, int64_t cap,
                             int64_t* n) {
  ST(check_ready(ctx));
  if (n) *n = ctx->n;
  if ((keys || levels || u) && cap < ctx->n)
    return fail(ctx, OFU_ECAPACITY, "export_leaves: capacity smaller than the leaf count");
  Leaves& L = ctx->L[ctx->cur];
  const size_t m = size_t(ctx->n);
  if (m) {
    if (keys) CU(cudaMemcpyAsync(keys, L.key, m * sizeof(uint64_t), cudaMemcpyDefault, ctx->stream));
    if (levels) CU(cudaMemcpyAsync(levels, L.level, m, cudaMemcpyDefault, ctx->stream));
    if (u) CU(cudaMemcpyAsync(u, L.u, m * sizeof(float), cudaMemcpyDefault, ctx->stream));
  }
  CU(cudaStreamSynchronize(ctx->stream));
  return OFU_OK;
}

ofu_status ofu_solve(ofu_ctx* ctx, int32_t iters, int32_t restructure_every, int32_t check_every,
                     double gap_tol, int32_t* iters_done, int64_t* leaf_iters, double* energies3) {
  ST(check_built(ctx));
  if (iters < 0 || restructure_every < 0 || check_every < 0)
    return fail(ctx, OFU_EINVAL, "solve: counts must be >= 0");
  int32_t done = 0;
  int64_t li = 0;
  double e[3] = {0.0, 0.0, 0.0};
  bool have_e = false;
  while (done < iters) {
    int32_t step = iters - done;
    if (restructure_every > 0) step = std::min(step, restructure_every);
    if (check_every > 0) step = std::min(step, check_every - (done % check_every));
    ST(ofu_iterate(ctx, step));
    li += int64_t(step) * ctx->n;
    done += step;
    have_e = false;
    if (check_every > 0 && done % check_every == 0) {
      ST(ofu_energy(ctx, &e[0], &e[1], &e[2]));
      have_e = true;
      if (gap_tol > 0 && e[2] / std::max(std::fabs(e[0]), 1.0) < gap_tol) break;
    }
    if (restructure_every > 0 && done % restructure_every == 0 && done < iters) {
      ST(ofu_restructure(ctx, nullptr, nullptr, nullptr));
      have_e = false;
    }
  }
  if (energies3) {
    if (!have_e) ST(ofu_energy(ctx, &e[0], &e[1], &e[2]));
    for (int k = 0; k < 3; ++k) energies3[k] = e[k];
  } else {
    CU(cudaStreamSynchronize(ctx->stream));
  }
  if (iters_done) *iters_done = done;
  if (leaf_iters) *leaf_iters = li;
  return OFU_OK;
}

ofu_status ofu_export_field(ofu_ctx* ctx, int32_t field, void* dst, int64_t cap_items,
                            int64_t* n_items) {
  ST(check_ready(ctx));
  const int64_t n = ctx->n;
  Leaves& L = ctx->L[ctx->cur];
  int64_t items;
  switch (field) {
    case OFU_FIELD_U: case OFU_FIELD_UBAR: case OFU_FIELD_TAU: case OFU_FIELD_SIGMA: case OFU_FIELD_W:
      items = n; break;
    case OFU_FIELD_P: items = 3 * n; break;
    case OFU_FIELD_SAMPLE_OFF: items = n + 1; break;
    case OFU_FIELD_SAMPLES: items = ctx->n_samples; break;
    default: return fail(ctx, OFU_EINVAL, "export_field: unknown field");
  }
  if (n_items) *n_items = items;
  if (!dst) return OFU_OK;
  if (cap_items < items) return fail(ctx, OFU_ECAPACITY, "export_field: capacity too small");
  if (n == 0) return OFU_OK;
  cudaStream_t s = ctx->stream;
  switch (field) {
    case OFU_FIELD_U: CU(cudaMemcpyAsync(dst, L.u, n * 4, cudaMemcpyDefault, s)); break;
    case OFU_FIELD_UBAR: CU(cudaMemcpyAsync(dst, L.ubar, n * 4, cudaMemcpyDefault, s)); break;
    case OFU_FIELD_TAU: CU(cudaMemcpyAsync(dst, L.tau, n * 4, cudaMemcpyDefault, s)); break;
    case OFU_FIELD_SIGMA: CU(cudaMemcpyAsync(dst, L.sigma, n * 4, cudaMemcpyDefault, s)); break;
    case OFU_FIELD_P:
      for (int d = 0; d < 3; ++d)
        CU(cudaMemcpyAsync(reinterpret_cast<float*>(dst) + d * n, L.p + d * L.cap, n * 4, cudaMemcpyDefault, s));
      break;
    case OFU_FIELD_SAMPLE_OFF: CU(cudaMemcpyAsync(dst, L.soff, (n + 1) * 4, cudaMemcpyDefault, s)); break;
    case OFU_FIELD_W: {
      int32_t* w;
      ST(ensure(ctx, B_CNT, size_t(n), &w));
      CU(launch_w_from_soff(L.soff, n, w, s));
      CU(cudaMemcpyAsync(dst, w, n * 4, cudaMemcpyDefault, s));
      break;
    }
    case OFU_FIELD_SAMPLES: {
      float* w;
      ST(ensure(ctx, B_CNT, size_t(items), &w));
      CU(launch_widen_samples(ctx->samp[ctx->cur], ctx->prm.sample_fp16 != 0, items, w, s));
      CU(cudaMemcpyAsync(dst, w, items * 4, cudaMemcpyDefault, s));
      break;
    }
  }
  CU(cudaStreamSynchronize(s));
  return OFU_OK;
}

ofu_status ofu_export_neighbours(ofu_ctx* ctx, int32_t face, int64_t* off, int64_t* idx, int64_t cap,
                                 int64_t* nnz) {
  ST(check_built(ctx));
  if (face < 0 || face > 5) return fail(ctx, OFU_EINVAL, "export_neighbours: face must be 0..5");
  const int64_t n = ctx->n;
  Leaves& L = ctx->L[ctx->cur];
  std::vector<int32_t> e(n);
  CU(cudaMemcpyAsync(e.data(), L.nbr + int64_t(face) * L.cap, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<int32_t> ov(L.ovf_cap > 0 ? size_t(L.ovf_cap) : 0);
  if (!ov.empty()) CU(cudaMemcpyAsync(ov.data(), L.ovf, ov.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  std::vector<int64_t> ho(n + 1), hx;
  ho[0] = 0;
  for (int64_t l = 0; l < n; ++l) {
    const int32_t x = e[l];
    if (x == kEmpty) {
    } else if (x >= 0) {
      hx.push_back(entry_idx(x));
    } else {
      const uint32_t st = list_start(x);
      for (int32_t k = 0; k < ov[st]; ++k) hx.push_back(entry_idx(ov[st + 1 + k]));
    }
    ho[l + 1] = int64_t(hx.size());
  }
  if (nnz) *nnz = int64_t(hx.size());
  if (idx && cap < int64_t(hx.size())) return fail(ctx, OFU_ECAPACITY, "export_neighbours: capacity too small");
  if (off) CU(cudaMemcpy(off, ho.data(), ho.size() * 8, cudaMemcpyDefault));
  if (idx && !hx.empty()) CU(cudaMemcpy(idx, hx.data(), hx.size() * 8, cudaMemcpyDefault));
  return OFU_OK;
}

ofu_status ofu_import_leaves(ofu_ctx* ctx, const uint64_t* keys, const uint8_t* levels, int64_t n,
                             const float* u, const float* p) {
  ST(check_ready(ctx));
  if (!ctx->have_frames) return fail(ctx, OFU_ESTATE, "import_leaves: call ofu_integrate_frames first");
  if (n < 1 || !keys || !levels) return fail(ctx, OFU_EINVAL, "import_leaves: need n >= 1 leaves");
  if (n > max_leaves(ctx)) return fail(ctx, OFU_ECAPACITY, "import_leaves: more than max_leaves");
  if (!samples_fit(n, ctx->F)) return fail(ctx, OFU_ECAPACITY, "sample count may exceed 2^32");
  // stage into the spare buffer, check, then make it current
  const int nx = 1 - ctx->cur;
  ST(ensure_leaves(ctx, nx, n));
  Leaves& L = ctx->L[nx];
  CU(cudaMemcpyAsync(L.key, keys, n * 8, cudaMemcpyDefault, ctx->stream));
  CU(cudaMemcpyAsync(L.level, levels, n, cudaMemcpyDefault, ctx->stream));
  uint32_t* bad;
  ST(ensure(ctx, B_CNT, 1, &bad));
  CU(cudaMemsetAsync(bad, 0, 4, ctx->stream));
  CU(launch_check_tiling(L.key, L.level, n, ctx->prm.max_depth, bad, ctx->stream));
  uint32_t hb = 0;
  ST(read_back(ctx, bad, 4, &hb));
  if (hb) return fail(ctx, OFU_EINVAL, "import_leaves: leaves do not tile the domain in key order");
  ctx->cur = nx;
  ctx->n = n;
  ST(integrate_all(ctx, true));
  if (u) {
    CU(cudaMemcpyAsync(L.u, u, n * 4, cudaMemcpyDefault, ctx->stream));
    CU(cudaMemcpyAsync(L.ubar, u, n * 4, cudaMemcpyDefault, ctx->stream));
  }
  if (p) {
    for (int d = 0; d < 3; ++d)
      CU(cudaMemcpyAsync(L.p + d * L.cap, p + d * n, n * 4, cudaMemcpyDefault, ctx->stream));
  }
  ST(rebuild_topology(ctx));
  CU(cudaStreamSynchronize(ctx->stream));
  return OFU_OK;
}

ofu_status ofu_set_state(ofu_ctx* ctx, const float* u, const float* ubar, const float* p, int64_t n) {
  ST(check_built(ctx));
  if (n != ctx->n || !u || !p) return fail(ctx, OFU_EINVAL, "set_state: n must equal the leaf count; u and p required");
  Leaves& L = ctx->L[ctx->cur];
  CU(cudaMemcpyAsync(L.u, u, n * 4, cudaMemcpyDefault, ctx->stream));
  CU(cudaMemcpyAsync(L.ubar, ubar ? ubar : u, n * 4, cudaMemcpyDefault, ctx->stream));
  for (int d = 0; d < 3; ++d)
    CU(cudaMemcpyAsync(L.p + d * L.cap, p + d * n, n * 4, cudaMemcpyDefault, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return OFU_OK;
}

ofu_status ofu_energy_static(ofu_ctx* ctx, double* out3) {
  ST(check_built(ctx));
  if (!out3) return fail(ctx, OFU_EINVAL, "energy_static: out3 is NULL");
  if (ctx->n > energy_static_max_leaves())
    return fail(ctx, OFU_ECAPACITY, "energy_static: " + std::to_string(ctx->n) +
                                        " leaves exceed its fixed scratch limit of " +
                                        std::to_string(energy_static_max_leaves()) + " leaves");
  int dev = -1;
  CU(cudaGetDevice(&dev));
  if (dev != ctx->device)
    return fail(ctx, OFU_EINVAL, "energy_static: the context's device (" + std::to_string(ctx->device) +
                                     ") must be the current device (" + std::to_string(dev) + ")");
  double* scratch = nullptr;
  CU(energy_static_scratch(&scratch));
  Leaves& L = ctx->L[ctx->cur];
  CU(launch_energy_static(view_of(ctx), L.u, L.p, L.soff, ctx->samp[ctx->cur],
                          ctx->prm.sample_fp16 != 0, ctx->prm.lambda, ctx->prm.gamma,
                          primal_sets(ctx), scratch, ctx->stream));
  CU(cudaMemcpyAsync(out3, scratch + energy_static_result_offset(), 3 * sizeof(double),
                     cudaMemcpyDefault, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return OFU_OK;
}

// ---- warm-start network ----------------------------------------------------

#define MCU(call)                                                        \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) {                                             \
      net->poisoned = true;                                              \
      net->err = std::string(#call) + ": " + cudaGetErrorString(e_);     \
      cudaGetLastError();                                                \
      return e_ == cudaErrorMemoryAllocation ? OFU_ENOMEM : OFU_ECUDA;   \
    }                                                                    \
  } while (0)

// Gradient magnitude (truncation units per finest voxel) above which the
// warm start sets p to lambda times the field's normal: the true TSDF ramps
// at 1/delta = 1/4 per voxel, prediction noise on flat regions stays far below.
constexpr float kWarmEdge = 0.05f;

static ofu_status mlp_ready(ofu_mlp* net) {
  if (!net) return OFU_EINVAL;
  if (net->poisoned) {
    net->err = "network object poisoned by an earlier CUDA error";
    return OFU_ESTATE;
  }
  return OFU_OK;
}

static ofu_status mlp_partials(ofu_mlp* net, int64_t B) {
  const int64_t nb = mlp_grad_blocks(B);
  if (nb <= net->partial_blocks) return OFU_OK;
  if (net->partial) MCU(cudaFree(net->partial));
  if (net->sums) MCU(cudaFree(net->sums));
  net->partial = nullptr;
  net->sums = nullptr;
  net->partial_blocks = 0;
  MCU(cudaMalloc(&net->partial, size_t(nb) * kMlpParams * sizeof(float)));
  MCU(cudaMalloc(&net->sums, (2 * size_t(nb) + 2) * sizeof(double)));
  net->partial_blocks = nb;
  return OFU_OK;
}

int64_t ofu_mlp_num_params(void) { return kMlpParams; }

ofu_status ofu_mlp_create(void* cuda_stream, ofu_mlp** out) {
  if (!out) return OFU_EINVAL;
  *out = nullptr;
  ofu_mlp* net = new ofu_mlp();
  net->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  const size_t pb = size_t(kMlpParams) * sizeof(float);
  cudaError_t e = cudaMalloc(&net->params, pb);
  if (e == cudaSuccess) e = cudaMalloc(&net->m, pb);
  if (e == cudaSuccess) e = cudaMalloc(&net->v, pb);
  if (e == cudaSuccess) e = cudaMalloc(&net->grad, pb);
  if (e == cudaSuccess) e = cudaMallocHost(&net->pinned, 64);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->params, 0, pb, net->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->m, 0, pb, net->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->v, 0, pb, net->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->stream);
  if (e != cudaSuccess) {
    g_create_error = std::string("ofu_mlp_create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    ofu_mlp_destroy(net);
    return e == cudaErrorMemoryAllocation ? OFU_ENOMEM : OFU_ECUDA;
  }
  *out = net;
  return OFU_OK;
}

void ofu_mlp_destroy(ofu_mlp* net) {
  if (!net) return;
  cudaStreamSynchronize(net->stream);
  cudaFree(net->params);
  cudaFree(net->m);
  cudaFree(net->v);
  cudaFree(net->grad);
  cudaFree(net->partial);
  cudaFree(net->sums);
  if (net->pinned) cudaFreeHost(net->pinned);
  cudaGetLastError();
  delete net;
}

const char* ofu_mlp_last_error(const ofu_mlp* net) { return net ? net->err.c_str() : g_create_error.c_str(); }

ofu_status ofu_mlp_set_params(ofu_mlp* net, const float* params) {
  ST(mlp_ready(net));
  if (!params) {
    net->err = "set_params: params is NULL";
    return OFU_EINVAL;
  }
  const size_t pb = size_t(kMlpParams) * sizeof(float);
  MCU(cudaMemcpyAsync(net->params, params, pb, cudaMemcpyDefault, net->stream));
  MCU(cudaMemsetAsync(net->m, 0, pb, net->stream));
  MCU(cudaMemsetAsync(net->v, 0, pb, net->stream));
  MCU(cudaStreamSynchronize(net->stream));
  net->step = 0;
  return OFU_OK;
}

ofu_status ofu_mlp_get_params(ofu_mlp* net, float* params) {
  ST(mlp_ready(net));
  if (!params) {
    net->err = "get_params: params is NULL";
    return OFU_EINVAL;
  }
  MCU(cudaMemcpyAsync(params, net->params, size_t(kMlpParams) * sizeof(float), cudaMemcpyDefault,
                      net->stream));
  MCU(cudaStreamSynchronize(net->stream));
  return OFU_OK;
}

ofu_status ofu_mlp_forward(ofu_mlp* net, const float* X, int64_t B, float* y) {
  ST(mlp_ready(net));
  if (B < 0 || (B > 0 && (!X || !y))) {
    net->err = "forward: need B >= 0 and device X, y";
    return OFU_EINVAL;
  }
  MCU(launch_mlp_forward(net->params, X, B, y, net->stream));
  return OFU_OK;
}

static ofu_status mlp_grad(ofu_mlp* net, const float* X, const float* t, const float* w,
                           const int32_t* rows, int64_t B) {
  if (B < 1 || !X || !t || !w) {
    net->err = "gradient: need B >= 1 and device X, t, w";
    return OFU_EINVAL;
  }
  ST(mlp_partials(net, B));
  MCU(launch_mlp_grad(net->params, X, t, w, rows, B, net->partial, net->sums, net->grad,
                      net->sums + 2 * net->partial_blocks, net->stream));
  return OFU_OK;
}

ofu_status ofu_mlp_gradient(ofu_mlp* net, const float* X, const float* t, const float* w,
                            const int32_t* rows, int64_t B, float* grad, double* loss) {
  ST(mlp_ready(net));
  ST(mlp_grad(net, X, t, w, rows, B));
  if (grad)
    MCU(cudaMemcpyAsync(grad, net->grad, size_t(kMlpParams) * sizeof(float), cudaMemcpyDefault,
                        net->stream));
  MCU(cudaMemcpyAsync(net->pinned, net->sums + 2 * net->partial_blocks, sizeof(double),
                      cudaMemcpyDeviceToHost, net->stream));
  MCU(cudaStreamSynchronize(net->stream));
  if (loss) *loss = *reinterpret_cast<double*>(net->pinned);
  return OFU_OK;
}

ofu_status ofu_mlp_train_step(ofu_mlp* net, const float* X, const float* t, const float* w,
                              const int32_t* rows, int64_t B, float lr, double* loss) {
  ST(mlp_ready(net));
  if (!(lr > 0.0f)) {
    net->err = "train_step: lr must be > 0";
    return OFU_EINVAL;
  }
  ST(mlp_grad(net, X, t, w, rows, B));
  net->step += 1;
  MCU(launch_adam(net->params, net->m, net->v, net->grad, lr, net->step, net->stream));
  if (loss) {
    MCU(cudaMemcpyAsync(net->pinned, net->sums + 2 * net->partial_blocks, sizeof(double),
                        cudaMemcpyDeviceToHost, net->stream));
    MCU(cudaStreamSynchronize(net->stream));
    *loss = *reinterpret_cast<double*>(net->pinned);
  }
  return OFU_OK;
}

ofu_status ofu_features(ofu_ctx* ctx, float* X, int64_t cap_rows) {
  ST(check_built(ctx));
  if (!X || cap_rows < ctx->n)
    return fail(ctx, OFU_ECAPACITY, "features: X must hold N x 39 floats on the device");
  Leaves& L = ctx->L[ctx->cur];
  CU(launch_features(view_of(ctx), L.u, L.soff, ctx->samp[ctx->cur], ctx->prm.sample_fp16 != 0, X,
                     ctx->stream));
  return OFU_OK;
}

ofu_status ofu_warm_start(ofu_ctx* ctx, const ofu_mlp* net) {
  ST(check_built(ctx));
  if (!net) return fail(ctx, OFU_EINVAL, "warm_start: network is NULL");
  CU(cudaStreamSynchronize(net->stream));   // the network's last update is complete
  Leaves& L = ctx->L[ctx->cur];
  CU(launch_warm_start(view_of(ctx), L.u, L.soff, ctx->samp[ctx->cur], ctx->prm.sample_fp16 != 0,
                       net->params, L.ubar, ctx->stream));
  CU(cudaMemcpyAsync(L.u, L.ubar, size_t(ctx->n) * sizeof(float), cudaMemcpyDeviceToDevice,
                     ctx->stream));
  // dual start consistent with the new field: lambda n on its edges
  CU(launch_dual_init(view_of(ctx), L.u, L.p, float(ctx->prm.lambda), kWarmEdge, dual_sets(ctx),
                      nbr_recs(ctx, true), ctx->stream));
  return OFU_OK;
}

// ---- checkpoint -------------------------------------------------------------

namespace {
const char kCkptMagic[8] = {'O', 'F', 'U', 'C', 'K', 'P', 'T', '1'};

bool put(FILE* f, const void* p, size_t n) { return n == 0 || std::fwrite(p, 1, n, f) == n; }
bool get(FILE* f, void* p, size_t n) { return n == 0 || std::fread(p, 1, n, f) == n; }
}  // namespace

ofu_status ofu_save(ofu_ctx* ctx, const char* path) {
  ST(check_built(ctx));
  if (!path) return fail(ctx, OFU_EINVAL, "save: path is NULL");
  const int64_t n = ctx->n;
  const size_t fr = size_t(ctx->F) * ctx->H * ctx->W;
  Leaves& L = ctx->L[ctx->cur];
  std::vector<float> rmap(fr), u(n), ub(n), p(3 * size_t(n));
  std::vector<Cam> cams(ctx->F);
  std::vector<uint64_t> keys(n);
  std::vector<uint8_t> lv(n);
  cudaStream_t s = ctx->stream;
  CU(cudaMemcpyAsync(rmap.data(), ctx->depth, fr * 4, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(cams.data(), ctx->cams, cams.size() * sizeof(Cam), cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(keys.data(), L.key, n * 8, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(lv.data(), L.level, n, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(u.data(), L.u, n * 4, cudaMemcpyDeviceToHost, s));
  CU(cudaMemcpyAsync(ub.data(), L.ubar, n * 4, cudaMemcpyDeviceToHost, s));
  for (int d = 0; d < 3; ++d)
    CU(cudaMemcpyAsync(p.data() + d * n, L.p + d * L.cap, n * 4, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(ctx, OFU_EINVAL, std::string("save: cannot open ") + path);
  const int32_t dims[3] = {ctx->F, ctx->H, ctx->W};
  bool ok = put(f, kCkptMagic, 8) && put(f, &ctx->prm, sizeof(ofu_params)) && put(f, dims, 12) &&
            put(f, cams.data(), cams.size() * sizeof(Cam)) && put(f, rmap.data(), fr * 4) &&
            put(f, &n, 8) && put(f, keys.data(), n * 8) && put(f, lv.data(), n) &&
            put(f, u.data(), n * 4) && put(f, ub.data(), n * 4) && put(f, p.data(), 3 * n * 4);
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(ctx, OFU_EINVAL, std::string("save: write failed for ") + path);
  return OFU_OK;
}

ofu_status ofu_load(ofu_ctx* ctx, const char* path) {
  ST(check_ready(ctx));
  if (!path) return fail(ctx, OFU_EINVAL, "load: path is NULL");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(ctx, OFU_EINVAL, std::string("load: cannot open ") + path);
  char magic[8];
  ofu_params prm;
  int32_t dims[3];
  int64_t n = 0;
  bool ok = get(f, magic, 8) && std::memcmp(magic, kCkptMagic, 8) == 0 &&
            get(f, &prm, sizeof(prm)) && get(f, dims, 12);
  std::string why;
  ok = ok && validate(&prm, &why) == OFU_OK && dims[0] >= 1 && dims[0] <= 512 && dims[1] >= 1 &&
       dims[2] >= 1;
  std::vector<Cam> cams;
  std::vector<float> rmap, u, ub, p;
  std::vector<uint64_t> keys;
  std::vector<uint8_t> lv;
  if (ok) {
    cams.resize(dims[0]);
    rmap.resize(size_t(dims[0]) * dims[1] * dims[2]);
    ok = get(f, cams.data(), cams.size() * sizeof(Cam)) && get(f, rmap.data(), rmap.size() * 4) &&
         get(f, &n, 8) && n >= 1 && n <= kMaxLeaves;
  }
  if (ok) {
    keys.resize(n);
    lv.resize(n);
    u.resize(n);
    ub.resize(n);
    p.resize(3 * size_t(n));
    ok = get(f, keys.data(), n * 8) && get(f, lv.data(), n) && get(f, u.data(), n * 4) &&
         get(f, ub.data(), n * 4) && get(f, p.data(), 3 * n * 4);
  }
  std::fclose(f);
  if (!ok) return fail(ctx, OFU_EINVAL, std::string("load: not a valid checkpoint: ") + path);
  // frames (range maps) and parameters, then the structure and the iterate
  ctx->prm = prm;
  const size_t fr = rmap.size();
  if (ctx->depth) CU(dfree(ctx, ctx->depth));
  if (ctx->cams) CU(dfree(ctx, ctx->cams));
  if (ctx->map) CU(dfree(ctx, ctx->map));
  ctx->depth = nullptr;
  ctx->cams = nullptr;
  ctx->map = nullptr;
  CU(dalloc(ctx, &ctx->depth, fr * 4));
  CU(dalloc(ctx, &ctx->cams, cams.size() * sizeof(Cam)));
  CU(cudaMemcpy(ctx->depth, rmap.data(), fr * 4, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(ctx->cams, cams.data(), cams.size() * sizeof(Cam), cudaMemcpyHostToDevice));
  ctx->F = dims[0];
  ctx->H = dims[1];
  ctx->W = dims[2];
  ctx->have_frames = true;
  ctx->n = 0;
  free_frame_trees(ctx);
  if (ctx->prm.data_term == 1) ST(build_frame_trees(ctx));
  ST(ofu_import_leaves(ctx, keys.data(), lv.data(), n, u.data(), p.data()));
  Leaves& L = ctx->L[ctx->cur];
  CU(cudaMemcpyAsync(L.ubar, ub.data(), n * 4, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return OFU_OK;
}

int64_t ofu_kernel_launches(void) { return launches_so_far(); }

ofu_status ofu_profile(ofu_ctx* ctx, int32_t enable) {
  ST(check_ready(ctx));
  // the event pool is created here, outside any timed work, and only grows
  if (enable < 0 || enable > kProfMaxIters)
    return fail(ctx, OFU_EINVAL, "profile: enable must be 0, 1 or an iteration count <= 2^20");
  const size_t want = std::max(kProfEvents, 3 * size_t(enable));
  while (enable && ctx->prof_ev.size() < want) {
    cudaEvent_t e;
    CU(cudaEventCreate(&e));
    ctx->prof_ev.push_back(e);
  }
  ctx->prof_on = enable != 0;
  if (enable) {
    ctx->prof_used = 0;
    ctx->prof_bytes[0] = ctx->prof_bytes[1] = 0.0;
    ctx->prof_launches[0] = ctx->prof_launches[1] = 0;
  }
  return OFU_OK;
}

ofu_status ofu_profile_read(ofu_ctx* ctx, double* ms, int64_t* launches, double* bytes) {
  ST(check_ready(ctx));
  CU(cudaStreamSynchronize(ctx->stream));
  double t[2] = {0.0, 0.0};
  for (size_t i = 0; i + 3 <= ctx->prof_used; i += 3) {
    float a = 0.0f, b = 0.0f;
    CU(cudaEventElapsedTime(&a, ctx->prof_ev[i], ctx->prof_ev[i + 1]));
    CU(cudaEventElapsedTime(&b, ctx->prof_ev[i + 1], ctx->prof_ev[i + 2]));
    t[0] += a;
    t[1] += b;
  }
  for (int k = 0; k < 2; ++k) {
    if (ms) ms[k] = t[k];
    if (launches) launches[k] = ctx->prof_launches[k];
    if (bytes) bytes[k] = ctx->prof_bytes[k];
  }
  return OFU_OK;
}

}  // extern "C"
