// batch.cu -- many independent contexts advanced in lock step (host
// driver; kernels in batch_a.cu, batch_b.cu, batch_c.cu).
//
// Every pass of every Dormand-Prince stage runs over a work list of
// (member, tile) items of all active members: pass A (stage assembly +
// forward x FFT) over their y tiles, pass B over their kx planes, pass C
// (inverse x FFT + field + torque + error) over their tiles.  One block per
// item.  A pass is one launch per (z-extent group for pass B, whose z
// transform is specialised per nz; block-size class: each member's own block
// size rounded up to 128, 256 or 512), and these launches run concurrently
// on side streams, so small items run in small blocks several to an SM.
// Each list is sorted by decreasing work, so uneven members share the GPU
// without a tail per member.  Stream order makes pass B wait for pass A and
// pass C for pass B.
// A fixed-step lock step (6 stages and the accept) is one CUDA graph,
// replayed.
//
// Each member runs exactly the arithmetic of its own context path (the same
// device bodies, FFT plans and FP32 stage coefficients formed from the same
// FP64 step), so a member's trajectory is bitwise the same alone and in any
// batch.  The batched pass B is one CTA per kx plane (R = 1) reading the
// kernel rows from L2; members must use that shape (mmp_set_shape, or
// mmp_autotune with MMP_TUNE_BATCH).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <tuple>
#include <vector>

#include "batch.h"
#include "ctx.h"
#include "dp45.h"
#include "kernels.h"
#include "pass_a.cuh"
#include "plan.h"

using namespace mmp;

namespace {

int berr(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return report_error(code, buf);
}

struct Member {
  mmp_ctx* ctx;
  int goal;            // MMP_GOAL_*
  double a, c;         // goal arguments
  double until;        // RUN / RELAX: end time
  long long left;      // STEPS: accepted steps still to do
  int done = 0;
  int status = MMP_OK;
  int par = 0;         // ping-pong parity inside an advance call
};

// Dynamic shared memory of a member's items in each pass.
size_t smem_a(const Grid& g) { return passa_inv_offset(g.Px, g.ty, g.xb) + (size_t)g.ty * g.nx * sizeof(float); }
size_t smem_b(const Grid& g) { return passb_smem(g.ny, g.nz, g.Py, g.kzn, 1, false).total; }
size_t smem_c(const Grid& g) { return smem_field(g, true); }

// z-extent group of pass B (the specialised z transforms).
int nz_group(int nz) { return (nz == 1 || nz == 2 || nz == 4 || nz == 8) ? nz : 0; }

double item_cost(const Grid& g, int pass) {
  auto lg = [](double v) { return v > 1 ? log2(v) : 1.0; };
  if (pass == 1) return 3.0 * g.nz * g.Py * lg(g.Py) + 60.0 * g.Py * g.nz;
  if (pass == 2) return (double)g.tyc * g.Px * lg(g.Px) + 40.0 * g.tyc * g.nx;
  return (double)g.ty * g.Px * lg(g.Px);
}

// Block size class of an item: the member's own block size for the pass
// (launch_threads), rounded up to 128, 256 or 512 threads, so small items
// run in small blocks and several share an SM.
int thread_class(int t) { return t <= 128 ? 128 : (t <= 256 ? 256 : 512); }

// One launch of a stage: pass kind (0 = A, 1 = B, 2 = C), z group of pass B,
// block size, and its slice of the item array.
struct Launch {
  int kind, group, threads;
  int off, cnt;
  size_t smem;
  int warp = -1;   // >= 0: the warp-engine launch of this pass for descriptor `warp`
  Grid g{};        // its grid
  int R = 1;       // its ky classes (pass B)
};

struct ListSet {
  std::vector<int> members;     // member indices; descriptor k is members[k]
  std::vector<Launch> launches; // grouped by kind (A, then B, then C)
  int total = 0;
};

}  // namespace

struct mmp_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;      // created here (the caller gave the legacy default stream)
  std::vector<Member> members;
  // device buffers
  BatchInst* d_inst = nullptr;
  size_t cap_inst = 0;
  BatchItem* d_items = nullptr;
  size_t cap_items = 0;
  unsigned* d_red = nullptr;
  size_t cap_red = 0;
  unsigned* h_red = nullptr;
  size_t cap_hred = 0;
  std::vector<BatchInst> h_inst;
  ListSet list;
  std::vector<cudaStream_t> aux;   // side streams: the launches of one pass run concurrently
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  bool list_valid = false;
  int sms = 0;
  // fixed-step graph of one lock step over the current list
  cudaGraphExec_t graph = nullptr;
  bool graph_valid = false;
  long long per_step = 0;       // kernel launches of one graph replay
  long long launches = 0;
  // tracing: events around every pass launch (lock steps then launch
  // directly instead of through the graph)
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events[3];
  size_t prof_used[3] = {0, 0, 0};
};

namespace {

int cuda_fail(cudaError_t e, const char* what) {
  return berr(MMP_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}
#define BCK(expr, what)                                   \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return cuda_fail(_e, what);    \
  } while (0)
#define BTRY(expr)                                        \
  do {                                                    \
    int _rc = (expr);                                     \
    if (_rc != MMP_OK) return _rc;                        \
  } while (0)

template <typename T>
int grow_buf(T*& p, size_t& cap, size_t need) {
  if (need <= cap && p) return MMP_OK;
  if (p) cudaFree(p);
  p = nullptr;
  size_t n = std::max<size_t>(need, 16);
  if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    cap = 0;
    return berr(MMP_E_OOM, "batch: device allocation of %zu bytes failed", n * sizeof(T));
  }
  cap = n;
  return MMP_OK;
}

// A member that runs the warp passes A, B and C (its shape: engine 3 with
// Py / R = 1024, no staged kernel rows), one launch per pass of its own.
bool warp_member(const mmp_ctx* c) {
  return c->engine == (MMP_ENGINE_WARP_B | MMP_ENGINE_WARP_X) && c->ks == 0 && batch_warp_supported(c->g, c->R);
}

bool eligible(const mmp_ctx* c, const char** why) {
  if (c->nsub != 1) { *why = "batch members have one sublattice"; return false; }
  if (!c->uniform) { *why = "batch members have one region"; return false; }
  if (!(c->terms & MMP_T_DEMAG)) { *why = "batch members have the demag term on"; return false; }
  if (c->terms & (MMP_T_AFM | MMP_T_MEL | MMP_T_ELASTIC)) {
    *why = "batch members have no AFM, magnetoelastic or elastic term";
    return false;
  }
  if (c->method != MMP_DP45) { *why = "batch members use the Dormand-Prince solver"; return false; }
  if (warp_member(c)) return true;
  if (c->R != 1 || c->ks != 0 || c->engine != 0) {
    *why = "batch members use the shape R = 1, stage_kernel = 0, engine = 0, or the warp passes A, B and C "
           "with Py / R = 1024";
    return false;
  }
  const Grid& g = c->g;
  if ((long long)g.xb * (g.ty / 2) * g.Px > (long long)fft_cap_a(c->plan_x) * kBatchThreads ||
      (long long)g.xbc * (g.tyc / 2) * g.Px > (long long)fft_cap(c->plan_x) * kBatchThreads ||
      (long long)3 * g.nz * g.Py > 2LL * fft_cap(c->plan_ly) * kBatchThreads) {
    *why = "member tiles or planes exceed the FFT capacity of one batched block";
    return false;
  }
  const size_t lim = 227 * 1024 - 2048;   // static shared memory of the batched kernels
  if (smem_a(g) > lim || smem_b(g) > lim || smem_c(g) > lim) {
    *why = "member too large for one batched block";
    return false;
  }
  return true;
}

// Descriptor of member m for the next launches (parity, coefficients of
// step h, relax flag).
BatchInst make_inst(const Member& m, unsigned* red, double h, int relax) {
  mmp_ctx* c = m.ctx;
  BatchInst I;
  memset(&I, 0, sizeof I);
  I.g = c->g;
  I.d.T = c->d_T;
  I.d.khat = c->d_khat;
  I.d.tw_x = c->d_tw_x;
  I.d.tw_y = c->d_tw_y;
  I.d.tw_ly = c->d_tw_ly;
  I.d.tw_z = c->d_tw_z;
  I.d.plan_x = c->plan_x;
  I.d.plan_ly = c->plan_ly;
  I.d.R = 1;
  I.d.ks = 0;
  if (warp_member(c)) {   // the warp passes' tables and ky classes
    I.d.R = c->R;
    I.d.tw_wy = c->d_tw_wy;
    I.d.tw_wx = c->d_tw_wx;
    I.d.tw_wx2 = c->d_tw_wx2;
    I.d.err = c->d_flag;
    I.d.engine = 1;
  }
  I.co.reg = c->d_coef;
  I.co.regions = nullptr;
  I.co.hA = nullptr;
  I.co.uniform = 1;
  I.ybuf[0] = c->d_y;
  I.ybuf[1] = c->d_stage;
  I.kbuf[0] = c->d_k[0];
  I.kbuf[1] = c->d_k[6];
  for (int j = 0; j < 5; ++j) I.kmid[j] = c->d_k[j + 1];
  I.red = red;
  I.terms = kernel_terms(c);
  I.relax = relax;
  I.par = m.par;
  for (int i = 1; i <= 6; ++i) stage_coefs(h, i, I.coef[i]);
  error_coefs(h, I.ecoef);
  return I;
}

// Work lists over `mem` (member indices): per pass kind, z group (pass B)
// and block-size class, one launch over its items sorted longest first;
// uploaded to d_items.
int build_list(mmp_batch* b, const std::vector<int>& mem) {
  ListSet L;
  L.members = mem;
  std::map<std::tuple<int, int, int>, std::vector<std::pair<double, BatchItem>>> sec;
  std::map<std::tuple<int, int, int>, size_t> smem;
  std::vector<Launch> warp;   // the warp-engine members' launches
  for (int k = 0; k < (int)mem.size(); ++k) {
    const mmp_ctx* c = b->members[mem[k]].ctx;
    const Grid& g = c->g;
    if (warp_member(c)) {
      for (int kind = 0; kind < 3; ++kind) {
        Launch l{};
        l.kind = kind;
        l.warp = k;
        l.g = g;
        l.R = c->R;
        warp.push_back(l);
      }
      continue;
    }
    const int tiles = (g.ny + g.ty - 1) / g.ty;       // pass A
    const int tiles_c = (g.ny + g.tyc - 1) / g.tyc;   // pass C
    const auto ka = std::make_tuple(0, 0, thread_class(c->thrA));
    const auto kb = std::make_tuple(1, nz_group(g.nz), thread_class(c->thrB));
    const auto kc = std::make_tuple(2, 0, thread_class(c->thrC));
    smem[ka] = std::max(smem[ka], smem_a(g));
    smem[kb] = std::max(smem[kb], smem_b(g));
    smem[kc] = std::max(smem[kc], smem_c(g));
    for (int z = 0; z < g.nz; ++z) {
      for (int t = 0; t < tiles; ++t) sec[ka].push_back({item_cost(g, 0), BatchItem{k, t, z}});
      for (int t = 0; t < tiles_c; ++t) sec[kc].push_back({item_cost(g, 2), BatchItem{k, t, z}});
    }
    for (int kx = 0; kx < g.kxn; ++kx) sec[kb].push_back({item_cost(g, 1), BatchItem{k, kx, 0}});
  }
  std::vector<BatchItem> items;
  for (auto& kv : sec) {   // std::map order: kind, then group, then block size
    auto& v = kv.second;
    std::stable_sort(v.begin(), v.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    Launch l;
    l.kind = std::get<0>(kv.first);
    l.group = std::get<1>(kv.first);
    l.threads = std::get<2>(kv.first);
    l.off = (int)items.size();
    l.cnt = (int)v.size();
    l.smem = smem[kv.first];
    for (auto& e : v) items.push_back(e.second);
    L.launches.push_back(l);
  }
  for (const Launch& l : warp) L.launches.push_back(l);
  if (!warp.empty()) BCK(batch_warp_prepare(), "batch: warp-pass attributes");
  L.total = (int)items.size();
  BTRY(grow_buf(b->d_items, b->cap_items, items.size()));
  BTRY(grow_buf(b->d_inst, b->cap_inst, mem.size()));
  BCK(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice,
                      b->stream),
      "batch: upload work list");
  // side streams and events for the widest pass
  size_t widest = 0;
  for (int kind = 0; kind < 3; ++kind) {
    size_t n = 0;
    for (const Launch& l : L.launches) n += l.kind == kind;
    widest = std::max(widest, n);
  }
  if (!b->fork) BCK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "batch: event");
  while (b->aux.size() + 1 < widest) {
    cudaStream_t st;
    cudaEvent_t ev;
    BCK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "batch: side stream");
    BCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "batch: event");
    b->aux.push_back(st);
    b->join.push_back(ev);
  }
  b->list = L;
  b->list_valid = true;
  b->graph_valid = false;
  return MMP_OK;
}

// Events around the launches of pass kind k (0 = A, 1 = B, 2 = C) when tracing.
struct BTraced {
  mmp_batch* b;
  cudaEvent_t stop = nullptr;
  BTraced(mmp_batch* bb, int k) : b(bb) {
    if (!b->prof) return;
    auto& v = b->prof_events[k];
    if (b->prof_used[k] == v.size()) {
      cudaEvent_t x, y;
      cudaEventCreate(&x);
      cudaEventCreate(&y);
      v.push_back({x, y});
    }
    auto& pr = v[b->prof_used[k]++];
    cudaEventRecord(pr.first, b->stream);
    stop = pr.second;
  }
  ~BTraced() {
    if (stop) cudaEventRecord(stop, b->stream);
  }
};

cudaError_t launch_one(mmp_batch* b, const Launch& l, int stage, cudaStream_t s) {
  if (l.warp >= 0) return launch_batch_warp(l.kind, b->d_inst, l.warp, l.g, l.R, stage, s);
  const BatchItem* it = b->d_items + l.off;
  if (l.kind == 0) return launch_batch_passA(b->d_inst, it, l.cnt, stage, l.threads, l.smem, s);
  if (l.kind == 1) return launch_batch_passB(l.group, b->d_inst, it, l.cnt, l.threads, l.smem, s);
  return launch_batch_field(b->d_inst, it, l.cnt, stage, l.threads, l.smem, s);
}

// Enqueue stage `stage` of the current list: the launches of pass A, then
// of pass B, then of pass C; the launches of one pass run concurrently on
// side streams forked from and joined back into the batch stream.
int launch_stage(mmp_batch* b, int stage) {
  for (int kind = 0; kind < 3; ++kind) {
    std::vector<const Launch*> ls;
    for (const Launch& l : b->list.launches)
      if (l.kind == kind) ls.push_back(&l);
    if (ls.empty()) continue;
    BTraced t(b, kind);
    if (ls.size() > 1) BCK(cudaEventRecord(b->fork, b->stream), "batch: fork");
    for (size_t i = 0; i < ls.size(); ++i) {
      cudaStream_t s = i == 0 ? b->stream : b->aux[i - 1];
      if (i > 0) BCK(cudaStreamWaitEvent(s, b->fork, 0), "batch: fork wait");
      BCK(launch_one(b, *ls[i], stage, s), "batch: pass launch");
      b->launches++;
      if (i > 0) {
        BCK(cudaEventRecord(b->join[i - 1], s), "batch: join");
        BCK(cudaStreamWaitEvent(b->stream, b->join[i - 1], 0), "batch: join wait");
      }
    }
  }
  return MMP_OK;
}

int upload_insts(mmp_batch* b) {
  BCK(cudaMemcpyAsync(b->d_inst, b->h_inst.data(), b->h_inst.size() * sizeof(BatchInst), cudaMemcpyHostToDevice,
                      b->stream),
      "batch: upload descriptors");
  return MMP_OK;
}

// Write the ping-pong parity back into the member contexts (canonical
// buffers outside advance calls).
void settle(mmp_batch* b) {
  for (Member& m : b->members) {
    if (m.par) {
      std::swap(m.ctx->d_y, m.ctx->d_stage);
      std::swap(m.ctx->d_k[0], m.ctx->d_k[6]);
      m.par = 0;
    }
  }
}

bool member_done(const Member& m) {
  if (m.done) return true;
  if (m.goal == MMP_GOAL_STEPS) return m.left <= 0;
  return m.ctx->t >= m.until * (1.0 - 1e-15);
}

// Step of member m in the next attempt (RUN / RELAX land on their end time).
double member_h(const Member& m) {
  double h = m.ctx->dt;
  if (m.goal != MMP_GOAL_STEPS && m.ctx->t + h > m.until) h = m.until - m.ctx->t;
  return h;
}

}  // namespace

extern "C" {

int mmp_batch_create(mmp_batch** out, void* stream) {
  if (!out) return berr(MMP_E_INVAL, "out is null");
  *out = nullptr;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return berr(MMP_E_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  mmp_batch* b = new mmp_batch();
  b->stream = static_cast<cudaStream_t>(stream);
  if (!b->stream) {   // graphs cannot be captured on the legacy default stream
    e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaGetLastError();
      delete b;
      return berr(MMP_E_CUDA, "batch: stream creation failed: %s", cudaGetErrorString(e));
    }
    b->own_stream = true;
  }
  b->sms = sms;
  *out = b;
  return MMP_OK;
}

int mmp_batch_destroy(mmp_batch* b) {
  if (!b) return MMP_OK;
  cudaStreamSynchronize(b->stream);
  settle(b);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  for (cudaStream_t st : b->aux) cudaStreamDestroy(st);
  for (cudaEvent_t ev : b->join) cudaEventDestroy(ev);
  if (b->fork) cudaEventDestroy(b->fork);
  for (auto& v : b->prof_events)
    for (auto& pr : v) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  void* bufs[] = {b->d_inst, b->d_items, b->d_red};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (b->h_red) cudaFreeHost(b->h_red);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return MMP_OK;
}

int mmp_batch_add(mmp_batch* b, mmp_ctx* ctx, int goal, double a, double c) {
  if (!b || !ctx) return berr(MMP_E_INVAL, "null batch or context");
  if (ctx->poisoned) return berr(MMP_E_STATE, "context poisoned by an earlier CUDA error");
  for (const Member& m : b->members)
    if (m.ctx == ctx) return berr(MMP_E_INVAL, "context already in the batch");
  if (goal < MMP_GOAL_STEPS || goal > MMP_GOAL_RELAX) return berr(MMP_E_INVAL, "unknown goal %d", goal);
  if (goal == MMP_GOAL_STEPS && !(a >= 0)) return berr(MMP_E_INVAL, "steps must be >= 0");
  if (goal == MMP_GOAL_RUN && !(a >= 0)) return berr(MMP_E_INVAL, "duration must be >= 0");
  if (goal == MMP_GOAL_RELAX && (!(a > 0) || !(c > 0))) return berr(MMP_E_INVAL, "bad relax settings");
  BTRY(ctx_prepare(ctx));
  const char* why = "";
  if (!eligible(ctx, &why)) return berr(MMP_E_INVAL, "%s", why);
  BCK(cudaStreamSynchronize(ctx->stream), "batch: member stream");
  Member m;
  m.ctx = ctx;
  m.goal = goal;
  m.a = a;
  m.c = c;
  m.left = goal == MMP_GOAL_STEPS ? (long long)a : 0;
  m.until = goal == MMP_GOAL_RUN ? ctx->t + a : (goal == MMP_GOAL_RELAX ? ctx->t + c : 0.0);
  b->members.push_back(m);
  b->list_valid = false;
  return MMP_OK;
}

int mmp_batch_remove(mmp_batch* b, mmp_ctx* ctx) {
  if (!b || !ctx) return berr(MMP_E_INVAL, "null batch or context");
  for (size_t i = 0; i < b->members.size(); ++i)
    if (b->members[i].ctx == ctx) {
      BCK(cudaStreamSynchronize(b->stream), "batch: sync");
      b->members.erase(b->members.begin() + i);
      b->list_valid = false;
      return MMP_OK;
    }
  return berr(MMP_E_INVAL, "context not in the batch");
}

int mmp_batch_size(mmp_batch* b, int* n) {
  if (!b || !n) return berr(MMP_E_INVAL, "null argument");
  *n = (int)b->members.size();
  return MMP_OK;
}

int mmp_batch_status(mmp_batch* b, mmp_ctx* ctx, int* done, int* status) {
  if (!b || !ctx) return berr(MMP_E_INVAL, "null batch or context");
  for (const Member& m : b->members)
    if (m.ctx == ctx) {
      if (done) *done = member_done(m) ? 1 : 0;
      if (status) *status = m.status;
#ifdef MMP_CHECK_BOUNDS
      // the member's index checks report into its context's flag word
      if (status && ctx->d_flag) {
        unsigned f = 0;
        BCK(cudaStreamSynchronize(b->stream), "batch: sync");
        BCK(cudaMemcpy(&f, ctx->d_flag, sizeof f, cudaMemcpyDeviceToHost), "batch: read flag");
        if (f & 2u) *status = MMP_E_BOUNDS;
      }
#endif
      return MMP_OK;
    }
  return berr(MMP_E_INVAL, "context not in the batch");
}

int mmp_batch_profile(mmp_batch* b, int enable) {
  if (!b) return berr(MMP_E_INVAL, "null batch");
  BCK(cudaStreamSynchronize(b->stream), "batch: sync");
  for (size_t& u : b->prof_used) u = 0;
  b->prof = enable != 0;
  return MMP_OK;
}

int mmp_batch_profile_read(mmp_batch* b, int pass, long long* launches, double* total_ms) {
  if (!b) return berr(MMP_E_INVAL, "null batch");
  if (pass < 0 || pass > 2) return berr(MMP_E_INVAL, "pass must be 0 (A), 1 (B) or 2 (C)");
  BCK(cudaStreamSynchronize(b->stream), "batch: sync");
  double tot = 0.0;
  for (size_t i = 0; i < b->prof_used[pass]; ++i) {
    float ms = 0.0f;
    BCK(cudaEventElapsedTime(&ms, b->prof_events[pass][i].first, b->prof_events[pass][i].second), "event time");
    tot += ms;
  }
  if (launches) *launches = (long long)b->prof_used[pass];
  if (total_ms) *total_ms = tot;
  return MMP_OK;
}

int mmp_batch_launches(mmp_batch* b, long long* n) {
  if (!b || !n) return berr(MMP_E_INVAL, "null argument");
  *n = b->launches;
  return MMP_OK;
}

namespace {

// The lock-step loop of mmp_batch_advance (parities stay in the members).
int advance_loop(mmp_batch* b, int max_attempts) {
  const size_t nm = b->members.size();
  BTRY(grow_buf(b->d_red, b->cap_red, 2 * std::max<size_t>(nm, 1)));
  if (b->cap_hred < b->cap_red) {
    if (b->h_red) cudaFreeHost(b->h_red);
    b->h_red = nullptr;
    b->cap_hred = 0;
    if (cudaMallocHost(&b->h_red, b->cap_red * sizeof(unsigned)) != cudaSuccess) {
      cudaGetLastError();
      return berr(MMP_E_OOM, "batch: pinned allocation failed");
    }
    b->cap_hred = b->cap_red;
  }
  int attempts = 0;
  while (attempts < max_attempts) {
    std::vector<int> act;
    for (int i = 0; i < (int)nm; ++i)
      if (!member_done(b->members[i])) act.push_back(i);
    if (act.empty()) break;
    // first stages (k1) that are not cached, in their relax mode
    std::vector<int> need_k1;
    for (int i : act) {
      const Member& m = b->members[i];
      const int relax = m.goal == MMP_GOAL_RELAX;
      if (!(m.ctx->k1_valid && m.ctx->k1_relax == relax)) need_k1.push_back(i);
    }
    if (!need_k1.empty()) {
      BTRY(build_list(b, need_k1));
      b->h_inst.resize(need_k1.size());
      for (size_t k = 0; k < need_k1.size(); ++k) {
        const Member& m = b->members[need_k1[k]];
        b->h_inst[k] = make_inst(m, b->d_red, member_h(m), m.goal == MMP_GOAL_RELAX);
      }
      BTRY(upload_insts(b));
      BTRY(launch_stage(b, 0));
      for (int i : need_k1) {
        Member& m = b->members[i];
        m.ctx->k1_valid = true;
        m.ctx->k1_relax = m.goal == MMP_GOAL_RELAX;
        m.ctx->evals++;
      }
      b->list_valid = false;
    }
    if (!b->list_valid || b->list.members != act) BTRY(build_list(b, act));
    b->h_inst.resize(act.size());
    bool fixed = true;   // every active member takes fixed steps without read-back
    for (size_t k = 0; k < act.size(); ++k) {
      const Member& m = b->members[act[k]];
      b->h_inst[k] = make_inst(m, b->d_red + 2 * k, member_h(m), m.goal == MMP_GOAL_RELAX);
      if (m.ctx->adaptive || m.goal != MMP_GOAL_STEPS) fixed = false;
    }
    BTRY(upload_insts(b));
    if (fixed && b->prof) {
      // traced: one lock step of direct launches
      for (int s = 1; s <= 6; ++s) BTRY(launch_stage(b, s));
      BCK(launch_batch_accept(b->d_inst, (int)act.size(), b->stream), "batch: accept");
      b->launches++;
      for (int i : act) {
        Member& m = b->members[i];
        m.par ^= 1;
        m.left--;
        m.ctx->t += m.ctx->dt;
        m.ctx->steps++;
        m.ctx->evals += 6;
      }
      attempts++;
      continue;
    }
    if (fixed) {
      // whole lock steps from one graph: every member takes K steps
      long long K = max_attempts - attempts;
      for (int i : act) K = std::min(K, b->members[i].left);
      if (!b->graph_valid) {
        if (b->graph) cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        const long long before = b->launches;
        BCK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeRelaxed), "batch: begin capture");
        int rc = MMP_OK;
        for (int s = 1; s <= 6 && rc == MMP_OK; ++s) rc = launch_stage(b, s);
        if (rc == MMP_OK) rc = launch_batch_accept(b->d_inst, (int)act.size(), b->stream) == cudaSuccess
                                   ? MMP_OK
                                   : cuda_fail(cudaGetLastError(), "batch: accept");
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &gr);
        b->per_step = b->launches - before + 1;
        b->launches = before;
        BTRY(rc);
        BCK(e, "batch: end capture");
        e = cudaGraphInstantiate(&b->graph, gr, 0);
        cudaGraphDestroy(gr);
        BCK(e, "batch: instantiate");
        b->graph_valid = true;
      }
      for (long long s = 0; s < K; ++s) {
        BCK(cudaGraphLaunch(b->graph, b->stream), "batch: graph launch");
        b->launches += b->per_step;
      }
      for (int i : act) {
        Member& m = b->members[i];
        m.par ^= (int)(K & 1);
        m.left -= K;
        for (long long s = 0; s < K; ++s) m.ctx->t += m.ctx->dt;   // as K single steps add it
        m.ctx->steps += K;
        m.ctx->evals += 6 * K;
      }
      attempts += (int)K;
      continue;
    }
    // one lock step with the errors read back
    BCK(cudaMemsetAsync(b->d_red, 0, 2 * act.size() * sizeof(unsigned), b->stream), "batch: reset errors");
    for (int s = 1; s <= 6; ++s) BTRY(launch_stage(b, s));
    BCK(cudaMemcpyAsync(b->h_red, b->d_red, 2 * act.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream),
        "batch: read errors");
    BCK(cudaStreamSynchronize(b->stream), "batch: sync");
    for (size_t k = 0; k < act.size(); ++k) {
      Member& m = b->members[act[k]];
      mmp_ctx* c = m.ctx;
      const int relax = m.goal == MMP_GOAL_RELAX;
      const double h = member_h(m);
      c->evals += 6;
      if (!(c->adaptive || relax)) {   // fixed step: always accepted
        m.par ^= 1;
        c->t += h;
        c->steps++;
        m.left--;
        continue;
      }
      float e, tm;
      memcpy(&e, &b->h_red[2 * k], 4);
      memcpy(&tm, &b->h_red[2 * k + 1], 4);
      const double err = e;
      if (!std::isfinite(err)) {   // state and k1 untouched (the ping-pong is not flipped)
        m.done = 1;
        m.status = MMP_E_NONFINITE;
        continue;
      }
      const bool ok = err <= c->tol || h <= c->dt_min;
      const double fac = grow(err, c->tol);
      if (ok) {
        m.par ^= 1;
        c->t += h;
        c->steps++;
        m.left--;
      } else {
        c->rejected++;
      }
      c->dt = std::min(std::max(h * fac, c->dt_min), c->dt_max);
      if (relax && ok && tm <= m.a) m.done = 1;
    }
    attempts++;
  }
  return MMP_OK;
}

}  // namespace

int mmp_batch_advance(mmp_batch* b, int max_attempts, int* n_active) {
  if (!b) return berr(MMP_E_INVAL, "null batch");
  if (max_attempts < 0) return berr(MMP_E_INVAL, "max_attempts < 0");
  int rc = advance_loop(b, max_attempts);
  cudaError_t se = cudaStreamSynchronize(b->stream);
  settle(b);
  b->list_valid = false;   // parities were written back: descriptors are rebuilt next time
  if (se != cudaSuccess && rc == MMP_OK) rc = cuda_fail(se, "batch: sync");
  for (Member& m : b->members)
    if (m.goal == MMP_GOAL_RELAX && member_done(m)) m.ctx->k1_valid = false;   // k1 holds the damping-only torque
  if (n_active) {
    int n = 0;
    for (const Member& m : b->members) n += !member_done(m);
    *n_active = n;
  }
  return rc;
}

}  // extern "C"
