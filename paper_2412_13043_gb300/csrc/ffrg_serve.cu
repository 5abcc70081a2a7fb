// Serving: continuous batching of RG-flow requests on one GPU.
//
// A scheduler thread owns up to max_slots device-resident flows ("slots").
// Each slot holds its request's dressing tables, its DP5(4) state and its own
// RHS scratch.  Every tick advances all resident flows by one adaptive step
// with batched launches (one precompute, one persistent integrand launch per
// model over the combined work list, one finalize and one derivative kernel
// per stage, one control kernel with a CTA per flow).  Flows retire when
// their control block says done; queued requests are admitted as soon as a
// slot and enough of the HBM budget are free, so new flows join while others
// are mid-flight.  Ticks are pipelined two deep: the next tick is queued
// before the host reads the previous tick's control blocks, retires, admits
// and rebuilds.  Each flow's reductions and step control depend only on its
// own data, so its result does not depend on what it is batched with.
//
// Requests: frozen-background flows (d_t y = -Flow, Sec. 5.2.2 Eqs. assVar /
// flowVar) of the d=3 and finite-T models, mixed precision.
//
// Memory: the HBM budget is reserved once, at start, and slot buffers are
// carved from that reservation on the host (first fit, coalesced on return),
// so admitting and retiring flows never calls a device allocator: nothing on
// the tick path synchronises the device.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ffrg_internal.cuh"

namespace ffrg {

using Clock = std::chrono::steady_clock;

enum { kQueued = 0, kResident = 1, kDone = 2 };

struct ServeReq {
  unsigned long long id;
  ffrg_problem pb;
  ffrg_table_desc td;
  ffrg_step_opts opts;
  double Lambda;
  std::vector<double> tab, y0, result;
  int state = kQueued;
  int status = FFRG_OK;
  bool cancel = false;
  ffrg_flow_stats stats{};
  double latency = 0.0;
  Clock::time_point t_submit;
  size_t need = 0;   // device bytes while resident
  int ny = 0;
};

// Geometry and device layout of one resident flow (segments of one buffer).
struct SlotLayout {
  Plan pl;
  int ny, npsi;
  size_t bytes;
  size_t o_tab, o_tab32, o_y, o_ys, o_K, o_raw, o_radF, o_radF32, o_radq, o_radq32, o_kc, o_extp, o_psis, o_part;
  size_t o_kbuf;
  size_t o_rx, o_rw, o_a1x, o_a1w, o_a2x, o_a2w, o_psx, o_psw;
};

static size_t seg(size_t &used, size_t bytes) {
  size_t off = (used + 255) & ~(size_t)255;
  used = off + std::max<size_t>(bytes, 16);
  return off;
}

static void slot_layout(const ffrg_problem *pb, const ffrg_table_desc *td, SlotLayout &L) {
  Plan &pl = L.pl;
  pl = Plan();
  plan_geometry(&pl, pb, td);
  pl.sum_w2 = 2.0;
  L.ny = pl.n_ext;
  L.npsi = std::max(1, pl.n_ext_ang);
  const size_t d = sizeof(double);
  size_t u = 0;
  L.o_tab = seg(u, (size_t)pl.tab_count * d);
  L.o_tab32 = seg(u, (size_t)pl.tab32_count * sizeof(float2));
  L.o_y = seg(u, (size_t)L.ny * d);
  L.o_ys = seg(u, (size_t)L.ny * d);
  L.o_K = seg(u, (size_t)7 * L.ny * d);
  L.o_raw = seg(u, (size_t)pl.n_ext * d);
  L.o_radF = seg(u, (size_t)pl.nr * pl.nfreq * d);
  L.o_radq = seg(u, (size_t)pl.nr * d);
  L.o_radq32 = seg(u, (size_t)pl.nr * sizeof(float));
  L.o_radF32 = seg(u, (size_t)pl.nr * pl.nfreq * sizeof(float));
  L.o_kc = seg(u, kKConstBytes);
  L.o_kbuf = seg(u, pl.kbuf_count * sizeof(float));   // finite T: K in FP32 (serving is mixed)
  L.o_extp = seg(u, (size_t)pl.n_ext_p * d);
  L.o_psis = seg(u, (size_t)L.npsi * d);
  L.o_part = seg(u, (size_t)pl.fn_items * d);
  L.o_rx = seg(u, (size_t)pl.nr * d);
  L.o_rw = seg(u, (size_t)pl.nr * d);
  L.o_a1x = seg(u, (size_t)pl.na1 * d);
  L.o_a1w = seg(u, (size_t)pl.na1 * d);
  L.o_a2x = seg(u, d);
  L.o_a2w = seg(u, d);
  L.o_psx = seg(u, (size_t)L.npsi * d);
  L.o_psw = seg(u, (size_t)L.npsi * d);
  L.bytes = u;
}

// First-fit allocator over one device reservation; host bookkeeping only.
// Offsets and sizes are multiples of 256 bytes.
struct Arena {
  unsigned char *base = nullptr;
  size_t size = 0, used = 0;
  std::map<size_t, size_t> free_list;  // offset -> length, no two adjacent
  static size_t round(size_t n) { return (std::max<size_t>(n, 1) + 255) & ~(size_t)255; }
  void init(unsigned char *b, size_t n) {
    base = b;
    size = n;
    used = 0;
    free_list.clear();
    if (n) free_list[0] = n;
  }
  unsigned char *take(size_t n) {
    n = round(n);
    for (auto it = free_list.begin(); it != free_list.end(); ++it)
      if (it->second >= n) {
        const size_t off = it->first, len = it->second;
        free_list.erase(it);
        if (len > n) free_list[off + n] = len - n;
        used += n;
        return base + off;
      }
    return nullptr;
  }
  void give(unsigned char *p, size_t n) {
    if (!p) return;
    n = round(n);
    used -= n;
    auto it = free_list.emplace((size_t)(p - base), n).first;
    auto nx = std::next(it);
    if (nx != free_list.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_list.erase(nx);
    }
    if (it != free_list.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_list.erase(it);
      }
    }
  }
};

struct Slot {
  ServeReq *req = nullptr;
  unsigned char *buf = nullptr;
  size_t cap = 0;
  SlotLayout L;
  RhsArgs ra;
  FlowArgs fa;
  bool fresh = false;    // admitted, first derivative not yet taken
  bool cooling = false;  // retired while a tick that still lists it is in flight
};

// Compact device copies of the descriptors of one launch set.
struct LaunchSet {
  RhsArgs *descs = nullptr;
  FlowArgs *fa = nullptr;
  int *lists = nullptr;  // [all | d3 flows | d3 start | ft flows | ft start]
  BatchList bl{};
  int n = 0, max_ny = 0;
};

// Ticks in flight at most: while the GPU runs one tick, the next is queued
// behind it and the host reads the control blocks of the one before, retires,
// admits and rebuilds the launch set for the tick after.
constexpr int kTickDepth = 2;

struct Server {
  ffrg_ctx lc;  // launch context of the scheduler thread (no allocations behind it)
  ffrg_serve_opts opts{};
  std::thread th;
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  std::deque<ServeReq *> queue;
  std::unordered_map<unsigned long long, ServeReq *> reqs;
  unsigned long long next_id = 1;
  std::vector<Slot> slots;
  unsigned char *arena_mem = nullptr;  // the reserved HBM budget
  Arena arena;                         // slot buffers carved from it
  cudaStream_t st = nullptr;  // ticks: batched steps and first derivatives
  cudaStream_t io = nullptr;  // request uploads and result copies
  FlowCtl *ctl_dev = nullptr;
  FlowCtl *ctl_host = nullptr;        // pinned, kTickDepth snapshots of the control blocks
  cudaEvent_t tick_ev[kTickDepth] = {};  // end of the tick whose snapshot is in buffer b
  unsigned *status_dev = nullptr;
  LaunchSet step_set, init_set;
  unsigned char *stage_host = nullptr;  // pinned staging of descriptor uploads, two buffers
  cudaEvent_t stage_ev[2] = {};         // end of the last upload from staging buffer 0 / 1
  int stage_i = 0;
  size_t stage_bytes = 0;
  ffrg_serve_stats stats{};
  int fatal = FFRG_OK;
};

}  // namespace ffrg

namespace ffrg {

// Fill a slot's device buffer from its request and build its descriptors.
static int slot_setup(Server &S, int si) {
  Slot &sl = S.slots[si];
  ServeReq *r = sl.req;
  SlotLayout &L = sl.L;
  Plan &pl = L.pl;
  unsigned char *b = sl.buf;
  const size_t d = sizeof(double);
  std::vector<double> rx(pl.nr), rw(pl.nr), x1(pl.na1), w1(pl.na1), xp(L.npsi), wp(L.npsi);
  double x2 = 0.0, w2 = 2.0;
  host_gauss_legendre(pl.nr, 0.0, 1.0, rx.data(), rw.data());
  host_gauss_legendre(pl.na1, -1.0, 1.0, x1.data(), w1.data());
  host_gauss_legendre(L.npsi, -1.0, 1.0, xp.data(), wp.data());
  pl.rad_x = (double *)(b + L.o_rx);
  pl.rad_w = (double *)(b + L.o_rw);
  pl.a1_x = (double *)(b + L.o_a1x);
  pl.a1_w = (double *)(b + L.o_a1w);
  pl.a2_x = (double *)(b + L.o_a2x);
  pl.a2_w = (double *)(b + L.o_a2w);
  pl.psi_x = (double *)(b + L.o_psx);
  pl.psi_w = (double *)(b + L.o_psw);
  pl.radF = (double *)(b + L.o_radF);
  pl.radq = (double *)(b + L.o_radq);
  pl.radq32 = (float *)(b + L.o_radq32);
  pl.radF32 = (float *)(b + L.o_radF32);
  pl.kconst = b + L.o_kc;
  pl.kbuf = pl.kbuf_count ? (double *)(b + L.o_kbuf) : nullptr;
  pl.ext_pd = (double *)(b + L.o_extp);
  pl.psi_s = (double *)(b + L.o_psis);
  pl.partial = (double *)(b + L.o_part);
  pl.tab32 = (float2 *)(b + L.o_tab32);
  struct Up { void *dst; const void *src; size_t n; } ups[] = {
      {b + L.o_tab, r->tab.data(), r->tab.size() * d}, {b + L.o_y, r->y0.data(), r->y0.size() * d},
      {pl.rad_x, rx.data(), rx.size() * d},           {pl.rad_w, rw.data(), rw.size() * d},
      {pl.a1_x, x1.data(), x1.size() * d},            {pl.a1_w, w1.data(), w1.size() * d},
      {pl.a2_x, &x2, d},                              {pl.a2_w, &w2, d},
      {pl.psi_x, xp.data(), xp.size() * d},           {pl.psi_w, wp.data(), wp.size() * d}};
  for (auto &u : ups) {
    cudaError_t e = cudaMemcpyAsync(u.dst, u.src, u.n, cudaMemcpyHostToDevice, S.io);
    if (e != cudaSuccess) return set_cuda_error(&S.lc, e, "serve upload");
  }
  FlowCtl hc;
  memset(&hc, 0, sizeof(hc));
  const ffrg_step_opts &o = r->opts;
  hc.t = o.t0;
  hc.t0 = o.t0;
  hc.t1 = o.t1;
  hc.dt = fmin(fmax(o.dt0, o.dt_min), o.dt_max);
  hc.dt_min = o.dt_min;
  hc.dt_max = o.dt_max;
  hc.atol = o.atol;
  hc.rtol = o.rtol;
  hc.end_tol = 1e-13 * fmax(fabs(o.t1 - o.t0), 1.0);
  hc.Lambda = r->Lambda;
  hc.max_steps = o.max_steps;
  FlowCtl *ctl = S.ctl_dev + si;
  cudaError_t e = cudaMemcpyAsync(ctl, &hc, sizeof(hc), cudaMemcpyHostToDevice, S.io);
  if (e != cudaSuccess) return set_cuda_error(&S.lc, e, "serve ctl upload");
  // The host copies above come from pageable memory and the stack: wait for
  // them.  The slot is listed in no launch set of a tick in flight (slots
  // cool down until those ticks end), and the flow's first launch on the
  // tick stream is issued after this wait.
  e = cudaStreamSynchronize(S.io);
  if (e != cudaSuccess) return set_cuda_error(&S.lc, e, "serve upload sync");
  fill_args(&pl, &r->pb, &r->td, (const double *)(b + L.o_tab), r->Lambda, sl.ra);
  sl.ra.fused_ctr = nullptr;   // batched kernels only
  sl.ra.out = (double *)(b + L.o_raw);
  sl.ra.status = S.status_dev;
  sl.ra.k_dev = &ctl->k_stage;
  sl.ra.skip = &ctl->done;
  FlowArgs &f = sl.fa;
  memset(&f, 0, sizeof(f));
  f.ny = L.ny;
  f.mode = 0;
  f.n = r->td.n_pts;
  f.npsi = r->pb.n_ext_ang;
  f.p_min = r->pb.p_min;
  f.p_step = r->pb.n_ext_p > 1 ? log(r->pb.p_max / r->pb.p_min) / (r->pb.n_ext_p - 1) : 0.0;
  f.psi_w = pl.psi_w;
  f.y = (double *)(b + L.o_y);
  f.ys = (double *)(b + L.o_ys);
  f.K = (double *)(b + L.o_K);
  f.raw = (double *)(b + L.o_raw);
  f.ctl = ctl;
  sl.fresh = true;
  return FFRG_OK;
}

static size_t smem32_of(const Plan &pl) {
  return pl.smem32;
}

// Launch set layout: descs | fa | lists (cap ints: all flows, then per group
// cap flow indices and cap + 1 item offsets; padded to an even count so that
// what follows is 8-byte aligned) | per group cap + 1 cost prefixes.
static int list_ints(int cap) { return (cap + kMaxBatchGroups * (2 * cap + 1) + 1) & ~1; }
static size_t set_bytes_of(int cap) {
  return (sizeof(RhsArgs) + sizeof(FlowArgs)) * cap + sizeof(int) * list_ints(cap) +
         sizeof(long long) * kMaxBatchGroups * (cap + 1);
}

// Upload the descriptors of the given slots as one compact launch set.
static int build_set(Server &S, const std::vector<int> &ids, LaunchSet &ls) {
  const int n = (int)ids.size(), cap = (int)S.slots.size();
  ls.n = n;
  ls.max_ny = 0;
  BatchList &bl = ls.bl;
  bl = BatchList();
  if (n == 0) return FFRG_OK;
  // host staging: descs | fa | lists | costs, in the staging buffer whose
  // previous upload has ended (two buffers used in turn)
  unsigned char *stage = S.stage_host + (size_t)S.stage_i * S.stage_bytes;
  cudaError_t e = cudaEventSynchronize(S.stage_ev[S.stage_i]);
  if (e != cudaSuccess) return set_cuda_error(&S.lc, e, "serve staging wait");
  RhsArgs *hd = (RhsArgs *)stage;
  FlowArgs *hf = (FlowArgs *)(stage + sizeof(RhsArgs) * cap);
  int *hl = (int *)(stage + (sizeof(RhsArgs) + sizeof(FlowArgs)) * cap);
  long long *hc = (long long *)(hl + list_ints(cap));
  int gn[kMaxBatchGroups] = {}, gitems[kMaxBatchGroups] = {};
  size_t gsmem[kMaxBatchGroups] = {};
  auto gflows = [&](int g) { return hl + cap + g * (2 * cap + 1); };
  auto gstart = [&](int g) { return gflows(g) + cap; };
  auto gcost = [&](int g) { return hc + (size_t)g * (cap + 1); };
  for (int g = 0; g < kMaxBatchGroups; ++g) {
    gstart(g)[0] = 0;
    gcost(g)[0] = 0;
  }
  for (int i = 0; i < n; ++i) {
    const Slot &sl = S.slots[ids[i]];
    hd[i] = sl.ra;
    hf[i] = sl.fa;
    hl[i] = ids[i];
    ls.max_ny = std::max(ls.max_ny, sl.L.ny);
    bl.max_ext = std::max(bl.max_ext, sl.L.pl.n_ext);
    bl.max_pre = std::max(bl.max_pre, precompute_blocks(sl.ra, 64));
    const size_t smem = smem32_of(sl.L.pl);
    const int occ = std::max(1, std::min(4, batched_ctas_per_sm(&S.lc, sl.L.pl.model, smem)));
    const int g = (sl.L.pl.model == FFRG_MODEL_D3 ? 0 : 4) + occ - 1;
    // estimated cost of one item: rows x (angle nodes per row + per-row work)
    const long long cost = (long long)sl.L.pl.fn_items * sl.L.pl.fcr * (sl.L.pl.fjb + 1);
    const int k = gn[g]++;
    gflows(g)[k] = i;
    gitems[g] += sl.L.pl.fn_items;
    gstart(g)[k + 1] = gitems[g];
    gcost(g)[k + 1] = gcost(g)[k] + cost;
    gsmem[g] = std::max(gsmem[g], smem);
  }
  // stream order on the tick stream: after every tick that reads the old set
  e = cudaMemcpyAsync(ls.descs, stage, set_bytes_of(cap), cudaMemcpyHostToDevice, S.st);
  if (e == cudaSuccess) e = cudaEventRecord(S.stage_ev[S.stage_i], S.st);
  if (e != cudaSuccess) return set_cuda_error(&S.lc, e, "serve descriptor upload");
  S.stage_i ^= 1;
  int *dl = ls.lists;
  const long long *dc = (const long long *)(dl + list_ints(cap));
  bl.descs = ls.descs;
  bl.n_flows = n;
  for (int g = 0; g < kMaxBatchGroups; ++g) {
    if (gn[g] == 0) continue;
    BatchGroup &G = bl.groups[bl.n_groups++];
    G.model = g < 4 ? FFRG_MODEL_D3 : FFRG_MODEL_FINITE_T;
    G.flows = dl + cap + g * (2 * cap + 1);
    G.start = G.flows + cap;
    G.cost = dc + (size_t)g * (cap + 1);
    G.n = gn[g];
    G.items = gitems[g];
    G.smem = gsmem[g];
  }
  return FFRG_OK;
}

}  // namespace ffrg

namespace ffrg {

static void finish_req(Server &S, ServeReq *r, int status) {
  r->status = status;
  r->state = kDone;
  r->latency = std::chrono::duration<double>(Clock::now() - r->t_submit).count();
  if (status == FFRG_ECANCELED) S.stats.cancelled++;
  else S.stats.completed++;
}

// Retire slot si after the tick whose control blocks are c: copy the state
// back (unless cancelled) and let the slot cool down.  A finished flow's state
// no longer changes (its later launches return at once), so the copy may run
// beside the tick in flight.
static int retire(Server &S, int si, const FlowCtl &c, int status) {
  Slot &sl = S.slots[si];
  ServeReq *r = sl.req;
  if (status != FFRG_ECANCELED) {
    r->result.resize(sl.L.ny);
    cudaError_t e = cudaMemcpyAsync(r->result.data(), sl.fa.y, sl.L.ny * sizeof(double), cudaMemcpyDeviceToHost, S.io);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S.io);
    if (e != cudaSuccess) return set_cuda_error(&S.lc, e, "serve result copy");
    r->stats.steps = c.steps;
    r->stats.rejects = c.rejects;
    r->stats.rhs_evals = 1 + 6 * (c.steps + c.rejects);
    r->stats.integrand_evals = (double)r->stats.rhs_evals * ffrg_evals(&r->pb);
    r->stats.t_reached = c.t;
  }
  std::lock_guard<std::mutex> lock(S.mu);
  finish_req(S, r, status);
  sl.req = nullptr;
  sl.fresh = false;
  sl.cooling = true;
  return FFRG_OK;
}

// Admit queued requests (first come, first served) while a slot is free and
// the reserved HBM budget has a contiguous range for the request's buffers;
// otherwise the head of the queue waits for retiring flows to return theirs.
// Host bookkeeping only: no device allocation or free.
static int admit(Server &S) {
  for (;;) {
    ServeReq *r = nullptr;
    int si = -1;
    {
      std::lock_guard<std::mutex> lock(S.mu);
      while (!S.queue.empty() && S.queue.front()->cancel) {
        ServeReq *c = S.queue.front();
        S.queue.pop_front();
        finish_req(S, c, FFRG_ECANCELED);
      }
      if (S.queue.empty()) return FFRG_OK;
      r = S.queue.front();
      for (int i = 0; i < (int)S.slots.size() && si < 0; ++i)
        if (!S.slots[i].req && !S.slots[i].cooling) si = i;
      if (si < 0) return FFRG_OK;
      unsigned char *buf = S.arena.take(r->need);
      if (!buf) return FFRG_OK;
      S.queue.pop_front();
      r->state = kResident;
      Slot &sl = S.slots[si];
      sl.req = r;
      sl.buf = buf;
      sl.cap = r->need;
    }
    Slot &sl = S.slots[si];
    slot_layout(&r->pb, &r->td, sl.L);
    int st = slot_setup(S, si);
    if (st) return st;
    std::lock_guard<std::mutex> lock(S.mu);
    S.stats.admitted++;
  }
}

struct Tick {
  long long id;
  std::vector<int> live;  // slots in this tick's launch set
};

static void scheduler(Server *Sp) {
  Server &S = *Sp;
  cudaSetDevice(S.lc.device);
  bool changed = true;
  std::deque<Tick> inflight;
  std::vector<std::pair<int, long long>> cooling;  // (slot, last tick that lists it)
  long long launched = 0;                           // ids of issued ticks: 1, 2, ...
  int st = FFRG_OK;
  while (true) {
    {
      std::unique_lock<std::mutex> lock(S.mu);
      if (S.stop) break;
    }
    std::vector<int> live;
    for (int i = 0; i < (int)S.slots.size(); ++i)
      if (S.slots[i].req) live.push_back(i);
    // the oldest tick, once the pipeline is full or nothing is left to issue
    if (!inflight.empty() && ((int)inflight.size() >= kTickDepth || live.empty())) {
      Tick T = std::move(inflight.front());
      inflight.pop_front();
      const int b = (int)(T.id % kTickDepth);
      cudaError_t e = cudaEventSynchronize(S.tick_ev[b]);
      if (e != cudaSuccess) {
        st = set_cuda_error(&S.lc, e, "serve tick");
        break;
      }
      {
        std::lock_guard<std::mutex> lock(S.mu);
        S.stats.ticks++;
        S.stats.resident = (int)T.live.size();
        S.stats.peak_resident = std::max(S.stats.peak_resident, (int)T.live.size());
        S.stats.hbm_in_use = S.arena.used;
      }
      const FlowCtl *ctl = S.ctl_host + (size_t)b * S.slots.size();
      for (int i : T.live) {
        Slot &sl = S.slots[i];
        if (!sl.req) continue;  // retired after an earlier tick
        bool cancel;
        {
          std::lock_guard<std::mutex> lock(S.mu);
          cancel = sl.req->cancel;
        }
        if (ctl[i].done || cancel) {
          st = retire(S, i, ctl[i], cancel ? FFRG_ECANCELED : ctl[i].status);
          if (st) break;
          cooling.push_back({i, launched});
          changed = true;
        }
      }
      if (st) break;
      for (size_t k = 0; k < cooling.size();)
        if (cooling[k].second <= T.id) {
          // no tick in flight reads the slot any more: its range returns to the arena
          Slot &cs = S.slots[cooling[k].first];
          cs.cooling = false;
          S.arena.give(cs.buf, cs.cap);
          cs.buf = nullptr;
          cs.cap = 0;
          cooling[k] = cooling.back();
          cooling.pop_back();
        } else {
          ++k;
        }
      S.cv.notify_all();
      continue;  // re-read the slots before admitting
    }
    st = admit(S);
    if (st) break;
    // new flows: first derivative and first step size, queued before the next tick
    std::vector<int> fresh;
    live.clear();
    for (int i = 0; i < (int)S.slots.size(); ++i) {
      if (!S.slots[i].req) continue;
      live.push_back(i);
      if (S.slots[i].fresh) fresh.push_back(i);
    }
    if (!fresh.empty()) {
      st = build_set(S, fresh, S.init_set);
      if (!st) st = launch_flow_batched_init(&S.lc, S.init_set.fa, S.init_set.n, S.init_set.max_ny, S.init_set.bl,
                                            S.st);
      if (st) break;
      for (int i : fresh) S.slots[i].fresh = false;
      changed = true;
    }
    if (live.empty()) {
      if (!inflight.empty()) continue;
      std::unique_lock<std::mutex> lock(S.mu);
      S.cv.wait_for(lock, std::chrono::milliseconds(2), [&] { return S.stop || !S.queue.empty(); });
      continue;
    }
    if (changed) {
      st = build_set(S, live, S.step_set);
      if (st) break;
      changed = false;
    }
    // one tick: a batched step of every flow in the set, then a snapshot of
    // the control blocks into this tick's host buffer
    const long long id = ++launched;
    const int b = (int)(id % kTickDepth);
    st = launch_flow_batched_step(&S.lc, S.step_set.fa, S.step_set.n, S.step_set.max_ny, S.step_set.bl, S.st);
    if (st) break;
    cudaError_t e = cudaMemcpyAsync(S.ctl_host + (size_t)b * S.slots.size(), S.ctl_dev,
                                    sizeof(FlowCtl) * S.slots.size(), cudaMemcpyDeviceToHost, S.st);
    if (e == cudaSuccess) e = cudaEventRecord(S.tick_ev[b], S.st);
    if (e != cudaSuccess) {
      st = set_cuda_error(&S.lc, e, "serve tick");
      break;
    }
    inflight.push_back({id, std::move(live)});
  }
  // drain: nothing of this server stays in flight; everything still queued or
  // resident is cancelled (or failed with the fatal status)
  if (st) S.fatal = st;
  cudaStreamSynchronize(S.st);
  cudaStreamSynchronize(S.io);
  std::lock_guard<std::mutex> lock(S.mu);
  for (auto &sl : S.slots)
    if (sl.req) {
      finish_req(S, sl.req, S.fatal ? S.fatal : FFRG_ECANCELED);
      sl.req = nullptr;
    }
  while (!S.queue.empty()) {
    finish_req(S, S.queue.front(), S.fatal ? S.fatal : FFRG_ECANCELED);
    S.queue.pop_front();
  }
  S.stop = true;
  S.cv.notify_all();
}

}  // namespace ffrg

using namespace ffrg;

static Server *server_of(ffrg_ctx *ctx) { return ctx ? (Server *)ctx->server : nullptr; }

extern "C" int ffrg_serve_start(ffrg_ctx *ctx, const ffrg_serve_opts *opts) {
  if (!ctx || !opts) return FFRG_EINVAL;
  if (ctx->server) return FFRG_EBUSY;
  if (opts->max_slots < 1 || opts->max_slots > 256 || opts->max_queue < 1) return FFRG_EINVAL;
  cudaSetDevice(ctx->device);
  Server *S = new Server();
  S->opts = *opts;
  if (!S->opts.hbm_budget_bytes) S->opts.hbm_budget_bytes = size_t(1) << 30;
  S->lc.device = ctx->device;
  S->lc.num_sms = ctx->num_sms;
  S->lc.budget = 0;
  S->lc.used = 0;
  S->lc.status_dev = nullptr;
  S->lc.status_host = nullptr;
  S->lc.server = nullptr;
  S->lc.profiling = 0;
  S->lc.prof_used = 0;
  const int cap = opts->max_slots;
  S->slots.resize(cap);
  const size_t set_bytes = set_bytes_of(cap);
  S->stage_bytes = set_bytes;
  cudaError_t e = cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->io, cudaStreamNonBlocking);
  for (int b = 0; b < kTickDepth; ++b)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->tick_ev[b], cudaEventDisableTiming);
  for (int b = 0; b < 2; ++b)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->stage_ev[b], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc((void **)&S->ctl_dev, sizeof(FlowCtl) * cap);
  if (e == cudaSuccess) e = cudaMemset(S->ctl_dev, 0, sizeof(FlowCtl) * cap);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&S->ctl_host, sizeof(FlowCtl) * cap * kTickDepth);
  if (e == cudaSuccess) e = cudaMalloc((void **)&S->status_dev, 16);
  if (e == cudaSuccess) e = cudaMemset(S->status_dev, 0, 16);
  if (e == cudaSuccess) e = cudaMallocHost((void **)&S->stage_host, set_bytes * 2);
  // the whole HBM budget of the resident flows, reserved once
  const size_t arena_bytes = S->opts.hbm_budget_bytes & ~(size_t)255;
  if (e == cudaSuccess) e = cudaMalloc((void **)&S->arena_mem, std::max<size_t>(arena_bytes, 256));
  if (e == cudaSuccess) S->arena.init(S->arena_mem, arena_bytes);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();  // the memsets above ran on the legacy stream
  for (LaunchSet *ls : {&S->step_set, &S->init_set}) {
    unsigned char *blk = nullptr;
    if (e == cudaSuccess) e = cudaMalloc((void **)&blk, set_bytes);
    ls->descs = (RhsArgs *)blk;
    ls->fa = (FlowArgs *)(blk + sizeof(RhsArgs) * cap);
    ls->lists = (int *)(blk + (sizeof(RhsArgs) + sizeof(FlowArgs)) * cap);
  }
  if (e != cudaSuccess) {
    int st = set_cuda_error(ctx, e, "ffrg_serve_start");
    cudaFree(S->ctl_dev);
    cudaFreeHost(S->ctl_host);
    cudaFree(S->status_dev);
    cudaFreeHost(S->stage_host);
    cudaFree(S->arena_mem);
    cudaFree(S->step_set.descs);
    cudaFree(S->init_set.descs);
    for (int b = 0; b < kTickDepth; ++b)
      if (S->tick_ev[b]) cudaEventDestroy(S->tick_ev[b]);
    for (int b = 0; b < 2; ++b)
      if (S->stage_ev[b]) cudaEventDestroy(S->stage_ev[b]);
    if (S->io) cudaStreamDestroy(S->io);
    if (S->st) cudaStreamDestroy(S->st);
    delete S;
    return st;
  }
  ctx->server = S;
  S->th = std::thread(scheduler, S);
  return FFRG_OK;
}

extern "C" int ffrg_serve_submit(ffrg_ctx *ctx, const ffrg_problem *pb, const ffrg_table_desc *desc,
                                 const double *tables_host, const double *y0_host, double Lambda,
                                 const ffrg_step_opts *o, unsigned long long *ticket) {
  Server *S = server_of(ctx);
  if (!S) return FFRG_EINVAL;
  if (!pb || !desc || !tables_host || !y0_host || !o || !ticket) return FFRG_EINVAL;
  if (pb->model != FFRG_MODEL_D3 && pb->model != FFRG_MODEL_FINITE_T) return FFRG_EINVAL;
  if (validate_problem(pb, desc) != FFRG_OK) return FFRG_EINVAL;
  if (!(Lambda > 0.0) || !isfinite(Lambda) || !(o->t1 >= o->t0) || !(o->dt0 > 0.0) || !(o->dt_min > 0.0) ||
      !(o->dt_max >= o->dt_min) || !(o->atol >= 0.0) || !(o->rtol >= 0.0) || !(o->atol + o->rtol > 0.0) ||
      o->max_steps < 1)
    return FFRG_EINVAL;
  SlotLayout L;
  slot_layout(pb, desc, L);
  if (smem32_of(L.pl) > 227 * 1024) return FFRG_EINVAL;
  ServeReq *r = new ServeReq();
  r->pb = *pb;
  r->td = *desc;
  r->opts = *o;
  r->Lambda = Lambda;
  r->tab.assign(tables_host, tables_host + (size_t)L.pl.tab_count);
  r->y0.assign(y0_host, y0_host + L.ny);
  r->need = L.bytes;
  r->ny = L.ny;
  std::lock_guard<std::mutex> lock(S->mu);
  if (S->stop) {
    delete r;
    return S->fatal ? S->fatal : FFRG_EINVAL;
  }
  if (Arena::round(r->need) > S->arena.size) {
    S->stats.rejected++;
    delete r;
    return FFRG_ENOMEM;
  }
  if ((int)S->queue.size() >= S->opts.max_queue) {
    S->stats.rejected++;
    delete r;
    return FFRG_EBUSY;
  }
  r->id = S->next_id++;
  r->t_submit = Clock::now();
  S->queue.push_back(r);
  S->reqs[r->id] = r;
  S->stats.submitted++;
  *ticket = r->id;
  S->cv.notify_all();
  return FFRG_OK;
}

extern "C" int ffrg_serve_poll(ffrg_ctx *ctx, unsigned long long ticket, double *result_host, ffrg_flow_stats *stats,
                               double *latency_s) {
  Server *S = server_of(ctx);
  if (!S) return FFRG_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return FFRG_ENOTFOUND;
  ServeReq *r = it->second;
  if (r->state != kDone) return FFRG_EPENDING;
  if (result_host && !r->result.empty()) memcpy(result_host, r->result.data(), r->result.size() * sizeof(double));
  if (stats) *stats = r->stats;
  if (latency_s) *latency_s = r->latency;
  const int st = r->status;
  S->reqs.erase(it);
  delete r;
  return st;
}

extern "C" int ffrg_serve_cancel(ffrg_ctx *ctx, unsigned long long ticket) {
  Server *S = server_of(ctx);
  if (!S) return FFRG_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) return FFRG_ENOTFOUND;
  it->second->cancel = true;
  S->cv.notify_all();
  return FFRG_OK;
}

extern "C" int ffrg_serve_get_stats(ffrg_ctx *ctx, ffrg_serve_stats *out) {
  Server *S = server_of(ctx);
  if (!S || !out) return FFRG_EINVAL;
  std::lock_guard<std::mutex> lock(S->mu);
  *out = S->stats;
  out->queued = (int)S->queue.size();
  return FFRG_OK;
}

extern "C" int ffrg_serve_stop(ffrg_ctx *ctx) {
  Server *S = server_of(ctx);
  if (!S) return FFRG_EINVAL;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
    S->cv.notify_all();
  }
  if (S->th.joinable()) S->th.join();
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(S->st);
  cudaStreamSynchronize(S->io);
  for (auto &kv : S->reqs) delete kv.second;
  cudaFree(S->arena_mem);
  cudaFree(S->ctl_dev);
  cudaFreeHost(S->ctl_host);
  cudaFree(S->status_dev);
  cudaFreeHost(S->stage_host);
  cudaFree(S->step_set.descs);
  cudaFree(S->init_set.descs);
  for (int b = 0; b < kTickDepth; ++b) cudaEventDestroy(S->tick_ev[b]);
  for (int b = 0; b < 2; ++b) cudaEventDestroy(S->stage_ev[b]);
  cudaStreamDestroy(S->io);
  cudaStreamDestroy(S->st);
  const int fatal = S->fatal;
  if (fatal) ctx->last_error = S->lc.last_error;
  delete S;
  ctx->server = nullptr;
  return fatal;
}
