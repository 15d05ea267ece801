// C ABI for ensembles of independent lattices of uneven size (the batched
// configuration): per-box handles, coefficient tables, work-item schedules,
// the three scheduling modes and their CUDA-graph capture.
#include <cuda_runtime.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <numeric>
#include <vector>

#include "../../include/u1u1.h"
#include "host_internal.h"
#include "u1u1_internal.cuh"

using namespace u1u1;

namespace {

// Device copy of one run's schedule (sorted order, prefix tables).
struct Schedule {
  std::vector<int> steps;
  int* d_order = nullptr;
  int* d_steps = nullptr;
  long long* d_box_prefix = nullptr;
  long long* d_step_off = nullptr;
  EnsSched sc{};
  std::vector<long long> items_per_step;  // for the per-step mode
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};

  ~Schedule() {
    for (auto& g : graph)
      if (g) cudaGraphExecDestroy(g);
    dev_free(d_order);
    dev_free(d_steps);
    dev_free(d_box_prefix);
    dev_free(d_step_off);
  }
};

// One detection step k of a run: the boxes detecting at k and the prefix
// sums of their work items in each batched pass (offsets into the plan's
// device arrays).
struct DetGroup {
  int k = 0;
  int nlist = 0;
  size_t list = 0;                      // ints: box indices
  size_t pm = 0, pw = 0, pc = 0, po = 0;  // long longs: nlist + 1 prefix sums each
  long long m_items = 0, w_items = 0, c_items = 0, o_items = 0;
  bool stage = false;                   // some box has more partials than one finalize CTA takes
};
// A launch of plain steps: its schedule view (order, prefix tables) and,
// for persistent segments, each box's first run step.
struct PlainLaunch {
  int k = 0;               // per-step mode: the run step
  size_t order = 0, steps = 0, kstart = 0;  // ints
  size_t prefix = 0, step_off = 0;          // long longs
  int nboxes = 0, smax = 0;
  long long total = 0;     // items (persistent: all steps of the segment)
  long long items = 0;     // per-step mode: items of step k
};

// Device plan of a run with detection every `de` steps: per-step plain
// launches and detection groups (per-step mode), persistent segments between
// the detection steps and the same groups (persistent mode).
struct DetPlan {
  std::vector<DetGroup> groups;
  std::vector<PlainLaunch> per_step;   // one per run step
  std::vector<PlainLaunch> segments;   // groups.size() + 1 persistent segments
  int* d_int = nullptr;
  long long* d_ll = nullptr;
  cudaGraphExec_t graph[3] = {nullptr, nullptr, nullptr};
  ~DetPlan() {
    for (auto& g : graph)
      if (g) cudaGraphExecDestroy(g);
    dev_free(d_int);
    dev_free(d_ll);
  }
};

}  // namespace

struct u1u1_ensemble {
  int nboxes = 0;
  int precision = U1U1_FP32;
  int horizon = 0;
  std::vector<u1u1_lattice*> boxes;
  void* d_boxes = nullptr;  // EnsBox<T>[nboxes]
  TmaPlan* d_tma = nullptr;  // tensor maps, two position buffers per box
  EnsDyn* d_dyn = nullptr;
  void* d_coef = nullptr;   // Coef<T>[nboxes * horizon]
  unsigned long long* d_ticket = nullptr;
  unsigned* d_done = nullptr;
  int* d_err = nullptr;      // [0]: persistent-kernel error, [1]: tensor-copy timeout of the per-step kernel
  std::vector<int> ntiles;
  // host view of the device step indices after every enqueued run
  std::vector<long long> shadow_n;
  std::vector<int> shadow_cur;
  long long wait_limit_ns = 2000000000LL;
  int inject = 0;
  int poisoned = 0;
  int item_lz = ENS_LZ;  // z-chunk of a work item (tuning knob)
  int persistent_tma = 1;  // the persistent kernel fills interior tiles by tensor copies (tuning knob)
  std::map<std::vector<int>, std::unique_ptr<Schedule>> schedules;
  cudaStream_t capture_stream = nullptr;
  // detection inside runs: per-box resources and plans keyed by
  // (steps, detect_every, each box's step index modulo detect_every)
  EnsDet* d_det = nullptr;
  std::vector<EnsDet> hdet;
  std::vector<long long> shadow_rec;
  std::map<std::vector<int>, std::unique_ptr<DetPlan>> det_plans;
  // the boxes' step views (an EnsViews<T>, host memory) passed to the step
  // kernels as a parameter; empty above ENS_VIEW_MAX boxes
  std::vector<unsigned char> views;
};

namespace {

template <typename T>
const EnsViews<T>* host_views(const u1u1_ensemble* e) {
  return e->views.empty() ? nullptr : reinterpret_cast<const EnsViews<T>*>(e->views.data());
}

template <typename T>
int build_tables(u1u1_ensemble* e, cudaStream_t st) {
  const int nb = e->nboxes;
  std::vector<EnsBox<T>> hb(nb);
  for (int b = 0; b < nb; ++b) {
    u1u1_lattice* h = e->boxes[b];
    EnsBox<T>& B = hb[b];
    for (int k = 0; k < 2; ++k)
      for (int f = 0; f < U1U1_NPOS; ++f) B.pos[k][f] = (T*)h->pos[k][f];
    for (int f = 0; f < U1U1_NMOM; ++f) B.mom[f] = (T*)h->mom[f];
    B.nx = h->p.nx;
    B.ny = h->p.ny;
    B.nz = h->p.nz;
    B.dx = (T)h->p.dx;
    e->ntiles[b] = ens_tile_grid(B.nx, B.ny, B.nz, &B.gx, &B.gy, &B.lz, &B.gz, e->item_lz);
    B.ntiles = e->ntiles[b];
    B.coef0 = (long long)b * e->horizon;
  }
  e->views.clear();
  if (nb <= ENS_VIEW_MAX) {
    e->views.assign(sizeof(EnsViews<T>), 0);
    EnsViews<T>* V = reinterpret_cast<EnsViews<T>*>(e->views.data());
    for (int b = 0; b < nb; ++b)
      for (int k = 0; k < 2; ++k) {
        LatticeView<T>& v = V->v[b][k];
        for (int f = 0; f < U1U1_NPOS; ++f) {
          v.pin[f] = hb[b].pos[k][f];
          v.pout[f] = hb[b].pos[k ^ 1][f];
        }
        for (int f = 0; f < U1U1_NMOM; ++f) v.mom[f] = hb[b].mom[f];
        v.nx = hb[b].nx;
        v.ny = hb[b].ny;
        v.nz = hb[b].nz;
      }
  }
  // tensor maps of each box's two position buffers (FP32; disabled plans
  // otherwise), read by the kernels from device memory
  std::vector<TmaPlan> hp((size_t)2 * nb);
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 2; ++k) {
      make_tma_plan<T>(hb[b].pos[k], hb[b].nx, hb[b].ny, hb[b].nz, &hp[2 * b + k]);
      hp[2 * b + k].status = e->d_err + 1;  // a copy timeout is this ensemble's, reported by its status
    }
  if (!e->d_tma) U1U1_CUDA_TRY(dev_alloc(&e->d_tma, sizeof(TmaPlan) * hp.size()), "ensemble tensor maps");
  U1U1_CUDA_TRY(cudaMemcpyAsync(e->d_tma, hp.data(), sizeof(TmaPlan) * hp.size(), cudaMemcpyHostToDevice, st),
                "tensor map copy");
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 2; ++k) hb[b].tma[k] = e->d_tma + 2 * b + k;
  if (!e->d_boxes) U1U1_CUDA_TRY(dev_alloc(&e->d_boxes, sizeof(EnsBox<T>) * nb), "ensemble box table");
  U1U1_CUDA_TRY(cudaMemcpyAsync(e->d_boxes, hb.data(), sizeof(EnsBox<T>) * nb, cudaMemcpyHostToDevice, st),
                "box table copy");
  // detection resources: each box's own handle scratch, and the grids of a
  // single lattice's measuring and windings passes of its shape
  e->hdet.assign(nb, EnsDet{});
  for (int b = 0; b < nb; ++b) {
    u1u1_lattice* h = e->boxes[b];
    EnsDet& D = e->hdet[b];
    D.part = h->partials;
    D.faces = h->faces;
    D.masks = h->masks;
    D.counts = h->cpartials;
    D.ge4 = h->ge4;
    D.ring = h->ring;
    tiled_grid_dims(h->p.nx, h->p.ny, h->p.nz, (int)sizeof(T), TILE_WAVES_DEFAULT, &D.mgx, &D.mgy, &D.mgz, &D.mlz);
    wind_grid_dims(h->p.nx, h->p.ny, h->p.nz, &D.wtx, &D.wty, &D.wtz, &D.wlz);
    D.nmeas = D.mgx * D.mgy * D.mgz;
    D.nwind = D.wtx * D.wty * D.wtz;
    D.words = (h->p.nx + 31) / 32;
    D.tol = h->overlap_tol;
    D.nx = h->p.nx;
    D.ny = h->p.ny;
    D.nz = h->p.nz;
    if (D.nmeas + D.nwind > h->npartials)
      return fail(U1U1_ERR_STATE, "box %d: detection partials exceed the handle's buffer", b);
  }
  if (!e->d_det) U1U1_CUDA_TRY(dev_alloc(&e->d_det, sizeof(EnsDet) * nb), "detection table");
  U1U1_CUDA_TRY(cudaMemcpyAsync(e->d_det, e->hdet.data(), sizeof(EnsDet) * nb, cudaMemcpyHostToDevice, st),
                "detection table copy");
  if (e->d_coef) return U1U1_OK;  // a re-tiling keeps the coefficient table
  // per-step coefficients of every box up to the horizon
  std::vector<Coef<T>> hc((size_t)nb * e->horizon);
  for (int b = 0; b < nb; ++b)
    for (int n = 0; n < e->horizon; ++n) hc[(size_t)b * e->horizon + n] = make_coef<T>(&e->boxes[b]->p, n);
  U1U1_CUDA_TRY(dev_alloc(&e->d_coef, sizeof(Coef<T>) * hc.size()), "coefficient table");
  U1U1_CUDA_TRY(cudaMemcpyAsync(e->d_coef, hc.data(), sizeof(Coef<T>) * hc.size(), cudaMemcpyHostToDevice, st),
                "coefficient copy");
  return U1U1_OK;
}

int make_schedule(u1u1_ensemble* e, const std::vector<int>& steps, Schedule** out, cudaStream_t st) {
  auto it = e->schedules.find(steps);
  if (it != e->schedules.end()) {
    *out = it->second.get();
    return U1U1_OK;
  }
  const int nb = e->nboxes;
  std::unique_ptr<Schedule> s(new Schedule());
  s->steps = steps;
  std::vector<int> order(nb);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return steps[a] > steps[b]; });
  std::vector<long long> prefix(nb + 1, 0);
  for (int i = 0; i < nb; ++i) prefix[i + 1] = prefix[i] + e->ntiles[order[i]];
  const int smax = nb ? steps[order[0]] : 0;
  std::vector<long long> off(smax + 1, 0);
  s->items_per_step.assign(smax, 0);
  int active = nb;
  for (int k = 0; k < smax; ++k) {
    while (active > 0 && steps[order[active - 1]] <= k) --active;
    s->items_per_step[k] = prefix[active];
    off[k + 1] = off[k] + prefix[active];
  }
  U1U1_CUDA_TRY(dev_alloc(&s->d_order, sizeof(int) * std::max(nb, 1)), "schedule");
  U1U1_CUDA_TRY(dev_alloc(&s->d_steps, sizeof(int) * std::max(nb, 1)), "schedule");
  U1U1_CUDA_TRY(dev_alloc(&s->d_box_prefix, sizeof(long long) * (nb + 1)), "schedule");
  U1U1_CUDA_TRY(dev_alloc(&s->d_step_off, sizeof(long long) * (smax + 1)), "schedule");
  U1U1_CUDA_TRY(cudaMemcpyAsync(s->d_order, order.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st), "schedule");
  U1U1_CUDA_TRY(cudaMemcpyAsync(s->d_steps, steps.data(), sizeof(int) * nb, cudaMemcpyHostToDevice, st), "schedule");
  U1U1_CUDA_TRY(cudaMemcpyAsync(s->d_box_prefix, prefix.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice,
                                st),
                "schedule");
  U1U1_CUDA_TRY(cudaMemcpyAsync(s->d_step_off, off.data(), sizeof(long long) * (smax + 1), cudaMemcpyHostToDevice, st),
                "schedule");
  s->sc.order = s->d_order;
  s->sc.steps = s->d_steps;
  s->sc.box_prefix = s->d_box_prefix;
  s->sc.step_off = s->d_step_off;
  s->sc.nboxes = nb;
  s->sc.smax = smax;
  s->sc.total = off[smax];
  *out = s.get();
  e->schedules[steps] = std::move(s);
  return U1U1_OK;
}

// Enqueue the device work of one run without detection, or the unbatched
// loop with it (no host bookkeeping).
template <typename T>
int enqueue_run(u1u1_ensemble* e, Schedule* s, int mode, int de, cudaStream_t st) {
  const EnsBox<T>* boxes = (const EnsBox<T>*)e->d_boxes;
  const Coef<T>* coef = (const Coef<T>*)e->d_coef;
  cudaError_t err = cudaSuccess;
  if (mode == U1U1_ENS_PERSISTENT) {
    U1U1_CUDA_TRY(cudaMemsetAsync(e->d_ticket, 0, sizeof(unsigned long long), st), "ticket reset");
    U1U1_CUDA_TRY(cudaMemsetAsync(e->d_done, 0, sizeof(unsigned) * e->nboxes, st), "counter reset");
    U1U1_CUDA_TRY(cudaMemsetAsync(e->d_err, 0, sizeof(int), st), "status reset");
    err = launch_ens_persistent<T>(boxes, e->d_dyn, coef, s->sc, nullptr, e->d_ticket, e->d_done, e->d_err,
                                   e->wait_limit_ns, e->inject, e->persistent_tma, host_views<T>(e), st);
    if (err != cudaSuccess) return cuda_fail(err, "persistent ensemble kernel");
  } else if (mode == U1U1_ENS_PER_STEP) {
    for (int k = 0; k < s->sc.smax; ++k) {
      err = launch_ens_step<T>(boxes, e->d_dyn, coef, s->sc, k, s->items_per_step[k], host_views<T>(e), st);
      if (err != cudaSuccess) return cuda_fail(err, "ensemble step kernel");
    }
  } else {
    // the per-box handles advance their own host bookkeeping here
    for (int b = 0; b < e->nboxes; ++b) {
      const int rc = u1u1_step(e->boxes[b], s->steps[b], de, st);
      if (rc) return rc;
    }
  }
  err = launch_ens_advance(e->d_dyn, s->d_steps, e->nboxes, de, st);
  if (err != cudaSuccess) return cuda_fail(err, "ensemble advance kernel");
  return U1U1_OK;
}

int enqueue(u1u1_ensemble* e, Schedule* s, int mode, int de, cudaStream_t st) {
  return e->precision == U1U1_FP64 ? enqueue_run<double>(e, s, mode, de, st)
                                   : enqueue_run<float>(e, s, mode, de, st);
}

// box b, at step index n0 when the run starts, detects at run step k
bool detects(long long n0, int k, int steps, int de) { return de > 0 && k < steps && (n0 + k) % de == 0; }

// Plan of a run with detection every de steps (host tables, then one upload).
int make_det_plan(u1u1_ensemble* e, const std::vector<int>& steps, int de, DetPlan** out, cudaStream_t st) {
  const int nb = e->nboxes;
  std::vector<int> key(steps);
  key.push_back(de);
  std::vector<long long> n0(nb);
  for (int b = 0; b < nb; ++b) {
    n0[b] = e->boxes[b]->n;
    key.push_back((int)(n0[b] % de));
  }
  auto it = e->det_plans.find(key);
  if (it != e->det_plans.end()) {
    *out = it->second.get();
    return U1U1_OK;
  }
  std::unique_ptr<DetPlan> P(new DetPlan());
  std::vector<int> ints;
  std::vector<long long> lls;
  auto push_ints = [&](const std::vector<int>& v) {
    const size_t off = ints.size();
    ints.insert(ints.end(), v.begin(), v.end());
    if (v.empty()) ints.push_back(0);  // keep every view's offset valid
    return off;
  };
  auto push_prefix = [&](const std::vector<long long>& c) {
    const size_t off = lls.size();
    lls.push_back(0);
    for (long long v : c) lls.push_back(lls.back() + v);
    return off;
  };
  int smax = 0;
  for (int b = 0; b < nb; ++b) smax = std::max(smax, steps[b]);
  // detection groups
  for (int k = 0; k < smax; ++k) {
    std::vector<int> list;
    for (int b = 0; b < nb; ++b)
      if (detects(n0[b], k, steps[b], de)) list.push_back(b);
    if (list.empty()) continue;
    DetGroup g;
    g.k = k;
    g.nlist = (int)list.size();
    g.list = push_ints(list);
    std::vector<long long> m, w, c, o;
    for (int b : list) {
      const EnsDet& D = e->hdet[b];
      const long long words = (long long)D.words * D.ny * D.nz;
      m.push_back(D.nmeas);
      w.push_back(D.nwind);
      c.push_back(words);
      o.push_back((words + 31) / 32);
      g.m_items += D.nmeas;
      g.w_items += D.nwind;
      g.c_items += words;
      g.o_items += (words + 31) / 32;
      if (D.nmeas + D.nwind > FIN_STAGE_MIN) g.stage = true;
    }
    g.pm = push_prefix(m);
    g.pw = push_prefix(w);
    g.pc = push_prefix(c);
    g.po = push_prefix(o);
    P->groups.push_back(g);
  }
  // per-step mode: the plain steps of each run step
  for (int k = 0; k < smax; ++k) {
    std::vector<int> plain;
    std::vector<long long> tiles;
    for (int b = 0; b < nb; ++b)
      if (k < steps[b] && !detects(n0[b], k, steps[b], de)) {
        plain.push_back(b);
        tiles.push_back(e->ntiles[b]);
      }
    PlainLaunch L;
    L.k = k;
    L.nboxes = (int)plain.size();
    L.order = push_ints(plain);
    L.prefix = push_prefix(tiles);
    for (long long t : tiles) L.items += t;
    P->per_step.push_back(L);
  }
  // persistent mode: segments of plain steps between detection steps; the
  // boxes that detect at a step start the next segment one step later
  const int ng = (int)P->groups.size();
  for (int j = 0; j <= ng; ++j) {
    std::vector<int> cnt(nb), kst(nb);
    for (int b = 0; b < nb; ++b) {
      const int g0 = j == 0 ? 0 : P->groups[j - 1].k;
      const int start = j == 0 ? 0 : g0 + (detects(n0[b], g0, steps[b], de) ? 1 : 0);
      const int end = std::min(j < ng ? P->groups[j].k : steps[b], steps[b]);
      cnt[b] = std::max(0, end - start);
      kst[b] = start;
    }
    std::vector<int> order(nb);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cnt[a] > cnt[b]; });
    std::vector<long long> tiles(nb);
    for (int i = 0; i < nb; ++i) tiles[i] = e->ntiles[order[i]];
    const int sm = nb ? cnt[order[0]] : 0;
    std::vector<long long> per(sm, 0);
    int active = nb;
    for (int k = 0; k < sm; ++k) {
      while (active > 0 && cnt[order[active - 1]] <= k) --active;
      for (int i = 0; i < active; ++i) per[k] += e->ntiles[order[i]];
    }
    PlainLaunch L;
    L.order = push_ints(order);
    L.steps = push_ints(cnt);
    L.kstart = push_ints(kst);
    L.prefix = push_prefix(tiles);
    L.step_off = push_prefix(per);
    L.nboxes = nb;
    L.smax = sm;
    for (long long v : per) L.total += v;
    P->segments.push_back(L);
  }
  U1U1_CUDA_TRY(dev_alloc(&P->d_int, sizeof(int) * std::max<size_t>(ints.size(), 1)), "detection plan");
  U1U1_CUDA_TRY(dev_alloc(&P->d_ll, sizeof(long long) * std::max<size_t>(lls.size(), 1)), "detection plan");
  U1U1_CUDA_TRY(cudaMemcpyAsync(P->d_int, ints.data(), sizeof(int) * ints.size(), cudaMemcpyHostToDevice, st),
                "plan copy");
  U1U1_CUDA_TRY(cudaMemcpyAsync(P->d_ll, lls.data(), sizeof(long long) * lls.size(), cudaMemcpyHostToDevice, st),
                "plan copy");
  *out = P.get();
  e->det_plans[key] = std::move(P);
  return U1U1_OK;
}

EnsSched view(const DetPlan* P, const PlainLaunch& L) {
  EnsSched sc{};
  sc.order = P->d_int + L.order;
  sc.steps = P->d_int + L.steps;
  sc.box_prefix = P->d_ll + L.prefix;
  sc.step_off = P->d_ll + L.step_off;
  sc.nboxes = L.nboxes;
  sc.smax = L.smax;
  sc.total = L.total;
  return sc;
}

// the batched detection of one group: measuring step, windings, cells and
// overlap, finalize into each box's record ring
template <typename T>
int enqueue_group(u1u1_ensemble* e, const DetPlan* P, const DetGroup& g, int de, cudaStream_t st) {
  const EnsBox<T>* boxes = (const EnsBox<T>*)e->d_boxes;
  const Coef<T>* coef = (const Coef<T>*)e->d_coef;
  const int* list = P->d_int + g.list;
  cudaError_t err = launch_ens_measure<T>(boxes, e->d_det, e->d_dyn, coef, list, P->d_ll + g.pm, g.nlist, g.m_items,
                                          g.k, host_views<T>(e), st);
  if (err != cudaSuccess) return cuda_fail(err, "ensemble measuring step");
  err = launch_ens_windings<T>(boxes, e->d_det, e->d_dyn, list, P->d_ll + g.pw, g.nlist, g.w_items, g.k, st);
  if (err != cudaSuccess) return cuda_fail(err, "ensemble windings");
  err = launch_ens_cells(e->d_det, list, P->d_ll + g.pc, P->d_ll + g.po, g.nlist, g.c_items, g.o_items, st);
  if (err != cudaSuccess) return cuda_fail(err, "ensemble cells and overlap");
  err = launch_ens_finalize(e->d_det, e->d_dyn, list, g.nlist, g.k, de, g.stage, st);
  if (err != cudaSuccess) return cuda_fail(err, "ensemble finalize");
  return U1U1_OK;
}

// Enqueue the device work of one batched run with detection.
template <typename T>
int enqueue_det_run(u1u1_ensemble* e, Schedule* s, DetPlan* P, int mode, int de, cudaStream_t st) {
  const EnsBox<T>* boxes = (const EnsBox<T>*)e->d_boxes;
  const Coef<T>* coef = (const Coef<T>*)e->d_coef;
  cudaError_t err = cudaSuccess;
  if (mode == U1U1_ENS_PERSISTENT) {
    U1U1_CUDA_TRY(cudaMemsetAsync(e->d_err, 0, sizeof(int), st), "status reset");
    for (size_t j = 0; j < P->segments.size(); ++j) {
      const PlainLaunch& L = P->segments[j];
      if (L.total > 0) {
        U1U1_CUDA_TRY(cudaMemsetAsync(e->d_ticket, 0, sizeof(unsigned long long), st), "ticket reset");
        U1U1_CUDA_TRY(cudaMemsetAsync(e->d_done, 0, sizeof(unsigned) * e->nboxes, st), "counter reset");
        err = launch_ens_persistent<T>(boxes, e->d_dyn, coef, view(P, L), P->d_int + L.kstart, e->d_ticket,
                                       e->d_done, e->d_err, e->wait_limit_ns, e->inject, e->persistent_tma,
                                       host_views<T>(e), st);
        if (err != cudaSuccess) return cuda_fail(err, "persistent ensemble kernel");
      }
      if (j < P->groups.size()) {
        const int rc = enqueue_group<T>(e, P, P->groups[j], de, st);
        if (rc) return rc;
      }
    }
  } else {
    size_t gi = 0;
    for (const PlainLaunch& L : P->per_step) {
      if (L.items > 0) {
        err = launch_ens_step<T>(boxes, e->d_dyn, coef, view(P, L), L.k, L.items, host_views<T>(e), st);
        if (err != cudaSuccess) return cuda_fail(err, "ensemble step kernel");
      }
      if (gi < P->groups.size() && P->groups[gi].k == L.k) {
        const int rc = enqueue_group<T>(e, P, P->groups[gi++], de, st);
        if (rc) return rc;
      }
    }
  }
  err = launch_ens_advance(e->d_dyn, s->d_steps, e->nboxes, de, st);
  if (err != cudaSuccess) return cuda_fail(err, "ensemble advance kernel");
  return U1U1_OK;
}

int enqueue_det(u1u1_ensemble* e, Schedule* s, DetPlan* P, int mode, int de, cudaStream_t st) {
  return e->precision == U1U1_FP64 ? enqueue_det_run<double>(e, s, P, mode, de, st)
                                   : enqueue_det_run<float>(e, s, P, mode, de, st);
}

// bring the device step table in line with the per-box handles (a box may
// have been stepped or loaded through its borrowed handle)
int sync_dyn(u1u1_ensemble* e, cudaStream_t st) {
  bool stale = false;
  for (int b = 0; b < e->nboxes; ++b)
    if (e->boxes[b]->n != e->shadow_n[b] || e->boxes[b]->cur != e->shadow_cur[b] ||
        e->boxes[b]->rec_written != e->shadow_rec[b])
      stale = true;
  if (!stale) return U1U1_OK;
  std::vector<EnsDyn> hd(e->nboxes);
  for (int b = 0; b < e->nboxes; ++b) {
    hd[b].n = e->boxes[b]->n;
    hd[b].rec = e->boxes[b]->rec_written;
    hd[b].cur = e->boxes[b]->cur;
    hd[b].pad = 0;
    e->shadow_n[b] = hd[b].n;
    e->shadow_cur[b] = hd[b].cur;
    e->shadow_rec[b] = hd[b].rec;
  }
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  U1U1_CUDA_TRY(cudaMemcpyAsync(e->d_dyn, hd.data(), sizeof(EnsDyn) * e->nboxes, cudaMemcpyHostToDevice, st),
                "step table");
  return U1U1_OK;
}

}  // namespace

extern "C" void u1u1_ensemble_destroy(u1u1_ensemble* e) {
  if (!e) return;
  e->schedules.clear();
  e->det_plans.clear();
  for (u1u1_lattice* h : e->boxes) lattice_destroy(h);
  dev_free(e->d_boxes);
  dev_free(e->d_tma);
  dev_free(e->d_dyn);
  dev_free(e->d_coef);
  dev_free(e->d_ticket);
  dev_free(e->d_done);
  dev_free(e->d_err);
  dev_free(e->d_det);
  if (e->capture_stream) cudaStreamDestroy(e->capture_stream);
  delete e;
}

extern "C" int u1u1_ensemble_create(const u1u1_params* per_box, int nboxes, const u1u1_buffers* buffers, int horizon,
                                    void* stream, u1u1_ensemble** out) {
  if (!per_box || !buffers || !out) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (nboxes < 1) return fail(U1U1_ERR_INVALID_ARG, "nboxes must be >= 1");
  if (horizon < 0) return fail(U1U1_ERR_INVALID_ARG, "horizon must be >= 0");
  for (int b = 1; b < nboxes; ++b)
    if (per_box[b].precision != per_box[0].precision)
      return fail(U1U1_ERR_INVALID_ARG, "all boxes of an ensemble share one precision");
  cudaStream_t st = (cudaStream_t)stream;
  u1u1_ensemble* e = new u1u1_ensemble();
  e->nboxes = nboxes;
  e->precision = per_box[0].precision;
  e->horizon = horizon ? horizon : 8192;
  e->ntiles.assign(nboxes, 0);
  e->shadow_n.assign(nboxes, 0);
  e->shadow_cur.assign(nboxes, 0);
  e->shadow_rec.assign(nboxes, 0);
  for (int b = 0; b < nboxes; ++b) {
    u1u1_lattice* h = nullptr;
    int rc = u1u1_init_lattice(&per_box[b], &buffers[b], stream, &h);
    if (rc) {
      u1u1_ensemble_destroy(e);
      return rc;
    }
    h->kernel = U1U1_KERNEL_TILED;
    h->ensemble_box = 1;
    e->boxes.push_back(h);
  }
  int rc = U1U1_OK;
  cudaError_t err = cudaSuccess;
  if (err == cudaSuccess) err = dev_alloc(&e->d_err, 2 * sizeof(int));
  if (err == cudaSuccess) err = cudaMemsetAsync(e->d_err, 0, 2 * sizeof(int), st);
  if (err != cudaSuccess) rc = cuda_fail(err, "ensemble allocation");
  if (!rc) rc = e->precision == U1U1_FP64 ? build_tables<double>(e, st) : build_tables<float>(e, st);
  if (!rc) {
    if (err == cudaSuccess) err = dev_alloc(&e->d_dyn, sizeof(EnsDyn) * nboxes);
    if (err == cudaSuccess) err = dev_alloc(&e->d_ticket, sizeof(unsigned long long));
    if (err == cudaSuccess) err = dev_alloc(&e->d_done, sizeof(unsigned) * nboxes);
    if (err == cudaSuccess) err = cudaMemsetAsync(e->d_dyn, 0, sizeof(EnsDyn) * nboxes, st);
    if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&e->capture_stream, cudaStreamNonBlocking);
    if (err != cudaSuccess) rc = cuda_fail(err, "ensemble allocation");
  }
  if (rc) {
    u1u1_ensemble_destroy(e);
    return rc;
  }
  *out = e;
  return U1U1_OK;
}

extern "C" int u1u1_ensemble_run(u1u1_ensemble* e, const int* steps, int detect_every, int mode, int use_graph,
                                 void* stream) {
  const NvtxRange range("u1u1_ensemble_run");
  if (!e || !steps) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (mode < U1U1_ENS_PERSISTENT || mode > U1U1_ENS_UNBATCHED) return fail(U1U1_ERR_INVALID_ARG, "unknown mode %d", mode);
  if (detect_every < 0) return fail(U1U1_ERR_INVALID_ARG, "detect_every must be >= 0");
  const int de = detect_every;
  if (e->poisoned) return fail(U1U1_ERR_STATE, "an earlier persistent run timed out; the ensemble state is incomplete");
  std::vector<int> sv(steps, steps + e->nboxes);
  for (int b = 0; b < e->nboxes; ++b) {
    if (sv[b] < 0) return fail(U1U1_ERR_INVALID_ARG, "steps[%d] must be >= 0", b);
    const u1u1_params& p = e->boxes[b]->p;
    if (e->boxes[b]->n + sv[b] > e->horizon)
      return fail(U1U1_ERR_STATE, "box %d would pass the step horizon %d", b, e->horizon);
    if (p.m != 0.0 && !(p.eta0 + (double)e->boxes[b]->n * p.deta > 0.0))
      return fail(U1U1_ERR_INVALID_ARG, "conformal time of box %d must stay > 0", b);
  }
  if (use_graph && mode == U1U1_ENS_UNBATCHED)
    return fail(U1U1_ERR_NOT_SUPPORTED,
                "the unbatched loop bakes each box's buffers and coefficients into its launches; run it without a graph");
  cudaStream_t st = (cudaStream_t)stream;
  if (de > 0) {
    // the overlap tolerance of each box's handle, as set when the run is enqueued
    bool changed = false;
    for (int b = 0; b < e->nboxes; ++b)
      if (e->hdet[b].tol != e->boxes[b]->overlap_tol) {
        e->hdet[b].tol = e->boxes[b]->overlap_tol;
        changed = true;
      }
    if (changed) {
      U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
      U1U1_CUDA_TRY(cudaMemcpyAsync(e->d_det, e->hdet.data(), sizeof(EnsDet) * e->nboxes, cudaMemcpyHostToDevice,
                                    st),
                    "detection table copy");
    }
  }
  int rc = sync_dyn(e, st);
  if (rc) return rc;
  Schedule* s = nullptr;
  rc = make_schedule(e, sv, &s, st);
  if (rc) return rc;
  DetPlan* P = nullptr;
  if (de > 0 && mode != U1U1_ENS_UNBATCHED) {
    rc = make_det_plan(e, sv, de, &P, st);
    if (rc) return rc;
  }
  auto run_on = [&](cudaStream_t q) { return P ? enqueue_det(e, s, P, mode, de, q) : enqueue(e, s, mode, de, q); };
  if (!use_graph) {
    rc = run_on(st);
    if (rc) return rc;
  } else {
    cudaGraphExec_t& g = P ? P->graph[mode] : s->graph[mode];
    if (!g) {
      // capture on a private stream so the caller's stream may be the legacy one
      cudaGraph_t graph = nullptr;
      U1U1_CUDA_TRY(cudaStreamBeginCapture(e->capture_stream, cudaStreamCaptureModeThreadLocal), "graph capture");
      int crc = run_on(e->capture_stream);
      cudaError_t ce = cudaStreamEndCapture(e->capture_stream, &graph);
      if (crc) {
        if (graph) cudaGraphDestroy(graph);
        return crc;
      }
      if (ce != cudaSuccess) return cuda_fail(ce, "graph capture");
      ce = cudaGraphInstantiate(&g, graph, 0);
      cudaGraphDestroy(graph);
      if (ce != cudaSuccess) {
        g = nullptr;
        return cuda_fail(ce, "graph instantiate");
      }
    }
    U1U1_CUDA_TRY(cudaGraphLaunch(g, st), "graph launch");
  }
  if (mode != U1U1_ENS_UNBATCHED) {
    for (int b = 0; b < e->nboxes; ++b) {
      u1u1_lattice* h = e->boxes[b];
      if (de > 0) {  // records appended to the box's ring by the batched detection
        const long long k1 = (de - h->n % de) % de;
        if (sv[b] > k1) h->rec_written += (sv[b] - 1 - k1) / de + 1;
      }
      h->n += sv[b];
      h->cur ^= (sv[b] & 1);
    }
  }
  for (int b = 0; b < e->nboxes; ++b) {
    e->shadow_n[b] = e->boxes[b]->n;
    e->shadow_cur[b] = e->boxes[b]->cur;
    e->shadow_rec[b] = e->boxes[b]->rec_written;
  }
  return U1U1_OK;
}

extern "C" int u1u1_ensemble_lattice(u1u1_ensemble* e, int box, u1u1_lattice** h) {
  if (!e || !h) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (box < 0 || box >= e->nboxes) return fail(U1U1_ERR_INVALID_ARG, "box %d out of range", box);
  *h = e->boxes[box];
  return U1U1_OK;
}

extern "C" int u1u1_ensemble_status(u1u1_ensemble* e, int* status, void* stream) {
  if (!e || !status) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  int w[2] = {0, 0};
  U1U1_CUDA_TRY(cudaMemcpyAsync(w, e->d_err, sizeof(w), cudaMemcpyDeviceToHost, (cudaStream_t)stream), "status");
  U1U1_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream), "stream synchronize");
  // a wait for a tensor copy that ran out counts as a timeout too
  const int v = w[0] != 0 ? w[0] : w[1];
  *status = v;
  if (v != 0) e->poisoned = 1;
  return U1U1_OK;
}

extern "C" int u1u1_ensemble_set_wait_limit(u1u1_ensemble* e, int64_t ns) {
  if (!e) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (ns < 1000) return fail(U1U1_ERR_INVALID_ARG, "wait limit must be >= 1000 ns");
  e->wait_limit_ns = ns;
  for (auto& kv : e->schedules)
    for (auto& g : kv.second->graph)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  e->det_plans.clear();
  return U1U1_OK;
}

extern "C" int u1u1_ensemble_inject_unreachable_wait(u1u1_ensemble* e, int enable) {
  if (!e) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  e->inject = enable ? 1 : 0;
  for (auto& kv : e->schedules)
    for (auto& g : kv.second->graph)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
  e->det_plans.clear();
  return U1U1_OK;
}

// ---------------------------------------------------------------------------
// autotuner: work-item z-chunk and schedule
// ---------------------------------------------------------------------------

extern "C" int u1u1_ensemble_get_tuning(const u1u1_ensemble* e, int* item_lz, int* persistent_tma) {
  if (!e) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (item_lz) *item_lz = e->item_lz;
  if (persistent_tma) *persistent_tma = e->persistent_tma;
  return U1U1_OK;
}

extern "C" int u1u1_ensemble_set_tuning(u1u1_ensemble* e, int item_lz, int persistent_tma, void* stream) {
  if (!e) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (item_lz != 16 && item_lz != 32 && item_lz != 64 && item_lz != 128)
    return fail(U1U1_ERR_INVALID_ARG, "item_lz must be 16, 32, 64 or 128 (got %d)", item_lz);
  if (persistent_tma != 0 && persistent_tma != 1) return fail(U1U1_ERR_INVALID_ARG, "persistent_tma must be 0 or 1");
  cudaStream_t st = (cudaStream_t)stream;
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  e->item_lz = item_lz;
  e->persistent_tma = persistent_tma;
  e->schedules.clear();  // tile grids and captured graphs change
  e->det_plans.clear();
  return e->precision == U1U1_FP64 ? build_tables<double>(e, st) : build_tables<float>(e, st);
}

extern "C" int u1u1_ensemble_autotune(u1u1_ensemble* e, int probe_steps, int* mode_out, int* item_lz_out,
                                      void* stream) {
  if (!e) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (probe_steps < 1) return fail(U1U1_ERR_INVALID_ARG, "probe_steps must be >= 1");
  if (e->poisoned) return fail(U1U1_ERR_STATE, "an earlier persistent run timed out");
  cudaStream_t st = (cudaStream_t)stream;
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  // save every box's state (current positions and momenta) and step index
  const int nb = e->nboxes;
  // (a box whose copy did not complete is left alone by the restore: nothing
  // has run on it yet)
  std::vector<void*> saves(nb, nullptr);
  std::vector<char> saved(nb, 0);
  std::vector<long long> n0(nb);
  std::vector<int> c0(nb);
  for (int b = 0; b < nb; ++b) {
    n0[b] = e->boxes[b]->n;
    c0[b] = e->boxes[b]->cur;
  }
  int rc = U1U1_OK;
  for (int b = 0; b < nb && !rc; ++b) {
    u1u1_lattice* h = e->boxes[b];
    const size_t bytes = h->V * h->esize;
    cudaError_t err = dev_alloc(&saves[b], bytes * U1U1_NFIELDS);
    if (err != cudaSuccess) {
      cudaGetLastError();
      rc = fail(U1U1_ERR_OUT_OF_MEMORY, "autotune needs a copy of the ensemble state");
      break;
    }
    for (int f = 0; f < U1U1_NFIELDS && !rc; ++f) {
      void* src = f < U1U1_NPOS ? h->pos[h->cur][f] : h->mom[f - U1U1_NPOS];
      err = cudaMemcpyAsync((char*)saves[b] + f * bytes, src, bytes, cudaMemcpyDeviceToDevice, st);
      if (err != cudaSuccess) rc = cuda_fail(err, "autotune save");
    }
    saved[b] = rc ? 0 : 1;
  }
  auto restore = [&]() -> int {
    for (int b = 0; b < nb; ++b) {
      if (!saved[b]) continue;
      u1u1_lattice* h = e->boxes[b];
      h->n = n0[b];
      h->cur = c0[b];
      const size_t bytes = h->V * h->esize;
      for (int f = 0; f < U1U1_NFIELDS; ++f) {
        void* dst = f < U1U1_NPOS ? h->pos[h->cur][f] : h->mom[f - U1U1_NPOS];
        U1U1_CUDA_TRY(cudaMemcpyAsync(dst, (char*)saves[b] + f * bytes, bytes, cudaMemcpyDeviceToDevice, st),
                      "autotune restore");
      }
    }
    return U1U1_OK;
  };
  const int lz0 = e->item_lz, tma0 = e->persistent_tma;
  const int lzs[] = {16, 32, 64, 128};
  // (mode, tensor copies in the persistent kernel)
  const int modes[][2] = {{U1U1_ENS_PERSISTENT, 1}, {U1U1_ENS_PERSISTENT, 0}, {U1U1_ENS_PER_STEP, 1}};
  float best = 1e30f;
  int best_mode = U1U1_ENS_PERSISTENT, best_lz = lz0, best_tma = tma0;
  std::vector<int> steps(nb);
  for (int b = 0; b < nb; ++b) steps[b] = (int)std::min<long long>(probe_steps, e->horizon - n0[b]);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (!rc && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess))
    rc = fail(U1U1_ERR_CUDA, "events");
  for (int lz : lzs) {
    if (rc) break;
    e->item_lz = lz;
    e->schedules.clear();
    e->det_plans.clear();
    rc = e->precision == U1U1_FP64 ? build_tables<double>(e, st) : build_tables<float>(e, st);
    for (const auto& mt : modes) {
      if (rc) break;
      const int mode = mt[0];
      e->persistent_tma = mt[1];
      e->schedules.clear();  // graphs captured with another choice
      float ms_best = 1e30f;
      // timed as graph replays, as the runs it tunes are meant to be made:
      // the first repetition captures the graph and warms up
      for (int rep = 0; rep < 2 && !rc; ++rep) {
        rc = restore();
        if (rc) break;
        cudaEventRecord(ev0, st);
        rc = u1u1_ensemble_run(e, steps.data(), 0, mode, 1, stream);
        cudaEventRecord(ev1, st);
        if (rc) break;
        if (cudaEventSynchronize(ev1) != cudaSuccess) {
          rc = fail(U1U1_ERR_CUDA, "autotune sync");
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        if (rep > 0) ms_best = ms;
      }
      int status = 0;
      if (!rc) rc = u1u1_ensemble_status(e, &status, stream);
      if (!rc && status != 0) rc = fail(status, "autotune run failed on the device");
      if (!rc && ms_best < best) {
        best = ms_best;
        best_mode = mode;
        best_lz = lz;
        best_tma = mt[1];
      }
    }
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  int rrc = restore();
  // the restore's copies read the saves on the stream: let them finish first
  if (cudaStreamSynchronize(st) != cudaSuccess && !rrc) rrc = cuda_fail(cudaGetLastError(), "stream synchronize");
  for (void* s : saves) dev_free(s);
  if (!rc) rc = rrc;
  e->item_lz = rc ? lz0 : best_lz;
  e->persistent_tma = rc ? tma0 : best_tma;
  e->schedules.clear();
  e->det_plans.clear();
  const int brc = e->precision == U1U1_FP64 ? build_tables<double>(e, st) : build_tables<float>(e, st);
  // re-sync the device step table with the restored host bookkeeping
  for (int b = 0; b < nb; ++b) e->shadow_n[b] = -1;  // forces the upload (records included)
  const int src = sync_dyn(e, st);
  if (rc) return rc;
  if (brc) return brc;
  if (src) return src;
  if (mode_out) *mode_out = best_mode;
  if (item_lz_out) *item_lz_out = best_lz;
  return U1U1_OK;
}
