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
    cudaFree(d_order);
    cudaFree(d_steps);
    cudaFree(d_box_prefix);
    cudaFree(d_step_off);
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
  std::map<std::vector<int>, std::unique_ptr<Schedule>> schedules;
  cudaStream_t capture_stream = nullptr;
};

namespace {

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
    e->ntiles[b] = ens_tile_grid(B.nx, B.ny, B.nz, &B.gx, &B.gy, &B.lz, &B.gz, e->item_lz);
    B.ntiles = e->ntiles[b];
    B.coef0 = (long long)b * e->horizon;
  }
  // tensor maps of each box's two position buffers (FP32; disabled plans
  // otherwise), read by the kernels from device memory
  std::vector<TmaPlan> hp((size_t)2 * nb);
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 2; ++k) {
      make_tma_plan<T>(hb[b].pos[k], hb[b].nx, hb[b].ny, hb[b].nz, &hp[2 * b + k]);
      hp[2 * b + k].status = e->d_err + 1;  // a copy timeout is this ensemble's, reported by its status
    }
  if (!e->d_tma) U1U1_CUDA_TRY(cudaMalloc((void**)&e->d_tma, sizeof(TmaPlan) * hp.size()), "ensemble tensor maps");
  U1U1_CUDA_TRY(cudaMemcpy(e->d_tma, hp.data(), sizeof(TmaPlan) * hp.size(), cudaMemcpyHostToDevice),
                "tensor map copy");
  for (int b = 0; b < nb; ++b)
    for (int k = 0; k < 2; ++k) hb[b].tma[k] = e->d_tma + 2 * b + k;
  if (!e->d_boxes) U1U1_CUDA_TRY(cudaMalloc(&e->d_boxes, sizeof(EnsBox<T>) * nb), "ensemble box table");
  U1U1_CUDA_TRY(cudaMemcpy(e->d_boxes, hb.data(), sizeof(EnsBox<T>) * nb, cudaMemcpyHostToDevice), "box table copy");
  if (e->d_coef) return U1U1_OK;  // a re-tiling keeps the coefficient table
  // per-step coefficients of every box up to the horizon
  std::vector<Coef<T>> hc((size_t)nb * e->horizon);
  for (int b = 0; b < nb; ++b)
    for (int n = 0; n < e->horizon; ++n) hc[(size_t)b * e->horizon + n] = make_coef<T>(&e->boxes[b]->p, n);
  U1U1_CUDA_TRY(cudaMalloc(&e->d_coef, sizeof(Coef<T>) * hc.size()), "coefficient table");
  U1U1_CUDA_TRY(cudaMemcpy(e->d_coef, hc.data(), sizeof(Coef<T>) * hc.size(), cudaMemcpyHostToDevice),
                "coefficient copy");
  (void)st;
  return U1U1_OK;
}

int make_schedule(u1u1_ensemble* e, const std::vector<int>& steps, Schedule** out) {
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
  U1U1_CUDA_TRY(cudaMalloc(&s->d_order, sizeof(int) * std::max(nb, 1)), "schedule");
  U1U1_CUDA_TRY(cudaMalloc(&s->d_steps, sizeof(int) * std::max(nb, 1)), "schedule");
  U1U1_CUDA_TRY(cudaMalloc(&s->d_box_prefix, sizeof(long long) * (nb + 1)), "schedule");
  U1U1_CUDA_TRY(cudaMalloc(&s->d_step_off, sizeof(long long) * (smax + 1)), "schedule");
  U1U1_CUDA_TRY(cudaMemcpy(s->d_order, order.data(), sizeof(int) * nb, cudaMemcpyHostToDevice), "schedule");
  U1U1_CUDA_TRY(cudaMemcpy(s->d_steps, steps.data(), sizeof(int) * nb, cudaMemcpyHostToDevice), "schedule");
  U1U1_CUDA_TRY(cudaMemcpy(s->d_box_prefix, prefix.data(), sizeof(long long) * (nb + 1), cudaMemcpyHostToDevice),
                "schedule");
  U1U1_CUDA_TRY(cudaMemcpy(s->d_step_off, off.data(), sizeof(long long) * (smax + 1), cudaMemcpyHostToDevice),
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

// Enqueue the device work of one run (no host bookkeeping).
template <typename T>
int enqueue_run(u1u1_ensemble* e, Schedule* s, int mode, cudaStream_t st) {
  const EnsBox<T>* boxes = (const EnsBox<T>*)e->d_boxes;
  const Coef<T>* coef = (const Coef<T>*)e->d_coef;
  cudaError_t err = cudaSuccess;
  if (mode == U1U1_ENS_PERSISTENT) {
    U1U1_CUDA_TRY(cudaMemsetAsync(e->d_ticket, 0, sizeof(unsigned long long), st), "ticket reset");
    U1U1_CUDA_TRY(cudaMemsetAsync(e->d_done, 0, sizeof(unsigned) * e->nboxes, st), "counter reset");
    U1U1_CUDA_TRY(cudaMemsetAsync(e->d_err, 0, sizeof(int), st), "status reset");
    err = launch_ens_persistent<T>(boxes, e->d_dyn, coef, s->sc, e->d_ticket, e->d_done, e->d_err, e->wait_limit_ns,
                                   e->inject, st);
    if (err != cudaSuccess) return cuda_fail(err, "persistent ensemble kernel");
  } else if (mode == U1U1_ENS_PER_STEP) {
    for (int k = 0; k < s->sc.smax; ++k) {
      err = launch_ens_step<T>(boxes, e->d_dyn, coef, s->sc, k, s->items_per_step[k], st);
      if (err != cudaSuccess) return cuda_fail(err, "ensemble step kernel");
    }
  } else {
    // the per-box handles advance their own host bookkeeping here
    for (int b = 0; b < e->nboxes; ++b) {
      const int rc = u1u1_step(e->boxes[b], s->steps[b], 0, st);
      if (rc) return rc;
    }
  }
  err = launch_ens_advance(e->d_dyn, s->d_steps, e->nboxes, st);
  if (err != cudaSuccess) return cuda_fail(err, "ensemble advance kernel");
  return U1U1_OK;
}

int enqueue(u1u1_ensemble* e, Schedule* s, int mode, cudaStream_t st) {
  return e->precision == U1U1_FP64 ? enqueue_run<double>(e, s, mode, st) : enqueue_run<float>(e, s, mode, st);
}

// bring the device step table in line with the per-box handles (a box may
// have been stepped or loaded through its borrowed handle)
int sync_dyn(u1u1_ensemble* e, cudaStream_t st) {
  bool stale = false;
  for (int b = 0; b < e->nboxes; ++b)
    if (e->boxes[b]->n != e->shadow_n[b] || e->boxes[b]->cur != e->shadow_cur[b]) stale = true;
  if (!stale) return U1U1_OK;
  std::vector<EnsDyn> hd(e->nboxes);
  for (int b = 0; b < e->nboxes; ++b) {
    hd[b].n = e->boxes[b]->n;
    hd[b].cur = e->boxes[b]->cur;
    hd[b].pad = 0;
    e->shadow_n[b] = hd[b].n;
    e->shadow_cur[b] = hd[b].cur;
  }
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  U1U1_CUDA_TRY(cudaMemcpy(e->d_dyn, hd.data(), sizeof(EnsDyn) * e->nboxes, cudaMemcpyHostToDevice), "step table");
  return U1U1_OK;
}

}  // namespace

extern "C" void u1u1_ensemble_destroy(u1u1_ensemble* e) {
  if (!e) return;
  e->schedules.clear();
  for (u1u1_lattice* h : e->boxes) u1u1_destroy(h);
  cudaFree(e->d_boxes);
  cudaFree(e->d_tma);
  cudaFree(e->d_dyn);
  cudaFree(e->d_coef);
  cudaFree(e->d_ticket);
  cudaFree(e->d_done);
  cudaFree(e->d_err);
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
  for (int b = 0; b < nboxes; ++b) {
    u1u1_lattice* h = nullptr;
    int rc = u1u1_init_lattice(&per_box[b], &buffers[b], stream, &h);
    if (rc) {
      u1u1_ensemble_destroy(e);
      return rc;
    }
    h->kernel = U1U1_KERNEL_TILED;
    e->boxes.push_back(h);
  }
  int rc = U1U1_OK;
  cudaError_t err = cudaSuccess;
  if (err == cudaSuccess) err = cudaMalloc((void**)&e->d_err, 2 * sizeof(int));
  if (err == cudaSuccess) err = cudaMemset(e->d_err, 0, 2 * sizeof(int));
  if (err != cudaSuccess) rc = cuda_fail(err, "ensemble allocation");
  if (!rc) rc = e->precision == U1U1_FP64 ? build_tables<double>(e, st) : build_tables<float>(e, st);
  if (!rc) {
    if (err == cudaSuccess) err = cudaMalloc((void**)&e->d_dyn, sizeof(EnsDyn) * nboxes);
    if (err == cudaSuccess) err = cudaMalloc((void**)&e->d_ticket, sizeof(unsigned long long));
    if (err == cudaSuccess) err = cudaMalloc((void**)&e->d_done, sizeof(unsigned) * nboxes);
    if (err == cudaSuccess) err = cudaMemset(e->d_dyn, 0, sizeof(EnsDyn) * nboxes);
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

extern "C" int u1u1_ensemble_run(u1u1_ensemble* e, const int* steps, int mode, int use_graph, void* stream) {
  if (!e || !steps) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (mode < U1U1_ENS_PERSISTENT || mode > U1U1_ENS_UNBATCHED) return fail(U1U1_ERR_INVALID_ARG, "unknown mode %d", mode);
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
  int rc = sync_dyn(e, st);
  if (rc) return rc;
  Schedule* s = nullptr;
  rc = make_schedule(e, sv, &s);
  if (rc) return rc;
  if (!use_graph) {
    rc = enqueue(e, s, mode, st);
    if (rc) return rc;
  } else {
    cudaGraphExec_t& g = s->graph[mode];
    if (!g) {
      // capture on a private stream so the caller's stream may be the legacy one
      cudaGraph_t graph = nullptr;
      U1U1_CUDA_TRY(cudaStreamBeginCapture(e->capture_stream, cudaStreamCaptureModeThreadLocal), "graph capture");
      int crc = enqueue(e, s, mode, e->capture_stream);
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
      e->boxes[b]->n += sv[b];
      e->boxes[b]->cur ^= (sv[b] & 1);
    }
  }
  for (int b = 0; b < e->nboxes; ++b) {
    e->shadow_n[b] = e->boxes[b]->n;
    e->shadow_cur[b] = e->boxes[b]->cur;
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
  return U1U1_OK;
}

// ---------------------------------------------------------------------------
// autotuner: work-item z-chunk and schedule
// ---------------------------------------------------------------------------

extern "C" int u1u1_ensemble_autotune(u1u1_ensemble* e, int probe_steps, int* mode_out, int* item_lz_out,
                                      void* stream) {
  if (!e) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (probe_steps < 1) return fail(U1U1_ERR_INVALID_ARG, "probe_steps must be >= 1");
  if (e->poisoned) return fail(U1U1_ERR_STATE, "an earlier persistent run timed out");
  cudaStream_t st = (cudaStream_t)stream;
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  // save every box's state (current positions and momenta) and step index
  const int nb = e->nboxes;
  std::vector<void*> saves(nb, nullptr);
  std::vector<long long> n0(nb);
  std::vector<int> c0(nb);
  int rc = U1U1_OK;
  for (int b = 0; b < nb && !rc; ++b) {
    u1u1_lattice* h = e->boxes[b];
    n0[b] = h->n;
    c0[b] = h->cur;
    const size_t bytes = h->V * h->esize;
    cudaError_t err = cudaMalloc(&saves[b], bytes * U1U1_NFIELDS);
    if (err != cudaSuccess) {
      cudaGetLastError();
      rc = fail(U1U1_ERR_OUT_OF_MEMORY, "autotune needs a copy of the ensemble state");
      break;
    }
    for (int f = 0; f < U1U1_NFIELDS && !rc; ++f) {
      void* src = f < U1U1_NPOS ? h->pos[h->cur][f] : h->mom[f - U1U1_NPOS];
      err = cudaMemcpy((char*)saves[b] + f * bytes, src, bytes, cudaMemcpyDeviceToDevice);
      if (err != cudaSuccess) rc = cuda_fail(err, "autotune save");
    }
  }
  auto restore = [&]() -> int {
    for (int b = 0; b < nb; ++b) {
      u1u1_lattice* h = e->boxes[b];
      h->n = n0[b];
      h->cur = c0[b];
      const size_t bytes = h->V * h->esize;
      for (int f = 0; f < U1U1_NFIELDS; ++f) {
        void* dst = f < U1U1_NPOS ? h->pos[h->cur][f] : h->mom[f - U1U1_NPOS];
        U1U1_CUDA_TRY(cudaMemcpy(dst, (char*)saves[b] + f * bytes, bytes, cudaMemcpyDeviceToDevice), "autotune restore");
      }
    }
    return U1U1_OK;
  };
  const int lz0 = e->item_lz;
  const int lzs[] = {16, 32, 64, 128};
  const int modes[] = {U1U1_ENS_PERSISTENT, U1U1_ENS_PER_STEP};
  float best = 1e30f;
  int best_mode = U1U1_ENS_PERSISTENT, best_lz = lz0;
  std::vector<int> steps(nb);
  for (int b = 0; b < nb; ++b) steps[b] = (int)std::min<long long>(probe_steps, e->horizon - n0[b]);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (!rc && (cudaEventCreate(&ev0) != cudaSuccess || cudaEventCreate(&ev1) != cudaSuccess))
    rc = fail(U1U1_ERR_CUDA, "events");
  for (int lz : lzs) {
    if (rc) break;
    e->item_lz = lz;
    e->schedules.clear();
    rc = e->precision == U1U1_FP64 ? build_tables<double>(e, st) : build_tables<float>(e, st);
    for (int mode : modes) {
      if (rc) break;
      float ms_best = 1e30f;
      for (int rep = 0; rep < 2 && !rc; ++rep) {  // the first repetition also warms up
        rc = restore();
        if (rc) break;
        cudaEventRecord(ev0, st);
        rc = u1u1_ensemble_run(e, steps.data(), mode, 0, stream);
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
      }
    }
  }
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  const int rrc = restore();
  for (void* s : saves) cudaFree(s);
  if (!rc) rc = rrc;
  e->item_lz = rc ? lz0 : best_lz;
  e->schedules.clear();
  const int brc = e->precision == U1U1_FP64 ? build_tables<double>(e, st) : build_tables<float>(e, st);
  // re-sync the device step table with the restored host bookkeeping
  for (int b = 0; b < nb; ++b) e->shadow_n[b] = -1;
  const int src = sync_dyn(e, st);
  if (rc) return rc;
  if (brc) return brc;
  if (src) return src;
  if (mode_out) *mode_out = best_mode;
  if (item_lz_out) *item_lz_out = best_lz;
  return U1U1_OK;
}
