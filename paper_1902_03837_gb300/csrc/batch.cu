// Batched execution of many independent chi0 / eps~^-1 problems.
//
// The paper distributes the response function over q points and over the
// k, c, v transition indices (Parallelism section, linear response) and
// notes the load imbalance of q-point distribution "since the number of
// possible transitions varies".  On one GPU the independent problems (a
// system at one q point each, with its own grid sizes, response set,
// frequency count and ragged transition count) are run as one unit:
//
//   1. every problem's host set-up runs once (chi0_batch_create).  The
//      problems of one system (one context at several q indices) share its
//      coefficients and its mixed grids, computed once per system;
//   2. the oscillator strengths of all problems run in ONE persistent launch
//      over a device task table: blocks take the next (problem, k-pair, n,
//      m-chunk) work item from a counter, so uneven problems balance;
//   3. the remaining kernels of every problem (weights, operand split,
//      contraction, reduction, Dyson) go on a few helper streams.  Problems
//      are assigned to the streams longest first, each to the stream with the
//      least estimated work so far; the problems of one stream run one after
//      the other and share one set of scratch buffers (operands, partials,
//      chi0, Dyson panels), sized for the largest of them;
//   4. all of it is captured once into a CUDA graph and replayed by every
//      chi0_batch_run.
// Autotuning on the batch's own data at creation: the tile width of the
// persistent rho launch (m bands per block), remembered per geometry for the
// rest of the process, and the transition split of every problem's
// contraction (the planned split, half and twice as many, timed).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ctx.cuh"

struct chi0_batch {
  std::vector<chi0_ctx*> items;  // one problem context per (context, q index) pair
  std::vector<chi0_ctx*> bases;  // the distinct caller contexts whose coefficients the problems read
  cudaEvent_t ev_up = nullptr;   // their pending coefficient copies, ahead of a replay
  std::vector<int> iqs;
  std::vector<void*> outs;       // eps~^-1 per problem (NULL: no Dyson step)
  std::vector<void*> chi_outs;   // chi0 per problem (NULL: not copied out)
  std::vector<int> stream_of;    // helper stream of each problem
  std::vector<int> order;        // problems in launch order (per stream: longest first)
  std::vector<double> cost;      // estimated device time of each problem (model units)
  std::vector<std::vector<DevBuf>> arena;  // [helper stream][scratch slot] shared buffers
  float tuned_split_ms = 0.f;    // summed best contraction time of the split tuning
  std::vector<cudaStream_t> helpers;
  std::vector<cudaEvent_t> evs;  // fork/join events
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  bool fp64 = false;
  DevBuf tasks, counter;
  int ntasks = 0;
  int64_t total_blocks = 0;
  int jm = 4;
  size_t smem = 0;
  int nsm = 148;
  cudaStream_t last_stream = nullptr;  // stream of the last replay
  bool replayed = false;
  std::string err;
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;  // geometry key -> chosen m bands per block

template <typename T, typename TOUT>
chi0_status build_tasks(chi0_batch* b, int jm_max, std::vector<chi0::RhoTask<T, TOUT>>& tasks,
                        size_t* smem, int64_t* total) {
  tasks.clear();
  *smem = 0;
  *total = 0;
  for (chi0_ctx* c : b->items) {
    if (c->nt == 0) continue;
    chi0::RhoTask<T, TOUT> tk;
    size_t sm = 0;
    int64_t nb = 0;
    cudaError_t e = chi0::rho_task_make<T, TOUT>(
        c->geom, (const typename chi0::C2<T>::t*)c->d_U.p, (const int32_t*)c->d_kq.p,
        (const int32_t*)c->d_g0.p, (const int32_t*)c->d_gresp.p, (const int32_t*)c->d_gperm.p,
        (const typename chi0::C2<T>::t*)c->d_tw1.p, (const typename chi0::C2<T>::t*)c->d_tw2.p,
        (TOUT*)c->d_R.p, jm_max, &tk, &sm, &nb);
    if (e != cudaSuccess) return CHI0_EUNSUPPORTED;
    tk.block0 = *total;
    *total += nb;
    *smem = std::max(*smem, sm);
    tasks.push_back(tk);
  }
  if (*smem > 227 * 1024) return CHI0_EUNSUPPORTED;
  return CHI0_OK;
}

template <typename T, typename TOUT>
chi0_status upload_tasks(chi0_batch* b, int jm) {
  std::vector<chi0::RhoTask<T, TOUT>> tasks;
  size_t smem = 0;
  int64_t total = 0;
  chi0_status s = build_tasks<T, TOUT>(b, jm, tasks, &smem, &total);
  if (s != CHI0_OK) return s;
  chi0_ctx* c0 = b->items[0];
  if ((s = chi0::ctx_ensure(c0, b->tasks, tasks.size() * sizeof(tasks[0]) + 16, "batch tasks")) != CHI0_OK) return s;
  if ((s = chi0::ctx_ensure(c0, b->counter, 16, "batch counter")) != CHI0_OK) return s;
  if (!tasks.empty() &&
      cudaMemcpy(b->tasks.p, tasks.data(), tasks.size() * sizeof(tasks[0]), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  b->ntasks = (int)tasks.size();
  b->total_blocks = total;
  b->jm = jm;
  b->smem = smem;
  return CHI0_OK;
}

template <typename T, typename TOUT>
cudaError_t launch_tasks(chi0_batch* b, cudaStream_t st) {
  return chi0::launch_rho_batch<T, TOUT>((const chi0::RhoTask<T, TOUT>*)b->tasks.p, b->ntasks,
                                         b->total_blocks, b->jm, b->smem,
                                         (unsigned long long*)b->counter.p, b->nsm, st);
}

cudaError_t launch_batched_rho(chi0_batch* b, cudaStream_t st) {
  return b->fp64 ? launch_tasks<double, double2>(b, st) : launch_tasks<float, float2>(b, st);
}

chi0_status set_tasks(chi0_batch* b, int jm) {
  return b->fp64 ? upload_tasks<double, double2>(b, jm) : upload_tasks<float, float2>(b, jm);
}

std::string tune_key(const chi0_batch* b) {
  std::string k = b->fp64 ? "f64" : "f32";
  for (const chi0_ctx* c : b->items) {
    const RhoGeom& g = c->geom;
    char buf[160];
    snprintf(buf, sizeof(buf), "|%d,%d,%d,%d,%d,%d,%d,%d,%d,%d,%d", g.N1, g.N2, g.NZ, g.HX, g.HY, g.HZ,
             g.ng, g.nk, g.Nn, g.Nm, g.nb);
    k += buf;
  }
  return k;
}

// time the persistent rho launch for every admissible width and keep the best
chi0_status autotune(chi0_batch* b, cudaStream_t st) {
  const std::string key = tune_key(b);
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return set_tasks(b, it->second);
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  int best = -1;
  float best_ms = 1e30f;
  for (int jm : {4, 2, 1}) {
    if (set_tasks(b, jm) != CHI0_OK) continue;
    if (launch_batched_rho(b, st) != cudaSuccess) {  // warm-up
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(e0, st);
    cudaError_t le = launch_batched_rho(b, st);
    cudaEventRecord(e1, st);
    float ms = 0.f;
    if (le != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = jm;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 0) return CHI0_EUNSUPPORTED;
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = best;
  }
  return set_tasks(b, best);
}

void destroy_batch(chi0_batch* b) {
  if (!b) return;
  if (b->replayed) cudaStreamSynchronize(b->last_stream);
  for (cudaStream_t s : b->helpers) cudaStreamSynchronize(s);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->evs) cudaEventDestroy(e);
  if (b->ev_up) cudaEventDestroy(b->ev_up);
  if (b->tasks.p) cudaFree(b->tasks.p);
  if (b->counter.p) cudaFree(b->counter.p);
  b->tasks = b->counter = DevBuf{};
  // the problem contexts first (their shared buffers are only borrowed), then
  // the shared scratch
  for (chi0_ctx* c : b->items) chi0_destroy(c);
  for (auto& slots : b->arena)
    for (DevBuf& d : slots)
      if (d.p) cudaFree(d.p);
  for (cudaStream_t s : b->helpers) cudaStreamDestroy(s);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  delete b;
}

// Estimated device time of a problem (seconds): the tensor-core contraction
// (3 BF16 products over the lower-triangle tiles, at about 1.1 PFLOP/s
// issued) or the FP64 one, plus the FP64 Dyson step (about 4 N_G^3 complex
// flops executed per frequency at about 1 TFLOP/s).
double problem_cost(const chi0_ctx* c, bool with_dyson) {
  const double ng = c->cfg.ng, nw = c->cfg.nw, nt = (double)c->nt;
  const double t_con = c->fp64 ? 4.0 * ng * (ng + 1) * nt * nw / 0.8e12
                               : 3.0 * 4.0 * ng * ng * 1.2 * nt * nw / 1.1e15;
  const double t_dys = with_dyson ? 4.0 * ng * ng * ng * nw / 1.0e12 : 0.0;
  return t_con + t_dys + 5e-5;
}

}  // namespace

extern "C" {

chi0_status chi0_batch_create(chi0_ctx* const* ctxs, const int* iqs, void* const* chi_out, void* const* eps_out,
                              int n, int nstreams, chi0_batch** out) {
  if (!out) return CHI0_EINVAL;
  *out = nullptr;
  if (!ctxs || !iqs || n < 1 || nstreams < 1 || nstreams > 32) return CHI0_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return CHI0_EINVAL;
    if (iqs[i] < 0 || iqs[i] >= ctxs[i]->cfg.nq) return CHI0_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] && iqs[j] == iqs[i]) return CHI0_EINVAL;  // each (context, q) once
    if (ctxs[i]->fp64 != ctxs[0]->fp64) return CHI0_EUNSUPPORTED;
    if (!(chi_out && chi_out[i]) && !(eps_out && eps_out[i])) return CHI0_EINVAL;  // nothing to return
  }
  chi0_batch* b = new (std::nothrow) chi0_batch();
  if (!b) return CHI0_ENOMEM;
  b->fp64 = ctxs[0]->fp64;
  b->iqs.assign(iqs, iqs + n);
  b->outs.assign(n, nullptr);
  b->chi_outs.assign(n, nullptr);
  if (eps_out) b->outs.assign(eps_out, eps_out + n);
  if (chi_out) b->chi_outs.assign(chi_out, chi_out + n);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
  }
  chi0_status s = CHI0_OK;
  // one problem context per (context, q index), sharing the context's inputs
  for (int i = 0; i < n && s == CHI0_OK; ++i) {
    for (int k = 0; k < ctxs[i]->nk; ++k)
      if (!ctxs[i]->wf_set[k] || !ctxs[i]->energies_set) s = CHI0_ESTATE;
    chi0_ctx* c = s == CHI0_OK ? chi0::make_problem_ctx(ctxs[i]) : nullptr;
    if (s == CHI0_OK && !c) s = CHI0_ENOMEM;
    if (s == CHI0_OK && std::find(b->bases.begin(), b->bases.end(), ctxs[i]) == b->bases.end()) {
      b->bases.push_back(ctxs[i]);
      // coefficient copies still on the caller context's upload stream land
      // before the planning and tuning below read the coefficients
      if (ctxs[i]->s_up && cudaStreamSynchronize(ctxs[i]->s_up) != cudaSuccess) s = CHI0_ECUDA;
    }
    if (c) {
      c->group_cap = 4;
      b->items.push_back(c);
    }
  }
  // plan rho; the first problem of a system with transitions owns the mixed
  // grids, the system's other problems borrow them
  std::vector<chi0_ctx*> owner(n, nullptr);
  for (int i = 0; i < n && s == CHI0_OK; ++i) {
    chi0_ctx* c = b->items[i];
    chi0_ctx* own = nullptr;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i] && owner[j]) own = owner[j];
    if (own) {
      c->d_U = DevBuf{own->d_U.p, own->d_U.bytes, true};
      c->grid_shared = true;
    }
    if ((s = chi0::plan_rho(c, b->iqs[i])) != CHI0_OK) break;
    owner[i] = own ? own : (c->nt > 0 ? c : nullptr);
    if (!own) s = chi0::launch_rho(c, false);   // the mixed grids (used by the tuning below)
  }
  // sizing pass: plan the rest of each problem with its own scratch, note the
  // sizes and free them again (one problem's scratch at a time)
  std::vector<std::vector<size_t>> need(n);
  for (int i = 0; i < n && s == CHI0_OK; ++i) {
    chi0_ctx* c = b->items[i];
    if ((s = chi0::plan_chi0(c, b->iqs[i])) != CHI0_OK) break;
    if (b->outs[i] && (s = chi0::plan_eps(c, b->iqs[i], (double2*)b->outs[i])) != CHI0_OK) break;
    if (cudaStreamSynchronize(c->st) != cudaSuccess) s = CHI0_ECUDA;
    for (DevBuf* d : chi0::scratch_slots(c)) {
      need[i].push_back(d->bytes);
      if (d->p && !d->borrowed) cudaFree(d->p);
      *d = DevBuf{};
    }
    b->cost.push_back(problem_cost(c, b->outs[i] != nullptr));
  }
  // longest first, each to the helper stream with the least work so far
  const int ns = std::min(nstreams, n);
  if (s == CHI0_OK) {
    b->order.resize(n);
    for (int i = 0; i < n; ++i) b->order[i] = i;
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
    std::vector<double> load(ns, 0.0);
    b->stream_of.assign(n, 0);
    for (int i : b->order) {
      const int h = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      b->stream_of[i] = h;
      load[h] += b->cost[i];
    }
    // shared scratch of each stream: every slot as large as its largest user
    const size_t nslot = need[0].size();
    b->arena.assign(ns, std::vector<DevBuf>(nslot));
    for (int h = 0; h < ns && s == CHI0_OK; ++h)
      for (size_t k = 0; k < nslot && s == CHI0_OK; ++k) {
        size_t mx = 0;
        for (int i = 0; i < n; ++i)
          if (b->stream_of[i] == h) mx = std::max(mx, need[i][k]);
        if (mx == 0) continue;
        if (cudaMalloc(&b->arena[h][k].p, mx) != cudaSuccess) {
          cudaGetLastError();
          s = CHI0_ENOMEM;
        } else {
          b->arena[h][k].bytes = mx;
        }
      }
    // re-plan every problem on its stream's shared scratch (no allocation)
    for (int i = 0; i < n && s == CHI0_OK; ++i) {
      chi0_ctx* c = b->items[i];
      std::vector<DevBuf*> slots = chi0::scratch_slots(c);
      for (size_t k = 0; k < nslot; ++k) {
        const DevBuf& a = b->arena[b->stream_of[i]][k];
        *slots[k] = a.p ? DevBuf{a.p, a.bytes, true} : DevBuf{};
      }
      ++c->plan_epoch;
      if ((s = chi0::plan_rho(c, b->iqs[i])) != CHI0_OK) break;
      if ((s = chi0::plan_chi0(c, b->iqs[i])) != CHI0_OK) break;
      if (b->outs[i] && (s = chi0::plan_eps(c, b->iqs[i], (double2*)b->outs[i])) != CHI0_OK) break;
    }
  }
  for (chi0_ctx* c : b->items)
    if (s == CHI0_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = CHI0_ECUDA;
  cudaStream_t st0 = b->items.empty() ? nullptr : b->items[0]->st;
  if (s == CHI0_OK) s = autotune(b, st0);   // also leaves every problem's rho computed
  if (s == CHI0_OK && cudaStreamSynchronize(st0) != cudaSuccess) s = CHI0_ECUDA;
  // the transition split of every contraction, on the problem's own data
  for (int i = 0; i < n && s == CHI0_OK && !b->fp64; ++i) {
    chi0_ctx* c = b->items[i];
    if (c->nt == 0) continue;
    if ((s = chi0::launch_weights_stage(c)) != CHI0_OK) break;
    float ms = 0.f;
    if ((s = chi0::tc_tune_split(c, &ms)) != CHI0_OK) break;
    if (ms < 1e29f) b->tuned_split_ms += ms;
  }
  for (int k = 0; k < ns && s == CHI0_OK; ++k) {
    cudaStream_t hs = nullptr;
    if (cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking) != cudaSuccess) s = CHI0_ECUDA;
    else b->helpers.push_back(hs);
  }
  for (int k = 0; k < 2 * ns + 2 && s == CHI0_OK; ++k) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) s = CHI0_ECUDA;
    else b->evs.push_back(e);
  }
  for (chi0_ctx* c : b->items)
    if (s == CHI0_OK && (cudaStreamSynchronize(c->st) != cudaSuccess || chi0_synchronize(c) != CHI0_OK))
      s = CHI0_ECUDA;
  if (s != CHI0_OK) {
    cudaGetLastError();
    // report the failing problem's message on the first context
    for (chi0_ctx* c : b->items)
      if (!c->err.empty()) {
        ctxs[0]->err = "batch problem: " + c->err;
        break;
      }
    destroy_batch(b);
    return s;
  }
  *out = b;
  return CHI0_OK;
}

chi0_status chi0_batch_run(chi0_batch* b, void* stream) {
  if (!b) return CHI0_EINVAL;
  if (!b->exec) {
    // the work is recorded on an internal stream (the caller's stream may be
    // the legacy default stream, which cannot be captured); the graph is then
    // launched on the caller's stream
    if (!b->capture_stream &&
        cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      return CHI0_ECUDA;
    }
    cudaStream_t st = b->capture_stream;
    const int ns = (int)b->helpers.size();
    std::vector<cudaStream_t> saved;
    for (chi0_ctx* c : b->items) saved.push_back(c->st);
    auto restore = [&]() {
      for (size_t i = 0; i < b->items.size(); ++i) {
        b->items[i]->st = saved[i];
        b->items[i]->capturing = false;
      }
    };
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      return CHI0_ECUDA;
    }
    chi0_status s = CHI0_OK;
    auto fork = [&](cudaEvent_t e) {
      cudaEventRecord(e, st);
      for (cudaStream_t h : b->helpers) cudaStreamWaitEvent(h, e, 0);
    };
    auto join = [&](int first_event) {
      for (int k = 0; k < ns; ++k) {
        cudaEventRecord(b->evs[first_event + k], b->helpers[k]);
        cudaStreamWaitEvent(st, b->evs[first_event + k], 0);
      }
    };
    // the mixed grids of every system (its grid owner), spread over the streams
    fork(b->evs[2 * ns]);
    int nown = 0;
    for (size_t i = 0; i < b->items.size() && s == CHI0_OK; ++i) {
      chi0_ctx* c = b->items[i];
      c->capturing = true;
      if (c->grid_shared || c->nt == 0) continue;
      c->st = b->helpers[nown++ % ns];
      s = chi0::launch_rho(c, false);
    }
    join(0);
    if (s == CHI0_OK && launch_batched_rho(b, st) != cudaSuccess) s = CHI0_ECUDA;
    if (!b->items.empty()) b->items[0]->launches += 1;
    // the rest of every problem on its stream, in the planned order
    fork(b->evs[2 * ns + 1]);
    for (int i : b->order) {
      if (s != CHI0_OK) break;
      chi0_ctx* c = b->items[i];
      c->st = b->helpers[b->stream_of[i]];
      c->rho_iq = c->plan_rho_iq;
      s = b->outs[i] ? chi0::launch_chi0_eps(c) : chi0::launch_chi0(c);
      if (s == CHI0_OK && b->chi_outs[i] &&
          cudaMemcpyAsync(b->chi_outs[i], c->d_chi.p, (size_t)c->cfg.ng * c->cfg.ng * c->cfg.nw * 16,
                          cudaMemcpyDeviceToDevice, c->st) != cudaSuccess)
        s = CHI0_ECUDA;
    }
    join(ns);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    restore();
    if (s != CHI0_OK || ce != cudaSuccess) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      return s != CHI0_OK ? s : CHI0_ECUDA;
    }
    b->graph = g;
    // node priorities let the overlapped Dyson step go ahead of the contraction
    if (cudaGraphInstantiateWithFlags(&b->exec, g, cudaGraphInstantiateFlagUseNodePriority) != cudaSuccess) {
      cudaGetLastError();
      return CHI0_ECUDA;
    }
  }
  // the replay reads the callers' coefficients: it follows their copies on
  // the upload streams, and their next copies wait for it (ev_wf_done)
  for (chi0_ctx* base : b->bases) {
    if (!base->s_up) continue;
    if ((!b->ev_up && cudaEventCreateWithFlags(&b->ev_up, cudaEventDisableTiming) != cudaSuccess) ||
        cudaEventRecord(b->ev_up, base->s_up) != cudaSuccess ||
        cudaStreamWaitEvent((cudaStream_t)stream, b->ev_up, 0) != cudaSuccess) {
      cudaGetLastError();
      return CHI0_ECUDA;
    }
  }
  if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  for (chi0_ctx* base : b->bases)
    if ((!base->ev_wf_done && cudaEventCreateWithFlags(&base->ev_wf_done, cudaEventDisableTiming) != cudaSuccess) ||
        cudaEventRecord(base->ev_wf_done, (cudaStream_t)stream) != cudaSuccess) {
      cudaGetLastError();
      return CHI0_ECUDA;
    }
  b->last_stream = (cudaStream_t)stream;
  b->replayed = true;
  return CHI0_OK;
}

int chi0_batch_rho_width(const chi0_batch* b) { return b ? b->jm : 0; }

chi0_status chi0_batch_info(const chi0_batch* b, int* stream_of, double* tuned_split_ms) {
  if (!b) return CHI0_EINVAL;
  if (stream_of)
    for (size_t i = 0; i < b->stream_of.size(); ++i) stream_of[i] = b->stream_of[i];
  if (tuned_split_ms) *tuned_split_ms = b->tuned_split_ms;
  return CHI0_OK;
}

chi0_status chi0_batch_synchronize(chi0_batch* b) {
  if (!b) return CHI0_EINVAL;
  chi0_status s = CHI0_OK;
  if (b->replayed && cudaStreamSynchronize(b->last_stream) != cudaSuccess) {
    cudaGetLastError();
    s = CHI0_ECUDA;
  }
  for (chi0_ctx* c : b->items) {
    const chi0_status e = chi0_synchronize(c);
    if (e != CHI0_OK && s == CHI0_OK) s = e;
  }
  return s;
}

void chi0_batch_destroy(chi0_batch* b) { destroy_batch(b); }

}  // extern "C"
