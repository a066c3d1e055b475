// Batched execution of many independent chi0 / eps~^-1 problems.
//
// The paper distributes the response function over q points and over the
// k, c, v transition indices (Parallelism section, linear response) and
// notes the load imbalance of q-point distribution "since the number of
// possible transitions varies".  On one GPU the independent problems (a
// system at one q point each, with its own grid sizes, response set,
// frequency count and ragged transition count) are run as one unit:
//
//   1. every problem's host set-up runs once (chi0_batch_create);
//   2. the oscillator strengths of all problems run in ONE persistent launch
//      over a device task table: blocks take the next (problem, k-pair, n,
//      m-chunk) work item from a counter, so uneven problems balance;
//   3. the remaining kernels of every problem (weights, contraction,
//      reduction, Dyson) go on a few helper streams so that small problems
//      overlap;
//   4. all of it is captured once into a CUDA graph and replayed by every
//      chi0_batch_run.
// The tile width of the persistent rho launch (m bands per block) is chosen
// by timing the candidates on the batch's own data at creation, and the
// choice is remembered per geometry for the rest of the process.
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
  std::vector<chi0_ctx*> items;
  std::vector<int> iqs;
  std::vector<void*> outs;
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
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaEvent_t e : b->evs) cudaEventDestroy(e);
  for (cudaStream_t s : b->helpers) cudaStreamDestroy(s);
  if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  if (b->tasks.p) cudaFree(b->tasks.p);
  if (b->counter.p) cudaFree(b->counter.p);
  delete b;
}

}  // namespace

extern "C" {

chi0_status chi0_batch_create(chi0_ctx* const* ctxs, const int* iqs, void* const* eps_out, int n,
                              int nstreams, chi0_batch** out) {
  if (!out) return CHI0_EINVAL;
  *out = nullptr;
  if (!ctxs || !iqs || n < 1 || nstreams < 1 || nstreams > 32) return CHI0_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return CHI0_EINVAL;
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return CHI0_EINVAL;  // one problem per context
    if (ctxs[i]->fp64 != ctxs[0]->fp64) return CHI0_EUNSUPPORTED;
  }
  chi0_batch* b = new (std::nothrow) chi0_batch();
  if (!b) return CHI0_ENOMEM;
  b->fp64 = ctxs[0]->fp64;
  b->items.assign(ctxs, ctxs + n);
  b->iqs.assign(iqs, iqs + n);
  b->outs.assign(n, nullptr);
  if (eps_out) b->outs.assign(eps_out, eps_out + n);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
  }
  chi0_status s = CHI0_OK;
  for (int i = 0; i < n && s == CHI0_OK; ++i) {
    chi0_ctx* c = b->items[i];
    if ((s = chi0::plan_rho(c, b->iqs[i])) != CHI0_OK) break;
    // the mixed grids are needed to tune and to plan the contraction
    if ((s = chi0::launch_rho(c, false)) != CHI0_OK) break;
    if ((s = chi0::plan_chi0(c, b->iqs[i])) != CHI0_OK) break;
    if (b->outs[i]) s = chi0::plan_eps(c, b->iqs[i], (double2*)b->outs[i]);
  }
  cudaStream_t st0 = b->items[0]->st;
  for (chi0_ctx* c : b->items)
    if (s == CHI0_OK && cudaStreamSynchronize(c->st) != cudaSuccess) s = CHI0_ECUDA;
  if (s == CHI0_OK) s = autotune(b, st0);
  for (int k = 0; k < nstreams && s == CHI0_OK; ++k) {
    cudaStream_t hs = nullptr;
    if (cudaStreamCreateWithFlags(&hs, cudaStreamNonBlocking) != cudaSuccess) s = CHI0_ECUDA;
    else b->helpers.push_back(hs);
  }
  for (int k = 0; k < 2 * nstreams + 2 && s == CHI0_OK; ++k) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) s = CHI0_ECUDA;
    else b->evs.push_back(e);
  }
  if (s == CHI0_OK && cudaStreamSynchronize(st0) != cudaSuccess) s = CHI0_ECUDA;
  if (s != CHI0_OK) {
    cudaGetLastError();
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
    // capture: fork to the helper streams, per-problem kernels, batched rho, join
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
    fork(b->evs[2 * ns]);
    for (size_t i = 0; i < b->items.size() && s == CHI0_OK; ++i) {
      chi0_ctx* c = b->items[i];
      c->st = b->helpers[i % ns];
      c->capturing = true;
      s = chi0::launch_rho(c, false);
    }
    join(0);
    if (s == CHI0_OK && launch_batched_rho(b, st) != cudaSuccess) s = CHI0_ECUDA;
    for (chi0_ctx* c : b->items) c->launches += 1;
    fork(b->evs[2 * ns + 1]);
    for (size_t i = 0; i < b->items.size() && s == CHI0_OK; ++i) {
      chi0_ctx* c = b->items[i];
      c->rho_iq = c->plan_rho_iq;
      s = b->outs[i] ? chi0::launch_chi0_eps(c) : chi0::launch_chi0(c);
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
  if (cudaGraphLaunch(b->exec, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  return CHI0_OK;
}

int chi0_batch_rho_width(const chi0_batch* b) { return b ? b->jm : 0; }

void chi0_batch_destroy(chi0_batch* b) { destroy_batch(b); }

}  // extern "C"
