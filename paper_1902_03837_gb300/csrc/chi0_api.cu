// C ABI of libchi0 (declared in include/chi0.h): argument checking, the host
// side of the q-point setup (k - q folding, response G set, transition block,
// twiddle tables) and the stream-ordered sequence of kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/chi0.h"
#include "ctx.cuh"

using chi0::RhoGeom;

namespace {

chi0_status fail(chi0_ctx* c, chi0_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

chi0_status cuda_fail(chi0_ctx* c, cudaError_t e, const char* what) {
  return fail(c, e == cudaErrorMemoryAllocation ? CHI0_ENOMEM : CHI0_ECUDA, "%s: %s", what,
              cudaGetErrorString(e));
}

#define CK(call, what)                                \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

chi0_status ensure(chi0_ctx* c, DevBuf& b, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return CHI0_OK;
  if (b.borrowed)  // memory owned elsewhere cannot grow here
    return fail(c, CHI0_ESTATE, "%s: shared buffer of %zu bytes, %zu needed", what, b.bytes, bytes);
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (std::getenv("CHI0_FAULT") && std::strcmp(std::getenv("CHI0_FAULT"), "alloc") == 0)
    return fail(c, CHI0_ENOMEM, "%s: injected allocation failure (CHI0_FAULT=alloc)", what);
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CHI0_ENOMEM, "%s: cudaMalloc(%zu) failed: %s", what, bytes,
                cudaGetErrorString(e));
  }
  b.bytes = bytes;
  return CHI0_OK;
}

}  // namespace

namespace chi0 {
void stage_begin(chi0_ctx* c, int stage) {
  if (c->capturing) return;
  auto& st = c->stage[stage];
  if (st.used + 2 > st.ev.size()) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      return;
    }
    st.ev.push_back(a);
    st.ev.push_back(b);
  }
  cudaEventRecord(st.ev[st.used], c->st);
}
void stage_end(chi0_ctx* c, int stage, int kernels) {
  auto& st = c->stage[stage];
  if (c->capturing) {
    st.launches += kernels;
    c->launches += kernels;
    return;
  }
  if (st.used + 2 > st.ev.size()) return;  // begin failed to get events
  cudaEventRecord(st.ev[st.used + 1], c->st);
  st.used += 2;
  st.launches += kernels;
  c->launches += kernels;
}
chi0_status ctx_fail(chi0_ctx* c, chi0_status s, const char* msg) { c->err = msg; return s; }
chi0_status ctx_ensure(chi0_ctx* c, DevBuf& b, size_t bytes, const char* what) { return ensure(c, b, bytes, what); }
}  // namespace chi0

namespace {

void release(DevBuf& b) {
  if (b.p && !b.borrowed) cudaFree(b.p);
  b = DevBuf{};
}

size_t cplx_bytes(const chi0_ctx* c) { return c->fp64 ? 16 : 8; }

// |q+G|^2 scaled to an exact integer for a cubic cell: sum_a (L q_a + L G_a)^2
// with L = lcm of the k grid (q is a grid vector, so L q_a is an integer).
int64_t lcm64(int64_t a, int64_t b) {
  int64_t x = a, y = b;
  while (y) {
    int64_t t = x % y;
    x = y;
    y = t;
  }
  return a / x * b;
}

bool q_integers(const chi0_ctx* c, int iq, int64_t qi[3]) {
  for (int d = 0; d < 3; ++d) {
    const double x = c->q[3 * iq + d] * c->cfg.kgrid[d];
    const double r = std::nearbyint(x);
    if (std::fabs(x - r) > 1e-9) return false;
    qi[d] = (int64_t)r;
  }
  return true;
}

void response_set(const chi0_ctx* c, int iq, std::vector<int32_t>& out) {
  int64_t qi[3];
  q_integers(c, iq, qi);
  const int64_t L = lcm64(lcm64(c->cfg.kgrid[0], c->cfg.kgrid[1]), c->cfg.kgrid[2]);
  int64_t lq[3];
  for (int d = 0; d < 3; ++d) lq[d] = qi[d] * (L / c->cfg.kgrid[d]);
  const int ng = c->cfg.ng;
  const int m = (int)std::ceil(std::cbrt(3.0 * ng / (4.0 * M_PI))) + 3;
  std::vector<std::tuple<int64_t, int, int, int>> cand;
  cand.reserve((size_t)(2 * m + 1) * (2 * m + 1) * (2 * m + 1));
  for (int x = -m; x <= m; ++x)
    for (int y = -m; y <= m; ++y)
      for (int z = -m; z <= m; ++z) {
        const int64_t a = lq[0] + L * x, b = lq[1] + L * y, d = lq[2] + L * z;
        cand.emplace_back(a * a + b * b + d * d, x, y, z);
      }
  std::sort(cand.begin(), cand.end());
  out.resize((size_t)ng * 3);
  for (int i = 0; i < ng; ++i) {
    out[3 * i] = std::get<1>(cand[i]);
    out[3 * i + 1] = std::get<2>(cand[i]);
    out[3 * i + 2] = std::get<3>(cand[i]);
  }
}

void kpairs(const chi0_ctx* c, int iq, std::vector<int32_t>& kq, std::vector<int32_t>& g0) {
  int64_t qi[3];
  q_integers(c, iq, qi);
  const int* n = c->cfg.kgrid;
  kq.resize(c->nk);
  g0.resize((size_t)c->nk * 3);
  for (int i = 0; i < n[0]; ++i)
    for (int j = 0; j < n[1]; ++j)
      for (int l = 0; l < n[2]; ++l) {
        const int ik = (i * n[1] + j) * n[2] + l;
        const int64_t src[3] = {i - qi[0], j - qi[1], l - qi[2]};
        int64_t rep[3];
        for (int d = 0; d < 3; ++d) {
          rep[d] = ((src[d] % n[d]) + n[d]) % n[d];
          g0[3 * ik + d] = (int32_t)((src[d] - rep[d]) / n[d]);
        }
        kq[ik] = (int32_t)((rep[0] * n[1] + rep[1]) * n[2] + rep[2]);
      }
}

template <typename T2>
void twiddles(int n, std::vector<T2>& out) {
  out.resize(n);
  for (int j = 0; j < n; ++j) {
    const double ang = 2.0 * M_PI * (double)j / (double)n;
    out[j].x = std::cos(ang);
    out[j].y = std::sin(ang);
  }
}

chi0_status check_device_error(chi0_ctx* c) {
  if (!c->d_err.p) return CHI0_OK;
  int h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, c->d_err.p, sizeof(h), cudaMemcpyDeviceToHost, c->st), "read error flag");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  if (h[0] || h[1]) {
    CK(cudaMemsetAsync(c->d_err.p, 0, sizeof(h), c->st), "clear error flag");
    if (h[1]) return fail(c, CHI0_ETIMEOUT, "a bounded device-side wait gave up (code %d)", h[1]);
    return fail(c, CHI0_ENOTPD, "Dyson elimination met a non-positive (Hermitian) or vanishing (general) pivot");
  }
  return CHI0_OK;
}

}  // namespace

namespace chi0 {

chi0_status plan_rho(chi0_ctx* c, int iq) {
  if (!c) return CHI0_EINVAL;
  if (iq < 0 || iq >= c->cfg.nq) return fail(c, CHI0_EINVAL, "iq %d out of range", iq);
  for (int ik = 0; ik < c->nk; ++ik)
    if (!c->wf_set[ik]) return fail(c, CHI0_ESTATE, "wavefunctions of k %d not set", ik);
  if (!c->energies_set) return fail(c, CHI0_ESTATE, "energies not set");
  if (c->rho_planned_epoch == c->plan_epoch && c->plan_rho_iq == iq) {
    c->rho_iq = c->chi_iq = c->eps_iq = -1;   // the plan holds; the results are stale
    return CHI0_OK;
  }
  chi0_status s;
  // ---- q-point setup on the host
  response_set(c, iq, c->h_gresp);
  kpairs(c, iq, c->h_kq, c->h_g0);
  const double tol = c->cfg.occ_drop_tol;
  int mmax = -1, nmin = c->nb;
  for (int ik = 0; ik < c->nk; ++ik)
    for (int b = 0; b < c->nb; ++b) {
      const double f = c->h_occ[(size_t)ik * c->nb + b];
      if (f > tol) mmax = std::max(mmax, b);
      if (f < 1.0 - tol) nmin = std::min(nmin, b);
    }
  // the extrapolar correction subtracts every band n < nb at k (closure)
  if (c->bg_on) nmin = 0;
  c->Nm = mmax + 1;
  c->n_lo = nmin;
  c->Nn = c->nb - nmin;
  c->nt = (int64_t)c->nk * c->Nn * c->Nm;
  RhoGeom& g = c->geom;
  g = RhoGeom{};
  g.N1 = c->cfg.fft[0];
  g.N2 = c->cfg.fft[1];
  g.N3 = c->cfg.fft[2];
  int L[3] = {0, 0, 0};
  for (int ik = 0; ik < c->nk; ++ik)
    for (int p = 0; p < c->h_npw[ik]; ++p)
      for (int d = 0; d < 3; ++d)
        L[d] = std::max(L[d], std::abs(c->h_gvec[((size_t)ik * c->npw_max + p) * 3 + d]));
  g.Lx = L[0];
  g.Ly = L[1];
  g.Lz = L[2];
  g.NX = 2 * L[0] + 1;
  g.NY = 2 * L[1] + 1;
  g.NZ = 2 * L[2] + 1;
  g.nk = c->nk;
  g.nb = c->nb;
  g.npw_max = c->npw_max;
  g.ng = c->cfg.ng;
  int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
  for (int i = 0; i < g.ng; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], c->h_gresp[3 * i + d]);
      hi[d] = std::max(hi[d], c->h_gresp[3 * i + d]);
    }
  g.Mx_lo = lo[0];
  g.My_lo = lo[1];
  g.Mz_lo = lo[2];
  g.HX = hi[0] - lo[0] + 1;
  g.HY = hi[1] - lo[1] + 1;
  g.HZ = hi[2] - lo[2] + 1;
  g.n_lo = c->n_lo;
  g.Nn = c->Nn;
  g.Nm = c->Nm;
  int g0max = 0;
  for (int v : c->h_g0) g0max = std::max(g0max, std::abs(v));
  g.g0max = g0max;
  g.g0z_min = 1 << 30;
  g.g0z_max = -(1 << 30);
  for (int ik = 0; ik < c->nk; ++ik) {
    g.g0z_min = std::min(g.g0z_min, c->h_g0[3 * ik + 2]);
    g.g0z_max = std::max(g.g0z_max, c->h_g0[3 * ik + 2]);
  }
  // response indices in (Gy, Gz, Gx) order
  c->h_gperm.resize(g.ng);
  for (int i = 0; i < g.ng; ++i) c->h_gperm[i] = i;
  std::stable_sort(c->h_gperm.begin(), c->h_gperm.end(), [&](int a, int b) {
    const int32_t* A = &c->h_gresp[3 * a];
    const int32_t* B = &c->h_gresp[3 * b];
    if (A[1] != B[1]) return A[1] < B[1];
    if (A[2] != B[2]) return A[2] < B[2];
    return A[0] < B[0];
  });
  // the real-space product must not alias onto the response set
  for (int d = 0; d < 3; ++d) {
    const int n = c->cfg.fft[d];
    const int hmax = std::max(std::abs(lo[d]), std::abs(hi[d])) + g0max;
    if (n <= 2 * L[d] + hmax)
      return fail(c, CHI0_EINVAL,
                  "fft[%d] = %d aliases: need > 2*%d + %d for these spheres and response set", d,
                  n, L[d], hmax);
  }
  const bool streamed = c->stream_nb > 0;
  if (streamed) {
    if (c->bg_on || c->term_params || c->grp_thresh > 0.0)
      return fail(c, CHI0_EUNSUPPORTED,
                  "band-block streaming excludes the extrapolar correction, the learned terminator and pole grouping");
    c->blk_nb = std::max(1, std::min(c->stream_nb, c->Nn));
    c->blk_nk = std::max(1, std::min(c->stream_nk > 0 ? c->stream_nk : c->nk, c->nk));
    c->nt_blk = (int64_t)c->blk_nk * c->blk_nb * c->Nm;
  }
  c->rho_iq = c->chi_iq = c->eps_iq = -1;
  c->plan_rho_iq = iq;
  if (c->nt == 0) {
    c->rho_planned_epoch = c->plan_epoch;
    ++c->rho_plan_serial;
    return CHI0_OK;
  }
  // ---- device buffers
  const size_t cb = cplx_bytes(c);
  const size_t plane_bytes = (size_t)g.N1 * g.NZ * g.N2 * cb;
  // streamed: the m-band grids of every k (resident) and one block's n grids
  const size_t ubytes = streamed ? (size_t)c->nk * c->Nm * plane_bytes : (size_t)c->nk * c->nb * plane_bytes;
  if ((s = ensure(c, c->d_U, ubytes, "mixed-grid wavefunctions")) != CHI0_OK) return s;
  if (streamed &&
      (s = ensure(c, c->d_Ublk, (size_t)c->blk_nk * c->blk_nb * plane_bytes, "mixed grids of a band block")) != CHI0_OK)
    return s;
  if ((s = ensure(c, c->d_R, (size_t)(streamed ? c->nt_blk : c->nt) * g.ng * cb, "rho")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_gresp, (size_t)g.ng * 12, "G set")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_gperm, (size_t)g.ng * 4, "G order")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_kq, (size_t)c->nk * 4, "k pairs")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_g0, (size_t)c->nk * 12, "umklapp")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_tw1, (size_t)g.N1 * cb, "twiddles")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_tw2, (size_t)g.N2 * cb, "twiddles")) != CHI0_OK) return s;
  CK(cudaMemcpyAsync(c->d_gresp.p, c->h_gresp.data(), (size_t)g.ng * 12, cudaMemcpyHostToDevice, c->st), "G set H2D");
  CK(cudaMemcpyAsync(c->d_kq.p, c->h_kq.data(), (size_t)c->nk * 4, cudaMemcpyHostToDevice, c->st), "kq H2D");
  CK(cudaMemcpyAsync(c->d_gperm.p, c->h_gperm.data(), (size_t)g.ng * 4, cudaMemcpyHostToDevice, c->st), "G order H2D");
  CK(cudaMemcpyAsync(c->d_g0.p, c->h_g0.data(), (size_t)c->nk * 12, cudaMemcpyHostToDevice, c->st), "g0 H2D");
  if (c->fp64) {
    std::vector<double2> t1, t2;
    twiddles(g.N1, t1);
    twiddles(g.N2, t2);
    CK(cudaMemcpyAsync(c->d_tw1.p, t1.data(), t1.size() * 16, cudaMemcpyHostToDevice, c->st), "tw H2D");
    CK(cudaMemcpyAsync(c->d_tw2.p, t2.data(), t2.size() * 16, cudaMemcpyHostToDevice, c->st), "tw H2D");
    CK(cudaStreamSynchronize(c->st), "synchronize");
  } else {
    std::vector<double2> t1d, t2d;
    twiddles(g.N1, t1d);
    twiddles(g.N2, t2d);
    std::vector<float2> t1(t1d.size()), t2(t2d.size());
    for (size_t i = 0; i < t1d.size(); ++i) t1[i] = make_float2((float)t1d[i].x, (float)t1d[i].y);
    for (size_t i = 0; i < t2d.size(); ++i) t2[i] = make_float2((float)t2d[i].x, (float)t2d[i].y);
    CK(cudaMemcpyAsync(c->d_tw1.p, t1.data(), t1.size() * 8, cudaMemcpyHostToDevice, c->st), "tw H2D");
    CK(cudaMemcpyAsync(c->d_tw2.p, t2.data(), t2.size() * 8, cudaMemcpyHostToDevice, c->st), "tw H2D");
    CK(cudaStreamSynchronize(c->st), "synchronize");
  }
  // mixed grid: coefficients in, U out; transforms along y (NX N2 NY per gz
  // plane) and x (N1 N2 NX per gz plane)
  {
    auto& a1 = c->stage[CHI0_STAGE_WF_GRID];
    a1.bytes = (double)c->nk * c->nb * ((double)c->npw_max * (cb + 12) + ubytes / ((double)c->nk * c->nb));
    a1.flops = 8.0 * (double)c->nk * c->nb * g.NZ *
               ((double)g.NX * g.N2 * g.NY + (double)g.N1 * g.N2 * g.NX);
    // rho: every transition reads two N1 x NZ x N2 mixed grids and writes ng values;
    // executed work per transition and x plane: the z correlation (N2 HZ NZ
    // complex multiply-adds), the pruned y transform (HY HZ N2 / 4 multiply-adds
    // plus 6 HZ N2 flops of radix-4 butterflies when N2 % 4 == 0, else HY HZ N2
    // multiply-adds), the x accumulation (ng multiply-adds)
    auto& a2 = c->stage[CHI0_STAGE_RHO];
    a2.bytes = (double)c->nt * g.ng * cb + (double)ubytes;
    const double ywork = (g.N2 % 4 == 0) ? 8.0 * g.HY * g.HZ * (g.N2 / 4) + 6.0 * g.HZ * g.N2
                                         : 8.0 * g.HY * g.HZ * g.N2;
    a2.flops = (double)c->nt * g.N1 *
               (8.0 * g.N2 * g.HZ * g.NZ + ywork + 8.0 * g.ng);
  }
  c->rho_planned_epoch = c->plan_epoch;
  ++c->rho_plan_serial;
  return CHI0_OK;
}

// wavefunctions to the mixed grid: every k and band (nkr = 0), or the k
// points k0 .. k0 + nkr - 1 and bands b0 .. b0 + nbo - 1 into U[k - k0][b - b0]
cudaError_t launch_wf_range(chi0_ctx* c, void* U, int k0, int nkr, int b0, int nbo) {
  const RhoGeom& g = c->geom;
  chi0::stage_begin(c, CHI0_STAGE_WF_GRID);
  cudaError_t e;
  if (c->fp64)
    e = chi0::launch_wf_to_mixed<double>(g, (const int32_t*)c->d_gvec.p, (const int32_t*)c->d_npw.p,
                                         (const double2*)c->d_coef.p, (const double2*)c->d_tw1.p,
                                         (const double2*)c->d_tw2.p, (double2*)U, c->st, k0, nkr, b0, nbo);
  else
    e = chi0::launch_wf_to_mixed<float>(g, (const int32_t*)c->d_gvec.p, (const int32_t*)c->d_npw.p,
                                        (const float2*)c->d_coef.p, (const float2*)c->d_tw1.p,
                                        (const float2*)c->d_tw2.p, (float2*)U, c->st, k0, nkr, b0, nbo);
  if (e == cudaSuccess) chi0::stage_end(c, CHI0_STAGE_WF_GRID, 1);
  // the coefficients have been read up to here: the next copy on the upload
  // stream waits for this point
  if (e == cudaSuccess && c->ev_wf_done && !c->capturing) e = cudaEventRecord(c->ev_wf_done, c->st);
  return e;
}

// kernels of compute_rho (wavefunctions to the mixed grid; rho unless the
// caller runs rho for many problems in one batched launch, or the
// transitions are streamed in band blocks by build_chi0)
// rho of the whole problem, pipelined with the coefficient upload: the k
// points in kWfChunks chunks, each transformed once its copies have landed
// (the event of its latest copy on the upload stream), and rho launched on a
// chunk of k-pairs right after the transform that completes the grids of
// its k and k - q points.  The blocks compute the same transitions as one
// launch over all k-pairs, so the result is the same.
constexpr int kWfChunks = 8;

chi0_status launch_rho_pipelined(chi0_ctx* c) {
  const int nk = c->nk;
  const int per = (nk + kWfChunks - 1) / kWfChunks;   // k points per chunk
  const int nch = (nk + per - 1) / per;                // chunks (the last may be short)
  auto chunk_of = [&](int k) { return k / per; };
  // the transform chunk each rho chunk waits for
  std::vector<int> need(nch, 0);
  for (int k = 0; k < nk; ++k) {
    const int ch = chunk_of(k);
    need[ch] = std::max(need[ch], std::max(ch, chunk_of(c->h_kq[k])));
  }
  const RhoGeom& g0 = c->geom;
  const size_t band = (size_t)g0.N1 * g0.NZ * g0.N2;   // complex entries of one band's mixed grid
  const size_t cbytes = cplx_bytes(c);
  for (int w = 0; w < nch; ++w) {
    const int k0 = w * per, k1 = std::min(nk, k0 + per);
    if (!c->ev_up.empty()) {   // the chunk's latest copy
      int last = -1;
      for (int k = k0; k < k1; ++k)
        if (c->up_seq[k] >= 0 && (last < 0 || c->up_seq[k] > c->up_seq[last])) last = k;
      if (last >= 0) CK(cudaStreamWaitEvent(c->st, c->ev_up[last], 0), "upload wait");
    }
    // the transform of k0 .. k1 - 1, written at its global place in U
    cudaError_t e = launch_wf_range(c, (char*)c->d_U.p + (size_t)k0 * c->nb * band * cbytes, k0, k1 - k0, 0, c->nb);
    if (e != cudaSuccess) return cuda_fail(c, e, "wf_to_mixed launch");
    for (int r = 0; r < nch; ++r) {
      if (need[r] != w) continue;
      const int r0 = r * per, r1 = std::min(nk, r0 + per);
      RhoGeom g = g0;
      g.k0 = r0;
      g.nk = r1 - r0;
      g.nbu = c->nb;
      g.bu0 = 0;
      g.nbm = c->nb;
      const size_t roff = (size_t)r0 * c->Nn * c->Nm * g0.ng;
      const size_t uoff = (size_t)r0 * c->nb * band;
      chi0::stage_begin(c, CHI0_STAGE_RHO);
      if (c->fp64)
        e = chi0::launch_rho_pairs<double, double2>(
            g, (const double2*)c->d_U.p + uoff, (const int32_t*)c->d_kq.p, (const int32_t*)c->d_g0.p,
            (const int32_t*)c->d_gresp.p, (const int32_t*)c->d_gperm.p, (const double2*)c->d_tw1.p,
            (const double2*)c->d_tw2.p, (double2*)c->d_R.p + roff, c->st, (const double2*)c->d_U.p);
      else
        e = chi0::launch_rho_pairs<float, float2>(
            g, (const float2*)c->d_U.p + uoff, (const int32_t*)c->d_kq.p, (const int32_t*)c->d_g0.p,
            (const int32_t*)c->d_gresp.p, (const int32_t*)c->d_gperm.p, (const float2*)c->d_tw1.p,
            (const float2*)c->d_tw2.p, (float2*)c->d_R.p + roff, c->st, (const float2*)c->d_U.p);
      if (e != cudaSuccess) return cuda_fail(c, e, "rho_pairs launch");
      chi0::stage_end(c, CHI0_STAGE_RHO, 1);
    }
  }
  return CHI0_OK;
}

chi0_status launch_rho(chi0_ctx* c, bool with_pairs) {
  const int iq = c->plan_rho_iq;
  if (iq < 0) return fail(c, CHI0_ESTATE, "rho not planned");
  if (with_pairs && c->nt > 0 && !c->grid_shared && c->stream_nb == 0 && c->nk >= 2 * kWfChunks) {
    chi0_status s = launch_rho_pipelined(c);
    if (s != CHI0_OK) return s;
    c->rho_iq = iq;
    c->chi_iq = c->eps_iq = -1;
    return CHI0_OK;
  }
  if (c->nt > 0 && !c->grid_shared) {
    // streamed: the grids of the m bands 0 .. Nm - 1 at every k only
    const int nkr = c->stream_nb > 0 ? c->nk : 0, nbo = c->stream_nb > 0 ? c->Nm : 0;
    if (!c->ev_up.empty()) {   // every copy on the upload stream first
      int last = -1;
      for (int k = 0; k < c->nk; ++k)
        if (c->up_seq[k] >= 0 && (last < 0 || c->up_seq[k] > c->up_seq[last])) last = k;
      if (last >= 0) CK(cudaStreamWaitEvent(c->st, c->ev_up[last], 0), "upload wait");
    }
    cudaError_t e = launch_wf_range(c, c->d_U.p, 0, nkr, 0, nbo);
    if (e != cudaSuccess) return cuda_fail(c, e, "wf_to_mixed launch");
  }
  if (c->nt > 0 && c->stream_nb == 0) {
    const RhoGeom& g = c->geom;
    cudaError_t e;
    if (with_pairs) {
      chi0::stage_begin(c, CHI0_STAGE_RHO);
      if (c->fp64)
        e = chi0::launch_rho_pairs<double, double2>(
            g, (const double2*)c->d_U.p, (const int32_t*)c->d_kq.p, (const int32_t*)c->d_g0.p,
            (const int32_t*)c->d_gresp.p, (const int32_t*)c->d_gperm.p, (const double2*)c->d_tw1.p,
            (const double2*)c->d_tw2.p, (double2*)c->d_R.p, c->st);
      else
        e = chi0::launch_rho_pairs<float, float2>(
            g, (const float2*)c->d_U.p, (const int32_t*)c->d_kq.p, (const int32_t*)c->d_g0.p,
            (const int32_t*)c->d_gresp.p, (const int32_t*)c->d_gperm.p, (const float2*)c->d_tw1.p,
            (const float2*)c->d_tw2.p, (float2*)c->d_R.p, c->st);
      if (e != cudaSuccess) return cuda_fail(c, e, "rho_pairs launch");
      chi0::stage_end(c, CHI0_STAGE_RHO, 1);
    }
  }
  c->rho_iq = iq;
  c->chi_iq = c->eps_iq = -1;
  return CHI0_OK;
}

// Frequency factor of a transition with energy difference d (the weights
// kernel's form): kind 0 the imaginary axis, kinds 1 / 2 the real / imaginary
// part on the real axis.
static double pole_weight_host(int kind, double om, double eta, double d) {
  if (kind == 0) {
    const double sw = om + eta;
    const double den = d * d + sw * sw;
    return den > 0.0 ? 2.0 * d / den : 0.0;
  }
  const double a = om + d, b = om - d;
  const double da = a * a + eta * eta, db = b * b + eta * eta;
  if (!(da > 0.0) || !(db > 0.0)) return 0.0;
  return kind == 1 ? a / da - b / db : eta / db - eta / da;
}

// Sign shared by every imaginary-axis transition weight (the kind-0 weights of
// k_weights).  pref (f_m - f_n) 2d/(d^2 + s^2) has the sign of its pole d at
// every frequency (pref > 0, f_m - f_n > tol), and the extrapolar term
// -pref f_m 2dbar/(dbar^2 + s^2) the sign of -dbar.  Returns -1 or +1 when no
// nonzero term has the other sign, 0 when they are mixed or when a dense grid
// makes the factor a mean over poles that are not known here.  dpole: the
// pole energy each transition uses (its group representative's), or NULL for
// its own.
static int weight_sign(const chi0_ctx* c, const std::vector<double>* dpole) {
  if (c->dg_nd > 0) return 0;
  bool pos = false, neg = false;
  const int nb = c->nb;
  for (int64_t t = 0; t < c->nt; ++t) {
    const int m = (int)(t % c->Nm);
    const int64_t r = t / c->Nm;
    const int n = c->n_lo + (int)(r % c->Nn);
    const int ik = (int)(r / c->Nn), ikp = c->h_kq[ik];
    const double fm = c->h_occ[(size_t)ikp * nb + m];
    if (fm - c->h_occ[(size_t)ik * nb + n] > c->cfg.occ_drop_tol) {
      const double d = dpole ? (*dpole)[t] : c->h_eps[(size_t)ikp * nb + m] - c->h_eps[(size_t)ik * nb + n];
      pos |= d > 0.0;
      neg |= d < 0.0;
    }
    if (c->bg_on && fm > c->cfg.occ_drop_tol) {
      const double dbar = c->h_eps[(size_t)ikp * nb + m] - c->bg_eps;
      pos |= dbar < 0.0;
      neg |= dbar > 0.0;
    }
    if (pos && neg) return 0;
  }
  return neg ? -1 : 1;
}

// ---- Bruneval-Gonze extrapolar correction: planning and launch
// Difference vectors d = G_i - G_j of the response set, ordered by (y, z, x)
// (the order the rho kernel visits its G set in), cut into chunks of at most
// 4096 (the rho kernel's register accumulators at one m band per block).
chi0_status plan_bg(chi0_ctx* c) {
  const int ng = c->cfg.ng, nw = c->nwv;
  const RhoGeom& g = c->geom;
  auto less_yzx = [](const std::array<int32_t, 3>& A, const std::array<int32_t, 3>& B) {
    if (A[1] != B[1]) return A[1] < B[1];
    if (A[2] != B[2]) return A[2] < B[2];
    return A[0] < B[0];
  };
  std::vector<std::array<int32_t, 3>> dv((size_t)ng * ng);
  for (int i = 0; i < ng; ++i)
    for (int j = 0; j < ng; ++j)
      for (int a = 0; a < 3; ++a)
        dv[(size_t)i * ng + j][a] = c->h_gresp[3 * i + a] - c->h_gresp[3 * j + a];
  std::vector<std::array<int32_t, 3>> D(dv);
  std::sort(D.begin(), D.end(), less_yzx);
  D.erase(std::unique(D.begin(), D.end()), D.end());
  const int nd = (int)D.size();
  std::vector<int32_t> didx((size_t)ng * ng);
  for (size_t e = 0; e < dv.size(); ++e)
    didx[e] = (int32_t)(std::lower_bound(D.begin(), D.end(), dv[e], less_yzx) - D.begin());
  // the densities' products must not alias onto the difference set
  for (int a = 0; a < 3; ++a) {
    int dmax = 0;
    for (const auto& d : D) dmax = std::max(dmax, std::abs(d[a]));
    const int L = a == 0 ? g.Lx : a == 1 ? g.Ly : g.Lz;
    if (c->cfg.fft[a] <= 2 * L + dmax)
      return fail(c, CHI0_EINVAL,
                  "fft[%d] = %d aliases for the extrapolar densities: need > 2*%d + %d", a,
                  c->cfg.fft[a], L, dmax);
  }
  constexpr int kChunk = 4096;
  const int nch = (nd + kChunk - 1) / kChunk;
  if (nch > chi0::kBgMaxChunks)
    return fail(c, CHI0_EUNSUPPORTED, "%d difference vectors: more than %d chunks", nd, chi0::kBgMaxChunks);
  const int64_t ntd = (int64_t)c->nk * c->Nm;
  chi0::BgChunks ch{};
  ch.n = nch;
  c->bg_geom.assign(nch, g);
  for (int k = 0; k < nch; ++k) {
    const int a0 = k * kChunk, a1 = std::min(nd, a0 + kChunk);
    ch.start[k] = a0;
    ch.off[k] = ntd * a0;
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-(1 << 30), -(1 << 30), -(1 << 30)};
    for (int e = a0; e < a1; ++e)
      for (int a = 0; a < 3; ++a) {
        lo[a] = std::min(lo[a], D[e][a]);
        hi[a] = std::max(hi[a], D[e][a]);
      }
    RhoGeom& gc = c->bg_geom[k];
    gc.ng = a1 - a0;
    gc.Mx_lo = lo[0];
    gc.My_lo = lo[1];
    gc.Mz_lo = lo[2];
    gc.HX = hi[0] - lo[0] + 1;
    gc.HY = hi[1] - lo[1] + 1;
    gc.HZ = hi[2] - lo[2] + 1;
    gc.n_lo = 0;
    gc.Nn = c->Nm;
    gc.Nm = 1;
    gc.diag = 1;
    gc.g0max = 0;
    gc.g0z_min = 0;
    gc.g0z_max = 0;
  }
  ch.start[nch] = nd;
  // extrapolar weights wbar[iw][k * Nm + m] (same pole form as the weights kernel)
  const double pref = c->cfg.spin_factor / ((double)c->nk * c->omega_cell);
  const double tol = c->cfg.occ_drop_tol;
  std::vector<double> wbar((size_t)nw * ntd, 0.0);
  for (int iw = 0; iw < nw; ++iw)
    for (int ik = 0; ik < c->nk; ++ik)
      for (int m = 0; m < c->Nm; ++m) {
        const double f = c->h_occ[(size_t)ik * c->nb + m];
        if (!(f > tol)) continue;
        const double dbar = c->h_eps[(size_t)ik * c->nb + m] - c->bg_eps;
        wbar[(size_t)iw * ntd + (size_t)ik * c->Nm + m] =
            pref * f * pole_weight_host(c->h_vkind[iw], c->h_vval[iw], c->cfg.eta, dbar);
      }
  std::vector<int32_t> dflat((size_t)nd * 3), ident(std::min(nd, kChunk)), kid(c->nk), zero((size_t)c->nk * 3, 0);
  for (int e = 0; e < nd; ++e)
    for (int a = 0; a < 3; ++a) dflat[(size_t)e * 3 + a] = D[e][a];
  for (size_t e = 0; e < ident.size(); ++e) ident[e] = (int32_t)e;
  for (int ik = 0; ik < c->nk; ++ik) kid[ik] = ik;
  chi0_status s;
  const size_t cb = cplx_bytes(c);
  if ((s = ensure(c, c->d_bgd, dflat.size() * 4, "difference vectors")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_bgperm, ident.size() * 4, "difference order")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_bgkq, kid.size() * 4, "k map")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_bgg0, zero.size() * 4, "zero umklapp")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_bgrd, (size_t)ntd * nd * cb, "diagonal densities")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_bgw, wbar.size() * 8, "extrapolar weights")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_bgP, (size_t)nw * nd * 16, "extrapolar term")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_bgidx, didx.size() * 4, "difference index")) != CHI0_OK) return s;
  CK(cudaMemcpyAsync(c->d_bgd.p, dflat.data(), dflat.size() * 4, cudaMemcpyHostToDevice, c->st), "d H2D");
  CK(cudaMemcpyAsync(c->d_bgperm.p, ident.data(), ident.size() * 4, cudaMemcpyHostToDevice, c->st), "order H2D");
  CK(cudaMemcpyAsync(c->d_bgkq.p, kid.data(), kid.size() * 4, cudaMemcpyHostToDevice, c->st), "k map H2D");
  CK(cudaMemcpyAsync(c->d_bgg0.p, zero.data(), zero.size() * 4, cudaMemcpyHostToDevice, c->st), "G0 H2D");
  CK(cudaMemcpyAsync(c->d_bgw.p, wbar.data(), wbar.size() * 8, cudaMemcpyHostToDevice, c->st), "wbar H2D");
  CK(cudaMemcpyAsync(c->d_bgidx.p, didx.data(), didx.size() * 4, cudaMemcpyHostToDevice, c->st), "index H2D");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  c->bg_nd = nd;
  c->bg_ntd = ntd;
  c->bg_ch = ch;
  return CHI0_OK;
}

// diagonal densities (rho kernel, same-band mode) and their weighted sum
// P[w][d]; independent of the contraction, so launched before it (the
// Hermitised gather into chi0 follows each frequency's reduction)
chi0_status launch_bg(chi0_ctx* c) {
  const RhoGeom& g = c->geom;
  const int ng = c->cfg.ng, nw = c->nwv;
  const size_t cb = cplx_bytes(c);
  chi0::stage_begin(c, CHI0_STAGE_RHO);
  for (int k = 0; k < c->bg_ch.n; ++k) {
    const RhoGeom& gc = c->bg_geom[k];
    const int32_t* dset = (const int32_t*)c->d_bgd.p + 3 * (size_t)c->bg_ch.start[k];
    char* out = (char*)c->d_bgrd.p + (size_t)c->bg_ch.off[k] * cb;
    cudaError_t e;
    if (c->fp64)
      e = chi0::launch_rho_pairs<double, double2>(gc, (const double2*)c->d_U.p, (const int32_t*)c->d_bgkq.p,
                                                  (const int32_t*)c->d_bgg0.p, dset,
                                                  (const int32_t*)c->d_bgperm.p, (const double2*)c->d_tw1.p,
                                                  (const double2*)c->d_tw2.p, (double2*)out, c->st);
    else
      e = chi0::launch_rho_pairs<float, float2>(gc, (const float2*)c->d_U.p, (const int32_t*)c->d_bgkq.p,
                                                (const int32_t*)c->d_bgg0.p, dset,
                                                (const int32_t*)c->d_bgperm.p, (const float2*)c->d_tw1.p,
                                                (const float2*)c->d_tw2.p, (float2*)out, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "extrapolar densities launch");
  }
  chi0::stage_end(c, CHI0_STAGE_RHO, c->bg_ch.n);
  (void)g;
  chi0::stage_begin(c, CHI0_STAGE_REDUCE);
  cudaError_t e = c->fp64 ? chi0::launch_bg_sum<double2>((const double2*)c->d_bgrd.p, c->bg_ch,
                                                        (const double*)c->d_bgw.p, c->bg_ntd, c->bg_nd, nw,
                                                        (double2*)c->d_bgP.p, c->st)
                          : chi0::launch_bg_sum<float2>((const float2*)c->d_bgrd.p, c->bg_ch,
                                                       (const double*)c->d_bgw.p, c->bg_ntd, c->bg_nd, nw,
                                                       (double2*)c->d_bgP.p, c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "extrapolar term launch");
  chi0::stage_end(c, CHI0_STAGE_REDUCE, 1);
  return CHI0_OK;
}

chi0_status plan_chi0(chi0_ctx* c, int iq) {
  if (iq != c->plan_rho_iq || iq < 0) return fail(c, CHI0_ESTATE, "chi0_compute_rho(%d) must come first", iq);
  if (c->chi_planned_epoch == c->plan_epoch && c->plan_chi_iq == iq && c->chi_for_rho_serial == c->rho_plan_serial)
    return CHI0_OK;
  const int nw0 = c->cfg.nw, ng = c->cfg.ng;
  // frequency list of the contraction (see chi0_ctx::nwv)
  c->h_vval.clear();
  c->h_vkind.clear();
  c->h_vr.assign(nw0, -1);
  c->h_vi.assign(nw0, -1);
  c->has_real = false;
  for (int iw = 0; iw < nw0; ++iw) {
    const double re = c->om[2 * iw], im = c->om[2 * iw + 1];
    if (re == 0.0) {
      c->h_vr[iw] = (int)c->h_vval.size();
      c->h_vval.push_back(im);
      c->h_vkind.push_back(0);
      continue;
    }
    if (im != 0.0 || !(re > 0.0) || !(c->cfg.eta > 0.0))
      return fail(c, CHI0_EUNSUPPORTED,
                  "frequency %d: off the imaginary axis only real frequencies > 0 with eta > 0 are supported", iw);
    c->has_real = true;
    c->h_vr[iw] = (int)c->h_vval.size();
    c->h_vval.push_back(re);
    c->h_vkind.push_back(1);
    c->h_vi[iw] = (int)c->h_vval.size();
    c->h_vval.push_back(re);
    c->h_vkind.push_back(2);
  }
  if (c->has_real && c->term_params)
    return fail(c, CHI0_EUNSUPPORTED, "the learned terminator is for imaginary-axis frequencies only");
  c->nwv = (int)c->h_vval.size();
  const int nw = c->nwv;
  chi0_status s;
  const size_t n2 = (size_t)ng * ng;
  if ((s = ensure(c, c->d_chi, n2 * nw0 * 16, "chi0")) != CHI0_OK) return s;
  if (c->has_real) {
    if ((s = ensure(c, c->d_chiv, n2 * nw * 16, "chi0 parts")) != CHI0_OK) return s;
    if ((s = ensure(c, c->d_vr, (size_t)nw0 * 4, "frequency map")) != CHI0_OK) return s;
    if ((s = ensure(c, c->d_vi, (size_t)nw0 * 4, "frequency map")) != CHI0_OK) return s;
    CK(cudaMemcpyAsync(c->d_vr.p, c->h_vr.data(), (size_t)nw0 * 4, cudaMemcpyHostToDevice, c->st), "map H2D");
    // the mixed form contracts a real frequency once with its complex weights
    // (chi0 at its first entry): the combine then only copies it
    c->h_vi_dev = c->h_vi;
    if (!c->fp64) std::fill(c->h_vi_dev.begin(), c->h_vi_dev.end(), -1);
    CK(cudaMemcpyAsync(c->d_vi.p, c->h_vi_dev.data(), (size_t)nw0 * 4, cudaMemcpyHostToDevice, c->st), "map H2D");
  }
  if (!c->d_err.p) {
    if ((s = ensure(c, c->d_err, 16, "error flag")) != CHI0_OK) return s;
    CK(cudaMemsetAsync(c->d_err.p, 0, 16, c->st), "clear error flag");
  }
  c->plan_chi_iq = -1;
  // degenerate-pole grouping (Appendix B): sort the contributing poles by
  // energy (stable in the transition order), open a group at the smallest
  // pole not yet taken and give it every following pole within grp_thresh;
  // each transition then uses its representative's pole energy
  if (c->grp_thresh > 0.0 && c->nt > 0) {
    const int64_t nt = c->nt;
    const int nb = c->nb;
    std::vector<double> d(nt);
    std::vector<int64_t> order;
    order.reserve(nt);
    for (int64_t t = 0; t < nt; ++t) {
      const int m = (int)(t % c->Nm);
      const int64_t r = t / c->Nm;
      const int n = c->n_lo + (int)(r % c->Nn);
      const int ik = (int)(r / c->Nn), ikp = c->h_kq[ik];
      d[t] = c->h_eps[(size_t)ikp * nb + m] - c->h_eps[(size_t)ik * nb + n];
      if (c->h_occ[(size_t)ikp * nb + m] - c->h_occ[(size_t)ik * nb + n] > c->cfg.occ_drop_tol) order.push_back(t);
    }
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return d[a] < d[b]; });
    std::vector<double> dp(d);   // transitions without weight keep their own energy
    std::vector<size_t> gstart;  // first position in `order` of every group
    for (size_t i = 0; i < order.size();) {
      const double dr = d[order[i]];
      gstart.push_back(i);
      size_t j = i;
      do {
        dp[order[j]] = dr;
        ++j;
      } while (j < order.size() && d[order[j]] - dr < c->grp_thresh);
      i = j;
    }
    c->herk_sign = weight_sign(c, &dp);
    chi0_status s0 = ensure(c, c->d_dpole, (size_t)nt * 8, "pole energies");
    if (s0 != CHI0_OK) return s0;
    CK(cudaMemcpyAsync(c->d_dpole.p, dp.data(), (size_t)nt * 8, cudaMemcpyHostToDevice, c->st), "poles H2D");
    CK(cudaStreamSynchronize(c->st), "synchronize");
    // The grouped contraction (Appendix B, Eqs. X_IP_split1/2: a factor per
    // group times the frequency-independent sum of its rho rho^* terms) pays
    // when the groups are large: one contraction over all transitions gives
    // the group sums, and each frequency is then a sum over the groups.
    c->ngroups = (int)std::min<size_t>(gstart.size(), 0x7fffffff);
    gstart.push_back(order.size());
    int64_t kgrp = 0;
    for (int g = 0; g < c->ngroups; ++g) kgrp += (int64_t)((gstart[g + 1] - gstart[g] + 63) / 64) * 64;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    const int nTt = (2 * ng + 127) / 128;
    const double part_bytes = (double)c->ngroups * (nTt * (nTt + 1) / 2) * 65536.0;
    c->grouped = !c->fp64 && !c->has_real && !c->bg_on && !c->term_params && c->stream_nb == 0 &&
                 c->ngroups > 0 && (int64_t)c->ngroups * 32 <= nt && kgrp <= 2 * nt &&
                 part_bytes <= 0.3 * (double)free_b;
    if (c->grouped) {
      c->kgrp = kgrp;
      std::vector<int64_t> perm((size_t)kgrp, -1);
      std::vector<int2> ranges(c->ngroups);
      std::vector<double> ga((size_t)nt, 0.0);
      std::vector<float> fac((size_t)c->nwv * c->ngroups);
      const double pref = c->cfg.spin_factor / ((double)c->nk * c->omega_cell);
      int64_t row = 0;
      for (int g = 0; g < c->ngroups; ++g) {
        ranges[g] = make_int2((int)(row / 64), (int)((gstart[g + 1] - gstart[g] + 63) / 64));
        for (size_t p = gstart[g]; p < gstart[g + 1]; ++p) perm[(size_t)row + (p - gstart[g])] = order[p];
        row += (int64_t)ranges[g].y * 64;
        const double drep = d[order[gstart[g]]];
        for (int v = 0; v < c->nwv; ++v)
          fac[(size_t)v * c->ngroups + g] = (float)pole_weight_host(0, c->h_vval[v], c->cfg.eta, drep);
      }
      for (int64_t t = 0; t < nt; ++t) {
        const int m = (int)(t % c->Nm);
        const int64_t r = t / c->Nm;
        const int n = c->n_lo + (int)(r % c->Nn);
        const int ik = (int)(r / c->Nn), ikp = c->h_kq[ik];
        ga[t] = pref * (c->h_occ[(size_t)ikp * nb + m] - c->h_occ[(size_t)ik * nb + n]);
      }
      if ((s0 = ensure(c, c->d_tperm, (size_t)kgrp * 8, "group order")) != CHI0_OK) return s0;
      if ((s0 = ensure(c, c->d_grange, (size_t)c->ngroups * 8, "group ranges")) != CHI0_OK) return s0;
      if ((s0 = ensure(c, c->d_ga, (size_t)nt * 8, "group weights")) != CHI0_OK) return s0;
      if ((s0 = ensure(c, c->d_gfac, fac.size() * 4, "group factors")) != CHI0_OK) return s0;
      CK(cudaMemcpyAsync(c->d_tperm.p, perm.data(), perm.size() * 8, cudaMemcpyHostToDevice, c->st), "order H2D");
      CK(cudaMemcpyAsync(c->d_grange.p, ranges.data(), ranges.size() * 8, cudaMemcpyHostToDevice, c->st),
         "ranges H2D");
      CK(cudaMemcpyAsync(c->d_ga.p, ga.data(), ga.size() * 8, cudaMemcpyHostToDevice, c->st), "weights H2D");
      CK(cudaMemcpyAsync(c->d_gfac.p, fac.data(), fac.size() * 4, cudaMemcpyHostToDevice, c->st), "factors H2D");
      CK(cudaStreamSynchronize(c->st), "synchronize");
    }
  } else {
    c->grouped = false;
    c->ngroups = 0;
    c->herk_sign = weight_sign(c, nullptr);
  }
  if (c->nt > 0) {
    // transitions per contraction: all of them, or one band block's
    const int64_t ntc = c->stream_nb > 0 ? c->nt_blk : c->nt;
    if ((s = ensure(c, c->d_w, (size_t)ntc * nw * 8, "weights")) != CHI0_OK) return s;
    if ((s = ensure(c, c->d_omim, (size_t)nw * 8, "frequencies")) != CHI0_OK) return s;
    if ((s = ensure(c, c->d_vkind, (size_t)nw * 4, "frequency kinds")) != CHI0_OK) return s;
    CK(cudaMemcpyAsync(c->d_omim.p, c->h_vval.data(), nw * 8, cudaMemcpyHostToDevice, c->st), "omega H2D");
    CK(cudaMemcpyAsync(c->d_vkind.p, c->h_vkind.data(), nw * 4, cudaMemcpyHostToDevice, c->st), "kinds H2D");
    CK(cudaStreamSynchronize(c->st), "synchronize");
    if (c->fp64) {
      // split the transitions into chunks so that the grid fills the GPU
      const int nT = (ng + 31) / 32;
      const int64_t tiles = (int64_t)nT * (nT + 1) / 2 * nw;
      int64_t want = std::max<int64_t>(1, (4 * 152 + tiles - 1) / tiles);
      const int64_t mem_cap = std::max<int64_t>(1, (int64_t)(8ull << 30) / (int64_t)(n2 * nw * 16));
      want = std::min<int64_t>({want, mem_cap, (ntc + 63) / 64});
      c->nchunks = (int)std::max<int64_t>(1, want);
      c->kchunk = (int)((ntc + c->nchunks - 1) / c->nchunks);
      if ((s = ensure(c, c->d_part, n2 * nw * c->nchunks * 16, "chi0 partials")) != CHI0_OK) return s;
    } else if (c->grouped) {
      if ((s = chi0::tc_plan_grouped(c, ng, nw)) != CHI0_OK) return s;
    } else {
      if ((s = chi0::tc_plan(c, ntc, ng, nw)) != CHI0_OK) return s;
    }
    if (c->term_params && (s = chi0::term_plan(c, iq)) != CHI0_OK) return s;
    if (c->bg_on && (s = plan_bg(c)) != CHI0_OK) return s;
  }
  c->plan_chi_iq = iq;
  c->chi_planned_epoch = c->plan_epoch;
  c->chi_for_rho_serial = c->rho_plan_serial;
  ++c->chi_plan_serial;
  return CHI0_OK;
}

// the transition weights of every entry of the frequency list (a3)
chi0_status launch_weights_stage(chi0_ctx* c) {
  const double pref = c->cfg.spin_factor / ((double)c->nk * c->omega_cell);
  chi0::stage_begin(c, CHI0_STAGE_WEIGHTS);
  cudaError_t e = chi0::launch_weights(c->nk, c->n_lo, c->Nn, c->Nm, c->nb, (const int32_t*)c->d_kq.p,
                                       (const double*)c->d_eps.p, (const double*)c->d_occ.p,
                                       (const double*)c->d_omim.p, (const int*)c->d_vkind.p, c->nwv, c->cfg.eta,
                                       pref, c->cfg.occ_drop_tol, c->bg_on, c->bg_eps,
                                       c->grp_thresh > 0.0 ? (const double*)c->d_dpole.p : nullptr,
                                       c->dg_nd > 0 ? (const double*)c->d_epsd.p : nullptr, c->dg_nd,
                                       (double*)c->d_w.p, c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "weights launch");
  chi0::stage_end(c, CHI0_STAGE_WEIGHTS, 1);
  return CHI0_OK;
}

// Band-block streaming: for every block of blk_nk k points and blk_nb n
// bands, the n grids of the block, its rho (m grids from the resident d_U),
// its weights and its contraction, summed into chi0 (the first block writes,
// the later ones add).  The blocks partition the transition set of the
// unstreamed form, so the sum is the same chi0 (Eq. X_IP is a sum over
// transitions) up to the order of the additions.
chi0_status launch_chi0_streamed(chi0_ctx* c) {
  const int nw = c->nwv, ng = c->cfg.ng;
  const size_t n2 = (size_t)ng * ng;
  double2* chiv = c->has_real ? (double2*)c->d_chiv.p : (double2*)c->d_chi.p;
  const double pref = c->cfg.spin_factor / ((double)c->nk * c->omega_cell);
  int blk = 0;
  double bytes = 0.0;
  for (int k0 = 0; k0 < c->nk; k0 += c->blk_nk) {
    const int nkb = std::min(c->blk_nk, c->nk - k0);
    for (int b0 = c->n_lo; b0 < c->nb; b0 += c->blk_nb, ++blk) {
      const int nbb = std::min(c->blk_nb, c->nb - b0);
      const int64_t ntb = (int64_t)nkb * nbb * c->Nm;
      cudaError_t e = launch_wf_range(c, c->d_Ublk.p, k0, nkb, b0, nbb);
      if (e != cudaSuccess) return cuda_fail(c, e, "wf_to_mixed launch (band block)");
      RhoGeom gb = c->geom;
      gb.nk = nkb;
      gb.k0 = k0;
      gb.n_lo = b0;
      gb.Nn = nbb;
      gb.nbu = nbb;
      gb.bu0 = b0;
      gb.nbm = c->Nm;
      chi0::stage_begin(c, CHI0_STAGE_RHO);
      if (c->fp64)
        e = chi0::launch_rho_pairs<double, double2>(
            gb, (const double2*)c->d_Ublk.p, (const int32_t*)c->d_kq.p, (const int32_t*)c->d_g0.p,
            (const int32_t*)c->d_gresp.p, (const int32_t*)c->d_gperm.p, (const double2*)c->d_tw1.p,
            (const double2*)c->d_tw2.p, (double2*)c->d_R.p, c->st, (const double2*)c->d_U.p);
      else
        e = chi0::launch_rho_pairs<float, float2>(
            gb, (const float2*)c->d_Ublk.p, (const int32_t*)c->d_kq.p, (const int32_t*)c->d_g0.p,
            (const int32_t*)c->d_gresp.p, (const int32_t*)c->d_gperm.p, (const float2*)c->d_tw1.p,
            (const float2*)c->d_tw2.p, (float2*)c->d_R.p, c->st, (const float2*)c->d_U.p);
      if (e != cudaSuccess) return cuda_fail(c, e, "rho_pairs launch (band block)");
      chi0::stage_end(c, CHI0_STAGE_RHO, 1);
      chi0::stage_begin(c, CHI0_STAGE_WEIGHTS);
      e = chi0::launch_weights(nkb, b0, nbb, c->Nm, c->nb, (const int32_t*)c->d_kq.p, (const double*)c->d_eps.p,
                               (const double*)c->d_occ.p, (const double*)c->d_omim.p, (const int*)c->d_vkind.p, nw,
                               c->cfg.eta, pref, c->cfg.occ_drop_tol, 0, 0.0, nullptr,
                               c->dg_nd > 0 ? (const double*)c->d_epsd.p : nullptr, c->dg_nd, (double*)c->d_w.p,
                               c->st, k0);
      if (e != cudaSuccess) return cuda_fail(c, e, "weights launch (band block)");
      chi0::stage_end(c, CHI0_STAGE_WEIGHTS, 1);
      chi0_status s;
      if (c->fp64) {
        chi0::stage_begin(c, CHI0_STAGE_CONTRACT);
        e = chi0::launch_chi0_fp64_partials((const double2*)c->d_R.p, (const double*)c->d_w.p, ntb, ng, nw,
                                            c->kchunk, c->nchunks, (double2*)c->d_part.p, c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "chi0 fp64 launch (band block)");
        chi0::stage_end(c, CHI0_STAGE_CONTRACT, 1);
        chi0::stage_begin(c, CHI0_STAGE_REDUCE);
        e = chi0::launch_chi0_reduce((const double2*)c->d_part.p, c->nchunks, ng, nw, chiv, c->st, blk > 0);
        if (e != cudaSuccess) return cuda_fail(c, e, "chi0 reduce launch (band block)");
        chi0::stage_end(c, CHI0_STAGE_REDUCE, 1);
      } else {
        s = chi0::tc_launch(c, c->d_R.p, (const double*)c->d_w.p, ntb, ng, nw, chiv, nullptr, nullptr, nullptr,
                            c->has_real ? c->h_vkind.data() : nullptr, blk > 0);
        if (s != CHI0_OK) return s;
        bytes += c->stage[CHI0_STAGE_CONTRACT].bytes;
      }
    }
  }
  c->stage[CHI0_STAGE_CONTRACT].flops = 4.0 * (double)ng * (ng + 1) * (double)c->nt * nw;
  if (!c->fp64) c->stage[CHI0_STAGE_CONTRACT].bytes = bytes;
  else c->stage[CHI0_STAGE_CONTRACT].bytes = (double)c->nt * ng * 16 + (double)c->nt * nw * 8;
  c->stage[CHI0_STAGE_WEIGHTS].bytes = (double)c->nt * nw * 8;
  (void)n2;
  return CHI0_OK;
}

// kernels of build_chi0 (weights, contraction, reduction, terminator)
chi0_status launch_chi0(chi0_ctx* c, const cudaEvent_t* ev_freq, const cudaEvent_t* ev_prep, bool defer_combine) {
  const int iq = c->plan_chi_iq;
  if (iq < 0) return fail(c, CHI0_ESTATE, "chi0 not planned");
  const int nw0 = c->cfg.nw, nw = c->nwv, ng = c->cfg.ng;
  const size_t n2 = (size_t)ng * ng;
  chi0_status s;
  if (c->nt == 0) {
    CK(cudaMemsetAsync(c->d_chi.p, 0, n2 * nw0 * 16, c->st), "zero chi0");
  } else if (c->grouped) {
    if ((s = chi0::tc_launch_grouped(c, (double2*)c->d_chi.p, ev_freq)) != CHI0_OK) return s;
    if (ev_prep)
      for (int v = 0; v < nw; ++v) cudaEventRecord(ev_prep[v], c->st);
  } else if (c->stream_nb > 0) {
    if ((s = launch_chi0_streamed(c)) != CHI0_OK) return s;
    if (c->has_real && !defer_combine) {
      double2* chiv = (double2*)c->d_chiv.p;
      chi0::stage_begin(c, CHI0_STAGE_REDUCE);
      cudaError_t e = chi0::launch_combine_freq(chiv, (const int*)c->d_vr.p, (const int*)c->d_vi.p, ng, nw0,
                                                (double2*)c->d_chi.p, c->st);
      if (e != cudaSuccess) return cuda_fail(c, e, "frequency combine launch");
      chi0::stage_end(c, CHI0_STAGE_REDUCE, 1);
    }
  } else {
    // the contraction's output: chi0 itself, or its parts H_r, H_i per real frequency
    double2* chiv = c->has_real ? (double2*)c->d_chiv.p : (double2*)c->d_chi.p;
    if ((s = launch_weights_stage(c)) != CHI0_OK) return s;
    cudaError_t e;
    c->stage[CHI0_STAGE_WEIGHTS].bytes = (double)c->nt * nw * 8;
    c->stage[CHI0_STAGE_WEIGHTS].flops = 6.0 * (double)c->nt * nw;
    // chi0 algorithmic flops (Hermitian half): 4 ng (ng + 1) nt per frequency
    c->stage[CHI0_STAGE_CONTRACT].flops = 4.0 * (double)ng * (ng + 1) * (double)c->nt * nw;
    c->stage[CHI0_STAGE_CONTRACT].bytes = (double)c->nt * ng * cplx_bytes(c) + (double)c->nt * nw * 8;
    c->stage[CHI0_STAGE_REDUCE].bytes = (double)n2 * nw * 16;
    c->stage[CHI0_STAGE_REDUCE].flops = 0;
    if (c->bg_on && (s = launch_bg(c)) != CHI0_OK) return s;
    const chi0::BgApply bga{(const double2*)c->d_bgP.p, (const int32_t*)c->d_bgidx.p, c->bg_nd};
    if (c->fp64) {
      chi0::stage_begin(c, CHI0_STAGE_CONTRACT);
      e = chi0::launch_chi0_fp64_partials((const double2*)c->d_R.p, (const double*)c->d_w.p, c->nt, ng,
                                          nw, c->kchunk, c->nchunks, (double2*)c->d_part.p, c->st);
      if (e != cudaSuccess) return cuda_fail(c, e, "chi0 fp64 launch");
      chi0::stage_end(c, CHI0_STAGE_CONTRACT, 1);
      chi0::stage_begin(c, CHI0_STAGE_REDUCE);
      e = chi0::launch_chi0_reduce((const double2*)c->d_part.p, c->nchunks, ng, nw, chiv, c->st);
      if (e != cudaSuccess) return cuda_fail(c, e, "chi0 reduce launch");
      chi0::stage_end(c, CHI0_STAGE_REDUCE, 1);
      c->stage[CHI0_STAGE_REDUCE].bytes += (double)n2 * nw * c->nchunks * 16;
      if (c->bg_on) {
        chi0::stage_begin(c, CHI0_STAGE_REDUCE);
        e = chi0::launch_bg_apply(bga.P, bga.didx, ng, bga.nd, nw, chiv, c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "extrapolar term launch");
        chi0::stage_end(c, CHI0_STAGE_REDUCE, 1);
      }
    } else {
      s = chi0::tc_launch(c, c->d_R.p, (const double*)c->d_w.p, c->nt, ng, nw, chiv,
                          c->term_params ? nullptr : ev_freq, c->term_params ? nullptr : ev_prep,
                          c->bg_on ? &bga : nullptr, c->has_real ? c->h_vkind.data() : nullptr);
      if (s != CHI0_OK) return s;
    }
    if (c->has_real && !defer_combine) {
      chi0::stage_begin(c, CHI0_STAGE_REDUCE);
      e = chi0::launch_combine_freq(chiv, (const int*)c->d_vr.p, (const int*)c->d_vi.p, ng, nw0,
                                    (double2*)c->d_chi.p, c->st);
      if (e != cudaSuccess) return cuda_fail(c, e, "frequency combine launch");
      chi0::stage_end(c, CHI0_STAGE_REDUCE, 1);
    }
    if (c->term_params) {
      s = chi0::term_launch(c, (double2*)c->d_chi.p);
      if (s != CHI0_OK) return s;
    }
  }
  c->chi_iq = iq;
  c->eps_iq = -1;
  return CHI0_OK;
}

chi0_status plan_eps(chi0_ctx* c, int iq, double2* A) {
  if (iq != c->plan_chi_iq || iq < 0) return fail(c, CHI0_ESTATE, "chi0_build_chi0(%d) must come first", iq);
  if (c->eps_planned_epoch == c->plan_epoch && c->plan_eps_iq == iq && c->plan_eps_out == A &&
      c->eps_for_chi_serial == c->chi_plan_serial)
    return CHI0_OK;
  const int nw = c->cfg.nw, ng = c->cfg.ng;
  chi0_status s;
  if ((s = ensure(c, c->d_vsqrt, (size_t)ng * 8, "coulomb")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_colp, (size_t)nw * ng * 32 * 16, "panels")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_rowp, (size_t)nw * ng * 32 * 16, "panels")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_pinv, (size_t)nw * 32 * 32 * 16, "pivot blocks")) != CHI0_OK) return s;
  std::vector<double> v(ng);
  int64_t qi[3];
  q_integers(c, iq, qi);
  for (int i = 0; i < ng; ++i) {
    double q2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double comp = (double)qi[d] / c->cfg.kgrid[d] + c->h_gresp[3 * i + d];
      q2 += comp * comp;
    }
    const double qg = (2.0 * M_PI / c->a) * std::sqrt(q2);
    if (qg == 0.0) return fail(c, CHI0_EINVAL, "|q+G| = 0: bare Coulomb interaction diverges");
    v[i] = std::sqrt(4.0 * M_PI) / qg;
  }
  CK(cudaMemcpyAsync(c->d_vsqrt.p, v.data(), ng * 8, cudaMemcpyHostToDevice, c->st), "v H2D");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  CK(chi0::dyson_prepare(), "Dyson kernel attributes");
  if (!c->s_ct) {
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
    // The Dyson blocks go first whenever they are pending: blocks of a
    // lower-priority grid are only dispatched while no higher-priority block
    // waits, so at the lower priority the Dyson step would run only in the
    // gaps between contraction launches.
    CK(cudaStreamCreateWithPriority(&c->s_ct, cudaStreamNonBlocking, least), "pipeline stream");
    CK(cudaStreamCreateWithPriority(&c->s_dy, cudaStreamNonBlocking, greatest), "pipeline stream");
    CK(cudaStreamCreateWithPriority(&c->s_dy2, cudaStreamNonBlocking, greatest), "pipeline stream");
    cudaEvent_t* evs[] = {&c->ev_fork, &c->ev_join_ct, &c->ev_join_dy, &c->ev_join_dy2};
    for (cudaEvent_t* e : evs) CK(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "pipeline event");
  }
  // one event per entry of the contraction's frequency list
  while ((int)c->ev_freq.size() < std::max(nw, c->nwv)) {
    cudaEvent_t e = nullptr, f = nullptr;
    CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "pipeline event");
    c->ev_freq.push_back(e);
    CK(cudaEventCreateWithFlags(&f, cudaEventDisableTiming), "pipeline event");
    c->ev_prep.push_back(f);
  }
  c->plan_eps_out = A;
  c->plan_eps_iq = iq;
  c->eps_planned_epoch = c->plan_epoch;
  c->eps_for_chi_serial = c->chi_plan_serial;
  return CHI0_OK;
}

// kernels of invert_eps (eps~ and the Gauss-Jordan inverse into the planned output)
chi0_status launch_eps(chi0_ctx* c) {
  const int iq = c->plan_eps_iq;
  if (iq < 0) return fail(c, CHI0_ESTATE, "Dyson step not planned");
  const int nw = c->cfg.nw, ng = c->cfg.ng;
  const size_t n2 = (size_t)ng * ng;
  chi0::stage_begin(c, CHI0_STAGE_DYSON);
  // runs of imaginary-axis frequencies (Hermitian eps~) and of real-axis ones
  // (general eps~), each run in one launch sequence
  int nlaunch = 0;
  for (int i0 = 0; i0 < nw;) {
    const bool general = c->has_real && c->h_vi[i0] >= 0;
    int i1 = i0 + 1;
    while (i1 < nw && (c->has_real && c->h_vi[i1] >= 0) == general) ++i1;
    const double2* chi = (const double2*)c->d_chi.p + (size_t)i0 * n2;
    double2* out = c->plan_eps_out + (size_t)i0 * n2;
    cudaError_t e = general
        ? chi0::launch_dyson_general(chi, (const double*)c->d_vsqrt.p, ng, i1 - i0, out, (double2*)c->d_colp.p,
                                     (double2*)c->d_rowp.p, (double2*)c->d_pinv.p, (int*)c->d_err.p, c->st)
        : chi0::launch_dyson(chi, (const double*)c->d_vsqrt.p, ng, i1 - i0, out, (double2*)c->d_colp.p,
                             (double2*)c->d_rowp.p, (double2*)c->d_pinv.p, (int*)c->d_err.p, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "dyson launch");
    nlaunch += (general ? 1 : 2) + 3 * ((ng + 31) / 32);
    i0 = i1;
  }
  chi0::stage_end(c, CHI0_STAGE_DYSON, nlaunch);
  // Gauss-Jordan inversion: ng^3 complex multiply-adds per frequency (about
  // half of them executed, the Hermitian lower tiles)
  c->stage[CHI0_STAGE_DYSON].flops = 8.0 * (double)ng * ng * ng * nw;
  c->stage[CHI0_STAGE_DYSON].bytes = 2.0 * (double)n2 * nw * 16;
  c->eps_iq = iq;
  return CHI0_OK;
}

chi0_status launch_chi0_eps(chi0_ctx* c, void* host_out, bool* copied) {
  const int iq = c->plan_chi_iq;
  if (copied) *copied = false;
  if (iq < 0 || c->plan_eps_iq != iq) return fail(c, CHI0_ESTATE, "build and Dyson step not planned");
  const int nw = c->cfg.nw, ng = c->cfg.ng;
  chi0_status s;
  if (c->fp64 || c->term_params || c->nt == 0 || nw < 2 || c->stream_nb > 0) {
    // FP64 contraction and Dyson share the FP64 pipe; the learned terminator
    // needs every frequency of chi0 first: no overlap to gain
    if ((s = launch_chi0(c)) != CHI0_OK) return s;
    return launch_eps(c);
  }
  const size_t n2 = (size_t)ng * ng;
  cudaStream_t base = c->st;
  cudaEventRecord(c->ev_fork, base);
  cudaStreamWaitEvent(c->s_ct, c->ev_fork, 0);
  cudaStreamWaitEvent(c->s_dy, c->ev_fork, 0);
  cudaStreamWaitEvent(c->s_dy2, c->ev_fork, 0);
  c->st = c->s_ct;
  s = launch_chi0(c, c->ev_freq.data(), c->ev_prep.data(), /*defer_combine=*/true);
  // Dyson steps in groups of 4 frequencies: the pivot-block inverses of a
  // group run side by side (one SM each), which a single frequency's chain
  // of 32 dependent pivot steps cannot hide.  The last four frequencies go
  // as 2, 1, 1, so that after the last contraction only one frequency's
  // Dyson step is left.  A group holds frequencies of one kind (imaginary
  // axis: Hermitian eps~; real axis: general eps~, whose chi0 is first
  // combined from its two contractions H_r + i H_i).
  // Consecutive groups alternate between two Dyson streams, each with its
  // own panel scratch (the group's slice of the per-frequency buffers), so
  // that the pivot-block inverses of one group (one SM per matrix) overlap
  // the rank-32 updates of the other.
  const int nT = (ng + 31) / 32;
  int grp = 0;
  auto general = [&](int iw) { return c->has_real && c->h_vi[iw] >= 0; };
  auto first_v = [&](int iw) { return c->has_real ? c->h_vr[iw] : iw; };   // list entries of frequency iw
  auto last_v = [&](int iw) { return general(iw) ? c->h_vi[iw] : first_v(iw); };
  for (int w0 = 0; w0 < nw && s == CHI0_OK;) {
    const int r = nw - w0;
    int gw = r > 4 ? std::min(4, r - 4) : (r == 4 ? 2 : 1);
    for (int g = 1; g < gw; ++g)
      if (general(w0 + g) != general(w0)) {
        gw = g;
        break;
      }
    c->st = (grp++ & 1) ? c->s_dy2 : c->s_dy;
    cudaStreamWaitEvent(c->st, c->ev_freq[last_v(w0 + gw - 1)], 0);
    // and, when a split pass follows, until it is done: the Dyson blocks then
    // share the SMs with the (tensor-bound) contraction, not with the
    // (bandwidth-bound) split
    if (w0 + gw < nw) cudaStreamWaitEvent(c->st, c->ev_prep[first_v(w0 + gw)], 0);
    cudaError_t e = cudaSuccess;
    if (c->has_real) {
      chi0::stage_begin(c, CHI0_STAGE_REDUCE);
      e = chi0::launch_combine_freq((const double2*)c->d_chiv.p, (const int*)c->d_vr.p + w0,
                                    (const int*)c->d_vi.p + w0, ng, gw, (double2*)c->d_chi.p + w0 * n2, c->st);
      chi0::stage_end(c, CHI0_STAGE_REDUCE, 1);
      if (e != cudaSuccess) s = cuda_fail(c, e, "frequency combine launch");
    }
    if (s != CHI0_OK) break;
    chi0::stage_begin(c, CHI0_STAGE_DYSON);
    const double2* chi = (const double2*)c->d_chi.p + w0 * n2;
    double2* out = c->plan_eps_out + w0 * n2;
    double2* colp = (double2*)c->d_colp.p + (size_t)w0 * ng * 32;
    double2* rowp = (double2*)c->d_rowp.p + (size_t)w0 * ng * 32;
    double2* pinv = (double2*)c->d_pinv.p + (size_t)w0 * 32 * 32;
    e = general(w0) ? chi0::launch_dyson_general(chi, (const double*)c->d_vsqrt.p, ng, gw, out, colp, rowp, pinv,
                                                 (int*)c->d_err.p, c->st)
                    : chi0::launch_dyson(chi, (const double*)c->d_vsqrt.p, ng, gw, out, colp, rowp, pinv,
                                         (int*)c->d_err.p, c->st);
    if (e != cudaSuccess) s = cuda_fail(c, e, "dyson launch");
    chi0::stage_end(c, CHI0_STAGE_DYSON, (general(w0) ? 1 : 2) + 3 * nT);
    // a host output receives each group as soon as it is inverted, so that
    // only the last group's copy follows the last contraction
    if (s == CHI0_OK && host_out) {
      e = cudaMemcpyAsync((char*)host_out + (size_t)w0 * n2 * 16, out, (size_t)gw * n2 * 16,
                          cudaMemcpyDeviceToHost, c->st);
      if (e != cudaSuccess) s = cuda_fail(c, e, "eps copy out");
    }
    w0 += gw;
  }
  c->st = base;
  // join (also on failure, so that a capture stays well formed)
  cudaEventRecord(c->ev_join_ct, c->s_ct);
  cudaEventRecord(c->ev_join_dy, c->s_dy);
  cudaEventRecord(c->ev_join_dy2, c->s_dy2);
  cudaStreamWaitEvent(base, c->ev_join_ct, 0);
  cudaStreamWaitEvent(base, c->ev_join_dy, 0);
  cudaStreamWaitEvent(base, c->ev_join_dy2, 0);
  if (s != CHI0_OK) return s;
  c->stage[CHI0_STAGE_DYSON].flops = 8.0 * (double)ng * ng * ng * nw;
  c->stage[CHI0_STAGE_DYSON].bytes = 2.0 * (double)n2 * nw * 16;
  c->eps_iq = iq;
  if (copied) *copied = host_out != nullptr;
  return CHI0_OK;
}

chi0_ctx* make_problem_ctx(const chi0_ctx* base) {
  chi0_ctx* c = new (std::nothrow) chi0_ctx();
  if (!c) return nullptr;
  c->cfg = base->cfg;
  c->q = base->q;
  c->om = base->om;
  c->cfg.q_frac = c->q.data();
  c->cfg.omega = c->om.data();
  c->nk = base->nk;
  c->nb = base->nb;
  c->npw_max = base->npw_max;
  c->a = base->a;
  c->omega_cell = base->omega_cell;
  c->st = base->st;
  c->fp64 = base->fp64;
  c->h_npw = base->h_npw;
  c->h_gvec = base->h_gvec;
  c->wf_set = base->wf_set;
  c->h_eps = base->h_eps;
  c->h_occ = base->h_occ;
  c->energies_set = base->energies_set;
  const DevBuf* src[] = {&base->d_gvec, &base->d_npw, &base->d_coef, &base->d_eps, &base->d_occ, &base->d_epsd};
  DevBuf* dst[] = {&c->d_gvec, &c->d_npw, &c->d_coef, &c->d_eps, &c->d_occ, &c->d_epsd};
  for (int i = 0; i < 6; ++i) *dst[i] = DevBuf{src[i]->p, src[i]->bytes, true};
  c->term_params = base->term_params;
  c->term_bf16 = base->term_bf16;
  c->bg_on = base->bg_on;
  c->bg_eps = base->bg_eps;
  c->grp_thresh = base->grp_thresh;
  c->dg_nd = base->dg_nd;
  return c;
}

std::vector<DevBuf*> scratch_slots(chi0_ctx* c) {
  std::vector<DevBuf*> v = {&c->d_w, &c->d_part, &c->d_chi, &c->d_chiv, &c->d_colp, &c->d_rowp, &c->d_pinv,
                            &c->d_termx, &c->d_termy};
  for (DevBuf* b : tc_scratch_slots(c)) v.push_back(b);
  return v;
}

}  // namespace chi0

extern "C" {

chi0_status chi0_create(const chi0_config* cfg, chi0_ctx** out) {
  if (!out) return CHI0_EINVAL;
  *out = nullptr;
  if (!cfg) return CHI0_EINVAL;
  chi0_ctx* c = new (std::nothrow) chi0_ctx();
  if (!c) return CHI0_ENOMEM;
  chi0_status s = CHI0_OK;
  auto bad = [&](chi0_status st, const char* m) {
    s = st;
    c->err = m;
  };
  const double a = cfg->lattice[0][0];
  for (int i = 0; i < 3 && s == CHI0_OK; ++i)
    for (int j = 0; j < 3; ++j)
      if (std::fabs(cfg->lattice[i][j] - (i == j ? a : 0.0)) > 1e-12 * std::fabs(a))
        bad(CHI0_EUNSUPPORTED, "only cubic cells a*I are supported");
  if (s == CHI0_OK && !(a > 0)) bad(CHI0_EINVAL, "lattice constant must be positive");
  for (int d = 0; d < 3 && s == CHI0_OK; ++d) {
    if (cfg->kgrid[d] < 1 || cfg->kgrid[d] > 1024) bad(CHI0_EINVAL, "kgrid out of range");
    if (cfg->fft[d] < 2 || cfg->fft[d] > 4096) bad(CHI0_EINVAL, "fft grid out of range");
  }
  if (s == CHI0_OK && (cfg->nbands < 1 || cfg->npw_max < 1 || cfg->ng < 1 || cfg->ng > 4096 ||
                       cfg->nq < 1 || cfg->nw < 1 || !cfg->q_frac || !cfg->omega))
    bad(CHI0_EINVAL, "nbands/npw_max/ng/nq/nw out of range or NULL q_frac/omega");
  if (s == CHI0_OK && cfg->time_reversal != 1)
    bad(CHI0_EUNSUPPORTED, "only time-reversal-symmetric inputs are supported");
  if (s == CHI0_OK && cfg->precision != CHI0_FP64 && cfg->precision != CHI0_MIXED_BF16X3)
    bad(CHI0_EINVAL, "unknown precision");
  if (s == CHI0_OK && (cfg->occ_drop_tol < 0 || cfg->eta < 0 || !(cfg->spin_factor > 0)))
    bad(CHI0_EINVAL, "occ_drop_tol, eta must be >= 0 and spin_factor > 0");
  if (s != CHI0_OK) {
    // the handle is not returned; the message cannot be read back
    delete c;
    return s;
  }
  c->cfg = *cfg;
  c->q.assign(cfg->q_frac, cfg->q_frac + 3 * cfg->nq);
  c->om.assign(cfg->omega, cfg->omega + 2 * cfg->nw);
  c->cfg.q_frac = nullptr;
  c->cfg.omega = nullptr;
  c->nk = cfg->kgrid[0] * cfg->kgrid[1] * cfg->kgrid[2];
  c->nb = cfg->nbands;
  c->npw_max = cfg->npw_max;
  c->a = a;
  c->omega_cell = a * a * a;
  c->st = (cudaStream_t)cfg->cuda_stream;
  c->fp64 = cfg->precision == CHI0_FP64;
  for (int iq = 0; iq < cfg->nq; ++iq) {
    int64_t qi[3];
    if (!q_integers(c, iq, qi)) {
      delete c;
      return CHI0_EINVAL;
    }
  }
  c->h_npw.assign(c->nk, 0);
  c->h_gvec.assign((size_t)c->nk * c->npw_max * 3, 0);
  c->wf_set.assign(c->nk, 0);
  *out = c;
  return CHI0_OK;
}

chi0_status chi0_set_wavefunctions(chi0_ctx* c, int ik, int npw, const int32_t* gvec,
                                   const void* coef, int coef_is_c64, int on_device) {
  if (!c) return CHI0_EINVAL;
  if (ik < 0 || ik >= c->nk) return fail(c, CHI0_EINVAL, "ik %d out of range", ik);
  if (npw < 1 || npw > c->npw_max) return fail(c, CHI0_EINVAL, "npw %d out of range", npw);
  if (!gvec || !coef) return fail(c, CHI0_EINVAL, "NULL gvec or coef");
  chi0_status s;
  const size_t cb = cplx_bytes(c);
  if ((s = ensure(c, c->d_coef, (size_t)c->nk * c->nb * c->npw_max * cb, "coefficients")) != CHI0_OK)
    return s;
  if ((s = ensure(c, c->d_gvec, (size_t)c->nk * c->npw_max * 3 * 4, "gvec")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_npw, (size_t)c->nk * 4, "npw")) != CHI0_OK) return s;
  // Miller indices: keep a host copy (sphere extents, alias checks)
  int32_t* hg = c->h_gvec.data() + (size_t)ik * c->npw_max * 3;
  std::vector<int32_t> incoming((size_t)npw * 3);
  if (on_device) {
    CK(cudaMemcpyAsync(incoming.data(), gvec, (size_t)npw * 12, cudaMemcpyDeviceToHost, c->st), "gvec D2H");
    CK(cudaStreamSynchronize(c->st), "synchronize");
  } else {
    std::memcpy(incoming.data(), gvec, (size_t)npw * 12);
  }
  for (int p = 0; p < npw * 3; ++p)
    if (incoming[p] < -1000 || incoming[p] > 1000) return fail(c, CHI0_EINVAL, "Miller index out of range");
  // a new sphere (or a first one) invalidates the plans; new coefficient
  // values on the same sphere do not, and then the Miller indices and the
  // zero padding on the device are already in place
  const bool new_sphere =
      !c->wf_set[ik] || c->h_npw[ik] != npw || std::memcmp(hg, incoming.data(), (size_t)npw * 12) != 0;
  const bool same = (coef_is_c64 != 0) == !c->fp64;
  char* dst = (char*)c->d_coef.p + (size_t)ik * c->nb * c->npw_max * cb;
  // a copy of this k point still queued on the upload stream comes first
  if (!c->ev_up.empty() && !(same && !on_device && !new_sphere))
    CK(cudaStreamWaitEvent(c->st, c->ev_up[ik], 0), "upload wait");
  if (new_sphere) {
    ++c->plan_epoch;
    std::memcpy(hg, incoming.data(), (size_t)npw * 12);
    std::memset(hg + (size_t)npw * 3, 0, (size_t)(c->npw_max - npw) * 12);
    c->h_npw[ik] = npw;
    CK(cudaMemcpyAsync((char*)c->d_gvec.p + (size_t)ik * c->npw_max * 12, hg,
                       (size_t)c->npw_max * 12, cudaMemcpyHostToDevice, c->st),
       "gvec H2D");
    CK(cudaMemcpyAsync((char*)c->d_npw.p + (size_t)ik * 4, &c->h_npw[ik], 4, cudaMemcpyHostToDevice,
                       c->st),
       "npw H2D");
    // coefficients: rows of npw, padded to npw_max
    CK(cudaMemsetAsync(dst, 0, (size_t)c->nb * c->npw_max * cb, c->st), "zero coefficients");
  }
  if (same && !on_device && !new_sphere) {
    // new values on the same sphere: copy on the upload stream (see s_up)
    if (!c->s_up) CK(cudaStreamCreateWithFlags(&c->s_up, cudaStreamNonBlocking), "upload stream");
    if (!c->ev_wf_done) {   // the first copy waits for everything queued on the context's stream
      CK(cudaEventCreateWithFlags(&c->ev_wf_done, cudaEventDisableTiming), "upload event");
      CK(cudaEventRecord(c->ev_wf_done, c->st), "upload event");
    }
    if (c->ev_up.empty()) {
      c->ev_up.assign(c->nk, nullptr);
      c->up_seq.assign(c->nk, -1);
      for (int k = 0; k < c->nk; ++k)
        CK(cudaEventCreateWithFlags(&c->ev_up[k], cudaEventDisableTiming), "upload event");
    }
    CK(cudaStreamWaitEvent(c->s_up, c->ev_wf_done, 0), "upload wait");
    CK(cudaMemcpy2DAsync(dst, (size_t)c->npw_max * cb, coef, (size_t)npw * cb, (size_t)npw * cb, c->nb,
                         cudaMemcpyHostToDevice, c->s_up),
       "coefficients copy");
    CK(cudaEventRecord(c->ev_up[ik], c->s_up), "upload event");
    c->up_seq[ik] = c->up_count++;
  } else if (same) {
    CK(cudaMemcpy2DAsync(dst, (size_t)c->npw_max * cb, coef, (size_t)npw * cb, (size_t)npw * cb,
                         c->nb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                         c->st),
       "coefficients copy");
  } else {
    // convert on the host (device sources are staged through the host)
    const size_t in_cb = coef_is_c64 ? 8 : 16;
    std::vector<char> src((size_t)c->nb * npw * in_cb);
    if (on_device) {
      CK(cudaMemcpyAsync(src.data(), coef, src.size(), cudaMemcpyDeviceToHost, c->st), "coef D2H");
      CK(cudaStreamSynchronize(c->st), "synchronize");
    } else {
      std::memcpy(src.data(), coef, src.size());
    }
    std::vector<char> conv((size_t)c->nb * npw * cb);
    const size_t n = (size_t)c->nb * npw * 2;
    if (coef_is_c64) {
      const float* f = (const float*)src.data();
      double* d = (double*)conv.data();
      for (size_t i = 0; i < n; ++i) d[i] = f[i];
    } else {
      const double* d = (const double*)src.data();
      float* f = (float*)conv.data();
      for (size_t i = 0; i < n; ++i) f[i] = (float)d[i];
    }
    CK(cudaMemcpy2DAsync(dst, (size_t)c->npw_max * cb, conv.data(), (size_t)npw * cb,
                         (size_t)npw * cb, c->nb, cudaMemcpyHostToDevice, c->st),
       "coefficients copy");
    CK(cudaStreamSynchronize(c->st), "synchronize");
  }
  c->wf_set[ik] = 1;
  c->rho_iq = c->chi_iq = c->eps_iq = -1;
  return CHI0_OK;
}

chi0_status chi0_set_energies(chi0_ctx* c, const double* eps, const double* occ) {
  if (!c) return CHI0_EINVAL;
  if (!eps || !occ) return fail(c, CHI0_EINVAL, "NULL eps or occ");
  const size_t n = (size_t)c->nk * c->nb;
  for (size_t i = 0; i < n; ++i) {
    if (!std::isfinite(eps[i])) return fail(c, CHI0_EINVAL, "non-finite energy at %zu", i);
    if (!(occ[i] >= 0.0 && occ[i] <= 1.0)) return fail(c, CHI0_EINVAL, "occupation outside [0,1] at %zu", i);
  }
  // changed energies or occupations invalidate the plans (the transition
  // set and the pole grouping are planned from them); unchanged ones are
  // already on the device
  if (c->energies_set && c->h_eps.size() == n && c->h_occ.size() == n &&
      std::memcmp(c->h_eps.data(), eps, n * 8) == 0 && std::memcmp(c->h_occ.data(), occ, n * 8) == 0)
    return CHI0_OK;
  ++c->plan_epoch;
  c->h_eps.assign(eps, eps + n);
  c->h_occ.assign(occ, occ + n);
  chi0_status s;
  if ((s = ensure(c, c->d_eps, n * 8, "eps")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_occ, n * 8, "occ")) != CHI0_OK) return s;
  CK(cudaMemcpyAsync(c->d_eps.p, c->h_eps.data(), n * 8, cudaMemcpyHostToDevice, c->st), "eps H2D");
  CK(cudaMemcpyAsync(c->d_occ.p, c->h_occ.data(), n * 8, cudaMemcpyHostToDevice, c->st), "occ H2D");
  c->energies_set = true;
  c->rho_iq = c->chi_iq = c->eps_iq = -1;
  return CHI0_OK;
}

chi0_status chi0_compute_rho(chi0_ctx* c, int iq) {
  if (!c) return CHI0_EINVAL;
  chi0_status s;
  if ((s = chi0::plan_rho(c, iq)) != CHI0_OK) return s;
  return chi0::launch_rho(c, true);
}

chi0_status chi0_build_chi0(chi0_ctx* c, int iq, void* out, int out_on_device) {
  if (!c) return CHI0_EINVAL;
  if (iq != c->rho_iq || iq < 0) return fail(c, CHI0_ESTATE, "chi0_compute_rho(%d) must come first", iq);
  chi0_status s;
  if ((s = chi0::plan_chi0(c, iq)) != CHI0_OK) return s;
  if ((s = chi0::launch_chi0(c)) != CHI0_OK) return s;
  if (out) {
    const size_t bytes = (size_t)c->cfg.ng * c->cfg.ng * c->cfg.nw * 16;
    CK(cudaMemcpyAsync(out, c->d_chi.p, bytes,
                       out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st),
       "chi0 copy out");
    if (!out_on_device) {
      CK(cudaStreamSynchronize(c->st), "synchronize");
      return check_device_error(c);
    }
  }
  return CHI0_OK;
}

chi0_status chi0_invert_eps(chi0_ctx* c, int iq, void* out, int out_on_device) {
  if (!c) return CHI0_EINVAL;
  if (iq != c->chi_iq || iq < 0) return fail(c, CHI0_ESTATE, "chi0_build_chi0(%d) must come first", iq);
  if (!out) return fail(c, CHI0_EINVAL, "NULL output");
  const size_t bytes = (size_t)c->cfg.ng * c->cfg.ng * c->cfg.nw * 16;
  chi0_status s;
  double2* A;
  if (out_on_device) {
    A = (double2*)out;
  } else {
    if ((s = ensure(c, c->d_A, bytes, "eps")) != CHI0_OK) return s;
    A = (double2*)c->d_A.p;
  }
  if ((s = chi0::plan_eps(c, iq, A)) != CHI0_OK) return s;
  if ((s = chi0::launch_eps(c)) != CHI0_OK) return s;
  if (!out_on_device) {
    CK(cudaMemcpyAsync(out, A, bytes, cudaMemcpyDeviceToHost, c->st), "eps copy out");
    CK(cudaStreamSynchronize(c->st), "synchronize");
    return check_device_error(c);
  }
  return CHI0_OK;
}

chi0_status chi0_build_invert(chi0_ctx* c, int iq, void* chi_out, void* eps_out, int out_on_device) {
  if (!c) return CHI0_EINVAL;
  if (iq != c->rho_iq || iq < 0) return fail(c, CHI0_ESTATE, "chi0_compute_rho(%d) must come first", iq);
  if (!eps_out) return fail(c, CHI0_EINVAL, "NULL output");
  const size_t bytes = (size_t)c->cfg.ng * c->cfg.ng * c->cfg.nw * 16;
  chi0_status s;
  double2* A;
  if (out_on_device) {
    A = (double2*)eps_out;
  } else {
    if ((s = ensure(c, c->d_A, bytes, "eps")) != CHI0_OK) return s;
    A = (double2*)c->d_A.p;
  }
  if ((s = chi0::plan_chi0(c, iq)) != CHI0_OK) return s;
  if ((s = chi0::plan_eps(c, iq, A)) != CHI0_OK) return s;
  bool copied = false;
  if ((s = chi0::launch_chi0_eps(c, out_on_device ? nullptr : eps_out, &copied)) != CHI0_OK) return s;
  const cudaMemcpyKind kind = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (chi_out) CK(cudaMemcpyAsync(chi_out, c->d_chi.p, bytes, kind, c->st), "chi0 copy out");
  if (!out_on_device) {
    if (!copied) CK(cudaMemcpyAsync(eps_out, A, bytes, cudaMemcpyDeviceToHost, c->st), "eps copy out");
    CK(cudaStreamSynchronize(c->st), "synchronize");
    return check_device_error(c);
  }
  return CHI0_OK;
}

chi0_status chi0_set_bg_terminator(chi0_ctx* c, int on, double eps_bar) {
  if (!c) return CHI0_EINVAL;
  if (on && !std::isfinite(eps_bar)) return fail(c, CHI0_EINVAL, "extrapolar energy must be finite");
  if (on && c->term_params)
    return fail(c, CHI0_EINVAL, "the learned terminator is set: the two corrections exclude each other");
  c->bg_on = on ? 1 : 0;
  c->bg_eps = eps_bar;
  ++c->plan_epoch;
  // the transition block changes (every band n): compute_rho must run again
  c->rho_iq = c->chi_iq = c->eps_iq = -1;
  c->plan_rho_iq = c->plan_chi_iq = c->plan_eps_iq = -1;
  return CHI0_OK;
}

chi0_status chi0_build_sigma_i(chi0_ctx* c, int iq, int qp_lo, int qp_hi, const void* eps_inv, int nw,
                               void* out, int out_on_device) {
  if (!c) return CHI0_EINVAL;
  if (iq < 0 || iq >= c->cfg.nq) return fail(c, CHI0_EINVAL, "iq %d out of range", iq);
  if (qp_lo < 0 || qp_hi > c->nb || qp_hi <= qp_lo)
    return fail(c, CHI0_EINVAL, "quasiparticle window [%d, %d) is empty or outside [0, %d)", qp_lo, qp_hi, c->nb);
  if (!eps_inv || !out || nw < 1) return fail(c, CHI0_EINVAL, "NULL eps~^-1 or output, or nw < 1");
  const int nqp = qp_hi - qp_lo;
  if (nqp > 64) return fail(c, CHI0_EUNSUPPORTED, "at most 64 bands in the quasiparticle window");
  if (iq != c->rho_iq) return fail(c, CHI0_ESTATE, "chi0_compute_rho(%d) must come first", iq);
  if (c->stream_nb > 0)
    return fail(c, CHI0_EUNSUPPORTED, "the self-energy kernel needs every band's mixed grids (no band-block streaming)");
  if (c->nt == 0)
    return fail(c, CHI0_ESTATE, "no transitions at this q: the mixed-grid wavefunctions were not built");
  const int ng = c->cfg.ng, nb = c->nb;
  const int64_t T = (int64_t)c->nk * nb * nqp;
  const size_t cb = cplx_bytes(c);
  chi0_status s;
  // rho geometry of the window: n in [qp_lo, qp_hi) at k, every band m at k - q
  RhoGeom& g = c->sig_geom;
  g = c->geom;
  g.n_lo = qp_lo;
  g.Nn = nqp;
  g.Nm = nb;
  g.diag = 0;
  const int64_t nI = (ng + 63) / 64, nJ = (T + 63) / 64;
  const size_t osz = (size_t)c->nk * nb * nqp * nqp * 16;   // I of one frequency
  if ((s = ensure(c, c->d_sigR, (size_t)T * ng * cb, "quasiparticle rho")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_sigY, (size_t)nI * nJ * 4096 * cb * 2, "W^delta rho* tiles")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_sigRT, (size_t)nI * nJ * 4096 * cb, "rho tiles")) != CHI0_OK) return s;
  if (!out_on_device && (s = ensure(c, c->d_sigI, osz, "I staging")) != CHI0_OK) return s;
  if ((s = ensure(c, c->d_vsqrt, (size_t)ng * 8, "coulomb")) != CHI0_OK) return s;
  if (c->fp64) {
    if ((s = ensure(c, c->d_sigWd, (size_t)ng * ng * 16, "W^delta")) != CHI0_OK) return s;
  } else if ((s = chi0::sig_tc_plan(c, T, ng)) != CHI0_OK) {
    return s;
  }
  if (!c->d_err.p) {
    if ((s = ensure(c, c->d_err, 16, "error flag")) != CHI0_OK) return s;
    CK(cudaMemsetAsync(c->d_err.p, 0, 16, c->st), "clear error flag");
  }
  // V_i = sqrt(4 pi) / |q + G_i| on the response set of iq
  {
    std::vector<double> v(ng);
    int64_t qi[3];
    q_integers(c, iq, qi);
    for (int i = 0; i < ng; ++i) {
      double q2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double comp = (double)qi[d] / c->cfg.kgrid[d] + c->h_gresp[3 * i + d];
        q2 += comp * comp;
      }
      const double qg = (2.0 * M_PI / c->a) * std::sqrt(q2);
      if (qg == 0.0) return fail(c, CHI0_EINVAL, "|q+G| = 0: bare Coulomb interaction diverges");
      v[i] = std::sqrt(4.0 * M_PI) / qg;
    }
    CK(cudaMemcpyAsync(c->d_vsqrt.p, v.data(), (size_t)ng * 8, cudaMemcpyHostToDevice, c->st), "v H2D");
    CK(cudaStreamSynchronize(c->st), "synchronize");
  }
  cudaError_t e;
  chi0::stage_begin(c, CHI0_STAGE_RHO);
  if (c->fp64)
    e = chi0::launch_rho_pairs<double, double2>(g, (const double2*)c->d_U.p, (const int32_t*)c->d_kq.p,
                                                (const int32_t*)c->d_g0.p, (const int32_t*)c->d_gresp.p,
                                                (const int32_t*)c->d_gperm.p, (const double2*)c->d_tw1.p,
                                                (const double2*)c->d_tw2.p, (double2*)c->d_sigR.p, c->st);
  else
    e = chi0::launch_rho_pairs<float, float2>(g, (const float2*)c->d_U.p, (const int32_t*)c->d_kq.p,
                                              (const int32_t*)c->d_g0.p, (const int32_t*)c->d_gresp.p,
                                              (const int32_t*)c->d_gperm.p, (const float2*)c->d_tw1.p,
                                              (const float2*)c->d_tw2.p, (float2*)c->d_sigR.p, c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "quasiparticle rho launch");
  e = c->fp64 ? chi0::launch_sig_rhot<double2>((const double2*)c->d_sigR.p, T, nqp, nb, ng, (double2*)c->d_sigRT.p,
                                               c->st)
              : chi0::launch_sig_rhot<float2>((const float2*)c->d_sigR.p, T, nqp, nb, ng, (float2*)c->d_sigRT.p,
                                              c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "rho tile copy launch");
  chi0::stage_end(c, CHI0_STAGE_RHO, 2);
  if (!c->fp64) {
    chi0::stage_begin(c, CHI0_STAGE_WEIGHTS);
    if ((e = chi0::sig_tc_split_b(c, (const float2*)c->d_sigR.p, nqp, nb)) != cudaSuccess)
      return cuda_fail(c, e, "rho split launch");
    chi0::stage_end(c, CHI0_STAGE_WEIGHTS, 1);
  }
  const double pref = -1.0 / ((double)c->nk * c->omega_cell);   // Eq. (I_c)
  const size_t n2 = (size_t)ng * ng;
  const double* v = (const double*)c->d_vsqrt.p;
  void* Y = c->d_sigY.p;   // FP64 (FP64 form) or FP32 (mixed form) tiles
  for (int iw = 0; iw < nw; ++iw) {
    const double2* E = (const double2*)eps_inv + iw * n2;
    double2* I = out_on_device ? (double2*)((char*)out + iw * osz) : (double2*)c->d_sigI.p;
    chi0::stage_begin(c, CHI0_STAGE_WEIGHTS);
    e = c->fp64 ? chi0::launch_sig_wd64(E, v, ng, (double2*)c->d_sigWd.p, c->st) : chi0::sig_tc_split_a(c, E, v);
    if (e != cudaSuccess) return cuda_fail(c, e, "W^delta launch");
    chi0::stage_end(c, CHI0_STAGE_WEIGHTS, 1);
    chi0::stage_begin(c, CHI0_STAGE_CONTRACT);
    e = c->fp64 ? chi0::launch_sig_gemm64((const double2*)c->d_sigWd.p, (const double2*)c->d_sigR.p, ng, T, nqp, nb,
                                          (double2*)Y, c->st)
                : chi0::sig_tc_contract(c, (float2*)Y);
    if (e != cudaSuccess) return cuda_fail(c, e, "W^delta rho* contraction launch");
    chi0::stage_end(c, CHI0_STAGE_CONTRACT, 1);
    chi0::stage_begin(c, CHI0_STAGE_REDUCE);
    e = c->fp64 ? chi0::launch_sig_dot<double2, double2>((const double2*)c->d_sigRT.p, (const double2*)Y, ng, T, nqp,
                                                         pref, I, c->st)
                : chi0::launch_sig_dot<float2, float2>((const float2*)c->d_sigRT.p, (const float2*)Y, ng, T, nqp, pref,
                                                       I, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "I launch");
    chi0::stage_end(c, CHI0_STAGE_REDUCE, 1);
    if (!out_on_device)
      CK(cudaMemcpyAsync((char*)out + iw * osz, I, osz, cudaMemcpyDeviceToHost, c->st), "I copy out");
  }
  // algorithmic work of the last call: rho of the window, one complex
  // contraction of N_G^2 T multiply-adds and one of N_G T nqp per frequency
  c->stage[CHI0_STAGE_RHO].bytes = (double)T * ng * cb;
  c->stage[CHI0_STAGE_CONTRACT].flops = 8.0 * (double)ng * ng * (double)T * nw;
  c->stage[CHI0_STAGE_CONTRACT].bytes = ((double)ng * ng * 16 + (double)T * ng * cb + (double)T * ng * 2 * cb) * nw;
  c->stage[CHI0_STAGE_REDUCE].flops = 8.0 * (double)ng * (double)T * nqp * nw;
  c->stage[CHI0_STAGE_REDUCE].bytes = ((double)T * ng * 2 * cb + (double)osz) * nw;
  if (!out_on_device) {
    CK(cudaStreamSynchronize(c->st), "synchronize");
    return check_device_error(c);
  }
  return CHI0_OK;
}

chi0_status chi0_set_band_blocks(chi0_ctx* c, int bands_per_block, int k_per_block) {
  if (!c) return CHI0_EINVAL;
  if (bands_per_block < 0 || k_per_block < 0)
    return fail(c, CHI0_EINVAL, "band and k block sizes must be >= 0");
  c->stream_nb = bands_per_block;
  c->stream_nk = bands_per_block > 0 ? k_per_block : 0;
  ++c->plan_epoch;
  c->rho_iq = c->chi_iq = c->eps_iq = -1;
  c->plan_rho_iq = c->plan_chi_iq = c->plan_eps_iq = -1;
  return CHI0_OK;
}

chi0_status chi0_get_pole_groups(chi0_ctx* c, int64_t* ngroups, int* grouped_contraction) {
  if (!c) return CHI0_EINVAL;
  if (c->plan_chi_iq < 0) return fail(c, CHI0_ESTATE, "no chi0 planned yet");
  if (ngroups) *ngroups = c->grp_thresh > 0.0 ? c->ngroups : 0;
  if (grouped_contraction) *grouped_contraction = c->grouped ? 1 : 0;
  return CHI0_OK;
}

chi0_status chi0_set_pole_grouping(chi0_ctx* c, double eps_thresh) {
  if (!c) return CHI0_EINVAL;
  if (!std::isfinite(eps_thresh) || eps_thresh < 0.0)
    return fail(c, CHI0_EINVAL, "degeneracy threshold must be finite and >= 0");
  if (eps_thresh > 0.0 && c->dg_nd > 0)
    return fail(c, CHI0_EINVAL, "the double grid is set: pole grouping and the double grid exclude each other");
  if (eps_thresh != c->grp_thresh) ++c->plan_epoch;
  c->grp_thresh = eps_thresh;
  return CHI0_OK;
}

chi0_status chi0_set_double_grid(chi0_ctx* c, int nd, const double* eps_dense) {
  if (!c) return CHI0_EINVAL;
  if (nd < 0 || nd > 4096 || (nd > 0 && !eps_dense)) return fail(c, CHI0_EINVAL, "nd out of range or NULL energies");
  if (nd > 0 && c->grp_thresh > 0.0)
    return fail(c, CHI0_EINVAL, "pole grouping is set: pole grouping and the double grid exclude each other");
  ++c->plan_epoch;
  if (nd == 0) {
    c->dg_nd = 0;
    return CHI0_OK;
  }
  const size_t n = (size_t)c->nk * nd * c->nb;
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(eps_dense[i])) return fail(c, CHI0_EINVAL, "dense-grid energy %zu not finite", i);
  chi0_status s = ensure(c, c->d_epsd, n * 8, "dense-grid energies");
  if (s != CHI0_OK) return s;
  CK(cudaMemcpyAsync(c->d_epsd.p, eps_dense, n * 8, cudaMemcpyHostToDevice, c->st), "dense energies H2D");
  CK(cudaStreamSynchronize(c->st), "synchronize");
  c->dg_nd = nd;
  return CHI0_OK;
}

chi0_status chi0_get_response_gvectors(chi0_ctx* c, int iq, int32_t* out) {
  if (!c) return CHI0_EINVAL;
  if (iq < 0 || iq >= c->cfg.nq || !out) return fail(c, CHI0_EINVAL, "bad iq or NULL out");
  std::vector<int32_t> g;
  response_set(c, iq, g);
  std::memcpy(out, g.data(), g.size() * 4);
  return CHI0_OK;
}

chi0_status chi0_get_transitions(chi0_ctx* c, int64_t* nt, int32_t* out) {
  if (!c) return CHI0_EINVAL;
  if (c->rho_iq < 0) return fail(c, CHI0_ESTATE, "no transitions before chi0_compute_rho");
  if (nt) *nt = c->nt;
  if (out) {
    int64_t t = 0;
    for (int ik = 0; ik < c->nk; ++ik)
      for (int n = 0; n < c->Nn; ++n)
        for (int m = 0; m < c->Nm; ++m, ++t) {
          out[3 * t] = ik;
          out[3 * t + 1] = c->n_lo + n;
          out[3 * t + 2] = m;
        }
  }
  return CHI0_OK;
}

chi0_status chi0_get_rho(chi0_ctx* c, void* out) {
  if (!c) return CHI0_EINVAL;
  if (c->rho_iq < 0) return fail(c, CHI0_ESTATE, "no rho before chi0_compute_rho");
  if (c->stream_nb > 0) return fail(c, CHI0_ESTATE, "rho is not kept when the transitions are streamed in band blocks");
  if (!out) return fail(c, CHI0_EINVAL, "NULL out");
  const size_t n = (size_t)c->nt * c->cfg.ng;
  if (n == 0) return CHI0_OK;
  if (c->fp64) {
    CK(cudaMemcpyAsync(out, c->d_R.p, n * 16, cudaMemcpyDeviceToHost, c->st), "rho D2H");
    CK(cudaStreamSynchronize(c->st), "synchronize");
  } else {
    std::vector<float2> tmp(n);
    CK(cudaMemcpyAsync(tmp.data(), c->d_R.p, n * 8, cudaMemcpyDeviceToHost, c->st), "rho D2H");
    CK(cudaStreamSynchronize(c->st), "synchronize");
    double2* o = (double2*)out;
    for (size_t i = 0; i < n; ++i) o[i] = make_double2(tmp[i].x, tmp[i].y);
  }
  return CHI0_OK;
}

chi0_status chi0_get_rho_rows(chi0_ctx* c, const int64_t* rows, int64_t nrows, void* out) {
  if (!c) return CHI0_EINVAL;
  if (c->rho_iq < 0) return fail(c, CHI0_ESTATE, "no rho before chi0_compute_rho");
  if (c->stream_nb > 0) return fail(c, CHI0_ESTATE, "rho is not kept when the transitions are streamed in band blocks");
  if (nrows < 0 || (nrows > 0 && (!rows || !out))) return fail(c, CHI0_EINVAL, "bad rows/out");
  const int ng = c->cfg.ng;
  const size_t cb = cplx_bytes(c);
  std::vector<char> tmp((size_t)ng * cb);
  double2* o = (double2*)out;
  for (int64_t r = 0; r < nrows; ++r) {
    if (rows[r] < 0 || rows[r] >= c->nt) return fail(c, CHI0_EINVAL, "row %lld out of range", (long long)rows[r]);
    CK(cudaMemcpyAsync(tmp.data(), (const char*)c->d_R.p + (size_t)rows[r] * ng * cb, (size_t)ng * cb,
                       cudaMemcpyDeviceToHost, c->st),
       "rho row D2H");
    CK(cudaStreamSynchronize(c->st), "synchronize");
    for (int i = 0; i < ng; ++i) {
      if (c->fp64) {
        o[(size_t)r * ng + i] = ((const double2*)tmp.data())[i];
      } else {
        const float2 v = ((const float2*)tmp.data())[i];
        o[(size_t)r * ng + i] = make_double2(v.x, v.y);
      }
    }
  }
  return CHI0_OK;
}

chi0_status chi0_check_bounded_wait(chi0_ctx* c) {
  if (!c) return CHI0_EINVAL;
  chi0_status s;
  if (!c->d_err.p) {
    if ((s = ensure(c, c->d_err, 16, "error flag")) != CHI0_OK) return s;
    CK(cudaMemsetAsync(c->d_err.p, 0, 16, c->st), "clear error flag");
  }
  cudaError_t e = chi0::launch_wait_probe((int*)c->d_err.p, c->st);
  if (e != cudaSuccess) return cuda_fail(c, e, "wait probe launch");
  return CHI0_OK;
}

chi0_status chi0_synchronize(chi0_ctx* c) {
  if (!c) return CHI0_EINVAL;
  if (c->s_up) CK(cudaStreamSynchronize(c->s_up), "synchronize");   // coefficient copies in flight
  CK(cudaStreamSynchronize(c->st), "synchronize");
  CK(cudaGetLastError(), "pending error");
  return check_device_error(c);
}

chi0_status chi0_get_stats(chi0_ctx* c, double* ms, double* bytes, double* flops,
                           int64_t* launches) {
  if (!c) return CHI0_EINVAL;
  CK(cudaStreamSynchronize(c->st), "synchronize");
  for (int k = 0; k < CHI0_NSTAGES; ++k) {
    auto& st = c->stage[k];
    if (st.used) {
      double tot = 0.0;
      for (size_t p = 0; p + 1 < st.used; p += 2) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, st.ev[p], st.ev[p + 1]) == cudaSuccess) tot += t;
        cudaGetLastError();
      }
      st.ms = tot;
      st.used = 0;
    } else {
      st.ms = 0.0;
    }
    if (ms) ms[k] = st.ms;
    if (bytes) bytes[k] = st.bytes;
    if (flops) flops[k] = st.flops;
  }
  if (launches) *launches = c->launches;
  return CHI0_OK;
}

const char* chi0_last_error(const chi0_ctx* c) {
  if (!c) return "NULL context";
  return c->err.c_str();
}

void chi0_destroy(chi0_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->st);
  DevBuf* bufs[] = {&c->d_gvec, &c->d_npw, &c->d_coef, &c->d_eps, &c->d_occ, &c->d_stage,
                    &c->d_gresp, &c->d_gperm, &c->d_kq, &c->d_g0, &c->d_tw1, &c->d_tw2, &c->d_U, &c->d_R,
                    &c->d_w, &c->d_part, &c->d_chi, &c->d_A, &c->d_colp, &c->d_rowp, &c->d_pinv,
                    &c->d_err, &c->d_vsqrt, &c->d_omim, &c->d_tc, &c->d_termx, &c->d_termy,
                    &c->d_termq, &c->d_termw, &c->d_termc, &c->d_bgd, &c->d_bgperm, &c->d_bgkq,
                    &c->d_bgg0, &c->d_bgrd, &c->d_bgw, &c->d_bgP, &c->d_bgidx, &c->d_sigR, &c->d_sigWd,
                    &c->d_sigY, &c->d_sigI, &c->d_sigRT, &c->d_dpole, &c->d_epsd, &c->d_Ublk,
                    &c->d_tperm, &c->d_grange, &c->d_ga, &c->d_gfac};
  for (DevBuf* b : bufs) release(*b);
  for (auto& st : c->stage)
    for (cudaEvent_t e : st.ev)
      if (e) cudaEventDestroy(e);
  chi0::tc_release(c);
  chi0::sig_tc_release(c);
  cudaStream_t pst[] = {c->s_ct, c->s_dy, c->s_dy2, c->s_up};
  for (cudaStream_t t : pst)
    if (t) {
      cudaStreamSynchronize(t);
      cudaStreamDestroy(t);
    }
  cudaEvent_t pev[] = {c->ev_fork, c->ev_join_ct, c->ev_join_dy, c->ev_join_dy2};
  for (cudaEvent_t e : pev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_freq)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_prep)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : c->ev_up)
    if (e) cudaEventDestroy(e);
  if (c->ev_wf_done) cudaEventDestroy(c->ev_wf_done);
  delete c;
}

}  // extern "C"
