// Learned band-sum terminator: a small network predicts the contribution of
// the bands left out of a truncated chi0.
//
// The paper corrects a band-truncated chi0 with the Bruneval-Gonze
// X-terminator (Eq. X_term_def, Appendix C): chi0 = chi0^trunc + Delta chi.
// Here Delta chi_{GG'}(w) is predicted per matrix entry from the features
//     x = (|q+G| / Kn, |q+G'| / Kn, Im w / Wn, Re chi0^trunc / c, Im chi0^trunc / c)
// (Kn = largest |q+G| of the response set, Wn = largest |Im w|, c = mean
// |chi0^trunc_GG(w_0)|), and the prediction c (y_0 + i y_1) is Hermitised
// before it is added.  The network: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 +
// b2), y = W3 h2 + b3 (5 -> 128 -> 128 -> 2); parameters packed as W1, b1,
// W2, b2, W3, b3 in FP32 (master copy).  In BF16 mode every matrix product
// takes BF16-rounded operands and accumulates in FP32.  Training: loss
// L = 1/(2B) sum (y - t)^2, gradients by backpropagation, Adam updates.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "ctx.cuh"

namespace chi0 {

namespace {

constexpr int kI = 5, kH = 128, kO = 2;
constexpr int kP = kH * kI + kH + kH * kH + kH + kO * kH + kO;  // 17538
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kI, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kO * kH;
constexpr int kS = 32;         // samples per block
constexpr int kThreads = 256;

__device__ __forceinline__ float rb(float v, int bf16) {
  return bf16 ? __bfloat162float(__float2bfloat16_rn(v)) : v;
}

// Forward (and optionally backward) for kS samples per block.  Gradients of
// the block go to part[block][kP] (summed later in a fixed order).
template <bool kBackward>
__global__ void __launch_bounds__(kThreads)
k_mlp(const float* __restrict__ prm, const float* __restrict__ x, const float* __restrict__ t,
      int64_t batch, int bf16, float* __restrict__ part, float* __restrict__ y_out,
      float* __restrict__ loss_part) {
  extern __shared__ float sm[];
  float* W2 = sm;                       // [H][H+1] (rounded)
  float* h1 = W2 + kH * (kH + 1);       // [S][H]
  float* h2 = h1 + kS * kH;             // [S][H]
  float* xs = h2 + kS * kH;             // [S][I]
  float* ys = xs + kS * kI;             // [S][O] -> dy
  float* dz2 = ys + kS * kO;            // [S][H]
  float* dz1 = dz2 + kS * kH;           // [S][H]
  float* red = dz1 + kS * kH;           // [kThreads]
  const int tid = threadIdx.x;
  const int64_t s0 = (int64_t)blockIdx.x * kS;
  const int ns = (batch - s0 < kS) ? (int)(batch - s0) : kS;
  for (int e = tid; e < kH * kH; e += kThreads) {
    const int r = e / kH, c = e % kH;
    W2[r * (kH + 1) + c] = rb(prm[kOffW2 + e], bf16);
  }
  for (int e = tid; e < kS * kI; e += kThreads) {
    const int s = e / kI;
    xs[e] = (s < ns) ? rb(x[(s0 + s) * kI + e % kI], bf16) : 0.f;
  }
  __syncthreads();
  // layer 1
  for (int e = tid; e < kS * kH; e += kThreads) {
    const int s = e / kH, h = e % kH;
    float z = prm[kOffB1 + h];
    for (int i = 0; i < kI; ++i) z = fmaf(rb(prm[kOffW1 + h * kI + i], bf16), xs[s * kI + i], z);
    h1[e] = tanhf(z);
  }
  __syncthreads();
  // layer 2
  for (int e = tid; e < kS * kH; e += kThreads) {
    const int s = e / kH, h = e % kH;
    float z = prm[kOffB2 + h];
    const float* w = W2 + h * (kH + 1);
    const float* a = h1 + s * kH;
    for (int k = 0; k < kH; ++k) z = fmaf(w[k], rb(a[k], bf16), z);
    h2[e] = tanhf(z);
  }
  __syncthreads();
  // layer 3
  for (int e = tid; e < kS * kO; e += kThreads) {
    const int s = e / kO, o = e % kO;
    float z = prm[kOffB3 + o];
    for (int k = 0; k < kH; ++k) z = fmaf(rb(prm[kOffW3 + o * kH + k], bf16), rb(h2[s * kH + k], bf16), z);
    ys[e] = z;
    if (!kBackward && s < ns) y_out[(s0 + s) * kO + o] = z;
  }
  if (!kBackward) return;
  __syncthreads();
  // loss and dy = (y - t) / B
  float lsum = 0.f;
  for (int e = tid; e < kS * kO; e += kThreads) {
    const int s = e / kO;
    float r = 0.f;
    if (s < ns) r = ys[e] - t[(s0 + s) * kO + e % kO];
    lsum += r * r;
    ys[e] = r / (float)batch;
  }
  red[tid] = lsum;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (tid < w) red[tid] += red[tid + w];
    __syncthreads();
  }
  if (tid == 0) loss_part[blockIdx.x] = 0.5f * red[0] / (float)batch;
  // dz2 = (dy W3) * (1 - h2^2)
  for (int e = tid; e < kS * kH; e += kThreads) {
    const int s = e / kH, h = e % kH;
    float g = 0.f;
    for (int o = 0; o < kO; ++o) g = fmaf(rb(ys[s * kO + o], bf16), rb(prm[kOffW3 + o * kH + h], bf16), g);
    const float hv = h2[e];
    dz2[e] = (s < ns) ? g * (1.f - hv * hv) : 0.f;
  }
  __syncthreads();
  // dz1 = (dz2 W2) * (1 - h1^2)
  for (int e = tid; e < kS * kH; e += kThreads) {
    const int s = e / kH, k = e % kH;
    float g = 0.f;
    for (int h = 0; h < kH; ++h) g = fmaf(rb(dz2[s * kH + h], bf16), W2[h * (kH + 1) + k], g);
    const float hv = h1[e];
    dz1[e] = (s < ns) ? g * (1.f - hv * hv) : 0.f;
  }
  __syncthreads();
  float* gp = part + (size_t)blockIdx.x * kP;
  // dW3[o][h] = sum_s dy[s][o] h2[s][h];  db3
  for (int e = tid; e < kO * kH; e += kThreads) {
    const int o = e / kH, h = e % kH;
    float g = 0.f;
    for (int s = 0; s < kS; ++s) g = fmaf(rb(ys[s * kO + o], bf16), rb(h2[s * kH + h], bf16), g);
    gp[kOffW3 + e] = g;
  }
  if (tid < kO) {
    float g = 0.f;
    for (int s = 0; s < kS; ++s) g += ys[s * kO + tid];
    gp[kOffB3 + tid] = g;
  }
  // dW2[h][k] = sum_s dz2[s][h] h1[s][k];  db2
  for (int e = tid; e < kH * kH; e += kThreads) {
    const int h = e / kH, k = e % kH;
    float g = 0.f;
    for (int s = 0; s < kS; ++s) g = fmaf(rb(dz2[s * kH + h], bf16), rb(h1[s * kH + k], bf16), g);
    gp[kOffW2 + e] = g;
  }
  for (int h = tid; h < kH; h += kThreads) {
    float g2 = 0.f, g1 = 0.f;
    for (int s = 0; s < kS; ++s) {
      g2 += dz2[s * kH + h];
      g1 += dz1[s * kH + h];
    }
    gp[kOffB2 + h] = g2;
    gp[kOffB1 + h] = g1;
  }
  // dW1[h][i] = sum_s dz1[s][h] x[s][i]
  for (int e = tid; e < kH * kI; e += kThreads) {
    const int h = e / kI, i = e % kI;
    float g = 0.f;
    for (int s = 0; s < kS; ++s) g = fmaf(rb(dz1[s * kH + h], bf16), xs[s * kI + i], g);
    gp[kOffW1 + e] = g;
  }
}

__global__ void k_mlp_reduce(const float* __restrict__ part, int nblk, const float* __restrict__ lpart,
                             float* __restrict__ grad, float* __restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kP) {
    float g = 0.f;
    for (int b = 0; b < nblk; ++b) g += part[(size_t)b * kP + p];
    grad[p] = g;
  }
  if (p == 0 && loss) {
    float l = 0.f;
    for (int b = 0; b < nblk; ++b) l += lpart[b];
    *loss = l;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  p[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

size_t mlp_smem() {
  return sizeof(float) * ((size_t)kH * (kH + 1) + 4 * (size_t)kS * kH + kS * kI + kS * kO + kThreads);
}

}  // namespace

int mlp_nparams() { return kP; }

cudaError_t mlp_loss_grad(const float* prm, const float* x, const float* t, int64_t batch, int bf16,
                          float* grad, float* loss, float* part, float* lpart, cudaStream_t st) {
  const int nblk = (int)((batch + kS - 1) / kS);
  const size_t smem = mlp_smem();
  cudaError_t e = cudaFuncSetAttribute(k_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_mlp<true><<<nblk, kThreads, smem, st>>>(prm, x, t, batch, bf16, part, nullptr, lpart);
  k_mlp_reduce<<<(kP + 255) / 256, 256, 0, st>>>(part, nblk, lpart, grad, loss);
  return cudaGetLastError();
}

cudaError_t mlp_predict(const float* prm, const float* x, int64_t batch, int bf16, float* y,
                        cudaStream_t st) {
  const int64_t nblk = (batch + kS - 1) / kS;
  const size_t smem = mlp_smem();
  cudaError_t e = cudaFuncSetAttribute(k_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_mlp<false><<<(unsigned)nblk, kThreads, smem, st>>>(prm, x, nullptr, batch, bf16, nullptr, y, nullptr);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* p, const float* g, float* m, float* v, int64_t n, float lr, float b1,
                     float b2, float eps, int step, cudaStream_t st) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace chi0

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace chi0 {
namespace {

// c = mean |chi_ii(w_0)| and 1/c (device, no host round trip)
__global__ void k_diag_scale(const double2* __restrict__ chi, int ng, double* __restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < ng; i += 256) {
    const double2 v = chi[(size_t)i * ng + i];
    s += sqrt(v.x * v.x + v.y * v.y);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double c = red[0] / ng;
    out[0] = c > 0.0 ? c : 1.0;
    out[1] = 1.0 / out[0];
  }
}

__global__ void k_term_features_dev(const double2* __restrict__ chi, const double2* __restrict__ full,
                                    const double* __restrict__ qgn, const double* __restrict__ wn,
                                    int ng, int nw, const double* __restrict__ cs, float* __restrict__ x,
                                    float* __restrict__ t) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n2 = (int64_t)ng * ng;
  if (e >= n2 * nw) return;
  const double inv_c = cs[1];
  const int iw = (int)(e / n2);
  const int64_t ij = e - iw * n2;
  const int i = (int)(ij / ng), j = (int)(ij % ng);
  const double2 c = chi[e];
  float* xo = x + e * kI;
  xo[0] = (float)qgn[i];
  xo[1] = (float)qgn[j];
  xo[2] = (float)wn[iw];
  xo[3] = (float)(c.x * inv_c);
  xo[4] = (float)(c.y * inv_c);
  if (full && t) {
    const double2 f = full[e];
    t[e * kO] = (float)((f.x - c.x) * inv_c);
    t[e * kO + 1] = (float)((f.y - c.y) * inv_c);
  }
}

__global__ void k_term_apply_dev(double2* __restrict__ chi, const float* __restrict__ y, int ng, int nw,
                                 const double* __restrict__ cs) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n2 = (int64_t)ng * ng;
  if (e >= n2 * nw) return;
  const double c = cs[0];
  const int iw = (int)(e / n2);
  const int64_t ij = e - iw * n2;
  const int i = (int)(ij / ng), j = (int)(ij % ng);
  const int64_t ji = (int64_t)iw * n2 + (int64_t)j * ng + i;
  const double dre = 0.5 * ((double)y[e * kO] + (double)y[ji * kO]);
  const double dim = 0.5 * ((double)y[e * kO + 1] - (double)y[ji * kO + 1]);
  double2 v = chi[e];
  v.x += c * dre;
  v.y += (i == j) ? 0.0 : c * dim;
  chi[e] = v;
}

// host tables of the feature normalisation for q point iq
void term_tables(chi0_ctx* c, int iq, std::vector<double>& qgn, std::vector<double>& wn) {
  const int ng = c->cfg.ng, nw = c->cfg.nw;
  qgn.resize(ng);
  wn.resize(nw);
  double qmax = 0.0;
  for (int i = 0; i < ng; ++i) {
    double q2 = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double comp = c->q[3 * iq + d] + c->h_gresp[3 * i + d];
      q2 += comp * comp;
    }
    qgn[i] = std::sqrt(q2);
    qmax = std::max(qmax, qgn[i]);
  }
  for (auto& v : qgn) v = qmax > 0 ? v / qmax : 0.0;
  double wmax = 0.0;
  for (int iw = 0; iw < nw; ++iw) wmax = std::max(wmax, std::fabs(c->om[2 * iw + 1]));
  for (int iw = 0; iw < nw; ++iw) wn[iw] = wmax > 0 ? std::fabs(c->om[2 * iw + 1]) / wmax : 0.0;
}

}  // namespace

// tables of the feature normalisation for q point iq (host set-up)
chi0_status term_tables_upload(chi0_ctx* c, int iq) {
  const int ng = c->cfg.ng, nw = c->cfg.nw;
  chi0_status s;
  if ((s = ctx_ensure(c, c->d_termq, (size_t)ng * 8, "terminator tables")) != CHI0_OK) return s;
  if ((s = ctx_ensure(c, c->d_termw, (size_t)nw * 8, "terminator tables")) != CHI0_OK) return s;
  if ((s = ctx_ensure(c, c->d_termc, 16, "terminator scale")) != CHI0_OK) return s;
  std::vector<double> qgn, wn;
  term_tables(c, iq, qgn, wn);
  if (cudaMemcpyAsync(c->d_termq.p, qgn.data(), ng * 8, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
      cudaMemcpyAsync(c->d_termw.p, wn.data(), nw * 8, cudaMemcpyHostToDevice, c->st) != cudaSuccess ||
      cudaStreamSynchronize(c->st) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, CHI0_ECUDA, "terminator tables upload failed");
  }
  return CHI0_OK;
}

// kernels: scale c, features (and targets) of chi
chi0_status term_features_launch(chi0_ctx* c, const double2* chi, const double2* full, float* x, float* t) {
  const int ng = c->cfg.ng, nw = c->cfg.nw;
  k_diag_scale<<<1, 256, 0, c->st>>>(chi, ng, (double*)c->d_termc.p);
  const int64_t n = (int64_t)ng * ng * nw;
  k_term_features_dev<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(
      chi, full, (const double*)c->d_termq.p, (const double*)c->d_termw.p, ng, nw,
      (const double*)c->d_termc.p, x, t);
  if (cudaGetLastError() != cudaSuccess) return ctx_fail(c, CHI0_ECUDA, "terminator features launch failed");
  return CHI0_OK;
}

chi0_status term_plan(chi0_ctx* c, int iq) {
  const int64_t n = (int64_t)c->cfg.ng * c->cfg.ng * c->cfg.nw;
  chi0_status s;
  if ((s = ctx_ensure(c, c->d_termx, (size_t)n * kI * 4, "terminator features")) != CHI0_OK) return s;
  if ((s = ctx_ensure(c, c->d_termy, (size_t)n * kO * 4, "terminator prediction")) != CHI0_OK) return s;
  return term_tables_upload(c, iq);
}

// chi += Hermitised network correction (build_chi0 with a terminator set)
chi0_status term_launch(chi0_ctx* c, double2* chi) {
  const int ng = c->cfg.ng, nw = c->cfg.nw;
  const int64_t n = (int64_t)ng * ng * nw;
  chi0_status s;
  if ((s = term_features_launch(c, chi, nullptr, (float*)c->d_termx.p, nullptr)) != CHI0_OK) return s;
  if (mlp_predict(c->term_params, (const float*)c->d_termx.p, n, c->term_bf16, (float*)c->d_termy.p,
                  c->st) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, CHI0_ECUDA, "terminator prediction launch failed");
  }
  k_term_apply_dev<<<(unsigned)((n + 255) / 256), 256, 0, c->st>>>(chi, (const float*)c->d_termy.p, ng, nw,
                                                                   (const double*)c->d_termc.p);
  if (cudaGetLastError() != cudaSuccess) return ctx_fail(c, CHI0_ECUDA, "terminator apply launch failed");
  c->launches += 4;
  return CHI0_OK;
}

}  // namespace chi0

extern "C" {

int chi0_mlp_nparams(void) { return chi0::kP; }

int64_t chi0_mlp_workspace_floats(int64_t batch) {
  const int64_t nblk = (batch + chi0::kS - 1) / chi0::kS;
  return nblk * chi0::kP + nblk;
}

chi0_status chi0_mlp_loss_grad(const float* params, const float* x, const float* t, int64_t batch,
                               int bf16, float* grad, float* loss, float* work, void* stream) {
  if (!params || !x || !t || !grad || !work || batch < 1) return CHI0_EINVAL;
  const int64_t nblk = (batch + chi0::kS - 1) / chi0::kS;
  if (nblk > 0x7fffffff) return CHI0_EINVAL;
  if (chi0::mlp_loss_grad(params, x, t, batch, bf16, grad, loss, work, work + nblk * chi0::kP,
                          (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  return CHI0_OK;
}

chi0_status chi0_mlp_adam(float* params, const float* grad, float* m, float* v, int64_t n, float lr,
                          float beta1, float beta2, float eps, int step, void* stream) {
  if (!params || !grad || !m || !v || n < 1 || step < 1) return CHI0_EINVAL;
  if (chi0::mlp_adam(params, grad, m, v, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  return CHI0_OK;
}

chi0_status chi0_mlp_predict(const float* params, const float* x, int64_t batch, int bf16, float* y,
                             void* stream) {
  if (!params || !x || !y || batch < 1) return CHI0_EINVAL;
  if (chi0::mlp_predict(params, x, batch, bf16, y, (cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return CHI0_ECUDA;
  }
  return CHI0_OK;
}

chi0_status chi0_term_features(chi0_ctx* c, int iq, const void* chi_trunc, const void* chi_full, float* x,
                               float* t, double* scale) {
  if (!c) return CHI0_EINVAL;
  if (iq < 0 || iq >= c->cfg.nq || !chi_trunc || !x || (chi_full && !t))
    return chi0::ctx_fail(c, CHI0_EINVAL, "bad iq or NULL buffer");
  if (c->h_gresp.empty() || c->rho_iq != iq)
    return chi0::ctx_fail(c, CHI0_ESTATE, "chi0_compute_rho(iq) must come first (response G set)");
  chi0_status s = chi0::term_tables_upload(c, iq);
  if (s != CHI0_OK) return s;
  s = chi0::term_features_launch(c, (const double2*)chi_trunc, (const double2*)chi_full, x, t);
  if (s != CHI0_OK) return s;
  if (scale) {
    double cs[2];
    if (cudaMemcpyAsync(cs, c->d_termc.p, 16, cudaMemcpyDeviceToHost, c->st) != cudaSuccess ||
        cudaStreamSynchronize(c->st) != cudaSuccess) {
      cudaGetLastError();
      return chi0::ctx_fail(c, CHI0_ECUDA, "scale read back failed");
    }
    *scale = cs[0];
  }
  return CHI0_OK;
}

chi0_status chi0_set_terminator(chi0_ctx* c, const float* params, int bf16) {
  if (!c) return CHI0_EINVAL;
  if (params && c->bg_on)
    return chi0::ctx_fail(c, CHI0_EINVAL, "the extrapolar terminator is set: the two corrections exclude each other");
  c->term_params = params;
  c->term_bf16 = bf16;
  c->chi_iq = c->eps_iq = -1;
  ++c->plan_epoch;
  return CHI0_OK;
}

}  // extern "C"
