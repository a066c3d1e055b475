// Godby-Needs plasmon-pole model of eps~^-1 (Full frequency GW subsection).
//
// Per element, with x(w) = eps^-1_GG'(w) - delta_GG', the model is one pole
// pair in the retarded form of the chi0 weights,
//     x(w) = R [1/(w - wt + i eta) - 1/(w + wt + i eta)],
// which equals -2 R wt / (nu^2 + wt^2) at w = i nu.  Fixing it at w = 0 and
// w = i w_p gives
//     wt^2 = w_p^2 x(i w_p) / (x(0) - x(i w_p)),   R = -x(0) wt / 2,
// wt the principal square root.  Elements where Re wt^2 <= 0 (or where x does
// not change between the two points) have no real pole; they keep their
// static value, recorded as wt = 0, R = x(0).
//
// Both kernels are elementwise.  The fit moves 64 bytes per element (two
// inputs, two outputs); the evaluation reads 32 bytes per element per chunk
// of frequencies and writes 16 bytes per element and frequency.  Both are
// bound by the FP64 units rather than by HBM (about 20 FP64 operations per
// element and frequency in the evaluation, counting the reciprocal as one).
#include <cmath>

#include "chi0.h"
#include "internal.cuh"

namespace {

constexpr int kPpaThreads = 256;
constexpr int kPpaMaxFreq = 32;   // frequencies per evaluation launch (kernel parameter)

struct FreqChunk {
  double re[kPpaMaxFreq];
  double im[kPpaMaxFreq];
  int n;
};

// a / b by Smith's method (R. L. Smith, CACM 5, 435 (1962)): scales by the
// larger component of b, so |b|^2 is never formed.
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  if (fabs(b.x) >= fabs(b.y)) {
    const double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  }
  const double r = b.x / b.y, d = b.x * r + b.y;
  return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Principal square root of z with Re z > 0: with t = sqrt((|z| + Re z)/2),
// sqrt(z) = t + i Im z / (2 t) (no cancellation in that half plane).
__device__ __forceinline__ double2 csqrt_right(double2 z) {
  const double t = sqrt(0.5 * (hypot(z.x, z.y) + z.x));
  return make_double2(t, z.y / (2.0 * t));
}

__global__ void __launch_bounds__(kPpaThreads) k_ppa_fit(const double2* __restrict__ e0,
                                                         const double2* __restrict__ ep, int ng, double wp2,
                                                         double2* __restrict__ wt, double2* __restrict__ R) {
  const size_t n2 = (size_t)ng * ng;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += stride) {
    double2 x0 = e0[idx], xp = ep[idx];
    if (idx % (size_t)(ng + 1) == 0) {  // diagonal: subtract delta
      x0.x -= 1.0;
      xp.x -= 1.0;
    }
    const double2 den = make_double2(x0.x - xp.x, x0.y - xp.y);
    double2 w = make_double2(0.0, 0.0), r = x0;
    if (den.x != 0.0 || den.y != 0.0) {
      const double2 q = cdiv(xp, den);
      const double2 w2 = make_double2(wp2 * q.x, wp2 * q.y);
      if (w2.x > 0.0) {
        w = csqrt_right(w2);
        const double2 p = cmul(x0, w);
        r = make_double2(-0.5 * p.x, -0.5 * p.y);
      }
    }
    wt[idx] = w;
    R[idx] = r;
  }
}

// The evaluation uses the equivalent form x(a) = x0 / (1 - a^2 p), with
// a = w + i eta, x0 = -2 R / wt (= x(0)) and p = 1 / wt^2 formed once per
// element and a^2 once per frequency (on the host): per element and
// frequency one complex product, one real reciprocal and four products, in
// place of two complex divisions.  Near a pole 1 - a^2 p ~ 2 eta / wt, so the
// rounding error of the subtraction grows like wt / eta -- a few 1e-14
// relative at eta = 0.1 eV.
__global__ void __launch_bounds__(kPpaThreads) k_ppa_eval(const double2* __restrict__ wt,
                                                          const double2* __restrict__ R, int ng, FreqChunk fc,
                                                          double2* __restrict__ out) {
  const size_t n2 = (size_t)ng * ng;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += stride) {
    const double2 w = wt[idx], r = R[idx];
    const double dg = idx % (size_t)(ng + 1) == 0 ? 1.0 : 0.0;
    double2* o = out + idx;
    if (w.x == 0.0 && w.y == 0.0) {  // no real pole: the static value at every frequency
      for (int f = 0; f < fc.n; ++f) o[(size_t)f * n2] = make_double2(r.x + dg, r.y);
      continue;
    }
    const double2 x0 = cdiv(make_double2(-2.0 * r.x, -2.0 * r.y), w);
    const double2 p = cdiv(make_double2(1.0, 0.0), cmul(w, w));
    for (int f = 0; f < fc.n; ++f) {
      const double2 a2 = make_double2(fc.re[f], fc.im[f]);
      const double2 e = make_double2(1.0 - (a2.x * p.x - a2.y * p.y), -(a2.x * p.y + a2.y * p.x));
      const double inv = 1.0 / (e.x * e.x + e.y * e.y);
      const double vx = (x0.x * e.x + x0.y * e.y) * inv;
      const double vy = (x0.y * e.x - x0.x * e.y) * inv;
      o[(size_t)f * n2] = make_double2(vx + dg, vy);
    }
  }
}

int ppa_grid(size_t n2) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms < 1) sms = 1;
  const size_t need = (n2 + kPpaThreads - 1) / kPpaThreads;
  const size_t cap = (size_t)sms * 8;   // 8 blocks of 256 threads fill an SM
  return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

}  // namespace

extern "C" chi0_status chi0_ppa_fit(const void* eps_inv_0, const void* eps_inv_p, int ng, double omega_p,
                                    void* omega_t, void* R, void* cuda_stream) {
  if (!eps_inv_0 || !eps_inv_p || !omega_t || !R || ng < 1 || !std::isfinite(omega_p) || !(omega_p > 0.0))
    return CHI0_EINVAL;
  const size_t n2 = (size_t)ng * ng;
  k_ppa_fit<<<ppa_grid(n2), kPpaThreads, 0, (cudaStream_t)cuda_stream>>>(
      (const double2*)eps_inv_0, (const double2*)eps_inv_p, ng, omega_p * omega_p, (double2*)omega_t,
      (double2*)R);
  if (cudaGetLastError() != cudaSuccess) return CHI0_ECUDA;
  return CHI0_OK;
}

extern "C" chi0_status chi0_ppa_eval(const void* omega_t, const void* R, int ng, const double* freqs, int nf,
                                     double eta, void* out, void* cuda_stream) {
  if (!omega_t || !R || !out || ng < 1 || nf < 0 || (nf > 0 && !freqs) || !std::isfinite(eta) || eta < 0.0)
    return CHI0_EINVAL;
  for (int f = 0; f < nf; ++f)
    if (!std::isfinite(freqs[2 * f]) || !std::isfinite(freqs[2 * f + 1])) return CHI0_EINVAL;
  const size_t n2 = (size_t)ng * ng;
  const int grid = ppa_grid(n2);
  for (int f0 = 0; f0 < nf; f0 += kPpaMaxFreq) {
    FreqChunk fc;
    fc.n = nf - f0 < kPpaMaxFreq ? nf - f0 : kPpaMaxFreq;
    for (int f = 0; f < fc.n; ++f) {  // a^2, a = w + i eta
      const double ar = freqs[2 * (f0 + f)], ai = freqs[2 * (f0 + f) + 1] + eta;
      fc.re[f] = ar * ar - ai * ai;
      fc.im[f] = 2.0 * ar * ai;
    }
    k_ppa_eval<<<grid, kPpaThreads, 0, (cudaStream_t)cuda_stream>>>(
        (const double2*)omega_t, (const double2*)R, ng, fc, (double2*)out + (size_t)f0 * n2);
    if (cudaGetLastError() != cudaSuccess) return CHI0_ECUDA;
  }
  return CHI0_OK;
}
