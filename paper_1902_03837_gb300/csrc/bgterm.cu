// Bruneval-Gonze extrapolar correction (X-terminator): Eq. (X_term_def) and
// Appendix C (Eqs. rhotw-term, F-term, X-term).  The bands left out of the
// sum get one energy eps_bar and no occupation; by the closure relation over
// all bands at k,
//
//   sum_{n >= nb} rho_nm(G) conj(rho_nm(G'))
//       = rho~_{m,k-q}(G - G') - sum_{n < nb} rho_nm(G) conj(rho_nm(G')),
//
// so the corrected chi0 is the contraction over every band n < nb with the
// weights w_t - wbar_m (done by the weights kernel and the usual contraction)
// plus sum_{k', m} wbar_{mk'}(w) rho~_{mk'}(G - G').  The diagonal densities
// rho~ come from the rho kernel in its same-band mode on the set of
// difference vectors d = G_i - G_j; the two kernels here form that last term.
#include "internal.cuh"

namespace chi0 {

namespace {

template <typename TOUT>
__global__ void __launch_bounds__(128)
k_bg_sum(const TOUT* __restrict__ rd, const BgChunks ch, const double* __restrict__ wbar, int64_t ntd,
         int nd, double2* __restrict__ P) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  const int iw = blockIdx.y;
  if (d >= nd) return;
  int c = 0;
  while (c + 1 < ch.n && d >= ch.start[c + 1]) ++c;
  const int64_t stride = ch.start[c + 1] - ch.start[c];
  const TOUT* p = rd + ch.off[c] + (d - ch.start[c]);
  const double* w = wbar + (size_t)iw * ntd;
  double sx = 0.0, sy = 0.0;
  for (int64_t t = 0; t < ntd; ++t) {
    const double wt = w[t];
    const TOUT v = p[t * stride];
    sx = fma(wt, (double)v.x, sx);
    sy = fma(wt, (double)v.y, sy);
  }
  P[(size_t)iw * nd + d] = make_double2(sx, sy);
}

// chi[iw][i][j] += v, chi[iw][j][i] += conj(v) for i >= j, with
// v = (P[d_ij] + conj(P[d_ji])) / 2 (exactly Hermitian; real on the diagonal)
// imag = 1 adds i times the Hermitised term (the imaginary parts of complex
// weights, added to a full complex chi0 of a real-axis frequency)
__global__ void k_bg_apply(const double2* __restrict__ P, const int32_t* __restrict__ didx, int ng, int nd,
                           double2* __restrict__ chi, int imag) {
  const int iw = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ng * ng) return;
  const int i = (int)(e / ng), j = (int)(e % ng);
  if (i < j) return;
  const double2* Pw = P + (size_t)iw * nd;
  const double2 a = Pw[didx[(size_t)i * ng + j]], b = Pw[didx[(size_t)j * ng + i]];
  double vx = 0.5 * (a.x + b.x), vy = 0.5 * (a.y - b.y);
  double2* cw = chi + (size_t)iw * ng * ng;
  if (i == j) vy = 0.0;
  // lower entry += v, upper entry += conj(v); times i when imag
  const double2 lo = imag ? make_double2(-vy, vx) : make_double2(vx, vy);
  const double2 up = imag ? make_double2(vy, vx) : make_double2(vx, -vy);
  double2 x = cw[(size_t)i * ng + j];
  cw[(size_t)i * ng + j] = make_double2(x.x + lo.x, x.y + lo.y);
  if (i != j) {
    x = cw[(size_t)j * ng + i];
    cw[(size_t)j * ng + i] = make_double2(x.x + up.x, x.y + up.y);
  }
}

}  // namespace

template <typename TOUT>
cudaError_t launch_bg_sum(const TOUT* rd, const BgChunks& ch, const double* wbar, int64_t ntd, int nd,
                          int nw, double2* P, cudaStream_t s) {
  if (nd <= 0 || nw <= 0) return cudaSuccess;
  k_bg_sum<TOUT><<<dim3((unsigned)((nd + 127) / 128), (unsigned)nw), 128, 0, s>>>(rd, ch, wbar, ntd, nd, P);
  return cudaGetLastError();
}

cudaError_t launch_bg_apply(const double2* P, const int32_t* didx, int ng, int nd, int nw, double2* chi,
                            cudaStream_t s, int imag) {
  if (ng <= 0 || nw <= 0) return cudaSuccess;
  const int64_t n = (int64_t)ng * ng;
  k_bg_apply<<<dim3((unsigned)((n + 255) / 256), (unsigned)nw), 256, 0, s>>>(P, didx, ng, nd, chi, imag);
  return cudaGetLastError();
}

template cudaError_t launch_bg_sum<float2>(const float2*, const BgChunks&, const double*, int64_t, int, int,
                                           double2*, cudaStream_t);
template cudaError_t launch_bg_sum<double2>(const double2*, const BgChunks&, const double*, int64_t, int, int,
                                            double2*, cudaStream_t);

}  // namespace chi0
