// Transition weights and the FP64 form of the chi0 contraction.
//
// Appendix B of the paper writes chi0 as frequency factors F_{nmk}(w) times
// frequency-independent products R^{nmk}_{GG'} = f_s/(N_k Omega) x (occupation
// factor) x rho rho^* (Eqs. X_IP_split, X_IP_split1, X_IP_split2).  Here the
// occupation factor, prefactor and two-pole frequency factor of each
// transition are folded into one real weight per (w, t), and
//
//     chi0(w) = sum_t w_t(w) rho_t rho_t^H   (Hermitian),
//
// is accumulated over bounded transition chunks (the paper's reduction over
// the k/c/v distribution becomes an on-device sum of chunk partials).
#include "internal.cuh"

namespace chi0 {

namespace {

// w_t = pref (f_m - f_n) [1/(z + D) - 1/(z - D)] with z = w + i eta purely
// imaginary (z = i s): the bracket is 2 D / (D^2 + s^2), real.
// Frequency factor of one transition with energy difference d = e_m - e_n:
//   1/(w + d + i eta) - 1/(w - d + i eta)
// kind 0: w = i om (imaginary axis; the factor is real, 2d/(d^2 + (om+eta)^2));
// kind 1 / 2: w = om on the real axis, the real / imaginary part.
__device__ __forceinline__ double pole_weight(int kind, double om, double eta, double d) {
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

__global__ void k_weights(int nk, int n_lo, int Nn, int Nm, int nb, const int32_t* __restrict__ kq,
                          const double* __restrict__ eps, const double* __restrict__ occ,
                          const double* __restrict__ omega_im, const int* __restrict__ vkind, int nw,
                          double eta, double pref, double occ_tol, int bg, double eps_bar,
                          const double* __restrict__ dpole, const double* __restrict__ epsd, int nd,
                          double* __restrict__ w, int k0) {
  const int64_t nt = (int64_t)nk * Nn * Nm;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int m = (int)(t % Nm);
  const int64_t r = t / Nm;
  const int n = n_lo + (int)(r % Nn);
  const int ik = k0 + (int)(r / Nn);   // global k (the transitions cover k0 .. k0 + nk - 1)
  const int ikp = kq[ik];
  const double df = occ[(size_t)ikp * nb + m] - occ[(size_t)ik * nb + n];
  const double d = eps[(size_t)ikp * nb + m] - eps[(size_t)ik * nb + n];
  const double fm = occ[(size_t)ikp * nb + m];
  const double dbar = eps[(size_t)ikp * nb + m] - eps_bar;  // m into an empty state at eps_bar
  for (int iw = 0; iw < nw; ++iw) {
    // kind 0: imaginary-axis frequency i omega_im (+ i eta), real weight;
    // kinds 1 / 2: real part / imaginary part of the complex weight at the
    // real frequency omega_im[iw] with broadening eta
    const int kind = vkind ? vkind[iw] : 0;
    double v = 0.0;
    if (df > occ_tol) {
      double f;
      if (dpole) {
        f = pole_weight(kind, omega_im[iw], eta, dpole[t]);
      } else if (nd > 0) {
        f = 0.0;
        for (int j = 0; j < nd; ++j)
          f += pole_weight(kind, omega_im[iw], eta,
                           epsd[((size_t)ikp * nd + j) * nb + m] - epsd[((size_t)ik * nd + j) * nb + n]);
        f /= nd;
      } else {
        f = pole_weight(kind, omega_im[iw], eta, d);
      }
      v = pref * df * f;
    }
    if (bg && fm > occ_tol) v -= pref * fm * pole_weight(kind, omega_im[iw], eta, dbar);
    w[(size_t)iw * nt + t] = v;
  }
}

constexpr int kT = 32;   // output tile (complex entries per side)
constexpr int kKB = 16;  // transitions per shared-memory stage

__device__ __forceinline__ void tri_decode(int tile, int& I, int& J) {
  int i = (int)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= tile) ++i;
  while (i * (i + 1) / 2 > tile) --i;
  I = i;
  J = tile - i * (i + 1) / 2;
}

// part[kc][iw][i][j] = sum_{t in chunk kc} w_t R_ti conj(R_tj) on lower tiles I >= J.
__global__ void __launch_bounds__(256)
k_chi0_fp64(const double2* __restrict__ R, const double* __restrict__ w, int64_t nt, int ng,
            int nw, int kchunk, double2* __restrict__ part) {
  __shared__ double2 As[kKB][kT];
  __shared__ double2 Bs[kKB][kT];
  __shared__ double ws[kKB];
  int I, J;
  tri_decode(blockIdx.x, I, J);
  const int kc = blockIdx.y, iw = blockIdx.z;
  const int64_t t0 = (int64_t)kc * kchunk;
  const int64_t t1 = min(nt, t0 + kchunk);
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  double2 acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = make_double2(0.0, 0.0);
  const double* wv = w + (size_t)iw * nt;
  for (int64_t tt = t0; tt < t1; tt += kKB) {
    for (int e = tid; e < kKB * kT; e += 256) {
      const int r = e / kT, c = e % kT;
      const int64_t t = tt + r;
      const int ia = I * kT + c, ib = J * kT + c;
      As[r][c] = (t < t1 && ia < ng) ? R[t * ng + ia] : make_double2(0.0, 0.0);
      Bs[r][c] = (t < t1 && ib < ng) ? R[t * ng + ib] : make_double2(0.0, 0.0);
    }
    if (tid < kKB) ws[tid] = (tt + tid < t1) ? wv[tt + tid] : 0.0;
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kKB; ++r) {
      const double wt = ws[r];
      double2 a[2], b[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const double2 av = As[r][ty * 2 + u];
        a[u] = make_double2(wt * av.x, wt * av.y);
        b[u] = Bs[r][tx * 2 + u];
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {  // acc += a conj(b)
          acc[u][v].x = fma(a[u].x, b[v].x, acc[u][v].x);
          acc[u][v].x = fma(a[u].y, b[v].y, acc[u][v].x);
          acc[u][v].y = fma(a[u].y, b[v].x, acc[u][v].y);
          acc[u][v].y = fma(-a[u].x, b[v].y, acc[u][v].y);
        }
    }
    __syncthreads();
  }
  double2* out = part + ((size_t)kc * nw + iw) * (size_t)ng * ng;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = I * kT + ty * 2 + u, j = J * kT + tx * 2 + v;
      if (i < ng && j < ng) out[(size_t)i * ng + j] = acc[u][v];
    }
}

// chi[iw][i][j] (i >= j) = sum_kc part, then chi[iw][j][i] = conj(chi[iw][i][j]).
__global__ void k_chi0_reduce(const double2* __restrict__ part, int nchunks, int ng, int nw,
                              double2* __restrict__ chi, int accumulate) {
  const int64_t n2 = (int64_t)ng * ng;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n2 * nw) return;
  const int iw = (int)(e / n2);
  const int64_t ij = e - (int64_t)iw * n2;
  const int i = (int)(ij / ng), j = (int)(ij - (int64_t)i * ng);
  if (i < j) return;
  double sx = 0.0, sy = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const double2 v = part[((size_t)c * nw + iw) * n2 + ij];
    sx += v.x;
    sy += v.y;
  }
  double2* o = chi + (size_t)iw * n2;
  if (i == j) sy = 0.0;  // Hermitian: real diagonal
  if (accumulate) {      // add to the sum of the earlier transition blocks
    const double2 a = o[(size_t)i * ng + j];
    sx += a.x;
    sy += a.y;
  }
  o[(size_t)i * ng + j] = make_double2(sx, sy);
  if (i != j) o[(size_t)j * ng + i] = make_double2(sx, -sy);
}

}  // namespace

cudaError_t launch_weights(int nk, int n_lo, int Nn, int Nm, int nb, const int32_t* kq,
                           const double* eps, const double* occ, const double* omega_im,
                           const int* vkind, int nw, double eta, double pref,
                           double occ_tol, int bg, double eps_bar, const double* dpole, const double* epsd,
                           int nd, double* w, cudaStream_t s, int k0) {
  const int64_t nt = (int64_t)nk * Nn * Nm;
  if (nt == 0) return cudaSuccess;
  const int64_t blocks = (nt + 255) / 256;
  k_weights<<<(unsigned)blocks, 256, 0, s>>>(nk, n_lo, Nn, Nm, nb, kq, eps, occ, omega_im, vkind, nw, eta,
                                            pref, occ_tol, bg, eps_bar, dpole, epsd, nd, w, k0);
  return cudaGetLastError();
}

cudaError_t launch_chi0_fp64_partials(const double2* R, const double* w, int64_t nt, int ng,
                                      int nw, int kchunk, int nchunks, double2* part,
                                      cudaStream_t s) {
  const int nT = (ng + kT - 1) / kT;
  dim3 grid(nT * (nT + 1) / 2, nchunks, nw);
  k_chi0_fp64<<<grid, 256, 0, s>>>(R, w, nt, ng, nw, kchunk, part);
  return cudaGetLastError();
}

// chi[iw] = H[v] (imaginary-axis frequency) or H[vr] + i H[vi] (real axis)
__global__ void k_combine_freq(const double2* __restrict__ H, const int* __restrict__ vr,
                               const int* __restrict__ vi, int64_t n2, double2* __restrict__ chi) {
  const int iw = blockIdx.y;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n2) return;
  const double2 a = H[(size_t)vr[iw] * n2 + e];
  double2 v = a;
  if (vi[iw] >= 0) {
    const double2 b = H[(size_t)vi[iw] * n2 + e];
    v = make_double2(a.x - b.y, a.y + b.x);
  }
  chi[(size_t)iw * n2 + e] = v;
}

cudaError_t launch_combine_freq(const double2* H, const int* vr, const int* vi, int ng, int nw, double2* chi,
                                cudaStream_t s) {
  const int64_t n2 = (int64_t)ng * ng;
  k_combine_freq<<<dim3((unsigned)((n2 + 255) / 256), (unsigned)nw), 256, 0, s>>>(H, vr, vi, n2, chi);
  return cudaGetLastError();
}

cudaError_t launch_chi0_reduce(const double2* part, int nchunks, int ng, int nw, double2* chi,
                               cudaStream_t s, int accumulate) {
  const int64_t n = (int64_t)ng * ng * nw;
  k_chi0_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, nchunks, ng, nw, chi, accumulate);
  return cudaGetLastError();
}

}  // namespace chi0
