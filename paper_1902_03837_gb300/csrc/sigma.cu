// Self-energy kernel I of the full-frequency GW step (Eqs. W_def, W_delta, I_c):
//
//   I^{ab k}_{m q}(w) = -1/(N_k Omega) sum_{G,G'} W^d_GG'(q,w) rho_{amk}(q,G) conj(rho_{bmk}(q,G')),
//
// W = V eps~^-1 V (the symmetric form of Eq. W_def), W^d its delta-like part
// (Eq. W_delta), a and b two bands of the quasiparticle window at k, m any
// band at k - q.  With Y(i, t) = sum_j W^d_ij conj(rho_t(j)) (the contraction:
// tensor cores in the mixed form, tc.cu; the plain FP64 kernel below in the
// FP64 form) every entry is one dot product over i:
//
//   I[k][m][a][b] = -1/(N_k Omega) sum_i rho_{(k,m,a)}(i) Y(i, (k,m,b)).
//
// Transitions of the window are ordered t = ((k nb) + m) nqp + a (partners of
// one (k, m) adjacent); the rho kernel writes them in the order
// ((k nqp) + a) nb + m.  Y is stored as 64 x 64 complex tiles, tile
// (i / 64) + (t / 64) * nI, nI = ceil(ng / 64), entry (i % 64) * 64 + t % 64.
#include "internal.cuh"

namespace chi0 {

namespace {

__device__ __forceinline__ int64_t rho_row(int64_t t, int nqp, int nb) {
  const int64_t a = t % nqp, g = t / nqp;
  return ((g / nb) * nqp + a) * nb + g % nb;
}

// W^d_ij = V_i V_j [ (Im E_ij + Im E_ji) / 2 - i (Re E_ij - Re E_ji) / 2 ] in FP64
__global__ void k_sig_wd64(const double2* __restrict__ E, const double* __restrict__ v, int ng,
                           double2* __restrict__ Wd) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ng * ng) return;
  const int i = (int)(e / ng), j = (int)(e % ng);
  const double2 a = E[e], b = E[(size_t)j * ng + i];
  const double f = 0.5 * v[i] * v[j];
  Wd[e] = make_double2(f * (a.y + b.y), -f * (a.x - b.x));
}

// Y(i, t) = sum_j W^d_ij conj(rho_t(j)), plain FP64: 16 x 16 outputs per
// block, 16-wide slices of j staged in shared memory.
__global__ void __launch_bounds__(256)
k_sig_gemm64(const double2* __restrict__ Wd, const double2* __restrict__ R, int ng, int64_t T, int nqp, int nb,
             int nI, double2* __restrict__ Y) {
  __shared__ double2 ws[16][17], rs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.y * 16;
  const int64_t t0 = (int64_t)blockIdx.x * 16;
  const int i = i0 + ty;
  const int64_t t = t0 + tx;
  const int64_t lrow = (t0 + ty < T) ? rho_row(t0 + ty, nqp, nb) : -1;   // the row this thread stages
  double sx = 0.0, sy = 0.0;
  for (int j0 = 0; j0 < ng; j0 += 16) {
    const int j = j0 + tx;
    ws[ty][tx] = (i0 + ty < ng && j < ng) ? Wd[(size_t)(i0 + ty) * ng + j] : make_double2(0.0, 0.0);
    const double2 r = (lrow >= 0 && j < ng) ? R[lrow * ng + j] : make_double2(0.0, 0.0);
    rs[ty][tx] = make_double2(r.x, -r.y);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const double2 a = ws[ty][q], b = rs[tx][q];
      sx += a.x * b.x - a.y * b.y;
      sy += a.x * b.y + a.y * b.x;
    }
    __syncthreads();
  }
  if (i < ng && t < T)
    Y[((size_t)(t / 64) * nI + i / 64) * 4096 + (size_t)(i % 64) * 64 + t % 64] = make_double2(sx, sy);
}

constexpr int kDotChunk = 32;   // values of i staged per pass
constexpr int kDotA = 8;        // partners a per pass

// I[g][a][b] = pref sum_i rho_{(g,a)}(i) Y(i, (g,b)), g = (k, m): one block
// per 64 columns t = (g, b); 256 threads = 64 columns x 4 phases over i.
// The rho rows of the groups these columns touch are staged in shared memory
// per 32 values of i.  Products in the element type of rho (FP32 in the mixed
// form: at most 8 terms per thread and chunk), sums over chunks in FP64.
template <typename TR>
__global__ void __launch_bounds__(256)
k_sig_dot(const TR* __restrict__ R, const double2* __restrict__ Y, int ng, int64_t T, int nqp, int nb, int nI,
          double pref, double2* __restrict__ out) {
  using F = decltype(TR::x);
  extern __shared__ __align__(16) unsigned char sm_raw[];
  TR* rs = reinterpret_cast<TR*>(sm_raw);   // [rows][kDotChunk]
  const int64_t c0 = (int64_t)blockIdx.x * 64;
  const int64_t c1 = c0 + 64 < T ? c0 + 64 : T;
  const int64_t g_lo = c0 / nqp, g_hi = (c1 - 1) / nqp;
  const int rows = (int)(g_hi - g_lo + 1) * nqp;
  const int jl = threadIdx.x & 63, ph = threadIdx.x >> 6;
  const int64_t tcol = c0 + jl;
  const bool live = tcol < T;
  const int64_t g = live ? tcol / nqp : g_lo;
  const int b = live ? (int)(tcol % nqp) : 0;
  const int lrow0 = (int)(g - g_lo) * nqp;
  const double2* Ycol = Y + (size_t)(c0 / 64) * nI * 4096 + jl;
  for (int a0 = 0; a0 < nqp; a0 += kDotA) {
    double sx[kDotA], sy[kDotA];
#pragma unroll
    for (int q = 0; q < kDotA; ++q) sx[q] = sy[q] = 0.0;
    for (int i0 = 0; i0 < ng; i0 += kDotChunk) {
      __syncthreads();
      for (int e = threadIdx.x; e < rows * kDotChunk; e += 256) {
        const int r = e / kDotChunk, il = e % kDotChunk;
        const int i = i0 + il;
        TR v;
        v.x = 0;
        v.y = 0;
        if (i < ng) v = R[rho_row((g_lo + r / nqp) * nqp + r % nqp, nqp, nb) * ng + i];
        rs[e] = v;
      }
      __syncthreads();
      if (live) {
        F cx[kDotA], cy[kDotA];
#pragma unroll
        for (int q = 0; q < kDotA; ++q) cx[q] = cy[q] = 0;
        for (int il = ph; il < kDotChunk && i0 + il < ng; il += 4) {
          const int i = i0 + il;
          const double2 yd = Ycol[(size_t)(i >> 6) * 4096 + (size_t)(i & 63) * 64];
          const F yx = (F)yd.x, yy = (F)yd.y;
#pragma unroll
          for (int q = 0; q < kDotA; ++q)
            if (a0 + q < nqp) {
              const TR r = rs[(lrow0 + a0 + q) * kDotChunk + il];
              cx[q] += r.x * yx - r.y * yy;
              cy[q] += r.x * yy + r.y * yx;
            }
        }
#pragma unroll
        for (int q = 0; q < kDotA; ++q) {
          sx[q] += (double)cx[q];
          sy[q] += (double)cy[q];
        }
      }
    }
    // sum the four phases
    __syncthreads();
    double2* red = reinterpret_cast<double2*>(sm_raw);   // [4][64][kDotA]
#pragma unroll
    for (int q = 0; q < kDotA; ++q) red[(ph * 64 + jl) * kDotA + q] = make_double2(sx[q], sy[q]);
    __syncthreads();
    if (ph == 0 && live)
      for (int q = 0; q < kDotA && a0 + q < nqp; ++q) {
        double x = 0.0, y = 0.0;
        for (int p = 0; p < 4; ++p) {
          const double2 v = red[(p * 64 + jl) * kDotA + q];
          x += v.x;
          y += v.y;
        }
        out[((size_t)g * nqp + a0 + q) * nqp + b] = make_double2(pref * x, pref * y);
      }
  }
}

template <typename TR>
size_t dot_smem(int nqp) {
  const size_t rows = (size_t)(63 / nqp + 2) * nqp;
  const size_t a = rows * kDotChunk * sizeof(TR), r = (size_t)4 * 64 * kDotA * 16;
  return a > r ? a : r;
}

}  // namespace

cudaError_t launch_sig_wd64(const double2* E, const double* vsqrt, int ng, double2* Wd, cudaStream_t s) {
  const int64_t n = (int64_t)ng * ng;
  k_sig_wd64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(E, vsqrt, ng, Wd);
  return cudaGetLastError();
}

cudaError_t launch_sig_gemm64(const double2* Wd, const double2* R, int ng, int64_t T, int nqp, int nb,
                              double2* Y, cudaStream_t s) {
  const int nI = (ng + 63) / 64;
  k_sig_gemm64<<<dim3((unsigned)((T + 15) / 16), (unsigned)((ng + 15) / 16)), 256, 0, s>>>(Wd, R, ng, T, nqp,
                                                                                          nb, nI, Y);
  return cudaGetLastError();
}

template <typename TR>
cudaError_t launch_sig_dot(const TR* R, const double2* Y, int ng, int64_t T, int nqp, int nb, double pref,
                           double2* out, cudaStream_t s) {
  const int nI = (ng + 63) / 64;
  const size_t smem = dot_smem<TR>(nqp);
  cudaError_t e = cudaFuncSetAttribute(k_sig_dot<TR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_sig_dot<TR><<<(unsigned)((T + 63) / 64), 256, smem, s>>>(R, Y, ng, T, nqp, nb, nI, pref, out);
  return cudaGetLastError();
}

template cudaError_t launch_sig_dot<float2>(const float2*, const double2*, int, int64_t, int, int, double, double2*,
                                            cudaStream_t);
template cudaError_t launch_sig_dot<double2>(const double2*, const double2*, int, int64_t, int, int, double,
                                             double2*, cudaStream_t);

}  // namespace chi0
