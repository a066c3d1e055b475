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
// (i / 64) + (t / 64) * nI, nI = ceil(ng / 64), entry (i % 64) * 64 + t % 64,
// in FP32 (mixed form) or FP64; rho is copied once per call into the same
// layout (RT) for the dot products.
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

constexpr int kDotUnroll = 8;   // values of i per thread between FP64 sums

__device__ __forceinline__ size_t tile_off(int64_t t, int i, int nI) {
  return ((size_t)(t >> 6) * nI + (i >> 6)) * 4096 + (size_t)(i & 63) * 64 + (t & 63);
}

// rho of the window in the tile layout of Y: RT(i, t) = rho_t(i), t in the
// group-major order (one pass per call; the dot then reads its columns
// coalesced).  32 x 32 blocks through shared memory.
template <typename TR>
__global__ void __launch_bounds__(256)
k_sig_rhot(const TR* __restrict__ R, int64_t T, int nqp, int nb, int ng, int nI, TR* __restrict__ RT) {
  __shared__ TR tl[32][33];
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  const int i0 = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows per pass
  for (int r = ty; r < 32; r += 8) {
    const int64_t t = t0 + r;
    const int i = i0 + tx;
    TR v;
    v.x = 0;
    v.y = 0;
    if (t < T && i < ng) v = R[rho_row(t, nqp, nb) * ng + i];
    tl[r][tx] = v;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + r;
    const int64_t t = t0 + tx;
    if (t < T && i < ng) RT[tile_off(t, i, nI)] = tl[tx][r];
  }
}

// Running sum of the dot products: FP64 in the FP64 form; in the mixed form
// FP32 with Neumaier compensation (GB300's FP64 units are too few to convert
// and add every partial sum in FP64 at the rate the loads arrive).
template <typename F>
struct DotSum {
  F s = 0, c = 0;
  __device__ __forceinline__ void add(F x) {
    if constexpr (sizeof(F) == 4) {
      const F t = s + x;
      c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
      s = t;
    } else {
      s += x;
    }
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// I[g][a][b] = pref sum_i rho_{(g,a)}(i) Y(i, (g,b)), g = (k, m): one block
// per 64 columns t = (g, b); 256 threads = 64 columns x 4 phases over i.
// Each thread reads its column of Y and the columns (g, a) of RT (tile
// layout, both coalesced across the warp), A partners per pass.  Products in
// the element type of rho, summed kDotUnroll at a time into a DotSum.
template <typename TR, typename TY, int A>
__global__ void __launch_bounds__(256, (sizeof(TR) == 8 && A == 4) ? 3 : 1)
k_sig_dot(const TR* __restrict__ RT, const TY* __restrict__ Y, int ng, int64_t T, int nqp, int nI, double pref,
          double2* __restrict__ out) {
  using F = decltype(TR::x);
  __shared__ double2 red[4][64][A];
  const int jl = threadIdx.x & 63, ph = threadIdx.x >> 6;
  const int64_t t = (int64_t)blockIdx.x * 64 + jl;
  const bool live = t < T;
  const int64_t g = live ? t / nqp : 0;
  const int b = live ? (int)(t % nqp) : 0;
  const TY* Ycol = Y + tile_off(t, 0, nI);
  for (int a0 = 0; a0 < nqp; a0 += A) {
    const TR* col[A];   // the partners (g, a0 + q) in RT
#pragma unroll
    for (int q = 0; q < A; ++q) col[q] = RT + tile_off(g * nqp + ((a0 + q < nqp) ? a0 + q : 0), 0, nI);
    DotSum<F> sx[A], sy[A];
    if (live) {
      for (int i0 = ph; i0 < ng; i0 += 4 * kDotUnroll) {
        F cx[A], cy[A];
#pragma unroll
        for (int q = 0; q < A; ++q) cx[q] = cy[q] = 0;
        if (i0 + 4 * (kDotUnroll - 1) < ng) {
          // a full block of kDotUnroll values of i: no guards, so that every
          // load of the block can be in flight at once
          TY yv[kDotUnroll];
#pragma unroll
          for (int r = 0; r < kDotUnroll; ++r) {
            const int i = i0 + 4 * r;
            yv[r] = Ycol[(size_t)(i >> 6) * 4096 + (size_t)(i & 63) * 64];
          }
#pragma unroll
          for (int r = 0; r < kDotUnroll; ++r) {
            const int i = i0 + 4 * r;
            const size_t ro = (size_t)(i >> 6) * 4096 + (size_t)(i & 63) * 64;
            const F yx = (F)yv[r].x, yy = (F)yv[r].y;
#pragma unroll
            for (int q = 0; q < A; ++q)
              if (a0 + q < nqp) {
                const TR v = col[q][ro];
                cx[q] += v.x * yx - v.y * yy;
                cy[q] += v.x * yy + v.y * yx;
              }
          }
        } else {
          for (int r = 0; r < kDotUnroll; ++r) {
            const int i = i0 + 4 * r;
            if (i >= ng) break;
            const size_t ro = (size_t)(i >> 6) * 4096 + (size_t)(i & 63) * 64;
            const TY yd = Ycol[ro];
            const F yx = (F)yd.x, yy = (F)yd.y;
#pragma unroll
            for (int q = 0; q < A; ++q)
              if (a0 + q < nqp) {
                const TR v = col[q][ro];
                cx[q] += v.x * yx - v.y * yy;
                cy[q] += v.x * yy + v.y * yx;
              }
          }
        }
#pragma unroll
        for (int q = 0; q < A; ++q) {
          sx[q].add(cx[q]);
          sy[q].add(cy[q]);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < A; ++q) red[ph][jl][q] = make_double2(sx[q].value(), sy[q].value());
    __syncthreads();
    if (ph == 0 && live)
      for (int q = 0; q < A && a0 + q < nqp; ++q) {
        const double x = red[0][jl][q].x + red[1][jl][q].x + red[2][jl][q].x + red[3][jl][q].x;
        const double y = red[0][jl][q].y + red[1][jl][q].y + red[2][jl][q].y + red[3][jl][q].y;
        out[((size_t)g * nqp + a0 + q) * nqp + b] = make_double2(pref * x, pref * y);
      }
  }
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
cudaError_t launch_sig_rhot(const TR* R, int64_t T, int nqp, int nb, int ng, TR* RT, cudaStream_t s) {
  const int nI = (ng + 63) / 64;
  k_sig_rhot<TR><<<dim3((unsigned)((T + 31) / 32), (unsigned)((ng + 31) / 32)), 256, 0, s>>>(R, T, nqp, nb, ng, nI,
                                                                                              RT);
  return cudaGetLastError();
}

template <typename TR, typename TY>
cudaError_t launch_sig_dot(const TR* RT, const TY* Y, int ng, int64_t T, int nqp, double pref, double2* out,
                           cudaStream_t s) {
  const int nI = (ng + 63) / 64;
  const unsigned grid = (unsigned)((T + 63) / 64);
  if (nqp <= 4)   // fewer partners per pass: fewer registers, more resident blocks
    k_sig_dot<TR, TY, 4><<<grid, 256, 0, s>>>(RT, Y, ng, T, nqp, nI, pref, out);
  else
    k_sig_dot<TR, TY, 8><<<grid, 256, 0, s>>>(RT, Y, ng, T, nqp, nI, pref, out);
  return cudaGetLastError();
}

template cudaError_t launch_sig_rhot<float2>(const float2*, int64_t, int, int, int, float2*, cudaStream_t);
template cudaError_t launch_sig_rhot<double2>(const double2*, int64_t, int, int, int, double2*, cudaStream_t);
template cudaError_t launch_sig_dot<float2, float2>(const float2*, const float2*, int, int64_t, int, double,
                                                    double2*, cudaStream_t);
template cudaError_t launch_sig_dot<double2, double2>(const double2*, const double2*, int, int64_t, int, double,
                                                      double2*, cudaStream_t);

}  // namespace chi0
