// Dyson step of the Linear Algebra subsection (Eqs. X_rpa, X_rpa_inv) in the
// symmetric form used for W (Eq. W_def):
//
//     eps~ = 1 - V chi0 V,   V = diag(sqrt(4 pi) / |q+G|),   out = eps~^-1,
//
// one matrix per frequency, all frequencies of a q point in one batch.  eps~
// is Hermitian positive definite here (chi0 is negative semidefinite), so the
// inverse is taken by blocked in-place Gauss-Jordan elimination without
// pivoting.  For the pivot block b (width nb), with P = A_bb^-1:
//
//     A_ij <- A_ij - A_ib P A_bj     (i, j outside b)
//     A_bj <- P A_bj,   A_ib <- -A_ib P,   A_bb <- P,
//
// and after the last block A holds eps~^-1.  Each step is three launches: the
// pivot-block inverse (one block per matrix), the two panels, and the rank-nb
// update.  FP64 throughout.
//
// Symmetry halves the work: once the rows/columns of a set S have been swept,
// A_ji = s conj(A_ij) with s = -1 when exactly one of i, j lies in S and +1
// otherwise.  Only the tiles on and below the diagonal are updated; the
// panels read entries above the diagonal through that rule, and a final pass
// copies the conjugate of the lower tiles into the upper ones.
#include "internal.cuh"

namespace chi0 {

namespace {

constexpr int kNB = 32;  // pivot block width
constexpr int kUT = 32;  // update tile

// complex arithmetic as fused multiply-adds (4 per multiply-add): the FP64
// units are the bound of this step
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ void cmac(double2& acc, double2 a, double2 b) {  // acc += a b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cmsub(double2& acc, double2 a, double2 b) {  // acc -= a b
  acc.x = fma(-a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

__global__ void k_build_eps(const double2* __restrict__ chi, const double* __restrict__ v, int ng,
                            int nw, double2* __restrict__ A) {
  const int64_t n2 = (int64_t)ng * ng;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n2 * nw) return;
  const int64_t ij = e % n2;
  const int i = (int)(ij / ng), j = (int)(ij % ng);
  const double s = -v[i] * v[j];
  const double2 c = chi[e];
  A[e] = make_double2((i == j ? 1.0 : 0.0) + s * c.x, s * c.y);
}

// P = inverse of the nb x nb pivot block (scalar Gauss-Jordan in shared memory).
__global__ void __launch_bounds__(128)
k_gj_pivot(double2* __restrict__ A, int ng, int b0, int nb, double2* __restrict__ pinv,
           int* __restrict__ err, int general) {
  __shared__ double2 P[kNB][kNB + 1];
  const int iw = blockIdx.x;
  const double2* Am = A + (size_t)iw * ng * ng;
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    P[r][c] = Am[(size_t)(b0 + r) * ng + b0 + c];
  }
  __syncthreads();
  __shared__ double2 prow[kNB];
  __shared__ double2 pcol[kNB];
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  __shared__ double2 dinv;
  for (int p = 0; p < nb; ++p) {
    if (tid == 0) {
      // Hermitian positive definite => real positive pivots
      const double2 d = P[p][p];
      const double mag = d.x * d.x + d.y * d.y;
      if (!((general || d.x > 0.0) && mag > 1e-300)) bad = 1;
      else dinv = make_double2(d.x / mag, -d.y / mag);  // 1/d
    }
    __syncthreads();
    if (bad) break;
    const double inv_re = dinv.x, inv_im = dinv.y;
    if (tid < nb) {
      const double2 rv = P[p][tid];
      const double2 cv = P[tid][p];
      prow[tid] = cmul(rv, make_double2(inv_re, inv_im));  // a_pj / d
      pcol[tid] = cv;                                     // a_ip
    }
    __syncthreads();
    for (int e = tid; e < nb * nb; e += blockDim.x) {
      const int r = e / nb, c = e % nb;
      double2 val = P[r][c];
      if (r == p && c == p) {
        val = make_double2(inv_re, inv_im);
      } else if (r == p) {
        val = prow[c];
      } else if (c == p) {  // -a_ip / d
        const double2 a = cmul(pcol[r], make_double2(inv_re, inv_im));
        val = make_double2(-a.x, -a.y);
      } else {              // a_ij - a_ip a_pj / d
        cmsub(val, pcol[r], prow[c]);
      }
      P[r][c] = val;
    }
    __syncthreads();
  }
  if (bad) {
    if (tid == 0) atomicExch(err, 1);
    return;
  }
  double2* po = pinv + (size_t)iw * kNB * kNB;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int r = e / nb, c = e % nb;
    po[r * kNB + c] = P[r][c];
  }
}

// colpanel[iw][i][k] = A_i,b0+k (all i);  rowpanel[iw][k][j] = sum_l P_kl A_b0+l,j (all j).
// Entries above the diagonal tiles are not maintained; they follow from the
// stored ones: A_i,b = -conj(A_b,i) for i < b0 (i swept, b not), and
// A_b,j = conj(A_j,b) for j beyond the pivot block (neither swept).
// One thread per (column e, k): four columns per block, so that the panels
// of one matrix spread over ng / 4 blocks (the FP64 rate of a single SM is
// low, and this step sits on the critical path of every pivot block).
constexpr int kPE = 4;

__global__ void __launch_bounds__(128)
k_gj_panels(const double2* __restrict__ A, int ng, int b0, int nb, const double2* __restrict__ pinv,
            double2* __restrict__ colp, double2* __restrict__ rowp, int full) {
  __shared__ double2 base[kPE][kNB];  // A_b0+l,e of the block's columns
  const int iw = blockIdx.y;
  const double2* Am = A + (size_t)iw * ng * ng;
  const double2* P = pinv + (size_t)iw * kNB * kNB;
  double2* cp = colp + (size_t)iw * ng * kNB;
  double2* rp = rowp + (size_t)iw * kNB * ng;
  const int k = threadIdx.x & (kNB - 1), jj = threadIdx.x / kNB;
  const int e = blockIdx.x * kPE + jj;
  const bool live = e < ng && k < nb;
  if (live) {
    double2 v;
    if (full || e >= b0) {
      v = Am[(size_t)e * ng + b0 + k];
    } else {
      const double2 u = Am[(size_t)(b0 + k) * ng + e];
      v = make_double2(-u.x, u.y);
    }
    cp[(size_t)e * kNB + k] = v;
    base[jj][k] = (full || e < b0 + nb) ? Am[(size_t)(b0 + k) * ng + e] : make_double2(v.x, -v.y);
  }
  __syncthreads();
  if (!live) return;
  double2 acc = make_double2(0.0, 0.0);
  for (int l = 0; l < nb; ++l) cmac(acc, P[k * kNB + l], base[jj][l]);
  rp[(size_t)k * ng + e] = acc;
}

// Update blocks are small enough to run on an SM beside a tensor-core
// contraction CTA, so that the Dyson step of one frequency can use the FP64
// units while the contraction of the next occupies the tensor cores: 128
// threads of at most 64 registers, 13 KB of shared memory.  Each block takes
// 16 rows of a 32 x 32 lower tile (kUR) and the k range in two halves (kKH).
// Pivot blocks start at multiples of 32 = kUT, so a tile lies either wholly
// inside or wholly outside the pivot rows (and columns).
constexpr int kUR = 16;
constexpr int kKH = kNB / 2;

__global__ void __launch_bounds__(128, 8)
k_gj_update(double2* __restrict__ A, int ng, int b0, int nb, const double2* __restrict__ pinv,
            const double2* __restrict__ colp, const double2* __restrict__ rowp, int full) {
  __shared__ double2 Cs[kUR][kKH + 1];  // rows i of the block, k (one half)
  __shared__ double2 Rs[kKH][kUT + 1];  // k (one half), columns j of the tile
  const int iw = blockIdx.y;
  int I, J;  // lower tile: I >= J
  {
    const int t = blockIdx.x >> 1;
    if (full) {  // every tile (general matrices)
      const int nT = (ng + kUT - 1) / kUT;
      I = t / nT;
      J = t - I * nT;
    } else {     // tiles on and below the diagonal (Hermitian sweep rule)
      int r = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
      while ((r + 1) * (r + 2) / 2 <= t) ++r;
      while (r * (r + 1) / 2 > t) --r;
      I = r;
      J = t - r * (r + 1) / 2;
    }
  }
  const int i0 = I * kUT + (blockIdx.x & 1) * kUR, j0 = J * kUT;
  if (i0 >= ng) return;  // the whole block lies below the matrix
  const int pt = b0 / kUT;
  const bool ib = (I == pt), jb = (J == pt);
  double2* Am = A + (size_t)iw * ng * ng;
  const double2* cp = colp + (size_t)iw * ng * kNB;
  const double2* rp = rowp + (size_t)iw * kNB * ng;
  const double2* P = pinv + (size_t)iw * kNB * kNB;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;  // columns 2 tx + v, rows 2 ty + u
  double2 val[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + ty * 2 + u, j = j0 + tx * 2 + v;
      double2 x = make_double2(0.0, 0.0);
      if (i < ng && j < ng) {
        if (ib && jb)
          x = P[(i - b0) * kNB + (j - b0)];   // pivot block: P
        else if (ib)
          x = rp[(size_t)(i - b0) * ng + j];  // pivot rows: P A_bj
        else if (!jb)
          x = Am[(size_t)i * ng + j];         // elsewhere: A_ij - A_ib (P A_bj)
      }                                       // pivot columns: -A_ib P
      val[u][v] = x;
    }
  if (!ib) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int kb = h * kKH;
      if (kb >= nb) break;
      for (int e = tid; e < kUR * kKH; e += 128) {
        const int r = e / kKH, k = e % kKH;
        const int i = i0 + r;
        Cs[r][k] = (i < ng && kb + k < nb) ? cp[(size_t)i * kNB + kb + k] : make_double2(0.0, 0.0);
      }
      for (int e = tid; e < kKH * kUT; e += 128) {
        const int k = e / kUT, c = e % kUT;
        const int j = j0 + c;
        double2 x = make_double2(0.0, 0.0);
        if (j < ng && kb + k < nb) x = jb ? P[(kb + k) * kNB + c] : rp[(size_t)(kb + k) * ng + j];
        Rs[k][c] = x;
      }
      __syncthreads();
      const int kn = min(kKH, nb - kb);  // P beyond nb is not defined: never read it
      for (int k = 0; k < kn; ++k) {
        const double2 a0 = Cs[ty * 2][k], a1 = Cs[ty * 2 + 1][k];
        const double2 c0 = Rs[k][tx * 2], c1 = Rs[k][tx * 2 + 1];
        cmsub(val[0][0], a0, c0);
        cmsub(val[0][1], a0, c1);
        cmsub(val[1][0], a1, c0);
        cmsub(val[1][1], a1, c1);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + ty * 2 + u, j = j0 + tx * 2 + v;
      if (i < ng && j < ng) Am[(size_t)i * ng + j] = val[u][v];
    }
}

// upper tiles <- conjugate transpose of the lower tiles
__global__ void k_gj_mirror(double2* __restrict__ A, int ng) {
  const int iw = blockIdx.y;
  double2* Am = A + (size_t)iw * ng * ng;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ng * ng) return;
  const int i = (int)(e / ng), j = (int)(e % ng);
  if (i / kUT < j / kUT) {
    const double2 v = Am[(size_t)j * ng + i];
    Am[(size_t)i * ng + j] = make_double2(v.x, -v.y);
  }
}

}  // namespace

cudaError_t dyson_prepare() {
  const void* fns[] = {(const void*)k_build_eps, (const void*)k_gj_pivot, (const void*)k_gj_panels,
                       (const void*)k_gj_update, (const void*)k_gj_mirror};
  for (const void* f : fns) {
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                               cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_dyson(const double2* chi, const double* vsqrt, int ng, int nw, double2* A,
                         double2* colp, double2* rowp, double2* pinv, int* err, cudaStream_t s) {
  const int64_t n = (int64_t)ng * ng * nw;
  k_build_eps<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(chi, vsqrt, ng, nw, A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nt = (ng + kUT - 1) / kUT;
  for (int b0 = 0; b0 < ng; b0 += kNB) {
    const int nb = min(kNB, ng - b0);
    k_gj_pivot<<<nw, 128, 0, s>>>(A, ng, b0, nb, pinv, err, 0);
    k_gj_panels<<<dim3((ng + kPE - 1) / kPE, nw), kPE * kNB, 0, s>>>(A, ng, b0, nb, pinv, colp, rowp, 0);
    k_gj_update<<<dim3(nt * (nt + 1), nw), 128, 0, s>>>(A, ng, b0, nb, pinv, colp, rowp, 0);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_gj_mirror<<<dim3((unsigned)(((int64_t)ng * ng + 255) / 256), nw), 256, 0, s>>>(A, ng);
  return cudaGetLastError();
}

// General (non-Hermitian) eps~ of real-axis frequencies: the same blocked
// Gauss-Jordan over every tile, reading A directly, with no mirror pass.
// Pivoting is not needed there: for w > 0 with eta > 0 every weight's
// imaginary part is <= 0, so eps~ has a positive semidefinite imaginary
// (anti-Hermitian) part, which every Schur complement inherits; a pivot that
// vanishes all the same is reported through the error flag.
cudaError_t launch_dyson_general(const double2* chi, const double* vsqrt, int ng, int nw, double2* A,
                                 double2* colp, double2* rowp, double2* pinv, int* err, cudaStream_t s) {
  const int64_t n = (int64_t)ng * ng * nw;
  k_build_eps<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(chi, vsqrt, ng, nw, A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nt = (ng + kUT - 1) / kUT;
  for (int b0 = 0; b0 < ng; b0 += kNB) {
    const int nb = min(kNB, ng - b0);
    k_gj_pivot<<<nw, 128, 0, s>>>(A, ng, b0, nb, pinv, err, 1);
    k_gj_panels<<<dim3((ng + kPE - 1) / kPE, nw), kPE * kNB, 0, s>>>(A, ng, b0, nb, pinv, colp, rowp, 1);
    k_gj_update<<<dim3(2 * nt * nt, nw), 128, 0, s>>>(A, ng, b0, nb, pinv, colp, rowp, 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace chi0
