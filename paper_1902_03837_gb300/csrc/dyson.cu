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
__global__ void __launch_bounds__(256)
k_gj_pivot(double2* __restrict__ A, int ng, int b0, int nb, double2* __restrict__ pinv,
           int* __restrict__ err) {
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
  for (int p = 0; p < nb; ++p) {
    const double2 d = P[p][p];
    // Hermitian positive definite => real positive pivots
    const double mag = d.x * d.x + d.y * d.y;
    if (tid == 0 && !(d.x > 0.0 && mag > 1e-300)) bad = 1;
    __syncthreads();
    if (bad) break;
    const double inv_re = d.x / mag, inv_im = -d.y / mag;  // 1/d
    if (tid < nb) {
      const double2 rv = P[p][tid];
      const double2 cv = P[tid][p];
      prow[tid] = make_double2(rv.x * inv_re - rv.y * inv_im, rv.x * inv_im + rv.y * inv_re);  // a_pj / d
      pcol[tid] = cv;                                                                          // a_ip
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
        const double2 a = pcol[r];
        val = make_double2(-(a.x * inv_re - a.y * inv_im), -(a.x * inv_im + a.y * inv_re));
      } else {              // a_ij - a_ip a_pj / d
        const double2 a = pcol[r], b = prow[c];
        val.x -= a.x * b.x - a.y * b.y;
        val.y -= a.x * b.y + a.y * b.x;
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
__global__ void k_gj_panels(const double2* __restrict__ A, int ng, int b0, int nb,
                            const double2* __restrict__ pinv, double2* __restrict__ colp,
                            double2* __restrict__ rowp) {
  const int iw = blockIdx.y;
  const double2* Am = A + (size_t)iw * ng * ng;
  const double2* P = pinv + (size_t)iw * kNB * kNB;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ng) return;
  double2* cp = colp + (size_t)iw * ng * kNB;
  double2* rp = rowp + (size_t)iw * kNB * ng;
  double2 col[kNB];
  for (int k = 0; k < nb; ++k) {
    double2 v;
    if (e >= b0) {
      v = Am[(size_t)e * ng + b0 + k];
    } else {
      const double2 u = Am[(size_t)(b0 + k) * ng + e];
      v = make_double2(-u.x, u.y);
    }
    cp[(size_t)e * kNB + k] = v;
    // base of the row panel: A_b0+k,e
    col[k] = (e < b0 + nb) ? Am[(size_t)(b0 + k) * ng + e] : make_double2(v.x, -v.y);
  }
  for (int k = 0; k < nb; ++k) {
    double sx = 0.0, sy = 0.0;
    for (int l = 0; l < nb; ++l) {
      const double2 p = P[k * kNB + l], a = col[l];
      sx += p.x * a.x - p.y * a.y;
      sy += p.x * a.y + p.y * a.x;
    }
    rp[(size_t)k * ng + e] = make_double2(sx, sy);
  }
}

__global__ void __launch_bounds__(256)
k_gj_update(double2* __restrict__ A, int ng, int b0, int nb, const double2* __restrict__ pinv,
            const double2* __restrict__ colp, const double2* __restrict__ rowp) {
  __shared__ double2 Cs[kUT][kNB + 1];  // rows i of the tile, k
  __shared__ double2 Rs[kNB][kUT + 1];  // k, columns j of the tile
  const int iw = blockIdx.y;
  int I, J;  // lower tile: I >= J
  {
    const int t = blockIdx.x;
    int r = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    while (r * (r + 1) / 2 > t) --r;
    I = r;
    J = t - r * (r + 1) / 2;
  }
  const int i0 = I * kUT, j0 = J * kUT;
  double2* Am = A + (size_t)iw * ng * ng;
  const double2* cp = colp + (size_t)iw * ng * kNB;
  const double2* rp = rowp + (size_t)iw * kNB * ng;
  const double2* P = pinv + (size_t)iw * kNB * kNB;
  const int tid = threadIdx.x;
  for (int e = tid; e < kUT * kNB; e += 256) {
    const int r = e / kNB, k = e % kNB;
    const int i = i0 + r;
    Cs[r][k] = (i < ng && k < nb) ? cp[(size_t)i * kNB + k] : make_double2(0.0, 0.0);
  }
  for (int e = tid; e < kNB * kUT; e += 256) {
    const int k = e / kUT, c = e % kUT;
    const int j = j0 + c;
    Rs[k][c] = (j < ng && k < nb) ? rp[(size_t)k * ng + j] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  for (int u = 0; u < 2; ++u) {
    for (int v = 0; v < 2; ++v) {
      const int r = ty * 2 + u, c = tx * 2 + v;
      const int i = i0 + r, j = j0 + c;
      if (i >= ng || j >= ng) continue;
      const bool ib = (i >= b0 && i < b0 + nb), jb = (j >= b0 && j < b0 + nb);
      double2 val;
      if (ib && jb) {
        val = P[(i - b0) * kNB + (j - b0)];
      } else if (ib) {
        val = Rs[i - b0][c];
      } else if (jb) {  // -A_ib P_bj
        double sx = 0.0, sy = 0.0;
        for (int k = 0; k < nb; ++k) {
          const double2 a = Cs[r][k], p = P[k * kNB + (j - b0)];
          sx += a.x * p.x - a.y * p.y;
          sy += a.x * p.y + a.y * p.x;
        }
        val = make_double2(-sx, -sy);
      } else {          // A_ij - A_ib (P A_bj)
        val = Am[(size_t)i * ng + j];
        for (int k = 0; k < nb; ++k) {
          const double2 a = Cs[r][k], b = Rs[k][c];
          val.x -= a.x * b.x - a.y * b.y;
          val.y -= a.x * b.y + a.y * b.x;
        }
      }
      Am[(size_t)i * ng + j] = val;
    }
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

cudaError_t launch_dyson(const double2* chi, const double* vsqrt, int ng, int nw, double2* A,
                         double2* colp, double2* rowp, double2* pinv, int* err, cudaStream_t s) {
  const int64_t n = (int64_t)ng * ng * nw;
  k_build_eps<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(chi, vsqrt, ng, nw, A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nt = (ng + kUT - 1) / kUT;
  for (int b0 = 0; b0 < ng; b0 += kNB) {
    const int nb = min(kNB, ng - b0);
    k_gj_pivot<<<nw, 256, 0, s>>>(A, ng, b0, nb, pinv, err);
    k_gj_panels<<<dim3((ng + 127) / 128, nw), 128, 0, s>>>(A, ng, b0, nb, pinv, colp, rowp);
    k_gj_update<<<dim3(nt * (nt + 1) / 2, nw), 256, 0, s>>>(A, ng, b0, nb, pinv, colp, rowp);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_gj_mirror<<<dim3((unsigned)(((int64_t)ng * ng + 255) / 256), nw), 256, 0, s>>>(A, ng);
  return cudaGetLastError();
}

}  // namespace chi0
