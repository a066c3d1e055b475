// Internal declarations shared by the translation units of libchi0.
// Not part of the public ABI (see include/chi0.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace chi0 {

template <typename T> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float> { using t = float2; };

// Geometry of the oscillator-strength computation for one q point.
//
// The real-space grid is (N1, N2, N3) = (x, y, z).  Wavefunctions are held in
// a mixed representation U_n(x, y, gz): the inverse transform is done along x
// and y only, z stays in reciprocal space (gz in [-Lz, Lz], NZ = 2 Lz + 1).
// The response vectors G_i are used through h_i = G_i - G0 (G0: umklapp of
// the k-pair); hz_rel = G_i,z - Mz_lo in [0, HZ), and likewise for y.
struct RhoGeom {
  int N1, N2, N3;
  int Lx, Ly, Lz;          // largest |G_a| over every wavefunction sphere
  int NX, NY, NZ;          // 2 L + 1
  int nk, nb, npw_max;
  int ng;
  int Mx_lo, My_lo, Mz_lo; // smallest G_a over the response set
  int HX, HY, HZ;          // extent of the response set along each axis
  int n_lo, Nn;            // n bands (at k): [n_lo, n_lo + Nn)
  int Nm;                  // m bands (at k - q): [0, Nm)
  int g0max;               // largest |G0_a| over the k-pairs (umklapp)
  int g0z_min, g0z_max;    // range of G0_z over the k-pairs
  int diag;                // 1: the m grid is band n_lo + n at the same k (Nm = 1):
                           // diagonal densities <n k| e^{i G.r} |n k>
  // Band/k blocks (0 = the whole problem): the transitions cover the k
  // points k0 .. k0 + nk - 1; the n grids sit in an array of nbu bands per
  // local k whose first band is bu0; the m grids in an array of nbm bands per
  // (global) k, separate from the n grids when the task's Um is set.
  int k0, nbu, bu0, nbm;
};

// Zero padding of the n plane in the rho kernel's shared memory.
struct RhoSmem {
  int padz;      // zero rows below the n plane
  int unp_rows;  // rows of the padded n plane (zero outside [padz, padz + NZ))
};

// One independent rho problem (a system at one q point) for the rho kernels.
template <typename T, typename TOUT>
struct RhoTask {
  RhoGeom g;
  RhoSmem sm;
  const typename C2<T>::t* U;
  const typename C2<T>::t* Um;  // m grids (NULL: in U)
  const int32_t* kq;
  const int32_t* g0;
  const int32_t* gresp;
  const int32_t* gperm;
  const typename C2<T>::t* tw1;
  const typename C2<T>::t* tw2;
  TOUT* R;
  int jm;          // m bands per block (<= the kernel's JM)
  int64_t block0;  // first global block of this task in a batched launch
};

// ---- launchers (stream-ordered; return cudaGetLastError()) ----

// a1: sphere -> mixed grid U[k][band][x][gz][y] for every k and band, or
// (nkr > 0) for the k points k0 .. k0 + nkr - 1 and bands b0 .. b0 + nbo - 1
// only, written as U[k - k0][band - b0] (coefficients indexed globally).
template <typename T>
cudaError_t launch_wf_to_mixed(const RhoGeom& g, const int32_t* gvec, const int32_t* npw,
                               const typename C2<T>::t* coef, const typename C2<T>::t* tw1,
                               const typename C2<T>::t* tw2, typename C2<T>::t* U,
                               cudaStream_t s, int k0 = 0, int nkr = 0, int b0 = 0, int nbo = 0);

// a2: rho for every transition of the dense (k, n, m) block, written to
// R[t][i], t = ((ik * Nn) + (n - n_lo)) * Nm + m.  gperm: the response indices
// ordered by (Gy, Gz, Gx) (the order in which a block's threads visit them).
// Um (optional): the m grids in an array of their own (see RhoGeom::nbm).
template <typename T, typename TOUT>
cudaError_t launch_rho_pairs(const RhoGeom& g, const typename C2<T>::t* U, const int32_t* kq,
                             const int32_t* g0, const int32_t* gresp, const int32_t* gperm,
                             const typename C2<T>::t* tw1, const typename C2<T>::t* tw2,
                             TOUT* R, cudaStream_t s, const typename C2<T>::t* Um = nullptr);

// Fill a task for the rho kernels with at most jm_max m bands per block;
// *smem = its shared memory with a JM = jm_max kernel, *nblocks its blocks.
template <typename T, typename TOUT>
cudaError_t rho_task_make(const RhoGeom& g, const typename C2<T>::t* U, const int32_t* kq,
                          const int32_t* g0, const int32_t* gresp, const int32_t* gperm,
                          const typename C2<T>::t* tw1, const typename C2<T>::t* tw2, TOUT* R,
                          int jm_max, RhoTask<T, TOUT>* tk, size_t* smem, int64_t* nblocks);

// Persistent rho over many tasks in one launch (tasks_dev: device array with
// block0 prefix offsets; total: all blocks; counter: device scratch).
template <typename T, typename TOUT>
cudaError_t launch_rho_batch(const RhoTask<T, TOUT>* tasks_dev, int ntasks, int64_t total, int jm,
                             size_t smem, unsigned long long* counter, int nsm, cudaStream_t s);

// a3: real transition weights w[iw][t] (FP64).
// With bg != 0 each weight is reduced by the extrapolar weight of its m
// (a transition from m into an empty state at eps_bar): the closure form of
// the Bruneval-Gonze correction.
// omega_im[iw] and vkind[iw] (NULL: all kind 0) describe the contraction's
// frequency list: kind 0 an imaginary-axis frequency i omega_im (real
// weights); kinds 1 and 2 the real and imaginary parts of the complex weights
// at the real frequency omega_im.
// The frequency factor takes the pole energy d = eps_{m,k-q} - eps_{n,k}
// unless dpole (one pole energy per transition: its degenerate group's
// representative, Appendix B) or epsd (nd dense-grid energies per k and band,
// [k][j][band]: the factor becomes its mean over the nd dense transitions) is
// given.
cudaError_t launch_weights(int nk, int n_lo, int Nn, int Nm, int nb, const int32_t* kq,
                           const double* eps, const double* occ, const double* omega_im,
                           const int* vkind, int nw, double eta, double pref,
                           double occ_tol, int bg, double eps_bar, const double* dpole, const double* epsd,
                           int nd, double* w, cudaStream_t s, int k0 = 0);
// chi[iw] = H[vr[iw]] + i H[vi[iw]] (vi[iw] < 0: chi[iw] = H[vr[iw]])
cudaError_t launch_combine_freq(const double2* H, const int* vr, const int* vi, int ng, int nw, double2* chi,
                                cudaStream_t s);

// Bruneval-Gonze correction, the two steps after the contraction:
// P[iw][d] = sum_t wbar[iw][t] rd(t, d) over the diagonal densities rd of the
// states t = (k, m) on the difference vectors d (stored in chunks: chunk c
// holds d in [start[c], start[c + 1]) as [t][d - start[c]] at offset off[c]),
// then chi[iw][i][j] += P[iw][didx[i][j]] (Hermitised).
constexpr int kBgMaxChunks = 16;
struct BgChunks {
  int n;
  int start[kBgMaxChunks + 1];
  int64_t off[kBgMaxChunks];
};
template <typename TOUT>
cudaError_t launch_bg_sum(const TOUT* rd, const BgChunks& ch, const double* wbar, int64_t ntd, int nd,
                          int nw, double2* P, cudaStream_t s);
cudaError_t launch_bg_apply(const double2* P, const int32_t* didx, int ng, int nd, int nw, double2* chi,
                            cudaStream_t s, int imag = 0);
// The extrapolar term of every frequency, applied by the contraction right
// after its own reduction of that frequency (before its per-frequency event).
struct BgApply {
  const double2* P;      // [nw][nd]
  const int32_t* didx;   // [ng][ng]
  int nd;
};

// a4 (FP64 form): split-K partials of chi0 = sum_t w_t R_t R_t^H, lower
// triangle tiles; part[kc][iw][i][j] (complex128).
cudaError_t launch_chi0_fp64_partials(const double2* R, const double* w, int64_t nt, int ng,
                                      int nw, int kchunk, int nchunks, double2* part,
                                      cudaStream_t s);
// Sum of the partials, Hermitian completion: chi[iw][i][j] (accumulate: added
// to what chi holds, the sum over earlier transition blocks).
cudaError_t launch_chi0_reduce(const double2* part, int nchunks, int ng, int nw, double2* chi,
                               cudaStream_t s, int accumulate = 0);

// a5: eps~ = 1 - V chi V, then in-place blocked Gauss-Jordan inverse.
cudaError_t launch_dyson(const double2* chi, const double* vsqrt, int ng, int nw, double2* A,
                         double2* colpanel, double2* rowpanel, double2* pinv, int* err_flag,
                         cudaStream_t s);
// The same for general eps~ (real-axis frequencies): every tile, no symmetry.
cudaError_t launch_dyson_general(const double2* chi, const double* vsqrt, int ng, int nw, double2* A,
                                 double2* colpanel, double2* rowpanel, double2* pinv, int* err_flag,
                                 cudaStream_t s);
// The Dyson kernels prefer the whole shared-memory carveout, the setting of
// the tensor-core contraction, so that both can share an SM.
cudaError_t dyson_prepare();

// Self-energy kernel I (Eq. I_c; sigma.cu).  W^d of one frequency in FP64
// from eps~^-1 (E) and V; Y(i, t) = sum_j W^d_ij conj(rho_t(j)) in plain
// FP64 (rho in the rho kernel's order of the quasiparticle window, Y in
// 64 x 64 tiles); I[g][a][b] = pref sum_i rho_(g,a)(i) Y(i, (g,b)).
cudaError_t launch_sig_wd64(const double2* E, const double* vsqrt, int ng, double2* Wd, cudaStream_t s);
cudaError_t launch_sig_gemm64(const double2* Wd, const double2* R, int ng, int64_t T, int nqp, int nb,
                              double2* Y, cudaStream_t s);
// rho of the window (rho kernel order) into the tile layout of Y (RT)
template <typename TR>
cudaError_t launch_sig_rhot(const TR* R, int64_t T, int nqp, int nb, int ng, TR* RT, cudaStream_t s);
template <typename TR, typename TY>
cudaError_t launch_sig_dot(const TR* RT, const TY* Y, int ng, int64_t T, int nqp, double pref, double2* out,
                           cudaStream_t s);

}  // namespace chi0
