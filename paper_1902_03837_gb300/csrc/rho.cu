// Oscillator strengths rho_{nmk}(q,G) = <n k| e^{i(q+G).r} |m k-q>
// (Linear Response section, Eq. rhotw), through the real-space product of the
// two states and a Fourier transform, as the paper describes.
//
// GB300 design.  With u_n(r) = sum_G c_n(G) e^{iG.r} on the N1 x N2 x N3 grid
// and h = G - G0 (k - q = k' + G0):
//
//   rho(G) = 1/(N1 N2 N3) sum_r conj(u_n(r)) u_m(r) e^{i h.r}.
//
// The orbitals are transformed back along x and y only (kernel a1), so along
// z they stay band-limited spectra U(x, y, gz), gz in [-Lz, Lz].  For one
// (x, y) column the z part of the product and its forward transform collapse
// into a short correlation of the two spectra:
//
//   sum_z conj(u_n) u_m e^{2 pi i hz z / N3} = N3 sum_b conj(U_n(b + hz)) U_m(b),
//
// (exact while |b + hz - b'| < N3, i.e. on any alias-free grid), which costs
// NZ multiply-adds per output instead of an N3-point transform.  The y and x
// transforms of the product are then pruned DFTs onto the response set only
// (kernel a2, stages Y and X).  A thread block owns one k-pair, one n band
// and JM m bands, streams the x planes of the two mixed grids through shared
// memory and accumulates rho for all its transitions in registers, so the
// large intermediate of a staged FFT never reaches HBM.
#include "internal.cuh"

namespace chi0 {

namespace {

template <typename T2>
__device__ __forceinline__ void cmac(T2& acc, const T2 a, const T2 b) {  // acc += a * b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}

template <typename T2>
__device__ __forceinline__ void cjmac(T2& acc, const T2 a, const T2 b) {  // acc += conj(a) * b
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

// Stage Z step conj(a) b with packed FP32 arithmetic: per component the same
// fused multiply-adds as cjmac, in the same order, issued two at a time:
//   acc += (a.x, a.x) * (b.x, b.y),  acc += (a.y, a.y) * (b.y, -b.x).
// A U_n value enters the z window once as (a.x, a.x), (a.y, a.y); the FP64
// kernel keeps the scalar form.
template <typename T2> struct ZRow { T2 v; };
template <> struct ZRow<float2> { float2 xx, yy; };
__device__ __forceinline__ ZRow<float2> zrow(const float2 a) {
  ZRow<float2> r;
  r.xx = make_float2(a.x, a.x);
  r.yy = make_float2(a.y, a.y);
  return r;
}
__device__ __forceinline__ ZRow<double2> zrow(const double2 a) { return ZRow<double2>{a}; }
__device__ __forceinline__ float2 zrot(const float2 b) { return make_float2(b.y, -b.x); }
__device__ __forceinline__ double2 zrot(const double2 b) { return b; }
__device__ __forceinline__ void zmac(float2& acc, const ZRow<float2>& a, const float2 b, const float2 rb) {
  acc = __ffma2_rn(a.xx, b, acc);
  acc = __ffma2_rn(a.yy, rb, acc);
}
__device__ __forceinline__ void zmac(double2& acc, const ZRow<double2>& a, const double2 b, const double2) {
  cjmac(acc, a.v, b);
}

template <typename T2>
__device__ __forceinline__ T2 czero() {
  T2 z;
  z.x = 0;
  z.y = 0;
  return z;
}

// asynchronous global -> shared copies (bypass registers; many in flight)
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}
// copy n bytes (a multiple of 8) with cp.async; 16-byte pieces when both ends allow
__device__ __forceinline__ void async_copy(void* dst, const void* src, int nbytes, int tid, int nth) {
  if ((((uintptr_t)dst | (uintptr_t)src | (uintptr_t)nbytes) & 15) == 0) {
    for (int i = tid; i < nbytes / 16; i += nth)
      cp_async16(static_cast<char*>(dst) + 16 * i, static_cast<const char*>(src) + 16 * i);
  } else {
    for (int i = tid; i < nbytes / 8; i += nth)
      cp_async8(static_cast<char*>(dst) + 8 * i, static_cast<const char*>(src) + 8 * i);
  }
}

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

// ---------------------------------------------------------------------------
// a1: c_{nk}(G) on the k sphere -> U[k][band][x][gz][y]
//     U(x, y, gz) = sum_{gx, gy} c(gx, gy, gz) e^{2 pi i (gx x / N1 + gy y / N2)}
// One block per (k, band); the sphere is scattered into a (NZ, NX, NY) box in
// shared memory, then each gz plane is transformed along y and then x.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_wf_to_mixed(RhoGeom g, const int32_t* __restrict__ gvec, const int32_t* __restrict__ npw,
              const typename C2<T>::t* __restrict__ coef, const typename C2<T>::t* __restrict__ tw1,
              const typename C2<T>::t* __restrict__ tw2, typename C2<T>::t* __restrict__ U, int k0,
              int b0, int nbo) {
  using T2 = typename C2<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* box = reinterpret_cast<T2*>(smem_raw);  // [NZ][NX][NY]
  T2* t1 = box + g.NZ * g.NX * g.NY;          // [NX][N2]
  const int tid = threadIdx.x, nth = blockDim.x;
  const int ikl = blockIdx.x / nbo;           // local k and band of the output
  const int bl = blockIdx.x - ikl * nbo;
  const int ik = k0 + ikl;                    // global k and band of the coefficients
  const int band = b0 + bl;
  const int nbox = g.NZ * g.NX * g.NY;
  for (int i = tid; i < nbox; i += nth) box[i] = czero<T2>();
  __syncthreads();
  const int np = npw[ik];
  const int32_t* gv = gvec + (size_t)ik * g.npw_max * 3;
  const T2* c = coef + ((size_t)ik * g.nb + band) * g.npw_max;
  for (int p = tid; p < np; p += nth) {
    const int gx = gv[3 * p], gy = gv[3 * p + 1], gz = gv[3 * p + 2];
    box[((gz + g.Lz) * g.NX + (gx + g.Lx)) * g.NY + (gy + g.Ly)] = c[p];
  }
  __syncthreads();
  T2* out = U + ((size_t)ikl * nbo + bl) * ((size_t)g.N1 * g.NZ * g.N2);
  if (g.N1 % 4 == 0 && g.N2 % 4 == 0) {
    // Radix-4 on the output side: with N = 4 Q and x = x0 + Q x1,
    //   u(x0 + Q x1) = sum_c i^{c x1} S_c(x0),  S_c(x0) = sum_{g = c mod 4} a(g) e^{2 pi i g x0 / N},
    // so each work item takes one x0 (all inputs once, into four partial
    // sums) and writes four outputs.
    const int Q1 = g.N1 / 4, Q2 = g.N2 / 4;
    // P[k] sums the inputs of index = k mod 4; their frequency class is
    // (c0 + k) mod 4, c0 = the class of index 0
    auto by_class = [](const T2 (&P)[4], int c0, T2 (&S)[4]) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int k = (c - c0) & 3;
        S[c] = k == 0 ? P[0] : k == 1 ? P[1] : k == 2 ? P[2] : P[3];
      }
    };
    auto emit4 = [](const T2 (&S)[4], T2 (&o)[4]) {
      o[0].x = (S[0].x + S[2].x) + (S[1].x + S[3].x);  // x1 = 0
      o[0].y = (S[0].y + S[2].y) + (S[1].y + S[3].y);
      o[1].x = (S[0].x - S[2].x) - (S[1].y - S[3].y);  // x1 = 1: S0 + i S1 - S2 - i S3
      o[1].y = (S[0].y - S[2].y) + (S[1].x - S[3].x);
      o[2].x = (S[0].x + S[2].x) - (S[1].x + S[3].x);  // x1 = 2
      o[2].y = (S[0].y + S[2].y) - (S[1].y + S[3].y);
      o[3].x = (S[0].x - S[2].x) + (S[1].y - S[3].y);  // x1 = 3: S0 - i S1 - S2 + i S3
      o[3].y = (S[0].y - S[2].y) - (S[1].x - S[3].x);
    };
    for (int zz = 0; zz < g.NZ; ++zz) {
      const T2* bz = box + zz * g.NX * g.NY;
      for (int it = tid; it < g.NX * Q2; it += nth) {
        const int gxr = it / Q2, y0 = it - gxr * Q2;
        int idx = pmod(-g.Ly * y0, g.N2);
        T2 P[4] = {czero<T2>(), czero<T2>(), czero<T2>(), czero<T2>()};  // by gyr mod 4
        const T2* brow = bz + gxr * g.NY;
        int gyr = 0;
        for (; gyr + 4 <= g.NY; gyr += 4) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            cmac(P[k], brow[gyr + k], tw2[idx]);
            idx += y0;
            if (idx >= g.N2) idx -= g.N2;
          }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (gyr + k < g.NY) {
            cmac(P[k], brow[gyr + k], tw2[idx]);
            idx += y0;
            if (idx >= g.N2) idx -= g.N2;
          }
        T2 S[4], o[4];
        by_class(P, pmod(-g.Ly, 4), S);
        emit4(S, o);
#pragma unroll
        for (int y1 = 0; y1 < 4; ++y1) t1[gxr * g.N2 + y0 + Q2 * y1] = o[y1];
      }
      __syncthreads();
      for (int it = tid; it < Q1 * g.N2; it += nth) {
        const int x0 = it / g.N2, y = it - x0 * g.N2;
        int idx = pmod(-g.Lx * x0, g.N1);
        T2 P[4] = {czero<T2>(), czero<T2>(), czero<T2>(), czero<T2>()};  // by gxr mod 4
        int gxr = 0;
        for (; gxr + 4 <= g.NX; gxr += 4) {
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            cmac(P[k], t1[(gxr + k) * g.N2 + y], tw1[idx]);
            idx += x0;
            if (idx >= g.N1) idx -= g.N1;
          }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (gxr + k < g.NX) {
            cmac(P[k], t1[(gxr + k) * g.N2 + y], tw1[idx]);
            idx += x0;
            if (idx >= g.N1) idx -= g.N1;
          }
        T2 S[4], o[4];
        by_class(P, pmod(-g.Lx, 4), S);
        emit4(S, o);
#pragma unroll
        for (int x1 = 0; x1 < 4; ++x1) out[((size_t)(x0 + Q1 * x1) * g.NZ + zz) * g.N2 + y] = o[x1];
      }
      __syncthreads();
    }
    return;
  }
  for (int zz = 0; zz < g.NZ; ++zz) {
    const T2* bz = box + zz * g.NX * g.NY;
    for (int it = tid; it < g.NX * g.N2; it += nth) {
      const int gxr = it / g.N2, y = it - gxr * g.N2;
      int idx = pmod(-g.Ly * y, g.N2);
      T2 acc = czero<T2>();
      for (int gyr = 0; gyr < g.NY; ++gyr) {
        cmac(acc, bz[gxr * g.NY + gyr], tw2[idx]);
        idx += y;
        if (idx >= g.N2) idx -= g.N2;
      }
      t1[gxr * g.N2 + y] = acc;
    }
    __syncthreads();
    for (int it = tid; it < g.N1 * g.N2; it += nth) {
      const int x = it / g.N2, y = it - x * g.N2;
      int idx = pmod(-g.Lx * x, g.N1);
      T2 acc = czero<T2>();
      for (int gxr = 0; gxr < g.NX; ++gxr) {
        cmac(acc, t1[gxr * g.N2 + y], tw1[idx]);
        idx += x;
        if (idx >= g.N1) idx -= g.N1;
      }
      out[((size_t)x * g.NZ + zz) * g.N2 + y] = acc;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// a2: rho for JM transitions (one n at k, JM consecutive m at k - q).
// ---------------------------------------------------------------------------
constexpr int kRhoThreads = 256;
constexpr int kAccMax = 16;   // register accumulators per thread
constexpr int kHZT = 3;       // hz outputs per stage-Z work item
constexpr int kHYT = 4;       // hy outputs per stage-Y work item
constexpr int kHZY = 2;       // hz columns per stage-Y work item


template <typename T2, typename TOUT>
__device__ __forceinline__ void store_out(TOUT* p, const T2 v, double scale);
template <>
__device__ __forceinline__ void store_out<double2, double2>(double2* p, const double2 v, double s) {
  *p = make_double2(v.x * s, v.y * s);
}
template <>
__device__ __forceinline__ void store_out<float2, float2>(float2* p, const float2 v, double s) {
  *p = make_float2((float)(v.x * s), (float)(v.y * s));
}

// One block of transitions (one n at k, up to JM consecutive m at k - q) of
// one task; blk is the block index within the task.
template <typename T, int JM, typename TOUT>
__device__ __forceinline__ void rho_block(const RhoTask<T, TOUT>& tk, int64_t blk,
                                          unsigned char* smem_raw) {
  using T2 = typename C2<T>::t;
  const RhoGeom& g = tk.g;
  const RhoSmem& sm = tk.sm;
  const T2* __restrict__ U = tk.U;
  const int32_t* __restrict__ kq = tk.kq;
  const int32_t* __restrict__ g0 = tk.g0;
  const int32_t* __restrict__ gresp = tk.gresp;
  const int32_t* __restrict__ gperm = tk.gperm;
  const T2* __restrict__ tw1 = tk.tw1;
  const T2* __restrict__ tw2 = tk.tw2;
  TOUT* __restrict__ R = tk.R;
  const int jm = tk.jm;
  const int tid = threadIdx.x;
  // block order: m chunk fastest, then n, then the k-pair, so that the blocks
  // resident at one time share the mixed grids of one k-pair in L2
  const int nmc = (g.Nm + jm - 1) / jm;
  const int mc = (int)(blk % nmc);
  const int nrel = (int)((blk / nmc) % g.Nn);
  const int ik = (int)(blk / ((int64_t)nmc * g.Nn));
  const int m0 = mc * jm;
  const int cm = min(jm, g.Nm - m0);
  const int ikg = g.k0 + ik;  // global k of the transition (ik is local to the block)
  const int ikp = kq[ikg];
  const int G0x = g0[3 * ikg], G0y = g0[3 * ikg + 1], G0z = g0[3 * ikg + 2];
  const int NZ = g.NZ, N2 = g.N2, HZ = g.HZ, HY = g.HY;
  const int N2P = N2 + 1;  // padded row of zs: column reads in stage Y hit distinct banks
  const size_t plane = (size_t)NZ * N2;

  T2* unp = reinterpret_cast<T2*>(smem_raw);          // [unp_rows][N2]
  T2* ums = unp + (size_t)sm.unp_rows * N2;            // [JM][NZ][N2]
  T2* zs = ums + (size_t)JM * plane;                   // [JM][HZ][N2P]
  T2* ys = zs + (size_t)JM * HZ * N2P;                 // [2][JM][HY][HZ] (two halves of y)
  T2* twx = ys + (size_t)2 * JM * HY * HZ;             // [2][HX] (double buffered)
  T2* twy = twx + 2 * g.HX;                            // [HY][N2P]: e^{2 pi i hy y / N2}
  int* gtab = reinterpret_cast<int*>(twy + (size_t)HY * N2P);  // [ng]: (hx_rel << 16) | (hy_rel * HZ + hz_rel)
  int* gout = gtab + g.ng;                             // [ng]: response index of gtab entry

  for (int i = tid; i < sm.unp_rows * N2; i += kRhoThreads) unp[i] = czero<T2>();
  // stage-X entries visit the response set in ys order (hy, hz, then hx), so
  // that neighbouring threads read neighbouring ys words; gperm holds that order
  for (int i = tid; i < g.ng; i += kRhoThreads) {
    const int p = gperm[i];
    const int hxr = gresp[3 * p] - g.Mx_lo;
    const int hyr = gresp[3 * p + 1] - g.My_lo;
    const int hzr = gresp[3 * p + 2] - g.Mz_lo;
    gtab[i] = (hxr << 16) | (hyr * HZ + hzr);
    gout[i] = p;
  }
  const int hz_base = g.Mz_lo - G0z;  // hz of hz_rel = 0
  const int hy_base = g.My_lo - G0y;
  const int hx_base = g.Mx_lo - G0x;
  for (int i = tid; i < HY * N2; i += kRhoThreads) {
    const int hyr = i / N2, y = i - hyr * N2;
    twy[hyr * N2P + y] = tw2[pmod((hy_base + hyr) * y, N2)];
  }

  // register accumulators: entry e <-> (j, i) = divmod(tid + e * threads, ng);
  // ent[e] packs its ys offset (low 20 bits) and x-twiddle row (high bits), or -1
  T2 acc[kAccMax];
  int ent[kAccMax];
  __syncthreads();  // gtab ready
#pragma unroll
  for (int e = 0; e < kAccMax; ++e) {
    acc[e] = czero<T2>();
    const int idx = tid + e * kRhoThreads;
    const int j = idx / g.ng;
    const int i = idx - j * g.ng;
    if (j < cm) {
      const int gt = gtab[i];
      ent[e] = ((gt >> 16) << 20) | (j * HY * HZ + (gt & 0xffff));
    } else {
      ent[e] = -1;
    }
  }

  const int nbu = g.nbu ? g.nbu : g.nb, nbm = g.nbm ? g.nbm : g.nb;
  const T2* Un = U + ((size_t)ik * nbu + (g.n_lo - g.bu0 + nrel)) * ((size_t)g.N1 * plane);
  const T2* Um = (tk.Um ? tk.Um : U) +
                 ((size_t)ikp * nbm + m0 + (g.diag ? g.n_lo + nrel : 0)) * ((size_t)g.N1 * plane);
  const size_t band_stride = (size_t)g.N1 * plane;
  const int nhb = (HZ + kHZT - 1) / kHZT;
  const int nyb = (HY + kHYT - 1) / kHYT;
  const int nzb = (HZ + kHZY - 1) / kHZY;
  const int yhalf = (N2 + 1) / 2;
  // radix-4 stage Y when N2 is a multiple of 4: Q4 = N2 / 4 points per
  // residue; the hy of one class mod 4 are ceil(HY / 4) at most, taken kHYT
  // at a time (ncc chunks)
  const bool radix4 = (N2 % 4) == 0;
  const int Q4 = N2 / 4;
  const int qhalf = (Q4 + 1) / 2;
  const int ncc = ((HY + 3) / 4 + kHYT - 1) / kHYT;
  __syncthreads();

  // plane loads: the n band into the padded rows, the m bands, and the
  // x twiddles; issued asynchronously (the next plane's copies overlap stages Y and X)
  auto issue_plane = [&](int x) {
    async_copy(unp + (size_t)sm.padz * N2, Un + (size_t)x * plane, (int)(plane * sizeof(T2)), tid,
               kRhoThreads);
    for (int j = 0; j < cm; ++j)
      async_copy(ums + (size_t)j * plane, Um + (size_t)j * band_stride + (size_t)x * plane,
                 (int)(plane * sizeof(T2)), tid, kRhoThreads);
  };
  issue_plane(0);
  // This thread's first work item of stages Z, Y1 and Y2 is the same for
  // every x plane: decode it once (packed), so that the plane loop divides
  // only for later rounds.
  const int zpack = (tid / N2) << 16 | (tid % N2);                 // stage Z: hb, y
  const int y1pack = radix4 ? ((tid / Q4) << 16 | (tid % Q4)) : 0;  // stage Y1: row, r
  int y2pack = 0;                                                   // stage Y2 (bit fields)
  if (radix4) {
    int r0 = tid;
    const int j = r0 % cm; r0 /= cm;
    const int c = r0 % 4; r0 /= 4;
    const int zb = r0 % nzb; r0 /= nzb;
    const int mc = r0 % ncc;
    const int half = r0 / ncc;
    y2pack = j | c << 4 | zb << 8 | mc << 16 | half << 24;
  }
  cp_async_wait_all();
  __syncthreads();

  for (int x = 0; x < g.N1; ++x) {
    T2* tx = twx + (x & 1) * g.HX;
    for (int i = tid; i < g.HX; i += kRhoThreads) tx[i] = tw1[pmod((hx_base + i) * x, g.N1)];

    // ---- stage Z: zs[j][hz][y] = sum_b conj(U_n(y, b + hz)) U_m,j(y, b)
    for (int it = tid; it < N2 * nhb; it += kRhoThreads) {
      const int hb = it == tid ? zpack >> 16 : it / N2;
      const int y = it == tid ? zpack & 0xffff : it - hb * N2;
      T2 a[JM][kHZT];
#pragma unroll
      for (int j = 0; j < JM; ++j)
#pragma unroll
        for (int h = 0; h < kHZT; ++h) a[j][h] = czero<T2>();
      // row of U_n(b + hz) in the padded array: b + hz + Lz + padz (b from -Lz)
      const T2* pn = unp + (size_t)(sm.padz + hz_base + hb * kHZT) * N2 + y;
      const T2* pm = ums + y;
      if (cm == JM) {
        // U_n rows hz .. hz + kHZT - 1 at b slide by one row per b: keep the
        // window in registers (three names, rotated by unrolling) and load
        // one new row per b
        static_assert(kHZT == 3, "the rotation below is written for three rows");
        ZRow<T2> w0 = zrow(pn[0]), w1 = zrow(pn[N2]), w2;
        const T2* pl = pn + 2 * N2;  // next row of U_n to load
        int b = 0;
        auto step = [&](const ZRow<T2>& r0, const ZRow<T2>& r1, const ZRow<T2>& r2) {
#pragma unroll
          for (int j = 0; j < JM; ++j) {
            const T2 um = pm[j * (int)plane];
            const T2 rm = zrot(um);
            zmac(a[j][0], r0, um, rm);
            zmac(a[j][1], r1, um, rm);
            zmac(a[j][2], r2, um, rm);
          }
          pm += N2;
        };
        for (; b + 3 <= NZ; b += 3) {
          w2 = zrow(pl[0]);
          step(w0, w1, w2);
          w0 = zrow(pl[N2]);
          step(w1, w2, w0);
          w1 = zrow(pl[2 * N2]);
          step(w2, w0, w1);
          pl += 3 * N2;
        }
        for (; b < NZ; ++b) {
          w2 = zrow(pl[0]);
          step(w0, w1, w2);
          w0 = w1;
          w1 = w2;
          pl += N2;
        }
      } else {
        for (int b = 0; b < NZ; ++b, pn += N2, pm += N2) {
          T2 um[JM], un[kHZT];
#pragma unroll
          for (int j = 0; j < JM; ++j) um[j] = (j < cm) ? pm[j * (int)plane] : czero<T2>();
#pragma unroll
          for (int h = 0; h < kHZT; ++h) un[h] = pn[h * N2];
#pragma unroll
          for (int j = 0; j < JM; ++j)
#pragma unroll
            for (int h = 0; h < kHZT; ++h) cjmac(a[j][h], un[h], um[j]);
        }
      }
#pragma unroll
      for (int h = 0; h < kHZT; ++h) {
        const int hzr = hb * kHZT + h;
        if (hzr < HZ) {
#pragma unroll
          for (int j = 0; j < JM; ++j)
            if (j < cm) zs[((size_t)j * HZ + hzr) * N2P + y] = a[j][h];
        }
      }
    }
    __syncthreads();

    // the planes of x are no longer read (stages Y and X use zs, ys and the
    // twiddles): start copying those of x + 1, hidden behind stages Y and X
    if (x + 1 < g.N1) issue_plane(x + 1);

    if (radix4) {
      // ---- stage Y, radix-4 form (N2 = 4 Q): with y = Q s + r,
      //   Y(hy) = sum_r e^{2 pi i hy r / N2} W_c(r),  W_c(r) = sum_s i^{c s} z(Q s + r),
      // c = hy mod 4.  Y1 replaces each zs row by W_0..W_3 (butterflies, no
      // multiplies); Y2 takes the hy of one residue class together, so that
      // they share the W_c loads, over half of the r range per work item.
      for (int it = tid; it < cm * HZ * Q4; it += kRhoThreads) {
        const int r = it == tid ? y1pack & 0xffff : it % Q4;
        const int row = it == tid ? y1pack >> 16 : it / Q4;
        T2* zr = zs + (size_t)row * N2P;
        const T2 z0 = zr[r], z1 = zr[Q4 + r], z2 = zr[2 * Q4 + r], z3 = zr[3 * Q4 + r];
        T2 w;
        w.x = (z0.x + z2.x) + (z1.x + z3.x);  // c = 0
        w.y = (z0.y + z2.y) + (z1.y + z3.y);
        zr[r] = w;
        w.x = (z0.x - z2.x) - (z1.y - z3.y);  // c = 1: z0 + i z1 - z2 - i z3
        w.y = (z0.y - z2.y) + (z1.x - z3.x);
        zr[Q4 + r] = w;
        w.x = (z0.x + z2.x) - (z1.x + z3.x);  // c = 2
        w.y = (z0.y + z2.y) - (z1.y + z3.y);
        zr[2 * Q4 + r] = w;
        w.x = (z0.x - z2.x) + (z1.y - z3.y);  // c = 3: z0 - i z1 - z2 + i z3
        w.y = (z0.y - z2.y) - (z1.x - z3.x);
        zr[3 * Q4 + r] = w;
      }
      __syncthreads();
      const int nit = 2 * cm * 4 * ncc * nzb;
      for (int it = tid; it < nit; it += kRhoThreads) {
        // j fastest, then the residue class: the 16 threads of a half-warp
        // read rows at offsets 13 j + 12 c (mod 16 words), all distinct
        int j, c, zb, mc, half;
        if (it == tid) {
          j = y2pack & 15;
          c = (y2pack >> 4) & 15;
          zb = (y2pack >> 8) & 255;
          mc = (y2pack >> 16) & 255;
          half = y2pack >> 24;
        } else {
          int r0 = it;
          j = r0 % cm; r0 /= cm;
          c = r0 % 4; r0 /= 4;
          zb = r0 % nzb; r0 /= nzb;
          mc = r0 % ncc;
          half = r0 / ncc;
        }
        const int c0 = pmod(c - hy_base, 4);  // first hy_rel of the class
        T2 a[kHYT][kHZY];
#pragma unroll
        for (int h = 0; h < kHYT; ++h)
#pragma unroll
          for (int z = 0; z < kHZY; ++z) a[h][z] = czero<T2>();
        const int hz0 = min(zb * kHZY, HZ - 1);
        const int hz1 = min(zb * kHZY + 1, HZ - 1);
        const T2* w0p = zs + ((size_t)j * HZ + hz0) * N2P + c * Q4;
        const T2* w1p = zs + ((size_t)j * HZ + hz1) * N2P + c * Q4;
        const T2* tp[kHYT];
#pragma unroll
        for (int h = 0; h < kHYT; ++h)
          tp[h] = twy + (size_t)min(c0 + 4 * (mc * kHYT + h), HY - 1) * N2P;
        const int rlo = half * qhalf, rhi = min(Q4, rlo + qhalf);
        for (int r = rlo; r < rhi; ++r) {
          const T2 v0 = w0p[r], v1 = w1p[r];
#pragma unroll
          for (int h = 0; h < kHYT; ++h) {
            const T2 t = tp[h][r];
            cmac(a[h][0], t, v0);
            cmac(a[h][1], t, v1);
          }
        }
        T2* yo = ys + (size_t)half * JM * HY * HZ;
#pragma unroll
        for (int h = 0; h < kHYT; ++h) {
          const int hyr = c0 + 4 * (mc * kHYT + h);
          if (hyr < HY) {
            yo[((size_t)j * HY + hyr) * HZ + hz0] = a[h][0];
            if (zb * kHZY + 1 < HZ) yo[((size_t)j * HY + hyr) * HZ + hz1] = a[h][1];
          }
        }
      }
      __syncthreads();
    } else {
      // ---- stage Y: ys[half][j][hy][hz] = sum_{y in half} e^{2 pi i hy y / N2} zs[j][hz][y]
      for (int it = tid; it < 2 * cm * nyb * nzb; it += kRhoThreads) {
        const int half = it / (cm * nyb * nzb);
        const int r0 = it - half * (cm * nyb * nzb);
        const int j = r0 / (nyb * nzb);
        const int r = r0 - j * (nyb * nzb);
        const int zb = r / nyb, yb = r - zb * nyb;
        T2 a[kHYT][kHZY];
  #pragma unroll
        for (int h = 0; h < kHYT; ++h)
  #pragma unroll
          for (int z = 0; z < kHZY; ++z) a[h][z] = czero<T2>();
        const int hz0 = min(zb * kHZY, HZ - 1);
        const int hz1 = min(zb * kHZY + 1, HZ - 1);
        const T2* z0p = zs + ((size_t)j * HZ + hz0) * N2P;
        const T2* z1p = zs + ((size_t)j * HZ + hz1) * N2P;
        const int hy0 = yb * kHYT;
        const int ylo = half * yhalf, yhi = min(N2, ylo + yhalf);
        const T2* tp[kHYT];
  #pragma unroll
        for (int h = 0; h < kHYT; ++h) tp[h] = twy + (size_t)min(hy0 + h, HY - 1) * N2P;
        for (int y = ylo; y < yhi; ++y) {
          const T2 v0 = z0p[y], v1 = z1p[y];
  #pragma unroll
          for (int h = 0; h < kHYT; ++h) {
            const T2 t = tp[h][y];
            cmac(a[h][0], t, v0);
            cmac(a[h][1], t, v1);
          }
        }
        T2* yo = ys + (size_t)half * JM * HY * HZ;
  #pragma unroll
        for (int h = 0; h < kHYT; ++h) {
          const int hyr = hy0 + h;
          if (hyr < HY) {
            yo[((size_t)j * HY + hyr) * HZ + hz0] = a[h][0];
            if (zb * kHZY + 1 < HZ) yo[((size_t)j * HY + hyr) * HZ + hz1] = a[h][1];
          }
        }
      }
      __syncthreads();
    }

    // ---- stage X: rho(G_i) += e^{2 pi i hx x / N1} (ys[0] + ys[1])[j][hy_i][hz_i]
    const T2* ys1 = ys + (size_t)JM * HY * HZ;
#pragma unroll
    for (int e = 0; e < kAccMax; ++e) {
      if (ent[e] >= 0) {
        const int o = ent[e] & 0xfffff;
        T2 v = ys[o];
        const T2 v1 = ys1[o];
        v.x += v1.x;
        v.y += v1.y;
        cmac(acc[e], tx[ent[e] >> 20], v);
      }
    }
    cp_async_wait_all();
    __syncthreads();
  }

  const double scale = 1.0 / ((double)g.N1 * (double)g.N2);
  const int64_t tbase = ((int64_t)ik * g.Nn + nrel) * g.Nm + m0;
#pragma unroll
  for (int e = 0; e < kAccMax; ++e) {
    if (ent[e] >= 0) {
      const int idx = tid + e * kRhoThreads;
      const int j = idx / g.ng;
      const int i = idx - j * g.ng;
      store_out<T2, TOUT>(R + (tbase + j) * g.ng + gout[i], acc[e], scale);
    }
  }
}

template <typename T, int JM, typename TOUT>
__global__ void __launch_bounds__(kRhoThreads, sizeof(T) == 4 ? 2 : 1) k_rho_pairs(const RhoTask<T, TOUT> tk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rho_block<T, JM, TOUT>(tk, blockIdx.x, smem_raw);
}

// Persistent form: every block takes the next global block index from a
// device counter until all tasks' blocks are done.  Tasks are independent
// problems (systems / q points) with their own geometry; task i owns global
// blocks [block0_i, block0_{i+1}).
template <typename T, int JM, typename TOUT>
__global__ void __launch_bounds__(kRhoThreads, sizeof(T) == 4 ? 2 : 1)
k_rho_batch(const RhoTask<T, TOUT>* __restrict__ tasks, int ntasks, int64_t total,
            unsigned long long* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RhoTask<T, TOUT> stk;
  __shared__ long long snext;
  for (;;) {
    if (threadIdx.x == 0) snext = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long gb = snext;
    if (gb >= total) break;
    if (threadIdx.x == 0) {
      int lo = 0, hi = ntasks - 1;  // last task with block0 <= gb
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (tasks[mid].block0 <= gb) lo = mid; else hi = mid - 1;
      }
      stk = tasks[lo];
    }
    __syncthreads();
    rho_block<T, JM, TOUT>(stk, gb - stk.block0, smem_raw);
    __syncthreads();
  }
}

template <typename T>
size_t rho_smem_bytes(const RhoGeom& g, const RhoSmem& sm, int jm) {
  using T2 = typename C2<T>::t;
  size_t n = (size_t)sm.unp_rows * g.N2 + (size_t)jm * g.NZ * g.N2 + (size_t)jm * g.HZ * (g.N2 + 1) +
             (size_t)2 * jm * g.HY * g.HZ + 2 * (size_t)g.HX + (size_t)g.HY * (g.N2 + 1);
  return n * sizeof(T2) + 2 * (size_t)g.ng * sizeof(int);
}

}  // namespace

template <typename T>
cudaError_t launch_wf_to_mixed(const RhoGeom& g, const int32_t* gvec, const int32_t* npw,
                               const typename C2<T>::t* coef, const typename C2<T>::t* tw1,
                               const typename C2<T>::t* tw2, typename C2<T>::t* U,
                               cudaStream_t s, int k0, int nkr, int b0, int nbo) {
  using T2 = typename C2<T>::t;
  const size_t smem = ((size_t)g.NZ * g.NX * g.NY + (size_t)g.NX * g.N2) * sizeof(T2);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (nkr <= 0) {  // every k and band
    k0 = 0;
    nkr = g.nk;
    b0 = 0;
    nbo = g.nb;
  }
  if (k0 < 0 || b0 < 0 || nbo <= 0 || k0 + nkr > g.nk || b0 + nbo > g.nb) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_wf_to_mixed<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  k_wf_to_mixed<T><<<nkr * nbo, 256, smem, s>>>(g, gvec, npw, coef, tw1, tw2, U, k0, b0, nbo);
  return cudaGetLastError();
}

template <typename T, int JM, typename TOUT>
static cudaError_t launch_rho_jm(const RhoTask<T, TOUT>& tk, size_t smem, int64_t nblocks, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_rho_pairs<T, JM, TOUT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (nblocks > 0x7fffffff) return cudaErrorInvalidValue;
  k_rho_pairs<T, JM, TOUT><<<(unsigned)nblocks, kRhoThreads, smem, s>>>(tk);
  return cudaGetLastError();
}

template <typename T, typename TOUT>
cudaError_t rho_task_make(const RhoGeom& g, const typename C2<T>::t* U, const int32_t* kq,
                          const int32_t* g0, const int32_t* gresp, const int32_t* gperm,
                          const typename C2<T>::t* tw1, const typename C2<T>::t* tw2, TOUT* R,
                          int jm_max, RhoTask<T, TOUT>* tk, size_t* smem, int64_t* nblocks) {
  if (g.Nn > 65535 || g.HX >= 32768 || g.HY * g.HZ >= 65536) return cudaErrorInvalidValue;
  RhoSmem sm;
  // rows of the zero-padded n plane: row = padz + hz + b, b in [0, NZ), hz over
  // every tile of every k-pair: [Mz_lo - G0z_max, Mz_lo + nhb * kHZT - 1 - G0z_min]
  const int nhb = (g.HZ + kHZT - 1) / kHZT;
  const int hz_min = g.Mz_lo - g.g0z_max;
  const int hz_max = g.Mz_lo + nhb * kHZT - 1 - g.g0z_min;
  sm.padz = max(0, -hz_min);
  sm.unp_rows = max(sm.padz + hz_max + g.NZ, sm.padz + g.NZ);
  const int cap = kRhoThreads * kAccMax;
  int jm = jm_max;
  while (jm > 1 && jm > g.Nm) jm /= 2;  // no wider than the m bands there are
  while (jm > 1 && jm * g.ng > cap) jm /= 2;
  if (jm * g.ng > cap) return cudaErrorInvalidValue;  // ng > 4096
  *smem = rho_smem_bytes<T>(g, sm, jm_max);
  tk->g = g;
  tk->sm = sm;
  tk->U = U;
  tk->Um = nullptr;
  tk->kq = kq;
  tk->g0 = g0;
  tk->gresp = gresp;
  tk->gperm = gperm;
  tk->tw1 = tw1;
  tk->tw2 = tw2;
  tk->R = R;
  tk->jm = jm;
  tk->block0 = 0;
  *nblocks = (int64_t)g.nk * g.Nn * ((g.Nm + jm - 1) / jm);
  return cudaSuccess;
}

template <typename T, typename TOUT>
cudaError_t launch_rho_pairs(const RhoGeom& g, const typename C2<T>::t* U, const int32_t* kq,
                             const int32_t* g0, const int32_t* gresp, const int32_t* gperm,
                             const typename C2<T>::t* tw1, const typename C2<T>::t* tw2, TOUT* R,
                             cudaStream_t s, const typename C2<T>::t* Um) {
  if (g.Nn <= 0 || g.Nm <= 0 || g.nk <= 0) return cudaSuccess;
  for (int jm : {4, 2, 1}) {
    RhoTask<T, TOUT> tk;
    size_t smem = 0;
    int64_t nb = 0;
    cudaError_t e = rho_task_make<T, TOUT>(g, U, kq, g0, gresp, gperm, tw1, tw2, R, jm, &tk, &smem, &nb);
    if (e != cudaSuccess) return e;
    tk.Um = Um;
    if (tk.jm != jm || smem > 227 * 1024) continue;
    switch (jm) {
      case 4: return launch_rho_jm<T, 4, TOUT>(tk, smem, nb, s);
      case 2: return launch_rho_jm<T, 2, TOUT>(tk, smem, nb, s);
      default: return launch_rho_jm<T, 1, TOUT>(tk, smem, nb, s);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T, typename TOUT>
cudaError_t launch_rho_batch(const RhoTask<T, TOUT>* tasks_dev, int ntasks, int64_t total, int jm,
                             size_t smem, unsigned long long* counter, int nsm, cudaStream_t s) {
  if (ntasks == 0 || total == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  int per_sm = 1;
  const int grid = nsm * 2;
  (void)per_sm;
  switch (jm) {
    case 4:
      e = cudaFuncSetAttribute(k_rho_batch<T, 4, TOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_rho_batch<T, 4, TOUT><<<grid, kRhoThreads, smem, s>>>(tasks_dev, ntasks, total, counter);
      break;
    case 2:
      e = cudaFuncSetAttribute(k_rho_batch<T, 2, TOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_rho_batch<T, 2, TOUT><<<grid, kRhoThreads, smem, s>>>(tasks_dev, ntasks, total, counter);
      break;
    default:
      e = cudaFuncSetAttribute(k_rho_batch<T, 1, TOUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      k_rho_batch<T, 1, TOUT><<<grid, kRhoThreads, smem, s>>>(tasks_dev, ntasks, total, counter);
  }
  return cudaGetLastError();
}

template cudaError_t launch_wf_to_mixed<double>(const RhoGeom&, const int32_t*, const int32_t*,
                                                const double2*, const double2*, const double2*,
                                                double2*, cudaStream_t, int, int, int, int);
template cudaError_t launch_wf_to_mixed<float>(const RhoGeom&, const int32_t*, const int32_t*,
                                               const float2*, const float2*, const float2*,
                                               float2*, cudaStream_t, int, int, int, int);
template cudaError_t rho_task_make<double, double2>(const RhoGeom&, const double2*, const int32_t*,
                                                    const int32_t*, const int32_t*, const int32_t*,
                                                    const double2*, const double2*, double2*, int,
                                                    RhoTask<double, double2>*, size_t*, int64_t*);
template cudaError_t rho_task_make<float, float2>(const RhoGeom&, const float2*, const int32_t*,
                                                  const int32_t*, const int32_t*, const int32_t*,
                                                  const float2*, const float2*, float2*, int,
                                                  RhoTask<float, float2>*, size_t*, int64_t*);
template cudaError_t launch_rho_batch<double, double2>(const RhoTask<double, double2>*, int, int64_t, int,
                                                       size_t, unsigned long long*, int, cudaStream_t);
template cudaError_t launch_rho_batch<float, float2>(const RhoTask<float, float2>*, int, int64_t, int,
                                                     size_t, unsigned long long*, int, cudaStream_t);
template cudaError_t launch_rho_pairs<double, double2>(const RhoGeom&, const double2*,
                                                       const int32_t*, const int32_t*,
                                                       const int32_t*, const int32_t*,
                                                       const double2*, const double2*, double2*,
                                                       cudaStream_t, const double2*);
template cudaError_t launch_rho_pairs<float, float2>(const RhoGeom&, const float2*, const int32_t*,
                                                     const int32_t*, const int32_t*, const int32_t*,
                                                     const float2*, const float2*, float2*,
                                                     cudaStream_t, const float2*);

}  // namespace chi0
