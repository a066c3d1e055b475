// Mixed-precision chi0 contraction on the 5th-generation tensor cores
// (tcgen05 + TMEM + TMA, sm_103a).
//
// chi0(w) = sum_t w_t rho_t rho_t^H (Appendix B: frequency factors times
// frequency-independent rho rho^* products) is a Hermitian rank-K update with
// K = number of transitions.  It is computed in real arithmetic: with
// P_t = w_t rho_t and rows m = 2 i + c (c = 0 real, 1 imaginary part),
//
//     A[m][t] = P_t(i).c,   B[m][t] = rho_t(i).c,   D = A B^T  (2 N_G x 2 N_G),
//     Re chi_ij = D[2i][2j] + D[2i+1][2j+1],   Im chi_ij = D[2i+1][2j] - D[2i][2j+1].
//
// When every weight has one sign s (on the imaginary axis w_t has the sign of
// the pole, the same for all transitions unless occupations and energies are
// out of order or an extrapolar term is added), the Hermitian contraction
// takes the one-operand form chi0 = s S S^H with S_t = sqrt|w_t| rho_t: A and
// B are both S (one operand set per frequency, half the bytes the tiles
// stream), and the sign is applied when the partials are summed.
//
// Precision: each FP32 operand is split into two BF16 numbers, x = hi + lo
// (hi = bf16(x), lo = bf16(x - hi), together ~16 bits), and
// D = Ah Bh + Ah Bl + Al Bh (the lo*lo term, <= 2^-16 of a product, is
// dropped; in the one-operand form lo carries a correction that keeps the
// diagonal free of that term's bias, see k_prep).  The tensor core's FP32 accumulation loses low bits on every
// addition with a bias (measured: the error grows linearly with the number of
// accumulated transitions, ~2e-6 relative per 512), so each TMEM accumulation
// is limited to 128 transitions; the epilogue warps fold those sub-sums into
// compensated FP32 sums, and the per-CTA partials are added in FP64.  Only the
// lower-triangle 128 x 128 tiles of D are computed (chi0 is Hermitian).
//
// Kernel structure (one CTA = one tile x one range of transitions, 6 warps):
//   warp 0      TMA producer: Ah, Al, Bh, Bl tiles (128 x 64 BF16, 128-byte
//               swizzle) into a 3-stage shared-memory ring (mbarrier tx counts)
//   warp 1      TMEM allocation (2 x 128 columns); one elected thread issues
//               tcgen05.mma (M = N = 128, K = 16, BF16 -> FP32) into the two
//               accumulators in turn and tcgen05.commit
//   warps 2-5   epilogue: tcgen05.ld of a finished 128 x 128 accumulator,
//               combination of 2 x 2 real blocks into complex entries,
//               compensated accumulation in registers, final FP64 partial
// Every mbarrier wait is bounded: on timeout the kernel raises the device
// error flag (reported as CHI0_ETIMEOUT), skips the remaining work, frees its
// TMEM and returns.
// Every contraction now runs the wide variant of this kernel, k_herk_wide:
// 128 x 256 tiles, N = 256 products, twelve warps (see its comment), over the
// lower-triangle tiles (real weights), over every tile (the complex weights
// of a real frequency), or over every tile with FP32 tiles out (the
// self-energy product).  k_herk_bf16x3 below, the 128 x 128 form, is no longer
// launched; its comment describes the work units and the pipeline that
// k_herk_wide widens.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "ctx.cuh"

namespace chi0 {

namespace {

constexpr int kBM = 128;             // tile rows (real), = 64 complex G
constexpr int kBN = 128;             // tile cols (real)
constexpr int kBK = 64;              // transitions per pipeline stage (128 bytes of BF16)
constexpr int kStages = 3;
constexpr int kSubKB = 2;           // k-blocks per TMEM accumulation (128 transitions)
constexpr int kTileBytes = kBM * kBK * 2;         // 16 KB per operand tile
constexpr int kStageBytes = 4 * kTileBytes;       // Ah, Al, Bh, Bl
constexpr int kSmemBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
constexpr int kThreads = 192;
constexpr long long kSpinCycles = 4000000000LL;   // ~2 s at 2 GHz
constexpr int kErrTimeout = 2;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait on an mbarrier phase.  Gives up after kSpinCycles or when
// another role has already given up (abort flag in shared memory).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                          int* err) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (*(volatile int*)(err + 1)) {  // another CTA already gave up
      *abort_flag = 1;
      return false;
    }
    if (clock64() - t0 > kSpinCycles) {
      *abort_flag = 1;
      atomicExch(err + 1, kErrTimeout);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, BF16 inputs, FP32 accumulator
__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major tile of 128-byte rows written by
// TMA with 128-byte swizzle; 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
  d |= (uint64_t)1 << 16;                   // leading-dimension offset (unused with swizzle)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride-dimension offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // 128-byte swizzle
  return d;
}

// Instruction descriptor: kind::f16, A = B = BF16, D = F32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tri_decode(int tile, int& I, int& J) {
  int i = (int)((sqrt(8.0 * (double)tile + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= tile) ++i;
  while (i * (i + 1) / 2 > tile) --i;
  I = i;
  J = tile - i * (i + 1) / 2;
}

// Compensated accumulation (Neumaier): s + c carries the running sum.
__device__ __forceinline__ void nsum(float& s, float& c, float x) {
  const float t = s + x;
  c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
  s = t;
}

// Work unit = one lower-triangle tile (I, J) x one range of k-blocks (a
// split) -- or, with nI > 0, one tile of the full grid of nI row tiles of A
// by ntiles / nI row tiles of B (I = tile % nI, J = tile / nI; A and B then
// have their own row paddings mpad and mpad_b); unit u is tile u % ntiles of
// split u / ntiles, so the CTAs resident
// at one time read the same k-blocks (shared in L2).  The kernel is
// persistent: CTA c takes units c, c + gridDim.x, ...; the stage ring and the
// accumulator ping-pong run on across units, so the next unit's operands
// stream in while the epilogue finishes the last one, and the CTA holds its SM
// for the whole launch (blocks of a concurrent kernel fill what it leaves).
// The MMA thread alternates between two TMEM accumulators, one per sub-chunk
// of kSubKB k-blocks; the epilogue warps drain a finished sub-chunk (complex
// combination, compensated FP32 sums held in registers) while the other one
// fills, so the tensor core's FP32 accumulation never runs longer than
// kSubKB * 64 transitions.
// At most 224 registers: two warps of this CTA share a sub-partition, and
// 2 x 224 x 32 leaves 2048 of its 16384 registers for a 64-register warp of
// a concurrent Dyson block.
__global__ void __maxnreg__(224)
k_herk_bf16x3(const __grid_constant__ CUtensorMap tm_ah, const __grid_constant__ CUtensorMap tm_al,
              const __grid_constant__ CUtensorMap tm_bh, const __grid_constant__ CUtensorMap tm_bl,
              int total_kb, int kb_per_split, int mpad, double2* __restrict__ part, int ntiles,
              int nunits, int* __restrict__ err, int nI, int mpad_b, int f32out,
              const int2* __restrict__ ranges) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + kStages * kStageBytes);
  const uint32_t bar_full = smem_u32(bars);                   // [kStages]
  const uint32_t bar_empty = smem_u32(bars + kStages);        // [kStages]
  const uint32_t bar_accf = smem_u32(bars + 2 * kStages);     // [2] accumulator full
  const uint32_t bar_acce = smem_u32(bars + 2 * kStages + 2); // [2] accumulator drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {  // an earlier CTA timed out: skip the work (one read, so the whole CTA agrees)
    volatile int* skip = reinterpret_cast<volatile int*>(tmem_slot + 2);
    if (threadIdx.x == 0) *skip = *(volatile int*)(err + 1);
    __syncthreads();
    if (*skip) return;
  }
  // k-block range of a unit
  auto unit_range = [&](int u, int& kb0, int& nkb) {
    if (ranges) {  // k-block range of split u / ntiles from the table (a pole group)
      const int2 r = ranges[u / ntiles];
      kb0 = r.x;
      nkb = r.y;
      return;
    }
    kb0 = (u / ntiles) * kb_per_split;
    nkb = max(0, min(total_kb, kb0 + kb_per_split) - kb0);
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_accf + 8 * b, 1);
      mbar_init(bar_acce + 8 * b, 4);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0 && lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_ah) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_al) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_bh) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_bl) : "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), 2 * kBN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int gk = 0;  // k-blocks loaded by this CTA so far (stage ring position)
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int I, J, kb0, nkb;
        const int tile = u % ntiles;
        if (nI > 0) {
          I = tile % nI;
          J = tile / nI;
        } else {
          tri_decode(tile, I, J);
        }
        unit_range(u, kb0, nkb);
        for (int k = 0; k < nkb; ++k, ++gk) {
          const int s = gk % kStages;
          const uint32_t ph = (uint32_t)((gk / kStages) & 1);
          if (!mbar_wait(bar_empty + 8 * s, ph ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          const uint32_t st = base + s * kStageBytes;
          mbar_expect_tx(bar_full + 8 * s, kStageBytes);
          // k-blocked layout: block kb starts at row kb * mpad (A) and kb * mpad_b (B)
          const int row = (kb0 + k) * mpad, row_b = (kb0 + k) * mpad_b;
          tma_load_2d(st, &tm_ah, 0, row + I * kBM, bar_full + 8 * s);
          tma_load_2d(st + kTileBytes, &tm_al, 0, row + I * kBM, bar_full + 8 * s);
          tma_load_2d(st + 2 * kTileBytes, &tm_bh, 0, row_b + J * kBN, bar_full + 8 * s);
          tma_load_2d(st + 3 * kTileBytes, &tm_bl, 0, row_b + J * kBN, bar_full + 8 * s);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(kBM, kBN);
      int gk = 0, gsc = 0;  // stage ring position, sub-chunks issued by this CTA
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int kb0, nkb;
        unit_range(u, kb0, nkb);
        const int nsub = (nkb + kSubKB - 1) / kSubKB;
        int k = 0;
        for (int sc = 0; sc < nsub; ++sc, ++gsc) {
          const int b = gsc & 1;
          if (!mbar_wait(bar_acce + 8 * b, (uint32_t)(((gsc >> 1) & 1) ^ 1), abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)(b * kBN);
          const int kend = min(nkb, (sc + 1) * kSubKB);
          for (int kk0 = 0; k < kend; ++k, ++kk0, ++gk) {
            const int s = gk % kStages;
            const uint32_t ph = (uint32_t)((gk / kStages) & 1);
            if (!mbar_wait(bar_full + 8 * s, ph, abort_flag, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = base + s * kStageBytes;
            const uint64_t dah = desc_sw128(st);
            const uint64_t dal = desc_sw128(st + kTileBytes);
            const uint64_t dbh = desc_sw128(st + 2 * kTileBytes);
            const uint64_t dbl = desc_sw128(st + 3 * kTileBytes);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
              const uint64_t off = (uint64_t)((kk * 32) >> 4);  // 16 BF16 = 32 bytes along K
              umma_bf16(acc, dah + off, dbh + off, idesc, (kk0 > 0 || kk > 0) ? 1u : 0u);
              umma_bf16(acc, dah + off, dbl + off, idesc, 1u);
              umma_bf16(acc, dal + off, dbh + off, idesc, 1u);
            }
            umma_commit(bar_empty + 8 * s);  // stage free once these MMAs have read it
          }
          if (!ok) break;
          umma_commit(bar_accf + 8 * b);     // sub-chunk sum ready in accumulator b
        }
      }
    }
  } else {
    // ---------------- epilogue (warps 2..5 -> TMEM lane quadrants 2, 3, 0, 1)
    const int q = warp & 3;
    const bool odd = (lane & 1) != 0;
    int gsc = 0;  // sub-chunks drained by this CTA
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      int kb0, nkb;
      unit_range(u, kb0, nkb);
      const int nsub = (nkb + kSubKB - 1) / kSubKB;
      float accs[32][2], accc[32][2];  // compensated sums: [complex entry][re, im]
#pragma unroll
      for (int e = 0; e < 32; ++e) accs[e][0] = accs[e][1] = accc[e][0] = accc[e][1] = 0.f;
      for (int sc = 0; sc < nsub; ++sc, ++gsc) {
        const int b = gsc & 1;
        ok = __all_sync(0xffffffffu,
                        mbar_wait(bar_accf + 8 * b, (uint32_t)((gsc >> 1) & 1), abort_flag, err) ? 1 : 0) != 0;
        if (!ok) break;
        tc_fence_after();
        const uint32_t acc = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kBN);
#pragma unroll
        for (int cb = 0; cb < kBN / 16; ++cb) {
          uint32_t v[16];
          tmem_ld16(acc + (uint32_t)(cb * 16), v);
          // rows 2i (even lane) and 2i+1 (odd lane); each lane combines 4 of the 8 complex columns
          float recv[8];
#pragma unroll
          for (int k2 = 0; k2 < 8; ++k2) {
            const float send = __uint_as_float(odd ? v[k2] : v[8 + k2]);
            recv[k2] = __shfl_xor_sync(0xffffffffu, send, 1);
          }
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const float r0c0 = odd ? recv[2 * jj] : __uint_as_float(v[2 * jj]);           // D[2i][2j]
            const float r0c1 = odd ? recv[2 * jj + 1] : __uint_as_float(v[2 * jj + 1]);   // D[2i][2j+1]
            const float r1c0 = odd ? __uint_as_float(v[8 + 2 * jj]) : recv[2 * jj];       // D[2i+1][2j]
            const float r1c1 = odd ? __uint_as_float(v[9 + 2 * jj]) : recv[2 * jj + 1];   // D[2i+1][2j+1]
            const int e = cb * 4 + jj;
            nsum(accs[e][0], accc[e][0], r0c0 + r1c1);
            nsum(accs[e][1], accc[e][1], r1c0 - r0c1);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar_acce + 8 * b) : "memory");
      }
      if (!ok) break;
      const int il = (q * 32 + lane) >> 1;  // complex row of the tile
      const size_t obase = ((size_t)(u / ntiles) * ntiles + (u % ntiles)) * (size_t)(kBM / 2) * (kBN / 2) +
                           (size_t)il * (kBN / 2) + (odd ? 4 : 0);
      if (f32out) {  // the compensated sums rounded to FP32 (the tile layout of part, 8-byte entries)
        float2* out = reinterpret_cast<float2*>(part) + obase;
#pragma unroll
        for (int cb = 0; cb < kBN / 16; ++cb)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int e = cb * 4 + jj;
            out[cb * 8 + jj] = make_float2(accs[e][0] + accc[e][0], accs[e][1] + accc[e][1]);
          }
      } else {
        double2* out = part + obase;
#pragma unroll
        for (int cb = 0; cb < kBN / 16; ++cb)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int e = cb * 4 + jj;
            out[cb * 8 + jj] = make_double2((double)accs[e][0] + (double)accc[e][0],
                                            (double)accs[e][1] + (double)accc[e][1]);
          }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * kBN);
  }
}

// ---- wide tiles: 128 rows of A x 256 rows of B per unit ---------------------
// The Hermitian contraction with N = 256 per MMA: each k-block stages Ah, Al
// (128 rows) and Bh, Bl (256 rows, two TMA boxes each) and issues 12
// tcgen05.mma of 128 x 256 x 16, so one operand byte feeds twice the products
// of a 128 x 128 tile (half the shared-memory and L2 traffic per product of
// A, and twice the work per stage in flight).  Two stages of 96 KB.  The
// accumulators take all 512 TMEM columns (two of 256, ping-pong); eight
// epilogue warps drain them, two per TMEM lane quadrant, each holding the
// compensated sums of 128 of the 256 columns (as many as the narrow kernel's
// four).  Warps 0..3 (producer, MMA issuer, two idle) give registers to the
// epilogue warpgroups: 384 threads launched at 144 registers (55,296), then
// 4 x 32 x 40 + 8 x 32 x 192 = 54,272 after the hand-over, which leaves a
// 128-thread, 64-register Dyson block room beside it (10,240 registers,
// 2,816 per sub-partition).
// Tiles: (I, J) with I in [2J, nI), nI = mpad / 128 row tiles of A and nJ =
// mpad / 256 column tiles of B (mpad a multiple of 256): every real entry
// (r, c) with r >= c lies in one of them.  Tile index = sum_{J' < J} (nI - 2J')
// + (I - 2J).  Partial output: 64 complex rows x 128 complex columns per
// unit.
constexpr int kWN = 256;                          // tile cols (real)
constexpr int kWStages = 2;
constexpr int kWTileA = kBM * kBK * 2;            // 16 KB
constexpr int kWTileB = kWN * kBK * 2;            // 32 KB
constexpr int kWStageBytes = 2 * kWTileA + 2 * kWTileB;   // 96 KB
constexpr int kWSmemBytes = kWStages * kWStageBytes + 1024 + 256;
constexpr int kWThreads = 384;
constexpr int kWPart = (kBM / 2) * (kWN / 2);     // complex entries of a partial tile

__device__ __forceinline__ void wide_decode(int tile, int nI, int& I, int& J) {
  int J0 = 0, base = 0;
  while (base + (nI - 2 * J0) <= tile) {
    base += nI - 2 * J0;
    ++J0;
  }
  J = J0;
  I = 2 * J0 + (tile - base);
}

__device__ __forceinline__ void setmaxnreg_dec40() {
  asm volatile("setmaxnreg.dec.sync.aligned.u32 40;" ::: "memory");
}
__device__ __forceinline__ void setmaxnreg_inc192() {
  asm volatile("setmaxnreg.inc.sync.aligned.u32 192;" ::: "memory");
}

__global__ void __maxnreg__(144)
k_herk_wide(const __grid_constant__ CUtensorMap tm_ah, const __grid_constant__ CUtensorMap tm_al,
            const __grid_constant__ CUtensorMap tm_bh, const __grid_constant__ CUtensorMap tm_bl, int total_kb,
            int kb_per_split, int mpad, double2* __restrict__ part, int ntiles, int nunits,
            int* __restrict__ err, int nI, const int2* __restrict__ ranges, int full, int mpad_b,
            int f32out) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + kWStages * kWStageBytes);
  const uint32_t bar_full = smem_u32(bars);                    // [kWStages]
  const uint32_t bar_empty = smem_u32(bars + kWStages);        // [kWStages]
  const uint32_t bar_accf = smem_u32(bars + 2 * kWStages);     // [2] accumulator full
  const uint32_t bar_acce = smem_u32(bars + 2 * kWStages + 2); // [2] accumulator drained
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kWStages + 4);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  {  // an earlier CTA timed out: skip the work (one read, so the whole CTA agrees)
    volatile int* skip = reinterpret_cast<volatile int*>(tmem_slot + 2);
    if (threadIdx.x == 0) *skip = *(volatile int*)(err + 1);
    __syncthreads();
    if (*skip) return;
  }
  auto unit_range = [&](int u, int& kb0, int& nkb) {
    if (ranges) {
      const int2 r = ranges[u / ntiles];
      kb0 = r.x;
      nkb = r.y;
      return;
    }
    kb0 = (u / ntiles) * kb_per_split;
    nkb = max(0, min(total_kb, kb0 + kb_per_split) - kb0);
  };

  if (threadIdx.x == 0) {
    for (int st = 0; st < kWStages; ++st) {
      mbar_init(bar_full + 8 * st, 1);
      mbar_init(bar_empty + 8 * st, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_accf + 8 * b, 1);
      mbar_init(bar_acce + 8 * b, 8);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0 && lane == 0) {
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_ah) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_al) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_bh) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tm_bl) : "memory");
  }
  if (warp == 1) tmem_alloc(smem_u32(tmem_slot), 2 * kWN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp < 4) {
    setmaxnreg_dec40();
    if (warp == 0 && lane == 0) {
      // ---------------- TMA producer
      int gk = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int I, J, kb0, nkb;
        if (full) {   // every tile: I fastest
          I = (u % ntiles) % nI;
          J = (u % ntiles) / nI;
        } else {
          wide_decode(u % ntiles, nI, I, J);
        }
        unit_range(u, kb0, nkb);
        for (int k = 0; k < nkb; ++k, ++gk) {
          const int st = gk % kWStages;
          const uint32_t ph = (uint32_t)((gk / kWStages) & 1);
          if (!mbar_wait(bar_empty + 8 * st, ph ^ 1u, abort_flag, err)) {
            ok = false;
            break;
          }
          const uint32_t sb = base + st * kWStageBytes;
          mbar_expect_tx(bar_full + 8 * st, kWStageBytes);
          const int row = (kb0 + k) * mpad, rowb = (kb0 + k) * mpad_b;
          tma_load_2d(sb, &tm_ah, 0, row + I * kBM, bar_full + 8 * st);
          tma_load_2d(sb + kWTileA, &tm_al, 0, row + I * kBM, bar_full + 8 * st);
          tma_load_2d(sb + 2 * kWTileA, &tm_bh, 0, rowb + J * kWN, bar_full + 8 * st);
          tma_load_2d(sb + 2 * kWTileA + kWTileA, &tm_bh, 0, rowb + J * kWN + kBM, bar_full + 8 * st);
          tma_load_2d(sb + 2 * kWTileA + kWTileB, &tm_bl, 0, rowb + J * kWN, bar_full + 8 * st);
          tma_load_2d(sb + 2 * kWTileA + kWTileB + kWTileA, &tm_bl, 0, rowb + J * kWN + kBM, bar_full + 8 * st);
        }
      }
    } else if (warp == 1 && lane == 0) {
      // ---------------- MMA issuer
      constexpr uint32_t idesc = idesc_bf16(kBM, kWN);
      int gk = 0, gsc = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
        int kb0, nkb;
        unit_range(u, kb0, nkb);
        const int nsub = (nkb + kSubKB - 1) / kSubKB;
        int k = 0;
        for (int sc = 0; sc < nsub; ++sc, ++gsc) {
          const int b = gsc & 1;
          if (!mbar_wait(bar_acce + 8 * b, (uint32_t)(((gsc >> 1) & 1) ^ 1), abort_flag, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + (uint32_t)(b * kWN);
          const int kend = min(nkb, (sc + 1) * kSubKB);
          for (int kk0 = 0; k < kend; ++k, ++kk0, ++gk) {
            const int st = gk % kWStages;
            const uint32_t ph = (uint32_t)((gk / kWStages) & 1);
            if (!mbar_wait(bar_full + 8 * st, ph, abort_flag, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t sb = base + st * kWStageBytes;
            const uint64_t dah = desc_sw128(sb);
            const uint64_t dal = desc_sw128(sb + kWTileA);
            const uint64_t dbh = desc_sw128(sb + 2 * kWTileA);
            const uint64_t dbl = desc_sw128(sb + 2 * kWTileA + kWTileB);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
              const uint64_t off = (uint64_t)((kk * 32) >> 4);
              umma_bf16(acc, dah + off, dbh + off, idesc, (kk0 > 0 || kk > 0) ? 1u : 0u);
              umma_bf16(acc, dah + off, dbl + off, idesc, 1u);
              umma_bf16(acc, dal + off, dbh + off, idesc, 1u);
            }
            umma_commit(bar_empty + 8 * st);
          }
          if (!ok) break;
          umma_commit(bar_accf + 8 * b);
        }
      }
    }
  } else {
    setmaxnreg_inc192();
    // ---------------- epilogue: warps 4..11; TMEM lane quadrant warp % 4,
    // column half (warp - 4) / 4 of the 256 accumulator columns
    const int q = warp & 3;
    const int hcol = (warp - 4) >> 2;
    const bool odd = (lane & 1) != 0;
    int gsc = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok; u += gridDim.x) {
      int kb0, nkb;
      unit_range(u, kb0, nkb);
      const int nsub = (nkb + kSubKB - 1) / kSubKB;
      float accs[32][2], accc[32][2];
#pragma unroll
      for (int e = 0; e < 32; ++e) accs[e][0] = accs[e][1] = accc[e][0] = accc[e][1] = 0.f;
      for (int sc = 0; sc < nsub; ++sc, ++gsc) {
        const int b = gsc & 1;
        ok = __all_sync(0xffffffffu,
                        mbar_wait(bar_accf + 8 * b, (uint32_t)((gsc >> 1) & 1), abort_flag, err) ? 1 : 0) != 0;
        if (!ok) break;
        tc_fence_after();
        const uint32_t acc = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * kWN + hcol * kBN);
#pragma unroll
        for (int cb = 0; cb < kBN / 16; ++cb) {
          uint32_t v[16];
          tmem_ld16(acc + (uint32_t)(cb * 16), v);
          float recv[8];
#pragma unroll
          for (int k2 = 0; k2 < 8; ++k2) {
            const float send = __uint_as_float(odd ? v[k2] : v[8 + k2]);
            recv[k2] = __shfl_xor_sync(0xffffffffu, send, 1);
          }
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const float r0c0 = odd ? recv[2 * jj] : __uint_as_float(v[2 * jj]);
            const float r0c1 = odd ? recv[2 * jj + 1] : __uint_as_float(v[2 * jj + 1]);
            const float r1c0 = odd ? __uint_as_float(v[8 + 2 * jj]) : recv[2 * jj];
            const float r1c1 = odd ? __uint_as_float(v[9 + 2 * jj]) : recv[2 * jj + 1];
            const int e = cb * 4 + jj;
            nsum(accs[e][0], accc[e][0], r0c0 + r1c1);
            nsum(accs[e][1], accc[e][1], r1c0 - r0c1);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar_acce + 8 * b) : "memory");
      }
      if (!ok) break;
      const int il = (q * 32 + lane) >> 1;  // complex row of the tile
      if (f32out) {
        // the compensated sums rounded to FP32, written as the 64 x 64
        // complex tiles of the full grid of 128-row B tiles: this warp's 64
        // columns are tile I + (2 J + hcol) nI (one k range per tile), which
        // exists while its B rows lie within mpad_b
        const int tile = u % ntiles, I = tile % nI, Jn = 2 * (tile / nI) + hcol;
        if (Jn * kBN < mpad_b) {
          float2* out = reinterpret_cast<float2*>(part) + ((size_t)Jn * nI + I) * (size_t)(kBM / 2) * (kBN / 2) +
                        (size_t)il * (kBN / 2) + (odd ? 4 : 0);
#pragma unroll
          for (int cb = 0; cb < kBN / 16; ++cb)
#pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
              const int e = cb * 4 + jj;
              out[cb * 8 + jj] = make_float2(accs[e][0] + accc[e][0], accs[e][1] + accc[e][1]);
            }
        }
      } else {
        double2* out = part + (size_t)u * kWPart + (size_t)il * (kWN / 2) + hcol * (kBN / 2) + (odd ? 4 : 0);
#pragma unroll
        for (int cb = 0; cb < kBN / 16; ++cb)
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int e = cb * 4 + jj;
            out[cb * 8 + jj] = make_double2((double)accs[e][0] + (double)accc[e][0],
                                            (double)accs[e][1] + (double)accc[e][1]);
          }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, 2 * kWN);
  }
}

// hi/lo BF16 split of the real operand in k-blocked layout: element (m, t),
// m = 2 i + c, sits at [t / 64][m][t % 64] (each block of 64 transitions holds
// all rows, 128 bytes per row), so one 128-row TMA box is one contiguous 16 KB
// chunk.  value = (w_t if w else 1) * R[t][i].c; zero outside (nt, ng).
constexpr int kPT = 64;  // transitions per tile (= one k-block)
constexpr int kPI = 32;  // complex G per tile

// Up to kPrepGroup operands are split in one pass, so that R is read once
// for all of them (the split is bound by HBM traffic: R in, hi/lo out).
// Operand g is R scaled by the weights wr[g][t] (NULL: unit weights), by
// sqrt|wr[g][t]| when sq[g] is set (the one-operand form S = rho diag(sqrt|w|)
// of a contraction whose weights share one sign), or, with wi[g] given, by the
// complex weights wr[g][t] + i wi[g][t] (a real-axis frequency: A = w rho with
// rows Re = wr x - wi y, Im = wr y + wi x).  In the one-operand form the
// dropped lo lo^T is a sum of squares on the diagonal (a bias of about
// -2.8e-6 relative on every chi0_ii, where the two-operand form's dropped
// terms have no sign); the split then stores lo' = lo + lo^2 / (2 hi) in
// place of lo, which makes the diagonal's products hi^2 + 2 hi lo' = x^2.
constexpr int kPrepGroup = 8;
struct PrepOut {
  __nv_bfloat16* hi[kPrepGroup];
  __nv_bfloat16* lo[kPrepGroup];
  const double* wr[kPrepGroup];
  const double* wi[kPrepGroup];
  int sq[kPrepGroup];
};

// perm (optional): row t of the operand is transition perm[t] of R (-1: a
// zero row), for nt rows; without it row t is transition t.
__global__ void __launch_bounds__(256)
k_prep(const float2* __restrict__ R, int ngrp, int64_t nt, int ng, int mpad, const __grid_constant__ PrepOut out,
       const int64_t* __restrict__ perm) {
  __shared__ float tile[2 * kPI][kPT + 1];
  __shared__ float ws[kPrepGroup][kPT];   // weights converted once per transition (FP64 is slow here)
  __shared__ float wsi[kPrepGroup][kPT];  // imaginary parts of complex weights
  __shared__ float rs[kPrepGroup][kPT];   // one-operand form: 0.5 / sqrt|w| (0 for w = 0)
  __shared__ int64_t src[kPT];            // transition of each row (-1: zero row)
  const int64_t kb = blockIdx.x;
  const int64_t t0 = kb * kPT;
  const int i0 = blockIdx.y * kPI;
  for (int tl = threadIdx.x; tl < kPT; tl += 256) {
    const int64_t t = t0 + tl;
    src[tl] = t < nt ? (perm ? perm[t] : t) : -1;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < ngrp * kPT; e += 256) {
    const int g = e / kPT, tl = e % kPT;
    const int64_t t = src[tl];
    if (out.wr[g] && t >= 0) {
      const double wv = out.wr[g][t];
      // sqrt|w| in FP32 (2^-24 relative, far below the split's 2^-17; the
      // FP64 square root is slow on this part)
      const float sw = sqrtf(fabsf((float)wv));
      ws[g][tl] = out.sq[g] ? sw : (float)wv;
      rs[g][tl] = sw > 0.f ? 0.5f / sw : 0.f;
    } else {
      ws[g][tl] = 1.f;
      rs[g][tl] = 0.f;
    }
    wsi[g][tl] = (out.wi[g] && t >= 0) ? (float)out.wi[g][t] : 0.f;
  }
  for (int e = threadIdx.x; e < kPT * kPI; e += 256) {
    const int tl = e / kPI, il = e % kPI;
    const int64_t t = src[tl];
    const int i = i0 + il;
    const float2 v = (t >= 0 && i < ng) ? R[t * ng + i] : make_float2(0.f, 0.f);
    tile[2 * il][tl] = v.x;
    tile[2 * il + 1][tl] = v.y;
  }
  __syncthreads();
  const size_t blk = (size_t)kb * mpad * kPT;
  // every element pair once, through all operands of the pass: the R values
  // and their reciprocals (for the one-operand correction) are shared
  for (int e = threadIdx.x; e < 2 * kPI * (kPT / 2); e += 256) {
    const int ml = e / (kPT / 2), tp = e % (kPT / 2);
    const size_t off = blk + (size_t)(2 * i0 + ml) * kPT + 2 * tp;
    const float y0 = tile[ml][2 * tp], y1 = tile[ml][2 * tp + 1];
    const float ry0 = y0 != 0.f ? __fdividef(1.f, y0) : 0.f;
    const float ry1 = y1 != 0.f ? __fdividef(1.f, y1) : 0.f;
    for (int g = 0; g < ngrp; ++g) {
      float x0, x1;
      if (out.wi[g]) {
        // row 2 i: Re(w rho) = wr x - wi y; row 2 i + 1: Im(w rho) = wr y + wi x
        const int mr = ml & ~1;
        const float a0 = tile[mr][2 * tp], b0 = tile[mr + 1][2 * tp];
        const float a1 = tile[mr][2 * tp + 1], b1 = tile[mr + 1][2 * tp + 1];
        if (ml & 1) {
          x0 = fmaf(ws[g][2 * tp], b0, wsi[g][2 * tp] * a0);
          x1 = fmaf(ws[g][2 * tp + 1], b1, wsi[g][2 * tp + 1] * a1);
        } else {
          x0 = fmaf(ws[g][2 * tp], a0, -wsi[g][2 * tp] * b0);
          x1 = fmaf(ws[g][2 * tp + 1], a1, -wsi[g][2 * tp + 1] * b1);
        }
      } else {
        x0 = y0 * ws[g][2 * tp];
        x1 = y1 * ws[g][2 * tp + 1];
      }
      const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
      float r0 = x0 - __low2float(h), r1 = x1 - __high2float(h);   // exact
      if (out.sq[g]) {
        // one-operand form: lo' = lo + lo^2 / (2 hi), so that the products
        // taken, hi^2 + 2 hi lo', equal x^2 up to the (unbiased) rounding of
        // lo'; otherwise the dropped lo^2 would bias every diagonal entry.
        // 1 / (2 x) = (1 / R) (0.5 / sqrt|w|) stands in for 1 / (2 hi): they
        // differ by 2^-9 relative, far below what the correction needs
        r0 = fmaf(r0 * r0, ry0 * rs[g][2 * tp], r0);
        r1 = fmaf(r1 * r1, ry1 * rs[g][2 * tp + 1], r1);
      }
      const __nv_bfloat162 l = __floats2bfloat162_rn(r0, r1);
      *reinterpret_cast<__nv_bfloat162*>(out.hi[g] + off) = h;
      *reinterpret_cast<__nv_bfloat162*>(out.lo[g] + off) = l;
    }
  }
}

// chi[i][j] (i >= j) = sum over chunks of the partials (FP64), mirrored.
// Position of the complex entry (i, j), i >= j, among the Hermitian
// contraction's partial tiles: narrow 64 x 64 tiles in lower-triangle order,
// or wide 64 x 128 tiles (I = i / 64, J = j / 128, I >= 2J) column by column.
__device__ __forceinline__ void herm_pos(int i, int j, int wide, int nI, int& tile, size_t& off) {
  if (wide) {
    const int I = i / (kBM / 2), J = j / (kWN / 2);
    tile = J * nI - J * (J - 1) + (I - 2 * J);
    off = (size_t)(i % (kBM / 2)) * (kWN / 2) + (j % (kWN / 2));
  } else {
    const int I = i / (kBM / 2), J = j / (kBN / 2);
    tile = I * (I + 1) / 2 + J;
    off = (size_t)(i % (kBM / 2)) * (kBN / 2) + (j % (kBN / 2));
  }
}

__global__ void k_tc_reduce(const double2* __restrict__ part, int nchunks, int ntiles, int ng,
                            double2* __restrict__ chi, int accumulate, int wide, int nI, int tile_elems,
                            double sign) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ng * ng) return;
  const int i = (int)(e / ng), j = (int)(e % ng);
  if (i < j) return;
  int tile;
  size_t off;
  herm_pos(i, j, wide, nI, tile, off);
  double sx = 0.0, sy = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const double2 v = part[((size_t)c * ntiles + tile) * tile_elems + off];
    sx += v.x;
    sy += v.y;
  }
  if (i == j) sy = 0.0;  // Hermitian: real diagonal
  sx *= sign;            // the one-operand form sums sign S S^H
  sy *= sign;
  if (accumulate) {      // add to the sum of the earlier transition blocks
    const double2 a = chi[(size_t)i * ng + j];
    sx += a.x;
    sy += a.y;
  }
  chi[(size_t)i * ng + j] = make_double2(sx, sy);
  if (i != j) chi[(size_t)j * ng + i] = make_double2(sx, -sy);
}

// chi[i][j] = sum over chunks of the partials of the full tile grid (A rows i,
// B rows j: tile (i / 64) + (j / cols) nT with cols = 64 complex columns per
// 128 x 128 tile or 128 per 128 x 256 tile), every entry (no Hermitian
// symmetry).
__global__ void k_tc_reduce_full(const double2* __restrict__ part, int nchunks, int ntiles, int nT, int ng,
                                 double2* __restrict__ chi, int accumulate, int cols) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ng * ng) return;
  const int i = (int)(e / ng), j = (int)(e % ng);
  const int tile = i / (kBM / 2) + (j / cols) * nT;
  const size_t off = (size_t)(i % (kBM / 2)) * cols + (j % cols);
  double sx = 0.0, sy = 0.0;
  for (int c = 0; c < nchunks; ++c) {
    const double2 v = part[((size_t)c * ntiles + tile) * (kBM / 2) * cols + off];
    sx += v.x;
    sy += v.y;
  }
  if (accumulate) {
    sx += chi[e].x;
    sy += chi[e].y;
  }
  chi[e] = make_double2(sx, sy);
}

struct TcState {
  DevBuf ah[kPrepGroup], al[kPrepGroup], bh, bl, part;
  CUtensorMap m_ah[kPrepGroup], m_al[kPrepGroup], m_bh, m_bl;
  int64_t kpad = 0;
  int mpad = 0, ntiles = 0, total_kb = 0, kbpc = 0, nchunks = 0;
  int ntiles_f = 0, kbpc_f = 0, nchunks_f = 0;   // full tile grid (complex weights)
  int group = 1;  // frequencies per operand-split pass (A buffers in use)
  int nsm = 1;    // persistent contraction grid
  // Hermitian contraction: wide tiles (128 x 256, k_herk_wide) or narrow ones
  // (128 x 128, k_herk_bf16x3); nI row tiles of 128 (and nJ column tiles of
  // 256 when wide); tile_elems complex entries per partial tile
  int wide = 1, nI = 0, nJ = 0, tile_elems = (kBM / 2) * (kBN / 2);
};

// Tile layout of the Hermitian contraction for an operand of mpad rows.
void herm_tiles(TcState& t) {
  t.nI = t.mpad / kBM;
  if (t.wide) {
    t.nJ = t.mpad / kWN;
    t.ntiles = t.nI * t.nJ - t.nJ * (t.nJ - 1);
    t.tile_elems = kWPart;
  } else {
    t.nJ = t.nI;
    t.ntiles = t.nI * (t.nI + 1) / 2;
    t.tile_elems = (kBM / 2) * (kBN / 2);
  }
}

// One Hermitian contraction launch (lower-triangle tiles x transition splits).
// one_op: the one-operand form D = S S^T, both tiles read from operand g;
// otherwise A is operand g and B the unit-weight operand.
cudaError_t launch_herm(chi0_ctx* c, TcState& t, int g, int kbpc, int nunits, const int2* ranges, bool one_op) {
  const unsigned grid = (unsigned)std::min(nunits, std::max(1, t.nsm));
  const CUtensorMap& mbh = one_op ? t.m_ah[g] : t.m_bh;
  const CUtensorMap& mbl = one_op ? t.m_al[g] : t.m_bl;
  if (t.wide)
    k_herk_wide<<<grid, kWThreads, kWSmemBytes, c->st>>>(t.m_ah[g], t.m_al[g], mbh, mbl, t.total_kb, kbpc, t.mpad,
                                                          (double2*)t.part.p, t.ntiles, nunits, (int*)c->d_err.p,
                                                          t.nI, ranges, 0, t.mpad, 0);
  else
    k_herk_bf16x3<<<grid, kThreads, kSmemBytes, c->st>>>(t.m_ah[g], t.m_al[g], mbh, mbl, t.total_kb, kbpc, t.mpad,
                                                          (double2*)t.part.p, t.ntiles, nunits, (int*)c->d_err.p, 0,
                                                          t.mpad, 0, ranges);
  return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D map over the k-blocked operand viewed as [nkb * mpad rows][64 BF16]
bool make_map(CUtensorMap* m, void* ptr, int64_t kpad, int mpad) {
  auto enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kBK, (cuuint64_t)(kpad / kBK) * (cuuint64_t)mpad};
  cuuint64_t strides[1] = {(cuuint64_t)kBK * 2};
  cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

chi0_status tc_plan(chi0_ctx* c, int64_t nt, int ng, int nw) {
  if (!c->tc) c->tc = new TcState();
  TcState& t = *static_cast<TcState*>(c->tc);
  t.wide = 1;
  t.mpad = (2 * ng + kWN - 1) / kWN * kWN;   // a multiple of the wide tile's 256 columns
  t.kpad = (nt + kBK - 1) / kBK * kBK;
  const int nT = t.mpad / kBM;
  herm_tiles(t);
  t.total_kb = (int)(t.kpad / kBK);
  // split the transitions so that the grid fills whole waves of one CTA per SM
  int nsm = 148;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
  }
  t.nsm = nsm;
  auto choose_split = [&](int ntiles, int& kbpc, int& nchunks) {
    int nsplit = 1;
    double best = 1e30;
    for (int sp = 1; sp <= 64; ++sp) {
      const int kbps = (t.total_kb + sp - 1) / sp;
      if (sp > 1 && kbps < 8 * kSubKB) break;  // keep every CTA busy for a while
      const int ctas = ntiles * sp;
      const int waves = (ctas + nsm - 1) / nsm;
      // time ~ waves * work per CTA; prefer fewer partials on ties
      const double cost = (double)waves * kbps + 4.0 * sp;
      if (cost < best) {
        best = cost;
        nsplit = sp;
      }
    }
    kbpc = (t.total_kb + nsplit - 1) / nsplit;
    nchunks = (t.total_kb + kbpc - 1) / kbpc;
  };
  choose_split(t.ntiles, t.kbpc, t.nchunks);
  // the full tile grid of the complex contraction of a real-axis frequency
  // (128 x 256 tiles with the wide kernel)
  t.ntiles_f = t.wide ? nT * (t.mpad / kWN) : nT * nT;
  choose_split(t.ntiles_f, t.kbpc_f, t.nchunks_f);
  if (t.kpad / kPT > 0x7fffffff / t.mpad)
    return ctx_fail(c, CHI0_EUNSUPPORTED, "too many transitions for one contraction");
  const size_t opb = (size_t)t.mpad * t.kpad * 2;
  chi0_status s;
  // the unit-weight operand B is read only by the two-operand form (weights
  // of mixed signs) and by the complex contractions of real frequencies
  const bool need_b = c->herk_sign == 0 || c->has_real;
  if (need_b) {
    if ((s = ctx_ensure(c, t.bh, opb, "B hi")) != CHI0_OK) return s;
    if ((s = ctx_ensure(c, t.bl, opb, "B lo")) != CHI0_OK) return s;
  }
  // a batch problem (group_cap > 0) keeps room for twice the planned
  // partials, for the split candidates of tc_tune_split
  const size_t room = c->group_cap > 0 ? 2 : 1;
  const size_t nbytes = std::max((size_t)t.nchunks * t.ntiles * room * t.tile_elems,
                                  c->has_real ? (size_t)t.nchunks_f * t.ntiles_f * (kBM / 2) * (t.wide ? kWN : kBN) / 2
                                              : (size_t)0);
  if ((s = ctx_ensure(c, t.part, nbytes * 16, "chunk partials")) != CHI0_OK)
    return s;
  // A buffers for up to kPrepGroup frequencies, as far as half of the free
  // device memory allows (one pair is always needed)
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    int have = 0;
    while (have < kPrepGroup && t.ah[have].bytes >= opb && t.al[have].bytes >= opb) ++have;
    int g = std::min(kPrepGroup, std::max(1, nw));
    if (c->group_cap > 0) g = std::min(g, c->group_cap);
    while (g > std::max(1, have) && (double)(g - have) * 2.0 * (double)opb > 0.5 * (double)free_b) --g;
    t.group = g;
  }
  for (int g = 0; g < t.group; ++g) {
    if ((s = ctx_ensure(c, t.ah[g], opb, "A hi")) != CHI0_OK) return s;
    if ((s = ctx_ensure(c, t.al[g], opb, "A lo")) != CHI0_OK) return s;
    if (!make_map(&t.m_ah[g], t.ah[g].p, t.kpad, t.mpad) || !make_map(&t.m_al[g], t.al[g].p, t.kpad, t.mpad))
      return ctx_fail(c, CHI0_ECUDA, "cuTensorMapEncodeTiled failed");
  }
  if (need_b && (!make_map(&t.m_bh, t.bh.p, t.kpad, t.mpad) || !make_map(&t.m_bl, t.bl.p, t.kpad, t.mpad)))
    return ctx_fail(c, CHI0_ECUDA, "cuTensorMapEncodeTiled failed");
  cudaError_t e = cudaFuncSetAttribute(k_herk_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_herk_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_herk_wide, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  // The whole shared-memory carveout on every SM this path touches, so that
  // an SM running a contraction CTA (193 KB) keeps room for the small blocks
  // of the Dyson step of the previous frequency (a carveout sized to the CTA
  // alone would leave none).
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_herk_bf16x3, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_prep, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_reduce, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tc_reduce_full, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return ctx_fail(c, CHI0_ECUDA, cudaGetErrorString(e));
  return CHI0_OK;
}

namespace {

// Grouped contraction, per frequency: chi[i][j] (i >= j) = sum_g F_g(w) M_g[i][j]
// over the pole groups (Appendix B: a frequency factor per group times the
// frequency-independent sum of the group's rho rho^* terms), M_g read from
// the partial tiles of the group's contraction unit; up to kCombW
// frequencies per launch, compensated FP32 sums, Hermitian mirror.
constexpr int kCombW = 8;
__global__ void __launch_bounds__(256)
k_grp_combine(const double2* __restrict__ part, const float* __restrict__ F, int ngroups, int ntiles, int ng,
              int w0, int nwc, double2* __restrict__ chi, int wide, int nI, int tile_elems) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)ng * ng) return;
  const int i = (int)(e / ng), j = (int)(e % ng);
  if (i < j) return;
  int tile;
  size_t off;
  herm_pos(i, j, wide, nI, tile, off);
  float sx[kCombW], sy[kCombW], cx[kCombW], cy[kCombW];
#pragma unroll
  for (int w = 0; w < kCombW; ++w) sx[w] = sy[w] = cx[w] = cy[w] = 0.f;
  for (int g = 0; g < ngroups; ++g) {
    const double2 p = part[((size_t)g * ntiles + tile) * tile_elems + off];
    const float px = (float)p.x, py = (float)p.y;
#pragma unroll
    for (int w = 0; w < kCombW; ++w) {
      if (w < nwc) {
        const float f = F[(size_t)(w0 + w) * ngroups + g];
        nsum(sx[w], cx[w], f * px);
        nsum(sy[w], cy[w], f * py);
      }
    }
  }
  const size_t n2 = (size_t)ng * ng;
#pragma unroll
  for (int w = 0; w < kCombW; ++w) {
    if (w < nwc) {
      const double x = (double)sx[w] + (double)cx[w];
      const double y = i == j ? 0.0 : (double)sy[w] + (double)cy[w];
      double2* o = chi + (size_t)(w0 + w) * n2;
      o[(size_t)i * ng + j] = make_double2(x, y);
      if (i != j) o[(size_t)j * ng + i] = make_double2(x, -y);
    }
  }
}

}  // namespace

chi0_status tc_plan_grouped(chi0_ctx* c, int ng, int nw) {
  if (!c->tc) c->tc = new TcState();
  TcState& t = *static_cast<TcState*>(c->tc);
  t.wide = 1;
  t.mpad = (2 * ng + kWN - 1) / kWN * kWN;
  t.kpad = c->kgrp;
  herm_tiles(t);
  t.total_kb = (int)(t.kpad / kBK);
  t.group = 1;
  int nsm = 148, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  t.nsm = nsm;
  if (t.kpad / kPT > 0x7fffffff / t.mpad || (int64_t)c->ngroups * t.ntiles > 0x7fffffff)
    return ctx_fail(c, CHI0_EUNSUPPORTED, "too many grouped transitions for one contraction");
  const size_t opb = (size_t)t.mpad * t.kpad * 2;
  chi0_status s;
  DevBuf* ops[] = {&t.ah[0], &t.al[0]};   // one operand (S S^H form)
  for (DevBuf* b : ops)
    if ((s = ctx_ensure(c, *b, opb, "grouped operands")) != CHI0_OK) return s;
  if ((s = ctx_ensure(c, t.part, (size_t)c->ngroups * t.ntiles * t.tile_elems * 16, "group sums")) != CHI0_OK)
    return s;
  if (!make_map(&t.m_ah[0], t.ah[0].p, t.kpad, t.mpad) || !make_map(&t.m_al[0], t.al[0].p, t.kpad, t.mpad))
    return ctx_fail(c, CHI0_ECUDA, "cuTensorMapEncodeTiled failed");
  cudaError_t e = cudaFuncSetAttribute(k_herk_bf16x3, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_herk_bf16x3, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_herk_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_herk_wide, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return ctx_fail(c, CHI0_ECUDA, cudaGetErrorString(e));
  (void)nw;
  return CHI0_OK;
}

chi0_status tc_launch_grouped(chi0_ctx* c, double2* chi, const cudaEvent_t* ev_freq) {
  if (!c->tc) return ctx_fail(c, CHI0_ESTATE, "grouped contraction not planned");
  TcState& t = *static_cast<TcState*>(c->tc);
  const int ng = c->cfg.ng, nw = c->nwv;
  const int64_t n2 = (int64_t)ng * ng;
  const dim3 pgrid((unsigned)(t.kpad / kPT), (unsigned)(t.mpad / 2 / kPI));
  const int64_t* perm = (const int64_t*)c->d_tperm.p;
  // one operand in group order, S = rho diag(sqrt(pref (f_m - f_n))) (frequency
  // independent; every grouped transition has f_m - f_n > 0), so that the
  // group sums are M_g = S_g S_g^H
  PrepOut oa{};
  oa.hi[0] = (__nv_bfloat16*)t.ah[0].p;
  oa.lo[0] = (__nv_bfloat16*)t.al[0].p;
  oa.wr[0] = (const double*)c->d_ga.p;
  oa.sq[0] = 1;
  stage_begin(c, CHI0_STAGE_WEIGHTS);
  k_prep<<<pgrid, 256, 0, c->st>>>((const float2*)c->d_R.p, 1, t.kpad, ng, t.mpad, oa, perm);
  stage_end(c, CHI0_STAGE_WEIGHTS, 1);
  // one unit per (tile, group): the group sums M_g, tile by tile
  const int nunits = t.ntiles * c->ngroups;
  stage_begin(c, CHI0_STAGE_CONTRACT);
  launch_herm(c, t, 0, t.total_kb, nunits, (const int2*)c->d_grange.p, true);
  stage_end(c, CHI0_STAGE_CONTRACT, 1);
  // chi0 at every frequency from the group sums and the groups' factors
  const unsigned cgrid = (unsigned)((n2 + 255) / 256);
  int nlaunch = 0;
  stage_begin(c, CHI0_STAGE_REDUCE);
  for (int w0 = 0; w0 < nw; w0 += kCombW, ++nlaunch) {
    const int nwc = std::min(kCombW, nw - w0);
    k_grp_combine<<<cgrid, 256, 0, c->st>>>((const double2*)t.part.p, (const float*)c->d_gfac.p, c->ngroups,
                                            t.ntiles, ng, w0, nwc, chi, t.wide, t.nI, t.tile_elems);
    if (ev_freq)
      for (int w = w0; w < w0 + nwc; ++w) cudaEventRecord(ev_freq[w], c->st);
  }
  stage_end(c, CHI0_STAGE_REDUCE, nlaunch);
  const double tile_bytes = (double)t.tile_elems * 16;
  c->stage[CHI0_STAGE_WEIGHTS].bytes = (double)c->nt * ng * 8 + 4.0 * t.mpad * t.kpad;
  c->stage[CHI0_STAGE_CONTRACT].bytes = 4.0 * t.mpad * t.kpad + (double)nunits * tile_bytes;
  // the work done: one Hermitian contraction over the transitions in group
  // order (not one per frequency), then the combination per frequency
  c->stage[CHI0_STAGE_CONTRACT].flops = 4.0 * (double)ng * (ng + 1) * (double)t.kpad;
  c->stage[CHI0_STAGE_REDUCE].flops = 2.0 * (double)ng * (ng + 1) * (double)c->ngroups * nw;
  c->stage[CHI0_STAGE_REDUCE].bytes = (double)nlaunch * nunits * tile_bytes + (double)n2 * nw * 16;
  c->tc_issued_flops = 3.0 * 2.0 * kBM * (t.wide ? kWN : kBN) * (double)t.kpad * t.ntiles;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(c, CHI0_ECUDA, cudaGetErrorString(e));
  return CHI0_OK;
}

chi0_status tc_launch(chi0_ctx* c, const void* R, const double* w, int64_t nt, int ng, int nw,
                      double2* chi, const cudaEvent_t* ev_freq, const cudaEvent_t* ev_prep,
                      const BgApply* bg, const int* vkind, int accumulate) {
  if (!c->tc) return ctx_fail(c, CHI0_ESTATE, "tensor-core contraction not planned");
  TcState& t = *static_cast<TcState*>(c->tc);
  const dim3 pgrid((unsigned)(t.kpad / kPT), (unsigned)(t.mpad / 2 / kPI));
  const int64_t n2 = (int64_t)ng * ng;
  const int nT = t.mpad / kBM;
  // jobs: an entry of the frequency list with real weights is one Hermitian
  // contraction (lower-triangle tiles); a real-axis frequency (entries of
  // kinds 1 and 2: the real and imaginary parts of its complex weights) is one
  // contraction with complex weights over the full tile grid, whose result is
  // chi0 of that frequency, written at its first entry
  struct Job {
    int v;
    bool cplx;
  };
  std::vector<Job> jobs;
  for (int v = 0; v < nw; ++v) {
    const bool cplx = vkind && vkind[v] == 1 && v + 1 < nw && vkind[v + 1] == 2;
    jobs.push_back({v, cplx});
    if (cplx) ++v;
  }
  // A Hermitian job whose weights share one sign takes the one-operand form
  // chi0 = sign S S^H with S = rho diag(sqrt|w|): one operand set per
  // frequency, read for both tiles.  Otherwise (mixed signs) A = w rho and
  // B = rho; the complex jobs also read B.
  const bool one_op = c->herk_sign != 0;
  bool need_b = !one_op;
  for (const Job& jb : jobs) need_b |= jb.cplx;
  if (need_b) {   // B = rho (frequency independent)
    PrepOut ob{};
    ob.hi[0] = (__nv_bfloat16*)t.bh.p;
    ob.lo[0] = (__nv_bfloat16*)t.bl.p;
    stage_begin(c, CHI0_STAGE_WEIGHTS);
    k_prep<<<pgrid, 256, 0, c->st>>>((const float2*)R, 1, nt, ng, t.mpad, ob, nullptr);
    stage_end(c, CHI0_STAGE_WEIGHTS, 1);
  }
  const int nunits = t.ntiles * t.nchunks, nunits_f = t.ntiles_f * t.nchunks_f;
  const unsigned hgrid = (unsigned)std::min(nunits, std::max(1, t.nsm));
  const unsigned hgrid_f = (unsigned)std::min(nunits_f, std::max(1, t.nsm));
  int passes = 0, nherm = 0, nfull = 0;
  for (size_t j0 = 0; j0 < jobs.size(); j0 += t.group, ++passes) {
    const int gw = (int)std::min<size_t>(t.group, jobs.size() - j0);
    PrepOut oa{};
    for (int g = 0; g < gw; ++g) {
      const Job& jb = jobs[j0 + g];
      oa.hi[g] = (__nv_bfloat16*)t.ah[g].p;
      oa.lo[g] = (__nv_bfloat16*)t.al[g].p;
      oa.wr[g] = w + (size_t)jb.v * nt;
      oa.wi[g] = jb.cplx ? w + (size_t)(jb.v + 1) * nt : nullptr;
      oa.sq[g] = one_op && !jb.cplx;
    }
    stage_begin(c, CHI0_STAGE_WEIGHTS);
    k_prep<<<pgrid, 256, 0, c->st>>>((const float2*)R, gw, nt, ng, t.mpad, oa, nullptr);
    stage_end(c, CHI0_STAGE_WEIGHTS, 1);
    if (ev_prep)
      for (int g = 0; g < gw; ++g) {
        cudaEventRecord(ev_prep[jobs[j0 + g].v], c->st);
        if (jobs[j0 + g].cplx) cudaEventRecord(ev_prep[jobs[j0 + g].v + 1], c->st);
      }
    for (int g = 0; g < gw; ++g) {
      const Job& jb = jobs[j0 + g];
      double2* out = chi + (size_t)jb.v * n2;
      stage_begin(c, CHI0_STAGE_CONTRACT);
      if (jb.cplx) {
        if (t.wide)
          k_herk_wide<<<hgrid_f, kWThreads, kWSmemBytes, c->st>>>(
              t.m_ah[g], t.m_al[g], t.m_bh, t.m_bl, t.total_kb, t.kbpc_f, t.mpad, (double2*)t.part.p, t.ntiles_f,
              nunits_f, (int*)c->d_err.p, nT, nullptr, 1, t.mpad, 0);
        else
          k_herk_bf16x3<<<hgrid_f, kThreads, kSmemBytes, c->st>>>(
              t.m_ah[g], t.m_al[g], t.m_bh, t.m_bl, t.total_kb, t.kbpc_f, t.mpad, (double2*)t.part.p, t.ntiles_f,
              nunits_f, (int*)c->d_err.p, nT, t.mpad, 0, nullptr);
        ++nfull;
      } else {
        launch_herm(c, t, g, t.kbpc, nunits, nullptr, one_op);
        ++nherm;
      }
      stage_end(c, CHI0_STAGE_CONTRACT, 1);
      stage_begin(c, CHI0_STAGE_REDUCE);
      if (jb.cplx)
        k_tc_reduce_full<<<(unsigned)((n2 + 255) / 256), 256, 0, c->st>>>(
            (const double2*)t.part.p, t.nchunks_f, t.ntiles_f, nT, ng, out, accumulate, (t.wide ? kWN : kBN) / 2);
      else
        k_tc_reduce<<<(unsigned)((n2 + 255) / 256), 256, 0, c->st>>>((const double2*)t.part.p, t.nchunks, t.ntiles,
                                                                      ng, out, accumulate, t.wide, t.nI,
                                                                      t.tile_elems, one_op ? (double)c->herk_sign : 1.0);
      int nk = 1;
      if (bg) {
        launch_bg_apply(bg->P + (size_t)jb.v * bg->nd, bg->didx, ng, bg->nd, 1, out, c->st, 0);
        ++nk;
        if (jb.cplx) {   // + i (Hermitised P of the imaginary parts)
          launch_bg_apply(bg->P + (size_t)(jb.v + 1) * bg->nd, bg->didx, ng, bg->nd, 1, out, c->st, 1);
          ++nk;
        }
      }
      stage_end(c, CHI0_STAGE_REDUCE, nk);
      if (ev_freq) {
        cudaEventRecord(ev_freq[jb.v], c->st);
        if (jb.cplx) cudaEventRecord(ev_freq[jb.v + 1], c->st);
      }
    }
  }
  const double tile_bytes = (double)t.tile_elems * 16;
  const double tile_bytes_f = (double)(kBM / 2) * ((t.wide ? kWN : kBN) / 2) * 16;
  // operand split: R read once per pass, hi/lo written (B once if needed, A per job)
  c->stage[CHI0_STAGE_WEIGHTS].bytes += (double)(passes + (need_b ? 1 : 0)) * nt * ng * 8 +
                                        (double)(jobs.size() + (need_b ? 1 : 0)) * 4.0 * t.mpad * t.kpad;
  // contraction: each launch streams its operands (hi and lo) once, one set
  // in the one-operand form and two otherwise, and writes its chunk partials
  c->stage[CHI0_STAGE_CONTRACT].bytes =
      (double)nherm * (one_op ? 4.0 : 8.0) * t.mpad * t.kpad + (double)nfull * 8.0 * t.mpad * t.kpad +
      (double)nherm * t.nchunks * t.ntiles * tile_bytes + (double)nfull * t.nchunks_f * t.ntiles_f * tile_bytes_f;
  c->stage[CHI0_STAGE_REDUCE].bytes =
      (double)nherm * t.nchunks * t.ntiles * tile_bytes + (double)nfull * t.nchunks_f * t.ntiles_f * tile_bytes_f +
      (double)(nherm + nfull) * n2 * 16;
  // tensor-core work actually issued: 3 BF16 products over the tiles of each launch
  c->tc_issued_flops = 3.0 * 2.0 * kBM * (double)t.kpad *
                      ((double)(t.wide ? kWN : kBN) * (t.ntiles * nherm + t.ntiles_f * nfull));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ctx_fail(c, CHI0_ECUDA, cudaGetErrorString(e));
  return CHI0_OK;
}

void tc_release(chi0_ctx* c) {
  if (!c->tc) return;
  TcState* t = static_cast<TcState*>(c->tc);
  DevBuf* bufs[] = {&t->bh, &t->bl, &t->part};
  for (DevBuf* b : bufs)
    if (b->p && !b->borrowed) cudaFree(b->p);
  for (int g = 0; g < kPrepGroup; ++g) {
    if (t->ah[g].p && !t->ah[g].borrowed) cudaFree(t->ah[g].p);
    if (t->al[g].p && !t->al[g].borrowed) cudaFree(t->al[g].p);
  }
  delete t;
  c->tc = nullptr;
}

std::vector<DevBuf*> tc_scratch_slots(chi0_ctx* c) {
  std::vector<DevBuf*> v;
  if (!c->tc) c->tc = new TcState();
  TcState& t = *static_cast<TcState*>(c->tc);
  v.push_back(&t.bh);
  v.push_back(&t.bl);
  v.push_back(&t.part);
  for (int g = 0; g < kPrepGroup; ++g) {
    v.push_back(&t.ah[g]);
    v.push_back(&t.al[g]);
  }
  return v;
}

// The contraction of the first entry of the frequency list (its operands
// split as tc_launch does) timed for the planned transition split and for
// half and twice as many splits; the fastest is kept for the later launches.
chi0_status tc_tune_split(chi0_ctx* c, float* best_ms) {
  if (!c->tc || c->nt == 0) return CHI0_OK;
  TcState& t = *static_cast<TcState*>(c->tc);
  const int ng = c->cfg.ng;
  const dim3 pgrid((unsigned)(t.kpad / kPT), (unsigned)(t.mpad / 2 / kPI));
  const bool one_op = c->herk_sign != 0;
  if (!one_op) {
    PrepOut ob{};
    ob.hi[0] = (__nv_bfloat16*)t.bh.p;
    ob.lo[0] = (__nv_bfloat16*)t.bl.p;
    k_prep<<<pgrid, 256, 0, c->st>>>((const float2*)c->d_R.p, 1, c->nt, ng, t.mpad, ob, nullptr);
  }
  PrepOut oa{};
  oa.hi[0] = (__nv_bfloat16*)t.ah[0].p;
  oa.lo[0] = (__nv_bfloat16*)t.al[0].p;
  oa.wr[0] = (const double*)c->d_w.p;
  oa.sq[0] = one_op;
  k_prep<<<pgrid, 256, 0, c->st>>>((const float2*)c->d_R.p, 1, c->nt, ng, t.mpad, oa, nullptr);
  const size_t cap = t.part.bytes / ((size_t)t.tile_elems * 16);
  const int base_split = (t.total_kb + t.kbpc - 1) / t.kbpc;
  int best_kbpc = t.kbpc, best_n = t.nchunks;
  float best = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, CHI0_ECUDA, "events for the split tuning");
  }
  for (int sp : {base_split, std::max(1, base_split / 2), 2 * base_split}) {
    const int kbpc = (t.total_kb + sp - 1) / sp;
    const int nchunks = (t.total_kb + kbpc - 1) / kbpc;
    if ((size_t)nchunks * t.ntiles > cap) continue;
    const int nunits = t.ntiles * nchunks;
    const unsigned grid = (unsigned)std::min(nunits, std::max(1, t.nsm));
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {   // the first run warms the caches
      cudaEventRecord(e0, c->st);
      launch_herm(c, t, 0, kbpc, nunits, nullptr, one_op);
      (void)grid;
      cudaEventRecord(e1, c->st);
      if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        cudaGetLastError();
        ms = 1e30f;
      }
    }
    if (ms < best) {
      best = ms;
      best_kbpc = kbpc;
      best_n = nchunks;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  t.kbpc = best_kbpc;
  t.nchunks = best_n;
  if (best_ms) *best_ms = best;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CHI0_OK : ctx_fail(c, CHI0_ECUDA, cudaGetErrorString(e));
}

// ---- failure detection: the bounded wait ---------------------------------------
// One thread waits on an mbarrier that nothing arrives on, through the same
// bounded wait as the contraction's producer, MMA and epilogue roles: after
// kSpinCycles it gives up, raises the device error flag (reported as
// CHI0_ETIMEOUT by the next synchronising call) and the kernel returns.

namespace {

__global__ void k_wait_probe(int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    mbar_wait(smem_u32(&bar), 0u, &abort_flag, err);
  }
}

}  // namespace

cudaError_t launch_wait_probe(int* err, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(err);
  return cudaGetLastError();
}

// ---- self-energy kernel I (Eq. I_c) -----------------------------------------
// Y(i, t) = sum_j W^d_ij conj(rho_t(j)) is the same complex product as the
// chi0 contraction, C_ij = sum_K A_K(i) conj(B_K(j)), with K = G' (ng values)
// instead of the transitions: A = W^d (rows 2 i + c), B = rho of the
// transitions t of the quasiparticle window (rows 2 t + c), the full grid of
// 128 x 128 tiles, one k range per tile (no chunk partials: each tile's sum
// is Y itself, rounded to FP32).  Transitions are ordered t = ((k nb) + m) nqp + a,
// so that the partners a of one (k, m) are adjacent columns of Y.

namespace {

struct SigTc {
  DevBuf ah, al, bh, bl;
  CUtensorMap m_ah, m_al, m_bh, m_bl;
  int64_t kpad = 0, T = 0, mpad_b = 0;
  int ng = 0, mpad_a = 0, nI = 0, nJ = 0, nsm = 1;
};

__device__ __forceinline__ void split_store(float x0, float x1, __nv_bfloat16* hi, __nv_bfloat16* lo, size_t off) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
  const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - __low2float(h), x1 - __high2float(h));
  *reinterpret_cast<__nv_bfloat162*>(hi + off) = h;
  *reinterpret_cast<__nv_bfloat162*>(lo + off) = l;
}

// B: row 2 t + c, column j holds rho_t(j).c (zero outside t < T, j < ng); the
// rho kernel's row of transition t = ((k nb) + m) nqp + a is ((k nqp) + a) nb + m.
__global__ void __launch_bounds__(256)
k_sig_bsplit(const float2* __restrict__ R, int64_t T, int nqp, int nb, int ng, int64_t mpad_b,
             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t r0 = (int64_t)blockIdx.x * 64;  // 64 rows = 32 transitions
  const int kb = blockIdx.y;                    // 64 values of j
  for (int e = threadIdx.x; e < 64 * 32; e += 256) {
    const int ml = e >> 5, jp = e & 31;
    const int64_t m = r0 + ml, t = m >> 1;
    const int j = kb * 64 + 2 * jp;
    float x0 = 0.f, x1 = 0.f;
    if (t < T) {
      const int64_t a = t % nqp, g = t / nqp;
      const float2* row = R + (((g / nb) * nqp + a) * nb + g % nb) * (int64_t)ng;
      if (j < ng) x0 = (m & 1) ? row[j].y : row[j].x;
      if (j + 1 < ng) x1 = (m & 1) ? row[j + 1].y : row[j + 1].x;
    }
    split_store(x0, x1, hi, lo, ((size_t)kb * mpad_b + m) * 64 + 2 * jp);
  }
}

// A: row 2 i + c, column j holds W^d_ij.c, Eq. (W_delta) with W = V E V:
// W^d_ij = V_i V_j [ (Im E_ij + Im E_ji) / 2 - i (Re E_ij - Re E_ji) / 2 ].
__global__ void __launch_bounds__(256)
k_sig_asplit(const double2* __restrict__ E, const double* __restrict__ v, int ng, int mpad_a,
             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int r0 = blockIdx.x * 64;
  const int kb = blockIdx.y;
  for (int e = threadIdx.x; e < 64 * 32; e += 256) {
    const int ml = e >> 5, jp = e & 31;
    const int m = r0 + ml, i = m >> 1;
    const int j = kb * 64 + 2 * jp;
    float x[2] = {0.f, 0.f};
    if (i < ng) {
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        const int jj = j + q;
        if (jj < ng) {
          const double2 a = E[(size_t)i * ng + jj], b = E[(size_t)jj * ng + i];
          const double f = 0.5 * v[i] * v[jj];
          x[q] = (float)((m & 1) ? -f * (a.x - b.x) : f * (a.y + b.y));
        }
      }
    }
    split_store(x[0], x[1], hi, lo, ((size_t)kb * mpad_a + m) * 64 + 2 * jp);
  }
}

}  // namespace

chi0_status sig_tc_plan(chi0_ctx* c, int64_t T, int ng) {
  if (!c->sig_tc) c->sig_tc = new SigTc();
  SigTc& t = *static_cast<SigTc*>(c->sig_tc);
  t.T = T;
  t.ng = ng;
  t.kpad = (ng + kBK - 1) / kBK * kBK;
  t.nI = (ng + 63) / 64;
  t.nJ = (int)std::min<int64_t>((T + 63) / 64, 0x7fffffff);
  t.mpad_a = t.nI * kBM;
  t.mpad_b = (int64_t)t.nJ * kBN;
  // TMA row coordinates and tile indices are 32-bit
  if ((T + 63) / 64 > 0x7fffffff / t.nI || (t.kpad / kBK) * t.mpad_b > 0x7fffffff)
    return ctx_fail(c, CHI0_EUNSUPPORTED, "too many transitions in the quasiparticle window for one contraction");
  chi0_status s;
  const size_t opa = (size_t)t.mpad_a * t.kpad * 2, opb = (size_t)t.mpad_b * t.kpad * 2;
  if ((s = ctx_ensure(c, t.ah, opa, "W^delta hi")) != CHI0_OK) return s;
  if ((s = ctx_ensure(c, t.al, opa, "W^delta lo")) != CHI0_OK) return s;
  if ((s = ctx_ensure(c, t.bh, opb, "rho hi")) != CHI0_OK) return s;
  if ((s = ctx_ensure(c, t.bl, opb, "rho lo")) != CHI0_OK) return s;
  if (!make_map(&t.m_ah, t.ah.p, t.kpad, t.mpad_a) || !make_map(&t.m_al, t.al.p, t.kpad, t.mpad_a) ||
      !make_map(&t.m_bh, t.bh.p, t.kpad, (int)t.mpad_b) || !make_map(&t.m_bl, t.bl.p, t.kpad, (int)t.mpad_b))
    return ctx_fail(c, CHI0_ECUDA, "cuTensorMapEncodeTiled failed");
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  t.nsm = std::max(1, nsm);
  cudaError_t e = cudaFuncSetAttribute(k_herk_wide, cudaFuncAttributeMaxDynamicSharedMemorySize, kWSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_herk_wide, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return ctx_fail(c, CHI0_ECUDA, cudaGetErrorString(e));
  return CHI0_OK;
}

cudaError_t sig_tc_split_b(chi0_ctx* c, const float2* R, int nqp, int nb) {
  SigTc& t = *static_cast<SigTc*>(c->sig_tc);
  k_sig_bsplit<<<dim3((unsigned)(t.mpad_b / 64), (unsigned)(t.kpad / 64)), 256, 0, c->st>>>(
      R, t.T, nqp, nb, t.ng, t.mpad_b, (__nv_bfloat16*)t.bh.p, (__nv_bfloat16*)t.bl.p);
  return cudaGetLastError();
}

cudaError_t sig_tc_split_a(chi0_ctx* c, const double2* E, const double* vsqrt) {
  SigTc& t = *static_cast<SigTc*>(c->sig_tc);
  k_sig_asplit<<<dim3((unsigned)(t.mpad_a / 64), (unsigned)(t.kpad / 64)), 256, 0, c->st>>>(
      E, vsqrt, t.ng, t.mpad_a, (__nv_bfloat16*)t.ah.p, (__nv_bfloat16*)t.al.p);
  return cudaGetLastError();
}

// Y on the wide kernel: 128 x 256 tiles over the full grid (nJ / 2 wide
// column tiles, rounded up), one k range per tile, written as Y's 64 x 64
// complex FP32 tiles; the half of a last wide tile beyond the B rows is not
// written.
cudaError_t sig_tc_contract(chi0_ctx* c, float2* Y) {
  SigTc& t = *static_cast<SigTc*>(c->sig_tc);
  const int ntiles = t.nI * ((t.nJ + 1) / 2);
  const int total_kb = (int)(t.kpad / kBK);
  const unsigned grid = (unsigned)std::min(ntiles, t.nsm);
  k_herk_wide<<<grid, kWThreads, kWSmemBytes, c->st>>>(t.m_ah, t.m_al, t.m_bh, t.m_bl, total_kb, total_kb, t.mpad_a,
                                                        reinterpret_cast<double2*>(Y), ntiles, ntiles,
                                                        (int*)c->d_err.p, t.nI, nullptr, 1, (int)t.mpad_b, 1);
  return cudaGetLastError();
}

void sig_tc_release(chi0_ctx* c) {
  if (!c->sig_tc) return;
  SigTc* t = static_cast<SigTc*>(c->sig_tc);
  DevBuf* bufs[] = {&t->ah, &t->al, &t->bh, &t->bl};
  for (DevBuf* b : bufs)
    if (b->p) cudaFree(b->p);
  delete t;
  c->sig_tc = nullptr;
}

}  // namespace chi0
